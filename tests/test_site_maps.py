"""The site-to-thread maps of the hop (the autotuner's candidates) on the
host: a small C++ program built with nvcc from the library's device header
checks that every linear and box map covers every site exactly once on
several lattice shapes and that the box numbering's division by invariant
integers is exact.  No GPU needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1311_4521_gb300", "csrc")


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_site_maps_cover_every_site_once(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    exe = tmp_path / "site_map_check"
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, os.path.join(HERE, "host", "site_map_check.cu"),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "0 failures" in out.stdout


def test_batched_work_orders_and_stage_slots(tmp_path):
    """The batched hops' work orders on the host: the banded tile order is a
    permutation of the tiles, the staged hop's boxes cover every site once,
    and every stage slot a consumer reads holds the neighbour it wants, by
    the content the producer's tensor copies put there (12 lattice shapes,
    both output parities, including 32^3x64)."""
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    include = os.path.join(os.path.dirname(HERE), "include")
    exe = tmp_path / "tile_order_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-I", CSRC, "-I", include,
                    os.path.join(HERE, "host", "tile_order_check.cu"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip().endswith("OK"), out.stdout
