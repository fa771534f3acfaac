// tm_stage_host.h -- host entry points of the staged batched hop (tm_stage.cu).
#pragma once

#include <cuda.h>

#include "tm_internal.h"

namespace twm {

// Storage formats the staged hop is built for (FP32 12/18-real, FP16 12-real links).
bool stage_supported(int prec, int recon);
// Lattices it tiles: Lx a multiple of 16 (boxes of 8 half-sites in x).
bool stage_geometry_ok(const Geom &g);
// Boxes per z block of the staged hop's traversal order on lattice g: x
// fastest, then y, z inside the block, t, and the z blocks, with blocks of
// at most 128 boxes per time layer pair: the t faces of a box are the own
// sites of a box at most 128 work items away (read again from L2, not from
// memory), and only the z faces at block edges are read from memory twice.
// (Measured on 32^3x64, 12 FP32 right-hand sides: 64, 128, 256 or 1024
// boxes move launch B by less than 2 %.)
int stage_zblock(const Geom &g);
// Whether the driver provides the tensor-map encoder.
bool stage_available();
// Builds U's site-complete link copy (its 8 links per site: twice the
// handle's link bytes, for FP32 handles all 18 reals of each link) on stream
// s, once per handle.
cudaError_t stage_links8(const tm_gauge *U, cudaStream_t s);
// The 5 box maps of a packed field of lattice g (and for FP16 the 5 maps of
// its site norms) into maps[0 .. 2*5).
bool stage_field_maps(int prec, const Geom &g, const void *field, CUtensorMap *maps);
// The map of U's site-complete links (stage_links8 first).
bool stage_link_map(const tm_gauge *U, CUtensorMap &m);

}  // namespace twm
