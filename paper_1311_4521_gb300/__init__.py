"""GB300 (sm_103a) library for the even-odd preconditioned Wilson twisted-mass operator.

``tmhop`` is the ctypes binding of the C ABI in include/tmhop.h (it needs the
compiled ``libtmhop.so``; build it with :func:`build.build`), ``autograd``
the torch.autograd Functions over it, and ``fields`` the seeded synthetic
input generators.
"""
__all__ = ["fields", "build", "tmhop", "autograd"]
