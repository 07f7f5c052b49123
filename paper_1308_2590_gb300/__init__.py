"""GB300 (sm_103a) implementation of the implicit 2D3V PIC particle loop and
field solve of Petrov & Davis (arXiv 1308.2590), behind the C ABI of
include/pic.h.

Submodules: ``build`` (compiles libpic.so), ``pic`` (ctypes binding with the
C entry-point names), ``workloads`` (seeded synthetic runs).
"""
