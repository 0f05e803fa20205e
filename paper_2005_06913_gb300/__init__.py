"""GB300-native minimum spanning trees by data-parallel Boruvka rounds.

The compute path is libmst.so (hand-written sm_103a CUDA kernels behind the
C ABI of include/mst.h); ``binding`` is its thin Python interface and
``graphgen`` the seeded synthetic workloads.
"""
from . import binding  # noqa: F401
from .binding import *  # noqa: F401,F403
