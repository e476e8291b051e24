"""GB300-native checkerboard Metropolis sweeps, replica exchange and
reductions for Ising, +-J Edwards-Anderson and Heisenberg lattices
(Weigel, arXiv:1101.1427), behind the C ABI of include/spin.h.

``Lattice`` owns the device buffers (PyTorch tensors: memory and streams
only) of one library handle; every computation is a call into the CUDA
library through the binding in ``_binding``.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import lib  # noqa: F401
from .lattice import BatchGraph, Lattice, batch_run  # noqa: F401
