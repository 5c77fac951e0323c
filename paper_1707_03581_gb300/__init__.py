"""GB300-native IMEX multi-rate SDC for the coupled stand/stock FEM heat equation.

The compute path is the C-ABI library libsdcheat.so (CUDA kernels for
sm_103a, built in-tree by `build.build()`); `binding.Solver` is its Python
face. Nothing here runs the simulation on the CPU.
"""

from .binding import LIB_PATH, Batch, SdcError, Solver, load_library  # noqa: F401
