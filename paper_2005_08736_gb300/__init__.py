"""GB300 (sm_103a) implementation of the step of the high-order gas-kinetic
scheme of Cao, Pan & Xu (arXiv:2005.08736): WENO5 reconstruction, BGK
interface flux at 2x2 Gauss points and the two-stage fourth-order update, as
CUDA kernels behind the C ABI of include/hgks.h.

Submodules: ``_lib`` (ctypes binding of the ABI), ``solver`` (Python API with
torch streams), ``inputs`` (seeded synthetic initial fields), ``build``
(nvcc build of libhgks.so).  Importing the package does not load the CUDA
library; the first Simulation does, and raises if it is missing.
"""

__all__ = ["build", "inputs", "solver"]
