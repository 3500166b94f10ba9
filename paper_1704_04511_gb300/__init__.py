"""GB300 (sm_103a) IRLS reconstruction of damped-exponential image series by structured
low-rank matrix completion (arXiv 1704.04511, Algorithm 1).

The compute path is librecon.so (CUDA kernels behind the C ABI of include/recon.h); `recon`
is its thin ctypes binding and `serve` the request loop built on it.
"""

from . import recon  # noqa: F401  (loads nothing until the first call)

__all__ = ["recon"]
