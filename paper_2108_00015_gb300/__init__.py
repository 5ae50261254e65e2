"""GB300 (sm_103a) implementation of the ConKer n-point correlation hot path
(arXiv 2108.00015): gridding, FFT shell convolution and n-point product sums
behind a C ABI (include/conker.h).  ``conker`` is the ctypes binding."""
from .conker import CkError, Plan, batch_compute, load, order_mask, sky_to_cartesian  # noqa: F401
