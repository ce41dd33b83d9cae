"""GB300-native all-pairs library: f(l(i), l(j)) for every pair i < j.

The compute path is the CUDA library ``libap.so`` (C ABI in
``include/allpairs.h``); this package is its thin binding:

* ``binding``  -- ctypes marshalling of the C ABI (``Items`` handle class);
* ``autograd`` -- ``OverlapAlign``, a torch.autograd.Function over the overlap
  cost and its hand-written adjoint.
"""
from .binding import (AP_FN_BHATTACHARYYA, AP_FN_COSINE, AP_FN_COVERAGE,  # noqa: F401
                      AP_FN_GMM_L2,
                      AP_FN_OVERLAP, AP_FN_PEARSON, AP_PREC_FP32,
                      AP_PREC_SPLIT_BF16, APError, Items, lib, pair_count, pair_index,
                      plan_tiles)
