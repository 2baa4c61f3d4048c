"""GB300 clover-Wilson Dirac operator, SAP smoother, FP64 flexible outer solver
and link force (arXiv:2112.00501: the fine-grid operator of Eq. (1) and the
QWS smoother M_SAP of Sec. 2, used as the post-smoother of Sec. 3).

The compute path is libmgc.so (hand-written sm_103a CUDA behind the C ABI in
include/mgc.h); the Python modules only marshal arguments.  Importing the
package does not load the library: `api` and `autograd` do, and fail loudly
if it is missing.
"""

__all__ = ["api", "autograd", "synth", "build"]
