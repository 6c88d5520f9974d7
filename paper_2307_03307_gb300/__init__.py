"""GB300 (sm_103a) MWU solver for positive LPs (arXiv 2307.03307).

The hot path (constraint evaluation, exp weights with shifted log-sum-exp,
transpose gradients, the gradient test and multiplicative update, and the
K-candidate and Newton step-size searches) runs in hand-written CUDA kernels inside
``_lib/libmwu.so``, behind the C ABI of ``include/mwu.h``.  ``mwu`` is the thin
ctypes binding with the same names, ``lpspec`` marshals the paper's graph LPs,
and ``autograd`` wraps the smoothed potential as a torch.autograd.Function.
"""
import os

# mwu_solve_batch runs instances concurrently, three streams each (the
# context's own, and the two that capture its search loop): give the process
# more hardware work queues than the driver's default 8, so that the streams
# do not share queues.  The driver reads this when CUDA initialises, so it
# takes effect only if the process has not initialised CUDA yet.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from . import mwu  # noqa: F401,E402
from . import lpspec  # noqa: F401,E402
from . import autograd  # noqa: F401,E402

__all__ = ["mwu", "lpspec", "autograd"]
