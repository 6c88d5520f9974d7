"""GB300 (sm_103a) MWU solver for positive LPs (arXiv 2307.03307).

The hot path (constraint evaluation, exp weights with shifted log-sum-exp,
transpose gradients, the gradient test and multiplicative update, and the
K-candidate and Newton step-size searches) runs in hand-written CUDA kernels inside
``_lib/libmwu.so``, behind the C ABI of ``include/mwu.h``.  ``mwu`` is the thin
ctypes binding with the same names, ``lpspec`` marshals the paper's graph LPs,
and ``autograd`` wraps the smoothed potential as a torch.autograd.Function.
"""
from . import mwu  # noqa: F401
from . import lpspec  # noqa: F401
from . import autograd  # noqa: F401

__all__ = ["mwu", "lpspec", "autograd"]
