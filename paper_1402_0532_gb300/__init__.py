"""GB300 (sm_103a) implementation of the multiplication-free nonlinear DFT of
arXiv 1402.0532: the NDFT (Eq. 8), the (x)-butterfly NFFT (Sec. 3) and the
nonlinear cross-ambiguity function (Eq. 12a), behind the C ABI of
include/ndft.h.  ``api`` is the thin PyTorch binding; ``scenes`` the seeded
synthetic inputs; ``build`` compiles libndft.so."""

__all__ = ["Plan", "BatchedPlan", "argmax", "CafFunction", "caf_autograd"]


def __getattr__(name):
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
