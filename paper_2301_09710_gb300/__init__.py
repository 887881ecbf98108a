"""GB300 (sm_103a) rotation-based SPECT projector, its exact adjoint and the
MLEM update (arXiv 2301.09710, Section II-A and Eqs. (7)-(8)).

Submodules are imported lazily so that ``paper_2301_09710_gb300.synthetic``
(seeded inputs) can be used without torch or the CUDA library.
"""
__all__ = ["SpectPlan", "SpectBatch", "build", "synthetic"]


def __getattr__(name):
    if name == "SpectPlan":
        from .projector import SpectPlan
        return SpectPlan
    if name == "SpectBatch":
        from .projector import SpectBatch
        return SpectBatch
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
