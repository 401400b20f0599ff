"""GB300 (sm_103a) implementation of the Lya M1 substep of the Lydion method
(arXiv 2606.02711): C ABI in include/lym1.h, CUDA library liblym1.so built by
``build.build()``, Python binding in ``lym1``."""
from . import build  # noqa: F401

__all__ = ["build", "lym1"]


def __getattr__(name):
    if name == "lym1":
        from . import lym1 as m
        return m
    raise AttributeError(name)
