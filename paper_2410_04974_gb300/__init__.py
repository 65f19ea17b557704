"""GB300-native differentiable render of 6D Gaussian scenes (6DGS, arXiv 2410.04974).

The work happens in ``libsixdgs.so`` (hand-written sm_103a CUDA behind the C
ABI of ``include/sixdgs.h``); this package marshals arguments to it.
"""

from . import _lib
from ._lib import SixDGSError, load
from .render import (PARAM_NAMES, Renderer, RenderFunction, make_plan, make_settings, params_to_device, render,
                     condition_cache, scale_rotation)

__all__ = ["SixDGSError", "load", "Renderer", "RenderFunction", "render", "make_plan", "make_settings",
           "params_to_device", "PARAM_NAMES", "scale_rotation", "condition_cache", "_lib"]
