"""GB300-native tropical tensor-network contraction for spin-glass ground states.

The compute path is libtn.so (CUDA for sm_103a, C ABI in include/tn.h); this
package only marshals arguments (binding.py) and wraps the ground-state
traceback as a torch.autograd.Function (autograd.py).  There is no CPU
fallback: without the built library or a CUDA device every compute call fails.
"""
from .binding import *  # noqa: F401,F403
from .binding import Max2SAT, SpinGlass, TNError, lib  # noqa: F401

__all__ = [n for n in dir() if n.startswith("tn_") or n.startswith("TN_")] + [
    "SpinGlass", "Max2SAT", "TNError", "lib", "TropicalEnergy"]


def __getattr__(name):
    if name == "TropicalEnergy":
        from .autograd import TropicalEnergy
        return TropicalEnergy
    raise AttributeError(name)
