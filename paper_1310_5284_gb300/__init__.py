"""GB300-native energy-conserving 1D PIC/MCC for RF discharges.

The hot path (charge assignment, energy-conserving gather and leapfrog or
direct-implicit push, electrode absorption, null-collision Monte Carlo with
ionisation, tridiagonal field solve with the RF electrode) runs in the CUDA
kernels of libpic.so behind the C ABI of include/pic.h.  This package holds
the library sources (csrc/), its build step and a thin ctypes binding.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Sim", "make_config", "required_sizes", "philox_fill"):
        from . import sim
        return getattr(sim, name)
    raise AttributeError(name)
