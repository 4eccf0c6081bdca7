"""GB300 (sm_103a) entropic lattice Boltzmann for the full-tensor anisotropic
advection-diffusion equation.

The compute path is the C-ABI library ``libelbm.so`` (hand-written CUDA);
:mod:`paper_2605_01774_gb300.elbm` is a thin ctypes binding with the same
function names as ``include/elbm.h``.  There is no CPU fallback: importing the
binding without the built library raises.
"""
__all__ = ["elbm", "build"]
