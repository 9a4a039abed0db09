"""GPU (sm_103a) low-rank all-at-once solver for the stochastic unsteady
Navier-Stokes problem (Elman & Su): tensor-train GMRES inside truncated
inexact Picard, behind the C ABI of include/tt_stochns.h.

`binding` is the ctypes layer over lib/libttns.so; `build` compiles it.
There is no CPU fallback: without the library or a GPU, `binding.Context()`
raises.
"""
__all__ = ["binding", "build"]
