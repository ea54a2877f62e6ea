"""GB300 (sm_103a) implementation of one method-of-lines RK stage of the Valencia GRMHD equations on uniform
Cartesian blocks over a frozen metric (AsterX, arXiv:2406.11669).

`asterx` is the binding of the C ABI (include/asterx.h); `workloads` generates seeded synthetic inputs.
"""
__all__ = ["asterx", "workloads", "build"]
