"""GB300 amplitude solver for the point-source Helmholtz equation.

Implements the hot path of Treister & Haber, "A multigrid solver to the
Helmholtz equation with a point source based on travel time and amplitude":
the multigrid-preconditioned flexible GMRES solve of the complex ADR
equation for the amplitude a given the travel time tau, and the
reconstruction u = a exp(-i w tau).  The computation lives in hand-written
CUDA kernels for sm_103a behind the C ABI of include/adr.h (libadr.so);
`adr` is its Python binding and `workloads` builds seeded synthetic inputs.

Submodules are imported lazily so that `workloads` can be used without the
compiled library.
"""

__all__ = ["adr", "workloads", "build"]
