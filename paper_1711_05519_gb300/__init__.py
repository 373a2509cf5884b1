"""GB300 (sm_103a) implementation of accelerated alternating projections (AccAltProj) for
fully observed robust PCA, behind the C ABI of include/rpca.h."""
from .rpca import (Solver, RpcaError, solve, solve_host, solve_host_release, selftest_waits, lib, status_string, header_functions,  # noqa: F401
                   OK, INVALID_ARG, CUDA_ERR, NUMERICAL, CAPACITY, NOT_CONVERGED, TIMEOUT, STATE)
