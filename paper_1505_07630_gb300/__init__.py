"""GB300-native Jacobi / pipelined PCG for OpenFOAM-style LDU matrices.

The compute path is libldupcg (hand-written sm_103a CUDA behind a C ABI,
include/ldupcg.h); this package holds its build script, the ctypes binding
and the autograd wrapper.  PyTorch supplies device memory and streams only.
"""
from .ldupcg import (LduAmg, LduError, LduMatrix, amg_from_system, amg_pcg_solve,  # noqa: F401
                     amg_pipecg_solve,
                     ldu_amg_aggregates, ldu_amg_create, ldu_amg_destroy, ldu_amg_info,
                     ldu_amg_vcycle)
from .ldupcg import (from_system, from_systems, ldu_batch_info,  # noqa: F401
                     ldu_batch_results, ldu_batch_schedule, ldu_create, ldu_create_batched,
                     ldu_destroy, ldu_diag_grad, ldu_harmonic_coeffs, ldu_harmonic_grad,
                     ldu_heat_steps, ldu_piso_pressure, ldu_value_grad,
                     pcg_solve_batched, pcg_solve_batched_async,
                     ldu_face_grad, ldu_set_face_coeffs, ldu_spmv, ldu_update_values, lib,
                     library_path, pcg_solve, pcg_solve_ldu_noalloc, pipecg_solve,
                     status_string)
from .autograd import (HarmonicCoeffs, LduSolve, LduSolveValues, harmonic_coeffs,  # noqa: F401,E402
                       ldu_solve, ldu_solve_values)
