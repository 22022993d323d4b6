// Declarations of the adjoint's global solve for implicit transport
// (tfs_implicit.cu), kept apart from the step kernel's shared header.
#pragma once

#include <cuda_runtime.h>

#include "tfs_internal.h"

namespace tfs {

// One implicit step (stress form) solves Op sigma^{n+1} = R with Op = M_p +
// dt (u.grad - eps Lap), M_p = a I - dt L(kappa*) per point.  Its adjoint needs
// lamR = Op^-T v, v = s1 + sum_j rho_j z_j (z_j = b1 lamQ'_j + b2 lamQ''_j of the
// mode adjoint ring ell_prev / ell_prev2).  This solves that system with the
// step's Krylov solver on the transposed operator (the point blocks and their
// inverses transposed in place, the tap coefficients gathered from the
// neighbours into cfT, 4 dim N doubles) and then rewrites s1 in place as
// M_p^T lamR - sum_j rho_j z_j, so that the pointwise adjoint kernel, which
// forms M_p^-T (s1 + sum_j rho_j z_j), recovers lamR and does the rest of the
// step's adjoint unchanged.  `a` is filled as for the forward step (kry,
// partials, tolerance, iteration limit, grid, stencil, velocity, kappa).
cudaError_t run_implicit_adjoint_f64(const ImpArgs<double>& a, double* s1, const double* ell_prev,
                                     const double* ell_prev2, double* cfT, cudaStream_t s, int* iters,
                                     double* relres);
cudaError_t run_implicit_adjoint_f32(const ImpArgs<float>& a, double* s1, const float* ell_prev,
                                     const float* ell_prev2, double* cfT, cudaStream_t s, int* iters,
                                     double* relres);

}  // namespace tfs
