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
//
// The paper's variable (lp_out given): the operator is a I - dt xi L + dt xi T
// on Phi with -dt T(h) on the right-hand side, v = s1 + xi lamPsi + sum_j dt c_j
// z_j (lam_psi: the adjoint of Psi, or nullptr), and the adjoint of h gains
// -dt T^T lamR = -(v - M_p^T lamR)/xi.  s1 is left as it is and lp_out receives
// lamPsi - (v - M_p^T lamR)/xi: the paper-variable adjoint kernel, given that in
// place of lamPsi, recovers lamR from M_p^-T (s1 + xi lp_out + sum_j dt c_j z_j)
// and adds the transport's term to the adjoint of h.
cudaError_t run_implicit_adjoint_f64(const ImpArgs<double>& a, double* s1, const double* ell_prev,
                                     const double* ell_prev2, double* cfT, const double* lam_psi, double xi,
                                     double* lp_out, cudaStream_t s, int* iters, double* relres);
cudaError_t run_implicit_adjoint_f32(const ImpArgs<float>& a, double* s1, const float* ell_prev,
                                     const float* ell_prev2, double* cfT, const double* lam_psi, double xi,
                                     double* lp_out, cudaStream_t s, int* iters, double* relres);

// Adjoint of the SDIRK2 first step with implicit transport (zero initial
// modes): stage 1 solved again for S1 (into S1), then the two
// transposed stage systems (lamr2 kept in s0_out until the end), then the
// adjoint of sigma0 into s1_out (s0_out set to 0) and the parameter terms into
// g_kap and the adjoint's 32-point partials.  s1 / s0in: adjoints of sigma^1
// and (partial) sigma^0; ell_prev / ell_prev2: the two later mode-ring levels;
// S2: sigma^1 of the recomputed step; cfT: 4 dim N doubles.  `a` as for the
// forward start (a = dt W + dt/Wi); iters sums the three solves, relres the
// largest residual.
template <typename T>
struct StartImpAdj {
    const double* s1;
    const double* s0in;
    const T* ell_prev;
    const T* ell_prev2;
    const T* S2;
    double* S1;
    double* s1_out;
    double* s0_out;
    double* g_kap;
    double* partials;
    double* cfT;
    double Wi, Re;
    // the paper's variable (paper = 1): lam_psi the adjoint of Psi^1 (one-step
    // run, else nullptr), phi0 = Phi(0) (nullptr: 0), dt the time step (a.dt is
    // gamma dt W there); S2 is then Psi^1 and S1 receives Phi^(1)
    int paper;
    const double* lam_psi;
    const T* phi0;
    double dt;
};
cudaError_t run_start_implicit_adjoint_f64(const ImpArgs<double>& a, const StartConsts& c,
                                           const StartImpAdj<double>& j, cudaStream_t s, int* iters,
                                           double* relres);
cudaError_t run_start_implicit_adjoint_f32(const ImpArgs<float>& a, const StartConsts& c,
                                           const StartImpAdj<float>& j, cudaStream_t s, int* iters,
                                           double* relres);

}  // namespace tfs
