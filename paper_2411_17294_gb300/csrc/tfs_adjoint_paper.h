// Declarations of the adjoint of the paper's variable (tfs_adjoint_paper.cu),
// kept apart from the step kernel's shared header.
#pragma once

#include <cuda_runtime.h>

#include "tfs_internal.h"

namespace tfs {

// Adjoint of one BDF2 step in the paper's variable (pointwise law).  psi is the
// step's output Psi^{n+1}; lam_psi the adjoint of Psi at the final step (else
// nullptr); s1 / s0 the adjoints of Phi^{n+1} and (partial) of Phi^n, s1_out /
// s0_out those of Phi^n and (partial) Phi^{n-1}; the mode adjoint ring as in the
// stress form (lamQ written over ell_prev2).  mc / mcf: c_j, dt c_j, w_j mu_j c_j.
// With explicit transport (acting on 2 Psi^n - Psi^{n-1}) the adjoint of Psi has
// a ring too: t1 the full adjoint of Psi^{n+1} (it then replaces lam_psi), t0
// the partial one of Psi^n; the kernel sets t1_out = t0, t0_out = 0 and writes
// lamR to lamR_out, and the transposed stencil adds its terms to t1_out, t0_out.
template <typename T>
struct PaperAdjArgs {
    const T* kap;
    const T* psi;
    const double* lam_psi;
    const double* s1;
    const double* s0;
    const T* ell_prev;
    T* ell_prev2;
    double* s1_out;
    double* s0_out;
    double* g_kap;
    const double* t1;
    const double* t0;
    double* t1_out;
    double* t0_out;
    double* lamR_out;
    double* partials;
    unsigned* flags;
    long long N;
    int m;
    double dt, a, xi, G, psi0, Wi, Re;
    ModeConstsD mc;
    ModeConstsF mcf;
};
// Adjoint of the SDIRK2 first step in the paper's variable (pointwise law, zero
// initial modes): sigma0 is Phi(0) (nullptr: 0), lam_psi the adjoint of Psi^1
// when the run has one step (else nullptr), s1 / s0 the adjoints of Phi^1 and
// (partial) of Phi^0, ell_prev / ell_prev2 the two later levels of the mode
// adjoint ring; s1_out receives the whole adjoint of Phi^0 and s0_out 0.
// a = 1 + gamma dt W/Wi.
template <typename T>
struct PaperStartAdjArgs {
    const T* kap0;
    const T* sigma0;
    const double* lam_psi;
    const double* s1;
    const double* s0;
    const T* ell_prev;
    const T* ell_prev2;
    double* s1_out;
    double* s0_out;
    double* g_kap;
    double* partials;
    unsigned* flags;
    long long N;
    int m;
    double dt, a, G, Wi, Re;
};
cudaError_t launch_paper_start_adjoint_f64(const PaperStartAdjArgs<double>& a, const StartConsts& c, int dim,
                                           cudaStream_t s);
cudaError_t launch_paper_start_adjoint_f32(const PaperStartAdjArgs<float>& a, const StartConsts& c, int dim,
                                           cudaStream_t s);
cudaError_t launch_paper_adjoint_f64(const PaperAdjArgs<double>& a, int dim, cudaStream_t s);
cudaError_t launch_paper_adjoint_f32(const PaperAdjArgs<float>& a, int dim, cudaStream_t s);

}  // namespace tfs
