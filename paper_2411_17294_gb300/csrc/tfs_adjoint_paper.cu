// Adjoint of one BDF2 step in the paper's variable (Section 3.4), pointwise
// law, one thread per point.
//
// Forward step at a point (h = sum_j w_j mu_j c_j Q_j, Q_j = b1 phi_j^n + b2 phi_j^{n-1}):
//   R = -b1 Phi^n - b2 Phi^{n-1} + dt (L(kappa) h - h/Wi) + dt G k Psi0,   k = kappa + kappa^T
//   Phi^{n+1} = M^-1 R,   M = (b0 + dt xi/Wi) I - dt xi L(kappa)
//   phi_j^{n+1} = -c_j Q_j + dt c_j Phi^{n+1},   Psi^{n+1} = xi Phi^{n+1} + h
// Reverse, given the adjoints s1 of Phi^{n+1}, z_j of phi_j^{n+1} (z_j = b1 lamQ_j'
// + b2 lamQ_j'' from the two later steps) and, at the final step, lamPsi of Psi:
//   lamPhi = s1 + xi lamPsi + sum_j dt c_j z_j;   lamR = M^-T lamPhi
//   lamh = dt (L(kappa)^T lamR - lamR/Wi) + lamPsi
//   lamQ_j = w_j mu_j c_j lamh - c_j z_j          (the new level of the mode ring)
//   adjoint of Phi^n += -b1 lamR, of Phi^{n-1} += -b2 lamR
// Parameter terms: since xi Phi^{n+1} + h = Psi^{n+1}, the kappa terms of M and of
// dt L(kappa) h combine into dt lamR^T (dL/dkappa) Psi^{n+1}, and the Wi terms of M
// and of -dt h/Wi into (dt/Wi^2) <lamR, Psi^{n+1}>: the stress form's formulas
// with sigma^{n+1} replaced by Psi^{n+1}; the source adds dt G Psi0 (sym) to
// dJ/dkappa, -(G/Wi) dt Psi0 <lamR, k> to dJ/dWi and -dt Psi0 <lamR, k>/(Wi Re) to
// dJ/dbeta.  Only Psi^{n+1} of the forward step is needed.
#include <cuda_runtime.h>

#include <type_traits>

#include "tfs_device.cuh"
#include "tfs_internal.h"
#include "tfs_adjoint_paper.h"

namespace tfs {
namespace {

// 64 threads per block: z_j of a block (m nc 64 floats, 24 KB at m = 32 in 2D)
// lets nine blocks share an SM where 128-thread blocks fit four (measured on
// the 2D 512^2 m = 32 FP32 adjoint workload: 16.4 ms against 18.6 ms for the
// 100-step reverse sweep with its recompute)
constexpr int kThreads = 64;

// Entry (r, k) of the packed matrix of S -> kappa S + S kappa^T (as uc_entry,
// in the arithmetic type R; r and k fold at compile time under static_for).
template <int DIM, typename R>
__device__ __forceinline__ R uc_r(const R K[3][3], int r, int k) {
    const int ro = Packed<DIM>::I(r), so = Packed<DIM>::J(r);
    const int i = Packed<DIM>::I(k), j = Packed<DIM>::J(k);
    R v = R(0);
    if (so == j) v += K[ro][i];
    if (i != j && so == i) v += K[ro][j];
    if (ro == i) v += K[so][j];
    if (i != j && ro == j) v += K[so][i];
    return v;
}

// One thread per point, partials per 32-point warp (the layout of the other
// adjoint kernels).  FP64 storage: FP64 throughout.  FP32 storage: the mode
// passes and the point system in FP32 (compensated sum of dt c_j z_j; z_j kept
// in shared memory between the two passes, so that the ring is read once), the
// adjoint fields and the gradient accumulations in FP64.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) paper_adjoint_kernel(const PaperAdjArgs<T> A) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr bool F32 = sizeof(T) == 4;
    using R = typename std::conditional<F32, float, double>::type;
    extern __shared__ float zs[];           // FP32: z_j [m][NC][kThreads]
    const long long N = A.N;
    const int tid = threadIdx.x;
    const long long p = (long long)blockIdx.x * kThreads + tid;
    double gWi = 0.0, gbeta = 0.0;
    if (p < N) {
        R K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (R)A.kap[(long long)(i * DIM + j) * N + p];
        double lamd[NC];
        R lp[NC], psi[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long q = (long long)c * N + p;
            const double l = A.t1 ? A.t1[q] : A.lam_psi ? A.lam_psi[q] : 0.0;
            if (A.t1) {
                A.t1_out[q] = A.t0[q];
                A.t0_out[q] = 0.0;
            }
            lp[c] = (R)l;
            psi[c] = (R)A.psi[q];
            lamd[c] = A.s1[q] + A.xi * l;
        }
        // + sum_j dt c_j z_j per component, z_j = b1 lamQ'_j + b2 lamQ''_j
        if constexpr (F32) {
            float ss[NC], comp[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) ss[c] = comp[c] = 0.0f;
#pragma unroll 4
            for (int jj = 0; jj < A.m; ++jj) {
                const float rh = A.mcf.rho[jj];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const long long q = mode_index(p, jj * NC + c, A.m * NC);
                    const float z = __fmaf_rn(0.5f, (float)A.ell_prev2[q], -2.0f * (float)A.ell_prev[q]);
                    zs[(jj * NC + c) * kThreads + tid] = z;
                    const float yv = __fmaf_rn(rh, z, -comp[c]);
                    const float t = __fadd_rn(ss[c], yv);
                    comp[c] = __fsub_rn(__fsub_rn(t, ss[c]), yv);
                    ss[c] = t;
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) lamd[c] += (double)ss[c] - (double)comp[c];
        } else {
            double ss[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) ss[c] = 0.0;
#pragma unroll 2
            for (int jj = 0; jj < A.m; ++jj) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const long long q = mode_index(p, jj * NC + c, A.m * NC);
                    const double zj = kB1 * (double)A.ell_prev[q] + kB2 * (double)A.ell_prev2[q];
                    ss[c] = fma(A.mc.rho[jj], zj, ss[c]);        // rho_j = dt c_j in this variable
                }
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) lamd[c] += ss[c];
        }
        // lamR = M^{-T} lamPhi, M = a I - dt xi L(kappa)
        R lam[NC];
        bool ok;
        if constexpr (F32) {
            LU32<NC> F;
            const float a = (float)A.a, dx = (float)(A.dt * A.xi);
            static_for<0, NC>([&](auto rr) {
                constexpr int r = decltype(rr)::value;
                static_for<0, NC>([&](auto kk) {
                    constexpr int k = decltype(kk)::value;
                    const float v = uc_r<DIM, float>(K, k, r);       // entry (r, k) of M^T
                    F.a[r][k] = (r == k) ? __fmaf_rn(-dx, v, a) : -dx * v;
                });
            });
#pragma unroll
            for (int c = 0; c < NC; ++c) lam[c] = (float)lamd[c];
            ok = lu32_factor<NC>(F, 1e-30f);
            lu32_solve<NC>(F, lam);
        } else {
            double M[NC][NC], Mt[NC][NC];
            assemble_M<DIM>(K, A.a, A.dt * A.xi, M);
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int k = 0; k < NC; ++k) Mt[r][k] = M[k][r];
#pragma unroll
            for (int c = 0; c < NC; ++c) lam[c] = lamd[c];
            ok = gauss_pp<NC>(Mt, lam, 1e-300);
        }
        // lamh = dt (L^T lamR - lamR/Wi) + lamPsi
        R lh[NC];
        const R dtr = (R)A.dt, iwi = (R)(1.0 / A.Wi);
        static_for<0, NC>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            R acc = -lam[k] * iwi;
            static_for<0, NC>([&](auto rr) {
                constexpr int r = decltype(rr)::value;
                acc += uc_r<DIM, R>(K, r, k) * lam[r];
            });
            lh[k] = dtr * acc + lp[k];
        });
        // new mode-ring level lamQ_j = w_j mu_j c_j lamh - c_j z_j (over ell_prev2)
        if constexpr (F32) {
#pragma unroll 4
            for (int jj = 0; jj < A.m; ++jj) {
                const float eh = A.mcf.eta_hi[jj], el = A.mcf.eta_lo[jj], cj = A.mcf.c[jj];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const long long q = mode_index(p, jj * NC + c, A.m * NC);
                    const float z = zs[(jj * NC + c) * kThreads + tid];
                    A.ell_prev2[q] = (T)__fmaf_rn(eh, lh[c], __fmaf_rn(el, lh[c], -cj * z));
                }
            }
        } else {
#pragma unroll 2
            for (int jj = 0; jj < A.m; ++jj) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const long long q = mode_index(p, jj * NC + c, A.m * NC);
                    const double zj = kB1 * (double)A.ell_prev[q] + kB2 * (double)A.ell_prev2[q];
                    A.ell_prev2[q] = (T)(A.mc.eta[jj] * (double)lh[c] - A.mc.c[jj] * zj);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long q = (long long)c * N + p;
            A.s1_out[q] = A.s0[q] - kB1 * (double)lam[c];
            A.s0_out[q] = -kB2 * (double)lam[c];
            if (A.lamR_out) A.lamR_out[q] = (double)lam[c];
        }
        // parameter derivatives (the stress form's with sigma^{n+1} -> Psi^{n+1})
        R S3[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
            S3[i][j] = psi[r];
            S3[j][i] = psi[r];
        }
        R gK[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        const R src = (R)(A.dt * A.G * A.psi0);
        R sym_dot = 0, psi_dot = 0;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            const int r = Packed<DIM>::I(cc), s2 = Packed<DIM>::J(cc);
            const R l = lam[cc];
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                gK[r][b] += dtr * l * S3[b][s2];
                gK[s2][b] += dtr * l * S3[r][b];
            }
            gK[r][s2] += src * l;
            gK[s2][r] += src * l;
            sym_dot += l * (K[r][s2] + K[s2][r]);
            psi_dot += l * psi[cc];
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) A.g_kap[(long long)(a * DIM + b) * N + p] += (double)gK[a][b];
        const double lam_G = A.dt * A.psi0 * (double)sym_dot;
        gWi = A.dt / (A.Wi * A.Wi) * (double)psi_dot - A.G / A.Wi * lam_G;
        gbeta = -lam_G / (A.Wi * A.Re);
        if (!ok) atomicOr(A.flags, 2u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gWi += __shfl_xor_sync(0xffffffffu, gWi, off);
        gbeta += __shfl_xor_sync(0xffffffffu, gbeta, off);
    }
    // partials of the 32-point group (p >> 5); groups past the last point hold none
    const long long grp = p >> 5;
    if ((tid & 31) == 0 && grp * 32 < N) {
        A.partials[2 * grp + 0] += gWi;
        A.partials[2 * grp + 1] += gbeta;
    }
}

// Terms of one implicit stage F = P - Z - s [L(kappa) Y - Y/Wi + G k g] = 0 in
// the parameters, given its adjoint lamr: dJ/dkappa += s (dL/dkappa)^T(lamr, Y) +
// s G g sym(lamr), dJ/dWi += s/Wi^2 <lamr, Y> - (G/Wi) s g <lamr, k>,
// dJ/dbeta += -s g <lamr, k>/(Wi Re)  (G = (1 - beta)/(Wi Re), k = kappa + kappa^T).
template <int DIM>
__device__ __forceinline__ void stage_param_terms(const double K[3][3], const double* lamr, const double* Y,
                                                  double sc, double G, double g, double Wi, double Re,
                                                  double gK[3][3], double& gWi, double& gbeta) {
    constexpr int NC = Packed<DIM>::NC;
    double Y3[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int r = 0; r < NC; ++r) {
        const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
        Y3[i][j] = Y[r];
        Y3[j][i] = Y[r];
    }
    double sym_dot = 0.0, y_dot = 0.0;
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
        const int r = Packed<DIM>::I(cc), s2 = Packed<DIM>::J(cc);
        const double l = lamr[cc];
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
            gK[r][b] += sc * l * Y3[b][s2];
            gK[s2][b] += sc * l * Y3[r][b];
        }
        gK[r][s2] += sc * G * g * l;
        gK[s2][r] += sc * G * g * l;
        sym_dot += l * (K[r][s2] + K[s2][r]);
        y_dot += l * Y[cc];
    }
    const double lam_G = sc * g * sym_dot;
    gWi += sc / (Wi * Wi) * y_dot - G / Wi * lam_G;
    gbeta += -lam_G / (Wi * Re);
}

// Adjoint of the SDIRK2 first step in the paper's variable for zero initial
// modes, one thread per point, FP64.  With phi_j^0 = 0 (iota_j = 1/(1 + gamma
// mu_j dt), W = sum_j w_j iota_j, S = sum_j w_j mu_j iota_j^2, gd = gamma dt,
// f1 = (1 - gamma) dt, M = a I - gd W L(kappa)) the forward reads
//   P1 = M^-1 (P0 + gd G k g0)                          (stage 1: h = 0)
//   h2 = f1 S P1,  zP = P0 + (f1/gd)(P1 - P0)
//   P2 = M^-1 (zP - gd (L h2 - h2/Wi) + gd G k g1)     (stage 2)
//   phi_j^1 = iota_j (f1 iota_j P1 + gd P2),  Phi^1 = P2,  Psi^1 = W P2 - h2
// Since a P - gd W L P = P + gd (W P/Wi - L W P), each stage is
// P - Z - gd [L Y - Y/Wi + G k g] = 0 with Y = W P1 (stage 1) and Y = Psi^1
// (stage 2).  Reverse, z_j the adjoint of phi_j^1:
//   lamP2 = s1 + W lamPsi + gd sum_j iota_j z_j,  lamr2 = M^-T lamP2
//   lamh2 = -lamPsi - gd (L^T lamr2 - lamr2/Wi)
//   lamP1 = f1 sum_j iota_j^2 z_j + f1 S lamh2 + (f1/gd) lamr2,  lamr1 = M^-T lamP1
//   adjoint of Phi^0 = s0 + lamr1 + (1 - f1/gd) lamr2
// and the stage terms of stage_param_terms with (lamr1, W P1, g0), (lamr2, Psi^1, g1).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) paper_start_adjoint_kernel(const PaperStartAdjArgs<T> A,
                                                                       const StartConsts C) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
    double gWi = 0.0, gbeta = 0.0;
    if (p < N) {
        const double gd = C.gam * A.dt, f1 = (1.0 - C.gam) * A.dt;
        double S = 0.0;
        for (int jj = 0; jj < A.m; ++jj) S += C.w[jj] * C.mu[jj] * C.inv_den[jj] * C.inv_den[jj];
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (double)A.kap0[(long long)(i * DIM + j) * N + p];
        double M0[NC][NC], M[NC][NC];
        assemble_M<DIM>(K, A.a, gd * C.W, M0);
        double P0[NC], src[NC], P1[NC], P2[NC], h2[NC], Y1[NC], Psi1[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            P0[c] = A.sigma0 ? (double)A.sigma0[(long long)c * N + p] : 0.0;
            src[c] = A.G * (K[i][j] + K[j][i]);
            P1[c] = P0[c] + gd * src[c] * C.g[0];
        }
        // forward, recomputed
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int k = 0; k < NC; ++k) M[r][k] = M0[r][k];
        bool ok = gauss_pp<NC>(M, P1, 1e-300);
#pragma unroll
        for (int c = 0; c < NC; ++c) h2[c] = f1 * S * P1[c];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            double Lh = -h2[r] / A.Wi;
#pragma unroll
            for (int k = 0; k < NC; ++k) Lh = fma(uc_entry<DIM>(K, r, k), h2[k], Lh);
            P2[r] = P0[r] + (f1 / gd) * (P1[r] - P0[r]) - gd * Lh + gd * src[r] * C.g[1];
        }
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int k = 0; k < NC; ++k) M[r][k] = M0[r][k];
        ok = gauss_pp<NC>(M, P2, 1e-300) && ok;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            Y1[c] = C.W * P1[c];
            Psi1[c] = C.W * P2[c] - h2[c];
        }
        // reverse
        double lamP2[NC], lamP1[NC], lamPsi[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long q = (long long)c * N + p;
            lamPsi[c] = A.lam_psi ? A.lam_psi[q] : 0.0;
            double a2 = 0.0, a1 = 0.0;
            for (int jj = 0; jj < A.m; ++jj) {
                const long long qm = mode_index(p, jj * NC + c, A.m * NC);
                const double z = kB1 * (double)A.ell_prev[qm] + kB2 * (double)A.ell_prev2[qm];
                a2 = fma(C.inv_den[jj], z, a2);
                a1 = fma(C.inv_den[jj] * C.inv_den[jj], z, a1);
            }
            lamP2[c] = A.s1[q] + C.W * lamPsi[c] + gd * a2;
            lamP1[c] = f1 * a1;
        }
        double Mt[NC][NC];
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int k = 0; k < NC; ++k) Mt[r][k] = M0[k][r];
        ok = gauss_pp<NC>(Mt, lamP2, 1e-300) && ok;          // lamP2 = lamr2
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            double lt = -lamP2[k] / A.Wi;
#pragma unroll
            for (int r = 0; r < NC; ++r) lt = fma(uc_entry<DIM>(K, r, k), lamP2[r], lt);
            const double lamh2 = -lamPsi[k] - gd * lt;
            lamP1[k] += f1 * S * lamh2 + (f1 / gd) * lamP2[k];
        }
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int k = 0; k < NC; ++k) Mt[r][k] = M0[k][r];
        ok = gauss_pp<NC>(Mt, lamP1, 1e-300) && ok;          // lamP1 = lamr1
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long q = (long long)c * N + p;
            A.s1_out[q] = A.s0[q] + lamP1[c] + (1.0 - f1 / gd) * lamP2[c];
            A.s0_out[q] = 0.0;
        }
        double gK[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        stage_param_terms<DIM>(K, lamP1, Y1, gd, A.G, C.g[0], A.Wi, A.Re, gK, gWi, gbeta);
        stage_param_terms<DIM>(K, lamP2, Psi1, gd, A.G, C.g[1], A.Wi, A.Re, gK, gWi, gbeta);
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) A.g_kap[(long long)(a * DIM + b) * N + p] += gK[a][b];
        if (!ok) atomicOr(A.flags, 2u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gWi += __shfl_xor_sync(0xffffffffu, gWi, off);
        gbeta += __shfl_xor_sync(0xffffffffu, gbeta, off);
    }
    const long long grp = p >> 5;
    if ((threadIdx.x & 31) == 0 && grp * 32 < N) {
        A.partials[2 * grp + 0] += gWi;
        A.partials[2 * grp + 1] += gbeta;
    }
}

template <typename T>
cudaError_t launch_start(const PaperStartAdjArgs<T>& a, const StartConsts& c, int dim, cudaStream_t s) {
    const long long blocks = (a.N + kThreads - 1) / kThreads;
    if (blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (a.m < 0 || a.m > kMaxModes) return cudaErrorInvalidValue;
    if (dim == 2) paper_start_adjoint_kernel<T, 2><<<(unsigned)blocks, kThreads, 0, s>>>(a, c);
    else paper_start_adjoint_kernel<T, 3><<<(unsigned)blocks, kThreads, 0, s>>>(a, c);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch(const PaperAdjArgs<T>& a, int dim, cudaStream_t s) {
    const long long blocks = (a.N + kThreads - 1) / kThreads;
    if (blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (a.m < 0 || a.m > kMaxModes) return cudaErrorInvalidValue;
    const int nc = dim == 2 ? 3 : 6;
    const size_t smem = sizeof(T) == 4 ? (size_t)a.m * nc * kThreads * sizeof(float) : 0;   // <= 196608
    auto kern = dim == 2 ? paper_adjoint_kernel<T, 2> : paper_adjoint_kernel<T, 3>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)blocks, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_paper_start_adjoint_f64(const PaperStartAdjArgs<double>& a, const StartConsts& c, int dim,
                                           cudaStream_t s) {
    return launch_start(a, c, dim, s);
}

cudaError_t launch_paper_start_adjoint_f32(const PaperStartAdjArgs<float>& a, const StartConsts& c, int dim,
                                           cudaStream_t s) {
    return launch_start(a, c, dim, s);
}

cudaError_t launch_paper_adjoint_f64(const PaperAdjArgs<double>& a, int dim, cudaStream_t s) {
    return launch(a, dim, s);
}

cudaError_t launch_paper_adjoint_f32(const PaperAdjArgs<float>& a, int dim, cudaStream_t s) {
    return launch(a, dim, s);
}

}  // namespace tfs
