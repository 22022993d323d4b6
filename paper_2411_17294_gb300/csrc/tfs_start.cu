// First step t_0 -> t_1 by two-stage SDIRK2 for the pointwise law (transport
// off), the start the paper uses for non-trivial initial data (Section 5.1)
// in place of BDF2 with an empty past.  SDIRK2 with gamma = 1 - 1/sqrt2 is
// stiffly accurate and L-stable.
//
// The kernel-compressed law is the system of mode ODEs
//   d sigma_j/dt = -mu_j sigma_j + w_j (sigma - sigma0)
// (those whose BDF2 discretisation is eq. BDF_Phi_k_n+1) constrained by
//   sum_j d sigma_j/dt = L(kappa) sigma - sigma/Wi + G (kappa + kappa^T) g_alpha(t),
// the mode sum standing for the Caputo derivative (Section 2.2).  At a stage
// with explicit mode part Z_j the implicit relation K_j = (-mu_j (Z_j + gamma dt
// K_j) + w_j (S - sigma0)) gives K_j = (-mu_j Z_j + w_j (S - sigma0)) / (1 +
// gamma mu_j dt), and the constraint becomes the point system
//   (dt W + dt/Wi) S - dt L(kappa^0) S = dt W sigma0 + dt sum_j mu_j Z_j/(1 + gamma mu_j dt)
//                                        + dt G (kappa^0 + kappa^0T) g_alpha(t_i),
// W = sum_j w_j / (1 + gamma mu_j dt).  Stage 1: t_1 = gamma dt, Z_j = sigma_j^0.
// Stage 2: t_2 = dt, Z_j = sigma_j^0 + dt (1 - gamma) K_j^(1).  Result: sigma^1 =
// S^(2), sigma_j^1 = Z_j^(2) + gamma dt K_j^(2).  kappa^0 is the velocity
// gradient of the first step (no past to extrapolate from).
//
// One thread per point; every quantity is formed in FP64 whatever the storage
// (one launch per run, so its cost does not matter), the stage-2 explicit part
// is recomputed from sigma_j^0 instead of stored.
#include <cuda_runtime.h>

#include "tfs_device.cuh"
#include "tfs_internal.h"

namespace tfs {
namespace {

constexpr int kThreads = 128;

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) start_point_kernel(const StartArgs<T> A, const StartConsts C) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (double)A.kap0[(long long)(i * DIM + j) * N + p];
        double M0[NC][NC];
        assemble_M<DIM>(K, A.a, A.dt, M0);
        double s0[NC], src[NC], S1[NC], S2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            s0[c] = A.sigma0 ? (double)A.sigma0[(long long)c * N + p] : 0.0;
            src[c] = A.G * (K[i][j] + K[j][i]);
        }
        bool ok = true;
        // stage 1: Z_j = sigma_j^0
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double zs = 0.0;
            for (int jj = 0; jj < A.m; ++jj)
                zs = fma(C.mu[jj] * C.inv_den[jj], (double)A.modes0[mode_index(p, jj * NC + c, A.m * NC)], zs);
            S1[c] = A.dt * (C.W * s0[c] + zs + src[c] * C.g[0]);
        }
        {
            double M[NC][NC];
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int k = 0; k < NC; ++k) M[r][k] = M0[r][k];
            ok = gauss_pp<NC>(M, S1, 1e-300) && ok;
        }
        // stage 2: Z_j = sigma_j^0 + dt (1 - gamma) K_j^(1)
        const double f1 = A.dt * (1.0 - C.gam);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double d = S1[c] - s0[c];
            double zs = 0.0;
            for (int jj = 0; jj < A.m; ++jj) {
                const double z0 = (double)A.modes0[mode_index(p, jj * NC + c, A.m * NC)];
                const double z = fma(f1, (-C.mu[jj] * z0 + C.w[jj] * d) * C.inv_den[jj], z0);
                zs = fma(C.mu[jj] * C.inv_den[jj], z, zs);
            }
            S2[c] = A.dt * (C.W * s0[c] + zs + src[c] * C.g[1]);
        }
        ok = gauss_pp<NC>(M0, S2, 1e-300) && ok;
        // sigma_j^1 = Z_j^(2) + gamma dt K_j^(2)
        const double f2 = A.dt * C.gam;
        bool finite = true;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double d1 = S1[c] - s0[c], d2 = S2[c] - s0[c];
            for (int jj = 0; jj < A.m; ++jj) {
                const long long q = mode_index(p, jj * NC + c, A.m * NC);
                const double z0 = (double)A.modes0[q];
                const double z = fma(f1, (-C.mu[jj] * z0 + C.w[jj] * d1) * C.inv_den[jj], z0);
                A.modes1[q] = (T)fma(f2, (-C.mu[jj] * z + C.w[jj] * d2) * C.inv_den[jj], z);
            }
            const T out = (T)S2[c];
            finite = finite && isfinite((double)out);
            A.sig1[(long long)c * N + p] = out;
            if (A.sig_copy) A.sig_copy[(long long)c * N + p] = out;
        }
        if (!ok) atomicOr(A.flags, 2u);
        if (!finite) atomicOr(A.flags, 1u);
    }
}

// The same start in the paper's variable (Section 3.4): the ODE system
//   d Phi/dt = (L(kappa) - I/Wi) Psi + G (kappa + kappa^T) Psi0,   d phi_j/dt = -mu_j phi_j + Phi,
//   Psi = sum_j w_j (-mu_j phi_j + Phi).
// At a stage with explicit parts ZPhi, Zphi_j the implicit mode relation gives
// phi_j = (Zphi_j + gamma dt Phi) / (1 + gamma mu_j dt), hence Psi = W Phi - h,
// h = sum_j w_j mu_j Zphi_j / (1 + gamma mu_j dt), W = sum_j w_j / (1 + gamma mu_j dt), and
//   (1 + gamma dt W/Wi) Phi - gamma dt W L(kappa^0) Phi
//       = ZPhi - gamma dt (L(kappa^0) h - h/Wi) + gamma dt G (kappa^0 + kappa^0T) Psi0(t_i).
// Stage 2 takes ZPhi = Phi^0 + dt (1 - gamma) (Phi^(1) - Phi^0)/(gamma dt) and
// Zphi_j = phi_j^0 + dt (1 - gamma) (-mu_j phi_j^(1) + Phi^(1)); the result is
// Phi^1 = Phi^(2), phi_j^1 = (Zphi_j^(2) + gamma dt Phi^1)/(1 + gamma mu_j dt),
// Psi^1 = W Phi^1 - h^(2).  Psi0 at the stages comes from the host (the same
// recurrence on Phi0 == 1).
template <int DIM>
__device__ __forceinline__ void upper_convected_minus(const double K[3][3], const double* h, double inv_wi,
                                                      double* out) {
    constexpr int NC = Packed<DIM>::NC;
    double H[3][3];
#pragma unroll
    for (int r = 0; r < NC; ++r) {
        H[Packed<DIM>::I(r)][Packed<DIM>::J(r)] = h[r];
        H[Packed<DIM>::J(r)][Packed<DIM>::I(r)] = h[r];
    }
#pragma unroll
    for (int r = 0; r < NC; ++r) {
        const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
        double v = -inv_wi * h[r];
#pragma unroll
        for (int l = 0; l < DIM; ++l) v = fma(K[i][l], H[l][j], fma(H[i][l], K[j][l], v));
        out[r] = v;
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) start_paper_kernel(const StartArgs<T> A, const StartConsts C) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double gd = C.gam * A.dt;
    const double f1 = A.dt * (1.0 - C.gam);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (double)A.kap0[(long long)(i * DIM + j) * N + p];
        double M0[NC][NC];
        assemble_M<DIM>(K, A.a, gd * C.W, M0);
        double P0[NC], src[NC], h[NC], Lh[NC], P1[NC], P2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            P0[c] = A.sigma0 ? (double)A.sigma0[(long long)c * N + p] : 0.0;
            src[c] = A.G * (K[i][j] + K[j][i]);
        }
        bool ok = true;
        // stage 1: ZPhi = Phi^0, Zphi_j = phi_j^0
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double hs = 0.0;
            for (int jj = 0; jj < A.m; ++jj)
                hs = fma(C.w[jj] * C.mu[jj] * C.inv_den[jj], (double)A.modes0[mode_index(p, jj * NC + c, A.m * NC)], hs);
            h[c] = hs;
        }
        upper_convected_minus<DIM>(K, h, A.inv_wi, Lh);
#pragma unroll
        for (int c = 0; c < NC; ++c) P1[c] = P0[c] - gd * Lh[c] + gd * src[c] * C.g[0];
        {
            double M[NC][NC];
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int k = 0; k < NC; ++k) M[r][k] = M0[r][k];
            ok = gauss_pp<NC>(M, P1, 1e-300) && ok;
        }
        // stage 2 explicit parts (Zphi_j recomputed from phi_j^0 and Phi^(1) when needed)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double hs = 0.0;
            for (int jj = 0; jj < A.m; ++jj) {
                const double z0 = (double)A.modes0[mode_index(p, jj * NC + c, A.m * NC)];
                const double ph = fma(gd, P1[c], z0) * C.inv_den[jj];
                const double z = fma(f1, P1[c] - C.mu[jj] * ph, z0);
                hs = fma(C.w[jj] * C.mu[jj] * C.inv_den[jj], z, hs);
            }
            h[c] = hs;
        }
        upper_convected_minus<DIM>(K, h, A.inv_wi, Lh);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double zP = P0[c] + f1 * (P1[c] - P0[c]) / gd;
            P2[c] = zP - gd * Lh[c] + gd * src[c] * C.g[1];
        }
        ok = gauss_pp<NC>(M0, P2, 1e-300) && ok;
        bool finite = true;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            for (int jj = 0; jj < A.m; ++jj) {
                const long long q = mode_index(p, jj * NC + c, A.m * NC);
                const double z0 = (double)A.modes0[q];
                const double ph = fma(gd, P1[c], z0) * C.inv_den[jj];
                const double z = fma(f1, P1[c] - C.mu[jj] * ph, z0);
                A.modes1[q] = (T)(fma(gd, P2[c], z) * C.inv_den[jj]);
            }
            const T phi = (T)P2[c];
            const T psi = (T)fma(C.W, P2[c], -h[c]);
            finite = finite && isfinite((double)phi) && isfinite((double)psi);
            A.sig1[(long long)c * N + p] = phi;
            A.psi[(long long)c * N + p] = psi;
            if (A.sig_copy) A.sig_copy[(long long)c * N + p] = psi;
        }
        if (!ok) atomicOr(A.flags, 2u);
        if (!finite) atomicOr(A.flags, 1u);
    }
}

// Adjoint of start_point_kernel for zero initial modes (the state tfs_set_state
// leaves).  With Z_j^(1) = 0 the forward reads
//   r1 = dt (W s0 + G k g1),                      S1 = M^-1 r1
//   Z2_j = dt (1 - gamma) w_j iota_j (S1 - s0),    iota_j = 1/(1 + gamma mu_j dt)
//   r2 = dt (W s0 + sum_j mu_j iota_j Z2_j + G k g2),  S2 = M^-1 r2
//   sigma_j^1 = Z2_j (1 - gamma dt mu_j iota_j) + gamma dt w_j iota_j (S2 - s0),  sigma^1 = S2
// (M = (dt W + dt/Wi) I - dt L(kappa^0), k = kappa^0 + kappa^0T, s0 = sigma0 = sigma^0), and
// its reverse, given the adjoints lam1 of sigma^1, z_j of sigma_j^1 and s0in of
// sigma^0 (as the next step's level n-1):
//   lamS2 = lam1 + sum_j z_j gamma dt w_j iota_j;    lamZ2_j = z_j (1 - gamma dt mu_j iota_j)
//   lamr2 = M^-T lamS2;  lamZ2_j += dt mu_j iota_j lamr2
//   lamS1 = sum_j lamZ2_j dt (1 - gamma) w_j iota_j;  lamr1 = M^-T lamS1
//   dJ/dsigma0 = s0in + dt W (lamr1 + lamr2) - sum_j (z_j gamma dt + lamZ2_j dt (1 - gamma)) w_j iota_j
// and for each stage i the terms of the BDF2 adjoint with (lamR, sigma, g) =
// (lamr_i, S_i, g_i): dJ/dkappa += dt lamr_i-weighted (S kappa-derivatives) + dt G g_i
// (sym), dJ/dWi += (dt/Wi^2) <lamr_i, S_i> - (G/Wi) dt g_i <lamr_i, k>, dJ/dbeta +=
// -dt g_i <lamr_i, k> / (Wi Re).  FP64 per point whatever the storage.
template <typename T, int DIM>
__global__ void __launch_bounds__(32) start_adjoint_kernel(const StartAdjArgs<T> A, const StartConsts C) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const long long p = (long long)blockIdx.x * 32 + threadIdx.x;
    double gWi = 0.0, gbeta = 0.0;
    if (p < N) {
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (double)A.kap0[(long long)(i * DIM + j) * N + p];
        double M0[NC][NC];
        assemble_M<DIM>(K, A.a, A.dt, M0);
        const double f1 = A.dt * (1.0 - C.gam), f2 = A.dt * C.gam;
        double s0[NC], ks[NC], S1[NC], S2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            s0[c] = A.sigma0 ? (double)A.sigma0[(long long)c * N + p] : 0.0;
            ks[c] = K[i][j] + K[j][i];
        }
        bool ok = true;
        // forward stages (zero initial modes)
#pragma unroll
        for (int c = 0; c < NC; ++c) S1[c] = A.dt * (C.W * s0[c] + A.G * ks[c] * C.g[0]);
        {
            double M[NC][NC];
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int k = 0; k < NC; ++k) M[r][k] = M0[r][k];
            ok = gauss_pp<NC>(M, S1, 1e-300) && ok;
        }
        double c1 = 0.0;     // sum_j mu_j iota_j f1 w_j iota_j: Z2 enters r2 through it
        for (int jj = 0; jj < A.m; ++jj) c1 += C.mu[jj] * C.inv_den[jj] * f1 * C.w[jj] * C.inv_den[jj];
#pragma unroll
        for (int c = 0; c < NC; ++c) S2[c] = A.dt * (C.W * s0[c] + c1 * (S1[c] - s0[c]) + A.G * ks[c] * C.g[1]);
        {
            double M[NC][NC];
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int k = 0; k < NC; ++k) M[r][k] = M0[r][k];
            ok = gauss_pp<NC>(M, S2, 1e-300) && ok;
        }
        // reverse
        double lamS2[NC], lamS1[NC], gs0[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            lamS2[c] = A.s1[(long long)c * N + p];
            gs0[c] = A.s0[(long long)c * N + p];
        }
        // lamZ2_j = z_j (1 - f2 mu_j iota_j) + dt mu_j iota_j lamr2 needs lamr2 first:
        // accumulate the z-only parts now, the lamr2 part after the solve
        double zq[NC];   // sum_j z_j (1 - f2 mu_j iota_j) f1 w_j iota_j
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double a1 = 0.0, a2 = 0.0;
            for (int jj = 0; jj < A.m; ++jj) {
                const long long q = mode_index(p, jj * NC + c, A.m * NC);
                const double z = kB1 * (double)A.ell_prev[q] + kB2 * (double)A.ell_prev2[q];
                const double wi = C.w[jj] * C.inv_den[jj];
                a1 = fma(z, f2 * wi, a1);
                a2 = fma(z * (1.0 - f2 * C.mu[jj] * C.inv_den[jj]), f1 * wi, a2);
            }
            zq[c] = a2;
            lamS2[c] += a1;
            gs0[c] -= a1;
        }
        double Mt[NC][NC];
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int k = 0; k < NC; ++k) Mt[r][k] = M0[k][r];
        double lr2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) lr2[c] = lamS2[c];
        {
            double M[NC][NC];
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int k = 0; k < NC; ++k) M[r][k] = Mt[r][k];
            ok = gauss_pp<NC>(M, lr2, 1e-300) && ok;
        }
        // lamS1 = sum_j lamZ2_j f1 w_j iota_j = zq + dt c1 lamr2
#pragma unroll
        for (int c = 0; c < NC; ++c) lamS1[c] = zq[c] + A.dt * c1 * lr2[c];
        double lr1[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) lr1[c] = lamS1[c];
        ok = gauss_pp<NC>(Mt, lr1, 1e-300) && ok;
        // dJ/dsigma0
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            gs0[c] += A.dt * C.W * (lr1[c] + lr2[c]) - lamS1[c];
            A.s1_out[(long long)c * N + p] = gs0[c];
            A.s0_out[(long long)c * N + p] = 0.0;
        }
        // parameter derivatives, per stage
        double gK[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int st = 0; st < 2; ++st) {
            const double* lam = st == 0 ? lr1 : lr2;
            const double* sig = st == 0 ? S1 : S2;
            double S3[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
                S3[i][j] = sig[r];
                S3[j][i] = sig[r];
            }
            const double src = A.dt * A.G * C.g[st];
            double sym_dot = 0.0, sig_dot = 0.0;
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) {
                const int r = Packed<DIM>::I(cc), s2 = Packed<DIM>::J(cc);
                const double l = lam[cc];
#pragma unroll
                for (int b = 0; b < DIM; ++b) {
                    gK[r][b] += A.dt * l * S3[b][s2];
                    gK[s2][b] += A.dt * l * S3[r][b];
                }
                gK[r][s2] += src * l;
                gK[s2][r] += src * l;
                sym_dot += l * ks[cc];
                sig_dot += l * sig[cc];
            }
            const double lam_a = -sig_dot;
            const double lam_G = A.dt * C.g[st] * sym_dot;
            gWi += -A.dt / (A.Wi * A.Wi) * lam_a - A.G / A.Wi * lam_G;
            gbeta += -lam_G / (A.Wi * A.Re);
        }
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
    if (threadIdx.x == 0) {
        A.partials[2 * (long long)blockIdx.x + 0] += gWi;
        A.partials[2 * (long long)blockIdx.x + 1] += gbeta;
    }
}

template <typename T>
cudaError_t launch_adj(const StartAdjArgs<T>& a, const StartConsts& c, int dim, cudaStream_t s) {
    const long long blocks = (a.N + 31) / 32;
    if (blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (dim == 2) start_adjoint_kernel<T, 2><<<(unsigned)blocks, 32, 0, s>>>(a, c);
    else start_adjoint_kernel<T, 3><<<(unsigned)blocks, 32, 0, s>>>(a, c);
    return cudaGetLastError();
}

template <typename T, bool PAPER>
cudaError_t launch(const StartArgs<T>& a, const StartConsts& c, int dim, cudaStream_t s) {
    long long blocks = (a.N + kThreads - 1) / kThreads;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (blocks < 1) blocks = 1;
    if (PAPER && !a.psi) return cudaErrorInvalidValue;
    if (dim == 2) {
        if (PAPER) start_paper_kernel<T, 2><<<(unsigned)blocks, kThreads, 0, s>>>(a, c);
        else start_point_kernel<T, 2><<<(unsigned)blocks, kThreads, 0, s>>>(a, c);
    } else {
        if (PAPER) start_paper_kernel<T, 3><<<(unsigned)blocks, kThreads, 0, s>>>(a, c);
        else start_point_kernel<T, 3><<<(unsigned)blocks, kThreads, 0, s>>>(a, c);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_start_point_f64(const StartArgs<double>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch<double, false>(a, c, dim, s);
}

cudaError_t launch_start_point_f32(const StartArgs<float>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch<float, false>(a, c, dim, s);
}

cudaError_t launch_start_adjoint_f64(const StartAdjArgs<double>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch_adj(a, c, dim, s);
}

cudaError_t launch_start_adjoint_f32(const StartAdjArgs<float>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch_adj(a, c, dim, s);
}

cudaError_t launch_start_paper_f64(const StartArgs<double>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch<double, true>(a, c, dim, s);
}

cudaError_t launch_start_paper_f32(const StartArgs<float>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch<float, true>(a, c, dim, s);
}

}  // namespace tfs
