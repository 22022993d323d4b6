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
                zs = fma(C.mu[jj] * C.inv_den[jj], (double)A.modes0[((long long)jj * NC + c) * N + p], zs);
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
                const double z0 = (double)A.modes0[((long long)jj * NC + c) * N + p];
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
                const long long q = ((long long)jj * NC + c) * N + p;
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
                hs = fma(C.w[jj] * C.mu[jj] * C.inv_den[jj], (double)A.modes0[((long long)jj * NC + c) * N + p], hs);
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
                const double z0 = (double)A.modes0[((long long)jj * NC + c) * N + p];
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
                const long long q = ((long long)jj * NC + c) * N + p;
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

cudaError_t launch_start_paper_f64(const StartArgs<double>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch<double, true>(a, c, dim, s);
}

cudaError_t launch_start_paper_f32(const StartArgs<float>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch<float, true>(a, c, dim, s);
}

}  // namespace tfs
