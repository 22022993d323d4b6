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

template <typename T>
cudaError_t launch(const StartArgs<T>& a, const StartConsts& c, int dim, cudaStream_t s) {
    long long blocks = (a.N + kThreads - 1) / kThreads;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (blocks < 1) blocks = 1;
    if (dim == 2) start_point_kernel<T, 2><<<(unsigned)blocks, kThreads, 0, s>>>(a, c);
    else start_point_kernel<T, 3><<<(unsigned)blocks, kThreads, 0, s>>>(a, c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_start_point_f64(const StartArgs<double>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch(a, c, dim, s);
}

cudaError_t launch_start_point_f32(const StartArgs<float>& a, const StartConsts& c, int dim, cudaStream_t s) {
    return launch(a, c, dim, s);
}

}  // namespace tfs
