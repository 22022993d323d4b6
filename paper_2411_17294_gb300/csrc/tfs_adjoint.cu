// Adjoint (reverse-mode derivative) of one forward stress step.
//
// The forward step maps (sigma^n, sigma^{n-1}, modes^n, modes^{n-1}) to
// (sigma^{n+1}, sigma^n, modes^{n+1}, modes^n).  Its push-forward
// modes_j^{n+1} = -c_j Q_j + rho_j (sigma^{n+1} - sigma0), Q_j = b1 modes_j^n + b2 modes_j^{n-1},
// is linear, so the adjoint of the mode history needs only one new value per
// (mode, component, point) and step:
//     lamQ_j = -c_j z_j - eta_j lamR,     z_j = b1 lamQ_j' + b2 lamQ_j''
// where lamQ' and lamQ'' are the values of the two later steps (zero at the
// final time) and z_j is the adjoint of modes_j^{n+1}.  The adjoint modes are
// therefore a two-level ring like the forward modes: read two levels, write
// one.  The stress part per point:
//     lam_sigma^{n+1} = s1 + sum_j rho_j z_j
//     M(kappa*)^T lamR = lam_sigma^{n+1}          (FP64 point solve)
//     dJ/dsigma0 += eta lamR - sum_j rho_j z_j
//     dJ/dkappa* += dt <lamR, dM/dkappa sigma^{n+1}>-terms + dt G g d(kappa+kappa^T)^T lamR
//     dJ/dWi     += -dt/Wi^2 (-<lamR, sigma^{n+1}>) - G/Wi (dt g <lamR, sym kappa*>)
//     dJ/dbeta   += -(dt g <lamR, sym kappa*>) / (Wi Re)
// and the transport term A = dt (u.grad_h - eps Lap_h)(2 sigma^n - sigma^{n-1})
// sends -lamR back through the transposed stencil (second kernel).
// The forward modes themselves are never needed: only sigma^{n+1} and kappa.
#include <cuda_runtime.h>

#include "tfs_device.cuh"
#include "tfs_internal.h"

namespace tfs {
namespace {

template <typename T, int DIM, int MT>
__global__ void __launch_bounds__(32 * Packed<DIM>::NC)
adj_kernel(const AdjArgs<T> A, const int classic) {
    constexpr int NC = Packed<DIM>::NC;
    __shared__ double sS[NC][32];     // sum_j rho_j z_j per component
    __shared__ double sL[NC][32];     // lamR per component
    __shared__ double sRed[2][NC];    // block reduction of the scalar gradients

    const int lane = threadIdx.x;
    const int c = threadIdx.y;
    const long long N = A.N;
    const long long p = (long long)blockIdx.x * 32 + lane;
    const bool active = p < N;
    const long long pc = active ? p : 0;
    const long long stride = (long long)NC * N;

    // ---- z_j and sum_j rho_j z_j for component c --------------------------
    double Z[MT > 0 ? MT : 1];
    double S = 0.0;
    if (!classic) {
        const T* e1 = A.ell_prev + (long long)c * N + pc;
        const T* e2 = A.ell_prev2 + (long long)c * N + pc;
#pragma unroll
        for (int j = 0; j < MT; ++j) {
            if (j < A.m) {
                double z = 0.0;
                if (!A.first) z = kB1 * to_d(__ldcs(e1 + j * stride)) + kB2 * to_d(__ldcs(e2 + j * stride));
                Z[j] = z;
                S = fma(A.mc.rho[j], z, S);
            }
        }
    }
    sS[c][lane] = S;
    __syncthreads();

    double gWi = 0.0, gbeta = 0.0;
    if (c == 0 && active) {
        double K[3][3];
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                const long long q = (long long)(a * DIM + b) * N + p;
                K[a][b] = 2.0 * to_d(A.kap_n[q]) - to_d(A.kap_nm1[q]);
            }
        double sig[NC], lam[NC];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            sig[r] = to_d(A.sig_np1[(long long)r * N + p]);
            lam[r] = A.s1[(long long)r * N + p] + sS[r][lane];
        }
        double M[NC][NC], Mt[NC][NC];
        assemble_M<DIM>(K, A.a, A.dt, M);
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int k = 0; k < NC; ++k) Mt[r][k] = M[k][r];
        const bool ok = gauss_pp<NC>(Mt, lam, 1e-300);
        if (!ok) atomicOr(A.flags, 2u);
        // lam now holds lamR

        // d/dkappa* of <lamR, M sigma> and of the source term
        double gK[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) gK[a][b] = 0.0;
        double S3[3][3];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
            S3[i][j] = sig[r];
            S3[j][i] = sig[r];
        }
        const double src = A.dt * A.G * A.g;
        double sym_dot = 0.0, sig_dot = 0.0;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            const int r = Packed<DIM>::I(cc), s = Packed<DIM>::J(cc);
            const double l = lam[cc];
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                gK[r][b] += A.dt * l * S3[b][s];
                gK[s][b] += A.dt * l * S3[r][b];
            }
            gK[r][s] += src * l;
            gK[s][r] += src * l;
            sym_dot += l * (K[r][s] + K[s][r]);
            sig_dot += l * sig[cc];
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                const long long q = (long long)(a * DIM + b) * N + p;
                A.g_kap[q] += gK[a][b];
            }
        const double lam_a = -sig_dot;
        const double lam_G = A.dt * A.g * sym_dot;
        gWi = -A.dt / (A.Wi * A.Wi) * lam_a - A.G / A.Wi * lam_G;
        gbeta = -lam_G / (A.Wi * A.Re);

#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const long long q = (long long)r * N + p;
            sL[r][lane] = lam[r];
            A.lamR[q] = lam[r];
            double gs = A.eta * lam[r] - sS[r][lane];
            double s1o = A.s0[q];
            double s0o = 0.0;
            if (classic) {
                const double lamH = -lam[r];
                s1o += kB1 * lamH;
                s0o += kB2 * lamH;
                gs += kB0 * lamH;
            }
            A.g_sigma0[q] += gs;
            A.s1_out[q] = s1o;
            A.s0_out[q] = s0o;
        }
    }

    // block reduction of the two scalar gradients (warp 0 holds them)
    if (c == 0) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            gWi += __shfl_xor_sync(0xffffffffu, gWi, off);
            gbeta += __shfl_xor_sync(0xffffffffu, gbeta, off);
        }
        if (lane == 0) {
            A.partials[2 * (long long)blockIdx.x + 0] += gWi;
            A.partials[2 * (long long)blockIdx.x + 1] += gbeta;
        }
    }
    (void)sRed;
    __syncthreads();

    // ---- new adjoint mode level: lamQ_j = -c_j z_j - eta_j lamR ---------------
    if (!classic && active) {
        const double l = sL[c][lane];
        T* out = A.ell_prev2 + (long long)c * N + p;
#pragma unroll
        for (int j = 0; j < MT; ++j)
            if (j < A.m) __stcs(out + j * stride, (T)fma(-A.mc.eta[j], l, -A.mc.c[j] * Z[j]));
    }
}

// Transposed stencil: the forward step added  -dt (u.grad_h - eps Lap_h) E  to
// R at point p, E = 2 sigma^n - sigma^{n-1}; so each point q receives
// lamE(q) = sum over points p whose stencil reads q of  -coef * lamR(p).
template <typename TU, int DIM>
__global__ void adj_transport_kernel(const AdjArgs<double> A, const TU* __restrict__ u, const int stencil) {
    constexpr int NC = Packed<DIM>::NC;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.N) return;
    GridIdx g;
    g.n0 = A.n0; g.n1 = A.n1; g.n2 = A.n2;
    g.x = q % A.n0;
    g.y = (q / A.n0) % A.n1;
    g.z = q / ((long long)A.n0 * A.n1);
    double lamE[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) lamE[c] = 0.0;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        const double ih = A.inv_h[ax];
        // the point p = q - k e_ax read q with its tap k
#pragma unroll
        for (int k = -2; k <= 2; ++k) {
            const long long pnb = g.at(ax, -k);
            const double ua = (double)u[(long long)ax * A.N + pnb];
            double coef;
            if (stencil == 1) {
                coef = (k == 1) ? 0.5 * ih : (k == -1) ? -0.5 * ih : 0.0;
            } else if (ua >= 0.0) {
                coef = (k == -2) ? ih / 6.0 : (k == -1) ? -ih : (k == 0) ? 0.5 * ih : (k == 1) ? ih / 3.0 : 0.0;
            } else {
                coef = (k == -1) ? -ih / 3.0 : (k == 0) ? -0.5 * ih : (k == 1) ? ih : (k == 2) ? -ih / 6.0 : 0.0;
            }
            double lapc = 0.0;
            if (A.eps != 0.0) lapc = (k == 0) ? -2.0 * ih * ih : (k == 1 || k == -1) ? ih * ih : 0.0;
            const double w = A.dt * (ua * coef - A.eps * lapc);
            if (w != 0.0) {
#pragma unroll
                for (int c = 0; c < NC; ++c) lamE[c] -= w * A.lamR[(long long)c * A.N + pnb];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const long long i = (long long)c * A.N + q;
        A.s1_out[i] += 2.0 * lamE[c];
        A.s0_out[i] -= lamE[c];
    }
}

__global__ void reduce_partials_kernel(const double* __restrict__ partials, int count, double* out2) {
    __shared__ double s[2][256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            s[0][threadIdx.x] += s[0][threadIdx.x + off];
            s[1][threadIdx.x] += s[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = s[0][0];
        out2[1] = s[1][0];
    }
}

template <typename T, int DIM, int MT>
cudaError_t launch_adj(const AdjArgs<T>& a, const LaunchCfg& cfg, cudaStream_t s) {
    constexpr int NC = Packed<DIM>::NC;
    const long long blocks = (a.N + 31) / 32;
    adj_kernel<T, DIM, MT><<<dim3((unsigned)blocks), dim3(32, NC), 0, s>>>(a, cfg.classic ? 1 : 0);
    return cudaGetLastError();
}

template <typename T, int DIM>
cudaError_t dispatch_mt(const AdjArgs<T>& a, const LaunchCfg& cfg, cudaStream_t s) {
    const int m = cfg.classic ? 0 : a.m;
    if (m <= 8) return launch_adj<T, DIM, 8>(a, cfg, s);
    if (m <= 16) return launch_adj<T, DIM, 16>(a, cfg, s);
    if (m <= 32) return launch_adj<T, DIM, 32>(a, cfg, s);
    if (m <= 48) return launch_adj<T, DIM, 48>(a, cfg, s);
    return launch_adj<T, DIM, 64>(a, cfg, s);
}

}  // namespace

cudaError_t launch_adjoint_f64(const AdjArgs<double>& a, const LaunchCfg& cfg, cudaStream_t s) {
    return cfg.dim == 2 ? dispatch_mt<double, 2>(a, cfg, s) : dispatch_mt<double, 3>(a, cfg, s);
}

cudaError_t launch_adjoint_f32(const AdjArgs<float>& a, const LaunchCfg& cfg, cudaStream_t s) {
    return cfg.dim == 2 ? dispatch_mt<float, 2>(a, cfg, s) : dispatch_mt<float, 3>(a, cfg, s);
}

cudaError_t launch_adjoint_transport(const AdjArgs<double>& a, const void* u, bool u_is_double,
                                     const LaunchCfg& cfg, cudaStream_t s) {
    const int threads = 256;
    const long long blocks = (a.N + threads - 1) / threads;
    if (cfg.dim == 2) {
        if (u_is_double) adj_transport_kernel<double, 2><<<(unsigned)blocks, threads, 0, s>>>(a, (const double*)u, cfg.stencil);
        else adj_transport_kernel<float, 2><<<(unsigned)blocks, threads, 0, s>>>(a, (const float*)u, cfg.stencil);
    } else {
        if (u_is_double) adj_transport_kernel<double, 3><<<(unsigned)blocks, threads, 0, s>>>(a, (const double*)u, cfg.stencil);
        else adj_transport_kernel<float, 3><<<(unsigned)blocks, threads, 0, s>>>(a, (const float*)u, cfg.stencil);
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, int count, double* out2, cudaStream_t s) {
    reduce_partials_kernel<<<1, 256, 0, s>>>(partials, count, out2);
    return cudaGetLastError();
}

}  // namespace tfs
