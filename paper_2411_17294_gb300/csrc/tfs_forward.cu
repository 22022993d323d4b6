// Forward stress step: one launch advances every grid point from t_n to t_{n+1}.
//
// Per point (Section 4.1 with the kernel compression of Section 2.2):
//   kappa* = 2 kappa^n - kappa^{n-1}, E = 2 sigma^n - sigma^{n-1}
//   A  = dt sum_a u_a D_a(E) - eps dt Lap(E)           (periodic stencil, explicit)
//   H  = sum_j eta_j (b1 sigma_j^n + b2 sigma_j^{n-1})  (mode history sum)
//   R  = eta sigma0 - H + dt G (kappa* + kappa*^T) g - A
//   solve (eta + dt/Wi) s - dt (kappa* s + s kappa*^T) = R   -> sigma^{n+1}
//   sigma_j^{n+1} = -c_j (b1 sigma_j^n + b2 sigma_j^{n-1}) + rho_j (sigma^{n+1} - sigma0)
//
// Thread layout: a block covers 32 consecutive points; warp c of the block
// handles stress component c for those points (lane = point).  Mode arrays are
// [m][nc][N], so every warp load/store of one (mode, component) plane is a
// single 128-byte line.  Each thread keeps the m history terms Q_j of its
// (point, component) in registers between the history sum and the push-forward,
// so every mode value is read once and written once per step.  The nc x nc
// point systems of the block are solved by warp 0 (lane = point) in FP64; the
// other warps exchange R and sigma^{n+1} - sigma0 through shared memory.
#include <cuda_runtime.h>

#include "tfs_device.cuh"
#include "tfs_internal.h"

namespace tfs {
namespace {

template <typename T, int DIM, bool TRANSPORT>
__device__ __forceinline__ double transport_term(const FwdArgs<T>& A, const GridIdx& g, int c,
                                                 int stencil, long long p) {
    // E = 2 sigma^n - sigma^{n-1} at a neighbour, in the storage precision
    const T* sn = A.sig_n + (long long)c * A.N;
    const T* sm = A.sig_nm1 + (long long)c * A.N;
    auto E = [&](long long q) -> T { return (T)2 * __ldg(sn + q) - __ldg(sm + q); };
    T adv = (T)0, lap = (T)0;
    const T e0 = E(p);
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        const T ua = __ldg(A.u + (long long)ax * A.N + p);
        const T ih = (T)A.inv_h[ax];
        const T em1 = E(g.at(ax, -1)), ep1 = E(g.at(ax, 1));
        T d;
        if (stencil == 1) {
            d = (ep1 - em1) * ((T)0.5 * ih);
        } else if (ua >= (T)0) {
            const T em2 = E(g.at(ax, -2));
            d = (em2 - (T)6 * em1 + (T)3 * e0 + (T)2 * ep1) * (ih / (T)6);
        } else {
            const T ep2 = E(g.at(ax, 2));
            d = ((T)-2 * em1 - (T)3 * e0 + (T)6 * ep1 - ep2) * (ih / (T)6);
        }
        adv += ua * d;
        if (A.eps != 0.0) lap += (em1 - (T)2 * e0 + ep1) * (ih * ih);
    }
    return A.dt * to_d(adv) - A.eps * A.dt * to_d(lap);
}

template <typename T, int DIM, int MT, bool TRANSPORT, bool COMP>
__global__ void __launch_bounds__(32 * Packed<DIM>::NC)
fwd_kernel(const FwdArgs<T> A, const int stencil, const int classic) {
    constexpr int NC = Packed<DIM>::NC;
    __shared__ double sR[NC][32];
    __shared__ double sD[NC][32];

    const int lane = threadIdx.x;
    const int c = threadIdx.y;
    const long long N = A.N;
    const long long p = (long long)blockIdx.x * 32 + lane;
    const bool active = p < N;
    const long long pc = active ? p : 0;   // clamped index for inactive lanes

    // ---- (a4) history sum over the modes of component c -------------------
    T Q[MT > 0 ? MT : 1];
    double H = 0.0;
    if (classic) {
        if (active) {
            const long long q = (long long)c * N + p;
            const double s0 = A.sigma0 ? to_d(A.sigma0[q]) : 0.0;
            H = kB1 * to_d(A.sig_n[q]) + kB2 * to_d(A.sig_nm1[q]) + kB0 * s0;
        }
    } else {
        const T* mn = A.modes_n + (long long)c * N + pc;
        const T* mm = A.modes_nm1 + (long long)c * N + pc;
        const long long stride = (long long)NC * N;
        if constexpr (sizeof(T) == 4 && COMP) {
            // compensated dot product (Ogita-Rump-Oishi Dot2): exact products by
            // FMA, error-free sums, eta_j carried as hi + lo floats
            float hs = 0.f, he = 0.f;
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                if (j < A.m) {
                    const float x = __ldcs(mn + j * stride);
                    const float y = __ldcs(mm + j * stride);
                    const float qj = __fmaf_rn(0.5f, y, -2.0f * x);   // b1 x + b2 y, one rounding
                    Q[j] = qj;
                    const float pr = __fmul_rn(A.mc.eta_hi[j], qj);
                    const float pe = __fmaf_rn(A.mc.eta_hi[j], qj, -pr);
                    float s, e;
                    two_sum(hs, pr, s, e);
                    hs = s;
                    he = __fadd_rn(he, __fadd_rn(e, __fmaf_rn(A.mc.eta_lo[j], qj, pe)));
                }
            }
            H = (double)hs + (double)he;
        } else if constexpr (sizeof(T) == 4) {
            float hs = 0.f;
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                if (j < A.m) {
                    const float x = __ldcs(mn + j * stride);
                    const float y = __ldcs(mm + j * stride);
                    const float qj = __fmaf_rn(0.5f, y, -2.0f * x);
                    Q[j] = qj;
                    hs = __fmaf_rn(A.mc.eta_hi[j], qj, hs);
                }
            }
            H = (double)hs;
        } else {
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                if (j < A.m) {
                    const double x = __ldcs(mn + j * stride);
                    const double y = __ldcs(mm + j * stride);
                    const double qj = kB1 * x + kB2 * y;
                    Q[j] = (T)qj;
                    H = fma(A.mc.eta[j], qj, H);
                }
            }
        }
    }

    // ---- right-hand side component c ------------------------------------
    double R = 0.0;
    const double s0c = (active && A.sigma0) ? to_d(A.sigma0[(long long)c * N + p]) : 0.0;
    if (active) {
        const int ci = Packed<DIM>::I(c), cj = Packed<DIM>::J(c);
        const long long kij = (long long)(ci * DIM + cj) * N + p;
        const long long kji = (long long)(cj * DIM + ci) * N + p;
        const double ks = (2.0 * to_d(A.kap_n[kij]) - to_d(A.kap_nm1[kij])) +
                          (2.0 * to_d(A.kap_n[kji]) - to_d(A.kap_nm1[kji]));
        R = A.eta * s0c - H + A.dt * A.G * A.g * ks;
        if constexpr (TRANSPORT) {
            GridIdx g;
            g.n0 = A.n0; g.n1 = A.n1; g.n2 = A.n2;
            g.x = p % A.n0;
            g.y = (p / A.n0) % A.n1;
            g.z = p / ((long long)A.n0 * A.n1);
            R -= transport_term<T, DIM, TRANSPORT>(A, g, c, stencil, p);
        }
    }
    sR[c][lane] = R;
    __syncthreads();

    // ---- (a2) + (a5) per-point solve by warp 0 ---------------------------
    if (c == 0) {
        double x[NC];
#pragma unroll
        for (int r = 0; r < NC; ++r) x[r] = sR[r][lane];
        bool ok = true;
        if (active) {
            double K[3][3];
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
                for (int b = 0; b < DIM; ++b) {
                    const long long q = (long long)(a * DIM + b) * N + p;
                    K[a][b] = 2.0 * to_d(A.kap_n[q]) - to_d(A.kap_nm1[q]);
                }
            double M[NC][NC];
            assemble_M<DIM>(K, A.a, A.dt, M);
            ok = gauss_pp<NC>(M, x, 1e-300);
            bool finite = true;
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                const T v = (T)x[r];
                finite = finite && isfinite(to_d(v));
                A.sig_np1[(long long)r * N + p] = v;
                if (A.sig_copy) A.sig_copy[(long long)r * N + p] = v;
            }
            unsigned fl = (ok ? 0u : 2u) | (finite ? 0u : 1u);
            if (TRANSPORT && A.courant_coef > 0.0) {
                double cr = 0.0;
#pragma unroll
                for (int ax = 0; ax < DIM; ++ax) cr += fabs(to_d(A.u[(long long)ax * N + p])) * A.inv_h[ax];
                if (A.courant_coef * cr > A.courant_limit) fl |= 4u;
            }
            if (fl) atomicOr(A.flags, fl);
        }
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const double s0r = (active && A.sigma0) ? to_d(A.sigma0[(long long)r * N + pc]) : 0.0;
            // the push-forward uses the stored (rounded) value of sigma^{n+1}
            sD[r][lane] = to_d((T)x[r]) - s0r;
        }
    }
    __syncthreads();

    // ---- (a6) mode push-forward over the oldest level ---------------------
    if (!classic && active) {
        const double d = sD[c][lane];
        T* out = A.modes_nm1 + (long long)c * N + p;
        const long long stride = (long long)NC * N;
        if constexpr (sizeof(T) == 4) {
            const float df = (float)d;
#pragma unroll
            for (int j = 0; j < MT; ++j)
                if (j < A.m) __stcs(out + j * stride, __fmaf_rn(A.mc.rho[j], df, -A.mc.c[j] * Q[j]));
        } else {
#pragma unroll
            for (int j = 0; j < MT; ++j)
                if (j < A.m) __stcs(out + j * stride, (T)fma(A.mc.rho[j], d, -A.mc.c[j] * (double)Q[j]));
        }
    }
}

template <typename T, int DIM, int MT, bool TRANSPORT, bool COMP>
cudaError_t launch_one(const FwdArgs<T>& a, const LaunchCfg& cfg, cudaStream_t s) {
    constexpr int NC = Packed<DIM>::NC;
    const long long blocks = (a.N + 31) / 32;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)blocks), block(32, NC);
    fwd_kernel<T, DIM, MT, TRANSPORT, COMP><<<grid, block, 0, s>>>(a, cfg.stencil, cfg.classic ? 1 : 0);
    return cudaGetLastError();
}

template <typename T, int DIM, bool TRANSPORT, bool COMP>
cudaError_t dispatch_mt(const FwdArgs<T>& a, const LaunchCfg& cfg, cudaStream_t s) {
    const int m = cfg.classic ? 0 : a.m;
    if (m <= 8) return launch_one<T, DIM, 8, TRANSPORT, COMP>(a, cfg, s);
    if (m <= 16) return launch_one<T, DIM, 16, TRANSPORT, COMP>(a, cfg, s);
    if (m <= 32) return launch_one<T, DIM, 32, TRANSPORT, COMP>(a, cfg, s);
    if (m <= 48) return launch_one<T, DIM, 48, TRANSPORT, COMP>(a, cfg, s);
    return launch_one<T, DIM, 64, TRANSPORT, COMP>(a, cfg, s);
}

template <typename T, bool COMP>
cudaError_t dispatch(const FwdArgs<T>& a, const LaunchCfg& cfg, cudaStream_t s) {
    if (cfg.dim == 2)
        return cfg.transport ? dispatch_mt<T, 2, true, COMP>(a, cfg, s) : dispatch_mt<T, 2, false, COMP>(a, cfg, s);
    return cfg.transport ? dispatch_mt<T, 3, true, COMP>(a, cfg, s) : dispatch_mt<T, 3, false, COMP>(a, cfg, s);
}

}  // namespace

cudaError_t launch_forward_f64(const FwdArgs<double>& a, const LaunchCfg& cfg, cudaStream_t s) {
    return dispatch<double, false>(a, cfg, s);
}

cudaError_t launch_forward_f32(const FwdArgs<float>& a, const LaunchCfg& cfg, cudaStream_t s) {
    return cfg.compensated ? dispatch<float, true>(a, cfg, s) : dispatch<float, false>(a, cfg, s);
}

}  // namespace tfs
