// Step with implicit transport: u.grad and eps Lap act on sigma^{n+1} inside
// the solve, the form in which the paper's scheme carries them (eq.
// FP_discrete), instead of the explicit extrapolation of the default step.
// The per-point relation becomes one linear system over the grid,
//
//   Op(sigma)_p = M_p sigma_p + dt [ sum_a u_a(p) D_a(sigma) - eps Lap(sigma) ]_p = R_p,
//   M_p = (eta + dt/Wi) I - dt L(kappa*_p),   L(k) s = k s + s k^T,
//   R_p = eta sigma0_p - H_p + dt G (kappa*_p + kappa*_p^T) g_alpha(t_{n+1}),
//
// with the stencils of the explicit form (D_a upwinded on the sign of u_a(p))
// acting on every stress component.  It is solved by BiCGStab (van der Vorst,
// 1992) preconditioned on the right by block Jacobi: the nc x nc block of each
// point, M_p plus the diagonal of the transport stencil.  Krylov vectors are
// FP64 in both storage modes.
//
// Kernels: rhs (history sum H over the modes, Q_j = b1 x + b2 y written over
// the oldest mode level, R, initial guess E = 2 sigma^n - sigma^{n-1}), apply
// (Op), precond (block solves), vector updates and dot products (per-block
// partial sums added on the host in a fixed order), push (sigma^{n+1} and the
// new mode level from Q_j).  One thread per point, grid-stride loops.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "tfs_device.cuh"
#include "tfs_internal.h"

namespace tfs {
namespace {

constexpr int kThreads = 256;

template <typename T, int DIM, bool COMP>
__global__ void __launch_bounds__(kThreads) imp_rhs_kernel(const ImpArgs<T> A, double* b, double* x0) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr bool F32 = sizeof(T) == 4;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) {
                const long long q = (long long)(i * DIM + j) * N + p;
                K[i][j] = 2.0 * (double)A.kap_n[q] - (double)A.kap_nm1[q];
            }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const double s0 = A.sigma0 ? (double)A.sigma0[qc] : 0.0;
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            const double ks = K[i][j] + K[j][i];
            double R;
            if (A.classic) {
                const double H = kB1 * (double)A.sig_n[qc] + kB2 * (double)A.sig_nm1[qc] + kB0 * s0;
                R = A.eta * s0 - H + A.dt * A.G * A.g * ks;
            } else if constexpr (F32) {
                // compensated sum as in the default step, then one rounding to double
                float hs = 0.0f, comp = 0.0f;
                for (int jj = 0; jj < A.m; ++jj) {
                    const long long q = ((long long)jj * NC + c) * N + p;
                    const float qj = __fmaf_rn(0.5f, (float)A.modes_nm1[q], -2.0f * (float)A.modes_n[q]);
                    A.modes_nm1[q] = (T)qj;
                    if (COMP) {
                        const float yv = __fmaf_rn(A.mc.eta_hi[jj], qj, __fmaf_rn(A.mc.eta_lo[jj], qj, -comp));
                        const float t = __fadd_rn(hs, yv);
                        comp = __fsub_rn(__fsub_rn(t, hs), yv);
                        hs = t;
                    } else {
                        hs = __fmaf_rn(A.mc.eta_hi[jj], qj, hs);
                    }
                }
                const double H = (double)hs - (double)comp;
                R = A.eta * s0 - H + A.dt * A.G * A.g * ks;
            } else {
                double H = 0.0;
                for (int jj = 0; jj < A.m; ++jj) {
                    const long long q = ((long long)jj * NC + c) * N + p;
                    const double qj = kB1 * (double)A.modes_n[q] + kB2 * (double)A.modes_nm1[q];
                    A.modes_nm1[q] = (T)qj;
                    H = fma(A.mcd.eta[jj], qj, H);
                }
                R = A.eta * s0 - H + A.dt * A.G * A.g * ks;
            }
            b[qc] = R;
            x0[qc] = 2.0 * (double)A.sig_n[qc] - (double)A.sig_nm1[qc];
        }
    }
}

template <typename T, int DIM>
__device__ __forceinline__ void point_block(const ImpArgs<T>& A, long long p, double M[Packed<DIM>::NC][Packed<DIM>::NC]) {
    double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const long long q = (long long)(i * DIM + j) * A.N + p;
            K[i][j] = 2.0 * (double)A.kap_n[q] - (double)A.kap_nm1[q];
        }
    assemble_M<DIM>(K, A.a, A.dt, M);
}

// first derivative along axis ax of field f at point p (taps -2..2), upwinded on the sign of v
template <int DIM>
__device__ __forceinline__ double deriv_at(const double* f, const GridIdx& g, int ax, int stencil, double v,
                                           double ih) {
    const double fm1 = f[g.at(ax, -1)], fp1 = f[g.at(ax, 1)];
    if (stencil == 1) return (fp1 - fm1) * (0.5 * ih);
    const double f0 = f[g.at(ax, 0)];
    if (v >= 0.0) return (f[g.at(ax, -2)] - 6.0 * fm1 + 3.0 * f0 + 2.0 * fp1) * (ih / 6.0);
    return (-2.0 * fm1 - 3.0 * f0 + 6.0 * fp1 - f[g.at(ax, 2)]) * (ih / 6.0);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_apply_kernel(const ImpArgs<T> A, const double* x, double* y) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        double M[NC][NC];
        point_block<T, DIM>(A, p, M);
        GridIdx g;
        g.n0 = A.n0;
        g.n1 = A.n1;
        g.n2 = A.n2;
        g.x = p % A.n0;
        g.y = (p / A.n0) % A.n1;
        g.z = p / ((long long)A.n0 * A.n1);
        double u[3] = {0, 0, 0};
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) u[ax] = (double)A.u[(long long)ax * N + p];
        double xp[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) xp[c] = x[(long long)c * N + p];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < NC; ++k) acc = fma(M[r][k], xp[k], acc);
            const double* f = x + (long long)r * N;
            double t = 0.0;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) {
                t += u[ax] * deriv_at<DIM>(f, g, ax, A.stencil, u[ax], A.inv_h[ax]);
                if (A.eps != 0.0)
                    t -= A.eps * (f[g.at(ax, -1)] - 2.0 * xp[r] + f[g.at(ax, 1)]) * (A.inv_h[ax] * A.inv_h[ax]);
            }
            y[(long long)r * N + p] = acc + A.dt * t;
        }
    }
}

// z = P^-1 r: the point block M_p plus the diagonal of the transport stencil
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_precond_kernel(const ImpArgs<T> A, const double* r, double* z) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        double M[NC][NC];
        point_block<T, DIM>(A, p, M);
        double diag = 0.0;
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) {
            const double ua = (double)A.u[(long long)ax * N + p];
            if (A.stencil == 0) diag += fabs(ua) * 0.5 * A.inv_h[ax];
            diag += 2.0 * A.eps * A.inv_h[ax] * A.inv_h[ax];
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) M[c][c] += A.dt * diag;
        double v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = r[(long long)c * N + p];
        if (!gauss_pp<NC>(M, v, 1e-300)) atomicOr(A.flags, 2u);
#pragma unroll
        for (int c = 0; c < NC; ++c) z[(long long)c * N + p] = v[c];
    }
}

// per-block partial sums of x.y (x.x when y == x), block reduce in shared memory
__global__ void __launch_bounds__(kThreads) imp_dot_kernel(const double* x, const double* y, long long n,
                                                           double* partials) {
    __shared__ double sh[kThreads];
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc = fma(x[i], y[i], acc);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// y = a x + b y + c z (any of the inputs may alias y)
__global__ void __launch_bounds__(kThreads) imp_axpbypcz_kernel(double a, const double* x, double b, double* y, double c,
                                                                const double* z, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double xv = x ? x[i] : 0.0, zv = z ? z[i] : 0.0;
        y[i] = a * xv + b * y[i] + c * zv;
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_push_kernel(const ImpArgs<T> A, const double* x) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr bool F32 = sizeof(T) == 4;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        bool finite = true;
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const T out = (T)x[qc];
            finite = finite && isfinite((double)out);
            A.sig_np1[qc] = out;
            if (A.sig_copy) A.sig_copy[qc] = out;
            const T s0 = A.sigma0 ? A.sigma0[qc] : (T)0;
            if (A.classic) continue;
            if constexpr (F32) {
                const float d = __fsub_rn((float)out, (float)s0);
                for (int j = 0; j < A.m; ++j) {
                    const long long q = ((long long)j * NC + c) * N + p;
                    A.modes_nm1[q] = __fmaf_rn(A.mc.rho[j], d, -A.mc.c[j] * (float)A.modes_nm1[q]);
                }
            } else {
                const double d = (double)out - (double)s0;
                for (int j = 0; j < A.m; ++j) {
                    const long long q = ((long long)j * NC + c) * N + p;
                    A.modes_nm1[q] = (T)fma(A.mcd.rho[j], d, -A.mcd.c[j] * (double)A.modes_nm1[q]);
                }
            }
        }
        if (!finite) atomicOr(A.flags, 1u);
    }
}

// ------------------------------------------------------------------ host side
struct Krylov {
    double *b, *x, *r, *rh, *p, *v, *s, *t, *ph, *sh;
};

template <typename T, int DIM, bool COMP>
cudaError_t run_implicit(const ImpArgs<T>& a, cudaStream_t st, int* iters, double* relres) {
    constexpr int NC = Packed<DIM>::NC;
    const long long n = (long long)NC * a.N;
    const long long bs = (long long)kImpBlocks;
    Krylov K;
    double* base = a.kry;
    double** slots[] = {&K.b, &K.x, &K.r, &K.rh, &K.p, &K.v, &K.s, &K.t, &K.ph, &K.sh};
    for (int i = 0; i < 10; ++i) *slots[i] = base + (size_t)i * (size_t)n;
    std::vector<double> host(kImpBlocks);
    cudaError_t e = cudaSuccess;
    auto check = [&]() { if (e == cudaSuccess) e = cudaGetLastError(); return e == cudaSuccess; };
    // dot product: partial sums on the device, added on the host in block order
    auto dot = [&](const double* x, const double* y, double* out) {
        if (e != cudaSuccess) return;
        imp_dot_kernel<<<(unsigned)bs, kThreads, 0, st>>>(x, y, n, a.partials);
        if (!check()) return;
        e = cudaMemcpyAsync(host.data(), a.partials, sizeof(double) * kImpBlocks, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        double acc = 0.0;
        for (int i = 0; i < kImpBlocks; ++i) acc += host[i];
        *out = acc;
    };
    auto lin = [&](double ca, const double* x, double cb, double* y, double cc, const double* z) {
        if (e != cudaSuccess) return;
        imp_axpbypcz_kernel<<<(unsigned)bs, kThreads, 0, st>>>(ca, x, cb, y, cc, z, n);
        check();
    };
    auto apply = [&](const double* x, double* y) {
        if (e != cudaSuccess) return;
        imp_apply_kernel<T, DIM><<<(unsigned)bs, kThreads, 0, st>>>(a, x, y);
        check();
    };
    auto precond = [&](const double* r, double* z) {
        if (e != cudaSuccess) return;
        imp_precond_kernel<T, DIM><<<(unsigned)bs, kThreads, 0, st>>>(a, r, z);
        check();
    };

    imp_rhs_kernel<T, DIM, COMP><<<(unsigned)bs, kThreads, 0, st>>>(a, K.b, K.x);
    check();
    double bnorm2 = 0.0;
    dot(K.b, K.b, &bnorm2);
    const double bnorm = std::sqrt(bnorm2);
    int it = 0;
    double res = 0.0;
    bool converged = false;
    if (e == cudaSuccess && bnorm == 0.0) {
        lin(0.0, nullptr, 0.0, K.x, 0.0, nullptr);   // R = 0: sigma^{n+1} = 0
        converged = true;
    } else if (e == cudaSuccess) {
        apply(K.x, K.r);
        lin(1.0, K.b, -1.0, K.r, 0.0, nullptr);      // r = b - Op(x0)
        lin(1.0, K.r, 0.0, K.rh, 0.0, nullptr);      // shadow residual
        lin(0.0, nullptr, 0.0, K.p, 0.0, nullptr);
        lin(0.0, nullptr, 0.0, K.v, 0.0, nullptr);
        double rr = 0.0;
        dot(K.r, K.r, &rr);
        res = std::sqrt(rr) / bnorm;
        converged = res <= a.tol;
        double rho = 1.0, alpha = 1.0, omega = 1.0;
        while (e == cudaSuccess && !converged && it < a.maxit) {
            ++it;
            double rho_new = 0.0;
            dot(K.rh, K.r, &rho_new);
            if (rho_new == 0.0 || omega == 0.0) break;   // breakdown
            const double beta = (rho_new / rho) * (alpha / omega);
            rho = rho_new;
            lin(-beta * omega, K.v, beta, K.p, 1.0, K.r);   // p = r + beta (p - omega v)
            precond(K.p, K.ph);
            apply(K.ph, K.v);
            double rhv = 0.0;
            dot(K.rh, K.v, &rhv);
            if (rhv == 0.0) break;
            alpha = rho / rhv;
            lin(1.0, K.r, 0.0, K.s, -alpha, K.v);          // s = r - alpha v
            double ss = 0.0;
            dot(K.s, K.s, &ss);
            if (std::sqrt(ss) / bnorm <= a.tol) {
                lin(alpha, K.ph, 1.0, K.x, 0.0, nullptr);   // x += alpha ph
                res = std::sqrt(ss) / bnorm;
                converged = true;
                break;
            }
            precond(K.s, K.sh);
            apply(K.sh, K.t);
            double ts = 0.0, tt = 0.0;
            dot(K.t, K.s, &ts);
            dot(K.t, K.t, &tt);
            omega = tt > 0.0 ? ts / tt : 0.0;
            lin(alpha, K.ph, 1.0, K.x, omega, K.sh);        // x += alpha ph + omega sh
            lin(1.0, K.s, 0.0, K.r, -omega, K.t);           // r = s - omega t
            dot(K.r, K.r, &rr);
            res = std::sqrt(rr) / bnorm;
            converged = res <= a.tol;
        }
    }
    if (e == cudaSuccess && !converged) {
        unsigned nc_flag = 16u;
        e = cudaMemcpyAsync(host.data(), a.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        unsigned f = 0u;
        memcpy(&f, host.data(), sizeof(unsigned));
        f |= nc_flag;
        if (e == cudaSuccess) e = cudaMemcpyAsync(a.flags, &f, sizeof(unsigned), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) {
        imp_push_kernel<T, DIM><<<(unsigned)bs, kThreads, 0, st>>>(a, K.x);
        check();
    }
    *iters = it;
    *relres = res;
    return e;
}

}  // namespace

cudaError_t run_implicit_f64(const ImpArgs<double>& a, cudaStream_t s, int* iters, double* relres) {
    return a.dim == 2 ? run_implicit<double, 2, false>(a, s, iters, relres)
                      : run_implicit<double, 3, false>(a, s, iters, relres);
}

cudaError_t run_implicit_f32(const ImpArgs<float>& a, cudaStream_t s, bool comp, int* iters, double* relres) {
    if (a.dim == 2)
        return comp ? run_implicit<float, 2, true>(a, s, iters, relres) : run_implicit<float, 2, false>(a, s, iters, relres);
    return comp ? run_implicit<float, 3, true>(a, s, iters, relres) : run_implicit<float, 3, false>(a, s, iters, relres);
}

}  // namespace tfs
