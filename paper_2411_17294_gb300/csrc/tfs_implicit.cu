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
// 1992) preconditioned on the right by block Jacobi (the nc x nc block of
// each point, M_p plus the diagonal of the transport stencil), inside a
// mixed-precision defect correction: FP64 residuals of the FP64 system, the
// BiCGStab iterations on a float copy of it for the corrections.
//
// Kernels: rhs (history sum H over the modes, Q_j = b1 x + b2 y written over
// the oldest mode level, R, initial guess E = 2 sigma^n - sigma^{n-1}), apply
// (Op), precond (block solves), vector updates and dot products (per-block
// partial sums added on the host in a fixed order), push (sigma^{n+1} and the
// new mode level from Q_j).  One thread per point, grid-stride loops.
#include <cuda_runtime.h>

#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "tfs_device.cuh"
#include "tfs_internal.h"
#include "tfs_adjoint_implicit.h"

namespace tfs {
namespace {

constexpr int kThreads = 256;
constexpr int kMB = 8;   // mode values a thread reads before it writes the first back

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
                // compensated sum as in the default step, then one rounding to double;
                // the modes are read kMB at a time, before the first of them is
                // written back (the sum keeps its order)
                float hs = 0.0f, comp = 0.0f;
                for (int j0 = 0; j0 < A.m; j0 += kMB) {
                    float vn1[kMB], vn[kMB];
#pragma unroll
                    for (int k = 0; k < kMB; ++k)
                        if (j0 + k < A.m) {
                            const long long q = mode_index(p, (j0 + k) * NC + c, A.m * NC);
                            vn1[k] = (float)A.modes_nm1[q];
                            vn[k] = (float)A.modes_n[q];
                        }
#pragma unroll
                    for (int k = 0; k < kMB; ++k) {
                        const int jj = j0 + k;
                        if (jj >= A.m) break;
                        const float qj = __fmaf_rn(0.5f, vn1[k], -2.0f * vn[k]);
                        A.modes_nm1[mode_index(p, jj * NC + c, A.m * NC)] = (T)qj;
                        if (COMP) {
                            const float yv = __fmaf_rn(A.mc.eta_hi[jj], qj, __fmaf_rn(A.mc.eta_lo[jj], qj, -comp));
                            const float t = __fadd_rn(hs, yv);
                            comp = __fsub_rn(__fsub_rn(t, hs), yv);
                            hs = t;
                        } else {
                            hs = __fmaf_rn(A.mc.eta_hi[jj], qj, hs);
                        }
                    }
                }
                const double H = (double)hs - (double)comp;
                R = A.eta * s0 - H + A.dt * A.G * A.g * ks;
            } else {
                double H = 0.0;
                for (int j0 = 0; j0 < A.m; j0 += kMB) {
                    double vn1[kMB], vn[kMB];
#pragma unroll
                    for (int k = 0; k < kMB; ++k)
                        if (j0 + k < A.m) {
                            const long long q = mode_index(p, (j0 + k) * NC + c, A.m * NC);
                            vn1[k] = (double)A.modes_nm1[q];
                            vn[k] = (double)A.modes_n[q];
                        }
#pragma unroll
                    for (int k = 0; k < kMB; ++k) {
                        const int jj = j0 + k;
                        if (jj >= A.m) break;
                        const double qj = kB1 * vn[k] + kB2 * vn1[k];
                        A.modes_nm1[mode_index(p, jj * NC + c, A.m * NC)] = (T)qj;
                        H = fma(A.mcd.eta[jj], qj, H);
                    }
                }
                R = A.eta * s0 - H + A.dt * A.G * A.g * ks;
            }
            b[qc] = R;
            x0[qc] = 2.0 * (double)A.sig_n[qc] - (double)A.sig_nm1[qc];
        }
    }
}

// Per step: the point blocks P_p = M_p + dt c0_p I, M_p = a I - dt L(kappa*_p),
// c0_p the centre coefficient of the transport stencil at p (sum over the axes),
// and their inverses (the block-Jacobi preconditioner), stored [nc*nc][N]
// (entry r*nc + k of point p at (r*nc + k) N + p); and the four off-centre tap
// coefficients of every axis times dt, Cf[(a*4 + t) N + p] for the taps -2, -1,
// +1, +2 (the stencils of deriv_at, upwinded on the sign of u_a(p), and eps Lap).
// The operator is then Op(x)_p = P_p x_p + sum_a sum_t Cf x_{p + tap}, the same
// for every Krylov iteration of the step.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_setup_kernel(const ImpArgs<T> A, double* Mb, double* Pinv,
                                                             double* Cf) {
    constexpr int NC = Packed<DIM>::NC;
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
        double M[NC][NC];
        assemble_M<DIM>(K, A.a, A.dt, M);
        double diag = 0.0;
        constexpr double kSixth = 1.0 / 6.0;
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) {
            const double ua = (double)A.u[(long long)ax * N + p];
            const double ih = A.inv_h[ax];
            const double e = A.eps * ih * ih;
            if (A.stencil == 0) diag += fabs(ua) * 0.5 * ih;
            diag += 2.0 * e;
            double c[4];   // taps -2, -1, +1, +2
            if (A.stencil == 1) {
                const double h2 = 0.5 * ua * ih;
                c[0] = 0.0; c[1] = -h2 - e; c[2] = h2 - e; c[3] = 0.0;
            } else if (ua >= 0.0) {
                const double s6 = ua * ih * kSixth;
                c[0] = s6; c[1] = -6.0 * s6 - e; c[2] = 2.0 * s6 - e; c[3] = 0.0;
            } else {
                const double s6 = ua * ih * kSixth;
                c[0] = 0.0; c[1] = -2.0 * s6 - e; c[2] = 6.0 * s6 - e; c[3] = -s6;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) Cf[(long long)(ax * 4 + t) * N + p] = A.dt * c[t];
        }
#pragma unroll
        for (int r = 0; r < NC; ++r) M[r][r] += A.dt * diag;
        // the inverse, column by column of the identity; in 2D one elimination
        // for all three (3D: the 6 x 6 blocks of both would not fit the registers)
        constexpr int NR = NC <= 3 ? NC : 1;
        bool ok = true;
#pragma unroll
        for (int k0 = 0; k0 < NC; k0 += NR) {
            double P[NC][NC], X[NC][NR];
#pragma unroll
            for (int r = 0; r < NC; ++r) {
#pragma unroll
                for (int c = 0; c < NC; ++c) P[r][c] = M[r][c];
#pragma unroll
                for (int k = 0; k < NR; ++k) X[r][k] = r == k0 + k ? 1.0 : 0.0;
            }
            ok = gauss_pp_multi<NC, NR>(P, X, 1e-300) && ok;
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int k = 0; k < NR; ++k) Pinv[(long long)(r * NC + k0 + k) * N + p] = X[r][k];
        }
        if (!ok) atomicOr(A.flags, 2u);
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int c = 0; c < NC; ++c) Mb[(long long)(r * NC + c) * N + p] = M[r][c];
    }
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

// Device scalars of the iteration.
enum : int { S_RHO = 0, S_RHO_NEW, S_ALPHA, S_OMEGA, S_BETA, S_RHV, S_TS, S_TT, S_RR, S_BNORM2, S_DONE, S_ITERS,
             S_BREAK, S_TOL2, S_COUNT };
constexpr int kPartialSets = 2;    // dot products reduced in one pass

__device__ __forceinline__ bool done(const double* sc) { return sc[S_DONE] != 0.0; }

constexpr int kWarps = kThreads / 32;

// sum over the 32 lanes of a warp in a fixed order (lane 0 holds it)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// sums of two values over the block (every thread calls), in thread 0; the
// per-warp sums pass through sh
__device__ __forceinline__ void block_sum2(double& a0, double& a1, double (*sh)[kWarps]) {
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a0;
        sh[1][threadIdx.x >> 5] = a1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a0 = a1 = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            a0 += sh[0][w];
            a1 += sh[1][w];
        }
    }
}

// block-level reduction of two values into partials[set * kImpBlocks + block]
__device__ __forceinline__ void block_partials(double a0, double a1, int nsets, double* partials) {
    __shared__ double sh[2][kWarps];
    block_sum2(a0, a1, sh);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = a0;
        if (nsets > 1) partials[kImpBlocks + blockIdx.x] = a1;
    }
}

// After block_partials: true in every thread of the block that finishes last
// (a ticket drawn after a fence that publishes the block's partial sums), which
// then resets the ticket for the next launch.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (last) *ticket = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// One block: add the partial sums of nparts blocks in a fixed order into scalar
// slots, then the scalar step of the iteration.
//   op 0: RR, RHO_NEW <- (r, r), (rh, r); convergence test; beta and rho of the next direction
//   op 1: RHV <- (rh, v); alpha
//   op 2: TS, TT <- (t, s), (t, t); omega
//   op 3: BNORM2 <- (b, b)
//   op 4: RR, RHO_NEW <- (r, r), (rh, r) at the start; beta and rho of the first direction
__device__ void scalar_step(const double* partials, int nparts, double* sc, int op) {
    __shared__ double sh[2][kWarps];
    static_assert(kImpBlocks <= 4 * kThreads, "at most four partial sums per thread");
    // thread 0 reads the scalars it needs together with the partial sums (no
    // other block writes them during the launch): one round trip, not two
    double s_done = 0.0, s_rho = 0.0, s_alpha = 0.0, s_omega = 0.0, s_lim = 0.0, s_iters = 0.0;
    if (threadIdx.x == 0 && op != 3) {
        s_done = sc[S_DONE];
        s_rho = sc[S_RHO];
        s_alpha = sc[S_ALPHA];
        s_omega = sc[S_OMEGA];
        s_lim = sc[S_TOL2] * sc[S_BNORM2];
        s_iters = sc[S_ITERS];
    }
    // the (at most) four partial sums of a thread are loaded together; written by
    // other blocks of this launch, they are read from L2
    double p0[4], p1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = threadIdx.x + k * kThreads;
        p0[k] = i < nparts ? __ldcg(partials + i) : 0.0;
        p1[k] = i < nparts ? __ldcg(partials + kImpBlocks + i) : 0.0;
    }
    double v0 = (p0[0] + p0[1]) + (p0[2] + p0[3]);
    double v1 = (p1[0] + p1[1]) + (p1[2] + p1[3]);
    block_sum2(v0, v1, sh);
    if (threadIdx.x != 0) return;
    if (op == 3) {
        sc[S_BNORM2] = v0;
        return;
    }
    // beta and rho of the next direction, once (r, r) = v0 and (rh, r) = v1 are
    // known and the iteration goes on
    auto next_direction = [&](bool done_now) {
        if (done_now) return;
        sc[S_BETA] = (v1 / s_rho) * (s_alpha / s_omega);
        sc[S_RHO] = v1;
    };
    if (op == 4) {
        sc[S_RR] = v0;
        sc[S_RHO_NEW] = v1;
        const bool conv = v0 <= s_lim;
        if (conv) sc[S_DONE] = 1.0;
        next_direction(s_done != 0.0 || conv);
        return;
    }
    if (s_done != 0.0) return;
    if (op == 1) {
        sc[S_RHV] = v0;
        if (v0 == 0.0) {
            sc[S_BREAK] = 1.0;
            sc[S_DONE] = 1.0;
        } else {
            sc[S_ALPHA] = s_rho / v0;
        }
    } else if (op == 2) {
        sc[S_TS] = v0;
        sc[S_TT] = v1;
        sc[S_OMEGA] = v1 > 0.0 ? v0 / v1 : 0.0;
    } else {
        sc[S_RR] = v0;
        sc[S_RHO_NEW] = v1;
        sc[S_ITERS] = s_iters + 1.0;
        bool stop = false;
        if (v0 <= s_lim) {
            sc[S_DONE] = 1.0;
            stop = true;
        } else if (v1 == 0.0 || s_omega == 0.0) {
            sc[S_BREAK] = 1.0;
            sc[S_DONE] = 1.0;
            stop = true;
        }
        next_direction(stop);
    }
}

// Grid of the operator kernels (all they take of a step's arguments)
struct ImpGrid {
    long long N;
    int n0, n1, n2;
    unsigned* flags;   // TFS_FLAG_TIMEOUT of a copy wait that gave up
};

// Index of coefficient k of point p: FP64 coefficients (the step's system) are
// [k][N]; the float copies of the inner solve are tile-major (mode_index over
// 32-point tiles, K coefficients per point), so that the K loads of a point share
// one base address and differ by constants.
template <typename V, int K>
__device__ __forceinline__ long long coef_at(long long p, int k, long long N) {
    if constexpr (sizeof(V) == 4) return mode_index(p, k, K);
    else return (long long)k * N + p;
}

// y = Op(x) = P_p x_p + sum_a sum_t Cf x_{p + tap} with the per-step blocks and
// coefficients of imp_setup_kernel (float: blocks and taps of a point in one
// tile-major array, Cf = Mb + nc^2 tile rows); partial sums of (w0, y) and (w1, y) when
// w0 / w1 are given (w1 may be y itself: the (t, t) product), and with op >= 0
// the scalar step op of scalar_step in the block that finishes last.  The
// periodic neighbour offsets are 32-bit (an implicit-transport workspace for
// 2^31 points would not fit any device).
template <int DIM, typename V>
__global__ void __launch_bounds__(kThreads) imp_apply_kernel(const ImpGrid A, const V* __restrict__ Mb,
                                                             const V* __restrict__ Cf, const V* __restrict__ x, V* y,
                                                             const V* w0, const V* w1, double* partials, double* sc,
                                                             int op, unsigned* ticket) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr int KA = NC * NC + 4 * DIM;   // coefficients per point (float layout)
    if (done(sc)) return;
    const long long N = A.N;
    const int n0 = A.n0, n1 = A.n1, n2 = A.n2;
    const bool w1y = w1 == y;   // (y, y): from the register, not read back
    V a0 = (V)0, a1 = (V)0;   // per-thread dot products (a few points each), then double per block
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const unsigned pp = (unsigned)p;
        const unsigned q1 = pp / (unsigned)n0;
        const int c[3] = {(int)(pp - q1 * (unsigned)n0), (int)(q1 % (unsigned)n1), (int)(q1 / (unsigned)n1)};
        const int len[3] = {n0, n1, n2};
        const int str[3] = {1, n0, n0 * n1};
        int off[3][4];
        V cf[3][4];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int k = t < 2 ? t - 2 : t - 1;
                int v = c[a] + k;
                if (v < 0) v += len[a];
                if (v < 0) v += len[a];
                if (v >= len[a]) v -= len[a];
                if (v >= len[a]) v -= len[a];
                off[a][t] = (v - c[a]) * str[a];
                cf[a][t] = Cf[coef_at<V, KA>(p, a * 4 + t, N)];
            }
        }
        V xp[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) xp[k] = x[(long long)k * N + p];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            V acc = (V)0;
#pragma unroll
            for (int k = 0; k < NC; ++k) acc = fma(Mb[coef_at<V, KA>(p, r * NC + k, N)], xp[k], acc);
            const V* f = x + (long long)r * N + p;
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (cf[a][t] != (V)0) acc = fma(cf[a][t], f[off[a][t]], acc);
            const long long q = (long long)r * N + p;
            y[q] = acc;
            if (w0) a0 = fma(w0[q], acc, a0);
            if (w1) a1 = fma(w1y ? acc : w1[q], acc, a1);
        }
    }
    if (w0) {
        block_partials((double)a0, (double)a1, w1 ? 2 : 1, partials);
        if (op >= 0 && last_block(ticket)) scalar_step(partials, gridDim.x, sc, op);
    }
}

// The same operator on grids with n0 % 32 == 0 and n1 % 8 == 0, tiled: a unit
// is a 32 x 8 (x, y) tile and a chunk of kZc z planes (one plane in 2D); the
// block stages the tile of x with a 2-cell halo in x and y in shared memory
// once per plane (every x value loaded once per tile instead of at nine taps),
// keeps x at z-2 .. z+2 of its own column in registers (3D), and applies the
// taps without branches (a zero coefficient adds nothing).  The point's
// coefficients (and w0) are loaded before the staging barrier, so that their
// loads and those of the tile are in flight together.  Units are handed out
// grid-stride over a fixed grid, so that the partial sums are those of fixed
// blocks, reduced in a fixed order as everywhere else.
constexpr int kAX = 32, kAY = 8, kAH = 2, kAZc = 8;
constexpr int kASX = kAX + 2 * kAH, kASY = kAY + 2 * kAH;

template <int DIM, typename V>
__global__ void __launch_bounds__(kThreads, DIM == 2 && sizeof(V) == 4 ? 6 : 1)
    imp_apply_tiled_kernel(const ImpGrid A, const V* __restrict__ Mb, const V* __restrict__ Cf,
                                                                    const V* __restrict__ x, V* y, const V* w0,
                                                                    const V* w1, double* partials, double* sc,
                                                                    int op, unsigned* ticket) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr int KA = NC * NC + 4 * DIM;   // coefficients per point (float layout)
    constexpr bool kPreMb = NC <= 3;   // the 2D blocks in registers across the barrier (3D: too many)
    __shared__ V Xs[NC][kASY][kASX];
    if (done(sc)) return;
    const bool w1y = w1 == y;
    const long long N = A.N;
    const int n0 = A.n0, n1 = A.n1, n2 = DIM == 3 ? A.n2 : 1;
    const long long plane = (long long)n0 * n1;
    static_assert(kAX * kAY == kThreads, "one thread per tile point (block_partials reduces kThreads values)");
    const int tid = threadIdx.x, tx = tid % kAX, ty = tid / kAX;
    const int tiles_x = n0 / kAX, tiles = tiles_x * (n1 / kAY);
    const int zchunks = (n2 + kAZc - 1) / kAZc;
    const int units = tiles * zchunks;   // 32-bit: a unit holds at least 256 points
    auto wrap = [](int v, int n) { v %= n; return v < 0 ? v + n : v; };
    auto wrap1 = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };   // -n <= v < 2n
    // the halo cell this thread stages: the ring of width kAH around the tile
    // (kAH rows above, kAH rows below, kAH columns left and right), one cell per
    // thread of the first kHalo
    constexpr int kHalo = kASX * kASY - kAX * kAY;
    static_assert(kHalo <= kThreads, "one halo cell per thread");
    const bool halo = tid < kHalo;
    int hx, hy;
    {
        int t = tid;
        if (t < kAH * kASX) {
            hy = t / kASX; hx = t % kASX;
        } else if ((t -= kAH * kASX) < kAH * kASX) {
            hy = kAH + kAY + t / kASX; hx = t % kASX;
        } else if ((t -= kAH * kASX) < kAY * kAH) {
            hy = kAH + t / kAH; hx = t % kAH;
        } else {
            t -= kAY * kAH;
            hy = kAH + t / kAH; hx = kAH + kAX + t % kAH;
        }
    }
    V a0 = (V)0, a1 = (V)0;
    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int txy = zchunks == 1 ? unit : unit % tiles;
        const int zc = zchunks == 1 ? 0 : unit / tiles;
        const int x0 = (txy % tiles_x) * kAX, y0 = (txy / tiles_x) * kAY;
        const int gx = x0 + tx, gy = y0 + ty;
        const long long qxy = gx + (long long)n0 * gy;
        const int zb = zc * kAZc, ze = min(zb + kAZc, n2);
        V qz[NC][5];   // x of this column at z-2 .. z+2 (3D)
        if (DIM == 3) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long o = plane * wrap(zb - 2 + k, n2) + qxy;
#pragma unroll
                for (int c = 0; c < NC; ++c) qz[c][k] = x[(long long)c * N + o];
            }
        }
        for (int z = zb; z < ze; ++z) {
            const long long zo = plane * z;
            const long long p = zo + qxy;
            V cf[DIM][4], mb[kPreMb ? NC : 1][kPreMb ? NC : 1], wv[NC];
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
                for (int t = 0; t < 4; ++t) cf[a][t] = Cf[coef_at<V, KA>(p, a * 4 + t, N)];
            if constexpr (kPreMb) {
#pragma unroll
                for (int r = 0; r < NC; ++r)
#pragma unroll
                    for (int k = 0; k < NC; ++k) mb[r][k] = Mb[coef_at<V, KA>(p, r * NC + k, N)];
            }
#pragma unroll
            for (int r = 0; r < NC; ++r) wv[r] = w0 ? w0[(long long)r * N + p] : (V)0;
            V xin[NC], xh[NC];   // this point's x (2D) and the halo cell's, loaded before the barrier
            if (DIM == 3) {
                const long long o = plane * wrap(z + 2, n2) + qxy;
#pragma unroll
                for (int c = 0; c < NC; ++c) qz[c][4] = x[(long long)c * N + o];
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) xin[c] = x[(long long)c * N + p];
            }
            if (halo) {
                const long long o = zo + wrap1(x0 + hx - kAH, n0) + (long long)n0 * wrap1(y0 + hy - kAH, n1);
#pragma unroll
                for (int c = 0; c < NC; ++c) xh[c] = x[(long long)c * N + o];
            }
            __syncthreads();   // the previous plane's reads of Xs are done
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                Xs[c][ty + kAH][tx + kAH] = DIM == 3 ? qz[c][2] : xin[c];
                if (halo) Xs[c][hy][hx] = xh[c];
            }
            __syncthreads();
            V xp[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) xp[k] = Xs[k][ty + kAH][tx + kAH];
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                V acc = (V)0;
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    V m;
                    if constexpr (kPreMb) m = mb[r][k];
                    else m = Mb[coef_at<V, KA>(p, r * NC + k, N)];
                    acc = fma(m, xp[k], acc);
                }
                const int sy = ty + kAH, sx = tx + kAH;
                // taps -2, -1, +1, +2 along x, y (and z from the registers)
                acc = fma(cf[0][0], Xs[r][sy][sx - 2], acc);
                acc = fma(cf[0][1], Xs[r][sy][sx - 1], acc);
                acc = fma(cf[0][2], Xs[r][sy][sx + 1], acc);
                acc = fma(cf[0][3], Xs[r][sy][sx + 2], acc);
                acc = fma(cf[1][0], Xs[r][sy - 2][sx], acc);
                acc = fma(cf[1][1], Xs[r][sy - 1][sx], acc);
                acc = fma(cf[1][2], Xs[r][sy + 1][sx], acc);
                acc = fma(cf[1][3], Xs[r][sy + 2][sx], acc);
                if (DIM == 3) {
                    acc = fma(cf[DIM - 1][0], qz[r][0], acc);
                    acc = fma(cf[DIM - 1][1], qz[r][1], acc);
                    acc = fma(cf[DIM - 1][2], qz[r][3], acc);
                    acc = fma(cf[DIM - 1][3], qz[r][4], acc);
                }
                const long long q = (long long)r * N + p;
                y[q] = acc;
                if (w0) a0 = fma(wv[r], acc, a0);
                if (w1) a1 = fma(w1y ? acc : w1[q], acc, a1);
            }
            if (DIM == 3) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int k = 0; k < 4; ++k) qz[c][k] = qz[c][k + 1];
            }
        }
    }
    if (w0) {
        block_partials((double)a0, (double)a1, w1 ? 2 : 1, partials);
        if (op >= 0 && last_block(ticket)) scalar_step(partials, gridDim.x, sc, op);
    }
}

constexpr int kPX = kAX + 8;   // staged x row: x0 - 4 .. x0 + 35
constexpr int kPipeFull = 9 + 8;   // 2D: nc^2 block entries and 4 taps x 2 axes per point
constexpr int kPipeCompact = 6;    // 2D: the extrapolated velocity gradient (4) and the velocity (2)
template <int KC>
struct PipeStage {
    float X[3][kASY][kPX];
    float C[kAY][KC][kAX];
    float W[3][kAY][kAX];
};
template <int KC>
constexpr size_t pipe_smem() { return 2 * sizeof(PipeStage<KC>); }

// Scalars of the compact float operator: the step's a and dt, and per axis
// eps/h^2, 1/(6h) and 1/(2h), with the stencil (imp_setup_kernel's formulas).
struct CompactConsts {
    float dt, a;
    float e[2], ih6[2], ih2[2];
    int stencil;
};

// The 2D point block M and taps cf[axis][-2, -1, +1, +2] of the compact float
// operator from the point's values kc (kappa_00, kappa_01, kappa_10, kappa_11 of
// the extrapolated gradient, u_0, u_1): imp_setup_kernel's formulas in float.
__device__ __forceinline__ void compact_operator(const float kc[kPipeCompact], const CompactConsts& Q, float M[3][3],
                                                 float cf[2][4]) {
    const float K[3][3] = {{kc[0], kc[1], 0.f}, {kc[2], kc[3], 0.f}, {0.f, 0.f, 0.f}};
    float diag = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float ua = kc[4 + a], e = Q.e[a];
        if (Q.stencil == 0) diag += fabsf(ua) * Q.ih2[a];
        diag += 2.f * e;
        float c[4];
        if (Q.stencil == 1) {
            const float h2 = ua * Q.ih2[a];
            c[0] = 0.f; c[1] = -h2 - e; c[2] = h2 - e; c[3] = 0.f;
        } else if (ua >= 0.f) {
            const float s6 = ua * Q.ih6[a];
            c[0] = s6; c[1] = -6.f * s6 - e; c[2] = 2.f * s6 - e; c[3] = 0.f;
        } else {
            const float s6 = ua * Q.ih6[a];
            c[0] = 0.f; c[1] = -2.f * s6 - e; c[2] = 6.f * s6 - e; c[3] = -s6;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) cf[a][t] = Q.dt * c[t];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float l = uc_entry<2>(K, r, k);
            M[r][k] = r == k ? fmaf(-Q.dt, l, Q.a) + Q.dt * diag : -Q.dt * l;
        }
}

// The compact float operator on 2D grids with n0 % 32 == 0 and n1 % 8 == 0,
// without staging: a block applies 32 x 8 tiles (a warp per row segment),
// grid-stride, every thread loading its point's values, x at the point and at
// its eight taps (the neighbours' rows are those of the block's other warps or
// the tile's margin: L1 serves most) and w0, with no barrier between tiles, so
// that the loads of every resident warp stay in flight together.  (Staging the
// tile in shared memory by bulk and cp.async copies, as imp_apply_pipe2d_kernel
// does, measured slower for these 6 values per point: 23.3 against 22.3 us at
// 1024^2.)
__global__ void __launch_bounds__(kThreads) imp_apply_l1_kernel(const ImpGrid A, const CompactConsts Q,
                                                                const float* __restrict__ Cc,
                                                                const float* __restrict__ x, float* y,
                                                                const float* w0, const float* w1, double* partials,
                                                                double* sc, int op, unsigned* ticket) {
    constexpr int NC = 3;
    if (done(sc)) return;
    const bool w1y = w1 == y;
    const long long N = A.N;
    const int n0 = A.n0, n1 = A.n1;
    const int tid = threadIdx.x, tx = tid % kAX, ty = tid / kAX;
    const int tiles_x = n0 / kAX, units = tiles_x * (n1 / kAY);
    auto wrap1 = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };   // -n <= v < 2n
    float a0 = 0.f, a1 = 0.f;
    for (int unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int gx = (unit % tiles_x) * kAX + tx, gy = (unit / tiles_x) * kAY + ty;
        const long long p = (long long)gy * n0 + gx;
        float kc[kPipeCompact];
#pragma unroll
        for (int k = 0; k < kPipeCompact; ++k) kc[k] = Cc[mode_index(p, k, kPipeCompact)];
        // offsets of the taps -2, -1, +1, +2 along x, then y
        const long long row = (long long)gy * n0;
        long long off[8];
        off[0] = row + wrap1(gx - 2, n0); off[1] = row + wrap1(gx - 1, n0);
        off[2] = row + wrap1(gx + 1, n0); off[3] = row + wrap1(gx + 2, n0);
        off[4] = (long long)wrap1(gy - 2, n1) * n0 + gx; off[5] = (long long)wrap1(gy - 1, n1) * n0 + gx;
        off[6] = (long long)wrap1(gy + 1, n1) * n0 + gx; off[7] = (long long)wrap1(gy + 2, n1) * n0 + gx;
        float xp[NC], xt[NC][8], wv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float* xc = x + (long long)c * N;
            xp[c] = xc[p];
#pragma unroll
            for (int t = 0; t < 8; ++t) xt[c][t] = xc[off[t]];
            wv[c] = w0 ? w0[(long long)c * N + p] : 0.f;
        }
        float M[NC][NC], cf[2][4];
        compact_operator(kc, Q, M, cf);
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < NC; ++k) acc = fmaf(M[r][k], xp[k], acc);
#pragma unroll
            for (int t = 0; t < 8; ++t) acc = fmaf(cf[t / 4][t % 4], xt[r][t], acc);
            const long long q = (long long)r * N + p;
            y[q] = acc;
            if (w0) a0 = fmaf(wv[r], acc, a0);
            if (w1) a1 = fmaf(w1y ? acc : w1[q], acc, a1);
        }
    }
    if (w0) {
        block_partials((double)a0, (double)a1, w1 ? 2 : 1, partials);
        if (op >= 0 && last_block(ticket)) scalar_step(partials, gridDim.x, sc, op);
    }
}

// The float operator on 2D grids with n0 % 32 == 0 and n1 % 8 == 0 (16-byte
// aligned vectors), software-pipelined: a unit is one 32 x 8 tile, staged into
// one of two shared-memory stages while the previous unit is applied from the
// other.  The tile's coefficient rows (tile-major: 8 contiguous rows of KC
// values x 32 points: the rounded blocks and taps of imp_setup_kernel) arrive by
// bulk copies (cp.async.bulk, one per row from lanes of warp 0, completing on
// the stage's mbarrier); its x rows with a margin of 4 cells in x and 2 in y
// (whole 16-byte chunks, wrapped periodically) and its w0 rows by 16-byte
// cp.async copies of every thread.  Every entry of y is formed in the order of
// imp_apply_tiled_kernel (the two give the same y).  It serves the float
// operators that are not compact (the transposed ones of adjoint solves).
// A wait that gives up latches TFS_FLAG_TIMEOUT, lets the copies in flight land
// (bounded) and ends the block's units; the block still adds its partial sums,
// so the last-block count stays whole.
template <int KC>
__global__ void __launch_bounds__(kThreads) imp_apply_pipe2d_kernel(const ImpGrid A, const float* __restrict__ Af,
                                                                    const float* __restrict__ x, float* y,
                                                                    const float* w0, const float* w1,
                                                                    double* partials, double* sc, int op,
                                                                    unsigned* ticket) {
    constexpr int NC = 3;
    using Stage = PipeStage<KC>;
    extern __shared__ __align__(128) unsigned char pipe_smem_buf[];
    __shared__ __align__(8) uint64_t bars[2];
    Stage* stage = reinterpret_cast<Stage*>(pipe_smem_buf);
    if (done(sc)) return;
    const bool w1y = w1 == y;
    const long long N = A.N;
    const int n0 = A.n0, n1 = A.n1;
    const int tid = threadIdx.x, tx = tid % kAX, ty = tid / kAX;
    const int tiles_x = n0 / kAX, units = tiles_x * (n1 / kAY);
    auto wrap1 = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };   // -n <= v < 2n
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // stage unit `unit` into stage sidx (its earlier reads are done: a block barrier precedes)
    auto issue = [&](int unit, int sidx) {
        Stage& S = stage[sidx];
        const int x0 = (unit % tiles_x) * kAX, y0 = (unit / tiles_x) * kAY;
        if (tid < 32) {
            // coefficients: the tile's 8 row segments, KC x 32 floats each, contiguous
            fence_proxy_async_smem();
            if (tid == 0) mbar_arrive_expect_tx(&bars[sidx], (unsigned)sizeof(S.C));
            __syncwarp();
            if (tid < kAY) {
                const long long p0 = (long long)(y0 + tid) * n0 + x0;
                bulk_load(&S.C[tid][0][0], Af + (p0 >> 5) * (KC * kAX), KC * kAX * sizeof(float), &bars[sidx]);
            }
        }
        // x: nc x 12 rows x 10 chunks (chunk 0: x0-4 .. x0-1, chunk 9: x0+32 .. x0+35, wrapped)
        constexpr int kXc = kPX / 4, kXrow = kASY * kXc;
        for (int i = tid; i < NC * kXrow; i += kThreads) {
            const int c = i / kXrow, rem = i - c * kXrow, row = rem / kXc, ch = rem - row * kXc;
            const int gy = wrap1(y0 + row - kAH, n1);
            const int gx = ch == 0 ? wrap1(x0 - 4, n0) : (ch == kXc - 1 ? wrap1(x0 + kAX, n0) : x0 + 4 * (ch - 1));
            cp_async16(&S.X[c][row][4 * ch], x + (long long)c * N + (long long)gy * n0 + gx, 16);
        }
        if (w0) {
            constexpr int kWc = kAX / 4, kWrow = kAY * kWc;
            for (int i = tid; i < NC * kWrow; i += kThreads) {
                const int c = i / kWrow, rem = i - c * kWrow, row = rem / kWc, ch = rem - row * kWc;
                cp_async16(&S.W[c][row][4 * ch], w0 + (long long)c * N + (long long)(y0 + row) * n0 + x0 + 4 * ch, 16);
            }
        }
        cp_async_commit();
    };
    float a0 = 0.f, a1 = 0.f;
    int unit = blockIdx.x;
    if (unit < units) issue(unit, 0);
    for (int it = 0; unit < units; ++it, unit += gridDim.x) {
        const int sidx = it & 1;
        const int next = unit + gridDim.x;
        if (next < units) {
            issue(next, sidx ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        const unsigned parity = (unsigned)(it >> 1) & 1u;
        const bool ok = mbar_wait(&bars[sidx], parity);
        if (__syncthreads_or(!ok)) {   // (also: this unit's stage is complete for every thread)
            if (tid == 0) atomicOr(A.flags, 8u);
            mbar_wait(&bars[sidx], parity);
            if (next < units) mbar_wait(&bars[sidx ^ 1], (unsigned)((it + 1) >> 1) & 1u);
            cp_async_wait<0>();
            break;
        }
        const Stage& S = stage[sidx];
        const int x0 = (unit % tiles_x) * kAX, y0 = (unit / tiles_x) * kAY;
        const long long p = (long long)(y0 + ty) * n0 + x0 + tx;
        const int sy = ty + kAH, sx = tx + 4;
        // the point's block M and taps cf[axis][-2, -1, +1, +2]
        static_assert(KC == kPipeFull, "nc^2 block entries and 8 taps per point");
        float M[NC][NC], cf[2][4];
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int k = 0; k < NC; ++k) M[r][k] = S.C[ty][r * NC + k][tx];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int t = 0; t < 4; ++t) cf[a][t] = S.C[ty][NC * NC + 4 * a + t][tx];
        float xp[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) xp[k] = S.X[k][sy][sx];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < NC; ++k) acc = fmaf(M[r][k], xp[k], acc);
            acc = fmaf(cf[0][0], S.X[r][sy][sx - 2], acc);
            acc = fmaf(cf[0][1], S.X[r][sy][sx - 1], acc);
            acc = fmaf(cf[0][2], S.X[r][sy][sx + 1], acc);
            acc = fmaf(cf[0][3], S.X[r][sy][sx + 2], acc);
            acc = fmaf(cf[1][0], S.X[r][sy - 2][sx], acc);
            acc = fmaf(cf[1][1], S.X[r][sy - 1][sx], acc);
            acc = fmaf(cf[1][2], S.X[r][sy + 1][sx], acc);
            acc = fmaf(cf[1][3], S.X[r][sy + 2][sx], acc);
            const long long q = (long long)r * N + p;
            y[q] = acc;
            if (w0) a0 = fmaf(S.W[r][ty][tx], acc, a0);
            if (w1) a1 = fmaf(w1y ? acc : w1[q], acc, a1);
        }
        __syncthreads();   // every read of this stage is done before it is refilled
    }
    if (w0) {
        block_partials((double)a0, (double)a1, w1 ? 2 : 1, partials);
        if (op >= 0 && last_block(ticket)) scalar_step(partials, gridDim.x, sc, op);
    }
}

// Blocks of a grid-stride kernel resident at once on this device (one wave), at
// most kImpBlocks: a partial second wave would stream its share of the vectors
// with a fraction of the SMs.  The count depends only on the device and the
// kernel, so the partial sums stay those of fixed blocks.
template <typename Kern>
unsigned resident_blocks(Kern kernel, size_t dyn = 0) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kThreads, dyn) != cudaSuccess) {
        (void)cudaGetLastError();
        return (unsigned)kImpBlocks;
    }
    const long long g = (long long)sms * per;
    return (unsigned)(g < 1 ? 1 : (g > kImpBlocks ? kImpBlocks : g));
}

// Op x -> y (with the partial dot products; with op >= 0 the scalar step op in
// the last block, ticket its counter): the tiled kernel where the grid tiles,
// the per-point one elsewhere.  Both compute every entry in the same order, so
// the result does not depend on which one runs.
template <int DIM, typename V>
unsigned apply_blocks(bool tiled) {
    static const unsigned gt = resident_blocks(imp_apply_tiled_kernel<DIM, V>);
    static const unsigned gp = resident_blocks(imp_apply_kernel<DIM, V>);
    return tiled ? gt : gp;
}

// blocks of the pipelined 2D kernel (its dynamic shared-memory limit raised
// once, before the occupancy query; 0 if that fails)
template <int KC>
unsigned pipe_blocks() {
    static const unsigned g = []() {
        if (cudaFuncSetAttribute(imp_apply_pipe2d_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pipe_smem<KC>()) != cudaSuccess) {
            (void)cudaGetLastError();
            return 0u;
        }
        return resident_blocks(imp_apply_pipe2d_kernel<KC>, pipe_smem<KC>());
    }();
    return g;
}

inline unsigned l1_blocks() {
    static const unsigned g = resident_blocks(imp_apply_l1_kernel);
    return g;
}

// whether the pipelined kernel serves this 2D float operator (whole tiles,
// 16-byte aligned vectors)
template <typename T>
bool pipe_fits(const ImpArgs<T>& a, const void* x, const void* w0, const void* coef) {
    auto al16 = [](const void* q) { return q == nullptr || reinterpret_cast<uintptr_t>(q) % 16 == 0; };
    return a.n0 % kAX == 0 && a.n1 % kAY == 0 && al16(x) && al16(w0) && al16(coef);
}

// cc: the compact float operator (Mb then holds its per-point values), which
// only imp_apply_l1_kernel applies
template <typename T, int DIM, typename V>
void launch_apply(const ImpArgs<T>& a, const V* Mb, const V* Cf, const V* x, V* y, const V* w0, const V* w1,
                  double* partials, double* sc, int op, unsigned* ticket, const CompactConsts* cc, cudaStream_t st) {
    const ImpGrid G{a.N, a.n0, a.n1, a.n2, a.flags};
    const bool tiled = a.n0 % kAX == 0 && a.n1 % kAY == 0;
    if constexpr (DIM == 2 && std::is_same<V, float>::value) {
        if (cc) {
            imp_apply_l1_kernel<<<l1_blocks(), kThreads, 0, st>>>(G, *cc, Mb, x, y, w0, w1, partials, sc, op, ticket);
            return;
        }
        if (pipe_fits(a, x, w0, Mb) && Cf == Mb + 32 * 9 && pipe_blocks<kPipeFull>() > 0) {
            imp_apply_pipe2d_kernel<kPipeFull><<<pipe_blocks<kPipeFull>(), kThreads, pipe_smem<kPipeFull>(), st>>>(
                G, Mb, x, y, w0, w1, partials, sc, op, ticket);
            return;
        }
    }
    const unsigned g = apply_blocks<DIM, V>(tiled);
    if (tiled)
        imp_apply_tiled_kernel<DIM, V><<<g, kThreads, 0, st>>>(G, Mb, Cf, x, y, w0, w1, partials, sc, op, ticket);
    else
        imp_apply_kernel<DIM, V><<<g, kThreads, 0, st>>>(G, Mb, Cf, x, y, w0, w1, partials, sc, op, ticket);
}

// The combination and the block-Jacobi step of imp_comb_precond_kernel with the
// compact float operator of a 2D forward solve: the point block M (with the
// centre taps) is formed from the point's 6 values as imp_apply_l1_kernel forms
// it, and M z = w is solved by cofactors, instead of reading 9 stored inverse
// entries (the preconditioner is then M^-1 of the float operator itself).
__global__ void __launch_bounds__(kThreads) imp_comb_compact_kernel(long long N, const float* __restrict__ Cc,
                                                                    const CompactConsts Q, int mode,
                                                                    float* __restrict__ p,
                                                                    const float* __restrict__ r,
                                                                    const float* __restrict__ v,
                                                                    float* __restrict__ z, const double* sc) {
    if (done(sc)) return;
    // mode 0: p = r + beta (p - omega v);  mode 1: p (as s) = r - alpha v
    const float beta = (float)sc[S_BETA], omega = (float)sc[S_OMEGA], alpha = (float)sc[S_ALPHA];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        float kc[kPipeCompact], w[3];
#pragma unroll
        for (int k = 0; k < kPipeCompact; ++k) kc[k] = Cc[mode_index(i, k, kPipeCompact)];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long q = (long long)c * N + i;
            const float nv = mode == 0 ? fmaf(beta, p[q] - omega * v[q], r[q]) : fmaf(-alpha, v[q], r[q]);
            p[q] = nv;
            w[c] = nv;
        }
        float M[3][3], cf[2][4];
        compact_operator(kc, Q, M, cf);
        // cofactors C[i][j] of M; z = C^T w / det
        const float c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1], c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2],
                    c02 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
        const float c10 = M[0][2] * M[2][1] - M[0][1] * M[2][2], c11 = M[0][0] * M[2][2] - M[0][2] * M[2][0],
                    c12 = M[0][1] * M[2][0] - M[0][0] * M[2][1];
        const float c20 = M[0][1] * M[1][2] - M[0][2] * M[1][1], c21 = M[0][2] * M[1][0] - M[0][0] * M[1][2],
                    c22 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
        const float inv = 1.f / (M[0][0] * c00 + M[0][1] * c01 + M[0][2] * c02);
        z[i] = (c00 * w[0] + c10 * w[1] + c20 * w[2]) * inv;
        z[N + i] = (c01 * w[0] + c11 * w[1] + c21 * w[2]) * inv;
        z[2 * N + i] = (c02 * w[0] + c12 * w[1] + c22 * w[2]) * inv;
    }
}

// z = P^-1 v with v = a x + b y (+ c w): forms the combination, stores it in
// `comb` (when given) and its preconditioned image in z
// (every call passes distinct p, r, v, z)
template <int NC, typename V>
__global__ void __launch_bounds__(kThreads) imp_comb_precond_kernel(long long N, const V* __restrict__ Pinv, int mode,
                                                                    V* __restrict__ p, const V* __restrict__ r,
                                                                    const V* __restrict__ v, V* __restrict__ z,
                                                                    const double* sc) {
    if (done(sc)) return;
    // mode 0: p = r + beta (p - omega v);  mode 1: p (as s) = r - alpha v
    const V beta = (V)sc[S_BETA], omega = (V)sc[S_OMEGA], alpha = (V)sc[S_ALPHA];
#pragma unroll 2
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        V w[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long q = (long long)c * N + i;
            const V nv = mode == 0 ? fma(beta, p[q] - omega * v[q], r[q]) : fma(-alpha, v[q], r[q]);
            p[q] = nv;
            w[c] = nv;
        }
#pragma unroll
        for (int rr = 0; rr < NC; ++rr) {
            V acc = (V)0;
#pragma unroll
            for (int k = 0; k < NC; ++k) acc = fma(Pinv[coef_at<V, NC * NC>(i, rr * NC + k, N)], w[k], acc);
            z[(long long)rr * N + i] = acc;
        }
    }
}

// x += alpha ph + omega sh;  r = s - omega t;  partial sums of (r, r) and (rh, r),
// then scalar step 0 in the block that finishes last
// (every call passes seven distinct vectors)
template <typename V>
__global__ void __launch_bounds__(kThreads) imp_xr_kernel(long long n, V* __restrict__ x, const V* __restrict__ ph,
                                                          const V* __restrict__ sh, V* __restrict__ r,
                                                          const V* __restrict__ s, const V* __restrict__ t,
                                                          const V* __restrict__ rh, double* partials, double* sc,
                                                          unsigned* ticket) {
    if (done(sc)) return;
    const V alpha = (V)sc[S_ALPHA], omega = (V)sc[S_OMEGA];
    V a0 = (V)0, a1 = (V)0;
    // kB elements per thread and pass, all their loads issued before the first
    // store (kB runs of kThreads, each coalesced, at constant offsets)
    constexpr int kB = 4;
    const long long stride = (long long)gridDim.x * kThreads * kB;
    for (long long i0 = (long long)blockIdx.x * kThreads * kB + threadIdx.x; i0 < n; i0 += stride) {
        const long long lim = n - i0;
        V xv[kB], pv[kB], hv[kB], sv[kB], tv[kB], qv[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            const long long i = i0 + k * kThreads;
            if (k * kThreads < lim) {
                xv[k] = x[i]; pv[k] = ph[i]; hv[k] = sh[i]; sv[k] = s[i]; tv[k] = t[i]; qv[k] = rh[i];
            }
        }
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            const long long i = i0 + k * kThreads;
            if (k * kThreads < lim) {
                x[i] = fma(alpha, pv[k], fma(omega, hv[k], xv[k]));
                const V rv = fma(-omega, tv[k], sv[k]);
                r[i] = rv;
                a0 = fma(rv, rv, a0);
                a1 = fma(qv[k], rv, a1);
            }
        }
    }
    block_partials((double)a0, (double)a1, 2, partials);
    if (last_block(ticket)) scalar_step(partials, gridDim.x, sc, 0);
}

// The same update on float vectors of 16-byte aligned storage with n % 4 == 0,
// four elements per thread and pass in 16-byte loads and stores
__global__ void __launch_bounds__(kThreads) imp_xr4_kernel(long long n, float4* __restrict__ x,
                                                           const float4* __restrict__ ph,
                                                           const float4* __restrict__ sh, float4* __restrict__ r,
                                                           const float4* __restrict__ s,
                                                           const float4* __restrict__ t,
                                                           const float4* __restrict__ rh, double* partials,
                                                           double* sc, unsigned* ticket) {
    if (done(sc)) return;
    const float alpha = (float)sc[S_ALPHA], omega = (float)sc[S_OMEGA];
    float a0 = 0.f, a1 = 0.f;
    const long long n4 = n / 4;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n4; i += (long long)gridDim.x * kThreads) {
        const float4 xv = x[i], pv = ph[i], hv = sh[i], sv = s[i], tv = t[i], qv = rh[i];
        float4 xo, ro;
        xo.x = fmaf(alpha, pv.x, fmaf(omega, hv.x, xv.x));
        xo.y = fmaf(alpha, pv.y, fmaf(omega, hv.y, xv.y));
        xo.z = fmaf(alpha, pv.z, fmaf(omega, hv.z, xv.z));
        xo.w = fmaf(alpha, pv.w, fmaf(omega, hv.w, xv.w));
        ro.x = fmaf(-omega, tv.x, sv.x);
        ro.y = fmaf(-omega, tv.y, sv.y);
        ro.z = fmaf(-omega, tv.z, sv.z);
        ro.w = fmaf(-omega, tv.w, sv.w);
        x[i] = xo;
        r[i] = ro;
        a0 = fmaf(ro.x, ro.x, a0); a0 = fmaf(ro.y, ro.y, a0); a0 = fmaf(ro.z, ro.z, a0); a0 = fmaf(ro.w, ro.w, a0);
        a1 = fmaf(qv.x, ro.x, a1); a1 = fmaf(qv.y, ro.y, a1); a1 = fmaf(qv.z, ro.z, a1); a1 = fmaf(qv.w, ro.w, a1);
    }
    block_partials((double)a0, (double)a1, 2, partials);
    if (last_block(ticket)) scalar_step(partials, gridDim.x, sc, 0);
}

// per-block partial sums of x.y and x.z (z may be null), for the start of the iteration
template <typename V>
__global__ void __launch_bounds__(kThreads) imp_dot2_kernel(const V* x, const V* y, const V* z, long long n,
                                                            double* partials) {
    V a0 = (V)0, a1 = (V)0;
#pragma unroll 4
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        a0 = fma(x[i], y[i], a0);
        if (z) a1 = fma(x[i], z[i], a1);
    }
    block_partials((double)a0, (double)a1, z ? 2 : 1, partials);
}

// The scalar step alone, after a kernel that leaves its kImpBlocks partial sums
__global__ void __launch_bounds__(kThreads) imp_scalar_kernel(const double* partials, double* sc, int op) {
    scalar_step(partials, kImpBlocks, sc, op);
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
            // the modes read kMB at a time before the first is written back
            for (int j0 = 0; j0 < A.m; j0 += kMB) {
                T qv[kMB];
#pragma unroll
                for (int k = 0; k < kMB; ++k)
                    if (j0 + k < A.m) qv[k] = A.modes_nm1[mode_index(p, (j0 + k) * NC + c, A.m * NC)];
#pragma unroll
                for (int k = 0; k < kMB; ++k) {
                    const int j = j0 + k;
                    if (j >= A.m) break;
                    const long long q = mode_index(p, j * NC + c, A.m * NC);
                    if constexpr (F32) {
                        const float d = __fsub_rn((float)out, (float)s0);
                        A.modes_nm1[q] = __fmaf_rn(A.mc.rho[j], d, -A.mc.c[j] * (float)qv[k]);
                    } else {
                        const double d = (double)out - (double)s0;
                        A.modes_nm1[q] = (T)fma(A.mcd.rho[j], d, -A.mcd.c[j] * (double)qv[k]);
                    }
                }
            }
        }
        if (!finite) atomicOr(A.flags, 1u);
    }
}

// r = b - r (r holds Op(x0)), or r = b when x0 = 0 (zero: x set to 0 too);
// rh = r; p = v = 0
template <typename V>
__global__ void __launch_bounds__(kThreads) imp_init_kernel(long long n, const V* b, V* r, V* rh, V* p, V* v,
                                                            V* x, int zero) {
#pragma unroll 4
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const V rv = zero ? b[i] : b[i] - r[i];
        r[i] = rv;
        rh[i] = rv;
        p[i] = (V)0;
        v[i] = (V)0;
        if (zero) x[i] = (V)0;
    }
}

// Outer step of the mixed-precision solve: r64 = b - r64 (r64 holds Op(x) in
// FP64), its float copy rf, and the partial sums of (r64, r64)
__global__ void __launch_bounds__(kThreads) imp_resid_kernel(long long n, const double* b, double* r64, float* rf,
                                                             double* partials) {
    double a0 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double rv = b[i] - r64[i];
        r64[i] = rv;
        rf[i] = (float)rv;
        a0 = fma(rv, rv, a0);
    }
    block_partials(a0, 0.0, 1, partials);
}

// x += d (the FP32 correction of the inner solve)
__global__ void __launch_bounds__(kThreads) imp_correct_kernel(long long n, double* x, const float* d) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

// float tile-major copies of the step's operator (the point blocks and the tap
// coefficients, nc^2 + 4 d per point, in Af) and of the block-Jacobi inverses
// (nc^2 per point, in Pf), from the FP64 [k][N] arrays
template <int NC, int DIM>
__global__ void __launch_bounds__(kThreads) imp_float_operator_kernel(long long N, const double* Mb, const double* Cf,
                                                                      const double* Pinv, float* Af, float* Pf) {
    constexpr int KA = NC * NC + 4 * DIM, KP = NC * NC;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            Af[mode_index(p, k, KA)] = (float)Mb[(long long)k * N + p];
            Pf[mode_index(p, k, KP)] = (float)Pinv[(long long)k * N + p];
        }
#pragma unroll
        for (int k = 0; k < 4 * DIM; ++k) Af[mode_index(p, KP + k, KA)] = (float)Cf[(long long)k * N + p];
    }
}

// The compact float operator of a 2D forward solve: per point (tile-major, 6
// values) the extrapolated velocity gradient 2 kappa^n - kappa^{n-1} and the
// velocity, as imp_setup_kernel takes them, rounded to float (the operator and
// its block-Jacobi preconditioner are formed from them where they are applied)
template <typename T>
__global__ void __launch_bounds__(kThreads) imp_float_compact_kernel(const ImpArgs<T> A, float* Cc) {
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int ij = 0; ij < 4; ++ij) {
            const long long q = (long long)ij * N + p;
            Cc[mode_index(p, ij, kPipeCompact)] = (float)(2.0 * (double)A.kap_n[q] - (double)A.kap_nm1[q]);
        }
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) Cc[mode_index(p, 4 + ax, kPipeCompact)] = (float)A.u[(long long)ax * N + p];
    }
}

// ------------------------------------------------------------------ the paper's variable
// Right-hand side of the implicit step in the paper's variable, per point:
//   h = sum_j w_j mu_j c_j Q_j, Q_j = b1 phi_j^n + b2 phi_j^{n-1} (written over the oldest level),
//   b = -b1 Phi^n - b2 Phi^{n-1} + dt (L(kappa*) h - h/Wi) + dt G (kappa* + kappa*^T) Psi0
// (the transport of h is subtracted by imp_sub_transport_kernel); h is kept for
// Psi^{n+1} = xi Phi^{n+1} + h, and the initial guess is 2 Phi^n - Phi^{n-1}.
template <typename T, int DIM, bool COMP>
__global__ void __launch_bounds__(kThreads) imp_rhs_paper_kernel(const ImpArgs<T> A, double* b, double* x0,
                                                                 double* H) {
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
        double h[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if constexpr (F32) {
                float hs = 0.0f, comp = 0.0f;
                for (int jj = 0; jj < A.m; ++jj) {
                    const long long q = mode_index(p, jj * NC + c, A.m * NC);
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
                h[c] = (double)hs - (double)comp;
            } else {
                double hs = 0.0;
                for (int jj = 0; jj < A.m; ++jj) {
                    const long long q = mode_index(p, jj * NC + c, A.m * NC);
                    const double qj = kB1 * (double)A.modes_n[q] + kB2 * (double)A.modes_nm1[q];
                    A.modes_nm1[q] = (T)qj;
                    hs = fma(A.mcd.eta[jj], qj, hs);
                }
                h[c] = hs;
            }
        }
        double Hs[3][3];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            Hs[Packed<DIM>::I(r)][Packed<DIM>::J(r)] = h[r];
            Hs[Packed<DIM>::J(r)][Packed<DIM>::I(r)] = h[r];
        }
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
            double lh = -A.inv_wi * h[r];
#pragma unroll
            for (int l = 0; l < DIM; ++l) lh = fma(K[i][l], Hs[l][j], fma(Hs[i][l], K[j][l], lh));
            const long long q = (long long)r * N + p;
            const double pn = (double)A.sig_n[q], pm = (double)A.sig_nm1[q];
            b[q] = (2.0 * pn - 0.5 * pm) + A.dt_rhs * lh + A.dt_rhs * A.G * A.g * (K[i][j] + K[j][i]);
            x0[q] = 2.0 * pn - pm;
            H[q] = h[r];
        }
    }
}

// b -= scale (u.grad - eps Lap) H, the stencils of the operator
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_sub_transport_kernel(const ImpArgs<T> A, const double* H, double* b,
                                                                     double scale) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
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
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const double* f = H + (long long)r * N;
            const double f0 = f[p];
            double t = 0.0;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) {
                t += u[ax] * deriv_at<DIM>(f, g, ax, A.stencil, u[ax], A.inv_h[ax]);
                if (A.eps != 0.0)
                    t -= A.eps * (f[g.at(ax, -1)] - 2.0 * f0 + f[g.at(ax, 1)]) * (A.inv_h[ax] * A.inv_h[ax]);
            }
            b[(long long)r * N + p] -= scale * t;
        }
    }
}

// Psi^{n+1} = xi Phi^{n+1} + h into psi (and the caller's copy)
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_psi_kernel(const ImpArgs<T> A, const double* x, const double* H) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        bool finite = true;
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const long long q = (long long)r * N + p;
            const T v = (T)fma(A.xi, x[q], H[q]);
            finite = finite && isfinite((double)v);
            A.psi[q] = v;
            if (A.sig_copy) A.sig_copy[q] = v;
        }
        if (!finite) atomicOr(A.flags, 1u);
    }
}

// ------------------------------------------------------------------ first step (SDIRK2)
// Stage right-hand side over the grid: b = dt W sigma0 + dt sum_j mu_j Z_j/(1 + gamma mu_j dt)
// + dt G (kappa^0 + kappa^0T) g_alpha(t_i), Z the explicit mode stage; x0 = sigma^0 when given.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) start_rhs_kernel(const ImpArgs<T> A, const StartConsts C, int stage,
                                                             const T* Z, double* b, double* x0) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double gs = C.g[stage - 1];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            const double ks = (double)A.kap_n[(long long)(i * DIM + j) * N + p] +
                              (double)A.kap_n[(long long)(j * DIM + i) * N + p];
            const double s0 = A.sigma0 ? (double)A.sigma0[qc] : 0.0;
            double zs = 0.0;
            for (int jj = 0; jj < A.m; ++jj)
                zs = fma(C.mu[jj] * C.inv_den[jj], (double)Z[mode_index(p, jj * NC + c, A.m * NC)], zs);
            b[qc] = A.dt * (C.W * s0 + zs + A.G * ks * gs);
            if (x0) x0[qc] = (double)A.sig_n[qc];
        }
    }
}

// After stage 1 (x = S1): the level-(n-1) slot receives the stage-2 explicit part
//   Z_j = sigma_j^0 + dt (1 - gamma) K_j,  K_j = (-mu_j sigma_j^0 + w_j (S1 - sigma0)) / (1 + gamma mu_j dt).
// After stage 2 (x = S2): sigma^1 = S2 and sigma_j^1 = Z_j + gamma dt K_j with K_j from Z_j and S2.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) start_push_kernel(const ImpArgs<T> A, const StartConsts C, int stage,
                                                              const double* x) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double f = stage == 1 ? A.dt * (1.0 - C.gam) : A.dt * C.gam;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        bool finite = true;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const double s0 = A.sigma0 ? (double)A.sigma0[qc] : 0.0;
            const double d = x[qc] - s0;
            for (int jj = 0; jj < A.m; ++jj) {
                const long long q = mode_index(p, jj * NC + c, A.m * NC);
                const double z = stage == 1 ? (double)A.modes_n[q] : (double)A.modes_nm1[q];
                const double kj = (-C.mu[jj] * z + C.w[jj] * d) * C.inv_den[jj];
                A.modes_nm1[q] = (T)fma(f, kj, z);
            }
            if (stage == 2) {
                const T out = (T)x[qc];
                finite = finite && isfinite((double)out);
                A.sig_np1[qc] = out;
                if (A.sig_copy) A.sig_copy[qc] = out;
            }
        }
        if (!finite) atomicOr(A.flags, 1u);
    }
}

// ------------------------------------------------------------------ adjoint
// Right-hand side of the adjoint's global solve, v = s1 [+ xi lamPsi] + sum_j
// rho_j z_j with z_j = b1 lamQ'_j + b2 lamQ''_j (FP64), and the initial guess 0.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_adj_rhs_kernel(const ImpArgs<T> A, const double* s1,
                                                               const T* ell_prev, const T* ell_prev2,
                                                               const double* lam_psi, double xi, double* b,
                                                               double* x) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double acc = 0.0;
            for (int jj = 0; jj < A.m; ++jj) {
                const long long q = mode_index(p, jj * NC + c, A.m * NC);
                acc = fma(A.mcd.rho[jj], kB1 * (double)ell_prev[q] + kB2 * (double)ell_prev2[q], acc);
            }
            const long long qc = (long long)c * N + p;
            b[qc] = s1[qc] + acc + (lam_psi ? xi * lam_psi[qc] : 0.0);
            x[qc] = 0.0;
        }
    }
}

// Op -> Op^T, part 1: every point block P_p and its inverse transposed in place.
template <int NC>
__global__ void __launch_bounds__(kThreads) imp_transpose_blocks_kernel(long long N, double* Mb, double* Pinv) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int r = 0; r < NC; ++r)
#pragma unroll
            for (int k = r + 1; k < NC; ++k) {
                const long long i = (long long)(r * NC + k) * N + p, j = (long long)(k * NC + r) * N + p;
                const double m0 = Mb[i], m1 = Mb[j];
                Mb[i] = m1;
                Mb[j] = m0;
                const double q0 = Pinv[i], q1 = Pinv[j];
                Pinv[i] = q1;
                Pinv[j] = q0;
            }
    }
}

// Op -> Op^T, part 2: Op couples p to p + k e_a with Cf_{a,k}(p) (the same on
// every component), so Op^T couples p to p - k e_a with Cf_{a,k}(p - k e_a):
// the taps -2, -1, +1, +2 (t = 0..3) map to t' = 3 - t.
template <int DIM>
__global__ void __launch_bounds__(kThreads) imp_transpose_taps_kernel(long long N, int n0, int n1, int n2,
                                                                      const double* __restrict__ Cf,
                                                                      double* __restrict__ CfT) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        GridIdx g;
        g.n0 = n0;
        g.n1 = n1;
        g.n2 = n2;
        g.x = p % n0;
        g.y = (p / n0) % n1;
        g.z = p / ((long long)n0 * n1);
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int k = t < 2 ? t - 2 : t - 1;
                CfT[(long long)(a * 4 + (3 - t)) * N + p] = Cf[(long long)(a * 4 + t) * N + g.at(a, -k)];
            }
    }
}

// s1 <- M_p^T y - sum_j rho_j z_j (M_p = a I - dt L(kappa*), the pointwise part
// of the operator), so that the pointwise adjoint kernel's own M_p^-T (s1 +
// sum_j rho_j z_j) is y.
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_adj_fix_kernel(const ImpArgs<T> A, const double* y, double* s1,
                                                               const T* ell_prev, const T* ell_prev2) {
    constexpr int NC = Packed<DIM>::NC;
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
        double M[NC][NC], yp[NC];
        assemble_M<DIM>(K, A.a, A.dt, M);
#pragma unroll
        for (int c = 0; c < NC; ++c) yp[c] = y[(long long)c * N + p];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double acc = 0.0;
            for (int jj = 0; jj < A.m; ++jj) {
                const long long q = mode_index(p, jj * NC + c, A.m * NC);
                acc = fma(A.mcd.rho[jj], kB1 * (double)ell_prev[q] + kB2 * (double)ell_prev2[q], acc);
            }
            double mty = 0.0;
#pragma unroll
            for (int r = 0; r < NC; ++r) mty = fma(M[r][c], yp[r], mty);
            s1[(long long)c * N + p] = mty - acc;
        }
    }
}

// The paper's variable: lp = lamPsi - (v - M_p^T y)/xi with v = s1 + xi lamPsi +
// sum_j dt c_j z_j (y solves Op^T y = v, so v - M_p^T y = dt xi T^T y).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) imp_adj_paper_fix_kernel(const ImpArgs<T> A, const double* y,
                                                                     const double* s1, const double* lam_psi,
                                                                     double xi, const T* ell_prev,
                                                                     const T* ell_prev2, double* lp) {
    constexpr int NC = Packed<DIM>::NC;
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
        double M[NC][NC], yp[NC];
        assemble_M<DIM>(K, A.a, A.dt, M);
#pragma unroll
        for (int c = 0; c < NC; ++c) yp[c] = y[(long long)c * N + p];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            double acc = 0.0;
            for (int jj = 0; jj < A.m; ++jj) {
                const long long q = mode_index(p, jj * NC + c, A.m * NC);
                acc = fma(A.mcd.rho[jj], kB1 * (double)ell_prev[q] + kB2 * (double)ell_prev2[q], acc);
            }
            const double lpc = lam_psi ? lam_psi[qc] : 0.0;
            const double v = s1[qc] + acc + xi * lpc;
            double mty = 0.0;
#pragma unroll
            for (int r = 0; r < NC; ++r) mty = fma(M[r][c], yp[r], mty);
            lp[qc] = lpc - (v - mty) / xi;
        }
    }
}

// Adjoint of the SDIRK2 first step with implicit transport (stress form, zero
// initial modes).  The forward is the pointwise start's with M replaced by
// Op = (dt W + dt/Wi) I - dt L(kappa^0) + dt (u.grad - eps Lap):
//   S1 = Op^-1 dt (W s0 + G k g1),  S2 = Op^-1 dt (W s0 + c1 (S1 - s0) + G k g2),
//   c1 = sum_j mu_j iota_j dt (1 - gamma) w_j iota_j,  sigma^1 = S2,
//   sigma_j^1 = dt (1 - gamma) w_j iota_j (S1 - s0)(1 - gamma dt mu_j iota_j) + gamma dt w_j iota_j (S2 - s0),
// and its reverse the pointwise one with Op^-T in place of M^-T: lamr2 = Op^-T
// (s1 + a1), lamr1 = Op^-T (zq + dt c1 lamr2), with a1 = sum_j z_j gamma dt w_j
// iota_j and zq = sum_j z_j (1 - gamma dt mu_j iota_j) dt (1 - gamma) w_j iota_j.

// right-hand side of stage 1 (zero initial modes), initial guess 0
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) sta_r1_kernel(const ImpArgs<T> A, const StartConsts C, double* b,
                                                          double* x) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            const double ks = (double)A.kap_n[(long long)(i * DIM + j) * N + p] +
                              (double)A.kap_n[(long long)(j * DIM + i) * N + p];
            const double s0 = A.sigma0 ? (double)A.sigma0[qc] : 0.0;
            b[qc] = A.dt * (C.W * s0 + A.G * ks * C.g[0]);
            x[qc] = 0.0;
        }
    }
}

// the two ring sums of the start's adjoint at point p, component c
template <typename T, int NC>
__device__ __forceinline__ void sta_ring_sums(const StartConsts& C, int m, double dt, const T* ell_prev,
                                              const T* ell_prev2, long long N, long long p, int c, double& a1,
                                              double& zq) {
    const double f1 = dt * (1.0 - C.gam), f2 = dt * C.gam;
    a1 = 0.0;
    zq = 0.0;
    for (int jj = 0; jj < m; ++jj) {
        const long long q = mode_index(p, jj * NC + c, m * NC);
        const double z = kB1 * (double)ell_prev[q] + kB2 * (double)ell_prev2[q];
        const double wi = C.w[jj] * C.inv_den[jj];
        a1 = fma(z, f2 * wi, a1);
        zq = fma(z * (1.0 - f2 * C.mu[jj] * C.inv_den[jj]), f1 * wi, zq);
    }
}

__device__ __forceinline__ double sta_c1(const StartConsts& C, int m, double dt) {
    const double f1 = dt * (1.0 - C.gam);
    double c1 = 0.0;
    for (int jj = 0; jj < m; ++jj) c1 += C.mu[jj] * C.inv_den[jj] * f1 * C.w[jj] * C.inv_den[jj];
    return c1;
}

// b = s1 + a1 (stage 2's adjoint system), or b = zq + dt c1 lr2 (stage 1's) when lr2 is given
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) sta_lam_rhs_kernel(const ImpArgs<T> A, const StartConsts C,
                                                               const double* s1, const double* lr2,
                                                               const T* ell_prev, const T* ell_prev2, double* b,
                                                               double* x) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double c1 = sta_c1(C, A.m, A.dt);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            double a1, zq;
            sta_ring_sums<T, NC>(C, A.m, A.dt, ell_prev, ell_prev2, N, p, c, a1, zq);
            b[qc] = lr2 ? zq + A.dt * c1 * lr2[qc] : s1[qc] + a1;
            x[qc] = 0.0;
        }
    }
}

// adjoint of sigma0 into s1_out (s0_out, which held lamr2, set to 0) and the
// parameter terms of both stages, as in the pointwise start adjoint
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) sta_final_kernel(const ImpArgs<T> A, const StartConsts C,
                                                             const double* s0in, const T* ell_prev,
                                                             const T* ell_prev2, const double* S1, const T* S2,
                                                             const double* lr1, double* lr2_s0out, double* s1_out,
                                                             double* g_kap, double* partials, double Wi, double Re) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double c1 = sta_c1(C, A.m, A.dt);
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double gWi = 0.0, gbeta = 0.0;
    if (p < N) {
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (double)A.kap_n[(long long)(i * DIM + j) * N + p];
        double l1[NC], l2[NC], st1[NC], st2[NC], ks[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            ks[c] = K[i][j] + K[j][i];
            l1[c] = lr1[qc];
            l2[c] = lr2_s0out[qc];
            st1[c] = S1[qc];
            st2[c] = (double)S2[qc];
            double a1, zq;
            sta_ring_sums<T, NC>(C, A.m, A.dt, ell_prev, ell_prev2, N, p, c, a1, zq);
            const double lamS1 = zq + A.dt * c1 * l2[c];
            s1_out[qc] = s0in[qc] - a1 + A.dt * C.W * (l1[c] + l2[c]) - lamS1;
            lr2_s0out[qc] = 0.0;
        }
        double gK[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int stg = 0; stg < 2; ++stg) {
            const double* lam = stg == 0 ? l1 : l2;
            const double* sig = stg == 0 ? st1 : st2;
            double S3[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
                S3[i][j] = sig[r];
                S3[j][i] = sig[r];
            }
            const double src = A.dt * A.G * C.g[stg];
            double sym_dot = 0.0, sig_dot = 0.0;
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) {
                const int r = Packed<DIM>::I(cc), s2 = Packed<DIM>::J(cc);
                const double l = lam[cc];
#pragma unroll
                for (int bb = 0; bb < DIM; ++bb) {
                    gK[r][bb] += A.dt * l * S3[bb][s2];
                    gK[s2][bb] += A.dt * l * S3[r][bb];
                }
                gK[r][s2] += src * l;
                gK[s2][r] += src * l;
                sym_dot += l * ks[cc];
                sig_dot += l * sig[cc];
            }
            const double lam_G = A.dt * C.g[stg] * sym_dot;
            gWi += A.dt / (Wi * Wi) * sig_dot - A.G / Wi * lam_G;
            gbeta += -lam_G / (Wi * Re);
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int bb = 0; bb < DIM; ++bb) g_kap[(long long)(a * DIM + bb) * N + p] += gK[a][bb];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gWi += __shfl_xor_sync(0xffffffffu, gWi, off);
        gbeta += __shfl_xor_sync(0xffffffffu, gbeta, off);
    }
    const long long grp = p >> 5;     // the 32-point group of this warp
    if ((threadIdx.x & 31) == 0 && grp * 32 < N) {
        partials[2 * grp + 0] += gWi;
        partials[2 * grp + 1] += gbeta;
    }
}

// The same in the paper's variable (zero initial modes).  With gd = gamma dt,
// f1 = (1 - gamma) dt, S = sum_j w_j mu_j iota_j^2, Op = a I - gd W L(kappa^0) +
// gd W T (a = 1 + gd W/Wi) and M_p its pointwise part, the forward is
//   P1 = Op^-1 (P0 + gd G k g0),  h2 = f1 S P1,  zP = P0 + (f1/gd)(P1 - P0),
//   P2 = Op^-1 (zP - gd (L h2 - h2/Wi) + gd G k g1 + gd T h2),  Psi^1 = W P2 - h2,
// and the reverse the pointwise one (paper_start_adjoint_kernel) with Op^-T and
// one more term in the adjoint of h2, + gd T^T lamr2 = (lamP2 - M_p^T lamr2)/W.

// stage 1 of the forward: b = P0 + gd G k g0, x = 0
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) stp_r1_kernel(const ImpArgs<T> A, const StartConsts C, const T* phi0,
                                                          double dt, double* b, double* x) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double gd = C.gam * dt;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            const double ks = (double)A.kap_n[(long long)(i * DIM + j) * N + p] +
                              (double)A.kap_n[(long long)(j * DIM + i) * N + p];
            b[qc] = (phi0 ? (double)phi0[qc] : 0.0) + gd * A.G * ks * C.g[0];
            x[qc] = 0.0;
        }
    }
}

// lamP2 = s1 + W lamPsi + gd sum_j iota_j z_j at (p, c), and sum_j iota_j^2 z_j
template <typename T, int NC>
__device__ __forceinline__ double stp_lamP2(const StartConsts& C, int m, double gd, const double* s1,
                                            const double* lam_psi, const T* ell_prev, const T* ell_prev2, long long N,
                                            long long p, int c, double& a1) {
    double a2 = 0.0;
    a1 = 0.0;
    for (int jj = 0; jj < m; ++jj) {
        const long long q = mode_index(p, jj * NC + c, m * NC);
        const double z = kB1 * (double)ell_prev[q] + kB2 * (double)ell_prev2[q];
        a2 = fma(C.inv_den[jj], z, a2);
        a1 = fma(C.inv_den[jj] * C.inv_den[jj], z, a1);
    }
    const long long qc = (long long)c * N + p;
    return s1[qc] + C.W * (lam_psi ? lam_psi[qc] : 0.0) + gd * a2;
}

// b = lamP2 (lr2 == nullptr), else b = lamP1 = f1 sum_j iota_j^2 z_j + f1 S lamh2 + (f1/gd) lr2
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) stp_lam_rhs_kernel(const ImpArgs<T> A, const StartConsts C,
                                                               const double* s1, const double* lam_psi,
                                                               const double* lr2, const T* ell_prev,
                                                               const T* ell_prev2, double dt, double Wi, double* b,
                                                               double* x) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double gd = C.gam * dt, f1 = (1.0 - C.gam) * dt;
    double S = 0.0;
    for (int jj = 0; jj < A.m; ++jj) S += C.w[jj] * C.mu[jj] * C.inv_den[jj] * C.inv_den[jj];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        double lamP2[NC], a1[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) lamP2[c] = stp_lamP2<T, NC>(C, A.m, gd, s1, lam_psi, ell_prev, ell_prev2, N, p, c, a1[c]);
        if (!lr2) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                b[(long long)c * N + p] = lamP2[c];
                x[(long long)c * N + p] = 0.0;
            }
            continue;
        }
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (double)A.kap_n[(long long)(i * DIM + j) * N + p];
        double M[NC][NC], l2[NC];
        assemble_M<DIM>(K, A.a, A.dt, M);
#pragma unroll
        for (int c = 0; c < NC; ++c) l2[c] = lr2[(long long)c * N + p];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            double mty = 0.0, lt = -l2[k] / Wi;
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                mty = fma(M[r][k], l2[r], mty);
                lt = fma(uc_entry<DIM>(K, r, k), l2[r], lt);
            }
            const long long qc = (long long)k * N + p;
            const double lamh2 = -(lam_psi ? lam_psi[qc] : 0.0) - gd * lt + (lamP2[k] - mty) / C.W;
            b[qc] = f1 * a1[k] + f1 * S * lamh2 + (f1 / gd) * l2[k];
            x[qc] = 0.0;
        }
    }
}

// adjoint of Phi(0) into s1_out (s0_out, which held lamr2, set to 0) and the
// parameter terms of both stages (Y1 = W P1, Y2 = Psi^1; scale gd)
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) stp_final_kernel(const ImpArgs<T> A, const StartConsts C,
                                                             const double* s0in, const double* P1, const T* Psi1,
                                                             const double* lr1, double* lr2_s0out, double* s1_out,
                                                             double* g_kap, double* partials, double dt, double Wi,
                                                             double Re) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double gd = C.gam * dt, f1 = (1.0 - C.gam) * dt;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double gWi = 0.0, gbeta = 0.0;
    if (p < N) {
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (double)A.kap_n[(long long)(i * DIM + j) * N + p];
        double l1[NC], l2[NC], Y1[NC], Y2[NC], ks[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
            ks[c] = K[i][j] + K[j][i];
            l1[c] = lr1[qc];
            l2[c] = lr2_s0out[qc];
            Y1[c] = C.W * P1[qc];
            Y2[c] = (double)Psi1[qc];
            s1_out[qc] = s0in[qc] + l1[c] + (1.0 - f1 / gd) * l2[c];
            lr2_s0out[qc] = 0.0;
        }
        double gK[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int stg = 0; stg < 2; ++stg) {
            const double* lam = stg == 0 ? l1 : l2;
            const double* Y = stg == 0 ? Y1 : Y2;
            double Y3[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
                Y3[i][j] = Y[r];
                Y3[j][i] = Y[r];
            }
            const double src = gd * A.G * C.g[stg];
            double sym_dot = 0.0, y_dot = 0.0;
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) {
                const int r = Packed<DIM>::I(cc), s2 = Packed<DIM>::J(cc);
                const double l = lam[cc];
#pragma unroll
                for (int bb = 0; bb < DIM; ++bb) {
                    gK[r][bb] += gd * l * Y3[bb][s2];
                    gK[s2][bb] += gd * l * Y3[r][bb];
                }
                gK[r][s2] += src * l;
                gK[s2][r] += src * l;
                sym_dot += l * ks[cc];
                y_dot += l * Y[cc];
            }
            const double lam_G = gd * C.g[stg] * sym_dot;
            gWi += gd / (Wi * Wi) * y_dot - A.G / Wi * lam_G;
            gbeta += -lam_G / (Wi * Re);
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int bb = 0; bb < DIM; ++bb) g_kap[(long long)(a * DIM + bb) * N + p] += gK[a][bb];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gWi += __shfl_xor_sync(0xffffffffu, gWi, off);
        gbeta += __shfl_xor_sync(0xffffffffu, gbeta, off);
    }
    const long long grp = p >> 5;
    if ((threadIdx.x & 31) == 0 && grp * 32 < N) {
        partials[2 * grp + 0] += gWi;
        partials[2 * grp + 1] += gbeta;
    }
}

// ------------------------------------------------------------------ host side
// Krylov workspace views (10 vectors of nc N, the point blocks and the
// preconditioner inverses, the tap coefficients, the FP32 section of the inner
// solve, the paper's variable's h, partial sums, device scalars)
template <int NC>
struct KryView {
    double *b, *x, *r, *rh, *p, *v, *sv, *t, *ph, *sh, *Mb, *Pinv, *Cf, *H, *partials, *sc;
    float *Af, *Pf;   // float tile-major copies: blocks and taps (nc^2 + 4 d per point), inverses (nc^2)
    float *xf, *rf, *rhf, *pf, *vf, *svf, *tf, *phf, *shf;   // inner-solve vectors
    unsigned* ticket;
    bool transposed = false;   // the taps and blocks of an adjoint solve (no compact float operator)
    KryView(double* w, double* parts, long long N) {
        constexpr int D = NC == 3 ? 2 : 3;
        const long long n = (long long)NC * N;
        b = w; x = w + n; r = w + 2 * n; rh = w + 3 * n; p = w + 4 * n; v = w + 5 * n; sv = w + 6 * n;
        t = w + 7 * n; ph = w + 8 * n; sh = w + 9 * n;
        Mb = w + 10 * n;
        Pinv = Mb + (long long)NC * NC * N;
        Cf = Pinv + (long long)NC * NC * N;                  // 4 taps x dim axes
        // the float section starts on a 128-byte boundary (its tile rows are 128 bytes)
        double* fd = Cf + 4LL * D * N;
        fd += (16 - (long long)((reinterpret_cast<uintptr_t>(fd) / sizeof(double)) % 16)) % 16;
        const long long Np = mode_points(N);
        Af = reinterpret_cast<float*>(fd);
        Pf = Af + (long long)(NC * NC + 4 * D) * Np;
        float* fv = Pf + (long long)NC * NC * Np;
        xf = fv; rf = fv + n; rhf = fv + 2 * n; pf = fv + 3 * n; vf = fv + 4 * n; svf = fv + 5 * n;
        tf = fv + 6 * n; phf = fv + 7 * n; shf = fv + 8 * n;
        H = Cf + 4LL * D * N + kry_float_doubles(NC, D, N);   // the paper's variable only
        partials = parts;
        sc = parts + kPartialSets * kImpBlocks;
        ticket = reinterpret_cast<unsigned*>(sc + 31);   // last-block counter (the outer scalars: sc + 16)
    }
};

// One BiCGStab run (right block-Jacobi preconditioning) on Op x = b with
// vectors and coefficients of type V (FP64: the step's operator; FP32: its
// float copy in the inner solve), from x (x_zero: from 0), to the relative
// residual tol (|r| <= tol |b|) or maxit iterations.  The iteration runs on the
// device scalars sc; the host looks at them every kCheck passes.  Returns the
// iterations, the last recursive (r, r) and (b, b); synchronises st.
template <typename V>
struct BiVecs {
    const V* b;
    V *x, *r, *rh, *p, *v, *sv, *t, *ph, *sh;
    const V *Mb, *Pinv, *Cf;
    const CompactConsts* cc;   // the compact float operator (Mb holds its values), or null
};

template <typename T, int DIM, typename V>
cudaError_t bicgstab(const ImpArgs<T>& a, const BiVecs<V>& K, double* partials, double* sc, unsigned* ticket,
                     double tol, int maxit, bool x_zero, cudaStream_t st, int* iters, double* rr_out,
                     double* bnorm2_out) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = a.N;
    const long long n = (long long)NC * N;
    const unsigned bs = (unsigned)kImpBlocks;
    static const unsigned g_comb = resident_blocks(imp_comb_precond_kernel<NC, V>);
    static const unsigned g_combc = resident_blocks(imp_comb_compact_kernel);
    // the combination and the preconditioner (compact: from the operator's values)
    auto comb = [&](int mode, V* pv, V* z, cudaStream_t s) {
        if constexpr (std::is_same<V, float>::value && DIM == 2) {
            if (K.cc) {
                imp_comb_compact_kernel<<<g_combc, kThreads, 0, s>>>(N, K.Mb, *K.cc, mode, pv, K.r, K.v, z, sc);
                return;
            }
        }
        imp_comb_precond_kernel<NC, V><<<g_comb, kThreads, 0, s>>>(N, K.Pinv, mode, pv, K.r, K.v, z, sc);
    };
    static const unsigned g_xr = resident_blocks(imp_xr_kernel<V>);
    static const unsigned g_xr4 = resident_blocks(imp_xr4_kernel);
    // the float update in 16-byte accesses where every vector allows it
    bool xr4 = false;
    if constexpr (std::is_same<V, float>::value) {
        auto al16 = [](const void* q) { return reinterpret_cast<uintptr_t>(q) % 16 == 0; };
        xr4 = n % 4 == 0 && al16(K.x) && al16(K.ph) && al16(K.sh) && al16(K.r) && al16(K.sv) && al16(K.t) &&
              al16(K.rh);
    }
    cudaError_t e = cudaSuccess;
    auto ok = [&]() {
        if (e == cudaSuccess) e = cudaGetLastError();
        return e == cudaSuccess;
    };
    double hs[S_COUNT] = {};
    hs[S_RHO] = hs[S_ALPHA] = hs[S_OMEGA] = 1.0;
    hs[S_TOL2] = tol * tol;
    e = cudaMemcpyAsync(sc, hs, sizeof(hs), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    imp_dot2_kernel<V><<<bs, kThreads, 0, st>>>(K.b, K.b, nullptr, n, partials);
    if (!ok()) return e;
    imp_scalar_kernel<<<1, kThreads, 0, st>>>(partials, sc, 3);
    if (!ok()) return e;
    e = cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    *bnorm2_out = hs[S_BNORM2];
    if (hs[S_BNORM2] == 0.0) {
        e = cudaMemsetAsync(K.x, 0, sizeof(V) * (size_t)n, st);   // b = 0: x = 0
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        *iters = 0;
        *rr_out = 0.0;
        return e;
    }
    if (!x_zero) {
        launch_apply<T, DIM, V>(a, K.Mb, K.Cf, K.x, K.r, nullptr, nullptr, partials, sc, -1, ticket, K.cc, st);
        if (!ok()) return e;
    }
    imp_init_kernel<V><<<bs, kThreads, 0, st>>>(n, K.b, K.r, K.rh, K.p, K.v, K.x, x_zero ? 1 : 0);
    if (!ok()) return e;
    imp_dot2_kernel<V><<<bs, kThreads, 0, st>>>(K.r, K.r, K.rh, n, partials);
    if (!ok()) return e;
    imp_scalar_kernel<<<1, kThreads, 0, st>>>(partials, sc, 4);
    if (!ok()) return e;
    // one iteration, five launches: the scalar steps run in the last block of the
    // kernel that leaves their partial sums
    auto iteration = [&](cudaStream_t s) {
        comb(0, K.p, K.ph, s);
        launch_apply<T, DIM, V>(a, K.Mb, K.Cf, K.ph, K.v, K.rh, nullptr, partials, sc, 1, ticket, K.cc, s);
        comb(1, K.sv, K.sh, s);
        launch_apply<T, DIM, V>(a, K.Mb, K.Cf, K.sh, K.t, K.sv, K.t, partials, sc, 2, ticket, K.cc, s);
        if (xr4)
            imp_xr4_kernel<<<g_xr4, kThreads, 0, s>>>(
                n, reinterpret_cast<float4*>(K.x), reinterpret_cast<const float4*>(K.ph),
                reinterpret_cast<const float4*>(K.sh), reinterpret_cast<float4*>(K.r),
                reinterpret_cast<const float4*>(K.sv), reinterpret_cast<const float4*>(K.t),
                reinterpret_cast<const float4*>(K.rh), partials, sc, ticket);
        else
            imp_xr_kernel<V><<<g_xr, kThreads, 0, s>>>(n, K.x, K.ph, K.sh, K.r, K.sv, K.t, K.rh, partials, sc,
                                                       ticket);
    };
    // The kCheck iterations between two looks at the scalars run as one CUDA
    // graph, captured once per device, grid and workspace and kept (per host
    // thread): the kernels take nothing else, and a finished iteration makes the
    // remaining launches return at once.
    constexpr int kCheck = 8;
    using Key = std::array<long long, 34>;
    static thread_local Key key{};
    static thread_local cudaGraphExec_t exec = nullptr;
    if (maxit >= kCheck) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        // everything the captured launches take: the grid, the vectors, the
        // scalars, and the compact operator's constants (by value in the graph)
        CompactConsts q{};
        if (K.cc) q = *K.cc;
        auto bits = [](float f) { long long b = 0; std::memcpy(&b, &f, sizeof(f)); return b; };
        const Key k{dev, N, a.n0, a.n1, a.n2, (long long)g_comb, (long long)g_xr,
                    (long long)K.x, (long long)K.r, (long long)K.rh, (long long)K.p, (long long)K.v,
                    (long long)K.sv, (long long)K.t, (long long)K.ph, (long long)K.sh, (long long)K.Mb,
                    (long long)K.Pinv, (long long)K.Cf, (long long)partials, (long long)sc, (long long)ticket,
                    (long long)a.flags, K.cc ? 1 : 0, bits(q.dt), bits(q.a), bits(q.e[0]), bits(q.e[1]),
                    bits(q.ih6[0]), bits(q.ih6[1]), bits(q.ih2[0]), bits(q.ih2[1]), q.stencil, 0};
        if (!exec || k != key) {
            if (exec) (void)cudaGraphExecDestroy(exec);
            exec = nullptr;
            (void)apply_blocks<DIM, V>(true);   // the occupancy queries before the capture
            (void)pipe_blocks<kPipeFull>();
            (void)l1_blocks();
            cudaStream_t cs = nullptr;
            e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
            cudaGraph_t gr = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int i = 0; i < kCheck; ++i) iteration(cs);
                e = cudaStreamEndCapture(cs, &gr);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, gr, 0);
            if (gr) (void)cudaGraphDestroy(gr);
            (void)cudaStreamDestroy(cs);
            if (e != cudaSuccess) {
                exec = nullptr;
                (void)cudaGetLastError();
                return e;
            }
            key = k;
        }
    }
    for (int it = 0; it < maxit; it += kCheck) {
        if (it + kCheck <= maxit) {
            e = cudaGraphLaunch(exec, st);
        } else {
            for (int i = it; i < maxit; ++i) iteration(st);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        if (hs[S_DONE] != 0.0) break;
    }
    e = cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *iters = (int)hs[S_ITERS];
    *rr_out = hs[S_RR];
    return e;
}

// Op x = b to the relative residual a.tol (|b - Op x| <= tol |b|, Op in FP64)
// from the initial guess in x (b, x filled; Mb, Pinv, Cf set up, all on st),
// by mixed-precision defect correction: the FP64 residual r = b - Op x, an
// inner BiCGStab on the float copy of the operator for the correction d
// (Op d = r to the relative residual the outer target asks for, at most 1e-4
// below |r| per pass), x += d, until the FP64 residual
// meets the target.  The inner iterations then run on float vectors and float
// coefficients (FP32 arithmetic and half the bytes; on this GPU FP64 runs at
// 1/64 of the FP32 rate); the FP64 residual keeps the accuracy of the result
// that of the FP64 system.  If an outer pass gains less than a factor 16, the
// FP64 BiCGStab finishes from the current x.  Leaves the result in x,
// latches TFS_FLAG_NOCONV when the tolerance was not reached; synchronises st.
// Returns the iterations (inner and FP64 ones) and the final FP64 relative
// residual.
template <typename T, int DIM>
cudaError_t krylov_solve(const ImpArgs<T>& a, const KryView<Packed<DIM>::NC>& K, cudaStream_t st, int* iters,
                         double* relres) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = a.N;
    const long long n = (long long)NC * N;
    const unsigned bs = (unsigned)kImpBlocks;
    double* partials = K.partials;
    double* sc = K.sc;
    cudaError_t e = cudaSuccess;
    auto ok = [&]() {
        if (e == cudaSuccess) e = cudaGetLastError();
        return e == cudaSuccess;
    };
    // the float operator: on whole 2D tiles of a forward solve the compact one
    // (velocity gradient and velocity per point, from which imp_apply_l1_kernel
    // forms the operator and imp_comb_compact_kernel the preconditioner), else
    // float copies of the blocks, the taps (which may be the transposed ones of
    // an adjoint solve, kept elsewhere) and the block inverses
    CompactConsts q{};
    bool compact = false;
    if constexpr (DIM == 2) {
        compact = !K.transposed && a.n0 % kAX == 0 && a.n1 % kAY == 0;
        if (compact) {
            q.dt = (float)a.dt;
            q.a = (float)a.a;
            for (int ax = 0; ax < 2; ++ax) {
                q.e[ax] = (float)(a.eps * a.inv_h[ax] * a.inv_h[ax]);
                q.ih6[ax] = (float)(a.inv_h[ax] / 6.0);
                q.ih2[ax] = (float)(0.5 * a.inv_h[ax]);
            }
            q.stencil = a.stencil;
        }
    }
    if (compact)
        imp_float_compact_kernel<T><<<bs, kThreads, 0, st>>>(a, K.Af);
    else
        imp_float_operator_kernel<NC, DIM><<<bs, kThreads, 0, st>>>(N, K.Mb, K.Cf, K.Pinv, K.Af, K.Pf);
    if (!ok()) return e;
    // device scalars of the outer FP64 residual (never "done": the FP64 operator
    // kernel skips its work once the scalars it is given say so)
    double* sco = sc + 16;
    {
        double z[S_COUNT] = {};
        e = cudaMemcpyAsync(sco, z, sizeof(z), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    // inner solve: right-hand side rf (overwritten by the residual: b is read
    // only before the init kernel sets r = b), correction xf
    const BiVecs<float> Fv{K.rf,  K.xf,  K.rf,  K.rhf, K.pf,  K.vf, K.svf, K.tf,
                           K.phf, K.shf, K.Af,  K.Pf,  K.Af + 32LL * NC * NC,   // taps: nc^2 tile rows on
                           compact ? &q : nullptr};
    double hs[S_COUNT] = {};
    double bnorm2 = 0.0, rr = 0.0;
    int total = 0;
    bool converged = false;
    // (b, b)
    imp_dot2_kernel<double><<<bs, kThreads, 0, st>>>(K.b, K.b, nullptr, n, partials);
    if (!ok()) return e;
    imp_scalar_kernel<<<1, kThreads, 0, st>>>(partials, sc, 3);
    if (!ok()) return e;
    e = cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    bnorm2 = hs[S_BNORM2];
    if (bnorm2 == 0.0) {
        e = cudaMemsetAsync(K.x, 0, sizeof(double) * (size_t)n, st);   // b = 0: x = 0
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        *iters = 0;
        *relres = 0.0;
        return e;
    }
    const double tol2 = a.tol * a.tol * bnorm2;
    // each float pass reduces the residual by 1e-4: in float arithmetic
    // BiCGStab's convergence turns erratic well before 1e-6 (measured on the
    // 2D 1024^2 workload: passes to 1e-4 took 230-500 iterations, to 1e-6 often
    // ran into the iteration limit), so more passes of fewer iterations win
    constexpr double kInnerFloor = 1e-4;
    double prev_rr = -1.0;
    constexpr int kOuterMax = 12;
    for (int outer = 0; outer < kOuterMax; ++outer) {
        // r = b - Op x in FP64, its float copy, (r, r)
        launch_apply<T, DIM, double>(a, K.Mb, K.Cf, K.x, K.r, nullptr, nullptr, partials, sco, -1, K.ticket, nullptr,
                                     st);
        imp_resid_kernel<<<bs, kThreads, 0, st>>>(n, K.b, K.r, K.rf, partials);
        imp_scalar_kernel<<<1, kThreads, 0, st>>>(partials, sco, 3);
        if (!ok()) return e;
        e = cudaMemcpyAsync(hs, sco, sizeof(hs), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        rr = hs[S_BNORM2];
        if (rr <= tol2) {
            converged = true;
            break;
        }
        if (prev_rr >= 0.0 && rr > prev_rr / 16.0) break;   // the float inner solve no longer gains: FP64 below
        prev_rr = rr;
        // inner: Op d = r in float, to the target relative to |r| (not below 1e-6),
        // at most maxit iterations per pass
        double inner_tol = std::sqrt(tol2 / rr) * 0.5;
        if (inner_tol < kInnerFloor) inner_tol = kInnerFloor;
        int it = 0;
        double irr = 0.0, ib2 = 0.0;
        e = bicgstab<T, DIM, float>(a, Fv, partials, sc, K.ticket, inner_tol, a.maxit, true, st, &it, &irr, &ib2);
        if (e != cudaSuccess) return e;
        total += it;
        imp_correct_kernel<<<bs, kThreads, 0, st>>>(n, K.x, K.xf);
        if (!ok()) return e;
    }
    if (!converged) {
        // FP64 BiCGStab from the current iterate
        const BiVecs<double> D{K.b, K.x, K.r, K.rh, K.p, K.v, K.sv, K.t, K.ph, K.sh, K.Mb, K.Pinv, K.Cf, nullptr};
        int it = 0;
        double b2 = 0.0;
        e = bicgstab<T, DIM, double>(a, D, partials, sc, K.ticket, a.tol, a.maxit, false, st, &it, &rr, &b2);
        if (e != cudaSuccess) return e;
        total += it;
        converged = rr <= tol2;
    }
    if (!converged) {
        unsigned f = 0u;
        e = cudaMemcpyAsync(&f, a.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        f |= 16u;
        if (e == cudaSuccess) e = cudaMemcpyAsync(a.flags, &f, sizeof(unsigned), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
    }
    *iters = total;
    *relres = std::sqrt(rr / bnorm2);
    return e;
}

template <typename T, int DIM, bool COMP>
cudaError_t run_implicit(const ImpArgs<T>& a, cudaStream_t st, int* iters, double* relres) {
    constexpr int NC = Packed<DIM>::NC;
    const KryView<NC> K(a.kry, a.partials, a.N);
    const unsigned bs = (unsigned)kImpBlocks;
    // the paper's variable keeps h after the preconditioner blocks
    double* H = K.H;
    imp_setup_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, K.Mb, K.Pinv, K.Cf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.paper) {
        imp_rhs_paper_kernel<T, DIM, COMP><<<bs, kThreads, 0, st>>>(a, K.b, K.x, H);
        imp_sub_transport_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, H, K.b, a.dt_rhs);
    } else {
        imp_rhs_kernel<T, DIM, COMP><<<bs, kThreads, 0, st>>>(a, K.b, K.x);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = krylov_solve<T, DIM>(a, K, st, iters, relres);
    if (e != cudaSuccess) return e;
    if (a.paper) {
        // Phi^{n+1} and the modes by the stress form's push (sigma0 = 0, rho_j = dt c_j), then Psi
        ImpArgs<T> pa = a;
        pa.sig_copy = nullptr;
        imp_push_kernel<T, DIM><<<bs, kThreads, 0, st>>>(pa, K.x);
        imp_psi_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, K.x, H);
    } else {
        imp_push_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, K.x);
    }
    return cudaGetLastError();
}

// The SDIRK2 first step in the paper's variable with implicit transport.  At a
// stage with explicit parts ZPhi, Zphi_j, phi_j = (Zphi_j + gamma dt Phi)/(1 +
// gamma mu_j dt), Psi = W Phi - h, h = sum_j w_j mu_j Zphi_j/(1 + gamma mu_j dt), and
//   (1 + gamma dt W/Wi) Phi - gamma dt W L(kappa^0) Phi + gamma dt W T(Phi)
//       = ZPhi - gamma dt (L(kappa^0) h - h/Wi) + gamma dt G (kappa^0 + kappa^0T) Psi0(t_i) + gamma dt T(h),
// T = u.grad - eps Lap: the stress form's operator with a = 1 + gamma dt W/Wi and
// scale gamma dt W (set by the caller).  Stage 2 takes ZPhi = Phi^0 + dt (1 -
// gamma)(Phi^(1) - Phi^0)/(gamma dt), Zphi_j = phi_j^0 + dt (1 - gamma)(Phi^(1) -
// mu_j phi_j^(1)); Phi^(1) is kept in the Psi output buffer until the end.
// Right-hand side without the transport of h (added by imp_sub_transport_kernel
// with scale -gamma dt); h goes to H; x0 = Phi^0 at stage 1 (stage 2 starts
// from Phi^(1), left in x).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) start_rhs_paper_kernel(const ImpArgs<T> A, const StartConsts C, int stage,
                                                                   double* b, double* x0, double* H) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double gd = C.gam * A.dt_rhs, f1 = A.dt_rhs * (1.0 - C.gam);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) K[i][j] = (double)A.kap_n[(long long)(i * DIM + j) * N + p];
        double h[NC], zP[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            const double P0 = (double)A.sig_n[qc];
            const double P1 = stage == 2 ? (double)A.psi[qc] : 0.0;
            zP[c] = stage == 1 ? P0 : P0 + f1 * (P1 - P0) / gd;
            double hs = 0.0;
            for (int jj = 0; jj < A.m; ++jj) {
                const double z0 = (double)A.modes_n[mode_index(p, jj * NC + c, A.m * NC)];
                double z = z0;
                if (stage == 2) z = fma(f1, P1 - C.mu[jj] * (fma(gd, P1, z0) * C.inv_den[jj]), z0);
                hs = fma(C.w[jj] * C.mu[jj] * C.inv_den[jj], z, hs);
            }
            h[c] = hs;
        }
        double Hs[3][3];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            Hs[Packed<DIM>::I(r)][Packed<DIM>::J(r)] = h[r];
            Hs[Packed<DIM>::J(r)][Packed<DIM>::I(r)] = h[r];
        }
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
            double lh = -A.inv_wi * h[r];
#pragma unroll
            for (int l = 0; l < DIM; ++l) lh = fma(K[i][l], Hs[l][j], fma(Hs[i][l], K[j][l], lh));
            const long long q = (long long)r * N + p;
            b[q] = zP[r] - gd * lh + gd * A.G * (K[i][j] + K[j][i]) * C.g[stage - 1];
            if (x0) x0[q] = (double)A.sig_n[q];
            H[q] = h[r];
        }
    }
}

// After a stage solve (x = Phi of the stage): stage 1 keeps Phi^(1) in the Psi
// buffer; stage 2 writes Phi^1 = x, phi_j^1 = (Zphi_j + gamma dt Phi^1)/(1 + gamma
// mu_j dt) (Zphi_j from phi_j^0 and Phi^(1)), and Psi^1 = W Phi^1 - h over Phi^(1).
template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) start_push_paper_kernel(const ImpArgs<T> A, const StartConsts C, int stage,
                                                                    const double* x, const double* H) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const double gd = C.gam * A.dt_rhs, f1 = A.dt_rhs * (1.0 - C.gam);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        bool finite = true;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long qc = (long long)c * N + p;
            if (stage == 1) {
                A.psi[qc] = (T)x[qc];
                continue;
            }
            const double P1 = (double)A.psi[qc], P2 = x[qc];
            for (int jj = 0; jj < A.m; ++jj) {
                const long long q = mode_index(p, jj * NC + c, A.m * NC);
                const double z0 = (double)A.modes_n[q];
                const double z = fma(f1, P1 - C.mu[jj] * (fma(gd, P1, z0) * C.inv_den[jj]), z0);
                A.modes_nm1[q] = (T)(fma(gd, P2, z) * C.inv_den[jj]);
            }
            const T phi = (T)P2, psi = (T)fma(C.W, P2, -H[qc]);
            finite = finite && isfinite((double)phi) && isfinite((double)psi);
            A.sig_np1[qc] = phi;
            A.psi[qc] = psi;
            if (A.sig_copy) A.sig_copy[qc] = psi;
        }
        if (!finite) atomicOr(A.flags, 1u);
    }
}

template <typename T, int DIM>
cudaError_t run_start_implicit(const ImpArgs<T>& a, const StartConsts& c, cudaStream_t st, int* iters,
                               double* relres) {
    constexpr int NC = Packed<DIM>::NC;
    const KryView<NC> K(a.kry, a.partials, a.N);
    const unsigned bs = (unsigned)kImpBlocks;
    imp_setup_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, K.Mb, K.Pinv, K.Cf);
    cudaError_t e = cudaGetLastError();
    *iters = 0;
    *relres = 0.0;
    double* H = K.H;     // the paper's variable: h of the stage
    for (int stage = 1; stage <= 2 && e == cudaSuccess; ++stage) {
        // stage 1 reads the level-0 modes and starts from sigma^0; stage 2 reads the
        // explicit part written by the first push and starts from S1 (left in x)
        if (a.paper) {
            start_rhs_paper_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, c, stage, K.b, stage == 1 ? K.x : nullptr, H);
            imp_sub_transport_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, H, K.b, -c.gam * a.dt_rhs);
        } else {
            start_rhs_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, c, stage, stage == 1 ? a.modes_n : a.modes_nm1, K.b,
                                                              stage == 1 ? K.x : nullptr);
        }
        e = cudaGetLastError();
        int it = 0;
        double rr = 0.0;
        if (e == cudaSuccess) e = krylov_solve<T, DIM>(a, K, st, &it, &rr);
        *iters += it;
        *relres = rr > *relres ? rr : *relres;
        if (e == cudaSuccess) {
            if (a.paper) start_push_paper_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, c, stage, K.x, H);
            else start_push_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, c, stage, K.x);
            e = cudaGetLastError();
        }
    }
    return e;
}

template <typename T, int DIM>
cudaError_t run_implicit_adjoint(const ImpArgs<T>& a, double* s1, const T* ell_prev, const T* ell_prev2, double* cfT,
                                 const double* lam_psi, double xi, double* lp_out, cudaStream_t st, int* iters,
                                 double* relres) {
    constexpr int NC = Packed<DIM>::NC;
    KryView<NC> K(a.kry, a.partials, a.N);
    const unsigned bs = (unsigned)kImpBlocks;
    imp_setup_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, K.Mb, K.Pinv, K.Cf);
    imp_transpose_blocks_kernel<NC><<<bs, kThreads, 0, st>>>(a.N, K.Mb, K.Pinv);
    imp_transpose_taps_kernel<DIM><<<bs, kThreads, 0, st>>>(a.N, a.n0, a.n1, a.n2, K.Cf, cfT);
    imp_adj_rhs_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, s1, ell_prev, ell_prev2, lp_out ? lam_psi : nullptr, xi,
                                                        K.b, K.x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    K.Cf = cfT;
    K.transposed = true;
    e = krylov_solve<T, DIM>(a, K, st, iters, relres);
    if (e != cudaSuccess) return e;
    if (lp_out)
        imp_adj_paper_fix_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, K.x, s1, lam_psi, xi, ell_prev, ell_prev2,
                                                                  lp_out);
    else
        imp_adj_fix_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, K.x, s1, ell_prev, ell_prev2);
    return cudaGetLastError();
}

}  // namespace

template <typename T, int DIM>
cudaError_t run_start_implicit_adjoint(const ImpArgs<T>& a, const StartConsts& C, const StartImpAdj<T>& J,
                                       cudaStream_t st, int* iters, double* relres) {
    constexpr int NC = Packed<DIM>::NC;
    KryView<NC> K(a.kry, a.partials, a.N);
    const unsigned bs = (unsigned)kImpBlocks;
    const size_t vb = sizeof(double) * (size_t)NC * (size_t)a.N;
    int it = 0, tot = 0;
    double rr = 0.0, worst = 0.0;
    // stage 1 of the forward again: S1
    imp_setup_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, K.Mb, K.Pinv, K.Cf);
    if (J.paper) stp_r1_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, C, J.phi0, J.dt, K.b, K.x);
    else sta_r1_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, C, K.b, K.x);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = krylov_solve<T, DIM>(a, K, st, &it, &rr);
    if (e != cudaSuccess) return e;
    tot += it;
    worst = rr > worst ? rr : worst;
    e = cudaMemcpyAsync(J.S1, K.x, vb, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    // the transposed operator
    imp_transpose_blocks_kernel<NC><<<bs, kThreads, 0, st>>>(a.N, K.Mb, K.Pinv);
    imp_transpose_taps_kernel<DIM><<<bs, kThreads, 0, st>>>(a.N, a.n0, a.n1, a.n2, K.Cf, J.cfT);
    K.Cf = J.cfT;
    K.transposed = true;
    // lamr2 (kept in s0_out until the end)
    if (J.paper)
        stp_lam_rhs_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, C, J.s1, J.lam_psi, nullptr, J.ell_prev, J.ell_prev2,
                                                            J.dt, J.Wi, K.b, K.x);
    else
        sta_lam_rhs_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, C, J.s1, nullptr, J.ell_prev, J.ell_prev2, K.b, K.x);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = krylov_solve<T, DIM>(a, K, st, &it, &rr);
    if (e != cudaSuccess) return e;
    tot += it;
    worst = rr > worst ? rr : worst;
    e = cudaMemcpyAsync(J.s0_out, K.x, vb, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    // lamr1
    if (J.paper)
        stp_lam_rhs_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, C, J.s1, J.lam_psi, J.s0_out, J.ell_prev,
                                                            J.ell_prev2, J.dt, J.Wi, K.b, K.x);
    else
        sta_lam_rhs_kernel<T, DIM><<<bs, kThreads, 0, st>>>(a, C, nullptr, J.s0_out, J.ell_prev, J.ell_prev2, K.b,
                                                            K.x);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = krylov_solve<T, DIM>(a, K, st, &it, &rr);
    if (e != cudaSuccess) return e;
    tot += it;
    worst = rr > worst ? rr : worst;
    const long long blocks = (a.N + kThreads - 1) / kThreads;
    if (J.paper)
        stp_final_kernel<T, DIM><<<(unsigned)blocks, kThreads, 0, st>>>(a, C, J.s0in, J.S1, J.S2, K.x, J.s0_out,
                                                                       J.s1_out, J.g_kap, J.partials, J.dt, J.Wi,
                                                                       J.Re);
    else
        sta_final_kernel<T, DIM><<<(unsigned)blocks, kThreads, 0, st>>>(a, C, J.s0in, J.ell_prev, J.ell_prev2, J.S1,
                                                                       J.S2, K.x, J.s0_out, J.s1_out, J.g_kap,
                                                                       J.partials, J.Wi, J.Re);
    *iters = tot;
    *relres = worst;
    return cudaGetLastError();
}

cudaError_t run_start_implicit_adjoint_f64(const ImpArgs<double>& a, const StartConsts& c,
                                           const StartImpAdj<double>& j, cudaStream_t s, int* iters,
                                           double* relres) {
    return a.dim == 2 ? run_start_implicit_adjoint<double, 2>(a, c, j, s, iters, relres)
                      : run_start_implicit_adjoint<double, 3>(a, c, j, s, iters, relres);
}

cudaError_t run_start_implicit_adjoint_f32(const ImpArgs<float>& a, const StartConsts& c,
                                           const StartImpAdj<float>& j, cudaStream_t s, int* iters,
                                           double* relres) {
    return a.dim == 2 ? run_start_implicit_adjoint<float, 2>(a, c, j, s, iters, relres)
                      : run_start_implicit_adjoint<float, 3>(a, c, j, s, iters, relres);
}

cudaError_t run_implicit_adjoint_f64(const ImpArgs<double>& a, double* s1, const double* ell_prev,
                                     const double* ell_prev2, double* cfT, const double* lam_psi, double xi,
                                     double* lp_out, cudaStream_t s, int* iters, double* relres) {
    return a.dim == 2
               ? run_implicit_adjoint<double, 2>(a, s1, ell_prev, ell_prev2, cfT, lam_psi, xi, lp_out, s, iters, relres)
               : run_implicit_adjoint<double, 3>(a, s1, ell_prev, ell_prev2, cfT, lam_psi, xi, lp_out, s, iters, relres);
}

cudaError_t run_implicit_adjoint_f32(const ImpArgs<float>& a, double* s1, const float* ell_prev,
                                     const float* ell_prev2, double* cfT, const double* lam_psi, double xi,
                                     double* lp_out, cudaStream_t s, int* iters, double* relres) {
    return a.dim == 2
               ? run_implicit_adjoint<float, 2>(a, s1, ell_prev, ell_prev2, cfT, lam_psi, xi, lp_out, s, iters, relres)
               : run_implicit_adjoint<float, 3>(a, s1, ell_prev, ell_prev2, cfT, lam_psi, xi, lp_out, s, iters, relres);
}

cudaError_t run_implicit_f64(const ImpArgs<double>& a, cudaStream_t s, int* iters, double* relres) {
    return a.dim == 2 ? run_implicit<double, 2, false>(a, s, iters, relres)
                      : run_implicit<double, 3, false>(a, s, iters, relres);
}

cudaError_t run_implicit_f32(const ImpArgs<float>& a, cudaStream_t s, bool comp, int* iters, double* relres) {
    if (a.dim == 2)
        return comp ? run_implicit<float, 2, true>(a, s, iters, relres) : run_implicit<float, 2, false>(a, s, iters, relres);
    return comp ? run_implicit<float, 3, true>(a, s, iters, relres) : run_implicit<float, 3, false>(a, s, iters, relres);
}

cudaError_t run_start_implicit_f64(const ImpArgs<double>& a, const StartConsts& c, cudaStream_t s, int* iters,
                                   double* relres) {
    return a.dim == 2 ? run_start_implicit<double, 2>(a, c, s, iters, relres)
                      : run_start_implicit<double, 3>(a, c, s, iters, relres);
}

cudaError_t run_start_implicit_f32(const ImpArgs<float>& a, const StartConsts& c, cudaStream_t s, int* iters,
                                   double* relres) {
    return a.dim == 2 ? run_start_implicit<float, 2>(a, c, s, iters, relres)
                      : run_start_implicit<float, 3>(a, c, s, iters, relres);
}

}  // namespace tfs
