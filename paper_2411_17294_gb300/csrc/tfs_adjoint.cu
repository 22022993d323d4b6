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
//     M(kappa*)^T lamR = lam_sigma^{n+1}          (point solve: FP64, or FP32 in FP32 storage)
//     dJ/dsigma0 += eta lamR - sum_j rho_j z_j
//     dJ/dkappa* += dt <lamR, dM/dkappa sigma^{n+1}>-terms + dt G g d(kappa+kappa^T)^T lamR
//     dJ/dWi     += -dt/Wi^2 (-<lamR, sigma^{n+1}>) - G/Wi (dt g <lamR, sym kappa*>)
//     dJ/dbeta   += -(dt g <lamR, sym kappa*>) / (Wi Re)
// and the transport term A = dt (u.grad_h - eps Lap_h)(2 sigma^n - sigma^{n-1})
// sends -lamR back through the transposed stencil (second kernel).
// The forward modes themselves are never needed: only sigma^{n+1} and kappa.
#include <cuda_runtime.h>

#include <type_traits>

#include "tfs_device.cuh"
#include "tfs_internal.h"

namespace tfs {
namespace {

constexpr int kTileA = 32;

// Shared-memory stage of one adjoint tile (32 points).  Planes of 32 T values:
//   lamQ' [m][nc], lamQ'' [m][nc], kappa^n [d*d], kappa^{n-1} [d*d], sigma^{n+1} [nc];
// then planes of 32 doubles:
//   s1 [nc], s0 [nc], dJ/dsigma0 [nc], dJ/dkappa [d*d].
struct AdjStageMap {
    int e1, e2, kn, km, sig, tplanes;   // T planes
    int s1, s0, gs, gk, dplanes;        // double planes
};

template <int DIM>
__host__ __device__ __forceinline__ AdjStageMap adj_stage_map(int m) {
    constexpr int NC = DIM == 2 ? 3 : 6;
    AdjStageMap S;
    S.e1 = 0;
    S.e2 = m * NC;
    S.kn = 2 * m * NC;
    S.km = S.kn + DIM * DIM;
    S.sig = S.km + DIM * DIM;
    S.tplanes = S.sig + NC;
    S.s1 = 0;
    S.s0 = NC;
    S.gs = 2 * NC;
    S.gk = 3 * NC;
    S.dplanes = 3 * NC + DIM * DIM;
    return S;
}

template <typename T>
__host__ __device__ __forceinline__ size_t adj_stage_bytes(const AdjStageMap& S) {
    return (size_t)S.tplanes * kTileA * sizeof(T) + (size_t)S.dplanes * kTileA * sizeof(double);
}

template <typename T, int DIM>
__device__ __forceinline__ const T* adj_tsrc(const AdjArgs<T>& A, const AdjStageMap& S, int plane) {
    const long long N = A.N;
    if (plane < S.km) return A.kap_n + (long long)(plane - S.kn) * N;
    if (plane < S.sig) return A.kap_nm1 + (long long)(plane - S.km) * N;
    return A.sig_np1 + (long long)(plane - S.sig) * N;
}

template <typename T, int DIM>
__device__ __forceinline__ const double* adj_dsrc(const AdjArgs<T>& A, const AdjStageMap& S, int plane) {
    constexpr int NC = DIM == 2 ? 3 : 6;
    const long long N = A.N;
    if (plane < S.s0) return A.s1 + (long long)plane * N;
    if (plane < S.gs) return A.s0 + (long long)(plane - S.s0) * N;
    if (plane < S.gk) return A.g_sigma0 + (long long)(plane - S.gs) * N;
    (void)NC;
    return A.g_kap + (long long)(plane - S.gk) * N;
}

// Copy planes [p_begin, p_end) of one plane family (32-element segments
// starting at t0) into shared memory.
template <typename E, typename Src>
__device__ __forceinline__ void stage_planes(E* dst, int p_begin, int p_end, Src src_of, long long t0, long long N,
                                             int tid, int nthr, bool vec16) {
    if (vec16) {
        constexpr int EPC = 16 / sizeof(E);
        constexpr int CPP = kTileA / EPC;
        const int total = (p_end - p_begin) * CPP;
        for (int q = tid; q < total; q += nthr) {
            const int plane = p_begin + q / CPP;
            const int k = q - (plane - p_begin) * CPP;
            const long long p0 = t0 + (long long)k * EPC;
            long long valid = N - p0;
            valid = valid < 0 ? 0 : (valid > EPC ? EPC : valid);
            const E* base = src_of(plane);
            cp_async16(dst + plane * kTileA + k * EPC, base + (valid > 0 ? p0 : 0), (int)(valid * sizeof(E)));
        }
    } else {
        const int total = (p_end - p_begin) * kTileA;
        for (int q = tid; q < total; q += nthr) {
            const int plane = p_begin + q / kTileA;
            const int l = q - (plane - p_begin) * kTileA;
            const long long p = t0 + l;
            const E* base = src_of(plane);
            cp_async_small<sizeof(E)>(dst + plane * kTileA + l, base + (p < N ? p : 0), p < N ? (int)sizeof(E) : 0);
        }
    }
}

// Stage T planes [tb_begin, tb_end) of a tile, and the double planes if asked.
template <typename T, int DIM>
__device__ __forceinline__ void adj_issue(const AdjArgs<T>& A, const AdjStageMap& S, unsigned char* buf, long long t0,
                                          int tid, int nthr, bool vec16, int tb_begin, int tb_end, bool doubles) {
    T* tb = reinterpret_cast<T*>(buf);
    double* db = reinterpret_cast<double*>(buf + (size_t)S.tplanes * kTileA * sizeof(T));
    // the adjoint mode ring is tile-major (mode_index): each of its rows is 32
    // stored elements (padding past N included), copied in 16-byte chunks
    {
        constexpr int EPC = 16 / sizeof(T);
        constexpr int CPP = kTileA / EPC;
        const int mnc = S.e2;
        const int lo = tb_begin, hi = min(tb_end, S.kn);
        for (int q = tid; q < (hi - lo) * CPP; q += nthr) {
            const int plane = lo + q / CPP;
            const int k = q % CPP;
            const T* row = plane < mnc ? A.ell_prev + mode_index(t0, plane, mnc)
                                       : A.ell_prev2 + mode_index(t0, plane - mnc, mnc);
            cp_async16(tb + plane * kTileA + k * EPC, row + k * EPC, 16);
        }
    }
    if (max(tb_begin, S.kn) < tb_end)
        stage_planes<T>(tb, max(tb_begin, S.kn), tb_end, [&](int pl) { return adj_tsrc<T, DIM>(A, S, pl); }, t0,
                        A.N, tid, nthr, vec16);
    if (doubles)
        stage_planes<double>(db, 0, S.dplanes, [&](int pl) { return adj_dsrc<T, DIM>(A, S, pl); }, t0, A.N, tid,
                             nthr, vec16);
}

template <typename T, int DIM>
__device__ __forceinline__ void adj_issue_all(const AdjArgs<T>& A, const AdjStageMap& S, unsigned char* buf,
                                              long long t0, int tid, int nthr, bool vec16) {
    adj_issue<T, DIM>(A, S, buf, t0, tid, nthr, vec16, 0, S.tplanes, true);
}

template <int DIM>
struct AdjShape {
    static constexpr int NC = Packed<DIM>::NC;
    static constexpr int W = 3;
    static constexpr int CPW = NC / W;
};

// Resident blocks asked of the register allocator: the most that compile
// without spills (2D: 6; 3D: 5 in FP32, 4 in FP64).
template <typename T, int DIM>
constexpr int adj_min_blocks() {
    return DIM == 2 ? 6 : (sizeof(T) == 4 ? 5 : 4);
}

// One tile.  `after_pass1` runs on all threads right after the barrier that
// ends the first pass, when the lamQ' planes are no longer read.
template <typename T, int DIM, typename Hook>
__device__ __forceinline__ void adj_tile(const AdjArgs<T>& A, const AdjStageMap& S, unsigned char* buf,
                                         long long t0, int classic, double* sS, double* sL, double& gWi,
                                         double& gbeta, Hook after_pass1) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr int W = AdjShape<DIM>::W;
    constexpr int CPW = AdjShape<DIM>::CPW;
    constexpr bool F32 = sizeof(T) == 4;
    T* tb = reinterpret_cast<T*>(buf);
    const double* db = reinterpret_cast<const double*>(buf + (size_t)S.tplanes * kTileA * sizeof(T));
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const long long N = A.N;
    const long long p = t0 + lane;
    const bool active = p < N;
    const int m = A.m;

    // ---- z_j = b1 lamQ'_j + b2 lamQ''_j (stored in place of lamQ''), S = sum_j rho_j z_j
    if (!classic) {
        const T* e1 = tb + (S.e1 + w) * kTileA + lane;
        T* e2 = tb + (S.e2 + w) * kTileA + lane;
        if constexpr (F32) {
            float ss[CPW], comp[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) ss[cc] = comp[cc] = 0.0f;
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const float rh = A.mcf.rho[j];
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc) {
                    const int o = (j * NC + cc * W) * kTileA;
                    const float z = A.first ? 0.0f : __fmaf_rn(0.5f, e2[o], -2.0f * e1[o]);
                    e2[o] = z;
                    const float yv = __fmaf_rn(rh, z, -comp[cc]);
                    const float t = __fadd_rn(ss[cc], yv);
                    comp[cc] = __fsub_rn(__fsub_rn(t, ss[cc]), yv);
                    ss[cc] = t;
                }
            }
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) sS[(w + cc * W) * kTileA + lane] = (double)ss[cc] - (double)comp[cc];
        } else {
            double ss[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) ss[cc] = 0.0;
#pragma unroll 2
            for (int j = 0; j < m; ++j) {
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc) {
                    const int o = (j * NC + cc * W) * kTileA;
                    const double z = A.first ? 0.0 : kB1 * (double)e1[o] + kB2 * (double)e2[o];
                    e2[o] = (T)z;
                    ss[cc] = fma(A.mc.rho[j], z, ss[cc]);
                }
            }
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) sS[(w + cc * W) * kTileA + lane] = ss[cc];
        }
    } else {
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) sS[(w + cc * W) * kTileA + lane] = 0.0;
    }
    __syncthreads();
    after_pass1();

    // ---- point system and parameter derivatives by warp 0.  FP64 storage:
    //      FP64 throughout.  FP32 storage: the per-point arithmetic in FP32 (FP32
    //      LU of M^T with partial pivoting), accumulations into the FP64 fields.
    if (w == 0) {
        using R = typename std::conditional<F32, float, double>::type;
        R K[3][3];
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int b = 0; b < DIM; ++b)
                K[a][b] = (R)2 * (R)tb[(S.kn + a * DIM + b) * kTileA + lane] - (R)tb[(S.km + a * DIM + b) * kTileA + lane];
        R sig[NC], lam[NC];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            sig[r] = (R)tb[(S.sig + r) * kTileA + lane];
            lam[r] = (R)(db[(S.s1 + r) * kTileA + lane] + sS[r * kTileA + lane]);
        }
        bool ok;
        if constexpr (F32) {
            LU32<NC> F;
            static_for<0, NC>([&](auto rr) {
                constexpr int r = decltype(rr)::value;
                static_for<0, NC>([&](auto kk) {
                    constexpr int k = decltype(kk)::value;
                    // transpose: entry (r, k) of M^T is entry (k, r) of M
                    constexpr int ro = Packed<DIM>::I(k), so = Packed<DIM>::J(k);
                    constexpr int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
                    float v = 0.0f;
                    if (so == j) v += K[ro][i];
                    if (i != j && so == i) v += K[ro][j];
                    if (ro == i) v += K[so][j];
                    if (i != j && ro == j) v += K[so][i];
                    F.a[r][k] = (r == k) ? __fmaf_rn(-(float)A.dt, v, (float)A.a) : -(float)A.dt * v;
                });
            });
            ok = lu32_factor<NC>(F, 1e-30f);
            lu32_solve<NC>(F, lam);
        } else {
            double M[NC][NC], Mt[NC][NC];
            assemble_M<DIM>(K, A.a, A.dt, M);
#pragma unroll
            for (int r = 0; r < NC; ++r)
#pragma unroll
                for (int k = 0; k < NC; ++k) Mt[r][k] = M[k][r];
            ok = gauss_pp<NC>(Mt, lam, 1e-300);
        }
        // lam now holds lamR
        R gK[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) gK[a][b] = (R)0;
        R S3[3][3];
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
            S3[i][j] = sig[r];
            S3[j][i] = sig[r];
        }
        const R dtR = (R)A.dt;
        const R src = (R)(A.dt * A.G * A.g);
        R sym_dot = (R)0, sig_dot = (R)0;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            const int r = Packed<DIM>::I(cc), s2 = Packed<DIM>::J(cc);
            const R l = lam[cc];
#pragma unroll
            for (int b = 0; b < DIM; ++b) {
                gK[r][b] += dtR * l * S3[b][s2];
                gK[s2][b] += dtR * l * S3[r][b];
            }
            gK[r][s2] += src * l;
            gK[s2][r] += src * l;
            sym_dot += l * (K[r][s2] + K[s2][r]);
            sig_dot += l * sig[cc];
        }
        if (active) {
            if (!ok) atomicOr(A.flags, 2u);
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
                for (int b = 0; b < DIM; ++b) {
                    const int q = a * DIM + b;
                    A.g_kap[(long long)q * N + p] = db[(S.gk + q) * kTileA + lane] + (double)gK[a][b];
                }
            const double lam_a = -(double)sig_dot;
            const double lam_G = A.dt * A.g * (double)sym_dot;
            gWi += -A.dt / (A.Wi * A.Wi) * lam_a - A.G / A.Wi * lam_G;
            gbeta += -lam_G / (A.Wi * A.Re);
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                const long long q = (long long)r * N + p;
                const double lr = (double)lam[r];
                A.lamR[q] = lr;
                double gs = A.eta * lr - sS[r * kTileA + lane];
                double s1o = db[(S.s0 + r) * kTileA + lane];
                double s0o = 0.0;
                if (classic) {
                    s1o += kB1 * -lr;
                    s0o += kB2 * -lr;
                    gs += kB0 * -lr;
                }
                A.g_sigma0[q] = db[(S.gs + r) * kTileA + lane] + gs;
                A.s1_out[q] = s1o;
                A.s0_out[q] = s0o;
            }
        }
#pragma unroll
        for (int r = 0; r < NC; ++r) sL[r * kTileA + lane] = (double)lam[r];
    }
    __syncthreads();

    // ---- new adjoint mode level: lamQ_j = -c_j z_j - eta_j lamR, over the oldest slot
    if (!classic && active) {
        const T* zv = tb + (S.e2 + w) * kTileA + lane;
        T* out = A.ell_prev2 + mode_index(p, w, m * NC);   // tile-major ring, row j NC + c
        constexpr long long stride = (long long)NC * kTileA;
        if constexpr (F32) {
            float l[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) l[cc] = (float)sL[(w + cc * W) * kTileA + lane];
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const float ej = A.mcf.eta_hi[j], cjf = A.mcf.c[j];
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc)
                    __stcs(out + j * stride + (long long)cc * W * kTileA,
                           __fmaf_rn(-ej, l[cc], -cjf * zv[(j * NC + cc * W) * kTileA]));
            }
        } else {
            double l[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) l[cc] = sL[(w + cc * W) * kTileA + lane];
#pragma unroll 2
            for (int j = 0; j < m; ++j)
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc)
                    __stcs(out + j * stride + (long long)cc * W * kTileA,
                           (T)fma(-A.mc.eta[j], l[cc], -A.mc.c[j] * (double)zv[(j * NC + cc * W) * kTileA]));
        }
    }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(32 * AdjShape<DIM>::W, adj_min_blocks<T, DIM>())
adj_kernel(const AdjArgs<T> A, const int classic, const long long num_tiles, const int stages, const int vec16) {
    constexpr int NC = Packed<DIM>::NC;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) double sS[NC * kTileA];
    __shared__ __align__(16) double sL[NC * kTileA];
    __shared__ double sRed[2][AdjShape<DIM>::W];
    const AdjStageMap S = adj_stage_map<DIM>(classic ? 0 : A.m);
    const size_t sb = adj_stage_bytes<T>(S);
    unsigned char* buf0 = smem;
    unsigned char* buf1 = smem + sb;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int nthr = 32 * AdjShape<DIM>::W;
    double gWi = 0.0, gbeta = 0.0;

    const bool v16 = vec16 != 0;
    if (stages == 2) {
        long long tile = blockIdx.x;
        if (tile < num_tiles) adj_issue_all<T, DIM>(A, S, buf0, tile * kTileA, tid, nthr, v16);
        cp_async_commit();
        for (int it = 0; tile < num_tiles; ++it, tile += gridDim.x) {
            const long long next = tile + gridDim.x;
            unsigned char* cur = (it & 1) ? buf1 : buf0;
            unsigned char* nxt = (it & 1) ? buf0 : buf1;
            if (next < num_tiles) adj_issue_all<T, DIM>(A, S, nxt, next * kTileA, tid, nthr, v16);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            adj_tile<T, DIM>(A, S, cur, tile * kTileA, classic, sS, sL, gWi, gbeta, [] {});
            __syncthreads();
        }
        cp_async_wait<0>();
    } else {
        // One stage: the next tile's lamQ' planes are fetched while this tile
        // solves and writes its new level; the other planes after it is done.
        long long tile = blockIdx.x;
        if (tile < num_tiles) adj_issue_all<T, DIM>(A, S, buf0, tile * kTileA, tid, nthr, v16);
        cp_async_commit();
        for (; tile < num_tiles; tile += gridDim.x) {
            const long long next = tile + gridDim.x;
            cp_async_wait<0>();
            __syncthreads();
            adj_tile<T, DIM>(A, S, buf0, tile * kTileA, classic, sS, sL, gWi, gbeta, [&] {
                if (next < num_tiles) adj_issue<T, DIM>(A, S, buf0, next * kTileA, tid, nthr, v16, 0, S.e2, false);
                cp_async_commit();
            });
            __syncthreads();
            if (next < num_tiles) adj_issue<T, DIM>(A, S, buf0, next * kTileA, tid, nthr, v16, S.e2, S.tplanes, true);
            cp_async_commit();
        }
        cp_async_wait<0>();
    }
    // per-block sums of the two scalar derivatives (warp 0 holds them)
    if (threadIdx.y == 0) {
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
    (void)sRed;
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

template <typename T, int DIM>
cudaError_t launch_adj(const AdjArgs<T>& a, const LaunchCfg& cfg, cudaStream_t s) {
    auto kern = adj_kernel<T, DIM>;
    const AdjStageMap S = adj_stage_map<DIM>(cfg.classic ? 0 : a.m);
    const size_t sb = adj_stage_bytes<T>(S);
    const size_t static_bytes = 2 * Packed<DIM>::NC * kTileA * sizeof(double) + 64;
    PersistPlan plan;
    cudaError_t e = persistent_plan(reinterpret_cast<const void*>(kern), 32 * AdjShape<DIM>::W, sb, static_bytes, 2,
                                    &plan);
    if (e != cudaSuccess) return e;
    const int best_stages = plan.stages;
    const size_t dyn = plan.dyn;
    const long long num_tiles = (a.N + kTileA - 1) / kTileA;
    long long grid = (long long)plan.per_sm * plan.sms;
    if (grid > num_tiles) grid = num_tiles;
    if (grid < 1) grid = 1;
    const int vec16 = (a.N % (16 / (long long)sizeof(T))) == 0 && (a.N % 2) == 0;
    kern<<<dim3((unsigned)grid), dim3(32, AdjShape<DIM>::W), dyn, s>>>(a, cfg.classic ? 1 : 0, num_tiles,
                                                                       best_stages, vec16);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_f64(const AdjArgs<double>& a, const LaunchCfg& cfg, cudaStream_t s) {
    return cfg.dim == 2 ? launch_adj<double, 2>(a, cfg, s) : launch_adj<double, 3>(a, cfg, s);
}

cudaError_t launch_adjoint_f32(const AdjArgs<float>& a, const LaunchCfg& cfg, cudaStream_t s) {
    return cfg.dim == 2 ? launch_adj<float, 2>(a, cfg, s) : launch_adj<float, 3>(a, cfg, s);
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
