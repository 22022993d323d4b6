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
// Structure.  When transport is on, a pre-pass evaluates the stencil term A
// at every point (a 32 x 8 tile of E = 2 sigma^n - sigma^{n-1} with a 2-cell
// halo in shared memory, marching over z with the z taps in registers:
// transport_staged in 3D, its planes copied by cp.async two planes ahead,
// transport_tiled in 2D or for buffers off 16-byte boundaries; transport_kernel,
// one thread per point, for grids that do not tile) and the step kernel reads
// it like any other per-point input.  The
// step kernel is persistent: each block of 3 warps loops over tiles of 32
// consecutive points, and everything a tile reads is staged global -> shared
// by one thread before the compute phase: both mode levels by untiled bulk
// copies (cp.async.bulk; the mode levels are stored tile-major, so a tile's
// m nc rows of 32 values are one contiguous block per level), and kappa^n,
// kappa^{n-1}, A, sigma0 and, for alpha = 1 or the paper's variable, the two
// levels of the carried field by tensor-map tiles (cp.async.bulk.tensor.2d;
// cp.async on grids whose plane length is not a multiple of 16 bytes), with
// completion counted on mbarriers whose waits are bounded.  The mode stream
// (94% of the bytes) and every per-point input are in flight without holding
// registers, and the compute phase makes no global loads.  Inside a tile,
// warp w handles stress components w and w + 3 in 3D (w in 2D), lane = point:
// it forms Q_j = b1 x + b2 y from shared memory, the history sum H (FP32
// storage: Kahan summation of terms formed exactly by FMA, eta_j split
// hi + lo) and its components of the right-hand side.  Warp 0 then solves the
// 32 point systems with lane = point; all warps write the new mode level from
// the Q_j with streaming stores.  Every mode value is read once and written
// once.
//
// Point solve.  FP64 storage: FP64 Gaussian elimination with partial
// pivoting.  FP32 storage: FP32 LU with partial pivoting, one refinement step
// whose residual R - M x0 is evaluated in double-float arithmetic (TwoSum /
// TwoProd, ~44-bit), correction through the same factors: the solution of the
// system as given is accurate far beyond the FP32 rounding of the stored
// result, and the FP64 pipe (1/64 of the FP32 rate on this GPU) stays free.
#include <cuda_runtime.h>

#include <cstring>

#include "tfs_device.cuh"
#include "tfs_internal.h"

namespace tfs {
namespace {

constexpr int kTile = 32;

// Shared-memory stage of one tile: planes of 32 elements, in this order
//   modes level n [m][nc], modes level n-1 [m][nc], kappa^n [d*d], kappa^{n-1} [d*d],
//   A [nc] (transport), sigma0 [nc] (nonzero initial stress), sigma^n, sigma^{n-1} [nc] (alpha = 1;
//   the levels of Phi in the paper's variable).
struct StageMap {
    int modes;          // first plane of each group
    int kn, km, tr, s0, sig;
    int planes;         // total
};

template <int DIM>
__host__ __device__ __forceinline__ StageMap stage_map(int m, bool transport, bool sigma0, bool levels) {
    constexpr int NC = DIM == 2 ? 3 : 6;
    StageMap S;
    S.modes = 0;
    S.kn = 2 * m * NC;
    S.km = S.kn + DIM * DIM;
    S.tr = S.km + DIM * DIM;
    S.s0 = S.tr + (transport ? NC : 0);
    S.sig = S.s0 + (sigma0 ? NC : 0);
    S.planes = S.sig + (levels ? 2 * NC : 0);
    return S;
}

// Global source of stage plane `plane` for the tile starting at point t0: the
// first of its 32 elements.  Mode rows come from the tile-major levels (always
// 32 stored elements, padding past N included); every other plane is a field
// [.][N] read at t0 (elements past N are zero-filled by the caller).
template <typename T, int DIM>
__device__ __forceinline__ const T* row_src(const FwdArgs<T>& A, const StageMap& S, int plane, long long t0) {
    constexpr int NC = DIM == 2 ? 3 : 6;
    const long long N = A.N;
    if (plane < S.kn) {
        const int mnc = A.m * NC;
        const T* lv = plane < mnc ? A.modes_n : A.modes_nm1;
        const int row = plane < mnc ? plane : plane - mnc;
        return lv + mode_index(t0, row, mnc);
    }
    if (plane < S.km) return A.kap_n + (long long)(plane - S.kn) * N + t0;
    if (plane < S.tr) return A.kap_nm1 + (long long)(plane - S.km) * N + t0;
    if (plane < S.s0) return A.trans + (long long)(plane - S.tr) * N + t0;
    if (plane < S.sig) return A.sigma0 + (long long)(plane - S.s0) * N + t0;
    const int k = plane - S.sig;
    return (k < NC ? A.sig_n + (long long)k * N : A.sig_nm1 + (long long)(k - NC) * N) + t0;
}

// Copy the stage planes [pb, pe) of the tile starting at point t0 (cp.async).
template <typename T, int DIM>
__device__ __forceinline__ void issue_planes(const FwdArgs<T>& A, const StageMap& S, T* buf, long long t0, int tid,
                                             int nthr, bool vec16, int pb, int pe) {
    const long long N = A.N;
    const int mnc = A.m * (DIM == 2 ? 3 : 6);
    const int mend = 2 * mnc;   // mode planes [0, 2 mnc): whole rows, always 16-byte chunks
    constexpr int EPC = 16 / sizeof(T);    // elements per chunk
    constexpr int CPP = kTile / EPC;       // chunks per plane row
    {
        const int lo = pb, hi = min(pe, mend);
        for (int q = tid; q < (hi - lo) * CPP; q += nthr) {
            const int plane = lo + q / CPP;
            const int k = q % CPP;
            cp_async16(buf + plane * kTile + k * EPC, row_src<T, DIM>(A, S, plane, t0) + k * EPC, 16);
        }
    }
    const int b0 = max(pb, mend);
    if (b0 >= pe) return;
    if (vec16) {
        const int total = (pe - b0) * CPP;
        for (int q = tid; q < total; q += nthr) {
            const int plane = b0 + q / CPP;
            const int k = q % CPP;
            const long long p0 = t0 + (long long)k * EPC;
            long long valid = N - p0;
            valid = valid < 0 ? 0 : (valid > EPC ? EPC : valid);
            const T* base = row_src<T, DIM>(A, S, plane, 0);
            cp_async16(buf + plane * kTile + k * EPC, base + (valid > 0 ? p0 : 0), (int)(valid * sizeof(T)));
        }
    } else {
        const int total = (pe - b0) * kTile;
        for (int q = tid; q < total; q += nthr) {
            const int plane = b0 + q / kTile;
            const int l = q % kTile;
            const long long p = t0 + l;
            const T* base = row_src<T, DIM>(A, S, plane, 0);
            cp_async_small<sizeof(T)>(buf + plane * kTile + l, base + (p < N ? p : 0), p < N ? (int)sizeof(T) : 0);
        }
    }
}

// TMA staging (one thread issues): the level-n mode rows complete on bar_e,
// everything else (level n-1, kappa levels, A, sigma0, stress levels) on bar_l.
// Each mode level of a tile is one contiguous block (tile-major storage),
// fetched by untiled bulk copies of at most 32 KB; the per-point fields by
// tensor-map tiles of 32 points.
constexpr unsigned kBulkChunk = 32768;

template <typename T>
__device__ __forceinline__ void bulk_level(T* dst, const T* src, unsigned bytes, uint64_t* bar) {
    for (unsigned off = 0; off < bytes; off += kBulkChunk) {
        const unsigned b = bytes - off < kBulkChunk ? bytes - off : kBulkChunk;
        bulk_load(reinterpret_cast<char*>(dst) + off, reinterpret_cast<const char*>(src) + off, b, bar);
    }
}

template <typename T, int DIM, bool TRANSPORT>
__device__ __forceinline__ void tma_issue(const FwdArgs<T>& A, const TmaPlan& tp, const StageMap& S, T* buf,
                                          long long t0, int mnc, bool has_s0, bool levels, bool early, bool late,
                                          uint64_t* bar_e, uint64_t* bar_l) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr unsigned kPlaneBytes = kTile * sizeof(T);
    const int x = (int)t0;
    const unsigned level_bytes = (unsigned)mnc * kPlaneBytes;
    fence_proxy_async_smem();
    if (early && mnc > 0) {
        mbar_arrive_expect_tx(bar_e, level_bytes);
        bulk_level(buf, A.modes_n + mode_index(t0, 0, mnc), level_bytes, bar_e);
    }
    if (late) {
        mbar_arrive_expect_tx(bar_l, (unsigned)(S.planes - mnc) * kPlaneBytes);
        if (mnc > 0) bulk_level(buf + (size_t)mnc * kTile, A.modes_nm1 + mode_index(t0, 0, mnc), level_bytes, bar_l);
        tma_load_2d(buf + (size_t)S.kn * kTile, &tp.kn, x, 0, bar_l);
        tma_load_2d(buf + (size_t)S.km * kTile, &tp.km, x, 0, bar_l);
        if (TRANSPORT) tma_load_2d(buf + (size_t)S.tr * kTile, &tp.tr, x, 0, bar_l);
        if (has_s0) tma_load_2d(buf + (size_t)S.s0 * kTile, &tp.s0, x, 0, bar_l);
        if (levels) {
            tma_load_2d(buf + (size_t)S.sig * kTile, &tp.sn, x, 0, bar_l);
            tma_load_2d(buf + (size_t)(S.sig + NC) * kTile, &tp.sm, x, 0, bar_l);
        }
    }
}

// First derivative of E at a point: upwind3 (biased by the sign of u) or central2
template <typename T>
__device__ __forceinline__ T stencil_deriv(int stencil, T ua, T em2, T em1, T e0, T ep1, T ep2, T ih) {
    if (stencil == 1) return (ep1 - em1) * ((T)0.5 * ih);
    if (ua >= (T)0) return (em2 - (T)6 * em1 + (T)3 * e0 + (T)2 * ep1) * (ih / (T)6);
    return ((T)-2 * em1 - (T)3 * e0 + (T)6 * ep1 - ep2) * (ih / (T)6);
}

// Transport stencil of component c at point p = (x, y, z), in two halves: the
// loads (E = 2 sigma^n - sigma^{n-1} at the taps, u at the point) are issued
// before the mode sweep so that their latency overlaps it; the arithmetic runs
// after it.  Both upwind sides are loaded so that no load waits for u.
template <typename T, int DIM>
struct StencilLoads {
    T n0, m0;                // sigma^n, sigma^{n-1} at the point
    T n[DIM][4], m[DIM][4];  // taps -2, -1, +1, +2 along each axis
    T u[DIM];
};

template <typename T, int DIM>
__device__ __forceinline__ void load_stencil(const FwdArgs<T>& A, int c, int stencil, unsigned x, unsigned y,
                                             unsigned z, long long p, StencilLoads<T, DIM>& L) {
    const T* sn = A.sig_n + (long long)c * A.N;
    const T* sm = A.sig_nm1 + (long long)c * A.N;
    const unsigned nn[3] = {(unsigned)A.n0, (unsigned)A.n1, (unsigned)A.n2};
    const unsigned co[3] = {x, y, z};
    const long long strides[3] = {1, (long long)A.n0, (long long)A.n0 * A.n1};
    L.n0 = __ldg(sn + p);
    L.m0 = __ldg(sm + p);
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        // both levels at offset off (|off| <= 2) along ax: periodic wrap, or on a
        // slab the slowest axis beyond the grid from the halo planes
        auto load2 = [&](int off, T& vn, T& vm) {
            int v = (int)co[ax] + off;
            const int nax = (int)nn[ax];
            if ((v < 0 || v >= nax) && ax == DIM - 1 && A.halo_lo) {
                const long long pl = ax == 2 ? (long long)nn[0] * nn[1] : (long long)nn[0];
                const long long in_plane = p - (long long)co[ax] * pl;
                const T* hb = v < 0 ? A.halo_lo : A.halo_hi;
                const int k = v < 0 ? v + A.halo_r : v - nax;
                const long long q = ((long long)c * A.halo_r + k) * pl + in_plane;
                vn = __ldg(hb + q);
                vm = __ldg(hb + (long long)(DIM == 2 ? 3 : 6) * A.halo_r * pl + q);
                return;
            }
            if (v < 0) v += nax;
            if (v < 0) v += nax;
            if (v >= nax) v -= nax;
            if (v >= nax) v -= nax;
            const long long q = p + ((long long)v - (long long)co[ax]) * strides[ax];
            vn = __ldg(sn + q);
            vm = __ldg(sm + q);
        };
        L.u[ax] = __ldg(A.u + (long long)ax * A.N + p);
        load2(-1, L.n[ax][1], L.m[ax][1]);
        load2(1, L.n[ax][2], L.m[ax][2]);
        if (stencil == 0) {
            load2(-2, L.n[ax][0], L.m[ax][0]);
            load2(2, L.n[ax][3], L.m[ax][3]);
        } else {
            L.n[ax][0] = L.m[ax][0] = L.n[ax][3] = L.m[ax][3] = (T)0;
        }
    }
}

template <typename T, int DIM>
__device__ __forceinline__ T finish_stencil(const FwdArgs<T>& A, int stencil, const StencilLoads<T, DIM>& L) {
    const T e0 = (T)2 * L.n0 - L.m0;
    T adv = (T)0, lap = (T)0;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
        const T em2 = (T)2 * L.n[ax][0] - L.m[ax][0];
        const T em1 = (T)2 * L.n[ax][1] - L.m[ax][1];
        const T ep1 = (T)2 * L.n[ax][2] - L.m[ax][2];
        const T ep2 = (T)2 * L.n[ax][3] - L.m[ax][3];
        const T ih = (T)A.inv_h[ax];
        adv += L.u[ax] * stencil_deriv<T>(stencil, L.u[ax], em2, em1, e0, ep1, ep2, ih);
        if (A.eps != 0.0) lap += (em1 - (T)2 * e0 + ep1) * (ih * ih);
    }
    return (T)A.dt * adv - (T)(A.eps * A.dt) * lap;
}

// ----------------------------------------------------------- FP32 point solve
// Packed residual r = R - a x + dt (K x + x K^T) with R, a, dt, K as double-float
// and x a float vector.  R - a x is formed exactly (TwoProd); the operator term
// is a compensated dot product (Ogita-Rump-Oishi Dot2) of the K entries with x.
template <int DIM>
__device__ __forceinline__ void residual_f2(const f2 K[3][3], F2c a, F2c dt, const f2 R[Packed<DIM>::NC],
                                            const float x[Packed<DIM>::NC], f2 r[Packed<DIM>::NC]) {
    constexpr int NC = Packed<DIM>::NC;
    float S[3][3];
    static_for<0, NC>([&](auto cc) {
        constexpr int c = decltype(cc)::value;
        S[Packed<DIM>::I(c)][Packed<DIM>::J(c)] = x[c];
        S[Packed<DIM>::J(c)][Packed<DIM>::I(c)] = x[c];
    });
    const f2 dtf{dt.hi, dt.lo};
    static_for<0, NC>([&](auto cc) {
        constexpr int c = decltype(cc)::value;
        constexpr int i = Packed<DIM>::I(c), j = Packed<DIM>::J(c);
        float bs = 0.0f, be = 0.0f;
        auto term = [&](const f2 k, float v) {
            const f2 pr = two_prod(k.hi, v);
            const f2 sm = two_sum_f2(bs, pr.hi);
            bs = sm.hi;
            be = __fadd_rn(be, __fadd_rn(sm.lo, __fmaf_rn(k.lo, v, pr.lo)));
        };
        static_for<0, DIM>([&](auto ll) {
            constexpr int l = decltype(ll)::value;
            term(K[i][l], S[l][j]);
            term(K[j][l], S[i][l]);
        });
        const f2 ax = [&] {
            f2 pr = two_prod(a.hi, x[c]);
            pr.lo = __fmaf_rn(a.lo, x[c], pr.lo);
            return pr;
        }();
        const f2 t = f2_add(R[c], f2_neg(ax));
        r[c] = f2_add(t, f2_mul(dtf, fast_two_sum(bs, be)));
    });
}

template <int DIM>
__device__ __forceinline__ bool solve_point_f32(const f2 K[3][3], F2c a, F2c dt, const f2 R[Packed<DIM>::NC],
                                                f2 x[Packed<DIM>::NC]) {
    constexpr int NC = Packed<DIM>::NC;
    LU32<NC> F;
    const float af = a.hi, dtf = dt.hi;
    static_for<0, NC>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        static_for<0, NC>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            constexpr int ro = Packed<DIM>::I(r), so = Packed<DIM>::J(r);
            constexpr int i = Packed<DIM>::I(k), j = Packed<DIM>::J(k);
            float v = 0.0f;
            if (so == j) v += K[ro][i].hi;
            if (i != j && so == i) v += K[ro][j].hi;
            if (ro == i) v += K[so][j].hi;
            if (i != j && ro == j) v += K[so][i].hi;
            F.a[r][k] = (r == k) ? __fmaf_rn(-dtf, v, af) : -dtf * v;
        });
    });
    // row diagonal dominance (the usual case: a = eta + dt/Wi against dt |kappa*|)
    // allows elimination without row exchanges; otherwise partial pivoting
    const bool ok = row_dominant<NC>(F) ? lu32_factor_nopivot<NC>(F, 1e-30f) : lu32_factor<NC>(F, 1e-30f);
    float x0[NC];
    static_for<0, NC>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        x0[r] = R[r].hi + R[r].lo;
    });
    lu32_solve<NC>(F, x0);
    f2 res[NC];
    residual_f2<DIM>(K, a, dt, R, x0, res);
    float d[NC];
    static_for<0, NC>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        d[r] = res[r].hi + res[r].lo;
    });
    lu32_solve<NC>(F, d);
    static_for<0, NC>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        x[r] = two_sum_f2(x0[r], d[r]);
    });
    return ok;
}

// ----------------------------------------------------------------- the kernels
// Transport pre-pass: A_c(p) = dt sum_a u_a D_a(E_c) - eps dt Lap(E_c) for all
// components at point p (one thread per point), and the Courant flag.
// Per-point fallback (any grid size): one thread per point, all components.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) transport_kernel(const FwdArgs<T> A, const int stencil) {
    constexpr int NC = Packed<DIM>::NC;
    const long long N = A.N;
    const float ccoef = (float)A.courant_coef, climit = (float)A.courant_limit;
    bool over = false;   // a point above the Courant limit (latched once per block)
    const float ihf[3] = {(float)A.inv_h[0], (float)A.inv_h[1], (float)A.inv_h[2]};
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const unsigned pu = (unsigned)p;
        const unsigned px = pu % (unsigned)A.n0;
        const unsigned r1 = pu / (unsigned)A.n0;
        const unsigned py = r1 % (unsigned)A.n1;
        const unsigned pz = r1 / (unsigned)A.n1;
#pragma unroll 1
        for (int c = 0; c < NC; ++c) {
            StencilLoads<T, DIM> SL;
            load_stencil<T, DIM>(A, c, stencil, px, py, pz, p, SL);
            A.trans[(long long)c * N + p] = finish_stencil<T, DIM>(A, stencil, SL);
        }
        if (ccoef > 0.0f) {
            float cr = 0.0f;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) cr += fabsf((float)A.u[(long long)ax * N + p]) * ihf[ax];
            over = over || ccoef * cr > climit;
        }
    }
    if (__syncthreads_or(over) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(A.flags, 4u);
}

// Tiled transport pre-pass for grids with n0 % 32 == 0 and n1 % 8 == 0.
// A block owns a 32 x 8 (x, y) tile; E = 2 sigma^n - sigma^{n-1} is formed once
// per value into a shared tile with a 2-cell halo in x and y, and in 3D the
// block marches over a chunk of z planes keeping E at z-2 .. z+2 of its own
// column in registers.  Arithmetic per point is that of finish_stencil.
constexpr int kTX = 32, kTY = 8, kHalo = 2;
constexpr int kSX = kTX + 2 * kHalo, kSY = kTY + 2 * kHalo;

template <typename T>
__device__ __forceinline__ int wrapi(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kTX * kTY) transport_tiled(const FwdArgs<T> A, const int stencil, const int zchunk) {
    constexpr int NC = Packed<DIM>::NC;
    __shared__ T Es[NC][kSY][kSX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int n0 = A.n0, n1 = A.n1, n2 = A.n2;
    const long long N = A.N;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int x = x0 + tx, y = y0 + ty;
    const long long plane = (long long)n0 * n1;
    const T ih[3] = {(T)A.inv_h[0], (T)A.inv_h[1], (T)A.inv_h[2]};
    const T dtT = (T)A.dt, edt = (T)(A.eps * A.dt);
    const bool lap = A.eps != 0.0;
    const float ccoef = (float)A.courant_coef, climit = (float)A.courant_limit;
    bool over = false;   // a point above the Courant limit (latched once per block)
    const float ihf[3] = {(float)A.inv_h[0], (float)A.inv_h[1], (float)A.inv_h[2]};
    // Both stress levels of the slowest-axis plane sl (z in 3D, a y row in 2D),
    // resolved once per plane: sl may lie up to kHalo outside the grid, where
    // it wraps, or on a slab comes from the halo planes; then E at a point of
    // that plane is 2 n[c cstride + q] - m[c cstride + q].
    struct PlanePtr {
        const T* n;
        const T* m;
        long long cstride;
    };
    const int ns = DIM == 3 ? n2 : n1;
    const long long pl = DIM == 3 ? plane : (long long)n0;
    auto plane_at = [&](int sl) -> PlanePtr {
        if ((sl < 0 || sl >= ns) && A.halo_lo) {
            const T* hb = sl < 0 ? A.halo_lo : A.halo_hi;
            const long long k = sl < 0 ? sl + A.halo_r : sl - ns;
            return {hb + k * pl, hb + ((long long)NC * A.halo_r + k) * pl, (long long)A.halo_r * pl};
        }
        const long long w = wrapi<T>(sl, ns);
        return {A.sig_n + w * pl, A.sig_nm1 + w * pl, N};
    };
    auto E_in = [&](const PlanePtr& P, int c, long long q) -> T {
        const long long o = (long long)c * P.cstride + q;
        return (T)2 * __ldg(P.n + o) - __ldg(P.m + o);
    };
    const int zbeg = DIM == 3 ? blockIdx.z * zchunk : 0;
    const int zend = DIM == 3 ? min(zbeg + zchunk, n2) : 1;
    const long long q_xy = x + (long long)n0 * y;   // this thread's column within a z plane (3D)
    T qz[NC][5];   // E of this column at z-2 .. z+2 (3D)
    if (DIM == 3) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const PlanePtr P = plane_at(zbeg - 2 + k);
#pragma unroll
            for (int c = 0; c < NC; ++c) qz[c][k] = E_in(P, c, q_xy);
        }
    }
    for (int z = zbeg; z < zend; ++z) {
        if (DIM == 3) {
            const PlanePtr P = plane_at(z + 2);
#pragma unroll
            for (int c = 0; c < NC; ++c) qz[c][4] = E_in(P, c, q_xy);
        }
        // own cell and halo cells of the shared tile at plane z
        if (DIM == 3) {
#pragma unroll
            for (int c = 0; c < NC; ++c) Es[c][ty + kHalo][tx + kHalo] = qz[c][2];
        } else {
            const PlanePtr P = plane_at(y);
#pragma unroll
            for (int c = 0; c < NC; ++c) Es[c][ty + kHalo][tx + kHalo] = E_in(P, c, x);
        }
        {
            const PlanePtr Pz = plane_at(DIM == 3 ? z : 0);   // 3D: the plane z (inside the grid)
            for (int h = tid; h < kSX * kSY; h += kTX * kTY) {
                const int hy = h / kSX, hx = h - hy * kSX;
                const bool inner = hx >= kHalo && hx < kHalo + kTX && hy >= kHalo && hy < kHalo + kTY;
                if (!inner) {
                    const int gx = wrapi<T>(x0 + hx - kHalo, n0);
                    if (DIM == 3) {
                        const int gy = wrapi<T>(y0 + hy - kHalo, n1);
#pragma unroll
                        for (int c = 0; c < NC; ++c) Es[c][hy][hx] = E_in(Pz, c, gx + (long long)n0 * gy);
                    } else {
                        // in 2D the rows are the slowest axis: wrapped, or a halo row on a slab
                        const PlanePtr P = plane_at(y0 + hy - kHalo);
#pragma unroll
                        for (int c = 0; c < NC; ++c) Es[c][hy][hx] = E_in(P, c, gx);
                    }
                }
            }
        }
        __syncthreads();
        const long long p = x + (long long)n0 * y + plane * z;
        T u[DIM];
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) u[ax] = __ldg(A.u + (long long)ax * N + p);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int sy = ty + kHalo, sx = tx + kHalo;
            const T e0 = Es[c][sy][sx];
            T tap[DIM][4];
            tap[0][0] = Es[c][sy][sx - 2];
            tap[0][1] = Es[c][sy][sx - 1];
            tap[0][2] = Es[c][sy][sx + 1];
            tap[0][3] = Es[c][sy][sx + 2];
            tap[1][0] = Es[c][sy - 2][sx];
            tap[1][1] = Es[c][sy - 1][sx];
            tap[1][2] = Es[c][sy + 1][sx];
            tap[1][3] = Es[c][sy + 2][sx];
            if (DIM == 3) {
                tap[DIM - 1][0] = qz[c][0];
                tap[DIM - 1][1] = qz[c][1];
                tap[DIM - 1][2] = qz[c][3];
                tap[DIM - 1][3] = qz[c][4];
            }
            T adv = (T)0, lp = (T)0;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) {
                adv += u[ax] * stencil_deriv<T>(stencil, u[ax], tap[ax][0], tap[ax][1], e0, tap[ax][2], tap[ax][3],
                                                ih[ax]);
                if (lap) lp += (tap[ax][1] - (T)2 * e0 + tap[ax][2]) * (ih[ax] * ih[ax]);
            }
            A.trans[(long long)c * N + p] = dtT * adv - edt * lp;
        }
        if (ccoef > 0.0f) {
            float cr = 0.0f;
#pragma unroll
            for (int ax = 0; ax < DIM; ++ax) cr += fabsf((float)u[ax]) * ihf[ax];
            over = over || ccoef * cr > climit;
        }
        __syncthreads();
        if (DIM == 3) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int k = 0; k < 4; ++k) qz[c][k] = qz[c][k + 1];
        }
    }
    if (__syncthreads_or(over) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(A.flags, 4u);
}

// Staged 3D transport pre-pass (grids with n0 % 32 == 0, n1 % 8 == 0 and
// n0 n1 < 2^31 whose transported levels, halo planes and velocity start on
// 16-byte boundaries).  Same tile and z march as transport_tiled, but the
// values a plane needs are copied global -> shared by cp.async two planes
// ahead, into one of two stage buffers, so that the loads of planes z+1 and
// z+2 are in flight while plane z is evaluated and no register holds a load in
// flight.  For the plane z a stage holds: both stress levels of the block's
// own 32 x 8 columns at z+2 (the z taps, kept in registers), both levels of the
// 4 halo rows (y0-2, y0-1, y0+8, y0+9) and of the x halo pairs (x0-2, x0-1 and
// x0+32, x0+33) at z, and u at z.  Rows move as 16-byte pieces, the x halo as
// pairs of values.  The copies have fixed roles: warp c < 6 fetches component
// c's rows (own columns and y halo), warps 6 and 7 the velocity and the x halo,
// so that every address is a per-thread constant plus a per-plane base.
// E = 2 sigma^n - sigma^{n-1} is formed once per value into the shared tile.
// The stencil is applied as 13 per-point coefficients (the upwind3 or central2
// weights times dt u_a / h_a, with the Laplacian's weights times eps dt / h_a^2)
// shared by the six components.
template <typename T>
struct StagedTile {
    static constexpr int NC = 6;
    static constexpr int kPer = 16 / (int)sizeof(T);           // values per 16-byte piece
    static constexpr int kRowChunks = kTX / kPer;              // pieces of a 32-value row
    static constexpr int kRowsPerPass = 32 / kRowChunks;       // rows one warp copies per instruction
    // stage layout (values): col[2][NC][kTY][32], yh[2][NC][4][32], u[3][kTY][32], xh[2][NC][kTY][2][2]
    static constexpr int kOffYh = 2 * NC * kTY * kTX;
    static constexpr int kOffU = kOffYh + 2 * NC * 4 * kTX;
    static constexpr int kOffXh = kOffU + 3 * kTY * kTX;
    static constexpr int kStageVals = kOffXh + 2 * NC * kTY * 4;
    static constexpr size_t kStageBytes = (size_t)kStageVals * sizeof(T);
    static constexpr size_t kTileBytes = (size_t)NC * kSY * kSX * sizeof(T);
    static constexpr size_t kSmemBytes = 2 * kStageBytes + kTileBytes;
};

template <typename T>
__global__ void __launch_bounds__(kTX * kTY, sizeof(T) == 4 ? 3 : 2)
    transport_staged(const FwdArgs<T> A, const int stencil, const int zchunk) {
    using L = StagedTile<T>;
    constexpr int NC = L::NC;
    constexpr int kPer = L::kPer, kRC = L::kRowChunks, kRP = L::kRowsPerPass;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stage0 = reinterpret_cast<T*>(smem_raw);
    T (*Es)[kSY][kSX] = reinterpret_cast<T (*)[kSY][kSX]>(smem_raw + 2 * L::kStageBytes);
    const int tx = threadIdx.x, ty = threadIdx.y;   // ty = warp
    const int n0 = A.n0, n1 = A.n1, n2 = A.n2;
    const long long N = A.N;
    const long long plane = (long long)n0 * n1;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const float ccoef = (float)A.courant_coef, climit = (float)A.courant_limit;
    bool over = false;   // a point above the Courant limit (latched once per block)
    const float ihf[3] = {(float)A.inv_h[0], (float)A.inv_h[1], (float)A.inv_h[2]};
    // per-axis stencil scales: g_a = dt u_a (1/h_a)/6 multiplies the derivative
    // weights, Lw_a = eps dt / h_a^2 the Laplacian's
    const T ih6[3] = {(T)(A.inv_h[0] / 6.0), (T)(A.inv_h[1] / 6.0), (T)(A.inv_h[2] / 6.0)};
    const T dtT = (T)A.dt;
    const T Lw[3] = {(T)(A.eps * A.dt * A.inv_h[0] * A.inv_h[0]), (T)(A.eps * A.dt * A.inv_h[1] * A.inv_h[1]),
                     (T)(A.eps * A.dt * A.inv_h[2] * A.inv_h[2])};
    struct PlanePtr {
        const T* n;
        const T* m;
        long long cstride;
    };
    // both stress levels of plane sl, -kHalo <= sl < n2 + kHalo: inside the
    // grid, wrapped, or on a slab the neighbours' planes from the halo buffers
    auto plane_at = [&](int sl) -> PlanePtr {
        if ((sl < 0 || sl >= n2) && A.halo_lo) {
            const T* hb = sl < 0 ? A.halo_lo : A.halo_hi;
            const long long k = sl < 0 ? sl + A.halo_r : sl - n2;
            return {hb + k * plane, hb + ((long long)NC * A.halo_r + k) * plane, (long long)A.halo_r * plane};
        }
        while (sl < 0) sl += n2;
        while (sl >= n2) sl -= n2;
        return {A.sig_n + sl * plane, A.sig_nm1 + sl * plane, N};
    };
    // per-thread copy roles (in-plane offsets; fit in 32 bits: n0 n1 < 2^31).
    // Warps c < NC: offA = own-column row rsub, offB (offB2) = y halo row rsub
    // (rsub + kRP).  Warps NC, NC + 1 (l = 0..63): offA = u row l / kRC,
    // offB = x halo pair of row (l >> 1) & 7 on side l & 1, lcb = l >> 4 (the
    // pair's level * NC + component is lcb + 4 i for its three copies i).
    const int lane = tx, w = ty;
    unsigned offA, offB, offB2 = 0;
    int lcb = 0;
    if (w < NC) {
        const int ch = lane % kRC, rsub = lane / kRC;
        offA = (unsigned)((y0 + rsub) * n0 + x0 + ch * kPer);
        // y halo rows k: y0-2, y0-1, y0+8, y0+9 wrapped
        auto gy = [&](int k) {
            int y = k < 2 ? y0 - 2 + k : y0 + kTY - 2 + k;
            if (y < 0) y += n1;
            if (y >= n1) y -= n1;
            return y;
        };
        offB = (unsigned)(gy(rsub) * n0 + x0 + ch * kPer);
        if (kRP < 4) offB2 = (unsigned)(gy(rsub + kRP) * n0 + x0 + ch * kPer);
    } else {
        const int l = lane + 32 * (w - NC);
        offA = (unsigned)((y0 + l / kRC) * n0 + x0 + (l % kRC) * kPer);
        const int side = l & 1, r = (l >> 1) & 7;
        int xs = side ? x0 + kTX : x0 - kHalo;
        if (xs < 0) xs += n0;
        if (xs >= n0) xs -= n0;
        offB = (unsigned)((y0 + r) * n0 + xs);
        lcb = l >> 4;
    }
    auto issue = [&](int st, int z) {
        T* S = stage0 + (size_t)st * L::kStageVals;
        if (w < NC) {
            const int c = w;
            const int ch = lane % kRC, rsub = lane / kRC;
            const PlanePtr Pc = plane_at(z + 2);
            const T* cn = Pc.n + c * Pc.cstride;
            const T* cm = Pc.m + c * Pc.cstride;
            // own columns at z + 2: rows rsub + kRP i
#pragma unroll
            for (int i = 0; i < kTY / kRP; ++i) {
                const unsigned o = offA + (unsigned)(i * kRP * n0);
                const int d = ((c * kTY) + rsub + i * kRP) * kTX + ch * kPer;
                cp_async16(S + d, cn + o, 16);
                cp_async16(S + NC * kTY * kTX + d, cm + o, 16);
            }
            const T* hn = A.sig_n + (long long)z * plane + c * N;   // plane z is inside the grid
            const T* hm = A.sig_nm1 + (long long)z * plane + c * N;
#pragma unroll
            for (int i = 0; i < (kRP < 4 ? 2 : 1); ++i) {
                const int k = rsub + i * kRP;
                if (k < 4) {
                    const unsigned o = i == 0 ? offB : offB2;
                    const int d = L::kOffYh + (c * 4 + k) * kTX + ch * kPer;
                    cp_async16(S + d, hn + o, 16);
                    cp_async16(S + NC * 4 * kTX + d, hm + o, 16);
                }
            }
        } else {
            const int l = lane + 32 * (w - NC);
            const T* ub = A.u + (long long)z * plane;
            // u rows l / kRC + (64 / kRC) i of the three axes
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
#pragma unroll
                for (int i = 0; i < kTY * kRC / 64; ++i) {
                    const unsigned o = offA + (unsigned)(i * (64 / kRC) * n0);
                    const int d = L::kOffU + (ax * kTY + l / kRC + i * (64 / kRC)) * kTX + (l % kRC) * kPer;
                    cp_async16(S + d, ub + ax * N + o, 16);
                }
            const T* hn = A.sig_n + (long long)z * plane;
            const T* hm = A.sig_nm1 + (long long)z * plane;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int lc = lcb + 4 * i;
                const int lev = lc >= NC, c = lc - (lev ? NC : 0);
                const T* src = (lev ? hm : hn) + c * N + offB;
                cp_async_small<2 * sizeof(T)>(S + L::kOffXh + (size_t)(l + 64 * i) * 2, src, 2 * sizeof(T));
            }
        }
    };
    const int zbeg = blockIdx.z * zchunk;
    const int zend = min(zbeg + zchunk, n2);
    const long long q_xy = (tx + x0) + (long long)n0 * (ty + y0);
    T qz[NC][5];   // E of this column at z-2 .. z+2
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const PlanePtr P = plane_at(zbeg - 2 + k);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const long long o = (long long)c * P.cstride + q_xy;
            qz[c][k] = (T)2 * __ldg(P.n + o) - __ldg(P.m + o);
        }
    }
    issue(0, zbeg);
    cp_async_commit();
    if (zbeg + 1 < zend) issue(1, zbeg + 1);
    cp_async_commit();
    for (int z = zbeg, it = 0; z < zend; ++z, ++it) {
        const T* S = stage0 + (size_t)(it & 1) * L::kStageVals;
        cp_async_wait<1>();
        __syncthreads();   // the stage of plane z has landed; the tile is free
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int o = (c * kTY + ty) * kTX + tx;
            qz[c][4] = (T)2 * S[o] - S[NC * kTY * kTX + o];
            Es[c][ty + kHalo][tx + kHalo] = qz[c][2];
        }
        T u[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) u[ax] = S[L::kOffU + (ax * kTY + ty) * kTX + tx];
        if (w < NC) {
            // component w's halo cells: the 4 y rows (lane = x), then the x pairs
            const int c = w;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int o = L::kOffYh + (c * 4 + k) * kTX + lane;
                Es[c][k < 2 ? k : kTY + k][lane + kHalo] = (T)2 * S[o] - S[o + NC * 4 * kTX];
            }
            const int r = lane >> 2, e = lane & 3;   // e: x0-2, x0-1, x0+32, x0+33
            const int o = L::kOffXh + ((c * kTY + r) * 2 + (e >> 1)) * 2 + (e & 1);
            Es[c][r + kHalo][e < 2 ? e : kTX + e] = (T)2 * S[o] - S[o + NC * kTY * 4];
        }
        __syncthreads();   // the tile is complete and the stage has been read
        if (z + 2 < zend) issue(it & 1, z + 2);
        cp_async_commit();
        // the 13 stencil coefficients of this point: taps -2, -1, +1, +2 along
        // each axis and the centre
        T cf[3][4], c0 = (T)0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const T g = dtT * u[ax] * ih6[ax];
            T wm2, wm1, w0, wp1, wp2;
            if (stencil == 1) {
                wm2 = (T)0; wm1 = (T)-3; w0 = (T)0; wp1 = (T)3; wp2 = (T)0;
            } else if (u[ax] >= (T)0) {
                wm2 = (T)1; wm1 = (T)-6; w0 = (T)3; wp1 = (T)2; wp2 = (T)0;
            } else {
                wm2 = (T)0; wm1 = (T)-2; w0 = (T)-3; wp1 = (T)6; wp2 = (T)-1;
            }
            cf[ax][0] = g * wm2;
            cf[ax][1] = g * wm1 - Lw[ax];
            cf[ax][2] = g * wp1 - Lw[ax];
            cf[ax][3] = g * wp2;
            c0 += g * w0 + (T)2 * Lw[ax];
        }
        const long long p = q_xy + plane * z;
        const int sy = ty + kHalo, sx = tx + kHalo;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            T acc = c0 * qz[c][2];
            acc += cf[0][0] * Es[c][sy][sx - 2];
            acc += cf[0][1] * Es[c][sy][sx - 1];
            acc += cf[0][2] * Es[c][sy][sx + 1];
            acc += cf[0][3] * Es[c][sy][sx + 2];
            acc += cf[1][0] * Es[c][sy - 2][sx];
            acc += cf[1][1] * Es[c][sy - 1][sx];
            acc += cf[1][2] * Es[c][sy + 1][sx];
            acc += cf[1][3] * Es[c][sy + 2][sx];
            acc += cf[2][0] * qz[c][0];
            acc += cf[2][1] * qz[c][1];
            acc += cf[2][2] * qz[c][3];
            acc += cf[2][3] * qz[c][4];
            A.trans[(long long)c * N + p] = acc;
        }
        if (ccoef > 0.0f) {
            float cr = 0.0f;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) cr += fabsf((float)u[ax]) * ihf[ax];
            over = over || ccoef * cr > climit;
        }
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int k = 0; k < 4; ++k) qz[c][k] = qz[c][k + 1];
    }
    cp_async_wait<0>();
    if (__syncthreads_or(over) && threadIdx.x == 0 && threadIdx.y == 0) atomicOr(A.flags, 4u);
}

// Warps per block of the step kernel: each warp handles NC / kWarps stress
// components of the tile's 32 points (3D: 2 components per warp, 2D: 1).
template <int DIM>
struct StepShape {
    static constexpr int NC = Packed<DIM>::NC;
    static constexpr int W = 3;
    static constexpr int CPW = NC / W;
};

// Modes whose Q_j a thread keeps in registers when the stage buffer is to be
// refilled right after the history sums (QR variant of the step kernel).
constexpr int kQR = 32;

// Packed index of the symmetric pair (a, b) (inverse of Packed<DIM>::I, J)
template <int DIM>
__device__ __forceinline__ int packed_index(int a, int b) {
    if (a == b) return DIM == 2 ? 2 * a : a;
    if (DIM == 2) return 1;
    return a + b == 3 ? 3 : (a + b == 2 ? 4 : 5);   // yz, xz, xy
}

// Right-hand side component r of the paper's variable in FP32 storage (the
// solving warp's system):
//   -b1 Phi^n - b2 Phi^{n-1} + dt G (kappa* + kappa*^T) Psi0 [- A] + dt (L(kappa*) h - h/Wi)
// Kat(a, b): kappa*_ab in double-float; Hat(a, b): the leading part of the
// history sum h_ab.  One definition for the solving warp (all r, values in
// registers) and for the per-warp form of the register variant (its own r,
// values read from shared memory), so both give the same bits.
template <int DIM, bool TRANSPORT, typename KA, typename HA>
__device__ __forceinline__ f2 paper_rhs_f32(const FwdArgs<float>& A, const StageMap& S, const float* buf, int lane,
                                            KA Kat, HA Hat, int r) {
    constexpr int NC = Packed<DIM>::NC;
    const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
    const f2 src{A.src_f2.hi, A.src_f2.lo};
    const float dtf = A.dt_f2.hi, iwi = (float)A.inv_wi;
    const float pn = buf[(S.sig + r) * kTile + lane];
    const float pm = buf[(S.sig + NC + r) * kTile + lane];
    f2 v = two_sum_f2(2.0f * pn, -0.5f * pm);
    v = f2_add(v, f2_mul(src, f2_add(Kat(i, j), Kat(j, i))));
    if constexpr (TRANSPORT) v = f2_add_f(v, -buf[(S.tr + r) * kTile + lane]);
    // the operator on h enters scaled by dt: float accuracy suffices
    float lh = -iwi * Hat(i, j);
#pragma unroll
    for (int l = 0; l < DIM; ++l) lh = __fmaf_rn(Kat(i, l).hi, Hat(l, j), __fmaf_rn(Hat(i, l), Kat(j, l).hi, lh));
    return f2_add_f(v, dtf * lh);
}

// One tile.  QR (FP32 storage, alpha < 1, m <= kQR): the Q_j of a thread's
// components stay in registers and the solving warp copies its kappa and
// sigma0 values out of the stage before the hook (in the paper's variable every
// warp first forms its components' right-hand side from the stage, kept in
// sD until the solve), so the hook may refill the whole stage buffer with the
// next tile while this one is solved and pushed forward; otherwise Q_j is
// stored over level n-1 in the stage and the hook may refill only the level-n
// mode planes.
template <typename T, int DIM, bool TRANSPORT, bool COMP, bool PAPER, bool QR, typename Hook>
__device__ __forceinline__ void compute_tile(const FwdArgs<T>& A, const StageMap& S, T* buf, long long t0,
                                             int classic, void* sR_raw, float* sD, Hook after_pass1) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr int W = StepShape<DIM>::W;
    constexpr int CPW = StepShape<DIM>::CPW;
    constexpr bool F32 = sizeof(T) == 4;
    static_assert(!QR || F32, "the register variant serves FP32 storage");
    float qr[QR ? CPW : 1][QR ? kQR : 1];   // Q_j in registers (QR)
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const long long N = A.N;
    const long long p = t0 + lane;
    const bool active = p < N;
    const int m = A.m;
    const bool has_s0 = A.sigma0 != nullptr;

    // ---- (a4) history sums over the modes of this thread's components
    //      (Q_j stored in place of level n-1)
    double Hd[CPW];
    f2 Hf[CPW];
    T s0c[CPW];
#pragma unroll
    for (int cc = 0; cc < CPW; ++cc) {
        const int c = w + cc * W;
        Hd[cc] = 0.0;
        Hf[cc] = f2{0.0f, 0.0f};
        s0c[cc] = has_s0 ? buf[(S.s0 + c) * kTile + lane] : (T)0;
    }
    if (classic) {
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            const int c = w + cc * W;
            const T sn = buf[(S.sig + c) * kTile + lane];
            const T sm = buf[(S.sig + NC + c) * kTile + lane];
            if constexpr (F32) {
                // b1 sigma^n + b2 sigma^{n-1} + b0 sigma0: exact products by powers of two, TwoProd for b0
                const f2 h = two_sum_f2(-2.0f * (float)sn, 0.5f * (float)sm);
                Hf[cc] = f2_add(h, two_prod(1.5f, (float)s0c[cc]));
            } else {
                Hd[cc] = kB1 * (double)sn + kB2 * (double)sm + kB0 * (double)s0c[cc];
            }
        }
    } else {
        const T* lv0 = buf + (w * kTile + lane);
        T* lv1 = buf + ((m * NC + w) * kTile + lane);
        if constexpr (F32 && COMP) {
            // Kahan summation of the terms eta_j Q_j: each term enters as
            // fma(eta_hi, Q, fma(eta_lo, Q, -comp)) -- the product is exact inside
            // the FMA, so the term is rounded once -- and the rounding error of
            // every addition is carried in `comp` (adds that are never contracted)
            float hs[CPW], comp[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) hs[cc] = comp[cc] = 0.0f;
            auto kahan_term = [&](int j, int cc, float qj) {
                const float yv = __fmaf_rn(A.mc.eta_hi[j], qj, __fmaf_rn(A.mc.eta_lo[j], qj, -comp[cc]));
                const float t = __fadd_rn(hs[cc], yv);
                comp[cc] = __fsub_rn(__fsub_rn(t, hs[cc]), yv);
                hs[cc] = t;
            };
            if constexpr (QR) {
#pragma unroll
                for (int j = 0; j < kQR; ++j) {
                    if (j < m) {
#pragma unroll
                        for (int cc = 0; cc < CPW; ++cc) {
                            const int o = (j * NC + cc * W) * kTile;
                            const float qj = __fmaf_rn(0.5f, (float)lv1[o], -2.0f * (float)lv0[o]);
                            qr[cc][j] = qj;
                            kahan_term(j, cc, qj);
                        }
                    }
                }
            } else {
#pragma unroll 4
                for (int j = 0; j < m; ++j) {
#pragma unroll
                    for (int cc = 0; cc < CPW; ++cc) {
                        const int o = (j * NC + cc * W) * kTile;
                        const float x = lv0[o];
                        const float y = lv1[o];
                        const float qj = __fmaf_rn(0.5f, y, -2.0f * x);
                        lv1[o] = qj;
                        kahan_term(j, cc, qj);
                    }
                }
            }
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) Hf[cc] = fast_two_sum(hs[cc], -comp[cc]);
        } else if constexpr (F32) {
            float hs[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) hs[cc] = 0.0f;
            if constexpr (QR) {
#pragma unroll
                for (int j = 0; j < kQR; ++j) {
                    if (j < m) {
#pragma unroll
                        for (int cc = 0; cc < CPW; ++cc) {
                            const int o = (j * NC + cc * W) * kTile;
                            const float qj = __fmaf_rn(0.5f, (float)lv1[o], -2.0f * (float)lv0[o]);
                            qr[cc][j] = qj;
                            hs[cc] = __fmaf_rn(A.mc.eta_hi[j], qj, hs[cc]);
                        }
                    }
                }
            } else {
#pragma unroll 4
                for (int j = 0; j < m; ++j) {
#pragma unroll
                    for (int cc = 0; cc < CPW; ++cc) {
                        const int o = (j * NC + cc * W) * kTile;
                        const float qj = __fmaf_rn(0.5f, lv1[o], -2.0f * lv0[o]);
                        lv1[o] = qj;
                        hs[cc] = __fmaf_rn(A.mc.eta_hi[j], qj, hs[cc]);
                    }
                }
            }
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) Hf[cc] = f2_from(hs[cc]);
        } else {
#pragma unroll 2
            for (int j = 0; j < m; ++j) {
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc) {
                    const int o = (j * NC + cc * W) * kTile;
                    const double qj = kB1 * (double)lv0[o] + kB2 * (double)lv1[o];
                    lv1[o] = (T)qj;
                    Hd[cc] = fma(A.mc.eta[j], qj, Hd[cc]);
                }
            }
        }
    }

    // ---- right-hand side components (the paper's variable: the history sums h
    //      themselves; its right-hand side couples the components and is formed
    //      by the solving warp)
#pragma unroll
    for (int cc = 0; cc < CPW && PAPER; ++cc) {
        const int c = w + cc * W;
        if constexpr (F32) reinterpret_cast<f2*>(sR_raw)[c * kTile + lane] = Hf[cc];
        else reinterpret_cast<double*>(sR_raw)[c * kTile + lane] = Hd[cc];
    }
#pragma unroll
    for (int cc = 0; cc < CPW && !PAPER; ++cc) {
        const int c = w + cc * W;
        const int ci = Packed<DIM>::I(c), cj = Packed<DIM>::J(c);
        const T kn_ij = buf[(S.kn + ci * DIM + cj) * kTile + lane];
        const T km_ij = buf[(S.km + ci * DIM + cj) * kTile + lane];
        const T kn_ji = buf[(S.kn + cj * DIM + ci) * kTile + lane];
        const T km_ji = buf[(S.km + cj * DIM + ci) * kTile + lane];
        if constexpr (F32) {
            const f2 kab = two_sum_f2(2.0f * (float)kn_ij, -(float)km_ij);
            const f2 kba = two_sum_f2(2.0f * (float)kn_ji, -(float)km_ji);
            const f2 ks = f2_add(kab, kba);
            const f2 eta{A.eta_f2.hi, A.eta_f2.lo}, src{A.src_f2.hi, A.src_f2.lo};
            f2 R = f2_add(f2_mul_f(eta, (float)s0c[cc]), f2_neg(Hf[cc]));
            R = f2_add(R, f2_mul(src, ks));
            if constexpr (TRANSPORT) R = f2_add_f(R, -(float)buf[(S.tr + c) * kTile + lane]);
            reinterpret_cast<f2*>(sR_raw)[c * kTile + lane] = R;
        } else {
            const double ks = (2.0 * (double)kn_ij - (double)km_ij) + (2.0 * (double)kn_ji - (double)km_ji);
            double R = A.eta * (double)s0c[cc] - Hd[cc] + A.dt * A.G * A.g * ks;
            if constexpr (TRANSPORT) R -= (double)buf[(S.tr + c) * kTile + lane];
            reinterpret_cast<double*>(sR_raw)[c * kTile + lane] = R;
        }
    }
    // QR: the solving warp's stage inputs in registers, so that the hook may
    // refill the whole stage
    float kn_r[QR ? DIM * DIM : 1], km_r[QR ? DIM * DIM : 1], s0_r[QR ? NC : 1];
    if constexpr (QR) {
        if (w == 0) {
#pragma unroll
            for (int i = 0; i < DIM * DIM; ++i) {
                kn_r[i] = (float)buf[(S.kn + i) * kTile + lane];
                km_r[i] = (float)buf[(S.km + i) * kTile + lane];
            }
#pragma unroll
            for (int r = 0; r < NC; ++r) s0_r[r] = has_s0 ? (float)buf[(S.s0 + r) * kTile + lane] : 0.0f;
        }
    }
    auto kn_at = [&](int i) -> float {
        if constexpr (QR) return kn_r[i];
        else return (float)buf[(S.kn + i) * kTile + lane];
    };
    auto km_at = [&](int i) -> float {
        if constexpr (QR) return km_r[i];
        else return (float)buf[(S.km + i) * kTile + lane];
    };
    if constexpr (PAPER && QR) {
        // every h is in sR: each warp forms its components' right-hand side
        // from the stage (into sD, which the solving warp reads before it
        // writes its own values there)
        __syncthreads();
        const f2* sH = reinterpret_cast<const f2*>(sR_raw);
        const float* fb = reinterpret_cast<const float*>(buf);
        auto Kat = [&](int a, int b) {
            return two_sum_f2(2.0f * fb[(S.kn + a * DIM + b) * kTile + lane], -fb[(S.km + a * DIM + b) * kTile + lane]);
        };
        auto Hat = [&](int a, int b) { return sH[packed_index<DIM>(a, b) * kTile + lane].hi; };
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            const int c = w + cc * W;
            reinterpret_cast<f2*>(sD)[c * kTile + lane] = paper_rhs_f32<DIM, TRANSPORT>(A, S, fb, lane, Kat, Hat, c);
        }
    }
    __syncthreads();
    // level n of the mode planes (QR: the whole stage) is no longer read in this tile
    after_pass1();

    // ---- (a2) + (a5) point solve by warp 0
    if (w == 0) {
        T out[NC];
        T psi[NC];
        unsigned fl = 0u;
        if constexpr (PAPER) {
            // (b0 + dt xi/Wi) Phi - dt xi L(kappa*) Phi
            //     = -b1 Phi^n - b2 Phi^{n-1} + dt (L(kappa*) h - h/Wi) + dt G (kappa* + kappa*^T) Psi0 [- A]
            // (A: the transport of E = 2 Psi^n - Psi^{n-1}, from the pre-pass)
            // Psi^{n+1} = xi Phi^{n+1} + h
            if constexpr (F32) {
                f2 K[3][3];
                float Kf[3][3];
#pragma unroll
                for (int a = 0; a < DIM; ++a)
#pragma unroll
                    for (int b = 0; b < DIM; ++b) {
                        K[a][b] = two_sum_f2(2.0f * kn_at(a * DIM + b), -km_at(a * DIM + b));
                        Kf[a][b] = K[a][b].hi;
                    }
                const f2* sH = reinterpret_cast<const f2*>(sR_raw);
                f2 h[NC], R[NC], x[NC];
                if constexpr (QR) {
                    // h is read after the solve (fewer live registers during it)
#pragma unroll
                    for (int r = 0; r < NC; ++r) R[r] = reinterpret_cast<const f2*>(sD)[r * kTile + lane];
                } else {
                    float Hs[3][3];
#pragma unroll
                    for (int r = 0; r < NC; ++r) {
                        h[r] = sH[r * kTile + lane];
                        Hs[Packed<DIM>::I(r)][Packed<DIM>::J(r)] = h[r].hi;
                        Hs[Packed<DIM>::J(r)][Packed<DIM>::I(r)] = h[r].hi;
                    }
                    auto Kat = [&](int a, int b) { return K[a][b]; };
                    auto Hat = [&](int a, int b) { return Hs[a][b]; };
#pragma unroll
                    for (int r = 0; r < NC; ++r)
                        R[r] = paper_rhs_f32<DIM, TRANSPORT>(A, S, reinterpret_cast<const float*>(buf), lane, Kat, Hat,
                                                             r);
                }
                if (!solve_point_f32<DIM>(K, A.a_f2, A.dtxi_f2, R, x)) fl |= 2u;
                const f2 xi{A.xi_f2.hi, A.xi_f2.lo};
#pragma unroll
                for (int r = 0; r < NC; ++r) {
                    if constexpr (QR) h[r] = sH[r * kTile + lane];
                    out[r] = (T)(x[r].hi + x[r].lo);
                    const f2 ps = f2_add(f2_mul(xi, x[r]), h[r]);
                    psi[r] = (T)(ps.hi + ps.lo);
                }
            } else {
                double K[3][3], Hs[3][3];
#pragma unroll
                for (int a = 0; a < DIM; ++a)
#pragma unroll
                    for (int b = 0; b < DIM; ++b)
                        K[a][b] = 2.0 * (double)buf[(S.kn + a * DIM + b) * kTile + lane] -
                                  (double)buf[(S.km + a * DIM + b) * kTile + lane];
                const double* sH = reinterpret_cast<const double*>(sR_raw);
                double h[NC], x[NC];
#pragma unroll
                for (int r = 0; r < NC; ++r) {
                    h[r] = sH[r * kTile + lane];
                    Hs[Packed<DIM>::I(r)][Packed<DIM>::J(r)] = h[r];
                    Hs[Packed<DIM>::J(r)][Packed<DIM>::I(r)] = h[r];
                }
#pragma unroll
                for (int r = 0; r < NC; ++r) {
                    const int i = Packed<DIM>::I(r), j = Packed<DIM>::J(r);
                    double lh = -A.inv_wi * Hs[i][j];
#pragma unroll
                    for (int l = 0; l < DIM; ++l) lh = fma(K[i][l], Hs[l][j], fma(Hs[i][l], K[j][l], lh));
                    const double pn = (double)buf[(S.sig + r) * kTile + lane];
                    const double pm = (double)buf[(S.sig + NC + r) * kTile + lane];
                    x[r] = (2.0 * pn - 0.5 * pm) + A.dt * lh + A.dt * A.G * A.g * (K[i][j] + K[j][i]);
                    if constexpr (TRANSPORT) x[r] -= (double)buf[(S.tr + r) * kTile + lane];
                }
                double M[NC][NC];
                assemble_M<DIM>(K, A.a, A.dt * A.xi, M);
                if (!gauss_pp<NC>(M, x, 1e-300)) fl |= 2u;
#pragma unroll
                for (int r = 0; r < NC; ++r) {
                    out[r] = (T)x[r];
                    psi[r] = (T)fma(A.xi, x[r], h[r]);
                }
            }
        } else if constexpr (F32) {
            f2 K[3][3];
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
                for (int b = 0; b < DIM; ++b)
                    K[a][b] = two_sum_f2(2.0f * kn_at(a * DIM + b), -km_at(a * DIM + b));
            const f2* sR = reinterpret_cast<const f2*>(sR_raw);
            f2 R[NC], x[NC];
#pragma unroll
            for (int r = 0; r < NC; ++r) R[r] = sR[r * kTile + lane];
            if (!solve_point_f32<DIM>(K, A.a_f2, A.dt_f2, R, x)) fl |= 2u;
#pragma unroll
            for (int r = 0; r < NC; ++r) out[r] = (T)(x[r].hi + x[r].lo);
        } else {
            double K[3][3];
#pragma unroll
            for (int a = 0; a < DIM; ++a)
#pragma unroll
                for (int b = 0; b < DIM; ++b)
                    K[a][b] = 2.0 * (double)buf[(S.kn + a * DIM + b) * kTile + lane] -
                              (double)buf[(S.km + a * DIM + b) * kTile + lane];
            const double* sR = reinterpret_cast<const double*>(sR_raw);
            double x[NC];
#pragma unroll
            for (int r = 0; r < NC; ++r) x[r] = sR[r * kTile + lane];
            double M[NC][NC];
            assemble_M<DIM>(K, A.a, A.dt, M);
            if (!gauss_pp<NC>(M, x, 1e-300)) fl |= 2u;
#pragma unroll
            for (int r = 0; r < NC; ++r) out[r] = (T)x[r];
        }
        bool finite = true;
#pragma unroll
        for (int r = 0; r < NC; ++r) {
            finite = finite && isfinite((double)out[r]);
            T s0r;
            if constexpr (QR) s0r = (T)s0_r[r];
            else s0r = has_s0 ? buf[(S.s0 + r) * kTile + lane] : (T)0;
            // the push-forward uses the stored value of sigma^{n+1}
            if constexpr (F32) sD[r * kTile + lane] = __fsub_rn((float)out[r], (float)s0r);
            else reinterpret_cast<double*>(sD)[r * kTile + lane] = (double)out[r] - (double)s0r;
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < NC; ++r) {
                A.sig_np1[(long long)r * N + p] = out[r];
                if constexpr (PAPER) {
                    finite = finite && isfinite((double)psi[r]);
                    A.psi[(long long)r * N + p] = psi[r];
                    if (A.sig_copy) A.sig_copy[(long long)r * N + p] = psi[r];
                } else {
                    if (A.sig_copy) A.sig_copy[(long long)r * N + p] = out[r];
                }
            }
            if (!finite) fl |= 1u;
            if (fl) atomicOr(A.flags, fl);
        }
    }
    __syncthreads();

    // ---- (a6) push-forward of the modes over the oldest level
    if (!classic && active) {
        const T* qv = buf + ((m * NC + w) * kTile + lane);
        // row j NC + c of this tile's block in the tile-major level
        T* out = A.modes_nm1 + mode_index(p, w, m * NC);
        constexpr long long stride = (long long)NC * kTile;
        if constexpr (QR) {
            float d[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) d[cc] = sD[(w + cc * W) * kTile + lane];
#pragma unroll
            for (int j = 0; j < kQR; ++j) {
                if (j < m) {
                    const float rho = A.mc.rho[j], cj = A.mc.c[j];
#pragma unroll
                    for (int cc = 0; cc < CPW; ++cc)
                        __stcs(out + j * stride + (long long)cc * W * kTile, __fmaf_rn(rho, d[cc], -cj * qr[cc][j]));
                }
            }
        } else if constexpr (F32) {
            float d[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) d[cc] = sD[(w + cc * W) * kTile + lane];
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const float rho = A.mc.rho[j], cj = A.mc.c[j];
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc)
                    __stcs(out + j * stride + (long long)cc * W * kTile,
                           __fmaf_rn(rho, d[cc], -cj * qv[(j * NC + cc * W) * kTile]));
            }
        } else {
            double d[CPW];
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) d[cc] = reinterpret_cast<const double*>(sD)[(w + cc * W) * kTile + lane];
#pragma unroll 2
            for (int j = 0; j < m; ++j)
#pragma unroll
                for (int cc = 0; cc < CPW; ++cc)
                    __stcs(out + j * stride + (long long)cc * W * kTile,
                           (T)fma(A.mc.rho[j], d[cc], -A.mc.c[j] * (double)qv[(j * NC + cc * W) * kTile]));
        }
    }
}

// Persistent step kernel.  Tiles are staged either by TMA (tp.on: one thread
// issues tensor-map copies that complete on mbarriers; every wait is bounded
// and a wait that gives up latches TFS_FLAG_TIMEOUT) or by cp.async (any grid).
// Two stage buffers double-buffer whole tiles; with one, the next tile's
// level-n mode planes are fetched as soon as the current tile has read its
// own (after its history sums) and the rest after its push-forward.  One loop
// serves every variant, so that the tile code is instantiated once.
template <typename T, int DIM, bool TRANSPORT, bool COMP, bool PAPER, bool QR>
__global__ void __launch_bounds__(32 * StepShape<DIM>::W, 4)
fwd_kernel(const FwdArgs<T> A, const __grid_constant__ TmaPlan tp, const int classic, const long long num_tiles,
           const int stages, const int vec16) {
    constexpr int NC = Packed<DIM>::NC;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) double sR_store[NC * kTile];       // R per (component, point): double or f2
    __shared__ __align__(16) double sD_store[NC * kTile];       // sigma^{n+1} - sigma0 (float or double)
    __shared__ __align__(8) uint64_t bars[2][2];                // TMA: [stage buffer][early, late]
    const StageMap S = stage_map<DIM>(classic ? 0 : A.m, TRANSPORT, A.sigma0 != nullptr, classic != 0 || PAPER);
    const size_t stage_elems = (size_t)S.planes * kTile;
    // stage buffers start on a 128-byte boundary (TMA destination)
    T* buf0 = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(smem) + 127) & ~uintptr_t(127));
    T* buf1 = buf0 + stage_elems;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int nthr = 32 * StepShape<DIM>::W;
    float* sD = reinterpret_cast<float*>(sD_store);
    const bool use_tma = tp.on != 0;
    const bool v16 = vec16 != 0;
    const int mnc = (classic ? 0 : A.m) * NC;
    const bool has_s0 = A.sigma0 != nullptr;
    const bool two = stages == 2;

    if (use_tma) {
        if (tid == 0) {
            mbar_init(&bars[0][0], 1);
            mbar_init(&bars[0][1], 1);
            mbar_init(&bars[1][0], 1);
            mbar_init(&bars[1][1], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    // stage planes of tile t into buffer b: early = level-n mode planes, late = the rest
    auto issue = [&](int b, long long t, bool early, bool late) {
        T* dst = b ? buf1 : buf0;
        if (use_tma) {
            if (tid == 0)
                tma_issue<T, DIM, TRANSPORT>(A, tp, S, dst, t * kTile, mnc, has_s0, classic != 0 || PAPER, early, late,
                                             &bars[b][0], &bars[b][1]);
        } else {
            issue_planes<T, DIM>(A, S, dst, t * kTile, tid, nthr, v16, early ? 0 : mnc, late ? S.planes : mnc);
            cp_async_commit();
        }
    };
    // each TMA barrier completes one phase per tile staged in its buffer
    auto wait_tma = [&](int b, unsigned parity) -> bool {
        bool ok = true;
        if (mnc > 0) ok = mbar_wait(&bars[b][0], parity);
        return mbar_wait(&bars[b][1], parity) && ok;
    };

    long long tile = blockIdx.x;
    if (tile < num_tiles) issue(0, tile, true, true);
    for (int it = 0; tile < num_tiles; ++it, tile += gridDim.x) {
        const long long next = tile + gridDim.x;
        const int b = two ? (it & 1) : 0;
        if (two && next < num_tiles) issue(b ^ 1, next, true, true);
        if (use_tma) {
            const unsigned parity = two ? ((unsigned)(it >> 1) & 1u) : ((unsigned)it & 1u);
            const bool ok = wait_tma(b, parity);
            if (__syncthreads_or(!ok)) {
                // give up: flag it and let the copies still in flight land (bounded) before exiting
                if (tid == 0) atomicOr(A.flags, 8u);
                wait_tma(b, parity);
                if (two && next < num_tiles) wait_tma(b ^ 1, (unsigned)((it + 1) >> 1) & 1u);
                return;
            }
        } else {
            if (two && next < num_tiles) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncthreads();
        }
        // one buffer: the next tile's level-n mode planes as soon as the history
        // sums have read them (QR: the whole next tile), the rest after the push
        auto early = [&] {
            if (!two && next < num_tiles) issue(0, next, true, QR);
        };
        compute_tile<T, DIM, TRANSPORT, COMP, PAPER, QR>(A, S, b ? buf1 : buf0, tile * kTile, classic, sR_store,
                                                         sD, early);
        __syncthreads();
        if (!QR && !two && next < num_tiles) issue(0, next, false, true);
    }
    if (!use_tma) cp_async_wait<0>();
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Raises the dynamic shared-memory limit of transport_staged<T> once per
// device (the attribute belongs to the device's copy of the kernel).
template <typename T>
cudaError_t staged_smem_ready() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(transport_staged<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)StagedTile<T>::kSmemBytes);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template <typename T, int DIM, bool TRANSPORT, bool COMP, bool PAPER>
cudaError_t launch_one(const FwdArgs<T>& a, const LaunchCfg& cfg, cudaStream_t s) {
    constexpr int NC = Packed<DIM>::NC;
    constexpr bool kQRok = sizeof(T) == 4;
    cudaError_t e;
    auto kern = fwd_kernel<T, DIM, TRANSPORT, COMP, PAPER, false>;
    const long long num_tiles = (a.N + kTile - 1) / kTile;
    const bool levels = cfg.classic || PAPER;
    if (PAPER && (cfg.classic || !a.psi)) return cudaErrorInvalidValue;
    const StageMap S = stage_map<DIM>(cfg.classic ? 0 : a.m, TRANSPORT, a.sigma0 != nullptr, levels);
    const size_t stage_bytes = (size_t)S.planes * kTile * sizeof(T);
    const size_t static_bytes = 2 * NC * kTile * sizeof(double) + 32;
    PersistPlan plan;
    e = persistent_plan(reinterpret_cast<const void*>(kern), 32 * StepShape<DIM>::W, stage_bytes, static_bytes, 2,
                        &plan);
    if (e != cudaSuccess) return e;
    if (TRANSPORT) {
        if (!a.trans) return cudaErrorInvalidValue;
        // the transported field: sigma, or Psi in the paper's variable
        FwdArgs<T> ta = a;
        if (PAPER) {
            if (!a.psi_n || !a.psi_nm1) return cudaErrorInvalidValue;
            ta.sig_n = a.psi_n;
            ta.sig_nm1 = a.psi_nm1;
        }
        if (a.n0 % kTX == 0 && a.n1 % kTY == 0) {
            // z planes per block: 16 for the staged kernel (measured at 256^3 with 3 blocks per SM:
            // 0.39 ms against 0.45 with 8), 8 for the plain one
            const int zs = 16, zt = 8;
            const dim3 block(kTX, kTY);
            bool staged = false;
            if constexpr (DIM == 3) {
                staged = (long long)a.n0 * a.n1 < (1ll << 31) && aligned16(ta.sig_n) && aligned16(ta.sig_nm1) &&
                         aligned16(ta.u) &&
                         (!ta.halo_lo || (aligned16(ta.halo_lo) && aligned16(ta.halo_hi)));
                if (staged) {
                    e = staged_smem_ready<T>();
                    if (e != cudaSuccess) return e;
                    const dim3 grid(a.n0 / kTX, a.n1 / kTY, (a.n2 + zs - 1) / zs);
                    transport_staged<T><<<grid, block, StagedTile<T>::kSmemBytes, s>>>(ta, cfg.stencil, zs);
                }
            }
            if (!staged) {
                const dim3 grid(a.n0 / kTX, a.n1 / kTY, DIM == 3 ? (a.n2 + zt - 1) / zt : 1);
                transport_tiled<T, DIM><<<grid, block, 0, s>>>(ta, cfg.stencil, zt);
            }
        } else {
            const int threads = 256;
            long long blocks = (a.N + threads - 1) / threads;
            if (blocks > (long long)plan.sms * 16) blocks = (long long)plan.sms * 16;
            transport_kernel<T, DIM><<<(unsigned)blocks, threads, 0, s>>>(ta, cfg.stencil);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // one stage buffer per block: the variant that keeps Q_j in registers
    // refills the whole buffer right after the history sums
    bool qr = false;
    if constexpr (kQRok) {
        if (!cfg.classic && a.m <= kQR && plan.stages == 1) {
            PersistPlan qp;
            e = persistent_plan(reinterpret_cast<const void*>(fwd_kernel<T, DIM, TRANSPORT, COMP, PAPER, true>),
                                32 * StepShape<DIM>::W, stage_bytes, static_bytes, 1, &qp);
            if (e != cudaSuccess) return e;
            if (qp.stages * qp.per_sm >= plan.stages * plan.per_sm) {
                qr = true;
                plan = qp;
            }
        }
    }
    const int stages = plan.stages;
    const size_t dyn = plan.dyn;
    long long grid = (long long)plan.per_sm * plan.sms;
    if (grid > num_tiles) grid = num_tiles;
    if (grid < 1) grid = 1;
    const int vec16 = (a.N % (16 / (long long)sizeof(T))) == 0;
    // tensor maps of every staged plane group; any refusal selects cp.async
    TmaPlan tp;
    memset(&tp, 0, sizeof(tp));
    {
        const bool dbl = sizeof(T) == 8;
        bool ok = a.N < (1ll << 31);
        ok = ok && encode_plane_map(&tp.kn, a.kap_n, a.N, DIM * DIM, DIM * DIM, dbl) &&
             encode_plane_map(&tp.km, a.kap_nm1, a.N, DIM * DIM, DIM * DIM, dbl);
        if (ok && TRANSPORT) ok = encode_plane_map(&tp.tr, a.trans, a.N, NC, NC, dbl);
        if (ok && a.sigma0) ok = encode_plane_map(&tp.s0, a.sigma0, a.N, NC, NC, dbl);
        if (ok && levels)
            ok = encode_plane_map(&tp.sn, a.sig_n, a.N, NC, NC, dbl) &&
                 encode_plane_map(&tp.sm, a.sig_nm1, a.N, NC, NC, dbl);
        tp.on = ok ? 1 : 0;
    }
    if (cfg.ev_before) {
        e = cudaEventRecord(cfg.ev_before, s);
        if (e != cudaSuccess) return e;
    }
    if (qr)
        fwd_kernel<T, DIM, TRANSPORT, COMP, PAPER, kQRok><<<dim3((unsigned)grid), dim3(32, StepShape<DIM>::W), dyn, s>>>(
            a, tp, 0, num_tiles, stages, vec16);
    else
        kern<<<dim3((unsigned)grid), dim3(32, StepShape<DIM>::W), dyn, s>>>(a, tp, cfg.classic ? 1 : 0, num_tiles,
                                                                           stages, vec16);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (cfg.ev_after) e = cudaEventRecord(cfg.ev_after, s);
    return e;
}

template <typename T, bool COMP>
cudaError_t dispatch(const FwdArgs<T>& a, const LaunchCfg& cfg, cudaStream_t s) {
    if (cfg.paper) {
        if (cfg.dim == 2)
            return cfg.transport ? launch_one<T, 2, true, COMP, true>(a, cfg, s)
                                 : launch_one<T, 2, false, COMP, true>(a, cfg, s);
        return cfg.transport ? launch_one<T, 3, true, COMP, true>(a, cfg, s) : launch_one<T, 3, false, COMP, true>(a, cfg, s);
    }
    if (cfg.dim == 2)
        return cfg.transport ? launch_one<T, 2, true, COMP, false>(a, cfg, s)
                             : launch_one<T, 2, false, COMP, false>(a, cfg, s);
    return cfg.transport ? launch_one<T, 3, true, COMP, false>(a, cfg, s) : launch_one<T, 3, false, COMP, false>(a, cfg, s);
}

}  // namespace

cudaError_t launch_forward_f64(const FwdArgs<double>& a, const LaunchCfg& cfg, cudaStream_t s) {
    return dispatch<double, false>(a, cfg, s);
}

cudaError_t launch_forward_f32(const FwdArgs<float>& a, const LaunchCfg& cfg, cudaStream_t s) {
    return cfg.compensated ? dispatch<float, true>(a, cfg, s) : dispatch<float, false>(a, cfg, s);
}

}  // namespace tfs
