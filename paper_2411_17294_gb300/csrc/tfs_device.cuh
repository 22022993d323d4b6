// Device-side building blocks of the stress step: packed component tables,
// the per-point upper-convected operator, the small dense solve, and the
// periodic stencil.  Used by tfs_forward.cu and tfs_adjoint.cu.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "tfs_internal.h"

namespace tfs {

// Compile-time loop: calls f(std::integral_constant<int, I>) for I in [B, E).
// Keeps every array index a constant so small matrices stay in registers.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

template <int DIM> struct Packed;
// 2D packed order (xx, xy, yy)
template <> struct Packed<2> {
    static constexpr int NC = 3;
    __host__ __device__ static constexpr int I(int c) { return c == 0 ? 0 : (c == 1 ? 0 : 1); }
    __host__ __device__ static constexpr int J(int c) { return c == 0 ? 0 : (c == 1 ? 1 : 1); }
};
// 3D packed order (xx, yy, zz, yz, xz, xy)
template <> struct Packed<3> {
    static constexpr int NC = 6;
    __host__ __device__ static constexpr int I(int c) {
        return c == 0 ? 0 : c == 1 ? 1 : c == 2 ? 2 : c == 3 ? 1 : c == 4 ? 0 : 0;
    }
    __host__ __device__ static constexpr int J(int c) {
        return c == 0 ? 0 : c == 1 ? 1 : c == 2 ? 2 : c == 3 ? 2 : c == 4 ? 2 : 1;
    }
};

// Entry (r, k) of the packed matrix of  S -> kappa S + S kappa^T, i.e. the
// r-th packed component of kappa E_k + E_k kappa^T where E_k is the symmetric
// unit matrix of packed component k.  All index tests fold at compile time
// once the loops over r and k are unrolled.
template <int DIM, typename R>
__device__ __forceinline__ R uc_entry(const R K[3][3], int r, int k) {
    const int ro = Packed<DIM>::I(r), so = Packed<DIM>::J(r);
    const int i = Packed<DIM>::I(k), j = Packed<DIM>::J(k);
    R v = R(0);
    // (kappa E)_{ro,so} = sum_l K[ro][l] E[l][so];  (E kappa^T)_{ro,so} = sum_l E[ro][l] K[so][l]
    // E[l][s] = 1 for (l,s) in {(i,j), (j,i)}
    if (so == j) v += K[ro][i];
    if (i != j && so == i) v += K[ro][j];
    if (ro == i) v += K[so][j];
    if (i != j && ro == j) v += K[so][i];
    return v;
}

// M = a I - dt L(kappa) in packed coordinates.
template <int DIM>
__device__ __forceinline__ void assemble_M(const double K[3][3], double a, double dt,
                                           double M[Packed<DIM>::NC][Packed<DIM>::NC]) {
    constexpr int NC = Packed<DIM>::NC;
    static_for<0, NC>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        static_for<0, NC>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            const double l = uc_entry<DIM>(K, r, k);
            M[r][k] = (r == k) ? fma(-dt, l, a) : -dt * l;
        });
    });
}

// In-place Gaussian elimination with partial pivoting on a small dense system.
// Pivot search by compare-and-swap (no dynamic register indexing): the largest
// |entry| of column k among rows k.. ends up in row k, ties keep the earlier row.
// Returns false when a pivot is not larger than `tiny`.
template <int NC>
__device__ __forceinline__ bool gauss_pp(double M[NC][NC], double x[NC], double tiny) {
    bool ok = true;
    static_for<0, NC>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const bool sw = fabs(M[i][k]) > fabs(M[k][k]);
            static_for<k, NC>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                const double t0 = M[k][j], t1 = M[i][j];
                M[k][j] = sw ? t1 : t0;
                M[i][j] = sw ? t0 : t1;
            });
            const double t0 = x[k], t1 = x[i];
            x[k] = sw ? t1 : t0;
            x[i] = sw ? t0 : t1;
        });
        ok = ok && (fabs(M[k][k]) > tiny);
        const double inv = 1.0 / M[k][k];
        M[k][k] = inv;     // keep the reciprocal for back substitution
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const double f = M[i][k] * inv;
            static_for<k + 1, NC>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                M[i][j] = fma(-f, M[k][j], M[i][j]);
            });
            x[i] = fma(-f, x[k], x[i]);
        });
    });
    static_for<0, NC>([&](auto rr) {
        constexpr int i = NC - 1 - decltype(rr)::value;
        double acc = x[i];
        static_for<i + 1, NC>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            acc = fma(-M[i][j], x[j], acc);
        });
        x[i] = acc * M[i][i];
    });
    return ok;
}

// gauss_pp on NR right-hand sides at once (the columns of X): the elimination
// of M runs once, and every column goes through exactly the operations that
// gauss_pp applies to a single right-hand side, so each solution is bitwise
// that of gauss_pp.  Returns false when a pivot is not larger than `tiny`.
template <int NC, int NR>
__device__ __forceinline__ bool gauss_pp_multi(double M[NC][NC], double X[NC][NR], double tiny) {
    bool ok = true;
    static_for<0, NC>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const bool sw = fabs(M[i][k]) > fabs(M[k][k]);
            static_for<k, NC>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                const double t0 = M[k][j], t1 = M[i][j];
                M[k][j] = sw ? t1 : t0;
                M[i][j] = sw ? t0 : t1;
            });
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const double t0 = X[k][r], t1 = X[i][r];
                X[k][r] = sw ? t1 : t0;
                X[i][r] = sw ? t0 : t1;
            }
        });
        ok = ok && (fabs(M[k][k]) > tiny);
        const double inv = 1.0 / M[k][k];
        M[k][k] = inv;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const double f = M[i][k] * inv;
            static_for<k + 1, NC>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                M[i][j] = fma(-f, M[k][j], M[i][j]);
            });
#pragma unroll
            for (int r = 0; r < NR; ++r) X[i][r] = fma(-f, X[k][r], X[i][r]);
        });
    });
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        static_for<0, NC>([&](auto rr) {
            constexpr int i = NC - 1 - decltype(rr)::value;
            double acc = X[i][r];
            static_for<i + 1, NC>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                acc = fma(-M[i][j], X[j][r], acc);
            });
            X[i][r] = acc * M[i][i];
        });
    }
    return ok;
}

// FP32 LU factorisation with partial pivoting by compare-and-swap on whole
// rows (the multipliers move with their rows), recording every swap decision so
// that the factors can be applied to further right-hand sides:  P M = L U.
// The diagonal keeps 1/u_kk.  Returns false when a pivot is not above `tiny`.
template <int NC>
struct LU32 {
    float a[NC][NC];
    bool sw[NC][NC];   // sw[k][i]: rows k and i exchanged at elimination step k (i > k)
};

template <int NC>
__device__ __forceinline__ bool lu32_factor(LU32<NC>& F, float tiny) {
    bool ok = true;
    static_for<0, NC>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const bool sw = fabsf(F.a[i][k]) > fabsf(F.a[k][k]);
            F.sw[k][i] = sw;
            static_for<0, NC>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                const float t0 = F.a[k][j], t1 = F.a[i][j];
                F.a[k][j] = sw ? t1 : t0;
                F.a[i][j] = sw ? t0 : t1;
            });
        });
        ok = ok && (fabsf(F.a[k][k]) > tiny);
        const float inv = 1.0f / F.a[k][k];
        F.a[k][k] = inv;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const float f = F.a[i][k] * inv;
            F.a[i][k] = f;                     // multiplier of L
            static_for<k + 1, NC>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                F.a[i][j] = __fmaf_rn(-f, F.a[k][j], F.a[i][j]);
            });
        });
    });
    return ok;
}

// FP32 LU without row exchanges, for matrices that are strictly diagonally
// dominant by rows (Gaussian elimination is then stable without pivoting);
// the swap flags are cleared so that lu32_solve applies no permutation.
template <int NC>
__device__ __forceinline__ bool lu32_factor_nopivot(LU32<NC>& F, float tiny) {
    bool ok = true;
    static_for<0, NC>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            F.sw[k][i] = false;
        });
        ok = ok && (fabsf(F.a[k][k]) > tiny);
        const float inv = 1.0f / F.a[k][k];
        F.a[k][k] = inv;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const float f = F.a[i][k] * inv;
            F.a[i][k] = f;
            static_for<k + 1, NC>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                F.a[i][j] = __fmaf_rn(-f, F.a[k][j], F.a[i][j]);
            });
        });
    });
    return ok;
}

template <int NC>
__device__ __forceinline__ bool row_dominant(const LU32<NC>& F) {
    bool dom = true;
    static_for<0, NC>([&](auto rr) {
        constexpr int r = decltype(rr)::value;
        float off = 0.0f;
        static_for<0, NC>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            if (k != r) off += fabsf(F.a[r][k]);
        });
        dom = dom && (fabsf(F.a[r][r]) > off);
    });
    return dom;
}

// x <- M^{-1} x with the factors of lu32_factor (permutation, then L, then U).
template <int NC>
__device__ __forceinline__ void lu32_solve(const LU32<NC>& F, float x[NC]) {
    static_for<0, NC>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            const float t0 = x[k], t1 = x[i];
            x[k] = F.sw[k][i] ? t1 : t0;
            x[i] = F.sw[k][i] ? t0 : t1;
        });
    });
    static_for<0, NC>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        static_for<k + 1, NC>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            x[i] = __fmaf_rn(-F.a[i][k], x[k], x[i]);
        });
    });
    static_for<0, NC>([&](auto rr) {
        constexpr int i = NC - 1 - decltype(rr)::value;
        float acc = x[i];
        static_for<i + 1, NC>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            acc = __fmaf_rn(-F.a[i][j], x[j], acc);
        });
        x[i] = acc * F.a[i][i];
    });
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, ~44-bit
// significand, built from the error-free transformations TwoSum (Knuth) and
// TwoProd (exact product by FMA).  Used to assemble the right-hand side and the
// refinement residual of the point system in FP32 storage mode without the
// FP64 pipe.
struct f2 {
    float hi, lo;
};

__device__ __forceinline__ f2 f2_from(float a) { return {a, 0.0f}; }

__device__ __forceinline__ f2 two_sum_f2(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ f2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    const f2 s = two_sum_f2(a.hi, b.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, lo);
}

__device__ __forceinline__ f2 f2_add_f(f2 a, float b) {
    const f2 s = two_sum_f2(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ f2 f2_mul_f(f2 a, float b) {
    f2 p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, sm_80+).
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// 16-byte asynchronous copy global -> shared; bytes beyond src_bytes are zero.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Tensor-map (TMA) copies global -> shared that complete on an mbarrier.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes initialised mbarriers visible to the asynchronous proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// orders this thread's earlier shared-memory accesses (and, after a barrier,
// those of the block) before its later asynchronous-proxy copies
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the completion of phase `parity` of `bar`.  Bounded: gives up
// (returns false) after 2^24 tries or 2 s, whichever comes first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned i = 0; i < (1u << 24); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// Tiled 2D copy of the tensor map's box at (x, y) into shared memory; the
// transferred bytes are counted on `bar`.  The map must live in kernel
// parameter (__grid_constant__), constant or global memory.
// Untiled bulk copy global -> shared (cp.async.bulk): both addresses 16-byte
// aligned and `bytes` a multiple of 16; completion counted on the mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Periodic neighbour index along axis `ax` at offset `off` (|off| <= 2) from
// point (x, y, z); correct for any axis length >= 1.
struct GridIdx {
    long long n0, n1, n2;
    long long x, y, z;
    __device__ __forceinline__ static long long wrap(long long v, long long n) {
        if (v < 0) v += n;
        if (v < 0) v += n;
        if (v >= n) v -= n;
        if (v >= n) v -= n;
        return v;
    }
    __device__ __forceinline__ long long at(int ax, int off) const {
        const long long xx = ax == 0 ? wrap(x + off, n0) : x;
        const long long yy = ax == 1 ? wrap(y + off, n1) : y;
        const long long zz = ax == 2 ? wrap(z + off, n2) : z;
        return xx + n0 * (yy + n1 * zz);
    }
};

// two-sum of a and b (Knuth): s + e == a + b exactly.  __fadd_rn/__fsub_rn are
// never contracted into FMAs.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(double v) { return v; }

}  // namespace tfs
