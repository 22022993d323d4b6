// Internal declarations shared by the host API and the kernels of libtfs.
// Not part of the public ABI (see include/tfs.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tfs {

constexpr int kMaxModes = 64;
constexpr double kB0 = 1.5, kB1 = -2.0, kB2 = 0.5;   // BDF2 (Section 4.1)

// Storage of the forward mode levels, tile-major: the m nc rows (row j nc + c
// for mode j, component c) of the 32 consecutive points of tile p / 32 are
// contiguous, so that one tile's level is one contiguous block of m nc 32
// elements (a single bulk copy, and one DRAM stream instead of m nc of them);
// a level spans ceil(N / 32) whole tiles, the points past N being padding.
constexpr int kModeTile = 32;
__host__ __device__ __forceinline__ long long mode_index(long long p, int row, int rows) {
    return ((p >> 5) * rows + row) * kModeTile + (p & 31);
}
__host__ __device__ __forceinline__ long long mode_points(long long N) {
    return (N + kModeTile - 1) / kModeTile * kModeTile;
}

// Per-mode constants of the BDF2 push-forward (eq. BDF_Phi_k_n+1):
// c_j = 1/(b0 + mu_j dt), rho_j = w_j dt c_j, eta_j = mu_j dt c_j.
// The float copies carry a hi/lo split of eta_j for the compensated mode sum.
struct ModeConstsD {
    double c[kMaxModes], rho[kMaxModes], eta[kMaxModes];
};
struct ModeConstsF {
    float c[kMaxModes], rho[kMaxModes], eta_hi[kMaxModes], eta_lo[kMaxModes];
};

template <typename T> struct ModeConsts;
template <> struct ModeConsts<double> { using type = ModeConstsD; };
template <> struct ModeConsts<float> { using type = ModeConstsF; };

// A double scalar split into two floats, hi + lo (double-float arithmetic).
struct F2c {
    float hi, lo;
};

// Arguments of one forward step launch.  Field pointers follow the layouts of
// include/tfs.h; the mode levels are tile-major (mode_index).
template <typename T>
struct FwdArgs {
    const T* kap_n;        // [d*d][N]
    const T* kap_nm1;      // [d*d][N]
    const T* u;            // [d][N] (transport only)
    const T* sigma0;       // [nc][N] or nullptr for zero
    const T* sig_n;        // [nc][N]
    const T* sig_nm1;      // [nc][N]
    T* sig_np1;            // [nc][N]
    T* sig_copy;           // optional second destination of sigma^{n+1}
    T* trans;              // [nc][N] transport term A: written by the pre-pass, read by the step
    const T* modes_n;      // tile-major mode level n (mode_index)
    T* modes_nm1;          // level n-1, overwritten with level n+1
    unsigned* flags;       // latched device status
    long long N;
    int n0, n1, n2;
    int m;
    double dt, eta, a, G, g, eps;   // eta, a = eta + dt/Wi, G, g = g_alpha(t_{n+1})
    double inv_h[3];
    double courant_coef;   // per-point Courant number = coef * sum_a |u_a| / h_a (0: no check)
    double courant_limit;
    // double-float copies of the step scalars (FP32 storage modes)
    F2c eta_f2, a_f2, dt_f2, src_f2;   // src = dt G g
    typename ModeConsts<T>::type mc;
    // the paper's own variable (Section 3.4): sig_* hold the levels of Phi, g holds
    // Psi0^{n+1}, a = b0 + dt xi/Wi, mc holds c_j, dt c_j, w_j mu_j c_j; psi receives
    // the stress Psi^{n+1} = xi Phi^{n+1} + h
    T* psi;                // [nc][N]
    const T* psi_n;        // Psi^n, Psi^{n-1}: the transported field of this variable
    const T* psi_nm1;
    double xi, inv_wi;
    F2c xi_f2, dtxi_f2;    // xi, dt xi
    // slab of a larger periodic domain along the slowest axis (z in 3D, y in
    // 2D): the stencil's neighbours beyond the slab come from the neighbouring
    // slabs' boundary planes, [2 levels][nc][R][plane] (level 0 sigma^n, 1
    // sigma^{n-1}; R = halo_r planes of n0 (2D) or n0 n1 (3D) points; halo_lo
    // plane k is slab coordinate k - R, halo_hi plane k is n_s + k); both
    // nullptr: the slowest axis wraps periodically within the grid
    const T* halo_lo;
    const T* halo_hi;
    int halo_r;
};

// Tensor maps of the per-point plane groups a tile stages, each a 2D view
// [planes][N] (x = point, y = plane) with a box of 32 points; `on` = 0 selects
// the cp.async path (grids whose N * element size is not a multiple of 16
// bytes, or unaligned fields).  The tile-major mode levels need no map: each
// tile's level is one contiguous block, fetched by untiled bulk copies.
struct TmaPlan {
    CUtensorMap kn, km;         // velocity gradient levels [d*d]
    CUtensorMap tr, s0;         // transport term, initial stress [nc]
    CUtensorMap sn, sm;         // stress levels n, n-1 [nc] (alpha = 1)
    int on;
};

// Host: encode a [planes][N] tensor map with a box of 32 x box_h (false if the
// layout does not allow one).
bool encode_plane_map(CUtensorMap* map, const void* base, long long N, int planes, int box_h, bool dbl);

// Launch shape of a persistent tile kernel: stage buffers per block, resident
// blocks per SM, SM count and dynamic shared memory (stages * stage bytes +
// 128 bytes of alignment slack).  Computed once per kernel, device and stage
// size (the kernel's dynamic shared-memory limit is set then) and cached.
struct PersistPlan {
    int stages, per_sm, sms;
    size_t dyn;
};
cudaError_t persistent_plan(const void* kern, int threads, size_t stage_bytes, size_t static_bytes, int max_stages,
                            PersistPlan* out);

// Arguments of one step with implicit transport (tfs_implicit.cu).
template <typename T>
struct ImpArgs {
    const T* kap_n;
    const T* kap_nm1;
    const T* u;            // [d][N]
    const T* sigma0;       // [nc][N] or nullptr for zero
    const T* sig_n;
    const T* sig_nm1;
    T* sig_np1;
    T* sig_copy;           // optional second destination of sigma^{n+1}
    const T* modes_n;      // tile-major mode level n (mode_index)
    T* modes_nm1;          // level n-1 in; Q_j after the right-hand side; level n+1 out
    unsigned* flags;
    long long N;
    int dim, n0, n1, n2, m, stencil, classic;
    double dt, eta, a, G, g, eps;
    double inv_h[3];
    typename ModeConsts<T>::type mc;
    ModeConstsD mcd;
    F2c eta_f2, src_f2;
    double* kry;           // 10 vectors of nc N doubles (Krylov workspace)
    double* partials;      // reduction scratch, kImpBlocks doubles
    double tol;            // relative residual target
    int maxit;
    // the paper's variable (Section 3.4): the unknown is Phi^{n+1}, the operator's
    // transport acts on Psi^{n+1} = xi Phi + h, so dt above is dt xi (the transport
    // scale of the operator) and a = b0 + dt xi/Wi; g holds Psi0^{n+1}, mc the
    // per-mode constants c_j, dt c_j, w_j mu_j c_j; the right-hand side takes the
    // step's dt_rhs; psi receives Psi^{n+1}
    int paper;
    double dt_rhs, xi, inv_wi;
    T* psi;
};
constexpr int kImpBlocks = 1024;   // blocks of the implicit-step kernels (and reduction partials)

// FP32 section of the implicit-transport workspace (the inner solve of the
// mixed-precision Krylov scheme): tile-major float copies of the point blocks,
// the tap coefficients and the block inverses ((2 nc^2 + 4 d) per point over the
// points padded to whole 32-point tiles) and nine Krylov vectors (9 nc N),
// counted in doubles (rounded up), plus 16 for the section's 128-byte alignment.
__host__ __device__ __forceinline__ long long kry_float_doubles(int nc, int dim, long long N) {
    return ((2LL * nc * nc + 4LL * dim) * mode_points(N) + 9LL * nc * N + 1) / 2 + 16;
}

// host driver of one implicit step (BiCGStab, block-Jacobi preconditioned);
// synchronises `s`; returns the iterations used and the final relative residual
cudaError_t run_implicit_f64(const ImpArgs<double>& a, cudaStream_t s, int* iters, double* relres);
cudaError_t run_implicit_f32(const ImpArgs<float>& a, cudaStream_t s, bool compensated, int* iters, double* relres);

// First step t_0 -> t_1 by two-stage SDIRK2 (gamma = 1 - 1/sqrt2, stiffly
// accurate, L-stable; Section 5.1) on the mode ODEs
//   d sigma_j/dt = -mu_j sigma_j + w_j (sigma - sigma0),  sum_j d sigma_j/dt = F(sigma, t),
// each stage solving (dt W + dt/Wi) S - dt L(kappa^0) S [+ dt (u.grad - eps Lap) S]
//   = dt W sigma0 + dt sum_j mu_j Z_j / (1 + gamma mu_j dt) + dt G (kappa^0 + kappa^0T) g_alpha(t_i),
// W = sum_j w_j / (1 + gamma mu_j dt), Z_j the explicit part of the mode stage.
struct StartConsts {
    double mu[kMaxModes], w[kMaxModes];
    double inv_den[kMaxModes];   // 1 / (1 + gamma mu_j dt)
    double W, gam;
    double g[2];                 // g_alpha(gamma dt), g_alpha(dt)
};

// Arguments of the pointwise first step (transport off): level-0 fields in,
// sigma^1 and the level-1 modes out; all arithmetic in FP64.
template <typename T>
struct StartArgs {
    const T* kap0;         // [d*d][N]
    const T* sigma0;       // [nc][N] or nullptr for zero
    const T* modes0;       // tile-major mode level 0 (mode_index)
    T* modes1;             // level 1 (out)
    T* sig1;               // [nc][N] (out)
    T* sig_copy;           // optional second destination of sigma^1
    unsigned* flags;
    long long N;
    int m;
    double dt, a, G;       // a = dt W + dt/Wi (the paper's variable: 1 + gamma dt W/Wi)
    T* psi;                // the paper's variable: Psi^1 [nc][N] (out); sigma0 then points at Phi^0
    double inv_wi;
};

cudaError_t launch_start_point_f64(const StartArgs<double>& a, const StartConsts& c, int dim, cudaStream_t s);
cudaError_t launch_start_point_f32(const StartArgs<float>& a, const StartConsts& c, int dim, cudaStream_t s);
// the same first step in the paper's variable (c.g holds Psi0 at the two stage times)
cudaError_t launch_start_paper_f64(const StartArgs<double>& a, const StartConsts& c, int dim, cudaStream_t s);
cudaError_t launch_start_paper_f32(const StartArgs<float>& a, const StartConsts& c, int dim, cudaStream_t s);
// Adjoint of the pointwise SDIRK2 first step (transport off, zero initial modes):
// inputs the adjoints of sigma^1 (s1), of sigma^0 as the next step's level n-1
// (s0) and of the level-1 modes (z_j = b1 ell_prev + b2 ell_prev2); outputs the
// adjoint of sigma0 in s1_out (s0_out = 0), and adds dJ/dkappa^0 to g_kap and the
// per-block dJ/dWi, dJ/dbeta to partials[2 b], [2 b + 1] (b = point / 32).
template <typename T>
struct StartAdjArgs {
    const T* kap0;
    const T* sigma0;       // nullptr for zero
    const double* s1;
    const double* s0;
    const T* ell_prev;
    const T* ell_prev2;
    double* s1_out;
    double* s0_out;
    double* g_kap;
    double* partials;
    unsigned* flags;
    long long N;
    int m;
    double dt, a, G, Wi, Re;
};
cudaError_t launch_start_adjoint_f64(const StartAdjArgs<double>& a, const StartConsts& c, int dim, cudaStream_t s);
cudaError_t launch_start_adjoint_f32(const StartAdjArgs<float>& a, const StartConsts& c, int dim, cudaStream_t s);
// implicit transport: the two stage systems by the Krylov solver of the implicit step
// (a.a, a.kap_n = a.kap_nm1 = kappa^0 set by the caller); synchronises `s`;
// iterations summed and the larger relative residual of the two stages
cudaError_t run_start_implicit_f64(const ImpArgs<double>& a, const StartConsts& c, cudaStream_t s, int* iters,
                                   double* relres);
cudaError_t run_start_implicit_f32(const ImpArgs<float>& a, const StartConsts& c, cudaStream_t s, int* iters,
                                   double* relres);

struct LaunchCfg {
    int dim;
    int stencil;       // 0 upwind3, 1 central2
    bool transport;
    bool classic;      // alpha == 1
    bool compensated;  // FP32 compensated mode sum
    bool paper = false; // the paper's own variable (transport off only)
    cudaEvent_t ev_before = nullptr;   // recorded just before / after the step kernel
    cudaEvent_t ev_after = nullptr;    // (not around the transport pre-pass), if set
};

// forward launchers (tfs_forward.cu)
cudaError_t launch_forward_f64(const FwdArgs<double>& a, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_forward_f32(const FwdArgs<float>& a, const LaunchCfg& cfg, cudaStream_t s);

// Arguments of one adjoint step launch (see tfs_adjoint.cu).
template <typename T>
struct AdjArgs {
    const T* kap_n;        // [d*d][N] forward velocity gradient of the step
    const T* kap_nm1;
    const T* u;            // [d][N]
    const T* sig_np1;      // forward sigma^{n+1} of the step [nc][N]
    // adjoint stress state: s1 = adjoint of sigma^{n+1}, s0 = adjoint of the copied sigma^n
    const double* s1;      // [nc][N]
    const double* s0;      // [nc][N]
    double* s1_out;        // adjoint of sigma^n       (next step's s1)
    double* s0_out;        // adjoint of sigma^{n-1}   (next step's s0)
    double* lamR;          // [nc][N] scratch: adjoint of the right-hand side (for transport)
    // adjoint mode ring: ell_prev = lamQ of the previous adjoint step, ell_prev2 the one before
    const T* ell_prev;     // [m][nc][N]
    T* ell_prev2;          // [m][nc][N] read, then overwritten with this step's lamQ
    double* g_sigma0;      // [nc][N] accumulated
    double* g_kap;         // [d*d][N] accumulated (frozen gradient: coefficient +1)
    double* partials;      // [gridDim.x][2] per-block sums of dJ/dWi, dJ/dbeta
    unsigned* flags;
    long long N;
    int n0, n1, n2;
    int m;
    int first;             // 1 on the first adjoint step (no previous lamQ)
    double dt, eta, a, G, g, eps, Wi, Re;
    double inv_h[3];
    ModeConstsD mc;
    ModeConstsF mcf;       // float copies (FP32 storage: mode sweeps in float)
};

cudaError_t launch_adjoint_f64(const AdjArgs<double>& a, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_adjoint_f32(const AdjArgs<float>& a, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_adjoint_transport(const AdjArgs<double>& a, const void* u, bool u_is_double,
                                     const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_reduce_partials(const double* partials, int count, double* out2, cudaStream_t s);

// small utility kernels (tfs_util.cu)
cudaError_t launch_fill_levels(void* sig_n, void* sig_nm1, void* sigma0_copy, const void* sigma0,
                               long long count, bool is_double, cudaStream_t s);
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s);
cudaError_t launch_write_header(uint64_t* dst, const uint64_t* words, int count, cudaStream_t s);
cudaError_t launch_to_double(const void* src, double* dst, long long count, bool is_double, cudaStream_t s);
cudaError_t launch_add_initial(double* g_sigma0, const double* s1, const double* s0, long long count,
                               cudaStream_t s);

}  // namespace tfs
