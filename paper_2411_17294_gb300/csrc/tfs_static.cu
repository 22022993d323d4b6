// tfs_run_static: a run of the stress step whose state needs no allocation.
//
// Some callers cannot allocate device memory: code running where cudaMalloc is
// not allowed (inside a host framework that owns all device memory, a real-time
// loop that must not allocate, a plug-in without access to an allocator).  For
// them this entry point keeps the whole step state -- the stress ring, the
// initial-stress copy, the transport term, the status word and both mode
// levels -- in one
// file-scope device array of fixed size, kStaticBytes, instead of a
// caller-bound workspace.  The caller passes only inputs and the output.
//
// The array is part of the library image: every GPU that loads libtfs.so holds
// it until the process exits.  In host code its name only stands for the
// array; the device address is looked up with cudaGetSymbolAddress once per
// device and context (on the first call with that device current, and again
// when the current context is a different one, e.g. after cudaDeviceReset)
// and cached.  That first call on a device must therefore come before any
// stream capture.  All calls share the one array and each call starts by
// clearing what must start at zero (modes, flags) and writing the initial
// stress, so calls that overlap on the GPU (different streams, or host
// threads) race and must not be issued.  The status word the step kernels
// latch (non-finite result, singular point system, Courant limit, a bounded
// wait that gave up) stays in the array after the call; tfs_static_status
// reads it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <utility>

#include "../../include/tfs.h"
#include "tfs_internal.h"

using namespace tfs;

namespace {

constexpr size_t kStaticBytes = (size_t)64 << 20;   // 64 MiB
constexpr size_t kAlignS = 256;

__device__ __align__(256) unsigned char g_static_state[kStaticBytes];

constexpr int kMaxDevices = 64;
void* g_static_addr[kMaxDevices] = {};
unsigned long long g_static_ctx[kMaxDevices] = {};   // context the cached address belongs to
std::mutex g_static_mutex;

size_t up256(size_t v) { return (v + kAlignS - 1) / kAlignS * kAlignS; }

// Unique id of the calling thread's current CUDA context (0: none current, or
// the driver does not offer the query).  Context ids are never reused, so a
// cached address whose id differs from the current one belongs to a context
// that no longer exists (cudaDeviceReset) or to another one.
unsigned long long current_context_id() {
    using CtxCur = CUresult (*)(CUcontext*);
    using CtxId = CUresult (*)(CUcontext, unsigned long long*);
    static const std::pair<CtxCur, CtxId> fns = [] {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa = cudaDriverEntryPointSymbolNotFound, qb = qa;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
            qa != cudaDriverEntryPointSuccess)
            a = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
            qb != cudaDriverEntryPointSuccess)
            b = nullptr;
        return std::pair<CtxCur, CtxId>(reinterpret_cast<CtxCur>(a), reinterpret_cast<CtxId>(b));
    }();
    if (!fns.first || !fns.second) return 0;
    CUcontext c = nullptr;
    if (fns.first(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    if (fns.second(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_static_state for the current device, looked up once per
// device and context.
cudaError_t static_base(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_static_addr[dev] || ctx == 0 || ctx != g_static_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_state);   // makes the device's primary context current
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
        g_static_ctx[dev] = current_context_id();
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

template <typename T>
void fill_step_args(FwdArgs<T>& a, long long N, const long long n[3], const double L[3], int m, double dt,
                    double eta, double Wi, double beta, double alpha, long long step) {
    a.N = N;
    a.n0 = (int)n[0];
    a.n1 = (int)n[1];
    a.n2 = (int)n[2];
    a.m = m;
    a.dt = dt;
    a.eta = eta;
    a.a = eta + dt / Wi;
    a.G = (1.0 - beta) / Wi;          // Re = 1
    a.eps = 0.0;
    for (int i = 0; i < 3; ++i) a.inv_h[i] = (double)n[i] / L[i];
    a.g = alpha == 1.0 ? 1.0 : std::pow((double)(step + 1) * dt, alpha - 1.0) / std::tgamma(alpha);
    auto split = [](double v) {
        F2c r;
        r.hi = (float)v;
        r.lo = (float)(v - (double)r.hi);
        return r;
    };
    a.eta_f2 = split(a.eta);
    a.a_f2 = split(a.a);
    a.dt_f2 = split(a.dt);
    a.src_f2 = split(a.dt * a.G * a.g);
}

}  // namespace

extern "C" int tfs_run_static(const tfs_grid* grid, double alpha, double Wi, double beta, int m, double dt,
                              int precision, const double* mu, const double* w, const void* sigma0,
                              const void* grad_u, const void* u, int steps, void* sigma_out, void* stream) {
    // ---- arguments (same ranges as tfs_create)
    if (!grid || (grid->dim != 2 && grid->dim != 3)) return TFS_ERR_ARG;
    if (!(alpha > 0.0 && alpha <= 1.0) || !(Wi > 0.0) || !std::isfinite(Wi) || !(beta >= 0.0 && beta < 1.0) ||
        !(dt > 0.0) || !std::isfinite(dt))
        return TFS_ERR_ARG;
    if (m < 0 || m > kMaxModes || (alpha == 1.0 && m != 0) || (alpha < 1.0 && m < 1)) return TFS_ERR_ARG;
    if (precision != TFS_FP64 && precision != TFS_FP32 && precision != TFS_FP32_PLAIN) return TFS_ERR_ARG;
    if (!grad_u || !sigma_out || steps < 0) return TFS_ERR_ARG;
    if (alpha < 1.0 && (!mu || !w)) return TFS_ERR_ARG;
    long long n[3] = {1, 1, 1};
    double L[3] = {1.0, 1.0, 1.0};
    long long N = 1;
    for (int ax = 0; ax < grid->dim; ++ax) {
        if (grid->n[ax] < 1 || !(grid->L[ax] > 0.0) || !std::isfinite(grid->L[ax])) return TFS_ERR_ARG;
        n[ax] = grid->n[ax];
        L[ax] = grid->L[ax];
        N *= n[ax];
    }
    const int nc = grid->dim == 2 ? 3 : 6;
    const size_t es = precision == TFS_FP64 ? 8 : 4;
    const size_t field = (size_t)nc * (size_t)N * es;
    const size_t modes = (size_t)m * (size_t)nc * (size_t)mode_points(N) * es;   // tile-major levels
    const size_t need = kAlignS + 5 * up256(field) + 2 * up256(modes);
    if (need > kStaticBytes) return TFS_ERR_TOOBIG;

    // ---- SOE constants (FP64, as tfs_set_soe)
    ModeConstsD mcd{};
    ModeConstsF mcf{};
    double eta = kB0;
    if (alpha < 1.0) {
        eta = 0.0;
        for (int j = 0; j < m; ++j) {
            if (!(mu[j] >= 0.0) || !(w[j] >= 0.0) || !std::isfinite(mu[j]) || !std::isfinite(w[j]))
                return TFS_ERR_ARG;
            const double c = 1.0 / (kB0 + mu[j] * dt);
            const double rho = w[j] * dt * c;
            const double et = mu[j] * dt * c;
            eta += kB0 * rho;
            mcd.c[j] = c;
            mcd.rho[j] = rho;
            mcd.eta[j] = et;
            mcf.c[j] = (float)c;
            mcf.rho[j] = (float)rho;
            mcf.eta_hi[j] = (float)et;
            mcf.eta_lo[j] = (float)(et - (double)mcf.eta_hi[j]);
        }
    }

    // ---- state in the static array
    void* base_v = nullptr;
    if (static_base(&base_v) != cudaSuccess) return TFS_ERR_CUDA;
    char* p = (char*)base_v;
    unsigned* flags = (unsigned*)p;
    p += kAlignS;
    char* s0copy = p;
    p += up256(field);
    char* sig[3];
    for (int i = 0; i < 3; ++i) {
        sig[i] = p;
        p += up256(field);
    }
    char* trans = p;
    p += up256(field);
    char* md[2];
    for (int i = 0; i < 2; ++i) {
        md[i] = p;
        p += up256(modes);
    }
    // Courant flag of the explicit transport: a point is flagged when
    // sum_a |u_a|/h_a exceeds U sum_a 1/h_a, U the velocity limit of
    // tfs_transport_limit for this table (host computation, no device memory)
    double ccoef = 0.0;
    if (u) {
        tfs_handle hh = nullptr;
        double U = 0.0;
        int rc = tfs_create(&hh, grid, alpha, Wi, beta, m, dt, precision);
        if (rc == TFS_OK && alpha < 1.0) rc = tfs_set_soe(hh, mu, w, m);
        if (rc == TFS_OK) rc = tfs_transport_limit(hh, &U);
        if (hh) tfs_destroy(hh);
        if (rc != TFS_OK) return rc;
        double sih = 0.0;
        for (int ax = 0; ax < grid->dim; ++ax) sih += (double)n[ax] / L[ax];
        ccoef = U > 0.0 ? 1.0 / (U * sih) : 1e300;
    }

    cudaStream_t s = (cudaStream_t)stream;
    const bool dbl = precision == TFS_FP64;
    cudaError_t e = launch_fill_levels(sig[0], sig[1], s0copy, sigma0, (long long)nc * N, dbl, s);
    if (e == cudaSuccess && modes > 0) e = launch_zero(md[0], modes, s);
    if (e == cudaSuccess && modes > 0) e = launch_zero(md[1], modes, s);
    if (e == cudaSuccess) e = launch_zero(flags, kAlignS, s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;

    LaunchCfg cfg;
    cfg.dim = grid->dim;
    cfg.stencil = TFS_STENCIL_UPWIND3;
    cfg.transport = u != nullptr;
    cfg.classic = alpha == 1.0;
    cfg.compensated = precision == TFS_FP32;
    const int mm = alpha == 1.0 ? 0 : m;
    int cur = 0, prev = 1, cur_mode = 0;
    for (long long step = 0; step < steps; ++step) {
        const int nxt = 3 - cur - prev;
        if (dbl) {
            FwdArgs<double> a{};
            fill_step_args(a, N, n, L, mm, dt, eta, Wi, beta, alpha, step);
            a.courant_coef = ccoef;
            a.courant_limit = 1.0;
            a.kap_n = (const double*)grad_u;
            a.kap_nm1 = (const double*)grad_u;
            a.u = (const double*)u;
            a.sigma0 = sigma0 ? (const double*)s0copy : nullptr;
            a.sig_n = (const double*)sig[cur];
            a.sig_nm1 = (const double*)sig[prev];
            a.sig_np1 = (double*)sig[nxt];
            a.sig_copy = nullptr;
            a.trans = (double*)trans;
            a.modes_n = (const double*)md[cur_mode];
            a.modes_nm1 = (double*)md[1 - cur_mode];
            a.flags = flags;
            a.mc = mcd;
            e = launch_forward_f64(a, cfg, s);
        } else {
            FwdArgs<float> a{};
            fill_step_args(a, N, n, L, mm, dt, eta, Wi, beta, alpha, step);
            a.courant_coef = ccoef;
            a.courant_limit = 1.0;
            a.kap_n = (const float*)grad_u;
            a.kap_nm1 = (const float*)grad_u;
            a.u = (const float*)u;
            a.sigma0 = sigma0 ? (const float*)s0copy : nullptr;
            a.sig_n = (const float*)sig[cur];
            a.sig_nm1 = (const float*)sig[prev];
            a.sig_np1 = (float*)sig[nxt];
            a.sig_copy = nullptr;
            a.trans = (float*)trans;
            a.modes_n = (const float*)md[cur_mode];
            a.modes_nm1 = (float*)md[1 - cur_mode];
            a.flags = flags;
            a.mc = mcf;
            e = launch_forward_f32(a, cfg, s);
        }
        if (e != cudaSuccess) return TFS_ERR_CUDA;
        prev = cur;
        cur = nxt;
        if (mm > 0) cur_mode = 1 - cur_mode;
    }
    e = cudaMemcpyAsync(sigma_out, sig[cur], field, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? TFS_OK : TFS_ERR_CUDA;
}

extern "C" int tfs_static_status(unsigned* device_flags, void* stream) {
    if (!device_flags) return TFS_ERR_ARG;
    void* base_v = nullptr;
    if (static_base(&base_v) != cudaSuccess) return TFS_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned f = 0u;
    cudaError_t e = cudaMemcpyAsync(&f, base_v, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    *device_flags = f;
    return TFS_OK;
}
