// Host side of libtfs: the C ABI declared in include/tfs.h.
//
// The handle keeps the problem description, the FP64 SOE constants and the
// layout of the caller-bound workspace; the step itself is one kernel launch
// (tfs_forward.cu).  No device memory is allocated here.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <new>
#include <vector>

#include "../../include/tfs.h"
#include "tfs_internal.h"
#include "tfs_adjoint_paper.h"
#include "tfs_adjoint_implicit.h"

using namespace tfs;

namespace {

constexpr uint64_t kMagic = 0x3153464154434b50ull;   // checkpoint tag
constexpr uint64_t kVersion = 3;   // 3: tile-major mode levels
constexpr size_t kAlign = 256;
constexpr size_t kHeaderBytes = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int kHaloPlanes = 2;   // radius of the upwind3 stencil: the planes a slab's neighbours need

}  // namespace

struct tfs_ctx {
    int dim = 2;
    long long n[3] = {1, 1, 1};
    double L[3] = {1, 1, 1};
    long long N = 0;
    int nc = 3;
    double alpha = 1, Wi = 1, beta = 0, Re = 1, eps = 0, dt = 1;
    int m = 0;
    int precision = TFS_FP64;
    int stencil = TFS_STENCIL_UPWIND3;
    int transport = 1;
    int start = TFS_START_BDF2;    // first step from the initial state
    int form = TFS_FORM_STRESS;    // variable carried: the stress, or the paper's Phi
    double umax = -1.0;            // declared velocity bound (< 0: none)
    // SOE
    bool soe_set = false;
    std::vector<double> mu, w;
    ModeConstsD mcd{};
    ModeConstsF mcf{};
    double eta = 0.0;
    // the paper's variable: c_j, dt c_j, w_j mu_j c_j, xi = b0 sum_j w_j c_j, and the
    // modes of Phi0 == 1 (the same at every point; host FP64)
    ModeConstsD mcd_p{};
    ModeConstsF mcf_p{};
    double xi_p = 0.0;
    std::vector<double> phi0_n, phi0_nm1;
    // workspace
    char* ws = nullptr;
    size_t ws_bytes = 0;
    unsigned* flags = nullptr;
    char* sigma0 = nullptr;        // copy of the initial stress
    char* sig[3] = {nullptr, nullptr, nullptr};
    char* trans = nullptr;         // transport term A [nc][N] of the current step
    char* modes[2] = {nullptr, nullptr};
    int cur_sig = 0, prev_sig = 1; // ring slots of levels n and n-1
    char* psi[2] = {nullptr, nullptr};   // the paper's variable: Psi^n (psi[cur_psi]) and Psi^{n-1}
    int cur_psi = 0;
    int cur_mode = 0;              // ring slot of modes level n (n-1 in the other)
    bool sigma0_zero = true;
    bool state_set = false;
    long long step = 0;
    cudaStream_t last_stream = nullptr;
    // optional events recorded around the step kernel of every tfs_step
    cudaEvent_t ev_before = nullptr, ev_after = nullptr;
    // neighbours' boundary planes of a slab step (tfs_step_slab; null otherwise)
    const void* halo_lo = nullptr;
    const void* halo_hi = nullptr;
    // cached stability bounds of the explicit transport (invalidated by SOE and stencil changes)
    bool lim_valid = false;
    double lam_star = 0.0;   // advection: largest stable dt |u| / h (1D)
    double z_star = 0.0;     // diffusion: largest stable 4 eps dt / h^2 (1D)
    // implicit transport: Krylov workspace after the modes, solver controls, last solve
    double* kry = nullptr;
    double* partials = nullptr;
    double krylov_tol = -1.0;      // < 0: default for the precision
    int krylov_maxit = 500;
    int last_iters = 0;
    double last_relres = 0.0;
    // adjoint workspace
    char* aws = nullptr;
    size_t aws_bytes = 0;
    int seg_capacity = 0;

    size_t es() const { return precision == TFS_FP64 ? 8 : 4; }
    bool is_double() const { return precision == TFS_FP64; }
    bool classic() const { return alpha == 1.0; }
    size_t field_bytes() const { return (size_t)nc * (size_t)N * es(); }
    // forward mode levels: tile-major over ceil(N / 32) whole tiles (mode_index)
    size_t modes_bytes() const { return (size_t)m * (size_t)nc * (size_t)mode_points(N) * es(); }
    int third_sig() const { return 3 - cur_sig - prev_sig; }
    bool explicit_transport() const { return transport == 1; }
    // explicit transport: the Courant bound of the form carried applies
    bool checked_transport() const { return transport == 1; }
    bool implicit_transport() const { return transport == 2; }
    bool paper() const { return form == TFS_FORM_PAPER; }
    // slab decomposition along the slowest axis: points per plane of that axis
    // and its length
    long long slab_plane() const { return dim == 3 ? n[0] * n[1] : n[0]; }
    long long slab_len() const { return n[dim - 1]; }
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? TFS_OK : TFS_ERR_CUDA; }

double g_alpha(const tfs_ctx* h, long long step_index) {
    if (h->classic()) return 1.0;
    const double t = (double)(step_index + 1) * h->dt;
    return std::pow(t, h->alpha - 1.0) / std::tgamma(h->alpha);
}

// Stability of the explicit transport.  For one Fourier mode with stencil
// symbol s(theta) (D_h e^{i theta x/h} = s(theta)/h e^{i theta x/h}) and
// lambda = dt |u| / h, the generating function of the scheme's recursion is
//   (W(zeta) + lambda s(theta) zeta (2 - zeta)) y(zeta) = data,
//   W(zeta) = delta(zeta) sum_j w_j dt / (delta(zeta) + mu_j dt)   (alpha < 1),
//   W(zeta) = delta(zeta) = b0 + b1 zeta + b2 zeta^2               (alpha = 1).
// W is analytic in the closed unit disk (the roots of delta + mu dt lie
// outside it), so the step is stable while f = W + lambda s zeta (2 - zeta)
// has no zero in the disk, i.e. while the winding number of f(e^{i phi}),
// 0 <= phi < 2 pi, about 0 vanishes for every theta (argument principle).
// stability_bound() bisects for the largest such lambda along given directions.
// In the paper's variable the transport acts on Psi = V(zeta) Phi, V = sum_j w_j
// delta / (delta + mu_j dt) (the discrete D^{1-alpha} of the mode recursion), and
// the BDF2 equation on Phi gives f = delta + lambda s V zeta (2 - zeta): the same
// test with delta in place of W and V zeta (2 - zeta) in place of zeta (2 - zeta).
struct Cplx {
    double re, im;
};
inline Cplx cadd(Cplx a, Cplx b) { return {a.re + b.re, a.im + b.im}; }
inline Cplx csub(Cplx a, Cplx b) { return {a.re - b.re, a.im - b.im}; }
inline Cplx cmul(Cplx a, Cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline Cplx cdiv(Cplx a, Cplx b) {
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
inline Cplx cexpi(double t) { return {std::cos(t), std::sin(t)}; }

Cplx stencil_symbol(int stencil, double theta) {
    const Cplx e1 = cexpi(theta), em1 = cexpi(-theta), em2 = cexpi(-2 * theta);
    if (stencil == TFS_STENCIL_CENTRAL2) return {0.5 * (e1.re - em1.re), 0.5 * (e1.im - em1.im)};
    // (e^{-2it} - 6 e^{-it} + 3 + 2 e^{it}) / 6
    return {(em2.re - 6 * em1.re + 3 + 2 * e1.re) / 6.0, (em2.im - 6 * em1.im + 2 * e1.im) / 6.0};
}

// Largest t such that f = W + t d zeta (2 - zeta) keeps winding number 0 about
// the origin on |zeta| = 1 for every direction d in `dirs` (bisection).
double stability_bound(const tfs_ctx* h, const std::vector<Cplx>& dirs) {
    // contour |zeta| = 1, refined geometrically towards phi = 0 (zeta = 1)
    std::vector<double> phis;
    const int nlin = 2048, nlog = 200;
    for (int i = nlog; i >= 1; --i) phis.push_back(2 * M_PI / nlin * std::pow(1e-6, (double)i / nlog));
    for (int i = 1; i < nlin; ++i) phis.push_back(2 * M_PI * (double)i / nlin);
    for (int i = 1; i <= nlog; ++i) phis.push_back(2 * M_PI - 2 * M_PI / nlin * std::pow(1e-6, (double)i / nlog));
    const size_t K = phis.size();
    std::vector<Cplx> W(K), G(K);
    for (size_t k = 0; k < K; ++k) {
        const Cplx z = cexpi(phis[k]);
        const Cplx delta = cadd(cadd(Cplx{kB0, 0.0}, cmul(Cplx{kB1, 0.0}, z)), cmul(Cplx{kB2, 0.0}, cmul(z, z)));
        Cplx w{0.0, 0.0};
        const Cplx ext = cmul(z, csub(Cplx{2.0, 0.0}, z));
        if (h->paper()) {
            Cplx v{0.0, 0.0};
            for (int j = 0; j < h->m; ++j)
                v = cadd(v, cdiv(cmul(Cplx{h->w[j], 0.0}, delta), cadd(delta, Cplx{h->mu[j] * h->dt, 0.0})));
            W[k] = delta;
            G[k] = cmul(v, ext);
            continue;
        }
        if (h->classic()) {
            w = delta;
        } else {
            for (int j = 0; j < h->m; ++j)
                w = cadd(w, cdiv(Cplx{h->w[j] * h->dt, 0.0}, cadd(delta, Cplx{h->mu[j] * h->dt, 0.0})));
            w = cmul(w, delta);
        }
        W[k] = w;
        G[k] = ext;
    }
    auto stable = [&](double t) {
        for (const Cplx& sv : dirs) {
            const Cplx ls{t * sv.re, t * sv.im};
            double wind = 0.0;
            Cplx prev = cadd(W[K - 1], cmul(ls, G[K - 1]));
            for (size_t k = 0; k < K; ++k) {
                const Cplx f = cadd(W[k], cmul(ls, G[k]));
                const Cplx r = cdiv(f, prev);
                wind += std::atan2(r.im, r.re);
                prev = f;
            }
            if (std::fabs(wind) > M_PI) return false;   // winding number != 0
        }
        return true;
    };
    double lo = 1e-12, hi = 1e-6;
    if (!stable(lo)) return 0.0;
    while (stable(hi) && hi < 1e6) {
        lo = hi;
        hi *= 2.0;
    }
    for (int it = 0; it < 50 && hi - lo > 1e-7 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (stable(mid)) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Courant check.  With lambda_tot = dt sum_a |u_a|/h_a and nu_tot = eps dt sum_a 1/h_a^2
// the step is accepted while lambda_tot / lambda* + 4 nu_tot / z* <= 0.9, where
// lambda* bounds the advection symbol (directions s(theta)) and z* the
// diffusion symbol 4 nu sin^2(theta/2) (direction +1): 10% margin on the sum of
// the two fractions of the stable region.  The kernel flags points with
// courant_coef * sum_a |u_a| / h_a > courant_limit.
bool limits_known(const tfs_ctx* h) { return h->classic() || h->soe_set; }

void ensure_limits(tfs_ctx* h) {
    if (h->lim_valid) return;
    const int nth = 240;
    std::vector<Cplx> S;
    for (int t = 1; t < nth; ++t) S.push_back(stencil_symbol(h->stencil, 2 * M_PI * t / nth));
    h->lam_star = stability_bound(h, S);
    h->z_star = stability_bound(h, std::vector<Cplx>{Cplx{1.0, 0.0}});
    h->lim_valid = true;
}

double sum_inv_h(const tfs_ctx* h) {
    double s = 0.0;
    for (int a = 0; a < h->dim; ++a) s += (double)h->n[a] / h->L[a];
    return s;
}

double sum_inv_h2(const tfs_ctx* h) {
    double s = 0.0;
    for (int a = 0; a < h->dim; ++a) s += ((double)h->n[a] / h->L[a]) * ((double)h->n[a] / h->L[a]);
    return s;
}

// fraction of the stable region taken by the explicit diffusion term
double diffusion_fraction(tfs_ctx* h, double eps) {
    if (eps == 0.0 || !limits_known(h)) return 0.0;
    ensure_limits(h);
    if (!(h->z_star > 0.0)) return 1e300;
    return 4.0 * eps * h->dt * sum_inv_h2(h) / h->z_star;
}

double courant_coef(tfs_ctx* h) {
    if (!limits_known(h)) return 0.0;
    ensure_limits(h);
    return h->lam_star > 0.0 ? h->dt / h->lam_star : 1e300;
}

double courant_limit(tfs_ctx* h) {
    if (!limits_known(h)) return 1e300;
    return 0.9 - diffusion_fraction(h, h->eps);
}

// declared bounds (eps, and umax when given) exceed the limit
bool limits_violated(tfs_ctx* h) {
    if (!h->checked_transport() || !limits_known(h)) return false;
    const double lim = courant_limit(h);
    if (lim < 0.0) return true;
    return h->umax >= 0.0 && courant_coef(h) * h->umax * sum_inv_h(h) > lim;
}

// implicit transport: 10 Krylov vectors [nc][N] plus the point blocks and the
// preconditioner inverses [nc*nc][N], all FP64
size_t krylov_bytes_for(const tfs_ctx* h, int form) {
    // 10 vectors, the point blocks and their inverses, 4 stencil coefficients per
    // axis, the FP32 section of the inner solve, and (the paper's variable) h
    return (((10 + 2 * (size_t)h->nc + (form == TFS_FORM_PAPER ? 1 : 0)) * (size_t)h->nc + 4 * (size_t)h->dim) *
                (size_t)h->N +
            (size_t)kry_float_doubles(h->nc, h->dim, h->N)) *
           sizeof(double);
}
size_t krylov_bytes(const tfs_ctx* h) { return krylov_bytes_for(h, h->form); }
size_t forward_bytes_for(const tfs_ctx* h, int transport, int form);

void layout_forward(tfs_ctx* h, char* base) {
    char* p = base;
    h->flags = (unsigned*)p;
    p += kAlign;
    h->sigma0 = p;
    p += align_up(h->field_bytes());
    for (int i = 0; i < 3; ++i) {
        h->sig[i] = p;
        p += align_up(h->field_bytes());
    }
    h->trans = p;
    p += align_up(h->field_bytes());
    for (int i = 0; i < 2; ++i) {
        h->modes[i] = p;
        p += align_up(h->modes_bytes());
    }
    h->psi[0] = h->psi[1] = nullptr;
    if (h->paper()) {
        for (int i = 0; i < 2; ++i) {
            h->psi[i] = p;
            p += align_up(h->field_bytes());
        }
    }
    h->kry = nullptr;
    h->partials = nullptr;
    if (h->implicit_transport()) {
        h->kry = (double*)p;
        p += align_up(krylov_bytes(h));
        h->partials = (double*)p;
    }
}

size_t forward_bytes_for(const tfs_ctx* h, int transport, int form) {
    size_t b = kAlign + 5 * align_up(h->field_bytes()) + 2 * align_up(h->modes_bytes());
    if (form == TFS_FORM_PAPER) b += 2 * align_up(h->field_bytes());
    if (transport == 2) b += align_up(krylov_bytes_for(h, form)) + align_up(sizeof(double) * (2 * kImpBlocks + 32));
    return b;
}

size_t forward_bytes(const tfs_ctx* h) { return forward_bytes_for(h, h->transport, h->form); }

F2c split_f2(double v) {
    F2c r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

template <typename T>
void fill_common(tfs_ctx* h, FwdArgs<T>& a) {
    a.N = h->N;
    a.n0 = (int)h->n[0];
    a.n1 = (int)h->n[1];
    a.n2 = (int)h->n[2];
    a.m = h->classic() ? 0 : h->m;
    a.dt = h->dt;
    a.eta = h->classic() ? kB0 : h->eta;
    a.a = a.eta + h->dt / h->Wi;
    a.G = (1.0 - h->beta) / (h->Wi * h->Re);
    a.eps = h->eps;
    for (int i = 0; i < 3; ++i) a.inv_h[i] = (double)h->n[i] / h->L[i];
    a.courant_coef = (h->checked_transport() && limits_known(h)) ? courant_coef(h) : 0.0;
    a.courant_limit = courant_limit(h);
    a.flags = h->flags;
    a.eta_f2 = split_f2(a.eta);
    a.a_f2 = split_f2(a.a);
    a.dt_f2 = split_f2(a.dt);
}

LaunchCfg make_cfg(const tfs_ctx* h) {
    LaunchCfg cfg;
    cfg.dim = h->dim;
    cfg.stencil = h->stencil;
    cfg.transport = h->transport != 0;
    cfg.classic = h->classic();
    cfg.compensated = h->precision == TFS_FP32;
    cfg.ev_before = h->ev_before;
    cfg.ev_after = h->ev_after;
    return cfg;
}

// One forward step; sig_copy optionally receives sigma^{n+1} as well.
template <typename T>
void fill_implicit(tfs_ctx* h, ImpArgs<T>& a, const void* kn, const void* knm1, const void* u, void* sig_copy,
                   int nxt, int cm, int pm) {
    a.kap_n = (const T*)kn;
    a.kap_nm1 = (const T*)knm1;
    a.u = (const T*)u;
    a.sigma0 = h->sigma0_zero ? nullptr : (const T*)h->sigma0;
    a.sig_n = (const T*)h->sig[h->cur_sig];
    a.sig_nm1 = (const T*)h->sig[h->prev_sig];
    a.sig_np1 = (T*)h->sig[nxt];
    a.sig_copy = (T*)sig_copy;
    a.modes_n = (const T*)h->modes[cm];
    a.modes_nm1 = (T*)h->modes[pm];
    a.flags = h->flags;
    a.N = h->N;
    a.dim = h->dim;
    a.n0 = (int)h->n[0];
    a.n1 = (int)h->n[1];
    a.n2 = (int)h->n[2];
    a.m = h->classic() ? 0 : h->m;
    a.stencil = h->stencil;
    a.classic = h->classic() ? 1 : 0;
    a.dt = h->dt;
    a.eta = h->classic() ? kB0 : h->eta;
    a.a = a.eta + h->dt / h->Wi;
    a.G = (1.0 - h->beta) / (h->Wi * h->Re);
    a.g = g_alpha(h, h->step);
    a.eps = h->eps;
    for (int i = 0; i < 3; ++i) a.inv_h[i] = (double)h->n[i] / h->L[i];
    a.mcd = h->mcd;
    a.eta_f2 = split_f2(a.eta);
    a.src_f2 = split_f2(a.dt * a.G * a.g);
    a.kry = h->kry;
    a.partials = h->partials;
    a.tol = h->krylov_tol > 0.0 ? h->krylov_tol : (h->is_double() ? 1e-13 : 1e-9);
    a.maxit = h->krylov_maxit;
}

double paper_psi0(const tfs_ctx* h);
void paper_advance_phi0(tfs_ctx* h);

// The paper's variable with implicit transport: the operator is
// (b0 + dt xi/Wi) I - dt xi L(kappa*) + dt xi (u.grad - eps Lap), i.e. the stress
// form's with a = b0 + dt xi/Wi and transport scale dt xi.
template <typename T>
void fill_implicit_paper(tfs_ctx* h, ImpArgs<T>& a) {
    a.paper = 1;
    a.sigma0 = nullptr;
    a.classic = 0;
    a.dt_rhs = h->dt;
    a.dt = h->dt * h->xi_p;
    a.a = kB0 + h->dt * h->xi_p / h->Wi;
    a.g = paper_psi0(h);
    a.xi = h->xi_p;
    a.inv_wi = 1.0 / h->Wi;
    a.mcd = h->mcd_p;
    a.psi = (T*)h->psi[1 - h->cur_psi];
}

// One step with implicit transport (tfs_implicit.cu); synchronises the stream.
int do_step_implicit(tfs_ctx* h, const void* kn, const void* knm1, const void* u, void* sig_copy, cudaStream_t s) {
    if (!h->kry || h->ws_bytes < forward_bytes(h)) return TFS_ERR_NOWORKSPACE;
    const int nxt = h->third_sig();
    const int cm = h->cur_mode, pm = 1 - h->cur_mode;
    int iters = 0;
    double relres = 0.0;
    cudaError_t e;
    if (h->is_double()) {
        ImpArgs<double> a{};
        fill_implicit(h, a, kn, knm1, u, sig_copy, nxt, cm, pm);
        a.mc = h->mcd;
        if (h->paper()) {
            fill_implicit_paper(h, a);
            a.mc = h->mcd_p;
        }
        e = run_implicit_f64(a, s, &iters, &relres);
    } else {
        ImpArgs<float> a{};
        fill_implicit(h, a, kn, knm1, u, sig_copy, nxt, cm, pm);
        a.mc = h->mcf;
        if (h->paper()) {
            fill_implicit_paper(h, a);
            a.mc = h->mcf_p;
        }
        e = run_implicit_f32(a, s, h->precision == TFS_FP32, &iters, &relres);
    }
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    if (h->paper()) {
        paper_advance_phi0(h);
        h->cur_psi = 1 - h->cur_psi;
    }
    h->last_iters = iters;
    h->last_relres = relres;
    h->prev_sig = h->cur_sig;
    h->cur_sig = nxt;
    if (!h->classic()) h->cur_mode = pm;
    h->step += 1;
    h->last_stream = s;
    return TFS_OK;
}

// The paper's variable: Psi0^{n+1} = xi + sum_j w_j mu_j c_j (b1 phi0_j^n + b2 phi0_j^{n-1}),
// the discrete D^{1-alpha} 1 that multiplies the source, and the push-forward of
// the modes phi0_j of Phi0 == 1 after a step.
double paper_psi0(const tfs_ctx* h) {
    double s = h->xi_p;
    for (int j = 0; j < h->m; ++j) s += h->mcd_p.eta[j] * (kB1 * h->phi0_n[j] + kB2 * h->phi0_nm1[j]);
    return s;
}

void paper_advance_phi0(tfs_ctx* h) {
    for (int j = 0; j < h->m; ++j) {
        const double nx = h->mcd_p.c[j] * (-kB1 * h->phi0_n[j] - kB2 * h->phi0_nm1[j] + h->dt);
        h->phi0_nm1[j] = h->phi0_n[j];
        h->phi0_n[j] = nx;
    }
}

// SDIRK2 first step on the modes of Phi0 == 1 (the scalar case of the
// paper-variable start in tfs_start.cu): returns Psi0 at the two stage times
// in psi0[2] and advances phi0 to level 1.
void paper_sdirk2_phi0(tfs_ctx* h, double psi0[2]) {
    const double gam = 1.0 - std::sqrt(0.5), gd = gam * h->dt, f1 = h->dt * (1.0 - gam);
    double W = 0.0;
    for (int j = 0; j < h->m; ++j) W += h->w[j] / (1.0 + gam * h->mu[j] * h->dt);
    std::vector<double> z2(h->m);
    double s1 = W, s2 = W;
    for (int j = 0; j < h->m; ++j) {
        const double inv = 1.0 / (1.0 + gam * h->mu[j] * h->dt);
        const double z0 = h->phi0_n[j];
        s1 -= h->w[j] * h->mu[j] * z0 * inv;
        const double ph = (z0 + gd) * inv;
        z2[j] = z0 + f1 * (1.0 - h->mu[j] * ph);
        s2 -= h->w[j] * h->mu[j] * z2[j] * inv;
    }
    psi0[0] = s1;
    psi0[1] = s2;
    for (int j = 0; j < h->m; ++j) {
        h->phi0_nm1[j] = h->phi0_n[j];
        h->phi0_n[j] = (z2[j] + gd) / (1.0 + gam * h->mu[j] * h->dt);
    }
}

void paper_reset_phi0(tfs_ctx* h, long long steps) {
    h->phi0_n.assign(h->m, 0.0);
    h->phi0_nm1.assign(h->m, 0.0);
    for (long long k = 0; k < steps; ++k) {
        if (k == 0 && h->start == TFS_START_SDIRK2) {
            double unused[2];
            paper_sdirk2_phi0(h, unused);
        } else {
            paper_advance_phi0(h);
        }
    }
}

template <typename T>
void fill_paper(tfs_ctx* h, FwdArgs<T>& a) {
    const double psi0 = paper_psi0(h);
    a.sigma0 = nullptr;
    a.psi = (T*)h->psi[1 - h->cur_psi];          // Psi^{n+1} over Psi^{n-1}, after the pre-pass has read it
    a.psi_n = (const T*)h->psi[h->cur_psi];
    a.psi_nm1 = (const T*)h->psi[1 - h->cur_psi];
    a.xi = h->xi_p;
    a.inv_wi = 1.0 / h->Wi;
    a.a = kB0 + h->dt * h->xi_p / h->Wi;
    a.g = psi0;
    a.a_f2 = split_f2(a.a);
    a.dt_f2 = split_f2(h->dt);
    a.src_f2 = split_f2(h->dt * a.G * psi0);
    a.xi_f2 = split_f2(h->xi_p);
    a.dtxi_f2 = split_f2(h->dt * h->xi_p);
}

// SDIRK2 constants of the first step (Section 5.1): gamma = 1 - 1/sqrt2,
// 1/(1 + gamma mu_j dt), W = sum_j w_j/(1 + gamma mu_j dt), g_alpha at both stage times
StartConsts start_consts(const tfs_ctx* h) {
    StartConsts c{};
    c.gam = 1.0 - std::sqrt(0.5);
    c.W = 0.0;
    for (int j = 0; j < h->m; ++j) {
        c.mu[j] = h->mu[j];
        c.w[j] = h->w[j];
        c.inv_den[j] = 1.0 / (1.0 + c.gam * h->mu[j] * h->dt);
        c.W += h->w[j] * c.inv_den[j];
    }
    c.g[0] = std::pow(c.gam * h->dt, h->alpha - 1.0) / std::tgamma(h->alpha);
    c.g[1] = std::pow(h->dt, h->alpha - 1.0) / std::tgamma(h->alpha);
    return c;
}

// The first step by SDIRK2: pointwise (transport off, tfs_start.cu) or with the
// implicit transport inside both stage systems (tfs_implicit.cu).  The stress
// and mode rings then advance as after any step: level n-1 = the initial state.
int do_first_step_sdirk2(tfs_ctx* h, const void* kn, const void* u, void* sig_copy, cudaStream_t s) {
    if (h->explicit_transport()) return TFS_ERR_ARG;

    StartConsts c = start_consts(h);
    const int nxt = h->third_sig();
    const int cm = h->cur_mode, pm = 1 - h->cur_mode;
    const double a_stage = h->dt * c.W + h->dt / h->Wi;
    cudaError_t e;
    if (h->implicit_transport()) {
        if (!h->kry || h->ws_bytes < forward_bytes(h)) return TFS_ERR_NOWORKSPACE;
        int iters = 0;
        double relres = 0.0;
        // the paper's variable: stage operator a = 1 + gamma dt W/Wi, scale gamma dt W; Psi0 at the stages
        const std::vector<double> keep_n = h->phi0_n, keep_nm1 = h->phi0_nm1;
        if (h->paper()) paper_sdirk2_phi0(h, c.g);
        auto paper_stage = [&](auto& a) {
            a.paper = 1;
            a.sigma0 = nullptr;
            a.dt_rhs = h->dt;
            a.dt = c.gam * h->dt * c.W;
            a.a = 1.0 + c.gam * h->dt * c.W / h->Wi;
            a.inv_wi = 1.0 / h->Wi;
            a.xi = c.W;
            a.psi = (decltype(a.psi))h->psi[1 - h->cur_psi];
        };
        if (h->is_double()) {
            ImpArgs<double> a{};
            fill_implicit(h, a, kn, kn, u, sig_copy, nxt, cm, pm);
            a.mc = h->mcd;
            a.a = a_stage;
            if (h->paper()) paper_stage(a);
            e = run_start_implicit_f64(a, c, s, &iters, &relres);
        } else {
            ImpArgs<float> a{};
            fill_implicit(h, a, kn, kn, u, sig_copy, nxt, cm, pm);
            a.mc = h->mcf;
            a.a = a_stage;
            if (h->paper()) paper_stage(a);
            e = run_start_implicit_f32(a, c, s, &iters, &relres);
        }
        if (e != cudaSuccess && h->paper()) {
            h->phi0_n = keep_n;
            h->phi0_nm1 = keep_nm1;
        }
        h->last_iters = iters;
        h->last_relres = relres;
    } else if (h->paper()) {
        // Phi^0 is level n of the ring; Psi0 at the stage times from the host
        const std::vector<double> keep_n = h->phi0_n, keep_nm1 = h->phi0_nm1;
        paper_sdirk2_phi0(h, c.g);
        const double a_p = 1.0 + h->dt * c.gam * c.W / h->Wi;
        const double G = (1.0 - h->beta) / (h->Wi * h->Re);
        if (h->ev_before) e = cudaEventRecord(h->ev_before, s);
        else e = cudaSuccess;
        if (e == cudaSuccess && h->is_double()) {
            StartArgs<double> a{(const double*)kn, (const double*)h->sig[h->cur_sig], (const double*)h->modes[cm],
                                (double*)h->modes[pm], (double*)h->sig[nxt], (double*)sig_copy, h->flags, h->N, h->m,
                                h->dt, a_p, G, (double*)h->psi[1 - h->cur_psi], 1.0 / h->Wi};
            e = launch_start_paper_f64(a, c, h->dim, s);
        } else if (e == cudaSuccess) {
            StartArgs<float> a{(const float*)kn, (const float*)h->sig[h->cur_sig], (const float*)h->modes[cm],
                               (float*)h->modes[pm], (float*)h->sig[nxt], (float*)sig_copy, h->flags, h->N, h->m,
                               h->dt, a_p, G, (float*)h->psi[1 - h->cur_psi], 1.0 / h->Wi};
            e = launch_start_paper_f32(a, c, h->dim, s);
        }
        if (e == cudaSuccess && h->ev_after) e = cudaEventRecord(h->ev_after, s);
        if (e != cudaSuccess) {
            h->phi0_n = keep_n;
            h->phi0_nm1 = keep_nm1;
        }
    } else {
        if (h->ev_before) e = cudaEventRecord(h->ev_before, s);
        else e = cudaSuccess;
        if (e == cudaSuccess && h->is_double()) {
            StartArgs<double> a{(const double*)kn, h->sigma0_zero ? nullptr : (const double*)h->sigma0,
                                (const double*)h->modes[cm], (double*)h->modes[pm], (double*)h->sig[nxt],
                                (double*)sig_copy, h->flags, h->N, h->m, h->dt, a_stage,
                                (1.0 - h->beta) / (h->Wi * h->Re), nullptr, 1.0 / h->Wi};
            e = launch_start_point_f64(a, c, h->dim, s);
        } else if (e == cudaSuccess) {
            StartArgs<float> a{(const float*)kn, h->sigma0_zero ? nullptr : (const float*)h->sigma0,
                               (const float*)h->modes[cm], (float*)h->modes[pm], (float*)h->sig[nxt],
                               (float*)sig_copy, h->flags, h->N, h->m, h->dt, a_stage,
                               (1.0 - h->beta) / (h->Wi * h->Re), nullptr, 1.0 / h->Wi};
            e = launch_start_point_f32(a, c, h->dim, s);
        }
        if (e == cudaSuccess && h->ev_after) e = cudaEventRecord(h->ev_after, s);
    }
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    h->prev_sig = h->cur_sig;
    h->cur_sig = nxt;
    h->cur_mode = pm;
    if (h->paper()) h->cur_psi = 1 - h->cur_psi;
    h->step += 1;
    h->last_stream = s;
    return TFS_OK;
}

int do_step(tfs_ctx* h, const void* kn, const void* knm1, const void* u, void* sig_copy, cudaStream_t s) {
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    if (!h->state_set) return TFS_ERR_STATE;
    if (!h->classic() && !h->soe_set) return TFS_ERR_NOSOE;
    if (!kn) return TFS_ERR_ARG;
    if (h->transport && !u) return TFS_ERR_ARG;
    if (limits_violated(h)) return TFS_ERR_UNSTABLE;
    if (!knm1) knm1 = kn;
    if (h->start == TFS_START_SDIRK2 && h->step == 0) return do_first_step_sdirk2(h, kn, u, sig_copy, s);
    if (h->implicit_transport()) return do_step_implicit(h, kn, knm1, u, sig_copy, s);
    const int nxt = h->third_sig();
    const int cm = h->cur_mode, pm = 1 - h->cur_mode;
    cudaError_t e;
    LaunchCfg cfg = make_cfg(h);
    cfg.paper = h->paper();
    if (h->is_double()) {
        FwdArgs<double> a{};
        fill_common(h, a);
        a.kap_n = (const double*)kn;
        a.kap_nm1 = (const double*)knm1;
        a.u = (const double*)u;
        a.sigma0 = h->sigma0_zero ? nullptr : (const double*)h->sigma0;
        a.sig_n = (const double*)h->sig[h->cur_sig];
        a.sig_nm1 = (const double*)h->sig[h->prev_sig];
        a.sig_np1 = (double*)h->sig[nxt];
        a.sig_copy = (double*)sig_copy;
        a.trans = (double*)h->trans;
        a.modes_n = (const double*)h->modes[cm];
        a.modes_nm1 = (double*)h->modes[pm];
        a.halo_lo = (const double*)h->halo_lo;
        a.halo_hi = (const double*)h->halo_hi;
        a.halo_r = kHaloPlanes;
        a.g = g_alpha(h, h->step);
        a.mc = h->mcd;
        if (h->paper()) {
            a.mc = h->mcd_p;
            fill_paper(h, a);
        }
        e = launch_forward_f64(a, cfg, s);
    } else {
        FwdArgs<float> a{};
        fill_common(h, a);
        a.kap_n = (const float*)kn;
        a.kap_nm1 = (const float*)knm1;
        a.u = (const float*)u;
        a.sigma0 = h->sigma0_zero ? nullptr : (const float*)h->sigma0;
        a.sig_n = (const float*)h->sig[h->cur_sig];
        a.sig_nm1 = (const float*)h->sig[h->prev_sig];
        a.sig_np1 = (float*)h->sig[nxt];
        a.sig_copy = (float*)sig_copy;
        a.trans = (float*)h->trans;
        a.modes_n = (const float*)h->modes[cm];
        a.modes_nm1 = (float*)h->modes[pm];
        a.halo_lo = (const float*)h->halo_lo;
        a.halo_hi = (const float*)h->halo_hi;
        a.halo_r = kHaloPlanes;
        a.g = g_alpha(h, h->step);
        a.src_f2 = split_f2(a.dt * a.G * a.g);
        a.mc = h->mcf;
        if (h->paper()) {
            a.mc = h->mcf_p;
            fill_paper(h, a);
        }
        e = launch_forward_f32(a, cfg, s);
    }
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    if (h->paper()) {
        paper_advance_phi0(h);
        h->cur_psi = 1 - h->cur_psi;
    }
    h->prev_sig = h->cur_sig;
    h->cur_sig = nxt;
    if (!h->classic()) h->cur_mode = pm;
    h->step += 1;
    h->last_stream = s;
    return TFS_OK;
}

bool valid_handle(tfs_handle h) { return h != nullptr; }

}  // namespace

extern "C" {

int tfs_create(tfs_handle* out, const tfs_grid* grid, double alpha, double Wi, double beta, int m, double dt,
               int precision) {
    if (!out) return TFS_ERR_ARG;
    *out = nullptr;
    if (!grid || (grid->dim != 2 && grid->dim != 3)) return TFS_ERR_ARG;
    if (!(alpha > 0.0 && alpha <= 1.0)) return TFS_ERR_ARG;
    if (!(Wi > 0.0) || !std::isfinite(Wi)) return TFS_ERR_ARG;
    if (!(beta >= 0.0 && beta < 1.0)) return TFS_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return TFS_ERR_ARG;
    if (m < 0 || m > kMaxModes) return TFS_ERR_ARG;
    if (alpha == 1.0 && m != 0) return TFS_ERR_ARG;
    if (alpha < 1.0 && m < 1) return TFS_ERR_ARG;
    if (precision != TFS_FP64 && precision != TFS_FP32 && precision != TFS_FP32_PLAIN) return TFS_ERR_ARG;
    long long N = 1;
    for (int a = 0; a < grid->dim; ++a) {
        if (grid->n[a] < 1 || !(grid->L[a] > 0.0) || !std::isfinite(grid->L[a])) return TFS_ERR_ARG;
        N *= grid->n[a];
    }
    if ((N + 31) / 32 > 0x7fffffffLL) return TFS_ERR_ARG;
    tfs_ctx* h = new (std::nothrow) tfs_ctx();
    if (!h) return TFS_ERR_ARG;
    h->dim = grid->dim;
    for (int a = 0; a < 3; ++a) {
        h->n[a] = (a < grid->dim) ? grid->n[a] : 1;
        h->L[a] = (a < grid->dim) ? grid->L[a] : 1.0;
    }
    h->N = N;
    h->nc = grid->dim == 2 ? 3 : 6;
    h->alpha = alpha;
    h->Wi = Wi;
    h->beta = beta;
    h->dt = dt;
    h->m = m;
    h->precision = precision;
    *out = h;
    return TFS_OK;
}

int tfs_set_param(tfs_handle h, int key, double value) {
    if (!valid_handle(h)) return TFS_ERR_ARG;
    if (!std::isfinite(value)) return TFS_ERR_ARG;
    switch (key) {
        case TFS_PARAM_RE:
            if (!(value > 0.0)) return TFS_ERR_ARG;
            h->Re = value;
            return TFS_OK;
        case TFS_PARAM_EPS:
            if (!(value >= 0.0)) return TFS_ERR_ARG;
            if (h->checked_transport() && diffusion_fraction(h, value) > 0.9) return TFS_ERR_UNSTABLE;
            h->eps = value;
            return TFS_OK;
        case TFS_PARAM_STENCIL:
            if (value != TFS_STENCIL_UPWIND3 && value != TFS_STENCIL_CENTRAL2) return TFS_ERR_ARG;
            h->stencil = (int)value;
            h->lim_valid = false;
            return TFS_OK;
        case TFS_PARAM_TRANSPORT:
            if (value != 0.0 && value != 1.0 && value != 2.0) return TFS_ERR_ARG;
            if (h->ws && h->ws_bytes < forward_bytes_for(h, (int)value, h->form)) return TFS_ERR_NOWORKSPACE;
            h->transport = (int)value;
            if (h->ws) layout_forward(h, h->ws);
            return TFS_OK;
        case TFS_PARAM_UMAX: {
            if (!(value >= 0.0)) return TFS_ERR_ARG;
            if (h->checked_transport() && limits_known(h) && courant_coef(h) * value * sum_inv_h(h) > courant_limit(h))
                return TFS_ERR_UNSTABLE;
            h->umax = value;
            return TFS_OK;
        }
        case TFS_PARAM_KRYLOV_TOL:
            if (!(value > 0.0 && value < 1.0)) return TFS_ERR_ARG;
            h->krylov_tol = value;
            return TFS_OK;
        case TFS_PARAM_KRYLOV_MAXIT:
            if (!(value >= 1.0 && value <= 100000.0) || value != std::floor(value)) return TFS_ERR_ARG;
            h->krylov_maxit = (int)value;
            return TFS_OK;
        case TFS_PARAM_FORM:
            if (value != TFS_FORM_STRESS && value != TFS_FORM_PAPER) return TFS_ERR_ARG;
            if (value == TFS_FORM_PAPER && h->classic()) return TFS_ERR_ARG;
            if (h->ws && h->ws_bytes < forward_bytes_for(h, h->transport, (int)value)) return TFS_ERR_NOWORKSPACE;
            if ((int)value != h->form) h->state_set = false;   // the state means something else now
            h->form = (int)value;
            h->lim_valid = false;                              // the Courant bound depends on the form
            if (h->ws) layout_forward(h, h->ws);
            return TFS_OK;
        case TFS_PARAM_START:
            if (value != TFS_START_BDF2 && value != TFS_START_SDIRK2) return TFS_ERR_ARG;
            if (value == TFS_START_SDIRK2 && h->classic()) return TFS_ERR_ARG;
            h->start = (int)value;
            return TFS_OK;
        default:
            return TFS_ERR_ARG;
    }
}

int tfs_set_soe(tfs_handle h, const double* mu, const double* w, int m) {
    if (!valid_handle(h)) return TFS_ERR_ARG;
    if (h->classic()) return m == 0 ? TFS_OK : TFS_ERR_ARG;
    if (!mu || !w || m != h->m) return TFS_ERR_ARG;
    for (int j = 0; j < m; ++j)
        if (!(mu[j] >= 0.0) || !(w[j] >= 0.0) || !std::isfinite(mu[j]) || !std::isfinite(w[j])) return TFS_ERR_ARG;
    h->mu.assign(mu, mu + m);
    h->w.assign(w, w + m);
    double eta = 0.0;
    for (int j = 0; j < kMaxModes; ++j) {
        double c = 0.0, rho = 0.0, et = 0.0;
        if (j < m) {
            c = 1.0 / (kB0 + mu[j] * h->dt);
            rho = w[j] * h->dt * c;
            et = mu[j] * h->dt * c;
            eta += kB0 * rho;
        }
        h->mcd.c[j] = c;
        h->mcd.rho[j] = rho;
        h->mcd.eta[j] = et;
        h->mcf.c[j] = (float)c;
        h->mcf.rho[j] = (float)rho;
        const float hi = (float)et;
        h->mcf.eta_hi[j] = hi;
        h->mcf.eta_lo[j] = (float)(et - (double)hi);
    }
    h->eta = eta;
    double xi = 0.0;
    for (int j = 0; j < kMaxModes; ++j) {
        double c = 0.0, pe = 0.0;
        if (j < m) {
            c = 1.0 / (kB0 + mu[j] * h->dt);
            pe = w[j] * mu[j] * c;
            xi += kB0 * w[j] * c;
        }
        h->mcd_p.c[j] = c;
        h->mcd_p.rho[j] = c * h->dt;
        h->mcd_p.eta[j] = pe;
        h->mcf_p.c[j] = (float)c;
        h->mcf_p.rho[j] = (float)(c * h->dt);
        const float hi = (float)pe;
        h->mcf_p.eta_hi[j] = hi;
        h->mcf_p.eta_lo[j] = (float)(pe - (double)hi);
    }
    h->xi_p = xi;
    h->soe_set = true;
    h->lim_valid = false;
    return TFS_OK;
}

int tfs_set_step_events(tfs_handle h, void* ev_before, void* ev_after) {
    if (!valid_handle(h)) return TFS_ERR_ARG;
    if ((ev_before == nullptr) != (ev_after == nullptr)) return TFS_ERR_ARG;
    h->ev_before = (cudaEvent_t)ev_before;
    h->ev_after = (cudaEvent_t)ev_after;
    return TFS_OK;
}

int tfs_transport_limit(tfs_handle h, double* umax_out) {
    if (!valid_handle(h) || !umax_out) return TFS_ERR_ARG;
    if (!h->classic() && !h->soe_set) return TFS_ERR_NOSOE;
    const double lim = courant_limit(h);
    *umax_out = lim > 0.0 ? lim / (courant_coef(h) * sum_inv_h(h)) : 0.0;
    return TFS_OK;
}

size_t tfs_workspace_bytes(tfs_handle h) {
    if (!valid_handle(h)) return 0;
    return forward_bytes(h);
}

int tfs_bind_workspace(tfs_handle h, void* dev_ptr, size_t bytes) {
    if (!valid_handle(h) || !dev_ptr) return TFS_ERR_ARG;
    if (((uintptr_t)dev_ptr) % kAlign) return TFS_ERR_ARG;
    if (bytes < forward_bytes(h)) return TFS_ERR_NOWORKSPACE;
    h->ws = (char*)dev_ptr;
    h->ws_bytes = bytes;
    layout_forward(h, h->ws);
    h->state_set = false;
    return TFS_OK;
}

int tfs_set_state(tfs_handle h, const void* sigma0, void* stream) {
    if (!valid_handle(h)) return TFS_ERR_ARG;
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    h->cur_sig = 0;
    h->prev_sig = 1;
    h->cur_mode = 0;
    h->cur_psi = 0;
    const long long count = (long long)h->nc * h->N;
    cudaError_t e = launch_fill_levels(h->sig[0], h->sig[1], h->sigma0, sigma0, count, h->is_double(), s);
    if (e == cudaSuccess && h->m > 0) e = launch_zero(h->modes[0], h->modes_bytes(), s);
    if (e == cudaSuccess && h->m > 0) e = launch_zero(h->modes[1], h->modes_bytes(), s);
    if (e == cudaSuccess) e = launch_zero(h->flags, kAlign, s);
    for (int i = 0; i < 2 && h->paper(); ++i)    // Psi before the first step, and its past: 0
        if (e == cudaSuccess) e = launch_zero(h->psi[i], h->field_bytes(), s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    paper_reset_phi0(h, 0);
    h->sigma0_zero = (sigma0 == nullptr);
    h->step = 0;
    h->state_set = true;
    h->last_stream = s;
    return TFS_OK;
}

int tfs_step(tfs_handle h, const void* grad_u_n, const void* grad_u_nm1, const void* u, void* stream) {
    if (!valid_handle(h)) return TFS_ERR_ARG;
    return do_step(h, grad_u_n, grad_u_nm1, u, nullptr, (cudaStream_t)stream);
}

size_t tfs_halo_bytes(tfs_handle h) {
    if (!valid_handle(h)) return 0;
    return 2 * (size_t)h->nc * kHaloPlanes * (size_t)h->slab_plane() * h->es();
}

int tfs_get_halo(tfs_handle h, void* lo, void* hi, void* stream) {
    if (!valid_handle(h) || (!lo && !hi)) return TFS_ERR_ARG;
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    if (!h->state_set) return TFS_ERR_STATE;
    if (h->paper() || h->slab_len() < kHaloPlanes) return TFS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    h->last_stream = s;
    const size_t es = h->es();
    const size_t width = (size_t)kHaloPlanes * (size_t)h->slab_plane() * es;   // R planes of one component
    const char* lv[2] = {h->sig[h->cur_sig], h->sig[h->prev_sig]};
    for (int side = 0; side < 2; ++side) {
        char* dst = (char*)(side == 0 ? lo : hi);
        if (!dst) continue;
        const size_t first = side == 0 ? 0 : (size_t)(h->slab_len() - kHaloPlanes) * (size_t)h->slab_plane() * es;
        for (int l = 0; l < 2; ++l) {
            cudaError_t e = cudaMemcpy2DAsync(dst + (size_t)l * h->nc * width, width, lv[l] + first,
                                              (size_t)h->N * es, width, (size_t)h->nc, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return TFS_ERR_CUDA;
        }
    }
    return TFS_OK;
}

int tfs_step_slab(tfs_handle h, const void* grad_u_n, const void* grad_u_nm1, const void* u, const void* halo_lo,
                  const void* halo_hi, void* stream) {
    if (!valid_handle(h) || !halo_lo || !halo_hi) return TFS_ERR_ARG;
    if (h->paper() || h->implicit_transport() || h->slab_len() < kHaloPlanes) return TFS_ERR_ARG;
    h->halo_lo = halo_lo;
    h->halo_hi = halo_hi;
    const int rc = do_step(h, grad_u_n, grad_u_nm1, u, nullptr, (cudaStream_t)stream);
    h->halo_lo = h->halo_hi = nullptr;
    return rc;
}

int tfs_get_stress(tfs_handle h, void* out, void* stream) {
    if (!valid_handle(h) || !out) return TFS_ERR_ARG;
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    if (!h->state_set) return TFS_ERR_STATE;
    h->last_stream = (cudaStream_t)stream;
    const void* src = h->paper() ? (const void*)h->psi[h->cur_psi] : (const void*)h->sig[h->cur_sig];
    return cuda_err(cudaMemcpyAsync(out, src, h->field_bytes(), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

long tfs_step_index(tfs_handle h) { return valid_handle(h) ? (long)h->step : -1; }

int tfs_last_solve(tfs_handle h, int* iterations, double* relative_residual) {
    if (!valid_handle(h)) return TFS_ERR_ARG;
    if (iterations) *iterations = h->last_iters;
    if (relative_residual) *relative_residual = h->last_relres;
    return TFS_OK;
}

size_t tfs_checkpoint_bytes(tfs_handle h) {
    if (!valid_handle(h)) return 0;
    return kHeaderBytes + (h->paper() ? 5 : 3) * align_up(h->field_bytes()) + 2 * align_up(h->modes_bytes());
}

int tfs_save(tfs_handle h, void* dst, void* stream) {
    if (!valid_handle(h) || !dst) return TFS_ERR_ARG;
    if (((uintptr_t)dst) % 16) return TFS_ERR_ARG;
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    if (!h->state_set) return TFS_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t words[13] = {kMagic, kVersion, (uint64_t)h->dim, (uint64_t)h->n[0], (uint64_t)h->n[1],
                          (uint64_t)h->n[2], (uint64_t)h->m, (uint64_t)h->precision, (uint64_t)h->step,
                          (uint64_t)(h->sigma0_zero ? 1 : 0), 0, 0, (uint64_t)h->form};
    double scal[2] = {h->dt, h->alpha};
    memcpy(&words[10], &scal[0], 8);
    memcpy(&words[11], &scal[1], 8);
    char* p = (char*)dst;
    cudaError_t e = launch_write_header((uint64_t*)p, words, 13, s);
    p += kHeaderBytes;
    const size_t fb = h->field_bytes(), mb = h->modes_bytes();
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->sig[h->cur_sig], fb, cudaMemcpyDeviceToDevice, s);
    p += align_up(fb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->sig[h->prev_sig], fb, cudaMemcpyDeviceToDevice, s);
    p += align_up(fb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->sigma0, fb, cudaMemcpyDeviceToDevice, s);
    p += align_up(fb);
    if (mb > 0) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->modes[h->cur_mode], mb, cudaMemcpyDeviceToDevice, s);
        p += align_up(mb);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->modes[1 - h->cur_mode], mb, cudaMemcpyDeviceToDevice, s);
        p += align_up(mb);
    }
    if (h->paper()) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->psi[h->cur_psi], fb, cudaMemcpyDeviceToDevice, s);
        p += align_up(fb);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p, h->psi[1 - h->cur_psi], fb, cudaMemcpyDeviceToDevice, s);
    }
    h->last_stream = s;
    return cuda_err(e);
}

int tfs_load(tfs_handle h, const void* src, void* stream) {
    if (!valid_handle(h) || !src) return TFS_ERR_ARG;
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t words[13];
    cudaError_t e = cudaMemcpyAsync(words, src, sizeof(words), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    double scal[2];
    memcpy(&scal[0], &words[10], 8);
    memcpy(&scal[1], &words[11], 8);
    if (words[0] != kMagic || words[1] != kVersion || words[2] != (uint64_t)h->dim ||
        words[3] != (uint64_t)h->n[0] || words[4] != (uint64_t)h->n[1] || words[5] != (uint64_t)h->n[2] ||
        words[6] != (uint64_t)h->m || words[7] != (uint64_t)h->precision || scal[0] != h->dt ||
        scal[1] != h->alpha || words[12] != (uint64_t)h->form)
        return TFS_ERR_FORMAT;
    h->cur_sig = 0;
    h->prev_sig = 1;
    h->cur_mode = 0;
    const char* p = (const char*)src + kHeaderBytes;
    const size_t fb = h->field_bytes(), mb = h->modes_bytes();
    e = cudaMemcpyAsync(h->sig[0], p, fb, cudaMemcpyDeviceToDevice, s);
    p += align_up(fb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sig[1], p, fb, cudaMemcpyDeviceToDevice, s);
    p += align_up(fb);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->sigma0, p, fb, cudaMemcpyDeviceToDevice, s);
    p += align_up(fb);
    if (mb > 0) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->modes[0], p, mb, cudaMemcpyDeviceToDevice, s);
        p += align_up(mb);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->modes[1], p, mb, cudaMemcpyDeviceToDevice, s);
        p += align_up(mb);
    }
    if (h->paper()) {
        h->cur_psi = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->psi[0], p, fb, cudaMemcpyDeviceToDevice, s);
        p += align_up(fb);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->psi[1], p, fb, cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    h->step = (long long)words[8];
    if (h->paper()) paper_reset_phi0(h, h->step);
    h->sigma0_zero = words[9] != 0;
    h->state_set = true;
    h->last_stream = s;
    return TFS_OK;
}

// ------------------------------------------------------------------ adjoint
namespace {

struct AdjLayout {
    double* s[4];       // two ping-pong pairs (s1, s0)
    double* t[4];       // the paper's variable with transport: the same for the adjoint of Psi
    double* cfT;        // implicit transport: the transposed operator's tap coefficients
    double* lpp;        // implicit transport in the paper's variable: the modified adjoint of Psi
    double* lamR;
    char* ell[2];
    double* partials;   // 2 per block
    double* out2;
    char* seg;
    size_t seg_stride;
};

bool paper_psi_ring(const tfs_ctx* h) { return h->paper() && h->transport == 1; }

size_t adj_bytes(const tfs_ctx* h, int seg_steps) {
    const size_t dfield = (size_t)h->nc * (size_t)h->N * 8;
    const long long blocks = (h->N + 31) / 32;
    const size_t cft = h->implicit_transport() ? align_up(4 * (size_t)h->dim * (size_t)h->N * 8) : 0;
    const size_t lpp = (h->implicit_transport() && h->paper()) ? align_up(dfield) : 0;
    return (paper_psi_ring(h) ? 9 : 5) * align_up(dfield) + cft + lpp + 2 * align_up(h->modes_bytes()) + align_up((size_t)blocks * 16) + kAlign +
           (size_t)seg_steps * align_up(h->field_bytes());
}

AdjLayout adj_layout(const tfs_ctx* h) {
    AdjLayout L;
    const size_t dfield = (size_t)h->nc * (size_t)h->N * 8;
    const long long blocks = (h->N + 31) / 32;
    char* p = h->aws;
    for (int i = 0; i < 4; ++i) {
        L.s[i] = (double*)p;
        p += align_up(dfield);
    }
    L.lamR = (double*)p;
    p += align_up(dfield);
    for (int i = 0; i < 4; ++i) {
        L.t[i] = nullptr;
        if (paper_psi_ring(h)) {
            L.t[i] = (double*)p;
            p += align_up(dfield);
        }
    }
    L.cfT = nullptr;
    if (h->implicit_transport()) {
        L.cfT = (double*)p;
        p += align_up(4 * (size_t)h->dim * (size_t)h->N * 8);
    }
    L.lpp = nullptr;
    if (h->implicit_transport() && h->paper()) {
        L.lpp = (double*)p;
        p += align_up(dfield);
    }
    for (int i = 0; i < 2; ++i) {
        L.ell[i] = p;
        p += align_up(h->modes_bytes());
    }
    L.partials = (double*)p;
    p += align_up((size_t)blocks * 16);
    L.out2 = (double*)p;
    p += kAlign;
    L.seg = p;
    L.seg_stride = align_up(h->field_bytes());
    return L;
}

// One reverse step of the paper's variable (BDF2; pointwise law or explicit
// transport): psi is the step's Psi^{n+1}, lam_psi the adjoint of Psi at the
// final step (else null; with transport the Psi ring carries it), psi0 the
// step's Psi0^{n+1}.
extern "C++" template <typename T>
cudaError_t paper_adjoint_step(const tfs_ctx* h, const AdjLayout& L, int cur, int ell_prev, const void* grad_u,
                               const void* u, const void* psi, const double* lam_psi, double psi0, double* g_kap,
                               cudaStream_t s) {
    const int nxt = 1 - cur;
    PaperAdjArgs<T> a{};
    a.kap = (const T*)grad_u;
    a.psi = (const T*)psi;
    a.lam_psi = lam_psi;
    a.s1 = L.s[2 * cur];
    a.s0 = L.s[2 * cur + 1];
    a.ell_prev = (const T*)L.ell[ell_prev];
    a.ell_prev2 = (T*)L.ell[1 - ell_prev];
    a.s1_out = L.s[2 * nxt];
    a.s0_out = L.s[2 * nxt + 1];
    a.g_kap = g_kap;
    if (paper_psi_ring(h)) {
        a.t1 = L.t[2 * cur];
        a.t0 = L.t[2 * cur + 1];
        a.t1_out = L.t[2 * nxt];
        a.t0_out = L.t[2 * nxt + 1];
        a.lamR_out = L.lamR;
    }
    a.partials = L.partials;
    a.flags = h->flags;
    a.N = h->N;
    a.m = h->m;
    a.dt = h->dt;
    a.a = kB0 + h->dt * h->xi_p / h->Wi;
    a.xi = h->xi_p;
    a.G = (1.0 - h->beta) / (h->Wi * h->Re);
    a.psi0 = psi0;
    a.Wi = h->Wi;
    a.Re = h->Re;
    a.mc = h->mcd_p;
    a.mcf = h->mcf_p;
    cudaError_t e;
    if constexpr (sizeof(T) == 8) e = launch_paper_adjoint_f64(a, h->dim, s);
    else e = launch_paper_adjoint_f32(a, h->dim, s);
    if (e != cudaSuccess || !paper_psi_ring(h)) return e;
    // the transposed stencil of -dt (u.grad - eps Lap)(2 Psi^n - Psi^{n-1})
    AdjArgs<double> ad{};
    ad.N = h->N;
    ad.n0 = (int)h->n[0];
    ad.n1 = (int)h->n[1];
    ad.n2 = (int)h->n[2];
    ad.dt = h->dt;
    ad.eps = h->eps;
    for (int i = 0; i < 3; ++i) ad.inv_h[i] = (double)h->n[i] / h->L[i];
    ad.lamR = L.lamR;
    ad.s1_out = L.t[2 * nxt];
    ad.s0_out = L.t[2 * nxt + 1];
    return launch_adjoint_transport(ad, u, sizeof(T) == 8, make_cfg(h), s);
}

// Psi0^{n+1} of steps 0 .. steps-1 (with the SDIRK2 start: Psi0 at its two
// stage times in stage[2], out[0] unused), leaving the host modes of Phi0 as
// they were.
std::vector<double> paper_psi0_sequence(tfs_ctx* h, int steps, double stage[2]) {
    const std::vector<double> keep_n = h->phi0_n, keep_nm1 = h->phi0_nm1;
    paper_reset_phi0(h, 0);
    std::vector<double> out((size_t)steps);
    stage[0] = stage[1] = 0.0;
    for (int k = 0; k < steps; ++k) {
        if (k == 0 && h->start == TFS_START_SDIRK2) {
            paper_sdirk2_phi0(h, stage);
            out[0] = 0.0;
            continue;
        }
        out[(size_t)k] = paper_psi0(h);
        paper_advance_phi0(h);
    }
    h->phi0_n = keep_n;
    h->phi0_nm1 = keep_nm1;
    return out;
}

}  // namespace

size_t tfs_adjoint_workspace_bytes(tfs_handle h, int segment_steps) {
    if (!valid_handle(h) || segment_steps < 1) return 0;
    return adj_bytes(h, segment_steps);
}

int tfs_bind_adjoint_workspace(tfs_handle h, void* dev_ptr, size_t bytes) {
    if (!valid_handle(h) || !dev_ptr) return TFS_ERR_ARG;
    if (((uintptr_t)dev_ptr) % kAlign) return TFS_ERR_ARG;
    const size_t base = adj_bytes(h, 0);
    if (bytes < adj_bytes(h, 1)) return TFS_ERR_NOWORKSPACE;
    h->aws = (char*)dev_ptr;
    h->aws_bytes = bytes;
    h->seg_capacity = (int)((bytes - base) / align_up(h->field_bytes()));
    return TFS_OK;
}

int tfs_backward(tfs_handle h, const void* dJ_dsigma_T, const void* const* checkpoints, int K, int steps,
                 const void* grad_u, const void* u, double* dJ_dsigma0, double* dJ_dgrad_u, double* dJ_dWi,
                 double* dJ_dbeta, void* stream) {
    // the SDIRK2 first step's adjoint: pointwise law or implicit transport (the
    // forward refuses explicit transport with it)
    if (valid_handle(h) && h->start == TFS_START_SDIRK2 && h->explicit_transport()) return TFS_ERR_ARG;
    if (!valid_handle(h) || !dJ_dsigma_T || !checkpoints || !grad_u || !dJ_dsigma0 || !dJ_dgrad_u || !dJ_dWi ||
        !dJ_dbeta)
        return TFS_ERR_ARG;
    if (K < 1 || steps < 1) return TFS_ERR_ARG;
    if (h->transport && !u) return TFS_ERR_ARG;
    if (!h->ws || !h->aws) return TFS_ERR_NOWORKSPACE;
    if (h->aws_bytes < adj_bytes(h, K)) return TFS_ERR_NOWORKSPACE;   // also after a change of form
    if (!h->classic() && !h->soe_set) return TFS_ERR_NOSOE;
    cudaStream_t s = (cudaStream_t)stream;
    AdjLayout L = adj_layout(h);
    const size_t dfield = (size_t)h->nc * (size_t)h->N * 8;
    const long long blocks = (h->N + 31) / 32;
    const long long ncN = (long long)h->nc * h->N;
    cudaError_t e = cudaSuccess;
    e = launch_zero(dJ_dsigma0, dfield, s);
    if (e == cudaSuccess) e = launch_zero(dJ_dgrad_u, (size_t)h->dim * h->dim * h->N * 8, s);
    if (e == cudaSuccess) e = launch_zero(L.partials, (size_t)blocks * 16, s);
    for (int i = 0; i < 2 && e == cudaSuccess && h->modes_bytes() > 0; ++i) e = launch_zero(L.ell[i], h->modes_bytes(), s);
    // J = <dJ, sigma^T>, or in the paper's variable <dJ, Psi^T> (held in lamR, the
    // adjoint of Phi^T then starts at 0)
    double* dJ_into = h->paper() ? (paper_psi_ring(h) ? L.t[0] : L.lamR) : L.s[0];
    if (e == cudaSuccess) e = launch_to_double(dJ_dsigma_T, dJ_into, ncN, h->is_double(), s);
    if (e == cudaSuccess && h->paper()) e = launch_zero(L.s[0], dfield, s);
    if (e == cudaSuccess && paper_psi_ring(h)) e = launch_zero(L.t[1], dfield, s);
    if (e == cudaSuccess) e = launch_zero(L.s[1], dfield, s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    double psi0_stage[2] = {0.0, 0.0};
    const std::vector<double> psi0s = h->paper() ? paper_psi0_sequence(h, steps, psi0_stage) : std::vector<double>();
    int cur = 0;        // s[2*cur] = s1, s[2*cur+1] = s0
    int ell_prev = 0;   // slot of lamQ of the later step; the other slot holds the one before
    const LaunchCfg cfg = make_cfg(h);
    const int nseg = (steps + K - 1) / K;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int start = seg * K;
        const int end = (start + K < steps) ? start + K : steps;
        int rc = tfs_load(h, checkpoints[seg], stream);
        if (rc != TFS_OK) return rc;
        if (h->step != start) return TFS_ERR_FORMAT;
        for (int n = start; n < end; ++n) {
            rc = do_step(h, grad_u, grad_u, u, L.seg + (size_t)(n - start) * L.seg_stride, s);
            if (rc != TFS_OK) return rc;
        }
        for (int n = end - 1; n >= start; --n) {
            const void* sig_np1 = L.seg + (size_t)(n - start) * L.seg_stride;
            const int nxt = 1 - cur;
            if (h->paper() && n == 0 && h->start == TFS_START_SDIRK2) {
                // pointwise law (SDIRK2 refuses explicit transport, the adjoint implicit transport)
                StartConsts c = start_consts(h);
                c.g[0] = psi0_stage[0];
                c.g[1] = psi0_stage[1];
                const double a_p = 1.0 + h->dt * c.gam * c.W / h->Wi;
                const double G = (1.0 - h->beta) / (h->Wi * h->Re);
                const double* lam_psi = (steps == 1) ? L.lamR : nullptr;
                if (h->implicit_transport()) {
                    // both stage systems global; Phi^(1) of stage 1 kept in lpp
                    int it = 0;
                    double rr = 0.0;
                    if (h->is_double()) {
                        ImpArgs<double> ia{};
                        fill_implicit(h, ia, grad_u, grad_u, u, nullptr, h->third_sig(), h->cur_mode, 1 - h->cur_mode);
                        ia.a = a_p;
                        ia.dt = c.gam * h->dt * c.W;
                        StartImpAdj<double> j{L.s[2 * cur], L.s[2 * cur + 1], (const double*)L.ell[ell_prev],
                                              (const double*)L.ell[1 - ell_prev], (const double*)sig_np1, L.lpp,
                                              L.s[2 * nxt], L.s[2 * nxt + 1], dJ_dgrad_u, L.partials, L.cfT,
                                              h->Wi, h->Re, 1, lam_psi,
                                              h->sigma0_zero ? nullptr : (const double*)h->sigma0, h->dt};
                        e = run_start_implicit_adjoint_f64(ia, c, j, s, &it, &rr);
                    } else {
                        ImpArgs<float> ia{};
                        fill_implicit(h, ia, grad_u, grad_u, u, nullptr, h->third_sig(), h->cur_mode, 1 - h->cur_mode);
                        ia.a = a_p;
                        ia.dt = c.gam * h->dt * c.W;
                        StartImpAdj<float> j{L.s[2 * cur], L.s[2 * cur + 1], (const float*)L.ell[ell_prev],
                                             (const float*)L.ell[1 - ell_prev], (const float*)sig_np1, L.lpp,
                                             L.s[2 * nxt], L.s[2 * nxt + 1], dJ_dgrad_u, L.partials, L.cfT,
                                             h->Wi, h->Re, 1, lam_psi,
                                             h->sigma0_zero ? nullptr : (const float*)h->sigma0, h->dt};
                        e = run_start_implicit_adjoint_f32(ia, c, j, s, &it, &rr);
                    }
                    if (e != cudaSuccess) return TFS_ERR_CUDA;
                    h->last_iters = it;
                    h->last_relres = rr;
                    cur = nxt;
                    continue;
                }
                if (h->is_double()) {
                    PaperStartAdjArgs<double> a{(const double*)grad_u,
                                                h->sigma0_zero ? nullptr : (const double*)h->sigma0, lam_psi,
                                                L.s[2 * cur], L.s[2 * cur + 1], (const double*)L.ell[ell_prev],
                                                (const double*)L.ell[1 - ell_prev], L.s[2 * nxt], L.s[2 * nxt + 1],
                                                dJ_dgrad_u, L.partials, h->flags, h->N, h->m, h->dt, a_p, G, h->Wi,
                                                h->Re};
                    e = launch_paper_start_adjoint_f64(a, c, h->dim, s);
                } else {
                    PaperStartAdjArgs<float> a{(const float*)grad_u,
                                               h->sigma0_zero ? nullptr : (const float*)h->sigma0, lam_psi,
                                               L.s[2 * cur], L.s[2 * cur + 1], (const float*)L.ell[ell_prev],
                                               (const float*)L.ell[1 - ell_prev], L.s[2 * nxt], L.s[2 * nxt + 1],
                                               dJ_dgrad_u, L.partials, h->flags, h->N, h->m, h->dt, a_p, G, h->Wi,
                                               h->Re};
                    e = launch_paper_start_adjoint_f32(a, c, h->dim, s);
                }
                if (e != cudaSuccess) return TFS_ERR_CUDA;
                cur = nxt;
                continue;
            }
            if (h->paper()) {
                const double* lam_psi = (n == steps - 1 && !paper_psi_ring(h)) ? L.lamR : nullptr;
                if (h->implicit_transport()) {
                    // Op^T solve; the adjoint of Psi handed on carries the transport's term
                    int it = 0;
                    double rr = 0.0;
                    if (h->is_double()) {
                        ImpArgs<double> ia{};
                        fill_implicit(h, ia, grad_u, grad_u, u, nullptr, h->third_sig(), h->cur_mode, 1 - h->cur_mode);
                        fill_implicit_paper(h, ia);
                        e = run_implicit_adjoint_f64(ia, L.s[2 * cur], (const double*)L.ell[ell_prev],
                                                     (const double*)L.ell[1 - ell_prev], L.cfT, lam_psi, h->xi_p,
                                                     L.lpp, s, &it, &rr);
                    } else {
                        ImpArgs<float> ia{};
                        fill_implicit(h, ia, grad_u, grad_u, u, nullptr, h->third_sig(), h->cur_mode, 1 - h->cur_mode);
                        fill_implicit_paper(h, ia);
                        e = run_implicit_adjoint_f32(ia, L.s[2 * cur], (const float*)L.ell[ell_prev],
                                                     (const float*)L.ell[1 - ell_prev], L.cfT, lam_psi, h->xi_p,
                                                     L.lpp, s, &it, &rr);
                    }
                    if (e != cudaSuccess) return TFS_ERR_CUDA;
                    h->last_iters = it;
                    h->last_relres = rr;
                    lam_psi = L.lpp;
                }
                e = h->is_double() ? paper_adjoint_step<double>(h, L, cur, ell_prev, grad_u, u, sig_np1, lam_psi,
                                                                psi0s[(size_t)n], dJ_dgrad_u, s)
                                   : paper_adjoint_step<float>(h, L, cur, ell_prev, grad_u, u, sig_np1, lam_psi,
                                                               psi0s[(size_t)n], dJ_dgrad_u, s);
                if (e != cudaSuccess) return TFS_ERR_CUDA;
                cur = nxt;
                ell_prev = 1 - ell_prev;
                continue;
            }
            if (n == 0 && h->start == TFS_START_SDIRK2) {
                const StartConsts c = start_consts(h);
                const double a_stage = h->dt * c.W + h->dt / h->Wi;
                const double G = (1.0 - h->beta) / (h->Wi * h->Re);
                if (h->implicit_transport()) {
                    // both stage systems are global: two transposed solves, stage 1 solved again
                    int it = 0;
                    double rr = 0.0;
                    if (h->is_double()) {
                        ImpArgs<double> ia{};
                        fill_implicit(h, ia, grad_u, grad_u, u, nullptr, h->third_sig(), h->cur_mode, 1 - h->cur_mode);
                        ia.a = a_stage;
                        StartImpAdj<double> j{L.s[2 * cur], L.s[2 * cur + 1], (const double*)L.ell[ell_prev],
                                              (const double*)L.ell[1 - ell_prev], (const double*)sig_np1, L.lamR,
                                              L.s[2 * nxt], L.s[2 * nxt + 1], dJ_dgrad_u, L.partials, L.cfT,
                                              h->Wi, h->Re, 0, nullptr, nullptr, h->dt};
                        e = run_start_implicit_adjoint_f64(ia, c, j, s, &it, &rr);
                    } else {
                        ImpArgs<float> ia{};
                        fill_implicit(h, ia, grad_u, grad_u, u, nullptr, h->third_sig(), h->cur_mode, 1 - h->cur_mode);
                        ia.a = a_stage;
                        StartImpAdj<float> j{L.s[2 * cur], L.s[2 * cur + 1], (const float*)L.ell[ell_prev],
                                             (const float*)L.ell[1 - ell_prev], (const float*)sig_np1, L.lamR,
                                             L.s[2 * nxt], L.s[2 * nxt + 1], dJ_dgrad_u, L.partials, L.cfT,
                                             h->Wi, h->Re, 0, nullptr, nullptr, h->dt};
                        e = run_start_implicit_adjoint_f32(ia, c, j, s, &it, &rr);
                    }
                    if (e != cudaSuccess) return TFS_ERR_CUDA;
                    h->last_iters = it;
                    h->last_relres = rr;
                    cur = nxt;
                    continue;
                }
                if (h->is_double()) {
                    StartAdjArgs<double> a{(const double*)grad_u, h->sigma0_zero ? nullptr : (const double*)h->sigma0,
                                           L.s[2 * cur], L.s[2 * cur + 1], (const double*)L.ell[ell_prev],
                                           (const double*)L.ell[1 - ell_prev], L.s[2 * nxt], L.s[2 * nxt + 1],
                                           dJ_dgrad_u, L.partials, h->flags, h->N, h->m, h->dt, a_stage, G, h->Wi,
                                           h->Re};
                    e = launch_start_adjoint_f64(a, c, h->dim, s);
                } else {
                    StartAdjArgs<float> a{(const float*)grad_u, h->sigma0_zero ? nullptr : (const float*)h->sigma0,
                                          L.s[2 * cur], L.s[2 * cur + 1], (const float*)L.ell[ell_prev],
                                          (const float*)L.ell[1 - ell_prev], L.s[2 * nxt], L.s[2 * nxt + 1],
                                          dJ_dgrad_u, L.partials, h->flags, h->N, h->m, h->dt, a_stage, G, h->Wi,
                                          h->Re};
                    e = launch_start_adjoint_f32(a, c, h->dim, s);
                }
                if (e != cudaSuccess) return TFS_ERR_CUDA;
                cur = nxt;
                continue;
            }
            if (h->is_double()) {
                AdjArgs<double> a{};
                a.kap_n = (const double*)grad_u;
                a.kap_nm1 = (const double*)grad_u;
                a.u = (const double*)u;
                a.sig_np1 = (const double*)sig_np1;
                a.ell_prev = (const double*)L.ell[ell_prev];
                a.ell_prev2 = (double*)L.ell[1 - ell_prev];
                a.mc = h->mcd;
                a.s1 = L.s[2 * cur];
                a.s0 = L.s[2 * cur + 1];
                a.s1_out = L.s[2 * nxt];
                a.s0_out = L.s[2 * nxt + 1];
                a.lamR = L.lamR;
                a.g_sigma0 = dJ_dsigma0;
                a.g_kap = dJ_dgrad_u;
                a.partials = L.partials;
                a.flags = h->flags;
                a.N = h->N;
                a.n0 = (int)h->n[0];
                a.n1 = (int)h->n[1];
                a.n2 = (int)h->n[2];
                a.m = h->classic() ? 0 : h->m;
                a.first = (n == steps - 1);
                a.dt = h->dt;
                a.eta = h->classic() ? kB0 : h->eta;
                a.a = a.eta + h->dt / h->Wi;
                a.G = (1.0 - h->beta) / (h->Wi * h->Re);
                a.g = g_alpha(h, n);
                a.eps = h->eps;
                a.Wi = h->Wi;
                a.Re = h->Re;
                for (int i = 0; i < 3; ++i) a.inv_h[i] = (double)h->n[i] / h->L[i];
                if (h->implicit_transport()) {
                    ImpArgs<double> ia{};
                    fill_implicit(h, ia, grad_u, grad_u, u, nullptr, h->third_sig(), h->cur_mode, 1 - h->cur_mode);
                    int it = 0;
                    double rr = 0.0;
                    e = run_implicit_adjoint_f64(ia, L.s[2 * cur], a.ell_prev, a.ell_prev2, L.cfT, nullptr, 0.0,
                                                 nullptr, s, &it, &rr);
                    h->last_iters = it;
                    h->last_relres = rr;
                }
                if (e == cudaSuccess) e = launch_adjoint_f64(a, cfg, s);
                if (e == cudaSuccess && h->explicit_transport()) e = launch_adjoint_transport(a, u, true, cfg, s);
            } else {
                AdjArgs<float> a{};
                a.kap_n = (const float*)grad_u;
                a.kap_nm1 = (const float*)grad_u;
                a.u = (const float*)u;
                a.sig_np1 = (const float*)sig_np1;
                a.ell_prev = (const float*)L.ell[ell_prev];
                a.ell_prev2 = (float*)L.ell[1 - ell_prev];
                a.mc = h->mcd;
                a.mcf = h->mcf;
                a.s1 = L.s[2 * cur];
                a.s0 = L.s[2 * cur + 1];
                a.s1_out = L.s[2 * nxt];
                a.s0_out = L.s[2 * nxt + 1];
                a.lamR = L.lamR;
                a.g_sigma0 = dJ_dsigma0;
                a.g_kap = dJ_dgrad_u;
                a.partials = L.partials;
                a.flags = h->flags;
                a.N = h->N;
                a.n0 = (int)h->n[0];
                a.n1 = (int)h->n[1];
                a.n2 = (int)h->n[2];
                a.m = h->classic() ? 0 : h->m;
                a.first = (n == steps - 1);
                a.dt = h->dt;
                a.eta = h->classic() ? kB0 : h->eta;
                a.a = a.eta + h->dt / h->Wi;
                a.G = (1.0 - h->beta) / (h->Wi * h->Re);
                a.g = g_alpha(h, n);
                a.eps = h->eps;
                a.Wi = h->Wi;
                a.Re = h->Re;
                for (int i = 0; i < 3; ++i) a.inv_h[i] = (double)h->n[i] / h->L[i];
                if (h->implicit_transport()) {
                    ImpArgs<float> ia{};
                    fill_implicit(h, ia, grad_u, grad_u, u, nullptr, h->third_sig(), h->cur_mode, 1 - h->cur_mode);
                    int it = 0;
                    double rr = 0.0;
                    e = run_implicit_adjoint_f32(ia, L.s[2 * cur], a.ell_prev, a.ell_prev2, L.cfT, nullptr, 0.0,
                                                 nullptr, s, &it, &rr);
                    h->last_iters = it;
                    h->last_relres = rr;
                }
                if (e == cudaSuccess) e = launch_adjoint_f32(a, cfg, s);
                if (e == cudaSuccess && h->explicit_transport()) {
                    AdjArgs<double> ad{};
                    ad.N = a.N;
                    ad.n0 = a.n0;
                    ad.n1 = a.n1;
                    ad.n2 = a.n2;
                    ad.dt = a.dt;
                    ad.eps = a.eps;
                    for (int i = 0; i < 3; ++i) ad.inv_h[i] = a.inv_h[i];
                    ad.lamR = a.lamR;
                    ad.s1_out = a.s1_out;
                    ad.s0_out = a.s0_out;
                    e = launch_adjoint_transport(ad, u, false, cfg, s);
                }
            }
            if (e != cudaSuccess) return TFS_ERR_CUDA;
            cur = nxt;
            if (!h->classic()) ell_prev = 1 - ell_prev;
        }
    }
    // initial state sigma^0 = sigma^{-1} = sigma0
    e = launch_add_initial(dJ_dsigma0, L.s[2 * cur], L.s[2 * cur + 1], ncN, s);
    if (e == cudaSuccess) e = launch_reduce_partials(L.partials, (int)blocks, L.out2, s);
    double out2[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(out2, L.out2, sizeof(out2), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    *dJ_dWi = out2[0];
    *dJ_dbeta = out2[1];
    h->last_stream = s;
    return TFS_OK;
}

int tfs_status(tfs_handle h, unsigned* device_flags) {
    if (!valid_handle(h) || !device_flags) return TFS_ERR_ARG;
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->flags, sizeof(v), cudaMemcpyDeviceToHost, h->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->last_stream);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    *device_flags = v;
    return TFS_OK;
}

const char* tfs_strerror(int code) {
    switch (code) {
        case TFS_OK: return "ok";
        case TFS_ERR_ARG: return "invalid argument";
        case TFS_ERR_NOSOE: return "no SOE table set (alpha < 1)";
        case TFS_ERR_UNSTABLE: return "velocity bound exceeds the explicit-transport Courant limit";
        case TFS_ERR_CUDA: return "CUDA runtime error";
        case TFS_ERR_STATE: return "call out of order (state not set)";
        case TFS_ERR_NOWORKSPACE: return "workspace not bound or too small";
        case TFS_ERR_FORMAT: return "checkpoint does not match this handle";
        case TFS_ERR_TOOBIG: return "problem state exceeds the 64 MiB array of tfs_run_static";
        default: return "unknown status";
    }
}

int tfs_destroy(tfs_handle h) {
    if (!valid_handle(h)) return TFS_ERR_ARG;
    delete h;
    return TFS_OK;
}

}  // extern "C"
