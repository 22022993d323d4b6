// Navier-Stokes projection step on the periodic square (Section 4.1), the
// velocity the stress step is coupled to.  One step t_n -> t_{n+1}, BDF2 with
// the extrapolation E(f) = 2 f^n - f^{n-1} (eq. BDF_and_extrapolation),
// nu = beta/Re, sigma the polymer stress whose divergence drives the momentum
// equation (eq. Navier_Stokes):
//   Xi = (b1 u^n + b2 u^{n-1})/dt + E(nu curl curl u + (u.grad)u - div sigma)
//        (eq. time_discretization_NS; curl curl u = grad div u - Lap u, eq. velocity_correction)
//   Lap p = -div Xi, mean(p) = 0                                   (eq. NS_Poisson)
//   (b0/dt) u^{n+1} - nu Lap u^{n+1} = -grad p - (b1 u^n + b2 u^{n-1})/dt
//        + E(-(u.grad)u + div sigma)                               (eq. NS_Helmholtz)
// On the periodic grid every operator is diagonal in Fourier space: d/dx_a
// multiplies mode k by i k_a (zero at the Nyquist wavenumber of the axis), the
// Laplacian is the square of that, so Poisson and Helmholtz are divisions per
// mode and the result is divergence-free to rounding.  Products are formed on
// the grid.  The transforms are this file's own: a Stockham autosort FFT of
// each row in shared memory (the formulation of Govindaraju et al.,
// "High performance discrete Fourier transforms on graphics processors",
// SC 2008) in radix 4, FP64 complex, and a tiled transpose between the two axes; spectral
// arrays are kept transposed, [kx][ky].  Real fields go two to a complex
// transform (f + i g forward, split by the Hermitian symmetry of real spectra;
// A + i B inverse), so a step takes 6 two-dimensional transforms, not 11.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/tfs.h"
#include "tfs_internal.h"

namespace tfs {
namespace {

constexpr int kMaxLen = 1024;          // longest row transform (two rows of complex doubles in 32 KB)
constexpr int kNsThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// i d a for a real d (the first-derivative multiplier)
__device__ __forceinline__ double2 cimul(double d, double2 a) { return make_double2(-d * a.y, d * a.x); }

// DFT of each row of length n (a power of two, 2 .. kMaxLen) with
// exp(-+ 2 pi i j k / n) (forward / inverse), times `scale`; one block per row,
// rows of `in` and `out` n elements apart (in == out allowed: a row is read
// whole first).  tw[t] = exp(-2 pi i t / n), t < n (computed once on the host
// in FP64).  Stockham autosort, radix 4: stage Ns = 1, 4, 16, ... takes the
// four operands j + r n/4 (r = 0..3) of butterfly j, turns operand r by
// exp(-+ 2 pi i r k / (4 Ns)) = tw[r k n / (4 Ns)], k = j mod Ns, applies the
// 4-point DFT and writes output r to (j / Ns) 4 Ns + k + r Ns; a length that is
// not a power of four ends with one radix-2 stage (Ns = n/2).  The buffers
// ping-pong in shared memory; the result is in natural order.
__global__ void __launch_bounds__(kNsThreads) fft_rows_kernel(const double2* in, double2* out, int n,
                                                              const double2* __restrict__ tw, int inverse,
                                                              double scale) {
    extern __shared__ double2 fft_buf[];
    double2* x = fft_buf;
    double2* y = fft_buf + n;
    const double2* src = in + (long long)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = src[i];
    __syncthreads();
    const int quarter = n >> 2;
    int ns = 1;
    for (; 4 * ns <= n; ns <<= 2) {
        const int step = n / (4 * ns);
        for (int j = threadIdx.x; j < quarter; j += blockDim.x) {
            const int k = j & (ns - 1);
            const double2 v0 = x[j];
            double2 v1 = x[j + quarter], v2 = x[j + 2 * quarter], v3 = x[j + 3 * quarter];
            if (ns > 1) {   // the first stage's twiddles are all 1
                double2 t1 = __ldg(tw + k * step), t2 = __ldg(tw + 2 * k * step), t3 = __ldg(tw + 3 * k * step);
                if (inverse) {
                    t1.y = -t1.y;
                    t2.y = -t2.y;
                    t3.y = -t3.y;
                }
                v1 = cmul(v1, t1);
                v2 = cmul(v2, t2);
                v3 = cmul(v3, t3);
            }
            const double2 a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), d = csub(v1, v3);
            // (v1 - v3) times -i (forward) or +i (inverse)
            const double2 a3 = inverse ? make_double2(-d.y, d.x) : make_double2(d.y, -d.x);
            const int o = ((j - k) << 2) + k;
            y[o] = cadd(a0, a2);
            y[o + ns] = cadd(a1, a3);
            y[o + 2 * ns] = csub(a0, a2);
            y[o + 3 * ns] = csub(a1, a3);
        }
        __syncthreads();
        double2* tmp = x;
        x = y;
        y = tmp;
    }
    if (ns < n) {   // radix-2 stage, Ns = n/2
        const int half = n >> 1;
        const int step = half / ns;
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int k = j & (ns - 1);
            double2 t = __ldg(tw + k * step);
            if (inverse) t.y = -t.y;
            const double2 a = x[j];
            const double2 b = cmul(x[j + half], t);
            const int o = ((j - k) << 1) + k;
            y[o] = cadd(a, b);
            y[o + ns] = csub(a, b);
        }
        __syncthreads();
        double2* tmp = x;
        x = y;
        y = tmp;
    }
    double2* dst = out + (long long)blockIdx.x * n;
    if (scale == 1.0)
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = x[i];
    else
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = cscale(x[i], scale);
}

// out[c][r] = in[r][c] for a rows x cols complex matrix (32 x 32 tiles)
__global__ void transpose_kernel(const double2* in, double2* out, int rows, int cols) {
    __shared__ double2 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[(long long)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(long long)c * rows + r] = tile[threadIdx.x][k];
    }
}

// Two real fields per complex transform: z = f + i g on the grid (g absent: 0).
template <typename T>
__global__ void pack_pair_kernel(const T* f, const T* g, double2* z, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        z[i] = make_double2((double)f[i], g ? (double)g[i] : 0.0);
}

// Spectra of the two real fields of Z = DFT(f + i g) ([kx][ky], row kx of n1
// entries): with W = conj(Z(-k)), F = (Z + W)/2 and G = (Z - W)/(2i), the
// Hermitian and anti-Hermitian parts (G not written when absent).
__global__ void unpack_pair_kernel(const double2* Z, double2* F, double2* G, int n0, int n1) {
    const long long n = (long long)n0 * n1;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / n1), j = (int)(q - (long long)i * n1);
        const long long qm = (long long)(i == 0 ? 0 : n0 - i) * n1 + (j == 0 ? 0 : n1 - j);
        const double2 z = Z[q], zm = Z[qm];
        F[q] = make_double2(0.5 * (z.x + zm.x), 0.5 * (z.y - zm.y));
        if (G) G[q] = make_double2(0.5 * (z.y + zm.y), -0.5 * (z.x - zm.x));
    }
}

// Z = A + i B in spectral space (B absent: 0), for one inverse transform of two
// real fields: the real part of the result is a, the imaginary part b
__global__ void pack_spectra_kernel(const double2* A, const double2* B, double2* Z, long long n) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double2 a = A[q];
        Z[q] = B ? make_double2(a.x - B[q].y, a.y + B[q].x) : a;
    }
}

// real and imaginary parts of z into the FP64 fields da, db and the caller's
// fields ta, tb (each when given)
template <typename T>
__global__ void unpack_grid_kernel(const double2* z, double* da, T* ta, double* db, T* tb, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = z[i];
        if (da) da[i] = v.x;
        if (ta) ta[i] = (T)v.x;
        if (db) db[i] = v.y;
        if (tb) tb[i] = (T)v.y;
    }
}

// First-derivative multipliers d_x, d_y of spectral entry idx of the
// transposed layout [kx][ky] (row kx of n1 entries): wavenumber times 2 pi / L,
// zero at the Nyquist index of each axis.
__device__ __forceinline__ void wavenumbers(long long idx, int n0, int n1, double sx, double sy, double& dx,
                                            double& dy) {
    const int qi = (int)idx;   // n0 n1 <= kMaxLen^2
    const int i = qi / n1, j = qi - i * n1;
    dx = i == n0 / 2 ? 0.0 : (double)(i < n0 / 2 ? i : i - n0) * sx;
    dy = j == n1 / 2 ? 0.0 : (double)(j < n1 / 2 ? j : j - n1) * sy;
}

#define NS_LOOP(i, n) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
                           i += (long long)gridDim.x * blockDim.x)

// divergence-free part of (ux, uy) in place: u -= grad phi, Lap phi = div u (mode 0 kept)
__global__ void ns_project_kernel(double2* ux, double2* uy, int n0, int n1, double sx, double sy) {
    NS_LOOP(q, (long long)n0 * n1) {
        double dx, dy;
        wavenumbers(q, n0, n1, sx, sy, dx, dy);
        const double k2 = dx * dx + dy * dy;
        if (k2 <= 0.0) continue;
        const double2 div = cadd(cimul(dx, ux[q]), cimul(dy, uy[q]));
        const double2 phi = cscale(div, -1.0 / k2);
        ux[q] = csub(ux[q], cimul(dx, phi));
        uy[q] = csub(uy[q], cimul(dy, phi));
    }
}

// spectral velocity gradient: g0 = d_x ux, g1 = d_y ux, g2 = d_x uy, g3 = d_y uy
__global__ void ns_gradient_kernel(const double2* ux, const double2* uy, double2* g0, double2* g1, double2* g2,
                                   double2* g3, int n0, int n1, double sx, double sy) {
    NS_LOOP(q, (long long)n0 * n1) {
        double dx, dy;
        wavenumbers(q, n0, n1, sx, sy, dx, dy);
        g0[q] = cimul(dx, ux[q]);
        g1[q] = cimul(dy, ux[q]);
        g2[q] = cimul(dx, uy[q]);
        g3[q] = cimul(dy, uy[q]);
    }
}

// spectral divergence of the packed stress (xx, xy, yy): (d_x s_xx + d_y s_xy, d_x s_xy + d_y s_yy)
__global__ void ns_divstress_kernel(const double2* sxx, const double2* sxy, const double2* syy, double2* dx_out,
                                    double2* dy_out, int n0, int n1, double sx, double sy) {
    NS_LOOP(q, (long long)n0 * n1) {
        double dx, dy;
        wavenumbers(q, n0, n1, sx, sy, dx, dy);
        dx_out[q] = cadd(cimul(dx, sxx[q]), cimul(dy, sxy[q]));
        dy_out[q] = cadd(cimul(dx, sxy[q]), cimul(dy, syy[q]));
    }
}

// convective term on the grid: (u.grad)u_a = u_x kappa_a,x + u_y kappa_a,y (kappa [4][N] row-major)
__global__ void ns_convection_kernel(const double* u, const double* kap, double* cx, double* cy, long long N) {
    NS_LOOP(p, N) {
        const double ux = u[p], uy = u[N + p];
        cx[p] = ux * kap[p] + uy * kap[N + p];
        cy[p] = ux * kap[2 * N + p] + uy * kap[3 * N + p];
    }
}

// One step per Fourier mode.  a: u^n, b: u^{n-1}; c, d: the convective term and
// the stress divergence at levels n (0) and n-1 (1); out: u^{n+1}.
struct NsModes {
    const double2 *ax, *ay, *bx, *by;
    const double2 *c0x, *c0y, *c1x, *c1y;
    const double2 *d0x, *d0y, *d1x, *d1y;
    double2 *ox, *oy;
};

// Per mode, with h = (b1 u^n + b2 u^{n-1})/dt and w = h + E(conv - div sigma):
// Xi = h + E(nu curl curl u + conv - div sigma), p = i k.Xi / k^2 (Lap p =
// -div Xi), (b0/dt + nu k^2) u^{n+1} = -i k p - w.  In Fourier space
// k.(curl curl u) = k.(k^2 u - k (k.u)) = 0 for every k, so k.Xi = k.w and
//   u^{n+1} = -(w - k (k.w)/k^2) / (b0/dt + nu k^2),
// the projection of -w onto divergence-free fields, which the kernel forms
// directly (the rotational term changes the pressure of the scheme only on a
// bounded domain).  Mode 0: u^{n+1} = -w dt/b0.
__global__ void ns_update_kernel(const NsModes M, int n0, int n1, double sx, double sy, double nu, double dt) {
    const double idt = 1.0 / dt, b0dt = kB0 / dt;
    NS_LOOP(q, (long long)n0 * n1) {
        double dx, dy;
        wavenumbers(q, n0, n1, sx, sy, dx, dy);
        const double k2 = dx * dx + dy * dy;
        auto wcomp = [&](double2 a, double2 b, double2 c0, double2 c1, double2 d0, double2 d1) {
            const double2 h = cscale(cadd(cscale(a, kB1), cscale(b, kB2)), idt);
            return cadd(h, csub(cscale(csub(c0, d0), 2.0), csub(c1, d1)));
        };
        double2 wx = wcomp(M.ax[q], M.bx[q], M.c0x[q], M.c1x[q], M.d0x[q], M.d1x[q]);
        double2 wy = wcomp(M.ay[q], M.by[q], M.c0y[q], M.c1y[q], M.d0y[q], M.d1y[q]);
        double inv = dt / kB0;
        if (k2 > 0.0) {
            // one division gives both 1/k^2 and 1/(b0/dt + nu k^2)
            const double den = b0dt + nu * k2;
            const double r = 1.0 / (k2 * den);
            const double2 s = cscale(cadd(cscale(wx, dx), cscale(wy, dy)), den * r);   // (k.w)/k^2
            wx = csub(wx, cscale(s, dx));
            wy = csub(wy, cscale(s, dy));
            inv = k2 * r;
        }
        M.ox[q] = cscale(wx, -inv);
        M.oy[q] = cscale(wy, -inv);
    }
}

}  // namespace
}  // namespace tfs

using namespace tfs;

struct tfs_ns_ctx {
    int n0 = 0, n1 = 0;
    long long N = 0;
    double sx = 0, sy = 0;        // 2 pi / L per axis
    double nu = 0, dt = 0;
    int precision = TFS_FP64;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    // spectral (complex, [kx][ky]): velocity levels, convective term and stress
    // divergence levels, stress components, gradient components, transposes
    double2* uh[2][2] = {};       // [level slot][component]
    double2* ch[2][2] = {};
    double2* dh[2][2] = {};
    double2* sh[3] = {};
    double2* gh[4] = {};
    double2* tmp[2] = {};
    // grid fields (FP64): u^n [2][N], kappa^n [4][N], convective term [2][N]
    double* u = nullptr;
    double* kap = nullptr;
    double* conv = nullptr;
    double2* tw0 = nullptr;       // exp(-2 pi i t / n0), t < n0; and for n1
    double2* tw1 = nullptr;
    std::vector<double2> tw_host; // both tables, uploaded by tfs_ns_set_state
    int cur = 0;                  // slot of level n (n-1 in the other)
    bool have_prev_terms = false; // f^{n-1} exists (else the empty past: f^{n-1} = f^n)
    bool state_set = false;
    long long step = 0;
};

namespace {

constexpr size_t kNsAlign = 256;
size_t ns_up(size_t v) { return (v + kNsAlign - 1) / kNsAlign * kNsAlign; }

size_t ns_bytes(const tfs_ns_ctx* h) {
    const size_t cplx = ns_up(sizeof(double2) * (size_t)h->N), real = ns_up(sizeof(double) * (size_t)h->N);
    return 21 * cplx + 8 * real + ns_up(sizeof(double2) * (size_t)(h->n0 + h->n1));
}

void ns_layout(tfs_ns_ctx* h) {
    const size_t cplx = ns_up(sizeof(double2) * (size_t)h->N), real = ns_up(sizeof(double) * (size_t)h->N);
    char* p = h->ws;
    auto take_c = [&]() { double2* r = (double2*)p; p += cplx; return r; };
    for (int l = 0; l < 2; ++l)
        for (int a = 0; a < 2; ++a) h->uh[l][a] = take_c();
    for (int l = 0; l < 2; ++l)
        for (int a = 0; a < 2; ++a) h->ch[l][a] = take_c();
    for (int l = 0; l < 2; ++l)
        for (int a = 0; a < 2; ++a) h->dh[l][a] = take_c();
    for (int c = 0; c < 3; ++c) h->sh[c] = take_c();
    for (int c = 0; c < 4; ++c) h->gh[c] = take_c();
    for (int c = 0; c < 2; ++c) h->tmp[c] = take_c();
    h->u = (double*)p;
    p += 2 * real;
    h->kap = (double*)p;
    p += 4 * real;
    h->conv = (double*)p;
    p += 2 * real;
    h->tw0 = (double2*)p;
    h->tw1 = h->tw0 + h->n0;
}

unsigned ns_grid(long long n) {
    long long b = (n + kNsThreads - 1) / kNsThreads;
    return (unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

cudaError_t fft_rows(const tfs_ns_ctx* h, const double2* in, double2* out, int n, int rows, double sign,
                     double scale, cudaStream_t s) {
    const int threads = n / 2 < kNsThreads ? (n / 2 > 0 ? n / 2 : 1) : kNsThreads;
    const double2* tw = n == h->n0 ? h->tw0 : h->tw1;
    fft_rows_kernel<<<rows, threads, 2 * n * sizeof(double2), s>>>(in, out, n, tw, sign > 0 ? 1 : 0, scale);
    return cudaGetLastError();
}

cudaError_t transpose(const double2* in, double2* out, int rows, int cols, cudaStream_t s) {
    transpose_kernel<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, s>>>(in, out, rows, cols);
    return cudaGetLastError();
}

// spectra [kx][ky] of two real grid fields [y][x] (g absent: G not formed),
// by one complex transform of f + i g
template <typename T>
cudaError_t fft2_pair(tfs_ns_ctx* h, const T* f, const T* g, double2* F, double2* G, cudaStream_t s) {
    pack_pair_kernel<T><<<ns_grid(h->N), kNsThreads, 0, s>>>(f, g, h->tmp[0], h->N);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = fft_rows(h, h->tmp[0], h->tmp[0], h->n0, h->n1, -1.0, 1.0, s);
    if (e == cudaSuccess) e = transpose(h->tmp[0], h->tmp[1], h->n1, h->n0, s);
    if (e == cudaSuccess) e = fft_rows(h, h->tmp[1], h->tmp[1], h->n1, h->n0, -1.0, 1.0, s);
    if (e == cudaSuccess) {
        unpack_pair_kernel<<<ns_grid(h->N), kNsThreads, 0, s>>>(h->tmp[1], F, G, h->n0, h->n1);
        e = cudaGetLastError();
    }
    return e;
}

// real grid fields [y][x] of the spectra A and B ([kx][ky], both Hermitian; B
// may be absent), by one inverse transform of A + i B: a into da and/or ta, b
// into db and/or tb
template <typename T>
cudaError_t ifft2_pair(tfs_ns_ctx* h, const double2* A, const double2* B, double* da, T* ta, double* db, T* tb,
                       cudaStream_t s) {
    pack_spectra_kernel<<<ns_grid(h->N), kNsThreads, 0, s>>>(A, B, h->tmp[0], h->N);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = fft_rows(h, h->tmp[0], h->tmp[0], h->n1, h->n0, 1.0, 1.0, s);
    if (e == cudaSuccess) e = transpose(h->tmp[0], h->tmp[1], h->n0, h->n1, s);
    if (e == cudaSuccess) e = fft_rows(h, h->tmp[1], h->tmp[1], h->n0, h->n1, 1.0, 1.0 / (double)h->N, s);
    if (e == cudaSuccess) {
        unpack_grid_kernel<T><<<ns_grid(h->N), kNsThreads, 0, s>>>(h->tmp[1], da, ta, db, tb, h->N);
        e = cudaGetLastError();
    }
    return e;
}

// grid velocity and gradient of the spectral level (ux, uy) into the FP64
// fields u, kap and, when given, the caller's fields uo [2][N], ko [4][N]
template <typename T>
cudaError_t grid_fields(tfs_ns_ctx* h, double2* ux, double2* uy, double* u, double* kap, T* uo, T* ko,
                        cudaStream_t s) {
    const long long N = h->N;
    cudaError_t e = ifft2_pair<T>(h, ux, uy, u, uo, u + N, uo ? uo + N : nullptr, s);
    if (e != cudaSuccess) return e;
    ns_gradient_kernel<<<ns_grid(N), kNsThreads, 0, s>>>(ux, uy, h->gh[0], h->gh[1], h->gh[2], h->gh[3], h->n0, h->n1,
                                                         h->sx, h->sy);
    e = cudaGetLastError();
    for (int c = 0; c < 4 && e == cudaSuccess; c += 2)
        e = ifft2_pair<T>(h, h->gh[c], h->gh[c + 1], kap + c * N, ko ? ko + c * N : nullptr, kap + (c + 1) * N,
                          ko ? ko + (c + 1) * N : nullptr, s);
    return e;
}

// spectral convective term (u.grad)u of grid fields u, kap into (cx, cy)
cudaError_t convection(tfs_ns_ctx* h, const double* u, const double* kap, double2* cx, double2* cy, cudaStream_t s) {
    ns_convection_kernel<<<ns_grid(h->N), kNsThreads, 0, s>>>(u, kap, h->conv, h->conv + h->N, h->N);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = fft2_pair<double>(h, h->conv, h->conv + h->N, cx, cy, s);
    return e;
}

template <typename T>
int ns_set_state(tfs_ns_ctx* h, const T* u0, const T* uprev, cudaStream_t s) {
    const long long N = h->N;
    const int c = h->cur, o = 1 - c;
    cudaError_t e = cudaMemcpyAsync(h->tw0, h->tw_host.data(), sizeof(double2) * h->tw_host.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = fft2_pair<T>(h, u0, u0 + N, h->uh[c][0], h->uh[c][1], s);
    if (e == cudaSuccess) {
        ns_project_kernel<<<ns_grid(N), kNsThreads, 0, s>>>(h->uh[c][0], h->uh[c][1], h->n0, h->n1, h->sx, h->sy);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && uprev) {
        // the given level n-1 and its explicit terms (no stress)
        e = fft2_pair<T>(h, uprev, uprev + N, h->uh[o][0], h->uh[o][1], s);
        if (e == cudaSuccess) {
            ns_project_kernel<<<ns_grid(N), kNsThreads, 0, s>>>(h->uh[o][0], h->uh[o][1], h->n0, h->n1, h->sx, h->sy);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = grid_fields<T>(h, h->uh[o][0], h->uh[o][1], h->u, h->kap, nullptr, nullptr, s);
        if (e == cudaSuccess) e = convection(h, h->u, h->kap, h->ch[o][0], h->ch[o][1], s);
        for (int a = 0; a < 2 && e == cudaSuccess; ++a)
            e = cudaMemsetAsync(h->dh[o][a], 0, sizeof(double2) * (size_t)N, s);
    } else if (e == cudaSuccess) {
        for (int a = 0; a < 2 && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(h->uh[o][a], h->uh[c][a], sizeof(double2) * (size_t)N, cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = grid_fields<T>(h, h->uh[c][0], h->uh[c][1], h->u, h->kap, nullptr, nullptr, s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    h->have_prev_terms = uprev != nullptr;
    h->state_set = true;
    h->step = 0;
    return TFS_OK;
}

template <typename T>
int ns_step(tfs_ns_ctx* h, const T* sigma, T* u_out, T* kap_out, cudaStream_t s) {
    const long long N = h->N;
    const int c = h->cur, o = 1 - c;
    // explicit terms of level n: convection from the stored grid fields, stress divergence
    cudaError_t e = convection(h, h->u, h->kap, h->ch[c][0], h->ch[c][1], s);
    if (e == cudaSuccess && sigma) {
        e = fft2_pair<T>(h, sigma, sigma + N, h->sh[0], h->sh[1], s);
        if (e == cudaSuccess) e = fft2_pair<T>(h, sigma + 2 * N, (const T*)nullptr, h->sh[2], nullptr, s);
        if (e == cudaSuccess) {
            ns_divstress_kernel<<<ns_grid(N), kNsThreads, 0, s>>>(h->sh[0], h->sh[1], h->sh[2], h->dh[c][0],
                                                                  h->dh[c][1], h->n0, h->n1, h->sx, h->sy);
            e = cudaGetLastError();
        }
    } else {
        for (int a = 0; a < 2 && e == cudaSuccess; ++a)
            e = cudaMemsetAsync(h->dh[c][a], 0, sizeof(double2) * (size_t)N, s);
    }
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    // level n-1's terms (the empty past: level n's)
    const int pc = h->have_prev_terms ? o : c;
    NsModes M{h->uh[c][0], h->uh[c][1], h->uh[o][0], h->uh[o][1],
              h->ch[c][0], h->ch[c][1], h->ch[pc][0], h->ch[pc][1],
              h->dh[c][0], h->dh[c][1], h->dh[pc][0], h->dh[pc][1],
              h->uh[o][0], h->uh[o][1]};
    // u^{n+1} is written over u^{n-1}: each mode reads its own entries before writing them
    ns_update_kernel<<<ns_grid(N), kNsThreads, 0, s>>>(M, h->n0, h->n1, h->sx, h->sy, h->nu, h->dt);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = grid_fields<T>(h, h->uh[o][0], h->uh[o][1], h->u, h->kap, u_out, kap_out, s);
    if (e != cudaSuccess) return TFS_ERR_CUDA;
    h->cur = o;
    h->have_prev_terms = true;
    h->step += 1;
    return TFS_OK;
}

bool pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" {

int tfs_ns_create(tfs_ns_handle* out, int n0, int n1, double L0, double L1, double beta, double Re, double dt,
                  int precision) {
    if (!out) return TFS_ERR_ARG;
    *out = nullptr;
    if (!pow2(n0) || !pow2(n1) || n0 > kMaxLen || n1 > kMaxLen) return TFS_ERR_ARG;
    if (!(L0 > 0.0) || !(L1 > 0.0) || !std::isfinite(L0) || !std::isfinite(L1)) return TFS_ERR_ARG;
    if (!(beta > 0.0 && beta <= 1.0) || !(Re > 0.0) || !std::isfinite(Re) || !(dt > 0.0) || !std::isfinite(dt))
        return TFS_ERR_ARG;
    if (precision != TFS_FP64 && precision != TFS_FP32 && precision != TFS_FP32_PLAIN) return TFS_ERR_ARG;
    tfs_ns_ctx* h = new (std::nothrow) tfs_ns_ctx();
    if (!h) return TFS_ERR_ARG;
    h->n0 = n0;
    h->n1 = n1;
    h->N = (long long)n0 * n1;
    h->sx = 2.0 * 3.14159265358979323846 / L0;
    h->sy = 2.0 * 3.14159265358979323846 / L1;
    h->nu = beta / Re;
    h->dt = dt;
    h->precision = precision;
    // twiddle tables exp(-2 pi i t / n), t < n, of both axes (FP64, host)
    for (int n : {n0, n1})
        for (int t = 0; t < n; ++t) {
            const double a = -2.0 * 3.14159265358979323846 * (double)t / (double)n;
            h->tw_host.push_back(make_double2(std::cos(a), std::sin(a)));
        }
    *out = h;
    return TFS_OK;
}

size_t tfs_ns_workspace_bytes(tfs_ns_handle h) { return h ? ns_bytes(h) : 0; }

int tfs_ns_bind_workspace(tfs_ns_handle h, void* dev_ptr, size_t bytes) {
    if (!h || !dev_ptr || ((uintptr_t)dev_ptr % kNsAlign) != 0) return TFS_ERR_ARG;
    if (bytes < ns_bytes(h)) return TFS_ERR_NOWORKSPACE;
    h->ws = (char*)dev_ptr;
    h->ws_bytes = bytes;
    ns_layout(h);
    h->state_set = false;
    return TFS_OK;
}

int tfs_ns_set_state(tfs_ns_handle h, const void* u0, const void* u_prev, void* stream) {
    if (!h || !u0) return TFS_ERR_ARG;
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    return h->precision == TFS_FP64
               ? ns_set_state<double>(h, (const double*)u0, (const double*)u_prev, (cudaStream_t)stream)
               : ns_set_state<float>(h, (const float*)u0, (const float*)u_prev, (cudaStream_t)stream);
}

int tfs_ns_step(tfs_ns_handle h, const void* sigma, void* u_out, void* grad_u_out, void* stream) {
    if (!h) return TFS_ERR_ARG;
    if (!h->ws) return TFS_ERR_NOWORKSPACE;
    if (!h->state_set) return TFS_ERR_STATE;
    return h->precision == TFS_FP64
               ? ns_step<double>(h, (const double*)sigma, (double*)u_out, (double*)grad_u_out, (cudaStream_t)stream)
               : ns_step<float>(h, (const float*)sigma, (float*)u_out, (float*)grad_u_out, (cudaStream_t)stream);
}

int tfs_ns_destroy(tfs_ns_handle h) {
    delete h;
    return TFS_OK;
}

}  // extern "C"
