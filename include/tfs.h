/*
 * tfs.h -- C ABI of the time-fractional polymer-stress step (libtfs.so).
 *
 * The library advances the polymer extra stress of the macroscopic model of
 * Beddrich, Lunowa & Wohlmuth (arXiv 2411.17294) on a periodic grid, one time
 * step per call, on one CUDA GPU (sm_103a).  The law it integrates is the
 * stress form of the macroscopic Fokker-Planck system of Section 3.4
 * (eq. macroscopic_fokker_planck, coupling eqs. mm_contribution_order0 and
 * mm_coupling_order2, stress eq. mm_ExtraStress):
 *
 *   D^alpha_C (sigma - sigma0) = kappa sigma + sigma kappa^T - sigma / Wi
 *                                + G (kappa + kappa^T) t^(alpha-1)/Gamma(alpha)
 *                                - u . grad sigma + eps Lap sigma,
 *   G = (1 - beta) / (Wi Re),   kappa_ij = d u_i / d x_j,
 *
 * with the Caputo kernel t^-alpha/Gamma(1-alpha) compressed into a sum of m
 * exponentials (Section 2.2, eq. tf_approximate_kernel); every grid point
 * carries m mode tensors advanced by BDF2 (Section 4.1, eq. BDF_Phi_k_n+1) and
 * the stress solves, per point, the small system obtained by inserting that
 * push-forward into the mode sum (the eta, eta_k form of eq. FP_discrete):
 *
 *   (eta + dt/Wi) sigma^{n+1} - dt (kappa* sigma^{n+1} + sigma^{n+1} kappa*^T)
 *     = eta sigma0 - sum_j eta_j (b1 sigma_j^n + b2 sigma_j^{n-1})
 *       + dt G (kappa* + kappa*^T) g(t_{n+1}) - dt (u . grad_h - eps Lap_h) E,
 *   kappa* = 2 kappa^n - kappa^{n-1},  E = 2 sigma^n - sigma^{n-1}
 *   (extrapolation of eq. BDF_and_extrapolation).
 * alpha = 1 is plain BDF2 (Oldroyd-B) with no modes.
 *
 * Conventions
 *   Grid: periodic, n[0] x n[1] (x n[2]) points, x fastest: p = x + n0 (y + n1 z).
 *   Packed stress components nc = 3 in 2D (xx, xy, yy), 6 in 3D
 *   (xx, yy, zz, yz, xz, xy).  Stress fields are [nc][N] structure-of-arrays.
 *   Velocity gradient [d*d][N] with component i*d + j = d u_i / d x_j;
 *   velocity [d][N].
 *   Element type of every field pointer: double for TFS_FP64, float for
 *   TFS_FP32 / TFS_FP32_PLAIN.  Gradients returned by tfs_backward are double.
 *   All field pointers are device pointers owned by the caller; the library
 *   allocates no device memory: its state lives in a caller-bound workspace.
 *   Streams: a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls that take a stream only enqueue work on it; they do not synchronise.
 *
 * Errors: every call returns a TFS_* status (0 = TFS_OK).  Kernel-side
 * conditions (non-finite result, near-singular point system, Courant limit
 * exceeded) are latched in a device word and read by tfs_status.
 */
#ifndef TFS_H
#define TFS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tfs_ctx* tfs_handle;

/* status codes */
enum {
    TFS_OK = 0,
    TFS_ERR_ARG = 1,          /* invalid argument (size, range, NULL, alignment) */
    TFS_ERR_NOSOE = 2,        /* alpha < 1 and no SOE table set */
    TFS_ERR_UNSTABLE = 3,     /* declared velocity bound exceeds the explicit-transport limit
                                 (tfs_set_param(TFS_PARAM_UMAX) or, once the SOE is known, tfs_step) */
    TFS_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    TFS_ERR_STATE = 5,        /* call out of order (no state set, adjoint not begun, ...) */
    TFS_ERR_NOWORKSPACE = 6,  /* no (or too small a) workspace bound */
    TFS_ERR_FORMAT = 7,       /* checkpoint buffer does not match this handle */
    TFS_ERR_TOOBIG = 8        /* problem state exceeds the fixed array of tfs_run_static */
};

/* precision modes */
enum {
    TFS_FP64 = 0,             /* everything in double */
    TFS_FP32 = 1,             /* float storage, compensated mode sum, FP64-accurate point solve */
    TFS_FP32_PLAIN = 2        /* float storage, plain float mode sum (precision studies) */
};

/* tfs_set_param keys */
enum {
    TFS_PARAM_RE = 0,         /* Reynolds number, default 1 */
    TFS_PARAM_EPS = 1,        /* centre-of-mass diffusion eps >= 0, default 0 */
    TFS_PARAM_STENCIL = 2,    /* TFS_STENCIL_*, default upwind3 */
    TFS_PARAM_TRANSPORT = 3,  /* 0: pointwise law (u ignored); 1: explicit transport (default);
                                 2: implicit transport -- u.grad and eps Lap at t_{n+1} inside a global
                                 solve, the form of the paper's eq. FP_discrete: block-Jacobi
                                 preconditioned BiCGStab on a float copy of the system inside an FP64
                                 defect correction (the result meets the FP64 residual target; FP64
                                 BiCGStab finishes if the float passes stall), no Courant limit;
                                 the workspace grows by ((10 + 2 nc) nc + 4 d) N doubles plus
                                 (2 nc^2 + 4 d + 9 nc) N floats; tfs_step then synchronises its
                                 stream; tfs_backward solves the transposed system per step with the
                                 same solver (either form, either start) */
    TFS_PARAM_UMAX = 4,       /* declared bound U on |u_a|; checked against tfs_transport_limit */
    TFS_PARAM_KRYLOV_TOL = 5, /* implicit transport: relative residual target, default 1e-13 (FP64)
                                 or 1e-9 (FP32 storage) */
    TFS_PARAM_KRYLOV_MAXIT = 6, /* implicit transport: iteration limit of each Krylov run (each float
                                   pass of the defect correction, the FP64 finish), default 500 */
    TFS_PARAM_START = 7,      /* first step from the initial state, TFS_START_*: BDF2 with an empty
                                 past (default), or the two-stage SDIRK2 the paper takes for
                                 non-trivial initial data (Section 5.1; gamma = 1 - 1/sqrt2, stiffly
                                 accurate, L-stable; kappa of the first call, both stage systems solved
                                 in FP64).  SDIRK2 needs alpha < 1 (else TFS_ERR_ARG here) and transport
                                 0 or 2: with explicit transport the first tfs_step returns TFS_ERR_ARG.
                                 With transport 2 both stage systems go through the implicit solver
                                 (tfs_last_solve: iterations summed, larger residual).  With
                                 TFS_FORM_PAPER the same method on Phi and its modes.  tfs_backward
                                 differentiates the start (zero initial modes, as tfs_set_state leaves
                                 them) with transport 0 or 2 in either form */
    TFS_PARAM_FORM = 8        /* variable carried, TFS_FORM_*: the stress (default), or the paper's own
                                 variable (Section 3.4): Phi with d Phi/dt = (L(kappa) - I/Wi) Psi +
                                 G (kappa + kappa^T) Psi0, Psi = D^{1-alpha} Phi by kernel compression of
                                 g_alpha = t^(alpha-1)/Gamma(alpha), so the SOE table of tfs_set_soe
                                 approximates g_alpha (the Caputo kernel of order 1 - alpha); Psi0 =
                                 D^{1-alpha} 1 from the same modes, on the host.  The stress returned is
                                 Psi (zero before the first step); tfs_set_state sets Phi(0) (NULL: 0).
                                 BDF2 on Phi and the modes (Section 4.1), one point system per point.
                                 With transport 1 the operator u.grad - eps Lap acts on the
                                 extrapolation 2 Psi^n - Psi^{n-1}, explicitly, with the stencils of the
                                 stress form; tfs_transport_limit, the eps and umax checks and the
                                 Courant flag then use this variable's own bound (the transport acts on
                                 Psi = V Phi, V the discrete D^{1-alpha}, which makes it far tighter for
                                 small alpha).  With transport 2 it acts on
                                 Psi^{n+1} = xi Phi^{n+1} + h inside the solve (eq. FP_discrete): the
                                 operator (b0 + dt xi/Wi) I - dt xi L(kappa*) + dt xi (u.grad - eps Lap)
                                 through the same Krylov solver, and one more nc N FP64 vector.  Needs
                                 alpha < 1 (else TFS_ERR_ARG here); either start (SDIRK2 with transport
                                 0 or 2, else tfs_step returns TFS_ERR_ARG); tfs_backward takes it
                                 with every transport mode and start the step takes.  The workspace grows by 2 nc N elements (Psi^n, Psi^{n-1});
                                 with a workspace bound, a form it does not fit returns TFS_ERR_NOWORKSPACE.
                                 Changing the form discards the state (call tfs_set_state again) */
};

/* first-step methods (TFS_PARAM_START) */
enum { TFS_START_BDF2 = 0, TFS_START_SDIRK2 = 1 };

/* variables carried (TFS_PARAM_FORM) */
enum { TFS_FORM_STRESS = 0, TFS_FORM_PAPER = 1 };

enum { TFS_STENCIL_UPWIND3 = 0, TFS_STENCIL_CENTRAL2 = 1 };

/* device status flags (tfs_status) */
enum {
    TFS_FLAG_NONFINITE = 1u,  /* a new stress value was NaN or Inf */
    TFS_FLAG_SINGULAR = 2u,   /* a point system had a pivot below 1e-300 / relative 1e-14 */
    TFS_FLAG_COURANT = 4u,    /* a point had dt sum_a |u_a|/h_a above the limit of tfs_transport_limit */
    TFS_FLAG_TIMEOUT = 8u,    /* a kernel gave up waiting for its own tile copies (bounded wait; the
                                 step's output is then incomplete) */
    TFS_FLAG_NOCONV = 16u     /* an implicit-transport solve stopped above its tolerance (the best
                                 iterate was kept) */
};

typedef struct {
    int dim;        /* 2 or 3 */
    int n[3];       /* points per axis (n[2] ignored in 2D); each >= 1 */
    double L[3];    /* box lengths > 0 */
} tfs_grid;

/* Create a handle for the problem of Section 4.1 on the periodic grid:
   fractional order alpha and Weissenberg number Wi of the time-fractional
   Fokker-Planck equation (eq. timefractionalFokkerPlanck; Wi the relaxation
   time, the paper's 2 De), solvent fraction beta of the momentum equation
   (eq. Navier_Stokes: G = (1 - beta)/(Wi Re) scales the stress source), m
   kernel-compression modes (Section 2.2) and the step dt of eq.
   BDF_and_extrapolation.  alpha in (0, 1]; Wi > 0; beta in [0, 1); dt > 0;
   0 <= m <= 64 (m = 0 required when alpha == 1, m >= 1 otherwise);
   precision one of TFS_FP64, TFS_FP32, TFS_FP32_PLAIN.  No device memory is
   allocated.  On error *h is set to NULL. */
int tfs_create(tfs_handle* h, const tfs_grid* grid, double alpha, double Wi, double beta,
               int m, double dt, int precision);

/* Set an optional parameter (TFS_PARAM_*).  Re > 0, eps >= 0, umax >= 0.
   With transport on and the SOE known, an eps or umax beyond the stability
   limit of tfs_transport_limit returns TFS_ERR_UNSTABLE (and is not set). */
int tfs_set_param(tfs_handle h, int key, double value);

/* Kernel compression of Section 2.2 (eq. tf_approximate_kernel).
   Copy the SOE table: exponents mu_j >= 0 and weights w_j >= 0 (finite),
   j < m, approximating t^-alpha/Gamma(1-alpha) by sum_j w_j exp(-mu_j t)
   (Section 2.2).  Host arrays, copied; m must equal the handle's m.
   Precomputes c_j = 1/(b0 + mu_j dt), rho_j = w_j dt c_j, eta_j = mu_j dt c_j
   and eta = b0 sum_j rho_j in FP64. */
int tfs_set_soe(tfs_handle h, const double* mu, const double* w, int m);

/* Largest velocity bound U (TFS_PARAM_UMAX) for which the explicit transport
   is stable.  From a von Neumann analysis of the step with the handle's SOE
   table (relaxation and kappa ignored): lambda* is the largest dt|u|/h for
   which the stencil symbol keeps the step's characteristic function free of
   zeros in the unit disk, z* the same for the diffusion symbol; the step is
   accepted while dt U sum_a 1/h_a / lambda* + 4 eps dt sum_a 1/h_a^2 / z* <= 0.9.
   Returns U >= 0 (0 when eps alone uses the whole margin).  Requires the SOE
   when alpha < 1 (TFS_ERR_NOSOE).  Host only; computed once per SOE/stencil. */
int tfs_transport_limit(tfs_handle h, double* umax_out);

/* Bytes of device workspace the handle needs: 256 (status) + 5 fields of
   nc N elements (sigma0 copy, stress ring of 3, transport term) + 2 mode levels
   of m nc ceil(N/32)*32 elements (stored tile by tile: the m nc values of 32
   consecutive points are contiguous), each rounded up to 256 bytes; more with
   the paper's variable or implicit transport (see TFS_PARAM_FORM and
   TFS_PARAM_TRANSPORT). */
size_t tfs_workspace_bytes(tfs_handle h);

/* Bind caller-owned device memory of at least tfs_workspace_bytes bytes,
   256-byte aligned.  The library never frees it. */
int tfs_bind_workspace(tfs_handle h, void* dev_ptr, size_t bytes);

/* Initial conditions of eq. amnsfp_initial_conditions: the stress (or Phi
   with TFS_FORM_PAPER) starts at sigma0 [nc][N] (device, element type of the
   handle; NULL = zero stress, the paper's start from rest) and every
   fractional mode at zero; sigma^{-1} = sigma^0 (the empty past of the BDF2
   start), step counter 0, status flags cleared.  TFS_ERR_NOWORKSPACE without
   a workspace; enqueues on `stream`. */
int tfs_set_state(tfs_handle h, const void* sigma0, void* stream);

/* One step t_n -> t_{n+1} of eq. FP_discrete with the mode push-forward of
   eq. BDF_Phi_k_n+1 and the extrapolated gradient kappa* = 2 kappa^n -
   kappa^{n-1} of eq. BDF_and_extrapolation.  grad_u_n = kappa^n, grad_u_nm1
   = kappa^{n-1} [d*d][N] (NULL = same as grad_u_n); u = velocity [d][N]
   (NULL allowed when transport is off); device pointers of the handle's
   element type, read only.  Enqueues the step kernel, preceded by the
   transport pre-pass when transport is explicit (transport 2: the Krylov
   solve, which synchronises `stream`).  TFS_ERR_STATE before tfs_set_state,
   TFS_ERR_NOSOE without a table, TFS_ERR_UNSTABLE when a declared velocity
   bound exceeds the explicit limit, TFS_ERR_CUDA on a failed launch. */
int tfs_step(tfs_handle h, const void* grad_u_n, const void* grad_u_nm1, const void* u, void* stream);

/* Copy the current polymer stress to out [nc][N] (device, caller-owned,
   element type of the handle): sigma^n, the degree-2 part of Psi of eq.
   mm_ExtraStress in the packed units of eq. mm_coupling_order2; with
   TFS_FORM_PAPER the stress Psi^n = D^{1-alpha} Phi^n.  Enqueues a copy on
   `stream`; TFS_ERR_STATE before tfs_set_state. */
int tfs_get_stress(tfs_handle h, void* out, void* stream);

/* Slab decomposition (for running one periodic domain on several GPUs).  The
   paper's runtime partitions its meshes over MPI ranks (Section 5, the
   experimental setup); this is the library's counterpart for the periodic
   grid: the domain is cut along its slowest axis (z in 3D, y in 2D) into
   slabs, one handle per slab created with the slab's own grid (n[d-1] its
   plane count, L[d-1] its length, the other axes those of the whole domain).
   Every point's update is local except the transport stencil, which reaches
   R = 2 planes into the neighbouring slabs; each step therefore takes the
   neighbours' boundary planes of sigma^n and sigma^{n-1} (both enter E =
   2 sigma^n - sigma^{n-1}).  A slab step of the stress form with explicit
   transport (or none) gives, at every point, the same result as the step of
   the whole domain.
   A halo buffer is [2 levels][nc][R][plane] elements of the handle's type
   (level 0 sigma^n, level 1 sigma^{n-1}; plane = n[0] points in 2D, n[0] n[1]
   in 3D, x fastest), device memory owned by the caller; tfs_halo_bytes gives
   its size (0 for an invalid handle). */
size_t tfs_halo_bytes(tfs_handle h);

/* The slab's own boundary planes as its neighbours need them, after the last
   step (or tfs_set_state): lo <- its first R planes (the lower neighbour's
   halo_hi), hi <- its last R planes (the upper neighbour's halo_lo); either
   may be NULL.  Enqueues device copies on `stream`.  TFS_ERR_ARG for the
   paper's variable or a slab thinner than R planes. */
int tfs_get_halo(tfs_handle h, void* lo, void* hi, void* stream);

/* One step of a slab: tfs_step with the planes beyond the slab's ends read
   from halo_lo (the lower neighbour's last R planes: slab coordinates -R ..
   -1) and halo_hi (the upper neighbour's first R planes: n[d-1] .. n[d-1] + R
   - 1) instead of wrapping around the slab.  Stress form with transport 0 or
   1 (TFS_ERR_ARG otherwise, and for NULL halos); other errors as tfs_step.
   The halos are read by the transport pre-pass, on `stream`. */
int tfs_step_slab(tfs_handle h, const void* grad_u_n, const void* grad_u_nm1, const void* u, const void* halo_lo,
                  const void* halo_hi, void* stream);

/* Measurement hook (no counterpart in the paper): with two cudaEvent_t
   (passed as void*, both or neither), every later tfs_step records ev_before
   on its stream just before the step kernel and ev_after just after it (the
   transport pre-pass runs before ev_before), so that the step kernel alone
   can be timed.  NULL, NULL turns it off.  The events are not owned. */
int tfs_set_step_events(tfs_handle h, void* ev_before, void* ev_after);

/* Current step index n (number of completed steps since tfs_set_state). */
long tfs_step_index(tfs_handle h);

/* Check of the bounded device wait (no counterpart in the paper).  Every
   mbarrier wait of the library gives up after about 2 s, latches
   TFS_FLAG_TIMEOUT and lets its kernel return, so that a copy that never
   completes cannot hang the GPU.  This launches one block whose thread waits
   on an mbarrier that nothing arrives at, through that same wait, and reports
   the flag it latched (*flags, TFS_FLAG_TIMEOUT when the wait gave up) and the
   time the wait took (*seconds).  Synchronises `stream`; allocates nothing
   (a file-scope device array holds the result).  TFS_ERR_ARG for NULL
   pointers, TFS_ERR_CUDA if the launch or copy fails. */
int tfs_check_wait_bound(unsigned* flags, double* seconds, void* stream);

/* Iterations and final relative residual |b - Op x| / |b| of the last
   implicit-transport solve (TFS_PARAM_TRANSPORT = 2): a step's (the SDIRK2
   start: its two stages summed, the larger residual), or after tfs_backward
   its last reverse step's transposed solve(s); either pointer may be NULL.
   Host-side, no synchronisation. */
int tfs_last_solve(tfs_handle h, int* iterations, double* relative_residual);

/* Checkpoints: a device buffer holding the full state (header, stress at
   levels n and n-1, the initial stress, modes at levels n and n-1; with
   TFS_FORM_PAPER the levels of Phi in place of the stress, then Psi^n). */
size_t tfs_checkpoint_bytes(tfs_handle h);
int tfs_save(tfs_handle h, void* dst, void* stream);
/* Restore a checkpoint written by tfs_save on a handle of the same shape and
   precision (checked: TFS_ERR_FORMAT).  Synchronises `stream` to read the
   header. */
int tfs_load(tfs_handle h, const void* src, void* stream);

/* Adjoint workspace for checkpoint segments of `segment_steps` steps. */
size_t tfs_adjoint_workspace_bytes(tfs_handle h, int segment_steps);
int tfs_bind_adjoint_workspace(tfs_handle h, void* dev_ptr, size_t bytes);

/* Adjoint of the scheme of eq. FP_discrete / eq. BDF_Phi_k_n+1 (the paper
   computes no gradients: this is the exact reverse of the discrete steps that
   tfs_step takes).
   Reverse-mode derivative of J(sigma^T) for a run of `steps` steps from the
   state set by tfs_set_state, with a frozen velocity gradient grad_u [d*d][N]
   (and velocity u when transport is on), given dJ/dsigma(T) [nc][N] (element
   type of the handle).  checkpoints[k] must hold tfs_save of step k*K for
   k = 0 .. ceil(steps/K)-1; each segment is recomputed from its checkpoint
   and then differentiated backwards.  Outputs (device, double): dJ_dsigma0
   [nc][N], dJ_dgrad_u [d*d][N]; host doubles *dJ_dWi, *dJ_dbeta.  Synchronises
   `stream` at the end to return the two scalars.  The handle's forward state
   afterwards is that of the last recomputed segment.  With TFS_FORM_PAPER,
   J is a function of Psi(T) and dJ_dsigma0 is the derivative in Phi(0). */
int tfs_backward(tfs_handle h, const void* dJ_dsigma_T, const void* const* checkpoints, int K,
                 int steps, const void* grad_u, const void* u, double* dJ_dsigma0,
                 double* dJ_dgrad_u, double* dJ_dWi, double* dJ_dbeta, void* stream);

/* Read (and keep) the latched device flags; synchronises the last stream
   the handle used.  Returns TFS_OK or TFS_ERR_CUDA. */
int tfs_status(tfs_handle h, unsigned* device_flags);

/* Static description of a status code. */
const char* tfs_strerror(int code);

/* Free the handle (host memory only). */
int tfs_destroy(tfs_handle h);

/* Run `steps` steps from sigma0 without any workspace, for callers that cannot
   allocate device memory (code running where cudaMalloc is not allowed: a host
   framework that owns all device memory, an allocation-free real-time loop, a
   plug-in without an allocator).  The paper has no counterpart: this is an
   interface convenience around the same step kernel.
   The whole state (stress ring, sigma0 copy, transport term, status word, both mode levels)
   lives in one fixed device array of 64 MiB compiled into the library, which
   every GPU that loads the library holds until the process exits; problems
   whose state needs more (256 + 5 up256(nc N s) + 2 up256(m nc ceil(N/32)*32 s) bytes,
   s = element size, up256 = round up to 256) return TFS_ERR_TOOBIG before any
   device work.  Arguments as tfs_create / tfs_set_soe (mu, w: host, m
   entries, NULL when alpha == 1); Re = 1, eps = 0, upwind3 stencil, transport
   on iff u != NULL (points beyond the velocity limit of tfs_transport_limit
   latch TFS_FLAG_COURANT; nothing is refused); sigma0 [nc][N] (NULL = zero), grad_u
   [d*d][N] frozen for all steps, sigma_out [nc][N]: device pointers of the
   precision's element type.  Enqueues on `stream` and returns; the result is
   in sigma_out once the stream reaches it.  The array's device address is
   looked up on the first call on each device (with that device current): make
   that first call before any stream capture.  Every call shares the array and
   clears it at its start, so calls whose GPU work overlaps (other streams or
   host threads) race and must not be issued.  The device flags its kernels
   latch (TFS_FLAG_*) stay in the array: read them with tfs_static_status.
   Allocates nothing. */
int tfs_run_static(const tfs_grid* grid, double alpha, double Wi, double beta, int m, double dt,
                   int precision, const double* mu, const double* w, const void* sigma0,
                   const void* grad_u, const void* u, int steps, void* sigma_out, void* stream);

/* Device flags (TFS_FLAG_*) latched by the most recent tfs_run_static on the
   current device, which has no handle to ask through tfs_status: a non-finite
   result, a near-singular point system, the Courant limit exceeded, or a
   bounded wait that gave up.  Synchronises `stream` (pass the stream of that
   run) and copies the word from the library's fixed array into
   *device_flags; allocates nothing.  The paper has no counterpart.
   TFS_ERR_ARG for NULL, TFS_ERR_CUDA if the copy fails. */
int tfs_static_status(unsigned* device_flags, void* stream);

/* ---- The velocity the stress is coupled to: one Navier-Stokes projection
   step on the periodic square (Section 4.1: BDF2 with the extrapolation of
   eq. BDF_and_extrapolation, the rotational viscous term of eq.
   velocity_correction in the pressure equation eq. NS_Poisson, the velocity
   from the Helmholtz equation eq. NS_Helmholtz, the polymer stress entering as
   its divergence, eq. Navier_Stokes).  Fourier spectral derivatives (d/dx_a
   multiplies mode k by i k_a, zero at the Nyquist wavenumber; the Laplacian
   is its square), so Poisson and Helmholtz are divisions per mode and the
   velocity stays divergence-free; the transforms are the library's own FFT
   kernels.  Internal state FP64; the fields exchanged with the caller are of
   the precision given at creation (double for TFS_FP64, else float), so that
   they feed the stress handle directly.  A coupled step, in the paper's
   order: tfs_ns_step(sigma^n) -> u^{n+1}, kappa^{n+1}, then tfs_step(h,
   kappa^{n+1}, kappa^{n+1}, u^{n+1}) (the stress step with kappa* =
   kappa^{n+1}, the velocity already known). */
typedef struct tfs_ns_ctx* tfs_ns_handle;

/* Grid n0 x n1 (powers of two, 2 .. 1024), box L0 x L1, solvent fraction beta
   in (0, 1] and Reynolds number Re > 0 (viscosity beta/Re), step dt > 0,
   precision as tfs_create.  No device memory is allocated; on error *h = NULL. */
int tfs_ns_create(tfs_ns_handle* h, int n0, int n1, double L0, double L1, double beta, double Re, double dt,
                  int precision);

/* Device workspace of the handle: 21 complex and 8 real FP64 fields of n0 n1
   values and the transforms' twiddle tables (n0/2 + n1/2 complex), each
   rounded up to 256 bytes. */
size_t tfs_ns_workspace_bytes(tfs_ns_handle h);

/* Bind caller-owned device memory (256-byte aligned) of at least
   tfs_ns_workspace_bytes bytes; discards the state. */
int tfs_ns_bind_workspace(tfs_ns_handle h, void* dev_ptr, size_t bytes);

/* Initial velocity u0 [2][N] (device; x fastest, N = n0 n1), projected onto
   divergence-free fields.  u_prev = the level one step earlier (projected
   too) or NULL for an empty past (u^{-1} = u^0 and the previous explicit
   terms equal to the first ones).  Enqueues on `stream`. */
int tfs_ns_set_state(tfs_ns_handle h, const void* u0, const void* u_prev, void* stream);

/* One step with the polymer stress sigma^n [3][N] (packed xx, xy, yy, as
   tfs_get_stress returns it; NULL = no stress): writes u^{n+1} [2][N] and the
   velocity gradient kappa^{n+1} [4][N] (kappa_ij = du_i/dx_j at i*2 + j);
   either output may be NULL.  Enqueues on `stream`; TFS_ERR_STATE before
   tfs_ns_set_state, TFS_ERR_NOWORKSPACE without a workspace. */
int tfs_ns_step(tfs_ns_handle h, const void* sigma, void* u_out, void* grad_u_out, void* stream);

/* Free the handle (host memory only). */
int tfs_ns_destroy(tfs_ns_handle h);

#ifdef __cplusplus
}
#endif

#endif /* TFS_H */
