/*
 * Plain FP64 CPU oracle for one time step of the fractional polymer-stress law.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file; only the tests, the package smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes (Beddrich, Lunowa & Wohlmuth, arXiv 2411.17294):
 *
 *   The macroscopic system of Section 3.4 (eq. macroscopic_fokker_planck) with
 *   Psi := D^{1-alpha} Phi (the Riemann-Liouville derivative of Section 1,
 *   eq. RiemannLiouvilleFractionalDerivative) satisfies exactly
 *       D^alpha Psi + (u.grad - eps Lap) Psi = A(grad u) Psi,
 *   and the stress of eq. mm_ExtraStress is proportional to the degree-2 part of
 *   Psi.  Written for the symmetric stress sigma (units S_ii = sqrt2 phi_{2e_i},
 *   S_ij = phi_{e_i+e_j}, in which the 6x6 block A_2 of eq. mm_coupling_order2 is
 *   kappa S + S kappa^T and the vector K of eq. mm_contribution_order0, with the
 *   sqrt2 kappa_ii of eq. conf_op_tested, is kappa + kappa^T):
 *
 *     D^alpha_C (sigma - sigma0) = kappa sigma + sigma kappa^T - sigma / Wi
 *                                  + G (kappa + kappa^T) g_alpha(t)
 *                                  - u.grad sigma + eps Lap sigma,
 *     G = (1 - beta) / (Wi Re),   g_alpha(t) = t^(alpha-1) / Gamma(alpha),
 *     kappa_ij = d u_i / d x_j.
 *
 *   The Caputo kernel t^-alpha / Gamma(1-alpha) is replaced by the sum of
 *   exponentials sum_j w_j exp(-mu_j t) (Section 2.2, eq. tf_approximate_kernel),
 *   which turns the derivative into m mode ODEs (eq. fractional_modes_equations)
 *   and the derivative into sum_j (-mu_j f_j + w_j f)
 *   (eq. fractional_modes_fractional_derivative).  The modes are advanced by
 *   BDF2 (Section 4.1, eq. BDF_and_extrapolation with b = (3/2, -2, 1/2)) and
 *   solved for explicitly (eq. BDF_Phi_k_n+1).  Inserting the push-forward in the
 *   mode sum gives the eta and eta_k coefficients of eq. FP_discrete, with which
 *   the step for the stress becomes, at every grid point,
 *
 *     kappa* = 2 kappa^n - kappa^{n-1}            (extrapolation, a_1=2, a_2=-1)
 *     E      = 2 sigma^n - sigma^{n-1}
 *     A      = dt sum_a u_a D_a(E) - eps dt Lap(E) (explicit transport)
 *     H      = sum_j eta_j (b1 sigma_j^n + b2 sigma_j^{n-1})
 *     R      = eta sigma0 - H + dt G (kappa* + kappa*^T) g_alpha(t_{n+1}) - A
 *     (eta + dt/Wi) sigma^{n+1} - dt (kappa* sigma^{n+1} + sigma^{n+1} kappa*^T) = R
 *     sigma_j^{n+1} = c_j (-b1 sigma_j^n - b2 sigma_j^{n-1}) + rho_j (sigma^{n+1} - sigma0)
 *
 *   with c_j = 1/(b0 + mu_j dt), rho_j = w_j dt c_j, eta_j = mu_j dt c_j,
 *   eta = b0 sum_j rho_j.  For alpha = 1 (no memory) the derivative is plain BDF2:
 *   eta = b0, H = b1 sigma^n + b2 sigma^{n-1} + b0 sigma0, g = 1.
 *
 * Every operation is written out plainly: the small linear system is assembled
 * column by column by applying the operator to unit vectors and solved by
 * Gaussian elimination with partial pivoting; modes are summed in order
 * j = 0..m-1.  Compile with -O2 -ffp-contract=off and no fast-math.
 *
 * Layouts (all row-major, point index p = x + nx (y + ny z)):
 *   stress fields  [nc][N]   packed components, 2D (xx, xy, yy),
 *                             3D (xx, yy, zz, yz, xz, xy); or [d*d][N] when full
 *   modes          [m][nc][N]
 *   velocity grad  [d*d][N]  component i*d + j holds d u_i / d x_j
 *   velocity       [d][N]
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dim;          /* spatial dimension d: 2 or 3 */
    int n[3];         /* grid points per axis (x fastest); n[2] = 1 in 2D */
    double L[3];      /* periodic box lengths */
    double alpha;     /* fractional order, 0 < alpha <= 1 */
    double Wi;        /* relaxation time */
    double beta;      /* solvent viscosity ratio */
    double Re;        /* Reynolds number */
    double eps;       /* centre-of-mass diffusion coefficient */
    double dt;        /* time step */
    int m;            /* number of SOE terms (ignored when alpha == 1) */
    int stencil;      /* 0: third-order upwind-biased (radius 2); 1: central (radius 1) */
    int transport;    /* 0: pointwise law; 1: include u.grad and eps Lap */
    int full;         /* 0: packed symmetric components; 1: full d x d tensor */
} orc_params;

static const double B0 = 1.5, B1 = -2.0, B2 = 0.5;   /* BDF2, Section 4.1 */

/* packed component c -> tensor index pair */
static const int PK2[3][2] = {{0, 0}, {0, 1}, {1, 1}};
static const int PK3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};

static int ncomp(const orc_params* p) {
    if (p->full) return p->dim * p->dim;
    return p->dim == 2 ? 3 : 6;
}

static void comp_pair(const orc_params* p, int c, int* i, int* j) {
    if (p->full) { *i = c / p->dim; *j = c % p->dim; return; }
    if (p->dim == 2) { *i = PK2[c][0]; *j = PK2[c][1]; }
    else { *i = PK3[c][0]; *j = PK3[c][1]; }
}

/* vector of components -> d x d matrix (symmetric fill when packed) */
static void to_matrix(const orc_params* p, const double* v, double S[3][3]) {
    int nc = ncomp(p);
    memset(S, 0, sizeof(double) * 9);
    for (int c = 0; c < nc; ++c) {
        int i, j;
        comp_pair(p, c, &i, &j);
        S[i][j] = v[c];
        if (!p->full) S[j][i] = v[c];
    }
}

static void from_matrix(const orc_params* p, double S[3][3], double* v) {
    int nc = ncomp(p);
    for (int c = 0; c < nc; ++c) {
        int i, j;
        comp_pair(p, c, &i, &j);
        v[c] = S[i][j];
    }
}

/* out = kappa S + S kappa^T, in component form */
static void upper_convected(const orc_params* p, double K[3][3], const double* s, double* out) {
    int d = p->dim;
    double S[3][3], T[3][3];
    to_matrix(p, s, S);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double acc = 0.0;
            for (int l = 0; l < d; ++l) acc += K[i][l] * S[l][j] + S[i][l] * K[j][l];
            T[i][j] = acc;
        }
    from_matrix(p, T, out);
}

/* Gaussian elimination with partial pivoting; returns 0 on success */
static int gauss_solve(int n, double* A /* n x n row-major, destroyed */, double* b /* in: rhs, out: x */) {
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); piv = i; }
        if (best == 0.0) return 1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double f = A[i * n + k] / A[k * n + k];
            for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double acc = b[i];
        for (int j = i + 1; j < n; ++j) acc -= A[i * n + j] * b[j];
        b[i] = acc / A[i * n + i];
    }
    return 0;
}

/* Assemble the operator  s -> a s - dt (kappa s + s kappa^T)  as a matrix,
   column k = image of the k-th unit vector. */
static void assemble(const orc_params* p, double K[3][3], double a, double* M) {
    int nc = ncomp(p);
    double e[9], img[9];
    for (int k = 0; k < nc; ++k) {
        for (int c = 0; c < nc; ++c) e[c] = (c == k) ? 1.0 : 0.0;
        upper_convected(p, K, e, img);
        for (int r = 0; r < nc; ++r) M[r * nc + k] = a * e[r] - p->dt * img[r];
    }
}

static long wrap(long i, long n) { long r = i % n; return r < 0 ? r + n : r; }

static long pidx(const orc_params* p, long x, long y, long z) {
    return x + (long)p->n[0] * (y + (long)p->n[1] * z);
}

/* first derivative of field f along axis a at (x,y,z), upwinded on the sign of v */
static double deriv(const orc_params* p, const double* f, int a, long x, long y, long z, double v) {
    long c[3] = {x, y, z};
    double h = p->L[a] / p->n[a];
    double s[5];   /* f at offsets -2..2 along axis a */
    for (int k = -2; k <= 2; ++k) {
        long q[3] = {c[0], c[1], c[2]};
        q[a] = wrap(c[a] + k, p->n[a]);
        s[k + 2] = f[pidx(p, q[0], q[1], q[2])];
    }
    if (p->stencil == 1) return (s[3] - s[1]) / (2.0 * h);
    if (v >= 0.0) return (s[0] - 6.0 * s[1] + 3.0 * s[2] + 2.0 * s[3]) / (6.0 * h);
    return (-2.0 * s[1] - 3.0 * s[2] + 6.0 * s[3] - s[4]) / (6.0 * h);
}

static double laplace(const orc_params* p, const double* f, long x, long y, long z) {
    long c[3] = {x, y, z};
    double acc = 0.0;
    for (int a = 0; a < p->dim; ++a) {
        double h = p->L[a] / p->n[a];
        long qm[3] = {c[0], c[1], c[2]}, qp[3] = {c[0], c[1], c[2]};
        qm[a] = wrap(c[a] - 1, p->n[a]);
        qp[a] = wrap(c[a] + 1, p->n[a]);
        acc += (f[pidx(p, qm[0], qm[1], qm[2])] - 2.0 * f[pidx(p, x, y, z)] + f[pidx(p, qp[0], qp[1], qp[2])]) / (h * h);
    }
    return acc;
}

static long npoints(const orc_params* p) { return (long)p->n[0] * p->n[1] * (p->dim == 3 ? p->n[2] : 1); }

/* per-step scalars of Section 4.1 */
typedef struct { double eta, a, G, g; } step_scalars;

static step_scalars scalars(const orc_params* p, const double* mu, const double* w, long step_index) {
    step_scalars s;
    double t = (double)(step_index + 1) * p->dt;
    if (p->alpha == 1.0) {
        s.eta = B0;
        s.g = 1.0;
    } else {
        double eta = 0.0;
        for (int j = 0; j < p->m; ++j) {
            double c = 1.0 / (B0 + mu[j] * p->dt);
            eta += B0 * w[j] * p->dt * c;
        }
        s.eta = eta;
        s.g = pow(t, p->alpha - 1.0) / tgamma(p->alpha);
    }
    s.a = s.eta + p->dt / p->Wi;
    s.G = (1.0 - p->beta) / (p->Wi * p->Re);
    return s;
}

int orc_ncomp(const orc_params* p) { return ncomp(p); }

/*
 * One forward step t_n -> t_{n+1} on the whole grid.  Inputs are not modified;
 * sig_np1 [nc][N] and modes_np1 [m][nc][N] receive the new level.
 * u may be NULL when transport == 0.  Returns the number of singular systems.
 */
int orc_step(const orc_params* p, const double* mu, const double* w, long step_index,
             const double* sig_n, const double* sig_nm1,
             const double* modes_n, const double* modes_nm1,
             const double* sigma0,
             const double* kap_n, const double* kap_nm1, const double* u,
             double* sig_np1, double* modes_np1) {
    const int d = p->dim, nc = ncomp(p);
    const long N = npoints(p);
    const int classic = (p->alpha == 1.0);
    const int m = classic ? 0 : p->m;
    step_scalars s = scalars(p, mu, w, step_index);
    int failures = 0;

    /* extrapolated stress E = 2 sigma^n - sigma^{n-1}, needed at neighbours */
    double* E = (double*)malloc(sizeof(double) * (size_t)nc * (size_t)N);
    for (long q = 0; q < (long)nc * N; ++q) E[q] = 2.0 * sig_n[q] - sig_nm1[q];

#pragma omp parallel for schedule(static) reduction(+ : failures)
    for (long pt = 0; pt < N; ++pt) {
        long x = pt % p->n[0];
        long y = (pt / p->n[0]) % p->n[1];
        long z = (d == 3) ? pt / ((long)p->n[0] * p->n[1]) : 0;

        double K[3][3] = {{0}};
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                long q = (long)(i * d + j) * N + pt;
                K[i][j] = 2.0 * kap_n[q] - kap_nm1[q];
            }

        double R[9], sym[9], Kmat[9 * 9];
        double KS[3][3];
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) KS[i][j] = K[i][j] + K[j][i];
        from_matrix(p, KS, sym);

        for (int c = 0; c < nc; ++c) {
            double H;
            if (classic) {
                H = B1 * sig_n[(long)c * N + pt] + B2 * sig_nm1[(long)c * N + pt] + B0 * sigma0[(long)c * N + pt];
            } else {
                H = 0.0;
                for (int j = 0; j < m; ++j) {
                    double cj = 1.0 / (B0 + mu[j] * p->dt);
                    double etaj = mu[j] * p->dt * cj;
                    long q = ((long)j * nc + c) * N + pt;
                    H += etaj * (B1 * modes_n[q] + B2 * modes_nm1[q]);
                }
            }
            double A = 0.0;
            if (p->transport) {
                const double* Ec = E + (long)c * N;
                for (int a = 0; a < d; ++a) {
                    double va = u[(long)a * N + pt];
                    A += p->dt * va * deriv(p, Ec, a, x, y, z, va);
                }
                if (p->eps != 0.0) A -= p->eps * p->dt * laplace(p, Ec, x, y, z);
            }
            R[c] = s.eta * sigma0[(long)c * N + pt] - H + p->dt * s.G * sym[c] * s.g - A;
        }

        assemble(p, K, s.a, Kmat);
        double x_[9];
        for (int c = 0; c < nc; ++c) x_[c] = R[c];
        if (gauss_solve(nc, Kmat, x_)) failures += 1;
        for (int c = 0; c < nc; ++c) sig_np1[(long)c * N + pt] = x_[c];

        for (int j = 0; j < m; ++j) {
            double cj = 1.0 / (B0 + mu[j] * p->dt);
            double rhoj = w[j] * p->dt * cj;
            for (int c = 0; c < nc; ++c) {
                long q = ((long)j * nc + c) * N + pt;
                modes_np1[q] = cj * (-B1 * modes_n[q] - B2 * modes_nm1[q])
                             + rhoj * (x_[c] - sigma0[(long)c * N + pt]);
            }
        }
    }
    free(E);
    return failures;
}

/* Dense matrix of  S -> a S_p - dt L(kappa*_p) S_p + dt [sum_a u_a D_a(S) - eps Lap(S)]_p
   over the grid (n = nc N unknowns, unknown k = component * N + point), column by
   column: the image of each unit field.  unit is N doubles of zeros (scratch). */
static void assemble_global(const orc_params* p, const double* kap_n, const double* kap_nm1, const double* u,
                            double a, double* G, double* unit) {
    const int d = p->dim, nc = ncomp(p);
    const long N = npoints(p);
    const long n = (long)nc * N;
    /* columns: unknown k = (component ck, point pk) */
    for (long k = 0; k < n; ++k) {
        const int ck = (int)(k / N);
        const long pk = k % N;
        for (long r = 0; r < n; ++r) G[r * n + k] = 0.0;
        /* local part at point pk: the block a I - dt L(kappa*_pk) applied to e_ck */
        {
            double K[3][3] = {{0}};
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    long q = (long)(i * d + j) * N + pk;
                    K[i][j] = 2.0 * kap_n[q] - kap_nm1[q];
                }
            double e[9], img[9];
            for (int c = 0; c < nc; ++c) e[c] = (c == ck) ? 1.0 : 0.0;
            upper_convected(p, K, e, img);
            for (int c = 0; c < nc; ++c) G[((long)c * N + pk) * n + k] += a * e[c] - p->dt * img[c];
        }
        /* transport part: component ck of the unit field is 1 at pk; its image
           is nonzero at the points whose stencils reach pk */
        if (p->transport) {
            unit[pk] = 1.0;
            for (long pt = 0; pt < N; ++pt) {
                long x = pt % p->n[0];
                long y = (pt / p->n[0]) % p->n[1];
                long z = (d == 3) ? pt / ((long)p->n[0] * p->n[1]) : 0;
                double t = 0.0;
                for (int a = 0; a < d; ++a) {
                    double va = u[(long)a * N + pt];
                    t += va * deriv(p, unit, a, x, y, z, va);
                }
                if (p->eps != 0.0) t -= p->eps * laplace(p, unit, x, y, z);
                if (t != 0.0) G[((long)ck * N + pt) * n + k] += p->dt * t;
            }
            unit[pk] = 0.0;
        }
    }

}

/*
 * One step with the transport treated implicitly (the form in which the paper's
 * scheme, eq. FP_discrete, carries u.grad and eps Lap: at t_{n+1}, inside the
 * solve).  The per-point relation becomes a coupled system over the grid:
 *
 *   (eta + dt/Wi) sigma_p - dt (kappa*_p sigma_p + sigma_p kappa*_p^T)
 *     + dt [ sum_a u_a(p) D_a(sigma) - eps Lap(sigma) ]_p  =  R_p,
 *   R_p = eta sigma0_p - H_p + dt G (kappa*_p + kappa*_p^T) g_alpha(t_{n+1}),
 *
 * with the same stencils as the explicit form (D_a upwinded on the sign of
 * u_a at p), acting on each stress component.  The global matrix (nc N)^2 is
 * assembled column by column by applying the operator to unit fields and solved
 * by Gaussian elimination with partial pivoting: small grids only.  The modes
 * are then pushed forward exactly as in orc_step.  Returns 1 if the system was
 * singular.
 */
int orc_step_implicit(const orc_params* p, const double* mu, const double* w, long step_index,
                      const double* sig_n, const double* sig_nm1,
                      const double* modes_n, const double* modes_nm1,
                      const double* sigma0,
                      const double* kap_n, const double* kap_nm1, const double* u,
                      double* sig_np1, double* modes_np1) {
    const int d = p->dim, nc = ncomp(p);
    const long N = npoints(p);
    const long n = (long)nc * N;
    const int classic = (p->alpha == 1.0);
    const int m = classic ? 0 : p->m;
    step_scalars s = scalars(p, mu, w, step_index);

    double* G = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* rhs = (double*)malloc(sizeof(double) * (size_t)n);
    double* unit = (double*)calloc((size_t)N, sizeof(double));
    if (!G || !rhs || !unit) { free(G); free(rhs); free(unit); return 1; }

    assemble_global(p, kap_n, kap_nm1, u, s.a, G, unit);

    for (long pt = 0; pt < N; ++pt) {
        double K[3][3] = {{0}};
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                long q = (long)(i * d + j) * N + pt;
                K[i][j] = 2.0 * kap_n[q] - kap_nm1[q];
            }
        double KS[3][3], sym[9];
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) KS[i][j] = K[i][j] + K[j][i];
        from_matrix(p, KS, sym);
        for (int c = 0; c < nc; ++c) {
            double H;
            if (classic) {
                H = B1 * sig_n[(long)c * N + pt] + B2 * sig_nm1[(long)c * N + pt] + B0 * sigma0[(long)c * N + pt];
            } else {
                H = 0.0;
                for (int j = 0; j < m; ++j) {
                    double cj = 1.0 / (B0 + mu[j] * p->dt);
                    double etaj = mu[j] * p->dt * cj;
                    long q = ((long)j * nc + c) * N + pt;
                    H += etaj * (B1 * modes_n[q] + B2 * modes_nm1[q]);
                }
            }
            rhs[(long)c * N + pt] = s.eta * sigma0[(long)c * N + pt] - H + p->dt * s.G * sym[c] * s.g;
        }
    }
    int failed = gauss_solve((int)n, G, rhs);
    for (long q = 0; q < n; ++q) sig_np1[q] = rhs[q];

    for (long pt = 0; pt < N; ++pt)
        for (int j = 0; j < m; ++j) {
            double cj = 1.0 / (B0 + mu[j] * p->dt);
            double rhoj = w[j] * p->dt * cj;
            for (int c = 0; c < nc; ++c) {
                long q = ((long)j * nc + c) * N + pt;
                modes_np1[q] = cj * (-B1 * modes_n[q] - B2 * modes_nm1[q]) + rhoj * (rhs[(long)c * N + pt] - sigma0[(long)c * N + pt]);
            }
        }
    free(G);
    free(rhs);
    free(unit);
    return failed;
}

/*
 * First step t_0 -> t_1 by a two-stage SDIRK2 method (gamma = 1 - 1/sqrt2, L-stable,
 * stiffly accurate), as the paper does for non-trivial initial data (Section 5.1)
 * instead of BDF2 with an empty past.  Fractional order (alpha < 1) only.
 *
 * The kernel-compressed law is the system of mode equations
 *     d sigma_j/dt = -mu_j sigma_j + w_j (sigma - sigma0)
 * (the ODEs whose BDF2 discretisation is eq. BDF_Phi_k_n+1) with the constraint
 *     sum_j d sigma_j/dt = F(sigma, t) = L(kappa) sigma - sigma/Wi + G (kappa + kappa^T) g_alpha(t)
 *                                        - (u.grad - eps Lap) sigma,
 * the mode sum standing for the Caputo derivative.  At stage i (time t_i, stage
 * value S, Z_j the explicit part of the mode stage) the slopes are
 *     K_j = (-mu_j Z_j + w_j (S - sigma0)) / (1 + gamma mu_j dt),
 * and the constraint gives, over the grid (transport implicit),
 *     (dt W + dt/Wi) S - dt L(kappa) S + dt (u.grad - eps Lap) S
 *         = dt W sigma0 + dt sum_j mu_j Z_j / (1 + gamma mu_j dt) + dt G (kappa + kappa^T) g_alpha(t_i),
 *     W = sum_j w_j / (1 + gamma mu_j dt).
 * Stage 1: t_1 = gamma dt, Z_j = sigma_j^0.  Stage 2: t_2 = dt,
 * Z_j = sigma_j^0 + dt (1 - gamma) K_j^(1).  Result: sigma^1 = S^(2),
 * sigma_j^1 = Z_j^(2) + gamma dt K_j^(2).  kappa* = kappa^0 (no past).
 * Returns 1 if a system was singular.
 */
int orc_first_step_sdirk2(const orc_params* p, const double* mu, const double* w,
                          const double* sig_0, const double* modes_0, const double* sigma0,
                          const double* kap_0, const double* u, double* sig_1, double* modes_1) {
    const int d = p->dim, nc = ncomp(p);
    const long N = npoints(p);
    const long n = (long)nc * N;
    const int m = p->m;
    if (p->alpha == 1.0 || m < 1) return 1;
    const double gam = 1.0 - sqrt(0.5);
    const double dt = p->dt;
    double W = 0.0;
    for (int j = 0; j < m; ++j) W += w[j] / (1.0 + gam * mu[j] * dt);
    const double a = dt * W + dt / p->Wi;
    const double G = (1.0 - p->beta) / (p->Wi * p->Re);
    (void)sig_0;

    double* A = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* rhs = (double*)malloc(sizeof(double) * (size_t)n);
    double* unit = (double*)calloc((size_t)N, sizeof(double));
    double* Z = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    if (!A || !rhs || !unit || !Z) { free(A); free(rhs); free(unit); free(Z); return 1; }
    memcpy(Z, modes_0, sizeof(double) * (size_t)m * (size_t)n);
    int failed = 0;
    for (int stage = 1; stage <= 2; ++stage) {
        const double t = (stage == 1 ? gam : 1.0) * dt;
        const double g = pow(t, p->alpha - 1.0) / tgamma(p->alpha);
        assemble_global(p, kap_0, kap_0, u, a, A, unit);
        for (long pt = 0; pt < N; ++pt) {
            double K[3][3] = {{0}}, KS[3][3], sym[9];
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) K[i][j] = kap_0[(long)(i * d + j) * N + pt];
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) KS[i][j] = K[i][j] + K[j][i];
            from_matrix(p, KS, sym);
            for (int c = 0; c < nc; ++c) {
                double zsum = 0.0;
                for (int j = 0; j < m; ++j) zsum += mu[j] * Z[((long)j * nc + c) * N + pt] / (1.0 + gam * mu[j] * dt);
                rhs[(long)c * N + pt] = dt * W * sigma0[(long)c * N + pt] + dt * zsum + dt * G * sym[c] * g;
            }
        }
        if (gauss_solve((int)n, A, rhs)) failed = 1;
        /* slopes and the next mode stage */
        for (int j = 0; j < m; ++j)
            for (long q = 0; q < n; ++q) {
                const long jq = (long)j * n + q;
                const double Kj = (-mu[j] * Z[jq] + w[j] * (rhs[q] - sigma0[q])) / (1.0 + gam * mu[j] * dt);
                if (stage == 1) Z[jq] = modes_0[jq] + dt * (1.0 - gam) * Kj;
                else modes_1[jq] = Z[jq] + gam * dt * Kj;
            }
    }
    for (long q = 0; q < n; ++q) sig_1[q] = rhs[q];
    free(A);
    free(rhs);
    free(unit);
    free(Z);
    return failed;
}

/*
 * Reference adjoint (reverse-mode derivative) of orc_step, for packed storage.
 *
 * The step maps (sigma^n, sigma^{n-1}, modes^n, modes^{n-1}) to
 * (sigma^{n+1}, sigma^n, modes^{n+1}, modes^n).  Given the adjoints of the
 * outputs -- s1 (of sigma^{n+1}), s0 (of the copied sigma^n), z1 (of
 * modes^{n+1}) and z0 (of the copied modes^n) -- it writes the adjoints of the
 * inputs (s1_out of sigma^n, s0_out of sigma^{n-1}, z1_out of modes^n, z0_out of
 * modes^{n-1}) and adds the parameter derivatives to g_sigma0 [nc][N],
 * g_kap_n and g_kap_nm1 [d*d][N], *g_Wi and *g_beta.
 * sig_np1 is the forward result of this step.  The operations of orc_step are
 * differentiated in reverse order.
 */
int orc_adjoint_step(const orc_params* p, const double* mu, const double* w, long step_index,
                     const double* sig_np1, const double* sigma0,
                     const double* kap_n, const double* kap_nm1, const double* u,
                     const double* s1, const double* s0, const double* z1, const double* z0,
                     double* s1_out, double* s0_out, double* z1_out, double* z0_out,
                     double* g_sigma0, double* g_kap_n, double* g_kap_nm1,
                     double* g_Wi, double* g_beta) {
    const int d = p->dim, nc = ncomp(p);
    const long N = npoints(p);
    const int classic = (p->alpha == 1.0);
    const int m = classic ? 0 : p->m;
    step_scalars s = scalars(p, mu, w, step_index);
    int failures = 0;
    double gWi = 0.0, gbeta = 0.0;
    (void)sigma0;   /* sigma0 enters linearly; its derivative does not depend on it */

    double* lamA = (double*)calloc((size_t)nc * (size_t)N, sizeof(double));

#pragma omp parallel for schedule(static) reduction(+ : failures, gWi, gbeta)
    for (long pt = 0; pt < N; ++pt) {
        double K[3][3] = {{0}};
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                long q = (long)(i * d + j) * N + pt;
                K[i][j] = 2.0 * kap_n[q] - kap_nm1[q];
            }
        double sig[9];
        for (int c = 0; c < nc; ++c) sig[c] = sig_np1[(long)c * N + pt];

        /* modes^{n+1} = c_j(-b1 modes^n - b2 modes^{n-1}) + rho_j (sigma^{n+1} - sigma0) */
        double lam_sig[9];
        for (int c = 0; c < nc; ++c) lam_sig[c] = s1[(long)c * N + pt];
        for (int j = 0; j < m; ++j) {
            double cj = 1.0 / (B0 + mu[j] * p->dt);
            double rhoj = w[j] * p->dt * cj;
            for (int c = 0; c < nc; ++c) {
                long q = ((long)j * nc + c) * N + pt;
                lam_sig[c] += rhoj * z1[q];
                g_sigma0[(long)c * N + pt] -= rhoj * z1[q];
            }
        }

        /* sigma^{n+1} = M^{-1} R  ->  lamR = M^{-T} lam_sig */
        double M[81], Mt[81], lamR[9];
        assemble(p, K, s.a, M);
        for (int r = 0; r < nc; ++r)
            for (int c = 0; c < nc; ++c) Mt[r * nc + c] = M[c * nc + r];
        for (int c = 0; c < nc; ++c) lamR[c] = lam_sig[c];
        if (gauss_solve(nc, Mt, lamR)) failures += 1;

        /* dM sigma = da sigma - dt (dK sigma + sigma dK^T):
           lam_a = -<lamR, sigma>, lam_K_ab = dt <lamR, (E_ab sigma + sigma E_ab^T)> */
        double lam_a = 0.0;
        for (int c = 0; c < nc; ++c) lam_a -= lamR[c] * sig[c];
        double lamK[3][3] = {{0}};
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double E[3][3] = {{0}};
                E[a][b] = 1.0;
                double img[9];
                upper_convected(p, E, sig, img);
                double acc = 0.0;
                for (int c = 0; c < nc; ++c) acc += lamR[c] * img[c];
                lamK[a][b] += p->dt * acc;
            }

        /* R = eta sigma0 - H + dt G sym(K) g - A */
        double sym[9];
        {
            double KS[3][3];
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) KS[i][j] = K[i][j] + K[j][i];
            from_matrix(p, KS, sym);
        }
        double lam_G = 0.0;
        for (int c = 0; c < nc; ++c) lam_G += p->dt * s.g * sym[c] * lamR[c];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                /* d sym_c / d K_ab = [pair(c) == (a,b)] + [pair(c) == (b,a)] */
                double acc = 0.0;
                for (int c = 0; c < nc; ++c) {
                    int i, j;
                    comp_pair(p, c, &i, &j);
                    double dsym = ((i == a && j == b) ? 1.0 : 0.0) + ((j == a && i == b) ? 1.0 : 0.0);
                    acc += lamR[c] * dsym;
                }
                lamK[a][b] += p->dt * s.G * s.g * acc;
            }
        for (int c = 0; c < nc; ++c) {
            g_sigma0[(long)c * N + pt] += s.eta * lamR[c];
            lamA[(long)c * N + pt] = -lamR[c];
        }

        /* H and the mode recursion: lamQ_j = -c_j z1_j - eta_j lamR  (classic: H uses sigma levels) */
        for (int c = 0; c < nc; ++c) {
            s1_out[(long)c * N + pt] = s0[(long)c * N + pt];   /* copy slot */
            s0_out[(long)c * N + pt] = 0.0;
        }
        if (classic) {
            for (int c = 0; c < nc; ++c) {
                double lamH = -lamR[c];
                s1_out[(long)c * N + pt] += B1 * lamH;
                s0_out[(long)c * N + pt] += B2 * lamH;
                g_sigma0[(long)c * N + pt] += B0 * lamH;
            }
        }
        for (int j = 0; j < m; ++j) {
            double cj = 1.0 / (B0 + mu[j] * p->dt);
            double etaj = mu[j] * p->dt * cj;
            for (int c = 0; c < nc; ++c) {
                long q = ((long)j * nc + c) * N + pt;
                double lamQ = -cj * z1[q] - etaj * lamR[c];
                z1_out[q] = z0[q] + B1 * lamQ;
                z0_out[q] = B2 * lamQ;
            }
        }

        /* kappa* = 2 kappa^n - kappa^{n-1} */
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                long q = (long)(a * d + b) * N + pt;
                g_kap_n[q] += 2.0 * lamK[a][b];
                g_kap_nm1[q] -= lamK[a][b];
            }

        /* a = eta + dt/Wi, G = (1-beta)/(Wi Re) */
        gWi += -p->dt / (p->Wi * p->Wi) * lam_a - s.G / p->Wi * lam_G;
        gbeta += -lam_G / (p->Wi * p->Re);
    }

    /* A = dt sum_a u_a D_a(E) - eps dt Lap(E), E = 2 sigma^n - sigma^{n-1}:
       scatter lamA through the stencil to the points it read */
    if (p->transport) {
        double* lamE = (double*)calloc((size_t)nc * (size_t)N, sizeof(double));
        for (long pt = 0; pt < N; ++pt) {
            long c3[3];
            c3[0] = pt % p->n[0];
            c3[1] = (pt / p->n[0]) % p->n[1];
            c3[2] = (d == 3) ? pt / ((long)p->n[0] * p->n[1]) : 0;
            for (int c = 0; c < nc; ++c) {
                double la = lamA[(long)c * N + pt];
                if (la == 0.0) continue;
                double* le = lamE + (long)c * N;
                for (int a = 0; a < d; ++a) {
                    double va = u[(long)a * N + pt];
                    double h = p->L[a] / p->n[a];
                    double coef[5] = {0, 0, 0, 0, 0};
                    if (p->stencil == 1) { coef[1] = -1.0 / (2.0 * h); coef[3] = 1.0 / (2.0 * h); }
                    else if (va >= 0.0) {
                        coef[0] = 1.0 / (6.0 * h); coef[1] = -6.0 / (6.0 * h);
                        coef[2] = 3.0 / (6.0 * h); coef[3] = 2.0 / (6.0 * h);
                    } else {
                        coef[1] = -2.0 / (6.0 * h); coef[2] = -3.0 / (6.0 * h);
                        coef[3] = 6.0 / (6.0 * h); coef[4] = -1.0 / (6.0 * h);
                    }
                    for (int k = -2; k <= 2; ++k) {
                        if (coef[k + 2] == 0.0) continue;
                        long q[3] = {c3[0], c3[1], c3[2]};
                        q[a] = wrap(c3[a] + k, p->n[a]);
                        le[pidx(p, q[0], q[1], q[2])] += p->dt * va * coef[k + 2] * la;
                    }
                    if (p->eps != 0.0) {
                        double hh = h * h;
                        long qm[3] = {c3[0], c3[1], c3[2]}, qp[3] = {c3[0], c3[1], c3[2]};
                        qm[a] = wrap(c3[a] - 1, p->n[a]);
                        qp[a] = wrap(c3[a] + 1, p->n[a]);
                        le[pidx(p, qm[0], qm[1], qm[2])] -= p->eps * p->dt * la / hh;
                        le[pt] -= p->eps * p->dt * (-2.0) * la / hh;
                        le[pidx(p, qp[0], qp[1], qp[2])] -= p->eps * p->dt * la / hh;
                    }
                }
            }
        }
        for (long q = 0; q < (long)nc * N; ++q) {
            s1_out[q] += 2.0 * lamE[q];
            s0_out[q] -= lamE[q];
        }
        free(lamE);
    }
    free(lamA);
    *g_Wi += gWi;
    *g_beta += gbeta;
    return failures;
}
