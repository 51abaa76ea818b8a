/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, FP64 CPU implementation of the sparse-GP (GAP) fit of
 * Klawohn, Kermode and Bartok, "Massively Parallel Fitting of Gaussian
 * Approximation Potentials" (arXiv:2207.03803), Sec. II.  Only the test suite,
 * the package's smoke check and the benchmark's CPU-baseline leg may load this
 * file; the GPU library shares no code with it.
 *
 * Every loop sums in index order; OpenMP splits only independent outputs
 * (configurations, rows, columns), so results are bit-identical for any
 * thread count.  Build with -ffp-contract=off: no FMA contraction.
 *
 * Notation (paper, Sec. II): x_i descriptor of atom i (unit length here),
 * x_s sparse point, k(x, x_s) = delta^2 (x . x_s)^zeta the dot-product
 * covariance named by the appendix options (covariance_type=dot_product,
 * zeta, delta), integer zeta evaluated by repeated multiplication.  With
 * species labels, k = 0 between different species.
 *
 * Derivative rows (Sec. II: force observations enter through the kernel's gradients):
 * pair p = (target atom a, source atom i) carries J_p = d x_i / d r_a, layout
 * [pair][alpha][d].  The force on a is F_a = -dE/dr_a, so the design row of
 * force component (a, alpha) is
 *     K_{(a,alpha),s} = -delta^2 zeta sum_{p in pairs(a)} (x_i . x_s)^(zeta-1) (J_p[alpha] . x_s).
 *
 * Virial rows (Sec. II: derivatives with respect to lattice deformations):
 * pair p also carries u_p = r_a - r_i, the displacement of its target from its
 * source.  A homogeneous strain eps moves x_i by sum_p J_p eps u_p (first order), so
 * the virial W = -dE/d eps of configuration A, symmetrised, in Voigt order
 * (xx, yy, zz, yz, xz, xy) with (alpha, beta) the component's two indices, is
 *     K_{(A,v),s} = -delta^2 zeta sum_{p in pairs(A)} (x_i . x_s)^(zeta-1)
 *                   (1/2) [(J_p[alpha] . x_s) u_p[beta] + (J_p[beta] . x_s) u_p[alpha]].
 *
 * Parity status: every function below is pinned by the CPU test suite
 * (normal equations, exact rational solves, loss gradient, LAPACK Householder
 * convention, finite differences, closed forms for zeta = 1 and 2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

static double wall(void) {
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

static double dot(const double *a, const double *b, int64_t d) {
    double g = 0.0;
    for (int64_t k = 0; k < d; ++k) g += a[k] * b[k];
    return g;
}

static double ipow(double g, int zeta) {
    double p = 1.0;
    for (int z = 0; z < zeta; ++z) p *= g;
    return p;
}

static int same_species(const int32_t *sa, int64_t i, const int32_t *ss, int64_t s) {
    if (!sa || !ss) return 1;
    return sa[i] == ss[s];
}

/* Covariance k(x_i, x_s) = delta^2 (x_i . x_s)^zeta (appendix options). */
double or_kernel(const double *x, const double *xs, int64_t d, double delta, int zeta) {
    return delta * delta * ipow(dot(x, xs, d), zeta);
}

/* Energy rows of the design matrix, Eq. (6) summed over the atoms of each
 * configuration (Eq. 1) and scaled by Sigma^{-1/2} (Eq. 7):
 *     out[A, s] = (1/sigma_A) sum_{i in A} k(x_i, x_s).   out: [n_cfg x M]. */
void or_design_energy(int64_t n_cfg, const int64_t *cfg_ptr, int64_t d, const double *X,
                      const int32_t *atom_sp, int64_t M, const double *Xs, const int32_t *sparse_sp,
                      double delta, int zeta, const double *sigma_e, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t A = 0; A < n_cfg; ++A) {
        for (int64_t s = 0; s < M; ++s) {
            double e = 0.0;
            for (int64_t i = cfg_ptr[A]; i < cfg_ptr[A + 1]; ++i)
                if (same_species(atom_sp, i, sparse_sp, s)) e += or_kernel(X + i * d, Xs + s * d, d, delta, zeta);
            out[A * M + s] = e / sigma_e[A];
        }
    }
}

/* Force rows (derivative observations, Sec. II), scaled by Sigma^{-1/2}:
 *     out[3a+alpha, s] = -(delta^2 zeta / sigma) sum_p (x_i . x_s)^(zeta-1) (J_p[alpha] . x_s).
 * out: [3 n_atoms x M]. */
void or_design_force(int64_t n_atoms, const int64_t *pair_ptr, const int64_t *pair_src, const double *J,
                     int64_t d, const double *X, const int32_t *atom_sp, int64_t M, const double *Xs,
                     const int32_t *sparse_sp, double delta, int zeta, const double *sigma_f, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < n_atoms; ++a) {
        for (int64_t s = 0; s < M; ++s) {
            double f[3] = {0.0, 0.0, 0.0};
            for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p) {
                int64_t i = pair_src[p];
                if (!same_species(atom_sp, i, sparse_sp, s)) continue;
                double w = delta * delta * (double)zeta * ipow(dot(X + i * d, Xs + s * d, d), zeta - 1);
                for (int al = 0; al < 3; ++al) f[al] += w * dot(J + (p * 3 + al) * d, Xs + s * d, d);
            }
            for (int al = 0; al < 3; ++al) out[(3 * a + al) * M + s] = -f[al] / sigma_f[3 * a + al];
        }
    }
}

/* The Voigt components (xx, yy, zz, yz, xz, xy) of the symmetrised product of a
 * 3-vector g (alpha-indexed) and u (beta-indexed). */
static void voigt_sym(const double *g, const double *u, double *v) {
    v[0] = g[0] * u[0];
    v[1] = g[1] * u[1];
    v[2] = g[2] * u[2];
    v[3] = 0.5 * (g[1] * u[2] + g[2] * u[1]);
    v[4] = 0.5 * (g[0] * u[2] + g[2] * u[0]);
    v[5] = 0.5 * (g[0] * u[1] + g[1] * u[0]);
}

/* Virial rows (lattice-deformation derivatives, Sec. II), scaled by Sigma^{-1/2}:
 *     out[6A+v, s] = -(delta^2 zeta / sigma) sum over pairs p whose target atom is in A of
 *                    (x_i . x_s)^(zeta-1) sym(J_p x_s, u_p)_v.
 * out: [6 n_cfg x M]. */
void or_design_virial(int64_t n_cfg, const int64_t *cfg_ptr, const int64_t *pair_ptr, const int64_t *pair_src,
                      const double *J, const double *pair_u, int64_t d, const double *X, const int32_t *atom_sp,
                      int64_t M, const double *Xs, const int32_t *sparse_sp, double delta, int zeta,
                      const double *sigma_v, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t A = 0; A < n_cfg; ++A) {
        for (int64_t s = 0; s < M; ++s) {
            double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int64_t a = cfg_ptr[A]; a < cfg_ptr[A + 1]; ++a) {
                for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p) {
                    int64_t i = pair_src[p];
                    if (!same_species(atom_sp, i, sparse_sp, s)) continue;
                    double w = delta * delta * (double)zeta * ipow(dot(X + i * d, Xs + s * d, d), zeta - 1);
                    double g[3], t[6];
                    for (int al = 0; al < 3; ++al) g[al] = dot(J + (p * 3 + al) * d, Xs + s * d, d);
                    voigt_sym(g, pair_u + 3 * p, t);
                    for (int k = 0; k < 6; ++k) v[k] += w * t[k];
                }
            }
            for (int k = 0; k < 6; ++k) out[(6 * A + k) * M + s] = -v[k] / sigma_v[6 * A + k];
        }
    }
}

/* K_MM[s,t] = k(x_s, x_t), plus the absolute sparse_jitter on the diagonal
 * (appendix options: sparse_jitter=1.0E-8).  The upper triangle is computed
 * and mirrored, so the matrix is exactly symmetric. */
void or_kmm(int64_t M, int64_t d, const double *Xs, const int32_t *sparse_sp, double delta, int zeta,
            double jitter, double *K) {
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t s = 0; s < M; ++s) {
        for (int64_t t = s; t < M; ++t) {
            double v = same_species(sparse_sp, s, sparse_sp, t) ? or_kernel(Xs + s * d, Xs + t * d, d, delta, zeta) : 0.0;
            if (t == s) v += jitter;
            K[s * M + t] = v;
            K[t * M + s] = v;
        }
    }
}

/* Cholesky K = U^T U with U upper triangular (U = L_MM^T of Eq. 7).
 * Returns 0, or j+1 when pivot j is not positive.  U: [M x M], lower part zeroed. */
int or_cholesky_upper(int64_t M, const double *K, double *U) {
    memset(U, 0, sizeof(double) * (size_t)(M * M));
    for (int64_t j = 0; j < M; ++j) {
        double s = K[j * M + j];
        for (int64_t k = 0; k < j; ++k) s -= U[k * M + j] * U[k * M + j];
        if (!(s > 0.0)) return (int)(j + 1);
        double ujj = sqrt(s);
        U[j * M + j] = ujj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < M; ++i) {
            double t = K[j * M + i];
            for (int64_t k = 0; k < j; ++k) t -= U[k * M + j] * U[k * M + i];
            U[j * M + i] = t / ujj;
        }
    }
    return 0;
}

/* Householder QR A = QR (Eq. 11 and the text after it), in place on a
 * row-major [m x n] matrix, LAPACK geqrf convention: column j's reflector is
 * H_j = I - tau_j v v^T with v_j = 1 implicit, v_{j+1..m-1} stored below the
 * diagonal, R on and above the diagonal.  For x = A[j:m, j] with alpha = x_0:
 * beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta, v = x/(alpha - beta);
 * a zero sub-column gives tau = 0.  Columns are updated in blocks of 64, one
 * thread per block, each block sweeping the rows in order. */
void or_householder_qr(int64_t m, int64_t n, double *A, double *tau) {
    int64_t kmax = m < n ? m : n;
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < kmax; ++j) {
        double xnorm2 = 0.0;
        for (int64_t i = j + 1; i < m; ++i) xnorm2 += A[i * n + j] * A[i * n + j];
        double alpha = A[j * n + j];
        if (xnorm2 == 0.0) { tau[j] = 0.0; continue; }
        double beta = -copysign(sqrt(alpha * alpha + xnorm2), alpha);
        tau[j] = (beta - alpha) / beta;
        double scal = 1.0 / (alpha - beta);
        for (int64_t i = j + 1; i < m; ++i) A[i * n + j] *= scal;
        A[j * n + j] = beta;
        double tj = tau[j];
        int64_t nb = (n - (j + 1) + 63) / 64;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t b = 0; b < nb; ++b) {
            int64_t k0 = j + 1 + 64 * b, k1 = k0 + 64 < n ? k0 + 64 : n;
            for (int64_t k = k0; k < k1; ++k) w[k] = A[j * n + k];          /* v_j = 1 */
            for (int64_t i = j + 1; i < m; ++i) {
                double vi = A[i * n + j];
                for (int64_t k = k0; k < k1; ++k) w[k] += vi * A[i * n + k];
            }
            for (int64_t k = k0; k < k1; ++k) A[j * n + k] -= tj * w[k];
            for (int64_t i = j + 1; i < m; ++i) {
                double vi = A[i * n + j];
                for (int64_t k = k0; k < k1; ++k) A[i * n + k] -= tj * w[k] * vi;
            }
        }
    }
    free(w);
}

/* Q^T b with the reflectors stored by or_householder_qr (the pdormqr step of
 * Sec. III.B): b <- H_{k-1} ... H_1 H_0 ... applied as H_0 first. */
void or_apply_qt(int64_t m, int64_t n, const double *A, const double *tau, double *b) {
    int64_t kmax = m < n ? m : n;
    for (int64_t j = 0; j < kmax; ++j) {
        double w = b[j];
        for (int64_t i = j + 1; i < m; ++i) w += A[i * n + j] * b[i];
        double tw = tau[j] * w;
        b[j] -= tw;
        for (int64_t i = j + 1; i < m; ++i) b[i] -= tw * A[i * n + j];
    }
}

/* Q x for x of length m (the reflectors applied in reverse order). */
void or_apply_q(int64_t m, int64_t n, const double *A, const double *tau, double *x) {
    int64_t kmax = m < n ? m : n;
    for (int64_t j = kmax - 1; j >= 0; --j) {
        double w = x[j];
        for (int64_t i = j + 1; i < m; ++i) w += A[i * n + j] * x[i];
        double tw = tau[j] * w;
        x[j] -= tw;
        for (int64_t i = j + 1; i < m; ++i) x[i] -= tw * A[i * n + j];
    }
}

/* Back substitution c = R^{-1} z (Eq. 12, the pdtrtrs step), R the upper
 * triangle of the row-major [* x ldr] array.  Returns j+1 if R_jj == 0. */
int or_back_substitution(int64_t n, const double *R, int64_t ldr, const double *z, double *c) {
    for (int64_t j = n - 1; j >= 0; --j) {
        double t = z[j];
        for (int64_t k = j + 1; k < n; ++k) t -= R[j * ldr + k] * c[k];
        if (R[j * ldr + j] == 0.0) return (int)(j + 1);
        c[j] = t / R[j * ldr + j];
    }
    return 0;
}

/* Predictions of the fitted model (Eqs. 1 and 2): E_A = sum_{i in A} eps(x_i),
 * eps(x) = sum_s c_s k(x, x_s).  Forces, when pair data are given, follow the
 * chain rule: F_{a,alpha} = -sum_{p in pairs(a)} J_p[alpha] . grad eps(x_i),
 * grad eps(x) = sum_s c_s delta^2 zeta (x . x_s)^(zeta-1) x_s; virials, when the
 * pair displacements are given too: V_{A,v} = -sum over the pairs of A's atoms of
 * sym(J_p grad eps(x_i), u_p)_v.
 * E: [n_cfg], F: [3 n_atoms] (may be NULL), V: [6 n_cfg] (may be NULL). */
void or_predict(int64_t n_cfg, const int64_t *cfg_ptr, int64_t d, const double *X, const int32_t *atom_sp,
                int64_t M, const double *Xs, const int32_t *sparse_sp, double delta, int zeta, const double *c,
                const int64_t *pair_ptr, const int64_t *pair_src, const double *J, const double *pair_u, double *E,
                double *F, double *V) {
    int64_t n_atoms = cfg_ptr[n_cfg];
    double *eps = (double *)malloc(sizeof(double) * (size_t)(n_atoms > 0 ? n_atoms : 1));
    double *grad = NULL;
    int want_v = (V && pair_ptr && pair_src && J && pair_u);
    int want_f = (F && pair_ptr && pair_src && J) || want_v;
    if (want_f) grad = (double *)malloc(sizeof(double) * (size_t)(n_atoms > 0 ? n_atoms * d : 1));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_atoms; ++i) {
        double e = 0.0;
        double *gi = want_f ? grad + i * d : NULL;
        if (gi) memset(gi, 0, sizeof(double) * (size_t)d);
        for (int64_t s = 0; s < M; ++s) {
            if (!same_species(atom_sp, i, sparse_sp, s)) continue;
            double g = dot(X + i * d, Xs + s * d, d);
            e += c[s] * delta * delta * ipow(g, zeta);
            if (gi) {
                double w = c[s] * delta * delta * (double)zeta * ipow(g, zeta - 1);
                for (int64_t k = 0; k < d; ++k) gi[k] += w * Xs[s * d + k];
            }
        }
        eps[i] = e;
    }
    for (int64_t A = 0; A < n_cfg; ++A) {
        double e = 0.0;
        for (int64_t i = cfg_ptr[A]; i < cfg_ptr[A + 1]; ++i) e += eps[i];
        E[A] = e;
    }
    if (want_f && F) {
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < n_atoms; ++a) {
            for (int al = 0; al < 3; ++al) {
                double f = 0.0;
                for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p)
                    f += dot(J + (p * 3 + al) * d, grad + pair_src[p] * d, d);
                F[3 * a + al] = -f;
            }
        }
    }
    if (want_v) {
#pragma omp parallel for schedule(static)
        for (int64_t A = 0; A < n_cfg; ++A) {
            double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int64_t a = cfg_ptr[A]; a < cfg_ptr[A + 1]; ++a) {
                for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p) {
                    double g[3], t[6];
                    for (int al = 0; al < 3; ++al) g[al] = dot(J + (p * 3 + al) * d, grad + pair_src[p] * d, d);
                    voigt_sym(g, pair_u + 3 * p, t);
                    for (int k = 0; k < 6; ++k) v[k] += t[k];
                }
            }
            for (int k = 0; k < 6; ++k) V[6 * A + k] = -v[k];
        }
    }
    free(grad);
    free(eps);
}

/* The whole fit of Sec. II: A = [Sigma^{-1/2} K_NM ; U] (Eq. 7), b = [y/sigma ; 0]
 * (Eq. 8), Householder QR of A, Q^T b, back substitution (Eq. 12).
 * y: energies [n_cfg], then forces [3 n_atoms] (if pair data are given), then
 * virials [6 n_cfg] (if pair displacements are given too).
 * times[4] (optional): seconds for assembly, K_MM + Cholesky, QR, Q^T b + solve.
 * A_out (optional, [(N+M) x M]) receives the factored matrix (R and reflectors).
 * Returns 0, or -(pivot) for a Cholesky breakdown, or +j for a zero R_jj. */
int or_fit(int64_t n_cfg, const int64_t *cfg_ptr, int64_t d, const double *X, const int32_t *atom_sp,
           int64_t M, const double *Xs, const int32_t *sparse_sp, double delta, int zeta, double jitter,
           const int64_t *pair_ptr, const int64_t *pair_src, const double *J, const double *pair_u,
           const double *y, const double *sigma, double *c, double *times, double *A_out) {
    int64_t n_atoms = cfg_ptr[n_cfg];
    int64_t NF = n_cfg + (pair_ptr ? 3 * n_atoms : 0);
    int64_t N = NF + (pair_ptr && pair_u ? 6 * n_cfg : 0);
    int64_t rows = N + M;
    double *A = A_out ? A_out : (double *)malloc(sizeof(double) * (size_t)(rows * M));
    double *b = (double *)calloc((size_t)rows, sizeof(double));
    double *tau = (double *)malloc(sizeof(double) * (size_t)M);
    double *K = (double *)malloc(sizeof(double) * (size_t)(M * M));
    double t0 = wall();
    or_design_energy(n_cfg, cfg_ptr, d, X, atom_sp, M, Xs, sparse_sp, delta, zeta, sigma, A);
    if (pair_ptr)
        or_design_force(n_atoms, pair_ptr, pair_src, J, d, X, atom_sp, M, Xs, sparse_sp, delta, zeta,
                        sigma + n_cfg, A + n_cfg * M);
    if (pair_ptr && pair_u)
        or_design_virial(n_cfg, cfg_ptr, pair_ptr, pair_src, J, pair_u, d, X, atom_sp, M, Xs, sparse_sp, delta,
                         zeta, sigma + NF, A + NF * M);
    for (int64_t r = 0; r < N; ++r) b[r] = y[r] / sigma[r];
    double t1 = wall();
    or_kmm(M, d, Xs, sparse_sp, delta, zeta, jitter, K);
    int st = or_cholesky_upper(M, K, A + N * M);
    double t2 = wall();
    int rc = 0;
    if (st != 0) { rc = -st; goto done; }
    or_householder_qr(rows, M, A, tau);
    double t3 = wall();
    or_apply_qt(rows, M, A, tau, b);
    st = or_back_substitution(M, A, M, b, c);
    double t4 = wall();
    if (st != 0) rc = st;
    if (times) { times[0] = t1 - t0; times[1] = t2 - t1; times[2] = t3 - t2; times[3] = t4 - t3; }
done:
    free(K);
    free(tau);
    free(b);
    if (!A_out) free(A);
    return rc;
}
