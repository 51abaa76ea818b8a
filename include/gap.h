/*
 * libgap -- sparse Gaussian-process (GAP) fitting on one GB300 GPU (sm_103a).
 *
 * The library computes the fit of Klawohn, Kermode and Bartok, "Massively
 * Parallel Fitting of Gaussian Approximation Potentials" (arXiv:2207.03803),
 * Sec. II: the weights c minimising the loss of Eq. (3),
 *     L = (y - K_NM c)^T Sigma^{-1} (y - K_NM c) + c^T K_MM c,
 * through the stable least-squares form of Eqs. (7)-(12):
 *     A = [ Sigma^{-1/2} K_NM ; U ],  K_MM = U^T U (U = L_MM^T),  b = [ Sigma^{-1/2} y ; 0 ],
 *     A = QR,  c = R^{-1} Q^T b.
 * K_NM holds one row per target: total energies, Eq. (6), summed over the
 * atoms of a configuration, and force components (derivative observations,
 * Sec. II).  The covariance is the dot-product kernel of the appendix
 * options, k(x, x_s) = delta^2 (x . x_s)^zeta with integer zeta in 1..63.
 *
 * Conventions for every entry point:
 *   - Every call returns a gap_status; nothing aborts or throws across the ABI.
 *     gap_last_error() gives a one-line reason for the last failure on a ctx.
 *   - Work is ordered on the CUDA stream given to gap_create (NULL = legacy
 *     default stream).  Calls return after their work is enqueued, except
 *     where a host-visible result is needed (documented per call).
 *   - Input pointers are borrowed for the duration of the call only; what is
 *     needed later is copied or derived into workspaces the ctx owns.
 *     Outputs go to caller-allocated buffers.
 *   - Matrices in the problem description are row-major, FP64.
 *   - A ctx is not thread-safe; use one per host thread.
 */
#ifndef LIBGAP_GAP_H
#define LIBGAP_GAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gap_ctx gap_ctx;

typedef enum {
    GAP_OK = 0,
    GAP_ERR_INVALID = 1,        /* bad argument or inconsistent problem description   */
    GAP_ERR_NOMEM = 2,          /* device or host allocation failed                   */
    GAP_ERR_CUDA = 3,           /* a CUDA runtime call failed                         */
    GAP_ERR_NOT_SPD = 4,        /* Cholesky of K_MM met a non-positive pivot          */
    GAP_ERR_RANK = 5,           /* zero or non-finite diagonal entry of R             */
    GAP_ERR_NOT_CONVERGED = 6,  /* refinement stopped at its iteration limit          */
    GAP_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up                 */
    GAP_ERR_STATE = 8           /* calls out of order (assemble -> factor -> solve)   */
} gap_status;

typedef enum {
    /* A, K_MM, Cholesky, QR, Q^T b and back substitution all in FP64 SIMT kernels.
     * Reproducibility: the rows of a configuration or of a target atom cut by tile
     * edges are summed by atomic adds, one per tile.  With at most two parts (every
     * configuration of <= 128 atoms, every atom of <= 64 pairs) the sum does not
     * depend on their order and a fit is bit-for-bit the same on every run; longer
     * segments add three or more parts in arrival order, so their rows (and the fit)
     * agree between runs to FP64 rounding only. */
    GAP_PREC_FP64 = 0,
    /* Design-matrix dot products on tcgen05 tensor cores with FP32 accumulation: a
     * single-pass BF16 (or TF32) copy with an FP32 zeta-power epilogue feeds an FP32
     * Householder QR; a split-operand copy accurate to FP32, with its energy rows kept
     * in FP64 from a double-float epilogue, feeds the FP64 iterative refinement of c.
     * Its products: TF32, two slices and three products; BF16, three slices and six
     * products.
     * The K_MM Cholesky runs in double-float on the FP32 units; the refinement's
     * residuals and corrections and the final solves are FP64 (or double-float). */
    GAP_PREC_MIXED_BF16 = 1,
    GAP_PREC_MIXED_TF32 = 2,
    /* As GAP_PREC_MIXED_BF16, but the force rows -- nearly all of the design matrix --
     * come from FP16 products: each operand row is scaled by a power of two and split
     * into two FP16 slices, the single-pass FP16 product feeding the QR and three
     * products (error about 2^-22, as for TF32) the refinement.  Half the tensor-core
     * work of the BF16 force rows; energy rows and predictions as GAP_PREC_MIXED_BF16. */
    GAP_PREC_MIXED_FP16 = 3
} gap_precision;

typedef enum { GAP_MEM_DEVICE = 0, GAP_MEM_HOST = 1 } gap_memory;

/* One fitting problem.  n_pairs == 0 and pair_ptr == NULL mean energies only. */
typedef struct {
    int64_t n_cfg;            /* configurations (energy targets)                          */
    int64_t n_atoms;          /* atoms over all configurations (== cfg_ptr[n_cfg])        */
    int64_t d;                /* descriptor length                                        */
    int64_t n_pairs;          /* (target atom, source atom) pairs for force rows          */
    int64_t n_sparse;         /* sparse points M                                          */
    const int64_t *cfg_ptr;   /* [n_cfg+1] atoms of configuration A: [cfg_ptr[A], cfg_ptr[A+1]) */
    const double *X;          /* [n_atoms, d] unit-length descriptors x_i                 */
    const double *Xs;         /* [n_sparse, d] unit-length sparse points x_s              */
    const int32_t *atom_species;   /* [n_atoms] or NULL (one species); k = 0 across species */
    const int32_t *sparse_species; /* [n_sparse] or NULL                                  */
    const int64_t *pair_ptr;  /* [n_atoms+1] pairs of target atom a: [pair_ptr[a], pair_ptr[a+1]) */
    const int64_t *pair_src;  /* [n_pairs] source atom i of each pair (same configuration) */
    const double *J;          /* [n_pairs, 3, d] J_p[alpha] = d x_i / d r_{a,alpha}       */
    const double *y;          /* [N] targets: n_cfg energies, then 3 n_atoms forces (a-major),
                                 then 6 n_cfg virials (A-major, xx yy zz yz xz xy) if pair_u */
    const double *sigma;      /* [N] per-target sigma (> 0), same order as y              */
    double delta;             /* kernel scale delta                                       */
    int32_t zeta;             /* kernel power, integer 1..63                              */
    int32_t memory;           /* gap_memory of every pointer above                        */
    double jitter;            /* absolute diagonal jitter of K_MM (paper: 1e-8)           */
    /* [n_pairs, 3] displacement u_p = r_a - r_i of each pair's target from its source, or
     * NULL.  Given (with pair data), six virial rows per configuration follow the force
     * rows: the derivatives of the energy with respect to a homogeneous lattice strain
     * (Sec. II), under which x_i moves by sum over the pairs with source i of J_p eps u_p:
     *   K_{(A,v),s} = -delta^2 zeta sum_{p in pairs(A)} (x_i . x_s)^(zeta-1)
     *                 (1/2) [(J_p[alpha] . x_s) u_p[beta] + (J_p[beta] . x_s) u_p[alpha]]
     * for Voigt component v = (alpha, beta) in the order xx, yy, zz, yz, xz, xy. */
    const double *pair_u;
    /* Two-body sub-GAP (the appendix's distance_2b descriptors with covariance_type=ard_se)
     * summed into the same fit, or n_sparse_2b = 0.  Its n_sparse_2b sparse distances are
     * columns n_sparse .. n_sparse + n_sparse_2b - 1 of the design matrix (c and the
     * weights of gap_solve / gap_predict have n_sparse + n_sparse_2b entries), K_MM is block
     * diagonal over the two sets, and
     *   k(r, r') = delta_2b^2 exp(-(r - r')^2 / (2 theta_2b^2)) f(r) f(r'),
     *   f(r) = 1 below cutoff_2b - width_2b, (1 + cos(pi (r - cutoff_2b + width_2b) / width_2b)) / 2
     *          up to cutoff_2b, 0 beyond.
     * Bonds: every atom pair within the cutoff listed from both ends and grouped by atom --
     * the bonds of atom a are [bond_ptr[a], bond_ptr[a+1]) -- each with its length r and
     * unit vector u = (r_a - r_j) / r.  Rows, each scaled by 1/sigma like the others: energy
     * (1/2) sum over the configuration's bonds of k(r, r_t); force (a, alpha) -sum over a's
     * bonds of dk/dr(r, r_t) u[alpha]; virial (A, v) -(1/2) sum over A's bonds of
     * dk/dr(r, r_t) r u[alpha] u[beta]. */
    int64_t n_bonds, n_sparse_2b;
    const int64_t *bond_ptr;  /* [n_atoms + 1] */
    const double *bond_r;     /* [n_bonds] bond lengths (> 0)                       */
    const double *bond_u;     /* [n_bonds, 3] unit vectors (r_a - r_j) / r            */
    const double *sparse_r;   /* [n_sparse_2b] sparse distances                       */
    double delta_2b, theta_2b, cutoff_2b, width_2b;  /* theta, width > 0; width <= cutoff */
} gap_problem;

typedef struct {
    int32_t iterations;       /* refinement iterations run (0 in FP64 mode)               */
    int32_t converged;        /* 1 if the refinement met its tolerance                    */
    double rel_update;        /* last ||delta c|| / ||c||                                 */
    double residual_norm;     /* ||b - A c||_2 of the stacked system (FP64)               */
    double time_ms[4];        /* device time of assemble, factor, solve, refine          */
} gap_solve_info;

/* Device time per kernel class of the calls since the last gap_assemble on a
 * ctx, from CUDA events recorded on the ctx's stream around each launch group. */
typedef enum {
    GAP_PROF_COPY_IN = 0,     /* host-to-device staging of host-memory inputs          */
    GAP_PROF_PACK = 1,        /* operand splitting for the tensor cores                */
    GAP_PROF_GEMM_ENERGY = 2, /* energy rows and per-atom force weights (Eq. 6)        */
    GAP_PROF_GEMM_FORCE = 3,  /* force rows                                            */
    GAP_PROF_KMM_CHOL = 4,    /* K_MM + jitter, Cholesky, stacking U (Eq. 7)           */
    GAP_PROF_QR_PANEL = 5,    /* Householder panel factorisation                       */
    GAP_PROF_QR_UPDATE = 6,   /* compact-WY trailing updates (V^T C and C - V T^T W)   */
    GAP_PROF_SOLVE = 7,       /* back substitution (Eq. 12)                            */
    GAP_PROF_REFINE = 8,      /* FP64 refinement                                       */
    GAP_PROF_PREDICT = 9,     /* predictions (Eqs. 1, 2)                               */
    GAP_PROF_N = 10
} gap_prof_class;

typedef struct {
    double ms[GAP_PROF_N];      /* summed device milliseconds per class */
    int32_t groups[GAP_PROF_N]; /* timed launch groups per class        */
} gap_profile;

/* Create a context bound to `cuda_stream` (a cudaStream_t, or NULL) on the
 * current CUDA device.  Returns GAP_ERR_INVALID for an unknown precision. */
gap_status gap_create(gap_ctx **ctx, gap_precision prec, void *cuda_stream);

/* Release every workspace of the ctx (synchronises its stream first). */
void gap_destroy(gap_ctx *ctx);

/* One-line description of the last failure on this ctx ("" if none). */
const char *gap_last_error(const gap_ctx *ctx);

/* Tunables: "max_iter" (refinement iterations, default 30), "tol" (relative
 * update tolerance of the refinement, default 1e-10), "qr_nb" (QR panel width,
 * 16..128, multiple of 16; default 32), "qr_two_level" (mixed precisions: outer
 * QR panels of 128 applied on the tensor cores, default 1), "qr_passes" (mixed
 * precisions: tensor-core passes of those updates, 1 = plain TF32 or 3 = split
 * TF32 of about FP32 accuracy; default 1 — the FP32 QR only preconditions the
 * FP64 refinement, whose result does not depend on it), "cqr_passes" (mixed
 * precisions: CholeskyQR passes per 32-column QR panel, 1 or 2, default 1),
 * "batch_lanes" (fits in flight in gap_fit_batched, 1..16, default 4),
 * "force_walk" (mixed precisions: consecutive output tiles each CTA of the
 * tensor-core force pass takes per step of its walk, 1..32, default 4; a
 * schedule choice only, the rows do not depend on it),
 * "tsqr_shards" (0..64, default 0: factor the data rows as up to this many row
 * blocks and merge their R factors, see gap_factor),
 * "j_ring_rows" (mixed precisions only, 0 or a positive multiple of 128, default 0:
 * the J ring.  The tensor-core force pass then converts and multiplies this many
 * packed Jacobian rows at a time, 42 pairs per 128 rows, through one operand slot
 * instead of holding every pair's converted rows.  A host problem's J is copied
 * chunk by chunk through two FP64 slots of that many pairs, not staged whole: the
 * layout for problems whose Jacobians do not fit on the device, like the 132 GB of
 * the three-species d = 1024 workload of Sec. IV.  The fit does not depend on it.
 * Problems with virial rows are refused (GAP_ERR_INVALID).  gap_predict with a host
 * problem walks the same ring by whole atoms, so that no atom may have more pairs
 * than one slot holds.  "j_ring_direct" (0 or 1, default 0): a host J in page-locked
 * memory (cudaHostAlloc, or cudaHostRegister over the whole array) that the device
 * maps at the same address is read in place by the packing and prediction kernels.
 * There are then no FP64 slots and no copies.  The first and the last byte of J are
 * checked, and GAP_ERR_INVALID is returned when they are not such memory; the caller
 * makes sure that every byte between them is.  After a ring assembly of a host problem, gap_predict with
 * targets == NULL reads no Jacobians at all: see gap_predict.  Virial predictions
 * are refused for host targets.)
 * "graphs" (0 or 1, default 1): gap_factor's QR (without "tsqr_shards") runs as a CUDA graph
 * of its launches, captured the second time the ctx factors a problem of the same shape with
 * the same buffers and replayed after (up to 8 graphs per ctx; the QR's profile time is then
 * reported as GAP_PROF_QR_UPDATE only).  The result does not depend on it.
 * Unknown keys, and "j_ring_rows" > 0 on an FP64 ctx, give GAP_ERR_INVALID. */
gap_status gap_set_option(gap_ctx *ctx, const char *key, double value);

/* Device bytes the ctx will hold for this problem at this precision
 * (the (N+M) x M design matrix of Eq. (7) and every workspace), without the
 * option "tsqr_shards" = G's stack of (G+1) M rows x (M+1) columns. */
gap_status gap_workspace_size(const gap_problem *p, gap_precision prec, size_t *bytes);

/* gap_workspace_size with the option "j_ring_rows" = j_ring_rows.  The converted
 * Jacobian rows count as one slot, and a host problem adds the two FP64 slots.
 * GAP_ERR_INVALID for a value the option refuses.  Predictions' scratch space is
 * not counted; with forces it is about n_atoms x M x 12 bytes. */
gap_status gap_workspace_size_ring(const gap_problem *p, gap_precision prec, int64_t j_ring_rows, size_t *bytes);

/* Rows of the stacked matrix A of Eq. (7): N + M, with N = n_cfg + 3 n_atoms
 * (forces) or n_cfg (energies only). */
int64_t gap_design_rows(const gap_problem *p);

/* Assemble the data rows Sigma^{-1/2} K_NM (Eqs. 6, 7; energy and force rows,
 * the zeta-power and Sigma scaling fused into the GEMM epilogues) and the
 * right-hand side b = [Sigma^{-1/2} y ; 0] (Eq. 8).  Host pointers
 * (memory == GAP_MEM_HOST) are copied to the device inside this call.
 * Validates the problem on the host (sizes, monotone pointers, pair sources in
 * the target's configuration, sigma > 0, 1 <= zeta <= 63; in the mixed precisions at
 * most 16384 columns, n_sparse + n_sparse_2b, which the refinement pass holds per
 * thread); GAP_ERR_INVALID on failure. */
gap_status gap_assemble(gap_ctx *ctx, const gap_problem *p);

/* K_MM + jitter I, its Cholesky K_MM = U^T U (FP64), U stacked as the last M
 * rows of A (Eq. 7), then the blocked Householder QR A = QR (Eqs. 11, 12).
 * With the option "tsqr_shards" = G > 0, the row-block distribution of the
 * multi-process solver (Sec. III-B: configurations split over processes by rows,
 * the solution independent of the row order) runs on this GPU as a TSQR: the
 * data rows are cut into up to G blocks of whole 128-row tiles, each at least
 * M + 128 rows long (fewer blocks when N is short; none when N < M + 128 or
 * when N + M rounded up to a multiple of 128 is below N + 128); each
 * block [A_g | b_g] is factored on its own into R_g and Q_g^T b_g, and one QR of
 * the stack [R_1; ...; R_G; U] (right-hand side [Q_1^T b_1; ...; 0]) gives R and
 * Q^T b.  gap_tsqr_blocks reports the block count used.
 * Synchronises to report GAP_ERR_NOT_SPD (non-positive pivot). */
gap_status gap_factor(gap_ctx *ctx);

/* Row blocks of the last gap_factor's TSQR; 0 when A was factored as one
 * matrix (the option off, N too short, or the mixed precisions' fallback to
 * column panels for an ill-conditioned panel); -1 for a NULL ctx. */
int gap_tsqr_blocks(const gap_ctx *ctx);

/* The TSQR plan gap_factor uses for n_data_rows = N data rows, M sparse points and
 * "tsqr_shards" = want (host only, no GPU needed): returns the block count G (0: one
 * QR of the whole matrix) and, when row0 and rows are non-NULL (caller-owned, at
 * least 64 entries each), block g's first row and row count.  -1 for negative sizes. */
int gap_tsqr_plan(int64_t n_data_rows, int64_t M, int want, int64_t *row0, int64_t *rows);

/* c = R^{-1} Q^T b (Eq. 12) into c_dev ([M] FP64, device).  In the mixed
 * precisions this is the starting point of FP64 refinement against the
 * FP32-accurate design matrix.  If the refinement does not converge after a
 * factorisation with one-pass QR updates (the default), the FP32-accurate matrix
 * is refactored once with split-product updates and CholeskyQR2 panels and the
 * solve repeated.  Synchronises (fills *info if non-NULL).  GAP_ERR_RANK for a
 * zero R diagonal, GAP_ERR_NOT_CONVERGED if the refinement hit max_iter (c_dev
 * still holds the last iterate). */
gap_status gap_solve(gap_ctx *ctx, double *c_dev, gap_solve_info *info);

/* Predicted energies E_A = sum_{i in A} sum_s c_s k(x_i, x_s) (Eqs. 1, 2) and
 * forces F_a = -sum_{p in pairs(a)} J_p^T grad eps(x_i) for the configurations
 * in `targets` (y and sigma unused; pointers may be host or device per
 * targets->memory) with the sparse set of the last gap_assemble.  E_dev
 * [n_cfg] and F_dev [3 n_atoms] (may be NULL) are device buffers.
 * targets == NULL predicts for the problem of the last gap_assemble on this ctx
 * from its device copies: nothing is copied from the host again.  A device-memory
 * problem's arrays must still hold its data.  A gap_predict with host-memory
 * targets replaces those copies; a later NULL then fails with GAP_ERR_STATE until
 * the next gap_assemble.  When that problem was a host problem assembled through
 * the J ring (option "j_ring_rows"), its Jacobians are not on the device.  The
 * predictions are then its design rows times c_dev, scaled by sigma (Eq. 7: a data
 * row is its target's model value over sigma).  Energies use the FP64 energy rows.
 * Forces use the FP32-accurate rows, summed in double-float. */
gap_status gap_predict(gap_ctx *ctx, const gap_problem *targets, const double *c_dev, double *E_dev, double *F_dev);

/* gap_predict with the virials of the fitted model as well: V_dev [6 n_cfg] (device,
 * may be NULL; A-major, Voigt order xx yy zz yz xz xy) receives
 *   V_{A,v} = -sum over the pairs p of A's atoms of (1/2)
 *             [(J_p[alpha] . grad eps(x_i)) u_p[beta] + (J_p[beta] . grad eps(x_i)) u_p[alpha]],
 * the derivative of E_A with respect to a homogeneous lattice strain (Sec. II).
 * targets->pair_u (and its pair data) must be given when V_dev is; F_dev may be NULL. */
gap_status gap_predict_virial(gap_ctx *ctx, const gap_problem *targets, const double *c_dev, double *E_dev,
                              double *F_dev, double *V_dev);

/* Fill *out with the per-class device times of the calls since the last
 * gap_assemble on this ctx (synchronises the ctx's stream). */
gap_status gap_get_profile(gap_ctx *ctx, gap_profile *out);

/* Copy rows [row0, row0+nrows) of the current design matrix (Sigma^{-1/2} K_NM
 * stacked on zeros) into dst_dev as row-major FP64 [nrows x M].  `which` = 0:
 * the matrix the QR factors, readable between gap_assemble and gap_factor; 1: the
 * mixed precisions' residual matrix (FP32-accurate, its energy rows from their FP64
 * copy), readable from gap_assemble on.  FP64 mode keeps one matrix, factored in
 * place: either value reads it before gap_factor only.  GAP_ERR_STATE otherwise. */
gap_status gap_read_design(gap_ctx *ctx, int which, int64_t row0, int64_t nrows, double *dst_dev);

/* Copy the upper-triangular R (M x M) of the last gap_factor into dst_dev
 * (row-major FP64; entries below the diagonal are zero).  After a TSQR
 * factorisation this is the R of the merge QR. */
gap_status gap_read_r(gap_ctx *ctx, double *dst_dev);

/* Fit n independent problems (Sec. V: many fits for hyperparameter
 * exploration) with one call: each gets assemble -> factor -> solve.  Up to
 * "batch_lanes" fits (option, default 4) run at once, each lane a worker context
 * of the same precision and options with its own stream and host thread
 * (created on the first call, owned by ctx).  The fits are placed on the lanes
 * by greedy LPT on their estimated cost (rows x M^2, longest first), so the same
 * batch gives each lane the same fits in the same order on every call; a
 * fit's arithmetic does not depend on the lanes, so its result equals that of
 * a single fit.  The workers start after the work already queued on ctx's
 * stream; the call returns when every fit has finished.  c_dev[k] ([M_k] FP64,
 * device) receives fit k's weights, infos[k] (optional) its report.  The first
 * failure stops the remaining fits and is returned with the fit's index in
 * gap_last_error(ctx).  ctx's own matrices are not touched (gap_read_design and
 * gap_read_r keep referring to its last single fit). */
gap_status gap_fit_batched(gap_ctx *ctx, int n, const gap_problem *const *probs, double *const *c_dev,
                           gap_solve_info *infos);

/* ------------------------------------------- row blocks over several GPUs --
 * The row-block distribution of Sec. III-B as a TSQR over contexts (one per GPU or
 * process): each factors its own configurations' data rows, the R factors and
 * transformed right-hand sides are exchanged, and one QR of their stack with U gives
 * the fit.  The stack [R_1 z_1; ...; R_G z_G; U 0] has the same normal equations as the
 * whole [Sigma^{-1/2} K ; U | b], so c does not depend on how the configurations were
 * split (the paper notes the solution does not depend on the row order).  FP64 only
 * (GAP_ERR_INVALID otherwise): a mixed-precision refinement would need the residual of
 * every block's rows in each iteration.
 *
 * gap_tsqr_local: after gap_assemble of this block's configurations, the Householder QR
 * of its data rows [Sigma^{-1/2} K_g | b_g] (at least n_sparse of them; no U).  Rz_dev
 * receives [R_g | z_g], row-major FP64 [M x (M+1)] with zeros below the diagonal, and
 * *tail2 the squared norm of the rest of Q_g^T b_g (host).  Synchronises.  The ctx then
 * accepts gap_tsqr_merge only (gap_factor needs a new gap_assemble).
 * gap_tsqr_merge: with the sparse set of this ctx's last gap_assemble (every block must
 * use the same one), K_MM + jitter = U^T U (Eq. 7) and the QR of the stack of the G
 * blocks Rz_dev (device, row-major [G x M x (M+1)], in any order) on U; tail2 is the sum
 * of the blocks' *tail2.  gap_solve then gives c, with the residual norm of the whole
 * fit, and gap_read_r the merged R. */
gap_status gap_tsqr_local(gap_ctx *ctx, double *Rz_dev, double *tail2);
gap_status gap_tsqr_merge(gap_ctx *ctx, int G, const double *Rz_dev, double tail2);

/* ------------------------------------------------ CUR sparse-point selection --
 * Chooses the sparse set by leverage-score sampling (the cur_points choice of
 * Secs. III-A and III-C, after Mahoney and Drineas, PNAS 106 (2009) 697): for every species
 * t with n_select[t] > 0, the rows X_t of the descriptors of its atoms (in atom
 * order) give the rank-k leverage scores
 *     pi_i = |U_k[i, :]|^2 / k,   X_t = U S V^T,  U_k: k leading left singular vectors,
 * and n_select[t] distinct atoms of t are drawn without replacement with
 * probabilities proportional to pi: the atoms with the n_select[t] largest keys
 * log(u_i) / pi_i (Efraimidis and Spirakis, IPL 97 (2006) 181), ties to the
 * lower atom index, and -inf as the key of an atom with pi_i = 0.
 * U_k comes from a randomised range finder with test matrix omega and
 * power_iters power iterations (Halko, Martinsson and Tropp, SIAM Rev. 53 (2011)
 * 217, Algs. 4.4 and 5.1): Q = orth(X_t omega), then power_iters times
 * Q = orth(X_t (X_t^T Q)); B = Q^T X_t; U_k = Q W_k with W_k the eigenvectors
 * of B B^T for its k largest eigenvalues.  For X_t of rank <= l the scores are
 * the exact ones (with probability one over omega); otherwise they approach them
 * as power_iters grows.  All arithmetic is FP64.
 * Arguments (all arrays device memory except n_select):
 *   X [n_atoms x d] row-major descriptors; atom_species [n_atoms] in
 *   [0, n_species) (NULL when n_species == 1); n_select [n_species] (host) sparse
 *   points per species; 1 <= k <= l <= min(d, 128); 0 <= power_iters <= 64;
 *   omega [d x l] row-major (one test matrix for every species; draw it, e.g.
 *   standard normal); u [n_atoms] in (0, 1], one uniform per atom;
 *   selected [sum n_select] receives the chosen atom indices, species after
 *   species, ascending within each; leverage [n_atoms] (may be NULL) receives
 *   pi_i for the atoms of every species with n_select > 0 (other entries are
 *   not written).
 * Errors: GAP_ERR_INVALID for bad sizes, a species value out of range, or a
 * species with fewer atoms than n_select or than l; GAP_ERR_RANK when the
 * range finder's CholeskyQR meets a non-positive pivot (rows of a species that
 * span no direction; rows spanning fewer than l directions but at least k
 * usually still factor, after the first pass's shift, and then give exact
 * scores); GAP_ERR_NOMEM / GAP_ERR_CUDA.  err (may be NULL) gets a one-line reason.
 * Ordering: work goes on cuda_stream; temporaries (about
 * 8 (d + 3 l) n + 400 l max(d, l) bytes for the largest species, n its atoms)
 * come from the stream-ordered allocator and are freed before the call
 * returns, and the call synchronises the stream before it returns. */
gap_status gap_select_cur(const double *X, int64_t n_atoms, int64_t d, const int32_t *atom_species,
                          int32_t n_species, const int64_t *n_select, int32_t k, int32_t l, int32_t power_iters,
                          const double *omega, const double *u, int64_t *selected, double *leverage,
                          void *cuda_stream, char *err, size_t err_len);

/* ---------------------------------------------- allocation-free predictions --
 * Some callers cannot allocate device memory while they need predictions: a
 * molecular-dynamics engine or serving loop that asks for energies and forces
 * every step while its own allocator or memory pool owns the GPU's memory (so
 * cudaMalloc would fail, and cudaFree would synchronise the device in the
 * middle of a step), or code that runs inside another framework's fixed memory
 * budget.  gap_predict_static computes the predictions of gap_predict
 * (Eqs. 1, 2 and the force chain rule) for them without allocating: it calls
 * no cudaMalloc, cudaFree or allocating library routine and needs no ctx.
 * It always predicts in FP64 (the SIMT kernels of an FP64 context): its results
 * equal gap_predict's in an FP64 context, and match a mixed-precision context's
 * tensor-core predictions to that path's accuracy.
 * The paper has no counterpart; this is an interface of this library only.
 *
 * Scratch: one device array of GAP_PREDICT_STATIC_SCRATCH_BYTES compiled into
 * the library; every GPU that loads the library holds it until the process
 * exits.  A prediction must fit in it: 256 + 16 n_atoms bytes, plus
 * 8 n_atoms d + 8 n_sparse bytes when forces are requested; larger targets
 * are rejected with GAP_ERR_INVALID and a message (use gap_predict for them),
 * before any size product is formed.
 * Arguments: every pointer in *targets (targets->memory must be
 * GAP_MEM_DEVICE), c_dev, E_dev [n_cfg] and F_dev [3 n_atoms] (may be NULL) is
 * device memory; targets->Xs and targets->sparse_species are the fit's sparse
 * set and c_dev [n_sparse] its weights; y and sigma are not read.  err (may be
 * NULL) receives a one-line reason on failure.
 * Set-up: the first call on each device resolves the array's device address
 * (cudaGetSymbolAddress, with that device current).  The address is resolved
 * again when the device's context has changed (after a cudaDeviceReset).
 * Ordering: work goes on cuda_stream.  Every call synchronises that stream while
 * it validates the index arrays (it reads a status word back), so a call cannot
 * be captured in a CUDA graph; it returns with the prediction enqueued.
 * Sharing: all calls on a device use the same array, which keeps the last
 * call's contents; each call clears the status word it needs at zero and
 * writes every other region before reading it.  Calls whose work overlaps on
 * the GPU (other streams or host threads) race on the array: serialise them. */
#define GAP_PREDICT_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
gap_status gap_predict_static(const gap_problem *targets, const double *c_dev, double *E_dev, double *F_dev,
                              void *cuda_stream, char *err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* LIBGAP_GAP_H */
