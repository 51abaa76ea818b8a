// Internal declarations of libgap (not part of the C-ABI).
#pragma once

#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gap.h"

namespace gap {

// Device-side status word written by kernels (first error wins).
struct DevStatus {
    int code;      // gap_status
    int pad;
    int64_t index; // offending index (pivot, row, pair, ...)
};

// Growable device allocation owned by a ctx.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t b = bytes ? bytes : 256;
        cudaError_t e = cudaMalloc(&p, b);
        if (e == cudaSuccess) cap = b;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T> T *as() const { return reinterpret_cast<T *>(p); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
};

// CUDA-event timing of launch groups by kernel class (gap_prof_class).
struct Prof {
    cudaStream_t s = nullptr;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Mark { int cls; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    int open_cls = -1;
    cudaEvent_t open_ev = nullptr;
    cudaEvent_t get() {
        if (used == pool.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    void begin(int cls) {
        open_ev = get();
        open_cls = cls;
        if (open_ev) cudaEventRecord(open_ev, s);
    }
    void end() {
        cudaEvent_t e = get();
        if (e && open_ev) {
            cudaEventRecord(e, s);
            marks.push_back({open_cls, open_ev, e});
        }
        open_ev = nullptr;
    }
    void reset() {
        used = 0;
        marks.clear();
    }
    ~Prof() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

// Device view of one assembled problem.
struct Dims {
    int64_t n_cfg, n_atoms, d, n_pairs, M;  // M: every column (SOAP sparse points, then two-body ones)
    int64_t Ms, M2;  // SOAP sparse points (rows of X_s) and two-body sparse distances (M = Ms + M2)
    int64_t N;     // data rows
    int64_t rows;  // N + M
    int64_t ld;    // leading dimension of the column-major design matrix (>= rows)
    int zeta;
    double delta, jitter;
    bool forces, species;
    bool virials;  // six virial rows per configuration after the force rows
};

constexpr int kTsqrMax = 64;  // most row blocks of a TSQR factorisation

}  // namespace gap

struct gap_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    gap_precision prec = GAP_PREC_FP64;
    std::string err;
    int state = 0;  // 0 empty, 1 assembled, 2 factored
    // options
    int max_iter = 30;
    double tol = 1e-10;
    int qr_nb = 32;
    bool qr_two_level = true;
    int qr_passes = 1;  // tensor-core passes of the FP32 QR trailing updates (1 or 3)
    int cqr_passes = 1; // CholeskyQR passes per FP32 QR panel (1 or 2)
    int qr_fallbacks = 0;      // factorisations redone with column panels
    bool qr_lean = false;      // the last FP32 QR ran one-pass updates or one CholeskyQR pass
    int qr_refactors = 0;      // solves that refactored with the accurate QR after no convergence
    int batch_lanes = 4;       // gap_fit_batched: fits in flight at once (worker contexts)
    int force_walk = 4;        // tensor-core force pass: consecutive tiles per step of a CTA's walk
    // TSQR factorisation (the row-block distribution of Sec. III-B on one GPU): the data rows
    // in up to tsqr_shards row blocks, each factored on its own, then one QR of the stacked
    // [R_1; ...; R_G; U].  tsqr_used: blocks of the last factorisation (0: one QR of A)
    int tsqr_shards = 0;
    int tsqr_used = 0;
    // a merge of row blocks factored by other contexts (gap_tsqr_merge): their residual
    // tails are not in this ctx, only the sum of their squares
    bool tsqr_ext = false;
    double tsqr_ext_tail2 = 0.0;
    int64_t tsqr_r0[gap::kTsqrMax] = {}, tsqr_n[gap::kTsqrMax] = {};
    int64_t r_ld = 0;          // leading dimension of the matrix holding R (A or the stack)
    bool owns_stream = false;  // worker contexts own their streams
    std::vector<gap_ctx *> lanes;  // gap_fit_batched worker contexts (created on first use)
    gap::Dims dm{};
    // inputs kept after assemble (device)
    gap::DevBuf Xs, sparse_sp;
    // K_MM's diagonal blocks (ascending ends, the last M): the sparse points of one species
    // are contiguous and no species repeats (or the two-body block follows the SOAP one);
    // empty when K_MM is factored as one block
    std::vector<int64_t> kmm_ends;
    // the problem last assembled, as a device-memory problem (the staged copies of a host
    // problem, or the caller's device arrays): gap_predict with no targets uses it
    gap_problem last_dev{};
    bool have_last = false;
    // a host problem's J staged in chunks on a copy stream (mixed assembly): chunk i holds
    // the Jacobian rows [j_rows[i], j_rows[i+1]) once j_ev[i] has completed
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_stage = nullptr, j_ev[8] = {};
    int n_jchunks = 0;
    int64_t j_rows[9] = {};
    // J ring (option j_ring_rows, mixed precisions): the force pass packs and multiplies
    // j_ring_rows Jacobian rows at a time, and a host problem's J is copied through the
    // two FP64 slots of ring_J (events: slot landed, slot free) instead of staged whole
    int64_t j_ring_rows = 0;
    bool j_ring_direct = false;  // a page-locked host J is read in place by the kernels
    gap::DevBuf ring_J;
    cudaEvent_t ring_ev[4] = {};
    // staging of host inputs and derived index arrays
    gap::DevBuf h_cfg_ptr, h_X, h_atom_sp, h_pair_ptr, h_pair_src, h_J, h_y, h_sigma;
    gap::DevBuf atom_cfg, pair_tgt;
    // virial rows as force rows of pseudo-targets (k_virial.cu): index arrays and the
    // per-atom strain Jacobians G of the problem last assembled (or predicted)
    gap::DevBuf h_pair_u, vp_ptr, vp_src, vp_tgt, vG;
    gap::DevBuf h_bond_ptr, h_bond_r, h_bond_u, h_sparse_r;  // two-body inputs of a host problem
    gap::DevBuf sparse_r;  // the fit's two-body sparse distances, and its constants below
    double tb_delta = 0, tb_theta = 1, tb_cutoff = 1, tb_width = 1;
    // design matrices (column-major [ld x (M+1)], last column = b)
    gap::DevBuf A;       // FP64 (FP64 mode) or FP32 (mixed: QR matrix)
    gap::DevBuf Aacc;    // FP32 accurate residual matrix (mixed)
    gap::DevBuf b64;     // FP64 right-hand side [rows]
    gap::DevBuf Wf;      // per-atom force weights [n_atoms x M] (FP64 or FP32)
    gap::DevBuf tc_ops;  // tensor-core operand staging (converted descriptors / Jacobians)
    gap::DevBuf pred_work;  // prediction scratch of the mixed precisions (weights, gradients, partials)
    // factor workspaces
    gap::DevBuf Kmm, tau, T, Wpart, Wred, part, diagrow, status, qr_outer;
    gap::DevBuf tsqr;   // TSQR merge stack, column-major [round_up((G+1) M, 128) x (M+1)]
    // solve workspaces
    gap::DevBuf vecs;
    gap::DevBuf rinv;   // mixed refinement: R^{-1} and its transpose (FP32)
    gap::DevBuf cg_ws;  // mixed refinement: split vector and per-CTA partials of the fused pass
    gap::DevBuf E64;    // mixed: the accurate energy rows in FP64, row-major [n_cfg x M]
    gap::DevBuf head_t; // mixed refinement: residual of the head rows [round_up(n_cfg, 32)]
    gap::DevStatus *h_status = nullptr;  // pinned host mirror
    cudaEvent_t ev[8] = {};
    gap::Prof prof;
    // QR launch sequences captured as CUDA graphs (option "graphs"): one per problem shape
    // and set of buffers, captured the second time that key is factored, replayed after (up
    // to 8 per ctx: with tens of large graphs alive in a process their launches cost
    // milliseconds each, so a ctx cycling through many shapes keeps launching kernels)
    struct QrGraph {
        std::vector<uintptr_t> key;
        cudaGraphExec_t exec = nullptr;
        int uses = 0;
    };
    bool use_graphs = true;
    std::vector<QrGraph> qr_graphs;
    cudaStream_t gstream = nullptr;  // the stream the graphs are captured on
};

namespace gap {

// Error helpers used by the ABI layer.
gap_status fail(gap_ctx *c, gap_status s, const std::string &msg);
gap_status cuda_fail(gap_ctx *c, cudaError_t e, const char *where);

#define GAP_CUDA(ctx, call)                                                   \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return gap::cuda_fail((ctx), e_, #call);       \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// The tensor-core force pass packs the Jacobian rows in pair tiles: 128 rows holding 42
// consecutive pairs (three rows each) and two zero rows.  Packed rows of n_pairs pairs:
constexpr int kForcePairsPerTile = 42;
inline int64_t force_pack_rows(int64_t n_pairs) { return ceil_div(n_pairs, kForcePairsPerTile) * 128; }

// Layout of the FP32-accurate design matrix of the mixed precisions (read only by
// the refinement): blocks of ACC_RB = 32 rows, each stored column by column (32
// consecutive floats per column, nc columns per block), so that one block of rows
// is one contiguous stretch of memory.
constexpr int ACC_RB = 32;
__host__ __device__ inline int64_t acc_index(int64_t row, int64_t col, int64_t nc) {
    return (row / ACC_RB) * (ACC_RB * nc) + col * ACC_RB + (row % ACC_RB);
}

// ---- kernels launched by the ABI layer (each returns the launch error) ----

// index arrays: atom -> configuration, pair -> target atom; validation
cudaError_t launch_segment_ids(const int64_t *ptr, int64_t n_seg, int64_t *out_ids, cudaStream_t s);
cudaError_t launch_validate(const Dims &dm, const int64_t *cfg_ptr, const int64_t *pair_ptr, const int64_t *pair_src,
                            const int64_t *atom_cfg, const double *sigma, const int32_t *atom_sp,
                            const int32_t *sparse_sp, DevStatus *st, cudaStream_t s);

// SIMT assembly (T = double or float): energy rows + per-atom force weights, then force rows
template <class T>
cudaError_t launch_energy_simt(const Dims &dm, const double *X, const double *Xs, const int32_t *atom_sp,
                               const int32_t *sparse_sp, const int64_t *cfg_ptr, const int64_t *atom_cfg,
                               const double *sigma, T *A, T *Wf, cudaStream_t s);
template <class T>
cudaError_t launch_force_simt(const Dims &dm, const double *J, const double *Xs, const int64_t *pair_ptr,
                              const int64_t *pair_src, const int64_t *pair_tgt, const double *sigma, const T *Wf,
                              T *A, cudaStream_t s);

// rhs b = [y / sigma ; 0] (FP64) and its copy into column M of A
template <class T>
cudaError_t launch_rhs(const Dims &dm, const double *y, const double *sigma, double *b64, T *A, cudaStream_t s,
                       bool blocked = false);

// K_MM + jitter (FP64, column-major M x M).  double_float: dot products in double-float on
// the FP32 units, the lower triangle only, X_s split first into split_ws (2 M d floats).
cudaError_t launch_kmm(const Dims &dm, const double *Xs, const int32_t *sparse_sp, double *K, cudaStream_t s,
                       bool double_float = false, float *split_ws = nullptr);
// blocked Cholesky K = L L^T in place (lower, column-major); status on failure.  ends
// (n_ends ascending block ends, the last M; or none): K is block diagonal with those
// diagonal blocks, each factored on its own (no trailing update crosses a block end).
cudaError_t cholesky_lower(double *K, int64_t M, DevStatus *st, cudaStream_t s, const int64_t *ends = nullptr,
                           int n_ends = 0);
// The same factor with the trailing matrix in double-float (mixed precisions); ws holds
// cholesky_df_workspace_bytes(M).
size_t cholesky_df_workspace_bytes(int64_t M);
cudaError_t cholesky_lower_df(double *K, int64_t M, float *ws, DevStatus *st, cudaStream_t s,
                              const int64_t *ends = nullptr, int n_ends = 0);
// The ctx buffer that holds R^{-1} and R^{-T} (FP32, M x round_up(M, 32) each) in the
// refinement, and before it the double-float Cholesky's workspace and the split X_s of
// K_MM (d = the descriptor length).
inline size_t rinv_bytes(int64_t M, int64_t d = 0) {
    const size_t w = 2 * sizeof(float) * (size_t)round_up(M, 32) * (size_t)M, k = cholesky_df_workspace_bytes(M);
    const size_t x = 2 * sizeof(float) * (size_t)M * (size_t)d;  // split X_s for K_MM
    return std::max(std::max(w, k), x);
}
// A[N + i, j] = U[i, j] = L[j, i] (i <= j) for every target matrix
template <class T>
cudaError_t launch_stack_u(const Dims &dm, const double *L, T *A, cudaStream_t s, bool blocked = false);

// blocked Householder QR of the column-major [rows x ncols] matrix (ncols = M + 1:
// the last column is b and only receives the reflectors)
// (FP32 with outer_ws != NULL: two-level blocking, outer panels of 128 applied
// on the tensor cores; FP64: flat panels of nb)
template <class T>
cudaError_t householder_qr(T *A, int64_t rows, int64_t M, int64_t ld, int nb, T *tau, T *Tbuf, T *part,
                           T *diagrow, T *Wpart, T *Wred, int n_row_blocks, cudaStream_t s, Prof *prof,
                           void *outer_ws, int *status, int upd_passes, int cqr_passes);
// upd_passes: tensor-core passes of the two-level trailing updates (3: split TF32,
// about FP32 accuracy; 1: plain TF32)
cudaError_t householder_qr_two_level(float *A, int64_t rows, int64_t M, int64_t ld, int nb, float *tau, float *Tbuf,
                                     float *part, float *diagrow, float *Wpart, float *Wred, int n_row_blocks,
                                     cudaStream_t s, Prof *prof, void *outer_ws, int *status, int upd_passes,
                                     int cqr_passes);
size_t qr_outer_workspace_bytes(int64_t rows, int64_t M);
// TSQR merge: the M x (M+1) top of the row block at row r0 of the column-major A (R in
// the upper triangle of the first M columns, the transformed right-hand side in column
// M) into rows [srow, srow + M) of the stack S; zero below the diagonal, and in column M
// when zero_b (the block of U, whose right-hand side is zero).
template <class T>
cudaError_t tsqr_gather(const T *A, int64_t ld, int64_t r0, int64_t M, T *S, int64_t lds, int64_t srow, bool zero_b,
                        cudaStream_t s);

// Mixed refinement (k_refine.cu).  W = R^{-1} (FP32, column-major ldw, upper) and
// Wt = W^T from the FP32 R (upper part of the column-major [ldr x M] R) and the
// FP64 inverses of its 64 x 64 diagonal blocks (trsv_invert_blocks layout).
cudaError_t triangular_inverse(const float *R, int64_t ldr, int64_t M, const double *Dinv, float *W, float *Wt,
                               int64_t ldw, cudaStream_t s);
// One pass over the rows of the FP32-accurate matrix A (row-block layout, M + 1
// columns of which the first M are used): t = A u, or the residual t = rhs - A u
// when rhs is given; sq = |t|^2 and, when w is given, w = A^T t.  df: products and
// sums in double-float (about 48 bits), else plain FP32 (the recursive CGLS
// corrections).  ws: cgls_workspace_bytes(M); needs cgls_fused_fits(M).
size_t cgls_workspace_bytes(int64_t M);
bool cgls_fused_fits(int64_t M);
// status: the device status word (a bounded wait that runs out records GAP_ERR_TIMEOUT).
cudaError_t cgls_pass(const float *A, int64_t rows, int64_t M, const double *u, const double *rhs, double *w,
                      double *sq, void *ws, bool df, int *status, cudaStream_t s);
// Rows [row0, row0 + nrows) of the row-block matrix as row-major FP64 [nrows x M];
// and its column-major copy [ld x (M + 1)].
cudaError_t read_rows_acc(const float *A, int64_t M, int64_t row0, int64_t nrows, double *dst, cudaStream_t s);
// The same pass over the head rows [0, rh) in FP64: rows below n_e from E64 (the FP64
// energy rows, row-major [n_e x M]), the rest from the row-block matrix A.  ws
// (cgls_head_bytes) receives the head's residual t in its first rh doubles, then the
// column pass's partial sums; w and sq are added to (accumulate) or written.
size_t cgls_head_bytes(int64_t rh, int64_t M);
cudaError_t cgls_head(const double *E64, int64_t n_e, const float *A, int64_t rh, int64_t M, const double *u,
                      const double *rhs, double *w, double *sq, double *ws, bool accumulate, cudaStream_t s);
cudaError_t acc_to_colmajor(const float *A, int64_t ld, int64_t M, float *out, cudaStream_t s);
// Predictions of the assembled problem from its design rows (mixed precisions): E [n_e] =
// sigma * (E64 c) over the FP64 energy rows, and out [nrows] = sigma[row0 + i] * (A[row0 + i, :] . c)
// over rows [row0, row0 + nrows) of the FP32 row-block matrix A.  ws: 2 M floats.
cudaError_t predict_from_rows(const double *E64, int64_t n_e, const float *A, int64_t M, int64_t row0, int64_t nrows,
                              const double *sigma, const double *c, float *ws, double *E, double *out, cudaStream_t s);
size_t cqr_workspace_bytes(int64_t rows);
constexpr int kStatusCqrFallback = 100;  // internal: a CholeskyQR2 panel broke down

// back substitution c = R^{-1} z, R upper in A[0:M, 0:M] (column-major ld), z = A[0:M, M];
// work: ceil(M/64) 64^2 + M doubles (the first part keeps the diagonal-block inverses)
template <class T>
cudaError_t back_substitution(const T *A, int64_t M, int64_t ld, const T *z, double *c, double *work, DevStatus *st,
                              cudaStream_t s);
// triangular solves with R (upper, column-major ld) in FP64 arithmetic, blocked by
// TNB = 64 with the diagonal-block inverses Dinv (trsv_invert_blocks):
// trans = 0: x = R^{-1} x ; trans = 1: x = R^{-T} x ; work: M doubles
constexpr int kTrsvBlock = 64;
template <class T>
cudaError_t trsv_invert_blocks(const T *R, int64_t M, int64_t ld, double *Dinv, DevStatus *st, cudaStream_t s);
template <class T>
cudaError_t trsv_upper(const T *R, int64_t M, int64_t ld, int trans, double *x, const double *Dinv, double *work,
                       cudaStream_t s);

// t = A v (rows x M, FP64 accumulation); g = A^T r
template <class T>
cudaError_t gemv_n(const T *A, int64_t rows, int64_t M, int64_t ld, const double *v, double *t, cudaStream_t s);
template <class T>
cudaError_t gemv_t(const T *A, int64_t rows, int64_t M, int64_t ld, const double *r, double *g, float *rsplit,
                   cudaStream_t s);  // rsplit: 2 rows floats of scratch (FP32 matrices)

// small vector helpers (FP64)
cudaError_t vec_dot(const double *a, const double *b, int64_t n, double *out, cudaStream_t s);
cudaError_t vec_axpy(double alpha_sign, const double *num, const double *den, const double *x, double *y, int64_t n,
                     cudaStream_t s);  // y += sign * (num/den) * x (scalars on device)
cudaError_t vec_xpby(const double *x, const double *num, const double *den, double *p, int64_t n,
                     cudaStream_t s);  // p = x + (num/den) p
cudaError_t vec_sub(const double *b, const double *t, double *r, int64_t n, cudaStream_t s);  // r = b - t
cudaError_t convert_to_f64(const void *src, int is_f32, int64_t n, double *dst, cudaStream_t s);

// Virial rows as force rows of pseudo-targets (k_virial.cu): vp_ptr [2 n_cfg + 1],
// vp_src / vp_tgt [2 n_atoms], G [2 n_atoms x 3 x d] (FP64) from the pairs' Jacobians and
// displacements u [n_pairs x 3]; virial_dims gives the Dims under which the force kernels
// produce the virial rows (pseudo-targets as atoms, row base n_cfg + 3 n_atoms).
cudaError_t launch_virial_pseudo_pairs(const Dims &dm, const int64_t *cfg_ptr, const int64_t *atom_cfg,
                                       const int64_t *pair_ptr, const int64_t *pair_src, const double *J,
                                       const double *pair_u, int64_t *vp_ptr, int64_t *vp_src, int64_t *vp_tgt,
                                       double *G, cudaStream_t s);
Dims virial_dims(const Dims &dm);

// The two-body sub-GAP (k_two_body.cu): bonds grouped by atom, sparse distances, the
// covariance's constants (delta^2, 1 / (2 theta^2), cutoff, transition width) and the
// first design-matrix column of its block.
struct TwoBodyDev {
    const int64_t *bond_ptr;
    const double *bond_r, *bond_u, *sparse_r;
    int64_t M2, col0;
    double delta2, inv2t2, rc, w;
};
cudaError_t launch_2b_validate(int64_t n_atoms, int64_t n_bonds, const TwoBodyDev &tb, DevStatus *st, cudaStream_t s);
// the block's energy, force and virial rows into A (and, mixed, A_acc and the FP64 energy rows)
template <class T>
cudaError_t launch_2b_rows(const Dims &dm, const int64_t *cfg_ptr, const TwoBodyDev &tb, const double *sigma, T *A,
                           float *Aacc, double *E64, cudaStream_t s);
// its K_MM block (+ jitter on the diagonal) into K [M x M]
cudaError_t launch_2b_kmm(const TwoBodyDev &tb, double jitter, double *K, int64_t M, cudaStream_t s);
// its predictions added to E, F (may be null) and V (may be null) for its weights c2 [M2]
cudaError_t launch_2b_predict(int64_t n_cfg, int64_t n_atoms, const int64_t *cfg_ptr, const TwoBodyDev &tb,
                              const double *c2, double *E, double *F, double *V, cudaStream_t s);
// V[3 t + alpha] = -sum over the pseudo-pairs of target t of G . grad[src] (FP64), the
// virials of the per-atom gradients grad [n_atoms x d] that predict_simt leaves in grad_work
cudaError_t predict_virial_simt(const Dims &vdm, const int64_t *vp_ptr, const int64_t *vp_src, const double *G,
                                const double *grad, double *V, cudaStream_t s);

// predictions (FP64 SIMT): E [n_cfg], F [3 n_atoms] (F may be null)
cudaError_t predict_simt(const Dims &dm, const double *X, const double *Xs, const int32_t *atom_sp,
                         const int32_t *sparse_sp, const int64_t *cfg_ptr, const int64_t *pair_ptr,
                         const int64_t *pair_src, const double *J, const double *c, double *E, double *F,
                         double *eps_work, double *grad_work, double *wmat_work, int64_t atom_chunk,
                         cudaStream_t s);

// read-back helpers
template <class T>
cudaError_t launch_read_rows(const T *A, int64_t ld, int64_t M, int64_t row0, int64_t nrows, double *dst,
                             cudaStream_t s);
template <class T>
cudaError_t launch_read_r(const T *A, int64_t ld, int64_t M, double *dst, cudaStream_t s);

}  // namespace gap
