// Tensor-core (tcgen05) assembly of the design matrix for the mixed precisions.
#pragma once

#include "gap_internal.cuh"

namespace gap {

// operand schemes: BF16 (three-slice split), TF32 (two-slice split), FP16 (the BF16 scheme
// for energy rows and predictions, a scaled two-slice FP16 split for the force rows)
enum class TcMode { BF16, TF32, FP16 };

struct TcInputs {
    const double *X, *Xs, *J;
    const int64_t *cfg_ptr, *atom_cfg, *pair_ptr, *pair_src, *pair_tgt;
    const double *sigma;
    const int32_t *atom_sp, *sparse_sp;
    int *status;  // device status word (GAP_ERR_TIMEOUT on a bounded-wait timeout)
    // J still arriving in chunks (0 = all present): chunk i holds the Jacobian rows
    // [j_rows[i], j_rows[i+1]) (multiples of 128; the last is the padded row count) once
    // j_ev[i] has completed
    int n_jchunks;
    const int64_t *j_rows;
    const cudaEvent_t *j_ev;
    // zeroed FP64 [n_cfg x M] (row-major) for the accurate energy rows, or null
    double *E64;
    // force pass: consecutive tiles each CTA takes per step of its tile walk (option force_walk)
    int force_walk = 4;
    // virial rows (dm.virials): the pair displacements and the buffers of the strain
    // Jacobians and pseudo-pair index arrays (launch_virial_pseudo_pairs), or null
    const double *pair_u = nullptr;  // [n_pairs x 3] pair displacements
    double *vG = nullptr;            // written by tc_assemble once every J chunk has landed
    int64_t *vp_ptr = nullptr, *vp_src = nullptr, *vp_tgt = nullptr;
    // J ring (ring_rows > 0, no virial rows): the force pass streams its operands through
    // one packed slot of ring_rows Jacobian rows (a multiple of 128: 42 pairs per 128
    // rows), packing and multiplying one chunk of pair tiles at a time.  A device J is read
    // in place (J).  A host J (h_J set, J null) is first copied chunk by chunk into the two
    // FP64 slots of ring_buf (ring_slot_pairs(ring_rows) pairs each) on ring_stream:
    // ring_ev[s] marks slot s landed, ring_ev[2 + s] slot s read (free again).  h_pair_ptr:
    // the host problem's pair_ptr (predictions walk the ring by atoms).
    int64_t ring_rows = 0;
    const double *h_J = nullptr;
    // h_J page-locked as a whole and read in place by the kernels (no FP64 slots, no copies)
    bool h_J_direct = false;
    const int64_t *h_pair_ptr = nullptr;
    double *ring_buf = nullptr;
    cudaStream_t ring_stream = nullptr;
    const cudaEvent_t *ring_ev = nullptr;
};

// Pairs held by one slot of the J ring.
inline int64_t ring_slot_pairs(int64_t ring_rows) { return ring_rows / 128 * kForcePairsPerTile; }

// Device bytes of the operand staging buffers for this problem.
size_t tc_workspace_bytes(const Dims &dm, int64_t ring_rows = 0);

// A (QR matrix, single-pass BF16/TF32 products) and Aacc (split-TF32 products,
// FP32-accurate) data rows, Sigma-scaled, into zeroed column-major matrices;
// Wf receives the per-atom force weights of the accurate pass, in.E64 (if set) the
// accurate energy rows in FP64 (double-float epilogue).
cudaError_t tc_assemble(const Dims &dm, const TcInputs &in, TcMode mode, DevBuf &ops, float *A, float *Aacc,
                        float *Wf, cudaStream_t s, Prof *prof);

// Predictions (Eqs. 1, 2) for the mixed precisions: energies from a first
// split-precision GEMM (atoms x sparse points, epilogue eps partials and gradient
// weights), gradients from a second (atoms x descriptor entries over the sparse
// points), forces by contracting the Jacobians with the gradients in FP64.
size_t tc_predict_workspace_bytes(const Dims &dm);
// V (may be null): virials [6 n_cfg] from in.vG and the pseudo-pair arrays (needs F).
cudaError_t tc_predict(const Dims &dm, const TcInputs &in, TcMode mode, DevBuf &ops, DevBuf &work, const double *c,
                       double *E, double *F, cudaStream_t s, Prof *prof, double *V = nullptr);

// QR trailing update on the tensor cores: C[row_off + r, col_off + c] -= sum_a V[r, a] W2[a, c]
// for the column-major FP32 matrix A (leading dimension ld), with V given as
// row-major split-TF32 slices [R x kpad] (row stride v_ld, default kpad) and W2
// transposed as [nt x kpad] slices.
// passes = 3: hi.hi + hi.lo + lo.hi (about FP32 accuracy); passes = 1: hi.hi only
// (plain TF32; the lo slices are not read).
cudaError_t tc_qr_update(float *A, int64_t ld, int64_t row_off, int64_t R, int64_t col_off, int64_t nt,
                         const float *v_hi, const float *v_lo, const float *w_hi, const float *w_lo, int kpad,
                         int passes, int *status, cudaStream_t s, int v_ld = 0);

// QR trailing update, first product on the tensor cores.  tc_qr_pack_v copies the
// reflectors of columns [K0+coff, K0+coff+nbo) of A (rows K0 .. K0+R, unit diagonal,
// zero above it) into vws as n_rows reflector rows (zero past nbo): the TF32 hi slice,
// and with full also
// the lo slice and the unsplit copy, whose address it returns (column-major,
// leading dimension round_up(R, 32)).  tc_qr_y then computes, for a column-major
// FP32 source C, Yp[split][a][c] = sum over the split's rows r of
// V[r, a] C[crow0 + r, c0 + c], rows split into about n_split ranges (the number
// used is returned).  vws: tc_qr_y_workspace_bytes(R) bytes.
size_t tc_qr_y_workspace_bytes(int64_t R);
const float *tc_qr_pack_v(const float *A, int64_t ld, int64_t K0, int nbo, int64_t R, void *vws, int n_rows, bool full,
                          cudaStream_t s, int coff = 0);
cudaError_t tc_qr_y(const float *C, int64_t ldc, int64_t crow0, int64_t R, int64_t c0, int64_t nt, int n_split,
                    void *vws, float *Yp, int *status, cudaStream_t s, int *n_split_used);
// The same product in one plain-TF32 pass: V (the hi slice in vws, v_rows packed
// reflector rows) and C are both fetched by TMA, C straight from the column-major
// matrix (crow0 a multiple of 4, ldc a multiple of 4; the tensor cores use the TF32
// part of each C element).
cudaError_t tc_qr_y_tma(const float *C, int64_t ldc, int64_t crow0, int64_t R, int64_t c0, int64_t nt, int n_split,
                        void *vws, int v_rows, float *Yp, int *status, cudaStream_t s, int *n_split_used);
// Both products of a pair of outer panels in one pass over C: Yp[split][a][c] for the
// 128 reflector rows of v1 (a < 128) and the v2_rows of v2 (a = 128 + ..), each packed
// as by tc_qr_pack_v with the same R.
cudaError_t tc_qr_y2_tma(const float *C, int64_t ldc, int64_t crow0, int64_t R, int64_t c0, int64_t nt, int n_split,
                         const float *v1, const float *v2, int v2_rows, float *Yp, int *status, cudaStream_t s,
                         int *n_split_used);

}  // namespace gap
