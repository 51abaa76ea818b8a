// Tensor-core (tcgen05) assembly of the design matrix for the mixed precisions.
#pragma once

#include "gap_internal.cuh"

namespace gap {

enum class TcMode { BF16, TF32 };

struct TcInputs {
    const double *X, *Xs, *J;
    const int64_t *cfg_ptr, *atom_cfg, *pair_ptr, *pair_src, *pair_tgt;
    const double *sigma;
    const int32_t *atom_sp, *sparse_sp;
    int *status;  // device status word (GAP_ERR_TIMEOUT on a bounded-wait timeout)
};

// Device bytes of the operand staging buffers for this problem.
size_t tc_workspace_bytes(const Dims &dm);

// A (QR matrix, single-pass BF16/TF32 products) and Aacc (split-TF32 products,
// FP32-accurate) data rows, Sigma-scaled, into zeroed column-major matrices;
// Wf receives the per-atom force weights of the accurate pass.
cudaError_t tc_assemble(const Dims &dm, const TcInputs &in, TcMode mode, DevBuf &ops, float *A, float *Aacc,
                        float *Wf, cudaStream_t s, Prof *prof);

// Predictions (Eqs. 1, 2) for the mixed precisions: energies from a first
// split-precision GEMM (atoms x sparse points, epilogue eps partials and gradient
// weights), gradients from a second (atoms x descriptor entries over the sparse
// points), forces by contracting the Jacobians with the gradients in FP64.
size_t tc_predict_workspace_bytes(const Dims &dm);
cudaError_t tc_predict(const Dims &dm, const TcInputs &in, TcMode mode, DevBuf &ops, DevBuf &work, const double *c,
                       double *E, double *F, cudaStream_t s, Prof *prof);

}  // namespace gap
