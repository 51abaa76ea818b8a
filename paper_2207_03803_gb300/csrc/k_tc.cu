// Mixed-precision assembly entry (placeholder routing to the FP32 SIMT kernels).
#include "tc_gemm.cuh"

namespace gap {

size_t tc_workspace_bytes(const Dims &dm) {
    (void)dm;
    return 0;
}

cudaError_t tc_assemble(const Dims &dm, const TcInputs &in, TcMode mode, DevBuf &ops, float *A, float *Aacc,
                        float *Wf, cudaStream_t s) {
    (void)mode;
    (void)ops;
    cudaError_t e = launch_energy_simt<float>(dm, in.X, in.Xs, in.atom_sp, in.sparse_sp, in.cfg_ptr, in.atom_cfg,
                                              in.sigma, Aacc, Wf, s);
    if (e != cudaSuccess) return e;
    e = launch_force_simt<float>(dm, in.J, in.Xs, in.pair_ptr, in.pair_src, in.pair_tgt, in.sigma, Wf, Aacc, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(A, Aacc, sizeof(float) * (size_t)dm.ld * (size_t)dm.M, cudaMemcpyDeviceToDevice, s);
}

}  // namespace gap
