// Predictions of a fitted model (Sec. II, Eqs. 1 and 2), FP64 SIMT:
//   eps(x_i) = sum_s c_s delta^2 (x_i . x_s)^zeta,     E_A = sum_{i in A} eps(x_i),
//   grad eps(x_i) = sum_s c_s delta^2 zeta (x_i . x_s)^(zeta-1) x_s,
//   F_{a,alpha} = -sum_{p in pairs(a)} J_p[alpha] . grad eps(x_{i(p)}).
// Forces go through the per-atom gradient (an n_atoms x M x d GEMM) instead of
// per-pair design rows, which needs n_pairs/n_atoms times fewer products.
#include "gap_internal.cuh"

namespace gap {
namespace {

__device__ __forceinline__ double ipow(double g, int z) {
    double p = 1.0;
    for (int k = 0; k < z; ++k) p *= g;
    return p;
}

// Atoms [a_begin, a_begin + n) : eps[a] and wm[(a - a_begin) * M + s] = c_s delta^2 zeta u^(zeta-1).
// Grid: ceil(n / 128) blocks of 256 threads; each block sweeps every sparse tile.
__global__ void __launch_bounds__(256) k_pred_atoms(Dims dm, const double *__restrict__ X,
                                                    const double *__restrict__ Xs, const int32_t *__restrict__ atom_sp,
                                                    const int32_t *__restrict__ sparse_sp,
                                                    const double *__restrict__ c, int64_t a_begin, int64_t n,
                                                    double *__restrict__ eps, double *__restrict__ wm, int want_w) {
    __shared__ double As[16][128];
    __shared__ double Bs[16][64];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t a0 = a_begin + (int64_t)blockIdx.x * 128, a_end = a_begin + n;
    const int64_t d = dm.d, M = dm.M;
    const double d2 = dm.delta * dm.delta, zf = (double)dm.zeta;
    double e_acc[8] = {};
    for (int64_t s0 = 0; s0 < M; s0 += 64) {
        double acc[8][4] = {};
        for (int64_t k0 = 0; k0 < d; k0 += 16) {
            for (int e = tid; e < 128 * 16; e += 256) {
                int r = e / 16, kk = e % 16;
                int64_t a = a0 + r, k = k0 + kk;
                As[kk][r] = (a < a_end && k < d) ? X[a * d + k] : 0.0;
            }
            for (int e = tid; e < 64 * 16; e += 256) {
                int r = e / 16, kk = e % 16;
                int64_t s = s0 + r, k = k0 + kk;
                Bs[kk][r] = (s < M && k < d) ? Xs[s * d + k] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                double av[8], bv[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) av[i] = As[kk][ty * 8 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int64_t a = a0 + ty * 8 + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int64_t s = s0 + tx * 4 + j;
                if (a < a_end && s < M) {
                    bool same = !dm.species || atom_sp[a] == sparse_sp[s];
                    double u = acc[i][j];
                    double uz1 = ipow(u, dm.zeta - 1);
                    e_acc[i] += same ? c[s] * d2 * uz1 * u : 0.0;
                    if (want_w) wm[(a - a_begin) * M + s] = same ? c[s] * d2 * zf * uz1 : 0.0;
                }
            }
        }
    }
    // reduce the 16 column groups sharing each row (lanes tx = 0..15 of a half warp)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        double v = e_acc[i];
        for (int o = 8; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, 16);
        int64_t a = a0 + ty * 8 + i;
        if (tx == 0 && a < a_end) eps[a] = v;
    }
}

// grad[a, k] = sum_s wm[a - a_begin, s] Xs[s, k]; tile 128 atoms x 64 descriptor entries.
__global__ void __launch_bounds__(256) k_pred_grad(Dims dm, const double *__restrict__ wm,
                                                   const double *__restrict__ Xs, int64_t a_begin, int64_t n,
                                                   double *__restrict__ grad) {
    __shared__ double Ws[16][128];
    __shared__ double Bs[16][64];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t r0 = (int64_t)blockIdx.x * 128, k0 = (int64_t)blockIdx.y * 64;
    const int64_t d = dm.d, M = dm.M;
    double acc[8][4] = {};
    for (int64_t s0 = 0; s0 < M; s0 += 16) {
        for (int e = tid; e < 128 * 16; e += 256) {
            int r = e / 16, ss = e % 16;
            int64_t row = r0 + r, s = s0 + ss;
            Ws[ss][r] = (row < n && s < M) ? wm[row * M + s] : 0.0;
        }
        for (int e = tid; e < 64 * 16; e += 256) {
            int kk = e % 64, ss = e / 64;
            int64_t s = s0 + ss, k = k0 + kk;
            Bs[ss][kk] = (s < M && k < d) ? Xs[s * d + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int ss = 0; ss < 16; ++ss) {
            double av[8], bv[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) av[i] = Ws[ss][ty * 8 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[ss][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int64_t row = r0 + ty * 8 + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t k = k0 + tx * 4 + j;
            if (row < n && k < d) grad[(a_begin + row) * d + k] = acc[i][j];
        }
    }
}

// One warp per target atom: F[3a+alpha] = -sum_p J_p[alpha] . grad[src(p)].
__global__ void k_pred_force(Dims dm, const int64_t *__restrict__ pair_ptr, const int64_t *__restrict__ pair_src,
                             const double *__restrict__ J, const double *__restrict__ grad, double *__restrict__ F) {
    int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int lane = threadIdx.x % 32;
    if (a >= dm.n_atoms) return;
    const int64_t d = dm.d;
    double f[3] = {0.0, 0.0, 0.0};
    for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p) {
        const double *g = grad + pair_src[p] * d;
        for (int al = 0; al < 3; ++al) {
            const double *j = J + (p * 3 + al) * d;
            double s = 0.0;
            for (int64_t k = lane; k < d; k += 32) s += j[k] * g[k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            f[al] += s;
        }
    }
    if (lane == 0)
        for (int al = 0; al < 3; ++al) F[3 * a + al] = -f[al];
}

__global__ void k_pred_energy(int64_t n_cfg, const int64_t *__restrict__ cfg_ptr, const double *__restrict__ eps,
                              double *__restrict__ E) {
    int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (A >= n_cfg) return;
    double e = 0.0;
    for (int64_t i = cfg_ptr[A]; i < cfg_ptr[A + 1]; ++i) e += eps[i];
    E[A] = e;
}

}  // namespace

cudaError_t predict_simt(const Dims &dm, const double *X, const double *Xs, const int32_t *atom_sp,
                         const int32_t *sparse_sp, const int64_t *cfg_ptr, const int64_t *pair_ptr,
                         const int64_t *pair_src, const double *J, const double *c, double *E, double *F,
                         double *eps_work, double *grad_work, double *wmat_work, int64_t atom_chunk, cudaStream_t s) {
    const bool want_f = F != nullptr && pair_ptr != nullptr && dm.n_pairs > 0;
    for (int64_t a = 0; a < dm.n_atoms; a += atom_chunk) {
        int64_t n = min(atom_chunk, dm.n_atoms - a);
        k_pred_atoms<<<(unsigned)ceil_div(n, 128), 256, 0, s>>>(dm, X, Xs, atom_sp, sparse_sp, c, a, n, eps_work,
                                                                 wmat_work, want_f ? 1 : 0);
        if (want_f) {
            dim3 g((unsigned)ceil_div(n, 128), (unsigned)ceil_div(dm.d, 64));
            k_pred_grad<<<g, 256, 0, s>>>(dm, wmat_work, Xs, a, n, grad_work);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (dm.n_cfg > 0) k_pred_energy<<<(unsigned)ceil_div(dm.n_cfg, 256), 256, 0, s>>>(dm.n_cfg, cfg_ptr, eps_work, E);
    if (F != nullptr && dm.n_atoms > 0) {
        if (want_f) {
            k_pred_force<<<(unsigned)ceil_div(dm.n_atoms * 32, 256), 256, 0, s>>>(dm, pair_ptr, pair_src, J,
                                                                                 grad_work, F);
        } else {
            cudaMemsetAsync(F, 0, sizeof(double) * 3 * dm.n_atoms, s);
        }
    }
    return cudaGetLastError();
}

}  // namespace gap

namespace gap {
cudaError_t predict_virial_simt(const Dims &vdm, const int64_t *vp_ptr, const int64_t *vp_src, const double *G,
                                const double *grad, double *V, cudaStream_t s) {
    if (vdm.n_atoms <= 0) return cudaSuccess;
    k_pred_force<<<(unsigned)ceil_div(vdm.n_atoms * 32, 256), 256, 0, s>>>(vdm, vp_ptr, vp_src, G, grad, V);
    return cudaGetLastError();
}
}  // namespace gap
