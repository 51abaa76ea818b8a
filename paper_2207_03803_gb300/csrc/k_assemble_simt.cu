// SIMT assembly of the design-matrix data rows Sigma^{-1/2} K_NM (Sec. II,
// Eqs. 6 and 7) for the FP64 precision (and an FP32 variant).
//
// Energy rows: K_{A,s} = sum_{i in A} delta^2 (x_i . x_s)^zeta  (Eq. 6 with the
// dot-product covariance), divided by sigma_A.
// Force rows:  K_{(a,alpha),s} = -sum_{p in pairs(a)} W_{i(p),s} (J_p[alpha] . x_s),
// W_{i,s} = delta^2 zeta (x_i . x_s)^(zeta-1), divided by sigma_{(a,alpha)}.
// The energy kernel also stores W (per atom, per sparse point) for the force
// kernel, so the force GEMM contracts only the Jacobian rows.
//
// Both kernels are register-tiled GEMMs with the power, species mask and
// Sigma scaling in the epilogue, followed by a segmented sum over the atoms of
// a configuration (energy) or the pairs of a target atom (force) done in shared
// memory in index order.  A segment cut by a tile boundary gets one atomic add
// from each of its (at most two, for configurations of <= 128 atoms and atoms
// of <= 64 pairs) tiles; two-term sums are order-independent, so results are
// bit-reproducible.  The design matrix is column-major with leading dimension
// ld and is zeroed before these kernels run.
#include "gap_internal.cuh"

namespace gap {
namespace {

template <class T>
__device__ __forceinline__ T ipow(T g, int z) {
    T p = T(1);
    for (int k = 0; k < z; ++k) p *= g;
    return p;
}

__device__ __forceinline__ void atomic_add(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add(float *p, float v) { atomicAdd(p, v); }

constexpr int EBM = 128, EBN = 64, EBK = 16;  // energy tile: atoms x sparse points
constexpr int FBP = 64, FBN = 64, FBK = 16;   // force tile: pairs x sparse points

// Grid: (ceil(n_atoms/128), ceil(M/64)); 256 threads; dynamic smem = 128*65*sizeof(T).
template <class T>
__global__ void __launch_bounds__(256) k_energy_simt(Dims dm, const double *__restrict__ X,
                                                     const double *__restrict__ Xs, const int32_t *__restrict__ atom_sp,
                                                     const int32_t *__restrict__ sparse_sp,
                                                     const int64_t *__restrict__ cfg_ptr,
                                                     const int64_t *__restrict__ atom_cfg,
                                                     const double *__restrict__ sigma, T *__restrict__ A,
                                                     T *__restrict__ Wf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T As[EBK][EBM];
    __shared__ T Bs[EBK][EBN];
    T *Ks = reinterpret_cast<T *>(smem_raw);  // [EBM][EBN+1]
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t a0 = (int64_t)blockIdx.x * EBM, s0 = (int64_t)blockIdx.y * EBN;
    const int64_t d = dm.d, M = dm.M, na = dm.n_atoms;
    T acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int64_t k0 = 0; k0 < d; k0 += EBK) {
        for (int e = tid; e < EBM * EBK; e += 256) {
            int r = e / EBK, kk = e % EBK;
            int64_t a = a0 + r, k = k0 + kk;
            As[kk][r] = (a < na && k < d) ? T(X[a * d + k]) : T(0);
        }
        for (int e = tid; e < EBN * EBK; e += 256) {
            int r = e / EBK, kk = e % EBK;
            int64_t s = s0 + r, k = k0 + kk;
            Bs[kk][r] = (s < M && k < d) ? T(Xs[s * d + k]) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < EBK; ++kk) {
            T a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][ty * 8 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
    const T d2 = T(dm.delta * dm.delta), zf = T(dm.zeta);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int r = ty * 8 + i;
        int64_t a = a0 + r;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int c = tx * 4 + j;
            int64_t s = s0 + c;
            T kv = T(0);
            if (a < na && s < M) {
                bool same = !dm.species || atom_sp[a] == sparse_sp[s];
                T g = acc[i][j];
                T gz1 = ipow(g, dm.zeta - 1);
                Wf[a * M + s] = same ? d2 * zf * gz1 : T(0);
                kv = same ? d2 * gz1 * g : T(0);
            }
            Ks[r * (EBN + 1) + c] = kv;
        }
    }
    __syncthreads();
    // segmented sum over the atoms of each configuration present in this tile
    const int64_t a_last = min(a0 + EBM, na) - 1;
    if (a0 > a_last) return;
    const int64_t c_first = atom_cfg[a0], c_last = atom_cfg[a_last];
    const int n_seg = (int)(c_last - c_first + 1);
    for (int task = tid; task < n_seg * EBN; task += 256) {
        int seg = task / EBN, c = task % EBN;
        int64_t s = s0 + c;
        if (s >= M) continue;
        int64_t cfg = c_first + seg;
        int64_t lo = max(cfg_ptr[cfg], a0), hi = min(cfg_ptr[cfg + 1], a0 + EBM);
        T sum = T(0);
        for (int64_t a = lo; a < hi; ++a) sum += Ks[(a - a0) * (EBN + 1) + c];
        T v = sum / T(sigma[cfg]);
        bool partial = cfg_ptr[cfg] < a0 || cfg_ptr[cfg + 1] > a0 + EBM;
        T *dst = A + cfg + s * dm.ld;
        if (partial)
            atomic_add(dst, v);
        else
            *dst = v;
    }
}

// Grid: (ceil(n_pairs/64), ceil(M/64)); 256 threads; dynamic smem = 64*65*sizeof(T).
template <class T>
__global__ void __launch_bounds__(256) k_force_simt(Dims dm, const double *__restrict__ J,
                                                    const double *__restrict__ Xs, const int64_t *__restrict__ pair_ptr,
                                                    const int64_t *__restrict__ pair_src,
                                                    const int64_t *__restrict__ pair_tgt,
                                                    const double *__restrict__ sigma, const T *__restrict__ Wf,
                                                    T *__restrict__ A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T Js[FBK][3][FBP];
    __shared__ T Bs[FBK][FBN];
    T *Vs = reinterpret_cast<T *>(smem_raw);  // [FBP][FBN+1]
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t p0 = (int64_t)blockIdx.x * FBP, s0 = (int64_t)blockIdx.y * FBN;
    const int64_t d = dm.d, M = dm.M, np = dm.n_pairs;
    T acc[3][4][4];
#pragma unroll
    for (int al = 0; al < 3; ++al)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[al][i][j] = T(0);
    for (int64_t k0 = 0; k0 < d; k0 += FBK) {
        for (int e = tid; e < 3 * FBP * FBK; e += 256) {
            int row = e / FBK, kk = e % FBK;  // row = pair_local*3 + alpha
            int pl = row / 3, al = row % 3;
            int64_t p = p0 + pl, k = k0 + kk;
            Js[kk][al][pl] = (p < np && k < d) ? T(J[(p * 3 + al) * d + k]) : T(0);
        }
        for (int e = tid; e < FBN * FBK; e += 256) {
            int r = e / FBK, kk = e % FBK;
            int64_t s = s0 + r, k = k0 + kk;
            Bs[kk][r] = (s < M && k < d) ? T(Xs[s * d + k]) : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < FBK; ++kk) {
            T b[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int al = 0; al < 3; ++al) {
                T a[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = Js[kk][al][ty * 4 + i];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[al][i][j] += a[i] * b[j];
            }
        }
        __syncthreads();
    }
    // weights of the 4 pairs x 4 columns this thread holds
    T w[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t p = p0 + ty * 4 + i;
        int64_t src = p < np ? pair_src[p] : 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t s = s0 + tx * 4 + j;
            w[i][j] = (p < np && s < M) ? Wf[src * M + s] : T(0);
        }
    }
    const int64_t p_last = min(p0 + FBP, np) - 1;
    const int64_t t_first = pair_tgt[p0], t_last = pair_tgt[p_last];
    const int n_seg = (int)(t_last - t_first + 1);
    for (int al = 0; al < 3; ++al) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) Vs[(ty * 4 + i) * (FBN + 1) + tx * 4 + j] = -w[i][j] * acc[al][i][j];
        __syncthreads();
        for (int task = tid; task < n_seg * FBN; task += 256) {
            int seg = task / FBN, c = task % FBN;
            int64_t s = s0 + c;
            if (s >= M) continue;
            int64_t a = t_first + seg;
            int64_t lo = max(pair_ptr[a], p0), hi = min(pair_ptr[a + 1], p0 + FBP);
            if (lo >= hi) continue;  // atom without pairs in this tile
            T sum = T(0);
            for (int64_t p = lo; p < hi; ++p) sum += Vs[(p - p0) * (FBN + 1) + c];
            int64_t row = dm.n_cfg + 3 * a + al;
            T v = sum / T(sigma[row]);
            bool partial = pair_ptr[a] < p0 || pair_ptr[a + 1] > p0 + FBP;
            T *dst = A + row + s * dm.ld;
            if (partial)
                atomic_add(dst, v);
            else
                *dst = v;
        }
        __syncthreads();
    }
}

template <class T>
__global__ void k_rhs(Dims dm, const double *__restrict__ y, const double *__restrict__ sigma, double *__restrict__ b,
                      T *__restrict__ A, int blocked) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= dm.rows) return;
    double v = r < dm.N ? y[r] / sigma[r] : 0.0;
    b[r] = v;
    A[blocked ? acc_index(r, dm.M, dm.M + 1) : r + dm.M * dm.ld] = T(v);
}

// out[k] = segment id of element k for ptr[0..n_seg] (element k in [ptr[j], ptr[j+1]) -> j)
__global__ void k_segment_ids(const int64_t *__restrict__ ptr, int64_t n_seg, int64_t *__restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_seg) return;
    for (int64_t k = ptr[j]; k < ptr[j + 1]; ++k) out[k] = j;
}

__device__ void set_status(DevStatus *st, int code, int64_t idx) {
    if (atomicCAS(&st->code, 0, code) == 0) st->index = idx;
}

// Checks run on the device before any kernel indexes with these arrays.
__global__ void k_validate(Dims dm, const int64_t *__restrict__ cfg_ptr, const int64_t *__restrict__ pair_ptr,
                           const int64_t *__restrict__ pair_src, const int64_t *__restrict__ atom_cfg,
                           const double *__restrict__ sigma, const int32_t *__restrict__ atom_sp,
                           const int32_t *__restrict__ sparse_sp, DevStatus *st) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = t; j < dm.n_cfg; j += stride)
        if (cfg_ptr[j + 1] < cfg_ptr[j]) set_status(st, GAP_ERR_INVALID, j);
    if (t == 0 && (cfg_ptr[0] != 0 || cfg_ptr[dm.n_cfg] != dm.n_atoms)) set_status(st, GAP_ERR_INVALID, -1);
    if (sigma)
        for (int64_t r = t; r < dm.N; r += stride)
            if (!(sigma[r] > 0.0)) set_status(st, GAP_ERR_INVALID, r);
    if (dm.forces) {
        if (t == 0 && (pair_ptr[0] != 0 || pair_ptr[dm.n_atoms] != dm.n_pairs)) set_status(st, GAP_ERR_INVALID, -2);
        for (int64_t a = t; a < dm.n_atoms; a += stride)
            if (pair_ptr[a + 1] < pair_ptr[a]) set_status(st, GAP_ERR_INVALID, a);
    }
}

// second pass (needs monotone pointers and atom_cfg): pair sources in range and in
// the target's configuration; species labels non-negative
__global__ void k_validate_pairs(Dims dm, const int64_t *__restrict__ pair_ptr, const int64_t *__restrict__ pair_src,
                                 const int64_t *__restrict__ atom_cfg, const int32_t *__restrict__ atom_sp,
                                 const int32_t *__restrict__ sparse_sp, DevStatus *st) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (dm.forces) {
        for (int64_t a = t; a < dm.n_atoms; a += stride) {
            for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p) {
                int64_t i = pair_src[p];
                if (i < 0 || i >= dm.n_atoms || atom_cfg[i] != atom_cfg[a]) set_status(st, GAP_ERR_INVALID, p);
            }
        }
    }
    if (dm.species) {
        for (int64_t a = t; a < dm.n_atoms; a += stride)
            if (atom_sp[a] < 0) set_status(st, GAP_ERR_INVALID, a);
        for (int64_t s = t; s < dm.M; s += stride)
            if (sparse_sp[s] < 0) set_status(st, GAP_ERR_INVALID, s);
    }
}

}  // namespace

cudaError_t launch_segment_ids(const int64_t *ptr, int64_t n_seg, int64_t *out_ids, cudaStream_t s) {
    if (n_seg <= 0) return cudaSuccess;
    k_segment_ids<<<(unsigned)ceil_div(n_seg, 256), 256, 0, s>>>(ptr, n_seg, out_ids);
    return cudaGetLastError();
}

cudaError_t launch_validate(const Dims &dm, const int64_t *cfg_ptr, const int64_t *pair_ptr, const int64_t *pair_src,
                            const int64_t *atom_cfg, const double *sigma, const int32_t *atom_sp,
                            const int32_t *sparse_sp, DevStatus *st, cudaStream_t s) {
    if (atom_cfg == nullptr) {
        k_validate<<<304, 256, 0, s>>>(dm, cfg_ptr, pair_ptr, pair_src, atom_cfg, sigma, atom_sp, sparse_sp, st);
    } else {
        k_validate_pairs<<<304, 256, 0, s>>>(dm, pair_ptr, pair_src, atom_cfg, atom_sp, sparse_sp, st);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_energy_simt(const Dims &dm, const double *X, const double *Xs, const int32_t *atom_sp,
                               const int32_t *sparse_sp, const int64_t *cfg_ptr, const int64_t *atom_cfg,
                               const double *sigma, T *A, T *Wf, cudaStream_t s) {
    if (dm.n_atoms == 0 || dm.M == 0) return cudaSuccess;
    size_t smem = (size_t)EBM * (EBN + 1) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_energy_simt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)ceil_div(dm.n_atoms, EBM), (unsigned)ceil_div(dm.M, EBN));
    k_energy_simt<T><<<grid, 256, smem, s>>>(dm, X, Xs, atom_sp, sparse_sp, cfg_ptr, atom_cfg, sigma, A, Wf);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_force_simt(const Dims &dm, const double *J, const double *Xs, const int64_t *pair_ptr,
                              const int64_t *pair_src, const int64_t *pair_tgt, const double *sigma, const T *Wf,
                              T *A, cudaStream_t s) {
    if (!dm.forces || dm.n_pairs == 0 || dm.M == 0) return cudaSuccess;
    size_t smem = (size_t)FBP * (FBN + 1) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_force_simt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)ceil_div(dm.n_pairs, FBP), (unsigned)ceil_div(dm.M, FBN));
    k_force_simt<T><<<grid, 256, smem, s>>>(dm, J, Xs, pair_ptr, pair_src, pair_tgt, sigma, Wf, A);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_rhs(const Dims &dm, const double *y, const double *sigma, double *b64, T *A, cudaStream_t s,
                       bool blocked) {
    k_rhs<T><<<(unsigned)ceil_div(dm.rows, 256), 256, 0, s>>>(dm, y, sigma, b64, A, blocked ? 1 : 0);
    return cudaGetLastError();
}

template cudaError_t launch_energy_simt<double>(const Dims &, const double *, const double *, const int32_t *,
                                                const int32_t *, const int64_t *, const int64_t *, const double *,
                                                double *, double *, cudaStream_t);
template cudaError_t launch_energy_simt<float>(const Dims &, const double *, const double *, const int32_t *,
                                               const int32_t *, const int64_t *, const int64_t *, const double *,
                                               float *, float *, cudaStream_t);
template cudaError_t launch_force_simt<double>(const Dims &, const double *, const double *, const int64_t *,
                                               const int64_t *, const int64_t *, const double *, const double *,
                                               double *, cudaStream_t);
template cudaError_t launch_force_simt<float>(const Dims &, const double *, const double *, const int64_t *,
                                              const int64_t *, const int64_t *, const double *, const float *,
                                              float *, cudaStream_t);
template cudaError_t launch_rhs<double>(const Dims &, const double *, const double *, double *, double *,
                                        cudaStream_t, bool);
template cudaError_t launch_rhs<float>(const Dims &, const double *, const double *, double *, float *,
                                       cudaStream_t, bool);

}  // namespace gap
