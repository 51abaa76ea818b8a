// FP64 refinement of the mixed-precision fit (preconditioned CGLS on
// min || b - A_acc x ||, right preconditioner R from the FP32 QR of the
// single-pass matrix; Sec. II, Eq. 7 and the QR solve that follows it):
//
//  * the preconditioner is applied through an explicit inverse W = R^{-1}
//    (FP32, upper triangular) and its transpose, computed once per
//    factorisation by block columns of 64 from the FP64 inverses of R's
//    diagonal blocks: W[:, j] = [ -(W[0:j0, 0:j0] R[0:j0, j]) D_j ; D_j ];
//    each application is then one column-dot kernel instead of a sequence
//    of dependent block steps.  A fixed matrix, so CGLS sees one linear
//    operator throughout.
//  * one pass over the rows per iteration: for a block of 32 rows (one
//    contiguous stretch of the row-block layout), t = A u (double-float),
//    |t|^2, and w += A^T t from the same rows while they are still in cache,
//    so A_acc streams from HBM once instead of twice.
//    The CGLS gradient is then updated as s <- s - alpha W^T (A^T A u)
//    (= W^T A^T r after r <- r - alpha A u), exact in exact arithmetic; the
//    starting gradient comes from the true residual of the QR solution.
#include <algorithm>

#include "gap_internal.cuh"

namespace gap {
namespace {

constexpr int TIB = 64;  // block size of the inverse (= the diagonal blocks' size)

// Block column jb of W = R^{-1}: blockIdx.x = row tile (it <= jb).
// it == jb: the diagonal block (FP64 inverse -> FP32); it < jb:
// W[it, jb] = -(sum over k-tiles from it to jb-1 of W[it, k] R[k, jb]) D_jb.
// W is zero below the diagonal (the caller clears it first).
__global__ void __launch_bounds__(256) k_trinv_col(const float *R, int64_t ldr, int64_t M, const double *Dinv, int jb,
                                                   float *W, int64_t ldw) {
    __shared__ float As[TIB][TIB + 1];
    __shared__ float Bs[TIB][TIB + 1];
    const int64_t i0 = (int64_t)blockIdx.x * TIB, j0 = (int64_t)jb * TIB;
    const int nbj = (int)min((int64_t)TIB, M - j0);
    const double *D = Dinv + (int64_t)jb * TIB * TIB;  // column-major TIB x TIB, upper
    const int tid = threadIdx.x, tr = tid / 16, tcl = tid % 16;
    if (i0 == j0) {
        for (int e = tid; e < TIB * TIB; e += 256) {
            const int r = e % TIB, c = e / TIB;
            if (r < nbj && c < nbj) W[(j0 + r) + (j0 + c) * ldw] = r <= c ? (float)D[r + c * TIB] : 0.f;
        }
        return;
    }
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    for (int64_t k0 = i0; k0 < j0; k0 += TIB) {
        for (int e = tid; e < TIB * TIB; e += 256) {
            const int r = e % TIB, c = e / TIB;
            As[r][c] = W[(i0 + r) + (k0 + c) * ldw];
            Bs[r][c] = c < nbj ? R[(k0 + r) + (j0 + c) * ldr] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < TIB; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[tr * 4 + u][k];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = Bs[k][tcl * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
    // X = -Y D_jb
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) As[tr * 4 + u][tcl * 4 + v] = acc[u][v];
    for (int e = tid; e < TIB * TIB; e += 256) {
        const int r = e % TIB, c = e / TIB;
        Bs[r][c] = (r < nbj && c < nbj) ? (float)D[r + c * TIB] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int col = tcl * 4 + v;
            float x = 0.f;
            for (int k = 0; k <= col; ++k) x = fmaf(As[tr * 4 + u][k], Bs[k][col], x);
            if (col < nbj) W[(i0 + tr * 4 + u) + (j0 + col) * ldw] = -x;
        }
}

// Wt = W^T for the leading M x M block (32 x 32 shared-memory tiles).
__global__ void k_transpose_sq(const float *W, int64_t ldw, int64_t M, float *Wt) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
        const int64_t r = r0 + threadIdx.x, c = c0 + yy;
        tile[yy][threadIdx.x] = (r < M && c < M) ? W[r + c * ldw] : 0.f;
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
        const int64_t r = c0 + threadIdx.x, c = r0 + yy;  // Wt[r, c] = W[c, r]
        if (r < M && c < M) Wt[r + c * ldw] = tile[threadIdx.x][yy];
    }
}

// ------------------------------------------------------------ CGLS pass --
constexpr int CG_RB = 32;        // rows per block (one 128-byte segment per column)
constexpr int CG_THREADS = 512;  // 16 warps
constexpr int CG_NW = CG_THREADS / 32;

// Double-float accumulate hi + lo += a * (vh + vl): the product's rounding error
// by FMA, the sum's by TwoSum (Knuth).
__device__ __forceinline__ void dfa(float &hi, float &lo, float a, float vh, float vl) {
    const float p = a * vh;
    const float e = fmaf(a, vh, -p) + a * vl;
    const float s = hi + p;
    const float bp = s - hi;
    lo += ((hi - (s - bp)) + (p - bp)) + e;
    hi = s;
}
// hi + lo += (bh + bl), both double-float.
__device__ __forceinline__ void dfadd(float &hi, float &lo, float bh, float bl) {
    const float s = hi + bh;
    const float bp = s - hi;
    lo += ((hi - (s - bp)) + (bh - bp)) + bl;
    hi = s;
}

__global__ void k_split_f64(const double *v, int64_t n, float *vh, float *vl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h = (float)v[i];
    vh[i] = h;
    vl[i] = (float)(v[i] - (double)h);
}

// Persistent over blocks of ACC_RB = 32 rows of the row-block layout (a block is
// one contiguous stretch: 32 floats per column).  Shared memory: uh, ul [M].
//   t = A u for the block's rows (warp w: columns w, w + 16, ...; lane = row);
//   with rhs: t <- rhs - t (the residual); sq += t^2;
//   with want_w: w_j += sum_r A[r, j] t_r, thread tid owning columns tid + 512 c,
//   c < CPT, its double-float sums held in registers across all of its blocks.
// Outputs per CTA: wpart[2][grid][M] (hi, lo of its share of A^T t), tpart[grid].
template <int CPT>
__global__ void __launch_bounds__(CG_THREADS, CPT <= 8 ? 2 : 1) k_cgls_pass(const float *__restrict__ A, int64_t rows, int64_t M,
                                                          int64_t nc, const float *__restrict__ uh_g,
                                                          const float *__restrict__ ul_g,
                                                          const double *__restrict__ rhs, int want_w,
                                                          float *__restrict__ wpart, double *__restrict__ tpart) {
    extern __shared__ float sm[];
    float *s_uh = sm, *s_ul = sm + M;
    __shared__ float red_h[CG_NW][32], red_l[CG_NW][32];
    __shared__ float s_th[CG_RB], s_tl[CG_RB];
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    for (int64_t j = tid; j < M; j += CG_THREADS) {
        s_uh[j] = uh_g[j];
        s_ul[j] = ul_g[j];
    }
    float wh[CPT], wl[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) wh[c] = wl[c] = 0.f;
    __syncthreads();
    double tsq = 0.0;
    for (int64_t rb = blockIdx.x; rb * CG_RB < rows; rb += gridDim.x) {
        const float *blk = A + rb * CG_RB * nc;
        const int64_t i = rb * CG_RB + lane;
        float hi = 0.f, lo = 0.f;
        {
            const float *a = blk + lane;
            int64_t j = warp;
            constexpr int UN = CPT <= 4 ? 8 : 4;  // loads in flight per warp (register budget)
            for (; j + (UN - 1) * CG_NW < M; j += UN * CG_NW) {
                float x[UN];
#pragma unroll
                for (int u = 0; u < UN; ++u) x[u] = __ldg(a + (j + u * CG_NW) * CG_RB);
#pragma unroll
                for (int u = 0; u < UN; ++u) dfa(hi, lo, x[u], s_uh[j + u * CG_NW], s_ul[j + u * CG_NW]);
            }
            for (; j < M; j += CG_NW) dfa(hi, lo, __ldg(a + j * CG_RB), s_uh[j], s_ul[j]);
        }
        red_h[warp][lane] = hi;
        red_l[warp][lane] = lo;
        __syncthreads();
        if (warp == 0) {
            float h = 0.f, l = 0.f;
            for (int w = 0; w < CG_NW; ++w) dfadd(h, l, red_h[w][lane], red_l[w][lane]);
            double t = (double)h + (double)l;
            if (rhs) t = i < rows ? rhs[i] - t : 0.0;
            tsq = fma(t, t, tsq);
            const float th = (float)t;
            s_th[lane] = th;
            s_tl[lane] = (float)(t - (double)th);
        }
        __syncthreads();
        if (want_w) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int64_t j = tid + (int64_t)c * CG_THREADS;
                if (j < M) {
                    const float4 *col = reinterpret_cast<const float4 *>(blk + j * CG_RB);
                    constexpr int NQ = CPT <= 4 ? CG_RB / 4 : CG_RB / 8;  // float4 loads in flight
#pragma unroll
                    for (int h0 = 0; h0 < CG_RB / 4; h0 += NQ) {
                        float4 x[NQ];
#pragma unroll
                        for (int q = 0; q < NQ; ++q) x[q] = __ldg(col + h0 + q);
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            const int r = 4 * (h0 + q);
                            dfa(wh[c], wl[c], x[q].x, s_th[r], s_tl[r]);
                            dfa(wh[c], wl[c], x[q].y, s_th[r + 1], s_tl[r + 1]);
                            dfa(wh[c], wl[c], x[q].z, s_th[r + 2], s_tl[r + 2]);
                            dfa(wh[c], wl[c], x[q].w, s_th[r + 3], s_tl[r + 3]);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    const int64_t G = gridDim.x;
    if (want_w) {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int64_t j = tid + (int64_t)c * CG_THREADS;
            if (j < M) {
                wpart[(int64_t)blockIdx.x * M + j] = wh[c];
                wpart[(G + blockIdx.x) * M + j] = wl[c];
            }
        }
    }
    if (warp == 0) {
        for (int o = 16; o > 0; o >>= 1) tsq += __shfl_down_sync(0xffffffffu, tsq, o);
        if (lane == 0) tpart[blockIdx.x] = tsq;
    }
}

// w[j] = sum over CTAs (fixed order) of the double-float partials (skipped when w is
// null: the pass then wrote no partials); tsq = sum of tpart.
__global__ void k_cgls_reduce(const float *wpart, const double *tpart, int G, int64_t M, double *w, double *tsq) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w != nullptr && j < M) {
        float h = 0.f, l = 0.f;
        for (int b = 0; b < G; ++b) dfadd(h, l, wpart[(int64_t)b * M + j], wpart[((int64_t)G + b) * M + j]);
        w[j] = (double)h + (double)l;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < G; ++b) s += tpart[b];
        *tsq = s;
    }
}

int cgls_grid() {
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    return 2 * std::max(n_sm, 1);
}

}  // namespace

cudaError_t triangular_inverse(const float *R, int64_t ldr, int64_t M, const double *Dinv, float *W, float *Wt,
                               int64_t ldw, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(W, 0, sizeof(float) * (size_t)ldw * (size_t)M, s);
    if (e != cudaSuccess) return e;
    const int nblk = (int)ceil_div(M, TIB);
    for (int jb = 0; jb < nblk; ++jb) k_trinv_col<<<(unsigned)(jb + 1), 256, 0, s>>>(R, ldr, M, Dinv, jb, W, ldw);
    const unsigned nt = (unsigned)ceil_div(M, 32);
    k_transpose_sq<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(W, ldw, M, Wt);
    return cudaGetLastError();
}

size_t cgls_workspace_bytes(int64_t M) {
    const int G = cgls_grid();
    return sizeof(float) * (size_t)M * (2 + 2 * (size_t)G) + sizeof(double) * (size_t)G + 1024;
}

bool cgls_fused_fits(int64_t M) { return M <= 32 * CG_THREADS; }

namespace {
template <int CPT>
cudaError_t launch_cgls(const float *A, int64_t rows, int64_t M, const float *uh, const float *ul, const double *rhs,
                        bool want_w, float *wpart, double *tpart, int G, cudaStream_t s) {
    const size_t smem = 2 * sizeof(float) * (size_t)M;
    cudaError_t e = cudaFuncSetAttribute(k_cgls_pass<CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cgls_pass<CPT><<<G, CG_THREADS, smem, s>>>(A, rows, M, M + 1, uh, ul, rhs, want_w ? 1 : 0, wpart, tpart);
    return cudaGetLastError();
}
}  // namespace

cudaError_t cgls_pass(const float *A, int64_t rows, int64_t M, const double *u, const double *rhs, double *w,
                      double *sq, void *ws, cudaStream_t s) {
    if (!cgls_fused_fits(M)) return cudaErrorInvalidValue;
    const int G = cgls_grid();
    float *uh = (float *)ws, *ul = uh + M, *wpart = ul + M;
    double *tpart = (double *)(((uintptr_t)(wpart + 2 * (size_t)G * M) + 255) & ~(uintptr_t)255);
    k_split_f64<<<(unsigned)ceil_div(M, 256), 256, 0, s>>>(u, M, uh, ul);
    const int cpt = (int)ceil_div(M, CG_THREADS);
    const bool ww = w != nullptr;
    cudaError_t e = cpt <= 1   ? launch_cgls<1>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, s)
                    : cpt <= 2 ? launch_cgls<2>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, s)
                    : cpt <= 4 ? launch_cgls<4>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, s)
                    : cpt <= 8 ? launch_cgls<8>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, s)
                    : cpt <= 16 ? launch_cgls<16>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, s)
                                : launch_cgls<32>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, s);
    if (e != cudaSuccess) return e;
    k_cgls_reduce<<<(unsigned)ceil_div(M, 256), 256, 0, s>>>(wpart, tpart, G, M, w, sq);
    return cudaGetLastError();
}

namespace {
__global__ void k_read_rows_acc(const float *A, int64_t M, int64_t row0, int64_t nrows, double *dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nrows * M) return;
    const int64_t r = e / M, c = e % M;
    dst[e] = (double)A[acc_index(row0 + r, c, M + 1)];
}
// column-major copy [ld x nc] of the row-block layout (rows past `rows` are zero in both)
__global__ void k_acc_to_colmajor(const float *A, int64_t ld, int64_t nc, float *out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ld * nc) return;
    const int64_t r = e % ld, c = e / ld;
    out[e] = A[acc_index(r, c, nc)];
}
}  // namespace

cudaError_t read_rows_acc(const float *A, int64_t M, int64_t row0, int64_t nrows, double *dst, cudaStream_t s) {
    if (nrows * M == 0) return cudaSuccess;
    k_read_rows_acc<<<(unsigned)ceil_div(nrows * M, 256), 256, 0, s>>>(A, M, row0, nrows, dst);
    return cudaGetLastError();
}

cudaError_t acc_to_colmajor(const float *A, int64_t ld, int64_t M, float *out, cudaStream_t s) {
    k_acc_to_colmajor<<<(unsigned)ceil_div(ld * (M + 1), 256), 256, 0, s>>>(A, ld, M + 1, out);
    return cudaGetLastError();
}

}  // namespace gap
