// FP64 refinement of the mixed-precision fit (preconditioned CGLS on
// min || b - A_acc x ||, right preconditioner R from the FP32 QR of the
// single-pass matrix; Sec. II, Eq. 7 and the QR solve that follows it):
//
//  * the preconditioner is applied through an explicit inverse W = R^{-1}
//    (FP32, upper triangular) and its transpose, computed once per
//    factorisation from the FP64 inverses of R's 64 x 64 diagonal blocks by
//    recursive doubling: for R = [R11 R12; 0 R22], W12 = -W11 R12 W22, all
//    pairs of one block size in one launch; each application is then one
//    column-dot kernel instead of a sequence of dependent block steps.  A
//    fixed matrix, so CGLS sees one linear operator throughout.
//  * one pass over the rows per iteration: for a block of 32 rows (one
//    contiguous stretch of the row-block layout), t = A u (double-float),
//    |t|^2, and w += A^T t from the same rows while they are still in cache,
//    so A_acc streams from HBM once instead of twice.
//    The CGLS gradient is then updated as s <- s - alpha W^T (A^T A u)
//    (= W^T A^T r after r <- r - alpha A u), exact in exact arithmetic; the
//    starting gradient comes from the true residual of the QR solution.
#include <algorithm>

#include "gap_internal.cuh"
#include "tc_ptx.cuh"

namespace gap {
namespace {

constexpr int TIB = 64;  // block size of the inverse (= the diagonal blocks' size)

// Diagonal TIB x TIB blocks of W from the FP64 diagonal-block inverses.
__global__ void k_trinv_diag(const double *Dinv, int64_t M, float *W, int64_t ldw) {
    const int64_t j0 = (int64_t)blockIdx.x * TIB;
    const int nb = (int)min((int64_t)TIB, M - j0);
    const double *D = Dinv + (int64_t)blockIdx.x * TIB * TIB;  // column-major, upper
    for (int e = threadIdx.x; e < TIB * TIB; e += blockDim.x) {
        const int r = e % TIB, c = e / TIB;
        if (r < nb && c < nb) W[(j0 + r) + (j0 + c) * ldw] = r <= c ? (float)D[r + c * TIB] : 0.f;
    }
}

// One step of the recursive inverse for every pair of diagonal blocks of size bs
// at offsets o = 2 bs p: with R = [R11 R12; 0 R22] and W11 = R11^{-1}, W22 = R22^{-1}
// known, W12 = -W11 (R12 W22).  step 0: T = R12 W22 (into the scratch Tb at W12's
// position); step 1: W12 = -W11 T.  CTA tile 64 x 64 of the bs x n2 product
// (n2 = width of the second block), 256 threads with 4 x 4 each; the k range
// skips the zero triangle of the triangular factor.  Grid (bs/64, ceil(n2/64), pairs).
__global__ void __launch_bounds__(256) k_trinv_step(const float *R, int64_t ldr, int64_t M, int64_t bs, int step,
                                                    float *W, float *Tb, int64_t ldw) {
    __shared__ float As[TIB][TIB + 1];
    __shared__ float Bs[TIB][TIB + 1];
    const int64_t o = (int64_t)blockIdx.z * 2 * bs, o2 = o + bs;
    if (o2 >= M) return;
    const int64_t n2 = min(bs, M - o2);
    const int64_t i0 = (int64_t)blockIdx.x * TIB, j0 = (int64_t)blockIdx.y * TIB;
    if (j0 >= n2) return;
    // A: bs x K, B: K x n2 (column-major views)
    const float *Am = step == 0 ? R + o + o2 * ldr : W + o + o * ldw;
    const int64_t lda = step == 0 ? ldr : ldw;
    const float *Bm = step == 0 ? W + o2 + o2 * ldw : Tb + o + o2 * ldw;
    const int64_t K = step == 0 ? n2 : bs;
    // step 0: W22 upper -> B[k, j] = 0 for k > j; step 1: W11 upper -> A[i, k] = 0 for k < i
    const int64_t kb = step == 0 ? 0 : i0, ke = step == 0 ? min(K, j0 + TIB) : K;
    const int tid = threadIdx.x, tr = tid / 16, tcl = tid % 16;
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
    for (int64_t k0 = kb; k0 < ke; k0 += TIB) {
        for (int e = tid; e < TIB * TIB; e += 256) {
            const int r = e % TIB, c = e / TIB;
            As[r][c] = (k0 + c < ke) ? Am[(i0 + r) + (k0 + c) * lda] : 0.f;
            Bs[r][c] = (k0 + r < ke && j0 + c < n2) ? Bm[(k0 + r) + (j0 + c) * ldw] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < TIB; ++k) {
            float a[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[tr * 4 + u][k];
#pragma unroll
            for (int v = 0; v < 4; ++v) bv[v] = Bs[k][tcl * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }
    float *C = step == 0 ? Tb + o + o2 * ldw : W + o + o2 * ldw;
    const float sg = step == 0 ? 1.f : -1.f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t i = i0 + tr * 4 + u, j = j0 + tcl * 4 + v;
            if (j < n2) C[i + j * ldw] = sg * acc[u][v];
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
// The passes' multiply-accumulate: double-float (DF) or plain FP32 (lo untouched).
template <bool DF>
__device__ __forceinline__ void macc(float &hi, float &lo, float a, float vh, float vl) {
    if (DF)
        dfa(hi, lo, a, vh, vl);
    else
        hi = fmaf(a, vh, hi);
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
//   t = A u for the block's rows (each warp takes 4 columns per float4 load);
//   with rhs: t <- rhs - t (the residual); sq += t^2;
//   with want_w: w_j += sum_r A[r, j] t_r, thread tid owning columns tid + 512 c,
//   c < CPT, its double-float sums held in registers across all of its blocks.
// Outputs per CTA: wpart[2][grid][M] (hi, lo of its share of A^T t), tpart[grid].
template <int CPT, bool DF>
__global__ void __launch_bounds__(CG_THREADS, CPT <= 8 ? 2 : 1) k_cgls_pass(const float *__restrict__ A, int64_t rows, int64_t M,
                                                          int64_t nc, const float *__restrict__ uh_g,
                                                          const float *__restrict__ ul_g,
                                                          const double *__restrict__ rhs, int want_w,
                                                          float *__restrict__ wpart, double *__restrict__ tpart) {
    extern __shared__ float sm[];
    float *s_uh = sm, *s_ul = sm + M;
    // double-buffered by block parity: a warp may start the next block's first phase
    // while others still read this block's t (no barrier at the end of a block)
    __shared__ float red_hb[2][CG_NW][32], red_lb[2][CG_NW][32];
    __shared__ float s_thb[2][CG_RB], s_tlb[2][CG_RB];
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
    int par = 0;
    for (int64_t rb = blockIdx.x; rb * CG_RB < rows; rb += gridDim.x, par ^= 1) {
        float(*red_h)[32] = red_hb[par];
        float(*red_l)[32] = red_lb[par];
        float *s_th = s_thb[par], *s_tl = s_tlb[par];
        const float *blk = A + rb * CG_RB * nc;
        const int64_t i = rb * CG_RB + lane;
        constexpr int UNR = CPT <= 4 ? 4 : (CPT <= 8 ? 3 : 2);  // float4 loads in flight per lane
        // t for the block's 32 rows: lane l reads rows 4 (l % 8) .. +3 of column
        // 4 w + l / 8 (+ 64 k) as one float4, so a warp covers 4 columns (512
        // contiguous bytes) per load; the four column slots are then combined
        float h4[4] = {0.f, 0.f, 0.f, 0.f}, l4[4] = {0.f, 0.f, 0.f, 0.f};
        {
            const int r4 = (lane & 7) * 4;
            constexpr int STEP = 4 * CG_NW;
            int64_t j = 4 * warp + (lane >> 3);
            for (; j + (UNR - 1) * STEP < M; j += UNR * STEP) {
                float4 x[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) x[u] = __ldg(reinterpret_cast<const float4 *>(blk + (j + u * STEP) * CG_RB + r4));
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const float vh = s_uh[j + u * STEP], vl = s_ul[j + u * STEP];
                    macc<DF>(h4[0], l4[0], x[u].x, vh, vl);
                    macc<DF>(h4[1], l4[1], x[u].y, vh, vl);
                    macc<DF>(h4[2], l4[2], x[u].z, vh, vl);
                    macc<DF>(h4[3], l4[3], x[u].w, vh, vl);
                }
            }
            for (; j < M; j += STEP) {
                const float4 x = __ldg(reinterpret_cast<const float4 *>(blk + j * CG_RB + r4));
                const float vh = s_uh[j], vl = s_ul[j];
                macc<DF>(h4[0], l4[0], x.x, vh, vl);
                macc<DF>(h4[1], l4[1], x.y, vh, vl);
                macc<DF>(h4[2], l4[2], x.z, vh, vl);
                macc<DF>(h4[3], l4[3], x.w, vh, vl);
            }
#pragma unroll
            for (int o = 8; o <= 16; o <<= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float oh = __shfl_xor_sync(0xffffffffu, h4[q], o);
                    const float ol = __shfl_xor_sync(0xffffffffu, l4[q], o);
                    dfadd(h4[q], l4[q], oh, ol);
                }
            if (lane < 8)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    red_h[warp][r4 + q] = h4[q];
                    red_l[warp][r4 + q] = l4[q];
                }
        }
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
                            macc<DF>(wh[c], wl[c], x[q].x, s_th[r], s_tl[r]);
                            macc<DF>(wh[c], wl[c], x[q].y, s_th[r + 1], s_tl[r + 1]);
                            macc<DF>(wh[c], wl[c], x[q].z, s_th[r + 2], s_tl[r + 2]);
                            macc<DF>(wh[c], wl[c], x[q].w, s_th[r + 3], s_tl[r + 3]);
                        }
                    }
                }
            }
        }
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

// The same pass over slices of SUB rows of the 32-row blocks, for large M.  A block of 32
// rows spans 32 (M + 1) floats (2 MB at M = 16000): the 152 CTAs' blocks do not stay in L2
// between the two phases, so the second phase would read A from HBM again.  A slice of SUB = 8
// rows is one 32-byte sector per column (512 KB at M = 16000, 78 MB for all CTAs), and its
// second phase reads it from L2.
//   phase 1 (t = A u): lane l reads rows 4 (l % RQ) .. +3 of column CW w + l / RQ (+ CW NW k)
//            as one float4 (RQ = SUB / 4 lanes per column), four row accumulators per lane;
//   phase 2 (w += A^T t): thread tid owns columns tid + 512 c, c < CPT, as in k_cgls_pass.
template <int CPT, bool DF, int SUB>
__global__ void __launch_bounds__(CG_THREADS, 1) k_cgls_pass_sub(const float *__restrict__ A, int64_t rows,
                                                                 int64_t M, int64_t nc, const float *__restrict__ uh_g,
                                                                 const float *__restrict__ ul_g,
                                                                 const double *__restrict__ rhs, int want_w,
                                                                 float *__restrict__ wpart,
                                                                 double *__restrict__ tpart) {
    constexpr int RQ = SUB / 4, CW = 32 / RQ;  // lanes per column, columns per warp load
    extern __shared__ float sm[];
    float *s_uh = sm, *s_ul = sm + M;
    __shared__ float red_hb[2][CG_NW][SUB], red_lb[2][CG_NW][SUB];
    __shared__ float s_thb[2][SUB], s_tlb[2][SUB];
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
    int par = 0;
    const int rq = lane % RQ, r4 = 4 * rq;
    for (int64_t sb = blockIdx.x; sb * SUB < rows; sb += gridDim.x, par ^= 1) {
        float(*red_h)[SUB] = red_hb[par];
        float(*red_l)[SUB] = red_lb[par];
        float *s_th = s_thb[par], *s_tl = s_tlb[par];
        const int64_t r0 = sb * SUB;  // first row of the slice
        const float *blk = A + (r0 / CG_RB) * CG_RB * nc + (r0 % CG_RB);  // column j: blk + 32 j, SUB floats
        float h4[4] = {0.f, 0.f, 0.f, 0.f}, l4[4] = {0.f, 0.f, 0.f, 0.f};
        {
            constexpr int STEP = CW * CG_NW, UNR = 4;
            int64_t j = (int64_t)CW * warp + lane / RQ;
            for (; j + (UNR - 1) * STEP < M; j += UNR * STEP) {
                float4 x[UNR];
#pragma unroll
                for (int u = 0; u < UNR; ++u) x[u] = __ldg(reinterpret_cast<const float4 *>(blk + (j + u * STEP) * CG_RB + r4));
#pragma unroll
                for (int u = 0; u < UNR; ++u) {
                    const float vh = s_uh[j + u * STEP], vl = s_ul[j + u * STEP];
                    macc<DF>(h4[0], l4[0], x[u].x, vh, vl);
                    macc<DF>(h4[1], l4[1], x[u].y, vh, vl);
                    macc<DF>(h4[2], l4[2], x[u].z, vh, vl);
                    macc<DF>(h4[3], l4[3], x[u].w, vh, vl);
                }
            }
            for (; j < M; j += STEP) {
                const float4 x = __ldg(reinterpret_cast<const float4 *>(blk + j * CG_RB + r4));
                const float vh = s_uh[j], vl = s_ul[j];
                macc<DF>(h4[0], l4[0], x.x, vh, vl);
                macc<DF>(h4[1], l4[1], x.y, vh, vl);
                macc<DF>(h4[2], l4[2], x.z, vh, vl);
                macc<DF>(h4[3], l4[3], x.w, vh, vl);
            }
            // the lanes of one row chunk (equal l % RQ) hold different columns: add them up
#pragma unroll
            for (int o = RQ; o < 32; o <<= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float oh = __shfl_xor_sync(0xffffffffu, h4[q], o);
                    const float ol = __shfl_xor_sync(0xffffffffu, l4[q], o);
                    dfadd(h4[q], l4[q], oh, ol);
                }
            if (lane < RQ)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    red_h[warp][r4 + q] = h4[q];
                    red_l[warp][r4 + q] = l4[q];
                }
        }
        __syncthreads();
        if (warp == 0 && lane < SUB) {
            float h = 0.f, l = 0.f;
            for (int w = 0; w < CG_NW; ++w) dfadd(h, l, red_h[w][lane], red_l[w][lane]);
            const int64_t i = r0 + lane;
            double t = (double)h + (double)l;
            if (rhs) t = i < rows ? rhs[i] - t : 0.0;
            if (i >= rows) t = 0.0;
            tsq = fma(t, t, tsq);
            const float th = (float)t;
            s_th[lane] = th;
            s_tl[lane] = (float)(t - (double)th);
        }
        __syncthreads();
        if (want_w) {
            float th[SUB], tl[SUB];
#pragma unroll
            for (int r = 0; r < SUB; ++r) {
                th[r] = s_th[r];
                tl[r] = s_tl[r];
            }
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int64_t j = tid + (int64_t)c * CG_THREADS;
                if (j < M) {
                    const float4 *col = reinterpret_cast<const float4 *>(blk + j * CG_RB);
#pragma unroll
                    for (int q = 0; q < SUB / 4; ++q) {
                        const float4 x = __ldg(col + q);
                        macc<DF>(wh[c], wl[c], x.x, th[4 * q], tl[4 * q]);
                        macc<DF>(wh[c], wl[c], x.y, th[4 * q + 1], tl[4 * q + 1]);
                        macc<DF>(wh[c], wl[c], x.z, th[4 * q + 2], tl[4 * q + 2]);
                        macc<DF>(wh[c], wl[c], x.w, th[4 * q + 3], tl[4 * q + 3]);
                    }
                }
            }
        }
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

// ----------------------------------------------------- TMA-fed CGLS pass --
// The same pass with the data moved by TMA: one producer thread streams every 32-row
// block twice (once per phase) as tiles of 256 columns x 32 rows (32 KB, 128-byte
// swizzle: column c's 16-byte chunk q, rows 4q .. 4q + 3, sits at
// c * 128 + ((q ^ (c % 8)) * 16)) through a ring of TS_STAGES stages; sixteen consumer
// warps compute from shared memory.
//   phase 1 (t = A u): consumer warp g takes columns 16 g .. 16 g + 15 of each tile,
//            lane l chunk l % 8 of column 16 g + 4 j + l / 8 (j < 4) as one float4, four
//            row accumulators per lane, combined over lanes and warps at the block's end;
//   phase 2 (w += A^T t): consumer thread i takes column i % 256 of each tile, rows
//            16 (i / 256) .. + 15 (four float4), its 16 values of t held in registers;
//            w accumulated in shared memory per row half (double-float), the halves
//            added at the end.
// Shared memory: the stages, u as FP32 pairs [M] and w as FP32 pairs [2][M].
constexpr int TS_COLS = 256, TS_STAGES = 3, TS_CONS = 16;  // consumer warps
constexpr uint32_t TS_BYTES = TS_COLS * 32 * 4;
constexpr int TS_THREADS = 32 * (1 + TS_CONS);

__device__ __forceinline__ float4 ts_chunk(const unsigned char *tile, int c, int q) {
    return *reinterpret_cast<const float4 *>(tile + c * 128 + ((q ^ (c & 7)) * 16));
}
__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * TS_CONS) : "memory"); }

template <bool DF>
__global__ void __launch_bounds__(TS_THREADS, 1)
    k_cgls_tma(const __grid_constant__ CUtensorMap tA, int64_t rows, int64_t M, const float *__restrict__ uh_g,
               const float *__restrict__ ul_g, const double *__restrict__ rhs, int want_w, float *__restrict__ wpart,
               double *__restrict__ tpart, int *status) {
    extern __shared__ __align__(1024) unsigned char ts_raw[];
    unsigned char *stg = (unsigned char *)(((uintptr_t)ts_raw + 1023) & ~(uintptr_t)1023);
    float *s_uh = (float *)(stg + TS_STAGES * TS_BYTES), *s_ul = s_uh + M;
    float *s_wh = s_ul + M, *s_wl = s_wh + 2 * M;  // [2][M] each
    __shared__ float red_h[TS_CONS][32], red_l[TS_CONS][32];
    __shared__ float s_th[32], s_tl[32];
    __shared__ uint64_t full[TS_STAGES], empty[TS_STAGES];
    __shared__ int s_fail, s_stop;  // any role failed; the consumers' common decision to stop
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t nc = M + 1;
    const int nck = (int)((M + TS_COLS - 1) / TS_COLS);  // tiles per block and phase
    const int nph = want_w ? 2 : 1;                      // the second phase only forms A^T t
    if (threadIdx.x == 0) {
        for (int s = 0; s < TS_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TS_CONS);
        }
        s_fail = 0;
        s_stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int64_t j = threadIdx.x; j < M; j += blockDim.x) {
        s_uh[j] = uh_g[j];
        s_ul[j] = ul_g[j];
        s_wh[j] = s_wh[M + j] = 0.f;
        s_wl[j] = s_wl[M + j] = 0.f;
    }
    __syncthreads();
    const int64_t nblk = (rows + 31) / 32;
    double tsq = 0.0;
    if (warp == 0) {
        // ------------------------------------------------------ producer --
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int64_t rb = blockIdx.x; rb < nblk && ok; rb += gridDim.x)
                for (int ph = 0; ph < nph && ok; ++ph)
                    for (int k = 0; k < nck; ++k, ++it) {
                        const uint32_t s = it % TS_STAGES, par = (it / TS_STAGES) & 1;
                        if (!mbar_wait(&empty[s], par ^ 1, status)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(&full[s], TS_BYTES);
                        tma_load_2d(stg + s * TS_BYTES, &tA, &full[s], 0, (int)(rb * nc + (int64_t)k * TS_COLS));
                    }
            if (!ok) atomicExch(&s_fail, 1);
            // drain: every load issued must land before the CTA may exit
            if (it > 0) {
                const uint32_t last = it - 1;
                for (uint32_t q = (last >= (uint32_t)TS_STAGES ? last - TS_STAGES + 1 : 0); q <= last; ++q)
                    mbar_wait(&full[q % TS_STAGES], (q / TS_STAGES) & 1, status);
            }
        }
    } else {
        // ----------------------------------------------------- consumers --
        // Every consumer warp passes the same barriers in the same order; a wait that
        // times out only records the failure, and all of them stop together at the
        // next decision point (s_stop, written before a barrier, read after it).
        const int g = warp - 1, ci = threadIdx.x - 32, Mi = (int)M;
        const int q1 = lane & 7, c1 = 16 * g + (lane >> 3);  // phase 1: chunk, first column
        const int c2 = ci & (TS_COLS - 1), hh = ci / TS_COLS;  // phase 2: column, row half
        float *wh2 = s_wh + hh * M, *wl2 = s_wl + hh * M;
        // byte offsets of this thread's 16-byte chunks within a tile (the same in every tile)
        int off1[4], off2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c1 + 4 * j;
            off1[j] = c * 128 + ((q1 ^ (c & 7)) * 16);
            off2[j] = c2 * 128 + (((4 * hh + j) ^ (c2 & 7)) * 16);
        }
        uint32_t st = 0, par = 0;  // ring stage and its phase bit
        auto advance = [&]() {
            if (++st == TS_STAGES) {
                st = 0;
                par ^= 1u;
            }
        };
        for (int64_t rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
            const int64_t i = rb * 32 + lane;
            // the block's right-hand side, fetched before its tiles are consumed
            const double rv = (g == 0 && rhs != nullptr && i < rows) ? rhs[i] : 0.0;
            float h4[4] = {0.f, 0.f, 0.f, 0.f}, l4[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < nck; ++k, advance()) {
                if (!mbar_wait(&full[st], par, status)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                const unsigned char *tile = stg + st * TS_BYTES;
                const int cb = k * TS_COLS;
                const float *uh = s_uh + cb, *ul = s_ul + cb;
                if (cb + TS_COLS <= Mi) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float4 x = *reinterpret_cast<const float4 *>(tile + off1[j]);
                        const float vh = uh[c1 + 4 * j], vl = ul[c1 + 4 * j];
                        macc<DF>(h4[0], l4[0], x.x, vh, vl);
                        macc<DF>(h4[1], l4[1], x.y, vh, vl);
                        macc<DF>(h4[2], l4[2], x.z, vh, vl);
                        macc<DF>(h4[3], l4[3], x.w, vh, vl);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (cb + c1 + 4 * j < Mi) {
                            const float4 x = *reinterpret_cast<const float4 *>(tile + off1[j]);
                            const float vh = uh[c1 + 4 * j], vl = ul[c1 + 4 * j];
                            macc<DF>(h4[0], l4[0], x.x, vh, vl);
                            macc<DF>(h4[1], l4[1], x.y, vh, vl);
                            macc<DF>(h4[2], l4[2], x.z, vh, vl);
                            macc<DF>(h4[3], l4[3], x.w, vh, vl);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[st]);
            }
#pragma unroll
            for (int o = 8; o <= 16; o <<= 1)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float oh = __shfl_xor_sync(0xffffffffu, h4[q], o);
                    const float ol = __shfl_xor_sync(0xffffffffu, l4[q], o);
                    dfadd(h4[q], l4[q], oh, ol);
                }
            if (lane < 8)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    red_h[g][4 * q1 + q] = h4[q];
                    red_l[g][4 * q1 + q] = l4[q];
                }
            cons_sync();
            if (g == 0) {
                float th = 0.f, tl = 0.f;
                for (int w = 0; w < TS_CONS; ++w) dfadd(th, tl, red_h[w][lane], red_l[w][lane]);
                double t = (double)th + (double)tl;
                if (rhs) t = rv - t;
                if (i >= rows) t = 0.0;
                tsq = fma(t, t, tsq);
                const float fh = (float)t;
                s_th[lane] = fh;
                s_tl[lane] = (float)(t - (double)fh);
                if (lane == 0) s_stop = *(volatile int *)&s_fail;
            }
            cons_sync();
            if (s_stop) break;
            if (nph > 1) {
                float th[16], tl[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    th[r] = s_th[16 * hh + r];
                    tl[r] = s_tl[16 * hh + r];
                }
                for (int k = 0; k < nck; ++k, advance()) {
                    if (!mbar_wait(&full[st], par, status)) {
                        atomicExch(&s_fail, 1);
                        break;
                    }
                    const int col = k * TS_COLS + c2;
                    if (col < Mi) {
                        const unsigned char *tile = stg + st * TS_BYTES;
                        float wh = wh2[col], wl = wl2[col];
                        float4 x[4];
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) x[qq] = *reinterpret_cast<const float4 *>(tile + off2[qq]);
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            macc<DF>(wh, wl, x[qq].x, th[4 * qq], tl[4 * qq]);
                            macc<DF>(wh, wl, x[qq].y, th[4 * qq + 1], tl[4 * qq + 1]);
                            macc<DF>(wh, wl, x[qq].z, th[4 * qq + 2], tl[4 * qq + 2]);
                            macc<DF>(wh, wl, x[qq].w, th[4 * qq + 3], tl[4 * qq + 3]);
                        }
                        wh2[col] = wh;
                        wl2[col] = wl;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[st]);
                }
                if (g == 0 && lane == 0) s_stop = *(volatile int *)&s_fail;
                cons_sync();  // s_th is rewritten for the next block; s_stop is common
                if (s_stop) break;
            }
        }
    }
    __syncthreads();
    const int64_t G = gridDim.x;
    if (want_w)
        for (int64_t j = threadIdx.x; j < M; j += blockDim.x) {
            float h = s_wh[j], l = s_wl[j];
            dfadd(h, l, s_wh[M + j], s_wl[M + j]);
            wpart[(int64_t)blockIdx.x * M + j] = h;
            wpart[(G + blockIdx.x) * M + j] = l;
        }
    if (warp == 1) {
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
    k_trinv_diag<<<(unsigned)nblk, 256, 0, s>>>(Dinv, M, W, ldw);
    // W12 = -W11 R12 W22 for doubling block sizes (Wt is the scratch until the end)
    for (int64_t bs = TIB; bs < M; bs *= 2) {
        const unsigned pairs = (unsigned)ceil_div(M, 2 * bs);
        const dim3 grid((unsigned)(bs / TIB), (unsigned)ceil_div(bs, TIB), pairs);
        k_trinv_step<<<grid, 256, 0, s>>>(R, ldr, M, bs, 0, W, Wt, ldw);
        k_trinv_step<<<grid, 256, 0, s>>>(R, ldr, M, bs, 1, W, Wt, ldw);
    }
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
template <int CPT, bool DF>
cudaError_t launch_cgls_p(const float *A, int64_t rows, int64_t M, const float *uh, const float *ul, const double *rhs,
                          bool want_w, float *wpart, double *tpart, int G, cudaStream_t s) {
    const size_t smem = 2 * sizeof(float) * (size_t)M;
    // the limit is raised once to the largest launch (fits in flight on several host
    // threads must not lower it under one another)
    static const cudaError_t e_attr = cudaFuncSetAttribute(k_cgls_pass<CPT, DF>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)(2 * sizeof(float) * 32 * CG_THREADS));
    if (e_attr != cudaSuccess) return e_attr;
    k_cgls_pass<CPT, DF><<<G, CG_THREADS, smem, s>>>(A, rows, M, M + 1, uh, ul, rhs, want_w ? 1 : 0, wpart, tpart);
    return cudaGetLastError();
}
template <int CPT, bool DF>
cudaError_t launch_cgls_sub(const float *A, int64_t rows, int64_t M, const float *uh, const float *ul,
                            const double *rhs, bool want_w, float *wpart, double *tpart, int G, cudaStream_t s) {
    constexpr int SUB = 8;
    const size_t smem = 2 * sizeof(float) * (size_t)M;
    static const cudaError_t e_attr = cudaFuncSetAttribute(k_cgls_pass_sub<CPT, DF, SUB>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)(2 * sizeof(float) * 32 * CG_THREADS));
    if (e_attr != cudaSuccess) return e_attr;
    k_cgls_pass_sub<CPT, DF, SUB><<<G, CG_THREADS, smem, s>>>(A, rows, M, M + 1, uh, ul, rhs, want_w ? 1 : 0, wpart,
                                                              tpart);
    return cudaGetLastError();
}
template <int CPT>
cudaError_t launch_cgls(const float *A, int64_t rows, int64_t M, const float *uh, const float *ul, const double *rhs,
                        bool want_w, float *wpart, double *tpart, int G, bool df, cudaStream_t s) {
    if (CPT >= 16)  // M > 4096: a CTA's 32-row blocks would not stay in L2 between the phases
        return df ? launch_cgls_sub<CPT, true>(A, rows, M, uh, ul, rhs, want_w, wpart, tpart, G, s)
                  : launch_cgls_sub<CPT, false>(A, rows, M, uh, ul, rhs, want_w, wpart, tpart, G, s);
    return df ? launch_cgls_p<CPT, true>(A, rows, M, uh, ul, rhs, want_w, wpart, tpart, G, s)
              : launch_cgls_p<CPT, false>(A, rows, M, uh, ul, rhs, want_w, wpart, tpart, G, s);
}
}  // namespace

namespace {
constexpr int64_t TS_MAX_M = 5120;  // u and two halves of w as FP32 pairs next to the stages in shared memory

template <bool DF>
cudaError_t launch_cgls_tma(const float *A, int64_t rows, int64_t M, const float *uh, const float *ul,
                            const double *rhs, bool want_w, float *wpart, double *tpart, int G, int *status,
                            cudaStream_t s) {
    // the row-block layout as a 2-D tensor: 32 rows (contiguous) x (blocks x (M + 1)) columns
    auto fn = encode_fn();
    if (!fn) return cudaErrorInvalidValue;
    CUtensorMap tA;
    cuuint64_t dims[2] = {32u, (cuuint64_t)(((rows + 31) / 32) * (M + 1))};
    cuuint64_t strides[1] = {128u};
    cuuint32_t box[2] = {32u, (cuuint32_t)TS_COLS};
    cuuint32_t estr[2] = {1u, 1u};
    if (fn(&tA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)A, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = 1024 + (size_t)TS_STAGES * TS_BYTES + 24 * (size_t)M;
    // raised once to the largest launch (see launch_cgls_p)
    static const cudaError_t e_attr = cudaFuncSetAttribute(
        k_cgls_tma<DF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)(1024 + (size_t)TS_STAGES * TS_BYTES + 24 * (size_t)TS_MAX_M));
    if (e_attr != cudaSuccess) return e_attr;
    k_cgls_tma<DF><<<G, TS_THREADS, smem, s>>>(tA, rows, M, uh, ul, rhs, want_w ? 1 : 0, wpart, tpart, status);
    return cudaGetLastError();
}
}  // namespace

cudaError_t cgls_pass(const float *A, int64_t rows, int64_t M, const double *u, const double *rhs, double *w,
                      double *sq, void *ws, bool df, int *status, cudaStream_t s) {
    if (!cgls_fused_fits(M)) return cudaErrorInvalidValue;
    float *uh = (float *)ws, *ul = uh + M, *wpart = ul + M;
    if (M <= TS_MAX_M && status && ((rows + 31) / 32) * (M + 1) < ((int64_t)1 << 31)) {
        // one CTA per SM, data moved by TMA
        int dev = 0, n_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        const int G = std::max(n_sm, 1);
        double *tpart = (double *)(((uintptr_t)(wpart + 2 * (size_t)G * M) + 255) & ~(uintptr_t)255);
        k_split_f64<<<(unsigned)ceil_div(M, 256), 256, 0, s>>>(u, M, uh, ul);
        cudaError_t e = df ? launch_cgls_tma<true>(A, rows, M, uh, ul, rhs, w != nullptr, wpart, tpart, G, status, s)
                           : launch_cgls_tma<false>(A, rows, M, uh, ul, rhs, w != nullptr, wpart, tpart, G, status, s);
        if (e != cudaSuccess) return e;
        k_cgls_reduce<<<(unsigned)ceil_div(M, 256), 256, 0, s>>>(wpart, tpart, G, M, w, sq);
        return cudaGetLastError();
    }
    const int G = cgls_grid();
    double *tpart = (double *)(((uintptr_t)(wpart + 2 * (size_t)G * M) + 255) & ~(uintptr_t)255);
    k_split_f64<<<(unsigned)ceil_div(M, 256), 256, 0, s>>>(u, M, uh, ul);
    const int cpt = (int)ceil_div(M, CG_THREADS);
    const bool ww = w != nullptr;
    cudaError_t e = cpt <= 1   ? launch_cgls<1>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, df, s)
                    : cpt <= 2 ? launch_cgls<2>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, df, s)
                    : cpt <= 4 ? launch_cgls<4>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, df, s)
                    : cpt <= 8 ? launch_cgls<8>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, df, s)
                    : cpt <= 16 ? launch_cgls<16>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, df, s)
                                : launch_cgls<32>(A, rows, M, uh, ul, rhs, ww, wpart, tpart, G, df, s);
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

namespace {
// Entry (i, s) of the head rows: the FP64 energy rows below n_e, the row-block FP32
// matrix after them.
__device__ __forceinline__ double head_entry(const double *E64, int64_t n_e, const float *A, int64_t M, int64_t i,
                                             int64_t s) {
    return i < n_e ? E64[i * M + s] : (double)A[acc_index(i, s, M + 1)];
}

// t_i = rhs_i - A_i . u (or A_i . u without rhs) for the head row i = blockIdx.x, in
// FP64; the block's partial sums reduced in a fixed order.
__global__ void __launch_bounds__(256) k_cgls_head_rows(const double *__restrict__ E64, int64_t n_e,
                                                        const float *__restrict__ A, int64_t M,
                                                        const double *__restrict__ u, const double *__restrict__ rhs,
                                                        double *__restrict__ t) {
    __shared__ double red[256];
    const int64_t i = blockIdx.x;
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < M; k += 256) acc += head_entry(E64, n_e, A, M, i, k) * u[k];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) t[i] = rhs ? rhs[i] - red[0] : red[0];
}

constexpr int kHeadSlab = 64;  // head rows per partial sum of the column pass

// Partial column sums over slabs of kHeadSlab head rows: part[g * M + s] = sum over the
// rows i of slab g of A[i, s] t_i (one thread per column, blockIdx.y the slab).
__global__ void __launch_bounds__(256) k_cgls_head_cols(const double *__restrict__ E64, int64_t n_e,
                                                        const float *__restrict__ A, int64_t rh, int64_t M,
                                                        const double *__restrict__ t, double *__restrict__ part) {
    const int64_t s = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (s >= M) return;
    const int64_t i0 = (int64_t)blockIdx.y * kHeadSlab, i1 = min(rh, i0 + kHeadSlab);
    double v = 0.0;
    for (int64_t i = i0; i < i1; ++i) v += head_entry(E64, n_e, A, M, i, s) * t[i];
    part[(int64_t)blockIdx.y * M + s] = v;
}

// w_s (+)= the slabs' partial sums in slab order; block 0 also forms sq (+)= |t|^2 in a
// fixed order.  acc = 0 overwrites instead of adding.
__global__ void __launch_bounds__(256) k_cgls_head_sum(const double *__restrict__ part, int G, int64_t rh, int64_t M,
                                                       const double *__restrict__ t, double *__restrict__ w,
                                                       double *__restrict__ sq, int acc) {
    const int64_t s = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (w && s < M) {
        double v = 0.0;
        for (int g = 0; g < G; ++g) v += part[(int64_t)g * M + s];
        w[s] = acc ? w[s] + v : v;
    }
    if (blockIdx.x == 0) {
        __shared__ double red[256];
        double q = 0.0;
        for (int64_t i = threadIdx.x; i < rh; i += 256) q += t[i] * t[i];
        red[threadIdx.x] = q;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) *sq = acc ? *sq + red[0] : red[0];
    }
}
}  // namespace

size_t cgls_head_bytes(int64_t rh, int64_t M) {
    return sizeof(double) * (size_t)(std::max<int64_t>(1, rh) + ceil_div(std::max<int64_t>(1, rh), kHeadSlab) * M);
}

// ws: cgls_head_bytes(rh, M) bytes (t, then the column pass's partial sums).
cudaError_t cgls_head(const double *E64, int64_t n_e, const float *A, int64_t rh, int64_t M, const double *u,
                      const double *rhs, double *w, double *sq, double *ws, bool accumulate, cudaStream_t s) {
    if (rh <= 0) return cudaSuccess;
    double *t = ws, *part = ws + rh;
    const int G = (int)ceil_div(rh, kHeadSlab);
    const unsigned cb = (unsigned)std::max<int64_t>(1, ceil_div(M, 256));
    k_cgls_head_rows<<<(unsigned)rh, 256, 0, s>>>(E64, n_e, A, M, u, rhs, t);
    if (w) k_cgls_head_cols<<<dim3(cb, (unsigned)G), 256, 0, s>>>(E64, n_e, A, rh, M, t, part);
    k_cgls_head_sum<<<cb, 256, 0, s>>>(part, G, rh, M, t, w, sq, accumulate ? 1 : 0);
    return cudaGetLastError();
}

namespace {
// Predictions from design rows (Eq. 7: a data row is its target's model value over sigma).
// FP64 rows (the energy rows E64 [n x M]): one warp per row, FP64 dot with c.
__global__ void k_rows_dot_f64(const double *__restrict__ R, int64_t n, int64_t M, const double *__restrict__ c,
                               const double *__restrict__ sigma, double *__restrict__ out) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (i >= n) return;
    const double *r = R + i * M;
    double s = 0.0;
    for (int64_t j = lane; j < M; j += 32) s = fma(r[j], c[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = sigma[i] * s;
}

// Rows [row0, row0 + nrows) of the FP32 row-block matrix A (M + 1 columns): one warp per
// 32-row block, lane = row (32 consecutive floats per column), the dot product with c
// (as FP32 pairs) in double-float.  out[i - row0] = sigma[i] * (A[i, :] . c).
__global__ void k_acc_rows_dot(const float *__restrict__ A, int64_t M, int64_t row0, int64_t nrows,
                               const float *__restrict__ ch, const float *__restrict__ cl,
                               const double *__restrict__ sigma, double *__restrict__ out) {
    const int64_t b = row0 / ACC_RB + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    const int64_t i = b * ACC_RB + lane;
    if (b * ACC_RB >= row0 + nrows) return;
    const float *blk = A + b * ACC_RB * (M + 1) + lane;
    float h = 0.f, l = 0.f;
    int64_t j = 0;
    constexpr int U = 8;
    for (; j + U <= M; j += U) {
        float x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = __ldg(blk + (j + u) * ACC_RB);
#pragma unroll
        for (int u = 0; u < U; ++u) dfa(h, l, x[u], __ldg(ch + j + u), __ldg(cl + j + u));
    }
    for (; j < M; ++j) dfa(h, l, __ldg(blk + j * ACC_RB), __ldg(ch + j), __ldg(cl + j));
    if (i >= row0 && i < row0 + nrows) out[i - row0] = sigma[i] * ((double)h + (double)l);
}
}  // namespace

cudaError_t predict_from_rows(const double *E64, int64_t n_e, const float *A, int64_t M, int64_t row0, int64_t nrows,
                              const double *sigma, const double *c, float *ws, double *E, double *out, cudaStream_t s) {
    if (E && n_e > 0)
        k_rows_dot_f64<<<(unsigned)ceil_div(n_e * 32, 256), 256, 0, s>>>(E64, n_e, M, c, sigma, E);
    if (out && nrows > 0) {
        float *ch = ws, *cl = ws + M;
        k_split_f64<<<(unsigned)ceil_div(M, 256), 256, 0, s>>>(c, M, ch, cl);
        const int64_t nb = (row0 + nrows - 1) / ACC_RB - row0 / ACC_RB + 1;
        k_acc_rows_dot<<<(unsigned)ceil_div(nb * 32, 256), 256, 0, s>>>(A, M, row0, nrows, ch, cl, sigma, out);
    }
    return cudaGetLastError();
}

cudaError_t acc_to_colmajor(const float *A, int64_t ld, int64_t M, float *out, cudaStream_t s) {
    k_acc_to_colmajor<<<(unsigned)ceil_div(ld * (M + 1), 256), 256, 0, s>>>(A, ld, M + 1, out);
    return cudaGetLastError();
}

}  // namespace gap
