// Dense linear algebra of the fit (Sec. II, Eqs. 7-12), SIMT kernels for FP64
// and FP32 storage:
//   K_MM + jitter, blocked right-looking Cholesky K_MM = L L^T (U = L^T),
//   stacking U under the data rows, blocked Householder QR of the column-major
//   design matrix (the role pdgeqrf plays in Sec. III.B) with the right-hand
//   side carried as an extra column (Q^T b, the pdormqr step), back
//   substitution (pdtrtrs), and the GEMVs and triangular solves of the FP64
//   refinement.
//
// Householder convention (LAPACK geqrf): for x = A[j:, j], alpha = x_0,
// beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta, v = x / (alpha - beta)
// with v_0 = 1 implicit; a zero sub-column gives tau = 0.  A panel of nb
// columns is factored one column per launch: each launch finishes the
// reductions of its column (every block sums the per-block partials in the
// same fixed order), applies the reflector to its rows of the panel and
// produces the partial sums the next column needs.  The block of nb
// reflectors is then applied to the trailing columns in compact WY form,
// C <- C - V T^T (V^T C), as two GEMM-shaped kernels with a fixed-order
// reduction of V^T C over row blocks.
#include <math.h>

#include <algorithm>
#include <climits>

#include "gap_internal.cuh"
#include "tc_gemm.cuh"

namespace gap {
namespace {

template <class T>
__device__ __forceinline__ T ipow(T g, int z) {
    T p = T(1);
    for (int k = 0; k < z; ++k) p *= g;
    return p;
}

__device__ __forceinline__ bool status_bad(const DevStatus *st) { return st && *(volatile const int *)&st->code != 0; }

__device__ void set_status(DevStatus *st, int code, int64_t idx) {
    if (atomicCAS(&st->code, 0, code) == 0) st->index = idx;
}

// 1/sqrt(d) for d > 0 in FP64 from an FP32 seed and two Newton steps
// y <- y (3 - d y^2) / 2 (each step squares the relative error: 2^-23 -> 2^-46 -> below
// one FP64 ulp), a handful of FP64 multiplies instead of the long FP64 square-root and
// division sequences, which are slow on this GPU's FP64 units.
__device__ __forceinline__ double rsqrt_f64(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);  // outside the FP32 seed's range
    double y = (double)rsqrtf((float)d);
    y = y * (1.5 - 0.5 * d * y * y);
    y = y * (1.5 - 0.5 * d * y * y);
    return y;
}

// ------------------------------------------------------------------ K_MM --
// K[s + t*M] = delta^2 (x_s . x_t)^zeta (0 across species) + jitter [s == t].
// Products and sums are formed in the same order for (s,t) and (t,s), so K is
// exactly symmetric.
// A 64 x 64 tile of K_MM whose sparse points share no species is zero (the sub-GAPs of
// different species do not covary): true when species are given and no row's species equals
// a column's.  Every thread of the block calls it (a barrier).
__device__ __forceinline__ bool kmm_tile_cross(const Dims &dm, const int32_t *sp, int64_t s0, int64_t t0) {
    if (!dm.species) return false;
    __shared__ int rs[64], cs[64];
    const int tid = threadIdx.x;
    if (tid < 64) rs[tid] = s0 + tid < dm.M ? sp[s0 + tid] : INT_MIN;
    else if (tid < 128) cs[tid - 64] = t0 + tid - 64 < dm.M ? sp[t0 + tid - 64] : INT_MIN + 1;
    __syncthreads();
    int hit = 0;
    for (int e = tid; e < 64 * 64; e += blockDim.x) hit |= rs[e / 64] == cs[e % 64];
    return __syncthreads_or(hit) == 0;
}

__global__ void __launch_bounds__(256) k_kmm(Dims dm, const double *__restrict__ Xs,
                                             const int32_t *__restrict__ sp, double *__restrict__ K) {
    __shared__ double As[16][64];
    __shared__ double Bs[16][64];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t s0 = (int64_t)blockIdx.x * 64, t0 = (int64_t)blockIdx.y * 64, M = dm.M, d = dm.d;
    if (kmm_tile_cross(dm, sp, s0, t0)) {  // no dot products: the tile is zero (never on the diagonal)
        for (int e = tid; e < 64 * 64; e += 256) {
            const int64_t s = s0 + e % 64, t = t0 + e / 64;
            if (s < M && t < M) K[s + t * M] = 0.0;
        }
        return;
    }
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < d; k0 += 16) {
        for (int e = tid; e < 64 * 16; e += 256) {
            int r = e / 16, kk = e % 16;
            int64_t k = k0 + kk;
            As[kk][r] = (s0 + r < M && k < d) ? Xs[(s0 + r) * d + k] : 0.0;
            Bs[kk][r] = (t0 + r < M && k < d) ? Xs[(t0 + r) * d + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += As[kk][tx * 4 + i] * Bs[kk][ty * 4 + j];
        __syncthreads();
    }
    const double d2 = dm.delta * dm.delta;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int64_t t = t0 + ty * 4 + j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int64_t s = s0 + tx * 4 + i;
            if (s < M && t < M) {
                bool same = !dm.species || sp[s] == sp[t];
                double v = same ? d2 * ipow(acc[i][j], dm.zeta) : 0.0;
                if (s == t) v += dm.jitter;
                K[s + t * M] = v;
            }
        }
    }
}

// The same K_MM with the dot products in double-float on the FP32 units (the mixed
// precisions): each FP64 entry of X_s arrives split into an FP32 pair (about 48 bits,
// split once before the launch), each product of pairs is formed with its FMA rounding
// error, and the sums are kept as FP32 pairs by TwoSum (relative accuracy about 2^-44,
// far below the FP32 rounding the U rows get in the mixed matrices).  The power,
// species mask and jitter are FP64.  Only the tiles of the lower triangle (s >= t) are
// formed: the double-float factor reads nothing else.
__device__ __forceinline__ void df_fma_acc(float &hi, float &lo, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p) + (ah * bl + al * bh);
    const float s = hi + p;
    const float bp = s - hi;
    lo += ((hi - (s - bp)) + (p - bp)) + e;
    hi = s;
}

__global__ void __launch_bounds__(256) k_kmm_df(Dims dm, const float *__restrict__ Xh, const float *__restrict__ Xl,
                                                const int32_t *__restrict__ sp, double *__restrict__ K) {
    if (blockIdx.y > blockIdx.x) return;  // the factor reads the lower triangle only
    __shared__ float Ah[16][64], Al[16][64], Bh[16][64], Bl[16][64];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int64_t s0 = (int64_t)blockIdx.x * 64, t0 = (int64_t)blockIdx.y * 64, M = dm.M, d = dm.d;
    if (kmm_tile_cross(dm, sp, s0, t0)) {  // no dot products: the tile is zero (never on the diagonal)
        for (int e = tid; e < 64 * 64; e += 256) {
            const int64_t s = s0 + e % 64, t = t0 + e / 64;
            if (s < M && t < M) K[s + t * M] = 0.0;
        }
        return;
    }
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
    for (int64_t k0 = 0; k0 < d; k0 += 16) {
        for (int e = tid; e < 64 * 16; e += 256) {
            const int r = e / 16, kk = e % 16;
            const int64_t k = k0 + kk;
            const bool oa = s0 + r < M && k < d, ob = t0 + r < M && k < d;
            Ah[kk][r] = oa ? Xh[(s0 + r) * d + k] : 0.f;
            Al[kk][r] = oa ? Xl[(s0 + r) * d + k] : 0.f;
            Bh[kk][r] = ob ? Xh[(t0 + r) * d + k] : 0.f;
            Bl[kk][r] = ob ? Xl[(t0 + r) * d + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    df_fma_acc(hi[i][j], lo[i][j], Ah[kk][tx * 4 + i], Al[kk][tx * 4 + i], Bh[kk][ty * 4 + j],
                               Bl[kk][ty * 4 + j]);
        __syncthreads();
    }
    const double d2 = dm.delta * dm.delta;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t t = t0 + ty * 4 + j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t s = s0 + tx * 4 + i;
            if (s < M && t < M) {
                const bool same = !dm.species || sp[s] == sp[t];
                double v = same ? d2 * ipow((double)hi[i][j] + (double)lo[i][j], dm.zeta) : 0.0;
                if (s == t) v += dm.jitter;
                K[s + t * M] = v;
            }
        }
    }
}

// ------------------------------------------------------------ Cholesky --
constexpr int CNB = 32;

// Factor the diagonal block K[k0:k0+kb, k0:k0+kb] (lower) in shared memory.
__global__ void k_potrf_diag(double *K, int64_t M, int64_t k0, int kb, DevStatus *st) {
    __shared__ double a[CNB][CNB + 1];
    __shared__ double rdiag;
    __shared__ int bad;
    const int tx = threadIdx.x % CNB, ty = threadIdx.x / CNB;  // 32 x 32 threads
    if (threadIdx.x == 0) bad = status_bad(st) ? 1 : 0;
    if (tx < kb && ty < kb) a[ty][tx] = K[(k0 + ty) + (k0 + tx) * M];
    __syncthreads();
    if (bad) return;
    for (int j = 0; j < kb; ++j) {
        if (threadIdx.x == 0) {
            double p = a[j][j];
            if (!(p > 0.0) || !isfinite(p)) {
                set_status(st, GAP_ERR_NOT_SPD, k0 + j);
                bad = 1;
            } else {
                const double y = rsqrt_f64(p);
                a[j][j] = p * y;
                rdiag = y;
            }
        }
        __syncthreads();
        if (bad) return;
        if (ty == 0 && tx > j && tx < kb) a[tx][j] *= rdiag;
        __syncthreads();
        if (tx > j && ty > j && tx < kb && ty < kb && ty >= tx) a[ty][tx] -= a[ty][j] * a[tx][j];
        __syncthreads();
    }
    if (tx < kb && ty < kb) K[(k0 + ty) + (k0 + tx) * M] = (ty >= tx) ? a[ty][tx] : 0.0;
}

// Rows i >= k0+kb of the panel: solve x L_kk^T = K[i, k0:k0+kb].
__global__ void k_trsm_panel(double *K, int64_t M, int64_t k0, int kb, int64_t end, const DevStatus *st) {
    __shared__ double L[CNB][CNB + 1];
    __shared__ double rd[CNB];
    if (status_bad(st)) return;
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
        int r = e % kb, c = e / kb;
        L[r][c] = K[(k0 + r) + (k0 + c) * M];
    }
    __syncthreads();
    if (threadIdx.x < kb) rd[threadIdx.x] = 1.0 / L[threadIdx.x][threadIdx.x];
    __syncthreads();
    int64_t i = k0 + kb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= end) return;
    double x[CNB];
#pragma unroll
    for (int j = 0; j < CNB; ++j) {
        if (j < kb) {
            double t = K[i + (k0 + j) * M];
            for (int l = 0; l < j; ++l) t -= x[l] * L[j][l];
            x[j] = t * rd[j];
        }
    }
#pragma unroll
    for (int j = 0; j < CNB; ++j)
        if (j < kb) K[i + (k0 + j) * M] = x[j];
}

// Trailing update of the lower triangle: K[i,l] -= sum_j P[i,j] P[l,j], i >= l.
__global__ void __launch_bounds__(256) k_syrk_lower(double *K, int64_t M, int64_t k0, int kb, int64_t end,
                                                    const DevStatus *st) {
    if (blockIdx.y > blockIdx.x) return;
    if (status_bad(st)) return;
    __shared__ double Pi[CNB][64];
    __shared__ double Pl[CNB][64];
    const int64_t base = k0 + kb;
    const int64_t i0 = base + (int64_t)blockIdx.x * 64, l0 = base + (int64_t)blockIdx.y * 64;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    for (int e = tid; e < 64 * kb; e += 256) {
        int r = e % 64, j = e / 64;
        Pi[j][r] = (i0 + r < end) ? K[(i0 + r) + (k0 + j) * M] : 0.0;
        Pl[j][r] = (l0 + r < end) ? K[(l0 + r) + (k0 + j) * M] : 0.0;
    }
    __syncthreads();
    double acc[4][4] = {};
    for (int j = 0; j < kb; ++j)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += Pi[j][tx * 4 + a] * Pl[j][ty * 4 + b];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        int64_t l = l0 + ty * 4 + b;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            int64_t i = i0 + tx * 4 + a;
            if (i < end && l < end && i >= l) K[i + l * M] -= acc[a][b];
        }
    }
}

// ------------------------------------------------ Cholesky, double-float --
// The mixed precisions factor K_MM in double-float arithmetic (pairs hi + lo of FP32
// values, about 48 significant bits) on the FP32 units; this GPU's FP64 units are too
// slow for the O(M^3) work.  U = L^T enters the design matrices in FP32, so the factor's
// rounding is far below what the matrices carry.  Kh, Kl (M x M, column-major, lower
// triangle) hold K_MM, are overwritten by L panel by panel, and L is written back to
// the FP64 K at the end.

// Kh, Kl = the double-float split of the lower triangle of K.
__global__ void k_split_lower(const double *__restrict__ K, int64_t M, float *__restrict__ Kh,
                              float *__restrict__ Kl) {
    const int64_t l = blockIdx.y, i = l + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const double v = K[i + l * M];
    const float h = (float)v;
    Kh[i + l * M] = h;
    Kl[i + l * M] = (float)(v - (double)h);
}

// K = Kh + Kl on the lower triangle (L in FP64).
__global__ void k_merge_lower(double *__restrict__ K, int64_t M, const float *__restrict__ Kh,
                              const float *__restrict__ Kl) {
    const int64_t l = blockIdx.y, i = l + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    K[i + l * M] = (double)Kh[i + l * M] + (double)Kl[i + l * M];
}

// Double-float helpers.  A pair (h, l) stands for h + l; accumulators are renormalised
// only when stored.
// h + l rounded to a normalised pair (Fast2Sum: |l| is small against |h|).
__device__ __forceinline__ void df_norm(float &h, float &l) {
    const float s = h + l;
    l = l - (s - h);
    h = s;
}
// (sh, sl) += a * b: the product's rounding error by FMA, the cross terms a_h b_l +
// a_l b_h folded in (a_l b_l is below 2^-48), the sum's rounding error by TwoSum (Knuth).
__device__ __forceinline__ void df_fma(float &sh, float &sl, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = sh + p;
    const float bp = s - sh;
    sl += ((sh - (s - bp)) + (p - bp)) + e;
    sh = s;
}
// (h, l) = a * b, normalised.
__device__ __forceinline__ void df_mul(float &h, float &l, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    h = p;
    l = e;
    df_norm(h, l);
}
// (h, l) -= (bh, bl), renormalised (TwoSum, then Fast2Sum).
__device__ __forceinline__ void df_sub(float &h, float &l, float bh, float bl) {
    const float s = h - bh;
    const float bp = s - h;
    float lo = (l - bl) + ((h - (s - bp)) + (-bh - bp));
    float hn = s;
    df_norm(hn, lo);
    h = hn;
    l = lo;
}
// 1 / sqrt(d) for d = dh + dl > 0: the FP32 estimate, one FP32 Newton step
// y <- y (3 - d y^2) / 2, then one Newton step with the residual 1 - d y^2 formed in
// double-float (the error squares at each step: about 2^-22 -> 2^-24 -> below 2^-46).
__device__ __forceinline__ void df_rsqrt(float dh, float dl, float &yh, float &yl) {
    float y = rsqrtf(dh);
    y = y * fmaf(-0.5f * dh, y * y, 1.5f);
    float qh, ql;  // y^2 exactly
    qh = y * y;
    ql = fmaf(y, y, -qh);
    float ph, pl;  // d y^2
    df_mul(ph, pl, dh, dl, qh, ql);
    // r = 1 - d y^2 (small: |r| below about 2^-22)
    const float r = (1.f - ph) - pl;
    yh = y;
    yl = 0.5f * y * r;
    df_norm(yh, yl);
}

// Cholesky A = L L^T of a symmetric positive definite block (kb <= 32 rows and columns, its
// lower triangle in A) in double-float, and X = L^{-1}, by the 1024 threads of the CTA
// (thread (i, l) = entry (i, l)).  One barrier per step: every thread forms the pivot
// itself; column j of L goes to L while the trailing update reads A's column j unscaled
// (and scales it in registers), and row j of X goes to X while the rows below read B's
// row j unscaled.  A and B (work) are consumed; L and X come out normalised, zero outside
// the lower triangle; r = 1 / L_jj.  Returns false (the same in every thread) when a pivot
// is not positive and finite, its index in *jbad.  The caller synchronises after filling A.
typedef float DfTile[CNB][CNB + 1];
__device__ bool df_chol_inv32(DfTile &Ah, DfTile &Al, DfTile &Lh, DfTile &Ll, DfTile &Bh, DfTile &Bl, DfTile &Xh,
                              DfTile &Xl, float *rh, float *rl, int kb, int *jbad) {
    const int l = threadIdx.x % CNB, i = threadIdx.x / CNB;
    Bh[i][l] = (i == l && i < kb) ? 1.f : 0.f;
    Bl[i][l] = 0.f;
    Lh[i][l] = Ll[i][l] = Xh[i][l] = Xl[i][l] = 0.f;
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        float dh = Ah[j][j], dl = Al[j][j];
        df_norm(dh, dl);
        if (!(dh > 0.f) || !isfinite(dh)) {  // the same in every thread
            *jbad = j;
            return false;
        }
        // only the threads of column j and of the trailing block's lower triangle need 1 / sqrt(d)
        if (i >= l && l >= j) {
            float yh, yl;
            df_rsqrt(dh, dl, yh, yl);
            if (i == j && l == j) {
                rh[j] = yh;
                rl[j] = yl;
            }
            if (l == j && i < kb) {
                if (i == j) {
                    df_mul(Lh[j][j], Ll[j][j], dh, dl, yh, yl);  // L_jj = d / sqrt(d)
                } else {
                    float h = Ah[i][j], lo = Al[i][j];
                    df_norm(h, lo);
                    df_mul(Lh[i][j], Ll[i][j], h, lo, yh, yl);
                }
            }
            if (l > j && i >= l && i < kb) {
                float ah = Ah[i][j], al = Al[i][j], bh = Ah[l][j], bl = Al[l][j];
                df_norm(ah, al);
                df_norm(bh, bl);
                float sh, sl, th, tl;
                df_mul(sh, sl, ah, al, yh, yl);  // L[i, j]
                df_mul(th, tl, bh, bl, yh, yl);  // L[l, j]
                df_fma(Ah[i][l], Al[i][l], -sh, -sl, th, tl);
            }
        }
        __syncthreads();
    }
    for (int j = 0; j < kb; ++j) {
        if (l <= j && i >= j && i < kb) {
            float bh = Bh[j][l], bl = Bl[j][l];
            df_norm(bh, bl);
            float xh, xl;
            df_mul(xh, xl, bh, bl, rh[j], rl[j]);  // X[j, l] = B[j, l] / L_jj
            if (i == j) {
                Xh[j][l] = xh;
                Xl[j][l] = xl;
            } else {
                df_fma(Bh[i][l], Bl[i][l], -xh, -xl, Lh[i][j], Ll[i][j]);  // B[i, l] -= L[i, j] X[j, l]
            }
        }
        __syncthreads();
    }
    return true;
}

// The diagonal block of the K_MM factor: L_kk back to Kh / Kl, X = L_kk^{-1} to Xh / Xl
// (CNB x CNB, row-major) for the panel solve.
__global__ void __launch_bounds__(CNB *CNB) k_potrf_diag_df(float *__restrict__ Kh, float *__restrict__ Kl, int64_t M,
                                                           int64_t k0, int kb, float *__restrict__ Xh_g,
                                                           float *__restrict__ Xl_g, DevStatus *st) {
    __shared__ DfTile Ah, Al, Lh, Ll, Bh, Bl, Xh, Xl;
    __shared__ float rh[CNB], rl[CNB];
    __shared__ int bad;
    const int l = threadIdx.x % CNB, i = threadIdx.x / CNB;
    {
        const bool in = i < kb && l < kb && l <= i;
        const int64_t at = (k0 + i) + (k0 + l) * M;
        Ah[i][l] = in ? Kh[at] : 0.f;
        Al[i][l] = in ? Kl[at] : 0.f;
    }
    if (threadIdx.x == 0) bad = status_bad(st) ? 1 : 0;
    __syncthreads();
    if (bad) return;
    int jb = 0;
    if (!df_chol_inv32(Ah, Al, Lh, Ll, Bh, Bl, Xh, Xl, rh, rl, kb, &jb)) {
        if (threadIdx.x == 0) set_status(st, GAP_ERR_NOT_SPD, k0 + jb);
        return;
    }
    if (i < kb && l <= i) {
        const int64_t at = (k0 + i) + (k0 + l) * M;
        Kh[at] = Lh[i][l];
        Kl[at] = Ll[i][l];
        Xh_g[i * CNB + l] = Xh[i][l];
        Xl_g[i * CNB + l] = Xl[i][l];
    }
}

// Rows i >= k0 + kb of the panel: x = K[i, k0:k0+kb] L_kk^{-T}, i.e. x_j = sum_{q <= j}
// K[i, q] X[j, q], in place in Kh / Kl.  A CTA takes 32 rows; thread (row r, group g)
// forms the outputs j = g + 8 k, k < 4.
constexpr int TRS_ROWS = 32, TRS_GROUPS = 8;
__global__ void __launch_bounds__(TRS_ROWS *TRS_GROUPS) k_trsm_panel_df(float *__restrict__ Kh, float *__restrict__ Kl,
                                                                       int64_t M, int64_t k0, int kb, int64_t end,
                                                                       const float *__restrict__ Xh_g,
                                                                       const float *__restrict__ Xl_g,
                                                                       const DevStatus *st) {
    __shared__ float Bh[CNB][TRS_ROWS + 1], Bl[CNB][TRS_ROWS + 1], Xh[CNB][CNB + 1], Xl[CNB][CNB + 1];
    if (status_bad(st)) return;
    const int64_t r0 = k0 + kb + (int64_t)blockIdx.x * TRS_ROWS;
    for (int e = threadIdx.x; e < CNB * TRS_ROWS; e += blockDim.x) {
        const int r = e % TRS_ROWS, q = e / TRS_ROWS;
        const bool ok = q < kb && r0 + r < end;
        const int64_t at = (r0 + r) + (k0 + q) * M;
        Bh[q][r] = ok ? Kh[at] : 0.f;
        Bl[q][r] = ok ? Kl[at] : 0.f;
    }
    for (int e = threadIdx.x; e < CNB * CNB; e += blockDim.x) {
        const int j = e / CNB, q = e % CNB;
        const bool ok = j < kb && q <= j;
        Xh[j][q] = ok ? Xh_g[j * CNB + q] : 0.f;
        Xl[j][q] = ok ? Xl_g[j * CNB + q] : 0.f;
    }
    __syncthreads();
    const int r = threadIdx.x % TRS_ROWS, g = threadIdx.x / TRS_ROWS;
    float xh[CNB / TRS_GROUPS], xl[CNB / TRS_GROUPS];
#pragma unroll
    for (int k = 0; k < CNB / TRS_GROUPS; ++k) xh[k] = xl[k] = 0.f;
    for (int q = 0; q < kb; ++q) {
        const float bh = Bh[q][r], bl = Bl[q][r];
#pragma unroll
        for (int k = 0; k < CNB / TRS_GROUPS; ++k) {
            const int j = g + TRS_GROUPS * k;
            if (q <= j) df_fma(xh[k], xl[k], bh, bl, Xh[j][q], Xl[j][q]);
        }
    }
    const int64_t i = r0 + r;
    if (i < end)
#pragma unroll
        for (int k = 0; k < CNB / TRS_GROUPS; ++k) {
            const int j = g + TRS_GROUPS * k;
            if (j < kb) {
                float h = xh[k], lo = xl[k];
                df_norm(h, lo);
                Kh[i + (k0 + j) * M] = h;
                Kl[i + (k0 + j) * M] = lo;
            }
        }
}

// Trailing update of the lower triangle: K[i, l] -= sum_j L[i, j] L[l, j] over the panel's
// columns j, on the 64 x 64 tiles with i-tile >= l-tile (one CTA each, triangular
// numbering); thread (tx, ty) forms the 4 x 4 outputs rows 4 tx .., columns 4 ty ...
__global__ void __launch_bounds__(256) k_syrk_lower_df(float *__restrict__ Kh, float *__restrict__ Kl, int64_t M,
                                                       int64_t k0, int kb, int64_t end, const DevStatus *st) {
    if (status_bad(st)) return;
    const int64_t t = blockIdx.x;
    int64_t bx = (int64_t)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((bx + 1) * (bx + 2) / 2 <= t) ++bx;
    while (bx * (bx + 1) / 2 > t) --bx;
    const int64_t by = t - bx * (bx + 1) / 2;
    __shared__ __align__(16) float Aih[CNB][64], Ail[CNB][64], Alh[CNB][64], All[CNB][64];
    const int64_t base = k0 + kb, i0 = base + bx * 64, l0 = base + by * 64;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    for (int e = tid; e < 64 * kb; e += 256) {
        const int r = e % 64, j = e / 64;
        const int64_t ci = (k0 + j) * M;
        const bool okI = i0 + r < end, okL = l0 + r < end;
        Aih[j][r] = okI ? Kh[i0 + r + ci] : 0.f;
        Ail[j][r] = okI ? Kl[i0 + r + ci] : 0.f;
        Alh[j][r] = okL ? Kh[l0 + r + ci] : 0.f;
        All[j][r] = okL ? Kl[l0 + r + ci] : 0.f;
    }
    __syncthreads();
    float ah[4][4], al[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ah[a][b] = al[a][b] = 0.f;
    for (int j = 0; j < kb; ++j) {
        const float4 xh = *reinterpret_cast<const float4 *>(&Aih[j][tx * 4]);
        const float4 xl = *reinterpret_cast<const float4 *>(&Ail[j][tx * 4]);
        const float4 yh = *reinterpret_cast<const float4 *>(&Alh[j][ty * 4]);
        const float4 yl = *reinterpret_cast<const float4 *>(&All[j][ty * 4]);
        const float xa[4] = {xh.x, xh.y, xh.z, xh.w}, xb[4] = {xl.x, xl.y, xl.z, xl.w};
        const float ya[4] = {yh.x, yh.y, yh.z, yh.w}, yb[4] = {yl.x, yl.y, yl.z, yl.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) df_fma(ah[a][b], al[a][b], xa[a], xb[a], ya[b], yb[b]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int64_t l = l0 + ty * 4 + b;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t i = i0 + tx * 4 + a;
            if (i < end && l < end && i >= l) {
                float h = Kh[i + l * M], lo = Kl[i + l * M];
                df_sub(h, lo, ah[a][b], al[a][b]);
                Kh[i + l * M] = h;
                Kl[i + l * M] = lo;
            }
        }
    }
}

// A[N + i, j] = L[j, i] for i <= j (U = L^T); tile transpose through shared memory.
template <class T>
__global__ void k_stack_u(Dims dm, const double *__restrict__ L, T *__restrict__ A, int blocked) {
    __shared__ double tile[32][33];
    const int64_t M = dm.M;
    int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        int64_t i = i0 + r, j = j0 + tx;  // read L[j, i] = L[j + i*M]
        tile[r][tx] = (i < M && j < M) ? L[j + i * M] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        int64_t j = j0 + r, i = i0 + tx;
        if (i < M && j < M) {
            const int64_t at = blocked ? acc_index(dm.N + i, j, M + 1) : (dm.N + i) + j * dm.ld;
            A[at] = (i <= j) ? T(tile[tx][r]) : T(0);
        }
    }
}

// -------------------------------------------------------- Householder QR --
constexpr int QNB = 32;      // maximum panel width of the column kernels
constexpr int QTHREADS = 256;

template <class T>
__device__ __forceinline__ T block_sum_vec(T *vals, int n, T *red) {
    // reduce vals[0..n) (per thread) over the block into red[0..n); returns nothing useful
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = 0; q < n; ++q) {
        T v = vals[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * (QNB + 1) + q] = v;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        T s = T(0);
        for (int w = 0; w < nw; ++w) s += red[w * (QNB + 1) + threadIdx.x];
        red[8 * (QNB + 1) + threadIdx.x] = s;
    }
    __syncthreads();
    return T(0);
}

// Rows of the panel owned by block b: [lo, hi) within [k0, rows).
__device__ __forceinline__ void block_rows(int64_t k0, int64_t rows, int64_t &lo, int64_t &hi) {
    int64_t n = rows - k0, per = (n + gridDim.x - 1) / gridDim.x;
    lo = k0 + (int64_t)blockIdx.x * per;
    hi = min(rows, lo + per);
}

// Partial sums for column j: part[b*(QNB+1) + 0] = sum_{i>j} A[i,j]^2,
// part[..+1+q] = sum_{i>j} A[i,j] A[i,j+1+q]; diag[q] = A[j, j+q] (owner block).
template <class T>
__global__ void __launch_bounds__(QTHREADS) k_qr_col_init(const T *A, int64_t rows, int64_t ld, int64_t k0,
                                                           int64_t k1, T *part, T *diag) {
    __shared__ T red[9 * (QNB + 1)];
    int64_t lo, hi;
    block_rows(k0, rows, lo, hi);
    const int64_t j = k0;
    const int nq = (int)(k1 - j);  // values: norm + (nq-1) dots
    T acc[QNB];
#pragma unroll
    for (int q = 0; q < QNB; ++q) acc[q] = T(0);
    for (int64_t i = max(lo, j + 1) + threadIdx.x; i < hi; i += blockDim.x) {
        T x = A[i + j * ld];
        acc[0] += x * x;
#pragma unroll
        for (int q = 1; q < QNB; ++q)
            if (q < nq) acc[q] += x * A[i + (j + q) * ld];
    }
    block_sum_vec(acc, nq, red);
    if (threadIdx.x < nq) part[(int64_t)blockIdx.x * (QNB + 1) + threadIdx.x] = red[8 * (QNB + 1) + threadIdx.x];
    if (j >= lo && j < hi && threadIdx.x < nq) diag[threadIdx.x] = A[j + (j + threadIdx.x) * ld];
}

// One Householder step on column j of the panel [k0, k1).
template <class T>
__global__ void __launch_bounds__(QTHREADS) k_qr_col_step(T *A, int64_t rows, int64_t ld, int64_t k0, int64_t k1,
                                                           int64_t j, T *tau, const T *part_in, T *part_out,
                                                           const T *diag_in, T *diag_out) {
    __shared__ T red[9 * (QNB + 1)];
    __shared__ T sh_w[QNB];
    __shared__ T sh_par[3];  // tau, scale s, beta
    const int nq = (int)(k1 - j);  // columns j..k1-1
    // 1. finish the reductions for column j: 8 groups of 32 threads each sum every
    //    8th block's partials, then the 8 group sums are added in group order
    {
        const int q = threadIdx.x & 31, g = threadIdx.x >> 5;
        T s = T(0);
        if (q < nq) {
#pragma unroll 4
            for (int b = g; b < (int)gridDim.x; b += 8) s += part_in[b * (QNB + 1) + q];
        }
        red[g * (QNB + 1) + q] = s;
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        T s = T(0);
        for (int g = 0; g < 8; ++g) s += red[g * (QNB + 1) + threadIdx.x];
        red[8 * (QNB + 1) + threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x < nq) red[threadIdx.x] = red[8 * (QNB + 1) + threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        T norm2 = red[0], alpha = diag_in[0];
        T t = T(0), sc = T(0), beta = alpha;
        if (norm2 != T(0)) {
            beta = -copysign(sqrt(alpha * alpha + norm2), alpha);
            t = (beta - alpha) / beta;
            sc = T(1) / (alpha - beta);
        }
        sh_par[0] = t;
        sh_par[1] = sc;
        sh_par[2] = beta;
    }
    __syncthreads();
    const T t = sh_par[0], sc = sh_par[1];
    if (threadIdx.x >= 1 && threadIdx.x < nq) sh_w[threadIdx.x] = diag_in[threadIdx.x] + sc * red[threadIdx.x];
    __syncthreads();
    int64_t lo, hi;
    block_rows(k0, rows, lo, hi);
    // 2. the diagonal row j (owner block): R entries and tau
    if (j >= lo && j < hi) {
        if (threadIdx.x == 0) {
            A[j + j * ld] = sh_par[2];
            tau[j] = t;
        } else if (threadIdx.x < nq) {
            A[j + (j + threadIdx.x) * ld] = diag_in[threadIdx.x] - t * sh_w[threadIdx.x];
        }
    }
    // 3. rows i > j: scale v, update the panel columns, partials for column j+1
    const bool more = j + 1 < k1;
    const int nq2 = nq - 1;  // values for column j+1: norm + (nq2-1) dots
    T acc[QNB];
#pragma unroll
    for (int q = 0; q < QNB; ++q) acc[q] = T(0);
    for (int64_t i = max(lo, j + 1) + threadIdx.x; i < hi; i += blockDim.x) {
        T v = sc * A[i + j * ld];
        A[i + j * ld] = v;
        T y0 = T(0);
#pragma unroll
        for (int q = 1; q < QNB; ++q) {
            if (q < nq) {
                T aq = A[i + (j + q) * ld] - t * v * sh_w[q];
                A[i + (j + q) * ld] = aq;
                if (q == 1) y0 = aq;
                if (more && i > j + 1) {
                    if (q == 1)
                        acc[0] += aq * aq;
                    else
                        acc[q - 1] += y0 * aq;
                }
            }
        }
        if (more && i == j + 1) {
            // new diagonal row j+1: A[j+1, j+1 .. k1)
            for (int q = 1; q < nq; ++q) diag_out[q - 1] = A[i + (j + q) * ld];
        }
    }
    if (more) {
        block_sum_vec(acc, nq2, red);
        if (threadIdx.x < nq2)
            part_out[(int64_t)blockIdx.x * (QNB + 1) + threadIdx.x] = red[8 * (QNB + 1) + threadIdx.x];
    }
}

// V^T V partials of the panel: V[i, a] = 0 (i < k0+a), 1 (i == k0+a), A[i, k0+a] (i > k0+a).
template <class T>
__device__ __forceinline__ T vval(const T *A, int64_t ld, int64_t k0, int64_t i, int a) {
    int64_t c = k0 + a;
    return i < c ? T(0) : (i == c ? T(1) : A[i + c * ld]);
}

template <class T>
__global__ void __launch_bounds__(256) k_qr_vtv(const T *A, int64_t rows, int64_t ld, int64_t k0, int kb,
                                               T *part /* [grid][QNB*QNB] */) {
    __shared__ T Vs[64][QNB + 1];
    int64_t lo, hi;
    block_rows(k0, rows, lo, hi);
    // each thread owns (a, b) entries e = tid, tid+256, ... of the kb x kb Gram
    T acc[4] = {};
    for (int64_t r0 = lo; r0 < hi; r0 += 64) {
        for (int e = threadIdx.x; e < 64 * QNB; e += 256) {
            int r = e % 64, a = e / 64;
            int64_t i = r0 + r;
            Vs[r][a] = (i < hi && a < kb) ? vval(A, ld, k0, i, a) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = threadIdx.x + 256 * q;
            int a = e / QNB, b = e % QNB;
            T s = T(0);
            for (int r = 0; r < 64; ++r) s += Vs[r][a] * Vs[r][b];
            acc[q] += s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) part[(int64_t)blockIdx.x * QNB * QNB + threadIdx.x + 256 * q] = acc[q];
}

// T (upper, kb x kb, stored T[a + b*QNB]) from the Gram of V and tau (LAPACK larft, forward, columnwise):
// T[j,j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] (V^T V)[0:j, j].
template <class T>
__global__ void k_qr_tfactor(const T *part, int nparts, const T *tau, int64_t k0, int kb, T *Tm) {
    __shared__ T G[QNB][QNB + 1];
    __shared__ T Ts[QNB][QNB + 1];
    __shared__ T tmp[QNB];
    for (int e = threadIdx.x; e < QNB * QNB; e += blockDim.x) {
        T s = T(0);
        for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * QNB * QNB + e];
        G[e / QNB][e % QNB] = s;
        Ts[e / QNB][e % QNB] = T(0);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        T tj = tau[k0 + j];
        if (threadIdx.x < j) {
            T s = T(0);
            for (int l = threadIdx.x; l < j; ++l) s += Ts[threadIdx.x][l] * G[l][j];
            tmp[threadIdx.x] = -tj * s;
        }
        __syncthreads();
        if (threadIdx.x < j) Ts[threadIdx.x][j] = tmp[threadIdx.x];
        if (threadIdx.x == 0) Ts[j][j] = tj;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < QNB * QNB; e += blockDim.x) Tm[e] = Ts[e % QNB][e / QNB];
}

// W partials: Wpart[rb][a][c] = sum_{i in row block rb} V[i,a] C[i,c], C = A[:, c0 + c].
// Grid: (ceil(nt/64), n_rb); 256 threads; each thread 8 (a) x 1 (c) ... tile 32 x 64.
template <class T>
__global__ void __launch_bounds__(256) k_qr_vtc(const T *A, int64_t rows, int64_t ld, int64_t k0, int kb, int64_t c0,
                                               int64_t nt, T *Wpart) {
    __shared__ T Vs[32][QNB + 1];
    __shared__ T Cs[32][65];
    const int64_t cb = (int64_t)blockIdx.x * 64;
    const int64_t n = rows - k0, per = (n + gridDim.y - 1) / gridDim.y;
    const int64_t lo = k0 + (int64_t)blockIdx.y * per, hi = min(rows, lo + per);
    const int tid = threadIdx.x, tc = tid % 64, ta = tid / 64;  // ta: 0..3 -> a = ta*8 .. +8
    T acc[8] = {};
    for (int64_t r0 = lo; r0 < hi; r0 += 32) {
        for (int e = tid; e < 32 * QNB; e += 256) {
            int r = e % 32, a = e / 32;
            int64_t i = r0 + r;
            Vs[r][a] = (i < hi && a < kb) ? vval(A, ld, k0, i, a) : T(0);
        }
        for (int e = tid; e < 32 * 64; e += 256) {
            int r = e % 32, c = e / 32;
            int64_t i = r0 + r;
            Cs[r][c] = (i < hi && cb + c < nt) ? A[i + (c0 + cb + c) * ld] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
            T cv = Cs[r][tc];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] += Vs[r][ta * 8 + q] * cv;
        }
        __syncthreads();
    }
    if (cb + tc < nt) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int a = ta * 8 + q;
            if (a < kb) Wpart[((int64_t)blockIdx.y * QNB + a) * nt + cb + tc] = acc[q];
        }
    }
}

// W2[a][c] = sum_b T[b,a] W[b][c], W = sum over row blocks (fixed order).
// Block: 32 columns (threadIdx.x, coalesced) x 32 reflectors (threadIdx.y).
template <class T>
__global__ void __launch_bounds__(1024) k_qr_wreduce(const T *Wpart, int n_rb, const T *Tm, int kb, int64_t nt, T *W2) {
    __shared__ T ws[QNB][33];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int a = threadIdx.y;
    T s = T(0);
    if (c < nt && a < kb)
        for (int rb = 0; rb < n_rb; ++rb) s += Wpart[((int64_t)rb * QNB + a) * nt + c];
    ws[a][threadIdx.x] = s;
    __syncthreads();
    if (c < nt && a < kb) {
        T w = T(0);
        for (int b = 0; b <= a; ++b) w += Tm[b + a * QNB] * ws[b][threadIdx.x];
        W2[(int64_t)a * nt + c] = w;
    }
}

// C[i, c] -= sum_a V[i, a] W2[a, c] for rows i >= k0.  Tile 128 rows x 64 columns.
template <class T>
__global__ void __launch_bounds__(256) k_qr_update(T *A, int64_t rows, int64_t ld, int64_t k0, int kb, int64_t c0,
                                                  int64_t nt, const T *W2) {
    __shared__ T Vs[QNB][128];
    __shared__ T Ws[QNB][64];
    const int64_t i0 = k0 + (int64_t)blockIdx.x * 128, cb = (int64_t)blockIdx.y * 64;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;  // rows ty*8.., cols tx*4..
    for (int e = tid; e < 128 * QNB; e += 256) {
        int r = e % 128, a = e / 128;
        int64_t i = i0 + r;
        Vs[a][r] = (i < rows && a < kb) ? vval(A, ld, k0, i, a) : T(0);
    }
    for (int e = tid; e < 64 * QNB; e += 256) {
        int c = e % 64, a = e / 64;
        Ws[a][c] = (a < kb && cb + c < nt) ? W2[(int64_t)a * nt + cb + c] : T(0);
    }
    __syncthreads();
    T acc[8][4] = {};
    for (int a = 0; a < kb; ++a) {
        T v[8], w[4];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = Vs[a][ty * 8 + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) w[c] = Ws[a][tx * 4 + c];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] += v[r] * w[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int64_t col = cb + tx * 4 + c;
        if (col >= nt) continue;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int64_t i = i0 + ty * 8 + r;
            if (i < rows) A[i + (c0 + col) * ld] -= acc[r][c];
        }
    }
}

// Partial V^T C over one row block: Wpart[rb][a][c] = sum_{i in block rb} V[i,a] C[i,c],
// C = A[:, c0 + c].  CTA tile: 32 reflectors x QBN columns; thread tile 8 reflectors
// (8*ta + i) x QBN/64 columns (tc + 64 j); rows streamed in chunks of 16.
// Grid: (ceil(nt / QBN), n_rb); 256 threads; dynamic smem (16*32 + 16*QBN) elements.
template <class T>
__global__ void __launch_bounds__(256) k_qr_vtc2(const T *A, int64_t rows, int64_t ld, int64_t k0, int kb,
                                                int64_t c0, int64_t nt, T *Wpart) {
    constexpr int BK = 16, QBN = sizeof(T) == 4 ? 512 : 256, NJ = QBN / 64;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int VS = QNB + 1, CS = QBN + 1;  // padded strides: conflict-free row-wise fills
    T *Vs = reinterpret_cast<T *>(sm_raw);  // [BK][VS]
    T *Cs = Vs + BK * VS;                    // [BK][CS]
    const int64_t cb = (int64_t)blockIdx.x * QBN;
    const int64_t n = rows - k0, per = (n + gridDim.y - 1) / gridDim.y;
    const int64_t lo = k0 + (int64_t)blockIdx.y * per, hi = min(rows, lo + per);
    const int tid = threadIdx.x, ta = tid / 64, tc = tid % 64;
    T acc[8][NJ];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[i][j] = T(0);
    for (int64_t r0 = lo; r0 < hi; r0 += BK) {
        for (int e = tid; e < BK * QNB; e += 256) {
            const int r = e % BK, a = e / BK;
            const int64_t i = r0 + r;
            Vs[r * VS + a] = (i < hi && a < kb) ? vval(A, ld, k0, i, a) : T(0);
        }
        for (int e = tid; e < BK * QBN; e += 256) {
            const int r = e % BK, c = e / BK;
            const int64_t i = r0 + r;
            Cs[r * CS + c] = (i < hi && cb + c < nt) ? A[i + (c0 + cb + c) * ld] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < BK; ++k) {
            T v[8], cc[NJ];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = Vs[k * VS + ta * 8 + i];
#pragma unroll
            for (int j = 0; j < NJ; ++j) cc[j] = Cs[k * CS + tc + 64 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) acc[i][j] += v[i] * cc[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int a = ta * 8 + i;
        if (a >= kb) continue;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int64_t c = cb + tc + 64 * j;
            if (c < nt) Wpart[((int64_t)blockIdx.y * QNB + a) * nt + c] = acc[i][j];
        }
    }
}

// C[i, c] -= sum_a V[i, a] W2[a, c] for rows i >= k0.  CTA tile 128 rows x 128
// columns; thread tile 8 rows (tx + 16 i) x 8 columns (ty + 16 j), so a half warp
// touches 16 consecutive rows of one column.  Dynamic smem 2 * 32 * 128 elements.
template <class T>
__global__ void __launch_bounds__(256) k_qr_update2(T *A, int64_t rows, int64_t ld, int64_t k0, int kb, int64_t c0,
                                                   int64_t nt, const T *W2) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *Vs = reinterpret_cast<T *>(sm_raw);  // [QNB][128]
    T *Ws = Vs + QNB * 128;                  // [QNB][128]
    const int64_t i0 = k0 + (int64_t)blockIdx.x * 128, cb = (int64_t)blockIdx.y * 128;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    for (int e = tid; e < 128 * QNB; e += 256) {
        const int r = e % 128, a = e / 128;
        const int64_t i = i0 + r;
        Vs[a * 128 + r] = (i < rows && a < kb) ? vval(A, ld, k0, i, a) : T(0);
        const int c = e % 128;
        Ws[a * 128 + c] = (a < kb && cb + c < nt) ? W2[(int64_t)a * nt + cb + c] : T(0);
    }
    __syncthreads();
    T acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
    for (int a = 0; a < kb; ++a) {
        T v[8], w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = Vs[a * 128 + tx + 16 * i];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = Ws[a * 128 + ty + 16 * j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] += v[i] * w[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t col = cb + ty + 16 * j;
        if (col >= nt) continue;
        T *cp = A + (c0 + col) * ld;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t r = i0 + tx + 16 * i;
            if (r < rows) cp[r] -= acc[i][j];
        }
    }
}

// ---------------------------------------- two-level QR: outer panels of 128 --
// The FP32 factorisation factors outer panels of up to QNBO = 128 columns as
// four inner panels of 32 (column kernels + updates confined to the outer
// panel), then applies the 128 reflectors to the trailing columns once:
//   G = V^T V -> T (compact WY), Y = V^T C, W2 = T^T Y, C <- C - V W2,
// the last product on the tensor cores with split-TF32 operands.
constexpr int QNBO = 128;


// G = sum of the partials in block order.
__global__ void k_qr_gram_reduce(const float *Gp, int nparts, int nt, float *G) {
    // G[a][b] = sum over the split partials Yp[split][a][b] (stride nt); zero for b >= nt
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= QNBO * QNBO) return;
    const int a = e / QNBO, bb = e % QNBO;
    float s = 0.f;
    if (bb < nt)
        for (int p = 0; p < nparts; ++p) s += Gp[((int64_t)p * QNBO + a) * nt + bb];
    G[e] = s;
}

// Compact-WY T (upper, column-major T[a + b*QNBO]) from G = V^T V and tau (the LAPACK
// larft recurrence T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j], T[j, j] = tau_j).  G and T sit
// in shared memory; for each j, four threads per row i < j split the row's dot product and
// combine it by shuffles.  512 threads; dynamic smem 2 QNBO (QNBO + 1) floats.
__global__ void __launch_bounds__(512) k_qr_tfactor_big(const float *G, const float *tau, int64_t K0, int nbo,
                                                       float *Tm) {
    extern __shared__ float tsm[];
    float *Ts = tsm;                      // [QNBO][QNBO + 1], row-major T[i][j]
    float *Gs = tsm + QNBO * (QNBO + 1);  // [QNBO][QNBO + 1], Gs[l][j] = G[l, j]
    for (int e = threadIdx.x; e < QNBO * QNBO; e += blockDim.x) {
        const int l = e / QNBO, j = e % QNBO;
        Gs[l * (QNBO + 1) + j] = G[l * QNBO + j];
        Ts[l * (QNBO + 1) + j] = 0.f;
    }
    __syncthreads();
    const int i = threadIdx.x >> 2, sub = threadIdx.x & 3;
    for (int j = 0; j < nbo; ++j) {
        const float tj = tau[K0 + j];
        float s = 0.f;
        if (i < j)
            for (int l = i + sub; l < j; l += 4) s += Ts[i * (QNBO + 1) + l] * Gs[l * (QNBO + 1) + j];
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        __syncthreads();  // every read of column j's inputs is done
        if (sub == 0 && i < j) Ts[i * (QNBO + 1) + j] = -tj * s;
        if (threadIdx.x == 0) Ts[j * (QNBO + 1) + j] = tj;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < QNBO * QNBO; e += blockDim.x) Tm[e] = Ts[(e % QNBO) * (QNBO + 1) + e / QNBO];
}


__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float rest = x - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(rest));
    hi = __uint_as_float(h);
    lo = __uint_as_float(l);
}

// W2^T = (T^T Y)^T for the trailing columns: Y = sum of the n_split partials
// Yp[split][a][c] (fixed order, eight independent sums in flight), then
// W2[a, c] = sum_{b <= a} T[b, a] Y[b, c], stored transposed as Wt[c * kpad + a]
// (TF32 split into hi/lo; lo skipped when Wt_lo is null).  Block (32, 32): threadIdx.x
// = column, threadIdx.y + 32 q = reflector.
__global__ void __launch_bounds__(1024) k_qr_w2t(const float *Yp, int n_split, const float *Tm, int nbo, int64_t nt,
                                                int kpad, float *Wt_hi, float *Wt_lo) {
    __shared__ float Ys[QNBO][33];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    for (int q = 0; q < 4; ++q) {
        const int a = threadIdx.y + 32 * q;
        float s = 0.f;
        if (c < nt && a < nbo) {
            const float *y = Yp + (int64_t)a * nt + c;
            const int64_t stride = (int64_t)QNBO * nt;
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            int sp = 0;
            for (; sp + 8 <= n_split; sp += 8)
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] += y[(int64_t)(sp + u) * stride];
            for (; sp < n_split; ++sp) acc[0] += y[(int64_t)sp * stride];
            s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        }
        Ys[a][threadIdx.x] = s;
    }
    __syncthreads();
    if (c >= nt) return;
    for (int q = 0; q < 4; ++q) {
        const int a = threadIdx.y + 32 * q;
        if (a >= kpad) break;
        float w = 0.f;
        if (a < nbo)
            for (int bb = 0; bb <= a; ++bb) w += Tm[bb + a * QNBO] * Ys[bb][threadIdx.x];
        float h, lo;
        tf32_split(w, h, lo);
        Wt_hi[c * kpad + a] = h;
        if (Wt_lo) Wt_lo[c * kpad + a] = lo;
    }
}

// T12 = -T1 G12 T2 for a pair of outer panels (compact WY of the product of their
// block reflectors: T = [T1 T12; 0 T2]), with G12 = V1^T V2 row-major [a][b] and T1,
// T2, T12 column-major with stride QNBO.  Grid nb2 (column c), block QNBO (row a).
__global__ void __launch_bounds__(QNBO) k_qr_t12(const float *__restrict__ G12, const float *__restrict__ T1,
                                                 const float *__restrict__ T2, int nb2, float *__restrict__ T12) {
    __shared__ float xs[QNBO];
    const int a = threadIdx.x, c = blockIdx.x;
    float x = 0.f;  // (G12 T2)[a, c]
    for (int b = 0; b <= c; ++b) x += G12[a * QNBO + b] * T2[b + c * QNBO];
    xs[a] = x;
    __syncthreads();
    float t = 0.f;
    for (int b = a; b < QNBO; ++b) t += T1[a + b * QNBO] * xs[b];
    T12[a + c * QNBO] = -t;
}

// W2^T for a pair of outer panels (128 + nb2 reflectors): Y1 = V1^T C and Y2 = V2^T C
// summed from their split partials (split stride ystride floats), then W2 = T^T [Y1; Y2],
// i.e. rows a < 128:
// sum_{b <= a} T1[b, a] Y1[b, c]; rows 128 + a2: sum_b T12[b, a2] Y1[b, c] +
// sum_{b <= a2} T2[b, a2] Y2[b, c]; stored as Wt[c * kpad + a] (TF32 hi slice, zero
// for a >= 128 + nb2).  Block (32, 32): threadIdx.x = column.
__global__ void __launch_bounds__(1024) k_qr_w2t_pair(const float *Yp1, int ns1, const float *Yp2, int ns2,
                                                     int64_t ystride, const float *T1, const float *T12,
                                                     const float *T2, int nb2, int64_t nt, int kpad, float *Wt_hi) {
    __shared__ float Y1s[QNBO][33], Y2s[QNBO][33];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t stride = ystride;
    for (int q = 0; q < 4; ++q) {
        const int a = threadIdx.y + 32 * q;
        float s1 = 0.f, s2 = 0.f;
        if (c < nt) {
            float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const float *y = Yp1 + (int64_t)a * nt + c;
            int sp = 0;
            for (; sp + 8 <= ns1; sp += 8)
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] += y[(int64_t)(sp + u) * stride];
            for (; sp < ns1; ++sp) acc[0] += y[(int64_t)sp * stride];
            s1 = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
            if (a < nb2) {
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] = 0.f;
                y = Yp2 + (int64_t)a * nt + c;
                sp = 0;
                for (; sp + 8 <= ns2; sp += 8)
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc[u] += y[(int64_t)(sp + u) * stride];
                for (; sp < ns2; ++sp) acc[0] += y[(int64_t)sp * stride];
                s2 = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
            }
        }
        Y1s[a][threadIdx.x] = s1;
        Y2s[a][threadIdx.x] = s2;
    }
    __syncthreads();
    if (c >= nt) return;
    for (int q = 0; q < 8; ++q) {
        const int a = threadIdx.y + 32 * q;
        if (a >= kpad) break;
        float w = 0.f;
        if (a < QNBO) {
            for (int b = 0; b <= a; ++b) w += T1[b + a * QNBO] * Y1s[b][threadIdx.x];
        } else if (a - QNBO < nb2) {
            const int a2 = a - QNBO;
            for (int b = 0; b < QNBO; ++b) w += T12[b + a2 * QNBO] * Y1s[b][threadIdx.x];
            for (int b = 0; b <= a2; ++b) w += T2[b + a2 * QNBO] * Y2s[b][threadIdx.x];
        }
        float h, lo;
        tf32_split(w, h, lo);
        Wt_hi[c * kpad + a] = h;
    }
}

// Row-major split copy of the panel reflectors: Vr_hi/lo[r * vr_ld + a] = V[K0 + r, a]
// for reflectors a = a_begin + 32 blockIdx.y + .. (zero for a >= nbo; lo skipped when
// Vr_lo is null), through 32 x 32 shared-memory transposes (reads coalesced along
// rows, writes along reflectors).  Grid (ceil(R/128), reflectors / 32), block (32, 8).
__global__ void k_qr_pack_vrm(const float *A, int64_t rows, int64_t ld, int64_t K0, int nbo, int vr_ld, int a_begin,
                              float *Vr_hi, float *Vr_lo) {
    __shared__ float tile[32][33];
    const int64_t R = rows - K0;
    const int a0 = a_begin + blockIdx.y * 32;
    for (int sub = 0; sub < 4; ++sub) {  // four 32-row tiles per block
        const int64_t r0 = (int64_t)blockIdx.x * 128 + sub * 32;
        if (r0 >= R) break;
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            const int a = a0 + yy;
            const int64_t r = r0 + threadIdx.x;
            tile[yy][threadIdx.x] = (a < nbo && r < R) ? vval(A, ld, K0, K0 + r, a) : 0.f;
        }
        __syncthreads();
        for (int yy = threadIdx.y; yy < 32; yy += 8) {
            const int64_t r = r0 + yy;
            if (r >= R) continue;
            float h, lo;
            tf32_split(tile[threadIdx.x][yy], h, lo);
            Vr_hi[r * vr_ld + a0 + threadIdx.x] = h;
            if (Vr_lo) Vr_lo[r * vr_ld + a0 + threadIdx.x] = lo;
        }
        __syncthreads();
    }
}

// --------------------------------- FP32 panels: CholeskyQR2 + reconstruction --
// A panel P (m x b, b <= 32, column-major in A) is factored in a constant
// number of passes instead of one launch per column:
//   G1 = P^T P, R1 = chol(G1), Q1 = P R1^{-1};  G2 = Q1^T Q1, R2 = chol(G2),
//   Q = Q1 R2^{-1}, R = R2 R1      (mixed-precision CholeskyQR2: the Grams are
//   accumulated in double-float from FP32 data, the b x b work is FP64),
// then Householder vectors are reconstructed from the orthonormal Q
// (Ballard, Demmel, Grigori, Jacquelin, Nguyen, Solomonik, "Reconstructing
// Householder vectors from tall-skinny QR", IPDPS 2014): the LU factorisation
// without pivoting of Q - [S; 0], with signs S_i = -sign of the running
// diagonal, gives V = L (unit lower), T = -U S L_1^{-T}, tau_i = T_ii and the
// Householder R = S R, stored in the LAPACK layout the rest of the QR uses.
// A Cholesky breakdown (a panel too ill-conditioned for the Gram) sets the
// status word to kCqrFail; the caller then refactors with the column kernels.
constexpr int kCqrFail = 100;
constexpr int CQB = 32;

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float p, float e) {
    const float s = hi + p;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += err + e;
}

// Partial Grams over row ranges in double-float: Gph/Gpl[blk][i*32 + j] (both
// triangles) = hi/lo of sum_r X[r,i] X[r,j], each product split exactly by FMA and
// added by TwoSum.  CTA of 512 threads: 14 row groups x 36 threads, one thread per
// 4 x 4 block of the upper triangle of 8 x 8 blocks; group g takes rows g, g + 14, ...
// of each 256-row chunk.  Chunks are staged in shared memory, double-buffered: the next
// chunk's loads are in flight (registers) while the current one is used, and one barrier
// per chunk separates the buffers.  The groups' sums are combined by a fixed tree.
constexpr int CQ_CHUNK = 256, CQ_GROUPS = 14, CQ_LD = CQB + 4;
constexpr size_t cq_gram_smem() { return sizeof(float) * 2 * CQ_CHUNK * CQ_LD; }
__global__ void __launch_bounds__(512) k_cqr_gram(const float *X, int64_t ld, int64_t m, int b, float *Gph,
                                                  float *Gpl) {
    extern __shared__ __align__(16) float cq_sm[];  // [2][CQ_CHUNK][CQ_LD], then the combine
    const int tid = threadIdx.x, g = tid / 36;
    int q = tid % 36, bi = 0;
    while (q >= 8 - bi) {
        q -= 8 - bi;
        ++bi;
    }
    const int bj = bi + q;
    const int blk = tid % 36;  // this thread's 4 x 4 block
    const int64_t per = (m + gridDim.x - 1) / gridDim.x;
    const int64_t lo_r = (int64_t)blockIdx.x * per, hi_r = min(m, lo_r + per);
    float h[16], l[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) h[u] = l[u] = 0.f;
    constexpr int PER = CQ_CHUNK * CQB / 512;
    float nx[PER];
    auto load_chunk = [&](int64_t r0) {
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e2 = tid + 512 * u, r = e2 % CQ_CHUNK, c = e2 / CQ_CHUNK;
            const int64_t rr = r0 + r;
            nx[u] = (rr < hi_r && c < b) ? X[rr + c * ld] : 0.f;
        }
    };
    auto store_chunk = [&](int buf) {
        float *Xs = cq_sm + buf * CQ_CHUNK * CQ_LD;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e2 = tid + 512 * u;
            Xs[(e2 % CQ_CHUNK) * CQ_LD + e2 / CQ_CHUNK] = nx[u];
        }
    };
    if (lo_r < hi_r) {
        load_chunk(lo_r);
        store_chunk(0);
    }
    __syncthreads();
    int buf = 0;
    for (int64_t r0 = lo_r; r0 < hi_r; r0 += CQ_CHUNK, buf ^= 1) {
        const bool more = r0 + CQ_CHUNK < hi_r;
        if (more) load_chunk(r0 + CQ_CHUNK);
        if (g < CQ_GROUPS) {
            const float *Xs = cq_sm + buf * CQ_CHUNK * CQ_LD;
            for (int r = g; r < CQ_CHUNK; r += CQ_GROUPS) {
                const float4 xi = *reinterpret_cast<const float4 *>(&Xs[r * CQ_LD + 4 * bi]);
                const float4 xj = *reinterpret_cast<const float4 *>(&Xs[r * CQ_LD + 4 * bj]);
                const float a[4] = {xi.x, xi.y, xi.z, xi.w}, c4[4] = {xj.x, xj.y, xj.z, xj.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float p = a[u] * c4[v];
                        two_sum_acc(h[u * 4 + v], l[u * 4 + v], p, fmaf(a[u], c4[v], -p));
                    }
            }
        }
        // the other buffer was last read in the previous chunk, before the barrier below it
        if (more) store_chunk(buf ^ 1);
        __syncthreads();
    }
    // combine the groups by a fixed tree: S[g][blk][16] hi and lo (in the chunk buffers)
    float *Sh = cq_sm, *Sl = cq_sm + CQ_GROUPS * 36 * 16;
    if (g < CQ_GROUPS)
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            Sh[(g * 36 + blk) * 16 + u] = h[u];
            Sl[(g * 36 + blk) * 16 + u] = l[u];
        }
    __syncthreads();
    for (int half = 8; half > 0; half >>= 1) {  // groups g and g + half, for g < half
        if (g < half && g + half < CQ_GROUPS)
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                float sh = Sh[(g * 36 + blk) * 16 + u], sl = Sl[(g * 36 + blk) * 16 + u];
                two_sum_acc(sh, sl, Sh[((g + half) * 36 + blk) * 16 + u], Sl[((g + half) * 36 + blk) * 16 + u]);
                Sh[(g * 36 + blk) * 16 + u] = sh;
                Sl[(g * 36 + blk) * 16 + u] = sl;
            }
        __syncthreads();
    }
    // group 0 holds the block's sums: entry (i, j) of the upper triangle is block
    // (i / 4, j / 4), element (i % 4, j % 4)
    for (int e2 = tid; e2 < CQB * CQB; e2 += 512) {
        const int i = e2 / CQB, j = e2 % CQB;
        const int ii = min(i, j), jj = max(i, j);
        const int pb = ii / 4, pq = jj / 4;
        const int k = pb * 8 - pb * (pb - 1) / 2 + (pq - pb);  // block index, row-major over the triangle
        const int u = (ii % 4) * 4 + jj % 4;
        Gph[(int64_t)blockIdx.x * CQB * CQB + e2] = Sh[k * 16 + u];
        Gpl[(int64_t)blockIdx.x * CQB * CQB + e2] = Sl[k * 16 + u];
    }
}

// G = the Gram partials summed in double-float: block b takes entries 32 b .. 32 b + 31;
// thread group g (32 of them) sums partials g, g + 32, ... of its entry, and the groups are
// combined by a fixed tree.  Grid CQB, block 1024.
__global__ void __launch_bounds__(1024) k_cqr_gram_sum(const float *Gph, const float *Gpl, int nparts, float *Gh,
                                                      float *Gl) {
    __shared__ float Sh[32][33], Sl[32][33];
    const int x = threadIdx.x % 32, g = threadIdx.x / 32, e = blockIdx.x * 32 + x;
    float h = 0.f, l = 0.f;
    for (int p = g; p < nparts; p += 32) two_sum_acc(h, l, Gph[(int64_t)p * CQB * CQB + e], Gpl[(int64_t)p * CQB * CQB + e]);
    Sh[g][x] = h;
    Sl[g][x] = l;
    __syncthreads();
    for (int st = 16; st > 0; st >>= 1) {
        if (g < st) {
            float a = Sh[g][x], c = Sl[g][x];
            two_sum_acc(a, c, Sh[g + st][x], Sl[g + st][x]);
            Sh[g][x] = a;
            Sl[g][x] = c;
        }
        __syncthreads();
    }
    if (g == 0) {
        Gh[e] = Sh[0][x];
        Gl[e] = Sl[0][x];
    }
}

// R = chol(G) upper (R = L^T of the double-float Cholesky G = L L^T) as FP64, row-major
// R[i * 32 + j], and Rinv = R^{-1} = (L^{-1})^T as FP32, column-major Rinv[i + j * 32].
// One block of 1024 threads.  Breakdown -> status kCqrFail.
__global__ void __launch_bounds__(1024) k_cqr_chol(const float *Gh, const float *Gl, int b, double *R, float *Rinv,
                                                   DevStatus *st) {
    __shared__ DfTile Ah, Al, Lh, Ll, Bh, Bl, Xh, Xl;
    __shared__ float rh[CQB], rl[CQB];
    __shared__ int bad;
    const int l = threadIdx.x % CQB, i = threadIdx.x / CQB;
    {
        const bool in = i < b && l < b && l <= i;
        Ah[i][l] = in ? Gh[i * CQB + l] : 0.f;
        Al[i][l] = in ? Gl[i * CQB + l] : 0.f;
    }
    if (threadIdx.x == 0) bad = status_bad(st) ? 1 : 0;
    __syncthreads();
    if (bad) return;
    int jb = 0;
    if (!df_chol_inv32(Ah, Al, Lh, Ll, Bh, Bl, Xh, Xl, rh, rl, b, &jb)) {
        if (threadIdx.x == 0) set_status(st, kCqrFail, 0);
        return;
    }
    const bool up = i <= l && l < b;
    R[i * CQB + l] = up ? (double)Lh[l][i] + (double)Ll[l][i] : 0.0;
    Rinv[i + l * CQB] = up ? Xh[l][i] : 0.f;
}

// dst[r, :] = src[r, :] Minv for rows r in [r_begin, m); Minv upper b x b (FP32,
// column-major).  One thread per row; src may equal dst (each row is read before written).
// With vcm (the reflector rows of a panel): the rows also go, rounded to TF32, to the
// update's packed copies, vcm column-major [32][m_pad] and vr row-major [m_pad][32]
// (columns past b and rows m .. m_pad - 1 zero); the row-major copy is transposed through
// shared memory so that each block writes its rows as one contiguous stretch.
__global__ void __launch_bounds__(256) k_cqr_rows(const float *src, int64_t lds, float *dst, int64_t ldd, int64_t m,
                                                 int b, const float *Minv, int64_t r_begin, float *vcm = nullptr,
                                                 float *vr = nullptr, int64_t m_pad = 0) {
    __shared__ __align__(16) float Mi[CQB * CQB];
    __shared__ float tile[256][CQB + 1];
    for (int e = threadIdx.x; e < CQB * CQB; e += blockDim.x) Mi[e] = Minv[e];
    __syncthreads();
    const int64_t r0 = r_begin + (int64_t)blockIdx.x * blockDim.x, r = r0 + threadIdx.x;
    const bool live = r < m;
    float x[CQB];
#pragma unroll
    for (int c = 0; c < CQB; ++c) x[c] = (live && c < b) ? src[r + c * lds] : 0.f;
#pragma unroll
    for (int c = 0; c < CQB; ++c) {
        float y = 0.f;
        if (c < b) {
            // y = sum over k <= c of x[k] Mi[k, c], in ascending k, with the column of Mi
            // read four entries at a time (shared-memory broadcasts)
#pragma unroll
            for (int k4 = 0; k4 < CQB; k4 += 4) {
                if (k4 <= c) {
                    const float4 mv = *reinterpret_cast<const float4 *>(&Mi[k4 + c * CQB]);
                    y += x[k4] * mv.x;
                    if (k4 + 1 <= c) y += x[k4 + 1] * mv.y;
                    if (k4 + 2 <= c) y += x[k4 + 2] * mv.z;
                    if (k4 + 3 <= c) y += x[k4 + 3] * mv.w;
                }
            }
            if (live) dst[r + c * ldd] = y;
        }
        if (vcm) {
            float h, lo;
            tf32_split(y, h, lo);
            if (r < m_pad) vcm[c * m_pad + r] = h;
            tile[threadIdx.x][c] = h;
        }
    }
    if (vcm) {
        __syncthreads();
        const int64_t nrow = m_pad - r0 < 256 ? m_pad - r0 : 256;
        float *out = vr + r0 * CQB;
        for (int64_t e = threadIdx.x; e < nrow * CQB; e += blockDim.x) out[e] = tile[e / CQB][e % CQB];
    }
}

// Reconstruction on the top b x b block of Q (column-major in Q, ld ldq):
// modified LU of Q1 - S, T = -U S L1^{-T}, Householder R = S (R2 R1); writes the
// panel's top block of A (R upper, L1 strictly lower), tau, and Uinv (FP32, upper,
// column-major) for the rows below.  One block of 1024 threads, thread (i, j) = entry
// (i, j); one barrier per step: every thread forms the step's pivot itself, and the
// multipliers and pivots go to arrays of their own while the update reads the unscaled
// column.  The LU and the triangular inverses run in FP32 (the precision of Q and of the
// reflectors they produce); R = R2 R1 is formed in FP64.
__global__ void __launch_bounds__(1024) k_cqr_recon(const float *Q, int64_t ldq, int b, const double *R1,
                                                    const double *R2, float *A, int64_t ld, int64_t k0, float *tau,
                                                    float *Uinv, float *Tout, float *vcm, float *vr) {
    __shared__ float Z[CQB][CQB + 1];   // Q1, then the LU's trailing matrix (U above the diagonal)
    __shared__ float Lm[CQB][CQB + 1];  // multipliers: L1 strictly below the diagonal
    __shared__ double Rs[CQB][CQB + 1];
    __shared__ float Bu[CQB][CQB + 1], Ui[CQB][CQB + 1];  // U^{-1}: work, result
    __shared__ float Bl[CQB][CQB + 1], Li[CQB][CQB + 1];  // L1^{-1}: work, result
    __shared__ float S[CQB], Ud[CQB];
    const int t = threadIdx.x, i = t / CQB, j = t % CQB;
    Z[i][j] = (i < b && j < b) ? Q[i + j * ldq] : 0.f;
    Lm[i][j] = 0.f;
    Bu[i][j] = Bl[i][j] = (i == j && i < b) ? 1.f : 0.f;
    Ui[i][j] = Li[i][j] = 0.f;
    // R = R2 R1 (both upper), or R1 alone after a single CholeskyQR pass (R2 null)
    {
        double sacc = 0.0;
        if (i < b && j < b && i <= j) {
            if (R2)
                for (int k = i; k <= j; ++k) sacc += R2[i * CQB + k] * R1[k * CQB + j];
            else
                sacc = R1[i * CQB + j];
        }
        Rs[i][j] = sacc;
    }
    __syncthreads();
    // modified LU: S_k = -sign(Z_kk), pivot Z_kk - S_k; multipliers Z_ik / pivot; update
    for (int k = 0; k < b; ++k) {
        const float zkk = Z[k][k];
        const float sk = zkk >= 0.f ? -1.f : 1.f;
        const float piv = zkk - sk;
        const float zr = 1.f / piv;
        if (t == 0) {
            S[k] = sk;
            Ud[k] = piv;
        }
        if (j == k && i > k && i < b) Lm[i][k] = Z[i][k] * zr;
        if (i > k && j > k && i < b && j < b) Z[i][j] -= (Z[i][k] * zr) * Z[k][j];
        __syncthreads();
    }
    // U^{-1} by rows from the bottom (X[r, :] = B[r, :] / U_rr; B[i, :] -= U_ir X[r, :] for
    // i < r), L1^{-1} by rows from the top (unit diagonal), both in one loop
    for (int q = 0; q < b; ++q) {
        const int r = b - 1 - q;  // row of U^{-1} finished at this step
        if (j >= r && i <= r) {
            const float x = Bu[r][j] / Ud[r];
            if (i == r) Ui[r][j] = x;
            else Bu[i][j] -= Z[i][r] * x;
        }
        if (j <= q && i >= q && i < b) {
            const float x = Bl[q][j];
            if (i == q) Li[q][j] = x;
            else Bl[i][j] -= Lm[i][q] * x;
        }
        __syncthreads();
    }
    if (i < b && j < b) {
        // T = -U S L1^{-T}: T_ij = -sum_k U_ik S_k (L1^{-1})_jk, upper triangular
        if (i <= j) {
            float tij = -Ud[i] * S[i] * Li[j][i];
            for (int k = i + 1; k < b; ++k) tij -= Z[i][k] * S[k] * Li[j][k];
            if (i == j) tau[k0 + i] = tij;
            if (Tout) Tout[i + j * QNBO] = tij;
        } else if (Tout) {
            Tout[i + j * QNBO] = 0.f;
        }
        // panel top block: Householder R = S R above/on the diagonal, L1 below
        const float v = (i <= j) ? (float)((double)S[i] * Rs[i][j]) : Lm[i][j];
        A[(k0 + i) + (k0 + j) * ld] = v;
        Uinv[i + j * CQB] = (i <= j) ? Ui[i][j] : 0.f;
    } else if (i < CQB && j < CQB) {
        Uinv[i + j * CQB] = 0.f;
    }
    // the reflectors' top rows in the update's packed copies (unit diagonal, zero above)
    if (vcm && i < b) {
        float h = 0.f, lo;
        if (j < b) tf32_split(i < j ? 0.f : (i == j ? 1.f : Lm[i][j]), h, lo);
        vcm[j * ldq + i] = h;
        vr[i * CQB + j] = h;
    }
}

// ------------------------------------------------------ triangular solves --
constexpr int TNB = 64;

// Inverses of the diagonal TNB x TNB blocks of the upper-triangular R (FP64,
// column-major per block: Dinv[b][r + c*TNB]).  One block of TNB threads per
// diagonal block, thread c computing column c by back substitution.  A zero or
// non-finite diagonal entry sets GAP_ERR_RANK.
template <class T>
__global__ void k_trsv_invert(const T *R, int64_t ld, int64_t M, double *Dinv, DevStatus *st) {
    __shared__ double Rs[TNB][TNB + 1];
    __shared__ double Xi[TNB][TNB + 1];
    const int64_t b0 = (int64_t)blockIdx.x * TNB;
    const int nb = (int)min((int64_t)TNB, M - b0);
    for (int e = threadIdx.x; e < TNB * TNB; e += blockDim.x) {
        const int r = e % TNB, c = e / TNB;
        Rs[r][c] = (r < nb && c < nb) ? (double)R[(b0 + r) + (b0 + c) * ld] : 0.0;
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c < nb) {
        for (int r = c; r >= 0; --r) {
            double v = (r == c) ? 1.0 : 0.0;
            for (int k = r + 1; k <= c; ++k) v -= Rs[r][k] * Xi[k][c];
            const double d = Rs[r][r];
            if (d == 0.0 || !isfinite(d)) {
                if (st) set_status(st, GAP_ERR_RANK, b0 + r);
                v = 0.0;
            } else {
                v /= d;
            }
            Xi[r][c] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TNB * TNB; e += blockDim.x) {
        const int r = e % TNB, cc = e / TNB;
        Dinv[(int64_t)blockIdx.x * TNB * TNB + e] = (r <= cc && r < nb && cc < nb) ? Xi[r][cc] : 0.0;
    }
}

// One block step of a blocked triangular solve with the inverted diagonal blocks.
// trans = 0 (R x = z, blocks last to first): xb = D_b z_b; z[0:b0] -= R[0:b0, blk] xb.
// trans = 1 (R^T x = z, blocks first to last): xb = D_b^T z_b; z[b1:M] -= R[blk, b1:M]^T xb.
// Every block recomputes xb (z_b is not written in this launch); block 0 stores it in xs.
template <class T>
__global__ void __launch_bounds__(256) k_trsv_step(const T *R, int64_t ld, int64_t M, const double *Dinv, int blk,
                                                  int trans, double *z, double *xs) {
    __shared__ double zb[TNB], xb[TNB];
    const int64_t b0 = (int64_t)blk * TNB;
    const int nb = (int)min((int64_t)TNB, M - b0);
    const double *D = Dinv + (int64_t)blk * TNB * TNB;
    if (threadIdx.x < TNB) zb[threadIdx.x] = threadIdx.x < nb ? z[b0 + threadIdx.x] : 0.0;
    __syncthreads();
    if (threadIdx.x < TNB) {
        const int r = threadIdx.x;
        double s = 0.0;
        if (trans == 0)
            for (int c = r; c < nb; ++c) s += D[r + c * TNB] * zb[c];
        else
            for (int c = 0; c <= r && c < nb; ++c) s += D[c + r * TNB] * zb[c];
        xb[r] = r < nb ? s : 0.0;
        if (blockIdx.x == 0 && r < nb) xs[b0 + r] = s;
    }
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (trans == 0) {
        if (t >= b0) return;
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s += (double)R[t + (b0 + j) * ld] * xb[j];
        z[t] -= s;
    } else {
        const int64_t i = b0 + nb + t;
        if (i >= M) return;
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s += (double)R[(b0 + j) + i * ld] * xb[j];
        z[i] -= s;
    }
}

// x_blk = R_blk^{-1} x_blk (trans = 0) or R_blk^{-T} x_blk (trans = 1), one block.
template <class T>
__global__ void k_trsv_diag(const T *R, int64_t ld, int64_t b0, int nb, int trans, double *x, DevStatus *st) {
    __shared__ double Rs[TNB][TNB + 1];
    __shared__ double xs[TNB];
    const int t = threadIdx.x;  // TNB threads
    for (int e = t; e < nb * nb; e += blockDim.x) {
        int r = e % nb, c = e / nb;
        Rs[r][c] = (double)R[(b0 + r) + (b0 + c) * ld];
    }
    if (t < nb) xs[t] = x[b0 + t];
    __syncthreads();
    if (trans == 0) {
        for (int j = nb - 1; j >= 0; --j) {
            if (t == 0) {
                double rjj = Rs[j][j];
                if (rjj == 0.0 || !isfinite(rjj)) {
                    if (st) set_status(st, GAP_ERR_RANK, b0 + j);
                    xs[j] = 0.0;
                } else {
                    xs[j] /= rjj;
                }
            }
            __syncthreads();
            if (t < j) xs[t] -= Rs[t][j] * xs[j];
            __syncthreads();
        }
    } else {
        for (int j = 0; j < nb; ++j) {
            if (t == 0) {
                double rjj = Rs[j][j];
                if (rjj == 0.0 || !isfinite(rjj)) {
                    if (st) set_status(st, GAP_ERR_RANK, b0 + j);
                    xs[j] = 0.0;
                } else {
                    xs[j] /= rjj;
                }
            }
            __syncthreads();
            if (t > j && t < nb) xs[t] -= Rs[j][t] * xs[j];
            __syncthreads();
        }
    }
    if (t < nb) x[b0 + t] = xs[t];
}

// trans = 0: x[0:b0] -= R[0:b0, b0:b0+nb] x_blk ; trans = 1: x[b1:M] -= R[b0:b1, b1:M]^T x_blk
template <class T>
__global__ void k_trsv_update(const T *R, int64_t ld, int64_t M, int64_t b0, int nb, int trans, double *x) {
    __shared__ double xs[TNB];
    if (threadIdx.x < nb) xs[threadIdx.x] = x[b0 + threadIdx.x];
    __syncthreads();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (trans == 0) {
        if (k >= b0) return;
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s += (double)R[k + (b0 + j) * ld] * xs[j];
        x[k] -= s;
    } else {
        int64_t i = b0 + nb + k;
        if (i >= M) return;
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s += (double)R[(b0 + j) + i * ld] * xs[j];
        x[i] -= s;
    }
}

template <class T>
__global__ void k_copy_to_f64(const T *src, int64_t n, double *dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

// ----------------------------------------------------------------- GEMVs --
// For the FP32 design matrix the sums run in double-float (an FP32 pair, ~48-bit):
// each product a*v is split into its rounded value and exact error (FMA) with the
// FP64 vector entry given as an FP32 pair, and added by TwoSum.  FP64 matrices use FP64.
__device__ __forceinline__ void df_acc(float &hi, float &lo, float a, float vh, float vl) {
    const float p = a * vh;
    const float e = fmaf(a, vh, -p) + a * vl;
    const float s = hi + p;
    const float bp = s - hi;
    lo += ((hi - (s - bp)) + (p - bp)) + e;
    hi = s;
}

__global__ void k_split_vec(const double *v, int64_t n, float *vh, float *vl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h = (float)v[i];
    vh[i] = h;
    vl[i] = (float)(v[i] - (double)h);
}

// t[i] = sum_k A[i + k ld] v[k] over rows; v staged through shared memory.
template <class T>
__global__ void __launch_bounds__(256) k_gemv_n(const T *A, int64_t rows, int64_t M, int64_t ld, const double *v,
                                               double *t) {
    __shared__ float vsh[1024], vsl[1024];
    __shared__ double vs[1024];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float hi = 0.f, lo = 0.f;
    double s = 0.0;
    for (int64_t k0 = 0; k0 < M; k0 += 1024) {
        const int nk = (int)min((int64_t)1024, M - k0);
        __syncthreads();
        for (int e = threadIdx.x; e < nk; e += blockDim.x) {
            const double x = v[k0 + e];
            vs[e] = x;
            vsh[e] = (float)x;
            vsl[e] = (float)(x - (double)(float)x);
        }
        __syncthreads();
        if (i < rows) {
            if (sizeof(T) == 4) {
                for (int k = 0; k < nk; ++k) df_acc(hi, lo, (float)A[i + (k0 + k) * ld], vsh[k], vsl[k]);
            } else {
                for (int k = 0; k < nk; ++k) s += (double)A[i + (k0 + k) * ld] * vs[k];
            }
        }
    }
    if (i < rows) t[i] = sizeof(T) == 4 ? (double)hi + (double)lo : s;
}

// g[k] = sum_i A[i + k ld] r[i]; one block per column, fixed-order block reduction.
// For FP32 matrices rh/rl is the FP32-pair split of r.
template <class T>
__global__ void __launch_bounds__(256) k_gemv_t(const T *A, int64_t rows, int64_t ld, const double *r, const float *rh,
                                               const float *rl, double *g) {
    __shared__ double red[256];
    const int64_t k = blockIdx.x;
    double s = 0.0;
    if (sizeof(T) == 4) {
        float hi = 0.f, lo = 0.f;
        for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) df_acc(hi, lo, (float)A[i + k * ld], rh[i], rl[i]);
        s = (double)hi + (double)lo;
    } else {
        for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) s += (double)A[i + k * ld] * r[i];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[k] = red[0];
}

__global__ void __launch_bounds__(1024) k_dot(const double *a, const double *b, int64_t n, double *out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * b[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_axpy(double sign, const double *num, const double *den, const double *x, double *y, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a = (*den != 0.0) ? sign * (*num / *den) : 0.0;
    y[i] += a * x[i];
}

__global__ void k_xpby(const double *x, const double *num, const double *den, double *p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double b = (*den != 0.0) ? *num / *den : 0.0;
    p[i] = x[i] + b * p[i];
}

__global__ void k_sub(const double *b, const double *t, double *r, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - t[i];
}

template <class T>
__global__ void k_read_rows(const T *A, int64_t ld, int64_t M, int64_t row0, int64_t nrows, double *dst) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nrows * M) return;
    int64_t r = e % nrows, c = e / nrows;
    dst[r * M + c] = (double)A[(row0 + r) + c * ld];
}

template <class T>
__global__ void k_read_r(const T *A, int64_t ld, int64_t M, double *dst) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * M) return;
    int64_t r = e % M, c = e / M;
    dst[r * M + c] = (r <= c) ? (double)A[r + c * ld] : 0.0;
}

// one thread per entry of the M x (M+1) block, rows fastest (coalesced in both matrices)
template <class T>
__global__ void k_tsqr_gather(const T *__restrict__ A, int64_t ld, int64_t r0, int64_t M, T *__restrict__ S,
                              int64_t lds, int64_t srow, int zero_b) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * (M + 1)) return;
    const int64_t i = e % M, j = e / M;
    const bool keep = j < M ? i <= j : !zero_b;
    S[(srow + i) + j * lds] = keep ? A[(r0 + i) + j * ld] : T(0);
}

}  // namespace

// ============================================================ launchers ==
cudaError_t launch_kmm(const Dims &dm, const double *Xs, const int32_t *sparse_sp, double *K, cudaStream_t s,
                       bool double_float, float *split_ws) {
    if (dm.M == 0) return cudaSuccess;
    dim3 grid((unsigned)ceil_div(dm.M, 64), (unsigned)ceil_div(dm.M, 64));
    if (double_float) {
        const int64_t n = dm.M * dm.d;
        float *Xh = split_ws, *Xl = split_ws + n;
        k_split_vec<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(Xs, n, Xh, Xl);
        k_kmm_df<<<grid, 256, 0, s>>>(dm, Xh, Xl, sparse_sp, K);
    } else {
        k_kmm<<<grid, 256, 0, s>>>(dm, Xs, sparse_sp, K);
    }
    return cudaGetLastError();
}

size_t cholesky_df_workspace_bytes(int64_t M) { return sizeof(float) * (2 * (size_t)M * (size_t)M + 2 * CNB * CNB); }

// The end of the diagonal block holding column k0 (ends: ascending block ends, the last
// M; none: one block).
static int64_t block_end(int64_t k0, int64_t M, const int64_t *ends, int n_ends) {
    for (int b = 0; b < n_ends; ++b)
        if (ends[b] > k0) return std::min(ends[b], M);
    return M;
}

cudaError_t cholesky_lower_df(double *K, int64_t M, float *ws, DevStatus *st, cudaStream_t s, const int64_t *ends,
                              int n_ends) {
    if (M == 0) return cudaSuccess;
    float *Kh = ws, *Kl = Kh + M * M, *Xh = Kl + M * M, *Xl = Xh + CNB * CNB;
    const dim3 tri((unsigned)ceil_div(M, 256), (unsigned)M);
    k_split_lower<<<tri, 256, 0, s>>>(K, M, Kh, Kl);
    for (int64_t k0 = 0; k0 < M;) {
        // a block-diagonal K_MM (sparse points of different species, or of the two-body
        // block, do not covary) is factored block by block: the trailing updates stop at the
        // block's end, and the panels do not cross it
        const int64_t end = block_end(k0, M, ends, n_ends);
        const int kb = (int)min((int64_t)CNB, end - k0);
        k_potrf_diag_df<<<1, CNB * CNB, 0, s>>>(Kh, Kl, M, k0, kb, Xh, Xl, st);
        const int64_t rest = end - k0 - kb;
        if (rest > 0) {
            k_trsm_panel_df<<<(unsigned)ceil_div(rest, TRS_ROWS), TRS_ROWS * TRS_GROUPS, 0, s>>>(Kh, Kl, M, k0, kb, end,
                                                                                             Xh, Xl, st);
            const int64_t nbk = ceil_div(rest, 64);
            k_syrk_lower_df<<<(unsigned)(nbk * (nbk + 1) / 2), 256, 0, s>>>(Kh, Kl, M, k0, kb, end, st);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k0 += kb;
    }
    k_merge_lower<<<tri, 256, 0, s>>>(K, M, Kh, Kl);
    return cudaGetLastError();
}

cudaError_t cholesky_lower(double *K, int64_t M, DevStatus *st, cudaStream_t s, const int64_t *ends, int n_ends) {
    for (int64_t k0 = 0; k0 < M;) {
        const int64_t end = block_end(k0, M, ends, n_ends);
        int kb = (int)min((int64_t)CNB, end - k0);
        k_potrf_diag<<<1, CNB * CNB, 0, s>>>(K, M, k0, kb, st);
        int64_t rest = end - k0 - kb;
        if (rest > 0) {
            k_trsm_panel<<<(unsigned)ceil_div(rest, 128), 128, 0, s>>>(K, M, k0, kb, end, st);
            unsigned nbk = (unsigned)ceil_div(rest, 64);
            k_syrk_lower<<<dim3(nbk, nbk), 256, 0, s>>>(K, M, k0, kb, end, st);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k0 += kb;
    }
    return cudaSuccess;
}

template <class T>
cudaError_t launch_stack_u(const Dims &dm, const double *L, T *A, cudaStream_t s, bool blocked) {
    if (dm.M == 0) return cudaSuccess;
    dim3 grid((unsigned)ceil_div(dm.M, 32), (unsigned)ceil_div(dm.M, 32));
    k_stack_u<T><<<grid, dim3(32, 8), 0, s>>>(dm, L, A, blocked ? 1 : 0);
    return cudaGetLastError();
}

namespace {
// Panel [k0, k1) by column kernels (one launch per column).
template <class T>
cudaError_t qr_panel(T *A, int64_t rows, int64_t ld, int64_t k0, int64_t k1, T *tau, T *part, T *diagrow,
                     cudaStream_t s) {
    const int ncol_blocks = 304;  // 2 blocks per SM for the column kernels
    T *diag_a = diagrow, *diag_b = diagrow + (QNB + 1);
    T *part_a = part, *part_b = part + (int64_t)ncol_blocks * (QNB + 1);
    k_qr_col_init<T><<<ncol_blocks, QTHREADS, 0, s>>>(A, rows, ld, k0, k1, part_a, diag_a);
    for (int64_t j = k0; j < k1; ++j) {
        k_qr_col_step<T><<<ncol_blocks, QTHREADS, 0, s>>>(A, rows, ld, k0, k1, j, tau, part_a, part_b, diag_a, diag_b);
        T *t1 = part_a; part_a = part_b; part_b = t1;
        T *t2 = diag_a; diag_a = diag_b; diag_b = t2;
    }
    return cudaGetLastError();
}

// Row splits of a split-K product Y = V^T C over n_ct column tiles (at most cap): the
// persistent grid runs split x column tiles, so they should fill its last wave.  Of one
// to four waves, the split count whose tiles leave the fewest CTAs idle (fewer waves on a
// near tie).
int wave_splits(int64_t n_ct, int64_t cap) {
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    n_sm = std::max(n_sm, 1);
    int best = 1;
    double best_e = -1.0;
    for (int w = 1; w <= 4; ++w) {
        const int64_t sp = std::min<int64_t>((int64_t)w * n_sm / std::max<int64_t>(n_ct, 1), cap);
        if (sp < 1) continue;
        const int64_t tiles = sp * n_ct;
        const double e = (double)tiles / (double)(ceil_div(tiles, n_sm) * n_sm);
        if (e > best_e + 0.02) {
            best_e = e;
            best = (int)sp;
        }
    }
    return best;
}

// Compact-WY application of the reflectors of panel [k0, k1) to columns [k1, k1 + nt).
template <class T>
cudaError_t qr_apply(T *A, int64_t rows, int64_t ld, int64_t k0, int64_t k1, int64_t nt, T *tau, T *Tbuf, T *part,
                     T *Wpart, T *Wred, int n_row_blocks, int64_t wpart_cols, cudaStream_t s) {
    const int kb = (int)(k1 - k0);
    if (nt > 0) {
        // narrow updates get more row blocks (at least ~4 blocks per SM), within the
        // capacity of the partial buffer (n_row_blocks x QNB x wpart_cols)
        {
            constexpr int QBN0 = sizeof(T) == 4 ? 512 : 256;
            const int64_t col_tiles = ceil_div(nt, QBN0);
            int64_t want = std::max<int64_t>(n_row_blocks, ceil_div(608, col_tiles));
            want = std::min<int64_t>(want, 512);
            want = std::min<int64_t>(want, (int64_t)n_row_blocks * wpart_cols / nt);
            n_row_blocks = (int)std::max<int64_t>(1, want);
        }
        const int nvtv = 152;
        k_qr_vtv<T><<<nvtv, 256, 0, s>>>(A, rows, ld, k0, kb, part);
        k_qr_tfactor<T><<<1, 256, 0, s>>>(part, nvtv, tau, k0, kb, Tbuf);
        constexpr int QBN = sizeof(T) == 4 ? 512 : 256;
        const size_t sm1 = sizeof(T) * (16 * (QNB + 1) + 16 * (QBN + 1)), sm2 = sizeof(T) * 2 * QNB * 128;
        dim3 g1((unsigned)ceil_div(nt, QBN), (unsigned)n_row_blocks);
        k_qr_vtc2<T><<<g1, 256, sm1, s>>>(A, rows, ld, k0, kb, k1, nt, Wpart);
        k_qr_wreduce<T><<<(unsigned)ceil_div(nt, 32), dim3(32, QNB), 0, s>>>(Wpart, n_row_blocks, Tbuf, kb, nt, Wred);
        dim3 g2((unsigned)ceil_div(rows - k0, 128), (unsigned)ceil_div(nt, 128));
        k_qr_update2<T><<<g2, 256, sm2, s>>>(A, rows, ld, k0, kb, k1, nt, Wred);
    }
    return cudaGetLastError();
}

// The kernels' shared-memory limits, raised once per process (the values are constants;
// a per-call attribute change would take the driver's lock on every launch of every lane).
template <class T>
void qr_set_smem_attrs() {
    constexpr int QBN = sizeof(T) == 4 ? 512 : 256;
    static const bool once = [] {
        cudaFuncSetAttribute(k_qr_vtc2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(T) * (16 * (QNB + 1) + 16 * (QBN + 1))));
        cudaFuncSetAttribute(k_qr_update2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(T) * 2 * QNB * 128));
        return true;
    }();
    (void)once;
}
}  // namespace

// FP32 panel [k0, k1) by CholeskyQR2 + Householder reconstruction (see above).
// ws: cqr_workspace_bytes(rows) bytes.
cudaError_t qr_panel_cqr(float *A, int64_t rows, int64_t ld, int64_t k0, int64_t k1, float *tau, void *ws,
                         DevStatus *st, cudaStream_t s, float *Tout, int cqr_passes, float *vcm = nullptr,
                         float *vr = nullptr) {
    const int b = (int)(k1 - k0);
    const int64_t m = rows - k0;
    const int nparts = 152;  // Gram partials (one CTA each)
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    unsigned char *w = (unsigned char *)ws;
    float *Gph = (float *)w, *Gpl = Gph + (size_t)nparts * CQB * CQB;
    w += al(sizeof(double) * nparts * CQB * CQB);
    double *R1 = (double *)w;
    w += al(sizeof(double) * CQB * CQB);
    double *R2 = (double *)w;
    w += al(sizeof(double) * CQB * CQB);
    float *M1 = (float *)w;
    w += al(sizeof(float) * CQB * CQB);
    float *M2 = (float *)w;
    w += al(sizeof(float) * CQB * CQB);
    float *Uinv = (float *)w;
    w += al(sizeof(float) * CQB * CQB);
    float *Gh = (float *)w, *Gl = Gh + CQB * CQB;  // the summed Gram
    w += al(sizeof(double) * CQB * CQB);
    float *Qb = (float *)w;  // [m x b] column-major, ld = ldq
    const int64_t ldq = round_up(m, 32);
    float *P = A + k0 + k0 * ld;
    const unsigned rb = (unsigned)ceil_div(m, 256);
    static const cudaError_t gram_attr =
        cudaFuncSetAttribute(k_cqr_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cq_gram_smem());
    if (gram_attr != cudaSuccess) return gram_attr;
    k_cqr_gram<<<nparts, 512, cq_gram_smem(), s>>>(P, ld, m, b, Gph, Gpl);
    k_cqr_gram_sum<<<CQB, 1024, 0, s>>>(Gph, Gpl, nparts, Gh, Gl);
    k_cqr_chol<<<1, 1024, 0, s>>>(Gh, Gl, b, R1, M1, st);
    k_cqr_rows<<<rb, 256, 0, s>>>(P, ld, Qb, ldq, m, b, M1, 0);
    if (cqr_passes > 1) {
        // second pass: Q1 is orthonormal to about kappa^2 times the Gram's precision; one more
        // Gram / Cholesky / row pass brings it to working precision (R = R2 R1)
        k_cqr_gram<<<nparts, 512, cq_gram_smem(), s>>>(Qb, ldq, m, b, Gph, Gpl);
        k_cqr_gram_sum<<<CQB, 1024, 0, s>>>(Gph, Gpl, nparts, Gh, Gl);
        k_cqr_chol<<<1, 1024, 0, s>>>(Gh, Gl, b, R2, M2, st);
        k_cqr_rows<<<rb, 256, 0, s>>>(Qb, ldq, Qb, ldq, m, b, M2, 0);
    }
    // with vcm / vr: the reflectors also go to the packed copies of the panel's update
    // (TF32, column-major with leading dimension ldq and row-major with 32 columns)
    k_cqr_recon<<<1, 1024, 0, s>>>(Qb, ldq, b, R1, cqr_passes > 1 ? R2 : nullptr, A, ld, k0, tau, Uinv, Tout, vcm,
                                   vr);
    const int64_t r_end = vcm ? ldq : m;
    if (r_end > b)
        k_cqr_rows<<<(unsigned)ceil_div(r_end - b, 256), 256, 0, s>>>(Qb, ldq, P, ld, m, b, Uinv, b, vcm, vr, ldq);
    return cudaGetLastError();
}

// C[k0:, c0:c0+nt] -= V T^T V^T C for the reflectors in columns [k0, k0+nbo) of A
// (Tm column-major with stride QNBO), both products on the tensor cores.
cudaError_t qr_update_tc(float *A, int64_t rows, int64_t ld, int64_t k0, int nbo, int64_t c0, int64_t nt,
                         float *Tm, bool form_T, const float *tau, float *G, float *Yp, int64_t yp_cap, void *vcm,
                         float *Wt_hi, float *Wt_lo, float *Vr_hi, float *Vr_lo, int passes, int *status,
                         cudaStream_t s, int vr_ld = 0, bool prepacked = false) {
    const int64_t R = rows - k0;
    // row splits of Y = V^T C (128-column tiles), within the partials' capacity
    auto splits = [&](int64_t ncols) { return wave_splits(ceil_div(ncols, 128), yp_cap / (QNBO * ncols)); };
    // one pass: only the TF32 hi slice of the nbo live reflectors is packed (K = kpad), and
    // the Gram of an outer panel is formed from it in one plain-TF32 pass too; three
    // passes: hi, lo and unsplit copies of all QNBO
    const bool lean = passes == 1;
    const int kpad = lean ? (int)round_up(nbo, 32) : QNBO;
    // prepacked (one pass, a CholeskyQR inner panel): the panel kernels already wrote both
    // copies of its reflectors (column-major in vcm, row-major in Vr_hi with 32 columns)
    prepacked = prepacked && lean && kpad == 32;
    const float *Vf = prepacked ? nullptr : tc_qr_pack_v(A, ld, k0, nbo, R, vcm, lean ? kpad : QNBO, !lean, s);
    int n_split = 0;
    cudaError_t e;
    if (form_T) {
        // G = V^T V on the tensor cores (C = the reflector copy itself, column-major with
        // leading dimension round_up(R, 32)), then T
        if (lean)
            e = tc_qr_y_tma((const float *)vcm, round_up(R, 32), 0, R, 0, kpad, splits(kpad), vcm, kpad, Yp, status, s,
                            &n_split);
        else
            e = tc_qr_y(Vf, round_up(R, 32), 0, R, 0, QNBO, splits(QNBO), vcm, Yp, status, s, &n_split);
        if (e != cudaSuccess) return e;
        k_qr_gram_reduce<<<QNBO * QNBO / 256, 256, 0, s>>>(Yp, n_split, lean ? kpad : QNBO, G);
        k_qr_tfactor_big<<<1, 512, sizeof(float) * 2 * QNBO * (QNBO + 1), s>>>(G, tau, k0, nbo, Tm);
    }
    // Y = V^T C: split-TF32 (three passes) or plain TF32 with C fetched by TMA (one pass)
    e = passes == 1 ? tc_qr_y_tma(A, ld, k0, R, c0, nt, splits(nt), vcm, lean ? kpad : QNBO, Yp, status, s, &n_split)
                    : tc_qr_y(A, ld, k0, R, c0, nt, splits(nt), vcm, Yp, status, s, &n_split);
    if (e != cudaSuccess) return e;
    float *wlo = passes == 1 ? nullptr : Wt_lo, *vlo = passes == 1 ? nullptr : Vr_lo;
    k_qr_w2t<<<(unsigned)ceil_div(nt, 32), dim3(32, 32), 0, s>>>(Yp, n_split, Tm, nbo, nt, kpad, Wt_hi, wlo);
    if (vr_ld <= 0 || passes != 1) vr_ld = kpad;
    if (!prepacked)
        k_qr_pack_vrm<<<dim3((unsigned)ceil_div(R, 128), kpad / 32), dim3(32, 8), 0, s>>>(A, rows, ld, k0, nbo, vr_ld,
                                                                                        0, Vr_hi, vlo);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return tc_qr_update(A, ld, k0, R, c0, nt, Vr_hi, Vr_lo, Wt_hi, Wt_lo, kpad, passes, status, s, vr_ld);
}

// C[K0:, c0:c0+nt] -= V T^T V^T C for the 128 + nb2 reflectors of a pair of outer panels
// (columns [K0, K0+128) and [K0+128, K0+128+nb2) of A), one plain-TF32 pass: the columns
// of C are read and rewritten once for both panels.  T1 (of the first panel) is given,
// and so are V1's copies, packed by the first panel's update of the second: column-major
// in the first slot of vcm, row-major in columns 0..127 of Vr_hi (row stride
// 128 + round_up(nb2, 32)).  T2 and T12 = -T1 V1^T V2 T2 are formed here.  Vr_hi holds
// rows x 256 and Wt_hi (M+1) x 256 floats.
cudaError_t qr_update_tc_pair(float *A, int64_t rows, int64_t ld, int64_t K0, int nb2, int64_t c0, int64_t nt,
                              const float *T1, float *T2, float *T12, const float *tau, float *G, float *Yp,
                              int64_t yp_cap, void *vcm, float *Wt_hi, float *Vr_hi, int *status, cudaStream_t s) {
    const int64_t R = rows - K0, R_pad = round_up(R, 32);
    const int kpad2 = (int)round_up(nb2, 32), kpad = QNBO + kpad2;
    float *v1 = (float *)vcm, *v2 = v1 + (size_t)QNBO * R_pad;  // the hi slots of the two panels
    // row splits of the Gram products (128-column tiles) and of the pair's Y (256-column
    // tiles), within the partials' capacity
    auto splits = [&](int64_t ncols, int64_t cap) { return wave_splits(ceil_div(ncols, 128), cap / (QNBO * ncols)); };
    auto splits256 = [&](int64_t ncols, int64_t cap) {
        return wave_splits(ceil_div(ncols, 256), cap / (QNBO * ncols));
    };
    tc_qr_pack_v(A, ld, K0, nb2, R, v2, kpad2, false, s, QNBO);
    int ns = 0;
    // T2 from G22 = V2^T V2
    cudaError_t e = tc_qr_y_tma(v2, R_pad, 0, R, 0, kpad2, splits(kpad2, yp_cap), v2, kpad2, Yp, status, s, &ns);
    if (e != cudaSuccess) return e;
    k_qr_gram_reduce<<<QNBO * QNBO / 256, 256, 0, s>>>(Yp, ns, kpad2, G);
    k_qr_tfactor_big<<<1, 512, sizeof(float) * 2 * QNBO * (QNBO + 1), s>>>(G, tau, K0 + QNBO, nb2, T2);
    // G12 = V1^T V2, then T12
    e = tc_qr_y_tma(v2, R_pad, 0, R, 0, kpad2, splits(kpad2, yp_cap), v1, QNBO, Yp, status, s, &ns);
    if (e != cudaSuccess) return e;
    k_qr_gram_reduce<<<QNBO * QNBO / 256, 256, 0, s>>>(Yp, ns, kpad2, G);
    k_qr_t12<<<(unsigned)nb2, QNBO, 0, s>>>(G, T1, T2, nb2, T12);
    // Y1 = V1^T C and Y2 = V2^T C in one pass over C: Yp[split][256][nt]
    e = tc_qr_y2_tma(A, ld, K0, R, c0, nt, splits256(nt, yp_cap / 2), v1, v2, kpad2, Yp, status, s, &ns);
    if (e != cudaSuccess) return e;
    k_qr_w2t_pair<<<(unsigned)ceil_div(nt, 32), dim3(32, 32), 0, s>>>(Yp, ns, Yp + QNBO * nt, ns, 2 * QNBO * nt, T1,
                                                                      T12, T2, nb2, nt, kpad, Wt_hi);
    k_qr_pack_vrm<<<dim3((unsigned)ceil_div(R, 128), kpad2 / 32), dim3(32, 8), 0, s>>>(A, rows, ld, K0, QNBO + nb2,
                                                                                     kpad, QNBO, Vr_hi, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return tc_qr_update(A, ld, K0, R, c0, nt, Vr_hi, nullptr, Wt_hi, nullptr, kpad, 1, status, s);
}

size_t cqr_workspace_bytes(int64_t rows) {
    return 9 * 256 + sizeof(double) * (304 + 3) * CQB * CQB + sizeof(float) * 3 * CQB * CQB +
           sizeof(float) * (size_t)round_up(rows, 32) * CQB;
}

size_t qr_outer_workspace_bytes(int64_t rows, int64_t M) {
    const int n_rb = 64;
    return sizeof(float) * (5 * QNBO * QNBO + (size_t)n_rb * QNBO * (M + 1) + 2 * (size_t)rows * QNBO +
                            (size_t)rows * QNB + 2 * (size_t)(M + 1) * QNBO) + 12 * 256 +
           tc_qr_y_workspace_bytes(rows) + cqr_workspace_bytes(rows);
}

template <class T>
cudaError_t householder_qr(T *A, int64_t rows, int64_t M, int64_t ld, int nb, T *tau, T *Tbuf, T *part, T *diagrow,
                           T *Wpart, T *Wred, int n_row_blocks, cudaStream_t s, Prof *prof, void *outer_ws,
                           int *status, int upd_passes, int cqr_passes) {
    if (nb > QNB) nb = QNB;
    qr_set_smem_attrs<T>();
    const int64_t ncols = M + 1;  // last column: right-hand side
    if (sizeof(T) == 8 || outer_ws == nullptr) {
        // flat blocked Householder: panels of nb, each applied to all trailing columns
        for (int64_t k0 = 0; k0 < M; k0 += nb) {
            const int64_t k1 = min(M, k0 + nb), nt = ncols - k1;
            if (prof) prof->begin(GAP_PROF_QR_PANEL);
            cudaError_t e = qr_panel<T>(A, rows, ld, k0, k1, tau, part, diagrow, s);
            if (prof) prof->end();
            if (e != cudaSuccess) return e;
            if (nt > 0) {
                if (prof) prof->begin(GAP_PROF_QR_UPDATE);
                e = qr_apply<T>(A, rows, ld, k0, k1, nt, tau, Tbuf, part, Wpart, Wred, n_row_blocks, M + 1, s);
                if (prof) prof->end();
                if (e != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    } else {
        return householder_qr_two_level((float *)A, rows, M, ld, nb, (float *)tau, (float *)Tbuf, (float *)part,
                                        (float *)diagrow, (float *)Wpart, (float *)Wred, n_row_blocks, s, prof,
                                        outer_ws, status, upd_passes, cqr_passes);
    }
}

cudaError_t householder_qr_two_level(float *A, int64_t rows, int64_t M, int64_t ld, int nb, float *tau, float *Tbuf,
                                     float *part, float *diagrow, float *Wpart, float *Wred, int n_row_blocks,
                                     cudaStream_t s, Prof *prof, void *outer_ws, int *status, int upd_passes,
                                     int cqr_passes) {
    const int n_rb = 64;
    const int64_t ncols = M + 1;
    // outer workspace carve-up
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    unsigned char *w = (unsigned char *)outer_ws;
    float *G = (float *)w;
    w += al(sizeof(float) * QNBO * QNBO);
    float *To = (float *)w;
    w += al(sizeof(float) * QNBO * QNBO);
    float *Yp = (float *)w;
    w += al(sizeof(float) * (size_t)n_rb * QNBO * ncols);
    float *Vr_hi = (float *)w;
    w += al(sizeof(float) * (size_t)rows * QNBO);
    float *Vr_lo = (float *)w;
    w += al(sizeof(float) * (size_t)rows * QNBO);
    float *Wt_hi = (float *)w;
    w += al(sizeof(float) * (size_t)ncols * QNBO);
    float *Wt_lo = (float *)w;
    w += al(sizeof(float) * (size_t)ncols * QNBO);
    float *T1 = (float *)w;  // pairs of outer panels: T of the first, of the second, and T12
    w += al(sizeof(float) * QNBO * QNBO);
    float *T2 = (float *)w;
    w += al(sizeof(float) * QNBO * QNBO);
    float *T12 = (float *)w;
    w += al(sizeof(float) * QNBO * QNBO);
    float *Vr_in = (float *)w;  // row-major reflectors of the inner updates (one-pass pairs)
    w += al(sizeof(float) * (size_t)rows * QNB);
    void *vcm = (void *)w;  // column-major split copy of the outer-panel reflectors
    w += al(tc_qr_y_workspace_bytes(rows));
    void *cqr_ws = (void *)w;  // CholeskyQR2 panel workspace
    const int64_t yp_cap = (int64_t)n_rb * QNBO * ncols;  // capacity of Yp in floats
    static const cudaError_t tf_attr = cudaFuncSetAttribute(k_qr_tfactor_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                            (int)(sizeof(float) * 2 * QNBO * (QNBO + 1)));
    if (tf_attr != cudaSuccess) return tf_attr;
    // With one-pass updates, the inner updates pack their reflectors into the third slot of
    // vcm (unused then), so that the first slot keeps a pair's V1 from its mid-level update
    // to the pair's update.
    const bool pairs = upd_passes == 1;
    void *vcm_inner = pairs ? (void *)((float *)vcm + 2 * (size_t)QNBO * (size_t)round_up(rows, 32)) : vcm;
    // inner panels of nb over [K0, K1), their updates confined to [K0, K1)
    auto factor_outer = [&](int64_t K0, int64_t K1) -> cudaError_t {
        if (prof) prof->begin(GAP_PROF_QR_PANEL);
        for (int64_t k0 = K0; k0 < K1; k0 += nb) {
            const int64_t k1 = min(K1, k0 + nb);
            const bool cqr = rows - k0 >= 4 * CQB && k1 - k0 <= CQB;
            const int64_t nti = K1 - k1;
            // one pass: a CholeskyQR panel with an update to follow writes the update's packed
            // reflector copies itself
            const bool prepack = pairs && cqr && nti > 0;
            cudaError_t e = cqr ? qr_panel_cqr(A, rows, ld, k0, k1, tau, cqr_ws, (DevStatus *)status, s, To, cqr_passes,
                                               prepack ? (float *)vcm_inner : nullptr, prepack ? Vr_in : nullptr)
                                : qr_panel<float>(A, rows, ld, k0, k1, tau, part, diagrow, s);
            if (e != cudaSuccess) return e;
            if (nti <= 0) continue;
            if (cqr) {
                // inner update of the rest of the outer panel on the tensor cores, with the
                // compact-WY T the reconstruction produced (reflectors zero-padded to 128)
                e = qr_update_tc(A, rows, ld, k0, (int)(k1 - k0), k1, nti, To, false, tau, G, Yp, yp_cap, vcm_inner,
                                 Wt_hi, Wt_lo, pairs ? Vr_in : Vr_hi, Vr_lo, upd_passes, status, s, 0, prepack);
            } else {
                e = qr_apply<float>(A, rows, ld, k0, k1, nti, tau, Tbuf, part, Wpart, Wred, n_row_blocks, M + 1, s);
            }
            if (e != cudaSuccess) return e;
        }
        if (prof) prof->end();
        return cudaSuccess;
    };
    // With one-pass updates, outer panels go in pairs: the first panel's reflectors are
    // applied to the second panel's columns only, and the trailing columns receive both
    // panels' 256 reflectors in one update (their columns read and rewritten once).  The
    // lo halves of Vr and Wt, unused in one pass, extend their hi halves to 256 columns.
    for (int64_t K0 = 0; K0 < M;) {
        const int64_t K1 = min(M, K0 + QNBO);
        const int nbo = (int)(K1 - K0);
        cudaError_t e = factor_outer(K0, K1);
        if (e != cudaSuccess) return e;
        if (pairs && nbo == QNBO && K1 < M) {
            const int64_t K2 = min(M, K1 + QNBO);
            const int nb2 = (int)(K2 - K1);
            if (prof) prof->begin(GAP_PROF_QR_UPDATE);
            // V1's row-major copy goes straight into the pair's 256-wide layout
            e = qr_update_tc(A, rows, ld, K0, nbo, K1, nb2, T1, true, tau, G, Yp, yp_cap, vcm, Wt_hi, Wt_lo, Vr_hi,
                             Vr_lo, upd_passes, status, s, QNBO + (int)round_up(nb2, 32));
            if (prof) prof->end();
            if (e != cudaSuccess) return e;
            if ((e = factor_outer(K1, K2)) != cudaSuccess) return e;
            const int64_t nt = ncols - K2;
            if (nt > 0) {
                if (prof) prof->begin(GAP_PROF_QR_UPDATE);
                e = qr_update_tc_pair(A, rows, ld, K0, nb2, K2, nt, T1, T2, T12, tau, G, Yp, yp_cap, vcm, Wt_hi, Vr_hi,
                                      status, s);
                if (prof) prof->end();
                if (e != cudaSuccess) return e;
            }
            K0 = K2;
            continue;
        }
        const int64_t nt = ncols - K1;
        if (nt > 0) {
            if (prof) prof->begin(GAP_PROF_QR_UPDATE);
            e = qr_update_tc(A, rows, ld, K0, nbo, K1, nt, To, true, tau, G, Yp, yp_cap, vcm, Wt_hi, Wt_lo, Vr_hi,
                             Vr_lo, upd_passes, status, s);
            if (prof) prof->end();
            if (e != cudaSuccess) return e;
        }
        K0 = K1;
    }
    return cudaSuccess;
}

template <class T>
cudaError_t trsv_invert_blocks(const T *R, int64_t M, int64_t ld, double *Dinv, DevStatus *st, cudaStream_t s) {
    k_trsv_invert<T><<<(unsigned)ceil_div(M, TNB), TNB, 0, s>>>(R, ld, M, Dinv, st);
    return cudaGetLastError();
}

template <class T>
cudaError_t trsv_upper(const T *R, int64_t M, int64_t ld, int trans, double *x, const double *Dinv, double *work,
                       cudaStream_t s) {
    const int nblk = (int)ceil_div(M, TNB);
    for (int q = 0; q < nblk; ++q) {
        const int blk = trans == 0 ? nblk - 1 - q : q;
        const int64_t b0 = (int64_t)blk * TNB, nb = min((int64_t)TNB, M - b0);
        const int64_t rest = trans == 0 ? b0 : M - b0 - nb;
        k_trsv_step<T><<<(unsigned)std::max<int64_t>(1, ceil_div(rest, 256)), 256, 0, s>>>(R, ld, M, Dinv, blk, trans,
                                                                                           x, work);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(x, work, sizeof(double) * M, cudaMemcpyDeviceToDevice, s);
}

template <class T>
cudaError_t back_substitution(const T *A, int64_t M, int64_t ld, const T *z, double *c, double *work, DevStatus *st,
                              cudaStream_t s) {
    // work: Dinv (ceil(M/TNB) TNB^2 doubles) followed by M doubles
    double *Dinv = work, *xs = work + ceil_div(M, TNB) * TNB * TNB;
    k_copy_to_f64<T><<<(unsigned)ceil_div(M, 256), 256, 0, s>>>(z, M, c);
    cudaError_t e = trsv_invert_blocks<T>(A, M, ld, Dinv, st, s);
    if (e != cudaSuccess) return e;
    return trsv_upper<T>(A, M, ld, 0, c, Dinv, xs, s);
}

template <class T>
cudaError_t gemv_n(const T *A, int64_t rows, int64_t M, int64_t ld, const double *v, double *t, cudaStream_t s) {
    k_gemv_n<T><<<(unsigned)ceil_div(rows, 256), 256, 0, s>>>(A, rows, M, ld, v, t);
    return cudaGetLastError();
}

template <class T>
cudaError_t gemv_t(const T *A, int64_t rows, int64_t M, int64_t ld, const double *r, double *g, float *rsplit,
                   cudaStream_t s) {
    float *rh = rsplit, *rl = rsplit ? rsplit + rows : nullptr;
    if (sizeof(T) == 4) k_split_vec<<<(unsigned)ceil_div(rows, 256), 256, 0, s>>>(r, rows, rh, rl);
    k_gemv_t<T><<<(unsigned)M, 256, 0, s>>>(A, rows, ld, r, rh, rl, g);
    return cudaGetLastError();
}

cudaError_t vec_dot(const double *a, const double *b, int64_t n, double *out, cudaStream_t s) {
    k_dot<<<1, 1024, 0, s>>>(a, b, n, out);
    return cudaGetLastError();
}
cudaError_t vec_axpy(double sign, const double *num, const double *den, const double *x, double *y, int64_t n,
                     cudaStream_t s) {
    k_axpy<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(sign, num, den, x, y, n);
    return cudaGetLastError();
}
cudaError_t vec_xpby(const double *x, const double *num, const double *den, double *p, int64_t n, cudaStream_t s) {
    k_xpby<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(x, num, den, p, n);
    return cudaGetLastError();
}
cudaError_t vec_sub(const double *b, const double *t, double *r, int64_t n, cudaStream_t s) {
    k_sub<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(b, t, r, n);
    return cudaGetLastError();
}
cudaError_t convert_to_f64(const void *src, int is_f32, int64_t n, double *dst, cudaStream_t s) {
    if (is_f32)
        k_copy_to_f64<float><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>((const float *)src, n, dst);
    else
        k_copy_to_f64<double><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>((const double *)src, n, dst);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_read_rows(const T *A, int64_t ld, int64_t M, int64_t row0, int64_t nrows, double *dst,
                             cudaStream_t s) {
    int64_t n = nrows * M;
    if (n == 0) return cudaSuccess;
    k_read_rows<T><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(A, ld, M, row0, nrows, dst);
    return cudaGetLastError();
}
template <class T>
cudaError_t launch_read_r(const T *A, int64_t ld, int64_t M, double *dst, cudaStream_t s) {
    k_read_r<T><<<(unsigned)ceil_div(M * M, 256), 256, 0, s>>>(A, ld, M, dst);
    return cudaGetLastError();
}

template <class T>
cudaError_t tsqr_gather(const T *A, int64_t ld, int64_t r0, int64_t M, T *S, int64_t lds, int64_t srow, bool zero_b,
                        cudaStream_t s) {
    const int64_t n = M * (M + 1);
    if (n == 0) return cudaSuccess;
    k_tsqr_gather<T><<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(A, ld, r0, M, S, lds, srow, zero_b ? 1 : 0);
    return cudaGetLastError();
}

#define GAP_INST(T)                                                                                              \
    template cudaError_t launch_stack_u<T>(const Dims &, const double *, T *, cudaStream_t, bool);               \
    template cudaError_t householder_qr<T>(T *, int64_t, int64_t, int64_t, int, T *, T *, T *, T *, T *, T *,   \
                                           int, cudaStream_t, Prof *, void *, int *, int, int);                  \
    template cudaError_t trsv_upper<T>(const T *, int64_t, int64_t, int, double *, const double *, double *,    \
                                       cudaStream_t);                                                            \
    template cudaError_t trsv_invert_blocks<T>(const T *, int64_t, int64_t, double *, DevStatus *, cudaStream_t); \
    template cudaError_t back_substitution<T>(const T *, int64_t, int64_t, const T *, double *, double *,        \
                                              DevStatus *, cudaStream_t);                                        \
    template cudaError_t gemv_n<T>(const T *, int64_t, int64_t, int64_t, const double *, double *, cudaStream_t); \
    template cudaError_t gemv_t<T>(const T *, int64_t, int64_t, int64_t, const double *, double *, float *,      \
                                   cudaStream_t);                                                                \
    template cudaError_t launch_read_rows<T>(const T *, int64_t, int64_t, int64_t, int64_t, double *,            \
                                             cudaStream_t);                                                      \
    template cudaError_t launch_read_r<T>(const T *, int64_t, int64_t, double *, cudaStream_t);                  \
    template cudaError_t tsqr_gather<T>(const T *, int64_t, int64_t, int64_t, T *, int64_t, int64_t, bool,       \
                                        cudaStream_t);
GAP_INST(double)
GAP_INST(float)
#undef GAP_INST

}  // namespace gap
