// CUR sparse-point selection (the cur_points choice of the sparse set, Secs. III-A and III-C, after
// Mahoney and Drineas, PNAS 106 (2009) 697): per species, the M sparse points are M
// distinct atoms drawn without replacement with probabilities given by the rank-k
// leverage scores of that species' descriptor rows,
//     pi_i = |U_k[i, :]|^2 / k,   X = U S V^T,  U_k the k leading left singular vectors.
// U_k comes from a randomised range finder (Halko, Martinsson and Tropp, SIAM Rev. 53
// (2011) 217, Algs. 4.4 and 5.1): Q = orth(X Omega), q times Q = orth(X (X^T Q)),
// B = Q^T X, B B^T = W diag(lambda) W^T, U_k = Q W_k.  orth is shifted CholeskyQR3
// (G = Y^T Y (+ shift) = R^T R, Y <- Y R^{-1}, three times); the eigenvectors of B B^T
// come from cyclic Jacobi rotations in one block.  The draw without replacement keeps the M largest keys
// log(u_i) / pi_i (Efraimidis and Spirakis, IPL 97 (2006) 181), ties to the lower atom
// index.  Omega and u are inputs.  Every step is FP64 SIMT arithmetic.
#include <string>

#include "gap_internal.cuh"

namespace gap {
namespace {

constexpr int CUR_LMAX = 128;  // largest l = k + oversampling
constexpr int GT_M = 64, GT_N = 32, GT_K = 16;

// C[i, j] (slab z of a split-K sum) = sum over kk in slab z of A(i, kk) B(kk, j),
//   A(i, kk) = TA ? A[kk * lda + i] : A[i * lda + kk],   B(kk, j) = B[kk * sbk + j * sbc].
// Block tile 64 x 32, 256 threads with 2 x 4 outputs each; slab z covers kk in
// [z * kper, min(K, (z + 1) * kper)) and writes C + z * m * ldc.  Fixed summation order.
template <bool TA>
__global__ void __launch_bounds__(256) k_cur_gemm(int64_t m, int64_t n, int64_t K, int64_t kper,
                                                  const double *__restrict__ A, int64_t lda,
                                                  const double *__restrict__ B, int64_t sbk, int64_t sbc,
                                                  double *__restrict__ C, int64_t ldc) {
    __shared__ double As[GT_K][GT_M + 1];
    __shared__ double Bs[GT_K][GT_N + 1];
    const int t = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * GT_M, j0 = (int64_t)blockIdx.y * GT_N;
    const int64_t kb = (int64_t)blockIdx.z * kper, ke = min(K, kb + kper);
    C += (int64_t)blockIdx.z * m * ldc;
    const int ti = t >> 3, tj = t & 7;
    double acc[2][4] = {};
    for (int64_t k0 = kb; k0 < ke; k0 += GT_K) {
#pragma unroll
        for (int q = 0; q < GT_M * GT_K / 256; ++q) {
            const int e = t + q * 256;
            const int i = TA ? e % GT_M : e / GT_K, kk = TA ? e / GT_M : e % GT_K;
            const int64_t gi = i0 + i, gk = k0 + kk;
            As[kk][i] = (gi < m && gk < ke) ? (TA ? A[gk * lda + gi] : A[gi * lda + gk]) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < GT_N * GT_K / 256; ++q) {
            const int e = t + q * 256;
            const int j = sbc == 1 ? e % GT_N : e / GT_K, kk = sbc == 1 ? e / GT_N : e % GT_K;
            const int64_t gj = j0 + j, gk = k0 + kk;
            Bs[kk][j] = (gj < n && gk < ke) ? B[gk * sbk + gj * sbc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GT_K; ++kk) {
            const double a0 = As[kk][ti], a1 = As[kk][ti + 32];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double b = Bs[kk][tj + 8 * c];
                acc[0][c] = fma(a0, b, acc[0][c]);
                acc[1][c] = fma(a1, b, acc[1][c]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t gi = i0 + ti + 32 * r, gj = j0 + tj + 8 * c;
            if (gi < m && gj < n) C[gi * ldc + gj] = acc[r][c];
        }
}

// out[e] = sum over g of part[g * len + e], g ascending.
__global__ void k_cur_sum_slabs(const double *__restrict__ part, int G, int64_t len, double *__restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += part[(int64_t)g * len + e];
    out[e] = s;
}

// Atoms of species t (all atoms when species is NULL), ascending, into idx; their count
// into *count.  One block over chunks of blockDim atoms, a block-wide scan per chunk.
__global__ void __launch_bounds__(1024) k_cur_species_index(const int32_t *__restrict__ species, int32_t t,
                                                           int64_t n, int64_t *__restrict__ idx,
                                                           int64_t *__restrict__ count) {
    __shared__ int s_w[32];
    __shared__ int64_t s_base;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
        const int64_t a = c0 + tid;
        const bool in = a < n && (species == nullptr || species[a] == t);
        const unsigned b = __ballot_sync(0xffffffffu, in);
        if (lane == 0) s_w[w] = __popc(b);
        __syncthreads();
        int before = 0, total = 0;
        for (int i = 0; i < nw; ++i) {
            before += i < w ? s_w[i] : 0;
            total += s_w[i];
        }
        const int64_t base = s_base;
        if (in) idx[base + before + __popc(b & ((1u << lane) - 1u))] = a;
        __syncthreads();
        if (tid == 0) s_base = base + total;
        __syncthreads();
    }
    if (tid == 0) *count = s_base;
}

// Xs[r, :] = X[idx[r], :].
__global__ void k_cur_gather(const double *__restrict__ X, int64_t d, const int64_t *__restrict__ idx, int64_t n,
                             double *__restrict__ Xs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    const int64_t r = e / d, c = e % d;
    Xs[e] = X[idx[r] * d + c];
}

// One block: G + sigma I (l x l, symmetric positive definite) = R^T R with R upper
// triangular, and Rinv = R^{-1} (upper, l x l row-major, global).  sigma = 0, or with
// shift set the shift of shifted CholeskyQR for G = Y^T Y of an n x l matrix Y,
// sigma = 11 (n l + l (l + 1)) 2^-53 trace(G) (Fukaya, Kannan, Nakatsukasa, Yamamoto
// and Yanagisawa, SIAM J. Sci. Comput. 42 (2020) A477), which keeps the factor finite
// for Y of condition up to about 2^53.  Sets *status = 1 at a non-positive pivot; does
// nothing once *status is set.  Dynamic shared memory: l (l + 1) doubles.
__global__ void __launch_bounds__(1024) k_cur_chol_inv(const double *__restrict__ G, int l, int64_t n, int shift,
                                                      double *__restrict__ Rinv, int *status) {
    extern __shared__ double sh[];
    const int ld = l + 1;
    double *R = sh;
    __shared__ int bad;
    const int t = threadIdx.x, nt = blockDim.x;
    for (int e = t; e < l * l; e += nt) R[(e / l) * ld + e % l] = G[e];
    if (t == 0) bad = *status;
    __syncthreads();
    if (bad) return;
    if (shift && t == 0) {
        double tr = 0.0;
        for (int j = 0; j < l; ++j) tr += R[j * ld + j];
        const double sg = 11.0 * ((double)n * l + (double)l * (l + 1)) * 0x1p-53 * tr;
        for (int j = 0; j < l; ++j) R[j * ld + j] += sg;
    }
    __syncthreads();
    for (int j = 0; j < l; ++j) {
        if (t == 0) {
            const double pv = R[j * ld + j];
            if (!(pv > 0.0)) bad = 1;
            R[j * ld + j] = sqrt(pv > 0.0 ? pv : 1.0);
        }
        __syncthreads();
        if (bad) break;
        for (int c = j + 1 + t; c < l; c += nt) R[j * ld + c] /= R[j * ld + j];
        __syncthreads();
        const int w = l - j - 1;
        for (int e = t; e < w * w; e += nt) {
            const int a = j + 1 + e / w, c = j + 1 + e % w;
            if (c >= a) R[a * ld + c] -= R[j * ld + a] * R[j * ld + c];
        }
        __syncthreads();
    }
    if (bad) {
        if (t == 0) *status = 1;
        return;
    }
    // column c of R^{-1} solves R x = e_c (one thread per column, rows c down to 0)
    for (int c = t; c < l; c += nt) {
        for (int i = l - 1; i > c; --i) Rinv[i * l + c] = 0.0;
        for (int i = c; i >= 0; --i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int m = i + 1; m <= c; ++m) s -= R[i * ld + m] * Rinv[m * l + c];
            Rinv[i * l + c] = s / R[i * ld + i];
        }
    }
}

// One block: the eigenvectors of the symmetric positive semidefinite H (l x l) for its k
// largest eigenvalues, as the columns of W (l x k row-major), by cyclic Jacobi rotations
// in round-robin order (each step rotates l/2 disjoint index pairs at once; the rotations
// of one step commute).  A pair is rotated while |h_pq| > 2^-52 sqrt(h_pp h_qq) (the
// relative criterion of Demmel and Veselic, SIAM J. Matrix Anal. Appl. 13 (1992) 1204);
// the sweeps end when one rotates nothing (at most 60).  V (l x l, global) accumulates
// the rotations.  Skipped once *status is set.  Dynamic shared memory: l (l + 1) doubles.
__global__ void __launch_bounds__(1024) k_cur_eig(const double *__restrict__ H, int l, int k,
                                                 double *__restrict__ V, double *__restrict__ W,
                                                 const int *status) {
    extern __shared__ double sh[];
    const int ld = l + 1;
    double *C = sh;
    __shared__ double cs[CUR_LMAX / 2][2];
    __shared__ int pq[CUR_LMAX / 2][2];
    __shared__ int order[CUR_LMAX];
    __shared__ int rotated;
    const int t = threadIdx.x, nt = blockDim.x;
    if (*status) return;
    for (int e = t; e < l * l; e += nt) {
        const int i = e / l, j = e % l;
        C[i * ld + j] = 0.5 * (H[e] + H[j * l + i]);
        V[e] = (i == j) ? 1.0 : 0.0;
    }
    const int lp = l + (l & 1);  // with l odd, index l is a bye
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (t == 0) rotated = 0;
        __syncthreads();
        for (int step = 0; step < lp - 1; ++step) {
            if (t < lp / 2) {
                // circle method: position 0 keeps index 0, positions 1..lp-1 rotate
                const int pa = t, pb = lp - 1 - t;
                int p = pa == 0 ? 0 : 1 + (pa - 1 + step) % (lp - 1);
                int q = 1 + (pb - 1 + step) % (lp - 1);
                if (p > q) {
                    const int x = p;
                    p = q;
                    q = x;
                }
                double c = 1.0, s = 0.0;
                if (q < l) {
                    const double apq = C[p * ld + q], app = C[p * ld + p], aqq = C[q * ld + q];
                    if (fabs(apq) > 0x1p-52 * sqrt(fabs(app * aqq))) {
                        const double th = (aqq - app) / (2.0 * apq);
                        const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        s = tt * c;
                        rotated = 1;
                    }
                }
                pq[t][0] = p;
                pq[t][1] = q;
                cs[t][0] = c;
                cs[t][1] = s;
            }
            __syncthreads();
            // rows p, q of C  <-  J^T from the left
            for (int e = t; e < (lp / 2) * l; e += nt) {
                const int r = e / l, j = e % l, p = pq[r][0], q = pq[r][1];
                if (q < l && cs[r][1] != 0.0) {
                    const double c = cs[r][0], s = cs[r][1], a = C[p * ld + j], b = C[q * ld + j];
                    C[p * ld + j] = c * a - s * b;
                    C[q * ld + j] = s * a + c * b;
                }
            }
            __syncthreads();
            // columns p, q of C and of V  <-  J from the right
            for (int e = t; e < (lp / 2) * l; e += nt) {
                const int r = e / l, i = e % l, p = pq[r][0], q = pq[r][1];
                if (q < l && cs[r][1] != 0.0) {
                    const double c = cs[r][0], s = cs[r][1];
                    const double a = C[i * ld + p], b = C[i * ld + q];
                    C[i * ld + p] = c * a - s * b;
                    C[i * ld + q] = s * a + c * b;
                    const double va = V[i * l + p], vb = V[i * l + q];
                    V[i * l + p] = c * va - s * vb;
                    V[i * l + q] = s * va + c * vb;
                }
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();  // every thread has read the flag before the next sweep clears it
        if (!any) break;
    }
    // eigenvalues in decreasing order, ties to the lower index
    if (t == 0) {
        for (int j = 0; j < l; ++j) order[j] = j;
        for (int a = 1; a < l; ++a)
            for (int b = a; b > 0; --b) {
                const int x = order[b - 1], y = order[b];
                if (!(C[y * ld + y] > C[x * ld + x])) break;
                order[b - 1] = y;
                order[b] = x;
            }
    }
    __syncthreads();
    for (int e = t; e < l * k; e += nt) W[e] = V[(e / k) * l + order[e % k]];
}

// pi[r] = |L[r, :]|^2 / k for L = Q W_k (n x k); key[r] = log(u[idx[r]]) / pi[r]
// (-inf for pi = 0); the leverage also goes to lev[idx[r]] when lev is given.
__global__ void k_cur_leverage(const double *__restrict__ L, int k, int64_t n, const int64_t *__restrict__ idx,
                               const double *__restrict__ u, double *__restrict__ key, double *__restrict__ lev) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double s2 = 0.0;
    for (int j = 0; j < k; ++j) s2 = fma(L[r * k + j], L[r * k + j], s2);
    const double p = s2 / (double)k;
    key[r] = p > 0.0 ? log(u[idx[r]]) / p : -INFINITY;
    if (lev) lev[idx[r]] = p;
}

// Order-preserving image of a double in the unsigned 64-bit integers.
__device__ __forceinline__ unsigned long long key_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// One block: the atoms idx[r] of the m largest keys (1 <= m <= n; ties to the lower r),
// ascending, into out[0..m).  The threshold T (the largest value with at least m keys at
// or above it) is fixed bit by bit from the top; every key above T is taken, then the
// first m - (number above T) keys equal to T.  Exactly m entries are written.
__global__ void __launch_bounds__(1024) k_cur_select(const double *__restrict__ key, const int64_t *__restrict__ idx,
                                                    int64_t n, int64_t m, int64_t *__restrict__ out) {
    __shared__ unsigned long long s_w[32];
    __shared__ int s_e[32];
    __shared__ int64_t s_pos, s_eq;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    auto count_ge = [&](unsigned long long T) -> unsigned long long {
        unsigned long long c = 0;
        for (int64_t r = tid; r < n; r += blockDim.x) c += key_bits(key[r]) >= T ? 1ull : 0ull;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) s_w[w] = c;
        __syncthreads();
        unsigned long long tot = 0;
        for (int i = 0; i < nw; ++i) tot += s_w[i];
        __syncthreads();
        return tot;
    };
    unsigned long long T = 0;
    for (int bit = 63; bit >= 0; --bit) {
        const unsigned long long cand = T | (1ull << bit);
        if (count_ge(cand) >= (unsigned long long)m) T = cand;
    }
    const int64_t above = T == ~0ull ? 0 : (int64_t)count_ge(T + 1ull);
    const int64_t want_eq = m - above;
    if (tid == 0) s_pos = s_eq = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
        const int64_t r = c0 + tid;
        const unsigned long long kb = r < n ? key_bits(key[r]) : 0ull;
        const bool gt = r < n && kb > T, eq = r < n && kb == T;
        const unsigned be = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) s_e[w] = __popc(be);
        __syncthreads();
        int eq_before = 0, eq_total = 0;
        for (int i = 0; i < nw; ++i) {
            eq_before += i < w ? s_e[i] : 0;
            eq_total += s_e[i];
        }
        const int64_t eq_base = s_eq, pos = s_pos;
        const bool take = gt || (eq && eq_base + eq_before + __popc(be & ((1u << lane) - 1u)) < want_eq);
        const unsigned bt = __ballot_sync(0xffffffffu, take);
        __syncthreads();
        if (lane == 0) s_e[w] = __popc(bt);
        __syncthreads();
        int t_before = 0, t_total = 0;
        for (int i = 0; i < nw; ++i) {
            t_before += i < w ? s_e[i] : 0;
            t_total += s_e[i];
        }
        if (take) out[pos + t_before + __popc(bt & ((1u << lane) - 1u))] = idx[r];
        __syncthreads();
        if (tid == 0) {
            s_pos = pos + t_total;
            s_eq = eq_base + eq_total;
        }
        __syncthreads();
    }
}

void put_msg(char *buf, size_t len, const std::string &msg) {
    if (!buf || len == 0) return;
    const size_t n = msg.size() < len - 1 ? msg.size() : len - 1;
    msg.copy(buf, n);
    buf[n] = '\0';
}

struct CurWork {
    double *Xs, *Y, *Y2, *slab, *G, *Rinv, *P, *H, *V, *W, *L, *key;
    int *status;
};

constexpr int kSlabs = 48;  // split-K slabs of the sums over atoms

int64_t slab_rows(int64_t n) { return round_up(ceil_div(n, kSlabs), GT_K); }

// C (a x b) = A^T B over the n rows of A (n x a) and B (n x b), summed in fixed slabs.
void tn_sum(const double *A, int64_t a, const double *B, int64_t b, int64_t n, double *C, double *slab,
            cudaStream_t s) {
    const int64_t kper = slab_rows(n);
    const int G = (int)ceil_div(n, kper);
    dim3 grid((unsigned)ceil_div(a, GT_M), (unsigned)ceil_div(b, GT_N), (unsigned)G);
    k_cur_gemm<true><<<grid, 256, 0, s>>>(a, b, n, kper, A, a, B, b, 1, slab, b);
    k_cur_sum_slabs<<<(unsigned)ceil_div(a * b, 256), 256, 0, s>>>(slab, G, a * b, C);
}

// C (m x n) = A (m x K, row-major) B with B(kk, j) = B[kk * sbk + j * sbc].
void nn(const double *A, int64_t m, int64_t K, const double *B, int64_t sbk, int64_t sbc, int64_t n, double *C,
        cudaStream_t s) {
    dim3 grid((unsigned)ceil_div(m, GT_M), (unsigned)ceil_div(n, GT_N), 1);
    k_cur_gemm<false><<<grid, 256, 0, s>>>(m, n, K, K, A, K, B, sbk, sbc, C, n);
}

size_t smem_bytes(int l) { return (size_t)l * (l + 1) * sizeof(double); }

// Y (n x l) <- an orthonormal basis of its range: shifted CholeskyQR3 (one shifted
// pass, then two plain ones).
void orth(CurWork &w, double *&Y, double *&Y2, int64_t n, int l, cudaStream_t s) {
    for (int pass = 0; pass < 3; ++pass) {
        tn_sum(Y, l, Y, l, n, w.G, w.slab, s);
        k_cur_chol_inv<<<1, 1024, smem_bytes(l), s>>>(w.G, l, n, pass == 0, w.Rinv, w.status);
        nn(Y, n, l, w.Rinv, l, 1, l, Y2, s);
        std::swap(Y, Y2);
    }
}

}  // namespace

// Kernel launches of one species' selection (for launch counts).
int cur_launches_per_species(int power_iters) {
    const int orth = 3 * 4;  // per pass: split-K product, slab sum, Cholesky + inverse, product
    return 1 + 1 + orth + power_iters * (2 + 1 + orth) + 2 + 1 + 1 + 1 + 1 + 1;
}

}  // namespace gap

using namespace gap;

extern "C" gap_status gap_select_cur(const double *X, int64_t n_atoms, int64_t d, const int32_t *atom_species,
                                     int32_t n_species, const int64_t *n_select, int32_t k, int32_t l,
                                     int32_t power_iters, const double *omega, const double *u, int64_t *selected,
                                     double *leverage, void *cuda_stream, char *err, size_t err_len) {
    put_msg(err, err_len, "");
    if (!X || !n_select || !omega || !u || !selected || n_atoms <= 0 || d <= 0 || n_species < 1 ||
        n_species > 4096 || (n_species > 1 && !atom_species)) {
        put_msg(err, err_len, "X, n_select, omega, u and selected are required (atom_species too for several "
                              "species); n_atoms and d must be positive and 1 <= n_species <= 4096");
        return GAP_ERR_INVALID;
    }
    if (k < 1 || l < k || l > CUR_LMAX || l > d || power_iters < 0 || power_iters > 64) {
        put_msg(err, err_len, "need 1 <= k <= l <= min(d, " + std::to_string(CUR_LMAX) +
                                  ") and 0 <= power_iters <= 64");
        return GAP_ERR_INVALID;
    }
    if (d > 65536 || n_atoms > (int64_t(1) << 36) / d) {
        put_msg(err, err_len, "descriptor matrix too large (d above 65536 or n_atoms * d above 2^36)");
        return GAP_ERR_INVALID;
    }
    for (int t = 0; t < n_species; ++t)
        if (n_select[t] < 0) {
            put_msg(err, err_len, "n_select must be non-negative");
            return GAP_ERR_INVALID;
        }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (cudaFuncSetAttribute(k_cur_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(l)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_cur_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(l)) !=
            cudaSuccess) {
        put_msg(err, err_len, "cudaFuncSetAttribute failed");
        return GAP_ERR_CUDA;
    }
    gap_status rc = GAP_OK;
    auto fail = [&](gap_status code, const std::string &msg) {
        put_msg(err, err_len, msg);
        rc = code;
    };
    // the atoms of each species, ascending, one block of idx_all after another
    int64_t *idx_all = nullptr, *counts_d = nullptr;
    if (cudaMallocAsync((void **)&idx_all, sizeof(int64_t) * (size_t)n_atoms, s) != cudaSuccess ||
        cudaMallocAsync((void **)&counts_d, sizeof(int64_t) * (size_t)n_species, s) != cudaSuccess) {
        cudaGetLastError();
        if (idx_all) cudaFreeAsync(idx_all, s);
        put_msg(err, err_len, "device allocation failed");
        return GAP_ERR_NOMEM;
    }
    std::vector<int64_t> counts(n_species, 0);
    {
        // a species' block starts after all lower species' atoms: count first, then place
        for (int t = 0; t < n_species; ++t)
            k_cur_species_index<<<1, 1024, 0, s>>>(n_species > 1 ? atom_species : nullptr, t, n_atoms, idx_all,
                                                   counts_d + t);
        if (cudaMemcpyAsync(counts.data(), counts_d, sizeof(int64_t) * n_species, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            fail(GAP_ERR_CUDA, "species index pass failed");
        int64_t off = 0;
        for (int t = 0; t < n_species && rc == GAP_OK; ++t) {
            if (counts[t] > 0)
                k_cur_species_index<<<1, 1024, 0, s>>>(n_species > 1 ? atom_species : nullptr, t, n_atoms,
                                                       idx_all + off, counts_d + t);
            off += counts[t];
        }
        if (rc == GAP_OK && off != n_atoms) fail(GAP_ERR_INVALID, "atom_species holds values outside [0, n_species)");
    }
    int64_t nmax = 0;
    for (int t = 0; t < n_species && rc == GAP_OK; ++t) {
        if (n_select[t] > counts[t]) {
            fail(GAP_ERR_INVALID, "species " + std::to_string(t) + " has " + std::to_string((long long)counts[t]) +
                                      " atoms, fewer than its " + std::to_string((long long)n_select[t]) +
                                      " sparse points");
            break;
        }
        if (n_select[t] > 0 && counts[t] < l) {
            fail(GAP_ERR_INVALID, "species " + std::to_string(t) + " has fewer atoms than l");
            break;
        }
        if (n_select[t] > 0) nmax = std::max(nmax, counts[t]);
    }
    CurWork w{};
    void *pool = nullptr;
    if (rc == GAP_OK && nmax > 0) {
        const int64_t slabs = kSlabs;  // every species' split-K sum uses at most kSlabs slabs
        const int64_t dl = std::max<int64_t>(d, l);
        const int64_t doubles[12] = {nmax * d,       nmax * l,       nmax * l,       slabs * l * dl,
                                     (int64_t)l * l, (int64_t)l * l, (int64_t)l * d, (int64_t)l * l,
                                     (int64_t)l * l, (int64_t)l * k, nmax * k,       nmax};
        size_t bytes = 256;  // status word
        for (int64_t x : doubles) bytes += (size_t)round_up(x * 8, 256);
        if (cudaMallocAsync(&pool, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            pool = nullptr;
            fail(GAP_ERR_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        } else {
            char *q = (char *)pool;
            double **dst[12] = {&w.Xs, &w.Y, &w.Y2, &w.slab, &w.G, &w.Rinv, &w.P, &w.H, &w.V, &w.W, &w.L, &w.key};
            for (int i = 0; i < 12; ++i) {
                *dst[i] = (double *)q;
                q += round_up(doubles[i] * 8, 256);
            }
            w.status = (int *)q;
        }
    }
    int64_t off = 0, out_off = 0;
    for (int t = 0; t < n_species && rc == GAP_OK; ++t) {
        const int64_t n = counts[t], m = n_select[t];
        const int64_t *idx = idx_all + off;
        off += n;
        if (m == 0) continue;
        cudaMemsetAsync(w.status, 0, sizeof(int), s);
        k_cur_gather<<<(unsigned)ceil_div(n * d, 256), 256, 0, s>>>(X, d, idx, n, w.Xs);
        double *Y = w.Y, *Y2 = w.Y2;
        nn(w.Xs, n, d, omega, l, 1, l, Y, s);  // Y = Xs Omega
        orth(w, Y, Y2, n, l, s);
        for (int it = 0; it < power_iters; ++it) {
            tn_sum(Y, l, w.Xs, d, n, w.P, w.slab, s);  // P = Q^T Xs  (l x d)
            nn(w.Xs, n, d, w.P, 1, d, l, Y, s);         // Y = Xs P^T
            orth(w, Y, Y2, n, l, s);
        }
        tn_sum(Y, l, w.Xs, d, n, w.P, w.slab, s);  // B = Q^T Xs
        nn(w.P, l, d, w.P, 1, d, l, w.H, s);        // H = B B^T
        k_cur_eig<<<1, 1024, smem_bytes(l), s>>>(w.H, l, k, w.V, w.W, w.status);
        nn(Y, n, l, w.W, k, 1, k, w.L, s);  // L = Q W_k
        k_cur_leverage<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(w.L, k, n, idx, u, w.key, leverage);
        k_cur_select<<<1, 1024, 0, s>>>(w.key, idx, n, m, selected + out_off);
        out_off += m;
        int h_status = 0;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess ||
            cudaMemcpyAsync(&h_status, w.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            fail(GAP_ERR_CUDA, std::string("CUR selection failed: ") + cudaGetErrorString(e));
            break;
        }
        if (h_status) {
            fail(GAP_ERR_RANK, "the descriptor rows of species " + std::to_string(t) +
                                   " are too close to rank deficient for the range finder (CholeskyQR met a non-positive pivot)");
            break;
        }
    }
    if (pool) cudaFreeAsync(pool, s);
    cudaFreeAsync(counts_d, s);
    cudaFreeAsync(idx_all, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == GAP_OK) fail(GAP_ERR_CUDA, "CUR selection failed");
    return rc;
}
