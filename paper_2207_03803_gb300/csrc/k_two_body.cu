// Two-body sub-GAP (the appendix's distance_2b descriptors with covariance_type=ard_se),
// summed into the same fit as the SOAP block: one descriptor instance per atom pair within
// the cutoff (its distance r), the covariance
//     k(r, r') = delta^2 exp(-(r - r')^2 / (2 theta^2)) f(r) f(r'),
//     f(r) = 1 below r_c - w, (1 + cos(pi (r - r_c + w) / w)) / 2 up to r_c, 0 beyond,
// and its sparse distances r_t as the design matrix's columns col0 .. col0 + M2 - 1.  The
// bonds come listed from both ends and grouped by atom (length r, unit vector
// u = (r_a - r_j) / r), so a configuration's energy is half the sum over its bonds.  Rows
// (scaled by 1/sigma like the SOAP block's):
//     energy (A):         (1/2) sum_{b in A} k(r_b, r_t)
//     force (a, alpha):   -sum_{b of a} dk/dr(r_b, r_t) u_b[alpha]
//     virial (A, v):      -(1/2) sum_{b in A} dk/dr(r_b, r_t) r_b u_b[alpha] u_b[beta]
// The SOAP assembly sees the two-body columns as sparse points with zero descriptors (and
// a species no atom has), so it leaves them zero; these kernels then store them.  All
// arithmetic is FP64; the mixed precisions store FP32 copies in the QR matrix and the
// refinement's matrix and the FP64 energy rows.
#include "gap_internal.cuh"

namespace gap {
namespace {

__device__ void set_status(DevStatus *st, int code, int64_t idx) {
    if (atomicCAS(&st->code, 0, code) == 0) st->index = idx;
}

__device__ __forceinline__ void cutoff_fn(double r, const TwoBodyDev &tb, double &f, double &df) {
    if (r >= tb.rc) {
        f = 0.0;
        df = 0.0;
    } else if (r <= tb.rc - tb.w) {
        f = 1.0;
        df = 0.0;
    } else {
        const double x = (r - tb.rc + tb.w) / tb.w;
        f = 0.5 * (1.0 + cos(M_PI * x));
        df = -0.5 * M_PI / tb.w * sin(M_PI * x);
    }
}

// k(r, r_t) and dk/dr for the sparse distance r_t (its cutoff weight ft given).
__device__ __forceinline__ void kernel_2b(double r, double f, double df, double rt, double ft, const TwoBodyDev &tb,
                                          double &k, double &dk) {
    const double x = r - rt;
    const double g = tb.delta2 * exp(-x * x * tb.inv2t2);
    k = g * f * ft;
    dk = g * (-2.0 * tb.inv2t2 * x * f + df) * ft;
}

template <class T>
__device__ __forceinline__ void store_row(int64_t row, int64_t col, double v, T *A, int64_t ld, float *Aacc,
                                          int64_t nc, double *E64, int64_t M) {
    A[row + col * ld] = (T)v;
    if (Aacc) Aacc[acc_index(row, col, nc)] = (float)v;
    if (E64) E64[row * M + col] = v;
}

// Energy rows and (with virials) virial rows: one block per configuration, one thread per
// sparse distance (strided), the configuration's bonds in order.
template <class T>
__global__ void k_2b_cfg_rows(int64_t n_cfg, int64_t n_atoms, const int64_t *__restrict__ cfg_ptr, TwoBodyDev tb,
                              const double *__restrict__ sigma, bool virials, T *A, int64_t ld, float *Aacc,
                              double *E64, int64_t M) {
    const int64_t cf = blockIdx.x;
    const int64_t b0 = tb.bond_ptr[cfg_ptr[cf]], b1 = tb.bond_ptr[cfg_ptr[cf + 1]];
    for (int64_t t = threadIdx.x; t < tb.M2; t += blockDim.x) {
        const double rt = tb.sparse_r[t];
        double ft, dft;
        cutoff_fn(rt, tb, ft, dft);
        double e = 0.0, v[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t b = b0; b < b1; ++b) {
            const double r = tb.bond_r[b];
            double f, df, k, dk;
            cutoff_fn(r, tb, f, df);
            kernel_2b(r, f, df, rt, ft, tb, k, dk);
            e += k;
            if (virials) {
                const double ux = tb.bond_u[3 * b], uy = tb.bond_u[3 * b + 1], uz = tb.bond_u[3 * b + 2];
                const double w = dk * r;
                v[0] += w * ux * ux;
                v[1] += w * uy * uy;
                v[2] += w * uz * uz;
                v[3] += w * uy * uz;
                v[4] += w * ux * uz;
                v[5] += w * ux * uy;
            }
        }
        const int64_t col = tb.col0 + t;
        store_row<T>(cf, col, 0.5 * e / sigma[cf], A, ld, Aacc, M + 1, E64, M);
        if (virials)
            for (int c = 0; c < 6; ++c) {
                const int64_t row = n_cfg + 3 * n_atoms + 6 * cf + c;
                store_row<T>(row, col, -0.5 * v[c] / sigma[row], A, ld, Aacc, M + 1, nullptr, M);
            }
    }
}

// Force rows: one warp per atom, one lane per sparse distance (strided).
template <class T>
__global__ void k_2b_force_rows(int64_t n_cfg, int64_t n_atoms, TwoBodyDev tb, const double *__restrict__ sigma,
                                T *A, int64_t ld, float *Aacc, int64_t M) {
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a >= n_atoms) return;
    const int64_t b0 = tb.bond_ptr[a], b1 = tb.bond_ptr[a + 1];
    for (int64_t t = lane; t < tb.M2; t += 32) {
        const double rt = tb.sparse_r[t];
        double ft, dft;
        cutoff_fn(rt, tb, ft, dft);
        double g[3] = {0, 0, 0};
        for (int64_t b = b0; b < b1; ++b) {
            const double r = tb.bond_r[b];
            double f, df, k, dk;
            cutoff_fn(r, tb, f, df);
            kernel_2b(r, f, df, rt, ft, tb, k, dk);
            for (int al = 0; al < 3; ++al) g[al] += dk * tb.bond_u[3 * b + al];
        }
        for (int al = 0; al < 3; ++al) {
            const int64_t row = n_cfg + 3 * a + al;
            store_row<T>(row, tb.col0 + t, -g[al] / sigma[row], A, ld, Aacc, M + 1, nullptr, M);
        }
    }
}

// The two-body block of K_MM (column-major M x M) with the jitter on its diagonal.
__global__ void k_2b_kmm(TwoBodyDev tb, double jitter, double *K, int64_t M) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= tb.M2 * tb.M2) return;
    const int64_t t = e / tb.M2, u = e % tb.M2;
    double ft, dft, fu, dfu, k, dk;
    cutoff_fn(tb.sparse_r[t], tb, ft, dft);
    cutoff_fn(tb.sparse_r[u], tb, fu, dfu);
    kernel_2b(tb.sparse_r[t], ft, dft, tb.sparse_r[u], fu, tb, k, dk);
    K[(tb.col0 + t) + (tb.col0 + u) * M] = k + (t == u ? jitter : 0.0);
}

// eps(r) = sum_t c_t k(r, r_t) and its derivative, for bond b.
__device__ __forceinline__ void eps_2b(int64_t b, const TwoBodyDev &tb, const double *c2, double &e, double &de) {
    const double r = tb.bond_r[b];
    double f, df;
    cutoff_fn(r, tb, f, df);
    e = de = 0.0;
    for (int64_t t = 0; t < tb.M2; ++t) {
        double ft, dft, k, dk;
        cutoff_fn(tb.sparse_r[t], tb, ft, dft);
        kernel_2b(r, f, df, tb.sparse_r[t], ft, tb, k, dk);
        e += c2[t] * k;
        de += c2[t] * dk;
    }
}

// Predictions added to E [n_cfg] and V [6 n_cfg] (may be null): one thread per configuration.
__global__ void k_2b_predict_cfg(int64_t n_cfg, const int64_t *__restrict__ cfg_ptr, TwoBodyDev tb,
                                 const double *__restrict__ c2, double *E, double *V) {
    const int64_t cf = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (cf >= n_cfg) return;
    double e = 0.0, v[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t b = tb.bond_ptr[cfg_ptr[cf]]; b < tb.bond_ptr[cfg_ptr[cf + 1]]; ++b) {
        double eb, deb;
        eps_2b(b, tb, c2, eb, deb);
        e += eb;
        if (V) {
            const double ux = tb.bond_u[3 * b], uy = tb.bond_u[3 * b + 1], uz = tb.bond_u[3 * b + 2];
            const double w = deb * tb.bond_r[b];
            v[0] += w * ux * ux;
            v[1] += w * uy * uy;
            v[2] += w * uz * uz;
            v[3] += w * uy * uz;
            v[4] += w * ux * uz;
            v[5] += w * ux * uy;
        }
    }
    E[cf] += 0.5 * e;
    if (V)
        for (int c = 0; c < 6; ++c) V[6 * cf + c] -= 0.5 * v[c];
}

// Predictions added to F [3 n_atoms]: one thread per atom.
__global__ void k_2b_predict_atoms(int64_t n_atoms, TwoBodyDev tb, const double *__restrict__ c2, double *F) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_atoms) return;
    double g[3] = {0, 0, 0};
    for (int64_t b = tb.bond_ptr[a]; b < tb.bond_ptr[a + 1]; ++b) {
        double eb, deb;
        eps_2b(b, tb, c2, eb, deb);
        for (int al = 0; al < 3; ++al) g[al] += deb * tb.bond_u[3 * b + al];
    }
    for (int al = 0; al < 3; ++al) F[3 * a + al] -= g[al];
}

// Structure of the bond arrays: bond_ptr from 0 to n_bonds and monotone, lengths finite
// and positive, sparse distances finite.  Sets the status word (first bad index).
__global__ void k_2b_validate(int64_t n_atoms, int64_t n_bonds, TwoBodyDev tb, DevStatus *st) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    if (i0 == 0 && (tb.bond_ptr[0] != 0 || tb.bond_ptr[n_atoms] != n_bonds)) set_status(st, GAP_ERR_INVALID, 0);
    for (int64_t a = i0; a < n_atoms; a += stride)
        if (tb.bond_ptr[a + 1] < tb.bond_ptr[a]) set_status(st, GAP_ERR_INVALID, a);
    for (int64_t b = i0; b < n_bonds; b += stride)
        if (!(tb.bond_r[b] > 0.0) || !isfinite(tb.bond_r[b])) set_status(st, GAP_ERR_INVALID, b);
    for (int64_t t = i0; t < tb.M2; t += stride)
        if (!isfinite(tb.sparse_r[t])) set_status(st, GAP_ERR_INVALID, t);
}

}  // namespace

cudaError_t launch_2b_validate(int64_t n_atoms, int64_t n_bonds, const TwoBodyDev &tb, DevStatus *st, cudaStream_t s) {
    k_2b_validate<<<304, 256, 0, s>>>(n_atoms, n_bonds, tb, st);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_2b_rows(const Dims &dm, const int64_t *cfg_ptr, const TwoBodyDev &tb, const double *sigma, T *A,
                           float *Aacc, double *E64, cudaStream_t s) {
    if (tb.M2 <= 0) return cudaSuccess;
    k_2b_cfg_rows<T><<<(unsigned)dm.n_cfg, 64, 0, s>>>(dm.n_cfg, dm.n_atoms, cfg_ptr, tb, sigma, dm.virials, A, dm.ld,
                                                        Aacc, E64, dm.M);
    if (dm.forces)
        k_2b_force_rows<T><<<(unsigned)ceil_div(dm.n_atoms * 32, 256), 256, 0, s>>>(dm.n_cfg, dm.n_atoms, tb, sigma, A,
                                                                                    dm.ld, Aacc, dm.M);
    return cudaGetLastError();
}
template cudaError_t launch_2b_rows<double>(const Dims &, const int64_t *, const TwoBodyDev &, const double *, double *,
                                            float *, double *, cudaStream_t);
template cudaError_t launch_2b_rows<float>(const Dims &, const int64_t *, const TwoBodyDev &, const double *, float *,
                                           float *, double *, cudaStream_t);

cudaError_t launch_2b_kmm(const TwoBodyDev &tb, double jitter, double *K, int64_t M, cudaStream_t s) {
    if (tb.M2 <= 0) return cudaSuccess;
    k_2b_kmm<<<(unsigned)ceil_div(tb.M2 * tb.M2, 256), 256, 0, s>>>(tb, jitter, K, M);
    return cudaGetLastError();
}

cudaError_t launch_2b_predict(int64_t n_cfg, int64_t n_atoms, const int64_t *cfg_ptr, const TwoBodyDev &tb,
                              const double *c2, double *E, double *F, double *V, cudaStream_t s) {
    if (tb.M2 <= 0) return cudaSuccess;
    k_2b_predict_cfg<<<(unsigned)ceil_div(n_cfg, 128), 128, 0, s>>>(n_cfg, cfg_ptr, tb, c2, E, V);
    if (F) k_2b_predict_atoms<<<(unsigned)ceil_div(n_atoms, 128), 128, 0, s>>>(n_atoms, tb, c2, F);
    return cudaGetLastError();
}

}  // namespace gap
