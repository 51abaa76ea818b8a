// Virial rows (Sec. II: derivatives of the energy with respect to a homogeneous
// lattice deformation) as force rows of pseudo-targets.
//
// A strain eps moves descriptor x_i by sum over the pairs p with source i of
// J_p eps u_p (u_p = r_a - r_i, first order), so the virial -dE/d eps of
// configuration A, symmetrised, in Voigt order v = (xx, yy, zz, yz, xz, xy), is
//     V_{A,v} = -sum_{i in A} (G_i^v . grad eps(x_i)),
//     G_i^v   = sum_{p: src(p) = i} (1/2) (J_p[alpha] u_p[beta] + J_p[beta] u_p[alpha])
// with (alpha, beta) the two indices of v.  That is the force-row formula with
// "pairs" (target (A, h), source i) and "Jacobians" G_i^{3h + alpha}: each
// configuration becomes two pseudo-targets, h = 0 for (xx, yy, zz) and h = 1 for
// (yz, xz, xy), whose pseudo-pairs are its atoms in order.  The force-row kernels
// then produce the virial rows (and predictions) unchanged, with row base
// n_cfg + 3 n_atoms.  Pseudo-pair order: pseudo-target t = 2A + h holds the
// pseudo-pairs [2 cfg_ptr[A] + h n_A, 2 cfg_ptr[A] + (h + 1) n_A), one per atom of A.
#include "gap_internal.cuh"

namespace gap {
namespace {

// Pseudo-pair index arrays, one thread per atom i (configuration A = atom_cfg[i]).
__global__ void k_virial_index(int64_t n_cfg, int64_t n_atoms, const int64_t *__restrict__ cfg_ptr,
                               const int64_t *__restrict__ atom_cfg, int64_t *__restrict__ vp_ptr,
                               int64_t *__restrict__ vp_src, int64_t *__restrict__ vp_tgt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cfg) {
        const int64_t b = cfg_ptr[i], nA = cfg_ptr[i + 1] - b;
        vp_ptr[2 * i] = 2 * b;
        vp_ptr[2 * i + 1] = 2 * b + nA;
    }
    if (i == 0) vp_ptr[2 * n_cfg] = 2 * n_atoms;
    if (i >= n_atoms) return;
    const int64_t A = atom_cfg[i], b = cfg_ptr[A], nA = cfg_ptr[A + 1] - b, k = i - b;
    vp_src[2 * b + k] = i;
    vp_tgt[2 * b + k] = 2 * A;
    vp_src[2 * b + nA + k] = i;
    vp_tgt[2 * b + nA + k] = 2 * A + 1;
}

// G (FP64, [2 n_atoms][3][d] in pseudo-pair order): one warp per (atom i, 128-wide slice
// of d), lanes on 4 consecutive entries each.  The warp walks the pairs of i's
// configuration in index order, 32 at a time, and adds those whose source is i: the
// sums run in pair order, so G does not depend on the schedule.
constexpr int kVcols = 128;
__global__ void __launch_bounds__(256) k_virial_jacobians(int64_t n_atoms, int64_t d, const int64_t *__restrict__ cfg_ptr,
                                                          const int64_t *__restrict__ atom_cfg,
                                                          const int64_t *__restrict__ pair_ptr,
                                                          const int64_t *__restrict__ pair_src,
                                                          const double *__restrict__ J,
                                                          const double *__restrict__ pair_u, double *__restrict__ G) {
    const int lane = threadIdx.x & 31;
    const int64_t n_sl = (d + kVcols - 1) / kVcols;
    const int64_t n_work = n_atoms * n_sl;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wk < n_work; wk += nwarps) {
        const int64_t i = wk / n_sl, k0 = (wk % n_sl) * kVcols + 4 * lane;
        const int64_t A = atom_cfg[i], b = cfg_ptr[A], nA = cfg_ptr[A + 1] - b;
        const int64_t q0 = pair_ptr[b], q1 = pair_ptr[b + nA];
        double v[6][4];
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int u = 0; u < 4; ++u) v[c][u] = 0.0;
        for (int64_t qb = q0; qb < q1; qb += 32) {
            const int64_t q = qb + lane;
            unsigned m = __ballot_sync(0xffffffffu, q < q1 && pair_src[q] == i);
            while (m) {  // matching pairs in increasing index
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                const int64_t p = qb + bit;
                const double u0 = pair_u[3 * p], u1 = pair_u[3 * p + 1], u2 = pair_u[3 * p + 2];
                const double *j0 = J + (3 * p) * d, *j1 = j0 + d, *j2 = j1 + d;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t k = k0 + u;
                    if (k >= d) break;
                    const double a0 = j0[k], a1 = j1[k], a2 = j2[k];
                    v[0][u] += a0 * u0;
                    v[1][u] += a1 * u1;
                    v[2][u] += a2 * u2;
                    v[3][u] += 0.5 * (a1 * u2 + a2 * u1);
                    v[4][u] += 0.5 * (a0 * u2 + a2 * u0);
                    v[5][u] += 0.5 * (a0 * u1 + a1 * u0);
                }
            }
        }
        const int64_t pp0 = 2 * b + (i - b), pp1 = pp0 + nA;  // pseudo-pairs (A, h = 0) and (A, h = 1)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + u;
            if (k >= d) break;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                G[(3 * pp0 + c) * d + k] = v[c][u];
                G[(3 * pp1 + c) * d + k] = v[3 + c][u];
            }
        }
    }
}

}  // namespace

cudaError_t launch_virial_pseudo_pairs(const Dims &dm, const int64_t *cfg_ptr, const int64_t *atom_cfg,
                                       const int64_t *pair_ptr, const int64_t *pair_src, const double *J,
                                       const double *pair_u, int64_t *vp_ptr, int64_t *vp_src, int64_t *vp_tgt,
                                       double *G, cudaStream_t s) {
    const int64_t n = std::max(dm.n_cfg, dm.n_atoms);
    k_virial_index<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(dm.n_cfg, dm.n_atoms, cfg_ptr, atom_cfg, vp_ptr, vp_src,
                                                              vp_tgt);
    const int64_t warps = dm.n_atoms * ceil_div(dm.d, kVcols);
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps, 8), 16 * 152));
    k_virial_jacobians<<<nb, 256, 0, s>>>(dm.n_atoms, dm.d, cfg_ptr, atom_cfg, pair_ptr, pair_src, J, pair_u, G);
    return cudaGetLastError();
}

Dims virial_dims(const Dims &dm) {
    Dims v = dm;
    v.n_atoms = 2 * dm.n_cfg;            // pseudo-targets
    v.n_pairs = 2 * dm.n_atoms;          // pseudo-pairs
    v.n_cfg = dm.n_cfg + 3 * dm.n_atoms; // row base of the virial rows
    v.forces = true;
    return v;
}

}  // namespace gap
