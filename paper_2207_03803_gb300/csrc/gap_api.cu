// C-ABI of libgap (declarations and contracts in include/gap.h).
//
// Phases (Sec. II of arXiv:2207.03803):
//   gap_assemble : data rows Sigma^{-1/2} K_NM (Eqs. 6, 7) and b (Eq. 8)
//   gap_factor   : K_MM + jitter, Cholesky K_MM = U^T U, stack U (Eq. 7), Householder QR
//   gap_solve    : c = R^{-1} Q^T b (Eq. 12); in the mixed precisions, FP64
//                  refinement of c against the FP32-accurate design matrix
//   gap_predict  : energies and forces of the fitted model (Eqs. 1, 2)
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "gap_internal.cuh"
#include "tc_gemm.cuh"

namespace gap {

gap_status fail(gap_ctx *c, gap_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

gap_status cuda_fail(gap_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") at " + where;
    if (c) c->err = m;
    return e == cudaErrorMemoryAllocation ? GAP_ERR_NOMEM : GAP_ERR_CUDA;
}

namespace {

constexpr int kQrColBlocks = 304;
constexpr int kQrRowBlocks = 64;
constexpr int kQNB = 32;

bool is_mixed(gap_precision p) {
    return p == GAP_PREC_MIXED_BF16 || p == GAP_PREC_MIXED_TF32 || p == GAP_PREC_MIXED_FP16;
}
// tensor-core operand scheme of a mixed precision's assembly
TcMode tc_mode(gap_precision p) {
    return p == GAP_PREC_MIXED_TF32 ? TcMode::TF32 : (p == GAP_PREC_MIXED_FP16 ? TcMode::FP16 : TcMode::BF16);
}

int64_t data_rows(const gap_problem *p) {
    bool forces = p->pair_ptr != nullptr && p->n_pairs > 0;
    bool virials = forces && p->pair_u != nullptr;
    return p->n_cfg + (forces ? 3 * p->n_atoms : 0) + (virials ? 6 * p->n_cfg : 0);
}

gap_status check_scalars(gap_ctx *c, const gap_problem *p, bool need_targets) {
    if (!p) return fail(c, GAP_ERR_INVALID, "problem is NULL");
    if (p->n_cfg < 1 || p->n_atoms < 1 || p->d < 1 || p->n_sparse < 1 || p->n_pairs < 0)
        return fail(c, GAP_ERR_INVALID, "sizes must be positive (n_cfg, n_atoms, d, n_sparse) and n_pairs >= 0");
    if (p->zeta < 1 || p->zeta > 63) return fail(c, GAP_ERR_INVALID, "zeta must be an integer in 1..63");
    if (!isfinite(p->delta) || !isfinite(p->jitter) || p->jitter < 0)
        return fail(c, GAP_ERR_INVALID, "delta must be finite and jitter finite and >= 0");
    if (p->memory != GAP_MEM_DEVICE && p->memory != GAP_MEM_HOST)
        return fail(c, GAP_ERR_INVALID, "memory must be GAP_MEM_DEVICE or GAP_MEM_HOST");
    if (!p->cfg_ptr || !p->X || !p->Xs) return fail(c, GAP_ERR_INVALID, "cfg_ptr, X and Xs are required");
    if (need_targets && (!p->y || !p->sigma)) return fail(c, GAP_ERR_INVALID, "y and sigma are required");
    if ((p->atom_species == nullptr) != (p->sparse_species == nullptr))
        return fail(c, GAP_ERR_INVALID, "atom_species and sparse_species must both be given or both be NULL");
    bool forces = p->pair_ptr != nullptr && p->n_pairs > 0;
    if (forces && (!p->pair_src || !p->J)) return fail(c, GAP_ERR_INVALID, "force rows need pair_src and J");
    if (!forces && p->n_pairs > 0) return fail(c, GAP_ERR_INVALID, "n_pairs > 0 needs pair_ptr");
    if (!forces && p->pair_u) return fail(c, GAP_ERR_INVALID, "virial rows (pair_u) need pair data");
    if (p->n_sparse_2b < 0 || p->n_bonds < 0) return fail(c, GAP_ERR_INVALID, "n_sparse_2b and n_bonds must be >= 0");
    if (p->n_sparse_2b > 0) {
        if (!p->bond_ptr || !p->sparse_r || (p->n_bonds > 0 && (!p->bond_r || !p->bond_u)))
            return fail(c, GAP_ERR_INVALID, "a two-body block needs bond_ptr, sparse_r, and bond_r, bond_u for its bonds");
        if (!isfinite(p->delta_2b) || !(p->theta_2b > 0.0) || !(p->width_2b > 0.0) || !(p->cutoff_2b >= p->width_2b) ||
            !isfinite(p->theta_2b) || !isfinite(p->cutoff_2b))
            return fail(c, GAP_ERR_INVALID, "two-body constants: delta_2b finite, theta_2b > 0, 0 < width_2b <= cutoff_2b");
    }
    return GAP_OK;
}

// Host-side structural validation of a host-memory problem: the configuration and pair
// pointers (O(n_cfg + n_atoms)).  The per-row and per-pair checks (sigma > 0, each pair
// source in its target's configuration, species >= 0) run on the device on the staged
// copies, as for device-memory problems, before any kernel indexes with them.
gap_status validate_host(gap_ctx *c, const gap_problem *p, bool need_targets) {
    (void)need_targets;
    const int64_t *cp = p->cfg_ptr;
    if (cp[0] != 0 || cp[p->n_cfg] != p->n_atoms) return fail(c, GAP_ERR_INVALID, "cfg_ptr must run from 0 to n_atoms");
    for (int64_t j = 0; j < p->n_cfg; ++j)
        if (cp[j + 1] < cp[j]) return fail(c, GAP_ERR_INVALID, "cfg_ptr not monotone at " + std::to_string(j));
    if (p->pair_ptr && p->n_pairs > 0) {
        const int64_t *pp = p->pair_ptr;
        if (pp[0] != 0 || pp[p->n_atoms] != p->n_pairs)
            return fail(c, GAP_ERR_INVALID, "pair_ptr must run from 0 to n_pairs");
        for (int64_t a = 0; a < p->n_atoms; ++a)
            if (pp[a + 1] < pp[a]) return fail(c, GAP_ERR_INVALID, "pair_ptr not monotone at " + std::to_string(a));
    }
    if (p->n_sparse_2b > 0) {
        const int64_t *bp = p->bond_ptr;
        if (bp[0] != 0 || bp[p->n_atoms] != p->n_bonds) return fail(c, GAP_ERR_INVALID, "bond_ptr must run from 0 to n_bonds");
        for (int64_t a = 0; a < p->n_atoms; ++a)
            if (bp[a + 1] < bp[a]) return fail(c, GAP_ERR_INVALID, "bond_ptr not monotone at " + std::to_string(a));
    }
    return GAP_OK;
}

template <class T>
gap_status stage(gap_ctx *c, DevBuf &buf, const T *src, int64_t n, const T **dst) {
    GAP_CUDA(c, buf.ensure(sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
    GAP_CUDA(c, cudaMemcpyAsync(buf.p, src, sizeof(T) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    *dst = buf.as<T>();
    return GAP_OK;
}

// Device pointers of a problem (staged if it lives in host memory).
struct DevProblem {
    const int64_t *cfg_ptr, *pair_ptr, *pair_src;
    const double *X, *Xs, *J, *y, *sigma;
    const int32_t *atom_sp, *sparse_sp;
    const double *pair_u;  // virial rows: [n_pairs x 3] pair displacements, or null
    const int64_t *bond_ptr;                        // two-body block (or null)
    const double *bond_r, *bond_u, *sparse_r;
};

// J of a host problem in chunks on the ctx's copy stream, each chunk's completion an
// event (the assembly multiplies the chunks that have landed while the rest are copied).
// The copy stream first waits for the work already queued on the ctx's stream, which may
// still read the staging buffer.
gap_status stage_J_chunked(gap_ctx *c, const gap_problem *p, const double **dst) {
    const int64_t n_pairs = p->n_pairs, d = p->d, rJ = force_pack_rows(n_pairs);
    GAP_CUDA(c, c->h_J.ensure(sizeof(double) * (size_t)std::max<int64_t>(n_pairs * 3 * d, 1)));
    if (!c->cstream) GAP_CUDA(c, cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
    if (!c->ev_stage) GAP_CUDA(c, cudaEventCreateWithFlags(&c->ev_stage, cudaEventDisableTiming));
    for (auto &e : c->j_ev)
        if (!e) GAP_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    GAP_CUDA(c, cudaEventRecord(c->ev_stage, c->stream));
    GAP_CUDA(c, cudaStreamWaitEvent(c->cstream, c->ev_stage, 0));
    const int n = (int)std::min<int64_t>(8, rJ / 128);
    c->n_jchunks = n;
    for (int i = 0; i <= n; ++i) c->j_rows[i] = i == n ? rJ : round_up((int64_t)i * rJ / n, 128);
    double *J = c->h_J.as<double>();
    for (int i = 0; i < n; ++i) {
        // the pairs of this chunk's pair tiles (42 pairs per 128 packed rows)
        const int64_t p0 = std::min(n_pairs, c->j_rows[i] / 128 * kForcePairsPerTile);
        const int64_t p1 = std::min(n_pairs, c->j_rows[i + 1] / 128 * kForcePairsPerTile);
        if (p1 > p0)
            GAP_CUDA(c, cudaMemcpyAsync(J + p0 * 3 * d, p->J + p0 * 3 * d, sizeof(double) * (size_t)((p1 - p0) * 3 * d),
                                        cudaMemcpyHostToDevice, c->cstream));
        GAP_CUDA(c, cudaEventRecord(c->j_ev[i], c->cstream));
    }
    *dst = J;
    return GAP_OK;
}

// The J ring's FP64 slots and events for a host problem of descriptor length d.
gap_status ensure_ring(gap_ctx *c, int64_t d) {
    if (c->j_ring_direct)
        c->ring_J.release();  // a page-locked J is read in place: no slots
    else
        GAP_CUDA(c, c->ring_J.ensure(2 * sizeof(double) * 3 * (size_t)d * (size_t)ring_slot_pairs(c->j_ring_rows)));
    if (!c->cstream) GAP_CUDA(c, cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
    for (auto &e : c->ring_ev)
        if (!e) GAP_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->h_J.release();  // a J staged whole earlier is not needed any more
    return GAP_OK;
}

// skip_J: a host problem's J stays where it is (read through the J ring); dp->J is null.
gap_status to_device(gap_ctx *c, const gap_problem *p, bool need_targets, DevProblem *dp, bool chunk_J = false,
                     bool skip_J = false) {
    bool forces = p->pair_ptr != nullptr && p->n_pairs > 0;
    c->n_jchunks = 0;
    if (p->memory == GAP_MEM_DEVICE) {
        const bool tb = p->n_sparse_2b > 0;
        *dp = {p->cfg_ptr, forces ? p->pair_ptr : nullptr, forces ? p->pair_src : nullptr, p->X, p->Xs,
               forces ? p->J : nullptr, p->y, p->sigma, p->atom_species, p->sparse_species,
               forces ? p->pair_u : nullptr, tb ? p->bond_ptr : nullptr, tb ? p->bond_r : nullptr,
               tb ? p->bond_u : nullptr, tb ? p->sparse_r : nullptr};
        return GAP_OK;
    }
    gap_status st = validate_host(c, p, need_targets);
    if (st != GAP_OK) return st;
    *dp = {};
    int64_t N = data_rows(p);
    if ((st = stage(c, c->h_cfg_ptr, p->cfg_ptr, p->n_cfg + 1, &dp->cfg_ptr)) != GAP_OK) return st;
    if ((st = stage(c, c->h_X, p->X, p->n_atoms * p->d, &dp->X)) != GAP_OK) return st;
    dp->Xs = nullptr;  // staged by the caller into c->Xs when needed
    if (need_targets) {
        if ((st = stage(c, c->h_y, p->y, N, &dp->y)) != GAP_OK) return st;
        if ((st = stage(c, c->h_sigma, p->sigma, N, &dp->sigma)) != GAP_OK) return st;
    }
    if (p->atom_species) {
        if ((st = stage(c, c->h_atom_sp, p->atom_species, p->n_atoms, &dp->atom_sp)) != GAP_OK) return st;
    }
    if (forces) {
        if ((st = stage(c, c->h_pair_ptr, p->pair_ptr, p->n_atoms + 1, &dp->pair_ptr)) != GAP_OK) return st;
        if ((st = stage(c, c->h_pair_src, p->pair_src, p->n_pairs, &dp->pair_src)) != GAP_OK) return st;
        if (skip_J) {
            dp->J = nullptr;
            st = ensure_ring(c, p->d);
        } else {
            st = chunk_J ? stage_J_chunked(c, p, &dp->J) : stage(c, c->h_J, p->J, p->n_pairs * 3 * p->d, &dp->J);
        }
        if (st != GAP_OK) return st;
        if (p->pair_u && (st = stage(c, c->h_pair_u, p->pair_u, 3 * p->n_pairs, &dp->pair_u)) != GAP_OK) return st;
    }
    if (p->n_sparse_2b > 0) {
        if ((st = stage(c, c->h_bond_ptr, p->bond_ptr, p->n_atoms + 1, &dp->bond_ptr)) != GAP_OK) return st;
        if ((st = stage(c, c->h_bond_r, p->bond_r, p->n_bonds, &dp->bond_r)) != GAP_OK) return st;
        if ((st = stage(c, c->h_bond_u, p->bond_u, 3 * p->n_bonds, &dp->bond_u)) != GAP_OK) return st;
        if ((st = stage(c, c->h_sparse_r, p->sparse_r, p->n_sparse_2b, &dp->sparse_r)) != GAP_OK) return st;
    }
    return GAP_OK;
}

// The J ring's part of the tensor-core inputs (host problem p with dp->J null: the FP64
// slots; a device J is read in place).
gap_status set_ring(gap_ctx *c, const gap_problem *p, const DevProblem &dp, TcInputs &ti) {
    ti.ring_rows = c->j_ring_rows;
    if (!dp.J && p->memory == GAP_MEM_HOST) {
        ti.h_J = p->J;
        ti.h_pair_ptr = p->pair_ptr;
        ti.ring_buf = c->ring_J.as<double>();
        ti.ring_stream = c->cstream;
        ti.ring_ev = c->ring_ev;
        if (c->j_ring_direct) {
            // read in place: the first and the last byte must be page-locked host memory that
            // the device sees at the same address (the caller locks the whole array)
            const char *first = (const char *)p->J;
            const char *last = first + sizeof(double) * 3 * (size_t)p->d * (size_t)p->n_pairs - 1;
            cudaPointerAttributes a0{}, a1{};
            if (cudaPointerGetAttributes(&a0, first) != cudaSuccess ||
                cudaPointerGetAttributes(&a1, last) != cudaSuccess || a0.type != cudaMemoryTypeHost ||
                a1.type != cudaMemoryTypeHost || a0.devicePointer != (void *)first || a1.devicePointer != (void *)last) {
                cudaGetLastError();
                return fail(c, GAP_ERR_INVALID,
                            "j_ring_direct needs J in page-locked host memory mapped at the same address");
            }
            ti.h_J_direct = true;
        }
    }
    return GAP_OK;
}

// K_MM's diagonal blocks for the blocked Cholesky.  Sparse points of different species do
// not covary, nor do the two-body block's with the SOAP ones.  When each species' sparse
// points are contiguous and no species appears twice, K_MM is block diagonal with those
// runs as blocks (and the two-body block after them); otherwise one block.
gap_status set_kmm_blocks(gap_ctx *c, const gap_problem *p) {
    const Dims &dm = c->dm;
    c->kmm_ends.clear();
    if (dm.species) {
        std::vector<int32_t> sp((size_t)dm.Ms);
        GAP_CUDA(c, cudaMemcpyAsync(sp.data(), p->sparse_species, sizeof(int32_t) * (size_t)dm.Ms,
                                    p->memory == GAP_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost,
                                    c->stream));
        GAP_CUDA(c, cudaStreamSynchronize(c->stream));
        std::vector<int32_t> seen;
        for (int64_t i = 1; i <= dm.Ms; ++i)
            if (i == dm.Ms || sp[(size_t)i] != sp[(size_t)i - 1]) {
                const int32_t t = sp[(size_t)i - 1];
                if (std::find(seen.begin(), seen.end(), t) != seen.end() || seen.size() >= 64) {
                    c->kmm_ends.clear();  // a species in two runs (or too many runs): one block
                    break;
                }
                seen.push_back(t);
                c->kmm_ends.push_back(i);
            }
        if (c->kmm_ends.empty()) c->kmm_ends.push_back(dm.Ms);
    } else {
        c->kmm_ends.push_back(dm.Ms);
    }
    if (dm.M2 > 0) c->kmm_ends.push_back(dm.M);
    return GAP_OK;
}

// The two-body block of problem p on the device: its bonds (dp) and the sparse distances
// and constants sr, p (the fit's), its columns after the Ms SOAP sparse points.
TwoBodyDev two_body_dev(const gap_problem *p, const DevProblem &dp, const double *sr, int64_t Ms) {
    TwoBodyDev tb{};
    tb.bond_ptr = dp.bond_ptr;
    tb.bond_r = dp.bond_r;
    tb.bond_u = dp.bond_u;
    tb.sparse_r = sr;
    tb.M2 = p->n_sparse_2b;
    tb.col0 = Ms;
    tb.delta2 = p->delta_2b * p->delta_2b;
    tb.inv2t2 = 1.0 / (2.0 * p->theta_2b * p->theta_2b);
    tb.rc = p->cutoff_2b;
    tb.w = p->width_2b;
    return tb;
}

gap_status read_status(gap_ctx *c, const char *what) {
    GAP_CUDA(c, cudaMemcpyAsync(c->h_status, c->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
    GAP_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->h_status->code != 0) {
        gap_status s = (gap_status)c->h_status->code;
        char buf[160];
        snprintf(buf, sizeof buf, "%s: status %d at index %lld", what, c->h_status->code,
                 (long long)c->h_status->index);
        return fail(c, s, buf);
    }
    return GAP_OK;
}

gap_status clear_status(gap_ctx *c) {
    GAP_CUDA(c, c->status.ensure(sizeof(DevStatus)));
    GAP_CUDA(c, cudaMemsetAsync(c->status.p, 0, sizeof(DevStatus), c->stream));
    return GAP_OK;
}

size_t elt_size(gap_precision p) { return p == GAP_PREC_FP64 ? 8 : 4; }

Dims make_dims(const gap_problem *p) {
    Dims dm{};
    dm.n_cfg = p->n_cfg;
    dm.n_atoms = p->n_atoms;
    dm.d = p->d;
    dm.forces = p->pair_ptr != nullptr && p->n_pairs > 0;
    dm.n_pairs = dm.forces ? p->n_pairs : 0;
    dm.Ms = p->n_sparse;
    dm.M2 = p->n_sparse_2b > 0 ? p->n_sparse_2b : 0;
    dm.M = dm.Ms + dm.M2;
    dm.N = data_rows(p);
    dm.rows = dm.N + dm.M;
    dm.ld = round_up(dm.rows, 128);
    dm.zeta = p->zeta;
    dm.delta = p->delta;
    dm.jitter = p->jitter;
    dm.species = p->atom_species != nullptr;
    dm.virials = dm.forces && p->pair_u != nullptr;
    return dm;
}

// The pseudo-pair buffers of the virial rows (k_virial.cu) for a problem of these sizes.
gap_status ensure_virial_buffers(gap_ctx *c, const Dims &dm) {
    GAP_CUDA(c, c->vp_ptr.ensure(sizeof(int64_t) * (size_t)(2 * dm.n_cfg + 1)));
    GAP_CUDA(c, c->vp_src.ensure(sizeof(int64_t) * (size_t)(2 * dm.n_atoms)));
    GAP_CUDA(c, c->vp_tgt.ensure(sizeof(int64_t) * (size_t)(2 * dm.n_atoms)));
    GAP_CUDA(c, c->vG.ensure(sizeof(double) * (size_t)(6 * dm.n_atoms * dm.d)));
    return GAP_OK;
}

}  // namespace
}  // namespace gap

namespace gap {
namespace {
// The mixed precisions factor K_MM with a double-float trailing matrix while its
// entries (at most delta^2 + jitter in size) sit well inside the FP32 exponent range.
bool chol_df(gap_precision prec, const Dims &dm) {
    const double top = dm.delta * dm.delta + dm.jitter;
    return is_mixed(prec) && top > 1e-18 && top < 1e18;
}

template <class T>
gap_status factor_qr(gap_ctx *c, int passes, int cqr);

// The fit's two-body model (sparse distances and constants; no bonds).
TwoBodyDev fit_two_body(const gap_ctx *c) {
    TwoBodyDev tb{};
    tb.sparse_r = c->sparse_r.as<double>();
    tb.M2 = c->dm.M2;
    tb.col0 = c->dm.Ms;
    tb.delta2 = c->tb_delta * c->tb_delta;
    tb.inv2t2 = 1.0 / (2.0 * c->tb_theta * c->tb_theta);
    tb.rc = c->tb_cutoff;
    tb.w = c->tb_width;
    return tb;
}

template <class T>
gap_status factor_impl(gap_ctx *c) {
    const Dims &dm = c->dm;
    cudaStream_t s = c->stream;
    GAP_CUDA(c, cudaEventRecord(c->ev[2], s));
    if (clear_status(c) != GAP_OK) return GAP_ERR_CUDA;
    DevStatus *dst = c->status.as<DevStatus>();
    GAP_CUDA(c, c->Kmm.ensure(sizeof(double) * dm.M * dm.M));
    const int32_t *ssp = dm.species ? c->sparse_sp.as<int32_t>() : nullptr;
    c->prof.begin(GAP_PROF_KMM_CHOL);
    const bool mixed = is_mixed(c->prec);
    if (mixed) GAP_CUDA(c, c->rinv.ensure(rinv_bytes(dm.M, dm.d)));  // free until the refinement
    GAP_CUDA(c, launch_kmm(dm, c->Xs.as<double>(), ssp, c->Kmm.as<double>(), s, mixed,
                           mixed ? c->rinv.as<float>() : nullptr));
    if (dm.M2 > 0) GAP_CUDA(c, launch_2b_kmm(fit_two_body(c), dm.jitter, c->Kmm.as<double>(), dm.M, s));
    if (chol_df(c->prec, dm)) {
        GAP_CUDA(c, cholesky_lower_df(c->Kmm.as<double>(), dm.M, c->rinv.as<float>(), dst, s, c->kmm_ends.data(),
                                      (int)c->kmm_ends.size()));
    } else {
        GAP_CUDA(c, cholesky_lower(c->Kmm.as<double>(), dm.M, dst, s, c->kmm_ends.data(), (int)c->kmm_ends.size()));
    }
    gap_status st = read_status(c, "Cholesky of K_MM + jitter met a non-positive pivot");
    if (st != GAP_OK) return st;
    T *A = c->A.as<T>();
    GAP_CUDA(c, launch_stack_u<T>(dm, c->Kmm.as<double>(), A, s));
    if (is_mixed(c->prec)) GAP_CUDA(c, launch_stack_u<float>(dm, c->Kmm.as<double>(), c->Aacc.as<float>(), s, true));
    c->prof.end();
    return factor_qr<T>(c, c->qr_passes, c->cqr_passes);
}

// Row blocks of the data rows [0, N) for a TSQR factorisation: up to `want` blocks of
// whole 128-row tiles (the last one takes the remainder), none shorter than M + 128 rows,
// so that every block is tall for its QR and starts on a tile of A.  The tensor-core
// updates of a block add their 128-row tiles through a map of ld rows from the block's
// first row; a tile may run up to 127 rows past the block (adding zero there), so the
// last one must still end inside the column: ld >= N + 128.  Returns the block count, 0
// when N or ld is too short for that (one QR of the whole matrix then).
int tsqr_plan(int64_t N, int64_t M, int64_t ld, int want, int64_t *r0, int64_t *n) {
    if (want < 1 || N < M + 128 || ld < N + 128) return 0;
    int G = std::min(want, kTsqrMax);
    while (G > 1 && (N / G) / 128 * 128 < M + 128) --G;
    const int64_t nb = G > 1 ? (N / G) / 128 * 128 : N;
    for (int g = 0; g < G; ++g) {
        r0[g] = g * nb;
        n[g] = g + 1 < G ? nb : N - g * nb;
    }
    return G;
}

// The QR of c->A (one matrix, no TSQR) through a CUDA graph of its launches when the option
// "graphs" is on.  Its launch sequence depends only on the problem's shape and the ctx's
// buffers, so a graph captured once replays it with one launch: the thousand-odd kernels of a
// small fit's QR no longer take the driver's launch path one by one (lanes of a batch
// contend for it).  A key is captured the second time it is factored (the first call runs
// the kernels directly and settles one-time setup); a capture that fails runs directly.
template <class T>
cudaError_t qr_graphed(gap_ctx *c, T *A, int passes, int cqr, void *outer, int *code) {
    const Dims &dm = c->dm;
    cudaStream_t s = c->stream;
    auto run_on = [&](cudaStream_t st, Prof *prof) {
        return householder_qr<T>(A, dm.rows, dm.M, dm.ld, std::min(c->qr_nb, kQNB), c->tau.as<T>(), c->T.as<T>(),
                                 c->part.as<T>(), c->diagrow.as<T>(), c->Wpart.as<T>(), c->Wred.as<T>(), kQrRowBlocks, st,
                                 prof, outer, outer ? code : nullptr, passes, cqr);
    };
    auto run = [&](Prof *prof) { return run_on(s, prof); };
    if (!c->use_graphs) return run(&c->prof);
    const std::vector<uintptr_t> key = {
        (uintptr_t)dm.rows, (uintptr_t)dm.M, (uintptr_t)dm.ld, (uintptr_t)sizeof(T), (uintptr_t)passes, (uintptr_t)cqr,
        (uintptr_t)c->qr_nb, (uintptr_t)A, (uintptr_t)c->tau.p, (uintptr_t)c->T.p, (uintptr_t)c->part.p,
        (uintptr_t)c->diagrow.p, (uintptr_t)c->Wpart.p, (uintptr_t)c->Wred.p, (uintptr_t)outer, (uintptr_t)code};
    gap_ctx::QrGraph *hit = nullptr;
    for (auto &g : c->qr_graphs)
        if (g.key == key) hit = &g;
    if (hit == nullptr) {
        if (c->qr_graphs.size() >= 8) {  // the least used one makes room
            auto lo = std::min_element(c->qr_graphs.begin(), c->qr_graphs.end(),
                                       [](const gap_ctx::QrGraph &a, const gap_ctx::QrGraph &b) { return a.uses < b.uses; });
            if (lo->exec) cudaGraphExecDestroy(lo->exec);
            c->qr_graphs.erase(lo);
        }
        c->qr_graphs.push_back({key, nullptr, 0});
        hit = &c->qr_graphs.back();
    }
    hit->uses += 1;
    if (!hit->exec && hit->uses >= 2) {
        // captured on a stream of the ctx's own (the caller's may be the legacy default stream,
        // which cannot capture); the graph is then launched on the ctx's stream
        if (!c->gstream && cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess)
            c->gstream = nullptr;
        cudaGraph_t g = nullptr;
        if (c->gstream && cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t e = run_on(c->gstream, nullptr);
            const cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
            if (e == cudaSuccess && e2 == cudaSuccess && g &&
                cudaGraphInstantiate(&hit->exec, g, 0) != cudaSuccess)
                hit->exec = nullptr;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();  // a failed capture leaves no error behind: the kernels run directly
    }
    if (!hit->exec) return run(&c->prof);
    c->prof.begin(GAP_PROF_QR_UPDATE);  // the whole QR: panels and updates in one graph
    const cudaError_t e = cudaGraphLaunch(hit->exec, s);
    c->prof.end();
    return e;
}

// The QR of the stacked matrix in c->A (passes: tensor-core passes of the FP32 trailing
// updates; cqr: CholeskyQR passes of the FP32 panels).  With the "tsqr_shards" option the
// data rows are factored as the row-block distribution of Sec. III-B: every block of rows
// [r0, r0 + n) gets its own Householder QR in place, R_g with Q_g^T b_g in column M; the
// stack S = [R_1; ...; R_G; U] then has the same normal matrix and the same
// S^T [Q^T b] as [A | b] (the solution does not depend on which rows share a block),
// and the QR of S gives R and Q^T b.  The residual of the fit is spread over the block
// tails and the tail of S.
template <class T>
gap_status factor_qr(gap_ctx *c, int passes, int cqr) {
    const Dims &dm = c->dm;
    cudaStream_t s = c->stream;
    gap_status st = GAP_OK;
    T *A = c->A.as<T>();
    c->qr_lean = sizeof(T) == 4 && c->qr_two_level && (passes == 1 || cqr == 1);
    const size_t e = sizeof(T);
    const int64_t nc = dm.M + 1;
    c->tsqr_used = c->tsqr_shards > 0 ? tsqr_plan(dm.N, dm.M, dm.ld, c->tsqr_shards, c->tsqr_r0, c->tsqr_n) : 0;
    c->tsqr_ext = false;
    const int G = c->tsqr_used;
    const int64_t s_rows = (G + 1) * dm.M, s_ld = round_up(s_rows, 128);
    GAP_CUDA(c, c->tau.ensure(e * dm.M));
    GAP_CUDA(c, c->T.ensure(e * kQNB * kQNB));
    GAP_CUDA(c, c->part.ensure(e * std::max<size_t>(2 * kQrColBlocks * (kQNB + 1), 152 * kQNB * kQNB)));
    GAP_CUDA(c, c->diagrow.ensure(e * 2 * (kQNB + 1)));
    GAP_CUDA(c, c->Wpart.ensure(e * kQrRowBlocks * kQNB * nc));
    GAP_CUDA(c, c->Wred.ensure(e * kQNB * nc));
    void *outer = nullptr;
    if (sizeof(T) == 4 && c->qr_two_level) {
        GAP_CUDA(c, c->qr_outer.ensure(qr_outer_workspace_bytes(G ? std::max(dm.rows, s_rows) : dm.rows, dm.M)));
        outer = c->qr_outer.p;
    }
    int *code = &c->status.as<DevStatus>()->code;
    auto qr = [&](T *X, int64_t rows, int64_t ld) {
        return householder_qr<T>(X, rows, dm.M, ld, std::min(c->qr_nb, kQNB), c->tau.as<T>(), c->T.as<T>(),
                                 c->part.as<T>(), c->diagrow.as<T>(), c->Wpart.as<T>(), c->Wred.as<T>(), kQrRowBlocks,
                                 s, &c->prof, outer, outer ? code : nullptr, passes, cqr);
    };
    c->r_ld = dm.ld;
    if (G == 0) {
        GAP_CUDA(c, qr_graphed<T>(c, A, passes, cqr, outer, code));
    } else {
        GAP_CUDA(c, c->tsqr.ensure(e * s_ld * nc));
        T *S = c->tsqr.as<T>();
        GAP_CUDA(c, cudaMemsetAsync(S, 0, e * s_ld * nc, s));  // padding rows of the stack stay zero
        for (int g = 0; g < G; ++g) {
            GAP_CUDA(c, qr(A + c->tsqr_r0[g], c->tsqr_n[g], dm.ld));
            GAP_CUDA(c, tsqr_gather<T>(A, dm.ld, c->tsqr_r0[g], dm.M, S, s_ld, g * dm.M, false, s));
        }
        GAP_CUDA(c, tsqr_gather<T>(A, dm.ld, dm.N, dm.M, S, s_ld, G * dm.M, true, s));  // U, right-hand side 0
        GAP_CUDA(c, qr(S, s_rows, s_ld));
        c->r_ld = s_ld;
    }
    if (outer) {
        GAP_CUDA(c, cudaMemcpyAsync(c->h_status, c->status.p, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
        GAP_CUDA(c, cudaStreamSynchronize(s));
        if (c->h_status->code == kStatusCqrFallback) {
            // a panel was too ill-conditioned for CholeskyQR2: refactor the FP32-accurate
            // matrix with the column-by-column Householder panels (one QR of the whole matrix)
            GAP_CUDA(c, acc_to_colmajor(c->Aacc.as<float>(), dm.ld, dm.M, c->A.as<float>(), s));
            GAP_CUDA(c, cudaMemsetAsync(c->status.p, 0, sizeof(DevStatus), s));
            GAP_CUDA(c, householder_qr<T>(A, dm.rows, dm.M, dm.ld, std::min(c->qr_nb, kQNB), c->tau.as<T>(),
                                          c->T.as<T>(), c->part.as<T>(), c->diagrow.as<T>(), c->Wpart.as<T>(),
                                          c->Wred.as<T>(), kQrRowBlocks, s, &c->prof, nullptr, nullptr, 3, 2));
            c->qr_fallbacks += 1;
            c->tsqr_used = 0;
            c->r_ld = dm.ld;
        }
        st = read_status(c, "QR update (tensor cores)");
        if (st != GAP_OK) return st;
    }
    GAP_CUDA(c, cudaEventRecord(c->ev[3], s));
    return GAP_OK;
}

// The matrix whose top M x (M+1) holds R and Q^T b after the last factorisation.
template <class T>
T *r_matrix(gap_ctx *c) {
    return c->tsqr_used ? c->tsqr.as<T>() : c->A.as<T>();
}
}  // namespace

namespace {

// vector workspace layout (FP64): x[M] q[M] s[M] p[M] g[M] | r[rows] t[rows] | scalars[16]
struct RefVecs {
    double *x, *q, *s, *p, *g, *r, *t, *sc;
};

template <class T>
gap_status solve_impl(gap_ctx *c, double *c_dev, gap_solve_info *info) {
    const Dims &dm = c->dm;
    cudaStream_t s = c->stream;
    const int64_t M = dm.M, rows = dm.rows;
    GAP_CUDA(c, cudaEventRecord(c->ev[4], s));
    // vectors | scalars | diagonal-block inverses of R | triangular-solve scratch | split residual
    const int64_t ninv = ceil_div(M, kTrsvBlock) * kTrsvBlock * kTrsvBlock;
    GAP_CUDA(c, c->vecs.ensure(sizeof(double) * (5 * M + 2 * rows + 16 + ninv + M + rows)));
    double *base = c->vecs.as<double>();
    RefVecs v{base, base + M, base + 2 * M, base + 3 * M, base + 4 * M, base + 5 * M, base + 5 * M + rows,
              base + 5 * M + 2 * rows};
    double *Dinv = base + 5 * M + 2 * rows + 16, *xs = Dinv + ninv;
    float *rsplit = reinterpret_cast<float *>(xs + M);
    if (clear_status(c) != GAP_OK) return GAP_ERR_CUDA;
    const T *A = c->A.as<T>();
    // c0 = R^{-1} (Q^T b)[0:M]; the transformed b sits in column M of the factored matrix
    const T *Rm = r_matrix<T>(c);
    const int64_t ldr = c->r_ld;
    c->prof.begin(GAP_PROF_SOLVE);
    GAP_CUDA(c, back_substitution<T>(Rm, M, ldr, Rm + M * ldr, v.x, Dinv, c->status.as<DevStatus>(), s));
    c->prof.end();
    gap_status st = read_status(c, "R has a zero or non-finite diagonal entry");
    if (st != GAP_OK) return st;
    GAP_CUDA(c, cudaEventRecord(c->ev[5], s));
    gap_solve_info inf{};
    double hsc[8] = {};
    if (!is_mixed(c->prec)) {
        // ||b - A c|| = ||(Q^T b)[M:rows]|| (Householder transforms preserve norms); after a
        // TSQR the tail is the block tails below each R_g plus the tail of the stack
        int64_t nr = 0;
        if (c->tsqr_ext) {  // merged blocks of other contexts: the stack's tail here, theirs summed
            nr = (int64_t)c->tsqr_used * M;
            GAP_CUDA(c, convert_to_f64(Rm + M * ldr + M, sizeof(T) == 4, nr, v.r, s));
        } else if (c->tsqr_used) {
            for (int g = 0; g < c->tsqr_used; ++g) {
                const int64_t r0 = c->tsqr_r0[g], n = c->tsqr_n[g] - M;
                GAP_CUDA(c, convert_to_f64(A + M * dm.ld + r0 + M, sizeof(T) == 4, n, v.r + nr, s));
                nr += n;
            }
            const int64_t n = (c->tsqr_used + 1) * M - M;
            GAP_CUDA(c, convert_to_f64(Rm + M * ldr + M, sizeof(T) == 4, n, v.r + nr, s));
            nr += n;
        } else {
            nr = rows - M;
            GAP_CUDA(c, convert_to_f64(A + M * dm.ld + M, sizeof(T) == 4, nr, v.r, s));
        }
        GAP_CUDA(c, vec_dot(v.r, v.r, nr, v.sc, s));
        GAP_CUDA(c, cudaMemcpyAsync(hsc, v.sc, sizeof(double), cudaMemcpyDeviceToHost, s));
        GAP_CUDA(c, cudaStreamSynchronize(s));
        inf.residual_norm = sqrt(hsc[0] + (c->tsqr_ext ? c->tsqr_ext_tail2 : 0.0));
        inf.converged = 1;
    } else {
        // Preconditioned CGLS in FP64 on min ||b - Aacc x||, right preconditioner R
        // from the FP32 QR (applied as the explicit W = R^{-1}), starting from the QR
        // solution.  Per iteration: u = W p; w = A^T A u and |A u|^2 in one pass over A;
        // x += alpha u; s -= alpha W^T w (the gradient W^T A^T r after r -= alpha A u).
        const float *Aa = c->Aacc.as<float>();
        const T *R = Rm;
        const double *b = c->b64.as<double>();
        double *sc = v.sc;  // 0 gamma, 1 |A u|^2, 2 gamma_new, 3 |u|^2, 4 |x|^2, 5 |r|^2
        c->prof.begin(GAP_PROF_REFINE);
        const int64_t ldw = round_up(M, 32);
        GAP_CUDA(c, c->rinv.ensure(rinv_bytes(M)));
        float *W = c->rinv.as<float>(), *Wt = W + ldw * M;
        GAP_CUDA(c, triangular_inverse((const float *)R, ldr, M, Dinv, W, Wt, ldw, s));
        GAP_CUDA(c, c->cg_ws.ensure(cgls_workspace_bytes(M)));
        void *cw = c->cg_ws.p;
        // A pass over the residual matrix: its first block of 32 rows (the energy rows, in
        // FP64 from the assembly's double-float epilogue, and the force rows that share the
        // block) in FP64, the fused pass over A_acc for the rows after it.
        const int64_t rh = std::min<int64_t>(rows, round_up(dm.n_cfg, ACC_RB));
        GAP_CUDA(c, c->head_t.ensure(cgls_head_bytes(rh, M)));
        int *code = &c->status.as<DevStatus>()->code;
        auto pass = [&](const double *u, const double *rhs, double *w, double *sq, bool df) -> cudaError_t {
            const bool tail = rows > rh;
            if (tail) {
                cudaError_t e = cgls_pass(Aa + acc_index(rh, 0, M + 1), rows - rh, M, u, rhs ? rhs + rh : nullptr, w,
                                          sq, cw, df, code, s);
                if (e != cudaSuccess) return e;
            }
            return cgls_head(c->E64.as<double>(), dm.n_cfg, Aa, rh, M, u, rhs, w, sq, c->head_t.as<double>(), tail, s);
        };
        // gradient at the QR solution from its true residual
        GAP_CUDA(c, pass(v.x, b, v.g, sc + 5, true));  // g = A^T (b - A x)
        GAP_CUDA(c, gemv_t<float>(W, M, M, ldw, v.g, v.s, rsplit, s));   // s = W^T g
        GAP_CUDA(c, cudaMemcpyAsync(v.p, v.s, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
        GAP_CUDA(c, vec_dot(v.s, v.s, M, sc + 0, s));
        int it = 0;
        bool conv = false;
        double rel = 0.0;
        for (it = 0; it < c->max_iter; ++it) {
            GAP_CUDA(c, gemv_t<float>(Wt, M, M, ldw, v.p, v.q, rsplit, s));  // u = W p
            GAP_CUDA(c, pass(v.q, nullptr, v.g, sc + 1, true));  // A^T A u, |A u|^2
            GAP_CUDA(c, gemv_t<float>(W, M, M, ldw, v.g, v.t, rsplit, s));  // W^T A^T A u
            GAP_CUDA(c, vec_axpy(+1.0, sc + 0, sc + 1, v.q, v.x, M, s));     // x += alpha u
            GAP_CUDA(c, vec_axpy(-1.0, sc + 0, sc + 1, v.t, v.s, M, s));     // s -= alpha W^T A^T A u
            GAP_CUDA(c, vec_dot(v.s, v.s, M, sc + 2, s));
            GAP_CUDA(c, vec_dot(v.q, v.q, M, sc + 3, s));
            GAP_CUDA(c, vec_dot(v.x, v.x, M, sc + 4, s));
            GAP_CUDA(c, cudaMemcpyAsync(hsc, sc, sizeof(double) * 5, cudaMemcpyDeviceToHost, s));
            GAP_CUDA(c, cudaStreamSynchronize(s));
            double alpha = hsc[1] != 0.0 ? hsc[0] / hsc[1] : 0.0;
            rel = hsc[4] > 0 ? alpha * sqrt(hsc[3]) / sqrt(hsc[4]) : 0.0;
            GAP_CUDA(c, vec_xpby(v.s, sc + 2, sc + 0, v.p, M, s));   // p = s + beta p
            GAP_CUDA(c, cudaMemcpyAsync(sc + 0, sc + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
            if (!(rel >= c->tol) || hsc[2] == 0.0) {
                conv = true;
                ++it;
                break;
            }
        }
        // true residual of the final iterate
        GAP_CUDA(c, pass(v.x, b, nullptr, sc + 5, true));
        c->prof.end();
        GAP_CUDA(c, cudaMemcpyAsync(hsc + 5, sc + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
        GAP_CUDA(c, cudaStreamSynchronize(s));
        st = read_status(c, "refinement pass");
        if (st != GAP_OK) return st;
        inf.iterations = it;
        inf.converged = conv ? 1 : 0;
        inf.rel_update = rel;
        inf.residual_norm = sqrt(hsc[5]);
    }
    GAP_CUDA(c, cudaMemcpyAsync(c_dev, v.x, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
    GAP_CUDA(c, cudaEventRecord(c->ev[6], s));
    GAP_CUDA(c, cudaEventSynchronize(c->ev[6]));
    float t0 = 0, t1 = 0, t2 = 0, t3 = 0;
    // a phase whose events were not recorded reads 0 (its error is cleared, so that it does
    // not surface at a later launch check)
    if (cudaEventElapsedTime(&t0, c->ev[0], c->ev[1]) != cudaSuccess) t0 = 0.f;
    if (cudaEventElapsedTime(&t1, c->ev[2], c->ev[3]) != cudaSuccess) t1 = 0.f;
    if (cudaEventElapsedTime(&t2, c->ev[4], c->ev[5]) != cudaSuccess) t2 = 0.f;
    if (cudaEventElapsedTime(&t3, c->ev[5], c->ev[6]) != cudaSuccess) t3 = 0.f;
    (void)cudaGetLastError();
    inf.time_ms[0] = t0;
    inf.time_ms[1] = t1;
    inf.time_ms[2] = t2;
    inf.time_ms[3] = t3;
    if (info) *info = inf;
    if (is_mixed(c->prec) && !inf.converged) {
        char buf[128];
        snprintf(buf, sizeof buf, "refinement stopped after %d iterations (relative update %.3e)", inf.iterations,
                 inf.rel_update);
        return fail(c, GAP_ERR_NOT_CONVERGED, buf);
    }
    return GAP_OK;
}
}  // namespace
}  // namespace gap

using namespace gap;

namespace {
// assemble -> factor -> solve of one problem on ctx c
gap_status run_fit(gap_ctx *c, const gap_problem *p, double *c_dev, gap_solve_info *info) {
    gap_status st = gap_assemble(c, p);
    if (st == GAP_OK) st = gap_factor(c);
    if (st == GAP_OK) st = gap_solve(c, c_dev, info);
    return st;
}

// worker contexts for gap_fit_batched: same precision and options, own streams
gap_status ensure_lanes(gap_ctx *c, int L) {
    while ((int)c->lanes.size() < L) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return fail(c, GAP_ERR_CUDA, "cudaStreamCreateWithFlags failed");
        gap_ctx *w = nullptr;
        gap_status st = gap_create(&w, c->prec, s);
        if (st != GAP_OK) {
            cudaStreamDestroy(s);
            return fail(c, st, "creating a batch worker context failed");
        }
        w->owns_stream = true;
        c->lanes.push_back(w);
    }
    for (gap_ctx *w : c->lanes) {
        w->max_iter = c->max_iter;
        w->tol = c->tol;
        w->qr_nb = c->qr_nb;
        w->qr_two_level = c->qr_two_level;
        w->qr_passes = c->qr_passes;
        w->force_walk = c->force_walk;
        w->cqr_passes = c->cqr_passes;
        w->tsqr_shards = c->tsqr_shards;
        w->j_ring_rows = c->j_ring_rows;
        w->j_ring_direct = c->j_ring_direct;
        w->use_graphs = c->use_graphs;
    }
    return GAP_OK;
}
}  // namespace


extern "C" {

gap_status gap_create(gap_ctx **ctx, gap_precision prec, void *cuda_stream) {
    if (!ctx) return GAP_ERR_INVALID;
    *ctx = nullptr;
    if (prec != GAP_PREC_FP64 && !is_mixed(prec)) return GAP_ERR_INVALID;
    gap_ctx *c = new (std::nothrow) gap_ctx();
    if (!c) return GAP_ERR_NOMEM;
    c->prec = prec;
    c->stream = (cudaStream_t)cuda_stream;
    c->prof.s = c->stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaMallocHost((void **)&c->h_status, sizeof(DevStatus)) != cudaSuccess) {
        delete c;
        return GAP_ERR_CUDA;
    }
    for (auto &e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            delete c;
            return GAP_ERR_CUDA;
        }
    *ctx = c;
    return GAP_OK;
}

void gap_destroy(gap_ctx *c) {
    if (!c) return;
    for (gap_ctx *w : c->lanes) gap_destroy(w);
    c->lanes.clear();
    cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->Xs, &c->sparse_sp, &c->h_cfg_ptr, &c->h_X, &c->h_atom_sp, &c->h_pair_ptr, &c->h_pair_src,
                      &c->h_J, &c->h_y, &c->h_sigma, &c->atom_cfg, &c->pair_tgt, &c->A, &c->Aacc, &c->b64, &c->Wf,
                      &c->tc_ops, &c->pred_work, &c->Kmm, &c->tau, &c->T, &c->Wpart, &c->Wred, &c->part, &c->diagrow,
                      &c->status, &c->qr_outer, &c->vecs, &c->rinv, &c->cg_ws};
    for (DevBuf *b : bufs) b->release();
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->cstream) {
        cudaStreamSynchronize(c->cstream);
        cudaStreamDestroy(c->cstream);
    }
    if (c->ev_stage) cudaEventDestroy(c->ev_stage);
    for (auto &e : c->j_ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : c->ring_ev)
        if (e) cudaEventDestroy(e);
    for (auto &g : c->qr_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->owns_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *gap_last_error(const gap_ctx *c) { return c ? c->err.c_str() : "ctx is NULL"; }

gap_status gap_set_option(gap_ctx *c, const char *key, double value) {
    if (!c || !key) return GAP_ERR_INVALID;
    if (!strcmp(key, "max_iter")) {
        if (value < 0 || value > 10000) return fail(c, GAP_ERR_INVALID, "max_iter out of range");
        c->max_iter = (int)value;
    } else if (!strcmp(key, "tol")) {
        if (!(value > 0)) return fail(c, GAP_ERR_INVALID, "tol must be > 0");
        c->tol = value;
    } else if (!strcmp(key, "qr_two_level")) {
        c->qr_two_level = value != 0.0;
    } else if (!strcmp(key, "force_walk")) {
        if (value < 1 || value > 32 || value != (double)(int)value)
            return fail(c, GAP_ERR_INVALID, "force_walk must be an integer 1..32");
        c->force_walk = (int)value;
    } else if (!strcmp(key, "batch_lanes")) {
        if (value < 1 || value > 16) return fail(c, GAP_ERR_INVALID, "batch_lanes must be 1..16");
        c->batch_lanes = (int)value;
    } else if (!strcmp(key, "cqr_passes")) {
        if (value != 1.0 && value != 2.0) return fail(c, GAP_ERR_INVALID, "cqr_passes must be 1 or 2");
        c->cqr_passes = (int)value;
    } else if (!strcmp(key, "qr_passes")) {
        if (value != 1.0 && value != 3.0) return fail(c, GAP_ERR_INVALID, "qr_passes must be 1 or 3");
        c->qr_passes = (int)value;
    } else if (!strcmp(key, "tsqr_shards")) {
        if (value < 0 || value > kTsqrMax || value != (double)(int)value)
            return fail(c, GAP_ERR_INVALID, "tsqr_shards must be an integer 0..64");
        c->tsqr_shards = (int)value;
    } else if (!strcmp(key, "j_ring_rows")) {
        if (value < 0 || value > 1e12 || value != (double)(int64_t)value || ((int64_t)value) % 128 != 0)
            return fail(c, GAP_ERR_INVALID, "j_ring_rows must be 0 or a positive multiple of 128");
        if (value > 0 && !is_mixed(c->prec))
            return fail(c, GAP_ERR_INVALID, "the J ring is an option of the mixed precisions");
        c->j_ring_rows = (int64_t)value;
    } else if (!strcmp(key, "graphs")) {
        c->use_graphs = value != 0.0;
    } else if (!strcmp(key, "j_ring_direct")) {
        c->j_ring_direct = value != 0.0;
    } else if (!strcmp(key, "qr_nb")) {
        int nb = (int)value;
        if (nb < 16 || nb > 128 || nb % 16) return fail(c, GAP_ERR_INVALID, "qr_nb must be 16..128, multiple of 16");
        c->qr_nb = nb;
    } else {
        return fail(c, GAP_ERR_INVALID, std::string("unknown option ") + key);
    }
    return GAP_OK;
}

int64_t gap_design_rows(const gap_problem *p) {
    return p ? data_rows(p) + p->n_sparse + (p->n_sparse_2b > 0 ? p->n_sparse_2b : 0) : -1;
}

gap_status gap_workspace_size(const gap_problem *p, gap_precision prec, size_t *bytes) {
    return gap_workspace_size_ring(p, prec, 0, bytes);
}

gap_status gap_workspace_size_ring(const gap_problem *p, gap_precision prec, int64_t j_ring_rows, size_t *bytes) {
    if (!p || !bytes || j_ring_rows < 0 || j_ring_rows % 128 != 0 || (j_ring_rows > 0 && !is_mixed(prec)))
        return GAP_ERR_INVALID;
    gap_status st = check_scalars(nullptr, p, false);
    if (st != GAP_OK) return st;
    Dims dm = make_dims(p);
    size_t e = elt_size(prec);
    size_t a = (size_t)dm.ld * (size_t)(dm.M + 1) * e;       // design matrix + rhs column
    size_t total = a;
    if (is_mixed(prec)) total += a;                           // FP32-accurate residual copy
    total += (size_t)dm.n_atoms * dm.M * e;                   // per-atom force weights
    total += (size_t)dm.rows * 8;                             // b (FP64)
    total += (size_t)dm.M * dm.M * 8;                         // K_MM / L
    total += (size_t)kQrRowBlocks * kQNB * (dm.M + 1) * e;    // QR V^T C partials
    total += (size_t)kQNB * (dm.M + 1) * e;                   // QR T^T V^T C
    total += (size_t)dm.M * dm.d * 8 + (size_t)(dm.n_atoms + dm.n_pairs) * 8;  // Xs, index arrays
    if (dm.M2 > 0) total += (size_t)(dm.n_atoms + 1 + 4 * p->n_bonds + dm.M2) * 8;  // two-body inputs (host problems)
    total += (size_t)(6 * dm.rows + 8 * dm.M) * 8;            // refinement vectors
    if (is_mixed(prec)) total += qr_outer_workspace_bytes(dm.rows, dm.M);  // two-level QR
    if (is_mixed(prec)) total += tc_workspace_bytes(dm, j_ring_rows);  // tensor-core operand staging
    if (j_ring_rows > 0 && dm.forces && p->memory == GAP_MEM_HOST)    // the J ring's two FP64 slots
        total += 2 * sizeof(double) * 3 * (size_t)dm.d * (size_t)ring_slot_pairs(j_ring_rows);
    if (is_mixed(prec)) {                                     // refinement: R^{-1}, R^{-T}, pass partials
        total += rinv_bytes(dm.M, dm.d);
        total += cgls_workspace_bytes(dm.M);
        total += (size_t)dm.n_cfg * dm.M * 8 + (size_t)round_up(dm.n_cfg, ACC_RB) * 8;  // FP64 energy rows
    }
    *bytes = total;
    return GAP_OK;
}

namespace {
gap_status assemble_impl(gap_ctx *c, const gap_problem *p);
}

gap_status gap_assemble(gap_ctx *c, const gap_problem *p) {
    if (!c) return GAP_ERR_INVALID;
    const gap_status st = assemble_impl(c, p);
    // a host problem's J is borrowed: its chunked (or ring) copies end before the call returns
    if ((c->n_jchunks > 0 || c->j_ring_rows > 0) && c->cstream) cudaStreamSynchronize(c->cstream);
    return st;
}

namespace {
gap_status assemble_impl(gap_ctx *c, const gap_problem *p) {
    c->err.clear();
    c->state = 0;
    c->have_last = false;
    gap_status st = check_scalars(c, p, true);
    if (st != GAP_OK) return st;
    if (is_mixed(c->prec) && !cgls_fused_fits(p->n_sparse + std::max<int64_t>(0, p->n_sparse_2b)))
        return fail(c, GAP_ERR_INVALID, "the mixed precisions support at most 16384 sparse points");
    Dims dm = make_dims(p);
    c->dm = dm;
    cudaStream_t s = c->stream;
    c->prof.reset();
    GAP_CUDA(c, cudaEventRecord(c->ev[0], s));
    const bool ring = c->j_ring_rows > 0 && dm.forces;
    if (ring && dm.virials) return fail(c, GAP_ERR_INVALID, "the J ring does not take problems with virial rows");
    DevProblem dp{};
    if (p->memory == GAP_MEM_HOST) c->prof.begin(GAP_PROF_COPY_IN);
    st = to_device(c, p, true, &dp, is_mixed(c->prec) && !ring, ring);
    if (p->memory == GAP_MEM_HOST) c->prof.end();
    if (st != GAP_OK) return st;
    // sparse set (kept for K_MM and predictions).  A two-body block's columns follow as
    // sparse points with zero descriptors (and a species label no atom carries), for which
    // the SOAP kernels give zero rows and a zero K_MM block; its own kernels fill them.
    const cudaMemcpyKind kind = p->memory == GAP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    GAP_CUDA(c, c->Xs.ensure(sizeof(double) * dm.M * dm.d));
    GAP_CUDA(c, cudaMemcpyAsync(c->Xs.p, p->Xs, sizeof(double) * dm.Ms * dm.d, kind, s));
    if (dm.M2 > 0)
        GAP_CUDA(c, cudaMemsetAsync(c->Xs.as<double>() + dm.Ms * dm.d, 0, sizeof(double) * dm.M2 * dm.d, s));
    const int32_t *sparse_sp = nullptr;
    if (dm.species) {
        GAP_CUDA(c, c->sparse_sp.ensure(sizeof(int32_t) * dm.M));
        GAP_CUDA(c, cudaMemcpyAsync(c->sparse_sp.p, p->sparse_species, sizeof(int32_t) * dm.Ms, kind, s));
        if (dm.M2 > 0)  // label 0x7F7F7F7F: non-negative, and no atom's
            GAP_CUDA(c, cudaMemsetAsync(c->sparse_sp.as<int32_t>() + dm.Ms, 0x7F, sizeof(int32_t) * dm.M2, s));
        sparse_sp = c->sparse_sp.as<int32_t>();
    }
    if (dm.M2 > 0) {  // the fit's sparse distances and constants, kept for K_MM and predictions
        GAP_CUDA(c, c->sparse_r.ensure(sizeof(double) * dm.M2));
        GAP_CUDA(c, cudaMemcpyAsync(c->sparse_r.p, p->sparse_r, sizeof(double) * dm.M2, kind, s));
        c->tb_delta = p->delta_2b;
        c->tb_theta = p->theta_2b;
        c->tb_cutoff = p->cutoff_2b;
        c->tb_width = p->width_2b;
    }
    if ((st = set_kmm_blocks(c, p)) != GAP_OK) return st;
    const double *Xs = c->Xs.as<double>();
    // derived indices and device-side validation
    if ((st = clear_status(c)) != GAP_OK) return st;
    DevStatus *dst = c->status.as<DevStatus>();
    GAP_CUDA(c, c->atom_cfg.ensure(sizeof(int64_t) * dm.n_atoms));
    GAP_CUDA(c, c->pair_tgt.ensure(sizeof(int64_t) * std::max<int64_t>(dm.n_pairs, 1)));
    // host problems had their pointers checked on the host; their sigma, pair sources and
    // species are checked here, on the staged copies
    GAP_CUDA(c, launch_validate(dm, dp.cfg_ptr, dp.pair_ptr, dp.pair_src, nullptr, dp.sigma, dp.atom_sp, sparse_sp,
                                dst, s));
    if ((st = read_status(c, "invalid problem (pointers or sigma)")) != GAP_OK) return st;
    GAP_CUDA(c, launch_segment_ids(dp.cfg_ptr, dm.n_cfg, c->atom_cfg.as<int64_t>(), s));
    if (dm.forces) GAP_CUDA(c, launch_segment_ids(dp.pair_ptr, dm.n_atoms, c->pair_tgt.as<int64_t>(), s));
    GAP_CUDA(c, launch_validate(dm, dp.cfg_ptr, dp.pair_ptr, dp.pair_src, c->atom_cfg.as<int64_t>(), dp.sigma,
                                dp.atom_sp, sparse_sp, dst, s));
    if ((st = read_status(c, "invalid problem (pair sources or species)")) != GAP_OK) return st;
    const TwoBodyDev tb2 = two_body_dev(p, dp, c->sparse_r.as<double>(), dm.Ms);
    if (dm.M2 > 0) {
        GAP_CUDA(c, launch_2b_validate(dm.n_atoms, p->n_bonds, tb2, dst, s));
        if ((st = read_status(c, "invalid two-body bonds (bond_ptr, bond lengths or sparse distances)")) != GAP_OK)
            return st;
    }
    // design matrix buffers
    const size_t e = elt_size(c->prec);
    const size_t abytes = (size_t)dm.ld * (size_t)(dm.M + 1) * e;
    GAP_CUDA(c, c->A.ensure(abytes));
    GAP_CUDA(c, cudaMemsetAsync(c->A.p, 0, abytes, s));
    GAP_CUDA(c, c->Wf.ensure((size_t)dm.n_atoms * dm.M * e));
    GAP_CUDA(c, c->b64.ensure(sizeof(double) * dm.rows));
    if (c->prec == GAP_PREC_FP64) {
        double *A = c->A.as<double>(), *Wf = c->Wf.as<double>();
        c->prof.begin(GAP_PROF_GEMM_ENERGY);
        GAP_CUDA(c, launch_energy_simt<double>(dm, dp.X, Xs, dp.atom_sp, sparse_sp, dp.cfg_ptr,
                                               c->atom_cfg.as<int64_t>(), dp.sigma, A, Wf, s));
        c->prof.end();
        c->prof.begin(GAP_PROF_GEMM_FORCE);
        GAP_CUDA(c, launch_force_simt<double>(dm, dp.J, Xs, dp.pair_ptr, dp.pair_src, c->pair_tgt.as<int64_t>(),
                                              dp.sigma, Wf, A, s));
        if (dm.virials) {
            // virial rows: the force rows of each configuration's two pseudo-targets
            if ((st = ensure_virial_buffers(c, dm)) != GAP_OK) return st;
            GAP_CUDA(c, launch_virial_pseudo_pairs(dm, dp.cfg_ptr, c->atom_cfg.as<int64_t>(), dp.pair_ptr, dp.pair_src,
                                                   dp.J, dp.pair_u, c->vp_ptr.as<int64_t>(), c->vp_src.as<int64_t>(),
                                                   c->vp_tgt.as<int64_t>(), c->vG.as<double>(), s));
            GAP_CUDA(c, launch_force_simt<double>(virial_dims(dm), c->vG.as<double>(), Xs, c->vp_ptr.as<int64_t>(),
                                                  c->vp_src.as<int64_t>(), c->vp_tgt.as<int64_t>(), dp.sigma, Wf, A, s));
        }
        c->prof.end();
        if (dm.M2 > 0) GAP_CUDA(c, launch_2b_rows<double>(dm, dp.cfg_ptr, tb2, dp.sigma, A, nullptr, nullptr, s));
        GAP_CUDA(c, launch_rhs<double>(dm, dp.y, dp.sigma, c->b64.as<double>(), A, s));
    } else {
        GAP_CUDA(c, c->Aacc.ensure(abytes));
        GAP_CUDA(c, cudaMemsetAsync(c->Aacc.p, 0, abytes, s));
        const size_t ebytes = sizeof(double) * (size_t)std::max<int64_t>(1, dm.n_cfg * dm.M);
        GAP_CUDA(c, c->E64.ensure(ebytes));
        GAP_CUDA(c, cudaMemsetAsync(c->E64.p, 0, ebytes, s));
        float *A = c->A.as<float>(), *Aacc = c->Aacc.as<float>(), *Wf = c->Wf.as<float>();
        TcInputs ti{dp.X,      Xs,         dp.J,         dp.cfg_ptr, c->atom_cfg.as<int64_t>(),
                    dp.pair_ptr, dp.pair_src, c->pair_tgt.as<int64_t>(), dp.sigma, dp.atom_sp,
                    sparse_sp, &dst->code, c->n_jchunks, c->j_rows, c->j_ev, c->E64.as<double>()};
        ti.force_walk = c->force_walk;
        if (ring && (st = set_ring(c, p, dp, ti)) != GAP_OK) return st;
        if (dm.virials) {
            if ((st = ensure_virial_buffers(c, dm)) != GAP_OK) return st;
            ti.pair_u = dp.pair_u;
            ti.vG = c->vG.as<double>();
            ti.vp_ptr = c->vp_ptr.as<int64_t>();
            ti.vp_src = c->vp_src.as<int64_t>();
            ti.vp_tgt = c->vp_tgt.as<int64_t>();
        }
        const cudaError_t ea = tc_assemble(dm, ti, tc_mode(c->prec),
                                           c->tc_ops, A, Aacc, Wf, s, &c->prof);
        // the host's J is borrowed: its copies end before this call returns, also on failure
        if (c->n_jchunks > 0 || ti.h_J) GAP_CUDA(c, cudaStreamSynchronize(c->cstream));
        GAP_CUDA(c, ea);
        if (dm.M2 > 0)
            GAP_CUDA(c, launch_2b_rows<float>(dm, dp.cfg_ptr, tb2, dp.sigma, A, Aacc, c->E64.as<double>(), s));
        GAP_CUDA(c, launch_rhs<float>(dm, dp.y, dp.sigma, c->b64.as<double>(), A, s));
        GAP_CUDA(c, launch_rhs<float>(dm, dp.y, dp.sigma, c->b64.as<double>(), Aacc, s, true));
    }
    GAP_CUDA(c, cudaEventRecord(c->ev[1], s));
    // the status word also carries tensor-core timeouts; reading it synchronises,
    // which host-memory problems need anyway (their inputs are borrowed)
    if ((st = read_status(c, "assembly")) != GAP_OK) return st;
    // the assembled problem as device memory, for gap_predict without targets
    c->last_dev = *p;
    c->last_dev.memory = GAP_MEM_DEVICE;
    c->last_dev.cfg_ptr = dp.cfg_ptr;
    c->last_dev.X = dp.X;
    c->last_dev.Xs = Xs;
    c->last_dev.y = dp.y;
    c->last_dev.sigma = dp.sigma;
    c->last_dev.atom_species = dp.atom_sp;
    c->last_dev.sparse_species = sparse_sp;
    c->last_dev.pair_ptr = dp.pair_ptr;
    c->last_dev.pair_src = dp.pair_src;
    c->last_dev.J = dp.J;
    c->last_dev.pair_u = dp.pair_u;
    c->last_dev.bond_ptr = dp.bond_ptr;
    c->last_dev.bond_r = dp.bond_r;
    c->last_dev.bond_u = dp.bond_u;
    c->last_dev.sparse_r = dm.M2 > 0 ? c->sparse_r.as<double>() : nullptr;
    c->have_last = true;
    c->state = 1;
    return GAP_OK;
}
}  // namespace


gap_status gap_factor(gap_ctx *c) {
    if (!c) return GAP_ERR_INVALID;
    if (c->state != 1) return fail(c, GAP_ERR_STATE, "gap_factor needs a preceding gap_assemble");
    c->err.clear();
    gap_status st = c->prec == GAP_PREC_FP64 ? factor_impl<double>(c) : factor_impl<float>(c);
    if (st != GAP_OK) {
        c->state = 0;
        return st;
    }
    c->state = 2;
    return GAP_OK;
}


}  // extern "C"

namespace gap {
namespace {
// Rz [M x (M+1)], row-major FP64: the top M rows of the factored column-major A (R on and
// above the diagonal, zeros below it; column M the transformed right-hand side).
__global__ void k_read_rz(const double *__restrict__ A, int64_t ld, int64_t M, double *__restrict__ Rz) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * (M + 1)) return;
    const int64_t i = e / (M + 1), j = e % (M + 1);
    Rz[e] = (j < M && j < i) ? 0.0 : A[i + j * ld];
}
// The G blocks Rz_g (row-major [M x (M+1)] each) as rows g M .. g M + M - 1 of the
// column-major stack S (leading dimension lds).
__global__ void k_stack_rz(const double *__restrict__ Rz, int64_t G, int64_t M, double *__restrict__ S, int64_t lds) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= G * M * (M + 1)) return;
    const int64_t g = e / (M * (M + 1)), r = e % (M * (M + 1)), i = r / (M + 1), j = r % (M + 1);
    S[(g * M + i) + j * lds] = Rz[e];
}
// Householder QR (FP64, flat panels) of the column-major [rows x (M+1)] matrix X with the
// ctx's QR workspaces.
gap_status qr_f64(gap_ctx *c, double *X, int64_t rows, int64_t ld) {
    const Dims &dm = c->dm;
    const size_t e = sizeof(double);
    const int64_t nc = dm.M + 1;
    GAP_CUDA(c, c->tau.ensure(e * dm.M));
    GAP_CUDA(c, c->T.ensure(e * kQNB * kQNB));
    GAP_CUDA(c, c->part.ensure(e * std::max<size_t>(2 * kQrColBlocks * (kQNB + 1), 152 * kQNB * kQNB)));
    GAP_CUDA(c, c->diagrow.ensure(e * 2 * (kQNB + 1)));
    GAP_CUDA(c, c->Wpart.ensure(e * kQrRowBlocks * kQNB * nc));
    GAP_CUDA(c, c->Wred.ensure(e * kQNB * nc));
    GAP_CUDA(c, householder_qr<double>(X, rows, dm.M, ld, std::min(c->qr_nb, kQNB), c->tau.as<double>(),
                                       c->T.as<double>(), c->part.as<double>(), c->diagrow.as<double>(),
                                       c->Wpart.as<double>(), c->Wred.as<double>(), kQrRowBlocks, c->stream, &c->prof,
                                       nullptr, nullptr, 3, 2));
    return GAP_OK;
}
}  // namespace
}  // namespace gap

extern "C" {

gap_status gap_tsqr_local(gap_ctx *c, double *Rz_dev, double *tail2) {
    if (!c) return GAP_ERR_INVALID;
    if (c->state != 1) return fail(c, GAP_ERR_STATE, "gap_tsqr_local needs a preceding gap_assemble");
    if (!Rz_dev || !tail2) return fail(c, GAP_ERR_INVALID, "Rz_dev and tail2 are required");
    if (c->prec != GAP_PREC_FP64) return fail(c, GAP_ERR_INVALID, "the row-block merge runs in FP64 precision");
    const Dims &dm = c->dm;
    if (dm.N < dm.M) return fail(c, GAP_ERR_INVALID, "a row block needs at least n_sparse data rows");
    c->err.clear();
    cudaStream_t s = c->stream;
    double *A = c->A.as<double>();
    c->prof.begin(GAP_PROF_QR_UPDATE);
    gap_status st = qr_f64(c, A, dm.N, dm.ld);  // the data rows and b (column M), without U
    c->prof.end();
    if (st != GAP_OK) return st;
    const int64_t n = dm.M * (dm.M + 1);
    k_read_rz<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(A, dm.ld, dm.M, Rz_dev);
    GAP_CUDA(c, cudaGetLastError());
    // the block's residual tail: (Q^T b)[M:N]
    GAP_CUDA(c, c->vecs.ensure(sizeof(double) * 8));
    double *sq = c->vecs.as<double>(), h = 0.0;
    GAP_CUDA(c, vec_dot(A + dm.M * dm.ld + dm.M, A + dm.M * dm.ld + dm.M, dm.N - dm.M, sq, s));
    GAP_CUDA(c, cudaMemcpyAsync(&h, sq, sizeof(double), cudaMemcpyDeviceToHost, s));
    GAP_CUDA(c, cudaStreamSynchronize(s));
    *tail2 = h;
    c->state = 3;  // a factored row block: the merge may follow, a gap_factor needs a new gap_assemble
    return GAP_OK;
}

gap_status gap_tsqr_merge(gap_ctx *c, int G, const double *Rz_dev, double tail2) {
    if (!c) return GAP_ERR_INVALID;
    if (c->state != 1 && c->state != 3)
        return fail(c, GAP_ERR_STATE, "gap_tsqr_merge needs the sparse set of a gap_assemble");
    if (G < 1 || !Rz_dev || !(tail2 >= 0.0)) return fail(c, GAP_ERR_INVALID, "G >= 1, Rz_dev and tail2 >= 0 are required");
    if (c->prec != GAP_PREC_FP64) return fail(c, GAP_ERR_INVALID, "the row-block merge runs in FP64 precision");
    c->err.clear();
    const Dims &dm = c->dm;
    cudaStream_t s = c->stream;
    GAP_CUDA(c, cudaEventRecord(c->ev[2], s));  // the factor phase of gap_solve's report
    if (clear_status(c) != GAP_OK) return GAP_ERR_CUDA;
    // K_MM + jitter = U^T U (Eq. 7) from this ctx's sparse set, U into rows N .. N + M - 1 of A
    GAP_CUDA(c, c->Kmm.ensure(sizeof(double) * dm.M * dm.M));
    c->prof.begin(GAP_PROF_KMM_CHOL);
    GAP_CUDA(c, launch_kmm(dm, c->Xs.as<double>(), dm.species ? c->sparse_sp.as<int32_t>() : nullptr,
                           c->Kmm.as<double>(), s));
    if (dm.M2 > 0) GAP_CUDA(c, launch_2b_kmm(fit_two_body(c), dm.jitter, c->Kmm.as<double>(), dm.M, s));
    GAP_CUDA(c, cholesky_lower(c->Kmm.as<double>(), dm.M, c->status.as<DevStatus>(), s, c->kmm_ends.data(),
                               (int)c->kmm_ends.size()));
    c->prof.end();
    gap_status st = read_status(c, "Cholesky of K_MM + jitter met a non-positive pivot");
    if (st != GAP_OK) return st;
    double *A = c->A.as<double>();
    GAP_CUDA(c, launch_stack_u<double>(dm, c->Kmm.as<double>(), A, s));
    // the stack [R_1 z_1; ...; R_G z_G; U 0] and its QR
    const int64_t s_rows = ((int64_t)G + 1) * dm.M, s_ld = round_up(s_rows, 128);
    GAP_CUDA(c, c->tsqr.ensure(sizeof(double) * s_ld * (dm.M + 1)));
    double *S = c->tsqr.as<double>();
    GAP_CUDA(c, cudaMemsetAsync(S, 0, sizeof(double) * s_ld * (dm.M + 1), s));
    const int64_t n = (int64_t)G * dm.M * (dm.M + 1);
    k_stack_rz<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(Rz_dev, G, dm.M, S, s_ld);
    GAP_CUDA(c, cudaGetLastError());
    GAP_CUDA(c, tsqr_gather<double>(A, dm.ld, dm.N, dm.M, S, s_ld, (int64_t)G * dm.M, true, s));
    c->prof.begin(GAP_PROF_QR_UPDATE);
    st = qr_f64(c, S, s_rows, s_ld);
    c->prof.end();
    if (st != GAP_OK) return st;
    GAP_CUDA(c, cudaEventRecord(c->ev[3], s));
    c->tsqr_used = G;
    c->tsqr_ext = true;
    c->tsqr_ext_tail2 = tail2;
    c->r_ld = s_ld;
    c->state = 2;
    return GAP_OK;
}

gap_status gap_solve(gap_ctx *c, double *c_dev, gap_solve_info *info) {
    if (!c) return GAP_ERR_INVALID;
    if (c->state != 2) return fail(c, GAP_ERR_STATE, "gap_solve needs a preceding gap_factor");
    if (!c_dev) return fail(c, GAP_ERR_INVALID, "c_dev is NULL");
    c->err.clear();
    if (c->prec == GAP_PREC_FP64) return solve_impl<double>(c, c_dev, info);
    gap_status st = solve_impl<float>(c, c_dev, info);
    if (st == GAP_ERR_NOT_CONVERGED && c->qr_lean) {
        // the one-pass FP32 QR left too rough a preconditioner for this matrix: refactor the
        // FP32-accurate matrix with split-product updates and CholeskyQR2 panels, and solve
        // again from the new QR solution
        c->err.clear();
        GAP_CUDA(c, acc_to_colmajor(c->Aacc.as<float>(), c->dm.ld, c->dm.M, c->A.as<float>(), c->stream));
        if ((st = factor_qr<float>(c, 3, 2)) != GAP_OK) return st;
        c->qr_refactors += 1;
        st = solve_impl<float>(c, c_dev, info);
    }
    return st;
}

namespace gap {
namespace {
gap_status predict_impl(gap_ctx *c, const gap_problem *t, const double *c_dev, double *E_dev, double *F_dev,
                        double *V_dev);
}
}  // namespace gap

gap_status gap_predict(gap_ctx *c, const gap_problem *t, const double *c_dev, double *E_dev, double *F_dev) {
    return predict_impl(c, t, c_dev, E_dev, F_dev, nullptr);
}

gap_status gap_predict_virial(gap_ctx *c, const gap_problem *t, const double *c_dev, double *E_dev, double *F_dev,
                              double *V_dev) {
    return predict_impl(c, t, c_dev, E_dev, F_dev, V_dev);
}

namespace gap {
namespace {
// Predictions of the last assembled problem from its design rows (a mixed fit of a host
// problem whose J went through the J ring and is not on the device): the data rows of
// Eq. (7) are the targets' model values over sigma, so E = sigma_E (E64 c) with the FP64
// energy rows, and the force (and virial) values are sigma (A_acc c) over the FP32-accurate
// rows, in double-float.  No Jacobian is read again.
gap_status predict_from_design(gap_ctx *c, const double *c_dev, double *E_dev, double *F_dev, double *V_dev) {
    const Dims &dm = c->dm;
    const gap_problem &t = c->last_dev;
    if (V_dev && !dm.virials) return fail(c, GAP_ERR_INVALID, "virial predictions need pair data and pair_u");
    cudaStream_t s = c->stream;
    DevBuf ws;
    GAP_CUDA(c, ws.ensure(2 * sizeof(float) * (size_t)dm.M));
    c->prof.begin(GAP_PROF_PREDICT);
    cudaError_t e = predict_from_rows(c->E64.as<double>(), dm.n_cfg, c->Aacc.as<float>(), dm.M, dm.n_cfg,
                                      F_dev ? 3 * dm.n_atoms : 0, t.sigma, c_dev, ws.as<float>(), E_dev, F_dev, s);
    if (e == cudaSuccess && V_dev)
        e = predict_from_rows(nullptr, 0, c->Aacc.as<float>(), dm.M, dm.n_cfg + 3 * dm.n_atoms, 6 * dm.n_cfg, t.sigma,
                              c_dev, ws.as<float>(), nullptr, V_dev, s);
    c->prof.end();
    if (e != cudaSuccess) return cuda_fail(c, e, "predict from the design rows");
    GAP_CUDA(c, cudaStreamSynchronize(s));  // ws is freed on return
    return GAP_OK;
}

gap_status predict_impl(gap_ctx *c, const gap_problem *t, const double *c_dev, double *E_dev, double *F_dev,
                        double *V_dev) {
    if (!c) return GAP_ERR_INVALID;
    if (c->state < 1) return fail(c, GAP_ERR_STATE, "gap_predict needs the sparse set of a gap_assemble");
    if (!c_dev || !E_dev) return fail(c, GAP_ERR_INVALID, "c_dev and E_dev are required");
    c->err.clear();
    if (t == nullptr) {
        // the problem last assembled, from its device copies
        if (!c->have_last)
            return fail(c, GAP_ERR_STATE, "gap_predict without targets needs the problem of the last gap_assemble");
        if (c->last_dev.n_pairs > 0 && c->last_dev.J == nullptr && is_mixed(c->prec))
            return predict_from_design(c, c_dev, E_dev, F_dev, V_dev);
        t = &c->last_dev;
    } else if (t->memory == GAP_MEM_HOST) {
        c->have_last = false;  // staging this problem replaces the assembled problem's copies
    }
    gap_status st = check_scalars(c, t, false);
    if (st != GAP_OK) return st;
    if (t->d != c->dm.d || t->n_sparse != c->dm.Ms || std::max<int64_t>(0, t->n_sparse_2b) != c->dm.M2)
        return fail(c, GAP_ERR_INVALID, "targets must use the fitted descriptor length and sparse sets");
    if ((t->atom_species != nullptr) != c->dm.species)
        return fail(c, GAP_ERR_INVALID, "targets must carry species labels exactly when the fit does");
    Dims dm = make_dims(t);
    dm.M = c->dm.M;
    if (V_dev && !dm.virials) return fail(c, GAP_ERR_INVALID, "virial predictions need pair data and pair_u");
    // a host problem's J goes through the J ring (mixed precisions, option j_ring_rows)
    const bool ring = is_mixed(c->prec) && c->j_ring_rows > 0 && dm.forces && t->memory == GAP_MEM_HOST;
    if (ring && V_dev) return fail(c, GAP_ERR_INVALID, "the J ring does not take virial predictions");
    if (ring && (F_dev || V_dev)) {
        const int64_t cap = ring_slot_pairs(c->j_ring_rows);
        for (int64_t a = 0; a < t->n_atoms; ++a)
            if (t->pair_ptr[a + 1] - t->pair_ptr[a] > cap)
                return fail(c, GAP_ERR_INVALID, "j_ring_rows holds fewer pairs than atom " + std::to_string(a) + " has");
    }
    DevProblem dp{};
    if ((st = to_device(c, t, false, &dp, false, ring)) != GAP_OK) return st;
    cudaStream_t s = c->stream;
    // virials are contracted from the per-atom gradients that the force predictions form
    DevBuf ftmp;
    if (V_dev && !F_dev) {
        GAP_CUDA(c, ftmp.ensure(sizeof(double) * 3 * (size_t)dm.n_atoms));
        F_dev = ftmp.as<double>();
    }
    {  // pointers (device) and pair sources / species (every problem) checked on the device
        if ((st = clear_status(c)) != GAP_OK) return st;
        GAP_CUDA(c, launch_validate(dm, dp.cfg_ptr, dp.pair_ptr, dp.pair_src, nullptr, nullptr, dp.atom_sp, nullptr,
                                    c->status.as<DevStatus>(), s));
        if ((st = read_status(c, "invalid prediction targets")) != GAP_OK) return st;
    }
    const int64_t chunk = std::min<int64_t>(dm.n_atoms, 32768);
    DevBuf eps, grad, wm, cfgids;
    if (!is_mixed(c->prec)) {
        GAP_CUDA(c, eps.ensure(sizeof(double) * dm.n_atoms));
        GAP_CUDA(c, grad.ensure(sizeof(double) * (dm.forces ? dm.n_atoms * dm.d : 1)));
        GAP_CUDA(c, wm.ensure(sizeof(double) * (dm.forces ? chunk * dm.M : 1)));
    }
    if (dm.forces) {
        GAP_CUDA(c, cfgids.ensure(sizeof(int64_t) * dm.n_atoms));
        GAP_CUDA(c, launch_segment_ids(dp.cfg_ptr, dm.n_cfg, cfgids.as<int64_t>(), s));
        GAP_CUDA(c, launch_validate(dm, dp.cfg_ptr, dp.pair_ptr, dp.pair_src, cfgids.as<int64_t>(), nullptr,
                                    dp.atom_sp, dm.species ? c->sparse_sp.as<int32_t>() : nullptr,
                                    c->status.as<DevStatus>(), s));
        if ((st = read_status(c, "invalid prediction targets (pair sources)")) != GAP_OK) return st;
    }
    c->prof.begin(GAP_PROF_PREDICT);
    cudaError_t e = cudaSuccess;
    if (V_dev) {
        // the targets' pseudo-pairs and strain Jacobians (k_virial.cu)
        if ((st = ensure_virial_buffers(c, dm)) != GAP_OK) return st;
        GAP_CUDA(c, cfgids.ensure(sizeof(int64_t) * dm.n_atoms));
        GAP_CUDA(c, launch_segment_ids(dp.cfg_ptr, dm.n_cfg, cfgids.as<int64_t>(), s));
        e = launch_virial_pseudo_pairs(dm, dp.cfg_ptr, cfgids.as<int64_t>(), dp.pair_ptr, dp.pair_src, dp.J, dp.pair_u,
                                       c->vp_ptr.as<int64_t>(), c->vp_src.as<int64_t>(), c->vp_tgt.as<int64_t>(),
                                       c->vG.as<double>(), s);
    }
    if (e != cudaSuccess) {
    } else if (is_mixed(c->prec)) {
        // split-precision tensor-core products, FP64 sums (accurate to FP32 products)
        TcInputs ti{dp.X, c->Xs.as<double>(), dp.J, dp.cfg_ptr, nullptr, dp.pair_ptr, dp.pair_src, nullptr,
                    nullptr, dp.atom_sp, dm.species ? c->sparse_sp.as<int32_t>() : nullptr, &c->status.as<DevStatus>()->code};
        if (V_dev) {
            ti.vG = c->vG.as<double>();
            ti.vp_ptr = c->vp_ptr.as<int64_t>();
            ti.vp_src = c->vp_src.as<int64_t>();
        }
        if (ring && (st = set_ring(c, t, dp, ti)) != GAP_OK) {
            c->prof.end();
            return st;
        }
        e = tc_predict(dm, ti, tc_mode(c->prec) == TcMode::TF32 ? TcMode::TF32 : TcMode::BF16, c->tc_ops, c->pred_work,
                       c_dev, E_dev, F_dev, s, &c->prof, V_dev);
    } else {
        e = predict_simt(dm, dp.X, c->Xs.as<double>(), dp.atom_sp, dm.species ? c->sparse_sp.as<int32_t>() : nullptr,
                         dp.cfg_ptr, dp.pair_ptr, dp.pair_src, dp.J, c_dev, E_dev, F_dev, eps.as<double>(),
                         grad.as<double>(), wm.as<double>(), chunk, s);
        if (e == cudaSuccess && V_dev)
            e = predict_virial_simt(virial_dims(dm), c->vp_ptr.as<int64_t>(), c->vp_src.as<int64_t>(),
                                    c->vG.as<double>(), grad.as<double>(), V_dev, s);
    }
    if (e == cudaSuccess && dm.M2 > 0) {
        // the two-body model, with the fit's sparse distances and constants, on the targets' bonds
        TwoBodyDev tb = fit_two_body(c);
        tb.bond_ptr = dp.bond_ptr;
        tb.bond_r = dp.bond_r;
        tb.bond_u = dp.bond_u;
        if ((st = clear_status(c)) != GAP_OK) return st;
        GAP_CUDA(c, launch_2b_validate(dm.n_atoms, t->n_bonds, tb, c->status.as<DevStatus>(), s));
        if ((st = read_status(c, "invalid two-body bonds of the prediction targets")) != GAP_OK) return st;
        e = launch_2b_predict(dm.n_cfg, dm.n_atoms, dp.cfg_ptr, tb, c_dev + dm.Ms, E_dev, F_dev, V_dev, s);
    }
    c->prof.end();
    if (ring) cudaStreamSynchronize(c->cstream);  // the borrowed host J is read by the copies only until here
    if (e != cudaSuccess) return cuda_fail(c, e, "predict");
    GAP_CUDA(c, cudaStreamSynchronize(s));  // temporaries are freed on return
    eps.release();
    grad.release();
    wm.release();
    cfgids.release();
    return GAP_OK;
}
}  // namespace
}  // namespace gap

gap_status gap_get_profile(gap_ctx *c, gap_profile *out) {
    if (!c || !out) return GAP_ERR_INVALID;
    GAP_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = gap_profile{};
    for (const auto &m : c->prof.marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess && m.cls >= 0 && m.cls < GAP_PROF_N) {
            out->ms[m.cls] += ms;
            out->groups[m.cls] += 1;
        }
    }
    return GAP_OK;
}

gap_status gap_read_design(gap_ctx *c, int which, int64_t row0, int64_t nrows, double *dst) {
    if (!c || !dst) return GAP_ERR_INVALID;
    const Dims &dm = c->dm;
    if (row0 < 0 || nrows < 0 || row0 + nrows > dm.rows) return fail(c, GAP_ERR_INVALID, "row range out of bounds");
    if (which == 0 && c->state != 1) return fail(c, GAP_ERR_STATE, "the QR matrix is only readable before gap_factor");
    if (which == 1 && c->state < 1) return fail(c, GAP_ERR_STATE, "nothing assembled");
    if (which != 0 && which != 1) return fail(c, GAP_ERR_INVALID, "which must be 0 or 1");
    cudaError_t e;
    if (c->prec == GAP_PREC_FP64) {
        if (which == 1 && c->state != 1) return fail(c, GAP_ERR_STATE, "FP64 mode keeps one matrix (factored in place)");
        e = launch_read_rows<double>(c->A.as<double>(), dm.ld, dm.M, row0, nrows, dst, c->stream);
    } else {
        e = which == 0 ? launch_read_rows<float>(c->A.as<float>(), dm.ld, dm.M, row0, nrows, dst, c->stream)
                       : read_rows_acc(c->Aacc.as<float>(), dm.M, row0, nrows, dst, c->stream);
        if (e == cudaSuccess && which == 1 && row0 < dm.n_cfg) {
            // the energy rows of the residual matrix are the FP64 ones
            const int64_t n = std::min(nrows, dm.n_cfg - row0);
            e = cudaMemcpyAsync(dst, c->E64.as<double>() + row0 * dm.M, sizeof(double) * n * dm.M,
                                cudaMemcpyDeviceToDevice, c->stream);
        }
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "read_design");
    GAP_CUDA(c, cudaStreamSynchronize(c->stream));
    return GAP_OK;
}

int gap_tsqr_blocks(const gap_ctx *c) { return c ? c->tsqr_used : -1; }

int gap_tsqr_plan(int64_t n_data_rows, int64_t M, int want, int64_t *row0, int64_t *rows) {
    if (n_data_rows < 0 || M < 0) return -1;
    int64_t r0[kTsqrMax], n[kTsqrMax];
    const int64_t ld = round_up(n_data_rows + M, 128);
    const int G = tsqr_plan(n_data_rows, M, ld, want, r0, n);
    if (row0 && rows)
        for (int g = 0; g < G; ++g) {
            row0[g] = r0[g];
            rows[g] = n[g];
        }
    return G;
}

gap_status gap_read_r(gap_ctx *c, double *dst) {
    if (!c || !dst) return GAP_ERR_INVALID;
    if (c->state != 2) return fail(c, GAP_ERR_STATE, "R exists after gap_factor");
    cudaError_t e = c->prec == GAP_PREC_FP64
                        ? launch_read_r<double>(r_matrix<double>(c), c->r_ld, c->dm.M, dst, c->stream)
                        : launch_read_r<float>(r_matrix<float>(c), c->r_ld, c->dm.M, dst, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read_r");
    GAP_CUDA(c, cudaStreamSynchronize(c->stream));
    return GAP_OK;
}

gap_status gap_fit_batched(gap_ctx *c, int n, const gap_problem *const *probs, double *const *c_dev,
                           gap_solve_info *infos) {
    if (!c || n < 0 || (n > 0 && (!probs || !c_dev))) return GAP_ERR_INVALID;
    c->err.clear();
    // longest fits first (the greedy order of Sec. III.B)
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    // estimated cost of a fit: its QR, rows x M^2
    auto cost = [&](int k) { return (double)gap_design_rows(probs[k]) * (double)probs[k]->n_sparse * probs[k]->n_sparse; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    const int L = std::min(c->batch_lanes, n);
    if (L <= 1) {
        for (int k : order) {
            gap_status st = run_fit(c, probs[k], c_dev[k], infos ? &infos[k] : nullptr);
            if (st != GAP_OK) {
                c->err = "fit " + std::to_string(k) + ": " + c->err;
                return st;
            }
        }
        return GAP_OK;
    }
    // L fits in flight: worker contexts with their own streams, one host thread each,
    // taking the next fit in order; each fit's arithmetic is that of a single fit
    gap_status st = ensure_lanes(c, L);
    if (st != GAP_OK) return st;
    cudaEvent_t ready = nullptr;  // inputs written on the caller's stream come first
    GAP_CUDA(c, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    if (cudaEventRecord(ready, c->stream) != cudaSuccess) {
        cudaEventDestroy(ready);
        return fail(c, GAP_ERR_CUDA, "cudaEventRecord failed");
    }
    // each fit goes to the lane with the least estimated work so far, longest first (greedy
    // LPT, Sec. III.B): the same batch gives every lane the same fits in the same order on
    // every call, so a lane's buffers stay put after its first (largest) fit and its QR graphs
    // are replayed on later calls
    std::vector<std::vector<int>> plan(L);
    {
        std::vector<double> load(L, 0.0);
        for (int k : order) {
            const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            plan[l].push_back(k);
            load[l] += cost(k);
        }
    }
    std::atomic<bool> failed{false};
    std::mutex mu;
    gap_status first = GAP_OK;
    std::string first_err;
    std::vector<std::thread> th;
    for (int l = 0; l < L; ++l) {
        th.emplace_back([&, l]() {
            gap_ctx *w = c->lanes[l];
            gap_status ls = cudaSetDevice(c->device) == cudaSuccess &&
                                    cudaStreamWaitEvent(w->stream, ready, 0) == cudaSuccess
                                ? GAP_OK
                                : GAP_ERR_CUDA;
            int k = -1;
            for (size_t i = 0; i < plan[l].size() && ls == GAP_OK && !failed.load(); ++i) {
                k = plan[l][i];
                ls = run_fit(w, probs[k], c_dev[k], infos ? &infos[k] : nullptr);
            }
            if (ls != GAP_OK) {
                failed.store(true);
                std::lock_guard<std::mutex> g(mu);
                if (first == GAP_OK) {
                    first = ls;
                    first_err = (k >= 0 ? "fit " + std::to_string(k) + ": " : std::string()) + w->err;
                }
            }
        });
    }
    for (auto &t : th) t.join();
    cudaEventDestroy(ready);
    if (first != GAP_OK) return fail(c, first, first_err);
    return GAP_OK;
}

}  // extern "C"
