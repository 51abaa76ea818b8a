// gap_predict_static: predictions of a fitted model that allocate nothing.
//
// The scratch the prediction kernels need (a status word, configuration ids,
// per-atom energies, per-atom gradients and a block of per-sparse-point
// weights) lives in one file-scope device array of fixed size instead of
// memory from cudaMalloc.  Host code cannot use the array's name as a device
// address (it is a host-side stand-in), so its address is resolved with
// cudaGetSymbolAddress once per device, with that device current, and passed
// to the kernels.  The resolved address is kept with the driver context it
// belongs to: after a cudaDeviceReset the library's module is loaded again into
// a new context, and the address is resolved again.
#include <cuda.h>

#include <mutex>
#include <string>

#include "gap_internal.cuh"

namespace {

__device__ __align__(256) unsigned char g_predict_scratch[GAP_PREDICT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// The calling thread's current driver context (null if none is current yet).
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (Fn)p;
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

void put_err(char *buf, size_t len, const std::string &msg) {
    if (!buf || len == 0) return;
    size_t n = msg.size() < len - 1 ? msg.size() : len - 1;
    msg.copy(buf, n);
    buf[n] = '\0';
}

// Device address of the scratch array on the current device: resolved on the first
// call on each device, and again whenever that device's context has changed.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    const CUcontext cur = current_context();
    if (!g_scratch_addr[dev] || !cur || cur != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_predict_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_context();  // current now: the symbol lookup made it so
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

gap_status read_static_status(const gap::DevStatus *st, cudaStream_t s, char *err, size_t err_len, const char *what) {
    gap::DevStatus h{};
    if (cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        put_err(err, err_len, "CUDA error while reading the validation status");
        return GAP_ERR_CUDA;
    }
    if (h.code != 0) {
        put_err(err, err_len, std::string(what) + " (index " + std::to_string((long long)h.index) + ")");
        return (gap_status)h.code;
    }
    return GAP_OK;
}

}  // namespace

extern "C" gap_status gap_predict_static(const gap_problem *t, const double *c_dev, double *E_dev, double *F_dev,
                                         void *cuda_stream, char *err, size_t err_len) {
    put_err(err, err_len, "");
    if (!t || !c_dev || !E_dev) {
        put_err(err, err_len, "targets, c_dev and E_dev are required");
        return GAP_ERR_INVALID;
    }
    if (t->memory != GAP_MEM_DEVICE) {
        put_err(err, err_len, "gap_predict_static takes device pointers only (memory = GAP_MEM_DEVICE)");
        return GAP_ERR_INVALID;
    }
    if (t->n_sparse_2b > 0) {
        put_err(err, err_len, "gap_predict_static does not take a two-body block (use gap_predict)");
        return GAP_ERR_INVALID;
    }
    if (t->n_cfg < 1 || t->n_atoms < 1 || t->d < 1 || t->n_sparse < 1 || t->n_pairs < 0 || t->zeta < 1 ||
        !t->cfg_ptr || !t->X || !t->Xs || (t->atom_species == nullptr) != (t->sparse_species == nullptr)) {
        put_err(err, err_len, "invalid sizes or missing pointers in the prediction targets");
        return GAP_ERR_INVALID;
    }
    const bool forces = F_dev != nullptr && t->pair_ptr != nullptr && t->n_pairs > 0;
    if (forces && (!t->pair_src || !t->J)) {
        put_err(err, err_len, "force predictions need pair_src and J");
        return GAP_ERR_INVALID;
    }
    // scratch layout (bytes): status 256 | configuration ids 8 n_atoms | eps 8 n_atoms |
    //                         gradients 8 n_atoms d | weights 8 chunk M (chunk >= 1 atoms)
    const size_t cap = GAP_PREDICT_STATIC_SCRATCH_BYTES;
    // each factor is bounded before the products below are formed, so none of them wraps
    const bool too_big = (size_t)t->n_atoms > (cap - 256) / 16 || (size_t)t->n_sparse > cap / 8 ||
                         (forces && (size_t)t->d > (cap - 256 - 16 * (size_t)t->n_atoms) / (8 * (size_t)t->n_atoms));
    if (too_big) {
        put_err(err, err_len, "prediction needs more than the " + std::to_string(cap) +
                                  " bytes of scratch of gap_predict_static (use gap_predict)");
        return GAP_ERR_INVALID;
    }
    const size_t fixed = 256 + 16 * (size_t)t->n_atoms + (forces ? 8 * (size_t)t->n_atoms * (size_t)t->d : 0);
    const size_t per_chunk_atom = forces ? 8 * (size_t)t->n_sparse : 0;
    if (fixed + per_chunk_atom > cap) {
        put_err(err, err_len, "prediction needs " + std::to_string(fixed + per_chunk_atom) +
                                  " bytes of scratch, more than the " + std::to_string(cap) +
                                  " bytes of gap_predict_static (use gap_predict)");
        return GAP_ERR_INVALID;
    }
    int64_t chunk = t->n_atoms;
    if (forces) {
        chunk = (int64_t)((cap - fixed) / per_chunk_atom);
        if (chunk > t->n_atoms) chunk = t->n_atoms;
    }
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        put_err(err, err_len, "cudaGetSymbolAddress of the static scratch failed");
        return GAP_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char *b = (unsigned char *)base;
    gap::DevStatus *st = (gap::DevStatus *)b;
    int64_t *cfg_ids = (int64_t *)(b + 256);
    double *eps = (double *)(cfg_ids + t->n_atoms);
    double *grad = eps + t->n_atoms;
    double *wm = grad + (forces ? t->n_atoms * t->d : 0);

    gap::Dims dm{};
    dm.n_cfg = t->n_cfg;
    dm.n_atoms = t->n_atoms;
    dm.d = t->d;
    dm.forces = forces;
    dm.n_pairs = forces ? t->n_pairs : 0;
    dm.M = t->n_sparse;
    dm.N = t->n_cfg + (forces ? 3 * t->n_atoms : 0);
    dm.rows = dm.N + dm.M;
    dm.ld = dm.rows;
    dm.zeta = t->zeta;
    dm.delta = t->delta;
    dm.species = t->atom_species != nullptr;
    const int64_t *pair_ptr = forces ? t->pair_ptr : nullptr;
    const int64_t *pair_src = forces ? t->pair_src : nullptr;

    // the status word must start at zero: every call clears it
    if (cudaMemsetAsync(st, 0, sizeof(gap::DevStatus), s) != cudaSuccess) {
        put_err(err, err_len, "cudaMemsetAsync of the status word failed");
        return GAP_ERR_CUDA;
    }
    if (gap::launch_validate(dm, t->cfg_ptr, pair_ptr, pair_src, nullptr, nullptr, t->atom_species, nullptr, st, s) !=
        cudaSuccess) {
        put_err(err, err_len, "validation launch failed");
        return GAP_ERR_CUDA;
    }
    gap_status rc = read_static_status(st, s, err, err_len, "invalid configuration or pair pointers");
    if (rc != GAP_OK) return rc;
    if (forces) {
        if (gap::launch_segment_ids(t->cfg_ptr, dm.n_cfg, cfg_ids, s) != cudaSuccess ||
            gap::launch_validate(dm, t->cfg_ptr, pair_ptr, pair_src, cfg_ids, nullptr, t->atom_species,
                                 t->sparse_species, st, s) != cudaSuccess) {
            put_err(err, err_len, "validation launch failed");
            return GAP_ERR_CUDA;
        }
        rc = read_static_status(st, s, err, err_len, "a pair source is outside its target's configuration");
        if (rc != GAP_OK) return rc;
    }
    cudaError_t e = gap::predict_simt(dm, t->X, t->Xs, t->atom_species, t->sparse_species, t->cfg_ptr, pair_ptr,
                                      pair_src, t->J, c_dev, E_dev, forces ? F_dev : nullptr, eps, grad, wm, chunk, s);
    if (e == cudaSuccess && F_dev && !forces) e = cudaMemsetAsync(F_dev, 0, sizeof(double) * 3 * t->n_atoms, s);
    if (e != cudaSuccess) {
        put_err(err, err_len, std::string("prediction launch failed: ") + cudaGetErrorString(e));
        return GAP_ERR_CUDA;
    }
    return GAP_OK;
}
