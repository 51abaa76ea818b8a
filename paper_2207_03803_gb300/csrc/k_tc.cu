// tcgen05 (5th-generation tensor core) assembly of the design matrix for the
// mixed precisions: the K_NM tiles of Sec. II (Eqs. 6, 7) as GEMMs over the
// descriptor dimension d, operands staged by TMA into 128B-swizzled shared
// memory, accumulators in TMEM, the power / species / Sigma epilogue and the
// segmented sum over configurations (energies) or pairs (forces) fused in.
//
// Two GEMMs share one kernel template:
//   energy pass: rows = atoms,               G[a,s]  = x_a . x_s
//     epilogue: K = delta^2 G^zeta summed over the atoms of each configuration
//               -> energy rows; W = delta^2 zeta G^(zeta-1) stored per atom.
//   force pass : transposed tiles, rows = sparse points, columns = (pair, alpha)
//               = J rows, H[s,r] = x_s . J_p[alpha]
//     epilogue: -W[src(p), s] H summed over the pairs of each target atom
//               (a running sum along each thread's columns) -> force rows (a, alpha).
// Every operand is split into slices (two TF32 or three BF16) so that one pass
// yields both matrices of the mixed precisions:
//   accumulator 0 = hi.hi                 -> the single-pass BF16/TF32 product
//                                            (the QR matrix, FP32 storage)
//   accumulator 1 = the remaining terms   -> added to accumulator 0 gives a
//                                            product accurate to FP32 (the
//                                            refinement's residual matrix).
// TF32: x = hi + lo, products hi.hi | hi.lo + lo.hi (error ~2^-22).
// BF16: x = h + m + l, products h.h | h.m + m.h + h.l + l.h + m.m (~2^-24).
// FP16 (force pass of the FP16 precision): each operand row scaled by a power of two
// 2^e, x 2^e = f + g (FP16 hi and lo), products f.f | f.g + g.f (error ~2^-22, as for
// TF32, at the 16-bit rate: FP16 keeps 11 significant bits, so two slices carry about
// 22 where BF16 needs three); the epilogue undoes the scales 2^(e_row + e_col).
//
// Kernel organisation (persistent, one CTA per SM, 192 threads):
//   warp 0   : TMA producer (one elected thread), STAGES-deep smem ring
//   warp 1   : TMEM allocation and the MMA issuer (one elected thread)
//   warps 2-5: epilogue; warp w reads TMEM lanes 32*(w%4) .. +31 (force pass: warps 2-9,
//              warps 2-5 the single-pass matrix, 6-9 the accurate one)
// TMEM holds two tile buffers x two accumulators x 128 columns (512 columns),
// so the epilogue of tile i overlaps the MMAs of tile i+1.
// Every wait is bounded: on timeout the kernel records GAP_ERR_TIMEOUT in the
// status word, stops issuing work, and still frees its TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace gap {
namespace {

constexpr int BM = 128, BN = 128;
// pairs per 128-row tile of the force pass: 126 Jacobian rows (three per pair) and two zero rows
constexpr int PPT = kForcePairsPerTile;
// epilogue modes of the GEMM kernel
constexpr int MODE_ENERGY = 0;   // energy rows + per-atom force weights (segmented over configurations)
constexpr int MODE_PREDICT = 2;  // per-atom energy partials and gradient weights c_s delta^2 zeta u^(zeta-1)
constexpr int MODE_STORE = 3;    // plain row-major store of the accurate product
constexpr int MODE_QR_UPD = 4;   // QR trailing update: C[row_off + r, col_off + c] -= product (column-major C)
constexpr int MODE_FORCE = 5;  // force rows, transposed tile: lanes = sparse points, columns = pair rows
constexpr int MODE_YSTORE = 6;   // split-K row-major store: tile t = (split, column tile), rows 0..127
constexpr int MODE_Y2 = 7;       // the split-K store for two A operands (rows 0..127, 128..255) sharing B
// operand kinds: 0 = TF32 split (hi, lo), 1 = BF16 split (h, m, l), 2 = plain TF32 (one pass),
// 3 = scaled FP16 split (f, g: the force pass of the FP16 precision)
template <int KIND>
__host__ __device__ constexpr int n_slices() { return KIND == 0 || KIND == 3 ? 2 : (KIND == 1 ? 3 : 1); }
// elements of one 128-byte operand row (one k-block)
template <int KIND>
__host__ __device__ constexpr int kb_elems() { return KIND == 1 || KIND == 3 ? 64 : 32; }
// operand tiles per k-block: A slices, B slices (MODE_Y2: two A operands, one B)
template <int KIND, int MODE>
__host__ __device__ constexpr int na_tiles() { return MODE == MODE_Y2 ? 2 : n_slices<KIND>(); }
template <int KIND, int MODE>
__host__ __device__ constexpr int nb_tiles() { return MODE == MODE_Y2 ? 1 : n_slices<KIND>(); }
template <int MODE>
__host__ __device__ constexpr bool split_k() { return MODE == MODE_YSTORE || MODE == MODE_Y2; }
// tile columns (MMA N) and accumulator buffers: MODE_Y2 takes 256-column B tiles, its two
// accumulators then filling TMEM without double buffering (its tiles run long K ranges)
template <int MODE>
__host__ __device__ constexpr int bn_of() { return MODE == MODE_Y2 ? 256 : 128; }
template <int MODE>
__host__ __device__ constexpr int nbuf_of() { return MODE == MODE_Y2 ? 1 : 2; }
constexpr int EPI = 16;              // epilogue column chunk
constexpr int VSTR = 2 * EPI + 1;    // shared-memory row stride of the epilogue buffer
constexpr uint32_t TMEM_COLS = 512;  // 2 buffers x 2 accumulators x BN
constexpr int NTHREADS = 192;
// threads of the GEMM kernel: producer warp, MMA warp, then 4 epilogue warps (8 in the
// force pass: two per TMEM lane quarter, one per output matrix)
template <int MODE>
__host__ __device__ constexpr int epi_warps() { return MODE == MODE_FORCE ? 8 : 4; }
template <int MODE>
__host__ __device__ constexpr int gemm_threads() { return 64 + 32 * epi_warps<MODE>(); }
constexpr uint32_t SLICE_BYTES = BM * 128;  // one 128-row x 128-byte swizzled tile
// force pass: a tile's outputs per sparse point are one run of consecutive rows
// (consecutive target atoms); up to FSMAX of them are staged per lane, in a window of
// FSW rows starting at the run's first row rounded down to a multiple of 4, and the
// window is added to the output column by a bulk reduce-add.  Staging [32 lanes][FSW]
// floats per warp (one matrix each): warps 0-4 in the epilogue buffer V, warps 5-7 and
// the run's 1/sigma in an extra region.
constexpr int FSMAX = 21;
constexpr int FSW = 24;                 // window rows: FSMAX plus up to 3 of alignment
constexpr int FST1 = 32 * FSW;          // one warp's staging
template <int MODE>
constexpr size_t mode_extra_bytes() {
    // + 128: the region starts at the next 128-byte boundary (the staging windows are read by
    // tensor bulk copies, whose shared-memory side must be 128-byte aligned)
    return MODE == MODE_FORCE ? (size_t)(3 * FST1 + 64) * 4 + 128 : 0;
}

struct Params {
    int64_t R, M, ld, n_cfg, n_pairs;
    int w_vec4;  // rows of W are 16-byte aligned (M % 4 == 0)
    int n_kb, n_ct;
    int64_t n_tiles;
    int64_t t_begin;  // first tile of the launch (the force pass runs in chunks of pair tiles)
    int walk;         // force pass: consecutive tiles per step of the tile walk (tile_at)
    int zeta;
    float d2, zf;
    float d2l;           // delta^2 - d2 (the low half of delta^2 as a double-float pair)
    double *E64;         // MODE_ENERGY: the accurate energy rows in FP64, row-major [n_cfg x M] (or null)
    const int64_t *cfg_ptr, *atom_cfg, *pair_ptr, *pair_src, *pair_tgt;
    // force pass, precomputed per pair slot of the pair tiles: source atom, target slot in
    // the tile's run, flags (bit 0: the pair ends its target's run in the tile, bit 1: that
    // target has pairs outside the tile); per target: the three 1/sigma; per pair tile:
    // first output row, run length, first / last target partial
    const int32_t *m_src, *m_slot;
    const uint8_t *m_flag;
    const float *m_isc, *m_iss;  // KIND 3: inverse operand scales per pair slot / per sparse point
    const float *m_inv3;
    const int64_t *t_base;
    const int32_t *t_run;
    const double *sigma;
    const int32_t *atom_sp, *sparse_sp;
    float *A_lo, *A_acc, *W;  // A_acc: row-block layout (acc_index, M + 1 columns)
    // centred operands (energy and prediction passes): x = mu + (x - mu) per descriptor, the
    // GEMM forms the centred dot product and the epilogue adds d mu_atom mu_sparse; the means
    // as FP32 pairs (null: operands not centred), dd = d
    const float *mux_h, *mux_l, *mus_h, *mus_l;
    float dd;
    int64_t row_off, col_off;  // MODE_QR_UPD: position of the updated block in C
    int kb_split;              // MODE_YSTORE / MODE_Y2: k-blocks per split
    int kb_lo, kb_hi;          // other modes: k-blocks [kb_lo, kb_hi) of every tile (kb_hi = 0: all)
    int b_row0;                // MODE_FORCE: first Jacobian row in the B operand's map (a ring slot)
    const float *cvec_h, *cvec_l;  // MODE_PREDICT: weights c [M] as FP32 pairs
    double *eps_part;    // MODE_PREDICT: [n_ct][R] per-tile energy partials
    int *status;         // DevStatus::code
};

__device__ __forceinline__ int64_t row0_of(int64_t t, const Params &P) { return (t / P.n_ct) * 128; }

// k-blocks of tile t: all of them, or one split's share for the split-K store.
template <int MODE>
__device__ __forceinline__ void kb_range(int64_t t, const Params &P, int &kb0, int &kb1) {
    if (split_k<MODE>()) {
        kb0 = (int)(t / P.n_ct) * P.kb_split;
        kb1 = min(P.n_kb, kb0 + P.kb_split);
    } else {
        kb0 = P.kb_lo;
        kb1 = P.kb_hi > 0 ? min(P.n_kb, P.kb_hi) : P.n_kb;
    }
}

// The j-th tile of this CTA.  Tiles go in groups of k consecutive ones (k = P.walk in
// the force pass, else 1), the groups strided by the grid: CTA b takes groups b,
// b + gridDim.x, ...  The CTAs working at one time cover consecutive tiles, so in the
// force pass the sparse tiles of a pair tile run together and its Jacobian slices are
// read from HBM once; a group's tiles share their pair tile (when k divides the
// sparse-tile count), so its per-row metadata is fetched once per group.  Tile indices
// grow with j: the first one past n_tiles ends the walk.
template <int MODE>
__device__ __forceinline__ int64_t tile_at(int64_t j, const Params &P) {
    const int64_t k = MODE == MODE_FORCE ? P.walk : 1;
    return P.t_begin + ((j / k) * gridDim.x + blockIdx.x) * k + j % k;
}

// Shared-memory matrix descriptor (tcgen05): K-major operand in the 128-byte
// swizzle layout written by TMA: rows of 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);        // start address
    d |= (uint64_t)(16u >> 4) << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;               // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                          // descriptor version (tcgen05)
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulate, K-major A and B, M = 128, N = NN, operand
// format fmt (kind::f16: 0 = FP16, 1 = BF16; kind::tf32: 2 = TF32), the same for A and B.
template <int NN = BN>
__device__ __forceinline__ uint32_t instr_desc_fmt(uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
template <int KIND, int NN = BN>
__device__ __forceinline__ uint32_t instr_desc() {
    // FP16 or BF16 (kind::f16), or TF32 (kind::tf32)
    return instr_desc_fmt<NN>(KIND == 3 ? 0u : (KIND == 1 ? 1u : 2u));
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if (KIND == 0 || KIND == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Both accumulators' 16 columns with one wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float *va, float *vb) {
    uint32_t r[16], u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        va[j] = __uint_as_float(r[j]);
        vb[j] = __uint_as_float(u[j]);
    }
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// all epilogue threads of the kernel (128 or 256)
template <int N>
__device__ __forceinline__ void epi_sync_n() { asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void tf32_split_dev(float x, float &hi, float &lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float rest = x - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(rest));
    hi = __uint_as_float(h);
    lo = __uint_as_float(l);
}

// Double-float arithmetic on the FP32 units (a value is the unevaluated sum h + l,
// about 48 significant bits).  two_sum_f: a + b exactly as the rounded sum plus err
// (Knuth's TwoSum).  df_mul_f: (h, l) *= (bh, bl), the product's rounding error taken
// by an FMA (Dekker's product), renormalised.
__device__ __forceinline__ float two_sum_f(float a, float b, float &err) {
    const float s = a + b;
    const float bp = s - a;
    err = (a - (s - bp)) + (b - bp);
    return s;
}
__device__ __forceinline__ void df_mul_f(float &h, float &l, float bh, float bl) {
    const float p = h * bh;
    const float e = fmaf(h, bh, -p) + (h * bl + l * bh);
    h = p + e;
    l = e - (h - p);
}

// g^z for an integer z >= 0 by square-and-multiply over the bits of z: a fixed
// sequence of multiplies with uniform predicates (z is the same for every thread), no
// data-dependent loop.  z < 64.
__device__ __forceinline__ float ipowf(float g, int z) {
    float p = 1.f, sq = g;
#pragma unroll
    for (int bit = 0; bit < 6; ++bit) {
        if (z & (1 << bit)) p *= sq;
        sq *= sq;
    }
    return p;
}

// 8-column accumulator loads of this warp's 32 lanes with their wait in one asm statement,
// so that no use of the registers can be scheduled before the wait: n consecutive groups
// of 8 columns from ta (and from tb, the second accumulator).

__device__ __forceinline__ void tmem_ld24(uint32_t ta, float *va) {
    uint32_t r[24];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                   "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
                 : "r"(ta + 0u), "r"(ta + 8u), "r"(ta + 16u)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 24; ++j) va[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld24x2(uint32_t ta, float *va, uint32_t tb, float *vb) {
    uint32_t r[48];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%48];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%49];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%50];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%51];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32,%33,%34,%35,%36,%37,%38,%39}, [%52];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40,%41,%42,%43,%44,%45,%46,%47}, [%53];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                   "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                   "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]),
                   "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]),
                   "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
                 : "r"(ta + 0u), "r"(ta + 8u), "r"(ta + 16u), "r"(tb + 0u), "r"(tb + 8u), "r"(tb + 16u)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 24; ++j) va[j] = __uint_as_float(r[j]);
#pragma unroll
    for (int j = 0; j < 24; ++j) vb[j] = __uint_as_float(r[24 + j]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t ta, float *va) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(ta + 0u)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) va[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld8x2(uint32_t ta, float *va, uint32_t tb, float *vb) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta + 0u), "r"(tb + 0u)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) va[j] = __uint_as_float(r[j]);
#pragma unroll
    for (int j = 0; j < 8; ++j) vb[j] = __uint_as_float(r[8 + j]);
}

// ------------------------------------------------------ force epilogue --
// What a flush of the force epilogue needs besides the three sums.
struct FlushCtx {
    float *stg;            // this warp's staging [32 lanes][FSW] (window row, per lane)
    float *out;            // matrix m: A_lo (column-major, ld) or A_acc (row-block layout)
    const float *inv3;     // 1/sigma per target row (unstaged path)
    const float *sinv3;    // 1/sigma of the run's rows, in shared memory (staged path)
    int64_t ld, nc;        // leading dimension of A_lo; columns of the row-block layout
    int64_t s, base_row;   // this lane's sparse point; first output row of the tile's run
    int64_t kf;            // the tile's first target
    int off;               // the run's first row within the staging window (base_row mod 4)
    float iss;             // KIND 3: the inverse scale of the lane's sparse point (else 1)
    int lane;
    int sv, staged;
};

// The three component sums of one target (slot sl of the tile's run) leave the
// registers, scaled by -1/sigma: into the lane's staging window, or, for runs longer than
// the staging, straight to the output rows (added when the target has pairs outside the
// tile, or in a later K-chunk).  Out of line: the unrolled pair loop calls it at every
// pair that may end a target, and is taken about three times per tile.
template <int M, int ACC>
__device__ __noinline__ void force_flush(float c0, float c1, float c2, int sl, int part, FlushCtx fc) {
    const float v[3] = {c0 * fc.iss, c1 * fc.iss, c2 * fc.iss};
    if (fc.staged) {
        // lane windows are FSW = 24 words apart, so the 8 lanes of one residue mod 4 share
        // a bank per component: they write the three components in rotated order (3-way
        // instead of 8-way bank conflicts)
        const int rot = (fc.lane >> 2) % 3;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int qa = rot + j < 3 ? rot + j : rot + j - 3;
            const float x = qa == 0 ? v[0] : (qa == 1 ? v[1] : v[2]);
            fc.stg[fc.lane * FSW + fc.off + 3 * sl + qa] = -x * fc.sinv3[3 * sl + qa];
        }
        return;
    }
    if (!fc.sv) return;
#pragma unroll
    for (int qa = 0; qa < 3; ++qa) {
        const int64_t row = fc.base_row + 3 * sl + qa;
        const float x = -v[qa] * fc.inv3[3 * (fc.kf + sl) + qa];
        float *dst = M == 0 ? fc.out + row + fc.s * fc.ld : fc.out + acc_index(row, fc.s, fc.nc);
        if (part)
            atomicAdd(dst, x);
        else if (ACC)
            *dst += x;
        else
            *dst = x;
    }
}

// Warp (q, M) of a force tile: per pair k (columns 3k + alpha of the accumulators), the
// weighted products W[src_k, s] H[3k + alpha, s] of matrix M (0: accumulator 0, the
// single-pass product; 1: accumulators 0 + 1, the accurate product) summed per target,
// flushed at the pair that ends each target's run.  The pair loop is unrolled, so every
// accumulator column and weight register index is a constant; the columns come in
// groups of 8 pairs (three 8-column loads per accumulator).
template <int KIND, int M, int ACC>
__device__ __forceinline__ void force_sums(uint32_t tb, const float (&w)[PPT], const int *s_slot,
                                           const uint8_t *s_fl, const float *s_isc, const FlushCtx &fc) {
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
    for (int g = 0; g < (PPT + 7) / 8; ++g) {
        const int np = PPT - 8 * g < 8 ? PPT - 8 * g : 8;
        float a[24], b[24];
        if (np == 8) {
            if (M) tmem_ld24x2(tb + 24 * g, a, tb + BN + 24 * g, b);
            else tmem_ld24(tb + 24 * g, a);
        } else {
            if (M) tmem_ld8x2(tb + 24 * g, a, tb + BN + 24 * g, b);
            else tmem_ld8(tb + 24 * g, a);
        }
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            if (kk < np) {
                const int k = 8 * g + kk;
                float v0 = a[3 * kk], v1 = a[3 * kk + 1], v2 = a[3 * kk + 2];
                if (M) {
                    v0 += b[3 * kk];
                    v1 += b[3 * kk + 1];
                    v2 += b[3 * kk + 2];
                }
                const float wk = KIND == 3 ? w[k] * s_isc[k] : w[k];  // KIND 3: the pair's scale 2^-e
                c0 = fmaf(wk, v0, c0);
                c1 = fmaf(wk, v1, c1);
                c2 = fmaf(wk, v2, c2);
                const int f = s_fl[k];
                if (f & 1) {  // the same for every lane: no divergence
                    force_flush<M, ACC>(c0, c1, c2, s_slot[k], (f >> 1) & 1, fc);
                    __syncwarp();  // converged again before the next accumulator load
                    c0 = c1 = c2 = 0.f;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ kernel --
// ACC (MODE_FORCE): add the output rows to A and A_acc instead of storing them (the
// K-chunks after the first); a template parameter, so that the one-chunk kernel keeps
// its store path as it is.
template <int KIND, int STAGES, int MODE, int ACC = 0>
__global__ void __launch_bounds__(gemm_threads<MODE>(), 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
              const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
              const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2,
              const __grid_constant__ CUtensorMap tC, const __grid_constant__ CUtensorMap tD, Params P) {
    constexpr int S = n_slices<KIND>();    // operand slices
    constexpr int SA = na_tiles<KIND, MODE>(), SB = nb_tiles<KIND, MODE>();
    constexpr bool ACC1 = KIND != 2 || MODE == MODE_Y2;  // the second accumulator is used
    constexpr int BNm = bn_of<MODE>(), NBUF = nbuf_of<MODE>();
    constexpr uint32_t B_BYTES = BNm * 128;  // one B tile: BNm rows of 128 bytes
    constexpr uint32_t STAGE_BYTES = SA * SLICE_BYTES + SB * B_BYTES;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // epilogue staging: force-row runs, or the QR update's reduce-add tiles
    float *V = (float *)(smem + STAGES * STAGE_BYTES);  // [128 x VSTR] floats
    // per tile column (transposed passes): metadata arrays of 128 entries
    int64_t *skey = (int64_t *)(V + 128 * VSTR);  // force: output row
    int64_t *srow = skey + 128;                   // force: run descriptor; energy: atom species
    int *send = (int *)(srow + 128);              // force: source atom; energy: configuration
    int *spart = send + 128;                      // 1 if the segment reaches outside the tile
    float *sinv = (float *)(spart + 128);         // energy: 1/sigma of the segment's row
    unsigned *smask = (unsigned *)(sinv + 128);   // [4] segment ends, one bit per column
    int *sflag = (int *)(smask + 4);              // [4] shared abort flags
    uint64_t *bars = (uint64_t *)(sflag + 4);
    uint64_t *full = bars, *empty = bars + STAGES, *tfull = bars + 2 * STAGES, *tempty = bars + 2 * STAGES + 2;
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * STAGES + 4);
    // mode_extra_bytes<MODE>(), 128-byte aligned (tensor bulk copies read staging windows here)
    float *xtra = (float *)(((uintptr_t)(tmem_slot + 2) + 127) & ~(uintptr_t)127);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 32 * epi_warps<MODE>());
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------- TMA producer --
        if (lane == 0) {
            const CUtensorMap *ta[3] = {&tA0, &tA1, &tA2};
            const CUtensorMap *tb[3] = {&tB0, &tB1, &tB2};
            // split-K Y products: the reflector tiles (A) are read by every column tile of
            // their split, which run at the same time; the trailing matrix (B) is read once
            constexpr bool HINT = MODE == MODE_Y2 || MODE == MODE_YSTORE;
            const uint64_t pol_a = HINT ? l2_policy_evict_last() : 0, pol_b = HINT ? l2_policy_evict_first() : 0;
            uint32_t it = 0;
            bool ok = true;
            int64_t t;
            for (int64_t j = 0; (t = tile_at<MODE>(j, P)) < P.n_tiles && ok; ++j) {
                // A rows: the tile's row block (sparse points for the transposed force pass)
                const int rb = split_k<MODE>() ? 0 : (int)((t / P.n_ct) * BM), cb = (int)((t % P.n_ct) * BNm);
                constexpr bool TR = MODE == MODE_FORCE || MODE == MODE_ENERGY;  // transposed tiles
                const int row0 = TR ? cb : rb, col0 = TR ? rb - P.b_row0 : cb;
                int kb0, kb1;
                kb_range<MODE>(t, P, kb0, kb1);
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, P.status)) { ok = false; break; }
                    unsigned char *st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&full[s], STAGE_BYTES);
#pragma unroll
                    for (int i = 0; i < SA; ++i) {
                        if (HINT)
                            tma_load_2d_hint(st + i * SLICE_BYTES, ta[i], &full[s], kb * kb_elems<KIND>(), row0, pol_a);
                        else
                            tma_load_2d(st + i * SLICE_BYTES, ta[i], &full[s], kb * kb_elems<KIND>(), row0);
                    }
#pragma unroll
                    for (int i = 0; i < SB; ++i) {
                        if (HINT)
                            tma_load_2d_hint(st + SA * SLICE_BYTES + i * B_BYTES, tb[i], &full[s], kb * kb_elems<KIND>(),
                                             col0, pol_b);
                        else
                            tma_load_2d(st + SA * SLICE_BYTES + i * B_BYTES, tb[i], &full[s], kb * kb_elems<KIND>(),
                                        col0);
                    }
                }
            }
            // drain: every load issued must land before the CTA may exit
            if (it > 0) {
                const uint32_t last = it - 1;
                for (uint32_t k = (last >= (uint32_t)STAGES ? last - STAGES + 1 : 0); k <= last; ++k)
                    mbar_wait(&full[k % STAGES], (k / STAGES) & 1, P.status);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer --
        if (lane == 0) {
            const uint32_t idesc = instr_desc<KIND, BNm>();
            uint32_t it = 0, tc = 0;
            bool ok = true;
            int64_t t;
            for (int64_t j = 0; (t = tile_at<MODE>(j, P)) < P.n_tiles && ok; ++j, ++tc) {
                const uint32_t ab = tc % NBUF, aph = (tc / NBUF) & 1;
                if (!mbar_wait(&tempty[ab], aph ^ 1, P.status)) { ok = false; break; }
                fence_after();
                const uint32_t d0 = tmem + ab * (2 * BNm), d1 = d0 + BNm;
                int kb0, kb1;
                kb_range<MODE>(t, P, kb0, kb1);
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                    if (!mbar_wait(&full[s], ph, P.status)) { ok = false; break; }
                    fence_after();
                    const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {  // four MMA k-steps of 32 bytes per 128-byte row
                        uint64_t a[SA], b[SB];
#pragma unroll
                        for (int i = 0; i < SA; ++i) a[i] = smem_desc(base + i * SLICE_BYTES + k * 32);
#pragma unroll
                        for (int i = 0; i < SB; ++i) b[i] = smem_desc(base + SA * SLICE_BYTES + i * B_BYTES + k * 32);
                        const uint32_t first = (kb == kb0 && k == 0) ? 0u : 1u;
                        mma<KIND>(d0, a[0], b[0], idesc, first);
                        if (MODE == MODE_Y2) {
                            mma<KIND>(d1, a[SA - 1], b[0], idesc, first);
                        } else if (ACC1) {
                            mma<KIND>(d1, a[0], b[SB > 1 ? 1 : 0], idesc, first);
                            mma<KIND>(d1, a[SA > 1 ? 1 : 0], b[0], idesc, 1u);
                        }
                        if (KIND == 1 && MODE != MODE_Y2) {
                            mma<KIND>(d1, a[0], b[SB - 1], idesc, 1u);
                            mma<KIND>(d1, a[SA - 1], b[0], idesc, 1u);
                            mma<KIND>(d1, a[SA > 1 ? 1 : 0], b[SB > 1 ? 1 : 0], idesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);  // frees the stage once these MMAs complete
                }
                if (!ok) break;
                mma_commit(&tfull[ab]);
            }
            // drain: the last accumulator must be complete before TMEM is freed
            if (tc > 0) mbar_wait(&tfull[(tc - 1) % NBUF], ((tc - 1) / NBUF) & 1, P.status);
        }
    } else {
        // -------------------------------------------------------- epilogue --
        // Warp w reads TMEM lanes 32 (w % 4) .. +31.  The energy and force passes take
        // transposed tiles (lanes = sparse points) and run their segmented sums in
        // registers; the other modes own one output row per lane.
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int lt = q * 32 + lane;           // TMEM lane of this thread
        const int et = (warp - 2) * 32 + lane;  // epilogue thread id
        uint32_t tc = 0;
        if (MODE == MODE_FORCE) {
            // Transposed force tile: TMEM lane = sparse point s, accumulator column = row
            // 3k + alpha of the pair tile (pair k of its PPT consecutive pairs; the pairs of a
            // target atom adjacent).  Warp (q, m) forms matrix m for the 32 sparse points of
            // lane quarter q: m = 0 the single-pass product (the QR matrix), m = 1 the
            // accurate product (the refinement's matrix), so that every warp sees all columns
            // and writes each target's sums once, with plain stores:
            //   F[a, alpha, s] = -(1/sigma) sum over pairs p of a of W[src(p), s] H[3p+alpha, s].
            // The 32 lanes of a warp read W[src, s] for 32 consecutive s.  Per pair tile, the
            // pairs' metadata (source, target slot, flags) and the run's 1/sigma come into
            // shared memory once (consecutive tiles of a CTA's walk share their pair tile).
            constexpr int NE = 32 * epi_warps<MODE>();  // epilogue threads
            const int wi = warp - 2, m = wi >> 2;
            int *s_src = send;                                   // [PPT] source atom (-1: none)
            int *s_slot = spart;                                 // [PPT] target slot in the tile's run
            uint8_t *s_fl = reinterpret_cast<uint8_t *>(skey);   // [PPT] bit 0 end, bit 1 partial
            float *s_isc = sinv;                                 // [PPT] KIND 3: pair scales 2^-e
            float *s_inv3 = xtra + 3 * FST1;                     // [FSMAX]: 1/sigma of the run's rows
            int64_t *s_base = srow;
            int *s_run = (int *)(srow + 1);
            float *stg = wi < 5 ? V + wi * FST1 : xtra + (wi - 5) * FST1;
            float *mine = stg + lane * FSW;  // this lane's window (16-byte aligned: FSW % 4 == 0)
            float w[PPT];
            bool have_w = false;
            int64_t cur_pt = -1, t;
            for (int64_t j = 0; (t = tile_at<MODE>(j, P)) < P.n_tiles; ++j, ++tc) {
                const uint32_t ab = tc & 1, aph = (tc >> 1) & 1;
                const int64_t pt = t / P.n_ct, st = t % P.n_ct;
                if (pt != cur_pt) {
                    epi_sync_n<NE>();  // every reader of the previous pair tile's metadata is done
                    if (et < PPT) {
                        const int64_t i = pt * PPT + et;
                        s_src[et] = P.m_src[i];
                        s_slot[et] = P.m_slot[i];
                        s_fl[et] = P.m_flag[i];
                    }
                    if (KIND == 3 && et < PPT) s_isc[et] = P.m_isc[pt * PPT + et];
                    if (et == 0) {
                        *s_base = P.t_base[pt];
                        s_run[0] = P.t_run[3 * pt];
                        s_run[1] = P.t_run[3 * pt + 1];
                        s_run[2] = P.t_run[3 * pt + 2];
                    }
                    epi_sync_n<NE>();
                    // the run's 1/sigma (targets kf .. kf + L/3 - 1), when it fits the staging
                    const int L0 = s_run[0];
                    if (et < L0 && L0 <= FSMAX) s_inv3[et] = P.m_inv3[3 * ((*s_base - P.n_cfg) / 3) + et];
                    cur_pt = pt;
                    have_w = false;
                    epi_sync_n<NE>();
                }
                const int64_t s = st * BN + lt;
                const bool sv = s < P.M;
                if (!have_w) {  // the weights of this tile's pairs (else fetched during the last tile)
                    const float *wcol = P.W + (sv ? s : 0);
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const int src = s_src[k];
                        w[k] = (sv && src >= 0) ? __ldg(wcol + (int64_t)src * P.M) : 0.f;
                    }
                }
                const int L = s_run[0];
                const bool staged = L > 0 && L <= FSMAX;
                const int64_t base_row = *s_base;
                // the window starts zeroed: its rows outside the run, and the rows of targets
                // without pairs (atoms with no neighbours), add nothing.  The last tile's bulk
                // reduce-adds have read it by now; the wait makes sure.
                if (staged) {
                    bulk_wait_read0();  // this lane's reduce-adds (lane 0: the warp's tensor one)
                    __syncwarp();
#pragma unroll
                    for (int r = 0; r < FSW; r += 4) *reinterpret_cast<float4 *>(mine + r) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                int *fl = &sflag[tc & 1];
                if (et == 0) *fl = mbar_wait(&tfull[ab], aph, P.status) ? 0 : 1;
                epi_sync_n<NE>();
                if (*fl != 0) break;
                fence_after();
                const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + ab * (2 * BN);
                FlushCtx fc;
                fc.stg = stg;
                fc.out = m == 0 ? P.A_lo : P.A_acc;
                fc.inv3 = P.m_inv3;
                fc.sinv3 = s_inv3;
                fc.ld = P.ld;
                fc.nc = P.M + 1;
                fc.s = sv ? s : 0;
                fc.base_row = base_row;
                fc.kf = (base_row - P.n_cfg) / 3;
                fc.off = (int)(base_row & 3);
                fc.iss = (KIND == 3 && sv) ? P.m_iss[s] : 1.f;
                fc.lane = lane;
                fc.sv = sv;
                fc.staged = staged;
                if (m == 0)
                    force_sums<KIND, 0, ACC>(tb, w, s_slot, s_fl, s_isc, fc);
                else
                    force_sums<KIND, 1, ACC>(tb, w, s_slot, s_fl, s_isc, fc);
                fence_before();
                mbar_arrive(&tempty[ab]);  // TMEM is read: the MMAs may go on
                // the next tile of the walk on the same pair tile: its weights are fetched
                // now, while this tile's run is written out
                const int64_t tn = tile_at<MODE>(j + 1, P);
                have_w = tn < P.n_tiles && tn / P.n_ct == pt;
                if (have_w) {
                    const int64_t sn = (tn % P.n_ct) * BN + lt;
                    const bool svn = sn < P.M;
                    const float *wcol = P.W + (svn ? sn : 0);
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const int src = s_src[k];
                        w[k] = (svn && src >= 0) ? __ldg(wcol + (int64_t)src * P.M) : 0.f;
                    }
                }
                if (staged) {
                    // the warp's runs (scaled by -1/sigma at the flush) go to the output by the bulk
                    // copy engine as one tensor reduce-add of the staging [32 sparse points][FSW
                    // rows], the window starting at the run's first row rounded down to a
                    // multiple of 4: A_lo is column-major (rows past the matrix are dropped);
                    // A_acc in 32-row blocks is seen as 32 rows x (blocks x (M + 1)) columns, so
                    // a window crossing a block boundary sends its rows past the boundary by
                    // per-lane bulk reduce-adds.  Adding onto the zeroed matrices serves whole
                    // runs, the first / last target's partial sums and later K-chunks alike;
                    // lanes past the sparse points hold zeros.
                    const int off = (int)(base_row & 3);
                    fence_proxy_async();
                    __syncwarp();
                    const int64_t row0 = base_row - off, s0 = st * BN + q * 32;
                    if (m == 0) {
                        if (lane == 0) {
                            tma_reduce_add_2d(&tC, stg, (int)row0, (int)s0);
                            bulk_commit();
                        }
                    } else {
                        const int x0 = (int)(row0 % ACC_RB), n1 = ACC_RB - x0;
                        if (lane == 0) {
                            tma_reduce_add_2d(&tD, stg, x0, (int)((row0 / ACC_RB) * (P.M + 1) + s0));
                            bulk_commit();
                        }
                        // the window's rows in the next block (rounded up to 4, within ld)
                        const int64_t nw = min((int64_t)((off + L + 3) & ~3), P.ld - row0);
                        if (nw > n1 && sv) {
                            bulk_reduce_add_f32(P.A_acc + acc_index(row0 + n1, s, P.M + 1), mine + n1,
                                                (uint32_t)(4 * (nw - n1)));
                            bulk_commit();
                        }
                    }
                }
            }
            bulk_wait_all();  // every reduce-add of this lane has landed before the CTA ends
        } else if (MODE == MODE_PREDICT || MODE == MODE_STORE || MODE == MODE_QR_UPD || split_k<MODE>()) {
            // row-wise epilogues: no segments, each thread owns one output row
            for (int64_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x, ++tc) {
                const uint32_t ab = tc % NBUF, aph = (tc / NBUF) & 1;
                const int64_t ct = t % P.n_ct;
                // split-K store: tile row block 0 of split t / n_ct, written to that split's slab
                const int64_t row = (split_k<MODE>() ? 0 : (t / P.n_ct) * BM) + lt, col0 = ct * BNm;
                float *const Wout = split_k<MODE>() ? P.W + (t / P.n_ct) * P.R * P.M : P.W;
                const bool valid = row < P.R;
                const int32_t my_sp = (MODE == MODE_PREDICT && valid && P.atom_sp) ? P.atom_sp[row] : 0;
                // MODE_PREDICT: the tile's per-column values (c as an FP32 pair, the sparse
                // points' means, their species) into shared memory, one column per thread,
                // alternating by tile (the barrier below orders both uses)
                float *ctab = V + (tc & 1) * 5 * BM;
                int *ctab_sp = reinterpret_cast<int *>(ctab + 4 * BM);
                if (MODE == MODE_PREDICT) {
                    const int64_t sc = col0 + et;
                    const bool ok = sc < P.M;
                    ctab[et] = ok ? P.cvec_h[sc] : 0.f;
                    ctab[BM + et] = ok ? P.cvec_l[sc] : 0.f;
                    ctab[2 * BM + et] = ok && P.mux_h ? P.mus_h[sc] : 0.f;
                    ctab[3 * BM + et] = ok && P.mux_h ? P.mus_l[sc] : 0.f;
                    ctab_sp[et] = ok && P.sparse_sp ? P.sparse_sp[sc] : 0;
                }
                // no barrier separates consecutive tiles here, so the flag slot alternates
                int *fl = &sflag[tc & 1];
                if (et == 0) *fl = mbar_wait(&tfull[ab], aph, P.status) ? 0 : 1;
                epi_sync();
                if (*fl != 0) break;
                fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + ab * (2 * BNm);
                float eh = 0.f, el = 0.f;  // MODE_PREDICT: energy partial in double-float
                float pxh = 0.f, pxl = 0.f;  // MODE_PREDICT, centred operands: d mu_a as an FP32 pair
                if (MODE == MODE_PREDICT && P.mux_h && valid) {
                    pxh = P.dd * P.mux_h[row];
                    pxl = fmaf(P.dd, P.mux_h[row], -pxh) + P.dd * P.mux_l[row];
                }
                if (MODE == MODE_QR_UPD) {
                    // C -= D through the TMA: -D goes to a shared staging tile (column j's 128
                    // rows contiguous) and a bulk tensor reduce-add adds it to C in L2.  Two
                    // staging buffers; one elected thread issues, commits and drains the ops.
                    const int x0 = (int)(P.row_off + row0_of(t, P)), y0 = (int)(P.col_off + col0);
                    for (int ch = 0; ch < BN / EPI; ++ch) {
                        float *stg = V + (ch & 1) * (EPI * 128);
                        if (ch >= 2) {
                            if (et == 0) bulk_wait_read1();  // the op that read this buffer is done
                            epi_sync();
                        }
                        float a0[EPI], a1[EPI];
                        if (ACC1) {
                            tmem_ld16x2(tbase + ch * EPI, tbase + BN + ch * EPI, a0, a1);
                        } else {
                            tmem_ld16(tbase + ch * EPI, a0);
#pragma unroll
                            for (int j = 0; j < EPI; ++j) a1[j] = 0.f;
                        }
#pragma unroll
                        for (int j = 0; j < EPI; ++j) stg[j * 128 + lt] = -(a0[j] + a1[j]);
                        fence_proxy_async();
                        epi_sync();
                        if (et == 0) {
                            tma_reduce_add_2d(&tC, stg, x0, y0 + ch * EPI);
                            bulk_commit();
                        }
                    }
                    if (et == 0) bulk_wait_all();  // no reduce in flight past this tile
                    epi_sync();
                } else
                for (int ch = 0; ch < BNm / EPI; ++ch) {
                    float a0[EPI], a1[EPI];
                    if (ACC1) {
                        tmem_ld16x2(tbase + ch * EPI, tbase + BNm + ch * EPI, a0, a1);
                    } else {
                        tmem_ld16(tbase + ch * EPI, a0);
#pragma unroll
                        for (int j = 0; j < EPI; ++j) a1[j] = 0.f;
                    }
                    const int64_t s0 = col0 + ch * EPI;
#pragma unroll
                    for (int j = 0; j < EPI; ++j) {
                        const int64_t s = s0 + j;
                        float out = MODE == MODE_Y2 ? a0[j] : a0[j] + a1[j];  // Y2: two outputs
                        if (MODE == MODE_PREDICT && P.mux_h && valid && s < P.M) {
                            // centred operands: out += d mu_a mu_s (double-float bulk)
                            const float mh = ctab[2 * BM + ch * EPI + j], ml = ctab[3 * BM + ch * EPI + j];
                            const float ph = pxh * mh;
                            const float pe = fmaf(pxh, mh, -ph) + (pxh * ml + pxl * mh);
                            out = ph + (pe + out);
                        }
                        if (MODE == MODE_PREDICT) {
                            float wv = 0.f;
                            if (valid && s < P.M && (!P.atom_sp || ctab_sp[ch * EPI + j] == my_sp)) {
                                const float uz1 = ipowf(out, P.zeta - 1);
                                const float chv = ctab[ch * EPI + j], cl = ctab[BM + ch * EPI + j];
                                const float v = P.d2 * uz1 * out;
                                const float pr = chv * v;
                                const float er = fmaf(chv, v, -pr) + cl * v;
                                const float sm = eh + pr;
                                const float bp = sm - eh;
                                el += ((eh - (sm - bp)) + (pr - bp)) + er;
                                eh = sm;
                                wv = chv * P.d2 * P.zf * uz1;
                            }
                            out = wv;
                        }
                        a0[j] = out;
                    }
                    // ACC (MODE_STORE, K-chunks after the first): add to what is there
                    auto store = [&](float *dst, const float *v) {
                        if (s0 + EPI <= P.M && P.w_vec4) {
                            float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
                            for (int j4 = 0; j4 < EPI / 4; ++j4) {
                                float4 o = make_float4(v[4 * j4], v[4 * j4 + 1], v[4 * j4 + 2], v[4 * j4 + 3]);
                                if (ACC) {
                                    const float4 q = d4[j4];
                                    o.x += q.x;
                                    o.y += q.y;
                                    o.z += q.z;
                                    o.w += q.w;
                                }
                                d4[j4] = o;
                            }
                        } else {
                            for (int j = 0; j < EPI && s0 + j < P.M; ++j) dst[j] = ACC ? dst[j] + v[j] : v[j];
                        }
                    };
                    if (valid && Wout != nullptr) {
                        store(Wout + row * P.M + s0, a0);
                        if (MODE == MODE_Y2) store(Wout + (row + BM) * P.M + s0, a1);  // second A operand
                    }
                }
                if (MODE == MODE_PREDICT && valid) P.eps_part[ct * P.R + row] = (double)eh + (double)el;
                fence_before();
                mbar_arrive(&tempty[ab]);
            }
        } else {
            // Energy pass, transposed tile: TMEM lane = sparse point s, accumulator column
            // = atom a of the tile (the atoms of one configuration adjacent).  Per (a, s):
            // g = x_a . x_s (single-pass g0 and accurate g), W[a, s] = delta^2 zeta g^(zeta-1)
            // (stored: the 32 lanes of a warp write 32 consecutive s), and the running sums
            // of delta^2 g0^zeta and delta^2 g^zeta over the atoms of each configuration,
            // written (or added, when the configuration reaches outside the tile) with
            // 1/sigma at its last atom in the tile.  Per-atom metadata: thread et = atom et.
            int *s_cfg = send, *s_part = spart, *s_sp = (int *)srow;
            float *s_invl = (float *)srow + BM;                 // low half of 1/sigma (sinv: high)
            float *s_mxh = (float *)skey, *s_mxl = s_mxh + BM;  // atom means (centred operands)
            for (int64_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x, ++tc) {
                const uint32_t ab = tc & 1, aph = (tc >> 1) & 1;
                const int64_t a0 = (t / P.n_ct) * BM, st = t % P.n_ct;
                epi_sync();  // every reader of the previous tile's metadata is done
                {
                    const int64_t a = a0 + et;
                    int key = -1, part = 0, sp = 0;
                    bool end = false;
                    float inv = 0.f, invl = 0.f;
                    if (a < P.R) {
                        key = (int)P.atom_cfg[a];
                        if (P.atom_sp) sp = P.atom_sp[a];
                        end = et == BM - 1 || a + 1 >= P.R || P.atom_cfg[a + 1] != key;
                        if (end) {
                            part = (P.cfg_ptr[key] < a0 || P.cfg_ptr[key + 1] > a0 + BM) ? 1 : 0;
                            const double iv = 1.0 / P.sigma[key];
                            inv = (float)iv;
                            invl = (float)(iv - (double)inv);
                        }
                    }
                    s_cfg[et] = key;
                    s_part[et] = part;
                    s_sp[et] = sp;
                    sinv[et] = inv;
                    s_invl[et] = invl;
                    if (P.mux_h) {
                        s_mxh[et] = a < P.R ? P.mux_h[a] : 0.f;
                        s_mxl[et] = a < P.R ? P.mux_l[a] : 0.f;
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, end);
                    if (lane == 0) smask[et >> 5] = m;
                }
                int *fl = &sflag[tc & 1];
                if (et == 0) *fl = mbar_wait(&tfull[ab], aph, P.status) ? 0 : 1;
                epi_sync();
                if (*fl != 0) break;
                fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + ab * (2 * BN);
                const int64_t s = st * BN + lt;
                const bool sv = s < P.M;
                const int32_t my_sp = (sv && P.sparse_sp) ? P.sparse_sp[s] : 0;
                float *wcol = P.W + (sv ? s : 0) + a0 * P.M;  // W[a0 + r, s] = wcol[r * M]
                // centred operands: d mu_s as an FP32 pair for the bulk term d mu_a mu_s
                float dsh = 0.f, dsl = 0.f;
                if (P.mux_h && sv) {
                    dsh = P.dd * P.mus_h[s];
                    dsl = fmaf(P.dd, P.mus_h[s], -dsh) + P.dd * P.mus_l[s];
                }
                // The accurate energy rows run in double-float throughout: g as a pair from the
                // centred product and its bulk term, delta^2 g^zeta, the sum over the
                // configuration's atoms and the 1/sigma scaling.  Small energy sigmas weight
                // these few rows so heavily that their FP32 rounding alone (about 3e-8) moves
                // the fitted forces by several 1e-7; the refinement reads them from E64.
                float klo = 0.f, kah = 0.f, kal = 0.f;
                constexpr int EV = 8;  // atoms whose powers are formed together (independent chains)
#pragma unroll 1
                for (int ch = 0; ch < BN / EPI; ++ch) {
                    float a0v[EPI], a1v[EPI];
                    tmem_ld16x2(tbase + ch * EPI, tbase + BN + ch * EPI, a0v, a1v);
                    const unsigned ends = (smask[ch >> 1] >> ((ch & 1) * EPI)) & 0xFFFFu;
#pragma unroll
                    for (int hb = 0; hb < EPI; hb += EV) {
                        // g of EV atoms (single-pass g0, accurate pair g + gl), then their powers
                        // side by side: pz = g^(zeta-1), p0 = g0^zeta (square and multiply over
                        // the bits of zeta, uniform across the warp), th + tl = g^zeta in
                        // double-float
                        float g[EV], gl[EV], g0[EV], th[EV], tl[EV], pz[EV], p0[EV];
#pragma unroll
                        for (int u = 0; u < EV; ++u) {
                            const int r = ch * EPI + hb + u;
                            g0[u] = a0v[hb + u];
                            g[u] = a0v[hb + u] + a1v[hb + u];
                            gl[u] = 0.f;
                            if (P.mux_h) {
                                // g = d mu_a mu_s + (x_a - mu_a) . (x_s - mu_s): the bulk in
                                // double-float, the accurate g kept as the pair (g, gl)
                                const float xh = s_mxh[r], xl = s_mxl[r];
                                const float ph = dsh * xh;
                                const float pe = fmaf(dsh, xh, -ph) + (dsh * xl + dsl * xh);
                                g0[u] = ph + (pe + g0[u]);
                                float e1, e2;
                                const float s1 = two_sum_f(g[u], pe, e1);
                                g[u] = two_sum_f(ph, s1, e2);
                                gl[u] = e1 + e2;
                            }
                            th[u] = g[u];
                            tl[u] = gl[u];
                            pz[u] = 1.f;
                            p0[u] = 1.f;
                        }
                        {
                            float sa[EV], sb[EV];
#pragma unroll
                            for (int u = 0; u < EV; ++u) {
                                sa[u] = g[u];
                                sb[u] = g0[u];
                            }
#pragma unroll
                            for (int bit = 0; bit < 6; ++bit) {
                                if ((P.zeta >> bit) == 0) break;  // uniform
                                const bool ba = ((P.zeta - 1) >> bit) & 1, bb = (P.zeta >> bit) & 1;
#pragma unroll
                                for (int u = 0; u < EV; ++u) {
                                    if (ba) pz[u] *= sa[u];
                                    if (bb) p0[u] *= sb[u];
                                    sa[u] *= sa[u];
                                    sb[u] *= sb[u];
                                }
                            }
                        }
#pragma unroll 1
                        for (int k = 1; k < P.zeta; ++k)
#pragma unroll
                            for (int u = 0; u < EV; ++u) df_mul_f(th[u], tl[u], g[u], gl[u]);
#pragma unroll
                        for (int u = 0; u < EV; ++u) {
                            const int j = hb + u;
                            const int r = ch * EPI + j;
                            const int key = s_cfg[r];
                            const bool same = key >= 0 && sv && (!P.atom_sp || s_sp[r] == my_sp);
                            if (key >= 0 && sv) wcol[(int64_t)r * P.M] = same ? P.d2 * P.zf * pz[u] : 0.f;
                            if (same) {
                                klo += P.d2 * p0[u];
                                float t1 = th[u], t2 = tl[u];  // delta^2 g^zeta as a pair
                                df_mul_f(t1, t2, P.d2, P.d2l);
                                float e;
                                kah = two_sum_f(kah, t1, e);
                                kal += e + t2;
                            }
                            if ((ends >> j) & 1u) {  // the same for every lane: no divergence
                                if (sv) {
                                    const float inv = sinv[r];
                                    float vh = kah, vl = kal;
                                    df_mul_f(vh, vl, inv, s_invl[r]);
                                    const float kac = vh + vl;
                                    float *dl = P.A_lo + (int64_t)key + s * P.ld;
                                    float *da = P.A_acc + acc_index(key, s, P.M + 1);
                                    double *de = P.E64 ? P.E64 + (int64_t)key * P.M + s : nullptr;
                                    if (s_part[r]) {
                                        atomicAdd(dl, klo * inv);
                                        atomicAdd(da, kac);
                                        if (de) atomicAdd(de, (double)vh + (double)vl);
                                    } else {
                                        *dl = klo * inv;
                                        *da = kac;
                                        if (de) *de = (double)vh + (double)vl;
                                    }
                                }
                                klo = 0.f;
                                kah = kal = 0.f;
                            }
                        }
                    }
                }
                fence_before();
                mbar_arrive(&tempty[ab]);
            }
        }
    }
    // ------------------------------------------------------------ teardown --
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// ------------------------------------------------------------ packing --
// Element (r, kk) of a packed operand, read from its source:
//   PACK_ROWS   FP64 row-major [rows x K] (descriptors, sparse points)
//   PACK_JAC    FP64 Jacobians [n_pairs x 3 x K] in pair tiles (force_pack_row): row
//               128 pt + 3 k + alpha is component alpha of pair PPT pt + k; rows 126, 127
//               of a tile and the pairs at and past jpairs (the pairs src holds) are zero
//   PACK_F32    FP32 row-major [rows x ld]
//   PACK_TRANS  FP64 transposed: element (r, kk) = src[kk * ld + r]
enum { PACK_ROWS = 0, PACK_JAC = 1, PACK_F32 = 2, PACK_TRANS = 3, PACK_CENTER = 4 };

__device__ __forceinline__ float pack_load(const void *src, int mode, int64_t r, int64_t kk, int64_t K, int64_t ld,
                                           int64_t jpairs, const double *mu) {
    if (kk >= K) return 0.f;
    switch (mode) {
    case PACK_ROWS: return (float)((const double *)src)[r * ld + kk];
    case PACK_CENTER: return (float)(((const double *)src)[r * ld + kk] - mu[r]);
    case PACK_JAC: {
        const int64_t j = r % 128, p = r / 128 * PPT + j / 3;
        return (j < 3 * PPT && p < jpairs) ? (float)((const double *)src)[(3 * p + j % 3) * ld + kk] : 0.f;
    }
    case PACK_F32: return ((const float *)src)[r * ld + kk];
    default: return (float)((const double *)src)[kk * ld + r];
    }
}

// Split packed operand [rows x K_pad] into two TF32 slices (hi, lo) in FP32 containers.
// Grid-stride over groups of four consecutive entries of a row (K_pad % 4 == 0).
__global__ void k_pack_tf32(const void *__restrict__ src, int mode, int64_t rows, int64_t K, int64_t K_pad,
                            int64_t ld, int64_t jpairs, const double *__restrict__ mu, float *__restrict__ hi,
                            float *__restrict__ lo) {
    const int64_t ng = rows * (K_pad / 4);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = 4 * g, r = e / K_pad, kk = e % K_pad;
        float4 h, l;
        tf32_split_dev(pack_load(src, mode, r, kk, K, ld, jpairs, mu), h.x, l.x);
        tf32_split_dev(pack_load(src, mode, r, kk + 1, K, ld, jpairs, mu), h.y, l.y);
        tf32_split_dev(pack_load(src, mode, r, kk + 2, K, ld, jpairs, mu), h.z, l.z);
        tf32_split_dev(pack_load(src, mode, r, kk + 3, K, ld, jpairs, mu), h.w, l.w);
        *reinterpret_cast<float4 *>(hi + e) = h;
        *reinterpret_cast<float4 *>(lo + e) = l;
    }
}

// Split into three BF16 slices x = h + m + l; after the one FP32 rounding of x the
// residuals are exact in FP32 (no FP64 arithmetic).
// Grid-stride over groups of four consecutive entries of a row (K_pad % 4 == 0).
__global__ void k_pack_bf16x3(const void *__restrict__ src, int mode, int64_t rows, int64_t K, int64_t K_pad,
                              int64_t ld, int64_t jpairs, const double *__restrict__ mu, __nv_bfloat16 *__restrict__ s0,
                              __nv_bfloat16 *__restrict__ s1, __nv_bfloat16 *__restrict__ s2) {
    const int64_t ng = rows * (K_pad / 4);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = 4 * g, r = e / K_pad, kk = e % K_pad;
        __nv_bfloat16 h[4], m[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float x = pack_load(src, mode, r, kk + u, K, ld, jpairs, mu);
            h[u] = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(h[u]);
            m[u] = __float2bfloat16_rn(r1);
            l[u] = __float2bfloat16_rn(r1 - __bfloat162float(m[u]));
        }
        *reinterpret_cast<uint2 *>(s0 + e) = *reinterpret_cast<const uint2 *>(h);
        *reinterpret_cast<uint2 *>(s1 + e) = *reinterpret_cast<const uint2 *>(m);
        *reinterpret_cast<uint2 *>(s2 + e) = *reinterpret_cast<const uint2 *>(l);
    }
}

// Force-pass operands of the FP16 precision: the FP16 pair f + g of x 2^e, e the power of
// two that puts the largest magnitude of a scale group in [2^14, 2^15): f = FP16(x 2^e)
// and g = FP16(x 2^e - f).  x 2^e - f is exact in FP32, and g keeps it to FP16's 11
// significant bits, so f + g holds x 2^e to about 2^-22 of the group's scale.  A scale
// group is one row (PACK_ROWS: a sparse point), or the three Jacobian rows of a pair
// (PACK_JAC: pair slot k of pair tile pt, rows 128 pt + 3 k + alpha), so that the force
// epilogue applies one scale per pair, to the pair's weight.  isc[group] = 2^-e (1 for a
// group of zeros); the warp of a tile's last slot also writes the tile's two zero rows.
// One warp per group; its rows are read twice (largest magnitude first), the second time
// mostly from L1.
__global__ void k_pack_force_f16(const void *__restrict__ src, int mode, int64_t rows, int64_t K, int64_t K_pad,
                                 int64_t ld, int64_t jpairs, __half *__restrict__ s1, __half *__restrict__ s2,
                                 float *__restrict__ isc) {
    const int lane = threadIdx.x & 31;
    const bool jac = mode == PACK_JAC;
    const int64_t groups = jac ? rows / 128 * PPT : rows;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < groups; gi += nwarps) {
        const int k = (int)(gi % PPT);
        const int64_t r0 = jac ? gi / PPT * 128 + 3 * k : gi;
        const int nr = jac ? 3 : 1;                         // rows of the group
        const int nz = (jac && k == PPT - 1) ? 128 - 3 * PPT : 0;  // the tile's zero rows after it
        float mx = 0.f;
        for (int u = 0; u < nr; ++u)
            for (int64_t kk = lane; kk < K; kk += 32)
                mx = fmaxf(mx, fabsf(pack_load(src, mode, r0 + u, kk, K, ld, jpairs, nullptr)));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        // mx = 1.m 2^(E - 127) (E its biased exponent), so e = 141 - E puts mx 2^e in [2^14, 2^15)
        const int E = (int)((__float_as_uint(mx) >> 23) & 0xFFu);
        const int e = E == 0 ? 0 : max(-100, min(100, 141 - E));
        const float sc = __uint_as_float((uint32_t)(127 + e) << 23);
        if (lane == 0) isc[gi] = __uint_as_float((uint32_t)(127 - e) << 23);
        for (int u = 0; u < nr + nz; ++u) {
            const int64_t r = r0 + u;
            for (int64_t kk = 4 * lane; kk < K_pad; kk += 128) {
                __half f[4], g[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float xs = pack_load(src, mode, r, kk + v, K, ld, jpairs, nullptr) * sc;
                    f[v] = __float2half_rn(xs);
                    g[v] = __float2half_rn(xs - __half2float(f[v]));
                }
                const int64_t e0 = r * K_pad + kk;
                *reinterpret_cast<uint2 *>(s1 + e0) = *reinterpret_cast<const uint2 *>(f);
                *reinterpret_cast<uint2 *>(s2 + e0) = *reinterpret_cast<const uint2 *>(g);
            }
        }
    }
}

// Row means of an FP64 row-major matrix [rows x d] (one warp per row): mu64 for the
// centred packing, and the same as FP32 pairs (mh, ml) for the epilogues.
__global__ void k_row_means(const double *__restrict__ X, int64_t rows, int64_t d, double *__restrict__ mu64,
                            float *__restrict__ mh, float *__restrict__ ml) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (r >= rows) return;
    double acc = 0.0;
    for (int64_t k = lane; k < d; k += 32) acc += X[r * d + k];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const double m = acc / (double)d;
        mu64[r] = m;
        const float h = (float)m;
        mh[r] = h;
        ml[r] = (float)(m - (double)h);
    }
}

// c as FP32 pairs (hi, lo) for the prediction epilogue's double-float sums.
__global__ void k_split_c(const double *c, int64_t n, float *ch, float *cl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float h = (float)c[i];
    ch[i] = h;
    cl[i] = (float)(c[i] - (double)h);
}

// eps[a] = sum over column tiles (fixed order) of the per-tile partials.
__global__ void k_sum_eps(const double *__restrict__ part, int64_t n_ct, int64_t n, double *__restrict__ eps) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    double e = 0.0;
    for (int64_t c = 0; c < n_ct; ++c) e += part[c * n + a];
    eps[a] = e;
}

__global__ void k_energy_from_eps(int64_t n_cfg, const int64_t *__restrict__ cfg_ptr, const double *__restrict__ eps,
                                  double *__restrict__ E) {
    int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (A >= n_cfg) return;
    double e = 0.0;
    for (int64_t i = cfg_ptr[A]; i < cfg_ptr[A + 1]; ++i) e += eps[i];
    E[A] = e;
}

// x rounded to FP32 (to nearest; exact ties round away from zero) from its IEEE-754 bit
// pattern with integer operations, so that no FP64 instruction runs: the 23 mantissa bits
// below the leading one are the top 20 of the high word and the top 3 of the low word, the
// next bit rounds (a carry out of the mantissa raises the exponent).  Magnitudes below the
// FP32 normal range become zero, above it infinity.
__device__ __forceinline__ float f64_to_f32_bits(double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    unsigned v = ((unsigned)e << 23) + m + ((lo >> 28) & 1u);
    v = e <= 0 ? 0u : (e >= 255 ? 0x7F800000u : v);
    return __uint_as_float((hi & 0x80000000u) | v);
}

// F[a] = -sum over pairs p of a of J_p g_src(p) (three components), one warp per target
// atom.  J (FP64) is rounded to FP32 by bit operations, each product J g is split exactly by
// FMA and summed in double-float (TwoSum), so no FP64 instruction runs: the kernel is
// bound by the J reads.  Atoms [a0, a1); J holds the pairs from p_base on (all of them,
// or one slot of the J ring).
__global__ void k_force_from_grad(int64_t a0, int64_t a1, int64_t d, const int64_t *__restrict__ pair_ptr,
                                  const int64_t *__restrict__ pair_src, const double *__restrict__ J, int64_t p_base,
                                  const float *__restrict__ grad, double *__restrict__ F) {
    const int64_t a = a0 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    if (a >= a1) return;
    float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
    for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p) {
        const float *g = grad + pair_src[p] * d;
        const double *j = J + (p - p_base) * 3 * d;
#pragma unroll 4
        for (int64_t k = lane; k < d; k += 32) {
            const float gk = g[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float jc = f64_to_f32_bits(j[c * d + k]);
                const float pr = jc * gk;
                const float er = fmaf(jc, gk, -pr);
                const float sm = h[c] + pr;
                const float bp = sm - h[c];
                l[c] += ((h[c] - (sm - bp)) + (pr - bp)) + er;
                h[c] = sm;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, h[c], o), ol = __shfl_down_sync(0xffffffffu, l[c], o);
            const float sm = h[c] + oh;
            const float bp = sm - h[c];
            l[c] += ((h[c] - (sm - bp)) + (oh - bp)) + ol;
            h[c] = sm;
        }
    }
    if (lane == 0) {
        F[3 * a] = -((double)h[0] + (double)l[0]);
        F[3 * a + 1] = -((double)h[1] + (double)l[1]);
        F[3 * a + 2] = -((double)h[2] + (double)l[2]);
    }
}

// ------------------------------------------------ force-pass metadata --
// Pair tiles: 128 Jacobian rows holding PPT = 42 consecutive pairs (row 3k + alpha of
// the tile is component alpha of its k-th pair) and two zero rows.  Per pair slot
// i = PPT pt + k (slots past n_pairs are padding): its source atom, its target's slot in
// the tile (target minus the tile's first target) and flags: bit 0 = the pair ends its
// target's run in the tile (its last pair, or the tile's last pair), bit 1 = that target
// has pairs outside the tile (its sums are added, not stored).
__global__ void k_force_meta_pairs(int64_t n_pairs, int64_t n_slots, const int64_t *__restrict__ pair_src,
                                   const int64_t *__restrict__ pair_tgt, const int64_t *__restrict__ pair_ptr,
                                   int32_t *m_src, int32_t *m_slot, uint8_t *m_flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots) return;
    if (i >= n_pairs) {
        m_src[i] = -1;
        m_slot[i] = 0;
        m_flag[i] = 0;
        return;
    }
    const int64_t p0 = i / PPT * PPT, p1 = min(p0 + PPT, n_pairs);
    const int64_t key = pair_tgt[i], lo = pair_ptr[key], hi = pair_ptr[key + 1];
    const bool end = i == hi - 1 || i == p1 - 1;
    const bool part = lo < p0 || hi > p0 + PPT;
    m_src[i] = (int32_t)pair_src[i];
    m_slot[i] = (int32_t)(key - pair_tgt[p0]);
    m_flag[i] = (uint8_t)((end ? 1 : 0) | (part ? 2 : 0));
}

// Per target atom a: the three 1/sigma of its force rows.
__global__ void k_force_meta_inv(int64_t n_atoms, int64_t n_cfg, const double *__restrict__ sigma, float *inv3) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 3 * n_atoms) inv3[e] = 1.0f / (float)sigma[n_cfg + e];
}

// Per pair tile: the first output row of its run (the targets of its first to its last
// pair), the run length and whether the first / last target reaches outside the tile.
__global__ void k_force_meta_tiles(int64_t n_pairs, int64_t n_pt, int64_t n_cfg, const int64_t *__restrict__ pair_tgt,
                                   const int64_t *__restrict__ pair_ptr, int64_t *t_base, int32_t *t_run) {
    const int64_t pt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pt >= n_pt) return;
    const int64_t p0 = pt * PPT;
    int64_t base = 0;
    int L = 0, fp = 0, lp = 0;
    if (p0 < n_pairs) {
        const int64_t kf = pair_tgt[p0], kl = pair_tgt[min(p0 + PPT, n_pairs) - 1];
        base = n_cfg + 3 * kf;
        L = (int)min((int64_t)(1 << 20), 3 * (kl - kf + 1));
        fp = pair_ptr[kf] < p0 ? 1 : 0;
        lp = pair_ptr[kl + 1] > p0 + PPT ? 1 : 0;
    }
    t_base[pt] = base;
    t_run[3 * pt] = L;
    t_run[3 * pt + 1] = fp;
    t_run[3 * pt + 2] = lp;
}

// ---------------------------------------------------------- host side --
// 2-D map over a row-major [rows x d_pad] slice; boxes of 128 bytes x 128 rows.
bool make_map(CUtensorMap *m, const void *base, int64_t rows, int64_t d_pad, int kind, int64_t row_stride = 0) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int esz = kind == 0 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)d_pad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)((row_stride > 0 ? row_stride : d_pad) * esz)};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), 128u};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = fn(m, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int KIND, int STAGES, int MODE>
constexpr size_t smem_bytes() {
    return 1024 + (size_t)STAGES * (na_tiles<KIND, MODE>() * SLICE_BYTES + nb_tiles<KIND, MODE>() * bn_of<MODE>() * 128) +
           128 * VSTR * 4 + 2 * 128 * 8 +
           3 * 128 * 4 + 8 * 4 + (2 * STAGES + 4) * 8 + 16 + mode_extra_bytes<MODE>();
}

template <int KIND, int STAGES, int MODE, int ACC = 0>
cudaError_t launch_gemm(const CUtensorMap *ta, const CUtensorMap *tb, const Params &P, int n_sm, cudaStream_t s,
                        const CUtensorMap *tc = nullptr, const CUtensorMap *td = nullptr) {
    auto kern = k_tc_gemm<KIND, STAGES, MODE, ACC>;
    constexpr size_t smem = smem_bytes<KIND, STAGES, MODE>();
    // raised once per instantiation (a constant; not on every launch of every lane)
    static const cudaError_t e_attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e_attr != cudaSuccess) return e_attr;
    const int grid = (int)std::min<int64_t>(P.n_tiles - P.t_begin, n_sm);
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, gemm_threads<MODE>(), smem, s>>>(ta[0], ta[1], ta[2], tb[0], tb[1], tb[2], tc ? *tc : ta[0],
                                                  td ? *td : ta[0], P);
    return cudaGetLastError();
}

cudaError_t pack_slices(int kind, const void *src, int mode, int64_t rows, int64_t K, int64_t K_pad, int64_t ld,
                        int64_t jpairs, void *s0, void *s1, void *s2, cudaStream_t s, const double *mu = nullptr) {
    if (rows == 0) return cudaSuccess;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows * (K_pad / 4), 256), 8 * n_sm));
    if (kind == 0)
        k_pack_tf32<<<nb, 256, 0, s>>>(src, mode, rows, K, K_pad, ld, jpairs, mu, (float *)s0, (float *)s1);
    else
        k_pack_bf16x3<<<nb, 256, 0, s>>>(src, mode, rows, K, K_pad, ld, jpairs, mu, (__nv_bfloat16 *)s0,
                                         (__nv_bfloat16 *)s1, (__nv_bfloat16 *)s2);
    return cudaGetLastError();
}

cudaError_t pack_force_f16(const void *src, int mode, int64_t rows, int64_t K, int64_t K_pad, int64_t ld,
                           int64_t jpairs, void *s1, void *s2, float *isc, cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // 8 warps per block, 2 blocks per SM: each warp's rows (up to 24 KB in FP64) mostly stay
    // in L1 between their two reads
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, 8), 2 * n_sm));
    k_pack_force_f16<<<nb, 256, 0, s>>>(src, mode, rows, K, K_pad, ld, jpairs, (__half *)s1, (__half *)s2, isc);
    return cudaGetLastError();
}

}  // namespace

// force-pass metadata bytes (after the operand slices, 256-byte aligned parts); the
// last two parts, the inverse FP16 scales of the Jacobian rows and of the sparse points,
// are used by the BF16 precision only
size_t force_meta_bytes(const Dims &dm) {
    if (!dm.forces) return 0;
    const int64_t rJ = force_pack_rows(dm.n_pairs), n_pt = rJ / 128, ns = n_pt * PPT;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al(4 * (size_t)ns) * 2 + al((size_t)ns) + al(12 * (size_t)dm.n_atoms) + al(8 * (size_t)n_pt) +
           al(12 * (size_t)n_pt) + al(4 * (size_t)rJ) + al(4 * (size_t)dm.M);
}

// bytes of the descriptor means (centred operands): FP64 and FP32-pair copies
size_t means_bytes(int64_t n) { return ((size_t)n * 16 + 1023) & ~(size_t)255; }

size_t tc_workspace_bytes(const Dims &dm, int64_t ring_rows) {
    const int64_t d_pad = round_up(dm.d, 64);
    const int64_t rJ = force_pack_rows(dm.n_pairs), rJs = ring_rows > 0 ? std::min(rJ, ring_rows) : rJ;
    const int64_t rows = dm.n_atoms + dm.M + (dm.forces ? rJs + dm.M : 0) +
                         (dm.virials ? force_pack_rows(2 * dm.n_atoms) : 0);
    // 2 x FP32 or 3 x BF16 slices (at most 8 bytes per element), the force (and virial)
    // metadata, the means
    return (size_t)rows * d_pad * 8 + 1024 + force_meta_bytes(dm) + (dm.virials ? force_meta_bytes(virial_dims(dm)) : 0) +
           means_bytes(dm.n_atoms + dm.M) + 512;
}

cudaError_t tc_assemble(const Dims &dm, const TcInputs &in, TcMode mode, DevBuf &ops, float *A, float *Aacc,
                        float *Wf, cudaStream_t s, Prof *prof) {
    const int kind = mode == TcMode::TF32 ? 0 : 1;  // energy pass (and the force pass but for FP16)
    const int S = kind == 0 ? 2 : 3;
    const int esz = kind == 0 ? 4 : 2;
    const int64_t d_pad = round_up(dm.d, 64);
    // force operand rows: the Jacobian rows 3 p + alpha, padded to whole tiles; virial rows
    // (force rows of pseudo-targets, k_virial.cu): the strain Jacobian rows of their pseudo-pairs
    const bool vir = dm.forces && dm.virials && in.vG != nullptr;
    const Dims vdm = virial_dims(dm);
    const int64_t rJ = dm.forces ? force_pack_rows(dm.n_pairs) : 0;
    const int64_t rV = vir ? force_pack_rows(vdm.n_pairs) : 0;
    // J ring: one slot of ring_rows packed rows stands for the whole packed J
    const bool ring = rJ > 0 && in.ring_rows > 0;
    if (ring && (vir || in.ring_rows % BM != 0 ||
                 (!in.J && !(in.h_J && (in.h_J_direct || (in.ring_buf && in.ring_stream && in.ring_ev))))))
        return cudaErrorInvalidValue;
    const int64_t rJs = ring ? std::min(rJ, in.ring_rows) : rJ;
    // slice arrays: [S][rows_all][d_pad]: X and Xs centred (energy pass), J rows (or the
    // ring slot), Xs as given (force and virial passes), then the virial Jacobian rows
    const int64_t rows_all = dm.n_atoms + dm.M + rJs + (rJ > 0 ? dm.M : 0) + rV;
    const size_t slice_elems = (size_t)rows_all * d_pad;
    const size_t meta_off = (slice_elems * esz * S + 1023) & ~(size_t)255;
    const size_t vmeta_off = (meta_off + force_meta_bytes(dm) + 255) & ~(size_t)255;
    const size_t mean_off = (vmeta_off + (vir ? force_meta_bytes(vdm) : 0) + 255) & ~(size_t)255;
    cudaError_t e = ops.ensure(mean_off + means_bytes(dm.n_atoms + dm.M) + 256);
    if (e != cudaSuccess) return e;
    unsigned char *base = ops.as<unsigned char>();
    auto slice = [&](int i, int64_t row_off) { return base + ((size_t)i * slice_elems + (size_t)row_off * d_pad) * esz; };
    // descriptor means: FP64 [n_atoms + M], then FP32 pairs (atoms, sparse points)
    const int64_t nm = dm.n_atoms + dm.M;
    double *mu64 = (double *)(base + mean_off);
    float *mxh = (float *)(mu64 + nm), *mxl = mxh + nm, *msh = mxh + dm.n_atoms, *msl = mxl + dm.n_atoms;
    // rows of src into the slices from row_off; jac: Jacobian rows, zero at and past jlimit;
    // mu: centred rows
    auto pack = [&](const double *src, int64_t rows, int64_t row_off, bool jac, int64_t jlimit,
                    const double *mu = nullptr) -> cudaError_t {
        return pack_slices(kind, src, jac ? PACK_JAC : (mu ? PACK_CENTER : PACK_ROWS), rows, dm.d, d_pad, dm.d, jlimit,
                           slice(0, row_off), slice(1, row_off), slice(2, row_off), s, mu);
    };
    // force-pass metadata (force_meta_bytes): per Jacobian row source, target, flags; per
    // target 1/sigma; per pair tile run descriptors; the FP16 precision's inverse scales
    // (rows, sparse points).  One set for the force rows, one for the virial rows.
    struct Meta {
        int32_t *src, *key;
        uint8_t *flag;
        float *inv3;
        int64_t *t_base;
        int32_t *t_run;
        float *isc, *iss;
    };
    auto meta_at = [](unsigned char *mp, int64_t rows, int64_t n_targets) {
        auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
        const int64_t n_pt = rows / BM, ns = n_pt * PPT;
        Meta m;
        m.src = (int32_t *)mp;
        mp += al(4 * (size_t)ns);
        m.key = (int32_t *)mp;
        mp += al(4 * (size_t)ns);
        m.flag = (uint8_t *)mp;
        mp += al((size_t)ns);
        m.inv3 = (float *)mp;
        mp += al(12 * (size_t)n_targets);
        m.t_base = (int64_t *)mp;
        mp += al(8 * (size_t)n_pt);
        m.t_run = (int32_t *)mp;
        mp += al(12 * (size_t)n_pt);
        m.isc = (float *)mp;
        mp += al(4 * (size_t)rows);
        m.iss = (float *)mp;
        return m;
    };
    const Meta mf = meta_at(base + meta_off, rJ, dm.n_atoms);
    const Meta mv = meta_at(base + vmeta_off, rV, vdm.n_atoms);
    float *m_isc = mf.isc, *m_iss = mf.iss;
    // the force pass's operands: the FP16 precision packs a scaled FP16 pair (kind 3), the
    // others their split as for the energy pass
    const bool f16 = mode == TcMode::FP16;
    auto pack_force = [&](const double *src, int64_t rows, int64_t row_off, bool jac, int64_t jlimit,
                          float *isc) -> cudaError_t {
        if (!f16) return pack(src, rows, row_off, jac, jlimit);
        return pack_force_f16(src, jac ? PACK_JAC : PACK_ROWS, rows, dm.d, d_pad, dm.d, jlimit, slice(0, row_off),
                              slice(1, row_off), isc, s);
    };
    if (ring && in.h_J && !in.h_J_direct) {
        // the FP64 slots are free once the work queued so far on this stream is done (an
        // earlier call may still read them); the first two chunks' copies then overlap the
        // energy pass
        for (int sl = 0; sl < 2; ++sl)
            if ((e = cudaEventRecord(in.ring_ev[2 + sl], s)) != cudaSuccess) return e;
    }
    if (prof) prof->begin(GAP_PROF_PACK);
    // the energy pass multiplies centred descriptors: the sums of the tensor cores' FP32
    // accumulation then stay small, and their rounding (about 1e-7 of g = x.x_s otherwise,
    // all of one sign) no longer reaches the powers g^zeta and g^(zeta-1)
    k_row_means<<<(unsigned)ceil_div(dm.n_atoms * 32, 256), 256, 0, s>>>(in.X, dm.n_atoms, dm.d, mu64, mxh, mxl);
    k_row_means<<<(unsigned)ceil_div(dm.M * 32, 256), 256, 0, s>>>(in.Xs, dm.M, dm.d, mu64 + dm.n_atoms, msh, msl);
    if ((e = pack(in.X, dm.n_atoms, 0, false, 0, mu64)) != cudaSuccess) return e;
    if ((e = pack(in.Xs, dm.M, dm.n_atoms, false, 0, mu64 + dm.n_atoms)) != cudaSuccess) return e;
    if (rJ > 0 && (e = pack_force(in.Xs, dm.M, dm.n_atoms + dm.M + rJs, false, 0, m_iss)) != cudaSuccess) return e;
    const bool chunked = rJ > 0 && in.n_jchunks > 0 && !ring;
    if (rJ > 0 && !chunked && !ring &&
        (e = pack_force(in.J, rJ, dm.n_atoms + dm.M, true, dm.n_pairs, m_isc)) != cudaSuccess)
        return e;
    if (prof) prof->end();
    const int64_t vrow0 = dm.n_atoms + dm.M + rJs + dm.M;  // first virial Jacobian row of the slices

    CUtensorMap tX[3], tSc[3], tS[3], tJ[3], tV[3];
    for (int i = 0; i < 3; ++i) {
        const int si = i < S ? i : 0;  // unused third map for TF32 mirrors slice 0
        if (!make_map(&tX[i], slice(si, 0), dm.n_atoms, d_pad, kind)) return cudaErrorInvalidValue;
        if (!make_map(&tSc[i], slice(si, dm.n_atoms), dm.M, d_pad, kind)) return cudaErrorInvalidValue;
        if (rJ > 0 && !make_map(&tS[i], slice(si, dm.n_atoms + dm.M + rJs), dm.M, d_pad, kind))
            return cudaErrorInvalidValue;
        if (rJ > 0 && !make_map(&tJ[i], slice(si, dm.n_atoms + dm.M), rJs, d_pad, kind)) return cudaErrorInvalidValue;
        if (rV > 0 && !make_map(&tV[i], slice(si, vrow0), rV, d_pad, kind)) return cudaErrorInvalidValue;
    }
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);

    Params P{};
    P.M = dm.M;
    P.ld = dm.ld;
    P.n_cfg = dm.n_cfg;
    P.n_pairs = dm.n_pairs;
    P.w_vec4 = (dm.M % 4 == 0) ? 1 : 0;
    P.n_kb = (int)(d_pad * esz / 128);
    P.n_ct = (int)ceil_div(dm.M, BN);
    P.zeta = dm.zeta;
    P.d2 = (float)(dm.delta * dm.delta);
    P.d2l = (float)(dm.delta * dm.delta - (double)P.d2);
    P.zf = (float)dm.zeta;
    P.E64 = in.E64;
    P.walk = std::max(1, in.force_walk);
    P.cfg_ptr = in.cfg_ptr;
    P.atom_cfg = in.atom_cfg;
    P.pair_ptr = in.pair_ptr;
    P.pair_src = in.pair_src;
    P.pair_tgt = in.pair_tgt;
    P.sigma = in.sigma;
    P.atom_sp = in.atom_sp;
    P.sparse_sp = in.sparse_sp;
    P.A_lo = A;
    P.A_acc = Aacc;
    P.W = Wf;
    P.status = in.status;
    // energy pass (also writes the per-atom force weights W), on the centred operands
    P.R = dm.n_atoms;
    P.n_tiles = ceil_div(P.R, BM) * P.n_ct;
    P.mux_h = mxh;
    P.mux_l = mxl;
    P.mus_h = msh;
    P.mus_l = msl;
    P.dd = (float)dm.d;
    if (prof) prof->begin(GAP_PROF_GEMM_ENERGY);
    // transposed tiles: A = sparse points, B = atoms (tile index = atom tile x sparse tile)
    e = kind == 0 ? launch_gemm<0, 3, MODE_ENERGY>(tSc, tX, P, n_sm, s)
                  : launch_gemm<1, 2, MODE_ENERGY>(tSc, tX, P, n_sm, s);
    if (prof) prof->end();
    P.mux_h = P.mux_l = P.mus_h = P.mus_l = nullptr;
    if (e != cudaSuccess || rJ == 0) return e;
    // force pass (and the virial pass, the force rows of pseudo-targets): per-row /
    // per-target / per-tile metadata, then the GEMM.  fd: the rows' Dims (fd.n_cfg = the
    // first output row, fd.n_atoms = the targets), rows: Jacobian rows padded to tiles.
    auto set_meta = [&](const Dims &fd, int64_t rows, const int64_t *src, const int64_t *tgt, const int64_t *ptr,
                        const Meta &m) -> cudaError_t {
        const int64_t n_pt = rows / BM, ns = n_pt * PPT;
        k_force_meta_pairs<<<(unsigned)ceil_div(ns, 256), 256, 0, s>>>(fd.n_pairs, ns, src, tgt, ptr, m.src, m.key,
                                                                      m.flag);
        k_force_meta_inv<<<(unsigned)ceil_div(3 * fd.n_atoms, 256), 256, 0, s>>>(fd.n_atoms, fd.n_cfg, in.sigma, m.inv3);
        k_force_meta_tiles<<<(unsigned)ceil_div(n_pt, 256), 256, 0, s>>>(fd.n_pairs, n_pt, fd.n_cfg, tgt, ptr, m.t_base,
                                                                         m.t_run);
        P.n_cfg = fd.n_cfg;
        P.n_pairs = fd.n_pairs;
        P.m_src = m.src;
        P.m_slot = m.key;
        P.m_flag = m.flag;
        P.m_inv3 = m.inv3;
        P.t_base = m.t_base;
        P.t_run = m.t_run;
        P.m_isc = m.isc;
        P.m_iss = m_iss;  // the sparse points' scales: one X_s copy for both passes
        P.R = rows;
        return cudaGetLastError();
    };
    if ((e = set_meta(dm, rJ, in.pair_src, in.pair_tgt, in.pair_ptr, mf)) != cudaSuccess) return e;
    // transposed tiles: A = sparse points, B = Jacobian rows (tile index = pair tile x sparse tile)
    // The contraction over d runs in K-chunks of at most kKbChunk k-blocks (32 MMA steps),
    // each launch adding its sums to A and A_acc.  The tensor cores' FP32 accumulation
    // truncates at every step; over a long contraction the running sums mostly carry the
    // sign of the result, so the truncations add up to a bias of the force rows (measured:
    // -2.2e-6 of their scale at 128 steps, d = 1024 in TF32; -2e-7 at 32 steps).  BF16 at
    // d <= 512 stays one launch.
    constexpr int kKbChunk = 8;
    const int n_kc = (int)ceil_div(P.n_kb, kKbChunk);
    // the force epilogue's output maps: A_lo column-major [ld x (M + 1)] and A_acc's 32-row
    // blocks as 32 rows x (ld / 32 x (M + 1)) columns, boxes of FSW rows x 32 sparse points
    CUtensorMap tLo, tAcc;
    {
        auto fn = encode_fn();
        cuuint32_t box[2] = {(cuuint32_t)FSW, 32u}, estr[2] = {1u, 1u};
        cuuint64_t dlo[2] = {(cuuint64_t)dm.ld, (cuuint64_t)(dm.M + 1)}, slo[1] = {(cuuint64_t)dm.ld * 4};
        cuuint64_t dac[2] = {(cuuint64_t)ACC_RB, (cuuint64_t)(dm.ld / ACC_RB * (dm.M + 1))}, sac[1] = {ACC_RB * 4};
        if (!fn ||
            fn(&tLo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, A, dlo, slo, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
                CUDA_SUCCESS ||
            fn(&tAcc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Aacc, dac, sac, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
                CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    auto force = [&](int64_t r0, int64_t r1, const CUtensorMap *tB) -> cudaError_t {
        P.t_begin = r0 / BM * P.n_ct;
        P.n_tiles = r1 / BM * P.n_ct;
        if (prof) prof->begin(GAP_PROF_GEMM_FORCE);
        cudaError_t e2 = cudaSuccess;
        for (int kc = 0; kc < n_kc && e2 == cudaSuccess; ++kc) {
            P.kb_lo = kc * kKbChunk;
            P.kb_hi = std::min(P.n_kb, (kc + 1) * kKbChunk);
            if (kc == 0)
                e2 = f16 ? launch_gemm<3, 3, MODE_FORCE>(tS, tB, P, n_sm, s, &tLo, &tAcc)
                         : (kind == 0 ? launch_gemm<0, 3, MODE_FORCE>(tS, tB, P, n_sm, s, &tLo, &tAcc)
                                      : launch_gemm<1, 2, MODE_FORCE>(tS, tB, P, n_sm, s, &tLo, &tAcc));
            else
                e2 = f16 ? launch_gemm<3, 3, MODE_FORCE, 1>(tS, tB, P, n_sm, s, &tLo, &tAcc)
                         : (kind == 0 ? launch_gemm<0, 3, MODE_FORCE, 1>(tS, tB, P, n_sm, s, &tLo, &tAcc)
                                      : launch_gemm<1, 2, MODE_FORCE, 1>(tS, tB, P, n_sm, s, &tLo, &tAcc));
        }
        P.kb_lo = P.kb_hi = 0;
        if (prof) prof->end();
        return e2;
    };
    // the virial rows after the force rows: their strain Jacobians (k_virial.cu) packed
    // like J, their pseudo-pairs' metadata, the same GEMM
    auto virials = [&]() -> cudaError_t {
        if (!vir) return cudaSuccess;
        if (prof) prof->begin(GAP_PROF_PACK);
        cudaError_t e2 = launch_virial_pseudo_pairs(dm, in.cfg_ptr, in.atom_cfg, in.pair_ptr, in.pair_src, in.J,
                                                    in.pair_u, in.vp_ptr, in.vp_src, in.vp_tgt, in.vG, s);
        if (e2 == cudaSuccess) e2 = pack_force(in.vG, rV, vrow0, true, vdm.n_pairs, mv.isc);
        if (prof) prof->end();
        if (e2 != cudaSuccess) return e2;
        if ((e2 = set_meta(vdm, rV, in.vp_src, in.vp_tgt, in.vp_ptr, mv)) != cudaSuccess) return e2;
        return force(0, rV, tV);
    };
    if (ring) {
        // chunk ch: pair tiles [r0, r1) of the packed rows, pairs [q0, q1).  A host J
        // goes through FP64 slot ch % 2 on the copy stream (the copy of the next chunk
        // overlaps this one's packing and GEMM); the packed slot is reused in stream order.
        const int64_t slot_pairs = ring_slot_pairs(in.ring_rows);
        const size_t pair_bytes = sizeof(double) * 3 * (size_t)dm.d;
        for (int64_t r0 = 0, ch = 0; r0 < rJ; r0 += in.ring_rows, ++ch) {
            const int64_t r1 = std::min(rJ, r0 + in.ring_rows);
            const int64_t q0 = r0 / BM * PPT, q1 = std::min(dm.n_pairs, r1 / BM * PPT);
            const double *Jc = in.J ? in.J + q0 * 3 * dm.d : (in.h_J_direct ? in.h_J + q0 * 3 * dm.d : nullptr);
            const int sl = (int)(ch % 2);
            if (in.h_J && !in.h_J_direct) {
                double *dst = in.ring_buf + (size_t)sl * (size_t)slot_pairs * 3 * (size_t)dm.d;
                if ((e = cudaStreamWaitEvent(in.ring_stream, in.ring_ev[2 + sl], 0)) != cudaSuccess ||
                    (q1 > q0 && (e = cudaMemcpyAsync(dst, in.h_J + q0 * 3 * dm.d, pair_bytes * (size_t)(q1 - q0),
                                                     cudaMemcpyHostToDevice, in.ring_stream)) != cudaSuccess) ||
                    (e = cudaEventRecord(in.ring_ev[sl], in.ring_stream)) != cudaSuccess)
                    return e;
                // the time this stream waits for the chunk to land counts as copy-in
                if (prof) prof->begin(GAP_PROF_COPY_IN);
                e = cudaStreamWaitEvent(s, in.ring_ev[sl], 0);
                if (prof) prof->end();
                if (e != cudaSuccess) return e;
                Jc = dst;
            }
            if (prof) prof->begin(GAP_PROF_PACK);
            e = pack_force(Jc, r1 - r0, dm.n_atoms + dm.M, true, std::max<int64_t>(0, dm.n_pairs - q0), m_isc + q0);
            if (prof) prof->end();
            if (e == cudaSuccess && in.h_J && !in.h_J_direct) e = cudaEventRecord(in.ring_ev[2 + sl], s);
            P.b_row0 = (int)r0;
            if (e != cudaSuccess || (e = force(r0, r1, tJ)) != cudaSuccess) return e;
        }
        P.b_row0 = 0;
        return cudaSuccess;
    }
    if (!chunked) {
        if ((e = force(0, rJ, tJ)) != cudaSuccess) return e;
        return virials();
    }
    // J arrives in chunks: each is packed and its pair tiles multiplied once it has landed,
    // while the next chunks are still being copied
    for (int ch = 0; ch < in.n_jchunks; ++ch) {
        const int64_t r0 = in.j_rows[ch], r1 = in.j_rows[ch + 1];
        if (r1 <= r0) continue;
        if ((e = cudaStreamWaitEvent(s, in.j_ev[ch], 0)) != cudaSuccess) return e;
        if (prof) prof->begin(GAP_PROF_PACK);
        const int64_t q0 = r0 / BM * PPT;  // first pair of the chunk
        e = pack_force(in.J + q0 * 3 * dm.d, r1 - r0, dm.n_atoms + dm.M + r0, true,
                       std::max<int64_t>(0, dm.n_pairs - q0), m_isc + q0);
        if (prof) prof->end();
        if (e != cudaSuccess || (e = force(r0, r1, tJ)) != cudaSuccess) return e;
    }
    return virials();
}


size_t tc_predict_workspace_bytes(const Dims &dm) {
    const int64_t d_pad = round_up(dm.d, 64), M_pad = round_up(dm.M, 64);
    size_t b = (size_t)(dm.n_atoms + dm.M) * d_pad * 8;                 // operand slices, first GEMM
    if (dm.forces) b = std::max(b, (size_t)(dm.n_atoms + dm.d) * M_pad * 8);  // second GEMM
    return b + 1024;
}

cudaError_t tc_predict(const Dims &dm, const TcInputs &in, TcMode mode, DevBuf &ops, DevBuf &work, const double *c,
                       double *E, double *F, cudaStream_t s, Prof *prof, double *V) {
    const int kind = mode == TcMode::TF32 ? 0 : 1;
    const int S = kind == 0 ? 2 : 3;
    const int esz = kind == 0 ? 4 : 2;
    const int64_t d_pad = round_up(dm.d, 64), M_pad = round_up(dm.M, 64);
    const bool forces = F != nullptr && dm.forces && dm.n_pairs > 0;
    const int64_t n_ct1 = ceil_div(dm.M, BN);
    // work: W [n_atoms x M] f32 | grad [n_atoms x d] f32 | eps_part [n_ct1 x n_atoms] f64 | eps [n_atoms] f64
    //       | c as FP32 pairs [2 x M]
    const size_t wbytes = forces ? (size_t)dm.n_atoms * dm.M * 4 : 256;
    const size_t gbytes = forces ? (size_t)dm.n_atoms * dm.d * 4 : 256;
    const size_t pbytes = (size_t)n_ct1 * dm.n_atoms * 8, ebytes = (size_t)dm.n_atoms * 8;
    const size_t cbytes = (size_t)dm.M * 8;
    const int64_t nm = dm.n_atoms + dm.M;
    const size_t mbytes = (size_t)nm * 16;  // descriptor means: FP64, then FP32 pairs
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    cudaError_t e = work.ensure(al(wbytes) + al(gbytes) + al(pbytes) + al(ebytes) + al(cbytes) + al(mbytes));
    if (e != cudaSuccess) return e;
    unsigned char *wb = work.as<unsigned char>();
    float *W = (float *)wb;
    float *grad = (float *)(wb + al(wbytes));
    double *eps_part = (double *)(wb + al(wbytes) + al(gbytes));
    double *eps = (double *)(wb + al(wbytes) + al(gbytes) + al(pbytes));
    float *c_h = (float *)(wb + al(wbytes) + al(gbytes) + al(pbytes) + al(ebytes)), *c_l = c_h + dm.M;
    double *mu64 = (double *)(wb + al(wbytes) + al(gbytes) + al(pbytes) + al(ebytes) + al(cbytes));
    float *mxh = (float *)(mu64 + nm), *mxl = mxh + nm, *msh = mxh + dm.n_atoms, *msl = mxl + dm.n_atoms;
    k_split_c<<<(unsigned)ceil_div(dm.M, 256), 256, 0, s>>>(c, dm.M, c_h, c_l);
    if ((e = ops.ensure(tc_predict_workspace_bytes(dm))) != cudaSuccess) return e;
    unsigned char *base = ops.as<unsigned char>();
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);

    // first GEMM: u = x_a . x_s over atoms x sparse points
    {
        const size_t se = (size_t)(dm.n_atoms + dm.M) * d_pad;
        auto sl = [&](int i, int64_t row_off) { return base + ((size_t)i * se + (size_t)row_off * d_pad) * esz; };
        // centred operands, as in the energy pass (the epilogue adds d mu_a mu_s back)
        k_row_means<<<(unsigned)ceil_div(dm.n_atoms * 32, 256), 256, 0, s>>>(in.X, dm.n_atoms, dm.d, mu64, mxh, mxl);
        k_row_means<<<(unsigned)ceil_div(dm.M * 32, 256), 256, 0, s>>>(in.Xs, dm.M, dm.d, mu64 + dm.n_atoms, msh, msl);
        if ((e = pack_slices(kind, in.X, PACK_CENTER, dm.n_atoms, dm.d, d_pad, dm.d, 0, sl(0, 0), sl(1, 0), sl(2, 0), s,
                             mu64)) != cudaSuccess)
            return e;
        if ((e = pack_slices(kind, in.Xs, PACK_CENTER, dm.M, dm.d, d_pad, dm.d, 0, sl(0, dm.n_atoms), sl(1, dm.n_atoms),
                             sl(2, dm.n_atoms), s, mu64 + dm.n_atoms)) != cudaSuccess)
            return e;
        CUtensorMap tA[3], tB[3];
        for (int i = 0; i < 3; ++i) {
            const int si = i < S ? i : 0;
            if (!make_map(&tA[i], sl(si, 0), dm.n_atoms, d_pad, kind) ||
                !make_map(&tB[i], sl(si, dm.n_atoms), dm.M, d_pad, kind))
                return cudaErrorInvalidValue;
        }
        Params P{};
        P.R = dm.n_atoms;
        P.M = dm.M;
        P.n_kb = (int)(d_pad * esz / 128);
        P.n_ct = (int)n_ct1;
        P.n_tiles = ceil_div(P.R, BM) * P.n_ct;
        P.zeta = dm.zeta;
        P.d2 = (float)(dm.delta * dm.delta);
        P.zf = (float)dm.zeta;
        P.atom_sp = in.atom_sp;
        P.sparse_sp = in.sparse_sp;
        P.W = W;
        P.w_vec4 = (dm.M % 4 == 0) ? 1 : 0;
        P.cvec_h = c_h;
        P.cvec_l = c_l;
        P.eps_part = eps_part;
        P.mux_h = mxh;
        P.mux_l = mxl;
        P.mus_h = msh;
        P.mus_l = msl;
        P.dd = (float)dm.d;
        P.status = in.status;
        if (!forces) P.W = nullptr;  // energies only: the gradient weights are not needed
        e = kind == 0 ? launch_gemm<0, 3, MODE_PREDICT>(tA, tB, P, n_sm, s)
                      : launch_gemm<1, 2, MODE_PREDICT>(tA, tB, P, n_sm, s);
        if (e != cudaSuccess) return e;
    }
    k_sum_eps<<<(unsigned)ceil_div(dm.n_atoms, 256), 256, 0, s>>>(eps_part, n_ct1, dm.n_atoms, eps);
    k_energy_from_eps<<<(unsigned)ceil_div(dm.n_cfg, 256), 256, 0, s>>>(dm.n_cfg, in.cfg_ptr, eps, E);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!forces) {
        if (F) return cudaMemsetAsync(F, 0, sizeof(double) * 3 * dm.n_atoms, s);
        return cudaSuccess;
    }
    // second GEMM: grad = W X_s  (rows: atoms, columns: descriptor entries, K: sparse points)
    {
        const size_t se = (size_t)(dm.n_atoms + dm.d) * M_pad;
        auto sl = [&](int i, int64_t row_off) { return base + ((size_t)i * se + (size_t)row_off * M_pad) * esz; };
        if ((e = pack_slices(kind, W, PACK_F32, dm.n_atoms, dm.M, M_pad, dm.M, 0, sl(0, 0), sl(1, 0), sl(2, 0), s)) != cudaSuccess)
            return e;
        if ((e = pack_slices(kind, in.Xs, PACK_TRANS, dm.d, dm.M, M_pad, dm.d, 0, sl(0, dm.n_atoms), sl(1, dm.n_atoms),
                             sl(2, dm.n_atoms), s)) != cudaSuccess)
            return e;
        CUtensorMap tA[3], tB[3];
        for (int i = 0; i < 3; ++i) {
            const int si = i < S ? i : 0;
            if (!make_map(&tA[i], sl(si, 0), dm.n_atoms, M_pad, kind) ||
                !make_map(&tB[i], sl(si, dm.n_atoms), dm.d, M_pad, kind))
                return cudaErrorInvalidValue;
        }
        Params P{};
        P.R = dm.n_atoms;
        P.M = dm.d;  // output columns
        P.n_kb = (int)(M_pad * esz / 128);
        P.n_ct = (int)ceil_div(dm.d, BN);
        P.n_tiles = ceil_div(P.R, BM) * P.n_ct;
        P.W = grad;
        P.w_vec4 = (dm.d % 4 == 0) ? 1 : 0;
        P.status = in.status;
        // The contraction runs over all M sparse points; as in the force pass, K-chunks of at
        // most 8 k-blocks (32 MMA steps) keep the truncating accumulation from building a bias
        // (about 5e-6 of the forces at M = 4000 in one accumulator); later chunks add.
        constexpr int kKbChunk = 8;
        for (int kb = 0; kb < P.n_kb; kb += kKbChunk) {
            P.kb_lo = kb;
            P.kb_hi = std::min(P.n_kb, kb + kKbChunk);
            if (kb == 0)
                e = kind == 0 ? launch_gemm<0, 3, MODE_STORE>(tA, tB, P, n_sm, s)
                              : launch_gemm<1, 2, MODE_STORE>(tA, tB, P, n_sm, s);
            else
                e = kind == 0 ? launch_gemm<0, 3, MODE_STORE, 1>(tA, tB, P, n_sm, s)
                              : launch_gemm<1, 2, MODE_STORE, 1>(tA, tB, P, n_sm, s);
            if (e != cudaSuccess) return e;
        }
    }
    if (in.J || in.h_J_direct) {
        // J on the device, or a page-locked host J read in place
        k_force_from_grad<<<(unsigned)ceil_div(dm.n_atoms * 32, 256), 256, 0, s>>>(
            0, dm.n_atoms, dm.d, in.pair_ptr, in.pair_src, in.J ? in.J : in.h_J, 0, grad, F);
    } else {
        // a host J through the J ring's two FP64 slots, by runs of whole atoms whose pairs
        // fill at most one slot (the copy of the next run overlaps this one's kernel)
        if (!in.h_J || !in.h_pair_ptr || !in.ring_buf || !in.ring_stream || !in.ring_ev || in.ring_rows <= 0)
            return cudaErrorInvalidValue;
        const int64_t slot_pairs = ring_slot_pairs(in.ring_rows);
        const size_t pair_bytes = sizeof(double) * 3 * (size_t)dm.d;
        const int64_t *pp = in.h_pair_ptr;
        for (int sl = 0; sl < 2; ++sl)
            if ((e = cudaEventRecord(in.ring_ev[2 + sl], s)) != cudaSuccess) return e;
        int64_t ch = 0;
        for (int64_t a0 = 0; a0 < dm.n_atoms; ++ch) {
            // the last atom a1 with pp[a1] - pp[a0] <= slot_pairs
            const int64_t a1 = (int64_t)(std::upper_bound(pp + a0, pp + dm.n_atoms + 1, pp[a0] + slot_pairs) - pp) - 1;
            if (a1 <= a0) return cudaErrorInvalidValue;  // an atom with more pairs than a slot
            const int sl = (int)(ch % 2);
            double *dst = in.ring_buf + (size_t)sl * (size_t)slot_pairs * 3 * (size_t)dm.d;
            const int64_t q0 = pp[a0], q1 = pp[a1];
            if ((e = cudaStreamWaitEvent(in.ring_stream, in.ring_ev[2 + sl], 0)) != cudaSuccess ||
                (q1 > q0 && (e = cudaMemcpyAsync(dst, in.h_J + q0 * 3 * dm.d, pair_bytes * (size_t)(q1 - q0),
                                                 cudaMemcpyHostToDevice, in.ring_stream)) != cudaSuccess) ||
                (e = cudaEventRecord(in.ring_ev[sl], in.ring_stream)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, in.ring_ev[sl], 0)) != cudaSuccess)
                return e;
            k_force_from_grad<<<(unsigned)ceil_div((a1 - a0) * 32, 256), 256, 0, s>>>(a0, a1, dm.d, in.pair_ptr,
                                                                                     in.pair_src, dst, q0, grad, F);
            if ((e = cudaEventRecord(in.ring_ev[2 + sl], s)) != cudaSuccess) return e;
            a0 = a1;
        }
    }
    // virials: the same contraction over the pseudo-pairs of each configuration's two
    // pseudo-targets, with the strain Jacobians (k_virial.cu)
    if (V && in.vG) {
        const int64_t nt = 2 * dm.n_cfg;
        k_force_from_grad<<<(unsigned)ceil_div(nt * 32, 256), 256, 0, s>>>(0, nt, dm.d, in.vp_ptr, in.vp_src, in.vG, 0,
                                                                          grad, V);
    }
    (void)prof;
    return cudaGetLastError();
}


cudaError_t tc_qr_update(float *A, int64_t ld, int64_t row_off, int64_t R, int64_t col_off, int64_t nt,
                         const float *v_hi, const float *v_lo, const float *w_hi, const float *w_lo, int kpad,
                         int passes, int *status, cudaStream_t s, int v_ld) {
    if (R <= 0 || nt <= 0) return cudaSuccess;
    CUtensorMap tA[3], tB[3];
    if (!make_map(&tA[0], v_hi, R, kpad, 0, v_ld) || !make_map(&tB[0], w_hi, nt, kpad, 0)) return cudaErrorInvalidValue;
    if (passes == 1) {
        tA[1] = tA[0];
        tB[1] = tB[0];
    } else if (!make_map(&tA[1], v_lo, R, kpad, 0) || !make_map(&tB[1], w_lo, nt, kpad, 0)) {
        return cudaErrorInvalidValue;
    }
    tA[2] = tA[0];
    tB[2] = tB[0];
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    Params P{};
    P.R = R;
    P.M = nt;
    P.ld = ld;
    P.row_off = row_off;
    P.col_off = col_off;
    P.n_kb = kpad * 4 / 128;
    P.n_ct = (int)ceil_div(nt, BN);
    P.n_tiles = ceil_div(R, BM) * P.n_ct;
    P.A_lo = A;
    P.status = status;
    // C map over the whole column-major matrix: dims {ld rows, row_off + R rows used ... }
    CUtensorMap tC;
    {
        auto fn = encode_fn();
        if (!fn) return cudaErrorInvalidValue;
        cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)(col_off + nt)};
        cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
        cuuint32_t box[2] = {128u, (cuuint32_t)EPI};
        cuuint32_t estr[2] = {1u, 1u};
        if (fn(&tC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)A, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    return passes == 1 ? launch_gemm<2, 6, MODE_QR_UPD>(tA, tB, P, n_sm, s, &tC)
                       : launch_gemm<0, 3, MODE_QR_UPD>(tA, tB, P, n_sm, s, &tC);
}


// ------------------------------------------------------------------------
// Y = V^T C for the QR trailing update (outer panel of up to 128 reflectors):
// Y[a, c] = sum_r V[r, a] C[r, c] over the rows of one split of [row0, row0 + R),
// written as Yp[split][a][c] (the splits are summed afterwards in a fixed order).
// V arrives by TMA as split-TF32 slices of its column-major copy [128 x R]
// (K-major A operand).  C is read by the four loader warps straight from the
// column-major FP32 matrix (one thread per column, 32 consecutive rows = one
// 128-byte line per k-block), split into TF32 hi/lo in registers and written
// into the 128B-swizzled K-major layout of the B operand; a proxy fence and an
// mbarrier hand the tiles to the MMA thread.  D += Vhi.Chi + Vhi.Clo + Vlo.Chi.
namespace {

struct QrYParams {
    const float *A;      // column-major FP32 source of C
    int64_t ld, row0, R; // rows [row0, row0 + R) of C
    int64_t c0, nt;      // columns [c0, c0 + nt)
    int n_ct, n_split, kb_per_split, n_kb_total;
    int64_t n_tiles;
    float *Yp;           // [n_split][128][nt]
    int *status;
};

template <int STAGES>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc_qr_y(const __grid_constant__ CUtensorMap tVh,
                                                         const __grid_constant__ CUtensorMap tVl, QrYParams P) {
    constexpr uint32_t TILE = 128 * 128;         // 128 rows x 128 bytes
    constexpr uint32_t STAGE_BYTES = 4 * TILE;   // V hi, V lo, C hi, C lo
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *fullv = bars, *fullc = bars + STAGES, *empty = bars + 2 * STAGES;
    uint64_t *tfull = bars + 3 * STAGES, *tempty = bars + 3 * STAGES + 2;
    uint32_t *tmem_slot = (uint32_t *)(bars + 3 * STAGES + 4);
    int *sflag = (int *)(tmem_slot + 2);  // [4] shared wait outcomes
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&fullv[s], 1);
            mbar_init(&fullc[s], 128);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(256u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ----------------------------------------------- TMA producer (V) --
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < P.n_tiles && ok; t += gridDim.x) {
                const int split = (int)(t / P.n_ct);
                const int kb0 = split * P.kb_per_split, kb1 = min(P.n_kb_total, kb0 + P.kb_per_split);
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, P.status)) { ok = false; break; }
                    unsigned char *st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&fullv[s], 2 * TILE);
                    tma_load_2d(st, &tVh, &fullv[s], kb * 32, 0);
                    tma_load_2d(st + TILE, &tVl, &fullv[s], kb * 32, 0);
                }
            }
            if (it > 0) {
                const uint32_t last = it - 1;
                for (uint32_t q = (last >= (uint32_t)STAGES ? last - STAGES + 1 : 0); q <= last; ++q)
                    mbar_wait(&fullv[q % STAGES], (q / STAGES) & 1, P.status);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer --
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);  // TF32, M=128, N=128
            uint32_t it = 0, tc = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < P.n_tiles && ok; t += gridDim.x, ++tc) {
                const int split = (int)(t / P.n_ct);
                const int kb0 = split * P.kb_per_split, kb1 = min(P.n_kb_total, kb0 + P.kb_per_split);
                const uint32_t ab = tc & 1, aph = (tc >> 1) & 1;
                if (!mbar_wait(&tempty[ab], aph ^ 1, P.status)) { ok = false; break; }
                fence_after();
                const uint32_t d = tmem + ab * 128;
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                    if (!mbar_wait(&fullv[s], ph, P.status) || !mbar_wait(&fullc[s], ph, P.status)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint64_t vh = smem_desc(base + k * 32), vl = smem_desc(base + TILE + k * 32);
                        const uint64_t ch = smem_desc(base + 2 * TILE + k * 32), cl = smem_desc(base + 3 * TILE + k * 32);
                        const uint32_t first = (kb == kb0 && k == 0) ? 0u : 1u;
                        mma<0>(d, vh, ch, idesc, first);
                        mma<0>(d, vh, cl, idesc, 1u);
                        mma<0>(d, vl, ch, idesc, 1u);
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&tfull[ab]);
            }
            if (tc > 0) mbar_wait(&tfull[(tc - 1) & 1], ((tc - 1) >> 1) & 1, P.status);
        }
    } else {
        // --------------------------------------- C loaders, then epilogue --
        const int q = warp & 3;
        const int et = (warp - 2) * 32 + lane;  // 0..127: the column this thread loads
        const int lt = q * 32 + lane;           // TMEM lane (reflector) this thread reads
        uint32_t it = 0, tc = 0;
        for (int64_t t = blockIdx.x; t < P.n_tiles; t += gridDim.x, ++tc) {
            const int split = (int)(t / P.n_ct);
            const int64_t ct = t % P.n_ct;
            const int kb0 = split * P.kb_per_split, kb1 = min(P.n_kb_total, kb0 + P.kb_per_split);
            const int64_t col = ct * 128 + et;
            const bool cvalid = col < P.nt;
            const float *cp = P.A + (P.c0 + (cvalid ? col : 0)) * P.ld + P.row0;
            bool ok = true;
            // two-deep register pipeline: the loads of k-block kb+1 are in flight while
            // k-block kb is split and stored
            float4 cur[8], nxt[8];
            auto load_kb = [&](int kb, float4 *dst) {
                const int64_t r0 = (int64_t)kb * 32;
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) {
                    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (cvalid) {
                        if (r0 + c4 * 4 + 3 < P.R) {
                            x = *reinterpret_cast<const float4 *>(cp + r0 + c4 * 4);
                        } else {
                            float v[4];
                            for (int u = 0; u < 4; ++u) v[u] = (r0 + c4 * 4 + u < P.R) ? cp[r0 + c4 * 4 + u] : 0.f;
                            x = make_float4(v[0], v[1], v[2], v[3]);
                        }
                    }
                    dst[c4] = x;
                }
            };
            if (kb0 < kb1) load_kb(kb0, cur);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
                const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                if (kb + 1 < kb1) load_kb(kb + 1, nxt);
                // every loader thread waits (bounded) on the stage itself; a thread that
                // gives up leaves the k-loop and meets the others at the epilogue barrier
                if (!mbar_wait(&empty[s], ph ^ 1, P.status)) { ok = false; break; }
                unsigned char *hi = smem + s * STAGE_BYTES + 2 * TILE + et * 128;
                unsigned char *lo = hi + TILE;
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) {
                    const float4 x = cur[c4];
                    float4 h, l;
                    tf32_split_dev(x.x, h.x, l.x);
                    tf32_split_dev(x.y, h.y, l.y);
                    tf32_split_dev(x.z, h.z, l.z);
                    tf32_split_dev(x.w, h.w, l.w);
                    const int chunk = (c4 ^ (et & 7)) * 16;  // 128-byte swizzle
                    *reinterpret_cast<float4 *>(hi + chunk) = h;
                    *reinterpret_cast<float4 *>(lo + chunk) = l;
                }
                fence_proxy_async();
                mbar_arrive(&fullc[s]);
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) cur[c4] = nxt[c4];
            }
            (void)ok;
            // epilogue of this tile: TMEM lane = reflector, 128 columns
            const uint32_t ab = tc & 1, aph = (tc >> 1) & 1;
            int *fl = &sflag[2 + (tc & 1)];
            if (et == 0) *fl = mbar_wait(&tfull[ab], aph, P.status) ? 0 : 1;
            epi_sync();
            if (*fl != 0) break;
            fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + ab * 128;
            float *yrow = P.Yp + ((int64_t)split * 128 + lt) * P.nt + ct * 128;
            for (int ch = 0; ch < 128 / EPI; ++ch) {
                float v[EPI];
                tmem_ld16(tbase + ch * EPI, v);
                const int64_t cbase = ct * 128 + ch * EPI;
#pragma unroll
                for (int j = 0; j < EPI; ++j)
                    if (cbase + j < P.nt) yrow[ch * EPI + j] = v[j];
            }
            fence_before();
            mbar_arrive(&tempty[ab]);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u));
    }
}

// column-major-by-reflector copies of the panel reflectors: Vc[a][r] = V[K0 + r, a] for
// a < n_rows, split (Vh, Vl) for the A operand and unsplit (Vf) as a column-major C
// source for V^T V; with full == 0 only Vh is written.
// Grid (ceil(R_pad / 1024), n_rows): blockIdx.y = reflector a, four rows per thread.
__global__ void k_qr_pack_vcm(const float *A, int64_t ld, int64_t K0, int coff, int nbo, int64_t R, int64_t R_pad,
                              int n_rows, int full, float *Vh, float *Vl, float *Vf) {
    const int a = blockIdx.y;
    for (int u = 0; u < 4; ++u) {
    const int64_t r = (int64_t)blockIdx.x * 1024 + u * 256 + threadIdx.x;
    if (r >= R_pad) break;
    const int64_t e = (int64_t)a * R_pad + r, i = K0 + r, c = K0 + coff + a;
    float v = 0.f;
    if (a < nbo && r < R) v = i < c ? 0.f : (i == c ? 1.f : A[i + c * ld]);
    float h, l;
    tf32_split_dev(v, h, l);
    Vh[e] = h;
    if (full) {
        Vl[e] = l;
        Vf[e] = v;
    }
    }
}

}  // namespace

size_t tc_qr_y_workspace_bytes(int64_t R) { return sizeof(float) * 3 * 128 * (size_t)round_up(R, 32) + 512; }

const float *tc_qr_pack_v(const float *A, int64_t ld, int64_t K0, int nbo, int64_t R, void *vws, int n_rows, bool full,
                          cudaStream_t s, int coff) {
    const int64_t R_pad = round_up(R, 32);
    float *Vh = (float *)vws, *Vl = Vh + 128 * R_pad, *Vf = Vl + 128 * R_pad;
    k_qr_pack_vcm<<<dim3((unsigned)ceil_div(R_pad, 1024), (unsigned)n_rows), 256, 0, s>>>(
        A, ld, K0, coff, nbo, R, R_pad, n_rows, full ? 1 : 0, Vh, Vl, Vf);
    return Vf;
}

cudaError_t tc_qr_y(const float *C, int64_t ldc, int64_t crow0, int64_t R, int64_t c0, int64_t nt, int n_split,
                    void *vws, float *Yp, int *status, cudaStream_t s, int *n_split_used) {
    *n_split_used = 0;
    if (R <= 0 || nt <= 0) return cudaSuccess;
    const int64_t R_pad = round_up(R, 32);
    float *Vh = (float *)vws, *Vl = Vh + 128 * R_pad;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap tVh, tVl;
    if (!make_map(&tVh, Vh, 128, R_pad, 0) || !make_map(&tVl, Vl, 128, R_pad, 0)) return cudaErrorInvalidValue;
    QrYParams P{};
    P.A = C;
    P.ld = ldc;
    P.row0 = crow0;
    P.R = R;
    P.c0 = c0;
    P.nt = nt;
    P.n_ct = (int)ceil_div(nt, 128);
    P.n_kb_total = (int)(R_pad / 32);
    P.kb_per_split = (int)ceil_div(P.n_kb_total, n_split);
    P.n_split = (int)ceil_div(P.n_kb_total, P.kb_per_split);
    P.n_tiles = (int64_t)P.n_split * P.n_ct;
    *n_split_used = P.n_split;
    P.Yp = Yp;
    P.status = status;
    constexpr int STAGES = 3;
    const size_t smem = 1024 + (size_t)STAGES * 4 * 128 * 128 + (3 * STAGES + 4) * 8 + 64;
    static const cudaError_t y_attr =
        cudaFuncSetAttribute(k_tc_qr_y<STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (y_attr != cudaSuccess) return y_attr;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = (int)std::min<int64_t>(P.n_tiles, n_sm);
    k_tc_qr_y<STAGES><<<grid, NTHREADS, smem, s>>>(tVh, tVl, P);
    return cudaGetLastError();
}

cudaError_t tc_qr_y_tma(const float *C, int64_t ldc, int64_t crow0, int64_t R, int64_t c0, int64_t nt, int n_split,
                        void *vws, int v_rows, float *Yp, int *status, cudaStream_t s, int *n_split_used) {
    *n_split_used = 0;
    if (R <= 0 || nt <= 0) return cudaSuccess;
    if (crow0 % 4 != 0 || ldc % 4 != 0) return cudaErrorInvalidValue;  // 16-byte TMA origin and stride
    const int64_t R_pad = round_up(R, 32);
    const float *Vh = (const float *)vws;
    CUtensorMap tA[3], tB[3];
    // V rows past v_rows (reflectors beyond the panel's) read as zero
    if (!make_map(&tA[0], Vh, v_rows, R_pad, 0)) return cudaErrorInvalidValue;
    {
        // B operand: columns c0 .. c0 + nt of C, K = rows crow0 .. crow0 + R (contiguous
        // within a column: K-major); boxes of 32 rows (128 bytes) x 128 columns, rows
        // past R and columns past nt read as zero
        auto fn = encode_fn();
        if (!fn) return cudaErrorInvalidValue;
        cuuint64_t dims[2] = {(cuuint64_t)R, (cuuint64_t)nt};
        cuuint64_t strides[1] = {(cuuint64_t)(ldc * 4)};
        cuuint32_t box[2] = {32u, 128u};
        cuuint32_t estr[2] = {1u, 1u};
        if (fn(&tB[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)(C + crow0 + c0 * ldc), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    tA[1] = tA[2] = tA[0];
    tB[1] = tB[2] = tB[0];
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    Params P{};
    P.R = 128;
    P.M = nt;
    P.n_kb = (int)(R_pad / 32);
    P.kb_split = (int)ceil_div(P.n_kb, std::max(1, n_split));
    const int used = (int)ceil_div(P.n_kb, P.kb_split);  // every split has at least one k-block
    P.n_ct = (int)ceil_div(nt, BN);
    P.n_tiles = (int64_t)used * P.n_ct;
    P.W = Yp;
    P.w_vec4 = (nt % 4 == 0) ? 1 : 0;
    P.status = status;
    *n_split_used = used;
    return launch_gemm<2, 6, MODE_YSTORE>(tA, tB, P, n_sm, s);
}

cudaError_t tc_qr_y2_tma(const float *C, int64_t ldc, int64_t crow0, int64_t R, int64_t c0, int64_t nt, int n_split,
                         const float *v1, const float *v2, int v2_rows, float *Yp, int *status, cudaStream_t s,
                         int *n_split_used) {
    *n_split_used = 0;
    if (R <= 0 || nt <= 0) return cudaSuccess;
    if (crow0 % 4 != 0 || ldc % 4 != 0) return cudaErrorInvalidValue;  // 16-byte TMA origin and stride
    const int64_t R_pad = round_up(R, 32);
    CUtensorMap tA[3], tB[3];
    if (!make_map(&tA[0], v1, 128, R_pad, 0) || !make_map(&tA[1], v2, v2_rows, R_pad, 0)) return cudaErrorInvalidValue;
    {
        auto fn = encode_fn();
        if (!fn) return cudaErrorInvalidValue;
        cuuint64_t dims[2] = {(cuuint64_t)R, (cuuint64_t)nt};
        cuuint64_t strides[1] = {(cuuint64_t)(ldc * 4)};
        cuuint32_t box[2] = {32u, (cuuint32_t)bn_of<MODE_Y2>()};
        cuuint32_t estr[2] = {1u, 1u};
        if (fn(&tB[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)(C + crow0 + c0 * ldc), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    tA[2] = tA[0];
    tB[1] = tB[2] = tB[0];
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    Params P{};
    P.R = 256;
    P.M = nt;
    P.n_kb = (int)(R_pad / 32);
    P.kb_split = (int)ceil_div(P.n_kb, std::max(1, n_split));
    const int used = (int)ceil_div(P.n_kb, P.kb_split);
    P.n_ct = (int)ceil_div(nt, bn_of<MODE_Y2>());
    P.n_tiles = (int64_t)used * P.n_ct;
    P.W = Yp;
    P.w_vec4 = (nt % 4 == 0) ? 1 : 0;
    P.status = status;
    *n_split_used = used;
    return launch_gemm<2, 3, MODE_Y2>(tA, tB, P, n_sm, s);
}

}  // namespace gap
