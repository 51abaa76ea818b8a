/*
 * Seeded synthetic inputs for the sparse-GP (GAP) fit workloads.
 *
 * This file holds NO arithmetic of the fitting method (no kernel, no sums over
 * configurations, no linear algebra).  It draws the raw inputs a fit consumes:
 * configuration sizes, species labels, neighbour lists, descriptor vectors,
 * descriptor Jacobians, sparse-point indices, a hidden weight vector and noise.
 *
 * Every value is a pure function of (seed, array id, element index): a
 * counter-based generator built on the splitmix64 finaliser (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
 * Normal deviates use Marsaglia's polar method (Marsaglia and Bray, SIAM Rev.
 * 6, 1964) with a logarithm evaluated here from its atanh series using only
 * +, -, *, / and an exact binary exponent split, so the bits do not depend on
 * the platform's libm.  Build with -ffp-contract=off so that no FMA
 * contraction changes a rounding between compilers or architectures.
 */
#include <stdint.h>
#include <math.h>
#include <string.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ull

static inline uint64_t gg_mix(uint64_t z) {
    z += GG_GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* 64 random bits for element `idx`, attempt `k` of array `aid`. */
static inline uint64_t gg_bits(uint64_t seed, uint64_t aid, uint64_t idx, uint64_t k) {
    uint64_t s = gg_mix(seed ^ gg_mix(aid * 0xD1B54A32D192ED03ull));
    return gg_mix(s ^ gg_mix(idx * 0xA0761D6478BD642Full + k * 0xE7037ED1A0B428DBull));
}

/* Uniform in [0, 1) with 53 random bits. */
static inline double gg_unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* Uniform integer in [lo, hi] (inclusive). */
static inline int64_t gg_int(uint64_t r, int64_t lo, int64_t hi) {
    uint64_t span = (uint64_t)(hi - lo + 1);
    return lo + (int64_t)((double)(r >> 11) * (1.0 / 9007199254740992.0) * (double)span);
}

/* Natural log of x > 0 from x = m * 2^e (m in [sqrt(1/2), sqrt(2))) and
 * log m = 2 atanh(t), t = (m - 1)/(m + 1), |t| < 0.1716; 24 series terms
 * leave a truncation error far below one ulp. */
static double gg_log(double x) {
    int e;
    double m = frexp(x, &e); /* exact: x = m * 2^e, m in [0.5, 1) */
    if (m < 0.70710678118654752) { m *= 2.0; e -= 1; }
    double t = (m - 1.0) / (m + 1.0);
    double t2 = t * t, term = t, sum = 0.0;
    for (int n = 0; n < 24; ++n) {
        sum += term / (double)(2 * n + 1);
        term *= t2;
    }
    return 2.0 * sum + (double)e * 0.69314718055994530942;
}

/* Standard normal deviate for element idx of array aid (polar method). */
static double gg_normal(uint64_t seed, uint64_t aid, uint64_t idx) {
    for (uint64_t k = 0;; ++k) {
        double u = 2.0 * gg_unit(gg_bits(seed, aid, idx, 2 * k)) - 1.0;
        double v = 2.0 * gg_unit(gg_bits(seed, aid, idx, 2 * k + 1)) - 1.0;
        double s = u * u + v * v;
        if (s > 0.0 && s < 1.0) return u * sqrt(-2.0 * gg_log(s) / s);
    }
}

/* ---------------------------------------------------------------- API -- */

double gg_log_public(double x) { return gg_log(x); }

/* n draws of scale * N(0,1) from array `aid`, element ids offset..offset+n-1. */
void gg_normals(uint64_t seed, uint64_t aid, int64_t offset, int64_t n, double scale, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = scale * gg_normal(seed, aid, (uint64_t)(offset + i));
}

/* n uniform integers in [lo, hi] from array `aid`. */
void gg_ints(uint64_t seed, uint64_t aid, int64_t n, int64_t lo, int64_t hi, int64_t *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = gg_int(gg_bits(seed, aid, (uint64_t)i, 0), lo, hi);
}

/* n uniform doubles in [0, 1) from array `aid`. */
void gg_uniforms(uint64_t seed, uint64_t aid, int64_t n, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = gg_unit(gg_bits(seed, aid, (uint64_t)i, 0));
}

/* Descriptor rows [n x d]: N(0,1) entries (absolute value if absval != 0),
 * each row then scaled to unit Euclidean length.  Rows row0..row0+n-1 of the
 * array, so any subset of rows can be regenerated on its own. */
void gg_descriptors(uint64_t seed, uint64_t aid, int64_t row0, int64_t n, int64_t d, int absval, double *X) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
        double *x = X + r * d;
        double ss = 0.0;
        for (int64_t k = 0; k < d; ++k) {
            double z = gg_normal(seed, aid, (uint64_t)((row0 + r) * d + k));
            if (absval && z < 0.0) z = -z;
            x[k] = z;
            ss += z * z;
        }
        double inv = 1.0 / sqrt(ss);
        for (int64_t k = 0; k < d; ++k) x[k] *= inv;
    }
}

/* Descriptor rows at arbitrary row indices idx[0..n-1] of the same array
 * (identical to the rows gg_descriptors draws at those positions). */
void gg_descriptor_rows(uint64_t seed, uint64_t aid, const int64_t *idx, int64_t n, int64_t d, int absval,
                        double *X) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) gg_descriptors(seed, aid, idx[r], 1, d, absval, X + r * d);
}

/* Pair sources: for target atom a (in configuration cfg_of[a]) draw
 * pair_ptr[a+1]-pair_ptr[a] source atoms uniformly, with replacement, from
 * the atoms of that configuration (the target itself included). */
void gg_pair_src(uint64_t seed, uint64_t aid, int64_t n_atoms, const int64_t *cfg_ptr, const int64_t *cfg_of,
                 const int64_t *pair_ptr, int64_t *pair_src) {
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n_atoms; ++a) {
        int64_t c = cfg_of[a], lo = cfg_ptr[c], hi = cfg_ptr[c + 1] - 1;
        for (int64_t p = pair_ptr[a]; p < pair_ptr[a + 1]; ++p)
            pair_src[p] = gg_int(gg_bits(seed, aid, (uint64_t)p, 0), lo, hi);
    }
}

/* m distinct indices drawn from cand[0..n_cand-1] by a partial Fisher-Yates
 * shuffle (cand is permuted in place; the first m entries are the draw). */
int gg_subset(uint64_t seed, uint64_t aid, int64_t n_cand, int64_t *cand, int64_t m) {
    if (m > n_cand || m < 0) return -1;
    for (int64_t i = 0; i < m; ++i) {
        int64_t j = gg_int(gg_bits(seed, aid, (uint64_t)i, 0), i, n_cand - 1);
        int64_t t = cand[i];
        cand[i] = cand[j];
        cand[j] = t;
    }
    return 0;
}
