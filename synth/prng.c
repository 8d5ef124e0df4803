/*
 * Counter-based pseudo-random draws for the synthetic workloads.
 *
 * This file holds no arithmetic of the filter: it only turns (seed, stream,
 * index) triples into uniform and normal variates.  Both the CUDA path and the
 * oracle receive the same host arrays produced here, so neither side ever draws
 * its own random numbers.
 *
 * Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used in counter mode: draw i of stream s
 * under seed k is mix64(key(k, s) + (i + 1) * 0x9E3779B97F4A7C15), where
 * key(k, s) = mix64(k ^ mix64(s + 0x632BE59BD9B4E019)).  A uniform variate keeps
 * the top 53 bits, u = (z >> 11 + 0.5) * 2^-53, which lies strictly inside
 * (0, 1).  A normal variate pairs draws 2i and 2i+1 through the Box-Muller
 * transform, sqrt(-2 ln u1) * cos(2 pi u2).
 *
 * Every draw depends on its index only, so any slice can be produced
 * independently and the output does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return mix64(seed ^ mix64(stream + 0x632BE59BD9B4E019ULL));
}

static inline uint64_t draw_u64(uint64_t key, uint64_t i) {
    return mix64(key + (i + 1) * GOLDEN);
}

static inline double u01(uint64_t z) {
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static inline double normal_at(uint64_t key, uint64_t i) {
    const double two_pi = 6.283185307179586476925286766559;
    double a = u01(draw_u64(key, 2 * i));
    double b = u01(draw_u64(key, 2 * i + 1));
    return sqrt(-2.0 * log(a)) * cos(two_pi * b);
}

/* Raw 64-bit draws [offset, offset + n) of (seed, stream). */
void synth_u64(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n, uint64_t* out) {
    uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = draw_u64(key, offset + (uint64_t)i);
}

/* Uniform variates on (lo, hi). */
void synth_uniform(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n,
                   double lo, double hi, double* out) {
    uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * u01(draw_u64(key, offset + (uint64_t)i));
}

/*
 * Normal variates laid out as a column-major rows x cols matrix with leading
 * dimension ld: entry (j, c) is mean + scale[j] * N_{c*rows + j} (scale may be
 * NULL for 1).  Padding rows j >= rows are left untouched.
 */
void synth_normal_matrix(uint64_t seed, uint64_t stream, int64_t rows, int64_t cols, int64_t ld,
                         double mean, double stddev, const double* row_scale, double* out) {
    uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < cols; ++c) {
        for (int64_t j = 0; j < rows; ++j) {
            double s = stddev * (row_scale ? row_scale[j] : 1.0);
            out[c * ld + j] = mean + s * normal_at(key, (uint64_t)(c * rows + j));
        }
    }
}

/* Same draws as synth_normal_matrix, rounded once to float. */
void synth_normal_matrix_f32(uint64_t seed, uint64_t stream, int64_t rows, int64_t cols, int64_t ld,
                             double mean, double stddev, const double* row_scale, float* out) {
    uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < cols; ++c) {
        for (int64_t j = 0; j < rows; ++j) {
            double s = stddev * (row_scale ? row_scale[j] : 1.0);
            out[c * ld + j] = (float)(mean + s * normal_at(key, (uint64_t)(c * rows + j)));
        }
    }
}
