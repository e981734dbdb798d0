// sim.cuh -- the similarity functions of Table 1 as exact integer tests, and
// the length window of Table 2, for the kernels and the host code.
//
// A threshold is the rational p/q.  Each function's test sim(x, y) >= p/q is
// cleared of its fraction (and, for Cosine, of the square root):
//   Jaccard  o/(|x|+|y|-o) >= p/q    <=>  o*(p+q) >= p*(|x|+|y|)
//   Cosine   o/sqrt(|x|*|y|) >= p/q  <=>  o^2*q^2 >= p^2*|x|*|y|
//   Dice     2o/(|x|+|y|) >= p/q     <=>  2*o*q   >= p*(|x|+|y|)
//   Overlap  o >= p/q                <=>  o*q     >= p
// The Bitmap Filter (Eq. 2) keeps a pair iff its overlap bound reaches
// need(x, y), the smallest overlap that passes the test; need depends on
// |x|+|y| alone for Jaccard, Dice and Overlap, and on |x|*|y| for Cosine.
#pragma once

#include <math.h>
#include <stdint.h>

#include "../../include/bmj.h"

namespace bmj {

// p/q is a valid threshold for the function: 0 < p <= q (Overlap: any p, q >= 1,
// since its threshold counts tokens); Cosine also needs p, q <= 65535 so that
// q^2 fits the 32-bit window coefficient.
__host__ __device__ inline bool sim_valid(int sim, uint32_t p, uint32_t q) {
    if (p == 0 || q == 0) return false;
    switch (sim) {
        case BMJ_JACCARD: case BMJ_DICE: return p <= q && q < 0x80000000u;
        case BMJ_COSINE: return p <= q && q <= 65535u;
        case BMJ_OVERLAP: return q < 0x80000000u;
        default: return false;
    }
}

// Sizes a <= b can reach the threshold (Table 2) iff wa*a >= wb*b + wc, i.e. iff
// the test passes with the overlap at its maximum a.
struct SimWindow {
    uint32_t wa, wb, wc;
};

__host__ __device__ inline SimWindow sim_window(int sim, uint32_t p, uint32_t q) {
    switch (sim) {
        case BMJ_COSINE: return SimWindow{q * q, p * p, 0u};     // a*q^2 >= b*p^2
        case BMJ_DICE: return SimWindow{2u * q - p, p, 0u};      // a*(2q-p) >= b*p
        case BMJ_OVERLAP: return SimWindow{q, 0u, p};            // a*q >= p
        default: return SimWindow{q, p, 0u};                     // a*q >= b*p
    }
}

__host__ __device__ inline bool in_window(uint64_t a, uint64_t b, SimWindow w) {
    return (uint64_t)w.wa * a >= (uint64_t)w.wb * b + w.wc;
}

// Smallest size a (paired with a set of size s >= a) inside the window.
__host__ __device__ inline uint64_t window_low(uint64_t s, SimWindow w) {
    return ((uint64_t)w.wb * s + w.wc + w.wa - 1) / w.wa;
}

// Largest size b (paired with a set of size s <= b) inside the window; ~0 when
// the window has no upper bound (Overlap), 0 when even b = s is outside it.
__host__ __device__ inline uint64_t window_high(uint64_t s, SimWindow w) {
    const uint64_t lhs = (uint64_t)w.wa * s;
    if (lhs < w.wc) return 0;
    if (w.wb == 0) return ~0ull;
    return (lhs - w.wc) / w.wb;
}

// Smallest overlap passing the Cosine test: ceil(p*sqrt(x*y)/q), from a
// floating-point estimate corrected in exact 128-bit arithmetic.
__host__ __device__ inline int64_t cosine_need(uint32_t p, uint32_t q, int64_t x, int64_t y) {
    const unsigned __int128 rhs = (unsigned __int128)((uint64_t)p * p) * (uint64_t)(x * y);
    const uint64_t qq = (uint64_t)q * q;
    uint64_t o = (uint64_t)ceil((double)p * sqrt((double)x * (double)y) / (double)q);
    while (o > 0 && (unsigned __int128)(o - 1) * (o - 1) * qq >= rhs) o--;
    while ((unsigned __int128)o * o * qq < rhs) o++;
    return (int64_t)o;
}

// Smallest overlap passing the test for sizes whose sum is S (Jaccard, Dice,
// Overlap only).
__host__ __device__ inline int64_t need_of_sum(int sim, uint32_t p, uint32_t q, int64_t S) {
    switch (sim) {
        case BMJ_DICE: return ((uint64_t)p * S + 2ull * q - 1) / (2ull * q);
        case BMJ_OVERLAP: return ((uint64_t)p + q - 1) / q;
        default: return ((uint64_t)p * S + (uint64_t)p + q - 1) / ((uint64_t)p + q);
    }
}

__host__ __device__ inline int64_t sim_need(int sim, uint32_t p, uint32_t q, int64_t x, int64_t y) {
    return sim == BMJ_COSINE ? cosine_need(p, q, x, y) : need_of_sum(sim, p, q, x + y);
}

// The Eq. 2 limit: the pair survives iff the popcount of its xor is <= this
// (floor((x + y - h)/2) >= need  <=>  h <= x + y - 2*need).
__host__ __device__ inline int64_t sim_lim(int sim, uint32_t p, uint32_t q, int64_t x, int64_t y) {
    return x + y - 2 * sim_need(sim, p, q, x, y);
}

}  // namespace bmj
