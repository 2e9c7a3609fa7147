// gom_bitplane.cuh -- bit-plane arithmetic shared by the bit-sliced mixing
// path and Forced Improvement: one 32-bit register holds one bit of 32
// individuals, so one logic instruction works on 32 trials.  Weighted sums
// of bit-planes by ripple-carry adders, the signed delta T - 2N of a GOM
// step, and the per-lane bit-sliced fitness accumulator with its flush into
// the block's fitness accumulators.  Anonymous namespace: each translation
// unit that includes it compiles its own copy.
#pragma once

#include <cuda_runtime.h>

#include "gom_internal.h"

namespace {

constexpr int kFitPlanes = 24;  // bits of the per-lane bit-sliced fitness accumulator
constexpr int kWeightBits = 8;  // |w| < 2^8 on this path

// x & (bit t of u ? ~0 : 0), for a per-lane weight u.
__device__ __forceinline__ uint32_t bit_mask(uint32_t x, uint32_t u, int t) { return ((u >> t) & 1u) ? x : 0u; }

// acc += u * x over R bit-planes (ripple carry; u < 2^UB; the sum stays below
// 2^R by the caller's bound, so the last carry is always zero).
template <int R, int UB, int NA>
__device__ __forceinline__ void add_weighted(uint32_t (&acc)[NA], uint32_t x, uint32_t u)
{
    static_assert(NA >= R, "accumulator narrower than R");
    uint32_t carry = 0;
#pragma unroll
    for (int t = 0; t < R; ++t) {
        if (t < UB) {
            const uint32_t in = bit_mask(x, u, t);
            const uint32_t a = acc[t];
            acc[t] = a ^ in ^ carry;
            carry = (a & in) | (a & carry) | (in & carry);
        } else {
            const uint32_t a = acc[t];
            acc[t] = a ^ carry;
            carry = a & carry;
        }
    }
}

// Per-lane state of the bit-sliced path across the groups of a generation.
struct BsLane {
    uint32_t fit[kFitPlanes]; // accepted deltas of this lane's 32 individuals (word lane mod W), bit-sliced
    int since_flush;          // items added since the last flush (warp-uniform)
    unsigned n_dl, n_acc, n_imp;
};

__device__ __forceinline__ void bs_lane_zero(BsLane &L)
{
#pragma unroll
    for (int t = 0; t < kFitPlanes; ++t) L.fit[t] = 0;
    L.since_flush = 0;
    L.n_dl = L.n_acc = L.n_imp = 0;
}

// Adds the lane's accumulated deltas into the block's fitness accumulators
// s_f[32 w + b] (one shared atomic per individual with a non-zero sum) and
// clears them.  Warp-wide call.
__device__ __forceinline__ void bs_flush(const GomParams &P, BsLane &L, long long *s_f)
{
    const int lane = threadIdx.x & 31;
    const int w = lane & (P.W - 1);
    uint32_t any = 0;
#pragma unroll
    for (int t = 0; t < kFitPlanes; ++t) any |= L.fit[t];
    if (any) {
        for (int b = 0; b < 32; ++b) {
            if (!((any >> b) & 1u)) continue;
            unsigned v = 0;
#pragma unroll
            for (int t = 0; t < kFitPlanes; ++t) v |= ((L.fit[t] >> b) & 1u) << t;
            atomicAdd(reinterpret_cast<unsigned long long *>(&s_f[32 * w + b]), (unsigned long long)v);
        }
    }
#pragma unroll
    for (int t = 0; t < kFitPlanes; ++t) L.fit[t] = 0;
    L.since_flush = 0;
}

// delta = T - 2N over R + 2 bit-planes (two's complement), in place in T
// (T has R + 2 planes, its top two zero on entry).  Returns, as planes, the
// individuals whose delta is non-zero (*nz) and negative (*neg).
template <int R>
__device__ __forceinline__ void delta_planes(uint32_t (&T)[R + 2], const uint32_t (&N)[R], uint32_t *nz, uint32_t *neg)
{
    uint32_t carry = 0xFFFFFFFFu; // + 1 of the negation
#pragma unroll
    for (int t = 0; t < R + 2; ++t) {
        const uint32_t a = T[t];
        const uint32_t b = ~((t >= 1 && t - 1 < R) ? N[t - 1] : 0u);
        T[t] = a ^ b ^ carry;
        carry = (a & b) | (a & carry) | (b & carry);
    }
    uint32_t z = 0;
#pragma unroll
    for (int t = 0; t < R + 2; ++t) z |= T[t];
    *nz = z;
    *neg = T[R + 1];
}

// Adds the accepted deltas (non-negative: bits 0 .. R of D, masked by acc)
// into the lane's fitness accumulator.
template <int R>
__device__ __forceinline__ void fit_add(BsLane &L, const uint32_t (&D)[R + 2], uint32_t acc)
{
    uint32_t carry = 0;
#pragma unroll
    for (int t = 0; t < kFitPlanes; ++t) {
        const uint32_t in = t <= R ? (D[t] & acc) : 0u;
        const uint32_t a = L.fit[t];
        L.fit[t] = a ^ in ^ carry;
        carry = (a & in) | (a & carry) | (in & carry);
    }
}

} // namespace
