// gom_bitplane.cuh -- bit-plane arithmetic shared by the bit-sliced mixing
// path and Forced Improvement: one 32-bit register holds one bit of 32
// individuals, so one logic instruction works on 32 trials.  Weighted sums
// of bit-planes by ripple-carry adders (the signed delta of a GOM step in one
// chain per edge), and the per-lane bit-sliced fitness accumulator with its
// flush into the block's fitness accumulators.  Anonymous namespace: each translation
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

// D += u * pos - u * neg over NP bit-planes, two's complement (pos and neg
// disjoint; u < 2^UB).  A lane that subtracts adds the complement of u with a
// carry of one in: its planes are ~u below UB, all ones above (the sign
// extension), and a lane that adds has u below UB, zero above -- so plane t
// is (bit t of u ? pos : neg) below UB and neg above, and one ripple-carry
// chain serves both signs.  The caller keeps every partial sum inside
// [-2^(NP-1), 2^(NP-1)); the carry out of the top plane is dropped.
template <int NP, int UB>
__device__ __forceinline__ void add_signed(uint32_t (&D)[NP], uint32_t pos, uint32_t neg, uint32_t u)
{
    uint32_t carry = neg;
#pragma unroll
    for (int t = 0; t < NP; ++t) {
        const uint32_t in = t < UB ? (((u >> t) & 1u) ? pos : neg) : neg;
        const uint32_t a = D[t];
        D[t] = a ^ in ^ carry;
        carry = (a & in) | (a & carry) | (in & carry);
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

// Adds the accepted deltas (non-negative and below 2^R: planes 0 .. R - 1 of
// D, masked by acc) into the lane's fitness accumulator.
template <int R>
__device__ __forceinline__ void fit_add(BsLane &L, const uint32_t (&D)[R + 1], uint32_t acc)
{
    uint32_t carry = 0;
#pragma unroll
    for (int t = 0; t < kFitPlanes; ++t) {
        const uint32_t in = t < R ? (D[t] & acc) : 0u;
        const uint32_t a = L.fit[t];
        L.fit[t] = a ^ in ^ carry;
        carry = (a & in) | (a & carry) | (in & carry);
    }
}

} // namespace
