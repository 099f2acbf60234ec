// ltl_device.cuh -- device-side building blocks of the GB300 LTL learner.
//
// Characteristic sequences (CS, Section 4 of "LTL learning on GPUs") are kept
// as W uint64 words per trace, least significant bit = position 0.  With
// that bit order the paper's left shift for X (position i takes the value at
// i+1) is a right shift here, and a shift by s carries the low s bits of
// word w+1 into the top of word w.
//
// Every operator keeps sequences canonical: bits at positions >= the trace's
// length are 0 (every formula is false beyond the end of a trace, Section 2).
// X, F, U, And and Or preserve that on canonical inputs; Not and G are masked
// with the per-trace length mask.
#pragma once
#include <cstdint>

#include "ltl_types.h"

namespace ltl {

// out = cs shifted toward position 0 by s positions: out(pos) = cs(pos + s),
// zero past the last word.  s is a power of two; s < 64 when W == 1.
template <int W>
__device__ __forceinline__ void shr(const uint64_t (&cs)[W], uint32_t s, uint64_t (&out)[W]) {
    if (W == 1) {
        out[0] = cs[0] >> s;
        return;
    }
    if (s < 64) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t v = cs[w] >> s;
            if (w + 1 < W) v |= cs[w + 1] << (64 - s);
            out[w] = v;
        }
    } else {
        const uint32_t q = s >> 6;   // whole-word shift (s is a multiple of 64)
#pragma unroll
        for (int w = 0; w < W; ++w) {
            uint64_t v = 0;
#pragma unroll
            for (int k = 1; k < W; ++k)
                if (w + k < W && q == (uint32_t)k) v = cs[w + k];
            out[w] = v;
        }
    }
}

// X f: strong next (false at the last position), one shift (Section 4).
template <int W>
__device__ __forceinline__ void op_x(uint64_t (&c)[W]) {
    uint64_t t[W];
    shr<W>(c, 1u, t);
#pragma unroll
    for (int w = 0; w < W; ++w) c[w] = t[w];
}

// F f by exponential propagation (Section 4, Lemma 1 of Appendix B):
// after step i, position j holds iff f holds somewhere in [j, j + 2^i).
// nsteps = ceil(log2(max trace length)) reaches every later position.
template <int W>
__device__ __forceinline__ void op_f(uint64_t (&c)[W], int nsteps) {
    for (int i = 0; i < nsteps; ++i) {
        uint64_t t[W];
        shr<W>(c, 1u << i, t);
#pragma unroll
        for (int w = 0; w < W; ++w) c[w] |= t[w];
    }
}

// G f = not F not f, restricted to the trace (the paper gives no listing
// for G; this is the reading used throughout): G f holds at i iff f holds at
// every i <= j < |tr|.
template <int W>
__device__ __forceinline__ void op_g(uint64_t (&c)[W], const uint64_t (&m)[W], int nsteps) {
#pragma unroll
    for (int w = 0; w < W; ++w) c[w] = m[w] & ~c[w];
    op_f<W>(c, nsteps);
#pragma unroll
    for (int w = 0; w < W; ++w) c[w] = m[w] & ~c[w];
}

// f U g by exponential propagation (Section 4, Lemma 2 of Appendix B):
// c1 tracks "f holds on [j, j + 2^i)" and c2 tracks "f U g within 2^i".
template <int W>
__device__ __forceinline__ void op_u(uint64_t (&c1)[W], uint64_t (&c2)[W], int nsteps) {
    for (int i = 0; i < nsteps; ++i) {
        const uint32_t s = 1u << i;
        uint64_t t[W];
        shr<W>(c2, s, t);
#pragma unroll
        for (int w = 0; w < W; ++w) c2[w] |= c1[w] & t[w];
        if (i + 1 < nsteps) {
            shr<W>(c1, s, t);
#pragma unroll
            for (int w = 0; w < W; ++w) c1[w] &= t[w];
        }
    }
}

// One term of the NH universal hash (Black, Halevi, Krawczyk, Krovetz and
// Rogaway, "UMAC: fast and secure message authentication", CRYPTO 1999):
// ((lo(x) + lo(k)) mod 2^32) * ((hi(x) + hi(k)) mod 2^32) as a 64-bit product.
// Summed mod 2^64 over all words of a matrix with per-position keys it is a
// fingerprint that does not depend on how threads share the words.
__device__ __forceinline__ uint64_t nh_term(uint64_t x, uint64_t k) {
    const uint32_t a = (uint32_t)x + (uint32_t)k;
    const uint32_t b = (uint32_t)(x >> 32) + (uint32_t)(k >> 32);
    return (uint64_t)a * (uint64_t)b;
}

// SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014), a bijection
// on 64-bit words used to spread fingerprints over hash slots and to derive
// the NH keys.
__device__ __host__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace ltl
