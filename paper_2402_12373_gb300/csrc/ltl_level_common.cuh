// ltl_level_common.cuh -- pieces shared by the size-level candidate kernels.
//
// A candidate (Section 3, handleOp) is one connective applied to cached
// operands.  Its characteristic matrix (CM) is computed in registers, spread
// over the CTA: thread `tid` owns, in chunk c of group g, the traces
// t0 = 2 * ((g * C + c) * NT + tid) and t0 + 1, every bit-plane w of both.
// The check-and-cache step then needs three CTA-wide facts: the NH
// fingerprint (a sum, so the thread split does not matter), the soundness
// test of eq. (dagger) (an AND over traces), and -- after a hash-set probe --
// either a store of the new CM or a full compare with an equal-fingerprint
// entry.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ltl_device.cuh"
#include "ltl_types.h"

namespace ltl {
namespace lvl {

__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(volatile const int *)p; }

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    return *(volatile const unsigned long long *)p;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Publishes an entry.  No fence is needed before it: the matrix words were
// written before a barrier (CTA, mbarrier or cluster) that the publishing
// thread passed, and a release at GPU scope is cumulative over writes ordered
// before it that way; readers acquire the slot and then read the matrix
// (PTX memory model: base causality order is transitive through each
// release/acquire pair).
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// 128-bit compare-and-swap of a hash slot (acquire, GPU scope): if the slot
// holds {c_key, c_val} it becomes {n_key, n_val}; the slot's previous
// contents are returned either way.  With {0, 0} -> {0, 0} it is an atomic
// read of the slot.
__device__ __forceinline__ HSlot slot_cas(HSlot *p, unsigned long long c_key, unsigned long long c_val,
                                          unsigned long long n_key, unsigned long long n_val) {
    HSlot o;
    asm volatile(
        "{\n"
        "  .reg .b128 d, b, c;\n"
        "  mov.b128 b, {%2, %3};\n"
        "  mov.b128 c, {%4, %5};\n"
        "  atom.acquire.gpu.global.cas.b128 d, [%6], b, c;\n"
        "  mov.b128 {%0, %1}, d;\n"
        "}\n"
        : "=l"(o.key), "=l"(o.val)
        : "l"(c_key), "l"(c_val), "l"(n_key), "l"(n_val), "l"(p)
        : "memory");
    return o;
}

// Publishes a claimed slot: {key, val} by a 128-bit exchange with release
// semantics (GPU scope), so that a reader whose slot_cas returns the index
// also sees the entry's matrix and provenance written before.
__device__ __forceinline__ void slot_publish(const Problem &pb, unsigned long long h, unsigned long long key,
                                             unsigned long long val) {
    asm volatile(
        "{\n"
        "  .reg .b128 d, b;\n"
        "  mov.b128 b, {%0, %1};\n"
        "  atom.release.gpu.global.exch.b128 d, [%2], b;\n"
        "}\n" ::"l"(key),
        "l"(val), "l"(pb.hslots + h)
        : "memory");
}

template <int W, int C>
struct Frag {
    uint64_t v[C][2][W];   // [chunk][trace of the pair][word]
};

__host__ __device__ constexpr bool is_binary(int op) { return op == OP_AND || op == OP_OR || op == OP_U; }

// Loads one thread's share of a CM: `base` points at plane 0, planes are
// `plane` words apart, the thread's pair of chunk c starts at toff + c * cs.
template <int W, int C, bool kReadOnly>
__device__ __forceinline__ void load_frag(const uint64_t *base, uint64_t plane, uint64_t toff, uint64_t cs,
                                          Frag<W, C> &f) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(base + (uint64_t)w * plane + toff + c * cs);
            const ulonglong2 q = kReadOnly ? __ldg(p) : *p;
            f.v[c][0][w] = q.x;
            f.v[c][1][w] = q.y;
        }
    }
}

// Narrow layout: one uint64 word holds two traces of at most 32 positions
// (bits 0..31: the even trace, bits 32..63: the odd one).  A shift toward
// position 0 then acts on each 32-bit half separately.
__device__ __forceinline__ uint64_t shr_narrow(uint64_t x, uint32_t s) {
    const uint32_t lo = (uint32_t)x >> s, hi = (uint32_t)(x >> 32) >> s;
    return ((uint64_t)hi << 32) | (uint64_t)lo;
}

template <int W, bool NARROW>
__device__ __forceinline__ void shr_any(const uint64_t (&cs)[W], uint32_t s, uint64_t (&out)[W]) {
    if (NARROW) {
#pragma unroll
        for (int w = 0; w < W; ++w) out[w] = shr_narrow(cs[w], s);
    } else {
        shr<W>(cs, s, out);
    }
}

// Shift kinds of the log-step loops: 0 any run-time distance; 1 a run-time
// distance below 32; K >= 32 the constant distance K.
template <int K>
struct ShiftKind {
    static constexpr int value = K;
};

// A trace of W >= 2 words shifted by s < 32 positions toward position 0: as
// 32-bit halves, every half of the result is one funnel shift of two
// neighbouring halves.
template <int W>
__device__ __forceinline__ void shr_funnel(const uint64_t (&cs)[W], uint32_t s, uint64_t (&out)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t lo = (uint32_t)cs[w], hi = (uint32_t)(cs[w] >> 32);
        const uint32_t nlo = (w + 1 < W) ? (uint32_t)cs[w + 1] : 0u;
        out[w] = ((uint64_t)__funnelshift_r(hi, nlo, s) << 32) | (uint64_t)__funnelshift_r(lo, hi, s);
    }
}

template <int W, bool NARROW, int K>
__device__ __forceinline__ void shr_kind(const uint64_t (&cs)[W], uint32_t s, uint64_t (&out)[W]) {
    if constexpr (NARROW || W == 1 || K == 0) shr_any<W, NARROW>(cs, K >= 32 ? (uint32_t)K : s, out);
    else if constexpr (K == 1) shr_funnel<W>(cs, s, out);
    else shr<W>(cs, (uint32_t)K, out);   // a constant multiple of 32: word and half-word moves
}

// Runs step(kind, s, last) for s = 2^0 .. 2^(nsteps - 1) (last: the final
// step).  In the wide layouts the distances below 32 run in one loop of
// funnel shifts and the distances 32, 64, ... (one per word size, at most
// log2(64 W) steps in all) are peeled off as constant word moves, so no
// step needs a variable 64-bit shift with carry; narrow and one-word traces
// keep one loop.
template <int W, bool NARROW, class Step>
__device__ __forceinline__ void log_steps(int nsteps, Step &&step) {
    if constexpr (NARROW || W == 1) {
        for (int i = 0; i < nsteps; ++i) step(ShiftKind<0>{}, 1u << i, i + 1 == nsteps);
    } else {
        const int ns = nsteps < 5 ? nsteps : 5;
        for (int i = 0; i < ns; ++i) step(ShiftKind<1>{}, 1u << i, i + 1 == nsteps);
        if (nsteps > 5) step(ShiftKind<32>{}, 32u, nsteps == 6);
        if (nsteps > 6) step(ShiftKind<64>{}, 64u, nsteps == 7);
        if constexpr (W >= 4)
            if (nsteps > 7) step(ShiftKind<128>{}, 128u, nsteps == 8);
        if constexpr (W >= 8)
            if (nsteps > 8) step(ShiftKind<256>{}, 256u, nsteps == 9);
        for (int i = W >= 8 ? 9 : W >= 4 ? 8 : 7; i < nsteps; ++i) step(ShiftKind<0>{}, 1u << i, i + 1 == nsteps);
    }
}

// ---------------------------------------------------------------------------
// Carry-chain propagation: the same F, G and U as the exponential propagation
// of Section 4, in O(W) integer operations per trace instead of O(log n)
// steps.  With the positions of a trace reversed (the last position least
// significant), "at the next position" becomes "at the next less significant
// bit", the direction in which an integer addition carries.  U's finite-trace
// recursion r(i) = g(i) | (f(i) & r(i + 1)), r(|tr|) = 0, is then the carry
// recursion of the sum (f | g) + g -- generate where g holds, propagate where
// f holds -- so the carry into each bit is r at the next position and
//     f U g = g | (f & ~((f | g) + g)).
// F is the closure "at this position or a later one": x | -x sets every bit
// at or above the least significant set bit.  Positions past the end of a
// trace are zero in both operands, so no carry starts there, and the carry out
// of position 0 is dropped.

// Positions reversed: the W words of a wide trace in reverse order, each
// bit-reversed (the last position becomes bit 0 of word 0).  A narrow word
// holds two 32-bit traces: reversing the whole word reverses each and swaps
// the halves, and every operation below works on the halves separately, so the
// second reversal puts both back.
template <int W>
__device__ __forceinline__ void rev_trace(const uint64_t (&x)[W], uint64_t (&out)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) out[w] = __brevll(x[W - 1 - w]);
}

// a + b over a reversed trace (narrow: each 32-bit trace on its own).
template <int W, bool NARROW>
__device__ __forceinline__ void add_trace(const uint64_t (&a)[W], const uint64_t (&b)[W], uint64_t (&s)[W]) {
    if constexpr (NARROW) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t lo = (uint32_t)a[w] + (uint32_t)b[w];
            const uint32_t hi = (uint32_t)(a[w] >> 32) + (uint32_t)(b[w] >> 32);
            s[w] = ((uint64_t)hi << 32) | (uint64_t)lo;
        }
    } else if constexpr (W == 1) {
        s[0] = a[0] + b[0];
    } else if constexpr (W == 2) {
        asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;"
            : "=l"(s[0]), "=l"(s[1])
            : "l"(a[0]), "l"(a[1]), "l"(b[0]), "l"(b[1]));
    } else if constexpr (W == 4) {
        asm("add.cc.u64 %0, %4, %8;\n\taddc.cc.u64 %1, %5, %9;\n\taddc.cc.u64 %2, %6, %10;\n\taddc.u64 %3, %7, %11;"
            : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3])
            : "l"(a[0]), "l"(a[1]), "l"(a[2]), "l"(a[3]), "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]));
    } else {
        static_assert(W == 8, "traces of 1, 2, 4 or 8 words");
        asm("add.cc.u64 %0, %8, %16;\n\taddc.cc.u64 %1, %9, %17;\n\taddc.cc.u64 %2, %10, %18;\n\t"
            "addc.cc.u64 %3, %11, %19;\n\taddc.cc.u64 %4, %12, %20;\n\taddc.cc.u64 %5, %13, %21;\n\t"
            "addc.cc.u64 %6, %14, %22;\n\taddc.u64 %7, %15, %23;"
            : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3]), "=l"(s[4]), "=l"(s[5]), "=l"(s[6]), "=l"(s[7])
            : "l"(a[0]), "l"(a[1]), "l"(a[2]), "l"(a[3]), "l"(a[4]), "l"(a[5]), "l"(a[6]), "l"(a[7]), "l"(b[0]),
              "l"(b[1]), "l"(b[2]), "l"(b[3]), "l"(b[4]), "l"(b[5]), "l"(b[6]), "l"(b[7]));
    }
}

// -a over a reversed trace (narrow: each 32-bit trace on its own).
template <int W, bool NARROW>
__device__ __forceinline__ void neg_trace(const uint64_t (&a)[W], uint64_t (&s)[W]) {
    if constexpr (NARROW) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t lo = 0u - (uint32_t)a[w];
            const uint32_t hi = 0u - (uint32_t)(a[w] >> 32);
            s[w] = ((uint64_t)hi << 32) | (uint64_t)lo;
        }
    } else if constexpr (W == 1) {
        s[0] = 0ull - a[0];
    } else if constexpr (W == 2) {
        asm("sub.cc.u64 %0, 0, %2;\n\tsubc.u64 %1, 0, %3;" : "=l"(s[0]), "=l"(s[1]) : "l"(a[0]), "l"(a[1]));
    } else if constexpr (W == 4) {
        asm("sub.cc.u64 %0, 0, %4;\n\tsubc.cc.u64 %1, 0, %5;\n\tsubc.cc.u64 %2, 0, %6;\n\tsubc.u64 %3, 0, %7;"
            : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3])
            : "l"(a[0]), "l"(a[1]), "l"(a[2]), "l"(a[3]));
    } else {
        static_assert(W == 8, "traces of 1, 2, 4 or 8 words");
        asm("sub.cc.u64 %0, 0, %8;\n\tsubc.cc.u64 %1, 0, %9;\n\tsubc.cc.u64 %2, 0, %10;\n\t"
            "subc.cc.u64 %3, 0, %11;\n\tsubc.cc.u64 %4, 0, %12;\n\tsubc.cc.u64 %5, 0, %13;\n\t"
            "subc.cc.u64 %6, 0, %14;\n\tsubc.u64 %7, 0, %15;"
            : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3]), "=l"(s[4]), "=l"(s[5]), "=l"(s[6]), "=l"(s[7])
            : "l"(a[0]), "l"(a[1]), "l"(a[2]), "l"(a[3]), "l"(a[4]), "l"(a[5]), "l"(a[6]), "l"(a[7]));
    }
}

// F of one trace in place, by the carry chain.
template <int W, bool NARROW>
__device__ __forceinline__ void carry_f(uint64_t (&x)[W]) {
    uint64_t y[W], n[W];
    rev_trace<W>(x, y);
    neg_trace<W, NARROW>(y, n);
#pragma unroll
    for (int w = 0; w < W; ++w) y[w] |= n[w];
    rev_trace<W>(y, x);
}

// f U g of one trace into g, by the carry chain; fr = f with its positions
// reversed (rev_trace).
template <int W, bool NARROW>
__device__ __forceinline__ void carry_u(const uint64_t (&fr)[W], uint64_t (&g)[W]) {
    uint64_t gr[W], x[W], sm[W];
    rev_trace<W>(g, gr);
#pragma unroll
    for (int w = 0; w < W; ++w) x[w] = fr[w] | gr[w];
    add_trace<W, NARROW>(x, gr, sm);
#pragma unroll
    for (int w = 0; w < W; ++w) x[w] = gr[w] | (fr[w] & ~sm[w]);
    rev_trace<W>(x, g);
}

// The connective itself (Section 4) on all of a thread's traces at once: a =
// left operand (or the only one), r = right operand on entry for binary
// connectives, the result on exit; m = length mask (Not and G).  The
// exponential-propagation loops run step-outer, trace-inner, so each shift
// step issues 2 * C * W independent updates.
template <int OP, int W, int C, bool NARROW = false>
__device__ __forceinline__ void apply_op(Frag<W, C> &r, Frag<W, C> &a, const Frag<W, C> &m, int nsteps,
                                         bool logstep) {
    if (OP == OP_ATOM || OP == OP_X || OP == OP_F || OP == OP_G || OP == OP_NOT) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int w = 0; w < W; ++w)
                    r.v[c][j][w] = (OP == OP_NOT || OP == OP_G) ? (m.v[c][j][w] & ~a.v[c][j][w]) : a.v[c][j][w];
    }
    if (OP == OP_X) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint64_t t[W];
                shr_any<W, NARROW>(r.v[c][j], 1u, t);
#pragma unroll
                for (int w = 0; w < W; ++w) r.v[c][j][w] = t[w];
            }
    } else if ((OP == OP_F || OP == OP_G) && !logstep) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) carry_f<W, NARROW>(r.v[c][j]);
        if (OP == OP_G) {   // G f = not F not f within the trace
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int w = 0; w < W; ++w) r.v[c][j][w] = m.v[c][j][w] & ~r.v[c][j][w];
        }
    } else if (OP == OP_F || OP == OP_G) {
        log_steps<W, NARROW>(nsteps, [&](auto kind, uint32_t s, bool) {
            constexpr int K = decltype(kind)::value;
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    uint64_t t[W];
                    shr_kind<W, NARROW, K>(r.v[c][j], s, t);
#pragma unroll
                    for (int w = 0; w < W; ++w) r.v[c][j][w] |= t[w];
                }
        });
        if (OP == OP_G) {   // G f = not F not f within the trace
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int w = 0; w < W; ++w) r.v[c][j][w] = m.v[c][j][w] & ~r.v[c][j][w];
        }
    } else if (OP == OP_AND || OP == OP_OR) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int w = 0; w < W; ++w)
                    r.v[c][j][w] = (OP == OP_AND) ? (r.v[c][j][w] & a.v[c][j][w]) : (r.v[c][j][w] | a.v[c][j][w]);
    } else if (OP == OP_U && !logstep) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint64_t fr[W];
                rev_trace<W>(a.v[c][j], fr);
                carry_u<W, NARROW>(fr, r.v[c][j]);
            }
    } else if (OP == OP_U) {
        // a: "f holds on [j, j + 2^i)"; r: "f U g within 2^i" (Lemma 2)
        log_steps<W, NARROW>(nsteps, [&](auto kind, uint32_t s, bool last) {
            constexpr int K = decltype(kind)::value;
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    uint64_t t[W];
                    shr_kind<W, NARROW, K>(r.v[c][j], s, t);
#pragma unroll
                    for (int w = 0; w < W; ++w) r.v[c][j][w] |= a.v[c][j][w] & t[w];
                    if (!last) {
                        shr_kind<W, NARROW, K>(a.v[c][j], s, t);
#pragma unroll
                        for (int w = 0; w < W; ++w) a.v[c][j][w] &= t[w];
                    }
                }
        });
    }
}

// A binary connective on a batch of NB candidates that share the left operand
// a (r[k] = right operand k on entry, the result on exit).  For U the left
// operand's own propagation (Lemma 2: "f holds on [j, j + 2^i)") does not
// depend on the right operand, so it runs once per batch, and each step costs
// every candidate one shift and one three-input logic operation.  Slots
// k >= nb hold zeros and are computed like the others (uniform control flow).
template <int OP, int W, int C, int NB, bool NARROW = false>
__device__ __forceinline__ void apply_binary_batch(Frag<W, C> (&r)[NB], Frag<W, C> &a, int nsteps, bool logstep) {
    if (OP == OP_AND || OP == OP_OR) {
#pragma unroll
        for (int k = 0; k < NB; ++k)
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int w = 0; w < W; ++w)
                        r[k].v[c][j][w] =
                            (OP == OP_AND) ? (r[k].v[c][j][w] & a.v[c][j][w]) : (r[k].v[c][j][w] | a.v[c][j][w]);
    } else if (OP == OP_U && !logstep) {
        // the left operand is reversed once for the batch
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint64_t fr[W];
                rev_trace<W>(a.v[c][j], fr);
#pragma unroll
                for (int k = 0; k < NB; ++k) carry_u<W, NARROW>(fr, r[k].v[c][j]);
            }
    } else if (OP == OP_U) {
        log_steps<W, NARROW>(nsteps, [&](auto kind, uint32_t s, bool last) {
            constexpr int K = decltype(kind)::value;
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    uint64_t t[W];
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        shr_kind<W, NARROW, K>(r[k].v[c][j], s, t);
#pragma unroll
                        for (int w = 0; w < W; ++w) r[k].v[c][j][w] |= a.v[c][j][w] & t[w];
                    }
                    if (!last) {
                        shr_kind<W, NARROW, K>(a.v[c][j], s, t);
#pragma unroll
                        for (int w = 0; w < W; ++w) a.v[c][j][w] &= t[w];
                    }
                }
        });
    }
}

// Soundness bits of this thread's traces: the value at position 0 of trace
// slot (c, j) is bit 2c + j; in the narrow layout word (c, j) holds two
// traces, at bits 4c + 2j (even trace) and 4c + 2j + 1 (odd trace).
template <int W, int C, bool NARROW = false>
__device__ __forceinline__ uint32_t pos0_bits(const Frag<W, C> &r) {
    uint32_t b = 0;
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (NARROW) {
                b |= ((uint32_t)r.v[c][j][0] & 1u) << (4 * c + 2 * j);
                b |= ((uint32_t)(r.v[c][j][0] >> 32) & 1u) << (4 * c + 2 * j + 1);
            } else {
                b |= ((uint32_t)r.v[c][j][0] & 1u) << (2 * c + j);
            }
        }
    return b;
}

template <int W, int C>
__device__ __forceinline__ void store_frag(const Frag<W, C> &r, uint64_t *dst, uint64_t plane, uint64_t toff,
                                           uint64_t cs) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            ulonglong2 q;
            q.x = r.v[c][0][w];
            q.y = r.v[c][1][w];
            *reinterpret_cast<ulonglong2 *>(dst + (uint64_t)w * plane + toff + c * cs) = q;
        }
    }
}

// Entries published during this launch are read through L2 only (ld.cg).
template <int W, int C>
__device__ __forceinline__ bool equal_frag(const Frag<W, C> &r, const uint64_t *src, uint64_t plane, uint64_t toff,
                                           uint64_t cs) {
    bool eq = true;
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const ulonglong2 q =
                __ldcg(reinterpret_cast<const ulonglong2 *>(src + (uint64_t)w * plane + toff + c * cs));
            eq &= (q.x == r.v[c][0][w]) & (q.y == r.v[c][1][w]);
        }
    }
    return eq;
}

template <int W, int C>
__device__ __forceinline__ bool equal_regs(const Frag<W, C> &x, const Frag<W, C> &y) {
    bool eq = true;
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int w = 0; w < W; ++w) eq &= x.v[c][j][w] == y.v[c][j][w];
    return eq;
}

enum : int { DEC_NEW = 0, DEC_CMP = 1, DEC_FAIL = 2, DEC_ERR = 3, DEC_DUP = 4, DEC_WAIT = 5 };

// One probe run by a single thread from slot h: claims an empty slot
// (DEC_NEW, with a freshly allocated entry index), or stops at a slot holding
// the same fingerprint (DEC_CMP, with the entry to compare against).  If that
// slot's entry is not yet published, the blocking form waits (bounded); the
// non-blocking form returns DEC_WAIT with h left on the slot, for callers that
// may hold unpublished claims of their own (waiting there could deadlock two
// CTAs that each wait for the other's publication).  With kAlloc each lane
// takes its entry index with its own atomicAdd (the fused, streaming and
// cluster kernels: a warp-aggregated allocation measured slower in the fused
// kernel, since the warp's atomic waits for its slowest lane's CAS); without
// it a claim returns DEC_NEW and the caller allocates (claim_entry) -- the
// warp-specialised kernel's hash warps, whose lanes' claims complete together,
// take a round's claims with one atomic.
template <bool kBlocking, bool kAlloc = true>
__device__ __forceinline__ int probe(const Problem &pb, unsigned long long key, unsigned long long &h,
                                     unsigned long long &idx, bool full) {
    // while the cache has room (`full`: the caller's recent reading of the
    // cache-full flag), the 128-bit CAS itself reads the slot -- one round
    // trip for an empty slot, another key, or a match whose entry index is
    // already published; a full cache stores nothing more, so then the CAS
    // claims nothing and only reads
    for (unsigned long long n = 0; n <= pb.hmask; ++n) {
        HSlot *slot = pb.hslots + h;
        HSlot o = slot_cas(slot, 0ull, 0ull, full ? 0ull : key, full ? 0ull : kValPending);
        if (o.key == 0ull) {
            if (full) return DEC_FAIL;
            if (!kAlloc) return DEC_NEW;   // claimed; the caller allocates the entry (claim_entry)
            const unsigned long long i = atomicAdd(&pb.ctrl->n_entries, 1ull);
            if (i >= pb.max_entries) {
                slot_publish(pb, h, key, kValFail);
                atomicExch(&pb.ctrl->cap_hit, 1);
                return DEC_FAIL;
            }
            idx = i;
            return DEC_NEW;
        }
        if (o.key == key) {
            // relaxed admission: an equal key is a duplicate, whatever the matrix
            if (pb.ruc != RUC_EXACT) return DEC_DUP;
            unsigned long long spins = 0;
            while (o.val == kValPending) {
                if (!kBlocking) return DEC_WAIT;
                if (++spins > pb.spin_limit) {
                    atomicAdd(&pb.ctrl->timeouts, 1ull);
                    atomicCAS(&pb.ctrl->err, 0, -4 /* LTL_ERR_TIMEOUT */);
                    atomicExch(&pb.ctrl->stop, 1);
                    return DEC_ERR;
                }
                __nanosleep(64);
                o = slot_cas(slot, 0ull, 0ull, 0ull, 0ull);
            }
            if (o.val == kValFail) return DEC_FAIL;
            idx = o.val;
            return DEC_CMP;
        }
        h = (h + 1) & pb.hmask;
    }
    atomicExch(&pb.ctrl->cap_hit, 1);   // table full
    return DEC_FAIL;
}

// The entry of a slot claimed by probe<..., false>: index i from the
// problem's entry counter (result DEC_NEW), or, past the cache's capacity,
// the slot published as failed and the cache marked full (DEC_FAIL).
__device__ __forceinline__ int claim_entry(const Problem &pb, unsigned long long h, unsigned long long key,
                                           unsigned long long i, unsigned long long &idx) {
    if (i >= pb.max_entries) {
        slot_publish(pb, h, key, kValFail);
        atomicExch(&pb.ctrl->cap_hit, 1);
        return DEC_FAIL;
    }
    idx = i;
    return DEC_NEW;
}

// Sum mod 2^64 of a 64-bit value over the 32 lanes of a warp, by three
// 32-bit warp reductions: the high words mod 2^32, and the two 16-bit halves
// of the low words (each sum < 2^21, so exact); every lane gets the sum.
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    const uint32_t s_lo = __reduce_add_sync(0xffffffffu, lo & 0xFFFFu);
    const uint32_t s_mid = __reduce_add_sync(0xffffffffu, lo >> 16);
    const uint32_t s_hi = __reduce_add_sync(0xffffffffu, hi);
    return ((uint64_t)s_hi << 32) + ((uint64_t)s_mid << 16) + (uint64_t)s_lo;
}

// Records a separator (eq. (dagger)): the first one seen wins the atomic and
// its provenance is kept.  Callers skip the call once they know a separator
// of the problem has been recorded (its count is only read as a flag).
__device__ __forceinline__ void record_separator(const Problem &pb, int level, uint64_t prov) {
    if (atomicAdd(&pb.ctrl->found_count, 1u) == 0u) {
        pb.ctrl->found_prov = prov;
        pb.ctrl->found_level = level;
    }
    if (pb.stop_first) atomicExch(&pb.ctrl->stop, 1);
}

__device__ __forceinline__ unsigned long long fp_key(uint64_t s) {
    const unsigned long long key = mix64(s);
    return key ? key : 1ull;
}

// Hash-table key and first slot of a candidate from its reduced fingerprint s.
// Exact admission: the finalised NH sum (then a full compare on a match).
// Relaxed admission (Section 5): a 63-bit key -- the finalised NH sum, or the
// first-k-percent bits themselves -- with the masked-out bits zeroed; bit 63
// is set so that no key is 0 (the empty slot) and key equality is exactly
// equality of the 63-bit values; the slot comes from a finalised copy.
__device__ __forceinline__ unsigned long long admission_key(const Problem &pb, uint64_t s, unsigned long long &h) {
    if (pb.ruc == RUC_EXACT) {
        unsigned long long key = fp_key(s);
        // masked fingerprints (a stress setting): more equal keys of different
        // matrices, still told apart by the full compare
        if (pb.key_mask != kKey63) key = (key & pb.key_mask) | (1ull << 63);
        h = key & pb.hmask;
        return key;
    }
    const uint64_t v = (pb.ruc == RUC_HASH ? mix64(s) : s) & pb.key_mask;
    const unsigned long long key = v | (1ull << 63);
    h = mix64(key) & pb.hmask;
    return key;
}

// First-k-percent term of one word of plane 0: the first b positions of trace
// t go to bits [t*b, t*b + b) of the 63-bit key; what falls beyond bit 62 is
// dropped.  Terms of different traces do not overlap, so summing them (the
// reduction used for fingerprints) concatenates them.
__device__ __forceinline__ uint64_t fkp_term(uint64_t positions, uint64_t t, uint32_t b) {
    const uint64_t lo = t * (uint64_t)b;
    if (lo >= 63) return 0;
    const uint64_t v = b >= 64 ? positions : positions & ((1ull << b) - 1);
    return (v << lo) & kKey63;
}

// First-k-percent terms of the 2x2 words (c, j) of a thread's fragment: word
// (c, j) of plane 0 holds trace toff + c*cs + j (wide layout) or traces
// 2(toff + c*cs + j) and 2(toff + c*cs + j) + 1 in its low and high halves
// (narrow layout).
template <bool NARROW>
__device__ __forceinline__ uint64_t fkp_word(uint64_t w0, uint64_t word_index, uint32_t b) {
    if (NARROW)
        return fkp_term(w0 & 0xFFFFFFFFull, 2 * word_index, b) + fkp_term(w0 >> 32, 2 * word_index + 1, b);
    return fkp_term(w0, word_index, b);
}

// Decodes tile k of a segment into operand ranges [a0, a1) x [b0, b1).
__device__ __forceinline__ void decode_tile(const Seg &sg, uint64_t k, uint64_t &a0, uint64_t &a1, uint64_t &b0,
                                            uint64_t &b1) {
    if (sg.kind == SEG_UNARY) {
        a0 = k * sg.ta;
        a1 = min(a0 + sg.ta, sg.a_count);
        b0 = 0;
        b1 = 1;
        return;
    }
    uint64_t ta, tb;
    if (sg.kind == SEG_RECT) {
        if (sg.a_inner) { ta = k % sg.n_ta; tb = k / sg.n_ta; }
        else { tb = k % sg.n_tb; ta = k / sg.n_tb; }
    } else {
        // upper-triangular tiles (ta <= tb), row-major: row ta holds n - ta tiles
        const int64_t n = (int64_t)sg.n_ta;
        const double dn = (double)n;
        double est = ((2.0 * dn + 1.0) - sqrt((2.0 * dn + 1.0) * (2.0 * dn + 1.0) - 8.0 * (double)k)) * 0.5;
        int64_t r = (int64_t)est;
        if (r < 0) r = 0;
        if (r > n - 1) r = n - 1;
        auto row_start = [&](int64_t x) -> int64_t { return x * n - x * (x - 1) / 2; };
        while (r > 0 && row_start(r) > (int64_t)k) --r;
        while (r + 1 < n && row_start(r + 1) <= (int64_t)k) ++r;
        ta = (uint64_t)r;
        tb = ta + ((uint64_t)k - (uint64_t)row_start(r));
    }
    a0 = ta * sg.ta;
    a1 = min(a0 + sg.ta, sg.a_count);
    b0 = tb * sg.tb;
    b1 = min(b0 + sg.tb, sg.b_count);
}

// The segment holding `tile`: the last one whose first tile is <= tile
// (binary search; a launch may carry the segments of many problems).
__device__ __forceinline__ int find_segment(const LevelArgs &la, unsigned long long tile) {
    int lo = 0, hi = la.n_segs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (la.segs[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace lvl
}  // namespace ltl
