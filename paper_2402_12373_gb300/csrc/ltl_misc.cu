// ltl_misc.cu -- the small kernels around the size-level kernels: trace
// packing (atoms and length masks), NH key generation, the provenance walk
// that rebuilds a formula, formula evaluation (ltl_eval) and the launchers.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdint>

#include "ltl_device.cuh"
#include "ltl_types.h"

namespace ltl {

// ---------------------------------------------------------------------------
// Trace packing: length masks and the atoms' characteristic matrices (and,
// given `keys`, the NH fingerprint keys, one per matrix word).  One thread per
// (plane w < Wt, trace slot t); every word of the mask, the atoms and the keys
// is written, the padding planes W..Wt-1 as zeros, so none needs clearing
// first.  Given `zero`, the launch also clears n_zero 16-byte units there
// (a problem's hash slots), grid-stride over all its threads.  Positions are read straight from the
// concatenated letters; a letter with a bit >= n_props, a decreasing offset
// or a trace longer than 64 * W marks the input invalid (a trace with bad
// offsets is then packed as empty).
// ---------------------------------------------------------------------------

// NH key of matrix word i: a SplitMix64 output of a fixed seed.
__device__ __forceinline__ uint64_t nh_key(uint64_t seed, uint64_t i) {
    return mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

__global__ void pack_kernel(const uint32_t *__restrict__ letters, const uint64_t *__restrict__ offsets,
                            uint32_t n_traces, uint64_t plane, int W, int Wt, int n_props, uint64_t *mask,
                            uint64_t *atoms, uint64_t stride, Ctrl *ctrl, uint64_t *keys, uint64_t seed,
                            uint4 *zero, uint64_t n_zero) {
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = idx; i < n_zero; i += (uint64_t)gridDim.x * blockDim.x) zero[i] = make_uint4(0, 0, 0, 0);
    if (idx >= plane * (uint64_t)Wt) return;
    if (keys) keys[idx] = nh_key(seed, idx);
    const uint64_t t = idx % plane, w = idx / plane;
    uint64_t off = 0, len = 0;
    if (t < n_traces) {
        off = offsets[t];
        const uint64_t end = offsets[t + 1];
        if (end < off || (t == 0 && off != 0)) {   // no letter of it is read
            atomicExch(&ctrl->invalid_letter, 1);
            off = 0;
        } else {
            len = end - off;
        }
        if (len > 64ull * (uint64_t)W) {
            atomicExch(&ctrl->invalid_letter, 1);
            len = 64ull * (uint64_t)W;
        }
    }
    const uint64_t lo = 64ull * w;
    const uint64_t n_here = len > lo ? min(len - lo, (uint64_t)64) : 0;
    mask[w * plane + t] = n_here == 64 ? ~0ull : ((1ull << n_here) - 1ull);
    uint32_t seen = 0;
    for (int p = 0; p < n_props; ++p) {
        uint64_t bits = 0;
        for (uint64_t i = 0; i < n_here; ++i) {
            const uint32_t l = letters[off + lo + i];
            seen |= l;
            bits |= (uint64_t)((l >> p) & 1u) << i;
        }
        atoms[(uint64_t)p * stride + w * plane + t] = bits;
    }
    if (n_props < 32 && (seen >> n_props)) atomicExch(&ctrl->invalid_letter, 1);
}

// Narrow layout (every trace at most 32 long): word q of a plane holds traces
// 2q (bits 0..31) and 2q + 1 (bits 32..63).  One thread per word.
__global__ void pack_narrow_kernel(const uint32_t *__restrict__ letters, const uint64_t *__restrict__ offsets,
                                   uint32_t n_traces, uint64_t plane, int n_props, uint64_t *mask, uint64_t *atoms,
                                   uint64_t stride, Ctrl *ctrl, uint64_t *keys, uint64_t seed, uint4 *zero,
                                   uint64_t n_zero) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = q; i < n_zero; i += (uint64_t)gridDim.x * blockDim.x) zero[i] = make_uint4(0, 0, 0, 0);
    if (q >= plane) return;
    if (keys) keys[q] = nh_key(seed, q);
    uint64_t off[2] = {0, 0}, len[2] = {0, 0};
    for (int h = 0; h < 2; ++h) {
        const uint64_t t = 2 * q + h;
        if (t < n_traces) {
            off[h] = offsets[t];
            const uint64_t end = offsets[t + 1];
            if (end < off[h] || (t == 0 && off[h] != 0)) {   // no letter of it is read
                atomicExch(&ctrl->invalid_letter, 1);
                off[h] = 0;
            } else {
                len[h] = end - off[h];
            }
            if (len[h] > 32) {
                atomicExch(&ctrl->invalid_letter, 1);
                len[h] = 32;
            }
        }
    }
    uint64_t mk = 0;
    for (int h = 0; h < 2; ++h) mk |= (len[h] == 32 ? 0xffffffffull : ((1ull << len[h]) - 1ull)) << (32 * h);
    mask[q] = mk;
    uint32_t seen = 0;
    for (int p = 0; p < n_props; ++p) {
        uint64_t bits = 0;
        for (int h = 0; h < 2; ++h)
            for (uint64_t i = 0; i < len[h]; ++i) {
                const uint32_t l = letters[off[h] + i];
                seen |= l;
                bits |= (uint64_t)((l >> p) & 1u) << (32 * h + i);
            }
        atoms[(uint64_t)p * stride + q] = bits;
    }
    if (n_props < 32 && (seen >> n_props)) atomicExch(&ctrl->invalid_letter, 1);
}

// ---------------------------------------------------------------------------
// Provenance walk: the syntax tree of a cache entry (or of a recorded
// separator) as a pre-order token list, op | (atom index << 8).  One thread
// per job; job j writes tokens[j * cap ...] and its count to n_out[j] (-1 if
// the provenance is inconsistent or the tree exceeds cap).
// ---------------------------------------------------------------------------
__global__ void walk_batch_kernel(const WalkJob *jobs, int n_jobs, uint32_t *tokens, int cap, int *n_out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_jobs) return;
    const WalkJob jb = jobs[j];
    uint32_t *tok = tokens + (uint64_t)j * cap;
    uint64_t stack[2 * kMaxLevels + 2];
    int sp = 0, n = 0;
    bool ok = true;
    stack[sp++] = jb.root;
    while (sp > 0 && n < cap && ok) {
        const uint64_t p = stack[--sp];
        const int op = prov_op(p);
        if (op > OP_U) { ok = false; break; }
        tok[n++] = (uint32_t)op | ((uint32_t)(op == OP_ATOM ? prov_a(p) : 0) << 8);
        if (op == OP_ATOM) continue;
        const bool binary = op == OP_AND || op == OP_OR || op == OP_U;
        if (prov_a(p) >= jb.n_entries || (binary && prov_b(p) >= jb.n_entries) || sp + 2 > 2 * kMaxLevels + 2) {
            ok = false;
            break;
        }
        if (binary) stack[sp++] = jb.prov[prov_b(p)];   // pushed first: visited after the left subtree
        stack[sp++] = jb.prov[prov_a(p)];
    }
    n_out[j] = (ok && sp == 0) ? n : -1;
}

// ---------------------------------------------------------------------------
// Formula evaluation (ltl_eval): a post-order program run per trace with an
// operand stack in device scratch memory; the same operator functions as the
// candidate kernels.  Program word: op | (atom << 8).
// ---------------------------------------------------------------------------
template <int W>
__global__ void eval_kernel(const uint32_t *__restrict__ prog, int n_instr, const uint64_t *__restrict__ atoms,
                            const uint64_t *__restrict__ mask, uint64_t stride, uint64_t plane,
                            uint64_t *stack, int nsteps, uint32_t n_traces, uint64_t *out, int out_words) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= plane) return;
    int sp = 0;
    for (int k = 0; k < n_instr; ++k) {
        const uint32_t ins = prog[k];
        const int op = (int)(ins & 0xffu);
        uint64_t r[W];
        if (op == OP_ATOM) {
            const uint64_t *src = atoms + (uint64_t)(ins >> 8) * stride;
#pragma unroll
            for (int w = 0; w < W; ++w) r[w] = src[(uint64_t)w * plane + t];
        } else if (op == OP_AND || op == OP_OR || op == OP_U) {
            uint64_t a[W];
            const uint64_t *sa = stack + (uint64_t)(sp - 2) * stride;
            const uint64_t *sb = stack + (uint64_t)(sp - 1) * stride;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                a[w] = sa[(uint64_t)w * plane + t];
                r[w] = sb[(uint64_t)w * plane + t];
            }
            if (op == OP_AND) {
#pragma unroll
                for (int w = 0; w < W; ++w) r[w] &= a[w];
            } else if (op == OP_OR) {
#pragma unroll
                for (int w = 0; w < W; ++w) r[w] |= a[w];
            } else {
                op_u<W>(a, r, nsteps);
            }
            sp -= 2;
        } else {
            const uint64_t *sa = stack + (uint64_t)(sp - 1) * stride;
#pragma unroll
            for (int w = 0; w < W; ++w) r[w] = sa[(uint64_t)w * plane + t];
            if (op == OP_NOT || op == OP_G) {
                uint64_t m[W];
#pragma unroll
                for (int w = 0; w < W; ++w) m[w] = mask[(uint64_t)w * plane + t];
                if (op == OP_NOT) {
#pragma unroll
                    for (int w = 0; w < W; ++w) r[w] = m[w] & ~r[w];
                } else {
                    op_g<W>(r, m, nsteps);
                }
            } else if (op == OP_X) {
                op_x<W>(r);
            } else {
                op_f<W>(r, nsteps);
            }
            sp -= 1;
        }
        uint64_t *dst = stack + (uint64_t)sp * stride;
#pragma unroll
        for (int w = 0; w < W; ++w) dst[(uint64_t)w * plane + t] = r[w];
        ++sp;
    }
    if (t < n_traces) {
        const uint64_t *res = stack;   // the single value left on the stack
        for (int w = 0; w < out_words; ++w)
            out[t * (uint64_t)out_words + w] = w < W ? res[(uint64_t)w * plane + t] : 0ull;
    }
}

// Characteristic matrix of one cache entry in the trace-major layout of ltl_eval.
__global__ void unpack_kernel(const uint64_t *src, uint64_t plane, int W, uint32_t n_traces, uint64_t *out,
                              int out_words) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_traces) return;
    for (int w = 0; w < out_words; ++w) out[t * (uint64_t)out_words + w] = w < W ? src[(uint64_t)w * plane + t] : 0ull;
}

// ---------------------------------------------------------------------------
// Host-callable launchers
// ---------------------------------------------------------------------------

// CTAs of a pack launch: enough for its words, and for clearing n_zero
// 16-byte units at about four per thread (at most 4096 CTAs; the clearing
// loop is grid-stride).
static unsigned pack_blocks(uint64_t units, uint64_t n_zero, int th) {
    const uint64_t b_pack = (units + th - 1) / th;
    const uint64_t b_zero = std::min<uint64_t>((n_zero + 4ull * th - 1) / (4ull * th), 4096);
    return (unsigned)std::max<uint64_t>(std::max(b_pack, b_zero), 1);
}

cudaError_t launch_pack(const uint32_t *letters, const uint64_t *offsets, uint32_t n_traces, uint64_t plane,
                        int W, int Wt, int n_props, uint64_t *mask, uint64_t *atoms, uint64_t stride, Ctrl *ctrl,
                        cudaStream_t s, uint64_t *keys, uint64_t seed, void *zero, uint64_t n_zero16) {
    const int th = 256;
    pack_kernel<<<pack_blocks(plane * (uint64_t)Wt, zero ? n_zero16 : 0, th), th, 0, s>>>(
        letters, offsets, n_traces, plane, W, Wt, n_props, mask, atoms, stride, ctrl, keys, seed, (uint4 *)zero,
        zero ? n_zero16 : 0);
    return cudaGetLastError();
}

cudaError_t launch_pack_narrow(const uint32_t *letters, const uint64_t *offsets, uint32_t n_traces, uint64_t plane,
                               int n_props, uint64_t *mask, uint64_t *atoms, uint64_t stride, Ctrl *ctrl,
                               cudaStream_t s, uint64_t *keys, uint64_t seed, void *zero, uint64_t n_zero16) {
    const int th = 256;
    pack_narrow_kernel<<<pack_blocks(plane, zero ? n_zero16 : 0, th), th, 0, s>>>(
        letters, offsets, n_traces, plane, n_props, mask, atoms, stride, ctrl, keys, seed, (uint4 *)zero,
        zero ? n_zero16 : 0);
    return cudaGetLastError();
}

cudaError_t launch_walk_batch(const WalkJob *jobs, int n_jobs, uint32_t *tokens, int cap, int *n_out, cudaStream_t s) {
    if (n_jobs <= 0) return cudaSuccess;
    const int th = 64;
    walk_batch_kernel<<<(n_jobs + th - 1) / th, th, 0, s>>>(jobs, n_jobs, tokens, cap, n_out);
    return cudaGetLastError();
}

cudaError_t launch_eval(int W, const uint32_t *prog, int n_instr, const uint64_t *atoms, const uint64_t *mask,
                        uint64_t stride, uint64_t plane, uint64_t *stack, int nsteps, uint32_t n_traces,
                        uint64_t *out, int out_words, cudaStream_t s) {
    const int th = 128;
    const unsigned grid = (unsigned)((plane + th - 1) / th);
#define LTL_EVAL_CASE(WW)                                                                                   \
    case WW:                                                                                                \
        eval_kernel<WW><<<grid, th, 0, s>>>(prog, n_instr, atoms, mask, stride, plane, stack, nsteps, n_traces, \
                                            out, out_words);                                                \
        break;
    switch (W) {
        LTL_EVAL_CASE(1)
        LTL_EVAL_CASE(2)
        LTL_EVAL_CASE(4)
        LTL_EVAL_CASE(8)
        LTL_EVAL_CASE(16)
    default:
        return cudaErrorInvalidValue;
    }
#undef LTL_EVAL_CASE
    return cudaGetLastError();
}

cudaError_t launch_unpack(const uint64_t *src, uint64_t plane, int W, uint32_t n_traces, uint64_t *out,
                          int out_words, cudaStream_t s) {
    const int th = 256;
    unpack_kernel<<<(n_traces + th - 1) / th, th, 0, s>>>(src, plane, W, n_traces, out, out_words);
    return cudaGetLastError();
}

}  // namespace ltl
