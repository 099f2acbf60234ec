// ltl_kernels.cu -- sm_103a kernels of the enumerative LTL learner.
//
// Layout in HBM (one learning problem):
//   characteristic matrix (CM) = W bit-planes of `plane` uint64 words; word t
//   of plane w holds positions 64w..64w+63 of trace t (plane >= |P|+|N| is a
//   multiple of 2 * threads * chunks; padding traces are all zero).
//   arena   : entries x stride words (stride = W * plane), append-only,
//             size levels stored as contiguous index ranges.
//   prov    : one packed (op, left, right) word per entry.
//   hkeys / hvals : open-addressing hash set, linear probing; a slot holds
//             a 64-bit fingerprint and the index of the entry it stands for.
//
// Thread mapping of a CTA working on one candidate: thread `tid` owns, in
// chunk c of group g, traces t0 = 2 * ((g * C + c) * NT + tid) and t0 + 1 in
// every plane (one 16-byte load per plane and chunk, coalesced across the
// warp).  With one group (groups == 1) the whole candidate CM lives in
// registers from its computation until it is written or compared; with
// more groups the CM is recomputed group by group in the second pass.
#include <cuda_runtime.h>

#include <cstdint>

#include "ltl_device.cuh"
#include "ltl_types.h"

namespace ltl {

namespace {

__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(volatile const int *)p; }

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    return *(volatile const unsigned long long *)p;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int W, int C>
struct Frag {
    uint64_t v[C][2][W];   // [chunk][trace of the pair][word]
};

__device__ __forceinline__ uint64_t pair_base(uint32_t g, int C, int c, int NT, int tid) {
    return 2ull * ((uint64_t)(g * (uint32_t)C + (uint32_t)c) * (uint64_t)NT + (uint64_t)tid);
}

// Read-only operand loads (entries of earlier levels: never written by this
// launch) go through the non-coherent read-only path.
template <int W, int C>
__device__ __forceinline__ void load_ro(const uint64_t *__restrict__ base, uint64_t plane, uint32_t g,
                                       int NT, int tid, Frag<W, C> &f) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint64_t t0 = pair_base(g, C, c, NT, tid);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2 *>(base + (uint64_t)w * plane + t0));
            f.v[c][0][w] = q.x;
            f.v[c][1][w] = q.y;
        }
    }
}

template <int W, int C>
__device__ __forceinline__ void compute_group(int op, const uint64_t *__restrict__ A,
                                              const uint64_t *__restrict__ B, const Problem &pb,
                                              uint32_t g, int NT, int tid, Frag<W, C> &r) {
    switch (op) {
    case OP_ATOM:
        load_ro<W, C>(A, pb.plane, g, NT, tid, r);
        break;
    case OP_NOT: {
        Frag<W, C> m;
        load_ro<W, C>(A, pb.plane, g, NT, tid, r);
        load_ro<W, C>(pb.mask, pb.plane, g, NT, tid, m);
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int w = 0; w < W; ++w) r.v[c][j][w] = m.v[c][j][w] & ~r.v[c][j][w];
        break;
    }
    case OP_X:
        load_ro<W, C>(A, pb.plane, g, NT, tid, r);
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) op_x<W>(r.v[c][j]);
        break;
    case OP_F:
        load_ro<W, C>(A, pb.plane, g, NT, tid, r);
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) op_f<W>(r.v[c][j], pb.nsteps);
        break;
    case OP_G: {
        Frag<W, C> m;
        load_ro<W, C>(A, pb.plane, g, NT, tid, r);
        load_ro<W, C>(pb.mask, pb.plane, g, NT, tid, m);
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) op_g<W>(r.v[c][j], m.v[c][j], pb.nsteps);
        break;
    }
    case OP_AND:
    case OP_OR: {
        Frag<W, C> b;
        load_ro<W, C>(A, pb.plane, g, NT, tid, r);
        load_ro<W, C>(B, pb.plane, g, NT, tid, b);
        if (op == OP_AND) {
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int w = 0; w < W; ++w) r.v[c][j][w] &= b.v[c][j][w];
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int w = 0; w < W; ++w) r.v[c][j][w] |= b.v[c][j][w];
        }
        break;
    }
    case OP_U: {
        Frag<W, C> a;
        load_ro<W, C>(A, pb.plane, g, NT, tid, a);
        load_ro<W, C>(B, pb.plane, g, NT, tid, r);
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) op_u<W>(a.v[c][j], r.v[c][j], pb.nsteps);
        break;
    }
    default:
        break;
    }
}

// NH fingerprint partial sum and the soundness test of eq. (dagger) on this
// thread's traces: every positive must hold at position 0, every negative not.
template <int W, int C>
__device__ __forceinline__ void digest_group(const Frag<W, C> &r, const Problem &pb, uint32_t g, int NT,
                                             int tid, uint64_t &fp, bool &bad) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint64_t t0 = pair_base(g, C, c, NT, tid);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const ulonglong2 k = __ldg(reinterpret_cast<const ulonglong2 *>(pb.keys + (uint64_t)w * pb.plane + t0));
            fp += nh_term(r.v[c][0][w], k.x) + nh_term(r.v[c][1][w], k.y);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint64_t t = t0 + (uint64_t)j;
            const bool v = (r.v[c][j][0] & 1ull) != 0;
            const bool want = t < pb.n_pos;
            bad |= (t < pb.n_traces) && (v != want);
        }
    }
}

template <int W, int C>
__device__ __forceinline__ void store_group(const Frag<W, C> &r, uint64_t *dst, uint64_t plane, uint32_t g,
                                            int NT, int tid) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint64_t t0 = pair_base(g, C, c, NT, tid);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            ulonglong2 q;
            q.x = r.v[c][0][w];
            q.y = r.v[c][1][w];
            *reinterpret_cast<ulonglong2 *>(dst + (uint64_t)w * plane + t0) = q;
        }
    }
}

// Entries written during this launch are read through L2 only (ld.cg):
// they were published by other CTAs after this SM may have started.
template <int W, int C>
__device__ __forceinline__ bool equal_group(const Frag<W, C> &r, const uint64_t *src, uint64_t plane,
                                            uint32_t g, int NT, int tid) {
    bool eq = true;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const uint64_t t0 = pair_base(g, C, c, NT, tid);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const ulonglong2 q = __ldcg(reinterpret_cast<const ulonglong2 *>(src + (uint64_t)w * plane + t0));
            eq &= (q.x == r.v[c][0][w]) & (q.y == r.v[c][1][w]);
        }
    }
    return eq;
}

enum : int { DEC_NEW = 0, DEC_CMP = 1, DEC_FAIL = 2, DEC_ERR = 3 };

// One probe run by a single thread, starting at slot h: claims an empty
// slot (DEC_NEW, with a freshly allocated entry index), or stops at a slot
// holding the same fingerprint (DEC_CMP, with the entry to compare against,
// waiting a bounded time for a pending publication).
__device__ int probe(const Problem &pb, unsigned long long key, unsigned long long &h, unsigned long long &idx) {
    for (unsigned long long n = 0; n <= pb.hmask; ++n) {
        unsigned long long k = ld_volatile_u64(pb.hkeys + h);
        if (k == 0ull) {
            k = atomicCAS(pb.hkeys + h, 0ull, key);
            if (k == 0ull) {
                const unsigned long long i = atomicAdd(&pb.ctrl->n_entries, 1ull);
                if (i >= pb.max_entries) {
                    st_release_u32(pb.hvals + h, kValFail);
                    atomicExch(&pb.ctrl->cap_hit, 1);
                    return DEC_FAIL;
                }
                idx = i;
                return DEC_NEW;
            }
        }
        if (k == key) {
            uint32_t v;
            unsigned long long spins = 0;
            while ((v = ld_acquire_u32(pb.hvals + h)) == kValPending) {
                if (++spins > pb.spin_limit) {
                    atomicAdd(&pb.ctrl->timeouts, 1ull);
                    atomicCAS(&pb.ctrl->err, 0, -4 /* LTL_ERR_TIMEOUT */);
                    atomicExch(&pb.ctrl->stop, 1);
                    return DEC_ERR;
                }
                __nanosleep(64);
            }
            if (v == kValFail) return DEC_FAIL;
            idx = v;
            return DEC_CMP;
        }
        h = (h + 1) & pb.hmask;
    }
    atomicExch(&pb.ctrl->cap_hit, 1);   // table full
    return DEC_FAIL;
}

struct Shared {
    unsigned long long fp[32];
    int bad[32];
    unsigned long long tile;
    unsigned long long idx;
    unsigned long long h;
    int dec;
};

// Check-and-cache of one candidate (Section 3): build it, test soundness,
// then admit it to the cache iff no equal matrix is there yet.
template <int W, int C>
__device__ __forceinline__ void process(const Problem &pb, int level, int op, uint64_t a, uint64_t b,
                                        Shared &sh, int NT, int tid) {
    const uint64_t *A = (op == OP_ATOM ? pb.atoms : pb.arena) + a * pb.stride;
    const uint64_t *B = pb.arena + b * pb.stride;
    const uint32_t G = pb.groups;
    Frag<W, C> r;
    uint64_t fp = 0;
    bool bad = false;
    for (uint32_t g = 0; g < G; ++g) {
        compute_group<W, C>(op, A, B, pb, g, NT, tid, r);
        digest_group<W, C>(r, pb, g, NT, tid, fp, bad);
    }
    // CTA reduction of the fingerprint (sum mod 2^64) and of the soundness test
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) fp += __shfl_xor_sync(0xffffffffu, fp, off);
    bad = __any_sync(0xffffffffu, bad);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        sh.fp[warp] = fp;
        sh.bad[warp] = bad;
    }
    __syncthreads();
    const uint64_t prov = prov_pack(op, a, op == OP_AND || op == OP_OR || op == OP_U ? b : 0);
    unsigned long long key = 0;
    if (tid == 0) {
        uint64_t s = 0;
        int anybad = 0;
        for (int w2 = 0; w2 < (NT >> 5); ++w2) {
            s += sh.fp[w2];
            anybad |= sh.bad[w2];
        }
        if (!anybad) {   // a separating formula: record the first one
            if (atomicAdd(&pb.ctrl->found_count, 1u) == 0u) {
                pb.ctrl->found_prov = prov;
                pb.ctrl->found_level = level;
            }
            if (pb.stop_first) atomicExch(&pb.ctrl->stop, 1);
        }
        key = mix64(s);
        if (key == 0ull) key = 1ull;
        sh.h = key & pb.hmask;
    }
    // probe / compare / append
    for (;;) {
        if (tid == 0) {
            unsigned long long h = sh.h, idx = 0;
            const int d = probe(pb, key, h, idx);
            sh.dec = d;
            sh.idx = idx;
            sh.h = h;
        }
        __syncthreads();
        const int d = sh.dec;
        if (d == DEC_NEW) {
            const uint64_t idx = sh.idx;
            uint64_t *dst = pb.arena + idx * pb.stride;
            for (uint32_t g = 0; g < G; ++g) {
                if (G > 1) compute_group<W, C>(op, A, B, pb, g, NT, tid, r);
                store_group<W, C>(r, dst, pb.plane, g, NT, tid);
            }
            if (tid == 0) pb.prov[idx] = prov;
            __threadfence();
            __syncthreads();
            if (tid == 0) st_release_u32(pb.hvals + sh.h, (uint32_t)idx);
            break;
        }
        if (d == DEC_CMP) {
            const uint64_t *src = pb.arena + sh.idx * pb.stride;
            bool eq = true;
            for (uint32_t g = 0; g < G; ++g) {
                if (G > 1) compute_group<W, C>(op, A, B, pb, g, NT, tid, r);
                eq &= equal_group<W, C>(r, src, pb.plane, g, NT, tid);
            }
            const int all_eq = __syncthreads_and(eq);
            if (tid == 0) atomicAdd(&pb.ctrl->compares, 1ull);
            if (all_eq) break;
            if (tid == 0) {
                atomicAdd(&pb.ctrl->collisions, 1ull);
                sh.h = (sh.h + 1) & pb.hmask;
            }
            continue;
        }
        break;   // cache full (candidate still tested) or error
    }
}

}  // namespace

template <int W, int C>
struct Bounds {
    static constexpr int kThreads = (W * C >= 8) ? 256 : (W * C >= 4) ? 512 : 1024;
    static constexpr int kMinBlocks = (W * C >= 8) ? 2 : 1;
};

// One launch per size level: a persistent grid pulls tiles of candidates
// from a counter and runs check-and-cache on each candidate.
template <int W, int C>
__global__ void __launch_bounds__(Bounds<W, C>::kThreads, Bounds<W, C>::kMinBlocks)
    level_kernel(Problem pb, LevelArgs la) {
    __shared__ Shared sh;
    const int tid = threadIdx.x, NT = blockDim.x;
    unsigned long long done = 0;
    for (;;) {
        if (tid == 0) {
            unsigned long long t = ~0ull;
            if (!ld_volatile_i32(&pb.ctrl->stop)) t = atomicAdd(&pb.ctrl->next_tile[la.level], 1ull);
            sh.tile = t;
        }
        __syncthreads();
        const unsigned long long tile = sh.tile;
        __syncthreads();
        if (tile >= la.total_tiles) break;
        int si = 0;
        while (si + 1 < la.n_segs && la.segs[si + 1].tile_begin <= tile) ++si;
        const Seg sg = la.segs[si];
        const uint64_t k = tile - sg.tile_begin;
        if (sg.kind == SEG_UNARY) {
            const uint64_t a0 = k * kTileU;
            const uint64_t a1 = min(a0 + kTileU, sg.a_count);
            for (uint64_t i = a0; i < a1; ++i) {
                process<W, C>(pb, la.level, sg.op, sg.a_begin + i, 0, sh, NT, tid);
                ++done;
            }
        } else {
            uint64_t ta, tb;
            if (sg.kind == SEG_RECT) {
                if (sg.a_inner) { ta = k % sg.n_ta; tb = k / sg.n_ta; }
                else { tb = k % sg.n_tb; ta = k / sg.n_tb; }
            } else {
                // upper-triangular tiles (ta <= tb), row-major: row ta holds n - ta tiles
                const double n = (double)sg.n_ta;
                double est = ((2.0 * n + 1.0) - sqrt((2.0 * n + 1.0) * (2.0 * n + 1.0) - 8.0 * (double)k)) * 0.5;
                int64_t r = (int64_t)est;
                if (r < 0) r = 0;
                auto row_start = [&](int64_t x) -> int64_t { return x * (int64_t)sg.n_ta - x * (x - 1) / 2; };
                while (r > 0 && row_start(r) > (int64_t)k) --r;
                while (row_start(r + 1) <= (int64_t)k) ++r;
                ta = (uint64_t)r;
                tb = ta + ((uint64_t)k - (uint64_t)row_start(r));
            }
            const uint64_t a0 = ta * kTileA, a1 = min(a0 + kTileA, sg.a_count);
            const uint64_t b0 = tb * kTileB, b1 = min(b0 + kTileB, sg.b_count);
            for (uint64_t i = a0; i < a1; ++i) {
                for (uint64_t j = b0; j < b1; ++j) {
                    if (sg.kind == SEG_TRI && j <= i) continue;
                    process<W, C>(pb, la.level, sg.op, sg.a_begin + i, sg.b_begin + j, sh, NT, tid);
                    ++done;
                }
            }
        }
    }
    if (tid == 0 && done) atomicAdd(&pb.ctrl->cands, done);
}

// ---------------------------------------------------------------------------
// Trace packing: length masks and the atoms' characteristic matrices.  One
// thread per (plane w, trace slot t).  Positions are read straight from the
// concatenated letters; a letter with a bit >= n_props, a decreasing offset
// or a trace longer than 64 * W marks the input invalid.
// ---------------------------------------------------------------------------
__global__ void pack_kernel(const uint32_t *__restrict__ letters, const uint64_t *__restrict__ offsets,
                            uint32_t n_traces, uint64_t plane, int W, int n_props, uint64_t *mask,
                            uint64_t *atoms, uint64_t stride, Ctrl *ctrl) {
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= plane * (uint64_t)W) return;
    const uint64_t t = idx % plane, w = idx / plane;
    uint64_t off = 0, len = 0;
    if (t < n_traces) {
        off = offsets[t];
        const uint64_t end = offsets[t + 1];
        if (end < off || (t == 0 && off != 0)) {
            atomicExch(&ctrl->invalid_letter, 1);
            return;
        }
        len = end - off;
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

// NH keys, one per word of a matrix: SplitMix64 outputs of a fixed seed.
__global__ void keys_kernel(uint64_t *keys, uint64_t n, uint64_t seed) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

// ---------------------------------------------------------------------------
// Provenance walk: the syntax tree of a cache entry (or of the recorded
// separator) as a pre-order token list, op | (atom index << 8).  One thread.
// ---------------------------------------------------------------------------
__global__ void walk_kernel(const uint64_t *prov, uint64_t n_entries, uint64_t root_prov, uint32_t *tokens,
                            int cap, int *n_out) {
    uint64_t stack[2 * kMaxLevels + 2];
    int sp = 0, n = 0;
    bool ok = true;
    stack[sp++] = root_prov;
    while (sp > 0 && n < cap && ok) {
        const uint64_t p = stack[--sp];
        const int op = prov_op(p);
        if (op > OP_U) { ok = false; break; }
        tokens[n++] = (uint32_t)op | ((uint32_t)(op == OP_ATOM ? prov_a(p) : 0) << 8);
        if (op == OP_ATOM) continue;
        const bool binary = op == OP_AND || op == OP_OR || op == OP_U;
        if (prov_a(p) >= n_entries || (binary && prov_b(p) >= n_entries) || sp + 2 > 2 * kMaxLevels + 2) {
            ok = false;
            break;
        }
        if (binary) stack[sp++] = prov[prov_b(p)];   // pushed first: visited after the left subtree
        stack[sp++] = prov[prov_a(p)];
    }
    *n_out = (ok && sp == 0) ? n : -1;
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

template <int W, int C>
static const void *level_fn() { return reinterpret_cast<const void *>(&level_kernel<W, C>); }

const void *level_kernel_ptr(int W, int C) {
    switch (W * 16 + C) {
    case 1 * 16 + 1: return level_fn<1, 1>();
    case 1 * 16 + 2: return level_fn<1, 2>();
    case 1 * 16 + 4: return level_fn<1, 4>();
    case 1 * 16 + 8: return level_fn<1, 8>();
    case 2 * 16 + 1: return level_fn<2, 1>();
    case 2 * 16 + 2: return level_fn<2, 2>();
    case 2 * 16 + 4: return level_fn<2, 4>();
    case 4 * 16 + 1: return level_fn<4, 1>();
    case 4 * 16 + 2: return level_fn<4, 2>();
    case 8 * 16 + 1: return level_fn<8, 1>();
    default: return nullptr;
    }
}

int level_kernel_max_threads(int W, int C) {
    switch (W * C) {
    case 8: return Bounds<1, 8>::kThreads;
    case 4: return Bounds<1, 4>::kThreads;
    default: return Bounds<1, 1>::kThreads;
    }
}

cudaError_t launch_level(int W, int C, int grid, int threads, const Problem &pb, const LevelArgs &la,
                         cudaStream_t s) {
    const void *fn = level_kernel_ptr(W, C);
    if (!fn) return cudaErrorInvalidValue;
    Problem p = pb;
    LevelArgs l = la;
    void *args[] = {&p, &l};
    return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, 0, s);
}

cudaError_t launch_pack(const uint32_t *letters, const uint64_t *offsets, uint32_t n_traces, uint64_t plane,
                        int W, int n_props, uint64_t *mask, uint64_t *atoms, uint64_t stride, Ctrl *ctrl,
                        cudaStream_t s) {
    const uint64_t n = plane * (uint64_t)W;
    const int th = 256;
    pack_kernel<<<(unsigned)((n + th - 1) / th), th, 0, s>>>(letters, offsets, n_traces, plane, W, n_props, mask,
                                                             atoms, stride, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_keys(uint64_t *keys, uint64_t n, uint64_t seed, cudaStream_t s) {
    const int th = 256;
    keys_kernel<<<(unsigned)((n + th - 1) / th), th, 0, s>>>(keys, n, seed);
    return cudaGetLastError();
}

cudaError_t launch_walk(const uint64_t *prov, uint64_t n_entries, uint64_t root_prov, uint32_t *tokens, int cap,
                        int *n_out, cudaStream_t s) {
    walk_kernel<<<1, 1, 0, s>>>(prov, n_entries, root_prov, tokens, cap, n_out);
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
