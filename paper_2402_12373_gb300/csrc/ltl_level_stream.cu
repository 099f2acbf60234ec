// ltl_level_stream.cu -- the size-level candidate kernel for characteristic
// matrices larger than one CTA holds in registers (more than 4096 / W traces).
//
// The matrix is cut into `groups` chunk groups.  Pass 1 streams the operands
// group by group, computing the NH fingerprint and the position-0 soundness
// bits without keeping the matrix; after the hash probe, pass 2 recomputes
// each group and either stores it (new entry) or compares it with the stored
// entry of equal fingerprint.
//
// The operands -- with the length mask of Not and G and, in pass 1, the NH
// fingerprint keys -- reach shared memory through a per-thread double-buffered
// ring (cp.async, 16 bytes per copy): every thread copies exactly the 16-byte
// pieces it will compute on, so a thread waits only for its own copies and no
// barrier guards the ring.  The pipeline runs across pass 1, the probe and
// pass 2 (pass 2's first group is requested before the probe), so the next
// group's loads are in flight while the registers hold the current one.
//
// Once the problem's cache is full, a candidate is only tested for
// separation: nothing can be stored, so it needs no fingerprint (no keys are
// staged and no NH term is computed), no probe and no second pass.
#include "ltl_level_common.cuh"

namespace ltl {
namespace lvl {
namespace {

constexpr int kStreamStages = 2;   // ring slots (groups in flight + the one being read)
constexpr int kStreamPieces = 3;   // per slot: left operand; right operand or length mask; NH keys
// Once the cache is full a candidate needs no keys: the same ring holds three
// slots of two pieces, one more group in flight.
constexpr int kCappedStages = 3;
constexpr int kCappedPieces = 2;
static_assert(kCappedStages * kCappedPieces == kStreamStages * kStreamPieces, "both rings fill the same memory");

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// A thread's 16-byte pieces of one group, in ring slot `stage`: piece
// (kind o, chunk c, plane w) of thread tid at
// ring[((stage * kStreamPieces + o) * C + c) * W + w][tid] (consecutive threads
// 16 bytes apart, so shared-memory accesses are conflict-free).  Kinds: 0 the
// left (or only) operand, 1 the right operand of a binary connective or the
// length mask of Not and G, 2 the NH fingerprint keys (pass 1 only).
template <int W, int C, int P = kStreamPieces>
__device__ __forceinline__ ulonglong2 *ring_piece(ulonglong2 *ring, int stage, int o, int c, int w, int NT, int tid) {
    return ring + ((((uint64_t)stage * P + o) * C + c) * W + w) * (uint64_t)NT + tid;
}

template <int W, int C, int OP, int P = kStreamPieces>
__device__ __forceinline__ void stage_group(const Problem &pb, const uint64_t *A, const uint64_t *B, uint32_t g,
                                            bool keys, int NT, int tid, ulonglong2 *ring, int stage) {
    constexpr bool BIN = is_binary(OP);
    constexpr bool MASKED = (OP == OP_NOT || OP == OP_G);
    const uint64_t cs = 2ull * (uint64_t)NT;
    const uint64_t toff = 2ull * ((uint64_t)g * C * NT + (uint64_t)tid);
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t off = (uint64_t)w * pb.plane + toff + c * cs;
            cp_async16(ring_piece<W, C, P>(ring, stage, 0, c, w, NT, tid), A + off);
            if (BIN) cp_async16(ring_piece<W, C, P>(ring, stage, 1, c, w, NT, tid), B + off);
            if (MASKED) cp_async16(ring_piece<W, C, P>(ring, stage, 1, c, w, NT, tid), pb.mask + off);
            if (P > 2 && keys) cp_async16(ring_piece<W, C, P>(ring, stage, 2, c, w, NT, tid), pb.keys + off);
        }
    cp_async_commit();
}

// Pieces of kind o into a fragment.
template <int W, int C, int P = kStreamPieces>
__device__ __forceinline__ void read_piece(ulonglong2 *ring, int stage, int o, int NT, int tid, Frag<W, C> &f) {
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const ulonglong2 q = *ring_piece<W, C, P>(ring, stage, o, c, w, NT, tid);
            f.v[c][0][w] = q.x;
            f.v[c][1][w] = q.y;
        }
}

struct StreamShared {
    unsigned long long fp[32];
    uint32_t err[32];
    unsigned long long tile;
    int skip;
    int found_seen;   // the tile's problem had a recorded separator when the tile was taken
    int capped;       // the problem's cache was full when the last decision was taken
    unsigned long long idx;
    unsigned long long h;
    int dec;
};

// The connective on one group, from ring slot `stage` (x: left or only
// operand; r: the right operand of a binary connective, the result on exit).
template <int OP, int W, int C, int P = kStreamPieces>
__device__ __forceinline__ void stream_compute(const Problem &pb, ulonglong2 *ring, int stage, int NT, int tid,
                                               Frag<W, C> &x, Frag<W, C> &r) {
    constexpr bool BIN = is_binary(OP);
    constexpr bool MASKED = (OP == OP_NOT || OP == OP_G);
    Frag<W, C> m;
    read_piece<W, C, P>(ring, stage, 0, NT, tid, x);
    if (BIN) read_piece<W, C, P>(ring, stage, 1, NT, tid, r);
    if (MASKED) read_piece<W, C, P>(ring, stage, 1, NT, tid, m);
    apply_op<OP, W, C>(r, x, m, pb.nsteps, pb.logstep != 0);
}

template <int W, int C, int OP>
__device__ __forceinline__ void stream_candidate(const Problem &pb, int level, uint64_t a, uint64_t b,
                                                 StreamShared &sh, int NT, int tid, ulonglong2 *ring) {
    constexpr bool BIN = is_binary(OP);
    const uint64_t *A = ((OP == OP_ATOM) ? pb.atoms : pb.arena) + a * pb.stride;
    const uint64_t *B = pb.arena + b * pb.stride;
    const uint32_t G = pb.groups;
    const uint64_t cs = 2ull * (uint64_t)NT;
    // a full cache (seen before this candidate) leaves only the soundness test
    const bool capped = sh.capped != 0;
    const bool nh = !capped && pb.ruc != RUC_FKP;
    // group sequence: pass 1 (i < G), then pass 2 (i - G); slot i % kStreamStages
    const uint32_t total = capped ? G : 2 * G;
    auto stage = [&](uint32_t i) {
        if (i < total)
            stage_group<W, C, OP>(pb, A, B, i % G, i < G && nh, NT, tid, ring, (int)(i % kStreamStages));
        else cp_async_commit();   // an empty group keeps the wait counts uniform
    };
    for (uint32_t i = 0; i < kStreamStages - 1; ++i) stage(i);
    Frag<W, C> x, r;
    uint64_t fp = 0;
    uint32_t nerr = 0;
    for (uint32_t g = 0; g < G; ++g) {
        const uint64_t toff = 2ull * ((uint64_t)g * C * NT + (uint64_t)tid);
        cp_async_wait<kStreamStages - 2>();   // this thread's pieces of group g have landed
        const int sl = (int)(g % kStreamStages);
        stage(g + kStreamStages - 1);         // into the slot group g - 1 used, read before
        stream_compute<OP, W, C>(pb, ring, sl, NT, tid, x, r);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (capped) {
            } else if (nh) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const ulonglong2 k = *ring_piece<W, C>(ring, sl, 2, c, w, NT, tid);
                    fp += nh_term(r.v[c][0][w], k.x) + nh_term(r.v[c][1][w], k.y);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 2; ++j) fp += fkp_word<false>(r.v[c][j][0], toff + c * cs + j, pb.fkp_b);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint64_t t = toff + c * cs + (uint64_t)j;
                const bool v = (r.v[c][j][0] & 1ull) != 0;
                nerr += ((t < pb.n_traces) && (v != (t < pb.n_pos))) ? 1u : 0u;
            }
        }
    }
    fp = warp_sum_u64(fp);
    nerr = __reduce_add_sync(0xffffffffu, nerr);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        sh.fp[warp] = fp;
        sh.err[warp] = nerr;
    }
    __syncthreads();
    const uint64_t prov = prov_pack(OP, a, BIN ? b : 0);
    unsigned long long key = 0;
    if (tid == 0) {
        uint64_t s = 0;
        uint32_t total_err = 0;
        for (int w2 = 0; w2 < (NT >> 5); ++w2) {
            s += sh.fp[w2];
            total_err += sh.err[w2];
        }
        if (total_err <= pb.max_errors && !sh.found_seen) record_separator(pb, level, prov);   // eq. (dagger), or noisy
        unsigned long long h0 = 0;
        key = admission_key(pb, s, h0);
        sh.h = h0;
    }
    for (uint32_t pass2 = 0;; ++pass2) {
        if (tid == 0) {
            unsigned long long h = sh.h, idx = 0;
            // Once the cache is full nothing more is stored: the candidate has
            // been checked for separation above, and whether it duplicates an
            // entry no longer matters, so neither the probe nor the second
            // pass (the compare) is run.
            const int cap = capped || ld_volatile_i32(&pb.ctrl->cap_hit);
            sh.capped = cap;
            sh.dec = cap ? (int)DEC_FAIL : probe<true>(pb, key, h, idx, false);
            sh.idx = idx;
            sh.h = h;
        }
        __syncthreads();
        const int d = sh.dec;
        if (d != DEC_NEW && d != DEC_CMP) break;   // cache full (candidate still tested) or error
        if (pass2 > 0) {   // probing on after a collision: pass 2 again, from a fresh pipeline
            cp_async_wait_all();
            for (uint32_t i = G; i < G + kStreamStages - 1; ++i) stage(i);
        }
        uint64_t *ent = pb.arena + sh.idx * pb.stride;
        bool eq = true;
        for (uint32_t g = 0; g < G; ++g) {
            const uint32_t i = G + g;
            const uint64_t toff = 2ull * ((uint64_t)g * C * NT + (uint64_t)tid);
            cp_async_wait<kStreamStages - 2>();
            const int sl = (int)(i % kStreamStages);
            stage(i + kStreamStages - 1);
            stream_compute<OP, W, C>(pb, ring, sl, NT, tid, x, r);
            if (d == DEC_NEW) store_frag<W, C>(r, ent, pb.plane, toff, cs);
            else eq &= equal_frag<W, C>(r, ent, pb.plane, toff, cs);
        }
        if (d == DEC_NEW) {
            __syncthreads();
            if (tid == 0) {
                pb.prov[sh.idx] = prov;
                slot_publish(pb, sh.h, key, sh.idx);
            }
            break;
        }
        const int all_eq = __syncthreads_and(eq);
        if (tid == 0) atomicAdd(&pb.ctrl->compares, 1ull);
        if (all_eq) break;
        if (tid == 0) {
            atomicAdd(&pb.ctrl->collisions, 1ull);
            sh.h = (sh.h + 1) & pb.hmask;
        }
    }
    cp_async_wait_all();   // no copy of this candidate is left in flight into the ring
    __syncthreads();
}

// A candidate once the problem's cache is full: only its soundness (eq.
// (dagger), or the noisy variant) is tested -- nothing can be stored, so it
// needs no fingerprint, no probe and no second pass -- with one more group of
// operands in flight than the two-pass ring holds.
template <int W, int C, int OP>
__device__ __forceinline__ void stream_candidate_capped(const Problem &pb, int level, uint64_t a, uint64_t b,
                                                        StreamShared &sh, int NT, int tid, ulonglong2 *ring) {
    constexpr bool BIN = is_binary(OP);
    constexpr int ST = kCappedStages, P = kCappedPieces;
    const uint64_t *A = ((OP == OP_ATOM) ? pb.atoms : pb.arena) + a * pb.stride;
    const uint64_t *B = pb.arena + b * pb.stride;
    const uint32_t G = pb.groups;
    const uint64_t cs = 2ull * (uint64_t)NT;
    auto stage = [&](uint32_t i) {
        if (i < G) stage_group<W, C, OP, P>(pb, A, B, i, false, NT, tid, ring, (int)(i % ST));
        else cp_async_commit();   // an empty group keeps the wait counts uniform
    };
    for (uint32_t i = 0; i < ST - 1; ++i) stage(i);
    Frag<W, C> x, r;
    uint32_t nerr = 0;
    for (uint32_t g = 0; g < G; ++g) {
        const uint64_t toff = 2ull * ((uint64_t)g * C * NT + (uint64_t)tid);
        cp_async_wait<ST - 2>();   // this thread's pieces of group g have landed
        const int sl = (int)(g % ST);
        stage(g + ST - 1);         // into the slot group g - 1 used, read before
        stream_compute<OP, W, C, P>(pb, ring, sl, NT, tid, x, r);
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint64_t t = toff + c * cs + (uint64_t)j;
                const bool v = (r.v[c][j][0] & 1ull) != 0;
                nerr += ((t < pb.n_traces) && (v != (t < pb.n_pos))) ? 1u : 0u;
            }
    }
    nerr = __reduce_add_sync(0xffffffffu, nerr);
    if ((tid & 31) == 0) sh.err[tid >> 5] = nerr;
    __syncthreads();
    if (tid == 0) {
        uint32_t total_err = 0;
        for (int w2 = 0; w2 < (NT >> 5); ++w2) total_err += sh.err[w2];
        if (total_err <= pb.max_errors && !sh.found_seen) record_separator(pb, level, prov_pack(OP, a, BIN ? b : 0));
    }
    cp_async_wait_all();   // no copy of this candidate is left in flight into the ring
    __syncthreads();
}

template <int W, int C, int OP>
__device__ __forceinline__ unsigned long long stream_tile(const Problem &pb, int level, const Seg &sg, uint64_t a0,
                                                          uint64_t a1, uint64_t b0, uint64_t b1, StreamShared &sh,
                                                          int NT, int tid, ulonglong2 *ring) {
    constexpr bool BIN = is_binary(OP);
    unsigned long long n = 0;
    // sh.capped is read after the barrier that ends the previous candidate (or
    // the tile fetch), so every thread takes the same path
    auto one = [&](uint64_t a, uint64_t b) {
        if (sh.capped) stream_candidate_capped<W, C, OP>(pb, level, a, b, sh, NT, tid, ring);
        else stream_candidate<W, C, OP>(pb, level, a, b, sh, NT, tid, ring);
    };
    for (uint64_t i = a0; i < a1; ++i) {
        if (!BIN) {
            one(sg.a_begin + i, 0);
            ++n;
            continue;
        }
        const uint64_t jb = (sg.kind == SEG_TRI) ? max(b0, i + 1) : b0;
        for (uint64_t j = jb; j < b1; ++j) {
            one(sg.a_begin + i, sg.b_begin + j);
            ++n;
        }
    }
    return n;
}

}  // namespace

// Dynamic shared memory: the ring, kStreamStages x kStreamPieces x C x W pieces of
// 16 bytes per thread (stream_smem_bytes).
template <int W, int C>
__global__ void __launch_bounds__(256) stream_level_kernel(LevelArgs la) {
    __shared__ StreamShared sh;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    ulonglong2 *ring = reinterpret_cast<ulonglong2 *>(dyn_smem);
    const int tid = threadIdx.x, NT = blockDim.x;
    uint32_t dsmem;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsmem));
    for (;;) {
        if (tid == 0) {
            const unsigned long long t = atomicAdd(la.tile_counter, 1ull);
            int skip = 1, found = 0, cap = 0;
            if (t < la.total_tiles) {
                const Ctrl *ctrl = la.probs[la.segs[find_segment(la, t)].prob].ctrl;
                skip = ld_volatile_i32(&ctrl->stop);
                found = ld_volatile_i32(reinterpret_cast<const int *>(&ctrl->found_count));
                cap = ld_volatile_i32(&ctrl->cap_hit);
            }
            // the ring must fit the launch's dynamic shared memory
            if (!skip && (uint64_t)dsmem < (uint64_t)kStreamStages * kStreamPieces * C * W * 16 * (uint64_t)NT) {
                atomicCAS(&la.probs[la.segs[find_segment(la, t)].prob].ctrl->err, 0, -1 /* LTL_ERR_INVALID */);
                skip = 1;
            }
            sh.tile = t;
            sh.skip = skip;
            sh.found_seen = found;
            sh.capped = cap;
        }
        __syncthreads();
        const unsigned long long tile = sh.tile;
        const int skip = sh.skip;
        __syncthreads();
        if (tile >= la.total_tiles) break;
        if (skip) continue;
        const Seg sg = la.segs[find_segment(la, tile)];
        const Problem pb = la.probs[sg.prob];
        uint64_t a0, a1, b0, b1;
        decode_tile(sg, tile - sg.tile_begin, a0, a1, b0, b1);
        unsigned long long done = 0;
        switch (sg.op) {
#define LTL_STREAM_CASE(OPV) \
    case OPV: done = stream_tile<W, C, OPV>(pb, sg.level, sg, a0, a1, b0, b1, sh, NT, tid, ring); break;
            LTL_STREAM_CASE(OP_ATOM)
            LTL_STREAM_CASE(OP_NOT)
            LTL_STREAM_CASE(OP_AND)
            LTL_STREAM_CASE(OP_OR)
            LTL_STREAM_CASE(OP_X)
            LTL_STREAM_CASE(OP_F)
            LTL_STREAM_CASE(OP_G)
            LTL_STREAM_CASE(OP_U)
#undef LTL_STREAM_CASE
        default: break;
        }
        if (tid == 0 && done) atomicAdd(&pb.ctrl->cands, done);
    }
}

}  // namespace lvl

template <int W, int C>
static const void *stream_fn() {
    return reinterpret_cast<const void *>(&lvl::stream_level_kernel<W, C>);
}

// Dynamic shared memory of the streaming kernel's operand ring.
size_t stream_smem_bytes(int W, int C, int NT) {
    return (size_t)lvl::kStreamStages * lvl::kStreamPieces * (size_t)C * (size_t)W * 16 * (size_t)NT;
}

// Streaming shapes: C * W == 8 words per thread, 128 threads per CTA.
const void *stream_kernel_ptr(int W, int C) {
    switch (W * 16 + C) {
    case 1 * 16 + 8: return stream_fn<1, 8>();
    case 2 * 16 + 4: return stream_fn<2, 4>();
    case 4 * 16 + 2: return stream_fn<4, 2>();
    case 8 * 16 + 1: return stream_fn<8, 1>();
    default: return nullptr;
    }
}

}  // namespace ltl
