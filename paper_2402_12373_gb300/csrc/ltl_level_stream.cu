// ltl_level_stream.cu -- the size-level candidate kernel for characteristic
// matrices larger than one CTA holds in registers (more than 4096 / W traces).
//
// The matrix is cut into `groups` chunk groups.  Pass 1 streams the operands
// group by group (coalesced 16-byte loads), computing the NH fingerprint and
// the position-0 soundness bits without keeping the matrix; after the hash
// probe, pass 2 recomputes each group and either stores it (new entry) or
// compares it with the stored entry of equal fingerprint.
#include "ltl_level_common.cuh"

namespace ltl {
namespace lvl {
namespace {

struct StreamShared {
    unsigned long long fp[32];
    uint32_t err[32];
    unsigned long long tile;
    int skip;
    unsigned long long idx;
    unsigned long long h;
    int dec;
};

template <int OP, int W, int C>
__device__ __forceinline__ void stream_compute(const Problem &pb, const uint64_t *A, const uint64_t *B,
                                               uint64_t toff, uint64_t cs, Frag<W, C> &r) {
    constexpr bool BIN = is_binary(OP);
    constexpr bool MASKED = (OP == OP_NOT || OP == OP_G);
    Frag<W, C> x, m;
    load_frag<W, C, true>(A, pb.plane, toff, cs, x);
    if (BIN) load_frag<W, C, true>(B, pb.plane, toff, cs, r);
    if (MASKED) load_frag<W, C, true>(pb.mask, pb.plane, toff, cs, m);
    apply_op<OP, W, C>(r, x, m, pb.nsteps);
}

template <int W, int C, int OP>
__device__ __forceinline__ void stream_candidate(const Problem &pb, int level, uint64_t a, uint64_t b,
                                                 StreamShared &sh, int NT, int tid) {
    constexpr bool BIN = is_binary(OP);
    const uint64_t *A = ((OP == OP_ATOM) ? pb.atoms : pb.arena) + a * pb.stride;
    const uint64_t *B = pb.arena + b * pb.stride;
    const uint32_t G = pb.groups;
    const uint64_t cs = 2ull * (uint64_t)NT;
    Frag<W, C> r;
    uint64_t fp = 0;
    uint32_t nerr = 0;
    for (uint32_t g = 0; g < G; ++g) {
        const uint64_t toff = 2ull * ((uint64_t)g * C * NT + (uint64_t)tid);
        stream_compute<OP, W, C>(pb, A, B, toff, cs, r);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (pb.ruc != RUC_FKP) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const ulonglong2 k =
                        __ldg(reinterpret_cast<const ulonglong2 *>(pb.keys + (uint64_t)w * pb.plane + toff + c * cs));
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
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) fp += __shfl_xor_sync(0xffffffffu, fp, off);
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
        if (total_err <= pb.max_errors) record_separator(pb, level, prov);   // eq. (dagger), or noisy
        unsigned long long h0 = 0;
        key = admission_key(pb, s, h0);
        sh.h = h0;
    }
    for (;;) {
        if (tid == 0) {
            unsigned long long h = sh.h, idx = 0;
            // Once the cache is full nothing more is stored: the candidate has
            // been checked for separation above, and whether it duplicates an
            // entry no longer matters, so neither the probe nor the second
            // pass (the compare) is run.
            sh.dec = ld_volatile_i32(&pb.ctrl->cap_hit) ? (int)DEC_FAIL : probe<true>(pb, key, h, idx, false);
            sh.idx = idx;
            sh.h = h;
        }
        __syncthreads();
        const int d = sh.dec;
        if (d == DEC_NEW) {
            uint64_t *dst = pb.arena + sh.idx * pb.stride;
            for (uint32_t g = 0; g < G; ++g) {
                const uint64_t toff = 2ull * ((uint64_t)g * C * NT + (uint64_t)tid);
                stream_compute<OP, W, C>(pb, A, B, toff, cs, r);
                store_frag<W, C>(r, dst, pb.plane, toff, cs);
            }
            __syncthreads();
            if (tid == 0) {
                pb.prov[sh.idx] = prov;
                st_release_u32(pb.hvals + sh.h, (uint32_t)sh.idx);
            }
            break;
        }
        if (d == DEC_CMP) {
            const uint64_t *src = pb.arena + sh.idx * pb.stride;
            bool eq = true;
            for (uint32_t g = 0; g < G; ++g) {
                const uint64_t toff = 2ull * ((uint64_t)g * C * NT + (uint64_t)tid);
                stream_compute<OP, W, C>(pb, A, B, toff, cs, r);
                eq &= equal_frag<W, C>(r, src, pb.plane, toff, cs);
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
    __syncthreads();
}

template <int W, int C, int OP>
__device__ __forceinline__ unsigned long long stream_tile(const Problem &pb, int level, const Seg &sg, uint64_t a0,
                                                          uint64_t a1, uint64_t b0, uint64_t b1, StreamShared &sh,
                                                          int NT, int tid) {
    constexpr bool BIN = is_binary(OP);
    unsigned long long n = 0;
    for (uint64_t i = a0; i < a1; ++i) {
        if (!BIN) {
            stream_candidate<W, C, OP>(pb, level, sg.a_begin + i, 0, sh, NT, tid);
            ++n;
            continue;
        }
        const uint64_t jb = (sg.kind == SEG_TRI) ? max(b0, i + 1) : b0;
        for (uint64_t j = jb; j < b1; ++j) {
            stream_candidate<W, C, OP>(pb, level, sg.a_begin + i, sg.b_begin + j, sh, NT, tid);
            ++n;
        }
    }
    return n;
}

}  // namespace

template <int W, int C>
__global__ void __launch_bounds__(256) stream_level_kernel(LevelArgs la) {
    __shared__ StreamShared sh;
    const int tid = threadIdx.x, NT = blockDim.x;
    for (;;) {
        if (tid == 0) {
            const unsigned long long t = atomicAdd(la.tile_counter, 1ull);
            int skip = 1;
            if (t < la.total_tiles) skip = ld_volatile_i32(&la.probs[la.segs[find_segment(la, t)].prob].ctrl->stop);
            sh.tile = t;
            sh.skip = skip;
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
    case OPV: done = stream_tile<W, C, OPV>(pb, sg.level, sg, a0, a1, b0, b1, sh, NT, tid); break;
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
