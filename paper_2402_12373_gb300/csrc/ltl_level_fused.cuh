// ltl_level_fused.cuh -- the size-level candidate kernel for matrices that fit
// in one CTA's registers (the common case: up to 4096 / W traces).
//
// Per size level one persistent launch; CTAs pull tiles (8 x 8 operand pairs,
// or 16 operands for unary connectives) from a counter.  Within a tile a CTA
// walks its candidates in batches of NB that share the left operand:
//
//   1. the batch's operand matrices arrive in shared memory by TMA bulk copies
//      (cp.async.bulk, completion on an mbarrier), issued while the previous
//      batch was in its hash phase;
//   2. every thread computes its share of each candidate's matrix in
//      registers (the connective by exponential propagation, Section 4), the
//      NH fingerprint partial sums and the position-0 soundness bits;
//   3. one CTA barrier reduces fingerprints and soundness over the CTA; a
//      separator is recorded (eq. (dagger)); the next batch's copies are issued;
//   4. lanes k < NB of warp 0 probe the device hash set in parallel, one
//      candidate each; the CTA then stores new matrices (and a lane publishes
//      the entry) or compares duplicates word by word with the stored entry.
//
// One kernel per connective (template OP): each launch of a level covers the
// segments (splits) of one connective, so the compiler allocates registers
// for that connective alone.
#pragma once
#include "ltl_level_common.cuh"

namespace ltl {
namespace lvl {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        "  .reg .pred p;\n"
        "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "  selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One-dimensional TMA bulk copy global -> shared, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// lane states of the hash phase (warp 0, one lane per candidate of the batch)
enum : int { S_PROBE = 0, S_STORE = 1, S_CMP = 2, S_DONE = 3 };

template <int NB>
struct FusedShared {
    unsigned long long fp[32][NB];
    uint32_t err[32][NB];
    unsigned long long tile;
    int skip;
    int cap_full;     // the tile's problem had a full cache when the tile was taken
    int found_seen;   // ... and a recorded separator
    unsigned long long idx[2][NB];
    int dec[2][NB];
    uint32_t neq[2];
    alignas(8) uint64_t bar;
};

struct LaneConst {
    uint64_t toff, cs, plane, stride;
    uint32_t want, care;
    int tid, lane, warp, nwarps;
};

// Returns false when an operand wait ran out (the CTA must take no more tiles).
template <int W, int C, int NB, int OP, bool NARROW>
__device__ __forceinline__ bool fused_tile(const Problem &pb, int level, const Seg &sg, uint64_t a0, uint64_t a1,
                                           uint64_t b0, uint64_t b1, FusedShared<NB> &sh, uint64_t *slots,
                                           uint32_t &phase, uint32_t &round, const LaneConst &lc,
                                           unsigned long long &done, unsigned long long &staged, bool cap_full) {
    constexpr bool BIN = is_binary(OP);
    const bool tri = sg.kind == SEG_TRI;
    const uint64_t *srcA = (OP == OP_ATOM) ? pb.atoms : pb.arena;
    const uint32_t cm_bytes = (uint32_t)(pb.stride * 8);
    uint64_t ci = a0, cj = b0, loaded_a = ~0ull;

    // next batch of the tile in (a outer, b inner) order; binary batches share a
    auto next = [&](uint64_t &a, uint64_t &bf, int &nb) -> bool {
        if constexpr (!BIN) {
            if (ci >= a1) return false;
            a = ci;
            bf = 0;
            nb = (int)min((uint64_t)NB, a1 - ci);
            ci += (uint64_t)nb;
            return true;
        }
        for (;;) {
            if (ci >= a1) return false;
            const uint64_t jb = tri ? max(b0, ci + 1) : b0;
            if (cj < jb) cj = jb;
            if (cj < b1) break;
            ++ci;
            cj = 0;
        }
        a = ci;
        bf = cj;
        nb = (int)min((uint64_t)NB, b1 - cj);
        cj += (uint64_t)nb;
        return true;
    };
    // thread 0 issues the TMA copies of a batch (all threads track loaded_a)
    auto issue = [&](uint64_t a, uint64_t bf, int nb) {
        const bool reload_a = BIN && (a != loaded_a);
        if (lc.tid == 0) {
            const uint32_t n = (uint32_t)nb + (reload_a ? 1u : 0u);
            staged += n;
            mbar_arrive_expect_tx(&sh.bar, n * cm_bytes);
            if (BIN) {
                if (reload_a) bulk_g2s(slots + (uint64_t)NB * lc.stride, srcA + (sg.a_begin + a) * pb.stride, cm_bytes, &sh.bar);
                for (int k = 0; k < nb; ++k)
                    bulk_g2s(slots + (uint64_t)k * lc.stride, pb.arena + (sg.b_begin + bf + k) * pb.stride, cm_bytes,
                             &sh.bar);
            } else {
                for (int k = 0; k < nb; ++k)
                    bulk_g2s(slots + (uint64_t)k * lc.stride, srcA + (sg.a_begin + a + k) * pb.stride, cm_bytes,
                             &sh.bar);
            }
        }
        if (BIN) loaded_a = a;
    };
    // false when the wait ran out: this thread has not seen the batch land,
    // and keeps the phase so that the copies can still be waited for
    auto wait_data = [&]() -> bool {
        unsigned long long spins = 0;
        while (!mbar_try_wait(&sh.bar, phase))
            if (++spins > pb.spin_limit) return false;
        phase ^= 1u;
        return true;
    };

    uint64_t a, bf;
    int nb;
    bool have = next(a, bf, nb);
    if (have) issue(a, bf, nb);
    while (have) {
        const bool landed = wait_data();
        // ---- 2. candidates of the batch in registers
        constexpr bool MASKED = (OP == OP_NOT || OP == OP_G);
        Frag<W, C> r[NB];
        uint64_t fp[NB];
        uint32_t errs[NB];
        if constexpr (OP == OP_U) {
            // the batch shares its left operand (slot NB); slots k >= nb hold
            // an earlier batch's operands, computed and then ignored
            Frag<W, C> x;
            load_frag<W, C, false>(slots + (uint64_t)NB * lc.stride, lc.plane, lc.toff, lc.cs, x);
#pragma unroll
            for (int k = 0; k < NB; ++k)
                load_frag<W, C, false>(slots + (uint64_t)k * lc.stride, lc.plane, lc.toff, lc.cs, r[k]);
            apply_binary_batch<OP, W, C, NB, NARROW>(r, x, pb.nsteps, pb.logstep != 0);
        }
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            fp[k] = 0;
            errs[k] = 0;
            if (k < nb) {
                if constexpr (OP != OP_U) {
                    Frag<W, C> x, m;
                    load_frag<W, C, false>(slots + (uint64_t)(BIN ? NB : k) * lc.stride, lc.plane, lc.toff, lc.cs, x);
                    if (BIN) load_frag<W, C, false>(slots + (uint64_t)k * lc.stride, lc.plane, lc.toff, lc.cs, r[k]);
                    if (MASKED) load_frag<W, C, true>(pb.mask, lc.plane, lc.toff, lc.cs, m);
                    apply_op<OP, W, C, NARROW>(r[k], x, m, pb.nsteps, pb.logstep != 0);
                }
                const uint32_t bits = pos0_bits<W, C, NARROW>(r[k]);
                errs[k] = (uint32_t)__popc((bits ^ lc.want) & lc.care);   // misclassified traces
            }
        }
        if (pb.ruc != RUC_FKP) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    const ulonglong2 key = __ldg(
                        reinterpret_cast<const ulonglong2 *>(pb.keys + (uint64_t)w * lc.plane + lc.toff + c * lc.cs));
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (k < nb) fp[k] += nh_term(r[k].v[c][0][w], key.x) + nh_term(r[k].v[c][1][w], key.y);
                }
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (k < nb) fp[k] += fkp_word<NARROW>(r[k].v[c][j][0], lc.toff + c * lc.cs + j, pb.fkp_b);
        }
        // ---- 3. CTA reduction (also frees the operand slots)
#pragma unroll
        for (int k = 0; k < NB; ++k) fp[k] = warp_sum_u64(fp[k]);
#pragma unroll
        for (int k = 0; k < NB; ++k) errs[k] = __reduce_add_sync(0xffffffffu, errs[k]);
        if (lc.lane == 0) {
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                sh.fp[lc.warp][k] = fp[k];
                sh.err[lc.warp][k] = errs[k];
            }
        }
        // the reduction's barrier also makes the wait's outcome uniform: if
        // any thread gave up, the batch's matrices may have been computed from
        // shared memory the copies had not filled yet, so nothing of it is
        // checked or admitted, no further copy is issued, and the CTA waits
        // (again bounded) for the copies still in flight before it stops
        if (__syncthreads_or(landed ? 0 : 1)) {
            if (lc.tid == 0) {
                atomicCAS(&pb.ctrl->err, 0, -4 /* LTL_ERR_TIMEOUT */);
                atomicExch(&pb.ctrl->stop, 1);
            }
            if (!landed) {
                unsigned long long spins = 0;
                while (!mbar_try_wait(&sh.bar, phase) && ++spins < (1ull << 26)) {
                }
            }
            __syncthreads();
            return false;
        }
        const uint64_t cur_a = a, cur_bf = bf;
        const int cur_nb = nb;
        have = next(a, bf, nb);
        if (have) issue(a, bf, nb);

        // ---- 4. hash phase: warp 0 lane k owns candidate k
        int state = S_DONE;
        unsigned long long key = 0, h = 0, idx = 0, waits = 0;
        uint64_t prov = 0;
        if (lc.warp == 0 && lc.lane < cur_nb) {
            uint64_t s = 0;
            uint32_t nerr = 0;
            for (int w2 = 0; w2 < lc.nwarps; ++w2) {
                s += sh.fp[w2][lc.lane];
                nerr += sh.err[w2][lc.lane];
            }
            if (BIN) prov = prov_pack(OP, sg.a_begin + cur_a, sg.b_begin + cur_bf + lc.lane);
            else prov = prov_pack(OP, sg.a_begin + cur_a + lc.lane, 0);
            // eq. (dagger), or noisy; no record once the tile's problem has one
            if (nerr <= pb.max_errors && !sh.found_seen) record_separator(pb, level, prov);
            key = admission_key(pb, s, h);
            state = S_PROBE;
        }
        for (;;) {
            const int slot = (int)(round & 1u);
            if (lc.warp == 0) {
                // a candidate waits while an earlier one of the batch with the
                // same fingerprint is unsettled (it may be its pending entry)
                bool blocked = false;
#pragma unroll
                for (int k2 = 0; k2 < NB; ++k2) {
                    const unsigned long long key2 = __shfl_sync(0xffffffffu, key, k2);
                    const int st2 = __shfl_sync(0xffffffffu, state, k2);
                    if (k2 < lc.lane && st2 != S_DONE && key2 == key) blocked = true;
                }
                int dec = DEC_DUP;
                if (state == S_PROBE && !blocked) dec = probe<false>(pb, key, h, idx, cap_full);
                if (state == S_PROBE) {
                    if (blocked || dec == DEC_WAIT) {
                        // retried next round, after every CTA has published the
                        // claims of its current round (bounded by spin_limit)
                        dec = DEC_WAIT;
                        if (++waits > pb.spin_limit) {
                            atomicAdd(&pb.ctrl->timeouts, 1ull);
                            atomicCAS(&pb.ctrl->err, 0, -4 /* LTL_ERR_TIMEOUT */);
                            atomicExch(&pb.ctrl->stop, 1);
                            dec = DEC_ERR;
                            state = S_DONE;
                        } else if (!blocked) {
                            __nanosleep(128);
                        }
                    } else {
                        state = dec == DEC_NEW ? S_STORE : dec == DEC_CMP ? S_CMP : S_DONE;
                    }
                }
                if (lc.lane < NB) {
                    sh.dec[slot][lc.lane] = (lc.lane < cur_nb) ? dec : DEC_DUP;
                    sh.idx[slot][lc.lane] = idx;
                }
            }
            __syncthreads();   // A: decisions visible
            if (lc.tid == 0) sh.neq[slot ^ 1] = 0u;
            uint32_t neq = 0;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int d = sh.dec[slot][k];
                if (d == DEC_NEW) {
                    store_frag<W, C>(r[k], pb.arena + sh.idx[slot][k] * pb.stride, lc.plane, lc.toff, lc.cs);
                } else if (d == DEC_CMP) {
                    if (!equal_frag<W, C>(r[k], pb.arena + sh.idx[slot][k] * pb.stride, lc.plane, lc.toff, lc.cs))
                        neq |= 1u << k;
                }
            }
            neq = __reduce_or_sync(0xffffffffu, neq);
            if (lc.lane == 0 && neq) atomicOr(&sh.neq[slot], neq);
            __syncthreads();   // B: stores issued, compare verdicts in
            const uint32_t nq = sh.neq[slot];
            bool more = false;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int d = sh.dec[slot][k];
                more |= (d == DEC_WAIT) || (d == DEC_CMP && ((nq >> k) & 1u));
            }
            if (lc.warp == 0) {
                // full compares done this round, counted once for the warp
                const uint32_t mcmp = __ballot_sync(0xffffffffu, state == S_CMP);
                if (lc.lane == 0 && mcmp) atomicAdd(&pb.ctrl->compares, (unsigned long long)__popc(mcmp));
                if (state == S_STORE) {
                    pb.prov[idx] = prov;
                    slot_publish(pb, h, key, idx);
                    state = S_DONE;
                } else if (state == S_CMP) {
                    if ((nq >> lc.lane) & 1u) {   // same fingerprint, different matrix
                        atomicAdd(&pb.ctrl->collisions, 1ull);
                        h = (h + 1) & pb.hmask;
                        state = S_PROBE;
                    } else {
                        state = S_DONE;
                    }
                }
                __syncwarp();
            }
            ++round;
            if (!more) break;
        }
        done += (unsigned long long)cur_nb;
    }
    return true;
}

}  // namespace

// Per-problem lane constants: plane geometry and which of the thread's trace
// slots are positive / real (for the soundness test of eq. (dagger)).
template <int C, bool NARROW>
__device__ __forceinline__ void set_lane_problem(const Problem &pb, LaneConst &lc) {
    lc.plane = pb.plane;
    lc.stride = pb.stride;
    lc.want = 0;
    lc.care = 0;
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint64_t word = lc.toff + c * lc.cs + j;
            if (NARROW) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint64_t t = 2 * word + h;
                    if (t < pb.n_pos) lc.want |= 1u << (4 * c + 2 * j + h);
                    if (t < pb.n_traces) lc.care |= 1u << (4 * c + 2 * j + h);
                }
            } else {
                if (word < pb.n_pos) lc.want |= 1u << (2 * c + j);
                if (word < pb.n_traces) lc.care |= 1u << (2 * c + j);
            }
        }
}

// Register cap: 168 for 8 words per thread and for the narrow layout's
// batches of four (three 128-thread CTAs per SM), 128 for the other shapes
// (at most 256 threads per CTA either way).
template <int W, int C, int NB, int OP, bool NARROW>
__global__ void __maxnreg__((NARROW || W * C >= 8) ? 168 : 128) fused_level_kernel(LevelArgs la) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    uint64_t *slots = reinterpret_cast<uint64_t *>(dyn_smem);
    __shared__ FusedShared<NB> sh;
    if (la.desc) {   // a level planned on the device: its extent is in memory
        la.n_segs = la.desc->n_segs;
        la.total_tiles = la.desc->total_tiles;
        if (la.total_tiles == 0) return;   // nothing of this connective (or the search has stopped)
    }
    LaneConst lc;
    lc.tid = threadIdx.x;
    lc.lane = lc.tid & 31;
    lc.warp = lc.tid >> 5;
    lc.nwarps = blockDim.x >> 5;
    lc.toff = 2ull * (uint64_t)lc.tid;
    lc.cs = 2ull * (uint64_t)blockDim.x;
    // the operand slots of every problem in the launch must fit its dynamic
    // shared memory (checked per tile below)
    uint32_t dsmem;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsmem));
    if (lc.tid == 0) {
        mbar_init(&sh.bar, 1);
        sh.neq[0] = sh.neq[1] = 0u;
    }
    __syncthreads();
    uint32_t phase = 0, round = 0;
    int cur_prob = -1;
    Problem pb;
    // candidates of the current problem finished by this CTA, added to the
    // problem's count when the CTA moves to another problem or ends
    unsigned long long cands_acc = 0;
    unsigned long long staged = 0;   // thread 0: operand matrices copied into shared memory
    for (;;) {
        // thread 0 takes a tile and reads its problem's stop flag
        if (lc.tid == 0) {
            const unsigned long long t = atomicAdd(la.tile_counter, 1ull);
            int skip = 1, cap = 0, found = 0;
            if (t < la.total_tiles) {
                const Ctrl *ctrl = la.probs[la.segs[find_segment(la, t)].prob].ctrl;
                skip = ld_volatile_i32(&ctrl->stop);
                cap = ld_volatile_i32(&ctrl->cap_hit);
                found = ld_volatile_i32(reinterpret_cast<const int *>(&ctrl->found_count));
            }
            sh.tile = t;
            sh.skip = skip;
            sh.cap_full = cap;
            sh.found_seen = found;
        }
        __syncthreads();
        const unsigned long long tile = sh.tile;
        const int skip = sh.skip;
        const bool cap_full = sh.cap_full != 0;
        __syncthreads();
        if (tile >= la.total_tiles) break;
        if (skip) continue;
        const Seg sg = la.segs[find_segment(la, tile)];
        if (sg.prob != cur_prob) {   // tiles of one problem usually come in runs
            if (lc.tid == 0 && cands_acc) atomicAdd(&pb.ctrl->cands, cands_acc);
            cands_acc = 0;
            cur_prob = sg.prob;
            pb = la.probs[sg.prob];
            set_lane_problem<C, NARROW>(pb, lc);
        }
        if ((uint64_t)dsmem < (uint64_t)(NB + 1) * pb.stride * 8ull) {   // slots must fit the launch's smem
            if (lc.tid == 0) atomicCAS(&pb.ctrl->err, 0, -1 /* LTL_ERR_INVALID */);
            continue;
        }
        uint64_t a0, a1, b0, b1;
        decode_tile(sg, tile - sg.tile_begin, a0, a1, b0, b1);
        unsigned long long done = 0;
        const bool ok =
            fused_tile<W, C, NB, OP, NARROW>(pb, sg.level, sg, a0, a1, b0, b1, sh, slots, phase, round, lc, done, staged,
                                             cap_full);
        cands_acc += done;
        if (!ok) break;
    }
    if (lc.tid == 0 && cands_acc) atomicAdd(&pb.ctrl->cands, cands_acc);
    if (lc.tid == 0 && staged && la.staged) atomicAdd(la.staged, staged);
}

}  // namespace lvl

// candidates per batch: 2 when a thread holds 8 words per candidate of the
// wide layout, else 4
template <int W, int C, bool NARROW>
struct FusedNB {
    static constexpr int value = (!NARROW && W * C >= 8) ? 2 : 4;
};

template <int W, int C, bool NARROW = false>
const void *fused_fn(int op) {
    constexpr int NB = FusedNB<W, C, NARROW>::value;
    switch (op) {
    case OP_ATOM: return reinterpret_cast<const void *>(&lvl::fused_level_kernel<W, C, NB, OP_ATOM, NARROW>);
    case OP_NOT: return reinterpret_cast<const void *>(&lvl::fused_level_kernel<W, C, NB, OP_NOT, NARROW>);
    case OP_AND: return reinterpret_cast<const void *>(&lvl::fused_level_kernel<W, C, NB, OP_AND, NARROW>);
    case OP_OR: return reinterpret_cast<const void *>(&lvl::fused_level_kernel<W, C, NB, OP_OR, NARROW>);
    case OP_X: return reinterpret_cast<const void *>(&lvl::fused_level_kernel<W, C, NB, OP_X, NARROW>);
    case OP_F: return reinterpret_cast<const void *>(&lvl::fused_level_kernel<W, C, NB, OP_F, NARROW>);
    case OP_G: return reinterpret_cast<const void *>(&lvl::fused_level_kernel<W, C, NB, OP_G, NARROW>);
    case OP_U: return reinterpret_cast<const void *>(&lvl::fused_level_kernel<W, C, NB, OP_U, NARROW>);
    default: return nullptr;
    }
}

}  // namespace ltl
