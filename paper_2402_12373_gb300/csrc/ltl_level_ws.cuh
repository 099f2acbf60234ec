// ltl_level_ws.cuh -- the size-level candidate kernel with warp-specialised
// hash warps (for matrices that fit in one CTA's registers).
//
// The same per-candidate work as the fused kernel (ltl_level_fused.cuh), but
// no compute thread ever waits for a global-memory round trip of the hash set:
//
//   * NT compute threads pull tiles, receive each batch's operands in shared
//     memory by TMA bulk copies (prefetched one batch ahead), compute the NB
//     candidates in registers (exponential propagation, Section 4) and stage
//     them -- with per-warp NH fingerprint partial sums and misclassification
//     counts -- in a ring slot in shared memory, then go on with the next
//     batch.
//   * Two hash warps, one per ring slot, settle a staged batch completely:
//     lane k sums the partials of candidate k, records a separator (eq.
//     (dagger), or the noisy variant) and probes the device hash set; a new
//     matrix leaves the ring slot for the cache by one TMA bulk copy issued by
//     its lane, the warp compares duplicates with the stored entries (a whole
//     8 KiB matrix of 16-byte loads in flight per round trip), and the lanes
//     publish their new entries once their copies are complete and probe on
//     after fingerprint collisions, before the slot is freed.
//
// Slots hand over through two mbarriers: full (batch staged, compute -> hash)
// and empty (slot free, hash -> compute).  Every wait is bounded; a timed-out
// wait in the compute threads is made the same in every compute thread
// (barrier reduction) before anyone acts on it, sets the problem's error flag
// and winds the kernel down.
//
// Progress: a probe never blocks on another CTA's unpublished entry (DEC_WAIT
// is retried in a later round), and a hash warp stores and publishes the
// entries it claims in the same round, before it can wait on anything.  So
// every entry a hash warp waits for is published without depending on that
// warp, and nothing a hash warp does waits on the compute threads.
#pragma once
#include "ltl_level_common.cuh"

namespace ltl {
namespace lvl {
namespace ws {

constexpr int kRing = 2;        // ring slots = hash warps
constexpr int kMaxCWarps = 8;   // compute warps per CTA (NT <= 256)

// lane states of the hash warps (one lane per candidate of the batch)
enum : int { S_PROBE = 0, S_STORE = 1, S_CMP = 2, S_DONE = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// One-dimensional TMA bulk copy shared -> global (a bulk async-group of the
// issuing thread), its commit, and the wait for its completion (the writes
// performed), followed by the fence that orders those async-proxy writes
// before this thread's later generic-proxy operations (the release store that
// publishes the entry).
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_s2g_complete() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// New matrices leave a ring slot by TMA bulk copies for every connective but
// U; U's compute threads are as busy as its hash warps, and the proxy fence
// the bulk copies need on the compute side measured slower there.
template <int OP>
constexpr bool kBulkStore = OP != OP_U;

// Named barrier over the compute threads only (the hash warps never join it).
__device__ __forceinline__ void compute_sync(int nt) { asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory"); }

// The same barrier, returning the AND of `v` over the compute threads, so that
// a decision taken after a bounded wait is the same in every compute thread.
__device__ __forceinline__ bool compute_all(int nt, bool v) {
    uint32_t r;
    asm volatile(
        "{\n"
        "  .reg .pred pi, po;\n"
        "  setp.ne.u32 pi, %1, 0;\n"
        "  bar.red.and.pred po, 1, %2, pi;\n"
        "  selp.u32 %0, 1, 0, po;\n"
        "}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(nt)
        : "memory");
    return r != 0;
}

// Bounded wait without side effects: false after `limit` tries.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, unsigned long long limit) {
    unsigned long long spins = 0;
    while (!mbar_try_wait(bar, parity))
        if (++spins > limit) return false;
    return true;
}

// What the compute threads leave in a ring slot for its hash warp.
template <int NB>
struct SlotMeta {
    unsigned long long fp[kMaxCWarps][NB];   // per compute warp: NH partial sums
    uint32_t err[kMaxCWarps][NB];            // per compute warp: misclassified traces
    int prob;                                // problem index; -1: no more batches
    int level;
    int nb;                                  // candidates in the batch
    uint64_t pa, pb;                         // provenance base: left operand, first right operand
};

template <int NB>
struct WsShared {
    SlotMeta<NB> meta[kRing];
    alignas(8) uint64_t full[kRing];      // batch staged (compute -> hash)
    alignas(8) uint64_t empty[kRing];     // slot free again (hash -> compute)
    alignas(8) uint64_t ops;
    unsigned long long tile;
    int skip;
    int bad_smem;
};

// Compute-side constants of the thread's share of a matrix.
struct CLane {
    uint64_t toff, cs, plane, stride;
    uint32_t want, care;
    int tid, lane, warp, nwarps, nt;
};

template <int C, bool NARROW>
__device__ __forceinline__ void set_clane_problem(const Problem &pb, CLane &lc) {
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

// ----------------------------------------------------------- compute role

template <int W, int C, int NB, int OP, bool NARROW>
__device__ __forceinline__ void compute_role(const LevelArgs &la, WsShared<NB> &sh, uint64_t *opslots,
                                             uint32_t dsmem, CLane &lc) {
    constexpr bool BIN = is_binary(OP);
    constexpr bool MASKED = (OP == OP_NOT || OP == OP_G);
    uint32_t ops_phase = 0;
    uint32_t batch = 0;   // batches handed over: slot = batch % 2, slot use = batch / 2
    int cur_prob = -1;
    Problem pb;
    bool alive = true;
    unsigned long long staged = 0;   // thread 0: operand matrices copied into shared memory
    bool inflight = false;   // operand copies issued and not yet waited for
    uint64_t *ring = nullptr;
    // a timed-out wait (same outcome in every compute thread) stops the launch's work
    auto give_up = [&]() {
        if (lc.tid == 0) {
            atomicCAS(&pb.ctrl->err, 0, -4 /* LTL_ERR_TIMEOUT */);
            atomicExch(&pb.ctrl->stop, 1);
        }
        alive = false;
    };
    // thread 0 reserves each tile one tile ahead, so that the counter's round
    // trip overlaps the tile before
    unsigned long long next_tile = 0;
    if (lc.tid == 0) next_tile = atomicAdd(la.tile_counter, 1ull);
    for (;;) {
        if (lc.tid == 0) {
            const unsigned long long t = next_tile;
            int skip = 1;
            if (t < la.total_tiles) {
                next_tile = atomicAdd(la.tile_counter, 1ull);
                const int si = find_segment(la, t);
                skip = ld_volatile_i32(&la.probs[la.segs[si].prob].ctrl->stop);
            }
            sh.tile = t;
            sh.skip = skip;
        }
        compute_sync(lc.nt);
        const unsigned long long tile = sh.tile;
        const int skip = sh.skip;
        compute_sync(lc.nt);
        if (tile >= la.total_tiles || !alive) break;
        if (skip) continue;
        const Seg sg = la.segs[find_segment(la, tile)];
        if (sg.prob != cur_prob) {
            cur_prob = sg.prob;
            pb = la.probs[sg.prob];
            set_clane_problem<C, NARROW>(pb, lc);
            // ring slots after the NB + 1 operand slots (every problem of a
            // launch has the launch's shape, hence the same stride)
            ring = opslots + (uint64_t)(NB + 1) * pb.stride;
        }
        if ((uint64_t)dsmem < (uint64_t)(NB + 1 + kRing * NB) * pb.stride * 8ull) {
            if (lc.tid == 0) atomicCAS(&pb.ctrl->err, 0, -1 /* LTL_ERR_INVALID */);
            continue;
        }
        uint64_t a0, a1, b0, b1;
        decode_tile(sg, tile - sg.tile_begin, a0, a1, b0, b1);
        const bool tri = sg.kind == SEG_TRI;
        const uint64_t *srcA = (OP == OP_ATOM) ? pb.atoms : pb.arena;
        const uint32_t cm_bytes = (uint32_t)(pb.stride * 8);
        uint64_t ci = a0, cj = b0, loaded_a = ~0ull;   // operand indices are relative to the segment
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
        auto issue = [&](uint64_t a, uint64_t bf, int nb) {
            const bool reload_a = BIN && (a != loaded_a);
            if (lc.tid == 0) {
                const uint32_t n = (uint32_t)nb + (reload_a ? 1u : 0u);
                staged += n;
                mbar_arrive_expect_tx(&sh.ops, n * cm_bytes);
                if (BIN) {
                    if (reload_a)
                        bulk_g2s(opslots + (uint64_t)NB * lc.stride, srcA + (sg.a_begin + a) * pb.stride, cm_bytes,
                                 &sh.ops);
                    for (int k = 0; k < nb; ++k)
                        bulk_g2s(opslots + (uint64_t)k * lc.stride, pb.arena + (sg.b_begin + bf + k) * pb.stride,
                                 cm_bytes, &sh.ops);
                } else {
                    for (int k = 0; k < nb; ++k)
                        bulk_g2s(opslots + (uint64_t)k * lc.stride, srcA + (sg.a_begin + a + k) * pb.stride,
                                 cm_bytes, &sh.ops);
                }
            }
            if (BIN) loaded_a = a;
            inflight = true;
        };
        uint64_t a, bf;
        int nb;
        bool have = next(a, bf, nb);
        if (have) issue(a, bf, nb);
        while (have) {
            if (!compute_all(lc.nt, mbar_wait_for(&sh.ops, ops_phase, pb.spin_limit))) {
                give_up();
                break;
            }
            inflight = false;
            ops_phase ^= 1u;
            Frag<W, C> r[NB];
            uint64_t fp[NB];
            uint32_t errs[NB];
            if constexpr (OP == OP_U) {
                // the batch shares its left operand (slot NB); slots k >= nb
                // hold an earlier batch's operands, computed and then ignored
                Frag<W, C> x;
                load_frag<W, C, false>(opslots + (uint64_t)NB * lc.stride, lc.plane, lc.toff, lc.cs, x);
#pragma unroll
                for (int k = 0; k < NB; ++k)
                    load_frag<W, C, false>(opslots + (uint64_t)k * lc.stride, lc.plane, lc.toff, lc.cs, r[k]);
                apply_binary_batch<OP, W, C, NB, NARROW>(r, x, pb.nsteps, pb.logstep != 0);
            }
            // the batch's shared left operand (And, Or) and the length mask
            // (Not, G) are read once per batch
            Frag<W, C> xs, m;
            if constexpr (OP != OP_U && BIN) load_frag<W, C, false>(opslots + (uint64_t)NB * lc.stride, lc.plane,
                                                                    lc.toff, lc.cs, xs);
            if constexpr (MASKED) load_frag<W, C, true>(pb.mask, lc.plane, lc.toff, lc.cs, m);
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                fp[k] = 0;
                errs[k] = 0;
                if (k < nb) {
                    if constexpr (OP != OP_U && BIN) {
                        load_frag<W, C, false>(opslots + (uint64_t)k * lc.stride, lc.plane, lc.toff, lc.cs, r[k]);
                        apply_op<OP, W, C, NARROW>(r[k], xs, m, pb.nsteps, pb.logstep != 0);
                    } else if constexpr (OP != OP_U) {
                        Frag<W, C> x;
                        load_frag<W, C, false>(opslots + (uint64_t)k * lc.stride, lc.plane, lc.toff, lc.cs, x);
                        apply_op<OP, W, C, NARROW>(r[k], x, m, pb.nsteps, pb.logstep != 0);
                    }
                    const uint32_t bits = pos0_bits<W, C, NARROW>(r[k]);
                    errs[k] = (uint32_t)__popc((bits ^ lc.want) & lc.care);
                }
            }
            // every compute thread is done with the operand slots: prefetch the next batch
            compute_sync(lc.nt);
            const uint64_t cur_a = a, cur_bf = bf;
            const int cur_nb = nb;
            have = next(a, bf, nb);
            if (have) issue(a, bf, nb);
            // fingerprints (NH, or first-k-percent under relaxed admission)
            if (pb.ruc != RUC_FKP) {
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        const ulonglong2 key = __ldg(reinterpret_cast<const ulonglong2 *>(
                            pb.keys + (uint64_t)w * lc.plane + lc.toff + c * lc.cs));
#pragma unroll
                        for (int k = 0; k < NB; ++k)
                            if (k < cur_nb) fp[k] += nh_term(r[k].v[c][0][w], key.x) + nh_term(r[k].v[c][1][w], key.y);
                    }
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int j = 0; j < 2; ++j)
#pragma unroll
                        for (int k = 0; k < NB; ++k)
                            if (k < cur_nb)
                                fp[k] += fkp_word<NARROW>(r[k].v[c][j][0], lc.toff + c * lc.cs + j, pb.fkp_b);
            }
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                fp[k] = warp_sum_u64(fp[k]);
                errs[k] = __reduce_add_sync(0xffffffffu, errs[k]);
            }
            // hand the batch to the slot's hash warp
            const int slot = (int)(batch & 1u);
            if (!compute_all(lc.nt, mbar_wait_for(&sh.empty[slot], ((batch >> 1) & 1u) ^ 1u, pb.spin_limit))) {
                give_up();
                break;
            }
            uint64_t *dst = ring + (uint64_t)slot * NB * lc.stride;
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (k < cur_nb) store_frag<W, C>(r[k], dst + (uint64_t)k * lc.stride, lc.plane, lc.toff, lc.cs);
            // the hash warp copies new matrices out of the slot with bulk
            // (async-proxy) copies (every connective but U): these
            // shared-memory writes must be visible to that proxy once the
            // slot is handed over
            if constexpr (kBulkStore<OP>) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            SlotMeta<NB> &mt = sh.meta[slot];
            if (lc.lane == 0) {
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    mt.fp[lc.warp][k] = fp[k];
                    mt.err[lc.warp][k] = errs[k];
                }
            }
            if (lc.tid == 0) {
                mt.prob = sg.prob;
                mt.level = sg.level;
                mt.nb = cur_nb;
                mt.pa = sg.a_begin + cur_a;
                mt.pb = BIN ? sg.b_begin + cur_bf : 0;
            }
            mbar_arrive(&sh.full[slot]);
            ++batch;
        }
        if (!alive) break;
    }
    if (lc.tid == 0 && staged && la.staged) atomicAdd(la.staged, staged);
    // a wait that gave up may leave this CTA's own operand copies in flight:
    // wait for them (bounded) before the CTA's shared memory goes away
    if (inflight) compute_all(lc.nt, mbar_wait_for(&sh.ops, ops_phase, 1ull << 26));
    // no more batches: one end marker per ring slot (after a timeout the
    // marker is sent without waiting: the hash warps stop on it or on their own
    // bounded waits)
    for (int s = 0; s < kRing; ++s, ++batch) {
        const int slot = (int)(batch & 1u);
        if (alive) compute_all(lc.nt, mbar_wait_for(&sh.empty[slot], ((batch >> 1) & 1u) ^ 1u, 1ull << 26));
        if (lc.tid == 0) sh.meta[slot].prob = -1;
        mbar_arrive(&sh.full[slot]);
    }
}

// ----------------------------------------------------------- hash role

// One probe round for the lanes in S_PROBE (lane k < nb owns candidate k): a
// candidate waits while an earlier one of the batch with the same key is
// unsettled; a probe that meets another CTA's unpublished entry is retried in
// a later round (DEC_WAIT).
__device__ __forceinline__ int probe_round(const Problem &pb, int lane, int nb_max, int &state,
                                           unsigned long long key, unsigned long long &h, unsigned long long &idx,
                                           unsigned long long &waits, bool cap_full) {
    bool blocked = false;
    for (int k2 = 0; k2 < nb_max; ++k2) {
        const unsigned long long key2 = __shfl_sync(0xffffffffu, key, k2);
        const int st2 = __shfl_sync(0xffffffffu, state, k2);
        if (k2 < lane && st2 != S_DONE && key2 == key) blocked = true;
    }
    int dec = DEC_DUP;
    if (state == S_PROBE && !blocked) dec = probe<false, false>(pb, key, h, idx, cap_full);
    if (state == S_PROBE) {
        if (blocked || dec == DEC_WAIT) {
            dec = DEC_WAIT;
            if (++waits > pb.spin_limit) {
                atomicAdd(&pb.ctrl->timeouts, 1ull);
                atomicCAS(&pb.ctrl->err, 0, -4 /* LTL_ERR_TIMEOUT */);
                atomicExch(&pb.ctrl->stop, 1);
                dec = DEC_ERR;
                state = S_DONE;
            }
        } else {
            state = dec == DEC_NEW ? S_STORE : dec == DEC_CMP ? S_CMP : S_DONE;
        }
    }
    return dec;
}

// One matrix from a ring slot (shared memory) into its cache entry, the
// warp's 32 lanes 16 bytes apart.
__device__ __forceinline__ void copy_matrix(const uint64_t *src, uint64_t *dst, uint64_t stride, int lane) {
    constexpr int kU = 8;
    for (uint64_t base = 2 * (uint64_t)lane; base < stride; base += 64 * kU) {
        ulonglong2 v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (base + 64 * u < stride) v[u] = *reinterpret_cast<const ulonglong2 *>(src + base + 64 * u);
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (base + 64 * u < stride) *reinterpret_cast<ulonglong2 *>(dst + base + 64 * u) = v[u];
    }
}

// Full compare of a staged matrix with a cache entry, in chunks of 16
// 16-byte pieces per lane (an 8 KiB matrix is one chunk, one global round
// trip).  load_chunk issues a chunk's loads; differs compares the chunk
// already in q (loaded by the caller) and then every later chunk.  Entries
// published during this launch are read through L2 only (ld.cg).
constexpr int kCmpUnroll = 16;

__device__ __forceinline__ void load_chunk(ulonglong2 (&q)[kCmpUnroll], const uint64_t *ent, uint64_t base0,
                                           uint64_t stride, int lane) {
    const uint64_t base = base0 + 2 * (uint64_t)lane;
#pragma unroll
    for (int u = 0; u < kCmpUnroll; ++u)
        if (base + 64 * u < stride) q[u] = __ldcg(reinterpret_cast<const ulonglong2 *>(ent + base + 64 * u));
}

__device__ __forceinline__ bool differs(ulonglong2 (&q)[kCmpUnroll], const uint64_t *src, const uint64_t *ent,
                                        uint64_t stride, int lane) {
    bool eq = true;
    for (uint64_t base0 = 0; base0 < stride; base0 += 64 * kCmpUnroll) {
        if (base0 > 0) load_chunk(q, ent, base0, stride, lane);
        const uint64_t base = base0 + 2 * (uint64_t)lane;
#pragma unroll
        for (int u = 0; u < kCmpUnroll; ++u)
            if (base + 64 * u < stride) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(src + base + 64 * u);
                eq &= (q[u].x == v.x) & (q[u].y == v.y);
            }
    }
    return __any_sync(0xffffffffu, !eq);
}

template <int NB, int OP>
__device__ __forceinline__ void hash_role(const LevelArgs &la, WsShared<NB> &sh, uint64_t *opslots, int slot,
                                          int lane, int ncw, unsigned long long spin_cap) {
    uint32_t uses = 0;
    int cur_prob = -1;
    bool found_seen = false;
    Problem pb;
    unsigned long long cands_acc = 0;   // lane 0: candidates of the current problem, added on a change or at the end
    auto flush = [&]() {
        if (lane == 0 && cands_acc) atomicAdd(&pb.ctrl->cands, cands_acc);
        cands_acc = 0;
    };
    auto wait_all = [&](uint64_t *bar, uint32_t parity) -> bool {
        const bool ok = __all_sync(0xffffffffu, mbar_wait_for(bar, parity, spin_cap));
        if (!ok && cur_prob >= 0 && lane == 0) {
            atomicCAS(&pb.ctrl->err, 0, -4 /* LTL_ERR_TIMEOUT */);
            atomicExch(&pb.ctrl->stop, 1);
        }
        return ok;
    };
    for (;;) {
        if (!wait_all(&sh.full[slot], uses & 1u)) {   // the compute threads always send an end marker
            flush();
            return;
        }
        SlotMeta<NB> &mt = sh.meta[slot];
        const int prob = mt.prob;
        if (prob < 0) {
            flush();
            return;
        }
        if (prob != cur_prob) {
            if (cur_prob >= 0) flush();
            cur_prob = prob;
            pb = la.probs[prob];
            // a recorded separator of the problem makes further records unnecessary
            found_seen = __shfl_sync(0xffffffffu,
                                     lane == 0 ? ld_volatile_i32(reinterpret_cast<const int *>(&pb.ctrl->found_count)) : 0,
                                     0) != 0;
        }
        // the cache-full flag, once per batch, read before the batch's setup so
        // that its latency overlaps it (a stale "not full" only costs a claim
        // that fails at allocation)
        const int cap_raw = lane == 0 ? ld_volatile_i32(&pb.ctrl->cap_hit) : 0;
        const int nb = mt.nb;
        const int level = mt.level;
        const uint64_t *cms = opslots + (uint64_t)(NB + 1 + slot * NB) * pb.stride;
        int state = S_DONE;
        unsigned long long key = 0, h = 0, idx = 0, waits = 0;
        uint64_t prov = 0;
        bool sep = false;
        if (lane < nb) {
            uint64_t s = 0;
            uint32_t nerr = 0;
            for (int w = 0; w < ncw; ++w) {
                s += mt.fp[w][lane];
                nerr += mt.err[w][lane];
            }
            prov = is_binary(OP) ? prov_pack(OP, mt.pa, mt.pb + (uint64_t)lane) : prov_pack(OP, mt.pa + (uint64_t)lane, 0);
            if (nerr <= pb.max_errors && !found_seen) record_separator(pb, level, prov);   // eq. (dagger), or noisy
            key = admission_key(pb, s, h);
            state = S_PROBE;
            sep = nerr <= pb.max_errors;
        }
        found_seen |= __any_sync(0xffffffffu, sep);
        // every round: probe the unsettled lanes, copy the new matrices into
        // the cache, compare the duplicates, publish, probe on after a
        // collision (a round that met another CTA's unpublished entry is
        // retried after a short sleep)
        const bool cap_full = __shfl_sync(0xffffffffu, cap_raw, 0) != 0;
        while (__any_sync(0xffffffffu, state != S_DONE)) {
            int dec = probe_round(pb, lane, NB, state, key, h, idx, waits, cap_full);
            // the round's claims take consecutive entry indices with one atomic
            // (the lanes' claims complete together, so nothing waits for a
            // slower lane)
            const uint32_t m_new = __ballot_sync(0xffffffffu, state == S_STORE);
            if (m_new) {
                const int leader = __ffs(m_new) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&pb.ctrl->n_entries, (unsigned long long)__popc(m_new));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (state == S_STORE) {
                    dec = claim_entry(pb, h, key, base + (unsigned long long)__popc(m_new & ((1u << lane) - 1u)), idx);
                    if (dec == DEC_FAIL) state = S_DONE;
                }
            }
            const uint32_t m_cmp = __ballot_sync(0xffffffffu, state == S_CMP);
            // the first duplicate's loads go out before the copies, which run
            // under their round trip
            uint32_t neq = 0;
            ulonglong2 q[kCmpUnroll];
            int kc = -1;
            if (m_cmp) {
                kc = __ffs(m_cmp) - 1;
                const unsigned long long ik = __shfl_sync(0xffffffffu, idx, kc);
                load_chunk(q, pb.arena + ik * pb.stride, 0, pb.stride, lane);
            }
            // each new matrix leaves the ring slot by one bulk copy issued by
            // the candidate's own lane -- or, for U, by the warp's 16-byte
            // stores, which keep the proxy fence off U's busier compute side
            if constexpr (kBulkStore<OP>) {
                if (state == S_STORE)
                    bulk_s2g(pb.arena + idx * pb.stride, cms + (uint64_t)lane * pb.stride, (uint32_t)(pb.stride * 8));
            } else {
                const uint32_t m_store = __ballot_sync(0xffffffffu, state == S_STORE);
                for (uint32_t m = m_store; m; m &= m - 1) {
                    const int k = __ffs(m) - 1;
                    const unsigned long long ik = __shfl_sync(0xffffffffu, idx, k);
                    copy_matrix(cms + (uint64_t)k * pb.stride, pb.arena + ik * pb.stride, pb.stride, lane);
                }
            }
            for (uint32_t m = m_cmp; m; m &= m - 1) {
                const int k = __ffs(m) - 1;
                const unsigned long long ik = __shfl_sync(0xffffffffu, idx, k);
                if (k != kc) load_chunk(q, pb.arena + ik * pb.stride, 0, pb.stride, lane);
                if (differs(q, cms + (uint64_t)k * pb.stride, pb.arena + ik * pb.stride, pb.stride, lane))
                    neq |= 1u << k;
            }
            if (kBulkStore<OP> && state == S_STORE) bulk_s2g_complete();   // the new matrix is in the cache
            __syncwarp();   // (U) every lane's share of the new matrices is written
            {
                const uint32_t mcmp = __ballot_sync(0xffffffffu, state == S_CMP);
                if (lane == 0 && mcmp) atomicAdd(&pb.ctrl->compares, (unsigned long long)__popc(mcmp));
            }
            if (state == S_STORE) {
                pb.prov[idx] = prov;
                slot_publish(pb, h, key, idx);
                state = S_DONE;
            } else if (state == S_CMP) {
                if ((neq >> lane) & 1u) {   // same fingerprint, different matrix
                    atomicAdd(&pb.ctrl->collisions, 1ull);
                    h = (h + 1) & pb.hmask;
                    state = S_PROBE;
                } else {
                    state = S_DONE;
                }
            }
            if (dec == DEC_WAIT) __nanosleep(128);
        }
        cands_acc += (unsigned long long)nb;
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.empty[slot]);
        ++uses;
    }
}

}  // namespace ws

// Block: NT compute threads (blockDim.x - 32 * kRing) then the hash warps.
// Register cap as the fused kernel's.
template <int W, int C, int NB, int OP, bool NARROW>
__global__ void __maxnreg__((NARROW || W * C >= 8) ? 168 : 128) ws_level_kernel(LevelArgs la) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ ws::WsShared<NB> sh;
    const int tid = threadIdx.x;
    const int nt = (int)blockDim.x - 32 * ws::kRing;
    uint32_t dsmem;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsmem));
    if (tid == 0) {
        for (int s = 0; s < ws::kRing; ++s) {
            ws::mbar_init(&sh.full[s], (uint32_t)nt);
            ws::mbar_init(&sh.empty[s], 1);
        }
        ws::mbar_init(&sh.ops, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (nt < 32 || nt > 32 * ws::kMaxCWarps) return;   // launch shape outside what the slots hold
    uint64_t *opslots = reinterpret_cast<uint64_t *>(dyn_smem);
    if (tid < nt) {
        ws::CLane lc;
        lc.tid = tid;
        lc.lane = tid & 31;
        lc.warp = tid >> 5;
        lc.nwarps = nt >> 5;
        lc.nt = nt;
        lc.toff = 2ull * (uint64_t)tid;
        lc.cs = 2ull * (uint64_t)nt;
        lc.plane = lc.stride = 0;
        ws::compute_role<W, C, NB, OP, NARROW>(la, sh, opslots, dsmem, lc);
    } else {
        const int hw = (tid - nt) >> 5;
        ws::hash_role<NB, OP>(la, sh, opslots, hw, tid & 31, nt >> 5, 1ull << 26);
    }
}

}  // namespace lvl
}  // namespace ltl

namespace ltl {

// candidates per batch: as the fused kernel (2 when a thread holds 8 words
// per candidate of the wide layout, else 4)
template <int W, int C, bool NARROW>
struct WsNB {
    static constexpr int value = (!NARROW && W * C >= 8) ? 2 : 4;
};

template <int W, int C, bool NARROW = false>
const void *ws_fn(int op) {
    constexpr int NB = WsNB<W, C, NARROW>::value;
    switch (op) {
    case OP_ATOM: return reinterpret_cast<const void *>(&lvl::ws_level_kernel<W, C, NB, OP_ATOM, NARROW>);
    case OP_NOT: return reinterpret_cast<const void *>(&lvl::ws_level_kernel<W, C, NB, OP_NOT, NARROW>);
    case OP_AND: return reinterpret_cast<const void *>(&lvl::ws_level_kernel<W, C, NB, OP_AND, NARROW>);
    case OP_OR: return reinterpret_cast<const void *>(&lvl::ws_level_kernel<W, C, NB, OP_OR, NARROW>);
    case OP_X: return reinterpret_cast<const void *>(&lvl::ws_level_kernel<W, C, NB, OP_X, NARROW>);
    case OP_F: return reinterpret_cast<const void *>(&lvl::ws_level_kernel<W, C, NB, OP_F, NARROW>);
    case OP_G: return reinterpret_cast<const void *>(&lvl::ws_level_kernel<W, C, NB, OP_G, NARROW>);
    case OP_U: return reinterpret_cast<const void *>(&lvl::ws_level_kernel<W, C, NB, OP_U, NARROW>);
    default: return nullptr;
    }
}

}  // namespace ltl
