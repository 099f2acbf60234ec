// ltl_level_cluster.cu -- the size-level candidate kernel for characteristic
// matrices larger than one CTA holds, on thread-block clusters.
//
// A cluster of CL CTAs (one candidate at a time) splits the matrix into CL
// slices of whole chunk groups; each CTA computes its slice of the candidate
// once -- operands read straight from the cache with coalesced 16-byte loads,
// the connective by exponential propagation (Section 4) -- and keeps it in
// its shared memory, together with its NH fingerprint partial sum and
// misclassification count.  The partials go to the leader CTA through
// distributed shared memory; the leader records a separator (eq. (dagger), or
// the noisy variant) and probes the device hash set; then every CTA stores its
// slice into the new entry, or compares it with the stored entry of equal
// fingerprint, and the leader publishes the entry or continues probing.
// Against the two-pass streaming kernel this reads the operands once instead
// of twice and spreads a candidate over CL SMs.
//
// Control decisions are read by every CTA from the leader's shared memory
// after a cluster barrier, so all threads of the cluster take the same path
// through every barrier.  The probe may wait (bounded) on another
// cluster's unpublished entry: a cluster holds no unpublished claim of its
// own while it probes, so no two clusters can wait on each other.
#include <cooperative_groups.h>

#include "ltl_level_common.cuh"

namespace cg = cooperative_groups;

namespace ltl {
namespace lvl {
namespace {

constexpr int kClusterMax = 16;


struct ClusterShared {
    unsigned long long fp_warp[8];           // block reduction scratch
    uint32_t err_warp[8];
    int eq_warp[8];
    unsigned long long part_fp[kClusterMax];  // leader: per-CTA partials (written remotely)
    uint32_t part_err[kClusterMax];
    uint32_t part_neq[kClusterMax];          // every CTA: per-CTA "slice differs" (written remotely)
    unsigned long long tile;                 // leader -> all
    int skip;
    int dec;                                 // leader -> all: DEC_NEW, DEC_CMP, or a terminal value
    unsigned long long idx;
};

template <int W, int C, int OP>
__device__ __forceinline__ void cluster_candidate(const Problem &pb, int level, uint64_t a, uint64_t b,
                                                  ClusterShared &sh, ClusterShared *lead, uint64_t *slice, int rank,
                                                  int ncta, int gpc, int tid, int NT, cg::cluster_group &cluster) {
    constexpr bool BIN = is_binary(OP);
    constexpr bool MASKED = (OP == OP_NOT || OP == OP_G);
    const uint64_t *A = ((OP == OP_ATOM) ? pb.atoms : pb.arena) + a * pb.stride;
    const uint64_t *B = pb.arena + b * pb.stride;
    const uint64_t cs = 2ull * (uint64_t)NT;
    const uint64_t sw = pb.plane / (uint64_t)ncta;   // words of each plane in this CTA's slice
    const uint64_t s0 = (uint64_t)rank * sw;         // first word of the slice
    const int lane = tid & 31, warp = tid >> 5;
    // 1. this CTA's slice of the candidate, into shared memory
    uint64_t fp = 0;
    uint32_t nerr = 0;
    for (int g = 0; g < gpc; ++g) {
        const uint64_t toff = 2ull * ((uint64_t)(rank * gpc + g) * C * NT + (uint64_t)tid);
        Frag<W, C> x, r, m;
        load_frag<W, C, true>(A, pb.plane, toff, cs, x);
        if (BIN) load_frag<W, C, true>(B, pb.plane, toff, cs, r);
        if (MASKED) load_frag<W, C, true>(pb.mask, pb.plane, toff, cs, m);
        apply_op<OP, W, C>(r, x, m, pb.nsteps, pb.logstep != 0);
        store_frag<W, C>(r, slice, sw, toff - s0, cs);
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
    if (lane == 0) {
        sh.fp_warp[warp] = fp;
        sh.err_warp[warp] = nerr;
    }
    __syncthreads();
    if (tid == 0) {
        uint64_t s = 0;
        uint32_t e = 0;
        for (int w2 = 0; w2 < (NT >> 5); ++w2) {
            s += sh.fp_warp[w2];
            e += sh.err_warp[w2];
        }
        lead->part_fp[rank] = s;
        lead->part_err[rank] = e;
    }
    cluster.sync();   // partials are in the leader
    // 2. the leader probes; every CTA stores or compares its slice
    const uint64_t prov = prov_pack(OP, a, BIN ? b : 0);
    const bool leader = rank == 0 && tid == 0;
    unsigned long long key = 0, h = 0, idx = 0;
    if (leader) {
        uint64_t s = 0;
        uint32_t e = 0;
        for (int q = 0; q < ncta; ++q) {
            s += sh.part_fp[q];
            e += sh.part_err[q];
        }
        if (e <= pb.max_errors) record_separator(pb, level, prov);   // eq. (dagger), or noisy
        key = admission_key(pb, s, h);
    }
    for (;;) {
        if (leader) {
            sh.dec = probe<true>(pb, key, h, idx, ld_volatile_i32(&pb.ctrl->cap_hit) != 0);
            sh.idx = idx;
        }
        cluster.sync();   // the decision is in the leader
        const int d = lead->dec;
        const unsigned long long ent_idx = lead->idx;
        if (d != DEC_NEW && d != DEC_CMP) break;   // duplicate of a settled entry, cache full, or error
        uint64_t *ent = pb.arena + ent_idx * pb.stride;
        bool eq = true;
        for (int g = 0; g < gpc; ++g) {
            const uint64_t toff = 2ull * ((uint64_t)(rank * gpc + g) * C * NT + (uint64_t)tid);
            Frag<W, C> v;
            load_frag<W, C, false>(slice, sw, toff - s0, cs, v);
            if (d == DEC_NEW) store_frag<W, C>(v, ent, pb.plane, toff, cs);
            else eq &= equal_frag<W, C>(v, ent, pb.plane, toff, cs);
        }
        if (d == DEC_CMP) {
            // this slice's verdict into every CTA of the cluster, so that all
            // of them settle the candidate alike after the next barrier
            const int all_eq = __syncthreads_and(eq);
            if (tid == 0)
                for (int q = 0; q < ncta; ++q) cluster.map_shared_rank(&sh, q)->part_neq[rank] = all_eq ? 0u : 1u;
        }
        cluster.sync();   // every slice stored or compared, every verdict everywhere
        if (d == DEC_NEW) {
            if (leader) {
                pb.prov[ent_idx] = prov;
                slot_publish(pb, h, key, ent_idx);
            }
            break;
        }
        uint32_t neq = 0;
        for (int q = 0; q < ncta; ++q) neq |= sh.part_neq[q];
        if (leader) {
            atomicAdd(&pb.ctrl->compares, 1ull);
            if (neq) {   // same fingerprint, different matrix: probe on
                atomicAdd(&pb.ctrl->collisions, 1ull);
                h = (h + 1) & pb.hmask;
            }
        }
        if (!neq) break;
    }
}

}  // namespace

template <int W, int C>
__global__ void __launch_bounds__(256) cluster_level_kernel(LevelArgs la) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    __shared__ ClusterShared sh;
    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x, NT = blockDim.x;
    const int rank = (int)cluster.block_rank();
    const int ncta = (int)cluster.num_blocks();
    ClusterShared *lead = cluster.map_shared_rank(&sh, 0);
    uint64_t *slice = reinterpret_cast<uint64_t *>(dyn_smem);
    uint32_t dsmem;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsmem));
    if (ncta > kClusterMax) return;   // every CTA of the cluster returns: no barrier is left waiting
    for (;;) {
        if (rank == 0 && tid == 0) {
            const unsigned long long t = atomicAdd(la.tile_counter, 1ull);
            int skip = 1;
            if (t < la.total_tiles) skip = ld_volatile_i32(&la.probs[la.segs[find_segment(la, t)].prob].ctrl->stop);
            sh.tile = t;
            sh.skip = skip;
        }
        cluster.sync();
        const unsigned long long tile = lead->tile;
        const int skip = lead->skip;
        cluster.sync();   // read before the leader takes the next tile
        if (tile >= la.total_tiles) break;
        if (skip) continue;
        const Seg sg = la.segs[find_segment(la, tile)];
        const Problem pb = la.probs[sg.prob];
        // the slices must be whole chunk groups and fit the launch's shared memory
        const int gpc = (int)(pb.groups / (uint32_t)ncta);
        if (pb.groups % (uint32_t)ncta != 0 || gpc < 1 ||
            (uint64_t)dsmem < (uint64_t)W * (pb.plane / (uint64_t)ncta) * 8ull) {
            if (rank == 0 && tid == 0) atomicCAS(&pb.ctrl->err, 0, -1 /* LTL_ERR_INVALID */);
            continue;
        }
        uint64_t a0, a1, b0, b1;
        decode_tile(sg, tile - sg.tile_begin, a0, a1, b0, b1);
        unsigned long long done = 0;
        for (uint64_t i = a0; i < a1; ++i) {
            const bool bin = is_binary(sg.op);
            const uint64_t jb = bin ? ((sg.kind == SEG_TRI) ? max(b0, i + 1) : b0) : 0;
            const uint64_t je = bin ? b1 : 1;
            for (uint64_t j = jb; j < je; ++j) {
                const uint64_t a = sg.a_begin + i, b = bin ? sg.b_begin + j : 0;
                switch (sg.op) {
#define LTL_CLUSTER_CASE(OPV)                                                                              \
    case OPV:                                                                                              \
        cluster_candidate<W, C, OPV>(pb, sg.level, a, b, sh, lead, slice, rank, ncta, gpc, tid, NT, cluster); \
        break;
                    LTL_CLUSTER_CASE(OP_ATOM)
                    LTL_CLUSTER_CASE(OP_NOT)
                    LTL_CLUSTER_CASE(OP_AND)
                    LTL_CLUSTER_CASE(OP_OR)
                    LTL_CLUSTER_CASE(OP_X)
                    LTL_CLUSTER_CASE(OP_F)
                    LTL_CLUSTER_CASE(OP_G)
                    LTL_CLUSTER_CASE(OP_U)
#undef LTL_CLUSTER_CASE
                default: break;
                }
                ++done;
            }
        }
        if (rank == 0 && tid == 0 && done) atomicAdd(&pb.ctrl->cands, done);
    }
}

}  // namespace lvl

template <int W, int C>
static const void *cluster_fn() {
    return reinterpret_cast<const void *>(&lvl::cluster_level_kernel<W, C>);
}

// Cluster shapes: as the streaming kernel's, C * W == 8 words per thread, 128
// threads per CTA.
const void *cluster_kernel_ptr(int W, int C) {
    switch (W * 16 + C) {
    case 1 * 16 + 8: return cluster_fn<1, 8>();
    case 2 * 16 + 4: return cluster_fn<2, 4>();
    case 4 * 16 + 2: return cluster_fn<4, 2>();
    case 8 * 16 + 1: return cluster_fn<8, 1>();
    default: return nullptr;
    }
}

}  // namespace ltl
