// ltl_plan.cu -- the device planner of small size levels.
//
// A level's candidate space depends on how many formulas every earlier level
// added, which is known only once those levels have run.  For levels that are
// small (launch-latency bound), a host round trip per level costs more than
// the level itself; the planner instead closes level k - 1 and plans level k
// on the device, from the counts the level kernels left in the control block,
// with the same segment and tile code the host planner uses (ltl_plan.h).
// The host enqueues a chain of levels back to back -- planner, then one
// persistent launch per connective that reads its extent from the planner's
// output -- and reads back one log per level at the end.
#include <cuda_runtime.h>

#include "ltl_internal.h"
#include "ltl_plan.h"

namespace ltl {
namespace {

struct GroupEmit {
    const PlanArgs *a;
    int k;
    uint32_t nseg[kPlanGroups];
    bool bad;
    __device__ void operator()(Seg sg) {
        int g = -1;
        for (int i = 0; i < a->n_groups; ++i)
            if (a->group_op[i] == sg.op) g = i;
        if (g < 0 || nseg[g] >= (uint32_t)kPlanSegsPerGroup) {
            bad = true;   // the host launched no group for this connective
            return;
        }
        sg.prob = a->prob_index;
        sg.level = k;
        a->segs[g * kPlanSegsPerGroup + nseg[g]++] = sg;
    }
};

// One thread.  close_prev: record level k - 1 (its launches have finished, in
// stream order) and halt the chain if the host would stop after it.
// plan_this: write level k's segments, launch extents and zeroed tile counters.
__global__ void plan_level_kernel(PlanArgs a, int k, int close_prev, int plan_this) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    PlanState &st = *a.state;
    const Problem &pb = *a.prob;
    const Ctrl c = *pb.ctrl;
    const uint64_t ent = plan_min(c.n_entries, pb.max_entries);
    if (close_prev) {
        const int j = k - 1;
        st.lvl_count[j] = ent - st.lvl_begin[j];
        PlanLog &lg = a.log[j];
        lg.snap = c;
        lg.count = st.lvl_count[j];
        lg.t_end = now;
        const bool found_stop = c.found_count > 0 && a.stop_mode != LTL_STOP_NONE;
        if (c.invalid_letter || c.err || c.cap_hit || found_stop) st.halted = 1;
    }
    if (!plan_this) return;
    for (int g = 0; g < a.n_groups; ++g) {
        a.desc[g].n_segs = 0;
        a.desc[g].total_tiles = 0;
        a.counters[g] = 0ull;
    }
    PlanLog &lg = a.log[k];
    lg.begin = ent;
    lg.count = 0;
    lg.n_segs = 0;
    lg.ran = 0;
    lg.t_begin = now;
    lg.t_end = now;
    if (st.halted) return;
    st.lvl_begin[k] = ent;
    lg.ran = 1;
    GroupEmit emit{&a, k, {}, false};
    plan_level_segments(a.ops, a.n_props, st.lvl_begin, st.lvl_count, k, a.cost, emit);
    if (emit.bad) {
        atomicCAS(&pb.ctrl->err, 0, (int)LTL_ERR_INVALID);
        st.halted = 1;
        return;
    }
    for (int g = 0; g < a.n_groups; ++g) {
        Seg *sg = a.segs + g * kPlanSegsPerGroup;
        uint64_t cands = 0;
        for (uint32_t i = 0; i < emit.nseg[g]; ++i) cands += seg_candidates(sg[i]);
        const uint32_t cpt = tile_target(cands, a.group_cap[g], a.nb, a.tiles_per_cta);
        uint64_t total = 0;
        for (uint32_t i = 0; i < emit.nseg[g]; ++i) {
            set_tiles(sg[i], cpt);
            sg[i].tile_begin = total;
            total += sg[i].n_tiles;
        }
        a.desc[g].n_segs = (int32_t)emit.nseg[g];
        a.desc[g].total_tiles = total;
        lg.n_segs += emit.nseg[g];
    }
}

}  // namespace

cudaError_t launch_plan(const PlanArgs &a, int k, bool close_prev, bool plan_this, cudaStream_t s) {
    plan_level_kernel<<<1, 32, 0, s>>>(a, k, close_prev ? 1 : 0, plan_this ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace ltl
