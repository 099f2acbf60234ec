// ltl_plan.h -- the candidate space of one size level and its tiling.
//
// Shared by the host planner (the engine plans a round from the level counts
// it read back) and the device planner (a one-thread kernel plans the next
// level from the counts left in device memory, so that small levels run back
// to back without a host round trip).  Both must cut a level into exactly the
// same segments and tiles, so the code is written once, for host and device.
#pragma once
#include <cstdint>

#include "ltl.h"
#include "ltl_types.h"

#ifdef __CUDACC__
#define LTL_HD __host__ __device__
#else
#define LTL_HD
#endif

namespace ltl {

// Cost of each connective (index = op; atoms at OP_ATOM), 0 read as 1.
struct Costs {
    int c[8];
};

LTL_HD inline uint64_t plan_pow2_ceil(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

LTL_HD inline uint64_t plan_min(uint64_t a, uint64_t b) { return a < b ? a : b; }
LTL_HD inline uint64_t plan_max(uint64_t a, uint64_t b) { return a > b ? a : b; }

// Tile extents for a launch of `cands` candidates on `slots` resident CTAs:
// about `tiles_per_cta` tiles per CTA, never fewer than `nb` candidates per tile.
LTL_HD inline uint32_t tile_target(uint64_t cands, uint64_t slots, int nb, int tiles_per_cta) {
    uint64_t cpt = cands / plan_max(1, (uint64_t)tiles_per_cta * slots);
    cpt = plan_max(cpt, (uint64_t)nb);
    return (uint32_t)plan_min(plan_pow2_ceil(cpt), (uint64_t)kTileA * kTileB);
}

LTL_HD inline void set_tiles(Seg &s, uint32_t cpt) {
    if (s.kind == SEG_UNARY) {
        s.ta = (uint32_t)plan_min(cpt, kTileU);
        s.tb = 1;
        s.n_tiles = (s.a_count + s.ta - 1) / s.ta;
        return;
    }
    if (s.kind == SEG_TRI) {
        uint32_t side = 2;
        while (side < kTileA && side * side < cpt) side *= 2;
        s.ta = s.tb = side;
        s.n_ta = s.n_tb = (uint32_t)((s.a_count + side - 1) / side);
        s.n_tiles = (uint64_t)s.n_ta * (s.n_ta + 1) / 2;
        return;
    }
    s.tb = (uint32_t)plan_min(cpt, kTileB);
    s.ta = (uint32_t)plan_max(1, plan_min(cpt / s.tb, kTileA));
    s.n_ta = (uint32_t)((s.a_count + s.ta - 1) / s.ta);
    s.n_tb = (uint32_t)((s.b_count + s.tb - 1) / s.tb);
    s.n_tiles = (uint64_t)s.n_ta * s.n_tb;
    s.a_inner = s.n_ta <= s.n_tb ? 1 : 0;
}

LTL_HD inline uint64_t seg_candidates(const Seg &s) {
    if (s.kind == SEG_UNARY) return s.a_count;
    if (s.kind == SEG_TRI) return s.a_count * (s.a_count - 1) / 2;
    return s.a_count * s.b_count;
}

// Candidate space of cost level k of one problem (Section 3, handleOp, with the
// cost homomorphism of Section 2; uniform cost = size), in the paper's
// connective order F, U, G, X, And, Or, Not: one segment per unary connective
// (all formulas of level k - cost) and one per split of a binary one (U over
// ordered splits, And and Or over splits i <= j with unordered pairs when
// i == j).  lvl_begin / lvl_count give each earlier level's entries.  `emit`
// receives each segment with op, kind and operand ranges set.
template <class Emit>
LTL_HD inline void plan_level_segments(uint32_t ops, int n_props, const uint64_t *lvl_begin, const uint64_t *lvl_count,
                                       int k, const Costs &cost, Emit &emit) {
    if (k == cost.c[OP_ATOM]) {
        Seg sg{};
        sg.op = OP_ATOM; sg.kind = SEG_UNARY; sg.a_begin = 0; sg.a_count = (uint64_t)n_props;
        emit(sg);
        return;   // no other formula has the atoms' cost
    }
    const int order[7] = {OP_F, OP_U, OP_G, OP_X, OP_AND, OP_OR, OP_NOT};
    const uint32_t bit[8] = {0, LTL_NOT, LTL_AND, LTL_OR, LTL_X, LTL_F, LTL_G, LTL_U};
    for (int oi = 0; oi < 7; ++oi) {
        const int op = order[oi];
        if (!(ops & bit[op])) continue;
        const int rest = k - cost.c[op];
        if (op == OP_F || op == OP_G || op == OP_X || op == OP_NOT) {
            if (rest < 1) continue;
            if (op == OP_NOT && (ops & LTL_NNF) && rest != cost.c[OP_ATOM]) continue;   // atoms only
            const uint64_t cnt = lvl_count[rest];
            if (!cnt) continue;
            Seg sg{};
            sg.op = op; sg.kind = SEG_UNARY; sg.a_begin = lvl_begin[rest]; sg.a_count = cnt;
            emit(sg);
            continue;
        }
        for (int cl = 1; cl <= rest - 1; ++cl) {
            const int cr = rest - cl;
            if (op != OP_U && cl > cr) continue;
            const uint64_t na = lvl_count[cl], nb = lvl_count[cr];
            if (!na || !nb) continue;
            Seg sg{};
            sg.op = op; sg.a_begin = lvl_begin[cl]; sg.a_count = na; sg.b_begin = lvl_begin[cr]; sg.b_count = nb;
            if (op != OP_U && cl == cr) {
                if (na < 2) continue;
                sg.kind = SEG_TRI;
            } else {
                sg.kind = SEG_RECT;
            }
            emit(sg);
        }
    }
}

// ----------------------------------------------------------------------------
// Device planning of a chain of small levels.  The host enqueues, per level,
// the planner and then one persistent launch per connective (group), and
// after the chain one more planner call that only closes the last level; one
// read-back then returns every level's log.
// ----------------------------------------------------------------------------
constexpr int kPlanGroups = 8;          // launches per level: atoms or the seven connectives
constexpr int kPlanSegsPerGroup = 64;   // segments per launch (binary splits of one level)

// Level table of the problem, continued on the device.
struct PlanState {
    uint64_t lvl_begin[kMaxLevels];
    uint64_t lvl_count[kMaxLevels];
    int32_t halted;   // a closed level ended the search: later levels plan nothing
    int32_t pad;
};

// What the host needs to close one level exactly as it closes a host-planned one.
struct PlanLog {
    Ctrl snap;         // control block when the level was closed
    uint64_t begin;    // first cache entry of the level
    uint64_t count;    // entries the level added
    uint64_t n_segs;   // segments planned (0: no candidate of this size)
    int32_t ran;       // 1: planned (0: the chain had halted before it)
    int32_t pad;
    uint64_t t_begin;  // device clock (ns) when the level was planned
    uint64_t t_end;    // device clock (ns) when it was closed
};

struct PlanArgs {
    const Problem *prob;               // the problem's device descriptor
    PlanState *state;
    PlanLog *log;                      // indexed by level
    Seg *segs;                         // group g's segments at segs + g * kPlanSegsPerGroup
    LevelDesc *desc;                   // per group: segments and tiles of its launch
    unsigned long long *counters;      // per group: tile counter, zeroed by the planner
    Costs cost;
    uint32_t ops;
    int32_t n_props;
    int32_t stop_mode;                 // LTL_STOP_*
    int32_t prob_index;                // Seg::prob of the problem
    int32_t n_groups;
    int32_t group_op[kPlanGroups];     // connective of each launch
    uint32_t group_cap[kPlanGroups];   // CTAs of each launch
    int32_t nb;                        // candidates per batch of the level kernel
    int32_t tiles_per_cta;
};

}  // namespace ltl
