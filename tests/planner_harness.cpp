// Test harness (host only): the number of candidates of one size level as the
// shared level planner cuts it into segments (paper_2402_12373_gb300/csrc/
// ltl_plan.h, the code both the host planner and the device planner run).
// tests/test_planner_cpu.py builds it with the host C++ compiler and checks
// it against the oracle's candidate counts.
#define __host__
#define __device__
#include "ltl_plan.h"

extern "C" uint64_t level_candidates(uint32_t ops, int n_props, const uint64_t *counts, int k, const int *costs) {
    ltl::Costs c;
    for (int i = 0; i < 8; ++i) c.c[i] = costs[i];
    uint64_t begin[ltl::kMaxLevels] = {}, cnt[ltl::kMaxLevels] = {};
    for (int j = 1; j < k && j < ltl::kMaxLevels; ++j) cnt[j] = counts[j];
    uint64_t total = 0;
    auto emit = [&](ltl::Seg s) { total += ltl::seg_candidates(s); };
    ltl::plan_level_segments(ops, n_props, begin, cnt, k, c, emit);
    return total;
}

// Tiles of one segment for a target of `cpt` candidates per tile: their count
// and whether they cover exactly the segment's candidates (each candidate in
// one tile, none outside), by walking every tile's candidate range.
extern "C" int tiles_cover(int kind, uint64_t a_count, uint64_t b_count, uint32_t cpt, uint64_t *n_tiles) {
    ltl::Seg s{};
    s.kind = kind;
    s.a_count = a_count;
    s.b_count = b_count;
    ltl::set_tiles(s, cpt);
    *n_tiles = s.n_tiles;
    uint64_t covered = 0;
    if (kind == ltl::SEG_UNARY) {
        for (uint64_t t = 0; t < s.n_tiles; ++t) {
            const uint64_t a0 = t * s.ta, a1 = a0 + s.ta < a_count ? a0 + s.ta : a_count;
            if (a0 >= a1) return 0;
            covered += a1 - a0;
        }
    } else if (kind == ltl::SEG_RECT) {
        for (uint64_t ia = 0; ia < s.n_ta; ++ia)
            for (uint64_t ib = 0; ib < s.n_tb; ++ib) {
                const uint64_t a0 = ia * s.ta, a1 = a0 + s.ta < a_count ? a0 + s.ta : a_count;
                const uint64_t b0 = ib * s.tb, b1 = b0 + s.tb < b_count ? b0 + s.tb : b_count;
                if (a0 >= a1 || b0 >= b1) return 0;
                covered += (a1 - a0) * (b1 - b0);
            }
        if (s.n_tiles != (uint64_t)s.n_ta * s.n_tb) return 0;
    } else {   // pairs a < b, tiles on and above the diagonal
        uint64_t tiles = 0;
        for (uint64_t ia = 0; ia < s.n_ta; ++ia)
            for (uint64_t ib = ia; ib < s.n_tb; ++ib) {
                ++tiles;
                const uint64_t a0 = ia * s.ta, a1 = a0 + s.ta < a_count ? a0 + s.ta : a_count;
                const uint64_t b0 = ib * s.tb, b1 = b0 + s.tb < a_count ? b0 + s.tb : a_count;
                for (uint64_t a = a0; a < a1; ++a)
                    for (uint64_t b = (b0 > a + 1 ? b0 : a + 1); b < b1; ++b) ++covered;
            }
        if (tiles != s.n_tiles) return 0;
    }
    return covered == ltl::seg_candidates(s) ? 1 : 0;
}
