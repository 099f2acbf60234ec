// ltl_autotune.h -- online tuning of the size-level launches.
//
// A level launch is a persistent grid whose CTAs pull tiles from a counter.
// Two choices decide its shape: how many tiles each resident CTA gets on
// average (fewer, larger tiles amortise the tile fetch and keep the left
// operand staged longer; more, smaller tiles balance the tail) and how many
// CTAs per SM run (the occupancy maximum, or one fewer when resident CTAs
// compete for L1, shared memory bandwidth or the hash-set atomics).  The tuner
// measures each choice on real launches -- per launch class: kernel shape,
// connective and candidate-count bucket -- with the launches' own CUDA-event
// times, and then keeps the fastest (time per candidate).  Only launches that
// run alone (not the concurrent launches of small levels) and carry enough
// candidates for a stable time are tuned.
#pragma once
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>

namespace ltl {

constexpr int kTuneConfigs = 6;
constexpr int kTuneDefault = 1;                  // 4 tiles per CTA, full occupancy
constexpr uint64_t kTuneMinCands = 1ull << 14;   // smaller launches keep the default

struct TuneChoice {
    int tiles_per_cta;   // tiles per resident CTA the tile size aims at
    int cta_less;        // resident CTAs per SM: the occupancy maximum minus this
};

inline TuneChoice tune_choice(int c) {
    static const int tpc[3] = {2, 4, 8};
    return TuneChoice{tpc[c % 3], c / 3};
}

class Tuner {
public:
    bool enabled = false;
    std::string path;   // empty: in memory only

    // The configuration to run for `key`: an untried one first (in order),
    // then the fastest measured.  `allow_less`: one fewer CTA per SM is possible.
    int pick(const std::string &key, bool allow_less) {
        Stat &s = stats[key];
        const int n = allow_less ? kTuneConfigs : kTuneConfigs / 2;
        for (int c = 0; c < n; ++c)
            if (s.tries[c] == 0) return c;
        int best = kTuneDefault;
        double bv = 1e300;
        for (int c = 0; c < n; ++c)
            if (s.tries[c] && s.ns_per_cand[c] < bv) {
                bv = s.ns_per_cand[c];
                best = c;
            }
        return best;
    }

    void record(const std::string &key, int c, double ns_per_cand) {
        Stat &s = stats[key];
        if (s.tries[c] == 0 || ns_per_cand < s.ns_per_cand[c]) s.ns_per_cand[c] = ns_per_cand;
        s.tries[c]++;
    }

    // Text form, one line per class: key, then per configuration its best
    // time per candidate in ns (0: untried) and its number of runs.
    std::string dump() const {
        std::string out;
        char buf[96];
        for (const auto &kv : stats) {
            out += kv.first;
            for (int c = 0; c < kTuneConfigs; ++c) {
                snprintf(buf, sizeof buf, " %.4f:%u", kv.second.tries[c] ? kv.second.ns_per_cand[c] : 0.0,
                         kv.second.tries[c]);
                out += buf;
            }
            out += "\n";
        }
        return out;
    }

    void load() {
        if (path.empty()) return;
        FILE *f = fopen(path.c_str(), "r");
        if (!f) return;   // no file yet: start untuned
        char key[128];
        while (fscanf(f, "%127s", key) == 1) {
            Stat s{};
            bool ok = true;
            for (int c = 0; c < kTuneConfigs && ok; ++c) ok = fscanf(f, " %lf:%u", &s.ns_per_cand[c], &s.tries[c]) == 2;
            if (!ok) break;
            stats[key] = s;
        }
        fclose(f);
    }

    void save() const {
        if (path.empty()) return;
        FILE *f = fopen(path.c_str(), "w");
        if (!f) return;
        const std::string text = dump();
        fwrite(text.data(), 1, text.size(), f);
        fclose(f);
    }

private:
    struct Stat {
        double ns_per_cand[kTuneConfigs] = {};
        uint32_t tries[kTuneConfigs] = {};
    };
    std::map<std::string, Stat> stats;
};

}  // namespace ltl
