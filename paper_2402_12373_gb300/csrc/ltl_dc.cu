// ltl_dc.cu -- the divide-and-conquer unit of Section 6 over the batched
// enumerator.
//
// A specification with more than `window` traces is split into
// sub-specifications; each one that fits the window is learned by the
// enumerator, and the partial formulae are combined as
// (f11 & f12) | (f21 & f22).  Deterministic splitting halves P and N in list
// order and learns the four parts one after another, each restricted by what
// the earlier parts already decide; random splitting learns f11 on a random
// balanced sample of at most `window` traces and then the three remaining
// parts (independent of each other) concurrently.  When the enumerator finds
// no formula within max_size or its memory, a sub-specification with a single
// positive trace is closed by that trace's overfitting formula (the fallback
// of Section 3); otherwise its window is halved, and a sub-specification of
// one positive and one negative trace that still fails is closed by a formula
// that distinguishes the two traces.
//
// Every sub-specification that is ready is queued on one batch runner, so the
// enumerations of independent parts share launches (continuous batching).
// Language membership of a partial formula is computed on the device for all
// traces at once: the traces are packed once, and each formula is one run of
// the evaluation kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "ltl_device.cuh"
#include "ltl_internal.h"

namespace ltl {
namespace {

// ------------------------------------------------------------ partial formulae

// A formula, or one of the constants true / false that the combination
// simplifies away (the grammar has no constants; see `to_text`).
struct Fml {
    enum Kind { TEXT, TRUE_, FALSE_ } kind = TEXT;
    std::string text;
};

Fml f_true() { return Fml{Fml::TRUE_, {}}; }
Fml f_false() { return Fml{Fml::FALSE_, {}}; }
Fml f_text(std::string s) { return Fml{Fml::TEXT, std::move(s)}; }

Fml f_and(const Fml &a, const Fml &b) {
    if (a.kind == Fml::FALSE_ || b.kind == Fml::FALSE_) return f_false();
    if (a.kind == Fml::TRUE_) return b;
    if (b.kind == Fml::TRUE_) return a;
    return f_text("(" + a.text + " & " + b.text + ")");
}

Fml f_or(const Fml &a, const Fml &b) {
    if (a.kind == Fml::TRUE_ || b.kind == Fml::TRUE_) return f_true();
    if (a.kind == Fml::FALSE_) return b;
    if (b.kind == Fml::FALSE_) return a;
    return f_text("(" + a.text + " | " + b.text + ")");
}

// The constants as formulae of the grammar (needed only when the whole
// specification has no negative or no positive trace).
std::string to_text(const Fml &f) {
    if (f.kind == Fml::TRUE_) return "(p0 | !p0)";
    if (f.kind == Fml::FALSE_) return "(p0 & !p0)";
    return f.text;
}

// Syntax-tree nodes of formula text: atoms plus connectives.
uint64_t text_size(const std::string &s) {
    uint64_t n = 0;
    for (char c : s) n += (c == 'p' || c == '!' || c == 'X' || c == 'F' || c == 'G' || c == '&' || c == '|' || c == 'U');
    return n;
}

// ------------------------------------------------------------ membership

// All traces of the specification packed once on the device (positives,
// then negatives); `member` evaluates a formula at position 0 of every trace
// with the evaluation kernel.
class Membership {
public:
    ~Membership() { release(); }

    ltl_status init(const std::vector<uint32_t> &letters, const std::vector<uint64_t> &offsets, int n_props,
                    cudaStream_t stream) {
        sm = stream;
        n_props_ = n_props;
        T = offsets.size() - 1;
        uint64_t ml = 0;
        for (uint64_t t = 0; t < T; ++t) ml = std::max<uint64_t>(ml, offsets[t + 1] - offsets[t]);
        const int W = (int)std::max<uint64_t>(1, (ml + 63) / 64);
        Wt = (int)pow2_ceil((uint64_t)W);
        if (Wt > 16) return fail(LTL_ERR_INVALID, "divide and conquer supports traces up to 1024 positions");
        nsteps = ceil_log2(ml);
        plane = round_up(std::max<uint64_t>(T, 1), 128);
        stride = (uint64_t)Wt * plane;
        const uint64_t total = offsets[T];
        size_t o = 0;
        auto take = [&](size_t b) {
            const size_t r = o;
            o = round_up(o + b, 256);
            return r;
        };
        o_ctrl = take(sizeof(Ctrl));
        o_let = take(4 * std::max<uint64_t>(total, 1));
        o_off = take(8 * (T + 1));
        o_mask = take(8 * stride);
        o_atoms = take(8 * stride * (uint64_t)n_props);
        o_out = take(8 * std::max<uint64_t>(T, 1));
        ltl_status s = grow(&base, base_bytes, o);
        if (s != LTL_OK) return s;
        LTL_CUDA_TRY(cudaMemsetAsync(base, 0, o, sm));
        if (total) LTL_CUDA_TRY(cudaMemcpyAsync(base + o_let, letters.data(), 4 * total, cudaMemcpyHostToDevice, sm));
        LTL_CUDA_TRY(cudaMemcpyAsync(base + o_off, offsets.data(), 8 * (T + 1), cudaMemcpyHostToDevice, sm));
        LTL_CUDA_TRY(launch_pack((const uint32_t *)(base + o_let), (const uint64_t *)(base + o_off), (uint32_t)T, plane,
                                 W, Wt, n_props, (uint64_t *)(base + o_mask), (uint64_t *)(base + o_atoms), stride,
                                 (Ctrl *)(base + o_ctrl), sm));
        Ctrl h;
        LTL_CUDA_TRY(cudaMemcpyAsync(&h, base + o_ctrl, sizeof h, cudaMemcpyDeviceToHost, sm));
        LTL_CUDA_TRY(cudaStreamSynchronize(sm));
        if (h.invalid_letter) return fail(LTL_ERR_INVALID, "trace letters use propositions >= n_props");
        return LTL_OK;
    }

    // at0[t] = 1 iff trace t satisfies f at position 0
    ltl_status member(const Fml &f, std::vector<uint8_t> &at0) {
        at0.assign(T, f.kind == Fml::TRUE_ ? 1 : 0);
        if (f.kind != Fml::TEXT || T == 0) return LTL_OK;
        std::vector<uint32_t> prog;
        int depth = 0, max_atom = -1;
        if (!compile_formula(f.text.c_str(), n_props_, prog, depth, max_atom))
            return fail(LTL_ERR_INVALID, "internal: cannot compile a partial formula");
        ltl_status s = grow(&prog_d, prog_bytes, 4 * prog.size());
        if (s != LTL_OK) return s;
        s = grow(&stack_d, stack_bytes, 8 * stride * (uint64_t)std::max(depth, 1));
        if (s != LTL_OK) return s;
        LTL_CUDA_TRY(cudaMemcpyAsync(prog_d, prog.data(), 4 * prog.size(), cudaMemcpyHostToDevice, sm));
        LTL_CUDA_TRY(launch_eval(Wt, (const uint32_t *)prog_d, (int)prog.size(), (const uint64_t *)(base + o_atoms),
                                 (const uint64_t *)(base + o_mask), stride, plane, (uint64_t *)stack_d, nsteps,
                                 (uint32_t)T, (uint64_t *)(base + o_out), 1, sm));
        host.resize(T);
        LTL_CUDA_TRY(cudaMemcpyAsync(host.data(), base + o_out, 8 * T, cudaMemcpyDeviceToHost, sm));
        LTL_CUDA_TRY(cudaStreamSynchronize(sm));
        for (uint64_t t = 0; t < T; ++t) at0[t] = (uint8_t)(host[t] & 1ull);
        ++evals;
        return LTL_OK;
    }

    uint64_t evals = 0;

private:
    ltl_status grow(char **p, size_t &have, size_t need) {
        if (*p && have >= need) return LTL_OK;
        if (*p) cudaFreeAsync(*p, sm);
        *p = nullptr;
        have = 0;
        cudaError_t e = cudaMallocAsync((void **)p, std::max<size_t>(need, 256), sm);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            *p = nullptr;
            return fail(LTL_ERR_OOM, "cudaMallocAsync(%zu) failed", need);
        }
        have = std::max<size_t>(need, 256);
        return LTL_OK;
    }
    void release() {
        for (char **p : {&base, &prog_d, &stack_d})
            if (*p) cudaFreeAsync(*p, sm);
        if (sm) cudaStreamSynchronize(sm);
        base = prog_d = stack_d = nullptr;
        (void)cudaGetLastError();
    }

    cudaStream_t sm = nullptr;
    char *base = nullptr, *prog_d = nullptr, *stack_d = nullptr;
    size_t base_bytes = 0, prog_bytes = 0, stack_bytes = 0;
    size_t o_ctrl = 0, o_let = 0, o_off = 0, o_mask = 0, o_atoms = 0, o_out = 0;
    uint64_t T = 0, plane = 0, stride = 0;
    int Wt = 1, nsteps = 0, n_props_ = 1;
    std::vector<uint64_t> host;
};

// ------------------------------------------------------------ the split tree

using Idx = std::vector<uint32_t>;   // trace indices: positives [0, nP), negatives [nP, nP + nN)

struct Node {
    int mode = LTL_DC_DETERMINISTIC;
    Idx P, N;
    uint64_t win = 2;
    int parent = -1, which = -1, depth = 0;
    int stage = 0;      // deterministic: next part to learn (0..3); random: parts outstanding
    Fml f[4];           // f11, f12, f21, f22
    Idx P0, N0;         // the sample sent to the enumerator
    Idx P2r;            // deterministic: P2 without the positives the first disjunct accepts
    std::vector<uint8_t> L11;
    std::vector<uint32_t> leaf_l[2];   // gathered traces of the queued enumeration
    std::vector<uint64_t> leaf_o[2];
};

class DivideAndConquer {
public:
    // specification
    std::vector<uint32_t> letters;
    std::vector<uint64_t> offsets;
    uint64_t nP = 0, nN = 0;
    int n_props = 1;
    uint32_t ops = LTL_ALL;
    int max_size = 1;
    uint64_t seed_state = 0;
    // machinery
    BatchRunner *runner = nullptr;
    Membership mem;
    std::deque<Node> nodes;
    std::unordered_map<uint64_t, int> leaf_owner;
    uint64_t next_leaf = 0;
    ltl_dc_stats st{};
    Fml result;
    bool have_result = false;
    ltl_status error = LTL_OK;

    ltl_status run(int mode, uint64_t window) {
        Idx P(nP), N(nN);
        for (uint64_t i = 0; i < nP; ++i) P[i] = (uint32_t)i;
        for (uint64_t i = 0; i < nN; ++i) N[i] = (uint32_t)(nP + i);
        st.min_window = window;
        ltl_status s = spawn(mode, std::move(P), std::move(N), window, -1, -1, 0);
        std::vector<ltl_result> done;
        while (s == LTL_OK && !have_result && runner_busy(runner)) {
            s = runner_step(runner, done);
            for (const ltl_result &r : done) {
                if (s != LTL_OK) break;
                auto it = leaf_owner.find(r.id);
                if (it == leaf_owner.end()) continue;
                const int ni = it->second;
                leaf_owner.erase(it);
                s = on_leaf(ni, r);
            }
            done.clear();
        }
        if (s != LTL_OK) return s;
        if (!have_result) return fail(LTL_ERR_INVALID, "internal: divide and conquer ended without a result");
        st.rounds = runner_rounds(runner);
        st.evals = mem.evals;
        return LTL_OK;
    }

private:
    uint64_t rnd() {   // SplitMix64 (Steele, Lea & Flood 2014)
        seed_state += 0x9E3779B97F4A7C15ull;
        return mix64(seed_state);
    }

    // a random subset of k of the indices (partial Fisher-Yates)
    Idx sample(const Idx &from, size_t k) {
        Idx v = from;
        for (size_t i = 0; i < k && i + 1 < v.size(); ++i) {
            const size_t j = i + (size_t)(rnd() % (uint64_t)(v.size() - i));
            std::swap(v[i], v[j]);
        }
        v.resize(std::min(k, v.size()));
        std::sort(v.begin(), v.end());
        return v;
    }

    ltl_status spawn(int mode, Idx P, Idx N, uint64_t win, int parent, int which, int depth) {
        nodes.emplace_back();
        const int ni = (int)nodes.size() - 1;
        Node &n = nodes.back();
        n.mode = mode;
        n.P = std::move(P);
        n.N = std::move(N);
        n.win = win;
        n.parent = parent;
        n.which = which;
        n.depth = depth;
        return start(ni);
    }

    ltl_status start(int ni) {
        Node &n = nodes[ni];
        if (n.N.empty()) return finish(ni, f_true());
        if (n.P.empty()) return finish(ni, f_false());
        const uint64_t card = n.P.size() + n.N.size();
        if (n.mode == LTL_DC_DETERMINISTIC) {
            if (card <= n.win) {
                n.P0 = n.P;
                n.N0 = n.N;
                return enumerate(ni);
            }
            n.stage = 0;
            st.max_depth = std::max(st.max_depth, n.depth);   // depth of parts that do work
            const size_t hp = (n.P.size() + 1) / 2, hn = (n.N.size() + 1) / 2;
            Idx P1(n.P.begin(), n.P.begin() + hp), N1(n.N.begin(), n.N.begin() + hn);
            return spawn(n.mode, std::move(P1), std::move(N1), n.win, ni, 0, n.depth + 1);
        }
        // random splitting: f11 from a balanced random sample of the window
        const uint64_t m = std::min<uint64_t>(n.win, card);
        size_t kp = std::min<size_t>(n.P.size(), (size_t)((m + 1) / 2));
        const size_t kn = std::min<size_t>(n.N.size(), (size_t)(m - kp));
        kp = std::min<size_t>(n.P.size(), (size_t)(m - kn));
        n.P0 = card <= m ? n.P : sample(n.P, kp);
        n.N0 = card <= m ? n.N : sample(n.N, kn);
        return enumerate(ni);
    }

    // queues the enumeration of (P0, N0) of node ni
    ltl_status enumerate(int ni) {
        Node &n = nodes[ni];
        const Idx *side[2] = {&n.P0, &n.N0};
        ltl_traces tr[2];
        for (int h = 0; h < 2; ++h) {
            n.leaf_l[h].clear();
            n.leaf_o[h].assign(1, 0);
            for (uint32_t t : *side[h]) {
                n.leaf_l[h].insert(n.leaf_l[h].end(), letters.begin() + offsets[t], letters.begin() + offsets[t + 1]);
                n.leaf_o[h].push_back(n.leaf_l[h].size());
            }
            if (n.leaf_l[h].empty()) n.leaf_l[h].push_back(0);
            tr[h].letters = n.leaf_l[h].data();
            tr[h].offsets = n.leaf_o[h].data();
            tr[h].n_traces = side[h]->size();
        }
        st.max_depth = std::max(st.max_depth, n.depth);
        const uint64_t id = next_leaf++;
        leaf_owner[id] = ni;
        st.enum_calls++;
        return runner_submit(runner, tr[0], tr[1], n_props, ops, max_size, 0, id, false);
    }

    ltl_status on_leaf(int ni, const ltl_result &r) {
        Node &n = nodes[ni];
        n.leaf_l[0].clear(); n.leaf_l[1].clear(); n.leaf_o[0].clear(); n.leaf_o[1].clear();
        if (r.status < 0 && r.status != LTL_ERR_OOM) return fail(r.status, "enumeration of a sub-specification failed");
        const uint64_t card = n.P0.size() + n.N0.size();
        if (r.status == LTL_OK) return learned(ni, f_text(r.formula));
        st.enum_failed++;
        if (n.P.size() == 1) {
            // one positive trace: its overfitting formula rejects every
            // negative of the part at once (Section 3's fallback)
            Fml f;
            if (overfit(n.P[0], n.N, f)) {
                st.fallbacks++;
                return learned(ni, f);
            }
        }
        if (card <= 2) {
            // one positive, one negative: the distinguishing formula
            Fml f;
            ltl_status s = distinguish(n.P0, n.N0, f);
            if (s != LTL_OK) return s;
            st.fallbacks++;
            return learned(ni, f);
        }
        n.win = std::max<uint64_t>(2, std::min<uint64_t>(n.win, card) / 2);
        st.min_window = std::min(st.min_window, n.win);
        return start(ni);
    }

    // the enumerator (or the fallback) produced a formula for (P0, N0)
    ltl_status learned(int ni, Fml f) {
        if (nodes[ni].mode == LTL_DC_DETERMINISTIC) return finish(ni, std::move(f));
        Node &n = nodes[ni];
        n.f[0] = std::move(f);
        std::vector<uint8_t> L;
        ltl_status s = mem.member(n.f[0], L);
        if (s != LTL_OK) return s;
        Idx Pin, Pout, Nin, Nout;
        for (uint32_t t : n.P) (L[t] ? Pin : Pout).push_back(t);
        for (uint32_t t : n.N) (L[t] ? Nin : Nout).push_back(t);
        n.stage = 3;
        const int mode = n.mode, depth = n.depth + 1;
        const uint64_t win = n.win;
        // f12 on L(f11), f21 outside it, f22: positives outside against negatives inside
        s = spawn(mode, Pin, Nin, win, ni, 1, depth);
        if (s != LTL_OK) return s;
        s = spawn(mode, Pout, std::move(Nout), win, ni, 2, depth);
        if (s != LTL_OK) return s;
        return spawn(mode, std::move(Pout), std::move(Nin), win, ni, 3, depth);
    }

    ltl_status finish(int ni, Fml f) {
        const int parent = nodes[ni].parent, which = nodes[ni].which;
        nodes[ni].P.clear(); nodes[ni].N.clear(); nodes[ni].P0.clear(); nodes[ni].N0.clear();
        if (parent < 0) {
            result = std::move(f);
            have_result = true;
            return LTL_OK;
        }
        return child_done(parent, which, std::move(f));
    }

    ltl_status child_done(int pi, int which, Fml f) {
        Node &p = nodes[pi];
        p.f[which] = std::move(f);
        if (p.mode == LTL_DC_RANDOM) {
            if (--p.stage > 0) return LTL_OK;
            return finish(pi, f_or(f_and(p.f[0], p.f[1]), f_and(p.f[2], p.f[3])));
        }
        // deterministic: the four parts in order, each restricted by the earlier ones
        const size_t hp = (p.P.size() + 1) / 2, hn = (p.N.size() + 1) / 2;
        const Idx P1(p.P.begin(), p.P.begin() + hp), P2(p.P.begin() + hp, p.P.end());
        const Idx N1(p.N.begin(), p.N.begin() + hn), N2(p.N.begin() + hn, p.N.end());
        const int depth = p.depth + 1, mode = p.mode;
        const uint64_t win = p.win;
        std::vector<uint8_t> L;
        ltl_status s;
        switch (which) {
        case 0: {   // f12 = DS(P1, N2 ∩ L(f11))
            s = mem.member(p.f[0], p.L11);
            if (s != LTL_OK) return s;
            Idx N2in;
            for (uint32_t t : N2)
                if (p.L11[t]) N2in.push_back(t);
            return spawn(mode, P1, std::move(N2in), win, pi, 1, depth);
        }
        case 1: {   // f21 = DS(P2 \ L(f11 & f12), N1)
            s = mem.member(p.f[1], L);
            if (s != LTL_OK) return s;
            p.P2r.clear();
            for (uint32_t t : P2)
                if (!(p.L11[t] && L[t])) p.P2r.push_back(t);
            p.L11.clear();
            return spawn(mode, p.P2r, N1, win, pi, 2, depth);
        }
        case 2: {   // f22 = DS(P2 \ L(f11 & f12), N2 ∩ L(f21))
            s = mem.member(p.f[2], L);
            if (s != LTL_OK) return s;
            Idx N2in;
            for (uint32_t t : N2)
                if (L[t]) N2in.push_back(t);
            Idx P2r = std::move(p.P2r);
            return spawn(mode, std::move(P2r), std::move(N2in), win, pi, 3, depth);
        }
        default:
            return finish(pi, f_or(f_and(p.f[0], p.f[1]), f_and(p.f[2], p.f[3])));
        }
    }

    // The overfitting formula of trace p: its letter at every position, under
    // nested X's, (l_0 & X (l_1 & X ( ... l_{n-1}))), l_i the conjunction of the
    // propositions' literals at position i; when a negative extends p, also
    // "no position after the last": l_{n-1} & !X (p0 | !p0).  It holds at
    // position 0 of p and of no negative.  False when it does not apply (a
    // negative equal to p; a negative extending p under NNF; a connective it
    // needs is not allowed).
    bool overfit(uint32_t p, const Idx &N, Fml &out) {
        const bool has_not = (ops & LTL_NOT) != 0, nnf = (ops & LTL_NNF) != 0;
        const uint64_t lp = offsets[p + 1] - offsets[p];
        if (lp == 0 || (lp > 1 && !(ops & LTL_X))) return false;
        bool need_end = false;   // some negative extends p: say that p ends
        for (uint32_t q : N) {
            const uint64_t lq = offsets[q + 1] - offsets[q];
            if (lq < lp) continue;
            bool prefix = true;
            for (uint64_t i = 0; i < lp && prefix; ++i) prefix = letters[offsets[p] + i] == letters[offsets[q] + i];
            if (prefix && lq == lp) return false;
            need_end |= prefix;
        }
        if (need_end && (nnf || !has_not)) return false;
        std::string f;
        for (uint64_t i = lp; i-- > 0;) {
            const uint32_t a = letters[offsets[p] + i];
            std::string lam;
            for (int b = n_props - 1; b >= 0; --b) {
                const bool pos = (a >> b) & 1u;
                if (!pos && !has_not) return false;
                const std::string lit = std::string(pos ? "" : "!") + "p" + std::to_string(b);
                lam = lam.empty() ? lit : "(" + lit + " & " + lam + ")";
            }
            if (i + 1 == lp) {
                f = need_end ? "(" + lam + " & !X (p0 | !p0))" : lam;
            } else {
                f = "(" + lam + " & X " + f + ")";
            }
        }
        out = f_text(f);
        return true;
    }

    // A formula true at position 0 of every positive and false on every
    // negative of a small sub-specification, built from the traces: for each
    // positive p, the conjunction over negatives n of a formula telling p from
    // n (the first position where they differ, by a literal under X's; or the
    // end of the shorter trace); the disjunction over positives.
    ltl_status distinguish(const Idx &P, const Idx &N, Fml &out) {
        const bool has_x = ops & LTL_X, has_not = (ops & LTL_NOT) != 0, nnf = (ops & LTL_NNF) != 0;
        Fml all = f_false();
        for (uint32_t p : P) {
            Fml conj = f_true();
            const uint64_t lp = offsets[p + 1] - offsets[p];
            for (uint32_t q : N) {
                const uint64_t lq = offsets[q + 1] - offsets[q];
                const uint64_t m = std::min(lp, lq);
                uint64_t i = 0;
                while (i < m && letters[offsets[p] + i] == letters[offsets[q] + i]) ++i;
                std::string f;
                if (i < m) {
                    const uint32_t d = letters[offsets[p] + i] ^ letters[offsets[q] + i];
                    int b = 0;
                    while (!((d >> b) & 1u)) ++b;
                    const bool pos = (letters[offsets[p] + i] >> b) & 1u;
                    if (!pos && !has_not) return fail(LTL_NOT_FOUND, "no formula: a trace pair needs negation");
                    f = std::string(pos ? "" : "!") + "p" + std::to_string(b);
                } else if (lq < lp) {   // q is a proper prefix of p: p has position lq
                    if (!has_not) return fail(LTL_NOT_FOUND, "no formula: a trace pair needs negation");
                    f = "(p0 | !p0)";
                    i = lq;
                } else {
                    if (lp == lq) return fail(LTL_NOT_FOUND, "no formula: a trace is both positive and negative");
                    // p is a proper prefix of q: only "p has no position lp" tells
                    // them apart, i.e. !X^lp (p0 | !p0); an empty p satisfies nothing
                    if (lp == 0) return fail(LTL_NOT_FOUND, "no formula: an empty positive trace satisfies nothing");
                    if (!has_not || nnf)
                        return fail(LTL_NOT_FOUND, "no formula: a positive trace is a prefix of a negative one");
                    if (!has_x) return fail(LTL_NOT_FOUND, "no formula: telling two traces apart needs X");
                    std::string x;
                    for (uint64_t k = 0; k < lp; ++k) x += "X ";
                    f = "!" + x + "(p0 | !p0)";
                    i = 0;
                }
                if (i > 0 && !has_x) return fail(LTL_NOT_FOUND, "no formula: telling two traces apart needs X");
                std::string g;
                for (uint64_t k = 0; k < i; ++k) g += "X ";
                conj = f_and(conj, f_text(g + f));
            }
            all = f_or(all, conj);
        }
        out = all;
        return LTL_OK;
    }
};

}  // namespace
}  // namespace ltl

using namespace ltl;

extern "C" ltl_status ltl_learn_dc(const ltl_traces *P, const ltl_traces *N, int n_props, uint32_t ops,
                                   int max_size, const ltl_opts *opts, const ltl_dc_opts *dc, char *formula_out,
                                   size_t formula_cap, ltl_dc_stats *stats) {
    const double t0 = wall_ms();
    if (stats) memset(stats, 0, sizeof *stats);
    if (formula_out && formula_cap) formula_out[0] = '\0';
    ltl_status s = check_common(n_props, ops, max_size);
    if (s != LTL_OK) return s;
    if ((s = check_traces(P, "P")) != LTL_OK) return s;
    if ((s = check_traces(N, "N")) != LTL_OK) return s;
    if (!dc) return fail(LTL_ERR_INVALID, "dc options are NULL");
    if (dc->mode != LTL_DC_DETERMINISTIC && dc->mode != LTL_DC_RANDOM) return fail(LTL_ERR_INVALID, "unknown split mode");
    if (dc->window < 2) return fail(LTL_ERR_INVALID, "the split window must be at least 2");
    if ((ops & (LTL_AND | LTL_OR)) != (LTL_AND | LTL_OR))
        return fail(LTL_ERR_INVALID, "divide and conquer combines with & and |: ops must allow both");
    ltl_opts o;
    if (opts) o = *opts;
    else {
        memset(&o, 0, sizeof o);
    }
    if (o.max_errors) return fail(LTL_ERR_INVALID, "divide and conquer needs exact separation (max_errors = 0)");
    o.stop_on_solution = LTL_STOP_FIRST;

    const int resident = dc->max_resident > 0 ? std::min(dc->max_resident, 4096) : 64;
    BatchRunner *r = nullptr;
    s = runner_create(o, resident, resident, &r);
    if (s != LTL_OK) return s;
    // declared after the runner: its device buffers live on the runner's
    // stream and are released before the runner is destroyed
    std::unique_ptr<BatchRunner, void (*)(BatchRunner *)> guard(r, runner_destroy);
    DivideAndConquer d;
    d.nP = P->n_traces;
    d.nN = N->n_traces;
    d.n_props = n_props;
    d.ops = ops;
    d.max_size = max_size;
    d.seed_state = dc->seed;
    const ltl_traces *side[2] = {P, N};
    d.offsets.assign(1, 0);
    for (int h = 0; h < 2; ++h) {
        const uint64_t n = side[h]->offsets[side[h]->n_traces];
        d.letters.insert(d.letters.end(), side[h]->letters, side[h]->letters + n);
        for (uint64_t t = 0; t < side[h]->n_traces; ++t)
            d.offsets.push_back(d.offsets.back() + side[h]->offsets[t + 1] - side[h]->offsets[t]);
    }
    if (d.offsets.size() - 1 > 0xFFFFFFFFull) return fail(LTL_ERR_INVALID, "too many traces");
    d.runner = r;
    s = d.mem.init(d.letters, d.offsets, n_props, runner_stream(r));
    if (s != LTL_OK) return s;
    s = d.run(dc->mode, dc->window);
    if (s != LTL_OK) return s;
    // the combination is sound by construction; check it anyway on every trace
    std::vector<uint8_t> at0;
    s = d.mem.member(d.result, at0);
    if (s != LTL_OK) return s;
    for (uint64_t t = 0; t < d.nP + d.nN; ++t)
        if ((at0[t] != 0) != (t < d.nP))
            return fail(LTL_ERR_INVALID, "internal: the combined formula does not separate trace %llu",
                        (unsigned long long)t);
    const std::string text = to_text(d.result);
    d.st.formula_size = text_size(text);
    d.st.formula_len = text.size();
    d.st.evals = d.mem.evals;
    d.st.total_ms = wall_ms() - t0;
    if (stats) *stats = d.st;
    return write_formula(text, formula_out, formula_cap);
}
