// ltl_host.cu -- host driver and C ABI of the GB300 LTL learner.
//
// Per learn call: validate, lay the problem out in the workspace, pack the
// traces into bit-planes (atoms + length masks), then run the size levels of
// Section 3's `enum` one kernel launch per level (every connective and split
// of the level in one persistent launch), reading back a small control block
// after each level (separator found, cache full, errors, counters).  The
// formula is rebuilt from the provenance of the recorded separator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <string>
#include <vector>

#include "ltl.h"
#include "ltl_types.h"

namespace ltl {
const void *fused_kernel_ptr_w1(int C, int op);
const void *fused_kernel_ptr_w2(int C, int op);
const void *fused_kernel_ptr_w48(int W, int C, int op);
const void *fused_kernel_ptr_narrow(int C, int op);
cudaError_t launch_pack_narrow(const uint32_t *letters, const uint64_t *offsets, uint32_t n_traces, uint64_t plane,
                               int n_props, uint64_t *mask, uint64_t *atoms, uint64_t stride, Ctrl *ctrl,
                               cudaStream_t s);
const void *stream_kernel_ptr(int W, int C);
inline const void *fused_kernel_ptr(int W, int C, int op) {
    return W == 1 ? fused_kernel_ptr_w1(C, op) : W == 2 ? fused_kernel_ptr_w2(C, op) : fused_kernel_ptr_w48(W, C, op);
}
int fused_kernel_batch(int W, int C, bool narrow);
cudaError_t launch_pack(const uint32_t *letters, const uint64_t *offsets, uint32_t n_traces, uint64_t plane,
                        int W, int n_props, uint64_t *mask, uint64_t *atoms, uint64_t stride, Ctrl *ctrl,
                        cudaStream_t s);
cudaError_t launch_keys(uint64_t *keys, uint64_t n, uint64_t seed, cudaStream_t s);
cudaError_t launch_walk(const uint64_t *prov, uint64_t n_entries, uint64_t root_prov, uint32_t *tokens, int cap,
                        int *n_out, cudaStream_t s);
cudaError_t launch_eval(int W, const uint32_t *prog, int n_instr, const uint64_t *atoms, const uint64_t *mask,
                        uint64_t stride, uint64_t plane, uint64_t *stack, int nsteps, uint32_t n_traces,
                        uint64_t *out, int out_words, cudaStream_t s);
}  // namespace ltl

using namespace ltl;

namespace {

thread_local std::string g_err;

ltl_status fail(ltl_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CUDA_TRY(x)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (x);                                                                    \
        if (e_ != cudaSuccess) {                                                                 \
            (void)cudaGetLastError();                                                            \
            return fail(LTL_ERR_CUDA, "%s failed: %s", #x, cudaGetErrorString(e_));              \
        }                                                                                        \
    } while (0)

constexpr uint64_t kKeySeed = 0x243F6A8885A308D3ull;   // NH key stream seed (digits of pi)
constexpr int kMaxSegs = 512;
constexpr int kMaxTokens = 256;

uint64_t round_up(uint64_t x, uint64_t m) { return (x + m - 1) / m * m; }
uint64_t pow2_ceil(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}
int ceil_log2(uint64_t x) {   // smallest k with 2^k >= x (0 for x <= 1)
    int k = 0;
    while ((1ull << k) < x) ++k;
    return k;
}

// ----------------------------------------------------------------- formula text
// f := '!' f | 'X' f | 'F' f | 'G' f | 'p' digits | '(' f ')' | '(' f op f ')'
struct Node {
    int op;
    int a, b;   // children (node ids) or, for atoms, a = proposition
};

struct FormulaParser {
    const char *s;
    std::vector<Node> nodes;
    bool err = false;
    void ws() {
        while (*s == ' ' || *s == '\t' || *s == '\n' || *s == '\r') ++s;
    }
    int node(int op, int a, int b) {
        nodes.push_back(Node{op, a, b});
        return (int)nodes.size() - 1;
    }
    int parse(int depth) {
        if (depth > 200000) { err = true; return -1; }
        ws();
        const char c = *s;
        if (c == '!' || c == 'X' || c == 'F' || c == 'G') {
            ++s;
            const int x = parse(depth + 1);
            if (err) return -1;
            const int op = c == '!' ? OP_NOT : c == 'X' ? OP_X : c == 'F' ? OP_F : OP_G;
            return node(op, x, -1);
        }
        if (c == 'p') {
            ++s;
            if (*s < '0' || *s > '9') { err = true; return -1; }
            long v = 0;
            while (*s >= '0' && *s <= '9') {
                v = v * 10 + (*s - '0');
                if (v > 31) { err = true; return -1; }
                ++s;
            }
            return node(OP_ATOM, (int)v, -1);
        }
        if (c == '(') {
            ++s;
            const int l = parse(depth + 1);
            if (err) return -1;
            ws();
            const char o = *s;
            if (o == ')') { ++s; return l; }
            if (o != '&' && o != '|' && o != 'U') { err = true; return -1; }
            ++s;
            const int r = parse(depth + 1);
            if (err) return -1;
            ws();
            if (*s != ')') { err = true; return -1; }
            ++s;
            return node(o == '&' ? OP_AND : o == '|' ? OP_OR : OP_U, l, r);
        }
        err = true;
        return -1;
    }
};

// Post-order program (op | atom << 8) and the operand-stack depth it needs.
bool compile_formula(const char *text, int n_props, std::vector<uint32_t> &prog, int &depth, int &max_atom) {
    if (!text) return false;
    FormulaParser P{text};
    const int root = P.parse(0);
    P.ws();
    if (P.err || root < 0 || *P.s != '\0') return false;
    prog.clear();
    depth = 0;
    max_atom = -1;
    int sp = 0;
    // iterative post-order over the node DAG (a tree: each parse node used once)
    std::vector<std::pair<int, int>> st;   // (node, state)
    st.push_back({root, 0});
    while (!st.empty()) {
        auto &top = st.back();
        const Node &nd = P.nodes[top.first];
        const bool binary = nd.op == OP_AND || nd.op == OP_OR || nd.op == OP_U;
        if (nd.op == OP_ATOM) {
            if (nd.a >= n_props) return false;
            max_atom = std::max(max_atom, nd.a);
            prog.push_back((uint32_t)OP_ATOM | ((uint32_t)nd.a << 8));
            depth = std::max(depth, ++sp);
            st.pop_back();
            continue;
        }
        if (top.second == 0) {
            top.second = 1;
            st.push_back({nd.a, 0});
            continue;
        }
        if (binary && top.second == 1) {
            top.second = 2;
            st.push_back({nd.b, 0});
            continue;
        }
        prog.push_back((uint32_t)nd.op);
        if (binary) --sp;
        st.pop_back();
    }
    return sp == 1;
}

// Pre-order token list -> text in the library's output syntax.
size_t tokens_to_text(const uint32_t *tok, int n, int i, std::string &out) {
    if (i >= n) return (size_t)n + 1;
    const int op = (int)(tok[i] & 0xffu);
    switch (op) {
    case OP_ATOM: out += "p" + std::to_string(tok[i] >> 8); return (size_t)i + 1;
    case OP_NOT: out += "!"; return tokens_to_text(tok, n, i + 1, out);
    case OP_X: out += "X "; return tokens_to_text(tok, n, i + 1, out);
    case OP_F: out += "F "; return tokens_to_text(tok, n, i + 1, out);
    case OP_G: out += "G "; return tokens_to_text(tok, n, i + 1, out);
    default: break;
    }
    out += "(";
    size_t j = tokens_to_text(tok, n, i + 1, out);
    out += op == OP_AND ? " & " : op == OP_OR ? " | " : " U ";
    j = tokens_to_text(tok, n, (int)j, out);
    out += ")";
    return j;
}

}  // namespace

// ------------------------------------------------------------------- context

struct Layout {
    int W = 0, Wt = 0, C = 0, NT = 0, NB = 1;
    bool narrow = false;   // two traces of <= 32 positions per word
    size_t smem = 0;
    uint32_t G = 0;
    uint32_t n_traces = 0, n_pos = 0;
    int n_props = 0, nsteps = 0;
    uint64_t plane = 0, stride = 0;
    uint64_t hslots = 0, max_entries = 0;
    // byte offsets in the workspace
    size_t o_ctrl, o_segs, o_tokens, o_ntok, o_letters, o_offsets, o_mask, o_keys, o_atoms, o_hkeys, o_hvals,
        o_prov, o_arena, end;
};

struct ltl_ctx {
    ltl_opts opts{};
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    Ctrl *h_ctrl = nullptr;
    Seg *h_segs = nullptr;
    uint32_t *h_tokens = nullptr;
    cudaEvent_t ev[2 * kMaxLevels + 2] = {};
    Layout L;
    bool have_result = false;
    uint64_t lvl_begin[kMaxLevels] = {}, lvl_count[kMaxLevels] = {};
    struct Occ {
        const void *fn;
        int nt;
        size_t smem;
        int blocks;
    };
    std::vector<Occ> occ;
};

namespace {

ltl_status ctx_alloc_ws(ltl_ctx *c, size_t bytes) {
    if (c->ws && c->ws_bytes >= bytes) return LTL_OK;
    if (c->opts.workspace) return fail(LTL_ERR_OOM, "workspace of %zu bytes too small (need %zu)", c->ws_bytes, bytes);
    if (c->ws_owned && c->ws) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (c->opts.free) c->opts.free(c->ws, c->stream, c->opts.user);
        else cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    void *p = nullptr;
    if (c->opts.alloc) {
        p = c->opts.alloc(bytes, c->stream, c->opts.user);
        if (!p) return fail(LTL_ERR_OOM, "allocator callback returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(LTL_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    c->ws = (char *)p;
    c->ws_bytes = bytes;
    c->ws_owned = true;
    return LTL_OK;
}

// Chooses the launch shape and carves the workspace.
ltl_status plan(ltl_ctx *c, uint64_t n_pos, uint64_t n_neg, uint64_t max_len, uint64_t total_pos, bool host_input,
                int n_props, Layout &L) {
    const uint64_t T = n_pos + n_neg;
    if (T > 0x7fffffffull) return fail(LTL_ERR_INVALID, "too many traces (%llu)", (unsigned long long)T);
    L = Layout{};
    L.n_traces = (uint32_t)T;
    L.n_pos = (uint32_t)n_pos;
    L.n_props = n_props;
    L.W = (int)std::max<uint64_t>(1, (max_len + 63) / 64);
    L.Wt = (int)pow2_ceil((uint64_t)L.W);
    if (L.Wt > 8) return fail(LTL_ERR_INVALID, "traces longer than 512 positions are not supported by ltl_learn");
    L.nsteps = ceil_log2(max_len);
    // Each thread holds C pairs of traces x W words (C * W <= 8) of a
    // candidate; a CTA of up to 256 threads holds a whole matrix of up to
    // 4096 / W traces (fused kernel), larger ones go through the two-pass
    // streaming kernel in `G` chunk groups.
    const int Cmax = 8 / L.Wt;
    const uint64_t maxNT = 256;
    const uint64_t pairs = std::max<uint64_t>(1, (T + 1) / 2);
    // narrow layout: every trace fits 32 bits and the matrix fits one CTA;
    // a thread then holds C words of two traces each per 16-byte chunk pair
    const uint64_t quads = std::max<uint64_t>(1, (T + 3) / 4);
    const uint64_t cap_c = c->opts.max_chunks ? pow2_ceil(c->opts.max_chunks) : 8;
    const uint64_t ncmax = std::min<uint64_t>(4, cap_c);
    // the smallest power-of-two thread count >= 32 that holds `units` with at
    // most `cmax` chunks per thread, and the chunk count it then needs
    auto shape = [&](uint64_t units, uint64_t cmax) {
        uint64_t nt = pow2_ceil((units + cmax - 1) / cmax);
        nt = std::min<uint64_t>(std::max<uint64_t>(nt, 32), maxNT);
        L.NT = (int)nt;
        L.C = (int)std::min<uint64_t>(pow2_ceil((units + nt - 1) / nt), cmax);
        L.G = 1;
    };
    if (max_len <= 32 && quads <= maxNT * ncmax) {
        shape(quads, ncmax);                       // narrow, fused
        L.narrow = true;
    } else if (pairs <= maxNT * std::min<uint64_t>(Cmax, cap_c)) {
        shape(pairs, std::min<uint64_t>(Cmax, cap_c));   // wide, fused, capped shape
    } else if (pairs <= maxNT * (uint64_t)Cmax) {
        shape(pairs, (uint64_t)Cmax);              // wide, fused (the cap cannot hold the matrix)
    } else {
        L.NT = (int)maxNT;                         // wide, two-pass streaming, >= 2 groups
        L.C = Cmax;
        L.G = (uint32_t)((pairs + maxNT * Cmax - 1) / (maxNT * Cmax));
    }
    // the batch size the fused kernel of this shape was compiled with (the
    // shared-memory operand slots are sized from it)
    L.NB = L.G == 1 ? fused_kernel_batch(L.Wt, L.C, L.narrow) : 1;
    if (L.G == 1 && L.NB < 1) return fail(LTL_ERR_INVALID, "no fused kernel for W=%d C=%d", L.Wt, L.C);
    L.plane = (uint64_t)L.G * L.C * 2 * L.NT;   // words per bit-plane
    L.stride = (uint64_t)L.Wt * L.plane;
    L.smem = L.G == 1 ? (size_t)(L.NB + 1) * 8 * L.stride : 0;

    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o = round_up(o + bytes, 256);
        return r;
    };
    L.o_ctrl = take(sizeof(Ctrl));
    L.o_segs = take(sizeof(Seg) * kMaxSegs);
    L.o_tokens = take(sizeof(uint32_t) * kMaxTokens);
    L.o_ntok = take(sizeof(int));
    L.o_letters = take(host_input ? sizeof(uint32_t) * std::max<uint64_t>(total_pos, 1) : 0);
    L.o_offsets = take(host_input ? sizeof(uint64_t) * (T + 1) : 0);
    L.o_mask = take(8 * L.stride);
    L.o_keys = take(8 * L.stride);
    L.o_atoms = take(8 * L.stride * (uint64_t)n_props);
    const size_t fixed = o;

    uint64_t budget = c->ws_bytes;
    if (!c->opts.workspace) {
        if (c->opts.mem_budget_bytes) budget = c->opts.mem_budget_bytes + fixed;
        else {
            size_t fr = 0, tot = 0;
            CUDA_TRY(cudaMemGetInfo(&fr, &tot));
            budget = (uint64_t)(0.4 * (double)(fr + (c->ws_owned ? c->ws_bytes : 0)));
        }
    } else if (c->opts.mem_budget_bytes) {
        budget = std::min<uint64_t>(budget, c->opts.mem_budget_bytes + fixed);
    }
    if (budget <= fixed + 4096) return fail(LTL_ERR_OOM, "workspace too small for the problem layout");
    const uint64_t R = budget - fixed - 4096;
    const uint64_t per = 8 * L.stride + 8;   // arena + provenance per entry
    uint64_t E = R / (per + 24);
    uint64_t slots = pow2_ceil(std::max<uint64_t>(2 * E, 1024));
    while (slots * 12 + E * per > R && E > 0) {
        E = (R > slots * 12) ? (R - slots * 12) / per : 0;
        if (slots > 1024 && slots / 2 >= 2 * E) slots /= 2;
    }
    E = std::min<uint64_t>(E, kMaxEntries);
    if (E < 1) return fail(LTL_ERR_OOM, "workspace too small for one cache entry");
    L.max_entries = E;
    L.hslots = slots;
    L.o_hkeys = take(8 * slots);
    L.o_hvals = take(4 * slots);
    L.o_prov = take(8 * E);
    L.o_arena = take(8 * L.stride * E);
    L.end = o;
    ltl_status st = ctx_alloc_ws(c, L.end);
    if (st != LTL_OK) return st;
    return LTL_OK;
}

const void *level_kernel_for(const Layout &L, int op) {
    if (L.narrow) return fused_kernel_ptr_narrow(L.C, op);
    return L.G == 1 ? fused_kernel_ptr(L.Wt, L.C, op) : stream_kernel_ptr(L.Wt, L.C);
}

// Resident CTAs per SM of a layout's kernel for one connective (dynamic
// shared memory opted in); cached per kernel.
ltl_status occupancy(ltl_ctx *c, const Layout &L, int op, int &blocks) {
    const void *fn = level_kernel_for(L, op);
    if (!fn) return fail(LTL_ERR_INVALID, "no kernel for W=%d C=%d", L.Wt, L.C);
    for (const auto &e : c->occ)
        if (e.fn == fn && e.nt == L.NT && e.smem == L.smem) {
            blocks = e.blocks;
            return LTL_OK;
        }
    if (L.smem > 0) CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
    int b = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, L.NT, L.smem));
    if (b < 1) return fail(LTL_ERR_INVALID, "level kernel cannot be resident (threads %d, smem %zu)", L.NT, L.smem);
    c->occ.push_back({fn, L.NT, L.smem, b});
    blocks = b;
    return LTL_OK;
}

// Candidate space of size level k (Section 3, handleOp) as segments, grouped
// by connective in the paper's order F, U, G, X, And, Or, Not.  Each group is
// one launch; tile ids restart at 0 in every group.
struct OpGroup {
    int op;
    int first, count;       // segments [first, first + count) of the level
    uint64_t tiles;
};

// Tile extents for a launch of `cands` candidates on `slots` resident CTAs:
// about four tiles per CTA, never fewer than `nb` candidates per tile.
uint32_t tile_target(uint64_t cands, uint64_t slots, int nb) {
    uint64_t cpt = cands / std::max<uint64_t>(1, 4 * slots);
    cpt = std::max<uint64_t>(cpt, (uint64_t)nb);
    return (uint32_t)std::min<uint64_t>(pow2_ceil(cpt), (uint64_t)kTileA * kTileB);
}

void set_tiles(Seg &s, uint32_t cpt) {
    if (s.kind == SEG_UNARY) {
        s.ta = std::min<uint32_t>(cpt, kTileU);
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
    s.tb = std::min<uint32_t>(cpt, kTileB);
    s.ta = std::max<uint32_t>(1, std::min<uint32_t>(cpt / s.tb, kTileA));
    s.n_ta = (uint32_t)((s.a_count + s.ta - 1) / s.ta);
    s.n_tb = (uint32_t)((s.b_count + s.tb - 1) / s.tb);
    s.n_tiles = (uint64_t)s.n_ta * s.n_tb;
    s.a_inner = s.n_ta <= s.n_tb ? 1 : 0;
}

uint64_t seg_candidates(const Seg &s) {
    if (s.kind == SEG_UNARY) return s.a_count;
    if (s.kind == SEG_TRI) return s.a_count * (s.a_count - 1) / 2;
    return s.a_count * s.b_count;
}

int build_segments(const ltl_ctx *c, int k, uint32_t ops, int n_props, uint64_t slots, int nb, Seg *segs,
                   OpGroup *groups, int &n_groups) {
    int n = 0;
    n_groups = 0;
    auto close_group = [&](int op, int first) {
        if (n <= first) return;
        uint64_t cands = 0;
        for (int i = first; i < n; ++i) cands += seg_candidates(segs[i]);
        const uint32_t cpt = tile_target(cands, slots, nb);
        uint64_t total = 0;
        for (int i = first; i < n; ++i) {
            set_tiles(segs[i], cpt);
            segs[i].tile_begin = total;
            total += segs[i].n_tiles;
        }
        groups[n_groups++] = OpGroup{op, first, n - first, total};
    };
    if (k == 1) {
        Seg s{};
        s.op = OP_ATOM; s.kind = SEG_UNARY; s.a_begin = 0; s.a_count = (uint64_t)n_props;
        segs[n++] = s;
        close_group(OP_ATOM, 0);
        return n;
    }
    const int order[7] = {OP_F, OP_U, OP_G, OP_X, OP_AND, OP_OR, OP_NOT};
    const uint32_t bit[8] = {0, LTL_NOT, LTL_AND, LTL_OR, LTL_X, LTL_F, LTL_G, LTL_U};
    for (int oi = 0; oi < 7; ++oi) {
        const int op = order[oi];
        if (!(ops & bit[op])) continue;
        const int first = n;
        if (op == OP_F || op == OP_G || op == OP_X || op == OP_NOT) {
            const uint64_t cnt = c->lvl_count[k - 1];
            if (cnt) {
                Seg s{};
                s.op = op; s.kind = SEG_UNARY; s.a_begin = c->lvl_begin[k - 1]; s.a_count = cnt;
                segs[n++] = s;
            }
            close_group(op, first);
            continue;
        }
        for (int cl = 1; cl <= k - 2; ++cl) {
            const int cr = k - 1 - cl;
            if (op != OP_U && cl > cr) continue;
            const uint64_t na = c->lvl_count[cl], nbb = c->lvl_count[cr];
            if (!na || !nbb) continue;
            Seg s{};
            s.op = op; s.a_begin = c->lvl_begin[cl]; s.a_count = na; s.b_begin = c->lvl_begin[cr]; s.b_count = nbb;
            if (op != OP_U && cl == cr) {
                if (na < 2) continue;
                s.kind = SEG_TRI;
            } else {
                s.kind = SEG_RECT;
            }
            segs[n++] = s;
        }
        close_group(op, first);
    }
    return n;
}

ltl_status check_common(int n_props, uint32_t ops, int max_size) {
    if (n_props < 1 || n_props > 32) return fail(LTL_ERR_INVALID, "n_props must be in 1..32");
    if (max_size < 1 || max_size >= kMaxLevels) return fail(LTL_ERR_INVALID, "max_size must be in 1..63");
    if (ops & ~(uint32_t)LTL_ALL) return fail(LTL_ERR_INVALID, "unknown connective bits in ops");
    return LTL_OK;
}

ltl_status check_traces(const ltl_traces *t, const char *name) {
    if (!t) return fail(LTL_ERR_INVALID, "%s is NULL", name);
    if (!t->offsets) return fail(LTL_ERR_INVALID, "%s.offsets is NULL", name);
    if (t->offsets[0] != 0) return fail(LTL_ERR_INVALID, "%s.offsets[0] must be 0", name);
    for (uint64_t i = 0; i < t->n_traces; ++i)
        if (t->offsets[i + 1] < t->offsets[i]) return fail(LTL_ERR_INVALID, "%s.offsets decrease at %llu", name,
                                                           (unsigned long long)i);
    if (t->offsets[t->n_traces] && !t->letters) return fail(LTL_ERR_INVALID, "%s.letters is NULL", name);
    return LTL_OK;
}

double wall_ms() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return 1e3 * (double)ts.tv_sec + 1e-6 * (double)ts.tv_nsec;
}

ltl_status write_formula(const std::string &s, char *out, size_t cap) {
    if (!out) return LTL_OK;
    if (s.size() + 1 > cap) {
        if (cap) out[0] = '\0';
        return fail(LTL_ERR_BUFSIZE, "formula needs %zu bytes", s.size() + 1);
    }
    memcpy(out, s.c_str(), s.size() + 1);
    return LTL_OK;
}

// Rebuilds the formula text of a provenance word (a cache entry's or the
// recorded separator's) from the cache's provenance array.
ltl_status formula_of(ltl_ctx *c, uint64_t root_prov, uint64_t n_entries, std::string &text) {
    const Layout &L = c->L;
    uint32_t *d_tok = (uint32_t *)(c->ws + L.o_tokens);
    int *d_n = (int *)(c->ws + L.o_ntok);
    CUDA_TRY(launch_walk((const uint64_t *)(c->ws + L.o_prov), n_entries, root_prov, d_tok, kMaxTokens, d_n,
                          c->stream));
    int n = 0;
    CUDA_TRY(cudaMemcpyAsync(c->h_tokens, d_tok, sizeof(uint32_t) * kMaxTokens, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(&c->h_tokens[kMaxTokens], d_n, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    memcpy(&n, &c->h_tokens[kMaxTokens], sizeof(int));
    if (n <= 0) return fail(LTL_ERR_CUDA, "provenance walk failed");
    text.clear();
    tokens_to_text(c->h_tokens, n, 0, text);
    return LTL_OK;
}

ltl_status run_learn(ltl_ctx *c, const uint32_t *d_letters_in, const uint64_t *d_offsets_in, const ltl_traces *P,
                     const ltl_traces *N, uint64_t n_pos, uint64_t n_neg, uint64_t max_len, int n_props,
                     uint32_t ops, int max_size, char *formula_out, size_t formula_cap, ltl_stats *stats) {
    const double t0 = wall_ms();
    ltl_stats st;
    memset(&st, 0, sizeof st);
    if (formula_out && formula_cap) formula_out[0] = '\0';
    c->have_result = false;
    const bool host_input = (P != nullptr);
    uint64_t total_pos = 0;
    if (host_input) total_pos = P->offsets[P->n_traces] + N->offsets[N->n_traces];
    Layout L;
    ltl_status s = plan(c, n_pos, n_neg, max_len, total_pos, host_input, n_props, L);
    if (s != LTL_OK) return s;
    c->L = L;
    char *ws = c->ws;
    Ctrl *d_ctrl = (Ctrl *)(ws + L.o_ctrl);
    Seg *d_segs = (Seg *)(ws + L.o_segs);
    uint64_t *d_mask = (uint64_t *)(ws + L.o_mask);
    uint64_t *d_keys = (uint64_t *)(ws + L.o_keys);
    uint64_t *d_atoms = (uint64_t *)(ws + L.o_atoms);
    cudaStream_t sm = c->stream;
    const uint64_t T = n_pos + n_neg;

    const uint32_t *d_letters = d_letters_in;
    const uint64_t *d_offsets = d_offsets_in;
    if (host_input) {
        // positives then negatives, offsets rebased into one prefix array
        uint32_t *dl = (uint32_t *)(ws + L.o_letters);
        uint64_t *dof = (uint64_t *)(ws + L.o_offsets);
        const uint64_t np = P->offsets[P->n_traces], nn = N->offsets[N->n_traces];
        std::vector<uint64_t> off(T + 1);
        for (uint64_t i = 0; i <= P->n_traces; ++i) off[i] = P->offsets[i];
        for (uint64_t i = 1; i <= N->n_traces; ++i) off[P->n_traces + i] = np + N->offsets[i];
        if (np) CUDA_TRY(cudaMemcpyAsync(dl, P->letters, 4 * np, cudaMemcpyHostToDevice, sm));
        if (nn) CUDA_TRY(cudaMemcpyAsync(dl + np, N->letters, 4 * nn, cudaMemcpyHostToDevice, sm));
        CUDA_TRY(cudaMemcpyAsync(dof, off.data(), 8 * (T + 1), cudaMemcpyHostToDevice, sm));
        st.h2d_bytes += 4 * (np + nn) + 8 * (T + 1);
        CUDA_TRY(cudaStreamSynchronize(sm));   // `off` is pageable and goes out of scope
        d_letters = dl;
        d_offsets = dof;
    }
    CUDA_TRY(cudaMemsetAsync(d_ctrl, 0, sizeof(Ctrl), sm));
    CUDA_TRY(cudaMemsetAsync(ws + L.o_hkeys, 0, 8 * L.hslots, sm));
    CUDA_TRY(cudaMemsetAsync(ws + L.o_hvals, 0xff, 4 * L.hslots, sm));
    CUDA_TRY(cudaMemsetAsync(d_mask, 0, 8 * L.stride, sm));
    CUDA_TRY(cudaMemsetAsync(d_atoms, 0, 8 * L.stride * (uint64_t)n_props, sm));
    if (L.narrow)
        CUDA_TRY(launch_pack_narrow(d_letters, d_offsets, (uint32_t)T, L.plane, n_props, d_mask, d_atoms, L.stride,
                                    d_ctrl, sm));
    else
        CUDA_TRY(launch_pack(d_letters, d_offsets, (uint32_t)T, L.plane, L.W, n_props, d_mask, d_atoms, L.stride,
                             d_ctrl, sm));
    CUDA_TRY(launch_keys(d_keys, L.stride, kKeySeed, sm));
    st.launches += 2;

    Problem pb{};
    pb.arena = (uint64_t *)(ws + L.o_arena);
    pb.stride = L.stride;
    pb.plane = L.plane;
    pb.mask = d_mask;
    pb.keys = d_keys;
    pb.atoms = d_atoms;
    pb.prov = (uint64_t *)(ws + L.o_prov);
    pb.hkeys = (unsigned long long *)(ws + L.o_hkeys);
    pb.hvals = (uint32_t *)(ws + L.o_hvals);
    pb.hmask = L.hslots - 1;
    pb.max_entries = L.max_entries;
    pb.ctrl = d_ctrl;
    pb.n_traces = (uint32_t)T;
    pb.n_pos = (uint32_t)n_pos;
    pb.nsteps = L.nsteps;
    const int stop_mode = c->opts.stop_on_solution;
    pb.stop_first = stop_mode == LTL_STOP_FIRST ? 1 : 0;
    pb.groups = L.G;
    pb.spin_limit = c->opts.spin_limit ? c->opts.spin_limit : (1ull << 20);

    int blocks_per_sm = 0;
    if ((s = occupancy(c, L, OP_U, blocks_per_sm)) != LTL_OK) return s;
    memset(c->lvl_begin, 0, sizeof c->lvl_begin);
    memset(c->lvl_count, 0, sizeof c->lvl_count);
    uint64_t prev_entries = 0, prev_cands = 0;
    bool found = false;
    ltl_status result = LTL_NOT_FOUND;
    OpGroup groups[8];
    for (int k = 1; k <= max_size; ++k) {
        int n_groups = 0;
        const int n_segs = build_segments(c, k, ops, n_props, (uint64_t)blocks_per_sm * (uint64_t)c->n_sm, L.NB,
                                          c->h_segs, groups, n_groups);
        c->lvl_begin[k] = prev_entries;
        if (n_segs == 0 || n_groups == 0) {
            // no candidate of this size (e.g. no connective allowed): the level is empty
            st.levels_done = k;
            continue;
        }
        CUDA_TRY(cudaMemcpyAsync(d_segs, c->h_segs, sizeof(Seg) * n_segs, cudaMemcpyHostToDevice, sm));
        CUDA_TRY(cudaEventRecord(c->ev[2 * k], sm));
        for (int gi = 0; gi < n_groups; ++gi) {
            const OpGroup &gr = groups[gi];
            LevelArgs la{};
            la.segs = d_segs + gr.first;
            la.n_segs = gr.count;
            la.level = k;
            la.total_tiles = gr.tiles;
            la.counter = k * 8 + gr.op;
            int bps = 0;
            if ((s = occupancy(c, L, gr.op, bps)) != LTL_OK) return s;
            const int grid = (int)std::min<uint64_t>(gr.tiles, (uint64_t)bps * (uint64_t)c->n_sm);
            void *args[] = {&pb, &la};
            CUDA_TRY(cudaLaunchKernel(level_kernel_for(L, gr.op), dim3(grid), dim3(L.NT), args, L.smem, sm));
            st.launches += 1;
        }
        CUDA_TRY(cudaEventRecord(c->ev[2 * k + 1], sm));
        CUDA_TRY(cudaMemcpyAsync(c->h_ctrl, d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, sm));
        CUDA_TRY(cudaStreamSynchronize(sm));
        st.d2h_bytes += sizeof(Ctrl);
        const Ctrl &h = *c->h_ctrl;
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
        st.ms[k] = ms;
        if (h.invalid_letter) return fail(LTL_ERR_INVALID, "trace letters use propositions >= n_props, offsets "
                                                           "decrease, or a trace exceeds max_len");
        if (h.err == LTL_ERR_INVALID) return fail(LTL_ERR_INVALID, "launch shape / shared memory mismatch");
        if (h.err) return fail((ltl_status)h.err, "device wait exceeded spin_limit (%llu timeouts)",
                               (unsigned long long)h.timeouts);
        const uint64_t ent = std::min<uint64_t>(h.n_entries, L.max_entries);
        c->lvl_count[k] = ent - prev_entries;
        st.unique[k] = ent - prev_entries;
        st.candidates[k] = h.cands - prev_cands;
        prev_entries = ent;
        prev_cands = h.cands;
        const bool stopped_early = (h.stop != 0) || h.cap_hit;
        if (!stopped_early) st.levels_done = k;
        if (h.found_count > 0) found = true;
        if (h.cap_hit) { result = LTL_CAP_REACHED; break; }
        if (found && stop_mode != LTL_STOP_NONE) break;
    }
    st.entries = prev_entries;
    st.n_traces = T;
    st.words_per_trace = (uint32_t)L.W;
    st.threads_per_cta = (uint32_t)L.NT;
    st.batch = (uint32_t)L.NB;
    st.ctas_per_sm = (uint32_t)blocks_per_sm;
    st.traces_per_thread = (uint32_t)(L.narrow ? 4 * L.C : 2 * L.C);
    st.traces_per_word = L.narrow ? 2u : 1u;
    st.chunk_groups = L.G;
    st.max_entries = L.max_entries;
    st.d2h_bytes += 0;
    c->have_result = true;
    if (found) {
        const Ctrl &h = *c->h_ctrl;
        std::string text;
        s = formula_of(c, h.found_prov, prev_entries, text);
        st.launches += 1;
        st.d2h_bytes += sizeof(uint32_t) * kMaxTokens + sizeof(int);
        if (s != LTL_OK) return s;
        st.found_size = h.found_level;
        s = write_formula(text, formula_out, formula_cap);
        if (s != LTL_OK) return s;
        result = LTL_OK;
    }
    st.total_ms = wall_ms() - t0;
    if (stats) *stats = st;
    return result;
}

ltl_opts default_opts() {
    ltl_opts o;
    memset(&o, 0, sizeof o);
    o.stop_on_solution = LTL_STOP_FIRST;
    return o;
}

uint64_t traces_max_len(const ltl_traces *t) {
    uint64_t m = 0;
    for (uint64_t i = 0; i < t->n_traces; ++i) m = std::max<uint64_t>(m, t->offsets[i + 1] - t->offsets[i]);
    return m;
}

}  // namespace

// ==================================================================== C ABI

extern "C" {

const char *ltl_last_error(void) { return g_err.c_str(); }

const char *ltl_version(void) { return "ltl-gb300 0.1 (sm_103a)"; }

ltl_status ltl_ctx_create(const ltl_opts *opts, ltl_ctx **out) {
    if (!out) return fail(LTL_ERR_INVALID, "out is NULL");
    *out = nullptr;
    ltl_ctx *c = new ltl_ctx();
    c->opts = opts ? *opts : default_opts();
    if (c->opts.stop_on_solution < 0 || c->opts.stop_on_solution > 2) {
        delete c;
        return fail(LTL_ERR_INVALID, "stop_on_solution must be 0, 1 or 2");
    }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return fail(LTL_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    if (c->opts.stream) c->stream = (cudaStream_t)c->opts.stream;
    else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = true;
    }
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_ctrl, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_segs, sizeof(Seg) * kMaxSegs);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_tokens, sizeof(uint32_t) * (kMaxTokens + 1));
    for (int i = 0; i < 2 * kMaxLevels + 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        ltl_ctx_destroy(c);
        return fail(LTL_ERR_CUDA, "context setup failed: %s", cudaGetErrorString(e));
    }
    if (c->opts.workspace) {
        if (((uintptr_t)c->opts.workspace & 255u) != 0) {
            ltl_ctx_destroy(c);
            return fail(LTL_ERR_INVALID, "workspace must be 256-byte aligned");
        }
        c->ws = (char *)c->opts.workspace;
        c->ws_bytes = c->opts.workspace_bytes;
        c->ws_owned = false;
    }
    *out = c;
    return LTL_OK;
}

void ltl_ctx_destroy(ltl_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->ws_owned && c->ws) {
        if (c->opts.free) c->opts.free(c->ws, c->stream, c->opts.user);
        else cudaFree(c->ws);
    }
    for (int i = 0; i < 2 * kMaxLevels + 2; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
    if (c->h_segs) cudaFreeHost(c->h_segs);
    if (c->h_tokens) cudaFreeHost(c->h_tokens);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    (void)cudaGetLastError();
    delete c;
}

ltl_status ltl_ctx_learn(ltl_ctx *c, const ltl_traces *P, const ltl_traces *N, int n_props, uint32_t ops,
                         int max_size, char *formula_out, size_t formula_cap, ltl_stats *stats) {
    if (!c) return fail(LTL_ERR_INVALID, "ctx is NULL");
    ltl_status s = check_common(n_props, ops, max_size);
    if (s != LTL_OK) return s;
    if ((s = check_traces(P, "P")) != LTL_OK) return s;
    if ((s = check_traces(N, "N")) != LTL_OK) return s;
    const uint64_t ml = std::max(traces_max_len(P), traces_max_len(N));
    return run_learn(c, nullptr, nullptr, P, N, P->n_traces, N->n_traces, ml, n_props, ops, max_size, formula_out,
                     formula_cap, stats);
}

ltl_status ltl_ctx_learn_device(ltl_ctx *c, const uint32_t *d_letters, const uint64_t *d_offsets, uint64_t n_pos,
                                uint64_t n_neg, uint32_t max_len, int n_props, uint32_t ops, int max_size,
                                char *formula_out, size_t formula_cap, ltl_stats *stats) {
    if (!c) return fail(LTL_ERR_INVALID, "ctx is NULL");
    ltl_status s = check_common(n_props, ops, max_size);
    if (s != LTL_OK) return s;
    if (!d_offsets || (!d_letters && max_len > 0)) return fail(LTL_ERR_INVALID, "device trace buffers are NULL");
    return run_learn(c, d_letters, d_offsets, nullptr, nullptr, n_pos, n_neg, max_len, n_props, ops, max_size,
                     formula_out, formula_cap, stats);
}

ltl_status ltl_learn(const ltl_traces *P, const ltl_traces *N, int n_props, uint32_t ops, int max_size,
                     const ltl_opts *opts, char *formula_out, size_t formula_cap, ltl_stats *stats) {
    ltl_ctx *c = nullptr;
    ltl_status s = ltl_ctx_create(opts, &c);
    if (s != LTL_OK) return s;
    s = ltl_ctx_learn(c, P, N, n_props, ops, max_size, formula_out, formula_cap, stats);
    ltl_ctx_destroy(c);
    return s;
}

ltl_status ltl_ctx_level_range(ltl_ctx *c, int level, uint64_t *begin, uint64_t *count) {
    if (!c || !begin || !count) return fail(LTL_ERR_INVALID, "NULL argument");
    if (!c->have_result) return fail(LTL_ERR_INVALID, "no learn result on this context");
    if (level < 1 || level >= kMaxLevels) return fail(LTL_ERR_INVALID, "level out of range");
    *begin = c->lvl_begin[level];
    *count = c->lvl_count[level];
    return LTL_OK;
}

ltl_status ltl_ctx_entry(ltl_ctx *c, uint64_t idx, char *formula_out, size_t formula_cap, uint64_t *cs_out,
                         int words_per_trace) {
    if (!c) return fail(LTL_ERR_INVALID, "ctx is NULL");
    if (!c->have_result) return fail(LTL_ERR_INVALID, "no learn result on this context");
    const Layout &L = c->L;
    uint64_t n_ent = 0;
    for (int k = 1; k < kMaxLevels; ++k) n_ent = std::max(n_ent, c->lvl_begin[k] + c->lvl_count[k]);
    if (idx >= n_ent) return fail(LTL_ERR_INVALID, "entry %llu out of range", (unsigned long long)idx);
    uint64_t p = 0;
    CUDA_TRY(cudaMemcpyAsync(&c->h_ctrl->found_prov, c->ws + L.o_prov + 8 * idx, 8, cudaMemcpyDeviceToHost,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    p = c->h_ctrl->found_prov;
    if (formula_out) {
        std::string text;
        ltl_status s = formula_of(c, p, n_ent, text);
        if (s != LTL_OK) return s;
        if ((s = write_formula(text, formula_out, formula_cap)) != LTL_OK) return s;
    }
    if (cs_out && L.narrow) {
        if (words_per_trace != 1) return fail(LTL_ERR_INVALID, "words_per_trace must be 1");
        // word q of the plane holds traces 2q (low half) and 2q + 1 (high half)
        const uint64_t nw = ((uint64_t)L.n_traces + 1) / 2;
        std::vector<uint64_t> words(nw ? nw : 1);
        CUDA_TRY(cudaMemcpyAsync(words.data(), c->ws + L.o_arena + 8 * L.stride * idx, 8 * nw, cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (uint64_t t = 0; t < L.n_traces; ++t) cs_out[t] = (words[t / 2] >> (32 * (t & 1))) & 0xffffffffull;
        return LTL_OK;
    }
    if (cs_out) {
        if (words_per_trace != L.W) return fail(LTL_ERR_INVALID, "words_per_trace must be %d", L.W);
        // plane w of the entry holds word w of every trace: a strided 2-D copy
        const char *src = c->ws + L.o_arena + 8 * L.stride * idx;
        for (int w = 0; w < L.W; ++w)
            CUDA_TRY(cudaMemcpy2DAsync(cs_out + w, 8 * (size_t)L.W, src + 8 * L.plane * w, 8, 8, (size_t)L.n_traces,
                                       cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return LTL_OK;
}

ltl_status ltl_eval(const char *formula, const ltl_traces *traces, int n_props, uint64_t *cs_out,
                    int words_per_trace) {
    if (n_props < 1 || n_props > 32) return fail(LTL_ERR_INVALID, "n_props must be in 1..32");
    ltl_status s = check_traces(traces, "traces");
    if (s != LTL_OK) return s;
    if (!cs_out && traces->n_traces) return fail(LTL_ERR_INVALID, "cs_out is NULL");
    std::vector<uint32_t> prog;
    int depth = 0, max_atom = -1;
    if (!compile_formula(formula, n_props, prog, depth, max_atom))
        return fail(LTL_ERR_INVALID, "cannot parse formula (or an atom >= n_props): %s", formula ? formula : "(null)");
    const uint64_t T = traces->n_traces;
    const uint64_t ml = traces_max_len(traces);
    const int W = (int)std::max<uint64_t>(1, (ml + 63) / 64);
    const int Wt = (int)pow2_ceil((uint64_t)W);
    if (Wt > 16) return fail(LTL_ERR_INVALID, "ltl_eval supports traces up to 1024 positions");
    if (words_per_trace < W) return fail(LTL_ERR_INVALID, "words_per_trace must be >= %d", W);
    if (T == 0) return LTL_OK;
    const uint64_t plane = round_up(T, 128), stride = (uint64_t)Wt * plane;
    const uint64_t total_pos = traces->offsets[T];
    // device scratch: ctrl | letters | offsets | mask | atoms | stack | program | out
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t r = o;
        o = round_up(o + b, 256);
        return r;
    };
    const size_t o_ctrl = take(sizeof(Ctrl)), o_let = take(4 * std::max<uint64_t>(total_pos, 1)),
                 o_off = take(8 * (T + 1)), o_mask = take(8 * stride), o_atoms = take(8 * stride * (uint64_t)n_props),
                 o_stack = take(8 * stride * (uint64_t)depth), o_prog = take(4 * prog.size()),
                 o_out = take(8 * T * (uint64_t)words_per_trace);
    char *d = nullptr;
    cudaStream_t sm = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&sm, cudaStreamNonBlocking));
    cudaError_t e = cudaMallocAsync(&d, o, sm);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        cudaStreamDestroy(sm);
        return fail(LTL_ERR_OOM, "cudaMallocAsync(%zu) failed", o);
    }
    Ctrl h_ctrl;
    auto done = [&](ltl_status st) {
        cudaFreeAsync(d, sm);
        cudaStreamSynchronize(sm);
        cudaStreamDestroy(sm);
        (void)cudaGetLastError();
        return st;
    };
#define EVAL_TRY(x)                                                                                      \
    do {                                                                                                 \
        cudaError_t e_ = (x);                                                                            \
        if (e_ != cudaSuccess) return done(fail(LTL_ERR_CUDA, "%s failed: %s", #x, cudaGetErrorString(e_))); \
    } while (0)
    EVAL_TRY(cudaMemsetAsync(d + o_ctrl, 0, sizeof(Ctrl), sm));
    if (total_pos) EVAL_TRY(cudaMemcpyAsync(d + o_let, traces->letters, 4 * total_pos, cudaMemcpyHostToDevice, sm));
    EVAL_TRY(cudaMemcpyAsync(d + o_off, traces->offsets, 8 * (T + 1), cudaMemcpyHostToDevice, sm));
    EVAL_TRY(cudaMemcpyAsync(d + o_prog, prog.data(), 4 * prog.size(), cudaMemcpyHostToDevice, sm));
    EVAL_TRY(launch_pack((const uint32_t *)(d + o_let), (const uint64_t *)(d + o_off), (uint32_t)T, plane, W, n_props,
                         (uint64_t *)(d + o_mask), (uint64_t *)(d + o_atoms), stride, (Ctrl *)(d + o_ctrl), sm));
    if (Wt > W) {
        // planes W..Wt-1 are padding: zero them for the operators
        for (int w = W; w < Wt; ++w) {
            EVAL_TRY(cudaMemsetAsync(d + o_mask + 8 * plane * w, 0, 8 * plane, sm));
            for (int p = 0; p < n_props; ++p)
                EVAL_TRY(cudaMemsetAsync(d + o_atoms + 8 * (stride * p + plane * w), 0, 8 * plane, sm));
        }
    }
    EVAL_TRY(launch_eval(Wt, (const uint32_t *)(d + o_prog), (int)prog.size(), (const uint64_t *)(d + o_atoms),
                         (const uint64_t *)(d + o_mask), stride, plane, (uint64_t *)(d + o_stack), ceil_log2(ml),
                         (uint32_t)T, (uint64_t *)(d + o_out), words_per_trace, sm));
    EVAL_TRY(cudaMemcpyAsync(&h_ctrl, d + o_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, sm));
    EVAL_TRY(cudaMemcpyAsync(cs_out, d + o_out, 8 * T * (uint64_t)words_per_trace, cudaMemcpyDeviceToHost, sm));
    EVAL_TRY(cudaStreamSynchronize(sm));
#undef EVAL_TRY
    if (h_ctrl.invalid_letter) return done(fail(LTL_ERR_INVALID, "trace letters use propositions >= n_props"));
    return done(LTL_OK);
}

}  // extern "C"

// Entry points for other translation units of the library.
namespace ltl {
bool compile_formula_program(const char *text, int n_props, std::vector<uint32_t> &prog, int &depth) {
    int max_atom = -1;
    return compile_formula(text, n_props, prog, depth, max_atom);
}
ltl_status set_error(ltl_status s, const char *msg) { return fail(s, "%s", msg); }
}  // namespace ltl
