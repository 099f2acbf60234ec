// ltl_host.cu -- host helpers shared by the library (errors, formula text,
// argument checks) and ltl_eval.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <string>
#include <vector>

#include "ltl_internal.h"

namespace ltl {

namespace {
thread_local std::string g_err;
}

ltl_status fail(ltl_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

ltl_status set_error(ltl_status s, const char *msg) { return fail(s, "%s", msg); }

const char *last_error_text() { return g_err.c_str(); }

double wall_ms() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return 1e3 * (double)ts.tv_sec + 1e-6 * (double)ts.tv_nsec;
}

// ----------------------------------------------------------------- formula text
// f := '!' f | 'X' f | 'F' f | 'G' f | 'p' digits | '(' f ')' | '(' f op f ')'
namespace {
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
}  // namespace

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


bool compile_formula_program(const char *text, int n_props, std::vector<uint32_t> &prog, int &depth) {
    int max_atom = -1;
    return compile_formula(text, n_props, prog, depth, max_atom);
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

ltl_status check_common(int n_props, uint32_t ops, int max_size) {
    if (n_props < 1 || n_props > 32) return fail(LTL_ERR_INVALID, "n_props must be in 1..32");
    if (max_size < 1 || max_size >= kMaxLevels) return fail(LTL_ERR_INVALID, "max_size must be in 1..63");
    if (ops & ~(uint32_t)(LTL_ALL | LTL_NNF)) return fail(LTL_ERR_INVALID, "unknown connective bits in ops");
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

uint64_t traces_max_len(const ltl_traces *t) {
    uint64_t m = 0;
    for (uint64_t i = 0; i < t->n_traces; ++i) m = std::max<uint64_t>(m, t->offsets[i + 1] - t->offsets[i]);
    return m;
}

}  // namespace ltl

using namespace ltl;

extern "C" {

const char *ltl_last_error(void) { return last_error_text(); }

const char *ltl_version(void) { return "ltl-gb300 0.3 (sm_103a)"; }

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
    LTL_CUDA_TRY(cudaStreamCreateWithFlags(&sm, cudaStreamNonBlocking));
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
    EVAL_TRY(launch_pack((const uint32_t *)(d + o_let), (const uint64_t *)(d + o_off), (uint32_t)T, plane, W, Wt, n_props,
                         (uint64_t *)(d + o_mask), (uint64_t *)(d + o_atoms), stride, (Ctrl *)(d + o_ctrl), sm));
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
