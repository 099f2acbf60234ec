/*
 * ltl_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * enumerative LTL learner of "LTL learning on GPUs" (arXiv 2402.12373).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * path: its own parser, its own data layout (one byte per trace position, no
 * bit packing, no shifts), its own hash table.
 *
 * What it computes (all citations are to the paper):
 *
 *  - Finite-trace LTL semantics, Section 2: tr,i |= X f iff tr,i+1 |= f;
 *    tr,i |= F f iff some i <= j < |tr| has tr,j |= f; tr,i |= f U g iff some
 *    i <= j < |tr| has tr,j |= g and tr,k |= f for all i <= k < j; and every
 *    formula is false at i >= |tr| (so X is a strong next, and negation and
 *    G are false beyond the end of a trace).  G f holds at i iff f holds at
 *    every i <= j < |tr| (G is in the grammar of Section 2; the paper gives
 *    no separate clause, this is the textbook one).  The clauses are written
 *    out literally, O(n^2) per trace for F, G and U.
 *
 *  - The characteristic matrix of a formula (Section 4): its truth value at
 *    every position of every trace, traces in the fixed order P then N.
 *
 *  - Soundness, eq. (dagger) of Section 4: P within lang(f) and N disjoint from
 *    lang(f), where tr in lang(f) iff tr,0 |= f.
 *
 *  - The bottom-up enumeration of Section 3 (the `enum`, `handleOp` and
 *    check-and-cache steps): level 1 holds the atoms; level c is built from the
 *    cached levels by every connective in the order F, U, G, X, And, Or, Not;
 *    each candidate is first checked for soundness, then admitted to the
 *    cache iff its characteristic matrix is new.  Admission here is the exact
 *    uniqueness check (Section 5 notes that the relaxed check is exact when no
 *    hashing is needed); equality is decided by comparing the whole matrix.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *  - candidate space: unary ops take every entry of level c-1; And/Or take
 *    splits (i, j), i + j = c-1, i <= j, all pairs when i < j and pairs a < b
 *    (cache order) when i == j; U takes every ordered split and every ordered
 *    pair, a == b included.
 *  - atoms are deduplicated too (level 1 holds the distinct atom matrices).
 *  - unique counts include separating candidates (set semantics).
 *  - stop modes: 1 = stop at the first separator; 2 = finish the level where the
 *    first separator was found; 0 = enumerate every level up to max_size.
 *  - ops mask bits: Not=1 And=2 Or=4 X=8 F=16 G=32 U=64.
 *
 * Variants the paper states (oracle_learn_ex):
 *  - cost homomorphism (Section 2): every connective and the atoms have a
 *    positive cost; a formula's cost is the sum over its syntax tree.  Levels
 *    are costs instead of sizes: atoms form level cost(atom); a unary
 *    connective of cost k builds level c from level c - k; a binary one from
 *    splits (i, j) with i + j = c - k.  Uniform cost (all 1) is the size.
 *  - negation normal form (Section 2; used for the comparisons of Section 7):
 *    negation is applied to atoms only.
 *  - noisy learning (Section 3, after relaxedCheckAndCache): a candidate
 *    separates when it misclassifies at most max_errors traces.
 */
#define _POSIX_C_SOURCE 200809L
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

enum { O_ATOM = 0, O_NOT, O_AND, O_OR, O_X, O_F, O_G, O_U };
enum { M_NOT = 1, M_AND = 2, M_OR = 4, M_X = 8, M_F = 16, M_G = 32, M_U = 64 };

/* return codes */
enum { OR_FOUND = 0, OR_NOT_FOUND = 1, OR_CAP = 2, OR_INVALID = -1, OR_NOMEM = -3, OR_BUFSIZE = -5 };

/* ------------------------------------------------------------------ */
/* traces                                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    const uint32_t *letters;   /* concatenated positions, bit p = p holds  */
    const uint64_t *offsets;   /* n+1 prefix offsets                        */
    uint64_t n;                /* number of traces                          */
    uint64_t total;            /* total number of positions                 */
} Traces;

static uint64_t tr_len(const Traces *S, uint64_t t) { return S->offsets[t + 1] - S->offsets[t]; }

/* ------------------------------------------------------------------ */
/* semantics on one matrix: out[offsets[t] + i] = (tr_t, i |= op(...)) */
/* ------------------------------------------------------------------ */

static void sem_atom(const Traces *S, int p, uint8_t *out) {
    for (uint64_t q = 0; q < S->total; q++) out[q] = (uint8_t)((S->letters[q] >> p) & 1u);
}

static void sem_not(const Traces *S, const uint8_t *a, uint8_t *out) {
    for (uint64_t q = 0; q < S->total; q++) out[q] = (uint8_t)!a[q];
}

static void sem_and(const Traces *S, const uint8_t *a, const uint8_t *b, uint8_t *out) {
    for (uint64_t q = 0; q < S->total; q++) out[q] = (uint8_t)(a[q] && b[q]);
}

static void sem_or(const Traces *S, const uint8_t *a, const uint8_t *b, uint8_t *out) {
    for (uint64_t q = 0; q < S->total; q++) out[q] = (uint8_t)(a[q] || b[q]);
}

static void sem_X(const Traces *S, const uint8_t *a, uint8_t *out) {
    for (uint64_t t = 0; t < S->n; t++) {
        uint64_t base = S->offsets[t], L = tr_len(S, t);
        for (uint64_t i = 0; i < L; i++) out[base + i] = (i + 1 < L) ? a[base + i + 1] : 0;
    }
}

static void sem_F(const Traces *S, const uint8_t *a, uint8_t *out) {
    for (uint64_t t = 0; t < S->n; t++) {
        uint64_t base = S->offsets[t], L = tr_len(S, t);
        for (uint64_t i = 0; i < L; i++) {
            uint8_t v = 0;                       /* exists i <= j < L with a at j */
            for (uint64_t j = i; j < L; j++)
                if (a[base + j]) { v = 1; break; }
            out[base + i] = v;
        }
    }
}

static void sem_G(const Traces *S, const uint8_t *a, uint8_t *out) {
    for (uint64_t t = 0; t < S->n; t++) {
        uint64_t base = S->offsets[t], L = tr_len(S, t);
        for (uint64_t i = 0; i < L; i++) {
            uint8_t v = 1;                       /* for all i <= j < L, a at j */
            for (uint64_t j = i; j < L; j++)
                if (!a[base + j]) { v = 0; break; }
            out[base + i] = v;
        }
    }
}

static void sem_U(const Traces *S, const uint8_t *a, const uint8_t *b, uint8_t *out) {
    for (uint64_t t = 0; t < S->n; t++) {
        uint64_t base = S->offsets[t], L = tr_len(S, t);
        for (uint64_t i = 0; i < L; i++) {
            /* exists i <= j < L: b at j and a at every k in [i, j).  Walk j up
             * from i: the first j with b decides true; a j without a (and
             * without b) rules out every later j. */
            uint8_t v = 0;
            for (uint64_t j = i; j < L; j++) {
                if (b[base + j]) { v = 1; break; }
                if (!a[base + j]) break;
            }
            out[base + i] = v;
        }
    }
}

/* eq. (dagger): every positive true at position 0, every negative false there.
 * An empty trace is false at position 0 (i >= |tr|).  With an error budget
 * (noisy learning) at most max_errors traces may be misclassified. */
static int separates(const Traces *S, uint64_t n_pos, const uint8_t *m, uint64_t max_errors) {
    uint64_t errors = 0;
    for (uint64_t t = 0; t < S->n; t++) {
        uint8_t v = tr_len(S, t) > 0 ? m[S->offsets[t]] : 0;
        if (t < n_pos ? !v : v) errors++;
    }
    return errors <= max_errors;
}

/* ------------------------------------------------------------------ */
/* formula text: parser and AST evaluation                             */
/*   f := '!' f | 'X' f | 'F' f | 'G' f | 'p' digits                    */
/*      | '(' f ')' | '(' f ('&' | '|' | 'U') f ')'                      */
/* ------------------------------------------------------------------ */

typedef struct { int op, a, b; } AstNode;   /* a: prop index for atoms */

typedef struct {
    const char *s;
    AstNode *nodes;
    int n, cap;
    int err;
} Parser;

static void skip_ws(Parser *P) { while (*P->s == ' ' || *P->s == '\t' || *P->s == '\n') P->s++; }

static int new_node(Parser *P, int op, int a, int b) {
    if (P->n == P->cap) {
        P->cap = P->cap ? 2 * P->cap : 64;
        P->nodes = (AstNode *)realloc(P->nodes, sizeof(AstNode) * (size_t)P->cap);
    }
    P->nodes[P->n].op = op; P->nodes[P->n].a = a; P->nodes[P->n].b = b;
    return P->n++;
}

static int parse_f(Parser *P, int depth);

static int parse_f(Parser *P, int depth) {
    if (depth > 100000) { P->err = 1; return -1; }
    skip_ws(P);
    char c = *P->s;
    if (c == '!' || c == 'X' || c == 'F' || c == 'G') {
        P->s++;
        int x = parse_f(P, depth + 1);
        if (P->err) return -1;
        int op = c == '!' ? O_NOT : c == 'X' ? O_X : c == 'F' ? O_F : O_G;
        return new_node(P, op, x, -1);
    }
    if (c == 'p') {
        P->s++;
        if (*P->s < '0' || *P->s > '9') { P->err = 1; return -1; }
        long v = 0;
        while (*P->s >= '0' && *P->s <= '9') { v = v * 10 + (*P->s - '0'); if (v > 31) { P->err = 1; return -1; } P->s++; }
        return new_node(P, O_ATOM, (int)v, -1);
    }
    if (c == '(') {
        P->s++;
        int l = parse_f(P, depth + 1);
        if (P->err) return -1;
        skip_ws(P);
        char o = *P->s;
        if (o == ')') { P->s++; return l; }
        if (o != '&' && o != '|' && o != 'U') { P->err = 1; return -1; }
        P->s++;
        int r = parse_f(P, depth + 1);
        if (P->err) return -1;
        skip_ws(P);
        if (*P->s != ')') { P->err = 1; return -1; }
        P->s++;
        return new_node(P, o == '&' ? O_AND : o == '|' ? O_OR : O_U, l, r);
    }
    P->err = 1;
    return -1;
}

/* Evaluates the AST bottom-up (nodes are created children-first). */
static int eval_ast(const Traces *S, int n_props, const AstNode *nodes, int n, int root, uint8_t *out) {
    uint64_t W = S->total ? S->total : 1;
    uint8_t *buf = (uint8_t *)malloc((size_t)n * W);
    if (!buf) return OR_NOMEM;
    for (int k = 0; k < n; k++) {
        uint8_t *o = buf + (size_t)k * W;
        const AstNode *nd = &nodes[k];
        const uint8_t *A = nd->a >= 0 ? buf + (size_t)nd->a * W : NULL;
        const uint8_t *B = nd->b >= 0 ? buf + (size_t)nd->b * W : NULL;
        switch (nd->op) {
        case O_ATOM:
            if (nd->a >= n_props) { free(buf); return OR_INVALID; }
            sem_atom(S, nd->a, o); break;
        case O_NOT: sem_not(S, A, o); break;
        case O_AND: sem_and(S, A, B, o); break;
        case O_OR:  sem_or(S, A, B, o); break;
        case O_X:   sem_X(S, A, o); break;
        case O_F:   sem_F(S, A, o); break;
        case O_G:   sem_G(S, A, o); break;
        case O_U:   sem_U(S, A, B, o); break;
        }
    }
    memcpy(out, buf + (size_t)root * W, (size_t)S->total);
    free(buf);
    return 0;
}

/* Truth of `formula` at every position of every trace: out has one byte per
 * position, in the order of `letters`.  Returns 0, or OR_INVALID on a parse
 * error or an atom index >= n_props. */
int oracle_eval(const char *formula, const uint32_t *letters, const uint64_t *offsets,
                uint64_t n_traces, int n_props, uint8_t *out) {
    Parser P = {formula, NULL, 0, 0, 0};
    int root = parse_f(&P, 0);
    skip_ws(&P);
    if (P.err || *P.s != '\0' || root < 0) { free(P.nodes); return OR_INVALID; }
    Traces S = {letters, offsets, n_traces, offsets[n_traces]};
    int rc = eval_ast(&S, n_props, P.nodes, P.n, root, out);
    free(P.nodes);
    return rc;
}

/* Syntax-tree size of `formula` (number of nodes), or -1 on a parse error. */
int oracle_size(const char *formula) {
    Parser P = {formula, NULL, 0, 0, 0};
    int root = parse_f(&P, 0);
    skip_ws(&P);
    int n = (P.err || *P.s != '\0' || root < 0) ? -1 : 0;
    if (n == 0) {
        /* count nodes reachable from root (parenthesised sub-formulae create no node) */
        int *stack = (int *)malloc(sizeof(int) * (size_t)(P.n + 1)), sp = 0;
        stack[sp++] = root;
        while (sp) {
            int k = stack[--sp];
            n++;
            if (P.nodes[k].op != O_ATOM) {
                stack[sp++] = P.nodes[k].a;
                if (P.nodes[k].b >= 0) stack[sp++] = P.nodes[k].b;
            }
        }
        free(stack);
    }
    free(P.nodes);
    return n;
}

/* ------------------------------------------------------------------ */
/* language cache with exact dedup                                     */
/* ------------------------------------------------------------------ */

typedef struct {
    uint8_t op;
    uint32_t a, b;     /* operand entry ids (prop index for atoms) */
} Prov;

typedef struct {
    uint64_t W;                 /* bytes per matrix            */
    uint8_t **mat;              /* entry -> matrix             */
    Prov *prov;
    uint64_t n, cap;
    /* open-addressing table of entry ids + 1 (0 = empty) */
    uint64_t *slot;
    uint64_t *slot_hash;
    uint64_t nslot;
} Cache;

/* FNV-1a over the matrix bytes: only a bucket index, equality is memcmp. */
static uint64_t fnv1a(const uint8_t *p, uint64_t n) {
    uint64_t h = 1469598103934665603ULL;
    for (uint64_t i = 0; i < n; i++) { h ^= p[i]; h *= 1099511628211ULL; }
    return h;
}

static int cache_grow_table(Cache *C) {
    uint64_t ns = C->nslot ? 2 * C->nslot : 1024;
    uint64_t *sl = (uint64_t *)calloc(ns, sizeof(uint64_t));
    uint64_t *sh = (uint64_t *)calloc(ns, sizeof(uint64_t));
    if (!sl || !sh) { free(sl); free(sh); return OR_NOMEM; }
    for (uint64_t i = 0; i < C->nslot; i++) {
        if (!C->slot[i]) continue;
        uint64_t h = C->slot_hash[i], k = h & (ns - 1);
        while (sl[k]) k = (k + 1) & (ns - 1);
        sl[k] = C->slot[i]; sh[k] = h;
    }
    free(C->slot); free(C->slot_hash);
    C->slot = sl; C->slot_hash = sh; C->nslot = ns;
    return 0;
}

/* Returns 1 if m was new (and is now entry C->n - 1), 0 if already present,
 * or a negative error. Takes ownership of m when new. */
static int cache_insert(Cache *C, uint8_t *m, Prov pv) {
    if (2 * (C->n + 1) > C->nslot) { int rc = cache_grow_table(C); if (rc) return rc; }
    uint64_t h = fnv1a(m, C->W), k = h & (C->nslot - 1);
    while (C->slot[k]) {
        if (C->slot_hash[k] == h && memcmp(C->mat[C->slot[k] - 1], m, (size_t)C->W) == 0) return 0;
        k = (k + 1) & (C->nslot - 1);
    }
    if (C->n == C->cap) {
        uint64_t nc = C->cap ? 2 * C->cap : 1024;
        uint8_t **nm = (uint8_t **)realloc(C->mat, sizeof(uint8_t *) * nc);
        if (!nm) return OR_NOMEM;
        C->mat = nm;
        Prov *np = (Prov *)realloc(C->prov, sizeof(Prov) * nc);
        if (!np) return OR_NOMEM;
        C->prov = np;
        C->cap = nc;
    }
    C->mat[C->n] = m; C->prov[C->n] = pv; C->n++;
    C->slot[k] = C->n; C->slot_hash[k] = h;
    return 1;
}

static void cache_free(Cache *C) {
    for (uint64_t i = 0; i < C->n; i++) free(C->mat[i]);
    free(C->mat); free(C->prov); free(C->slot); free(C->slot_hash);
}

/* formula text of an entry (or of a candidate given by its provenance) */
typedef struct { char *buf; size_t len, cap; } Str;

static void str_put(Str *s, const char *t) {
    size_t n = strlen(t);
    if (s->len + n + 1 > s->cap) {
        s->cap = (s->len + n + 1) * 2;
        s->buf = (char *)realloc(s->buf, s->cap);
    }
    memcpy(s->buf + s->len, t, n + 1);
    s->len += n;
}

static void print_prov(const Cache *C, Prov pv, Str *s) {
    char tmp[32];
    switch (pv.op) {
    case O_ATOM: snprintf(tmp, sizeof tmp, "p%u", pv.a); str_put(s, tmp); return;
    case O_NOT: str_put(s, "!"); print_prov(C, C->prov[pv.a], s); return;
    case O_X: str_put(s, "X "); print_prov(C, C->prov[pv.a], s); return;
    case O_F: str_put(s, "F "); print_prov(C, C->prov[pv.a], s); return;
    case O_G: str_put(s, "G "); print_prov(C, C->prov[pv.a], s); return;
    default: break;
    }
    str_put(s, "(");
    print_prov(C, C->prov[pv.a], s);
    str_put(s, pv.op == O_AND ? " & " : pv.op == O_OR ? " | " : " U ");
    print_prov(C, C->prov[pv.b], s);
    str_put(s, ")");
}

/* ------------------------------------------------------------------ */
/* the enumeration (Section 3)                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    const Traces *S;
    uint64_t n_pos;
    uint64_t max_errors;
    int cost[8];          /* per connective (index = O_*), atoms at O_ATOM */
    int nnf;              /* negation on atoms only */
    Cache C;
    uint64_t *lvl_begin, *lvl_end;   /* entries of level c: [begin, end) */
    uint64_t *unique, *cands;
    int stop_mode;
    uint64_t max_entries;
    int found;
    int found_size;
    Prov found_prov;
    int cap_hit;
    int err;
} Enum;

/* check-and-cache for one candidate matrix m (owned).  Returns 1 to stop. */
static int check_and_cache(Enum *E, int c, uint8_t *m, Prov pv) {
    E->cands[c]++;
    if (separates(E->S, E->n_pos, m, E->max_errors)) {
        if (!E->found) { E->found = 1; E->found_size = c; E->found_prov = pv; }
        if (E->stop_mode == 1) { free(m); return 1; }
    }
    if (E->C.n >= E->max_entries) {
        /* cache full: only a duplicate may pass; anything new sets cap_hit */
        uint64_t h = fnv1a(m, E->C.W), k = h & (E->C.nslot - 1);
        int dup = 0;
        while (E->C.slot[k]) {
            if (E->C.slot_hash[k] == h && memcmp(E->C.mat[E->C.slot[k] - 1], m, (size_t)E->C.W) == 0) { dup = 1; break; }
            k = (k + 1) & (E->C.nslot - 1);
        }
        free(m);
        if (!dup) E->cap_hit = 1;   /* the level goes on: candidates are still checked */
        return 0;
    }
    int rc = cache_insert(&E->C, m, pv);
    if (rc < 0) { free(m); E->err = rc; return 1; }
    if (rc == 1) E->unique[c]++;
    else free(m);
    return 0;
}

static uint8_t *new_mat(Enum *E) {
    uint8_t *m = (uint8_t *)malloc((size_t)(E->C.W ? E->C.W : 1));
    if (!m) E->err = OR_NOMEM;
    return m;
}

/* Builds level c with connective op; returns 1 to stop.  The operands come
 * from level c - cost(op) (unary) or from splits of c - cost(op) (binary). */
static int handle_op(Enum *E, int op, int c) {
    const Traces *S = E->S;
    const int rest = c - E->cost[op];
    if (op == O_F || op == O_G || op == O_X || op == O_NOT) {
        if (rest < 1) return 0;
        if (op == O_NOT && E->nnf && rest != E->cost[O_ATOM]) return 0;   /* only atoms are negated */
        for (uint64_t e = E->lvl_begin[rest]; e < E->lvl_end[rest]; e++) {
            uint8_t *m = new_mat(E);
            if (!m) return 1;
            const uint8_t *a = E->C.mat[e];
            if (op == O_F) sem_F(S, a, m);
            else if (op == O_G) sem_G(S, a, m);
            else if (op == O_X) sem_X(S, a, m);
            else sem_not(S, a, m);
            Prov pv = {(uint8_t)op, (uint32_t)e, 0};
            if (check_and_cache(E, c, m, pv)) return 1;
        }
        return 0;
    }
    /* binary: splits (cl, cr) with cl + cr = rest */
    for (int cl = 1; cl <= rest - 1; cl++) {
        int cr = rest - cl;
        if (op != O_U && cl > cr) continue;
        for (uint64_t a = E->lvl_begin[cl]; a < E->lvl_end[cl]; a++) {
            uint64_t b0 = E->lvl_begin[cr];
            if (op != O_U && cl == cr) b0 = a + 1;       /* unordered pairs a < b */
            for (uint64_t b = b0; b < E->lvl_end[cr]; b++) {
                uint8_t *m = new_mat(E);
                if (!m) return 1;
                if (op == O_AND) sem_and(S, E->C.mat[a], E->C.mat[b], m);
                else if (op == O_OR) sem_or(S, E->C.mat[a], E->C.mat[b], m);
                else sem_U(S, E->C.mat[a], E->C.mat[b], m);
                Prov pv = {(uint8_t)op, (uint32_t)a, (uint32_t)b};
                if (check_and_cache(E, c, m, pv)) return 1;
            }
        }
    }
    return 0;
}

static double now_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/*
 * oracle_learn_ex: minimal-cost separating formula by exhaustive enumeration.
 *   letters/offsets : n_pos + n_neg traces, positives first
 *   n_props         : alphabet size
 *   ops             : connective mask (Not=1 And=2 Or=4 X=8 F=16 G=32 U=64)
 *   max_size        : largest formula cost tried (inclusive, <= 63)
 *   stop_mode       : 1 first separator, 2 finish its level, 0 every level
 *   max_entries     : cache capacity in entries (0 = unlimited)
 *   costs           : 8 costs indexed atom, Not, And, Or, X, F, G, U (NULL: all 1)
 *   nnf             : nonzero = negation on atoms only
 *   max_errors      : misclassified traces a separator may have (0 = exact)
 *   formula_out     : text of the first separator found ("" if none)
 *   unique, cands, secs : per cost level 0..max_size (caller-allocated, max_size+1)
 *   levels_done     : number of levels fully enumerated
 * Returns OR_FOUND, OR_NOT_FOUND, OR_CAP, or an error.
 */
int oracle_learn_ex(const uint32_t *letters, const uint64_t *offsets, uint64_t n_pos, uint64_t n_neg,
                    int n_props, uint32_t ops, int max_size, int stop_mode, uint64_t max_entries,
                    const int *costs, int nnf, uint64_t max_errors,
                    char *formula_out, size_t formula_cap, int *found_size,
                    uint64_t *unique, uint64_t *cands, double *secs, int *levels_done) {
    if (n_props < 1 || n_props > 32 || max_size < 1 || max_size > 63 || !found_size || !levels_done)
        return OR_INVALID;
    Traces S = {letters, offsets, n_pos + n_neg, offsets[n_pos + n_neg]};
    for (uint64_t q = 0; q < S.total; q++)
        if (n_props < 32 && (letters[q] >> n_props)) return OR_INVALID;
    Enum E;
    memset(&E, 0, sizeof E);
    E.S = &S; E.n_pos = n_pos; E.stop_mode = stop_mode; E.max_errors = max_errors; E.nnf = nnf;
    for (int k = 0; k < 8; k++) {
        E.cost[k] = costs ? costs[k] : 1;
        if (E.cost[k] < 1) return OR_INVALID;
    }
    E.max_entries = max_entries ? max_entries : (uint64_t)-1;
    E.C.W = S.total;
    E.lvl_begin = (uint64_t *)calloc((size_t)max_size + 2, sizeof(uint64_t));
    E.lvl_end = (uint64_t *)calloc((size_t)max_size + 2, sizeof(uint64_t));
    E.unique = unique; E.cands = cands;
    for (int c = 0; c <= max_size; c++) { unique[c] = 0; cands[c] = 0; secs[c] = 0.0; }
    *levels_done = 0; *found_size = 0;
    if (formula_out && formula_cap) formula_out[0] = '\0';
    if (cache_grow_table(&E.C)) { free(E.lvl_begin); free(E.lvl_end); return OR_NOMEM; }

    static const int order[7] = {O_F, O_U, O_G, O_X, O_AND, O_OR, O_NOT};
    static const uint32_t bit_of[8] = {0, M_NOT, M_AND, M_OR, M_X, M_F, M_G, M_U};
    int stop = 0;
    for (int c = 1; c <= max_size && !stop && !E.err; c++) {
        double t0 = now_s();
        E.lvl_begin[c] = E.C.n;
        if (c == E.cost[O_ATOM]) {
            for (int p = 0; p < n_props && !stop; p++) {
                uint8_t *m = new_mat(&E);
                if (!m) { stop = 1; break; }
                sem_atom(&S, p, m);
                Prov pv = {O_ATOM, (uint32_t)p, 0};
                stop = check_and_cache(&E, c, m, pv);
            }
        } else {
            for (int k = 0; k < 7 && !stop; k++)
                if (ops & bit_of[order[k]]) stop = handle_op(&E, order[k], c);
        }
        E.lvl_end[c] = E.C.n;
        secs[c] = now_s() - t0;
        if (!stop && !E.err && !E.cap_hit) *levels_done = c;
        if (E.cap_hit) stop = 1;
        if (E.found && stop_mode != 0) stop = 1;
    }
    int rc;
    if (E.err) rc = E.err;
    else if (E.found) {
        rc = OR_FOUND;
        *found_size = E.found_size;
        Str s = {NULL, 0, 0};
        print_prov(&E.C, E.found_prov, &s);
        if (formula_out) {
            if (s.len + 1 > formula_cap) rc = OR_BUFSIZE;
            else memcpy(formula_out, s.buf, s.len + 1);
        }
        free(s.buf);
    } else if (E.cap_hit) rc = OR_CAP;
    else rc = OR_NOT_FOUND;
    cache_free(&E.C);
    free(E.lvl_begin); free(E.lvl_end);
    return rc;
}

/* oracle_learn: uniform cost, all connectives' negation, exact separation. */
int oracle_learn(const uint32_t *letters, const uint64_t *offsets, uint64_t n_pos, uint64_t n_neg,
                 int n_props, uint32_t ops, int max_size, int stop_mode, uint64_t max_entries,
                 char *formula_out, size_t formula_cap, int *found_size,
                 uint64_t *unique, uint64_t *cands, double *secs, int *levels_done) {
    return oracle_learn_ex(letters, offsets, n_pos, n_neg, n_props, ops, max_size, stop_mode, max_entries,
                           NULL, 0, 0, formula_out, formula_cap, found_size, unique, cands, secs, levels_done);
}
