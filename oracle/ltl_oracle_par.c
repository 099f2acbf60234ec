/*
 * ltl_oracle_par.c -- the oracle's enumeration on every host core.
 *
 * TEST INFRASTRUCTURE ONLY (like ltl_oracle.c, which this file includes
 * unchanged): used by the tests and by the benchmark's CPU-baseline timing.
 *
 * oracle_learn_par computes exactly what oracle_learn computes -- the same
 * Section 3 enumeration, candidates in the same order, the same exact
 * uniqueness check -- but builds the characteristic matrices of a block of
 * consecutive candidates in parallel (OpenMP threads, one candidate each, with
 * the literal clauses of ltl_oracle.c), together with their soundness verdict
 * (eq. (dagger)) and their hash-bucket index.  The block is then admitted to
 * the cache by one thread, candidate by candidate, in enumeration order, so
 * every count, the first separator and its formula text are those of the
 * serial oracle.  Uniform costs, all connectives' negation and exact
 * separation only (the benchmark's configuration).
 */
#include "ltl_oracle.c"

#include <omp.h>

typedef struct {
    int op;
    uint64_t a, b;
} Cand;

/* Candidates of level c with connective op, in the serial oracle's order
 * (handle_op): appended to *out. */
static int list_candidates(const Enum *E, int op, int c, Cand **out, uint64_t *n, uint64_t *cap) {
    const int rest = c - 1;
    if (rest < 1) return 0;
    if (op == O_F || op == O_G || op == O_X || op == O_NOT) {
        for (uint64_t e = E->lvl_begin[rest]; e < E->lvl_end[rest]; e++) {
            if (*n == *cap) {
                *cap = *cap ? 2 * *cap : 4096;
                Cand *m = (Cand *)realloc(*out, sizeof(Cand) * *cap);
                if (!m) return OR_NOMEM;
                *out = m;
            }
            (*out)[(*n)++] = (Cand){op, e, 0};
        }
        return 0;
    }
    for (int cl = 1; cl <= rest - 1; cl++) {
        int cr = rest - cl;
        if (op != O_U && cl > cr) continue;
        for (uint64_t a = E->lvl_begin[cl]; a < E->lvl_end[cl]; a++) {
            uint64_t b0 = E->lvl_begin[cr];
            if (op != O_U && cl == cr) b0 = a + 1;
            for (uint64_t b = b0; b < E->lvl_end[cr]; b++) {
                if (*n == *cap) {
                    *cap = *cap ? 2 * *cap : 4096;
                    Cand *m = (Cand *)realloc(*out, sizeof(Cand) * *cap);
                    if (!m) return OR_NOMEM;
                    *out = m;
                }
                (*out)[(*n)++] = (Cand){op, a, b};
            }
        }
    }
    return 0;
}

static void build_candidate(const Enum *E, const Cand *cd, uint8_t *m) {
    const Traces *S = E->S;
    const uint8_t *A = E->C.mat[cd->a];
    switch (cd->op) {
    case O_F: sem_F(S, A, m); break;
    case O_G: sem_G(S, A, m); break;
    case O_X: sem_X(S, A, m); break;
    case O_NOT: sem_not(S, A, m); break;
    case O_AND: sem_and(S, A, E->C.mat[cd->b], m); break;
    case O_OR: sem_or(S, A, E->C.mat[cd->b], m); break;
    default: sem_U(S, A, E->C.mat[cd->b], m); break;
    }
}

/* The admission step of check_and_cache for a candidate whose matrix m (owned),
 * soundness `sep` and FNV hash h were computed by a worker.  Returns 1 to stop. */
static int admit(Enum *E, int c, uint8_t *m, Prov pv, int sep, uint64_t h) {
    E->cands[c]++;
    if (sep) {
        if (!E->found) { E->found = 1; E->found_size = c; E->found_prov = pv; }
        if (E->stop_mode == 1) { free(m); return 1; }
    }
    if (2 * (E->C.n + 1) > E->C.nslot) {
        int rc = cache_grow_table(&E->C);
        if (rc) { free(m); E->err = rc; return 1; }
    }
    uint64_t k = h & (E->C.nslot - 1);
    while (E->C.slot[k]) {
        if (E->C.slot_hash[k] == h && memcmp(E->C.mat[E->C.slot[k] - 1], m, (size_t)E->C.W) == 0) {
            free(m);
            return 0;
        }
        k = (k + 1) & (E->C.nslot - 1);
    }
    if (E->C.n >= E->max_entries) {
        free(m);
        E->cap_hit = 1;
        return 0;
    }
    if (E->C.n == E->C.cap) {
        uint64_t nc = E->C.cap ? 2 * E->C.cap : 1024;
        uint8_t **nm = (uint8_t **)realloc(E->C.mat, sizeof(uint8_t *) * nc);
        Prov *np = nm ? (Prov *)realloc(E->C.prov, sizeof(Prov) * nc) : NULL;
        if (!nm || !np) { if (nm) E->C.mat = nm; free(m); E->err = OR_NOMEM; return 1; }
        E->C.mat = nm; E->C.prov = np; E->C.cap = nc;
    }
    E->C.mat[E->C.n] = m; E->C.prov[E->C.n] = pv; E->C.n++;
    E->C.slot[k] = E->C.n; E->C.slot_hash[k] = h;
    E->unique[c]++;
    return 0;
}

/*
 * oracle_learn_par: as oracle_learn (uniform cost, exact separation), with
 * up to `threads` OpenMP threads (0: the OpenMP default).  block_bytes bounds
 * the matrices built ahead of admission (0: 256 MiB).  threads_used receives
 * the team size.
 */
int oracle_learn_par(const uint32_t *letters, const uint64_t *offsets, uint64_t n_pos, uint64_t n_neg,
                     int n_props, uint32_t ops, int max_size, int stop_mode, uint64_t max_entries, int threads,
                     uint64_t block_bytes, char *formula_out, size_t formula_cap, int *found_size,
                     uint64_t *unique, uint64_t *cands, double *secs, int *levels_done, int *threads_used) {
    if (n_props < 1 || n_props > 32 || max_size < 1 || max_size > 63 || !found_size || !levels_done)
        return OR_INVALID;
    Traces S = {letters, offsets, n_pos + n_neg, offsets[n_pos + n_neg]};
    for (uint64_t q = 0; q < S.total; q++)
        if (n_props < 32 && (letters[q] >> n_props)) return OR_INVALID;
    if (threads > 0) omp_set_num_threads(threads);
    int team = 1;
#pragma omp parallel
    {
#pragma omp single
        team = omp_get_num_threads();
    }
    if (threads_used) *threads_used = team;
    Enum E;
    memset(&E, 0, sizeof E);
    E.S = &S; E.n_pos = n_pos; E.stop_mode = stop_mode; E.max_errors = 0; E.nnf = 0;
    for (int k = 0; k < 8; k++) E.cost[k] = 1;
    E.max_entries = max_entries ? max_entries : (uint64_t)-1;
    E.C.W = S.total;
    E.lvl_begin = (uint64_t *)calloc((size_t)max_size + 2, sizeof(uint64_t));
    E.lvl_end = (uint64_t *)calloc((size_t)max_size + 2, sizeof(uint64_t));
    E.unique = unique; E.cands = cands;
    for (int c = 0; c <= max_size; c++) { unique[c] = 0; cands[c] = 0; secs[c] = 0.0; }
    *levels_done = 0; *found_size = 0;
    if (formula_out && formula_cap) formula_out[0] = '\0';
    if (cache_grow_table(&E.C)) { free(E.lvl_begin); free(E.lvl_end); return OR_NOMEM; }
    const uint64_t Wb = E.C.W ? E.C.W : 1;
    uint64_t block = (block_bytes ? block_bytes : (256ull << 20)) / Wb;
    if (block < (uint64_t)team) block = (uint64_t)team;
    if (block > 65536) block = 65536;
    uint8_t **mats = (uint8_t **)calloc((size_t)block, sizeof(uint8_t *));
    int *sep = (int *)calloc((size_t)block, sizeof(int));
    uint64_t *hash = (uint64_t *)calloc((size_t)block, sizeof(uint64_t));
    Cand *list = NULL;
    uint64_t cap_list = 0;

    static const int order[7] = {O_F, O_U, O_G, O_X, O_AND, O_OR, O_NOT};
    static const uint32_t bit_of[8] = {0, M_NOT, M_AND, M_OR, M_X, M_F, M_G, M_U};
    int stop = 0;
    for (int c = 1; c <= max_size && !stop && !E.err; c++) {
        double t0 = now_s();
        E.lvl_begin[c] = E.C.n;
        if (c == 1) {
            for (int p = 0; p < n_props && !stop; p++) {
                uint8_t *m = new_mat(&E);
                if (!m) { stop = 1; break; }
                sem_atom(&S, p, m);
                Prov pv = {O_ATOM, (uint32_t)p, 0};
                stop = check_and_cache(&E, c, m, pv);
            }
        } else {
            for (int k = 0; k < 7 && !stop && !E.err; k++) {
                if (!(ops & bit_of[order[k]])) continue;
                uint64_t n = 0;
                if (list_candidates(&E, order[k], c, &list, &n, &cap_list)) { E.err = OR_NOMEM; break; }
                for (uint64_t base = 0; base < n && !stop && !E.err; base += block) {
                    const int64_t nb = (int64_t)(n - base < block ? n - base : block);
                    int oom = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : oom)
                    for (int64_t i = 0; i < nb; i++) {
                        uint8_t *m = (uint8_t *)malloc((size_t)Wb);
                        if (!m) { oom = 1; mats[i] = NULL; continue; }
                        build_candidate(&E, &list[base + (uint64_t)i], m);
                        mats[i] = m;
                        sep[i] = separates(&S, n_pos, m, 0);
                        hash[i] = fnv1a(m, E.C.W);
                    }
                    if (oom) {
                        for (int64_t i = 0; i < nb; i++) free(mats[i]);
                        E.err = OR_NOMEM;
                        break;
                    }
                    int64_t i = 0;
                    for (; i < nb && !stop; i++) {
                        const Cand *cd = &list[base + (uint64_t)i];
                        Prov pv = {(uint8_t)cd->op, (uint32_t)cd->a, (uint32_t)cd->b};
                        stop = admit(&E, c, mats[i], pv, sep[i], hash[i]);
                        mats[i] = NULL;
                    }
                    for (; i < nb; i++) { free(mats[i]); mats[i] = NULL; }
                }
            }
        }
        E.lvl_end[c] = E.C.n;
        secs[c] = now_s() - t0;
        if (!stop && !E.err && !E.cap_hit) *levels_done = c;
        if (E.cap_hit) stop = 1;
        if (E.found && stop_mode != 0) stop = 1;
    }
    free(list); free(mats); free(sep); free(hash);
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
