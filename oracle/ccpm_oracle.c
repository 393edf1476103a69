/*
 * ccpm_oracle.c -- CPU oracle for constraint-checking pattern matching.
 *
 * TEST INFRASTRUCTURE.  This file is not part of the product: only the tests,
 * the smoke check and the benchmark's CPU-baseline leg load it.  It is a plain,
 * slow, single-threaded restatement of the pruning steps of
 *   "Scalable Pattern Matching in Metadata Graphs via Constraint Checking"
 * and shares no code, header or table with the CUDA path.
 *
 * State (the paper's notation):
 *   omega[v]  -- bit q set  <=>  template vertex q is in omega(v)      (Alg. 3)
 *   A[e]      -- 1 byte per CSR entry e = (v, col[e]): edge still active,
 *                i.e. col[e] is in the active edge map epsilon(v)       (Alg. 3)
 * A vertex is active (alpha(v) = true) exactly when omega[v] != 0.
 *
 * Functions that are pinned only through the pipeline tests carry no extra
 * note; every function here is pinned (brute force, closed forms, Fig. 2
 * constructions, invariants) by the CPU test suite.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ENOMEM 2
#define OR_EBUDGET 6

static int popc32(uint32_t x) { int c = 0; while (x) { x &= x - 1; c++; } return c; }

/* Index of CSR entry (x, y), or -1.  Rows are sorted, so a plain binary
 * search over row x is exact. */
static int64_t entry_of(const int64_t *rp, const int32_t *col, int64_t x, int64_t y)
{
    int64_t lo = rp[x], hi = rp[x + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] == y) return mid;
        if (col[mid] < y) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3, INIT_VERTEX_STATE: omega(v) = {q : l(q) = l(v)}; an active vertex  */
/* keeps every incident edge, an inactive one keeps none.  An edge needs both */
/* endpoints active to carry a message, so A(v,u) = active(v) and active(u). */
/* ------------------------------------------------------------------------ */
void oracle_init(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *lab,
                 int n0, const uint8_t *tlab, uint32_t *omega, uint8_t *A)
{
    for (int64_t v = 0; v < n; v++) {
        uint32_t w = 0;
        for (int q = 0; q < n0; q++)
            if (tlab[q] == lab[v]) w |= 1u << q;
        omega[v] = w;
    }
    for (int64_t v = 0; v < n; v++)
        for (int64_t e = rp[v]; e < rp[v + 1]; e++)
            A[e] = (omega[v] != 0 && omega[col[e]] != 0) ? 1 : 0;
}

/* eta of Alg. 4: neighbour u can serve a local constraint of v iff some
 * template vertex a in omega(v) has a template neighbour b in omega(u). */
static int compatible(int n0, const uint32_t *tadj, uint32_t wv, uint32_t wu)
{
    for (int a = 0; a < n0; a++)
        if ((wv >> a) & 1u)
            if (tadj[a] & wu) return 1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One round of LOCAL_CONSTRAINT_CHECKING (Alg. 4 with the visitor of Alg. 5) */
/* in snapshot (Jacobi) form: every read uses round-k state (om_in, A_in),   */
/* every write goes to round-(k+1) state (om_out, A_out).                    */
/*                                                                           */
/* For an active v:                                                          */
/*  - edge elimination: entry (v,u) survives iff it was active and eta holds */
/*  - omega' = union of omega(u) over surviving entries (Alg. 4)             */
/*  - q stays in omega(v) iff adj(q) is a subset of omega' and, for every    */
/*    label L, at least |adj_L(q)| distinct surviving neighbours u have      */
/*    omega(u) meeting adj_L(q) (the "minimum number of distinct active      */
/*    neighbours with the same label", Section 4.1 and Section 4.3)          */
/*  - v is eliminated if omega(v) or its active edge map becomes empty.      */
/* Finally an entry is dropped if either endpoint was eliminated.            */
/* Returns 1 if omega or A changed.  *scanned += active entries read.        */
/* ------------------------------------------------------------------------ */
int oracle_lcc_round(int64_t n, const int64_t *rp, const int32_t *col,
                     int n0, const uint8_t *tlab, const uint32_t *tadj,
                     const uint32_t *om_in, const uint8_t *A_in,
                     uint32_t *om_out, uint8_t *A_out, int64_t *scanned)
{
    int changed = 0;
    int64_t sc = 0;
    /* every v writes only om_out[v]: the vertices can be processed in any
     * order, or in parallel when built with OpenMP */
#pragma omp parallel for schedule(dynamic, 4096) reduction(|:changed) reduction(+:sc)
    for (int64_t v = 0; v < n; v++) {
        uint32_t wv = om_in[v];
        if (wv == 0) { om_out[v] = 0; continue; }
        uint32_t omega_prime = 0;
        int64_t n_alive_edges = 0;
        for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
            if (!A_in[e]) continue;
            sc += 1;
            uint32_t wu = om_in[col[e]];
            if (!compatible(n0, tadj, wv, wu)) continue;
            omega_prime |= wu;
            n_alive_edges++;
        }
        uint32_t keep = 0;
        for (int q = 0; q < n0; q++) {
            if (!((wv >> q) & 1u)) continue;
            int ok = (tadj[q] & ~omega_prime) == 0;
            /* distinct-neighbour multiplicity, one label at a time */
            for (int b = 0; ok && b < n0; b++) {
                if (!((tadj[q] >> b) & 1u)) continue;
                uint32_t adj_L = 0;
                for (int c = 0; c < n0; c++)
                    if (((tadj[q] >> c) & 1u) && tlab[c] == tlab[b]) adj_L |= 1u << c;
                int need = popc32(adj_L);
                int have = 0;
                for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
                    if (!A_in[e]) continue;
                    uint32_t wu = om_in[col[e]];
                    if (!compatible(n0, tadj, wv, wu)) continue;
                    if (wu & adj_L) have++;
                }
                if (have < need) ok = 0;
            }
            if (ok) keep |= 1u << q;
        }
        if (n_alive_edges == 0) keep = 0;
        om_out[v] = keep;
        if (keep != wv) changed = 1;
    }
    *scanned += sc;
    /* every v writes only the entries of its own row */
#pragma omp parallel for schedule(dynamic, 4096) reduction(|:changed)
    for (int64_t v = 0; v < n; v++) {
        for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
            int64_t u = col[e];
            uint8_t a = A_in[e];
            if (a && !compatible(n0, tadj, om_in[v], om_in[u])) a = 0;
            if (om_out[v] == 0 || om_out[u] == 0) a = 0;
            A_out[e] = a;
            if (a != A_in[e]) changed = 1;
        }
    }
    return changed;
}

/* LCC repeated until a round eliminates nothing (Alg. 4's do-while).  Returns
 * the number of rounds executed, the final quiescent round included, or -1 on
 * allocation failure.  omega / A are updated in place. */
int64_t oracle_lcc(int64_t n, const int64_t *rp, const int32_t *col,
                   int n0, const uint8_t *tlab, const uint32_t *tadj,
                   uint32_t *omega, uint8_t *A, int64_t *scanned)
{
    int64_t m = rp[n];
    uint32_t *om2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *A2 = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    if (!om2 || !A2) { free(om2); free(A2); return -1; }
    int64_t rounds = 0;
    int changed;
    do {
        changed = oracle_lcc_round(n, rp, col, n0, tlab, tadj, omega, A, om2, A2, scanned);
        memcpy(omega, om2, sizeof(uint32_t) * (size_t)n);
        memcpy(A, A2, (size_t)m);
        rounds++;
    } while (changed);
    free(om2);
    free(A2);
    return rounds;
}

/* ------------------------------------------------------------------------ */
/* Rooted injective embedding of a substructure S of the template.           */
/* Used by NLCC (Alg. 6/7: does the token of head h issued at v come back /  */
/* get acknowledged?) and by the final template-driven search (Remark 1).    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
    const uint32_t *omega;
    const uint8_t *A;
    int k;                 /* |V_S| */
    int order[32];         /* template ids of S in visiting order, order[0] = root */
    int parent[32];        /* template id of an earlier S-neighbour, -1 for the root */
    uint32_t sadj[32];     /* S-adjacency of each template vertex (template-id masks) */
    int64_t psi[32];       /* current partial map: template id -> background vertex */
    /* enumeration outputs (final step only) */
    int enumerate;
    int64_t scanned;       /* CSR entries examined (edges-scanned metric) */
    uint64_t count;
    uint64_t cap;
    int over_budget;
    int n_e0;
    const int32_t *e0;     /* template edges, 2 per edge (enumeration marking) */
    uint32_t *om_mark;
    uint8_t *A_mark;
    /* listing (oracle_matches only) */
    int32_t *list;         /* row c = phi of the c-th match found, template id order */
    uint64_t list_cap;
    int n0;
    uint64_t *vcnt;        /* per vertex: matches that contain it */
    uint64_t *ecnt;        /* per CSR entry: matches that map a template edge onto it */
} search_t;

/* BFS over S from `root`, neighbours taken in increasing template id. */
static void make_order(search_t *s, uint32_t svert, int root)
{
    int head = 0, tail = 0;
    uint32_t seen = 1u << root;
    s->order[tail] = root; s->parent[tail] = -1; tail++;
    while (head < tail) {
        int x = s->order[head++];
        for (int y = 0; y < 32; y++) {
            if (!((svert >> y) & 1u) || ((seen >> y) & 1u)) continue;
            if (!((s->sadj[x] >> y) & 1u)) continue;
            seen |= 1u << y;
            s->order[tail] = y; s->parent[tail] = x; tail++;
        }
    }
    s->k = tail;
}

/* Order for a search rooted at the template edge (a, b): a, then b, then the
 * rest of the template breadth first (neighbours in increasing id). */
static void make_order_edge(search_t *s, uint32_t svert, int a, int b)
{
    int head = 0, tail = 0;
    uint32_t seen = (1u << a) | (1u << b);
    s->order[tail] = a; s->parent[tail] = -1; tail++;
    s->order[tail] = b; s->parent[tail] = a; tail++;
    while (head < tail) {
        int x = s->order[head++];
        for (int y = 0; y < 32; y++) {
            if (!((svert >> y) & 1u) || ((seen >> y) & 1u)) continue;
            if (!((s->sadj[x] >> y) & 1u)) continue;
            seen |= 1u << y;
            s->order[tail] = y; s->parent[tail] = x; tail++;
        }
    }
    s->k = tail;
}

static int extend(search_t *s, int i)
{
    if (i == s->k) {
        if (!s->enumerate) return 1;
        if (s->enumerate == 2) {
            if (s->list && s->count < s->list_cap)
                for (int q = 0; q < s->n0; q++) s->list[s->count * (uint64_t)s->n0 + (uint64_t)q] = (int32_t)s->psi[q];
            s->count++;
            for (int q = 0; q < s->n0; q++) s->vcnt[s->psi[q]] += 1;
            for (int t = 0; t < s->n_e0; t++) {
                int64_t x = s->psi[s->e0[2 * t]], y = s->psi[s->e0[2 * t + 1]];
                s->ecnt[entry_of(s->rp, s->col, x, y)] += 1;
                s->ecnt[entry_of(s->rp, s->col, y, x)] += 1;
            }
            return 0;
        }
        s->count++;
        for (int j = 0; j < s->k; j++) {
            int q = s->order[j];
            s->om_mark[s->psi[q]] |= 1u << q;
        }
        for (int t = 0; t < s->n_e0; t++) {
            int64_t x = s->psi[s->e0[2 * t]], y = s->psi[s->e0[2 * t + 1]];
            s->A_mark[entry_of(s->rp, s->col, x, y)] = 1;
            s->A_mark[entry_of(s->rp, s->col, y, x)] = 1;
        }
        if (s->count > s->cap) { s->over_budget = 1; return 1; }
        return 0;
    }
    int q = s->order[i];
    int64_t anchor = s->psi[s->parent[i]];
    for (int64_t e = s->rp[anchor]; e < s->rp[anchor + 1]; e++) {
        s->scanned++;
        if (!s->A[e]) continue;
        int64_t u = s->col[e];
        if (!((s->omega[u] >> q) & 1u)) continue;
        int ok = 1;
        for (int j = 0; j < i && ok; j++) {          /* injectivity */
            if (s->psi[s->order[j]] == u) ok = 0;
        }
        for (int j = 0; j < i && ok; j++) {          /* every S-edge to an earlier vertex */
            int b = s->order[j];
            if (!((s->sadj[q] >> b) & 1u)) continue;
            int64_t f = entry_of(s->rp, s->col, s->psi[b], u);
            if (f < 0 || !s->A[f]) ok = 0;
        }
        if (!ok) continue;
        s->psi[q] = u;
        if (extend(s, i + 1)) return 1;
    }
    s->psi[q] = -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* NON_LOCAL_CONSTRAINT_CHECKING for one constraint C0 (Alg. 6 and 7).        */
/* S = (svert, sadj) is a substructure of the template; `heads` are the       */
/* template vertices whose matches issue tokens.  Against one snapshot of     */
/* (omega, A): a vertex v with h in omega(v) keeps h iff some injective map   */
/* psi of S with psi(h) = v has q in omega(psi(q)) for every q and an active  */
/* edge for every edge of S.  Unsatisfied issuers lose h (Alg. 6); a vertex   */
/* whose omega empties is eliminated and its edges go with it.               */
/* Returns 1 if any omega changed, else 0; -1 on allocation failure.         */
/* ------------------------------------------------------------------------ */
int oracle_nlcc(int64_t n, const int64_t *rp, const int32_t *col,
                uint32_t svert, const uint32_t *sadj, uint32_t heads,
                uint32_t *omega, uint8_t *A, int64_t *n_tokens, int64_t *n_scanned)
{
    int64_t m = rp[n];
    uint32_t *om0 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *A0 = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    if (!om0 || !A0) { free(om0); free(A0); return -1; }
    memcpy(om0, omega, sizeof(uint32_t) * (size_t)n);
    memcpy(A0, A, (size_t)m);
    search_t s0;
    memset(&s0, 0, sizeof(s0));
    s0.n = n; s0.rp = rp; s0.col = col; s0.omega = om0; s0.A = A0;
    for (int q = 0; q < 32; q++) s0.sadj[q] = sadj[q] & svert;
    int64_t tokens = 0, scanned = 0;
    for (int h = 0; h < 32; h++) {
        if (!((heads >> h) & 1u) || !((svert >> h) & 1u)) continue;
        make_order(&s0, svert, h);
        /* every issuer is searched against the snapshot and writes only its
         * own omega word: issuers are independent */
#pragma omp parallel reduction(+:tokens, scanned)
        {
            search_t s = s0;
#pragma omp for schedule(dynamic, 256)
            for (int64_t v = 0; v < n; v++) {
                if (!((om0[v] >> h) & 1u)) continue;
                tokens += 1;
                for (int j = 0; j < 32; j++) s.psi[j] = -1;
                s.psi[h] = v;
                int sat = extend(&s, 1);
                if (!sat) omega[v] &= ~(1u << h);
            }
            scanned += s.scanned;
        }
    }
    *n_tokens += tokens;
    int changed = 0;
    for (int64_t v = 0; v < n; v++) {
        if (omega[v] != om0[v]) changed = 1;
        if (om0[v] != 0 && omega[v] == 0) {
            for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
                A[e] = 0;
                int64_t r = entry_of(rp, col, col[e], v);
                if (r >= 0) A[r] = 0;
            }
        }
    }
    *n_scanned += scanned;
    free(om0);
    free(A0);
    return changed;
}

/* ------------------------------------------------------------------------ */
/* Final template-driven search on the pruned graph (Remark 1; Section 4.7:  */
/* the walk covers the full template, work aggregation off, every match      */
/* verified).  Enumerates every injective phi with q in omega(phi(q)) and an  */
/* active edge for every template edge.  Outputs: om_out[v] = {q : some match */
/* has phi(q) = v}, A_out[e] = 1 iff e is the image of a template edge in    */
/* some match (both directions), *count = number of matches phi.             */
/* Returns OR_OK, or OR_EBUDGET once the count exceeds `cap`: the count is   */
/* then invalid, and om_out / A_out are finished by existence searches, one   */
/* per (vertex, template vertex) and one per (entry, template edge), so they  */
/* are exact all the same.                                                    */
/* ------------------------------------------------------------------------ */
int oracle_final(int64_t n, const int64_t *rp, const int32_t *col,
                 int n0, const uint32_t *tadj, int m0, const int32_t *tedges,
                 const uint32_t *omega, const uint8_t *A,
                 uint32_t *om_out, uint8_t *A_out, uint64_t *count, uint64_t cap,
                 int64_t *n_scanned)
{
    int64_t m = rp[n];
    memset(om_out, 0, sizeof(uint32_t) * (size_t)n);
    memset(A_out, 0, (size_t)m);
    search_t s;
    memset(&s, 0, sizeof(s));
    s.n = n; s.rp = rp; s.col = col; s.omega = omega; s.A = A;
    s.enumerate = 1; s.cap = cap; s.n_e0 = m0; s.e0 = tedges;
    s.om_mark = om_out; s.A_mark = A_out;
    uint32_t all = (n0 >= 32) ? 0xFFFFFFFFu : ((1u << n0) - 1u);
    for (int q = 0; q < n0; q++) s.sadj[q] = tadj[q];
    make_order(&s, all, 0);
    for (int64_t v = 0; v < n && !s.over_budget; v++) {
        if (!(omega[v] & 1u)) continue;
        for (int j = 0; j < 32; j++) s.psi[j] = -1;
        s.psi[0] = v;
        extend(&s, 1);
    }
    if (!s.over_budget) {
        *count = s.count;
        *n_scanned += s.scanned;
        return OR_OK;
    }
    memset(om_out, 0, sizeof(uint32_t) * (size_t)n);
    memset(A_out, 0, (size_t)m);
    s.enumerate = 0;
    int64_t scanned = s.scanned;
    /* existence searches are independent of each other: per (v, q) the only
     * write is om_out[v]; per entry the writes set flags to 1 (atomically,
     * as a reverse entry belongs to another row) */
    for (int q = 0; q < n0; q++) {
        make_order(&s, all, q);
#pragma omp parallel reduction(+:scanned)
        {
            search_t t = s;
            t.scanned = 0;
#pragma omp for schedule(dynamic, 256)
            for (int64_t v = 0; v < n; v++) {
                if (!((omega[v] >> q) & 1u)) continue;
                for (int j = 0; j < 32; j++) t.psi[j] = -1;
                t.psi[q] = v;
                if (extend(&t, 1)) om_out[v] |= 1u << q;
            }
            scanned += t.scanned;
        }
    }
    for (int te = 0; te < m0; te++) {
        int a = tedges[2 * te], b = tedges[2 * te + 1];
        make_order_edge(&s, all, a, b);
#pragma omp parallel reduction(+:scanned)
        {
            search_t t = s;
            t.scanned = 0;
#pragma omp for schedule(dynamic, 256)
            for (int64_t x = 0; x < n; x++) {
                if (!((omega[x] >> a) & 1u)) continue;
                for (int64_t e = rp[x]; e < rp[x + 1]; e++) {
                    int64_t y = col[e];
                    uint8_t done;
#pragma omp atomic read
                    done = A_out[e];
                    if (!A[e] || !((omega[y] >> b) & 1u) || done) continue;
                    for (int j = 0; j < 32; j++) t.psi[j] = -1;
                    t.psi[a] = x;
                    t.psi[b] = y;
                    if (extend(&t, 2)) {
                        int64_t r = entry_of(rp, col, y, x);
#pragma omp atomic write
                        A_out[e] = 1;
#pragma omp atomic write
                        A_out[r] = 1;
                    }
                }
            }
            scanned += t.scanned;
        }
    }
    *count = 0;
    *n_scanned += scanned;
    return OR_EBUDGET;
}

/* ------------------------------------------------------------------------ */
/* Every match of the template inside (omega, A), for the analyses the paper  */
/* names as the point of pruning (Introduction: listing the matches, and     */
/* per-vertex / per-edge participation, i.e. match-based centrality).  Plain */
/* backtracking from template vertex 0 over vertices in increasing id; a      */
/* match phi is listed as phi(0..n0-1) (the first list_cap of them, in the    */
/* order found).  vcnt[v] = number of matches with v in phi(V0); ecnt[e] =    */
/* number of matches that map a template edge onto the undirected edge of     */
/* entry e (both entries of an edge get the same count).  Returns the number  */
/* of matches.                                                               */
/* ------------------------------------------------------------------------ */
uint64_t oracle_matches(int64_t n, const int64_t *rp, const int32_t *col,
                        int n0, const uint32_t *tadj, int m0, const int32_t *tedges,
                        const uint32_t *omega, const uint8_t *A,
                        int32_t *list, uint64_t list_cap, uint64_t *vcnt, uint64_t *ecnt)
{
    int64_t m = rp[n];
    memset(vcnt, 0, sizeof(uint64_t) * (size_t)n);
    memset(ecnt, 0, sizeof(uint64_t) * (size_t)m);
    search_t s;
    memset(&s, 0, sizeof(s));
    s.n = n; s.rp = rp; s.col = col; s.omega = omega; s.A = A;
    s.enumerate = 2; s.cap = (uint64_t)-1; s.n_e0 = m0; s.e0 = tedges;
    s.list = list; s.list_cap = list_cap; s.n0 = n0; s.vcnt = vcnt; s.ecnt = ecnt;
    uint32_t all = (n0 >= 32) ? 0xFFFFFFFFu : ((1u << n0) - 1u);
    for (int q = 0; q < n0; q++) s.sadj[q] = tadj[q];
    make_order(&s, all, 0);
    for (int64_t v = 0; v < n; v++) {
        if (!(omega[v] & 1u)) continue;
        for (int j = 0; j < 32; j++) s.psi[j] = -1;
        s.psi[0] = v;
        extend(&s, 1);
    }
    return s.count;
}

/* ======================================================================== */
/* Wider templates and edge labels (the LCC phase only).                     */
/*                                                                          */
/* The paper's LCC storage estimate budgets eight bytes of omega per vertex  */
/* for a template of 64 vertices (Section 5.1), and its graphs carry         */
/* metadata on edges as well as vertices (Section 3).  Here omega is a       */
/* 64-bit word (bit q = template vertex q, n0 <= 64), graph entry e carries  */
/* the edge label el[e] (the same on both directions of an edge; all 0 when  */
/* el is NULL) and template edge i carries tel[i] (all 0 when tel is NULL).  */
/* A match must map every template edge onto a graph edge of the same label, */
/* so the local constraints of Alg. 4 read, per edge label L:                */
/*  - eta: entry (v,u) labelled L survives iff some a in omega(v) has a      */
/*    template neighbour b in omega(u) joined to a by an edge labelled L;    */
/*  - coverage: each template neighbour b of q, joined by label L, lies in   */
/*    omega(u) for some surviving entry (v,u) labelled L;                    */
/*  - multiplicity: for each pair (vertex label, edge label), at least as    */
/*    many distinct surviving neighbours u reached by that edge label have   */
/*    omega(u) meeting q's template neighbours of that pair as q has such    */
/*    neighbours.                                                            */
/* With every edge label 0 these are exactly the rules of oracle_lcc_round.  */
/* Rounds are snapshot (Jacobi) rounds, counted as in oracle_lcc.            */
/* ======================================================================== */

typedef struct {
    int n0;
    uint8_t tlab[64];
    uint64_t adj[256][64];   /* adj[L][q]: template neighbours of q via edges labelled L */
    uint64_t any[64];        /* template neighbours of q, any edge label */
    int n_used;              /* edge labels some template edge carries ... */
    uint8_t used[256];       /* ... (adj[L] is empty for every other L) */
} wide_tmpl_t;

static int popc64(uint64_t x) { int c = 0; while (x) { x &= x - 1; c++; } return c; }

static void wide_tables(int n0, const uint8_t *tlab, int m0, const int32_t *te, const uint8_t *tel,
                        wide_tmpl_t *t)
{
    memset(t, 0, sizeof(*t));
    t->n0 = n0;
    for (int q = 0; q < n0; q++) t->tlab[q] = tlab[q];
    for (int i = 0; i < m0; i++) {
        int a = te[2 * i], b = te[2 * i + 1];
        int L = tel ? tel[i] : 0;
        t->adj[L][a] |= 1ull << b;
        t->adj[L][b] |= 1ull << a;
        t->any[a] |= 1ull << b;
        t->any[b] |= 1ull << a;
    }
    for (int L = 0; L < 256; L++) {
        int nonempty = 0;
        for (int q = 0; q < n0; q++) nonempty |= t->adj[L][q] != 0;
        if (nonempty) t->used[t->n_used++] = (uint8_t)L;
    }
}

/* eta with an edge label: some a in wv has a template neighbour in wu via label L */
static int wide_compatible(const wide_tmpl_t *t, uint64_t wv, uint64_t wu, int L)
{
    for (int a = 0; a < t->n0; a++)
        if ((wv >> a) & 1ull)
            if (t->adj[L][a] & wu) return 1;
    return 0;
}

/* Alg. 3 with 64-bit omega: omega(v) = {q : l(q) = l(v)}; an entry is active
 * iff both of its ends are. */
void oracle_wide_init(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *lab,
                      int n0, const uint8_t *tlab, uint64_t *omega, uint8_t *A)
{
    for (int64_t v = 0; v < n; v++) {
        uint64_t w = 0;
        for (int q = 0; q < n0; q++)
            if (tlab[q] == lab[v]) w |= 1ull << q;
        omega[v] = w;
    }
    for (int64_t v = 0; v < n; v++)
        for (int64_t e = rp[v]; e < rp[v + 1]; e++)
            A[e] = (omega[v] != 0 && omega[col[e]] != 0) ? 1 : 0;
}

static int wide_round(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *el,
                      const wide_tmpl_t *t, const uint64_t *om_in, const uint8_t *A_in,
                      uint64_t *om_out, uint8_t *A_out, int64_t *scanned)
{
    int changed = 0;
    int64_t sc = 0;
    static uint64_t U[256];   /* omega' per edge label (single-threaded use) */
    for (int64_t v = 0; v < n; v++) {
        uint64_t wv = om_in[v];
        if (wv == 0) { om_out[v] = 0; continue; }
        memset(U, 0, sizeof(U));
        int64_t n_alive_edges = 0;
        for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
            if (!A_in[e]) continue;
            sc += 1;
            int L = el ? el[e] : 0;
            uint64_t wu = om_in[col[e]];
            if (!wide_compatible(t, wv, wu, L)) continue;
            U[L] |= wu;
            n_alive_edges++;
        }
        uint64_t keep = 0;
        for (int q = 0; q < t->n0; q++) {
            if (!((wv >> q) & 1ull)) continue;
            int ok = 1;
            /* coverage, edge label by edge label (labels no template edge
             * carries have no template neighbours to cover) */
            for (int i = 0; ok && i < t->n_used; i++) {
                int L = t->used[i];
                if (t->adj[L][q] & ~U[L]) ok = 0;
            }
            /* distinct-neighbour multiplicity per (vertex label, edge label) */
            for (int i = 0; ok && i < t->n_used; i++) {
                int L = t->used[i];
                for (int b = 0; ok && b < t->n0; b++) {
                    if (!((t->adj[L][q] >> b) & 1ull)) continue;
                    uint64_t cls = 0;
                    for (int c = 0; c < t->n0; c++)
                        if (((t->adj[L][q] >> c) & 1ull) && t->tlab[c] == t->tlab[b]) cls |= 1ull << c;
                    int need = popc64(cls);
                    int have = 0;
                    for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
                        if (!A_in[e]) continue;
                        if ((el ? el[e] : 0) != L) continue;
                        uint64_t wu = om_in[col[e]];
                        if (!wide_compatible(t, wv, wu, L)) continue;
                        if (wu & cls) have++;
                    }
                    if (have < need) ok = 0;
                }
            }
            if (ok) keep |= 1ull << q;
        }
        if (n_alive_edges == 0) keep = 0;
        om_out[v] = keep;
        if (keep != wv) changed = 1;
    }
    *scanned += sc;
    for (int64_t v = 0; v < n; v++) {
        for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
            int64_t u = col[e];
            uint8_t a = A_in[e];
            if (a && !wide_compatible(t, om_in[v], om_in[u], el ? el[e] : 0)) a = 0;
            if (om_out[v] == 0 || om_out[u] == 0) a = 0;
            A_out[e] = a;
            if (a != A_in[e]) changed = 1;
        }
    }
    return changed;
}

/* One snapshot round (for the tests of single rounds).  Returns 1 if omega or
 * A changed. */
int oracle_wide_lcc_round(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *el,
                          int n0, const uint8_t *tlab, int m0, const int32_t *te, const uint8_t *tel,
                          const uint64_t *om_in, const uint8_t *A_in, uint64_t *om_out, uint8_t *A_out,
                          int64_t *scanned)
{
    wide_tmpl_t *t = (wide_tmpl_t *)malloc(sizeof(wide_tmpl_t));
    if (!t) return -1;
    wide_tables(n0, tlab, m0, te, tel, t);
    int ch = wide_round(n, rp, col, el, t, om_in, A_in, om_out, A_out, scanned);
    free(t);
    return ch;
}

/* Init, then rounds until one changes nothing.  Returns the rounds executed
 * (the quiescent one included), or -1 on allocation failure. */
int64_t oracle_wide_lcc(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *lab, const uint8_t *el,
                        int n0, const uint8_t *tlab, int m0, const int32_t *te, const uint8_t *tel,
                        uint64_t *omega, uint8_t *A, int64_t *scanned)
{
    int64_t m = rp[n];
    wide_tmpl_t *t = (wide_tmpl_t *)malloc(sizeof(wide_tmpl_t));
    uint64_t *om2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *A2 = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    if (!t || !om2 || !A2) { free(t); free(om2); free(A2); return -1; }
    wide_tables(n0, tlab, m0, te, tel, t);
    oracle_wide_init(n, rp, col, lab, n0, tlab, omega, A);
    int64_t rounds = 0;
    int changed;
    do {
        changed = wide_round(n, rp, col, el, t, omega, A, om2, A2, scanned);
        memcpy(omega, om2, sizeof(uint64_t) * (size_t)n);
        memcpy(A, A2, (size_t)m);
        rounds++;
    } while (changed);
    free(t);
    free(om2);
    free(A2);
    return rounds;
}
