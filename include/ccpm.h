/*
 * ccpm.h -- C ABI of the GB300 constraint-checking pattern matcher.
 *
 * The library prunes a vertex-labelled background graph G down to exactly the
 * vertices and edges that take part in at least one exact match of a small
 * connected template G0 (Definition 1 of "Scalable Pattern Matching in
 * Metadata Graphs via Constraint Checking"): local constraint checking to a
 * fixpoint (Alg. 4), one non-local constraint at a time with LCC re-run after
 * any change (Alg. 1, Alg. 6/7), and a final template-driven search over the
 * whole template (Remark 1, Section 4.7) that also counts matches.
 *
 * Conventions
 *   - Every call returns an int status (CCPM_OK or a CCPM_E* code); no C++
 *     exception crosses this boundary.  ccpm_last_error() gives a message.
 *   - Graph layout: undirected simple graph in CSR, each undirected edge stored
 *     in both rows; row_ptr is int64 [n+1], col is int32 [m_dir] with every row
 *     sorted ascending, no self loops, no duplicates.  labels is uint8 [n].
 *   - omega layout: uint32 per vertex; bit q set <=> template vertex q is a
 *     possible match of that vertex (omega(v) of Section 3).
 *   - Edge bitmap layout: one bit per CSR entry e, bit (e & 31) of word e >> 5
 *     (uint32 words, ceil(m_dir / 32) of them); both directions of an
 *     undirected edge always carry the same value.
 *   - Calls run on the context's CUDA stream and return after the work they
 *     describe has completed, unless stated otherwise.
 *   - Calls that take a context (or a graph, template or result made with
 *     one) make the context's device current on the calling thread and leave
 *     it current; ccpm_lcc_fixpoint_noalloc, which takes no context, restores
 *     the caller's current device.
 *   - All handles are single-thread objects: do not use one handle from two
 *     host threads at once.
 */
#ifndef CCPM_H
#define CCPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCPM_OK        0
#define CCPM_EINVAL    1   /* bad argument, bad CSR, bad template             */
#define CCPM_ENOMEM    2   /* host or device allocation failed                 */
#define CCPM_ECUDA     3   /* a CUDA runtime call failed                       */
#define CCPM_ETIMEOUT  4   /* a device-side wait gave up (bounded spin)        */
#define CCPM_EOVERFLOW 5   /* a fixed-capacity device buffer would overflow    */
#define CCPM_EBUDGET   6   /* a search budget was exceeded; see ccpm_counts    */
#define CCPM_ESTATE    7   /* call made in the wrong order                     */

/* ccpm_graph_load_csr flags */
#define CCPM_HOST_PTRS    0  /* pointers are host memory; the library copies them     */
#define CCPM_DEVICE_PTRS  1  /* pointers are device memory on the context's device,
                                borrowed: they must stay valid until the graph is
                                destroyed and must not be modified meanwhile       */
#define CCPM_VALIDATE     2  /* check sortedness, symmetry, self loops, duplicates */

#define CCPM_MAX_TMPL_VERTICES 32
#define CCPM_MAX_TMPL_EDGES    496

/* constraint kinds (Table 3): path, cycle, and the three TDS unions */
#define CCPM_KIND_PC     0
#define CCPM_KIND_CC     1
#define CCPM_KIND_TDS_CC 2
#define CCPM_KIND_TDS_PC 3
#define CCPM_KIND_TDS    4

/* constraint order (Section 4.2 "Constraint Ordering Heuristics") */
#define CCPM_ORDER_FIXED    0  /* the paper's heuristic: paths and cycles first, shorter first */
#define CCPM_ORDER_EXPLICIT 1  /* the order given by ccpm_tmpl_set_order                       */
#define CCPM_ORDER_LEARNED  2  /* before each constraint, the remaining ones are scored by the
                                  ordering network (options.mlp) and the best runs next; every
                                  constraint still runs, so results equal the fixed order's     */

/* ordering network: 16 features -> 64 -> 64 -> 1 (ReLU) */
#define CCPM_MLP_IN      16
#define CCPM_MLP_HIDDEN  64
#define CCPM_MLP_PARAMS  (CCPM_MLP_IN * CCPM_MLP_HIDDEN + CCPM_MLP_HIDDEN + \
                          CCPM_MLP_HIDDEN * CCPM_MLP_HIDDEN + CCPM_MLP_HIDDEN + CCPM_MLP_HIDDEN + 1)

typedef struct ccpm_ctx    *ccpm_ctx_t;
typedef struct ccpm_graph  *ccpm_graph_t;
typedef struct ccpm_tmpl   *ccpm_tmpl_t;
typedef struct ccpm_result *ccpm_result_t;
typedef struct ccpm_mlp    *ccpm_mlp_t;

typedef struct {
    int      kind;                 /* CCPM_KIND_*                                  */
    int      n_verts;              /* |V_S|                                        */
    uint32_t vert_mask;            /* bit q: template vertex q is in S             */
    uint32_t head_mask;            /* template vertices whose matches issue tokens */
    int      n_edges;              /* |E_S|                                        */
    int32_t  edges[CCPM_MAX_TMPL_EDGES][2];   /* (a, b), a < b, sorted             */
} ccpm_constraint_info;

typedef struct {
    int      order_mode;           /* CCPM_ORDER_*                                  */
    int      run_final;            /* 1 (default): final exact search + counting   */
    uint64_t max_embeddings;       /* final search stops past this many matches    */
    uint64_t search_budget;        /* max 32-candidate windows one root may scan;  */
                                   /* 0 = library default                          */
    int      hub_degree;           /* rows longer than this are split across warps;*/
                                   /* 0 = library default (1024); values above    */
                                   /* 2^24 are treated as 2^24                     */
    int      batch_workers;        /* ccpm_prune_batch: concurrent workers, 0 = the */
                                   /* autotuned choice for this graph              */
    int      resume;               /* ccpm_prune: 1 = start from the state held in */
                                   /* *out (a result of this graph and template,  */
                                   /* e.g. one read back by ccpm_state_import)     */
                                   /* instead of from the initial state of Alg. 3  */
    int      compact;              /* row compaction between LCC rounds: 0 = when  */
                                   /* most entries of the live rows are inactive,  */
                                   /* 1 = after every round that leaves some, -1 = */
                                   /* never; results are the same in all modes     */
    int      search_split;         /* windows a search scans before it hands its   */
                                   /* untried candidates to other warps: 0 = the   */
                                   /* library default (2048), -1 = never; results  */
                                   /* are the same for every value                 */
    int      lcc_only;             /* 1: stop at the first LCC fixpoint (no non-   */
                                   /* local constraint, no final search); the     */
                                   /* result holds that fixpoint                   */
    int      short_rows;           /* rows up to this many entries are walked 32   */
                                   /* rows per warp as one stream; longer ones a   */
                                   /* warp per row: 0 = library default (64)      */
    int      no_edge_elimination;  /* 1: ablation: LCC counts every live neighbour */
                                   /* (no edge elimination by eta); ω*, E* and    */
                                   /* the count are unchanged, only the time      */
    int      entry_labels;         /* first LCC round reads a per-graph copy of the */
                                   /* neighbour labels in entry order (1 byte per  */
                                   /* entry, built once): 0 = when the initially   */
                                   /* active rows hold >= 1/8 of the entries and   */
                                   /* >= 2^22, 1 = always, -1 = never; same result */
    int      grid_share;           /* ccpm_prune_batch: while k workers are busy,  */
                                   /* each sizes its grids for 1/min(grid_share,k) */
                                   /* of the GPU's SMs, so that kernels of several */
                                   /* templates run side by side instead of one   */
                                   /* filling every SM, and the last templates of */
                                   /* a batch get the whole GPU back: 0 = the     */
                                   /* autotuned choice, 1 = the whole GPU always  */
    ccpm_mlp_t mlp;                /* ordering network for CCPM_ORDER_LEARNED       */
} ccpm_options;

/* What happened to one non-local constraint during a prune (the training log
 * of the ordering network).  features are the network's inputs at the moment
 * the constraint was chosen; bits_* are sums of |omega(v)| over all vertices
 * before the constraint and after its LCC re-run. */
typedef struct {
    int32_t  constraint;           /* index in the generated (fixed) order          */
    int32_t  position;             /* 0-based position at which it ran              */
    float    features[CCPM_MLP_IN];
    int64_t  bits_before, bits_after;
    int32_t  lcc_rounds;           /* LCC rounds of the re-run (0 if nothing changed)*/
    int32_t  tokens;               /* (vertex, head) walks it issued                 */
    double   ms_search, ms_lcc;    /* device time of its search and of the re-run   */
} ccpm_constraint_log;

typedef struct {
    int64_t  active_v;             /* vertices with omega != 0 at the end         */
    int64_t  active_e_dir;         /* set bits in the edge bitmap (2 x |E*|)      */
    int64_t  lcc_rounds_total;     /* LCC rounds over all phases, each phase      */
                                   /* counting its final quiescent round          */
    int32_t  n_phases;             /* 1 + number of non-local constraints         */
    int32_t  nlcc_constraints_run;
    uint64_t match_embeddings;     /* number of matches phi (valid if count_valid)*/
    uint64_t automorphisms;        /* label-preserving automorphisms of G0        */
    uint64_t match_subgraphs;      /* match_embeddings / automorphisms            */
    int32_t  count_valid;          /* 0 if the final search hit a budget          */
    int32_t  status;               /* status of the prune call                    */
    int64_t  tokens;               /* (vertex, head) token walks issued by NLCC   */
    int64_t  edges_scanned_lcc;    /* sum over LCC rounds of active CSR entries   */
    int64_t  edges_scanned_search; /* CSR entries examined by NLCC + final search */
    double   ms_total, ms_lcc, ms_nlcc, ms_final;   /* device time per stage     */
    /* measurement of the LCC round kernel (CUDA events around each launch on
     * the context stream) and the traffic the method itself needs per round
     * (Alg. 4 over n_a active vertices and M_a active CSR entries):
     *   16 B per active vertex (two 4-byte row offsets, omega read and write)
     * + 8.25 B per active entry (column index, gather of the neighbour's
     *   omega, read and write of its edge bit)                              */
    int64_t  lcc_launches;
    double   ms_lcc_kernel;
    int64_t  lcc_alg_bytes;        /* sum over rounds of 8.25 M_a + 16 n_a      */
    int64_t  lcc_row_entries;      /* CSR entries in rows of active vertices  */
    int64_t  lcc_active_vertices;  /* active vertices, summed over rounds      */
    int64_t  kernel_launches;      /* all kernels this call launched          */
    int64_t  lcc_compactions;      /* row compactions (K4) between LCC rounds */
    double   ms_search_kernel;     /* device time of the NLCC search kernels  */
    int64_t  search_launches;      /* their launches                          */
    int64_t  search_entries_nlcc;  /* row entries those kernels examined      */
    /* what the kernel itself reads and writes per round: 24 B per active
     * vertex (two int64 offsets, omega read and write) + 4.125 B per entry of
     * an active row (column index, edge bit) + 4 B per active entry (gather) */
    int64_t  lcc_kernel_bytes;
    int64_t  lcc_first_entries;    /* M_a of the first round after init       */
    double   ms_lcc_first;         /* device time of that round               */
    /* device time of the final step's parts: the enumerations that count (and
     * mark) matches, the per-(vertex, template vertex) existence searches and
     * the per-entry existence searches (both only when the count is capped)  */
    double   ms_final_count, ms_final_vertex, ms_final_edge;
} ccpm_counts;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA `device`.  `cuda_stream` (a cudaStream_t) may be
 * NULL, in which case the library creates and owns a stream.  A non-NULL
 * stream is borrowed and must outlive the context. */
int  ccpm_ctx_create(int device, void *cuda_stream, ccpm_ctx_t *out);
void ccpm_ctx_destroy(ccpm_ctx_t ctx);
/* Message for the last failing call on this context (never NULL). */
const char *ccpm_last_error(ccpm_ctx_t ctx);
void ccpm_options_default(ccpm_options *opt);

/* ------------------------------------------------------------------ graph */

/* Load the background graph G (Section 3; CSR + separate label store as in
 * Section 4.8).  n vertices, m_dir directed CSR entries.  With
 * CCPM_HOST_PTRS the arrays are copied to the device; with CCPM_DEVICE_PTRS
 * they are borrowed.  CCPM_VALIDATE adds an O(m) host check (host pointers
 * only) and returns CCPM_EINVAL on an unsorted row, self loop, duplicate or a
 * missing reverse entry.  n must be < 2^31. */
int  ccpm_graph_load_csr(ccpm_ctx_t ctx, int64_t n, int64_t m_dir,
                         const int64_t *row_ptr, const int32_t *col,
                         const uint8_t *labels, int flags, ccpm_graph_t *out);
void ccpm_graph_destroy(ccpm_graph_t g);

/* --------------------------------------------------------------- template */

/* Load template G0 (Section 3): n0 in [2, 32] vertices with labels, m0
 * undirected edges given as 2*m0 int32 (a, b) pairs.  CCPM_EINVAL if G0 is
 * disconnected (Section 3 assumes connected), has a self loop, a duplicate or
 * an out-of-range vertex. */
int  ccpm_tmpl_load(ccpm_ctx_t ctx, int n0, const uint8_t *labels, int m0,
                    const int32_t *edges, ccpm_tmpl_t *out);
void ccpm_tmpl_destroy(ccpm_tmpl_t t);

/* Generate the ordered non-local constraint set K0 (Table 3 Steps 1-5,
 * Alg. 2, ordering of Section 4.2).  The graph supplies background label
 * frequencies used to orient token walks (Section 4.2 "Constraint
 * Optimization"); it may be NULL.  Writes |K0| to *n_constraints. */
int  ccpm_constraints_generate(ccpm_tmpl_t t, ccpm_graph_t g, int *n_constraints);
/* Describe constraint i (0-based, in the current order). */
int  ccpm_constraints_describe(ccpm_tmpl_t t, int i, ccpm_constraint_info *out);
/* Explicit order: order[j] = index (in the generated order) of the constraint
 * to check j-th; must be a permutation of 0..n-1.  Used with
 * CCPM_ORDER_EXPLICIT. */
int  ccpm_tmpl_set_order(ccpm_tmpl_t t, int n, const int32_t *order);

/* ------------------------------------------------------------------ prune */

/* Run the whole pipeline (Alg. 1 plus the final search of Remark 1) for
 * template t over graph g.  If *out is NULL a result is created; a non-NULL
 * *out made by an earlier call on the same graph is reused (its buffers are
 * overwritten).  Returns CCPM_OK, CCPM_EBUDGET or an error.  CCPM_EBUDGET
 * means a budget was reached: past options.max_embeddings the match count is
 * not reported (count_valid = 0) while omega and the edge bitmap are still
 * the exact answer; past options.search_budget a search kept its root as
 * satisfied, so omega and the bitmap are a superset of the exact answer. */
int  ccpm_prune(ccpm_ctx_t ctx, ccpm_graph_t g, ccpm_tmpl_t t,
                const ccpm_options *opt, ccpm_result_t *out);

/* Prune T templates over the same resident graph (the exploratory-search
 * workload of Section 6.7: many variants of one query).  Each template's
 * results are exactly those ccpm_prune gives for it.  The templates run
 * concurrently on worker streams of this context, each with its own scratch,
 * so that small phases of different templates overlap on the GPU.  With
 * options.batch_workers = 0 the settings come from an autotuner: on the first
 * call for this graph it prunes one slice of the batch (32 templates spread
 * evenly over it) once per candidate setting and keeps the fastest, choosing
 * in turn the worker count (1, 2, 4, 8, 16), options.grid_share (1, 2, 4),
 * options.search_split (2048, 512, 8192), options.short_rows (64, 32, 256)
 * and options.hub_degree (1024, 4096); the choice is kept on the graph and
 * applies to options left at 0.  When every outs[i] holds a result of an
 * earlier call, the templates start longest first by that result's time.
 * Every setting gives the same results.  outs[i] follows the same
 * create-or-reuse rule as ccpm_prune.  Returns CCPM_OK, CCPM_EBUDGET if any template hit a budget
 * (see each result's counts), or the first error. */
int  ccpm_prune_batch(ccpm_ctx_t ctx, ccpm_graph_t g, int T, const ccpm_tmpl_t *tmpls,
                      const ccpm_options *opt, ccpm_result_t *outs);
/* The worker count the autotuner chose for batches over g (0 before the first
 * autotuned ccpm_prune_batch call, or with NULL). */
int  ccpm_graph_batch_workers(ccpm_graph_t g);
/* All the autotuner's choices for g (zeros before the first autotuned batch;
 * 0 for search_split, short_rows or hub_degree = the library default) and
 * the chosen setting's wall time on the tuning slice in milliseconds.  Any
 * pointer may be NULL. */
int  ccpm_graph_batch_tuning(ccpm_graph_t g, int *workers, int *grid_share, int *search_split, int *short_rows,
                             int *hub_degree, double *slice_ms);

/* ----------------------------------------------------------------- result */

/* Copy omega (n uint32) to dst (host memory, or device memory when
 * dst_on_device != 0). */
int  ccpm_result_omega(ccpm_result_t r, uint32_t *dst, int64_t n, int dst_on_device);
/* Copy the edge bitmap (ceil(m_dir/32) words) to dst. */
int  ccpm_result_edge_bitmap(ccpm_result_t r, uint32_t *dst, int64_t words, int dst_on_device);
int  ccpm_result_counts(ccpm_result_t r, ccpm_counts *out);
/* LCC rounds per phase: [initial LCC, after constraint 1, ...]; a phase whose
 * constraint changed nothing has 0 rounds.  Writes min(cap, n_phases). */
int  ccpm_result_phase_rounds(ccpm_result_t r, int32_t *dst, int cap);
/* Every match of the template within a result of this graph and template
 * (the listing and the per-vertex / per-edge participation counts that the
 * Introduction names as what pruning is for; Section 4.7: the full-template
 * search verifies each match).  A match phi is an injective, label-preserving
 * map of the template vertices that sends every template edge onto a graph
 * edge (Definition 1); all matches lie inside the pruned state, so the search
 * runs only there (on omega of the result; the final state is the fastest).
 *   list           n0 int32 per match: phi(0), ..., phi(n0-1); the first
 *                  min(*n_matches, list_cap) matches found, in no set order
 *                  (nullable when list_cap == 0)
 *   vertex_counts  uint64 [n] (nullable): matches that contain the vertex
 *   entry_counts   uint64 [m_dir] (nullable): matches that map a template edge
 *                  onto the edge of that CSR entry (both entries of an edge
 *                  get the same count)
 *   *n_matches     the number of matches (all of them, beyond list_cap too)
 * Outputs are device pointers on the context's device if dst_on_device, else
 * host memory (staged through temporary device buffers).  `opt` (nullable):
 * search_budget bounds the windows one search may scan (0: unbounded),
 * search_split as for ccpm_prune.  Errors: CCPM_EINVAL for a result of another
 * graph, template or device; CCPM_EBUDGET if a search ran out of its budget
 * (the outputs are then incomplete); CCPM_ENOMEM / CCPM_ECUDA. */
/* Exploratory search (Section 6.7, "Exploratory Search"; "Interactive
 * Incremental Search" for the candidate set): the base template is relaxed
 * level by level, level k holding every variant with k template edges
 * removed that stays connected (vertices and labels are kept, so template
 * vertex q means the same in every variant); the search stops after the
 * first level at which some variant has a match.
 * First the candidate set is built with local constraints only: the union of
 * the LCC fixpoints of every variant up to max_removed, which holds every
 * match of every variant.  Each variant is then pruned from the candidate set
 * (as with options.resume) instead of from the label-initial state; its omega*,
 * E* and count equal those of a prune of that variant alone.
 *   variants   per variant examined, in level order (nullable if variants_cap
 *              is 0): its level, the removed edges (bit i = edge i of the base
 *              in input order), |V*|, E* entries, count, status, time
 *   *out       the union of omega* and of E* over the variants with a match at
 *              the first such level (a new result, or one of this graph to
 *              reuse); all zero, and *level_found = -1, if no variant up to
 *              max_removed has a match.  ccpm_result_counts gives its active_v
 *              and active_e_dir only.
 * `opt` (nullable) applies to every variant's prune.  The base template may
 * have at most 64 edges.  Errors as for ccpm_prune; CCPM_EBUDGET if any
 * variant's prune hit a budget (its outputs are then supersets). */
typedef struct {
    int32_t  level;              /* template edges removed                     */
    int32_t  n_edges;            /* edges of the variant                       */
    uint64_t removed;            /* bit i: edge i of the base removed          */
    int64_t  active_v, active_e_dir;
    uint64_t match_embeddings;
    int32_t  count_valid, status;
    double   ms_total;
} ccpm_explore_variant;
int  ccpm_explore(ccpm_ctx_t ctx, ccpm_graph_t g, ccpm_tmpl_t base, int max_removed, const ccpm_options *opt,
                  ccpm_explore_variant *variants, int variants_cap, int *n_variants, int *level_found,
                  double *ms_candidates, ccpm_result_t *out);
int  ccpm_result_matches(ccpm_ctx_t ctx, ccpm_result_t r, ccpm_tmpl_t t, const ccpm_options *opt,
                         int32_t *list, uint64_t list_cap, uint64_t *vertex_counts, uint64_t *entry_counts,
                         int dst_on_device, uint64_t *n_matches);
/* Device pointers owned by the result (valid until it is destroyed). */
/* Log record of the i-th constraint in the order it ran (0 <= i < n_phases-1). */
int  ccpm_result_constraint_log(ccpm_result_t r, int i, ccpm_constraint_log *out);
const uint32_t *ccpm_result_omega_device(ccpm_result_t r);
const uint32_t *ccpm_result_edge_bitmap_device(ccpm_result_t r);
void ccpm_result_destroy(ccpm_result_t r);

/* ------------------------------------------------------ checkpoint/resume */

/* A pruning state (omega, edge bitmap, counts, per-phase rounds) as one
 * self-describing host byte blob: a 96-byte little-endian header (magic
 * "CCPMSTAT", version, n, m_dir, bitmap words, fingerprints of the graph -- n,
 * m_dir and its label histogram -- and of the template -- labels and sorted
 * edges --, sizes and an FNV-1a 64 checksum of the payload), then the counts,
 * the phase rounds (int32), omega (n uint32) and the bitmap (words uint32).
 * Constraint logs are not part of it.
 *
 * ccpm_state_export: with buf == NULL sets *len to the size needed and
 * returns CCPM_OK; otherwise writes the blob to buf (host memory of *len
 * bytes) and sets *len to the bytes written, or returns CCPM_EINVAL with *len
 * set to the size needed when *len is too small.
 *
 * ccpm_state_import: checks the blob against g and t (CCPM_EINVAL on a wrong
 * magic, version, size, fingerprint or checksum) and returns a new result in
 * *out holding that state, owned by the caller like any result.  Pruning
 * removes only candidates that no match uses (Section 4), so any state this
 * library produced for (g, t) contains every match; ccpm_prune with
 * options.resume = 1 continues from it (LCC, the non-local constraints and
 * the final search) and ends in the same omega*, E* and match count as a
 * fresh run; round counts may differ. */
int  ccpm_state_export(ccpm_result_t r, void *buf, size_t *len);
int  ccpm_state_import(ccpm_ctx_t ctx, ccpm_graph_t g, ccpm_tmpl_t t, const void *buf, size_t len,
                       ccpm_result_t *out);

/* ------------------------------------------------------ ordering network */

/* A 3-layer perceptron that scores non-local constraints for
 * CCPM_ORDER_LEARNED (the paper orders constraints by a fixed heuristic,
 * Section 4.2, and leaves learned orders to future work, Section 8).
 * Parameters: FP32 master copy of CCPM_MLP_PARAMS floats laid out as
 * W1[16][64], b1[64], W2[64][64], b2[64], w3[64], b3 (W[i][j]: input i to
 * unit j).  Products run on BF16 tensor cores with FP32 accumulation:
 * X, W1, W2 and the first hidden layer are rounded to BF16 before each product.
 * All host arrays are row-major FP32; calls are synchronous on the stream of
 * the context the network was created on. */
int  ccpm_mlp_create(ccpm_ctx_t ctx, uint64_t seed, ccpm_mlp_t *out);
void ccpm_mlp_destroy(ccpm_mlp_t m);
int  ccpm_mlp_set_params(ccpm_mlp_t m, const float *params);
int  ccpm_mlp_get_params(ccpm_mlp_t m, float *params);
/* y[b] = network(x[b][0..15]) for b < B. */
int  ccpm_mlp_forward(ccpm_mlp_t m, int B, const float *x, float *y);
/* Gradient of 0.5 * mean_b (y[b] - t[b])^2 with respect to every parameter
 * (same layout as the parameters) and the loss itself. */
int  ccpm_mlp_gradient(ccpm_mlp_t m, int B, const float *x, const float *t, float *grad, float *loss);
/* `steps` Adam steps (beta 0.9 / 0.999) on minibatches of `batch` rows drawn
 * with replacement from the N rows of (x, t) by a seeded counter-based hash;
 * *final_loss (nullable) gets the last minibatch's loss. */
int  ccpm_mlp_train(ccpm_mlp_t m, int N, const float *x, const float *t, int steps, int batch, float lr,
                    uint64_t seed, float *final_loss);

/* ------------------------------------ wider templates and edge labels */

/* Edge labels of a loaded graph (Section 3: the background graph carries
 * metadata on its edges as well as on its vertices).  edge_labels[e] is the
 * label of CSR entry e, uint8 [m_dir]; both entries of an undirected edge
 * must carry the same label (checked with CCPM_VALIDATE, host pointers only:
 * CCPM_EINVAL otherwise).  CCPM_HOST_PTRS copies the array to the device;
 * CCPM_DEVICE_PTRS borrows it (it must outlive the graph).  A later call
 * replaces the labels; NULL removes them (every edge label is then 0).  Only
 * ccpm_lcc_wide reads them. */
int  ccpm_graph_set_edge_labels(ccpm_graph_t g, const uint8_t *edge_labels, int flags);

typedef struct {
    int64_t rounds;          /* LCC rounds executed, the final quiescent one included */
    int64_t edges_scanned;   /* active entries read, summed over the rounds           */
    int64_t vertices_scanned;/* active vertices read, summed over the rounds          */
    int64_t active_v;        /* vertices whose omega is not empty at the fixpoint     */
    int64_t active_e_dir;    /* CSR entries whose bit is set at the fixpoint          */
    double  ms;              /* device time of the call (events on the ctx stream)    */
} ccpm_wide_stats;

/* Local constraint checking to its fixpoint for templates of up to 64
 * vertices, with edge labels.  The paper sizes LCC state at eight bytes of
 * omega per vertex for a 64-vertex template (Section 5.1, "Complexity
 * Analysis"), and a match must preserve edge metadata as well as vertex
 * labels (Section 3).
 *   template: n0 (2..64) vertex labels, m0 (1..2016) edges as 2*m0 int32
 *             (endpoints in range, no self loop or duplicate, connected), and
 *             tmpl_edge_labels (nullable: all 0), one label per edge; at most
 *             8 distinct edge labels and 64 label-multiplicity classes
 *   graph:    its edge labels from ccpm_graph_set_edge_labels (all 0 if none)
 * Per edge label L, the rules of Alg. 4 read: an active entry (v,u) labelled L
 * stays active iff some a in omega(v) has a template neighbour b in omega(u)
 * joined to a by an edge labelled L; q stays in omega(v) iff every template
 * neighbour b of q (joined by label L) lies in omega(u) for some entry (v,u)
 * labelled L that stays active, and, for every pair (vertex label, edge
 * label), at least as many distinct such neighbours u reached by that edge
 * label have omega(u) meeting q's template neighbours of that pair as q has
 * such neighbours.  Rounds are snapshot rounds.  With every edge label 0 and
 * n0 <= 32 the result equals the first LCC fixpoint of ccpm_prune.
 * Outputs: omega uint64 [n] (bit q = template vertex q) and the edge bitmap
 * (ceil(m_dir/32) uint32 words, layout as above), device pointers on the
 * context's device if out_on_device, else host memory; stats (nullable).  No
 * non-local constraint and no final search run: the result holds every match
 * (a superset of omega* and E*; exact for acyclic templates with unique
 * vertex labels).  Synchronous on the context's stream.  Errors: CCPM_EINVAL
 * (template, with a message in ccpm_last_error), CCPM_ENOMEM, CCPM_ECUDA. */
int  ccpm_lcc_wide(ccpm_ctx_t ctx, ccpm_graph_t g, int n0, const uint8_t *tmpl_labels, int m0,
                   const int32_t *tmpl_edges, const uint8_t *tmpl_edge_labels, uint64_t *omega,
                   uint32_t *ebits, int out_on_device, ccpm_wide_stats *stats);

/* ------------------------------------------------- allocation-free LCC */

/* Local constraint checking to its fixpoint without allocating anything.
 * The paper has no counterpart to this call; it exists for callers that must
 * not allocate device memory while they run (a memory budget fixed up front,
 * an allocator owned by someone else, or host code that may not block inside
 * cudaMalloc).
 *
 * Inputs are device pointers on `device`: the CSR graph (row_ptr int64 [n+1],
 * col int32 [m_dir], labels uint8 [n], same rules as ccpm_graph_load_csr) and
 * the template as host arrays (n0 labels, m0 edges as 2*m0 int32).  Outputs:
 * omega (device, n uint32) and ebits (device, ceil(m_dir/32) uint32 words),
 * both in the layouts described at the top of this file; *rounds (host,
 * nullable) gets the LCC rounds executed including the final quiescent one,
 * *edges_scanned (host, nullable) the active entries read over all rounds.
 * The result equals the LCC fixpoint ccpm_prune reaches before any
 * non-local constraint.  Work runs on `cuda_stream` (NULL: the legacy default
 * stream) and the call returns when it is done.
 *
 * Scratch lives in a fixed 16 MiB area compiled into the library, enough for
 * roughly n <= 500,000 vertices and m_dir <= 16,000,000 entries; larger graphs
 * are rejected with CCPM_EINVAL and a message in errbuf (nullable, errlen
 * bytes, written by every call).  The first call on a device looks up the
 * area's device address (make that first call before any stream capture).
 * All calls share the one area: calls whose GPU work overlaps in time, on any
 * streams, corrupt each other's results, so serialise them.  The call reads
 * row_ptr[0] and row_ptr[n] first and returns CCPM_EINVAL unless they are 0
 * and m_dir.  It makes `device` current while it runs and makes the caller's
 * current device current again before it returns. */
int  ccpm_lcc_fixpoint_noalloc(int device, void *cuda_stream, int64_t n, int64_t m_dir,
                               const int64_t *row_ptr, const int32_t *col, const uint8_t *labels,
                               int n0, const uint8_t *tmpl_labels, int m0, const int32_t *tmpl_edges,
                               uint32_t *omega, uint32_t *ebits, int32_t *rounds,
                               int64_t *edges_scanned, char *errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif
#endif /* CCPM_H */
