// ccpm_internal.h -- structures shared by the host engine and the CUDA kernels.
// Not part of the public ABI (see include/ccpm.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ccpm.h"

namespace ccpm {

constexpr int kMaxT = 32;           // template vertices (omega is one uint32)
constexpr int kMaxCls = 32;         // label-multiplicity classes per template
constexpr int kSmallDeg = 64;       // rows up to this length: the flat short-row path
constexpr int kDefaultHubDeg = 1024;// longer rows are split into chunks of this size
constexpr int kMaxHubDeg = 1 << 24; // larger hub_degree options are clamped to this
constexpr int64_t kEntryLabelRows = (int64_t)1 << 22;   // first-round rows that pay for the entry labels
constexpr uint64_t kDefaultSearchBudget = 1ull << 22;

// Template tables for the LCC kernels.  A "class" is (q, L) with
// |adj_L(q)| >= 2: vertex q of the template needs at least `need` distinct
// active neighbours whose omega meets `mask` = adj_L(q) (Section 4.1 / Section 4.3).
struct DevTmpl {
    int n0;
    int n_cls;
    uint32_t adj[kMaxT];
    uint32_t cls_mask[kMaxCls];
    uint32_t cls_need[kMaxCls];
    uint32_t cls_q[kMaxCls];
};

// Search plan of a rooted injective embedding of a substructure S: positions
// 0..k-1, position 0 is the root.  Position i > 0 is found among the active
// neighbours of position par[i]; back[i] lists earlier positions that must be
// joined to it by an active edge; same[i] lists earlier positions whose
// template vertex has the same label (injectivity only needs those).
struct DevPlan {
    int k;
    int8_t q[kMaxT];
    int8_t par[kMaxT];
    uint8_t lab[kMaxT];       // label of the template vertex at each position
    uint32_t nbr[kMaxT];      // earlier positions joined to position i in S
    uint32_t back[kMaxT];
    uint32_t same[kMaxT];
    // full-template enumeration marks these (position, position) edges
    int n_marks;
    int8_t mark_a[CCPM_MAX_TMPL_EDGES];
    int8_t mark_b[CCPM_MAX_TMPL_EDGES];
};

struct HostConstraint {
    int kind;
    uint32_t vmask;
    uint32_t hmask;
    std::vector<std::pair<int, int>> edges;   // a < b, sorted
    int gen_index;
};

struct Template {
    int n0 = 0;
    uint8_t labels[kMaxT] = {};
    std::vector<std::pair<int, int>> edges;   // a < b, input order
    uint32_t adj[kMaxT] = {};
    std::vector<HostConstraint> k0;           // generated, fixed heuristic order
    std::vector<int> order;                   // explicit order (indices into k0)
    bool generated = false;
    uint64_t automorphisms = 0;
    std::string err;
};

// glue between translation units (ccpm_kernels.cu, ccpm_mlp.cu, ccpm_wide.cu)
int ctx_device(ccpm_ctx *ctx);
void *ctx_stream_ptr(ccpm_ctx *ctx);
int ctx_num_sms(ccpm_ctx *ctx);
int ctx_set_err(ccpm_ctx *ctx, int code, const char *msg);
// device arrays of a loaded graph (el: edge labels, NULL if none were set)
struct GraphView {
    int64_t n, m;
    const int64_t *rp;
    const int32_t *col;
    const uint8_t *lab;
    const uint8_t *el;
    ccpm_ctx *ctx;
};
GraphView graph_view(ccpm_graph *g);
// Scoring scratch of one caller (a context, or the network's own public
// forward call): device inputs and outputs plus pinned host staging, grown on
// demand.  Each batch worker scores with its own, so concurrent workers share
// only the network's parameters, which scoring only reads.
struct MlpScratch {
    float *dx = nullptr, *dy = nullptr;   // device [cap * CCPM_MLP_IN], [cap]
    float *hx = nullptr, *hy = nullptr;   // pinned host staging of the same sizes
    int cap = 0;
};
void mlp_scratch_free(MlpScratch &sc);
// wait_ev (a cudaEvent_t, nullable): wait by polling it and yielding the
// core (batch workers), instead of the runtime's spinning stream wait.
int mlp_score(ccpm_mlp *m, int B, const float *host_x, float *host_y, void *stream, MlpScratch &sc,
              void *wait_ev = nullptr);

// host helpers (ccpm_host.cpp)
int  template_build(Template &t, int n0, const uint8_t *labels, int m0, const int32_t *edges);
int  constraints_generate(Template &t, std::string &err);
uint64_t count_automorphisms(const Template &t);
void build_dev_tmpl(const Template &t, DevTmpl &d);
// order[] of S's vertices from `root`: greedy, most back edges first, then
// fewest live candidates (qlive[q]: vertices whose omega holds q, when given;
// otherwise the background frequency of q's label), then lowest id.
// second >= 0 fixes position 1 (a template neighbour of root): plans rooted at
// a template edge.
void build_plan(const Template &t, uint32_t svert, const uint32_t *sadj, int root,
                const int64_t *label_freq, bool with_marks, DevPlan &p, int second = -1,
                const unsigned long long *qlive = nullptr);

}  // namespace ccpm
