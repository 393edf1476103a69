// ccpm_wide.cu -- local constraint checking (Alg. 3 and Alg. 4) for templates
// of up to 64 vertices, with omega in 64-bit words (the paper's LCC state
// estimate budgets eight bytes per vertex for 64 template vertices, Section
// 5.1), and with edge labels (Section 3: edges carry metadata too).
//
// The rules of Alg. 4 are read per edge label L: an entry (v,u) labelled L
// stays active iff some a in omega(v) has a template neighbour b in omega(u)
// joined to a by an edge labelled L (eta); q stays in omega(v) iff every
// template neighbour b of q, joined by label L, lies in omega(u) of a kept
// entry labelled L (the union omega' taken per edge label), and for each
// pair (vertex label, edge label) enough distinct kept neighbours reached by
// that label meet q's template neighbours of the pair (the multiplicity rule
// of Section 4.1).  With every edge label 0 these are the rules of the 32-bit
// pipeline.
//
// Layout and schedule: one warp per listed vertex (one block per vertex whose
// row is longer than 1024 entries); its entries are read in windows aligned
// to the 32-entry words of the edge bitmap, so lane i of a window owns bit i
// of one word (one broadcast load of the bits, one atomic to clear the
// failing ones).  Rounds are snapshot rounds over two omega
// buffers; each round lists the vertices that were active at its start for
// the next round, which writes 0 for those that died and drops them.  The
// host reads one small counter block per round.  No kernel waits on another
// block: every loop is bounded by the list or row it walks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "ccpm.h"
#include "ccpm_internal.h"

namespace ccpm {
namespace {

constexpr int kWT = 64;        // template vertices
constexpr int kWEL = 8;        // distinct edge labels one template may use
constexpr int kWCls = 64;      // label-multiplicity classes (need >= 2)
constexpr int kWEdges = 2016;  // 64 * 63 / 2
constexpr int kWHub = 1024;    // rows longer than this are walked by a whole block
constexpr unsigned FULL = 0xFFFFFFFFu;

// Template tables of one call (device copy, loaded into shared memory).
struct __align__(16) WideTab {
    int n0, n_el, n_cls, pad;
    uint8_t el_index[256];         // graph edge label -> edge-label index j, 0xFF: used by no template edge
    uint64_t adj[kWEL][kWT];       // adj[j][q]: template neighbours of q joined by an edge of label index j
    uint64_t cls_mask[kWCls];      // template neighbours of cls_q with one vertex label, joined by label cls_j
    uint32_t cls_need[kWCls];      // their number (at least 2; a class of one is the coverage rule)
    uint8_t cls_q[kWCls];
    uint8_t cls_j[kWCls];
};

struct WideCounters {
    unsigned long long n_next;     // vertices listed for the next round (rows up to kWHub entries)
    unsigned long long n_hub_next; // ... with longer rows
    unsigned long long scanned;    // active entries read (both ends live, bit set)
    unsigned long long alive;      // active vertices read
    unsigned long long active_v, active_e;   // hand-back totals
    unsigned int changed;
    unsigned int pad;
};

struct WideArgs {
    const int64_t *rp;
    const int32_t *col;
    const uint8_t *el;             // edge label per entry, or NULL (all 0)
    const uint64_t *om_in;
    uint64_t *om_out;
    uint32_t *ebits;
    const int32_t *list_in;
    int64_t n_in;
    int32_t *list_out;
    const int32_t *hub_in;         // vertices whose rows are longer than kWHub entries
    int64_t n_hub;
    int32_t *hub_out;
    WideCounters *st;
    const WideTab *tab;
};

__device__ __forceinline__ uint64_t warp_or64(uint64_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(FULL, x, o);
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

__device__ __forceinline__ void load_tab(WideTab &dst, const WideTab *src) {
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(WideTab) / 4); i += blockDim.x) d[i] = s[i];
}

// Warp-aggregated append of v (lanes with `take`) to list[*count ...].
__device__ __forceinline__ void push_list(bool take, int32_t v, int32_t *list, unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    const uint32_t act = __ballot_sync(FULL, take);
    if (!act) return;
    unsigned long long base = 0;
    const int leader = __ffs(act) - 1;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(act));
    base = __shfl_sync(FULL, base, leader);
    if (take) list[base + __popc(act & ((1u << lane) - 1u))] = v;
}

// Alg. 3: omega_0(v) = {q : l(q) = l(v)} in both snapshot buffers; every
// initially active vertex is listed for the first round, on the list of its
// row length.
__global__ void __launch_bounds__(256)
k_wide_init(int64_t n, const int64_t *__restrict__ rp, const uint8_t *__restrict__ lab,
            const uint64_t *__restrict__ lmask, uint64_t *om0, uint64_t *om1, int32_t *list, int32_t *hub,
            WideCounters *st) {
    __shared__ uint64_t sl[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sl[i] = lmask[i];
    __syncthreads();
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = v0 + threadIdx.x;
        uint64_t w = 0;
        bool long_row = false;
        if (v < n) {
            w = sl[lab[v]];
            om0[v] = w;
            om1[v] = w;
            if (w) long_row = rp[v + 1] - rp[v] > kWHub;
        }
        push_list(w != 0 && !long_row, (int32_t)v, list, &st->n_next);
        push_list(w != 0 && long_row, (int32_t)v, hub, &st->n_hub_next);
    }
}

// The template neighbours of omega(v) per edge-label index (every lane of
// the warp gets them).
__device__ __forceinline__ void nbr_masks(const WideTab &T, uint64_t wv, uint64_t (&nb)[kWEL]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < kWEL; j++) nb[j] = 0;
    for (int q = lane; q < T.n0; q += 32)
        if ((wv >> q) & 1ull) {
#pragma unroll
            for (int j = 0; j < kWEL; j++)
                if (j < T.n_el) nb[j] |= T.adj[j][q];
        }
#pragma unroll
    for (int j = 0; j < kWEL; j++) nb[j] = warp_or64(nb[j]);
}

// One warp's share of a row: windows first_w, first_w + w_step, ... (each a
// group of four 32-entry windows aligned to the bitmap words, all loaded
// before any is used).  Per lane: the unions per edge-label index, the
// surviving entries, the eta change; per class, the count of surviving
// entries meeting it is added to cnt[c] by lane 0 (atomically when several
// warps share cnt).
__device__ __forceinline__ void scan_windows(const WideArgs &a, const WideTab &T, uint64_t wv,
                                             const uint64_t (&nb)[kWEL], int64_t beg, int64_t end,
                                             int64_t first_w, int64_t w_step, uint64_t (&U)[kWEL],
                                             uint32_t &nN, uint32_t &achg, uint32_t *cnt, bool shared_cnt,
                                             unsigned long long &scanned) {
    constexpr int WU = 4;
    const int lane = threadIdx.x & 31;
    const int n_cls = T.n_cls;
    for (int64_t w0 = first_w; (w0 << 5) < end; w0 += w_step) {
        bool bit[WU];
        int32_t u[WU];
        uint8_t lb[WU];
        uint64_t wn[WU];
#pragma unroll
        for (int k = 0; k < WU; k++) {
            const int64_t e = ((w0 + k) << 5) + lane;
            const uint32_t word = ((w0 + k) << 5) < end ? a.ebits[w0 + k] : 0u;
            bit[k] = e >= beg && e < end && ((word >> lane) & 1u);
        }
#pragma unroll
        for (int k = 0; k < WU; k++) {
            const int64_t e = ((w0 + k) << 5) + lane;
            u[k] = bit[k] ? a.col[e] : 0;
            lb[k] = (bit[k] && a.el) ? a.el[e] : (uint8_t)0;
        }
#pragma unroll
        for (int k = 0; k < WU; k++) wn[k] = bit[k] ? a.om_in[u[k]] : 0ull;
#pragma unroll
        for (int k = 0; k < WU; k++) {
            if (((w0 + k) << 5) >= end) break;          // past the row (warp-uniform)
            const uint64_t wu = wn[k];
            const int j = bit[k] ? (int)T.el_index[lb[k]] : 0xFF;
            uint64_t m = 0;
#pragma unroll
            for (int jj = 0; jj < kWEL; jj++)
                if (j == jj) m = nb[jj];
            const bool live = bit[k] && wu != 0;     // both ends active: the entry is active
            const bool pass = live && (wu & m) != 0;
            scanned += live ? 1ull : 0ull;
            if (live && !pass) achg = 1;             // eta eliminates an active entry
            if (pass) {
                nN++;
#pragma unroll
                for (int jj = 0; jj < kWEL; jj++)
                    if (j == jj) U[jj] |= wu;
            }
            // the bit goes with the failing entries and with those whose
            // other end is inactive already (no change: that entry is inactive)
            const uint32_t drop = __ballot_sync(FULL, bit[k] && !pass);
            if (drop && lane == 0) atomicAnd(&a.ebits[w0 + k], ~drop);
            for (int c = 0; c < n_cls; c++) {
                if (!((wv >> T.cls_q[c]) & 1ull)) continue;
                const uint32_t hit = __ballot_sync(FULL, pass && j == (int)T.cls_j[c] && (wu & T.cls_mask[c]) != 0);
                if (lane == 0 && hit) {
                    if (shared_cnt) atomicAdd(&cnt[c], (uint32_t)__popc(hit));
                    else cnt[c] += (uint32_t)__popc(hit);
                }
            }
        }
    }
}

// The vertex rule: q stays iff every template neighbour joined by edge
// label j lies in U[j] and every class of q has enough distinct neighbours;
// nothing stays without a surviving entry.
__device__ __forceinline__ uint64_t decide_wide(const WideTab &T, uint64_t wv, const uint64_t (&U)[kWEL], uint32_t nN,
                                                const uint32_t *cnt) {
    uint64_t keep = 0;
    if (nN == 0) return 0;
    for (int q = 0; q < T.n0; q++) {
        if (!((wv >> q) & 1ull)) continue;
        bool ok = true;
#pragma unroll
        for (int j = 0; j < kWEL; j++)
            if (j < T.n_el && (T.adj[j][q] & ~U[j])) ok = false;
        for (int c = 0; c < T.n_cls && ok; c++)
            if (T.cls_q[c] == q && cnt[c] < T.cls_need[c]) ok = false;
        if (ok) keep |= 1ull << q;
    }
    return keep;
}

// One snapshot round.  Rows of at most kWHub entries: one warp each.  Longer
// rows (list hub_in): one block each, its warps taking interleaved window
// groups, the partial results combined in shared memory.  Every vertex
// listed at the start of the round is listed again (the next round writes
// its zero if it died here); a vertex stays on the list of its row length.
__global__ void __launch_bounds__(256)
k_wide_round(WideArgs a) {
    __shared__ WideTab T;
    __shared__ uint32_t cnt[8][kWCls];
    __shared__ uint32_t bcnt[kWCls];
    __shared__ unsigned long long bU[kWEL];
    __shared__ uint32_t bN, bchg;
    load_tab(T, a.tab);
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nwb = (int)(blockDim.x >> 5);
    unsigned long long scanned = 0, alive = 0;
    unsigned int changed = 0;
    // (1) rows up to kWHub entries, one warp each
    for (int64_t i = gw; i < a.n_in; i += nw) {
        const int32_t v = a.list_in[i];
        const uint64_t wv = a.om_in[v];
        if (wv == 0) {
            // died in the previous round: its zero goes to this buffer too
            if (lane == 0) a.om_out[v] = 0;
            continue;
        }
        if (lane == 0) alive++;
        uint64_t nb[kWEL];
        nbr_masks(T, wv, nb);
        for (int c = lane; c < T.n_cls; c += 32) cnt[wib][c] = 0;
        __syncwarp();
        const int64_t beg = a.rp[v], end = a.rp[(int64_t)v + 1];
        uint64_t U[kWEL];
#pragma unroll
        for (int j = 0; j < kWEL; j++) U[j] = 0;
        uint32_t nN = 0, achg = 0;
        scan_windows(a, T, wv, nb, beg, end, beg >> 5, 4, U, nN, achg, cnt[wib], false, scanned);
#pragma unroll
        for (int j = 0; j < kWEL; j++) U[j] = warp_or64(U[j]);
        nN = __reduce_add_sync(FULL, nN);
        achg = __reduce_or_sync(FULL, achg);
        __syncwarp();
        const uint64_t keep = decide_wide(T, wv, U, nN, cnt[wib]);
        if (keep != wv || achg) changed = 1;
        if (lane == 0) {
            a.om_out[v] = keep;
            const unsigned long long pos = atomicAdd(&a.st->n_next, 1ull);
            a.list_out[pos] = v;
        }
        __syncwarp();
    }
    // (2) longer rows, one block each (block-uniform loop)
    for (int64_t i = blockIdx.x; i < a.n_hub; i += gridDim.x) {
        const int32_t v = a.hub_in[i];
        const uint64_t wv = a.om_in[v];
        if (wv == 0) {
            if (threadIdx.x == 0) a.om_out[v] = 0;
            continue;
        }
        if (threadIdx.x == 0) alive++;
        uint64_t nb[kWEL];
        nbr_masks(T, wv, nb);
        for (int c = threadIdx.x; c < T.n_cls; c += blockDim.x) bcnt[c] = 0;
        if (threadIdx.x < kWEL) bU[threadIdx.x] = 0ull;
        if (threadIdx.x == 0) { bN = 0; bchg = 0; }
        __syncthreads();
        const int64_t beg = a.rp[v], end = a.rp[(int64_t)v + 1];
        uint64_t U[kWEL];
#pragma unroll
        for (int j = 0; j < kWEL; j++) U[j] = 0;
        uint32_t nN = 0, achg = 0;
        scan_windows(a, T, wv, nb, beg, end, (beg >> 5) + 4 * wib, 4 * nwb, U, nN, achg, bcnt, true, scanned);
#pragma unroll
        for (int j = 0; j < kWEL; j++) U[j] = warp_or64(U[j]);
        nN = __reduce_add_sync(FULL, nN);
        achg = __reduce_or_sync(FULL, achg);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < kWEL; j++)
                if (U[j]) atomicOr(&bU[j], (unsigned long long)U[j]);
            if (nN) atomicAdd(&bN, nN);
            if (achg) atomicOr(&bchg, 1u);
        }
        __syncthreads();
        if (wib == 0) {
            uint64_t Ub[kWEL];
#pragma unroll
            for (int j = 0; j < kWEL; j++) Ub[j] = bU[j];
            const uint64_t keep = decide_wide(T, wv, Ub, bN, bcnt);
            if (keep != wv || bchg) changed = 1;
            if (lane == 0) {
                a.om_out[v] = keep;
                const unsigned long long pos = atomicAdd(&a.st->n_hub_next, 1ull);
                a.hub_out[pos] = v;
            }
        }
        __syncthreads();                          // bcnt / bU / bN are reused
    }
    scanned = warp_sum64(scanned);
    alive = warp_sum64(alive);
    changed = __reduce_or_sync(FULL, changed);
    if (lane == 0) {
        if (scanned) atomicAdd(&a.st->scanned, scanned);
        if (alive) atomicAdd(&a.st->alive, alive);
        if (changed) atomicOr(&a.st->changed, 1u);
    }
}

// Hand-back: an entry keeps its bit only if both of its ends are active
// (rows of dead vertices and entries to dead neighbours are cleared; so are
// the rows of vertices that were never active).  Counts the active vertices
// and entries.
__global__ void __launch_bounds__(256)
k_wide_clear(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
             const uint64_t *__restrict__ om, uint32_t *ebits, WideCounters *st) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long av = 0, ae = 0;
    for (int64_t v = gw; v < n; v += nw) {
        const bool vlive = om[v] != 0;
        if (lane == 0 && vlive) av++;
        const int64_t beg = rp[v], end = rp[v + 1];
        for (int64_t w0 = beg >> 5; (w0 << 5) < end; w0++) {
            const int64_t e = (w0 << 5) + lane;
            const uint32_t word = ebits[w0];
            const bool bit = e >= beg && e < end && ((word >> lane) & 1u);
            const bool keep = bit && vlive && om[col[e]] != 0;
            ae += keep ? 1ull : 0ull;
            const uint32_t drop = __ballot_sync(FULL, bit && !keep);
            if (drop && lane == 0) atomicAnd(&ebits[w0], ~drop);
        }
    }
    av = warp_sum64(av);
    ae = warp_sum64(ae);
    if (lane == 0) {
        if (av) atomicAdd(&st->active_v, av);
        if (ae) atomicAdd(&st->active_e, ae);
    }
}

// Every entry's bit set; the bits past the last entry stay 0.
__global__ void k_wide_fill(int64_t words, int64_t m, uint32_t *ebits) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t left = m - (w << 5);
        ebits[w] = left >= 32 ? FULL : ((1u << (uint32_t)left) - 1u);
    }
}

int grid_of(ccpm_ctx *ctx, int64_t items, int per_block, int per_sm) {
    const int64_t need = std::max<int64_t>(1, (items + per_block - 1) / per_block);
    return (int)std::min<int64_t>(need, (int64_t)ctx_num_sms(ctx) * per_sm);
}

int popc64(uint64_t x) { return __builtin_popcountll(x); }

// Checks the template and fills the tables; returns CCPM_OK or CCPM_EINVAL
// with a message.
int build_tab(int n0, const uint8_t *labels, int m0, const int32_t *edges, const uint8_t *elab, WideTab &t,
              uint64_t *lmask, std::string &err) {
    if (n0 < 2 || n0 > kWT) { err = "wide template must have 2..64 vertices"; return CCPM_EINVAL; }
    if (m0 < 1 || m0 > kWEdges || !labels || !edges) {
        err = "wide template needs 1..2016 edges and non-NULL arrays";
        return CCPM_EINVAL;
    }
    std::memset(&t, 0, sizeof(t));
    std::memset(t.el_index, 0xFF, sizeof(t.el_index));
    t.n0 = n0;
    uint64_t any[kWT] = {};
    for (int i = 0; i < m0; i++) {
        const int a = edges[2 * i], b = edges[2 * i + 1];
        if (a < 0 || b < 0 || a >= n0 || b >= n0) { err = "template edge endpoint out of range"; return CCPM_EINVAL; }
        if (a == b) { err = "template self loop"; return CCPM_EINVAL; }
        if ((any[a] >> b) & 1ull) { err = "duplicate template edge"; return CCPM_EINVAL; }
        any[a] |= 1ull << b;
        any[b] |= 1ull << a;
        const uint8_t L = elab ? elab[i] : 0;
        if (t.el_index[L] == 0xFF) {
            if (t.n_el == kWEL) { err = "template uses more than 8 edge labels"; return CCPM_EINVAL; }
            t.el_index[L] = (uint8_t)t.n_el++;
        }
        const int j = t.el_index[L];
        t.adj[j][a] |= 1ull << b;
        t.adj[j][b] |= 1ull << a;
    }
    // connected
    uint64_t seen = 1, frontier = 1;
    while (frontier) {
        uint64_t next = 0;
        for (int q = 0; q < n0; q++)
            if ((frontier >> q) & 1ull) next |= any[q];
        frontier = next & ~seen;
        seen |= next;
    }
    const uint64_t all = n0 == 64 ? ~0ull : ((1ull << n0) - 1ull);
    if ((seen & all) != all) { err = "template is not connected"; return CCPM_EINVAL; }
    // multiplicity classes: q's neighbours of one vertex label joined by one edge label
    for (int q = 0; q < n0; q++)
        for (int j = 0; j < t.n_el; j++) {
            uint64_t done = 0;
            for (int b = 0; b < n0; b++) {
                if (!((t.adj[j][q] >> b) & 1ull) || ((done >> b) & 1ull)) continue;
                uint64_t grp = 0;
                for (int c = 0; c < n0; c++)
                    if (((t.adj[j][q] >> c) & 1ull) && labels[c] == labels[b]) grp |= 1ull << c;
                done |= grp;
                if (popc64(grp) < 2) continue;
                if (t.n_cls == kWCls) { err = "template has more than 64 label-multiplicity classes"; return CCPM_EINVAL; }
                t.cls_mask[t.n_cls] = grp;
                t.cls_need[t.n_cls] = (uint32_t)popc64(grp);
                t.cls_q[t.n_cls] = (uint8_t)q;
                t.cls_j[t.n_cls] = (uint8_t)j;
                t.n_cls++;
            }
        }
    std::memset(lmask, 0, sizeof(uint64_t) * 256);
    for (int q = 0; q < n0; q++) lmask[labels[q]] |= 1ull << q;
    return CCPM_OK;
}

// Device buffers of one call, freed on every return path.
struct WideBufs {
    WideTab *tab = nullptr;
    uint64_t *lmask = nullptr;
    uint64_t *om[2] = {nullptr, nullptr};
    int32_t *list[2] = {nullptr, nullptr};
    int32_t *hub[2] = {nullptr, nullptr};
    uint32_t *bits = nullptr;
    WideCounters *st = nullptr;
    WideCounters *st_h = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~WideBufs() {
        cudaFree(tab); cudaFree(lmask); cudaFree(om[0]); cudaFree(om[1]);
        cudaFree(list[0]); cudaFree(list[1]); cudaFree(hub[0]); cudaFree(hub[1]); cudaFree(bits); cudaFree(st);
        if (st_h) cudaFreeHost(st_h);
        for (auto e : ev) if (e) cudaEventDestroy(e);
    }
};

}  // namespace
}  // namespace ccpm

using namespace ccpm;

extern "C" int ccpm_lcc_wide(ccpm_ctx_t ctx, ccpm_graph_t g, int n0, const uint8_t *tmpl_labels, int m0,
                             const int32_t *tmpl_edges, const uint8_t *tmpl_edge_labels, uint64_t *omega,
                             uint32_t *ebits, int out_on_device, ccpm_wide_stats *stats) {
    if (!ctx || !g || !omega || !ebits) return CCPM_EINVAL;
    const GraphView G = graph_view(g);
    if (G.ctx != ctx) return ctx_set_err(ctx, CCPM_EINVAL, "lcc_wide: graph of another context");
    WideTab tab;
    uint64_t lmask[256];
    std::string err;
    int rc = build_tab(n0, tmpl_labels, m0, tmpl_edges, tmpl_edge_labels, tab, lmask, err);
    if (rc) return ctx_set_err(ctx, rc, err.c_str());
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) return ctx_set_err(ctx, CCPM_ECUDA, "lcc_wide: device");
    cudaStream_t s = (cudaStream_t)ctx_stream_ptr(ctx);
    const int64_t n = G.n, m = G.m, words = (m + 31) / 32;
    WideBufs B;
    auto fail = [&](cudaError_t e, const char *what) {
        return ctx_set_err(ctx, e == cudaErrorMemoryAllocation ? CCPM_ENOMEM : CCPM_ECUDA,
                           (std::string("lcc_wide: ") + what + ": " + cudaGetErrorString(e)).c_str());
    };
#define WCU(call, what)                          \
    do {                                         \
        cudaError_t e_ = (call);                 \
        if (e_ != cudaSuccess) return fail(e_, what); \
    } while (0)
    WCU(cudaMalloc(&B.tab, sizeof(WideTab)), "alloc");
    WCU(cudaMalloc(&B.lmask, sizeof(lmask)), "alloc");
    for (int i = 0; i < 2; i++) {
        WCU(cudaMalloc(&B.om[i], sizeof(uint64_t) * (size_t)std::max<int64_t>(n, 1)), "alloc");
        WCU(cudaMalloc(&B.list[i], sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)), "alloc");
        WCU(cudaMalloc(&B.hub[i], sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)), "alloc");
    }
    WCU(cudaMalloc(&B.bits, sizeof(uint32_t) * (size_t)std::max<int64_t>(words, 1)), "alloc");
    WCU(cudaMalloc(&B.st, sizeof(WideCounters)), "alloc");
    WCU(cudaMallocHost(&B.st_h, sizeof(WideCounters)), "alloc");
    WCU(cudaEventCreate(&B.ev[0]), "event");
    WCU(cudaEventCreate(&B.ev[1]), "event");
    WCU(cudaMemcpyAsync(B.tab, &tab, sizeof(WideTab), cudaMemcpyHostToDevice, s), "copy");
    WCU(cudaMemcpyAsync(B.lmask, lmask, sizeof(lmask), cudaMemcpyHostToDevice, s), "copy");
    WCU(cudaEventRecord(B.ev[0], s), "event");
    WCU(cudaMemsetAsync(B.st, 0, sizeof(WideCounters), s), "memset");
    if (words > 0) {
        k_wide_fill<<<grid_of(ctx, words, 256, 8), 256, 0, s>>>(words, m, B.bits);
        WCU(cudaGetLastError(), "launch");
    }
    k_wide_init<<<grid_of(ctx, n, 256, 8), 256, 0, s>>>(n, G.rp, G.lab, B.lmask, B.om[0], B.om[1], B.list[0],
                                                         B.hub[0], B.st);
    WCU(cudaGetLastError(), "launch");
    WCU(cudaMemcpyAsync(B.st_h, B.st, sizeof(WideCounters), cudaMemcpyDeviceToHost, s), "copy");
    WCU(cudaStreamSynchronize(s), "sync");
    int64_t n_in = (int64_t)B.st_h->n_next, n_hub = (int64_t)B.st_h->n_hub_next;
    int64_t rounds = 0, scanned = 0, alive = 0;
    int cur = 0, li = 0;
    for (;;) {
        WCU(cudaMemsetAsync(B.st, 0, sizeof(WideCounters), s), "memset");
        WideArgs a;
        a.rp = G.rp;
        a.col = G.col;
        a.el = G.el;
        a.om_in = B.om[cur];
        a.om_out = B.om[cur ^ 1];
        a.ebits = B.bits;
        a.list_in = B.list[li];
        a.n_in = n_in;
        a.list_out = B.list[li ^ 1];
        a.hub_in = B.hub[li];
        a.n_hub = n_hub;
        a.hub_out = B.hub[li ^ 1];
        a.st = B.st;
        a.tab = B.tab;
        const int grid = std::max(grid_of(ctx, n_in * 32, 256, 8), grid_of(ctx, n_hub * 256, 256, 8));
        k_wide_round<<<grid, 256, 0, s>>>(a);
        WCU(cudaGetLastError(), "launch");
        WCU(cudaMemcpyAsync(B.st_h, B.st, sizeof(WideCounters), cudaMemcpyDeviceToHost, s), "copy");
        WCU(cudaStreamSynchronize(s), "sync");
        rounds++;
        scanned += (int64_t)B.st_h->scanned;
        alive += (int64_t)B.st_h->alive;
        cur ^= 1;                  // omega of the round just run
        li ^= 1;
        n_in = (int64_t)B.st_h->n_next;
        n_hub = (int64_t)B.st_h->n_hub_next;
        if (!B.st_h->changed) break;
    }
    WCU(cudaMemsetAsync(B.st, 0, sizeof(WideCounters), s), "memset");
    k_wide_clear<<<grid_of(ctx, n * 32, 256, 8), 256, 0, s>>>(n, G.rp, G.col, B.om[cur], B.bits, B.st);
    WCU(cudaGetLastError(), "launch");
    WCU(cudaEventRecord(B.ev[1], s), "event");
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (n > 0) WCU(cudaMemcpyAsync(omega, B.om[cur], sizeof(uint64_t) * (size_t)n, kind, s), "copy");
    if (words > 0) WCU(cudaMemcpyAsync(ebits, B.bits, sizeof(uint32_t) * (size_t)words, kind, s), "copy");
    WCU(cudaMemcpyAsync(B.st_h, B.st, sizeof(WideCounters), cudaMemcpyDeviceToHost, s), "copy");
    WCU(cudaStreamSynchronize(s), "sync");
#undef WCU
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, B.ev[0], B.ev[1]);
        stats->rounds = rounds;
        stats->edges_scanned = scanned;
        stats->vertices_scanned = alive;
        stats->active_v = (int64_t)B.st_h->active_v;
        stats->active_e_dir = (int64_t)B.st_h->active_e;
        stats->ms = ms;
    }
    return CCPM_OK;
}
