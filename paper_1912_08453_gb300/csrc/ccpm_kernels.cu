// ccpm_kernels.cu -- sm_103a kernels of the constraint-checking pipeline and
// the C ABI that drives them.
//
// Device state of one prune (the paper's vertex state, Alg. 3):
//   omega[2][n]  uint32  omega(v) for rounds k and k+1 (snapshot/Jacobi LCC)
//   ebits[W]     uint32  1 bit per CSR entry: the active edge map epsilon(v)
// A vertex is active exactly when omega(v) != 0.
//
// Edge bits are kept exact for rows of active vertices only.  A bit in the row
// of an active v that points to a vertex u eliminated in the previous round is
// cleared lazily: the next round sees omega(u) = 0, treats the entry as
// inactive and clears the bit.  Rows of eliminated vertices are zeroed when
// they die; rows of vertices that never become active are zeroed only when
// the edge bitmap is handed back without the final search.  Once the rows are
// compacted (K4) the rounds read the compacted rows and their own bitmap; the
// full bitmap is then frozen and handed back in its fixpoint form (bit, both
// ends live, compatible omegas).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>


#include <atomic>
#include <climits>
#include <cmath>
#include <chrono>
#include <mutex>
#include <thread>

#include "ccpm_internal.h"

namespace ccpm {

#define FULL_MASK 0xFFFFFFFFu

// -------------------------------------------------------------------------
// device-side bookkeeping
// -------------------------------------------------------------------------

struct RoundStats {
    unsigned long long scanned;   // active CSR entries read this round
    unsigned long long windows;   // CSR entries examined by searches
    unsigned long long matches;   // final search: matches found
    unsigned long long tokens;    // NLCC: (vertex, head) searches issued
    unsigned long long row_entries;   // CSR entries in rows of active vertices
    unsigned long long alive;         // active vertices processed
    unsigned long long kept;          // entries still active after the round (rows of survivors)
    unsigned long long rows_next;     // CSR entries in the rows of the survivors
    unsigned int changed;         // any omega or edge changed
    unsigned int n_small, n_med, n_chunk;   // next frontier sizes
    unsigned int n_hub_slots;
    unsigned int n_roots;
    unsigned int n_items;         // (root, head, first candidate) search items
    unsigned int overflow;        // a search hit its budget
    unsigned int n_spill;         // items handed on by searches that ran long (reserved)
    unsigned int spill_stop;      // the spill list is valid below this index (see spill)
    unsigned int skipped;         // LCC round queued after the fixpoint: did nothing
};

struct HubAcc {                   // partial LCC state of one split row
    uint32_t U, nN, flags, done;
    uint32_t cnt[kMaxCls];
    uint32_t pbase;               // index of the row's first piece when the pieces were made
};

struct ChunkItem {                // one piece of a long row
    int32_t v, c, slot, nchunks;
};

struct SmemTmpl {
    uint32_t adj[kMaxT];
    uint32_t cls_mask[kMaxCls];
    uint32_t cls_need[kMaxCls];
    uint32_t cls_q[kMaxCls];
    int n_cls;
};

// Per warp: the rows of one batch of the short-row path.
struct ShortRows {
    int64_t off[32];      // row i's entry k of the batch stream is CSR entry off[i] + k
    uint32_t nbr[32];     // template neighbours of omega(v_i)
    int row[32];          // row whose piece of the current step starts at this lane
};

__device__ __forceinline__ void load_tmpl(SmemTmpl &s, const DevTmpl &t) {
    for (int i = threadIdx.x; i < kMaxT; i += blockDim.x) s.adj[i] = t.adj[i];
    for (int i = threadIdx.x; i < kMaxCls; i += blockDim.x) {
        s.cls_mask[i] = t.cls_mask[i];
        s.cls_need[i] = t.cls_need[i];
        s.cls_q[i] = t.cls_q[i];
    }
    if (threadIdx.x == 0) s.n_cls = t.n_cls;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Per-warp staging buffer for frontier appends: one global atomic per 32 items.
template <typename T>
struct WarpBuf {
    T *buf;          // 32 slots in shared memory
    int *cnt;        // shared counter
    T *out;          // global list
    unsigned int *gcount;
    unsigned long long cap = ~0ull;   // items past this index are counted, not stored

    __device__ __forceinline__ void flush() {
        int c = *cnt;
        if (c == 0) return;
        unsigned int base = 0;
        if (lane_id() == 0) base = atomicAdd(gcount, (unsigned int)c);
        base = __shfl_sync(FULL_MASK, base, 0);
        if ((int)lane_id() < c && (unsigned long long)base + lane_id() < cap) out[base + lane_id()] = buf[lane_id()];
        __syncwarp();
        if (lane_id() == 0) *cnt = 0;
        __syncwarp();
    }
    // warp-uniform call; lanes with pred push val
    __device__ __forceinline__ void push(bool pred, const T &val) {
        uint32_t m = __ballot_sync(FULL_MASK, pred);
        if (!m) return;
        int n = __popc(m);
        if (*cnt + n > 32) flush();
        int c = *cnt;
        if (pred) buf[c + __popc(m & ((1u << lane_id()) - 1u))] = val;
        __syncwarp();
        if (lane_id() == 0) *cnt = c + n;
        __syncwarp();
    }
};

// Zero the bits of CSR entries [beg, end); `G` lanes cooperate.  Words fully
// inside the range belong to this row alone and are stored; the two boundary
// words are shared with neighbouring rows and are cleared atomically.
template <int G>
__device__ __forceinline__ void clear_row(uint32_t *ebits, int64_t beg, int64_t end, int lane_g) {
    if (beg >= end) return;
    int64_t w0 = beg >> 5, w1 = (end - 1) >> 5;
    for (int64_t w = w0 + lane_g; w <= w1; w += G) {
        int64_t lo = w << 5;
        uint32_t keep = 0;
        if (beg > lo) keep |= (1u << (uint32_t)(beg - lo)) - 1u;
        if (end < lo + 32) keep |= ~((1u << (uint32_t)(end - lo)) - 1u);
        if (keep) atomicAnd(&ebits[w], keep);
        else ebits[w] = 0u;
    }
}

// OR / sum over aligned groups of G lanes (whole warp: one redux instruction)
template <int G>
__device__ __forceinline__ uint32_t grp_or(uint32_t x) {
    if constexpr (G == 32) {
        return __reduce_or_sync(FULL_MASK, x);
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) x |= __shfl_xor_sync(FULL_MASK, x, o);
        return x;
    }
}
template <int G>
__device__ __forceinline__ uint32_t grp_sum(uint32_t x) {
    if constexpr (G == 32) {
        return __reduce_add_sync(FULL_MASK, x);
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
        return x;
    }
}

// -------------------------------------------------------------------------
// K1: INIT_VERTEX_STATE (Alg. 3) and the first frontier
// -------------------------------------------------------------------------

struct LabelMask { uint32_t m[256]; };

__global__ void __launch_bounds__(256)
k_init(int64_t n, const int64_t *__restrict__ rp, const uint8_t *__restrict__ lab, LabelMask lm,
       const uint32_t *__restrict__ om_in, uint32_t *om0, uint32_t *om1, int32_t *small_out, int32_t *med_out,
       ChunkItem *chunk_out, HubAcc *acc, RoundStats *st, int hub_deg, int short_max) {
    __shared__ uint32_t slm[256];
    __shared__ int32_t sbuf[2][8][32];
    __shared__ int scnt[2][8];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) slm[i] = lm.m[i];
    const int wib = threadIdx.x >> 5;
    if (lane_id() == 0) { scnt[0][wib] = 0; scnt[1][wib] = 0; }
    __syncthreads();
    WarpBuf<int32_t> bs{sbuf[0][wib], &scnt[0][wib], small_out, &st->n_small};
    WarpBuf<int32_t> bm{sbuf[1][wib], &scnt[1][wib], med_out, &st->n_med};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_pad = (n + 31) & ~(int64_t)31;
    unsigned long long rows = 0;          // entries in the rows of the active vertices
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_pad; v += stride) {
        uint32_t w = 0;
        int64_t deg = 0;
        if (v < n) {
            w = slm[lab[v]];
            if (om_in) w &= om_in[v];     // resumed state, kept inside the initial one
            om0[v] = w;
            om1[v] = w;
            if (w) deg = rp[v + 1] - rp[v];
        }
        rows += (unsigned long long)deg;
        // buckets: short rows (4 lanes each), medium rows (a warp each), long
        // rows (split into pieces of hub_deg entries); every active vertex is
        // in exactly one of them
        const int64_t small_max = hub_deg < short_max ? hub_deg : short_max;
        bs.push(w && deg <= small_max, (int32_t)v);
        bm.push(w && deg > small_max && deg <= hub_deg, (int32_t)v);
        if (w && deg > hub_deg) {
            int nch = (int)((deg + hub_deg - 1) / hub_deg);
            int slot = (int)atomicAdd(&st->n_hub_slots, 1u);
            unsigned int base = atomicAdd(&st->n_chunk, (unsigned int)nch);
            acc[slot].pbase = base;
            for (int c = 0; c < nch; c++) chunk_out[base + c] = ChunkItem{(int32_t)v, c, slot, nch};
        }
    }
    bs.flush();
    bm.flush();
    for (int o = 16; o > 0; o >>= 1) rows += __shfl_xor_sync(FULL_MASK, rows, o);
    if (lane_id() == 0 && rows) atomicAdd(&st->row_entries, rows);
}

// -------------------------------------------------------------------------
// K2/K3: one LCC round (Alg. 4 with Alg. 5), snapshot form
// -------------------------------------------------------------------------

struct LccArgs {
    const int64_t *rp;
    const int32_t *col;
    const uint32_t *om_cur;
    uint32_t *om_next;
    uint32_t *ebits;
    const int32_t *small_in;
    const int32_t *med_in;
    const ChunkItem *chunk_in;
    int64_t n_small, n_med, n_chunk;
    int32_t *small_out;
    int32_t *med_out;
    ChunkItem *chunk_out;
    HubAcc *acc;
    RoundStats *st;
    int hub_deg;
    int64_t *deg;                 // entries each listed vertex keeps (0 if it dies), or nullptr
    int med_chunk;                // medium vertices a warp prefetches together (1..16)
    int small_chunk;              // unused by the short-row path (32 rows per batch)
    // first round after a fresh init: omega(u) is the initial mask of u's
    // label, so the neighbour gather reads the 1-byte label instead of the
    // 4-byte omega word (lab0 = labels, lmask = label -> initial omega)
    const uint8_t *lab0;
    LabelMask lmask;
    // with lab0: the neighbours' labels in CSR entry order (one byte per
    // entry, built once per graph), so the first round reads neither the
    // column index nor the neighbour's label: omega(u) = lmask[elab[e]]
    const uint8_t *elab;
    // later rounds over the full rows: warp-per-row paths visit only the set
    // bits (most entries of a live row are inactive by then)
    int sparse;
    // rounds queued without a host round trip: the list sizes come from the
    // previous round's counters, and a round after the fixpoint does nothing
    const RoundStats *prev;       // nullable: sizes are the fields above
    int resident_warps;           // warps of one resident wave (medium prefetch unit)
    uint32_t eta_off;             // ~0: ablation without edge elimination (every live
                                  // neighbour passes eta); 0: the method
    // a narrow copy of omega for the neighbour gathers (templates of at most
    // 8 / 16 vertices: 1 / 2 bytes per vertex, 4x / 2x fewer bytes than the
    // 32-bit words, so it stays in L2 at scale 25): read nw_cur, written to
    // nw_next beside om_next; nw_bytes 0 = no copy (gather om_cur)
    const void *nw_cur;
    void *nw_next;
    int nw_bytes;
};

// A neighbour's omega for the LCC gathers: from the narrow copy when there is one.
__device__ __forceinline__ uint32_t gather_om(const uint32_t *__restrict__ om, const void *nw, int nwb, int32_t u) {
    if (nwb == 1) return __ldg((const uint8_t *)nw + u);
    if (nwb == 2) return __ldg((const uint16_t *)nw + u);
    return __ldg(om + u);
}

// omega'(v) of the next round, and its narrow copy.
__device__ __forceinline__ void store_om(const LccArgs &a, int32_t v, uint32_t w) {
    a.om_next[v] = w;
    if (a.nw_bytes == 1) ((uint8_t *)a.nw_next)[v] = (uint8_t)w;
    else if (a.nw_bytes == 2) ((uint16_t *)a.nw_next)[v] = (uint16_t)w;
}

template <int MAXC>
struct Partial {
    uint32_t U = 0, nN = 0, achg = 0;
    uint32_t cnt[MAXC > 0 ? MAXC : 1];
    __device__ __forceinline__ Partial() {
#pragma unroll
        for (int c = 0; c < (MAXC > 0 ? MAXC : 1); c++) cnt[c] = 0;
    }
};

// Position of the r-th (0-based) set bit of x (x has more than r set bits):
// halve the range, keeping the half that holds it.
__device__ __forceinline__ uint32_t select_bit(uint32_t x, uint32_t r) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t w = 16; w > 0; w >>= 1) {
        const uint32_t low = __popc(x & ((1u << w) - 1u));
        if (low <= r) { r -= low; x >>= w; pos += w; }
    }
    return pos;
}

template <int MAXC>
__device__ __forceinline__ void tally_entry(uint32_t w, uint32_t nbr_v, const SmemTmpl &s, const uint32_t (&cm)[4],
                                            Partial<MAXC> &p, uint32_t &scanned, bool &keep) {
    keep = (w & nbr_v) != 0u;
    scanned += w != 0u;
    if (w != 0u && !keep) p.achg = 1u;  // eta eliminates the entry
    if (keep) {
        p.U |= w;
        p.nN++;
        if constexpr (MAXC > 0 && MAXC <= 4) {
#pragma unroll
            for (int c = 0; c < MAXC; c++) p.cnt[c] += (w & cm[c]) ? 1u : 0u;
        } else {
#pragma unroll
            for (int c = 0; c < MAXC; c++)
                if (c < s.n_cls) p.cnt[c] += (w & s.cls_mask[c]) ? 1u : 0u;
        }
    }
}

// Later rounds over the full rows, where most entries of a live row are
// already inactive: only the entries whose bit is set are visited, 32 per
// step (one per lane).  The bits of up to 1024 entries are read per load (one
// word per lane); lane k takes the k-th set bit of the group by a search over
// the words' prefix counts.  The next step's entries are located and their
// column indices loaded while the current step's neighbour omegas are
// gathered.  A failing entry's bit is cleared with an atomic (the words at
// the ends of the range are shared with other rows).
template <int MAXC>
__device__ __forceinline__ void scan_row_sparse(int64_t beg, int64_t end, uint32_t nbr_v,
                                                const int32_t *__restrict__ col, const uint32_t *__restrict__ om,
                                                uint32_t *ebits, const SmemTmpl &s, Partial<MAXC> &p,
                                                uint32_t &scanned, const uint32_t (&cm)[4], const void *nw, int nwb) {
    const int lane = (int)lane_id();
    const int64_t wb = beg >> 5, we = (end + 31) >> 5;
    for (int64_t g0 = wb; g0 < we; g0 += 32) {
        const int64_t wi = g0 + lane;
        uint32_t word = 0u;
        if (wi < we) {
            word = ebits[wi];
            const int64_t e0 = wi << 5;
            if (e0 < beg) word &= ~0u << (uint32_t)(beg - e0);
            if (end - e0 < 32) word &= (1u << (uint32_t)(end - e0)) - 1u;
        }
        const uint32_t c = __popc(word);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
        const uint32_t excl = incl - c;
        // lane k of a step: the (k0 + k)-th set entry of the group, and its column
        auto locate = [&](uint32_t k0, int64_t &e, int32_t &u) {
            const uint32_t k = k0 + (uint32_t)lane;
            int i = 0;                                  // last word whose prefix is <= k
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t ex = __shfl_sync(FULL_MASK, excl, i + step);
                if (ex <= k) i += step;
            }
            const uint32_t wd = __shfl_sync(FULL_MASK, word, i);
            const uint32_t ex_i = __shfl_sync(FULL_MASK, excl, i);
            e = -1;
            u = 0;
            if (k < total) {
                e = ((g0 + i) << 5) + (int64_t)select_bit(wd, k - ex_i);
                u = __ldcs(col + e);
            }
        };
        int64_t e_c = -1;
        int32_t u_c = 0;
        if (total) locate(0, e_c, u_c);
        for (uint32_t k0 = 0; k0 < total; k0 += 32) {
            const uint32_t w = e_c >= 0 ? gather_om(om, nw, nwb, u_c) : 0u;
            int64_t e_n = -1;
            int32_t u_n = 0;
            if (k0 + 32 < total) locate(k0 + 32, e_n, u_n);
            bool keep;
            tally_entry<MAXC>(w, nbr_v, s, cm, p, scanned, keep);
            if (e_c >= 0 && !keep) atomicAnd(&ebits[e_c >> 5], ~(1u << (uint32_t)(e_c & 31)));
            e_c = e_n;
            u_c = u_n;
        }
    }
}

// Stream the CSR entries [beg, end) of an active vertex: edge elimination by
// eta (entry kept iff the neighbour's omega contains a template neighbour of
// some q in omega(v)), the union omega' of Alg. 4 and the per-class counts of
// distinct compatible neighbours.
//
// Warp form: all 32 lanes walk the row together in windows aligned to the
// 32-entry words of the edge bitmap, so lane i of a window always owns bit i
// of one word: the bits of a window are one broadcast load and its failing
// entries are cleared with one ballot and one atomic.  Entry offsets are kept
// relative to the first window (32-bit), so the loads of a step use one base
// pointer with constant offsets.
// DENSE: every edge bit of the rows read is still set (the first round after
// init), so the bits are not loaded; otherwise a column index is only loaded
// for entries whose bit is set.
template <int MAXC, bool DENSE>
__device__ __forceinline__ void scan_row_warp(int64_t beg, int64_t end, uint32_t nbr_v,
                                              const int32_t *__restrict__ col,
                                              const uint32_t *__restrict__ om, uint32_t *ebits,
                                              const SmemTmpl &s, Partial<MAXC> &p,
                                              uint32_t &scanned, const uint8_t *__restrict__ lab0,
                                              const uint32_t *slm, const uint32_t (&cm)[4], const void *nw,
                                              int nwb, const uint8_t *__restrict__ elab, bool sparse) {
    if constexpr (!DENSE) {
        if (sparse) {
            scan_row_sparse<MAXC>(beg, end, nbr_v, col, om, ebits, s, p, scanned, cm, nw, nwb);
            return;
        }
    }
    constexpr int UNR = 4;   // windows per step
    const int lane = (int)lane_id();
    const int64_t w0 = beg >> 5;
    const int nwin = (int)(((end + 31) >> 5) - w0);
    const int lo = (int)(beg - (w0 << 5));          // entries before lo belong to the previous row
    const int hi = (int)(end - (w0 << 5));          // entries from hi on belong to the next row
    const int32_t *cb = col + (w0 << 5) + lane;
    const uint8_t *lb = (DENSE && elab) ? elab + (w0 << 5) + lane : nullptr;   // first round only
    uint32_t *eb = ebits + w0;
    // the column indices of the next step are loaded while the neighbour
    // omegas of the current step are gathered
    bool act[UNR];
    int32_t u[UNR];
    auto load_step = [&](int k0) {
        const int rel0 = k0 * 32 + lane;
        const int32_t *c0 = cb + k0 * 32;
        uint32_t word[UNR];
#pragma unroll
        for (int j = 0; j < UNR; j++) {
            word[j] = ~0u;
            if (!DENSE) word[j] = (k0 + j < nwin) ? eb[k0 + j] : 0u;
        }
#pragma unroll
        for (int j = 0; j < UNR; j++) {
            const int rel = rel0 + j * 32;
            act[j] = rel >= lo && rel < hi && ((word[j] >> lane) & 1u);
            // the column index, or the neighbour's label when the entry labels are given
            if (lb) u[j] = act[j] ? (int32_t)__ldcs(lb + k0 * 32 + j * 32) : 0;
            else u[j] = act[j] ? __ldcs(c0 + j * 32) : 0;
        }
    };
    load_step(0);
    for (int k0 = 0; k0 < nwin; k0 += UNR) {
        uint32_t wu[UNR];
        bool was[UNR];
#pragma unroll
        for (int j = 0; j < UNR; j++) {
            was[j] = act[j];
            if (lb) wu[j] = act[j] ? slm[u[j]] : 0u;
            else if (lab0) wu[j] = act[j] ? slm[__ldg(lab0 + u[j])] : 0u;
            else wu[j] = act[j] ? gather_om(om, nw, nwb, u[j]) : 0u;
        }
        if (k0 + UNR < nwin) load_step(k0 + UNR);
#pragma unroll
        for (int j = 0; j < UNR; j++) {
            if (k0 + j >= nwin) break;          // past the row's last window (warp-uniform)
            const uint32_t w = wu[j];
            const bool keep = (w & nbr_v) != 0u;
            scanned += w != 0u;
            if (w != 0u && !keep) p.achg = 1u;  // eta eliminates the entry
            if (keep) {
                p.U |= w;
                p.nN++;
                if constexpr (MAXC > 0 && MAXC <= 4) {
#pragma unroll
                    for (int c = 0; c < MAXC; c++) p.cnt[c] += (w & cm[c]) ? 1u : 0u;
                } else {
#pragma unroll
                    for (int c = 0; c < MAXC; c++)
                        if (c < s.n_cls) p.cnt[c] += (w & s.cls_mask[c]) ? 1u : 0u;
                }
            }
            // the bit goes with the failing entries and with those whose other
            // end is already inactive (no change of the state A: that entry is
            // inactive already), so later rounds and compaction see only live
            // compatible entries
            const uint32_t drop = __ballot_sync(FULL_MASK, was[j] && !keep);
            if (drop) {
                const int k = k0 + j;
                if (k * 32 >= lo && k * 32 + 32 <= hi) {
                    // the word holds entries of this row only
                    const uint32_t kept = __ballot_sync(FULL_MASK, keep);
                    if (lane == 0) eb[k] = kept;
                } else if (lane == 0) {
                    atomicAnd(&eb[k], ~drop);
                }
            }
        }
    }
}

// Clear the entries of a row (at most 32 long) given by a row-relative mask.
__device__ __forceinline__ void clear_rel(uint32_t *ebits, int64_t beg, uint32_t clr) {
    if (!clr) return;
    const uint32_t sh = (uint32_t)(beg & 31);
    atomicAnd(&ebits[beg >> 5], ~(clr << sh));
    if (sh && (clr >> (32 - sh))) atomicAnd(&ebits[(beg >> 5) + 1], ~(clr >> (32 - sh)));
}

// The vertex-elimination rule of Alg. 4 plus the multiplicity rule of
// Section 4.1: q survives iff adj(q) is inside omega' and every class of q
// has enough distinct neighbours; no surviving edge eliminates the vertex.
template <int MAXC>
__device__ __forceinline__ uint32_t decide(uint32_t wv, const Partial<MAXC> &p, const SmemTmpl &s) {
    uint32_t keep = 0;
    for (uint32_t m = wv; m; m &= m - 1u) {
        int q = __ffs(m) - 1;
        if ((s.adj[q] & ~p.U) == 0u) keep |= 1u << q;
    }
#pragma unroll
    for (int c = 0; c < MAXC; c++)
        if (c < s.n_cls && p.cnt[c] < s.cls_need[c]) keep &= ~(1u << s.cls_q[c]);
    if (p.nN == 0u) keep = 0u;
    return keep;
}

__device__ __forceinline__ uint32_t nbr_mask(uint32_t wv, const SmemTmpl &s) {
    uint32_t m = 0;
    for (uint32_t x = wv; x; x &= x - 1u) m |= s.adj[__ffs(x) - 1];
    return m;
}

// Round counters one warp accumulates (summed once at the end of the kernel).
struct LccTally {
    uint32_t scanned = 0;          // per lane
    unsigned long long rows = 0, alive = 0, kept = 0, rows_next = 0;   // lane 0 (or the row lanes)
    uint32_t changed = 0;
};

// Short rows, 32 per warp batch (lane i owns row i of the batch).  The rows'
// entries are walked as one stream, 32 per step with one entry per lane, so
// lanes stay busy whatever the row lengths.  A step holds pieces of several
// rows: every lane finds its row from the piece starts, and per-row sums are
// segmented warp reductions whose result each row's lane collects.
//
// The walk is software-pipelined: while the neighbour omegas (or labels) of
// one step are gathered, the next step's rows are located and its edge bits
// and column indices are loaded, and the next batch's list entries, omegas
// and row offsets are loaded during the current batch.  The column loads
// stream past the caches (read once per round).

// Where the entries of one step lie: lane k holds stream entry k0 + k.
struct ShortStep {
    uint32_t seg;        // lanes of this lane's row piece
    int seg_lo;          // first lane of the piece
    int64_t e;           // CSR entry
    uint32_t nb;         // template neighbours of its row's omega
    bool act;            // a live entry (in range, bit set)
    int32_t u;           // its column index (valid when act)
    bool ov;             // row lane: its row has a piece in this step ...
    int lo;              // ... starting at this lane
};

template <bool DENSE>
__device__ __forceinline__ void short_locate(const LccArgs &a, ShortRows &sr, int k0, int T, int start, int d,
                                             ShortStep &st) {
    const int lane = (int)lane_id();
    const int lo = max(start, k0) - k0, hi = min(start + d, k0 + 32) - k0;
    st.ov = lo < hi;
    st.lo = lo;
    if (st.ov) sr.row[lo] = lane;
    const uint32_t H = __reduce_or_sync(FULL_MASK, st.ov ? (1u << lo) : 0u);   // piece starts (bit 0 always)
    __syncwarp();
    const uint32_t upto = lane == 31 ? FULL_MASK : ((2u << lane) - 1u);
    st.seg_lo = 31 - __clz(H & upto);
    const uint32_t above = H & ~upto;
    const int seg_hi = above ? __ffs(above) - 1 : 32;
    st.seg = (seg_hi == 32 ? FULL_MASK : ((1u << seg_hi) - 1u)) & ~((1u << st.seg_lo) - 1u);
    const int r = sr.row[st.seg_lo];
    const int k = k0 + lane;
    const bool valid = k < T;
    st.e = sr.off[r] + k;
    st.nb = sr.nbr[r];
    st.act = valid;
    if (!DENSE && valid) st.act = (__ldg(a.ebits + (st.e >> 5)) >> (uint32_t)(st.e & 31)) & 1u;
    if (DENSE && a.elab) st.u = st.act ? (int32_t)__ldcs(a.elab + st.e) : 0;   // the neighbour's label
    else st.u = st.act ? __ldcs(a.col + st.e) : 0;
    __syncwarp();                                // sr.row is rewritten by the next step
}

template <int MAXC, bool DENSE>
__device__ __forceinline__ void short_rows(const LccArgs &a, const SmemTmpl &s, const uint32_t *slm,
                                           const uint32_t (&cm)[4], ShortRows &sr, int64_t first, int64_t stride,
                                           int64_t n_small, WarpBuf<int32_t> &bs, LccTally &tl) {
    const int lane = (int)lane_id();
    const int64_t n_batch = (n_small + 31) / 32;
    auto load_v = [&](int64_t ch) -> int32_t {
        const int64_t idx = ch * 32 + lane;
        return (ch < n_batch && idx < n_small) ? a.small_in[idx] : -1;
    };
    int32_t v_nx = load_v(first);
    uint32_t wv_nx = 0u;
    int64_t b_nx = 0;
    int d_nx = 0;
    auto load_row = [&]() {
        wv_nx = 0u; b_nx = 0; d_nx = 0;
        if (v_nx >= 0) {
            wv_nx = __ldg(a.om_cur + v_nx);
            if (wv_nx) {
                b_nx = a.rp[v_nx];
                d_nx = (int)(a.rp[v_nx + 1] - b_nx);
            }
        }
    };
    load_row();
    for (int64_t ch = first; ch < n_batch; ch += stride) {
        const int32_t v = v_nx;
        const uint32_t wv = wv_nx;
        const int64_t b = b_nx;
        const int d = d_nx;
        v_nx = load_v(ch + stride);              // in flight during this batch
        const uint32_t nbr = wv ? (nbr_mask(wv, s) | a.eta_off) : 0u;
        int S = d;                               // inclusive prefix of the row lengths
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL_MASK, S, o);
            if (lane >= o) S += t;
        }
        const int T = __shfl_sync(FULL_MASK, S, 31);
        const int start = S - d;
        sr.off[lane] = b - start;
        sr.nbr[lane] = nbr;
        uint32_t U = 0u, N = 0u;
        uint32_t cnt[MAXC > 0 ? MAXC : 1];
#pragma unroll
        for (int c = 0; c < (MAXC > 0 ? MAXC : 1); c++) cnt[c] = 0u;
        __syncwarp();
        ShortStep cur;
        if (T > 0) short_locate<DENSE>(a, sr, 0, T, start, d, cur);
        load_row();                              // the next batch's omegas and offsets
        for (int k0 = 0; k0 < T; k0 += 32) {
            uint32_t w = 0u;
            if (cur.act)
                w = (DENSE && a.elab) ? slm[cur.u]
                           : (a.lab0 ? slm[__ldg(a.lab0 + cur.u)] : gather_om(a.om_cur, a.nw_cur, a.nw_bytes, cur.u));
            ShortStep nx;
            if (k0 + 32 < T) short_locate<DENSE>(a, sr, k0 + 32, T, start, d, nx);
            const bool keep = (w & cur.nb) != 0u;
            tl.scanned += w != 0u;
            if (w != 0u && !keep) tl.changed = 1u;       // eta eliminates a live entry
            // entries whose other end is already inactive lose their bit too (no
            // change of the state: such an entry is inactive already)
            const uint32_t dm = __ballot_sync(FULL_MASK, cur.act && !keep) & cur.seg;
            uint32_t gk[MAXC > 4 ? MAXC : 1];
            uint32_t rk;
            const uint32_t ru = __reduce_or_sync(cur.seg, keep ? w : 0u);
            if constexpr (MAXC <= 4) {
                // the kept count and up to four class counts of a piece (each at
                // most 32) packed in 6-bit fields
                uint32_t pk = keep ? 1u : 0u;
#pragma unroll
                for (int c = 0; c < MAXC; c++)
                    if (keep && (w & cm[c])) pk += 1u << (6 * (c + 1));
                rk = __reduce_add_sync(cur.seg, pk);
            } else {
                rk = __reduce_add_sync(cur.seg, keep ? 1u : 0u);
#pragma unroll
                for (int c = 0; c < MAXC; c++)
                    gk[c] = c < s.n_cls ? __reduce_add_sync(cur.seg, (keep && (w & s.cls_mask[c])) ? 1u : 0u) : 0u;
            }
            if (lane == cur.seg_lo && dm) {
                // the piece's entries are consecutive from e: at most two words
                const uint32_t bits = dm >> cur.seg_lo;
                const uint32_t sh = (uint32_t)(cur.e & 31);
                atomicAnd(&a.ebits[cur.e >> 5], ~(bits << sh));
                if (sh && (bits >> (32 - sh))) atomicAnd(&a.ebits[(cur.e >> 5) + 1], ~(bits >> (32 - sh)));
            }
            // each row's lane takes the sums of its piece
            const int src = cur.ov ? cur.lo : 0;
            const uint32_t gu = __shfl_sync(FULL_MASK, ru, src);
            const uint32_t gr = __shfl_sync(FULL_MASK, rk, src);
            if constexpr (MAXC <= 4) {
                if (cur.ov) {
                    U |= gu;
                    N += gr & 63u;
#pragma unroll
                    for (int c = 0; c < MAXC; c++) cnt[c] += (gr >> (6 * (c + 1))) & 63u;
                }
            } else {
                uint32_t gc[MAXC];
#pragma unroll
                for (int c = 0; c < MAXC; c++) gc[c] = __shfl_sync(FULL_MASK, gk[c], src);
                if (cur.ov) {
                    U |= gu;
                    N += gr;
#pragma unroll
                    for (int c = 0; c < MAXC; c++) cnt[c] += gc[c];
                }
            }
            cur = nx;
        }
        if (v >= 0) {
            uint32_t keep = 0u;
            if (wv) {
                Partial<MAXC> p;
                p.U = U;
                p.nN = N;
#pragma unroll
                for (int c = 0; c < (MAXC > 0 ? MAXC : 1); c++) p.cnt[c] = cnt[c];
                keep = decide<MAXC>(wv, p, s);
                tl.rows += (unsigned long long)d;
                tl.alive++;
                if (keep) { tl.kept += N; tl.rows_next += (unsigned long long)d; }
                if (keep != wv) tl.changed = 1u;
                if (keep == 0u) clear_row<1>(a.ebits, b, b + d, 0);
            }
            store_om(a, v, keep);
            if (a.deg) a.deg[v] = keep ? (int64_t)N : 0;
        }
        // the batch's vertices that were active at the start of the round
        bs.push(v >= 0 && wv != 0u, v);
        __syncwarp();                            // sr.off / sr.nbr are rewritten by the next batch
    }
}

template <int MAXC, bool DENSE>
__global__ void __launch_bounds__(256, 4)
k_lcc_round(LccArgs a, DevTmpl t) {
    int64_t n_small = a.n_small, n_med = a.n_med, n_chunk = a.n_chunk;
    int MB = a.med_chunk;
    if (a.prev) {
        if (a.prev->changed == 0u) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.st->skipped = 1u;
            return;
        }
        n_small = a.prev->n_small;
        n_med = a.prev->n_med;
        n_chunk = a.prev->n_chunk;
        MB = (int)max((int64_t)1, min((int64_t)16, n_med / (4 * (int64_t)a.resident_warps)));
    }
    __shared__ SmemTmpl s;
    __shared__ uint32_t slm[256];
    __shared__ int32_t sbuf[2][8][32];
    __shared__ ChunkItem cbuf[8][32];
    __shared__ ShortRows srows[8];
    __shared__ int scnt[3][8];
    load_tmpl(s, t);
    if (a.lab0)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) slm[i] = a.lmask.m[i];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    if (lane == 0) { scnt[0][wib] = 0; scnt[1][wib] = 0; scnt[2][wib] = 0; }
    __syncthreads();
    WarpBuf<int32_t> bs{sbuf[0][wib], &scnt[0][wib], a.small_out, &a.st->n_small};
    WarpBuf<int32_t> bm{sbuf[1][wib], &scnt[1][wib], a.med_out, &a.st->n_med};
    WarpBuf<ChunkItem> bc{cbuf[wib], &scnt[2][wib], a.chunk_out, &a.st->n_chunk};
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    LccTally tl;
    // masks of the first four label-multiplicity classes in registers (0 for
    // classes the template does not have: they never count)
    uint32_t cm[4];
#pragma unroll
    for (int c = 0; c < 4; c++) cm[c] = s.cls_mask[c];

    // (1) pieces of long rows: one warp per piece, combined through HubAcc;
    // the last piece to finish decides for the vertex.
    for (int64_t it = gwarp; it < n_chunk; it += nwarps) {
        ChunkItem ci = a.chunk_in[it];
        const uint32_t wv = __ldg(a.om_cur + ci.v);
        if (wv == 0u) {
            if (ci.c == 0 && lane == 0) {
                store_om(a, ci.v, 0u);
                if (a.deg) a.deg[ci.v] = 0;
            }
            continue;
        }
        const int64_t rbeg = a.rp[ci.v], rend = a.rp[ci.v + 1];
        const int64_t beg = rbeg + (int64_t)ci.c * a.hub_deg;
        const int64_t end = min(rend, beg + (int64_t)a.hub_deg);
        if (lane == 0) { tl.rows += (unsigned long long)(end - beg); tl.alive += ci.c == 0; }
        Partial<MAXC> p;
        scan_row_warp<MAXC, DENSE>(beg, end, nbr_mask(wv, s) | a.eta_off, a.col, a.om_cur, a.ebits, s, p, tl.scanned, a.lab0,
                                   slm, cm, a.nw_cur, a.nw_bytes, a.elab, a.sparse != 0);
        p.U = grp_or<32>(p.U);
        p.nN = grp_sum<32>(p.nN);
        p.achg = grp_or<32>(p.achg);
#pragma unroll
        for (int c = 0; c < MAXC; c++) p.cnt[c] = grp_sum<32>(p.cnt[c]);
        HubAcc *h = a.acc + ci.slot;
        unsigned int ticket = 0;
        if (lane == 0) {
            if (p.U) atomicOr(&h->U, p.U);
            if (p.nN) atomicAdd(&h->nN, p.nN);
            if (p.achg) atomicOr(&h->flags, 1u);
#pragma unroll
            for (int c = 0; c < MAXC; c++)
                if (p.cnt[c]) atomicAdd(&h->cnt[c], p.cnt[c]);
            __threadfence();
            ticket = atomicAdd(&h->done, 1u);
        }
        ticket = __shfl_sync(FULL_MASK, ticket, 0);
        if (ticket == (unsigned int)(ci.nchunks - 1)) {
            __threadfence();
            Partial<MAXC> tot;
            tot.U = atomicOr(&h->U, 0u);
            tot.nN = atomicAdd(&h->nN, 0u);
            tot.achg = atomicOr(&h->flags, 0u);
#pragma unroll
            for (int c = 0; c < MAXC; c++) tot.cnt[c] = atomicAdd(&h->cnt[c], 0u);
            uint32_t keep = decide<MAXC>(wv, tot, s);
            if (lane == 0) {
                store_om(a, ci.v, keep);
                if (a.deg) a.deg[ci.v] = keep ? (int64_t)tot.nN : 0;
            }
            if (lane == 0 && keep) { tl.kept += tot.nN; tl.rows_next += (unsigned long long)(rend - rbeg); }
            if (keep != wv || tot.achg) tl.changed = 1u;
            if (keep == 0u) clear_row<32>(a.ebits, rbeg, rend, lane);
            __syncwarp();
            if (lane == 0) {
                h->U = 0u; h->nN = 0u; h->flags = 0u; h->done = 0u;
                for (int c = 0; c < MAXC; c++) h->cnt[c] = 0u;
            }
        }
        bc.push(lane == 0, ci);
    }

    // (2) medium rows: one warp per vertex, taken 16 at a time: the list
    // entries, omega and row offsets of the next 16 vertices are loaded by 16
    // lanes at once, so each row walk starts from registers
    const int64_t n_mchunks = (n_med + MB - 1) / MB;
    for (int64_t ch = gwarp; ch < n_mchunks; ch += nwarps) {
        const int64_t idx = ch * MB + lane;
        int32_t vl = -1;
        uint32_t wl = 0u;
        int64_t bl = 0, el = 0;
        if (lane < MB && idx < n_med) {
            vl = a.med_in[idx];
            wl = __ldg(a.om_cur + vl);
            if (wl) { bl = a.rp[vl]; el = a.rp[vl + 1]; }
        }
        for (int j = 0; j < MB; j++) {
            const int32_t v = __shfl_sync(FULL_MASK, vl, j);
            if (v < 0) break;
            const uint32_t wv = __shfl_sync(FULL_MASK, wl, j);
            const int64_t beg = __shfl_sync(FULL_MASK, bl, j), end = __shfl_sync(FULL_MASK, el, j);
            uint32_t keep = 0u, p_nN = 0u;
            if (wv) {
                if (lane == 0) { tl.rows += (unsigned long long)(end - beg); tl.alive++; }
                Partial<MAXC> p;
                scan_row_warp<MAXC, DENSE>(beg, end, nbr_mask(wv, s) | a.eta_off, a.col, a.om_cur, a.ebits, s, p, tl.scanned,
                                           a.lab0, slm, cm, a.nw_cur, a.nw_bytes, a.elab, a.sparse != 0);
                p.U = grp_or<32>(p.U);
                p.nN = grp_sum<32>(p.nN);
                p.achg = grp_or<32>(p.achg);
#pragma unroll
                for (int c = 0; c < MAXC; c++) p.cnt[c] = grp_sum<32>(p.cnt[c]);
                keep = decide<MAXC>(wv, p, s);
                p_nN = p.nN;
                if (lane == 0 && keep) { tl.kept += p.nN; tl.rows_next += (unsigned long long)(end - beg); }
                if (keep != wv || p.achg) tl.changed = 1u;
                if (keep == 0u) clear_row<32>(a.ebits, beg, end, lane);
            }
            if (lane == 0) {
                store_om(a, v, keep);
                if (a.deg) a.deg[v] = keep ? (int64_t)p_nN : 0;
            }
        }
        // the chunk's vertices that were active at the start of the round, in one push
        bm.push(vl >= 0 && wl != 0u, vl);
    }

    // (3) short rows: 32 vertices per warp batch, entries streamed flat
    short_rows<MAXC, DENSE>(a, s, slm, cm, srows[wib], gwarp, nwarps, n_small, bs, tl);

    bs.flush();
    bm.flush();
    bc.flush();
    // warp totals
    unsigned long long scanned64 = tl.scanned;
    for (int o = 16; o > 0; o >>= 1) {
        scanned64 += __shfl_xor_sync(FULL_MASK, scanned64, o);
        tl.rows += __shfl_xor_sync(FULL_MASK, tl.rows, o);
        tl.alive += __shfl_xor_sync(FULL_MASK, tl.alive, o);
        tl.kept += __shfl_xor_sync(FULL_MASK, tl.kept, o);
        tl.rows_next += __shfl_xor_sync(FULL_MASK, tl.rows_next, o);
        tl.changed |= __shfl_xor_sync(FULL_MASK, tl.changed, o);
    }
    if (lane == 0) {
        if (scanned64) atomicAdd(&a.st->scanned, scanned64);
        if (tl.rows) atomicAdd(&a.st->row_entries, tl.rows);
        if (tl.alive) atomicAdd(&a.st->alive, tl.alive);
        if (tl.kept) atomicAdd(&a.st->kept, tl.kept);
        if (tl.rows_next) atomicAdd(&a.st->rows_next, tl.rows_next);
        if (tl.changed) atomicOr(&a.st->changed, 1u);
    }
}

// -------------------------------------------------------------------------
// K4: row compaction between LCC rounds (frontier and edge-bitmap compaction)
//
// Later rounds touch only the survivors, but the rows of the survivors still
// hold every neighbour they started with; once most of those entries are
// inactive a round spends its time skipping them.  Compaction writes a new
// CSR whose rows keep, in the same (ascending id) order, only the entries
// whose bit is set and whose other end point is still active: exactly the
// entries the next round would examine.  Ids stay the original vertex ids;
// the new bitmap starts with every bit set.  Entries left out are inactive
// for good (bits are only ever cleared and omega only shrinks), so every
// later round, and every search at a fixpoint, sees the same active entries
// as on the full rows.
//
// The frontier is rebuilt first (k_init over the live vertices) so that the
// pieces of a long row are consecutive in the piece list, in piece order:
// piece c's output offset is then the row's offset plus the counts of pieces
// 0..c-1.
// -------------------------------------------------------------------------

struct CompactArgs {
    const int64_t *rp;            // rows being compacted
    const int32_t *col;
    const uint32_t *bits;         // set exactly for the entries to keep
    const uint8_t *lab;
    const uint32_t *om;           // omega after the last round
    const int32_t *small_in;
    const int32_t *med_in;
    const ChunkItem *chunk_in;
    const HubAcc *acc;            // first-piece index of each long row (pbase)
    const RoundStats *lists;      // sizes of the three lists (written by the rebuild before)
    int hub_deg;
    int n_rank;                   // distinct labels of the template
    uint8_t lab_rank[256];        // rank of a template label among them
    uint8_t rank_label[kMaxT];
    uint32_t *piece_cnt;          // kept entries per (piece, rank) of long rows
    const int64_t *sub_rp;        // offsets of the new rows
    int32_t *sub_col;             // the new rows, grouped by label, ids ascending
    uint8_t *sub_nlab;            // inside a group, and their labels
    int32_t *dslot;               // per live vertex: its slot in gdir
    int64_t *gdir;                // per slot: start of each label group, then the row end
    unsigned int *n_slots;        // slot counter (zeroed before)
};

// Visit the entries of [beg, end) whose bit is set, 32 at a time and in
// ascending order: f(e, valid) is called by all lanes, lane i with the i-th
// set entry of the batch (valid) or none.  The bits are read 32 words
// (1024 entries) per load, so long runs of inactive entries cost little.
template <typename F>
__device__ __forceinline__ void for_set_bits(const uint32_t *bits, int64_t beg, int64_t end, F &&f) {
    const int lane = (int)lane_id();
    const int64_t wb = beg >> 5, we = (end + 31) >> 5;
    for (int64_t w0 = wb; w0 < we; w0 += 32) {
        const int64_t wi = w0 + lane;
        uint32_t word = 0u;
        if (wi < we) {
            word = bits[wi];
            const int64_t e0 = wi << 5;
            if (e0 < beg) word &= ~0u << (uint32_t)(beg - e0);
            if (end - e0 < 32) word &= (1u << (uint32_t)(end - e0)) - 1u;
        }
        const uint32_t c = __popc(word);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
        const uint32_t excl = incl - c;
        for (uint32_t k0 = 0; k0 < total; k0 += 32) {
            const uint32_t k = k0 + (uint32_t)lane;
            int i = 0;                                // last word whose prefix is <= k
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t ex = __shfl_sync(FULL_MASK, excl, i + step);
                if (ex <= k) i += step;
            }
            const uint32_t wd = __shfl_sync(FULL_MASK, word, i);
            const uint32_t ex_i = __shfl_sync(FULL_MASK, excl, i);
            const bool valid = k < total;
            int64_t e = -1;
            if (valid) e = ((w0 + i) << 5) + (int64_t)select_bit(wd, k - ex_i);
            f(e, valid);
        }
    }
}

__device__ __forceinline__ uint32_t lane_rank_count(int r, int n_rank) {
    uint32_t rc = 0;
    for (int rr = 0; rr < n_rank; rr++) {
        const uint32_t m = __ballot_sync(FULL_MASK, r == rr);
        if ((int)lane_id() == rr) rc = __popc(m);
    }
    return rc;
}

// Kept entries of [beg, end) per label rank, summed into lane r (r < n_rank).
__device__ __forceinline__ uint32_t rank_counts(const CompactArgs &a, int64_t beg, int64_t end) {
    uint32_t rc = 0;
    for_set_bits(a.bits, beg, end, [&](int64_t e, bool valid) {
        int r = valid ? (int)a.lab_rank[__ldg(a.lab + __ldg(a.col + e))] : -1;
        if (r >= a.n_rank) r = -1;           // never: kept entries have template labels
        rc += lane_rank_count(r, a.n_rank);
    });
    return rc;
}

// Write the kept entries of [beg, end): lane r holds the next output index of
// label rank r.  Order inside a rank is the visiting order (ascending).
__device__ __forceinline__ void place_ranked(const CompactArgs &a, int64_t beg, int64_t end, int64_t cur) {
    const int lane = (int)lane_id();
    const uint32_t below = (1u << lane) - 1u;
    for_set_bits(a.bits, beg, end, [&](int64_t e, bool valid) {
        int32_t u = -1;
        int r = -1;
        if (valid) {
            u = __ldg(a.col + e);
            r = (int)a.lab_rank[__ldg(a.lab + u)];
            if (r >= a.n_rank) r = -1;
        }
        int64_t pos = -1;
        for (int rr = 0; rr < a.n_rank; rr++) {
            const uint32_t m = __ballot_sync(FULL_MASK, r == rr);
            const int64_t base = __shfl_sync(FULL_MASK, cur, rr);
            if (r == rr) pos = base + __popc(m & below);
            if (lane == rr) cur += __popc(m);
        }
        if (r >= 0) {
            a.sub_col[pos] = u;
            a.sub_nlab[pos] = a.rank_label[r];
        }
    });
}

// Exclusive prefix over lanes.
__device__ __forceinline__ uint32_t lane_excl(uint32_t x) {
    const int lane = (int)lane_id();
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    return incl - x;
}

// Per-(piece, rank) kept entries of the pieces of long rows.
__global__ void __launch_bounds__(256)
k_compact_count(CompactArgs a) {
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    const int64_t n_chunk = a.lists->n_chunk;
    for (int64_t it = gwarp; it < n_chunk; it += nwarps) {
        const ChunkItem ci = a.chunk_in[it];
        if (__ldg(a.om + ci.v) == 0u) continue;
        const int64_t rbeg = a.rp[ci.v], rend = a.rp[ci.v + 1];
        const int64_t beg = rbeg + (int64_t)ci.c * a.hub_deg;
        const int64_t end = min(rend, beg + (int64_t)a.hub_deg);
        const uint32_t rc = rank_counts(a, beg, end);
        const int64_t p = (int64_t)a.acc[ci.slot].pbase + ci.c;
        if (lane < a.n_rank) a.piece_cnt[p * a.n_rank + lane] = rc;
    }
}

// Write the new rows and their label-group directory.  Pieces of long rows:
// rank r's group starts after the lower ranks of the whole row, and a piece's
// entries of rank r follow those of the row's earlier pieces.  Whole rows:
// by one lane when the row keeps at most 16 entries, else by the warp.
__global__ void __launch_bounds__(256)
k_compact_fill(CompactArgs a) {
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    const int64_t n_chunk = a.lists->n_chunk, n_med = a.lists->n_med, n_small = a.lists->n_small;
    for (int64_t it = gwarp; it < n_chunk; it += nwarps) {
        const ChunkItem ci = a.chunk_in[it];
        if (__ldg(a.om + ci.v) == 0u) continue;
        const int64_t rbeg = a.rp[ci.v], rend = a.rp[ci.v + 1];
        const int64_t beg = rbeg + (int64_t)ci.c * a.hub_deg;
        const int64_t end = min(rend, beg + (int64_t)a.hub_deg);
        const int64_t p0 = (int64_t)a.acc[ci.slot].pbase;
        // per rank, the row's total and the part in pieces before this one
        // (lanes stride over the pieces; lane r keeps rank r's sums)
        uint32_t tot = 0, before = 0;
        for (int r = 0; r < a.n_rank; r++) {
            uint32_t t = 0, b = 0;
            for (int c2 = lane; c2 < ci.nchunks; c2 += 32) {
                const uint32_t x = a.piece_cnt[(p0 + c2) * a.n_rank + r];
                t += x;
                if (c2 < ci.c) b += x;
            }
            t = __reduce_add_sync(FULL_MASK, t);
            b = __reduce_add_sync(FULL_MASK, b);
            if (lane == r) { tot = t; before = b; }
        }
        const int64_t gstart = a.sub_rp[ci.v] + (int64_t)lane_excl(tot);
        if (ci.c == 0) {
            unsigned int slot = 0;
            if (lane == 0) {
                slot = atomicAdd(a.n_slots, 1u);
                a.dslot[ci.v] = (int32_t)slot;
            }
            slot = __shfl_sync(FULL_MASK, slot, 0);
            if (lane <= a.n_rank) a.gdir[(int64_t)slot * (a.n_rank + 1) + lane] = gstart;
        }
        place_ranked(a, beg, end, gstart + before);
    }
    // whole rows, 32 list entries per warp step.  A row keeping at most 16
    // entries (most of them, once the first round has run) is written by its
    // own lane, one pass per label rank; the others by the whole warp in turn.
    const int64_t n_rows = n_med + n_small;
    for (int64_t b = gwarp * 32; b < n_rows; b += nwarps * 32) {
        const int64_t idx = b + lane;
        int32_t vl = -1;
        int64_t beg = 0, end = 0, out = 0, k = 0;
        if (idx < n_rows) {
            vl = idx < n_med ? a.med_in[idx] : a.small_in[idx - n_med];
            if (__ldg(a.om + vl) == 0u) vl = -1;
        }
        if (vl >= 0) {
            beg = a.rp[vl];
            end = a.rp[vl + 1];
            out = a.sub_rp[vl];
            k = a.sub_rp[vl + 1] - out;
        }
        // one directory slot per live row, one atomic per warp step
        const uint32_t live = __ballot_sync(FULL_MASK, vl >= 0);
        unsigned int slot0 = 0;
        if (lane == 0 && live) slot0 = atomicAdd(a.n_slots, (unsigned int)__popc(live));
        const unsigned int slot = __shfl_sync(FULL_MASK, slot0, 0) + (unsigned int)__popc(live & ((1u << lane) - 1u));
        if (vl >= 0) a.dslot[vl] = (int32_t)slot;
        if (vl >= 0 && k <= 16) {
            const int64_t stop = out + k;
            int64_t *dir = a.gdir + (int64_t)slot * (a.n_rank + 1);
            // the row's kept entries (at most 16): positions from the bit words
            // (four words per step), then their columns, then their labels, each
            // as independent loads; then placed label by label
            int32_t eu[16];
            uint8_t er[16];
            int n = 0;
            for (int64_t wi = beg >> 5; (wi << 5) < end && n < 16; wi += 4) {
                uint32_t wd[4];
#pragma unroll
                for (int j = 0; j < 4; j++) wd[j] = ((wi + j) << 5) < end ? a.bits[wi + j] : 0u;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    uint32_t word = wd[j];
                    const int64_t e0 = (wi + j) << 5;
                    if (e0 < beg) word &= ~0u << (uint32_t)(beg - e0);
                    if (end - e0 < 32) word &= end > e0 ? (1u << (uint32_t)(end - e0)) - 1u : 0u;
                    for (; word && n < 16; word &= word - 1u) eu[n++] = (int32_t)(e0 + __ffs(word) - 1 - beg);
                }
            }
#pragma unroll
            for (int i = 0; i < 16; i++)
                if (i < n) eu[i] = __ldg(a.col + beg + eu[i]);
#pragma unroll
            for (int i = 0; i < 16; i++)
                er[i] = i < n ? a.lab_rank[__ldg(a.lab + eu[i])] : (uint8_t)0xFF;
            for (int r = 0; r < a.n_rank; r++) {
                dir[r] = out;
                const uint8_t L = a.rank_label[r];
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    if (er[i] == r && out < stop) {
                        a.sub_col[out] = eu[i];
                        a.sub_nlab[out] = L;
                        out++;
                    }
                }
            }
            dir[a.n_rank] = stop;
        }
        for (uint32_t big = __ballot_sync(FULL_MASK, vl >= 0 && k > 16); big; big &= big - 1u) {
            const int src = __ffs(big) - 1;
            const int64_t rb = __shfl_sync(FULL_MASK, beg, src), re = __shfl_sync(FULL_MASK, end, src);
            const int64_t ro = __shfl_sync(FULL_MASK, out, src);
            const unsigned int rslot = __shfl_sync(FULL_MASK, slot, src);
            const uint32_t rc = rank_counts(a, rb, re);
            const int64_t gstart = ro + (int64_t)lane_excl(lane < a.n_rank ? rc : 0u);
            if (lane <= a.n_rank) a.gdir[(int64_t)rslot * (a.n_rank + 1) + lane] = gstart;
            place_ranked(a, rb, re, gstart);
        }
    }
}

// Bits of the compacted rows: every entry active, nothing past the last one.
__global__ void k_compact_bits(uint32_t *bits, const int64_t *total) {
    const int64_t m2 = *total;
    const int64_t words = (m2 + 31) / 32;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= words; i += stride) {
        uint32_t v = 0u;
        if (i < words) v = (i == words - 1 && (m2 & 31)) ? (1u << (uint32_t)(m2 & 31)) - 1u : ~0u;
        bits[i] = v;
    }
}

// Edge map of the final state when it is handed back without the final
// search: at an LCC fixpoint an entry between two active vertices is active
// iff their omegas are compatible (eta); entries cleared earlier stay
// cleared.  One warp per vertex, over the full rows.
__global__ void __launch_bounds__(256)
k_materialize_fix(int64_t n, const uint32_t *__restrict__ om, const int64_t *__restrict__ rp,
                  const int32_t *__restrict__ col, uint32_t *ebits, DevTmpl t) {
    __shared__ uint32_t sadj[kMaxT];
    for (int i = threadIdx.x; i < kMaxT; i += blockDim.x) sadj[i] = t.adj[i];
    __syncthreads();
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    for (int64_t v = gwarp; v < n; v += nwarps) {
        const int64_t beg = rp[v], end = rp[v + 1];
        if (beg == end) continue;
        const uint32_t wv = om[v];
        if (wv == 0u) {
            clear_row<32>(ebits, beg, end, lane);
            continue;
        }
        uint32_t nb = 0;
        for (uint32_t x = wv; x; x &= x - 1u) nb |= sadj[__ffs(x) - 1];
        for (int64_t w0 = beg >> 5; (w0 << 5) < end; w0++) {
            const int64_t e = (w0 << 5) + lane;
            const uint32_t word = ebits[w0];
            bool drop = false;
            if (e >= beg && e < end && ((word >> lane) & 1u)) drop = (__ldg(om + __ldg(col + e)) & nb) == 0u;
            const uint32_t dm = __ballot_sync(FULL_MASK, drop);
            if (dm && lane == 0) atomicAnd(&ebits[w0], ~dm);
        }
    }
}

// Zero the rows of the inactive vertices (one thread per vertex; the rows of
// vertices that were never active, or that a non-local check emptied, still
// carry bits the rounds never read).
__global__ void __launch_bounds__(256)
k_clear_dead_rows(int64_t n, const uint32_t *__restrict__ om, const int64_t *__restrict__ rp, uint32_t *ebits) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (om[v] == 0u) clear_row<1>(ebits, rp[v], rp[v + 1], 0);
}

// -------------------------------------------------------------------------
// Rooted injective embedding search (NLCC token walk, Alg. 6/7, and the
// final template-driven search, Remark 1).  One warp per root vertex, roots
// handed out dynamically; the warp walks the plan depth first, testing 32
// candidates at a time in parallel.
//
// Searches run only at LCC fixpoints.  There an entry (x, u) is active
// exactly when some template edge joins omega(x) and omega(u) (edge
// elimination has removed every other entry and keeps every such one), so a
// search needs adjacency and omega only: a candidate u for template vertex q
// next to a placed x with q_x in omega(x) is joined to x by an active entry
// iff u is a neighbour of x with q in omega(u).  Candidates are read from a
// copy of every row grouped by neighbour label (label, then id), so only the
// neighbours that carry label(q) are ever scanned.
// -------------------------------------------------------------------------

// A partial embedding of a search plan: positions 0..depth-1 placed.
constexpr int kItemMaxDepth = 7;
struct __align__(16) SearchItem {
    int32_t psi[kItemMaxDepth];
    int32_t hd;               // head | depth << 8
};

struct SearchArgs {
    const int64_t *rp;
    const int32_t *col;       // id-sorted rows (edge-bitmap indexing)
    const int32_t *dslot;     // compacted rows: slot of a live vertex in gdir
    const int64_t *gdir;      // per slot: start of each label group, then the row end
    int n_rank;               // distinct template labels (groups per compacted row)
    uint8_t lab_rank[256];    // rank of a template label among them
    const int64_t *rl;        // offsets of the rows the searches scan:
    const int32_t *lcol;      // the full rows grouped by neighbour label, ids ascending
    const uint8_t *nlab;      // inside a group, with nlab = label of lcol[e]; or
                              // compacted rows (ids ascending) with nlab = nullptr
    const uint32_t *om;
    const int32_t *roots;
    int64_t n_roots;
    unsigned long long *next_root;   // dynamic work counter
    const DevPlan *plans;     // plans[h] for each head h (NLCC) or plans[0] (final)
    uint32_t heads;           // NLCC: heads of the constraint; final: 1 << plans[0].q[0]
    uint32_t *sat;            // NLCC output: satisfied heads per vertex
    uint32_t *om_out;         // final: omega*
    uint32_t *eb_out;         // final: edge bitmap of E*
    RoundStats *st;
    uint64_t budget;          // windows per (root, head)
    uint64_t cap;             // final: stop past this many matches
    SearchItem *items;        // split search work: partial embeddings
    int64_t n_items;
    int64_t items_cap;
    SearchItem *spill;        // a search that has scanned spill_after windows hands its
    int64_t spill_cap;        // untried candidates on here as new items (0: never)
    uint64_t spill_after;
    int enum_heads;           // k_expand: 1 = final search (one head), 0 = NLCC
    const uint32_t *sat_seed; // existence passes: heads already known satisfied (nullable)
    // listing (mode kList): every match found gets an index from list_count;
    // the first list_cap are written as n0 vertex ids in template order; vcnt
    // and ecnt (nullable) count the matches per vertex and per CSR entry
    int32_t *list_out;
    uint64_t list_cap;
    int list_n0;
    unsigned long long *list_count;
    unsigned long long *vcnt;
    unsigned long long *ecnt;
};

constexpr int kMaxBack = 4;  // joins per level whose label group is kept in shared memory

struct WarpSearch {
    int32_t psi[kMaxT];
    int64_t pos[kMaxT];       // next window start inside the chosen label range
    int64_t end[kMaxT];
    int64_t wbase[kMaxT];     // start of the window the mask refers to
    uint32_t mask[kMaxT];     // untried valid candidates of that window
    uint32_t chk[kMaxT];      // further joins, looked up from scratch per candidate
    int nb[kMaxT];            // joins with a stored label group
    int64_t blo[kMaxT][kMaxBack], bhi[kMaxT][kMaxBack];
    const uint32_t *done_word;  // existence: the answer is known once this bit is set
    uint32_t done_bit;          // (by another warp's embedding); nullptr: never
    int head;                   // plan slot of the running item (spilled items keep it)
    // the first kJoinCache stored join groups of one level, copied to shared
    // memory when they are short: join tests at that level search them there
    int jc_level;
    int jc_len[2];
    int32_t jc[2][128];
    // the last match this warp marked (by plan position) and its plan: a
    // match found next in depth-first order usually differs from it only at
    // its last positions, and only what differs needs marking
    const DevPlan *last_plan;
    int32_t last[kMaxT];
    unsigned long long pub;     // matches of this warp already added to the global count
};
constexpr int kJoinCache = 2, kJoinCacheLen = 128;

// [lo, hi) of the label-L group in the label-grouped row of x: read from the
// group directory of the compacted rows, else found by binary search in the
// full rows.
__device__ __forceinline__ void label_range(const SearchArgs &a, int32_t x, uint32_t L, int64_t &lo, int64_t &hi) {
    if (a.gdir) {
        const int64_t *d = a.gdir + (int64_t)__ldg(a.dslot + x) * (a.n_rank + 1) + a.lab_rank[L];
        lo = __ldg(d);
        hi = __ldg(d + 1);
        return;
    }
    const int64_t b0 = a.rl[x], b1 = a.rl[x + 1];
    int64_t l = b0, h = b1;
    while (l < h) {
        int64_t m = (l + h) >> 1;
        if ((uint32_t)__ldg(a.nlab + m) < L) l = m + 1; else h = m;
    }
    lo = l;
    h = b1;
    while (l < h) {
        int64_t m = (l + h) >> 1;
        if ((uint32_t)__ldg(a.nlab + m) <= L) l = m + 1; else h = m;
    }
    hi = l;
}

// Is u (label L) a neighbour of x?  Binary search inside x's label-L group.
__device__ __forceinline__ bool adjacent(const SearchArgs &a, int32_t x, int32_t u, uint32_t L) {
    int64_t lo, hi;
    label_range(a, x, L, lo, hi);
    const int64_t stop = hi;
    while (lo < hi) {
        int64_t m = (lo + hi) >> 1;
        if (__ldg(a.lcol + m) < u) lo = m + 1; else hi = m;
    }
    return lo < stop && __ldg(a.lcol + lo) == u;
}

// CSR entry index of (x, y) in the id-sorted rows, or -1.
__device__ __forceinline__ int64_t find_entry(const int64_t *rp, const int32_t *col, int32_t x, int32_t y) {
    int64_t lo = rp[x], hi = rp[x + 1];
    const int64_t stop = hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(col + mid) < y) lo = mid + 1; else hi = mid;
    }
    return (lo < stop && __ldg(col + lo) == y) ? lo : -1;
}

// Open level d: among the placed neighbours of position d pick the one whose
// label group is shortest; scan that group, look the others up.
__device__ __forceinline__ void open_level(const SearchArgs &a, const DevPlan &P, WarpSearch &W, int d) {
    const int lane = (int)lane_id();
    // level d gets new groups: a join cache of this or a deeper level is stale
    if (lane == 0 && W.jc_level >= d) W.jc_level = -1;
    const uint32_t cm = P.nbr[d];
    const int cnt = __popc(cm);
    int64_t lo = 0, hi = 0, len = INT64_MAX;
    int j = -1;
    if (lane < cnt) {
        uint32_t m = cm;
        for (int i = 0; i < lane; i++) m &= m - 1u;
        j = __ffs(m) - 1;
        label_range(a, W.psi[j], P.lab[d], lo, hi);
        len = hi - lo;
    }
    int best = lane;
    for (int o = 16; o > 0; o >>= 1) {
        int64_t ol = __shfl_xor_sync(FULL_MASK, len, o);
        int ob = __shfl_xor_sync(FULL_MASK, best, o);
        if (ol < len || (ol == len && ob < best)) { len = ol; best = ob; }
    }
    // the other placed neighbours are joins: keep their label groups
    const int slot = lane < best ? lane : lane - 1;
    const bool join = lane < cnt && lane != best;
    if (join && slot < kMaxBack) {
        W.blo[d][slot] = lo;
        W.bhi[d][slot] = hi;
    }
    const uint32_t extra = __reduce_or_sync(FULL_MASK, (join && slot >= kMaxBack) ? (1u << j) : 0u);
    if (lane == best) {
        W.pos[d] = lo;
        W.end[d] = hi;
        W.mask[d] = 0u;
        W.chk[d] = extra;
        W.nb[d] = min(cnt - 1, kMaxBack);
    }
    __syncwarp();
}

// Returns true if an embedding exists (ENUM = false) / after enumerating all
// embeddings from this root (ENUM = true).  `over` is set when the window
// budget ran out; for existence the root is then reported as satisfied, which
// keeps the result a superset of the exact answer.
// Both directions of every template edge of the embedding in W.psi get their
// bit in the output edge map (id-sorted entry indices).
__device__ __forceinline__ void mark_edges(const SearchArgs &a, const DevPlan &P, const WarpSearch &W) {
    const int lane = (int)lane_id();
    for (int t = lane; t < P.n_marks; t += 32) {
        int32_t x = W.psi[P.mark_a[t]], y = W.psi[P.mark_b[t]];
        int64_t e1 = find_entry(a.rp, a.col, x, y);
        int64_t e2 = find_entry(a.rp, a.col, y, x);
        if (e1 >= 0) {
            uint32_t b1 = 1u << (uint32_t)(e1 & 31);
            if (!(a.eb_out[e1 >> 5] & b1)) atomicOr(&a.eb_out[e1 >> 5], b1);
        }
        if (e2 >= 0) {
            uint32_t b2 = 1u << (uint32_t)(e2 & 31);
            if (!(a.eb_out[e2 >> 5] & b2)) atomicOr(&a.eb_out[e2 >> 5], b2);
        }
    }
    __syncwarp();
}

// A match found by a listing search: stored (if its index is below the cap)
// and counted on every vertex and on both entries of every edge it uses.
__device__ __forceinline__ void list_embedding(const SearchArgs &a, const DevPlan &P, const WarpSearch &W) {
    const int lane = (int)lane_id();
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(a.list_count, 1ull);
    idx = __shfl_sync(FULL_MASK, idx, 0);
    if (lane < P.k) {
        const int32_t x = W.psi[lane];
        if (idx < a.list_cap) a.list_out[idx * (unsigned long long)a.list_n0 + (unsigned long long)P.q[lane]] = x;
        if (a.vcnt) atomicAdd(&a.vcnt[x], 1ull);
    }
    if (a.ecnt) {
        for (int t = lane; t < P.n_marks; t += 32) {
            const int32_t x = W.psi[P.mark_a[t]], y = W.psi[P.mark_b[t]];
            const int64_t e1 = find_entry(a.rp, a.col, x, y), e2 = find_entry(a.rp, a.col, y, x);
            if (e1 >= 0) atomicAdd(&a.ecnt[e1], 1ull);
            if (e2 >= 0) atomicAdd(&a.ecnt[e2], 1ull);
        }
    }
    __syncwarp();
}

// Is the entry e of the scanned label group a valid image u for position d?
// Its omega must hold q_d, it must differ from earlier same-label images, and
// it must be joined to every other placed neighbour of position d.
// Warp-uniform: make the join cache hold level d's first stored groups.
__device__ __forceinline__ void join_cache(const SearchArgs &a, WarpSearch &W, int d) {
    if (W.jc_level == d) return;
    const int lane = (int)lane_id();
    const int nb = min(W.nb[d], kJoinCache);
    for (int b = 0; b < kJoinCache; b++) {
        const int64_t lo = W.blo[d][b], len = W.bhi[d][b] - lo;
        const bool fits = b < nb && len <= kJoinCacheLen;
        if (fits)
            for (int i = lane; i < (int)len; i += 32) W.jc[b][i] = __ldg(a.lcol + lo + i);
        if (lane == 0) W.jc_len[b] = fits ? (int)len : -1;
    }
    if (lane == 0) W.jc_level = d;
    __syncwarp();
}

__device__ __forceinline__ bool test_candidate(const SearchArgs &a, const DevPlan &P, WarpSearch &W,
                                               int d, int64_t e, int64_t end, int32_t &u) {
    if (W.nb[d] > 0) join_cache(a, W, d);
    u = -1;
    if (e >= end) return false;
    u = __ldg(a.lcol + e);
    if (!((__ldg(a.om + u) >> P.q[d]) & 1u)) return false;
    for (uint32_t sm = P.same[d]; sm; sm &= sm - 1u)
        if (W.psi[__ffs(sm) - 1] == u) return false;
    for (int b = 0; b < W.nb[d]; b++) {
        if (b < kJoinCache && W.jc_len[b] >= 0) {
            int lo = 0, hi = W.jc_len[b];
            const int stop = hi;
            while (lo < hi) {
                const int m2 = (lo + hi) >> 1;
                if (W.jc[b][m2] < u) lo = m2 + 1; else hi = m2;
            }
            if (!(lo < stop && W.jc[b][lo] == u)) return false;
            continue;
        }
        int64_t lo = W.blo[d][b], hi = W.bhi[d][b];
        const int64_t stop = hi;
        while (lo < hi) {
            int64_t m2 = (lo + hi) >> 1;
            if (__ldg(a.lcol + m2) < u) lo = m2 + 1; else hi = m2;
        }
        if (!(lo < stop && __ldg(a.lcol + lo) == u)) return false;
    }
    for (uint32_t bm = W.chk[d]; bm; bm &= bm - 1u)
        if (!adjacent(a, W.psi[__ffs(bm) - 1], u, P.lab[d])) return false;
    return true;
}

// omega*(psi(i)) gets q_i for every position of the match in W.psi.
__device__ __forceinline__ void mark_vertices(const SearchArgs &a, const DevPlan &P, const WarpSearch &W) {
    const int lane = (int)lane_id();
    if (lane < P.k) {
        const int32_t x = W.psi[lane];
        const uint32_t bit = 1u << P.q[lane];
        if (!(a.om_out[x] & bit)) atomicOr(&a.om_out[x], bit);
    }
    __syncwarp();
}

// Mark a match found by a marking enumeration: every (vertex, template
// vertex) pair and both entries of every template edge, skipping those the
// warp's previous match (same plan) already marked: marks are only ever set,
// so a pair or an edge whose positions hold the same vertices as in that
// match is marked already.
__device__ __forceinline__ void mark_match(const SearchArgs &a, const DevPlan &P, WarpSearch &W) {
    const int lane = (int)lane_id();
    const bool same_plan = W.last_plan == &P;
    if (lane < P.k) {
        const int32_t x = W.psi[lane];
        if (!(same_plan && W.last[lane] == x)) {
            const uint32_t bit = 1u << P.q[lane];
            if (!(a.om_out[x] & bit)) atomicOr(&a.om_out[x], bit);
        }
    }
    for (int t = lane; t < P.n_marks; t += 32) {
        const int pa = P.mark_a[t], pb = P.mark_b[t];
        const int32_t x = W.psi[pa], y = W.psi[pb];
        if (same_plan && W.last[pa] == x && W.last[pb] == y) continue;
        const int64_t e1 = find_entry(a.rp, a.col, x, y);
        const int64_t e2 = find_entry(a.rp, a.col, y, x);
        if (e1 >= 0) {
            const uint32_t b1 = 1u << (uint32_t)(e1 & 31);
            if (!(a.eb_out[e1 >> 5] & b1)) atomicOr(&a.eb_out[e1 >> 5], b1);
        }
        if (e2 >= 0) {
            const uint32_t b2 = 1u << (uint32_t)(e2 & 31);
            if (!(a.eb_out[e2 >> 5] & b2)) atomicOr(&a.eb_out[e2 >> 5], b2);
        }
    }
    __syncwarp();
    if (lane < P.k) W.last[lane] = W.psi[lane];
    if (lane == 0) W.last_plan = &P;
    __syncwarp();
}

// Search modes: does an embedding exist / count the embeddings / count them
// and mark the vertices and edges of every one / count them and list them.
constexpr int kExist = 0, kCount = 1, kMark = 2, kList = 3;

// Hand the rest of a long search to other warps: for every open level L
// (d0..d) each untried candidate c -- the remaining bits of the level's
// tested window and every valid entry of its untested range -- becomes an item
// (psi[0..L-1], c) of depth L+1 in the spill list; for counting, candidates
// of the last position are counted here instead.  The items are counted
// first and written only if they all fit.  Returns false (the search goes on
// where it is) when they do not.  Reservations only ever add to the counter:
// the successful ones are exactly those ending at or below the capacity, and
// they fill the list up to the lowest start of a failed one (spill_stop), so
// the list is valid below min(counter, spill_stop).
template <int MODE>
__device__ bool spill(const SearchArgs &a, const DevPlan &P, WarpSearch &W, int d0, int d,
                      unsigned long long &matches) {
    const int lane = (int)lane_id();
    const uint32_t below = (1u << lane) - 1u;
    const int k = P.k;
    unsigned long long total = 0, direct = 0;
    for (int L = d0; L <= d; L++) {
        unsigned long long cnt = (unsigned long long)__popc(W.mask[L]);
        for (int64_t pos = W.pos[L]; pos < W.end[L]; pos += 32) {
            int32_t u;
            const bool ok = test_candidate(a, P, W, L, pos + lane, W.end[L], u);
            cnt += (unsigned long long)__popc(__ballot_sync(FULL_MASK, ok));
        }
        if (MODE == kCount && L == k - 1) direct += cnt; else total += cnt;
    }
    unsigned long long base = 0;
    unsigned int fits = 1;
    if (lane == 0 && total) {
        if (*(volatile const unsigned int *)&a.st->n_spill >= (unsigned long long)a.spill_cap) {
            fits = 0;                               // full already: do not grow the counter
        } else {
            base = atomicAdd(&a.st->n_spill, (unsigned int)total);
            if (base + total > (unsigned long long)a.spill_cap) {
                atomicMin(&a.st->spill_stop, (unsigned int)base);
                fits = 0;
            }
        }
    }
    if (!__shfl_sync(FULL_MASK, fits, 0)) return false;
    base = __shfl_sync(FULL_MASK, base, 0);
    for (int L = d0; L <= d; L++) {
        if (MODE == kCount && L == k - 1) continue;
        SearchItem si;
        for (int j = 0; j < kItemMaxDepth; j++) si.psi[j] = j < L ? W.psi[j] : 0;
        si.hd = W.head | ((L + 1) << 8);
        const uint32_t m = W.mask[L];
        if ((m >> lane) & 1u) {
            si.psi[L] = __ldg(a.lcol + W.wbase[L] + lane);
            a.spill[base + __popc(m & below)] = si;
        }
        base += (unsigned long long)__popc(m);
        for (int64_t pos = W.pos[L]; pos < W.end[L]; pos += 32) {
            int32_t u;
            const bool ok = test_candidate(a, P, W, L, pos + lane, W.end[L], u);
            const uint32_t vm = __ballot_sync(FULL_MASK, ok);
            if (ok) {
                si.psi[L] = u;
                a.spill[base + __popc(vm & below)] = si;
            }
            base += (unsigned long long)__popc(vm);
        }
    }
    matches += direct;
    __syncwarp();
    return true;
}

// Depth-first search from positions 0..d0-1 already placed in W.psi.
template <int MODE>
__device__ bool search_from(const SearchArgs &a, const DevPlan &P, int d0, WarpSearch &W,
                            unsigned long long &entries, unsigned long long &matches, bool &over) {
    const int lane = (int)lane_id();
    const int k = P.k;
    uint64_t used = 0;
    if (d0 >= k) {                                  // the placed prefix is already a full map
        if (MODE == kExist) return true;
        matches++;
        if (MODE == kMark) mark_match(a, P, W);
        if (MODE == kList) list_embedding(a, P, W);
        return false;
    }
    open_level(a, P, W, d0);
    int d = d0;
    while (d >= d0) {
        const uint32_t m = W.mask[d];
        if (m == 0u) {
            const int64_t pos = W.pos[d], end = W.end[d];
            if (pos >= end) { d--; continue; }
            if (++used > a.budget) { over = true; return MODE == kExist; }
            if ((used & 31u) == 0u) {
                // every 32 windows: has another warp answered this existence
                // question already, or has the count run past its cap?
                unsigned int stop = 0;
                if (lane == 0) {
                    if (MODE == kExist) {
                        stop = W.done_word && (*(volatile const uint32_t *)W.done_word & W.done_bit);
                    } else if (MODE == kCount || MODE == kMark) {
                        // counting (and marking) stops as soon as the total passes
                        // the cap: publish this warp's new matches and read the
                        // total, so that no warp runs on to the cap by itself
                        const unsigned long long d = matches - W.pub;
                        const unsigned long long tot =
                            d ? atomicAdd(&a.st->matches, d) + d : *(volatile const unsigned long long *)&a.st->matches;
                        W.pub = matches;
                        stop = tot > a.cap || *(volatile const unsigned int *)&a.st->overflow;
                    } else {
                        stop = matches > a.cap || *(volatile const unsigned int *)&a.st->overflow;
                    }
                }
                if (__shfl_sync(FULL_MASK, stop, 0)) {
                    // past the cap (the matches are published already, so the
                    // caller's batch-end check would not see it)
                    if (MODE == kCount || MODE == kMark) over = true;
                    return false;
                }
            }
            if (a.spill_after && used > a.spill_after && d < kItemMaxDepth &&
                spill<MODE>(a, P, W, d0, d, matches))
                return false;                       // the rest runs as new items
            entries += (unsigned long long)min((int64_t)32, end - pos);
            int32_t u;
            const bool ok = test_candidate(a, P, W, d, pos + lane, end, u);
            const uint32_t vm = __ballot_sync(FULL_MASK, ok);
            if (MODE == kCount && d == k - 1) {
                // counting: every valid image of the last position completes a match
                matches += (unsigned long long)__popc(vm);
                if (lane == 0) { W.mask[d] = 0u; W.pos[d] = pos + 32; }
                __syncwarp();
                continue;
            }
            if (lane == 0) { W.mask[d] = vm; W.wbase[d] = pos; W.pos[d] = pos + 32; }
            __syncwarp();
            continue;
        }
        const int b = __ffs(m) - 1;
        if (lane == 0) { W.mask[d] = m & (m - 1u); W.psi[d] = __ldg(a.lcol + W.wbase[d] + b); }
        __syncwarp();
        if (d == k - 1) {
            if (MODE == kExist) return true;
            matches++;                              // kMark / kList (counting never stores last-level masks)
            if (MODE == kList) list_embedding(a, P, W);
            else mark_match(a, P, W);
            continue;
        }
        d++;
        open_level(a, P, W, d);
    }
    return false;
}

__device__ __forceinline__ int64_t grab_root(const SearchArgs &a) {
    unsigned long long r = 0;
    if (lane_id() == 0) r = atomicAdd(a.next_root, 1ull);
    return (int64_t)__shfl_sync(FULL_MASK, r, 0);
}

__global__ void __launch_bounds__(128)
k_nlcc_search(SearchArgs a) {
    __shared__ WarpSearch ws[4];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    WarpSearch &W = ws[wib];
    unsigned long long entries = 0, matches = 0;
    bool over = false;
    for (int64_t it = grab_root(a); it < a.n_roots; it = grab_root(a)) {
        const int32_t v = a.roots[it];
        const uint32_t seed = a.sat_seed ? __ldg(a.sat_seed + v) : 0u;
        const uint32_t hv = __ldg(a.om + v) & a.heads & ~seed;
        uint32_t sat = seed;
        for (uint32_t hm = hv; hm; hm &= hm - 1u) {
            const int h = __ffs(hm) - 1;
            if (lane == 0) { W.psi[0] = v; W.done_word = nullptr; }
            __syncwarp();
            if (search_from<kExist>(a, a.plans[h], 1, W, entries, matches, over)) sat |= 1u << h;
            __syncwarp();
        }
        if (lane == 0) a.sat[v] = sat;
    }
    // entries, tokens and over are identical in every lane of the warp
    if (lane == 0) {
        if (entries) atomicAdd(&a.st->windows, entries);
        if (over) atomicOr(&a.st->overflow, 1u);
    }
}

template <int MODE>
__global__ void __launch_bounds__(128)
k_final_search(SearchArgs a) {
    __shared__ WarpSearch ws[4];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    WarpSearch &W = ws[wib];
    if (lane == 0) { W.last_plan = nullptr; W.pub = 0; }
    __syncwarp();
    unsigned long long entries = 0, matches = 0;
    bool over = false;
    for (int64_t it = grab_root(a); it < a.n_roots; it = grab_root(a)) {
        unsigned int stop = 0;
        if (lane == 0) stop = *(volatile unsigned int *)&a.st->overflow;
        if (__shfl_sync(FULL_MASK, stop, 0)) break;
        const int32_t v = a.roots[it];
        if (lane == 0) { W.psi[0] = v; W.done_word = nullptr; }
        __syncwarp();
        search_from<MODE>(a, a.plans[0], 1, W, entries, matches, over);
        __syncwarp();
        const unsigned long long pub = W.pub;     // read by every lane before lane 0 moves it
        __syncwarp();
        if (matches != pub) {
            unsigned long long tot = 0;
            if (lane == 0) {
                tot = atomicAdd(&a.st->matches, matches - pub) + (matches - pub);
                W.pub = matches;
            }
            tot = __shfl_sync(FULL_MASK, tot, 0);
            __syncwarp();
            if (tot > a.cap) over = true;
        }
        if (over) {
            if (lane == 0) atomicOr(&a.st->overflow, 1u);
            break;
        }
    }
    if (lane == 0 && entries) atomicAdd(&a.st->windows, entries);
}

// Split search work by the first level: every (root, head) becomes one item per
// candidate for position 1, so expensive roots spread over many warps.
__global__ void __launch_bounds__(256)
k_expand(SearchArgs a) {
    __shared__ SearchItem sbuf[8][32];
    __shared__ int scnt[8];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    if (lane == 0) scnt[wib] = 0;
    __syncthreads();
    WarpBuf<SearchItem> b{sbuf[wib], &scnt[wib], a.items, &a.st->n_items};
    b.cap = (unsigned long long)a.items_cap;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long entries = 0, tokens = 0;
    for (int64_t it = gwarp; it < a.n_roots; it += nwarps) {
        const int32_t v = a.roots[it];
        const uint32_t seed = (!a.enum_heads && a.sat_seed) ? __ldg(a.sat_seed + v) : 0u;
        const uint32_t hv = a.enum_heads ? a.heads : (__ldg(a.om + v) & a.heads & ~seed);
        if (!a.enum_heads && lane == 0) a.sat[v] = seed;
        tokens += (unsigned long long)__popc(hv);
        for (uint32_t hm = hv; hm; hm &= hm - 1u) {
            const int h = __ffs(hm) - 1;
            const DevPlan &P = a.plans[a.enum_heads ? 0 : h];
            const int q1 = P.q[1];
            int64_t lo, hi;
            label_range(a, v, P.lab[1], lo, hi);
            entries += (unsigned long long)(hi - lo);
            for (int64_t base = lo; base < hi; base += 32) {
                const int64_t e = base + lane;
                bool ok = false;
                int32_t u = -1;
                if (e < hi) {
                    u = __ldg(a.lcol + e);
                    ok = ((__ldg(a.om + u) >> q1) & 1u) && !((P.same[1] & 1u) && u == v);
                }
                SearchItem si;
                si.psi[0] = v;
                si.psi[1] = u;
                si.hd = h | (2 << 8);
                b.push(ok, si);
            }
        }
    }
    b.flush();
    if (lane == 0) {
        if (entries) atomicAdd(&a.st->windows, entries);
        if (tokens) atomicAdd(&a.st->tokens, tokens);
    }
}

// When there are too few items to fill the GPU, place one more position:
// every input item of depth D becomes one item per valid image of position D.
// Items that already place every position pass through.
__global__ void __launch_bounds__(128)
k_expand_next(SearchArgs a, const SearchItem *in, int64_t n_in) {
    __shared__ WarpSearch ws[4];
    __shared__ SearchItem sbuf[4][32];
    __shared__ int scnt[4];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    WarpSearch &W = ws[wib];
    if (lane == 0) scnt[wib] = 0;
    __syncthreads();
    WarpBuf<SearchItem> b{sbuf[wib], &scnt[wib], a.items, &a.st->n_items};
    b.cap = (unsigned long long)a.items_cap;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long entries = 0;
    for (int64_t it = gwarp; it < n_in; it += nwarps) {
        const SearchItem item = in[it];
        const int h = item.hd & 0xff, depth = item.hd >> 8;
        const DevPlan &P = a.plans[a.enum_heads ? 0 : h];
        if (depth >= P.k || depth >= kItemMaxDepth) {
            b.push(lane == 0, item);
            continue;
        }
        if (lane < depth) W.psi[lane] = item.psi[lane];
        __syncwarp();
        open_level(a, P, W, depth);
        const int64_t lo = W.pos[depth], hi = W.end[depth];
        entries += (unsigned long long)(hi - lo);
        for (int64_t base = lo; base < hi; base += 32) {
            int32_t u;
            const bool ok = test_candidate(a, P, W, depth, base + lane, hi, u);
            SearchItem si = item;
            si.psi[depth] = u;
            si.hd = h | ((depth + 1) << 8);
            b.push(ok, si);
        }
    }
    b.flush();
    if (lane == 0 && entries) atomicAdd(&a.st->windows, entries);
}

__device__ __forceinline__ int64_t grab_items(const SearchArgs &a, int batch) {
    unsigned long long r = 0;
    if (lane_id() == 0) r = atomicAdd(a.next_root, (unsigned long long)batch);
    return (int64_t)__shfl_sync(FULL_MASK, r, 0);
}

constexpr int kItemBatch = 4;
constexpr int kMaxPlans = 64;      // plan slots (heads, or oriented template edges)
constexpr uint64_t kMarkCap = 1ull << 20;   // matches one marking enumeration handles
constexpr uint64_t kFewMatches = 1ull << 16;   // marked during the first enumeration itself
// Below this many first-level items the searches place position 2 as well.
constexpr int64_t kExpandBelow = 16384;

__global__ void __launch_bounds__(128)
k_nlcc_items(SearchArgs a) {
    __shared__ WarpSearch ws[4];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    WarpSearch &W = ws[wib];
    unsigned long long entries = 0, matches = 0;
    bool over = false;
    for (int64_t it0 = grab_items(a, kItemBatch); it0 < a.n_items; it0 = grab_items(a, kItemBatch)) {
        const int64_t it1 = min(a.n_items, it0 + kItemBatch);
        for (int64_t it = it0; it < it1; it++) {
            const SearchItem item = a.items[it];
            const int h = item.hd & 0xff, depth = item.hd >> 8;
            const uint32_t bit = 1u << h;
            uint32_t done = 0;                                       // satisfied by another item?
            if (lane == 0) done = *(volatile uint32_t *)&a.sat[item.psi[0]] & bit;
            if (__shfl_sync(FULL_MASK, done, 0)) continue;
            if (lane < depth) W.psi[lane] = item.psi[lane];
            if (lane == 0) { W.done_word = &a.sat[item.psi[0]]; W.done_bit = bit; W.head = h; }
            __syncwarp();
            bool ran_out = false;
            if (search_from<kExist>(a, a.plans[h], depth, W, entries, matches, ran_out)) {
                const DevPlan &P = a.plans[h];
                if (ran_out) {
                    // budget exhausted: keep the head (a superset of the exact answer)
                    if (lane == 0) atomicOr(&a.sat[item.psi[0]], bit);
                } else {
                    // the embedding found satisfies every head it places, not only h
                    if (lane < P.k) {
                        const int q = P.q[lane];
                        if ((a.heads >> q) & 1u) atomicOr(&a.sat[W.psi[lane]], 1u << q);
                    }
                    if (a.eb_out) mark_edges(a, P, W);
                }
            }
            over = over || ran_out;
            __syncwarp();
        }
    }
    if (lane == 0) {
        if (entries) atomicAdd(&a.st->windows, entries);
        if (over) atomicOr(&a.st->overflow, 1u);
    }
}

template <int MODE>
__global__ void __launch_bounds__(128)
k_final_items(SearchArgs a) {
    __shared__ WarpSearch ws[4];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    WarpSearch &W = ws[wib];
    if (lane == 0) { W.last_plan = nullptr; W.pub = 0; }
    __syncwarp();
    unsigned long long entries = 0, matches = 0;
    bool over = false;
    for (int64_t it0 = grab_items(a, kItemBatch); it0 < a.n_items; it0 = grab_items(a, kItemBatch)) {
        unsigned int stop = 0;
        if (lane == 0) stop = *(volatile unsigned int *)&a.st->overflow;
        if (__shfl_sync(FULL_MASK, stop, 0)) break;
        const int64_t it1 = min(a.n_items, it0 + kItemBatch);
        for (int64_t it = it0; it < it1 && !over; it++) {
            const SearchItem item = a.items[it];
            const int depth = item.hd >> 8;
            if (lane < depth) W.psi[lane] = item.psi[lane];
            if (lane == 0) { W.done_word = nullptr; W.head = item.hd & 0xff; }
            __syncwarp();
            search_from<MODE>(a, a.plans[0], depth, W, entries, matches, over);
            __syncwarp();
        }
        const unsigned long long pub = W.pub;     // read by every lane before lane 0 moves it
        __syncwarp();
        if (matches != pub) {
            unsigned long long tot = 0;
            if (lane == 0) {
                tot = atomicAdd(&a.st->matches, matches - pub) + (matches - pub);
                W.pub = matches;
            }
            tot = __shfl_sync(FULL_MASK, tot, 0);
            __syncwarp();
            if (tot > a.cap) over = true;
        }
        if (over) {
            if (lane == 0) atomicOr(&a.st->overflow, 1u);
            break;
        }
    }
    if (lane == 0 && entries) atomicAdd(&a.st->windows, entries);
}

// Edge pass of the final step: every entry (x, y), x < y, whose ends hold
// omega* sets joined by some template edge and that no embedding found so far
// has marked becomes one item per orientation (a, b) of a template edge with
// a in omega*(x), b in omega*(y); plans[o] is rooted at that oriented edge.
struct EdgeTab {
    int n;                       // oriented template edges in this pass
    int8_t a[32], b[32];
};

__global__ void __launch_bounds__(256)
k_edge_items(SearchArgs a, EdgeTab tab) {
    __shared__ SearchItem sbuf[8][32];
    __shared__ int scnt[8];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    if (lane == 0) scnt[wib] = 0;
    __syncthreads();
    WarpBuf<SearchItem> b{sbuf[wib], &scnt[wib], a.items, &a.st->n_items};
    b.cap = (unsigned long long)a.items_cap;
    // one block per root: its warps take every (blockDim/32)-th window of the
    // root's row, so the rows of hubs are split across the block
    const int nwb = (int)(blockDim.x >> 5);
    for (int64_t it = blockIdx.x; it < a.n_roots; it += gridDim.x) {
        const int32_t x = a.roots[it];
        const uint32_t wx = __ldg(a.om + x);
        const int64_t beg = a.rp[x], end = a.rp[x + 1];
        for (int64_t base = beg + (int64_t)wib * 32; base < end; base += (int64_t)nwb * 32) {
            const int64_t e = base + lane;
            int32_t y = -1;
            uint32_t wy = 0u;
            if (e < end) {
                y = __ldg(a.col + e);
                if (y > x && !((a.eb_out[e >> 5] >> (uint32_t)(e & 31)) & 1u)) wy = __ldg(a.om + y);
            }
            // most neighbours of a hub are outside omega*: nothing to push
            if (!__any_sync(FULL_MASK, wy != 0u)) continue;
            for (int o = 0; o < tab.n; o++) {
                const bool ok = wy && ((wx >> tab.a[o]) & 1u) && ((wy >> tab.b[o]) & 1u);
                SearchItem si;
                for (int j = 0; j < kItemMaxDepth; j++) si.psi[j] = 0;
                si.psi[0] = x;
                si.psi[1] = y;
                si.hd = o | (2 << 8);
                b.push(ok, si);
            }
        }
    }
    b.flush();
}

__global__ void __launch_bounds__(128)
k_edge_search(SearchArgs a) {
    __shared__ WarpSearch ws[4];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    WarpSearch &W = ws[wib];
    unsigned long long entries = 0, matches = 0;
    bool over = false;
    for (int64_t it0 = grab_items(a, kItemBatch); it0 < a.n_items; it0 = grab_items(a, kItemBatch)) {
        const int64_t it1 = min(a.n_items, it0 + kItemBatch);
        for (int64_t it = it0; it < it1; it++) {
            const SearchItem item = a.items[it];
            const int o = item.hd & 0xff, depth = item.hd >> 8;
            // the entry of the item's template edge: psi[0], psi[1] are its
            // ends (items handed on by long searches keep them)
            int64_t e = 0;
            if (lane == 0) e = find_entry(a.rp, a.col, item.psi[0], item.psi[1]);
            e = __shfl_sync(FULL_MASK, e, 0);
            uint32_t done = 0;                          // marked by an embedding found meanwhile?
            if (lane == 0) done = (*(volatile uint32_t *)&a.eb_out[e >> 5] >> (uint32_t)(e & 31)) & 1u;
            if (__shfl_sync(FULL_MASK, done, 0)) continue;
            if (lane < depth) W.psi[lane] = item.psi[lane];
            if (lane == 0) { W.done_word = &a.eb_out[e >> 5]; W.done_bit = 1u << (uint32_t)(e & 31); W.head = o; }
            __syncwarp();
            const DevPlan &P = a.plans[o];
            bool ran_out = false;
            if (search_from<kExist>(a, P, depth, W, entries, matches, ran_out)) {
                if (!ran_out) {
                    mark_edges(a, P, W);
                } else if (lane == 0) {
                    // budget exhausted: keep the edge (a superset of the exact answer)
                    const int64_t e2 = find_entry(a.rp, a.col, item.psi[1], item.psi[0]);
                    atomicOr(&a.eb_out[e >> 5], 1u << (uint32_t)(e & 31));
                    if (e2 >= 0) atomicOr(&a.eb_out[e2 >> 5], 1u << (uint32_t)(e2 & 31));
                }
            }
            over = over || ran_out;
        }
    }
    if (lane == 0) {
        if (entries) atomicAdd(&a.st->windows, entries);
        if (over) atomicOr(&a.st->overflow, 1u);
    }
}

// omega* of the roots from their satisfied bits.
__global__ void k_sat_to_omega(const int32_t *roots, int64_t n_roots, const uint32_t *sat, const uint32_t *om,
                               uint32_t *om_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_roots; i += stride) {
        const int32_t v = roots[i];
        om_out[v] = sat[v] & om[v];
    }
}

// Label of the neighbour at every CSR entry (sort keys for the grouped rows).
__global__ void __launch_bounds__(256)
k_gather_labels(int64_t m, const int32_t *__restrict__ col, const uint8_t *__restrict__ lab, uint8_t *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        out[e] = __ldg(lab + __ldg(col + e));
}

// Label-grouped rows (once per graph): every row's entries stably sorted by
// their neighbour's label, by a counting sort per row.  One warp per row: a
// histogram of the row's labels in shared memory (256 bins), its exclusive
// scan, then the entries in order, 32 at a time, each placed at its label's
// next slot (lanes with equal labels are ranked by lane order, so equal
// labels keep their order).  keys: the labels in entry order, or NULL to
// gather them.
__device__ __forceinline__ uint32_t row_label(const uint8_t *keys, const int32_t *col, const uint8_t *lab,
                                              int64_t e, int64_t end) {
    if (e >= end) return 256u;                    // no entry: a value no label has
    return keys ? (uint32_t)keys[e] : (uint32_t)__ldg(lab + __ldg(col + e));
}

__global__ void __launch_bounds__(256)
k_label_sort(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
             const uint8_t *__restrict__ lab, const uint8_t *__restrict__ keys, uint8_t *nlab, int32_t *lcol) {
    __shared__ uint32_t bins[8][256];
    const int wib = threadIdx.x >> 5;
    const int lane = (int)lane_id();
    uint32_t *h = bins[wib];
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = gw; v < n; v += nw) {
        const int64_t beg = rp[v], end = rp[v + 1];
        if (end <= beg) continue;
#pragma unroll
        for (int k = 0; k < 8; k++) h[lane * 8 + k] = 0u;
        __syncwarp();
        for (int64_t c = beg; c < end; c += 32) {
            const uint32_t L = row_label(keys, col, lab, c + lane, end);
            const uint32_t grp = __match_any_sync(FULL_MASK, L);
            if (L < 256u && lane == __ffs(grp) - 1) h[L] += (uint32_t)__popc(grp);
            __syncwarp();
        }
        // exclusive scan of the 256 bins: 8 per lane, then across lanes
        uint32_t loc[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) { loc[k] = sum; sum += h[lane * 8 + k]; }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t excl = incl - sum;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) h[lane * 8 + k] = excl + loc[k];
        __syncwarp();
        for (int64_t c = beg; c < end; c += 32) {
            const int64_t e = c + lane;
            const uint32_t L = row_label(keys, col, lab, e, end);
            const uint32_t grp = __match_any_sync(FULL_MASK, L);
            if (L < 256u) {
                const uint32_t below = grp & ((1u << lane) - 1u);
                const int64_t pos = beg + (int64_t)h[L] + __popc(below);
                nlab[pos] = (uint8_t)L;
                lcol[pos] = __ldg(col + e);
            }
            __syncwarp();
            if (L < 256u && lane == __ffs(grp) - 1) h[L] += (uint32_t)__popc(grp);
            __syncwarp();
        }
    }
}

// Exclusive prefix sum of n int64 values, in three passes: each block scans
// a tile of kScanTile values and writes its total, one block scans the tile
// totals (in tiles of its own, carrying the running sum), and each tile adds
// its offset.
constexpr int kScanTile = 2048;                 // 256 threads x 8 values

__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t &total) {
    __shared__ int64_t warp_tot[8];
    const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wib] = incl;
    __syncthreads();
    int64_t before = 0;
    total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        if (w < wib) before += warp_tot[w];
        total += warp_tot[w];
    }
    __syncthreads();
    return before + incl - x;
}

__global__ void __launch_bounds__(256)
k_scan_tiles(int64_t n, const int64_t *__restrict__ in, int64_t *out, int64_t *tile_sum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * 8;
    int64_t v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t run = block_excl_scan(s, total);
#pragma unroll
    for (int k = 0; k < 8; k++) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256)
k_scan_sums(int64_t tiles, int64_t *tile_sum) {
    int64_t carry = 0;
    for (int64_t t0 = 0; t0 < tiles; t0 += kScanTile) {
        const int64_t base = t0 + (int64_t)threadIdx.x * 8;
        int64_t v[8], s = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            v[k] = base + k < tiles ? tile_sum[base + k] : 0;
            s += v[k];
        }
        int64_t total;
        int64_t run = carry + block_excl_scan(s, total);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (base + k < tiles) tile_sum[base + k] = run;
            run += v[k];
        }
        carry += total;
    }
}

__global__ void __launch_bounds__(256)
k_scan_add(int64_t n, int64_t *out, const int64_t *__restrict__ tile_off) {
    const int64_t off = tile_off[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
        if (base + i < n) out[base + i] += off;
}

// Roots of a search: every vertex whose omega meets `heads`.
__global__ void __launch_bounds__(256)
k_collect_roots(int64_t n, const uint32_t *__restrict__ om, uint32_t heads, int32_t *roots, RoundStats *st) {
    __shared__ int32_t sbuf[8][32];
    __shared__ int scnt[8];
    const int wib = threadIdx.x >> 5;
    if (lane_id() == 0) scnt[wib] = 0;
    __syncthreads();
    WarpBuf<int32_t> b{sbuf[wib], &scnt[wib], roots, &st->n_roots};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_pad = (n + 31) & ~(int64_t)31;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_pad; v += stride) {
        bool p = v < n && (__ldg(om + v) & heads);
        b.push(p, (int32_t)v);
    }
    b.flush();
}

// Alg. 6 lines 5-11: issuers whose token failed lose the head; a vertex whose
// omega empties is eliminated with its edges.  Both omega buffers are kept
// equal (they are equal at an LCC fixpoint).
__global__ void __launch_bounds__(256)
k_nlcc_apply(const int32_t *__restrict__ roots, int64_t n_roots, uint32_t heads,
             const uint32_t *__restrict__ sat, uint32_t *om0, uint32_t *om1,
             const int64_t *__restrict__ rp, uint32_t *ebits, RoundStats *st) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t changed = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_roots; i += stride) {
        const int32_t v = roots[i];
        const uint32_t w = om0[v];
        const uint32_t nw = w & ~(heads & ~sat[v]);
        if (nw != w) {
            om0[v] = nw;
            om1[v] = nw;
            changed = 1u;
            if (nw == 0u) clear_row<1>(ebits, rp[v], rp[v + 1], 0);
        }
    }
    if (__any_sync(FULL_MASK, changed) && lane_id() == 0) atomicOr(&st->changed, 1u);
}

__device__ __forceinline__ bool ebit(const uint32_t *eb, int64_t e) {
    return (eb[e >> 5] >> (uint32_t)(e & 31)) & 1u;
}

// Make the edge map exact everywhere (used when it is handed back without the
// final search): rows of inactive vertices are zeroed, and in live rows the
// bits of entries whose other end is inactive are cleared.  One warp per vertex.
__global__ void __launch_bounds__(256)
k_materialize(int64_t n, const uint32_t *__restrict__ om, const int64_t *__restrict__ rp,
              const int32_t *__restrict__ col, uint32_t *ebits) {
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    for (int64_t v = gwarp; v < n; v += nwarps) {
        const int64_t beg = rp[v], end = rp[v + 1];
        if (beg == end) continue;
        if (om[v] == 0u) {
            clear_row<32>(ebits, beg, end, lane);
            continue;
        }
        for (int64_t e = beg + lane; e < end; e += 32) {
            if (ebit(ebits, e) && om[col[e]] == 0u)
                atomicAnd(&ebits[e >> 5], ~(1u << (uint32_t)(e & 31)));
        }
    }
}

// Both narrow copies of omega from the current omega (an LCC phase starts
// with the two omega buffers equal).
__global__ void __launch_bounds__(256)
k_narrow(int64_t n, const uint32_t *__restrict__ om, void *nw0, void *nw1, int bytes) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t w = om[v];
        if (bytes == 1) {
            ((uint8_t *)nw0)[v] = (uint8_t)w;
            ((uint8_t *)nw1)[v] = (uint8_t)w;
        } else {
            ((uint16_t *)nw0)[v] = (uint16_t)w;
            ((uint16_t *)nw1)[v] = (uint16_t)w;
        }
    }
}

__global__ void k_set_word(uint32_t *p, uint32_t v) { *p = v; }
__global__ void k_and_word(uint32_t *p, uint32_t v) { *p &= v; }

// Per template vertex q: number of vertices with q in omega(v); slot 32: the
// total of |omega(v)|.  Inputs of the ordering features and the logs.
__global__ void __launch_bounds__(256)
k_omega_hist(int64_t n, const uint32_t *__restrict__ om, int n0, unsigned long long *hist) {
    unsigned int cnt[kMaxT];
#pragma unroll
    for (int q = 0; q < kMaxT; q++) cnt[q] = 0u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t w = __ldg(om + v);
#pragma unroll
        for (int q = 0; q < kMaxT; q++) cnt[q] += (w >> q) & 1u;
    }
    unsigned long long total = 0;
    for (int q = 0; q < n0; q++) {
        unsigned int c = __reduce_add_sync(FULL_MASK, cnt[q]);
        total += c;
        if (lane_id() == 0 && c) atomicAdd(&hist[q], (unsigned long long)c);
    }
    if (lane_id() == 0 && total) atomicAdd(&hist[kMaxT], total);
}

// Population counts for the result summary.
__global__ void __launch_bounds__(256)
k_count(int64_t n, const uint32_t *__restrict__ om, int64_t words, const uint32_t *__restrict__ eb,
        unsigned long long *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long av = 0, ae = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) av += om[i] != 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) ae += __popc(eb[i]);
    for (int o = 16; o > 0; o >>= 1) {
        av += __shfl_xor_sync(FULL_MASK, av, o);
        ae += __shfl_xor_sync(FULL_MASK, ae, o);
    }
    if (lane_id() == 0) {
        if (av) atomicAdd(&out[0], av);
        if (ae) atomicAdd(&out[1], ae);
    }
}

}  // namespace ccpm

// ===========================================================================
// C ABI
// ===========================================================================

using namespace ccpm;

// LCC rounds queued per host round trip.
constexpr int kLccGroup = 4;

struct Workspace {
    int64_t n = 0, m = 0, words = 0;
    int hub_deg = 0;
    uint32_t *om[2] = {nullptr, nullptr};
    uint16_t *nw[2] = {nullptr, nullptr};   // narrow copies of omega (up to 16 template vertices)
    uint32_t *ebits = nullptr;
    int32_t *small[2] = {nullptr, nullptr};
    int32_t *med[2] = {nullptr, nullptr};
    ChunkItem *chunk[2] = {nullptr, nullptr};
    int64_t chunk_cap = 0;
    HubAcc *acc = nullptr;
    int64_t acc_cap = 0;
    int32_t *roots = nullptr;
    uint32_t *sat = nullptr;
    SearchItem *items = nullptr;     // split search work
    int64_t items_cap = 0;
    SearchItem *items2 = nullptr;    // input of a further expansion
    SearchItem *spill_items = nullptr;   // items handed on by long searches
    int64_t spill_cap = 0;
    DevPlan *plans = nullptr;
    RoundStats *st = nullptr;        // device
    RoundStats *st_ring = nullptr;   // counters of a group of queued LCC rounds
    RoundStats *st_ring_h = nullptr; // pinned host mirror
    unsigned long long *next_root = nullptr;   // dynamic root counter of the searches
    RoundStats *st_h = nullptr;      // pinned host mirror
    unsigned long long *cnt = nullptr;
    unsigned long long *cnt_h = nullptr;
    unsigned long long *hist = nullptr;      // 33 counters (k_omega_hist)
    unsigned long long *hist_h = nullptr;
    DevPlan *plans_h = nullptr;      // pinned staging for plan uploads
    unsigned long long *aux_h = nullptr;     // pinned: counters snapshotted in stream order
    cudaEvent_t ev[12] = {};
    // compacted rows (K4), two generations; allocated at the first compaction
    int64_t *sub_rp[2] = {nullptr, nullptr};
    int32_t *sub_col[2] = {nullptr, nullptr};
    uint32_t *sub_bits[2] = {nullptr, nullptr};
    int64_t sub_cap[2] = {0, 0};     // entries sub_col / sub_bits can hold
    int64_t *deg = nullptr;          // n + 1 kept-entry counts, scanned into sub_rp
    uint8_t *sub_nlab[2] = {nullptr, nullptr};
    int32_t *sub_dslot[2] = {nullptr, nullptr};   // live vertex -> label-group directory slot
    int64_t *sub_gdir[2] = {nullptr, nullptr};
    int64_t gdir_cap[2] = {0, 0};
    unsigned int *slot_ctr = nullptr;
    uint32_t *piece_cnt = nullptr;   // kept entries per (piece, label rank) of long rows
    int64_t piece_cap = 0;
    void *scan_tmp = nullptr;
    size_t scan_tmp_bytes = 0;
    MlpScratch mlp;                  // scoring scratch of the learned order
};

struct ccpm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;                      // SMs this context sizes its grids for
    int sm_total = 0;                     // SMs of the device
    std::string err;
    Workspace ws;                         // scratch of prunes issued on this context
    std::vector<ccpm_ctx *> workers;      // contexts of concurrent batch workers
    cudaEvent_t wait_ev = nullptr;        // batch workers: waits poll this event and yield
    // batch workers: grids are sized for sm_total / min(batch_share, workers
    // busy right now), so the last templates of a batch get the whole GPU back
    const std::atomic<int> *batch_busy = nullptr;
    int batch_share = 1;
};

// SMs a launch of this context sizes its grid for.
int grid_sms(const ccpm_ctx *ctx) {
    if (!ctx->batch_busy) return ctx->num_sms;
    const int busy = std::max(1, std::min(ctx->batch_share, ctx->batch_busy->load(std::memory_order_relaxed)));
    return std::max(1, ctx->sm_total / busy);
}

struct ccpm_graph {
    ccpm_ctx *ctx = nullptr;
    int64_t n = 0, m = 0;
    int64_t *rp = nullptr;
    int32_t *col = nullptr;
    uint8_t *lab = nullptr;
    bool borrowed = false;
    int64_t label_freq[256] = {};
    int32_t *lcol = nullptr;      // rows grouped by neighbour label (built on first search)
    uint8_t *nlab = nullptr;
    std::mutex lrow_mu;           // concurrent batch workers build the grouped rows once
    int tuned_workers = 0;        // batch settings chosen by the autotuner (0: not tuned yet)
    int tuned_split = 0, tuned_short = 0, tuned_hub = 0, tuned_share = 0;
    double tuned_ms = 0.0;        // the chosen setting's time on the tuning slice
    std::atomic<int> prunes{0};   // prunes started on this graph
    std::atomic<bool> lrows_ready{false};   // lcol/nlab built (read without the lock)
    uint8_t *elab = nullptr;      // label of each entry's neighbour, CSR order (built on first use)
    uint8_t *edge_lab = nullptr;  // edge label of each entry (ccpm_graph_set_edge_labels), or none
    bool edge_lab_borrowed = false;
};

struct ccpm_tmpl {
    ccpm_ctx *ctx = nullptr;
    Template t;
};

struct ccpm_result {
    ccpm_graph *g = nullptr;
    uint64_t tmpl_fp = 0;           // fingerprint of the template it was made for
    uint32_t *om = nullptr;
    uint32_t *eb = nullptr;
    ccpm_counts counts{};
    std::vector<int32_t> phase_rounds;
    std::vector<ccpm_constraint_log> logs;
};

namespace {

int set_err(ccpm_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

// Wait for the work queued on the context's stream.  A batch worker polls an
// event and yields its core between polls: the runtime's own wait spins, and
// a dozen workers spinning at once would hold the host cores that the other
// workers need to launch their next kernels (a worker whose GPU work is done
// could then wait a scheduler time slice for a core).
cudaError_t ctx_sync(ccpm_ctx *ctx) {
    if (!ctx->wait_ev) return cudaStreamSynchronize(ctx->stream);
    cudaError_t e = cudaEventRecord(ctx->wait_ev, ctx->stream);
    if (e != cudaSuccess) return e;
    while ((e = cudaEventQuery(ctx->wait_ev)) == cudaErrorNotReady) std::this_thread::yield();
    return e;
}

// FNV-1a 64 over a byte range (fingerprints and the checksum of saved states)
uint64_t fnv1a(const void *p, size_t len, uint64_t h = 0xcbf29ce484222325ull) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t i = 0; i < len; i++) { h ^= b[i]; h *= 0x100000001b3ull; }
    return h;
}

// the template as labels and sorted edge list: equal for the same template
// however its edges were listed
uint64_t tmpl_fingerprint(const Template &t) {
    std::vector<std::pair<int, int>> e = t.edges;
    std::sort(e.begin(), e.end());
    uint64_t h = fnv1a(&t.n0, sizeof(t.n0));
    h = fnv1a(t.labels, (size_t)t.n0, h);
    for (auto &x : e) { int32_t ab[2] = {x.first, x.second}; h = fnv1a(ab, sizeof(ab), h); }
    return h;
}

uint64_t graph_fingerprint(const ccpm_graph &g) {
    uint64_t h = fnv1a(&g.n, sizeof(g.n));
    h = fnv1a(&g.m, sizeof(g.m), h);
    return fnv1a(g.label_freq, sizeof(g.label_freq), h);
}

#define CU(ctx, call)                                                                 \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return set_err((ctx), e_ == cudaErrorMemoryAllocation ? CCPM_ENOMEM : CCPM_ECUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

template <typename T>
int dalloc(ccpm_ctx *ctx, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        return set_err(ctx, CCPM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return CCPM_OK;
}

void ws_free(Workspace &w) {
    cudaFree(w.om[0]); cudaFree(w.om[1]); cudaFree(w.nw[0]); cudaFree(w.nw[1]); cudaFree(w.ebits);
    cudaFree(w.small[0]); cudaFree(w.small[1]); cudaFree(w.med[0]); cudaFree(w.med[1]);
    cudaFree(w.chunk[0]); cudaFree(w.chunk[1]); cudaFree(w.acc); cudaFree(w.roots);
    cudaFree(w.sat); cudaFree(w.items); cudaFree(w.items2); cudaFree(w.spill_items); cudaFree(w.plans); cudaFree(w.st); cudaFree(w.cnt); cudaFree(w.next_root);
    if (w.st_h) cudaFreeHost(w.st_h);
    cudaFree(w.st_ring);
    if (w.st_ring_h) cudaFreeHost(w.st_ring_h);
    if (w.cnt_h) cudaFreeHost(w.cnt_h);
    cudaFree(w.hist);
    if (w.hist_h) cudaFreeHost(w.hist_h);
    if (w.plans_h) cudaFreeHost(w.plans_h);
    if (w.aux_h) cudaFreeHost(w.aux_h);
    for (auto &e : w.ev) if (e) cudaEventDestroy(e);
    for (int i = 0; i < 2; i++) { cudaFree(w.sub_rp[i]); cudaFree(w.sub_col[i]); cudaFree(w.sub_bits[i]); }
    for (int i = 0; i < 2; i++) { cudaFree(w.sub_nlab[i]); cudaFree(w.sub_dslot[i]); cudaFree(w.sub_gdir[i]); }
    cudaFree(w.slot_ctr);
    cudaFree(w.deg); cudaFree(w.piece_cnt); cudaFree(w.scan_tmp);
    mlp_scratch_free(w.mlp);
    w = Workspace{};
}

int ws_ensure(ccpm_ctx *ctx, ccpm_graph *g, int hub_deg) {
    Workspace &w = ctx->ws;
    if (w.om[0] && w.hub_deg == hub_deg && w.n == g->n && w.m == g->m) return CCPM_OK;
    ws_free(w);
    w.n = g->n;
    w.m = g->m;
    w.words = (g->m + 31) / 32;
    w.hub_deg = hub_deg;
    w.chunk_cap = 2 * (g->m / hub_deg) + 16;
    w.acc_cap = g->m / hub_deg + 16;
    int rc;
    if ((rc = dalloc(ctx, &w.om[0], (size_t)g->n))) return rc;
    if ((rc = dalloc(ctx, &w.om[1], (size_t)g->n))) return rc;
    if ((rc = dalloc(ctx, &w.nw[0], (size_t)g->n))) return rc;
    if ((rc = dalloc(ctx, &w.nw[1], (size_t)g->n))) return rc;
    if ((rc = dalloc(ctx, &w.ebits, (size_t)w.words + 1))) return rc;
    for (int i = 0; i < 2; i++) {
        if ((rc = dalloc(ctx, &w.small[i], (size_t)g->n))) return rc;
        if ((rc = dalloc(ctx, &w.med[i], (size_t)g->n))) return rc;
        if ((rc = dalloc(ctx, &w.chunk[i], (size_t)w.chunk_cap))) return rc;
    }
    if ((rc = dalloc(ctx, &w.acc, (size_t)w.acc_cap))) return rc;
    if ((rc = dalloc(ctx, &w.roots, (size_t)g->n))) return rc;
    if ((rc = dalloc(ctx, &w.sat, (size_t)g->n))) return rc;
    w.items_cap = std::min<int64_t>(std::max<int64_t>(g->m, (int64_t)1 << 22), (int64_t)1 << 24);
    if ((rc = dalloc(ctx, &w.items, (size_t)w.items_cap))) return rc;
    if ((rc = dalloc(ctx, &w.items2, (size_t)kExpandBelow))) return rc;
    w.spill_cap = std::max<int64_t>(w.items_cap / 4, (int64_t)1 << 20);
    if ((rc = dalloc(ctx, &w.spill_items, (size_t)w.spill_cap))) return rc;
    if ((rc = dalloc(ctx, &w.plans, (size_t)kMaxPlans))) return rc;
    if ((rc = dalloc(ctx, &w.st, 1))) return rc;
    if ((rc = dalloc(ctx, &w.st_ring, (size_t)kLccGroup))) return rc;
    CU(ctx, cudaMallocHost((void **)&w.st_ring_h, sizeof(RoundStats) * kLccGroup));
    if ((rc = dalloc(ctx, &w.cnt, 2))) return rc;
    if ((rc = dalloc(ctx, &w.next_root, 1))) return rc;
    CU(ctx, cudaMallocHost((void **)&w.st_h, sizeof(RoundStats)));
    CU(ctx, cudaMallocHost((void **)&w.cnt_h, 2 * sizeof(unsigned long long)));
    CU(ctx, cudaMalloc((void **)&w.hist, (kMaxT + 1) * sizeof(unsigned long long)));
    CU(ctx, cudaMallocHost((void **)&w.hist_h, (kMaxT + 1) * sizeof(unsigned long long)));
    CU(ctx, cudaMallocHost((void **)&w.plans_h, kMaxPlans * sizeof(DevPlan)));
    CU(ctx, cudaMallocHost((void **)&w.aux_h, 4 * sizeof(unsigned long long)));
    CU(ctx, cudaMemsetAsync(w.acc, 0, sizeof(HubAcc) * (size_t)w.acc_cap, ctx->stream));
    for (auto &e : w.ev) CU(ctx, cudaEventCreate(&e));
    return CCPM_OK;
}

// Label-grouped copy of the rows: a stable segmented sort of every row by the
// neighbours' labels keeps ids ascending inside each label group.  Built once
// per graph, the first time a search needs it.
int ensure_label_rows(ccpm_ctx *ctx, ccpm_graph *g) {
    std::lock_guard<std::mutex> lock(g->lrow_mu);
    if (g->lcol || g->m == 0) return CCPM_OK;
    int rc;
    if ((rc = dalloc(ctx, &g->lcol, (size_t)g->m))) return rc;
    if ((rc = dalloc(ctx, &g->nlab, (size_t)g->m))) {
        cudaFree(g->lcol);
        g->lcol = nullptr;
        return rc;
    }
    // a counting sort of every row by neighbour label; its keys are the entry
    // labels (gathered here into a temporary array when they are not built:
    // the sort reads them twice)
    uint8_t *keys = g->elab;
    if (!keys) {
        if ((rc = dalloc(ctx, &keys, (size_t)g->m))) {
            cudaFree(g->lcol); cudaFree(g->nlab);
            g->lcol = nullptr; g->nlab = nullptr;
            return rc;
        }
        const int gg = (int)std::min<int64_t>((g->m + 255) / 256, (int64_t)ctx->num_sms * 8);
        k_gather_labels<<<gg, 256, 0, ctx->stream>>>(g->m, g->col, g->lab, keys);
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((g->n + 7) / 8, (int64_t)grid_sms(ctx) * 8));
    k_label_sort<<<grid, 256, 0, ctx->stream>>>(g->n, g->rp, g->col, g->lab, keys, g->nlab, g->lcol);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (keys != g->elab) cudaFree(keys);
    if (e != cudaSuccess) {
        cudaFree(g->lcol); cudaFree(g->nlab);
        g->lcol = nullptr; g->nlab = nullptr;
        return set_err(ctx, CCPM_ECUDA, std::string("label-grouped rows: ") + cudaGetErrorString(e));
    }
    g->lrows_ready.store(true);
    return CCPM_OK;
}

// The label of every entry's neighbour in CSR order (one byte per entry):
// the first LCC round after init reads it instead of the column index and the
// neighbour's label.  Built once per graph, the first time a first round
// covers a large share of the entries.
int ensure_entry_labels(ccpm_ctx *ctx, ccpm_graph *g) {
    std::lock_guard<std::mutex> lock(g->lrow_mu);
    if (g->elab || g->m == 0) return CCPM_OK;
    uint8_t *el = nullptr;
    int rc;
    if ((rc = dalloc(ctx, &el, (size_t)g->m))) return rc;
    int grid = (int)std::min<int64_t>((g->m + 255) / 256, (int64_t)ctx->num_sms * 8);
    k_gather_labels<<<grid, 256, 0, ctx->stream>>>(g->m, g->col, g->lab, el);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(el);
        return set_err(ctx, CCPM_ECUDA, std::string("entry labels: ") + cudaGetErrorString(e));
    }
    g->elab = el;
    return CCPM_OK;
}

// Split search work level by level while there is too little of it to fill
// the GPU (and the items still leave positions to place).
int expand_more(ccpm_ctx *ctx, Workspace &w, SearchArgs &a, int max_depth, int64_t &launches) {
    for (int depth = 2; depth < max_depth && depth < kItemMaxDepth; depth++) {
        if (a.n_items <= 0 || a.n_items >= kExpandBelow) return CCPM_OK;
        CU(ctx, cudaMemcpyAsync(w.items2, w.items, sizeof(SearchItem) * (size_t)a.n_items, cudaMemcpyDeviceToDevice,
                                ctx->stream));
        CU(ctx, cudaMemsetAsync(&w.st->n_items, 0, sizeof(unsigned int), ctx->stream));
        launches++;
        int grid = (int)std::max<int64_t>(1, std::min<int64_t>((a.n_items + 3) / 4, (int64_t)grid_sms(ctx) * 16));
        k_expand_next<<<grid, 128, 0, ctx->stream>>>(a, w.items2, a.n_items);
        CU(ctx, cudaGetLastError());
        unsigned int n2 = 0;
        CU(ctx, cudaMemcpyAsync(&n2, &w.st->n_items, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
        CU(ctx, ctx_sync(ctx));
        if ((int64_t)n2 > w.items_cap) return set_err(ctx, CCPM_EOVERFLOW, "search items overflow");
        a.n_items = n2;
    }
    return CCPM_OK;
}

// Grid of one resident wave for a 256-thread grid-stride kernel.
template <typename K>
int lcc_grid(ccpm_ctx *ctx, K kernel, int64_t warps) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 4;
    int64_t need = (warps + 7) / 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)grid_sms(ctx) * per_sm));
}

int grid_for(ccpm_ctx *ctx, int64_t work_items, int per_block, int blocks_per_sm) {
    int64_t need = (work_items + per_block - 1) / per_block;
    int64_t cap = (int64_t)grid_sms(ctx) * blocks_per_sm;
    if (need < 1) need = 1;
    return (int)std::min(need, cap);
}

// Windows a search scans before it hands the rest of its work to other warps.
constexpr uint64_t kSpillAfter = 2048;

// Run an item kernel, then again over the items long searches handed on, until
// none are left (each round of items is strictly deeper, so at most one pass
// per template position).  kind 0: NLCC existence (k_nlcc_items), 1: final
// count, 2: final count and mark, 3: count and list, 4: per-entry existence
// (k_edge_search).  Counting (and marking) stops once the cap
// is passed.
int item_passes(ccpm_ctx *ctx, Workspace &w, SearchArgs &a, int kind, uint64_t split, int64_t &launches,
                int64_t &passes) {
    cudaStream_t s = ctx->stream;
    SearchItem *bufs[2] = {w.items, w.spill_items};
    const int64_t caps[2] = {w.items_cap, w.spill_cap};
    int cur = 0;
    for (;;) {
        a.items = bufs[cur];
        a.spill = bufs[cur ^ 1];
        a.spill_cap = caps[cur ^ 1];
        a.spill_after = split;
        CU(ctx, cudaMemsetAsync(w.next_root, 0, sizeof(unsigned long long), s));
        CU(ctx, cudaMemsetAsync(&w.st->n_spill, 0, sizeof(unsigned int), s));
        CU(ctx, cudaMemsetAsync(&w.st->spill_stop, 0xFF, sizeof(unsigned int), s));
        const int gi = grid_for(ctx, (a.n_items + kItemBatch - 1) / kItemBatch * 32, 128, 16);
        launches++;
        passes++;
        if (kind == 0) k_nlcc_items<<<gi, 128, 0, s>>>(a);
        else if (kind == 1) k_final_items<kCount><<<gi, 128, 0, s>>>(a);
        else if (kind == 2) k_final_items<kMark><<<gi, 128, 0, s>>>(a);
        else if (kind == 3) k_final_items<kList><<<gi, 128, 0, s>>>(a);
        else k_edge_search<<<gi, 128, 0, s>>>(a);
        CU(ctx, cudaGetLastError());
        CU(ctx, cudaMemcpyAsync(&w.aux_h[1], &w.st->n_spill, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        CU(ctx, cudaMemcpyAsync(&w.aux_h[2], &w.st->overflow, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        CU(ctx, cudaMemcpyAsync(&w.aux_h[3], &w.st->spill_stop, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        CU(ctx, ctx_sync(ctx));
        const unsigned int spilled = std::min((unsigned int)(w.aux_h[1] & 0xFFFFFFFFull),
                                              (unsigned int)(w.aux_h[3] & 0xFFFFFFFFull));
        const unsigned int over = (unsigned int)(w.aux_h[2] & 0xFFFFFFFFull);
        if (spilled == 0 || (kind != 0 && kind != 4 && over)) break;
        a.n_items = spilled;
        cur ^= 1;
    }
    a.items = w.items;
    a.spill = nullptr;
    a.spill_after = 0;
    return CCPM_OK;
}


// Ordering features of one constraint in the current state (alive[q] =
// vertices with q in omega, total = sum of |omega|), step = constraints run.
void constraint_features(const Template &t, const HostConstraint &c, const unsigned long long *alive,
                         unsigned long long total, int step, int n_constraints, float *f) {
    for (int i = 0; i < CCPM_MLP_IN; i++) f[i] = 0.f;
    f[c.kind] = 1.f;
    const int nv = __builtin_popcount(c.vmask), ne = (int)c.edges.size(), nh = __builtin_popcount(c.hmask);
    f[5] = nv / 8.f;
    f[6] = ne / 8.f;
    f[7] = nh / 8.f;
    double sh = 0, sv = 0, mn = 1e300, mx = 0;
    for (int q = 0; q < t.n0; q++) {
        if ((c.hmask >> q) & 1u) sh += (double)alive[q];
        if ((c.vmask >> q) & 1u) {
            sv += (double)alive[q];
            mn = std::min(mn, (double)alive[q]);
            mx = std::max(mx, (double)alive[q]);
        }
    }
    if (mn > 1e299) mn = 0;
    f[8] = (float)(std::log2(1.0 + sh) / 32.0);
    f[9] = (float)(std::log2(1.0 + mn) / 32.0);
    f[10] = (float)(std::log2(1.0 + mx) / 32.0);
    f[11] = (float)(std::log2(1.0 + sv) / 32.0);
    f[12] = (float)nv / (float)t.n0;
    f[13] = (float)(ne - nv + 1) / 4.f;
    f[14] = n_constraints ? (float)step / (float)n_constraints : 0.f;
    f[15] = (float)(std::log2(1.0 + (double)total) / 32.0);
}

struct Pipeline {
    ccpm_ctx *ctx;
    ccpm_graph *g;
    const Template *t;
    DevTmpl dt;
    int cur = 0;            // omega buffer holding round-k state
    bool dense = true;      // next round is the first after init: all edge bits set
    bool from_labels = false;  // next round is the first after a fresh init: omega = initial label mask
    LabelMask lm0{};        // label -> initial omega (Alg. 3)
    int li = 0;             // frontier list parity
    int64_t n_small = 0, n_med = 0, n_chunk = 0;
    int64_t scanned = 0;
    int64_t windows = 0;
    int64_t rows = 0, alive = 0, launches = 0, lcc_launches = 0;
    int64_t alg_bytes = 0, kernel_bytes = 0, first_entries = 0, lcc_rounds_run = 0;
    double ms_first = 0.0;
    int rc_compact = 0;
    double ms_lcc_kernel = 0.0;
    double ms_search_kernel = 0.0;
    int64_t search_launches = 0, nlcc_entries = 0, item_passes = 0;
    int maxc = 0;
    int short_max = kSmallDeg;      // rows up to this length take the flat short-row path
    bool eta_off = false;           // ablation: no edge elimination
    int nw_bytes = 0;               // width of the narrow copy of omega (0: none)
    const uint8_t *elab = nullptr;  // the graph's entry labels for the first round (or none)
    int64_t first_rows = 0;         // entries in the rows of the initially active vertices
    // rows the LCC rounds read: the graph's, or the latest compacted ones (K4)
    const int64_t *lrp = nullptr;
    const int32_t *lcol = nullptr;
    uint32_t *lbits = nullptr;
    int gen = -1;                   // compacted generation in use, -1 = full rows
    int compact_mode = 0;           // options.compact
    int searches_ahead = 0;         // non-local constraints not yet checked
    int64_t compactions = 0;
    const uint8_t *lnlab = nullptr; // labels of lcol (compacted rows are label-grouped)
    const int32_t *ldslot = nullptr;  // their label-group directory
    const int64_t *lgdir = nullptr;
    int lnrank = 0;
    uint8_t llab_rank[256] = {};
    int64_t last_kept = -1, last_rows = -1;   // the latest round: entries still active, rows of the survivors

    // alive counts per template vertex (w.hist_h[0..31]) and total bits ([32])
    int omega_hist() {
        Workspace &w = ctx->ws;
        CU(ctx, cudaMemsetAsync(w.hist, 0, (kMaxT + 1) * sizeof(unsigned long long), ctx->stream));
        launches++;
        k_omega_hist<<<grid_for(ctx, g->n, 256, 4), 256, 0, ctx->stream>>>(g->n, w.om[cur], t->n0, w.hist);
        CU(ctx, cudaGetLastError());
        CU(ctx, cudaMemcpyAsync(w.hist_h, w.hist, (kMaxT + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                ctx->stream));
        CU(ctx, ctx_sync(ctx));
        return CCPM_OK;
    }

    int read_stats() {
        Workspace &w = ctx->ws;
        CU(ctx, cudaMemcpyAsync(w.st_h, w.st, sizeof(RoundStats), cudaMemcpyDeviceToHost, ctx->stream));
        CU(ctx, ctx_sync(ctx));
        return CCPM_OK;
    }

    // One LCC round.  slot: its counters; prev (nullable): the previous
    // round's counters, from which the round reads its list sizes on the
    // device (a round queued without a host round trip).  step: its place in
    // the group of queued rounds; round `step` of a group reads the omega and
    // list buffers the previous one wrote (the host flips cur / li only once
    // the group is done, by the number of rounds that ran).
    int launch_round(RoundStats *slot, const RoundStats *prev, int step = 0) {
        Workspace &w = ctx->ws;
        const int c = cur ^ (step & 1), l = li ^ (step & 1);
        LccArgs a;
        a.rp = lrp;
        a.col = lcol;
        a.om_cur = w.om[c];
        a.om_next = w.om[c ^ 1];
        a.ebits = lbits;
        a.small_in = w.small[l];
        a.med_in = w.med[l];
        a.chunk_in = w.chunk[l];
        a.n_small = n_small;
        a.n_med = n_med;
        a.n_chunk = n_chunk;
        a.small_out = w.small[l ^ 1];
        a.med_out = w.med[l ^ 1];
        a.chunk_out = w.chunk[l ^ 1];
        a.acc = w.acc;
        a.st = slot;
        a.prev = prev;
        a.resident_warps = grid_sms(ctx) * 32;
        a.hub_deg = w.hub_deg;
        a.deg = compact_mode >= 0 ? w.deg : nullptr;
        a.lab0 = from_labels ? g->lab : nullptr;
        a.elab = from_labels ? elab : nullptr;
        a.sparse = (!dense && gen < 0) ? 1 : 0;
        a.lmask = lm0;
        a.eta_off = eta_off ? ~0u : 0u;
        a.nw_bytes = nw_bytes;
        a.nw_cur = w.nw[c];
        a.nw_next = w.nw[c ^ 1];
        from_labels = false;
        // prefetch units: large enough to hide the per-vertex loads, small
        // enough that every resident warp gets several of them
        const int64_t resident = (int64_t)grid_sms(ctx) * 32;
        a.med_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(16, n_med / (4 * resident)));
        a.small_chunk = n_small >= 32 * 4 * resident ? 32 : (n_small >= 16 * 4 * resident ? 16 : 8);
        // a queued round does not know its sizes: one full resident wave
        int64_t warps = prev ? ((int64_t)1 << 40)
                             : n_chunk + (n_med + a.med_chunk - 1) / a.med_chunk + (n_small + a.small_chunk - 1) / a.small_chunk;
        launches++;
        lcc_launches++;
        // one resident wave: grid-stride work is split evenly over warps that all run at once
#define CCPM_LAUNCH_LCC(C, D) k_lcc_round<C, D><<<lcc_grid(ctx, k_lcc_round<C, D>, warps), 256, 0, ctx->stream>>>(a, dt)
        if (dense) {
            if (maxc == 0) CCPM_LAUNCH_LCC(0, true);
            else if (maxc <= 4) CCPM_LAUNCH_LCC(4, true);
            else CCPM_LAUNCH_LCC(32, true);
        } else {
            if (maxc == 0) CCPM_LAUNCH_LCC(0, false);
            else if (maxc <= 4) CCPM_LAUNCH_LCC(4, false);
            else CCPM_LAUNCH_LCC(32, false);
        }
#undef CCPM_LAUNCH_LCC
        dense = false;      // only the first round after init sees every bit set
        CU(ctx, cudaGetLastError());
        return CCPM_OK;
    }

    // LCC to fixpoint; returns rounds via *rounds.  Rounds are queued in
    // groups of up to kLccGroup with one host round trip per group: each
    // queued round reads its list sizes from the previous round's counters,
    // and rounds queued after the fixpoint return at once.  The first round
    // after init runs alone (its time is reported on its own, and a
    // compaction may follow it).  Compaction is considered between groups.
    int lcc(int64_t *rounds, bool first_alone = false) {
        Workspace &w = ctx->ws;
        int64_t r = 0;
        if (nw_bytes) {
            launches++;
            k_narrow<<<grid_for(ctx, g->n, 256, 8), 256, 0, ctx->stream>>>(g->n, w.om[cur], w.nw[0], w.nw[1], nw_bytes);
            CU(ctx, cudaGetLastError());
        }
        bool alone = first_alone;
        for (;;) {
            const int G = alone ? 1 : kLccGroup;
            alone = false;
            CU(ctx, cudaMemsetAsync(w.st_ring, 0, sizeof(RoundStats) * (size_t)G, ctx->stream));
            CU(ctx, cudaEventRecord(w.ev[4], ctx->stream));
            for (int i = 0; i < G; i++) {
                int rc = launch_round(w.st_ring + i, i ? w.st_ring + i - 1 : nullptr, i);
                if (rc) return rc;
            }
            CU(ctx, cudaEventRecord(w.ev[5], ctx->stream));
            CU(ctx, cudaMemcpyAsync(w.st_ring_h, w.st_ring, sizeof(RoundStats) * (size_t)G, cudaMemcpyDeviceToHost,
                                    ctx->stream));
            CU(ctx, ctx_sync(ctx));
            float ms = 0.f;
            CU(ctx, cudaEventElapsedTime(&ms, w.ev[4], w.ev[5]));
            ms_lcc_kernel += ms;
            bool done = false;
            int ran = 0;
            for (int i = 0; i < G; i++) {
                const RoundStats &h = w.st_ring_h[i];
                if (h.skipped) break;
                ran++;
                r++;
                scanned += (int64_t)h.scanned;
                rows += (int64_t)h.row_entries;
                alive += (int64_t)h.alive;
                alg_bytes += (33 * (int64_t)h.scanned) / 4 + 16 * (int64_t)h.alive;
                kernel_bytes += 24 * (int64_t)h.alive + (33 * (int64_t)h.row_entries) / 8 + 4 * (int64_t)h.scanned;
                if (lcc_rounds_run == 0) {
                    first_entries = (int64_t)h.scanned;
                    ms_first = ms;
                }
                lcc_rounds_run++;
                n_small = h.n_small;
                n_med = h.n_med;
                n_chunk = h.n_chunk;
                last_kept = (int64_t)h.kept;
                last_rows = (int64_t)h.rows_next;
                li ^= 1;
                cur ^= 1;
                if (!h.changed) { done = true; break; }
            }
            // launches that returned at once are not rounds
            lcc_launches -= G - ran;
            if (done) break;
            if (r > (int64_t)4 * (g->m + g->n) + 8)
                return set_err(ctx, CCPM_ETIMEOUT, "LCC did not converge");
            if (want_compact() && (rc_compact = compact())) return rc_compact;
        }
        *rounds = r;
        return CCPM_OK;
    }

    // Label-group directory of the compacted rows for the searches (none on
    // the full rows: they find groups by binary search).
    void directory(SearchArgs &a) const {
        a.dslot = gen >= 0 ? ldslot : nullptr;
        a.gdir = gen >= 0 ? lgdir : nullptr;
        a.n_rank = lnrank;
        std::memcpy(a.lab_rank, llab_rank, sizeof(llab_rank));
    }

    // Compact when most entries of the live rows are inactive: the next round
    // (or search) would mostly skip them.
    // Automatic mode compacts for searches: while non-local constraints are
    // still to run, and before the final search.  The LCC rounds alone barely
    // pay for the copy (measured on the scale-22 tree template), so an
    // LCC-only template is not compacted between its rounds.
    bool want_compact(bool final_search = false) const {
        if (compact_mode < 0 || last_rows <= 0) return false;
        if (compact_mode > 0) return last_kept < last_rows;
        return (final_search || searches_ahead > 0) && last_rows >= ((int64_t)1 << 21) &&
               last_kept * 8 < last_rows;
    }

    // A search needs label-grouped rows.  The grouped copy of the full rows
    // (a sort of every row, once per graph) pays off over many prunes of a
    // resident graph; for a graph's first prunes compacting the live rows is
    // far cheaper.
    bool cheaper_than_label_rows() const {
        return compact_mode >= 0 && gen < 0 && !g->lrows_ready.load() && g->prunes < 2 && last_rows > 0 &&
               last_kept < last_rows;
    }

    // Frontier of the live vertices over rows rp (the pieces of a long row
    // consecutive and in order); also makes both omega buffers equal.
    int rebucket(const int64_t *rp, bool sync = true) {
        Workspace &w = ctx->ws;
        LabelMask all;
        std::memset(&all, 0xFF, sizeof(all));
        CU(ctx, cudaMemsetAsync(w.st, 0, sizeof(RoundStats), ctx->stream));
        launches++;
        k_init<<<grid_for(ctx, g->n, 256, 8), 256, 0, ctx->stream>>>(g->n, rp, g->lab, all, w.om[cur], w.om[cur],
                                                                     w.om[cur ^ 1], w.small[li], w.med[li],
                                                                     w.chunk[li], w.acc, w.st, w.hub_deg, short_max);
        CU(ctx, cudaGetLastError());
        if (!sync) return CCPM_OK;
        int rc = read_stats();
        if (rc) return rc;
        n_small = w.st_h->n_small;
        n_med = w.st_h->n_med;
        n_chunk = w.st_h->n_chunk;
        if (w.st_h->n_hub_slots > (unsigned)w.acc_cap || n_chunk > w.chunk_cap)
            return set_err(ctx, CCPM_EOVERFLOW, "hub bookkeeping overflow");
        return CCPM_OK;
    }

    // K4: new rows holding only the entries the next round would examine,
    // grouped by label (the searches scan label groups).  The kept entries
    // are a subset of those the last round found compatible (last_kept), so
    // the new arrays are sized before anything runs; one host sync at the end
    // reads the new frontier sizes.
    int compact() {
        Workspace &w = ctx->ws;
        cudaStream_t s = ctx->stream;
        const int nb = gen < 0 ? 0 : (gen ^ 1);
        int rc;
        // label ranks of the template vertices
        uint8_t labs[kMaxT];
        int nl = 0;
        for (int q = 0; q < t->n0; q++) labs[nl++] = t->labels[q];
        std::sort(labs, labs + nl);
        nl = (int)(std::unique(labs, labs + nl) - labs);
        if (w.piece_cap < w.chunk_cap * nl) {
            cudaFree(w.piece_cnt);
            w.piece_cnt = nullptr;
            w.piece_cap = 0;
            if ((rc = dalloc(ctx, &w.piece_cnt, (size_t)(w.chunk_cap * kMaxT)))) return rc;
            w.piece_cap = w.chunk_cap * kMaxT;
        }
        if (!w.sub_rp[nb] && (rc = dalloc(ctx, &w.sub_rp[nb], (size_t)g->n + 1))) return rc;
        if (!w.sub_dslot[nb] && (rc = dalloc(ctx, &w.sub_dslot[nb], (size_t)g->n))) return rc;
        if (!w.slot_ctr && (rc = dalloc(ctx, &w.slot_ctr, 1))) return rc;
        // buffers grow to twice what is needed (a cudaFree waits for the whole
        // device, which would stall every other worker of a batch)
        const int64_t dir_need = (n_small + n_med + n_chunk + 1) * (int64_t)(nl + 1);
        if (dir_need > w.gdir_cap[nb]) {
            cudaFree(w.sub_gdir[nb]);
            w.sub_gdir[nb] = nullptr;
            w.gdir_cap[nb] = 0;
            const int64_t cap = std::max<int64_t>(2 * dir_need, w.gdir_cap[nb ^ 1]);
            if ((rc = dalloc(ctx, &w.sub_gdir[nb], (size_t)cap))) return rc;
            w.gdir_cap[nb] = cap;
        }
        const int64_t need = last_kept + 64;
        if (need > w.sub_cap[nb]) {
            cudaFree(w.sub_col[nb]);
            cudaFree(w.sub_nlab[nb]);
            cudaFree(w.sub_bits[nb]);
            w.sub_col[nb] = nullptr;
            w.sub_nlab[nb] = nullptr;
            w.sub_bits[nb] = nullptr;
            w.sub_cap[nb] = 0;
            const int64_t cap = std::max<int64_t>(std::min<int64_t>(2 * need, g->m + 64), w.sub_cap[nb ^ 1]);
            if ((rc = dalloc(ctx, &w.sub_col[nb], (size_t)cap))) return rc;
            if ((rc = dalloc(ctx, &w.sub_nlab[nb], (size_t)cap))) return rc;
            if ((rc = dalloc(ctx, &w.sub_bits[nb], (size_t)(cap / 32 + 2)))) return rc;
            w.sub_cap[nb] = cap;
        }
        // the lists name every vertex live at the start of the last round; the
        // rows to copy are those of the vertices live now: list only those (the
        // kernels read the new sizes on the device, no host sync)
        const int64_t listed = n_small + n_med + n_chunk;
        if ((rc = rebucket(lrp, false))) return rc;
        CompactArgs ca{};
        ca.rp = lrp;
        ca.col = lcol;
        ca.bits = lbits;
        ca.lab = g->lab;
        ca.om = w.om[cur];
        ca.small_in = w.small[li];
        ca.med_in = w.med[li];
        ca.chunk_in = w.chunk[li];
        ca.acc = w.acc;
        ca.lists = w.st;
        ca.hub_deg = w.hub_deg;
        ca.n_rank = nl;
        std::memset(ca.lab_rank, 0xFF, sizeof(ca.lab_rank));
        for (int r = 0; r < nl; r++) {
            ca.lab_rank[labs[r]] = (uint8_t)r;
            ca.rank_label[r] = labs[r];
        }
        ca.piece_cnt = w.piece_cnt;
        // offsets of the new rows from the entries each vertex kept in the last
        // round (0 for every vertex that is not live): exclusive prefix sum of
        // the kept counts (tile scans, a scan of the tile totals, the tile
        // offsets added)
        const int64_t cnt = g->n + 1, tiles = (cnt + kScanTile - 1) / kScanTile;
        const size_t tmp = sizeof(int64_t) * (size_t)tiles;
        if (tmp > w.scan_tmp_bytes) {
            cudaFree(w.scan_tmp);
            w.scan_tmp = nullptr;
            w.scan_tmp_bytes = 0;
            CU(ctx, cudaMalloc(&w.scan_tmp, tmp));
            w.scan_tmp_bytes = tmp;
        }
        int64_t *tile_sum = (int64_t *)w.scan_tmp;
        launches += 3;
        k_scan_tiles<<<(unsigned)tiles, 256, 0, s>>>(cnt, w.deg, w.sub_rp[nb], tile_sum);
        k_scan_sums<<<1, 256, 0, s>>>(tiles, tile_sum);
        k_scan_add<<<(unsigned)tiles, 256, 0, s>>>(cnt, w.sub_rp[nb], tile_sum);
        CU(ctx, cudaGetLastError());
        if (n_chunk > 0) {
            launches++;
            k_compact_count<<<grid_for(ctx, n_chunk * 32, 256, 8), 256, 0, s>>>(ca);
            CU(ctx, cudaGetLastError());
        }
        ca.sub_rp = w.sub_rp[nb];
        ca.sub_col = w.sub_col[nb];
        ca.sub_nlab = w.sub_nlab[nb];
        ca.dslot = w.sub_dslot[nb];
        ca.gdir = w.sub_gdir[nb];
        ca.n_slots = w.slot_ctr;
        CU(ctx, cudaMemsetAsync(w.slot_ctr, 0, sizeof(unsigned int), s));
        launches++;
        k_compact_fill<<<grid_for(ctx, listed * 32, 256, 8), 256, 0, s>>>(ca);
        CU(ctx, cudaGetLastError());
        launches++;
        k_compact_bits<<<grid_for(ctx, last_kept / 32 + 2, 256, 8), 256, 0, s>>>(w.sub_bits[nb], w.sub_rp[nb] + g->n);
        CU(ctx, cudaGetLastError());
        lrp = w.sub_rp[nb];
        lcol = w.sub_col[nb];
        lnlab = w.sub_nlab[nb];
        lbits = w.sub_bits[nb];
        ldslot = w.sub_dslot[nb];
        lgdir = w.sub_gdir[nb];
        lnrank = nl;
        std::memcpy(llab_rank, ca.lab_rank, sizeof(llab_rank));
        gen = nb;
        dense = true;
        compactions++;
        if ((rc = rebucket(lrp))) return rc;
        last_rows = last_kept;          // at most; every entry is now active
        return CCPM_OK;
    }
};

}  // namespace

namespace ccpm {
int ctx_device(ccpm_ctx *ctx) { return ctx->device; }
void *ctx_stream_ptr(ccpm_ctx *ctx) { return (void *)ctx->stream; }
int ctx_num_sms(ccpm_ctx *ctx) { return ctx->num_sms; }
int ctx_set_err(ccpm_ctx *ctx, int code, const char *msg) { return set_err(ctx, code, msg); }
GraphView graph_view(ccpm_graph *g) {
    GraphView v;
    v.n = g->n;
    v.m = g->m;
    v.rp = g->rp;
    v.col = g->col;
    v.lab = g->lab;
    v.el = g->edge_lab;
    v.ctx = g->ctx;
    return v;
}
}  // namespace ccpm

extern "C" {

void ccpm_options_default(ccpm_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->order_mode = CCPM_ORDER_FIXED;
    o->run_final = 1;
    o->max_embeddings = 1ull << 32;
    o->search_budget = 0;
    o->hub_degree = 0;
    o->batch_workers = 0;
}

int ccpm_ctx_create(int device, void *stream, ccpm_ctx_t *out) {
    if (!out) return CCPM_EINVAL;
    *out = nullptr;
    ccpm_ctx *c = new (std::nothrow) ccpm_ctx();
    if (!c) return CCPM_ENOMEM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    c->sm_total = c->num_sms;
    if (e == cudaSuccess) {
        if (stream) {
            c->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    if (e != cudaSuccess) {
        delete c;
        return CCPM_ECUDA;
    }
    *out = c;
    return CCPM_OK;
}

void ccpm_ctx_destroy(ccpm_ctx_t c) {
    if (!c) return;
    cudaSetDevice(c->device);
    for (ccpm_ctx *wk : c->workers) ccpm_ctx_destroy(wk);
    ws_free(c->ws);
    if (c->wait_ev) cudaEventDestroy(c->wait_ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *ccpm_last_error(ccpm_ctx_t c) { return c ? c->err.c_str() : "null context"; }

int ccpm_graph_load_csr(ccpm_ctx_t ctx, int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                        const uint8_t *labels, int flags, ccpm_graph_t *out) {
    if (!ctx || !out) return CCPM_EINVAL;
    *out = nullptr;
    if (n < 1 || n >= (int64_t)1 << 31 || m < 0 || !row_ptr || !labels || (m > 0 && !col))
        return set_err(ctx, CCPM_EINVAL, "graph: need 1 <= n < 2^31, m >= 0 and non-NULL arrays");
    CU(ctx, cudaSetDevice(ctx->device));
    const bool dev = (flags & CCPM_DEVICE_PTRS) != 0;
    if (!dev) {
        if (row_ptr[0] != 0 || row_ptr[n] != m)
            return set_err(ctx, CCPM_EINVAL, "graph: row_ptr[0] must be 0 and row_ptr[n] == m_dir");
        if (flags & CCPM_VALIDATE) {
            for (int64_t v = 0; v < n; v++)
                if (row_ptr[v + 1] < row_ptr[v]) return set_err(ctx, CCPM_EINVAL, "graph: row_ptr not monotone");
            for (int64_t v = 0; v < n; v++) {
                for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
                    int32_t u = col[e];
                    if (u < 0 || u >= n) return set_err(ctx, CCPM_EINVAL, "graph: column index out of range");
                    if (u == v) return set_err(ctx, CCPM_EINVAL, "graph: self loop");
                    if (e > row_ptr[v] && col[e - 1] >= u)
                        return set_err(ctx, CCPM_EINVAL, "graph: row not sorted or duplicate entry");
                    // reverse entry must exist
                    const int32_t *lo = col + row_ptr[u], *hi = col + row_ptr[u + 1];
                    const int32_t *f = std::lower_bound(lo, hi, (int32_t)v);
                    if (f == hi || *f != v) return set_err(ctx, CCPM_EINVAL, "graph: missing reverse entry");
                }
            }
        }
    } else if (flags & CCPM_VALIDATE) {
        return set_err(ctx, CCPM_EINVAL, "graph: CCPM_VALIDATE needs host pointers");
    }
    ccpm_graph *g = new (std::nothrow) ccpm_graph();
    if (!g) return set_err(ctx, CCPM_ENOMEM, "graph: host allocation");
    g->ctx = ctx;
    g->n = n;
    g->m = m;
    g->borrowed = dev;
    if (dev) {
        g->rp = const_cast<int64_t *>(row_ptr);
        g->col = const_cast<int32_t *>(col);
        g->lab = const_cast<uint8_t *>(labels);
        std::vector<uint8_t> h((size_t)n);
        cudaError_t e = cudaMemcpy(h.data(), labels, (size_t)n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { delete g; return set_err(ctx, CCPM_ECUDA, "graph: label readback"); }
        for (int64_t v = 0; v < n; v++) g->label_freq[h[v]]++;
    } else {
        int rc;
        if ((rc = dalloc(ctx, &g->rp, (size_t)n + 1)) || (rc = dalloc(ctx, &g->col, (size_t)m)) ||
            (rc = dalloc(ctx, &g->lab, (size_t)n))) {
            cudaFree(g->rp); cudaFree(g->col); cudaFree(g->lab);
            delete g;
            return rc;
        }
        cudaError_t e = cudaMemcpyAsync(g->rp, row_ptr, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess && m > 0)
            e = cudaMemcpyAsync(g->col, col, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->lab, labels, (size_t)n, cudaMemcpyHostToDevice, ctx->stream);
        // the offsets' check and the label histogram run while the copies do
        bool monotone = true;
        for (int64_t v = 0; v < n && monotone; v++) monotone = row_ptr[v + 1] >= row_ptr[v];
        for (int64_t v = 0; v < n; v++) g->label_freq[labels[v]]++;
        const cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess || !monotone) {
            cudaFree(g->rp); cudaFree(g->col); cudaFree(g->lab);
            delete g;
            if (!monotone) return set_err(ctx, CCPM_EINVAL, "graph: row_ptr not monotone");
            return set_err(ctx, CCPM_ECUDA, std::string("graph upload: ") + cudaGetErrorString(e));
        }
    }
    *out = g;
    return CCPM_OK;
}

void ccpm_graph_destroy(ccpm_graph_t g) {
    if (!g) return;
    cudaSetDevice(g->ctx->device);
    if (!g->borrowed) { cudaFree(g->rp); cudaFree(g->col); cudaFree(g->lab); }
    cudaFree(g->lcol);
    cudaFree(g->nlab);
    cudaFree(g->elab);
    if (!g->edge_lab_borrowed) cudaFree(g->edge_lab);
    delete g;
}

int ccpm_graph_set_edge_labels(ccpm_graph_t g, const uint8_t *edge_labels, int flags) {
    if (!g) return CCPM_EINVAL;
    ccpm_ctx *ctx = g->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    const bool dev = (flags & CCPM_DEVICE_PTRS) != 0;
    if (edge_labels && (flags & CCPM_VALIDATE)) {
        if (dev) return set_err(ctx, CCPM_EINVAL, "edge labels: CCPM_VALIDATE needs host pointers");
        // both entries of every edge carry the same label
        std::vector<int64_t> rp((size_t)g->n + 1);
        std::vector<int32_t> col((size_t)g->m);
        CU(ctx, cudaMemcpy(rp.data(), g->rp, sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost));
        if (g->m > 0) CU(ctx, cudaMemcpy(col.data(), g->col, sizeof(int32_t) * col.size(), cudaMemcpyDeviceToHost));
        for (int64_t v = 0; v < g->n; v++)
            for (int64_t e = rp[(size_t)v]; e < rp[(size_t)v + 1]; e++) {
                const int32_t u = col[(size_t)e];
                const int32_t *lo = col.data() + rp[(size_t)u], *hi = col.data() + rp[(size_t)u + 1];
                const int32_t *f = std::lower_bound(lo, hi, (int32_t)v);
                if (f == hi || *f != v) return set_err(ctx, CCPM_EINVAL, "edge labels: missing reverse entry");
                if (edge_labels[(size_t)(f - col.data())] != edge_labels[(size_t)e])
                    return set_err(ctx, CCPM_EINVAL, "edge labels: the two entries of an edge differ");
            }
    }
    if (!g->edge_lab_borrowed) cudaFree(g->edge_lab);
    g->edge_lab = nullptr;
    g->edge_lab_borrowed = false;
    if (!edge_labels) return CCPM_OK;
    if (dev) {
        g->edge_lab = const_cast<uint8_t *>(edge_labels);
        g->edge_lab_borrowed = true;
        return CCPM_OK;
    }
    int rc = dalloc(ctx, &g->edge_lab, (size_t)std::max<int64_t>(g->m, 1));
    if (rc) return rc;
    if (g->m > 0) CU(ctx, cudaMemcpyAsync(g->edge_lab, edge_labels, (size_t)g->m, cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return CCPM_OK;
}

int ccpm_tmpl_load(ccpm_ctx_t ctx, int n0, const uint8_t *labels, int m0, const int32_t *edges, ccpm_tmpl_t *out) {
    if (!out) return CCPM_EINVAL;
    *out = nullptr;
    ccpm_tmpl *t = new (std::nothrow) ccpm_tmpl();
    if (!t) return CCPM_ENOMEM;
    t->ctx = ctx;
    int rc = template_build(t->t, n0, labels, m0, edges);
    if (rc) {
        if (ctx) ctx->err = t->t.err;
        delete t;
        return rc;
    }
    *out = t;
    return CCPM_OK;
}

void ccpm_tmpl_destroy(ccpm_tmpl_t t) { delete t; }

int ccpm_constraints_generate(ccpm_tmpl_t t, ccpm_graph_t g, int *n) {
    (void)g;
    if (!t) return CCPM_EINVAL;
    std::string err;
    int rc = constraints_generate(t->t, err);
    if (rc) {
        t->t.err = err;
        if (t->ctx) t->ctx->err = err;
        return rc;
    }
    if (n) *n = (int)t->t.k0.size();
    return CCPM_OK;
}

int ccpm_constraints_describe(ccpm_tmpl_t t, int i, ccpm_constraint_info *out) {
    if (!t || !out || !t->t.generated) return CCPM_ESTATE;
    if (i < 0 || i >= (int)t->t.order.size()) return CCPM_EINVAL;
    const HostConstraint &c = t->t.k0[(size_t)t->t.order[(size_t)i]];
    std::memset(out, 0, sizeof(*out));
    out->kind = c.kind;
    out->vert_mask = c.vmask;
    out->head_mask = c.hmask;
    out->n_verts = __builtin_popcount(c.vmask);
    out->n_edges = (int)c.edges.size();
    for (size_t k = 0; k < c.edges.size(); k++) {
        out->edges[k][0] = c.edges[k].first;
        out->edges[k][1] = c.edges[k].second;
    }
    return CCPM_OK;
}

int ccpm_tmpl_set_order(ccpm_tmpl_t t, int n, const int32_t *order) {
    if (!t || !t->t.generated) return CCPM_ESTATE;
    if (n != (int)t->t.k0.size() || (n > 0 && !order)) return CCPM_EINVAL;
    std::vector<int> seen((size_t)n, 0), ord((size_t)n);
    for (int i = 0; i < n; i++) {
        if (order[i] < 0 || order[i] >= n || seen[(size_t)order[i]]) return CCPM_EINVAL;
        seen[(size_t)order[i]] = 1;
        ord[(size_t)i] = order[i];
    }
    t->t.order = ord;
    return CCPM_OK;
}

int ccpm_prune(ccpm_ctx_t ctx, ccpm_graph_t g, ccpm_tmpl_t tm, const ccpm_options *opt_in, ccpm_result_t *out) {
    if (!ctx || !g || !tm || !out) return CCPM_EINVAL;
    if (g->ctx->device != ctx->device) return set_err(ctx, CCPM_EINVAL, "graph lives on another device");
    ccpm_options opt;
    if (opt_in) opt = *opt_in; else ccpm_options_default(&opt);
    CU(ctx, cudaSetDevice(ctx->device));
    Template &t = tm->t;
    if (!t.generated) {
        std::string err;
        int rc = constraints_generate(t, err);
        if (rc) return set_err(ctx, rc, err);
    }
    const int hub_deg = opt.hub_degree > 0 ? std::min(opt.hub_degree, kMaxHubDeg) : kDefaultHubDeg;
    const uint64_t budget = opt.search_budget ? opt.search_budget : kDefaultSearchBudget;
    const uint64_t split = opt.search_split < 0 ? 0 : (opt.search_split == 0 ? kSpillAfter : (uint64_t)opt.search_split);
    int rc = ws_ensure(ctx, g, hub_deg);
    if (rc) return rc;
    Workspace &w = ctx->ws;
    ccpm_result *r = *out;
    if (r && r->g != g) return set_err(ctx, CCPM_EINVAL, "result was made for another graph");
    const uint64_t tfp = tmpl_fingerprint(t);
    const bool resume = opt.resume != 0;
    if (resume && (!r || r->tmpl_fp != tfp))
        return set_err(ctx, CCPM_EINVAL, "options.resume needs *out to hold a state of this graph and template");
    bool fresh = false;
    if (!r) {
        r = new (std::nothrow) ccpm_result();
        if (!r) return set_err(ctx, CCPM_ENOMEM, "result: host allocation");
        r->g = g;
        if ((rc = dalloc(ctx, &r->om, (size_t)g->n)) || (rc = dalloc(ctx, &r->eb, (size_t)w.words + 1))) {
            cudaFree(r->om); cudaFree(r->eb);
            delete r;
            return rc;
        }
        fresh = true;
    }
    auto fail = [&](int code) {
        if (fresh) { cudaFree(r->om); cudaFree(r->eb); delete r; }
        return code;
    };
    std::memset(&r->counts, 0, sizeof(r->counts));
    r->phase_rounds.clear();
    r->tmpl_fp = tfp;

    Pipeline P;
    P.ctx = ctx;
    P.g = g;
    P.t = &t;
    build_dev_tmpl(t, P.dt);
    P.maxc = P.dt.n_cls;
    P.lrp = g->rp;
    P.lcol = g->col;
    P.lbits = w.ebits;
    P.short_max = opt.short_rows > 0 ? std::min(opt.short_rows, kMaxHubDeg) : kSmallDeg;
    P.eta_off = opt.no_edge_elimination != 0;
    P.nw_bytes = t.n0 <= 8 ? 1 : (t.n0 <= 16 ? 2 : 0);
    g->prunes++;
    P.compact_mode = opt.compact;
    cudaStream_t s = ctx->stream;

#define CUF(call)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_err(ctx, CCPM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return fail(CCPM_ECUDA);                                                    \
        }                                                                               \
    } while (0)
#define RCF(expr)                     \
    do {                              \
        int rc_ = (expr);             \
        if (rc_) return fail(rc_);    \
    } while (0)

    if (P.compact_mode >= 0) {
        // kept-entry counts the rounds leave for a compaction: 0 for every vertex
        // no round has listed
        if (!w.deg) RCF(dalloc(ctx, &w.deg, (size_t)g->n + 1));
        CUF(cudaMemsetAsync(w.deg, 0, sizeof(int64_t) * (size_t)(g->n + 1), s));
    }
    CUF(cudaEventRecord(w.ev[0], s));
    // ---- init (Alg. 3)
    LabelMask lm;
    std::memset(&lm, 0, sizeof(lm));
    for (int q = 0; q < t.n0; q++) lm.m[t.labels[q]] |= 1u << q;
    P.lm0 = lm;
    P.from_labels = !resume;
    if (resume) {
        // a saved state: its edge bits, then (below) its omega inside the initial one
        CUF(cudaMemcpyAsync(w.ebits, r->eb, sizeof(uint32_t) * (size_t)w.words, cudaMemcpyDeviceToDevice, s));
    } else {
        CUF(cudaMemsetAsync(w.ebits, 0xFF, sizeof(uint32_t) * (size_t)w.words, s));
    }
    // no entries past m_dir: padding bits of the last word and the guard word stay 0
    k_set_word<<<1, 1, 0, s>>>(w.ebits + w.words, 0u);
    P.launches += 1 + ((g->m & 31) != 0);
    if (g->m & 31) {
        const uint32_t pad = (1u << (uint32_t)(g->m & 31)) - 1u;
        if (resume) k_and_word<<<1, 1, 0, s>>>(w.ebits + w.words - 1, pad);
        else k_set_word<<<1, 1, 0, s>>>(w.ebits + w.words - 1, pad);
    }
    CUF(cudaGetLastError());
    CUF(cudaMemsetAsync(w.st, 0, sizeof(RoundStats), s));
    {
        int grid = grid_for(ctx, g->n, 256, 8);
        P.launches++;
        k_init<<<grid, 256, 0, s>>>(g->n, g->rp, g->lab, lm, resume ? r->om : nullptr, w.om[0], w.om[1],
                                    w.small[0], w.med[0],
                                    w.chunk[0], w.acc, w.st, hub_deg, P.short_max);
        CUF(cudaGetLastError());
    }
    if (resume) {
        // entries with a dead end point carry no bit; the first round reads the bits
        P.launches++;
        k_materialize<<<grid_for(ctx, g->n * 32, 256, 8), 256, 0, s>>>(g->n, w.om[0], g->rp, g->col, w.ebits);
        CUF(cudaGetLastError());
        P.dense = false;
    }
    RCF(P.read_stats());
    P.cur = 0;
    P.li = 0;
    P.n_small = w.st_h->n_small;
    P.n_med = w.st_h->n_med;
    P.n_chunk = w.st_h->n_chunk;
    P.first_rows = (int64_t)w.st_h->row_entries;
    if (w.st_h->n_hub_slots > (unsigned)w.acc_cap || P.n_chunk > w.chunk_cap)
        return fail(set_err(ctx, CCPM_EOVERFLOW, "hub bookkeeping overflow"));
    // the first round reads the entry labels when its rows cover a large
    // share of the graph (building them is one pass over the entries)
    if (P.dense && (opt.entry_labels > 0 ||
                    (opt.entry_labels == 0 && P.first_rows >= kEntryLabelRows && P.first_rows * 8 >= g->m))) {
        RCF(ensure_entry_labels(ctx, g));
        P.elab = g->elab;
    }

    // ---- LCC to fixpoint (Alg. 4)
    P.searches_ahead = opt.lcc_only ? 0 : (int)t.order.size();
    int64_t rounds = 0;
    RCF(P.lcc(&rounds, true));
    r->phase_rounds.push_back((int32_t)rounds);
    int64_t total_rounds = rounds;
    CUF(cudaEventRecord(w.ev[1], s));

    // ---- non-local constraints, one at a time (Alg. 1, Alg. 6/7)
    int64_t tokens = 0;
    bool over = false;
    int nl_run = 0;
    std::vector<int> remaining = t.order;
    if (opt.lcc_only) {
        remaining.clear();
        opt.run_final = 0;
    }
    const int n_constraints = (int)remaining.size();
    const bool learned = opt.order_mode == CCPM_ORDER_LEARNED && opt.mlp;
    if (opt.order_mode == CCPM_ORDER_LEARNED && !opt.mlp)
        return fail(set_err(ctx, CCPM_EINVAL, "CCPM_ORDER_LEARNED needs options.mlp"));
    r->logs.clear();
    if (n_constraints > 0) RCF(P.omega_hist());
    for (int step = 0; step < n_constraints; step++) {
        // features of every remaining constraint in the current state
        std::vector<float> feats(remaining.size() * CCPM_MLP_IN);
        for (size_t i = 0; i < remaining.size(); i++)
            constraint_features(t, t.k0[(size_t)remaining[i]], w.hist_h, w.hist_h[kMaxT], step, n_constraints,
                                &feats[i * CCPM_MLP_IN]);
        // a constraint none of whose heads is matched by a live vertex issues no
        // token and changes nothing: it is checked without launching anything
        auto is_noop = [&](size_t i) {
            const uint32_t hm = t.k0[(size_t)remaining[i]].hmask;
            for (int q = 0; q < t.n0; q++)
                if (((hm >> q) & 1u) && w.hist_h[q]) return false;
            return true;
        };
        size_t pick = 0;
        if (learned && remaining.size() > 1) {
            size_t first_noop = remaining.size();
            for (size_t i = 0; i < remaining.size() && first_noop == remaining.size(); i++)
                if (is_noop(i)) first_noop = i;
            if (first_noop < remaining.size()) {
                pick = first_noop;
            } else {
                // the network predicts -log2(1 + microseconds) of running each
                // constraint now; a later constraint of the fixed order runs
                // first if it is predicted more than twice as cheap as the fixed
                // order's next one (the one predicted cheapest among those), so
                // expensive checks wait for a state that cheaper ones have shrunk
                std::vector<float> score(remaining.size());
                P.launches++;
                RCF(mlp_score(opt.mlp, (int)remaining.size(), feats.data(), score.data(), (void *)s, w.mlp,
                               (void *)ctx->wait_ev));
                for (size_t i = 1; i < remaining.size(); i++)
                    if (score[i] > score[0] + 1.f && score[i] > score[pick]) pick = i;
            }
        }
        const bool noop = is_noop(pick);
        const int chosen = remaining[pick];
        ccpm_constraint_log lg;
        std::memset(&lg, 0, sizeof(lg));
        lg.constraint = chosen;
        lg.position = step;
        std::memcpy(lg.features, &feats[pick * CCPM_MLP_IN], sizeof(lg.features));
        lg.bits_before = (int64_t)w.hist_h[kMaxT];
        remaining.erase(remaining.begin() + (long)pick);
        P.searches_ahead = (int)remaining.size() + 1;
        const HostConstraint &c = t.k0[(size_t)chosen];
        nl_run++;
        if (noop) {
            lg.bits_after = lg.bits_before;
            r->logs.push_back(lg);
            r->phase_rounds.push_back(0);
            continue;
        }
        CUF(cudaEventRecord(w.ev[6], s));
        const int64_t tokens_before = tokens;
        uint32_t sadj[kMaxT] = {};
        for (auto &e : c.edges) { sadj[e.first] |= 1u << e.second; sadj[e.second] |= 1u << e.first; }
        for (int h = 0; h < kMaxT; h++)
            if ((c.hmask >> h) & 1u) build_plan(t, c.vmask, sadj, h, g->label_freq, false, w.plans_h[h], -1, w.hist_h);
        CUF(cudaMemcpyAsync(w.plans, w.plans_h, sizeof(DevPlan) * kMaxT, cudaMemcpyHostToDevice, s));
        CUF(cudaMemsetAsync(w.st, 0, sizeof(RoundStats), s));
        P.launches++;
        k_collect_roots<<<grid_for(ctx, g->n, 256, 8), 256, 0, s>>>(g->n, w.om[P.cur], c.hmask, w.roots, w.st);
        CUF(cudaGetLastError());
        RCF(P.read_stats());
        const int64_t n_roots = w.st_h->n_roots;
        if (n_roots > 0) {
            if (P.want_compact() || P.cheaper_than_label_rows()) RCF(P.compact());
            if (P.gen < 0) RCF(ensure_label_rows(ctx, g));
            CUF(cudaMemsetAsync(w.next_root, 0, sizeof(unsigned long long), s));
            SearchArgs a{};
            a.rp = g->rp;
            a.col = g->col;
            a.rl = P.gen >= 0 ? P.lrp : g->rp;
            a.lcol = P.gen >= 0 ? P.lcol : g->lcol;
            a.nlab = P.gen >= 0 ? P.lnlab : g->nlab;
            P.directory(a);
            a.om = w.om[P.cur];
            a.roots = w.roots;
            a.n_roots = n_roots;
            a.next_root = w.next_root;
            a.plans = w.plans;
            a.heads = c.hmask;
            a.sat = w.sat;
            a.st = w.st;
            a.budget = budget;
            a.items = w.items;
            a.items_cap = w.items_cap;
            a.enum_heads = 0;
            // one item per (root, head, candidate for position 1)
            P.launches++;
            k_expand<<<grid_for(ctx, n_roots * 32, 256, 8), 256, 0, s>>>(a);
            CUF(cudaGetLastError());
            RCF(P.read_stats());
            a.n_items = w.st_h->n_items;
            if (a.n_items <= w.items_cap) RCF(expand_more(ctx, w, a, __builtin_popcount(c.vmask), P.launches));
            CUF(cudaMemsetAsync(w.next_root, 0, sizeof(unsigned long long), s));
            P.search_launches++;
            CUF(cudaMemcpyAsync(w.aux_h, &w.st->windows, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            CUF(cudaEventRecord(w.ev[10], s));
            if (a.n_items <= w.items_cap) {
                RCF(item_passes(ctx, w, a, 0, split, P.launches, P.item_passes));
            } else {
                P.launches++;
                k_nlcc_search<<<grid_for(ctx, n_roots * 32, 128, 16), 128, 0, s>>>(a);
            }
            CUF(cudaGetLastError());
            CUF(cudaEventRecord(w.ev[11], s));
            P.launches++;
            k_nlcc_apply<<<grid_for(ctx, n_roots, 256, 8), 256, 0, s>>>(w.roots, n_roots, c.hmask, w.sat,
                                                                        w.om[0], w.om[1], P.lrp, P.lbits, w.st);
            CUF(cudaGetLastError());
            RCF(P.read_stats());
            if (w.st_h->overflow) over = true;
            P.windows += (int64_t)w.st_h->windows;
            P.nlcc_entries += (int64_t)(w.st_h->windows - w.aux_h[0]);
            tokens += (int64_t)w.st_h->tokens;
            float ms_k = 0.f;
            CUF(cudaEventElapsedTime(&ms_k, w.ev[10], w.ev[11]));
            P.ms_search_kernel += ms_k;
        }
        bool changed = n_roots > 0 && w.st_h->changed;
        P.searches_ahead = (int)remaining.size();
        CUF(cudaEventRecord(w.ev[7], s));
        int64_t rr = 0;
        if (changed) {
            // the previous fixpoint's frontier holds every live vertex
            RCF(P.lcc(&rr));
        }
        CUF(cudaEventRecord(w.ev[8], s));
        r->phase_rounds.push_back((int32_t)rr);
        total_rounds += rr;
        if (changed) RCF(P.omega_hist());      // state for the next decision
        else CUF(ctx_sync(ctx));
        float ms_a = 0.f, ms_b = 0.f;
        cudaEventElapsedTime(&ms_a, w.ev[6], w.ev[7]);
        cudaEventElapsedTime(&ms_b, w.ev[7], w.ev[8]);
        lg.ms_search = ms_a;
        lg.ms_lcc = ms_b;
        lg.lcc_rounds = (int32_t)rr;
        lg.tokens = (int32_t)std::min<int64_t>(tokens - tokens_before, INT32_MAX);
        lg.bits_after = (int64_t)w.hist_h[kMaxT];
        r->logs.push_back(lg);
    }
    CUF(cudaEventRecord(w.ev[2], s));

    // ---- final template-driven search and match count (Remark 1, Sec. 4.7)
    // omega* and E* are existence questions answered exactly by searches over
    // the whole template; the number of matches is counted separately.
    bool count_valid = false;
    uint64_t matches = 0;
    bool final_done = false;
    float ms_fc = 0.f, ms_fv = 0.f, ms_fe = 0.f;
    cudaEvent_t fev[4] = {w.ev[6], w.ev[7], w.ev[8], w.ev[9]};
    if (opt.run_final) {
        const uint32_t all = t.n0 == 32 ? 0xFFFFFFFFu : ((1u << t.n0) - 1u);
        if (P.want_compact(true) || P.cheaper_than_label_rows()) RCF(P.compact());
        if (P.gen < 0) RCF(ensure_label_rows(ctx, g));
        CUF(cudaMemsetAsync(r->om, 0, sizeof(uint32_t) * (size_t)g->n, s));
        CUF(cudaMemsetAsync(r->eb, 0, sizeof(uint32_t) * (size_t)(w.words + 1), s));
        SearchArgs a{};
        a.rp = g->rp;
        a.col = g->col;
        a.rl = P.gen >= 0 ? P.lrp : g->rp;
        a.lcol = P.gen >= 0 ? P.lcol : g->lcol;
        a.nlab = P.gen >= 0 ? P.lnlab : g->nlab;
        P.directory(a);
        a.roots = w.roots;
        a.next_root = w.next_root;
        a.plans = w.plans;
        a.sat = w.sat;
        a.eb_out = r->eb;
        a.st = w.st;
        a.budget = budget;
        a.items = w.items;
        a.items_cap = w.items_cap;
        auto run_items = [&](bool edge_pass) -> int {
            int rc2 = item_passes(ctx, w, a, edge_pass ? 4 : 0, split, P.launches, P.item_passes);
            return rc2 ? rc2 : P.read_stats();
        };
        // the final enumeration keeps the background label frequencies (measured
        // faster than ordering by live candidates there)
        const unsigned long long *live = nullptr;
        int root = 0;
        for (int q = 1; q < t.n0; q++) {
            const bool fewer = live ? live[q] < live[root] : g->label_freq[t.labels[q]] < g->label_freq[t.labels[root]];
            if (fewer) root = q;
        }
        // one pass over every match from roots of `root`: count (mode kCount) or
        // count and mark (kMark); returns overflow of the cap
        auto count_pass = [&](int mode, const uint32_t *om_src, uint64_t cap, uint64_t &found, bool &capped) -> int {
            build_plan(t, all, t.adj, root, g->label_freq, true, w.plans_h[0], -1, live);
            CU(ctx, cudaMemcpyAsync(w.plans, w.plans_h, sizeof(DevPlan), cudaMemcpyHostToDevice, s));
            CU(ctx, cudaMemsetAsync(w.st, 0, sizeof(RoundStats), s));
            P.launches++;
            k_collect_roots<<<grid_for(ctx, g->n, 256, 8), 256, 0, s>>>(g->n, om_src, 1u << root, w.roots, w.st);
            CU(ctx, cudaGetLastError());
            int rc2 = P.read_stats();
            if (rc2) return rc2;
            const int64_t nr = w.st_h->n_roots;
            found = 0;
            capped = false;
            if (nr == 0) return CCPM_OK;
            a.om = om_src;
            a.n_roots = nr;
            a.heads = 1u << root;
            a.cap = cap;
            a.enum_heads = 1;
            a.om_out = r->om;
            a.eb_out = r->eb;
            P.launches++;
            k_expand<<<grid_for(ctx, nr * 32, 256, 8), 256, 0, s>>>(a);
            CU(ctx, cudaGetLastError());
            if ((rc2 = P.read_stats())) return rc2;
            a.n_items = w.st_h->n_items;
            if (a.n_items <= w.items_cap && (rc2 = expand_more(ctx, w, a, t.n0, P.launches))) return rc2;
            CU(ctx, cudaMemsetAsync(w.next_root, 0, sizeof(unsigned long long), s));
            const bool use_items = a.n_items <= w.items_cap;
            const int gr = grid_for(ctx, nr * 32, 128, 16);
            if (use_items) {
                if ((rc2 = item_passes(ctx, w, a, mode == kMark ? 2 : 1, split, P.launches, P.item_passes))) return rc2;
            } else if (mode == kMark) {
                P.launches++;
                k_final_search<kMark><<<gr, 128, 0, s>>>(a);
            } else {
                P.launches++;
                k_final_search<kCount><<<gr, 128, 0, s>>>(a);
            }
            CU(ctx, cudaGetLastError());
            if ((rc2 = P.read_stats())) return rc2;
            P.windows += (int64_t)w.st_h->windows;
            found = w.st_h->matches;
            capped = w.st_h->overflow != 0;
            return CCPM_OK;
        };
        // count the matches (every match lies inside the pruned state); with
        // few of them one more enumeration that marks each gives omega* and E*
        // few matches (at most kFewMatches): one enumeration counts and marks
        // them.  More: a counting enumeration up to the cap; then, up to
        // kMarkCap matches, one more enumeration marks them, and past that the
        // existence passes answer omega* and E*.
        bool capped = false;
        CUF(cudaEventRecord(fev[0], s));
        RCF(count_pass(kMark, w.om[P.cur], std::min<uint64_t>(opt.max_embeddings, kFewMatches), matches, capped));
        if (!capped) {
            count_valid = true;
            final_done = true;
        } else if (opt.max_embeddings > kFewMatches) {
            RCF(count_pass(kCount, w.om[P.cur], opt.max_embeddings, matches, capped));
            count_valid = !capped;
            if (!capped && matches <= kMarkCap) {
                uint64_t again = 0;
                CUF(cudaMemsetAsync(r->om, 0, sizeof(uint32_t) * (size_t)g->n, s));
                CUF(cudaMemsetAsync(r->eb, 0, sizeof(uint32_t) * (size_t)(w.words + 1), s));
                RCF(count_pass(kMark, w.om[P.cur], opt.max_embeddings, again, capped));
                final_done = true;
            }
        } else {
            count_valid = false;
        }
        CUF(cudaEventRecord(fev[1], s));
        if (!final_done) {
            // the capped enumeration's marks stay: every one belongs to a match
            // found, so the existence searches below skip those (vertex,
            // template vertex) pairs and entries
            a.om_out = nullptr;
            a.eb_out = r->eb;
            a.sat_seed = r->om;
        }
        if (!final_done) {
            // (A) every (v, q): some match has phi(q) = v?  Found embeddings also
            // satisfy the other (vertex, template vertex) pairs they place and mark
            // their edges.
            for (int q = 0; q < t.n0; q++) build_plan(t, all, t.adj, q, g->label_freq, true, w.plans_h[q], -1, live);
            CUF(cudaMemcpyAsync(w.plans, w.plans_h, sizeof(DevPlan) * (size_t)t.n0, cudaMemcpyHostToDevice, s));
            CUF(cudaMemsetAsync(w.st, 0, sizeof(RoundStats), s));
            P.launches++;
            k_collect_roots<<<grid_for(ctx, g->n, 256, 8), 256, 0, s>>>(g->n, w.om[P.cur], all, w.roots, w.st);
            CUF(cudaGetLastError());
            RCF(P.read_stats());
            int64_t n_roots = w.st_h->n_roots;
            if (n_roots > 0) {
                a.om = w.om[P.cur];
                a.n_roots = n_roots;
                a.heads = all;
                a.enum_heads = 0;
                P.launches++;
                k_expand<<<grid_for(ctx, n_roots * 32, 256, 8), 256, 0, s>>>(a);
                CUF(cudaGetLastError());
                RCF(P.read_stats());
                a.n_items = w.st_h->n_items;
                if (a.n_items <= w.items_cap) RCF(expand_more(ctx, w, a, t.n0, P.launches));
                if (a.n_items <= w.items_cap) {
                    RCF(run_items(false));
                } else {
                    CUF(cudaMemsetAsync(w.next_root, 0, sizeof(unsigned long long), s));
                    P.launches++;
                    k_nlcc_search<<<grid_for(ctx, n_roots * 32, 128, 16), 128, 0, s>>>(a);
                    CUF(cudaGetLastError());
                    RCF(P.read_stats());
                }
                if (w.st_h->overflow) over = true;
                P.windows += (int64_t)w.st_h->windows;
                P.launches++;
                k_sat_to_omega<<<grid_for(ctx, n_roots, 256, 8), 256, 0, s>>>(w.roots, n_roots, w.sat, w.om[P.cur], r->om);
                CUF(cudaGetLastError());
            }
            a.sat_seed = nullptr;
            CUF(cudaEventRecord(fev[2], s));
            // (B) every entry between omega* vertices that no embedding has marked
            // yet: some match maps a template edge onto it?
            std::vector<std::pair<int, int>> oriented;
            for (auto &e : t.edges) { oriented.push_back(e); oriented.push_back({e.second, e.first}); }
            if (n_roots > 0) {
                CUF(cudaMemsetAsync(w.st, 0, sizeof(RoundStats), s));
                P.launches++;
                k_collect_roots<<<grid_for(ctx, g->n, 256, 8), 256, 0, s>>>(g->n, r->om, all, w.roots, w.st);
                CUF(cudaGetLastError());
                RCF(P.read_stats());
                n_roots = w.st_h->n_roots;
            }
            for (size_t o0 = 0; n_roots > 0 && o0 < oriented.size(); o0 += 32) {
                EdgeTab tab;
                std::memset(&tab, 0, sizeof(tab));
                tab.n = (int)std::min<size_t>(32, oriented.size() - o0);
                for (int o = 0; o < tab.n; o++) {
                    tab.a[o] = (int8_t)oriented[o0 + (size_t)o].first;
                    tab.b[o] = (int8_t)oriented[o0 + (size_t)o].second;
                    build_plan(t, all, t.adj, tab.a[o], g->label_freq, true, w.plans_h[o], tab.b[o], live);
                }
                CUF(cudaMemcpyAsync(w.plans, w.plans_h, sizeof(DevPlan) * (size_t)tab.n, cudaMemcpyHostToDevice, s));
                a.om = r->om;
                // the candidate entries of a range of roots become items; a range
                // whose items do not fit is halved and made again (the bits marked
                // so far stay: every one of them is a found match's edge)
                int64_t span = n_roots;
                for (int64_t r0 = 0; r0 < n_roots;) {
                    const int64_t r1 = std::min(n_roots, r0 + span);
                    CUF(cudaMemsetAsync(w.st, 0, sizeof(RoundStats), s));
                    a.roots = w.roots + r0;
                    a.n_roots = r1 - r0;
                    P.launches++;
                    k_edge_items<<<grid_for(ctx, a.n_roots * 256, 256, 8), 256, 0, s>>>(a, tab);
                    CUF(cudaGetLastError());
                    RCF(P.read_stats());
                    a.n_items = w.st_h->n_items;
                    if (a.n_items > w.items_cap) {
                        if (r1 - r0 == 1)
                            return fail(set_err(ctx, CCPM_EOVERFLOW, "edge pass: one vertex has too many candidate edges"));
                        span = std::max<int64_t>(1, (r1 - r0) / 2);
                        continue;
                    }
                    if (a.n_items > 0) {
                        RCF(run_items(true));
                        if (w.st_h->overflow) over = true;
                        P.windows += (int64_t)w.st_h->windows;
                    }
                    r0 = r1;
                }
                a.roots = w.roots;
                a.n_roots = n_roots;
            }
            CUF(cudaEventRecord(fev[3], s));
            CUF(ctx_sync(ctx));
            cudaEventElapsedTime(&ms_fv, fev[1], fev[2]);
            cudaEventElapsedTime(&ms_fe, fev[2], fev[3]);
        } else {
            CUF(ctx_sync(ctx));
        }
        cudaEventElapsedTime(&ms_fc, fev[0], fev[1]);
        final_done = true;
    }
    if (!final_done) {
        // hand back the pruned state: exact edge map for live rows, dead rows
        // zeroed.  When every round ran on the full rows with edge
        // elimination, the last (quiescent) round has already left the live
        // rows exact, and only the rows of dead vertices are cleared.
        P.launches++;
        if (P.gen < 0 && !P.eta_off)
            k_clear_dead_rows<<<grid_for(ctx, g->n, 256, 8), 256, 0, s>>>(g->n, w.om[P.cur], g->rp, w.ebits);
        else
            k_materialize_fix<<<grid_for(ctx, g->n * 32, 256, 8), 256, 0, s>>>(g->n, w.om[P.cur], g->rp, g->col,
                                                                               w.ebits, P.dt);
        CUF(cudaGetLastError());
        CUF(cudaMemcpyAsync(r->om, w.om[P.cur], sizeof(uint32_t) * (size_t)g->n, cudaMemcpyDeviceToDevice, s));
        CUF(cudaMemcpyAsync(r->eb, w.ebits, sizeof(uint32_t) * (size_t)w.words, cudaMemcpyDeviceToDevice, s));
    }
    CUF(cudaEventRecord(w.ev[3], s));
    CUF(cudaMemsetAsync(w.cnt, 0, 2 * sizeof(unsigned long long), s));
    P.launches++;
    k_count<<<grid_for(ctx, std::max<int64_t>(g->n, w.words), 256, 8), 256, 0, s>>>(g->n, r->om, w.words, r->eb, w.cnt);
    CUF(cudaGetLastError());
    CUF(cudaMemcpyAsync(w.cnt_h, w.cnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CUF(ctx_sync(ctx));
    float ms_lcc = 0, ms_nlcc = 0, ms_final = 0;
    cudaEventElapsedTime(&ms_lcc, w.ev[0], w.ev[1]);
    cudaEventElapsedTime(&ms_nlcc, w.ev[1], w.ev[2]);
    cudaEventElapsedTime(&ms_final, w.ev[2], w.ev[3]);

    ccpm_counts &cn = r->counts;
    cn.active_v = (int64_t)w.cnt_h[0];
    cn.active_e_dir = (int64_t)w.cnt_h[1];
    cn.lcc_rounds_total = total_rounds;
    cn.n_phases = (int32_t)r->phase_rounds.size();
    cn.nlcc_constraints_run = nl_run;
    cn.count_valid = count_valid ? 1 : 0;
    cn.match_embeddings = count_valid ? matches : 0;
    cn.automorphisms = t.automorphisms;
    cn.match_subgraphs = (count_valid && t.automorphisms) ? matches / t.automorphisms : 0;
    cn.tokens = tokens;
    cn.edges_scanned_lcc = P.scanned;
    cn.edges_scanned_search = P.windows;
    cn.ms_lcc = ms_lcc;
    cn.ms_nlcc = ms_nlcc;
    cn.ms_final = ms_final;
    cn.ms_total = (double)ms_lcc + ms_nlcc + ms_final;
    cn.lcc_launches = P.lcc_launches;
    cn.ms_lcc_kernel = P.ms_lcc_kernel;
    cn.lcc_row_entries = P.rows;
    cn.lcc_active_vertices = P.alive;
    cn.lcc_alg_bytes = P.alg_bytes;
    cn.lcc_kernel_bytes = P.kernel_bytes;
    cn.lcc_first_entries = P.first_entries;
    cn.ms_lcc_first = P.ms_first;
    cn.ms_final_count = ms_fc;
    cn.ms_final_vertex = ms_fv;
    cn.ms_final_edge = ms_fe;
    cn.kernel_launches = P.launches;
    cn.lcc_compactions = P.compactions;
    cn.ms_search_kernel = P.ms_search_kernel;
    cn.search_launches = P.search_launches;
    cn.search_entries_nlcc = P.nlcc_entries;
    int status = CCPM_OK;
    if (over || (opt.run_final && !count_valid)) status = CCPM_EBUDGET;
    cn.status = status;
    *out = r;
    if (status == CCPM_EBUDGET) set_err(ctx, CCPM_EBUDGET, "a search budget was exceeded");
    return status;
#undef CUF
#undef RCF
}

// Run the templates tmpls[order[0..)] of a batch on `W` worker contexts, one
// host thread each, taking templates from a shared counter in that order.
// Returns the first error.
static int run_batch(ccpm_ctx *ctx, ccpm_graph *g, const std::vector<int> &order, const ccpm_tmpl_t *tmpls,
                     const ccpm_options *opt, ccpm_result_t *outs, int W, int *budget_hit) {
    const int hi = (int)order.size();
    W = std::max(1, std::min(W, hi));
    while ((int)ctx->workers.size() < W) {
        ccpm_ctx *wk = nullptr;
        int rc = ccpm_ctx_create(ctx->device, nullptr, &wk);
        if (rc) return set_err(ctx, rc, "batch: worker context");
        ctx->workers.push_back(wk);
        if (cudaEventCreateWithFlags(&wk->wait_ev, cudaEventDisableTiming) != cudaSuccess)
            return set_err(ctx, CCPM_ECUDA, "batch: worker event");
    }
    // grid share: while k workers are busy a worker sizes its grids for
    // 1/min(share, k) of the SMs (the persistent-style search kernels would
    // otherwise hold every SM until they finish, and the small kernels of
    // other templates would wait behind them); the last templates of the
    // batch get the whole GPU back
    const int share = std::max(1, opt->grid_share);
    std::atomic<int> busy(0);
    // workers start after everything already queued on the caller's stream
    cudaEvent_t ready;
    CU(ctx, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    if (cudaEventRecord(ready, ctx->stream) != cudaSuccess) {
        cudaEventDestroy(ready);
        return set_err(ctx, CCPM_ECUDA, "batch: event record");
    }
    for (int i = 0; i < W; i++)
        if (cudaStreamWaitEvent(ctx->workers[(size_t)i]->stream, ready, 0) != cudaSuccess) {
            cudaEventDestroy(ready);
            return set_err(ctx, CCPM_ECUDA, "batch: stream wait");
        }
    // the counter lives on this call's stack: the workers see it only
    // while their threads run
    for (int i = 0; i < W; i++) {
        ccpm_ctx *wk = ctx->workers[(size_t)i];
        wk->batch_busy = &busy;
        wk->batch_share = share;
    }
    std::atomic<int> next(0);
    std::atomic<int> first_err(0);
    std::atomic<int> budget(0);
    std::mutex err_mu;
    std::string err_msg;
    std::vector<std::thread> pool;
    for (int i = 0; i < W; i++) {
        ccpm_ctx *wk = ctx->workers[(size_t)i];
        pool.emplace_back([&, wk]() {
            cudaSetDevice(wk->device);
            for (int i = next.fetch_add(1); i < hi; i = next.fetch_add(1)) {
                if (first_err.load()) break;
                const int k = order[(size_t)i];
                busy.fetch_add(1);
                int rc = ccpm_prune(wk, g, tmpls[k], opt, &outs[k]);
                busy.fetch_sub(1);
                if (rc == CCPM_EBUDGET) {
                    budget.store(1);
                } else if (rc) {
                    int zero = 0;
                    if (first_err.compare_exchange_strong(zero, rc)) {
                        std::lock_guard<std::mutex> lk(err_mu);
                        err_msg = wk->err;
                    }
                }
            }
        });
    }
    for (auto &t : pool) t.join();
    for (int i = 0; i < W; i++) ctx->workers[(size_t)i]->batch_busy = nullptr;
    cudaEventDestroy(ready);
    if (budget.load()) *budget_hit = 1;
    if (first_err.load()) return set_err(ctx, first_err.load(), "batch: " + err_msg);
    return CCPM_OK;
}

int ccpm_prune_batch(ccpm_ctx_t ctx, ccpm_graph_t g, int T, const ccpm_tmpl_t *tmpls, const ccpm_options *opt_in,
                     ccpm_result_t *outs) {
    if (!ctx || !g || T < 0 || (T > 0 && (!tmpls || !outs))) return CCPM_EINVAL;
    for (int i = 0; i < T; i++)
        if (!tmpls[i]) return set_err(ctx, CCPM_EINVAL, "batch: NULL template");
    ccpm_options opt;
    if (opt_in) opt = *opt_in; else ccpm_options_default(&opt);
    CU(ctx, cudaSetDevice(ctx->device));
    // constraint generation is host work: do it here, not inside the workers
    for (int i = 0; i < T; i++) {
        if (!tmpls[i]->t.generated) {
            std::string err;
            int rc = constraints_generate(tmpls[i]->t, err);
            if (rc) return set_err(ctx, rc, err);
        }
    }
    int rc = ensure_label_rows(ctx, g);
    if (rc) return rc;
    int budget_hit = 0;
    const bool tune = opt.batch_workers <= 0 && g->tuned_workers <= 0;
    if (tune) {
        // autotune on one slice of this batch, the same templates for every
        // candidate (results are the same whatever the setting, so the slice's
        // results are simply made again): first the worker count, then the
        // windows a search scans before it hands work on, then the row length
        // of the flat short-row path, then the piece length of long rows.  The
        // choice is kept on the graph.
        // the slice: 32 templates spread evenly over the batch (long enough
        // for workers to queue, as they do on the whole batch)
        const int slice = std::max(1, std::min(T, 32));
        std::vector<int> sl;
        for (int i = 0; i < slice; i++) sl.push_back((int)((int64_t)i * T / slice));
        ccpm_options cand = opt;
        cand.search_split = 0;
        cand.short_rows = 0;
        cand.hub_degree = 0;
        cand.grid_share = 1;
        int best_w = 8;
        double best = 1e300;
        auto time_slice = [&](const ccpm_options &o, int W, double &ms) -> int {
            auto t0 = std::chrono::steady_clock::now();
            int rc2 = run_batch(ctx, g, sl, tmpls, &o, outs, W, &budget_hit);
            ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            return rc2;
        };
        double ms = 0;
        int rc;
        for (int Wc : {1, 2, 4, 8, 16}) {
            if ((rc = time_slice(cand, Wc, ms))) return rc;
            if (ms < best) { best = ms; best_w = Wc; }
        }
        for (int gs : {2, 4}) {
            ccpm_options o = cand;
            o.grid_share = gs;
            if ((rc = time_slice(o, best_w, ms))) return rc;
            if (ms < best) { best = ms; cand.grid_share = gs; }
        }
        for (int sp : {512, 8192}) {
            ccpm_options o = cand;
            o.search_split = sp;
            if ((rc = time_slice(o, best_w, ms))) return rc;
            if (ms < best) { best = ms; cand.search_split = sp; }
        }
        for (int sr : {32, 256}) {
            ccpm_options o = cand;
            o.short_rows = sr;
            if ((rc = time_slice(o, best_w, ms))) return rc;
            if (ms < best) { best = ms; cand.short_rows = sr; }
        }
        for (int hd : {4096}) {
            ccpm_options o = cand;
            o.hub_degree = hd;
            if ((rc = time_slice(o, best_w, ms))) return rc;
            if (ms < best) { best = ms; cand.hub_degree = hd; }
        }
        g->tuned_workers = best_w;
        g->tuned_split = cand.search_split;
        g->tuned_short = cand.short_rows;
        g->tuned_hub = cand.hub_degree;
        g->tuned_share = cand.grid_share;
        g->tuned_ms = best;
    }
    int W = opt.batch_workers > 0 ? opt.batch_workers : g->tuned_workers;
    if (opt.batch_workers <= 0) {
        // the tuned settings apply where the caller left the library default
        if (opt.search_split == 0) opt.search_split = g->tuned_split;
        if (opt.short_rows == 0) opt.short_rows = g->tuned_short;
        if (opt.hub_degree == 0) opt.hub_degree = g->tuned_hub;
        if (opt.grid_share == 0) opt.grid_share = g->tuned_share;
    }
    if (T > 0) {
        // longest first when the results of an earlier call give each
        // template's time (the tail of the batch is then short templates)
        std::vector<int> order(T);
        for (int i = 0; i < T; i++) order[(size_t)i] = i;
        bool timed = true;
        for (int i = 0; i < T && timed; i++) timed = outs[i] && outs[i]->counts.ms_total > 0.0;
        if (timed)
            std::stable_sort(order.begin(), order.end(),
                             [&](int x, int y) { return outs[x]->counts.ms_total > outs[y]->counts.ms_total; });
        int rc = run_batch(ctx, g, order, tmpls, &opt, outs, W, &budget_hit);
        if (rc) return rc;
    }
    if (budget_hit) return set_err(ctx, CCPM_EBUDGET, "a search budget was exceeded in the batch");
    return CCPM_OK;
}

}  // extern "C"

namespace {

__global__ void k_or_words(uint32_t *dst, const uint32_t *src, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] |= src[i];
}

// A result on graph g for template t holding (om, eb) copied from `src`
// arrays (the candidate set), ready for a resumed prune.
int result_from(ccpm_ctx *ctx, ccpm_graph *g, const Template &t, const uint32_t *om, const uint32_t *eb,
                int64_t words, ccpm_result **out) {
    ccpm_result *r = new (std::nothrow) ccpm_result();
    if (!r) return set_err(ctx, CCPM_ENOMEM, "result: host allocation");
    r->g = g;
    int rc;
    if ((rc = dalloc(ctx, &r->om, (size_t)g->n)) || (rc = dalloc(ctx, &r->eb, (size_t)words + 1))) {
        cudaFree(r->om); cudaFree(r->eb);
        delete r;
        return rc;
    }
    r->tmpl_fp = tmpl_fingerprint(t);
    cudaError_t e = cudaMemcpyAsync(r->om, om, sizeof(uint32_t) * (size_t)g->n, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->eb, eb, sizeof(uint32_t) * (size_t)(words + 1), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(r->om); cudaFree(r->eb);
        delete r;
        return set_err(ctx, CCPM_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
    }
    *out = r;
    return CCPM_OK;
}

}  // namespace

extern "C" {

int ccpm_explore(ccpm_ctx_t ctx, ccpm_graph_t g, ccpm_tmpl_t base, int max_removed, const ccpm_options *opt_in,
                 ccpm_explore_variant *variants, int variants_cap, int *n_variants, int *level_found,
                 double *ms_candidates, ccpm_result_t *out) {
    if (!ctx || !g || !base || !out || max_removed < 0 || (variants_cap > 0 && !variants)) return CCPM_EINVAL;
    if (g->ctx->device != ctx->device) return set_err(ctx, CCPM_EINVAL, "graph lives on another device");
    const Template &B = base->t;
    const int m0 = (int)B.edges.size();
    if (m0 > 64) return set_err(ctx, CCPM_EINVAL, "explore: the base template may have at most 64 edges");
    ccpm_options opt;
    if (opt_in) opt = *opt_in; else ccpm_options_default(&opt);
    opt.resume = 0;
    CU(ctx, cudaSetDevice(ctx->device));
    if (n_variants) *n_variants = 0;
    if (level_found) *level_found = -1;
    if (ms_candidates) *ms_candidates = 0.0;
    cudaStream_t s = ctx->stream;
    const int64_t words = (g->m + 31) / 32;
    // connected variants by level: every set of `k` template edges whose
    // removal leaves the template connected (vertices are never removed, so
    // template vertex q means the same in every variant)
    struct Variant { int level; uint64_t removed; Template t; };
    std::vector<Variant> vs;
    for (int k = 0; k <= std::min(max_removed, m0 - 1); k++) {
        std::vector<int> pick(k);
        for (int i = 0; i < k; i++) pick[i] = i;
        for (;;) {
            uint64_t mask = 0;
            for (int i : pick) mask |= 1ull << i;
            std::vector<int32_t> ed;
            for (int e = 0; e < m0; e++)
                if (!((mask >> e) & 1ull)) { ed.push_back(B.edges[(size_t)e].first); ed.push_back(B.edges[(size_t)e].second); }
            Variant v{k, mask, Template{}};
            if (template_build(v.t, B.n0, B.labels, (int)ed.size() / 2, ed.data()) == CCPM_OK) vs.push_back(std::move(v));
            int i = k - 1;
            while (i >= 0 && pick[(size_t)i] == m0 - k + i) i--;
            if (i < 0) break;
            pick[(size_t)i]++;
            for (int j = i + 1; j < k; j++) pick[(size_t)j] = pick[(size_t)j - 1] + 1;
        }
    }
    // the candidate set: the union of the LCC fixpoints of every variant (local
    // constraints only, so each costs one LCC to fixpoint); it holds every
    // match of every variant
    uint32_t *c_om = nullptr, *c_eb = nullptr;
    int rc;
    if ((rc = dalloc(ctx, &c_om, (size_t)g->n)) || (rc = dalloc(ctx, &c_eb, (size_t)words + 1))) {
        cudaFree(c_om); cudaFree(c_eb);
        return rc;
    }
    auto cleanup = [&]() { cudaFree(c_om); cudaFree(c_eb); };
    auto fail_c = [&](int code) { cleanup(); return code; };
    if (cudaMemsetAsync(c_om, 0, sizeof(uint32_t) * (size_t)g->n, s) != cudaSuccess ||
        cudaMemsetAsync(c_eb, 0, sizeof(uint32_t) * (size_t)(words + 1), s) != cudaSuccess)
        return fail_c(set_err(ctx, CCPM_ECUDA, "explore: memset"));
    ccpm_options lcc_only = opt;
    lcc_only.run_final = 0;
    lcc_only.order_mode = CCPM_ORDER_FIXED;
    auto t_start = std::chrono::steady_clock::now();
    for (auto &v : vs) {
        ccpm_tmpl tl;
        tl.ctx = ctx;
        tl.t = v.t;
        tl.t.generated = true;          // no non-local constraint: LCC only
        tl.t.k0.clear();
        tl.t.order.clear();
        ccpm_result *r = nullptr;
        rc = ccpm_prune(ctx, g, &tl, &lcc_only, &r);
        if (rc && rc != CCPM_EBUDGET) return fail_c(rc);
        const int gr = grid_for(ctx, std::max<int64_t>(g->n, words), 256, 8);
        k_or_words<<<gr, 256, 0, s>>>(c_om, r->om, g->n);
        k_or_words<<<gr, 256, 0, s>>>(c_eb, r->eb, words);
        ccpm_result_destroy(r);
        if (cudaGetLastError() != cudaSuccess) return fail_c(set_err(ctx, CCPM_ECUDA, "explore: union"));
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail_c(set_err(ctx, CCPM_ECUDA, "explore: sync"));
    if (ms_candidates)
        *ms_candidates = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    // the union of the matching variants' omega* and E* at the first level
    // with a match
    ccpm_result *u = *out;
    if (u && u->g != g) return fail_c(set_err(ctx, CCPM_EINVAL, "explore: result was made for another graph"));
    if (!u) {
        if ((rc = result_from(ctx, g, B, c_om, c_eb, words, &u))) return fail_c(rc);
    }
    u->tmpl_fp = tmpl_fingerprint(B);
    u->phase_rounds.clear();
    u->logs.clear();
    std::memset(&u->counts, 0, sizeof(u->counts));
    cudaMemsetAsync(u->om, 0, sizeof(uint32_t) * (size_t)g->n, s);
    cudaMemsetAsync(u->eb, 0, sizeof(uint32_t) * (size_t)(words + 1), s);
    int found = -1, nv = 0;
    bool budget = false;
    ccpm_options resumed = opt;
    resumed.resume = 1;
    for (int k = 0; k <= max_removed && found < 0; k++) {
        bool any = false;
        for (auto &v : vs) {
            if (v.level != k) continue;
            ccpm_tmpl tv;
            tv.ctx = ctx;
            tv.t = v.t;
            ccpm_result *r = nullptr;
            if ((rc = result_from(ctx, g, tv.t, c_om, c_eb, words, &r))) return fail_c(rc);
            rc = ccpm_prune(ctx, g, &tv, &resumed, &r);
            if (rc == CCPM_EBUDGET) budget = true;
            else if (rc) { ccpm_result_destroy(r); return fail_c(rc); }
            const ccpm_counts &c = r->counts;
            if (c.active_v > 0) {
                any = true;
                const int gr = grid_for(ctx, std::max<int64_t>(g->n, words), 256, 8);
                k_or_words<<<gr, 256, 0, s>>>(u->om, r->om, g->n);
                k_or_words<<<gr, 256, 0, s>>>(u->eb, r->eb, words);
            }
            if (nv < variants_cap) {
                ccpm_explore_variant &o = variants[nv];
                o.level = k;
                o.n_edges = (int32_t)v.t.edges.size();
                o.removed = v.removed;
                o.active_v = c.active_v;
                o.active_e_dir = c.active_e_dir;
                o.match_embeddings = c.match_embeddings;
                o.count_valid = c.count_valid;
                o.status = c.status;
                o.ms_total = c.ms_total;
            }
            nv++;
            ccpm_result_destroy(r);
        }
        if (any) found = k;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail_c(set_err(ctx, CCPM_ECUDA, "explore: sync"));
    cleanup();
    if (n_variants) *n_variants = nv;
    if (level_found) *level_found = found;
    *out = u;
    // counts of the union
    CU(ctx, cudaMemsetAsync(ctx->ws.cnt, 0, 2 * sizeof(unsigned long long), s));
    k_count<<<grid_for(ctx, std::max<int64_t>(g->n, words), 256, 8), 256, 0, s>>>(g->n, u->om, words, u->eb, ctx->ws.cnt);
    CU(ctx, cudaGetLastError());
    CU(ctx, cudaMemcpyAsync(ctx->ws.cnt_h, ctx->ws.cnt, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    u->counts.active_v = (int64_t)ctx->ws.cnt_h[0];
    u->counts.active_e_dir = (int64_t)ctx->ws.cnt_h[1];
    if (budget) return set_err(ctx, CCPM_EBUDGET, "explore: a search budget was exceeded");
    return CCPM_OK;
}

int ccpm_result_omega(ccpm_result_t r, uint32_t *dst, int64_t n, int dst_on_device) {
    if (!r || !dst || n != r->g->n) return CCPM_EINVAL;
    ccpm_ctx *ctx = r->g->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaMemcpyAsync(dst, r->om, sizeof(uint32_t) * (size_t)n,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return CCPM_OK;
}

int ccpm_result_edge_bitmap(ccpm_result_t r, uint32_t *dst, int64_t words, int dst_on_device) {
    if (!r || !dst || words != (r->g->m + 31) / 32) return CCPM_EINVAL;
    ccpm_ctx *ctx = r->g->ctx;
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaMemcpyAsync(dst, r->eb, sizeof(uint32_t) * (size_t)words,
                            dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return CCPM_OK;
}

int ccpm_result_constraint_log(ccpm_result_t r, int i, ccpm_constraint_log *out) {
    if (!r || !out || i < 0 || i >= (int)r->logs.size()) return CCPM_EINVAL;
    *out = r->logs[(size_t)i];
    return CCPM_OK;
}

int ccpm_result_counts(ccpm_result_t r, ccpm_counts *out) {
    if (!r || !out) return CCPM_EINVAL;
    *out = r->counts;
    return CCPM_OK;
}

int ccpm_result_phase_rounds(ccpm_result_t r, int32_t *dst, int cap) {
    if (!r || (!dst && cap > 0)) return CCPM_EINVAL;
    int k = std::min(cap, (int)r->phase_rounds.size());
    for (int i = 0; i < k; i++) dst[i] = r->phase_rounds[(size_t)i];
    return CCPM_OK;
}

int ccpm_result_matches(ccpm_ctx_t ctx, ccpm_result_t r, ccpm_tmpl_t tm, const ccpm_options *opt_in,
                        int32_t *list, uint64_t list_cap, uint64_t *vertex_counts, uint64_t *entry_counts,
                        int dst_on_device, uint64_t *n_matches) {
    if (!ctx || !r || !tm || !n_matches || (list_cap > 0 && !list)) return CCPM_EINVAL;
    *n_matches = 0;
    ccpm_graph *g = r->g;
    if (g->ctx->device != ctx->device) return set_err(ctx, CCPM_EINVAL, "result lives on another device");
    Template &t = tm->t;
    if (r->tmpl_fp != tmpl_fingerprint(t)) return set_err(ctx, CCPM_EINVAL, "result was made for another template");
    ccpm_options opt;
    if (opt_in) opt = *opt_in; else ccpm_options_default(&opt);
    CU(ctx, cudaSetDevice(ctx->device));
    const int hub_deg = opt.hub_degree > 0 ? std::min(opt.hub_degree, kMaxHubDeg) : kDefaultHubDeg;
    const uint64_t budget = opt.search_budget ? opt.search_budget : ~0ull;
    const uint64_t split = opt.search_split < 0 ? 0 : (opt.search_split == 0 ? kSpillAfter : (uint64_t)opt.search_split);
    int rc = ws_ensure(ctx, g, hub_deg);
    if (rc) return rc;
    if ((rc = ensure_label_rows(ctx, g))) return rc;
    Workspace &w = ctx->ws;
    cudaStream_t s = ctx->stream;
    // host outputs are filled through device buffers of this call
    int32_t *d_list = list;
    unsigned long long *d_vc = (unsigned long long *)vertex_counts, *d_ec = (unsigned long long *)entry_counts;
    bool own = false;
    auto release = [&]() {
        if (own) { cudaFree(d_list); cudaFree(d_vc); cudaFree(d_ec); }
    };
    if (!dst_on_device) {
        own = true;
        d_list = nullptr; d_vc = nullptr; d_ec = nullptr;
        if ((list_cap && (rc = dalloc(ctx, &d_list, (size_t)(list_cap * (uint64_t)t.n0)))) ||
            (vertex_counts && (rc = dalloc(ctx, &d_vc, (size_t)g->n))) ||
            (entry_counts && (rc = dalloc(ctx, &d_ec, (size_t)std::max<int64_t>(g->m, 1))))) {
            release();
            return rc;
        }
    }
#define CUR(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            release();                                                                   \
            return set_err(ctx, CCPM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                \
    } while (0)
    if (d_vc) CUR(cudaMemsetAsync(d_vc, 0, sizeof(unsigned long long) * (size_t)g->n, s));
    if (d_ec) CUR(cudaMemsetAsync(d_ec, 0, sizeof(unsigned long long) * (size_t)g->m, s));
    CUR(cudaMemsetAsync(w.cnt, 0, sizeof(unsigned long long), s));
    // the root is the template vertex with the rarest label
    int root = 0;
    for (int q = 1; q < t.n0; q++)
        if (g->label_freq[t.labels[q]] < g->label_freq[t.labels[root]]) root = q;
    const uint32_t all = t.n0 == 32 ? 0xFFFFFFFFu : ((1u << t.n0) - 1u);
    build_plan(t, all, t.adj, root, g->label_freq, true, w.plans_h[0], -1, nullptr);
    CUR(cudaMemcpyAsync(w.plans, w.plans_h, sizeof(DevPlan), cudaMemcpyHostToDevice, s));
    CUR(cudaMemsetAsync(w.st, 0, sizeof(RoundStats), s));
    k_collect_roots<<<grid_for(ctx, g->n, 256, 8), 256, 0, s>>>(g->n, r->om, 1u << root, w.roots, w.st);
    CUR(cudaGetLastError());
    CUR(cudaMemcpyAsync(w.st_h, w.st, sizeof(RoundStats), cudaMemcpyDeviceToHost, s));
    CUR(cudaStreamSynchronize(s));
    const int64_t n_roots = w.st_h->n_roots;
    bool over = false;
    if (n_roots > 0) {
        SearchArgs a{};
        a.rp = g->rp;
        a.col = g->col;
        a.rl = g->rp;
        a.lcol = g->lcol;
        a.nlab = g->nlab;
        a.om = r->om;
        a.roots = w.roots;
        a.n_roots = n_roots;
        a.next_root = w.next_root;
        a.plans = w.plans;
        a.heads = 1u << root;
        a.sat = w.sat;
        a.st = w.st;
        a.budget = budget;
        a.cap = ~0ull;
        a.items = w.items;
        a.items_cap = w.items_cap;
        a.enum_heads = 1;
        a.list_out = d_list;
        a.list_cap = list_cap;
        a.list_n0 = t.n0;
        a.list_count = w.cnt;
        a.vcnt = d_vc;
        a.ecnt = d_ec;
        int64_t launches = 0, passes = 0;
        k_expand<<<grid_for(ctx, n_roots * 32, 256, 8), 256, 0, s>>>(a);
        CUR(cudaGetLastError());
        CUR(cudaMemcpyAsync(w.st_h, w.st, sizeof(RoundStats), cudaMemcpyDeviceToHost, s));
        CUR(cudaStreamSynchronize(s));
        a.n_items = w.st_h->n_items;
        if (a.n_items <= w.items_cap && (rc = expand_more(ctx, w, a, t.n0, launches))) { release(); return rc; }
        CUR(cudaMemsetAsync(w.next_root, 0, sizeof(unsigned long long), s));
        if (a.n_items <= w.items_cap) {
            if ((rc = item_passes(ctx, w, a, 3, split, launches, passes))) { release(); return rc; }
        } else {
            k_final_search<kList><<<grid_for(ctx, n_roots * 32, 128, 16), 128, 0, s>>>(a);
            CUR(cudaGetLastError());
        }
        CUR(cudaMemcpyAsync(w.st_h, w.st, sizeof(RoundStats), cudaMemcpyDeviceToHost, s));
        CUR(cudaStreamSynchronize(s));
        over = w.st_h->overflow != 0;
    }
    unsigned long long found = 0;
    CUR(cudaMemcpyAsync(&found, w.cnt, sizeof(found), cudaMemcpyDeviceToHost, s));
    CUR(cudaStreamSynchronize(s));
    if (!dst_on_device) {
        const uint64_t rows = std::min<uint64_t>((uint64_t)found, list_cap);
        if (rows) CUR(cudaMemcpyAsync(list, d_list, sizeof(int32_t) * (size_t)(rows * (uint64_t)t.n0), cudaMemcpyDeviceToHost, s));
        if (d_vc) CUR(cudaMemcpyAsync(vertex_counts, d_vc, sizeof(uint64_t) * (size_t)g->n, cudaMemcpyDeviceToHost, s));
        if (d_ec) CUR(cudaMemcpyAsync(entry_counts, d_ec, sizeof(uint64_t) * (size_t)g->m, cudaMemcpyDeviceToHost, s));
        CUR(cudaStreamSynchronize(s));
    }
#undef CUR
    release();
    *n_matches = found;
    if (over) return set_err(ctx, CCPM_EBUDGET, "a listing search ran out of its window budget: outputs incomplete");
    return CCPM_OK;
}

const uint32_t *ccpm_result_omega_device(ccpm_result_t r) { return r ? r->om : nullptr; }
const uint32_t *ccpm_result_edge_bitmap_device(ccpm_result_t r) { return r ? r->eb : nullptr; }

int ccpm_graph_batch_workers(ccpm_graph_t g) { return g ? g->tuned_workers : 0; }

int ccpm_graph_batch_tuning(ccpm_graph_t g, int *workers, int *grid_share, int *search_split, int *short_rows,
                            int *hub_degree, double *slice_ms) {
    if (!g) return CCPM_EINVAL;
    if (workers) *workers = g->tuned_workers;
    if (grid_share) *grid_share = g->tuned_share;
    if (search_split) *search_split = g->tuned_split;
    if (short_rows) *short_rows = g->tuned_short;
    if (hub_degree) *hub_degree = g->tuned_hub;
    if (slice_ms) *slice_ms = g->tuned_ms;
    return CCPM_OK;
}

void ccpm_result_destroy(ccpm_result_t r) {
    if (!r) return;
    cudaSetDevice(r->g->ctx->device);
    cudaFree(r->om);
    cudaFree(r->eb);
    delete r;
}

// ---- checkpoint/resume: one host blob per state (layout in ccpm.h)

namespace {
struct StateHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int64_t n, m_dir, words;
    uint64_t graph_fp, tmpl_fp;
    uint32_t counts_bytes, n_phases;
    uint64_t payload_bytes;
    uint64_t payload_fnv;
    uint64_t reserved[2];
};
static_assert(sizeof(StateHeader) == 96, "state header layout");
constexpr char kStateMagic[8] = {'C', 'C', 'P', 'M', 'S', 'T', 'A', 'T'};
constexpr uint32_t kStateVersion = 1;

size_t state_payload_bytes(int64_t n, int64_t words, size_t n_phases) {
    return sizeof(ccpm_counts) + sizeof(int32_t) * n_phases + sizeof(uint32_t) * (size_t)(n + words);
}
}  // namespace

int ccpm_state_export(ccpm_result_t r, void *buf, size_t *len) {
    if (!r || !len) return CCPM_EINVAL;
    ccpm_graph *g = r->g;
    ccpm_ctx *ctx = g->ctx;
    const int64_t words = (g->m + 31) / 32;
    const size_t payload = state_payload_bytes(g->n, words, r->phase_rounds.size());
    const size_t need = sizeof(StateHeader) + payload;
    if (!buf) { *len = need; return CCPM_OK; }
    if (*len < need) {
        *len = need;
        return set_err(ctx, CCPM_EINVAL, "state buffer too small");
    }
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kStateMagic, 8);
    h.version = kStateVersion;
    h.header_bytes = sizeof(StateHeader);
    h.n = g->n;
    h.m_dir = g->m;
    h.words = words;
    h.graph_fp = graph_fingerprint(*g);
    h.tmpl_fp = r->tmpl_fp;
    h.counts_bytes = sizeof(ccpm_counts);
    h.n_phases = (uint32_t)r->phase_rounds.size();
    h.payload_bytes = payload;
    unsigned char *p = (unsigned char *)buf + sizeof(StateHeader);
    std::memcpy(p, &r->counts, sizeof(ccpm_counts));
    p += sizeof(ccpm_counts);
    if (!r->phase_rounds.empty()) std::memcpy(p, r->phase_rounds.data(), sizeof(int32_t) * r->phase_rounds.size());
    p += sizeof(int32_t) * r->phase_rounds.size();
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaMemcpy(p, r->om, sizeof(uint32_t) * (size_t)g->n, cudaMemcpyDeviceToHost));
    p += sizeof(uint32_t) * (size_t)g->n;
    CU(ctx, cudaMemcpy(p, r->eb, sizeof(uint32_t) * (size_t)words, cudaMemcpyDeviceToHost));
    h.payload_fnv = fnv1a((const unsigned char *)buf + sizeof(StateHeader), payload);
    std::memcpy(buf, &h, sizeof(h));
    *len = need;
    return CCPM_OK;
}

int ccpm_state_import(ccpm_ctx_t ctx, ccpm_graph_t g, ccpm_tmpl_t tm, const void *buf, size_t len,
                      ccpm_result_t *out) {
    if (!ctx || !g || !tm || !buf || !out) return CCPM_EINVAL;
    *out = nullptr;
    if (g->ctx->device != ctx->device) return set_err(ctx, CCPM_EINVAL, "graph lives on another device");
    StateHeader h;
    if (len < sizeof(h)) return set_err(ctx, CCPM_EINVAL, "state: truncated header");
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != kStateVersion ||
        h.header_bytes != sizeof(StateHeader) || h.counts_bytes != sizeof(ccpm_counts))
        return set_err(ctx, CCPM_EINVAL, "state: not a saved state of this library version");
    const int64_t words = (g->m + 31) / 32;
    if (h.n != g->n || h.m_dir != g->m || h.words != words || h.graph_fp != graph_fingerprint(*g))
        return set_err(ctx, CCPM_EINVAL, "state: saved for another graph");
    if (h.tmpl_fp != tmpl_fingerprint(tm->t)) return set_err(ctx, CCPM_EINVAL, "state: saved for another template");
    if (h.n_phases > (1u << 20)) return set_err(ctx, CCPM_EINVAL, "state: bad phase count");
    const size_t payload = state_payload_bytes(g->n, words, h.n_phases);
    if (h.payload_bytes != payload || len < sizeof(h) + payload) return set_err(ctx, CCPM_EINVAL, "state: truncated");
    const unsigned char *p = (const unsigned char *)buf + sizeof(h);
    if (fnv1a(p, payload) != h.payload_fnv) return set_err(ctx, CCPM_EINVAL, "state: checksum mismatch");
    CU(ctx, cudaSetDevice(ctx->device));
    ccpm_result *r = new (std::nothrow) ccpm_result();
    if (!r) return set_err(ctx, CCPM_ENOMEM, "result: host allocation");
    r->g = g;
    r->tmpl_fp = h.tmpl_fp;
    int rc = dalloc(ctx, &r->om, (size_t)g->n);
    if (!rc) rc = dalloc(ctx, &r->eb, (size_t)words + 1);
    if (rc) {
        cudaFree(r->om); cudaFree(r->eb);
        delete r;
        return rc;
    }
    std::memcpy(&r->counts, p, sizeof(ccpm_counts));
    p += sizeof(ccpm_counts);
    r->phase_rounds.resize(h.n_phases);
    if (h.n_phases) std::memcpy(r->phase_rounds.data(), p, sizeof(int32_t) * h.n_phases);
    p += sizeof(int32_t) * h.n_phases;
    cudaError_t e = cudaMemcpy(r->om, p, sizeof(uint32_t) * (size_t)g->n, cudaMemcpyHostToDevice);
    p += sizeof(uint32_t) * (size_t)g->n;
    if (e == cudaSuccess) e = cudaMemcpy(r->eb, p, sizeof(uint32_t) * (size_t)words, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(r->eb + words, 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        cudaFree(r->om); cudaFree(r->eb);
        delete r;
        return set_err(ctx, CCPM_ECUDA, std::string("state import: ") + cudaGetErrorString(e));
    }
    *out = r;
    return CCPM_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free LCC entry point
//
// Some callers cannot allocate device memory while they run: code that works
// inside a memory budget reserved up front, host code holding a lock in which
// cudaMalloc may block on the driver, or applications whose allocator is
// owned by someone else.  ccpm_lcc_fixpoint_noalloc runs local constraint
// checking to its fixpoint using only the caller's inputs and outputs plus a
// fixed scratch area compiled into this library.
// ===========================================================================

#include <mutex>

namespace {

// Scratch of the allocation-free entry point: the second omega buffer, the
// frontier lists, the split-row accumulators and the round counters.  It is
// part of the library image, so every GPU on which the library's kernels are
// loaded holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NoAllocLayout {
    size_t om2, small[2], med[2], chunk[2], acc, st, total;
    int64_t chunk_cap, acc_cap;
};

NoAllocLayout noalloc_layout(int64_t n, int64_t m, int hub) {
    NoAllocLayout L{};
    L.chunk_cap = 2 * (m / hub) + 16;
    L.acc_cap = m / hub + 16;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = up256(off + bytes); return at; };
    L.om2 = take(sizeof(uint32_t) * (size_t)n);
    for (int i = 0; i < 2; i++) L.small[i] = take(sizeof(int32_t) * (size_t)n);
    for (int i = 0; i < 2; i++) L.med[i] = take(sizeof(int32_t) * (size_t)n);
    for (int i = 0; i < 2; i++) L.chunk[i] = take(sizeof(ChunkItem) * (size_t)L.chunk_cap);
    L.acc = take(sizeof(HubAcc) * (size_t)L.acc_cap);
    L.st = take(sizeof(RoundStats));
    L.total = off;
    return L;
}

// Template tables straight from the caller's arrays (no heap use).
const char *noalloc_template(int n0, const uint8_t *labels, int m0, const int32_t *edges,
                             DevTmpl &d, LabelMask &lm) {
    if (n0 < 2 || n0 > kMaxT) return "template must have 2..32 vertices";
    if (m0 < 1 || m0 > CCPM_MAX_TMPL_EDGES || !labels || !edges) return "template needs 1..496 edges";
    std::memset(&d, 0, sizeof(d));
    std::memset(&lm, 0, sizeof(lm));
    d.n0 = n0;
    for (int i = 0; i < m0; i++) {
        int a = edges[2 * i], b = edges[2 * i + 1];
        if (a < 0 || b < 0 || a >= n0 || b >= n0 || a == b) return "bad template edge";
        if ((d.adj[a] >> b) & 1u) return "duplicate template edge";
        d.adj[a] |= 1u << b;
        d.adj[b] |= 1u << a;
    }
    uint32_t seen = 1u, fr = 1u;
    while (fr) {
        uint32_t nx = 0;
        for (int q = 0; q < n0; q++) if ((fr >> q) & 1u) nx |= d.adj[q];
        nx &= ~seen;
        seen |= nx;
        fr = nx;
    }
    if (seen != (n0 == 32 ? 0xFFFFFFFFu : ((1u << n0) - 1u))) return "template is not connected";
    for (int q = 0; q < n0; q++) {
        lm.m[labels[q]] |= 1u << q;
        uint32_t done = 0;
        for (int b = 0; b < n0; b++) {
            if (!((d.adj[q] >> b) & 1u) || ((done >> b) & 1u)) continue;
            uint32_t grp = 0;
            for (int c = 0; c < n0; c++)
                if (((d.adj[q] >> c) & 1u) && labels[c] == labels[b]) grp |= 1u << c;
            done |= grp;
            if (__builtin_popcount(grp) >= 2) {
                if (d.n_cls >= kMaxCls) return "template has more than 32 label-multiplicity classes";
                d.cls_mask[d.n_cls] = grp;
                d.cls_need[d.n_cls] = (uint32_t)__builtin_popcount(grp);
                d.cls_q[d.n_cls] = (uint32_t)q;
                d.n_cls++;
            }
        }
    }
    return nullptr;
}

// The body of the entry point below; it may leave another device current.
int lcc_fixpoint_noalloc_body(int device, void *cuda_stream, int64_t n, int64_t m_dir,
                              const int64_t *row_ptr, const int32_t *col, const uint8_t *labels,
                              int n0, const uint8_t *tmpl_labels, int m0, const int32_t *tmpl_edges,
                              uint32_t *omega, uint32_t *ebits, int32_t *rounds,
                              int64_t *edges_scanned, char *errbuf, size_t errlen) {
    auto fail = [&](int code, const char *msg) {
        if (errbuf && errlen) std::snprintf(errbuf, errlen, "%s", msg);
        return code;
    };
    if (device < 0 || device >= kNoAllocMaxDevices) return fail(CCPM_EINVAL, "device index out of range");
    if (n < 1 || n >= ((int64_t)1 << 31) || m_dir < 0 || !row_ptr || !labels || !omega ||
        (m_dir > 0 && (!col || !ebits)))
        return fail(CCPM_EINVAL, "need 1 <= n < 2^31, m_dir >= 0 and non-NULL device arrays");
    DevTmpl dt;
    LabelMask lm;
    if (const char *why = noalloc_template(n0, tmpl_labels, m0, tmpl_edges, dt, lm)) return fail(CCPM_EINVAL, why);
    const int hub = kDefaultHubDeg;
    const NoAllocLayout L = noalloc_layout(n, m_dir, hub);
    if (L.total > kNoAllocScratchBytes) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "graph too large for the allocation-free entry point: needs %zu bytes of scratch, "
                      "the fixed area holds %zu", L.total, kNoAllocScratchBytes);
        return fail(CCPM_EINVAL, msg);
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(CCPM_ECUDA, cudaGetErrorString(e));
    unsigned char *base = nullptr;
    {
        // once per device, with that device current: the device address of the
        // scratch array (the host-side symbol is only a stand-in)
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[device]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return fail(CCPM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
            g_noalloc_addr[device] = p;
        }
        base = (unsigned char *)g_noalloc_addr[device];
    }
    int num_sms = 0;
    e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return fail(CCPM_ECUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    {
        // the scratch is sized from m_dir: the offsets must agree with it
        // before any kernel writes there (two 8-byte reads into the stack)
        int64_t ends[2] = {-1, -1};
        e = cudaMemcpyAsync(&ends[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(CCPM_ECUDA, cudaGetErrorString(e));
        if (ends[0] != 0 || ends[1] != m_dir) return fail(CCPM_EINVAL, "row_ptr[0] must be 0 and row_ptr[n] == m_dir");
    }
    uint32_t *om[2] = {omega, (uint32_t *)(base + L.om2)};
    int32_t *small[2] = {(int32_t *)(base + L.small[0]), (int32_t *)(base + L.small[1])};
    int32_t *med[2] = {(int32_t *)(base + L.med[0]), (int32_t *)(base + L.med[1])};
    ChunkItem *chunk[2] = {(ChunkItem *)(base + L.chunk[0]), (ChunkItem *)(base + L.chunk[1])};
    HubAcc *acc = (HubAcc *)(base + L.acc);
    RoundStats *st = (RoundStats *)(base + L.st);
    RoundStats hs;
    auto grid = [&](int64_t items, int per_block) {
        int64_t need = (items + per_block - 1) / per_block;
        return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms * 8));
    };
    auto read_stats = [&]() {
        cudaError_t r = cudaMemcpyAsync(&hs, st, sizeof(RoundStats), cudaMemcpyDeviceToHost, s);
        if (r == cudaSuccess) r = cudaStreamSynchronize(s);
        return r;
    };
#define NA_CU(call)                                          \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return fail(CCPM_ECUDA, cudaGetErrorString(e_)); \
    } while (0)
    const int64_t words = (m_dir + 31) / 32;
    // the scratch keeps whatever the previous call left: clear what must start at zero
    NA_CU(cudaMemsetAsync(acc, 0, sizeof(HubAcc) * (size_t)L.acc_cap, s));
    NA_CU(cudaMemsetAsync(st, 0, sizeof(RoundStats), s));
    if (words > 0) {
        NA_CU(cudaMemsetAsync(ebits, 0xFF, sizeof(uint32_t) * (size_t)words, s));
        if (m_dir & 31) k_set_word<<<1, 1, 0, s>>>(ebits + words - 1, (1u << (uint32_t)(m_dir & 31)) - 1u);
    }
    k_init<<<grid(n, 256), 256, 0, s>>>(n, row_ptr, labels, lm, nullptr, om[0], om[1], small[0], med[0], chunk[0], acc,
                                        st, hub, kSmallDeg);
    NA_CU(cudaGetLastError());
    NA_CU(read_stats());
    if (hs.n_hub_slots > (unsigned)L.acc_cap || (int64_t)hs.n_chunk > L.chunk_cap)
        return fail(CCPM_EOVERFLOW, "split-row bookkeeping overflow");
    int64_t n_small = hs.n_small, n_med = hs.n_med, n_chunk = hs.n_chunk, scanned = 0;
    int cur = 0, li = 0;
    int32_t r = 0;
    for (;;) {
        NA_CU(cudaMemsetAsync(st, 0, sizeof(RoundStats), s));
        LccArgs a;
        a.rp = row_ptr;
        a.col = col;
        a.om_cur = om[cur];
        a.om_next = om[cur ^ 1];
        a.ebits = ebits;
        a.small_in = small[li];
        a.med_in = med[li];
        a.chunk_in = chunk[li];
        a.n_small = n_small;
        a.n_med = n_med;
        a.n_chunk = n_chunk;
        a.small_out = small[li ^ 1];
        a.med_out = med[li ^ 1];
        a.chunk_out = chunk[li ^ 1];
        a.acc = acc;
        a.st = st;
        a.hub_deg = hub;
        a.deg = nullptr;
        a.med_chunk = 1;
        a.small_chunk = 8;
        a.lab0 = nullptr;
        a.elab = nullptr;
        a.sparse = 0;
        a.prev = nullptr;
        a.resident_warps = num_sms * 32;
        a.eta_off = 0u;
        a.nw_bytes = 0;
        a.nw_cur = nullptr;
        a.nw_next = nullptr;
        const int g = grid((n_chunk + n_med + (n_small + 7) / 8) * 32, 256);
        if (dt.n_cls == 0) k_lcc_round<0, false><<<g, 256, 0, s>>>(a, dt);
        else if (dt.n_cls <= 4) k_lcc_round<4, false><<<g, 256, 0, s>>>(a, dt);
        else k_lcc_round<32, false><<<g, 256, 0, s>>>(a, dt);
        NA_CU(cudaGetLastError());
        NA_CU(read_stats());
        r++;
        scanned += (int64_t)hs.scanned;
        n_small = hs.n_small;
        n_med = hs.n_med;
        n_chunk = hs.n_chunk;
        li ^= 1;
        cur ^= 1;
        if (!hs.changed) break;
        if (r > 4 * (m_dir + n) + 8) return fail(CCPM_ETIMEOUT, "LCC did not converge");
    }
    // both omega buffers agree at the fixpoint; the caller's buffer must hold it
    if (cur != 0) NA_CU(cudaMemcpyAsync(omega, om[cur], sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    if (m_dir > 0) {
        k_materialize<<<grid(n * 32, 256), 256, 0, s>>>(n, omega, row_ptr, col, ebits);
        NA_CU(cudaGetLastError());
    }
    NA_CU(cudaStreamSynchronize(s));
#undef NA_CU
    if (rounds) *rounds = r;
    if (edges_scanned) *edges_scanned = scanned;
    return CCPM_OK;
}

}  // namespace

// The caller's current device is the same after the call as before it.
extern "C" int ccpm_lcc_fixpoint_noalloc(int device, void *cuda_stream, int64_t n, int64_t m_dir,
                                         const int64_t *row_ptr, const int32_t *col, const uint8_t *labels,
                                         int n0, const uint8_t *tmpl_labels, int m0, const int32_t *tmpl_edges,
                                         uint32_t *omega, uint32_t *ebits, int32_t *rounds,
                                         int64_t *edges_scanned, char *errbuf, size_t errlen) {
    if (errbuf && errlen) errbuf[0] = '\0';
    int prev = -1;
    const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
    const int rc = lcc_fixpoint_noalloc_body(device, cuda_stream, n, m_dir, row_ptr, col, labels, n0, tmpl_labels,
                                             m0, tmpl_edges, omega, ebits, rounds, edges_scanned, errbuf, errlen);
    if (have_prev && prev != device) cudaSetDevice(prev);
    return rc;
}
