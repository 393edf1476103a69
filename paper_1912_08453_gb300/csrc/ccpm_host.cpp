// ccpm_host.cpp -- host-side template logic: validation, non-local constraint
// generation (Table 3 Steps 1-5 with Alg. 2, ordering of Section 4.2),
// label-preserving automorphisms, and the search plans the kernels walk.
//
// Everything here is integer work on a template of at most 32 vertices; it runs
// in microseconds and needs no GPU.
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <set>

#include "ccpm_internal.h"

namespace ccpm {

namespace {

using Edge = std::pair<int, int>;

inline Edge norm(int a, int b) { return a < b ? Edge(a, b) : Edge(b, a); }

inline int popc(uint32_t x) { return __builtin_popcount(x); }

bool connected(int n0, const uint32_t *adj) {
    uint32_t seen = 1u, frontier = 1u;
    while (frontier) {
        uint32_t next = 0;
        for (int q = 0; q < n0; q++)
            if ((frontier >> q) & 1u) next |= adj[q];
        next &= ~seen;
        seen |= next;
        frontier = next;
    }
    uint32_t all = n0 == 32 ? 0xFFFFFFFFu : ((1u << n0) - 1u);
    return seen == all;
}

// Canonical simple cycles of the subgraph induced by `vset` (edges `eset`):
// each cycle once, written from its smallest vertex with the second vertex
// smaller than the last; returned in lexicographic order of that sequence.
void cycles_of(const uint32_t *adj_sub, uint32_t vset, std::vector<std::vector<int>> &out,
               size_t cap, bool &too_many) {
    std::vector<int> path;
    uint32_t onpath = 0;
    auto rec = [&](auto &&self, int start) -> void {
        int x = path.back();
        for (int y = 0; y < kMaxT; y++) {
            if (!((adj_sub[x] >> y) & 1u)) continue;
            if (y == start) {
                if (path.size() >= 3 && path[1] < path.back()) {
                    out.push_back(path);
                    if (out.size() > cap) { too_many = true; return; }
                }
            } else if (y > start && !((onpath >> y) & 1u)) {
                path.push_back(y);
                onpath |= 1u << y;
                self(self, start);
                onpath &= ~(1u << y);
                path.pop_back();
                if (too_many) return;
            }
        }
    };
    for (int s = 0; s < kMaxT && !too_many; s++) {
        if (!((vset >> s) & 1u)) continue;
        path.assign(1, s);
        onpath = 1u << s;
        rec(rec, s);
    }
    std::sort(out.begin(), out.end());
}

// Lexicographically smallest shortest path src -> dst in the template, or
// empty if unreachable.
std::vector<int> lex_shortest_path(int n0, const uint32_t *adj, int src, int dst) {
    int dist[kMaxT];
    for (int i = 0; i < kMaxT; i++) dist[i] = -1;
    std::deque<int> q;
    dist[dst] = 0;
    q.push_back(dst);
    while (!q.empty()) {
        int x = q.front();
        q.pop_front();
        for (int y = 0; y < n0; y++)
            if (((adj[x] >> y) & 1u) && dist[y] < 0) { dist[y] = dist[x] + 1; q.push_back(y); }
    }
    std::vector<int> path;
    if (dist[src] < 0) return path;
    int x = src;
    path.push_back(x);
    while (x != dst) {
        int nxt = -1;
        for (int y = 0; y < n0; y++)
            if (((adj[x] >> y) & 1u) && dist[y] == dist[x] - 1) { nxt = y; break; }
        x = nxt;
        path.push_back(x);
    }
    return path;
}

struct Sub {
    uint32_t v = 0;
    std::set<Edge> e;
};

// BFS spanning tree of a substructure from its lowest-id vertex, neighbours
// visited in increasing id (Alg. 2's SPANNING_TREE for path-derived unions).
std::set<Edge> spanning_tree(const Sub &s) {
    uint32_t adj[kMaxT] = {};
    for (auto &e : s.e) { adj[e.first] |= 1u << e.second; adj[e.second] |= 1u << e.first; }
    int root = __builtin_ctz(s.v);
    uint32_t seen = 1u << root;
    std::deque<int> q{root};
    std::set<Edge> tree;
    while (!q.empty()) {
        int x = q.front();
        q.pop_front();
        for (int y = 0; y < kMaxT; y++) {
            if (((adj[x] >> y) & 1u) && !((seen >> y) & 1u)) {
                seen |= 1u << y;
                tree.insert(norm(x, y));
                q.push_back(y);
            }
        }
    }
    return tree;
}

bool share_edge(const std::set<Edge> &a, const std::set<Edge> &b) {
    for (auto &e : a) if (b.count(e)) return true;
    return false;
}

// Alg. 2 with the reading: merge the first mergeable pair in index order,
// repeat until none merges.  mode 0: cycles (shared vertex and shared edge),
// 1: paths (shared vertex; spanning tree afterwards), 2: mixed (shared vertex).
std::vector<Sub> tds_union(std::vector<Sub> w, int mode) {
    for (;;) {
        bool merged = false;
        for (size_t i = 0; i < w.size() && !merged; i++) {
            for (size_t j = i + 1; j < w.size(); j++) {
                if (!(w[i].v & w[j].v)) continue;
                if (mode == 0 && !share_edge(w[i].e, w[j].e)) continue;
                w[i].v |= w[j].v;
                w[i].e.insert(w[j].e.begin(), w[j].e.end());
                w.erase(w.begin() + (long)j);
                merged = true;
                break;
            }
        }
        if (!merged) break;
    }
    if (mode == 1)
        for (auto &s : w) s.e = spanning_tree(s);
    return w;
}

}  // namespace

int template_build(Template &t, int n0, const uint8_t *labels, int m0, const int32_t *edges) {
    if (n0 < 2 || n0 > kMaxT) { t.err = "template must have 2..32 vertices"; return CCPM_EINVAL; }
    if (m0 < 1 || m0 > CCPM_MAX_TMPL_EDGES || !labels || !edges) {
        t.err = "template needs 1..496 edges and non-NULL arrays";
        return CCPM_EINVAL;
    }
    t.n0 = n0;
    std::memcpy(t.labels, labels, (size_t)n0);
    std::memset(t.adj, 0, sizeof(t.adj));
    t.edges.clear();
    for (int i = 0; i < m0; i++) {
        int a = edges[2 * i], b = edges[2 * i + 1];
        if (a < 0 || b < 0 || a >= n0 || b >= n0) { t.err = "template edge endpoint out of range"; return CCPM_EINVAL; }
        if (a == b) { t.err = "template self loop"; return CCPM_EINVAL; }
        if ((t.adj[a] >> b) & 1u) { t.err = "duplicate template edge"; return CCPM_EINVAL; }
        t.adj[a] |= 1u << b;
        t.adj[b] |= 1u << a;
        t.edges.push_back(norm(a, b));
    }
    if (!connected(n0, t.adj)) { t.err = "template is not connected"; return CCPM_EINVAL; }
    int n_cls = 0;
    for (int q = 0; q < n0; q++) {
        uint32_t done = 0;
        for (int b = 0; b < n0; b++) {
            if (!((t.adj[q] >> b) & 1u) || ((done >> b) & 1u)) continue;
            uint32_t grp = 0;
            for (int c = 0; c < n0; c++)
                if (((t.adj[q] >> c) & 1u) && labels[c] == labels[b]) grp |= 1u << c;
            done |= grp;
            if (popc(grp) >= 2) n_cls++;
        }
    }
    if (n_cls > kMaxCls) { t.err = "template has more than 32 label-multiplicity classes"; return CCPM_EINVAL; }
    t.automorphisms = count_automorphisms(t);
    t.generated = false;
    t.k0.clear();
    t.order.clear();
    return CCPM_OK;
}

uint64_t count_automorphisms(const Template &t) {
    int img[kMaxT];
    uint32_t used = 0;
    uint64_t total = 0;
    auto rec = [&](auto &&self, int i) -> void {
        if (i == t.n0) { total++; return; }
        for (int x = 0; x < t.n0; x++) {
            if (((used >> x) & 1u) || t.labels[x] != t.labels[i]) continue;
            bool ok = true;
            for (int j = 0; j < i && ok; j++)
                if ((((t.adj[i] >> j) & 1u) != 0) != (((t.adj[x] >> img[j]) & 1u) != 0)) ok = false;
            if (!ok) continue;
            img[i] = x;
            used |= 1u << x;
            self(self, i + 1);
            used &= ~(1u << x);
        }
    };
    rec(rec, 0);
    return total;
}

int constraints_generate(Template &t, std::string &err) {
    const int n0 = t.n0;
    int label_count[256] = {};
    for (int q = 0; q < n0; q++) label_count[t.labels[q]]++;
    // Step 1: vertices with a unique label that are leaves are left to LCC.
    uint32_t v_u = 0, v_ul = 0;
    for (int q = 0; q < n0; q++) {
        if (label_count[t.labels[q]] == 1) {
            v_u |= 1u << q;
            if (popc(t.adj[q]) == 1) v_ul |= 1u << q;
        }
    }
    uint32_t all = n0 == 32 ? 0xFFFFFFFFu : ((1u << n0) - 1u);
    uint32_t v1 = all & ~v_ul;
    uint32_t adj1[kMaxT] = {};
    for (int q = 0; q < n0; q++)
        if ((v1 >> q) & 1u) adj1[q] = t.adj[q] & v1;
    // Step 2: duplicate-label vertices.
    uint32_t v_d = all & ~v_u;
    // Step 3: one cycle constraint per simple cycle of G'_0.
    std::vector<std::vector<int>> cyc;
    bool too_many = false;
    cycles_of(adj1, v1, cyc, 4096, too_many);
    if (too_many) { err = "template has more than 4096 simple cycles"; return CCPM_EINVAL; }
    std::vector<Sub> cc, pc;
    for (auto &c : cyc) {
        Sub s;
        for (size_t i = 0; i < c.size(); i++) {
            s.v |= 1u << c[i];
            s.e.insert(norm(c[i], c[(i + 1) % c.size()]));
        }
        cc.push_back(s);
    }
    // Step 4: a shortest path for every same-label pair three or more hops
    // apart, unless one cycle constraint already covers all its edges.
    for (int i = 0; i < n0; i++) {
        if (!((v_d >> i) & 1u)) continue;
        for (int j = i + 1; j < n0; j++) {
            if (!((v_d >> j) & 1u) || t.labels[i] != t.labels[j]) continue;
            std::vector<int> p = lex_shortest_path(n0, t.adj, i, j);
            if (p.size() < 4) continue;   // fewer than 3 hops
            Sub s;
            for (size_t k = 0; k < p.size(); k++) {
                s.v |= 1u << p[k];
                if (k + 1 < p.size()) s.e.insert(norm(p[k], p[k + 1]));
            }
            bool covered = false;
            for (auto &c : cc) {
                bool all_in = true;
                for (auto &e : s.e) if (!c.e.count(e)) { all_in = false; break; }
                if (all_in) { covered = true; break; }
            }
            if (!covered) pc.push_back(s);
        }
    }
    // Step 5: TDS unions.
    std::vector<Sub> tcc = tds_union(cc, 0);
    std::vector<Sub> tpc = tds_union(pc, 1);
    std::vector<Sub> mix = tcc;
    mix.insert(mix.end(), tpc.begin(), tpc.end());
    std::vector<Sub> tds = tds_union(mix, 2);
    // K0 = PC + CC + TDS_CC + TDS_PC + TDS without exact duplicates.
    std::vector<HostConstraint> k0;
    std::set<std::pair<uint32_t, std::set<Edge>>> seen;
    auto add = [&](const std::vector<Sub> &lst, int kind) {
        for (auto &s : lst) {
            auto key = std::make_pair(s.v, s.e);
            if (seen.count(key)) continue;
            seen.insert(key);
            HostConstraint c;
            c.kind = kind;
            c.vmask = s.v;
            c.edges.assign(s.e.begin(), s.e.end());
            c.gen_index = (int)k0.size();
            // token issuers (Section 4.2 "Token Generation")
            if (kind == CCPM_KIND_CC || kind == CCPM_KIND_TDS_CC) {
                c.hmask = s.v;
            } else if (kind == CCPM_KIND_PC) {
                uint32_t ends = 0;
                for (int q = 0; q < kMaxT; q++) {
                    if (!((s.v >> q) & 1u)) continue;
                    int d = 0;
                    for (auto &e : s.e) d += (e.first == q) + (e.second == q);
                    if (d == 1) ends |= 1u << q;
                }
                c.hmask = ends;
            } else {
                uint32_t dup = s.v & v_d;
                c.hmask = dup ? dup : s.v;
            }
            k0.push_back(c);
        }
    };
    add(pc, CCPM_KIND_PC);
    add(cc, CCPM_KIND_CC);
    add(tcc, CCPM_KIND_TDS_CC);
    add(tpc, CCPM_KIND_TDS_PC);
    add(tds, CCPM_KIND_TDS);
    // Section 4.2: paths and cycles before TDS, shorter walks first.
    std::stable_sort(k0.begin(), k0.end(), [](const HostConstraint &a, const HostConstraint &b) {
        int ta = a.kind >= CCPM_KIND_TDS_CC, tb = b.kind >= CCPM_KIND_TDS_CC;
        if (ta != tb) return ta < tb;
        if (a.edges.size() != b.edges.size()) return a.edges.size() < b.edges.size();
        if (a.kind != b.kind) return a.kind < b.kind;
        return a.gen_index < b.gen_index;
    });
    t.k0 = k0;
    t.order.clear();
    for (int i = 0; i < (int)k0.size(); i++) t.order.push_back(i);
    t.generated = true;
    return CCPM_OK;
}

void build_dev_tmpl(const Template &t, DevTmpl &d) {
    std::memset(&d, 0, sizeof(d));
    d.n0 = t.n0;
    for (int q = 0; q < t.n0; q++) d.adj[q] = t.adj[q];
    int n = 0;
    for (int q = 0; q < t.n0; q++) {
        uint32_t done = 0;
        for (int b = 0; b < t.n0; b++) {
            if (!((t.adj[q] >> b) & 1u) || ((done >> b) & 1u)) continue;
            uint32_t grp = 0;
            for (int c = 0; c < t.n0; c++)
                if (((t.adj[q] >> c) & 1u) && t.labels[c] == t.labels[b]) grp |= 1u << c;
            done |= grp;
            if (popc(grp) >= 2 && n < kMaxCls) {
                d.cls_mask[n] = grp;
                d.cls_need[n] = (uint32_t)popc(grp);
                d.cls_q[n] = (uint32_t)q;
                n++;
            }
        }
    }
    d.n_cls = n;
}

void build_plan(const Template &t, uint32_t svert, const uint32_t *sadj, int root,
                const int64_t *label_freq, bool with_marks, DevPlan &p, int second,
                const unsigned long long *qlive) {
    std::memset(&p, 0, sizeof(p));
    int pos_of[kMaxT];
    for (int i = 0; i < kMaxT; i++) pos_of[i] = -1;
    int k = 0;
    p.q[k] = (int8_t)root;
    p.lab[k] = t.labels[root];
    p.par[k] = -1;
    pos_of[root] = k++;
    uint32_t placed = 1u << root;
    while (placed != svert) {
        int best = -1, best_links = -1;
        int64_t best_freq = 0;
        for (int q = 0; q < kMaxT; q++) {
            if (!((svert >> q) & 1u) || ((placed >> q) & 1u)) continue;
            int links = popc(sadj[q] & placed);
            if (links == 0) continue;
            int64_t f = qlive ? (int64_t)qlive[q] : (label_freq ? label_freq[t.labels[q]] : 0);
            if (links > best_links || (links == best_links && f < best_freq)) {
                best = q; best_links = links; best_freq = f;
            }
        }
        if (k == 1 && second >= 0) best = second;    // edge-rooted plan: position 1 is fixed
        if (best < 0) break;   // S disconnected: cannot happen for generated constraints
        int parent_pos = kMaxT;
        uint32_t back = 0, same = 0;
        for (int j = 0; j < k; j++) {
            int qj = p.q[j];
            if ((sadj[best] >> qj) & 1u) {
                if (parent_pos == kMaxT) parent_pos = j; else back |= 1u << j;
            }
            if (t.labels[qj] == t.labels[best]) same |= 1u << j;
        }
        p.q[k] = (int8_t)best;
        p.lab[k] = t.labels[best];
        p.nbr[k] = back | (1u << parent_pos);
        p.par[k] = (int8_t)parent_pos;
        p.back[k] = back;
        p.same[k] = same;
        pos_of[best] = k++;
        placed |= 1u << best;
    }
    p.k = k;
    if (with_marks) {
        int n = 0;
        for (auto &e : t.edges) {
            if (pos_of[e.first] < 0 || pos_of[e.second] < 0) continue;
            p.mark_a[n] = (int8_t)pos_of[e.first];
            p.mark_b[n] = (int8_t)pos_of[e.second];
            n++;
        }
        p.n_marks = n;
    }
}

}  // namespace ccpm
