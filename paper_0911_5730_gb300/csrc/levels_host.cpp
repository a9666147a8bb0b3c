// levels_host.cpp - host-side structure of one decomposition level.
//
// Everything here is index bookkeeping done once per setup: which DOFs each
// substructure holds, the interface / corner / edge classification, the
// interior ordering with its block structure, and the flattened per-
// substructure index maps uploaded to the device.  No floating-point work of
// the method happens here.
#include "levels_host.h"

#include <algorithm>
#include <map>
#include <numeric>
#include <queue>
#include <stdexcept>

namespace bddc {

namespace {

struct DSU {
    std::vector<int> p;
    explicit DSU(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
    int find(int x) {
        while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
        return x;
    }
    void unite(int a, int b) {
        a = find(a); b = find(b);
        if (a != b) { if (a < b) p[b] = a; else p[a] = b; }
    }
};

// Bandwidth of an ordering (ord[k] = node) on an undirected graph.
int bandwidth(const std::vector<std::vector<int>> &adj, const std::vector<int> &ord) {
    std::vector<int> pos(adj.size());
    for (size_t k = 0; k < ord.size(); ++k) pos[ord[k]] = (int)k;
    int bw = 0;
    for (size_t u = 0; u < adj.size(); ++u)
        for (int v : adj[u]) bw = std::max(bw, std::abs(pos[u] - pos[v]));
    return bw;
}

// Reverse Cuthill-McKee ordering, every connected component in turn.
std::vector<int> rcm(const std::vector<std::vector<int>> &adj) {
    const int n = (int)adj.size();
    std::vector<int> order;
    std::vector<char> seen(n, 0);
    std::vector<int> deg(n);
    for (int i = 0; i < n; ++i) deg[i] = (int)adj[i].size();
    auto bfs_last = [&](int start, std::vector<int> &lev) {
        std::vector<int> dist(n, -1);
        std::queue<int> q;
        q.push(start); dist[start] = 0;
        int last = start;
        while (!q.empty()) {
            int u = q.front(); q.pop();
            last = u;
            for (int v : adj[u]) if (dist[v] < 0) { dist[v] = dist[u] + 1; q.push(v); }
        }
        lev = dist;
        return last;
    };
    for (int root = 0; root < n; ++root) {
        if (seen[root]) continue;
        // pseudo-peripheral start: two BFS sweeps from the lowest-degree node of the component
        std::vector<int> lev;
        bfs_last(root, lev);
        int start = root;
        for (int i = 0; i < n; ++i)
            if (lev[i] >= 0 && deg[i] < deg[start]) start = i;
        int far = bfs_last(start, lev);
        bfs_last(far, lev);
        start = far;
        std::vector<int> comp;
        std::queue<int> q;
        q.push(start); seen[start] = 1;
        while (!q.empty()) {
            int u = q.front(); q.pop();
            comp.push_back(u);
            std::vector<int> nb;
            for (int v : adj[u]) if (!seen[v]) { seen[v] = 1; nb.push_back(v); }
            std::sort(nb.begin(), nb.end(), [&](int a, int b) {
                return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
            });
            for (int v : nb) q.push(v);
        }
        std::reverse(comp.begin(), comp.end());
        order.insert(order.end(), comp.begin(), comp.end());
    }
    return order;
}

// Smallest uniform block size b for which every coupling stays within the
// same or the neighbouring block.
int min_block(const std::vector<std::vector<int>> &adj, const std::vector<int> &ord) {
    const int n = (int)ord.size();
    if (n == 0) return 1;
    std::vector<int> pos(n), first(n);
    for (int k = 0; k < n; ++k) pos[ord[k]] = k;
    for (int k = 0; k < n; ++k) {
        int f = k;
        for (int v : adj[ord[k]]) f = std::min(f, pos[v]);
        first[k] = f;
    }
    for (int b = 1; b <= n; ++b) {
        bool ok = true;
        for (int k = 0; k < n && ok; ++k) ok = (k / b - first[k] / b) <= 1;
        if (ok) return b;
    }
    return n;
}

}  // namespace

void HLevel::build() {
    if ((int)esub.size() != nelem || (int64_t)eptr.size() != nelem + 1)
        throw Error(BDDC_E_ARG, "level: inconsistent element arrays");
    sub_elems.assign(nsub, {});
    for (int e = 0; e < nelem; ++e) {
        if (esub[e] < 0 || esub[e] >= nsub) throw Error(BDDC_E_ARG, "element assigned to an invalid substructure");
        sub_elems[esub[e]].push_back(e);
    }
    sub_dofs.assign(nsub, {});
    for (int s = 0; s < nsub; ++s) {
        if (sub_elems[s].empty()) throw Error(BDDC_E_ARG, "empty substructure " + std::to_string(s));
        auto &d = sub_dofs[s];
        for (int e : sub_elems[s])
            for (int64_t k = eptr[e]; k < eptr[e + 1]; ++k)
                if (eslot[k] >= 0) d.push_back(eslot[k]);
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
    }
    subs_ptr.assign(n + 1, 0);
    for (int s = 0; s < nsub; ++s) for (int g : sub_dofs[s]) subs_ptr[g + 1]++;
    for (int g = 0; g < n; ++g) subs_ptr[g + 1] += subs_ptr[g];
    subs_idx.assign(subs_ptr[n], 0);
    {
        std::vector<int64_t> fill(subs_ptr.begin(), subs_ptr.end() - 1);
        for (int s = 0; s < nsub; ++s) for (int g : sub_dofs[s]) subs_idx[fill[g]++] = s;
    }
    if (!dbnd.empty() && (int)dbnd.size() != n) throw Error(BDDC_E_ARG, "level: boundary flags of the wrong size");
    if (!comp.empty() && (int)comp.size() != n) throw Error(BDDC_E_ARG, "level: components of the wrong size");
    is_iface.assign(n, 0); is_corner.assign(n, 0);
    corners.clear();
    // corners: in three or more substructures, or an interface DOF on the
    // boundary of the domain (where an edge ends on a free side)
    for (int g = 0; g < n; ++g) {
        const int m = mult(g);
        is_iface[g] = m >= 2;
        is_corner[g] = m >= 3 || (m >= 2 && !dbnd.empty() && dbnd[g]);
        if (is_corner[g]) corners.push_back(g);
    }
    // Edges: connected chains of non-corner interface DOFs shared by one pair.
    DSU dsu(n);
    for (int e = 0; e < nelem; ++e) {
        for (int64_t a = eptr[e]; a < eptr[e + 1]; ++a) {
            const int ga = eslot[a];
            if (ga < 0 || !is_iface[ga] || is_corner[ga]) continue;
            for (int64_t b = a + 1; b < eptr[e + 1]; ++b) {
                const int gb = eslot[b];
                if (gb < 0 || !is_iface[gb] || is_corner[gb]) continue;
                if (subs(ga) == subs(gb)) dsu.unite(ga, gb);
            }
        }
    }
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;   // (s, t, root)
    for (int g = 0; g < n; ++g) {
        if (!is_iface[g] || is_corner[g]) continue;
        auto sv = subs(g);
        groups[{sv[0], sv[1], dsu.find(g)}].push_back(g);
    }
    edges.clear();
    for (auto &kv : groups) {
        Edge ed;
        ed.s = std::get<0>(kv.first);
        ed.t = std::get<1>(kv.first);
        ed.dofs = kv.second;   // ascending
        edges.push_back(std::move(ed));
    }
    // map keys are (s, t, root) with root = smallest DOF of the chain, so the
    // edges come out ordered by pair, then by lowest DOF.
    floating.assign(nsub, 1);
    for (int e = 0; e < nelem; ++e) if (ebnd[e]) floating[esub[e]] = 0;

    // interior / interface orderings and block structure
    Iord.assign(nsub, {}); Gord.assign(nsub, {});
    bw.assign(nsub, 0); bsz.assign(nsub, 1); nblk.assign(nsub, 0);
    std::vector<int> loc(n, -1);
    std::vector<std::vector<int>> first_all(nsub);   // lowest coupled position per row
    for (int s = 0; s < nsub; ++s) {
        std::vector<int> I;
        for (int g : sub_dofs[s]) (is_iface[g] ? Gord[s] : I).push_back(g);
        for (size_t k = 0; k < I.size(); ++k) loc[I[k]] = (int)k;
        std::vector<std::vector<int>> adj(I.size());
        for (int e : sub_elems[s]) {
            for (int64_t a = eptr[e]; a < eptr[e + 1]; ++a) {
                const int ga = eslot[a];
                if (ga < 0 || loc[ga] < 0) continue;
                for (int64_t b = eptr[e]; b < eptr[e + 1]; ++b) {
                    const int gb = eslot[b];
                    if (gb < 0 || loc[gb] < 0 || gb == ga) continue;
                    adj[loc[ga]].push_back(loc[gb]);
                }
            }
        }
        for (auto &v : adj) { std::sort(v.begin(), v.end()); v.erase(std::unique(v.begin(), v.end()), v.end()); }
        std::vector<int> natural(I.size());
        std::iota(natural.begin(), natural.end(), 0);
        std::vector<int> best = natural;
        int bwn = bandwidth(adj, natural);
        int bn = min_block(adj, natural);
        if (!I.empty()) {
            std::vector<int> r = rcm(adj);
            const int br = min_block(adj, r);
            if (br < bn) { best = r; bn = br; bwn = bandwidth(adj, r); }
        }
        Iord[s].resize(I.size());
        for (size_t k = 0; k < I.size(); ++k) Iord[s][k] = I[best[k]];
        {
            std::vector<int> pos(I.size());
            for (size_t k = 0; k < I.size(); ++k) pos[best[k]] = (int)k;
            auto &fst = first_all[s];
            fst.resize(I.size());
            for (size_t k = 0; k < I.size(); ++k) {
                int f = (int)k;
                for (int v : adj[best[k]]) f = std::min(f, pos[v]);
                fst[k] = f;
            }
        }
        for (int g : I) loc[g] = -1;
        bw[s] = std::max(bwn, 0);
        bsz[s] = std::max(bn, 1);
        nblk[s] = I.empty() ? 0 : (int)((I.size() + bsz[s] - 1) / bsz[s]);
    }
    // Prefer one power-of-two block size for the whole level (the apply
    // kernels then unroll the block solves completely).
    block_uniform = 0;
    int bmax = 1;
    for (int s = 0; s < nsub; ++s) bmax = std::max(bmax, bsz[s]);
    int bp = 1;
    while (bp < bmax) bp *= 2;
    if (bp < 8) bp = 8;
    if (bp <= 32) {
        bool ok = true;
        for (int s = 0; s < nsub && ok; ++s) {
            const auto &fst = first_all[s];
            for (size_t k = 0; k < fst.size() && ok; ++k) ok = ((int)k / bp - fst[k] / bp) <= 1;
        }
        if (ok) {
            block_uniform = bp;
            for (int s = 0; s < nsub; ++s) {
                bsz[s] = bp;
                nblk[s] = Iord[s].empty() ? 0 : (int)((Iord[s].size() + bp - 1) / bp);
            }
        }
    }
    iface_id.assign(n, -1);
    iface_dof.clear();
    for (int g = 0; g < n; ++g)
        if (is_iface[g]) { iface_id[g] = (int)iface_dof.size(); iface_dof.push_back(g); }
}

std::vector<int> HLevel::subs(int g) const {
    return std::vector<int>(subs_idx.begin() + subs_ptr[g], subs_idx.begin() + subs_ptr[g + 1]);
}

}  // namespace bddc
