// partition.cpp - the graph partitioner of Algorithm 2's first step:
// substructures with roughly equal weight (DOFs), few cut edges, weights on
// vertices and on edges.  Multilevel recursive bisection, host code:
//   coarsen   heavy-edge matching, visiting vertices in a seeded order, until
//             the graph is small or stops shrinking;
//   bisect    greedy graph growing from several peripheral seeds to the
//             target weight, the lowest cut kept;
//   refine    Fiduccia-Mattheyses passes at every level on the way back up
//             (boundary vertices in a max-gain heap, moves within the balance
//             bound, the best prefix of each pass kept);
//   k parts   recursive bisection with targets in proportion to the parts on
//             each side;
//   connect   pieces of a part that are not connected to its largest piece
//             join the neighbouring part they share most edge weight with.
#include "partition.h"

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <queue>
#include <vector>

namespace bddc {

namespace {

struct G {
    int n = 0;
    std::vector<int64_t> xadj;   // n + 1
    std::vector<int> adj, ew;    // edges (both directions)
    std::vector<int64_t> vw;     // vertex weights
    int64_t total() const { return std::accumulate(vw.begin(), vw.end(), int64_t(0)); }
};

// splitmix64: a seeded, platform-independent order for the matching
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// One level of heavy-edge matching; cmap[v] = coarse vertex of v.
G coarsen_once(const G &g, Rng &rng, std::vector<int> &cmap) {
    std::vector<int> order(g.n);
    std::iota(order.begin(), order.end(), 0);
    for (int i = g.n - 1; i > 0; --i) std::swap(order[i], order[(int)(rng.next() % (uint64_t)(i + 1))]);
    std::vector<int> match(g.n, -1);
    for (int v : order) {
        if (match[v] >= 0) continue;
        int best = v, bw = -1;
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
            const int u = g.adj[e];
            if (match[u] < 0 && u != v && g.ew[e] > bw) { bw = g.ew[e]; best = u; }
        }
        match[v] = best;
        match[best] = v;
    }
    cmap.assign(g.n, -1);
    int nc = 0;
    for (int v = 0; v < g.n; ++v)
        if (cmap[v] < 0) { cmap[v] = nc; cmap[match[v]] = nc; ++nc; }
    G c;
    c.n = nc;
    c.vw.assign(nc, 0);
    for (int v = 0; v < g.n; ++v) c.vw[cmap[v]] += g.vw[v];
    std::vector<std::vector<int>> members(nc);
    for (int v = 0; v < g.n; ++v) members[cmap[v]].push_back(v);
    std::vector<int> mark(nc, -1), pos(nc, 0);
    c.xadj.assign(nc + 1, 0);
    for (int cv = 0; cv < nc; ++cv) {
        for (int v : members[cv])
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
                const int cu = cmap[g.adj[e]];
                if (cu == cv) continue;
                if (mark[cu] != cv) {
                    mark[cu] = cv;
                    pos[cu] = (int)c.adj.size();
                    c.adj.push_back(cu);
                    c.ew.push_back(g.ew[e]);
                } else {
                    c.ew[pos[cu]] += g.ew[e];
                }
            }
        c.xadj[cv + 1] = (int64_t)c.adj.size();
    }
    return c;
}

int64_t cut_of(const G &g, const std::vector<char> &side) {
    int64_t c = 0;
    for (int v = 0; v < g.n; ++v)
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e)
            if (side[v] != side[g.adj[e]]) c += g.ew[e];
    return c / 2;
}

// A vertex far from `start` (the last one a breadth-first search reaches).
int far_vertex(const G &g, int start) {
    std::vector<int> dist(g.n, -1);
    std::queue<int> q;
    q.push(start);
    dist[start] = 0;
    int last = start;
    while (!q.empty()) {
        const int v = q.front();
        q.pop();
        last = v;
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e)
            if (dist[g.adj[e]] < 0) { dist[g.adj[e]] = dist[v] + 1; q.push(g.adj[e]); }
    }
    return last;
}

// Fiduccia-Mattheyses refinement of a bisection: side 0 should weigh
// target0, each side at most its target times (1 + eps).
void fm_refine(const G &g, std::vector<char> &side, int64_t target0, double eps, int passes) {
    const int64_t tot = g.total();
    const int64_t max0 = (int64_t)((double)target0 * (1.0 + eps)) + 1;
    const int64_t max1 = (int64_t)((double)(tot - target0) * (1.0 + eps)) + 1;
    std::vector<int64_t> gain(g.n);
    for (int pass = 0; pass < passes; ++pass) {
        int64_t w0 = 0;
        for (int v = 0; v < g.n; ++v) if (!side[v]) w0 += g.vw[v];
        for (int v = 0; v < g.n; ++v) {
            int64_t gv = 0;
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) gv += side[g.adj[e]] != side[v] ? g.ew[e] : -g.ew[e];
            gain[v] = gv;
        }
        using Item = std::pair<int64_t, int>;          // (gain, vertex), max first
        std::priority_queue<Item> heap[2];
        for (int v = 0; v < g.n; ++v) {
            bool bnd = false;
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1] && !bnd; ++e) bnd = side[g.adj[e]] != side[v];
            if (bnd) heap[(int)side[v]].push({gain[v], v});
        }
        std::vector<char> locked(g.n, 0);
        std::vector<int> moved;
        int64_t cur = 0, best = 0;
        size_t best_len = 0;
        // the balance improves or stays in bounds with every kept move
        auto over = [&](int64_t a0) { return std::max<int64_t>(0, a0 - max0) + std::max<int64_t>(0, (tot - a0) - max1); };
        int64_t best_over = over(w0);
        int stall = 0;
        const int limit = std::min(1000, std::max(64, g.n / 50));   // moves past the best before giving up
        while (stall < limit) {
            // pick the side to move from: the heavier one if out of balance,
            // else the better top gain that keeps the balance
            int from = -1;
            Item top[2] = {{INT64_MIN, -1}, {INT64_MIN, -1}};
            for (int sd = 0; sd < 2; ++sd) {
                while (!heap[sd].empty()) {
                    const Item it = heap[sd].top();
                    if (locked[it.second] || side[it.second] != sd || it.first != gain[it.second]) { heap[sd].pop(); continue; }
                    top[sd] = it;
                    break;
                }
            }
            const int64_t vwt[2] = {top[0].second >= 0 ? g.vw[top[0].second] : 0,
                                    top[1].second >= 0 ? g.vw[top[1].second] : 0};
            // a move keeps the other side in bounds and never empties a side
            const bool can0 = top[0].second >= 0 && w0 - vwt[0] > 0;
            const bool can1 = top[1].second >= 0 && tot - w0 - vwt[1] > 0;
            const bool ok0 = can0 && tot - w0 + vwt[0] <= max1;
            const bool ok1 = can1 && w0 + vwt[1] <= max0;
            if (w0 > max0 && can0) from = 0;
            else if (tot - w0 > max1 && can1) from = 1;
            else if (ok0 && ok1) from = top[0].first >= top[1].first ? 0 : 1;
            else if (ok0) from = 0;
            else if (ok1) from = 1;
            if (from < 0) break;
            const int v = top[from].second;
            heap[from].pop();
            locked[v] = 1;
            side[v] = (char)(1 - from);
            w0 += from == 0 ? -g.vw[v] : g.vw[v];
            cur += gain[v];
            moved.push_back(v);
            gain[v] = -gain[v];
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
                const int u = g.adj[e];
                gain[u] += side[u] == side[v] ? -2 * g.ew[e] : 2 * g.ew[e];
                if (!locked[u]) heap[(int)side[u]].push({gain[u], u});
            }
            const int64_t ov = over(w0);
            if (ov < best_over || (ov == best_over && cur > best)) {
                best = cur;
                best_over = ov;
                best_len = moved.size();
                stall = 0;
            } else {
                ++stall;
            }
        }
        for (size_t i = moved.size(); i > best_len; --i) side[moved[i - 1]] ^= 1;   // undo past the best
        if (best_len == 0) break;
    }
}

// Each side of a bisection keeps only its largest connected piece; the other
// pieces cross to the other side (which they touch: the graph is connected),
// so that every side, and in the end every part, is connected.
bool connect_sides(const G &g, std::vector<char> &side) {
    std::vector<int> comp(g.n, -1);
    std::vector<int64_t> cw;
    std::vector<char> cside;
    for (int v = 0; v < g.n; ++v) {
        if (comp[v] >= 0) continue;
        const int id = (int)cw.size();
        cw.push_back(0);
        cside.push_back(side[v]);
        std::queue<int> q;
        q.push(v);
        comp[v] = id;
        while (!q.empty()) {
            const int x = q.front();
            q.pop();
            cw[id] += g.vw[x] + 1;
            for (int64_t e = g.xadj[x]; e < g.xadj[x + 1]; ++e) {
                const int u = g.adj[e];
                if (comp[u] < 0 && side[u] == side[x]) { comp[u] = id; q.push(u); }
            }
        }
    }
    int keep[2] = {-1, -1};
    for (int c = 0; c < (int)cw.size(); ++c)
        if (keep[(int)cside[c]] < 0 || cw[c] > cw[keep[(int)cside[c]]]) keep[(int)cside[c]] = c;
    bool moved = false;
    for (int v = 0; v < g.n; ++v)
        if (keep[(int)cside[comp[v]]] != comp[v]) { side[v] = (char)(1 - cside[comp[v]]); moved = true; }
    return moved;
}

// Refinement that keeps the sides connected: a repair that moved a piece is
// followed by another balancing refinement (refinement can cut a narrow neck
// of a side in two), a few times at most.
void refine_connected(const G &g, std::vector<char> &side, int64_t target0, double eps, int passes) {
    fm_refine(g, side, target0, eps, passes);
    for (int t = 0; t < 3 && connect_sides(g, side); ++t) fm_refine(g, side, target0, eps, 2);
}

// Greedy graph growing from a few peripheral seeds; the lowest cut wins.
std::vector<char> initial_bisection(const G &g, int64_t target0, double eps, Rng &rng) {
    std::vector<char> best_side;
    int64_t best_cut = INT64_MAX;
    const int trials = std::min(g.n, 4);
    for (int t = 0; t < trials; ++t) {
        const int seed = far_vertex(g, (int)(rng.next() % (uint64_t)g.n));
        std::vector<char> side(g.n, 1);
        std::vector<int64_t> conn(g.n, 0);     // edge weight into side 0
        using Item = std::pair<int64_t, int>;
        std::priority_queue<Item> heap;
        int64_t w0 = 0;
        heap.push({0, seed});
        std::vector<char> in(g.n, 0);
        while (w0 < target0) {
            int v = -1;
            while (!heap.empty()) {
                const Item it = heap.top();
                heap.pop();
                if (!in[it.second]) { v = it.second; break; }
            }
            if (v < 0) {                     // a disconnected remainder: any vertex not in side 0
                for (int u = 0; u < g.n && v < 0; ++u) if (!in[u]) v = u;
                if (v < 0) break;
            }
            in[v] = 1;
            side[v] = 0;
            w0 += g.vw[v];
            for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
                const int u = g.adj[e];
                if (in[u]) continue;
                conn[u] += g.ew[e];
                heap.push({conn[u], u});
            }
        }
        // growing can enclose a pocket of the other side: pockets cross over
        // here, on the coarse graph, and the finer levels' refinement
        // restores the balance
        connect_sides(g, side);
        refine_connected(g, side, target0, eps, 4);
        const int64_t c = cut_of(g, side);
        if (c < best_cut) { best_cut = c; best_side = side; }
    }
    return best_side;
}

std::vector<char> multilevel_bisection(const G &g, int64_t target0, double eps, Rng &rng) {
    if (g.n <= 96) return initial_bisection(g, target0, eps, rng);
    std::vector<int> cmap;
    G c = coarsen_once(g, rng, cmap);
    if (c.n > (int)(0.9 * g.n)) return initial_bisection(g, target0, eps, rng);
    std::vector<char> cs = multilevel_bisection(c, target0, eps, rng);
    std::vector<char> side(g.n);
    for (int v = 0; v < g.n; ++v) side[v] = cs[cmap[v]];
    refine_connected(g, side, target0, eps, 4);
    return side;
}

G induced(const G &g, const std::vector<int> &verts, std::vector<int> &local) {
    G s;
    s.n = (int)verts.size();
    for (int i = 0; i < s.n; ++i) local[verts[i]] = i;
    s.xadj.assign(s.n + 1, 0);
    s.vw.resize(s.n);
    for (int i = 0; i < s.n; ++i) {
        const int v = verts[i];
        s.vw[i] = g.vw[v];
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e) {
            const int u = g.adj[e];
            if (local[u] >= 0) { s.adj.push_back(local[u]); s.ew.push_back(g.ew[e]); }
        }
        s.xadj[i + 1] = (int64_t)s.adj.size();
    }
    for (int v : verts) local[v] = -1;
    return s;
}

void recurse(const G &g, const std::vector<int> &verts, int k, int first, double eps, Rng &rng,
             std::vector<int> &part, std::vector<int> &local) {
    if (k == 1) {
        for (int v : verts) part[v] = first;
        return;
    }
    G s = induced(g, verts, local);
    const int k0 = k / 2;
    const int64_t target0 = (int64_t)((double)s.total() * k0 / k + 0.5);
    // split the balance tolerance over the levels of the recursion
    int depth = 0;
    for (int t = k; t > 1; t = (t + 1) / 2) ++depth;
    const double e = eps / std::max(1, depth);
    std::vector<char> side = s.n > 1 ? multilevel_bisection(s, target0, e, rng) : std::vector<char>(s.n, 0);
    if (s.n > 1) connect_sides(s, side);
    std::vector<int> a, b;
    for (int i = 0; i < s.n; ++i) (side[i] ? b : a).push_back(verts[i]);
    recurse(g, a, k0, first, eps, rng, part, local);
    recurse(g, b, k - k0, first + k0, eps, rng, part, local);
}

// Every part connected: smaller pieces join the neighbouring part they share
// the most edge weight with (repeated until no part has a second piece).
void connect_parts(const G &g, int k, std::vector<int> &part) {
    for (int round = 0; round < 64; ++round) {
        std::vector<int> comp(g.n, -1);
        std::vector<int64_t> cw;
        std::vector<int> cpart;
        for (int v = 0; v < g.n; ++v) {
            if (comp[v] >= 0) continue;
            const int id = (int)cw.size();
            cw.push_back(0);
            cpart.push_back(part[v]);
            std::queue<int> q;
            q.push(v);
            comp[v] = id;
            while (!q.empty()) {
                const int x = q.front();
                q.pop();
                cw[id] += g.vw[x];
                for (int64_t e = g.xadj[x]; e < g.xadj[x + 1]; ++e) {
                    const int u = g.adj[e];
                    if (comp[u] < 0 && part[u] == part[x]) { comp[u] = id; q.push(u); }
                }
            }
        }
        std::vector<int> keep(k, -1);
        for (int c = 0; c < (int)cw.size(); ++c) {
            const int p = cpart[c];
            if (keep[p] < 0 || cw[c] > cw[keep[p]]) keep[p] = c;
        }
        std::vector<std::vector<int>> members(cw.size());
        for (int v = 0; v < g.n; ++v)
            if (keep[cpart[comp[v]]] != comp[v]) members[comp[v]].push_back(v);
        bool changed = false;
        std::vector<int64_t> share(k, 0);
        for (int c = 0; c < (int)cw.size(); ++c) {
            if (members[c].empty()) continue;
            std::fill(share.begin(), share.end(), 0);
            for (int v : members[c])
                for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e)
                    if (comp[g.adj[e]] != c) share[part[g.adj[e]]] += g.ew[e];
            const int to = (int)(std::max_element(share.begin(), share.end()) - share.begin());
            if (share[to] == 0) continue;    // an isolated piece of a disconnected graph
            for (int v : members[c]) part[v] = to;
            changed = true;
        }
        if (!changed) return;
    }
}

}  // namespace

int64_t partition_graph(int n, const int64_t *xadj, const int *adjncy, const int *vwgt, const int *adjwgt,
                        int nparts, double imbalance, uint64_t seed, int *part_out) {
    G g;
    g.n = n;
    g.xadj.assign(xadj, xadj + n + 1);
    g.adj.assign(adjncy, adjncy + xadj[n]);
    g.ew.resize(g.adj.size());
    for (size_t e = 0; e < g.adj.size(); ++e) g.ew[e] = adjwgt ? adjwgt[e] : 1;
    g.vw.resize(n);
    for (int v = 0; v < n; ++v) g.vw[v] = vwgt ? vwgt[v] : 1;
    std::vector<int> part(n, 0), local(n, -1), verts(n);
    std::iota(verts.begin(), verts.end(), 0);
    Rng rng{seed};
    recurse(g, verts, nparts, 0, imbalance, rng, part, local);
    connect_parts(g, nparts, part);
    std::copy(part.begin(), part.end(), part_out);
    int64_t cut = 0;
    for (int v = 0; v < n; ++v)
        for (int64_t e = g.xadj[v]; e < g.xadj[v + 1]; ++e)
            if (part[v] != part[g.adj[e]]) cut += g.ew[e];
    return cut / 2;
}

}  // namespace bddc
