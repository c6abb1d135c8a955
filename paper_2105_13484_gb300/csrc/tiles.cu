// tiles.cu -- host-side plan for the tiled barotropic sub-cycle.
//
// The cells are split into P compact patches (recursive bisection on BFS
// distances of the cell adjacency graph).  Each patch is extended by a halo
// of K cell rings; after one forward-Euler sub-stage of the 2-D system only
// values one ring further in are still exact, so K sub-stages can run on the
// patch alone before the owned values must be exchanged.  Every edge is
// owned by the patch of its first cell.  Local indices are 16-bit; each
// patch has one extra "dummy" edge and cell slot (value 0) that stands in
// for neighbours outside the halo (those results are never used).
#include <algorithm>
#include <climits>
#include <cstdint>
#include <deque>
#include <numeric>
#include <vector>

#include "tiles.h"

namespace sse {

namespace {

// BFS distances from `src` restricted to cells with mask[c] == tag
void bfs(const std::vector<std::vector<int>> &adj, const std::vector<int> &mask, int tag, int src,
         std::vector<int> &dist, const std::vector<int> &cells) {
    for (int c : cells) dist[c] = INT_MAX;
    std::deque<int> q;
    dist[src] = 0;
    q.push_back(src);
    while (!q.empty()) {
        int c = q.front();
        q.pop_front();
        for (int o : adj[c])
            if (mask[o] == tag && dist[o] == INT_MAX) {
                dist[o] = dist[c] + 1;
                q.push_back(o);
            }
    }
}

void bisect(const std::vector<std::vector<int>> &adj, std::vector<int> cells, int parts,
            std::vector<int> &owner, int &next, std::vector<int> &mask, int &tagctr,
            std::vector<int> &da, std::vector<int> &db) {
    if (parts <= 1 || cells.size() <= 1) {
        const int id = next++;
        for (int c : cells) owner[c] = id;
        // empty parts still get ids so that exactly `parts` ids are used
        for (int k = 1; k < parts; k++) next++;
        return;
    }
    const int tag = ++tagctr;
    for (int c : cells) mask[c] = tag;
    // pseudo-peripheral pair: farthest from cells[0], then farthest from that
    bfs(adj, mask, tag, cells[0], da, cells);
    int a = cells[0];
    for (int c : cells)
        if (da[c] != INT_MAX && da[c] > da[a]) a = c;
    bfs(adj, mask, tag, a, da, cells);
    int b = a;
    for (int c : cells)
        if (da[c] != INT_MAX && da[c] > da[b]) b = c;
    bfs(adj, mask, tag, b, db, cells);
    const long long big = 1LL << 40;
    std::vector<std::pair<long long, int>> key;
    key.reserve(cells.size());
    for (int c : cells) {
        long long ka = da[c] == INT_MAX ? big : da[c];
        long long kb = db[c] == INT_MAX ? big : db[c];
        key.push_back({ka - kb, c});
    }
    std::sort(key.begin(), key.end());
    const int p1 = parts / 2;
    const size_t n1 = (size_t)((double)cells.size() * p1 / parts + 0.5);
    std::vector<int> left, right;
    for (size_t k = 0; k < key.size(); k++) (k < n1 ? left : right).push_back(key[k].second);
    bisect(adj, left, p1, owner, next, mask, tagctr, da, db);
    bisect(adj, right, parts - p1, owner, next, mask, tagctr, da, db);
}

}  // namespace

bool tile_stencil_ok(const HostMesh &hm) {
    for (int e = 0; e < hm.E; e++)
        for (int j = 0; j < hm.neoe[e]; j++) {
            const int ep = hm.eoe[(size_t)e * hm.maxE2 + j];
            const int a = hm.c1[ep], b = hm.c2[ep];
            if (a != hm.c1[e] && a != hm.c2[e] && b != hm.c1[e] && b != hm.c2[e]) return false;
        }
    return true;
}

bool build_tile_plan(const HostMesh &hm, int P, int K, TilePlan &plan) {
    const int C = hm.C, E = hm.E;
    // cell adjacency through edges
    std::vector<std::vector<int>> adj(C);
    for (int e = 0; e < E; e++) {
        adj[hm.c1[e]].push_back(hm.c2[e]);
        adj[hm.c2[e]].push_back(hm.c1[e]);
    }
    std::vector<int> owner(C, -1), mask(C, 0), da(C), db(C);
    std::vector<int> all(C);
    std::iota(all.begin(), all.end(), 0);
    int next = 0, tagctr = 0;
    bisect(adj, all, P, owner, next, mask, tagctr, da, db);

    plan = TilePlan();
    plan.P = P;
    plan.K = K;
    std::vector<std::vector<int>> own(P);
    for (int c = 0; c < C; c++) own[owner[c]].push_back(c);
    std::vector<int> dist(C, INT_MAX), lc(C, -1), le(E, -1);
    plan.cell_off.push_back(0);
    plan.edge_off.push_back(0);
    for (int p = 0; p < P; p++) {
        // cells within K rings of the owned set, ordered by distance
        std::vector<int> X = own[p];
        for (int c : X) dist[c] = 0;
        size_t head = 0;
        while (head < X.size()) {
            int c = X[head++];
            if (dist[c] >= K) continue;
            for (int o : adj[c])
                if (dist[o] == INT_MAX) {
                    dist[o] = dist[c] + 1;
                    X.push_back(o);
                }
        }
        std::sort(X.begin() + own[p].size(), X.end(), [&](int a, int b) {
            return dist[a] != dist[b] ? dist[a] < dist[b] : a < b;
        });
        const int nc = (int)X.size();
        for (int k = 0; k < nc; k++) lc[X[k]] = k;
        // edges of those cells: owned ones (first cell owned here) first
        std::vector<int> Eo, Eh;
        for (int c : X)
            for (int j = 0; j < hm.neoc[c]; j++) {
                int e = hm.eoc[(size_t)c * hm.maxE + j];
                if (le[e] != -1) continue;
                le[e] = 0;
                (owner[hm.c1[e]] == p ? Eo : Eh).push_back(e);
            }
        // ring of an edge: the larger ring of its cells (outside the patch: K+1)
        auto ering = [&](int e) {
            const int a = dist[hm.c1[e]], b = dist[hm.c2[e]];
            return std::max(a == INT_MAX ? K + 1 : a, b == INT_MAX ? K + 1 : b);
        };
        // owned edges of ring 0 (both cells owned) first: their next forward-Euler
        // stage reads only values that are exact before the halo is refreshed
        std::sort(Eo.begin(), Eo.end(), [&](int a, int b) {
            const int ra = ering(a), rb = ering(b);
            return ra != rb ? ra < rb : a < b;
        });
        std::sort(Eh.begin(), Eh.end(), [&](int a, int b) {
            const int ra = ering(a), rb = ering(b);
            return ra != rb ? ra < rb : a < b;
        });
        std::vector<int> Ed = Eo;
        Ed.insert(Ed.end(), Eh.begin(), Eh.end());
        const int ne = (int)Ed.size();
        for (int k = 0; k < ne; k++) le[Ed[k]] = k;
        if (nc + 1 > 32767 || ne + 1 > 32767) {
            for (int c : X) { dist[c] = INT_MAX; lc[c] = -1; }
            for (int e : Ed) le[e] = -1;
            return false;
        }
        const int dummyC = nc, dummyE = ne;
        // per-patch arrays
        TilePatch tp;
        tp.nc = nc; tp.ne = ne;
        tp.n_own_c = (int)own[p].size();
        tp.n_own_e = (int)Eo.size();
        tp.n_int_e = 0;
        for (int e : Eo) tp.n_int_e += ering(e) == 0;
        tp.cell_gid = X;
        tp.edge_gid = Ed;
        tp.c12.resize(ne);
        tp.n2.resize(ne);
        tp.eoe.assign((size_t)hm.maxE2 * ne, (int16_t)dummyE);   // [ne][maxE2]
        tp.cfc.assign((size_t)hm.maxE2 * ne, 0.0);
        tp.invdc.resize(ne);
        for (int k = 0; k < ne; k++) {
            const int e = Ed[k];
            const int a = lc[hm.c1[e]] >= 0 ? lc[hm.c1[e]] : dummyC;
            const int b = lc[hm.c2[e]] >= 0 ? lc[hm.c2[e]] : dummyC;
            tp.c12[k] = (int32_t)((uint32_t)a | ((uint32_t)b << 16));
            tp.n2[k] = (int16_t)hm.neoe[e];
            tp.invdc[k] = hm.invdc[e];
            for (int j = 0; j < hm.neoe[e]; j++) {
                const int ep = hm.eoe[(size_t)e * hm.maxE2 + j];
                tp.eoe[(size_t)k * hm.maxE2 + j] = (int16_t)(le[ep] >= 0 ? le[ep] : dummyE);
                tp.cfc[(size_t)k * hm.maxE2 + j] = le[ep] >= 0 ? hm.cfc[(size_t)e * hm.maxE2 + j] : 0.0;
            }
        }
        tp.nce.resize(nc);
        tp.ce.assign((size_t)hm.maxE * nc, (int16_t)dummyE);      // [nc][maxE]
        tp.divc.assign((size_t)hm.maxE * nc, 0.0);
        tp.H.resize(nc + 1);
        for (int k = 0; k < nc; k++) {
            const int c = X[k];
            tp.H[k] = hm.H[c];
            tp.nce[k] = (int16_t)hm.neoc[c];
            for (int j = 0; j < hm.neoc[c]; j++) {
                const int e = hm.eoc[(size_t)c * hm.maxE + j];
                tp.ce[(size_t)k * hm.maxE + j] = (int16_t)le[e];
                tp.divc[(size_t)k * hm.maxE + j] = hm.divc[(size_t)c * hm.maxE + j];
            }
        }
        tp.H[nc] = 1.0;  // dummy cell: finite depth
        // prefix counts by ring (owned edges have ring 0 or 1)
        for (int r = 0; r < 3; r++) {
            int n = tp.n_own_e;
            for (int e : Eh) n += ering(e) <= r + 1;
            tp.ne_ring[r] = n;
            int c = 0;
            for (int x : X) c += dist[x] <= r;
            tp.nc_ring[r] = c;
        }
        plan.patches.push_back(std::move(tp));
        plan.cell_off.push_back(plan.cell_off.back() + nc);
        plan.edge_off.push_back(plan.edge_off.back() + ne);
        for (int c : X) { dist[c] = INT_MAX; lc[c] = -1; }
        for (int e : Ed) le[e] = -1;
    }
    return true;
}

size_t tile_smem_bytes(const TilePlan &plan, int maxE, int maxE2, size_t sR) {
    (void)maxE;
    (void)maxE2;
    size_t best = 0;
    for (const TilePatch &t : plan.patches) {
        const size_t ne = t.ne + 1, nc = t.nc + 1;
        size_t b = 0;
        b += sR * (4 * ne);                 // u0, ua, uh, flux
        b += sR * ne;                       // 1/d_e
        b += sR * (3 * nc);                 // z0, za, zh
        b += sR * (ne + nc);                // G, H
        b += 4 * ne;                        // packed local byte offsets of (c1, c2)
        b += 2 * TILE_NE2P * ne;            // edgesOnEdge byte offsets, padded
        b += 2 * TILE_NCEP * nc;            // edgesOnCell byte offsets, padded
        b += 64 * 16;                       // alignment slack
        best = std::max(best, b);
    }
    return best;
}

}  // namespace sse
