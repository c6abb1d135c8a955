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

std::vector<int> partition_cells(const HostMesh &hm, int P) {
    const int C = hm.C;
    std::vector<std::vector<int>> adj(C);
    for (int e = 0; e < hm.E; e++) {
        adj[hm.c1[e]].push_back(hm.c2[e]);
        adj[hm.c2[e]].push_back(hm.c1[e]);
    }
    std::vector<int> owner(C, -1), mask(C, 0), da(C), db(C), all(C);
    std::iota(all.begin(), all.end(), 0);
    int next = 0, tagctr = 0;
    bisect(adj, all, P, owner, next, mask, tagctr, da, db);
    return owner;
}

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

std::vector<int> cell_locality_order(int C, const std::vector<int> &c1,
                                     const std::vector<int> &c2, int leaf) {
    std::vector<std::vector<int>> adj(C);
    for (size_t e = 0; e < c1.size(); e++) {
        adj[c1[e]].push_back(c2[e]);
        adj[c2[e]].push_back(c1[e]);
    }
    std::vector<int> owner(C, -1), mask(C, 0), da(C), db(C), all(C);
    std::iota(all.begin(), all.end(), 0);
    int next = 0, tagctr = 0;
    const int parts = std::max(1, (C + std::max(leaf, 1) - 1) / std::max(leaf, 1));
    // part ids are handed out depth first: the left half of every bisection
    // gets the lower ids
    bisect(adj, all, parts, owner, next, mask, tagctr, da, db);
    std::vector<int> order(C);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return owner[a] < owner[b]; });
    return order;
}

bool build_bcl_plan(const HostMesh &hm, int Pc, int max_e0, int max_c1, BclPlan &plan) {
    const int C = hm.C, E = hm.E, V = hm.V;
    if (Pc < 1) return false;
    for (int c = 0; c < C; c++) if (hm.neoc[c] > BCL_NCEP) return false;
    for (int e = 0; e < E; e++) if (hm.neoe[e] > BCL_NE2P) return false;
    plan = BclPlan();
    plan.Pc = Pc;
    plan.P = (C + Pc - 1) / Pc;
    const int P = plan.P;
    // compact patches: a recursive bisection of the cell graph into P parts;
    // an edge belongs to the patch of its lower-numbered cell
    plan.owner = partition_cells(hm, P);
    std::vector<std::vector<int>> own_e(P);
    for (int e = 0; e < E; e++) own_e[plan.owner[std::min(hm.c1[e], hm.c2[e])]].push_back(e);
    std::vector<int> le(E, -1), lc(C, -1), lv(V, -1);
    for (auto *o : {&plan.off_e0, &plan.off_e1, &plan.off_e2, &plan.off_c1, &plan.off_c2,
                    &plan.off_v})
        o->push_back(0);
    for (int p = 0; p < P; p++) {
        std::vector<int> Ed, Cd, Vd;   // local -> internal
        auto add_e = [&](int e) { if (e >= 0 && le[e] < 0) { le[e] = (int)Ed.size(); Ed.push_back(e); } };
        auto add_c = [&](int c) { if (c >= 0 && lc[c] < 0) { lc[c] = (int)Cd.size(); Cd.push_back(c); } };
        auto add_v = [&](int v) { if (v >= 0 && lv[v] < 0) { lv[v] = (int)Vd.size(); Vd.push_back(v); } };
        auto sorted_add = [](std::vector<int> x, auto &&fn) {
            std::sort(x.begin(), x.end());
            for (int y : x) fn(y);
        };
        for (int e : own_e[p]) add_e(e);
        const int nE0 = (int)Ed.size();
        {   // C1: the cells of the owned edges
            std::vector<int> x;
            for (int e : own_e[p]) { x.push_back(hm.c1[e]); x.push_back(hm.c2[e]); }
            sorted_add(x, add_c);
        }
        const int nC1 = (int)Cd.size();
        {   // E1: the edges of C1's cells
            std::vector<int> x;
            for (int k = 0; k < nC1; k++)
                for (int j = 0; j < hm.neoc[Cd[k]]; j++) x.push_back(hm.eoc[(size_t)Cd[k] * hm.maxE + j]);
            sorted_add(x, add_e);
        }
        const int nE1 = (int)Ed.size();
        {   // V: the vertices of E1's edges
            std::vector<int> x;
            for (int k = 0; k < nE1; k++) { x.push_back(hm.v1[Ed[k]]); x.push_back(hm.v2[Ed[k]]); }
            sorted_add(x, add_v);
        }
        const int nV = (int)Vd.size();
        {   // E2: plus the edges of V's vertices; C2: plus the cells of E1's
            // edges and of V's vertices
            std::vector<int> x, y;
            for (int k = 0; k < nV; k++)
                for (int j = 0; j < 3; j++) {
                    x.push_back(hm.eov[3 * (size_t)Vd[k] + j]);
                    y.push_back(hm.cov[3 * (size_t)Vd[k] + j]);
                }
            for (int k = 0; k < nE1; k++) { y.push_back(hm.c1[Ed[k]]); y.push_back(hm.c2[Ed[k]]); }
            x.erase(std::remove(x.begin(), x.end(), -1), x.end());
            y.erase(std::remove(y.begin(), y.end(), -1), y.end());
            sorted_add(x, add_e);
            sorted_add(y, add_c);
        }
        const int nE2 = (int)Ed.size(), nC2 = (int)Cd.size();
        auto reset = [&]() {
            for (int e : Ed) le[e] = -1;
            for (int c : Cd) lc[c] = -1;
            for (int v : Vd) lv[v] = -1;
        };
        if (nE0 > max_e0 || nC1 > max_c1 || nE2 + 1 > 65535 || nC2 + 1 > 65535 || nV > 65535) {
            reset();
            return false;
        }
        // owned edges: edgesOnEdge must lie in E1
        bool ok = true;
        for (int k = 0; k < nE0 && ok; k++) {
            const int e = Ed[k];
            if (hm.neoe[e] > BCL_NE2P) ok = false;
            for (int j = 0; j < hm.neoe[e] && ok; j++) {
                const int l = le[hm.eoe[(size_t)e * hm.maxE2 + j]];
                if (l < 0 || l >= nE1) ok = false;
            }
        }
        if (!ok) { reset(); return false; }
        plan.cnt.insert(plan.cnt.end(), {nE0, nE1, nE2, nC1, nC2, nV, 0, 0});
        plan.maxE0 = std::max(plan.maxE0, nE0); plan.maxE1 = std::max(plan.maxE1, nE1);
        plan.maxE2 = std::max(plan.maxE2, nE2); plan.maxC1 = std::max(plan.maxC1, nC1);
        plan.maxC2 = std::max(plan.maxC2, nC2); plan.maxV = std::max(plan.maxV, nV);
        plan.egid.insert(plan.egid.end(), Ed.begin(), Ed.end());
        plan.cgid.insert(plan.cgid.end(), Cd.begin(), Cd.end());
        // owned edges, term-major
        const size_t b10 = plan.e0_eoe.size();
        plan.e0_eoe.resize(b10 + (size_t)BCL_NE2P * nE0, (uint16_t)nE1);
        plan.e0_wl.resize(b10 + (size_t)BCL_NE2P * nE0, 0.0);
        plan.e0_cfc.resize(b10 + (size_t)BCL_NE2P * nE0, 0.0);
        for (int k = 0; k < nE0; k++) {
            const int e = Ed[k];
            for (int j = 0; j < hm.neoe[e]; j++) {
                const size_t x = b10 + (size_t)j * nE0 + k;
                plan.e0_eoe[x] = (uint16_t)le[hm.eoe[(size_t)e * hm.maxE2 + j]];
                plan.e0_wl[x] = hm.wl[(size_t)e * hm.maxE2 + j];
                plan.e0_cfc[x] = hm.cfc[(size_t)e * hm.maxE2 + j];
            }
            plan.e0_c12.push_back(lc[hm.c1[e]] | (lc[hm.c2[e]] << 16));
            plan.e0_v12.push_back(lv[hm.v1[e]] | (lv[hm.v2[e]] << 16));
            plan.e0_n2.push_back(hm.neoe[e]);
            plan.e0_invdc.push_back(hm.invdc[e]);
            plan.e0_invdv.push_back(hm.invdv[e]);
        }
        for (int k = 0; k < nE1; k++) {
            const int e = Ed[k];
            plan.e1_c12.push_back(lc[hm.c1[e]] | (lc[hm.c2[e]] << 16));
            plan.e1_v12.push_back(lv[hm.v1[e]] | (lv[hm.v2[e]] << 16));
        }
        // C1 cells: edges (dummy: the zero velocity slot nE2) and the cell
        // across each (dummy: the cell itself), term-major
        const size_t b6 = plan.c1_e.size();
        plan.c1_e.resize(b6 + (size_t)BCL_NCEP * nC1, (uint16_t)nE2);
        plan.c1_o.resize(b6 + (size_t)BCL_NCEP * nC1, 0);
        plan.c1_divc.resize(b6 + (size_t)BCL_NCEP * nC1, 0.0);
        plan.c1_kec.resize(b6 + (size_t)BCL_NCEP * nC1, 0.0);
        for (int k = 0; k < nC1; k++) {
            const int c = Cd[k];
            for (int j = 0; j < BCL_NCEP; j++) plan.c1_o[b6 + (size_t)j * nC1 + k] = (uint16_t)k;
            for (int j = 0; j < hm.neoc[c]; j++) {
                const int e = hm.eoc[(size_t)c * hm.maxE + j];
                const int o = hm.c1[e] == c ? hm.c2[e] : hm.c1[e];
                const size_t x = b6 + (size_t)j * nC1 + k;
                plan.c1_e[x] = (uint16_t)le[e];
                plan.c1_o[x] = (uint16_t)lc[o];
                plan.c1_divc[x] = hm.divc[(size_t)c * hm.maxE + j];
                plan.c1_kec[x] = hm.kec[(size_t)c * hm.maxE + j];
            }
        }
        // vertices (absent edge: the zero velocity slot; absent cell: the zero
        // thickness slot nC2, weight 0)
        const size_t b3 = plan.v_e.size();
        plan.v_e.resize(b3 + (size_t)3 * nV, (uint16_t)nE2);
        plan.v_c.resize(b3 + (size_t)3 * nV, (uint16_t)nC2);
        plan.v_curl.resize(b3 + (size_t)3 * nV, 0.0);
        plan.v_kw.resize(b3 + (size_t)3 * nV, 0.0);
        for (int k = 0; k < nV; k++) {
            const int v = Vd[k];
            for (int j = 0; j < 3; j++) {
                const size_t x = b3 + (size_t)j * nV + k;
                const int e = hm.eov[3 * (size_t)v + j], c = hm.cov[3 * (size_t)v + j];
                if (e >= 0) {
                    plan.v_e[x] = (uint16_t)le[e];
                    plan.v_curl[x] = hm.curlc[3 * (size_t)v + j];
                }
                if (c >= 0) {
                    plan.v_c[x] = (uint16_t)lc[c];
                    plan.v_kw[x] = hm.kw[3 * (size_t)v + j];
                }
            }
            plan.v_f.push_back(hm.fV[v]);
        }
        plan.off_e0.push_back(plan.off_e0.back() + nE0);
        plan.off_e1.push_back(plan.off_e1.back() + nE1);
        plan.off_e2.push_back(plan.off_e2.back() + nE2);
        plan.off_c1.push_back(plan.off_c1.back() + nC1);
        plan.off_c2.push_back(plan.off_c2.back() + nC2);
        plan.off_v.push_back(plan.off_v.back() + nV);
        reset();
    }
    return true;
}

bool build_thick_plan(const HostMesh &hm, int Pc, ThickPlan &plan) {
    const int C = hm.C, E = hm.E;
    if (Pc < 1) return false;
    for (int c = 0; c < C; c++) if (hm.neoc[c] > BCL_NCEP) return false;
    plan = ThickPlan();
    plan.Pc = Pc;
    // compact patches of at most Pc cells: a recursive bisection into parts
    // of about 31/32 Pc cells (the bisection balances the parts to within a few
    // cells)
    plan.P = (int)(((long long)C * 32 + 31LL * Pc - 1) / (31LL * Pc));
    plan.owner = partition_cells(hm, plan.P);
    std::vector<std::vector<int>> own_c(plan.P);
    for (int c = 0; c < C; c++) own_c[plan.owner[c]].push_back(c);
    for (const auto &o : own_c) if ((int)o.size() > Pc) return false;
    std::vector<int> le(E, -1), lc(C, -1);
    plan.off_eo.push_back(0);
    plan.off_c1.push_back(0);
    for (int p = 0; p < plan.P; p++) {
        const std::vector<int> &own = own_c[p];
        const int nO = (int)own.size();
        std::vector<int> Ed, Cd;
        for (int l = 0; l < nO; l++) { lc[own[l]] = l; Cd.push_back(own[l]); }
        std::vector<int> x;
        for (int l = 0; l < nO; l++)
            for (int j = 0; j < hm.neoc[own[l]]; j++) x.push_back(hm.eoc[(size_t)own[l] * hm.maxE + j]);
        std::sort(x.begin(), x.end());
        x.erase(std::unique(x.begin(), x.end()), x.end());
        for (int e : x) { le[e] = (int)Ed.size(); Ed.push_back(e); }
        std::vector<int> y;
        for (int e : Ed) { y.push_back(hm.c1[e]); y.push_back(hm.c2[e]); }
        std::sort(y.begin(), y.end());
        y.erase(std::unique(y.begin(), y.end()), y.end());
        for (int c : y) if (lc[c] < 0) { lc[c] = (int)Cd.size(); Cd.push_back(c); }
        const int nEO = (int)Ed.size(), nC1 = (int)Cd.size();
        auto reset = [&]() {
            for (int e : Ed) le[e] = -1;
            for (int c : Cd) lc[c] = -1;
        };
        if (nEO + 1 > 65535 || nC1 > 65535) { reset(); return false; }
        plan.cnt.insert(plan.cnt.end(), {nO, nEO, nC1, 0});
        plan.maxEO = std::max(plan.maxEO, nEO);
        plan.maxC1 = std::max(plan.maxC1, nC1);
        plan.eogid.insert(plan.eogid.end(), Ed.begin(), Ed.end());
        plan.c1gid.insert(plan.c1gid.end(), Cd.begin(), Cd.end());
        for (int e : Ed) plan.eo_c12.push_back(lc[hm.c1[e]] | (lc[hm.c2[e]] << 16));
        const size_t b = plan.o_e.size();
        plan.o_e.resize(b + (size_t)BCL_NCEP * Pc, (uint16_t)nEO);
        plan.o_o.resize(b + (size_t)BCL_NCEP * Pc, 0);
        for (int l = 0; l < Pc; l++)
            for (int j = 0; j < BCL_NCEP; j++) plan.o_o[b + (size_t)j * Pc + l] = (uint16_t)(l < nO ? l : 0);
        for (int l = 0; l < nO; l++) {
            const int c = own[l];
            for (int j = 0; j < hm.neoc[c]; j++) {
                const int e = hm.eoc[(size_t)c * hm.maxE + j];
                const int o = hm.c1[e] == c ? hm.c2[e] : hm.c1[e];
                plan.o_e[b + (size_t)j * Pc + l] = (uint16_t)le[e];
                plan.o_o[b + (size_t)j * Pc + l] = (uint16_t)lc[o];
            }
        }
        plan.off_eo.push_back(plan.off_eo.back() + nEO);
        plan.off_c1.push_back(plan.off_c1.back() + nC1);
        reset();
    }
    return true;
}

size_t tile_smem_bytes(const TilePlan &plan, int maxE, int maxE2, size_t sR, bool eoe_smem) {
    (void)maxE;
    (void)maxE2;
    size_t best = 0;
    for (const TilePatch &t : plan.patches) {
        const size_t ne = t.ne + 1, nc = t.nc + 1;
        size_t b = 0;
        b += sR * (4 * ne);                 // u0, ua, uh, flux (increments)
        b += sR * (3 * nc);                 // z0, za, zh (increments)
        b += sR * (2 * ne + nc);            // starting forcing and ubar, starting depth
        b += 4 * ne;                        // packed local byte offsets of (c1, c2)
        if (eoe_smem) b += 2 * TILE_NE2P * ne;   // edgesOnEdge byte offsets, padded
        b += 2 * TILE_NCEP * nc;            // edgesOnCell byte offsets, padded
        b += 64 * 16;                       // alignment slack
        best = std::max(best, b);
    }
    return best;
}

}  // namespace sse
