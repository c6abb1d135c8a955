// Checks the invariants of a tile plan of the tiled barotropic sub-cycle
// (csrc/tiles.cu) on one mesh: ownership, local order, and the closure that
// makes the communication-avoiding scheme exact -- every entry a sub-stage
// computes reads only entries that are exact after the sub-stage before.
// Usage: tile_plan_check <mesh dir> <patches>; prints "ok" or the first
// violation (exit status 1).
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../paper_2105_13484_gb300/csrc/tiles.h"

using namespace sse;

template <class T> static std::vector<T> rd(const std::string &f, size_t n) {
    std::vector<T> v(n);
    FILE *fp = fopen(f.c_str(), "rb");
    if (!fp || fread(v.data(), sizeof(T), n, fp) != n) {
        fprintf(stderr, "cannot read %s\n", f.c_str());
        exit(2);
    }
    fclose(fp);
    return v;
}

static int fail(const char *what, int p, int l) {
    printf("violation: %s (patch %d, local %d)\n", what, p, l);
    return 1;
}

int main(int argc, char **argv) {
    if (argc != 3) return 2;
    const std::string d = argv[1];
    const int P = atoi(argv[2]);
    int C, E, mE, mE2;
    FILE *fp = fopen((d + "/hdr.txt").c_str(), "r");
    if (!fp || fscanf(fp, "%d %d %d %d", &C, &E, &mE, &mE2) != 4) return 2;
    fclose(fp);
    HostMesh hm;
    hm.C = C; hm.E = E; hm.maxE = mE; hm.maxE2 = mE2;
    auto coe = rd<int>(d + "/coe.bin", 2 * (size_t)E);
    hm.c1.resize(E); hm.c2.resize(E);
    for (int e = 0; e < E; e++) { hm.c1[e] = coe[2 * e]; hm.c2[e] = coe[2 * e + 1]; }
    hm.neoc = rd<int>(d + "/neoc.bin", C);
    hm.eoc = rd<int>(d + "/eoc.bin", (size_t)C * mE);
    hm.neoe = rd<int>(d + "/neoe.bin", E);
    hm.eoe = rd<int>(d + "/eoe.bin", (size_t)E * mE2);
    hm.cfc.assign((size_t)E * mE2, 1.0); hm.divc.assign((size_t)C * mE, 1.0);
    hm.invdc.assign(E, 1.0); hm.H.assign(C, 1.0);
    if (!tile_stencil_ok(hm)) { printf("violation: not a TRiSK stencil\n"); return 1; }
    TilePlan plan;
    if (!build_tile_plan(hm, P, 3, plan)) { printf("violation: no plan\n"); return 1; }
    if ((int)plan.patches.size() != P) { printf("violation: patch count\n"); return 1; }

    std::vector<int> cell_owner(C, -1), edge_owner(E, -1);
    for (int p = 0; p < P; p++) {
        const TilePatch &t = plan.patches[p];
        for (int l = 0; l < t.n_own_c; l++) {
            if (cell_owner[t.cell_gid[l]] != -1) return fail("cell owned twice", p, l);
            cell_owner[t.cell_gid[l]] = p;
        }
        for (int l = 0; l < t.n_own_e; l++) {
            if (edge_owner[t.edge_gid[l]] != -1) return fail("edge owned twice", p, l);
            edge_owner[t.edge_gid[l]] = p;
        }
    }
    for (int c = 0; c < C; c++) if (cell_owner[c] < 0) return fail("cell not owned", -1, c);
    for (int e = 0; e < E; e++) {
        if (edge_owner[e] < 0) return fail("edge not owned", -1, e);
        if (edge_owner[e] != cell_owner[hm.c1[e]]) return fail("edge not owned by its first cell", -1, e);
    }

    for (int p = 0; p < P; p++) {
        const TilePatch &t = plan.patches[p];
        const int ne = t.ne, nc = t.nc;
        // exact after sub-stage s (s = -1: after the halo refresh, everything local)
        const int neA = t.ne_ring[2], neB = t.ne_ring[1], neC = t.ne_ring[0];
        const int ncA = t.nc_ring[2], ncB = t.nc_ring[1], ncC = t.nc_ring[0];
        const int ne_lim[3] = {neA, neB, neC}, nc_lim[3] = {ncA, ncB, ncC};
        const int ne_in[3] = {ne, neA, neB}, nc_in[3] = {nc, ncA, ncB};
        if (!(neC <= neB && neB <= neA && neA <= ne && ncC <= ncB && ncB <= ncA && ncA <= nc))
            return fail("ring counts not nested", p, -1);
        if (ncC != t.n_own_c) return fail("cells exact after the last sub-stage != owned", p, -1);
        if (t.n_own_e > neC) return fail("owned edges beyond the last sub-stage", p, -1);
        for (int l = t.n_own_c; l < nc; l++)
            if (cell_owner[t.cell_gid[l]] == p) return fail("halo cell owned here", p, l);
        for (int l = t.n_own_e; l < ne; l++)
            if (edge_owner[t.edge_gid[l]] == p) return fail("halo edge owned here", p, l);
        for (int l = 0; l < t.n_int_e; l++) {
            const int e = t.edge_gid[l];
            if (cell_owner[hm.c1[e]] != p || cell_owner[hm.c2[e]] != p)
                return fail("interior edge with a cell not owned", p, l);
        }
        for (int l = t.n_int_e; l < t.n_own_e; l++) {
            const int e = t.edge_gid[l];
            if (cell_owner[hm.c1[e]] == p && cell_owner[hm.c2[e]] == p)
                return fail("owned edge with both cells owned after the interior ones", p, l);
        }
        auto cells_of = [&](int l, int &a, int &b) {
            const unsigned x = (unsigned)t.c12[l];
            a = (int)(x & 0xffffu); b = (int)(x >> 16);
        };
        for (int s = 0; s < 3; s++) {
            for (int l = 0; l < ne_lim[s]; l++) {
                for (int j = 0; j < t.n2[l]; j++)
                    if (t.eoe[(size_t)l * mE2 + j] >= ne_in[s])
                        return fail("edge sub-stage reads an inexact edge", p, l);
                int a, b;
                cells_of(l, a, b);
                if (a >= nc_in[s] || b >= nc_in[s])
                    return fail("edge sub-stage reads an inexact cell", p, l);
            }
            for (int l = 0; l < nc_lim[s]; l++)
                for (int j = 0; j < t.nce[l]; j++)
                    if (t.ce[(size_t)l * mE + j] >= ne_lim[s])
                        return fail("cell sub-stage reads an edge not computed in it", p, l);
        }
        // the interior edges' first sub-stage runs before the halo refresh:
        // it may read only what the last sub-stage left exact
        for (int l = 0; l < t.n_int_e; l++) {
            for (int j = 0; j < t.n2[l]; j++)
                if (t.eoe[(size_t)l * mE2 + j] >= neC)
                    return fail("interior edge reads an edge not exact before the refresh", p, l);
            int a, b;
            cells_of(l, a, b);
            if (a >= ncC || b >= ncC)
                return fail("interior edge reads a cell not exact before the refresh", p, l);
        }
    }
    printf("ok\n");
    return 0;
}
