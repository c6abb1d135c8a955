// Checks the patch plan of the fused baroclinic kernel (csrc/tiles.cu,
// build_bcl_plan) on one mesh, numbered the way the library numbers it
// (cells in the locality order of cell_locality_order, edges by their lower
// cell).  Every owned edge belongs to exactly one patch; every local index the
// kernel dereferences lies inside its patch's list (or is that list's zero
// slot); every neighbour an owned edge, a C1 cell, a vertex or an E1 edge
// reads is the one the global mesh names; the plan's maxima bound every
// patch; and the same for the fused thickness kernel's plan (owned cells
// contiguous, each cell's edges and neighbours the mesh's, absent ones the zero
// slot).  Usage: bcl_plan_check <mesh dir> <cells per patch>; prints "ok" or
// the first violation (exit status 1).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <numeric>
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
    const int Pc = atoi(argv[2]);
    int C, E, V, mE, mE2;
    FILE *fp = fopen((d + "/hdr.txt").c_str(), "r");
    if (!fp || fscanf(fp, "%d %d %d %d %d", &C, &E, &mE, &mE2, &V) != 5) return 2;
    fclose(fp);
    const auto coe = rd<int>(d + "/coe.bin", 2 * (size_t)E);
    const auto voe = rd<int>(d + "/voe.bin", 2 * (size_t)E);
    const auto neoc = rd<int>(d + "/neoc.bin", C);
    const auto eoc = rd<int>(d + "/eoc.bin", (size_t)C * mE);
    const auto neoe = rd<int>(d + "/neoe.bin", E);
    const auto eoe = rd<int>(d + "/eoe.bin", (size_t)E * mE2);
    const auto eov = rd<int>(d + "/eov.bin", 3 * (size_t)V);
    const auto cov = rd<int>(d + "/cov.bin", 3 * (size_t)V);

    // the library's numbering: cells by locality, edges by their lower cell
    std::vector<int> a(E), b(E);
    for (int e = 0; e < E; e++) { a[e] = coe[2 * e]; b[e] = coe[2 * e + 1]; }
    const std::vector<int> cold = cell_locality_order(C, a, b, 8);
    std::vector<int> cnew(C, -1);
    for (int i = 0; i < C; i++) cnew[cold[i]] = i;
    for (int c = 0; c < C; c++) if (cnew[c] < 0) return fail("locality order is not a permutation", -1, c);
    std::vector<int> eold(E), enew(E);
    std::iota(eold.begin(), eold.end(), 0);
    std::sort(eold.begin(), eold.end(), [&](int p, int q) {
        const int mp = std::min(cnew[a[p]], cnew[b[p]]), mq = std::min(cnew[a[q]], cnew[b[q]]);
        if (mp != mq) return mp < mq;
        const int Mp = std::max(cnew[a[p]], cnew[b[p]]), Mq = std::max(cnew[a[q]], cnew[b[q]]);
        return Mp != Mq ? Mp < Mq : p < q;
    });
    for (int e = 0; e < E; e++) enew[eold[e]] = e;

    HostMesh hm;
    hm.C = C; hm.E = E; hm.V = V; hm.maxE = mE; hm.maxE2 = mE2;
    hm.c1.resize(E); hm.c2.resize(E); hm.v1.resize(E); hm.v2.resize(E); hm.neoe.resize(E);
    hm.eoe.assign((size_t)E * mE2, 0);
    for (int e = 0; e < E; e++) {
        const int o = eold[e];
        hm.c1[e] = cnew[coe[2 * o]]; hm.c2[e] = cnew[coe[2 * o + 1]];
        hm.v1[e] = voe[2 * o]; hm.v2[e] = voe[2 * o + 1];
        hm.neoe[e] = neoe[o];
        for (int j = 0; j < neoe[o]; j++) hm.eoe[(size_t)e * mE2 + j] = enew[eoe[(size_t)o * mE2 + j]];
    }
    hm.neoc.resize(C); hm.eoc.assign((size_t)C * mE, 0);
    for (int i = 0; i < C; i++) {
        const int o = cold[i];
        hm.neoc[i] = neoc[o];
        for (int j = 0; j < neoc[o]; j++) hm.eoc[(size_t)i * mE + j] = enew[eoc[(size_t)o * mE + j]];
    }
    hm.eov.resize(3 * (size_t)V); hm.cov.resize(3 * (size_t)V);
    for (int x = 0; x < 3 * V; x++) {
        hm.eov[x] = eov[x] >= 0 ? enew[eov[x]] : -1;
        hm.cov[x] = cov[x] >= 0 ? cnew[cov[x]] : -1;
    }
    // coefficients carry an identity tag so that the test can see that each
    // one went with its entry
    hm.cfc.resize((size_t)E * mE2); hm.wl.resize((size_t)E * mE2);
    for (size_t x = 0; x < hm.wl.size(); x++) { hm.wl[x] = 1.0 + (double)x; hm.cfc[x] = -1.0 - (double)x; }
    hm.divc.resize((size_t)C * mE); hm.kec.resize((size_t)C * mE);
    for (size_t x = 0; x < hm.divc.size(); x++) { hm.divc[x] = 1.0 + (double)x; hm.kec[x] = 2.0 + (double)x; }
    hm.curlc.resize(3 * (size_t)V); hm.kw.resize(3 * (size_t)V); hm.fV.resize(V);
    for (size_t x = 0; x < hm.curlc.size(); x++) { hm.curlc[x] = 1.0 + (double)x; hm.kw[x] = 3.0 + (double)x; }
    for (int v = 0; v < V; v++) hm.fV[v] = 5.0 + v;
    hm.invdc.resize(E); hm.invdv.resize(E);
    for (int e = 0; e < E; e++) { hm.invdc[e] = 1.0 + e; hm.invdv[e] = 2.0 + e; }
    hm.H.assign(C, 1.0);

    BclPlan pl;
    if (!build_bcl_plan(hm, Pc, 512, 512, pl)) { printf("violation: no plan\n"); return 1; }
    if (pl.P != (C + Pc - 1) / Pc) return fail("patch count", -1, -1);
    if ((int)pl.owner.size() != C) return fail("owner size", -1, -1);
    for (int c = 0; c < C; c++) if (pl.owner[c] < 0 || pl.owner[c] >= pl.P) return fail("cell owner", -1, c);
    std::vector<int> owner(E, -1);
    for (int p = 0; p < pl.P; p++) {
        const int *n = &pl.cnt[8 * p];
        const int nE0 = n[0], nE1 = n[1], nE2 = n[2], nC1 = n[3], nC2 = n[4], nV = n[5];
        if (!(nE0 <= nE1 && nE1 <= nE2 && nC1 <= nC2)) return fail("lists not nested", p, -1);
        if (nE0 > pl.maxE0 || nE1 > pl.maxE1 || nE2 > pl.maxE2 || nC1 > pl.maxC1 ||
            nC2 > pl.maxC2 || nV > pl.maxV)
            return fail("a count above the plan's maximum", p, -1);
        if (nE0 > 512 || nC1 > 512) return fail("a count above the kernel's slots", p, -1);
        if (pl.off_e0[p + 1] - pl.off_e0[p] != nE0 || pl.off_e1[p + 1] - pl.off_e1[p] != nE1 ||
            pl.off_e2[p + 1] - pl.off_e2[p] != nE2 || pl.off_c1[p + 1] - pl.off_c1[p] != nC1 ||
            pl.off_c2[p + 1] - pl.off_c2[p] != nC2 || pl.off_v[p + 1] - pl.off_v[p] != nV)
            return fail("offsets disagree with the counts", p, -1);
        const int *eg = &pl.egid[pl.off_e2[p]], *cg = &pl.cgid[pl.off_c2[p]];
        for (int l = 0; l < nE2; l++) if (eg[l] < 0 || eg[l] >= E) return fail("edge gid", p, l);
        for (int l = 0; l < nC2; l++) if (cg[l] < 0 || cg[l] >= C) return fail("cell gid", p, l);
        // owned edges: those whose lower cell is in this patch's part
        for (int l = 0; l < nE0; l++) {
            const int e = eg[l];
            if (owner[e] != -1) return fail("edge owned twice", p, l);
            owner[e] = p;
            if (pl.owner[std::min(hm.c1[e], hm.c2[e])] != p)
                return fail("edge owner is not its lower cell's patch", p, l);
        }
        // the lookup of a global vertex in V (by its E1 edges)
        std::vector<int> vg(nV, -1);
        for (int l = 0; l < nE1; l++) {
            const unsigned cc = (unsigned)pl.e1_c12[pl.off_e1[p] + l];
            const unsigned vv = (unsigned)pl.e1_v12[pl.off_e1[p] + l];
            const int ca = cc & 0xffff, cb = cc >> 16, va = vv & 0xffff, vb = vv >> 16;
            if (ca >= nC2 || cb >= nC2) return fail("E1 cell outside C2", p, l);
            if (va >= nV || vb >= nV) return fail("E1 vertex outside V", p, l);
            const int e = eg[l];
            if (cg[ca] != hm.c1[e] || cg[cb] != hm.c2[e]) return fail("E1 cells wrong", p, l);
            for (int s = 0; s < 2; s++) {
                const int vl = s ? vb : va, v = s ? hm.v2[e] : hm.v1[e];
                if (vg[vl] != -1 && vg[vl] != v) return fail("V local index maps two vertices", p, l);
                vg[vl] = v;
            }
        }
        for (int l = 0; l < nV; l++) if (vg[l] < 0) return fail("vertex not reached from E1", p, l);
        for (int l = 0; l < nE0; l++) {
            const int e = eg[l];
            const unsigned cc = (unsigned)pl.e0_c12[pl.off_e0[p] + l];
            const unsigned vv = (unsigned)pl.e0_v12[pl.off_e0[p] + l];
            const int ca = cc & 0xffff, cb = cc >> 16;
            if (ca >= nC1 || cb >= nC1) return fail("owned edge cell outside C1", p, l);
            if (cg[ca] != hm.c1[e] || cg[cb] != hm.c2[e]) return fail("owned edge cells wrong", p, l);
            if ((int)(vv & 0xffff) >= nV || (int)(vv >> 16) >= nV) return fail("owned edge vertex outside V", p, l);
            if (vg[vv & 0xffff] != hm.v1[e] || vg[vv >> 16] != hm.v2[e]) return fail("owned edge vertices wrong", p, l);
            if (pl.e0_n2[pl.off_e0[p] + l] != hm.neoe[e]) return fail("edgesOnEdge count", p, l);
            if (pl.e0_invdc[pl.off_e0[p] + l] != hm.invdc[e] || pl.e0_invdv[pl.off_e0[p] + l] != hm.invdv[e])
                return fail("owned edge 1/d or 1/l", p, l);
            for (int j = 0; j < BCL_NE2P; j++) {
                const size_t x = (size_t)BCL_NE2P * pl.off_e0[p] + (size_t)j * nE0 + l;
                const int le = pl.e0_eoe[x];
                if (j < hm.neoe[e]) {
                    if (le >= nE1) return fail("edgesOnEdge outside E1", p, l);
                    if (eg[le] != hm.eoe[(size_t)e * mE2 + j]) return fail("edgesOnEdge wrong", p, l);
                    if (pl.e0_wl[x] != hm.wl[(size_t)e * mE2 + j] || pl.e0_cfc[x] != hm.cfc[(size_t)e * mE2 + j])
                        return fail("edgesOnEdge coefficient", p, l);
                } else if (le != nE1 || pl.e0_wl[x] != 0.0 || pl.e0_cfc[x] != 0.0) {
                    return fail("edgesOnEdge padding is not the zero slot", p, l);
                }
            }
        }
        for (int l = 0; l < nC1; l++) {
            const int c = cg[l];
            for (int j = 0; j < BCL_NCEP; j++) {
                const size_t x = (size_t)6 * pl.off_c1[p] + (size_t)j * nC1 + l;
                const int le = pl.c1_e[x], lo = pl.c1_o[x];
                if (j < hm.neoc[c]) {
                    const int e = hm.eoc[(size_t)c * mE + j];
                    if (le >= nE1) return fail("C1 cell edge outside E1", p, l);
                    if (eg[le] != e) return fail("C1 cell edge wrong", p, l);
                    if (lo >= nC2 || cg[lo] != (hm.c1[e] == c ? hm.c2[e] : hm.c1[e]))
                        return fail("C1 cell neighbour wrong", p, l);
                    if (pl.c1_divc[x] != hm.divc[(size_t)c * mE + j] || pl.c1_kec[x] != hm.kec[(size_t)c * mE + j])
                        return fail("C1 cell coefficient", p, l);
                } else if (le != nE2 || lo != l || pl.c1_divc[x] != 0.0 || pl.c1_kec[x] != 0.0) {
                    return fail("C1 cell padding is not the zero slot", p, l);
                }
            }
        }
        for (int l = 0; l < nV; l++) {
            const int v = vg[l];
            if (pl.v_f[pl.off_v[p] + l] != hm.fV[v]) return fail("vertex f", p, l);
            for (int j = 0; j < 3; j++) {
                const size_t x = (size_t)3 * pl.off_v[p] + (size_t)j * nV + l;
                const int le = pl.v_e[x], lc = pl.v_c[x];
                const int e = hm.eov[3 * (size_t)v + j], c = hm.cov[3 * (size_t)v + j];
                if (e >= 0) {
                    if (le >= nE2 || eg[le] != e) return fail("vertex edge", p, l);
                    if (pl.v_curl[x] != hm.curlc[3 * (size_t)v + j]) return fail("vertex curl coefficient", p, l);
                } else if (le != nE2 || pl.v_curl[x] != 0.0) {
                    return fail("absent vertex edge is not the zero slot", p, l);
                }
                if (c >= 0) {
                    if (lc >= nC2 || cg[lc] != c) return fail("vertex cell", p, l);
                    if (pl.v_kw[x] != hm.kw[3 * (size_t)v + j]) return fail("vertex kite weight", p, l);
                } else if (lc != nC2 || pl.v_kw[x] != 0.0) {
                    return fail("absent vertex cell is not the zero slot", p, l);
                }
            }
        }
    }
    for (int e = 0; e < E; e++) if (owner[e] < 0) return fail("edge not owned", -1, e);

    // the fused thickness kernel's plan (128 cells per patch, as the library uses)
    ThickPlan tp;
    const int Tc = 128;
    if (!build_thick_plan(hm, Tc, tp)) { printf("violation: no thickness plan\n"); return 1; }
    std::vector<int> towned(C, 0);
    for (int p = 0; p < tp.P; p++) {
        const int nO = tp.cnt[4 * p], nEO = tp.cnt[4 * p + 1], nC1 = tp.cnt[4 * p + 2];
        if (nO > Tc) return fail("thickness patch above the kernel's threads", p, -1);
        if (nEO > tp.maxEO || nC1 > tp.maxC1 || nO > nC1) return fail("thickness counts", p, -1);
        if (tp.off_eo[p + 1] - tp.off_eo[p] != nEO || tp.off_c1[p + 1] - tp.off_c1[p] != nC1)
            return fail("thickness offsets", p, -1);
        const int *eg = &tp.eogid[tp.off_eo[p]], *cg = &tp.c1gid[tp.off_c1[p]];
        for (int l = 0; l < nEO; l++) if (eg[l] < 0 || eg[l] >= E) return fail("thickness edge gid", p, l);
        for (int l = 0; l < nC1; l++) if (cg[l] < 0 || cg[l] >= C) return fail("thickness cell gid", p, l);
        for (int l = 0; l < nO; l++) {
            if (tp.owner[cg[l]] != p) return fail("owned cell of another patch", p, l);
            if (towned[cg[l]]++) return fail("cell owned twice", p, l);
        }
        for (int l = 0; l < Tc; l++) {
            const int c = l < nO ? cg[l] : -1;
            for (int j = 0; j < BCL_NCEP; j++) {
                const size_t x = (size_t)BCL_NCEP * Tc * p + (size_t)j * Tc + l;
                const int le = tp.o_e[x], lo = tp.o_o[x];
                if (l < nO && j < hm.neoc[c]) {
                    const int e = hm.eoc[(size_t)c * mE + j];
                    if (le >= nEO || eg[le] != e) return fail("thickness cell edge", p, l);
                    if (lo >= nC1 || cg[lo] != (hm.c1[e] == c ? hm.c2[e] : hm.c1[e]))
                        return fail("thickness cell neighbour", p, l);
                } else if (le != nEO || lo >= nC1) {
                    return fail("thickness padding is not the zero slot", p, l);
                }
            }
        }
    }
    for (int c = 0; c < C; c++) if (!towned[c]) return fail("cell not owned by a thickness patch", -1, c);
    printf("ok\n");
    return 0;
}
