// api.cu -- C ABI of libsse.so (include/sse.h): mesh validation and upload,
// state management and the SSPRK2-SE / SSPRK3-SE step driver.
//
// The driver issues, per large step, the stage kernels in the order of the
// paper's schemes (Sec. 3.2 for SSPRK2-SE, Sec. 3.3 for SSPRK3-SE, with the
// reconciliation of Sec. 3.4).  The state is kept as (ubar, utilde, h,
// tracers, zeta) on the device; u = ubar + utilde is formed where it is read.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <type_traits>

#include <nvtx3/nvToolsExt.h>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/sse.h"
#include "sse_internal.cuh"
#include "tiles.h"

using namespace sse;

namespace {

// No exception crosses the C ABI: the entry points run their bodies through
// this.  The library's host containers (plans, staging vectors, graph and
// arena caches) report a failed allocation by throwing std::bad_alloc, which
// becomes SSE_ERR_OOM; anything else thrown becomes SSE_ERR_INTERNAL.
template <class F> int guarded(F &&f) noexcept {
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return SSE_ERR_OOM;
    } catch (...) {
        return SSE_ERR_INTERNAL;
    }
}

// an NVTX range that closes however its scope is left
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

constexpr int kAlign = 32;
inline int pad(int n) { return (n + kAlign - 1) / kAlign * kAlign; }

// RAII list of device allocations.  Meshes allocate with cudaMalloc; states
// allocate stream-ordered on their own stream (cudaMallocAsync / cudaFreeAsync)
// so that creating or destroying one state never synchronises the device
// while others run.  In counting mode nothing is allocated: the arena only
// sums the sizes (the footprint of a state before it is made).
struct DevArena {
    std::vector<void *> ptrs;
    bool failed = false;
    bool async = false;
    bool count_only = false;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;
    template <class T> T *alloc(size_t n) {
        const size_t nb = std::max<size_t>(n, 1) * sizeof(T);
        bytes += (nb + 255) / 256 * 256;
        if (count_only) return reinterpret_cast<T *>((uintptr_t)256);  // never dereferenced
        void *p = nullptr;
        const cudaError_t e = async ? cudaMallocAsync(&p, nb, stream) : cudaMalloc(&p, nb);
        if (e != cudaSuccess) {
            failed = true;
            cudaGetLastError();
            return nullptr;
        }
        if (async) cudaMemsetAsync(p, 0, nb, stream);
        else cudaMemset(p, 0, nb);
        ptrs.push_back(p);
        return (T *)p;
    }
    template <class T> T *upload(const std::vector<T> &v) {
        T *d = alloc<T>(v.size());
        if (count_only || !d || v.empty()) return d;
        const cudaError_t e =
            async ? cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, stream)
                  : cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) failed = true;
        return d;
    }
    ~DevArena() {
        for (void *p : ptrs) {
            if (async) cudaFreeAsync(p, stream);
            else cudaFree(p);
        }
    }
};

}  // namespace

struct sse_mesh {
    DMesh dm;
    DevArena arena;
    int device = 0;
    HostMesh host;  // connectivity kept for the tiled sub-cycle plan
    // tile plans already built for this mesh, by patch count (host data only;
    // every state uploads its own copy)
    std::mutex plan_mu;
    std::map<int, std::shared_ptr<const TilePlan>> plans;
    // fused baroclinic plans already built, by cells per patch (null: no fit)
    std::map<int, std::shared_ptr<const BclPlan>> bcl_plans;
    // fused thickness plan (null: no fit), built once
    std::shared_ptr<const ThickPlan> thick_plan;
    bool thick_tried = false;
    std::map<int, int> tuned;   // autotuned patch size by (precision, objective)
};

// ---------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------
static int mesh_create_impl(const sse_mesh_desc *d, sse_mesh **out) {
    if (!d || !out) return SSE_ERR_INVALID_ARG;
    *out = nullptr;
    const int C = d->nCells, E = d->nEdges, V = d->nVertices, mE = d->maxEdges,
              mE2 = d->maxEdges2, L = d->nLayers;
    if (C < 1 || E < 1 || V < 1 || mE < 3 || mE2 < 1 || L < 1) return SSE_ERR_INVALID_ARG;
    if (mE > MAXE || mE2 > MAXE2 || L > LMAX) return SSE_ERR_UNSUPPORTED;
    if (!d->cellsOnEdge || !d->verticesOnEdge || !d->nEdgesOnCell || !d->edgesOnCell ||
        !d->cellsOnVertex || !d->edgesOnVertex || !d->nEdgesOnEdge || !d->edgesOnEdge ||
        !d->weightsOnEdge || !d->dcEdge || !d->dvEdge || !d->areaCell || !d->areaTriangle ||
        !d->kiteAreasOnVertex || !d->fEdge || !d->fVertex || !d->bottomDepth ||
        !d->restThicknessFrac)
        return SSE_ERR_INVALID_ARG;
    // ---- validation
    for (int e = 0; e < E; e++) {
        for (int s = 0; s < 2; s++) {
            int c = d->cellsOnEdge[2 * e + s], v = d->verticesOnEdge[2 * e + s];
            if (c < 0 || c >= C || v < 0 || v >= V) return SSE_ERR_BAD_MESH;
        }
        if (d->cellsOnEdge[2 * e] == d->cellsOnEdge[2 * e + 1]) return SSE_ERR_BAD_MESH;
        if (!(d->dcEdge[e] > 0) || !(d->dvEdge[e] > 0) || !isfinite(d->fEdge[e]))
            return SSE_ERR_BAD_MESH;
        int n = d->nEdgesOnEdge[e];
        if (n < 0 || n > mE2) return SSE_ERR_BAD_MESH;
        for (int j = 0; j < n; j++) {
            int ep = d->edgesOnEdge[(size_t)e * mE2 + j];
            if (ep < 0 || ep >= E || !isfinite(d->weightsOnEdge[(size_t)e * mE2 + j]))
                return SSE_ERR_BAD_MESH;
        }
    }
    for (int i = 0; i < C; i++) {
        int n = d->nEdgesOnCell[i];
        if (n < 1 || n > mE || !(d->areaCell[i] > 0) || !(d->bottomDepth[i] > 0))
            return SSE_ERR_BAD_MESH;
        for (int j = 0; j < n; j++) {
            int e = d->edgesOnCell[(size_t)i * mE + j];
            if (e < 0 || e >= E) return SSE_ERR_BAD_MESH;
            if (d->cellsOnEdge[2 * e] != i && d->cellsOnEdge[2 * e + 1] != i) return SSE_ERR_BAD_MESH;
        }
    }
    for (int v = 0; v < V; v++) {
        double ksum = 0.0;
        if (!(d->areaTriangle[v] > 0) || !isfinite(d->fVertex[v])) return SSE_ERR_BAD_MESH;
        for (int j = 0; j < 3; j++) {
            int c = d->cellsOnVertex[3 * v + j], e = d->edgesOnVertex[3 * v + j];
            if (c < -1 || c >= C || e < -1 || e >= E) return SSE_ERR_BAD_MESH;
            if (e >= 0 && d->verticesOnEdge[2 * e] != v && d->verticesOnEdge[2 * e + 1] != v)
                return SSE_ERR_BAD_MESH;
            if (c >= 0) {
                if (!(d->kiteAreasOnVertex[3 * v + j] >= 0)) return SSE_ERR_BAD_MESH;
                ksum += d->kiteAreasOnVertex[3 * v + j];
            }
        }
        if (!(ksum > 0)) return SSE_ERR_BAD_MESH;
    }
    {
        double s = 0.0;
        for (int k = 0; k < L; k++) {
            if (!(d->restThicknessFrac[k] > 0)) return SSE_ERR_BAD_MESH;
            s += d->restThicknessFrac[k];
        }
        if (fabs(s - 1.0) > 1e-12) return SSE_ERR_BAD_MESH;
    }
    const bool partial = d->maxLevelCell != nullptr;
    if (partial != (d->restThickness != nullptr)) return SSE_ERR_INVALID_ARG;
    if (partial)
        for (int i = 0; i < C; i++) {
            const int K = d->maxLevelCell[i];
            if (K < 1 || K > L) return SSE_ERR_BAD_MESH;
            double s = 0.0;
            for (int k = 0; k < L; k++) {
                const double r = d->restThickness[(size_t)i * L + k];
                if (k < K ? !(r > 0) : r != 0.0) return SSE_ERR_BAD_MESH;
                s += r;
            }
            if (!(fabs(s - d->bottomDepth[i]) <= 1e-10 * d->bottomDepth[i])) return SSE_ERR_BAD_MESH;
        }

    // ---- internal numbering of cells and edges.  Cells follow the depth-first
    // order of a recursive bisection of the cell graph (any run of consecutive
    // cells is a compact region), edges the order of their lower-numbered
    // cell, vertices (below) the order of their lowest cell: a block of
    // consecutive columns then gathers its neighbours from a few cache lines
    // whatever the caller's numbering.  Every per-cell and per-edge field
    // crosses the API in the caller's numbering (the set/get kernels permute);
    // everything below works on the renumbered copy of the description.
    std::vector<int> cold, cnew(C), eold(E), enew(E);
    {
        std::vector<int> a(E), b(E);
        for (int e = 0; e < E; e++) { a[e] = d->cellsOnEdge[2 * e]; b[e] = d->cellsOnEdge[2 * e + 1]; }
        cold = cell_locality_order(C, a, b, 8);
        for (int i = 0; i < C; i++) cnew[cold[i]] = i;
        std::vector<long long> key(E);
        for (int e = 0; e < E; e++) {
            const long long x = cnew[a[e]], y = cnew[b[e]];
            key[e] = (std::min(x, y) * C + std::max(x, y)) * (long long)E + e;
        }
        std::iota(eold.begin(), eold.end(), 0);
        std::sort(eold.begin(), eold.end(), [&](int p, int q) { return key[p] < key[q]; });
        for (int e = 0; e < E; e++) enew[eold[e]] = e;
    }
    std::vector<int32_t> r_coe(2 * E), r_voe(2 * E), r_neoc(C), r_eoc((size_t)C * mE, 0);
    std::vector<int32_t> r_cov(3 * V), r_eov(3 * V), r_neoe(E), r_eoe((size_t)E * mE2, 0);
    std::vector<double> r_woe((size_t)E * mE2, 0.0), r_dc(E), r_dv(E), r_area(C), r_fE(E), r_H(C);
    std::vector<int32_t> r_mlc;
    std::vector<double> r_rest;
    for (int e = 0; e < E; e++) {
        const int o = eold[e];
        for (int s = 0; s < 2; s++) {
            r_coe[2 * e + s] = cnew[d->cellsOnEdge[2 * o + s]];
            r_voe[2 * e + s] = d->verticesOnEdge[2 * o + s];
        }
        r_neoe[e] = d->nEdgesOnEdge[o];
        for (int j = 0; j < r_neoe[e]; j++) {
            r_eoe[(size_t)e * mE2 + j] = enew[d->edgesOnEdge[(size_t)o * mE2 + j]];
            r_woe[(size_t)e * mE2 + j] = d->weightsOnEdge[(size_t)o * mE2 + j];
        }
        r_dc[e] = d->dcEdge[o]; r_dv[e] = d->dvEdge[o]; r_fE[e] = d->fEdge[o];
    }
    for (int i = 0; i < C; i++) {
        const int o = cold[i];
        r_neoc[i] = d->nEdgesOnCell[o];
        for (int j = 0; j < r_neoc[i]; j++)
            r_eoc[(size_t)i * mE + j] = enew[d->edgesOnCell[(size_t)o * mE + j]];
        r_area[i] = d->areaCell[o]; r_H[i] = d->bottomDepth[o];
    }
    for (int v = 0; v < 3 * V; v++) {
        r_cov[v] = d->cellsOnVertex[v] >= 0 ? cnew[d->cellsOnVertex[v]] : -1;
        r_eov[v] = d->edgesOnVertex[v] >= 0 ? enew[d->edgesOnVertex[v]] : -1;
    }
    if (partial) {
        r_mlc.resize(C);
        r_rest.resize((size_t)C * L);
        for (int i = 0; i < C; i++) {
            r_mlc[i] = d->maxLevelCell[cold[i]];
            for (int k = 0; k < L; k++)
                r_rest[(size_t)i * L + k] = d->restThickness[(size_t)cold[i] * L + k];
        }
    }
    sse_mesh_desc rd = *d;
    rd.cellsOnEdge = r_coe.data(); rd.verticesOnEdge = r_voe.data();
    rd.nEdgesOnCell = r_neoc.data(); rd.edgesOnCell = r_eoc.data();
    rd.cellsOnVertex = r_cov.data(); rd.edgesOnVertex = r_eov.data();
    rd.nEdgesOnEdge = r_neoe.data(); rd.edgesOnEdge = r_eoe.data();
    rd.weightsOnEdge = r_woe.data(); rd.dcEdge = r_dc.data(); rd.dvEdge = r_dv.data();
    rd.areaCell = r_area.data(); rd.fEdge = r_fE.data(); rd.bottomDepth = r_H.data();
    if (partial) { rd.maxLevelCell = r_mlc.data(); rd.restThickness = r_rest.data(); }
    d = &rd;

    // ---- derived, padded, layer-major arrays
    const int Cp = pad(C), Ep = pad(E), Vp = pad(V);
    std::vector<int2> coe(Ep, make_int2(0, 0)), voe(Ep, make_int2(0, 0));
    std::vector<int> neoc(Cp, 0), eoc((size_t)mE * Cp, 0), ooc((size_t)mE * Cp, 0);
    std::vector<int> neoe(Ep, 0), eoe((size_t)mE2 * Ep, 0), eov(3 * Vp, 0), cov(3 * Vp, 0);
    std::vector<double> H(Cp, 1.0), sfrac(d->restThicknessFrac, d->restThicknessFrac + L);
    std::vector<double> divc((size_t)mE * Cp, 0.0), kec((size_t)mE * Cp, 0.0);
    std::vector<double> wl((size_t)mE2 * Ep, 0.0), cfc((size_t)mE2 * Ep, 0.0);
    std::vector<double> curlc(3 * Vp, 0.0), kw(3 * Vp, 0.0), invdc(Ep, 1.0), invdv(Ep, 1.0);
    std::vector<double> fV(Vp, 0.0), area(Cp, 0.0), ld2(Ep, 0.0);
    // Vertices are numbered internally in the order of their lowest cell, so that
    // a warp of consecutive vertices gathers from nearby cells and edges (the
    // caller's numbering may be arbitrary; vertex data never crosses the API).
    std::vector<int> vold(V), vnew(V);
    {
        std::vector<long long> key(V);
        for (int v = 0; v < V; v++) {
            int lo = C;
            for (int j = 0; j < 3; j++) {
                const int c = d->cellsOnVertex[3 * v + j];
                if (c >= 0 && c < lo) lo = c;
            }
            key[v] = (long long)lo * V + v;   // ties keep the caller's order
        }
        std::iota(vold.begin(), vold.end(), 0);
        std::sort(vold.begin(), vold.end(), [&](int a, int b) { return key[a] < key[b]; });
        for (int nv = 0; nv < V; nv++) vnew[vold[nv]] = nv;
    }
    for (int e = 0; e < E; e++) {
        coe[e] = make_int2(d->cellsOnEdge[2 * e], d->cellsOnEdge[2 * e + 1]);
        voe[e] = make_int2(vnew[d->verticesOnEdge[2 * e]], vnew[d->verticesOnEdge[2 * e + 1]]);
        invdc[e] = 1.0 / d->dcEdge[e];
        invdv[e] = 1.0 / d->dvEdge[e];
        ld2[e] = 0.5 * d->dvEdge[e] * d->dcEdge[e];
        neoe[e] = d->nEdgesOnEdge[e];
        for (int j = 0; j < neoe[e]; j++) {
            int ep = d->edgesOnEdge[(size_t)e * mE2 + j];
            eoe[(size_t)j * Ep + e] = ep;
            double w = d->weightsOnEdge[(size_t)e * mE2 + j] * d->dvEdge[ep] / d->dcEdge[e];
            wl[(size_t)j * Ep + e] = w;
            cfc[(size_t)j * Ep + e] = w * 0.5 * (d->fEdge[e] + d->fEdge[ep]);
        }
    }
    for (int i = 0; i < C; i++) {
        H[i] = d->bottomDepth[i];
        area[i] = d->areaCell[i];
        neoc[i] = d->nEdgesOnCell[i];
        for (int j = 0; j < neoc[i]; j++) {
            int e = d->edgesOnCell[(size_t)i * mE + j];
            int c1 = d->cellsOnEdge[2 * e], c2 = d->cellsOnEdge[2 * e + 1];
            eoc[(size_t)j * Cp + i] = e;
            ooc[(size_t)j * Cp + i] = (c1 == i) ? c2 : c1;
            divc[(size_t)j * Cp + i] = ((c1 == i) ? 1.0 : -1.0) * d->dvEdge[e] / d->areaCell[i];
            kec[(size_t)j * Cp + i] = 0.25 * d->dvEdge[e] * d->dcEdge[e] / d->areaCell[i];
        }
    }
    for (int nv = 0; nv < V; nv++) {
        const int v = vold[nv];   // the caller's index
        fV[nv] = d->fVertex[v];
        double ksum = 0.0;
        for (int j = 0; j < 3; j++)
            if (d->cellsOnVertex[3 * v + j] >= 0) ksum += d->kiteAreasOnVertex[3 * v + j];
        for (int j = 0; j < 3; j++) {
            int e = d->edgesOnVertex[3 * v + j], c = d->cellsOnVertex[3 * v + j];
            if (e >= 0) {
                eov[(size_t)j * Vp + nv] = e;
                double sign = (d->verticesOnEdge[2 * e + 1] == v) ? 1.0 : -1.0;
                curlc[(size_t)j * Vp + nv] = sign * d->dcEdge[e] / d->areaTriangle[v];
            }
            if (c >= 0) {
                cov[(size_t)j * Vp + nv] = c;
                kw[(size_t)j * Vp + nv] = d->kiteAreasOnVertex[3 * v + j] / ksum;
            }
        }
    }
    auto tof = [](const std::vector<double> &x) {
        return std::vector<float>(x.begin(), x.end());
    };

    // owned here until it is handed out, so that a failure on the way frees it
    std::unique_ptr<sse_mesh> hold(new (std::nothrow) sse_mesh());
    sse_mesh *m = hold.get();
    if (!m) return SSE_ERR_OOM;
    {
        HostMesh &hm = m->host;
        hm.C = C; hm.E = E; hm.V = V; hm.maxE = mE; hm.maxE2 = mE2;
        hm.c1.resize(E); hm.c2.resize(E); hm.v1.resize(E); hm.v2.resize(E);
        hm.neoe.resize(E); hm.invdc.resize(E); hm.invdv.resize(E);
        hm.eoe.assign((size_t)E * mE2, 0); hm.cfc.assign((size_t)E * mE2, 0.0);
        hm.wl.assign((size_t)E * mE2, 0.0);
        for (int e = 0; e < E; e++) {
            hm.c1[e] = coe[e].x; hm.c2[e] = coe[e].y; hm.neoe[e] = neoe[e];
            hm.v1[e] = voe[e].x; hm.v2[e] = voe[e].y;
            hm.invdc[e] = invdc[e]; hm.invdv[e] = invdv[e];
            for (int j = 0; j < neoe[e]; j++) {
                hm.eoe[(size_t)e * mE2 + j] = eoe[(size_t)j * Ep + e];
                hm.cfc[(size_t)e * mE2 + j] = cfc[(size_t)j * Ep + e];
                hm.wl[(size_t)e * mE2 + j] = wl[(size_t)j * Ep + e];
            }
        }
        hm.neoc.resize(C); hm.eoc.assign((size_t)C * mE, 0); hm.divc.assign((size_t)C * mE, 0.0);
        hm.kec.assign((size_t)C * mE, 0.0);
        hm.H.resize(C);
        for (int i = 0; i < C; i++) {
            hm.neoc[i] = neoc[i]; hm.H[i] = H[i];
            for (int j = 0; j < neoc[i]; j++) {
                hm.eoc[(size_t)i * mE + j] = eoc[(size_t)j * Cp + i];
                hm.divc[(size_t)i * mE + j] = divc[(size_t)j * Cp + i];
                hm.kec[(size_t)i * mE + j] = kec[(size_t)j * Cp + i];
            }
        }
        // vertices in the internal numbering; absent edges and cells -1
        hm.eov.assign(3 * (size_t)V, -1); hm.cov.assign(3 * (size_t)V, -1);
        hm.curlc.assign(3 * (size_t)V, 0.0); hm.kw.assign(3 * (size_t)V, 0.0);
        hm.fV.resize(V);
        for (int nv = 0; nv < V; nv++) {
            const int v = vold[nv];
            hm.fV[nv] = fV[nv];
            for (int j = 0; j < 3; j++) {
                if (d->edgesOnVertex[3 * v + j] >= 0) {
                    hm.eov[3 * (size_t)nv + j] = eov[(size_t)j * Vp + nv];
                    hm.curlc[3 * (size_t)nv + j] = curlc[(size_t)j * Vp + nv];
                }
                if (d->cellsOnVertex[3 * v + j] >= 0) {
                    hm.cov[3 * (size_t)nv + j] = cov[(size_t)j * Vp + nv];
                    hm.kw[3 * (size_t)nv + j] = kw[(size_t)j * Vp + nv];
                }
            }
        }
    }
    cudaGetDevice(&m->device);
    DevArena &A = m->arena;
    DMesh &dm = m->dm;
    dm.C = C; dm.E = E; dm.V = V; dm.L = L; dm.Cp = Cp; dm.Ep = Ep; dm.Vp = Vp;
    dm.maxE = mE; dm.maxE2 = mE2;
    dm.coe = A.upload(coe); dm.voe = A.upload(voe);
    dm.neoc = A.upload(neoc); dm.eoc = A.upload(eoc); dm.ooc = A.upload(ooc);
    dm.neoe = A.upload(neoe); dm.eoe = A.upload(eoe); dm.eov = A.upload(eov);
    dm.cov = A.upload(cov); dm.H = A.upload(H); dm.sfrac = A.upload(sfrac);
    dm.sfrac_f = A.upload(tof(sfrac));
    dm.divc_d = A.upload(divc); dm.area = A.upload(area); dm.ld2 = A.upload(ld2);
    dm.d.divc = dm.divc_d; dm.d.kec = A.upload(kec); dm.d.wl = A.upload(wl);
    dm.d.cfc = A.upload(cfc); dm.d.curlc = A.upload(curlc); dm.d.kw = A.upload(kw);
    dm.d.invdc = A.upload(invdc); dm.d.invdv = A.upload(invdv); dm.d.fV = A.upload(fV);
    dm.d.H = dm.H; dm.f.H = A.upload(tof(H));
    dm.f.divc = A.upload(tof(divc)); dm.f.kec = A.upload(tof(kec)); dm.f.wl = A.upload(tof(wl));
    dm.f.cfc = A.upload(tof(cfc)); dm.f.curlc = A.upload(tof(curlc)); dm.f.kw = A.upload(tof(kw));
    dm.f.invdc = A.upload(tof(invdc)); dm.f.invdv = A.upload(tof(invdv));
    dm.f.fV = A.upload(tof(fV));
    // caller index -> internal index (set/get) and internal -> caller
    cnew.resize(Cp, 0); enew.resize(Ep, 0);
    cold.resize(Cp, 0); eold.resize(Ep, 0);
    dm.cperm = A.upload(cnew); dm.eperm = A.upload(enew);
    dm.cinv = A.upload(cold); dm.einv = A.upload(eold);
    dm.partial = partial ? 1 : 0;
    dm.kc = nullptr; dm.ke = nullptr; dm.sfc = nullptr; dm.sfc_f = nullptr;
    if (partial) {
        std::vector<int> kc(Cp, L), ke(Ep, L);
        std::vector<double> sfc((size_t)L * Cp, 0.0);
        for (int i = 0; i < C; i++) {
            kc[i] = d->maxLevelCell[i];
            for (int k = 0; k < L; k++)
                sfc[(size_t)k * Cp + i] = d->restThickness[(size_t)i * L + k] / d->bottomDepth[i];
        }
        for (int e = 0; e < E; e++) ke[e] = std::min(kc[coe[e].x], kc[coe[e].y]);
        dm.kc = A.upload(kc); dm.ke = A.upload(ke);
        dm.sfc = A.upload(sfc); dm.sfc_f = A.upload(tof(sfc));
    }
    if (A.failed) return SSE_ERR_OOM;
    *out = hold.release();
    return SSE_OK;
}

extern "C" int sse_mesh_create(const sse_mesh_desc *d, sse_mesh **out) {
    return guarded([&] { return mesh_create_impl(d, out); });
}

extern "C" void sse_mesh_destroy(sse_mesh *m) { delete m; }

const sse::DMesh *sse_internal_dmesh(const sse_mesh *m) { return &m->dm; }
int sse_internal_device(const sse_mesh *m) { return m->device; }

// ---------------------------------------------------------------------------
// Device address of page-locked host memory (cudaHostAlloc, cudaHostRegister)
// mapped for the current device, or null for any other pointer.  The state's
// set/get kernels then read or write such host buffers directly, which saves
// the staging copy through device memory.
static void *host_alias(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || at.type != cudaMemoryTypeHost ||
        at.device != dev || !at.devicePointer)
        return nullptr;
    return at.devicePointer;
}

// state: a precision-specific engine behind a small virtual interface
// ---------------------------------------------------------------------------
struct EngineBase {
    virtual int set(int field, const double *host) = 0;
    virtual int get(int field, double *host) = 0;
    virtual int set_f32(int field, const float *host) = 0;
    virtual int get_f32(int field, float *host) = 0;
    virtual int transfer(int field, void *host, int flags) = 0;   // sse_state_transfer
    virtual int sync() = 0;                                       // sse_state_sync
    virtual int step(int order, double dt, int M) = 0;
    virtual int step2(int order, double dt, int M) = 0;   // two steps, replayed from a graph
    virtual int graph_count() const = 0;                  // step-pair graphs held
    virtual int bcl_feuler(double dt) = 0;
    virtual int btr_substep(int order, double dt, int M) = 0;
    virtual int patches() const = 0;       // tiled sub-cycle patches (0: global kernel)
    virtual int patch_threads() const = 0; // threads per patch of the tiled sub-cycle
    virtual int patch_tmem() const = 0;    // 1: the tiled sub-cycle's edge data in tensor memory
    virtual int bcl_patch_cells() const = 0;   // cells per fused baroclinic patch (0: unfused)
    virtual int bcl_patch_count() const = 0;   // fused baroclinic patches (0: unfused)
    unsigned int inject_stall = 0;         // sse_state_inject(SSE_INJECT_BARRIER_STALL)
    virtual bool has_del4() const = 0;     // biharmonic viscosity on
    virtual bool fused_bcl() const = 0;    // the fused baroclinic stage is used
    virtual int diagnostics(sse_diag *out) = 0;
    long long steps = 0;

    // ---- optional per-launch event timing
    bool prof = false;
    std::vector<cudaEvent_t> pool;
    struct Rec { int cls; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    cudaStream_t ps = nullptr;
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // An NVTX range per kernel class (visible to nsys and other NVTX tools,
    // no-ops otherwise); with profiling on, CUDA events around the launch.
    void pbeg(int cls) {
        static const char *const names[SSE_K_NCLASS] = {
            "sse cell_diag", "sse vertex", "sse edge_pre", "sse bcl_edge", "sse btr",
            "sse transport", "sse thickness", "sse combine", "sse del4"};
        nvtxRangePushA(names[cls]);
        if (!prof) return;
        Rec r{cls, take(), take()};
        cudaEventRecord(r.a, ps);
        recs.push_back(r);
    }
    void pend() {
        nvtxRangePop();
        if (!prof || recs.empty()) return;
        cudaEventRecord(recs.back().b, ps);
    }
    void prof_clear() {
        for (auto &r : recs) { pool.push_back(r.a); pool.push_back(r.b); }
        recs.clear();
    }
    int prof_read(double *ms, int32_t *n) {
        for (int c = 0; c < SSE_K_NCLASS; c++) { ms[c] = 0.0; n[c] = 0; }
        if (cudaStreamSynchronize(ps) != cudaSuccess) return SSE_ERR_CUDA;
        for (auto &r : recs) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return SSE_ERR_CUDA;
            ms[r.cls] += t;
            n[r.cls] += 1;
        }
        return SSE_OK;
    }
    virtual ~EngineBase() {
        prof_clear();
        for (auto e : pool) cudaEventDestroy(e);
    }
};

#define CK(x)                                                        \
    do {                                                             \
        cudaError_t _e = (x);                                        \
        if (_e != cudaSuccess) {                                     \
            fprintf(stderr, "libsse: %s -> %s\n", #x, cudaGetErrorString(_e)); \
            return SSE_ERR_CUDA;                                     \
        }                                                            \
    } while (0)

// One launch of a step, recorded instead of issued (sse_step_batch): the
// batched driver replays the i-th launch of every state as one grid.
enum RecClass { REC_COLFLUX, REC_BCL, REC_BTR, REC_TRANSPORT, REC_THICK, REC_COMBINE };
template <class R> struct CombineJob {
    const R *a, *b, *c;
    R *out;
    double wa, wb, wc;
    int n, pad_;
};
template <class R> struct LaunchRec {
    int cls = 0;
    size_t smem = 0;
    union U {
        ColfluxJob<R> cf;
        BclJob<R> bcl;
        TransportJob<R> tr;
        ThickJob<R> th;
        BtrArgs<R> btr;
        CombineJob<R> cmb;
        U() {}
    } u;
};

template <class R>
struct Engine : EngineBase {
    std::vector<LaunchRec<R>> *rec = nullptr;   // set: record launches, do not issue them
    DMesh m;
    DParams p{};
    int recon = SSE_RECON_CONSISTENT;
    bool mixed = false;
    bool vmix = false;   // Algorithm 2 in every baroclinic stage
    int patch_cells = 0;   // target cells per sub-cycle patch (sse_tuning; 0: default)
    int bcl_cells = 0;     // cells per fused baroclinic patch (sse_tuning; 0: default)
    int bcl_pc = 0;        // the patch size the fused baroclinic plan uses (0: unfused)
    int bcl_patch_cells() const override { return fused ? bcl_pc : 0; }
    int bcl_patch_count() const override { return fused ? bcl.P : 0; }
    cudaStream_t s = nullptr;
    DevArena A;
    // state
    R *ubar_n, *ut_n;
    double *h_n, *zeta_n;
    R *hR_n, *tr_n;
    double toff[2] = {0.0, 0.0};   // tracer t is held as tracer - toff[t]
    // stage buffers
    R *ut_1, *ut_c, *ut_3, *ubar_1, *ubar_h, *ubar_np1;
    R *G0, *G1, *G2, *Gw;
    double *Fz1, *Fz2, *Fz3, *S1, *S2, *zeta_sub, *last_Fz;
    double *h_1, *h_h, *zeta_1, *zeta_h;
    R *hR_1, *hR_h, *tr_1, *tr_h;
    R *flux;
    double *Fcol;
    DiagBufs<R> db;
    R *bu0, *bua, *buh, *bz0, *bza, *bzh;
    unsigned int *barwords;
    int *barerr;
    double *stage;   // staging for host transfers
    double *wind, *wind_d;
    float *wind_f;
    double *dpart, *dout;
    int dparts = 0;
    int btr_blocks = 1;
    bool tiled = false;
    DTiles<R> tiles{};
    bool fused = false;   // the baroclinic stage as k_colflux + k_bcl_fused
    DBcl<R> bcl{};
    R *Fc = nullptr;      // [Ep] column transport of the stage (k_colflux)
    bool fused_th = false;   // the thickness stage as k_transport_cols + k_thick_fused
    DThick thk{};
    R *uA_e = nullptr;       // [Ep] transport adjustment u^A of the stage
    TransportArgs<R> last_ta{};   // the transport velocity the next thickness stage uses

    // Plan the tiled sub-cycle: patches of about patch_cells owned cells, halo
    // of 3 rings (one SSPRK3 sub-step per exchange).  The default (0) is one
    // patch per SM (at most nSM patches of >= 64 cells) in 1024-thread
    // blocks.  An explicit patch size may ask for up to two patches per SM:
    // those run as 512-thread blocks holding at most half an SM's shared
    // memory each.  Patches small enough that 512 threads do the same work
    // per thread as 1024 (at most 512 entries of each kind) also take
    // 512-thread blocks, so that the sub-cycles of two states can share an SM.
    int plan_tiles(const sse_mesh *mesh, int dev, int nsm) {
        const char *env = getenv("SSE_BTR_KERNEL");
        if (env && strcmp(env, "global") == 0) return SSE_OK;
        int smem_block = 0, smem_sm = 0;
        CK(cudaDeviceGetAttribute(&smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        if (m.maxE2 > 10 || m.maxE > TILE_NCEP) return SSE_OK;
        if (!tile_stencil_ok(mesh->host)) return SSE_OK;   // the global sub-cycle is exact for any stencil
        // a plan whose patches are too large for their block is retried with
        // more patches
        const int Pmax = patch_cells > 0 ? 2 * nsm : nsm;
        const int pc = patch_cells > 0 ? patch_cells : 64;
        int P0 = std::max(1, std::min(Pmax, m.C / pc));
        for (int k = 1, P = P0; P > 0;
             k++, P = (P >= Pmax) ? 0 : std::min(Pmax, std::max(P + 1, P * 5 / 4))) {
            const bool verbose = getenv("SSE_VERBOSE") != nullptr;
            std::shared_ptr<const TilePlan> cached;
            {
                sse_mesh *mm = const_cast<sse_mesh *>(mesh);
                std::lock_guard<std::mutex> lk(mm->plan_mu);
                auto it = mm->plans.find(P);
                if (it != mm->plans.end()) {
                    cached = it->second;
                } else {
                    auto fresh = std::make_shared<TilePlan>();
                    if (!build_tile_plan(mesh->host, P, 3, *fresh)) fresh.reset();
                    mm->plans[P] = fresh;
                    cached = fresh;
                }
            }
            if (!cached) {
                if (verbose) fprintf(stderr, "libsse: tile plan k=%d: 16-bit local index overflow\n", k);
                continue;
            }
            const TilePlan &plan = *cached;
            // 16-bit byte offsets; at most 3 entries of each kind per thread
            int most = 0;
            bool small = true;
            for (const TilePatch &t : plan.patches) {
                if ((size_t)(t.ne + 1) * sizeof(R) >= 65536 || (size_t)(t.nc + 1) * sizeof(R) >= 65536)
                    small = false;
                most = std::max(most, std::max(std::max(t.n_own_e, t.ne - t.n_own_e),
                                               std::max(t.n_own_c, t.nc - t.n_own_c)));
            }
            const size_t smem = tile_smem_bytes(plan, m.maxE, m.maxE2, sizeof(R));
            // the runtime reserves 1 KB of shared memory per block
            const bool half_sm = most <= 3 * 512 && smem <= (size_t)smem_block &&
                                 2 * (smem + 1024) <= (size_t)smem_sm;
            const bool whole_sm = P <= nsm && most <= 3 * 1024 && smem <= (size_t)smem_block &&
                                  smem + 1024 <= (size_t)smem_sm;
            int nthreads = 0;
            if (half_sm && (P > nsm || most <= 512)) nthreads = 512;
            else if (whole_sm) nthreads = 1024;
            if (!small || nthreads == 0) {
                if (verbose)
                    fprintf(stderr, "libsse: tile plan k=%d P=%d: patch too large (%d entries, "
                            "smem %zu, limits %d/%d)\n", k, P, most, smem, smem_block, smem_sm);
                continue;
            }
            const int own = std::max(2, (most + nthreads - 1) / nthreads);
            // FP32 1024-thread patches keep their edges' constant data in
            // tensor memory when every patch has at most that variant's slots
            // of edges per thread (SSE_BTR_TMEM=0 turns it off)
            const char *tenv = getenv("SSE_BTR_TMEM");
            int mne = 0;
            for (const TilePatch &t : plan.patches) mne = std::max(mne, t.ne);
            const bool tm = sizeof(R) == 4 && nthreads == 1024 && mne <= btr_tiled_tmem_slots() * 1024 &&
                            !(tenv && strcmp(tenv, "0") == 0);

            // the attribute belongs to the kernel, not to this state: allow the
            // device's whole opt-in size so that states of other meshes, whose
            // plans need less or more, never lower it under each other
            int static_smem = 0;
            for (int o = 2; o <= 3; o++) {
                cudaFuncAttributes fa;
                CK(cudaFuncGetAttributes(&fa, btr_tiled_kernel_ptr<R>(o, own, nthreads, tm)));
                CK(cudaFuncSetAttribute(btr_tiled_kernel_ptr<R>(o, own, nthreads, tm),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        smem_block - (int)fa.sharedSizeBytes));
                static_smem = std::max(static_smem, (int)fa.sharedSizeBytes);
            }
            size_t smem_launch = smem;
            if (tm) {
                // The kernel allocates all 512 columns of its SM's tensor
                // memory, an allocation that would wait for another holder:
                // asking for more than half the SM's shared memory keeps any
                // second such CTA off the SM, so the allocation never waits.
                smem_launch = tile_smem_bytes(plan, m.maxE, m.maxE2, sizeof(R), false);
                const size_t fixed = (size_t)static_smem + 1024, half = (size_t)smem_sm / 2 + 1;
                if (smem_launch + fixed < half) smem_launch = half - fixed;
            }
            int occ = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &occ, btr_tiled_kernel_ptr<R>(3, own, nthreads, tm), nthreads, smem_launch));
            if (occ * nsm < P) {
                if (verbose)
                    fprintf(stderr, "libsse: tile plan k=%d P=%d: occupancy %d x %d SMs\n", k, P,
                            occ, nsm);
                continue;
            }
            if (verbose) {
                int mnc = 0, moe = 0;
                long long tne = 0, tnc = 0;
                for (const TilePatch &t : plan.patches) {
                    mnc = std::max(mnc, t.nc);
                    moe = std::max(moe, t.n_own_e); tne += t.ne; tnc += t.nc;
                }
                fprintf(stderr, "libsse: tiled sub-cycle P=%d threads=%d own=%d smem=%zu tmem=%d "
                        "max(ne,nc,own_e)=(%d,%d,%d) halo overhead edges %.2f cells %.2f\n", P,
                        nthreads, own, smem_launch, (int)tm, mne, mnc, moe,
                        (double)tne / m.E, (double)tnc / m.C);
            }
            return upload_tiles(plan, nthreads, own, smem_launch, tm);
        }
        return SSE_OK;  // no plan fits: the global-memory sub-cycle is used
    }

    // Plan the fused baroclinic stage: patches of Pc consecutive cells of the
    // internal numbering, Pc the largest of a few sizes whose patches fit the
    // kernel's limits and whose shared memory fits a CTA.  Meshes with partial
    // bottom cells, Algorithm 2 or biharmonic viscosity keep the unfused
    // kernels, and so does any mesh no plan fits.
    int plan_bcl(const sse_mesh *mesh, int dev) {
        const char *env = getenv("SSE_BCL_KERNEL");
        if (env && strcmp(env, "unfused") == 0) return SSE_OK;
        if (m.partial || vmix || p.nu_4 > 0.0) return SSE_OK;
        int smem_block = 0, smem_sm = 0;
        CK(cudaDeviceGetAttribute(&smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        // the requested patch size if its plan fits; else the largest patches
        // of which as many CTAs fit an SM as the kernel is built for (two in
        // FP32, one in FP64); else the largest that fit at all
        for (int pass = bcl_cells > 0 ? -1 : 0; pass < 2; pass++)
        for (int Pc : {160, 128, 112, 96, 80, 64, 48, 32}) {
            if (pass == -1 && Pc != bcl_cells) continue;
            std::shared_ptr<const BclPlan> cached;
            {
                sse_mesh *mm = const_cast<sse_mesh *>(mesh);
                std::lock_guard<std::mutex> lk(mm->plan_mu);
                auto it = mm->bcl_plans.find(Pc);
                if (it != mm->bcl_plans.end()) {
                    cached = it->second;
                } else {
                    auto fresh = std::make_shared<BclPlan>();
                    if (!build_bcl_plan(mesh->host, Pc, bcl_max_edges_per_patch(),
                                        bcl_max_cells_per_patch(), *fresh))
                        fresh.reset();
                    mm->bcl_plans[Pc] = fresh;
                    cached = fresh;
                }
            }
            if (!cached) continue;
            const size_t smem = bcl_smem_bytes<R>(*cached, m.L);
            if (smem + 1024 + sizeof(BclJob<R>) + 64 > (size_t)smem_block) continue;
            if (pass <= 0 && (size_t)bcl_blocks_per_sm<R>() * (smem + 1024 + sizeof(BclJob<R>)) >
                                 (size_t)smem_sm)
                continue;
            bcl_pc = Pc;
            // both kernels hold a job descriptor in static shared memory
            CK(cudaFuncSetAttribute(bcl_fused_kernel_ptr<R>(),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem_block - (int)sizeof(BclJob<R>) - 64));
            CK(cudaFuncSetAttribute(bcl_fused_batch_kernel_ptr<R>(),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem_block - (int)sizeof(BclJob<R>) - 64));
            return upload_bcl(*cached, smem);
        }
        return SSE_OK;
    }

    // Plan the fused thickness stage (full columns only): patches of
    // thick_cells_per_patch() consecutive cells, built once per mesh.
    int plan_thick(const sse_mesh *mesh, int dev) {
        const char *env = getenv("SSE_THICK_KERNEL");
        if (env && strcmp(env, "unfused") == 0) return SSE_OK;
        if (m.partial) return SSE_OK;
        std::shared_ptr<const ThickPlan> pl;
        {
            sse_mesh *mm = const_cast<sse_mesh *>(mesh);
            std::lock_guard<std::mutex> lk(mm->plan_mu);
            if (!mm->thick_tried) {
                auto fresh = std::make_shared<ThickPlan>();
                if (!build_thick_plan(mesh->host, thick_cells_per_patch(), *fresh)) fresh.reset();
                mm->thick_plan = fresh;
                mm->thick_tried = true;
            }
            pl = mm->thick_plan;
        }
        if (!pl) return SSE_OK;
        int smem_block = 0;
        CK(cudaDeviceGetAttribute(&smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        DThick t{};
        t.P = pl->P; t.Pc = pl->Pc; t.maxEO = pl->maxEO; t.maxC1 = pl->maxC1;
        if (thick_smem_bytes(t, p.nT, true, true, sizeof(R)) + 1024 + sizeof(ThickJob<R>) + 64 >
            (size_t)smem_block)
            return SSE_OK;
        CK(cudaFuncSetAttribute(thick_fused_kernel_ptr<R>(),
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_block - (int)sizeof(ThickJob<R>) - 64));
        CK(cudaFuncSetAttribute(thick_fused_batch_kernel_ptr<R>(),
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_block - (int)sizeof(ThickJob<R>) - 64));
        t.cnt = A.upload(pl->cnt);
        t.off_eo = A.upload(pl->off_eo); t.off_c1 = A.upload(pl->off_c1);
        t.eogid = A.upload(pl->eogid); t.c1gid = A.upload(pl->c1gid);
        t.o_e = A.upload(pl->o_e); t.o_o = A.upload(pl->o_o);
        uA_e = A.alloc<R>(m.Ep);
        if (A.failed) return SSE_ERR_OOM;
        thk = t;
        fused_th = true;
        return SSE_OK;
    }

    int upload_bcl(const BclPlan &pl, size_t smem) {
        auto toR = [](const std::vector<double> &x) { return std::vector<R>(x.begin(), x.end()); };
        DBcl<R> &t = bcl;
        t.P = pl.P; t.maxE0 = pl.maxE0; t.maxE1 = pl.maxE1; t.maxE2 = pl.maxE2; t.maxC1 = pl.maxC1;
        t.maxC2 = pl.maxC2; t.maxV = pl.maxV; t.smem = smem;
        t.cnt = A.upload(pl.cnt);
        t.off_e0 = A.upload(pl.off_e0); t.off_v = A.upload(pl.off_v);
        t.e0_eoe = A.upload(pl.e0_eoe);
        t.e0_cfc = A.upload(toR(pl.e0_cfc)); t.e0_c12 = A.upload(pl.e0_c12);
        t.e0_v12 = A.upload(pl.e0_v12); t.e0_invdc = A.upload(toR(pl.e0_invdc));
        t.e0_invdv = A.upload(toR(pl.e0_invdv));
        t.v_f = A.upload(toR(pl.v_f));
        std::vector<unsigned char> img;
        std::vector<long long> img_off;
        t.img_max = bcl_build_image<R>(pl, img, img_off);
        t.img = A.upload(img); t.img_off = A.upload(img_off);
        Fc = A.alloc<R>(m.Ep);
        if (A.failed) return SSE_ERR_OOM;
        fused = true;
        return SSE_OK;
    }

    int upload_tiles(const TilePlan &plan, int nthreads, int own, size_t smem, bool tm) {
        const unsigned int sR = sizeof(R);
        std::vector<int> noc, noe, nie, cg, eg, c12, nel, ncl;
        std::vector<unsigned short> eo, ce;
        std::vector<R> cf, dv, Hh;
        for (const TilePatch &t : plan.patches) {
            noc.push_back(t.n_own_c); noe.push_back(t.n_own_e); nie.push_back(t.n_int_e);
            // sub-stage s of a sub-step needs edges of ring <= K - s and cells of
            // ring <= K - 1 - s (K = 3): the later sub-stages skip the outer rings
            for (int r = 2; r >= 0; r--) { nel.push_back(t.ne_ring[r]); ncl.push_back(t.nc_ring[r]); }
            cg.insert(cg.end(), t.cell_gid.begin(), t.cell_gid.end());
            eg.insert(eg.end(), t.edge_gid.begin(), t.edge_gid.end());
            for (int32_t x : t.c12) {
                const unsigned int a = (unsigned int)x & 0xffffu, b = (unsigned int)x >> 16;
                c12.push_back((int)((a * sR) | ((b * sR) << 16)));
            }
            // connectivity per entry (rows, copied to shared memory); coefficients
            // term-major within the patch ([j][ne], [j][nc]) so that a warp's
            // load of term j of 32 consecutive entries is one contiguous segment
            const size_t cf0 = cf.size(), dv0 = dv.size();
            cf.resize(cf0 + (size_t)t.ne * TILE_CFR, R(0));
            dv.resize(dv0 + (size_t)t.nc * TILE_NCEP, R(0));
            for (int k = 0; k < t.ne; k++) {
                for (int j = 0; j < TILE_NE2P; j++) {
                    const bool on = j < t.n2[k];
                    const int le = on ? t.eoe[(size_t)k * m.maxE2 + j] : t.ne;
                    eo.push_back((unsigned short)(le * sR));
                    if (on) cf[cf0 + (size_t)j * t.ne + k] = (R)t.cfc[(size_t)k * m.maxE2 + j];
                }
                cf[cf0 + (size_t)TILE_NE2P * t.ne + k] = (R)t.invdc[k];
            }
            for (int k = 0; k < t.nc; k++)
                for (int j = 0; j < TILE_NCEP; j++) {
                    const bool on = j < t.nce[k];
                    const int le = on ? t.ce[(size_t)k * m.maxE + j] : t.ne;
                    ce.push_back((unsigned short)(le * sR));
                    if (on) dv[dv0 + (size_t)j * t.nc + k] = (R)t.divc[(size_t)k * m.maxE + j];
                }
            for (double x : t.H) Hh.push_back((R)x);
        }
        DTiles<R> &t = tiles;
        t.P = plan.P; t.nthreads = nthreads; t.own = own; t.smem = smem; t.tm = tm ? 1 : 0;
        t.cell_off = A.upload(plan.cell_off); t.edge_off = A.upload(plan.edge_off);
        t.n_own_c = A.upload(noc); t.n_own_e = A.upload(noe); t.n_int_e = A.upload(nie);
        t.ne_lim = A.upload(nel); t.nc_lim = A.upload(ncl);
        t.cell_gid = A.upload(cg); t.edge_gid = A.upload(eg); t.c12 = A.upload(c12);
        t.eoe = A.upload(eo); t.cfc = A.upload(cf);
        t.ce = A.upload(ce); t.divc = A.upload(dv); t.H = A.upload(Hh);
        for (int b = 0; b < 2; b++) {
            t.xu[b] = A.alloc<R>(m.Ep);
            t.xz[b] = A.alloc<R>(m.Cp);
        }
        if (A.failed) return SSE_ERR_OOM;
        tiled = true;
        return SSE_OK;
    }

    int init(const sse_mesh *mesh, const sse_params *prm, cudaStream_t st,
             bool count_only = false) {
        m = mesh->dm;
        s = st;
        ps = st;
        A.async = true;
        A.stream = st;
        A.count_only = count_only;
        mixed = (prm->precision == SSE_MIXED);
        recon = prm->recon;
        vmix = (prm->options & SSE_OPT_VMIX) != 0;
        p.g = prm->g; p.rho0 = prm->rho0; p.nu_h = prm->nu_h; p.nu_v = prm->nu_v;
        p.kappa_h = prm->kappa_h; p.kappa_v = prm->kappa_v; p.c_drag = prm->c_drag;
        p.nu_4 = prm->nu_4;
        // The FP32 tracers of the mixed form are held as anomalies from the
        // EOS reference values (full columns): the density anomaly depends on
        // differences of T and S between neighbouring columns that are 1e-3 to
        // 1e-4 of S itself, which an FP32 S of about 35 does not resolve.
        // Transport, mixing and the stage combinations are linear in the
        // tracer and conserve it with the same mass fluxes, so the anomaly
        // obeys the same equations; the kernels' EOS references become the
        // remainder (zero).
        toff[0] = toff[1] = 0.0;
        if (mixed && !m.partial) {
            toff[0] = prm->eos_T_ref;
            toff[1] = prm->eos_S_ref;
        }
        p.alpha = prm->eos_alpha; p.beta = prm->eos_beta; p.T_ref = prm->eos_T_ref - toff[0];
        p.S_ref = prm->eos_S_ref - toff[1];
        p.zcoef = prm->g * (1.0 - prm->eos_rho_ref / prm->rho0);
        p.nT = prm->nTracers; p.recon = prm->recon; p.wind = nullptr; p.wind_f = nullptr;
        fill_phys(p.pd);
        fill_phys(p.pf);
        const size_t EL = (size_t)m.L * m.Ep, CL = (size_t)m.L * m.Cp, VL = (size_t)m.L * m.Vp;
        const int nT = p.nT;
        ubar_n = A.alloc<R>(m.Ep); ut_n = A.alloc<R>(EL);
        h_n = A.alloc<double>(CL); zeta_n = A.alloc<double>(m.Cp);
        tr_n = A.alloc<R>(nT * CL);
        ut_1 = A.alloc<R>(EL); ut_c = A.alloc<R>(EL); ut_3 = A.alloc<R>(EL);
        ubar_1 = A.alloc<R>(m.Ep); ubar_h = A.alloc<R>(m.Ep); ubar_np1 = A.alloc<R>(m.Ep);
        G0 = A.alloc<R>(m.Ep); G1 = A.alloc<R>(m.Ep); G2 = A.alloc<R>(m.Ep); Gw = A.alloc<R>(m.Ep);
        Fz1 = A.alloc<double>(m.Ep); Fz2 = A.alloc<double>(m.Ep); Fz3 = A.alloc<double>(m.Ep);
        S1 = A.alloc<double>(m.Ep); S2 = A.alloc<double>(m.Ep);
        zeta_sub = A.alloc<double>(m.Cp);
        last_Fz = Fz1;
        h_1 = A.alloc<double>(CL); h_h = A.alloc<double>(CL);
        zeta_1 = A.alloc<double>(m.Cp); zeta_h = A.alloc<double>(m.Cp);
        if (mixed) {
            hR_n = A.alloc<R>(CL); hR_1 = A.alloc<R>(CL); hR_h = A.alloc<R>(CL);
        } else {
            hR_n = (R *)h_n; hR_1 = (R *)h_1; hR_h = (R *)h_h;
        }
        tr_1 = A.alloc<R>(nT * CL); tr_h = A.alloc<R>(nT * CL);
        flux = A.alloc<R>(EL);
        Fcol = A.alloc<double>(m.Ep);
        db.delta = A.alloc<R>(CL); db.w = A.alloc<R>(CL); db.cq = A.alloc<V4<R>>(CL);
        db.omega = A.alloc<R>(VL); db.q = A.alloc<R>(VL);
        db.hq = A.alloc<V2<R>>(EL);
        db.del2 = db.delta2 = db.omega2 = nullptr;
        if (p.nu_4 > 0.0) {
            db.del2 = A.alloc<R>(EL); db.delta2 = A.alloc<R>(CL); db.omega2 = A.alloc<R>(VL);
        }
        bu0 = A.alloc<R>(m.Ep); bua = A.alloc<R>(m.Ep); buh = A.alloc<R>(m.Ep);
        bz0 = A.alloc<R>(m.Cp); bza = A.alloc<R>(m.Cp); bzh = A.alloc<R>(m.Cp);
        barwords = A.alloc<unsigned int>(2);
        barerr = A.alloc<int>(1);
        stage = A.alloc<double>((size_t)std::max(m.Ep, m.Cp) * m.L);
        wind = A.alloc<double>(m.Ep);
        wind_d = A.alloc<double>(m.Ep);
        wind_f = A.alloc<float>(m.Ep);
        dparts = 256;
        dpart = A.alloc<double>((size_t)dparts * 9);
        dout = A.alloc<double>(9);
        if (A.failed) return SSE_ERR_OOM;
        // persistent sub-cycle grid: all co-resident blocks, no more than needed
        int dev = 0, nsm = 0, occ = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int bt = btr_block_size<R>();
        int occ2 = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, btr_kernel_ptr<R>(2, m.maxE2), bt, 0));
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, btr_kernel_ptr<R>(3, m.maxE2), bt, 0));
        occ = std::min(occ, occ2);
        if (occ < 1) return SSE_ERR_UNSUPPORTED;
        const int need = (std::max(m.E, m.C) + bt - 1) / bt;
        btr_blocks = std::max(1, std::min(need, occ * nsm));
        // every thread keeps at most btr_max_items_per_thread() edges in registers
        if ((long long)btr_blocks * bt * btr_max_items_per_thread() < std::max(m.E, m.C))
            return SSE_ERR_UNSUPPORTED;
        int rc = plan_tiles(mesh, dev, nsm);
        if (rc) return rc;
        rc = plan_bcl(mesh, dev);
        if (rc) return rc;
        rc = plan_thick(mesh, dev);
        if (rc) return rc;
        CK(cudaStreamSynchronize(s));
        return SSE_OK;
    }

    Barrier bar() const { return Barrier{barwords, barwords + 1, barerr}; }

    template <class T> void fill_phys(PhysR<T> &q) const {
        q.g = (T)p.g; q.inv_rho0 = (T)(1.0 / p.rho0); q.nu_h = (T)p.nu_h; q.nu_v = (T)p.nu_v;
        q.kappa_h = (T)p.kappa_h; q.kappa_v = (T)p.kappa_v; q.c_drag = (T)p.c_drag;
        q.nu_4 = (T)p.nu_4;
        q.alpha = (T)p.alpha; q.beta = (T)p.beta; q.T_ref = (T)p.T_ref; q.S_ref = (T)p.S_ref;
        q.zcoef = (T)p.zcoef;
    }

    int check_launch() {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            fprintf(stderr, "libsse: launch failed: %s\n", cudaGetErrorString(e));
            return SSE_ERR_CUDA;
        }
        return SSE_OK;
    }

    // ---- host <-> device
    int set(int field, const double *host) override { return set_t<double>(field, host); }
    int get(int field, double *host) override { return get_t<double>(field, host); }
    int set_f32(int field, const float *host) override { return set_t<float>(field, host); }
    int get_f32(int field, float *host) override { return get_t<float>(field, host); }
    int transfer(int field, void *host, int flags) override {
        const bool get = flags & SSE_XFER_GET, sync = !(flags & SSE_XFER_ASYNC);
        if (flags & SSE_XFER_F32)
            return get ? get_t<float>(field, (float *)host, sync)
                       : set_t<float>(field, (const float *)host, sync);
        return get ? get_t<double>(field, (double *)host, sync)
                   : set_t<double>(field, (const double *)host, sync);
    }
    int sync() override {
        CK(cudaStreamSynchronize(s));
        return barrier_status();
    }

    // Host transfers in precision H: FP64 for every field; FP32 for the fields
    // held in the tendency precision (u, utilde, ubar, G, tracers).
    template <class H> int set_t(int field, const H *host, bool sync = true) {
        constexpr bool f64 = std::is_same<H, double>::value;
        const int L = m.L;
        // page-locked host buffers are read by the conversion kernels directly
        const H *direct = (const H *)host_alias(host);
        const H *in = direct ? direct : (const H *)stage;
        switch (field) {
        case SSE_FIELD_U:
        case SSE_FIELD_UTILDE:
            if (!direct) CK(cudaMemcpyAsync(stage, host, sizeof(H) * m.E * L, cudaMemcpyHostToDevice, s));
            launch_to_device<R>(in, ut_n, m.E, L, m.Ep, m.eperm, s);
            if (m.partial) launch_mask_layers<R>(ut_n, m.E, L, m.Ep, m.ke, s);
            if (field == SSE_FIELD_U) CK(cudaMemsetAsync(ubar_n, 0, sizeof(R) * m.Ep, s));
            break;
        case SSE_FIELD_UBAR:
        case SSE_FIELD_G:
            if (!direct) CK(cudaMemcpyAsync(stage, host, sizeof(H) * m.E, cudaMemcpyHostToDevice, s));
            launch_to_device<R>(in, field == SSE_FIELD_UBAR ? ubar_n : G0, m.E, 1, m.Ep, m.eperm, s);
            break;
        case SSE_FIELD_H:
            if constexpr (f64) {
                if (!direct)
                    CK(cudaMemcpyAsync(stage, host, sizeof(double) * m.C * L,
                                       cudaMemcpyHostToDevice, s));
                launch_to_device<double>(in, h_n, m.C, L, m.Cp, m.cperm, s);
                if (m.partial) launch_mask_layers<double>(h_n, m.C, L, m.Cp, m.kc, s);
                if (mixed) launch_h_to_float(h_n, (float *)hR_n, L * m.Cp, s);
                launch_ssh(m, h_n, zeta_n, s);
                break;
            } else {
                return SSE_ERR_INVALID_ARG;   // h is FP64 state in both forms
            }
        case SSE_FIELD_TRACER0:
        case SSE_FIELD_TRACER1: {
            const int t = field - SSE_FIELD_TRACER0;
            if (t >= p.nT) return SSE_ERR_INVALID_ARG;
            if (!direct) CK(cudaMemcpyAsync(stage, host, sizeof(H) * m.C * L, cudaMemcpyHostToDevice, s));
            launch_to_device<R>(in, tr_n + (size_t)t * L * m.Cp, m.C, L, m.Cp, m.cperm, s, toff[t]);
            if (m.partial) launch_mask_layers<R>(tr_n + (size_t)t * L * m.Cp, m.C, L, m.Cp, m.kc, s);
            break;
        }
        case SSE_FIELD_WIND:
            if constexpr (f64) {
                CK(cudaMemcpyAsync(wind, host, sizeof(double) * m.E, cudaMemcpyHostToDevice, s));
                launch_scale(wind, 1.0 / p.rho0, wind_d, wind_f, m.E, m.eperm, s);
                p.wind = wind_d;
                p.wind_f = wind_f;
                graphs_clear();   // the step's kernel arguments changed
                break;
            } else {
                return SSE_ERR_INVALID_ARG;
            }
        default:
            return SSE_ERR_INVALID_ARG;
        }
        CK(cudaMemsetAsync(barerr, 0, sizeof(int), s));
        steps = 0;
        int rc = check_launch();
        if (rc) return rc;
        if (sync) CK(cudaStreamSynchronize(s));
        return SSE_OK;
    }

    template <class H> int get_t(int field, H *host, bool sync = true) {
        constexpr bool f64 = std::is_same<H, double>::value;
        const int L = m.L;
        size_t n = 0;
        // the conversion kernels write page-locked host buffers directly
        H *direct = (H *)host_alias(host);
        H *out = direct ? direct : (H *)stage;
        if (!f64 && (field == SSE_FIELD_H || field == SSE_FIELD_ZETA ||
                     field == SSE_FIELD_ZETA_SUB || field == SSE_FIELD_FZETA ||
                     field == SSE_FIELD_WIND))
            return SSE_ERR_INVALID_ARG;   // FP64 state in both forms
        switch (field) {
        case SSE_FIELD_U:
            launch_add_bar<R>(ubar_n, ut_n, out, m.E, L, m.Ep, m.partial ? m.ke : nullptr, m.eperm, s);
            n = (size_t)m.E * L;
            break;
        case SSE_FIELD_UTILDE:
            launch_from_device<R>(ut_n, out, m.E, L, m.Ep, m.eperm, s);
            n = (size_t)m.E * L;
            break;
        case SSE_FIELD_UBAR:
        case SSE_FIELD_G:
            launch_from_device<R>(field == SSE_FIELD_UBAR ? ubar_n : G0, out, m.E, 1, m.Ep, m.eperm, s);
            n = m.E;
            break;
        case SSE_FIELD_H:
            if constexpr (f64) launch_from_device<double>(h_n, out, m.C, L, m.Cp, m.cperm, s);
            n = (size_t)m.C * L;
            break;
        case SSE_FIELD_TRACER0:
        case SSE_FIELD_TRACER1: {
            const int t = field - SSE_FIELD_TRACER0;
            if (t >= p.nT) return SSE_ERR_INVALID_ARG;
            launch_from_device<R>(tr_n + (size_t)t * L * m.Cp, out, m.C, L, m.Cp, m.cperm, s,
                                  toff[t]);
            n = (size_t)m.C * L;
            break;
        }
        case SSE_FIELD_ZETA:
            if constexpr (f64) launch_from_device<double>(zeta_n, out, m.C, 1, m.Cp, m.cperm, s);
            n = m.C;
            break;
        case SSE_FIELD_ZETA_SUB:
            if constexpr (f64) launch_from_device<double>(zeta_sub, out, m.C, 1, m.Cp, m.cperm, s);
            n = m.C;
            break;
        case SSE_FIELD_FZETA:
            if constexpr (f64) launch_from_device<double>(last_Fz, out, m.E, 1, m.Ep, m.eperm, s);
            n = m.E;
            break;
        case SSE_FIELD_WIND:
            if constexpr (f64) CK(cudaMemcpyAsync(out, wind, sizeof(double) * m.E, cudaMemcpyDefault, s));
            n = m.E;
            break;
        default:
            return SSE_ERR_INVALID_ARG;
        }
        int rc = check_launch();
        if (rc) return rc;
        if (!direct) CK(cudaMemcpyAsync(host, stage, sizeof(H) * n, cudaMemcpyDeviceToHost, s));
        if (!sync) return SSE_OK;
        CK(cudaStreamSynchronize(s));
        return barrier_status();
    }

    int barrier_status() {
        int err = 0;
        CK(cudaMemcpyAsync(&err, barerr, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return err ? SSE_ERR_SYNC_TIMEOUT : SSE_OK;
    }

    // ---- pieces
    void bcl_stage(R *ubar, R *ut, R *hR, R *tr, const double *zeta, bool split, const R *utn,
                   double a, double b, double dt, R *out, R *G) {
        if (fused && rec) {
            LaunchRec<R> r1;
            r1.cls = REC_COLFLUX;
            r1.u.cf = ColfluxJob<R>{m, ubar, ut, hR, Fc, split ? 1 : 0, 0};
            rec->push_back(r1);
            LaunchRec<R> r2;
            r2.cls = REC_BCL;
            r2.smem = bcl.smem;
            BclArgs<R> x{};
            x.ubar = ubar; x.ut = ut; x.hR = hR; x.tr = tr; x.zeta = zeta; x.Fc = Fc;
            x.ut_n = utn; x.a = (R)a; x.b = (R)b; x.dt = (R)dt; x.ut_out = out; x.G = G;
            r2.u.bcl = BclJob<R>{m, p, bcl, x};
            rec->push_back(r2);
            return;
        }
        if (fused) {
            // the column pre-pass (and the split at stage 1) counts as the edge
            // pre-pass class, the fused kernel as the baroclinic-edge class
            pbeg(SSE_K_EDGE_PRE);
            launch_colflux<R>(m, ubar, ut, hR, split, Fc, s);
            pend();
            BclArgs<R> x{};
            x.ubar = ubar; x.ut = ut; x.hR = hR; x.tr = tr; x.zeta = zeta; x.Fc = Fc;
            x.ut_n = utn; x.a = (R)a; x.b = (R)b; x.dt = (R)dt; x.ut_out = out; x.G = G;
            pbeg(SSE_K_BCL_EDGE);
            launch_bcl_fused<R>(bcl, m, p, x, s);
            pend();
            return;
        }
        pbeg(SSE_K_CELL_DIAG);
        launch_cell_diag<R>(m, p, ubar, ut, hR, tr, db, s);
        pend();
        pbeg(SSE_K_VERTEX);
        launch_vertex<R>(m, ubar, ut, hR, db, s);
        pend();
        pbeg(SSE_K_EDGE_PRE);
        launch_edge_pre<R>(m, ubar, ut, hR, db, split, s);
        pend();
        if (db.del2) {
            pbeg(SSE_K_DEL4);
            launch_del2_divcurl<R>(m, db, s);
            pend();
        }
        pbeg(SSE_K_BCL_EDGE);
        // Algorithm 2 keeps its modified super-diagonal in `flux`, which is
        // free until the stage's transport kernel writes it
        launch_bcl_edge<R>(m, p, ubar, ut, hR, zeta, db, utn, a, b, dt, out, G,
                           vmix ? flux : nullptr, s);
        pend();
    }

    cudaError_t btr(int order, const R *ub_start, const double *z_start, const R *Ga,
                    double tau_dt, int M, const R *X, double al, double be, R *ub_out,
                    double *Fz, double *z_out) {
        BtrArgs<R> a{};
        a.ub_start = ub_start; a.z_start = z_start; a.G = Ga; a.X = X; a.alpha = al;
        a.beta = be; a.ub_out = ub_out; a.Fz = Fz; a.z_out = z_out;
        a.u0 = bu0; a.ua = bua; a.uh = buh; a.z0 = bz0; a.za = bza; a.zh = bzh;
        a.tau = tau_dt / M; a.g = p.g; a.M = M; a.order = order; a.stall = inject_stall;
        last_Fz = Fz;
        if (rec) {
            LaunchRec<R> r;
            r.cls = REC_BTR;
            r.u.btr = a;
            rec->push_back(r);
            return cudaSuccess;
        }
        return issue_btr(a);
    }
    // the sub-cycle's launch on the state's own stream
    cudaError_t issue_btr(const BtrArgs<R> &a) {
        // the barrier reset (a memset) sits outside the timed pair
        cudaError_t me = cudaMemsetAsync(barwords, 0, 2 * sizeof(unsigned int), s);
        if (me != cudaSuccess) return me;
        pbeg(SSE_K_BTR);
        cudaError_t e = tiled ? launch_btr_tiled<R>(tiles, a, bar(), s)
                              : launch_btr<R>(m, a, bar(), btr_blocks, btr_block_size<R>(), s);
        pend();
        return e;
    }

    void transport(const R *hR, const double *zeta, const R *ubA, const R *utA, double wA,
                   const R *ubB, const R *utB, double wB, const double *Fz, const double *e1,
                   const double *e2, double cF, double cE, double cA, double *S_out) {
        TransportArgs<R> a{};
        a.hR = hR; a.zeta = zeta; a.Fcol = Fcol; a.ubA = ubA; a.utA = utA; a.ubB = ubB; a.utB = utB; a.wA = wA; a.wB = wB;
        a.Fz = Fz; a.ex1 = e1; a.ex2 = e2; a.cF = cF; a.cE = cE; a.cA = cA;
        a.recon = (recon != SSE_RECON_OFF); a.S_out = S_out; a.flux = flux;
        if (fused_th && rec) {
            LaunchRec<R> r;
            r.cls = REC_TRANSPORT;
            r.u.tr = TransportJob<R>{m, a, uA_e};
            rec->push_back(r);
            last_ta = a;
            return;
        }
        pbeg(SSE_K_TRANSPORT);
        if (fused_th) {
            // columns only; the thickness kernel forms the per-layer flux itself
            launch_transport_cols<R>(m, a, uA_e, s);
            last_ta = a;
        } else {
            launch_transport<R>(m, a, s);
        }
        pend();
    }

    void thickness(const double *h_s, const R *hR_s, const R *tr_s, double a, double b, double dt,
                   double *h_out, R *hR_out, R *tr_out, double *zeta_out) {
        ThickArgs<R> t{};
        t.flux = flux; t.Fcol = Fcol; t.h_s = h_s; t.hR_s = hR_s; t.tr_s = tr_s; t.h_n = h_n;
        t.hR_n = hR_n; t.tr_n = tr_n;
        t.a = a; t.b = b; t.dt = dt; t.h_out = h_out; t.hR_out = mixed ? hR_out : nullptr;
        t.tr_out = tr_out; t.zeta_out = zeta_out;
        pbeg(SSE_K_THICKNESS);
        if (fused_th) {
            ThickFArgs<R> f{};
            f.ubA = last_ta.ubA; f.utA = last_ta.utA; f.ubB = last_ta.ubB; f.utB = last_ta.utB;
            f.wA = last_ta.wA; f.wB = last_ta.wB; f.uA = uA_e; f.Fcol = Fcol;
            f.h_s = h_s; f.hR_s = hR_s; f.tr_s = tr_s; f.h_n = h_n; f.hR_n = hR_n; f.tr_n = tr_n;
            f.a = a; f.b = b; f.dt = dt; f.h_out = h_out; f.hR_out = t.hR_out; f.tr_out = tr_out;
            f.zeta_out = zeta_out;
            const size_t smem = thick_smem_bytes(thk, p.nT, f.utB != nullptr, a != 0.0, sizeof(R));
            if (rec) {
                pend();
                LaunchRec<R> r;
                r.cls = REC_THICK;
                r.smem = smem;
                r.u.th = ThickJob<R>{m, p, thk, f};
                rec->push_back(r);
                return;
            }
            launch_thick_fused<R>(thk, m, p, f, smem, s);
        } else {
            launch_thickness<R>(m, p, t, s);
        }
        pend();
    }

    // combined forcing for the corrector: Gw = w0 G0 + w1 G1 (+ w2 G2)
    void combine_G(double w0, double w1, double w2);

    int step(int order, double dt, int M) override {
        const bool consistent = (recon == SSE_RECON_CONSISTENT);
        if (order == 2) {
            // Stage 1 (Sec. 3.2): Algorithm 1, predictor sub-cycle, thickness
            bcl_stage(ubar_n, ut_n, hR_n, tr_n, zeta_n, true, nullptr, 0.0, 1.0, dt, ut_1, G0);
            CK(btr(2, ubar_n, zeta_n, G0, dt, M, nullptr, 0, 1, ubar_1, Fz1, nullptr));
            transport(hR_n, zeta_n, ubar_n, ut_n, 1.0, nullptr, nullptr, 0.0, Fz1, nullptr,
                      nullptr, 1.0, 0.0, 1.0, S1);
            thickness(h_n, hR_n, tr_n, 0.0, 1.0, dt, h_1, hR_1, tr_1, zeta_1);
            // Stage 2: baroclinic, utilde^{n+1} = (ut^n + ut^{n+2})/2
            bcl_stage(ubar_1, ut_1, hR_1, tr_1, zeta_1, false, ut_n, 0.5, 0.5, dt, ut_c, G1);
            // Step 2: corrector with Interp_2(G0, G1)
            combine_G(0.5, 0.5, 0.0);
            CK(btr(2, ubar_n, zeta_n, Gw, dt, M, nullptr, 0, 1, ubar_np1, Fz2, zeta_sub));
            // Step 3: thickness stage 2 with F^h_2 and the factor 2 of Sec. 3.4
            transport(hR_1, zeta_1, ubar_np1, ut_c, 1.0, nullptr, nullptr, 0.0, Fz2,
                      consistent ? Fz1 : S1, nullptr, 0.5, 0.5, 2.0, nullptr);
            thickness(h_1, hR_1, tr_1, 0.5, 0.5, dt, h_n, hR_n, tr_n, zeta_n);
        } else {
            // Stage 1 (Sec. 3.3)
            bcl_stage(ubar_n, ut_n, hR_n, tr_n, zeta_n, true, nullptr, 0.0, 1.0, dt, ut_1, G0);
            CK(btr(3, ubar_n, zeta_n, G0, dt, M, nullptr, 0, 1, ubar_1, Fz1, nullptr));
            transport(hR_n, zeta_n, ubar_n, ut_n, 1.0, nullptr, nullptr, 0.0, Fz1, nullptr,
                      nullptr, 1.0, 0.0, 1.0, S1);
            thickness(h_n, hR_n, tr_n, 0.0, 1.0, dt, h_1, hR_1, tr_1, zeta_1);
            // Stage 2
            bcl_stage(ubar_1, ut_1, hR_1, tr_1, zeta_1, false, ut_n, 0.75, 0.25, dt, ut_c, G1);
            CK(btr(3, ubar_1, zeta_1, G1, dt, M, ubar_n, 0.75, 0.25, ubar_h, Fz2, nullptr));
            transport(hR_1, zeta_1, ubar_1, ut_1, 1.0, nullptr, nullptr, 0.0, Fz2, nullptr,
                      nullptr, 1.0, 0.0, 1.0, S2);
            thickness(h_1, hR_1, tr_1, 0.75, 0.25, dt, h_h, hR_h, tr_h, zeta_h);
            // Stage 3
            bcl_stage(ubar_h, ut_c, hR_h, tr_h, zeta_h, false, ut_n, 1.0 / 3.0, 2.0 / 3.0, dt,
                      ut_3, G2);
            // Step 2: corrector with Interp_3(G0, G1, G_{1/2})
            combine_G(1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0);
            CK(btr(3, ubar_n, zeta_n, Gw, dt, M, nullptr, 0, 1, ubar_np1, Fz3, zeta_sub));
            // Step 3: F^h_3 of Sec. 3.4 and the factor 3/2
            transport(hR_h, zeta_h, ubar_n, ut_n, 0.5, ubar_np1, ut_3, 0.5, Fz3,
                      consistent ? Fz1 : S1, consistent ? Fz2 : S2, 2.0 / 3.0, 1.0 / 6.0, 1.5,
                      nullptr);
            thickness(h_h, hR_h, tr_h, 1.0 / 3.0, 2.0 / 3.0, dt, h_n, hR_n, tr_n, zeta_n);
        }
        advance(order);
        return check_launch();
    }

    // The host side of the end of a step: the new levels become level n.
    void advance(int order) {
        std::swap(ut_n, order == 2 ? ut_c : ut_3);
        std::swap(ubar_n, ubar_np1);
        steps++;
    }

    // ---- CUDA graphs of two large steps (sse_step with n_steps >= 2): the
    // launches of step() twice, captured once per (order, dt, M) and buffer
    // assignment (two steps bring the rotating buffers back), then replayed
    // with one cudaGraphLaunch.  Not used while profiling or with the barrier
    // stall hook on; given up for good if a capture fails (the legacy default
    // stream cannot be captured), in which case the steps run launch by launch.
    struct StepGraph {
        int order, M;
        double dt;
        const void *key[5];
        cudaGraphExec_t exec;
    };
    std::vector<StepGraph> graphs;
    bool graphs_ok = true;
    void graphs_clear() {
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
    }
    ~Engine() override { graphs_clear(); }
    int graph_count() const override { return (int)graphs.size(); }

    int step2(int order, double dt, int M) override {
        if (!graphs_ok || prof || inject_stall) {
            int rc = step(order, dt, M);
            return rc ? rc : step(order, dt, M);
        }
        const void *key[5] = {ut_n, ut_c, ut_3, ubar_n, ubar_np1};
        for (auto &g : graphs)
            if (g.order == order && g.dt == dt && g.M == M &&
                std::equal(key, key + 5, g.key)) {
                CK(cudaGraphLaunch(g.exec, s));
                advance(order);
                advance(order);
                return check_launch();
            }
        R *k_ut_n = ut_n, *k_ut_c = ut_c, *k_ut_3 = ut_3, *k_ub = ubar_n, *k_ubp = ubar_np1;
        const long long steps0 = steps;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            graphs_ok = false;
            return step2(order, dt, M);
        }
        int rc = step(order, dt, M);
        if (!rc) rc = step(order, dt, M);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        cudaGraphExec_t x = nullptr;
        if (!rc && e == cudaSuccess && g) e = cudaGraphInstantiate(&x, g, 0);
        if (g) cudaGraphDestroy(g);
        // capturing ran the host side of the two steps: undo it; the launch redoes it
        ut_n = k_ut_n; ut_c = k_ut_c; ut_3 = k_ut_3; ubar_n = k_ub; ubar_np1 = k_ubp;
        steps = steps0;
        if (rc || e != cudaSuccess || !x) {
            if (x) cudaGraphExecDestroy(x);
            cudaGetLastError();
            graphs_ok = false;
            return step2(order, dt, M);
        }
        if (graphs.size() >= 8) graphs_clear();
        StepGraph sg{order, M, dt, {}, x};
        std::copy(key, key + 5, sg.key);
        graphs.push_back(sg);
        CK(cudaGraphLaunch(x, s));
        advance(order);
        advance(order);
        return check_launch();
    }

    int bcl_feuler(double dt) override {
        launch_ssh(m, h_n, zeta_n, s);
        bcl_stage(ubar_n, ut_n, hR_n, tr_n, zeta_n, false, nullptr, 0.0, 1.0, dt, ut_1, G0);
        CK(cudaMemcpyAsync(ut_n, ut_1, sizeof(R) * m.L * m.Ep, cudaMemcpyDeviceToDevice, s));
        return check_launch();
    }

    int patches() const override { return tiled ? tiles.P : 0; }
    int patch_threads() const override { return tiled ? tiles.nthreads : 0; }
    int patch_tmem() const override { return tiled ? tiles.tm : 0; }
    bool has_del4() const override { return db.del2 != nullptr; }
    bool fused_bcl() const override { return fused; }

    int btr_substep(int order, double dt, int M) override {
        launch_ssh(m, h_n, zeta_n, s);
        CK(btr(order, ubar_n, zeta_n, G0, dt, M, nullptr, 0, 1, ubar_1, Fz1, zeta_sub));
        CK(cudaMemcpyAsync(ubar_n, ubar_1, sizeof(R) * m.Ep, cudaMemcpyDeviceToDevice, s));
        return check_launch();
    }

    int diagnostics(sse_diag *out) override {
        launch_diag<R>(m, ubar_n, ut_n, h_n, tr_n, p.nT, toff, zeta_n, dpart, dparts, dout, s);
        int rc = check_launch();
        if (rc) return rc;
        double v[9];
        CK(cudaMemcpyAsync(v, dout, sizeof(v), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        memset(out, 0, sizeof(*out));
        out->volume = v[0];
        out->tracer_content[0] = v[1];
        out->tracer_content[1] = v[2];
        out->kinetic_energy = v[3];
        out->max_speed = v[4];
        out->min_thickness = v[5];
        out->zeta_min = v[6];
        out->zeta_max = v[7];
        out->nonfinite = v[8] != 0.0;
        out->step = steps;
        rc = barrier_status();
        if (rc) return rc;
        return out->nonfinite ? SSE_ERR_NONFINITE : SSE_OK;
    }
};

// the Interp forcing of the corrector, Gw = w0 G0 + w1 G1 + w2 G2; the single
// and the batched kernel run the same per-edge function on a shared-memory
// copy of their descriptor (the same bits alone or in a batch)
template <class R> __device__ __forceinline__ void combine_edge(const CombineJob<R> &J, int e) {
    if (e >= J.n) return;
    J.out[e] = (R)(J.wa * (double)J.a[e] + J.wb * (double)J.b[e] + J.wc * (double)J.c[e]);
}
template <class R> __global__ void k_combine_G(const CombineJob<R> job) {
    __shared__ CombineJob<R> J;
    if (threadIdx.x == 0) J = job;
    __syncthreads();
    combine_edge<R>(J, blockIdx.x * blockDim.x + threadIdx.x);
}

template <class R> void Engine<R>::combine_G(double w0, double w1, double w2) {
    if (rec) {
        LaunchRec<R> r;
        r.cls = REC_COMBINE;
        r.u.cmb = CombineJob<R>{G0, G1, G2, Gw, w0, w1, w2, m.E, 0};
        rec->push_back(r);
        return;
    }
    pbeg(SSE_K_COMBINE);
    k_combine_G<R><<<(m.E + 255) / 256, 256, 0, s>>>(CombineJob<R>{G0, G1, G2, Gw, w0, w1, w2,
                                                                   m.E, 0});
    pend();
}

struct sse_state {
    std::unique_ptr<EngineBase> eng;
    int device = 0;
};

static bool params_ok(const sse_params *prm) {
    return !((prm->precision != SSE_FP64 && prm->precision != SSE_MIXED) || prm->recon < 0 ||
             prm->recon > 2 || prm->nTracers < 1 || prm->nTracers > 2 ||
             (prm->options & ~SSE_OPT_VMIX) != 0 || !(prm->g > 0) || !(prm->rho0 > 0) ||
             !(prm->nu_h >= 0) || !(prm->nu_v >= 0) || !(prm->kappa_h >= 0) ||
             !(prm->kappa_v >= 0) || !(prm->c_drag >= 0) || !(prm->nu_4 >= 0) ||
             !isfinite(prm->nu_4) || !isfinite(prm->eos_rho_ref) ||
             !isfinite(prm->eos_alpha) || !isfinite(prm->eos_beta) || !isfinite(prm->eos_T_ref) ||
             !isfinite(prm->eos_S_ref));
}

static bool tuning_ok(const sse_tuning *t) {
    if (!t) return true;
    if (t->patch_cells < 0) return false;
    if (t->bcl_patch_cells != 0) {
        bool known = false;
        for (int pc : {160, 128, 112, 96, 80, 64, 48, 32}) known = known || t->bcl_patch_cells == pc;
        if (!known) return false;
    }
    for (int k = 0; k < 6; k++)
        if (t->reserved[k] != 0) return false;
    return true;
}

static int make_state(const sse_mesh *mesh, const sse_params *prm, const sse_tuning *tun,
                      void *stream, bool count_only, sse_state **out, size_t *bytes) {
    // the state's kernels dereference the mesh's device arrays: the device
    // current now must be the one the mesh was made on
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SSE_ERR_CUDA;
    if (dev != mesh->device) return SSE_ERR_INVALID_ARG;
    std::unique_ptr<sse_state> hold(new (std::nothrow) sse_state());
    sse_state *st = hold.get();
    if (!st) return SSE_ERR_OOM;
    st->device = dev;
    const int pc = (tun && tun->patch_cells > 0) ? tun->patch_cells : 0;
    const int bpc = tun ? tun->bcl_patch_cells : 0;
    int rc;
    size_t b = 0;
    if (prm->precision == SSE_FP64) {
        auto *e = new (std::nothrow) Engine<double>();
        if (!e) return SSE_ERR_OOM;
        st->eng.reset(e);
        e->patch_cells = pc;
        e->bcl_cells = bpc;
        rc = e->init(mesh, prm, (cudaStream_t)stream, count_only);
        b = e->A.bytes;
    } else {
        auto *e = new (std::nothrow) Engine<float>();
        if (!e) return SSE_ERR_OOM;
        st->eng.reset(e);
        e->patch_cells = pc;
        e->bcl_cells = bpc;
        rc = e->init(mesh, prm, (cudaStream_t)stream, count_only);
        b = e->A.bytes;
    }
    if (bytes) *bytes = b;
    if (rc != SSE_OK || count_only) return rc;
    *out = hold.release();
    return SSE_OK;
}

extern "C" int sse_state_create(const sse_mesh *mesh, const sse_params *prm, void *stream,
                                sse_state **out) {
    return sse_state_create_ex(mesh, prm, nullptr, stream, out);
}

extern "C" int sse_state_create_ex(const sse_mesh *mesh, const sse_params *prm,
                                   const sse_tuning *tuning, void *stream, sse_state **out) {
    return guarded([&] {
        if (!mesh || !prm || !out) return SSE_ERR_INVALID_ARG;
        *out = nullptr;
        if (!params_ok(prm) || !tuning_ok(tuning)) return SSE_ERR_INVALID_ARG;
        return make_state(mesh, prm, tuning, stream, false, out, nullptr);
    });
}

extern "C" int sse_state_init(const sse_mesh *mesh, const sse_params *prm, const double *u,
                              const double *h, const double *tracers, const double *windStress,
                              void *stream, sse_state **out) {
    if (!mesh || !prm || !u || !h || !tracers || !out) return SSE_ERR_INVALID_ARG;
    *out = nullptr;
    sse_state *st = nullptr;
    int rc = sse_state_create(mesh, prm, stream, &st);
    if (rc) return rc;
    const size_t CL = (size_t)mesh->dm.C * mesh->dm.L;
    rc = sse_state_set(st, SSE_FIELD_U, u);
    if (!rc) rc = sse_state_set(st, SSE_FIELD_H, h);
    for (int t = 0; !rc && t < prm->nTracers; t++)
        rc = sse_state_set(st, SSE_FIELD_TRACER0 + t, tracers + t * CL);
    if (!rc && windStress) rc = sse_state_set(st, SSE_FIELD_WIND, windStress);
    if (rc) {
        sse_state_destroy(st);
        return rc;
    }
    *out = st;
    return SSE_OK;
}

extern "C" int sse_state_footprint(const sse_mesh *mesh, const sse_params *prm, size_t *bytes) {
    return sse_state_footprint_ex(mesh, prm, nullptr, bytes);
}

extern "C" int sse_state_footprint_ex(const sse_mesh *mesh, const sse_params *prm,
                                      const sse_tuning *tuning, size_t *bytes) {
    return guarded([&] {
        if (!mesh || !prm || !bytes) return SSE_ERR_INVALID_ARG;
        if (!params_ok(prm) || !tuning_ok(tuning)) return SSE_ERR_INVALID_ARG;
        return make_state(mesh, prm, tuning, nullptr, true, nullptr, bytes);
    });
}

extern "C" int sse_mesh_dims(const sse_mesh *mesh, int32_t dims[4]) {
    if (!mesh || !dims) return SSE_ERR_INVALID_ARG;
    dims[0] = mesh->dm.C; dims[1] = mesh->dm.E; dims[2] = mesh->dm.V; dims[3] = mesh->dm.L;
    return SSE_OK;
}

extern "C" int sse_state_inject(sse_state *st, int what, int value) {
    if (!st || what != SSE_INJECT_BARRIER_STALL || (value != 0 && value != 1))
        return SSE_ERR_INVALID_ARG;
    st->eng->inject_stall = (unsigned int)value;
    return SSE_OK;
}

extern "C" int sse_state_graphs(const sse_state *st, int *graphs) {
    if (!st || !graphs) return SSE_ERR_INVALID_ARG;
    *graphs = st->eng->graph_count();
    return SSE_OK;
}

extern "C" int sse_state_patches(const sse_state *st, int *patches) {
    if (!st || !patches) return SSE_ERR_INVALID_ARG;
    *patches = st->eng->patches();
    return SSE_OK;
}

extern "C" int sse_state_subcycle_shape(const sse_state *st, int *threads, int *tmem) {
    if (!st) return SSE_ERR_INVALID_ARG;
    if (threads) *threads = st->eng->patch_threads();
    if (tmem) *tmem = st->eng->patch_tmem();
    return SSE_OK;
}

// Measured choice of the sub-cycle patch size: the Algorithm 3/4 sub-cycle
// (M = 20 sub-steps, the kernel every large step calls two or three times)
// is timed with CUDA events for each candidate patch size on a zero state of
// this mesh; LATENCY keeps the fastest, THROUGHPUT the one with the least
// SM-time (duration x the SMs the patches hold: one per 1024-thread patch,
// half per 512-thread patch), among those within twice the fastest.  Results
// are cached per mesh, precision and objective.
static int tune_impl(const sse_mesh *mesh, const sse_params *prm, int objective,
                     sse_tuning *out) {
    if (!mesh || !prm || !out || (objective != SSE_TUNE_LATENCY &&
                                  objective != SSE_TUNE_THROUGHPUT))
        return SSE_ERR_INVALID_ARG;
    if (!params_ok(prm)) return SSE_ERR_INVALID_ARG;
    sse_mesh *mm = const_cast<sse_mesh *>(mesh);
    const int key = -(1 + prm->precision * 2 + objective);   // negative: not a patch count
    const int bkey = key - 100;                                // the baroclinic patch size
    {
        std::lock_guard<std::mutex> lk(mm->plan_mu);
        auto it = mm->tuned.find(key), jt = mm->tuned.find(bkey);
        if (it != mm->tuned.end() && jt != mm->tuned.end()) {
            memset(out, 0, sizeof(*out));
            out->patch_cells = it->second;
            out->bcl_patch_cells = jt->second;
            return SSE_OK;
        }
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SSE_ERR_CUDA;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int C = mesh->dm.C;
    const int cands[] = {64, 128, 256, 384, 512, 768, 1024, 1536};
    std::vector<std::pair<int, std::pair<float, double>>> res;   // (cells, (ms, SMs held))
    int last_P = -1, rc = SSE_OK;
    for (int pc : cands) {
        if (pc > 64 && C / pc < 1) break;
        sse_tuning t{};
        t.patch_cells = pc;
        sse_state *st = nullptr;
        rc = make_state(mesh, prm, &t, s, false, &st, nullptr);
        if (rc) break;
        const int P = st->eng->patches();
        const double sms = P * (st->eng->patch_threads() / 1024.0);
        if (P == 0 || P == last_P) {     // no tiled plan, or the same plan again
            delete st;
            if (P == 0) break;
            continue;
        }
        last_P = P;
        float best = 1e30f;
        for (int rep = 0; rep < 4 && !rc; rep++) {
            cudaEventRecord(e0, s);
            rc = st->eng->btr_substep(3, 600.0, 20);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);   // the first run warms up
        }
        delete st;
        if (rc) break;
        res.push_back({pc, {best, sms}});
    }
    // LATENCY: the fastest; THROUGHPUT: the least SM-time among candidates
    // within twice the fastest
    auto pick = [objective](const std::vector<std::pair<int, std::pair<float, double>>> &cand) {
        int c = 0;
        if (cand.empty()) return c;
        float fastest = 1e30f;
        for (auto &r : cand) fastest = std::min(fastest, r.second.first);
        double best_cost = 1e300;
        for (auto &r : cand) {
            const double cost = objective == SSE_TUNE_LATENCY
                                    ? r.second.first
                                    : (double)r.second.first * r.second.second;
            if (r.second.first <= 2.0f * fastest && cost < best_cost) {
                best_cost = cost;
                c = r.first;
            }
        }
        return c;
    };
    const int choice = rc ? 0 : pick(res);
    // the fused baroclinic kernel's patch size: Algorithm 1 of the same zero
    // state for each size whose plan fits (a size that falls back is skipped)
    std::vector<std::pair<int, std::pair<float, double>>> bres;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, mesh->device);
    const int per_sm = prm->precision == SSE_FP64 ? 1 : 2;   // CTAs per SM of the kernel
    for (int pc : {160, 128, 112, 96, 80, 64, 48, 32}) {
        if (rc) break;
        sse_tuning t{};
        t.patch_cells = choice;
        t.bcl_patch_cells = pc;
        sse_state *st = nullptr;
        rc = make_state(mesh, prm, &t, s, false, &st, nullptr);
        if (rc) break;
        if (st->eng->bcl_patch_cells() != pc) {
            delete st;
            continue;
        }
        const double sms = std::min((double)nsm,
                                    (double)((st->eng->bcl_patch_count() + per_sm - 1) / per_sm));
        float best = 1e30f;
        for (int rep = 0; rep < 4 && !rc; rep++) {
            cudaEventRecord(e0, s);
            rc = st->eng->bcl_feuler(600.0);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);   // the first run warms up
        }
        delete st;
        if (rc) break;
        bres.push_back({pc, {best, sms}});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc) return rc;
    const int bchoice = pick(bres);
    {
        std::lock_guard<std::mutex> lk(mm->plan_mu);
        mm->tuned[key] = choice;
        mm->tuned[bkey] = bchoice;
    }
    memset(out, 0, sizeof(*out));
    out->patch_cells = choice;
    out->bcl_patch_cells = bchoice;
    return SSE_OK;
}

extern "C" int sse_tune(const sse_mesh *mesh, const sse_params *prm, int objective,
                        sse_tuning *out) {
    return guarded([&] { return tune_impl(mesh, prm, objective, out); });
}

extern "C" void sse_state_destroy(sse_state *st) { delete st; }

extern "C" int sse_state_set(sse_state *st, int field, const double *host) {
    return guarded([&] {
        if (!st || !host) return SSE_ERR_INVALID_ARG;
        return st->eng->set(field, host);
    });
}

extern "C" int sse_state_get(sse_state *st, int field, double *host) {
    return guarded([&] {
        if (!st || !host) return SSE_ERR_INVALID_ARG;
        return st->eng->get(field, host);
    });
}

extern "C" int sse_state_transfer(sse_state *st, int field, void *host, int flags) {
    return guarded([&] {
        if (!st || !host || (flags & ~(SSE_XFER_GET | SSE_XFER_F32 | SSE_XFER_ASYNC)) != 0)
            return SSE_ERR_INVALID_ARG;
        return st->eng->transfer(field, host, flags);
    });
}

extern "C" int sse_state_sync(sse_state *st) {
    return guarded([&] {
        if (!st) return SSE_ERR_INVALID_ARG;
        return st->eng->sync();
    });
}

extern "C" int sse_state_set_f32(sse_state *st, int field, const float *host) {
    return guarded([&] {
        if (!st || !host) return SSE_ERR_INVALID_ARG;
        return st->eng->set_f32(field, host);
    });
}

extern "C" int sse_state_get_f32(sse_state *st, int field, float *host) {
    return guarded([&] {
        if (!st || !host) return SSE_ERR_INVALID_ARG;
        return st->eng->get_f32(field, host);
    });
}

extern "C" int sse_step(sse_state *st, int order, double dt, int n_substeps, int n_steps) {
    return guarded([&] {
        if (!st || (order != 2 && order != 3) || !(dt > 0) || !isfinite(dt) || n_substeps < 1 ||
            n_steps < 0)
            return SSE_ERR_INVALID_ARG;
        NvtxScope range("sse_step");
        int i = 0, rc = SSE_OK;
        for (; !rc && i + 2 <= n_steps; i += 2) rc = st->eng->step2(order, dt, n_substeps);
        for (; !rc && i < n_steps; i++) rc = st->eng->step(order, dt, n_substeps);
        return rc;
    });
}

// ---------------------------------------------------------------------------
// Batched steps: several states advance in lock-step; the i-th launch of every
// state's step (recorded by Engine::step with `rec` set) is issued as one grid
// for the 3-D kernels, and each state's sub-cycle runs on its own stream
// between fork and join events.  Per-state arithmetic is unchanged.
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_combine_G_batch(const CombineJob<R> *__restrict__ jobs,
                                  const int *__restrict__ first, int njobs) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    __shared__ CombineJob<R> J;
    if (threadIdx.x == 0) J = jobs[lo];
    __syncthreads();
    combine_edge<R>(J, (blockIdx.x - first[lo]) * blockDim.x + threadIdx.x);
}

namespace {
// staging of the job descriptors: two regions (steps alternate), pinned host
// and device, grown on demand; one per (device, stream), used under its mutex.
// Work on one stream is ordered, so the upload of step s + 2 into a region
// follows the kernels of step s that read it; batches on other streams have
// arenas of their own.
struct BatchArena {
    std::mutex mu;
    size_t cap = 0;
    char *host[2] = {nullptr, nullptr};
    char *dev[2] = {nullptr, nullptr};
    cudaEvent_t uploaded[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    int reserve(size_t bytes, int n, cudaStream_t ms) {
        if (!fork && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
            return SSE_ERR_CUDA;
        while ((int)join.size() < n + 1) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return SSE_ERR_CUDA;
            join.push_back(e);
        }
        if (bytes <= cap) return SSE_OK;
        // the old regions may still feed kernels queued on this stream
        if (cap && cudaStreamSynchronize(ms) != cudaSuccess) return SSE_ERR_CUDA;
        for (int b = 0; b < 2; b++) {
            if (uploaded[b]) cudaEventSynchronize(uploaded[b]);
            if (host[b]) cudaFreeHost(host[b]);
            if (dev[b]) cudaFree(dev[b]);
            host[b] = nullptr; dev[b] = nullptr;
        }
        cap = 0;
        for (int b = 0; b < 2; b++) {
            if (cudaMallocHost(&host[b], bytes) != cudaSuccess || cudaMalloc(&dev[b], bytes) != cudaSuccess)
                return SSE_ERR_OOM;
            if (!uploaded[b] && cudaEventCreateWithFlags(&uploaded[b], cudaEventDisableTiming) != cudaSuccess)
                return SSE_ERR_CUDA;
        }
        cap = bytes;
        return SSE_OK;
    }
};
std::mutex g_arena_mu;
std::map<std::pair<int, cudaStream_t>, std::unique_ptr<BatchArena>> g_arenas;

size_t align64(size_t x) { return (x + 63) / 64 * 64; }

template <class R> size_t job_size(int cls) {
    switch (cls) {
    case REC_COLFLUX: return sizeof(ColfluxJob<R>);
    case REC_BCL: return sizeof(BclJob<R>);
    case REC_TRANSPORT: return sizeof(TransportJob<R>);
    case REC_THICK: return sizeof(ThickJob<R>);
    case REC_COMBINE: return sizeof(CombineJob<R>);
    default: return 0;
    }
}
template <class R> const void *job_ptr(const LaunchRec<R> &r) {
    switch (r.cls) {
    case REC_COLFLUX: return &r.u.cf;
    case REC_BCL: return &r.u.bcl;
    case REC_TRANSPORT: return &r.u.tr;
    case REC_THICK: return &r.u.th;
    case REC_COMBINE: return &r.u.cmb;
    default: return nullptr;
    }
}
// blocks of one state's launch of class cls
template <class R> int job_blocks(const LaunchRec<R> &r) {
    switch (r.cls) {
    case REC_COLFLUX: return colflux_blocks(r.u.cf.m);
    case REC_BCL: return r.u.bcl.t.P;
    case REC_TRANSPORT: return (r.u.tr.m.E + 127) / 128;
    case REC_THICK: return r.u.th.t.P;
    case REC_COMBINE: return (r.u.cmb.n + 255) / 256;
    default: return 0;
    }
}

template <class R>
int step_batch_t(std::vector<Engine<R> *> &E, int order, const double *dt, const int32_t *M,
                 int n_steps, cudaStream_t ms) {
    const int n = (int)E.size();
    int dev = 0;
    CK(cudaGetDevice(&dev));
    BatchArena *A = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_arena_mu);
        auto &slot = g_arenas[std::make_pair(dev, ms)];
        if (!slot) slot.reset(new BatchArena());
        A = slot.get();
    }
    std::lock_guard<std::mutex> lk(A->mu);
    std::vector<std::vector<LaunchRec<R>>> rec(n);
    for (int st = 0; st < n_steps; st++) {
        // record the step of every state (this also advances their buffers)
        for (int i = 0; i < n; i++) {
            rec[i].clear();
            E[i]->rec = &rec[i];
            const int rc = E[i]->step(order, dt[i], M[i]);
            E[i]->rec = nullptr;
            if (rc) return rc;
        }
        const size_t nl = rec[0].size();
        for (int i = 1; i < n; i++) {
            if (rec[i].size() != nl) return SSE_ERR_UNSUPPORTED;
            for (size_t k = 0; k < nl; k++)
                if (rec[i][k].cls != rec[0][k].cls) return SSE_ERR_UNSUPPORTED;
        }
        // lay out the step's job arrays: per launch, n descriptors and n + 1 block starts
        std::vector<size_t> off(nl, 0), foff(nl, 0);
        size_t bytes = 0;
        for (size_t k = 0; k < nl; k++) {
            const size_t js = job_size<R>(rec[0][k].cls);
            if (!js) continue;
            off[k] = bytes;
            bytes = align64(bytes + js * n);
            foff[k] = bytes;
            bytes = align64(bytes + sizeof(int) * (n + 1));
        }
        int rc = A->reserve(std::max<size_t>(bytes, 64), n, ms);
        if (rc) return rc;
        const int b = st & 1;
        // the host region may still feed the upload of two steps ago
        CK(cudaEventSynchronize(A->uploaded[b]));
        std::vector<int> blocks(nl, 0);
        for (size_t k = 0; k < nl; k++) {
            const size_t js = job_size<R>(rec[0][k].cls);
            if (!js) continue;
            int *first = (int *)(A->host[b] + foff[k]);
            int acc = 0;
            for (int i = 0; i < n; i++) {
                memcpy(A->host[b] + off[k] + js * i, job_ptr<R>(rec[i][k]), js);
                first[i] = acc;
                acc += job_blocks<R>(rec[i][k]);
            }
            first[n] = acc;
            blocks[k] = acc;
        }
        CK(cudaMemcpyAsync(A->dev[b], A->host[b], bytes, cudaMemcpyHostToDevice, ms));
        CK(cudaEventRecord(A->uploaded[b], ms));
        for (size_t k = 0; k < nl; k++) {
            const int cls = rec[0][k].cls;
            const char *d = A->dev[b];
            if (cls == REC_BTR) {
                // fork: every sub-cycle on its own state's stream, then join
                CK(cudaEventRecord(A->fork, ms));
                for (int i = 0; i < n; i++) {
                    CK(cudaStreamWaitEvent(E[i]->s, A->fork, 0));
                    CK(E[i]->issue_btr(rec[i][k].u.btr));
                    CK(cudaEventRecord(A->join[i], E[i]->s));
                }
                for (int i = 0; i < n; i++) CK(cudaStreamWaitEvent(ms, A->join[i], 0));
                continue;
            }
            const int *first = (const int *)(d + foff[k]);
            size_t smem = 0;
            for (int i = 0; i < n; i++) smem = std::max(smem, rec[i][k].smem);
            switch (cls) {
            case REC_COLFLUX:
                launch_colflux_batch<R>((const ColfluxJob<R> *)(d + off[k]), first, n, blocks[k], ms);
                break;
            case REC_BCL:
                launch_bcl_fused_batch<R>((const BclJob<R> *)(d + off[k]), first, n, blocks[k], smem, ms);
                break;
            case REC_TRANSPORT:
                launch_transport_cols_batch<R>((const TransportJob<R> *)(d + off[k]), first, n,
                                               blocks[k], ms);
                break;
            case REC_THICK:
                launch_thick_fused_batch<R>((const ThickJob<R> *)(d + off[k]), first, n, blocks[k],
                                            smem, ms);
                break;
            case REC_COMBINE:
                k_combine_G_batch<R><<<blocks[k], 256, 0, ms>>>((const CombineJob<R> *)(d + off[k]),
                                                                first, n);
                break;
            }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                fprintf(stderr, "libsse: batched launch failed: %s\n", cudaGetErrorString(e));
                return SSE_ERR_CUDA;
            }
        }
    }
    // later work on each state's own stream follows the batch
    CK(cudaEventRecord(A->join[n], ms));
    for (int i = 0; i < n; i++) CK(cudaStreamWaitEvent(E[i]->s, A->join[n], 0));
    return SSE_OK;
}
}  // namespace

extern "C" int sse_step_batch(sse_state *const *states, int n, int order, const double *dt,
                              const int32_t *n_substeps, int n_steps, void *cuda_stream) {
    return guarded([&] {
        if (!states || n < 1 || !dt || !n_substeps || (order != 2 && order != 3) || n_steps < 0)
            return SSE_ERR_INVALID_ARG;
        for (int i = 0; i < n; i++) {
            if (!states[i] || !(dt[i] > 0) || !isfinite(dt[i]) || n_substeps[i] < 1)
                return SSE_ERR_INVALID_ARG;
            for (int j = 0; j < i; j++)
                if (states[j] == states[i]) return SSE_ERR_INVALID_ARG;
        }
        if (n_steps == 0) return SSE_OK;
        NvtxScope range("sse_step_batch");
        int rc = SSE_ERR_UNSUPPORTED;
        auto run = [&](auto *proto) {
            using Eng = std::remove_pointer_t<decltype(proto)>;
            std::vector<Eng *> E;
            for (int i = 0; i < n; i++) {
                Eng *e = dynamic_cast<Eng *>(states[i]->eng.get());
                if (!e || !e->fused || !e->fused_th || e->prof || e->inject_stall) return SSE_ERR_UNSUPPORTED;
                E.push_back(e);
            }
            for (int i = 1; i < n; i++)
                if (states[i]->device != states[0]->device) return SSE_ERR_INVALID_ARG;
            return step_batch_t(E, order, dt, n_substeps, n_steps, (cudaStream_t)cuda_stream);
        };
        if (dynamic_cast<Engine<float> *>(states[0]->eng.get()))
            rc = run((Engine<float> *)nullptr);
        else if (dynamic_cast<Engine<double> *>(states[0]->eng.get()))
            rc = run((Engine<double> *)nullptr);
        return rc;
    });
}

extern "C" int sse_baroclinic_feuler(sse_state *st, double dt) {
    return guarded([&] {
        if (!st || !(dt > 0) || !isfinite(dt)) return SSE_ERR_INVALID_ARG;
        return st->eng->bcl_feuler(dt);
    });
}

extern "C" int sse_barotropic_substep(sse_state *st, int order, double dt, int n_substeps) {
    return guarded([&] {
        if (!st || (order != 2 && order != 3) || !(dt > 0) || !isfinite(dt) || n_substeps < 1)
            return SSE_ERR_INVALID_ARG;
        return st->eng->btr_substep(order, dt, n_substeps);
    });
}

extern "C" int sse_diagnostics(sse_state *st, sse_diag *out) {
    return guarded([&] {
        if (!st || !out) return SSE_ERR_INVALID_ARG;
        return st->eng->diagnostics(out);
    });
}

extern "C" int sse_kernels_per_step(const sse_state *st, int order) {
    if (!st) return SSE_ERR_INVALID_ARG;
    // 4 per baroclinic stage (5 with biharmonic viscosity; 2 when fused), 1
    // per sub-cycle, 2 per thickness stage, 1 forcing combination
    const int bcl = st->eng->fused_bcl() ? 2 : 4 + (st->eng->has_del4() ? 1 : 0);
    return order == 2 ? 2 * bcl + 2 + 2 * 2 + 1 : 3 * bcl + 3 + 3 * 2 + 1;
}

extern "C" int sse_profile(sse_state *st, int enable) {
    if (!st) return SSE_ERR_INVALID_ARG;
    st->eng->prof_clear();
    st->eng->prof = (enable != 0);
    return SSE_OK;
}

extern "C" int sse_profile_read(sse_state *st, double *ms, int32_t *launches) {
    return guarded([&] {
        if (!st || !ms || !launches) return SSE_ERR_INVALID_ARG;
        return st->eng->prof_read(ms, launches);
    });
}

extern "C" const char *sse_strerror(int code) {
    switch (code) {
    case SSE_OK: return "ok";
    case SSE_ERR_INVALID_ARG: return "invalid argument";
    case SSE_ERR_BAD_MESH: return "invalid mesh (index out of range or non-positive geometry)";
    case SSE_ERR_OOM: return "out of memory";
    case SSE_ERR_CUDA: return "CUDA error";
    case SSE_ERR_NONFINITE: return "non-finite value in the state";
    case SSE_ERR_SYNC_TIMEOUT: return "grid barrier of the barotropic sub-cycle timed out";
    case SSE_ERR_UNSUPPORTED: return "size beyond a compiled limit";
    case SSE_ERR_TIMEOUT: return "request not finished within the timeout";
    case SSE_ERR_CANCELLED: return "request cancelled when its server stopped";
    case SSE_ERR_INTERNAL: return "unexpected host-side failure in the library";
    default: return "unknown error";
    }
}
