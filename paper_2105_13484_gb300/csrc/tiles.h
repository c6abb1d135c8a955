// tiles.h -- host-side patch plan of the tiled barotropic sub-cycle.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace sse {

// padded per-entry strides of the tiled sub-cycle's local connectivity
constexpr int TILE_NE2P = 10;  // edgesOnEdge per edge (hexagon/pentagon meshes: <= 10)
constexpr int TILE_NCEP = 6;   // edgesOnCell per cell (<= 6)

// host copy of the connectivity and coefficients the plan needs
struct HostMesh {
    int C = 0, E = 0, maxE = 0, maxE2 = 0;
    std::vector<int> c1, c2;      // [E]
    std::vector<int> neoc, eoc;   // [C], [C][maxE]
    std::vector<int> neoe, eoe;   // [E], [E][maxE2]
    std::vector<double> cfc;      // [E][maxE2] w l'/d (f+f')/2
    std::vector<double> divc;     // [C][maxE]  n l / A
    std::vector<double> invdc;    // [E]
    std::vector<double> H;        // [C]
};

struct TilePatch {
    int nc = 0, ne = 0, n_own_c = 0, n_own_e = 0;
    int n_int_e = 0;                       // owned edges with both cells owned (first)
    std::vector<int> cell_gid, edge_gid;   // local -> global (owned first)
    std::vector<int32_t> c12;              // [ne] local c1 | c2 << 16
    std::vector<int16_t> n2;               // [ne]
    std::vector<int16_t> eoe;              // [ne][maxE2] local (dummy = ne)
    std::vector<double> cfc;               // [ne][maxE2]
    std::vector<double> invdc;             // [ne]
    std::vector<int16_t> nce;              // [nc]
    std::vector<int16_t> ce;               // [nc][maxE] local edges (dummy = ne)
    std::vector<double> divc;              // [nc][maxE]
    std::vector<double> H;                 // [nc + 1]
    // prefix counts by halo ring: local edges with ring <= r+1 (r = 0..2; an
    // edge's ring is the larger ring of its two cells, cells outside the patch
    // count K+1) and local cells with ring <= r (r = 0..2)
    int ne_ring[3] = {0, 0, 0}, nc_ring[3] = {0, 0, 0};
};

struct TilePlan {
    int P = 0, K = 0;
    std::vector<TilePatch> patches;
    std::vector<int> cell_off, edge_off;   // [P + 1] prefix sums of nc, ne
};

// Partition into P patches with halos of K rings; false if a patch would
// need more than 32766 local entries.  Local order: owned cells, then halo
// cells by ring; owned edges (first cell owned: those with both cells owned,
// then the others), then halo edges by ring.
bool build_tile_plan(const HostMesh &hm, int P, int K, TilePlan &plan);
// True if every edgesOnEdge entry of an edge is an edge of one of its two
// cells (the TRiSK stencil): the ring counts of a plan, which decide which
// halo values are exact after each sub-stage, rely on it.
bool tile_stencil_ok(const HostMesh &hm);
// Dynamic shared memory of the largest patch for element size sR.
size_t tile_smem_bytes(const TilePlan &plan, int maxE, int maxE2, size_t sR);

}  // namespace sse
