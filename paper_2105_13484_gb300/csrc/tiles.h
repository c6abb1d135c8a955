// tiles.h -- host-side patch plan of the tiled barotropic sub-cycle.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace sse {

// padded per-entry strides of the tiled sub-cycle's local connectivity
constexpr int TILE_NE2P = 10;  // edgesOnEdge per edge (hexagon/pentagon meshes: <= 10)
// rows of a patch's streamed per-edge coefficient block: the TILE_NE2P
// Coriolis coefficients, then 1 / d_e
constexpr int TILE_CFR = TILE_NE2P + 1;
constexpr int TILE_NCEP = 6;   // edgesOnCell per cell (<= 6)

// host copy of the connectivity and coefficients the plans need (the
// library's internal numbering)
struct HostMesh {
    int C = 0, E = 0, V = 0, maxE = 0, maxE2 = 0;
    std::vector<int> c1, c2;      // [E]
    std::vector<int> v1, v2;      // [E]
    std::vector<int> neoc, eoc;   // [C], [C][maxE]
    std::vector<int> neoe, eoe;   // [E], [E][maxE2]
    std::vector<int> eov, cov;    // [V][3], -1 = absent
    std::vector<double> cfc;      // [E][maxE2] w l'/d (f+f')/2
    std::vector<double> wl;       // [E][maxE2] w l'/d
    std::vector<double> divc;     // [C][maxE]  n l / A
    std::vector<double> kec;      // [C][maxE]  l d / (4 A)
    std::vector<double> curlc;    // [V][3]     t d / A_v (0 where absent)
    std::vector<double> kw;       // [V][3]     normalised kite weight (0 where absent)
    std::vector<double> fV;       // [V]
    std::vector<double> invdc;    // [E]
    std::vector<double> invdv;    // [E]
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
// Dynamic shared memory of the largest patch for element size sR; without
// the edgesOnEdge offsets when eoe_smem is false (they live in tensor memory).
size_t tile_smem_bytes(const TilePlan &plan, int maxE, int maxE2, size_t sR, bool eoe_smem = true);

// Locality order of the cells of a mesh given by the cells of its edges:
// the parts (about `leaf` cells each) of a recursive bisection of the cell
// graph, in depth-first order, each part in increasing index.  Returns
// new -> old: any run of consecutive cells in this order covers a compact
// region, which the library uses as its internal cell numbering.
std::vector<int> cell_locality_order(int C, const std::vector<int> &c1,
                                     const std::vector<int> &c2, int leaf);

// Patch plan of the fused baroclinic kernel (one CTA per patch, the stage's
// cell, vertex and edge diagnostics of a layer in shared memory).  The cells
// are cut into ceil(C / Pc) compact parts by recursive bisection; patch p
// owns the edges whose lower-numbered cell lies in part p (E0).
// Local index spaces, each listing its smaller set first:
//   E0 <= E1 <= E2 (edges): E1 = the edges of C1's cells (edgesOnEdge of E0
//   lies in E1 for TRiSK stencils), E2 = E1 plus the edges of V's vertices;
//   C1 <= C2 (cells): C1 = the cells of E0's edges, C2 = C1 plus the cells of
//   E1's edges and of V's vertices; V = the vertices of E1's edges.
// Per-item arrays of a patch are term-major ([j][n]) so that a warp reading
// term j of consecutive items reads one contiguous run.  Local indices are
// 16-bit; a dummy slot after the last entry of E1 (hq), E2 (velocity) and C2
// (thickness) holds zero and stands in for absent neighbours.
// Cells into P compact parts (recursive bisection of the cell graph); the
// part of each cell.
std::vector<int> partition_cells(const HostMesh &hm, int P);

struct BclPlan {
    int P = 0, Pc = 0;
    std::vector<int> owner;                        // [C] patch of each cell
    int maxE0 = 0, maxE1 = 0, maxE2 = 0, maxC1 = 0, maxC2 = 0, maxV = 0;
    std::vector<int> cnt;                          // [P][8]: nE0 nE1 nE2 nC1 nC2 nV 0 0
    std::vector<int> off_e0, off_e1, off_e2;       // [P + 1] prefix sums
    std::vector<int> off_c1, off_c2, off_v;        // [P + 1]
    std::vector<int> egid, cgid;                   // [sum nE2], [sum nC2] local -> internal
    std::vector<uint16_t> e0_eoe;                  // [sum 10 nE0] local E1 index of edgesOnEdge
    std::vector<double> e0_wl, e0_cfc;             // [sum 10 nE0]
    std::vector<int> e0_c12, e0_v12;               // [sum nE0] c1 | c2 << 16 (C1), v1 | v2 << 16 (V)
    std::vector<int> e0_n2;                        // [sum nE0] edgesOnEdge count
    std::vector<double> e0_invdc, e0_invdv;        // [sum nE0]
    std::vector<int> e1_c12, e1_v12;               // [sum nE1] cells (C2), vertices (V)
    std::vector<uint16_t> c1_e, c1_o;              // [sum 6 nC1] local edge (E2), other cell (C2)
    std::vector<double> c1_divc, c1_kec;           // [sum 6 nC1]
    std::vector<uint16_t> v_e, v_c;                // [sum 3 nV] local edge (E2), cell (C2)
    std::vector<double> v_curl, v_kw;              // [sum 3 nV]
    std::vector<double> v_f;                       // [sum nV]
};
constexpr int BCL_NE2P = 10;   // edgesOnEdge slots of the fused kernel
constexpr int BCL_NCEP = 6;    // edgesOnCell slots of the fused kernel
// Patches of Pc cells with at most max_e0 owned edges and max_c1 cells in C1
// each; false if a patch breaks a limit, a local index needs more than 16
// bits, a cell has more than 6 edges, an edge more than 10 edgesOnEdge, or
// edgesOnEdge leaves E1.
bool build_bcl_plan(const HostMesh &hm, int Pc, int max_e0, int max_c1, BclPlan &plan);

// Patch plan of the fused thickness/tracer kernel (one CTA per patch).  The
// cells are cut into compact parts of at most Pc cells by recursive
// bisection; patch p owns part p's cells (local cells 0 .. nO - 1); EO = the
// edges of the owned cells, C1 = the owned cells followed by the cells across
// EO's edges.  Per owned cell, term-major ([j][Pc]): its edges
// (local EO index; a zero slot after EO's last entry for absent ones) and
// the cell across each (local C1 index; the cell itself for absent ones).
struct ThickPlan {
    int P = 0, Pc = 0, maxEO = 0, maxC1 = 0;
    std::vector<int> owner;                // [C] patch of each cell
    std::vector<int> cnt;                  // [P][4]: nO nEO nC1 0
    std::vector<int> off_eo, off_c1;       // [P + 1]
    std::vector<int> eogid, c1gid;         // [sum nEO], [sum nC1] local -> internal
    std::vector<int> eo_c12;               // [sum nEO] c1 | c2 << 16 (C1 indices)
    std::vector<uint16_t> o_e, o_o;        // [P][6][Pc] local edge, local cell across
};
bool build_thick_plan(const HostMesh &hm, int Pc, ThickPlan &plan);

}  // namespace sse
