// sse_internal.cuh -- device data structures shared by the kernels and the
// host driver of libsse.so.  Device arrays are layer-major and padded:
// X[k * Ep + e] for edge fields, X[k * Cp + i] for cell fields,
// X[k * Vp + v] for vertex fields (Ep, Cp, Vp multiples of 32).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace sse {

constexpr int MAXE = 8;    // edges per cell
constexpr int MAXE2 = 16;  // edges on edge
constexpr int LMAX = 64;   // layers

// Mesh coefficients in one precision (R = double or float).
template <class R>
struct Coef {
    const R *divc;   // [maxE][Cp]  n_{e,i} l_e / A_i
    const R *kec;    // [maxE][Cp]  l_e d_e / (4 A_i)
    const R *wl;     // [maxE2][Ep] w_{e,e'} l_{e'} / d_e
    const R *cfc;    // [maxE2][Ep] w_{e,e'} l_{e'} / d_e * (f_e + f_{e'}) / 2
    const R *curlc;  // [3][Vp]     t_{e,v} d_e / A_v (0 where absent)
    const R *kw;     // [3][Vp]     kite / sum(kites of ocean cells) (0 where land)
    const R *invdc;  // [Ep]        1 / d_e
    const R *invdv;  // [Ep]        1 / l_e
    const R *fV;     // [Vp]        f at vertices
    const R *H;      // [Cp]        resting depth
};

struct DMesh {
    int C, E, V, L, Cp, Ep, Vp, maxE, maxE2;
    const int2 *coe;    // [Ep] cells on edge
    const int2 *voe;    // [Ep] vertices on edge
    const int *neoc;    // [Cp]
    const int *eoc;     // [maxE][Cp] edges on cell
    const int *ooc;     // [maxE][Cp] the other cell across that edge
    const int *neoe;    // [Ep]
    const int *eoe;     // [maxE2][Ep]
    const int *eov;     // [3][Vp] (absent -> 0, with zero coefficient)
    const int *cov;     // [3][Vp] (land -> 0, with zero weight)
    // numbering: the caller's cell / edge index -> the internal one, and back
    // (padding entries map to 0)
    const int *cperm, *eperm;   // [Cp], [Ep] caller -> internal
    const int *cinv, *einv;     // [Cp], [Ep] internal -> caller
    const double *H;    // [Cp] resting depth
    const double *sfrac;  // [L] z-star fractions
    const float *sfrac_f; // [L] the same in FP32
    // partial bottom cells (partial = 1): layers per cell and per edge, and the
    // per-column z-star shares [L][Cp] (0 below the column's bottom)
    int partial;
    const int *kc;        // [Cp]
    const int *ke;        // [Ep]
    const double *sfc;    // [L][Cp]
    const float *sfc_f;   // [L][Cp]
    const double *divc_d; // [maxE][Cp] divergence coefficients in FP64
    const double *area;   // [Cp]
    const double *ld2;    // [Ep] l_e d_e / 2 (energy weight)
    Coef<double> d;
    Coef<float> f;
};

template <class R> __host__ __device__ inline const Coef<R> &coef(const DMesh &m);
template <> __host__ __device__ inline const Coef<double> &coef<double>(const DMesh &m) { return m.d; }
template <> __host__ __device__ inline const Coef<float> &coef<float>(const DMesh &m) { return m.f; }

// physical constants in one precision (converted once on the host)
template <class R> struct PhysR {
    R g, inv_rho0, nu_h, nu_v, kappa_h, kappa_v, c_drag, nu_4;
    R alpha, beta, T_ref, S_ref;  // rho' = rho - rho_ref = -alpha (T - T_ref) + beta (S - S_ref)
    R zcoef;                      // g (1 - rho_ref / rho0)
};

struct DParams {
    double g, rho0, nu_h, nu_v, kappa_h, kappa_v, c_drag, nu_4;
    double alpha, beta, T_ref, S_ref;
    double zcoef;                      // g (1 - rho_ref / rho0)
    int nT, recon;
    const double *wind;                // [Ep] wind stress / rho0, or nullptr
    const float *wind_f;               // the same in FP32
    PhysR<double> pd;
    PhysR<float> pf;
};

template <class R> __host__ __device__ inline const PhysR<R> &phys(const DParams &p);
template <> __host__ __device__ inline const PhysR<double> &phys<double>(const DParams &p) { return p.pd; }
template <> __host__ __device__ inline const PhysR<float> &phys<float>(const DParams &p) { return p.pf; }
template <class R> __device__ inline const R *wind_over_rho0(const DParams &p);
template <> __device__ inline const double *wind_over_rho0<double>(const DParams &p) { return p.wind; }
template <> __device__ inline const float *wind_over_rho0<float>(const DParams &p) { return p.wind_f; }

// Grid barrier words of the persistent sub-cycle kernel.
struct Barrier {
    unsigned int *count;  // arrivals in the current generation (gen == count + 1)
    unsigned int *gen;    // generation counter, zeroed with count before each launch
    int *err;             // nonzero after a timeout
};

// ---- stage kernels (layer-major), launched by the driver -----------------
// two and four values of one precision stored together, loaded as one vector
struct __align__(32) double4x { double x, y, z, w; };
template <class R> struct VecT;
template <> struct VecT<float> { using V2 = float2; using V4 = float4; };
template <> struct VecT<double> { using V2 = double2; using V4 = double4x; };
template <class R> using V2 = typename VecT<R>::V2;
template <class R> using V4 = typename VecT<R>::V4;

// Sum of tendency-precision terms, read out in FP64.  FP32 terms go into an
// unevaluated pair of floats with Knuth's TwoSum, which carries the rounding
// error of every addition exactly in the low part (about 48 significant bits
// in all), so no FP64 instruction runs per term: GB300 runs FP64 and the
// f32->f64 conversion at about 1/67 of the FP32 rate.  FP64 terms are summed
// in a double.
template <class R> struct PairSum;
template <> struct PairSum<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x, bp = s - hi;
        lo += (hi - (s - bp)) + (x - bp);
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <> struct PairSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

template <class R> struct DiagBufs {
    R *delta, *w;                        // [L][Cp] div u; div(h_e u), then w at the top of k
    V4<R> *cq;                           // [L][Cp] (K, p', rho', z_mid), gathered as one
    R *omega, *q;                        // [L][Vp]
    V2<R> *hq;                           // [L][Ep] (h_e u, q_e), gathered as one
    // biharmonic viscosity only (nullptr otherwise): del^2 u on edges, its
    // divergence on cells and its curl on vertices
    R *del2, *delta2, *omega2;
};

// hR is the stage thickness in the tendency precision (the FP64 array itself
// in SSE_FP64, an FP32 copy in SSE_MIXED).
template <class R>
void launch_cell_diag(const DMesh &m, const DParams &p, const R *ubar, const R *ut,
                      const R *hR, const R *tr, const DiagBufs<R> &b, cudaStream_t s);
template <class R>
void launch_vertex(const DMesh &m, const R *ubar, const R *ut, const R *hR,
                   const DiagBufs<R> &b, cudaStream_t s);
template <class R>
void launch_del2_divcurl(const DMesh &m, const DiagBufs<R> &b, cudaStream_t s);
template <class R>
void launch_edge_pre(const DMesh &m, R *ubar, R *ut, const R *hR, const DiagBufs<R> &b,
                     bool split, cudaStream_t s);
template <class R>
void launch_bcl_edge(const DMesh &m, const DParams &p, const R *ubar, const R *ut,
                     const R *hR, const double *zeta, const DiagBufs<R> &b, const R *ut_n,
                     double a, double bcoef, double dt, R *ut_out, R *G, R *vmc,
                     cudaStream_t s);

// ---- the fused baroclinic stage (bcl_fused.cu); plan from build_bcl_plan
template <class R> struct DBcl {
    int P = 0;
    int maxE0 = 0, maxE1 = 0, maxE2 = 0, maxC1 = 0, maxC2 = 0, maxV = 0;
    size_t smem = 0;
    const int *cnt = nullptr;                 // [P][8]
    const int *off_e0, *off_v;
    const unsigned short *e0_eoe;             // [sum 10 nE0]
    const R *e0_cfc;                          // [sum 10 nE0]
    const int *e0_c12, *e0_v12;               // [sum nE0]
    const R *e0_invdc, *e0_invdv;             // [sum nE0]
    const R *v_f;                             // [sum nV]
    // per patch, the connectivity and coefficients the kernel keeps in shared
    // memory, packed by the host in the kernel's layout (bcl_build_image)
    const unsigned char *img;                 // 16-byte aligned blocks
    const long long *img_off;                 // [P + 1] byte offsets
    size_t img_max = 0;                       // the largest block
};
template <class R> struct BclArgs {
    const R *ubar, *ut, *hR, *tr;  // stage input (ubar, utilde, thickness, tracers)
    const double *zeta;            // stage SSH
    const R *Fc;                   // [Ep] column transport sum_k h_e u_k (k_colflux)
    const R *ut_n;                 // old level for the convex combination, or null
    R a, b, dt;                    // out = a ut_n + b (ut1 - dt G)
    R *ut_out, *G;
};
// one state's share of a batched launch
template <class R> struct BclJob { DMesh m; DParams p; DBcl<R> t; BclArgs<R> a; };
template <class R> struct ColfluxJob {
    DMesh m;
    R *ubar, *ut;
    const R *hR;
    R *Fc;
    int split, pad_;
};
template <class R>
void launch_colflux_batch(const ColfluxJob<R> *jobs, const int *first, int njobs, int blocks,
                          cudaStream_t s);
int colflux_blocks(const DMesh &m);
template <class R>
void launch_bcl_fused_batch(const BclJob<R> *jobs, const int *first, int njobs, int blocks,
                            size_t smem, cudaStream_t s);
template <class R> const void *bcl_fused_batch_kernel_ptr();
struct BclPlan;
template <class R> size_t bcl_smem_bytes(const BclPlan &plan, int L);
// the per-patch shared-memory images of a plan (byte offsets [P + 1]); the
// largest image's size is returned
template <class R>
size_t bcl_build_image(const BclPlan &plan, std::vector<unsigned char> &img,
                       std::vector<long long> &off);
// CTAs per SM the fused baroclinic kernel is compiled for (its launch bounds)
template <class R> int bcl_blocks_per_sm();
int bcl_max_edges_per_patch();
int bcl_max_cells_per_patch();
template <class R> const void *bcl_fused_kernel_ptr();
template <class R>
void launch_colflux(const DMesh &m, R *ubar, R *ut, const R *hR, bool split, R *Fc,
                    cudaStream_t s);
template <class R>
void launch_bcl_fused(const DBcl<R> &t, const DMesh &m, const DParams &p, const BclArgs<R> &a,
                      cudaStream_t s);

template <class R> struct BtrArgs {
    const R *ub_start;     // [Ep]
    const double *z_start; // [Cp]
    const R *G;            // [Ep]
    const R *X;            // [Ep] for the epilogue ub_out = alpha X + beta ubar^M (may be null)
    double alpha, beta;
    R *ub_out;             // [Ep]
    double *Fz;            // [Ep]
    double *z_out;         // [Cp] or null
    R *u0, *ua, *uh;       // work [Ep]
    R *z0, *za, *zh;       // work [Cp]
    double tau, g;
    int M, order;
    unsigned int stall;    // test hook: arrivals every grid barrier waits for beyond the grid (0)
    // global-memory kernel only: internal -> caller index of the edge and cell
    // arrays above (ub_start ... z_out) when they are in the caller's
    // numbering (null: internal numbering)
    const int *einv, *cinv;
};
template <class R>
cudaError_t launch_btr(const DMesh &m, const BtrArgs<R> &a, const Barrier &bar, int nblocks,
                       int nthreads, cudaStream_t s);
template <class R> int btr_block_size();
template <class R> const void *btr_kernel_ptr(int order, int maxE2);
int btr_max_items_per_thread();

// Device copy of the tiled sub-cycle plan (see tiles.h): per-patch arrays
// flattened with the offsets cell_off / edge_off.
template <class R> struct DTiles {
    int P, nthreads, own;            // patches, threads per patch, entries per thread
    const int *cell_off, *edge_off;  // [P + 1]
    const int *n_own_c, *n_own_e;    // [P]
    const int *n_int_e;              // [P] owned edges with both cells owned (local 0..)
    const int *ne_lim, *nc_lim;      // [P][3] local edges / cells exact after 0, 1, 2 sub-stages
    const int *cell_gid, *edge_gid;  // local -> global
    const int *c12;                  // [sum ne] byte offsets of local (c1, c2): c1 | c2 << 16
    const unsigned short *eoe;       // [sum ne][TILE_NE2P] byte offsets of local edgesOnEdge
    const R *cfc;                    // per patch [TILE_CFR][ne]: Coriolis coefficients (0 on
                                     // padding), then 1 / d_e
    const unsigned short *ce;        // [sum nc][TILE_NCEP] byte offsets of local edgesOnCell
    const R *divc;                   // per patch [TILE_NCEP][nc] divergence coefficients
    const R *H;                      // patch p at cell_off[p] + p: [nc_p + 1]
    R *xu[2];                        // [Ep] exchange of owned ubar, double-buffered
    R *xz[2];                        // [Cp] exchange of owned zeta
    size_t smem;                     // dynamic shared memory per block
    int tm;                          // 1: the edges' constant data in tensor memory (FP32,
                                     // 1024 threads; eoe then not in shared memory)
};
template <class R>
cudaError_t launch_btr_tiled(const DTiles<R> &t, const BtrArgs<R> &a, const Barrier &bar,
                             cudaStream_t s);
// kernel of the tiled sub-cycle for (order, entries per thread, threads per
// patch: 512 or 1024, edge data in tensor memory); null for a combination
// that has no kernel (tensor memory: FP32 and 1024 threads only)
template <class R> const void *btr_tiled_kernel_ptr(int order, int own, int nthreads, bool tm);
// edges per thread the tensor-memory variant holds (a patch's edges <= this x 1024)
int btr_tiled_tmem_slots();

template <class R> struct TransportArgs {
    const R *hR;              // stage thickness [L][Cp] in the tendency precision
    const double *zeta;       // stage SSH [Cp] (sum h - H)
    const R *ubA, *utA;       // v = wA (ubA + utA) + wB (ubB + utB)
    const R *ubB, *utB;
    double wA, wB;
    const double *Fz, *ex1, *ex2;  // F^zeta and extra F^h terms
    double cF, cE, cA;
    int recon;
    double *S_out;            // sum_k v h_e (or null)
    double *Fcol;             // [Ep] column-integrated mass flux, FP64
    R *flux;                  // [L][Ep] h_e (v + uA)
};
template <class R>
void launch_transport(const DMesh &m, const TransportArgs<R> &a, cudaStream_t s);

template <class R> struct ThickArgs {
    const R *flux;            // [L][Ep]
    const double *Fcol;       // [Ep] column-integrated flux (FP64)
    const double *h_s;        // stage thickness
    const R *hR_s;            // stage thickness in the tendency precision
    const R *tr_s;            // stage tracers [nT][L][Cp]
    const double *h_n;        // h^n (convex combination)
    const R *hR_n;            // h^n in the tendency precision
    const R *tr_n;
    double a, b, dt;          // out = a * (h^n) + b * (FE result)
    double *h_out;
    R *hR_out;                // FP32 copy of h_out (SSE_MIXED) or null
    R *tr_out;
    double *zeta_out;
};
template <class R>
void launch_thickness(const DMesh &m, const DParams &p, const ThickArgs<R> &a, cudaStream_t s);

// ---- the fused thickness/tracer stage (thick_fused.cu); plan from build_thick_plan
struct DThick {
    int P = 0, Pc = 0, maxEO = 0, maxC1 = 0;
    const int *cnt = nullptr;            // [P][4]
    const int *off_eo, *off_c1;          // [P + 1]
    const int *eogid, *c1gid;            // local -> internal
    const unsigned short *o_e, *o_o;     // [P][6][Pc]
};
template <class R> struct ThickFArgs {
    // transport velocity v = wA (ubA + utA) + wB (ubB + utB) + u^A (utB may be null)
    const R *ubA, *utA, *ubB, *utB;
    double wA, wB;
    const R *uA;              // [Ep] from k_transport_cols
    const double *Fcol;       // [Ep] column-integrated flux (FP64)
    const double *h_s;        // stage thickness (FP64) and its tendency-precision copy
    const R *hR_s, *tr_s;
    const double *h_n;        // h^n for the convex combination (unused when a == 0)
    const R *hR_n, *tr_n;
    double a, b, dt;          // out = a (h^n) + b (FE result)
    double *h_out;
    R *hR_out;                // tendency-precision copy of h_out (SSE_MIXED) or null
    R *tr_out;
    double *zeta_out;
};
template <class R> struct ThickJob { DMesh m; DParams p; DThick t; ThickFArgs<R> a; };
template <class R> struct TransportJob { DMesh m; TransportArgs<R> a; R *uA; };
template <class R>
void launch_transport_cols_batch(const TransportJob<R> *jobs, const int *first, int njobs,
                                 int blocks, cudaStream_t s);
template <class R>
void launch_thick_fused_batch(const ThickJob<R> *jobs, const int *first, int njobs, int blocks,
                              size_t smem, cudaStream_t s);
template <class R> const void *thick_fused_batch_kernel_ptr();
size_t thick_smem_bytes(const DThick &plan, int nT, bool twoB, bool comb, size_t sR);
int thick_cells_per_patch();
template <class R> const void *thick_fused_kernel_ptr();
template <class R>
void launch_transport_cols(const DMesh &m, const TransportArgs<R> &a, R *uA, cudaStream_t s);
template <class R>
void launch_thick_fused(const DThick &t, const DMesh &m, const DParams &p, const ThickFArgs<R> &a,
                        size_t smem, cudaStream_t s);


// layout conversion: host-order [n][L] in precision H (FP64 or FP32) <->
// device layer-major R [L][np]
// (perm: the caller's index -> the internal one, DMesh::cperm / eperm); the
// device holds the value minus `off` (a tracer's storage offset), the way
// back adds it
template <class R, class H>
void launch_to_device(const H *src, R *dst, int n, int L, int np, const int *perm,
                      cudaStream_t s, double off = 0.0);
template <class R, class H>
void launch_from_device(const R *src, H *dst, int n, int L, int np, const int *perm,
                        cudaStream_t s, double off = 0.0);
template <class R, class H>
void launch_add_bar(const R *ubar, const R *ut, H *dst, int E, int L, int Ep,
                    const int *kmax, const int *perm, cudaStream_t s);
template <class R>
void launch_mask_layers(R *x, int n, int L, int np, const int *kmax, cudaStream_t s);
void launch_h_to_float(const double *h, float *hf, int n, cudaStream_t s);
void launch_scale(const double *src, double scale, double *dst_d, float *dst_f, int n,
                  const int *perm, cudaStream_t s);
void launch_ssh(const DMesh &m, const double *h, double *zeta, cudaStream_t s);

template <class R>
void launch_diag(const DMesh &m, const R *ubar, const R *ut, const double *h, const R *tr,
                 int nT, const double *toff, const double *zeta, double *partials, int nparts,
                 double *out, cudaStream_t s);

}  // namespace sse
