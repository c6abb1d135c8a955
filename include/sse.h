/*
 * sse.h -- C ABI of libsse.so: GB300 (sm_103a) multirate split-explicit
 * SSPRK2-SE / SSPRK3-SE time stepping of the layered primitive equations on
 * an unstructured TRiSK C-grid (Lan, Ju, Wang, Gunzburger, Jones, "High-order
 * multirate explicit time-stepping schemes for the baroclinic-barotropic
 * split dynamics in primitive equations").
 *
 * Conventions
 *   - Indices are 0-based int32; -1 marks an absent entry where allowed.
 *   - All host arrays passed in are owned by the caller and only read during
 *     the call.  All device memory is owned by the library.
 *   - Field arrays on the host are layer-fastest: X[i*nLayers + k], k = 0 is
 *     the top layer.  The device layout is the library's own (layer-major,
 *     padded); it is never exposed.
 *   - Every function returns SSE_OK (0) or a negative SSE_ERR_* code and
 *     never throws; sse_strerror() names the code.  A host allocation that
 *     fails inside the library (mesh plans, staging buffers) is SSE_ERR_OOM
 *     like a device one; any other unexpected host-side failure is
 *     SSE_ERR_INTERNAL.  After a non-fatal error
 *     (INVALID_ARG, BAD_MESH, NONFINITE) the objects stay valid.  After
 *     SSE_ERR_CUDA or SSE_ERR_SYNC_TIMEOUT the state must be re-set with
 *     sse_state_set before it is stepped again.
 *   - Work is issued on the stream given at sse_state_create (NULL = the
 *     legacy default stream).  sse_step is asynchronous; sse_state_get and
 *     sse_diagnostics synchronise that stream.
 */
#ifndef SSE_H
#define SSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define SSE_OK 0
#define SSE_ERR_INVALID_ARG (-1)   /* bad pointer, size, order, dt or M        */
#define SSE_ERR_BAD_MESH (-2)      /* index out of range, non-positive geometry */
#define SSE_ERR_OOM (-3)           /* device or host allocation failed          */
#define SSE_ERR_CUDA (-4)          /* a CUDA call failed                        */
#define SSE_ERR_NONFINITE (-5)     /* NaN/Inf found by sse_diagnostics          */
#define SSE_ERR_SYNC_TIMEOUT (-6)  /* a grid barrier of the sub-cycle timed out */
#define SSE_ERR_UNSUPPORTED (-7)   /* size beyond a compiled limit              */
#define SSE_ERR_TIMEOUT (-8)       /* sse_server_wait: the request is not done  */
#define SSE_ERR_CANCELLED (-9)     /* request dropped when its server stopped   */
#define SSE_ERR_INTERNAL (-10)     /* unexpected host-side failure in the library */

/* ---- precision of the device arithmetic ---- */
#define SSE_FP64 0   /* everything in FP64                                       */
#define SSE_MIXED 1  /* FP32 tendencies, velocities and tracers; FP64 layer
                        thickness, SSH, accumulated barotropic flux, flux
                        deficits and global sums                                 */

/* ---- SSH reconciliation (Sec. 3.4) ---- */
#define SSE_RECON_OFF 0         /* no transport-velocity adjustment             */
#define SSE_RECON_PAPER 1       /* F^h exactly as printed in Sec. 3.4           */
#define SSE_RECON_CONSISTENT 2  /* F^h from the already adjusted stage fluxes,
                                   so sum(h) - H equals the sub-cycle SSH       */

/* ---- fields for sse_state_set / sse_state_get ---- */
#define SSE_FIELD_U 0        /* normal velocity u      [nEdges][nLayers]        */
#define SSE_FIELD_H 1        /* layer thickness h      [nCells][nLayers]        */
#define SSE_FIELD_TRACER0 2  /* temperature            [nCells][nLayers]        */
#define SSE_FIELD_TRACER1 3  /* salinity (nTracers=2)  [nCells][nLayers]        */
#define SSE_FIELD_WIND 4     /* normal wind stress     [nEdges], N m^-2 (set)   */
#define SSE_FIELD_ZETA 5     /* SSH zeta = sum h - H   [nCells] (get)           */
#define SSE_FIELD_UBAR 6     /* barotropic velocity    [nEdges]                 */
#define SSE_FIELD_UTILDE 7   /* baroclinic velocity    [nEdges][nLayers]        */
#define SSE_FIELD_G 8        /* barotropic forcing G   [nEdges]                 */
#define SSE_FIELD_FZETA 9    /* accumulated sub-cycle flux F^zeta [nEdges] (get)*/
#define SSE_FIELD_ZETA_SUB 10 /* SSH at the end of the last sub-cycle [nCells]  */

typedef struct sse_mesh sse_mesh;
typedef struct sse_state sse_state;

/* Unstructured C-grid (MPAS/TRiSK conventions).  Edge normal n_e points from
 * cellsOnEdge[e][0] to cellsOnEdge[e][1]; tangent k x n_e points from
 * verticesOnEdge[e][0] to verticesOnEdge[e][1].  The tangential velocity is
 * u^t_e = (1/dcEdge_e) sum_j weightsOnEdge[e][j] dvEdge_{e'} u_{e'} over
 * e' = edgesOnEdge[e][j], j < nEdgesOnEdge[e] (TRiSK, Sec. 5 of the paper).
 * Land is expressed by leaving it out: every listed cell is ocean and every
 * listed edge joins two ocean cells; cellsOnVertex / edgesOnVertex may hold
 * -1 where the vertex touches land.  Limits: maxEdges <= 8,
 * maxEdges2 <= 16, 1 <= nLayers <= 64. */
typedef struct {
    int32_t nCells, nEdges, nVertices, maxEdges, maxEdges2, nLayers;
    const int32_t *cellsOnEdge;      /* [nEdges][2]                        */
    const int32_t *verticesOnEdge;   /* [nEdges][2]                        */
    const int32_t *nEdgesOnCell;     /* [nCells]                           */
    const int32_t *edgesOnCell;      /* [nCells][maxEdges]                 */
    const int32_t *cellsOnVertex;    /* [nVertices][3], -1 = land          */
    const int32_t *edgesOnVertex;    /* [nVertices][3], -1 = absent        */
    const int32_t *nEdgesOnEdge;     /* [nEdges]                           */
    const int32_t *edgesOnEdge;      /* [nEdges][maxEdges2]                */
    const double *weightsOnEdge;     /* [nEdges][maxEdges2]                */
    const double *dcEdge;            /* [nEdges] cell-centre distance (m)  */
    const double *dvEdge;            /* [nEdges] edge length (m)           */
    const double *areaCell;          /* [nCells] (m^2)                     */
    const double *areaTriangle;      /* [nVertices] dual-cell area (m^2)   */
    const double *kiteAreasOnVertex; /* [nVertices][3] (m^2)               */
    const double *fEdge;             /* [nEdges] Coriolis parameter (1/s)  */
    const double *fVertex;           /* [nVertices]                        */
    const double *bottomDepth;       /* [nCells] resting depth H (m) > 0   */
    const double *restThicknessFrac; /* [nLayers] z-star fractions, sum 1  */
    /* Partial bottom cells (both NULL: every column has all nLayers layers
     * with thicknesses restThicknessFrac x bottomDepth).  maxLevelCell[i] in
     * 1..nLayers is the number of layers of column i; restThickness[i][k] > 0
     * for k < maxLevelCell[i], 0 below, sums to bottomDepth[i] (relative
     * 1e-10); the z-star stretching of layer k of column i is
     * restThickness[i][k] / bottomDepth[i].  An edge has the layers both its
     * cells have.  State values in missing layers are ignored and read back
     * as 0. */
    const int32_t *maxLevelCell;     /* [nCells] or NULL                   */
    const double *restThickness;     /* [nCells][nLayers] or NULL          */
} sse_mesh_desc;

/* SSE_OPT_VMIX: every baroclinic stage uses Algorithm 2
 * (Baroclinic_FEuler_Mixing) instead of Algorithm 1: D^u leaves the explicit
 * tendency and (I - dt D^u) u1 = ut1 + ubar is solved down every edge column
 * (tridiagonal), wind stress explicit at the top, bottom drag linearised about
 * the speed of the stage's input velocity; then ut1 = u1 - ubar. */
#define SSE_OPT_VMIX 1

/* Physics and numerics.  Linear equation of state (Eq. eqstate):
 *   rho = eos_rho_ref - eos_alpha (T - eos_T_ref) + eos_beta (S - eos_S_ref). */
typedef struct {
    int32_t precision;  /* SSE_FP64 or SSE_MIXED                             */
    int32_t recon;      /* SSE_RECON_*                                        */
    int32_t nTracers;   /* 1 (T) or 2 (T, S)                                  */
    int32_t options;    /* bit set of SSE_OPT_* (other bits: SSE_ERR_INVALID_ARG) */
    double g, rho0;     /* gravity (m s^-2), reference density (kg m^-3)      */
    double nu_h, nu_v;  /* horizontal / vertical viscosity (m^2 s^-1)         */
    double kappa_h, kappa_v; /* tracer diffusivities (m^2 s^-1)               */
    double c_drag;      /* quadratic bottom-drag coefficient                  */
    double eos_rho_ref, eos_alpha, eos_beta, eos_T_ref, eos_S_ref;
    double nu_4;        /* biharmonic viscosity (m^4 s^-1): -nu_4 del^4 u in T^u, the
                           hyperviscosity of the paper's global setup (Sec. 2)  */
} sse_params;

/* Global diagnostics, reduced on the device in a fixed order (FP64). */
typedef struct {
    double volume;            /* sum_i A_i sum_k h_ik (m^3)                   */
    double tracer_content[2]; /* sum_i A_i sum_k h_ik phi_ik                  */
    double kinetic_energy;    /* sum_e (l_e d_e / 2) sum_k h_e u_ek^2 / 2     */
    double max_speed;         /* max |u_ek|                                    */
    double min_thickness;     /* min h_ik                                      */
    double zeta_min, zeta_max;
    int64_t step;             /* large steps taken since the last state set    */
    int32_t nonfinite;        /* 1 if any u, h or tracer is NaN/Inf            */
    int32_t reserved;
} sse_diag;

/* Copy and validate a mesh; uploads connectivity and derived coefficients
 * (divergence, curl, kinetic-energy, TRiSK and Coriolis coefficients) to the
 * current CUDA device.  *out receives the handle.  BAD_MESH on any index out
 * of range or non-positive geometry; UNSUPPORTED beyond the stated limits.
 * The library numbers cells, edges and vertices internally in a locality
 * order of its own (a recursive bisection of the cell graph); every per-cell
 * and per-edge array of this API, on the host or on the device, stays in the
 * caller's numbering. */
int sse_mesh_create(const sse_mesh_desc *desc, sse_mesh **out);
void sse_mesh_destroy(sse_mesh *mesh);

/* Allocate a model state on `mesh` with parameters `params`; `cuda_stream`
 * is a cudaStream_t (or NULL).  The state starts at rest with h = 0 and must
 * be filled with sse_state_set (at least U, H and the tracers).  The device
 * current at the call must be the one the mesh was made on (else
 * SSE_ERR_INVALID_ARG). */
int sse_state_create(const sse_mesh *mesh, const sse_params *params, void *cuda_stream,
                     sse_state **out);
void sse_state_destroy(sse_state *state);

/* sse_state_create followed by sse_state_set of U, H, each tracer and (if not
 * NULL) the wind stress: the whole initial state of Sec. 3 in one call.
 *   u           host [nEdges][nLayers] normal velocity (split into ubar and
 *               utilde by Eq. BBspl at the first step)
 *   h           host [nCells][nLayers] layer thickness (zeta = sum h - H)
 *   tracers     host [nTracers][nCells][nLayers] (T, then S)
 *   windStress  host [nEdges] normal wind stress (N m^-2) or NULL
 * On any error nothing is left allocated and *out is NULL. */
int sse_state_init(const sse_mesh *mesh, const sse_params *params, const double *u,
                   const double *h, const double *tracers, const double *windStress,
                   void *cuda_stream, sse_state **out);

/* Host -> device copy of one field (FP64 host array, layout per SSE_FIELD_*).
 * Setting U splits it into barotropic and baroclinic parts at the next step
 * (Eq. BBspl); setting H recomputes zeta.  Settable: U, H, TRACER0/1, WIND,
 * UBAR, UTILDE, G (the last three feed the algorithm-level calls below). */
int sse_state_set(sse_state *state, int field, const double *host);
/* Device -> host copy of one field as FP64; synchronises the stream. */
int sse_state_get(sse_state *state, int field, double *host_out);
/* The same transfers with FP32 host arrays, for the fields a state holds in
 * its tendency precision: U, UTILDE, UBAR, G, TRACER0/1 (FP32 in the mixed
 * form, so nothing is rounded there; the FP64 form rounds on the way out and
 * widens on the way in).  H, ZETA, ZETA_SUB, FZETA and WIND are FP64 state in
 * both forms: SSE_ERR_INVALID_ARG.  Both calls return once the host array has
 * been read or written.  With page-locked host memory (cudaHostAlloc,
 * cudaHostRegister) the conversion kernels access the host array directly,
 * for sse_state_set/get as well; the array must then hold the whole field. */
int sse_state_set_f32(sse_state *state, int field, const float *host);
int sse_state_get_f32(sse_state *state, int field, float *host_out);

/* One entry point for all four transfers, with a stream-ordered option.
 * flags: SSE_XFER_GET (device -> host; else host -> device), SSE_XFER_F32
 * (an FP32 host array, same fields as sse_state_set_f32; else FP64) and
 * SSE_XFER_ASYNC: the call returns without synchronising the state's
 * stream.  Then the host array is read or written when the stream reaches
 * the transfer: it must stay valid, and unchanged for a set, until then, and
 * its contents after a get are defined only once the stream has passed it
 * (sse_state_sync).  A pageable host array makes the copy synchronous all the
 * same (the CUDA copy semantics of pageable memory); page-locked memory does
 * not.  A barrier timeout is reported by the next synchronising call.
 * SSE_ERR_INVALID_ARG for unknown flags or a field the precision excludes. */
#define SSE_XFER_GET 1
#define SSE_XFER_F32 2
#define SSE_XFER_ASYNC 4
int sse_state_transfer(sse_state *state, int field, void *host, int flags);
/* Synchronise the state's stream; returns SSE_ERR_SYNC_TIMEOUT if a grid
 * barrier of the sub-cycle timed out since the state was last set. */
int sse_state_sync(sse_state *state);

/* Advance n_steps large steps of SSPRK{order}-SE (order 2: Sec. 3.2 with
 * Algorithm 3; order 3: Sec. 3.3 with Algorithm 4), time step dt (s) and
 * n_substeps barotropic sub-steps of dt/n_substeps, with the reconciliation
 * of Sec. 3.4 chosen in params.  Asynchronous on the state's stream.
 * INVALID_ARG for order not in {2,3}, dt <= 0 or non-finite, n_substeps < 1,
 * n_steps < 0. */
int sse_step(sse_state *state, int order, double dt, int n_substeps, int n_steps);

/* The same steps for n states at once, in lock-step (Sec. 3.2 / 3.3 per state,
 * with each state's own dt[i] and n_substeps[i]): the 3-D kernels of all n
 * states are issued as one launch per kernel and stage on `cuda_stream`, each
 * state's barotropic sub-cycle (Algorithm 3 / 4) runs on the state's own
 * stream between events that fork from and join back into `cuda_stream`, and
 * every state's stream waits for the batch at the end.  Each state's results
 * are bit-identical to sse_step on it alone.  The states must have been made
 * on the current device, share the precision, and use the fused baroclinic
 * and thickness kernels (full columns, Algorithm 1, no biharmonic viscosity)
 * with profiling and test hooks off; otherwise SSE_ERR_UNSUPPORTED and no
 * state is stepped.  INVALID_ARG as for sse_step, for n < 1 or for a state
 * listed twice.  Asynchronous. */
int sse_step_batch(sse_state *const *states, int n, int order, const double *dt,
                   const int32_t *n_substeps, int n_steps, void *cuda_stream);

/* Algorithm 1 (Baroclinic_FEuler) alone, on the state's u (= UBAR + UTILDE),
 * UTILDE, h, tracers and zeta = sum h - H: overwrites UTILDE with the
 * output tilde-u^1 and G with the barotropic forcing. */
int sse_baroclinic_feuler(sse_state *state, double dt);
/* Algorithm 3 (order 2) or Algorithm 4 (order 3) alone: sub-cycles UBAR and
 * zeta with frozen G; overwrites UBAR with ubar^1, FZETA with the
 * accumulated flux of Sec. 3.4 and ZETA_SUB with the sub-cycle's own SSH. */
int sse_barotropic_substep(sse_state *state, int order, double dt, int n_substeps);

/* Global sums and extrema (synchronises the stream).  Returns NONFINITE if
 * any u, h or tracer value is NaN or Inf (out is filled either way). */
int sse_diagnostics(sse_state *state, sse_diag *out);

/* Number of kernels sse_step launches per large step for `order`. */
int sse_kernels_per_step(const sse_state *state, int order);

/* Per-kernel timing with CUDA events on the state's stream.  Kernel classes: */
#define SSE_K_CELL_DIAG 0   /* cell diagnostics (K, div u, rho', p', z, w)   */
#define SSE_K_VERTEX 1      /* vorticity and potential vorticity             */
#define SSE_K_EDGE_PRE 2    /* edge mass flux, q_e, split (Eq. BBspl)        */
#define SSE_K_BCL_EDGE 3    /* Algorithm 1 edge kernel                        */
#define SSE_K_BTR 4         /* Algorithms 3/4 persistent sub-cycle            */
#define SSE_K_TRANSPORT 5   /* Sec. 3.4 adjustment and edge mass flux         */
#define SSE_K_THICKNESS 6   /* thickness and tracer stage                     */
#define SSE_K_COMBINE 7     /* Interp_2 / Interp_3 forcing combination        */
#define SSE_K_DEL4 8        /* div and curl of del^2 u (biharmonic viscosity)  */
#define SSE_K_NCLASS 9
/* enable != 0 starts recording an event pair around every launch of sse_step
 * (and clears earlier records); enable == 0 stops recording. */
int sse_profile(sse_state *state, int enable);
/* Synchronises the stream; fills ms[SSE_K_NCLASS] with the summed device time
 * of each class and launches[SSE_K_NCLASS] with the launch counts recorded
 * since the last sse_profile(state, 1). */
int sse_profile_read(sse_state *state, double *ms, int32_t *launches);

/* Measurement utility (no counterpart in the paper): the fused multiply-add
 * rate of the current GPU in TFLOP/s (2 flops per FMA), FP64 for
 * precision = SSE_FP64 and FP32 for SSE_MIXED, timed with CUDA events over
 * many independent FMA chains on every SM.  It allocates a few bytes, runs
 * on a private stream and synchronises it; the benchmark uses it as the
 * denominator of the FP64 form's arithmetic roofline. */
int sse_probe_fma_rate(int precision, double *tflops);

/* Allocation-free variant of sse_barotropic_substep (FP64), for callers that
 * must not allocate device memory at the point where they run the sub-cycle:
 * code running inside a device-memory allocator or memory-pool callback, a
 * host runtime that reserves all of its device memory up front and forbids
 * later cudaMalloc calls, or a latency-critical loop that cannot accept the
 * device-wide synchronisation cudaMalloc and cudaFree may imply.  The paper
 * has no counterpart; it computes the same Algorithm 3 (order 2) or
 * Algorithm 4 (order 3) sub-cycle as sse_barotropic_substep.
 *   mesh       a mesh made earlier by sse_mesh_create
 *   ubar_in    device [nEdges] barotropic velocity at the start
 *   zeta_in    device [nCells] SSH at the start
 *   G          device [nEdges] frozen barotropic forcing
 *   ubar_out   device [nEdges] ubar after n_substeps sub-steps of dt/n_substeps
 *   Fzeta_out  device [nEdges] accumulated flux F^zeta of Sec. 3.4
 *   zeta_out   device [nCells] the sub-cycle's own final SSH, or NULL
 *   cuda_stream  cudaStream_t (NULL = legacy default stream)
 * The caller owns all these arrays; the library allocates nothing in this
 * call.  Its work buffers live in one file-scope device array of fixed size
 * (limits: nEdges <= 393216, nCells <= 131072, about 12.6 MB) that every GPU
 * loading the library holds until the process exits; larger meshes return
 * SSE_ERR_UNSUPPORTED.  The first call on a device looks up that array's
 * device address and the launch shape (the first call of each order); make
 * it before any stream capture.  The device current at the call must be the
 * one the mesh was made on (else SSE_ERR_INVALID_ARG).  All calls share the
 * array, so calls that overlap on the GPU (on different streams or devices'
 * shared context) race and must be serialised by the caller; each call clears
 * the barrier and error words itself.  The call copies the barrier status to
 * host memory and synchronises `cuda_stream` before it returns, and returns
 * SSE_ERR_SYNC_TIMEOUT if a grid barrier timed out. */
int sse_barotropic_substep_noalloc(const sse_mesh *mesh, int order, double dt, int n_substeps,
                                   double g, const double *ubar_in, const double *zeta_in,
                                   const double *G, double *ubar_out, double *Fzeta_out,
                                   double *zeta_out, void *cuda_stream);

/* Launch-shape choices of a state.  patch_cells: target cells per patch of
 * the tiled barotropic sub-cycle.  0 (the default): one patch per SM, at most
 * one patch per 64 cells.  A positive value asks for about that many cells per
 * patch, up to two patches per SM (more than one patch per SM run as 512-thread
 * blocks holding at most half an SM's shared memory each).  Larger patches use
 * fewer SMs for longer, which lets the sub-cycles of several states run side
 * by side.  bcl_patch_cells: cells per patch of the fused baroclinic kernel
 * (Algorithm 1), one of 160, 128, 112, 96, 80, 64, 48, 32; 0 (the default):
 * the largest whose patches fit the kernel with as many CTAs per SM as it is
 * compiled for.  A size whose plan does not fit falls back to the default.
 * Smaller patches give a small mesh more CTAs (shorter latency when it runs
 * alone) at the cost of more halo work.  Results are the same bits for every
 * choice of either size. */
typedef struct {
    int32_t patch_cells;
    int32_t bcl_patch_cells;
    int32_t reserved[6];     /* must be 0 */
} sse_tuning;

#define SSE_TUNE_LATENCY 0     /* the fastest sub-cycle                          */
#define SSE_TUNE_THROUGHPUT 1  /* the least SM-time (duration x SMs held: one
                                  per 1024-thread patch, half per 512-thread
                                  patch) within twice the fastest              */

int sse_state_create_ex(const sse_mesh *mesh, const sse_params *params,
                        const sse_tuning *tuning, void *cuda_stream, sse_state **out);
/* Patches of the state's tiled sub-cycle (0: the global-memory sub-cycle). */
int sse_state_patches(const sse_state *state, int *patches);
/* The tiled sub-cycle's launch shape (Algorithms 3 and 4): threads per patch
 * (0 without a tiled sub-cycle), and 1 if each thread's edge coefficients and
 * edgesOnEdge offsets sit in the SM's tensor memory for the whole sub-cycle
 * (FP32 form, 1024-thread patches of at most 4096 edges; the environment
 * variable SSE_BTR_TMEM=0, read when the state is created, turns it off),
 * else 0 (streamed from L2).  Both shapes give the same bits.  Any output
 * pointer may be null.  SSE_ERR_INVALID_ARG for a null state. */
int sse_state_subcycle_shape(const sse_state *state, int *threads, int *tmem);
/* CUDA graphs the state holds.  sse_step with n_steps >= 2 runs the steps in
 * pairs, each pair replayed from a graph captured (once per order, dt,
 * n_substeps and buffer assignment) from the launches a single step makes;
 * an odd last step runs launch by launch.  Graphs are not used while
 * profiling is on or the test hook below is set, and not at all on the
 * legacy default stream (a NULL cuda_stream), which cannot be captured.
 * Results are the same bits either way.  While a capture is in progress,
 * work that another thread puts on the legacy default stream would have to
 * wait for the state's stream; give a state stepped in pairs a stream created
 * with cudaStreamNonBlocking (the request runtime's streams are) when other
 * threads use the legacy default stream. */
int sse_state_graphs(const sse_state *state, int *graphs);

/* Test hook for the failure path of the sub-cycle's grid barriers (no
 * counterpart in the paper).  With SSE_INJECT_BARRIER_STALL set to 1, every
 * grid-barrier wait of the state's sub-cycle waits for one arrival more than
 * its grid provides, so that the wait runs out its bounded budget (2 s), the
 * kernel sets the state's error word and returns: the next sse_state_get or
 * sse_diagnostics returns SSE_ERR_SYNC_TIMEOUT and the CUDA context stays
 * usable.  Set it back to 0 and re-set the state (sse_state_set) to continue.
 * Returns SSE_ERR_INVALID_ARG for another `what` or a value other than 0/1. */
#define SSE_INJECT_BARRIER_STALL 1
int sse_state_inject(sse_state *state, int what, int value);
/* Autotuner: times the Algorithm 3/4 sub-cycle (M = 20) of a zero state of
 * this mesh for each candidate patch size, then Algorithm 1 for each fused
 * baroclinic patch size whose plan fits, and returns the best of each for the
 * objective (SSE_TUNE_*: LATENCY the fastest; THROUGHPUT the least SM-time,
 * duration x the SMs the launch holds, among candidates within twice the
 * fastest).  Runs GPU work on a private stream; the result is cached in the
 * mesh. */
int sse_tune(const sse_mesh *mesh, const sse_params *params, int objective, sse_tuning *out);

/* Device bytes a state of this mesh and parameter set would allocate
 * (everything sse_state_create allocates; nothing is allocated here). */
int sse_state_footprint(const sse_mesh *mesh, const sse_params *params, size_t *bytes);
int sse_state_footprint_ex(const sse_mesh *mesh, const sse_params *params,
                           const sse_tuning *tuning, size_t *bytes);

/* dims = {nCells, nEdges, nVertices, nLayers} of a mesh. */
int sse_mesh_dims(const sse_mesh *mesh, int32_t dims[4]);

/* ---------------------------------------------------------------------------
 * Request runtime: continuous batching of independent solves on one GPU.
 *
 * A request is one solve: an initial state (u [nEdges][nLayers], h
 * [nCells][nLayers], tracers [nTracers][nCells][nLayers], host, FP64,
 * layer-fastest; copied at submission; wind_stress [nEdges] or NULL, as
 * SSE_FIELD_WIND) advanced n_steps SSPRK{order}-SE steps
 * of dt with n_substeps barotropic sub-steps (Sec. 3.2 / 3.3).  A worker
 * thread admits requests in arrival order while the sum of their
 * sse_state_footprint stays within hbm_budget_bytes and at most max_active
 * run; each admitted request gets its own stream and a device-resident state
 * and is advanced steps_per_launch steps at a time, its work overlapping with
 * that of the other active requests.  When it reaches its horizon the final
 * (u, h, tracers) are written to the caller's output buffers (same layouts;
 * they must stay valid until the request is done) and its memory is released,
 * so waiting requests are admitted as slots and memory free up.  The mesh
 * must outlive every request that uses it.  Results do not depend on what else
 * runs: each request's arithmetic is exactly that of sse_step on its state. */
typedef struct sse_server sse_server;

#define SSE_REQ_DONE 0       /* finished; outputs written                       */
#define SSE_REQ_PENDING 1    /* waiting for admission                           */
#define SSE_REQ_ACTIVE 2     /* admitted, stepping (negative: failed, SSE_ERR_*) */

typedef struct {
    int64_t id;
    int32_t status;          /* SSE_REQ_* or a negative SSE_ERR_* code        */
    int32_t steps_done;
    double t_submit, t_admit, t_done;   /* seconds since the server started     */
    size_t footprint;        /* device bytes the request holds while active   */
} sse_request_info;

typedef struct {
    int32_t pending, active, max_active_seen, reserved;
    size_t used_bytes, peak_bytes, budget_bytes;
} sse_server_info;

/* tune_objective: -1 = default launch shapes, else SSE_TUNE_* (sse_tune is
 * run once per mesh and precision, at the first submission that uses it). */
int sse_server_create(int device, size_t hbm_budget_bytes, int max_active,
                      int steps_per_launch, int tune_objective, sse_server **out);
/* flags = SSE_SERVER_PACKED: the active requests of one precision and order
 * advance in rounds of up to steps_per_launch steps, all of them in one
 * sse_step_batch call (one 3-D launch per kernel and stage for the whole
 * round); between rounds finished requests retire and waiting ones join.
 * Requests whose states cannot be packed step alone.  flags = 0 is
 * sse_server_create: every request steps on its own stream. */
#define SSE_SERVER_PACKED 1
int sse_server_create_ex(int device, size_t hbm_budget_bytes, int max_active,
                         int steps_per_launch, int tune_objective, int flags,
                         sse_server **out);
/* Queue a request; *id_out identifies it.  SSE_ERR_OOM if it alone exceeds
 * the budget. */
int sse_server_submit(sse_server *server, const sse_mesh *mesh, const sse_params *params,
                      const double *u, const double *h, const double *tracers,
                      const double *wind_stress, int order, double dt, int n_substeps,
                      int n_steps, double *u_out, double *h_out, double *tracers_out,
                      int64_t *id_out);
int sse_server_query(sse_server *server, int64_t id, sse_request_info *info);
/* Block until the request is done or failed (SSE_OK) or timeout_s passes
 * (SSE_ERR_TIMEOUT; timeout_s < 0 waits forever). */
int sse_server_wait(sse_server *server, int64_t id, double timeout_s, sse_request_info *info);
int sse_server_stats(sse_server *server, sse_server_info *info);
/* Forget a finished (or failed, or cancelled) request's record so that a
 * long-running server does not accumulate them; SSE_ERR_INVALID_ARG if the
 * request is still waiting or running or the id is unknown. */
int sse_server_release(sse_server *server, int64_t id);
/* Cancel the requests still waiting (SSE_ERR_CANCELLED), let the admitted ones
 * finish, stop the worker and free everything. */
void sse_server_destroy(sse_server *server);

const char *sse_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SSE_H */
