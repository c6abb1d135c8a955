/*
 * sse_oracle.h -- plain FP64 CPU oracle of the SSPRK2-SE / SSPRK3-SE schemes
 * (Lan, Ju, Wang, Gunzburger, Jones: multirate split-explicit SSPRK time
 * stepping for the layered primitive equations).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA path.  It is
 * used by the tests, by the smoke check and by the benchmark's CPU-baseline
 * leg; the product path never calls it.  It shares no code with the CUDA
 * library.
 *
 * Arrays are layer-fastest: X[i*L + k] is layer k (0 = top) of mesh entity i.
 * Mesh conventions follow paper_2105_13484_gb300/mesh.py (cellsOnEdge = c1,c2,
 * normal from c1 to c2; verticesOnEdge = v1,v2 with v2 in the +k x n
 * direction; -1 marks an absent entry).
 */
#ifndef SSE_ORACLE_H
#define SSE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nCells, nEdges, nVertices, maxEdges, maxEdges2, nLayers;
    const int *cellsOnEdge;       /* [E][2] */
    const int *verticesOnEdge;    /* [E][2] */
    const int *nEdgesOnCell;      /* [C] */
    const int *edgesOnCell;       /* [C][maxEdges] */
    const int *cellsOnVertex;     /* [V][3] */
    const int *edgesOnVertex;     /* [V][3] */
    const int *nEdgesOnEdge;      /* [E] */
    const int *edgesOnEdge;       /* [E][maxEdges2] */
    const double *weightsOnEdge;  /* [E][maxEdges2] */
    const double *dcEdge, *dvEdge, *areaCell, *areaTriangle;
    const double *kiteAreasOnVertex; /* [V][3] */
    const double *fEdge, *fVertex, *bottomDepth;
    const double *restThicknessFrac; /* [L], sums to 1 */
    /* partial bottom cells (both NULL: every column has all L layers with the
     * fractions above): active layers per cell, and the rest thickness of
     * each cell's layers ([C][L], 0 below maxLevelCell, summing to H) */
    const int *maxLevelCell;
    const double *restThickness;
} om_mesh;

typedef struct {
    int nTracers;          /* 1: temperature; 2: temperature, salinity */
    int recon;             /* 0 off, 1 as printed in Sec. 3.4, 2 consistent */
    double g, rho0, nu_h, nu_v, kappa_h, kappa_v, c_drag;
    double eos_rho_ref, eos_alpha, eos_beta, eos_T_ref, eos_S_ref;
    const double *windStress; /* [E] normal wind stress (N m^-2) or NULL */
    int vmix;              /* 1: Algorithm 2 (implicit vertical mixing) in every stage */
    double nu_4;           /* biharmonic viscosity: -nu_4 del^4 u in T^u (m^4 s^-1) */
} om_params;

/* optional per-step records for the tests (NULL members are skipped) */
typedef struct {
    double *zeta_sub;   /* [C] SSH at the end of the corrector sub-cycle */
    double *D1, *D2, *D3;        /* [E] flux deficits */
    double *Fz1, *Fz2, *Fz3;     /* [E] accumulated sub-cycle fluxes */
    double *G0, *G1, *G2;        /* [E] barotropic forcings of the stages */
} om_aux;

/* ---- TRiSK operators (layer-fastest, L layers) ---- */
void om_div(const om_mesh *m, int L, const double *F, double *out);
void om_grad(const om_mesh *m, int L, const double *phi, double *out);
void om_curl(const om_mesh *m, int L, const double *u, double *out);
void om_tangential(const om_mesh *m, int L, const double *u, double *out);
void om_kinetic_energy(const om_mesh *m, int L, const double *u, double *out);
void om_laplacian(const om_mesh *m, int L, const double *u, double *out);
/* del^4 u = Laplacian of the Laplacian (the hyperviscosity operator) */
void om_biharmonic(const om_mesh *m, int L, const double *u, double *out);
void om_coriolis(const om_mesh *m, int L, const double *x, double *out);
void om_edge_thickness(const om_mesh *m, int L, const double *h, double *out);
void om_vertex_thickness(const om_mesh *m, int L, const double *h, double *out);
void om_pv_flux(const om_mesh *m, int L, const double *u, const double *h, double *out);

/* ---- vertical pieces ---- */
void om_vertical_velocity(const om_mesh *m, const double *h, const double *v, double *w);
void om_density(const om_mesh *m, const om_params *p, const double *tr, double *rho);
void om_pressure(const om_mesh *m, const om_params *p, const double *h, const double *rho,
                 double *pres, double *zmid);

/* ---- the split system and its pieces ---- */
void om_split(const om_mesh *m, const double *u, const double *h, double *ubar, double *ut);
void om_baroclinic_rhs(const om_mesh *m, const om_params *p, const double *u, const double *ut,
                       const double *zeta, const double *h, const double *tr, double *rhs);
void om_baroclinic_feuler(const om_mesh *m, const om_params *p, const double *u,
                          const double *ut, const double *zeta, const double *h,
                          const double *tr, double dt, double *ut1, double *G);
/* implicit vertical diffusion (I - dt D^u) x = r per edge column, D^u with the
 * wind stress at the surface (explicit) and the bottom drag linearised about
 * the speed of u_drag (implicit) */
void om_vertical_mixing_solve(const om_mesh *m, const om_params *p, const double *u_drag,
                              const double *h, const double *r, double dt, double *x);
void om_baroclinic_feuler_mixing(const om_mesh *m, const om_params *p, const double *u,
                                 const double *ut, const double *ubar, const double *zeta,
                                 const double *h, const double *tr, double dt, double *ut1,
                                 double *G);
void om_barotropic_fe(const om_mesh *m, const om_params *p, const double *ubar,
                      const double *zeta, const double *G, double tau, double *ubar1,
                      double *zeta1, double *flux);
void om_barotropic_substep(const om_mesh *m, const om_params *p, int order,
                           const double *ubar, const double *zeta, const double *G, double dt,
                           int M, double *ubar1, double *Fzeta, double *zeta1);
void om_thickness_tracer_fe(const om_mesh *m, const om_params *p, const double *h,
                            const double *tr, const double *v, double dt, double *h1,
                            double *tr1);
void om_ssh(const om_mesh *m, const double *h, double *zeta);

/* one SSPRK{2,3}-SE step, in place on (u, h, tr); returns 0 or -1 (bad args) */
int om_sse_step(const om_mesh *m, const om_params *p, int order, double dt, int M,
                double *u, double *h, double *tr, om_aux *aux);

/* threads used by the OpenMP build of the oracle (ignored by the serial one) */
void om_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
