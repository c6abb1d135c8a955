/*
 * sse_oracle.c -- plain, slow FP64 CPU oracle of the SSPRK2-SE and SSPRK3-SE
 * multirate split-explicit schemes for the layered primitive equations.
 *
 * TEST INFRASTRUCTURE ONLY: called from tests/, from the smoke check and from
 * the benchmark's CPU-baseline leg.  No product code links it.  It shares no
 * source with the CUDA library.
 *
 * Everything is written in the order and notation of the paper:
 *   - layered equations and vertical operators        Sec. 2 (layered eqs)
 *   - baroclinic/barotropic split                      Eq. (BBspl), (bcl:btr:split)
 *   - Baroclinic_FEuler                                Algorithm 1
 *   - Barotropic_SSPRK2_Substep / SSPRK3_Substep       Algorithms 3 and 4
 *   - SSPRK2-SE / SSPRK3-SE steps                      Sec. 3.2, 3.3
 *   - SSH reconciliation                               Sec. 3.4
 * The horizontal (TRiSK) operators are not written out in the paper (Sec. 5
 * only cites the TRiSK scheme); they are the standard TRiSK definitions of
 * Thuburn et al. (2009) / Ringler et al. (2010).  Every array is
 * layer-fastest, X[i*L + k], k = 0 the top layer; interface k is the top of
 * layer k and interface L the bottom.
 *
 * Parity of each function is pinned by tests/test_oracle_*.py against
 * closed forms, invariants and brute-force cases.
 */
#include "sse_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Loops over mesh entities write only the entity's own outputs and read only
 * inputs, so built with -fopenmp (oracle/__init__.py builds a second library
 * that way) they run across threads with results bit-identical to the serial
 * build; without OpenMP the marker expands to nothing. */
#ifdef _OPENMP
#include <omp.h>
#define OMP_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OMP_FOR
#endif

/* threads of the OpenMP build (no effect in the serial build) */
void om_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

#define C1(e) (m->cellsOnEdge[2 * (e)])
#define C2(e) (m->cellsOnEdge[2 * (e) + 1])
#define V1(e) (m->verticesOnEdge[2 * (e)])
#define V2(e) (m->verticesOnEdge[2 * (e) + 1])

static double *vec(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

/* Partial bottom cells: a column i has kc(i) active layers; an edge is active
 * in the layers both its cells have (maxLevelEdgeTop in MPAS); the z-star
 * stretching of layer k of column i is its share of the column's rest
 * thickness.  Inactive layers hold h = 0, u = 0 and no tracer. */
static int kc(const om_mesh *m, int i) { return m->maxLevelCell ? m->maxLevelCell[i] : m->nLayers; }
static int ke(const om_mesh *m, int e) {
    int a = kc(m, C1(e)), b = kc(m, C2(e));
    return a < b ? a : b;
}
static double sfr(const om_mesh *m, int i, int k) {
    if (m->restThickness) return m->restThickness[(size_t)i * m->nLayers + k] / m->bottomDepth[i];
    return m->restThicknessFrac[k];
}

/* ======================================================================== */
/* TRiSK horizontal operators                                               */
/* ======================================================================== */

/* div_i(F) = (1/A_i) sum_{e in EC(i)} n_{e,i} l_e F_e, n_{e,i} = +1 if the edge
 * normal points out of cell i. */
void om_div(const om_mesh *m, int L, const double *F, double *out) {
    OMP_FOR
    for (int i = 0; i < m->nCells; i++)
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->nEdgesOnCell[i]; j++) {
                int e = m->edgesOnCell[i * m->maxEdges + j];
                double sign = (C1(e) == i) ? 1.0 : -1.0;
                s += sign * m->dvEdge[e] * F[(size_t)e * L + k];
            }
            out[(size_t)i * L + k] = s / m->areaCell[i];
        }
}

/* grad_e(phi) = (phi_c2 - phi_c1) / d_e */
void om_grad(const om_mesh *m, int L, const double *phi, double *out) {
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++)
        for (int k = 0; k < L; k++)
            out[(size_t)e * L + k] =
                (phi[(size_t)C2(e) * L + k] - phi[(size_t)C1(e) * L + k]) / m->dcEdge[e];
}

/* curl_v(u) = (1/A_v) sum_{e in EV(v)} t_{e,v} d_e u_e, t_{e,v} = +1 when the
 * edge normal circulates counter-clockwise around v (v = v2 of the edge). */
void om_curl(const om_mesh *m, int L, const double *u, double *out) {
    OMP_FOR
    for (int v = 0; v < m->nVertices; v++)
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < 3; j++) {
                int e = m->edgesOnVertex[3 * v + j];
                if (e < 0) continue;
                double sign = (V2(e) == v) ? 1.0 : -1.0;
                s += sign * m->dcEdge[e] * u[(size_t)e * L + k];
            }
            out[(size_t)v * L + k] = s / m->areaTriangle[v];
        }
}

/* tangential velocity u^t_e = (1/d_e) sum_{e'} w_{e,e'} l_{e'} u_{e'} along
 * t_e = k x n_e */
void om_tangential(const om_mesh *m, int L, const double *u, double *out) {
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++)
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->nEdgesOnEdge[e]; j++) {
                int ep = m->edgesOnEdge[e * m->maxEdges2 + j];
                s += m->weightsOnEdge[e * m->maxEdges2 + j] * m->dvEdge[ep] *
                     u[(size_t)ep * L + k];
            }
            out[(size_t)e * L + k] = s / m->dcEdge[e];
        }
}

/* K_i = (1/A_i) sum_{e in EC(i)} (l_e d_e / 4) u_e^2 */
void om_kinetic_energy(const om_mesh *m, int L, const double *u, double *out) {
    OMP_FOR
    for (int i = 0; i < m->nCells; i++)
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->nEdgesOnCell[i]; j++) {
                int e = m->edgesOnCell[i * m->maxEdges + j];
                double ue = u[(size_t)e * L + k];
                s += 0.25 * m->dvEdge[e] * m->dcEdge[e] * ue * ue;
            }
            out[(size_t)i * L + k] = s / m->areaCell[i];
        }
}

/* vector Laplacian, normal component: grad(div u) + k x grad(curl u)
 * = (delta_c2 - delta_c1)/d_e - (omega_v2 - omega_v1)/l_e */
void om_laplacian(const om_mesh *m, int L, const double *u, double *out) {
    double *delta = vec((size_t)m->nCells * L), *omega = vec((size_t)m->nVertices * L);
    om_div(m, L, u, delta);
    om_curl(m, L, u, omega);
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++)
        for (int k = 0; k < L; k++)
            out[(size_t)e * L + k] =
                (delta[(size_t)C2(e) * L + k] - delta[(size_t)C1(e) * L + k]) / m->dcEdge[e] -
                (omega[(size_t)V2(e) * L + k] - omega[(size_t)V1(e) * L + k]) / m->dvEdge[e];
    free(delta);
    free(omega);
}

/* del^4 u: the vector Laplacian applied twice (the hyperviscosity that
 * replaces nu_h del^2 u in the global setup, Sec. 2 remark on horizontal
 * dissipation) */
void om_biharmonic(const om_mesh *m, int L, const double *u, double *out) {
    double *l1 = vec((size_t)m->nEdges * L);
    om_laplacian(m, L, u, l1);
    /* del^2 u lives on the edge layers that exist (partial bottom cells) */
    if (L == m->nLayers)
        OMP_FOR
        for (int e = 0; e < m->nEdges; e++)
            for (int k = ke(m, e); k < L; k++) l1[(size_t)e * L + k] = 0.0;
    om_laplacian(m, L, l1, out);
    free(l1);
}

/* Coriolis tendency of a velocity x: normal component of -f k x x, in the
 * energy-neutral TRiSK form C_f(x)_e = (1/d_e) sum_{e'} w l_{e'} x_{e'} (f_e+f_{e'})/2 */
void om_coriolis(const om_mesh *m, int L, const double *x, double *out) {
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++)
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->nEdgesOnEdge[e]; j++) {
                int ep = m->edgesOnEdge[e * m->maxEdges2 + j];
                s += m->weightsOnEdge[e * m->maxEdges2 + j] * m->dvEdge[ep] *
                     x[(size_t)ep * L + k] * 0.5 * (m->fEdge[e] + m->fEdge[ep]);
            }
            out[(size_t)e * L + k] = s / m->dcEdge[e];
        }
}

/* centred edge thickness h_e = (h_c1 + h_c2)/2, 0 in layers where the edge is
 * not active (partial bottom cells) */
void om_edge_thickness(const om_mesh *m, int L, const double *h, double *out) {
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++) {
        int K = (L == m->nLayers) ? ke(m, e) : L;
        for (int k = 0; k < L; k++)
            out[(size_t)e * L + k] =
                k < K ? 0.5 * (h[(size_t)C1(e) * L + k] + h[(size_t)C2(e) * L + k]) : 0.0;
    }
}

/* kite-area-weighted vertex thickness over the ocean cells of the vertex that
 * are active in the layer (0 where none is) */
void om_vertex_thickness(const om_mesh *m, int L, const double *h, double *out) {
    OMP_FOR
    for (int v = 0; v < m->nVertices; v++)
        for (int k = 0; k < L; k++) {
            double s = 0.0, a = 0.0;
            for (int j = 0; j < 3; j++) {
                int c = m->cellsOnVertex[3 * v + j];
                if (c < 0) continue;
                if (L == m->nLayers && k >= kc(m, c)) continue;
                s += m->kiteAreasOnVertex[3 * v + j] * h[(size_t)c * L + k];
                a += m->kiteAreasOnVertex[3 * v + j];
            }
            out[(size_t)v * L + k] = a > 0.0 ? s / a : 0.0;
        }
}

/* potential-vorticity flux (energy-conserving TRiSK form):
 * Q_e = (1/d_e) sum_{e'} w_{e,e'} l_{e'} h_{e'} u_{e'} (q_e + q_{e'})/2,
 * q_v = (curl_v u + f_v)/h_v, q_e = (q_v1 + q_v2)/2.  It is the normal
 * component of -(omega + f) k x u. */
void om_pv_flux(const om_mesh *m, int L, const double *u, const double *h, double *out) {
    size_t EL = (size_t)m->nEdges * L, VL = (size_t)m->nVertices * L;
    double *omega = vec(VL), *hv = vec(VL), *he = vec(EL), *qe = vec(EL);
    om_curl(m, L, u, omega);
    om_vertex_thickness(m, L, h, hv);
    om_edge_thickness(m, L, h, he);
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++)
        for (int k = 0; k < L; k++) {
            int a = V1(e), b = V2(e);
            double ha = hv[(size_t)a * L + k], hb = hv[(size_t)b * L + k];
            double qa = ha > 0.0 ? (omega[(size_t)a * L + k] + m->fVertex[a]) / ha : 0.0;
            double qb = hb > 0.0 ? (omega[(size_t)b * L + k] + m->fVertex[b]) / hb : 0.0;
            qe[(size_t)e * L + k] = 0.5 * (qa + qb);
        }
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++)
        for (int k = 0; k < L; k++) {
            double s = 0.0;
            for (int j = 0; j < m->nEdgesOnEdge[e]; j++) {
                int ep = m->edgesOnEdge[e * m->maxEdges2 + j];
                s += m->weightsOnEdge[e * m->maxEdges2 + j] * m->dvEdge[ep] *
                     he[(size_t)ep * L + k] * u[(size_t)ep * L + k] * 0.5 *
                     (qe[(size_t)e * L + k] + qe[(size_t)ep * L + k]);
            }
            out[(size_t)e * L + k] = s / m->dcEdge[e];
        }
    free(omega);
    free(hv);
    free(he);
    free(qe);
}

/* ======================================================================== */
/* vertical pieces (Sec. 2, layered equations)                              */
/* ======================================================================== */

/* z-star vertical velocity at interfaces, w[i*(L+1) + k] (k = 0 surface,
 * k = K_i the column's bottom), from the thickness equation (layerthickness)
 * with dh_k/dt = s_k * d(sum_l h_l)/dt, s_k = rest-thickness fraction:
 *   w_K = 0,  w_k = w_{k+1} - div(h_e v)_k + s_k sum_l div(h_e v)_l,  w_0 = 0
 * (w = 0 below the bottom). */
void om_vertical_velocity(const om_mesh *m, const double *h, const double *v, double *w) {
    int L = m->nLayers;
    size_t EL = (size_t)m->nEdges * L, CL = (size_t)m->nCells * L;
    double *he = vec(EL), *F = vec(EL), *dv = vec(CL);
    om_edge_thickness(m, L, h, he);
    OMP_FOR
    for (size_t x = 0; x < EL; x++) F[x] = he[x] * v[x];
    om_div(m, L, F, dv);
    OMP_FOR
    for (int i = 0; i < m->nCells; i++) {
        int K = kc(m, i);
        double tot = 0.0;
        for (int k = 0; k < K; k++) tot += dv[(size_t)i * L + k];
        double *wi = w + (size_t)i * (L + 1);
        for (int k = K; k <= L; k++) wi[k] = 0.0;   /* the column's bottom and below */
        for (int k = K - 1; k >= 1; k--)
            wi[k] = wi[k + 1] - dv[(size_t)i * L + k] + sfr(m, i, k) * tot;
        wi[0] = 0.0;
    }
    free(he);
    free(F);
    free(dv);
}

/* linear equation of state, Eq. (eqstate): rho = rho_ref - alpha (T - T_ref)
 * + beta (S - S_ref); tracers are [nT][C][L] with T first, S second. */
void om_density(const om_mesh *m, const om_params *p, const double *tr, double *rho) {
    size_t CL = (size_t)m->nCells * m->nLayers;
    OMP_FOR
    for (size_t x = 0; x < CL; x++) {
        double r = p->eos_rho_ref - p->eos_alpha * (tr[x] - p->eos_T_ref);
        if (p->nTracers >= 2) r += p->eos_beta * (tr[CL + x] - p->eos_S_ref);
        rho[x] = r;
    }
}

/* hydrostatic pressure, Eq. (hydrocon), with p^s = 0:
 *   p_k = g (sum_{l<k} rho_l h_l + rho_k h_k / 2);
 * mid-layer height z_k = -H + sum_{l>k} h_l + h_k / 2. */
void om_pressure(const om_mesh *m, const om_params *p, const double *h, const double *rho,
                 double *pres, double *zmid) {
    int L = m->nLayers;
    OMP_FOR
    for (int i = 0; i < m->nCells; i++) {
        const double *hi = h + (size_t)i * L, *ri = rho + (size_t)i * L;
        double acc = 0.0;
        for (int k = 0; k < L; k++) {
            pres[(size_t)i * L + k] = p->g * (acc + 0.5 * ri[k] * hi[k]);
            acc += ri[k] * hi[k];
        }
        double below = 0.0;
        for (int k = L - 1; k >= 0; k--) {
            zmid[(size_t)i * L + k] = -m->bottomDepth[i] + below + 0.5 * hi[k];
            below += hi[k];
        }
    }
}

/* SSH from the layer thicknesses: zeta = sum_k h_k - H */
void om_ssh(const om_mesh *m, const double *h, double *zeta) {
    int L = m->nLayers;
    OMP_FOR
    for (int i = 0; i < m->nCells; i++) {
        double s = 0.0;
        for (int k = 0; k < L; k++) s += h[(size_t)i * L + k];
        zeta[i] = s - m->bottomDepth[i];
    }
}

/* ======================================================================== */
/* the split system                                                         */
/* ======================================================================== */

/* Eq. (BBspl): ubar = sum h_k u_k / sum h_k, utilde_k = u_k - ubar (edge h) */
void om_split(const om_mesh *m, const double *u, const double *h, double *ubar, double *ut) {
    int L = m->nLayers;
    double *he = vec((size_t)m->nEdges * L);
    om_edge_thickness(m, L, h, he);
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++) {
        double num = 0.0, den = 0.0;
        for (int k = 0; k < L; k++) {
            num += he[(size_t)e * L + k] * u[(size_t)e * L + k];
            den += he[(size_t)e * L + k];
        }
        ubar[e] = num / den;
        int K = ke(m, e);
        for (int k = 0; k < L; k++) ut[(size_t)e * L + k] = k < K ? u[(size_t)e * L + k] - ubar[e] : 0.0;
    }
    free(he);
}

/* Right-hand side of Algorithm 1, line 1:
 *   -f ut^perp + T^u(u) + D^u(u) + g grad(zeta)
 * with, per edge e and layer k,
 *   -f ut^perp           -> C_f(ut_k)
 *   -(curl u) u^perp     -> Q_k(u, h) - C_f(u_k)   (PV flux minus planetary part)
 *   -grad |u|^2 / 2      -> -grad(K_k)
 *   -(1/rho0) grad p_k   -> -(grad p_k + g rho_e grad z_k) / rho0 (layer form)
 *   -avg^m(w D_zt u)     -> -(w_k D_k + w_{k+1} D_{k+1}) / 2
 *   nu_h lap u           -> nu_h Laplacian
 *   D^u = D_zm(nu_v D_zt u) with wind stress tau/rho0 at the surface and
 *                           bottom drag c_drag |u| u at the bottom (Sec. 5)
 */
static void baroclinic_rhs(const om_mesh *m, const om_params *p, const double *u,
                           const double *ut, const double *zeta, const double *h,
                           const double *tr, double *rhs, int with_vvisc);

void om_baroclinic_rhs(const om_mesh *m, const om_params *p, const double *u, const double *ut,
                       const double *zeta, const double *h, const double *tr, double *rhs) {
    baroclinic_rhs(m, p, u, ut, zeta, h, tr, rhs, 1);
}

/* with_vvisc = 0 leaves out D^u (Algorithm 2 treats it implicitly) */
static void baroclinic_rhs(const om_mesh *m, const om_params *p, const double *u,
                           const double *ut, const double *zeta, const double *h,
                           const double *tr, double *rhs, int with_vvisc) {
    int L = m->nLayers;
    size_t EL = (size_t)m->nEdges * L, CL = (size_t)m->nCells * L;
    double *Q = vec(EL), *Cu = vec(EL), *Cut = vec(EL), *K = vec(CL), *gK = vec(EL);
    double *rho = vec(CL), *pres = vec(CL), *zmid = vec(CL), *gp = vec(EL), *gz = vec(EL);
    double *lap = vec(EL), *he = vec(EL), *w = vec((size_t)m->nCells * (L + 1));
    double *utan = vec(EL), *gzeta = vec(m->nEdges), *del4 = vec(EL);

    om_pv_flux(m, L, u, h, Q);
    om_coriolis(m, L, u, Cu);
    om_coriolis(m, L, ut, Cut);
    om_kinetic_energy(m, L, u, K);
    om_grad(m, L, K, gK);
    om_density(m, p, tr, rho);
    /* pressure-gradient force in the anomaly form: with rho = rho_ref + rho'
     * and zeta = sum h - H, Eq. (hydrocon) gives p_k = g rho_ref (zeta - z_k)
     * + p'_k (p' the pressure of rho'), so
     *   grad p_k + g rho_e grad z_k = g rho_ref grad zeta + grad p'_k + g rho'_e grad z_k.
     * Both forms are the same quantity; this one avoids cancelling two terms
     * of size g rho grad z over sloping bathymetry. */
    OMP_FOR
    for (size_t x = 0; x < CL; x++) rho[x] -= p->eos_rho_ref;
    om_pressure(m, p, h, rho, pres, zmid);
    om_grad(m, L, pres, gp);
    om_grad(m, L, zmid, gz);
    om_laplacian(m, L, u, lap);
    if (p->nu_4 != 0.0) om_biharmonic(m, L, u, del4);
    om_edge_thickness(m, L, h, he);
    om_vertical_velocity(m, h, u, w);
    om_tangential(m, L, u, utan);
    om_grad(m, 1, zeta, gzeta);

    OMP_FOR
    for (int e = 0; e < m->nEdges; e++) {
        int c1 = C1(e), c2 = C2(e), K = ke(m, e);
        const double *ue = u + (size_t)e * L, *hee = he + (size_t)e * L;
        for (int k = K; k < L; k++) rhs[(size_t)e * L + k] = 0.0;   /* below the edge's bottom */
        /* interface values: D_zt(u)_k and w_k at the edge, k = 0..K */
        for (int k = 0; k < K; k++) {
            size_t x = (size_t)e * L + k;
            double Dk = 0.0, Dk1 = 0.0, wk = 0.0, wk1 = 0.0;
            if (k >= 1) {
                Dk = (ue[k - 1] - ue[k]) / (0.5 * (hee[k - 1] + hee[k]));
                wk = 0.5 * (w[(size_t)c1 * (L + 1) + k] + w[(size_t)c2 * (L + 1) + k]);
            }
            if (k + 1 <= K - 1) {
                Dk1 = (ue[k] - ue[k + 1]) / (0.5 * (hee[k] + hee[k + 1]));
                wk1 = 0.5 * (w[(size_t)c1 * (L + 1) + k + 1] + w[(size_t)c2 * (L + 1) + k + 1]);
            }
            double vadv = 0.5 * (wk * Dk + wk1 * Dk1);
            /* viscous fluxes at the top (X_top) and bottom (X_bot) of layer k */
            double Xtop, Xbot;
            if (k == 0)
                Xtop = p->windStress ? p->windStress[e] / p->rho0 : 0.0;
            else
                Xtop = p->nu_v * Dk;
            if (k == K - 1) {
                double speed = sqrt(ue[k] * ue[k] + utan[x] * utan[x]);
                Xbot = p->c_drag * speed * ue[k];
            } else {
                Xbot = p->nu_v * Dk1;
            }
            double vvisc = with_vvisc ? (Xtop - Xbot) / hee[k] : 0.0;
            double rhoa_e = 0.5 * (rho[(size_t)c1 * L + k] + rho[(size_t)c2 * L + k]);
            double pgf = (p->g * p->eos_rho_ref * gzeta[e] + gp[x] + p->g * rhoa_e * gz[x]) / p->rho0;
            rhs[x] = Cut[x] + (Q[x] - Cu[x]) - gK[x] - pgf - vadv + p->nu_h * lap[x] + vvisc +
                     p->g * gzeta[e] - p->nu_4 * del4[x];
        }
    }
    free(Q); free(Cu); free(Cut); free(K); free(gK); free(rho); free(pres); free(zmid);
    free(gp); free(gz); free(lap); free(he); free(w); free(utan); free(gzeta); free(del4);
}

/* Algorithm 1, Baroclinic_FEuler(u, ut, zeta, h, dt) -> (ut1, G) */
void om_baroclinic_feuler(const om_mesh *m, const om_params *p, const double *u,
                          const double *ut, const double *zeta, const double *h,
                          const double *tr, double dt, double *ut1, double *G) {
    int L = m->nLayers;
    size_t EL = (size_t)m->nEdges * L;
    double *rhs = vec(EL), *he = vec(EL);
    om_baroclinic_rhs(m, p, u, ut, zeta, h, tr, rhs);
    om_edge_thickness(m, L, h, he);
    OMP_FOR
    for (size_t x = 0; x < EL; x++) ut1[x] = ut[x] + dt * rhs[x];
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++) {
        double num = 0.0, den = 0.0;
        for (int k = 0; k < L; k++) {
            num += he[(size_t)e * L + k] * ut1[(size_t)e * L + k];
            den += he[(size_t)e * L + k];
        }
        G[e] = num / den / dt;
        int K = ke(m, e);
        for (int k = 0; k < K; k++) ut1[(size_t)e * L + k] -= dt * G[e];
    }
    free(rhs);
    free(he);
}

/* Implicit vertical diffusion, the solve of Algorithm 2:
 *   x_k - dt D^u(x)_k = r_k,  D^u(x)_k = (X_k - X_{k+1}) / h_e,k,
 *   X_k = nu_v (x_{k-1} - x_k) / ((h_e,k-1 + h_e,k)/2) at interior interfaces,
 *   X_0 = tau_e / rho0 (wind stress, known), X_L = c_drag |u_drag| x_{L-1}
 * (bottom drag with the speed of u_drag, |u| = sqrt(u^2 + u_t^2) of the
 * bottom layer).  One tridiagonal system per edge column, solved by forward
 * elimination and back substitution (Thomas algorithm). */
void om_vertical_mixing_solve(const om_mesh *m, const om_params *p, const double *u_drag,
                              const double *h, const double *r, double dt, double *x) {
    int L = m->nLayers;
    size_t EL = (size_t)m->nEdges * L;
    double *he = vec(EL), *utan = vec(EL);
    double *lo = vec(L), *di = vec(L), *up = vec(L), *rr = vec(L), *cp = vec(L), *dp = vec(L);
    om_edge_thickness(m, L, h, he);
    om_tangential(m, L, u_drag, utan);
    for (int e = 0; e < m->nEdges; e++) {
        const double *hk = he + (size_t)e * L;
        const int K = ke(m, e);   /* the edge's active layers */
        for (int k = K; k < L; k++) x[(size_t)e * L + k] = 0.0;
        /* the matrix: lo_k x_{k-1} + di_k x_k + up_k x_{k+1} = rr_k */
        for (int k = 0; k < K; k++) {
            double a = 0.0, c = 0.0;
            if (k >= 1) a = dt * p->nu_v / (hk[k] * 0.5 * (hk[k - 1] + hk[k]));
            if (k + 1 <= K - 1) c = dt * p->nu_v / (hk[k] * 0.5 * (hk[k] + hk[k + 1]));
            lo[k] = -a;
            up[k] = -c;
            di[k] = 1.0 + a + c;
            rr[k] = r[(size_t)e * L + k];
        }
        if (p->windStress) rr[0] += dt * p->windStress[e] / p->rho0 / hk[0];
        {
            size_t xb = (size_t)e * L + (K - 1);
            double speed = sqrt(u_drag[xb] * u_drag[xb] + utan[xb] * utan[xb]);
            di[K - 1] += dt * p->c_drag * speed / hk[K - 1];
        }
        /* forward elimination */
        cp[0] = up[0] / di[0];
        dp[0] = rr[0] / di[0];
        for (int k = 1; k < K; k++) {
            double den = di[k] - lo[k] * cp[k - 1];
            cp[k] = up[k] / den;
            dp[k] = (rr[k] - lo[k] * dp[k - 1]) / den;
        }
        /* back substitution */
        x[(size_t)e * L + K - 1] = dp[K - 1];
        for (int k = K - 2; k >= 0; k--)
            x[(size_t)e * L + k] = dp[k] - cp[k] * x[(size_t)e * L + k + 1];
    }
    free(he); free(utan); free(lo); free(di); free(up); free(rr); free(cp); free(dp);
}

/* Algorithm 2, Baroclinic_FEuler_Mixing(u, ut, ubar, zeta, h, dt) -> (ut1, G):
 * the explicit stage of Algorithm 1 without D^u, G from it, then the
 * vertical diffusion solve on the whole velocity ut1 + ubar, and ut1 = u1 -
 * ubar (ubar: the stage's input barotropic velocity). */
void om_baroclinic_feuler_mixing(const om_mesh *m, const om_params *p, const double *u,
                                 const double *ut, const double *ubar, const double *zeta,
                                 const double *h, const double *tr, double dt, double *ut1,
                                 double *G) {
    int L = m->nLayers;
    size_t EL = (size_t)m->nEdges * L;
    double *rhs = vec(EL), *he = vec(EL), *r = vec(EL), *u1 = vec(EL);
    baroclinic_rhs(m, p, u, ut, zeta, h, tr, rhs, 0);
    om_edge_thickness(m, L, h, he);
    OMP_FOR
    for (size_t x = 0; x < EL; x++) ut1[x] = ut[x] + dt * rhs[x];
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++) {
        double num = 0.0, den = 0.0;
        for (int k = 0; k < L; k++) {
            num += he[(size_t)e * L + k] * ut1[(size_t)e * L + k];
            den += he[(size_t)e * L + k];
        }
        G[e] = num / den / dt;
        for (int k = 0; k < ke(m, e); k++) {
            ut1[(size_t)e * L + k] -= dt * G[e];
            r[(size_t)e * L + k] = ut1[(size_t)e * L + k] + ubar[e];
        }
    }
    om_vertical_mixing_solve(m, p, u, h, r, dt, u1);
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++)
        for (int k = 0; k < L; k++)
            ut1[(size_t)e * L + k] = k < ke(m, e) ? u1[(size_t)e * L + k] - ubar[e] : 0.0;
    free(rhs); free(he); free(r); free(u1);
}

/* the baroclinic stage of the step: Algorithm 1, or Algorithm 2 when mixing */
static void bcl_stage(const om_mesh *m, const om_params *p, const double *u, const double *ut,
                      const double *ubar, const double *zeta, const double *h, const double *tr,
                      double dt, double *ut1, double *G) {
    if (p->vmix)
        om_baroclinic_feuler_mixing(m, p, u, ut, ubar, zeta, h, tr, dt, ut1, G);
    else
        om_baroclinic_feuler(m, p, u, ut, zeta, h, tr, dt, ut1, G);
}

/* One forward-Euler stage of the barotropic mode, Eq. (eqtropic):
 *   ubar1 = ubar + tau (C_f(ubar) - g grad zeta + G)
 *   zeta1 = zeta - tau div(ubar (zeta + H)_e),  (zeta+H)_e centred.
 * `flux` returns ubar (zeta + H)_e, the flux this stage used. */
void om_barotropic_fe(const om_mesh *m, const om_params *p, const double *ubar,
                      const double *zeta, const double *G, double tau, double *ubar1,
                      double *zeta1, double *flux) {
    int E = m->nEdges, C = m->nCells;
    double *cf = vec(E), *gz = vec(E), *dv = vec(C);
    om_coriolis(m, 1, ubar, cf);
    om_grad(m, 1, zeta, gz);
    OMP_FOR
    for (int e = 0; e < E; e++) {
        double Hc1 = zeta[C1(e)] + m->bottomDepth[C1(e)];
        double Hc2 = zeta[C2(e)] + m->bottomDepth[C2(e)];
        flux[e] = ubar[e] * 0.5 * (Hc1 + Hc2);
    }
    om_div(m, 1, flux, dv);
    OMP_FOR
    for (int e = 0; e < E; e++) ubar1[e] = ubar[e] + tau * (cf[e] - p->g * gz[e] + G[e]);
    OMP_FOR
    for (int i = 0; i < C; i++) zeta1[i] = zeta[i] - tau * dv[i];
    free(cf);
    free(gz);
    free(dv);
}

/* Algorithm 3 (order 2) or Algorithm 4 (order 3): M sub-steps of length
 * dt/M with frozen G.  Returns ubar^{M/M}, the accumulated flux F^zeta of
 * Sec. 3.4 and (if zeta1 != NULL) the sub-cycle's own final SSH. */
void om_barotropic_substep(const om_mesh *m, const om_params *p, int order,
                           const double *ubar, const double *zeta, const double *G, double dt,
                           int M, double *ubar1, double *Fzeta, double *zeta1) {
    int E = m->nEdges, C = m->nCells;
    double tau = dt / M;
    double *u0 = vec(E), *z0 = vec(C);
    double *ua = vec(E), *za = vec(C), *ub = vec(E), *zb = vec(C), *uc = vec(E), *zc = vec(C);
    double *uh = vec(E), *zh = vec(C), *Fa = vec(E), *Fb = vec(E), *Fc = vec(E);
    memcpy(u0, ubar, sizeof(double) * E);
    memcpy(z0, zeta, sizeof(double) * C);
    for (int e = 0; e < E; e++) Fzeta[e] = 0.0;
    for (int j = 1; j <= M; j++) {
        /* hat{ubar}^{j/M}, hat{zeta}^{j/M} */
        om_barotropic_fe(m, p, u0, z0, G, tau, ua, za, Fa);
        /* hat{ubar}^{(j+1)/M}, hat{zeta}^{(j+1)/M} */
        om_barotropic_fe(m, p, ua, za, G, tau, ub, zb, Fb);
        if (order == 2) {
            OMP_FOR
            for (int e = 0; e < E; e++) {
                u0[e] = 0.5 * (u0[e] + ub[e]);
                Fzeta[e] += (Fa[e] + Fb[e]) / (2.0 * M);
            }
            OMP_FOR
            for (int i = 0; i < C; i++) z0[i] = 0.5 * (z0[i] + zb[i]);
        } else {
            /* hat{ubar}^{(j-1/2)/M} = 3/4 ubar^{(j-1)/M} + 1/4 hat{ubar}^{(j+1)/M} */
            OMP_FOR
            for (int e = 0; e < E; e++) uh[e] = 0.75 * u0[e] + 0.25 * ub[e];
            OMP_FOR
            for (int i = 0; i < C; i++) zh[i] = 0.75 * z0[i] + 0.25 * zb[i];
            /* hat{ubar}^{(j+1/2)/M} */
            om_barotropic_fe(m, p, uh, zh, G, tau, uc, zc, Fc);
            OMP_FOR
            for (int e = 0; e < E; e++) {
                u0[e] = u0[e] / 3.0 + 2.0 * uc[e] / 3.0;
                Fzeta[e] += (Fa[e] + Fb[e]) / (6.0 * M) + 2.0 * Fc[e] / (3.0 * M);
            }
            OMP_FOR
            for (int i = 0; i < C; i++) z0[i] = z0[i] / 3.0 + 2.0 * zc[i] / 3.0;
        }
    }
    memcpy(ubar1, u0, sizeof(double) * E);
    if (zeta1) memcpy(zeta1, z0, sizeof(double) * C);
    free(u0); free(z0); free(ua); free(za); free(ub); free(zb); free(uc); free(zc);
    free(uh); free(zh); free(Fa); free(Fb); free(Fc);
}

/* Forward-Euler thickness and tracer stage with transport velocity v:
 *   h1_k = h_k + dt T^h_k(h, v),  T^h_k = -div(h_e v)_k - (w_k - w_{k+1})
 *   (h phi)1_k = h phi + dt [ -div(h_e v phi_e)_k - (phibar^t_k w_k - phibar^t_{k+1} w_{k+1})
 *                + div(h_e kappa_h grad phi)_k + kappa_v (D_zt(phi)_k - D_zt(phi)_{k+1}) ]
 * (Eqs. layerthickness, tracer), phi_e centred, w from the same v. */
void om_thickness_tracer_fe(const om_mesh *m, const om_params *p, const double *h,
                            const double *tr, const double *v, double dt, double *h1,
                            double *tr1) {
    int L = m->nLayers;
    size_t EL = (size_t)m->nEdges * L, CL = (size_t)m->nCells * L;
    double *he = vec(EL), *F = vec(EL), *divF = vec(CL), *w = vec((size_t)m->nCells * (L + 1));
    double *Ft = vec(EL), *divFt = vec(CL), *gphi = vec(EL), *Fd = vec(EL), *divFd = vec(CL);
    om_edge_thickness(m, L, h, he);
    OMP_FOR
    for (size_t x = 0; x < EL; x++) F[x] = he[x] * v[x];
    om_div(m, L, F, divF);
    om_vertical_velocity(m, h, v, w);
    OMP_FOR
    for (int i = 0; i < m->nCells; i++)
        for (int k = 0; k < L; k++) {
            size_t x = (size_t)i * L + k;
            double wk = w[(size_t)i * (L + 1) + k], wk1 = w[(size_t)i * (L + 1) + k + 1];
            h1[x] = h[x] + dt * (-divF[x] - (wk - wk1));
        }
    for (int t = 0; t < p->nTracers; t++) {
        const double *phi = tr + (size_t)t * CL;
        double *phi1 = tr1 + (size_t)t * CL;
        OMP_FOR
        for (int e = 0; e < m->nEdges; e++)
            for (int k = 0; k < L; k++) {
                size_t x = (size_t)e * L + k;
                double phie = 0.5 * (phi[(size_t)C1(e) * L + k] + phi[(size_t)C2(e) * L + k]);
                Ft[x] = F[x] * phie;
            }
        om_div(m, L, Ft, divFt);
        om_grad(m, L, phi, gphi);
        OMP_FOR
        for (size_t x = 0; x < EL; x++) Fd[x] = he[x] * p->kappa_h * gphi[x];
        om_div(m, L, Fd, divFd);
        OMP_FOR
        for (int i = 0; i < m->nCells; i++) {
            const double *ph = phi + (size_t)i * L, *hi = h + (size_t)i * L;
            const double *wi = w + (size_t)i * (L + 1);
            const int K = kc(m, i);
            for (int k = K; k < L; k++) phi1[(size_t)i * L + k] = 0.0;   /* no water */
            for (int k = 0; k < K; k++) {
                size_t x = (size_t)i * L + k;
                double ftop = 0.0, fbot = 0.0, dtop = 0.0, dbot = 0.0;
                if (k >= 1) {
                    ftop = 0.5 * (ph[k - 1] + ph[k]) * wi[k];
                    dtop = (ph[k - 1] - ph[k]) / (0.5 * (hi[k - 1] + hi[k]));
                }
                if (k + 1 <= K - 1) {
                    fbot = 0.5 * (ph[k] + ph[k + 1]) * wi[k + 1];
                    dbot = (ph[k] - ph[k + 1]) / (0.5 * (hi[k] + hi[k + 1]));
                }
                double hphi = hi[k] * ph[k] +
                              dt * (-divFt[x] - (ftop - fbot) + divFd[x] + p->kappa_v * (dtop - dbot));
                phi1[x] = hphi / h1[x];
            }
        }
    }
    free(he); free(F); free(divF); free(w); free(Ft); free(divFt); free(gphi); free(Fd);
    free(divFd);
}

/* ======================================================================== */
/* SSPRK2-SE and SSPRK3-SE steps with SSH reconciliation                    */
/* ======================================================================== */

/* x = a*x1 + b*x2, elementwise */
static void comb(size_t n, double a, const double *x1, double b, const double *x2, double *x) {
    OMP_FOR
    for (size_t i = 0; i < n; i++) x[i] = a * x1[i] + b * x2[i];
}

/* convex combination of thickness-weighted tracers:
 * phi = (a h1 phi1 + b h2 phi2) / h, h = a h1 + b h2 (already formed) */
static void comb_tracer(size_t CL, int nT, double a, const double *h1, const double *p1, double b,
                        const double *h2, const double *p2, const double *h, double *phi) {
    for (int t = 0; t < nT; t++)
        OMP_FOR
        for (size_t x = 0; x < CL; x++) {
            size_t y = (size_t)t * CL + x;
            phi[y] = h[x] > 0.0 ? (a * h1[x] * p1[y] + b * h2[x] * p2[y]) / h[x] : 0.0;
        }
}

/* sum over layers of u_k * h_e,k and of h_e,k at every edge */
static void layer_flux(const om_mesh *m, const double *u, const double *h, double *Fh,
                       double *hs) {
    int L = m->nLayers;
    double *he = vec((size_t)m->nEdges * L);
    om_edge_thickness(m, L, h, he);
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++) {
        double f = 0.0, s = 0.0;
        for (int k = 0; k < L; k++) {
            f += u[(size_t)e * L + k] * he[(size_t)e * L + k];
            s += he[(size_t)e * L + k];
        }
        if (Fh) Fh[e] = f;
        if (hs) hs[e] = s;
    }
    free(he);
}

/* transport velocity v_k = u_k + c * D / hs (c = 0 when reconciliation is off) */
static void transport(const om_mesh *m, int recon, const double *u, const double *D,
                      const double *hs, double c, double *v) {
    int L = m->nLayers;
    OMP_FOR
    for (int e = 0; e < m->nEdges; e++) {
        double uA = recon ? c * D[e] / hs[e] : 0.0;
        int K = ke(m, e);
        for (int k = 0; k < L; k++) v[(size_t)e * L + k] = k < K ? u[(size_t)e * L + k] + uA : 0.0;
    }
}

static void cp_opt(double *dst, const double *src, size_t n) {
    if (dst) memcpy(dst, src, n * sizeof(double));
}

int om_sse_step(const om_mesh *m, const om_params *p, int order, double dt, int M, double *u,
                double *h, double *tr, om_aux *aux) {
    if ((order != 2 && order != 3) || !(dt > 0.0) || M < 1) return -1;
    int L = m->nLayers, E = m->nEdges, C = m->nCells, nT = p->nTracers;
    size_t EL = (size_t)E * L, CL = (size_t)C * L, TL = (size_t)nT * CL;
    double *zeta_n = vec(C), *ubar_n = vec(E), *ut_n = vec(EL);
    double *ut1 = vec(EL), *ut2 = vec(EL), *ut3 = vec(EL), *uth = vec(EL), *utn1 = vec(EL);
    double *G0 = vec(E), *G1 = vec(E), *G2 = vec(E), *Gi = vec(E);
    double *ubar1 = vec(E), *ubar2 = vec(E), *ubarh = vec(E), *ubarn1 = vec(E);
    double *Fz1 = vec(E), *Fz2 = vec(E), *Fz3 = vec(E), *Fh1 = vec(E), *Fh2 = vec(E);
    double *Fh3 = vec(E), *D1 = vec(E), *D2 = vec(E), *D3 = vec(E);
    double *hs_n = vec(E), *hs_1 = vec(E), *hs_h = vec(E);
    double *u1 = vec(EL), *uh = vec(EL), *un1 = vec(EL), *v = vec(EL);
    double *h1 = vec(CL), *h2 = vec(CL), *hh = vec(CL), *h3 = vec(CL);
    double *tr1 = vec(TL), *tr2 = vec(TL), *trh = vec(TL), *tr3 = vec(TL);
    double *zeta1 = vec(C), *zetah = vec(C), *zsub = vec(C), *he_n = vec(EL), *he_1 = vec(EL);
    double *he_h = vec(EL);

    /* Preprocessing: ubar^n, utilde^n by Eq. (BBspl) */
    om_ssh(m, h, zeta_n);
    om_split(m, u, h, ubar_n, ut_n);

    if (order == 2) {
        /* Stage 1 of SSPRK2-SE */
        bcl_stage(m, p, u, ut_n, ubar_n, zeta_n, h, tr, dt, ut1, G0);
        om_barotropic_substep(m, p, 2, ubar_n, zeta_n, G0, dt, M, ubar1, Fz1, NULL);
        OMP_FOR
        for (int e = 0; e < E; e++)
            for (int k = 0; k < L; k++) u1[(size_t)e * L + k] = k < ke(m, e) ? ubar1[e] + ut1[(size_t)e * L + k] : 0.0;
        layer_flux(m, u, h, Fh1, hs_n);
        for (int e = 0; e < E; e++) D1[e] = Fz1[e] - Fh1[e];
        transport(m, p->recon, u, D1, hs_n, 1.0, v);
        om_thickness_tracer_fe(m, p, h, tr, v, dt, h1, tr1);
        om_ssh(m, h1, zeta1);
        /* Stage 2 (baroclinic) */
        bcl_stage(m, p, u1, ut1, ubar1, zeta1, h1, tr1, dt, ut2, G1);
        comb(EL, 0.5, ut_n, 0.5, ut2, utn1);
        /* Step 2: corrector with Interp_2(G0, G1), Eq. (force2) */
        comb(E, 0.5, G0, 0.5, G1, Gi);
        om_barotropic_substep(m, p, 2, ubar_n, zeta_n, Gi, dt, M, ubarn1, Fz2, zsub);
        OMP_FOR
        for (int e = 0; e < E; e++)
            for (int k = 0; k < L; k++)
                un1[(size_t)e * L + k] = k < ke(m, e) ? ubarn1[e] + utn1[(size_t)e * L + k] : 0.0;
        /* Step 3: thickness stage 2 with reconciliation, F^h_2 of Sec. 3.4 */
        layer_flux(m, un1, h1, Fh2, hs_1);
        for (int e = 0; e < E; e++) {
            double a = (p->recon == 2) ? Fz1[e] : Fh1[e];
            Fh2[e] = 0.5 * (a + Fh2[e]);
            D2[e] = Fz2[e] - Fh2[e];
        }
        transport(m, p->recon, un1, D2, hs_1, 2.0, v);
        om_thickness_tracer_fe(m, p, h1, tr1, v, dt, h2, tr2);
        comb(CL, 0.5, h, 0.5, h2, hh);
        comb_tracer(CL, nT, 0.5, h, tr, 0.5, h2, tr2, hh, trh);
        memcpy(u, un1, EL * sizeof(double));
        memcpy(h, hh, CL * sizeof(double));
        memcpy(tr, trh, TL * sizeof(double));
        if (aux) {
            cp_opt(aux->D1, D1, E); cp_opt(aux->D2, D2, E);
            cp_opt(aux->Fz1, Fz1, E); cp_opt(aux->Fz2, Fz2, E);
            cp_opt(aux->G0, G0, E); cp_opt(aux->G1, G1, E);
        }
    } else {
        /* Stage 1 of SSPRK3-SE */
        bcl_stage(m, p, u, ut_n, ubar_n, zeta_n, h, tr, dt, ut1, G0);
        om_barotropic_substep(m, p, 3, ubar_n, zeta_n, G0, dt, M, ubar1, Fz1, NULL);
        OMP_FOR
        for (int e = 0; e < E; e++)
            for (int k = 0; k < L; k++) u1[(size_t)e * L + k] = k < ke(m, e) ? ubar1[e] + ut1[(size_t)e * L + k] : 0.0;
        layer_flux(m, u, h, Fh1, hs_n);
        for (int e = 0; e < E; e++) D1[e] = Fz1[e] - Fh1[e];
        transport(m, p->recon, u, D1, hs_n, 1.0, v);
        om_thickness_tracer_fe(m, p, h, tr, v, dt, h1, tr1);
        om_ssh(m, h1, zeta1);
        /* Stage 2 */
        bcl_stage(m, p, u1, ut1, ubar1, zeta1, h1, tr1, dt, ut2, G1);
        comb(EL, 0.75, ut_n, 0.25, ut2, uth);
        om_barotropic_substep(m, p, 3, ubar1, zeta1, G1, dt, M, ubar2, Fz2, NULL);
        comb(E, 0.75, ubar_n, 0.25, ubar2, ubarh);
        OMP_FOR
        for (int e = 0; e < E; e++)
            for (int k = 0; k < L; k++) uh[(size_t)e * L + k] = k < ke(m, e) ? ubarh[e] + uth[(size_t)e * L + k] : 0.0;
        layer_flux(m, u1, h1, Fh2, hs_1);
        for (int e = 0; e < E; e++) D2[e] = Fz2[e] - Fh2[e];
        transport(m, p->recon, u1, D2, hs_1, 1.0, v);
        om_thickness_tracer_fe(m, p, h1, tr1, v, dt, h2, tr2);
        comb(CL, 0.75, h, 0.25, h2, hh);
        comb_tracer(CL, nT, 0.75, h, tr, 0.25, h2, tr2, hh, trh);
        om_ssh(m, hh, zetah);
        /* Stage 3 (baroclinic) */
        bcl_stage(m, p, uh, uth, ubarh, zetah, hh, trh, dt, ut3, G2);
        comb(EL, 1.0 / 3.0, ut_n, 2.0 / 3.0, ut3, utn1);
        /* Step 2: corrector with Interp_3(G0, G1, G_{1/2}), Eq. (force3) */
        for (int e = 0; e < E; e++) Gi[e] = G0[e] / 6.0 + G1[e] / 6.0 + 2.0 * G2[e] / 3.0;
        om_barotropic_substep(m, p, 3, ubar_n, zeta_n, Gi, dt, M, ubarn1, Fz3, zsub);
        OMP_FOR
        for (int e = 0; e < E; e++)
            for (int k = 0; k < L; k++)
                un1[(size_t)e * L + k] = k < ke(m, e) ? ubarn1[e] + utn1[(size_t)e * L + k] : 0.0;
        /* Step 3: F^h_3 of Sec. 3.4, layer by layer */
        om_edge_thickness(m, L, h, he_n);
        om_edge_thickness(m, L, h1, he_1);
        om_edge_thickness(m, L, hh, he_h);
        OMP_FOR
        for (int e = 0; e < E; e++) {
            double s = 0.0, hs = 0.0;
            for (int k = 0; k < L; k++) {
                size_t x = (size_t)e * L + k;
                double a = u[x] * he_n[x], b = u1[x] * he_1[x];
                if (p->recon == 2) { a = 0.0; b = 0.0; }
                s += (a + b + 2.0 * (u[x] + un1[x]) * he_h[x]) / 6.0;
                hs += he_h[x];
            }
            if (p->recon == 2) s += (Fz1[e] + Fz2[e]) / 6.0;
            Fh3[e] = s;
            hs_h[e] = hs;
            D3[e] = Fz3[e] - Fh3[e];
        }
        OMP_FOR
        for (int e = 0; e < E; e++)
            for (int k = 0; k < L; k++) {
                size_t x = (size_t)e * L + k;
                v[x] = k < ke(m, e) ? 0.5 * (u[x] + un1[x]) + (p->recon ? 1.5 * D3[e] / hs_h[e] : 0.0)
                                    : 0.0;
            }
        om_thickness_tracer_fe(m, p, hh, trh, v, dt, h3, tr3);
        double *hn1 = h2; /* reuse */
        comb(CL, 1.0 / 3.0, h, 2.0 / 3.0, h3, hn1);
        double *trn1 = tr2;
        comb_tracer(CL, nT, 1.0 / 3.0, h, tr, 2.0 / 3.0, h3, tr3, hn1, trn1);
        memcpy(u, un1, EL * sizeof(double));
        memcpy(h, hn1, CL * sizeof(double));
        memcpy(tr, trn1, TL * sizeof(double));
        if (aux) {
            cp_opt(aux->D1, D1, E); cp_opt(aux->D2, D2, E); cp_opt(aux->D3, D3, E);
            cp_opt(aux->Fz1, Fz1, E); cp_opt(aux->Fz2, Fz2, E); cp_opt(aux->Fz3, Fz3, E);
            cp_opt(aux->G0, G0, E); cp_opt(aux->G1, G1, E); cp_opt(aux->G2, G2, E);
        }
    }
    if (aux) cp_opt(aux->zeta_sub, zsub, C);

    free(zeta_n); free(ubar_n); free(ut_n); free(ut1); free(ut2); free(ut3); free(uth);
    free(utn1); free(G0); free(G1); free(G2); free(Gi); free(ubar1); free(ubar2); free(ubarh);
    free(ubarn1); free(Fz1); free(Fz2); free(Fz3); free(Fh1); free(Fh2); free(Fh3); free(D1);
    free(D2); free(D3); free(hs_n); free(hs_1); free(hs_h); free(u1); free(uh); free(un1);
    free(v); free(h1); free(h2); free(hh); free(h3); free(tr1); free(tr2); free(trh);
    free(tr3); free(zeta1); free(zetah); free(zsub); free(he_n); free(he_1); free(he_h);
    return 0;
}
