// stage_kernels.cu -- 3-D kernels of one SSPRK-SE stage (sm_103a).
//
// One thread owns one column (cell, vertex or edge) and walks its layers from
// the top; column sums (thickness-weighted means, pressure, vertical velocity)
// are therefore sequential in k, in the same order as the definitions.  All
// arrays are layer-major, so at every k a warp reads 32 consecutive columns.
//
//   cell_diag  : per cell and layer  K, div u, rho', p', z_mid and the z-star w
//                (Sec. 2: layered equations, Eqs. hydrocon, eqstate)
//   vertex     : relative vorticity and potential vorticity q = (omega+f)/h_v
//   edge_pre   : edge mass flux h_e u and q_e; at stage 1 also Eq. (BBspl)
//   bcl_edge   : Algorithm 1 (Baroclinic_FEuler) with the SSPRK convex
//                combination of the stage
//   transport  : Sec. 3.4 flux deficit D = F^zeta - F^h, transport velocity
//                adjustment u^A and the edge mass flux h_e (u + u^A)
//   thickness  : thickness and tracer forward-Euler stage (Eqs. layerthickness,
//                tracer) with the convex combination and zeta = sum h - H
#include "sse_internal.cuh"

namespace sse {

template <class R> __device__ __forceinline__ R ld(const R *p) { return __ldg(p); }

template <class R> __device__ __forceinline__ const R *sfrac_of(const DMesh &m);
template <> __device__ __forceinline__ const double *sfrac_of<double>(const DMesh &m) { return m.sfrac; }
template <> __device__ __forceinline__ const float *sfrac_of<float>(const DMesh &m) { return m.sfrac_f; }
// per-column shares (partial bottom cells), [L][Cp]
template <class R> __device__ __forceinline__ const R *sfc_of(const DMesh &m);
template <> __device__ __forceinline__ const double *sfc_of<double>(const DMesh &m) { return m.sfc; }
template <> __device__ __forceinline__ const float *sfc_of<float>(const DMesh &m) { return m.sfc_f; }

// ---------------------------------------------------------------------------
// cell diagnostics
// ---------------------------------------------------------------------------
// PB: partial bottom cells -- the column's own layer count K and per-edge
// layer counts; u is 0 on edge layers that do not exist.
template <class R, int NCE, bool PB>
__global__ void __launch_bounds__(128) k_cell_diag(DMesh m, DParams p, const R *__restrict__ ubar,
                                                   const R *__restrict__ ut,
                                                   const R *__restrict__ hR,
                                                   const R *__restrict__ tr, DiagBufs<R> b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.C) return;
    const Coef<R> &c = coef<R>(m);
    const int Cp = m.Cp, Ep = m.Ep, L = m.L;
    const int ne = m.neoc[i];
    const int K = PB ? m.kc[i] : L;
    int es[NCE], os[NCE], kej[NCE];
    R dcf[NCE], kcf[NCE], ub[NCE];
#pragma unroll
    for (int j = 0; j < NCE; j++) {
        if (j < ne) {
            es[j] = m.eoc[j * Cp + i];
            os[j] = m.ooc[j * Cp + i];
            dcf[j] = c.divc[j * Cp + i];
            kcf[j] = c.kec[j * Cp + i];
            ub[j] = ld(ubar + es[j]);
            kej[j] = PB ? m.ke[es[j]] : L;
        } else {
            es[j] = 0; os[j] = i; dcf[j] = R(0); kcf[j] = R(0); ub[j] = R(0); kej[j] = 0;
        }
    }
    const PhysR<R> &q = phys<R>(p);
    const R g = q.g, alpha = q.alpha, beta = q.beta, Tref = q.T_ref, Sref = q.S_ref;
    const R *sfr = sfrac_of<R>(m);
    const R *sfc = sfc_of<R>(m);
    R accp = R(0), divsum = R(0);
    for (int k = 0; k < K; k++) {
        const R hk = ld(hR + k * Cp + i);
        R ke = R(0), dl = R(0), dv = R(0);
#pragma unroll
        for (int j = 0; j < NCE; j++) {
            if (j < ne && (!PB || k < kej[j])) {
                const R uk = ub[j] + ld(ut + k * Ep + es[j]);
                const R he = R(0.5) * (hk + ld(hR + k * Cp + os[j]));
                ke += kcf[j] * uk * uk;
                dl += dcf[j] * uk;
                dv += dcf[j] * (he * uk);
            }
        }
        R rp = -alpha * (ld(tr + k * Cp + i) - Tref);
        if (p.nT > 1) rp += beta * (ld(tr + (L + k) * Cp + i) - Sref);
        const int x = k * Cp + i;
        V4<R> cq;
        cq.x = ke;
        cq.y = g * (accp + R(0.5) * rp * hk);
        cq.z = rp;
        cq.w = R(0);    // z_mid, filled in on the way up
        b.cq[x] = cq;
        b.delta[x] = dl;
        accp += rp * hk;
        b.w[x] = dv;  // divergence of h_e u, finalised below
        divsum += dv;
    }
    // bottom -> top: z-star vertical velocity at the top of each layer and the
    // mid-layer height z_k = -H + sum_{l>k} h_l + h_k / 2
    R wk1 = R(0), below = R(0);
    const R Hi = (R)m.H[i];
    for (int k = K - 1; k >= 0; k--) {
        const int x = k * Cp + i;
        const R hk = ld(hR + x);
        b.cq[x].w = -Hi + below + R(0.5) * hk;
        below += hk;
        const R sk = PB ? sfc[x] : sfr[k];
        const R wk = (k == 0) ? R(0) : wk1 - b.w[x] + sk * divsum;
        b.w[x] = wk;
        wk1 = wk;
    }
}

// ---------------------------------------------------------------------------
// vertex vorticity and potential vorticity
// ---------------------------------------------------------------------------
template <class R, bool PB>
__global__ void __launch_bounds__(128) k_vertex(DMesh m, const R *__restrict__ ubar,
                                                const R *__restrict__ ut,
                                                const R *__restrict__ hR, DiagBufs<R> b) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    const Coef<R> &c = coef<R>(m);
    const int Vp = m.Vp, Ep = m.Ep, Cp = m.Cp, L = m.L;
    int e[3], ce[3], kej[3], kcj[3];
    R cc[3], kw[3], ub[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        e[j] = m.eov[j * Vp + v];
        ce[j] = m.cov[j * Vp + v];
        cc[j] = c.curlc[j * Vp + v];
        kw[j] = c.kw[j * Vp + v];
        ub[j] = ld(ubar + e[j]);
        kej[j] = PB ? m.ke[e[j]] : L;
        kcj[j] = PB ? m.kc[ce[j]] : L;
    }
    const R fv = c.fV[v];
    for (int k = 0; k < L; k++) {
        R om = R(0), hv = R(0), ws = R(0);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (!PB || k < kej[j]) om += cc[j] * (ub[j] + ld(ut + k * Ep + e[j]));
            hv += kw[j] * ld(hR + k * Cp + ce[j]);
            if (PB && k < kcj[j]) ws += kw[j];
        }
        b.omega[k * Vp + v] = om;
        if (PB) {
            // kite average over the cells that have this layer; none: q = 0
            hv = ws > R(0) ? hv / ws : R(0);
            b.q[k * Vp + v] = hv > R(0) ? (om + fv) / hv : R(0);
        } else {
            b.q[k * Vp + v] = (om + fv) / hv;
        }
    }
}

// ---------------------------------------------------------------------------
// edge pre-pass: h_e u, q_e; optional barotropic/baroclinic split (Eq. BBspl)
// ---------------------------------------------------------------------------
template <class R, bool PB>
__global__ void __launch_bounds__(128) k_edge_pre(DMesh m, R *__restrict__ ubar, R *__restrict__ ut,
                                                  const R *__restrict__ hR, DiagBufs<R> b,
                                                  int split) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const int Ep = m.Ep, Cp = m.Cp, Vp = m.Vp;
    const int2 cc = m.coe[e], vv = m.voe[e];
    const Coef<R> &c = coef<R>(m);
    const R invdc = c.invdc[e], invdv = c.invdv[e];
    R ub = ubar[e];
    R mean = R(0);
    // the edge's own layers; the rest of its column stays 0 (u, h_e u, del^2 u)
    const int K = PB ? m.ke[e] : m.L;
    if (PB && split)
        for (int k = K; k < m.L; k++) ut[k * Ep + e] = R(0);
    if (split) {
        R num = R(0), den = R(0);
        for (int k = 0; k < K; k++) {
            const R he = R(0.5) * (ld(hR + k * Cp + cc.x) + ld(hR + k * Cp + cc.y));
            num += he * ut[k * Ep + e];
            den += he;
        }
        mean = num / den;
        ub += mean;
        ubar[e] = ub;
    }
    for (int k = 0; k < K; k++) {
        const int x = k * Ep + e;
        R utk = ut[x];
        if (split) {
            utk -= mean;
            ut[x] = utk;
        }
        const R he = R(0.5) * (ld(hR + k * Cp + cc.x) + ld(hR + k * Cp + cc.y));
        V2<R> hq;
        hq.x = he * (ub + utk);
        hq.y = R(0.5) * (b.q[k * Vp + vv.x] + b.q[k * Vp + vv.y]);
        b.hq[x] = hq;
        if (b.del2)   // del^2 u = grad(div u) - k x grad(curl u), normal component
            b.del2[x] = (b.delta[k * Cp + cc.y] - b.delta[k * Cp + cc.x]) * invdc -
                        (b.omega[k * Vp + vv.y] - b.omega[k * Vp + vv.x]) * invdv;
    }
}

// Divergence (cells, items [0, C)) and curl (vertices, items [C, C + V)) of
// del^2 u, the inputs of del^4 u = del^2(del^2 u) in the baroclinic kernel.
template <class R, int NCE>
__global__ void __launch_bounds__(128) k_del2_divcurl(DMesh m, DiagBufs<R> b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const Coef<R> &c = coef<R>(m);
    const int Cp = m.Cp, Ep = m.Ep, Vp = m.Vp, L = m.L;
    if (t < m.C) {
        const int i = t, ne = m.neoc[i];
        int es[NCE];
        R dcf[NCE];
#pragma unroll
        for (int j = 0; j < NCE; j++) {
            es[j] = j < ne ? m.eoc[j * Cp + i] : 0;
            dcf[j] = j < ne ? c.divc[j * Cp + i] : R(0);
        }
        for (int k = 0; k < L; k++) {
            R d = R(0);
#pragma unroll
            for (int j = 0; j < NCE; j++)
                if (j < ne) d += dcf[j] * ld(b.del2 + k * Ep + es[j]);
            b.delta2[k * Cp + i] = d;
        }
    } else if (t < m.C + m.V) {
        const int v = t - m.C;
        int e[3];
        R cc[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            e[j] = m.eov[j * Vp + v];
            cc[j] = c.curlc[j * Vp + v];
        }
        for (int k = 0; k < L; k++) {
            R om = R(0);
#pragma unroll
            for (int j = 0; j < 3; j++) om += cc[j] * ld(b.del2 + k * Ep + e[j]);
            b.omega2[k * Vp + v] = om;
        }
    }
}

// ---------------------------------------------------------------------------
// Algorithm 1: baroclinic forward Euler, G, and the stage's convex combination
//   ut1_k = ut_k + dt ( C_f(ut_k) + [Q_k - C_f(u_k)] - grad K_k - PGF_k
//                       - avg^m(w D_zt u)_k + nu_h Lap u_k + D^u_k + g grad zeta )
//   G = (1/dt) sum_k h_k ut1_k / sum_k h_k ;  ut1_k -= dt G
//   out_k = a * ut_n_k + bcoef * ut1_k
// C_f(ut_k) - C_f(u_k) = -C_f(ubar): one 2-D sum per column.
// PGF in anomaly form: with rho = rho_ref + rho' and p' = g(sum_{l<k} rho'_l h_l
// + rho'_k h_k / 2),  grad p + g rho_e grad z = g rho_ref grad zeta + grad p'
// + g rho'_e grad z, so -PGF + g grad zeta = g (1 - rho_ref/rho0) grad zeta
// - (grad p' + g rho'_e grad z) / rho0.
// ---------------------------------------------------------------------------
// VMIX = false: Algorithm 1.  VMIX = true: Algorithm 2 -- the explicit stage
// without D^u, G, then (I - dt D^u) u1 = ut1 + ubar solved down each edge
// column (Thomas; the modified super-diagonal goes to the scratch vmc), with
// the wind explicit at the top and the bottom drag linearised about the speed
// of the stage's input velocity; ut1 = u1 - ubar.
// MINB: resident blocks per SM the kernel is compiled for (registers 65536 /
// (128 x MINB)): 8 for short columns; 6 for deep ones, whose longer sliding
// window over the layers would otherwise spill (measured on the 20-layer
// channel and the 60-layer sphere).
template <class R, int NE2, bool VMIX, bool PB, int MINB>
__global__ void __launch_bounds__(128, MINB) k_bcl_edge(DMesh m, DParams p, const R *__restrict__ ubar,
                                                  const R *__restrict__ ut,
                                                  const R *__restrict__ hR,
                                                  const double *__restrict__ zeta, DiagBufs<R> b,
                                                  const R *__restrict__ ut_n, R a, R bc, R dt,
                                                  R *__restrict__ ut_out, R *__restrict__ Gout,
                                                  R *__restrict__ vmc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const Coef<R> &c = coef<R>(m);
    const int Ep = m.Ep, Cp = m.Cp, Vp = m.Vp, L = m.L;
    const int2 cc = m.coe[e], vv = m.voe[e];
    const int c1 = cc.x, c2 = cc.y, v1 = vv.x, v2 = vv.y;
    const int n2 = m.neoe[e];
    int eo[NE2];
    R wl[NE2];
    R cbar = R(0);
    int kmin = L;   // the first layer some neighbour lacks (partial bottom cells)
#pragma unroll
    for (int j = 0; j < NE2; j++) {
        if (j < n2) {
            eo[j] = m.eoe[j * Ep + e];
            wl[j] = c.wl[j * Ep + e];
            cbar += c.cfc[j * Ep + e] * ld(ubar + eo[j]);
            if (PB) kmin = min(kmin, m.ke[eo[j]]);
        } else {
            eo[j] = e; wl[j] = R(0);
        }
    }
    const R invdc = c.invdc[e], invdv = c.invdv[e];
    const R ub = ubar[e];
    const PhysR<R> &q = phys<R>(p);
    const R dzeta = (R)(zeta[c2] - zeta[c1]);   // the difference taken in FP64
    const R gzeta = q.zcoef * dzeta * invdc;
    const R g = q.g, inv_rho0 = q.inv_rho0, nu_h = q.nu_h, nu_v = q.nu_v, nu_4 = q.nu_4;
    const R cdrag = q.c_drag;
    const R *wnd = wind_over_rho0<R>(p);
    const R wind = wnd ? wnd[e] : R(0);

    // the edge's own layers (partial bottom cells); below them nothing is written
    const int K = PB ? m.ke[e] : L;
    R ut_cur = ut[e];
    R u_cur = ub + ut_cur;
    R h1_cur = ld(hR + c1), h2_cur = ld(hR + c2);
    R he_cur = R(0.5) * (h1_cur + h2_cur);
    // pressure gradient from differences across the edge accumulated down the
    // column: dA = sum_{l<k} (rho' h)_c2 - (rho' h)_c1, dH = sum_{l<k} h_c2 - h_c1
    R dA = R(0), dH = R(0);
    // the top interface of layer k is the bottom interface of layer k - 1: its
    // shear D_zt(u) and edge w carry over from the previous layer (0 at k = 0)
    R Dk = R(0), wk = R(0);
    R num = R(0), den = R(0), speed_b = R(0);
    for (int k = 0; k < K; k++) {
        const int xe = k * Ep + e;
        R ut_next = R(0), u_next = R(0), h1_next = R(0), h2_next = R(0);
        if (k + 1 < K) {
            ut_next = ut[xe + Ep];
            u_next = ub + ut_next;
            h1_next = ld(hR + (k + 1) * Cp + c1);
            h2_next = ld(hR + (k + 1) * Cp + c2);
        }
        const R he_next = R(0.5) * (h1_next + h2_next);
        // potential-vorticity flux
        const R qk = b.hq[xe].y;
        R Q = R(0);
#pragma unroll
        for (int j = 0; j < NE2; j++)
            if (j < n2) {
                const V2<R> nb = b.hq[k * Ep + eo[j]];
                Q += wl[j] * nb.x * (R(0.5) * (qk + nb.y));
            }
        const int x1 = k * Cp + c1, x2 = k * Cp + c2;
        const V4<R> A = b.cq[x1], B = b.cq[x2];    // (K, p', rho', z_mid) of both cells
        const R gradK = (B.x - A.x) * invdc;
        // p'_2 - p'_1 and z_2 - z_1 (z = zeta - sum_{l<k} h_l - h_k / 2), the
        // same quantities as the differences of the two columns' values (Eq.
        // hydrocon) without cancelling two O(g rho' H) sums
        const R rh = B.z * h2_cur - A.z * h1_cur;
        const R dp = g * (dA + R(0.5) * rh);
        const R dz = dzeta - dH - R(0.5) * (h2_cur - h1_cur);
        const R pgf = (dp + g * (R(0.5) * (A.z + B.z)) * dz) * invdc * inv_rho0;
        dA += rh;
        dH += h2_cur - h1_cur;
        // vertical advection and viscosity at the top (k) and bottom (k+1) interfaces
        R Dk1 = R(0), wk1 = R(0);
        if (k + 1 < K) {
            Dk1 = (u_cur - u_next) / (R(0.5) * (he_cur + he_next));
            wk1 = R(0.5) * (b.w[x1 + Cp] + b.w[x2 + Cp]);
        }
        const R vadv = R(0.5) * (wk * Dk + wk1 * Dk1);
        const R Xtop = (k == 0) ? wind : nu_v * Dk;
        R Xbot;
        if (k == K - 1) {
            R utan = R(0);
#pragma unroll
            for (int j = 0; j < NE2; j++)
                if (j < n2 && (!PB || k < m.ke[eo[j]]))
                    utan += wl[j] * (ld(ubar + eo[j]) + ut[k * Ep + eo[j]]);
            speed_b = sqrt(u_cur * u_cur + utan * utan);
            Xbot = cdrag * speed_b * u_cur;
        } else {
            Xbot = nu_v * Dk1;
        }
        const R vvisc = VMIX ? R(0) : (Xtop - Xbot) / he_cur;
        const R lap = (b.delta[x2] - b.delta[x1]) * invdc -
                      (b.omega[k * Vp + v2] - b.omega[k * Vp + v1]) * invdv;
        // C_f(u_k) - C_f(ut_k) = C_f(ubar) over the neighbours that have layer k
        R cb = cbar;
        if (PB && k >= kmin) {
            cb = R(0);
#pragma unroll
            for (int j = 0; j < NE2; j++)
                if (j < n2 && k < m.ke[eo[j]]) cb += c.cfc[j * Ep + e] * ld(ubar + eo[j]);
        }
        R rhs = (Q - cb) - gradK - pgf - vadv + nu_h * lap + vvisc + gzeta;
        if (b.del2)
            rhs -= nu_4 * ((b.delta2[x2] - b.delta2[x1]) * invdc -
                           (b.omega2[k * Vp + v2] - b.omega2[k * Vp + v1]) * invdv);
        const R ut1 = ut_cur + dt * rhs;
        num += he_cur * ut1;
        den += he_cur;
        ut_out[xe] = ut1;
        Dk = Dk1; wk = wk1;
        ut_cur = ut_next; u_cur = u_next; he_cur = he_next;
        h1_cur = h1_next; h2_cur = h2_next;
    }
    const R G = num / den / dt;
    Gout[e] = G;
    if (!VMIX) {
        for (int k = 0; k < K; k++) {
            const int xe = k * Ep + e;
            const R x = ut_out[xe] - dt * G;
            ut_out[xe] = ut_n ? a * ut_n[xe] + bc * x : bc * x;
        }
        return;
    }
    // forward elimination down the column: row k is
    //   -lo x_{k-1} + (1 + lo + up [+ dt c_d |u| / h]) x_k - up x_{k+1} = r_k
    R cprev = R(0), dprev = R(0), hprev = R(0);
    R hk = R(0.5) * (ld(hR + c1) + ld(hR + c2));
    for (int k = 0; k < K; k++) {
        const int xe = k * Ep + e;
        const R hnext = (k + 1 < K)
            ? R(0.5) * (ld(hR + (k + 1) * Cp + c1) + ld(hR + (k + 1) * Cp + c2)) : R(0);
        const R lo = (k > 0) ? dt * nu_v / (hk * (R(0.5) * (hprev + hk))) : R(0);
        const R up = (k + 1 < K) ? dt * nu_v / (hk * (R(0.5) * (hk + hnext))) : R(0);
        R di = R(1) + lo + up;
        if (k == K - 1) di += dt * cdrag * speed_b / hk;
        R r = ut_out[xe] - dt * G + ub;
        if (k == 0) r += dt * wind / hk;
        // sub-diagonal -lo, super-diagonal -up: pivot di - (-lo) c'_{k-1}
        const R dn = di + lo * cprev;
        cprev = -up / dn;
        dprev = (r + lo * dprev) / dn;
        vmc[xe] = cprev;
        ut_out[xe] = dprev;
        hprev = hk;
        hk = hnext;
    }
    // back substitution up the column, then the convex combination
    R xnext = R(0);
    for (int k = K - 1; k >= 0; k--) {
        const int xe = k * Ep + e;
        const R x = ut_out[xe] - vmc[xe] * xnext;
        xnext = x;
        const R u1 = x - ub;
        ut_out[xe] = ut_n ? a * ut_n[xe] + bc * u1 : bc * u1;
    }
}

// ---------------------------------------------------------------------------
// Sec. 3.4: transport velocity adjustment and edge mass flux
//   F^h = cF * sum_k v_k h_e,k + cE * (extra terms), D = F^zeta - F^h,
//   u^A = cA * D / sum_k h_e,k,  flux_k = h_e,k (v_k + u^A)
// The column sums that decide D, u^A and the column-integrated flux F_col are
// read out in FP64 (PairSum: a float pair in the mixed form);
// sum_k h_e,k = ((zeta+H)_c1 + (zeta+H)_c2) / 2 because zeta = sum h - H.  The
// per-layer flux is stored in the tendency precision.
// ---------------------------------------------------------------------------
template <class R, bool PB>
__global__ void __launch_bounds__(128) k_transport(DMesh m, TransportArgs<R> a) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.E) return;
    const int Ep = m.Ep, Cp = m.Cp, L = m.L;
    const int2 cc = m.coe[e];
    const R ubA = a.ubA[e];
    const R ubB = a.ubB ? a.ubB[e] : R(0);
    const R wA = (R)a.wA, wB = (R)a.wB;
    const bool twoB = a.utB != nullptr;
    // with full columns the edge's total thickness is (zeta + H)_e; with partial
    // bottom cells it is the sum over the layers the edge has
    const int K = PB ? m.ke[e] : L;
    PairSum<R> Sacc, hacc;
    for (int k = 0; k < K; k++) {
        const R he = R(0.5) * (ld(a.hR + k * Cp + cc.x) + ld(a.hR + k * Cp + cc.y));
        R v = wA * (ubA + a.utA[k * Ep + e]);
        if (twoB) v += wB * (ubB + a.utB[k * Ep + e]);
        Sacc.add(v * he);
        if (PB) hacc.add(he);
    }
    const double S = Sacc.value();
    const double hs =
        PB ? hacc.value() : 0.5 * ((a.zeta[cc.x] + m.H[cc.x]) + (a.zeta[cc.y] + m.H[cc.y]));
    double Fh = a.cF * S;
    if (a.ex1) Fh += a.cE * a.ex1[e];
    if (a.ex2) Fh += a.cE * a.ex2[e];
    const double uA = a.recon ? a.cA * (a.Fz[e] - Fh) / hs : 0.0;
    if (a.S_out) a.S_out[e] = S;
    a.Fcol[e] = S + uA * hs;
    const R uAr = (R)uA;
    for (int k = 0; k < K; k++) {
        const R he = R(0.5) * (ld(a.hR + k * Cp + cc.x) + ld(a.hR + k * Cp + cc.y));
        R v = wA * (ubA + a.utA[k * Ep + e]);
        if (twoB) v += wB * (ubB + a.utB[k * Ep + e]);
        a.flux[k * Ep + e] = he * (v + uAr);
    }
}

// ---------------------------------------------------------------------------
// thickness and tracer stage (Eqs. layerthickness, tracer), z-star w from the
// same flux, convex combination with (h^n, phi^n), zeta = sum h - H.
// With z-star, -div(h u)_k - (w_k - w_{k+1}) = -s_k sum_l div(h u)_l, so the
// FP64 thickness update needs only the column-integrated edge flux F_col
// (FP64, from k_transport); the per-layer flux feeds w and the tracers in the
// tendency precision.
// ---------------------------------------------------------------------------
template <class R, int NCE, bool PB>
__global__ void __launch_bounds__(128, 6) k_thickness(DMesh m, DParams p, ThickArgs<R> a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.C) return;
    const Coef<R> &c = coef<R>(m);
    const int Cp = m.Cp, Ep = m.Ep, L = m.L;
    const int ne = m.neoc[i];
    const int K = PB ? m.kc[i] : L;     // the column's layers; below them nothing is written
    int es[NCE], os[NCE], kej[NCE];
    R dcf[NCE], idc[NCE];
    double D = 0.0;
#pragma unroll
    for (int j = 0; j < NCE; j++) {
        if (j < ne) {
            es[j] = m.eoc[j * Cp + i];
            os[j] = m.ooc[j * Cp + i];
            dcf[j] = c.divc[j * Cp + i];
            idc[j] = c.invdc[es[j]];
            D += m.divc_d[j * Cp + i] * a.Fcol[es[j]];
            kej[j] = PB ? m.ke[es[j]] : L;
        } else {
            es[j] = 0; os[j] = i; dcf[j] = R(0); idc[j] = R(0); kej[j] = 0;
        }
    }
    const R Dr = (R)D;
    const double dtD = a.dt * D;
    const PhysR<R> &q = phys<R>(p);
    const R *sfr = sfrac_of<R>(m);
    const R *sfcR = sfc_of<R>(m);
    const R dtR = (R)a.dt, aR = (R)a.a, bR = (R)a.b, kh = q.kappa_h, kv = q.kappa_v;
    const bool comb = a.a != 0.0;
    const bool khz = p.kappa_h != 0.0;
    const int nT = p.nT;
    double hsum = 0.0;
    // one pass from the top: w_0 = 0 and w_{k+1} = w_k + div_k - s_k D (the
    // z-star relation read downward, D = sum_l div_l), so w_k and w_{k+1} are
    // both at hand when layer k is updated
    R wk = R(0);
    R hs_prev = R(0), hs_cur = ld(a.hR_s + i);
    for (int k = 0; k < K; k++) {
        const int x = k * Cp + i;
        R divk = R(0);
#pragma unroll
        for (int j = 0; j < NCE; j++)
            if (j < ne) divk += dcf[j] * ld(a.flux + k * Ep + es[j]);
        const R sk = PB ? sfcR[x] : sfr[k];
        const R wk1 = (k + 1 < K) ? wk + divk - sk * Dr : R(0);
        const R hs_next = (k + 1 < K) ? ld(a.hR_s + x + Cp) : R(0);
        // thickness in FP64 from the column-integrated flux (volume conservation);
        // h_out may alias h_n, so h^n is read before the store
        const double h1 = a.h_s[x] - (PB ? m.sfc[x] : m.sfrac[k]) * dtD;
        const double hn = comb ? a.h_n[x] : 0.0;
        const double hout = comb ? a.a * hn + a.b * h1 : h1;
        // the tracer arithmetic uses the tendency precision
        const R h1r = hs_cur - sk * (dtR * Dr);
        const R hnr = comb ? ld(a.hR_n + x) : R(0);
        const R houtr = comb ? aR * hnr + bR * h1r : h1r;
        for (int t = 0; t < nT; t++) {
            const R *phi = a.tr_s + t * L * Cp;
            const R ph = ld(phi + x);
            R adv = R(0), dif = R(0);
#pragma unroll
            for (int j = 0; j < NCE; j++) {
                if (j < ne && (!PB || k < kej[j])) {
                    const R po = ld(phi + k * Cp + os[j]);
                    adv += dcf[j] * (ld(a.flux + k * Ep + es[j]) * (R(0.5) * (ph + po)));
                    if (khz) {
                        // n_{e,i} grad_e(phi) = (phi_other - phi_i) / d_e for either orientation
                        const R he = R(0.5) * (hs_cur + ld(a.hR_s + k * Cp + os[j]));
                        dif += fabs(dcf[j]) * he * kh * (po - ph) * idc[j];
                    }
                }
            }
            R ftop = R(0), fbot = R(0), dtop = R(0), dbot = R(0);
            if (k >= 1) {
                const R pu = ld(phi + x - Cp);
                ftop = R(0.5) * (pu + ph) * wk;
                dtop = (pu - ph) / (R(0.5) * (hs_prev + hs_cur));
            }
            if (k + 1 <= K - 1) {
                const R pd = ld(phi + x + Cp);
                fbot = R(0.5) * (ph + pd) * wk1;
                dbot = (ph - pd) / (R(0.5) * (hs_cur + hs_next));
            }
            const R hphi = hs_cur * ph + dtR * (-adv - (ftop - fbot) + dif + kv * (dtop - dbot));
            const R phi1 = hphi / h1r;
            R out;
            if (comb)
                out = (aR * hnr * a.tr_n[t * L * Cp + x] + bR * h1r * phi1) / houtr;
            else
                out = phi1;
            a.tr_out[t * L * Cp + x] = out;
        }
        a.h_out[x] = hout;
        if (a.hR_out) a.hR_out[x] = houtr;
        hsum += hout;
        wk = wk1;
        hs_prev = hs_cur;
        hs_cur = hs_next;
    }
    a.zeta_out[i] = hsum - m.H[i];
}

// ---------------------------------------------------------------------------
// small helpers: layout conversion, SSH
// ---------------------------------------------------------------------------
// host order [n][L] in precision H, the caller's numbering <-> device
// layer-major [L][np] in precision R, the internal numbering (perm: caller
// index -> internal index).  The device holds src - off (formed in FP64,
// rounded once to R); the way back adds off in FP64.
template <class H, class R>
__global__ void k_to_device(const H *__restrict__ src, R *__restrict__ dst, int n, int L,
                            int np, const int *__restrict__ perm, double off) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * L) return;
    const int i = (int)(t / L), k = (int)(t % L);
    dst[(long long)k * np + perm[i]] = (R)((double)src[t] - off);
}
template <class R, class H>
__global__ void k_from_device(const R *__restrict__ src, H *__restrict__ dst, int n, int L,
                              int np, const int *__restrict__ perm, double off) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * L) return;
    const int i = (int)(t / L), k = (int)(t % L);
    dst[t] = (H)((double)src[(long long)k * np + perm[i]] + off);
}
// u = ubar + utilde, summed in FP64 and rounded once to H
template <class R, class H>
__global__ void k_add_bar(const R *__restrict__ ubar, const R *__restrict__ ut,
                          H *__restrict__ dst, int E, int L, int Ep,
                          const int *__restrict__ kmax, const int *__restrict__ perm) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)E * L) return;
    const int e = perm[(int)(t / L)], k = (int)(t % L);
    dst[t] = (kmax && k >= kmax[e]) ? H(0)
                                    : (H)((double)ubar[e] + (double)ut[(long long)k * Ep + e]);
}
// zero the layers a column (or edge) does not have: x[k * np + i], k >= kmax[i]
template <class R>
__global__ void k_mask_layers(R *__restrict__ x, int n, int L, int np, const int *__restrict__ kmax) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * L) return;
    const int i = (int)(t % n), k = (int)(t / n);
    if (k >= kmax[i]) x[(long long)k * np + i] = R(0);
}
__global__ void k_h_to_float(const double *__restrict__ h, float *__restrict__ hf, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) hf[t] = (float)h[t];
}
// dd[perm[t]] = scale * src[t] (and its FP32 copy): a caller-ordered 2-D
// field into the internal numbering
__global__ void k_scale(const double *__restrict__ src, double scale, double *__restrict__ dd,
                        float *__restrict__ df, int n, const int *__restrict__ perm) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const double x = src[t] * scale;
        dd[perm[t]] = x;
        df[perm[t]] = (float)x;
    }
}
__global__ void k_ssh(DMesh m, const double *__restrict__ h, double *__restrict__ zeta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.C) return;
    double s = 0.0;
    for (int k = 0; k < m.L; k++) s += h[k * m.Cp + i];
    zeta[i] = s - m.H[i];
}

// ---------------------------------------------------------------------------
// deterministic diagnostics: fixed partition, fixed-order second pass
// out = [volume, tracer0, tracer1, KE, max|u|, min h, zeta min, zeta max, nonfinite]
// ---------------------------------------------------------------------------
constexpr int NDIAG = 9;
template <class R>
__global__ void k_diag_partial(DMesh m, const R *__restrict__ ubar, const R *__restrict__ ut,
                               const double *__restrict__ h, const R *__restrict__ tr, int nT,
                               double off0, double off1, const double *__restrict__ zeta,
                               double *__restrict__ part) {
    __shared__ double sh[NDIAG][256];
    const int tid = threadIdx.x;
    double v[NDIAG] = {0, 0, 0, 0, 0, 1e300, 1e300, -1e300, 0};
    const int L = m.L, Cp = m.Cp, Ep = m.Ep;
    for (int i = blockIdx.x * blockDim.x + tid; i < m.C; i += gridDim.x * blockDim.x) {
        double hs = 0.0, t0 = 0.0, t1 = 0.0;
        const int K = m.partial ? m.kc[i] : L;    // layers of the column
        for (int k = 0; k < K; k++) {
            const double hk = h[k * Cp + i];
            hs += hk;
            t0 += hk * ((double)tr[k * Cp + i] + off0);
            if (nT > 1) t1 += hk * ((double)tr[(L + k) * Cp + i] + off1);
            v[5] = fmin(v[5], hk);
            if (!isfinite(hk) || !isfinite((double)tr[k * Cp + i])) v[8] = 1.0;
        }
        v[0] += m.area[i] * hs;
        v[1] += m.area[i] * t0;
        v[2] += m.area[i] * t1;
        v[6] = fmin(v[6], zeta[i]);
        v[7] = fmax(v[7], zeta[i]);
    }
    for (int e = blockIdx.x * blockDim.x + tid; e < m.E; e += gridDim.x * blockDim.x) {
        const int2 cc = m.coe[e];
        double ke = 0.0;
        const int K = m.partial ? m.ke[e] : L;    // layers of the edge
        for (int k = 0; k < K; k++) {
            const double u = (double)ubar[e] + (double)ut[k * Ep + e];
            const double he = 0.5 * (h[k * Cp + cc.x] + h[k * Cp + cc.y]);
            ke += he * u * u;
            v[4] = fmax(v[4], fabs(u));
            if (!isfinite(u)) v[8] = 1.0;
        }
        v[3] += m.ld2[e] * 0.5 * ke;
    }
    for (int q = 0; q < NDIAG; q++) sh[q][tid] = v[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (tid < s) {
            for (int q = 0; q < 4; q++) sh[q][tid] += sh[q][tid + s];
            sh[4][tid] = fmax(sh[4][tid], sh[4][tid + s]);
            sh[5][tid] = fmin(sh[5][tid], sh[5][tid + s]);
            sh[6][tid] = fmin(sh[6][tid], sh[6][tid + s]);
            sh[7][tid] = fmax(sh[7][tid], sh[7][tid + s]);
            sh[8][tid] = fmax(sh[8][tid], sh[8][tid + s]);
        }
        __syncthreads();
    }
    if (tid == 0)
        for (int q = 0; q < NDIAG; q++) part[blockIdx.x * NDIAG + q] = sh[q][0];
}
__global__ void k_diag_final(const double *__restrict__ part, int nparts, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double v[NDIAG] = {0, 0, 0, 0, 0, 1e300, 1e300, -1e300, 0};
    for (int b = 0; b < nparts; b++) {
        for (int q = 0; q < 4; q++) v[q] += part[b * NDIAG + q];
        v[4] = fmax(v[4], part[b * NDIAG + 4]);
        v[5] = fmin(v[5], part[b * NDIAG + 5]);
        v[6] = fmin(v[6], part[b * NDIAG + 6]);
        v[7] = fmax(v[7], part[b * NDIAG + 7]);
        v[8] = fmax(v[8], part[b * NDIAG + 8]);
    }
    for (int q = 0; q < NDIAG; q++) out[q] = v[q];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

template <class R>
void launch_cell_diag(const DMesh &m, const DParams &p, const R *ubar, const R *ut, const R *hR,
                      const R *tr, const DiagBufs<R> &b, cudaStream_t s) {
    const int nb = nblk(m.C, 128);
    if (m.partial) {
        if (m.maxE <= 6) k_cell_diag<R, 6, true><<<nb, 128, 0, s>>>(m, p, ubar, ut, hR, tr, b);
        else k_cell_diag<R, MAXE, true><<<nb, 128, 0, s>>>(m, p, ubar, ut, hR, tr, b);
    } else {
        if (m.maxE <= 6) k_cell_diag<R, 6, false><<<nb, 128, 0, s>>>(m, p, ubar, ut, hR, tr, b);
        else k_cell_diag<R, MAXE, false><<<nb, 128, 0, s>>>(m, p, ubar, ut, hR, tr, b);
    }
}
template <class R>
void launch_vertex(const DMesh &m, const R *ubar, const R *ut, const R *hR, const DiagBufs<R> &b,
                   cudaStream_t s) {
    if (m.partial) k_vertex<R, true><<<nblk(m.V, 128), 128, 0, s>>>(m, ubar, ut, hR, b);
    else k_vertex<R, false><<<nblk(m.V, 128), 128, 0, s>>>(m, ubar, ut, hR, b);
}
template <class R>
void launch_del2_divcurl(const DMesh &m, const DiagBufs<R> &b, cudaStream_t s) {
    if (m.maxE <= 6)
        k_del2_divcurl<R, 6><<<nblk(m.C + m.V, 128), 128, 0, s>>>(m, b);
    else
        k_del2_divcurl<R, MAXE><<<nblk(m.C + m.V, 128), 128, 0, s>>>(m, b);
}
template <class R>
void launch_edge_pre(const DMesh &m, R *ubar, R *ut, const R *hR, const DiagBufs<R> &b,
                     bool split, cudaStream_t s) {
    if (m.partial)
        k_edge_pre<R, true><<<nblk(m.E, 128), 128, 0, s>>>(m, ubar, ut, hR, b, split ? 1 : 0);
    else
        k_edge_pre<R, false><<<nblk(m.E, 128), 128, 0, s>>>(m, ubar, ut, hR, b, split ? 1 : 0);
}
template <class R>
void launch_bcl_edge(const DMesh &m, const DParams &p, const R *ubar, const R *ut, const R *hR,
                     const double *zeta, const DiagBufs<R> &b, const R *ut_n, double a,
                     double bcoef, double dt, R *ut_out, R *G, R *vmc, cudaStream_t s) {
    const int nb = nblk(m.E, 128);
    const R ra = (R)a, rb = (R)bcoef, rdt = (R)dt;
#define SSE_BCL(NE2, VM, PB)                                                                   \
    do {                                                                                       \
        if (m.L >= 40)                                                                         \
            k_bcl_edge<R, NE2, VM, PB, 6><<<nb, 128, 0, s>>>(m, p, ubar, ut, hR, zeta, b, ut_n,  \
                                                             ra, rb, rdt, ut_out, G, vmc);     \
        else                                                                                   \
            k_bcl_edge<R, NE2, VM, PB, 8><<<nb, 128, 0, s>>>(m, p, ubar, ut, hR, zeta, b, ut_n,  \
                                                             ra, rb, rdt, ut_out, G, vmc);     \
    } while (0)
    const bool vm = vmc != nullptr, pb = m.partial != 0;
    if (m.maxE2 <= 10) {
        if (vm) { if (pb) SSE_BCL(10, true, true); else SSE_BCL(10, true, false); }
        else { if (pb) SSE_BCL(10, false, true); else SSE_BCL(10, false, false); }
    } else {
        if (vm) { if (pb) SSE_BCL(MAXE2, true, true); else SSE_BCL(MAXE2, true, false); }
        else { if (pb) SSE_BCL(MAXE2, false, true); else SSE_BCL(MAXE2, false, false); }
    }
#undef SSE_BCL
}
template <class R>
void launch_transport(const DMesh &m, const TransportArgs<R> &a, cudaStream_t s) {
    if (m.partial) k_transport<R, true><<<nblk(m.E, 128), 128, 0, s>>>(m, a);
    else k_transport<R, false><<<nblk(m.E, 128), 128, 0, s>>>(m, a);
}
template <class R>
void launch_thickness(const DMesh &m, const DParams &p, const ThickArgs<R> &a, cudaStream_t s) {
    const int nb = nblk(m.C, 128);
    if (m.partial) {
        if (m.maxE <= 6) k_thickness<R, 6, true><<<nb, 128, 0, s>>>(m, p, a);
        else k_thickness<R, MAXE, true><<<nb, 128, 0, s>>>(m, p, a);
    } else {
        if (m.maxE <= 6) k_thickness<R, 6, false><<<nb, 128, 0, s>>>(m, p, a);
        else k_thickness<R, MAXE, false><<<nb, 128, 0, s>>>(m, p, a);
    }
}
template <class R, class H>
void launch_to_device(const H *src, R *dst, int n, int L, int np, const int *perm,
                      cudaStream_t s, double off) {
    k_to_device<H, R><<<nblk((long long)n * L, 256), 256, 0, s>>>(src, dst, n, L, np, perm, off);
}
template <class R, class H>
void launch_from_device(const R *src, H *dst, int n, int L, int np, const int *perm,
                        cudaStream_t s, double off) {
    k_from_device<R, H><<<nblk((long long)n * L, 256), 256, 0, s>>>(src, dst, n, L, np, perm,
                                                                    off);
}
template <class R, class H>
void launch_add_bar(const R *ubar, const R *ut, H *dst, int E, int L, int Ep,
                    const int *kmax, const int *perm, cudaStream_t s) {
    k_add_bar<R, H><<<nblk((long long)E * L, 256), 256, 0, s>>>(ubar, ut, dst, E, L, Ep, kmax,
                                                                perm);
}
template <class R>
void launch_mask_layers(R *x, int n, int L, int np, const int *kmax, cudaStream_t s) {
    k_mask_layers<R><<<nblk((long long)n * L, 256), 256, 0, s>>>(x, n, L, np, kmax);
}
void launch_h_to_float(const double *h, float *hf, int n, cudaStream_t s) {
    k_h_to_float<<<nblk(n, 256), 256, 0, s>>>(h, hf, n);
}
void launch_scale(const double *src, double scale, double *dst_d, float *dst_f, int n,
                  const int *perm, cudaStream_t s) {
    k_scale<<<nblk(n, 256), 256, 0, s>>>(src, scale, dst_d, dst_f, n, perm);
}
void launch_ssh(const DMesh &m, const double *h, double *zeta, cudaStream_t s) {
    k_ssh<<<nblk(m.C, 128), 128, 0, s>>>(m, h, zeta);
}
template <class R>
void launch_diag(const DMesh &m, const R *ubar, const R *ut, const double *h, const R *tr, int nT,
                 const double *toff, const double *zeta, double *partials, int nparts,
                 double *out, cudaStream_t s) {
    k_diag_partial<R><<<nparts, 256, 0, s>>>(m, ubar, ut, h, tr, nT, toff[0], toff[1], zeta,
                                             partials);
    k_diag_final<<<1, 32, 0, s>>>(partials, nparts, out);
}

#define INST(R)                                                                                  \
    template void launch_cell_diag<R>(const DMesh &, const DParams &, const R *, const R *,      \
                                      const R *, const R *, const DiagBufs<R> &, cudaStream_t);  \
    template void launch_vertex<R>(const DMesh &, const R *, const R *, const R *,               \
                                   const DiagBufs<R> &, cudaStream_t);                           \
    template void launch_del2_divcurl<R>(const DMesh &, const DiagBufs<R> &, cudaStream_t);      \
    template void launch_edge_pre<R>(const DMesh &, R *, R *, const R *, const DiagBufs<R> &,    \
                                     bool, cudaStream_t);                                        \
    template void launch_bcl_edge<R>(const DMesh &, const DParams &, const R *, const R *,       \
                                     const R *, const double *, const DiagBufs<R> &, const R *,  \
                                     double, double, double, R *, R *, R *, cudaStream_t);       \
    template void launch_transport<R>(const DMesh &, const TransportArgs<R> &, cudaStream_t);    \
    template void launch_thickness<R>(const DMesh &, const DParams &, const ThickArgs<R> &,      \
                                      cudaStream_t);                                             \
    template void launch_to_device<R, double>(const double *, R *, int, int, int, const int *,   \
                                              cudaStream_t, double);                             \
    template void launch_to_device<R, float>(const float *, R *, int, int, int, const int *,     \
                                             cudaStream_t, double);                              \
    template void launch_from_device<R, double>(const R *, double *, int, int, int, const int *, \
                                                cudaStream_t, double);                           \
    template void launch_from_device<R, float>(const R *, float *, int, int, int, const int *,   \
                                               cudaStream_t, double);                            \
    template void launch_add_bar<R, double>(const R *, const R *, double *, int, int, int,       \
                                            const int *, const int *, cudaStream_t);             \
    template void launch_add_bar<R, float>(const R *, const R *, float *, int, int, int,         \
                                           const int *, const int *, cudaStream_t);              \
    template void launch_mask_layers<R>(R *, int, int, int, const int *, cudaStream_t);          \
    template void launch_diag<R>(const DMesh &, const R *, const R *, const double *, const R *, \
                                 int, const double *, const double *, double *, int, double *,  \
                                 cudaStream_t);
INST(double)
INST(float)

}  // namespace sse
