// bcl_fused.cu -- the baroclinic stage (Algorithm 1 with the stage's SSPRK
// convex combination) as one patch-tiled kernel (sm_103a).
//
// The unfused path runs four kernels per stage (cell diagnostics, vertex
// vorticity, edge pre-pass, edge tendency) that hand every diagnostic
// (K, p', rho', z_mid, w, div u, omega, q, h_e u, q_e) to the next through
// HBM.  Here one CTA owns a compact patch of edges (csrc/tiles.cu,
// build_bcl_plan) and walks the layers from the top: each layer's velocity
// and thickness over the patch and its halo are copied into shared memory
// (cp.async into a ring of four layers, two layers ahead of the one being
// computed), the cell, vertex and edge diagnostics of that layer are
// formed in shared memory, and the owned edges' tendencies follow.  Only the
// state itself crosses HBM: utilde, h and the tracers in, utilde out.
//
// Column sums.  The z-star vertical velocity at the top of layer k,
//   w_k = sum_{l<k} div(h_e u)_l - (sum_{l<k} s_l) sum_l div(h_e u)_l,
// is the bottom-up recurrence of Sec. 2 (w_L = 0, w_k = w_{k+1} - div_k +
// s_k sum div) read from the top; its depth integral sum_l div(h_e u)_l is
// the divergence of the column transport sum_k h_e u_k, which a light
// column pre-pass (k_colflux, which also performs the split of Eq. BBspl at
// stage 1) leaves per edge.  The mid-layer height of the pressure gradient
// is read from the top as z_k = zeta - sum_{l<k} h_l - h_k / 2 (zeta = sum h
// - H).  The pressure-gradient force is formed from differences across the
// edge: p'_c2 - p'_c1 = g (sum_{l<k} [(rho' h)_c2 - (rho' h)_c1]_l + half the
// layer's own difference) and z_c2 - z_c1 from the FP64 SSH difference and
// the accumulated thickness differences -- the same quantity as the
// difference of the two columns' pressures (Eq. hydrocon), but without
// cancelling two O(g rho' H) sums in FP32.  Algorithm 1's G needs the whole
// column of provisional values: they are written as the layers go, and one
// pass over the owned columns at the end subtracts dt G.
#include "sse_internal.cuh"
#include "tiles.h"

namespace sse {

namespace {

template <class R> __device__ __forceinline__ R ldg(const R *p) { return __ldg(p); }

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
// asynchronous 4- or 8-byte copy global -> shared (Ampere+ cp.async, cached in L1)
template <class R> __device__ __forceinline__ void cp_async(R *dst, const R *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "n"(sizeof(R)));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }
// wait until at most one committed group is still in flight
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
// layers staged in shared memory: k and k + 1 in use, k + 2 and k + 3 in flight
constexpr int NBUF = 4;

template <class R> __device__ __forceinline__ const R *sfrac_R(const DMesh &m);
template <> __device__ __forceinline__ const double *sfrac_R<double>(const DMesh &m) { return m.sfrac; }
template <> __device__ __forceinline__ const float *sfrac_R<float>(const DMesh &m) { return m.sfrac_f; }

// elements of R in n rounded up to 16 bytes
template <class R> __host__ __device__ __forceinline__ int pad16(int n) {
    return (int)(((size_t)n * sizeof(R) + 15) / 16 * 16 / sizeof(R));
}
// 16-byte aligned carve-out of dynamic shared memory
template <class T> __device__ __forceinline__ T *carve(char *&p, int n) {
    T *r = reinterpret_cast<T *>(p);
    p += ((size_t)n * sizeof(T) + 15) / 16 * 16;
    return r;
}

}  // namespace

// ---------------------------------------------------------------------------
// Column pre-pass: per edge, the column transport F_e = sum_k h_e,k u_k
// (h_e = (h_c1 + h_c2) / 2, u = ubar + utilde), the input of the depth
// integral of div(h_e u).  With `split` (stage 1) it first performs the
// barotropic/baroclinic split of Eq. (BBspl) in place:
//   ubar += sum_k h_e ut_k / sum_k h_e,  ut_k -= that mean.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void colflux_edge(const DMesh &m, R *__restrict__ ubar,
                                             R *__restrict__ ut, const R *__restrict__ hR,
                                             int split, R *__restrict__ Fc, const int e) {
    if (e >= m.E) return;
    const int Ep = m.Ep, Cp = m.Cp, L = m.L;
    const int2 cc = m.coe[e];
    R num = R(0), den = R(0);
    for (int k = 0; k < L; k++) {
        const R he = R(0.5) * (ldg(hR + k * Cp + cc.x) + ldg(hR + k * Cp + cc.y));
        num += he * ut[k * Ep + e];
        den += he;
    }
    R ub = ubar[e];
    if (!split) {
        Fc[e] = ub * den + num;
        return;
    }
    const R mean = num / den;
    ub += mean;
    ubar[e] = ub;
    R F = R(0);
    for (int k = 0; k < L; k++) {
        const R he = R(0.5) * (ldg(hR + k * Cp + cc.x) + ldg(hR + k * Cp + cc.y));
        const R x = ut[k * Ep + e] - mean;
        ut[k * Ep + e] = x;
        F += he * (ub + x);
    }
    Fc[e] = F;
}

// ---------------------------------------------------------------------------
// The fused stage kernel.  One CTA per patch, NT threads; owned edge i and C1
// cell i belong to thread i % NT, slot i / NT (at most NI slots).
//   ut1_k = ut_k + dt ( [Q_k - C_f(ubar)] - grad K_k - PGF_k - avg^m(w D_zt u)_k
//                       + nu_h Lap u_k + D^u_k + g grad zeta )
//   G = (1/dt) sum_k h_e,k ut1_k / sum_k h_e,k,  out_k = a ut_n,k + b (ut1_k - dt G)
// with the same operators, PGF anomaly form and boundary fluxes as the
// unfused kernels (stage_kernels.cu).
// ---------------------------------------------------------------------------
template <class R, int NT, int NI>
__device__ __forceinline__ void bcl_fused_patch(const DMesh &m, const DParams &p, const DBcl<R> &t,
                                                const BclArgs<R> &a, const int pid) {
    using R2 = V2<R>;
    const int tid = threadIdx.x;
    const int *cn = t.cnt + 8 * pid;
    const int nE0 = cn[0], nE1 = cn[1], nE2 = cn[2], nC1 = cn[3], nC2 = cn[4], nV = cn[5];
    const int *eg_g = t.egid + t.off_e2[pid];
    const int *cg_g = t.cgid + t.off_c2[pid];
    const int oe0 = t.off_e0[pid], oe1 = t.off_e1[pid], oc1 = t.off_c1[pid], ov = t.off_v[pid];
    const int Ep = m.Ep, Cp = m.Cp, L = m.L;
    const PhysR<R> &q = phys<R>(p);

    extern __shared__ __align__(16) char smem[];
    char *sp = smem;
    // three layers of utilde / h (k, k + 1 and k + 2 in flight), of the
    // tracers at C1 and of the old level at the owned edges
    R *ub_s = carve<R>(sp, t.maxE2 + 1);
    // buffer b of each ring starts at b times its stride (a multiple of 16 bytes)
    const int sE = pad16<R>(t.maxE2 + 1), sC = pad16<R>(t.maxC2 + 1);
    const int s1 = pad16<R>(t.maxC1), s0 = pad16<R>(t.maxE0);
    R *ut_r = carve<R>(sp, NBUF * sE);
    R *h_r = carve<R>(sp, NBUF * sC);
    R *T_r = carve<R>(sp, NBUF * s1);
    R *S_r = carve<R>(sp, NBUF * s1);
    R *un_r = carve<R>(sp, NBUF * s0);
    R *q_s = carve<R>(sp, t.maxV);
    R *om_s = carve<R>(sp, t.maxV);
    R2 *hq_s = carve<R2>(sp, t.maxE1 + 1);
    R *cK = carve<R>(sp, t.maxC1);
    R *cR = carve<R>(sp, t.maxC1);
    R *cW1 = carve<R>(sp, t.maxC1);
    R *cD = carve<R>(sp, t.maxC1);
    // the patch's connectivity and coefficients, read every layer: copied to
    // shared memory once (term-major, stride = the patch's own count)
    unsigned short *x_e0i = carve<unsigned short>(sp, BCL_NE2P * t.maxE0);
    R *x_e0w = carve<R>(sp, BCL_NE2P * t.maxE0);
    unsigned short *x_c1e = carve<unsigned short>(sp, BCL_NCEP * t.maxC1);
    unsigned short *x_c1o = carve<unsigned short>(sp, BCL_NCEP * t.maxC1);
    R *x_c1d = carve<R>(sp, BCL_NCEP * t.maxC1);
    R *x_c1k = carve<R>(sp, BCL_NCEP * t.maxC1);
    unsigned short *x_ve = carve<unsigned short>(sp, 3 * t.maxV);
    unsigned short *x_vc = carve<unsigned short>(sp, 3 * t.maxV);
    R *x_vcu = carve<R>(sp, 3 * t.maxV);
    R *x_vkw = carve<R>(sp, 3 * t.maxV);
    R *x_vf = carve<R>(sp, t.maxV);
    int *x_e1c = carve<int>(sp, t.maxE1);
    int *x_e1v = carve<int>(sp, t.maxE1);
    // the patch's internal edge and cell indices (each layer's copies use them)
    int *eg = carve<int>(sp, t.maxE2);
    int *cg = carve<int>(sp, t.maxC2);
    for (int j = tid; j < nE2; j += NT) eg[j] = eg_g[j];
    for (int j = tid; j < nC2; j += NT) cg[j] = cg_g[j];
    __syncthreads();
    for (int j = tid; j < BCL_NE2P * nE0; j += NT) {
        x_e0i[j] = t.e0_eoe[BCL_NE2P * oe0 + j];
        x_e0w[j] = ldg(t.e0_wl + BCL_NE2P * oe0 + j);
    }
    for (int j = tid; j < BCL_NCEP * nC1; j += NT) {
        x_c1e[j] = t.c1_e[BCL_NCEP * oc1 + j];
        x_c1o[j] = t.c1_o[BCL_NCEP * oc1 + j];
        x_c1d[j] = ldg(t.c1_divc + BCL_NCEP * oc1 + j);
        x_c1k[j] = ldg(t.c1_kec + BCL_NCEP * oc1 + j);
    }
    for (int j = tid; j < 3 * nV; j += NT) {
        x_ve[j] = t.v_e[3 * ov + j];
        x_vc[j] = t.v_c[3 * ov + j];
        x_vcu[j] = ldg(t.v_curl + 3 * ov + j);
        x_vkw[j] = ldg(t.v_kw + 3 * ov + j);
    }
    for (int j = tid; j < nV; j += NT) x_vf[j] = ldg(t.v_f + ov + j);
    for (int j = tid; j < nE1; j += NT) {
        x_e1c[j] = t.e1_c12[oe1 + j];
        x_e1v[j] = t.e1_v12[oe1 + j];
    }
    const bool two = p.nT > 1;
    const bool comb = a.ut_n != nullptr;
    // one layer's copies into buffer b
    auto issue = [&](int k, int b) {
        const R *un = a.ut + (size_t)k * Ep;
        const R *hn = a.hR + (size_t)k * Cp;
        R *ud = ut_r + b * sE, *hd = h_r + b * sC, *Td = T_r + b * s1, *Sd = S_r + b * s1;
        for (int j = tid; j < nE2; j += NT) cp_async(ud + j, un + eg[j]);
        for (int j = tid; j < nC2; j += NT) cp_async(hd + j, hn + cg[j]);
        for (int j = tid; j < nC1; j += NT) {
            cp_async(Td + j, a.tr + (size_t)k * Cp + cg[j]);
            if (two) cp_async(Sd + j, a.tr + (size_t)(L + k) * Cp + cg[j]);
        }
        if (comb) {
            R *nd = un_r + b * s0;
            for (int j = tid; j < nE0; j += NT) cp_async(nd + j, a.ut_n + (size_t)k * Ep + eg[j]);
        }
        cp_async_commit();
    };

    // ---- the layer-invariant 2-D data; layers 0 and 1 in flight
    for (int j = tid; j < nE2; j += NT) ub_s[j] = ldg(a.ubar + eg[j]);
    if (tid == 0) {
        ub_s[nE2] = R(0);
        for (int b = 0; b < NBUF; b++) { ut_r[b * sE + nE2] = R(0); h_r[b * sC + nC2] = R(0); }
        R2 z; z.x = R(0); z.y = R(0);
        hq_s[nE1] = z;
    }
    // layers 0, 1 and 2 in flight (one commit group each, empty past the bottom)
    for (int k = 0; k < NBUF - 1; k++) {
        if (k < L) issue(k, k);
        else cp_async_commit();
    }

    // cells of C1 held by this thread: global index, SSH, depth integral of
    // div(h_e u) and the running column sums
    int gc[NI];
    R dsum[NI], W[NI];
#pragma unroll
    for (int s = 0; s < NI; s++) {
        const int c = tid + s * NT;
        gc[s] = 0; dsum[s] = R(0); W[s] = R(0);
        if (c < nC1) {
            gc[s] = cg[c];
            R d = R(0);
#pragma unroll
            for (int j = 0; j < BCL_NCEP; j++) {
                const int el = t.c1_e[6 * oc1 + j * nC1 + c];
                if (el < nE2) d += ldg(t.c1_divc + 6 * oc1 + j * nC1 + c) * ldg(a.Fc + eg[el]);
            }
            dsum[s] = d;
        }
    }
    // owned edges held by this thread
    int ge[NI], c12[NI], v12[NI];
    R cbar[NI], gzeta[NI], wind[NI], idc[NI], idv[NI], Dk[NI], wk[NI], num[NI], den[NI];
    // pressure gradient from differences across the edge, accumulated down the
    // column: dA = sum_{l<k} (rho' h)_c2 - (rho' h)_c1, dH = sum_{l<k} h_c2 - h_c1
    R dA[NI], dH[NI], dzeta[NI];
    const R *wnd = wind_over_rho0<R>(p);
#pragma unroll
    for (int s = 0; s < NI; s++) {
        const int e = tid + s * NT;
        ge[s] = 0; c12[s] = 0; v12[s] = 0;
        gzeta[s] = R(0); wind[s] = R(0); idc[s] = R(0); idv[s] = R(0);
        Dk[s] = R(0); wk[s] = R(0); num[s] = R(0); den[s] = R(0); cbar[s] = R(0);
        dA[s] = R(0); dH[s] = R(0); dzeta[s] = R(0);
        if (e < nE0) {
            ge[s] = eg[e];
            c12[s] = t.e0_c12[oe0 + e];
            v12[s] = t.e0_v12[oe0 + e];
            idc[s] = ldg(t.e0_invdc + oe0 + e);
            idv[s] = ldg(t.e0_invdv + oe0 + e);
            const int g1 = cg[c12[s] & 0xffff], g2 = cg[c12[s] >> 16];
            dzeta[s] = (R)(a.zeta[g2] - a.zeta[g1]);   // the difference taken in FP64
            gzeta[s] = q.zcoef * dzeta[s] * idc[s];
            wind[s] = wnd ? wnd[ge[s]] : R(0);
        }
    }
    __syncthreads();   // ub_s
#pragma unroll
    for (int s = 0; s < NI; s++) {
        const int e = tid + s * NT;
        if (e < nE0) {
            // C_f(u_k) - C_f(ut_k) = C_f(ubar): one 2-D sum per column
            R cb = R(0);
#pragma unroll
            for (int j = 0; j < BCL_NE2P; j++) {
                const int x = BCL_NE2P * oe0 + j * nE0 + e;
                cb += ldg(t.e0_cfc + x) * ub_s[t.e0_eoe[x]];
            }
            cbar[s] = cb;
        }
    }
    const R g = q.g, alpha = q.alpha, beta = q.beta, Tref = q.T_ref, Sref = q.S_ref;
    const R inv_rho0 = q.inv_rho0, nu_h = q.nu_h, nu_v = q.nu_v, cdrag = q.c_drag;
    const R dt = a.dt, ca = a.a, cb = a.b;
    const R *sfr = sfrac_R<R>(m);
    R Sk = R(0);   // sum_{l<k} s_l

    for (int k = 0; k < L; k++) {
        const int bc = k % NBUF, bn = (k + 1) % NBUF;
        const R *ut_c = ut_r + bc * sE, *h_c = h_r + bc * sC;
        const R *ut_nx = ut_r + bn * sE, *h_nx = h_r + bn * sC;
        const R *T_c = T_r + bc * s1, *S_c = S_r + bc * s1, *un_c = un_r + bc * s0;
        cp_async_wait_1();
        __syncthreads();   // layers k and k + 1 in shared memory; layer k - 1's readers done
        if (k + 3 < L) issue(k + 3, (k + 3) % NBUF);
        else cp_async_commit();
        // ---- vertices: relative vorticity, kite-averaged thickness, PV
        for (int v = tid; v < nV; v += NT) {
            R om = R(0), hv = R(0);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int x = j * nV + v;
                const int el = x_ve[x], cl = x_vc[x];
                om += x_vcu[x] * (ub_s[el] + ut_c[el]);
                hv += x_vkw[x] * h_c[cl];
            }
            om_s[v] = om;
            q_s[v] = (om + x_vf[v]) / hv;
        }
        // ---- cells of C1: K, div u, div(h_e u), rho', p', z_mid, w
        const R sk = sfr[k];
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const int c = tid + s * NT;
            if (c < nC1) {
                const R hk = h_c[c];
                R ke = R(0), dl = R(0), dv = R(0);
#pragma unroll
                for (int j = 0; j < BCL_NCEP; j++) {
                    const int x = j * nC1 + c;
                    const int el = x_c1e[x], ol = x_c1o[x];
                    const R uk = ub_s[el] + ut_c[el];
                    const R he = R(0.5) * (hk + h_c[ol]);
                    const R dc = x_c1d[x];
                    ke += x_c1k[x] * uk * uk;
                    dl += dc * uk;
                    dv += dc * (he * uk);
                }
                R rp = -alpha * (T_c[c] - Tref);
                if (two) rp += beta * (S_c[c] - Sref);
                cK[c] = ke;
                cR[c] = rp;
                cD[c] = dl;
                W[s] += dv;
                // w at the top of layer k + 1
                cW1[c] = W[s] - (Sk + sk) * dsum[s];
            }
        }
        __syncthreads();
        // ---- edges of E1: (h_e u, q_e)
        for (int e = tid; e < nE1; e += NT) {
            const int cc = x_e1c[e], vv = x_e1v[e];
            R2 hq;
            hq.x = R(0.5) * (h_c[cc & 0xffff] + h_c[cc >> 16]) * (ub_s[e] + ut_c[e]);
            hq.y = R(0.5) * (q_s[vv & 0xffff] + q_s[vv >> 16]);
            hq_s[e] = hq;
        }
        __syncthreads();
        // ---- owned edges: the tendency of layer k
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const int e = tid + s * NT;
            if (e >= nE0) continue;
            const int c1 = c12[s] & 0xffff, c2 = c12[s] >> 16;
            const int v1 = v12[s] & 0xffff, v2 = v12[s] >> 16;
            const R ut_cur = ut_c[e], u_cur = ub_s[e] + ut_cur;
            const R he_cur = R(0.5) * (h_c[c1] + h_c[c2]);
            const R qk = hq_s[e].y;
            R Q = R(0);
#pragma unroll
            for (int j = 0; j < BCL_NE2P; j++) {
                const int x = j * nE0 + e;
                const R2 nb = hq_s[x_e0i[x]];
                Q += x_e0w[x] * nb.x * (R(0.5) * (qk + nb.y));
            }
            const R gradK = (cK[c2] - cK[c1]) * idc[s];
            // p'_2 - p'_1 and z_2 - z_1 (z = zeta - sum_{l<k} h_l - h_k / 2)
            const R h1 = h_c[c1], h2 = h_c[c2];
            const R rh = cR[c2] * h2 - cR[c1] * h1;
            const R dp = g * (dA[s] + R(0.5) * rh);
            const R dz = dzeta[s] - dH[s] - R(0.5) * (h2 - h1);
            const R pgf = (dp + g * (R(0.5) * (cR[c1] + cR[c2])) * dz) * idc[s] * inv_rho0;
            dA[s] += rh;
            dH[s] += h2 - h1;
            R Dk1 = R(0), wk1 = R(0);
            if (k + 1 < L) {
                const R u_next = ub_s[e] + ut_nx[e];
                const R he_next = R(0.5) * (h_nx[c1] + h_nx[c2]);
                Dk1 = (u_cur - u_next) / (R(0.5) * (he_cur + he_next));
                wk1 = R(0.5) * (cW1[c1] + cW1[c2]);
            }
            const R vadv = R(0.5) * (wk[s] * Dk[s] + wk1 * Dk1);
            const R Xtop = (k == 0) ? wind[s] : nu_v * Dk[s];
            R Xbot;
            if (k == L - 1) {
                R utan = R(0);
#pragma unroll
                for (int j = 0; j < BCL_NE2P; j++) {
                    const int x = j * nE0 + e;
                    const int el = x_e0i[x];
                    utan += x_e0w[x] * (ub_s[el] + ut_c[el]);
                }
                Xbot = cdrag * sqrt(u_cur * u_cur + utan * utan) * u_cur;
            } else {
                Xbot = nu_v * Dk1;
            }
            const R vvisc = (Xtop - Xbot) / he_cur;
            const R lap = (cD[c2] - cD[c1]) * idc[s] - (om_s[v2] - om_s[v1]) * idv[s];
            const R rhs = (Q - cbar[s]) - gradK - pgf - vadv + nu_h * lap + vvisc + gzeta[s];
            const R ut1 = ut_cur + dt * rhs;
            num[s] += he_cur * ut1;
            den[s] += he_cur;
            const size_t xo = (size_t)k * Ep + ge[s];
            a.ut_out[xo] = comb ? ca * un_c[e] + cb * ut1 : cb * ut1;
            Dk[s] = Dk1;
            wk[s] = wk1;
        }
        Sk += sk;
    }
    cp_async_wait_all();
    // ---- G and the subtraction of dt G over the owned columns
#pragma unroll
    for (int s = 0; s < NI; s++) {
        const int e = tid + s * NT;
        if (e >= nE0) continue;
        const R G = num[s] / den[s] / dt;
        a.G[ge[s]] = G;
        const R corr = cb * dt * G;
        for (int k = 0; k < L; k++) {
            const size_t xo = (size_t)k * Ep + ge[s];
            a.ut_out[xo] -= corr;
        }
    }
}


// ---------------------------------------------------------------------------
// Batched launches: the blocks of several states' launches of one kernel in
// one grid.  Job j owns the blocks [first[j], first[j + 1]); a block copies
// its job's descriptor into shared memory and runs the same per-block code as
// the single-state kernel, so every state's arithmetic is unchanged.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int job_of_block(const int *first, int njobs) {
    int lo = 0, hi = njobs - 1;
    const int b = blockIdx.x;
    while (lo < hi) {   // the last job whose first block is <= b
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}
template <class T> __device__ __forceinline__ void copy_job(T &dst, const T &src) {
    static_assert(sizeof(T) % 4 == 0, "job descriptors are copied in 4-byte words");
    const int *s = reinterpret_cast<const int *>(&src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}

// Both the single-state and the batched kernels copy their descriptor into
// shared memory and run the body on that copy, so that the body compiles to
// the same instructions in both and a state's results are the same bits
// whether it steps alone or in a batch.
template <class R, int NT, int NI>
__global__ void __launch_bounds__(NT, 2) k_bcl_fused(const BclJob<R> job) {
    __shared__ BclJob<R> J;
    copy_job(J, job);
    __syncthreads();
    bcl_fused_patch<R, NT, NI>(J.m, J.p, J.t, J.a, blockIdx.x);
}
template <class R, int NT, int NI>
__global__ void __launch_bounds__(NT, 2) k_bcl_fused_batch(const BclJob<R> *__restrict__ jobs,
                                                           const int *__restrict__ first,
                                                           int njobs) {
    __shared__ BclJob<R> J;
    const int j = job_of_block(first, njobs);
    copy_job(J, jobs[j]);
    __syncthreads();
    bcl_fused_patch<R, NT, NI>(J.m, J.p, J.t, J.a, blockIdx.x - first[j]);
}

template <class R>
__global__ void __launch_bounds__(128) k_colflux_one(const ColfluxJob<R> job) {
    __shared__ ColfluxJob<R> J;
    copy_job(J, job);
    __syncthreads();
    colflux_edge<R>(J.m, J.ubar, J.ut, J.hR, J.split, J.Fc, blockIdx.x * blockDim.x + threadIdx.x);
}
template <class R>
__global__ void __launch_bounds__(128) k_colflux_batch(const ColfluxJob<R> *__restrict__ jobs,
                                                       const int *__restrict__ first, int njobs) {
    __shared__ ColfluxJob<R> J;
    const int j = job_of_block(first, njobs);
    copy_job(J, jobs[j]);
    __syncthreads();
    colflux_edge<R>(J.m, J.ubar, J.ut, J.hR, J.split, J.Fc,
                    (blockIdx.x - first[j]) * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
constexpr int BCL_NT = 256;
constexpr int BCL_NI = 2;

template <class R> size_t bcl_smem_bytes(const BclPlan &plan) {
    auto a16 = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t sR = sizeof(R);
    size_t b = 0;
    b += (1 + NBUF) * a16(sR * (plan.maxE2 + 1));   // ubar, utilde (NBUF layers)
    b += NBUF * a16(sR * (plan.maxC2 + 1));         // h
    b += 2 * NBUF * a16(sR * plan.maxC1);           // T, S
    b += NBUF * a16(sR * plan.maxE0);               // old-level utilde
    // (each ring is carved as one block of NBUF 16-byte padded strides)
    b += 2 * a16(sR * plan.maxV);               // q, omega
    b += a16(2 * sR * (plan.maxE1 + 1));        // (h_e u, q_e)
    b += 4 * a16(sR * plan.maxC1);              // K, rho', w, div u
    // connectivity and coefficients of the patch
    b += a16(2 * BCL_NE2P * plan.maxE0) + a16(sR * BCL_NE2P * plan.maxE0);
    b += 2 * a16(2 * BCL_NCEP * plan.maxC1) + 2 * a16(sR * BCL_NCEP * plan.maxC1);
    b += 2 * a16(2 * 3 * plan.maxV) + 2 * a16(sR * 3 * plan.maxV) + a16(sR * plan.maxV);
    b += 2 * a16(4 * plan.maxE1);
    b += a16(4 * plan.maxE2) + a16(4 * plan.maxC2);   // internal indices
    return b;
}
int bcl_max_edges_per_patch() { return BCL_NT * BCL_NI; }
int bcl_max_cells_per_patch() { return BCL_NT * BCL_NI; }
template <class R> const void *bcl_fused_kernel_ptr() {
    return (const void *)k_bcl_fused<R, BCL_NT, BCL_NI>;
}

template <class R>
void launch_colflux(const DMesh &m, R *ubar, R *ut, const R *hR, bool split, R *Fc,
                    cudaStream_t s) {
    const ColfluxJob<R> job{m, ubar, ut, hR, Fc, split ? 1 : 0, 0};
    k_colflux_one<R><<<(m.E + 127) / 128, 128, 0, s>>>(job);
}
template <class R>
void launch_bcl_fused(const DBcl<R> &t, const DMesh &m, const DParams &p, const BclArgs<R> &a,
                      cudaStream_t s) {
    const BclJob<R> job{m, p, t, a};
    k_bcl_fused<R, BCL_NT, BCL_NI><<<t.P, BCL_NT, t.smem, s>>>(job);
}

template <class R>
void launch_colflux_batch(const ColfluxJob<R> *jobs, const int *first, int njobs, int blocks,
                          cudaStream_t s) {
    k_colflux_batch<R><<<blocks, 128, 0, s>>>(jobs, first, njobs);
}
int colflux_blocks(const DMesh &m) { return (m.E + 127) / 128; }
template <class R>
void launch_bcl_fused_batch(const BclJob<R> *jobs, const int *first, int njobs, int blocks,
                            size_t smem, cudaStream_t s) {
    k_bcl_fused_batch<R, BCL_NT, BCL_NI><<<blocks, BCL_NT, smem, s>>>(jobs, first, njobs);
}
template <class R> const void *bcl_fused_batch_kernel_ptr() {
    return (const void *)k_bcl_fused_batch<R, BCL_NT, BCL_NI>;
}
template void launch_colflux_batch<float>(const ColfluxJob<float> *, const int *, int, int,
                                          cudaStream_t);
template void launch_colflux_batch<double>(const ColfluxJob<double> *, const int *, int, int,
                                           cudaStream_t);
template void launch_bcl_fused_batch<float>(const BclJob<float> *, const int *, int, int, size_t,
                                            cudaStream_t);
template void launch_bcl_fused_batch<double>(const BclJob<double> *, const int *, int, int,
                                             size_t, cudaStream_t);
template const void *bcl_fused_batch_kernel_ptr<float>();
template const void *bcl_fused_batch_kernel_ptr<double>();
template size_t bcl_smem_bytes<float>(const BclPlan &);
template size_t bcl_smem_bytes<double>(const BclPlan &);
template const void *bcl_fused_kernel_ptr<float>();
template const void *bcl_fused_kernel_ptr<double>();
template void launch_colflux<float>(const DMesh &, float *, float *, const float *, bool, float *,
                                    cudaStream_t);
template void launch_colflux<double>(const DMesh &, double *, double *, const double *, bool,
                                     double *, cudaStream_t);
template void launch_bcl_fused<float>(const DBcl<float> &, const DMesh &, const DParams &,
                                      const BclArgs<float> &, cudaStream_t);
template void launch_bcl_fused<double>(const DBcl<double> &, const DMesh &, const DParams &,
                                       const BclArgs<double> &, cudaStream_t);

}  // namespace sse
