// bcl_fused.cu -- the baroclinic stage (Algorithm 1 with the stage's SSPRK
// convex combination) as one patch-tiled kernel (sm_103a).
//
// The unfused path runs four kernels per stage (cell diagnostics, vertex
// vorticity, edge pre-pass, edge tendency) that hand every diagnostic
// (K, p', rho', z_mid, w, div u, omega, q, h_e u, q_e) to the next through
// HBM.  Here one CTA owns a compact patch of edges (csrc/tiles.cu,
// build_bcl_plan) and walks the layers from the top, two at a time: each
// pair's velocity and thickness over the patch and its halo are copied into
// shared memory (cp.async into a ring of NB2 pairs, NB2 - 2 pairs ahead of
// the two in use), the cell, vertex and edge diagnostics of both layers are
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
#include <algorithm>
#include <cstring>
#include <vector>

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
// asynchronous 16-byte copy global -> shared, bypassing L1 (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }
// wait until at most N committed groups are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait_n() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
// layer pairs staged in shared memory: p and p + 1 in use, p + 2 .. p + NB2 - 1
// in flight (each pair's copies get NB2 - 2 pairs of compute to land)
constexpr int NB2 = 3;
// CTAs per SM of the fused kernel: two in FP32 (128 registers a thread); one
// in FP64, whose per-thread column state needs about 250 registers
template <class R> constexpr int bcl_min_blocks() { return sizeof(R) == 4 ? 2 : 1; }
// four values of one precision side by side in shared memory, at the 16-byte
// alignment a carve gives
struct __align__(16) dbl4s { double x, y, z, w; };
template <class R> struct Sh4 { using T = float4; };
template <> struct Sh4<double> { using T = dbl4s; };

template <class R> __device__ __forceinline__ const R *sfrac_R(const DMesh &m);
template <> __device__ __forceinline__ const double *sfrac_R<double>(const DMesh &m) { return m.sfrac; }
template <> __device__ __forceinline__ const float *sfrac_R<float>(const DMesh &m) { return m.sfrac_f; }

// a / b for the per-layer quotients: correctly rounded in FP64; in FP32 the
// reciprocal-multiply form (within 2 ulp for the divisors met here, thicknesses
// of 1e-3 to 1e4 m), whose error is far below the FP32 form's other rounding
template <class R> __device__ __forceinline__ R qdiv(R a, R b);
template <> __device__ __forceinline__ double qdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

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
//
// The layers are taken two at a time: shared memory holds each value of a
// pair of layers (k, k + 1) side by side, so one vector load serves both and
// every index and coefficient is read once per pair; the column recurrences
// (w, the pressure-gradient sums, D_zt u, G) then advance through the two
// layers in order.  A ring of NB2 pair buffers holds pair p (being
// computed), pair p + 1 (its first layer is the layer below pair p's second)
// and pairs p + 2 .. p + NB2 - 1 (in flight).
// ---------------------------------------------------------------------------
template <class R, int NT, int NI>
__device__ __forceinline__ void bcl_fused_patch(const DMesh &m, const DParams &p, const DBcl<R> &t,
                                                const BclArgs<R> &a, const int pid) {
    using R2 = V2<R>;
    using R4 = typename Sh4<R>::T;
    const int tid = threadIdx.x;
    // C1 cells are dealt from the last thread down, so that the threads that
    // hold a second vertex (the first ones) hold no cell
    const int ctid = NT - 1 - tid;
    const int *cn = t.cnt + 8 * pid;
    const int nE0 = cn[0], nE1 = cn[1], nE2 = cn[2], nC1 = cn[3], nC2 = cn[4], nV = cn[5];
    const int oe0 = t.off_e0[pid], ov = t.off_v[pid];
    const int Ep = m.Ep, Cp = m.Cp, L = m.L;
    const int NP = (L + 1) / 2;   // layer pairs (the second layer of the last is absent if L is odd)
    const PhysR<R> &q = phys<R>(p);

    extern __shared__ __align__(16) char smem[];
    char *sp = smem;
    R *ub_s = carve<R>(sp, t.maxE2 + 1);
    // buffer b of each ring starts at b times its stride (a multiple of 16 bytes)
    const int sE = pad16<R2>(t.maxE2 + 1), sC = pad16<R2>(t.maxC2 + 1);
    R2 *ut_r = carve<R2>(sp, NB2 * sE);
    R2 *h_r = carve<R2>(sp, NB2 * sC);
    R2 *q_s = carve<R2>(sp, t.maxV);
    R2 *om_s = carve<R2>(sp, t.maxV);
    R4 *hq_s = carve<R4>(sp, t.maxE1 + 1);   // (h_e u, q_e) of both layers
    R2 *cK = carve<R2>(sp, t.maxC1);
    R2 *cR = carve<R2>(sp, t.maxC1);
    R2 *cW1 = carve<R2>(sp, t.maxC1);
    R2 *cD = carve<R2>(sp, t.maxC1);
    R2 *x_vbf = carve<R2>(sp, t.maxV);   // (curl ubar, curl ubar + f): layer-invariant
    R *sf_s = carve<R>(sp, L);           // the layers' z-star stretching fractions s_k
    // the patch's connectivity and coefficients, read every pair: the host
    // packed them per patch in this layout (bcl_build_image), copied here in
    // 16-byte pieces; term-major with the patch's own counts as strides,
    // index pairs as lo | hi << 16, coefficient pairs side by side
    {
        const unsigned char *src = t.img + t.img_off[pid];
        const int n16 = (int)((t.img_off[pid + 1] - t.img_off[pid]) / 16);
        for (int i = tid; i < n16; i += NT) cp_async16(sp + 16 * i, src + 16 * i);
        cp_async_commit();
    }
    char *ip = sp;
    unsigned short *x_e0i = carve<unsigned short>(ip, BCL_NE2P * nE0);
    R *x_e0w = carve<R>(ip, BCL_NE2P * nE0);
    unsigned *x_c1eo = carve<unsigned>(ip, BCL_NCEP * nC1);
    R2 *x_c1dk = carve<R2>(ip, BCL_NCEP * nC1);
    unsigned *x_vec = carve<unsigned>(ip, 3 * nV);
    R2 *x_vck = carve<R2>(ip, 3 * nV);
    int *x_e1c = carve<int>(ip, nE1);
    int *x_e1v = carve<int>(ip, nE1);
    // the patch's internal edge and cell indices (each layer's copies use them)
    int *eg = carve<int>(ip, nE2);
    int *cg = carve<int>(ip, nC2);
    {
        const R *sfr = sfrac_R<R>(m);
        for (int k = tid; k < L; k += NT) sf_s[k] = sfr[k];
    }
    cp_async_wait_all();
    __syncthreads();
    const bool two = p.nT > 1;
    const bool comb = a.ut_n != nullptr;
    // one pair's copies into buffer b (the second layer's only if it exists)
    auto issue = [&](int pp, int b) {
        const int k0 = 2 * pp;
        const bool has1 = k0 + 1 < L;
        R *ud = reinterpret_cast<R *>(ut_r + b * sE), *hd = reinterpret_cast<R *>(h_r + b * sC);
        const R *u0 = a.ut + (size_t)k0 * Ep, *h0 = a.hR + (size_t)k0 * Cp;
        for (int j = tid; j < nE2; j += NT) {
            const int ge = eg[j];
            cp_async(ud + 2 * j, u0 + ge);
            if (has1) cp_async(ud + 2 * j + 1, u0 + Ep + ge);
        }
        for (int j = tid; j < nC2; j += NT) {
            const int gc = cg[j];
            cp_async(hd + 2 * j, h0 + gc);
            if (has1) cp_async(hd + 2 * j + 1, h0 + Cp + gc);
        }
        cp_async_commit();
    };

    // ---- the layer-invariant 2-D data; pairs 0 and 1 in flight
    for (int j = tid; j < nE2; j += NT) ub_s[j] = ldg(a.ubar + eg[j]);
    if (tid == 0) {
        R2 z2;
        z2.x = R(0); z2.y = R(0);
        ub_s[nE2] = R(0);
        for (int b = 0; b < NB2; b++) { ut_r[b * sE + nE2] = z2; h_r[b * sC + nC2] = z2; }
        R4 z4;
        z4.x = R(0); z4.y = R(0); z4.z = R(0); z4.w = R(0);
        hq_s[nE1] = z4;
    }
    // pairs 0 .. NB2 - 2 in flight (one commit group each, empty past the bottom)
    for (int pp = 0; pp < NB2 - 1; pp++) {
        if (pp < NP) issue(pp, pp);
        else cp_async_commit();
    }

    // cells of C1 held by this thread: the depth integral of div(h_e u) and
    // the running column sum
    R dsum[NI], W[NI];
#pragma unroll
    for (int s = 0; s < NI; s++) {
        const int c = ctid + s * NT;
        dsum[s] = R(0); W[s] = R(0);
        if (c < nC1) {
            R d = R(0);
#pragma unroll
            for (int j = 0; j < BCL_NCEP; j++) {
                const int el = x_c1eo[j * nC1 + c] & 0xffff;
                if (el < nE2) d += x_c1dk[j * nC1 + c].x * ldg(a.Fc + eg[el]);
            }
            dsum[s] = d;
        }
    }
    // owned edges held by this thread
    int ge[NI], c12[NI], v12[NI];
    R cbar[NI], idc[NI], idv[NI], Dk[NI], wk[NI], num[NI], den[NI];
    // pressure gradient from differences across the edge, accumulated down the
    // column: dA = sum_{l<k} (rho' h)_c2 - (rho' h)_c1, dH = sum_{l<k} h_c2 - h_c1
    R dA[NI], dH[NI], dzeta[NI];
    const R *wnd = wind_over_rho0<R>(p);
#pragma unroll
    for (int s = 0; s < NI; s++) {
        const int e = tid + s * NT;
        ge[s] = 0; c12[s] = 0; v12[s] = 0;
        idc[s] = R(0); idv[s] = R(0);
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
                cb += ldg(t.e0_cfc + BCL_NE2P * oe0 + j * nE0 + e) * ub_s[x_e0i[j * nE0 + e]];
            }
            cbar[s] = cb;
        }
    }
    // the relative vorticity of ubar at the vertices (every layer's omega is
    // this plus the curl of its utilde)
    for (int v = tid; v < nV; v += NT) {
        R ob = R(0);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int x = j * nV + v;
            ob += x_vck[x].x * ub_s[x_vec[x] & 0xffff];
        }
        R2 bf;
        bf.x = ob;
        bf.y = ob + ldg(t.v_f + ov + v);
        x_vbf[v] = bf;
    }
    const R g = q.g, alpha = q.alpha, beta = q.beta, Tref = q.T_ref, Sref = q.S_ref;
    const R inv_rho0 = q.inv_rho0, nu_h = q.nu_h, nu_v = q.nu_v, cdrag = q.c_drag;
    const R dt = a.dt, ca = a.a, cb = a.b;
    R Sk = R(0);   // sum_{l<k} s_l

    for (int pp = 0; pp < NP; pp++) {
        const int k0 = 2 * pp;
        const bool has1 = k0 + 1 < L;
        const int bc = pp % NB2, bn = (pp + 1) % NB2;
        const R2 *ut_c = ut_r + bc * sE, *h_c = h_r + bc * sC;
        const R2 *ut_nx = ut_r + bn * sE, *h_nx = h_r + bn * sC;

        cp_async_wait_n<NB2 - 3>();
        __syncthreads();   // pairs pp and pp + 1 in shared memory; pair pp - 1's readers done
        if (pp + NB2 - 1 < NP) issue(pp + NB2 - 1, (pp + NB2 - 1) % NB2);
        else cp_async_commit();
        // the old level at the owned edges (consecutive, so the loads
        // coalesce), read by the edge phase two barriers later
        R2 un2[NI];
#pragma unroll
        for (int s = 0; s < NI; s++) {
            un2[s].x = R(0); un2[s].y = R(0);
            if (comb && tid + s * NT < nE0) {
                un2[s].x = ldg(a.ut_n + (size_t)k0 * Ep + ge[s]);
                if (has1) un2[s].y = ldg(a.ut_n + (size_t)(k0 + 1) * Ep + ge[s]);
            }
        }
        // the tracers of this thread's C1 cells, read by the cell phase below
        // (the owned cells among them are consecutive)
        R2 T2s[NI], S2s[NI];
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const int c = ctid + s * NT;
            T2s[s].x = R(0); T2s[s].y = R(0); S2s[s] = T2s[s];
            if (c < nC1) {
                const R *T0 = a.tr + (size_t)k0 * Cp + cg[c];
                T2s[s].x = ldg(T0);
                if (has1) T2s[s].y = ldg(T0 + Cp);
                if (two) {
                    const R *S0 = T0 + (size_t)L * Cp;
                    S2s[s].x = ldg(S0);
                    if (has1) S2s[s].y = ldg(S0 + Cp);
                }
            }
        }
        // ---- vertices: relative vorticity, kite-averaged thickness, PV
        for (int v = tid; v < nV; v += NT) {
            R2 ot, hv;
            ot.x = R(0); ot.y = R(0); hv.x = R(0); hv.y = R(0);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int x = j * nV + v;
                const unsigned ec = x_vec[x];
                const R2 ck = x_vck[x];
                const R2 u2 = ut_c[ec & 0xffff], h2 = h_c[ec >> 16];
                ot.x += ck.x * u2.x;
                ot.y += ck.x * u2.y;
                hv.x += ck.y * h2.x;
                hv.y += ck.y * h2.y;
            }
            const R2 bf = x_vbf[v];
            R2 om, qv;
            om.x = bf.x + ot.x;
            om.y = bf.x + ot.y;
            qv.x = qdiv(bf.y + ot.x, hv.x);
            qv.y = qdiv(bf.y + ot.y, hv.y);
            om_s[v] = om;
            q_s[v] = qv;
        }
        // ---- cells of C1: K, div u, div(h_e u), rho', w
        const R sk0 = sf_s[k0], sk1 = has1 ? sf_s[k0 + 1] : R(0);
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const int c = ctid + s * NT;
            if (c < nC1) {
                const R2 hk = h_c[c];
                R2 ke, dl, dv;
                ke.x = R(0); ke.y = R(0); dl.x = R(0); dl.y = R(0); dv.x = R(0); dv.y = R(0);
#pragma unroll
                for (int j = 0; j < BCL_NCEP; j++) {
                    const int x = j * nC1 + c;
                    const unsigned eo = x_c1eo[x];
                    const int el = eo & 0xffff, ol = eo >> 16;
                    const R2 dk = x_c1dk[x];
                    const R ubl = ub_s[el];
                    const R2 ul = ut_c[el], ho = h_c[ol];
                    const R u0 = ubl + ul.x, u1 = ubl + ul.y;
                    const R he0 = R(0.5) * (hk.x + ho.x), he1 = R(0.5) * (hk.y + ho.y);
                    ke.x += dk.y * u0 * u0;
                    ke.y += dk.y * u1 * u1;
                    dl.x += dk.x * u0;
                    dl.y += dk.x * u1;
                    dv.x += dk.x * (he0 * u0);
                    dv.y += dk.x * (he1 * u1);
                }
                const R2 T2 = T2s[s];
                R2 rp;
                rp.x = -alpha * (T2.x - Tref);
                rp.y = -alpha * (T2.y - Tref);
                if (two) {
                    const R2 S2 = S2s[s];
                    rp.x += beta * (S2.x - Sref);
                    rp.y += beta * (S2.y - Sref);
                }
                cK[c] = ke;
                cR[c] = rp;
                cD[c] = dl;
                // w at the top of layers k0 + 1 and k0 + 2 (an absent second
                // layer's value is never read)
                R2 w1;
                W[s] += dv.x;
                w1.x = W[s] - (Sk + sk0) * dsum[s];
                W[s] += dv.y;
                w1.y = W[s] - (Sk + sk0 + sk1) * dsum[s];
                cW1[c] = w1;
            }
        }
        __syncthreads();
        // ---- edges of E1: (h_e u, q_e) of both layers
        for (int e = tid; e < nE1; e += NT) {
            const int cc = x_e1c[e], vv = x_e1v[e];
            const R2 h1 = h_c[cc & 0xffff], h2 = h_c[cc >> 16];
            const R2 qa = q_s[vv & 0xffff], qb = q_s[vv >> 16];
            const R ubl = ub_s[e];
            const R2 ul = ut_c[e];
            R4 hq;
            hq.x = R(0.5) * (h1.x + h2.x) * (ubl + ul.x);
            hq.y = R(0.5) * (qa.x + qb.x);
            hq.z = R(0.5) * (h1.y + h2.y) * (ubl + ul.y);
            hq.w = R(0.5) * (qa.y + qb.y);
            hq_s[e] = hq;
        }
        __syncthreads();
        // ---- owned edges: the tendencies of the pair's layers, in order
#pragma unroll
        for (int s = 0; s < NI; s++) {
            const int e = tid + s * NT;
            if (e >= nE0) continue;
            const int c1 = c12[s] & 0xffff, c2 = c12[s] >> 16;
            const int v1 = v12[s] & 0xffff, v2 = v12[s] >> 16;
            const R ube = ub_s[e];
            const R2 utc = ut_c[e];
            const R2 h1 = h_c[c1], h2 = h_c[c2];
            const R4 hqe = hq_s[e];
            R2 Q;
            Q.x = R(0); Q.y = R(0);
#pragma unroll
            for (int j = 0; j < BCL_NE2P; j++) {
                const int x = j * nE0 + e;
                const R w = x_e0w[x];
                const R4 nb = hq_s[x_e0i[x]];
                Q.x += w * nb.x * (R(0.5) * (hqe.y + nb.y));
                Q.y += w * nb.z * (R(0.5) * (hqe.w + nb.w));
            }
            const R2 K1 = cK[c1], K2 = cK[c2], P1 = cR[c1], P2 = cR[c2];
            const R2 D1 = cD[c1], D2 = cD[c2], o1 = om_s[v1], o2 = om_s[v2];
            const R2 W1 = cW1[c1], W2 = cW1[c2];
            // the layer below the pair: the first of the next pair
            R utn = R(0), h1n = R(0), h2n = R(0);
            if (k0 + 2 < L) {
                utn = ut_nx[e].x;
                h1n = h_nx[c1].x;
                h2n = h_nx[c2].x;
            }
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int k = k0 + i;
                if (k >= L) break;
                const R ut_cur = i ? utc.y : utc.x;
                const R hh1 = i ? h1.y : h1.x, hh2 = i ? h2.y : h2.x;
                const R u_cur = ube + ut_cur;
                const R he_cur = R(0.5) * (hh1 + hh2);
                const R gradK = ((i ? K2.y : K2.x) - (i ? K1.y : K1.x)) * idc[s];
                // p'_2 - p'_1 and z_2 - z_1 (z = zeta - sum_{l<k} h_l - h_k / 2)
                const R r1 = i ? P1.y : P1.x, r2 = i ? P2.y : P2.x;
                const R rh = r2 * hh2 - r1 * hh1;
                const R dp = g * (dA[s] + R(0.5) * rh);
                const R dz = dzeta[s] - dH[s] - R(0.5) * (hh2 - hh1);
                const R pgf = (dp + g * (R(0.5) * (r1 + r2)) * dz) * idc[s] * inv_rho0;
                dA[s] += rh;
                dH[s] += hh2 - hh1;
                R Dk1 = R(0), wk1 = R(0);
                if (k + 1 < L) {
                    const R u_next = ube + (i ? utn : utc.y);
                    const R he_next = R(0.5) * (i ? h1n + h2n : h1.y + h2.y);
                    Dk1 = qdiv(u_cur - u_next, R(0.5) * (he_cur + he_next));
                    wk1 = R(0.5) * (i ? W1.y + W2.y : W1.x + W2.x);
                }
                const R vadv = R(0.5) * (wk[s] * Dk[s] + wk1 * Dk1);
                R Xtop = nu_v * Dk[s];
                if (k == 0) Xtop = wnd ? wnd[ge[s]] : R(0);
                R Xbot;
                if (k == L - 1) {
                    R utan = R(0);
#pragma unroll
                    for (int j = 0; j < BCL_NE2P; j++) {
                        const int x = j * nE0 + e;
                        const int el = x_e0i[x];
                        const R2 ul = ut_c[el];
                        utan += x_e0w[x] * (ub_s[el] + (i ? ul.y : ul.x));
                    }
                    Xbot = cdrag * sqrt(u_cur * u_cur + utan * utan) * u_cur;
                } else {
                    Xbot = nu_v * Dk1;
                }
                const R vvisc = qdiv(Xtop - Xbot, he_cur);
                const R lap = ((i ? D2.y : D2.x) - (i ? D1.y : D1.x)) * idc[s] -
                              ((i ? o2.y : o2.x) - (i ? o1.y : o1.x)) * idv[s];
                const R gzeta = q.zcoef * dzeta[s] * idc[s];
                const R rhs = ((i ? Q.y : Q.x) - cbar[s]) - gradK - pgf - vadv + nu_h * lap +
                              vvisc + gzeta;
                const R ut1 = ut_cur + dt * rhs;
                num[s] += he_cur * ut1;
                den[s] += he_cur;
                const R unk = i ? un2[s].y : un2[s].x;
                a.ut_out[(size_t)k * Ep + ge[s]] = comb ? ca * unk + cb * ut1 : cb * ut1;
                Dk[s] = Dk1;
                wk[s] = wk1;
            }
        }
        Sk = (Sk + sk0) + sk1;
    }
    cp_async_wait_all();
    // ---- G and the subtraction of dt G over the owned columns.  The loads of
    // KB layers of both slots are issued before any store, so that a thread
    // waits for L / KB round trips to global memory instead of NI * L.
    R corr[NI];
#pragma unroll
    for (int s = 0; s < NI; s++) {
        const int e = tid + s * NT;
        corr[s] = R(0);
        if (e < nE0) {
            const R G = num[s] / den[s] / dt;
            a.G[ge[s]] = G;
            corr[s] = cb * dt * G;
        }
    }
    constexpr int KB = 4;
    for (int k0 = 0; k0 < L; k0 += KB) {
        R v[NI][KB];
#pragma unroll
        for (int s = 0; s < NI; s++) {
#pragma unroll
            for (int r = 0; r < KB; r++) {
                if (tid + s * NT < nE0 && k0 + r < L)
                    v[s][r] = a.ut_out[(size_t)(k0 + r) * Ep + ge[s]];
            }
        }
#pragma unroll
        for (int s = 0; s < NI; s++) {
#pragma unroll
            for (int r = 0; r < KB; r++) {
                if (tid + s * NT < nE0 && k0 + r < L)
                    a.ut_out[(size_t)(k0 + r) * Ep + ge[s]] = v[s][r] - corr[s];
            }
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
__global__ void __launch_bounds__(NT, bcl_min_blocks<R>()) k_bcl_fused(const BclJob<R> job) {
    __shared__ BclJob<R> J;
    copy_job(J, job);
    __syncthreads();
    bcl_fused_patch<R, NT, NI>(J.m, J.p, J.t, J.a, blockIdx.x);
}
template <class R, int NT, int NI>
__global__ void __launch_bounds__(NT, bcl_min_blocks<R>()) k_bcl_fused_batch(const BclJob<R> *__restrict__ jobs,
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

// bytes of one patch's shared-memory image: the arrays in the order the kernel
// carves them, each rounded up to 16 bytes
template <class R> static size_t image_bytes(int nE0, int nE1, int nE2, int nC1, int nC2, int nV) {
    auto a16 = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t sR = sizeof(R);
    return a16(2 * BCL_NE2P * (size_t)nE0) + a16(sR * BCL_NE2P * (size_t)nE0) +
           a16(4 * BCL_NCEP * (size_t)nC1) + a16(2 * sR * BCL_NCEP * (size_t)nC1) +
           a16(4 * 3 * (size_t)nV) + a16(2 * sR * 3 * (size_t)nV) + 2 * a16(4 * (size_t)nE1) +
           a16(4 * (size_t)nE2) + a16(4 * (size_t)nC2);
}

template <class R>
size_t bcl_build_image(const BclPlan &pl, std::vector<unsigned char> &img,
                       std::vector<long long> &off) {
    using R2 = V2<R>;
    img.clear();
    off.assign(1, 0);
    size_t best = 0;
    for (int p = 0; p < pl.P; p++) {
        const int *n = &pl.cnt[8 * p];
        const int nE0 = n[0], nE1 = n[1], nE2 = n[2], nC1 = n[3], nC2 = n[4], nV = n[5];
        const size_t bytes = image_bytes<R>(nE0, nE1, nE2, nC1, nC2, nV);
        best = std::max(best, bytes);
        const size_t base = img.size();
        img.resize(base + bytes, 0);
        unsigned char *q = img.data() + base;
        auto put = [&](const void *src, size_t len) {
            std::memcpy(q, src, len);
            q += (len + 15) / 16 * 16;
        };
        const int oe0 = pl.off_e0[p], oe1 = pl.off_e1[p], oc1 = pl.off_c1[p], ov = pl.off_v[p];
        put(&pl.e0_eoe[(size_t)BCL_NE2P * oe0], 2 * (size_t)BCL_NE2P * nE0);
        std::vector<R> w(pl.e0_wl.begin() + (size_t)BCL_NE2P * oe0,
                         pl.e0_wl.begin() + (size_t)BCL_NE2P * (oe0 + nE0));
        put(w.data(), sizeof(R) * w.size());
        std::vector<uint32_t> eo((size_t)BCL_NCEP * nC1);
        std::vector<R2> dk((size_t)BCL_NCEP * nC1);
        for (size_t j = 0; j < eo.size(); j++) {
            const size_t x = (size_t)BCL_NCEP * oc1 + j;
            eo[j] = (uint32_t)pl.c1_e[x] | ((uint32_t)pl.c1_o[x] << 16);
            dk[j].x = (R)pl.c1_divc[x];
            dk[j].y = (R)pl.c1_kec[x];
        }
        put(eo.data(), 4 * eo.size());
        put(dk.data(), sizeof(R2) * dk.size());
        std::vector<uint32_t> ec((size_t)3 * nV);
        std::vector<R2> ck((size_t)3 * nV);
        for (size_t j = 0; j < ec.size(); j++) {
            const size_t x = (size_t)3 * ov + j;
            ec[j] = (uint32_t)pl.v_e[x] | ((uint32_t)pl.v_c[x] << 16);
            ck[j].x = (R)pl.v_curl[x];
            ck[j].y = (R)pl.v_kw[x];
        }
        put(ec.data(), 4 * ec.size());
        put(ck.data(), sizeof(R2) * ck.size());
        put(&pl.e1_c12[oe1], 4 * (size_t)nE1);
        put(&pl.e1_v12[oe1], 4 * (size_t)nE1);
        put(&pl.egid[pl.off_e2[p]], 4 * (size_t)nE2);
        put(&pl.cgid[pl.off_c2[p]], 4 * (size_t)nC2);
        off.push_back((long long)img.size());
    }
    return best;
}

template <class R> size_t bcl_smem_bytes(const BclPlan &plan, int L) {
    auto a16 = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t sR = sizeof(R);
    size_t b = 0;
    b += a16(sR * (plan.maxE2 + 1));                   // ubar
    b += NB2 * a16(2 * sR * (plan.maxE2 + 1));         // utilde (pair ring)
    b += NB2 * a16(2 * sR * (plan.maxC2 + 1));         // h
    // (each ring is carved as one block of NB2 16-byte padded strides)
    b += 2 * a16(2 * sR * plan.maxV);                  // q, omega
    b += a16(4 * sR * (plan.maxE1 + 1));               // (h_e u, q_e) x 2
    b += 4 * a16(2 * sR * plan.maxC1);                 // K, rho', w, div u
    b += a16(2 * sR * plan.maxV);                      // curl ubar (+ f)
    b += a16(sR * L);                                  // s_k
    size_t img = 0;                                    // the largest patch image
    for (int p = 0; p < plan.P; p++) {
        const int *n = &plan.cnt[8 * p];
        img = std::max(img, image_bytes<R>(n[0], n[1], n[2], n[3], n[4], n[5]));
    }
    return b + img;
}
template <class R> int bcl_blocks_per_sm() { return bcl_min_blocks<R>(); }
template int bcl_blocks_per_sm<float>();
template int bcl_blocks_per_sm<double>();
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
template size_t bcl_smem_bytes<float>(const BclPlan &, int);
template size_t bcl_smem_bytes<double>(const BclPlan &, int);
template size_t bcl_build_image<float>(const BclPlan &, std::vector<unsigned char> &,
                                       std::vector<long long> &);
template size_t bcl_build_image<double>(const BclPlan &, std::vector<unsigned char> &,
                                        std::vector<long long> &);
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
