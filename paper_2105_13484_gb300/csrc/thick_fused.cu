// thick_fused.cu -- the thickness and tracer stage (Eqs. layerthickness,
// tracer, with the transport velocity of Sec. 3.4) as one patch-tiled kernel
// (sm_103a).
//
// The unfused path writes the per-layer edge mass flux h_e (v + u^A) from the
// transport kernel and gathers it back, six edges per cell-layer, in a
// one-thread-per-column kernel whose every layer waits on several rounds of
// gathers.  Here the transport kernel leaves only 2-D results (u^A and the
// FP64 column flux), and one CTA per patch of consecutive cells walks the
// layers from the top with each layer's velocities (at the patch's edges)
// and thickness and tracers (at its cells and their neighbours) staged in
// shared memory by cp.async (a ring of four layers, two ahead of the one
// being computed), and each owned cell's own stage and old levels loaded by
// its thread (the owned cells are consecutive, so those loads coalesce); the
// flux is formed in registers from them.  One barrier per layer.
#include "sse_internal.cuh"
#include "tiles.h"

namespace sse {

namespace {

template <class R> __device__ __forceinline__ R ldg(const R *p) { return __ldg(p); }

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
template <class T> __device__ __forceinline__ void cp_async(T *dst, const T *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(src),
                 "n"(sizeof(T)));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
// layers staged in shared memory: k and k + 1 in use, k + 2 and k + 3 in flight
constexpr int NBUF = 4;

template <class R> __device__ __forceinline__ const R *sfr_of(const DMesh &m);
template <> __device__ __forceinline__ const double *sfr_of<double>(const DMesh &m) { return m.sfrac; }
template <> __device__ __forceinline__ const float *sfr_of<float>(const DMesh &m) { return m.sfrac_f; }

// a / b for the vertical-diffusion quotients: correctly rounded in FP64; in
// FP32 the reciprocal-multiply form (within 2 ulp for the divisors met here,
// thicknesses of 1e-3 to 1e4 m).  The tracer values themselves keep IEEE
// division.
template <class R> __device__ __forceinline__ R qdiv(R a, R b);
template <> __device__ __forceinline__ double qdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float qdiv<float>(float a, float b) { return __fdividef(a, b); }

// elements of T in n rounded up to 16 bytes
template <class T> __host__ __device__ __forceinline__ int pad16(int n) {
    return (int)(((size_t)n * sizeof(T) + 15) / 16 * 16 / sizeof(T));
}
template <class T> __device__ __forceinline__ T *carve(char *&p, int n) {
    T *r = reinterpret_cast<T *>(p);
    p += ((size_t)n * sizeof(T) + 15) / 16 * 16;
    return r;
}

}  // namespace

// ---------------------------------------------------------------------------
// Sec. 3.4 per edge, columns only: F^h = cF sum_k v_k h_e,k + cE (extra
// terms), D = F^zeta - F^h, u^A = cA D / sum_k h_e,k; the column flux
// F_col = sum_k v h_e + u^A sum_k h_e (FP64) and u^A in the tendency
// precision.  Sums as in k_transport (a float pair in the mixed form).
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void transport_cols_edge(const DMesh &m, const TransportArgs<R> &a,
                                                    R *uA_out, const int e) {
    if (e >= m.E) return;
    const int Ep = m.Ep, Cp = m.Cp, L = m.L;
    const int2 cc = m.coe[e];
    const R ubA = a.ubA[e];
    const R ubB = a.ubB ? a.ubB[e] : R(0);
    const R wA = (R)a.wA, wB = (R)a.wB;
    const bool twoB = a.utB != nullptr;
    PairSum<R> Sacc;
    // layers in chunks of KC, every load of a chunk issued before its sums
    // (which still run over k in order)
    constexpr int KC = 4;
    for (int k0 = 0; k0 < L; k0 += KC) {
        R h1[KC], h2[KC], xa[KC], xb[KC];
#pragma unroll
        for (int j = 0; j < KC; j++) {
            const int k = k0 + j < L ? k0 + j : L - 1;
            h1[j] = ldg(a.hR + k * Cp + cc.x);
            h2[j] = ldg(a.hR + k * Cp + cc.y);
            xa[j] = ldg(a.utA + k * Ep + e);
            xb[j] = twoB ? ldg(a.utB + k * Ep + e) : R(0);
        }
#pragma unroll
        for (int j = 0; j < KC; j++) {
            if (k0 + j >= L) break;
            const R he = R(0.5) * (h1[j] + h2[j]);
            R v = wA * (ubA + xa[j]);
            if (twoB) v += wB * (ubB + xb[j]);
            Sacc.add(v * he);
        }
    }
    const double S = Sacc.value();
    const double hs = 0.5 * ((a.zeta[cc.x] + m.H[cc.x]) + (a.zeta[cc.y] + m.H[cc.y]));
    double Fh = a.cF * S;
    if (a.ex1) Fh += a.cE * a.ex1[e];
    if (a.ex2) Fh += a.cE * a.ex2[e];
    const double uA = a.recon ? a.cA * (a.Fz[e] - Fh) / hs : 0.0;
    if (a.S_out) a.S_out[e] = S;
    a.Fcol[e] = S + uA * hs;
    uA_out[e] = (R)uA;
}

// ---------------------------------------------------------------------------
// The fused thickness/tracer stage.  One CTA of NT threads per patch; owned
// cell l is thread l.  Per layer, with flux_e = h_e (v_e + u^A_e):
//   w_{k+1} = w_k + div(flux)_k - s_k D,  D = div(F_col)   (z-star, from the top)
//   h1 = h_s - s_k dt D (FP64),  h_out = a h^n + b h1
//   (h phi)1 = h phi + dt (-div(flux phi_e) - (phibar_k w_k - phibar_{k+1} w_{k+1})
//              + div(h_e kappa_h grad phi) + kappa_v (D_zt phi_k - D_zt phi_{k+1}))
//   phi_out = (a h^n phi^n + b h1 phi1) / h_out
// the same arithmetic as k_thickness, in the same precisions.
// ---------------------------------------------------------------------------
template <class R, int NT>
__device__ __forceinline__ void thick_fused_patch(const DMesh &m, const DParams &p, const DThick &t,
                                                  const ThickFArgs<R> &a, const int pid) {
    const int l = threadIdx.x;
    const int *cn = t.cnt + 4 * pid;
    const int nO = cn[0], nEO = cn[1], nC1 = cn[2];
    const int *eg_g = t.eogid + t.off_eo[pid];
    const int *cg_g = t.c1gid + t.off_c1[pid];

    const int Ep = m.Ep, Cp = m.Cp, L = m.L, Pc = t.Pc;
    const int nT = p.nT;
    const bool twoB = a.utB != nullptr, comb = a.a != 0.0;
    const PhysR<R> &q = phys<R>(p);

    extern __shared__ __align__(16) char smem[];
    char *sp = smem;
    const int sE = pad16<R>(t.maxEO + 1), sC = pad16<R>(t.maxC1);
    R *vb_s = carve<R>(sp, t.maxEO + 1);       // wA ubA + wB ubB + u^A per edge (0: zero slot)
    R *uA_r = carve<R>(sp, NBUF * sE);            // utA, NBUF layers
    R *uB_r = carve<R>(sp, twoB ? NBUF * sE : 1); // utB
    R *h_r = carve<R>(sp, NBUF * sC);             // hR_s at C1
    R *tr_r = carve<R>(sp, NBUF * nT * sC);       // tracers at C1, [layer][t][C1]
    int *eg = carve<int>(sp, t.maxEO);   // the patch's internal indices
    int *cg = carve<int>(sp, t.maxC1);
    for (int j = l; j < nEO; j += NT) eg[j] = eg_g[j];
    for (int j = l; j < nC1; j += NT) cg[j] = cg_g[j];
    __syncthreads();

    auto issue = [&](int k, int b) {
        for (int j = l; j < nEO; j += NT) {
            cp_async(uA_r + b * sE + j, a.utA + (size_t)k * Ep + eg[j]);
            if (twoB) cp_async(uB_r + b * sE + j, a.utB + (size_t)k * Ep + eg[j]);
        }
        for (int j = l; j < nC1; j += NT) {
            cp_async(h_r + b * sC + j, a.hR_s + (size_t)k * Cp + cg[j]);
            for (int tt = 0; tt < nT; tt++)
                cp_async(tr_r + (b * nT + tt) * sC + j, a.tr_s + ((size_t)tt * L + k) * Cp + cg[j]);
        }
        cp_async_commit();
    };
    for (int k = 0; k < NBUF - 1; k++) {   // layers 0, 1, 2 in flight
        if (k < L) issue(k, k);
        else cp_async_commit();
    }
    // the per-edge 2-D part of the transport velocity
    const R wA = (R)a.wA, wB = (R)a.wB;
    for (int j = l; j < nEO; j += NT) {
        const int e = eg[j];
        R v = wA * ldg(a.ubA + e) + ldg(a.uA + e);
        if (twoB) v += wB * ldg(a.ubB + e);
        vb_s[j] = v;
    }
    if (l == 0) {
        // the zero slot that stands in for a pentagon's absent sixth edge
        vb_s[nEO] = R(0);
        for (int b = 0; b < NBUF; b++) {
            uA_r[b * sE + nEO] = R(0);
            if (twoB) uB_r[b * sE + nEO] = R(0);
        }
    }

    // the owned cell's connectivity and column data
    const bool own = l < nO;
    const int i = own ? cg[l] : 0;
    int es[BCL_NCEP], os[BCL_NCEP];
    R dcf[BCL_NCEP], idc[BCL_NCEP];
    double D = 0.0;
#pragma unroll
    for (int j = 0; j < BCL_NCEP; j++) {
        es[j] = t.o_e[(size_t)BCL_NCEP * Pc * pid + (size_t)j * Pc + l];
        os[j] = t.o_o[(size_t)BCL_NCEP * Pc * pid + (size_t)j * Pc + l];
        dcf[j] = R(0); idc[j] = R(0);
        if (own && j < m.neoc[i]) {
            const int e = eg[es[j]];
            dcf[j] = coef<R>(m).divc[j * Cp + i];
            idc[j] = coef<R>(m).invdc[e];
            D += m.divc_d[j * Cp + i] * a.Fcol[e];
        }
    }
    const R Dr = (R)D;
    const double dtD = a.dt * D;
    const R *sfr = sfr_of<R>(m);
    const R dtR = (R)a.dt, aR = (R)a.a, bR = (R)a.b, kh = q.kappa_h, kv = q.kappa_v;
    const bool khz = p.kappa_h != 0.0;
    double hsum = 0.0;
    R wk = R(0), hs_prev = R(0);
    R ph_prev0 = R(0), ph_prev1 = R(0);   // the tracers one layer up

    for (int k = 0; k < L; k++) {
        const int bc = k % NBUF, bn = (k + 1) % NBUF;
        cp_async_wait_1();
        __syncthreads();   // layers k and k + 1 staged; layer k - 1's readers done
        if (k + 3 < L) issue(k + 3, (k + 3) % NBUF);
        else cp_async_commit();
        if (!own) continue;
        // the owned cell's own stage and old levels: coalesced loads (the
        // owned cells are consecutive), used after the flux loop below
        const size_t x = (size_t)k * Cp + i;
        const double hs_d = a.h_s[x];
        double hn = 0.0;
        R hnr = R(0), trn0 = R(0), trn1 = R(0);
        if (comb) {
            hn = a.h_n[x];
            hnr = a.hR_n[x];
            trn0 = a.tr_n[x];
            if (nT > 1) trn1 = a.tr_n[(size_t)L * Cp + x];
        }
        const R *uA_c = uA_r + bc * sE, *uB_c = uB_r + bc * sE, *h_c = h_r + bc * sC;
        const R hs_cur = h_c[l];
        const R hs_next = (k + 1 < L) ? h_r[bn * sC + l] : R(0);
        // flux at the cell's edges and its divergence
        R fl[BCL_NCEP];
        R divk = R(0);
#pragma unroll
        for (int j = 0; j < BCL_NCEP; j++) {
            const int el = es[j];
            R v = vb_s[el] + wA * uA_c[el];
            if (twoB) v += wB * uB_c[el];
            fl[j] = R(0.5) * (hs_cur + h_c[os[j]]) * v;
            divk += dcf[j] * fl[j];
        }
        const R sk = sfr[k];
        const R wk1 = (k + 1 < L) ? wk + divk - sk * Dr : R(0);
        // thickness in FP64 from the column-integrated flux (volume conservation)
        const double h1 = hs_d - m.sfrac[k] * dtD;
        const double hout = comb ? a.a * hn + a.b * h1 : h1;
        const R h1r = hs_cur - sk * (dtR * Dr);
        const R houtr = comb ? aR * hnr + bR * h1r : h1r;
#pragma unroll
        for (int tt = 0; tt < 2; tt++) {
            if (tt >= nT) break;
            const R *phi = tr_r + (bc * nT + tt) * sC;
            const R ph = phi[l];
            R adv = R(0), dif = R(0);
#pragma unroll
            for (int j = 0; j < BCL_NCEP; j++) {
                const R po = phi[os[j]];
                adv += dcf[j] * (fl[j] * (R(0.5) * (ph + po)));
                if (khz) {
                    const R he = R(0.5) * (hs_cur + h_c[os[j]]);
                    dif += fabs(dcf[j]) * he * kh * (po - ph) * idc[j];
                }
            }
            R ftop = R(0), fbot = R(0), dtop = R(0), dbot = R(0);
            if (k >= 1) {
                const R pu = tt ? ph_prev1 : ph_prev0;
                ftop = R(0.5) * (pu + ph) * wk;
                dtop = qdiv(pu - ph, R(0.5) * (hs_prev + hs_cur));
            }
            if (k + 1 < L) {
                const R pd = tr_r[(bn * nT + tt) * sC + l];
                fbot = R(0.5) * (ph + pd) * wk1;
                dbot = qdiv(ph - pd, R(0.5) * (hs_cur + hs_next));
            }
            const R hphi = hs_cur * ph + dtR * (-adv - (ftop - fbot) + dif + kv * (dtop - dbot));
            // the tracer itself: correctly rounded (a 2-ulp quotient here,
            // applied every stage, grows into the density and the velocity)
            const R phi1 = hphi / h1r;
            R out;
            if (comb)
                out = (aR * hnr * (tt ? trn1 : trn0) + bR * h1r * phi1) / houtr;
            else
                out = phi1;
            a.tr_out[(size_t)tt * L * Cp + x] = out;
            if (tt) ph_prev1 = ph; else ph_prev0 = ph;
        }
        a.h_out[x] = hout;
        if (a.hR_out) a.hR_out[x] = houtr;
        hsum += hout;
        wk = wk1;
        hs_prev = hs_cur;
    }
    cp_async_wait_all();
    if (own) a.zeta_out[i] = hsum - m.H[i];
}


// ---------------------------------------------------------------------------
// batched launches (see bcl_fused.cu): job j owns blocks [first[j], first[j+1])
// ---------------------------------------------------------------------------
__device__ __forceinline__ int job_of_block_t(const int *first, int njobs) {
    int lo = 0, hi = njobs - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}
template <class T> __device__ __forceinline__ void copy_job_t(T &dst, const T &src) {
    static_assert(sizeof(T) % 4 == 0, "job descriptors are copied in 4-byte words");
    const int *s = reinterpret_cast<const int *>(&src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
}
// single-state and batched kernels run the body on a shared-memory copy of
// their descriptor, so that the body compiles identically in both (a state's
// results are the same bits alone or in a batch)
//
// Resident CTAs per SM asked of the compiler.  A patch is 128 cells, so the
// level-7 sphere's 114,689 ocean cells make 925 CTAs: at the 96 registers the
// FP32 body takes unbounded, 5 CTAs fit an SM (760 on 152 SMs) and the launch
// runs 1.22 waves, its second a fifth full; at 7 (72 registers) the grid is
// one wave.  0 leaves the FP64 body's register count to the compiler.
template <class R> constexpr int thick_min_blocks() { return sizeof(R) == 4 ? 7 : 0; }
template <class R, int NT>
__global__ void __launch_bounds__(NT, thick_min_blocks<R>()) k_thick_fused(const ThickJob<R> job) {
    __shared__ ThickJob<R> J;
    copy_job_t(J, job);
    __syncthreads();
    thick_fused_patch<R, NT>(J.m, J.p, J.t, J.a, blockIdx.x);
}
template <class R, int NT>
__global__ void __launch_bounds__(NT, thick_min_blocks<R>()) k_thick_fused_batch(const ThickJob<R> *__restrict__ jobs,
                                                          const int *__restrict__ first,
                                                          int njobs) {
    __shared__ ThickJob<R> J;
    const int j = job_of_block_t(first, njobs);
    copy_job_t(J, jobs[j]);
    __syncthreads();
    thick_fused_patch<R, NT>(J.m, J.p, J.t, J.a, blockIdx.x - first[j]);
}
template <class R>
__global__ void __launch_bounds__(128) k_transport_cols(const TransportJob<R> job) {
    __shared__ TransportJob<R> J;
    copy_job_t(J, job);
    __syncthreads();
    transport_cols_edge<R>(J.m, J.a, J.uA, blockIdx.x * blockDim.x + threadIdx.x);
}
template <class R>
__global__ void __launch_bounds__(128) k_transport_cols_batch(const TransportJob<R> *__restrict__ jobs,
                                                              const int *__restrict__ first,
                                                              int njobs) {
    __shared__ TransportJob<R> J;
    const int j = job_of_block_t(first, njobs);
    copy_job_t(J, jobs[j]);
    __syncthreads();
    transport_cols_edge<R>(J.m, J.a, J.uA, (blockIdx.x - first[j]) * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
constexpr int THICK_NT = 128;   // = cells per patch

size_t thick_smem_bytes(const DThick &plan, int nT, bool twoB, bool comb, size_t sR) {
    auto a16 = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t Pc = plan.Pc;
    const size_t NB = NBUF;
    size_t b = a16(sR * (plan.maxEO + 1));
    b += NB * a16(sR * (plan.maxEO + 1)) * (twoB ? 2 : 1) + (twoB ? 0 : 16);
    b += NB * a16(sR * plan.maxC1) * (1 + nT);
    b += a16(4 * (size_t)plan.maxEO) + a16(4 * (size_t)plan.maxC1);
    (void)Pc;
    (void)comb;
    return b;
}
int thick_cells_per_patch() { return THICK_NT; }
template <class R> const void *thick_fused_kernel_ptr() { return (const void *)k_thick_fused<R, THICK_NT>; }

template <class R>
void launch_transport_cols(const DMesh &m, const TransportArgs<R> &a, R *uA, cudaStream_t s) {
    const TransportJob<R> job{m, a, uA};
    k_transport_cols<R><<<(m.E + 127) / 128, 128, 0, s>>>(job);
}
template <class R>
void launch_thick_fused(const DThick &t, const DMesh &m, const DParams &p, const ThickFArgs<R> &a,
                        size_t smem, cudaStream_t s) {
    const ThickJob<R> job{m, p, t, a};
    k_thick_fused<R, THICK_NT><<<t.P, THICK_NT, smem, s>>>(job);
}

template <class R>
void launch_transport_cols_batch(const TransportJob<R> *jobs, const int *first, int njobs,
                                 int blocks, cudaStream_t s) {
    k_transport_cols_batch<R><<<blocks, 128, 0, s>>>(jobs, first, njobs);
}
template <class R>
void launch_thick_fused_batch(const ThickJob<R> *jobs, const int *first, int njobs, int blocks,
                              size_t smem, cudaStream_t s) {
    k_thick_fused_batch<R, THICK_NT><<<blocks, THICK_NT, smem, s>>>(jobs, first, njobs);
}
template <class R> const void *thick_fused_batch_kernel_ptr() {
    return (const void *)k_thick_fused_batch<R, THICK_NT>;
}
template void launch_transport_cols_batch<float>(const TransportJob<float> *, const int *, int,
                                                 int, cudaStream_t);
template void launch_transport_cols_batch<double>(const TransportJob<double> *, const int *, int,
                                                  int, cudaStream_t);
template void launch_thick_fused_batch<float>(const ThickJob<float> *, const int *, int, int,
                                              size_t, cudaStream_t);
template void launch_thick_fused_batch<double>(const ThickJob<double> *, const int *, int, int,
                                               size_t, cudaStream_t);
template const void *thick_fused_batch_kernel_ptr<float>();
template const void *thick_fused_batch_kernel_ptr<double>();
template const void *thick_fused_kernel_ptr<float>();
template const void *thick_fused_kernel_ptr<double>();
template void launch_transport_cols<float>(const DMesh &, const TransportArgs<float> &, float *,
                                           cudaStream_t);
template void launch_transport_cols<double>(const DMesh &, const TransportArgs<double> &, double *,
                                            cudaStream_t);
template void launch_thick_fused<float>(const DThick &, const DMesh &, const DParams &,
                                        const ThickFArgs<float> &, size_t, cudaStream_t);
template void launch_thick_fused<double>(const DThick &, const DMesh &, const DParams &,
                                         const ThickFArgs<double> &, size_t, cudaStream_t);

}  // namespace sse
