// btr_kernel.cu -- the barotropic sub-cycle (Algorithms 3 and 4) as one
// persistent cooperative kernel (sm_103a).
//
// Every forward-Euler sub-stage of the 2-D system
//     ubar <- ubar + tau (C_f(ubar) - g grad zeta + G)
//     zeta <- zeta - tau div(ubar (zeta + H)_e)
// reads the previous sub-stage everywhere and writes only its own edges and
// cells, so one grid-wide barrier separates consecutive sub-stages: 2M
// barriers for Algorithm 3 and 3M for Algorithm 4.  The SSPRK convex
// combinations only touch a thread's own entries and are folded into the
// sub-stage that produces them.  The accumulated flux F^zeta of Sec. 3.4 is
// summed in FP64 by the owner of each edge.
//
// The barrier spins with a bounded budget: if it runs out (a block never
// arrives), the kernel records an error word and returns instead of hanging.
#include <mutex>

#include "../../include/sse.h"
#include "sse_internal.cuh"
#include "tiles.h"

namespace sse {

constexpr int BTR_THREADS = 512;
constexpr long long BARRIER_SPIN_NS = 2000000000LL;  // 2 s

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier.  `count` grows by one per arriving block and is never
// reset inside a launch: barrier number b (0-based) is complete when count
// reaches (b+1) * nblocks, which its last arriver publishes by releasing
// gen = b+1.  Waiters poll gen with acquire loads (no atomics).  Returns
// false, after setting *err, if the wait exceeded its budget.
__device__ __forceinline__ bool grid_barrier(const Barrier &bar, unsigned int &gen_local,
                                             unsigned int nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int g0 = gen_local;
        const unsigned int old = atom_add_acq_rel(bar.count, 1u);
        if (old == (g0 + 1) * nblocks - 1) {
            st_release(bar.gen, g0 + 1);
        } else {
            const unsigned long long t0 = gtimer();
            unsigned int spins = 0;
            while (ld_acquire(bar.gen) == g0) {
                if ((++spins & 255u) == 0) {
                    if (ld_acquire((const unsigned int *)bar.err) ||
                        gtimer() - t0 > (unsigned long long)BARRIER_SPIN_NS) {
                        atomicExch(bar.err, 1);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(20);
            }
        }
        gen_local = g0 + 1;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Split-phase grid barrier over the same count word: grid_arrive releases
// this block's earlier writes and adds one arrival without waiting for the
// reply; grid_wait returns once `target` arrivals are in (acquire), so a block
// can do work that needs no other block's data in between.  Both are called
// by every thread of the block; the block's last thread arrives and polls.
// grid_wait returns false, after setting *err, if the wait exceeded its
// budget.
__device__ __forceinline__ void grid_arrive(const Barrier &bar) {
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1)
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar.count) : "memory");
}
__device__ __forceinline__ bool grid_wait(const Barrier &bar, unsigned int target) {
    __shared__ int s_ok;
    if (threadIdx.x == blockDim.x - 1) {
        int ok = 1;
        const unsigned long long t0 = gtimer();
        unsigned int spins = 0;
        while (ld_acquire(bar.count) < target) {
            if ((++spins & 255u) == 0) {
                if (ld_acquire((const unsigned int *)bar.err) ||
                    gtimer() - t0 > (unsigned long long)BARRIER_SPIN_NS) {
                    atomicExch(bar.err, 1);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(20);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

constexpr int BTR_NIT = 8;    // edges (and cells) owned per thread, at most
constexpr int BTR_NE2 = 10;   // edgesOnEdge handled by the unrolled gather

// Per-edge forward-Euler stage of the barotropic momentum equation:
//   ubar_new = ubar + tau (C_f(ubar) - g grad zeta + G)
// and the flux ubar (zeta + H)_e of the input state.  Loads of the constant
// mesh data go through the read-only path; loads of the evolving 2-D state
// bypass L1 (__ldcg) because other blocks wrote them before the barrier.
template <class R, int NE2>
__device__ __forceinline__ R fe_edge(const DMesh &m, const Coef<R> &c, int e, const R *u,
                                     const R *z, R Ge, R tau, R g, R &flux) {
    const int Ep = m.Ep;
    const int n2 = __ldg(m.neoe + e);
    R cf = R(0);
#pragma unroll
    for (int j = 0; j < NE2; j++)
        if (j < n2) cf += __ldg(c.cfc + j * Ep + e) * __ldcg(u + __ldg(m.eoe + j * Ep + e));
    const int2 cc = __ldg(m.coe + e);
    const R ue = __ldcg(u + e);
    const R z1 = __ldcg(z + cc.x), z2 = __ldcg(z + cc.y);
    const R d1 = z1 + __ldg(c.H + cc.x), d2 = z2 + __ldg(c.H + cc.y);
    flux = ue * (R(0.5) * (d1 + d2));
    return ue + tau * (cf - g * (z2 - z1) * __ldg(c.invdc + e) + Ge);
}

// Per-cell forward-Euler stage of the barotropic continuity equation:
//   zeta_new = zeta - tau div(ubar (zeta + H)_e), the edge depth in c1,c2 order
template <class R>
__device__ __forceinline__ R fe_cell(const DMesh &m, const Coef<R> &c, int i, const R *u,
                                     const R *z, R tau) {
    const int Cp = m.Cp;
    const int ne = __ldg(m.neoc + i);
    const R zi = __ldcg(z + i), di = zi + __ldg(c.H + i);
    R dv = R(0);
#pragma unroll
    for (int j = 0; j < MAXE; j++) {
        if (j < ne) {
            const int e = __ldg(m.eoc + j * Cp + i), o = __ldg(m.ooc + j * Cp + i);
            const R cj = __ldg(c.divc + j * Cp + i);
            const R dov = __ldcg(z + o) + __ldg(c.H + o);
            const R de = (cj > R(0)) ? (di + dov) : (dov + di);
            dv += cj * (__ldcg(u + e) * (R(0.5) * de));
        }
    }
    return zi - tau * dv;
}

// The sub-cycle.  Thread t owns edges t, t+T, ... and cells t, t+T, ... (T =
// threads in the grid); its own ubar, zeta, G and this sub-step's partial
// F^zeta stay in registers, the 2-D state it shares goes through L2.
template <class R, int ORDER, int NE2>
__global__ void __launch_bounds__(BTR_THREADS) k_btr(DMesh m, BtrArgs<R> a, Barrier bar) {
    const Coef<R> &c = coef<R>(m);
    const unsigned int nb = gridDim.x + a.stall;   // arrivals a barrier waits for
    const int T = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int nit = ((m.E > m.C ? m.E : m.C) + T - 1) / T;  // <= BTR_NIT (host checks)
    // count and gen are zeroed on the stream right before the launch, so every
    // block starts from generation 0
    unsigned int gen = 0;
    const R tau = (R)a.tau, g = (R)a.g;
    const int M = a.M;
    R *u0 = a.u0, *ua = a.ua, *uh = a.uh, *z0 = a.z0, *za = a.za, *zh = a.zh;
    R u0r[BTR_NIT], z0r[BTR_NIT], Gr[BTR_NIT], Fs[BTR_NIT];
    double Fz[BTR_NIT];
#pragma unroll
    for (int s = 0; s < BTR_NIT; s++) {
        const int x = t0 + s * T;
        u0r[s] = R(0); z0r[s] = R(0); Gr[s] = R(0); Fz[s] = 0.0; Fs[s] = R(0);
        if (s < nit && x < m.E) {
            const int xa = a.einv ? a.einv[x] : x;   // the caller's numbering
            u0r[s] = a.ub_start[xa];
            Gr[s] = a.G[xa];
            u0[x] = u0r[s];
        }
        if (s < nit && x < m.C) {
            z0r[s] = (R)a.z_start[a.cinv ? a.cinv[x] : x];
            z0[x] = z0r[s];
        }
    }
    if (!grid_barrier(bar, gen, nb)) return;

    const R wAB = (ORDER == 2) ? R(0.5) : R(1.0 / 6.0);
    const R wC = R(2.0 / 3.0);
    const double invM = 1.0 / M;
    for (int j = 0; j < M; j++) {
        // stage a: (ua, za) = FE(u0, z0)
#pragma unroll
        for (int s = 0; s < BTR_NIT; s++) {
            const int x = t0 + s * T;
            if (s < nit) {
                if (x < m.E) {
                    R f;
                    ua[x] = fe_edge<R, NE2>(m, c, x, u0, z0, Gr[s], tau, g, f);
                    Fs[s] = wAB * f;
                }
                if (x < m.C) za[x] = fe_cell<R>(m, c, x, u0, z0, tau);
            }
        }
        if (!grid_barrier(bar, gen, nb)) return;
        // stage b: FE(ua, za), then the first convex combination
#pragma unroll
        for (int s = 0; s < BTR_NIT; s++) {
            const int x = t0 + s * T;
            if (s < nit) {
                if (x < m.E) {
                    R f;
                    const R ub = fe_edge<R, NE2>(m, c, x, ua, za, Gr[s], tau, g, f);
                    Fs[s] += wAB * f;
                    if (ORDER == 2) {
                        u0r[s] = R(0.5) * (u0r[s] + ub);
                        u0[x] = u0r[s];
                        Fz[s] += invM * (double)Fs[s];
                    } else {
                        uh[x] = R(0.75) * u0r[s] + R(0.25) * ub;
                    }
                }
                if (x < m.C) {
                    const R zb = fe_cell<R>(m, c, x, ua, za, tau);
                    if (ORDER == 2) {
                        z0r[s] = R(0.5) * (z0r[s] + zb);
                        z0[x] = z0r[s];
                    } else {
                        zh[x] = R(0.75) * z0r[s] + R(0.25) * zb;
                    }
                }
            }
        }
        if (!grid_barrier(bar, gen, nb)) return;
        if (ORDER == 3) {
            // stage c: FE(uh, zh), then the second convex combination
#pragma unroll
            for (int s = 0; s < BTR_NIT; s++) {
                const int x = t0 + s * T;
                if (s < nit) {
                    if (x < m.E) {
                        R f;
                        const R uc = fe_edge<R, NE2>(m, c, x, uh, zh, Gr[s], tau, g, f);
                        Fs[s] += wC * f;
                        u0r[s] = R(1.0 / 3.0) * u0r[s] + R(2.0 / 3.0) * uc;
                        u0[x] = u0r[s];
                        Fz[s] += invM * (double)Fs[s];
                    }
                    if (x < m.C) {
                        const R zc = fe_cell<R>(m, c, x, uh, zh, tau);
                        z0r[s] = R(1.0 / 3.0) * z0r[s] + R(2.0 / 3.0) * zc;
                        z0[x] = z0r[s];
                    }
                }
            }
            if (!grid_barrier(bar, gen, nb)) return;
        }
    }
#pragma unroll
    for (int s = 0; s < BTR_NIT; s++) {
        const int x = t0 + s * T;
        if (s < nit && x < m.E) {
            const int xa = a.einv ? a.einv[x] : x;
            a.Fz[xa] = Fz[s];
            a.ub_out[xa] = a.X ? (R)(a.alpha * (double)a.X[xa] + a.beta * (double)u0r[s]) : u0r[s];
        }
        if (s < nit && x < m.C && a.z_out) a.z_out[a.cinv ? a.cinv[x] : x] = (double)z0r[s];
    }
}

// ---------------------------------------------------------------------------
// Tiled, communication-avoiding sub-cycle.  One block per patch.  The patch's
// 2-D state (ubar, zeta and the sub-stage copies), forcing, depths and local
// connectivity live in shared memory; each edge's TRiSK Coriolis coefficients
// and edgesOnEdge offsets sit in tensor memory (FP32, 1024-thread patches) or
// stream from global memory and shared memory.  All forward-Euler sub-stages of one sub-step run on
// the patch with block-level barriers only (the halo of K >= 3 rings keeps
// the owned values exact); after each sub-step the owned ubar and zeta go
// through a double-buffered exchange array and one grid barrier refreshes the
// halo.  M grid barriers per call instead of 2M or 3M.
// ---------------------------------------------------------------------------
// threads per patch: one 1024-thread block per SM, or two 512-thread blocks
// (two patches) per SM whose block barriers overlap each other's work
constexpr int TILE_NE2 = 10;  // edgesOnEdge terms evaluated per edge (padding -> dummy, 0)

// The patch carries the sub-cycle as increments from its starting state:
// u* = ubar - ubar_start and z* = zeta - zeta_start.  The starting state's
// forcing F0 = C_f(ubar_start) - g grad zeta_start + G is formed once per
// launch from the FP64 starting SSH, and the starting column depth d0 =
// zeta_start + H is kept per cell, so that the sub-steps round only the
// (small) increments: in FP32 the full ubar and zeta would lose the 1e-3 to
// 1e-2 of themselves that their gradients and changes over a sub-cycle are.
// Every SSPRK combination has weights summing to one, so it applies to the
// increments unchanged.  (1/dc is stored with the Coriolis coefficients, as
// their last row, which keeps the patch's shared memory at its plain size.)
template <class R> struct TileSmem {
    R *u0, *ua, *uh, *fl, *z0, *za, *zh, *F0, *ub0, *d0;
    unsigned int *c12;                // packed byte offsets of (c1, c2) into the cell arrays
    unsigned short *eoe;              // [ne+1][TILE_NE2P] byte offsets into the edge arrays
                                      // (null when they live in tensor memory)
    unsigned short *ce;               // [nc+1][TILE_NCEP] byte offsets into fl
};

__device__ __forceinline__ char *align16(char *p) {
    return (char *)(((uintptr_t)p + 15) & ~(uintptr_t)15);
}

template <class R>
__device__ __forceinline__ TileSmem<R> carve(char *base, int ne, int nc, bool eoe_smem) {
    TileSmem<R> s;
    char *c = align16(base);
    const int ne1 = ne + 1, nc1 = nc + 1;
    R *r = (R *)c;
    s.u0 = r; r += ne1; s.ua = r; r += ne1; s.uh = r; r += ne1; s.fl = r; r += ne1;
    s.z0 = r; r += nc1; s.za = r; r += nc1; s.zh = r; r += nc1;
    s.F0 = r; r += ne1; s.ub0 = r; r += ne1; s.d0 = r; r += nc1;
    c = align16((char *)r);
    s.c12 = (unsigned int *)c; c = align16(c + 4 * ne1);
    s.eoe = nullptr;
    if (eoe_smem) { s.eoe = (unsigned short *)c; c = align16(c + 2 * TILE_NE2P * (size_t)ne1); }
    s.ce = (unsigned short *)c;
    return s;
}

template <class R> __device__ __forceinline__ R at(const R *base, unsigned int off) {
    return *(const R *)((const char *)base + off);
}

// ---- tensor memory as per-thread storage (FP32 form, 1024-thread patches).
// A thread's edges (l = tid + k * 1024, k < TM_SLOTS) never change during
// the sub-cycle, and neither do their Coriolis coefficients, 1/d_e and
// edgesOnEdge offsets: 16 words per edge, read every sub-stage.  Streamed
// from L2 they cost about a fifth of the sub-cycle (the patch's shared memory
// leaves L1 no room to keep them); held in tensor memory they are one
// 32x32b.x16 load per edge.  In that access shape thread i of warp w reads
// TMEM lane 32 (w % 4) + i, so the eight warps of a lane quadrant take
// disjoint 64-column ranges (w / 4) * 64 + 16 k: 512 columns in all.
constexpr int TM_SLOTS = 4;
constexpr int TM_COLS_SLOT = 16;   // 11 coefficients + 5 words of packed offsets
constexpr int TM_THREADS = 1024;
constexpr unsigned int TM_COLS = (TM_THREADS / 128) * TM_SLOTS * TM_COLS_SLOT;   // 512
static_assert(TILE_CFR + TILE_NE2P / 2 == TM_COLS_SLOT, "one TMEM slot per edge");

// Allocation by one whole warp; the address goes to shared memory.  The
// launch guarantees that no other CTA using tensor memory shares the SM (its
// shared memory exceeds half the SM's), so the allocation never waits.
__device__ __forceinline__ void tmem_alloc(unsigned int *dst, unsigned int ncols) {
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(dst);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(d), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned int taddr, unsigned int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_st16(unsigned int taddr, const unsigned int (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                 "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
                 "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
                 "r"(v[13]), "r"(v[14]), "r"(v[15]) : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// load and wait; the registers pass through the wait so that no use of them
// can be scheduled before it
__device__ __forceinline__ void tmem_ld16(unsigned int taddr, unsigned int (&v)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                   "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                   "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                   "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                   "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
                 :: "memory");
}

// An edge's constant data: TILE_CFR coefficients (the Coriolis terms, then
// 1/d_e) and its TILE_NE2P edgesOnEdge byte offsets.  From tensor memory (a
// warp-collective load: every lane of the warp calls it) or from the patch's
// global coefficient block and shared offsets (only for l < ne).
template <class R, bool TM>
__device__ __forceinline__ void edge_coefs(const TileSmem<R> &S, const R *__restrict__ cfc,
                                           int ne, int l, unsigned int taddr,
                                           R (&cf)[TILE_CFR], unsigned int (&o)[TILE_NE2P]) {
    if constexpr (TM) {
        unsigned int v[16];
        tmem_ld16(taddr, v);
#pragma unroll
        for (int j = 0; j < TILE_CFR; j++) cf[j] = __uint_as_float(v[j]);
#pragma unroll
        for (int i = 0; i < TILE_NE2P / 2; i++) {
            o[2 * i] = v[TILE_CFR + i] & 0xffffu; o[2 * i + 1] = v[TILE_CFR + i] >> 16;
        }
    } else {
#pragma unroll
        for (int j = 0; j < TILE_CFR; j++) cf[j] = __ldg(cfc + (size_t)j * ne + l);
        const unsigned int *eo = (const unsigned int *)(S.eoe + (size_t)l * TILE_NE2P);
#pragma unroll
        for (int i = 0; i < TILE_NE2P / 2; i++) {
            const unsigned int v = eo[i];
            o[2 * i] = v & 0xffffu; o[2 * i + 1] = v >> 16;
        }
    }
}

// The sub-stage arithmetic with every fused multiply-add spelled out: left to
// the compiler, a*x + b*y may fuse either product, and the choice can differ
// between the kernel's instantiations and between the owned and halo copies
// of one expression, which then round differently.  Written out, every code
// path that evaluates an edge or a cell rounds it the same way.
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_r(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_r(double a, double b) { return __dmul_rn(a, b); }
// a x + b y, the second product rounded first
template <class R> __device__ __forceinline__ R comb(R a, R x, R b, R y) {
    return fma_r(a, x, mul_r(b, y));
}

// forward-Euler edge update on the patch, on the increments u, z: returns the
// new ubar increment, sets the flux of the full state
template <class R>
__device__ __forceinline__ R tile_fe_edge(const TileSmem<R> &S, const R (&cf)[TILE_CFR],
                                          const unsigned int (&o)[TILE_NE2P], int l,
                                          const R *u, const R *z, R tau, R g, R &flux) {
    R acc = R(0);
#pragma unroll
    for (int j = 0; j < TILE_NE2; j++) acc = fma_r(cf[j], at(u, o[j]), acc);
    const unsigned int cc = S.c12[l];
    const unsigned int a = cc & 0xffffu, b = cc >> 16;
    const R za = at(z, a), zb = at(z, b);
    const R ue = u[l];
    flux = mul_r(S.ub0[l] + ue, mul_r(R(0.5), (at(S.d0, a) + at(S.d0, b)) + (za + zb)));
    const R rhs = fma_r(-mul_r(g, zb - za), cf[TILE_NE2P], S.F0[l] + acc);
    return fma_r(tau, rhs, ue);
}

// One forward-Euler sub-stage over this thread's edges in [lo, hi);
// fn(k, l, new increment, flux) stores the results, k < OWN for an owned edge
// in slot k (l = tid + k nt < noe), k = OWN for a halo edge.  With TM every
// edge has a slot (l = tid + k nt, k < KS): a warp whose 32 edges of slot k
// all lie outside [lo, hi) skips it, the others load the slot in every lane
// (the tensor-memory load is warp-collective) and compute only the lanes
// inside the range.  Without, the owned slots are unrolled and the halo edges
// (l = noe + tid + i nt) loop.
template <class R, bool TM, int KS, int OWN, class Fn>
__device__ __forceinline__ void edge_pass(const TileSmem<R> &S, const R *__restrict__ cfc,
                                          int ne, int noe, unsigned int tsl, int tid, int nt,
                                          int lo, int hi, const R *u, const R *z, R tau, R g,
                                          Fn &&fn) {
    if constexpr (TM) {
#pragma unroll
        for (int k = 0; k < KS; k++) {
            const int l = tid + k * nt, w0 = (tid & ~31) + k * nt;
            if (w0 >= hi || w0 + 32 <= lo) continue;
            R cf[TILE_CFR];
            unsigned int o[TILE_NE2P];
            __syncwarp();
            edge_coefs<R, true>(S, cfc, ne, l, tsl + (unsigned int)(k * TM_COLS_SLOT), cf, o);
            if (l >= lo && l < hi) {
                R f;
                const R r = tile_fe_edge<R>(S, cf, o, l, u, z, tau, g, f);
                fn(k < OWN && l < noe ? k : OWN, l, r, f);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < OWN; k++) {
            const int l = tid + k * nt;
            if (l >= lo && l < hi && l < noe) {
                R cf[TILE_CFR];
                unsigned int o[TILE_NE2P];
                edge_coefs<R, false>(S, cfc, ne, l, 0u, cf, o);
                R f;
                const R r = tile_fe_edge<R>(S, cf, o, l, u, z, tau, g, f);
                fn(k, l, r, f);
            }
        }
        for (int l = noe + tid; l < hi; l += nt) {
            R cf[TILE_CFR];
            unsigned int o[TILE_NE2P];
            edge_coefs<R, false>(S, cfc, ne, l, 0u, cf, o);
            R f;
            const R r = tile_fe_edge<R>(S, cf, o, l, u, z, tau, g, f);
            fn(OWN, l, r, f);
        }
    }
}

// term j of cell l's divergence coefficients at dvc[j * nc + l]
template <class R>
__device__ __forceinline__ R tile_fe_cell(const TileSmem<R> &S, const R *__restrict__ dvc, int nc,
                                          int l, const R *z, R tau) {
    R dc[TILE_NCEP];
#pragma unroll
    for (int j = 0; j < TILE_NCEP; j++) dc[j] = __ldg(dvc + (size_t)j * nc + l);
    const unsigned int *co = (const unsigned int *)(S.ce + (size_t)l * TILE_NCEP);
    unsigned int o[TILE_NCEP];
#pragma unroll
    for (int i = 0; i < TILE_NCEP / 2; i++) {
        const unsigned int v = co[i];
        o[2 * i] = v & 0xffffu; o[2 * i + 1] = v >> 16;
    }
    R dv = R(0);
#pragma unroll
    for (int j = 0; j < TILE_NCEP; j++) dv = fma_r(dc[j], at(S.fl, o[j]), dv);
    return fma_r(-tau, dv, z[l]);
}

// Accumulator of F^zeta = (1/M) sum_j (sub-step flux sum) for one owned
// edge.  FP64 form: a double.  Mixed form: the sub-step sums are FP32 and are
// added into an unevaluated pair of floats (hi, lo) with Knuth's TwoSum, which
// yields the exact rounding error of each addition; the pair carries about
// 48 significant bits, and FP64 is needed only once, at the end.  (FP64 adds
// run at a small fraction of the FP32 rate on this GPU; one per owned edge
// and sub-step costs more than a sub-stage's cell update.)
template <class R> struct FzAcc;
template <> struct FzAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x, double) {
        const float s = hi + x, bp = s - hi;
        lo += (hi - (s - bp)) + (x - bp);
        hi = s;
    }
    __device__ __forceinline__ double value(double invM) const {
        return invM * ((double)hi + (double)lo);
    }
};
template <> struct FzAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x, double invM) { s += invM * x; }
    __device__ __forceinline__ double value(double) const { return s; }
};

// The Coriolis term of the starting ubar, sum_j cf_j ub0_j, as the FP64 value
// the starting forcing adds.  FP64 form: FP64 products and sums.  Mixed form:
// the compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005, Algorithm Dot2): each product's
// rounding error from an FMA, each sum's from Knuth's TwoSum, the errors
// summed apart, so that the result is as accurate as if computed in twice
// FP32's precision -- without FP64 arithmetic, ten of whose operations per
// edge cost more than the whole FP32 evaluation.
template <class R>
__device__ __forceinline__ double coriolis_start(const R (&cf)[TILE_CFR],
                                                 const unsigned int (&o)[TILE_NE2P], const R *ub0) {
    if constexpr (sizeof(R) == 4) {
        float s = 0.f, c = 0.f;
#pragma unroll
        for (int j = 0; j < TILE_NE2; j++) {
            const float x = cf[j], y = at(ub0, o[j]);
            // __fmul_rn / __fadd_rn: never contracted into an FMA, which
            // would break the error-free transformations
            const float p = __fmul_rn(x, y), pe = fmaf(x, y, -p);
            const float t = __fadd_rn(s, p), z = __fsub_rn(t, s);
            const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
            s = t;
            c += pe + se;
        }
        return (double)s + (double)c;
    } else {
        double cb = 0.0;
#pragma unroll
        for (int j = 0; j < TILE_NE2; j++) cb += (double)cf[j] * (double)at(ub0, o[j]);
        return cb;
    }
}

// Each thread owns at most OWN owned edges, halo edges, owned cells and halo
// cells of its patch (the plan checks this); their global indices, the
// sub-step's partial F^zeta and the FP64 accumulators stay in registers.  The
// forward-Euler sub-stages take edge l = tid + k nt in slot k, owned edges
// (l < n_own_e) in the first OWN slots; with TM the slots' constant edge data
// live in tensor memory (FP32, 1024 threads, at most TM_SLOTS slots).
template <class R, int ORDER, int OWN, int NT, bool TM>
__global__ void __launch_bounds__(NT, 1024 / NT) k_btr_tiled(DTiles<R> t, BtrArgs<R> a,
                                                             Barrier bar) {
    static_assert(!TM || (sizeof(R) == 4 && NT == TM_THREADS), "tensor memory: FP32, 1024 threads");
    constexpr int KS = TM ? TM_SLOTS : 2 * OWN;   // edge slots per thread
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ unsigned int s_tmem;
    const int p = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    // tensor memory first, before any exit: warp 0 allocates, every thread
    // learns the base address, and every path out of the kernel frees it
    unsigned int tsl = 0;   // this thread's lane and first column
    if constexpr (TM) {
        if (tid < 32) tmem_alloc(&s_tmem, TM_COLS);
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        tsl = s_tmem + ((unsigned int)(32 * ((tid >> 5) & 3)) << 16) +
              (unsigned int)((tid >> 7) * (TM_SLOTS * TM_COLS_SLOT));
    }
    const int coff = t.cell_off[p], eoff = t.edge_off[p];
    const int nc = t.cell_off[p + 1] - coff, ne = t.edge_off[p + 1] - eoff;
    const int noc = t.n_own_c[p], noe = t.n_own_e[p], nint = t.n_int_e[p];
    const bool arriver = (tid >> 5) == ((nt - 1) >> 5);   // the warp of grid_arrive / grid_wait
    // sub-stage s only needs the edges and cells still exact after it (the
    // outer rings of the halo drop out one per sub-stage)
    const int neA = t.ne_lim[3 * p], neB = t.ne_lim[3 * p + 1], neC = t.ne_lim[3 * p + 2];
    const int ncA = t.nc_lim[3 * p], ncB = t.nc_lim[3 * p + 1], ncC = t.nc_lim[3 * p + 2];
    const TileSmem<R> S = carve<R>(smem_raw, ne, nc, !TM);
    const R *cfc = t.cfc + (size_t)eoff * TILE_CFR;
    const R *dvc = t.divc + (size_t)coff * TILE_NCEP;
    const unsigned short *eoe_g = t.eoe + (size_t)eoff * TILE_NE2P;
    const R tau = (R)a.tau, g = (R)a.g;
    const R third = R(1.0 / 3.0), two_thirds = R(2.0 / 3.0);
    // global indices of this thread's owned and halo entries
    int oe[OWN], he[OWN], oc[OWN], hc[OWN];
#pragma unroll
    for (int k = 0; k < OWN; k++) {
        const int lo = tid + k * nt, lh = noe + tid + k * nt;
        const int co = tid + k * nt, ch = noc + tid + k * nt;
        oe[k] = lo < noe ? t.edge_gid[eoff + lo] : -1;
        he[k] = lh < ne ? t.edge_gid[eoff + lh] : -1;
        oc[k] = co < noc ? t.cell_gid[coff + co] : -1;
        hc[k] = ch < nc ? t.cell_gid[coff + ch] : -1;
    }

    // ---- load the patch (the extra slot ne / nc is the zero-valued dummy);
    // the increments start at zero
    for (int l = tid; l <= ne; l += nt) {
        R u = R(0), d = R(0);
        double G = 0.0;
        unsigned int cc = (unsigned int)(nc * sizeof(R)) | ((unsigned int)(nc * sizeof(R)) << 16);
        if (l < ne) {
            const int gid = t.edge_gid[eoff + l];
            u = a.ub_start[gid];
            G = (double)a.G[gid];
            d = cfc[(size_t)TILE_NE2P * ne + l];
            cc = (unsigned int)t.c12[eoff + l];
        }
        // the SSH-gradient part of the starting forcing, from the FP64
        // starting SSH (the dummy cell: zeta = 0)
        const int ia = (int)((cc & 0xffffu) / sizeof(R)), ib = (int)((cc >> 16) / sizeof(R));
        const double za = ia < nc ? a.z_start[t.cell_gid[coff + ia]] : 0.0;
        const double zb = ib < nc ? a.z_start[t.cell_gid[coff + ib]] : 0.0;
        S.F0[l] = (R)(G - a.g * (zb - za) * (double)d);
        S.ub0[l] = u; S.c12[l] = cc;
        S.u0[l] = R(0); S.ua[l] = R(0); S.uh[l] = R(0); S.fl[l] = R(0);
    }
    if constexpr (!TM) {
        // rows are TILE_NE2P * 2 = 20 bytes: copy in 4-byte words (every row and the
        // patch base edge_off * 20 bytes are 4-byte aligned)
        const unsigned int *src = (const unsigned int *)eoe_g;
        unsigned int *dst = (unsigned int *)S.eoe;
        const int n4 = ne * (TILE_NE2P / 2);
        for (int x = tid; x < n4; x += nt) dst[x] = src[x];
        if (tid < TILE_NE2P) S.eoe[(size_t)ne * TILE_NE2P + tid] = (unsigned short)(ne * sizeof(R));
    }
    for (int l = tid; l <= nc; l += nt) {
        const double z = (l < nc) ? a.z_start[t.cell_gid[coff + l]] : 0.0;
        S.d0[l] = (R)(z + (double)t.H[coff + p + l]);
        S.z0[l] = R(0); S.za[l] = R(0); S.zh[l] = R(0);
    }
    {
        // rows of TILE_NCEP * 2 = 12 bytes, copied in 4-byte words
        const unsigned int *src = (const unsigned int *)(t.ce + (size_t)coff * TILE_NCEP);
        unsigned int *dst = (unsigned int *)S.ce;
        const int n4 = nc * (TILE_NCEP / 2);
        for (int x = tid; x < n4; x += nt) dst[x] = src[x];
    }
    R Fs[OWN];
    FzAcc<R> Fz[OWN];
#pragma unroll
    for (int k = 0; k < OWN; k++) Fs[k] = R(0);
    __syncthreads();
    // the Coriolis term of the starting ubar completes the starting forcing;
    // with TM the same pass moves each slot's constant edge data into tensor
    // memory (every lane stores every slot: the store is warp-collective)
#pragma unroll 1
    for (int k = 0; k < KS; k++) {
        const int l = tid + k * nt;
        if (!TM && l >= ne) break;
        R cf[TILE_CFR];
        unsigned int o[TILE_NE2P];
        unsigned int v[16];
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = 0u;
        if (l < ne) {
#pragma unroll
            for (int j = 0; j < TILE_CFR; j++) cf[j] = __ldg(cfc + (size_t)j * ne + l);
            const unsigned int *eo = (const unsigned int *)(eoe_g + (size_t)l * TILE_NE2P);
#pragma unroll
            for (int i = 0; i < TILE_NE2P / 2; i++) {
                const unsigned int w = __ldg(eo + i);
                o[2 * i] = w & 0xffffu; o[2 * i + 1] = w >> 16;
                v[TILE_CFR + i] = w;
            }
            S.F0[l] = (R)((double)S.F0[l] + coriolis_start<R>(cf, o, S.ub0));
            if constexpr (TM) {
#pragma unroll
                for (int j = 0; j < TILE_CFR; j++) v[j] = __float_as_uint(cf[j]);
            }
        }
        if constexpr (TM) {
            __syncwarp();
            tmem_st16(tsl + (unsigned int)(k * TM_COLS_SLOT), v);
        }
    }
    if constexpr (TM) tmem_st_wait();
    __syncthreads();

    const R wAB = (ORDER == 2) ? R(0.5) : R(1.0 / 6.0);
    const R wC = R(2.0 / 3.0);
    const double invM = 1.0 / a.M;
    int buf = 0;
    bool ok = true;
    for (int j = 0; j < a.M; j++) {
        // ---- stage a: (ua, za) = FE(u0, z0); after the first sub-step the owned
        // edges below nint were already done while the halo exchange was in
        // flight, except by the arriving warp
        const int lo = (j == 0 || arriver) ? 0 : nint;
        edge_pass<R, TM, KS, OWN>(S, cfc, ne, noe, tsl, tid, nt, lo, neA, S.u0, S.z0, tau, g,
                             [&](int k, int l, R r, R f) {
                                 S.ua[l] = r;
                                 S.fl[l] = f;
                                 if (k < OWN) Fs[k] = mul_r(wAB, f);
                             });
        __syncthreads();
        for (int l = tid; l < ncA; l += nt) S.za[l] = tile_fe_cell<R>(S, dvc, nc, l, S.z0, tau);
        __syncthreads();
        // ---- stage b: FE(ua, za), first convex combination
        edge_pass<R, TM, KS, OWN>(S, cfc, ne, noe, tsl, tid, nt, 0, neB, S.ua, S.za, tau, g,
                             [&](int k, int l, R ub, R f) {
                                 S.fl[l] = f;
                                 if (k < OWN) Fs[k] = fma_r(wAB, f, Fs[k]);
                                 if (ORDER == 2) S.u0[l] = mul_r(R(0.5), S.u0[l] + ub);
                                 else S.uh[l] = comb(R(0.75), S.u0[l], R(0.25), ub);
                             });
        __syncthreads();
        for (int l = tid; l < ncB; l += nt) {
            const R zb = tile_fe_cell<R>(S, dvc, nc, l, S.za, tau);
            if (ORDER == 2) S.z0[l] = mul_r(R(0.5), S.z0[l] + zb);
            else S.zh[l] = comb(R(0.75), S.z0[l], R(0.25), zb);
        }
        __syncthreads();
        if (ORDER == 3) {
            // ---- stage c: FE(uh, zh), second convex combination
            edge_pass<R, TM, KS, OWN>(S, cfc, ne, noe, tsl, tid, nt, 0, neC, S.uh, S.zh, tau, g,
                                 [&](int k, int l, R uc, R f) {
                                     S.fl[l] = f;
                                     if (k < OWN) Fs[k] = fma_r(wC, f, Fs[k]);
                                     S.u0[l] = comb(third, S.u0[l], two_thirds, uc);
                                 });
            __syncthreads();
            for (int l = tid; l < ncC; l += nt) {
                const R zc = tile_fe_cell<R>(S, dvc, nc, l, S.zh, tau);
                S.z0[l] = comb(third, S.z0[l], two_thirds, zc);
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < OWN; k++) Fz[k].add(Fs[k], invM);
        if (j + 1 == a.M) break;
        // ---- exchange the owned values, refresh the halo
        R *xu = t.xu[buf], *xz = t.xz[buf];
#pragma unroll
        for (int k = 0; k < OWN; k++) {
            if (oe[k] >= 0) xu[oe[k]] = S.u0[tid + k * nt];
            if (oc[k] >= 0) xz[oc[k]] = S.z0[tid + k * nt];
        }
        grid_arrive(bar);
        // Stage a of the next sub-step on the owned edges with both cells owned
        // (l < nint): it reads zeta at owned cells and ubar at edges of owned
        // cells (ring <= 1), all exact after this sub-step's last stage, and
        // writes only ua and the flux, which the refresh does not touch.  The
        // arriving warp, which waits for its release first, leaves its share
        // to the main stage a.
        if (!arriver)
            edge_pass<R, TM, KS, OWN>(S, cfc, ne, noe, tsl, tid, nt, 0, nint, S.u0, S.z0, tau, g,
                                 [&](int k, int l, R r, R f) {
                                     S.ua[l] = r;
                                     S.fl[l] = f;
                                     if (k < OWN) Fs[k] = mul_r(wAB, f);
                                 });
        if (!grid_wait(bar, (unsigned int)(j + 1) * gridDim.x + a.stall)) {
            ok = false;   // every thread: grid_wait's verdict is the block's
            break;
        }
#pragma unroll
        for (int k = 0; k < OWN; k++) {
            if (he[k] >= 0) S.u0[noe + tid + k * nt] = __ldcg(xu + he[k]);
            if (hc[k] >= 0) S.z0[noc + tid + k * nt] = __ldcg(xz + hc[k]);
        }
        buf ^= 1;
        __syncthreads();
    }
    if constexpr (TM) {
        // every warp's tensor-memory loads completed (each waited for its own)
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        if (tid < 32) tmem_dealloc(s_tmem, TM_COLS);
    }
    if (!ok) return;
    // ---- outputs for the owned edges and cells: starting state plus increment
#pragma unroll
    for (int k = 0; k < OWN; k++) {
        if (oe[k] >= 0) {
            const double u0 = (double)S.ub0[tid + k * nt] + (double)S.u0[tid + k * nt];
            a.Fz[oe[k]] = Fz[k].value(invM);
            a.ub_out[oe[k]] = a.X ? (R)(a.alpha * (double)a.X[oe[k]] + a.beta * u0) : (R)u0;
        }
        if (a.z_out && oc[k] >= 0)
            a.z_out[oc[k]] = a.z_start[oc[k]] + (double)S.z0[tid + k * nt];
    }
}

template <class R, int NT, bool TM> const void *btr_tiled_kernel_ptr_nt(int order, int own) {
    if (own == 2)
        return order == 2 ? (const void *)k_btr_tiled<R, 2, 2, NT, TM>
                          : (const void *)k_btr_tiled<R, 3, 2, NT, TM>;
    return order == 2 ? (const void *)k_btr_tiled<R, 2, 3, NT, TM>
                      : (const void *)k_btr_tiled<R, 3, 3, NT, TM>;
}
template <class R> const void *btr_tiled_kernel_ptr(int order, int own, int nthreads, bool tm) {
    if (tm) {
        if constexpr (sizeof(R) == 4) {
            if (nthreads == TM_THREADS) return btr_tiled_kernel_ptr_nt<R, TM_THREADS, true>(order, own);
        }
        return nullptr;
    }
    if (nthreads == 512) return btr_tiled_kernel_ptr_nt<R, 512, false>(order, own);
    if (nthreads == 1024) return btr_tiled_kernel_ptr_nt<R, 1024, false>(order, own);
    return nullptr;
}
int btr_tiled_tmem_slots() { return TM_SLOTS; }

template <class R>
cudaError_t launch_btr_tiled(const DTiles<R> &t, const BtrArgs<R> &a, const Barrier &bar,
                             cudaStream_t s) {
    DTiles<R> tt = t;
    BtrArgs<R> aa = a;
    Barrier bb = bar;
    void *args[] = {&tt, &aa, &bb};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(t.P);
    cfg.blockDim = dim3(t.nthreads);
    cfg.dynamicSmemBytes = t.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const void *fn = btr_tiled_kernel_ptr<R>(a.order, t.own, t.nthreads, t.tm != 0);
    if (!fn) return cudaErrorInvalidConfiguration;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

template const void *btr_tiled_kernel_ptr<double>(int, int, int, bool);
template const void *btr_tiled_kernel_ptr<float>(int, int, int, bool);
template cudaError_t launch_btr_tiled<double>(const DTiles<double> &, const BtrArgs<double> &,
                                              const Barrier &, cudaStream_t);
template cudaError_t launch_btr_tiled<float>(const DTiles<float> &, const BtrArgs<float> &,
                                             const Barrier &, cudaStream_t);

template <class R> int btr_block_size() { return BTR_THREADS; }
template <class R> const void *btr_kernel_ptr(int order, int maxE2) {
    if (maxE2 <= BTR_NE2)
        return order == 2 ? (const void *)k_btr<R, 2, BTR_NE2> : (const void *)k_btr<R, 3, BTR_NE2>;
    return order == 2 ? (const void *)k_btr<R, 2, MAXE2> : (const void *)k_btr<R, 3, MAXE2>;
}
int btr_max_items_per_thread() { return BTR_NIT; }

template <class R>
cudaError_t launch_btr(const DMesh &m, const BtrArgs<R> &a, const Barrier &bar, int nblocks,
                       int nthreads, cudaStream_t s) {
    DMesh mm = m;
    BtrArgs<R> aa = a;
    Barrier bb = bar;
    // the caller zeroes bar.count and bar.gen (adjacent words) on stream s
    // before every launch
    void *args[] = {&mm, &aa, &bb};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(nthreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, btr_kernel_ptr<R>(a.order, m.maxE2), args);
}

template int btr_block_size<double>();
template int btr_block_size<float>();
template const void *btr_kernel_ptr<double>(int, int);
template const void *btr_kernel_ptr<float>(int, int);
template cudaError_t launch_btr<double>(const DMesh &, const BtrArgs<double> &, const Barrier &,
                                        int, int, cudaStream_t);
template cudaError_t launch_btr<float>(const DMesh &, const BtrArgs<float> &, const Barrier &, int,
                                       int, cudaStream_t);

}  // namespace sse

// ===========================================================================
// Allocation-free sub-cycle: sse_barotropic_substep_noalloc
//
// For callers that must not allocate device memory at the point where they
// run the sub-cycle: code running inside a device-memory allocator or pool
// callback, a runtime that reserves all of its device memory up front and
// forbids later cudaMalloc calls, or a latency-critical loop in which the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// The work buffers live in one file-scope device array that every GPU
// loading this library holds until the process exits.  The first 256 bytes
// hold the grid-barrier words and the error word.
// ===========================================================================
namespace sse {

constexpr int NOALLOC_MAX_EDGES = 393216;
constexpr int NOALLOC_MAX_CELLS = 131072;
constexpr int NOALLOC_HEADER = 32;  // doubles (256 bytes) of barrier words
static __device__ __align__(256) double
    g_noalloc_scratch[NOALLOC_HEADER + 3 * NOALLOC_MAX_EDGES + 3 * NOALLOC_MAX_CELLS];

namespace {
constexpr int kMaxDevices = 64;
struct NoallocDevice {
    double *scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int sms = 0;
    // co-resident blocks per SM of each kernel variant the entry point may
    // launch, [order - 2][maxE2 <= BTR_NE2 ? 0 : 1] (0: not yet queried)
    int blocks_per_sm[2][2] = {{0, 0}, {0, 0}};
};
NoallocDevice g_noalloc_dev[kMaxDevices];
std::mutex g_noalloc_mutex;
}  // namespace

}  // namespace sse

const sse::DMesh *sse_internal_dmesh(const sse_mesh *m);
int sse_internal_device(const sse_mesh *m);

extern "C" int sse_barotropic_substep_noalloc(const sse_mesh *mesh, int order, double dt,
                                              int n_substeps, double g, const double *ubar_in,
                                              const double *zeta_in, const double *G,
                                              double *ubar_out, double *Fzeta_out,
                                              double *zeta_out, void *cuda_stream) {
    using namespace sse;
    if (!mesh || (order != 2 && order != 3) || !(dt > 0) || !isfinite(dt) || n_substeps < 1 ||
        !(g > 0) || !ubar_in || !zeta_in || !G || !ubar_out || !Fzeta_out)
        return SSE_ERR_INVALID_ARG;
    const DMesh &m = *sse_internal_dmesh(mesh);
    if (m.E > NOALLOC_MAX_EDGES || m.C > NOALLOC_MAX_CELLS) return SSE_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SSE_ERR_CUDA;
    // the mesh's arrays live on the device that was current at sse_mesh_create
    if (dev != sse_internal_device(mesh)) return SSE_ERR_INVALID_ARG;
    // the variant launch_btr picks for this mesh
    const int vi = m.maxE2 <= BTR_NE2 ? 0 : 1;
    NoallocDevice nd;
    int blocks_per_sm = 0;
    {
        // once per device, with that device current: the device address of the
        // array (the host-side symbol is only a stand-in for it); once per
        // kernel variant: its occupancy
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        NoallocDevice &d = g_noalloc_dev[dev];
        if (!d.scratch) {
            void *p = nullptr;
            int nsm = 0;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess ||
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return SSE_ERR_CUDA;
            d.sms = nsm;
            d.scratch = (double *)p;
        }
        int &occ = d.blocks_per_sm[order - 2][vi];
        if (occ == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &occ, btr_kernel_ptr<double>(order, m.maxE2), BTR_THREADS, 0) !=
                            cudaSuccess) {
            occ = 0;
            return SSE_ERR_CUDA;
        }
        blocks_per_sm = occ;
        nd = d;
    }
    if (blocks_per_sm < 1) return SSE_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *base = nd.scratch;
    unsigned int *words = (unsigned int *)base;
    double *work = base + NOALLOC_HEADER;
    BtrArgs<double> a{};
    a.ub_start = ubar_in; a.z_start = zeta_in; a.G = G; a.X = nullptr; a.alpha = 0.0;
    a.beta = 1.0; a.ub_out = ubar_out; a.Fz = Fzeta_out; a.z_out = zeta_out;
    // the caller's arrays are in the caller's numbering
    a.einv = m.einv; a.cinv = m.cinv;
    a.u0 = work; a.ua = work + NOALLOC_MAX_EDGES; a.uh = work + 2 * NOALLOC_MAX_EDGES;
    a.z0 = work + 3 * NOALLOC_MAX_EDGES; a.za = a.z0 + NOALLOC_MAX_CELLS;
    a.zh = a.z0 + 2 * NOALLOC_MAX_CELLS;
    a.tau = dt / n_substeps; a.g = g; a.M = n_substeps; a.order = order;
    Barrier bar{words, words + 1, (int *)(words + 2)};
    // the array keeps the previous call's contents: zero the barrier and error words
    if (cudaMemsetAsync(base, 0, NOALLOC_HEADER * sizeof(double), s) != cudaSuccess)
        return SSE_ERR_CUDA;
    const int need = ((m.E > m.C ? m.E : m.C) + BTR_THREADS - 1) / BTR_THREADS;
    int blocks = blocks_per_sm * nd.sms;
    if (need < blocks) blocks = need;
    if (blocks < 1) blocks = 1;
    if ((long long)blocks * BTR_THREADS * BTR_NIT < (m.E > m.C ? m.E : m.C))
        return SSE_ERR_UNSUPPORTED;
    if (launch_btr<double>(m, a, bar, blocks, BTR_THREADS, s) != cudaSuccess) return SSE_ERR_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, words + 2, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SSE_ERR_CUDA;
    return err ? SSE_ERR_SYNC_TIMEOUT : SSE_OK;
}
