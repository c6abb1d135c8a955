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

namespace sse {

constexpr int BTR_THREADS = 512;
constexpr long long BARRIER_SPIN_NS = 2000000000LL;  // 2 s

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// returns false (and sets *err) when the wait exceeded its budget
__device__ __forceinline__ bool grid_barrier(const Barrier &bar, unsigned int &gen_local,
                                             unsigned int nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int g0 = gen_local;
        __threadfence();
        const unsigned int arrived = atomicAdd(bar.count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar.count, 0u);
            __threadfence();
            atomicAdd(bar.gen, 1u);
        } else {
            const unsigned long long t0 = gtimer();
            unsigned int ns = 32;
            while (atomicAdd(bar.gen, 0u) == g0) {
                if (*((volatile int *)bar.err)) { ok = 0; break; }
                if (gtimer() - t0 > (unsigned long long)BARRIER_SPIN_NS) {
                    atomicExch(bar.err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 256) ns *= 2;
            }
        }
        __threadfence();
        gen_local = g0 + 1;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class R>
__device__ __forceinline__ R zh_edge(const DMesh &m, const R *z, int c1, int c2) {
    // barotropic column depth at the edge, (zeta + H)_e centred
    return R(0.5) * ((__ldcg(z + c1) + (R)m.H[c1]) + (__ldcg(z + c2) + (R)m.H[c2]));
}

// one forward-Euler sub-stage of the edge equation; returns the new ubar and
// the flux ubar (zeta + H)_e of the input state
template <class R>
__device__ __forceinline__ R fe_edge(const DMesh &m, const Coef<R> &c, int e, const R *u,
                                     const R *z, const R *G, R tau, R g, R &flux) {
    const int2 cc = m.coe[e];
    const int n2 = m.neoe[e];
    const int Ep = m.Ep;
    R cf = R(0);
    for (int j = 0; j < n2; j++) cf += c.cfc[j * Ep + e] * __ldcg(u + m.eoe[j * Ep + e]);
    const R ue = __ldcg(u + e);
    const R z1 = __ldcg(z + cc.x), z2 = __ldcg(z + cc.y);
    flux = ue * zh_edge<R>(m, z, cc.x, cc.y);
    return ue + tau * (cf - g * (z2 - z1) * c.invdc[e] + G[e]);
}

template <class R>
__device__ __forceinline__ R fe_cell(const DMesh &m, const Coef<R> &c, int i, const R *u,
                                     const R *z, R tau) {
    const int ne = m.neoc[i];
    const int Cp = m.Cp;
    R dv = R(0);
    for (int j = 0; j < ne; j++) {
        const int e = m.eoc[j * Cp + i];
        const int2 cc = m.coe[e];
        dv += c.divc[j * Cp + i] * (__ldcg(u + e) * zh_edge<R>(m, z, cc.x, cc.y));
    }
    return __ldcg(z + i) - tau * dv;
}

template <class R, int ORDER>
__global__ void __launch_bounds__(BTR_THREADS) k_btr(DMesh m, BtrArgs<R> a, Barrier bar) {
    const Coef<R> &c = coef<R>(m);
    const unsigned int nb = gridDim.x;
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    // count and gen are zeroed on the stream right before the launch, so every
    // block starts from generation 0
    unsigned int gen = 0;
    const R tau = (R)a.tau, g = (R)a.g;
    const int M = a.M;
    R *u0 = a.u0, *ua = a.ua, *uh = a.uh, *z0 = a.z0, *za = a.za, *zh = a.zh;

    for (int e = t0; e < m.E; e += stride) {
        u0[e] = a.ub_start[e];
        a.Fz[e] = 0.0;
    }
    for (int i = t0; i < m.C; i += stride) z0[i] = (R)a.z_start[i];
    if (!grid_barrier(bar, gen, nb)) return;

    const double wAB = (ORDER == 2) ? 1.0 / (2.0 * M) : 1.0 / (6.0 * M);
    const double wC = 2.0 / (3.0 * M);
    for (int j = 0; j < M; j++) {
        // stage a: (ua, za) = FE(u0, z0)
        for (int e = t0; e < m.E; e += stride) {
            R f;
            ua[e] = fe_edge<R>(m, c, e, u0, z0, a.G, tau, g, f);
            a.Fz[e] += wAB * (double)f;
        }
        for (int i = t0; i < m.C; i += stride) za[i] = fe_cell<R>(m, c, i, u0, z0, tau);
        if (!grid_barrier(bar, gen, nb)) return;
        // stage b: FE(ua, za), then the first convex combination
        for (int e = t0; e < m.E; e += stride) {
            R f;
            const R ub = fe_edge<R>(m, c, e, ua, za, a.G, tau, g, f);
            a.Fz[e] += wAB * (double)f;
            if (ORDER == 2)
                u0[e] = R(0.5) * (u0[e] + ub);
            else
                uh[e] = R(0.75) * u0[e] + R(0.25) * ub;
        }
        for (int i = t0; i < m.C; i += stride) {
            const R zb = fe_cell<R>(m, c, i, ua, za, tau);
            if (ORDER == 2)
                z0[i] = R(0.5) * (z0[i] + zb);
            else
                zh[i] = R(0.75) * z0[i] + R(0.25) * zb;
        }
        if (!grid_barrier(bar, gen, nb)) return;
        if (ORDER == 3) {
            // stage c: FE(uh, zh), then the second convex combination
            for (int e = t0; e < m.E; e += stride) {
                R f;
                const R uc = fe_edge<R>(m, c, e, uh, zh, a.G, tau, g, f);
                a.Fz[e] += wC * (double)f;
                u0[e] = u0[e] / R(3) + R(2) * uc / R(3);
            }
            for (int i = t0; i < m.C; i += stride) {
                const R zc = fe_cell<R>(m, c, i, uh, zh, tau);
                z0[i] = z0[i] / R(3) + R(2) * zc / R(3);
            }
            if (!grid_barrier(bar, gen, nb)) return;
        }
    }
    for (int e = t0; e < m.E; e += stride)
        a.ub_out[e] = a.X ? (R)(a.alpha * (double)a.X[e] + a.beta * (double)u0[e]) : u0[e];
    if (a.z_out)
        for (int i = t0; i < m.C; i += stride) a.z_out[i] = (double)z0[i];
}

template <class R> int btr_block_size() { return BTR_THREADS; }
template <class R> const void *btr_kernel_ptr(int order) {
    return order == 2 ? (const void *)k_btr<R, 2> : (const void *)k_btr<R, 3>;
}

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
    return cudaLaunchKernelExC(&cfg, btr_kernel_ptr<R>(a.order), args);
}

template int btr_block_size<double>();
template int btr_block_size<float>();
template const void *btr_kernel_ptr<double>(int);
template const void *btr_kernel_ptr<float>(int);
template cudaError_t launch_btr<double>(const DMesh &, const BtrArgs<double> &, const Barrier &,
                                        int, int, cudaStream_t);
template cudaError_t launch_btr<float>(const DMesh &, const BtrArgs<float> &, const Barrier &, int,
                                       int, cudaStream_t);

}  // namespace sse

// ===========================================================================
// Allocation-free sub-cycle: sse_barotropic_substep_noalloc
//
// For callers that cannot allocate device memory when they run the
// sub-cycle (for example code that executes while a CUDA stream is being
// captured into a graph, or inside an allocator callback or a memory pool
// that forbids new allocations): the work buffers live in one file-scope
// device array that every GPU loading this library holds until the process
// exits.  The first 256 bytes hold the grid-barrier words and the error word.
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
    int blocks_per_sm = 0, sms = 0;
};
NoallocDevice g_noalloc_dev[kMaxDevices];
std::mutex g_noalloc_mutex;
}  // namespace

}  // namespace sse

const sse::DMesh *sse_internal_dmesh(const sse_mesh *m);

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
    NoallocDevice nd;
    {
        // once per device, with that device current: the device address of the
        // array (the host-side symbol is only a stand-in for it)
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        NoallocDevice &d = g_noalloc_dev[dev];
        if (!d.scratch) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return SSE_ERR_CUDA;
            int occ2 = 0, occ3 = 0, nsm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_btr<double, 2>,
                                                              BTR_THREADS, 0) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ3, k_btr<double, 3>,
                                                              BTR_THREADS, 0) != cudaSuccess ||
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return SSE_ERR_CUDA;
            d.blocks_per_sm = occ2 < occ3 ? occ2 : occ3;
            d.sms = nsm;
            d.scratch = (double *)p;
        }
        nd = d;
    }
    if (nd.blocks_per_sm < 1) return SSE_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *base = nd.scratch;
    unsigned int *words = (unsigned int *)base;
    double *work = base + NOALLOC_HEADER;
    BtrArgs<double> a{};
    a.ub_start = ubar_in; a.z_start = zeta_in; a.G = G; a.X = nullptr; a.alpha = 0.0;
    a.beta = 1.0; a.ub_out = ubar_out; a.Fz = Fzeta_out; a.z_out = zeta_out;
    a.u0 = work; a.ua = work + NOALLOC_MAX_EDGES; a.uh = work + 2 * NOALLOC_MAX_EDGES;
    a.z0 = work + 3 * NOALLOC_MAX_EDGES; a.za = a.z0 + NOALLOC_MAX_CELLS;
    a.zh = a.z0 + 2 * NOALLOC_MAX_CELLS;
    a.tau = dt / n_substeps; a.g = g; a.M = n_substeps; a.order = order;
    Barrier bar{words, words + 1, (int *)(words + 2)};
    // the array keeps the previous call's contents: zero the barrier and error words
    if (cudaMemsetAsync(base, 0, NOALLOC_HEADER * sizeof(double), s) != cudaSuccess)
        return SSE_ERR_CUDA;
    const int need = ((m.E > m.C ? m.E : m.C) + BTR_THREADS - 1) / BTR_THREADS;
    int blocks = nd.blocks_per_sm * nd.sms;
    if (need < blocks) blocks = need;
    if (blocks < 1) blocks = 1;
    if (launch_btr<double>(m, a, bar, blocks, BTR_THREADS, s) != cudaSuccess) return SSE_ERR_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, words + 2, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SSE_ERR_CUDA;
    return err ? SSE_ERR_SYNC_TIMEOUT : SSE_OK;
}
