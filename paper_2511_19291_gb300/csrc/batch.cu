// batch.cu -- many independent circuits (the batch dimension of Sec. 4) in
// one CUDA-graph launch.
//
// Small circuits (complex64, width <= small_max_qubits, psi and lambda both
// fit in shared memory) run whole inside one block: a persistent kernel pulls
// circuit indices from a work queue, resets psi to |0...0>, applies the gates
// (each one the contraction M x_Q psi of Algorithm 1, done by all threads over
// the amplitude pairs or quads), forms lambda = H psi and E = Re<psi|lambda>,
// then sweeps the gates in reverse, reducing each angle derivative over the
// block and un-applying the gate from psi and lambda (Sec. 4.4).  Wider
// circuits run their own planned passes on several streams captured into the
// same graph.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "plan.h"
#include "prof.h"
#include "tile_dev.cuh"
#include "tile_plan.h"

namespace tqd {

struct SmallCirc {
    int n;
    int gate0, ngate;
    int term0, nterm;
    int poff;   // offset of this circuit's angles and gradients
    int index;  // position in the batch (energy output)
    int pad;
};

struct BGate {
    uint8_t kind, nw, w0, w1;
    int32_t param;  // local parameter index, -1 = none
    int32_t gen;    // generator class when the derivative is wanted, else 0
    int32_t pad;
};

struct BTerm {
    uint64_t x, z;
    double cre, cim;  // coeff * i^{|x & z|}
};

__device__ __forceinline__ float2 sm_m(const float *m, int idx) { return make_float2(m[2 * idx], m[2 * idx + 1]); }

// Apply gate (or its inverse) to one shared-memory state: the threads of the
// block share the pairs (1-qubit gates) or quads (2-qubit gates).
__device__ void small_apply(float2 *s, int n, const BGate &g, const float *m, bool dag) {
    const uint32_t N = 1u << n;
    if (g.nw == 1) {
        M2<float2> M;
        M.a = sm_m(m, 0); M.b = sm_m(m, 1); M.c = sm_m(m, 2); M.d = sm_m(m, 3);
        if (dag) M = dagger2(M);
        const uint32_t T = 1u << g.w0;
        for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
            const uint32_t b = (uint32_t)insert0(p, g.w0);
            float2 x0 = s[b], x1 = s[b | T];
            mv2(M, x0, x1);
            s[b] = x0;
            s[b | T] = x1;
        }
    } else {
        float2 M[16];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) M[r * 4 + c] = dag ? conjv(sm_m(m, c * 4 + r)) : sm_m(m, r * 4 + c);
        const int lo = min(g.w0, g.w1), hi = max(g.w0, g.w1);
        const uint32_t W0 = 1u << g.w0, W1 = 1u << g.w1;
        for (uint32_t p = threadIdx.x; p < N / 4; p += blockDim.x) {
            const uint32_t b = (uint32_t)insert00(p, lo, hi);
            const uint32_t idx[4] = {b, b | W1, b | W0, b | W0 | W1};
            float2 v[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) v[l] = s[idx[l]];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float2 acc = cmul(M[r * 4 + 0], v[0]);
#pragma unroll
                for (int c = 1; c < 4; ++c) acc = cfma(M[r * 4 + c], v[c], acc);
                s[idx[r]] = acc;
            }
        }
    }
}

// This thread's share of 2 Re<lambda| dG/dt |psi_before>, from the states after the gate.
__device__ double small_grad(const float2 *ps, const float2 *ls, int n, const BGate &g) {
    const uint32_t N = 1u << n;
    KSum<float> acc;
    if (g.nw == 1) {
        const uint32_t T = 1u << g.w0;
        for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
            const uint32_t b = (uint32_t)insert0(p, g.w0);
            const float2 p0 = ps[b], p1 = ps[b | T], l0 = ls[b], l1 = ls[b | T];
            switch (g.gen) {
            case GEN_X: acc.add(im_cdot(l0, p1) + im_cdot(l1, p0)); break;
            case GEN_Y: acc.add(re_cdot(l1, p0) - re_cdot(l0, p1)); break;
            case GEN_Z: acc.add(im_cdot(l0, p0) - im_cdot(l1, p1)); break;
            default: acc.add(-2.f * im_cdot(l1, p1)); break;  // GEN_P1
            }
        }
    } else {  // GEN_P11
        const uint32_t W = (1u << g.w0) | (1u << g.w1);
        const int lo = min(g.w0, g.w1), hi = max(g.w0, g.w1);
        for (uint32_t p = threadIdx.x; p < N / 4; p += blockDim.x) {
            const uint32_t b = (uint32_t)insert00(p, lo, hi) | W;
            acc.add(-2.f * im_cdot(ls[b], ps[b]));
        }
    }
    return acc.value();
}

// Block-wide FP64 sum, valid in thread 0; contains two barriers.
__device__ __forceinline__ double small_block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    __syncthreads();
    return r;
}

__global__ void k_batch_small(const SmallCirc *__restrict__ circs, int ncirc, const BGate *__restrict__ gates,
                              const float *__restrict__ mats, const BTerm *__restrict__ terms,
                              double *__restrict__ energies, double *__restrict__ grads, int *__restrict__ counter) {
    extern __shared__ float2 sbuf[];
    __shared__ int s_c;
    __shared__ double s_red[32];
    for (;;) {
        if (threadIdx.x == 0) s_c = atomicAdd(counter, 1);
        __syncthreads();
        const int c = s_c;
        __syncthreads();
        if (c >= ncirc) return;
        const SmallCirc C = circs[c];
        const uint32_t N = 1u << C.n;
        float2 *psi = sbuf, *lam = sbuf + N;
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) psi[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
        __syncthreads();
        for (int g = C.gate0; g < C.gate0 + C.ngate; ++g) {
            small_apply(psi, C.n, gates[g], mats + (size_t)g * MAT_STRIDE, false);
            __syncthreads();
        }
        // lambda = H psi and E = Re<psi|lambda>
        KSum<float> e;
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
            float2 l = make_float2(0.f, 0.f);
            for (int t = C.term0; t < C.term0 + C.nterm; ++t) {
                const BTerm T = terms[t];
                const uint32_t src = i ^ (uint32_t)T.x;
                const float s = (__popc(src & (uint32_t)T.z) & 1) ? -1.f : 1.f;
                l = cfma(make_float2(s * (float)T.cre, s * (float)T.cim), psi[src], l);
            }
            lam[i] = l;
            e.add(re_cdot(psi[i], l));
        }
        const double E = small_block_sum(e.value(), s_red);
        if (threadIdx.x == 0) energies[C.index] = E;
        __syncthreads();
        for (int g = C.gate0 + C.ngate - 1; g >= C.gate0; --g) {
            const BGate G = gates[g];
            const float *m = mats + (size_t)g * MAT_STRIDE;
            if (G.gen) {
                const double d = small_block_sum(small_grad(psi, lam, C.n, G), s_red);
                if (threadIdx.x == 0) grads[C.poff + G.param] += d;
            }
            small_apply(psi, C.n, G, m, true);
            small_apply(lam, C.n, G, m, true);
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------- wider circuits
// The wider circuits run from one persistent kernel that pulls work items
// from a queue in device memory.  A circuit goes through stages: reset psi,
// its forward passes, lambda = H psi with E, its reverse passes, then a
// closing step (E and the gradient summed).  Every stage but the last is
// split into `chunks` items over the circuit's tiles (or amplitudes); the
// block that finishes the last item of a stage pushes the items of the next
// one, so a block only ever waits for the queue itself, and other circuits'
// items fill the machine while a stage completes.  An item is processed by
// one block of two groups of 256 threads on a ring of tile buffers (the
// fused pass body of the single-circuit kernels, generic runner).
struct WideCirc {
    float2 *psi, *lam;          // its states
    const float *mats;          // its per-gate matrices (complex64 scalars)
    double *partials;           // [slot][pblk] gradient partials
    const int *param_ptr;       // CSR: parameter -> gradient slots
    const int *param_slots;
    int *err;                   // its device error word
    int n, n_params, pblk;
    int passes, pass0;          // its passes: WidePass[pass0 .. pass0 + passes)
    int chunks, tpc;            // items per stage, tiles per item
    int term0, nterm;           // its observable (BTerm)
    int poff, index;            // angle offset; position in the batch
    int stage0;                 // its first stage counter
    int e0;                     // its first energy partial
};

struct WidePass {
    const TilePassDev *desc;    // complex64 descriptor
    int map;                    // its psi tensor map (lambda's: map + 1)
    int pad;
};

constexpr int WIDE_THREADS = 2 * TILE_THREADS;
constexpr int WIDE_FWD_B = 6;   // forward ring: 6 buffers of 32 KiB
constexpr int WIDE_REV_B = 3;   // reverse ring: 3 buffers of 64 KiB (psi and lambda)
constexpr unsigned long long WIDE_VALID = 1ull << 63;

__host__ __device__ inline unsigned long long wide_item(int circ, int stage, int chunk) {
    return WIDE_VALID | ((unsigned long long)chunk << 40) | ((unsigned long long)stage << 20) | (unsigned)circ;
}

__global__ void __launch_bounds__(WIDE_THREADS, 1)
    k_batch_wide(const WideCirc *__restrict__ circs, const WidePass *__restrict__ passes,
                 const CUtensorMap *__restrict__ maps, const BTerm *__restrict__ terms,
                 unsigned long long *queue, unsigned *qctl, int *done, int total, double *eparts,
                 double *__restrict__ energies, double *__restrict__ grads, int *qerr) {
    __shared__ unsigned long long s_item;
    __shared__ double s_red[WIDE_THREADS / 32];
    const uint32_t tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            // next position of the queue; its item may not be pushed yet
            const unsigned pos = atomicAdd(qctl, 1u);
            unsigned long long it = 0;
            if (pos < (unsigned)total) {
                volatile unsigned long long *q = queue + pos;
                it = *q;
                if (!(it & WIDE_VALID)) {
                    const uint64_t t0 = gtimer_ns();
                    while (!((it = *q) & WIDE_VALID))
                        if (gtimer_ns() - t0 > WAIT_LIMIT_NS) {
                            atomicExch(qerr, 1);
                            it = 0;
                            break;
                        }
                }
                __threadfence();  // the item's data was written before it was pushed
            }
            s_item = it;
        }
        __syncthreads();
        const unsigned long long it = s_item;
        __syncthreads();
        if (!(it & WIDE_VALID)) return;
        // the tile copies below (async proxy) come after the acquire above
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const int ci = (int)(it & 0xFFFFF), stage = (int)((it >> 20) & 0xFFFFF), k = (int)((it >> 40) & 0xFFFFF);
        const WideCirc &C = circs[ci];
        const int P = C.passes;
        const uint64_t A = (uint64_t)1 << C.n;
        if (stage == 0) {
            // psi = |0...0> over this item's share of the amplitudes
            const uint64_t lo = A * k / C.chunks, hi = A * (k + 1) / C.chunks;
            for (uint64_t b = lo + tid; b < hi; b += blockDim.x) C.psi[b] = make_float2(b == 0 ? 1.f : 0.f, 0.f);
        } else if (stage <= P) {
            const WidePass W = passes[C.pass0 + stage - 1];
            tile_ring_tiles<float2, false, 2, WIDE_FWD_B, false, InterpRunner<float2, false>, true>(
                maps + W.map, maps + W.map, W.desc, C.mats, nullptr, 0, C.err, 0, (uint64_t)k * C.tpc, 1, C.tpc, 0);
        } else if (stage == P + 1) {
            // lambda = H psi on this item's amplitudes, and its share of
            // E = Re <psi|lambda> in FP64
            const uint64_t lo = A * k / C.chunks, hi = A * (k + 1) / C.chunks;
            double e = 0;
            for (uint64_t b = lo + tid; b < hi; b += blockDim.x) {
                float2 l = make_float2(0.f, 0.f);
                for (int t = C.term0; t < C.term0 + C.nterm; ++t) {
                    const BTerm T = terms[t];
                    const uint64_t src = b ^ T.x;
                    const float sg = (__popcll(src & T.z) & 1) ? -1.f : 1.f;
                    l = cfma(make_float2(sg * (float)T.cre, sg * (float)T.cim), C.psi[src], l);
                }
                C.lam[b] = l;
                e += (double)re_cdot(C.psi[b], l);
            }
            const double tot = block_sum(e, s_red);
            if (tid == 0) eparts[C.e0 + k] = tot;
        } else if (stage <= 2 * P + 1) {
            const WidePass W = passes[C.pass0 + (2 * P + 1 - stage)];
            tile_ring_tiles<float2, true, 2, WIDE_REV_B, false, InterpRunner<float2, true>, true>(
                maps + W.map, maps + W.map + 1, W.desc, C.mats, C.partials, C.pblk, C.err, 0, (uint64_t)k * C.tpc, 1,
                C.tpc, k);
        } else {
            // closing step: E and every parameter's derivative, summed in
            // FP64 in a fixed order (items, then the parameter's slots)
            if (tid == 0) {
                double e = 0;
                for (int j = 0; j < C.chunks; ++j) e += eparts[C.e0 + j];
                energies[C.index] = e;
            }
            for (int p = tid; p < C.n_params; p += blockDim.x) {
                double g = 0;
                for (int j = C.param_ptr[p]; j < C.param_ptr[p + 1]; ++j) {
                    const double *row = C.partials + (size_t)C.param_slots[j] * C.pblk;
                    for (int q = 0; q < C.chunks; ++q) g += row[q];
                }
                grads[C.poff + p] += g;
            }
        }
        // this item is done: the block that completes its stage pushes the
        // next stage's items (after its own writes and, through the stage
        // counter, everyone else's)
        __syncthreads();
        if (tid == 0 && stage < 2 * P + 2) {
            __threadfence();
            const int old = atomicAdd(done + C.stage0 + stage, 1);
            if (old == C.chunks - 1) {
                __threadfence();
                const int ns = stage + 1;
                const int cnt = ns == 2 * P + 2 ? 1 : C.chunks;
                const unsigned pos = atomicAdd(qctl + 1, (unsigned)cnt);
                for (int j = 0; j < cnt; ++j) atomicExch(queue + pos + j, wide_item(ci, ns, j));
            }
        }
    }
}

}  // namespace tqd

using namespace tqd;

struct tqd_batch {
    int device;
    tqd_batch_opts opts;
    std::vector<const tqd_circuit *> circuits;
    std::vector<std::vector<PauliGroup>> groups;
    std::vector<size_t> poff;
    size_t total_params;
    double *d_params, *d_energies, *d_grads;
    std::vector<int> small, large;
    // small-circuit data
    SmallCirc *d_small;
    BGate *d_bgates;
    BTerm *d_bterms;
    GateDev *d_bgdev;
    double *d_btable;
    double *d_bm64;
    float *d_bm32;
    int *d_counter;
    int n_bgates;
    int small_smem_q;  // largest small width
    // wider circuits
    void *d_arena;
    std::vector<tqd_state *> st_psi, st_lam;
    // ... on the persistent work-queue kernel (wide == true), else on streams
    bool wide;
    int tpc[27];                      // tiles per work item, by width
    WideCirc *d_wcircs;
    WidePass *d_wpasses;
    CUtensorMap *d_wmaps;
    BTerm *d_wterms;
    GateDev *d_wgdev;
    double *d_wtable, *d_wm64;
    float *d_wm32;
    int n_wgates;
    unsigned long long *d_queue, *d_qinit;
    unsigned *d_qctl, *d_qctl_init;
    int *d_done, *d_qerr;
    double *d_eparts;
    int total_items, n_init, n_counters, wide_smem;
    int tpc_used[27], items_used[27];  // the tiling each width got (0: none there)
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool captured;
    int graph_nodes;
};

namespace {

void free_wide(tqd_batch *b) {
    cudaFree(b->d_wcircs);
    cudaFree(b->d_wpasses);
    cudaFree(b->d_wmaps);
    cudaFree(b->d_wterms);
    cudaFree(b->d_wgdev);
    cudaFree(b->d_wtable);
    cudaFree(b->d_wm64);
    cudaFree(b->d_wm32);
    cudaFree(b->d_queue);
    cudaFree(b->d_qinit);
    cudaFree(b->d_qctl);
    cudaFree(b->d_qctl_init);
    cudaFree(b->d_done);
    cudaFree(b->d_qerr);
    cudaFree(b->d_eparts);
    b->d_wcircs = nullptr;
    b->d_wpasses = nullptr;
    b->d_wmaps = nullptr;
    b->d_wterms = nullptr;
    b->d_wgdev = nullptr;
    b->d_wtable = b->d_wm64 = nullptr;
    b->d_wm32 = nullptr;
    b->d_queue = b->d_qinit = nullptr;
    b->d_qctl = b->d_qctl_init = nullptr;
    b->d_done = b->d_qerr = nullptr;
    b->d_eparts = nullptr;
    b->wide = false;
}

void free_batch_device(tqd_batch *b) {
    cudaFree(b->d_params);
    cudaFree(b->d_energies);
    cudaFree(b->d_grads);
    cudaFree(b->d_small);
    cudaFree(b->d_bgates);
    cudaFree(b->d_bterms);
    cudaFree(b->d_bgdev);
    cudaFree(b->d_btable);
    cudaFree(b->d_bm64);
    cudaFree(b->d_bm32);
    cudaFree(b->d_counter);
    for (auto *s : b->st_psi) tqd_state_free(s);
    for (auto *s : b->st_lam) tqd_state_free(s);
    b->st_psi.clear();
    b->st_lam.clear();
    cudaFree(b->d_arena);
    free_wide(b);
    b->d_params = b->d_energies = b->d_grads = nullptr;
    b->d_small = nullptr;
    b->d_bgates = nullptr;
    b->d_bterms = nullptr;
    b->d_bgdev = nullptr;
    b->d_btable = nullptr;
    b->d_bm64 = nullptr;
    b->d_bm32 = nullptr;
    b->d_counter = nullptr;
    b->d_arena = nullptr;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->captured = false;
}

template <typename T>
cudaError_t up(T **dst, const std::vector<T> &v) {
    *dst = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)dst, v.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Tiles per work item of the wider circuits' stages, by default: at least 2
// (one per group of the block), about 8 items per stage, at most 16 tiles.
int default_tpc(int n) {
    const int tiles = 1 << std::max(0, n - TILE_K);
    return std::max(std::min(tiles, 2), std::min(16, tiles / 8));
}

// The persistent kernel's tables for the wider circuits: circuits, passes,
// tensor maps, concatenated gate records (one matrix preparation launch for
// all of them), observables, and the work queue.  Leaves b->wide false (the
// circuits then run on streams) when a circuit has no fused plan of complex64
// tile passes or a pass's ring does not fit in shared memory.
cudaError_t build_wide(tqd_batch *b) {
    free_wide(b);
    if (b->large.empty()) return cudaSuccess;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    std::vector<WideCirc> wc;
    std::vector<WidePass> wp;
    std::vector<CUtensorMap> maps;
    std::vector<BTerm> bt;
    std::vector<GateDev> gd;
    std::vector<double> table;
    std::vector<int> goff;
    int smem = 0, counters = 0, eparts = 0, total = 0;
    for (int w = 0; w < 27; ++w) b->tpc_used[w] = b->items_used[w] = 0;
    for (size_t i = 0; i < b->large.size(); ++i) {
        const tqd_circuit *C = b->circuits[b->large[i]];
        if (!C->fused || C->tile_passes.empty()) return cudaSuccess;
        for (const auto &pp : C->tile_passes)
            if (pp.tc >= 0) return cudaSuccess;
        const int c = b->large[i];
        WideCirc w;
        memset(&w, 0, sizeof(w));
        w.psi = (float2 *)b->st_psi[i]->amps;
        w.lam = (float2 *)b->st_lam[i]->amps;
        w.partials = C->d_partials;
        w.param_ptr = C->d_param_ptr;
        w.param_slots = C->d_param_slots;
        w.err = C->d_err;
        w.n = C->n;
        w.n_params = C->n_params;
        w.pblk = C->pblk;
        w.passes = (int)C->tile_passes.size();
        w.pass0 = (int)wp.size();
        const int tiles = 1 << (C->n - TILE_K);
        w.tpc = std::min(tiles, std::max(1, b->tpc[C->n] > 0 ? b->tpc[C->n] : default_tpc(C->n)));
        w.chunks = std::min((tiles + w.tpc - 1) / w.tpc, std::max(1, C->pblk));
        w.tpc = (tiles + w.chunks - 1) / w.chunks;
        w.chunks = (tiles + w.tpc - 1) / w.tpc;
        b->tpc_used[C->n] = w.tpc;
        b->items_used[C->n] = w.chunks;
        w.term0 = (int)bt.size();
        w.poff = (int)b->poff[c];
        w.index = c;
        w.stage0 = counters;
        w.e0 = eparts;
        counters += 2 * w.passes + 2;
        eparts += w.chunks;
        total += w.chunks * (2 * w.passes + 2) + 1;
        for (int p = 0; p < w.passes; ++p) {
            const TilePlanPass &pp = C->tile_passes[p];
            const TileHead &h = pp.dev[0].h;
            smem = std::max<int>(smem, (int)tile_smem_ring<float2, false, WIDE_FWD_B>(h).total);
            smem = std::max<int>(smem, (int)tile_smem_ring<float2, true, WIDE_REV_B>(h).total);
            WidePass x;
            x.desc = C->d_tile_desc + 2 * p;
            x.map = (int)maps.size();
            x.pad = 0;
            wp.push_back(x);
            CUtensorMap m[2];
            cudaError_t e = tile_tensor_map(&m[0], w.psi, pp, 0);
            if (e == cudaSuccess) e = tile_tensor_map(&m[1], w.lam, pp, 0);
            if (e != cudaSuccess) return cudaSuccess;  // no tensor map: streams
            maps.push_back(m[0]);
            maps.push_back(m[1]);
        }
        int nt = 0;
        for (const auto &grp : b->groups[c])
            for (const auto &t : grp.terms) {
                BTerm T;
                T.x = grp.xmask;
                T.z = t.zmask;
                T.cre = t.pre * t.coeff;
                T.cim = t.pim * t.coeff;
                bt.push_back(T);
                ++nt;
            }
        w.nterm = nt;
        goff.push_back((int)gd.size());
        const int toff = (int)table.size() / 2;
        table.insert(table.end(), C->table.begin(), C->table.end());
        for (const GateH &h : C->gates) {
            GateDev d;
            d.kind = h.kind;
            d.param = h.param >= 0 ? (int)(h.param + b->poff[c]) : -1;
            d.mat = h.mat >= 0 ? h.mat + toff : -1;
            d.pad = 0;
            d.fixed = h.fixed;
            gd.push_back(d);
        }
        wc.push_back(w);
    }
    // the ring's static part (descriptor head, barriers, counters) comes on top
    if (smem + 4096 > optin) return cudaSuccess;
    cudaError_t e;
    b->n_wgates = (int)gd.size();
    if ((e = up(&b->d_wgdev, gd)) != cudaSuccess) return e;
    if ((e = up(&b->d_wtable, table.empty() ? std::vector<double>(2, 0.0) : table)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&b->d_wm64, gd.size() * MAT_STRIDE * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&b->d_wm32, gd.size() * MAT_STRIDE * sizeof(float))) != cudaSuccess) return e;
    for (size_t i = 0; i < wc.size(); ++i) wc[i].mats = b->d_wm32 + (size_t)goff[i] * MAT_STRIDE;
    if ((e = up(&b->d_wcircs, wc)) != cudaSuccess) return e;
    if ((e = up(&b->d_wpasses, wp)) != cudaSuccess) return e;
    if ((e = up(&b->d_wmaps, maps)) != cudaSuccess) return e;
    if ((e = up(&b->d_wterms, bt.empty() ? std::vector<BTerm>(1) : bt)) != cudaSuccess) return e;
    // the first items: every circuit's reset, the costliest circuits first
    std::vector<int> order(wc.size());
    for (size_t i = 0; i < wc.size(); ++i) order[i] = (int)i;
    auto cost = [&](int i) {
        return (double)((uint64_t)1 << wc[i].n) * (double)b->circuits[b->large[i]]->gates.size();
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::vector<unsigned long long> init;
    for (int i : order)
        for (int k = 0; k < wc[i].chunks; ++k) init.push_back(wide_item(i, 0, k));
    if ((e = up(&b->d_qinit, init)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&b->d_queue, (size_t)total * sizeof(unsigned long long))) != cudaSuccess) return e;
    const std::vector<unsigned> qctl = {0u, (unsigned)init.size()};
    if ((e = up(&b->d_qctl_init, qctl)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&b->d_qctl, 2 * sizeof(unsigned))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&b->d_done, (size_t)counters * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&b->d_eparts, (size_t)std::max(1, eparts) * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&b->d_qerr, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemset(b->d_qerr, 0, sizeof(int))) != cudaSuccess) return e;
    b->total_items = total;
    b->n_init = (int)init.size();
    b->n_counters = counters;
    b->wide_smem = smem + 1024;
    if ((e = cudaFuncSetAttribute(k_batch_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, b->wide_smem)) !=
        cudaSuccess)
        return e;
    b->wide = true;
    return cudaSuccess;
}

// Split circuits into the small set and the wider set, build the
// small-circuit arrays and the states of the wider circuits.
cudaError_t layout_batch(tqd_batch *b, int small_max) {
    b->small.clear();
    b->large.clear();
    const int nc = (int)b->circuits.size();
    for (int c = 0; c < nc; ++c) {
        if (!b->opts.plain && b->circuits[c]->n <= small_max) b->small.push_back(c);
        else b->large.push_back(c);
    }
    // small circuits: concatenated gates, terms and matrices
    std::vector<SmallCirc> sc;
    std::vector<BGate> bg;
    std::vector<BTerm> bt;
    std::vector<GateDev> gd;
    std::vector<double> table;
    b->small_smem_q = 1;
    for (int c : b->small) {
        const tqd_circuit *C = b->circuits[c];
        SmallCirc s;
        s.n = C->n;
        s.gate0 = (int)bg.size();
        s.ngate = (int)C->gates.size();
        s.term0 = (int)bt.size();
        s.poff = (int)b->poff[c];
        s.index = c;
        s.pad = 0;
        b->small_smem_q = std::max(b->small_smem_q, C->n);
        const int toff = (int)table.size() / 2;
        table.insert(table.end(), C->table.begin(), C->table.end());
        for (size_t g = 0; g < C->gates.size(); ++g) {
            const GateH &h = C->gates[g];
            BGate x;
            x.kind = (uint8_t)h.kind;
            x.nw = (uint8_t)h.nw;
            x.w0 = (uint8_t)h.w[0];
            x.w1 = (uint8_t)(h.nw > 1 ? h.w[1] : 0);
            x.param = h.param;
            x.gen = C->grad_slot[g] >= 0 ? gate_gen(h.kind) : 0;
            x.pad = 0;
            bg.push_back(x);
            GateDev d;
            d.kind = h.kind;
            d.param = h.param >= 0 ? (int)(h.param + b->poff[c]) : -1;
            d.mat = h.mat >= 0 ? h.mat + toff : -1;
            d.pad = 0;
            d.fixed = h.fixed;
            gd.push_back(d);
        }
        int nt = 0;
        for (const auto &grp : b->groups[c])
            for (const auto &t : grp.terms) {
                BTerm T;
                T.x = grp.xmask;
                T.z = t.zmask;
                T.cre = t.pre * t.coeff;
                T.cim = t.pim * t.coeff;
                bt.push_back(T);
                ++nt;
            }
        s.nterm = nt;
        sc.push_back(s);
    }
    b->n_bgates = (int)bg.size();
    cudaError_t e;
    if ((e = up(&b->d_small, sc)) != cudaSuccess) return e;
    if ((e = up(&b->d_bgates, bg)) != cudaSuccess) return e;
    if ((e = up(&b->d_bterms, bt)) != cudaSuccess) return e;
    if ((e = up(&b->d_bgdev, gd)) != cudaSuccess) return e;
    if ((e = up(&b->d_btable, table)) != cudaSuccess) return e;
    if (!bg.empty()) {
        if ((e = cudaMalloc((void **)&b->d_bm64, bg.size() * MAT_STRIDE * sizeof(double))) != cudaSuccess) return e;
        if ((e = cudaMalloc((void **)&b->d_bm32, bg.size() * MAT_STRIDE * sizeof(float))) != cudaSuccess) return e;
    }
    // states of the wider circuits: one arena, 256-byte aligned slices
    size_t bytes = 0;
    std::vector<size_t> off;
    for (int c : b->large) {
        off.push_back(bytes);
        bytes += ((size_t)8 << b->circuits[c]->n) * 2;
        bytes = (bytes + 255) & ~(size_t)255;
    }
    if (bytes) {
        if ((e = cudaMalloc(&b->d_arena, bytes)) != cudaSuccess) return e;
    }
    for (size_t i = 0; i < b->large.size(); ++i) {
        const int n = b->circuits[b->large[i]]->n;
        const size_t sb = (size_t)8 << n;
        tqd_state *p = nullptr, *l = nullptr;
        char *base = (char *)b->d_arena + off[i];
        if (tqd_state_alloc(n, TQD_C64, base, sb, &p) != TQD_OK) return cudaErrorInvalidValue;
        if (tqd_state_alloc(n, TQD_C64, base + ((sb + 255) & ~(size_t)255), sb, &l) != TQD_OK)
            return cudaErrorInvalidValue;
        b->st_psi.push_back(p);
        b->st_lam.push_back(l);
    }
    return b->opts.plain ? cudaSuccess : build_wide(b);
}

// Everything one batch run does, enqueued on `s` (and the worker streams).
cudaError_t enqueue_batch(tqd_batch *b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->d_grads, 0, b->total_params * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int nstreams = (int)b->streams.size();
    if (nstreams > 0) {
        if ((e = cudaEventRecord(b->events[0], s)) != cudaSuccess) return e;
        for (int i = 0; i < nstreams; ++i)
            if ((e = cudaStreamWaitEvent(b->streams[i], b->events[0], 0)) != cudaSuccess) return e;
    }
    // small circuits on the origin stream
    if (!b->small.empty()) {
        ProfScope ps(PK_BATCH, 0.0, s);
        if ((e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s)) != cudaSuccess) return e;
        if ((e = launch_prep_raw(b->d_bgdev, b->n_bgates, b->d_params, b->d_btable, b->d_bm64, b->d_bm32, s)) !=
            cudaSuccess)
            return e;
        const size_t smem = 2 * ((size_t)8 << b->small_smem_q);
        const int threads = (int)b->opts.small_threads;
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_small, threads, smem);
        if (nb < 1) nb = 1;
        int grid = device_sm_count() * nb;
        if (grid > (int)b->small.size()) grid = (int)b->small.size();
        k_batch_small<<<grid, threads, smem, s>>>(b->d_small, (int)b->small.size(), b->d_bgates, b->d_bm32,
                                                  b->d_bterms, b->d_energies, b->d_grads, b->d_counter);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // wider circuits: the persistent work-queue kernel
    if (b->wide) {
        ProfScope ps(PK_BATCH, 0.0, s);
        const size_t qbytes = (size_t)b->total_items * sizeof(unsigned long long);
        if ((e = cudaMemsetAsync(b->d_queue, 0, qbytes, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(b->d_queue, b->d_qinit, (size_t)b->n_init * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpyAsync(b->d_qctl, b->d_qctl_init, 2 * sizeof(unsigned), cudaMemcpyDeviceToDevice, s)) !=
            cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(b->d_done, 0, (size_t)b->n_counters * sizeof(int), s)) != cudaSuccess) return e;
        if ((e = launch_prep_raw(b->d_wgdev, b->n_wgates, b->d_params, b->d_wtable, b->d_wm64, b->d_wm32, s)) !=
            cudaSuccess)
            return e;
        k_batch_wide<<<device_sm_count(), WIDE_THREADS, b->wide_smem, s>>>(
            b->d_wcircs, b->d_wpasses, b->d_wmaps, b->d_wterms, b->d_queue, b->d_qctl, b->d_done, b->total_items,
            b->d_eparts, b->d_energies, b->d_grads, b->d_qerr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (nstreams > 0) {
            for (int i = 0; i < nstreams; ++i) {
                if ((e = cudaEventRecord(b->events[1 + i], b->streams[i])) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(s, b->events[1 + i], 0)) != cudaSuccess) return e;
            }
        }
        return cudaSuccess;
    }
    // wider circuits round-robin over the worker streams
    for (size_t i = 0; i < b->large.size(); ++i) {
        const int c = b->large[i];
        cudaStream_t ws = nstreams > 0 ? b->streams[i % nstreams] : s;
        const tqd_circuit *C = b->circuits[c];
        const double *p = b->d_params + b->poff[c];
        if ((e = launch_reset(b->st_psi[i], 0, ws)) != cudaSuccess) return e;
        if ((e = run_forward(b->st_psi[i], C, p, ws)) != cudaSuccess) return e;
        if ((e = launch_expval(b->st_psi[i], b->groups[c], 0, 0, b->d_energies + c, ws)) != cudaSuccess) return e;
        if ((e = run_backward(b->st_psi[i], b->st_lam[i], C, p, b->groups[c], nullptr, 1.0, b->d_grads + b->poff[c],
                              ws)) != cudaSuccess)
            return e;
    }
    if (nstreams > 0) {
        for (int i = 0; i < nstreams; ++i) {
            if ((e = cudaEventRecord(b->events[1 + i], b->streams[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, b->events[1 + i], 0)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

double time_batch(tqd_batch *b, cudaStream_t s) {
    cudaStreamSynchronize(s);
    auto t0 = std::chrono::steady_clock::now();
    for (int r = 0; r < 2; ++r)
        if (enqueue_batch(b, s) != cudaSuccess) return 1e30;
    cudaStreamSynchronize(s);
    for (auto ws : b->streams) cudaStreamSynchronize(ws);
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" {

tqd_status tqd_batch_create(int n_circuits, const tqd_circuit *const *circuits, const tqd_pauli_term *const *terms,
                            const size_t *n_terms, const tqd_batch_opts *opts, tqd_batch **out) {
    if (!out || n_circuits < 1 || !circuits || !terms || !n_terms) {
        set_error("tqd_batch_create: bad arguments");
        return TQD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    tqd_batch_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    for (int i = 0; i < 3; ++i)
        if (o.reserved[i]) {
            set_error("tqd_batch_create: reserved opts not zero");
            return TQD_ERR_INVALID_ARG;
        }
    if (o.small_max_qubits > 13) {
        set_error("tqd_batch_create: small_max_qubits %u > 13 (psi and lambda must fit in shared memory)",
                  o.small_max_qubits);
        return TQD_ERR_INVALID_ARG;
    }
    if (o.small_threads && (o.small_threads % 32 || o.small_threads > 1024)) {
        set_error("tqd_batch_create: small_threads must be a multiple of 32 up to 1024");
        return TQD_ERR_INVALID_ARG;
    }
    for (int c = 0; c < n_circuits; ++c) {
        if (!circuits[c] || (n_terms[c] && !terms[c])) {
            set_error("tqd_batch_create: circuit or terms %d missing", c);
            return TQD_ERR_INVALID_ARG;
        }
        if (circuits[c]->n > 26) {
            set_error("tqd_batch_create: circuit %d has %d qubits (at most 26 in a batch)", c, circuits[c]->n);
            return TQD_ERR_INVALID_ARG;
        }
        for (int d = 0; d < c; ++d)
            if (circuits[d] == circuits[c]) {
                set_error("tqd_batch_create: circuit %d appears twice (each entry needs its own circuit)", c);
                return TQD_ERR_INVALID_ARG;
            }
        for (size_t j = 0; j < n_terms[c]; ++j)
            if ((terms[c][j].xmask | terms[c][j].zmask) >> circuits[c]->n) {
                set_error("tqd_batch_create: circuit %d term %zu acts outside its qubits", c, j);
                return TQD_ERR_INVALID_ARG;
            }
    }
    tqd_batch *b = new (std::nothrow) tqd_batch();
    if (!b) {
        set_error("tqd_batch_create: out of host memory");
        return TQD_ERR_OOM;
    }
    cudaGetDevice(&b->device);
    b->opts = o;
    if (!b->opts.small_threads) b->opts.small_threads = 256;
    if (!b->opts.small_max_qubits) b->opts.small_max_qubits = 13;
    if (!b->opts.streams) b->opts.streams = 16;
    if (b->opts.plain) b->opts.streams = 1;
    b->circuits.assign(circuits, circuits + n_circuits);
    b->total_params = 0;
    for (int c = 0; c < n_circuits; ++c) {
        b->poff.push_back(b->total_params);
        b->total_params += circuits[c]->n_params;
        b->groups.push_back(group_terms(terms[c], n_terms[c]));
    }
    auto fail = [&](cudaError_t e) {
        set_error("tqd_batch_create: %s", cudaGetErrorString(e));
        free_batch_device(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? TQD_ERR_OOM : TQD_ERR_CUDA;
    };
    cudaError_t e;
    const size_t np = std::max<size_t>(1, b->total_params);
    if ((e = cudaMalloc((void **)&b->d_params, np * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(b->d_params, 0, np * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc((void **)&b->d_grads, np * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc((void **)&b->d_energies, n_circuits * sizeof(double))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc((void **)&b->d_counter, sizeof(int))) != cudaSuccess) return fail(e);
    for (uint32_t i = 0; i < b->opts.streams; ++i) {
        cudaStream_t s;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
        b->streams.push_back(s);
    }
    for (uint32_t i = 0; i < b->opts.streams + 1; ++i) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
        b->events.push_back(ev);
    }
    // shared memory for the largest small circuit (psi + lambda)
    cudaFuncSetAttribute(k_batch_small, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * (8 << 13));
    if ((e = layout_batch(b, (int)b->opts.small_max_qubits)) != cudaSuccess) return fail(e);
    if (o.autotune && !o.plain) {
        // block size of the small kernel, then the width cutoff
        cudaStream_t s = b->streams.empty() ? nullptr : b->streams[0];
        cudaStream_t ts;
        cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
        double best = 1e30;
        uint32_t best_t = b->opts.small_threads, best_q = b->opts.small_max_qubits;
        const uint32_t th[3] = {128, 256, 512};
        for (uint32_t t : th) {
            b->opts.small_threads = t;
            time_batch(b, ts);  // warm-up
            const double dt = time_batch(b, ts);
            if (dt < best) { best = dt; best_t = t; }
        }
        b->opts.small_threads = best_t;
        best = 1e30;
        const uint32_t qs[3] = {11, 12, 13};
        for (uint32_t q : qs) {
            free_batch_device(b);
            if ((e = cudaMalloc((void **)&b->d_params, np * sizeof(double))) != cudaSuccess) return fail(e);
            cudaMemset(b->d_params, 0, np * sizeof(double));
            if ((e = cudaMalloc((void **)&b->d_grads, np * sizeof(double))) != cudaSuccess) return fail(e);
            if ((e = cudaMalloc((void **)&b->d_energies, n_circuits * sizeof(double))) != cudaSuccess) return fail(e);
            if ((e = cudaMalloc((void **)&b->d_counter, sizeof(int))) != cudaSuccess) return fail(e);
            if ((e = layout_batch(b, (int)q)) != cudaSuccess) return fail(e);
            time_batch(b, ts);
            const double dt = time_batch(b, ts);
            if (dt < best) { best = dt; best_q = q; }
        }
        (void)s;
        cudaStreamDestroy(ts);
        b->opts.small_max_qubits = best_q;
        free_batch_device(b);
        if ((e = cudaMalloc((void **)&b->d_params, np * sizeof(double))) != cudaSuccess) return fail(e);
        if ((e = cudaMemset(b->d_params, 0, np * sizeof(double))) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc((void **)&b->d_grads, np * sizeof(double))) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc((void **)&b->d_energies, n_circuits * sizeof(double))) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc((void **)&b->d_counter, sizeof(int))) != cudaSuccess) return fail(e);
        if ((e = layout_batch(b, (int)best_q)) != cudaSuccess) return fail(e);
        // the wider circuits' work items: tiles per item, width by width
        if (b->wide) {
            cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
            for (int w = TILE_K; w <= 26; ++w) {
                if (!b->items_used[w]) continue;
                const int tiles = 1 << (w - TILE_K);
                int best_c = b->tpc_used[w];
                best = 1e30;
                for (int cand = 1; cand <= 32 && cand <= tiles; cand *= 2) {
                    b->tpc[w] = cand;
                    if ((e = build_wide(b)) != cudaSuccess) return fail(e);
                    if (!b->wide) break;
                    time_batch(b, ts);
                    const double dt = time_batch(b, ts);
                    if (dt < best) { best = dt; best_c = cand; }
                }
                b->tpc[w] = best_c;
            }
            if ((e = build_wide(b)) != cudaSuccess) return fail(e);
            cudaStreamDestroy(ts);
        }
    }
    *out = b;
    return TQD_OK;
}

tqd_status tqd_batch_buffers(tqd_batch *b, double **dev_params, double **dev_energies, double **dev_grads,
                             size_t *param_offset) {
    if (!b) {
        set_error("tqd_batch_buffers: batch is NULL");
        return TQD_ERR_INVALID_ARG;
    }
    if (dev_params) *dev_params = b->d_params;
    if (dev_energies) *dev_energies = b->d_energies;
    if (dev_grads) *dev_grads = b->d_grads;
    if (param_offset)
        for (size_t c = 0; c < b->poff.size(); ++c) param_offset[c] = b->poff[c];
    return TQD_OK;
}

tqd_status tqd_batch_run(tqd_batch *b, void *stream) {
    if (!b) {
        set_error("tqd_batch_run: batch is NULL");
        return TQD_ERR_INVALID_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (b->opts.plain) {
        e = enqueue_batch(b, s);  // the baseline: every launch issued by the host
    } else {
        if (!b->captured) {
            // eager run first: sizes the workspaces and sets kernel attributes
            e = enqueue_batch(b, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            for (auto ws : b->streams)
                if (e == cudaSuccess) e = cudaStreamSynchronize(ws);
            cudaStream_t cap = nullptr;
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue_batch(b, cap);
                e = cudaStreamEndCapture(cap, &b->graph);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e == cudaSuccess) {
                size_t nn = 0;
                cudaGraphGetNodes(b->graph, nullptr, &nn);
                b->graph_nodes = (int)nn;
                b->captured = true;
            }
            if (cap) cudaStreamDestroy(cap);
        }
        if (e == cudaSuccess) {
            ProfScope ps(PK_BATCH, 0.0, s);
            e = cudaGraphLaunch(b->exec, s);
        }
    }
    if (prev != b->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        set_error("tqd_batch_run: %s", cudaGetErrorString(e));
        return TQD_ERR_CUDA;
    }
    return TQD_OK;
}

tqd_status tqd_batch_info(const tqd_batch *b, int *n_small, int *n_large, int *small_max_qubits, int *small_threads,
                          int *graph_nodes) {
    if (!b) {
        set_error("tqd_batch_info: batch is NULL");
        return TQD_ERR_INVALID_ARG;
    }
    if (n_small) *n_small = (int)b->small.size();
    if (n_large) *n_large = (int)b->large.size();
    if (small_max_qubits) *small_max_qubits = (int)b->opts.small_max_qubits;
    if (small_threads) *small_threads = (int)b->opts.small_threads;
    if (graph_nodes) *graph_nodes = b->graph_nodes;
    return TQD_OK;
}

tqd_status tqd_batch_tiling(const tqd_batch *b, int width, int *tiles_per_item, int *items_per_stage) {
    if (!b || width < 0 || width > 26) {
        set_error("tqd_batch_tiling: NULL batch or width outside 0..26");
        return TQD_ERR_INVALID_ARG;
    }
    const bool on = b->wide && b->items_used[width] > 0;
    if (tiles_per_item) *tiles_per_item = on ? b->tpc_used[width] : 0;
    if (items_per_stage) *items_per_stage = on ? b->items_used[width] : 0;
    return TQD_OK;
}

tqd_status tqd_batch_free(tqd_batch *b) {
    if (!b) return TQD_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    free_batch_device(b);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto ev : b->events) cudaEventDestroy(ev);
    if (prev != b->device) cudaSetDevice(prev);
    delete b;
    return TQD_OK;
}

}  // extern "C"
