// kernels_tile.cu -- the generic fused tile pass kernel and the host side of
// every tile pass launch (tensor maps, occupancy, grid, dispatch to the
// pass-specialised kernels when a circuit has them).  The device code is in
// tile_dev.cuh.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "jit.h"
#include "launch.h"
#include "prof.h"
#include "tile.h"
#include "tile_dev.cuh"
#include "tile_plan.h"

namespace tqd {

// The generic pass: positions, addresses and matrices read from the pass
// descriptor at run time.
template <typename V, bool ADJ, int NB>
__global__ void __launch_bounds__(TILE_THREADS, tile_min_blocks<V, ADJ, NB>())
    k_tile(const __grid_constant__ CUtensorMap map_psi, const __grid_constant__ CUtensorMap map_lam,
           const TilePassDev *__restrict__ Pg, const RT<V> *__restrict__ mats, double *__restrict__ partials,
           int pblk, int *__restrict__ err, int flags) {
    tile_pass_body<V, ADJ, NB, InterpRunner<V, ADJ>>(&map_psi, &map_lam, Pg, mats, partials, pblk, err, flags);
}

// The generic pass on a ring of tile buffers (one block per SM, G groups,
// TMAW: plus a TMA warp).
template <typename V, bool ADJ, bool TMAW>
__global__ void __launch_bounds__((TMAW ? RingCfg<ADJ>::THREADS_TMAW : RingCfg<ADJ>::THREADS), 1)
    k_tile_ring(const __grid_constant__ CUtensorMap map_psi, const __grid_constant__ CUtensorMap map_lam,
                const TilePassDev *__restrict__ Pg, const RT<V> *__restrict__ mats, double *__restrict__ partials,
                int pblk, int *__restrict__ err, int flags) {
    tile_pass_ring<V, ADJ, RingCfg<ADJ>::G, RingCfg<ADJ>::B, TMAW, InterpRunner<V, ADJ>>(
        &map_psi, &map_lam, Pg, mats, partials, pblk, err, flags);
}

// ------------------------------------------------------------------- host
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

cudaError_t tile_tensor_map(CUtensorMap *map, void *base, const TilePlanPass &pp, int dt) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const TileLayout &L = pp.layout;
    const int rank = L.rank[dt];
    const int amp = dt == 0 ? 8 : 16;
    const int epa = dt == 0 ? 1 : 2;  // 8-byte elements per amplitude
    cuuint64_t gdim[TILE_MAX_DIMS], gstride[TILE_MAX_DIMS];
    cuuint32_t box[TILE_MAX_DIMS], estr[TILE_MAX_DIMS];
    for (int d = 0; d < rank; ++d) {
        const uint64_t len = (uint64_t)1 << L.dim_len[dt][d];
        gdim[d] = d == 0 ? len * epa : len;
        box[d] = L.dim_in[dt][d] ? (cuuint32_t)(d == 0 ? len * epa : len) : 1u;
        estr[d] = 1;
        if (d > 0) gstride[d - 1] = ((uint64_t)1 << L.dim_lo[dt][d]) * amp;
    }
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, base, gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename V, bool ADJ, int NB>
static int occupancy_for(uint32_t smem) {
    static std::mutex mu;
    static uint32_t set_to = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (smem > set_to) {
            cudaFuncSetAttribute(k_tile<V, ADJ, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            set_to = smem;
        }
    }
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tile<V, ADJ, NB>, TILE_THREADS, smem);
    return nb > 0 ? nb : 1;
}

template <typename V, bool ADJ, int NB>
static uint32_t max_smem(const tqd_circuit *c, int dt) {
    uint32_t m = 0;
    for (const auto &p : c->tile_passes) {
        const TileSmem s = tile_smem<V, ADJ, NB>(p.dev[dt].h);
        if (s.total > m) m = s.total;
    }
    return m;
}

static int smem_optin_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return v;
}

// Tile buffers per block.  complex64 defaults to the ring (one block per SM
// whose groups share a ring of buffers refilled as soon as a tile is stored:
// the load latency hides behind other tiles' stages).  Otherwise one buffer:
// load, compute and store a tile, with several blocks per SM; two only when
// the caller asks for them and one block's shared memory holds them.
enum { TB_ONE = 1, TB_TWO = 2, TB_RING = 3, TB_RING_TMAW = 4 };

// Default ring flavour (set by measurement on the 26-qubit ansatz): with the
// TMA warpgroup both ways.
static int ring_default(bool) { return TB_RING_TMAW; }

template <typename V, bool ADJ>
static uint32_t max_smem_ring(const tqd_circuit *c, int dt) {
    uint32_t m = 0;
    for (const auto &p : c->tile_passes) {
        const TileSmem s = tile_smem_ring<V, ADJ, RingCfg<ADJ>::B>(p.dev[dt].h);
        if (s.total > m) m = s.total;
    }
    return m;
}

// Static shared memory of the ring body (descriptor head, barriers, counters).
template <bool ADJ> static constexpr uint32_t ring_static_smem() {
    return (uint32_t)(sizeof(TileHead) + RingCfg<ADJ>::B * (8 + 8 + 4) + RingCfg<ADJ>::G * 2 * 4 + 256);
}

template <typename V, bool ADJ>
static int buffers_for(const tqd_circuit *c, int dt) {
    const uint32_t want = c->opts.buffers;
    // the ring pays off once every block has several tiles (n >= 21: >= 1.7 per group)
    if (sizeof(V) == 8 && (want >= TB_RING || (want == 0 && c->n >= 21)) &&
        max_smem_ring<V, ADJ>(c, dt) + ring_static_smem<ADJ>() <= (uint32_t)smem_optin_limit())
        return want >= TB_RING ? (int)want : ring_default(ADJ);
    if (want != TB_TWO) return TB_ONE;
    return (int)max_smem<V, ADJ, 2>(c, dt) <= smem_optin_limit() ? TB_TWO : TB_ONE;
}

template <typename V, bool ADJ, int NB>
static int grid_nb(const tqd_circuit *c, int dt) {
    const uint64_t tiles = (uint64_t)1 << (c->n - TILE_K);
    const int nb = occupancy_for<V, ADJ, NB>(max_smem<V, ADJ, NB>(c, dt));
    uint64_t g = (uint64_t)device_sm_count() * nb;
    if (g > tiles) g = tiles;
    if (g > (uint64_t)c->pblk) g = c->pblk;
    if (c->opts.max_blocks && g > c->opts.max_blocks) g = c->opts.max_blocks;
    return (int)g;
}

// Ring: one block per SM.
static int grid_ring(const tqd_circuit *c) {
    const uint64_t tiles = (uint64_t)1 << (c->n - TILE_K);
    uint64_t g = (uint64_t)device_sm_count();
    if (g > tiles) g = tiles;
    if (g > (uint64_t)c->pblk) g = c->pblk;
    if (c->opts.max_blocks && g > c->opts.max_blocks) g = c->opts.max_blocks;
    return (int)g;
}

template <typename V, bool ADJ>
static int grid_for(const tqd_circuit *c, int dt) {
    switch (buffers_for<V, ADJ>(c, dt)) {
    case TB_RING: case TB_RING_TMAW: return grid_ring(c);
    case TB_TWO: return grid_nb<V, ADJ, 2>(c, dt);
    default: return grid_nb<V, ADJ, 1>(c, dt);
    }
}

int tile_grid(const tqd_circuit *c, int dt, bool adj) {
    if (dt == 0) return adj ? grid_for<float2, true>(c, 0) : grid_for<float2, false>(c, 0);
    return adj ? grid_for<double2, true>(c, 1) : grid_for<double2, false>(c, 1);
}

// Bytes a pass moves: psi read and written; in the reverse sweep lambda too,
// and psi only read when it comes from a forward checkpoint.
template <typename V, bool ADJ>
static double pass_bytes(const tqd_circuit *c, int flags) {
    const double state = (double)((uint64_t)1 << c->n) * sizeof(V);
    return state * (ADJ ? ((flags & TILE_PSI_RO) ? 3.0 : 4.0) : 2.0);
}

template <typename V, bool ADJ, int NB>
static cudaError_t launch_nb(const CUtensorMap &ma, const CUtensorMap &mb, const tqd_circuit *c, int pass,
                             int flags, cudaStream_t s) {
    const int dt = sizeof(V) == 8 ? 0 : 1;
    const TilePlanPass &pp = c->tile_passes[pass];
    const TileSmem sm = tile_smem<V, ADJ, NB>(pp.dev[dt].h);
    const int grid = grid_nb<V, ADJ, NB>(c, dt);
    ProfScope ps(ADJ ? PK_TILE_ADJ : PK_TILE_FWD, pass_bytes<V, ADJ>(c, flags), s);
    const RT<V> *mats = dt == 0 ? (const RT<V> *)c->d_mats32 : (const RT<V> *)c->d_mats64;
    k_tile<V, ADJ, NB><<<grid, TILE_THREADS, sm.total, s>>>(ma, mb, c->d_tile_desc + 2 * pass + dt, mats,
                                                            c->d_partials, c->pblk, c->d_err, flags);
    return cudaGetLastError();
}

// Registers per thread of the generic ring kernel with the TMA warpgroup.
template <typename V, bool ADJ>
static int ring_tmaw_regs() {
    if constexpr (sizeof(V) == 8) {
        static int regs = [] {
            cudaFuncAttributes a;
            return cudaFuncGetAttributes(&a, k_tile_ring<V, ADJ, true>) == cudaSuccess ? a.numRegs : -1;
        }();
        return regs;
    }
    return -1;
}

template <typename V, bool ADJ, bool TMAW>
static cudaError_t launch_ring_generic(const CUtensorMap &ma, const CUtensorMap &mb, const tqd_circuit *c, int pass,
                                       int flags, cudaStream_t s) {
    const int dt = sizeof(V) == 8 ? 0 : 1;
    static std::mutex mu;
    static uint32_t set_to = 0;
    const uint32_t need = max_smem_ring<V, ADJ>(c, dt);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (need > set_to) {
            cudaFuncSetAttribute(k_tile_ring<V, ADJ, TMAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            set_to = need;
        }
    }
    const TilePlanPass &pp = c->tile_passes[pass];
    const TileSmem sm = tile_smem_ring<V, ADJ, RingCfg<ADJ>::B>(pp.dev[dt].h);
    ProfScope ps(ADJ ? PK_TILE_ADJ : PK_TILE_FWD, pass_bytes<V, ADJ>(c, flags), s);
    const RT<V> *mats = dt == 0 ? (const RT<V> *)c->d_mats32 : (const RT<V> *)c->d_mats64;
    k_tile_ring<V, ADJ, TMAW><<<grid_ring(c), (TMAW ? RingCfg<ADJ>::THREADS_TMAW : RingCfg<ADJ>::THREADS), sm.total, s>>>(
        ma, mb, c->d_tile_desc + 2 * pass + dt, mats, c->d_partials, c->pblk, c->d_err, flags);
    return cudaGetLastError();
}

// Tensor maps: forward, ma = psi_src (loads) and mb = psi_dst (stores); the
// reverse sweep, ma = psi_src (loads, and stores unless TILE_PSI_RO) and mb
// = lambda.
template <typename V, bool ADJ>
static cudaError_t launch_t(const void *psi_src, void *psi_dst, tqd_state *lam, const tqd_circuit *c, int pass,
                            int flags, cudaStream_t s) {
    const int dt = sizeof(V) == 8 ? 0 : 1;
    const TilePlanPass &pp = c->tile_passes[pass];
    CUtensorMap ma, mb;
    cudaError_t e = tile_tensor_map(&ma, const_cast<void *>(psi_src), pp, dt);
    if (e != cudaSuccess) return e;
    if (ADJ) e = tile_tensor_map(&mb, lam->amps, pp, dt);
    else if (psi_dst != psi_src) e = tile_tensor_map(&mb, psi_dst, pp, dt);
    else mb = ma;
    if (e != cudaSuccess) return e;
    const int tb = buffers_for<V, ADJ>(c, dt);
    if (tb == TB_TWO) return launch_nb<V, ADJ, 2>(ma, mb, c, pass, flags, s);
    // the pass-specialised kernel when the circuit has one: same descriptor,
    // shared memory and grid as the generic kernel of the same kind
    const bool ring = tb == TB_RING || tb == TB_RING_TMAW, ro = (flags & TILE_PSI_RO) != 0;
    bool tmaw = tb == TB_RING_TMAW;
    CUfunction f = nullptr;
    e = jit_function(c, pass, dt, ADJ, ring, tmaw, ro, s, &f);
    if (e != cudaSuccess) return e;
    if (tmaw && (f ? jit_num_regs(f) : ring_tmaw_regs<V, ADJ>()) != RingCfg<ADJ>::REGS_LAUNCH) {
        // the TMA warpgroup's register shares add up only for a launch with
        // REGS_LAUNCH registers per thread: the ring without it instead
        tmaw = false;
        f = nullptr;
        e = jit_function(c, pass, dt, ADJ, ring, false, ro, s, &f);
        if (e != cudaSuccess) return e;
    }
    if (!f) {
        if constexpr (sizeof(V) == 8) {
            if (tmaw) return launch_ring_generic<V, ADJ, true>(ma, mb, c, pass, flags, s);
            if (ring) return launch_ring_generic<V, ADJ, false>(ma, mb, c, pass, flags, s);
        }
        return launch_nb<V, ADJ, 1>(ma, mb, c, pass, flags, s);
    }
    const TileSmem sm = ring ? tile_smem_ring<V, ADJ, RingCfg<ADJ>::B>(pp.dev[dt].h) : tile_smem<V, ADJ, 1>(pp.dev[dt].h);
    const int grid = ring ? grid_ring(c) : grid_nb<V, ADJ, 1>(c, dt);
    const int threads = ring ? (tmaw ? RingCfg<ADJ>::THREADS_TMAW : RingCfg<ADJ>::THREADS) : TILE_THREADS;
    ProfScope ps(ADJ ? PK_TILE_ADJ : PK_TILE_FWD, pass_bytes<V, ADJ>(c, flags), s);
    const void *mats = dt == 0 ? (const void *)c->d_mats32 : (const void *)c->d_mats64;
    return jit_launch(f, ma, mb, c->d_tile_desc + 2 * pass + dt, mats, c->d_partials, c->pblk, c->d_err, flags, grid,
                      threads, sm.total, s);
}

cudaError_t launch_tile_pass(tqd_state *psi, tqd_state *lam, const tqd_circuit *c, int pass, cudaStream_t s,
                             const void *psi_src, void *psi_dst) {
    const void *src = psi_src ? psi_src : psi->amps;
    void *dst = psi_dst ? psi_dst : psi->amps;
    // a reverse pass whose psi comes from elsewhere leaves it as it is
    const int flags = ((lam && psi_src) ? TILE_PSI_RO : 0) | (c->test_stall ? TILE_STALL_TEST : 0);
    if (psi->dtype == TQD_C64)
        return lam ? launch_t<float2, true>(src, dst, lam, c, pass, flags, s)
                   : launch_t<float2, false>(src, dst, lam, c, pass, flags, s);
    return lam ? launch_t<double2, true>(src, dst, lam, c, pass, flags, s)
               : launch_t<double2, false>(src, dst, lam, c, pass, flags, s);
}

}  // namespace tqd
