// kernels_tc.cu -- fused 6-qubit blocks on the tensor cores (complex64).
//
// All gates of a block act on qubits 0..5, so the block is one 64 x 64
// unitary U and the state, viewed as columns of 64 consecutive amplitudes,
// becomes Y = U X (the contraction M x_Q X of Algorithm 1 with |Q| = 6).  With
// interleaved (re, im) storage a column is 128 floats and the product is a
// real GEMM with the 128 x 128 embedding
//     U~[2r][2c] = Re U_rc   U~[2r][2c+1] = -Im U_rc
//     U~[2r+1][2c] = Im U_rc U~[2r+1][2c+1] = Re U_rc.
// tcgen05.mma (kind::tf32, M = 128, N = 64, K = 8 per instruction) takes U~
// from tensor memory (written there once per block) and a tile of 64 state
// columns from shared memory (K-major, 128-byte swizzle, loaded by TMA) and
// accumulates in TMEM.  TF32 keeps 10 mantissa
// bits, so both operands are split, a = a_hi + a_lo, and three products
// a_hi b_hi + a_hi b_lo + a_lo b_hi are accumulated in FP32 (split
// precision, about 21 bits per product).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "launch.h"
#include "prof.h"
#include "tc.h"

namespace tqd {

constexpr int TC_K = 128;                    // floats per column (64 complex amplitudes)
constexpr int TC_N = 64;                     // columns per tile
constexpr int TC_KB = TC_K / 32;             // 128-byte K blocks
constexpr int TC_B_BYTES = TC_N * TC_K * 4;  // 32 KiB
constexpr int TC_NB = 4;                     // state tile buffers (loads in flight)
constexpr int TC_NLO = 2;                    // lo-half buffers
// Tensor memory: the operand U~ as TF32 hi and lo halves (128 lanes = rows,
// one 32-bit column per K element), then two 64-column accumulators.
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint32_t TC_A_HI = 0, TC_A_LO = 128, TC_ACC = 256;
constexpr int TC_SMEM = (TC_NB + TC_NLO) * TC_B_BYTES + 1024 + 256;

__device__ __forceinline__ uint32_t tc_sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
// x rounded to the nearest TF32 value (10 stored mantissa bits; ties away from
// zero): half a TF32 unit in the last place added to the magnitude's bits,
// then the 13 low bits cleared.  The operand U~'s hi half uses it, so that its
// lo half has either sign and the split's error does not lean one way (the
// state's halves are split by truncation, as the tensor core reads a float).
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// ------------------------------------------------------------- block prep
// One block: thread c builds column c of U by applying the block's gates to
// e_c in FP64, then writes U~ row-major (row m, column k at m * 128 + k) as
// TF32 hi / lo halves.  adj: the embedding of U^dagger instead (the reverse
// sweep's x = U^dagger y, Sec. 4.4): row c of U^dagger is the conjugate of
// column c of U, so thread c writes rows 2c and 2c + 1.
__global__ void k_tc_prep(const TcGate *__restrict__ gates, int ng, const double *__restrict__ mats64,
                          float *__restrict__ a_hi, float *__restrict__ a_lo, int adj) {
    extern __shared__ double2 col[];  // [64 amplitudes][64 columns]: thread c owns column c
    const int c = threadIdx.x;        // 64 threads
#define V(r) col[(r) * 64 + c]
    for (int r = 0; r < 64; ++r) V(r) = make_double2(r == c ? 1.0 : 0.0, 0.0);
    for (int g = 0; g < ng; ++g) {
        const TcGate G = gates[g];
        const double *m = mats64 + (size_t)G.gate * MAT_STRIDE;
        if (G.nw == 1) {
            const M2<double2> M = load_m2<double2>(m);
            const int T = 1 << G.w0;
            for (int r = 0; r < 64; ++r) {
                if (r & T) continue;
                double2 x0 = V(r), x1 = V(r | T);
                mv2(M, x0, x1);
                V(r) = x0;
                V(r | T) = x1;
            }
        } else {
            const int W0 = 1 << G.w0, W1 = 1 << G.w1;
            for (int r = 0; r < 64; ++r) {
                if (r & (W0 | W1)) continue;
                const int idx[4] = {r, r | W1, r | W0, r | W0 | W1};
                double2 x[4], y[4];
                for (int l = 0; l < 4; ++l) x[l] = V(idx[l]);
                for (int i = 0; i < 4; ++i) {
                    double2 acc = make_double2(0.0, 0.0);
                    for (int j = 0; j < 4; ++j)
                        acc = cfma(make_double2(m[2 * (i * 4 + j)], m[2 * (i * 4 + j) + 1]), x[j], acc);
                    y[i] = acc;
                }
                for (int l = 0; l < 4; ++l) V(idx[l]) = y[l];
            }
        }
    }
    // U[r][c] = v[r]; the four real entries of each complex entry (of
    // U^dagger[c][r] = conj(v[r]) when adj)
    for (int r = 0; r < 64; ++r) {
        const double re = V(r).x, im = adj ? -V(r).y : V(r).y;
        const int i = adj ? c : r, j = adj ? r : c;  // the entry's row and column
        const double e[4] = {re, -im, im, re};  // (2i,2j) (2i,2j+1) (2i+1,2j) (2i+1,2j+1)
        const int rows[4] = {2 * i, 2 * i, 2 * i + 1, 2 * i + 1};
        const int ks[4] = {2 * j, 2 * j + 1, 2 * j, 2 * j + 1};
        for (int q = 0; q < 4; ++q) {
            const float hi = tf32_rn((float)e[q]);
            const float lo = (float)(e[q] - (double)hi);
            a_hi[rows[q] * TC_K + ks[q]] = hi;
            a_lo[rows[q] * TC_K + ks[q]] = lo;
        }
    }
#undef V
}

// ------------------------------------------------------------ TC apply
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);  // start address
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused with 128-byte swizzle, K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8-row atoms
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// Bounded wait for phase `parity` of `bar`: false once WAIT_LIMIT_NS of
// elapsed time passed without it.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity) {
    uint64_t t0 = 0;
    for (bool first = true;; first = false) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(tc_sptr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (first) t0 = gtimer_ns();
        else if (gtimer_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
}

// Warp-uniform bounded wait: lane 0 waits, the warp learns the outcome.
__device__ __forceinline__ bool tc_wait_warp(uint64_t *bar, uint32_t parity) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = tc_wait(bar, parity) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok && (threadIdx.x & 31) != 0) tc_wait(bar, parity);  // acquire the completed phase
    return ok != 0;
}

__device__ __forceinline__ void tc_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_sptr(bar)) : "memory");
}

// One block per SM over its tiles (blockIdx.x + k * gridDim.x).  U~ (hi and
// lo) sits in tensor memory for the whole kernel, which leaves the shared
// memory to four state-tile buffers and two lo-half buffers.  The warps have
// roles and meet only on mbarriers, never at a block barrier inside the loop:
//  - warp 13, lane 0 (loader): TMA loads of the state tiles, tile k into
//    buffer k % 4; tile k + 4 as soon as tile k's MMAs completed;
//  - warps 1..3 and 8..12 (split): the TF32 lo half of tile k into lo buffer
//    k % 2, once the tile has landed and tile k - 2's MMAs (which read that
//    lo buffer) completed; eight 16-byte values a thread;
//  - warp 0, lane 0 (MMA issuer): once tile k's lo half is written and its
//    accumulator (k % 2) has been read out, the 48 MMAs and their commits;
//  - warps 4..7 (epilogue, one per quarter of the TMEM lanes): tile k's result
//    from accumulator k % 2 to HBM once its MMAs completed, then release the
//    accumulator.
// Every wait is bounded in time; a role that gives up sets the error word and
// leaves, and the roles waiting on it then run out too.
constexpr int TC_THREADS = 448;
constexpr int TC_SPLIT_WARPS = 8;
constexpr int TC_SPLIT_THREADS = 32 * TC_SPLIT_WARPS;
constexpr int TC_SPLIT_PER = TC_B_BYTES / 16 / TC_SPLIT_THREADS;  // 16-byte values per split thread
constexpr int TC_EPI_THREADS = 128;
constexpr int TC_LOADER_WARP = 13;
static_assert(TC_SPLIT_PER * TC_SPLIT_THREADS * 16 == TC_B_BYTES, "split covers the tile");

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_apply(const __grid_constant__ CUtensorMap map, float *__restrict__ state, const float *__restrict__ a_hi,
               const float *__restrict__ a_lo, uint64_t n_tiles, int *__restrict__ err) {
    extern __shared__ unsigned char tc_raw[];
    const uint32_t pad = (1024u - (tc_sptr(tc_raw) & 1023u)) & 1023u;
    unsigned char *sm = tc_raw + pad;
    float *Bbuf = reinterpret_cast<float *>(sm);                          // TC_NB tiles
    float *Blo = reinterpret_cast<float *>(sm + TC_NB * TC_B_BYTES);      // TC_NLO tiles
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + (TC_NB + TC_NLO) * TC_B_BYTES);  // [TC_NB] tile landed
    uint64_t *lo_ready = full + TC_NB;      // [TC_NLO] lo half written (TC_SPLIT_THREADS arrivals)
    uint64_t *mma_done = lo_ready + TC_NLO; // [2] tile's MMAs completed, by accumulator
    uint64_t *epi_done = mma_done + 2;      // [2] accumulator read out (TC_EPI_THREADS arrivals)
    uint64_t *freeb = epi_done + 2;         // [TC_NB] tile's MMAs completed, by buffer
    uint64_t *drain = freeb + TC_NB;        // every MMA issued has completed
    uint32_t *slot = reinterpret_cast<uint32_t *>(drain + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < TC_NB; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_sptr(full + i)));
        for (int i = 0; i < TC_NLO; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_sptr(lo_ready + i)), "r"(TC_SPLIT_THREADS));
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_sptr(mma_done + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_sptr(epi_done + i)), "r"(TC_EPI_THREADS));
        }
        for (int i = 0; i < TC_NB; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_sptr(freeb + i)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_sptr(drain)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_sptr(slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *slot;
    // U~ into tensor memory: warp w < 8 writes rows 32 (w % 4) .. + 31 (its
    // lane quarter) of the hi half (w < 4) or the lo half, 32 columns at a time
    if (warp < 8) {
        const int q = warp & 3, h = warp >> 2;
        const float4 *src = reinterpret_cast<const float4 *>((h ? a_lo : a_hi) + (size_t)(32 * q + lane) * TC_K);
        for (int c = 0; c < TC_K / 32; ++c) {
            uint32_t r[32];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 v = src[c * 8 + j];
                r[4 * j] = __float_as_uint(v.x);
                r[4 * j + 1] = __float_as_uint(v.y);
                r[4 * j + 2] = __float_as_uint(v.z);
                r[4 * j + 3] = __float_as_uint(v.w);
            }
            const uint32_t ta = taddr + ((uint32_t)(32 * q) << 16) + (h ? TC_A_LO : TC_A_HI) + 32u * c;
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(ta),
                "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
                "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
                "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
                "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                : "memory");
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint64_t n_local = n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == TC_LOADER_WARP) {
        if (lane == 0) {
            // ---- loader
            const uint64_t m = reinterpret_cast<uint64_t>(&map);
            auto issue_load = [&](uint64_t k) {
                const int b = (int)(k % TC_NB);
                const uint64_t tile = blockIdx.x + k * gridDim.x;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_sptr(full + b)),
                             "r"((uint32_t)TC_B_BYTES)
                             : "memory");
                for (int kb = 0; kb < TC_KB; ++kb) {
                    const int c0 = kb * 32, c1 = (int)(tile * TC_N);
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                        "%3}], [%4];" ::"r"(tc_sptr(Bbuf + b * (TC_B_BYTES / 4)) + kb * TC_N * 128),
                        "l"(m), "r"(c0), "r"(c1), "r"(tc_sptr(full + b))
                        : "memory");
                }
            };
            uint64_t loads = 0;
            for (; loads < (uint64_t)TC_NB && loads < n_local; ++loads) issue_load(loads);
            for (uint64_t k = 0; loads < n_local; ++k) {
                // buffer k % TC_NB is free once tile k's MMAs completed; its
                // next phase needs the load issued here, so the wait cannot
                // fall a phase behind
                if (!tc_wait(freeb + (k % TC_NB), (uint32_t)(k / TC_NB) & 1u)) {
                    atomicExch(err, 1);
                    break;
                }
                issue_load(loads++);
            }
            // the copies still in flight land before the buffers go (at
            // most one per buffer; on success they all have already)
            for (uint64_t j = loads > (uint64_t)TC_NB ? loads - TC_NB : 0; j < loads; ++j)
                tc_wait(full + (j % TC_NB), (uint32_t)(j / TC_NB) & 1u);
        }
        __syncwarp();
    } else if (warp == 0) {
        if (lane == 0) {
            // ---- MMA issuer
            // instruction descriptor: D f32, A and B tf32, both K-major, N = 64, M = 128
            const uint32_t idesc =
                (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            bool failed = false;
            for (uint64_t k = 0; k < n_local; ++k) {
                const int d = (int)(k & 1), l = (int)(k % TC_NLO), b = (int)(k % TC_NB);
                // accumulator free, lo half ready (the split saw the tile land
                // before it wrote the lo half)
                if (k >= 2 && !tc_wait(epi_done + d, (uint32_t)((k - 2) >> 1) & 1u)) failed = true;
                if (!failed && !tc_wait(lo_ready + l, (uint32_t)(k / TC_NLO) & 1u)) failed = true;
                if (failed) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dcol = taddr + TC_ACC + (uint32_t)d * TC_N;
                const uint64_t dbhi = tc_desc(tc_sptr(Bbuf + b * (TC_B_BYTES / 4)));
                const uint64_t dblo = tc_desc(tc_sptr(Blo + l * (TC_B_BYTES / 4)));
#pragma unroll
                for (int p = 0; p < 3; ++p) {  // hi*hi, hi*lo, lo*hi
                    const uint32_t acol = taddr + (p == 2 ? TC_A_LO : TC_A_HI);
                    const uint64_t db = p == 1 ? dblo : dbhi;
#pragma unroll
                    for (int s = 0; s < TC_K / 8; ++s) {
                        const uint32_t a = acol + 8u * s;
                        const uint64_t bd = db + (uint64_t)(((s >> 2) * TC_N * 128 + (s & 3) * 32) >> 4);
                        const uint32_t acc = (p | s) != 0;
                        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, q;\n}" ::"r"(dcol),
                                     "r"(a), "l"(bd), "r"(idesc), "r"(acc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    tc_sptr(mma_done + d)));
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    tc_sptr(freeb + b)));
            }
            // every MMA issued ends before the tensor memory goes: one more
            // commit tracks them all
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tc_sptr(drain)));
            if (!tc_wait(drain, 0)) failed = true;
            if (failed) atomicExch(err, 1);
        }
        __syncwarp();
    } else if (warp < 4 || warp >= 8) {
        // ---- split
        const int st = (warp < 4 ? warp - 1 : warp - 5) * 32 + lane;
        for (uint64_t k = 0; k < n_local; ++k) {
            const int b = (int)(k % TC_NB), l = (int)(k % TC_NLO);
            if (!tc_wait_warp(full + b, (uint32_t)(k / TC_NB) & 1u)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            if (k >= 2 && !tc_wait_warp(mma_done + (k & 1), (uint32_t)((k - 2) >> 1) & 1u)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            const float4 *B = reinterpret_cast<const float4 *>(Bbuf + b * (TC_B_BYTES / 4));
            float4 *L = reinterpret_cast<float4 *>(Blo + l * (TC_B_BYTES / 4));
            float4 x[TC_SPLIT_PER];
#pragma unroll
            for (int j = 0; j < TC_SPLIT_PER; ++j) x[j] = B[st + j * TC_SPLIT_THREADS];
#pragma unroll
            for (int j = 0; j < TC_SPLIT_PER; ++j)
                L[st + j * TC_SPLIT_THREADS] = make_float4(x[j].x - tf32_hi(x[j].x), x[j].y - tf32_hi(x[j].y),
                                                           x[j].z - tf32_hi(x[j].z), x[j].w - tf32_hi(x[j].w));
            // the MMAs (async proxy) read what was written here
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_arrive(lo_ready + l);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (the
        // floats of a column), all 64 columns, 32 at a time
        const int q = warp & 3;
        for (uint64_t k = 0; k < n_local; ++k) {
            const int d = (int)(k & 1);
            if (!tc_wait_warp(mma_done + d, (uint32_t)(k >> 1) & 1u)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t tile = blockIdx.x + k * gridDim.x;
            float *out = state + tile * TC_N * TC_K;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint32_t r[32];
                const uint32_t ta = taddr + TC_ACC + (uint32_t)d * TC_N + ((uint32_t)(q * 32) << 16) + c * 32;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < 32; ++j) out[(c * 32 + j) * TC_K + q * 32 + lane] = __uint_as_float(r[j]);
            }
            // the accumulator's reads are done: the producer may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;");
            tc_arrive(epi_done + d);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_TMEM_COLS));
}

// ------------------------------------------------------------------- host
static cudaError_t tc_apply_state(tqd_state *psi, const tqd_circuit *c, const TcBlock &blk, cudaStream_t s);

static PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn() {
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

cudaError_t launch_tc_block(tqd_state *psi, const tqd_circuit *c, const TcBlock &blk, cudaStream_t s, bool adj,
                            tqd_state *second) {
    if (psi->dtype != TQD_C64 || psi->n < 6) return cudaErrorInvalidValue;
    if (second && (second->dtype != TQD_C64 || second->n != psi->n)) return cudaErrorInvalidValue;
    cudaError_t e;
    static std::once_flag prep_once;
    std::call_once(prep_once, [] {
        cudaFuncSetAttribute(k_tc_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * (int)sizeof(double2));
    });
    {
        ProfScope ps(PK_PREP, 0.0, s);
        k_tc_prep<<<1, 64, 64 * 64 * sizeof(double2), s>>>(blk.d_gates, blk.n_gates, c->d_mats64, blk.d_ahi, blk.d_alo,
                                                           adj ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    e = tc_apply_state(psi, c, blk, s);
    if (e == cudaSuccess && second) e = tc_apply_state(second, c, blk, s);
    return e;
}

// U~ (as last prepared) applied to every 64-amplitude column of one state.
static cudaError_t tc_apply_state(tqd_state *psi, const tqd_circuit *c, const TcBlock &blk, cudaStream_t s) {
    auto fn = tc_encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const uint64_t cols = ((uint64_t)1 << psi->n) / 64;
    CUtensorMap map;
    cuuint64_t gdim[2] = {(cuuint64_t)TC_K, (cuuint64_t)cols};
    cuuint64_t gstride[1] = {(cuuint64_t)TC_K * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)TC_N};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, psi->amps, gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int smem = TC_SMEM;
    static std::once_flag once;
    std::call_once(once, [&] { cudaFuncSetAttribute(k_tc_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); });
    const uint64_t tiles = cols / TC_N;
    uint64_t grid = (uint64_t)device_sm_count();
    if (grid > tiles) grid = tiles;
    if (c->opts.max_blocks && grid > c->opts.max_blocks) grid = c->opts.max_blocks;
    ProfScope ps(PK_TC_BLOCK, (double)((uint64_t)8 << psi->n) * 2.0, s);
    k_tc_apply<<<(int)grid, TC_THREADS, smem, s>>>(map, (float *)psi->amps, blk.d_ahi, blk.d_alo, tiles, c->d_err);
    return cudaGetLastError();
}

}  // namespace tqd
