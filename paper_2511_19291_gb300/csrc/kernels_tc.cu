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
// and a tile of 64 state columns from shared memory (K-major, 128-byte
// swizzle, loaded by TMA) and accumulates in TMEM.  TF32 keeps 10 mantissa
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

constexpr int TC_K = 128;                  // floats per column (64 complex amplitudes)
constexpr int TC_N = 64;                   // columns per tile
constexpr int TC_KB = TC_K / 32;           // 128-byte K blocks
constexpr int TC_A_BYTES = 128 * TC_K * 4; // 64 KiB
constexpr int TC_B_BYTES = TC_N * TC_K * 4;  // 32 KiB
constexpr int TC_THREADS = 256;

// Byte offset of element (row, k) of a K-major operand with `rows` rows:
// K blocks of 128 bytes, 8-row swizzle atoms of 1024 bytes, 16-byte chunk
// index XORed with the row inside the atom.
__host__ __device__ inline uint32_t tc_off(int row, int k, int rows) {
    const int kb = k >> 5, kk = k & 31;
    const int chunk = kk >> 2, within = (kk & 3) * 4;
    return (uint32_t)(kb * rows * 128 + (row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4) + within);
}

__device__ __forceinline__ uint32_t tc_sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// ------------------------------------------------------------- block prep
// One block: thread c builds column c of U by applying the block's gates to
// e_c in FP64, then writes U~ as TF32 hi / lo halves in the operand layout.
__global__ void k_tc_prep(const TcGate *__restrict__ gates, int ng, const double *__restrict__ mats64,
                          float *__restrict__ a_hi, float *__restrict__ a_lo) {
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
    // U[r][c] = v[r]; write the four real entries of each complex entry
    for (int r = 0; r < 64; ++r) {
        const double re = V(r).x, im = V(r).y;
        const double e[4] = {re, -im, im, re};  // (2r,2c) (2r,2c+1) (2r+1,2c) (2r+1,2c+1)
        const int rows[4] = {2 * r, 2 * r, 2 * r + 1, 2 * r + 1};
        const int ks[4] = {2 * c, 2 * c + 1, 2 * c, 2 * c + 1};
        for (int q = 0; q < 4; ++q) {
            const float hi = tf32_hi((float)e[q]);
            const float lo = (float)(e[q] - (double)hi);
            const uint32_t o = tc_off(rows[q], ks[q], 128) / 4;
            a_hi[o] = hi;
            a_lo[o] = lo;
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

// Pipelined over the block's tiles (one block per SM): two TMA buffers for
// the state tiles and two TMEM accumulators.  Iteration i: wait for tile i,
// split it (lo half into Blo), issue tile i's 48 MMAs into accumulator i % 2,
// write tile i - 1's result from the other accumulator to HBM while they
// run, wait for them, then refill tile i's buffer with tile i + 2.  So the
// MMAs of one tile overlap the previous tile's epilogue and the loads of the
// next two tiles.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_apply(const __grid_constant__ CUtensorMap map, float *__restrict__ state, const float *__restrict__ a_hi,
               const float *__restrict__ a_lo, uint64_t n_tiles, int *__restrict__ err) {
    extern __shared__ unsigned char tc_raw[];
    const uint32_t pad = (1024u - (tc_sptr(tc_raw) & 1023u)) & 1023u;
    unsigned char *sm = tc_raw + pad;
    float *Ahi = reinterpret_cast<float *>(sm);
    float *Alo = reinterpret_cast<float *>(sm + TC_A_BYTES);
    float *Bbuf = reinterpret_cast<float *>(sm + 2 * TC_A_BYTES);                  // 2 tiles
    float *Blo = reinterpret_cast<float *>(sm + 2 * TC_A_BYTES + 2 * TC_B_BYTES);  // 1 tile
    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sm + 2 * TC_A_BYTES + 3 * TC_B_BYTES);  // [2]
    uint64_t *bar_mma = bar_ld + 2;
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar_ld + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    {
        const uint4 *s0 = reinterpret_cast<const uint4 *>(a_hi), *s1 = reinterpret_cast<const uint4 *>(a_lo);
        uint4 *d0 = reinterpret_cast<uint4 *>(Ahi), *d1 = reinterpret_cast<uint4 *>(Alo);
        for (int i = tid; i < TC_A_BYTES / 16; i += TC_THREADS) {
            d0[i] = s0[i];
            d1[i] = s1[i];
        }
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_sptr(bar_ld)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_sptr(bar_ld + 1)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_sptr(bar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_sptr(slot)),
                     "r"(2 * TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = *slot;
    // instruction descriptor: D f32, A and B tf32, both K-major, N = 64, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    // this block's tiles: blockIdx.x + k * gridDim.x, k < n_local
    const uint64_t n_local = n_tiles > blockIdx.x ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto issue_load = [&](uint64_t k) {
        const int b = (int)(k & 1);
        const uint64_t tile = blockIdx.x + k * gridDim.x;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_sptr(bar_ld + b)),
                     "r"((uint32_t)TC_B_BYTES)
                     : "memory");
        const uint64_t m = reinterpret_cast<uint64_t>(&map);
        for (int kb = 0; kb < TC_KB; ++kb) {
            const int c0 = kb * 32, c1 = (int)(tile * TC_N);
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                ::"r"(tc_sptr(Bbuf + b * (TC_B_BYTES / 4)) + kb * TC_N * 128), "l"(m), "r"(c0), "r"(c1),
                "r"(tc_sptr(bar_ld + b))
                : "memory");
        }
    };
    // result of tile k (accumulator k % 2) to HBM: warp w reads TMEM lanes
    // 32 (w % 4) .. 32 (w % 4) + 31 (floats of a column) of columns
    // 32 (w / 4) .. 32 (w / 4) + 31
    auto epilogue = [&](uint64_t k) {
        const uint64_t tile = blockIdx.x + k * gridDim.x;
        float *out = state + tile * TC_N * TC_K;
        const uint32_t tcol = taddr + (uint32_t)(k & 1) * TC_N;
        const int q = warp & 3;
        {
            const int c = warp >> 2;
            uint32_t r[32];
            const uint32_t ta = tcol + ((uint32_t)(q * 32) << 16) + c * 32;
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
    };

    if (tid == 0) {
        if (n_local > 0) issue_load(0);
        if (n_local > 1) issue_load(1);
    }
    uint32_t ph_ld = 0, ph_mma = 0;  // bit b: phase parity of load barrier b
    bool failed = false;
    // Thread 0 waits (bounded) and the block learns the outcome at the
    // barrier, so every thread takes the same branch; the others then acquire
    // the completed phase themselves.
    // (one flag per barrier kind: a flag is rewritten only after two more
    // block barriers, so every thread has read it by then)
    __shared__ int s_ok[2];
    auto wait_all = [&](uint64_t *bar, uint32_t parity, int which) -> bool {
        if (tid == 0) s_ok[which] = tc_wait(bar, parity) ? 1 : 0;
        __syncthreads();
        const bool ok = s_ok[which] != 0;
        if (ok && tid != 0) tc_wait(bar, parity);
        return ok;
    };
    for (uint64_t k = 0; k < n_local; ++k) {
        const int b = (int)(k & 1);
        const float *B = Bbuf + b * (TC_B_BYTES / 4);
        if (!wait_all(bar_ld + b, (ph_ld >> b) & 1u, 0)) {
            failed = true;
            break;
        }
        ph_ld ^= 1u << b;
        // lo half of the state tile (same positions as B, 16 bytes at a
        // time); Blo is free: the previous tile's MMAs completed before the
        // last iteration ended
        for (int i = tid; i < TC_B_BYTES / 16; i += TC_THREADS) {
            const float4 x = reinterpret_cast<const float4 *>(B)[i];
            reinterpret_cast<float4 *>(Blo)[i] =
                make_float4(x.x - tf32_hi(x.x), x.y - tf32_hi(x.y), x.z - tf32_hi(x.z), x.w - tf32_hi(x.w));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t dcol = taddr + (uint32_t)b * TC_N;
            // operand descriptors: the start-address field (bits 0..13, in
            // 16-byte units) of each K step is the base plus a constant
            const uint64_t dahi = tc_desc(tc_sptr(Ahi)), dalo = tc_desc(tc_sptr(Alo));
            const uint64_t dbhi = tc_desc(tc_sptr(B)), dblo = tc_desc(tc_sptr(Blo));
#pragma unroll
            for (int p = 0; p < 3; ++p) {  // hi*hi, hi*lo, lo*hi
                const uint64_t da = p == 2 ? dalo : dahi;
                const uint64_t db = p == 1 ? dblo : dbhi;
#pragma unroll
                for (int s = 0; s < TC_K / 8; ++s) {
                    const uint64_t ad = da + (uint64_t)(((s >> 2) * 128 * 128 + (s & 3) * 32) >> 4);
                    const uint64_t bd = db + (uint64_t)(((s >> 2) * TC_N * 128 + (s & 3) * 32) >> 4);
                    const uint32_t acc = (p | s) != 0;
                    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}" ::"r"(dcol),
                                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tc_sptr(bar_mma)));
        }
        // the previous tile's result leaves while these MMAs run
        if (k > 0) epilogue(k - 1);
        if (!wait_all(bar_mma, ph_mma, 1)) {
            failed = true;
            break;
        }
        ph_mma ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // tile k's buffer (read by the MMAs just completed) takes tile k + 2
        if (tid == 0 && k + 2 < n_local) issue_load(k + 2);
    }
    if (!failed && n_local > 0) epilogue(n_local - 1);
    if (failed && tid == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(2 * TC_N));
}

// ------------------------------------------------------------------- host
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

cudaError_t launch_tc_block(tqd_state *psi, const tqd_circuit *c, const TcBlock &blk, cudaStream_t s) {
    if (psi->dtype != TQD_C64 || psi->n < 6) return cudaErrorInvalidValue;
    cudaError_t e;
    static std::once_flag prep_once;
    std::call_once(prep_once, [] {
        cudaFuncSetAttribute(k_tc_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 64 * (int)sizeof(double2));
    });
    {
        ProfScope ps(PK_PREP, 0.0, s);
        k_tc_prep<<<1, 64, 64 * 64 * sizeof(double2), s>>>(blk.d_gates, blk.n_gates, c->d_mats64, blk.d_ahi, blk.d_alo);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
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
    const int smem = 2 * TC_A_BYTES + 3 * TC_B_BYTES + 1024 + 64;
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
