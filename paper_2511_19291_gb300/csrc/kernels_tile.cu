// kernels_tile.cu -- the fused tile pass (forward and reverse sweep).
//
// One persistent block per tile slot: TMA (cp.async.bulk.tensor, 128-byte
// swizzle) brings the 2^12 amplitudes of a tile into shared memory; every
// stage then loads each thread's 16 amplitudes into registers in the stage's
// layout, applies the stage's gates there (Algorithm 1's contraction M x_Q X,
// with Q mapped onto register bits), and writes them back; a TMA store
// returns the tile to HBM.  The reverse sweep (Sec. 4.4: recompute the input
// of every gate as x = U^dagger y instead of storing it) does the same over
// psi and lambda, walking stages and gates backwards; before un-applying a
// parametric gate it reduces that gate's angle derivative
//   dE/dt = 2 Re <lambda| dG/dt |psi_before>
// (Im<lambda|P|psi> for R_P(t) = exp(-i t P/2), -2 Im<lambda|Pi|psi> for the
// phase gates) over the tile.
//
// Every wait is bounded: a TMA load that does not complete sets the error
// word and the block returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "launch.h"
#include "prof.h"
#include "tile.h"
#include "tile_plan.h"

namespace tqd {

template <typename V> using RT = typename Real<V>::T;
constexpr int NR = 1 << TILE_R;

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sptr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(sptr(bar)), "r"(parity)
        : "memory");
    return ok;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tma_load(int rank, const CUtensorMap *map, uint32_t dst, uint64_t *bar, const int *c) {
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    const uint32_t b = sptr(bar);
    switch (rank) {
    case 2:
        asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                     ::"r"(dst), "l"(m), "r"(c[0]), "r"(c[1]), "r"(b) : "memory");
        break;
    case 3:
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                     ::"r"(dst), "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(b) : "memory");
        break;
    case 4:
        asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
                     ::"r"(dst), "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(b) : "memory");
        break;
    default:
        asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                     ::"r"(dst), "l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(b) : "memory");
        break;
    }
}

__device__ __forceinline__ void tma_store(int rank, const CUtensorMap *map, uint32_t src, const int *c) {
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    switch (rank) {
    case 2:
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                     ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(src) : "memory");
        break;
    case 3:
        asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                     ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(src) : "memory");
        break;
    case 4:
        asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
                     ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(src) : "memory");
        break;
    default:
        asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];"
                     ::"l"(m), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(src) : "memory");
        break;
    }
}

// 128-byte swizzle of the TMA box, in amplitude units: the 16-byte chunk index
// inside a 128-byte row is XORed with the row index modulo 8.
template <typename V> __device__ __forceinline__ uint32_t swz(uint32_t l) {
    if constexpr (sizeof(V) == 8) return l ^ (((l >> 4) & 7u) << 1);
    else return l ^ ((l >> 3) & 7u);
}

// ----------------------------------------------------- register operations
template <int P> using IC = std::integral_constant<int, P>;

template <typename F> __device__ __forceinline__ void with_pos(int p, F &&f) {
    switch (p) {
    case 0: f(IC<0>{}); break;
    case 1: f(IC<1>{}); break;
    case 2: f(IC<2>{}); break;
    default: f(IC<3>{}); break;
    }
}
template <typename F> __device__ __forceinline__ void with_pos2(int p, int q, F &&f) {
    with_pos(p, [&](auto P_) { with_pos(q, [&](auto Q_) { f(P_, Q_); }); });
}

template <int P, typename V> __device__ __forceinline__ void rg1(V (&a)[NR], const M2<V> &m) {
#pragma unroll
    for (int j = 0; j < NR; ++j)
        if (!(j & (1 << P))) mv2(m, a[j], a[j | (1 << P)]);
}
template <int P, typename V> __device__ __forceinline__ void rd1(V (&a)[NR], V d0, V d1) {
#pragma unroll
    for (int j = 0; j < NR; ++j) a[j] = cmul(a[j], (j & (1 << P)) ? d1 : d0);
}
template <int P, typename V> __device__ __forceinline__ void rph(V (&a)[NR], V ph) {
#pragma unroll
    for (int j = 0; j < NR; ++j)
        if (j & (1 << P)) a[j] = cmul(a[j], ph);
}
template <int T, typename V> __device__ __forceinline__ void rx(V (&a)[NR]) {
#pragma unroll
    for (int j = 0; j < NR; ++j)
        if (!(j & (1 << T))) {
            V t = a[j];
            a[j] = a[j | (1 << T)];
            a[j | (1 << T)] = t;
        }
}
template <int C, int T, typename V> __device__ __forceinline__ void rcx(V (&a)[NR]) {
    if constexpr (C != T) {
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if ((j & (1 << C)) && !(j & (1 << T))) {
                V t = a[j];
                a[j] = a[j | (1 << T)];
                a[j | (1 << T)] = t;
            }
    }
}
template <int P, int Q, typename V> __device__ __forceinline__ void rsw(V (&a)[NR]) {
    if constexpr (P != Q) {
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if ((j & (1 << P)) && !(j & (1 << Q))) {
                const int k = (j ^ (1 << P)) | (1 << Q);
                V t = a[j];
                a[j] = a[k];
                a[k] = t;
            }
    }
}
template <int P, int Q, typename V> __device__ __forceinline__ void rd2(V (&a)[NR], V ph) {
    if constexpr (P != Q) {
#pragma unroll
        for (int j = 0; j < NR; ++j)
            if ((j & (1 << P)) && (j & (1 << Q))) a[j] = cmul(a[j], ph);
    }
}
// 4x4 with wires[0] on register position P (most significant local index bit).
template <int P, int Q, typename V> __device__ __forceinline__ void rg2(V (&a)[NR], const V (&m)[16]) {
    if constexpr (P != Q) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if ((j & (1 << P)) || (j & (1 << Q))) continue;
            const int i0 = j, i1 = j | (1 << Q), i2 = j | (1 << P), i3 = j | (1 << P) | (1 << Q);
            const V v0 = a[i0], v1 = a[i1], v2 = a[i2], v3 = a[i3];
            a[i0] = cfma(m[0], v0, cfma(m[1], v1, cfma(m[2], v2, cmul(m[3], v3))));
            a[i1] = cfma(m[4], v0, cfma(m[5], v1, cfma(m[6], v2, cmul(m[7], v3))));
            a[i2] = cfma(m[8], v0, cfma(m[9], v1, cfma(m[10], v2, cmul(m[11], v3))));
            a[i3] = cfma(m[12], v0, cfma(m[13], v1, cfma(m[14], v2, cmul(m[15], v3))));
        }
    }
}

template <typename V> __device__ __forceinline__ V pool_c(const RT<V> *pool, int off) {
    return mkc<V>(pool[off], pool[off + 1]);
}

template <int P, typename V> __device__ __forceinline__ void rg1r(V (&a)[NR], RT<V> m00, RT<V> m01, RT<V> m10,
                                                                 RT<V> m11) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        if (j & (1 << P)) continue;
        const V x0 = a[j], x1 = a[j | (1 << P)];
        a[j] = mkc<V>(fma(m00, x0.x, m01 * x1.x), fma(m00, x0.y, m01 * x1.y));
        a[j | (1 << P)] = mkc<V>(fma(m10, x0.x, m11 * x1.x), fma(m10, x0.y, m11 * x1.y));
    }
}

template <typename V, bool DAG>
__device__ __forceinline__ void apply_op_rest(const TileOp &op, V (&a)[NR], const RT<V> *pool, uint32_t tid);

// Per-thread factor of a diagonal run: the product of its gates whose
// positions are all thread bits.  *any tells whether there is one.
template <typename V>
__device__ __forceinline__ V dg_thread_factor(const TileOp &op, const TileSub *subs, const RT<V> *pool, uint32_t tid,
                                              bool &any) {
    V f = mkc<V>(1, 0);
    any = false;
    for (int i = op.sub0; i < op.sub0 + op.nsub; ++i) {
        const TileSub sb = subs[i];
        if (!(sb.a & 0x80)) continue;
        any = true;
        const int ba = (tid >> (sb.a & 0x7f)) & 1u;
        if (sb.type == TOP_D1) {
            f = cmul(f, pool_c<V>(pool, sb.moff + (ba ? 6 : 0)));
        } else if (ba && ((tid >> (sb.b & 0x7f)) & 1u)) {
            f = cmul(f, pool_c<V>(pool, sb.moff));
        }
    }
    return f;
}

// Apply one op (forward, or its inverse when DAG) to the 16 amplitudes of a,
// and of b too when TWO (the reverse sweep carries psi and lambda).
template <typename V, bool DAG, bool TWO>
__device__ __forceinline__ void apply_op(const TileOp &op, V (&a)[NR], V (&b)[NR], const RT<V> *pool, uint32_t tid,
                                         const TileSub *subs, const V *dgt) {
    switch (op.type) {
    case TOP_G1R: {
        RT<V> m00 = pool[op.moff], m01 = pool[op.moff + 2], m10 = pool[op.moff + 4], m11 = pool[op.moff + 6];
        if (DAG) { const RT<V> t = m01; m01 = m10; m10 = t; }
        with_pos(op.a, [&](auto P_) {
            rg1r<decltype(P_)::value>(a, m00, m01, m10, m11);
            if (TWO) rg1r<decltype(P_)::value>(b, m00, m01, m10, m11);
        });
        return;
    }
    case TOP_DG: {
        bool any;
        const V f = dg_thread_factor<V>(op, subs, pool, tid, any);
        const V *t = dgt + op.moff * NR;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            V ph = t[j];
            if (any) ph = cmul(ph, f);
            if (DAG) ph = conjv(ph);
            a[j] = cmul(a[j], ph);
            if (TWO) b[j] = cmul(b[j], ph);
        }
        return;
    }
    default:
        break;
    }
    apply_op_rest<V, DAG>(op, a, pool, tid);
    if (TWO) apply_op_rest<V, DAG>(op, b, pool, tid);
}

// The remaining op types, one register array at a time.
template <typename V, bool DAG>
__device__ __forceinline__ void apply_op_rest(const TileOp &op, V (&a)[NR], const RT<V> *pool, uint32_t tid) {
    switch (op.type) {
    case TOP_G1: {
        M2<V> m;
        m.a = pool_c<V>(pool, op.moff);
        m.b = pool_c<V>(pool, op.moff + 2);
        m.c = pool_c<V>(pool, op.moff + 4);
        m.d = pool_c<V>(pool, op.moff + 6);
        if (DAG) m = dagger2(m);
        with_pos(op.a, [&](auto P_) { rg1<decltype(P_)::value>(a, m); });
        break;
    }
    case TOP_D1: {
        V d0 = pool_c<V>(pool, op.moff), d1 = pool_c<V>(pool, op.moff + 6);
        if (DAG) { d0 = conjv(d0); d1 = conjv(d1); }
        if (op.a & 0x80) {
            const V d = ((tid >> (op.a & 0x7f)) & 1u) ? d1 : d0;
#pragma unroll
            for (int j = 0; j < NR; ++j) a[j] = cmul(a[j], d);
        } else {
            with_pos(op.a, [&](auto P_) { rd1<decltype(P_)::value>(a, d0, d1); });
        }
        break;
    }
    case TOP_CX:
        if (op.a & 0x80) {
            if ((tid >> (op.a & 0x7f)) & 1u) with_pos(op.b, [&](auto T_) { rx<decltype(T_)::value>(a); });
        } else {
            with_pos2(op.a, op.b, [&](auto C_, auto T_) { rcx<decltype(C_)::value, decltype(T_)::value>(a); });
        }
        break;
    case TOP_SW:
        with_pos2(op.a, op.b, [&](auto P_, auto Q_) { rsw<decltype(P_)::value, decltype(Q_)::value>(a); });
        break;
    case TOP_G2: {
        V m[16];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                m[r * 4 + c] = DAG ? conjv(pool_c<V>(pool, op.moff + 2 * (c * 4 + r)))
                                   : pool_c<V>(pool, op.moff + 2 * (r * 4 + c));
        with_pos2(op.a, op.b, [&](auto P_, auto Q_) { rg2<decltype(P_)::value, decltype(Q_)::value>(a, m); });
        break;
    }
    case TOP_D2: {
        V ph = pool_c<V>(pool, op.moff);
        if (DAG) ph = conjv(ph);
        const bool ta = op.a & 0x80, tb = op.b & 0x80;
        if (ta && tb) {
            if (((tid >> (op.a & 0x7f)) & 1u) && ((tid >> (op.b & 0x7f)) & 1u)) {
#pragma unroll
                for (int j = 0; j < NR; ++j) a[j] = cmul(a[j], ph);
            }
        } else if (ta) {
            if ((tid >> (op.a & 0x7f)) & 1u) with_pos(op.b, [&](auto P_) { rph<decltype(P_)::value>(a, ph); });
        } else if (tb) {
            if ((tid >> (op.b & 0x7f)) & 1u) with_pos(op.a, [&](auto P_) { rph<decltype(P_)::value>(a, ph); });
        } else {
            with_pos2(op.a, op.b, [&](auto P_, auto Q_) { rd2<decltype(P_)::value, decltype(Q_)::value>(a, ph); });
        }
        break;
    }
    default:
        break;
    }
}

// Angle derivative of one parametric op from the states after it (a = psi,
// b = lambda): this thread's share.
template <int P, typename V>
__device__ __forceinline__ RT<V> grad_g1(int gen, const V (&a)[NR], const V (&b)[NR]) {
    RT<V> s = 0;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        if (j & (1 << P)) continue;
        const V p0 = a[j], p1 = a[j | (1 << P)], l0 = b[j], l1 = b[j | (1 << P)];
        if (gen == GEN_X) s += im_cdot(l0, p1) + im_cdot(l1, p0);
        else s += re_cdot(l1, p0) - re_cdot(l0, p1);  // GEN_Y
    }
    return s;
}

// Share of one diagonal gate's derivative given w_j = Im(conj(lambda_j) psi_j)
// (unchanged by diagonal gates, so one w serves a whole run).
template <typename V>
__device__ __forceinline__ RT<V> grad_diag(uint8_t type, uint8_t pa, uint8_t pb, uint8_t gen, const RT<V> (&w)[NR],
                                           uint32_t tid) {
    using T = RT<V>;
    T s = 0;
    auto bit_of = [&](uint8_t pos, int j) -> int {
        return (pos & 0x80) ? (int)((tid >> (pos & 0x7f)) & 1u) : ((j >> pos) & 1);
    };
    if (type == TOP_D1) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const int bit = bit_of(pa, j);
            if (gen == GEN_Z) s += bit ? -w[j] : w[j];
            else if (bit) s += w[j];  // GEN_P1
        }
        return gen == GEN_P1 ? T(-2) * s : s;
    }
#pragma unroll
    for (int j = 0; j < NR; ++j)
        if (bit_of(pa, j) && bit_of(pb, j)) s += w[j];
    return T(-2) * s;
}

template <typename V>
__device__ __forceinline__ RT<V> grad_op(const TileOp &op, const V (&a)[NR], const V (&b)[NR], uint32_t tid) {
    using T = RT<V>;
    T s = 0;
    if (op.type == TOP_G1 || op.type == TOP_G1R) {
        with_pos(op.a, [&](auto P_) { s = grad_g1<decltype(P_)::value>(op.gen, a, b); });
        return s;
    }
    // diagonal generators: sum of Im(conj(lambda) psi) over the selected amplitudes
    T w[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) w[j] = im_cdot(b[j], a[j]);
    return grad_diag<V>(op.type, op.a, op.b, op.gen, w, tid);
}

template <typename T> __device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Matrix scalars copied into the pool for an op: (source offset, length).
__device__ __forceinline__ void op_pool_span(uint8_t type, int &src, int &len) {
    switch (type) {
    case TOP_G1: case TOP_G1R: case TOP_D1: src = 0; len = 8; break;
    case TOP_G2: src = 0; len = 32; break;
    case TOP_D2: src = 30; len = 2; break;
    default: src = 0; len = 0; break;
    }
}

struct TileSmem {
    uint32_t tiles, pool, gacc, dgt, tbt, stages, ops, subs, total;
};

template <typename V, bool ADJ>
__host__ __device__ inline TileSmem tile_smem(const TileHead &h) {
    const int pool_len = h.pool_len, n_grad = h.n_grad, n_dg = h.n_dg, n_stages = h.n_stages;
    TileSmem s;
    s.tiles = (ADJ ? 2u : 1u) * (1u << TILE_K) * (uint32_t)sizeof(V);
    s.pool = (uint32_t)((pool_len * sizeof(RT<V>) + 15) & ~15u);
    s.gacc = ADJ ? (uint32_t)(n_grad * TILE_THREADS * sizeof(RT<V>)) : 0u;
    s.gacc = (s.gacc + 15) & ~15u;
    s.dgt = (uint32_t)(n_dg * NR * sizeof(V));
    s.tbt = (uint32_t)((n_stages * TILE_TB * sizeof(uint16_t) + 15) & ~15u);
    s.stages = (uint32_t)(n_stages * sizeof(TileStage));
    s.ops = (uint32_t)((h.n_ops * sizeof(TileOp) + 15) & ~15u);
    s.subs = (uint32_t)((h.n_subs * sizeof(TileSub) + 15) & ~15u);
    s.total = 1024 + s.tiles + s.pool + s.gacc + s.dgt + s.tbt + s.stages + s.ops + s.subs + 16;
    return s;
}

// Bounds checks of the shared-memory indices, compiled in with TQD_CHECKED:
// a bad index is recorded in the error word (code 2) and the access skipped.
#ifdef TQD_CHECKED
#define TQD_IDX_OK(idx, lim) ((idx) < (lim) ? true : (atomicCAS(err, 0, 2), false))
#else
#define TQD_IDX_OK(idx, lim) true
#endif

// Copy `bytes` (a multiple of 4) from global to shared memory.
__device__ __forceinline__ void copy_words(void *dst, const void *src, uint32_t bytes) {
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = s[i];
}

template <typename V, bool ADJ>
__global__ void __launch_bounds__(TILE_THREADS, sizeof(V) == 8 ? (ADJ ? 2 : 3) : 1)
    k_tile(const __grid_constant__ CUtensorMap map_psi, const __grid_constant__ CUtensorMap map_lam,
           const TilePassDev *__restrict__ Pg, const RT<V> *__restrict__ mats, double *__restrict__ partials,
           int pblk, int *__restrict__ err) {
    using T = RT<V>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ TileHead P;
    copy_words(&P, &Pg->h, sizeof(TileHead));
    __syncthreads();
    const uint32_t pad = (1024u - (sptr(smem_raw) & 1023u)) & 1023u;
    unsigned char *sm = smem_raw + pad;
    const TileSmem L = tile_smem<V, ADJ>(P);
    V *tile_a = reinterpret_cast<V *>(sm);
    V *tile_b = tile_a + (1 << TILE_K);
    T *pool = reinterpret_cast<T *>(sm + L.tiles);
    T *gacc = reinterpret_cast<T *>(sm + L.tiles + L.pool);  // [grad op][thread]
    V *dgt = reinterpret_cast<V *>(sm + L.tiles + L.pool + L.gacc);
    uint16_t *tbt = reinterpret_cast<uint16_t *>(sm + L.tiles + L.pool + L.gacc + L.dgt);
    TileStage *stages = reinterpret_cast<TileStage *>(sm + L.tiles + L.pool + L.gacc + L.dgt + L.tbt);
    TileOp *ops = reinterpret_cast<TileOp *>(sm + L.tiles + L.pool + L.gacc + L.dgt + L.tbt + L.stages);
    TileSub *subs = reinterpret_cast<TileSub *>(sm + L.tiles + L.pool + L.gacc + L.dgt + L.tbt + L.stages + L.ops);
    uint64_t *bar =
        reinterpret_cast<uint64_t *>(sm + L.tiles + L.pool + L.gacc + L.dgt + L.tbt + L.stages + L.ops + L.subs);
    const uint32_t tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int TBS = TILE_TB;
    constexpr int NW = TILE_THREADS / 32;

    copy_words(stages, Pg->stages, P.n_stages * sizeof(TileStage));
    copy_words(ops, Pg->ops, P.n_ops * sizeof(TileOp));
    copy_words(subs, Pg->subs, P.n_subs * sizeof(TileSub));
    __syncthreads();

    // matrices of every op and diagonal sub-op, per-stage lane/warp offsets
    for (int k = 0; k < P.n_ops; ++k) {
        const TileOp op = ops[k];
        if (op.moff < 0 || op.type == TOP_DG) continue;
        int src, len;
        op_pool_span(op.type, src, len);
        for (int i = tid; i < len; i += blockDim.x)
            if (TQD_IDX_OK((uint32_t)(op.moff + i), (uint32_t)P.pool_len))
                pool[op.moff + i] = mats[(size_t)Pg->op_gate[k] * MAT_STRIDE + src + i];
    }
    for (int k = 0; k < P.n_subs; ++k) {
        const TileSub sb = subs[k];
        const int src = sb.type == TOP_D1 ? 0 : 30, len = sb.type == TOP_D1 ? 8 : 2;
        for (int i = tid; i < len; i += blockDim.x)
            if (TQD_IDX_OK((uint32_t)(sb.moff + i), (uint32_t)P.pool_len))
                pool[sb.moff + i] = mats[(size_t)Pg->sub_gate[k] * MAT_STRIDE + src + i];
    }
    for (int i = tid; i < P.n_stages * TBS; i += blockDim.x) {
        const int st = i / TBS, e = i % TBS;
        const TileStage &S = stages[st];
        tbt[i] = e < 32 ? S.ld_lo[e] : e < 32 + NW ? S.ld_hi[e - 32] : e < 64 + NW ? S.st_lo[e - 32 - NW] : S.st_hi[e - 64 - NW];
    }
    if (ADJ) {
        for (int i = tid; i < P.n_grad * TILE_THREADS; i += blockDim.x) gacc[i] = T(0);
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    // phase tables of the diagonal runs: entry j = product of the run's gates
    // whose positions are all register bits, evaluated at register index j
    for (int i = tid; i < P.n_dg * NR; i += blockDim.x) {
        const int d = i / NR, j = i % NR;
        const TileOp op = ops[Pg->dg_op[d]];
        V t = mkc<V>(1, 0);
        for (int q = op.sub0; q < op.sub0 + op.nsub; ++q) {
            const TileSub sb = subs[q];
            if (sb.a & 0x80) continue;
            if (sb.type == TOP_D1) t = cmul(t, pool_c<V>(pool, sb.moff + (((j >> sb.a) & 1) ? 6 : 0)));
            else if (((j >> sb.a) & 1) && ((j >> sb.b) & 1)) t = cmul(t, pool_c<V>(pool, sb.moff));
        }
        dgt[i] = t;
    }
    __syncthreads();

    const uint32_t tile_bytes = (1u << TILE_K) * (uint32_t)sizeof(V);
    const uint32_t box_bytes = tile_bytes >> P.n_extra;
    const uint64_t n_tiles = (uint64_t)1 << P.n_tiles_log2;
    uint32_t phase = 0;

    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        uint64_t g0 = 0;
        if (tid == 0) {
            for (int i = 0; i < P.n_tiles_log2; ++i) g0 |= ((tile >> i) & 1ull) << P.out_bits[i];
            mbar_expect_tx(bar, tile_bytes * (ADJ ? 2u : 1u));
            for (int e = 0; e < (1 << P.n_extra); ++e) {
                uint64_t g = g0;
                for (int i = 0; i < P.n_extra; ++i) g |= (uint64_t)((e >> i) & 1) << P.extra_bits[i];
                int c[TILE_MAX_DIMS];
#pragma unroll
                for (int d = 0; d < TILE_MAX_DIMS; ++d)
                    c[d] = d < P.rank ? (int)((g >> P.dim_lo[d]) & ((1ull << P.dim_len[d]) - 1)) : 0;
                tma_load(P.rank, &map_psi, sptr(tile_a) + e * box_bytes, bar, c);
                if (ADJ) tma_load(P.rank, &map_lam, sptr(tile_b) + e * box_bytes, bar, c);
            }
        }
        {
            uint32_t it = 0;
            while (!mbar_try_wait(bar, phase)) {
                if (++it > (1u << 26)) {
                    if (lane == 0) atomicExch(err, 1);
                    return;
                }
            }
        }
        phase ^= 1u;

        for (int si = 0; si < P.n_stages; ++si) {
            const int s = ADJ ? P.n_stages - 1 - si : si;
            const TileStage &st = stages[s];
            // forward: load through F, store through G; reverse: the other way
            const uint16_t *tl = tbt + s * TBS;
            const uint32_t base_ld = ADJ ? (uint32_t)(tl[32 + NW + lane] ^ tl[64 + NW + warp]) : (uint32_t)(tl[lane] ^ tl[32 + warp]);
            const uint32_t base_st = ADJ ? (uint32_t)(tl[lane] ^ tl[32 + warp]) : (uint32_t)(tl[32 + NW + lane] ^ tl[64 + NW + warp]);
            const uint16_t *roff_ld = ADJ ? st.st_roff : st.ld_roff;
            const uint16_t *roff_st = ADJ ? st.ld_roff : st.st_roff;
            V a[NR];
            V b[NR];
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const uint32_t ad = base_ld ^ roff_ld[j];
                if (TQD_IDX_OK(ad, (uint32_t)(1 << TILE_K))) {
                    a[j] = tile_a[ad];
                    if constexpr (ADJ) b[j] = tile_b[ad];
                }
            }
            if constexpr (!ADJ) {
                for (int k = st.op_begin; k < st.op_end; ++k)
                    apply_op<V, false, false>(ops[k], a, b, pool, tid, subs, dgt);
            } else {
                for (int k = (int)st.op_end - 1; k >= (int)st.op_begin; --k) {
                    const TileOp op = ops[k];
                    if (op.type == TOP_DG) {
                        T w[NR];
#pragma unroll
                        for (int j = 0; j < NR; ++j) w[j] = im_cdot(b[j], a[j]);
                        for (int q = op.sub0; q < op.sub0 + op.nsub; ++q) {
                            const TileSub sb = subs[q];
                            if (sb.gslot < 0) continue;
                            gacc[sb.gslot * TILE_THREADS + tid] += grad_diag<V>(sb.type, sb.a, sb.b, sb.gen, w, tid);
                        }
                    } else if (op.gslot >= 0) {
                        gacc[op.gslot * TILE_THREADS + tid] += grad_op<V>(op, a, b, tid);
                    }
                    apply_op<V, true, true>(op, a, b, pool, tid, subs, dgt);
                }
            }
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const uint32_t ad = base_st ^ roff_st[j];
                if (TQD_IDX_OK(ad, (uint32_t)(1 << TILE_K))) {
                    tile_a[ad] = a[j];
                    if constexpr (ADJ) tile_b[ad] = b[j];
                }
            }
            __syncthreads();
        }

        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            for (int e = 0; e < (1 << P.n_extra); ++e) {
                uint64_t g = g0;
                for (int i = 0; i < P.n_extra; ++i) g |= (uint64_t)((e >> i) & 1) << P.extra_bits[i];
                int c[TILE_MAX_DIMS];
#pragma unroll
                for (int d = 0; d < TILE_MAX_DIMS; ++d)
                    c[d] = d < P.rank ? (int)((g >> P.dim_lo[d]) & ((1ull << P.dim_len[d]) - 1)) : 0;
                tma_store(P.rank, &map_psi, sptr(tile_a) + e * box_bytes, c);
                if (ADJ) tma_store(P.rank, &map_lam, sptr(tile_b) + e * box_bytes, c);
            }
            bulk_commit();
            bulk_wait_read0();
        }
        __syncthreads();
    }
    if (tid == 0) bulk_wait0();
    if constexpr (ADJ) {
        __syncthreads();
        // per-thread partial sums (state precision, about 16 amplitudes x
        // the block's tiles each) are added in FP64, one warp per gradient op
        for (int k = warp; k < P.n_grad; k += NW) {
            double t = 0;
            for (int i = lane; i < TILE_THREADS; i += 32) t += (double)gacc[k * TILE_THREADS + i];
            t = warp_sum(t);
            if (lane == 0) partials[(size_t)Pg->grad_gate_slot[k] * pblk + blockIdx.x] = t;
        }
    }
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

static cudaError_t make_map(CUtensorMap *map, void *base, const TilePlanPass &pp, int dt) {
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

template <typename V, bool ADJ>
static int occupancy_for(uint32_t smem) {
    static std::mutex mu;
    static uint32_t set_to = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (smem > set_to) {
            cudaFuncSetAttribute(k_tile<V, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            set_to = smem;
        }
    }
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tile<V, ADJ>, TILE_THREADS, smem);
    return nb > 0 ? nb : 1;
}

template <typename V, bool ADJ>
static uint32_t max_smem(const tqd_circuit *c, int dt) {
    uint32_t m = 0;
    for (const auto &p : c->tile_passes) {
        const TileSmem s = tile_smem<V, ADJ>(p.dev[dt].h);
        if (s.total > m) m = s.total;
    }
    return m;
}

template <typename V, bool ADJ>
static int grid_for(const tqd_circuit *c, int dt) {
    const uint64_t tiles = (uint64_t)1 << (c->n - TILE_K);
    const int nb = occupancy_for<V, ADJ>(max_smem<V, ADJ>(c, dt));
    uint64_t g = (uint64_t)device_sm_count() * nb;
    if (g > tiles) g = tiles;
    if (g > (uint64_t)c->pblk) g = c->pblk;
    return (int)g;
}

int tile_grid(const tqd_circuit *c, int dt, bool adj) {
    if (dt == 0) return adj ? grid_for<float2, true>(c, 0) : grid_for<float2, false>(c, 0);
    return adj ? grid_for<double2, true>(c, 1) : grid_for<double2, false>(c, 1);
}

template <typename V, bool ADJ>
static cudaError_t launch_t(tqd_state *psi, tqd_state *lam, const tqd_circuit *c, int pass, cudaStream_t s) {
    const int dt = sizeof(V) == 8 ? 0 : 1;
    const TilePlanPass &pp = c->tile_passes[pass];
    CUtensorMap ma, mb;
    cudaError_t e = make_map(&ma, psi->amps, pp, dt);
    if (e != cudaSuccess) return e;
    if (ADJ) {
        e = make_map(&mb, lam->amps, pp, dt);
        if (e != cudaSuccess) return e;
    } else {
        mb = ma;
    }
    const TileSmem sm = tile_smem<V, ADJ>(pp.dev[dt].h);
    const int grid = grid_for<V, ADJ>(c, dt);
    const double bytes = (double)((uint64_t)1 << c->n) * sizeof(V) * 2.0 * (ADJ ? 2.0 : 1.0);
    ProfScope ps(ADJ ? PK_TILE_ADJ : PK_TILE_FWD, bytes, s);
    const RT<V> *mats = dt == 0 ? (const RT<V> *)c->d_mats32 : (const RT<V> *)c->d_mats64;
    k_tile<V, ADJ><<<grid, TILE_THREADS, sm.total, s>>>(ma, mb, c->d_tile_desc + 2 * pass + dt, mats, c->d_partials,
                                                        c->pblk, c->d_err);
    return cudaGetLastError();
}

cudaError_t launch_tile_pass(tqd_state *psi, tqd_state *lam, const tqd_circuit *c, int pass, cudaStream_t s) {
    if (psi->dtype == TQD_C64)
        return lam ? launch_t<float2, true>(psi, lam, c, pass, s) : launch_t<float2, false>(psi, lam, c, pass, s);
    return lam ? launch_t<double2, true>(psi, lam, c, pass, s) : launch_t<double2, false>(psi, lam, c, pass, s);
}

}  // namespace tqd
