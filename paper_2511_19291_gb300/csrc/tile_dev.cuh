// tile_dev.cuh -- device code of the fused tile pass (forward and reverse
// sweep), shared by the generic pass kernel and by the pass-specialised
// kernels that are compiled at run time (the same text is handed to NVRTC).
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
// Gradient partials: inside one tile a thread sums its amplitudes' products
// and the warp adds its 32 shares in state precision; across tiles every
// partial is added in FP64 (one shared-memory column per warp and gradient op).
//
// Every wait is bounded in time (WAIT_LIMIT_NS on the global timer): a TMA
// load that does not complete sets the error word and the block returns once
// the copies it issued have landed (or their waits have run out too).
#pragma once

#include "tile_desc.h"  // first: it supplies the fixed-width integer types under NVRTC
#include "common.cuh"

namespace tqd {

template <typename V> using RT = typename Real<V>::T;
constexpr int NR = 1 << TILE_R;

#ifdef __CUDACC_RTC__
// the tensor map as a kernel parameter (CUtensorMap's size and alignment)
struct alignas(64) TmaDesc {
    unsigned long long w[16];
};
#endif

template <typename A, typename B> struct same_type { static constexpr bool value = false; };
template <typename A> struct same_type<A, A> { static constexpr bool value = true; };
template <int P> struct IC { static constexpr int value = P; };

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
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(sptr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(bar)) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tma_load(int rank, const void *map, uint32_t dst, uint64_t *bar, const int *c) {
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

__device__ __forceinline__ void tma_store(int rank, const void *map, uint32_t src, const int *c) {
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
// Runtime position -> compile-time position (the generic kernel's dispatch).
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
    if constexpr (same_type<V, float2>::value) {
        // same roundings as the scalar form: m01 * x1 rounded, then fused with m00 * x0
        const float2 M00 = make_float2(m00, m00), M01 = make_float2(m01, m01);
        const float2 M10 = make_float2(m10, m10), M11 = make_float2(m11, m11);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j & (1 << P)) continue;
            const float2 x0 = a[j], x1 = a[j | (1 << P)];
            a[j] = f2_fma(M00, x0, f2_mul(M01, x1));
            a[j | (1 << P)] = f2_fma(M10, x0, f2_mul(M11, x1));
        }
    } else {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j & (1 << P)) continue;
            const V x0 = a[j], x1 = a[j | (1 << P)];
            a[j] = mkc<V>(fma(m00, x0.x, m01 * x1.x), fma(m00, x0.y, m01 * x1.y));
            a[j | (1 << P)] = mkc<V>(fma(m10, x0.x, m11 * x1.x), fma(m10, x0.y, m11 * x1.y));
        }
    }
}


// --------------------------------------------------------------- the ops
// One op with its positions fixed at compile time, applied forward or (DAG)
// inverted, to a and, when TWO, to b as well (the reverse sweep carries psi
// and lambda).  m points at the op's scalars in the pool; `bit` is the value
// of the thread-index bit an op position names.
template <typename V, bool DAG, bool TWO, int P>
__device__ __forceinline__ void op_g1(V (&a)[NR], V (&b)[NR], const RT<V> *m) {
    M2<V> M;
    M.a = pool_c<V>(m, 0);
    M.b = pool_c<V>(m, 2);
    M.c = pool_c<V>(m, 4);
    M.d = pool_c<V>(m, 6);
    if (DAG) M = dagger2(M);
    rg1<P>(a, M);
    if (TWO) rg1<P>(b, M);
}
template <typename V, bool DAG, bool TWO, int P>
__device__ __forceinline__ void op_g1r(V (&a)[NR], V (&b)[NR], const RT<V> *m) {
    RT<V> m00 = m[0], m01 = m[2], m10 = m[4], m11 = m[6];
    if (DAG) {
        const RT<V> t = m01;
        m01 = m10;
        m10 = t;
    }
    rg1r<P>(a, m00, m01, m10, m11);
    if (TWO) rg1r<P>(b, m00, m01, m10, m11);
}
template <typename V, bool DAG, bool TWO, int P>
__device__ __forceinline__ void op_d1r(V (&a)[NR], V (&b)[NR], const RT<V> *m) {
    V d0 = pool_c<V>(m, 0), d1 = pool_c<V>(m, 6);
    if (DAG) {
        d0 = conjv(d0);
        d1 = conjv(d1);
    }
    rd1<P>(a, d0, d1);
    if (TWO) rd1<P>(b, d0, d1);
}
template <typename V, bool DAG, bool TWO>
__device__ __forceinline__ void op_d1t(V (&a)[NR], V (&b)[NR], const RT<V> *m, uint32_t bit) {
    V d = pool_c<V>(m, bit ? 6 : 0);
    if (DAG) d = conjv(d);
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        a[j] = cmul(a[j], d);
        if (TWO) b[j] = cmul(b[j], d);
    }
}
template <bool TWO, int C, int T, typename V> __device__ __forceinline__ void op_cxr(V (&a)[NR], V (&b)[NR]) {
    rcx<C, T>(a);
    if (TWO) rcx<C, T>(b);
}
template <bool TWO, int T, typename V> __device__ __forceinline__ void op_cxt(V (&a)[NR], V (&b)[NR], uint32_t bit) {
    if (bit) {
        rx<T>(a);
        if (TWO) rx<T>(b);
    }
}
template <bool TWO, int P, int Q, typename V> __device__ __forceinline__ void op_sw(V (&a)[NR], V (&b)[NR]) {
    rsw<P, Q>(a);
    if (TWO) rsw<P, Q>(b);
}
template <typename V, bool DAG, bool TWO, int P, int Q>
__device__ __forceinline__ void op_g2(V (&a)[NR], V (&b)[NR], const RT<V> *m) {
    V M[16];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            M[r * 4 + c] = DAG ? conjv(pool_c<V>(m, 2 * (c * 4 + r))) : pool_c<V>(m, 2 * (r * 4 + c));
    rg2<P, Q>(a, M);
    if (TWO) rg2<P, Q>(b, M);
}
// phase on |11> of two register positions
template <typename V, bool DAG, bool TWO, int P, int Q>
__device__ __forceinline__ void op_d2rr(V (&a)[NR], V (&b)[NR], const RT<V> *m) {
    V ph = pool_c<V>(m, 0);
    if (DAG) ph = conjv(ph);
    rd2<P, Q>(a, ph);
    if (TWO) rd2<P, Q>(b, ph);
}
// one position is a thread bit (value `bit`), the other register position Q
template <typename V, bool DAG, bool TWO, int Q>
__device__ __forceinline__ void op_d2tr(V (&a)[NR], V (&b)[NR], const RT<V> *m, uint32_t bit) {
    if (bit) {
        V ph = pool_c<V>(m, 0);
        if (DAG) ph = conjv(ph);
        rph<Q>(a, ph);
        if (TWO) rph<Q>(b, ph);
    }
}
// both positions are thread bits; `bit` = both set
template <typename V, bool DAG, bool TWO>
__device__ __forceinline__ void op_d2tt(V (&a)[NR], V (&b)[NR], const RT<V> *m, uint32_t bit) {
    if (bit) {
        V ph = pool_c<V>(m, 0);
        if (DAG) ph = conjv(ph);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            a[j] = cmul(a[j], ph);
            if (TWO) b[j] = cmul(b[j], ph);
        }
    }
}
// Diagonal run: entry j of the run's phase table t (its gates on register
// positions), times the thread's factor f (its gates on thread bits) when ANY.
template <typename V, bool DAG, bool TWO, bool ANY>
__device__ __forceinline__ void op_dg(V (&a)[NR], V (&b)[NR], const V *t, V f) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        V ph = t[j];
        if (ANY) ph = cmul(ph, f);
        if (DAG) ph = conjv(ph);
        a[j] = cmul(a[j], ph);
        if (TWO) b[j] = cmul(b[j], ph);
    }
}

__device__ __forceinline__ uint32_t tbit(uint32_t tid, uint8_t pos) { return (tid >> (pos & 0x7f)) & 1u; }

// Tile-bit positions (qubits outside the pass's set): the bit of the tile's
// global origin.
__device__ __forceinline__ bool is_tile_pos(uint8_t pos) { return (pos & 0xC0) == TILE_POS_TILE; }
__device__ __forceinline__ uint32_t tile_bit(uint64_t torig, uint8_t pos) {
    return (uint32_t)(torig >> (pos & 0x3f)) & 1u;
}

// Phase e on the |1> half of register position P (psi, and lambda when TWO).
template <typename V, bool DAG, bool TWO, int P>
__device__ __forceinline__ void op_ph(V (&a)[NR], V (&b)[NR], V e) {
    if (DAG) e = conjv(e);
    rph<P>(a, e);
    if (TWO) rph<P>(b, e);
}

// The gates of a diagonal run that have a tile bit, at the current tile:
// those on tile bits only, or on a tile bit and a thread bit, multiply this
// thread's factor f; those on a tile bit and register position r multiply
// e[r] (bit r of emask set).  Tile bits are in sub-op position a.
template <typename V>
__device__ __forceinline__ void dg_tile_part(const TileOp &op, const TileSub *subs, const RT<V> *pool, uint32_t tid,
                                             uint64_t torig, V &f, V (&e)[TILE_R], uint32_t &emask) {
    for (int i = op.sub0; i < op.sub0 + op.nsub; ++i) {
        const TileSub sb = subs[i];
        if (!is_tile_pos(sb.a)) continue;
        const uint32_t ta = tile_bit(torig, sb.a);
        if (sb.type == TOP_D1) {
            f = cmul(f, pool_c<V>(pool, sb.moff + (ta ? 6 : 0)));
        } else if (ta) {
            const V ph = pool_c<V>(pool, sb.moff);
            if (is_tile_pos(sb.b)) {
                if (tile_bit(torig, sb.b)) f = cmul(f, ph);
            } else if (sb.b & 0x80) {
                if (tbit(tid, sb.b)) f = cmul(f, ph);
            } else {
                e[sb.b] = (emask >> sb.b) & 1u ? cmul(e[sb.b], ph) : ph;
                emask |= 1u << sb.b;
            }
        }
    }
}

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
        const uint32_t ba = tbit(tid, sb.a);
        if (sb.type == TOP_D1) {
            f = cmul(f, pool_c<V>(pool, sb.moff + (ba ? 6 : 0)));
        } else if (ba && tbit(tid, sb.b)) {
            f = cmul(f, pool_c<V>(pool, sb.moff));
        }
    }
    return f;
}

// The generic kernel's op: positions read from the descriptor.
template <typename V, bool DAG, bool TWO>
__device__ __forceinline__ void apply_op(const TileOp &op, V (&a)[NR], V (&b)[NR], const RT<V> *pool, uint32_t tid,
                                         const TileSub *subs, const V *dgt, uint64_t torig) {
    const RT<V> *m = pool + op.moff;
    switch (op.type) {
    case TOP_G1R:
        with_pos(op.a, [&](auto P_) { op_g1r<V, DAG, TWO, decltype(P_)::value>(a, b, m); });
        break;
    case TOP_DG: {
        bool any;
        V f = dg_thread_factor<V>(op, subs, pool, tid, any);
        if (op.b) {  // gates on tile bits
            V e[TILE_R];
            uint32_t em = 0;
            dg_tile_part<V>(op, subs, pool, tid, torig, f, e, em);
            op_dg<V, DAG, TWO, true>(a, b, dgt + op.moff * NR, f);
            if (em & 1u) op_ph<V, DAG, TWO, 0>(a, b, e[0]);
            if (em & 2u) op_ph<V, DAG, TWO, 1>(a, b, e[1]);
            if (em & 4u) op_ph<V, DAG, TWO, 2>(a, b, e[2]);
            if (em & 8u) op_ph<V, DAG, TWO, 3>(a, b, e[3]);
        } else if (any) {
            op_dg<V, DAG, TWO, true>(a, b, dgt + op.moff * NR, f);
        } else {
            op_dg<V, DAG, TWO, false>(a, b, dgt + op.moff * NR, f);
        }
        break;
    }
    case TOP_G1:
        with_pos(op.a, [&](auto P_) { op_g1<V, DAG, TWO, decltype(P_)::value>(a, b, m); });
        break;
    case TOP_D1:
        if (op.a & 0x80) op_d1t<V, DAG, TWO>(a, b, m, tbit(tid, op.a));
        else with_pos(op.a, [&](auto P_) { op_d1r<V, DAG, TWO, decltype(P_)::value>(a, b, m); });
        break;
    case TOP_CX:
        if (op.a & 0x80)
            with_pos(op.b, [&](auto T_) { op_cxt<TWO, decltype(T_)::value>(a, b, tbit(tid, op.a)); });
        else
            with_pos2(op.a, op.b, [&](auto C_, auto T_) {
                op_cxr<TWO, decltype(C_)::value, decltype(T_)::value>(a, b);
            });
        break;
    case TOP_SW:
        with_pos2(op.a, op.b, [&](auto P_, auto Q_) { op_sw<TWO, decltype(P_)::value, decltype(Q_)::value>(a, b); });
        break;
    case TOP_G2:
        with_pos2(op.a, op.b, [&](auto P_, auto Q_) {
            op_g2<V, DAG, TWO, decltype(P_)::value, decltype(Q_)::value>(a, b, m);
        });
        break;
    case TOP_D2: {
        const bool ta = op.a & 0x80, tb = op.b & 0x80;
        if (ta && tb) op_d2tt<V, DAG, TWO>(a, b, m, tbit(tid, op.a) & tbit(tid, op.b));
        else if (ta) with_pos(op.b, [&](auto Q_) { op_d2tr<V, DAG, TWO, decltype(Q_)::value>(a, b, m, tbit(tid, op.a)); });
        else if (tb) with_pos(op.a, [&](auto Q_) { op_d2tr<V, DAG, TWO, decltype(Q_)::value>(a, b, m, tbit(tid, op.b)); });
        else with_pos2(op.a, op.b, [&](auto P_, auto Q_) {
            op_d2rr<V, DAG, TWO, decltype(P_)::value, decltype(Q_)::value>(a, b, m);
        });
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
    if constexpr (same_type<V, float2>::value) {
        if (gen != GEN_X) {
            // Re(conj(l1) p0) - Re(conj(l0) p1), both dot products lane by lane
            float2 sp = make_float2(0.f, 0.f), sm = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                if (j & (1 << P)) continue;
                sp = f2_fma(b[j | (1 << P)], a[j], sp);
                sm = f2_fma(b[j], a[j | (1 << P)], sm);
            }
            return (sp.x + sp.y) - (sm.x + sm.y);
        }
    }
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
                                           uint32_t tid, uint64_t torig = 0) {
    using T = RT<V>;
    T s = 0;
    auto bit_of = [&](uint8_t pos, int j) -> int {
        return (pos & 0x80)       ? (int)((tid >> (pos & 0x7f)) & 1u)
               : is_tile_pos(pos) ? (int)tile_bit(torig, pos)
                                  : ((j >> pos) & 1);
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

// Total of w and its sums over the registers whose bit r is set, for every
// register bit r: halving the array by pair sums at each level costs
// 2^(R-1) + ... adds for the totals and 2^(R-1) - 1 + ... for the odd
// entries, 26 adds at R = 4 instead of 15 per gate of a diagonal run.
template <typename T>
__device__ __forceinline__ void diag_sums(const T (&w)[NR], T &tot, T (&S)[TILE_R]) {
    T cur[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) cur[j] = w[j];
#pragma unroll
    for (int r = 0; r < TILE_R; ++r) {
        const int m = NR >> r;
        T s = cur[1];
#pragma unroll
        for (int k = 3; k < m; k += 2) s += cur[k];
        S[r] = s;
#pragma unroll
        for (int k = 0; k < m / 2; ++k) cur[k] = cur[2 * k] + cur[2 * k + 1];
    }
    tot = cur[0];
}

// Share of a diagonal op's derivative (D1 or D2 outside a run).
template <typename V>
__device__ __forceinline__ RT<V> grad_diag_op(uint8_t type, uint8_t pa, uint8_t pb, uint8_t gen, const V (&a)[NR],
                                              const V (&b)[NR], uint32_t tid) {
    RT<V> w[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) w[j] = im_cdot(b[j], a[j]);
    return grad_diag<V>(type, pa, pb, gen, w, tid);
}

template <typename V>
__device__ __forceinline__ RT<V> grad_op(const TileOp &op, const V (&a)[NR], const V (&b)[NR], uint32_t tid) {
    RT<V> s = 0;
    if (op.type == TOP_G1 || op.type == TOP_G1R) {
        with_pos(op.a, [&](auto P_) { s = grad_g1<decltype(P_)::value>(op.gen, a, b); });
        return s;
    }
    return grad_diag_op<V>(op.type, op.a, op.b, op.gen, a, b, tid);
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

// Shared-memory layout of a block: `nbuf` tile buffers, each holding psi's
// tile (and lambda's in the reverse sweep), then the pass descriptor's parts;
// `gcols` FP64 gradient-partial columns (one per compute warp) per gradient op.
template <typename V, bool ADJ>
__host__ __device__ inline TileSmem tile_smem_n(const TileHead &h, int nbuf, int gcols) {
    const int pool_len = h.pool_len, n_grad = h.n_grad, n_dg = h.n_dg, n_stages = h.n_stages;
    TileSmem s;
    s.tiles = (uint32_t)nbuf * (ADJ ? 2u : 1u) * (1u << TILE_K) * (uint32_t)sizeof(V);
    s.pool = (uint32_t)((pool_len * sizeof(RT<V>) + 15) & ~15u);
    s.gacc = ADJ ? (uint32_t)(n_grad * gcols * sizeof(double)) : 0u;
    s.gacc = (s.gacc + 15) & ~15u;
    s.dgt = (uint32_t)(n_dg * NR * sizeof(V));
    s.tbt = (uint32_t)((n_stages * TILE_TB * sizeof(uint16_t) + 15) & ~15u);
    s.stages = (uint32_t)((n_stages * sizeof(TileStage) + 15) & ~15u);
    s.ops = (uint32_t)((h.n_ops * sizeof(TileOp) + 15) & ~15u);
    s.subs = (uint32_t)((h.n_subs * sizeof(TileSub) + 15) & ~15u);
    s.total = 1024 + s.tiles + s.pool + s.gacc + s.dgt + s.tbt + s.stages + s.ops + s.subs + 16;
    return s;
}
template <typename V, bool ADJ, int NB>
__host__ __device__ inline TileSmem tile_smem(const TileHead &h) {
    return tile_smem_n<V, ADJ>(h, NB, TILE_WARPS);
}
// Ring kernels: B buffers shared by the block's G groups (G * 8 warp columns).
template <typename V, bool ADJ, int B>
__host__ __device__ inline TileSmem tile_smem_ring(const TileHead &h) {
    return tile_smem_n<V, ADJ>(h, B, RingCfg<ADJ>::G * TILE_WARPS);
}

// Blocks per SM the register budget is sized for: what the shared memory of
// the common passes allows.
template <typename V, bool ADJ, int NB> __host__ __device__ constexpr int tile_min_blocks() {
    return sizeof(V) == 8 ? (NB == 1 ? (ADJ ? 2 : 3) : (ADJ ? 1 : 2)) : 1;
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

// What a stage runner sees of the current tile and the pass.
template <typename V> struct TileCtx {
    V *tile_a;               // psi's tile (2^K amplitudes, swizzled)
    V *tile_b;               // lambda's tile (reverse sweep)
    const RT<V> *pool;       // matrix scalars of the pass's ops
    double *gacc;            // [warp column][gradient op] FP64 partial derivatives
    const V *dgt;            // [diagonal run][16] phase tables
    const uint16_t *tbt;     // [stage][TILE_TB] lane / warp address tables
    const TileStage *stages;
    const TileOp *ops;
    const TileSub *subs;
    int n_stages;
    uint32_t tid;            // thread index within the group of 256 that works on the tile
    int lane, warp;
    int gcols, gcol;         // gradient columns of the block; this warp's column
    int n_grad;              // gradient ops of the pass
    uint64_t torig;          // global index of the current tile's local index 0 (its tile bits)
    uint32_t bar_id;         // named barrier of that group (0 = the whole block of 256)
    bool end_sync;           // the last stage ends with the group's barrier too (else each
                             // thread signals the tile's end itself, after its fence)
    int *err;
};

// End of a stage: the group's threads meet (bar.sync on the group's barrier).
template <typename V> __device__ __forceinline__ void tile_sync(const TileCtx<V> &c) {
    asm volatile("bar.sync %0, %1;" ::"r"(c.bar_id), "n"(TILE_THREADS) : "memory");
}

// A stage barrier of level lvl (SYNC_*): the group's, the warp's or none.
template <typename V> __device__ __forceinline__ void stage_sync(const TileCtx<V> &c, uint32_t lvl) {
    if (lvl == SYNC_GROUP) tile_sync(c);
    else if (lvl == SYNC_WARP) __syncwarp();
}

// ------------------------------------------------------ gradient partials
// A gradient value of a tile is one thread's share (its 16 amplitudes, state
// precision) of one angle derivative.  The warp's total of each value is
// added in FP64 to the warp's own column gacc[gcol][slot]: no atomics, and
// every sum across tiles is FP64.
//
// The warp totals come from a transposed butterfly.  Values are merged two at
// a time like the digits of a binary counter: merging two partial sums of
// level L (each already reduced over lane bits 0 .. L-1) exchanges over lane
// bit L; lanes with that bit clear keep the first value's half, the others
// the second's.  After 32 values -- or at the end of the tile, padded with
// zeros -- lane i holds the warp total of the chunk's value i: one shuffle
// per value instead of five.  The reverse sweep meets the pass's gradient ops
// in descending slot order, so value i of a tile belongs to slot
// n_grad - 1 - i.
template <typename T> struct GradAcc {
    T s[5];   // pending partial sums, s[L] of level L
    int cnt;  // values in the current chunk (runtime form)
    int done; // values of the tile already written (runtime form)
};

template <typename T> __device__ __forceinline__ T gmerge(T x, T y, int lane, int L) {
    const bool hi = (lane >> L) & 1;
    return (hi ? y : x) + __shfl_xor_sync(0xffffffffu, hi ? x : y, 1 << L);
}
template <typename T> __device__ __forceinline__ T gpad(T x, int lane, int L) {
    const T t = x + __shfl_xor_sync(0xffffffffu, x, 1 << L);
    return ((lane >> L) & 1) ? T(0) : t;
}
// Lanes i < m add their warp total v (value i of the chunk) to slot top - i.
template <typename V>
__device__ __forceinline__ void gwrite(const TileCtx<V> &c, int top, int m, RT<V> v) {
    if (c.lane < m) c.gacc[c.gcol * c.n_grad + (top - c.lane)] += (double)v;
}

// Value number C (0..31, compile time) of the chunk that ends at slot top.
template <int C, typename V>
__device__ __forceinline__ void gpush(GradAcc<RT<V>> &ga, RT<V> v, const TileCtx<V> &c, int top) {
    using T = RT<V>;
    T g = v;
    if constexpr (!(C & 1)) { ga.s[0] = g; return; }
    g = gmerge<T>(ga.s[0], g, c.lane, 0);
    if constexpr (!(C & 2)) { ga.s[1] = g; return; }
    g = gmerge<T>(ga.s[1], g, c.lane, 1);
    if constexpr (!(C & 4)) { ga.s[2] = g; return; }
    g = gmerge<T>(ga.s[2], g, c.lane, 2);
    if constexpr (!(C & 8)) { ga.s[3] = g; return; }
    g = gmerge<T>(ga.s[3], g, c.lane, 3);
    if constexpr (!(C & 16)) { ga.s[4] = g; return; }
    g = gmerge<T>(ga.s[4], g, c.lane, 4);
    gwrite<V>(c, top, 32, g);  // C == 31: the chunk is complete
}
// End of a chunk of M < 32 values (compile time): pad to 32 and write.
template <int M, typename V>
__device__ __forceinline__ void gflush(GradAcc<RT<V>> &ga, const TileCtx<V> &c, int top) {
    using T = RT<V>;
    if constexpr (M > 0) {
        T acc = T(0);
        bool have = false;
#pragma unroll
        for (int L = 0; L < 5; ++L) {
            if (M & (1 << L)) {
                acc = have ? gmerge<T>(ga.s[L], acc, c.lane, L) : gpad<T>(ga.s[L], c.lane, L);
                have = true;
            } else if (have) {
                acc = gpad<T>(acc, c.lane, L);
            }
        }
        gwrite<V>(c, top, M, acc);
    }
}
// Runtime forms (the generic runner): the counter is uniform over the warp,
// so every branch is too.
template <typename V>
__device__ __forceinline__ void gpush_rt(GradAcc<RT<V>> &ga, RT<V> v, const TileCtx<V> &c) {
    using T = RT<V>;
    T g = v;
#pragma unroll
    for (int L = 0; L < 5; ++L) {
        if (!(ga.cnt & (1 << L))) {
            ga.s[L] = g;
            ++ga.cnt;
            return;
        }
        g = gmerge<T>(ga.s[L], g, c.lane, L);
    }
    gwrite<V>(c, c.n_grad - 1 - ga.done, 32, g);
    ga.cnt = 0;
    ga.done += 32;
}
template <typename V>
__device__ __forceinline__ void gflush_rt(GradAcc<RT<V>> &ga, const TileCtx<V> &c) {
    using T = RT<V>;
    if (ga.cnt > 0) {
        T acc = T(0);
        bool have = false;
#pragma unroll
        for (int L = 0; L < 5; ++L) {
            if (ga.cnt & (1 << L)) {
                acc = have ? gmerge<T>(ga.s[L], acc, c.lane, L) : gpad<T>(ga.s[L], c.lane, L);
                have = true;
            } else if (have) {
                acc = gpad<T>(acc, c.lane, L);
            }
        }
        gwrite<V>(c, c.n_grad - 1 - ga.done, ga.cnt, acc);
    }
    ga.cnt = 0;
    ga.done = 0;
}

// Register j's tile index in a stage: lane and warp table entries XOR the
// register offset.  Forward loads through F and stores through G; the
// reverse sweep the other way.
template <bool ADJ>
__device__ __forceinline__ uint32_t stage_base_ld(const uint16_t *tl, int lane, int warp) {
    constexpr int NW = TILE_THREADS / 32;
    return ADJ ? (uint32_t)(tl[32 + NW + lane] ^ tl[64 + NW + warp]) : (uint32_t)(tl[lane] ^ tl[32 + warp]);
}
template <bool ADJ>
__device__ __forceinline__ uint32_t stage_base_st(const uint16_t *tl, int lane, int warp) {
    constexpr int NW = TILE_THREADS / 32;
    return ADJ ? (uint32_t)(tl[lane] ^ tl[32 + warp]) : (uint32_t)(tl[32 + NW + lane] ^ tl[64 + NW + warp]);
}

// Register j of a stage from / to the tile at index ad (psi, and lambda in
// the reverse sweep).
template <typename V, bool ADJ>
__device__ __forceinline__ void tile_ld(const TileCtx<V> &c, V (&a)[NR], V (&b)[NR], int j, uint32_t ad) {
    int *err = c.err;
    (void)err;
    if (TQD_IDX_OK(ad, (uint32_t)(1 << TILE_K))) {
        a[j] = c.tile_a[ad];
        if (ADJ) b[j] = c.tile_b[ad];
    }
}
template <typename V, bool ADJ>
__device__ __forceinline__ void tile_st(const TileCtx<V> &c, const V (&a)[NR], const V (&b)[NR], int j, uint32_t ad) {
    int *err = c.err;
    (void)err;
    if (TQD_IDX_OK(ad, (uint32_t)(1 << TILE_K))) {
        c.tile_a[ad] = a[j];
        if (ADJ) c.tile_b[ad] = b[j];
    }
}

// Registers j0 and j1 of a stage whose amplitudes are adjacent in the tile
// (indices ad and ad + 1, ad even: one 16-byte chunk of complex64 values)
// with one 16-byte shared-memory access per state.
template <typename V, bool ADJ>
__device__ __forceinline__ void tile_ld2(const TileCtx<V> &c, V (&a)[NR], V (&b)[NR], int j0, int j1, uint32_t ad) {
    static_assert(sizeof(V) == 8, "pairs of complex64 amplitudes");
    int *err = c.err;
    (void)err;
    if (TQD_IDX_OK(ad + 1, (uint32_t)(1 << TILE_K))) {
        const float4 x = *reinterpret_cast<const float4 *>(c.tile_a + ad);
        a[j0] = make_float2(x.x, x.y);
        a[j1] = make_float2(x.z, x.w);
        if (ADJ) {
            const float4 y = *reinterpret_cast<const float4 *>(c.tile_b + ad);
            b[j0] = make_float2(y.x, y.y);
            b[j1] = make_float2(y.z, y.w);
        }
    }
}
template <typename V, bool ADJ>
__device__ __forceinline__ void tile_st2(const TileCtx<V> &c, const V (&a)[NR], const V (&b)[NR], int j0, int j1,
                                         uint32_t ad) {
    static_assert(sizeof(V) == 8, "pairs of complex64 amplitudes");
    int *err = c.err;
    (void)err;
    if (TQD_IDX_OK(ad + 1, (uint32_t)(1 << TILE_K))) {
        *reinterpret_cast<float4 *>(c.tile_a + ad) = make_float4(a[j0].x, a[j0].y, a[j1].x, a[j1].y);
        if (ADJ) *reinterpret_cast<float4 *>(c.tile_b + ad) = make_float4(b[j0].x, b[j0].y, b[j1].x, b[j1].y);
    }
}

// Lambda only, as tile_st / tile_st2 (a reverse stage whose psi is not
// needed any more: the last stage of a pass that read psi from a forward
// checkpoint).
template <typename V, bool ADJ>
__device__ __forceinline__ void tile_stl(const TileCtx<V> &c, const V (&a)[NR], const V (&b)[NR], int j,
                                         uint32_t ad) {
    static_assert(ADJ, "lambda exists in the reverse sweep only");
    (void)a;
    int *err = c.err;
    (void)err;
    if (TQD_IDX_OK(ad, (uint32_t)(1 << TILE_K))) c.tile_b[ad] = b[j];
}
template <typename V, bool ADJ>
__device__ __forceinline__ void tile_stl2(const TileCtx<V> &c, const V (&a)[NR], const V (&b)[NR], int j0, int j1,
                                          uint32_t ad) {
    static_assert(ADJ && sizeof(V) == 8, "lambda pairs of complex64 amplitudes");
    (void)a;
    int *err = c.err;
    (void)err;
    if (TQD_IDX_OK(ad + 1, (uint32_t)(1 << TILE_K)))
        *reinterpret_cast<float4 *>(c.tile_b + ad) = make_float4(b[j0].x, b[j0].y, b[j1].x, b[j1].y);
}

// The generic stage runner: interprets the pass's stage and op lists.
// finish(c) ends a tile: the reverse sweep writes the last gradient chunk.
template <typename V, bool ADJ> struct InterpRunner {
    GradAcc<RT<V>> ga;
    __device__ __forceinline__ void init(const TileCtx<V> &) {
        ga.cnt = 0;
        ga.done = 0;
    }
    __device__ __forceinline__ void finish(const TileCtx<V> &c) {
        if (ADJ) gflush_rt<V>(ga, c);
    }
    __device__ __forceinline__ void run(const TileCtx<V> &c) {
        using T = RT<V>;
        int *err = c.err;
        for (int si = 0; si < c.n_stages; ++si) {
            const int s = ADJ ? c.n_stages - 1 - si : si;
            const TileStage &st = c.stages[s];
            const uint16_t *tl = c.tbt + s * TILE_TB;
            const uint32_t base_ld = stage_base_ld<ADJ>(tl, c.lane, c.warp);
            const uint32_t base_st = stage_base_st<ADJ>(tl, c.lane, c.warp);
            const uint16_t *roff_ld = ADJ ? st.st_roff : st.ld_roff;
            const uint16_t *roff_st = ADJ ? st.ld_roff : st.st_roff;
            V a[NR];
            V b[NR];
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const uint32_t ad = base_ld ^ roff_ld[j];
                if (TQD_IDX_OK(ad, (uint32_t)(1 << TILE_K))) {
                    a[j] = c.tile_a[ad];
                    if (ADJ) b[j] = c.tile_b[ad];
                }
            }
            if (!ADJ) {
                for (int k = st.op_begin; k < st.op_end; ++k)
                    apply_op<V, false, false>(c.ops[k], a, b, c.pool, c.tid, c.subs, c.dgt, c.torig);
            } else {
                for (int k = (int)st.op_end - 1; k >= (int)st.op_begin; --k) {
                    const TileOp op = c.ops[k];
                    if (op.type == TOP_DG) {
                        T w[NR];
#pragma unroll
                        for (int j = 0; j < NR; ++j) w[j] = im_cdot(b[j], a[j]);
                        // descending, so that the pass's gradient values arrive in
                        // descending slot order
                        for (int q = op.sub0 + op.nsub - 1; q >= op.sub0; --q) {
                            const TileSub sb = c.subs[q];
                            if (sb.gslot < 0) continue;
                            gpush_rt<V>(ga, grad_diag<V>(sb.type, sb.a, sb.b, sb.gen, w, c.tid, c.torig), c);
                        }
                    } else if (op.gslot >= 0) {
                        gpush_rt<V>(ga, grad_op<V>(op, a, b, c.tid), c);
                    }
                    apply_op<V, true, true>(op, a, b, c.pool, c.tid, c.subs, c.dgt, c.torig);
                }
            }
            stage_sync(c, st.sync_mid);
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const uint32_t ad = base_st ^ roff_st[j];
                if (TQD_IDX_OK(ad, (uint32_t)(1 << TILE_K))) {
                    c.tile_a[ad] = a[j];
                    if (ADJ) c.tile_b[ad] = b[j];
                }
            }
            // the last stage's writes are read next by the TMA store; between
            // stages s and s + 1 (either direction) the barrier of sync_end[s]
            if (si == c.n_stages - 1) fence_async_smem();
            if (si < c.n_stages - 1) stage_sync(c, c.stages[ADJ ? s - 1 : s].sync_end);
            else if (c.end_sync) tile_sync(c);
        }
    }
};

// Shared-memory pointers of a block, and the descriptor staged there.
template <typename V> struct TileShared {
    V *tiles;
    RT<V> *pool;
    double *gacc;
    V *dgt;
    uint16_t *tbt;
    TileStage *stages;
    TileOp *ops;
    TileSub *subs;
    uint64_t *bar;  // NB body: its tile barriers (dynamic part); unused by the ring
};

// Carves the dynamic shared memory by layout L, copies the pass descriptor
// into it, gathers the ops' matrices into the pool, builds the per-stage
// address tables and the diagonal runs' phase tables, and zeroes the
// gradient partials (gcols columns).  All threads of the block take part;
// ends with __syncthreads().
template <typename V, bool ADJ>
__device__ __forceinline__ TileShared<V> tile_setup(const TileHead &P, const TilePassDev *Pg, const RT<V> *mats,
                                                    const TileSmem &L, int gcols, int *err) {
    using T = RT<V>;
    extern __shared__ unsigned char smem_raw[];
    (void)err;
    const uint32_t pad = (1024u - (sptr(smem_raw) & 1023u)) & 1023u;
    unsigned char *sm = smem_raw + pad;
    TileShared<V> S;
    S.tiles = reinterpret_cast<V *>(sm);
    S.pool = reinterpret_cast<T *>(sm + L.tiles);
    S.gacc = reinterpret_cast<double *>(sm + L.tiles + L.pool);
    S.dgt = reinterpret_cast<V *>(sm + L.tiles + L.pool + L.gacc);
    S.tbt = reinterpret_cast<uint16_t *>(sm + L.tiles + L.pool + L.gacc + L.dgt);
    S.stages = reinterpret_cast<TileStage *>(sm + L.tiles + L.pool + L.gacc + L.dgt + L.tbt);
    S.ops = reinterpret_cast<TileOp *>(sm + L.tiles + L.pool + L.gacc + L.dgt + L.tbt + L.stages);
    S.subs = reinterpret_cast<TileSub *>(sm + L.tiles + L.pool + L.gacc + L.dgt + L.tbt + L.stages + L.ops);
    S.bar = reinterpret_cast<uint64_t *>(sm + L.tiles + L.pool + L.gacc + L.dgt + L.tbt + L.stages + L.ops + L.subs);
    const uint32_t tid = threadIdx.x;
    constexpr int TBS = TILE_TB;
    constexpr int NW = TILE_THREADS / 32;

    copy_words(S.stages, Pg->stages, P.n_stages * sizeof(TileStage));
    copy_words(S.ops, Pg->ops, P.n_ops * sizeof(TileOp));
    copy_words(S.subs, Pg->subs, P.n_subs * sizeof(TileSub));
    __syncthreads();

    // matrices of every op and diagonal sub-op, per-stage lane/warp offsets
    for (int k = 0; k < P.n_ops; ++k) {
        const TileOp op = S.ops[k];
        if (op.moff < 0 || op.type == TOP_DG) continue;
        int src, len;
        op_pool_span(op.type, src, len);
        for (int i = tid; i < len; i += blockDim.x)
            if (TQD_IDX_OK((uint32_t)(op.moff + i), (uint32_t)P.pool_len))
                S.pool[op.moff + i] = mats[(size_t)Pg->op_gate[k] * MAT_STRIDE + src + i];
    }
    for (int k = 0; k < P.n_subs; ++k) {
        const TileSub sb = S.subs[k];
        const int src = sb.type == TOP_D1 ? 0 : 30, len = sb.type == TOP_D1 ? 8 : 2;
        for (int i = tid; i < len; i += blockDim.x)
            if (TQD_IDX_OK((uint32_t)(sb.moff + i), (uint32_t)P.pool_len))
                S.pool[sb.moff + i] = mats[(size_t)Pg->sub_gate[k] * MAT_STRIDE + src + i];
    }
    for (int i = tid; i < P.n_stages * TBS; i += blockDim.x) {
        const int st = i / TBS, e = i % TBS;
        const TileStage &St = S.stages[st];
        S.tbt[i] = e < 32 ? St.ld_lo[e] : e < 32 + NW ? St.ld_hi[e - 32] : e < 64 + NW ? St.st_lo[e - 32 - NW]
                                                                                     : St.st_hi[e - 64 - NW];
    }
    if (ADJ) {
        for (int i = tid; i < P.n_grad * gcols; i += blockDim.x) S.gacc[i] = 0.0;
    }
    __syncthreads();
    // phase tables of the diagonal runs: entry j = product of the run's gates
    // whose positions are all register bits, evaluated at register index j
    for (int i = tid; i < P.n_dg * NR; i += blockDim.x) {
        const int d = i / NR, j = i % NR;
        const TileOp op = S.ops[Pg->dg_op[d]];
        V t = mkc<V>(1, 0);
        for (int q = op.sub0; q < op.sub0 + op.nsub; ++q) {
            const TileSub sb = S.subs[q];
            if (sb.a & 0xC0) continue;  // thread or tile bits
            if (sb.type == TOP_D1) t = cmul(t, pool_c<V>(S.pool, sb.moff + (((j >> sb.a) & 1) ? 6 : 0)));
            else if (((j >> sb.a) & 1) && ((j >> sb.b) & 1)) t = cmul(t, pool_c<V>(S.pool, sb.moff));
        }
        S.dgt[i] = t;
    }
    __syncthreads();
    return S;
}

// TMA coordinates of copy e of a tile: its global index origin plus the
// extra local bits, split into the tensor map's dimensions.
__device__ __forceinline__ void tile_coords(const TileHead &P, uint64_t tile, int e, int (&c)[TILE_MAX_DIMS]) {
    uint64_t g = 0;
    for (int i = 0; i < P.n_tiles_log2; ++i) g |= ((tile >> i) & 1ull) << P.out_bits[i];
    for (int i = 0; i < P.n_extra; ++i) g |= (uint64_t)((e >> i) & 1) << P.extra_bits[i];
#pragma unroll
    for (int d = 0; d < TILE_MAX_DIMS; ++d)
        c[d] = d < P.rank ? (int)((g >> P.dim_lo[d]) & ((1ull << P.dim_len[d]) - 1)) : 0;
}

// Global index of local index 0 of a tile (the values of the qubits outside
// the pass's set).
__device__ __forceinline__ uint64_t tile_origin(const TileHead &P, uint64_t tile) {
    uint64_t g = 0;
    for (int i = 0; i < P.n_tiles_log2; ++i) g |= ((tile >> i) & 1ull) << P.out_bits[i];
    return g;
}

// One thread: TMA loads of a tile (psi, and lambda when ADJ) into `dst`,
// completing on barrier `bar`.  stall (TILE_STALL_TEST): the barrier is armed
// for the tile's bytes but no copy is issued, so its phase never completes
// and the wait for it runs out (nothing is in flight for it either).
template <typename V, bool ADJ>
__device__ __forceinline__ void tile_issue_load(const TileHead &P, const void *map_psi, const void *map_lam, V *dst,
                                                uint64_t *bar, uint64_t tile, bool stall = false) {
    constexpr int TS = 1 << TILE_K;
    constexpr uint32_t NSTATE = ADJ ? 2u : 1u;
    const uint32_t tile_bytes = TS * (uint32_t)sizeof(V);
    const uint32_t box_bytes = tile_bytes >> P.n_extra;
    mbar_expect_tx(bar, tile_bytes * NSTATE);
    if (stall) return;
    for (int e = 0; e < (1 << P.n_extra); ++e) {
        int c[TILE_MAX_DIMS];
        tile_coords(P, tile, e, c);
        tma_load(P.rank, map_psi, sptr(dst) + e * box_bytes, bar, c);
        if (ADJ) tma_load(P.rank, map_lam, sptr(dst + TS) + e * box_bytes, bar, c);
    }
}

// One thread: TMA stores of the tile in `src`, as one bulk group.  The
// forward pass stores psi through map_lam (its destination: the source map
// itself in place, another state for a checkpoint); the reverse sweep stores
// psi through map_psi unless flags has TILE_PSI_RO (psi read from a forward
// checkpoint and not needed again) and lambda through map_lam.
template <typename V, bool ADJ>
__device__ __forceinline__ void tile_issue_store(const TileHead &P, const void *map_psi, const void *map_lam,
                                                 V *src, uint64_t tile, int flags) {
    constexpr int TS = 1 << TILE_K;
    const uint32_t box_bytes = (TS * (uint32_t)sizeof(V)) >> P.n_extra;
    for (int e = 0; e < (1 << P.n_extra); ++e) {
        int c[TILE_MAX_DIMS];
        tile_coords(P, tile, e, c);
        if (!ADJ) {
            tma_store(P.rank, map_lam, sptr(src) + e * box_bytes, c);
        } else {
            if (!(flags & TILE_PSI_RO)) tma_store(P.rank, map_psi, sptr(src) + e * box_bytes, c);
            tma_store(P.rank, map_lam, sptr(src + TS) + e * box_bytes, c);
        }
    }
    bulk_commit();
}

// Bounded wait of one thread for phase `parity` of barrier `bar`: 1 when the
// phase completed, 0 when WAIT_LIMIT_NS passed first.
__device__ __forceinline__ int mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return 1;
    const uint64_t t0 = gtimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (gtimer_ns() - t0 > WAIT_LIMIT_NS) return 0;
    return 1;
}

// Gradient partials of the block (gcols FP64 columns of n_grad entries)
// summed in FP64, one warp per gradient op.  Ends the pass.  nw: the warps taking
// part (the block's first nw).
__device__ __forceinline__ void tile_write_partials(const TileHead &P, const TilePassDev *Pg, const double *gacc,
                                                    int gcols, double *partials, int pblk, int nw, int pcol) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < P.n_grad; k += nw) {
        double t = 0;
        for (int i = lane; i < gcols; i += 32) t += gacc[i * P.n_grad + k];
        t = warp_sum(t);
        if (lane == 0) partials[(size_t)Pg->grad_gate_slot[k] * pblk + pcol] = t;
    }
}

// The whole pass for one block of 256 threads with NB tile buffers: stage the
// descriptor in shared memory, then load, run and store this block's tiles;
// in the reverse sweep, write the block's gradient partials.
// Runner::init(ctx) computes once per block what does not depend on the
// tile; run(ctx) applies every stage to the current tile and ends each stage
// with tile_sync(ctx) (the last one after fence.proxy.async).
template <typename V, bool ADJ, int NB, typename Runner>
__device__ __forceinline__ void tile_pass_body(const void *map_psi, const void *map_lam, const TilePassDev *Pg,
                                               const RT<V> *mats, double *partials, int pblk, int *err,
                                               int flags) {
    __shared__ TileHead P;
    __shared__ int s_timeout;
    copy_words(&P, &Pg->h, sizeof(TileHead));
    __syncthreads();
    const TileSmem L = tile_smem<V, ADJ, NB>(P);
    const uint32_t tid = threadIdx.x;
    const bool stall = (flags & TILE_STALL_TEST) && blockIdx.x == 0;
    if (tid == 0) {
        // the barriers sit after the descriptor parts; initialised before the
        // setup's first __syncthreads
        extern __shared__ unsigned char smem_raw[];
        const uint32_t pad = (1024u - (sptr(smem_raw) & 1023u)) & 1023u;
        uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + pad + L.total - 1024 - 16);
        for (int i = 0; i < NB; ++i) mbar_init(bar + i, 1);
        mbar_fence_init();
    }
    const TileShared<V> S = tile_setup<V, ADJ>(P, Pg, mats, L, TILE_WARPS, err);
    uint64_t *bar = S.bar;

    constexpr int TS = 1 << TILE_K;          // amplitudes per tile
    constexpr uint32_t NSTATE = ADJ ? 2u : 1u;
    const uint64_t n_tiles = (uint64_t)1 << P.n_tiles_log2;

    // Thread 0 waits (bounded) for buffer buf's copy; the block learns the
    // outcome at the barrier, so every thread takes the same branch.  The
    // other threads then acquire the completed phase themselves.
    uint32_t parity = 0;  // bit b: phase parity of buffer b's barrier
    auto wait_tile = [&](int buf) -> bool {
        const uint32_t ph = (parity >> buf) & 1u;
        if (tid == 0) s_timeout = !mbar_wait_bounded(bar + buf, ph);
        __syncthreads();
        if (s_timeout) return false;
        if (tid != 0) mbar_try_wait(bar + buf, ph);
        parity ^= 1u << buf;
        return true;
    };

    TileCtx<V> ctx;
    ctx.pool = S.pool;
    ctx.gacc = S.gacc;
    ctx.dgt = S.dgt;
    ctx.tbt = S.tbt;
    ctx.stages = S.stages;
    ctx.ops = S.ops;
    ctx.subs = S.subs;
    ctx.n_stages = P.n_stages;
    ctx.tid = tid;
    ctx.lane = tid & 31;
    ctx.warp = tid >> 5;
    ctx.gcols = TILE_WARPS;
    ctx.gcol = ctx.warp;
    ctx.n_grad = P.n_grad;
    ctx.bar_id = 0;
    ctx.end_sync = true;
    ctx.err = err;
    Runner runner;  // per-thread values of the pass that do not depend on the tile
    runner.init(ctx);

    // NB = 2: the next tile's copy is in flight while this one is computed;
    // a buffer is refilled only after its previous store has read it.
    if (NB == 2 && tid == 0 && blockIdx.x < n_tiles)
        tile_issue_load<V, ADJ>(P, map_psi, map_lam, S.tiles, bar, blockIdx.x, stall);
    int iter = 0;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++iter) {
        const int cur = NB == 2 ? (iter & 1) : 0;
        bool next_issued = false;
        if (tid == 0) {
            const uint64_t next = NB == 2 ? tile + gridDim.x : tile;
            if (next < n_tiles) {
                bulk_wait_read0();
                const int nb = NB == 2 ? cur ^ 1 : 0;
                tile_issue_load<V, ADJ>(P, map_psi, map_lam, S.tiles + (size_t)nb * NSTATE * TS, bar + nb, next,
                                        NB == 1 && stall && iter == 0);
                next_issued = NB == 2;
            }
        }
        if (!wait_tile(cur)) {
            if (tid == 0) {
                atomicExch(err, 1);
                // the other buffer's copy (NB = 2) lands before the block leaves
                if (next_issued) mbar_wait_bounded(bar + (cur ^ 1), (parity >> (cur ^ 1)) & 1u);
                bulk_wait0();
            }
            return;
        }
        ctx.tile_a = S.tiles + (size_t)cur * NSTATE * TS;
        ctx.tile_b = ctx.tile_a + TS;
        ctx.torig = tile_origin(P, tile);
        runner.run(ctx);
        if (tid == 0) tile_issue_store<V, ADJ>(P, map_psi, map_lam, ctx.tile_a, tile, flags);
        runner.finish(ctx);
    }
    if (tid == 0) bulk_wait0();
    if (ADJ) {
        __syncthreads();
        // the warps' FP64 columns, summed in FP64, one warp per gradient op
        tile_write_partials(P, Pg, S.gacc, TILE_WARPS, partials, pblk, TILE_WARPS, blockIdx.x);
    }
}

// Register shares of warp-specialised blocks (setmaxnreg, per warpgroup;
// every warp of the warpgroup executes it).
template <int N> __device__ __forceinline__ void reg_dealloc() {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}
template <int N> __device__ __forceinline__ void reg_alloc() {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}

// The whole pass for one block of G groups of 256 threads sharing a ring of
// B tile buffers, plus (TMAW) one TMA warpgroup (one block per SM).  Tile k of the
// block's sequence (global tile blockIdx.x + k * gridDim.x) goes through
// buffer k mod B and is computed by group k mod G.
//  - TMAW: the TMA warpgroup hands most of its registers to the groups
//    (setmaxnreg; RingCfg's shares) and issues every copy, from one thread
//    per group when B is a multiple of G (each group's copies then wait only
//    for its own stores), else from one thread: it loads the first B tiles
//    (its share), then for each of its k: waits until tile k is computed
//    (done[buffer]), stores it, waits until the store has read the buffer and
//    loads tile k + B into it.  The compute groups never wait for a store.
//  - A group's first thread waits (bounded) for its tile's load (full[buffer]);
//    the group runs every stage, meeting on its own named barrier after each
//    but the last; then (TMAW) each thread fences its writes and arrives on
//    done[buffer] (256 arrivals complete it) and goes on, or else the group
//    meets once more and its first thread stores the tile itself, waits until
//    the store has read the buffer and loads tile k + B into it.
// Up to B - G tiles are on their way in while G are computed.  A buffer passes
// between groups when B is not a multiple of G: the waiter for tile k + B
// first waits until tile k has been taken (gen[buffer] counts the tiles taken
// from each buffer), so the barrier parity it waits on is never a phase stale.
//
// The tiles are tbase + k * tstride for k < count (count < 0: every tile of
// the pass from tbase on), and the block's gradient partials go to column
// pcol.  REUSE: the function is called again by the same block (a persistent
// kernel); its barriers are invalidated at the end so that the next call
// initialises them afresh, and every thread of the block takes part.
template <typename V, bool ADJ, int G, int B, bool TMAW, typename Runner, bool REUSE = false>
__device__ __forceinline__ void tile_ring_tiles(const void *map_psi, const void *map_lam, const TilePassDev *Pg,
                                                const RT<V> *mats, double *partials, int pblk, int *err, int flags,
                                                uint64_t tbase, uint64_t tstride, int64_t count, int pcol) {
    static_assert(B >= G, "a ring needs a buffer per group");
    static_assert(!(REUSE && TMAW), "a reused ring has no TMA warpgroup");
    static_assert(!TMAW || G == RingCfg<ADJ>::G, "the register shares are set for RingCfg's groups");
    __shared__ TileHead P;
    __shared__ uint64_t fullb[B];
    __shared__ uint64_t doneb[B];
    __shared__ int gen[B];
    // per group and parity of its iteration: the first thread's wait outcome
    // (two slots, so a slot is rewritten only after every thread of the group
    // has passed the group barrier that follows its next read)
    __shared__ int s_timeout[G][2];
    copy_words(&P, &Pg->h, sizeof(TileHead));
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < B; ++i) {
            mbar_init(fullb + i, 1);
            mbar_init(doneb + i, TILE_THREADS);  // TMAW: every thread of the group arrives
            gen[i] = 0;
        }
        mbar_fence_init();
    }
    __syncthreads();
    const TileSmem L = tile_smem_ring<V, ADJ, B>(P);
    const TileShared<V> S = tile_setup<V, ADJ>(P, Pg, mats, L, G * TILE_WARPS, err);

    constexpr int TS = 1 << TILE_K;
    constexpr uint32_t NSTATE = ADJ ? 2u : 1u;
    const uint64_t n_tiles = (uint64_t)1 << P.n_tiles_log2;
    const uint64_t n_local = count >= 0 ? (uint64_t)count
                                        : (n_tiles > tbase ? (n_tiles - 1 - tbase) / tstride + 1 : 0);
    const int grp = (int)(tid >> 8);  // G: the TMA warp
    const bool stall = (flags & TILE_STALL_TEST) && blockIdx.x == 0;

    // Before a thread that issued loads leaves early: wait (bounded) until
    // the copies of tiles k0 .. k0 + B - 1 (its share: k = first mod step)
    // have landed, so no copy is still writing into the block's shared
    // memory when it exits.  A phase that already completed passes at once.
    auto drain = [&](uint64_t k0, uint64_t first, uint64_t step) {
        for (uint64_t k = k0; k < k0 + B && k < n_local; ++k)
            if (k % step == first % step) mbar_wait_bounded(fullb + (int)(k % B), (uint32_t)(k / B) & 1u);
    };

    if (!TMAW && tid == 0)
        for (int k = 0; k < B && (uint64_t)k < n_local; ++k)
            tile_issue_load<V, ADJ>(P, map_psi, map_lam, S.tiles + (size_t)k * NSTATE * TS, fullb + k,
                                    tbase + (uint64_t)k * tstride, stall && k == 0);
    if (TMAW && grp == G) {
        // the TMA warpgroup gives registers to the groups and leaves when its
        // copies are done (the groups write the gradient partials)
        reg_dealloc<RingCfg<ADJ>::REGS_TMA>();
        // NP copying threads, the first of warps 0 .. NP - 1 of the
        // warpgroup: one per group (thread p copies group p's tiles, k = p
        // mod G) when every buffer stays with one group (B a multiple of G),
        // else one for all tiles in their order.  Either way each thread
        // meets the tiles of a buffer in order, so done[buffer] is in tile
        // k's phase when its parity is tested.
        constexpr int NP = B % G == 0 ? G : 1;
        const uint32_t pw = (tid - (uint32_t)G * TILE_THREADS) >> 5;
        if ((tid & 31) == 0 && pw < (uint32_t)NP) {
            for (int k = (int)pw; k < B && (uint64_t)k < n_local; k += NP)
                tile_issue_load<V, ADJ>(P, map_psi, map_lam, S.tiles + (size_t)k * NSTATE * TS, fullb + k,
                                        tbase + (uint64_t)k * tstride, stall && k == 0);
            uint64_t k = pw;
            for (; k < n_local; k += NP) {
                const int slot = (int)(k % B);
                V *buf = S.tiles + (size_t)slot * NSTATE * TS;
                if (!mbar_wait_bounded(doneb + slot, (uint32_t)(k / B) & 1u)) {
                    atomicExch(err, 1);
                    break;
                }
                const uint64_t tile = tbase + k * tstride;
                tile_issue_store<V, ADJ>(P, map_psi, map_lam, buf, tile, flags);
                if (k + B < n_local) {
                    bulk_wait_read0();
                    tile_issue_load<V, ADJ>(P, map_psi, map_lam, buf, fullb + slot, tile + (uint64_t)B * tstride);
                }
            }
            // the loads this thread issued and nobody took: tiles k .. k + B - 1
            // of its share (none when the loop ran to the end)
            if (k < n_local) drain(k, pw, NP);
            bulk_wait0();
        }
        return;
    } else {
        if (TMAW) reg_alloc<RingCfg<ADJ>::REGS_GROUP>();
        const uint32_t gtid = tid & (TILE_THREADS - 1);
        TileCtx<V> ctx;
        ctx.pool = S.pool;
        ctx.gacc = S.gacc;
        ctx.dgt = S.dgt;
        ctx.tbt = S.tbt;
        ctx.stages = S.stages;
        ctx.ops = S.ops;
        ctx.subs = S.subs;
        ctx.n_stages = P.n_stages;
        ctx.tid = gtid;
        ctx.lane = gtid & 31;
        ctx.warp = gtid >> 5;
        ctx.gcols = G * TILE_WARPS;
        ctx.gcol = grp * TILE_WARPS + ctx.warp;
        ctx.n_grad = P.n_grad;
        ctx.bar_id = 1 + grp;
        ctx.end_sync = !TMAW;
        ctx.err = err;
        Runner runner;
        runner.init(ctx);
        uint32_t it = 0;  // this group's iteration count
        for (uint64_t k = grp; k < n_local; k += G, ++it) {
            const int slot = (int)(k % B);
            const uint32_t round = (uint32_t)(k / B);
            if (gtid == 0) {
                int ok = 1;
                // tile k - B taken (only needed when buffers pass between groups)
                if (B % G != 0) {
                    volatile int *gv = gen;
                    if (gv[slot] < (int)round) {
                        const uint64_t t0 = gtimer_ns();
                        while (gv[slot] < (int)round)
                            if (gtimer_ns() - t0 > WAIT_LIMIT_NS) {
                                ok = 0;
                                break;
                            }
                    }
                }
                if (ok) ok = mbar_wait_bounded(fullb + slot, round & 1u);
                if (ok && B % G != 0) {
                    volatile int *gv = gen;
                    gv[slot] = (int)round + 1;
                }
                s_timeout[grp][it & 1] = !ok;
            }
            asm volatile("bar.sync %0, %1;" ::"r"(ctx.bar_id), "n"(TILE_THREADS) : "memory");
            if (s_timeout[grp][it & 1]) {
                if (gtid == 0) {
                    atomicExch(err, 1);
                    // without the TMA warpgroup this thread issued refills:
                    // let every copy of the next B tiles land first
                    if (!TMAW) drain(k, 0, 1);
                }
                break;
            }
            if (gtid != 0) mbar_try_wait(fullb + slot, round & 1u);
            ctx.tile_a = S.tiles + (size_t)slot * NSTATE * TS;
            ctx.tile_b = ctx.tile_a + TS;
            ctx.torig = tile_origin(P, tbase + k * tstride);
            runner.run(ctx);
            if (TMAW) {
                // each thread has written its part of the tile and fenced it for
                // the async proxy: its arrival hands that part to the TMA
                // warpgroup (the tile is done when all 256 have arrived), and
                // the thread goes on to its next tile without meeting the others
                mbar_arrive(doneb + slot);
            } else if (gtid == 0) {
                // without a TMA warp the group's first thread stores the tile,
                // waits until the store has read the buffer and refills it
                const uint64_t tile = tbase + k * tstride;
                tile_issue_store<V, ADJ>(P, map_psi, map_lam, ctx.tile_a, tile, flags);
                if (k + B < n_local) {
                    bulk_wait_read0();
                    tile_issue_load<V, ADJ>(P, map_psi, map_lam, ctx.tile_a, fullb + slot,
                                            tile + (uint64_t)B * tstride);
                }
            }
            // the tile's last gradient values go to the warps' FP64 columns
            // after the tile has been handed on
            runner.finish(ctx);
        }
        if (!TMAW && gtid == 0) bulk_wait0();
    }
    if (ADJ) {
        // the groups only (the TMA warpgroup has left): named barrier 15
        asm volatile("bar.sync 15, %0;" ::"n"(G * TILE_THREADS) : "memory");
        tile_write_partials(P, Pg, S.gacc, G * TILE_WARPS, partials, pblk, G * TILE_WARPS, pcol);
    }
    if (REUSE) {
        // every copy has landed or been waited out and every wait is over:
        // the stores (async proxy) are ordered before what the caller does
        // next, and the barriers go back to uninitialised for the next call
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncthreads();
        if (tid == 0)
            for (int i = 0; i < B; ++i) {
                mbar_inval(fullb + i);
                mbar_inval(doneb + i);
            }
        __syncthreads();
    }
}

template <typename V, bool ADJ, int G, int B, bool TMAW, typename Runner>
__device__ __forceinline__ void tile_pass_ring(const void *map_psi, const void *map_lam, const TilePassDev *Pg,
                                               const RT<V> *mats, double *partials, int pblk, int *err,
                                               int flags) {
    tile_ring_tiles<V, ADJ, G, B, TMAW, Runner>(map_psi, map_lam, Pg, mats, partials, pblk, err, flags, blockIdx.x,
                                                gridDim.x, -1, blockIdx.x);
}

}  // namespace tqd
