// kernels_pauli_tile.cu -- Pauli sums over tiles: several x-mask groups per
// pass over the state.
//
// A term coeff * i^{|x&z|} X^x Z^z (Sec. 2.2.1's Z measurement generalised
// to Pauli strings) pairs amplitude b with b ^ x.  Take a set Q of 12 qubits:
// qubits 0..3 and 8 others.  Every group whose x mask lies inside Q pairs
// amplitudes of the same tile (the 2^12 amplitudes that agree outside Q), so
// one pass that stages each tile in shared memory serves all such groups:
//   E   = sum_b Re( conj(psi_{b^x}) psi_b D_x(b) ),
//   out_b (+)= sum_groups D_x(b ^ x) psi_{b^x},
// with D_x(b) = sum_{j in group} c_j i^{|x&z_j|} (-1)^{|b & z_j|}.  The sign
// splits into the tile's origin (bits outside Q, one factor per tile and
// term) and the local index.  The planner covers the groups with as few
// such sets Q as it can; groups that flip more than 8 qubits above qubit 3
// stay with the per-group kernels of kernels_pauli.cu.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "launch.h"
#include "pauli_tile.h"
#include "prof.h"

namespace tqd {

template <typename V> using RT = typename Real<V>::T;

namespace {

constexpr int PK = 12;                  // qubits per tile
constexpr int PTS = 1 << PK;            // amplitudes per tile
constexpr int PTHR = 256;               // threads per block
constexpr int PPER = PTS / PTHR;        // amplitudes per thread

// Copy `bytes` (a multiple of 4) into shared memory.
__device__ __forceinline__ void copy_in(void *dst, const void *src, uint32_t bytes) {
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t i = threadIdx.x; i < bytes / 4; i += blockDim.x) d[i] = s[i];
}

// Global index of the tile's origin: tile index bits scattered onto the
// qubits outside Q.
__device__ __forceinline__ uint64_t tile_origin(const PauliTileDesc &P, uint64_t tile) {
    uint64_t g = 0;
    for (int i = 0; i < P.n - PK; ++i) g |= ((tile >> i) & 1ull) << P.out_q[i];
    return g;
}

// Shared state of a block: the descriptor, the offsets of the 256 values of
// Q's high qubits, per-tile signed coefficients and the staged tile.
template <typename V> struct PauliSmem {
    PauliTileDesc P;
    uint64_t hoff[256];
    RT<V> cre[PT_MAXT], cim[PT_MAXT];
};

template <typename V> __device__ __forceinline__ void setup(PauliSmem<V> &S, const PauliTileDesc &Pg) {
    copy_in(&S.P, &Pg, sizeof(PauliTileDesc));
    __syncthreads();
    for (int h = threadIdx.x; h < 256; h += blockDim.x) {
        uint64_t o = 0;
        for (int i = 0; i < 8; ++i) o |= (uint64_t)((h >> i) & 1) << S.P.hi[i];
        S.hoff[h] = o;
    }
    __syncthreads();
}

// Coefficients of this tile: c_j w_j scale * (-1)^{|origin & z_j|}.
template <typename V>
__device__ __forceinline__ void tile_coeffs(PauliSmem<V> &S, uint64_t origin, const double *weights, double scale) {
    for (int j = threadIdx.x; j < S.P.n_terms; j += blockDim.x) {
        double w = scale;
        if (weights) w *= weights[S.P.idx[j]];
        if (__popcll(origin & S.P.zo[j]) & 1) w = -w;
        S.cre[j] = (RT<V>)(S.P.cre[j] * w);
        S.cim[j] = (RT<V>)(S.P.cim[j] * w);
    }
}

// D_g at the thread's 16 local indices l = r * 256 + tid (r = 0..15), the
// origin's sign already in the coefficients.  Bits 0..7 of l are the
// thread's, so a term's sign is a per-thread factor times (-1)^{|r & z_hi|}
// with z_hi its mask's bits 8..11; terms without such bits add one constant.
// With flip, D_g(l ^ x_g) instead: (l ^ x) & z has the parity of l & z plus
// that of x & z, a factor per term.
template <typename V>
__device__ __forceinline__ void group_Dr(const PauliSmem<V> &S, int g, uint32_t tid, bool flip, V (&D)[PPER]) {
    using T = RT<V>;
    T re0 = 0, im0 = 0;
#pragma unroll
    for (int r = 0; r < PPER; ++r) D[r] = mkc<V>(0, 0);
    const uint32_t xl = S.P.gx[g];
    for (int j = S.P.gfirst[g]; j < S.P.gfirst[g + 1]; ++j) {
        const uint32_t z = S.P.zl[j];
        T cr = S.cre[j], ci = S.cim[j];
        uint32_t par = __popc(tid & z & 0xFFu);
        if (flip) par += __popc(xl & z);
        if (par & 1u) {
            cr = -cr;
            ci = -ci;
        }
        const uint32_t zr = z >> 8;
        if (zr == 0) {
            re0 += cr;
            im0 += ci;
        } else {
#pragma unroll
            for (int r = 0; r < PPER; ++r) {
                const bool neg = __popc((uint32_t)r & zr) & 1;
                D[r].x += neg ? -cr : cr;
                D[r].y += neg ? -ci : ci;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < PPER; ++r) {
        D[r].x += re0;
        D[r].y += im0;
    }
}

// Local index l = r * 256 + tid: bits 0..3 are qubits 0..3 (16 consecutive
// amplitudes, one 128-byte run for complex64), bits 4..11 Q's high qubits.
__device__ __forceinline__ uint64_t global_of(const uint64_t *hoff, uint64_t origin, uint32_t l) {
    return origin | hoff[l >> 4] | (l & 15u);
}

template <typename V>
__global__ void __launch_bounds__(PTHR) k_pauli_tile_expval(const V *__restrict__ psi, const PauliTileDesc Pg,
                                                            double *__restrict__ partials) {
    __shared__ PauliSmem<V> S;
    __shared__ double sh[PTHR / 32];
    extern __shared__ __align__(16) unsigned char pt_dyn[];
    V *tile = reinterpret_cast<V *>(pt_dyn);  // PTS amplitudes
    setup<V>(S, Pg);
    const uint32_t tid = threadIdx.x;
    const uint64_t n_tiles = (uint64_t)1 << (S.P.n - PK);
    KSum<RT<V>> acc;
    for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const uint64_t origin = tile_origin(S.P, t);
        tile_coeffs<V>(S, origin, nullptr, 1.0);
#pragma unroll
        for (int r = 0; r < PPER; ++r) {
            const uint32_t l = r * PTHR + tid;
            tile[l] = psi[global_of(S.hoff, origin, l)];
        }
        __syncthreads();
        for (int g = 0; g < S.P.n_groups; ++g) {
            const uint32_t xl = S.P.gx[g];
            V D[PPER];
            group_Dr<V>(S, g, tid, false, D);
            RT<V> part = 0;
            if (xl == 0) {
#pragma unroll
                for (int r = 0; r < PPER; ++r) part = fma(norm2(tile[r * PTHR + tid]), D[r].x, part);
            } else {
#pragma unroll
                for (int r = 0; r < PPER; ++r) {
                    const uint32_t l = r * PTHR + tid;
                    const V a = tile[l], ap = tile[l ^ xl];
                    const RT<V> ur = re_cdot(ap, a), ui = im_cdot(ap, a);  // conj(psi_{b^x}) psi_b
                    part = fma(ur, D[r].x, fma(-ui, D[r].y, part));
                }
            }
            acc.add(part);
        }
        __syncthreads();
    }
    const double tot = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

template <typename V>
__global__ void __launch_bounds__(PTHR) k_pauli_tile_apply(const V *__restrict__ psi, V *__restrict__ out,
                                                           const PauliTileDesc Pg, const double *__restrict__ weights,
                                                           double scale) {
    __shared__ PauliSmem<V> S;
    extern __shared__ __align__(16) unsigned char pt_dyn[];
    V *tile = reinterpret_cast<V *>(pt_dyn);  // PTS amplitudes
    setup<V>(S, Pg);
    const uint32_t tid = threadIdx.x;
    const uint64_t n_tiles = (uint64_t)1 << (S.P.n - PK);
    for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const uint64_t origin = tile_origin(S.P, t);
        tile_coeffs<V>(S, origin, weights, scale);
#pragma unroll
        for (int r = 0; r < PPER; ++r) {
            const uint32_t l = r * PTHR + tid;
            tile[l] = psi[global_of(S.hoff, origin, l)];
        }
        __syncthreads();
        V o[PPER];
#pragma unroll
        for (int r = 0; r < PPER; ++r) o[r] = mkc<V>(0, 0);
        for (int g = 0; g < S.P.n_groups; ++g) {
            const uint32_t xl = S.P.gx[g];
            V D[PPER];
            group_Dr<V>(S, g, tid, true, D);
#pragma unroll
            for (int r = 0; r < PPER; ++r) o[r] = cfma(D[r], tile[(r * PTHR + tid) ^ xl], o[r]);
        }
#pragma unroll
        for (int r = 0; r < PPER; ++r) {
            const uint64_t b = global_of(S.hoff, origin, r * PTHR + tid);
            if (S.P.accumulate) o[r] = cadd(o[r], out[b]);
            out[b] = o[r];
        }
        __syncthreads();
    }
}

// ---------------------------------------- complex64: streamed, double-buffered
// The same sums for complex64 states, built for bandwidth.  Each block keeps
// two tile buffers: while one tile is evaluated, the next one arrives by
// cp.async (16-byte copies, 8 per thread).  In a tile a thread owns local
// indices l = r * 256 + tid (r = 0..15: local bits 8..11).  A term's sign
// (-1)^{|b & z|} splits into the tile origin's parity (per tile and term,
// from the term's z bits outside Q written as tile-index bits), the thread's
// (local bits 0..7) and the register index's, (-1)^{|r & zr|} with zr the
// term's local bits 8..11.  The host sorts every group's terms by zr, so a
// group's per-r factor D(r) = sum_j C_j (-1)^{|r & zr_j|} is a 16-point
// Walsh-Hadamard transform of the coefficients gathered by zr (and, the
// other way round, E needs the transform of the per-r products at the
// terms' zr), with every array index fixed at compile time.
//
// E also reads the tile in two more layouts.  Layout L keeps local bits
// 8..11 (L = 0, the one above), 4..7 (L = 1) or 0..3 (L = 2) in a thread's
// registers.  A group of X strings alone (no term has a z bit) whose x mask
// lies inside one layout's register bits then pairs registers of the same
// thread: its share of E is sum_j c_j * sum_b Re(conj(psi_{b^x}) psi_b), each
// pair once and doubled, with no sign, no shared-memory partner and no
// per-term work in the tile loop.  Taken for x masks of one qubit (X_i terms,
// the transverse fields of spin models); wider X strings stay in the loop over
// groups (their sixteen register cases would not fit the registers).
//
// Terms of a group with the same local z mask have the same sign at every
// local index: their coefficients, signed by the tile origin, are summed per
// tile into one class coefficient, and the E kernel's loops over a group run
// over its classes (the H psi kernel keeps one coefficient per term: its
// per-tile class sums would sit on the tile's critical path).
struct Pauli2Desc {
    PauliTileDesc P;                       // terms of each group sorted by local z mask
    uint16_t zfirst[PT_MAXG][17];          // classes of group g with zr == m: [zfirst[g][m], zfirst[g][m + 1])
    uint16_t tzfirst[PT_MAXG][17];         // terms of group g with zr == m (the H psi kernel works per term)
    uint16_t gcls[PT_MAXG + 1];            // classes of group g: [gcls[g], gcls[g + 1])
    uint16_t cfirst[PT_MAXT + 1];          // terms of class c: [cfirst[c], cfirst[c + 1])
    uint16_t czl[PT_MAXT];                 // local z mask of class c
    int n_cls;
    uint32_t real_groups;                  // bit g: every coefficient of group g is real
    uint32_t xonly;                        // bit g: group g is an X-only group of one layout (E only)
    uint8_t xfirst[4];                     // layout L's X-only groups: entries [xfirst[L], xfirst[L + 1])
    uint8_t xreg[PT_MAXG];                 // an entry's qubit: its bit on the layout's register index (0..3)
    float xcoef[PT_MAXG];                  // an entry's sum of coefficients
};

struct Pauli2Smem {
    Pauli2Desc D;
    uint64_t hoff[256];
    uint64_t tz[PT_MAXT];                  // z bits outside Q as tile-index bits
    float2 ce[PT_MAXT];                    // this tile's class coefficients (weights, scale, origin sign)
    float2 cw[PT_MAXT];                    // coefficients with weights and scale
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Unnormalised 16-point Walsh-Hadamard transform in place:
// v[m] <- sum_r v[r] (-1)^{|m & r|}.
template <typename T> __device__ __forceinline__ void wht16(T (&v)[16]) {
#pragma unroll
    for (int h = 1; h < 16; h <<= 1)
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (!(i & h)) {
                const T a = v[i], b = v[i | h];
                v[i] = a + b;
                v[i | h] = a - b;
            }
}

__device__ __forceinline__ void p2_setup(Pauli2Smem &S, const Pauli2Desc &Dg, const double *weights, double scale) {
    copy_in(&S.D, &Dg, sizeof(Pauli2Desc));
    __syncthreads();
    const PauliTileDesc &P = S.D.P;
    for (int h = threadIdx.x; h < 256; h += blockDim.x) {
        uint64_t o = 0;
        for (int i = 0; i < 8; ++i) o |= (uint64_t)((h >> i) & 1) << P.hi[i];
        S.hoff[h] = o;
    }
    for (int j = threadIdx.x; j < P.n_terms; j += blockDim.x) {
        uint64_t t = 0;
        for (int i = 0; i < P.n - PK; ++i) t |= ((P.zo[j] >> P.out_q[i]) & 1ull) << i;
        S.tz[j] = t;
        double w = scale;
        if (weights) w *= weights[P.idx[j]];
        S.cw[j] = make_float2((float)(P.cre[j] * w), (float)(P.cim[j] * w));
    }
    __syncthreads();
}

// Tile t's global origin and cp.async copies into buf (this thread's 8 chunks
// of 2 amplitudes: local indices k * 512 + 2 * tid, k = 0..7).
__device__ __forceinline__ void p2_load(const Pauli2Smem &S, const float2 *__restrict__ psi, float2 *buf,
                                        uint64_t origin, uint32_t tid) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t l = (uint32_t)k * 512u + 2u * tid;
        cp_async16(smem_u32(buf + l), psi + (origin | S.hoff[l >> 4] | (l & 15u)));
    }
}

// Tile t's term coefficients: weights, scale and the origin's sign, one
// thread per term (the H psi kernel).
__device__ __forceinline__ void p2_coeffs_terms(Pauli2Smem &S, uint64_t t) {
    for (int j = threadIdx.x; j < S.D.P.n_terms; j += blockDim.x) {
        const float2 c = S.cw[j];
        S.ce[j] = (__popcll(t & S.tz[j]) & 1) ? make_float2(-c.x, -c.y) : c;
    }
}

// Tile t's class coefficients: the class's terms with weights, scale and
// the origin's sign.
__device__ __forceinline__ void p2_coeffs(Pauli2Smem &S, uint64_t t) {
    for (int c = threadIdx.x; c < S.D.n_cls; c += blockDim.x) {
        float2 e = make_float2(0.f, 0.f);
        for (int j = S.D.cfirst[c]; j < S.D.cfirst[c + 1]; ++j) {
            const float2 w = S.cw[j];
            if (__popcll(t & S.tz[j]) & 1) {
                e.x -= w.x;
                e.y -= w.y;
            } else {
                e.x += w.x;
                e.y += w.y;
            }
        }
        S.ce[c] = e;
    }
}

template <int P> struct XI { static constexpr int value = P; };
// The partner of register r in a group with x bits xr on the register index
// is row r ^ xr.  Masks of at most one bit (all that single-qubit x strings
// give) become compile-time constants, so each partner load has a constant
// offset; other masks take the row index at run time (XI<-1>).
template <typename F> __device__ __forceinline__ void with_xr(uint32_t x, F &&f) {
    switch (x) {
    case 0: f(XI<0>{}); break;
    case 1: f(XI<1>{}); break;
    case 2: f(XI<2>{}); break;
    case 4: f(XI<4>{}); break;
    case 8: f(XI<8>{}); break;
    default: f(XI<-1>{}); break;
    }
}
template <int XR> __device__ __forceinline__ uint32_t prow(int r, uint32_t xr) {
    return XR >= 0 ? (uint32_t)(r ^ XR) : ((uint32_t)r ^ xr);
}

// Tile origins from three tables of 256 entries (tile-index bits 0..7,
// 8..15, 16..23 scattered onto the qubits outside Q).
struct P2Origin {
    uint64_t t[3][256];
};
__device__ __forceinline__ void p2_origin_tables(P2Origin &O, const PauliTileDesc &P) {
    for (int i = threadIdx.x; i < 3 * 256; i += blockDim.x) {
        const int k = i >> 8, v = i & 255;
        uint64_t g = 0;
        for (int b = 0; b < 8; ++b) {
            const int bit = 8 * k + b;
            if (bit < P.n - PK && ((v >> b) & 1)) g |= 1ull << P.out_q[bit];
        }
        O.t[k][v] = g;
    }
}
__device__ __forceinline__ uint64_t p2_origin_t(const P2Origin &O, uint64_t t) {
    return O.t[0][t & 255] | O.t[1][(t >> 8) & 255] | O.t[2][(t >> 16) & 255];
}

// sum_r Re(conj(a[r ^ XR]) a[r]) over the 16 registers: each pair {r, r ^ XR}
// once (r without XR's highest bit), doubled; two accumulators.
template <int XR> __device__ __forceinline__ float pair_dot(const float2 (&a)[PPER]) {
    constexpr int TOP = XR >= 8 ? 8 : XR >= 4 ? 4 : XR >= 2 ? 2 : 1;
    float2 s[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    int c = 0;
#pragma unroll
    for (int r = 0; r < PPER; ++r)
        if (!(r & TOP)) {
            s[c & 1] = f2_fma(a[r ^ XR], a[r], s[c & 1]);
            ++c;
        }
    return 2.f * ((s[0].x + s[1].x) + (s[0].y + s[1].y));
}
// E over the tiles of one launch (complex64).
__global__ void __launch_bounds__(PTHR, 2) k_pauli2_expval(const float2 *__restrict__ psi, const Pauli2Desc Dg,
                                                           double *__restrict__ partials) {
    __shared__ Pauli2Smem S;
    __shared__ P2Origin O;
    __shared__ double sh[PTHR / 32];
    extern __shared__ __align__(16) unsigned char pt_dyn[];
    float2 *bufs = reinterpret_cast<float2 *>(pt_dyn);  // 2 x PTS amplitudes
    p2_origin_tables(O, Dg.P);
    p2_setup(S, Dg, nullptr, 1.0);
    const PauliTileDesc &P = S.D.P;
    const uint32_t tid = threadIdx.x;
    const uint64_t n_tiles = (uint64_t)1 << (P.n - PK);
    // this thread's sign of every term (local bits 0..7 = thread bits)
    uint64_t tpar = 0;
    for (int c = 0; c < S.D.n_cls; ++c) tpar |= (uint64_t)(__popc(tid & S.D.czl[c] & 0xFFu) & 1) << c;
    uint64_t t = blockIdx.x;
    if (t < n_tiles) p2_load(S, psi, bufs, p2_origin_t(O, t), tid);
    cp_async_commit();
    double acc = 0;
    for (int cur = 0; t < n_tiles; t += gridDim.x, cur ^= 1) {
        const uint64_t tn = t + gridDim.x;
        if (tn < n_tiles) p2_load(S, psi, bufs + (cur ^ 1) * PTS, p2_origin_t(O, tn), tid);
        cp_async_commit();
        p2_coeffs(S, t);
        cp_async_wait1();
        __syncthreads();
        const float2 *tile = bufs + cur * PTS;
        float2 a[PPER];
        float part = 0.f;
        // X-only groups, layout by layout, layout 0 last (the loop over the
        // other groups below reads it too): layout 1 holds
        // l = (tid / 16) * 256 + r * 16 + tid % 16, layout 2
        // l = tid * 16 + (r ^ (tid % 16)) (the XOR spreads a half-warp's
        // loads over the banks; the pairs r, r ^ x are the same either way)
#pragma unroll
        for (int L = 2; L >= 0; --L) {
            const int i0 = S.D.xfirst[L], i1 = S.D.xfirst[L + 1];
            if (L > 0 && i0 == i1) continue;
#pragma unroll
            for (int r = 0; r < PPER; ++r)
                a[r] = tile[L == 0   ? (uint32_t)r * PTHR + tid
                            : L == 1 ? ((tid >> 4) << 8) | ((uint32_t)r << 4) | (tid & 15u)
                                     : (tid << 4) | ((uint32_t)r ^ (tid & 15u))];
            if (i0 == i1) continue;
            // the four one-qubit pair sums of this layout, then each group's
            const float d0 = pair_dot<1>(a), d1 = pair_dot<2>(a), d2 = pair_dot<4>(a), d3 = pair_dot<8>(a);
            for (int i = i0; i < i1; ++i) {
                const int k = S.D.xreg[i];
                part = fmaf(S.D.xcoef[i], k == 0 ? d0 : k == 1 ? d1 : k == 2 ? d2 : d3, part);
            }
        }
        for (int g = 0; g < P.n_groups; ++g) {
            if ((S.D.xonly >> g) & 1u) continue;  // below, in its layout
            const uint32_t xl = P.gx[g];
            const uint16_t *zf = S.D.zfirst[g];
            const int j0 = S.D.gcls[g], j1 = S.D.gcls[g + 1];
            const bool real = (S.D.real_groups >> g) & 1u;
            const bool any_zr = zf[16] > zf[1];
            // u_r = conj(psi_{l ^ x}) psi_l, l = r * 256 + tid; the partner
            // sits at register index r ^ xr of thread tid ^ xt (this
            // thread's own registers when xt = 0)
            const float2 *pt = tile + (tid ^ (xl & 0xFFu));
            const uint32_t xr = xl >> 8;
            const bool own = (xl & 0xFFu) == 0;
            if (!any_zr) {
                // every term's factor is constant over r: one sum of u
                float sr, si = 0.f;
                // four independent accumulators (r mod 4) keep the FMA chains short
                float2 s2[4], t2[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) s2[q] = t2[q] = make_float2(0.f, 0.f);
                if (xl == 0) {
#pragma unroll
                    for (int r = 0; r < PPER; ++r) s2[r & 3] = f2_fma(a[r], a[r], s2[r & 3]);
                } else if (real && own && (xr == 1 || xr == 2 || xr == 4 || xr == 8)) {
                    // partner in the same thread: each pair once, doubled
                    with_xr(xr, [&](auto XR_) {
                        constexpr int XR = decltype(XR_)::value;
                        if constexpr (XR > 0) {
#pragma unroll
                            for (int r = 0; r < PPER; ++r)
                                if (!(r & XR)) s2[r & 3] = f2_fma(a[r ^ XR], a[r], s2[r & 3]);
                        }
                    });
#pragma unroll
                    for (int q = 0; q < 4; ++q) s2[q] = make_float2(2.f * s2[q].x, 2.f * s2[q].y);
                } else if (real) {
                    with_xr(xr, [&](auto XR_) {
                        constexpr int XR = decltype(XR_)::value;
#pragma unroll
                        for (int r = 0; r < PPER; ++r) s2[r & 3] = f2_fma(pt[prow<XR>(r, xr) * PTHR], a[r], s2[r & 3]);
                    });
                } else {
                    with_xr(xr, [&](auto XR_) {
                        constexpr int XR = decltype(XR_)::value;
#pragma unroll
                        for (int r = 0; r < PPER; ++r) {
                            const float2 b = pt[prow<XR>(r, xr) * PTHR];
                            s2[r & 3] = f2_fma(b, a[r], s2[r & 3]);                          // b.x a.x, b.y a.y
                            t2[r & 3] = f2_fma(b, make_float2(a[r].y, -a[r].x), t2[r & 3]);  // b.x a.y, -b.y a.x
                        }
                    });
                }
                sr = ((s2[0].x + s2[1].x) + (s2[2].x + s2[3].x)) + ((s2[0].y + s2[1].y) + (s2[2].y + s2[3].y));
                if (xl != 0 && !real)
                    si = ((t2[0].x + t2[1].x) + (t2[2].x + t2[3].x)) + ((t2[0].y + t2[1].y) + (t2[2].y + t2[3].y));
                for (int j = j0; j < j1; ++j) {
                    float2 c = S.ce[j];
                    if ((tpar >> j) & 1) c = make_float2(-c.x, -c.y);
                    part = fmaf(c.x, sr, fmaf(-c.y, si, part));
                }
            } else {
                float ur[PPER], ui[PPER];
                if (xl == 0) {
#pragma unroll
                    for (int r = 0; r < PPER; ++r) {
                        ur[r] = fmaf(a[r].x, a[r].x, a[r].y * a[r].y);
                        ui[r] = 0.f;
                    }
                } else {
                    with_xr(xr, [&](auto XR_) {
                        constexpr int XR = decltype(XR_)::value;
#pragma unroll
                        for (int r = 0; r < PPER; ++r) {
                            const float2 b = pt[prow<XR>(r, xr) * PTHR];
                            ur[r] = fmaf(b.x, a[r].x, b.y * a[r].y);
                            ui[r] = fmaf(b.x, a[r].y, -b.y * a[r].x);
                        }
                    });
                }
                wht16(ur);
                if (real) {
                    // real coefficients: only the real parts meet
#pragma unroll
                    for (int m = 0; m < 16; ++m)
                        for (int j = zf[m]; j < zf[m + 1]; ++j) {
                            const float cx = S.ce[j].x;
                            part = fmaf((tpar >> j) & 1 ? -cx : cx, ur[m], part);
                        }
                } else {
                    if (xl != 0) wht16(ui);
#pragma unroll
                    for (int m = 0; m < 16; ++m) {
                        for (int j = zf[m]; j < zf[m + 1]; ++j) {
                            float2 c = S.ce[j];
                            if ((tpar >> j) & 1) c = make_float2(-c.x, -c.y);
                            part = fmaf(c.x, ur[m], fmaf(-c.y, ui[m], part));
                        }
                    }
                }
            }
        }
        acc += (double)part;
        __syncthreads();
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// E of a launch whose groups are X-only groups of the three layouts (one-qubit
// X terms; the transverse-field part of a spin Hamiltonian) and at most one
// diagonal group with real coefficients (the Z strings).  Nothing in the
// X-only part depends on a coefficient or a sign, so each thread only sums,
// per layout L and register bit k, sum_r Re(conj(a[r ^ 2^k]) a[r]) over its
// tiles, and weighs the twelve sums once at the end.  The diagonal group takes
// the thread's probabilities in layout 0 through the 16-point transform
// (like the loop over groups of k_pauli2_expval) with its class coefficients
// signed per tile.  Few registers: three blocks per SM, each with two tile
// buffers.
struct PauliXDesc {
    int n;                 // qubits of the state
    uint32_t lmask;        // bit L: some group lies in layout L
    uint8_t hi[8];         // Q's qubits above qubit 3
    uint8_t out_q[32];     // qubits outside Q (tile index bit i -> qubit)
    float coef[3][4];      // weight of layout L's pair sum over register bit k (0: no group)
    // the diagonal group (DIAG kernels): its classes of equal local z mask
    int n_cls;
    uint32_t mmask;              // bit m: some class has register mask m
    uint16_t zfirst[17];         // classes with register mask m: [zfirst[m], zfirst[m + 1])
    uint16_t czl[PT_MAXT];       // local z mask of class c
    uint16_t cfirst[PT_MAXT + 1];  // terms of class c: [cfirst[c], cfirst[c + 1])
    uint64_t tz[PT_MAXT];        // a term's z bits outside Q, as tile-index bits
    float cw[PT_MAXT];           // a term's coefficient
};

struct PauliXSmem {
    uint64_t hoff[256];    // offsets of the values of Q's high qubits
    uint64_t otab[6][16];  // tile origin, four tile-index bits at a time
};

template <bool DIAG>
__global__ void __launch_bounds__(PTHR, 3) k_pauli2_xonly(const float2 *__restrict__ psi, const __grid_constant__ PauliXDesc D,
                                                          double *__restrict__ partials) {
    __shared__ PauliXSmem S;
    __shared__ double sh[PTHR / 32];
    __shared__ float ce[DIAG ? PT_MAXT : 1];  // the tile's class coefficients
    extern __shared__ __align__(16) unsigned char pt_dyn[];
    float2 *bufs = reinterpret_cast<float2 *>(pt_dyn);  // 2 x PTS amplitudes
    const uint32_t tid = threadIdx.x;
    const int nt = D.n - PK;
    for (int h = tid; h < 256; h += PTHR) {
        uint64_t o = 0;
        for (int i = 0; i < 8; ++i) o |= (uint64_t)((h >> i) & 1) << D.hi[i];
        S.hoff[h] = o;
    }
    for (int i = tid; i < 6 * 16; i += PTHR) {
        const int k = i >> 4, v = i & 15;
        uint64_t g = 0;
        for (int b = 0; b < 4; ++b)
            if (4 * k + b < nt && ((v >> b) & 1)) g |= 1ull << D.out_q[4 * k + b];
        S.otab[k][v] = g;
    }
    // this thread's sign of every class (local bits 0..7 = thread bits)
    uint64_t tpar = 0;
    if (DIAG)
        for (int c = 0; c < D.n_cls; ++c) tpar |= (uint64_t)(__popc(tid & D.czl[c] & 0xFFu) & 1) << c;
    __syncthreads();
    auto origin = [&](uint64_t t) {
        uint64_t g = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) g |= S.otab[k][(t >> (4 * k)) & 15u];
        return g;
    };
    // this thread's 8 copies of 2 amplitudes: local indices k * 512 + 2 * tid
    auto load = [&](float2 *buf, uint64_t o) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t l = (uint32_t)k * 512u + 2u * tid;
            cp_async16(smem_u32(buf + l), psi + (o | S.hoff[l >> 4] | (l & 15u)));
        }
    };
    const uint64_t n_tiles = (uint64_t)1 << nt;
    uint64_t t = blockIdx.x;
    if (t < n_tiles) load(bufs, origin(t));
    cp_async_commit();
    float acc[3][4];
#pragma unroll
    for (int L = 0; L < 3; ++L)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[L][k] = 0.f;
    float dacc = 0.f;  // the diagonal group's share
    for (int cur = 0; t < n_tiles; t += gridDim.x, cur ^= 1) {
        const uint64_t tn = t + gridDim.x;
        if (tn < n_tiles) load(bufs + (cur ^ 1) * PTS, origin(tn));
        cp_async_commit();
        if (DIAG)
            // tile t's class coefficients: the class's terms signed by the origin
            for (int c = tid; c < D.n_cls; c += PTHR) {
                float e = 0.f;
                for (int j = D.cfirst[c]; j < D.cfirst[c + 1]; ++j)
                    e += (__popcll(t & D.tz[j]) & 1) ? -D.cw[j] : D.cw[j];
                ce[c] = e;
            }
        cp_async_wait1();
        __syncthreads();
        const float2 *tile = bufs + cur * PTS;
#pragma unroll
        for (int L = 2; L >= 0; --L) {
            if ((DIAG && L == 0) || ((D.lmask >> L) & 1u)) {
                float2 a[PPER];
#pragma unroll
                for (int r = 0; r < PPER; ++r)
                    a[r] = tile[L == 0   ? (uint32_t)r * PTHR + tid
                                : L == 1 ? ((tid >> 4) << 8) | ((uint32_t)r << 4) | (tid & 15u)
                                         : (tid << 4) | ((uint32_t)r ^ (tid & 15u))];
                if ((D.lmask >> L) & 1u) {
                    acc[L][0] += pair_dot<1>(a);
                    acc[L][1] += pair_dot<2>(a);
                    acc[L][2] += pair_dot<4>(a);
                    acc[L][3] += pair_dot<8>(a);
                }
                if (DIAG && L == 0) {
                    // probabilities at l = r * 256 + tid, transformed over r
                    float u[PPER];
#pragma unroll
                    for (int r = 0; r < PPER; ++r) u[r] = fmaf(a[r].x, a[r].x, a[r].y * a[r].y);
                    wht16(u);
                    float part = 0.f;
#pragma unroll
                    for (int m = 0; m < 16; ++m) {
                        if (!((D.mmask >> m) & 1u)) continue;
                        float cm = 0.f;
                        for (int c = D.zfirst[m]; c < D.zfirst[m + 1]; ++c)
                            cm += ((tpar >> c) & 1) ? -ce[c] : ce[c];
                        part = fmaf(cm, u[m], part);
                    }
                    dacc += part;
                }
            }
        }
        __syncthreads();
    }
    double part = (double)dacc;
#pragma unroll
    for (int L = 0; L < 3; ++L)
#pragma unroll
        for (int k = 0; k < 4; ++k) part += (double)D.coef[L][k] * (double)acc[L][k];
    const double tot = block_sum(part, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// out (+)= scale * sum_j w_j c_j P_j psi over the launch's groups (complex64):
// out_b += D_x(b ^ x) psi_{b ^ x} per group.
// eparts (may be null): the launch completes the output, and each block also
// writes its share of Re <psi|out> (the expectation value when out = H psi).
__global__ void __launch_bounds__(PTHR, 2) k_pauli2_apply(const float2 *__restrict__ psi, float2 *__restrict__ out,
                                                          const Pauli2Desc Dg, const double *__restrict__ weights,
                                                          double scale, int accumulate, double *__restrict__ eparts) {
    __shared__ Pauli2Smem S;
    __shared__ P2Origin O;
    __shared__ double sh[PTHR / 32];
    double eacc = 0;
    extern __shared__ __align__(16) unsigned char pt_dyn[];
    float2 *bufs = reinterpret_cast<float2 *>(pt_dyn);
    p2_origin_tables(O, Dg.P);
    p2_setup(S, Dg, weights, scale);
    const PauliTileDesc &P = S.D.P;
    const uint32_t tid = threadIdx.x;
    const uint64_t n_tiles = (uint64_t)1 << (P.n - PK);
    // sign of every term at the partner's local index l ^ x: thread bits of
    // (tid ^ x) and the register part x's own parity (group's x)
    uint64_t tpar = 0;
    for (int g = 0; g < P.n_groups; ++g)
        for (int j = P.gfirst[g]; j < P.gfirst[g + 1]; ++j) {
            const uint32_t z = P.zl[j];
            const int par = (__popc((tid ^ P.gx[g]) & z & 0xFFu) + __popc((P.gx[g] >> 8) & (z >> 8))) & 1;
            tpar |= (uint64_t)par << j;
        }
    uint64_t t = blockIdx.x;
    if (t < n_tiles) p2_load(S, psi, bufs, p2_origin_t(O, t), tid);
    cp_async_commit();
    for (int cur = 0; t < n_tiles; t += gridDim.x, cur ^= 1) {
        const uint64_t tn = t + gridDim.x;
        if (tn < n_tiles) p2_load(S, psi, bufs + (cur ^ 1) * PTS, p2_origin_t(O, tn), tid);
        cp_async_commit();
        const uint64_t origin = p2_origin_t(O, t);
        // this thread's outputs: 16 runs of 16 amplitudes, one per r
        const float2 *orow = out + (origin | (tid & 15u));
        float2 o[PPER];
        if (accumulate) {
#pragma unroll
            for (int r = 0; r < PPER; ++r) o[r] = orow[S.hoff[(r * PTHR + tid) >> 4]];
        } else {
#pragma unroll
            for (int r = 0; r < PPER; ++r) o[r] = make_float2(0.f, 0.f);
        }
        p2_coeffs_terms(S, t);
        cp_async_wait1();
        __syncthreads();
        const float2 *tile = bufs + cur * PTS;
        for (int g = 0; g < P.n_groups; ++g) {
            const uint32_t xl = P.gx[g];
            const uint16_t *zf = S.D.tzfirst[g];
            const int j0 = P.gfirst[g], j1 = P.gfirst[g + 1];
            const bool real = (S.D.real_groups >> g) & 1u;
            const float2 *pt = tile + (tid ^ (xl & 0xFFu));
            const uint32_t xr = xl >> 8;
            if (zf[16] <= zf[1]) {
                // D constant over r: the sum of the group's signed coefficients
                float dr = 0.f, di = 0.f;
                for (int j = j0; j < j1; ++j) {
                    float2 c = S.ce[j];
                    if ((tpar >> j) & 1) c = make_float2(-c.x, -c.y);
                    dr += c.x;
                    di += c.y;
                }
                const float2 d2 = make_float2(dr, dr);
                if (real) {
                    with_xr(xr, [&](auto XR_) {
                        constexpr int XR = decltype(XR_)::value;
#pragma unroll
                        for (int r = 0; r < PPER; ++r) o[r] = f2_fma(d2, pt[prow<XR>(r, xr) * PTHR], o[r]);
                    });
                } else {
                    const float2 e2 = make_float2(-di, di);
                    with_xr(xr, [&](auto XR_) {
                        constexpr int XR = decltype(XR_)::value;
#pragma unroll
                        for (int r = 0; r < PPER; ++r) {
                            const float2 b = pt[prow<XR>(r, xr) * PTHR];
                            o[r] = f2_fma(d2, b, f2_fma(e2, make_float2(b.y, b.x), o[r]));
                        }
                    });
                }
                continue;
            }
            // A_m = sum of the group's coefficients with zr == m (signed for
            // this thread and tile), D(r ^ xr) = its transform at r
            float dr[PPER], di[PPER];
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                float sr = 0.f, si = 0.f;
                for (int j = zf[m]; j < zf[m + 1]; ++j) {
                    float2 c = S.ce[j];
                    if ((tpar >> j) & 1) c = make_float2(-c.x, -c.y);
                    sr += c.x;
                    si += c.y;
                }
                dr[m] = sr;
                di[m] = si;
            }
            wht16(dr);
            if (real) {
                with_xr(xr, [&](auto XR_) {
                    constexpr int XR = decltype(XR_)::value;
#pragma unroll
                    for (int r = 0; r < PPER; ++r)
                        o[r] = f2_fma(make_float2(dr[r], dr[r]), pt[prow<XR>(r, xr) * PTHR], o[r]);
                });
            } else {
                wht16(di);
                with_xr(xr, [&](auto XR_) {
                    constexpr int XR = decltype(XR_)::value;
#pragma unroll
                    for (int r = 0; r < PPER; ++r) {
                        const float2 b = pt[prow<XR>(r, xr) * PTHR];
                        o[r] = f2_fma(make_float2(dr[r], dr[r]), b,
                                      f2_fma(make_float2(-di[r], di[r]), make_float2(b.y, b.x), o[r]));
                    }
                });
            }
        }
        float2 *wrow = out + (origin | (tid & 15u));
#pragma unroll
        for (int r = 0; r < PPER; ++r) wrow[S.hoff[(r * PTHR + tid) >> 4]] = o[r];
        if (eparts) {
            float2 e2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < PPER; ++r) e2 = f2_fma(tile[r * PTHR + tid], o[r], e2);  // Re(conj(psi) out)
            eacc += (double)e2.x + (double)e2.y;
        }
        __syncthreads();
    }
    if (eparts) {
        const double tot = block_sum(eacc, sh);
        if (threadIdx.x == 0) eparts[blockIdx.x] = tot;
    }
}

// ------------------------------------------------------------------ host
int high_count(uint64_t x) { return __builtin_popcountll(x >> 4); }

// complex64: 2 blocks per SM (two 32 KiB tile buffers and 128 registers a
// thread each); complex128: 4.
int tile_grid_pauli(int n, int dtype) {
    const uint64_t tiles = (uint64_t)1 << (n - PK);
    uint64_t g = (uint64_t)device_sm_count() * (dtype == TQD_C64 ? 2 : 4);
    return (int)std::min<uint64_t>(g, tiles);
}

// The complex64 kernels' descriptor: each group's terms sorted by their local
// z mask (so by its bits on the register index, local bits 8..11, first),
// runs of equal masks as classes, the range of classes of each register mask.
Pauli2Desc make_pauli2(const PauliTileDesc &src) {
    Pauli2Desc d;
    memset(&d, 0, sizeof(d));
    d.P = src;
    for (int g = 0; g < src.n_groups; ++g) {
        const int a = src.gfirst[g], b = src.gfirst[g + 1];
        std::vector<int> ord;
        for (int j = a; j < b; ++j) ord.push_back(j);
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return src.zl[x] < src.zl[y]; });
        for (int k = 0; k < b - a; ++k) {
            const int j = ord[k], t = a + k;
            d.P.zl[t] = src.zl[j];
            d.P.zo[t] = src.zo[j];
            d.P.cre[t] = src.cre[j];
            d.P.cim[t] = src.cim[j];
            d.P.idx[t] = src.idx[j];
        }
        bool real = true;
        for (int j = a; j < b; ++j) real = real && d.P.cim[j] == 0.0;
        if (real) d.real_groups |= 1u << g;
        d.gcls[g] = (uint16_t)d.n_cls;
        for (int j = a; j < b; ++j)
            if (j == a || d.P.zl[j] != d.P.zl[j - 1]) {
                d.czl[d.n_cls] = d.P.zl[j];
                d.cfirst[d.n_cls++] = (uint16_t)j;
            }
        d.gcls[g + 1] = (uint16_t)d.n_cls;
        d.cfirst[d.n_cls] = (uint16_t)b;
        int kt = a;
        for (int m = 0; m <= 16; ++m) {
            while (m < 16 && kt < b && (d.P.zl[kt] >> 8) < m) ++kt;
            d.tzfirst[g][m] = (uint16_t)(m == 16 ? b : kt);
        }
        int k = d.gcls[g];
        for (int m = 0; m <= 16; ++m) {
            while (m < 16 && k < d.gcls[g + 1] && (d.czl[k] >> 8) < m) ++k;
            d.zfirst[g][m] = (uint16_t)(m == 16 ? d.gcls[g + 1] : k);
        }
    }
    // X-only groups and their layouts
    int per[3][PT_MAXG], cnt[3] = {0, 0, 0};
    for (int g = 0; g < src.n_groups; ++g) {
        const uint32_t x = src.gx[g];
        bool xo = x != 0;
        for (int j = src.gfirst[g]; j < src.gfirst[g + 1] && xo; ++j)
            xo = d.P.zl[j] == 0 && d.P.zo[j] == 0 && d.P.cim[j] == 0.0;
        if (!xo) continue;
        const int L = (x & 0xF00u) == x ? 0 : (x & 0xF0u) == x ? 1 : (x & 0xFu) == x ? 2 : -1;
        if (L < 0 || __builtin_popcount(x) != 1) continue;
        per[L][cnt[L]++] = g;
        d.xonly |= 1u << g;
    }
    int e = 0;
    for (int L = 0; L < 3; ++L) {
        d.xfirst[L] = (uint8_t)e;
        for (int i = 0; i < cnt[L]; ++i, ++e) {
            const int g = per[L][i];
            double c = 0.0;
            for (int j = src.gfirst[g]; j < src.gfirst[g + 1]; ++j) c += d.P.cre[j];
            d.xreg[e] = (uint8_t)__builtin_ctz((src.gx[g] >> (L == 0 ? 8 : L == 1 ? 4 : 0)) & 15u);
            d.xcoef[e] = (float)c;
        }
    }
    d.xfirst[3] = (uint8_t)e;
    return d;
}

// The staged tile is dynamic shared memory (64 KiB for complex128).
template <typename K> void allow_tile_smem(K kernel, size_t bytes) {
    static std::once_flag once;
    std::call_once(once, [&] { cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); });
}

}  // namespace

std::vector<PauliTileDesc> plan_pauli_tiles(const std::vector<PauliGroup> &groups, int n,
                                            std::vector<int> *leftover) {
    leftover->clear();
    std::vector<PauliTileDesc> out;
    if (n < PK) {
        for (int g = 0; g < (int)groups.size(); ++g) leftover->push_back(g);
        return out;
    }
    // layouts: sets of at most 8 qubits above qubit 3; groups placed greedily,
    // the widest first
    std::vector<int> order;
    for (int g = 0; g < (int)groups.size(); ++g) {
        if (high_count(groups[g].xmask) > 8 || (groups[g].xmask >> n) != 0) leftover->push_back(g);
        else order.push_back(g);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return high_count(groups[a].xmask) > high_count(groups[b].xmask);
    });
    // Groups with x bits above qubit 3 go to the first set they fit in; those
    // without (the diagonal group, X/Y on qubits 0..3), which fit in any set
    // and come last in this order, go to the set with the least work so far
    // (16 per group, the Walsh-Hadamard transform, plus 1 per term), so that
    // the launches carry similar work.
    std::vector<uint64_t> sets;
    std::vector<std::vector<int>> members;
    std::vector<size_t> work;
    for (int g : order) {
        const uint64_t h = groups[g].xmask & ~(uint64_t)15;
        int placed = -1;
        if (h == 0) {
            for (size_t s = 0; s < sets.size(); ++s)
                if (placed < 0 || work[s] < work[placed]) placed = (int)s;
        } else {
            for (size_t s = 0; s < sets.size() && placed < 0; ++s)
                if (__builtin_popcountll(sets[s] | h) <= 8) placed = (int)s;
        }
        if (placed < 0) {
            sets.push_back(0);
            members.emplace_back();
            work.push_back(0);
            placed = (int)sets.size() - 1;
        }
        sets[placed] |= h;
        members[placed].push_back(g);
        work[placed] += 16 + groups[g].terms.size();
    }
    for (size_t s = 0; s < sets.size(); ++s) {
        // pad Q with unused qubits up to 8 high qubits
        uint64_t q = sets[s];
        for (int b = 4; b < n && __builtin_popcountll(q) < 8; ++b) q |= (uint64_t)1 << b;
        int hi[8], nh = 0, outq[64], no = 0;
        for (int b = 4; b < n; ++b) {
            if ((q >> b) & 1) hi[nh++] = b;
            else outq[no++] = b;
        }
        // local bit of each qubit in Q
        int local[64];
        for (int b = 0; b < 64; ++b) local[b] = -1;
        for (int b = 0; b < 4; ++b) local[b] = b;
        for (int i = 0; i < 8; ++i) local[hi[i]] = 4 + i;
        auto to_local = [&](uint64_t m) {
            uint32_t l = 0;
            for (int b = 0; b < n; ++b)
                if (((m >> b) & 1) && local[b] >= 0) l |= 1u << local[b];
            return l;
        };
        // split into launches of at most PT_MAXG groups and PT_MAXT terms
        PauliTileDesc d;
        auto fresh = [&]() {
            memset(&d, 0, sizeof(d));
            d.n = n;
            for (int i = 0; i < 8; ++i) d.hi[i] = (uint8_t)hi[i];
            for (int i = 0; i < no; ++i) d.out_q[i] = (uint8_t)outq[i];
        };
        fresh();
        for (int g : members[s]) {
            const PauliGroup &G = groups[g];
            for (size_t from = 0; from < G.terms.size();) {
                if (d.n_groups == PT_MAXG || d.n_terms == PT_MAXT) {
                    out.push_back(d);
                    fresh();
                }
                const size_t cnt = std::min<size_t>(G.terms.size() - from, PT_MAXT - d.n_terms);
                d.gx[d.n_groups] = (uint16_t)to_local(G.xmask);
                d.gfirst[d.n_groups] = (uint16_t)d.n_terms;
                for (size_t k = 0; k < cnt; ++k) {
                    const TermDev &t = G.terms[from + k];
                    const int j = d.n_terms++;
                    d.zl[j] = (uint16_t)to_local(t.zmask);
                    uint64_t zo = 0;
                    for (int b = 0; b < n; ++b)
                        if (((t.zmask >> b) & 1) && local[b] < 0) zo |= (uint64_t)1 << b;
                    d.zo[j] = zo;
                    d.cre[j] = t.pre * t.coeff;
                    d.cim[j] = t.pim * t.coeff;
                    d.idx[j] = t.index;
                }
                ++d.n_groups;
                d.gfirst[d.n_groups] = (uint16_t)d.n_terms;
                from += cnt;
            }
        }
        if (d.n_groups > 0) out.push_back(d);
    }
    return out;
}

// Blocks of the X-only launches (three per SM) and of the others (two).
static int xonly_grid(int n) {
    const uint64_t tiles = (uint64_t)1 << (n - PK);
    return (int)std::min<uint64_t>((uint64_t)device_sm_count() * 3, tiles);
}

static cudaError_t tile_expval_c64(const tqd_state *st, const std::vector<PauliTileDesc> &launches,
                                   double *partials, int pblk, cudaStream_t s) {
    const int grid = tile_grid_pauli(st->n, TQD_C64), xgrid = xonly_grid(st->n);
    const int width = std::max(grid, xgrid);  // partials summed per launch
    allow_tile_smem(k_pauli2_expval, 2 * PTS * sizeof(float2));
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_pauli2_xonly<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * PTS * (int)sizeof(float2));
        cudaFuncSetAttribute(k_pauli2_xonly<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * PTS * (int)sizeof(float2));
    });
    for (size_t i = 0; i < launches.size(); ++i) {
        const Pauli2Desc d = make_pauli2(launches[i]);
        double *row = partials + i * pblk;
        ProfScope ps(PK_EXPVAL, (double)((uint64_t)1 << st->n) * sizeof(float2), s);
        // every group X-only, or the diagonal group with real coefficients
        int diag = -1;
        bool lean = d.P.n_groups > 0;
        for (int g = 0; g < d.P.n_groups && lean; ++g) {
            if ((d.xonly >> g) & 1u) continue;
            if (d.P.gx[g] == 0 && ((d.real_groups >> g) & 1u) && diag < 0) diag = g;
            else lean = false;
        }
        int used;
        if (lean) {
            PauliXDesc x;
            memset(&x, 0, sizeof(x));
            x.n = d.P.n;
            memcpy(x.hi, d.P.hi, sizeof(x.hi));
            memcpy(x.out_q, d.P.out_q, sizeof(x.out_q));
            for (int L = 0; L < 3; ++L)
                for (int e = d.xfirst[L]; e < d.xfirst[L + 1]; ++e) {
                    x.coef[L][d.xreg[e]] += d.xcoef[e];
                    x.lmask |= 1u << L;
                }
            if (diag >= 0) {
                // the group's classes, renumbered from 0, and their terms
                const int c0 = d.gcls[diag], c1 = d.gcls[diag + 1], j0 = d.cfirst[c0];
                const int nt = d.P.n - PK;
                x.n_cls = c1 - c0;
                for (int c = c0; c < c1; ++c) {
                    x.czl[c - c0] = d.czl[c];
                    x.cfirst[c - c0] = (uint16_t)(d.cfirst[c] - j0);
                    x.mmask |= 1u << (d.czl[c] >> 8);
                }
                x.cfirst[c1 - c0] = (uint16_t)(d.cfirst[c1] - j0);
                for (int m = 0; m <= 16; ++m) x.zfirst[m] = (uint16_t)(d.zfirst[diag][m] - c0);
                for (int j = j0; j < d.cfirst[c1]; ++j) {
                    uint64_t tz = 0;
                    for (int b = 0; b < nt; ++b) tz |= ((d.P.zo[j] >> d.P.out_q[b]) & 1ull) << b;
                    x.tz[j - j0] = tz;
                    x.cw[j - j0] = (float)d.P.cre[j];
                }
                k_pauli2_xonly<true><<<xgrid, PTHR, 2 * PTS * sizeof(float2), s>>>((const float2 *)st->amps, x, row);
            } else {
                k_pauli2_xonly<false><<<xgrid, PTHR, 2 * PTS * sizeof(float2), s>>>((const float2 *)st->amps, x, row);
            }
            used = xgrid;
        } else {
            k_pauli2_expval<<<grid, PTHR, 2 * PTS * sizeof(float2), s>>>((const float2 *)st->amps, d, row);
            used = grid;
        }
        // the row's remaining entries count as zero
        if (used < width) {
            cudaError_t e = cudaMemsetAsync(row + used, 0, (size_t)(width - used) * sizeof(double), s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

template <typename V>
static cudaError_t tile_expval_t(const tqd_state *st, const std::vector<PauliTileDesc> &launches,
                                 double *partials, int pblk, cudaStream_t s) {
    const int grid = tile_grid_pauli(st->n, st->dtype);
    allow_tile_smem(k_pauli_tile_expval<V>, PTS * sizeof(V));
    for (size_t i = 0; i < launches.size(); ++i) {
        ProfScope ps(PK_EXPVAL, (double)((uint64_t)1 << st->n) * sizeof(V), s);
        k_pauli_tile_expval<V><<<grid, PTHR, PTS * sizeof(V), s>>>((const V *)st->amps, launches[i],
                                                                   partials + i * pblk);
    }
    return cudaGetLastError();
}

cudaError_t launch_pauli_tile_expval(const tqd_state *st, const std::vector<PauliTileDesc> &launches,
                                     double *partials, int pblk, cudaStream_t s) {
    if (st->dtype == TQD_C64) return tile_expval_c64(st, launches, partials, pblk, s);
    return tile_expval_t<double2>(st, launches, partials, pblk, s);
}

int pauli_tile_grid(int n, int dtype) { return tile_grid_pauli(n, dtype); }

int pauli_tile_expval_width(int n, int dtype) {
    return dtype == TQD_C64 ? std::max(tile_grid_pauli(n, dtype), xonly_grid(n)) : tile_grid_pauli(n, dtype);
}

static cudaError_t tile_apply_c64(const tqd_state *psi, const std::vector<PauliTileDesc> &launches,
                                  const double *weights, double scale, tqd_state *out, bool accumulate,
                                  double *eparts, cudaStream_t s) {
    const int grid = tile_grid_pauli(psi->n, TQD_C64);
    allow_tile_smem(k_pauli2_apply, 2 * PTS * sizeof(float2));
    const double N = (double)((uint64_t)1 << psi->n) * sizeof(float2);
    for (size_t i = 0; i < launches.size(); ++i) {
        const Pauli2Desc d = make_pauli2(launches[i]);
        const int acc = (accumulate || i > 0) ? 1 : 0;
        ProfScope ps(PK_APPLY_OBS, N * (acc ? 3 : 2), s);
        double *ep = i + 1 == launches.size() ? eparts : nullptr;
        k_pauli2_apply<<<grid, PTHR, 2 * PTS * sizeof(float2), s>>>((const float2 *)psi->amps, (float2 *)out->amps, d,
                                                                    weights, scale, acc, ep);
    }
    return cudaGetLastError();
}

template <typename V>
static cudaError_t tile_apply_t(const tqd_state *psi, const std::vector<PauliTileDesc> &launches,
                                const double *weights, double scale, tqd_state *out, bool accumulate,
                                cudaStream_t s) {
    const int grid = tile_grid_pauli(psi->n, psi->dtype);
    allow_tile_smem(k_pauli_tile_apply<V>, PTS * sizeof(V));
    const double N = (double)((uint64_t)1 << psi->n) * sizeof(V);
    for (size_t i = 0; i < launches.size(); ++i) {
        PauliTileDesc d = launches[i];
        d.accumulate = (accumulate || i > 0) ? 1 : 0;
        ProfScope ps(PK_APPLY_OBS, N * (d.accumulate ? 3 : 2), s);
        k_pauli_tile_apply<V><<<grid, PTHR, PTS * sizeof(V), s>>>((const V *)psi->amps, (V *)out->amps, d, weights,
                                                                  scale);
    }
    return cudaGetLastError();
}

cudaError_t launch_pauli_tile_apply(const tqd_state *psi, const std::vector<PauliTileDesc> &launches,
                                    const double *weights, double scale, tqd_state *out, bool accumulate,
                                    double *eparts, cudaStream_t s) {
    if (psi->dtype == TQD_C64) return tile_apply_c64(psi, launches, weights, scale, out, accumulate, eparts, s);
    return tile_apply_t<double2>(psi, launches, weights, scale, out, accumulate, s);
}

}  // namespace tqd
