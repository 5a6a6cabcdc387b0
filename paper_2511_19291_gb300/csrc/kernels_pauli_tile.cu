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

// ------------------------------------------------------------------ host
int high_count(uint64_t x) { return __builtin_popcountll(x >> 4); }

int tile_grid_pauli(int n) {
    const uint64_t tiles = (uint64_t)1 << (n - PK);
    uint64_t g = (uint64_t)device_sm_count() * 4;
    return (int)std::min<uint64_t>(g, tiles);
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
    std::vector<uint64_t> sets;
    std::vector<std::vector<int>> members;
    for (int g : order) {
        const uint64_t h = groups[g].xmask & ~(uint64_t)15;
        int placed = -1;
        for (size_t s = 0; s < sets.size() && placed < 0; ++s)
            if (__builtin_popcountll(sets[s] | h) <= 8) placed = (int)s;
        if (placed < 0) {
            sets.push_back(0);
            members.emplace_back();
            placed = (int)sets.size() - 1;
        }
        sets[placed] |= h;
        members[placed].push_back(g);
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

template <typename V>
static cudaError_t tile_expval_t(const tqd_state *st, const std::vector<PauliTileDesc> &launches,
                                 double *partials, int pblk, cudaStream_t s) {
    const int grid = tile_grid_pauli(st->n);
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
    if (st->dtype == TQD_C64) return tile_expval_t<float2>(st, launches, partials, pblk, s);
    return tile_expval_t<double2>(st, launches, partials, pblk, s);
}

int pauli_tile_grid(int n) { return tile_grid_pauli(n); }

template <typename V>
static cudaError_t tile_apply_t(const tqd_state *psi, const std::vector<PauliTileDesc> &launches,
                                const double *weights, double scale, tqd_state *out, bool accumulate,
                                cudaStream_t s) {
    const int grid = tile_grid_pauli(psi->n);
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
                                    cudaStream_t s) {
    if (psi->dtype == TQD_C64) return tile_apply_t<float2>(psi, launches, weights, scale, out, accumulate, s);
    return tile_apply_t<double2>(psi, launches, weights, scale, out, accumulate, s);
}

}  // namespace tqd
