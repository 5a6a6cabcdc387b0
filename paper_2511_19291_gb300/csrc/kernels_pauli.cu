// kernels_pauli.cu -- Pauli-sum expectation values and H psi.
//
// A term coeff * P with P = i^{|x&z|} X^x Z^z acts as
//   (P psi)_{b'} = i^{|x&z|} (-1)^{|(b' ^ x) & z|} psi_{b' ^ x},
// so <psi|P|psi> = sum_b conj(psi_{b^x}) i^{|x&z|} (-1)^{|b&z|} psi_b
// (measurement in the Z basis, Sec. 2.2.1, generalised to Pauli strings).
// Terms that share an x mask share one pass over the state: the pass reads
// each pair (b, b ^ x) once and evaluates D_x(b) = sum_j c_j (-1)^{|b & z_j|}.
// Reductions: per-thread Kahan-compensated sums in the state's precision,
// FP64 from the warp level on, per-block partials summed in a fixed order.
#include <algorithm>
#include <map>

#include "common.cuh"
#include "launch.h"
#include "pauli_tile.h"
#include "prof.h"

namespace tqd {

template <typename V> using RT = typename Real<V>::T;
constexpr int PT = 256;
constexpr int MAXT = 64;   // terms per launch
constexpr int MAXT1 = 8;   // terms per launch in per-term mode

struct TermPack {
    int nt;
    int pad;
    uint64_t x;
    uint64_t z[MAXT];
    double cre[MAXT];
    double cim[MAXT];
    int idx[MAXT];
};

std::vector<PauliGroup> group_terms(const tqd_pauli_term *terms, size_t n_terms) {
    std::map<uint64_t, size_t> where;
    std::vector<PauliGroup> groups;
    for (size_t j = 0; j < n_terms; ++j) {
        const uint64_t x = terms[j].xmask, z = terms[j].zmask;
        auto it = where.find(x);
        if (it == where.end()) {
            where[x] = groups.size();
            groups.push_back(PauliGroup{x, {}});
            it = where.find(x);
        }
        // i^{|x & z|}
        const int y = __builtin_popcountll(x & z) & 3;
        const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, 1, 0, -1};
        TermDev t;
        t.zmask = z;
        t.coeff = terms[j].coeff;
        t.pre = pr[y];
        t.pim = pi[y];
        t.index = (int)j;
        t.pad = 0;
        groups[it->second].terms.push_back(t);
    }
    return groups;
}

__device__ __forceinline__ float sgnf(uint64_t b, uint64_t z) { return (__popcll(b & z) & 1) ? -1.f : 1.f; }

// Coefficients in shared memory: c_j * w_j (or the bare phase in per-term mode).
template <typename T>
__device__ __forceinline__ void load_terms(const TermPack &tp, const double *weights, double scale, uint64_t *z,
                                           T *cr, T *ci) {
    for (int j = threadIdx.x; j < tp.nt; j += blockDim.x) {
        double w = scale;
        if (weights) w *= weights[tp.idx[j]];
        z[j] = tp.z[j];
        cr[j] = (T)(tp.cre[j] * w);
        ci[j] = (T)(tp.cim[j] * w);
    }
    __syncthreads();
}

template <typename V>
__device__ __forceinline__ V diagD(uint64_t b, int nt, const uint64_t *z, const RT<V> *cr, const RT<V> *ci) {
    RT<V> re = 0, im = 0;
    for (int j = 0; j < nt; ++j) {
        const RT<V> s = (__popcll(b & z[j]) & 1) ? RT<V>(-1) : RT<V>(1);
        re = fma(s, cr[j], re);
        im = fma(s, ci[j], im);
    }
    return mkc<V>(re, im);
}

// Total mode: one partial per block, sum_j c_j w_j <P_j> over this launch's terms.
template <typename V>
__global__ void __launch_bounds__(PT) k_expval_total(const V *__restrict__ psi, int n, TermPack tp,
                                                     double *__restrict__ partials) {
    __shared__ uint64_t z[MAXT];
    __shared__ RT<V> cr[MAXT], ci[MAXT];
    __shared__ double sh[PT / 32];
    load_terms<RT<V>>(tp, nullptr, 1.0, z, cr, ci);
    const int nt = tp.nt;
    KSum<RT<V>> acc;
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (tp.x == 0) {
        const uint64_t N = (uint64_t)1 << n;
        for (; i < N; i += S) {
            const V a = psi[i];
            const V D = diagD<V>(i, nt, z, cr, ci);
            acc.add(norm2(a) * D.x);
        }
    } else {
        const int h = 63 - __clzll((long long)tp.x);
        const uint64_t half = (uint64_t)1 << (n - 1);
        for (; i < half; i += S) {
            const uint64_t b = insert0(i, h), bp = b ^ tp.x;
            const V a = psi[b], ap = psi[bp];
            const V D = diagD<V>(b, nt, z, cr, ci), Dp = diagD<V>(bp, nt, z, cr, ci);
            const RT<V> ur = re_cdot(ap, a), ui = im_cdot(ap, a);  // u = conj(a') a
            acc.add(ur * (D.x + Dp.x) - ui * (D.y - Dp.y));
        }
    }
    const double tot = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Per-term mode: up to MAXT1 terms, one partial slot per term (slot = term index).
template <typename V>
__global__ void __launch_bounds__(PT) k_expval_terms(const V *__restrict__ psi, int n, TermPack tp,
                                                     double *__restrict__ partials, int pblk) {
    __shared__ double sh[PT / 32];
    KSum<RT<V>> acc[MAXT1];
    const int nt = tp.nt;
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (tp.x == 0) {
        const uint64_t N = (uint64_t)1 << n;
        for (; i < N; i += S) {
            const RT<V> p = norm2(psi[i]);
#pragma unroll
            for (int j = 0; j < MAXT1; ++j)
                if (j < nt) acc[j].add(((__popcll(i & tp.z[j]) & 1) ? -p : p) * (RT<V>)tp.cre[j]);
        }
    } else {
        const int h = 63 - __clzll((long long)tp.x);
        const uint64_t half = (uint64_t)1 << (n - 1);
        for (; i < half; i += S) {
            const uint64_t b = insert0(i, h), bp = b ^ tp.x;
            const V a = psi[b], ap = psi[bp];
            const RT<V> ur = re_cdot(ap, a), ui = im_cdot(ap, a);
#pragma unroll
            for (int j = 0; j < MAXT1; ++j) {
                if (j < nt) {
                    const RT<V> s = (__popcll(b & tp.z[j]) & 1) ? RT<V>(-1) : RT<V>(1);
                    const RT<V> sp = (__popcll(bp & tp.z[j]) & 1) ? RT<V>(-1) : RT<V>(1);
                    const RT<V> cr = (RT<V>)tp.cre[j], ci = (RT<V>)tp.cim[j];
                    acc[j].add(ur * (cr * (s + sp)) - ui * (ci * (s - sp)));
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MAXT1; ++j) {
        if (j < nt) {
            const double tot = block_sum(acc[j].value(), sh);
            if (threadIdx.x == 0) partials[(size_t)tp.idx[j] * pblk + blockIdx.x] = tot;
        }
    }
}

// out (+)= sum_j scale w_j c_j P_j psi over this launch's terms.
template <typename V>
__global__ void __launch_bounds__(PT) k_apply_obs(const V *__restrict__ psi, V *__restrict__ out, int n,
                                                  TermPack tp, const double *__restrict__ weights, double scale,
                                                  int accumulate) {
    __shared__ uint64_t z[MAXT];
    __shared__ RT<V> cr[MAXT], ci[MAXT];
    load_terms<RT<V>>(tp, weights, scale, z, cr, ci);
    const int nt = tp.nt;
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (tp.x == 0) {
        const uint64_t N = (uint64_t)1 << n;
        for (; i < N; i += S) {
            V o = cmul(diagD<V>(i, nt, z, cr, ci), psi[i]);
            if (accumulate) o = cadd(o, out[i]);
            out[i] = o;
        }
    } else {
        const int h = 63 - __clzll((long long)tp.x);
        const uint64_t half = (uint64_t)1 << (n - 1);
        for (; i < half; i += S) {
            const uint64_t b = insert0(i, h), bp = b ^ tp.x;
            const V a = psi[b], ap = psi[bp];
            V o = cmul(diagD<V>(bp, nt, z, cr, ci), ap);   // (P psi)_b from psi_{b^x}
            V op = cmul(diagD<V>(b, nt, z, cr, ci), a);
            if (accumulate) {
                o = cadd(o, out[b]);
                op = cadd(op, out[bp]);
            }
            out[b] = o;
            out[bp] = op;
        }
    }
}

__global__ void k_sum_rows(const double *__restrict__ partials, int pblk, int nblk, double *__restrict__ sums) {
    __shared__ double sh[PT / 32];
    const double *p = partials + (size_t)blockIdx.x * pblk;
    double v = 0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) v += p[i];
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_sum_all(const double *__restrict__ sums, int count, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0;
        for (int i = 0; i < count; ++i) acc += sums[i];
        out[0] = acc;
    }
}

__global__ void k_fill(double *__restrict__ out, int count, double v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = v;
}

// with_coeff: (cre, cim) = coeff * i^y; otherwise the bare phase i^y.
static void fill_pack(TermPack &tp, uint64_t x, const std::vector<TermDev> &terms, size_t from, size_t cnt,
                      bool with_coeff) {
    tp.nt = (int)cnt;
    tp.pad = 0;
    tp.x = x;
    for (size_t k = 0; k < cnt; ++k) {
        const TermDev &t = terms[from + k];
        const double c = with_coeff ? t.coeff : 1.0;
        tp.z[k] = t.zmask;
        tp.cre[k] = t.pre * c;
        tp.cim[k] = t.pim * c;
        tp.idx[k] = t.index;
    }
}

cudaError_t ensure_work(tqd_state *st, size_t len, cudaStream_t s) {
    st->work_stream = s;  // every user of the workspace passes here with its stream
    if (st->work_len >= len) return cudaSuccess;
    if (st->work) {
        cudaError_t e = cudaFreeAsync(st->work, s);
        if (e != cudaSuccess) return e;
        st->work = nullptr;
        st->work_len = 0;
    }
    cudaError_t e = cudaMallocAsync((void **)&st->work, len * sizeof(double), s);
    if (e != cudaSuccess) return e;
    st->work_len = len;
    return cudaSuccess;
}

template <typename V>
static cudaError_t expval_t(tqd_state *st, const std::vector<PauliGroup> &groups, int n_terms, int mode,
                            double *dev_out, cudaStream_t s) {
    const int n = st->n;
    const uint64_t N = (uint64_t)1 << n;
    const int grid = stream_grid(N / 2 > 0 ? N / 2 : 1, PT);
    const int pblk = grid;
    if (mode == 0) {
        // groups that fit a 12-qubit tile share passes; the rest one pass per group
        std::vector<int> left;
        const std::vector<PauliTileDesc> tiles = plan_pauli_tiles(groups, n, &left);
        const int tgrid = tiles.empty() ? 0 : pauli_tile_expval_width(n, st->dtype);
        size_t launches = 0;
        for (int gi : left) launches += (groups[gi].terms.size() + MAXT - 1) / MAXT;
        const size_t rows = tiles.size() + launches;
        if (rows == 0) {
            k_fill<<<1, 32, 0, s>>>(dev_out, 1, 0.0);
            return cudaGetLastError();
        }
        const int w = std::max(pblk, tgrid);
        cudaError_t e = ensure_work(st, rows * (size_t)w + rows, s);
        if (e != cudaSuccess) return e;
        double *parts = st->work, *sums = st->work + rows * (size_t)w;
        if (!tiles.empty()) {
            e = launch_pauli_tile_expval(st, tiles, parts, w, s);
            if (e != cudaSuccess) return e;
            ProfScope ps(PK_REDUCE, 0.0, s);
            k_sum_rows<<<(int)tiles.size(), PT, 0, s>>>(parts, w, tgrid, sums);
        }
        if (launches == 0) {
            ProfScope ps(PK_REDUCE, 0.0, s);
            k_sum_all<<<1, 32, 0, s>>>(sums, (int)rows, dev_out);
            return cudaGetLastError();
        }
        parts += tiles.size() * (size_t)w;
        size_t slot = 0;
        for (int gi : left) {
            const PauliGroup &g = groups[gi];
            for (size_t from = 0; from < g.terms.size(); from += MAXT) {
                TermPack tp;
                const size_t cnt = std::min((size_t)MAXT, g.terms.size() - from);
                fill_pack(tp, g.xmask, g.terms, from, cnt, true);
                ProfScope ps(PK_EXPVAL, (double)N * sizeof(V), s);
                k_expval_total<V><<<grid, PT, 0, s>>>((const V *)st->amps, n, tp, parts + slot * w);
                ++slot;
            }
        }
        ProfScope ps(PK_REDUCE, 0.0, s);
        k_sum_rows<<<(int)launches, PT, 0, s>>>(parts, w, grid, sums + tiles.size());
        k_sum_all<<<1, 32, 0, s>>>(sums, (int)rows, dev_out);
        return cudaGetLastError();
    }
    if (n_terms == 0) return cudaSuccess;
    cudaError_t e = ensure_work(st, (size_t)n_terms * pblk + n_terms, s);
    if (e != cudaSuccess) return e;
    double *parts = st->work;
    for (const auto &g : groups) {
        for (size_t from = 0; from < g.terms.size(); from += MAXT1) {
            TermPack tp;
            fill_pack(tp, g.xmask, g.terms, from, std::min((size_t)MAXT1, g.terms.size() - from), false);
            ProfScope ps(PK_EXPVAL_TERMS, (double)N * sizeof(V), s);
            k_expval_terms<V><<<grid, PT, 0, s>>>((const V *)st->amps, n, tp, parts, pblk);
        }
    }
    ProfScope ps(PK_REDUCE, 0.0, s);
    k_sum_rows<<<n_terms, PT, 0, s>>>(parts, pblk, grid, dev_out);
    return cudaGetLastError();
}

cudaError_t launch_expval(const tqd_state *st, const std::vector<PauliGroup> &groups, int n_terms, int mode,
                          double *dev_out, cudaStream_t s) {
    tqd_state *w = const_cast<tqd_state *>(st);
    if (st->dtype == TQD_C64) return expval_t<float2>(w, groups, n_terms, mode, dev_out, s);
    return expval_t<double2>(w, groups, n_terms, mode, dev_out, s);
}

// Re <psi|lam> per block (FP64), for the expectation value taken from
// lambda = H psi.
template <typename V>
__global__ void __launch_bounds__(PT) k_re_dot(const V *__restrict__ psi, const V *__restrict__ lam, uint64_t N,
                                               double *__restrict__ partials) {
    __shared__ double sh[PT / 32];
    double acc = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)PT + threadIdx.x; i < N; i += (uint64_t)gridDim.x * PT)
        acc += (double)re_cdot(psi[i], lam[i]);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

template <typename V>
static cudaError_t apply_obs_t(const tqd_state *psi, const std::vector<PauliGroup> &groups,
                               const double *weights, double scale, tqd_state *out, double *dev_energy,
                               cudaStream_t s) {
    const int n = psi->n;
    const uint64_t N = (uint64_t)1 << n;
    const int grid = stream_grid(N / 2 > 0 ? N / 2 : 1, PT);
    int accumulate = 0;
    std::vector<int> left;
    const std::vector<PauliTileDesc> tiles = plan_pauli_tiles(groups, n, &left);
    // E = Re <psi|out> from the last tile launch (complex64, nothing after it)
    // or from a separate pass over both states
    const bool fused_e = dev_energy && sizeof(V) == 8 && left.empty() && !tiles.empty();
    const int egrid = fused_e ? pauli_tile_grid(n, psi->dtype) : grid;
    if (dev_energy) {
        cudaError_t e = ensure_work(out, (size_t)egrid, s);
        if (e != cudaSuccess) return e;
    }
    if (!tiles.empty()) {
        cudaError_t e = launch_pauli_tile_apply(psi, tiles, weights, scale, out, false, fused_e ? out->work : nullptr, s);
        if (e != cudaSuccess) return e;
        accumulate = 1;
    }
    for (int gi : left) {
        const PauliGroup &g = groups[gi];
        for (size_t from = 0; from < g.terms.size(); from += MAXT) {
            TermPack tp;
            fill_pack(tp, g.xmask, g.terms, from, std::min((size_t)MAXT, g.terms.size() - from), true);
            ProfScope ps(PK_APPLY_OBS, (double)N * sizeof(V) * (accumulate ? 3 : 2), s);
            k_apply_obs<V><<<grid, PT, 0, s>>>((const V *)psi->amps, (V *)out->amps, n, tp, weights, scale,
                                               accumulate);
            accumulate = 1;
        }
    }
    if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(out->amps, 0, N * sizeof(V), s);
        if (e != cudaSuccess) return e;
    }
    if (dev_energy) {
        if (!fused_e) {
            ProfScope ps(PK_EXPVAL, 2.0 * (double)N * sizeof(V), s);
            k_re_dot<V><<<egrid, PT, 0, s>>>((const V *)psi->amps, (const V *)out->amps, N, out->work);
        }
        ProfScope ps(PK_REDUCE, 0.0, s);
        k_sum_rows<<<1, PT, 0, s>>>(out->work, egrid, egrid, dev_energy);
    }
    return cudaGetLastError();
}

cudaError_t launch_apply_observable(const tqd_state *psi, const std::vector<PauliGroup> &groups,
                                    const double *dev_weights, double scale, tqd_state *out, cudaStream_t s,
                                    double *dev_energy) {
    if (psi->dtype == TQD_C64) return apply_obs_t<float2>(psi, groups, dev_weights, scale, out, dev_energy, s);
    return apply_obs_t<double2>(psi, groups, dev_weights, scale, out, dev_energy, s);
}

}  // namespace tqd
