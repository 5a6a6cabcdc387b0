// shots.cu -- shot noise on the probability vector p = |psi|^2 (Sec. 4.3.2):
// probabilities, exact sampling, and the approximate Gaussian sample with
// its product with the state for the reverse sweep.
//
// Exact: shot s is the outcome b whose cumulative interval of the
// normalised p holds the caller's uniform u_s (inverse transform).  On one
// device the paper's hierarchy (group totals, then outcomes within the
// group) becomes a two-level cumulative sum: totals of chunks of
// consecutive outcomes and their exclusive prefix, a binary search over the
// chunks, then a scan inside the chunk.
//
// Approximate: y = n p + sqrt(n) D S z with D = diag(u), u = sqrt(p),
// S = I - 2 v v^T, v = vt / |vt|, vt = e_{N-1} - u, and z_{N-1} = 0; with
// B = vt . z and C = |vt|^2, y_i = n p_i + sqrt(n) u_i (z_i - 2 vt_i B / C).
// Its product with the state: for L = sum_i ybar_i y_i and A = sum_i ybar_i
// u_i vt_i,
//   dL/du_k = ybar_k (2 n u_k + sqrt(n) z_k)
//             - 2 sqrt(n) ([ybar_k (vt_k - u_k) B - A z_k] / C + 2 A B vt_k / C^2),
// and lambda_k = dL/d conj(psi_k) = (dL/du_k) psi_k / (2 |psi_k|) (0 where
// psi_k = 0), the seed of the reverse sweep for a loss of the shots.
// Reductions in FP64.
#include "common.cuh"
#include "internal.h"
#include "launch.h"
#include "prof.h"

namespace tqd {

namespace {

constexpr int ST = 256;  // threads per block

template <typename V> __device__ __forceinline__ double prob(const V &a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

template <typename V>
__global__ void __launch_bounds__(ST) k_probs(const V *__restrict__ psi, uint64_t N, double *__restrict__ p) {
    for (uint64_t i = blockIdx.x * (uint64_t)ST + threadIdx.x; i < N; i += (uint64_t)gridDim.x * ST) p[i] = prob(psi[i]);
}

// chunk totals: one warp per chunk of `csize` consecutive outcomes
template <typename V>
__global__ void __launch_bounds__(ST) k_chunk_sums(const V *__restrict__ psi, uint64_t n_chunks, uint64_t csize,
                                                   double *__restrict__ sums) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (ST / 32);
    for (uint64_t c = blockIdx.x * (uint64_t)(ST / 32) + (threadIdx.x >> 5); c < n_chunks; c += warps) {
        const V *q = psi + c * csize;
        double s = 0;
        for (uint64_t i = lane; i < csize; i += 32) s += prob(q[i]);
        s = warp_sum(s);
        if (lane == 0) sums[c] = s;
    }
}

// Exclusive prefix of x over blocks of 1024 (one block each): x <- prefix
// within the block, tot[block] = block total.
__global__ void __launch_bounds__(1024) k_scan_block(double *__restrict__ x, uint64_t n, double *__restrict__ tot) {
    __shared__ double sh[1024];
    const uint64_t i = blockIdx.x * 1024ull + threadIdx.x;
    const double v = i < n ? x[i] : 0.0;
    sh[threadIdx.x] = v;
    __syncthreads();
    // Hillis-Steele inclusive scan
    for (int o = 1; o < 1024; o <<= 1) {
        const double t = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0.0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) x[i] = sh[threadIdx.x] - v;
    if (threadIdx.x == 1023) tot[blockIdx.x] = sh[1023];
}

// adds each block's offset (exclusive prefix of the block totals, computed
// in order by one thread: at most 1024 blocks)
__global__ void k_scan_add(double *__restrict__ x, uint64_t n, const double *__restrict__ tot, int nblk,
                           double *__restrict__ total_out) {
    __shared__ double off;
    if (threadIdx.x == 0) {
        double o = 0;
        for (int b = 0; b < (int)blockIdx.x; ++b) o += tot[b];
        off = o;
        if (blockIdx.x == 0 && total_out) {
            double t = 0;
            for (int b = 0; b < nblk; ++b) t += tot[b];
            *total_out = t;
        }
    }
    __syncthreads();
    const uint64_t i = blockIdx.x * 1024ull + threadIdx.x;
    if (i < n) x[i] += off;
}

// one thread per shot: the outcome whose cumulative interval holds u * total
template <typename V>
__global__ void __launch_bounds__(ST) k_sample(const V *__restrict__ psi, const double *__restrict__ prefix,
                                               uint64_t n_chunks, uint64_t csize, const double *__restrict__ total,
                                               const double *__restrict__ uni, uint64_t n_shots,
                                               int64_t *__restrict__ out) {
    const double T = *total;
    for (uint64_t s = blockIdx.x * (uint64_t)ST + threadIdx.x; s < n_shots; s += (uint64_t)gridDim.x * ST) {
        const double t = uni[s] * T;
        // last chunk whose exclusive prefix is <= t (upper bound - 1)
        uint64_t lo = 0, hi = n_chunks;
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) >> 1;
            if (prefix[mid] <= t) lo = mid;
            else hi = mid;
        }
        const V *q = psi + lo * csize;
        double acc = prefix[lo];
        int64_t pick = -1, last = -1;
        for (uint64_t i = 0; i < csize; ++i) {
            const double pi = prob(q[i]);
            if (pi > 0) last = (int64_t)(lo * csize + i);
            acc += pi;
            if (acc > t && pi > 0) {
                pick = (int64_t)(lo * csize + i);
                break;
            }
        }
        // rounding left t past the chunk's last outcome: take that outcome
        out[s] = pick >= 0 ? pick : (last >= 0 ? last : (int64_t)(lo * csize + csize - 1));
    }
}

// FP64 partial sums of the Gaussian sample's scalars per block:
// [0] C = sum vt^2, [1] B = sum vt z, [2] A = sum ybar u vt (when ybar)
template <typename V>
__global__ void __launch_bounds__(ST) k_gauss_sums(const V *__restrict__ psi, uint64_t N, const double *__restrict__ z,
                                                   const double *__restrict__ ybar, double *__restrict__ parts) {
    __shared__ double sh[ST / 32];
    double c = 0, b = 0, a = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)ST + threadIdx.x; i < N; i += (uint64_t)gridDim.x * ST) {
        const double u = sqrt(prob(psi[i]));
        const double vt = (i == N - 1 ? 1.0 : 0.0) - u;
        const double zi = i == N - 1 ? 0.0 : z[i];
        c += vt * vt;
        b += vt * zi;
        if (ybar) a += ybar[i] * u * vt;
    }
    const double tc = block_sum(c, sh);
    const double tb = block_sum(b, sh);
    const double ta = ybar ? block_sum(a, sh) : 0.0;
    if (threadIdx.x == 0) {
        parts[blockIdx.x] = tc;
        parts[gridDim.x + blockIdx.x] = tb;
        parts[2 * gridDim.x + blockIdx.x] = ta;
    }
}

__global__ void k_gauss_reduce(const double *__restrict__ parts, int nblk, double *__restrict__ abc) {
    // one warp: fixed-order sums of the three rows
    const int lane = threadIdx.x;
    for (int r = 0; r < 3; ++r) {
        double s = 0;
        for (int i = lane; i < nblk; i += 32) s += parts[r * nblk + i];
        s = warp_sum(s);
        if (lane == 0) abc[r] = s;
    }
}

template <typename V>
__global__ void __launch_bounds__(ST) k_gauss_y(const V *__restrict__ psi, uint64_t N, double n_shots,
                                                const double *__restrict__ z, const double *__restrict__ abc,
                                                double *__restrict__ y) {
    const double C = abc[0], B = abc[1];
    const double f = C > 0 ? 2.0 * B / C : 0.0;
    const double sn = sqrt(n_shots);
    for (uint64_t i = blockIdx.x * (uint64_t)ST + threadIdx.x; i < N; i += (uint64_t)gridDim.x * ST) {
        const double p = prob(psi[i]);
        const double u = sqrt(p);
        const double vt = (i == N - 1 ? 1.0 : 0.0) - u;
        const double zi = i == N - 1 ? 0.0 : z[i];
        y[i] = n_shots * p + sn * u * (zi - vt * f);
    }
}

template <typename V>
__global__ void __launch_bounds__(ST) k_gauss_vjp(const V *__restrict__ psi, uint64_t N, double n_shots,
                                                  const double *__restrict__ z, const double *__restrict__ ybar,
                                                  const double *__restrict__ abc, V *__restrict__ lam) {
    const double C = abc[0], B = abc[1], A = abc[2];
    const double sn = sqrt(n_shots);
    for (uint64_t i = blockIdx.x * (uint64_t)ST + threadIdx.x; i < N; i += (uint64_t)gridDim.x * ST) {
        const V a = psi[i];
        const double u = sqrt(prob(a));
        const double vt = (i == N - 1 ? 1.0 : 0.0) - u;
        const double zi = i == N - 1 ? 0.0 : z[i];
        double ub = ybar[i] * (2.0 * n_shots * u + sn * zi);
        if (C > 0) ub -= 2.0 * sn * ((ybar[i] * (vt - u) * B - A * zi) / C + 2.0 * A * B * vt / (C * C));
        const double g = u > 0 ? ub / (2.0 * u) : 0.0;
        lam[i] = mkc<V>((typename Real<V>::T)(g * (double)a.x), (typename Real<V>::T)(g * (double)a.y));
    }
}

uint64_t chunk_size(uint64_t N) {
    uint64_t c = 256;
    while (N / c > (1ull << 20)) c <<= 1;
    return c < N ? c : N;
}

template <typename V>
cudaError_t sample_t(tqd_state *st, const double *uni, uint64_t n_shots, int64_t *out, cudaStream_t s) {
    const uint64_t N = (uint64_t)1 << st->n;
    const uint64_t cs = chunk_size(N), nc = N / cs;
    const int nblk = (int)((nc + 1023) / 1024);
    cudaError_t e = ensure_work(st, nc + (size_t)nblk + 1, s);
    if (e != cudaSuccess) return e;
    double *prefix = st->work, *tot = st->work + nc, *total = tot + nblk;
    const V *psi = (const V *)st->amps;
    ProfScope ps(PK_SHOTS, (double)N * sizeof(V), s);
    k_chunk_sums<V><<<stream_grid(nc * 32, ST), ST, 0, s>>>(psi, nc, cs, prefix);
    k_scan_block<<<nblk, 1024, 0, s>>>(prefix, nc, tot);
    k_scan_add<<<nblk, 1024, 0, s>>>(prefix, nc, tot, nblk, total);
    if (n_shots) k_sample<V><<<stream_grid(n_shots, ST), ST, 0, s>>>(psi, prefix, nc, cs, total, uni, n_shots, out);
    return cudaGetLastError();
}

template <typename V>
cudaError_t gauss_t(tqd_state *st, double n_shots, const double *z, const double *ybar, double *y, tqd_state *lam,
                    cudaStream_t s) {
    const uint64_t N = (uint64_t)1 << st->n;
    const int grid = stream_grid(N, ST);
    cudaError_t e = ensure_work(st, 3 * (size_t)grid + 3, s);
    if (e != cudaSuccess) return e;
    double *parts = st->work, *abc = st->work + 3 * (size_t)grid;
    const V *psi = (const V *)st->amps;
    ProfScope ps(PK_SHOTS, (double)N * (sizeof(V) * 2 + 16), s);
    k_gauss_sums<V><<<grid, ST, 0, s>>>(psi, N, z, ybar, parts);
    k_gauss_reduce<<<1, 32, 0, s>>>(parts, grid, abc);
    if (ybar) k_gauss_vjp<V><<<grid, ST, 0, s>>>(psi, N, n_shots, z, ybar, abc, (V *)lam->amps);
    else k_gauss_y<V><<<grid, ST, 0, s>>>(psi, N, n_shots, z, abc, y);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_probabilities(const tqd_state *st, double *p, cudaStream_t s) {
    const uint64_t N = (uint64_t)1 << st->n;
    const int grid = stream_grid(N, ST);
    ProfScope ps(PK_SHOTS, (double)N * ((st->dtype == TQD_C64 ? 8 : 16) + 8), s);
    if (st->dtype == TQD_C64) k_probs<float2><<<grid, ST, 0, s>>>((const float2 *)st->amps, N, p);
    else k_probs<double2><<<grid, ST, 0, s>>>((const double2 *)st->amps, N, p);
    return cudaGetLastError();
}

cudaError_t launch_sample(tqd_state *st, const double *uni, uint64_t n_shots, int64_t *out, cudaStream_t s) {
    return st->dtype == TQD_C64 ? sample_t<float2>(st, uni, n_shots, out, s) : sample_t<double2>(st, uni, n_shots, out, s);
}

cudaError_t launch_shots_gaussian(tqd_state *st, double n_shots, const double *z, const double *ybar, double *y,
                                  tqd_state *lam, cudaStream_t s) {
    return st->dtype == TQD_C64 ? gauss_t<float2>(st, n_shots, z, ybar, y, lam, s)
                                : gauss_t<double2>(st, n_shots, z, ybar, y, lam, s);
}

}  // namespace tqd
