// noalloc.cu -- tqd_expval_noalloc: the Pauli-sum expectation value with its
// reduction scratch in a fixed, file-scope device array instead of memory the
// library allocates.
//
// Who needs it: callers that may not allocate device memory once they are
// running -- a service that reserved its whole memory budget at start-up, a
// latency-sensitive loop where a cudaMalloc or cudaFree would stall the
// device, or a host framework that owns the device allocator and gives the
// library no hook into it.  tqd_expval grows a per-state workspace on demand;
// this entry point never does.
//
// The scratch array holds the per-block partial sums of one call.  It is
// sized for TQD_NOALLOC_SCRATCH_DOUBLES doubles (1 MiB); every GPU that
// loads the library keeps that much reserved until the process exits.  Every
// call on a device shares the same array: two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it.
#include <cuda.h>
#include <math.h>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace tqd {

static constexpr size_t kNoallocScratch = 131072;  // doubles (1 MiB); see TQD_NOALLOC_SCRATCH_DOUBLES
static constexpr int kTerms = 64;                    // terms per launch
static constexpr int kThreads = 256;

// The scratch.  In host code this name is only a stand-in for the symbol; the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_scratch[kNoallocScratch];

struct NaPack {
    int nt;
    int pad;
    uint64_t x;
    uint64_t z[kTerms];
    double cre[kTerms];
    double cim[kTerms];
};

template <typename V>
__device__ __forceinline__ V na_diag(uint64_t b, int nt, const uint64_t *z, const typename Real<V>::T *cr,
                                     const typename Real<V>::T *ci) {
    typename Real<V>::T re = 0, im = 0;
    for (int j = 0; j < nt; ++j) {
        const typename Real<V>::T s = (__popcll(b & z[j]) & 1) ? -1 : 1;
        re = fma(s, cr[j], re);
        im = fma(s, ci[j], im);
    }
    return mkc<V>(re, im);
}

// One partial per block into row[blockIdx.x]; same arithmetic and order as the
// allocating expectation kernel.
template <typename V>
__global__ void __launch_bounds__(kThreads) k_na_expval(const V *__restrict__ psi, int n, NaPack tp,
                                                        double *__restrict__ row) {
    using T = typename Real<V>::T;
    __shared__ uint64_t z[kTerms];
    __shared__ T cr[kTerms], ci[kTerms];
    __shared__ double sh[kThreads / 32];
    for (int j = threadIdx.x; j < tp.nt; j += blockDim.x) {
        z[j] = tp.z[j];
        cr[j] = (T)tp.cre[j];
        ci[j] = (T)tp.cim[j];
    }
    __syncthreads();
    KSum<T> acc;
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (tp.x == 0) {
        const uint64_t N = (uint64_t)1 << n;
        for (; i < N; i += S) {
            const V a = psi[i];
            acc.add(norm2(a) * na_diag<V>(i, tp.nt, z, cr, ci).x);
        }
    } else {
        const int h = 63 - __clzll((long long)tp.x);
        const uint64_t half = (uint64_t)1 << (n - 1);
        for (; i < half; i += S) {
            const uint64_t b = insert0(i, h), bp = b ^ tp.x;
            const V a = psi[b], ap = psi[bp];
            const V D = na_diag<V>(b, tp.nt, z, cr, ci), Dp = na_diag<V>(bp, tp.nt, z, cr, ci);
            const T ur = re_cdot(ap, a), ui = im_cdot(ap, a);
            acc.add(ur * (D.x + Dp.x) - ui * (D.y - Dp.y));
        }
    }
    const double tot = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) row[blockIdx.x] = tot;
}

__global__ void k_na_rows(const double *__restrict__ parts, int nblk, double *__restrict__ sums) {
    __shared__ double sh[kThreads / 32];
    const double *p = parts + (size_t)blockIdx.x * nblk;
    double v = 0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) v += p[i];
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_na_total(const double *__restrict__ sums, int count, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0;
        for (int i = 0; i < count; ++i) acc += sums[i];
        out[0] = acc;
    }
}

// Device address of g_scratch, looked up with the device current the first
// time a context of that device calls.  The cache is keyed on the driver's
// context ID, which is unique for the life of the process: after
// cudaDeviceReset (or any other end of the device's context) the next call
// finds a new ID and looks the address up again instead of reusing one that
// belonged to the destroyed context.
typedef CUresult (*FnCtxGetCurrent)(CUcontext *);
typedef CUresult (*FnCtxGetId)(CUcontext, unsigned long long *);

static std::mutex g_mu;
static double *g_addr[64] = {nullptr};
static unsigned long long g_ctx[64] = {0};

// ID of the calling thread's current context; 0 when there is none yet or
// the driver entry points are unavailable (the address is then looked up on
// every call).
static unsigned long long current_ctx_id() {
    static FnCtxGetCurrent get_current = nullptr;
    static FnCtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (FnCtxGetCurrent)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (FnCtxGetId)p;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

static cudaError_t scratch_address(int dev, double **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const unsigned long long id = current_ctx_id();
    if (!g_addr[dev] || id == 0 || id != g_ctx[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (double *)p;
        // the lookup makes the device's context current if it was not yet
        g_ctx[dev] = id != 0 ? id : current_ctx_id();
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

template <typename V>
static cudaError_t run_na(const tqd_state *st, const std::vector<PauliGroup> &groups, double *scratch,
                          int grid, size_t launches, double *dev_out, cudaStream_t s) {
    double *sums = scratch + launches * (size_t)grid;
    size_t slot = 0;
    for (const auto &g : groups) {
        for (size_t from = 0; from < g.terms.size(); from += kTerms) {
            NaPack tp;
            const size_t cnt = g.terms.size() - from < (size_t)kTerms ? g.terms.size() - from : (size_t)kTerms;
            tp.nt = (int)cnt;
            tp.pad = 0;
            tp.x = g.xmask;
            for (size_t k = 0; k < cnt; ++k) {
                const TermDev &t = g.terms[from + k];
                tp.z[k] = t.zmask;
                tp.cre[k] = t.pre * t.coeff;
                tp.cim[k] = t.pim * t.coeff;
            }
            k_na_expval<V><<<grid, kThreads, 0, s>>>((const V *)st->amps, st->n, tp, scratch + slot * grid);
            ++slot;
        }
    }
    k_na_rows<<<(int)launches, kThreads, 0, s>>>(scratch, grid, sums);
    k_na_total<<<1, 32, 0, s>>>(sums, (int)launches, dev_out);
    return cudaGetLastError();
}

}  // namespace tqd

using namespace tqd;

extern "C" tqd_status tqd_expval_noalloc(const tqd_state *state, const tqd_pauli_term *terms, size_t n_terms,
                                         double *dev_out, void *stream) {
    if (!state || !dev_out || (n_terms > 0 && !terms)) {
        set_error("tqd_expval_noalloc: NULL state, terms or dev_out");
        return TQD_ERR_INVALID_ARG;
    }
    const uint64_t lim = ((uint64_t)1 << state->n) - 1;
    for (size_t j = 0; j < n_terms; ++j) {
        if ((terms[j].xmask & ~lim) || (terms[j].zmask & ~lim)) {
            set_error("tqd_expval_noalloc: term %zu acts on a qubit >= %d", j, state->n);
            return TQD_ERR_INVALID_ARG;
        }
        if (!isfinite(terms[j].coeff)) {
            set_error("tqd_expval_noalloc: term %zu has a non-finite coefficient", j);
            return TQD_ERR_NUMERIC;
        }
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        set_error("tqd_expval_noalloc: cudaGetDevice failed");
        return TQD_ERR_CUDA;
    }
    if (prev != state->device && cudaSetDevice(state->device) != cudaSuccess) {
        set_error("tqd_expval_noalloc: cannot make device %d current", state->device);
        return TQD_ERR_CUDA;
    }
    tqd_status rc = TQD_OK;
    do {
        const std::vector<PauliGroup> groups = group_terms(terms, n_terms);
        size_t launches = 0;
        for (const auto &g : groups) launches += (g.terms.size() + kTerms - 1) / kTerms;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, state->device);
        if (sms <= 0) sms = 148;
        const uint64_t half = ((uint64_t)1 << state->n) / 2 > 0 ? ((uint64_t)1 << state->n) / 2 : 1;
        uint64_t grid = (half + kThreads - 1) / kThreads;
        if (grid > (uint64_t)sms * 8) grid = (uint64_t)sms * 8;
        const size_t need = launches * (size_t)grid + launches;
        if (need > kNoallocScratch) {
            set_error("tqd_expval_noalloc: %zu x-mask groups need %zu scratch doubles, the fixed scratch holds %zu "
                      "(TQD_NOALLOC_SCRATCH_DOUBLES); use tqd_expval", launches, need, kNoallocScratch);
            rc = TQD_ERR_INVALID_ARG;
            break;
        }
        double *scratch = nullptr;
        cudaError_t e = scratch_address(state->device, &scratch);
        if (e != cudaSuccess) {
            set_error("tqd_expval_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            rc = TQD_ERR_CUDA;
            break;
        }
        cudaStream_t s = (cudaStream_t)stream;
        if (launches == 0) {
            e = cudaMemsetAsync(dev_out, 0, sizeof(double), s);
        } else if (state->dtype == TQD_C64) {
            e = run_na<float2>(state, groups, scratch, (int)grid, launches, dev_out, s);
        } else {
            e = run_na<double2>(state, groups, scratch, (int)grid, launches, dev_out, s);
        }
        if (e != cudaSuccess) {
            set_error("tqd_expval_noalloc: %s", cudaGetErrorString(e));
            rc = TQD_ERR_CUDA;
        }
    } while (0);
    if (prev != state->device) cudaSetDevice(prev);
    return rc;
}
