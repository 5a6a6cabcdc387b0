// common.cuh -- device helpers shared by the libtqd kernels.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace tqd {

// ---------------------------------------------------------------- complex
template <typename V> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

template <typename V> __device__ __forceinline__ V mkc(typename Real<V>::T re, typename Real<V>::T im) {
    V r; r.x = re; r.y = im; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mkc<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mkc<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mkc<V>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a*b + c
template <typename V> __device__ __forceinline__ V cfma(V a, V b, V c) {
    return mkc<V>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
template <typename V> __device__ __forceinline__ V conjv(V a) { return mkc<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, typename Real<V>::T s) { return mkc<V>(a.x * s, a.y * s); }
// Re(conj(a) * b), Im(conj(a) * b)
template <typename V> __device__ __forceinline__ typename Real<V>::T re_cdot(V a, V b) { return fma(a.x, b.x, a.y * b.y); }
template <typename V> __device__ __forceinline__ typename Real<V>::T im_cdot(V a, V b) { return fma(a.x, b.y, -a.y * b.x); }
template <typename V> __device__ __forceinline__ typename Real<V>::T norm2(V a) { return fma(a.x, a.x, a.y * a.y); }

// 2x2 complex matrix held in registers.
template <typename V> struct M2 { V a, b, c, d; };  // [[a, b], [c, d]]

template <typename V> __device__ __forceinline__ void mv2(const M2<V> &m, V &x0, V &x1) {
    V y0 = cfma(m.a, x0, cmul(m.b, x1));
    V y1 = cfma(m.c, x0, cmul(m.d, x1));
    x0 = y0; x1 = y1;
}
template <typename V> __device__ __forceinline__ M2<V> dagger2(const M2<V> &m) {
    M2<V> r; r.a = conjv(m.a); r.b = conjv(m.c); r.c = conjv(m.b); r.d = conjv(m.d); return r;
}

// Matrices live in device memory as interleaved (re, im) scalars, row-major.
template <typename V> __device__ __forceinline__ M2<V> load_m2(const typename Real<V>::T *p) {
    M2<V> m;
    m.a = mkc<V>(p[0], p[1]); m.b = mkc<V>(p[2], p[3]);
    m.c = mkc<V>(p[4], p[5]); m.d = mkc<V>(p[6], p[7]);
    return m;
}

// --------------------------------------------------------------- indexing
// Insert a zero bit at position p (lower bits kept, upper bits shifted up).
__device__ __forceinline__ uint64_t insert0(uint64_t x, int p) {
    uint64_t lo = x & ((uint64_t(1) << p) - 1);
    return ((x >> p) << (p + 1)) | lo;
}
// Insert zero bits at p0 < p1.
__device__ __forceinline__ uint64_t insert00(uint64_t x, int p0, int p1) {
    return insert0(insert0(x, p0), p1);
}

__device__ __forceinline__ int parity64(uint64_t x) { return __popcll(x) & 1; }

// Packed pairs of float (Blackwell's f32x2 pipe): one instruction does the
// real and imaginary parts of a complex64 amplitude.
__device__ __forceinline__ uint64_t f2_pack(float2 v) {
    uint64_t u;
    asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(v.x), "f"(v.y));
    return u;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t u) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(u));
    return v;
}
// a * b + c, lane by lane
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
    return f2_unpack(d);
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(d);
}

// ---------------------------------------------------------- bounded waits
// Every spin wait of the library gives up after this much elapsed time on the
// device's global nanosecond timer (a poll count has no bound in time: one
// mbarrier.try_wait may suspend the thread for a hardware-chosen interval).
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;

__device__ __forceinline__ uint64_t gtimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------- reductions
// Kahan-compensated FP32 (or plain FP64) running sum.
template <typename T> struct KSum {
    T s = 0, c = 0;
    __device__ __forceinline__ void add(T v) {
        T y = v - c;
        T t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct KSum<double> {
    double s = 0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide FP64 sum; the result is valid in thread 0.  `sh` holds at least
// blockDim.x / 32 doubles.  Contains __syncthreads().
__device__ __forceinline__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) r += sh[i];
    }
    return r;
}

}  // namespace tqd
