// kernels_plain.cu -- gate matrices from angles, state reset, and the
// gate-by-gate path: one full-state streaming kernel per gate (Algorithm 1's
// contraction M x_Q X done in place with bit-index addressing), plus the
// gate-by-gate adjoint step of Sec. 4.4 (recompute x = U^dagger y instead of
// storing it) with the angle derivative reduced in the same sweep.
#include <stdio.h>

#include "common.cuh"
#include "gate_mat.h"
#include "launch.h"
#include "prof.h"

namespace tqd {

template <typename V> using RT = typename Real<V>::T;
constexpr int TPB = 256;

// Two consecutive amplitudes in one 16-byte (c64) or two 16-byte (c128) accesses.
__device__ __forceinline__ void ld2(const float2 *p, float2 &a, float2 &b) {
    float4 q = *reinterpret_cast<const float4 *>(p);
    a = make_float2(q.x, q.y);
    b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void st2(float2 *p, float2 a, float2 b) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void ld2(const double2 *p, double2 &a, double2 &b) { a = p[0]; b = p[1]; }
__device__ __forceinline__ void st2(double2 *p, double2 a, double2 b) { p[0] = a; p[1] = b; }

int stream_grid(uint64_t units, int threads) {
    const uint64_t cap = (uint64_t)device_sm_count() * 8;
    uint64_t need = (units + threads - 1) / threads;
    if (need > cap) need = cap;
    if (need < 1) need = 1;
    return (int)need;
}

// ------------------------------------------------------------------- prep
// Per-gate unitary from its angle; entry (r, c) of a d x d matrix at
// [2 (r d + c)], [2 (r d + c) + 1].  R_P(t) = exp(-i t P / 2).
__global__ void k_prep(const GateDev *__restrict__ gates, int ng, const double *__restrict__ params,
                       const double *__restrict__ table, double *__restrict__ m64, float *__restrict__ m32) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const GateDev gd = gates[g];
    const double th = gd.param >= 0 ? params[gd.param] : gd.fixed;
    double m[MAT_STRIDE];
    gate_matrix(gd.kind, th, table, gd.mat, m);
#pragma unroll
    for (int i = 0; i < MAT_STRIDE; ++i) {
        m64[(size_t)g * MAT_STRIDE + i] = m[i];
        m32[(size_t)g * MAT_STRIDE + i] = (float)m[i];
    }
}

cudaError_t launch_prep(const tqd_circuit *c, const double *dev_params, cudaStream_t s) {
    const int ng = (int)c->gates.size();
    if (ng == 0) return cudaSuccess;
    ProfScope ps(PK_PREP, 0.0, s);
    k_prep<<<(ng + 127) / 128, 128, 0, s>>>(c->d_gates, ng, dev_params, c->d_table, c->d_mats64, c->d_mats32);
    return cudaGetLastError();
}

cudaError_t launch_prep_raw(const GateDev *gates, int ng, const double *dev_params, const double *table,
                            double *m64, float *m32, cudaStream_t s) {
    if (ng == 0) return cudaSuccess;
    k_prep<<<(ng + 127) / 128, 128, 0, s>>>(gates, ng, dev_params, table, m64, m32);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ reset
template <typename V>
__global__ void k_reset(V *__restrict__ a, uint64_t N, uint64_t j) {
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    const V z = mkc<V>(0, 0);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; 2 * i < N; i += S) {
        V x = z, y = z;
        if (2 * i == j) x = mkc<V>(1, 0);
        if (2 * i + 1 == j) y = mkc<V>(1, 0);
        if (2 * i + 1 < N) st2(a + 2 * i, x, y);
        else a[2 * i] = x;
    }
}

cudaError_t launch_reset(tqd_state *st, uint64_t j, cudaStream_t s) {
    const uint64_t N = (uint64_t)1 << st->n;
    const int grid = stream_grid((N + 1) / 2, TPB);
    ProfScope ps(PK_RESET, (double)N * (st->dtype == TQD_C64 ? 8 : 16), s);
    if (st->dtype == TQD_C64) k_reset<float2><<<grid, TPB, 0, s>>>((float2 *)st->amps, N, j);
    else k_reset<double2><<<grid, TPB, 0, s>>>((double2 *)st->amps, N, j);
    return cudaGetLastError();
}

// -------------------------------------------------------- 1-qubit dense
// Pairs (b, b + 2^t).  For t >= 1 a unit is four amplitudes b, b+1 (bit 0
// vectorised) and their partners; for t = 0 a unit is two adjacent pairs.
// Complex64 with t <= 1 (n >= 6): each thread moves one 16-byte chunk (two
// amplitudes) per access and consecutive lanes consecutive chunks, so every
// warp access is one contiguous 512 bytes: for t = 0 the chunk is a pair; for
// t = 1 chunks 2k and 2k + 1 are partners, held by lanes 2k and 2k + 1, which
// exchange them with one shuffle per float.
template <typename V>
__global__ void __launch_bounds__(TPB) k_dense1(V *__restrict__ a, int n, int t, const RT<V> *__restrict__ mat,
                                                int dag) {
    M2<V> m = load_m2<V>(mat);
    if (dag) m = dagger2(m);
    const uint64_t units = (uint64_t)1 << (n - 2);
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if constexpr (sizeof(V) == 8) {
        if (t <= 1 && n >= 6) {
            // chunks: 2^(n-1), a multiple of 32, and every warp starts at a
            // multiple of 32, so the loop runs the same count in all its lanes
            const uint64_t C = (uint64_t)1 << (n - 1);
            const bool hi = threadIdx.x & 1;  // t = 1: this lane's chunk has bit 1 set
            for (uint64_t c = i; c < C; c += 2 * S) {
                const uint64_t c2 = c + S;
                const bool two = c2 < C;
                V x0, x1, y0, y1;
                ld2(a + 2 * c, x0, x1);
                if (two) ld2(a + 2 * c2, y0, y1);
                if (t == 0) {
                    mv2(m, x0, x1);
                    if (two) mv2(m, y0, y1);
                } else {
                    // partner chunk from the neighbouring lane (all lanes take part)
                    V p0, p1, q0 = x0, q1 = x1;
                    p0.x = __shfl_xor_sync(0xffffffffu, x0.x, 1);
                    p0.y = __shfl_xor_sync(0xffffffffu, x0.y, 1);
                    p1.x = __shfl_xor_sync(0xffffffffu, x1.x, 1);
                    p1.y = __shfl_xor_sync(0xffffffffu, x1.y, 1);
                    // bit-1 = 0 lane: a*mine + b*partner; bit-1 = 1 lane: c*partner + d*mine
                    x0 = hi ? cfma(m.c, p0, cmul(m.d, q0)) : cfma(m.a, q0, cmul(m.b, p0));
                    x1 = hi ? cfma(m.c, p1, cmul(m.d, q1)) : cfma(m.a, q1, cmul(m.b, p1));
                    if (two) {
                        V r0, r1;
                        q0 = y0;
                        q1 = y1;
                        r0.x = __shfl_xor_sync(0xffffffffu, y0.x, 1);
                        r0.y = __shfl_xor_sync(0xffffffffu, y0.y, 1);
                        r1.x = __shfl_xor_sync(0xffffffffu, y1.x, 1);
                        r1.y = __shfl_xor_sync(0xffffffffu, y1.y, 1);
                        y0 = hi ? cfma(m.c, r0, cmul(m.d, q0)) : cfma(m.a, q0, cmul(m.b, r0));
                        y1 = hi ? cfma(m.c, r1, cmul(m.d, q1)) : cfma(m.a, q1, cmul(m.b, r1));
                    }
                }
                st2(a + 2 * c, x0, x1);
                if (two) st2(a + 2 * c2, y0, y1);
            }
            return;
        }
    }
    if (t >= 1) {
        const uint64_t T = (uint64_t)1 << t;
        for (; i < units; i += S) {
            const uint64_t b = insert0(2 * i, t);
            V x0, y0, x1, y1;
            ld2(a + b, x0, y0);
            ld2(a + b + T, x1, y1);
            mv2(m, x0, x1);
            mv2(m, y0, y1);
            st2(a + b, x0, y0);
            st2(a + b + T, x1, y1);
        }
    } else {
        for (; i < units; i += S) {
            const uint64_t b = 4 * i;
            V x0, x1, y0, y1;
            ld2(a + b, x0, x1);
            ld2(a + b + 2, y0, y1);
            mv2(m, x0, x1);
            mv2(m, y0, y1);
            st2(a + b, x0, x1);
            st2(a + b + 2, y0, y1);
        }
    }
}

// ----------------------------------------------------- 1-qubit diagonal
// amp *= d0 or d1 by bit t.  only1: d0 == 1, so only amplitudes with bit t
// set are touched (half the traffic).
template <typename V>
__global__ void __launch_bounds__(TPB) k_diag1(V *__restrict__ a, int n, int t, const RT<V> *__restrict__ mat,
                                               int dag, int only1) {
    M2<V> m = load_m2<V>(mat);
    V d0 = m.a, d1 = m.d;
    if (dag) { d0 = conjv(d0); d1 = conjv(d1); }
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t T = (uint64_t)1 << t;
    if (only1) {
        if (t >= 1) {
            const uint64_t units = (uint64_t)1 << (n - 2);
            for (; i < units; i += S) {
                const uint64_t b = insert0(2 * i, t) | T;
                V x, y;
                ld2(a + b, x, y);
                st2(a + b, cmul(x, d1), cmul(y, d1));
            }
        } else {
            const uint64_t units = (uint64_t)1 << (n - 1);
            for (; i < units; i += S) a[2 * i + 1] = cmul(a[2 * i + 1], d1);
        }
    } else {
        const uint64_t units = (uint64_t)1 << (n - 1);
        for (; i < units; i += S) {
            const uint64_t b = 2 * i;
            V x, y;
            ld2(a + b, x, y);
            if (t >= 1) {
                const V d = ((b >> t) & 1) ? d1 : d0;
                x = cmul(x, d);
                y = cmul(y, d);
            } else {
                x = cmul(x, d0);
                y = cmul(y, d1);
            }
            st2(a + b, x, y);
        }
    }
}

// ------------------------------------------- 2-qubit permutations, phases
// CNOT(c, t): swap amplitudes (c=1, t=0) <-> (c=1, t=1).
// SWAP(p, q): swap amplitudes (p=1, q=0) <-> (p=0, q=1).
// kind 0 = CNOT, 1 = SWAP.
template <typename V>
__global__ void __launch_bounds__(TPB) k_perm2(V *__restrict__ a, int n, int p, int q, int kind) {
    const int lo = min(p, q), hi = max(p, q);
    const uint64_t P = (uint64_t)1 << p, Q = (uint64_t)1 << q;
    const uint64_t off0 = kind == 0 ? P : P;          // first element of the swapped pair
    const uint64_t off1 = kind == 0 ? (P | Q) : Q;    // second element
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (lo >= 1) {
        const uint64_t units = (uint64_t)1 << (n - 3);
        for (; i < units; i += S) {
            const uint64_t b = insert00(2 * i, lo, hi);
            V x0, y0, x1, y1;
            ld2(a + (b | off0), x0, y0);
            ld2(a + (b | off1), x1, y1);
            st2(a + (b | off0), x1, y1);
            st2(a + (b | off1), x0, y0);
        }
    } else {
        // one wire is qubit 0: work on 16-byte pairs (b, b+1) and (b|H, b|H+1)
        const uint64_t H = (uint64_t)1 << hi;
        const uint64_t units = (uint64_t)1 << (n - 2);
        for (; i < units; i += S) {
            const uint64_t b = insert0(2 * i, hi);
            if (kind == 0 && q == 0) {
                // CNOT with target 0: swap the two amplitudes of the pair at b|control
                V x, y;
                ld2(a + (b | H), x, y);
                st2(a + (b | H), y, x);
            } else {
                V x0, x1, y0, y1;
                ld2(a + b, x0, x1);
                ld2(a + (b | H), y0, y1);
                if (kind == 0) {  // CNOT with control 0: swap (b+1) <-> (b|T)+1
                    st2(a + b, x0, y1);
                    st2(a + (b | H), y0, x1);
                } else {          // SWAP(0, hi): swap (b+1) <-> (b|H)
                    st2(a + b, x0, y0);
                    st2(a + (b | H), x1, y1);
                }
            }
        }
    }
}

// amp *= ph for amplitudes with bits p and q both set (CZ, CPHASE).
template <typename V>
__global__ void __launch_bounds__(TPB) k_phase11(V *__restrict__ a, int n, int p, int q,
                                                 const RT<V> *__restrict__ mat, int dag) {
    V ph = mkc<V>(mat[30], mat[31]);  // entry (3, 3)
    if (dag) ph = conjv(ph);
    const int lo = min(p, q), hi = max(p, q);
    const uint64_t PQ = ((uint64_t)1 << p) | ((uint64_t)1 << q);
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (lo >= 1) {
        const uint64_t units = (uint64_t)1 << (n - 3);
        for (; i < units; i += S) {
            const uint64_t b = insert00(2 * i, lo, hi) | PQ;
            V x, y;
            ld2(a + b, x, y);
            st2(a + b, cmul(x, ph), cmul(y, ph));
        }
    } else {
        // one wire is qubit 0: the odd amplitude of the 16-byte pair at b|H
        const uint64_t H = (uint64_t)1 << hi;
        const uint64_t units = (uint64_t)1 << (n - 2);
        for (; i < units; i += S) {
            const uint64_t b = insert0(2 * i, hi) | H;
            V x, y;
            ld2(a + b, x, y);
            st2(a + b, x, cmul(y, ph));
        }
    }
}

// General 4x4 on wires (w0, w1), local index 2*bit(w0) + bit(w1).
template <typename V>
__global__ void __launch_bounds__(TPB) k_dense2(V *__restrict__ a, int n, int w0, int w1,
                                                const RT<V> *__restrict__ mat, int dag) {
    V m[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            V e = dag ? conjv(mkc<V>(mat[2 * (c * 4 + r)], mat[2 * (c * 4 + r) + 1]))
                      : mkc<V>(mat[2 * (r * 4 + c)], mat[2 * (r * 4 + c) + 1]);
            m[r][c] = e;
        }
    const int lo = min(w0, w1), hi = max(w0, w1);
    const uint64_t W0 = (uint64_t)1 << w0, W1 = (uint64_t)1 << w1;
    const uint64_t units = (uint64_t)1 << (n - 2);
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < units; i += S) {
        const uint64_t b = insert00(i, lo, hi);
        const uint64_t idx[4] = {b, b | W1, b | W0, b | W0 | W1};
        V v[4], w[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) v[l] = a[idx[l]];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            V acc = cmul(m[r][0], v[0]);
#pragma unroll
            for (int c = 1; c < 4; ++c) acc = cfma(m[r][c], v[c], acc);
            w[r] = acc;
        }
#pragma unroll
        for (int l = 0; l < 4; ++l) a[idx[l]] = w[l];
    }
}

// Small states (n < 4): one thread per pair or quad, any gate, dense.
template <typename V>
__global__ void k_small(V *__restrict__ a, int n, int k, int w0, int w1, const RT<V> *__restrict__ mat, int dag) {
    const uint64_t N = (uint64_t)1 << n;
    const int d = 1 << k;
    const uint64_t units = N >> k;
    for (uint64_t i = threadIdx.x; i < units; i += blockDim.x) {
        uint64_t idx[4];
        if (k == 1) {
            const uint64_t b = insert0(i, w0);
            idx[0] = b;
            idx[1] = b | ((uint64_t)1 << w0);
        } else {
            const uint64_t b = insert00(i, min(w0, w1), max(w0, w1));
            const uint64_t W0 = (uint64_t)1 << w0, W1 = (uint64_t)1 << w1;
            idx[0] = b; idx[1] = b | W1; idx[2] = b | W0; idx[3] = b | W0 | W1;
        }
        V v[4], w[4];
        for (int l = 0; l < d; ++l) v[l] = a[idx[l]];
        for (int r = 0; r < d; ++r) {
            V acc = mkc<V>(0, 0);
            for (int c = 0; c < d; ++c) {
                V e = dag ? conjv(mkc<V>(mat[2 * (c * d + r)], mat[2 * (c * d + r) + 1]))
                          : mkc<V>(mat[2 * (r * d + c)], mat[2 * (r * d + c) + 1]);
                acc = cfma(e, v[c], acc);
            }
            w[r] = acc;
        }
        for (int l = 0; l < d; ++l) a[idx[l]] = w[l];
    }
}

template <typename V>
static cudaError_t plain_gate_t(V *a, int n, const GateH &g, const RT<V> *mat, bool dag, cudaStream_t s) {
    const int k = gate_arity(g.kind);
    const double A = (double)sizeof(V) * ((uint64_t)1 << n);  // bytes of one full read (or write)
    if (n < 4) {
        ProfScope ps(PK_SMALL, 2 * A, s);
        k_small<V><<<1, 64, 0, s>>>(a, n, k, g.w[0], k == 2 ? g.w[1] : 0, mat, dag);
        return cudaGetLastError();
    }
    const uint64_t N = (uint64_t)1 << n;
    switch (g.kind) {
    case TQD_H: case TQD_X: case TQD_Y: case TQD_RX: case TQD_RY: case TQD_UNITARY1: {
        ProfScope ps(PK_DENSE1, 2 * A, s);
        k_dense1<V><<<stream_grid(N / 4, TPB), TPB, 0, s>>>(a, n, g.w[0], mat, dag);
        break;
    }
    case TQD_Z: case TQD_S: case TQD_T: case TQD_PHASE: {
        ProfScope ps(PK_DIAG1, A, s);
        k_diag1<V><<<stream_grid(g.w[0] >= 1 ? N / 4 : N / 2, TPB), TPB, 0, s>>>(a, n, g.w[0], mat, dag, 1);
        break;
    }
    case TQD_RZ: {
        ProfScope ps(PK_DIAG1, 2 * A, s);
        k_diag1<V><<<stream_grid(N / 2, TPB), TPB, 0, s>>>(a, n, g.w[0], mat, dag, 0);
        break;
    }
    case TQD_CNOT: case TQD_SWAP: {
        const int lo = g.w[0] < g.w[1] ? g.w[0] : g.w[1];
        ProfScope ps(PK_PERM2, A, s);
        k_perm2<V><<<stream_grid(lo >= 1 ? N / 8 : N / 4, TPB), TPB, 0, s>>>(a, n, g.w[0], g.w[1],
                                                                               g.kind == TQD_CNOT ? 0 : 1);
        break;
    }
    case TQD_CZ: case TQD_CPHASE: {
        const int lo = g.w[0] < g.w[1] ? g.w[0] : g.w[1];
        ProfScope ps(PK_PHASE11, A / 2, s);
        k_phase11<V><<<stream_grid(lo >= 1 ? N / 8 : N / 4, TPB), TPB, 0, s>>>(a, n, g.w[0], g.w[1], mat, dag);
        break;
    }
    case TQD_UNITARY2: {
        ProfScope ps(PK_DENSE2, 2 * A, s);
        k_dense2<V><<<stream_grid(N / 4, TPB), TPB, 0, s>>>(a, n, g.w[0], g.w[1], mat, dag);
        break;
    }
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_gate(tqd_state *st, const tqd_circuit *c, int g, bool adjoint, cudaStream_t s) {
    const GateH &gh = c->gates[g];
    if (st->dtype == TQD_C64)
        return plain_gate_t<float2>((float2 *)st->amps, st->n, gh, c->d_mats32 + (size_t)g * MAT_STRIDE, adjoint, s);
    return plain_gate_t<double2>((double2 *)st->amps, st->n, gh, c->d_mats64 + (size_t)g * MAT_STRIDE, adjoint, s);
}

// --------------------------------------------------------- adjoint steps
// Contribution of one 1-qubit parametric gate, from the states after it:
// dE/dt = Im<lam|P|psi> for R_P(t) = exp(-i t P/2), and -2 Im<lam|P1|psi>
// for PHASE (dG/dt = i P1 G).
template <typename V>
__device__ __forceinline__ RT<V> gen1(int gen, V l0, V l1, V p0, V p1) {
    switch (gen) {
    case GEN_X: return im_cdot(l0, p1) + im_cdot(l1, p0);
    case GEN_Y: return re_cdot(l1, p0) - re_cdot(l0, p1);
    case GEN_Z: return im_cdot(l0, p0) - im_cdot(l1, p1);
    case GEN_P1: return RT<V>(-2) * im_cdot(l1, p1);
    default: return RT<V>(0);
    }
}

template <typename V>
__global__ void __launch_bounds__(TPB) k_adj1(V *__restrict__ psi, V *__restrict__ lam, int n, int t,
                                              const RT<V> *__restrict__ mat, int gen, double *__restrict__ partials) {
    __shared__ double sh[TPB / 32];
    const M2<V> md = dagger2(load_m2<V>(mat));
    KSum<RT<V>> acc;
    const uint64_t units = (uint64_t)1 << (n - 2);
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= 1) {
        const uint64_t T = (uint64_t)1 << t;
        for (; i < units; i += S) {
            const uint64_t b = insert0(2 * i, t);
            V p0, q0, p1, q1, l0, m0, l1, m1;
            ld2(psi + b, p0, q0);
            ld2(psi + b + T, p1, q1);
            ld2(lam + b, l0, m0);
            ld2(lam + b + T, l1, m1);
            if (gen) acc.add(gen1(gen, l0, l1, p0, p1) + gen1(gen, m0, m1, q0, q1));
            mv2(md, p0, p1); mv2(md, q0, q1); mv2(md, l0, l1); mv2(md, m0, m1);
            st2(psi + b, p0, q0);
            st2(psi + b + T, p1, q1);
            st2(lam + b, l0, m0);
            st2(lam + b + T, l1, m1);
        }
    } else {
        for (; i < units; i += S) {
            const uint64_t b = 4 * i;
            V p0, p1, q0, q1, l0, l1, m0, m1;
            ld2(psi + b, p0, p1);
            ld2(psi + b + 2, q0, q1);
            ld2(lam + b, l0, l1);
            ld2(lam + b + 2, m0, m1);
            if (gen) acc.add(gen1(gen, l0, l1, p0, p1) + gen1(gen, m0, m1, q0, q1));
            mv2(md, p0, p1); mv2(md, q0, q1); mv2(md, l0, l1); mv2(md, m0, m1);
            st2(psi + b, p0, p1);
            st2(psi + b + 2, q0, q1);
            st2(lam + b, l0, l1);
            st2(lam + b + 2, m0, m1);
        }
    }
    if (partials) {
        const double tot = block_sum(acc.value(), sh);
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

// CPHASE step: contribution -2 Im<lam|P11|psi>, then both states times conj(ph)
// on the |11> amplitudes.
template <typename V>
__global__ void __launch_bounds__(TPB) k_adj_phase11(V *__restrict__ psi, V *__restrict__ lam, int n, int p, int q,
                                                     const RT<V> *__restrict__ mat, int gen,
                                                     double *__restrict__ partials) {
    __shared__ double sh[TPB / 32];
    const V ph = conjv(mkc<V>(mat[30], mat[31]));
    KSum<RT<V>> acc;
    const int lo = min(p, q), hi = max(p, q);
    const uint64_t PQ = ((uint64_t)1 << p) | ((uint64_t)1 << q);
    const uint64_t units = (uint64_t)1 << (n - 2);
    const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < units; i += S) {
        const uint64_t b = insert00(i, lo, hi) | PQ;
        V x = psi[b], l = lam[b];
        if (gen) acc.add(RT<V>(-2) * im_cdot(l, x));
        psi[b] = cmul(x, ph);
        lam[b] = cmul(l, ph);
    }
    if (partials) {
        const double tot = block_sum(acc.value(), sh);
        if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    }
}

// Tiny states (n < 4): one block, any gate; dense dagger on both states.
template <typename V>
__global__ void k_adj_small(V *__restrict__ psi, V *__restrict__ lam, int n, int k, int w0, int w1,
                            const RT<V> *__restrict__ mat, int gen, double *__restrict__ partials) {
    __shared__ double sh[2];
    const uint64_t N = (uint64_t)1 << n;
    const int d = 1 << k;
    const uint64_t units = N >> k;
    double acc = 0;
    for (uint64_t i = threadIdx.x; i < units; i += blockDim.x) {
        uint64_t idx[4];
        if (k == 1) {
            const uint64_t b = insert0(i, w0);
            idx[0] = b;
            idx[1] = b | ((uint64_t)1 << w0);
        } else {
            const uint64_t b = insert00(i, min(w0, w1), max(w0, w1));
            const uint64_t W0 = (uint64_t)1 << w0, W1 = (uint64_t)1 << w1;
            idx[0] = b; idx[1] = b | W1; idx[2] = b | W0; idx[3] = b | W0 | W1;
        }
        V v[4], l[4];
        for (int j = 0; j < d; ++j) { v[j] = psi[idx[j]]; l[j] = lam[idx[j]]; }
        if (gen == GEN_P11) acc += -2.0 * (double)im_cdot(l[3], v[3]);
        else if (gen) acc += (double)gen1(gen, l[0], l[1], v[0], v[1]);
        for (int which = 0; which < 2; ++which) {
            V *x = which ? l : v;
            V w[4];
            for (int r = 0; r < d; ++r) {
                V s = mkc<V>(0, 0);
                for (int c = 0; c < d; ++c)
                    s = cfma(conjv(mkc<V>(mat[2 * (c * d + r)], mat[2 * (c * d + r) + 1])), x[c], s);
                w[r] = s;
            }
            for (int j = 0; j < d; ++j) x[j] = w[j];
        }
        for (int j = 0; j < d; ++j) { psi[idx[j]] = v[j]; lam[idx[j]] = l[j]; }
    }
    if (partials) {
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) partials[0] = sh[0] + sh[1];
    }
}

template <typename V>
static cudaError_t plain_adjoint_t(V *psi, V *lam, int n, const GateH &g, const RT<V> *mat, double *partials,
                                   int pblk, cudaStream_t s) {
    const int k = gate_arity(g.kind);
    const bool grad = partials != nullptr && g.param >= 0 && gate_parametric(g.kind);
    const int gen = grad ? gate_gen(g.kind) : GEN_NONE;
    const uint64_t N = (uint64_t)1 << n;
    const double A = (double)sizeof(V) * N;
    if (k == 1 && n >= 4) {
        int grid = stream_grid(N / 4, TPB);
        if (grid > pblk) grid = pblk;
        ProfScope ps(PK_ADJ1, 4 * A, s);
        k_adj1<V><<<grid, TPB, 0, s>>>(psi, lam, n, g.w[0], mat, gen, grad ? partials : nullptr);
        return cudaGetLastError();
    }
    if ((g.kind == TQD_CPHASE || g.kind == TQD_CZ) && n >= 4) {
        int grid = stream_grid(N / 4, TPB);
        if (grid > pblk) grid = pblk;
        ProfScope ps(PK_ADJ_PHASE11, A, s);
        k_adj_phase11<V><<<grid, TPB, 0, s>>>(psi, lam, n, g.w[0], g.w[1], mat, gen, grad ? partials : nullptr);
        return cudaGetLastError();
    }
    if (n < 4) {
        ProfScope ps(PK_ADJ_SMALL, 4 * A, s);
        k_adj_small<V><<<1, 64, 0, s>>>(psi, lam, n, k, g.w[0], k == 2 ? g.w[1] : 0, mat, gen,
                                         grad ? partials : nullptr);
        return cudaGetLastError();
    }
    // Remaining non-parametric 2-qubit steps: un-apply on each state.
    cudaError_t e = plain_gate_t<V>(psi, n, g, mat, true, s);
    if (e != cudaSuccess) return e;
    return plain_gate_t<V>(lam, n, g, mat, true, s);
}

cudaError_t launch_plain_adjoint_gate(tqd_state *psi, tqd_state *lam, const tqd_circuit *c, int g,
                                      double *partials, int pblk, cudaStream_t s) {
    const GateH &gh = c->gates[g];
    if (psi->dtype == TQD_C64)
        return plain_adjoint_t<float2>((float2 *)psi->amps, (float2 *)lam->amps, psi->n, gh,
                                       c->d_mats32 + (size_t)g * MAT_STRIDE, partials, pblk, s);
    return plain_adjoint_t<double2>((double2 *)psi->amps, (double2 *)lam->amps, psi->n, gh,
                                    c->d_mats64 + (size_t)g * MAT_STRIDE, partials, pblk, s);
}

// ------------------------------------------------------ gradient finalize
// slot_sums[s] = sum over blocks of partials[s][.] (fixed tree order).
__global__ void k_slot_sum(const double *__restrict__ partials, int pblk, int nblk, double *__restrict__ slot_sums) {
    __shared__ double sh[TPB / 32];
    const double *p = partials + (size_t)blockIdx.x * pblk;
    double v = 0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) v += p[i];
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) slot_sums[blockIdx.x] = tot;
}

// grads[p] += sum of its slots, in gate order.
__global__ void k_param_sum(const int *__restrict__ ptr, const int *__restrict__ slots,
                            const double *__restrict__ slot_sums, int nparams, double *__restrict__ grads) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nparams) return;
    double acc = 0;
    for (int k = ptr[p]; k < ptr[p + 1]; ++k) acc += slot_sums[slots[k]];
    grads[p] += acc;
}

cudaError_t launch_grad_finalize(const tqd_circuit *c, int nblk, double *dev_grads, cudaStream_t s) {
    if (c->n_slots == 0 || c->n_params == 0) return cudaSuccess;
    ProfScope ps(PK_REDUCE, 0.0, s);
    k_slot_sum<<<c->n_slots, TPB, 0, s>>>(c->d_partials, c->pblk, nblk, c->d_slot_sums);
    k_param_sum<<<(c->n_params + 127) / 128, 128, 0, s>>>(c->d_param_ptr, c->d_param_slots, c->d_slot_sums,
                                                          c->n_params, dev_grads);
    return cudaGetLastError();
}

}  // namespace tqd
