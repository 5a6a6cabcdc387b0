// api.cu -- the extern "C" entry points of libtqd: argument validation on the
// host, handle management, and dispatch to the kernel launchers.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "jit.h"
#include "launch.h"
#include "plan.h"
#include "tile_plan.h"

namespace tqd {

static thread_local std::string g_error;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_error = buf;
}

int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        cache[dev] = v;
    }
    return cache[dev];
}

// Makes `dev` current for the scope of one call and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static size_t amp_bytes(tqd_dtype d) { return d == TQD_C64 ? 8 : 16; }

}  // namespace tqd

using namespace tqd;

#define CHECK_ARG(cond, ...)                  \
    do {                                      \
        if (!(cond)) {                        \
            tqd::set_error(__VA_ARGS__);      \
            return TQD_ERR_INVALID_ARG;       \
        }                                     \
    } while (0)

#define CHECK_CUDA(expr)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            /* the specialised-kernel errors keep the message they set */                 \
            if (e_ == cudaErrorNotSupported) return TQD_ERR_UNSUPPORTED;                  \
            if (e_ != cudaErrorInvalidSource && e_ != cudaErrorInvalidKernelImage)        \
                tqd::set_error("%s failed: %s", #expr, cudaGetErrorString(e_));           \
            return e_ == cudaErrorMemoryAllocation ? TQD_ERR_OOM : TQD_ERR_CUDA;          \
        }                                                                                 \
    } while (0)

#define GUARD(dev)                                                       \
    DeviceGuard guard_(dev);                                             \
    if (!guard_.ok) {                                                    \
        tqd::set_error("cannot make device %d current", (int)(dev));     \
        return TQD_ERR_CUDA;                                             \
    }

extern "C" {

const char *tqd_last_error(void) { return g_error.c_str(); }

const char *tqd_version(void) { return "tqd 0.1 (sm_103a)"; }

// ----------------------------------------------------------------- states
tqd_status tqd_state_alloc(int n_qubits, tqd_dtype dtype, void *dev_amps, size_t bytes, tqd_state **out) {
    CHECK_ARG(out != nullptr, "tqd_state_alloc: out is NULL");
    *out = nullptr;
    CHECK_ARG(n_qubits >= 1 && n_qubits <= 34, "tqd_state_alloc: n_qubits %d outside [1, 34]", n_qubits);
    CHECK_ARG(dtype == TQD_C64 || dtype == TQD_C128, "tqd_state_alloc: unknown dtype %d", (int)dtype);
    CHECK_ARG(dev_amps != nullptr, "tqd_state_alloc: dev_amps is NULL");
    CHECK_ARG(((uintptr_t)dev_amps & 255) == 0, "tqd_state_alloc: dev_amps is not 256-byte aligned");
    const size_t need = ((size_t)1 << n_qubits) * amp_bytes(dtype);
    CHECK_ARG(bytes >= need, "tqd_state_alloc: buffer of %zu bytes, %d qubits need %zu", bytes, n_qubits, need);
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, dev_amps);
    if (e != cudaSuccess) {
        set_error("tqd_state_alloc: cudaPointerGetAttributes: %s", cudaGetErrorString(e));
        return TQD_ERR_CUDA;
    }
    CHECK_ARG(attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged,
              "tqd_state_alloc: dev_amps is not device memory");
    tqd_state *s = new (std::nothrow) tqd_state;
    if (!s) {
        set_error("tqd_state_alloc: out of host memory");
        return TQD_ERR_OOM;
    }
    s->n = n_qubits;
    s->dtype = dtype;
    s->amps = dev_amps;
    s->bytes = bytes;
    s->device = attr.device;
    s->work = nullptr;
    s->work_len = 0;
    s->work_stream = nullptr;
    *out = s;
    return TQD_OK;
}

tqd_status tqd_state_reset(tqd_state *state, uint64_t basis_index, void *stream) {
    CHECK_ARG(state != nullptr, "tqd_state_reset: state is NULL");
    CHECK_ARG(basis_index < ((uint64_t)1 << state->n), "tqd_state_reset: basis index out of range");
    GUARD(state->device);
    CHECK_CUDA(launch_reset(state, basis_index, (cudaStream_t)stream));
    return TQD_OK;
}

tqd_status tqd_state_free(tqd_state *state) {
    if (!state) return TQD_OK;
    if (state->work) {
        // kernels queued on the workspace's stream may still use it: release
        // it in that stream's order (a plain cudaFree of a stream-ordered
        // allocation does not wait for them)
        DeviceGuard g(state->device);
        cudaFreeAsync(state->work, state->work_stream);
    }
    delete state;
    return TQD_OK;
}

// --------------------------------------------------------------- circuits
// Validates a gate list and the plan options; fills *o and *gs.
static tqd_status validate_circuit(int n_qubits, const tqd_gate *gates, size_t n_gates, int n_params,
                                   const double *matrices, size_t n_matrix_entries, const tqd_plan_opts *opts,
                                   tqd_plan_opts *o_out, std::vector<GateH> *gs_out) {
    CHECK_ARG(n_qubits >= 1 && n_qubits <= 34, "tqd_circuit_create: n_qubits %d outside [1, 34]", n_qubits);
    CHECK_ARG(n_gates == 0 || gates != nullptr, "tqd_circuit_create: gates is NULL");
    CHECK_ARG(n_gates <= (1u << 24), "tqd_circuit_create: too many gates");
    CHECK_ARG(n_params >= 0, "tqd_circuit_create: negative n_params");
    CHECK_ARG(n_matrix_entries == 0 || matrices != nullptr, "tqd_circuit_create: matrices is NULL");
    tqd_plan_opts &o = *o_out;
    memset(&o, 0, sizeof(o));
    o.mode = TQD_PLAN_FUSED;
    if (opts) {
        o = *opts;
        CHECK_ARG(o.mode == TQD_PLAN_PLAIN || o.mode == TQD_PLAN_FUSED || o.mode == TQD_PLAN_TC,
                  "tqd_circuit_create: unknown plan mode");
        CHECK_ARG(o.buffers <= 4, "tqd_circuit_create: buffers %u not in {0, ..., 4}", o.buffers);
        CHECK_ARG(o.jit <= 2, "tqd_circuit_create: jit %u not in {0, 1, 2}", o.jit);
        CHECK_ARG(o.tile_qubits == 0 || o.tile_qubits == (uint32_t)tqd::TILE_K,
                  "tqd_circuit_create: tile_qubits %u not in {0, %d} (the tile kernels hold 2^%d amplitudes)",
                  o.tile_qubits, tqd::TILE_K, tqd::TILE_K);
        CHECK_ARG(o.low_qubits == 0 || o.low_qubits == (uint32_t)tqd::TILE_LOW,
                  "tqd_circuit_create: low_qubits %u not in {0, %d}", o.low_qubits, tqd::TILE_LOW);
        CHECK_ARG(o.reserved[0] == 0, "tqd_circuit_create: reserved opts not zero");
    }
    std::vector<GateH> &gs = *gs_out;
    gs.assign(n_gates, GateH());
    for (size_t i = 0; i < n_gates; ++i) {
        const tqd_gate &g = gates[i];
        CHECK_ARG(g.kind <= TQD_UNITARY2, "gate %zu: unknown kind %u", i, g.kind);
        const int k = gate_arity((int)g.kind);
        CHECK_ARG((int)g.nwires == k, "gate %zu: kind %u takes %d wires, got %u", i, g.kind, k, g.nwires);
        for (int a = 0; a < k; ++a) {
            CHECK_ARG(g.wires[a] < (uint32_t)n_qubits, "gate %zu: wire %u >= n_qubits %d", i, g.wires[a], n_qubits);
            for (int b = 0; b < a; ++b)
                CHECK_ARG(g.wires[a] != g.wires[b], "gate %zu: duplicate wire %u", i, g.wires[a]);
        }
        if (g.param_idx >= 0) {
            CHECK_ARG(gate_parametric((int)g.kind), "gate %zu: kind %u takes no angle", i, g.kind);
            CHECK_ARG(g.param_idx < n_params, "gate %zu: param_idx %d >= n_params %d", i, g.param_idx, n_params);
        } else {
            CHECK_ARG(g.param_idx == -1, "gate %zu: param_idx %d (use -1 for a fixed angle)", i, g.param_idx);
        }
        if (!isfinite(g.fixed)) {
            set_error("gate %zu: non-finite fixed angle", i);
            return TQD_ERR_NUMERIC;
        }
        if (g.kind == TQD_UNITARY1 || g.kind == TQD_UNITARY2) {
            const size_t d2 = g.kind == TQD_UNITARY1 ? 4 : 16;
            CHECK_ARG(g.mat_idx >= 0 && (size_t)g.mat_idx + d2 <= n_matrix_entries,
                      "gate %zu: matrix index %d outside the table of %zu entries", i, g.mat_idx, n_matrix_entries);
        }
        GateH &h = gs[i];
        h.kind = (int)g.kind;
        h.nw = k;
        for (int a = 0; a < 3; ++a) h.w[a] = a < k ? (int)g.wires[a] : 0;
        h.param = g.param_idx;
        h.fixed = g.fixed;
        h.mat = (g.kind == TQD_UNITARY1 || g.kind == TQD_UNITARY2) ? g.mat_idx : -1;
    }
    for (size_t i = 0; i < 2 * n_matrix_entries; ++i) {
        if (!isfinite(matrices[i])) {
            set_error("tqd_circuit_create: non-finite matrix entry");
            return TQD_ERR_NUMERIC;
        }
    }
    return TQD_OK;
}

tqd_status tqd_circuit_create(int n_qubits, const tqd_gate *gates, size_t n_gates, int n_params,
                              const double *matrices, size_t n_matrix_entries, const tqd_plan_opts *opts,
                              tqd_circuit **out) {
    CHECK_ARG(out != nullptr, "tqd_circuit_create: out is NULL");
    *out = nullptr;
    tqd_plan_opts o;
    std::vector<GateH> gs;
    const tqd_status vs = validate_circuit(n_qubits, gates, n_gates, n_params, matrices, n_matrix_entries, opts, &o, &gs);
    if (vs != TQD_OK) return vs;
    tqd_circuit *c = new (std::nothrow) tqd_circuit();
    if (!c) {
        set_error("tqd_circuit_create: out of host memory");
        return TQD_ERR_OOM;
    }
    c->n = n_qubits;
    c->n_params = n_params;
    c->opts = o;
    c->gates = std::move(gs);
    c->table.assign(matrices ? matrices : (const double *)nullptr,
                    matrices ? matrices + 2 * n_matrix_entries : (const double *)nullptr);
    tqd_status st = build_circuit(c);
    if (st != TQD_OK) {
        tqd_circuit_free(c);
        return st;
    }
    *out = c;
    return TQD_OK;
}

tqd_status tqd_circuit_free(tqd_circuit *c) {
    if (!c) return TQD_OK;
    GUARD(c->device);  // its buffers (forward checkpoints included) belong to that device
    // work queued with the circuit may still read its buffers
    cudaDeviceSynchronize();
    release_circuit(c);
    delete c;
    return TQD_OK;
}

tqd_status tqd_jit_check(int n_qubits, const tqd_gate *gates, size_t n_gates, int n_params, const double *matrices,
                         size_t n_matrix_entries, int arch, int *n_kernels) {
    CHECK_ARG(n_kernels != nullptr, "tqd_jit_check: n_kernels is NULL");
    *n_kernels = 0;
    CHECK_ARG(arch >= 100 && arch < 1000, "tqd_jit_check: arch %d is not a compute capability like 103", arch);
    tqd_plan_opts o;
    std::vector<GateH> gs;
    const tqd_status vs = validate_circuit(n_qubits, gates, n_gates, n_params, matrices, n_matrix_entries, nullptr, &o,
                                           &gs);
    if (vs != TQD_OK) return vs;
    CHECK_ARG(n_qubits >= TILE_K && n_gates > 0, "tqd_jit_check: fused passes need >= %d qubits and a gate", TILE_K);
    tqd_circuit c;
    c.n = n_qubits;
    c.n_params = n_params;
    c.opts = o;
    c.gates = std::move(gs);
    return jit_check_host(&c, arch, n_kernels);
}

tqd_status tqd_plan_check(int n_qubits, const tqd_gate *gates, size_t n_gates, int n_params, const double *matrices,
                          size_t n_matrix_entries, const double *params, uint64_t seed, double *err_forward,
                          double *err_reverse, int *n_passes, int *n_stages) {
    CHECK_ARG(err_forward != nullptr && err_reverse != nullptr, "tqd_plan_check: NULL error output");
    tqd_plan_opts o;
    std::vector<GateH> gs;
    const tqd_status vs = validate_circuit(n_qubits, gates, n_gates, n_params, matrices, n_matrix_entries, nullptr, &o,
                                           &gs);
    if (vs != TQD_OK) return vs;
    CHECK_ARG(n_qubits >= TILE_K && n_qubits <= 20 && n_gates > 0,
              "tqd_plan_check: needs %d..20 qubits and a gate", TILE_K);
    CHECK_ARG(n_params == 0 || params != nullptr, "tqd_plan_check: params is NULL");
    tqd_circuit c;
    c.n = n_qubits;
    c.n_params = n_params;
    c.opts = o;
    c.gates = std::move(gs);
    c.table.assign(matrices ? matrices : (const double *)nullptr,
                   matrices ? matrices + 2 * n_matrix_entries : (const double *)nullptr);
    return tqd::plan_check_host(&c, params, seed, err_forward, err_reverse, n_passes, n_stages);
}

tqd_status tqd_circuit_info(const tqd_circuit *c, int *n_passes, int *n_launches_apply, int *n_launches_backward) {
    CHECK_ARG(c != nullptr, "tqd_circuit_info: circuit is NULL");
    if (n_passes) *n_passes = c->n_passes;
    if (n_launches_apply) *n_launches_apply = c->launches_apply;
    if (n_launches_backward) *n_launches_backward = c->launches_backward;
    return TQD_OK;
}

tqd_status tqd_circuit_check(const tqd_circuit *c, int *device_error) {
    CHECK_ARG(c != nullptr && device_error != nullptr, "tqd_circuit_check: NULL argument");
    GUARD(c->device);
    int v = 0;
    CHECK_CUDA(cudaMemcpy(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    *device_error = v;
    if (v != 0) CHECK_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
    if (v == 1) {
        tqd::set_error("tqd_circuit_check: a bounded wait for a tile copy gave up");
        return TQD_ERR_TIMEOUT;
    }
    if (v != 0) {
        tqd::set_error("tqd_circuit_check: a checked kernel found an index out of range (code %d)", v);
        return TQD_ERR_NUMERIC;
    }
    return TQD_OK;
}

tqd_status tqd_circuit_test_stall(tqd_circuit *c, int enable) {
    CHECK_ARG(c != nullptr, "tqd_circuit_test_stall: circuit is NULL");
    c->test_stall = enable != 0;
    return TQD_OK;
}

tqd_status tqd_apply_circuit(tqd_state *state, const tqd_circuit *c, const double *dev_params, void *stream) {
    CHECK_ARG(state != nullptr && c != nullptr, "tqd_apply_circuit: NULL state or circuit");
    CHECK_ARG(state->n == c->n, "tqd_apply_circuit: state has %d qubits, circuit %d", state->n, c->n);
    CHECK_ARG(c->n_params == 0 || dev_params != nullptr, "tqd_apply_circuit: dev_params is NULL");
    GUARD(state->device);
    CHECK_CUDA(run_forward(state, c, dev_params, (cudaStream_t)stream));
    return TQD_OK;
}

// ------------------------------------------------------------ observables
static tqd_status check_terms(const tqd_state *st, const tqd_pauli_term *terms, size_t n_terms, const char *who) {
    CHECK_ARG(n_terms == 0 || terms != nullptr, "%s: terms is NULL", who);
    const uint64_t lim = st->n >= 64 ? ~0ull : (((uint64_t)1 << st->n) - 1);
    for (size_t j = 0; j < n_terms; ++j) {
        CHECK_ARG((terms[j].xmask & ~lim) == 0 && (terms[j].zmask & ~lim) == 0,
                  "%s: term %zu acts on a qubit >= %d", who, j, st->n);
        if (!isfinite(terms[j].coeff)) {
            set_error("%s: term %zu has a non-finite coefficient", who, j);
            return TQD_ERR_NUMERIC;
        }
    }
    return TQD_OK;
}

tqd_status tqd_expval(const tqd_state *state, const tqd_pauli_term *terms, size_t n_terms, double *dev_out,
                      void *stream) {
    CHECK_ARG(state != nullptr, "tqd_expval: state is NULL");
    CHECK_ARG(dev_out != nullptr, "tqd_expval: dev_out is NULL");
    tqd_status st = check_terms(state, terms, n_terms, "tqd_expval");
    if (st != TQD_OK) return st;
    GUARD(state->device);
    CHECK_CUDA(launch_expval(state, group_terms(terms, n_terms), (int)n_terms, 0, dev_out, (cudaStream_t)stream));
    return TQD_OK;
}

tqd_status tqd_expval_terms(const tqd_state *state, const tqd_pauli_term *terms, size_t n_terms, double *dev_out,
                            void *stream) {
    CHECK_ARG(state != nullptr, "tqd_expval_terms: state is NULL");
    CHECK_ARG(n_terms == 0 || dev_out != nullptr, "tqd_expval_terms: dev_out is NULL");
    CHECK_ARG(n_terms < (1u << 20), "tqd_expval_terms: too many terms");
    tqd_status st = check_terms(state, terms, n_terms, "tqd_expval_terms");
    if (st != TQD_OK) return st;
    GUARD(state->device);
    CHECK_CUDA(launch_expval(state, group_terms(terms, n_terms), (int)n_terms, 1, dev_out, (cudaStream_t)stream));
    return TQD_OK;
}

tqd_status tqd_apply_observable(const tqd_state *psi, const tqd_pauli_term *terms, size_t n_terms,
                                const double *dev_weights, tqd_state *out, void *stream) {
    CHECK_ARG(psi != nullptr && out != nullptr, "tqd_apply_observable: NULL state");
    CHECK_ARG(psi != out && psi->amps != out->amps, "tqd_apply_observable: out must not alias psi");
    CHECK_ARG(psi->n == out->n && psi->dtype == out->dtype, "tqd_apply_observable: state shapes differ");
    tqd_status st = check_terms(psi, terms, n_terms, "tqd_apply_observable");
    if (st != TQD_OK) return st;
    GUARD(psi->device);
    CHECK_CUDA(launch_apply_observable(psi, group_terms(terms, n_terms), dev_weights, 1.0, out,
                                       (cudaStream_t)stream));
    return TQD_OK;
}

// ---------------------------------------------------------------- adjoint
tqd_status tqd_backward(tqd_state *psi, tqd_state *lambda, const tqd_circuit *c, const double *dev_params,
                        const tqd_pauli_term *terms, size_t n_terms, const double *dev_term_weights,
                        double grad_scale, double *dev_grads, void *stream) {
    CHECK_ARG(psi != nullptr && lambda != nullptr && c != nullptr, "tqd_backward: NULL handle");
    CHECK_ARG(psi != lambda && psi->amps != lambda->amps, "tqd_backward: lambda must not alias psi");
    CHECK_ARG(psi->n == c->n && lambda->n == c->n, "tqd_backward: qubit counts differ");
    CHECK_ARG(psi->dtype == lambda->dtype, "tqd_backward: psi and lambda dtypes differ");
    CHECK_ARG(c->n_params == 0 || dev_params != nullptr, "tqd_backward: dev_params is NULL");
    CHECK_ARG(c->n_params == 0 || dev_grads != nullptr, "tqd_backward: dev_grads is NULL");
    if (!isfinite(grad_scale)) {
        tqd::set_error("tqd_backward: non-finite grad_scale");
        return TQD_ERR_NUMERIC;
    }
    tqd_status st = check_terms(psi, terms, n_terms, "tqd_backward");
    if (st != TQD_OK) return st;
    GUARD(psi->device);
    CHECK_CUDA(run_backward(psi, lambda, c, dev_params, group_terms(terms, n_terms), dev_term_weights, grad_scale,
                            dev_grads, (cudaStream_t)stream));
    return TQD_OK;
}

tqd_status tqd_backward_seeded(tqd_state *psi, tqd_state *lambda, const tqd_circuit *c, const double *dev_params,
                               double *dev_grads, void *stream) {
    CHECK_ARG(psi != nullptr && lambda != nullptr && c != nullptr, "tqd_backward_seeded: NULL handle");
    CHECK_ARG(psi != lambda && psi->amps != lambda->amps, "tqd_backward_seeded: lambda must not alias psi");
    CHECK_ARG(psi->n == c->n && lambda->n == c->n, "tqd_backward_seeded: qubit counts differ");
    CHECK_ARG(psi->dtype == lambda->dtype, "tqd_backward_seeded: psi and lambda dtypes differ");
    CHECK_ARG(c->n_params == 0 || dev_params != nullptr, "tqd_backward_seeded: dev_params is NULL");
    CHECK_ARG(c->n_params == 0 || dev_grads != nullptr, "tqd_backward_seeded: dev_grads is NULL");
    GUARD(psi->device);
    CHECK_CUDA(run_backward(psi, lambda, c, dev_params, {}, nullptr, 1.0, dev_grads, (cudaStream_t)stream, nullptr,
                            false, -1, true));
    return TQD_OK;
}

tqd_status tqd_probabilities(const tqd_state *state, double *dev_p, void *stream) {
    CHECK_ARG(state != nullptr && dev_p != nullptr, "tqd_probabilities: NULL argument");
    GUARD(state->device);
    CHECK_CUDA(launch_probabilities(state, dev_p, (cudaStream_t)stream));
    return TQD_OK;
}

tqd_status tqd_sample(tqd_state *state, const double *dev_uniforms, size_t n_shots, int64_t *dev_samples,
                      void *stream) {
    CHECK_ARG(state != nullptr, "tqd_sample: state is NULL");
    CHECK_ARG(n_shots == 0 || (dev_uniforms != nullptr && dev_samples != nullptr), "tqd_sample: NULL buffer");
    GUARD(state->device);
    CHECK_CUDA(launch_sample(state, dev_uniforms, n_shots, dev_samples, (cudaStream_t)stream));
    return TQD_OK;
}

tqd_status tqd_shots_gaussian(tqd_state *state, double n_shots, const double *dev_z, double *dev_y, void *stream) {
    CHECK_ARG(state != nullptr && dev_z != nullptr && dev_y != nullptr, "tqd_shots_gaussian: NULL argument");
    CHECK_ARG(isfinite(n_shots) && n_shots >= 0, "tqd_shots_gaussian: n_shots must be finite and >= 0");
    GUARD(state->device);
    CHECK_CUDA(launch_shots_gaussian(state, n_shots, dev_z, nullptr, dev_y, nullptr, (cudaStream_t)stream));
    return TQD_OK;
}

tqd_status tqd_shots_gaussian_backward(tqd_state *state, double n_shots, const double *dev_z,
                                       const double *dev_ybar, tqd_state *lambda, void *stream) {
    CHECK_ARG(state != nullptr && lambda != nullptr && dev_z != nullptr && dev_ybar != nullptr,
              "tqd_shots_gaussian_backward: NULL argument");
    CHECK_ARG(state != lambda && state->amps != lambda->amps, "tqd_shots_gaussian_backward: lambda must not alias psi");
    CHECK_ARG(state->n == lambda->n && state->dtype == lambda->dtype,
              "tqd_shots_gaussian_backward: lambda differs from psi in qubits or dtype");
    CHECK_ARG(isfinite(n_shots) && n_shots >= 0, "tqd_shots_gaussian_backward: n_shots must be finite and >= 0");
    GUARD(state->device);
    CHECK_CUDA(launch_shots_gaussian(state, n_shots, dev_z, dev_ybar, nullptr, lambda, (cudaStream_t)stream));
    return TQD_OK;
}

tqd_status tqd_value_and_grad(tqd_state *psi, tqd_state *lambda, const tqd_circuit *c, const double *dev_params,
                              const tqd_pauli_term *terms, size_t n_terms, double *dev_energy, double *dev_grads,
                              void *stream) {
    CHECK_ARG(psi != nullptr && lambda != nullptr && c != nullptr, "tqd_value_and_grad: NULL handle");
    CHECK_ARG(psi != lambda && psi->amps != lambda->amps, "tqd_value_and_grad: lambda must not alias psi");
    CHECK_ARG(psi->n == c->n && lambda->n == c->n, "tqd_value_and_grad: qubit counts differ");
    CHECK_ARG(psi->dtype == lambda->dtype, "tqd_value_and_grad: psi and lambda dtypes differ");
    CHECK_ARG(c->n_params == 0 || dev_params != nullptr, "tqd_value_and_grad: dev_params is NULL");
    CHECK_ARG(c->n_params == 0 || dev_grads != nullptr, "tqd_value_and_grad: dev_grads is NULL");
    CHECK_ARG(dev_energy != nullptr, "tqd_value_and_grad: dev_energy is NULL");
    tqd_status st = check_terms(psi, terms, n_terms, "tqd_value_and_grad");
    if (st != TQD_OK) return st;
    GUARD(psi->device);
    const cudaStream_t s = (cudaStream_t)stream;
    const bool tail = c->fused && c->prefix_passes < (int)c->tile_passes.size();
    const int np = c->fused ? (tail ? c->prefix_passes : (int)c->tile_passes.size()) : 0;
    // Passes before the first one with an angle have no derivative to take:
    // the reverse sweep ends there.  psi is then restored from a copy of the
    // input state kept in a checkpoint slot, when some pass runs in place.
    const int lead = c->fused ? std::min(c->first_grad_pass, np) : 0;
    // forward checkpoints of the passes that run (the last ones that fit)
    Checkpoints ck;
    CHECK_CUDA(checkpoints_for(c, psi, np, &ck, lead > 0));
    const bool in_place = np - ck.count > 0;
    const int pass_begin = lead > 0 && (!in_place || ck.psi0) ? lead : 0;
    const bool restore = pass_begin > 0 && in_place;
    const size_t sb = ((size_t)1 << psi->n) * (psi->dtype == TQD_C64 ? 8 : 16);
    if (restore) CHECK_CUDA(cudaMemcpyAsync(ck.psi0, psi->amps, sb, cudaMemcpyDeviceToDevice, s));
    if (tail) {
        // the circuit ends with a permutation P (its tail passes): E and its
        // gradient from psi' = U' psi (the gates before P) with
        // H' = P^dagger H P; the tail passes never run
        const std::vector<tqd_pauli_term> hp = conjugate_by_tail(c, terms, n_terms);
        CHECK_CUDA(run_forward(psi, c, dev_params, s, c->prefix_passes, &ck));
        CHECK_CUDA(run_backward(psi, lambda, c, dev_params, group_terms(hp.data(), hp.size()), nullptr, 1.0,
                                dev_grads, s, dev_energy, true, c->prefix_passes, false, &ck, pass_begin));
    } else {
        CHECK_CUDA(run_forward(psi, c, dev_params, s, -1, &ck));
        CHECK_CUDA(run_backward(psi, lambda, c, dev_params, group_terms(terms, n_terms), nullptr, 1.0, dev_grads, s,
                                dev_energy, true, -1, false, &ck, pass_begin));
    }
    if (restore) CHECK_CUDA(cudaMemcpyAsync(psi->amps, ck.psi0, sb, cudaMemcpyDeviceToDevice, s));
    return TQD_OK;
}

}  // extern "C"
