// internal.h -- host-side structures of libtqd (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "tile.h"
#include "tqd.h"

namespace tqd {

void set_error(const char *fmt, ...);
int device_sm_count();

// Gate as stored by the library (validated copy of tqd_gate).
struct GateH {
    int kind;
    int nw;
    int w[3];
    int param;
    double fixed;
    int mat;
};

// Record read by the matrix-preparation kernel.
struct GateDev {
    int32_t kind;
    int32_t param;
    int32_t mat;
    int32_t pad;
    double fixed;
};

__host__ __device__ inline int gate_arity(int kind) {
    switch (kind) {
    case TQD_CNOT: case TQD_CZ: case TQD_CPHASE: case TQD_SWAP: case TQD_UNITARY2: return 2;
    default: return 1;
    }
}
__host__ __device__ inline bool gate_parametric(int kind) {
    return kind == TQD_RX || kind == TQD_RY || kind == TQD_RZ || kind == TQD_PHASE || kind == TQD_CPHASE;
}
__host__ __device__ inline bool gate_diagonal(int kind) {
    return kind == TQD_Z || kind == TQD_S || kind == TQD_T || kind == TQD_RZ || kind == TQD_PHASE ||
           kind == TQD_CZ || kind == TQD_CPHASE;
}
__host__ __device__ inline int gate_gen(int kind) {
    switch (kind) {
    case TQD_RX: return GEN_X;
    case TQD_RY: return GEN_Y;
    case TQD_RZ: return GEN_Z;
    case TQD_PHASE: return GEN_P1;
    case TQD_CPHASE: return GEN_P11;
    default: return GEN_NONE;
    }
}

// Pauli term grouped for the kernels: a group shares one x mask.
struct TermDev {
    uint64_t zmask;
    double coeff;
    double pre, pim;  // i^{|x&z|}
    int32_t index;    // position in the caller's term list (weights, per-term outputs)
    int32_t pad;
};

struct PauliGroup {
    uint64_t xmask;
    std::vector<TermDev> terms;
};
std::vector<PauliGroup> group_terms(const tqd_pauli_term *terms, size_t n_terms);

}  // namespace tqd

struct tqd_state {
    int n;
    tqd_dtype dtype;
    void *amps;
    size_t bytes;
    int device;
    double *work;       // reduction workspace (device, stream-ordered allocation), grown on demand
    size_t work_len;    // doubles
    cudaStream_t work_stream;  // stream of the workspace's last use: it is released in that stream's order
};

struct tqd_circuit {
    int n;
    int n_params;
    int device;
    tqd_plan_opts opts;
    std::vector<tqd::GateH> gates;
    std::vector<double> table;
    // device copies
    tqd::GateDev *d_gates;
    double *d_table;
    double *d_mats64;  // [n_gates][MAT_STRIDE]
    float *d_mats32;   // [n_gates][MAT_STRIDE]
    // gradient bookkeeping: one slot per parametric gate with param >= 0
    std::vector<int> grad_slot;  // per gate: slot index or -1
    int n_slots;
    int pblk;                    // partials per slot
    double *d_partials;          // [n_slots][pblk]
    double *d_slot_sums;         // [n_slots]
    int *d_param_ptr;            // CSR: param -> slots (n_params + 1)
    int *d_param_slots;
    int launches_apply;
    int launches_backward;
    int n_passes;
    bool fused;                  // tile passes (n >= 12) instead of the gate-by-gate plan
    int prefix_passes;           // fused: passes of the gates before the permutation tail
    int tail_gate;               // fused: first gate of the permutation tail (gates.size(): none)
    int first_grad_pass;         // fused: first pass with an angle (passes before it have none)
    std::vector<tqd::TilePlanPass> tile_passes;
    std::vector<void *> tc_blocks;   // tqd::TcBlock*, forward of passes whose gates all act on qubits 0..5
    tqd::TilePassDev *d_tile_desc;  // [pass][c64, c128] descriptors in device memory
    int *d_err;                  // device error word (bounded waits that gave up, failed checks)
    mutable int test_stall = 0;  // tqd_circuit_test_stall: tile passes launch with TILE_STALL_TEST
    // pass-specialised kernels (CUfunction) per [precision][direction][kind][pass]
    // (kind: tqd::jit_kind of the buffer layout and whether psi is read-only),
    // compiled on first use; nullptr entries run the generic kernel
    mutable std::mutex jit_mu;
    mutable std::vector<void *> jit_fn[2][2][6];
    mutable bool jit_ready[2][2][6] = {};
    // forward checkpoints of tqd_value_and_grad (device memory, sized on first use)
    mutable std::mutex ck_mu;
    mutable void *ck_buf = nullptr;
    mutable size_t ck_bytes = 0;        // allocated
    mutable size_t ck_state_bytes = 0;  // state size the allocation was sized for
};
