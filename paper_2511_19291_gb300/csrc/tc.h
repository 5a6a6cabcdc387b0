// tc.h -- fused 6-qubit blocks on the tensor cores (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace tqd {

// One gate of a block: wires are qubits 0..5 (local index bits).
struct TcGate {
    int32_t gate;  // circuit gate index (row of the per-gate matrices)
    uint8_t nw, w0, w1, pad;
};

// Device buffers of one block: its gates and the 128 x 128 real embedding of
// the fused unitary, TF32 hi / lo halves in the tensor-core operand layout.
struct TcBlock {
    TcGate *d_gates;
    int n_gates;
    float *d_ahi;
    float *d_alo;
};

// Builds the block's fused unitary U from the current angles (U^dagger when
// adj) and applies it to every 64-amplitude column of psi (complex64,
// n >= 12), then of `second` when given (the reverse sweep's lambda).
cudaError_t launch_tc_block(tqd_state *psi, const tqd_circuit *c, const TcBlock &blk, cudaStream_t s,
                            bool adj = false, tqd_state *second = nullptr);

// A pass the reverse sweep runs on the tensor cores: a tensor-core block with
// no angle derivative to take (its gates are fixed), so un-applying it is one
// product with U^dagger per state.
inline bool tc_reverse_pass(const TilePlanPass &p) { return p.tc >= 0 && p.dev[0].h.n_grad == 0; }

}  // namespace tqd
