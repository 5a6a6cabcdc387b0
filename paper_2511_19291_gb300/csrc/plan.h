// plan.h -- circuit planning and the forward / backward executors (internal).
#pragma once

#include <vector>

#include "internal.h"

namespace tqd {

// Gradient slot of every parametric gate that reads the parameter vector
// (c->grad_slot, c->n_slots); returns the slots of each parameter.
std::vector<std::vector<int>> assign_grad_slots(tqd_circuit *c);

// Validated circuit -> device buffers and launch plan.
tqd_status build_circuit(tqd_circuit *c);
void release_circuit(tqd_circuit *c);

// Forward checkpoints of a gradient evaluation over fused passes [0, np):
// the state after pass np - count + k is at at(k), k < count.
struct Checkpoints {
    char *base = nullptr;
    size_t stride = 0;
    int count = 0;
    void *psi0 = nullptr;  // a slot for a copy of the input state (want_psi0), else null
    void *at(int k) const { return base + (size_t)k * stride; }
};

// Checkpoint memory of circuit c for states like psi over np passes, sized
// by the circuit's option and half the free device memory the first time a
// state size is seen (cudaMalloc then, so not inside a stream capture);
// count 0 when the plan is not fused or nothing fits.  want_psi0: when some
// pass would still run in place, one slot (the last) holds a copy of the
// input state instead of a pass's output (psi0; null when there is no slot).
cudaError_t checkpoints_for(const tqd_circuit *c, const tqd_state *psi, int np, Checkpoints *out,
                            bool want_psi0 = false);

// psi <- U psi (prep + plain or fused passes); pass_end >= 0: only the fused
// passes [0, pass_end).  ck (fused): the last ck->count passes write their
// states to the checkpoints instead of psi, which keeps the state before them.
cudaError_t run_forward(tqd_state *psi, const tqd_circuit *c, const double *dev_params, cudaStream_t s,
                        int pass_end = -1, const Checkpoints *ck = nullptr);

// lambda = scale * H psi, reverse sweep, gradients accumulated into dev_grads.
// dev_energy (may be null): Re <psi|lambda> before the sweep.  prepared: the
// gate matrices of dev_params are already on the device (skip the prep).
// pass_end >= 0: the sweep starts at fused pass pass_end - 1; it ends at
// pass_begin (the passes before it are not un-applied).  seeded: lam
// already holds the seed (groups, weights and scale are not used).  ck: the
// checkpoints run_forward wrote (the final state is the last one; those
// passes read psi there and leave it; the earlier ones recompute psi in
// place, which ends as the input state of the forward run either way).
cudaError_t run_backward(tqd_state *psi, tqd_state *lam, const tqd_circuit *c, const double *dev_params,
                         const std::vector<PauliGroup> &groups, const double *dev_weights, double scale,
                         double *dev_grads, cudaStream_t s, double *dev_energy = nullptr, bool prepared = false,
                         int pass_end = -1, bool seeded = false, const Checkpoints *ck = nullptr,
                         int pass_begin = 0);

// The Pauli terms of P^dagger H P for the circuit's permutation tail P
// (gates tail_gate.. in order): masks and signs after conjugation by each
// CNOT, SWAP and X.  E = <P psi|H|P psi> = <psi|H'|psi>.
std::vector<tqd_pauli_term> conjugate_by_tail(const tqd_circuit *c, const tqd_pauli_term *terms, size_t n_terms);

}  // namespace tqd
