// launch.h -- host launchers of the libtqd kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace tqd {

// Grid for the full-state streaming kernels: a multiple of the SM count.
int stream_grid(uint64_t units, int threads);

// Per-gate matrices from the angles (double and float copies).
cudaError_t launch_prep(const tqd_circuit *c, const double *dev_params, cudaStream_t s);

// Matrices for an explicit gate-record array (used by batches).
cudaError_t launch_prep_raw(const GateDev *gates, int ng, const double *dev_params, const double *table,
                            double *m64, float *m32, cudaStream_t s);

// psi = e_j.
cudaError_t launch_reset(tqd_state *st, uint64_t j, cudaStream_t s);

// Gate-by-gate path: one full-state kernel for gate g (adjoint: its inverse).
cudaError_t launch_plain_gate(tqd_state *st, const tqd_circuit *c, int g, bool adjoint, cudaStream_t s);

// Gate-by-gate reverse step: contribution of gate g to its parameter's
// gradient from (psi, lambda), then both un-applied.  partials: pblk doubles.
cudaError_t launch_plain_adjoint_gate(tqd_state *psi, tqd_state *lam, const tqd_circuit *c, int g,
                                      double *partials, int pblk, cudaStream_t s);

// Sum gradient partials into grads (fixed order).
cudaError_t launch_grad_finalize(const tqd_circuit *c, int nblk, double *dev_grads, cudaStream_t s);

// Pauli sums.  mode 0: total E; mode 1: per-term values.
cudaError_t launch_expval(const tqd_state *st, const std::vector<PauliGroup> &groups, int n_terms,
                          int mode, double *dev_out, cudaStream_t s);
// out = scale * sum_j w_j c_j P_j psi.  dev_energy (may be null): also
// Re <psi|out> into dev_energy[0] (the expectation value when the weights
// and scale are 1); uses out's workspace.
cudaError_t launch_apply_observable(const tqd_state *psi, const std::vector<PauliGroup> &groups,
                                    const double *dev_weights, double scale, tqd_state *out,
                                    cudaStream_t s, double *dev_energy = nullptr);

// Shot noise (shots.cu): p = |psi|^2 (FP64); exact samples from the caller's
// uniforms; the Gaussian sample y (ybar == null) or, with ybar, the seed
// lambda = d(sum ybar y)/d conj(psi).  Use st's workspace.
cudaError_t launch_probabilities(const tqd_state *st, double *p, cudaStream_t s);
cudaError_t launch_sample(tqd_state *st, const double *uniforms, uint64_t n_shots, int64_t *out, cudaStream_t s);
cudaError_t launch_shots_gaussian(tqd_state *st, double n_shots, const double *z, const double *ybar, double *y,
                                  tqd_state *lam, cudaStream_t s);

// Grows st->work to at least `len` doubles (stream-ordered).
cudaError_t ensure_work(tqd_state *st, size_t len, cudaStream_t s);

}  // namespace tqd
