// tile_plan.h -- host-side plan of the fused tile passes (internal).
#pragma once

#include <cuda.h>

#include <vector>

#include "internal.h"
#include "tile.h"

namespace tqd {

bool tile_layout(int n, const std::vector<char> &inQ, TileLayout &L);
// Empty result: the circuit cannot be planned into tiles (the caller falls
// back to the gate-by-gate plan).  Plans gates [g_begin, g_end) (g_end < 0:
// to the end).
std::vector<TilePlanPass> plan_tile_passes(const tqd_circuit *c, int g_begin = 0, int g_end = -1);

// Lazy qubit order for the fused plans: every SWAP of the gate list becomes a
// relabelling of the qubits of the gates after it, and the permutation left
// at the end is appended as SWAP gates (part of the permutation tail).
// Returns whether the list changed.
bool relabel_swaps(std::vector<GateH> &gates, int n);

// First gate of the circuit's permutation tail: the longest suffix of CNOT,
// SWAP and X gates (gates.size() when the circuit does not end with one).
int permutation_tail(const tqd_circuit *c);

// The fused plan: the gates before the permutation tail, then the tail on
// its own passes (*prefix_passes: the passes of the first part).
std::vector<TilePlanPass> plan_fused(const tqd_circuit *c, int *prefix_passes);
bool encode_tile_pass(const tqd_circuit *c, TilePlanPass &P);

// Launch one pass (forward: lam == nullptr; reverse sweep with gradients
// into the circuit's partials when lam != nullptr).  Forward: psi is read
// from psi_src and written to psi_dst (each psi->amps when NULL; both hold
// psi's qubit count and dtype and do not overlap unless equal).  Reverse: psi
// is read from psi_src when given and then not written (a forward
// checkpoint), otherwise read and written in place.
cudaError_t launch_tile_pass(tqd_state *psi, tqd_state *lam, const tqd_circuit *c, int pass, cudaStream_t s,
                             const void *psi_src = nullptr, void *psi_dst = nullptr);
int tile_grid(const tqd_circuit *c, int dtype, bool adj);
// The TMA tensor map of pass pp over a state at `base` (dt 0: complex64).
cudaError_t tile_tensor_map(CUtensorMap *map, void *base, const TilePlanPass &pp, int dt);

// Host execution of circuit c's fused plan from its descriptors against the
// gates applied one by one (tqd_plan_check).
tqd_status plan_check_host(tqd_circuit *c, const double *params, uint64_t seed, double *err_fwd, double *err_rev,
                           int *n_passes, int *n_stages);

}  // namespace tqd
