// pauli_tile.h -- Pauli sums over 12-qubit tiles (internal).
#pragma once

#include <stdint.h>

#include <vector>

#include "internal.h"

namespace tqd {

constexpr int PT_MAXG = 32;  // x-mask groups per launch
constexpr int PT_MAXT = 64;  // terms per launch

// One launch: a set Q (qubits 0..3 and the 8 qubits hi[]) and the groups
// whose x masks lie inside Q, with masks in local bits (bit i < 4: qubit i;
// bit 4 + k: qubit hi[k]).
struct PauliTileDesc {
    int n;                           // qubits of the state (>= 12)
    int n_groups;
    int n_terms;
    int accumulate;                  // H psi: add into the output
    uint8_t hi[8];                   // Q's qubits above qubit 3, ascending
    uint8_t out_q[32];               // qubits outside Q, ascending (tile index bit i -> qubit)
    uint16_t gx[PT_MAXG];            // local x mask of each group
    uint16_t gfirst[PT_MAXG + 1];    // terms of group g: [gfirst[g], gfirst[g + 1])
    uint16_t zl[PT_MAXT];            // local z mask of each term
    uint16_t pad[3];
    uint64_t zo[PT_MAXT];            // z bits outside Q (signs fixed per tile)
    double cre[PT_MAXT], cim[PT_MAXT];  // coeff * i^{|x & z|}
    int32_t idx[PT_MAXT];            // the term's position in the caller's list (weights)
};

// Launches covering every group that flips at most 8 qubits above qubit 3;
// *leftover gets the indices of the other groups (and all groups when n < 12).
std::vector<PauliTileDesc> plan_pauli_tiles(const std::vector<PauliGroup> &groups, int n, std::vector<int> *leftover);

// Blocks of one tile launch; launch i writes partials[i * pblk + block].
int pauli_tile_grid(int n, int dtype);
// Partials of one expectation launch: launch i fills partials[i * pblk + j]
// for j < this width (blocks it did not have are written as zero).
int pauli_tile_expval_width(int n, int dtype);
cudaError_t launch_pauli_tile_expval(const tqd_state *st, const std::vector<PauliTileDesc> &launches,
                                     double *partials, int pblk, cudaStream_t s);
// out = (accumulate ? out : 0) + scale * sum w_j c_j P_j psi over the launches' groups.
// eparts (complex64 only, else ignored; may be null): the last launch also
// writes each block's share of Re <psi|out> to eparts[block].
cudaError_t launch_pauli_tile_apply(const tqd_state *psi, const std::vector<PauliTileDesc> &launches,
                                    const double *weights, double scale, tqd_state *out, bool accumulate,
                                    double *eparts, cudaStream_t s);

}  // namespace tqd
