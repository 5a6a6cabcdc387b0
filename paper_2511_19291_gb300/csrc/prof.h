// prof.h -- optional per-launch CUDA-event timing (internal).
#pragma once

#include <cuda_runtime.h>

namespace tqd {

enum ProfKind {
    PK_PREP = 0, PK_RESET, PK_DENSE1, PK_DIAG1, PK_PERM2, PK_PHASE11, PK_DENSE2, PK_SMALL,
    PK_ADJ1, PK_ADJ_PHASE11, PK_ADJ_SMALL, PK_EXPVAL, PK_EXPVAL_TERMS, PK_APPLY_OBS, PK_REDUCE,
    PK_TILE_FWD, PK_TILE_ADJ, PK_DIAG_RUN, PK_PAULI_TILE, PK_BATCH, PK_TC_BLOCK, PK_SHOTS, PK_NKINDS
};

bool prof_on();
// Records an event on s before the launch; returns a slot id (or -1 when off).
int prof_begin(int kind, cudaStream_t s);
// Records the end event and the launch's algorithmic bytes.
void prof_end(int slot, double bytes, cudaStream_t s);

struct ProfScope {
    int slot;
    double bytes;
    cudaStream_t s;
    ProfScope(int kind, double b, cudaStream_t st) : slot(prof_on() ? prof_begin(kind, st) : -1), bytes(b), s(st) {}
    ~ProfScope() {
        if (slot >= 0) prof_end(slot, bytes, s);
    }
};

}  // namespace tqd
