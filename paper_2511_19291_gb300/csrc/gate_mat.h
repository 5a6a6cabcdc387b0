// gate_mat.h -- the unitary of one gate from its angle (host and device).
#pragma once

#include <math.h>

#include "internal.h"

namespace tqd {

// Entry (r, c) of the d x d matrix (d = 2 or 4, wires[0] the most
// significant bit) at m[2 (r d + c)], m[2 (r d + c) + 1]; the rest of the
// MAT_STRIDE slots are zero.  R_P(t) = exp(-i t P / 2); PHASE(t) =
// diag(1, e^{it}); CPHASE(t) = diag(1, 1, 1, e^{it}).  table: the circuit's
// matrix entries (UNITARY1 / UNITARY2 read 4 / 16 complex entries at `mat`).
__host__ __device__ inline void gate_matrix(int kind, double th, const double *table, int mat, double *m) {
    for (int i = 0; i < MAT_STRIDE; ++i) m[i] = 0.0;
    const int d = gate_arity(kind) == 2 ? 4 : 2;
    auto set = [&](int r, int c, double re, double im) {
        m[2 * (r * d + c)] = re;
        m[2 * (r * d + c) + 1] = im;
    };
    double s, c, s1, c1;
#ifdef __CUDA_ARCH__
    sincos(0.5 * th, &s, &c);
    sincos(th, &s1, &c1);
#else
    s = sin(0.5 * th);
    c = cos(0.5 * th);
    s1 = sin(th);
    c1 = cos(th);
#endif
    const double r2 = 0.70710678118654752440;
    switch (kind) {
    case TQD_H: set(0, 0, r2, 0); set(0, 1, r2, 0); set(1, 0, r2, 0); set(1, 1, -r2, 0); break;
    case TQD_X: set(0, 1, 1, 0); set(1, 0, 1, 0); break;
    case TQD_Y: set(0, 1, 0, -1); set(1, 0, 0, 1); break;
    case TQD_Z: set(0, 0, 1, 0); set(1, 1, -1, 0); break;
    case TQD_S: set(0, 0, 1, 0); set(1, 1, 0, 1); break;
    case TQD_T: set(0, 0, 1, 0); set(1, 1, r2, r2); break;
    case TQD_RX: set(0, 0, c, 0); set(0, 1, 0, -s); set(1, 0, 0, -s); set(1, 1, c, 0); break;
    case TQD_RY: set(0, 0, c, 0); set(0, 1, -s, 0); set(1, 0, s, 0); set(1, 1, c, 0); break;
    case TQD_RZ: set(0, 0, c, -s); set(1, 1, c, s); break;
    case TQD_PHASE: set(0, 0, 1, 0); set(1, 1, c1, s1); break;
    case TQD_UNITARY1:
        for (int i = 0; i < 8; ++i) m[i] = table[2 * mat + i];
        break;
    case TQD_CNOT: set(0, 0, 1, 0); set(1, 1, 1, 0); set(2, 3, 1, 0); set(3, 2, 1, 0); break;
    case TQD_CZ: set(0, 0, 1, 0); set(1, 1, 1, 0); set(2, 2, 1, 0); set(3, 3, -1, 0); break;
    case TQD_CPHASE: set(0, 0, 1, 0); set(1, 1, 1, 0); set(2, 2, 1, 0); set(3, 3, c1, s1); break;
    case TQD_SWAP: set(0, 0, 1, 0); set(1, 2, 1, 0); set(2, 1, 1, 0); set(3, 3, 1, 0); break;
    case TQD_UNITARY2:
        for (int i = 0; i < 32; ++i) m[i] = table[2 * mat + i];
        break;
    default: break;
    }
}

}  // namespace tqd
