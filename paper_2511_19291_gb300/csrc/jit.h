// jit.h -- pass-specialised tile kernels (internal).
//
// The generic tile kernel reads every op's type, positions and matrix offset,
// and every register address, from the pass descriptor while it runs.  A
// specialised kernel has them fixed: its stage runner is generated as
// straight-line code (one helper call per op with compile-time positions,
// constant pool offsets and register addresses) and compiled at run time
// with NVRTC for the device's architecture.  It uses the same device code
// (tile_dev.cuh), shared-memory layout, descriptor and launch grid as the
// generic kernel, so the two are interchangeable pass by pass.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "internal.h"

namespace tqd {

// Whether circuit c runs its fused passes through specialised kernels.
bool jit_wanted(const tqd_circuit *c);

// Source text of pass `pass`'s specialised kernel (dt: 0 complex64, 1 complex128).
// `ring`: the kernel runs on a ring of tile buffers (tile_pass_ring) instead of
// one buffer per block (tile_pass_body); `tmaw`: the ring has a TMA warpgroup;
// `psi_ro` (reverse sweep): psi comes from a forward checkpoint and is not
// written back, so the last stage stores lambda only.
std::string jit_source(const tqd_circuit *c, int pass, int dt, bool adj, bool ring, bool tmaw, bool psi_ro);

// Index of a kernel kind in tqd_circuit::jit_fn.
inline int jit_kind(bool ring, bool tmaw, bool psi_ro) { return (ring ? (tmaw ? 2 : 1) : 0) + (psi_ro ? 3 : 0); }

// The specialised kernel of pass `pass`, compiling every pass of (dt, adj,
// kind) on first use.  *out = nullptr means "run the generic kernel": the circuit
// does not want specialised kernels, NVRTC is unavailable in the default
// mode, the pass is replaced by a tensor-core block, or s is capturing a
// graph before the kernels exist.  Errors: NVRTC missing when the circuit
// requires it (cudaErrorNotSupported) or a failed compile / module load.
cudaError_t jit_function(const tqd_circuit *c, int pass, int dt, bool adj, bool ring, bool tmaw, bool psi_ro,
                         cudaStream_t s, CUfunction *out);

// Registers per thread kernel f launches with (-1 when unknown).
int jit_num_regs(CUfunction f);

// Launches a specialised kernel with the generic kernel's arguments.
cudaError_t jit_launch(CUfunction f, const CUtensorMap &ma, const CUtensorMap &mb, const TilePassDev *desc,
                       const void *mats, double *partials, int pblk, int *err, int flags, int grid, int threads,
                       uint32_t smem, cudaStream_t s);

// Host only (no GPU): plans circuit c's fused passes, generates every
// specialised kernel (both precisions, both directions) and compiles the
// distinct ones for compute capability `arch`.  *n_kernels = their number.
tqd_status jit_check_host(tqd_circuit *c, int arch, int *n_kernels);

// Frees nothing (modules are shared by every circuit with the same pass
// shapes and live until the process exits); clears the circuit's table.
void jit_release(tqd_circuit *c);

}  // namespace tqd
