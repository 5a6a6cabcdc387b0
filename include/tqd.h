/*
 * tqd.h -- C ABI of libtqd, a single-GPU differentiable state-vector
 * simulator for GB300 (sm_103a).
 *
 * The library applies the gates of a parameterised circuit to a 2^n complex
 * amplitude vector, evaluates Pauli-sum expectation values, and takes the
 * adjoint (reverse-sweep) gradient of an expectation with respect to the gate
 * angles, recomputing intermediate states instead of storing them.
 *
 * Paper: "TorchQuantumDistributed" (arXiv 2511.19291).
 *   - state vector and gate (M, Q): Sec. 4.1, "Tensor dimension order";
 *   - gate application Y = M x_Q X: Sec. 2.2 (contraction notation) and
 *     Algorithm 1;
 *   - measurement in the Z basis and expectation values: Sec. 2.2.1;
 *   - backpropagation through unitaries by recomputation x = U^* y: Sec. 4.4.
 *
 * Conventions for every entry point:
 *   - Qubit i is bit i of the flat amplitude index.  Amplitudes are
 *     interleaved (re, im): float2 for TQD_C64, double2 for TQD_C128.
 *   - For a k-qubit gate, wires[0] is the most significant bit of the gate's
 *     local index; CNOT takes wires = {control, target}.
 *   - R_P(t) = exp(-i t P / 2) for RX, RY, RZ; PHASE(t) = diag(1, e^{it});
 *     CPHASE(t) = diag(1, 1, 1, e^{it}).
 *   - Every call that takes a stream is asynchronous on that stream
 *     (a cudaStream_t passed as void*; NULL is the legacy default stream).
 *   - Arguments are validated on the host before any launch.  On error the
 *     call returns a non-zero tqd_status, launches nothing and leaves a
 *     message for tqd_last_error() (thread-local).  No C++ exception crosses
 *     the ABI.
 *   - Device pointers passed in are owned by the caller and must stay valid
 *     until the work enqueued on the stream has finished.  Handles
 *     (tqd_state, tqd_circuit) are owned by the caller and freed with the
 *     matching *_free call; they may not be used by two streams at once.
 */
#ifndef LIBTQD_TQD_H_
#define LIBTQD_TQD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TQD_OK = 0,
    TQD_ERR_INVALID_ARG = 1, /* bad pointer, size, wire, index or alignment */
    TQD_ERR_UNSUPPORTED = 2, /* valid request this build does not implement */
    TQD_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    TQD_ERR_OOM = 4,         /* device or host allocation failed */
    TQD_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    TQD_ERR_NUMERIC = 6      /* non-finite or out-of-range numeric input */
} tqd_status;

typedef enum { TQD_C64 = 0, TQD_C128 = 1 } tqd_dtype;

typedef enum {
    TQD_H = 0, TQD_X = 1, TQD_Y = 2, TQD_Z = 3, TQD_S = 4, TQD_T = 5,
    TQD_RX = 6, TQD_RY = 7, TQD_RZ = 8, TQD_PHASE = 9,
    TQD_CNOT = 10, TQD_CZ = 11, TQD_CPHASE = 12, TQD_SWAP = 13,
    TQD_UNITARY1 = 14, /* arbitrary 2x2 unitary from the circuit's matrix table */
    TQD_UNITARY2 = 15  /* arbitrary 4x4 unitary from the circuit's matrix table */
} tqd_gate_kind;

/* One gate (M, Q) of Sec. 4.1.  The angle of a parametric gate is
 * dev_params[param_idx] when param_idx >= 0, otherwise `fixed`.  mat_idx is
 * the offset, in complex entries, of a UNITARY1/UNITARY2 matrix (row-major)
 * in the table given to tqd_circuit_create; -1 otherwise. */
typedef struct {
    uint32_t kind;
    uint32_t nwires;
    uint32_t wires[3];
    int32_t param_idx;
    double fixed;
    int32_t mat_idx;
    uint32_t reserved;
} tqd_gate;

/* coeff * i^{|x & z|} X^x Z^z: X on the bits of xmask, Z on the bits of
 * zmask, a bit in both masks is Y. */
typedef struct {
    uint64_t xmask;
    uint64_t zmask;
    double coeff;
} tqd_pauli_term;

typedef enum {
    TQD_PLAN_PLAIN = 0, /* one full-state sweep per gate (gate-by-gate path) */
    TQD_PLAN_FUSED = 1, /* fused passes: low-qubit and mixed tiles, diagonal runs */
    TQD_PLAN_TC = 2     /* as FUSED, and runs of >= 16 gates on qubits 0..5 become one fused
                           64 x 64 unitary applied on the tensor cores (complex64, split-
                           precision TF32 products): in the forward pass, and in the reverse
                           sweep when the block's gates are fixed (no angle: un-applying it is
                           one product with U^dagger per state; a block with angles is
                           un-applied by a tile pass, which also takes its derivatives) */
} tqd_plan_mode;

typedef struct {
    uint32_t mode;        /* tqd_plan_mode */
    uint32_t tile_qubits; /* fused tiles hold 2^tile_qubits amplitudes: 0 or 12, the width the
                             tile kernels are laid out for (16 amplitudes in registers x 256
                             threads); other values are TQD_ERR_INVALID_ARG */
    uint32_t low_qubits;  /* contiguous low qubits in every tile (128-byte runs of complex64):
                             0 or 4; other values are TQD_ERR_INVALID_ARG */
    uint32_t buffers;     /* tile buffers in the fused passes: 1 = each block loads, computes and
                             stores one tile at a time; 2 = each block loads its next tile while
                             the current one is computed (twice the shared memory); 3 = ring:
                             one block per SM whose groups of 256 threads share a ring of tile
                             buffers, each refilled by TMA as soon as its tile is stored
                             (complex64 only; complex128 uses 1); 4 = the ring with one more
                             warpgroup that issues every store and refill, so the groups never
                             wait for a store, and hands most of its registers to the groups;
                             0 = default: 4 for complex64 states of 21 qubits and more, else 1 */
    uint32_t jit;         /* fused passes run 1 = the generic pass kernel, which reads positions,
                             addresses and matrices from the pass descriptor; 2 = kernels
                             specialised per pass (straight-line code with those fixed, compiled
                             at run time with NVRTC on first use; TQD_ERR_UNSUPPORTED when NVRTC
                             cannot be loaded); 0 = default: specialised from 22 qubits up, when
                             NVRTC can be loaded */
    uint32_t max_blocks;  /* cap on the blocks of a fused pass launch (0 = no cap: one per SM for
                             the ring, the occupancy limit otherwise); a smaller grid gives each
                             block more tiles */
    uint32_t checkpoints; /* forward checkpoints of tqd_value_and_grad (fused plan): the states
                             after the last K passes are kept in device memory the circuit owns,
                             so the reverse sweep reads psi there instead of writing it back
                             (3 instead of 4 state transfers per reverse pass).  0 = default: as
                             many passes as fit in half the device memory free at the first
                             call; TQD_CHECKPOINTS_NONE = none (psi recomputed in place all the
                             way); other values = at most that many passes */
    uint32_t reserved[1]; /* must be zero */
} tqd_plan_opts;

#define TQD_CHECKPOINTS_NONE 0xFFFFFFFFu

typedef struct tqd_state tqd_state;
typedef struct tqd_circuit tqd_circuit;

/* ---------------------------------------------------------------- states */

/* Wrap caller-owned device memory (e.g. a torch tensor) as an n-qubit state.
 * dev_amps: device pointer, 256-byte aligned, at least 2^n * 8 (C64) or
 * 2^n * 16 (C128) bytes.  1 <= n_qubits <= 34.  The handle never frees
 * dev_amps.  Allocates only the small host handle. */
tqd_status tqd_state_alloc(int n_qubits, tqd_dtype dtype, void *dev_amps, size_t bytes,
                           tqd_state **out);

/* psi = e_{basis_index} (the |0...0> reset of the appendix listings when
 * basis_index = 0).  basis_index < 2^n. */
tqd_status tqd_state_reset(tqd_state *state, uint64_t basis_index, void *stream);

/* Frees the handle, never the amplitudes. The handle's reduction workspace
 * (allocated stream-ordered on first use) is released in the order of the
 * stream that used it last, so work still queued there may keep running; that
 * stream must still exist. NULL is accepted. */
tqd_status tqd_state_free(tqd_state *state);

/* -------------------------------------------------------------- circuits */

/* Validate a gate list and build its launch plan (host work only, plus one
 * device buffer for the per-gate matrices that tqd_apply_circuit fills from
 * the angles on the device, so a captured CUDA graph stays valid as the
 * angles change).  gates: host array of n_gates gates.  matrices: host array
 * of n_matrix_entries complex entries as interleaved (re, im) doubles, read
 * by UNITARY1/UNITARY2 gates; may be NULL when none is used.  opts may be
 * NULL (fused plan, default tiles).  The library keeps its own copies. */
tqd_status tqd_circuit_create(int n_qubits, const tqd_gate *gates, size_t n_gates, int n_params,
                              const double *matrices, size_t n_matrix_entries,
                              const tqd_plan_opts *opts, tqd_circuit **out);

/* Waits for the circuit's device to finish its queued work (which may read the
 * circuit's buffers), then frees the circuit and its device buffers (forward
 * checkpoints included). NULL is accepted. */
tqd_status tqd_circuit_free(tqd_circuit *circuit);

/* Diagnostics that need no GPU: validates the gate list as tqd_circuit_create
 * does, plans its fused passes on the host (n_qubits >= 12), generates every
 * pass-specialised kernel (both precisions, both directions; see
 * tqd_plan_opts.jit) and compiles the distinct ones with NVRTC for compute
 * capability `arch` (103 for sm_103a).  *n_kernels receives their number.
 * TQD_ERR_UNSUPPORTED when NVRTC cannot be loaded; TQD_ERR_CUDA when a kernel
 * fails to compile (tqd_last_error holds the start of the compiler log).  With
 * the environment variable TQD_JIT_DUMP_DIR set to a directory, every distinct
 * generated source is also written there (pass_<i>.cu).  The paper has no
 * counterpart: this checks code the library writes at run time. */
tqd_status tqd_jit_check(int n_qubits, const tqd_gate *gates, size_t n_gates, int n_params,
                         const double *matrices, size_t n_matrix_entries, int arch, int *n_kernels);

/* Diagnostics that need no GPU: plans the circuit into fused passes as
 * tqd_circuit_create does (12 <= n_qubits <= 20), then runs the encoded plan
 * on the host on a random state drawn from `seed`: every tile gathered by its
 * pass's qubit set, every stage's amplitudes loaded and stored through the
 * address tables the kernels read, every op applied at the register and
 * thread positions it encodes (params: host array of n_params angles).  It
 * compares the result with the gates applied one by one
 * (*err_forward: largest amplitude difference), runs the reverse sweep's
 * stages and inverse ops back to the start state (*err_reverse), and does
 * this for the complex64 and complex128 descriptors.  *n_passes and
 * *n_stages (may be NULL) receive the plan's size.  TQD_ERR_NUMERIC when a
 * stage moves amplitudes between threads without the barrier between its
 * loads and stores.  The paper has no counterpart: this checks the library's
 * own planner. */
tqd_status tqd_plan_check(int n_qubits, const tqd_gate *gates, size_t n_gates, int n_params,
                          const double *matrices, size_t n_matrix_entries, const double *params,
                          uint64_t seed, double *err_forward, double *err_reverse, int *n_passes,
                          int *n_stages);

/* Number of device launches one tqd_apply_circuit enqueues (for accounting). */
tqd_status tqd_circuit_info(const tqd_circuit *circuit, int *n_passes, int *n_launches_apply,
                            int *n_launches_backward);

/* Synchronizes the device, reads the circuit's device error word and clears
 * it: *device_error = 0 when every launch of this circuit since the last
 * check completed normally, 1 when a bounded wait for a tile copy gave up
 * (every device wait gives up after about one second of elapsed time; that
 * launch's results are invalid, the context stays usable), 2 when a kernel
 * built with TQD_CHECKED found an index out of range.  Returns
 * TQD_ERR_TIMEOUT for 1, TQD_ERR_NUMERIC for 2. */
tqd_status tqd_circuit_check(const tqd_circuit *circuit, int *device_error);

/* Test hook of the give-up path (the paper has no counterpart): while
 * enabled, every fused tile pass of this circuit arms the barrier of block
 * 0's first tile without issuing its copy, so that block's wait runs out its
 * time limit (about one second per launch, and as long again for the waits
 * that depend on that tile), the block returns, and tqd_circuit_check then
 * reports TQD_ERR_TIMEOUT.  The launch's results are invalid.  Other
 * launches (gate-by-gate kernels, tensor-core blocks, observables) are not
 * affected. */
tqd_status tqd_circuit_test_stall(tqd_circuit *circuit, int enable);

/* psi <- G_L ... G_1 psi (Sec. 4.1; gate semantics of Algorithm 1).
 * dev_params: device array of n_params doubles (may be NULL when n_params
 * is 0).  The state must have the circuit's qubit count. */
tqd_status tqd_apply_circuit(tqd_state *state, const tqd_circuit *circuit, const double *dev_params,
                             void *stream);

/* ----------------------------------------------------------- observables */

/* E = sum_j coeff_j <psi|P_j|psi> (Sec. 2.2.1), reduced in FP64, written to
 * dev_out[0] (device).  terms: host array, copied into the launch.  Masks
 * must lie below 2^n. */
tqd_status tqd_expval(const tqd_state *state, const tqd_pauli_term *terms, size_t n_terms,
                      double *dev_out, void *stream);

/* Per-term values <psi|P_j|psi> (without coeff_j) to dev_out[0..n_terms);
 * with Z_i terms this is measure_allZ of the appendix listings. */
tqd_status tqd_expval_terms(const tqd_state *state, const tqd_pauli_term *terms, size_t n_terms,
                            double *dev_out, void *stream);

/* out = sum_j w_j coeff_j P_j psi.  dev_weights: device array of n_terms
 * doubles, or NULL for all ones.  out must differ from psi and have the same
 * qubit count and dtype. */
tqd_status tqd_apply_observable(const tqd_state *psi, const tqd_pauli_term *terms, size_t n_terms,
                                const double *dev_weights, tqd_state *out, void *stream);

/* --------------------------------------------------------------- adjoint */

/* Adjoint gradient (Sec. 4.4): with psi holding psi_L = U psi_0 (the state
 * tqd_apply_circuit left), sets lambda = H psi_L for
 * H = grad_scale * sum_j w_j coeff_j P_j, then sweeps the circuit in reverse,
 * un-applying every gate from psi and lambda and adding
 * 2 Re <lambda| dG/dtheta |psi_before> for every parametric gate to
 * dev_grads[param_idx] (device, n_params doubles, accumulated, not zeroed).
 * On return psi holds psi_0 again (the recomputation that replaces stored
 * activations) and lambda holds U^dagger H psi_L.  lambda: a state of the
 * same qubit count and dtype used as scratch.  dev_term_weights may be NULL
 * (all ones). */
tqd_status tqd_backward(tqd_state *psi, tqd_state *lambda, const tqd_circuit *circuit,
                        const double *dev_params, const tqd_pauli_term *terms, size_t n_terms,
                        const double *dev_term_weights, double grad_scale, double *dev_grads,
                        void *stream);

/* Same result as tqd_expval, for callers that may not allocate device memory
 * while they run: a service that reserved its whole memory budget at
 * start-up, a latency-sensitive loop where cudaMalloc/cudaFree would stall the
 * device, or a framework that owns the device allocator.  (The paper has no
 * counterpart; this is a library convenience.)
 *
 * The reduction's per-block partial sums go to a fixed scratch array inside
 * the library, TQD_NOALLOC_SCRATCH_DOUBLES doubles (1 MiB) per GPU, reserved
 * from library load until process exit.  This call makes no cudaMalloc,
 * cudaFree or other allocating call.  Requests whose partials do not fit are
 * rejected with TQD_ERR_INVALID_ARG: they need (number of 64-term chunks of
 * distinct x masks) x (blocks + 1) doubles, blocks <= 8 x the SM count; on a
 * 152-SM GB300 about 100 chunks fit.  Every slot a call reads is written
 * earlier in the same call, so nothing has to be cleared between calls.
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The address is kept per device context: after
 * cudaDeviceReset (or whatever else ends the device's context) the next call
 * looks it up again, so that call too must come before any capture.  All
 * calls on a device share the one array: calls whose GPU work overlaps
 * (different streams or host threads) race. */
#define TQD_NOALLOC_SCRATCH_DOUBLES 131072
tqd_status tqd_expval_noalloc(const tqd_state *state, const tqd_pauli_term *terms, size_t n_terms,
                              double *dev_out, void *stream);

/* One gradient evaluation in one call: psi <- U psi (as tqd_apply_circuit),
 * E = <psi_L|H|psi_L> for H = sum_j coeff_j P_j written to dev_energy[0]
 * (device, FP64), and the adjoint gradient of E added to dev_grads (as
 * tqd_backward with unit weights and grad_scale 1); on return psi holds its
 * input state again and lambda holds the reverse sweep's adjoint state
 * V^dagger H psi_L, where V is U less the fused passes before its first
 * pass with an angle (V = U for the gate-by-gate plan, and whenever the
 * first pass has an angle).  E is read off lambda = H psi_L as Re <psi_L|lambda>, the seed the
 * reverse sweep needs anyway (Sec. 2.2.1, Sec. 4.4), so no separate
 * expectation pass runs; it equals tqd_expval's value up to rounding.
 *
 * Fused plans keep forward checkpoints (tqd_plan_opts.checkpoints): the
 * states after the last K passes go to device memory the circuit owns, the
 * reverse sweep reads psi there, and psi itself is only read when K covers
 * every pass.  The reverse sweep ends at the first pass with an angle (the
 * passes before it have no derivative to take, e.g. a QFT that prepares the
 * ansatz's input); when some pass runs in place, one checkpoint slot then
 * keeps a copy of the input state, copied back at the end, instead of a
 * pass's output.  The first call for a state size allocates that memory
 * (cudaMemGetInfo, cudaMalloc): make it outside any stream capture.  Calls on
 * one circuit whose GPU work overlaps race on it (as on its gradient
 * partials). */
tqd_status tqd_value_and_grad(tqd_state *psi, tqd_state *lambda, const tqd_circuit *circuit,
                              const double *dev_params, const tqd_pauli_term *terms, size_t n_terms,
                              double *dev_energy, double *dev_grads, void *stream);

/* The reverse sweep of tqd_backward from a seed the caller placed in lambda:
 * lambda must hold dL/d conj(psi_L) for a real loss L of the final state
 * (so that dL/dtheta = 2 Re <lambda| d psi_L/dtheta>); psi holds psi_L.
 * Adds dL/dtheta to dev_grads; on return psi holds psi_0 again.  With
 * lambda = H psi_L this is tqd_backward; tqd_shots_gaussian_backward writes
 * the seed of a loss of the Gaussian shots (Sec. 4.4 with a general seed). */
tqd_status tqd_backward_seeded(tqd_state *psi, tqd_state *lambda, const tqd_circuit *circuit,
                               const double *dev_params, double *dev_grads, void *stream);

/* ------------------------------------------------------------ shot noise */

/* p_b = |psi_b|^2 for every outcome b, FP64, to dev_p (2^n doubles)
 * (measurement in the Z basis, Sec. 2.2.1). */
tqd_status tqd_probabilities(const tqd_state *state, double *dev_p, void *stream);

/* Exact sampling of measurement outcomes (Sec. 4.3.2, "Exact"): shot s is
 * the outcome b with CDF(b-1) <= u_s < CDF(b) for the normalised cumulative
 * distribution of p = |psi|^2 (inverse transform), u_s = dev_uniforms[s] in
 * [0, 1) drawn by the caller; the outcome indices go to dev_samples
 * (n_shots int64, device).  Two-level cumulative sums (chunk totals, then
 * outcomes within the chunk), the single-device form of the paper's
 * hierarchical scheme.  Uses the state's workspace. */
tqd_status tqd_sample(tqd_state *state, const double *dev_uniforms, size_t n_shots, int64_t *dev_samples,
                      void *stream);

/* Approximate, differentiable shots (Sec. 4.3.2, "Approximate"):
 * y = n p + sqrt(n) D S z with p = |psi|^2, D = diag(sqrt(p)),
 * S = I - 2 v v^T, v = (e_{N-1} - sqrt(p)) / |e_{N-1} - sqrt(p)| (v = 0 in
 * the degenerate case) and z = (z_0, ..., z_{N-2}, 0): dev_z holds N - 1 or N
 * unit normals drawn by the caller (entry N - 1 is not read); y (N doubles)
 * sums to n sum(p).  The printed S = I - v v^T lacks the factor 2 of the
 * Householder reflection that gives the multinomial covariance. */
tqd_status tqd_shots_gaussian(tqd_state *state, double n_shots, const double *dev_z, double *dev_y, void *stream);

/* The seed of the reverse sweep for L = sum_i ybar_i y_i:
 * lambda_b = dL/d conj(psi_b) = (dL/du_b) psi_b / (2 |psi_b|) with
 * u = |psi| (0 where psi_b = 0), written to lambda (same qubits and dtype
 * as state).  Follow with tqd_backward_seeded for dL/dtheta. */
tqd_status tqd_shots_gaussian_backward(tqd_state *state, double n_shots, const double *dev_z,
                                       const double *dev_ybar, tqd_state *lambda, void *stream);

/* ---------------------------------------------------------------- batches */

/* Many independent circuits of uneven width and depth (the batch dimension of
 * Sec. 4, every circuit with its own state) evaluated together: forward,
 * E_c = <H_c>, and the adjoint gradient of every E_c, all from one CUDA-graph
 * launch.  Circuits of complex64 width up to `small_max_qubits` run whole in
 * one block's shared memory (psi and lambda resident) from a persistent
 * work-queue kernel.  Wider circuits run from a second persistent kernel:
 * each circuit's stages (reset, its fused tile passes, lambda = H psi with
 * E, its reverse passes, the closing sums) are split into work items of a
 * few tiles; a device work queue hands items to the blocks, and the block
 * that completes a stage queues the next one.  Wider circuits whose plan is
 * not all complex64 tile passes (or a tensor-core block) run their passes on
 * `streams` concurrent streams inside the same graph instead. */
typedef struct tqd_batch tqd_batch;

typedef struct {
    uint32_t small_max_qubits; /* 0 = default (13) or the autotuned value */
    uint32_t small_threads;    /* block size of the small-circuit kernel; 0 = default / autotuned */
    uint32_t streams;          /* concurrent streams for the wider circuits; 0 = default (16) */
    uint32_t autotune;         /* non-zero: time the candidates once at creation and keep the best
                                  (the small kernel's block size, its width cutoff, then the tiles
                                  per work item of the wider circuits, width by width) */
    uint32_t plain;            /* non-zero: every circuit gate by gate, one launch per gate (baseline) */
    uint32_t reserved[3];      /* must be zero */
} tqd_batch_opts;

/* circuits: n_circuits planned circuits (complex64 widths 1..26); terms[c],
 * n_terms[c]: circuit c's observable (host arrays, copied).  The batch owns
 * its states and its device buffers for angles, energies and gradients (see
 * tqd_batch_buffers); the circuits must outlive the batch. */
tqd_status tqd_batch_create(int n_circuits, const tqd_circuit *const *circuits,
                            const tqd_pauli_term *const *terms, const size_t *n_terms,
                            const tqd_batch_opts *opts, tqd_batch **out);

/* Device buffers owned by the batch: params (sum of the circuits' n_params
 * doubles, circuit c's angles at param_offset[c]), energies (n_circuits
 * doubles), grads (same layout as params, overwritten by every run).  Any
 * pointer may be NULL.  param_offset (host, n_circuits entries) may be NULL. */
tqd_status tqd_batch_buffers(tqd_batch *batch, double **dev_params, double **dev_energies, double **dev_grads,
                             size_t *param_offset);

/* One forward + expectation + adjoint gradient of every circuit, as one
 * CUDA-graph launch on `stream`; the first call on a batch captures the graph
 * (and warms the workspaces up), later calls replay it. */
tqd_status tqd_batch_run(tqd_batch *batch, void *stream);

tqd_status tqd_batch_info(const tqd_batch *batch, int *n_small, int *n_large, int *small_max_qubits,
                          int *small_threads, int *graph_nodes);

/* Work items of the wider circuits of width `width` (0..26) on the
 * persistent kernel: *tiles_per_item tiles of 2^12 amplitudes per item and
 * *items_per_stage items per stage; both 0 when no circuit of that width runs
 * there.  The paper has no counterpart: this reports the batch's schedule. */
tqd_status tqd_batch_tiling(const tqd_batch *batch, int width, int *tiles_per_item, int *items_per_stage);

tqd_status tqd_batch_free(tqd_batch *batch);

/* -------------------------------------------------------------- profiling */

/* Per-kernel-class timing, summed over launches: CUDA events recorded on the
 * launching stream around every kernel (the paper's Sec. 5 records walltime
 * per step; this splits it by kernel).  bytes is the algorithmic traffic of
 * those launches (amplitudes each launch must read and write). */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
    double bytes;
} tqd_profile_entry;

/* Turn recording on (non-zero) or off, discarding earlier records.  Recording
 * adds two event records per launch; it is off by default. */
tqd_status tqd_profile_enable(int enable);

/* Wait for the recorded events, write up to `capacity` entries (one per
 * kernel class that launched) and their total count to *n_out, then discard
 * the records. */
tqd_status tqd_profile_read(tqd_profile_entry *out, int capacity, int *n_out);

/* ------------------------------------------------------------------ misc */

/* Message of the last failed call on this thread ("" if none). */
const char *tqd_last_error(void);
const char *tqd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBTQD_TQD_H_ */
