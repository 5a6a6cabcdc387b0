// tile_desc.h -- descriptors of a fused tile pass as the kernels read them
// (plain structs; compiled by nvcc and by the runtime compiler alike).
//
// A pass holds K = 12 qubits Q (always the low qubits 0..3 plus up to 8
// others).  Every tile of the state -- the 2^K amplitudes that share the
// values of the qubits outside Q -- is brought into shared memory by TMA,
// every gate of the pass is applied there, and the tile is written back: one
// HBM read and write of the state per pass instead of one per gate.
//
// Inside the tile, local bit i stands for qubit q[i].  The 256 threads of a
// block each hold 2^R = 16 amplitudes in registers.  A pass is split into
// stages; in a stage, R chosen local bits are "register bits" (the bits of
// the register index j) and the other 8 are "thread bits" (bits of the
// thread index).  Dense gates need their qubits on register bits; diagonal
// gates and CNOT controls work on any bit.  Between stages the tile goes
// through shared memory, so each stage may pick new register bits.
#pragma once

#ifdef __CUDACC_RTC__
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef short int16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
#else
#include <stdint.h>
#endif

namespace tqd {

// Generator class of a parametric gate: dG/dt = i * gen_factor * P * G.
enum Gen { GEN_NONE = 0, GEN_X = 1, GEN_Y = 2, GEN_Z = 3, GEN_P1 = 4, GEN_P11 = 5 };

constexpr int MAT_STRIDE = 32;  // scalars per gate slot: 4x4 complex, interleaved

constexpr int TILE_K = 12;        // qubits per tile
constexpr int TILE_R = 4;         // register bits (amplitudes per thread = 16)
constexpr int TILE_T = 8;         // thread bits (256 threads)
constexpr int TILE_THREADS = 1 << TILE_T;
constexpr int TILE_LOW = 4;       // qubits 0..3 are in every tile (128-byte runs for c64)
constexpr int TILE_MAX_STAGES = 40;
constexpr int TILE_MAX_OPS = 240;
constexpr int TILE_MAX_GATES = 480;  // gates absorbed by one pass (ops and diagonal sub-ops)
constexpr int TILE_MAX_DIMS = 5;  // TMA tensor rank limit

// Launch flags of a tile pass.  TILE_PSI_RO (reverse sweep): psi is read from
// a forward checkpoint and only lambda is written back.  TILE_STALL_TEST:
// block 0 arms the barrier of its first tile without issuing the copy, so the
// wait for that tile runs out its time limit (the test of the give-up path).
constexpr int TILE_PSI_RO = 1;
constexpr int TILE_STALL_TEST = 2;

// Op types.  Positions are resolved per stage: `pos` < 0x40 is a register
// position (bit of the register index), `pos` >= 0x80 is thread-index bit
// (pos & 0x7f), and 0x40 <= `pos` < 0x80 is a qubit outside the pass's set,
// qubit (pos & 0x3f): a tile bit, the same for every amplitude of a tile (a
// bit of the tile's global origin).  Only diagonal gates of a run (TOP_DG)
// have tile bits; a two-qubit one has its tile bit in `a`.
enum TileOpType : uint8_t {
    TOP_G1 = 0,  // dense 2x2 on register position a
    TOP_D1 = 1,  // diagonal diag(m00, m11) on position a (register or thread)
    TOP_CX = 2,  // NOT on register position b when position a (register or thread) is 1
    TOP_SW = 3,  // swap register positions a, b
    TOP_G2 = 4,  // dense 4x4, wires[0] on register position a (MSB), wires[1] on b
    TOP_D2 = 5,  // phase m33 when positions a and b are both 1 (CZ, CPHASE)
    TOP_G1R = 6, // real 2x2 (RY, H) on register position a
    TOP_DG = 7,  // run of diagonal gates: subs[sub0 .. sub0 + nsub), one phase per amplitude
};

struct TileOp {
    uint8_t type;
    uint8_t a, b;
    uint8_t gen;     // generator class for the angle derivative (Gen), 0 = none
    int16_t moff;    // matrix offset in the pool (scalars), or the DG table index; -1 = none
    int16_t gslot;   // index among this pass's gradient ops, -1 = none
    int16_t sub0;    // TOP_DG: first sub-op
    int16_t nsub;    // TOP_DG: number of sub-ops
};

// One diagonal gate inside a TOP_DG run (type TOP_D1 or TOP_D2).
struct TileSub {
    uint8_t type;
    uint8_t a, b;
    uint8_t gen;
    int16_t moff;    // d0, d1 (D1: scalars 0..7 of the 2x2) or ph (D2) in the pool
    int16_t gslot;
};

constexpr int TILE_MAX_SUBS = 448;
constexpr uint8_t TILE_POS_TILE = 0x40;  // tile-bit position flag (see the op types)
constexpr int TILE_MAX_DG = 64;

// Shared-memory addresses of a stage.  Register j of thread (lane, warp)
// holds local index y = tlo[lane] ^ thi[warp] ^ roff[j].  Permutation gates
// (CNOT, SWAP, X) at the start of a stage are folded into the load address
// F(y) and those at its end into the store address G(y); F and G are affine
// maps over GF(2), so each address is an XOR of three table entries (already
// swizzled).  The reverse sweep loads with G and stores with F.
struct TileStage {
    uint8_t reg[TILE_R];      // local bit of register-index bit r
    uint8_t thr[TILE_T];      // local bit of thread-index bit u
    uint16_t op_begin, op_end;
    // Barriers (SYNC_*): sync_mid between the stage's loads and its stores;
    // sync_end between its stores and the next stage's loads (in either
    // direction of the sweep; unused after the last stage).  SYNC_NONE: every
    // thread only meets amplitudes it holds itself; SYNC_WARP: every warp
    // only meets its own (__syncwarp); SYNC_GROUP: the group of 256 meets.
    uint16_t sync_mid;
    uint16_t sync_end;
    uint16_t ld_roff[1 << TILE_R];
    uint16_t st_roff[1 << TILE_R];
    uint16_t ld_lo[32], ld_hi[TILE_THREADS / 32];
    uint16_t st_lo[32], st_hi[TILE_THREADS / 32];
};
static_assert(sizeof(TileStage) % 4 == 0, "stages are copied to shared memory in 4-byte words");
enum : uint16_t { SYNC_NONE = 0, SYNC_GROUP = 1, SYNC_WARP = 2 };
constexpr int TILE_TB = 2 * (32 + TILE_THREADS / 32);  // per-stage lane/warp table entries
constexpr int TILE_MAX_GRAD = 32;                        // gradient ops per pass
// States of at most this many qubits (4 tiles, so launches of at most 4 blocks,
// where the shared memory of the gradient columns costs no occupancy) take up
// to TILE_MAX_GRAD_SMALL gradient ops per pass: fewer, longer passes where
// launch latency, not HBM, sets the time.
constexpr int TILE_SMALL_QUBITS = 14;
constexpr int TILE_MAX_GRAD_SMALL = 104;

// Ring kernels (complex64): groups of 256 threads per block, plus one warp
// that issues the TMA copies, and tile buffers in the ring.  Forward: 3 groups, 6 buffers of 32 KiB (three tiles being
// computed, three loading).  Reverse sweep: 2 groups, 3 buffers of 64 KiB
// (psi and lambda).
template <bool ADJ> struct RingCfg {
    static constexpr int G = ADJ ? 2 : 3;
    static constexpr int B = ADJ ? 3 : 6;
    // threads of a block: the groups, and the TMA warpgroup when there is one
    static constexpr int THREADS = G * TILE_THREADS;
    static constexpr int THREADS_TMAW = G * TILE_THREADS + 128;
    // With the TMA warpgroup: registers per thread at launch (the most the
    // launch bounds allow with THREADS_TMAW threads: five or seven warps per
    // scheduler), then moved from the TMA warpgroup (setmaxnreg.dec to
    // REGS_TMA) to the groups (setmaxnreg.inc to REGS_GROUP).  The two shares
    // add up to the launch's registers exactly:
    //   G * 256 * REGS_GROUP + 128 * REGS_TMA == THREADS_TMAW * REGS_LAUNCH.
    static constexpr int REGS_LAUNCH = ADJ ? 96 : 72;
    static constexpr int REGS_TMA = ADJ ? 32 : 24;
    static constexpr int REGS_GROUP = ADJ ? 112 : 80;
};
static_assert(RingCfg<true>::G * TILE_THREADS * RingCfg<true>::REGS_GROUP + 128 * RingCfg<true>::REGS_TMA ==
                  RingCfg<true>::THREADS_TMAW * RingCfg<true>::REGS_LAUNCH,
              "register shares of the reverse ring");
static_assert(RingCfg<false>::G * TILE_THREADS * RingCfg<false>::REGS_GROUP + 128 * RingCfg<false>::REGS_TMA ==
                  RingCfg<false>::THREADS_TMAW * RingCfg<false>::REGS_LAUNCH,
              "register shares of the forward ring");
// Gradient partials of the reverse sweep: one FP64 column per compute warp of
// a block and gradient op.
constexpr int TILE_WARPS = TILE_THREADS / 32;

// Scalar part of a pass descriptor.
struct TileHead {
    int n;                 // qubits of the state
    int n_tiles_log2;      // n - K
    int n_extra;           // top local bits not covered by the TMA box (2^n_extra copies per tile)
    int rank;              // tensor-map rank
    int dim_lo[TILE_MAX_DIMS];    // lowest qubit of each tensor dimension
    int dim_len[TILE_MAX_DIMS];   // qubits in each tensor dimension
    int out_bits[40];      // qubits outside Q, ascending (tile index bit i -> qubit out_bits[i])
    int extra_bits[8];     // qubits of the extra local bits, ascending
    int n_stages;
    int n_ops;
    int n_grad;
    int pool_len;          // matrix pool length (scalars)
    int n_subs;
    int n_dg;              // diagonal runs (each has a 16-entry phase table)
    int pad[4];
};

// Everything a tile kernel needs for one pass.  It lives in device memory
// (uploaded once per circuit); each block copies the parts it uses into
// shared memory.
struct TilePassDev {
    TileHead h;
    TileStage stages[TILE_MAX_STAGES];
    TileOp ops[TILE_MAX_OPS];
    TileSub subs[TILE_MAX_SUBS];
    int32_t op_gate[TILE_MAX_OPS];        // circuit gate index of each op (matrix row)
    int32_t sub_gate[TILE_MAX_SUBS];      // circuit gate index of each diagonal sub-op
    int32_t grad_gate_slot[TILE_MAX_OPS]; // circuit gradient slot of each gradient op
    int16_t dg_op[TILE_MAX_DG];           // op index of each diagonal run
};

}  // namespace tqd
