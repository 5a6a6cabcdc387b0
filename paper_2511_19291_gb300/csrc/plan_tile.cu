// plan_tile.cu -- host planner of the fused tile passes.
//
// 1. Passes.  Starting at the first gate not yet done, the pass's qubit set Q
//    is qubits 0..3 plus the first other qubits touched, in gate order, by
//    gates that are not diagonal (up to 12).  Gates are then absorbed in
//    order: a gate joins the pass when no earlier gate left out of the pass
//    touches any of its wires and either all its wires are in Q or it is
//    diagonal.  A diagonal gate on a qubit outside Q multiplies each
//    amplitude by a phase of its index bits, and the bits outside Q are the
//    same for all amplitudes of a tile, so the kernels apply it from the
//    tile's origin.  Every gate left out commutes with every absorbed gate
//    after it, so executing the pass before the rest preserves the circuit;
//    two absorbed gates on the same qubit outside Q are both diagonal and
//    commute.  A pass whose ops do not fit the descriptor is cut back to a
//    prefix of its gates (the rest stay for later passes).
// 2. TMA box.  Q's qubits above 3 are grouped into runs; the tensor map has at
//    most 5 dimensions, so runs that do not fit become "extra" bits, copied by
//    2^extra TMA operations per tile.
// 3. Stages.  A stage fixes 4 register bits and takes, in gate order, every
//    gate whose predecessors are scheduled or taken by the same stage and
//    whose dense qubits fit in the register set.  Thread-index bits are
//    assigned so that a half-warp's shared-memory accesses fall in different
//    banks under the 128-byte swizzle.
// 4. Barriers.  Between a stage's loads and stores, and between one stage's
//    stores and the next one's loads, the group of 256 threads meets unless
//    every warp (then __syncwarp) or every thread (then nothing) accesses the
//    same addresses on both sides, which the address tables decide exactly.
//    Warp bits fixed to three bankless bits that are thread bits in every
//    stage make more points warp-local; that choice is taken when it needs
//    fewer group barriers.  (Taking warp bits among the bank-relevant bits
//    instead made about half the stage changes of the 26-qubit ansatz
//    warp-local but slowed its passes by about 30 %: bank conflicts cost more
//    than the barriers saved.)
#include <string.h>

#include <algorithm>
#include <array>
#include <vector>

#include "launch.h"
#include "tile.h"
#include "tile_plan.h"

namespace tqd {

constexpr int TC_QUBITS = 6;       // qubits of a tensor-core block
constexpr int TC_MIN_GATES = 16;   // shortest run worth a block

namespace {

// Register bits a gate needs in its stage (local bits).
void dense_needs(const GateH &g, const int *loc, int *out, int &cnt) {
    cnt = 0;
    switch (g.kind) {
    case TQD_H: case TQD_X: case TQD_Y: case TQD_RX: case TQD_RY: case TQD_UNITARY1:
        out[cnt++] = loc[g.w[0]];
        break;
    case TQD_CNOT:
        out[cnt++] = loc[g.w[1]];
        break;
    case TQD_SWAP: case TQD_UNITARY2:
        out[cnt++] = loc[g.w[0]];
        out[cnt++] = loc[g.w[1]];
        break;
    default:
        break;  // diagonal gates: any bit
    }
}

uint8_t op_type_of(int kind) {
    switch (kind) {
    case TQD_H: case TQD_X: case TQD_Y: case TQD_RX: case TQD_RY: case TQD_UNITARY1: return TOP_G1;
    case TQD_Z: case TQD_S: case TQD_T: case TQD_RZ: case TQD_PHASE: return TOP_D1;
    case TQD_CNOT: return TOP_CX;
    case TQD_SWAP: return TOP_SW;
    case TQD_UNITARY2: return TOP_G2;
    default: return TOP_D2;  // CZ, CPHASE
    }
}

// Segments of [from, n): maximal runs of equal membership, in-runs capped at 8.
struct Seg {
    int lo, len;
    bool in;
};
std::vector<Seg> segments(const std::vector<char> &box, int from, int n) {
    std::vector<Seg> out;
    int b = from;
    while (b < n) {
        const bool in = box[b] != 0;
        int e = b;
        while (e < n && (box[e] != 0) == in && (!in || e - b < 8)) ++e;
        out.push_back(Seg{b, e - b, in});
        b = e;
    }
    return out;
}

// Swizzled shared-memory offset of local index l (units of amplitudes).
uint32_t swz_host(uint32_t l, int amp_bytes) {
    return amp_bytes == 8 ? (l ^ (((l >> 4) & 7u) << 1)) : (l ^ ((l >> 3) & 7u));
}

// Affine map over GF(2) on 12-bit local indices: x -> L x ^ v.
struct Aff {
    uint32_t col[TILE_K];
    uint32_t v;
    Aff() : v(0) {
        for (int i = 0; i < TILE_K; ++i) col[i] = 1u << i;
    }
    uint32_t lin(uint32_t x) const {
        uint32_t r = 0;
        for (int i = 0; i < TILE_K; ++i)
            if ((x >> i) & 1) r ^= col[i];
        return r;
    }
    uint32_t operator()(uint32_t x) const { return lin(x) ^ v; }
};
// (f o h)(x) = f(h(x))
Aff compose(const Aff &f, const Aff &h) {
    Aff r;
    for (int i = 0; i < TILE_K; ++i) r.col[i] = f.lin(h.col[i]);
    r.v = f(h.v);
    return r;
}
bool is_perm_gate(int kind) { return kind == TQD_CNOT || kind == TQD_SWAP || kind == TQD_X; }
// The permutation of local indices a CNOT / SWAP / X performs (each is its own inverse).
Aff perm_map(const GateH &g, const int *loc) {
    Aff m;
    if (g.kind == TQD_CNOT) {
        const int c = loc[g.w[0]], t = loc[g.w[1]];
        m.col[c] ^= 1u << t;
    } else if (g.kind == TQD_SWAP) {
        const int p = loc[g.w[0]], q = loc[g.w[1]];
        m.col[p] = 1u << q;
        m.col[q] = 1u << p;
    } else {
        m.v = 1u << loc[g.w[0]];
    }
    return m;
}

// Lowest local bit that plays no part in the shared-memory bank of an
// amplitude under the 128-byte swizzle (complex64: bits 0..6; complex128:
// bits 0..5).
int first_bankless_bit(int dt) { return dt == 0 ? 7 : 6; }

// Thread bits of a stage (u -> local bit): the lane bits first, one
// representative of each bank class under the swizzle, so that a half-warp's
// accesses fall in different banks, then the other free bits in ascending
// order; the last three are the warp bits.  `warp` (3 bits, free in the
// stage, bankless) fixes the warp bits instead; the lanes are then the other
// free bits.
std::vector<int> thread_bits(const bool *is_reg, int dt, const std::vector<int> &warp) {
    std::vector<int> lanes;
    auto taken = [&](int b) {
        return std::find(lanes.begin(), lanes.end(), b) != lanes.end() ||
               std::find(warp.begin(), warp.end(), b) != warp.end();
    };
    const int classes64[4][2] = {{0, -1}, {1, 4}, {2, 5}, {3, 6}};
    const int classes128[3][2] = {{0, 3}, {1, 4}, {2, 5}};
    const int ncls = dt == 0 ? 4 : 3;
    for (int k = 0; k < ncls; ++k)
        for (int t = 0; t < 2; ++t) {
            const int b = dt == 0 ? classes64[k][t] : classes128[k][t];
            if (b >= 0 && !is_reg[b] && !taken(b)) {
                lanes.push_back(b);
                break;
            }
        }
    for (int b = 0; b < TILE_K; ++b)
        if (!is_reg[b] && !taken(b)) lanes.push_back(b);
    if (!warp.empty()) {
        lanes.resize(TILE_T - 3);
        lanes.insert(lanes.end(), warp.begin(), warp.end());
    }
    lanes.resize(TILE_T);
    return lanes;
}

// Local indices each thread of a stage loads or stores (through map M):
// out[t] = the 16 indices of thread t, sorted.
void thread_sets(const Aff &M, const int *reg, const std::vector<int> &thr,
                 std::vector<std::array<uint32_t, 1 << TILE_R>> &out) {
    out.resize(TILE_THREADS);
    for (int t = 0; t < TILE_THREADS; ++t) {
        uint32_t ot = 0;
        for (int u = 0; u < TILE_T; ++u)
            if ((t >> u) & 1) ot |= 1u << thr[u];
        for (int j = 0; j < (1 << TILE_R); ++j) {
            uint32_t o = ot;
            for (int r = 0; r < TILE_R; ++r)
                if ((j >> r) & 1) o |= 1u << reg[r];
            out[t][j] = M(o);
        }
        std::sort(out[t].begin(), out[t].end());
    }
}

// The barrier a point between two accesses of the tile needs, from the
// index sets before (a) and after (b) it: SYNC_NONE when every thread's two
// sets are equal (each thread only meets its own amplitudes), SYNC_WARP when
// every warp's are (each warp only meets its own), else SYNC_GROUP.
uint16_t sync_level(const std::vector<std::array<uint32_t, 1 << TILE_R>> &a,
                    const std::vector<std::array<uint32_t, 1 << TILE_R>> &b) {
    bool per_thread = true;
    for (int t = 0; t < TILE_THREADS && per_thread; ++t) per_thread = a[t] == b[t];
    if (per_thread) return SYNC_NONE;
    for (int w = 0; w < TILE_THREADS / 32; ++w) {
        std::vector<uint32_t> x, y;
        for (int l = 0; l < 32; ++l) {
            x.insert(x.end(), a[w * 32 + l].begin(), a[w * 32 + l].end());
            y.insert(y.end(), b[w * 32 + l].begin(), b[w * 32 + l].end());
        }
        std::sort(x.begin(), x.end());
        std::sort(y.begin(), y.end());
        if (x != y) return SYNC_GROUP;
    }
    return SYNC_WARP;
}

}  // namespace

// Box bits of a tile for a tensor map whose inner dimension holds the qubits
// below `low`: all of Q, less the extras, taken from the top runs until the
// map has <= 5 dimensions.  The extras are always Q's highest runs.
static bool tile_box(int n, const std::vector<char> &inQ, int low, std::vector<char> &box, std::vector<int> &extra) {
    box = inQ;
    extra.clear();
    for (int iter = 0; iter < 16; ++iter) {
        const std::vector<Seg> s = segments(box, low, n);
        const int dims = 1 + (int)s.size();
        if (dims <= TILE_MAX_DIMS) break;
        // move the highest in-run of the box to the extras
        int hi = -1;
        for (int i = (int)s.size() - 1; i >= 0; --i)
            if (s[i].in) { hi = i; break; }
        if (hi < 0) return false;
        for (int b = s[hi].lo; b < s[hi].lo + s[hi].len; ++b) {
            box[b] = 0;
            extra.push_back(b);
        }
    }
    std::sort(extra.begin(), extra.end());
    return (int)extra.size() <= 4;
}

bool tile_layout(int n, const std::vector<char> &inQ, TileLayout &L) {
    // Extras per precision: complex128's 3-bit inner dimension can need more
    // dimensions than complex64's 4-bit one, so complex64 takes its own (a
    // subset: both are Q's highest runs).  The local order is box bits
    // ascending, then extra bits ascending; extras being the highest runs,
    // that is Q ascending either way, so both precisions share it.
    std::vector<char> box[2];
    for (int dt = 0; dt < 2; ++dt)
        if (!tile_box(n, inQ, dt == 0 ? TILE_LOW : TILE_LOW - 1, box[dt], L.extra_dt[dt])) return false;
    L.extra = L.extra_dt[1];
    L.qubit_of_local.clear();
    for (int b = 0; b < n; ++b)
        if (box[1][b]) L.qubit_of_local.push_back(b);
    for (int b : L.extra) L.qubit_of_local.push_back(b);
    if ((int)L.qubit_of_local.size() != TILE_K) return false;
    for (size_t i = 1; i < L.qubit_of_local.size(); ++i)
        if (L.qubit_of_local[i] <= L.qubit_of_local[i - 1]) return false;  // not Q ascending
    for (int dt = 0; dt < 2; ++dt) {
        const int low = dt == 0 ? TILE_LOW : TILE_LOW - 1;
        const std::vector<Seg> s = segments(box[dt], low, n);
        L.rank[dt] = 1 + (int)s.size();
        if (L.rank[dt] > TILE_MAX_DIMS) return false;
        L.dim_lo[dt][0] = 0;
        L.dim_len[dt][0] = low;
        L.dim_in[dt][0] = 1;
        for (size_t i = 0; i < s.size(); ++i) {
            L.dim_lo[dt][i + 1] = s[i].lo;
            L.dim_len[dt][i + 1] = s[i].len;
            L.dim_in[dt][i + 1] = s[i].in ? 1 : 0;
        }
    }
    L.out.clear();
    for (int b = 0; b < n; ++b)
        if (!inQ[b]) L.out.push_back(b);
    return true;
}

std::vector<TilePlanPass> plan_tile_passes(const tqd_circuit *c, int g_begin, int g_end) {
    const int n = c->n;
    const int L = (int)c->gates.size();
    if (g_end < 0 || g_end > L) g_end = L;
    std::vector<TilePlanPass> passes;
    // gates outside [g_begin, g_end) count as done
    std::vector<char> done(L, 0);
    for (int g = 0; g < L; ++g) done[g] = g < g_begin || g >= g_end;
    int first = g_begin;
    while (first < L && done[first]) ++first;
    while (first < L) {
        // --- tensor-core block: a long run of gates on qubits 0..5
        if (c->opts.mode == TQD_PLAN_TC) {
            std::vector<int> blk;
            std::vector<char> blocked(n, 0);
            int nb = 0;
            for (int g = first; g < L && nb < TC_QUBITS && (int)blk.size() < TILE_MAX_OPS; ++g) {
                if (done[g]) continue;
                const GateH &gh = c->gates[g];
                bool ok = c->grad_slot[g] < 0 || true;
                for (int a = 0; a < gh.nw && ok; ++a) ok = gh.w[a] < TC_QUBITS && !blocked[gh.w[a]];
                if (ok) {
                    blk.push_back(g);
                } else {
                    for (int a = 0; a < gh.nw; ++a)
                        if (!blocked[gh.w[a]]) {
                            blocked[gh.w[a]] = 1;
                            if (gh.w[a] < TC_QUBITS) ++nb;
                        }
                }
            }
            int ngrad = 0;
            for (int g : blk) ngrad += c->grad_slot[g] >= 0 ? 1 : 0;
            if ((int)blk.size() >= TC_MIN_GATES && ngrad <= TILE_MAX_GRAD) {
                std::vector<char> inQ(n, 0);
                for (int q = 0; q < TILE_K; ++q) inQ[q] = 1;
                TilePlanPass P;
                if (!tile_layout(n, inQ, P.layout)) return {};
                P.gates = blk;
                P.tc = 0;  // marked; the circuit builder assigns the block
                for (int g : blk) done[g] = 1;
                passes.push_back(P);
                while (first < L && done[first]) ++first;
                continue;
            }
        }
        // --- qubit set: low qubits, then the qubits of gates in order, each
        // addition accepted only if the TMA box still fits
        std::vector<char> inQ(n, 0);
        int qn = 0;
        for (int q = 0; q < TILE_LOW; ++q) { inQ[q] = 1; ++qn; }
        TileLayout lay;
        // strict: refuse qubits whose padded set needs separate box copies in
        // complex64 (such passes copy each tile as 2^e small boxes, several
        // times slower than one box); the first gate's qubits are always taken
        auto try_add = [&](const int *ws, int cnt, bool strict) {
            int newq = 0;
            for (int a = 0; a < cnt; ++a) newq += inQ[ws[a]] ? 0 : 1;
            if (newq == 0) return true;
            if (qn + newq > TILE_K) return false;
            std::vector<char> t(inQ);
            for (int a = 0; a < cnt; ++a) t[ws[a]] = 1;
            // the layout needs exactly K bits: check with the set padded by the
            // lowest free qubits above the highest run (contiguous padding adds
            // no segments below it)
            std::vector<char> pad(t);
            int have = qn + newq;
            for (int q = TILE_LOW; q < n && have < TILE_K; ++q)
                if (!pad[q] && pad[q - 1]) { pad[q] = 1; ++have; }
            for (int q = TILE_LOW; q < n && have < TILE_K; ++q)
                if (!pad[q]) { pad[q] = 1; ++have; }
            TileLayout tl;
            if (!tile_layout(n, pad, tl)) return false;
            if (strict && !tl.extra_dt[0].empty()) return false;
            inQ.swap(t);
            qn += newq;
            return true;
        };
        int scanned = 0;
        for (int g = first; g < L && qn < TILE_K && scanned < 4096; ++g) {
            if (done[g]) continue;
            ++scanned;
            const GateH &gh = c->gates[g];
            if (gate_diagonal(gh.kind)) continue;  // needs none of its qubits in Q
            if (!try_add(gh.w, gh.nw, g != first) && g == first) break;
        }
        // fill: qubits that extend an existing run first, then any; without
        // box copies if possible
        for (int pass2 = 0; pass2 < 4 && qn < TILE_K; ++pass2)
            for (int q = TILE_LOW; q < n && qn < TILE_K; ++q)
                if (!inQ[q] && ((pass2 & 1) || inQ[q - 1] || (q + 1 < n && inQ[q + 1]))) try_add(&q, 1, pass2 < 2);
        if (qn < TILE_K || !tile_layout(n, inQ, lay)) return {};
        {
            const GateH &g0 = c->gates[first];
            for (int a = 0; a < g0.nw && !gate_diagonal(g0.kind); ++a)
                if (!inQ[g0.w[a]]) return {};
        }
        // --- absorb gates
        TilePlanPass P;
        P.layout = lay;
        std::vector<char> blocked(n, 0);
        int blocked_in_q = 0, ngrad = 0, ndiag = 0;
        const int max_grad = n <= TILE_SMALL_QUBITS ? TILE_MAX_GRAD_SMALL : TILE_MAX_GRAD;
        for (int g = first; g < L; ++g) {
            if (done[g]) continue;
            const GateH &gh = c->gates[g];
            const bool is_grad = c->grad_slot[g] >= 0;
            const bool diag = gate_diagonal(gh.kind);
            bool ok = (int)P.gates.size() < TILE_MAX_GATES && (!is_grad || ngrad < max_grad) &&
                      (diag ? ndiag < TILE_MAX_SUBS : (int)P.gates.size() - ndiag < TILE_MAX_OPS);
            for (int a = 0; a < gh.nw && ok; ++a) ok = (diag || inQ[gh.w[a]]) && !blocked[gh.w[a]];
            if (ok) {
                P.gates.push_back(g);
                done[g] = 1;
                if (is_grad) ++ngrad;
                if (diag) ++ndiag;
            } else {
                for (int a = 0; a < gh.nw; ++a) {
                    if (!blocked[gh.w[a]]) {
                        blocked[gh.w[a]] = 1;
                        if (inQ[gh.w[a]]) ++blocked_in_q;
                    }
                }
                if (blocked_in_q == TILE_K) break;
            }
        }
        // a pass whose ops do not fit the descriptor (too many diagonal runs,
        // sub-ops or stages) keeps a prefix of its gates, in circuit order:
        // the gates cut off run in later passes, after every gate kept
        {
            TilePlanPass T = P;
            while (!encode_tile_pass(c, T)) {
                if (P.gates.size() <= 1) return {};
                const size_t keep = P.gates.size() * 3 / 4;
                for (size_t i = keep; i < P.gates.size(); ++i) done[P.gates[i]] = 0;
                P.gates.resize(keep);
                T = P;
            }
        }
        passes.push_back(P);
        while (first < L && done[first]) ++first;
    }
    return passes;
}

// Lazy qubit order (the idea of Algorithm 2, MoveDim^-1 deferred: keep the
// permutation pending instead of moving data).  pi[q] is the bit of the
// stored index that holds qubit q.  A SWAP(a, b) exchanges pi[a] and pi[b]
// and moves no amplitude; every other gate acts on the bits pi of its wires.
// At the end the stored state is the true one with its index bits permuted
// by pi; the SWAPs appended here put every qubit back on its own bit.  They
// end the circuit, so they are its permutation tail: tqd_value_and_grad
// conjugates the observable through them instead of running them, and a run
// of the whole circuit moves the amplitudes once at the end.
bool relabel_swaps(std::vector<GateH> &gates, int n) {
    bool any = false;
    for (const GateH &g : gates) any = any || g.kind == TQD_SWAP;
    if (!any) return false;
    std::vector<int> pi(n);
    for (int q = 0; q < n; ++q) pi[q] = q;
    std::vector<GateH> out;
    out.reserve(gates.size() + n);
    for (GateH g : gates) {
        if (g.kind == TQD_SWAP) {
            std::swap(pi[g.w[0]], pi[g.w[1]]);
            continue;
        }
        for (int a = 0; a < g.nw; ++a) g.w[a] = pi[g.w[a]];
        out.push_back(g);
    }
    for (int q = 0; q < n; ++q) {
        if (pi[q] == q) continue;
        int r = 0;  // the qubit held by bit q
        while (pi[r] != q) ++r;
        GateH s;
        s.kind = TQD_SWAP;
        s.nw = 2;
        s.w[0] = q;
        s.w[1] = pi[q];
        s.w[2] = 0;
        s.param = -1;
        s.fixed = 0.0;
        s.mat = -1;
        out.push_back(s);
        pi[r] = pi[q];
        pi[q] = q;
    }
    gates.swap(out);
    return true;
}

int permutation_tail(const tqd_circuit *c) {
    int t = (int)c->gates.size();
    while (t > 0 && is_perm_gate(c->gates[t - 1].kind)) --t;
    return t;
}

std::vector<TilePlanPass> plan_fused(const tqd_circuit *c, int *prefix_passes) {
    const int tail = permutation_tail(c), L = (int)c->gates.size();
    std::vector<TilePlanPass> passes;
    if (tail > 0) {
        passes = plan_tile_passes(c, 0, tail);
        if (passes.empty()) return passes;
    }
    *prefix_passes = (int)passes.size();
    if (tail < L) {
        std::vector<TilePlanPass> t = plan_tile_passes(c, tail, L);
        if (t.empty()) return t;
        for (auto &p : t) passes.push_back(std::move(p));
    }
    return passes;
}

// Stage scheduling + op encoding for one pass.
bool encode_tile_pass(const tqd_circuit *c, TilePlanPass &P) {
    const int n = c->n;
    const TileLayout &lay = P.layout;
    std::vector<int> loc(n, -1);
    for (int i = 0; i < TILE_K; ++i) loc[lay.qubit_of_local[i]] = i;
    const int m = (int)P.gates.size();
    // dependencies inside the pass (shared local bits)
    std::vector<std::vector<int>> preds(m);
    {
        std::vector<int> last(TILE_K, -1);
        for (int i = 0; i < m; ++i) {
            const GateH &g = c->gates[P.gates[i]];
            for (int a = 0; a < g.nw; ++a) {
                const int lb = loc[g.w[a]];
                if (lb < 0) continue;  // outside Q: diagonal gates, which commute
                if (last[lb] >= 0) preds[i].push_back(last[lb]);
                last[lb] = i;
            }
        }
    }
    std::vector<char> sched(m, 0);
    int nsched = 0;
    std::vector<int> order;  // execution order (indices into P.gates)
    struct StageH {
        int reg[TILE_R];
        int begin, end;
    };
    std::vector<StageH> stages;
    while (nsched < m) {
        // Closure in gate order: a gate joins the stage when each of its
        // predecessors is scheduled or joined earlier in this stage and its
        // dense qubits fit in the stage's register set together with those
        // of the gates already joined.  Joined gates run in gate order.
        // A CNOT, SWAP or X whose predecessors are all scheduled or such
        // leading gates of this stage needs no register bit: the stage runs
        // the leading gates first, folded into its load address map.
        std::vector<int> rs;
        std::vector<char> fit(m, 0), lead(m, 0);
        for (int i = 0; i < m; ++i) {
            if (sched[i]) continue;
            bool preds_ok = true, preds_lead = true;
            for (int p : preds[i]) {
                preds_ok = preds_ok && (sched[p] || fit[p]);
                preds_lead = preds_lead && (sched[p] || lead[p]);
            }
            if (!preds_ok) continue;
            if (preds_lead && is_perm_gate(c->gates[P.gates[i]].kind)) {
                lead[i] = 1;
                fit[i] = 1;
                continue;
            }
            int need[2], cnt;
            dense_needs(c->gates[P.gates[i]], loc.data(), need, cnt);
            std::vector<int> u(rs);
            for (int k = 0; k < cnt; ++k)
                if (std::find(u.begin(), u.end(), need[k]) == u.end()) u.push_back(need[k]);
            if ((int)u.size() > TILE_R) continue;
            rs = u;
            fit[i] = 1;
        }
        // Then trailing permutation gates: a CNOT, SWAP or X that did not fit,
        // whose predecessors are all scheduled, taken or trailing, joins the
        // stage's end (its store address map).  Gates taken above that come
        // later in gate order share no qubit with it (they would depend on
        // it), so moving it after them keeps the circuit.
        std::vector<char> trail(m, 0);
        for (int i = 0; i < m; ++i) {
            if (sched[i] || fit[i] || !is_perm_gate(c->gates[P.gates[i]].kind)) continue;
            bool ok = true;
            for (int p : preds[i]) ok = ok && (sched[p] || fit[p] || trail[p]);
            if (ok) trail[i] = 1;
        }
        StageH st;
        st.begin = (int)order.size();
        for (int part = 0; part < 3; ++part)  // leading, taken, trailing; each in gate order
            for (int i = 0; i < m; ++i) {
                const int which = lead[i] ? 0 : trail[i] ? 2 : fit[i] ? 1 : -1;
                if (which != part) continue;
                sched[i] = 1;
                ++nsched;
                order.push_back(i);
            }
        st.end = (int)order.size();
        if (st.end == st.begin) return false;  // cannot happen: the first ready gate always fits
        // pad the register set: local bit 0 first (registers j and j ^ 1 then
        // hold adjacent amplitudes, one 16-byte access for complex64), then
        // the highest free local bits (they do not help bank spreading as
        // lane bits)
        if ((int)rs.size() < TILE_R && std::find(rs.begin(), rs.end(), 0) == rs.end()) rs.push_back(0);
        for (int b = TILE_K - 1; b >= 0 && (int)rs.size() < TILE_R; --b)
            if (std::find(rs.begin(), rs.end(), b) == rs.end()) rs.push_back(b);
        std::sort(rs.begin(), rs.end());
        for (int r = 0; r < TILE_R; ++r) st.reg[r] = rs[r];
        stages.push_back(st);
    }
    if ((int)stages.size() > TILE_MAX_STAGES) return false;
    const int S = (int)stages.size();

    // Load and store maps of every stage: the permutation gates at its start
    // become the load map F = f1 o f2 o ..., those at its end the store map
    // G = ... o g2 o g1.
    std::vector<Aff> Fm(S), Gm(S);
    std::vector<int> lead_ends(S), trail_begins(S);
    for (int s = 0; s < S; ++s) {
        const StageH &sh = stages[s];
        int lead_end = sh.begin;
        while (lead_end < sh.end && is_perm_gate(c->gates[P.gates[order[lead_end]]].kind)) ++lead_end;
        int trail_begin = sh.end;
        while (trail_begin > lead_end && is_perm_gate(c->gates[P.gates[order[trail_begin - 1]]].kind))
            --trail_begin;
        for (int q = sh.begin; q < lead_end; ++q) Fm[s] = compose(Fm[s], perm_map(c->gates[P.gates[order[q]]], loc.data()));
        for (int q = trail_begin; q < sh.end; ++q) Gm[s] = compose(perm_map(c->gates[P.gates[order[q]]], loc.data()), Gm[s]);
        lead_ends[s] = lead_end;
        trail_begins[s] = trail_begin;
    }

    // Thread bits of every stage and the barriers they need, per precision.
    // Two candidates: the bank-spreading default of each stage, and the same
    // lanes with the warp bits fixed to three bankless bits that are thread
    // bits in every stage (a warp then keeps its part of the tile from stage
    // to stage unless a permutation moves it).  The one with fewer group
    // barriers (then fewer warp barriers) wins.
    struct ThreadPlan {
        std::vector<std::vector<int>> thr;     // [stage][u]
        std::vector<uint16_t> mid, end;        // sync levels
        int cost = 0;
    };
    auto make_plan = [&](int dt, const std::vector<int> &warp) {
        ThreadPlan tp;
        tp.thr.resize(S);
        tp.mid.resize(S);
        tp.end.assign(S, SYNC_GROUP);
        std::vector<std::array<uint32_t, 1 << TILE_R>> ld, st, prev_st;
        for (int s = 0; s < S; ++s) {
            bool is_reg[TILE_K] = {false};
            for (int r = 0; r < TILE_R; ++r) is_reg[stages[s].reg[r]] = true;
            tp.thr[s] = thread_bits(is_reg, dt, warp);
            thread_sets(Fm[s], stages[s].reg, tp.thr[s], ld);
            thread_sets(Gm[s], stages[s].reg, tp.thr[s], st);
            tp.mid[s] = sync_level(ld, st);
            if (s > 0) tp.end[s - 1] = sync_level(prev_st, ld);
            prev_st.swap(st);
        }
        auto weight = [](uint16_t l) { return l == SYNC_GROUP ? 16 : l == SYNC_WARP ? 1 : 0; };
        for (int s = 0; s < S; ++s) tp.cost += weight(tp.mid[s]) + (s + 1 < S ? weight(tp.end[s]) : 0);
        return tp;
    };
    ThreadPlan tplan[2];
    for (int dt = 0; dt < 2; ++dt) {
        tplan[dt] = make_plan(dt, {});
        std::vector<int> common;  // bankless bits that are thread bits in every stage, highest first
        for (int b = TILE_K - 1; b >= first_bankless_bit(dt); --b) {
            bool free_all = true;
            for (int s = 0; s < S && free_all; ++s)
                for (int r = 0; r < TILE_R; ++r) free_all = free_all && stages[s].reg[r] != b;
            if (free_all) common.push_back(b);
        }
        if (common.size() >= 3) {
            ThreadPlan alt = make_plan(dt, std::vector<int>(common.begin(), common.begin() + 3));
            if (alt.cost < tplan[dt].cost) tplan[dt] = std::move(alt);
        }
    }

    // --- encode for both dtypes
    for (int dt = 0; dt < 2; ++dt) {
        TilePassDev &D = P.dev[dt];
        memset(&D, 0, sizeof(D));
        D.h.n = n;
        D.h.n_tiles_log2 = n - TILE_K;
        D.h.n_extra = (int)lay.extra_dt[dt].size();
        D.h.rank = lay.rank[dt];
        for (int d = 0; d < TILE_MAX_DIMS; ++d) {
            D.h.dim_lo[d] = d < D.h.rank ? lay.dim_lo[dt][d] : 0;
            D.h.dim_len[d] = d < D.h.rank ? lay.dim_len[dt][d] : 0;
        }
        for (size_t i = 0; i < lay.out.size(); ++i) D.h.out_bits[i] = lay.out[i];
        for (size_t i = 0; i < lay.extra_dt[dt].size(); ++i) D.h.extra_bits[i] = lay.extra_dt[dt][i];
        D.h.n_stages = (int)stages.size();
        int pool = 0, ngrad = 0, nops = 0, nsubs = 0;
        D.h.n_dg = 0;
        const int amp_bytes = dt == 0 ? 8 : 16;
        for (size_t s = 0; s < stages.size(); ++s) {
            const StageH &sh = stages[s];
            TileStage &ts = D.stages[s];
            bool is_reg[TILE_K] = {false};
            for (int r = 0; r < TILE_R; ++r) {
                ts.reg[r] = (uint8_t)sh.reg[r];
                is_reg[sh.reg[r]] = true;
            }
            for (int u = 0; u < TILE_T; ++u) ts.thr[u] = (uint8_t)tplan[dt].thr[s][u];
            const int lead_end = lead_ends[s], trail_begin = trail_begins[s];
            const Aff &F = Fm[s], &G = Gm[s];
            for (int j = 0; j < (1 << TILE_R); ++j) {
                uint32_t o = 0;
                for (int r = 0; r < TILE_R; ++r)
                    if ((j >> r) & 1) o |= 1u << sh.reg[r];
                ts.ld_roff[j] = (uint16_t)swz_host(F(o), amp_bytes);
                ts.st_roff[j] = (uint16_t)swz_host(G(o), amp_bytes);
            }
            for (int l = 0; l < 32; ++l) {
                uint32_t o = 0;
                for (int u = 0; u < 5; ++u)
                    if ((l >> u) & 1) o |= 1u << ts.thr[u];
                ts.ld_lo[l] = (uint16_t)swz_host(F.lin(o), amp_bytes);
                ts.st_lo[l] = (uint16_t)swz_host(G.lin(o), amp_bytes);
            }
            for (int w = 0; w < TILE_THREADS / 32; ++w) {
                uint32_t o = 0;
                for (int u = 5; u < TILE_T; ++u)
                    if ((w >> (u - 5)) & 1) o |= 1u << ts.thr[u];
                ts.ld_hi[w] = (uint16_t)swz_host(F.lin(o), amp_bytes);
                ts.st_hi[w] = (uint16_t)swz_host(G.lin(o), amp_bytes);
            }
            // barriers from the thread plan: between this stage's loads and
            // stores, and between its stores and the next stage's loads
            ts.sync_mid = tplan[dt].mid[s];
            ts.sync_end = tplan[dt].end[s];
            auto pos = [&](int lb) -> uint8_t {
                for (int r = 0; r < TILE_R; ++r)
                    if (ts.reg[r] == lb) return (uint8_t)r;
                for (int u = 0; u < TILE_T; ++u)
                    if (ts.thr[u] == lb) return (uint8_t)(0x80 | u);
                return 0xff;
            };
            // position of qubit q: a local bit's, or a tile bit's outside Q
            auto posq = [&](int q) -> uint8_t {
                return loc[q] >= 0 ? pos(loc[q]) : (uint8_t)(TILE_POS_TILE | q);
            };
            auto is_tile = [](uint8_t p) { return (p & 0xC0) == TILE_POS_TILE; };
            auto grad_of = [&](int gi, uint8_t &gen, int16_t &gslot) -> bool {
                const int slot = c->grad_slot[gi];
                gen = slot >= 0 ? (uint8_t)gate_gen(c->gates[gi].kind) : 0;
                gslot = -1;
                if (slot >= 0) {
                    if (ngrad >= TILE_MAX_OPS) return false;
                    gslot = (int16_t)ngrad;
                    D.grad_gate_slot[ngrad] = slot;
                    ++ngrad;
                }
                return true;
            };
            // a diagonal gate that can join a run: 1-qubit, or 2-qubit with a
            // tile bit, or with both positions on register bits or both on
            // thread bits
            auto runnable = [&](int gi) {
                const GateH &g = c->gates[gi];
                if (!gate_diagonal(g.kind)) return false;
                if (g.nw == 1) return true;
                const uint8_t pa = posq(g.w[0]), pb = posq(g.w[1]);
                if (is_tile(pa) || is_tile(pb)) return true;
                return ((pa & 0x80) != 0) == ((pb & 0x80) != 0);
            };
            // gates on tile bits exist only inside runs (a run of one, if need be)
            auto on_tile = [&](int gi) {
                const GateH &g = c->gates[gi];
                for (int a = 0; a < g.nw; ++a)
                    if (loc[g.w[a]] < 0) return true;
                return false;
            };
            ts.op_begin = (uint16_t)nops;
            int k = lead_end;
            while (k < trail_begin) {
                const int gi0 = P.gates[order[k]];
                int run_end = k;
                bool run_tile = false;
                while (run_end < trail_begin && runnable(P.gates[order[run_end]])) {
                    run_tile = run_tile || on_tile(P.gates[order[run_end]]);
                    ++run_end;
                }
                if (nops >= TILE_MAX_OPS) return false;
                TileOp &op = D.ops[nops];
                memset(&op, 0, sizeof(op));
                op.moff = -1;
                op.gslot = -1;
                op.sub0 = -1;
                if (run_end - k >= 2 || run_tile) {
                    // diagonal run (b = 1: some of its gates are on tile bits)
                    if (D.h.n_dg >= TILE_MAX_DG || nsubs + (run_end - k) > TILE_MAX_SUBS) return false;
                    op.type = TOP_DG;
                    op.b = run_tile ? 1 : 0;
                    op.moff = (int16_t)D.h.n_dg;
                    op.sub0 = (int16_t)nsubs;
                    op.nsub = (int16_t)(run_end - k);
                    D.dg_op[D.h.n_dg++] = (int16_t)nops;
                    for (int q = k; q < run_end; ++q) {
                        const int gi = P.gates[order[q]];
                        const GateH &g = c->gates[gi];
                        TileSub &sb = D.subs[nsubs];
                        sb.type = g.nw == 1 ? TOP_D1 : TOP_D2;
                        sb.a = posq(g.w[0]);
                        sb.b = g.nw > 1 ? posq(g.w[1]) : 0;
                        // a two-qubit gate on a tile bit has it in a (the phase
                        // is symmetric in the two bits)
                        if (g.nw > 1 && is_tile(sb.b) && !is_tile(sb.a)) {
                            const uint8_t t = sb.a;
                            sb.a = sb.b;
                            sb.b = t;
                        }
                        if (sb.a == 0xff || (g.nw > 1 && sb.b == 0xff)) return false;
                        if (!grad_of(gi, sb.gen, sb.gslot)) return false;
                        const int len = sb.type == TOP_D1 ? 8 : 2;
                        sb.moff = (int16_t)pool;
                        pool += len;
                        D.sub_gate[nsubs] = gi;
                        ++nsubs;
                    }
                    D.op_gate[nops] = gi0;
                    ++nops;
                    k = run_end;
                    continue;
                }
                const GateH &g = c->gates[gi0];
                op.type = op_type_of(g.kind);
                if (op.type == TOP_G1 && (g.kind == TQD_RY || g.kind == TQD_H || g.kind == TQD_X)) op.type = TOP_G1R;
                op.a = pos(loc[g.w[0]]);
                op.b = g.nw > 1 ? pos(loc[g.w[1]]) : 0;
                if (!grad_of(gi0, op.gen, op.gslot)) return false;
                int len = 0;
                switch (op.type) {
                case TOP_G1: case TOP_G1R: case TOP_D1: len = 8; break;
                case TOP_G2: len = 32; break;
                case TOP_D2: len = 2; break;
                default: len = 0; break;
                }
                op.moff = len ? (int16_t)pool : (int16_t)-1;
                pool += len;
                D.op_gate[nops] = gi0;
                if (op.a == 0xff || op.b == 0xff) return false;
                if ((op.type == TOP_G1 || op.type == TOP_G1R || op.type == TOP_SW || op.type == TOP_G2) &&
                    (op.a & 0x80))
                    return false;
                if ((op.type == TOP_CX || op.type == TOP_SW || op.type == TOP_G2) && (op.b & 0x80)) return false;
                ++nops;
                ++k;
            }
            ts.op_end = (uint16_t)nops;
        }
        D.h.n_ops = nops;
        D.h.n_subs = nsubs;
        D.h.n_grad = ngrad;
        D.h.pool_len = pool;
        if (pool > 32000) return false;
    }
    P.order.clear();
    for (int k = 0; k < m; ++k) P.order.push_back(P.gates[order[k]]);
    return true;
}

}  // namespace tqd
