// plan_check.cu -- tqd_plan_check: the fused plan executed on the host from
// its encoded descriptors, against applying the gates one by one.
//
// Host code only.  It reads the descriptors the tile kernels read (qubit set
// of each pass, every stage's load and store address tables, every op's
// positions and gate) and moves amplitudes the way the kernels do, so a
// planning or encoding mistake shows up as a wrong amplitude without a GPU.
// Stage semantics: register j of thread (lane, warp) holds the amplitude at
// local index unswizzle(lo[lane] ^ hi[warp] ^ roff[j]); ops act on the local
// bits their positions name (register position r -> reg[r], thread position
// u -> thr[u]); the reverse sweep loads through the store tables, applies
// the inverse ops in reverse order and stores through the load tables.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "gate_mat.h"
#include "plan.h"
#include "tile_plan.h"

namespace tqd {
namespace {

typedef std::complex<double> cplx;

// swizzled tile offset -> local index (the swizzle is an involution)
uint32_t unswizzle(uint32_t v, int dt) { return dt == 0 ? (v ^ (((v >> 4) & 7u) << 1)) : (v ^ ((v >> 3) & 7u)); }

struct Mat {
    cplx e[4][4];
    int d;
};

Mat matrix_of_gate(const tqd_circuit *c, const GateH &h, const double *params) {
    double m[MAT_STRIDE];
    gate_matrix(h.kind, h.param >= 0 ? params[h.param] : h.fixed, c->table.data(), h.mat, m);
    Mat r;
    r.d = gate_arity(h.kind) == 2 ? 4 : 2;
    for (int i = 0; i < r.d; ++i)
        for (int j = 0; j < r.d; ++j) r.e[i][j] = cplx(m[2 * (i * r.d + j)], m[2 * (i * r.d + j) + 1]);
    return r;
}
Mat matrix_of(const tqd_circuit *c, int g, const double *params) { return matrix_of_gate(c, c->gates[g], params); }

// v <- M v (or M^dagger v) on bit positions b0 (most significant) and b1.
void apply_bits(std::vector<cplx> &v, const Mat &M, int b0, int b1, bool dag) {
    const size_t N = v.size();
    if (M.d == 2) {
        const size_t T = (size_t)1 << b0;
        for (size_t i = 0; i < N; ++i) {
            if (i & T) continue;
            const cplx x0 = v[i], x1 = v[i | T];
            cplx y[2] = {0, 0};
            for (int r = 0; r < 2; ++r) {
                const cplx a = dag ? std::conj(M.e[0][r]) : M.e[r][0], b = dag ? std::conj(M.e[1][r]) : M.e[r][1];
                y[r] = a * x0 + b * x1;
            }
            v[i] = y[0];
            v[i | T] = y[1];
        }
        return;
    }
    const size_t P = (size_t)1 << b0, Q = (size_t)1 << b1;
    for (size_t i = 0; i < N; ++i) {
        if ((i & P) || (i & Q)) continue;
        const size_t idx[4] = {i, i | Q, i | P, i | P | Q};
        cplx x[4], y[4];
        for (int k = 0; k < 4; ++k) x[k] = v[idx[k]];
        for (int r = 0; r < 4; ++r) {
            y[r] = 0;
            for (int k = 0; k < 4; ++k) y[r] += (dag ? std::conj(M.e[k][r]) : M.e[r][k]) * x[k];
        }
        for (int k = 0; k < 4; ++k) v[idx[k]] = y[k];
    }
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One pass over every tile of psi, forward or reverse, from descriptor D.
// Returns false when a barrier flag is weaker than the address tables allow
// (a point marked SYNC_NONE where a thread meets another thread's amplitudes,
// or SYNC_WARP where a warp meets another warp's).
bool run_pass(const tqd_circuit *c, const TilePlanPass &P, int dt, const double *params, bool rev,
              std::vector<cplx> &psi) {
    const TilePassDev &D = P.dev[dt];
    const TileLayout &L = P.layout;
    const int n = c->n, nt = n - TILE_K;
    const int TS = 1 << TILE_K;
    std::vector<cplx> tile(TS), a(TS);
    // the gates of the pass's ops and diagonal sub-ops, once
    std::vector<Mat> op_m(D.h.n_ops), sub_m(D.h.n_subs);
    for (int k = 0; k < D.h.n_ops; ++k)
        if (D.ops[k].type != TOP_DG && D.ops[k].type != TOP_CX && D.ops[k].type != TOP_SW)
            op_m[k] = matrix_of(c, D.op_gate[k], params);
    for (int k = 0; k < D.h.n_subs; ++k) sub_m[k] = matrix_of(c, D.sub_gate[k], params);
    // the barrier flags, from the tables: at a point marked SYNC_NONE every
    // thread accesses the same addresses on both sides, at one marked
    // SYNC_WARP every warp does (a warp's 512 addresses)
    auto addr_set = [&](const TileStage &st, bool ld, int t0, int nthr) {
        std::vector<uint32_t> v;
        for (int t = t0; t < t0 + nthr; ++t)
            for (int j = 0; j < (1 << TILE_R); ++j)
                v.push_back(ld ? (st.ld_lo[t & 31] ^ st.ld_hi[t >> 5] ^ st.ld_roff[j])
                               : (st.st_lo[t & 31] ^ st.st_hi[t >> 5] ^ st.st_roff[j]));
        std::sort(v.begin(), v.end());
        return v;
    };
    auto point_ok = [&](uint16_t lvl, const TileStage &a, bool a_ld, const TileStage &b, bool b_ld) {
        if (lvl == SYNC_GROUP) return true;
        if (lvl != SYNC_NONE && lvl != SYNC_WARP) return false;
        const int width = lvl == SYNC_NONE ? 1 : 32;
        for (int t0 = 0; t0 < TILE_THREADS; t0 += width)
            if (addr_set(a, a_ld, t0, width) != addr_set(b, b_ld, t0, width)) return false;
        return true;
    };
    for (int s = 0; s < D.h.n_stages; ++s) {
        const TileStage &st = D.stages[s];
        if (!point_ok(st.sync_mid, st, true, st, false)) return false;
        if (s + 1 < D.h.n_stages && !point_ok(st.sync_end, st, false, D.stages[s + 1], true)) return false;
    }
    for (uint64_t t = 0; t < (1ull << nt); ++t) {
        uint64_t origin = 0;
        for (int i = 0; i < nt; ++i)
            if ((t >> i) & 1) origin |= 1ull << L.out[i];
        auto gidx = [&](uint32_t l) {
            uint64_t g = origin;
            for (int i = 0; i < TILE_K; ++i)
                if ((l >> i) & 1) g |= 1ull << L.qubit_of_local[i];
            return g;
        };
        for (int l = 0; l < TS; ++l) tile[l] = psi[gidx(l)];
        for (int si = 0; si < D.h.n_stages; ++si) {
            const TileStage &st = D.stages[rev ? D.h.n_stages - 1 - si : si];
            auto addr = [&](uint32_t y, bool load_tables) {
                uint32_t lane = 0, warp = 0, j = 0;
                for (int u = 0; u < 5; ++u) lane |= ((y >> st.thr[u]) & 1u) << u;
                for (int u = 5; u < TILE_T; ++u) warp |= ((y >> st.thr[u]) & 1u) << (u - 5);
                for (int r = 0; r < TILE_R; ++r) j |= ((y >> st.reg[r]) & 1u) << r;
                const uint32_t v = load_tables ? (st.ld_lo[lane] ^ st.ld_hi[warp] ^ st.ld_roff[j])
                                               : (st.st_lo[lane] ^ st.st_hi[warp] ^ st.st_roff[j]);
                return unswizzle(v, dt);
            };
            for (int y = 0; y < TS; ++y) a[y] = tile[addr(y, !rev)];
            auto bit = [&](uint8_t pos) { return (pos & 0x80) ? (int)st.thr[pos & 0x7f] : (int)st.reg[pos]; };
            auto is_tile = [](uint8_t pos) { return (pos & 0xC0) == TILE_POS_TILE; };
            auto tile_bit = [&](uint8_t pos) { return (int)((origin >> (pos & 0x3f)) & 1u); };
            auto one = [&](int k) {
                const TileOp &op = D.ops[k];
                if (op.type == TOP_DG) {
                    for (int i = 0; i < op.nsub; ++i) {
                        const int q = rev ? op.sub0 + op.nsub - 1 - i : op.sub0 + i;
                        const TileSub &sb = D.subs[q];
                        if (is_tile(sb.a)) {
                            // a qubit outside the pass's set: its bit is the tile's
                            const Mat &M = sub_m[q];
                            const int ta = tile_bit(sb.a);
                            if (sb.type == TOP_D1) {
                                const cplx d = ta ? M.e[1][1] : M.e[0][0];
                                for (auto &x : a) x *= rev ? std::conj(d) : d;
                            } else if (is_tile(sb.b)) {
                                if (ta && tile_bit(sb.b))
                                    for (auto &x : a) x *= rev ? std::conj(M.e[3][3]) : M.e[3][3];
                            } else if (ta) {
                                Mat P1;
                                P1.d = 2;
                                P1.e[0][0] = 1;
                                P1.e[0][1] = P1.e[1][0] = 0;
                                P1.e[1][1] = M.e[3][3];
                                apply_bits(a, P1, bit(sb.b), 0, rev);
                            }
                            continue;
                        }
                        apply_bits(a, sub_m[q], bit(sb.a), sb.type == TOP_D2 ? bit(sb.b) : 0, rev);
                    }
                    return;
                }
                if (op.type == TOP_CX || op.type == TOP_SW) {
                    Mat M;
                    M.d = 4;
                    for (auto &row : M.e)
                        for (auto &x : row) x = 0;
                    if (op.type == TOP_CX) M.e[0][0] = M.e[1][1] = M.e[2][3] = M.e[3][2] = 1;
                    else M.e[0][0] = M.e[1][2] = M.e[2][1] = M.e[3][3] = 1;
                    apply_bits(a, M, bit(op.a), bit(op.b), rev);
                    return;
                }
                apply_bits(a, op_m[k], bit(op.a), op_m[k].d == 4 ? bit(op.b) : 0, rev);
            };
            if (!rev)
                for (int k = st.op_begin; k < st.op_end; ++k) one(k);
            else
                for (int k = (int)st.op_end - 1; k >= (int)st.op_begin; --k) one(k);
            for (int y = 0; y < TS; ++y) tile[addr(y, rev)] = a[y];
        }
        for (int l = 0; l < TS; ++l) psi[gidx(l)] = tile[l];
    }
    return true;
}

}  // namespace

tqd_status plan_check_host(tqd_circuit *c, const double *params, uint64_t seed, double *err_fwd, double *err_rev,
                           int *n_passes, int *n_stages) {
    c->opts.mode = TQD_PLAN_FUSED;
    // the reference applies the gate list as given; the plan runs it with
    // the qubit order kept lazily (SWAPs relabel the gates after them)
    const std::vector<GateH> given = c->gates;
    relabel_swaps(c->gates, c->n);
    assign_grad_slots(c);
    int prefix = 0;
    std::vector<TilePlanPass> passes = plan_fused(c, &prefix);
    if (passes.empty()) {
        set_error("tqd_plan_check: the circuit could not be planned into fused passes");
        return TQD_ERR_UNSUPPORTED;
    }
    int stages = 0;
    for (auto &p : passes) {
        if (!encode_tile_pass(c, p)) {
            set_error("tqd_plan_check: a pass could not be encoded");
            return TQD_ERR_UNSUPPORTED;
        }
        stages += p.dev[0].h.n_stages;
    }
    const size_t N = (size_t)1 << c->n;
    std::vector<cplx> psi0(N);
    double nrm = 0;
    for (auto &x : psi0) {
        const double re = (double)(splitmix(seed) >> 11) * 0x1.0p-53 - 0.5;
        const double im = (double)(splitmix(seed) >> 11) * 0x1.0p-53 - 0.5;
        x = cplx(re, im);
        nrm += std::norm(x);
    }
    for (auto &x : psi0) x /= sqrt(nrm);
    std::vector<cplx> ref = psi0;
    for (const GateH &h : given) apply_bits(ref, matrix_of_gate(c, h, params), h.w[0], h.nw > 1 ? h.w[1] : 0, false);
    double ef = 0, er = 0;
    for (int dt = 0; dt < 2; ++dt) {
        std::vector<cplx> psi = psi0;
        for (auto &p : passes)
            if (!run_pass(c, p, dt, params, false, psi)) {
                set_error("tqd_plan_check: a stage moves amplitudes between threads without its mid-stage barrier");
                return TQD_ERR_NUMERIC;
            }
        for (size_t i = 0; i < N; ++i) ef = std::max(ef, std::abs(psi[i] - ref[i]));
        for (int p = (int)passes.size() - 1; p >= 0; --p) run_pass(c, passes[p], dt, params, true, psi);
        for (size_t i = 0; i < N; ++i) er = std::max(er, std::abs(psi[i] - psi0[i]));
    }
    *err_fwd = ef;
    *err_rev = er;
    if (n_passes) *n_passes = (int)passes.size();
    if (n_stages) *n_stages = stages;
    return TQD_OK;
}

}  // namespace tqd
