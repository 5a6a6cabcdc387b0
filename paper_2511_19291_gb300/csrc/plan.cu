// plan.cu -- circuit planning (host) and the forward / backward executors.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "jit.h"
#include "launch.h"
#include "plan.h"
#include "tc.h"
#include "tile_plan.h"

namespace tqd {

template <typename T>
static cudaError_t upload(T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Blocks used by every gate-by-gate adjoint step of an n-qubit state.
static int plain_adjoint_blocks(int n) {
    if (n < 4) return 1;
    return stream_grid(((uint64_t)1 << n) / 4, 256);
}

std::vector<std::vector<int>> assign_grad_slots(tqd_circuit *c) {
    // gradient slots: one per parametric gate that reads the parameter vector
    const int ng = (int)c->gates.size();
    c->grad_slot.assign(ng, -1);
    c->n_slots = 0;
    std::vector<std::vector<int>> by_param(c->n_params);
    for (int g = 0; g < ng; ++g) {
        const GateH &h = c->gates[g];
        if (h.param >= 0 && gate_parametric(h.kind)) {
            c->grad_slot[g] = c->n_slots;
            by_param[h.param].push_back(c->n_slots);
            ++c->n_slots;
        }
    }
    return by_param;
}

tqd_status build_circuit(tqd_circuit *c) {
    // fused plans keep the qubit order lazily: SWAPs relabel the gates after them
    if ((c->opts.mode == TQD_PLAN_FUSED || c->opts.mode == TQD_PLAN_TC) && c->n >= TILE_K)
        relabel_swaps(c->gates, c->n);
    const int ng = (int)c->gates.size();
    int dev = 0;
    cudaGetDevice(&dev);
    c->device = dev;
    c->d_gates = nullptr;
    c->d_table = nullptr;
    c->d_mats64 = nullptr;
    c->d_mats32 = nullptr;
    c->d_partials = nullptr;
    c->d_slot_sums = nullptr;
    c->d_param_ptr = nullptr;
    c->d_param_slots = nullptr;
    c->d_err = nullptr;
    c->d_tile_desc = nullptr;
    c->fused = false;
    c->prefix_passes = 0;
    c->tail_gate = (int)c->gates.size();
    c->first_grad_pass = 0;

    std::vector<std::vector<int>> by_param = assign_grad_slots(c);
    std::vector<int> ptr(c->n_params + 1, 0), slots;
    for (int p = 0; p < c->n_params; ++p) {
        ptr[p + 1] = ptr[p] + (int)by_param[p].size();
        for (int s : by_param[p]) slots.push_back(s);
    }
    c->pblk = plain_adjoint_blocks(c->n);

    std::vector<GateDev> gd(ng);
    for (int g = 0; g < ng; ++g) {
        gd[g].kind = c->gates[g].kind;
        gd[g].param = c->gates[g].param;
        gd[g].mat = c->gates[g].mat;
        gd[g].pad = 0;
        gd[g].fixed = c->gates[g].fixed;
    }
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err) {
        set_error("tqd_circuit_create: %s", cudaGetErrorString(err));
        return err == cudaErrorMemoryAllocation ? TQD_ERR_OOM : TQD_ERR_CUDA;
    };
    if ((e = upload(&c->d_gates, gd)) != cudaSuccess) return fail(e);
    if ((e = upload(&c->d_table, c->table)) != cudaSuccess) return fail(e);
    if (ng > 0) {
        if ((e = cudaMalloc((void **)&c->d_mats64, (size_t)ng * MAT_STRIDE * sizeof(double))) != cudaSuccess)
            return fail(e);
        if ((e = cudaMalloc((void **)&c->d_mats32, (size_t)ng * MAT_STRIDE * sizeof(float))) != cudaSuccess)
            return fail(e);
    }
    if (c->n_slots > 0) {
        if ((e = cudaMalloc((void **)&c->d_partials, (size_t)c->n_slots * c->pblk * sizeof(double))) != cudaSuccess)
            return fail(e);
        if ((e = cudaMalloc((void **)&c->d_slot_sums, (size_t)c->n_slots * sizeof(double))) != cudaSuccess)
            return fail(e);
    }
    if ((e = upload(&c->d_param_ptr, ptr)) != cudaSuccess) return fail(e);
    if ((e = upload(&c->d_param_slots, slots)) != cudaSuccess) return fail(e);

    if ((e = cudaMalloc((void **)&c->d_err, sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(c->d_err, 0, sizeof(int))) != cudaSuccess) return fail(e);

    // fused plan: tile passes, when the state holds at least one full tile
    if ((c->opts.mode == TQD_PLAN_FUSED || c->opts.mode == TQD_PLAN_TC) && c->n >= TILE_K && ng > 0) {
        int prefix = 0;
        std::vector<TilePlanPass> passes = plan_fused(c, &prefix);
        bool ok = !passes.empty();
        for (auto &p : passes) ok = ok && encode_tile_pass(c, p);
        if (ok) {
            std::vector<TilePassDev> desc;
            for (auto &p : passes) {
                desc.push_back(p.dev[0]);
                desc.push_back(p.dev[1]);
            }
            if ((e = upload(&c->d_tile_desc, desc)) != cudaSuccess) return fail(e);
            // tensor-core blocks: gate list and operand buffers per marked pass
            for (auto &p : passes) {
                if (p.tc < 0) continue;
                std::vector<TcGate> tg;
                for (int g : p.gates) {
                    const GateH &h = c->gates[g];
                    TcGate t;
                    t.gate = g;
                    t.nw = (uint8_t)h.nw;
                    t.w0 = (uint8_t)h.w[0];
                    t.w1 = (uint8_t)(h.nw > 1 ? h.w[1] : 0);
                    t.pad = 0;
                    tg.push_back(t);
                }
                TcBlock *b = new (std::nothrow) TcBlock();
                if (!b) return fail(cudaErrorMemoryAllocation);
                c->tc_blocks.push_back(b);
                b->n_gates = (int)tg.size();
                if ((e = upload(&b->d_gates, tg)) != cudaSuccess) return fail(e);
                if ((e = cudaMalloc((void **)&b->d_ahi, 128 * 128 * sizeof(float))) != cudaSuccess) return fail(e);
                if ((e = cudaMalloc((void **)&b->d_alo, 128 * 128 * sizeof(float))) != cudaSuccess) return fail(e);
                p.tc = (int)c->tc_blocks.size() - 1;
            }
            c->tile_passes = std::move(passes);
            c->prefix_passes = prefix;
            c->tail_gate = permutation_tail(c);
            c->first_grad_pass = 0;
            while (c->first_grad_pass < (int)c->tile_passes.size() &&
                   c->tile_passes[c->first_grad_pass].dev[0].h.n_grad == 0)
                ++c->first_grad_pass;
            c->fused = true;
            c->n_passes = (int)c->tile_passes.size();
            c->launches_apply = c->n_passes + 1;
            c->launches_backward = c->n_passes + 1 + (c->n_slots > 0 ? 2 : 0);  // + the H psi launches
            return TQD_OK;
        }
    }

    // plain plan: one launch per gate (two for 2-qubit permutations in reverse)
    c->n_passes = ng;
    c->launches_apply = ng + (ng > 0 ? 1 : 0);
    int back = 0;
    for (int g = 0; g < ng; ++g) {
        const GateH &h = c->gates[g];
        const bool one = gate_arity(h.kind) == 1 || h.kind == TQD_CPHASE || h.kind == TQD_CZ || c->n < 4;
        back += one ? 1 : 2;
    }
    c->launches_backward = back + (ng > 0 ? 1 : 0) + (c->n_slots > 0 ? 2 : 0);
    return TQD_OK;
}

void release_circuit(tqd_circuit *c) {
    jit_release(c);
    cudaFree(c->d_gates);
    cudaFree(c->d_table);
    cudaFree(c->d_mats64);
    cudaFree(c->d_mats32);
    cudaFree(c->d_partials);
    cudaFree(c->d_slot_sums);
    cudaFree(c->d_param_ptr);
    cudaFree(c->d_param_slots);
    cudaFree(c->d_err);
    cudaFree(c->d_tile_desc);
    for (void *v : c->tc_blocks) {
        TcBlock *b = (TcBlock *)v;
        cudaFree(b->d_gates);
        cudaFree(b->d_ahi);
        cudaFree(b->d_alo);
        delete b;
    }
    c->tc_blocks.clear();
    cudaFree(c->ck_buf);
    c->ck_buf = nullptr;
    c->ck_bytes = c->ck_state_bytes = 0;
}

cudaError_t checkpoints_for(const tqd_circuit *c, const tqd_state *psi, int np, Checkpoints *out, bool want_psi0) {
    *out = Checkpoints();
    const uint32_t opt = c->opts.checkpoints;
    if (!c->fused || np <= 0 || opt == TQD_CHECKPOINTS_NONE) return cudaSuccess;
    const size_t sb = ((size_t)1 << c->n) * (psi->dtype == TQD_C64 ? 8 : 16);
    int want = np;
    if (opt != 0 && opt < (uint32_t)np) want = (int)opt;
    std::lock_guard<std::mutex> lk(c->ck_mu);
    if (c->ck_state_bytes != sb) {
        // sized once per state size: up to `want` states in half the free memory
        if (c->ck_buf) {
            cudaError_t e = cudaFree(c->ck_buf);
            if (e != cudaSuccess) return e;
            c->ck_buf = nullptr;
            c->ck_bytes = 0;
        }
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) return e;
        size_t k = std::min<size_t>((size_t)want, fr / 2 / sb);
        // a budget the allocator cannot meet in one piece: fewer passes
        for (; k > 0; k /= 2) {
            if (cudaMalloc(&c->ck_buf, k * sb) == cudaSuccess) break;
            (void)cudaGetLastError();
            c->ck_buf = nullptr;
        }
        c->ck_bytes = k * sb;
        c->ck_state_bytes = sb;
    }
    out->base = (char *)c->ck_buf;
    out->stride = sb;
    const int slots = c->ck_buf ? (int)(c->ck_bytes / sb) : 0;
    out->count = std::min(want, slots);
    if (want_psi0 && out->count < np && slots > 0) {
        // some pass runs in place: the last slot keeps the input state
        if (out->count == slots) --out->count;
        out->psi0 = out->at(slots - 1);
    }
    return cudaSuccess;
}

cudaError_t run_forward(tqd_state *psi, const tqd_circuit *c, const double *dev_params, cudaStream_t s,
                        int pass_end, const Checkpoints *ck) {
    cudaError_t e = launch_prep(c, dev_params, s);
    if (e != cudaSuccess) return e;
    if (c->fused) {
        const int np = pass_end < 0 ? (int)c->tile_passes.size() : pass_end;
        const int first = ck ? np - ck->count : np;  // first checkpointed pass
        for (int p = 0; p < np; ++p) {
            const TilePlanPass &pp = c->tile_passes[p];
            const bool tc = pp.tc >= 0 && psi->dtype == TQD_C64;
            if (p < first) {
                e = tc ? launch_tc_block(psi, c, *(const TcBlock *)c->tc_blocks[pp.tc], s)
                       : launch_tile_pass(psi, nullptr, c, p, s);
            } else {
                const void *src = p == first ? psi->amps : ck->at(p - first - 1);
                void *dst = ck->at(p - first);
                if (tc) {
                    // the tensor-core kernel works in place: on a copy
                    e = cudaMemcpyAsync(dst, src, ck->stride, cudaMemcpyDeviceToDevice, s);
                    tqd_state v = *psi;
                    v.amps = dst;
                    if (e == cudaSuccess) e = launch_tc_block(&v, c, *(const TcBlock *)c->tc_blocks[pp.tc], s);
                } else {
                    e = launch_tile_pass(psi, nullptr, c, p, s, src, dst);
                }
            }
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    for (int g = 0; g < (int)c->gates.size(); ++g) {
        e = launch_plain_gate(psi, c, g, false, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t run_backward(tqd_state *psi, tqd_state *lam, const tqd_circuit *c, const double *dev_params,
                         const std::vector<PauliGroup> &groups, const double *dev_weights, double scale,
                         double *dev_grads, cudaStream_t s, double *dev_energy, bool prepared, int pass_end,
                         bool seeded, const Checkpoints *ck, int pass_begin) {
    cudaError_t e = prepared ? cudaSuccess : launch_prep(c, dev_params, s);
    if (e != cudaSuccess) return e;
    const bool use_ck = c->fused && ck && ck->count > 0;
    if (!seeded) {
        // the final state: psi, or the last checkpoint
        tqd_state fin = *psi;
        if (use_ck) fin.amps = ck->at(ck->count - 1);
        e = launch_apply_observable(&fin, groups, dev_weights, scale, lam, s, dev_energy);
    }
    if (e != cudaSuccess) return e;
    if (c->fused) {
        const int np = pass_end < 0 ? (int)c->tile_passes.size() : pass_end;
        const int first = use_ck ? np - ck->count : np;
        for (int p = np - 1; p >= pass_begin; --p) {
            const TilePlanPass &pp = c->tile_passes[p];
            if (psi->dtype == TQD_C64 && tc_reverse_pass(pp)) {
                // no derivative to take: lambda <- U^dagger lambda on the tensor
                // cores, and psi too unless it is read from a checkpoint
                const TcBlock &b = *(const TcBlock *)c->tc_blocks[pp.tc];
                e = p >= first ? launch_tc_block(lam, c, b, s, true) : launch_tc_block(psi, c, b, s, true, lam);
            } else {
                e = p >= first ? launch_tile_pass(psi, lam, c, p, s, ck->at(p - first))
                               : launch_tile_pass(psi, lam, c, p, s);
            }
            if (e != cudaSuccess) return e;
        }
        return launch_grad_finalize(c, tile_grid(c, psi->dtype == TQD_C64 ? 0 : 1, true), dev_grads, s);
    }
    const int nblk = plain_adjoint_blocks(c->n);
    for (int g = (int)c->gates.size() - 1; g >= 0; --g) {
        const int slot = c->grad_slot[g];
        double *part = slot >= 0 ? c->d_partials + (size_t)slot * c->pblk : nullptr;
        e = launch_plain_adjoint_gate(psi, lam, c, g, part, c->pblk, s);
        if (e != cudaSuccess) return e;
    }
    return launch_grad_finalize(c, nblk, dev_grads, s);
}

std::vector<tqd_pauli_term> conjugate_by_tail(const tqd_circuit *c, const tqd_pauli_term *terms, size_t n_terms) {
    std::vector<tqd_pauli_term> out(terms, terms + n_terms);
    const int L = (int)c->gates.size();
    for (auto &t : out) {
        uint64_t x = t.xmask, z = t.zmask;
        double coeff = t.coeff;
        // P^dagger Q P with P = G_L ... G_tail: conjugate by the last gate first
        for (int g = L - 1; g >= c->tail_gate; --g) {
            const GateH &h = c->gates[g];
            const int y0 = __builtin_popcountll(x & z);
            if (h.kind == TQD_CNOT) {
                // X_c -> X_c X_t, Z_t -> Z_c Z_t
                const uint64_t cb = 1ull << h.w[0], tb = 1ull << h.w[1];
                if (x & cb) x ^= tb;
                if (z & tb) z ^= cb;
            } else if (h.kind == TQD_SWAP) {
                const uint64_t pb = 1ull << h.w[0], qb = 1ull << h.w[1];
                auto sw = [&](uint64_t v) {
                    const bool a = v & pb, b = v & qb;
                    v &= ~(pb | qb);
                    return v | (a ? qb : 0) | (b ? pb : 0);
                };
                x = sw(x);
                z = sw(z);
            } else {  // X_q: X_q Z^z X_q = (-1)^{z_q} Z^z
                if ((z >> h.w[0]) & 1) coeff = -coeff;
            }
            // X^x Z^z keeps its order under these maps; the term's phase
            // i^{|x & z|} becomes i^{|x' & z'|} times i^{d}, d even
            const int d = (y0 - __builtin_popcountll(x & z)) & 3;
            if (d == 2) coeff = -coeff;
        }
        t.xmask = x;
        t.zmask = z;
        t.coeff = coeff;
    }
    return out;
}

}  // namespace tqd
