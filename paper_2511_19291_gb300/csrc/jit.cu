// jit.cu -- generation, run-time compilation (NVRTC) and launch of the
// pass-specialised tile kernels.
//
// NVRTC is loaded with dlopen, so the library also loads where it is absent
// (the default mode then keeps the generic kernel).  Compiled modules are
// cached per device by source text: passes of the same shape (an ansatz
// repeats its layers) share one kernel, whatever their angles, which stay in
// the matrix buffer.
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

#include "jit.h"
#include "tc.h"
#include "plan.h"
#include "prof.h"
#include "tile.h"
#include "tile_plan.h"

#include "tqd_jit_headers.inc"  // k_jit_header_names / k_jit_header_srcs / k_jit_n_headers

namespace tqd {

// --------------------------------------------------------------- loading
namespace {

struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcVersion) version = nullptr;
    bool ok = false;
};

const Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        n.create = (decltype(n.create))dlsym(h, "nvrtcCreateProgram");
        n.compile = (decltype(n.compile))dlsym(h, "nvrtcCompileProgram");
        n.log_size = (decltype(n.log_size))dlsym(h, "nvrtcGetProgramLogSize");
        n.log = (decltype(n.log))dlsym(h, "nvrtcGetProgramLog");
        n.cubin_size = (decltype(n.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
        n.cubin = (decltype(n.cubin))dlsym(h, "nvrtcGetCUBIN");
        n.destroy = (decltype(n.destroy))dlsym(h, "nvrtcDestroyProgram");
        n.version = (decltype(n.version))dlsym(h, "nvrtcVersion");
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    });
    return n;
}

typedef CUresult (*FnModuleLoadData)(CUmodule *, const void *);
typedef CUresult (*FnModuleGetFunction)(CUfunction *, CUmodule, const char *);
typedef CUresult (*FnFuncSetAttribute)(CUfunction, CUfunction_attribute, int);
typedef CUresult (*FnFuncGetAttribute)(int *, CUfunction_attribute, CUfunction);
typedef CUresult (*FnLaunchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                                   CUstream, void **, void **);

struct Driver {
    FnModuleLoadData load = nullptr;
    FnModuleGetFunction get = nullptr;
    FnFuncSetAttribute attr = nullptr;
    FnFuncGetAttribute get_attr = nullptr;
    FnLaunchKernel launch = nullptr;
    bool ok = false;
};

void *driver_sym(const char *name, int version) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return p;
}

const Driver &driver() {
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        d.load = (FnModuleLoadData)driver_sym("cuModuleLoadData", 12000);
        d.get = (FnModuleGetFunction)driver_sym("cuModuleGetFunction", 12000);
        d.attr = (FnFuncSetAttribute)driver_sym("cuFuncSetAttribute", 12000);
        d.get_attr = (FnFuncGetAttribute)driver_sym("cuFuncGetAttribute", 12000);
        d.launch = (FnLaunchKernel)driver_sym("cuLaunchKernel", 12000);
        d.ok = d.load && d.get && d.attr && d.get_attr && d.launch;
    });
    return d;
}

// ------------------------------------------------------------ generation
void put(std::string &o, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    o += buf;
}

const char *tf(bool b) { return b ? "true" : "false"; }

// Registers per thread a TMA-warpgroup ring kernel launches with.
int tmaw_launch_regs(bool adj) { return adj ? RingCfg<true>::REGS_LAUNCH : RingCfg<false>::REGS_LAUNCH; }

// Whether a diagonal run has gates on thread bits (a per-thread factor).
bool dg_has_thread_subs(const TilePassDev &D, const TileOp &op) {
    for (int q = op.sub0; q < op.sub0 + op.nsub; ++q)
        if (D.subs[q].a & 0x80) return true;
    return false;
}

// The runner's init: every diagonal run's thread factor (the product of its
// gates on thread bits at this thread's bit values) into member f<run>.  It
// depends only on the thread and the pass, not on the tile.
void emit_init(std::string &o, const TilePassDev &D) {
    for (int k = 0; k < D.h.n_ops; ++k) {
        const TileOp &op = D.ops[k];
        if (op.type == TOP_DG && dg_has_thread_subs(D, op)) put(o, "TV f%d;\n", op.moff);
    }
    o += "__device__ __forceinline__ void init(const TileCtx<TV> &c) {\nconst uint32_t tid = c.tid;\n(void)tid;\n";
    for (int k = 0; k < D.h.n_ops; ++k) {
        const TileOp &op = D.ops[k];
        if (op.type != TOP_DG || !dg_has_thread_subs(D, op)) continue;
        put(o, "{\nTV f = mkc<TV>(1, 0);\n");
        for (int q = op.sub0; q < op.sub0 + op.nsub; ++q) {
            const TileSub &sb = D.subs[q];
            if (!(sb.a & 0x80)) continue;
            if (sb.type == TOP_D1)
                put(o, "f = cmul(f, pool_c<TV>(c.pool, %d + (tbit(tid, %d) ? 6 : 0)));\n", sb.moff, sb.a);
            else
                put(o, "if (tbit(tid, %d) & tbit(tid, %d)) f = cmul(f, pool_c<TV>(c.pool, %d));\n", sb.a, sb.b,
                    sb.moff);
        }
        put(o, "f%d = f;\n}\n", op.moff);
    }
    o += "}\n";
}

// One op applied forward (or inverted in the reverse sweep, where it acts on
// psi and lambda): the generic kernel's apply_op with every field constant.
void emit_apply(std::string &o, const TilePassDev &D, const TileOp &op, bool adj) {
    const char *dg = tf(adj), *two = tf(adj);
    const int ta = op.a & 0x80, tb = op.b & 0x80;
    switch (op.type) {
    case TOP_G1R:
        put(o, "op_g1r<TV, %s, %s, %d>(a, b, c.pool + %d);\n", dg, two, op.a, op.moff);
        break;
    case TOP_G1:
        put(o, "op_g1<TV, %s, %s, %d>(a, b, c.pool + %d);\n", dg, two, op.a, op.moff);
        break;
    case TOP_D1:
        if (ta) put(o, "op_d1t<TV, %s, %s>(a, b, c.pool + %d, tbit(tid, %d));\n", dg, two, op.moff, op.a);
        else put(o, "op_d1r<TV, %s, %s, %d>(a, b, c.pool + %d);\n", dg, two, op.a, op.moff);
        break;
    case TOP_CX:
        if (ta) put(o, "op_cxt<%s, %d>(a, b, tbit(tid, %d));\n", two, op.b, op.a);
        else put(o, "op_cxr<%s, %d, %d>(a, b);\n", two, op.a, op.b);
        break;
    case TOP_SW:
        put(o, "op_sw<%s, %d, %d>(a, b);\n", two, op.a, op.b);
        break;
    case TOP_G2:
        put(o, "op_g2<TV, %s, %s, %d, %d>(a, b, c.pool + %d);\n", dg, two, op.a, op.b, op.moff);
        break;
    case TOP_D2:
        if (ta && tb)
            put(o, "op_d2tt<TV, %s, %s>(a, b, c.pool + %d, tbit(tid, %d) & tbit(tid, %d));\n", dg, two, op.moff, op.a,
                op.b);
        else if (ta)
            put(o, "op_d2tr<TV, %s, %s, %d>(a, b, c.pool + %d, tbit(tid, %d));\n", dg, two, op.b, op.moff, op.a);
        else if (tb)
            put(o, "op_d2tr<TV, %s, %s, %d>(a, b, c.pool + %d, tbit(tid, %d));\n", dg, two, op.a, op.moff, op.b);
        else
            put(o, "op_d2rr<TV, %s, %s, %d, %d>(a, b, c.pool + %d);\n", dg, two, op.a, op.b, op.moff);
        break;
    case TOP_DG:
        if (op.b) {
            // gates on tile bits: at this tile, those on tile bits only or on
            // a tile bit and a thread bit multiply the thread factor, those on
            // a tile bit and register position r a phase e<r> on r
            bool reg_used[TILE_R] = {false};
            for (int q = op.sub0; q < op.sub0 + op.nsub; ++q) {
                const TileSub &sb = D.subs[q];
                if ((sb.a & 0xC0) == TILE_POS_TILE && sb.type == TOP_D2 && !(sb.b & 0xC0)) reg_used[sb.b] = true;
            }
            o += "{\n";
            if (dg_has_thread_subs(D, op)) put(o, "TV tf = f%d;\n", op.moff);
            else o += "TV tf = mkc<TV>(1, 0);\n";
            for (int r = 0; r < TILE_R; ++r)
                if (reg_used[r]) put(o, "TV e%d = mkc<TV>(1, 0);\n", r);
            for (int q = op.sub0; q < op.sub0 + op.nsub; ++q) {
                const TileSub &sb = D.subs[q];
                if ((sb.a & 0xC0) != TILE_POS_TILE) continue;
                if (sb.type == TOP_D1)
                    put(o, "tf = cmul(tf, pool_c<TV>(c.pool, %d + (tile_bit(c.torig, %d) ? 6 : 0)));\n", sb.moff,
                        sb.a);
                else if ((sb.b & 0xC0) == TILE_POS_TILE)
                    put(o, "if (tile_bit(c.torig, %d) & tile_bit(c.torig, %d)) tf = cmul(tf, pool_c<TV>(c.pool, %d));\n",
                        sb.a, sb.b, sb.moff);
                else if (sb.b & 0x80)
                    put(o, "if (tile_bit(c.torig, %d) & tbit(tid, %d)) tf = cmul(tf, pool_c<TV>(c.pool, %d));\n",
                        sb.a, sb.b, sb.moff);
                else
                    put(o, "if (tile_bit(c.torig, %d)) e%d = cmul(e%d, pool_c<TV>(c.pool, %d));\n", sb.a, sb.b, sb.b,
                        sb.moff);
            }
            put(o, "op_dg<TV, %s, %s, true>(a, b, c.dgt + %d * NR, tf);\n", dg, two, op.moff);
            for (int r = 0; r < TILE_R; ++r)
                if (reg_used[r]) put(o, "op_ph<TV, %s, %s, %d>(a, b, e%d);\n", dg, two, r, r);
            o += "}\n";
            break;
        }
        // the table, times the run's thread factor (computed once per block by init)
        if (dg_has_thread_subs(D, op)) put(o, "op_dg<TV, %s, %s, true>(a, b, c.dgt + %d * NR, f%d);\n", dg, two, op.moff, op.moff);
        else put(o, "op_dg<TV, %s, %s, false>(a, b, c.dgt + %d * NR, mkc<TV>(1, 0));\n", dg, two, op.moff);
        break;
    default:
        break;
    }
}

// Gradient values of a tile in the order the reverse sweep meets them: value
// i goes to the warp reduction as number i % 32 of its chunk (gpush), whose
// warp totals are written to slots top - lane (top = n_grad - 1 - the values
// of earlier chunks).  The encoder numbers a pass's gradient ops in forward
// order, so the reverse order is slot n_grad - 1 - i; a pass that breaks
// that order gets a source that does not compile.
struct GradEmit {
    int n_grad = 0;
    int idx = 0;
};

void emit_push(std::string &o, GradEmit &ge, int slot, const char *expr) {
    const int top = ge.n_grad - 1 - (ge.idx & ~31);
    if (slot != ge.n_grad - 1 - ge.idx) put(o, "#error \"gradient slot %d out of order\"\n", slot);
    put(o, "gpush<%d, TV>(ga, %s, c, %d);\n", ge.idx & 31, expr, top);
    ++ge.idx;
}

// Reverse sweep: the op's angle derivatives from (psi, lambda) after it.
void emit_grad(std::string &o, const TilePassDev &D, const TileOp &op, GradEmit &ge) {
    if (op.type == TOP_DG) {
        bool need = false;
        for (int q = op.sub0; q < op.sub0 + op.nsub; ++q) need |= D.subs[q].gslot >= 0;
        if (!need) return;
        // Every derivative of the run is a signed sum of w: from the total wt
        // and the per-register-bit sums ws[r] each costs at most one fma.
        o += "{\nTT w[NR];\nfor (int j = 0; j < NR; ++j) w[j] = im_cdot(b[j], a[j]);\n"
             "TT wt, ws[TILE_R];\ndiag_sums<TT>(w, wt, ws);\n";
        // a thread or tile bit's value as an expression; "" for a register position
        auto bit = [](uint8_t p, char *buf, size_t len) {
            if (p & 0x80) snprintf(buf, len, "((tid >> %d) & 1u)", p & 0x7f);
            else if ((p & 0xC0) == TILE_POS_TILE) snprintf(buf, len, "tile_bit(c.torig, %d)", p);
            else buf[0] = 0;
        };
        // descending: the pass's values arrive in descending slot order
        for (int q = op.sub0 + op.nsub - 1; q >= op.sub0; --q) {
            const TileSub &sb = D.subs[q];
            if (sb.gslot < 0) continue;
            char ta[48], tb[48], e[200];
            bit(sb.a, ta, sizeof ta);
            if (sb.type == TOP_D1 && (sb.gen == GEN_Z || sb.gen == GEN_P1)) {
                const bool z = sb.gen == GEN_Z;
                if (ta[0]) snprintf(e, sizeof e, z ? "(%s ? -wt : wt)" : "(%s ? TT(-2) * wt : TT(0))", ta);
                else snprintf(e, sizeof e, z ? "fma(TT(-2), ws[%d], wt)" : "TT(-2) * ws[%d]", sb.a);
            } else if (sb.type == TOP_D2) {
                bit(sb.b, tb, sizeof tb);
                if (ta[0] && tb[0]) snprintf(e, sizeof e, "((%s & %s) ? TT(-2) * wt : TT(0))", ta, tb);
                else if (ta[0] || tb[0])
                    snprintf(e, sizeof e, "(%s ? TT(-2) * ws[%d] : TT(0))", ta[0] ? ta : tb, ta[0] ? sb.b : sb.a);
                else snprintf(e, sizeof e, "grad_diag<TV>(%d, %d, %d, %d, w, tid, c.torig)", sb.type, sb.a, sb.b, sb.gen);
            } else {
                snprintf(e, sizeof e, "grad_diag<TV>(%d, %d, %d, %d, w, tid, c.torig)", sb.type, sb.a, sb.b, sb.gen);
            }
            emit_push(o, ge, sb.gslot, e);
        }
        o += "}\n";
        return;
    }
    if (op.gslot < 0) return;
    char e[160];
    if (op.type == TOP_G1 || op.type == TOP_G1R)
        snprintf(e, sizeof e, "grad_g1<%d, TV>(%d, a, b)", op.a, op.gen);
    else
        snprintf(e, sizeof e, "grad_diag_op<TV>(%d, %d, %d, %d, a, b, tid)", op.type, op.a, op.b, op.gen);
    emit_push(o, ge, op.gslot, e);
}

// The 16 shared-memory accesses of a stage: register j of the thread sits at
// tile index base ^ roff[j], base = lo[lane] ^ hi[warp].  Every bit base can
// have lies in TB (the union of the lo and hi entries), so with u = roff[j] & TB
// the index is (base ^ u) + (roff[j] & ~TB): the sum of a per-thread value and
// a constant with disjoint bits.  Each distinct u gets one XOR; the constant
// becomes the access's immediate offset.
//
// complex64: when every lane and warp entry is even and registers j and j ^ 1
// sit at offsets r and r ^ 1 with r even (local bit 0 is register bit 0 and
// the map keeps it), the pair is one 16-byte access (tile_ld2 / tile_st2).
void emit_access(std::string &o, const char *fn, const char *base, const uint16_t *lo, const uint16_t *hi,
                 const uint16_t *roff, int dt) {
    uint32_t tb = 0;
    for (int l = 0; l < 32; ++l) tb |= lo[l];
    for (int w = 0; w < TILE_THREADS / 32; ++w) tb |= hi[w];
    bool pair = dt == 0 && !(tb & 1u);
    for (int j = 0; j < (1 << TILE_R) && pair; j += 2)
        pair = !(roff[j] & 1u) && roff[j + 1] == (roff[j] ^ 1u);
    std::vector<uint32_t> us;
    int idx[1 << TILE_R];
    for (int j = 0; j < (1 << TILE_R); ++j) {
        const uint32_t u = roff[j] & tb;
        int k = 0;
        while (k < (int)us.size() && us[k] != u) ++k;
        if (k == (int)us.size()) {
            us.push_back(u);
            put(o, "const uint32_t %s%d = %s ^ %uu;\n", base, k, base, u);
        }
        idx[j] = k;
    }
    if (pair) {
        for (int j = 0; j < (1 << TILE_R); j += 2)
            put(o, "%s2<TV, KADJ>(c, a, b, %d, %d, %s%d + %uu);\n", fn, j, j + 1, base, idx[j],
                (unsigned)(roff[j] & ~tb));
        return;
    }
    for (int j = 0; j < (1 << TILE_R); ++j)
        put(o, "%s<TV, KADJ>(c, a, b, %d, %s%d + %uu);\n", fn, j, base, idx[j], (unsigned)(roff[j] & ~tb));
}

std::string generate(const TilePassDev &D, int dt, bool adj, bool ring, bool tmaw, bool psi_ro) {
    const TileHead &h = D.h;
    std::string o;
    o.reserve(1 << 16);
    o += "#include \"tile_dev.cuh\"\nnamespace tqd {\n";
    put(o, "typedef %s TV;\ntypedef %s TT;\nconstexpr bool KADJ = %s;\n", dt == 0 ? "float2" : "double2",
        dt == 0 ? "float" : "double", tf(adj));
    o += "struct PassRunner {\nGradAcc<TT> ga;\n";
    emit_init(o, D);
    GradEmit ge;
    ge.n_grad = h.n_grad;
    o += "__device__ __forceinline__ void run(const TileCtx<TV> &c) {\n"
         "int *err = c.err;\n(void)err;\nconst uint32_t tid = c.tid;\n(void)tid;\nTV a[NR];\nTV b[NR];\n";
    for (int si = 0; si < h.n_stages; ++si) {
        const int s = adj ? h.n_stages - 1 - si : si;
        const TileStage &st = D.stages[s];
        put(o, "{\nconst uint16_t *tl = c.tbt + %d * TILE_TB;\n", s);
        o += "const uint32_t bl = stage_base_ld<KADJ>(tl, c.lane, c.warp);\n";
        // the reverse sweep loads through the store map and stores through the load map
        const uint16_t *rl = adj ? st.st_roff : st.ld_roff;
        const uint16_t *rs = adj ? st.ld_roff : st.st_roff;
        emit_access(o, "tile_ld", "bl", adj ? st.st_lo : st.ld_lo, adj ? st.st_hi : st.ld_hi, rl, dt);
        if (!adj) {
            for (int k = st.op_begin; k < st.op_end; ++k) emit_apply(o, D, D.ops[k], false);
        } else {
            for (int k = (int)st.op_end - 1; k >= (int)st.op_begin; --k) {
                emit_grad(o, D, D.ops[k], ge);
                emit_apply(o, D, D.ops[k], true);
            }
        }
        if (st.sync_mid == SYNC_GROUP) o += "tile_sync(c);\n";
        else if (st.sync_mid == SYNC_WARP) o += "__syncwarp();\n";
        o += "const uint32_t bs = stage_base_st<KADJ>(tl, c.lane, c.warp);\n";
        // psi read-only: its last stage leaves psi in registers (what it would
        // store is never read), so the compiler drops its dead un-applications
        const char *stfn = (adj && psi_ro && si == h.n_stages - 1) ? "tile_stl" : "tile_st";
        emit_access(o, stfn, "bs", adj ? st.ld_lo : st.st_lo, adj ? st.ld_hi : st.st_hi, rs, dt);
        // the ring with a TMA warpgroup: after the last stage each thread
        // signals the tile's end itself (no barrier)
        if (si == h.n_stages - 1) o += "fence_async_smem();\n";
        if (si < h.n_stages - 1) {
            // between stages s and s + 1 of either direction: sync_end[s]
            const uint16_t lvl = D.stages[adj ? s - 1 : s].sync_end;
            if (lvl == SYNC_GROUP) o += "tile_sync(c);\n";
            else if (lvl == SYNC_WARP) o += "__syncwarp();\n";
        } else if (!(ring && tmaw)) {
            o += "tile_sync(c);\n";
        }
        o += "}\n";
    }
    o += "}\n";
    // end of a tile: the last chunk of gradient values (after the tile has
    // been handed on)
    if (adj && ge.n_grad > 0 && (ge.idx & 31) != 0)
        put(o, "__device__ __forceinline__ void finish(const TileCtx<TV> &c) { gflush<%d, TV>(ga, c, %d); }\n",
            ge.idx & 31, ge.n_grad - 1 - (ge.idx & ~31));
    else
        o += "__device__ __forceinline__ void finish(const TileCtx<TV> &) {}\n";
    if (adj && ge.idx != ge.n_grad) put(o, "#error \"%d gradient values for %d slots\"\n", ge.idx, ge.n_grad);
    o += "};\n}  // namespace tqd\n";
    // the generic kernels' launch bounds (tile_min_blocks<V, ADJ, 1>; ring: one block of G groups)
    const int minb = dt == 0 ? (adj ? 2 : 3) : 1;
    put(o,
        "extern \"C\" __global__ void __launch_bounds__(%d, %d)\n"
        "tqd_pass(const __grid_constant__ tqd::TmaDesc mp, const __grid_constant__ tqd::TmaDesc ml,\n"
        "         const tqd::TilePassDev *__restrict__ Pg, const tqd::TT *__restrict__ mats,\n"
        "         double *__restrict__ partials, int pblk, int *__restrict__ err, int flags) {\n",
        ring ? (adj ? (tmaw ? RingCfg<true>::THREADS_TMAW : RingCfg<true>::THREADS) : (tmaw ? RingCfg<false>::THREADS_TMAW : RingCfg<false>::THREADS)) : TILE_THREADS, ring ? 1 : minb);
    if (ring)
        put(o, "    tqd::tile_pass_ring<tqd::TV, tqd::KADJ, tqd::RingCfg<tqd::KADJ>::G, tqd::RingCfg<tqd::KADJ>::B, %s,\n"
               "                        tqd::PassRunner>(&mp, &ml, Pg, mats, partials, pblk, err, flags);\n}\n", tf(tmaw));
    else
        o += "    tqd::tile_pass_body<tqd::TV, tqd::KADJ, 1, tqd::PassRunner>(&mp, &ml, Pg, mats, partials, pblk, err, flags);\n}\n";
    return o;
}

// ----------------------------------------------------------- compilation
int device_arch(int dev) {
    int mj = 0, mn = 0;
    cudaDeviceGetAttribute(&mj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mn, cudaDevAttrComputeCapabilityMinor, dev);
    return mj * 10 + mn;
}

// Source -> cubin; empty with the log in *log on failure.  info: ptxas
// reports resources (registers, spills) and the log is returned in *log on
// success too.
std::string compile_cubin(const std::string &src, int arch, std::string *log, bool info = false) {
    const Nvrtc &N = nvrtc();
    nvrtcProgram prog;
    if (N.create(&prog, src.c_str(), "tqd_pass.cu", k_jit_n_headers, k_jit_header_srcs, k_jit_header_names) !=
        NVRTC_SUCCESS) {
        *log = "nvrtcCreateProgram failed";
        return std::string();
    }
    char archopt[64];
    snprintf(archopt, sizeof(archopt), "--gpu-architecture=sm_%da", arch);
    // TQD_JIT_VERBOSE=1: ptxas reports registers and spills into the log
    const bool verbose = getenv("TQD_JIT_VERBOSE") && getenv("TQD_JIT_VERBOSE")[0] == '1';
    const char *opts[] = {archopt, "-std=c++17", "-DNDEBUG", (verbose || info) ? "--ptxas-options=-v" : "-DTQD_QUIET",
#ifdef TQD_CHECKED
                          "-DTQD_CHECKED",
#endif
    };
    const nvrtcResult r = N.compile(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    std::string out;
    if (verbose) {
        size_t n = 0;
        N.log_size(prog, &n);
        std::string lg(n, '\0');
        if (n) N.log(prog, &lg[0]);
        fprintf(stderr, "[tqd jit] %s\n", lg.c_str());
    }
    if (r != NVRTC_SUCCESS || info) {
        size_t n = 0;
        N.log_size(prog, &n);
        log->assign(n, '\0');
        if (n) N.log(prog, &(*log)[0]);
    }
    if (r == NVRTC_SUCCESS) {
        size_t n = 0;
        N.cubin_size(prog, &n);
        out.assign(n, '\0');
        if (n) N.cubin(prog, &out[0]);
    }
    N.destroy(&prog);
    return out;
}

std::mutex g_cache_mu;
std::map<std::pair<int, std::string>, CUfunction> g_cache;  // (device, source) -> kernel

}  // namespace

bool jit_wanted(const tqd_circuit *c) {
    if (!c->fused || c->opts.jit == 1) return false;
    if (c->opts.jit == 2) return true;
    return c->n >= 22 && nvrtc().ok && driver().ok;
}

std::string jit_source(const tqd_circuit *c, int pass, int dt, bool adj, bool ring, bool tmaw, bool psi_ro) {
    return generate(c->tile_passes[pass].dev[dt], dt, adj, ring, tmaw, adj && psi_ro);
}

// ----------------------------------------------------------- disk cache
// Compiled kernels persist across processes in a cache directory
// (TQD_JIT_CACHE_DIR, else $XDG_CACHE_HOME/tqd-jit, else $HOME/.cache/tqd-jit;
// TQD_JIT_CACHE=0 turns it off).  An entry stores its whole key: the target,
// the compiler version, the build's options, the device headers the source
// includes and the generated source itself; it is used only when all of it
// matches byte for byte, so another library build or compiler never reuses
// a kernel.  Entries are written to a temporary file and renamed into place;
// anything unreadable, mismatched or unwritable is simply compiled again.
namespace {

uint64_t fnv1a(const char *p, size_t n, uint64_t h = 1469598103934665603ull) {
    for (size_t i = 0; i < n; ++i) h = (h ^ (unsigned char)p[i]) * 1099511628211ull;
    return h;
}

const std::string &cache_dir() {
    static std::string dir;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *off = getenv("TQD_JIT_CACHE");
        if (off && off[0] == '0') return;
        if (const char *d = getenv("TQD_JIT_CACHE_DIR")) dir = d;
        else if (const char *x = getenv("XDG_CACHE_HOME")) dir = std::string(x) + "/tqd-jit";
        else if (const char *h = getenv("HOME")) dir = std::string(h) + "/.cache/tqd-jit";
        if (dir.empty()) return;
        // create every missing component
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
        struct stat st;
        if (stat(dir.c_str(), &st) != 0 || !S_ISDIR(st.st_mode)) dir.clear();
    });
    return dir;
}

// Everything besides the source that decides what the compiler produces.
const std::string &cache_key_prefix() {
    static std::string prefix;
    static std::once_flag once;
    std::call_once(once, [] {
        int mj = 0, mn = 0;
        if (nvrtc().version) nvrtc().version(&mj, &mn);
        std::ostringstream o;
        o << "tqd-jit 1\nnvrtc " << mj << "." << mn << "\n";
#ifdef TQD_CHECKED
        o << "checked\n";
#endif
        for (int i = 0; i < k_jit_n_headers; ++i)
            o << k_jit_header_names[i] << " " << std::hex
              << fnv1a(k_jit_header_srcs[i], strlen(k_jit_header_srcs[i])) << std::dec << "\n";
        prefix = o.str();
    });
    return prefix;
}

bool read_u64(std::istream &in, uint64_t &v) { return (bool)in.read(reinterpret_cast<char *>(&v), sizeof(v)); }

bool cache_load(const std::string &path, const std::string &key, std::string *cubin) {
    std::ifstream in(path, std::ios::binary);
    uint64_t klen = 0, clen = 0;
    if (!in || !read_u64(in, klen) || klen != key.size()) return false;
    std::string k(klen, '\0');
    if (!in.read(&k[0], (std::streamsize)klen) || k != key) return false;
    if (!read_u64(in, clen) || clen == 0 || clen > (1u << 26)) return false;
    cubin->assign(clen, '\0');
    return (bool)in.read(&(*cubin)[0], (std::streamsize)clen);
}

void cache_store(const std::string &path, const std::string &key, const std::string &cubin) {
    std::ostringstream tmpname;
    tmpname << path << ".tmp." << getpid() << "." << std::hash<std::thread::id>()(std::this_thread::get_id());
    const std::string tmp = tmpname.str();
    {
        std::ofstream out(tmp, std::ios::binary | std::ios::trunc);
        const uint64_t klen = key.size(), clen = cubin.size();
        out.write(reinterpret_cast<const char *>(&klen), sizeof(klen));
        out.write(key.data(), (std::streamsize)klen);
        out.write(reinterpret_cast<const char *>(&clen), sizeof(clen));
        out.write(cubin.data(), (std::streamsize)clen);
        if (!out) {
            out.close();
            unlink(tmp.c_str());
            return;
        }
    }
    if (rename(tmp.c_str(), path.c_str()) != 0) unlink(tmp.c_str());
}

// compile_cubin through the disk cache.
std::string compile_cached(const std::string &src, int arch, std::string *log) {
    const std::string &dir = cache_dir();
    if (dir.empty()) return compile_cubin(src, arch, log);
    std::string key = cache_key_prefix();
    key += "sm_" + std::to_string(arch) + "a\n";
    key += src;
    char name[40];
    snprintf(name, sizeof(name), "/%016llx.cubin", (unsigned long long)fnv1a(key.data(), key.size()));
    const std::string path = dir + name;
    std::string cubin;
    if (cache_load(path, key, &cubin)) return cubin;
    cubin = compile_cubin(src, arch, log);
    if (!cubin.empty()) cache_store(path, key, cubin);
    return cubin;
}

}  // namespace

static cudaError_t prepare(const tqd_circuit *c, int dt, bool adj, bool ring, bool tmaw, bool psi_ro) {
    if (!nvrtc().ok || !driver().ok) {
        set_error("specialised pass kernels: NVRTC or the CUDA driver entry points are unavailable");
        return cudaErrorNotSupported;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaFree(nullptr);  // the device's primary context is current from here on
    const int np = (int)c->tile_passes.size();
    std::vector<std::string> srcs(np);
    std::vector<int> need;  // passes whose source is not cached yet (first of each shape)
    std::unordered_map<std::string, int> first;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        for (int p = 0; p < np; ++p) {
            // forward (and, for fixed gates, reverse) runs on the tensor cores
            if (dt == 0 && (adj ? tc_reverse_pass(c->tile_passes[p]) : c->tile_passes[p].tc >= 0)) continue;
            srcs[p] = jit_source(c, p, dt, adj, ring, tmaw, psi_ro);
            if (g_cache.count({dev, srcs[p]}) || first.count(srcs[p])) continue;
            first[srcs[p]] = p;
            need.push_back(p);
        }
    }
    // compile the new shapes in parallel
    const int arch = device_arch(dev);
    std::vector<std::string> cubins(need.size()), logs(need.size());
    {
        const int nt = std::max(1, std::min<int>((int)need.size(), (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        std::atomic<int> next(0);
        for (int t = 0; t < nt; ++t)
            th.emplace_back([&] {
                for (int i; (i = next.fetch_add(1)) < (int)need.size();)
                    cubins[i] = compile_cached(srcs[need[i]], arch, &logs[i]);
            });
        for (auto &t : th) t.join();
    }
    const Driver &D = driver();
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (size_t i = 0; i < need.size(); ++i) {
        if (cubins[i].empty()) {
            set_error("specialised pass kernel failed to compile: %.400s", logs[i].c_str());
            return cudaErrorInvalidSource;
        }
        CUmodule mod;
        CUfunction f;
        CUresult r = D.load(&mod, cubins[i].data());
        if (r == CUDA_SUCCESS) r = D.get(&f, mod, "tqd_pass");
        if (r != CUDA_SUCCESS) {
            set_error("specialised pass kernel: module load failed (CUresult %d)", (int)r);
            return cudaErrorInvalidKernelImage;
        }
        // dynamic shared memory up to the opt-in limit less the static part
        int optin = 0, stat = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        r = D.get_attr(&stat, CU_FUNC_ATTRIBUTE_SHARED_SIZE_BYTES, f);
        if (r == CUDA_SUCCESS) r = D.attr(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, optin - stat);
        if (r != CUDA_SUCCESS) {
            set_error("specialised pass kernel: shared-memory attribute rejected (CUresult %d)", (int)r);
            return cudaErrorInvalidKernelImage;
        }
        g_cache[{dev, srcs[need[i]]}] = f;
    }
    const int kind = jit_kind(ring, tmaw, psi_ro);
    std::vector<void *> &tab = c->jit_fn[dt][adj ? 1 : 0][kind];
    tab.assign(np, nullptr);
    for (int p = 0; p < np; ++p)
        if (!srcs[p].empty()) tab[p] = (void *)g_cache.at({dev, srcs[p]});
    c->jit_ready[dt][adj ? 1 : 0][kind] = true;
    return cudaSuccess;
}

cudaError_t jit_function(const tqd_circuit *c, int pass, int dt, bool adj, bool ring, bool tmaw, bool psi_ro,
                         cudaStream_t s, CUfunction *out) {
    *out = nullptr;
    if (!jit_wanted(c)) return cudaSuccess;
    psi_ro = adj && psi_ro;
    std::lock_guard<std::mutex> lk(c->jit_mu);
    const int di = adj ? 1 : 0, kind = jit_kind(ring, tmaw, psi_ro);
    if (!c->jit_ready[dt][di][kind]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
            return cudaSuccess;  // no module loads inside a capture: generic kernel
        const cudaError_t e = prepare(c, dt, adj, ring, tmaw, psi_ro);
        if (e != cudaSuccess) return e;
    }
    const std::vector<void *> &tab = c->jit_fn[dt][di][kind];
    if (pass < (int)tab.size()) *out = (CUfunction)tab[pass];
    return cudaSuccess;
}

int jit_num_regs(CUfunction f) {
    int v = -1;
    if (!driver().ok || driver().get_attr(&v, CU_FUNC_ATTRIBUTE_NUM_REGS, f) != CUDA_SUCCESS) return -1;
    return v;
}

cudaError_t jit_launch(CUfunction f, const CUtensorMap &ma, const CUtensorMap &mb, const TilePassDev *desc,
                       const void *mats, double *partials, int pblk, int *err, int flags, int grid, int threads,
                       uint32_t smem, cudaStream_t s) {
    CUtensorMap a = ma, b = mb;
    const void *m = mats;
    void *args[] = {&a, &b, (void *)&desc, (void *)&m, (void *)&partials, (void *)&pblk, (void *)&err, (void *)&flags};
    const CUresult r = driver().launch(f, (unsigned)grid, 1, 1, (unsigned)threads, 1, 1, smem, (CUstream)s, args, nullptr);
    if (r == CUDA_SUCCESS) return cudaSuccess;
    // a launch the driver refused (nothing ran); the code names the reason
    set_error("specialised pass kernel launch refused (CUresult %d, grid %d, %u B shared memory)", (int)r, grid, smem);
    return cudaErrorInvalidKernelImage;
}

tqd_status jit_check_host(tqd_circuit *c, int arch, int *n_kernels) {
    *n_kernels = 0;
    if (!nvrtc().ok) {
        set_error("tqd_jit_check: NVRTC cannot be loaded");
        return TQD_ERR_UNSUPPORTED;
    }
    c->opts.mode = TQD_PLAN_FUSED;
    relabel_swaps(c->gates, c->n);
    assign_grad_slots(c);
    int prefix = 0;
    std::vector<TilePlanPass> passes = plan_fused(c, &prefix);
    for (auto &p : passes)
        if (!encode_tile_pass(c, p)) {
            set_error("tqd_jit_check: a pass could not be encoded");
            return TQD_ERR_INVALID_ARG;
        }
    std::vector<std::string> srcs;
    std::vector<int> launch_regs;  // registers the kernel must launch with (TMA warpgroup), else 0
    {
        std::unordered_map<std::string, int> seen;
        for (auto &p : passes)
            for (int dt = 0; dt < 2; ++dt)
                for (int adj = 0; adj < 2; ++adj)
                    for (int ring = 0; ring < (dt == 0 ? 3 : 1); ++ring)
                        for (int ro = 0; ro < (adj ? 2 : 1); ++ro) {
                            std::string src = generate(p.dev[dt], dt, adj != 0, ring != 0, ring == 2, ro != 0);
                            if (seen.emplace(src, 1).second) {
                                srcs.push_back(std::move(src));
                                launch_regs.push_back(ring == 2 ? tmaw_launch_regs(adj != 0) : 0);
                            }
                        }
    }
    // TQD_JIT_DUMP_DIR: write every distinct generated source there (pass_<i>.cu)
    if (const char *dir = getenv("TQD_JIT_DUMP_DIR")) {
        for (size_t i = 0; i < srcs.size(); ++i) {
            std::ofstream f(std::string(dir) + "/pass_" + std::to_string(i) + ".cu");
            f << srcs[i];
        }
    }
    std::vector<std::string> logs(srcs.size());
    std::vector<char> ok(srcs.size(), 0);
    const int nt = std::max(1, std::min<int>((int)srcs.size(), (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    std::atomic<int> next(0);
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&] {
            for (int i; (i = next.fetch_add(1)) < (int)srcs.size();)
                ok[i] = !compile_cubin(srcs[i], arch, &logs[i], true).empty();
        });
    for (auto &t : th) t.join();
    for (size_t i = 0; i < srcs.size(); ++i) {
        if (!ok[i]) {
            set_error("tqd_jit_check: kernel %zu of %zu failed to compile: %.400s", i, srcs.size(), logs[i].c_str());
            return TQD_ERR_CUDA;
        }
        // the register shares of a TMA-warpgroup kernel assume it launches
        // with exactly REGS_LAUNCH registers per thread
        const char *u = strstr(logs[i].c_str(), "Used ");
        const int regs = u ? atoi(u + 5) : -1;
        if (launch_regs[i] && regs != launch_regs[i]) {
            set_error("tqd_jit_check: TMA-warpgroup kernel %zu launches with %d registers per thread, not %d", i,
                      regs, launch_regs[i]);
            return TQD_ERR_CUDA;
        }
    }
    *n_kernels = (int)srcs.size();
    return TQD_OK;
}

void jit_release(tqd_circuit *c) {
    for (auto &d : c->jit_fn)
        for (auto &k : d)
            for (auto &v : k) v.clear();
}

}  // namespace tqd
