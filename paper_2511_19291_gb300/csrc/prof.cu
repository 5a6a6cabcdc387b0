// prof.cu -- per-launch CUDA-event timing: an event pair on the launching
// stream around every kernel, summed per kernel class with the launch's
// algorithmic bytes.  Off by default; tqd_profile_enable turns it on.
#include <mutex>
#include <string.h>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace tqd {

static const char *kNames[PK_NKINDS] = {
    "prep", "reset", "dense1", "diag1", "perm2", "phase11", "dense2", "small",
    "adj1", "adj_phase11", "adj_small", "expval", "expval_terms", "apply_obs", "reduce",
    "tile_fwd", "tile_adj", "diag_run", "pauli_tile", "batch", "tc_block", "shots",
};

struct Rec {
    int kind;
    double bytes;
    cudaEvent_t a, b;
};

static std::mutex g_mu;
static bool g_on = false;
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

bool prof_on() { return g_on; }

int prof_begin(int kind, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return -1;
    Rec r;
    r.kind = kind;
    r.bytes = 0;
    r.a = take_event();
    r.b = take_event();
    cudaEventRecord(r.a, s);
    g_recs.push_back(r);
    return (int)g_recs.size() - 1;
}

void prof_end(int slot, double bytes, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot < 0 || slot >= (int)g_recs.size()) return;
    g_recs[slot].bytes = bytes;
    cudaEventRecord(g_recs[slot].b, s);
}

static void recycle_locked() {
    for (auto &r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}

}  // namespace tqd

using namespace tqd;

extern "C" {

tqd_status tqd_profile_enable(int enable) {
    std::lock_guard<std::mutex> lk(g_mu);
    recycle_locked();
    g_on = enable != 0;
    return TQD_OK;
}

tqd_status tqd_profile_read(tqd_profile_entry *out, int capacity, int *n_out) {
    if (!n_out || (capacity > 0 && !out)) {
        set_error("tqd_profile_read: NULL output");
        return TQD_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    double ms[PK_NKINDS] = {0}, bytes[PK_NKINDS] = {0};
    long long cnt[PK_NKINDS] = {0};
    for (auto &r : g_recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) {
            set_error("tqd_profile_read: %s", cudaGetErrorString(e));
            return TQD_ERR_CUDA;
        }
        float t = 0;
        cudaEventElapsedTime(&t, r.a, r.b);
        ms[r.kind] += t;
        bytes[r.kind] += r.bytes;
        cnt[r.kind] += 1;
    }
    int n = 0;
    for (int k = 0; k < PK_NKINDS; ++k) {
        if (cnt[k] == 0) continue;
        if (n < capacity) {
            memset(&out[n], 0, sizeof(out[n]));
            strncpy(out[n].name, kNames[k], sizeof(out[n].name) - 1);
            out[n].launches = cnt[k];
            out[n].total_ms = ms[k];
            out[n].bytes = bytes[k];
        }
        ++n;
    }
    *n_out = n;
    recycle_locked();
    return TQD_OK;
}

}  // extern "C"
