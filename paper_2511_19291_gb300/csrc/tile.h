// tile.h -- fused tile passes: the host planner's view (internal).  The
// descriptors the kernels read are in tile_desc.h.
#pragma once

#include <stdint.h>

#include <vector>

#include "tile_desc.h"

namespace tqd {

// Host-side plan of one pass.
struct TileLayout {
    std::vector<int> qubit_of_local;  // local bit -> qubit (box bits ascending, then extras)
    std::vector<int> extra;           // Q qubits copied by separate TMA operations (complex128)
    std::vector<int> extra_dt[2];     // the same per precision: complex64's wider inner dimension
                                      // leaves fewer dimensions, so fewer (or no) separate copies
    std::vector<int> out;             // qubits outside Q, ascending
    int rank[2];                      // tensor-map rank for c64 / c128
    int dim_lo[2][TILE_MAX_DIMS];
    int dim_len[2][TILE_MAX_DIMS];
    int dim_in[2][TILE_MAX_DIMS];     // 1 = dimension inside the box
};

struct TilePlanPass {
    TileLayout layout;
    std::vector<int> gates;  // absorbed gates, circuit order
    std::vector<int> order;  // absorbed gates, execution order (stage schedule)
    TilePassDev dev[2];      // kernel descriptor for c64 / c128
    int tc = -1;             // index of the tensor-core block that replaces this pass's forward (c64), or -1
};

}  // namespace tqd
