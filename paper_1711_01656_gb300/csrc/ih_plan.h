// ih_plan.h -- tile-grid choice for one plane set.
//
// Larger tiles mean fewer carry bytes (the carries are about 1/R + 1/Wc of
// the output per pass); smaller tiles mean more independent warps.  The
// default rule takes the largest tile that still gives every SM at least
// `kWarpsPerSm` warps of work; an explicit override (set by the autotuner
// through ih_plan_override) replaces it for matching shapes.
#pragma once

#include "ih_internal.cuh"

namespace ih {

TileGrid choose_grid(int H, int W, int B, int kind, int nsm);

}  // namespace ih
