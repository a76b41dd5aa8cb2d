// ih_plan.h -- tile-grid choice for one build.
//
// Larger tiles mean fewer carry bytes (the carries are about 1/R + 1/Wc of
// the output); smaller tiles mean more independent warps.  The default rule
// takes the largest tile that still gives every SM `kWarpsPerSm` warps of
// count-tile work.  A tuned choice (ih_tune) overrides it for a shape.
#pragma once

#include "ih_internal.cuh"

namespace ih {

// groups: warps of count-tile work per tile (the number of bin groups).
TileGrid choose_grid(int H, int W, int groups, int nsm);

// Tile grid with explicit band rows and strip width (clamped to the frame).
TileGrid make_grid(int H, int W, int R, int Wc);

// The grids of the n plane sets of one batch: when the batch fills the GPU
// even with the largest tiles, every frame takes them (else the sets keep
// their grids).  Call before the carries are sized.
void batch_grids(PlaneSet *sets, int n, int nsm);

}  // namespace ih
