// Format selection (exhaustive search, selector network) and the block
// sequence state, shared between host translation units.
#pragma once

#include "ff_plan.h"

namespace ff {

// Pick one format per row bin with `selector` (FFSPMV_SEL_LEARNED or
// FFSPMV_SEL_EXHAUSTIVE).  bins[kBins] receives the choice.  layout (may be
// null) receives the network's whole-plan layout (FFSPMV_LAYOUT_*), or -1
// when no network answered (no weights installed, or the exhaustive search);
// alt (may be null) the best layout of the other family (x-panel / binned)
// when the two are predicted within FFSPMV_SEL_VERIFY_MARGIN, else -1.
ffspmv_status choose_bins(int selector, long long nrows, long long ncols,
                          const long long *ptr, const int *col, const u32 *val,
                          u32 m, const ffspmv_options &o, BinChoice *bins,
                          int *layout = nullptr, int *alt = nullptr);

void free_sequence_state(ffspmv_handle *h);
void batch_forget(ffspmv_handle *h);
void free_gf2(ffspmv_handle *h);

}  // namespace ff
