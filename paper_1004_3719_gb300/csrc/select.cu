// Format selection per row bin.
#include "ff_select.h"

namespace ff {

ffspmv_status choose_bins(int selector, long long nrows, long long ncols,
                          const long long *ptr, const int *col, const u32 *val,
                          u32 m, const ffspmv_options &o, BinChoice *bins)
{
    (void)selector; (void)ncols; (void)col;
    std::vector<long long> nnzb(kBins, 0), pmb(kBins, 0);
    for (long long i = 0; i < nrows; ++i) {
        int b = bin_of_length(ptr[i + 1] - ptr[i]);
        for (long long k = ptr[i]; k < ptr[i + 1]; ++k) {
            u32 v = val[k] % m;
            pmb[b] += (v == 1u) || (m > 2u && v == m - 1u);
        }
        nnzb[b] += ptr[i + 1] - ptr[i];
    }
    for (int b = 0; b < kBins; ++b)
        bins[b] = heuristic_bin_choice(b, nnzb[b] ? (double)pmb[b] / nnzb[b] : 0.0, o.use_pm1);
    return FFSPMV_OK;
}

}  // namespace ff
