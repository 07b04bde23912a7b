// Plan-building entry points shared between the host translation units.
#pragma once

#include <vector>

#include "ff_internal.cuh"

namespace ff {

// Row-length bins of the BINNED layout: bin 0 holds the empty rows, bin b >= 1
// the rows with 2^(b-2) < length <= 2^(b-1); the last bin also takes every
// longer row.
constexpr int kBins = 17;

struct BinChoice {
    int kind = SEG_CSR;  // SEG_CSR, SEG_CSRBLK, SEG_ELLR or SEG_COO
    int group = 1;       // lanes per row for SEG_CSR
    int pm = 0;          // segregate +-1 entries
};

int bin_of_length(long long L);
long long bin_upper(int b);
BinChoice heuristic_bin_choice(int b, double pm_fraction, int use_pm1);

ffspmv_status build_plan_ex(Plan &P, long long nrows, long long ncols,
                            const long long *ptr, const int *col, const u32 *val,
                            u32 m, const ffspmv_options &opt, const BinChoice *bins);

// Sub-plans over a subset of rows (the exhaustive search).
struct PlanSource;
PlanSource *make_source(long long nrows, long long ncols, const long long *ptr, const int *col,
                        const u32 *val, u32 m);
void free_source(PlanSource *s);
ffspmv_status build_rows_plan(Plan &P, const PlanSource &src, const std::vector<u32> &rows,
                              const BinChoice &c);

// The candidate formats of a bin (index f of ffspmv_select.h) and their validity.
constexpr int kFormats = 10;
BinChoice format_choice(int f, int pm);
bool format_valid(int f, int bin, long long maxlen);

void transpose_csr(long long nrows, long long ncols, const long long *ptr,
                   const int *col, const u32 *val, std::vector<long long> &tptr,
                   std::vector<int> &tcol, std::vector<u32> &tval);

}  // namespace ff
