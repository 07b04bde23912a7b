// Plan-building entry points shared between the host translation units.
#pragma once

#include <functional>
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

// panel_nv: vectors per pass of an x-panel plan (1, 2, or 4 when m <= 2^16)
ffspmv_status build_plan_ex(Plan &P, long long nrows, long long ncols,
                            const long long *ptr, const int *col, const u32 *val,
                            u32 m, const ffspmv_options &opt, const BinChoice *bins,
                            int panel_nv = 1);

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

// Host half of the x-panel layout (panel.cu): geometry, stage descriptors,
// entry words and values (u32 here; stored as u16 when m <= 2^16).
struct PanelHost {
    bool small = true;
    bool tiny = false;  // m <= 256, one vector per pass: u8 x and values
    bool mont = false;  // odd 2^16 < m < 2^31: values stored as v 2^32 mod m (Montgomery form)
    int nv = 1;
    int q = 1, ngroup = 0, rows_max = 0, resident = 0, px = 0, pe = 0, eb = 0;
    size_t smem = 0;
    long long pcols = 0, nstage = 0, npm = 0, npad = 0;
    std::vector<u32> grp_row0, stage_ptr;
    std::vector<PanelStage> stage;
    std::vector<u32> ent, val;
};

// Rows longer than kPanelLong are left out (the caller adds split CSR
// segments for them).  pm_on: +-1 entries (cls != 0) go to value-free
// sections.  force_q: 1, 2 or 4 forces the cluster size, else the builder
// picks it; nv: vectors per pass (1, 2, or 4 when m <= 2^16), x and the row
// sums interleaved by vector; max_clusters(q, small) gives the clusters of q
// CTAs resident at once.  False when the matrix has nothing to stage or exceeds the layout's
// limits.
bool panel_layout(long long n, long long nc, const long long *ptr, const u32 *col, const u32 *val,
                  const unsigned char *cls, u32 m, bool pm_on, int force_q, int nv,
                  const std::function<int(int, bool)> &max_clusters, PanelHost &H);

void transpose_csr(long long nrows, long long ncols, const long long *ptr,
                   const int *col, const u32 *val, std::vector<long long> &tptr,
                   std::vector<int> &tcol, std::vector<u32> &tval);

}  // namespace ff
