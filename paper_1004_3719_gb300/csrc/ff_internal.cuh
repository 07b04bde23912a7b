// Internal definitions shared by the CUDA translation units of libffspmv.
//
// Residue arithmetic (Sec. 2.2): sums of products are formed exactly in
// integer accumulators and reduced once per output.  The reduction is
// Barrett's (P. Barrett, "Implementing the Rivest Shamir and Adleman public
// key encryption algorithm on a standard digital signal processor", CRYPTO
// 1986) with the 64-bit reciprocal mu = floor(2^64 / m).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ffspmv.h"

namespace ff {

typedef unsigned long long u64;
typedef unsigned int u32;

// ---------------------------------------------------------------------------
// Modulus parameters.
struct Mod {
    u32 m;      // modulus, 2 <= m <= 2^32 - 1
    u32 c64;    // 2^64 mod m
    u64 mu;     // floor(2^64 / m)
    u32 alpha;  // < m
    u32 beta;   // < m
};

Mod make_mod(u32 m, u32 alpha, u32 beta);  // host

// x mod m for any 64-bit x.  With mu = floor(2^64/m), q = floor(x*mu/2^64)
// lies in {floor(x/m) - 1, floor(x/m)}, so one conditional subtraction ends
// in [0, m).
__device__ __forceinline__ u32 red64(u64 x, const Mod &M)
{
    u64 q = __umul64hi(x, M.mu);
    u64 r = x - q * (u64)M.m;
    if (r >= M.m) r -= M.m;
    return (u32)r;
}

__device__ __forceinline__ u32 addmod(u32 a, u32 b, u32 m)
{
    u64 s = (u64)a + b;
    return (u32)(s >= m ? s - m : s);
}

// y_new = alpha*r + beta*y_old (first writer of a row) or y_old + alpha*r
// (a later part adding into the same row).  r < m.
__device__ __forceinline__ u32 combine(u32 r, const u32 *yp, bool accum,
                                       const Mod &M)
{
    u32 a = (M.alpha == 1u) ? r : red64((u64)M.alpha * r, M);
    if (accum) return addmod(*yp, a, M.m);
    if (M.beta == 0u) return a;
    u32 b = (M.beta == 1u) ? *yp : red64((u64)M.beta * (*yp), M);
    return addmod(a, b, M.m);
}

// ---------------------------------------------------------------------------
// Accumulators.  AccSmall is one 64-bit word and is used when the plan has
// checked that no output sums more than floor((2^64-1)/B) terms, B the
// largest term (Sec. 2.2's M/m^2 bound with M = 2^64 - 1); AccWide carries
// into a third 32-bit word and never overflows for rows below 2^34 entries.
struct AccSmall {
    u64 v;
    __device__ __forceinline__ void zero() { v = 0; }
    __device__ __forceinline__ void mad(u32 a, u32 b) { v += (u64)a * b; }
    __device__ __forceinline__ void add(u32 a) { v += a; }
    // a 64-bit value congruent to the sum; group sums of these stay exact
    __device__ __forceinline__ u64 partial(const Mod &) const { return v; }
};

struct AccWide {
    u32 w0, w1, w2;
    __device__ __forceinline__ void zero() { w0 = w1 = w2 = 0; }
    __device__ __forceinline__ void mad(u32 a, u32 b)
    {
        asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
            "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+r"(w0), "+r"(w1), "+r"(w2)
            : "r"(a), "r"(b));
    }
    __device__ __forceinline__ void add(u32 a)
    {
        asm("add.cc.u32 %0, %0, %3;\n\t"
            "addc.cc.u32 %1, %1, 0;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+r"(w0), "+r"(w1), "+r"(w2)
            : "r"(a));
    }
    // (w2*2^64 + w1*2^32 + w0) mod m, a value below m
    __device__ __forceinline__ u64 partial(const Mod &M) const
    {
        u32 lo = red64(((u64)w1 << 32) | w0, M);
        u32 hi = red64((u64)w2 * M.c64, M);
        return addmod(lo, hi, M.m);
    }
};

// ---------------------------------------------------------------------------
// Plan segments.  A plan is a list of segments; each covers a set of rows
// (or of entries, for COO) in one storage format.  Segments of one phase own
// disjoint rows and run in one launch; phase 2 segments add into rows that a
// phase 1 segment has already written (the column split of Sec. 2.4.4, Hybridization).
enum SegKind : int {
    SEG_CSR = 0,     // `group` lanes per row
    SEG_CSRBLK = 1,  // one CTA per row
    SEG_ELLR = 2,    // one thread per row: DIA diagonals + ELL_R columns
    SEG_COO = 3,     // element-parallel segmented sums over sorted entries
    SEG_EMPTY = 4,   // rows with no entry: y <- beta*y
    SEG_CSRSPLIT = 5 // long rows cut into chunks, one CTA per chunk, exact atomic sums
};

constexpr int kThreads = 256;        // threads per CTA for every plan kernel
constexpr int kCooRuns = 8;          // 32-entry runs per warp chunk (COO)
constexpr u32 kClassShift = 30;      // +-1 class in the top two bits of col
constexpr u32 kColMask = (1u << kClassShift) - 1u;
constexpr u32 kPlus = 1u, kMinus = 2u;
constexpr int kMaxSeg = 24;
constexpr int kSplitChunk = 4096;   // entries per CTA of a split long row

struct SegDesc {
    int kind;
    int accum;       // 0: first writer (applies beta), 1: adds into y
    int group;       // CSR lanes per row (power of two, 1..32)
    int vbytes;      // bytes per stored value: 0 (all +-1), 2 or 4
    int pm;          // column words carry the +-1 class bits
    int ndiag;       // DIA diagonals (SEG_ELLR)
    int width;       // ELL_R columns (SEG_ELLR)
    int dvbytes;     // bytes per DIA value: 2 or 4
    long long nrows;     // rows in the segment (SEG_COO: rows spanned)
    long long nnz;       // entries in the segment
    long long row0;      // first row when `rows` is NULL
    long long ld;        // ELL_R / DIA leading dimension (>= nrows)
    long long block0;    // first CTA of this segment in its launch
    long long nblocks;
    const u32 *rows;     // local row -> matrix row, or NULL (row0 + local)
    const u32 *ptr;      // CSR: local offsets, nrows + 1
    const u32 *vptr;     // CSR with +-1 and values: value offsets, nrows + 1
    const u32 *col;      // column words
    const void *val;     // u16 or u32 values
    const u32 *rowid;    // COO: matrix row of each entry (sorted)
    const u32 *rownb;    // ELL_R: entries per row
    const int *doff;     // DIA offsets (column - row)
    const void *dval;    // DIA values [ndiag][ld]
    long long ncols;     // columns of the matrix (DIA bounds)
    const u32 *chunk_row;  // SEG_CSRSPLIT: local row of each chunk
    const u32 *chunk_beg;  // SEG_CSRSPLIT: first entry of each chunk (nchunks + 1)
};

struct PlanParams {
    int nseg;
    int acc_wide;
    long long total_blocks;
    SegDesc seg[kMaxSeg];
};

struct Phase {
    std::vector<SegDesc> segs;
    std::vector<u32> split_rows_host;  // rows summed through `carry` (COO, CSRSPLIT)
    const u32 *split_rows = nullptr;   // device copy
    long long nsplit = 0;
    bool has_atomic = false;           // one vector per launch (carry holds one)
};

// x-panel layout (FFSPMV_FMT_PANEL).  Rows are cut into `ngroup` row groups
// and columns into `q` column groups, both balanced by entries; CTA
// g * q + j (rank j of a cluster of q CTAs) sums the entries of row group g
// that fall in column group j.  It walks the panels (`px` bytes of staged x)
// of its column group that hold any of its entries, starting at a panel that
// depends on g so that the CTAs do not all read the same x at once.  A stage
// is at most `pe` entries of one panel; kPanelStages stages are in flight in
// shared memory, and kPanelStages x slots hold the panels they use (a panel
// is copied once, with its first stage).  One warp of the CTA issues the bulk
// copies of each stage once the buffer's previous stage is done with; the
// other warps wait for the copies and sum.
//
// Every CTA first converts its share of x into the staged copy (u16 or u32,
// contiguous) and meets the others at a grid barrier before the first panel
// is copied in; the launch is one CTA per SM, all resident.
//
// A stage is a list of lanes of eight entries each, in four sections:
// general packs, general singles, +-1 packs, +-1 singles.  A pack holds eight
// entries of one row: the lane sums them and the lanes of one warp that
// carry the same row add their sums together (a segmented warp sum) before
// one shared-memory atomic.  Single lanes add each of their eight terms.  The
// host orders the entries of every 32 lanes so that, slot by slot, the x
// words and the row sums a warp touches fall in distinct shared-memory banks
// as far as it can.  The +-1 sections carry no values (Sec. 2.4.2): bit 15
// of the entry word gives the sign.  In memory the eight entries of lane j
// of a 32-lane block of c lanes sit at 4j..4j+3 and 4c+4j..4c+4j+3 of the
// block (each 16-byte load of a warp reads 512 contiguous bytes); values
// (general lanes only) are lane by lane for u16, interleaved the same way
// for u32.  Entry word: (row in group << 16) | (sign << 15) | x element of
// the panel.  Row sums stay in shared memory (u32 sums of terms below 2m when
// m <= 2^16 -- at most kPanelLong of them, so below 2^32 -- u64 sums of terms
// below 2^32 otherwise); the q CTAs of a cluster add their partial sums
// through distributed shared memory.
constexpr int kPanelConsumers = 512;          // 16 warps sum entries
constexpr int kPanelStages = 3;
constexpr int kPanelThreads = kPanelConsumers + 32 * kPanelStages;  // + one copy warp per stage buffer
constexpr int kPanelPerThread = 8;            // entries a lane takes per step
constexpr int kPanelBarBytes = 128;           // full and empty mbarrier of each stage buffer
constexpr int kPanelDescBytes = 128;          // (entries, general, packs, x slot) of each buffer
constexpr u32 kPanelSlotMask = 7u;            // PanelStage::xs: x slot
constexpr u32 kPanelNewX = 8u;                // PanelStage::xs: the panel is copied in with this stage
static_assert(16 * kPanelStages + 8 <= kPanelBarBytes && kPanelStages <= 7,
              "full and empty mbarriers of the stage buffers, the epilogue's receive mbarrier, x slots");
constexpr unsigned kPanelSpin = 1u << 20;     // polls of an mbarrier before giving up
constexpr unsigned kPanelGridSpin = 1u << 20; // polls of the grid barrier before giving up
constexpr u32 kPanelIdxMask = 0x7fffu;        // x element of the panel
constexpr u32 kPanelNeg = 0x8000u;            // a -1 entry (+-1 sections)
constexpr long long kPanelLong = 32768;       // longer rows go to split CSR segments
constexpr int kPanelSmemMax = 227 * 1024;
constexpr int kPanelMaxPe = 32760;            // stage entries (fits the 16-bit pack counts)
static_assert(16 * kPanelStages + 4 <= kPanelDescBytes, "stage descriptors and the grid generation word");

struct PanelStage {
    u32 xoff;  // first staged-x element of the panel (16-byte aligned)
    u32 k0;    // first entry (a multiple of 8)
    u32 v0;    // first value (a multiple of 8): values of the general lanes only
    u32 nent;  // entries, a multiple of 8, at most pe
    u32 ngen;  // entries of the general sections (a multiple of 8), first in the stage
    u32 npg;   // entries of the general packs, first in the general sections
    u32 npp;   // entries of the +-1 packs, first in the +-1 sections
    u32 xs;    // x slot (kPanelSlotMask); kPanelNewX set: the panel is copied in with this stage
};

struct PanelPart {
    bool on = false;
    bool small = true;   // m <= 2^16: u16 x and values, u32 row sums
    bool tiny = false;   // m <= 256, one vector per pass: u8 x and values, u32 row sums
    bool mont = false;   // odd 2^16 < m < 2^31: values in Montgomery form (v 2^32 mod m)
    int nv = 1;          // vectors per pass: x and row sums interleaved by vector
    int q = 1;           // CTAs per cluster (column groups)
    int ngroup = 0;      // row groups
    int rows_max = 0;    // most rows in one group
    int resident = 0;    // clusters of q CTAs of the panel kernel resident at once
    int px = 0;          // bytes of x per panel (a multiple of 128)
    int pe = 0;          // entry capacity of a stage (a multiple of 8)
    int eb = 0;          // bytes per stage's entry buffer (a multiple of 128)
    long long ncols = 0; // x elements to stage
    long long nstage = 0;
    long long npm = 0;   // entries in the +-1 sections
    long long npad = 0;  // zero entries padding the general sections
    size_t smem = 0;     // dynamic shared memory per CTA
    const u32 *grp_row0 = nullptr;    // [ngroup + 1]
    const u32 *stage_ptr = nullptr;   // [ngroup * q + 1]
    const PanelStage *stage = nullptr;
    const u32 *ent = nullptr;
    const void *val = nullptr;
    void *xh = nullptr;  // staged x: u16 / u32, nv vectors interleaved, zero padded; xcols copies
    long long xstride = 0; // elements from one staged copy to the next
    int xcols = 1;         // staged copies (vectors staged by one launch when nv = 1)
    u32 *gbar = nullptr; // grid barrier: arrivals, generation
};

// Most clusters of q CTAs of the panel kernel for nv vectors per pass
// resident at once with `smem` bytes of dynamic shared memory each (0 when
// the launch cannot fit).
int panel_max_clusters(bool small, int nv, int q, size_t smem, bool tiny = false);

// One matrix plan (A or A^T).
struct Plan {
    PanelPart panel;
    long long nrows = 0, ncols = 0, nnz = 0;
    int acc_wide = 0;
    int format = 0;
    std::vector<Phase> phases;  // 1 or 2
    void *arena = nullptr;      // one device allocation for all parts
    size_t arena_bytes = 0;
    u64 *carry = nullptr;       // COO carries, zero between calls (nrows)
    std::string summary;
    long long max_row = 0;
    double pm_fraction = 0.0;
};

}  // namespace ff

namespace ff {
struct Gf2Pattern;
}

struct ffspmv_handle {
    ff::Plan A;
    ff::Plan AT;
    bool has_T = false;
    int transpose_mode = 0;
    ffspmv_options opt;
    uint32_t m = 0;
    int device = 0;
    // transpose by atomics: exact 64-bit sums per column
    ff::u64 *scatter = nullptr;
    size_t scatter_elems = 0;
    // host copy of the CSR for the atomic transpose (device arrays)
    void *csr_arena = nullptr;
    const long long *d_rowptr = nullptr;
    const int *d_col = nullptr;
    const ff::u32 *d_val = nullptr;
    // host copy of the CSR (values reduced mod m), for layouts built later
    std::vector<long long> h_ptr;
    std::vector<int> h_col;
    std::vector<ff::u32> h_val;
    // block sequence state
    void *seq_state = nullptr;
    int *d_status = nullptr;   // device status word (timeouts)
    // patterns of the odd entries of A and A^T for the GF(2) products
    ff::Gf2Pattern *gf2[2] = {nullptr, nullptr};
    // x-panel plans of A and A^T for 2 and 4 vectors per pass, built on the
    // first block that uses them when the plan is the x-panel layout
    ff::Plan *multi[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
};

namespace ff {

// plan.cu
ffspmv_status build_plan(Plan &P, long long nrows, long long ncols,
                         const long long *ptr, const int *col, const u32 *val,
                         u32 m, const ffspmv_options &opt, cudaStream_t st);
void free_plan(Plan &P);

// kernels.cu
// Run-time controls of the x-panel kernel's bounded waits.
struct PanelCtl {
    int *status = nullptr;  // device word: bit 0 set when a wait ran out
    int skip_stage = -1;    // testing only: the copies of this stage of every CTA are never issued
};

ffspmv_status run_plan(const Plan &P, const u32 *x, long long ldx, u32 *y,
                       long long ldy, int nvec, u32 m, u32 alpha, u32 beta,
                       cudaStream_t st, const PanelCtl *ctl = nullptr);
ffspmv_status run_scatter_transpose(ffspmv_handle *h, const u32 *x,
                                    long long ldx, u32 *y, long long ldy,
                                    int nvec, u32 alpha, u32 beta,
                                    cudaStream_t st);
long long count_plan_launches(const Plan &P, int nvec);
ffspmv_status check_range(const u32 *x, long long rows, long long ld,
                          int nvec, u32 m, int *d_flag, cudaStream_t st,
                          bool *bad);

}  // namespace ff

namespace ff {
// Records the failing CUDA call (per host thread) for ffspmv_last_error().
void note_cuda_error(cudaError_t e, const char *file, int line);
}

#define FF_CUDA(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) {                                 \
            ff::note_cuda_error(e_, __FILE__, __LINE__);         \
            return FFSPMV_ERR_CUDA;                              \
        }                                                        \
    } while (0)
