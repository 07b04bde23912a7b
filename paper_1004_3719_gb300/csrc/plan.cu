// Host-side plan construction: split a CSR matrix into the storage formats
// of Sec. 2.1 and 2.4 and lay every part out for the device.
//
//   CSR     plain row-wise storage, `group` lanes per row
//   ELLR    ELL_R, column-major with per-row counts (Sec. 2.4.3, Basic formats)
//   COO     coordinate triples (Sec. 2.1), element-parallel
//   COOS    COO_S: CSR over the non-empty rows only (Sec. 2.4.4, Hybridization)
//   DIA     diagonals stored densely with their offsets (Sec. 2.1)
//   HYBRID  the heuristic chooser of Sec. 2.4.5: dense diagonals to DIA, the
//           first w entries of every row to ELL_R, the residue to CSR, COO or
//           COO_S by its number of non-empty rows and entries per row
//   BINNED  rows binned by length, one format per bin (the library's own
//           layout; the bin formats come from the heuristic table, the
//           exhaustive search or the selector network)
//
// +-1 entries (Sec. 2.4.2) are moved to the front of each row's tail and
// flagged in the two top bits of the column word; value arrays then hold the
// general entries only, or nothing when a part is all +-1.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <numeric>

#include "ff_internal.cuh"
#include "ff_plan.h"

namespace ff {

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kNo = (size_t)-1;

struct Blob {
    std::vector<unsigned char> host;
    size_t put(const void *p, size_t n)
    {
        size_t off = (host.size() + kAlign - 1) / kAlign * kAlign;
        host.resize(off + (n ? n : 1));
        if (n) memcpy(host.data() + off, p, n);
        return off;
    }
    template <class T>
    size_t putv(const std::vector<T> &v)
    {
        return put(v.data(), v.size() * sizeof(T));
    }
};

struct SegBuild {
    SegDesc d;
    size_t o_rows = kNo, o_ptr = kNo, o_vptr = kNo, o_col = kNo, o_val = kNo;
    size_t o_rowid = kNo, o_rownb = kNo, o_doff = kNo, o_dval = kNo;
    size_t o_crow = kNo, o_cbeg = kNo;
    std::vector<u32> split;
    SegBuild() { memset(&d, 0, sizeof(d)); }
};

// A CSR matrix on the host with per-entry +-1 class (values already < m).
struct Mat {
    long long nrows = 0, ncols = 0;
    std::vector<long long> ptr;
    std::vector<u32> col;
    std::vector<u32> val;
    std::vector<unsigned char> cls;  // 0 general, kPlus, kMinus
};

unsigned char classify(u32 v, u32 m)
{
    if (v == 1u) return (unsigned char)kPlus;
    if (m > 2u && v == m - 1u) return (unsigned char)kMinus;
    return 0;
}

// Rows of a segment: identity range [row0, row0 + n) or an explicit list.
struct Rows {
    std::vector<u32> ids;
    long long row0 = 0, n = 0;
    long long at(long long r) const { return ids.empty() ? row0 + r : (long long)ids[r]; }
};

int value_bytes(u32 m) { return m <= 65536u ? 2 : 4; }

void push_val(std::vector<unsigned char> &out, u32 v, int vb)
{
    if (vb == 2) {
        unsigned short s = (unsigned short)v;
        const unsigned char *p = (const unsigned char *)&s;
        out.insert(out.end(), p, p + 2);
    } else {
        const unsigned char *p = (const unsigned char *)&v;
        out.insert(out.end(), p, p + 4);
    }
}

bool want_pm(int use_pm1, long long npm, long long total, long long ncols)
{
    if (npm == 0 || ncols > (long long)kColMask + 1) return false;
    if (use_pm1 == 1) return true;
    if (use_pm1 == 0) return false;
    return total > 0 && (double)npm >= 0.1 * (double)total;
}

// ---------------------------------------------------------------------------
// CSR-like segment (SEG_CSR / SEG_CSRBLK) over rows `R` of matrix `A`.
bool make_csr(Blob &B, const Mat &A, const Rows &R, int kind, int group,
              int use_pm1, int accum, u32 m, SegBuild &S, std::vector<u32> *ptr_out = nullptr)
{
    long long total = 0, npm = 0;
    for (long long r = 0; r < R.n; ++r) {
        long long i = R.at(r);
        for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) npm += A.cls[k] != 0;
        total += A.ptr[i + 1] - A.ptr[i];
    }
    if (total >= (1LL << 32)) return false;
    const bool pm = want_pm(use_pm1, npm, total, A.ncols);
    const long long ngen = pm ? total - npm : total;
    const int vb = (pm && ngen == 0) ? 0 : value_bytes(m);
    std::vector<u32> ptr(R.n + 1), vptr, col;
    std::vector<unsigned char> val;
    col.reserve(total);
    val.reserve((size_t)ngen * (vb ? vb : 1));
    if (pm && vb) vptr.resize(R.n + 1);
    u32 pos = 0, vpos = 0;
    for (long long r = 0; r < R.n; ++r) {
        long long i = R.at(r);
        ptr[r] = pos;
        if (!vptr.empty()) vptr[r] = vpos;
        if (!pm) {
            for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                col.push_back(A.col[k]);
                push_val(val, A.val[k], vb);
            }
            pos += (u32)(A.ptr[i + 1] - A.ptr[i]);
            continue;
        }
        for (int want = 0; want < 3; ++want) {
            for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                if (A.cls[k] != want) continue;
                col.push_back(A.col[k] | ((u32)want << kClassShift));
                if (want == 0) {
                    if (vb) push_val(val, A.val[k], vb);
                    ++vpos;
                }
                ++pos;
            }
        }
    }
    ptr[R.n] = pos;
    if (!vptr.empty()) vptr[R.n] = vpos;
    SegDesc &d = S.d;
    d.kind = kind;
    d.accum = accum;
    d.group = group;
    d.vbytes = vb;
    d.pm = pm ? 1 : 0;
    d.nrows = R.n;
    d.nnz = total;
    d.row0 = R.row0;
    d.ncols = A.ncols;
    d.nblocks = kind == SEG_CSRBLK ? R.n : (R.n + (kThreads / group) - 1) / (kThreads / group);
    if (!R.ids.empty()) S.o_rows = B.putv(R.ids);
    S.o_ptr = B.putv(ptr);
    if (ptr_out) *ptr_out = ptr;
    if (!vptr.empty()) S.o_vptr = B.putv(vptr);
    S.o_col = B.putv(col);
    if (vb) S.o_val = B.putv(val);
    return true;
}

// Long rows `R` cut into chunks of kSplitChunk entries (SEG_CSRSPLIT).
bool make_csrsplit(Blob &B, const Mat &A, const Rows &R, int use_pm1, int accum, u32 m,
                   SegBuild &S)
{
    std::vector<u32> ptr;
    if (!make_csr(B, A, R, SEG_CSRSPLIT, 1, use_pm1, accum, m, S, &ptr)) return false;
    std::vector<u32> crow, cbeg;
    for (long long r = 0; r < R.n; ++r)
        for (u32 k = ptr[r]; k < ptr[r + 1]; k += kSplitChunk) {
            crow.push_back((u32)r);
            cbeg.push_back(k);
        }
    cbeg.push_back(ptr[R.n]);
    S.d.kind = SEG_CSRSPLIT;
    S.d.nblocks = (long long)crow.size();
    S.o_crow = B.putv(crow);
    S.o_cbeg = B.putv(cbeg);
    for (long long r = 0; r < R.n; ++r) S.split.push_back((u32)R.at(r));
    return true;
}

// CSR over rows `R`, with the rows longer than `split_at` entries moved to a
// SEG_CSRSPLIT segment.  Appends one or two segments to `out`.
bool make_csr_with_split(Blob &B, const Mat &A, const Rows &R, int group, int use_pm1,
                         int accum, u32 m, long long split_at, std::vector<SegBuild> &out)
{
    Rows shortr, longr;
    for (long long r = 0; r < R.n; ++r) {
        long long i = R.at(r);
        (A.ptr[i + 1] - A.ptr[i] > split_at ? longr : shortr).ids.push_back((u32)i);
    }
    shortr.n = (long long)shortr.ids.size();
    longr.n = (long long)longr.ids.size();
    if (longr.n == 0) {
        SegBuild s;
        if (!make_csr(B, A, R, SEG_CSR, group, use_pm1, accum, m, s)) return false;
        out.push_back(s);
        return true;
    }
    if (shortr.n) {
        SegBuild s;
        if (!make_csr(B, A, shortr, SEG_CSR, group, use_pm1, accum, m, s)) return false;
        out.push_back(s);
    }
    SegBuild s;
    if (!make_csrsplit(B, A, longr, use_pm1, accum, m, s)) return false;
    out.push_back(s);
    return true;
}

// One thread per row: `diag` offsets (values gathered into [ndiag][ld]) and
// the first `width` entries of each row in ELL_R (column-major).  Entries on
// the chosen diagonals must already be absent from `A` (see split_diagonals);
// `D` holds them.
bool make_ellr(Blob &B, const Mat &A, const Rows &R, const std::vector<int> &diag,
               const Mat *D, int use_pm1, int accum, u32 m, long long guard,
               SegBuild &S)
{
    long long width = 0, total = 0, npm = 0;
    bool uniform = true;
    for (long long r = 0; r < R.n; ++r) {
        long long i = R.at(r);
        long long L = A.ptr[i + 1] - A.ptr[i];
        if (r > 0 && L != width) uniform = false;
        width = std::max(width, L);
        total += L;
        for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) npm += A.cls[k] != 0;
    }
    const long long ld = (R.n + 31) / 32 * 32;
    const int vb0 = value_bytes(m);
    const bool pm = want_pm(use_pm1, npm, total, A.ncols);
    const int vb = (pm && npm == total) ? 0 : vb0;
    const double bytes = (double)width * ld * (4 + vb) + (double)diag.size() * ld * vb0;
    if (bytes > (double)guard) return false;
    std::vector<u32> col((size_t)(width * ld), 0u), rownb;
    std::vector<unsigned char> val((size_t)(width * ld) * (vb ? vb : 1), 0);
    if (!uniform) rownb.resize(R.n);
    for (long long r = 0; r < R.n; ++r) {
        long long i = R.at(r);
        long long j = 0;
        for (int want = 0; want < (pm ? 3 : 1); ++want) {
            for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                if (pm && A.cls[k] != want) continue;
                size_t idx = (size_t)(j * ld + r);
                col[idx] = A.col[k] | (pm ? ((u32)A.cls[k] << kClassShift) : 0u);
                if (vb == 2) ((unsigned short *)val.data())[idx] = (unsigned short)A.val[k];
                else if (vb == 4) ((u32 *)val.data())[idx] = A.val[k];
                ++j;
            }
        }
        if (!uniform) rownb[r] = (u32)j;
    }
    std::vector<unsigned char> dval;
    if (!diag.empty()) {
        dval.assign((size_t)diag.size() * ld * vb0, 0);
        for (long long r = 0; r < R.n; ++r) {
            long long i = R.at(r);
            for (long long k = D->ptr[i]; k < D->ptr[i + 1]; ++k) {
                long long off = (long long)D->col[k] - i;
                size_t di = std::find(diag.begin(), diag.end(), (int)off) - diag.begin();
                size_t idx = di * ld + r;
                u32 cur = vb0 == 2 ? ((unsigned short *)dval.data())[idx] : ((u32 *)dval.data())[idx];
                u32 nv = (u32)(((unsigned long long)cur + D->val[k]) % m);
                if (vb0 == 2) ((unsigned short *)dval.data())[idx] = (unsigned short)nv;
                else ((u32 *)dval.data())[idx] = nv;
            }
        }
    }
    SegDesc &d = S.d;
    d.kind = SEG_ELLR;
    d.accum = accum;
    d.vbytes = vb;
    d.dvbytes = vb0;
    d.pm = pm ? 1 : 0;
    d.ndiag = (int)diag.size();
    d.width = (int)width;
    d.nrows = R.n;
    d.nnz = total + (D ? (long long)D->col.size() : 0);
    d.row0 = R.row0;
    d.ld = ld;
    d.ncols = A.ncols;
    d.nblocks = (R.n + kThreads - 1) / kThreads;
    if (!R.ids.empty()) S.o_rows = B.putv(R.ids);
    if (width > 0) {
        S.o_col = B.putv(col);
        if (vb) S.o_val = B.putv(val);
        if (!uniform) S.o_rownb = B.putv(rownb);
    }
    if (!diag.empty()) {
        S.o_doff = B.putv(diag);
        S.o_dval = B.putv(dval);
    }
    return true;
}

// COO over rows `R` (their entries in row order).
bool make_coo(Blob &B, const Mat &A, const Rows &R, int use_pm1, int accum, u32 m,
              SegBuild &S)
{
    long long total = 0, npm = 0;
    for (long long r = 0; r < R.n; ++r) {
        long long i = R.at(r);
        total += A.ptr[i + 1] - A.ptr[i];
        for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) npm += A.cls[k] != 0;
    }
    if (total >= (1LL << 32)) return false;
    const bool pm = want_pm(use_pm1, npm, total, A.ncols);
    const int vb = (pm && npm == total) ? 0 : value_bytes(m);
    std::vector<u32> rowid, col;
    std::vector<unsigned char> val;
    rowid.reserve(total);
    col.reserve(total);
    for (long long r = 0; r < R.n; ++r) {
        long long i = R.at(r);
        for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            rowid.push_back((u32)i);
            col.push_back(A.col[k] | (pm ? ((u32)A.cls[k] << kClassShift) : 0u));
            if (vb) push_val(val, A.val[k], vb);
        }
    }
    const long long chunk = 32LL * kCooRuns;
    for (long long b = chunk; b < total; b += chunk)
        if (rowid[b - 1] == rowid[b] && (S.split.empty() || S.split.back() != rowid[b]))
            S.split.push_back(rowid[b]);
    SegDesc &d = S.d;
    d.kind = SEG_COO;
    d.accum = accum;
    d.vbytes = vb;
    d.pm = pm ? 1 : 0;
    d.nrows = R.n;
    d.nnz = total;
    d.ncols = A.ncols;
    long long nchunks = (total + chunk - 1) / chunk;
    d.nblocks = (nchunks + (kThreads / 32) - 1) / (kThreads / 32);
    S.o_rowid = B.putv(rowid);
    S.o_col = B.putv(col);
    if (vb) S.o_val = B.putv(val);
    return true;
}

void make_empty(Blob &B, const Rows &R, SegBuild &S)
{
    SegDesc &d = S.d;
    d.kind = SEG_EMPTY;
    d.nrows = R.n;
    d.row0 = R.row0;
    d.nblocks = (R.n + kThreads - 1) / kThreads;
    if (!R.ids.empty()) S.o_rows = B.putv(R.ids);
}

// ---------------------------------------------------------------------------
Mat load_matrix(long long nrows, long long ncols, const long long *ptr,
                const int *col, const u32 *val, u32 m)
{
    Mat A;
    A.nrows = nrows;
    A.ncols = ncols;
    A.ptr.assign(ptr, ptr + nrows + 1);
    const long long nnz = ptr[nrows];
    A.col.resize(nnz);
    A.val.resize(nnz);
    A.cls.resize(nnz);
    for (long long k = 0; k < nnz; ++k) {
        A.col[k] = (u32)col[k];
        u32 v = val[k] % m;
        A.val[k] = v;
        A.cls[k] = classify(v, m);
    }
    return A;
}

// Move the entries on the offsets `diag` into D; the rest stays in R.
void split_diagonals(const Mat &A, const std::vector<int> &diag, Mat &R, Mat &D)
{
    R.nrows = D.nrows = A.nrows;
    R.ncols = D.ncols = A.ncols;
    R.ptr.assign(A.nrows + 1, 0);
    D.ptr.assign(A.nrows + 1, 0);
    for (long long i = 0; i < A.nrows; ++i) {
        for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            long long off = (long long)A.col[k] - i;
            bool on = std::find(diag.begin(), diag.end(), (int)off) != diag.end();
            Mat &T = on ? D : R;
            T.col.push_back(A.col[k]);
            T.val.push_back(A.val[k]);
            T.cls.push_back(A.cls[k]);
        }
        R.ptr[i + 1] = (long long)R.col.size();
        D.ptr[i + 1] = (long long)D.col.size();
    }
}

// First `w` entries of each row into E, the rest into T.
void split_width(const Mat &A, long long w, Mat &E, Mat &T)
{
    E.nrows = T.nrows = A.nrows;
    E.ncols = T.ncols = A.ncols;
    E.ptr.assign(A.nrows + 1, 0);
    T.ptr.assign(A.nrows + 1, 0);
    for (long long i = 0; i < A.nrows; ++i) {
        for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            Mat &X = (k - A.ptr[i] < w) ? E : T;
            X.col.push_back(A.col[k]);
            X.val.push_back(A.val[k]);
            X.cls.push_back(A.cls[k]);
        }
        E.ptr[i + 1] = (long long)E.col.size();
        T.ptr[i + 1] = (long long)T.col.size();
    }
}

int pow2_floor(double x)
{
    int g = 1;
    while (g * 2 <= x && g < 32) g *= 2;
    return g;
}

int default_group(const Mat &A, long long nonempty)
{
    double mean = nonempty > 0 ? (double)A.col.size() / (double)nonempty : 1.0;
    return pow2_floor(mean);
}

Rows all_rows(long long n)
{
    Rows R;
    R.n = n;
    return R;
}

void split_rows_by_empty(const Mat &A, Rows &full, Rows &empty)
{
    for (long long i = 0; i < A.nrows; ++i)
        (A.ptr[i + 1] > A.ptr[i] ? full : empty).ids.push_back((u32)i);
    full.n = (long long)full.ids.size();
    empty.n = (long long)empty.ids.size();
}

// Offsets of the most filled diagonals: at least half their length filled and
// at least n/4 long, at most 8 of them (the DIA part of the hybrid).
std::vector<int> dense_diagonals(const Mat &A)
{
    std::vector<int> out;
    if (A.nrows < 1 || A.ncols < 1) return out;
    std::vector<long long> cnt((size_t)(A.nrows + A.ncols - 1), 0);
    for (long long i = 0; i < A.nrows; ++i)
        for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
            cnt[(size_t)((long long)A.col[k] - i + A.nrows - 1)]++;
    std::vector<std::pair<long long, int>> cand;
    for (size_t t = 0; t < cnt.size(); ++t) {
        if (!cnt[t]) continue;
        long long off = (long long)t - (A.nrows - 1);
        long long len = off >= 0 ? std::min(A.nrows, A.ncols - off) : std::min(A.nrows + off, A.ncols);
        if (len * 4 >= A.nrows && cnt[t] * 2 >= len) cand.push_back({cnt[t], (int)off});
    }
    std::sort(cand.begin(), cand.end(), [](auto &a, auto &b) { return a.first > b.first; });
    for (size_t i = 0; i < cand.size() && i < 8; ++i) out.push_back(cand[i].second);
    std::sort(out.begin(), out.end());
    return out;
}

std::vector<int> all_diagonals(const Mat &A)
{
    std::vector<char> seen((size_t)(A.nrows + A.ncols + 1), 0);
    std::vector<int> out;
    for (long long i = 0; i < A.nrows; ++i)
        for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            size_t t = (size_t)((long long)A.col[k] - i + A.nrows);
            if (!seen[t]) {
                seen[t] = 1;
                out.push_back((int)((long long)A.col[k] - i));
            }
        }
    std::sort(out.begin(), out.end());
    return out;
}

// Upload the blob, patch the segment pointers and lay out the CTA ranges.
ffspmv_status finish(Plan &P, Blob &B, std::vector<std::vector<SegBuild>> &phases)
{
    // split-row lists live in the same arena
    std::vector<size_t> o_split(phases.size(), kNo);
    bool any_coo = false;
    for (size_t p = 0; p < phases.size(); ++p) {
        std::vector<u32> all;
        for (auto &s : phases[p]) {
            all.insert(all.end(), s.split.begin(), s.split.end());
            if (s.d.kind == SEG_COO || s.d.kind == SEG_CSRSPLIT) any_coo = true;
        }
        if (!all.empty()) o_split[p] = B.putv(all);
        Phase ph;
        ph.nsplit = (long long)all.size();
        ph.split_rows_host = all;
        P.phases.push_back(ph);
    }
    P.arena_bytes = B.host.size();
    if (P.arena_bytes) {
        if (cudaMalloc(&P.arena, P.arena_bytes) != cudaSuccess) {
            P.arena = nullptr;
            return FFSPMV_ERR_OOM;
        }
        FF_CUDA(cudaMemcpy(P.arena, B.host.data(), P.arena_bytes, cudaMemcpyHostToDevice));
    }
    unsigned char *base = (unsigned char *)P.arena;
    auto at = [&](size_t o) -> void * { return o == kNo ? nullptr : (void *)(base + o); };
    for (size_t p = 0; p < phases.size(); ++p) {
        Phase &ph = P.phases[p];
        ph.split_rows = (const u32 *)at(o_split[p]);
        long long block = 0;
        if (phases[p].size() > (size_t)kMaxSeg) return FFSPMV_ERR_UNSUPPORTED;
        for (auto &s : phases[p]) {
            if (s.d.nblocks <= 0) continue;
            SegDesc d = s.d;
            d.rows = (const u32 *)at(s.o_rows);
            d.ptr = (const u32 *)at(s.o_ptr);
            d.vptr = (const u32 *)at(s.o_vptr);
            d.col = (const u32 *)at(s.o_col);
            d.val = at(s.o_val);
            d.rowid = (const u32 *)at(s.o_rowid);
            d.rownb = (const u32 *)at(s.o_rownb);
            d.doff = (const int *)at(s.o_doff);
            d.dval = at(s.o_dval);
            d.chunk_row = (const u32 *)at(s.o_crow);
            d.chunk_beg = (const u32 *)at(s.o_cbeg);
            d.block0 = block;
            block += d.nblocks;
            if (d.kind == SEG_COO || d.kind == SEG_CSRSPLIT) ph.has_atomic = true;
            ph.segs.push_back(d);
        }
    }
    if (any_coo && P.nrows > 0) {
        if (cudaMalloc(&P.carry, (size_t)P.nrows * sizeof(u64)) != cudaSuccess) {
            P.carry = nullptr;
            return FFSPMV_ERR_OOM;
        }
        FF_CUDA(cudaMemset(P.carry, 0, (size_t)P.nrows * sizeof(u64)));
    }
    return FFSPMV_OK;
}

const char *kind_name(const SegDesc &d)
{
    switch (d.kind) {
    case SEG_CSR: return "CSR";
    case SEG_CSRBLK: return "CSR-CTA";
    case SEG_ELLR: return d.width ? (d.ndiag ? "DIA+ELL_R" : "ELL_R") : "DIA";
    case SEG_COO: return "COO";
    case SEG_CSRSPLIT: return "CSR-split";
    default: return "EMPTY";
    }
}

void describe(Plan &P, const char *fmt_name)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %lld x %lld, nnz %lld, acc %s, %.1f MB\n", fmt_name,
             P.nrows, P.ncols, P.nnz, P.acc_wide ? "96-bit" : "64-bit",
             (double)P.arena_bytes / 1e6);
    P.summary = buf;
    for (size_t p = 0; p < P.phases.size(); ++p) {
        for (auto &d : P.phases[p].segs) {
            snprintf(buf, sizeof buf,
                     "  phase %zu %-9s rows %lld nnz %lld group %d width %d diag %d pm %d vbytes %d%s\n",
                     p + 1, kind_name(d), d.nrows, d.nnz, d.group, d.width, d.ndiag, d.pm,
                     d.vbytes, d.accum ? " (adds)" : "");
            P.summary += buf;
        }
        if (P.phases[p].nsplit) {
            snprintf(buf, sizeof buf, "  phase %zu COO rows split between warps: %lld\n", p + 1,
                     P.phases[p].nsplit);
            P.summary += buf;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
int bin_of_length(long long L)
{
    if (L <= 0) return 0;
    int b = 1;
    long long u = 1;
    while (u < L && b < kBins - 1) {
        u <<= 1;
        ++b;
    }
    return b;
}

long long bin_upper(int b) { return b <= 0 ? 0 : (1LL << (b - 1)); }

// The heuristic table of the binned layout.  Sec. 2.4.5 leaves the chooser's
// constants to per-architecture tuning; these are the per-bin formats that
// won most often (weighted by entries) in the exhaustive search over the
// 2000-matrix training family on GB300: ELL_R for single-entry rows, CSR with
// 2 to 32 lanes per row (about a quarter to half the bin's longest row) up to
// 512 entries, one CTA per row up to 8192 entries, rows split across CTAs
// beyond.
BinChoice heuristic_bin_choice(int b, double pm_fraction, int use_pm1)
{
    BinChoice c;
    const long long U = bin_upper(b);
    if (U <= 1) {
        c.kind = SEG_ELLR;
        c.group = 1;
    } else if (U <= 512) {
        // lanes per row for U = 2, 4, ..., 512
        static const int lanes[] = {2, 4, 4, 8, 8, 16, 16, 32, 32};
        int k = 0;
        while ((2LL << k) < U) ++k;
        c.kind = SEG_CSR;
        c.group = lanes[k];
    } else if (U <= 8192) {
        c.kind = SEG_CSRBLK;
        c.group = 32;
    } else {
        c.kind = SEG_CSRSPLIT;
        c.group = 32;
    }
    c.pm = use_pm1 == 1 ? 1 : use_pm1 == 0 ? 0 : (pm_fraction >= 0.1 ? 1 : 0);
    return c;
}

// x-panel layout: the host half (geometry, stages, entry order) is
// panel_layout (panel.cu); this puts it into the plan's arena.
bool make_panel(Blob &B, const Mat &A, u32 m, int use_pm1, int force_q, int nv, PanelPart &pp, size_t &o_grp,
                size_t &o_sptr, size_t &o_stage, size_t &o_ent, size_t &o_val, size_t &o_xh, size_t &o_bar)
{
    long long npm = 0;
    for (auto c : A.cls) npm += c != 0;
    const long long nnz = (long long)A.col.size();
    // +-1 sections: forced on or off by use_pm1, else when +-1 entries are
    // at least 5% of the matrix
    const bool pm_on = use_pm1 == 1 || (use_pm1 < 0 && nnz > 0 && npm * 20 >= nnz);
    PanelHost H;
    if (!panel_layout(A.nrows, A.ncols, A.ptr.data(), A.col.data(), A.val.data(), A.cls.data(), m, pm_on,
                      force_q, nv,
                      [nv, m](int q, bool small) {
                          return panel_max_clusters(small, nv, q, kPanelSmemMax, m <= 256u && nv == 1);
                      },
                      H))
        return false;
    const int vb = H.tiny ? 1 : H.small ? 2 : 4, xb = vb;
    std::vector<unsigned char> vbytes(H.val.size() * vb + 64, 0);
    for (size_t t = 0; t < H.val.size(); ++t) {
        if (vb == 1) vbytes[t] = (unsigned char)H.val[t];
        else if (vb == 2) ((unsigned short *)vbytes.data())[t] = (unsigned short)H.val[t];
        else ((u32 *)vbytes.data())[t] = H.val[t];
    }
    H.ent.resize(H.ent.size() + 16, 0);
    pp.on = true;
    pp.small = H.small;
    pp.tiny = H.tiny;
    pp.mont = H.mont;
    pp.nv = H.nv;
    pp.q = H.q;
    pp.ngroup = H.ngroup;
    pp.rows_max = H.rows_max;
    pp.resident = H.resident;
    pp.px = H.px;
    pp.pe = H.pe;
    pp.eb = H.eb;
    pp.ncols = A.ncols;
    pp.nstage = H.nstage;
    pp.npm = H.npm;
    pp.npad = H.npad;
    pp.smem = H.smem;
    o_grp = B.putv(H.grp_row0);
    o_sptr = B.putv(H.stage_ptr);
    o_stage = B.putv(H.stage);
    o_ent = B.putv(H.ent);
    o_val = B.putv(vbytes);
    // staged x: four copies (one per vector of a group) for one-vector passes
    pp.xcols = H.nv == 1 ? 4 : 1;
    pp.xstride = (A.ncols + H.pcols + 64 + 63) / 64 * 64 * H.nv;
    std::vector<unsigned char> z((size_t)pp.xstride * pp.xcols * xb, 0);
    o_xh = B.putv(z);
    std::vector<u32> bar(2, 0);  // grid barrier: arrivals, generation
    o_bar = B.putv(bar);
    return true;
}

ffspmv_status build_plan_ex(Plan &P, long long nrows, long long ncols,
                            const long long *ptr, const int *col, const u32 *val,
                            u32 m, const ffspmv_options &opt, const BinChoice *bins, int panel_nv)
{
    const Mat A = load_matrix(nrows, ncols, ptr, col, val, m);
    P.nrows = nrows;
    P.ncols = ncols;
    P.nnz = (long long)A.col.size();
    long long maxlen = 0, nonempty = 0, npm = 0;
    for (long long i = 0; i < nrows; ++i) {
        long long L = A.ptr[i + 1] - A.ptr[i];
        maxlen = std::max(maxlen, L);
        nonempty += L > 0;
    }
    for (auto c : A.cls) npm += c != 0;
    P.max_row = maxlen;
    P.pm_fraction = P.nnz ? (double)npm / (double)P.nnz : 0.0;
    // Sec. 2.2: at most floor((2^64-1)/B) terms fit a 64-bit accumulator.
    {
        unsigned __int128 B = (unsigned __int128)(m - 1) * (m - 1);
        if (B < m) B = m;
        unsigned __int128 kmax = (~(unsigned __int128)0 >> 64) / B;
        P.acc_wide = (unsigned __int128)maxlen > kmax ? 1 : 0;
    }
    const long long guard = opt.guard_bytes > 0 ? opt.guard_bytes : (32LL << 30);
    const int upm = opt.use_pm1;
    int fmt = opt.priority_format;
    if (fmt == FFSPMV_FMT_AUTO) fmt = FFSPMV_FMT_BINNED;
    P.format = fmt;
    Blob B;
    std::vector<std::vector<SegBuild>> phases(1);
    const char *name = "?";
    Rows full, empty;
    split_rows_by_empty(A, full, empty);
    auto add_empty_rows = [&](std::vector<SegBuild> &ph) {
        if (empty.n) {
            SegBuild s;
            make_empty(B, empty, s);
            ph.push_back(s);
        }
    };
    const int G = opt.group_width > 0 ? pow2_floor(opt.group_width) : default_group(A, nonempty);

    switch (fmt) {
    case FFSPMV_FMT_CSR: {
        name = "CSR";
        SegBuild s;
        if (!make_csr(B, A, all_rows(nrows), SEG_CSR, G, upm, 0, m, s)) return FFSPMV_ERR_UNSUPPORTED;
        phases[0].push_back(s);
        break;
    }
    case FFSPMV_FMT_COOS: {
        name = "COO_S";
        if (full.n) {
            SegBuild s;
            if (!make_csr(B, A, full, SEG_CSR, G, upm, 0, m, s)) return FFSPMV_ERR_UNSUPPORTED;
            phases[0].push_back(s);
        }
        add_empty_rows(phases[0]);
        break;
    }
    case FFSPMV_FMT_COO: {
        name = "COO";
        if (full.n) {
            SegBuild s;
            if (!make_coo(B, A, full, upm, 0, m, s)) return FFSPMV_ERR_UNSUPPORTED;
            phases[0].push_back(s);
        }
        add_empty_rows(phases[0]);
        break;
    }
    case FFSPMV_FMT_ELLR: {
        name = "ELL_R";
        SegBuild s;
        if (!make_ellr(B, A, all_rows(nrows), {}, nullptr, upm, 0, m, guard, s))
            return FFSPMV_ERR_UNSUPPORTED;
        phases[0].push_back(s);
        break;
    }
    case FFSPMV_FMT_DIA: {
        name = "DIA";
        std::vector<int> diag = all_diagonals(A);
        long long ld = (nrows + 31) / 32 * 32;
        if ((double)diag.size() * ld * value_bytes(m) > (double)guard) return FFSPMV_ERR_UNSUPPORTED;
        Mat R, D;
        split_diagonals(A, diag, R, D);
        SegBuild s;
        if (!make_ellr(B, R, all_rows(nrows), diag, &D, 0, 0, m, guard, s)) return FFSPMV_ERR_UNSUPPORTED;
        phases[0].push_back(s);
        break;
    }
    case FFSPMV_FMT_HYBRID: {
        // Sec. 2.4.5: DIA for dense diagonals; if the matrix is large enough
        // and most rows are filled, an ELL_R part of width w; the residue to
        // CSR, COO or COO_S by its empty rows and entries per row.
        name = "HYBRID";
        std::vector<int> diag = dense_diagonals(A);
        Mat R, D;
        split_diagonals(A, diag, R, D);
        long long ne = 0;
        std::vector<long long> lens;
        for (long long i = 0; i < nrows; ++i) {
            long long L = R.ptr[i + 1] - R.ptr[i];
            ne += L > 0;
            lens.push_back(L);
        }
        long long w = 0;
        if (opt.ell_width >= 0) {
            w = opt.ell_width;
        } else if (nrows >= 10000 && ne * 10 >= nrows * 9) {
            std::vector<long long> s = lens;
            size_t q = s.size() / 10;
            std::nth_element(s.begin(), s.begin() + q, s.end());
            w = s[q];
        }
        Mat E, T;
        split_width(R, w, E, T);
        const bool has_first = w > 0 || !diag.empty();
        if (has_first) {
            SegBuild s;
            if (!make_ellr(B, E, all_rows(nrows), diag, &D, upm, 0, m, guard, s))
                return FFSPMV_ERR_UNSUPPORTED;
            phases[0].push_back(s);
        }
        Rows tf, te;
        split_rows_by_empty(T, tf, te);
        if (tf.n) {
            const int acc = has_first ? 1 : 0;
            std::vector<SegBuild> &ph = has_first ? (phases.resize(2), phases[1]) : phases[0];
            const long long tnnz = (long long)T.col.size();
            SegBuild s;
            bool ok;
            if (tf.n * 2 < nrows) {  // COO_S: CSR over the non-empty residue rows
                ok = make_csr_with_split(B, T, tf, default_group(T, tf.n), upm, acc, m,
                                         kSplitChunk / 2, ph);
            } else if (tnnz < 2 * tf.n) {
                ok = make_coo(B, T, tf, upm, acc, m, s);
                if (ok) ph.push_back(s);
            } else {
                ok = make_csr_with_split(B, T, all_rows(nrows), default_group(T, tf.n), upm, acc,
                                         m, kSplitChunk / 2, ph);
            }
            if (!ok) return FFSPMV_ERR_UNSUPPORTED;
            if (!has_first && !(tf.n * 2 >= nrows && tnnz >= 2 * tf.n)) {
                Rows e2;
                for (long long i = 0; i < nrows; ++i)
                    if (T.ptr[i + 1] == T.ptr[i]) e2.ids.push_back((u32)i);
                e2.n = (long long)e2.ids.size();
                if (e2.n) {
                    SegBuild se;
                    make_empty(B, e2, se);
                    phases[0].push_back(se);
                }
            }
        } else if (!has_first) {
            SegBuild se;
            make_empty(B, all_rows(nrows), se);
            phases[0].push_back(se);
        }
        break;
    }
    case FFSPMV_FMT_BINNED: {
        name = "BINNED";
        std::vector<Rows> rb(kBins);
        std::vector<long long> bpm(kBins, 0), bnnz(kBins, 0);
        for (long long i = 0; i < nrows; ++i) {
            long long L = A.ptr[i + 1] - A.ptr[i];
            int b = bin_of_length(L);
            rb[b].ids.push_back((u32)i);
            bnnz[b] += L;
            for (long long k = A.ptr[i]; k < A.ptr[i + 1]; ++k) bpm[b] += A.cls[k] != 0;
        }
        // longest rows first: their CTAs start early and the short bins fill in
        for (int b = kBins - 1; b >= 0; --b) {
            Rows &R = rb[b];
            R.n = (long long)R.ids.size();
            if (!R.n) continue;
            SegBuild s;
            if (b == 0) {
                make_empty(B, R, s);
                phases[0].push_back(s);
                continue;
            }
            BinChoice c = bins ? bins[b] : heuristic_bin_choice(b, bnnz[b] ? (double)bpm[b] / bnnz[b] : 0.0, upm);
            int pmode = c.pm ? 1 : 0;
            bool ok;
            if (c.kind == SEG_ELLR)
                ok = make_ellr(B, A, R, {}, nullptr, pmode, 0, m, guard, s);
            else if (c.kind == SEG_COO)
                ok = make_coo(B, A, R, pmode, 0, m, s);
            else if (c.kind == SEG_CSRSPLIT)
                ok = make_csrsplit(B, A, R, pmode, 0, m, s);
            else
                ok = make_csr(B, A, R, c.kind == SEG_CSRBLK ? SEG_CSRBLK : SEG_CSR,
                              std::max(1, std::min(32, c.group)), pmode, 0, m, s);
            if (!ok) return FFSPMV_ERR_UNSUPPORTED;
            phases[0].push_back(s);
        }
        break;
    }
    case FFSPMV_FMT_PANEL: {
        name = "PANEL";
        size_t o_grp, o_sptr, o_stage, o_ent, o_val, o_xh, o_bar;
        if (make_panel(B, A, m, upm, opt.panel_cluster, panel_nv, P.panel, o_grp, o_sptr, o_stage, o_ent, o_val,
                       o_xh, o_bar)) {
            // rows beyond kPanelLong: split CSR segments adding into y after the panels
            Rows huge;
            for (long long i = 0; i < nrows; ++i)
                if (A.ptr[i + 1] - A.ptr[i] > kPanelLong) huge.ids.push_back((u32)i);
            huge.n = (long long)huge.ids.size();
            if (huge.n) {
                SegBuild sh;
                if (!make_csrsplit(B, A, huge, upm, 1, m, sh)) return FFSPMV_ERR_UNSUPPORTED;
                phases[0].push_back(sh);
            }
        } else {
            // nothing to stage: a plain CSR plan
            SegBuild s;
            if (!make_csr(B, A, all_rows(nrows), SEG_CSR, G, upm, 0, m, s)) return FFSPMV_ERR_UNSUPPORTED;
            phases[0].push_back(s);
            P.panel = PanelPart();
            break;
        }
        ffspmv_status st = finish(P, B, phases);
        if (st != FFSPMV_OK) return st;
        unsigned char *base = (unsigned char *)P.arena;
        P.panel.grp_row0 = (const u32 *)(base + o_grp);
        P.panel.stage_ptr = (const u32 *)(base + o_sptr);
        P.panel.stage = (const PanelStage *)(base + o_stage);
        P.panel.ent = (const u32 *)(base + o_ent);
        P.panel.val = base + o_val;
        P.panel.xh = base + o_xh;
        P.panel.gbar = (u32 *)(base + o_bar);
        describe(P, name);
        char buf[400];
        snprintf(buf, sizeof buf,
                 "  panels: %d row groups x %d column groups (clusters of %d, %d resident), %lld stages of %d B x"
                 " + %d entries, x staged as %s, %s row sums, %d vector(s) per pass, %lld entries in +-1 sections,"
                 " %lld padding\n",
                 P.panel.ngroup, P.panel.q, P.panel.q, P.panel.resident, P.panel.nstage, P.panel.px, P.panel.pe,
                 P.panel.tiny ? "u8" : P.panel.small ? "u16" : "u32", P.panel.small ? "u32" : P.panel.mont ? "2 x u32 (Montgomery terms)" : "2 x u32", P.panel.nv, P.panel.npm,
                 P.panel.npad);
        P.summary += buf;
        return FFSPMV_OK;
    }
    default:
        return FFSPMV_ERR_ARG;
    }
    ffspmv_status st = finish(P, B, phases);
    if (st != FFSPMV_OK) return st;
    describe(P, name);
    return FFSPMV_OK;
}

// ---------------------------------------------------------------------------
// Sub-plans over a row subset, for the exhaustive search.
struct PlanSource {
    Mat A;
    u32 m;
};

PlanSource *make_source(long long nrows, long long ncols, const long long *ptr, const int *col,
                        const u32 *val, u32 m)
{
    PlanSource *s = new PlanSource();
    s->A = load_matrix(nrows, ncols, ptr, col, val, m);
    s->m = m;
    return s;
}

void free_source(PlanSource *s) { delete s; }

ffspmv_status build_rows_plan(Plan &P, const PlanSource &src, const std::vector<u32> &rows,
                              const BinChoice &c)
{
    const Mat &A = src.A;
    P.nrows = A.nrows;
    P.ncols = A.ncols;
    P.nnz = 0;
    long long maxlen = 0;
    for (u32 i : rows) {
        long long L = A.ptr[i + 1] - A.ptr[i];
        maxlen = std::max(maxlen, L);
        P.nnz += L;
    }
    {
        const u32 m = src.m;
        unsigned __int128 B = (unsigned __int128)(m - 1) * (m - 1);
        if (B < m) B = m;
        unsigned __int128 kmax = (~(unsigned __int128)0 >> 64) / B;
        P.acc_wide = (unsigned __int128)maxlen > kmax ? 1 : 0;
    }
    Rows R;
    R.ids = rows;
    R.n = (long long)rows.size();
    Blob B;
    std::vector<std::vector<SegBuild>> phases(1);
    SegBuild s;
    bool ok;
    const int pm = c.pm ? 1 : 0;
    if (c.kind == SEG_ELLR)
        ok = make_ellr(B, A, R, {}, nullptr, pm, 0, src.m, 1LL << 32, s);
    else if (c.kind == SEG_COO)
        ok = make_coo(B, A, R, pm, 0, src.m, s);
    else if (c.kind == SEG_CSRSPLIT)
        ok = make_csrsplit(B, A, R, pm, 0, src.m, s);
    else
        ok = make_csr(B, A, R, c.kind == SEG_CSRBLK ? SEG_CSRBLK : SEG_CSR,
                      std::max(1, std::min(32, c.group)), pm, 0, src.m, s);
    if (!ok) return FFSPMV_ERR_UNSUPPORTED;
    phases[0].push_back(s);
    return finish(P, B, phases);
}

ffspmv_status build_plan(Plan &P, long long nrows, long long ncols,
                         const long long *ptr, const int *col, const u32 *val,
                         u32 m, const ffspmv_options &opt, cudaStream_t)
{
    return build_plan_ex(P, nrows, ncols, ptr, col, val, m, opt, nullptr);
}

void free_plan(Plan &P)
{
    if (P.arena) cudaFree(P.arena);
    if (P.carry) cudaFree(P.carry);
    P.arena = nullptr;
    P.carry = nullptr;
    P.phases.clear();
}

// CSR of A^T by a counting sort over columns (rows of A^T in column order,
// entries of each row of A^T in increasing row index of A).
void transpose_csr(long long nrows, long long ncols, const long long *ptr,
                   const int *col, const u32 *val, std::vector<long long> &tptr,
                   std::vector<int> &tcol, std::vector<u32> &tval)
{
    const long long nnz = ptr[nrows];
    tptr.assign(ncols + 1, 0);
    for (long long k = 0; k < nnz; ++k) tptr[col[k] + 1]++;
    for (long long j = 0; j < ncols; ++j) tptr[j + 1] += tptr[j];
    std::vector<long long> pos(tptr.begin(), tptr.end() - 1);
    tcol.resize(nnz);
    tval.resize(nnz);
    for (long long i = 0; i < nrows; ++i)
        for (long long k = ptr[i]; k < ptr[i + 1]; ++k) {
            long long p = pos[col[k]]++;
            tcol[p] = (int)i;
            tval[p] = val[k];
        }
}

}  // namespace ff
