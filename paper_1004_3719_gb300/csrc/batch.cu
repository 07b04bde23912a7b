// Many independent products Y_j = A_j X_j (mod m_j) in one launch.
//
// The work list holds items of two kinds:
//   rows     a tile of consecutive short rows of one matrix; a group of G
//            lanes (G = the matrix's block width rounded up to a power of two)
//            handles one row, lane v accumulating component v, so the x loads
//            of an entry are contiguous across the group and need no
//            cross-lane reduction;
//   long row one row with at least `long_at` entries; the whole CTA shares
//            its entries (256/G entry lanes x G component lanes) and sums the
//            partials in shared memory.
// Each matrix brings its own modulus and Barrett constants (Sec. 2.2).  Items
// are ordered by decreasing estimated cost so that the longest start first.
// The tile height and the long-row threshold are picked by timing: the first
// call for a new set of handles and block widths tries a few shapes and
// keeps the fastest.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "ff_internal.cuh"
#include "ff_select.h"

namespace ff {

namespace {

constexpr int kBatchThreads = 256;
constexpr int kMaxBatch = 512;  // matrices per launch (pointer table in the launch parameters)

struct BMat {
    const long long *ptr;
    const int *col;
    const u32 *val;
    long long nrows;
    Mod M;
    int nvec;
    int G;
};

struct BItem {
    int mat;
    int rows;        // rows in this item; 0 marks a long-row item
    long long row0;
};

struct BPtrs {
    const u32 *x[kMaxBatch];
    u32 *y[kMaxBatch];
};

// acc += sum of val[k] * x[col[k] * nvec + lane] for k = k0, k0 + stride, ...
// below e, four entries at a time so that four gathers are in flight.
__device__ __forceinline__ void batch_entries(AccWide &acc, const BMat &A, const u32 *__restrict__ x,
                                              int lane, long long k0, long long e, long long stride)
{
    constexpr int U = 4;
    for (long long k = k0; k < e; k += U * stride) {
        long long c[U];
        u32 a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long kk = k + u * stride;
            c[u] = kk < e ? (long long)__ldg(A.col + kk) : -1;
            a[u] = kk < e ? __ldg(A.val + kk) : 0u;
        }
        u32 xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u] * A.nvec + lane) : 0u;
#pragma unroll
        for (int u = 0; u < U; ++u) acc.mad(a[u], xv[u]);
    }
}

__global__ void __launch_bounds__(kBatchThreads)
k_batch(const BMat *__restrict__ mats, const BItem *__restrict__ items, int mat0,
        const __grid_constant__ BPtrs P)
{
    __shared__ u64 red[kBatchThreads];
    const BItem it = items[blockIdx.x];
    const BMat &A = mats[it.mat];
    const u32 *__restrict__ x = P.x[it.mat - mat0];
    u32 *__restrict__ y = P.y[it.mat - mat0];
    const int G = A.G;
    const int lane = threadIdx.x & (G - 1);
    const int grp = threadIdx.x / G;
    const int groups = kBatchThreads / G;
    const bool active_lane = lane < A.nvec;
    if (it.rows > 0) {
        for (int r = grp; r < it.rows; r += groups) {
            const long long row = it.row0 + r;
            const long long s = __ldg(A.ptr + row), e = __ldg(A.ptr + row + 1);
            AccWide acc;
            acc.zero();
            if (active_lane) {
                batch_entries(acc, A, x, lane, s, e, 1);
                y[row * A.nvec + lane] = (u32)acc.partial(A.M);
            }
        }
        return;
    }
    // one long row shared by the whole CTA
    const long long row = it.row0;
    const long long s = __ldg(A.ptr + row), e = __ldg(A.ptr + row + 1);
    AccWide acc;
    acc.zero();
    if (active_lane) batch_entries(acc, A, x, lane, s + grp, e, groups);
    red[threadIdx.x] = active_lane ? acc.partial(A.M) : 0;  // each below m
    __syncthreads();
    for (int half = groups >> 1; half > 0; half >>= 1) {
        if (grp < half) red[threadIdx.x] += red[threadIdx.x + half * G];
        __syncthreads();
    }
    if (grp == 0 && active_lane) y[row * A.nvec + lane] = red64(red[threadIdx.x], A.M);
}

struct Shape {
    int tile_mult;     // rows per item = tile_mult * (256 / G)
    long long long_at; // rows with at least this many entries get a CTA
};

const Shape kShapes[] = {{1, 256}, {1, 1024}, {1, 1LL << 40}, {2, 256}, {2, 1024}, {4, 512}};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

struct WorkList {
    std::vector<BItem> items;
    std::vector<int> chunk_item0;  // first item of each chunk of kMaxBatch matrices
};

struct BatchCache {
    std::vector<ffspmv_handle *> hs;
    std::vector<int> nvec;
    std::vector<BMat> mats_host;
    void *dev = nullptr;
    size_t dev_bytes = 0;
    BMat *d_mats = nullptr;
    BItem *d_items = nullptr;
    int nitems = 0;
    std::vector<int> chunk_item0;
    int shape = -1;
};

BatchCache g_cache;

ffspmv_status ensure_csr_copy(ffspmv_handle *h)
{
    if (h->csr_arena) return FFSPMV_OK;
    const long long nrows = h->A.nrows, nnz = (long long)h->h_col.size();
    size_t b_ptr = (size_t)(nrows + 1) * 8, b_col = (size_t)nnz * 4, b_val = (size_t)nnz * 4;
    size_t o_col = (b_ptr + 255) / 256 * 256, o_val = o_col + (b_col + 255) / 256 * 256;
    if (cudaMalloc(&h->csr_arena, o_val + b_val + 4) != cudaSuccess) {
        h->csr_arena = nullptr;
        return FFSPMV_ERR_OOM;
    }
    char *base = (char *)h->csr_arena;
    FF_CUDA(cudaMemcpy(base, h->h_ptr.data(), b_ptr, cudaMemcpyHostToDevice));
    if (nnz) {
        FF_CUDA(cudaMemcpy(base + o_col, h->h_col.data(), b_col, cudaMemcpyHostToDevice));
        FF_CUDA(cudaMemcpy(base + o_val, h->h_val.data(), b_val, cudaMemcpyHostToDevice));
    }
    h->d_rowptr = (const long long *)base;
    h->d_col = (const int *)(base + o_col);
    h->d_val = (const u32 *)(base + o_val);
    return FFSPMV_OK;
}

int pow2_ceil(int v)
{
    int g = 1;
    while (g < v) g <<= 1;
    return g;
}

// Items for one shape, each chunk of kMaxBatch matrices ordered by cost.
WorkList make_items(const std::vector<ffspmv_handle *> &hs, const std::vector<BMat> &mats,
                    const Shape &sh)
{
    WorkList W;
    std::vector<std::pair<double, BItem>> items;
    size_t chunk_begin = 0;
    const int count = (int)hs.size();
    auto sort_chunk = [&]() {
        std::stable_sort(items.begin() + chunk_begin, items.end(),
                         [](const auto &a, const auto &b) { return a.first > b.first; });
    };
    for (int j = 0; j < count; ++j) {
        if (j % kMaxBatch == 0) {
            sort_chunk();
            chunk_begin = items.size();
            W.chunk_item0.push_back((int)items.size());
        }
        const BMat &b = mats[j];
        const long long tile = (long long)sh.tile_mult * (kBatchThreads / b.G);
        const long long *p = hs[j]->h_ptr.data();
        long long r0 = 0;
        while (r0 < b.nrows) {
            const long long L0 = p[r0 + 1] - p[r0];
            if (L0 >= sh.long_at) {
                BItem it;
                it.mat = j;
                it.row0 = r0;
                it.rows = 0;
                items.push_back({(double)L0 / (kBatchThreads / b.G), it});
                ++r0;
                continue;
            }
            long long r1 = r0;
            double cost = 0;
            while (r1 < b.nrows && r1 - r0 < tile && p[r1 + 1] - p[r1] < sh.long_at) {
                cost = std::max(cost, (double)(p[r1 + 1] - p[r1]));
                ++r1;
            }
            BItem it;
            it.mat = j;
            it.row0 = r0;
            it.rows = (int)(r1 - r0);
            items.push_back({cost * sh.tile_mult, it});
            r0 = r1;
        }
    }
    sort_chunk();
    W.chunk_item0.push_back((int)items.size());
    W.items.resize(items.size());
    for (size_t i = 0; i < items.size(); ++i) W.items[i] = items[i].second;
    return W;
}

ffspmv_status upload_items(BatchCache &C, const WorkList &W, int count)
{
    const size_t bm = (sizeof(BMat) * count + 255) / 256 * 256;
    const size_t need = bm + sizeof(BItem) * std::max<size_t>(W.items.size(), 1) + 256;
    if (need > C.dev_bytes) {
        if (C.dev) cudaFree(C.dev);
        C.dev = nullptr;
        C.dev_bytes = 0;
        if (cudaMalloc(&C.dev, need) != cudaSuccess) return FFSPMV_ERR_OOM;
        C.dev_bytes = need;
    }
    C.d_mats = (BMat *)C.dev;
    C.d_items = (BItem *)((char *)C.dev + bm);
    FF_CUDA(cudaMemcpy(C.d_mats, C.mats_host.data(), sizeof(BMat) * count, cudaMemcpyHostToDevice));
    if (!W.items.empty())
        FF_CUDA(cudaMemcpy(C.d_items, W.items.data(), sizeof(BItem) * W.items.size(),
                           cudaMemcpyHostToDevice));
    C.nitems = (int)W.items.size();
    C.chunk_item0 = W.chunk_item0;
    return FFSPMV_OK;
}

ffspmv_status launch(const BatchCache &C, int count, const uint32_t *const *d_x,
                     uint32_t *const *d_y, cudaStream_t st)
{
    for (int c = 0; c * kMaxBatch < count; ++c) {
        const int i0 = C.chunk_item0[c], i1 = C.chunk_item0[c + 1];
        if (i1 <= i0) continue;
        BPtrs P;
        memset(&P, 0, sizeof(P));
        for (int j = c * kMaxBatch; j < count && j < (c + 1) * kMaxBatch; ++j) {
            P.x[j - c * kMaxBatch] = d_x[j];
            P.y[j - c * kMaxBatch] = d_y[j];
        }
        k_batch<<<(unsigned)(i1 - i0), kBatchThreads, 0, st>>>(C.d_mats, C.d_items + i0,
                                                                c * kMaxBatch, P);
        FF_CUDA(cudaGetLastError());
    }
    return FFSPMV_OK;
}

}  // namespace

// Drop the cached work list if it refers to a handle being destroyed.
void batch_forget(ffspmv_handle *h)
{
    for (auto *x : g_cache.hs)
        if (x == h) {
            g_cache.hs.clear();
            g_cache.nvec.clear();
            return;
        }
}

}  // namespace ff

using namespace ff;

extern "C" ffspmv_status spmv_batch_apply(int32_t count, const ffspmv_t *hs,
                                          const uint32_t *const *d_x, uint32_t *const *d_y,
                                          const int32_t *nvec, ffspmv_stream_t stream)
{
    if (count < 0 || (count > 0 && (!hs || !d_x || !d_y || !nvec))) return FFSPMV_ERR_ARG;
    if (count == 0) return FFSPMV_OK;
    cudaStream_t st = (cudaStream_t)stream;
    BatchCache &C = g_cache;
    for (int j = 0; j < count; ++j) {
        if (!hs[j] || nvec[j] < 1 || nvec[j] > 32) return FFSPMV_ERR_ARG;
        if ((hs[j]->A.nrows > 0 && !d_y[j]) || (hs[j]->A.ncols > 0 && !d_x[j])) return FFSPMV_ERR_ARG;
    }
    bool same = (int)C.hs.size() == count;
    for (int j = 0; j < count && same; ++j) same = C.hs[j] == hs[j] && C.nvec[j] == nvec[j];
    if (same) return launch(C, count, d_x, d_y, st);

    C.hs.assign(hs, hs + count);
    C.nvec.assign(nvec, nvec + count);
    C.mats_host.assign(count, BMat());
    for (int j = 0; j < count; ++j) {
        ffspmv_status r = ensure_csr_copy(hs[j]);
        if (r != FFSPMV_OK) {
            C.hs.clear();
            return r;
        }
        BMat &b = C.mats_host[j];
        memset(&b, 0, sizeof(b));
        b.ptr = hs[j]->d_rowptr;
        b.col = hs[j]->d_col;
        b.val = hs[j]->d_val;
        b.nrows = hs[j]->A.nrows;
        b.M = make_mod(hs[j]->m, 1, 0);
        b.nvec = nvec[j];
        b.G = pow2_ceil(nvec[j]);
    }
    // time every shape on this batch (the outputs are written each time, with
    // the same values) and keep the fastest
    cudaEvent_t e0, e1;
    FF_CUDA(cudaEventCreate(&e0));
    FF_CUDA(cudaEventCreate(&e1));
    float best_ms = 0;
    int best = -1;
    for (int k = 0; k < kNumShapes; ++k) {
        WorkList W = make_items(C.hs, C.mats_host, kShapes[k]);
        ffspmv_status r = upload_items(C, W, count);
        if (r == FFSPMV_OK) r = launch(C, count, d_x, d_y, st);  // warm-up
        if (r != FFSPMV_OK) {
            C.hs.clear();
            return r;
        }
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2; ++rep) launch(C, count, d_x, d_y, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            C.hs.clear();
            return FFSPMV_ERR_CUDA;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0 || ms < best_ms) {
            best = k;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    C.shape = best;
    WorkList W = make_items(C.hs, C.mats_host, kShapes[best]);
    ffspmv_status r = upload_items(C, W, count);
    if (r != FFSPMV_OK) {
        C.hs.clear();
        return r;
    }
    return launch(C, count, d_x, d_y, st);
}
