// Many independent products Y_j = A_j X_j (mod m_j) in one launch.
//
// The work list holds one item per tile of rows of one matrix.  A CTA runs one
// item: a group of G lanes (G = the matrix's block width rounded up to a power
// of two) handles one row, lane v accumulating component v of the row, so the
// x loads of an entry are contiguous across the group and no cross-lane
// reduction is needed.  Each matrix brings its own modulus and Barrett
// constants (Sec. 2.2).  Items are ordered by decreasing estimated cost so
// that the longest tiles start first.
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
    int rows;        // rows in this item
    long long row0;
};

struct BPtrs {
    const u32 *x[kMaxBatch];
    u32 *y[kMaxBatch];
};

__global__ void __launch_bounds__(kBatchThreads)
k_batch(const BMat *__restrict__ mats, const BItem *__restrict__ items, int mat0,
        const __grid_constant__ BPtrs P)
{
    const BItem it = items[blockIdx.x];
    const BMat &A = mats[it.mat];
    const u32 *__restrict__ x = P.x[it.mat - mat0];
    u32 *__restrict__ y = P.y[it.mat - mat0];
    const int G = A.G;
    const int lane = threadIdx.x & (G - 1);
    const int grp = threadIdx.x / G;
    const int groups = kBatchThreads / G;
    const bool active_lane = lane < A.nvec;
    for (int r = grp; r < it.rows; r += groups) {
        const long long row = it.row0 + r;
        const long long s = __ldg(A.ptr + row), e = __ldg(A.ptr + row + 1);
        AccWide acc;
        acc.zero();
        if (active_lane) {
            for (long long k = s; k < e; ++k) {
                const long long c = __ldg(A.col + k);
                const u32 a = __ldg(A.val + k);
                acc.mad(a, __ldg(x + c * A.nvec + lane));
            }
            y[row * A.nvec + lane] = (u32)acc.partial(A.M);
        }
    }
}

struct BatchCache {
    std::vector<ffspmv_handle *> hs;
    std::vector<int> nvec;
    std::vector<BMat> mats_host;
    void *dev = nullptr;
    size_t dev_bytes = 0;
    BMat *d_mats = nullptr;
    BItem *d_items = nullptr;
    int nitems = 0;
    std::vector<int> chunk_item0;  // first item of each chunk of kMaxBatch matrices
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
    bool same = (int)C.hs.size() == count;
    for (int j = 0; j < count && same; ++j) same = C.hs[j] == hs[j] && C.nvec[j] == nvec[j];
    for (int j = 0; j < count; ++j) {
        if (!hs[j] || nvec[j] < 1 || nvec[j] > 32) return FFSPMV_ERR_ARG;
        if ((hs[j]->A.nrows > 0 && !d_y[j]) || (hs[j]->A.ncols > 0 && !d_x[j])) return FFSPMV_ERR_ARG;
    }
    if (!same) {
        C.hs.assign(hs, hs + count);
        C.nvec.assign(nvec, nvec + count);
        C.mats_host.assign(count, BMat());
        std::vector<std::pair<double, BItem>> items;
        C.chunk_item0.clear();
        size_t chunk_begin = 0;
        for (int j = 0; j < count; ++j) {
            if (j % kMaxBatch == 0) {
                // order the previous chunk's items by decreasing cost
                std::stable_sort(items.begin() + chunk_begin, items.end(),
                                 [](const auto &a, const auto &b) { return a.first > b.first; });
                chunk_begin = items.size();
                C.chunk_item0.push_back((int)items.size());
            }
            ffspmv_handle *h = hs[j];
            ffspmv_status r = ensure_csr_copy(h);
            if (r != FFSPMV_OK) return r;
            BMat &b = C.mats_host[j];
            memset(&b, 0, sizeof(b));
            b.ptr = h->d_rowptr;
            b.col = h->d_col;
            b.val = h->d_val;
            b.nrows = h->A.nrows;
            b.M = make_mod(h->m, 1, 0);
            b.nvec = nvec[j];
            b.G = pow2_ceil(nvec[j]);
            const int groups = kBatchThreads / b.G;
            const long long *p = h->h_ptr.data();
            for (long long r0 = 0; r0 < b.nrows; r0 += groups) {
                long long r1 = std::min(b.nrows, r0 + groups);
                BItem it;
                it.mat = j;
                it.row0 = r0;
                it.rows = (int)(r1 - r0);
                double cost = 0;
                for (long long i = r0; i < r1; ++i) cost = std::max(cost, (double)(p[i + 1] - p[i]));
                items.push_back({cost, it});
            }
        }
        std::stable_sort(items.begin() + chunk_begin, items.end(),
                         [](const auto &a, const auto &b) { return a.first > b.first; });
        C.nitems = (int)items.size();
        C.chunk_item0.push_back(C.nitems);
        size_t bm = (sizeof(BMat) * count + 255) / 256 * 256;
        size_t need = bm + sizeof(BItem) * items.size() + 256;
        if (need > C.dev_bytes) {
            if (C.dev) cudaFree(C.dev);
            C.dev = nullptr;
            C.dev_bytes = 0;
            if (cudaMalloc(&C.dev, need) != cudaSuccess) return FFSPMV_ERR_OOM;
            C.dev_bytes = need;
        }
        C.d_mats = (BMat *)C.dev;
        C.d_items = (BItem *)((char *)C.dev + bm);
        std::vector<BItem> flat(items.size());
        for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].second;
        FF_CUDA(cudaMemcpy(C.d_items, flat.data(), sizeof(BItem) * flat.size(), cudaMemcpyHostToDevice));
    }
    if (!same) {
        FF_CUDA(cudaMemcpy(C.d_mats, C.mats_host.data(), sizeof(BMat) * count, cudaMemcpyHostToDevice));
    }
    for (int c = 0; c * kMaxBatch < count; ++c) {
        const int i0 = C.chunk_item0[c], i1 = C.chunk_item0[c + 1];
        if (i1 <= i0) continue;
        BPtrs P;
        memset(&P, 0, sizeof(P));
        for (int j = c * kMaxBatch; j < count && j < (c + 1) * kMaxBatch; ++j) {
            P.x[j - c * kMaxBatch] = d_x[j];
            P.y[j - c * kMaxBatch] = d_y[j];
        }
        k_batch<<<(unsigned)(i1 - i0), kBatchThreads, 0, st>>>(C.d_mats, C.d_items + i0, c * kMaxBatch, P);
        FF_CUDA(cudaGetLastError());
    }
    return FFSPMV_OK;
}
