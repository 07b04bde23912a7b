// Many independent products Y_j = A_j X_j (mod m_j) in one launch.
//
// The work list holds items of two kinds:
//   rows     a tile of consecutive short rows of one matrix; a group of G
//            lanes handles one row, lane l accumulating the V consecutive
//            components l*V ... l*V+V-1 (V = 4, 2 or 1, the largest dividing
//            the block width; G = block width / V rounded up to a power of
//            two), so the x loads of an entry are contiguous across the group
//            and need no cross-lane reduction;
//   long row one row with at least `long_at` entries; the whole CTA shares
//            its entries (256/G entry lanes x G component lanes) and sums the
//            partials in shared memory.
// Each matrix brings its own modulus and Barrett constants (Sec. 2.2).  When
// m <= 2^31 four products (each below 2^62) are summed in a 64-bit word before
// they are carried into the 96-bit accumulator.  Items
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
    int G;      // lanes per row
    int V;      // components per lane (the last active lane may have fewer: ragged)
    int ragged; // nvec is not a multiple of V
    int fold4;  // m <= 2^31: four products fit a 64-bit word
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

__device__ __forceinline__ void acc_add64(AccWide &acc, u64 v)
{
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(acc.w0), "+r"(acc.w1), "+r"(acc.w2)
        : "r"((u32)v), "r"((u32)(v >> 32)));
}

// p[0 ... V - 1] (the first `cnt` of them when RAG), one vector load when aligned
template <int V, bool RAG>
__device__ __forceinline__ void load_x(u32 (&xv)[V], const u32 *__restrict__ p, bool aligned, int cnt)
{
    if (RAG) {
#pragma unroll
        for (int v = 0; v < V; ++v) xv[v] = v < cnt ? __ldg(p + v) : 0u;
    } else if (V == 4 && aligned) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p));
        xv[0] = w.x; xv[1] = w.y; xv[2 % V] = w.z; xv[3 % V] = w.w;
    } else if (V == 2 && aligned) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
        xv[0] = w.x; xv[1 % V] = w.y;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) xv[v] = __ldg(p + v);
    }
}

// acc[v] += sum of val[k] * xb[col[k] * nvec + v] over k = k0, k0 + stride, ...
// below L (indices relative to the row's first entry; xb = x + this lane's
// first component): whole blocks of four entries, four gathers in flight,
// then the remainder.
template <int V, bool RAG>
__device__ __forceinline__ void batch_entries(AccWide (&acc)[V], const BMat &A, const u32 *__restrict__ xb,
                                              bool aligned, int cnt, const int *__restrict__ colp,
                                              const u32 *__restrict__ valp, int k0, int L, int stride)
{
    constexpr int U = 4;
    const u32 nv = (u32)A.nvec;
    int k = k0;
    for (; k + (U - 1) * stride < L; k += U * stride) {
        u32 c[U], a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            c[u] = (u32)__ldg(colp + k + u * stride);
            a[u] = __ldg(valp + k + u * stride);
        }
        u32 xv[U][V];
#pragma unroll
        for (int u = 0; u < U; ++u) load_x<V, RAG>(xv[u], xb + (size_t)c[u] * nv, aligned, cnt);
        if (A.fold4) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                u64 sum = 0;
#pragma unroll
                for (int u = 0; u < U; ++u) sum += (u64)a[u] * xv[u][v];
                acc_add64(acc[v], sum);
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v].mad(a[u], xv[u][v]);
        }
    }
    for (; k < L; k += stride) {
        const u32 c = (u32)__ldg(colp + k), a = __ldg(valp + k);
        u32 xv[V];
        load_x<V, RAG>(xv, xb + (size_t)c * nv, aligned, cnt);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v].mad(a, xv[v]);
    }
}

template <int V, bool RAG>
__device__ __forceinline__ void batch_item(const BItem &it, const BMat &A, const u32 *__restrict__ x,
                                           u32 *__restrict__ y, u64 *red)
{
    const int G = A.G;
    const int lane = threadIdx.x & (G - 1);
    const int grp = threadIdx.x / G;
    const int groups = kBatchThreads / G;
    const int comp = lane * V;
    const int cnt = min(V, A.nvec - comp);  // components of this lane
    const bool active_lane = cnt > 0;
    const bool aligned = ((reinterpret_cast<uintptr_t>(x) | (uintptr_t)(A.nvec * 4)) & (4 * V - 1)) == 0;
    if (it.rows > 0) {
        for (int r = grp; r < it.rows; r += groups) {
            const long long row = it.row0 + r;
            const long long s = __ldg(A.ptr + row), e = __ldg(A.ptr + row + 1);
            AccWide acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v].zero();
            if (active_lane) {
                batch_entries<V, RAG>(acc, A, x + comp, aligned, cnt, A.col + s, A.val + s, 0, (int)(e - s), 1);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    if (!RAG || v < cnt) y[row * A.nvec + comp + v] = (u32)acc[v].partial(A.M);
            }
        }
        return;
    }
    // one long row shared by the whole CTA
    const long long row = it.row0;
    const long long s = __ldg(A.ptr + row), e = __ldg(A.ptr + row + 1);
    AccWide acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v].zero();
    if (active_lane) batch_entries<V, RAG>(acc, A, x + comp, aligned, cnt, A.col + s, A.val + s, grp, (int)(e - s), groups);
#pragma unroll
    for (int v = 0; v < V; ++v) red[v * kBatchThreads + threadIdx.x] = active_lane ? acc[v].partial(A.M) : 0;  // each below m
    __syncthreads();
    for (int half = groups >> 1; half > 0; half >>= 1) {
        if (grp < half)
#pragma unroll
            for (int v = 0; v < V; ++v) red[v * kBatchThreads + threadIdx.x] += red[v * kBatchThreads + threadIdx.x + half * G];
        __syncthreads();
    }
    if (grp == 0 && active_lane)
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (!RAG || v < cnt) y[row * A.nvec + comp + v] = red64(red[v * kBatchThreads + threadIdx.x], A.M);
}

__global__ void __launch_bounds__(kBatchThreads)
k_batch(const BMat *__restrict__ mats, const BItem *__restrict__ items, int mat0,
        const __grid_constant__ BPtrs P)
{
    __shared__ u64 red[4 * kBatchThreads];
    const BItem it = items[blockIdx.x];
    const BMat &A = mats[it.mat];
    const u32 *__restrict__ x = P.x[it.mat - mat0];
    u32 *__restrict__ y = P.y[it.mat - mat0];
    if (A.ragged) batch_item<4, true>(it, A, x, y, red);
    else if (A.V == 4) batch_item<4, false>(it, A, x, y, red);
    else if (A.V == 2) batch_item<2, false>(it, A, x, y, red);
    else batch_item<1, false>(it, A, x, y, red);
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
    // recorded on the stream of the last launch; the work list is not
    // overwritten before it completes (a launch on another stream may still
    // be reading it)
    cudaEvent_t done = nullptr;
    bool pending = false;
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
    if (C.pending) {
        FF_CUDA(cudaEventSynchronize(C.done));
        C.pending = false;
    }
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

ffspmv_status launch(BatchCache &C, int count, const uint32_t *const *d_x,
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
    FF_CUDA(cudaEventRecord(C.done, st));
    C.pending = true;
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
    if (!C.done) FF_CUDA(cudaEventCreateWithFlags(&C.done, cudaEventDisableTiming));
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
        // entry indices within a row are 32-bit in the kernel
        if (hs[j]->A.max_row >= (1LL << 31)) {
            C.hs.clear();
            return FFSPMV_ERR_UNSUPPORTED;
        }
        b.nvec = nvec[j];
        // four components per lane; widths 1 and 2 exactly, others not a
        // multiple of 4 with a shorter last lane
        b.V = nvec[j] <= 2 ? nvec[j] : 4;
        b.ragged = nvec[j] > 2 && nvec[j] % 4 != 0;
        b.G = pow2_ceil((nvec[j] + b.V - 1) / b.V);
        b.fold4 = hs[j]->m <= (1u << 31) ? 1 : 0;
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
