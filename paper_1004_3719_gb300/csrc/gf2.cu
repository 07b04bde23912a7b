// Products over GF(2) = Z/2Z with bit-packed vectors: Y = A X or A^T X (or
// Y ^= ...), X holding 64 components per 64-bit word.  This is Sec. 2's
// y_i = sum_j A_ij x_j at m = 2, where a sum is an exclusive or and an entry
// counts when its value is odd; packing the components of a block of vectors
// into words is the binary case the paper's closing remarks point to.
//
// Only the pattern of the odd entries is kept (built on the first call, for A
// or A^T).  Rows of at most kGf2Long entries: G lanes per row (G from the mean
// row length), each lane over every G-th entry, then an exclusive or across
// the group.  Longer rows are cut into chunks of kGf2Chunk entries, one warp
// each, whose results meet in y by atomic exclusive or (the row kernel first
// clears those rows of y, unless accumulating).  A lane gathers W words of
// each x row it names (the host walks the words four at a time).
#include <algorithm>
#include <cstring>

#include "ff_internal.cuh"
#include "ff_plan.h"
#include "ff_select.h"

namespace ff {

constexpr int kGf2Threads = 256;
constexpr long long kGf2Long = 32;
constexpr long long kGf2Chunk = 1024;

struct Gf2Pattern {
    void *arena = nullptr;
    const long long *ptr = nullptr;  // [n + 1]
    const u32 *col = nullptr;        // odd entries only
    const long long *chunks = nullptr;  // [nlong][3]: row, first entry, end of a long-row chunk
    long long n = 0, ncols = 0, nnz = 0, nlong = 0;  // nlong: chunks
    int G = 1;
};

void free_gf2(ffspmv_handle *h)
{
    for (int t = 0; t < 2; ++t) {
        if (h->gf2[t]) {
            if (h->gf2[t]->arena) cudaFree(h->gf2[t]->arena);
            delete h->gf2[t];
            h->gf2[t] = nullptr;
        }
    }
}

namespace {

template <int W>
__global__ void __launch_bounds__(kGf2Threads)
k_gf2_rows(const long long *__restrict__ ptr, const u32 *__restrict__ col, long long n, int G,
           const u64 *__restrict__ X, u64 *__restrict__ Y, int w, int w0, int accumulate)
{
    const int lane = threadIdx.x & (G - 1);
    const int grp = (threadIdx.x & 31) / G, gpw = 32 / G;
    const long long wid = ((long long)blockIdx.x * kGf2Threads + threadIdx.x) >> 5;
    const long long nw = (long long)gridDim.x * kGf2Threads / 32;
    // warp-uniform loop: every lane takes part in the shuffles
    for (long long base = wid * gpw; base < n; base += nw * gpw) {
        const long long row = base + grp;
        u64 a[W];
#pragma unroll
        for (int v = 0; v < W; ++v) a[v] = 0;
        bool mine = false;
        if (row < n) {
            const long long s = __ldg(ptr + row), e = __ldg(ptr + row + 1);
            mine = e - s <= kGf2Long;  // longer rows: the warp kernel
            if (mine) {
                for (long long k = s + lane; k < e; k += 4LL * G) {
                    u32 c[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) c[u] = k + u * G < e ? __ldg(col + k + u * G) : 0xffffffffu;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (c[u] != 0xffffffffu)
#pragma unroll
                            for (int v = 0; v < W; ++v) a[v] ^= __ldg(X + (size_t)c[u] * w + w0 + v);
                }
            }
        }
        for (int off = G >> 1; off > 0; off >>= 1)
#pragma unroll
            for (int v = 0; v < W; ++v) a[v] ^= __shfl_xor_sync(0xffffffffu, a[v], off);
        if (row < n && lane == 0) {
#pragma unroll
            for (int v = 0; v < W; ++v) {
                u64 *yp = Y + (size_t)row * w + w0 + v;
                if (mine) *yp = accumulate ? (*yp ^ a[v]) : a[v];
                else if (!accumulate) *yp = 0;  // the chunks of a long row xor into it
            }
        }
    }
}

template <int W>
__global__ void __launch_bounds__(kGf2Threads)
k_gf2_long(const u32 *__restrict__ col, const long long *__restrict__ chunks, long long nchunks,
           const u64 *__restrict__ X, u64 *__restrict__ Y, int w, int w0)
{
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * kGf2Threads + threadIdx.x) >> 5;
    const long long nw = (long long)gridDim.x * kGf2Threads / 32;
    for (long long r = wid; r < nchunks; r += nw) {  // warp-uniform
        const long long row = __ldg(chunks + 3 * r), s = __ldg(chunks + 3 * r + 1), e = __ldg(chunks + 3 * r + 2);
        u64 a[W];
#pragma unroll
        for (int v = 0; v < W; ++v) a[v] = 0;
        for (long long k = s + lane; k < e; k += 128) {
            u32 c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) c[u] = k + 32 * u < e ? __ldg(col + k + 32 * u) : 0xffffffffu;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (c[u] != 0xffffffffu)
#pragma unroll
                    for (int v = 0; v < W; ++v) a[v] ^= __ldg(X + (size_t)c[u] * w + w0 + v);
        }
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int v = 0; v < W; ++v) a[v] ^= __shfl_xor_sync(0xffffffffu, a[v], off);
        if (lane == 0)
#pragma unroll
            for (int v = 0; v < W; ++v) atomicXor(reinterpret_cast<unsigned long long *>(Y + (size_t)row * w + w0 + v),
                                                  (unsigned long long)a[v]);
    }
}

// The pattern of the odd entries of A (or of A^T) from the handle's host CSR.
ffspmv_status build_gf2(ffspmv_handle *h, int transpose, Gf2Pattern *&out)
{
    const long long nr = h->A.nrows, nc = h->A.ncols;
    std::vector<long long> ptr(1, 0);
    std::vector<int> col;
    std::vector<u32> one;
    ptr.reserve(nr + 1);
    for (long long i = 0; i < nr; ++i) {
        for (long long k = h->h_ptr[i]; k < h->h_ptr[i + 1]; ++k)
            if (h->h_val[k] & 1u) col.push_back(h->h_col[k]);
        ptr.push_back((long long)col.size());
    }
    long long n = nr, ncols = nc;
    if (transpose) {
        one.assign(col.size(), 1u);
        std::vector<long long> tptr;
        std::vector<int> tcol;
        std::vector<u32> tval;
        transpose_csr(nr, nc, ptr.data(), col.data(), one.data(), tptr, tcol, tval);
        ptr.swap(tptr);
        col.swap(tcol);
        n = nc;
        ncols = nr;
    }
    const long long nnz = (long long)col.size();
    if (ncols >= (1LL << 32) - 1) return FFSPMV_ERR_UNSUPPORTED;
    std::vector<long long> chunks;
    long long short_entries = 0, short_rows = 0;
    for (long long i = 0; i < n; ++i) {
        const long long L = ptr[i + 1] - ptr[i];
        if (L > kGf2Long) {
            for (long long k = ptr[i]; k < ptr[i + 1]; k += kGf2Chunk) {
                chunks.push_back(i);
                chunks.push_back(k);
                chunks.push_back(std::min(ptr[i + 1], k + kGf2Chunk));
            }
        } else {
            short_entries += L;
            ++short_rows;
        }
    }
    Gf2Pattern *g = new Gf2Pattern();
    g->n = n;
    g->ncols = ncols;
    g->nnz = nnz;
    g->nlong = (long long)chunks.size() / 3;
    // lanes per short row: about four entries each
    const double mean = short_rows ? (double)short_entries / (double)short_rows : 1.0;
    while (g->G < 32 && 4.0 * g->G < mean) g->G <<= 1;
    const size_t b_ptr = (size_t)(n + 1) * 8, b_col = (size_t)std::max<long long>(nnz, 1) * 4;
    const size_t o_col = (b_ptr + 255) / 256 * 256, o_long = o_col + (b_col + 255) / 256 * 256;
    const size_t bytes = o_long + (size_t)std::max<long long>(g->nlong, 1) * 24;
    if (cudaMalloc(&g->arena, bytes) != cudaSuccess) {
        delete g;
        return FFSPMV_ERR_OOM;
    }
    char *base = (char *)g->arena;
    cudaMemcpy(base, ptr.data(), b_ptr, cudaMemcpyHostToDevice);
    if (nnz) cudaMemcpy(base + o_col, col.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice);
    if (g->nlong) cudaMemcpy(base + o_long, chunks.data(), (size_t)g->nlong * 24, cudaMemcpyHostToDevice);
    if (cudaGetLastError() != cudaSuccess) {
        cudaFree(g->arena);
        delete g;
        return FFSPMV_ERR_CUDA;
    }
    g->ptr = (const long long *)base;
    g->col = (const u32 *)(base + o_col);
    g->chunks = (const long long *)(base + o_long);
    out = g;
    return FFSPMV_OK;
}

template <int W>
ffspmv_status launch_gf2(const Gf2Pattern &g, const u64 *X, u64 *Y, int w, int w0, int acc, int nsm,
                         cudaStream_t st)
{
    if (g.n > 0) {
        const long long want = (g.n * g.G + kGf2Threads - 1) / kGf2Threads;
        const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>(want, 16LL * nsm));
        k_gf2_rows<W><<<blocks, kGf2Threads, 0, st>>>(g.ptr, g.col, g.n, g.G, X, Y, w, w0, acc);
        FF_CUDA(cudaGetLastError());
    }
    if (g.nlong > 0) {
        const long long want = (g.nlong * 32 + kGf2Threads - 1) / kGf2Threads;
        const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>(want, 16LL * nsm));
        k_gf2_long<W><<<blocks, kGf2Threads, 0, st>>>(g.col, g.chunks, g.nlong, X, Y, w, w0);
        FF_CUDA(cudaGetLastError());
    }
    return FFSPMV_OK;
}

}  // namespace
}  // namespace ff

using namespace ff;

extern "C" ffspmv_status spmv_apply_gf2(ffspmv_t h, int32_t transpose, const uint64_t *d_X, uint64_t *d_Y,
                                        int32_t words, int32_t accumulate, ffspmv_stream_t stream)
{
    if (!h || words < 1 || (transpose != 0 && transpose != 1)) return FFSPMV_ERR_ARG;
    if (h->m != 2u) return FFSPMV_ERR_UNSUPPORTED;
    const long long in_rows = transpose ? h->A.nrows : h->A.ncols;
    const long long out_rows = transpose ? h->A.ncols : h->A.nrows;
    if ((in_rows > 0 && !d_X) || (out_rows > 0 && !d_Y)) return FFSPMV_ERR_ARG;
    if (!h->gf2[transpose]) {
        Gf2Pattern *g = nullptr;
        ffspmv_status r = build_gf2(h, transpose, g);
        if (r != FFSPMV_OK) return r;
        h->gf2[transpose] = g;
    }
    const Gf2Pattern &g = *h->gf2[transpose];
    if (out_rows == 0) return FFSPMV_OK;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm = std::max(nsm, 1);
    cudaStream_t st = (cudaStream_t)stream;
    const u64 *X = (const u64 *)d_X;
    u64 *Y = (u64 *)d_Y;
    for (int w0 = 0; w0 < words; w0 += 4) {
        const int W = std::min(4, words - w0);
        ffspmv_status r = W == 4   ? launch_gf2<4>(g, X, Y, words, w0, accumulate ? 1 : 0, nsm, st)
                          : W == 3 ? launch_gf2<3>(g, X, Y, words, w0, accumulate ? 1 : 0, nsm, st)
                          : W == 2 ? launch_gf2<2>(g, X, Y, words, w0, accumulate ? 1 : 0, nsm, st)
                                   : launch_gf2<1>(g, X, Y, words, w0, accumulate ? 1 : 0, nsm, st);
        if (r != FFSPMV_OK) return r;
    }
    return FFSPMV_OK;
}
