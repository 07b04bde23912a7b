// spmv_apply_transpose_noalloc: the transpose product by exact 64-bit atomic
// scatter, with its scratch in a fixed array of this library instead of a
// buffer allocated on demand.
//
// Some callers cannot let a library allocate device memory while they run: a
// serving process that reserved its whole device-memory budget up front for
// its own pool has nothing left for a cudaMalloc, and a latency-bound caller
// cannot afford the implicit device-wide synchronisation of a cudaFree.  This
// entry point makes no cudaMalloc, cudaFree or other allocating call; the
// scratch (the exact per-column sums) lives in `g_scratch` below, which every
// GPU that loads the library holds until the process exits.
#include <atomic>
#include <cstring>

#include "ff_internal.cuh"

namespace ff {

namespace {

// 2^20 64-bit sums: 8 MiB per device, enough for ncols * min(nvec, 16) <= 2^20.
constexpr long long kScratchElems = 1LL << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) u64 g_scratch[kScratchElems];

// Device address of g_scratch per device, filled on the first call made with
// that device current (in host code the name g_scratch is only a stand-in).
// Host threads that race on the first call all store the same address.
std::atomic<u64 *> g_scratch_ptr[kMaxDevices] = {};

__global__ void k_zero(u64 *__restrict__ p, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) p[t] = 0;
}

// Every entry of row i of A adds val * x[i][v] (reduced) into acc[col][v].
__global__ void k_scatter(long long nrows, const long long *__restrict__ ptr,
                          const int *__restrict__ col, const u32 *__restrict__ val,
                          const u32 *__restrict__ x, long long ldx, int nv,
                          u64 *__restrict__ acc, const Mod M)
{
    const int G = 8;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x & (G - 1);
    if (i >= nrows) return;
    for (long long k = ptr[i] + lane; k < ptr[i + 1]; k += G) {
        const long long j = col[k];
        const u32 a = val[k];
        for (int v = 0; v < nv; ++v) {
            const u32 t = red64((u64)a * __ldg(x + i * ldx + v), M);
            if (t) atomicAdd(acc + j * nv + v, (u64)t);
        }
    }
}

__global__ void k_finish(long long ncols, int nv, const u64 *__restrict__ acc,
                         u32 *__restrict__ y, long long ldy, const Mod M)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncols * nv) return;
    const long long j = t / nv;
    const int v = (int)(t - j * nv);
    u32 *yp = y + j * ldy + v;
    *yp = combine(red64(acc[t], M), yp, false, M);
}

// The array of device `dev`, which must be the current device.
ffspmv_status scratch_for_device(int dev, u64 **out)
{
    if (dev < 0 || dev >= kMaxDevices) return FFSPMV_ERR_UNSUPPORTED;
    u64 *p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        FF_CUDA(cudaGetSymbolAddress((void **)&p, g_scratch));
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return FFSPMV_OK;
}

}  // namespace

}  // namespace ff

using namespace ff;

extern "C" ffspmv_status spmv_apply_transpose_noalloc(ffspmv_t h, const uint32_t *d_x,
                                                      int64_t ldx, uint32_t *d_y,
                                                      int64_t ldy, int32_t nvec,
                                                      uint32_t alpha, uint32_t beta,
                                                      ffspmv_stream_t stream)
{
    if (!h || nvec < 1 || ldx < nvec || ldy < nvec) return FFSPMV_ERR_ARG;
    const long long nrows = h->A.nrows, ncols = h->A.ncols;
    if ((nrows > 0 && !d_x) || (ncols > 0 && !d_y)) return FFSPMV_ERR_ARG;
    // the device copy of A's CSR exists only for FFSPMV_TRANSPOSE_ATOMIC handles
    if (!h->d_rowptr) return FFSPMV_ERR_UNSUPPORTED;
    if (ncols == 0) return FFSPMV_OK;
    if (ncols > kScratchElems) return FFSPMV_ERR_UNSUPPORTED;  // beyond the fixed scratch
    long long chunk = kScratchElems / ncols;
    if (chunk > 16) chunk = 16;
    if (chunk > nvec) chunk = nvec;
    // the handle's arrays live on h->device; the kernels run on the current one
    int dev = 0;
    FF_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) return FFSPMV_ERR_ARG;
    u64 *acc = nullptr;
    ffspmv_status st = scratch_for_device(dev, &acc);
    if (st != FFSPMV_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->opt.value_check && nrows > 0) {
        // the same input check as spmv_apply_transpose (a preallocated flag word)
        bool bad = false;
        st = check_range(d_x, nrows, ldx, nvec, h->m, h->d_status + 1, s, &bad);
        if (st != FFSPMV_OK) return st;
        if (bad) return FFSPMV_ERR_RANGE;
    }
    const Mod M = make_mod(h->m, alpha, beta);
    for (long long c0 = 0; c0 < nvec; c0 += chunk) {
        const int nv = (int)(nvec - c0 < chunk ? nvec - c0 : chunk);
        const long long t = ncols * nv;
        // the array keeps the previous call's sums: clear the part used here
        k_zero<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(acc, t);
        FF_CUDA(cudaGetLastError());
        if (nrows > 0) {
            const long long threads = nrows * 8;
            k_scatter<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
                nrows, h->d_rowptr, h->d_col, h->d_val, d_x + c0, ldx, nv, acc, M);
            FF_CUDA(cudaGetLastError());
        }
        k_finish<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(ncols, nv, acc, d_y + c0, ldy, M);
        FF_CUDA(cudaGetLastError());
    }
    return FFSPMV_OK;
}
