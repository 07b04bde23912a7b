// Format selection for the binned layout: matrix features on the device, the
// exhaustive per-bin search (timed sub-plans), and the selector network (a
// 22-64-64-11 MLP in fp32 with forward, loss, backward, Adam and inference
// kernels).  The selector replaces the heuristic chooser of Sec. 2.4.5 and
// only picks formats: every plan computes the same exact result.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/ffspmv_select.h"
#include "ff_select.h"

namespace ff {

// ---------------------------------------------------------------------------
// Candidate formats (index f of ffspmv_select.h).
BinChoice format_choice(int f, int pm)
{
    BinChoice c;
    c.pm = pm;
    c.group = 1;
    switch (f) {
    case 0: c.kind = SEG_ELLR; break;
    case 1: case 2: case 3: case 4: case 5: case 6:
        c.kind = SEG_CSR;
        c.group = 1 << (f - 1);
        break;
    case 7: c.kind = SEG_CSRBLK; c.group = 32; break;
    case 8: c.kind = SEG_CSRSPLIT; c.group = 32; break;
    default: c.kind = SEG_COO; break;
    }
    return c;
}

bool format_valid(int f, int bin, long long maxlen)
{
    const long long U = bin_upper(bin);
    if (bin <= 0) return false;
    switch (f) {
    case 0: return maxlen <= 128;
    case 1: case 2: case 3: case 4: case 5: case 6: return (1LL << (f - 1)) <= 2 * std::max(1LL, U);
    case 7: return U >= 32;
    case 8: return U >= 512;
    default: return true;
    }
}

namespace {

// ---------------------------------------------------------------------------
// Features.
struct FeatAcc {
    unsigned long long sum_len, sum_len2, max_len, n_empty, n_le4, n_ge64;
    unsigned long long n_pm, n_band, n_diag0, n_local, sum_dist, n_halfdiag;
    double sum_len3;
    unsigned long long bin_rows[kBins], bin_nnz[kBins], bin_pm[kBins];
};

__device__ __forceinline__ int dev_bin_of_length(long long L)
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

// One warp per row (grid-stride over rows).
__global__ void k_features_rows(long long nrows, long long ncols, const long long *__restrict__ ptr,
                                const int *__restrict__ col, const u32 *__restrict__ val, u32 m,
                                unsigned *__restrict__ hist, FeatAcc *acc)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long n = nrows > ncols ? nrows : ncols;
    const long long local = n / 64 > 1 ? n / 64 : 1;
    unsigned long long pm = 0, band = 0, d0 = 0, loc = 0, dist = 0;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nrows; i += warps) {
        const long long s = ptr[i], e = ptr[i + 1];
        const long long L = e - s;
        unsigned long long rpm = 0;
        for (long long k = s + lane; k < e; k += 32) {
            const long long j = col[k];
            const u32 v = val[k] % m;
            const bool ispm = v == 1u || (m > 2u && v == m - 1u);
            rpm += ispm;
            const long long dd = j - i;
            const long long ad = dd < 0 ? -dd : dd;
            band += ad <= 64;
            d0 += dd == 0;
            loc += ad <= local;
            dist += (unsigned long long)ad;
            atomicAdd(hist + (dd + nrows - 1), 1u);
        }
        for (int off = 16; off > 0; off >>= 1) rpm += __shfl_xor_sync(0xffffffffu, rpm, off);
        pm += (lane == 0) ? rpm : 0;
        if (lane == 0) {
            atomicAdd(&acc->sum_len, (unsigned long long)L);
            atomicAdd(&acc->sum_len2, (unsigned long long)(L * L));
            atomicAdd(&acc->sum_len3, (double)L * (double)L * (double)L);
            atomicMax(&acc->max_len, (unsigned long long)L);
            if (L == 0) atomicAdd(&acc->n_empty, 1ull);
            if (L > 0 && L <= 4) atomicAdd(&acc->n_le4, 1ull);
            if (L >= 64) atomicAdd(&acc->n_ge64, 1ull);
            const int b = dev_bin_of_length(L);
            atomicAdd(&acc->bin_rows[b], 1ull);
            atomicAdd(&acc->bin_nnz[b], (unsigned long long)L);
            atomicAdd(&acc->bin_pm[b], rpm);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        band += __shfl_xor_sync(0xffffffffu, band, off);
        d0 += __shfl_xor_sync(0xffffffffu, d0, off);
        loc += __shfl_xor_sync(0xffffffffu, loc, off);
        dist += __shfl_xor_sync(0xffffffffu, dist, off);
    }
    if (lane == 0) {
        atomicAdd(&acc->n_pm, pm);
        atomicAdd(&acc->n_band, band);
        atomicAdd(&acc->n_diag0, d0);
        atomicAdd(&acc->n_local, loc);
        atomicAdd(&acc->sum_dist, dist);
    }
}

// Entries on diagonals that are at least half full.
__global__ void k_features_diag(long long nrows, long long ncols, const unsigned *__restrict__ hist,
                                FeatAcc *acc)
{
    const long long nd = nrows + ncols - 1;
    unsigned long long s = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nd;
         t += (long long)gridDim.x * blockDim.x) {
        const long long off = t - (nrows - 1);
        const long long len = off >= 0 ? (nrows < ncols - off ? nrows : ncols - off)
                                        : (nrows + off < ncols ? nrows + off : ncols);
        const unsigned long long c = hist[t];
        if (c > 0 && 2 * c >= (unsigned long long)len) s += c;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(&acc->n_halfdiag, s);
}

// Matrix features (n rows, N columns, row lengths L, nnz, mean = nnz/n; "+-1"
// means value mod m equal to 1 or m-1):
//   0 log2(n)/32               1 log2(N)/32              2 log2(1+mean)/16
//   3 min(std(L)/mean,10)/10   4 log2(1+max L)/32        5 share of empty rows
//   6 share of rows with 1 <= L <= 4                     7 share of rows with L >= 64
//   8 share of +-1 entries     9 log2(m)/32              10 share with |j-i| <= 64
//  11 share with j == i       12 share with |j-i| <= max(1, max(n,N)/64)
//  13 mean |j-i| / max(n,N)   14 skewness of L, clipped to [-10,10], /10
//  15 share of entries on diagonals that hold at least half their length
// Bin features of bin b: b/16, rows share, nnz share, +-1 share in the bin,
// (nnz_b/rows_b)/2^(b-1), log2(1+rows_b)/32.
__global__ void k_features_final(long long nrows, long long ncols, u32 m, const FeatAcc *acc,
                                 float *feat, float *binfeat)
{
    if (threadIdx.x != 0) return;
    const double n = (double)(nrows > 0 ? nrows : 1);
    const double nnz = (double)acc->sum_len;
    const double nz = nnz > 0 ? nnz : 1.0;
    const double mean = nnz / n;
    const double ex2 = (double)acc->sum_len2 / n;
    const double ex3 = acc->sum_len3 / n;
    const double var = ex2 - mean * mean > 0 ? ex2 - mean * mean : 0.0;
    const double sd = sqrt(var);
    double cv = mean > 0 ? sd / mean : 0.0;
    if (cv > 10) cv = 10;
    double sk = 0;
    if (sd > 0) {
        sk = (ex3 - 3 * mean * ex2 + 2 * mean * mean * mean) / (sd * sd * sd);
        sk = sk > 10 ? 10 : (sk < -10 ? -10 : sk);
    }
    const double big = (double)(nrows > ncols ? nrows : ncols);
    feat[0] = (float)(log2(n) / 32);
    feat[1] = (float)(log2((double)(ncols > 0 ? ncols : 1)) / 32);
    feat[2] = (float)(log2(1 + mean) / 16);
    feat[3] = (float)(cv / 10);
    feat[4] = (float)(log2(1 + (double)acc->max_len) / 32);
    feat[5] = (float)(acc->n_empty / n);
    feat[6] = (float)(acc->n_le4 / n);
    feat[7] = (float)(acc->n_ge64 / n);
    feat[8] = (float)(acc->n_pm / nz);
    feat[9] = (float)(log2((double)m) / 32);
    feat[10] = (float)(acc->n_band / nz);
    feat[11] = (float)(acc->n_diag0 / nz);
    feat[12] = (float)(acc->n_local / nz);
    feat[13] = (float)(((double)acc->sum_dist / nz) / (big > 0 ? big : 1));
    feat[14] = (float)(sk / 10);
    feat[15] = (float)(acc->n_halfdiag / nz);
    for (int b = 0; b < kBins; ++b) {
        const double r = (double)acc->bin_rows[b], z = (double)acc->bin_nnz[b];
        float *f = binfeat + b * FFSPMV_NUM_BIN_FEATURES;
        f[0] = (float)(b / 16.0);
        f[1] = (float)(r / n);
        f[2] = (float)(z / nz);
        f[3] = (float)(z > 0 ? acc->bin_pm[b] / z : 0.0);
        f[4] = (float)(b > 0 && r > 0 ? (z / r) / (double)(1LL << (b - 1)) : 0.0);
        f[5] = (float)(log2(1 + r) / 32);
    }
}

// ---------------------------------------------------------------------------
// Selector network.
constexpr int kIn = FFSPMV_MLP_IN, kH = FFSPMV_MLP_HIDDEN, kOut = FFSPMV_MLP_OUT;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kOut * kH;
static_assert(kOffB3 + kOut == FFSPMV_MLP_PARAMS, "parameter layout");

// out[b][o] = act(sum_i W[o][i] * in[b][i] + bias[o]), one thread per (b, o).
__global__ void k_dense(const float *__restrict__ W, const float *__restrict__ bias,
                        const float *__restrict__ in, int ldin, int batch, int I, int O,
                        float *__restrict__ out, int ldout, int relu)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)batch * O) return;
    const int b = (int)(t / O), o = (int)(t % O);
    float s = bias[o];
    const float *w = W + (long long)o * I;
    const float *x = in + (long long)b * ldin;
    for (int i = 0; i < I; ++i) s = fmaf(w[i], x[i], s);
    out[(long long)b * ldout + o] = relu ? fmaxf(s, 0.f) : s;
}

// gW[o][i] = sum_b dz[b][o] * in[b][i], gb[o] = sum_b dz[b][o]; block o,
// thread i (i == I gives the bias).
__global__ void k_grad_w(const float *__restrict__ dz, int lddz, const float *__restrict__ in,
                         int ldin, int batch, int I, float *__restrict__ gW, float *__restrict__ gb)
{
    const int o = blockIdx.x, i = threadIdx.x;
    if (i > I) return;
    float s = 0.f;
    for (int b = 0; b < batch; ++b) {
        const float d = dz[(long long)b * lddz + o];
        s = fmaf(d, i < I ? in[(long long)b * ldin + i] : 1.f, s);
    }
    if (i < I) gW[(long long)o * I + i] = s;
    else gb[o] = s;
}

// dh[b][i] = (sum_o W[o][i] * dz[b][o]) * (h[b][i] > 0)
__global__ void k_grad_in(const float *__restrict__ W, const float *__restrict__ dz, int lddz,
                          const float *__restrict__ h, int ldh, int batch, int I, int O,
                          float *__restrict__ dh, int lddh)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)batch * I) return;
    const int b = (int)(t / I), i = (int)(t % I);
    float s = 0.f;
    for (int o = 0; o < O; ++o) s = fmaf(W[(long long)o * I + i], dz[(long long)b * lddz + o], s);
    dh[(long long)b * lddh + i] = h[(long long)b * ldh + i] > 0.f ? s : 0.f;
}

__global__ void k_mask_sum(const float *__restrict__ mask, long long n, float *cnt)
{
    float s = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        s += mask[t];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(cnt, s);
}

__global__ void k_loss_grad(const float *__restrict__ out, const float *__restrict__ target,
                            const float *__restrict__ mask, long long n, const float *cnt,
                            float *__restrict__ dout, float *loss)
{
    const float c = fmaxf(*cnt, 1.f);
    float s = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const float d = mask[t] * (out[t] - target[t]);
        dout[t] = 2.f * d / c;
        s += d * d;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / c);
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float a = b1 * m1[t] + (1.f - b1) * gt;
    const float b = b2 * m2[t] + (1.f - b2) * gt * gt;
    m1[t] = a;
    m2[t] = b;
    p[t] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// Inference inputs: row b = [matrix features, features of bin b].
// Rows 0..kBins-1: the (matrix, bin) inputs; row kBins: the matrix-level
// input, its bin features all FFSPMV_MATRIX_INPUT.
__global__ void k_selector_inputs(const float *__restrict__ feat, const float *__restrict__ binfeat,
                                  float *__restrict__ in)
{
    const int b = blockIdx.x, i = threadIdx.x;
    if (b > kBins || i >= kIn) return;
    in[b * kIn + i] = i < FFSPMV_NUM_FEATURES ? feat[i]
                      : b == kBins            ? FFSPMV_MATRIX_INPUT
                                              : binfeat[b * FFSPMV_NUM_BIN_FEATURES + i - FFSPMV_NUM_FEATURES];
}

unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

ffspmv_status mlp_forward(const float *P, const float *in, int batch, float *act, float *out,
                          cudaStream_t st)
{
    if (batch <= 0) return FFSPMV_OK;
    k_dense<<<blocks_for((long long)batch * kH, 256), 256, 0, st>>>(P + kOffW1, P + kOffB1, in, kIn,
                                                                    batch, kIn, kH, act, 2 * kH, 1);
    k_dense<<<blocks_for((long long)batch * kH, 256), 256, 0, st>>>(P + kOffW2, P + kOffB2, act, 2 * kH,
                                                                    batch, kH, kH, act + kH, 2 * kH, 1);
    k_dense<<<blocks_for((long long)batch * kOut, 256), 256, 0, st>>>(P + kOffW3, P + kOffB3, act + kH,
                                                                      2 * kH, batch, kH, kOut, out, kOut, 0);
    FF_CUDA(cudaGetLastError());
    return FFSPMV_OK;
}

// ---------------------------------------------------------------------------
// Installed selector weights (host copy; uploaded per device on use).
std::mutex g_sel_mu;
std::vector<float> g_sel_host;

struct DevCSR {
    void *mem = nullptr;
    const long long *ptr = nullptr;
    const int *col = nullptr;
    const u32 *val = nullptr;
    ~DevCSR()
    {
        if (mem) cudaFree(mem);
    }
};

bool is_dev(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ffspmv_status upload_csr(long long nrows, long long nnz, const long long *ptr, const int *col,
                         const u32 *val, DevCSR &d)
{
    if (is_dev(ptr) && (nnz == 0 || (is_dev(col) && is_dev(val)))) {
        d.ptr = ptr;
        d.col = col;
        d.val = val;
        return FFSPMV_OK;
    }
    const size_t bp = ((size_t)(nrows + 1) * 8 + 255) / 256 * 256, bc = ((size_t)nnz * 4 + 255) / 256 * 256;
    if (cudaMalloc(&d.mem, bp + 2 * bc + 256) != cudaSuccess) {
        d.mem = nullptr;
        return FFSPMV_ERR_OOM;
    }
    char *b = (char *)d.mem;
    FF_CUDA(cudaMemcpy(b, ptr, (size_t)(nrows + 1) * 8, cudaMemcpyHostToDevice));
    if (nnz) {
        FF_CUDA(cudaMemcpy(b + bp, col, (size_t)nnz * 4, cudaMemcpyHostToDevice));
        FF_CUDA(cudaMemcpy(b + bp + bc, val, (size_t)nnz * 4, cudaMemcpyHostToDevice));
    }
    d.ptr = (const long long *)b;
    d.col = (const int *)(b + bp);
    d.val = (const u32 *)(b + bp + bc);
    return FFSPMV_OK;
}

ffspmv_status features_device(long long nrows, long long ncols, const long long *ptr, const int *col,
                              const u32 *val, u32 m, float *feat, float *binfeat, cudaStream_t st)
{
    const long long nd = nrows + ncols > 1 ? nrows + ncols - 1 : 1;
    void *scratch = nullptr;
    const size_t ab = (sizeof(FeatAcc) + 255) / 256 * 256;
    if (cudaMalloc(&scratch, ab + (size_t)nd * 4) != cudaSuccess) return FFSPMV_ERR_OOM;
    FeatAcc *acc = (FeatAcc *)scratch;
    unsigned *hist = (unsigned *)((char *)scratch + ab);
    ffspmv_status rs = FFSPMV_OK;
    do {
        if (cudaMemsetAsync(scratch, 0, ab + (size_t)nd * 4, st) != cudaSuccess) { rs = FFSPMV_ERR_CUDA; break; }
        if (nrows > 0) {
            const long long warps = std::min<long long>(nrows, 152LL * 64);
            k_features_rows<<<blocks_for(warps * 32, 256), 256, 0, st>>>(nrows, ncols, ptr, col, val, m,
                                                                         hist, acc);
            k_features_diag<<<std::min<unsigned>(blocks_for(nd, 256), 152u * 8), 256, 0, st>>>(nrows, ncols,
                                                                                              hist, acc);
        }
        k_features_final<<<1, 32, 0, st>>>(nrows, ncols, m, acc, feat, binfeat);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rs = FFSPMV_ERR_CUDA;
    } while (0);
    cudaFree(scratch);
    return rs;
}

// Bin occupancy on the host: max row length per bin and whether it holds +-1.
void bin_stats(long long nrows, const long long *ptr, const u32 *val, u32 m,
               std::vector<long long> &maxlen, std::vector<long long> &rows, std::vector<long long> &pm)
{
    maxlen.assign(kBins, 0);
    rows.assign(kBins, 0);
    pm.assign(kBins, 0);
    for (long long i = 0; i < nrows; ++i) {
        const long long L = ptr[i + 1] - ptr[i];
        const int b = bin_of_length(L);
        rows[b]++;
        maxlen[b] = std::max(maxlen[b], L);
        for (long long k = ptr[i]; k < ptr[i + 1]; ++k) {
            const u32 v = val[k] % m;
            pm[b] += v == 1u || (m > 2u && v == m - 1u);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// The exhaustive search.
ffspmv_status tune_bins(long long nrows, long long ncols, const long long *ptr, const int *col,
                        const u32 *val, u32 m, int max_rows, long long max_nnz, int reps,
                        float *times, float *pm_times, long long *sample_nnz, int *best)
{
    const float nanv = std::nanf("");
    for (int i = 0; i < kBins * kFormats; ++i) times[i] = nanv;
    for (int i = 0; i < kBins * 2; ++i) pm_times[i] = nanv;
    for (int b = 0; b < kBins; ++b) {
        sample_nnz[b] = 0;
        best[3 * b] = 0;
        best[3 * b + 1] = 0;
        best[3 * b + 2] = 0;
    }
    std::vector<std::vector<u32>> rows(kBins);
    for (long long i = 0; i < nrows; ++i) rows[bin_of_length(ptr[i + 1] - ptr[i])].push_back((u32)i);
    PlanSource *src = make_source(nrows, ncols, ptr, col, val, m);
    u32 *x = nullptr, *y = nullptr;
    ffspmv_status rs = FFSPMV_OK;
    if (cudaMalloc(&x, (size_t)std::max<long long>(ncols, 1) * 4) != cudaSuccess ||
        cudaMalloc(&y, (size_t)std::max<long long>(nrows, 1) * 4) != cudaSuccess) {
        rs = FFSPMV_ERR_OOM;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rs == FFSPMV_OK) {
        cudaMemset(x, 0, (size_t)std::max<long long>(ncols, 1) * 4);  // x = 0 < m: a valid input
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    auto time_plan = [&](const std::vector<u32> &r, const BinChoice &c, float *ms) -> ffspmv_status {
        Plan P;
        ffspmv_status s = build_rows_plan(P, *src, r, c);
        if (s != FFSPMV_OK) {
            free_plan(P);
            return s;
        }
        for (int w = 0; w < 2; ++w) run_plan(P, x, 1, y, 1, 1, m, 1, 0, st);
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps; ++k) run_plan(P, x, 1, y, 1, 1, m, 1, 0, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            free_plan(P);
            return FFSPMV_ERR_CUDA;
        }
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= (float)reps;
        free_plan(P);
        return FFSPMV_OK;
    };
    for (int b = 1; b < kBins && rs == FFSPMV_OK; ++b) {
        if (rows[b].empty()) continue;
        // evenly spaced sample of at most max_rows rows and about max_nnz entries
        std::vector<u32> smp;
        const long long nb = (long long)rows[b].size();
        long long want = std::min<long long>(nb, max_rows);
        long long avg = 0;
        for (u32 i : rows[b]) avg += ptr[i + 1] - ptr[i];
        avg = avg / nb + 1;
        want = std::max<long long>(1, std::min<long long>(want, max_nnz / avg + 1));
        for (long long k = 0; k < want; ++k) smp.push_back(rows[b][(size_t)(k * nb / want)]);
        long long maxlen = 0, snnz = 0, spm = 0;
        for (u32 i : smp) {
            maxlen = std::max(maxlen, ptr[i + 1] - ptr[i]);
            snnz += ptr[i + 1] - ptr[i];
            for (long long k = ptr[i]; k < ptr[i + 1]; ++k) {
                const u32 v = val[k] % m;
                spm += v == 1u || (m > 2u && v == m - 1u);
            }
        }
        sample_nnz[b] = snnz;
        int fbest = -1;
        float tbest = 0;
        for (int f = 0; f < kFormats; ++f) {
            if (!format_valid(f, b, maxlen)) continue;
            float ms = 0;
            ffspmv_status s = time_plan(smp, format_choice(f, 0), &ms);
            if (s == FFSPMV_ERR_CUDA) {
                rs = s;
                break;
            }
            if (s != FFSPMV_OK) continue;
            times[b * kFormats + f] = ms;
            if (fbest < 0 || ms < tbest) {
                fbest = f;
                tbest = ms;
            }
        }
        if (fbest < 0 || rs != FFSPMV_OK) continue;
        best[3 * b] = fbest;
        best[3 * b + 2] = 1;
        pm_times[2 * b] = tbest;
        if (spm > 0) {
            float ms = 0;
            if (time_plan(smp, format_choice(fbest, 1), &ms) == FFSPMV_OK) {
                pm_times[2 * b + 1] = ms;
                if (ms < tbest) best[3 * b + 1] = 1;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (x) cudaFree(x);
    if (y) cudaFree(y);
    free_source(src);
    return rs;
}

ffspmv_status selector_choose(long long nrows, long long ncols, long long nnz, const long long *hptr,
                              const int *hcol, const u32 *hval, u32 m, int *best, int *layout, int *alt = nullptr)
{
    std::vector<float> w;
    {
        std::lock_guard<std::mutex> lk(g_sel_mu);
        w = g_sel_host;
    }
    if (w.size() != (size_t)FFSPMV_MLP_PARAMS) return FFSPMV_ERR_UNSUPPORTED;
    DevCSR d;
    ffspmv_status rs = upload_csr(nrows, nnz, hptr, hcol, hval, d);
    if (rs != FFSPMV_OK) return rs;
    float *buf = nullptr;
    constexpr int kRows = kBins + 1;  // the bins, then the matrix-level input
    const size_t nf = FFSPMV_MLP_PARAMS + FFSPMV_NUM_FEATURES + kBins * FFSPMV_NUM_BIN_FEATURES +
                      kRows * kIn + kRows * 2 * kH + kRows * kOut;
    if (cudaMalloc(&buf, nf * sizeof(float)) != cudaSuccess) return FFSPMV_ERR_OOM;
    float *P = buf, *feat = P + FFSPMV_MLP_PARAMS, *binf = feat + FFSPMV_NUM_FEATURES;
    float *in = binf + kBins * FFSPMV_NUM_BIN_FEATURES, *act = in + kRows * kIn, *out = act + kRows * 2 * kH;
    std::vector<float> hout(kRows * kOut);
    do {
        if (cudaMemcpy(P, w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) { rs = FFSPMV_ERR_CUDA; break; }
        if ((rs = features_device(nrows, ncols, d.ptr, d.col, d.val, m, feat, binf, nullptr)) != FFSPMV_OK) break;
        k_selector_inputs<<<kRows, 32>>>(feat, binf, in);
        if ((rs = mlp_forward(P, in, kRows, act, out, nullptr)) != FFSPMV_OK) break;
        if (cudaMemcpy(hout.data(), out, hout.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rs = FFSPMV_ERR_CUDA;
    } while (0);
    cudaFree(buf);
    if (rs != FFSPMV_OK) return rs;
    // host CSR for bin occupancy (the input may be device memory)
    std::vector<long long> tptr;
    std::vector<u32> tval;
    const long long *pp = hptr;
    const u32 *vv = hval;
    if (is_dev(hptr)) {
        tptr.resize(nrows + 1);
        tval.resize(nnz);
        cudaMemcpy(tptr.data(), hptr, (nrows + 1) * 8, cudaMemcpyDeviceToHost);
        if (nnz) cudaMemcpy(tval.data(), hval, nnz * 4, cudaMemcpyDeviceToHost);
        pp = tptr.data();
        vv = tval.data();
    }
    std::vector<long long> maxlen, rows, pm;
    bin_stats(nrows, pp, vv, m, maxlen, rows, pm);
    for (int b = 0; b < kBins; ++b) {
        best[3 * b] = 0;
        best[3 * b + 1] = 0;
        best[3 * b + 2] = 0;
        if (b == 0 || rows[b] == 0) continue;
        int fb = -1;
        for (int f = 0; f < kFormats; ++f)
            if (format_valid(f, b, maxlen[b]) && (fb < 0 || hout[b * kOut + f] < hout[b * kOut + fb])) fb = f;
        if (fb < 0) continue;
        best[3 * b] = fb;
        best[3 * b + 1] = (pm[b] > 0 && hout[b * kOut + FFSPMV_OUT_PM] < 0.f) ? 1 : 0;
        best[3 * b + 2] = 1;
    }
    if (layout) {
        // least predicted whole-plan time, relative to the heuristic binned
        // plan (0), between the two families: x-panel (a cluster size only
        // past FFSPMV_SEL_Q_MARGIN) and binned (the network's own table only
        // past FFSPMV_SEL_NET_MARGIN)
        const float *o = &hout[kBins * kOut];
        int kq = 0;
        for (int k = 1; k < 3; ++k)
            if (o[FFSPMV_OUT_PANEL + k] < o[FFSPMV_OUT_PANEL + kq]) kq = k;
        float second = 1e30f;
        for (int k = 0; k < 3; ++k)
            if (k != kq) second = fminf(second, o[FFSPMV_OUT_PANEL + k]);
        const float vp = o[FFSPMV_OUT_PANEL + kq];
        const int lp = second - vp > FFSPMV_SEL_Q_MARGIN ? FFSPMV_LAYOUT_PANEL_Q1 + kq : FFSPMV_LAYOUT_PANEL;
        const bool net = o[FFSPMV_OUT_NETBINS] < -FFSPMV_SEL_NET_MARGIN;
        const float vb = net ? o[FFSPMV_OUT_NETBINS] : 0.f;
        const int lb = net ? FFSPMV_LAYOUT_NETBINS : FFSPMV_LAYOUT_BINNED;
        *layout = vp < vb ? lp : lb;
        if (alt) *alt = fabsf(vp - vb) < FFSPMV_SEL_VERIFY_MARGIN ? (vp < vb ? lb : lp) : -1;
    }
    return FFSPMV_OK;
}

ffspmv_status choose_bins(int selector, long long nrows, long long ncols, const long long *ptr,
                          const int *col, const u32 *val, u32 m, const ffspmv_options &o,
                          BinChoice *bins, int *layout, int *alt)
{
    const long long nnz = ptr[nrows];
    std::vector<int> best(3 * kBins, 0);
    ffspmv_status rs = FFSPMV_ERR_UNSUPPORTED;
    if (layout) *layout = -1;
    if (alt) *alt = -1;
    if (selector == FFSPMV_SEL_LEARNED)
        rs = selector_choose(nrows, ncols, nnz, ptr, col, val, m, best.data(), layout, alt);
    if (rs == FFSPMV_ERR_UNSUPPORTED || selector == FFSPMV_SEL_EXHAUSTIVE) {
        std::vector<float> t(kBins * kFormats), pt(kBins * 2);
        std::vector<long long> sn(kBins);
        rs = tune_bins(nrows, ncols, ptr, col, val, m, 16384, 1LL << 21, 5, t.data(), pt.data(),
                       sn.data(), best.data());
    }
    if (rs != FFSPMV_OK) return rs;
    std::vector<long long> maxlen, rows, pm;
    bin_stats(nrows, ptr, val, m, maxlen, rows, pm);
    for (int b = 0; b < kBins; ++b) {
        if (best[3 * b + 2]) {
            bins[b] = format_choice(best[3 * b], best[3 * b + 1]);
        } else {
            bins[b] = heuristic_bin_choice(b, 0.0, o.use_pm1);
        }
    }
    return FFSPMV_OK;
}

}  // namespace ff

using namespace ff;

extern "C" {

ffspmv_status ffspmv_matrix_features(int64_t nrows, int64_t ncols, const int64_t *d_row_ptr,
                                     const int32_t *d_col, const uint32_t *d_values, uint32_t modulus,
                                     float *d_feat, float *d_binfeat, ffspmv_stream_t stream)
{
    if (nrows < 0 || ncols < 0 || !d_row_ptr || !d_feat || !d_binfeat || modulus < 2u) return FFSPMV_ERR_ARG;
    return features_device(nrows, ncols, (const long long *)d_row_ptr, d_col, d_values, modulus, d_feat,
                           d_binfeat, (cudaStream_t)stream);
}

ffspmv_status ffspmv_tune_bins(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row_ptr,
                               const int32_t *col, const uint32_t *values, uint32_t modulus,
                               int32_t max_rows, int64_t max_nnz, int32_t reps, float *times,
                               float *pm_times, int64_t *sample_nnz, int32_t *best)
{
    if (nrows < 0 || ncols < 0 || nnz < 0 || !row_ptr || modulus < 2u || max_rows < 1 || max_nnz < 1 ||
        reps < 1 || !times || !pm_times || !sample_nnz || !best)
        return FFSPMV_ERR_ARG;
    if (nnz > 0 && (!col || !values)) return FFSPMV_ERR_ARG;
    std::vector<long long> hp;
    std::vector<int> hc;
    std::vector<u32> hv;
    const long long *p = (const long long *)row_ptr;
    const int *c = col;
    const u32 *v = values;
    if (is_dev(row_ptr)) {
        hp.resize(nrows + 1);
        hc.resize(nnz);
        hv.resize(nnz);
        FF_CUDA(cudaMemcpy(hp.data(), row_ptr, (nrows + 1) * 8, cudaMemcpyDeviceToHost));
        if (nnz) {
            FF_CUDA(cudaMemcpy(hc.data(), col, nnz * 4, cudaMemcpyDeviceToHost));
            FF_CUDA(cudaMemcpy(hv.data(), values, nnz * 4, cudaMemcpyDeviceToHost));
        }
        p = hp.data();
        c = hc.data();
        v = hv.data();
    }
    return tune_bins(nrows, ncols, p, c, v, modulus, max_rows, max_nnz, reps, times, pm_times,
                     (long long *)sample_nnz, best);
}

ffspmv_status ffspmv_mlp_forward(const float *d_params, const float *d_in, int32_t batch, float *d_act,
                                 float *d_out, ffspmv_stream_t stream)
{
    if (!d_params || !d_in || !d_act || !d_out || batch < 0) return FFSPMV_ERR_ARG;
    return mlp_forward(d_params, d_in, batch, d_act, d_out, (cudaStream_t)stream);
}

ffspmv_status ffspmv_mlp_loss(const float *d_out, const float *d_target, const float *d_mask, int32_t batch,
                              float *d_dout, float *d_loss, ffspmv_stream_t stream)
{
    if (!d_out || !d_target || !d_mask || !d_dout || !d_loss || batch < 0) return FFSPMV_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long n = (long long)batch * kOut;
    float *cnt = d_loss;  // the count is formed in d_loss[0] and then replaced by the loss
    float *tmp = nullptr;
    if (cudaMallocAsync((void **)&tmp, sizeof(float), st) != cudaSuccess) return FFSPMV_ERR_OOM;
    FF_CUDA(cudaMemsetAsync(tmp, 0, sizeof(float), st));
    FF_CUDA(cudaMemsetAsync(cnt, 0, sizeof(float), st));
    const unsigned nb = std::max(1u, std::min(blocks_for(n, 256), 1024u));
    k_mask_sum<<<nb, 256, 0, st>>>(d_mask, n, tmp);
    k_loss_grad<<<nb, 256, 0, st>>>(d_out, d_target, d_mask, n, tmp, d_dout, cnt);
    FF_CUDA(cudaGetLastError());
    FF_CUDA(cudaFreeAsync(tmp, st));
    return FFSPMV_OK;
}

ffspmv_status ffspmv_mlp_backward(const float *d_params, const float *d_in, int32_t batch, const float *d_act,
                                  const float *d_dout, float *d_grad, ffspmv_stream_t stream)
{
    if (!d_params || !d_in || !d_act || !d_dout || !d_grad || batch < 1) return FFSPMV_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const float *P = d_params;
    float *G = d_grad;
    float *dz = nullptr;  // [batch][2H]: dz2 then dz1
    if (cudaMallocAsync((void **)&dz, (size_t)batch * 2 * kH * sizeof(float), st) != cudaSuccess)
        return FFSPMV_ERR_OOM;
    const float *h1 = d_act, *h2 = d_act + kH;
    // layer 3
    k_grad_w<<<kOut, kH + 1, 0, st>>>(d_dout, kOut, h2, 2 * kH, batch, kH, G + kOffW3, G + kOffB3);
    k_grad_in<<<blocks_for((long long)batch * kH, 256), 256, 0, st>>>(P + kOffW3, d_dout, kOut, h2, 2 * kH,
                                                                      batch, kH, kOut, dz + kH, 2 * kH);
    // layer 2
    k_grad_w<<<kH, kH + 1, 0, st>>>(dz + kH, 2 * kH, h1, 2 * kH, batch, kH, G + kOffW2, G + kOffB2);
    k_grad_in<<<blocks_for((long long)batch * kH, 256), 256, 0, st>>>(P + kOffW2, dz + kH, 2 * kH, h1, 2 * kH,
                                                                      batch, kH, kH, dz, 2 * kH);
    // layer 1
    k_grad_w<<<kH, kIn + 1, 0, st>>>(dz, 2 * kH, d_in, kIn, batch, kIn, G + kOffW1, G + kOffB1);
    FF_CUDA(cudaGetLastError());
    FF_CUDA(cudaFreeAsync(dz, st));
    return FFSPMV_OK;
}

ffspmv_status ffspmv_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, int32_t step,
                              float lr, float beta1, float beta2, float eps, ffspmv_stream_t stream)
{
    if (!d_params || !d_grad || !d_m || !d_v || step < 1) return FFSPMV_ERR_ARG;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<blocks_for(FFSPMV_MLP_PARAMS, 256), 256, 0, (cudaStream_t)stream>>>(
        d_params, d_grad, d_m, d_v, FFSPMV_MLP_PARAMS, lr, beta1, beta2, eps, c1, c2);
    FF_CUDA(cudaGetLastError());
    return FFSPMV_OK;
}

ffspmv_status ffspmv_selector_load(const float *params, int64_t count)
{
    std::lock_guard<std::mutex> lk(g_sel_mu);
    if (!params) {
        g_sel_host.clear();
        return FFSPMV_OK;
    }
    if (count != FFSPMV_MLP_PARAMS) return FFSPMV_ERR_ARG;
    g_sel_host.assign(params, params + count);
    return FFSPMV_OK;
}

ffspmv_status ffspmv_heuristic_choose(int64_t nrows, const int64_t *row_ptr, const uint32_t *values,
                                      uint32_t modulus, int32_t use_pm1, int32_t *best)
{
    if (nrows < 0 || !row_ptr || !best || modulus < 2u) return FFSPMV_ERR_ARG;
    const long long *ptr = (const long long *)row_ptr;
    std::vector<long long> nnzb(kBins, 0), pmb(kBins, 0), rows(kBins, 0);
    for (long long i = 0; i < nrows; ++i) {
        const int b = bin_of_length(ptr[i + 1] - ptr[i]);
        rows[b]++;
        nnzb[b] += ptr[i + 1] - ptr[i];
        for (long long k = ptr[i]; k < ptr[i + 1]; ++k) {
            const u32 v = values[k] % modulus;
            pmb[b] += v == 1u || (modulus > 2u && v == modulus - 1u);
        }
    }
    for (int b = 0; b < kBins; ++b) {
        best[3 * b] = best[3 * b + 1] = best[3 * b + 2] = 0;
        if (b == 0 || rows[b] == 0) continue;
        const BinChoice c = heuristic_bin_choice(b, nnzb[b] ? (double)pmb[b] / nnzb[b] : 0.0, use_pm1);
        int f = 9;
        if (c.kind == SEG_ELLR) f = 0;
        else if (c.kind == SEG_CSR) { f = 1; for (int g = c.group; g > 1; g >>= 1) ++f; }
        else if (c.kind == SEG_CSRBLK) f = 7;
        else if (c.kind == SEG_CSRSPLIT) f = 8;
        best[3 * b] = f;
        best[3 * b + 1] = c.pm;
        best[3 * b + 2] = 1;
    }
    return FFSPMV_OK;
}

ffspmv_status ffspmv_selector_choose(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row_ptr,
                                     const int32_t *col, const uint32_t *values, uint32_t modulus,
                                     int32_t *best, int32_t *layout)
{
    if (nrows < 0 || ncols < 0 || nnz < 0 || !row_ptr || !best || modulus < 2u) return FFSPMV_ERR_ARG;
    return selector_choose(nrows, ncols, nnz, (const long long *)row_ptr, col, values, modulus, best, layout);
}

}  // extern "C"
