// deg det U and codeg det U of the matrix generator that a block-Wiedemann
// sigma-basis gives (Sec. 3, step 3 and Sec. 3.3, "determinant co-degree":
// the rank of a suitably preconditioned A is deg det U - codeg det U).
//
// Both are x-adic valuations of a determinant.  codeg det U = v(det U), the
// multiplicity of x in det U.  With D_r the degree of row r of U and
// U~_r(x) = x^{D_r} U_r(1/x) (row r's coefficients reversed against D_r),
// det U~(x) = x^{sum D_r} det U(1/x), so deg det U = sum D_r - v(det U~).
//
// v(det H) is read off Gaussian elimination over the power series F_p[[x]],
// truncated at x^K: in column c the entry of least valuation among the rows
// not yet used is the pivot, x^v u with u(0) != 0; every other entry a of the
// column has valuation >= v, so a / (x^v u) is a power series and
// row_r -= (a / (x^v u)) row_c changes no determinant.  The determinant is
// then the product of the pivots up to sign, and v(det H) = sum of the pivot
// valuations.  Dividing by x^v loses v coefficients, so after each pivot the
// rows are known modulo x^(prec - v); a pivot found below the precision is
// exact.  When some column has no entry known to be nonzero the precision
// was too small (or det H = 0): the elimination runs again with K doubled.
#include <algorithm>
#include <vector>

#include "ff_internal.cuh"
#include "../../include/ffspmv_sigma.h"

namespace ff {
namespace {

constexpr int kGdMaxN = 32;        // generator order (the sigma-basis takes m <= 32)
constexpr int kGdThreads = 256;
constexpr int kGdStartPrec = 32;   // first truncation order
constexpr int kGdDefaultPrec = 4096;
constexpr int kGdMaxPrec = 1 << 16;

struct GdRows {
    int r[kGdMaxN];  // physical row of each position of the elimination
};

__device__ __forceinline__ u32 mulmod(u32 a, u32 b, u32 p) { return (u32)((u64)a * b % p); }

// W[i][c][k], k < K: coefficient k of U_ic (rev = 0) or of U~_ic (rev = 1),
// U_ic = entry (sel[i], c) of the basis P ((d+1) x m x m, coefficient-major).
__global__ void k_gd_gather(const u32 *__restrict__ P, long long d, int m, int n, const int *__restrict__ sel,
                            const int *__restrict__ rowdeg, int rev, int K, u32 p, u32 *__restrict__ W)
{
    const long long total = (long long)n * n * K;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % K);
        const int c = (int)((e / K) % n);
        const int i = (int)(e / ((long long)K * n));
        const long long t = rev ? (long long)rowdeg[i] - k : (long long)k;
        u32 v = 0;
        if (t >= 0 && t <= d) v = P[(t * m + sel[i]) * m + c] % p;
        W[e] = v;
    }
}

// Degree of row sel[i] of U (columns < n): the largest t <= d with a nonzero
// coefficient, -1 for a zero row.  One CTA per row.
__global__ void k_gd_rowdeg(const u32 *__restrict__ P, long long d, int m, int n, const int *__restrict__ sel,
                            u32 p, int *__restrict__ rowdeg)
{
    __shared__ int best;
    if (threadIdx.x == 0) best = -1;
    __syncthreads();
    const int i = blockIdx.x;
    int mine = -1;
    for (long long e = threadIdx.x; e < (d + 1) * n; e += blockDim.x) {
        const long long t = e / n;
        const int c = (int)(e % n);
        if (P[(t * m + sel[i]) * m + c] % p) mine = max(mine, (int)t);
    }
    atomicMax(&best, mine);
    __syncthreads();
    if (threadIdx.x == 0) rowdeg[i] = best;
}

// Valuation (first nonzero coefficient below prec, else prec) of column c in
// the rows at positions c.. of the elimination; one CTA per position.
__global__ void k_gd_val(const u32 *__restrict__ W, int n, int K, int c, int prec, GdRows R, int *__restrict__ val)
{
    __shared__ int best;
    if (threadIdx.x == 0) best = prec;
    __syncthreads();
    const int pos = c + blockIdx.x;
    const u32 *w = W + ((long long)R.r[pos] * n + c) * K;
    int mine = prec;
    for (int k = threadIdx.x; k < prec; k += blockDim.x)
        if (w[k]) {
            mine = k;
            break;
        }
    atomicMin(&best, mine);
    __syncthreads();
    if (threadIdx.x == 0) val[blockIdx.x] = best;
}

// inv = 1 / u mod x^L, u_k = coefficient v + k of the pivot entry: inv_0 =
// u_0^(p-2) (Fermat), inv_k = -inv_0 sum_{j=1..k} u_j inv_{k-j}.  One CTA.
__global__ void k_gd_inv(const u32 *__restrict__ W, int n, int K, int c, int v, int L, GdRows R, u32 p,
                         u32 *__restrict__ inv)
{
    __shared__ u64 part[kGdThreads / 32];
    __shared__ u32 inv0;
    const u32 *u = W + ((long long)R.r[c] * n + c) * K + v;
    if (threadIdx.x == 0) {
        u32 b = u[0], e = p - 2, r = 1;
        while (e) {
            if (e & 1u) r = mulmod(r, b, p);
            b = mulmod(b, b, p);
            e >>= 1;
        }
        inv0 = r;
        inv[0] = r;
    }
    __syncthreads();
    for (int k = 1; k < L; ++k) {
        u64 s = 0;  // below L 2^31 < 2^47
        for (int j = 1 + threadIdx.x; j <= k; j += blockDim.x) s += mulmod(u[j], inv[k - j], p);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            u64 t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
            inv[k] = mulmod(inv0, (p - (u32)(t % p)) % p, p);
        }
        __syncthreads();
    }
}

// f_pos = (entry (pos, c) / x^v) * inv mod x^L for the positions below c
// (CTA b: position c + 1 + b).
__global__ void k_gd_factor(const u32 *__restrict__ W, int n, int K, int c, int v, int L, GdRows R, u32 p,
                            const u32 *__restrict__ inv, u32 *__restrict__ F)
{
    const int pos = c + 1 + blockIdx.x;
    const u32 *a = W + ((long long)R.r[pos] * n + c) * K + v;
    u32 *f = F + (long long)pos * K;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        u64 s = 0;
        for (int j = 0; j <= k; ++j) s += mulmod(a[j], inv[k - j], p);
        f[k] = (u32)(s % p);
    }
}

// row_pos -= f_pos row_c (columns > c, coefficients < L); CTA (b, j): position
// c + 1 + b, column c + 1 + j.
__global__ void k_gd_update(u32 *__restrict__ W, int n, int K, int c, int L, GdRows R, u32 p,
                            const u32 *__restrict__ F)
{
    const int w = n - c - 1;
    const int pos = c + 1 + blockIdx.x / w, col = c + 1 + blockIdx.x % w;
    u32 *t = W + ((long long)R.r[pos] * n + col) * K;
    const u32 *q = W + ((long long)R.r[c] * n + col) * K;
    const u32 *f = F + (long long)pos * K;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        u64 s = 0;
        for (int j = 0; j <= k; ++j) s += mulmod(f[j], q[k - j], p);
        t[k] = (u32)(((u64)t[k] + p - (u32)(s % p)) % p);
    }
}

// deterministic Miller-Rabin for q < 2^32 with bases 2, 3, 5, 7 (enough below
// 3 215 031 751; larger q also get base 11)
bool gd_prime(u64 q)
{
    if (q < 2) return false;
    const u64 small[] = {2, 3, 5, 7, 11};
    for (u64 b : small)
        if (q % b == 0) return q == b;
    u64 dd = q - 1;
    int s = 0;
    while (!(dd & 1)) {
        dd >>= 1;
        ++s;
    }
    for (u64 a : small) {
        u64 x = 1, b = a % q, e = dd;
        while (e) {
            if (e & 1) x = x * b % q;
            b = b * b % q;
            e >>= 1;
        }
        if (x == 1 || x == q - 1) continue;
        bool comp = true;
        for (int r = 1; r < s && comp; ++r) {
            x = x * x % q;
            if (x == q - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

struct GdRun {
    u32 p = 0;
    int m = 0, n = 0;
    long long d = 0;
    const u32 *P = nullptr;
    int *d_sel = nullptr, *d_rowdeg = nullptr, *d_val = nullptr;
    u32 *W = nullptr, *F = nullptr, *inv = nullptr;
    int cap = 0;  // precision the buffers hold
    cudaStream_t st = nullptr;
};

// v(det) of U (rev = 0) or U~ (rev = 1) at precision K; *ok = false when a
// column had no entry known to be nonzero.
ffspmv_status gd_valuation(GdRun &G, int rev, int K, long long *out, bool *ok)
{
    const int n = G.n;
    const long long total = (long long)n * n * K;
    const unsigned gb = (unsigned)std::min<long long>((total + kGdThreads - 1) / kGdThreads, 4096);
    k_gd_gather<<<gb, kGdThreads, 0, G.st>>>(G.P, G.d, G.m, n, G.d_sel, G.d_rowdeg, rev, K, G.p, G.W);
    FF_CUDA(cudaGetLastError());
    GdRows R;
    for (int i = 0; i < kGdMaxN; ++i) R.r[i] = i < n ? i : 0;
    int prec = K;
    long long sum = 0;
    std::vector<int> val(n);
    *ok = false;
    for (int c = 0; c < n; ++c) {
        k_gd_val<<<n - c, kGdThreads, 0, G.st>>>(G.W, n, K, c, prec, R, G.d_val);
        FF_CUDA(cudaGetLastError());
        FF_CUDA(cudaMemcpyAsync(val.data(), G.d_val, sizeof(int) * (n - c), cudaMemcpyDeviceToHost, G.st));
        FF_CUDA(cudaStreamSynchronize(G.st));
        int b = 0;
        for (int i = 1; i < n - c; ++i)
            if (val[i] < val[b]) b = i;
        const int v = val[b];
        if (v >= prec) return FFSPMV_OK;  // precision too small (or det = 0)
        std::swap(R.r[c], R.r[c + b]);
        sum += v;
        const int L = prec - v;
        if (c + 1 < n) {
            k_gd_inv<<<1, kGdThreads, 0, G.st>>>(G.W, n, K, c, v, L, R, G.p, G.inv);
            FF_CUDA(cudaGetLastError());
            k_gd_factor<<<n - c - 1, kGdThreads, 0, G.st>>>(G.W, n, K, c, v, L, R, G.p, G.inv, G.F);
            FF_CUDA(cudaGetLastError());
            k_gd_update<<<(n - c - 1) * (n - c - 1), kGdThreads, 0, G.st>>>(G.W, n, K, c, L, R, G.p, G.F);
            FF_CUDA(cudaGetLastError());
        }
        prec = L;
    }
    *ok = true;
    *out = sum;
    return FFSPMV_OK;
}

void gd_free(GdRun &G)
{
    cudaFree(G.d_sel);
    cudaFree(G.W);
    G.d_sel = nullptr;
    G.W = nullptr;
}

ffspmv_status gd_alloc(GdRun &G, int K)
{
    gd_free(G);
    const size_t ints = 3 * (size_t)kGdMaxN * sizeof(int);
    if (cudaMalloc(&G.d_sel, ints) != cudaSuccess) {
        cudaGetLastError();
        G.d_sel = nullptr;
        return FFSPMV_ERR_OOM;
    }
    G.d_rowdeg = G.d_sel + kGdMaxN;
    G.d_val = G.d_sel + 2 * kGdMaxN;
    const size_t words = (size_t)G.n * G.n * K + (size_t)G.n * K + (size_t)K;
    if (cudaMalloc(&G.W, words * sizeof(u32)) != cudaSuccess) {
        cudaGetLastError();
        G.W = nullptr;
        return FFSPMV_ERR_OOM;
    }
    G.F = G.W + (size_t)G.n * G.n * K;
    G.inv = G.F + (size_t)G.n * K;
    G.cap = K;
    return FFSPMV_OK;
}

// The valuation at the smallest doubling of kGdStartPrec that determines it.
ffspmv_status gd_valuation_auto(GdRun &G, int rev, int max_prec, const std::vector<int> &sel,
                                const std::vector<int> &rowdeg, long long *out)
{
    for (int K = std::min(kGdStartPrec, max_prec);; K = std::min(2 * K, max_prec)) {
        if (K > G.cap) {
            ffspmv_status s = gd_alloc(G, K);
            if (s != FFSPMV_OK) return s;
            FF_CUDA(cudaMemcpyAsync(G.d_sel, sel.data(), sizeof(int) * G.n, cudaMemcpyHostToDevice, G.st));
            FF_CUDA(cudaMemcpyAsync(G.d_rowdeg, rowdeg.data(), sizeof(int) * G.n, cudaMemcpyHostToDevice, G.st));
        }
        bool ok = false;
        ffspmv_status s = gd_valuation(G, rev, K, out, &ok);
        if (s != FFSPMV_OK) return s;
        if (ok) return FFSPMV_OK;
        if (K >= max_prec) return FFSPMV_ERR_UNSUPPORTED;
    }
}

}  // namespace
}  // namespace ff

using namespace ff;

extern "C" ffspmv_status sigma_generator_degrees(uint32_t p, int32_t m, int32_t n, int64_t d, const uint32_t *d_P,
                                                 const int32_t *h_delta, int32_t max_precision, int64_t *h_deg,
                                                 int64_t *h_codeg, ffspmv_stream_t stream)
{
    if (p < 2 || p > (1u << 31) || !gd_prime(p) || n < 1 || m < n || m > kGdMaxN || d < 0 || !d_P || !h_delta ||
        !h_deg || !h_codeg || max_precision < 0 || max_precision > kGdMaxPrec)
        return FFSPMV_ERR_ARG;
    const int max_prec = max_precision ? max_precision : kGdDefaultPrec;
    // the generator: the n rows of least (delta_i, i)
    std::vector<int> order(m);
    for (int i = 0; i < m; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h_delta[a] < h_delta[b]; });
    std::vector<int> sel(order.begin(), order.begin() + n);
    GdRun G;
    G.p = p;
    G.m = m;
    G.n = n;
    G.d = d;
    G.P = d_P;
    G.st = (cudaStream_t)stream;
    ffspmv_status s = gd_alloc(G, std::min(kGdStartPrec, max_prec));
    if (s != FFSPMV_OK) {
        gd_free(G);
        return s;
    }
    std::vector<int> rowdeg(n);
    auto run = [&]() -> ffspmv_status {
        FF_CUDA(cudaMemcpyAsync(G.d_sel, sel.data(), sizeof(int) * n, cudaMemcpyHostToDevice, G.st));
        k_gd_rowdeg<<<n, kGdThreads, 0, G.st>>>(d_P, d, m, n, G.d_sel, p, G.d_rowdeg);
        FF_CUDA(cudaGetLastError());
        FF_CUDA(cudaMemcpyAsync(rowdeg.data(), G.d_rowdeg, sizeof(int) * n, cudaMemcpyDeviceToHost, G.st));
        FF_CUDA(cudaStreamSynchronize(G.st));
        long long dsum = 0;
        for (int i = 0; i < n; ++i) {
            if (rowdeg[i] < 0) return FFSPMV_ERR_UNSUPPORTED;  // a zero row: det U = 0
            dsum += rowdeg[i];
        }
        long long codeg = 0, vrev = 0;
        ffspmv_status r = gd_valuation_auto(G, 0, max_prec, sel, rowdeg, &codeg);
        if (r != FFSPMV_OK) return r;
        r = gd_valuation_auto(G, 1, max_prec, sel, rowdeg, &vrev);
        if (r != FFSPMV_OK) return r;
        *h_codeg = codeg;
        *h_deg = dsum - vrev;
        return FFSPMV_OK;
    };
    s = run();
    gd_free(G);
    return s;
}
