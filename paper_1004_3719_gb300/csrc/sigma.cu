// Sigma-bases over F_p for the second step of block Wiedemann (Sec. 3.2,
// "Parallelization of the sigma-basis computation"): PM-Basis (Giorgi,
// Jeannerod and Villard, ISSAC 2003) as a host recursion on the order whose
// work is polynomial-matrix products on the GPU (polymat_mul, Sec. 3.2.1's
// evaluation / pointwise / interpolation scheme), and M-Basis, the iterative
// algorithm Sec. 3.2.2 recommends at small orders, as one CTA per leaf.
//
// M-Basis leaf.  For an order-d problem (d <= 32) the CTA keeps in shared
// memory the residual R = P F (coefficients k..d-1, m x n each) and the basis
// P (coefficients 0..k, m x m).  At order k one warp eliminates the m x n
// matrix R_k column by column (rows ordered by (delta_i, i), pivot = the
// first non-pivot row nonzero in the column); the whole CTA then applies the
// same row operations to every coefficient of R and P, one thread per
// (coefficient, column) position and thread-local in it, and multiplies the
// pivot rows by x.  The elimination is fraction free -- row r becomes
// a r - b q with a the pivot's entry and b row r's entry -- so no inverse is
// taken inside the loop; each row of P is then a known nonzero multiple c_r
// of the row that the elimination with division gives, and one inversion per
// row at the end of the leaf divides it out, which makes the result the same
// as the plain algorithm's.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "ff_internal.cuh"
#include "ffspmv_polymat.h"
#include "ffspmv_sigma.h"

namespace ff {
namespace {

constexpr int kSbMaxM = 32;                 // rows of F and of P (the polynomial-matrix product's limit)
constexpr int kSbMaxBase = 32;              // largest leaf order
constexpr int kSbThreads = 512;
constexpr size_t kSbSmemMax = 227 * 1024;
constexpr size_t kSbAlign = 256;
constexpr int kSbMaxShift = 1 << 24;

struct SbLeaf {
    const u32 *F;   // d x m x ldf, columns < n used
    u32 *P;         // out: (d+1) x m x m
    int *delta;     // out: m
    int shift[kSbMaxM];
    int m, n, d, ldf;
    Mod M;
};

// shared memory of one leaf: R (d x m x n), P ((d+1) x m x m), the column
// operations (multiplier and addend pairs, kSbMaxM x kSbMaxM), pivots, degrees,
// pivot flags and the inverse row scales
// words before the op table: R and P, rounded up to an even count so that the
// 8-byte pairs are aligned
__host__ __device__ inline size_t sb_op_offset(int m, int n, long long d)
{
    return ((size_t)d * m * n + (size_t)(d + 1) * m * m + 1) & ~(size_t)1;
}

size_t sb_leaf_smem(int m, int n, long long d)
{
    return (sb_op_offset(m, n, d) + 2 * kSbMaxM * kSbMaxM + 4 * kSbMaxM) * 4;
}

__device__ u32 sb_pow(u32 a, u32 e, const Mod &M)
{
    u32 r = 1u % M.m;
    while (e) {
        if (e & 1u) r = red64((u64)r * a, M);
        a = red64((u64)a * a, M);
        e >>= 1;
    }
    return r;
}

__global__ void __launch_bounds__(kSbThreads, 1) k_sb_mbasis(const __grid_constant__ SbLeaf a)
{
    extern __shared__ __align__(16) u32 sb_sm[];
    const int m = a.m, n = a.n, d = a.d;
    const u32 p = a.M.m;
    u32 *R = sb_sm;                                   // R[t][i][j] at (t m + i) n + j
    u32 *P = R + (size_t)d * m * n;                   // P[t][i][l] at (t m + i) m + l
    uint2 *sop = reinterpret_cast<uint2 *>(sb_sm + sb_op_offset(m, n, d));  // (multiplier, addend) of row r at column j: sop[j][r]
    int *spiv = (int *)(sop + kSbMaxM * kSbMaxM);     // pivot row of column j, -1 if none
    int *sdelta = spiv + kSbMaxM;
    int *sisp = sdelta + kSbMaxM;                     // row is a pivot at this order
    u32 *sinv = (u32 *)(sisp + kSbMaxM);              // 1 / c_r
    const int tid = threadIdx.x;

    for (long long i = tid; i < (long long)d * m * n; i += blockDim.x) {
        const long long t = i / ((long long)m * n);
        const int r = (int)((i / n) % m), c = (int)(i % n);
        R[i] = red64(a.F[((size_t)t * m + r) * a.ldf + c], a.M);
    }
    for (long long i = tid; i < (long long)(d + 1) * m * m; i += blockDim.x) P[i] = 0;
    __syncthreads();
    if (tid < m) {
        P[(size_t)tid * m + tid] = 1u;
        sdelta[tid] = a.shift[tid];
    }
    __syncthreads();

    u32 cs = 1u;   // warp 0, lane r < m: c_r, the product of the multipliers applied to row r
    for (int k = 0; k < d; ++k) {
        if (tid < 32) {
            // lane c holds column c of R_k; every lane holds the order positions
            // of all rows; rows are indexed by constants only (registers)
            const int lane = tid;
            const int dl = lane < m ? sdelta[lane] : INT_MAX;
            int myrank = 0;   // position of row `lane` in the order by (delta, index)
#pragma unroll
            for (int j = 0; j < kSbMaxM; ++j) {
                const int dj = __shfl_sync(0xffffffffu, dl, j);
                myrank += (j < m && (dj < dl || (dj == dl && j < lane))) ? 1 : 0;
            }
            int rk[kSbMaxM];
            u32 v[kSbMaxM];
#pragma unroll
            for (int r = 0; r < kSbMaxM; ++r) {
                rk[r] = __shfl_sync(0xffffffffu, myrank, r);
                v[r] = (r < m && lane < n) ? R[((size_t)k * m + r) * n + lane] : 0u;
            }
            u32 pivots = 0u;   // bit r: row r is a pivot at this order
            for (int j = 0; j < n; ++j) {
                // lane j: the first row in the order, not yet a pivot, nonzero in column j
                int best = 64, q = -1;
#pragma unroll
                for (int r = 0; r < kSbMaxM; ++r) {
                    if (r < m && !((pivots >> r) & 1u) && v[r] != 0u && rk[r] < best) {
                        best = rk[r];
                        q = r;
                    }
                }
                q = __shfl_sync(0xffffffffu, q, j);
                best = __shfl_sync(0xffffffffu, best, j);
                if (q < 0) {   // column j is already zero in every non-pivot row
                    if (lane == 0) spiv[j] = -1;
                    continue;
                }
                u32 vq = 0u;   // this lane's entry of the pivot row
#pragma unroll
                for (int r = 0; r < kSbMaxM; ++r) vq = (r == q) ? v[r] : vq;
                const u32 av = __shfl_sync(0xffffffffu, vq, j);
                u32 gmine = 0u;   // the addend coefficient of row `lane`
#pragma unroll
                for (int r = 0; r < kSbMaxM; ++r) {
                    const u32 br = __shfl_sync(0xffffffffu, v[r], j);
                    const bool upd = r < m && !((pivots >> r) & 1u) && br != 0u && rk[r] > best;
                    const u32 g = upd ? p - br : 0u;   // nonzero exactly when row r is updated
                    if (upd && lane > j && lane < n) v[r] = red64((u64)av * v[r] + (u64)g * vq, a.M);
                    gmine = (lane == r) ? g : gmine;
                }
                if (lane < m) {
                    sop[j * kSbMaxM + lane] = make_uint2(gmine ? av : 1u, gmine);
                    if (gmine) cs = red64((u64)cs * av, a.M);
                }
                pivots |= 1u << q;
                if (lane == 0) spiv[j] = q;
            }
            if (lane < m) {
                const int ip = (pivots >> lane) & 1u;
                sisp[lane] = ip;
                if (ip) sdelta[lane] = dl + 1;
            }
        }
        __syncthreads();
        // the column operations, in order, on R's coefficients k..d-1 and P's 0..k
        const int nr = (d - k) * n, np = (k + 1) * m;
        for (int pos = tid; pos < nr + np; pos += blockDim.x) {
            u32 *base;
            int stride;
            if (pos < nr) {
                base = R + ((size_t)(k + pos / n) * m) * n + (pos % n);
                stride = n;
            } else {
                const int w = pos - nr;
                base = P + ((size_t)(w / m) * m) * m + (w % m);
                stride = m;
            }
            u32 v[kSbMaxM];
#pragma unroll
            for (int r = 0; r < kSbMaxM; ++r) v[r] = r < m ? base[r * stride] : 0u;
            for (int j = 0; j < n; ++j) {
                const int q = spiv[j];
                if (q < 0) continue;
                u32 vq = 0u;
#pragma unroll
                for (int r = 0; r < kSbMaxM; ++r) vq = (r == q) ? v[r] : vq;
#pragma unroll
                for (int r = 0; r < kSbMaxM; ++r) {
                    if (r < m) {
                        const uint2 op = sop[j * kSbMaxM + r];
                        if (op.y) v[r] = red64((u64)op.x * v[r] + (u64)op.y * vq, a.M);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kSbMaxM; ++r)
                if (r < m) base[r * stride] = v[r];
        }
        __syncthreads();
        // pivot rows times x: R's coefficients k..d-1 and P's 0..k+1 move up by one
        for (int w = tid; w < m * (n + m); w += blockDim.x) {
            const int q = w / (n + m), c = w % (n + m);
            if (!sisp[q]) continue;
            if (c < n) {
                for (int t = d - 1; t > k; --t)
                    R[((size_t)t * m + q) * n + c] = R[((size_t)(t - 1) * m + q) * n + c];
                R[((size_t)k * m + q) * n + c] = 0u;
            } else {
                const int l = c - n;
                for (int t = k + 1; t > 0; --t)
                    P[((size_t)t * m + q) * m + l] = P[((size_t)(t - 1) * m + q) * m + l];
                P[(size_t)q * m + l] = 0u;
            }
        }
        __syncthreads();
    }
    if (tid < m) sinv[tid] = sb_pow(cs, p - 2u, a.M);   // c_r != 0 in the field F_p
    __syncthreads();
    for (long long i = tid; i < (long long)(d + 1) * m * m; i += blockDim.x) {
        const int r = (int)((i / m) % m);
        a.P[i] = red64((u64)P[i] * sinv[r], a.M);
    }
    if (tid < m) a.delta[tid] = sdelta[tid];
}

// Fp[k][i][j] = F[k][i][j] mod p for j < n, 0 for n <= j < m (square for the products)
__global__ void k_sb_pad(const u32 *__restrict__ F, long long d, int m, int n, u32 *__restrict__ Fp, const Mod M)
{
    const long long total = d * m * m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i % m);
        const long long ki = i / m;   // k m + i
        Fp[i] = j < n ? red64(F[ki * n + j], M) : 0u;
    }
}

__global__ void k_sb_wiedemann(const u32 *__restrict__ S, long long L, int s, u32 *__restrict__ F, u32 p)
{
    const long long total = L * 2 * s * s;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i % s);
        const int r = (int)((i / s) % (2 * s));
        const long long k = i / (2LL * s * s);
        u32 v;
        if (r < s) v = S[(k * s + r) * s + j];
        else v = (k == 0 && r - s == j) ? p - 1u : 0u;
        F[i] = v;
    }
}

bool sb_is_prime(u64 q)
{
    // deterministic Miller-Rabin: bases 2, 3, 5, 7 decide every q < 3 215 031 751
    if (q < 2) return false;
    for (u64 sp : {2ull, 3ull, 5ull, 7ull}) {
        if (q == sp) return true;
        if (q % sp == 0) return false;
    }
    u64 dd = q - 1;
    int r = 0;
    while (!(dd & 1)) {
        dd >>= 1;
        ++r;
    }
    auto mulm = [q](u64 x, u64 y) { return (u64)((unsigned __int128)x * y % q); };
    for (u64 b : {2ull, 3ull, 5ull, 7ull}) {
        u64 x = 1, e = dd, base = b % q;
        while (e) {
            if (e & 1) x = mulm(x, base);
            base = mulm(base, base);
            e >>= 1;
        }
        if (x == 1 || x == q - 1) continue;
        bool comp = true;
        for (int i = 1; i < r && comp; ++i) {
            x = mulm(x, x);
            if (x == q - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

size_t sb_round(size_t b) { return (b + kSbAlign - 1) / kSbAlign * kSbAlign; }

int sb_default_base(int m, int n)
{
    int b = kSbMaxBase;
    while (b > 1 && sb_leaf_smem(m, n, b) > kSbSmemMax) b >>= 1;
    return sb_leaf_smem(m, n, b) <= kSbSmemMax ? b : 0;
}

// stack bytes of the recursion at order d (degrees at their bound)
size_t sb_stack_bytes(int m, long long d, int base)
{
    if (d <= base) return 0;
    const long long d1 = (d + 1) / 2, d2 = d - d1;
    const size_t mm = (size_t)m * m * 4;
    const size_t P1 = sb_round((d1 + 1) * mm), C = sb_round((d1 + d) * mm), P2 = sb_round((d2 + 1) * mm);
    return std::max(P1 + sb_stack_bytes(m, d1, base), P1 + C + P2 + sb_stack_bytes(m, d2, base));
}

struct SbRun {
    u32 p;
    int m, n, base;
    Mod M;
    cudaStream_t st;
    char *stack;
    size_t cap, top;
    void *pm_work;
    int64_t pm_bytes;
    int *d_delta;
};

u32 *sb_alloc(SbRun &R, size_t elems)
{
    const size_t b = sb_round(elems * 4);
    if (R.top + b > R.cap) return nullptr;
    u32 *ptr = reinterpret_cast<u32 *>(R.stack + R.top);
    R.top += b;
    return ptr;
}

long long sb_degree_bound(const int *delta, const int *shift, int m, long long d)
{
    int dmax = INT_MIN, smin = INT_MAX;
    for (int i = 0; i < m; ++i) {
        dmax = std::max(dmax, delta[i]);
        smin = std::min(smin, shift[i]);
    }
    return std::max(0LL, std::min(d, (long long)dmax - smin));
}

ffspmv_status sb_leaf(SbRun &R, const u32 *F, long long d, const int *shift, u32 *P, int *delta)
{
    SbLeaf a;
    memset(&a, 0, sizeof(a));
    a.F = F;
    a.P = P;
    a.delta = R.d_delta;
    for (int i = 0; i < R.m; ++i) a.shift[i] = shift[i];
    a.m = R.m;
    a.n = R.n;
    a.d = (int)d;
    a.ldf = R.m;
    a.M = R.M;
    k_sb_mbasis<<<1, kSbThreads, sb_leaf_smem(R.m, R.n, d), R.st>>>(a);
    FF_CUDA(cudaGetLastError());
    FF_CUDA(cudaMemcpyAsync(delta, R.d_delta, sizeof(int) * R.m, cudaMemcpyDeviceToHost, R.st));
    FF_CUDA(cudaStreamSynchronize(R.st));
    return FFSPMV_OK;
}

// order-d basis of F (d coefficients of m x m, columns >= n zero) into P
// ((d+1) coefficients, zero above the degree); delta and the degree bound out
ffspmv_status sb_rec(SbRun &R, const u32 *F, long long d, const int *shift, u32 *P, int *delta, long long *e)
{
    ffspmv_status st;
    if (d <= R.base) {
        if ((st = sb_leaf(R, F, d, shift, P, delta)) != FFSPMV_OK) return st;
        *e = sb_degree_bound(delta, shift, R.m, d);
        return FFSPMV_OK;
    }
    const long long d1 = (d + 1) / 2, d2 = d - d1;
    const size_t mm = (size_t)R.m * R.m;
    const size_t mark = R.top;
    std::vector<int> delta1(R.m), delta2(R.m);
    long long e1 = 0, e2 = 0;
    u32 *P1 = sb_alloc(R, (d1 + 1) * mm);
    if (!P1) return FFSPMV_ERR_ARG;
    if ((st = sb_rec(R, F, d1, shift, P1, delta1.data(), &e1)) != FFSPMV_OK) return st;
    // the residual: coefficients d1..d-1 of P1 F
    u32 *C = sb_alloc(R, (e1 + d) * mm);
    u32 *P2 = sb_alloc(R, (d2 + 1) * mm);
    if (!C || !P2) return FFSPMV_ERR_ARG;
    st = polymat_mul(R.p, R.m, e1, d - 1, P1, F, C, R.pm_work, R.pm_bytes, (ffspmv_stream_t)R.st);
    if (st != FFSPMV_OK) return st;
    if ((st = sb_rec(R, C + d1 * mm, d2, delta1.data(), P2, delta2.data(), &e2)) != FFSPMV_OK) return st;
    st = polymat_mul(R.p, R.m, e2, e1, P2, P1, P, R.pm_work, R.pm_bytes, (ffspmv_stream_t)R.st);
    if (st != FFSPMV_OK) return st;
    if (e1 + e2 < d)
        FF_CUDA(cudaMemsetAsync(P + (e1 + e2 + 1) * mm, 0, (size_t)(d - e1 - e2) * mm * 4, R.st));
    for (int i = 0; i < R.m; ++i) delta[i] = delta2[i];
    *e = std::min(e1 + e2, sb_degree_bound(delta, shift, R.m, d));
    R.top = mark;
    return FFSPMV_OK;
}

struct SbLayout {
    int base;
    int64_t pm, fpad, dl, stack, total;
};

ffspmv_status sb_layout(int32_t m, int32_t n, int64_t d, int32_t base, SbLayout *out)
{
    if (m < 1 || m > kSbMaxM || n < 1 || n > m || d < 1 || base < 0 || base > kSbMaxBase) return FFSPMV_ERR_ARG;
    const int b = base ? base : sb_default_base(m, n);
    if (b < 1 || sb_leaf_smem(m, n, b) > kSbSmemMax) return FFSPMV_ERR_UNSUPPORTED;
    SbLayout L;
    L.base = b;
    L.pm = 0;
    if (d > b) {   // the largest product: (ceil(d/2) + 1) by d coefficients
        const ffspmv_status st = polymat_mul_workspace(m, (d + 1) / 2, d - 1, &L.pm);
        if (st != FFSPMV_OK) return st;
    }
    L.pm = (int64_t)sb_round((size_t)L.pm);
    L.fpad = (int64_t)sb_round((size_t)d * m * m * 4);
    L.dl = (int64_t)sb_round(kSbMaxM * 4);
    L.stack = (int64_t)sb_stack_bytes(m, d, b);
    L.total = L.pm + L.fpad + L.dl + L.stack;
    *out = L;
    return FFSPMV_OK;
}

}  // namespace
}  // namespace ff

using namespace ff;

extern "C" ffspmv_status sigma_basis_workspace(int32_t m, int32_t n, int64_t d, int32_t base, int64_t *bytes)
{
    if (!bytes) return FFSPMV_ERR_ARG;
    SbLayout L;
    const ffspmv_status st = sb_layout(m, n, d, base, &L);
    if (st != FFSPMV_OK) return st;
    *bytes = L.total;
    return FFSPMV_OK;
}

extern "C" ffspmv_status sigma_basis(uint32_t p, int32_t m, int32_t n, int64_t d, int32_t base,
                                     const uint32_t *d_F, const int32_t *h_shift, uint32_t *d_P,
                                     int32_t *h_delta, int64_t *h_degree, void *d_work, int64_t work_bytes,
                                     ffspmv_stream_t stream)
{
    if (p < 2 || p > (1u << 31) || !sb_is_prime(p) || !d_F || !d_P || !h_delta || !d_work) return FFSPMV_ERR_ARG;
    SbLayout L;
    ffspmv_status st = sb_layout(m, n, d, base, &L);
    if (st != FFSPMV_OK) return st;
    if (work_bytes < L.total || ((uintptr_t)d_work & 15)) return FFSPMV_ERR_ARG;
    std::vector<int> shift(m, 0);
    if (h_shift) {
        for (int i = 0; i < m; ++i) {
            if (h_shift[i] > kSbMaxShift || h_shift[i] < -kSbMaxShift) return FFSPMV_ERR_ARG;
            shift[i] = h_shift[i];
        }
    }
    SbRun R;
    R.p = p;
    R.m = m;
    R.n = n;
    R.base = L.base;
    R.M = make_mod(p, 1, 0);
    R.st = (cudaStream_t)stream;
    char *w = static_cast<char *>(d_work);
    R.pm_work = w;
    R.pm_bytes = L.pm;
    u32 *Fp = reinterpret_cast<u32 *>(w + L.pm);
    R.d_delta = reinterpret_cast<int *>(w + L.pm + L.fpad);
    R.stack = w + L.pm + L.fpad + L.dl;
    R.cap = (size_t)L.stack;
    R.top = 0;
    FF_CUDA(cudaFuncSetAttribute(k_sb_mbasis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sb_leaf_smem(m, n, L.base)));
    const long long total = d * m * m;
    const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 4096);
    k_sb_pad<<<blocks, 256, 0, R.st>>>(d_F, d, m, n, Fp, R.M);
    FF_CUDA(cudaGetLastError());
    long long e = 0;
    std::vector<int> delta(m);
    st = sb_rec(R, Fp, d, shift.data(), d_P, delta.data(), &e);
    if (st != FFSPMV_OK) return st;
    FF_CUDA(cudaStreamSynchronize(R.st));
    for (int i = 0; i < m; ++i) h_delta[i] = delta[i];
    if (h_degree) *h_degree = e;
    return FFSPMV_OK;
}

extern "C" ffspmv_status sigma_wiedemann_input(uint32_t p, int32_t s, int64_t L, const uint32_t *d_S, uint32_t *d_F,
                                               ffspmv_stream_t stream)
{
    if (p < 2 || p > (1u << 31) || s < 1 || s > kSbMaxM / 2 || L < 1 || !d_S || !d_F) return FFSPMV_ERR_ARG;
    const long long total = L * 2 * s * s;
    const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 4096);
    k_sb_wiedemann<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_S, L, s, d_F, p);
    FF_CUDA(cudaGetLastError());
    return FFSPMV_OK;
}
