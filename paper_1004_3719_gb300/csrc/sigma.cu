// Sigma-bases over F_p for the second step of block Wiedemann (Sec. 3.2,
// "Parallelization of the sigma-basis computation"): PM-Basis (Giorgi,
// Jeannerod and Villard, ISSAC 2003) as a host recursion on the order whose
// work is polynomial-matrix products on the GPU (polymat_mul, Sec. 3.2.1's
// evaluation / pointwise / interpolation scheme), and M-Basis, the iterative
// algorithm Sec. 3.2.2 recommends at small orders, as one CTA per leaf.
//
// M-Basis leaf.  An order-d problem (d <= 32) runs on one cluster of CTAs
// that keep, column by column, the residual R = P F (coefficients k..d-1,
// m x n) and the basis P (coefficients 0..k, m x m) in shared memory.  At
// order k four warps eliminate the m x n matrix R_k column by column (rows
// ordered by (delta_i, i), pivot = the first non-pivot row nonzero in the
// column), one lane per row; every CTA then applies the same row operations
// to its coefficients of R and P, one warp per (coefficient, column)
// position, and multiplies the pivot rows by x.  The elimination is fraction
// free -- row r becomes a r - b q with a the pivot's entry and b row r's
// entry -- so no inverse is taken inside the loop; each row of P is then a
// known nonzero multiple c_r of the row that the elimination with division
// gives, and one inversion per row at the end of the leaf divides it out,
// which makes the result the same as the plain algorithm's.
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
constexpr int kSbWarps = kSbThreads / 32;
constexpr int kSbCluster = 8;               // CTAs of one leaf (portable cluster size)
constexpr int kSbElimWarps = 4;             // warps of the leader that eliminate R_k
constexpr size_t kSbSmemMax = 227 * 1024;
constexpr size_t kSbAlign = 256;
constexpr int kSbMaxShift = 1 << 24;
constexpr int kSbRkLd = kSbMaxM + 1;        // row stride of the leader's copy of R_k (no bank conflicts)

struct SbLeaf {
    const u32 *F;   // d x m x ldf, columns < n used
    u32 *P;         // out: (d+1) x m x m
    int *delta;     // out: m
    int shift[kSbMaxM];
    int m, n, d, ldf;
    Mod M;
};

// The operations of one order, as every CTA of the leaf receives them:
// (multiplier, addend) of row r at column j in op[j][r], the pivot row of
// column j (-1: none) and the pivot flags of the rows.
struct SbOps {
    uint2 op[kSbMaxM][kSbMaxM];
    int piv[kSbMaxM];
    int isp[kSbMaxM];
};

// CTAs of a leaf: one per column of [R | P] at most
__host__ __device__ inline int sb_cluster(int m, int n) { return n + m < kSbCluster ? n + m : kSbCluster; }

// Shared memory of one CTA of a leaf: the operations (two copies, by order
// parity), the leader's copy of R_k, the inverse row scales, then the CTA's
// columns of [R | P] (column w belongs to CTA w mod C), each (d+1) x m words
// coefficient-major: word (t m + r) of a column is row r of coefficient t.
constexpr size_t kSbOpsBytes = sizeof(SbOps);
constexpr size_t kSbRkOff = 2 * kSbOpsBytes;
constexpr size_t kSbInvOff = kSbRkOff + (size_t)kSbMaxM * kSbRkLd * 4;
constexpr size_t kSbColOff = kSbInvOff + kSbMaxM * 4;
static_assert(kSbOpsBytes % 16 == 0 && kSbColOff % 16 == 0, "16-byte blocks");

size_t sb_leaf_smem(int m, int n, long long d)
{
    const int C = sb_cluster(m, n), own = (n + m + C - 1) / C;
    return kSbColOff + (size_t)own * (size_t)(d + 1) * m * 4;
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

// The same shared-memory word in CTA `rank` of the cluster.
__device__ __forceinline__ u32 sb_remote(const void *local, u32 rank)
{
    u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((u32)__cvta_generic_to_shared(local)), "r"(rank));
    return r;
}

__device__ __forceinline__ void sb_st_remote(u32 addr, u32 v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ void sb_st_remote_v4(u32 addr, uint4 v)
{
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

// Every thread of every CTA of the cluster: writes before it are seen after it.
__device__ __forceinline__ void sb_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ u32 sb_cluster_rank()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ u32 sb_cluster_size()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// One M-Basis leaf on a cluster of C CTAs (C = min(8, n + m)).  Each CTA
// keeps its columns of [R | P] in shared memory; per order k:
//   1. four warps of the leader eliminate R_k (gathered in the leader), one
//      lane per row, the columns split between them, and send the
//      operations to every CTA;
//   2. every CTA applies them to its positions, one warp per (coefficient,
//      column) position (two at a time) and one lane per row (R:
//      coefficients k..d-1, P: 0..k);
//   3. the pivot rows of each column move up one coefficient (times x), and
//      the owners of R's columns send R_{k+1} to the leader.
// Two cluster barriers per order order these steps.
__global__ void __launch_bounds__(kSbThreads, 1) k_sb_mbasis(const __grid_constant__ SbLeaf a)
{
    extern __shared__ __align__(16) unsigned char sb_sm[];
    const int m = a.m, n = a.n, d = a.d;
    const u32 p = a.M.m;
    const u32 rank = sb_cluster_rank(), C = sb_cluster_size();
    const int own = (n + m - (int)rank + (int)C - 1) / (int)C;  // columns rank, rank + C, ...
    SbOps *ops = reinterpret_cast<SbOps *>(sb_sm);
    u32 *Rk = reinterpret_cast<u32 *>(sb_sm + kSbRkOff);   // leader: R_k row r at r * kSbRkLd
    u32 *sinv = reinterpret_cast<u32 *>(sb_sm + kSbInvOff);
    u32 *col = reinterpret_cast<u32 *>(sb_sm + kSbColOff);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cst = (d + 1) * m;   // words per column

    // column i of this CTA is column w = rank + i C of [R | P]: R's column w
    // (the input, reduced) when w < n, else P's column w - n (the identity)
    for (int i = 0; i < own; ++i) {
        const int w = (int)rank + i * (int)C;
        u32 *cb = col + (size_t)i * cst;
        for (int e = tid; e < cst; e += kSbThreads) {
            const int t = e / m, r = e % m;
            u32 v;
            if (w < n) v = t < d ? red64(a.F[((size_t)t * m + r) * a.ldf + w], a.M) : 0u;
            else v = (t == 0 && r == w - n) ? 1u : 0u;
            cb[e] = v;
        }
    }
    __syncthreads();
    sb_cluster_sync();   // every CTA of the leaf runs before any remote store
    for (int i = warp; i < own; i += kSbWarps) {
        const int w = (int)rank + i * (int)C;
        if (w < n && lane < m) sb_st_remote(sb_remote(Rk + lane * kSbRkLd + w, 0), col[(size_t)i * cst + lane]);
    }
    // leader's warp 0, lane r < m: delta_r and c_r, the product of the
    // multipliers applied to row r
    int dl = lane < m ? a.shift[lane] : 0;
    u32 cs = 1u;
    for (int k = 0; k < d; ++k) {
        SbOps &O = ops[k & 1];
        sb_cluster_sync();   // R_k is complete in the leader
        if (rank == 0 && warp < kSbElimWarps) {
            // rows ordered by (delta_i, i); the pivot of column j is the first
            // row in that order, not yet a pivot, nonzero in the column.  The
            // elimination warps each hold one row per lane and update the
            // columns c = warp (mod kSbElimWarps); every one of them finds the
            // same pivots, and a named barrier ends each column
            const bool row = lane < m;
            int myrank = 0;
#pragma unroll
            for (int j = 0; j < kSbMaxM; ++j) {
                const int dj = __shfl_sync(0xffffffffu, dl, j);
                myrank += (j < m && (dj < dl || (dj == dl && j < lane))) ? 1 : 0;
            }
            u32 *__restrict__ Rrow = Rk + lane * kSbRkLd;
            u32 piv = 0u;   // bit r: row r is a pivot at this order
            for (int j = 0; j < n; ++j) {
                const u32 x = row ? Rrow[j] : 0u;
                const bool cand = row && !((piv >> lane) & 1u) && x != 0u;
                const u32 key = cand ? (u32)myrank : 64u;
                const u32 mn = __reduce_min_sync(0xffffffffu, key);
                uint2 myop = make_uint2(1u, 0u);
                if (mn != 64u) {
                    const int q = __ffs(__ballot_sync(0xffffffffu, key == mn)) - 1;
                    const u32 av = __shfl_sync(0xffffffffu, x, q);
                    if (cand && lane != q) {
                        // row <- av row - x pivot row (fraction free); columns
                        // of this warp, their loads issued before the stores
                        const u32 g = p - x;
                        const u32 *__restrict__ Rq = Rk + q * kSbRkLd;
                        const int c0 = j + 1 + ((warp - (j + 1)) % kSbElimWarps + kSbElimWarps) % kSbElimWarps;
                        for (int cb = c0; cb < n; cb += 4 * kSbElimWarps) {
                            u32 ra[4], qa[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int c = cb + u * kSbElimWarps;
                                ra[u] = c < n ? Rrow[c] : 0u;
                                qa[u] = c < n ? Rq[c] : 0u;
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int c = cb + u * kSbElimWarps;
                                if (c < n) Rrow[c] = red64((u64)av * ra[u] + (u64)g * qa[u], a.M);
                            }
                        }
                        myop = make_uint2(av, g);
                        if (warp == 0) cs = red64((u64)cs * av, a.M);
                    }
                    piv |= 1u << q;
                    if (warp == 0 && lane == 0) O.piv[j] = q;
                } else if (warp == 0 && lane == 0) {
                    O.piv[j] = -1;   // column j is already zero in every non-pivot row
                }
                if (warp == 0 && row) O.op[j][lane] = myop;
                asm volatile("bar.sync 1, %0;" ::"n"(kSbElimWarps * 32) : "memory");   // column j done
            }
            if (row) {
                const int ip = (int)((piv >> lane) & 1u);
                if (warp == 0) O.isp[lane] = ip;
                dl += ip;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(kSbElimWarps * 32) : "memory");   // the operations are complete
            // the operations to the other CTAs (split over the elimination
            // warps): rows j < n of op[][], then piv and isp
            const uint4 *src = reinterpret_cast<const uint4 *>(&O);
            const uint4 *tail = reinterpret_cast<const uint4 *>(O.piv);
            const int nq = n * (int)(kSbMaxM * sizeof(uint2) / 16);
            for (u32 rr = 1 + (u32)warp; rr < C; rr += kSbElimWarps) {
                for (int e = lane; e < nq; e += 32) sb_st_remote_v4(sb_remote(src + e, rr), src[e]);
                if (lane < (int)(2 * kSbMaxM * sizeof(int) / 16)) sb_st_remote_v4(sb_remote(tail + lane, rr), tail[lane]);
            }
        }
        sb_cluster_sync();   // the operations of order k are in every CTA
        // positions: R's coefficients k..d-1 and P's 0..k of this CTA's
        // columns, two per warp at a time (two independent chains of
        // operations in flight)
        auto cell_of = [&](int pos) -> u32 * {
            for (int i = 0; i < own; ++i) {
                const int w = (int)rank + i * (int)C;
                const int cnt = w < n ? d - k : k + 1;
                if (pos < cnt) return col + (size_t)i * cst + (size_t)(w < n ? k + pos : pos) * m;
                pos -= cnt;
            }
            return nullptr;
        };
        for (int pos = warp;; pos += 2 * kSbWarps) {
            u32 *c0 = cell_of(pos);
            if (!c0) break;
            u32 *c1 = cell_of(pos + kSbWarps);
            u32 v0 = lane < m ? c0[lane] : 0u, v1 = (c1 && lane < m) ? c1[lane] : 0u;
            for (int j = 0; j < n; ++j) {
                const int q = O.piv[j];
                if (q < 0) continue;
                const u32 q0 = __shfl_sync(0xffffffffu, v0, q), q1 = __shfl_sync(0xffffffffu, v1, q);
                if (lane < m) {
                    const uint2 op = O.op[j][lane];
                    if (op.y) {
                        v0 = red64((u64)op.x * v0 + (u64)op.y * q0, a.M);
                        v1 = red64((u64)op.x * v1 + (u64)op.y * q1, a.M);
                    }
                }
            }
            if (lane < m) {
                c0[lane] = v0;
                if (c1) c1[lane] = v1;
            }
        }
        __syncthreads();
        // pivot rows times x: R's coefficients k..d-1 and P's 0..k+1 move up by one
        for (int i = warp; i < own; i += kSbWarps) {
            const int w = (int)rank + i * (int)C;
            u32 *cb = col + (size_t)i * cst;
            if (lane < m && O.isp[lane]) {
                if (w < n) {
                    for (int t = d - 1; t > k; --t) cb[t * m + lane] = cb[(t - 1) * m + lane];
                    cb[k * m + lane] = 0u;
                } else {
                    for (int t = k + 1; t > 0; --t) cb[t * m + lane] = cb[(t - 1) * m + lane];
                    cb[lane] = 0u;
                }
            }
            if (w < n && k + 1 < d && lane < m)
                sb_st_remote(sb_remote(Rk + lane * kSbRkLd + w, 0), cb[(k + 1) * m + lane]);
        }
    }
    sb_cluster_sync();
    if (rank == 0 && warp == 0 && lane < m) {
        const u32 inv = sb_pow(cs, p - 2u, a.M);   // c_r != 0 in the field F_p
        for (u32 rr = 0; rr < C; ++rr) sb_st_remote(sb_remote(sinv + lane, rr), inv);
        a.delta[lane] = dl;
    }
    sb_cluster_sync();   // the scales are in every CTA; no remote access after this
    for (int i = 0; i < own; ++i) {
        const int w = (int)rank + i * (int)C;
        if (w < n) continue;
        const u32 *cb = col + (size_t)i * cst;
        for (int e = tid; e < cst; e += kSbThreads) {
            const int t = e / m, r = e % m;
            a.P[((size_t)t * m + r) * m + (w - n)] = red64((u64)cb[e] * sinv[r], a.M);
        }
    }
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
    const unsigned C = (unsigned)sb_cluster(R.m, R.n);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(kSbThreads, 1, 1);
    cfg.dynamicSmemBytes = sb_leaf_smem(R.m, R.n, d);
    cfg.stream = R.st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FF_CUDA(cudaLaunchKernelEx(&cfg, k_sb_mbasis, a));
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
