// Products of s x s polynomial matrices over Z/pZ, C(x) = A(x) B(x): the
// multiplication that the sigma-basis / PM-Basis step of block Wiedemann
// (Sec. 3) is built from.  Coefficient-major arrays: A[k][i][j] is the
// coefficient of x^k in entry (i, j).
//
// The exact integer coefficients of C are below s * min(da, db + ...) * (p-1)^2
// < P0 P1 P2 for three NTT-friendly primes, so C is computed modulo each of
// them by number-theoretic transforms (length L, the power of two >= da+db+1;
// one CTA per polynomial, in shared memory), a pointwise s x s matrix product
// at each of the L points, and the inverse transforms, then brought back to
// Z/pZ by Garner's mixed-radix reconstruction.  Forward transforms are
// decimation in frequency (natural order in, bit-reversed out) and the inverse
// ones decimation in time (bit-reversed in, natural out), so no permutation
// pass is needed; the pointwise products do not care about the order.
#include <algorithm>
#include <cstring>

#include "ff_internal.cuh"
#include "ffspmv_polymat.h"

namespace ff {
namespace {

constexpr int kPmPrimes = 3;
constexpr u32 kPmP[kPmPrimes] = {998244353u, 167772161u, 469762049u};  // c 2^k + 1, k = 23, 25, 26
constexpr u32 kPmGen = 3;                                            // a primitive root of each
constexpr int kPmMaxLog = 15;                                        // L <= 2^15: 128 KB of shared memory
constexpr int kNttThreads = 512;

struct PmConsts {
    Mod P[kPmPrimes];
    u32 root[kPmPrimes], iroot[kPmPrimes], linv[kPmPrimes];
    Mod mp;              // the output modulus p
    u32 inv01, inv02, inv12;  // P0^-1 mod P1, P0^-1 mod P2, P1^-1 mod P2
    u32 p0_mod_p, p0p1_mod_p;
};

__device__ __forceinline__ u32 mulm(u32 a, u32 b, const Mod &M) { return red64((u64)a * b, M); }

__device__ u32 powm(u32 a, u32 e, const Mod &M)
{
    u32 r = 1u % M.m;
    while (e) {
        if (e & 1u) r = mulm(r, a, M);
        a = mulm(a, a, M);
        e >>= 1;
    }
    return r;
}

// tw[q][0][i] = root_q^i, tw[q][1][i] = root_q^-i, i < L/2
__global__ void k_pm_twiddles(u32 *tw, int L, const __grid_constant__ PmConsts c)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int h = L / 2;
    if (t >= (long long)kPmPrimes * 2 * h) return;
    const int i = (int)(t % h), dir = (int)(t / h % 2), q = (int)(t / (2 * h));
    tw[t] = powm(dir ? c.iroot[q] : c.root[q], (u32)i, c.P[q]);
}

// dst[q][e][k] = src[k][e] mod P_q for k <= d, 0 up to L
__global__ void k_pm_load(const u32 *__restrict__ src, long long d, int s2, int L, u32 *__restrict__ dst,
                          const __grid_constant__ PmConsts c)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)kPmPrimes * s2 * L) return;
    const int k = (int)(t % L);
    const long long qe = t / L;
    const int e = (int)(qe % s2), q = (int)(qe / s2);
    dst[t] = k <= d ? src[(long long)k * s2 + e] % c.P[q].m : 0u;
}

// One polynomial of length L per CTA, transformed in shared memory.
template <bool INV>
__global__ void __launch_bounds__(kNttThreads) k_ntt(u32 *__restrict__ data, int L, int s2, const u32 *__restrict__ tw,
                                                     const __grid_constant__ PmConsts c)
{
    extern __shared__ u32 a[];
    const int q = blockIdx.x / s2;
    const Mod &M = c.P[q];
    const u32 P = M.m;
    const u32 *w = tw + ((size_t)q * 2 + (INV ? 1 : 0)) * (L / 2);
    u32 *g = data + (size_t)blockIdx.x * L;
    for (int i = threadIdx.x; i < L; i += kNttThreads) a[i] = g[i];
    __syncthreads();
    const int h = L / 2;
    if (!INV) {
        for (int len = h; len >= 1; len >>= 1) {  // decimation in frequency
            const int step = h / len;
            for (int b = threadIdx.x; b < h; b += kNttThreads) {
                const int j = b % len, i0 = (b / len) * 2 * len + j, i1 = i0 + len;
                const u32 u = a[i0], v = a[i1];
                const u32 sum = u + v >= P ? u + v - P : u + v;
                a[i0] = sum;
                a[i1] = mulm(u >= v ? u - v : u + P - v, w[j * step], M);
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < L; i += kNttThreads) g[i] = a[i];
    } else {
        for (int len = 1; len <= h; len <<= 1) {  // decimation in time
            const int step = h / len;
            for (int b = threadIdx.x; b < h; b += kNttThreads) {
                const int j = b % len, i0 = (b / len) * 2 * len + j, i1 = i0 + len;
                const u32 u = a[i0], v = mulm(a[i1], w[j * step], M);
                a[i0] = u + v >= P ? u + v - P : u + v;
                a[i1] = u >= v ? u - v : u + P - v;
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < L; i += kNttThreads) g[i] = mulm(a[i], c.linv[q], M);
    }
}

// Ch[q][i s + j][t] = sum_k Ah[q][i s + k][t] Bh[q][k s + j][t] mod P_q
__global__ void k_pm_pointwise(const u32 *__restrict__ Ah, const u32 *__restrict__ Bh, u32 *__restrict__ Ch, int s,
                               int L, const __grid_constant__ PmConsts c)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int s2 = s * s;
    if (t >= (long long)kPmPrimes * s2 * L) return;
    const int pt = (int)(t % L);
    const long long qe = t / L;
    const int e = (int)(qe % s2), q = (int)(qe / s2);
    const int i = e / s, j = e % s;
    const Mod &M = c.P[q];
    const u32 *ar = Ah + ((size_t)q * s2 + (size_t)i * s) * L + pt;
    const u32 *bc = Bh + ((size_t)q * s2 + j) * L + pt;
    u64 acc = 0;
    u32 r = 0;
    for (int k = 0; k < s; ++k) {
        acc += (u64)__ldg(ar + (size_t)k * L) * __ldg(bc + (size_t)k * s * L);  // each below 2^60
        if ((k & 7) == 7) {
            r = red64((u64)r + red64(acc, M), M);
            acc = 0;
        }
    }
    Ch[t] = red64((u64)r + red64(acc, M), M);
}

// C[k][e] = the integer with residues Ch[0..2][e][k], mod p (Garner)
__global__ void k_pm_crt(const u32 *__restrict__ Ch, u32 *__restrict__ C, long long dc, int s2, int L,
                         const __grid_constant__ PmConsts c)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (dc + 1) * s2) return;
    const int e = (int)(t % s2);
    const long long k = t / s2;
    const size_t plane = (size_t)s2 * L;
    const u32 r0 = Ch[(size_t)e * L + k], r1 = Ch[plane + (size_t)e * L + k], r2 = Ch[2 * plane + (size_t)e * L + k];
    const Mod &M1 = c.P[1], &M2 = c.P[2];
    const u32 x1 = r0;                                           // < P0
    const u32 x1m1 = x1 % M1.m, x1m2 = x1 % M2.m;
    const u32 x2 = mulm(r1 >= x1m1 ? r1 - x1m1 : r1 + M1.m - x1m1, c.inv01, M1);  // < P1
    u32 t3 = mulm(r2 >= x1m2 ? r2 - x1m2 : r2 + M2.m - x1m2, c.inv02, M2);
    const u32 x2m2 = x2 % M2.m;
    t3 = t3 >= x2m2 ? t3 - x2m2 : t3 + M2.m - x2m2;
    const u32 x3 = mulm(t3, c.inv12, M2);                        // < P2
    // value = x1 + P0 x2 + P0 P1 x3, reduced mod p term by term
    const Mod &mp = c.mp;
    u64 v = (u64)(x1 % mp.m) + red64((u64)c.p0_mod_p * x2, mp) + red64((u64)c.p0p1_mod_p * x3, mp);
    C[(size_t)k * s2 + e] = red64(v, mp);
}

u32 powmod_host(u64 a, u64 e, u64 m)
{
    u64 r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = (unsigned __int128)r * a % m;
        a = (unsigned __int128)a * a % m;
        e >>= 1;
    }
    return (u32)r;
}

int pm_log2(long long da, long long db)
{
    int lg = 0;
    while ((1LL << lg) < da + db + 1) ++lg;
    return std::max(lg, 1);
}

}  // namespace
}  // namespace ff

using namespace ff;

extern "C" ffspmv_status polymat_mul_workspace(int32_t s, int64_t da, int64_t db, int64_t *bytes)
{
    if (!bytes || s < 1 || s > 32 || da < 0 || db < 0) return FFSPMV_ERR_ARG;
    const int lg = pm_log2(da, db);
    if (lg > kPmMaxLog) return FFSPMV_ERR_UNSUPPORTED;
    const long long L = 1LL << lg;
    *bytes = 3LL * kPmPrimes * s * s * L * 4 + (long long)kPmPrimes * L * 4 + 256;
    return FFSPMV_OK;
}

extern "C" ffspmv_status polymat_mul(uint32_t p, int32_t s, int64_t da, int64_t db, const uint32_t *d_A,
                                     const uint32_t *d_B, uint32_t *d_C, void *d_work, int64_t work_bytes,
                                     ffspmv_stream_t stream)
{
    if (p < 2 || p > (1u << 31) || s < 1 || s > 32 || da < 0 || db < 0 || !d_A || !d_B || !d_C || !d_work)
        return FFSPMV_ERR_ARG;
    int64_t need = 0;
    ffspmv_status r = polymat_mul_workspace(s, da, db, &need);
    if (r != FFSPMV_OK) return r;
    if (work_bytes < need || ((uintptr_t)d_work & 15)) return FFSPMV_ERR_ARG;
    // the exact coefficients must stay below P0 P1 P2
    const long double bound = (long double)s * (long double)(std::min(da, db) + 1) * (long double)(p - 1) *
                              (long double)(p - 1);
    const long double prod = (long double)kPmP[0] * kPmP[1] * kPmP[2];
    if (bound >= prod) return FFSPMV_ERR_UNSUPPORTED;
    const int lg = pm_log2(da, db);
    const int L = 1 << lg, s2 = s * s;
    PmConsts c;
    memset(&c, 0, sizeof(c));
    for (int q = 0; q < kPmPrimes; ++q) {
        const u64 P = kPmP[q];
        c.P[q] = make_mod((u32)P, 1, 0);
        c.root[q] = powmod_host(kPmGen, (P - 1) >> lg, P);
        // order exactly L: root^(L/2) = -1
        if (powmod_host(c.root[q], (u64)L / 2, P) != P - 1) return FFSPMV_ERR_UNSUPPORTED;
        c.iroot[q] = powmod_host(c.root[q], P - 2, P);
        c.linv[q] = powmod_host((u64)L, P - 2, P);
    }
    c.mp = make_mod(p, 1, 0);
    c.inv01 = powmod_host(kPmP[0] % kPmP[1], kPmP[1] - 2, kPmP[1]);
    c.inv02 = powmod_host(kPmP[0] % kPmP[2], kPmP[2] - 2, kPmP[2]);
    c.inv12 = powmod_host(kPmP[1] % kPmP[2], kPmP[2] - 2, kPmP[2]);
    c.p0_mod_p = (u32)(kPmP[0] % p);
    c.p0p1_mod_p = (u32)((unsigned __int128)kPmP[0] * kPmP[1] % p);

    cudaStream_t st = (cudaStream_t)stream;
    const size_t plane = (size_t)kPmPrimes * s2 * L;
    u32 *Ah = (u32 *)d_work, *Bh = Ah + plane, *Ch = Bh + plane, *tw = Ch + plane;
    const int T = 256;
    auto blocks = [&](long long n) { return (unsigned)((n + T - 1) / T); };
    k_pm_twiddles<<<blocks((long long)kPmPrimes * L), T, 0, st>>>(tw, L, c);
    k_pm_load<<<blocks(plane), T, 0, st>>>(d_A, da, s2, L, Ah, c);
    k_pm_load<<<blocks(plane), T, 0, st>>>(d_B, db, s2, L, Bh, c);
    FF_CUDA(cudaGetLastError());
    const size_t smem = (size_t)L * 4;
    FF_CUDA(cudaFuncSetAttribute(k_ntt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FF_CUDA(cudaFuncSetAttribute(k_ntt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_ntt<false><<<(unsigned)(kPmPrimes * s2), kNttThreads, smem, st>>>(Ah, L, s2, tw, c);
    k_ntt<false><<<(unsigned)(kPmPrimes * s2), kNttThreads, smem, st>>>(Bh, L, s2, tw, c);
    k_pm_pointwise<<<blocks(plane), T, 0, st>>>(Ah, Bh, Ch, s, L, c);
    k_ntt<true><<<(unsigned)(kPmPrimes * s2), kNttThreads, smem, st>>>(Ch, L, s2, tw, c);
    k_pm_crt<<<blocks((da + db + 1) * s2), T, 0, st>>>(Ch, d_C, da + db, s2, L, c);
    FF_CUDA(cudaGetLastError());
    return FFSPMV_OK;
}
