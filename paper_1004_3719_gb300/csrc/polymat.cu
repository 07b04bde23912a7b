// Products of s x s polynomial matrices over Z/pZ, C(x) = A(x) B(x): the
// multiplication that the sigma-basis / PM-Basis step of block Wiedemann is
// built from, by the fast algorithm of Sec. 3 (parallel polynomial matrix
// multiplication): evaluate both operands at the powers of a root of unity,
// multiply the matrices point by point, interpolate back.  Coefficient-major
// arrays: A[k][i][j] is the coefficient of x^k in entry (i, j).
//
// F_p itself has roots of unity of order at most 16 when p = 65521, so the
// transforms run over three primes with large power-of-two roots instead: the
// exact integer coefficients of C are below s * (min(da, db) + 1) * (p-1)^2
// < P0 P1 P2, so C is computed modulo each of
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
    u32 root[kPmPrimes], iroot[kPmPrimes], linv[kPmPrimes], linv_q[kPmPrimes];
    int reduce_input;    // p > the smallest prime: inputs need a reduction mod P_q
    Mod mp;              // the output modulus p
    u32 inv01, inv02, inv12;  // P0^-1 mod P1, P0^-1 mod P2, P1^-1 mod P2
    u32 p0_mod_p, p0p1_mod_p;
};

__device__ __forceinline__ u32 mulm(u32 a, u32 b, const Mod &M) { return red64((u64)a * b, M); }

// a * w mod P for a fixed w with wq = floor(w 2^32 / P), P < 2^31 (Shoup): the
// quotient estimate umulhi(a, wq) is the true quotient or one less, so the
// 32-bit remainder lies in [0, 2P).
__device__ __forceinline__ u32 mul_shoup(u32 a, u32 w, u32 wq, u32 P)
{
    const u32 r = a * w - __umulhi(a, wq) * P;
    return r >= P ? r - P : r;
}

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

// tw[q][0][i] = (root_q^i, its Shoup quotient), tw[q][1][i] the same for root_q^-i, i < L/2
__global__ void k_pm_twiddles(uint2 *tw, int L, const __grid_constant__ PmConsts c)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int h = L / 2;
    if (t >= (long long)kPmPrimes * 2 * h) return;
    const int i = (int)(t % h), dir = (int)(t / h % 2), q = (int)(t / (2 * h));
    const u32 w = powm(dir ? c.iroot[q] : c.root[q], (u32)i, c.P[q]);
    tw[t] = make_uint2(w, (u32)(((u64)w << 32) / c.P[q].m));
}

// dst[q][e][k] = src[k][e] mod P_q for k <= d, 0 up to L = 2^lg (all indices
// below 2^31: 3 * 32^2 * 2^15 entries at most)
__global__ void k_pm_load(const u32 *__restrict__ src, long long d, int s2, int lg, u32 *__restrict__ dst,
                          const __grid_constant__ PmConsts c)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kPmPrimes * s2 << lg) return;
    const int k = t & ((1 << lg) - 1), qe = t >> lg;
    const int e = qe % s2, q = qe / s2;
    const u32 v = k <= d ? src[(long long)k * s2 + e] : 0u;
    dst[t] = c.reduce_input ? v % c.P[q].m : v;
}

// One polynomial of length L per CTA, transformed in shared memory.
template <bool INV>
__global__ void __launch_bounds__(kNttThreads) k_ntt(u32 *__restrict__ data, int L, int s2, const uint2 *__restrict__ tw,
                                                     const __grid_constant__ PmConsts c)
{
    extern __shared__ u32 a[];
    const int q = blockIdx.x / s2;
    const u32 P = c.P[q].m;
    const uint2 *w = tw + ((size_t)q * 2 + (INV ? 1 : 0)) * (L / 2);
    u32 *g = data + (size_t)blockIdx.x * L;
    for (int i = threadIdx.x; i < L; i += kNttThreads) a[i] = g[i];
    __syncthreads();
    const int h = L / 2;
    if (!INV) {
        for (int lgl = __ffs(h) - 1; lgl >= 0; --lgl) {  // decimation in frequency, len = 2^lgl
            const int len = 1 << lgl, step = h >> lgl;
            for (int b0 = threadIdx.x; b0 < h; b0 += 8 * kNttThreads) {
                uint2 wv[8];  // this thread's twiddles, all requested before any is used
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int b = b0 + u * kNttThreads;
                    wv[u] = b < h ? __ldg(w + (b & (len - 1)) * step) : make_uint2(0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int b = b0 + u * kNttThreads;
                    if (b >= h) break;
                    const int j = b & (len - 1), i0 = ((b >> lgl) << (lgl + 1)) + j, i1 = i0 + len;
                    const u32 x0 = a[i0], x1 = a[i1];
                    a[i0] = x0 + x1 >= P ? x0 + x1 - P : x0 + x1;
                    a[i1] = mul_shoup(x0 >= x1 ? x0 - x1 : x0 + P - x1, wv[u].x, wv[u].y, P);
                }
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < L; i += kNttThreads) g[i] = a[i];
    } else {
        for (int lgl = 0; (1 << lgl) <= h; ++lgl) {  // decimation in time, len = 2^lgl
            const int len = 1 << lgl, step = h >> lgl;
            for (int b0 = threadIdx.x; b0 < h; b0 += 8 * kNttThreads) {
                uint2 wv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int b = b0 + u * kNttThreads;
                    wv[u] = b < h ? __ldg(w + (b & (len - 1)) * step) : make_uint2(0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int b = b0 + u * kNttThreads;
                    if (b >= h) break;
                    const int j = b & (len - 1), i0 = ((b >> lgl) << (lgl + 1)) + j, i1 = i0 + len;
                    const u32 x0 = a[i0], x1 = mul_shoup(a[i1], wv[u].x, wv[u].y, P);
                    a[i0] = x0 + x1 >= P ? x0 + x1 - P : x0 + x1;
                    a[i1] = x0 >= x1 ? x0 - x1 : x0 + P - x1;
                }
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < L; i += kNttThreads) g[i] = mul_shoup(a[i], c.linv[q], c.linv_q[q], P);
    }
}

// Ch[q][i s + j][t] = sum_k Ah[q][i s + k][t] Bh[q][k s + j][t] mod P_q.  A CTA
// takes TP consecutive points of one prime: the s x s matrices of A and B at
// those points are read once into shared memory, [entry][point], and every
// output is formed there.
constexpr int kPwThreads = 256;

__global__ void __launch_bounds__(kPwThreads) k_pm_pointwise(const u32 *__restrict__ Ah, const u32 *__restrict__ Bh,
                                                            u32 *__restrict__ Ch, int s, int L, int lgtp,
                                                            const __grid_constant__ PmConsts c)
{
    const int TP = 1 << lgtp;
    extern __shared__ u32 pw[];
    const int s2 = s * s;
    u32 *As = pw, *Bs = pw + (size_t)s2 * TP;
    const int nblk = (L + TP - 1) / TP;
    const int q = blockIdx.x / nblk, t0 = (blockIdx.x % nblk) * TP;
    const int tp = min(TP, L - t0);
    const Mod &M = c.P[q];
    const u32 *ag = Ah + (size_t)q * s2 * L + t0, *bg = Bh + (size_t)q * s2 * L + t0;
    for (int idx = threadIdx.x; idx < s2 * TP; idx += kPwThreads) {
        const int e = idx >> lgtp, tt = idx & (TP - 1);
        As[idx] = tt < tp ? ag[(size_t)e * L + tt] : 0u;
        Bs[idx] = tt < tp ? bg[(size_t)e * L + tt] : 0u;
    }
    __syncthreads();
    u32 *cg = Ch + (size_t)q * s2 * L + t0;
    for (int o = threadIdx.x; o < s2 * TP; o += kPwThreads) {
        const int e = o >> lgtp, tt = o & (TP - 1);
        if (tt >= tp) continue;
        const int i = e / s, j = e % s;
        const u32 *ar = As + (size_t)i * s * TP + tt, *bc = Bs + (size_t)j * TP + tt;
        u64 acc = 0;
        u32 r = 0;
        for (int k = 0; k < s; ++k) {
            acc += (u64)ar[(size_t)k * TP] * bc[(size_t)k * s * TP];  // each below 2^60
            if ((k & 7) == 7) {
                r = red64((u64)r + red64(acc, M), M);
                acc = 0;
            }
        }
        cg[(size_t)e * L + tt] = red64((u64)r + red64(acc, M), M);
    }
}

// C[k][e] = the integer with residues Ch[0..2][e][k], mod p (Garner)
__global__ void k_pm_crt(const u32 *__restrict__ Ch, u32 *__restrict__ C, long long dc, int s2, int L,
                         const __grid_constant__ PmConsts c)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int)(dc + 1) * s2) return;
    const int e = t % s2, k = t / s2;
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
    *bytes = 3LL * kPmPrimes * s * s * L * 4 + (long long)kPmPrimes * L * 8 + 256;
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
        c.linv_q[q] = (u32)(((u64)c.linv[q] << 32) / P);
    }
    c.reduce_input = p > std::min({kPmP[0], kPmP[1], kPmP[2]}) ? 1 : 0;
    c.mp = make_mod(p, 1, 0);
    c.inv01 = powmod_host(kPmP[0] % kPmP[1], kPmP[1] - 2, kPmP[1]);
    c.inv02 = powmod_host(kPmP[0] % kPmP[2], kPmP[2] - 2, kPmP[2]);
    c.inv12 = powmod_host(kPmP[1] % kPmP[2], kPmP[2] - 2, kPmP[2]);
    c.p0_mod_p = (u32)(kPmP[0] % p);
    c.p0p1_mod_p = (u32)((unsigned __int128)kPmP[0] * kPmP[1] % p);

    cudaStream_t st = (cudaStream_t)stream;
    const size_t plane = (size_t)kPmPrimes * s2 * L;
    u32 *Ah = (u32 *)d_work, *Bh = Ah + plane, *Ch = Bh + plane;
    uint2 *tw = reinterpret_cast<uint2 *>(Ch + plane);  // 8-byte aligned: plane is a multiple of 2
    const int T = 256;
    auto blocks = [&](long long n) { return (unsigned)((n + T - 1) / T); };
    k_pm_twiddles<<<blocks((long long)kPmPrimes * L), T, 0, st>>>(tw, L, c);
    k_pm_load<<<blocks(plane), T, 0, st>>>(d_A, da, s2, lg, Ah, c);
    k_pm_load<<<blocks(plane), T, 0, st>>>(d_B, db, s2, lg, Bh, c);
    FF_CUDA(cudaGetLastError());
    const size_t smem = (size_t)L * 4;
    FF_CUDA(cudaFuncSetAttribute(k_ntt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FF_CUDA(cudaFuncSetAttribute(k_ntt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_ntt<false><<<(unsigned)(kPmPrimes * s2), kNttThreads, smem, st>>>(Ah, L, s2, tw, c);
    k_ntt<false><<<(unsigned)(kPmPrimes * s2), kNttThreads, smem, st>>>(Bh, L, s2, tw, c);
    // points per CTA: both s x s tiles in at most 64 KB of shared memory
    int lgtp = 5;  // 32 points per CTA, fewer when s^2 is large
    while (lgtp > 0 && ((size_t)s2 << lgtp) > 8192) --lgtp;
    const int TP = 1 << lgtp;
    const size_t pw_smem = (size_t)2 * s2 * TP * 4;
    FF_CUDA(cudaFuncSetAttribute(k_pm_pointwise, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pw_smem));
    k_pm_pointwise<<<(unsigned)(kPmPrimes * ((L + TP - 1) / TP)), kPwThreads, pw_smem, st>>>(Ah, Bh, Ch, s, L, lgtp, c);
    k_ntt<true><<<(unsigned)(kPmPrimes * s2), kNttThreads, smem, st>>>(Ch, L, s2, tw, c);
    k_pm_crt<<<blocks((da + db + 1) * s2), T, 0, st>>>(Ch, d_C, da + db, s2, L, c);
    FF_CUDA(cudaGetLastError());
    return FFSPMV_OK;
}
