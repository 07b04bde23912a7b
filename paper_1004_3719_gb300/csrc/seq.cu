// The block Wiedemann matrix sequence S_i = X^T A^i Y (mod p), Sec. 3 step 1,
// kept on the device as Sec. 2.5.2 asks.
//
// Persistent path (p <= 2^16, s <= 16, A square and splittable into a few
// dense diagonals plus a narrow ELL_R part): one cooperative kernel runs every
// step.  CTA c owns a contiguous slice of rows; per step it forms its rows of
// V_{i+1} = A V_i (DIA + ELL_R, Sec. 2.4.4), stores them, and projects them on
// the matching rows of X with tensor-core MMAs on 8-bit limbs; a bounded grid
// barrier then publishes V_{i+1} and the per-CTA partial projections, which
// the CTAs sum into S_{i+1}.  The kernel is captured in a CUDA graph.
//
// Per-launch path (everything else): for every step one projection launch and
// the plan's SpMM launches.
//
// Exactness of the projection on tensor cores: a residue v < 2^16 splits as
// v = 256*h + l with h, l < 256, both exact in fp16; one m16n8k16 MMA sums 16
// products below 2^16 each, so its fp32 result (< 2^20) is an exact integer,
// converted to u64 at once and weighted by 1, 256 or 65536.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "ff_internal.cuh"
#include "ff_select.h"

namespace ff {

namespace {

constexpr int kSeqThreads = 512;
constexpr int kS = 16;                            // block width of the persistent kernel
constexpr int kCPT = 8;                           // components per thread
constexpr int kTPR = kS / kCPT;                   // threads per row
constexpr int kRowsPerPass = kSeqThreads / kTPR;  // 256
constexpr int kMaxEnt = 16;                       // DIA + ELL_R entries per row
constexpr int kBatch = 10;                        // entries gathered together per thread
constexpr int kVsStride = 20;                     // halves per staged row (no bank conflicts)
constexpr size_t kXfSmemMax = 160 * 1024;         // shared memory for resident X fragments
constexpr unsigned kDefaultSpins = 1u << 22;      // x <= 64 ns sleeps: well under a second

struct SeqArgs {
    long long n;
    int ndiag, width, s;
    long long ld;
    long long nsteps;
    const int *doff;
    const unsigned short *dval;
    const u32 *col;
    const unsigned short *val;
    const u32 *rownb;
    const uint4 *XF;           // X limbs in MMA A-fragment order: [n/16][limb][lane]
    unsigned short *V0, *V1;   // n x 16
    u32 *partial;              // [2][nblocks][256]
    u32 *S;
    u32 *Vnext;
    unsigned *bar;             // [0] arrivals, [1] generation
    int *status;               // [0] timeout flag
    unsigned spin_limit;
    int test_skip;
    int xf_smem;               // X fragments of the CTA's rows held in shared memory
    int mat_smem;              // the CTA's rows of the matrix held in shared memory
    int mrows;                 // rows of one CTA's resident matrix slice (capacity)
    int mat_off;               // byte offset of that slice in dynamic shared memory
    Mod M;
};

// A CTA's rows of the DIA + ELL_R layout, resident in shared memory for the
// whole launch (the matrix is the same at every step): entry-major like the
// global arrays, row index relative to the CTA's first row.
struct MatSlice {
    const unsigned short *dval;  // [ndiag][mrows]
    const u32 *col;              // [width][mrows]
    const unsigned short *val;   // [width][mrows]
    const u32 *rownb;            // [mrows], or null when all rows have `width` entries
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_int(const int *p)
{
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier with a bounded wait.  The arrival counter (zeroed before the
// launch) only grows: barrier number `epoch` is passed once it reaches
// epoch * gridDim.x.  One thread per CTA adds its arrival with release order
// (after the CTA's __syncthreads, so it publishes the whole CTA's writes) and
// polls with acquire loads.  Returns false (and sets status[0]) when the wait
// ran out or another CTA already gave up.
__device__ bool grid_barrier(const SeqArgs &a, bool skip, unsigned &epoch)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        ++epoch;
        if (!skip) {
            const unsigned target = epoch * gridDim.x;
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.bar) : "memory");
            unsigned it = 0;
            while ((int)(ld_acquire(a.bar) - target) < 0) {
                if (++it > a.spin_limit || ((it & 255u) == 0 && ld_volatile_int(a.status) != 0)) {
                    atomicExch(a.status, 1);
                    ok = 0;
                    break;
                }
                if (it > 64) __nanosleep(32);
            }
        } else {
            // test hook: never arrive; wait (bounded) for the others to give up
            unsigned it = 0;
            while (ld_volatile_int(a.status) == 0 && ++it <= a.spin_limit) __nanosleep(64);
            atomicExch(a.status, 1);
            ok = 0;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Two 8-bit integers (bits 0-7 and 16-23 of p) as an exact f16x2 pair:
// 0x6400 | b is the half 1024 + b, and subtracting 1024 is exact.
__device__ __forceinline__ u32 bytes_to_half2(u32 p)
{
    u32 r;
    asm("sub.f16x2 %0, %1, %2;" : "=r"(r) : "r"(p | 0x64006400u), "r"(0x64006400u));
    return r;
}

// An exact non-negative integer below 2^23 held in an fp32, as u32.
__device__ __forceinline__ u32 f32_to_u32(float f)
{
    return __float_as_uint(f + 8388608.0f) - 0x4B000000u;
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint4 &A, u32 b0, u32 b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(A.x), "r"(A.y), "r"(A.z), "r"(A.w), "r"(b0), "r"(b1),
          "f"(0.f), "f"(0.f), "f"(0.f), "f"(0.f));
}

struct __align__(16) SeqSmem {
    union {
        unsigned short vs[2][kRowsPerPass][kVsStride];  // staged V rows, double buffered
        u32 red[kSeqThreads / 32][kS * kS];             // per-warp partial projections
    };
    int doff[kMaxEnt];
};

// V_out rows [r0, r1) = A * V_in (when `compute`), and, when `project`, the
// partial X^T V_out over those rows accumulated in pacc.  Two threads share a
// row (8 components each); warp w then runs k-step w of every 256-row pass
// with both X limbs against both V limbs (8 MMAs).  Indices are 32-bit: the
// layout guarantees 16 n < 2^31.
__device__ void spmm_and_project(const SeqArgs &a, SeqSmem &sm, const uint4 *xfs, const MatSlice &ms,
                                 const unsigned short *Vin, unsigned short *Vout, int r0, int r1,
                                 bool compute, bool project, u32 (&pacc)[2][2][4])
{
    const int R = a.mrows;
    const int rip = threadIdx.x / kTPR;
    const int c0 = (threadIdx.x % kTPR) * kCPT;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int nd = a.ndiag, n = (int)a.n, ld = (int)a.ld;
    int pass = 0;
    for (int base = r0; base < r1; base += kRowsPerPass, ++pass) {
        const int row = base + rip;
        uint4 outq = make_uint4(0u, 0u, 0u, 0u);
        if (row < r1) {
            if (compute) {
                const int lr = row - r0;
                const int ntot =
                    nd + (a.rownb ? (a.mat_smem ? (int)ms.rownb[lr] : (int)__ldg(a.rownb + row)) : a.width);
                u64 acc[kCPT];
#pragma unroll
                for (int k = 0; k < kCPT; ++k) acc[k] = 0;
#pragma unroll
                for (int e0 = 0; e0 < kMaxEnt; e0 += kBatch) {
                    if (e0 >= ntot) break;
                    uint4 q[kBatch];
                    u32 v[kBatch];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const int e = e0 + u;
                        q[u] = make_uint4(0u, 0u, 0u, 0u);
                        v[u] = 0;
                        if (e < nd) {
                            const int j = row + sm.doff[e];
                            if ((unsigned)j < (unsigned)n) {
                                v[u] = a.mat_smem ? ms.dval[e * R + lr] : __ldg(a.dval + e * ld + row);
                                q[u] = __ldcg(reinterpret_cast<const uint4 *>(Vin + j * kS + c0));
                            }
                        } else if (e < ntot) {
                            int j;
                            if (a.mat_smem) {
                                const int li = (e - nd) * R + lr;
                                j = (int)ms.col[li];
                                v[u] = ms.val[li];
                            } else {
                                const int idx = (e - nd) * ld + row;
                                j = (int)__ldg(a.col + idx);
                                v[u] = __ldg(a.val + idx);
                            }
                            q[u] = __ldcg(reinterpret_cast<const uint4 *>(Vin + j * kS + c0));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const u32 qq[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            acc[2 * k] += (u64)v[u] * (qq[k] & 0xffffu);
                            acc[2 * k + 1] += (u64)v[u] * (qq[k] >> 16);
                        }
                    }
                }
                outq.x = red64(acc[0], a.M) | (red64(acc[1], a.M) << 16);
                outq.y = red64(acc[2], a.M) | (red64(acc[3], a.M) << 16);
                outq.z = red64(acc[4], a.M) | (red64(acc[5], a.M) << 16);
                outq.w = red64(acc[6], a.M) | (red64(acc[7], a.M) << 16);
                *reinterpret_cast<uint4 *>(Vout + row * kS + c0) = outq;
            } else {
                outq = __ldcg(reinterpret_cast<const uint4 *>(Vin + row * kS + c0));
            }
        }
        if (!project) continue;
        unsigned short(*vs)[kVsStride] = sm.vs[pass & 1];
        *reinterpret_cast<uint2 *>(&vs[rip][c0]) = make_uint2(outq.x, outq.y);
        *reinterpret_cast<uint2 *>(&vs[rip][c0 + 4]) = make_uint2(outq.z, outq.w);
        __syncthreads();
        // each pass adds below 2^29 per element: reduce every 4 passes
        if ((pass & 3) == 3) {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) pacc[i][j][e] = red64(pacc[i][j][e], a.M);
        }
        const int q16 = (base >> 4) + w;
        if (q16 * 16 < r1) {
            uint4 A0, A1;
            if (a.xf_smem) {
                const uint4 *f = xfs + ((size_t)(q16 - (r0 >> 4)) * 2) * 32 + lane;
                A0 = f[0];
                A1 = f[32];
            } else {
                A0 = __ldg(a.XF + ((size_t)q16 * 2 + 0) * 32 + lane);
                A1 = __ldg(a.XF + ((size_t)q16 * 2 + 1) * 32 + lane);
            }
            const int k0 = w * 16;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int nn = nt * 8 + g;
                const u32 p0 = vs[k0 + 2 * t][nn] | ((u32)vs[k0 + 2 * t + 1][nn] << 16);
                const u32 p1 = vs[k0 + 2 * t + 8][nn] | ((u32)vs[k0 + 2 * t + 9][nn] << 16);
#pragma unroll
                for (int vl = 0; vl < 2; ++vl) {
                    const u32 b0 = bytes_to_half2(vl ? (p0 >> 8) & 0x00ff00ffu : p0 & 0x00ff00ffu);
                    const u32 b1 = bytes_to_half2(vl ? (p1 >> 8) & 0x00ff00ffu : p1 & 0x00ff00ffu);
                    float d0[4], d1[4];
                    mma16816(d0, A0, b0, b1);
                    mma16816(d1, A1, b0, b1);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        pacc[vl][nt][e] += f32_to_u32(d0[e]) + (f32_to_u32(d1[e]) << 8);
                }
            }
        }
    }
}

// Add the warps' fragments into sm.acc, then write this CTA's partial
// projection (reduced) and clear the accumulators.
__device__ void publish_partial(const SeqArgs &a, SeqSmem &sm, int buf, u32 (&pacc)[2][2][4])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    __syncthreads();  // the last pass's MMAs have read the staged rows
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int b = nt * 8 + 2 * t;
        u32 c[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            c[e] = red64((u64)pacc[0][nt][e] + ((u64)pacc[1][nt][e] << 8), a.M);  // V limb weights 1, 256
            pacc[0][nt][e] = pacc[1][nt][e] = 0;
        }
        sm.red[w][g * kS + b] = c[0];
        sm.red[w][g * kS + b + 1] = c[1];
        sm.red[w][(g + 8) * kS + b] = c[2];
        sm.red[w][(g + 8) * kS + b + 1] = c[3];
    }
    __syncthreads();
    u32 *dst = a.partial + ((size_t)buf * gridDim.x + blockIdx.x) * (kS * kS);
    for (int o = threadIdx.x; o < kS * kS; o += blockDim.x) {
        u64 tot = 0;
#pragma unroll
        for (int i = 0; i < kSeqThreads / 32; ++i) tot += sm.red[i][o];
        dst[o] = red64(tot, a.M);
    }
    __syncthreads();  // sm.red aliases the staging rows of the next step
}

// S_step[o] = sum over CTAs of their partials (mod p); one warp per output,
// output o on warp o / gridDim.x of CTA o % gridDim.x, so that every CTA has
// at most two.
__device__ void reduce_step(const SeqArgs &a, int buf, long long step)
{
    const int nb = gridDim.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const u32 *src = a.partial + (size_t)buf * nb * (kS * kS);
    for (int o = blockIdx.x + w * nb; o < kS * kS; o += nb * nw) {
        u64 s = 0;
        for (int c = lane; c < nb; c += 32) s += __ldcg(src + (size_t)c * (kS * kS) + o);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        const int ai = o / kS, bi = o % kS;
        if (lane == 0 && ai < a.s && bi < a.s) a.S[(step * a.s + ai) * a.s + bi] = red64(s, a.M);
    }
}

__global__ void __launch_bounds__(kSeqThreads, 1) k_sequence(const __grid_constant__ SeqArgs a)
{
    __shared__ SeqSmem sm;
    extern __shared__ uint4 xfs[];  // X fragments of this CTA's 16-row groups (if they fit)
    if (threadIdx.x < kMaxEnt) sm.doff[threadIdx.x] = threadIdx.x < a.ndiag ? a.doff[threadIdx.x] : 0;
    __syncthreads();
    const long long nb = gridDim.x;
    // 16-row aligned slices, so that every k-step covers one 16-row group
    const int r0 = (int)(((a.n * blockIdx.x / nb) >> 4) << 4);
    const int r1 = blockIdx.x + 1 == nb ? (int)a.n : (int)(((a.n * (blockIdx.x + 1) / nb) >> 4) << 4);
    if (a.nsteps <= 0 && !a.Vnext) return;
    if (a.xf_smem) {
        // constant across steps: keep the CTA's X fragments resident
        const int q0 = r0 >> 4, q1 = (r1 + 15) >> 4;
        for (int t = threadIdx.x; t < (q1 - q0) * 64; t += blockDim.x) xfs[t] = __ldg(a.XF + (size_t)q0 * 64 + t);
    }
    MatSlice ms = {nullptr, nullptr, nullptr, nullptr};
    if (a.mat_smem) {
        // constant across steps too: the CTA's rows of the matrix
        unsigned char *base = reinterpret_cast<unsigned char *>(xfs) + a.mat_off;
        const int R = a.mrows, nr = r1 - r0, ld = (int)a.ld;
        const size_t b_d = ((size_t)a.ndiag * R * 2 + 15) / 16 * 16, b_c = (size_t)a.width * R * 4;
        const size_t b_v = ((size_t)a.width * R * 2 + 15) / 16 * 16;
        unsigned short *dv = reinterpret_cast<unsigned short *>(base);
        u32 *cl = reinterpret_cast<u32 *>(base + b_d);
        unsigned short *vl = reinterpret_cast<unsigned short *>(base + b_d + b_c);
        u32 *rb = a.rownb ? reinterpret_cast<u32 *>(base + b_d + b_c + b_v) : nullptr;
        for (int t = threadIdx.x; t < a.ndiag * nr; t += blockDim.x) {
            const int e = t / nr, r = t - e * nr;
            dv[e * R + r] = __ldg(a.dval + (size_t)e * ld + r0 + r);
        }
        for (int t = threadIdx.x; t < a.width * nr; t += blockDim.x) {
            const int e = t / nr, r = t - e * nr;
            cl[e * R + r] = __ldg(a.col + (size_t)e * ld + r0 + r);
            vl[e * R + r] = __ldg(a.val + (size_t)e * ld + r0 + r);
        }
        if (rb)
            for (int r = threadIdx.x; r < nr; r += blockDim.x) rb[r] = __ldg(a.rownb + r0 + r);
        ms.dval = dv;
        ms.col = cl;
        ms.val = vl;
        ms.rownb = rb;
    }
    __syncthreads();
    const bool skip = a.test_skip && blockIdx.x == 0;
    unsigned epoch = 0;  // grid barriers passed (thread 0)
    u32 pacc[2][2][4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int e = 0; e < 4; ++e) pacc[i][j][e] = 0;
    // The partials of S_j are summed during the next step, after its SpMM and
    // before its barrier (they sit in buffer j & 1, which is written again only
    // after that barrier), so no CTA starts a step late.
    long long pending = -1;  // step whose partials are published but not yet summed
    // S_0 = X^T Y
    if (a.nsteps > 0) {
        spmm_and_project(a, sm, xfs, ms, a.V0, a.V0, r0, r1, false, true, pacc);
        publish_partial(a, sm, 0, pacc);
        if (!grid_barrier(a, skip, epoch)) return;
        pending = 0;
    }
    long long done = 0;  // SpMMs done: V_done is current
    for (long long i = 0; i < a.nsteps; ++i) {
        const bool need = (i + 1 < a.nsteps) || a.Vnext;
        if (!need) break;
        const unsigned short *Vin = (i & 1) ? a.V1 : a.V0;
        unsigned short *Vout = (i & 1) ? a.V0 : a.V1;
        const bool proj = i + 1 < a.nsteps;
        spmm_and_project(a, sm, xfs, ms, Vin, Vout, r0, r1, true, proj, pacc);
        if (pending >= 0) reduce_step(a, (int)(pending & 1), pending);
        pending = -1;
        if (proj) publish_partial(a, sm, (int)((i + 1) & 1), pacc);
        if (!grid_barrier(a, false, epoch)) return;
        done = i + 1;
        if (proj) pending = i + 1;
    }
    if (pending >= 0) reduce_step(a, (int)(pending & 1), pending);
    if (a.Vnext) {
        const unsigned short *Vf = (done & 1) ? a.V1 : a.V0;
        for (long long t = (long long)r0 * a.s + threadIdx.x; t < (long long)r1 * a.s; t += blockDim.x) {
            const long long row = t / a.s;
            const int c = (int)(t - row * a.s);
            a.Vnext[t] = __ldcg(Vf + row * kS + c);
        }
    }
}

// Y (n x s, u32) -> V0 (n x 16, u16, zero padded, reduced mod p).
__global__ void k_seq_prepare_v(long long n, int s, const u32 *__restrict__ Y,
                                unsigned short *V0, const Mod M)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * kS) return;
    const long long row = t / kS;
    const int c = (int)(t - row * kS);
    V0[t] = (unsigned short)(c < s ? red64(Y[row * s + c], M) : 0u);
}

// X (n x s, u32) -> its 8-bit limbs in m16n8k16 A-fragment order: for the
// 16-row group q, limb l and lane (g = lane/4, t = lane%4) the four f16x2
// words hold A[g][2t..2t+1], A[g+8][2t..2t+1], A[g][2t+8..9], A[g+8][2t+8..9]
// with A[a][k] = limb l of X[16q + k][a] (rows past n are zero).
__global__ void k_seq_prepare_x(long long n, int s, const u32 *__restrict__ X, uint4 *XF,
                                const Mod M)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nq = (n + 15) / 16;
    if (t >= nq * 2 * 32) return;
    const int lane = (int)(t & 31);
    const int l = (int)((t >> 5) & 1);
    const long long q = t >> 6;
    const int g = lane >> 2, tt = lane & 3;
    auto limb = [&](int k, int col) -> u32 {
        const long long row = q * 16 + k;
        if (row >= n || col >= s) return 0u;
        const u32 v = red64(X[row * s + col], M);
        return l ? (v >> 8) & 255u : v & 255u;
    };
    auto pair = [&](int k, int col) -> u32 {
        return bytes_to_half2(limb(k, col) | (limb(k + 1, col) << 16));
    };
    uint4 r;
    r.x = pair(2 * tt, g);
    r.y = pair(2 * tt, g + 8);
    r.z = pair(2 * tt + 8, g);
    r.w = pair(2 * tt + 8, g + 8);
    XF[t] = r;
}

// ---------------------------------------------------------------------------
// Per-launch path: projection S_step = X^T V (any p, s <= 32).
template <class Acc>
__global__ void __launch_bounds__(256) k_project(long long n, int s, const u32 *__restrict__ X,
                                                 const u32 *__restrict__ V, u64 *__restrict__ Sacc,
                                                 const Mod M)
{
    const int outs = s * s;
    for (int o = threadIdx.x; o < outs; o += blockDim.x) {
        const int ai = o / s, bi = o % s;
        Acc acc;
        acc.zero();
        for (long long k = blockIdx.x; k < n; k += gridDim.x)
            acc.mad(__ldg(X + k * s + ai), __ldg(V + k * s + bi));
        u64 part = acc.partial(M);
        atomicAdd(Sacc + o, (u64)red64(part, M));
    }
}

__global__ void k_project_finish(int outs, u64 *Sacc, u32 *S, const Mod M)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= outs) return;
    S[o] = red64(Sacc[o], M);
    Sacc[o] = 0;
}

__global__ void k_reduce_copy(long long n, const u32 *__restrict__ src, u32 *__restrict__ dst,
                              const Mod M)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = red64(src[t], M);
}

}  // namespace

// ---------------------------------------------------------------------------
struct SeqState {
    // DIA + ELL_R layout
    bool layout_tried = false, layout_ok = false;
    long long n = 0;
    int ndiag = 0, width = 0;
    long long ld = 0;
    void *arena = nullptr;
    const int *doff = nullptr;
    const unsigned short *dval = nullptr;
    const u32 *col = nullptr;
    const unsigned short *val = nullptr;
    const u32 *rownb = nullptr;
    // work buffers
    void *work = nullptr;
    size_t work_bytes = 0;
    uint4 *XF = nullptr;
    unsigned short *V0 = nullptr, *V1 = nullptr;
    u32 *partial = nullptr;
    unsigned *bar = nullptr;
    int nblocks = 0;
    // per-launch path buffers
    void *gwork = nullptr;
    size_t gwork_bytes = 0;
    // graph cache: the kernel arguments and the two input blocks that the
    // captured preparation launches read
    cudaGraphExec_t exec = nullptr;
    SeqArgs key;
    const u32 *key_X = nullptr, *key_Y = nullptr;
};

void free_sequence_state(ffspmv_handle *h)
{
    SeqState *q = (SeqState *)h->seq_state;
    if (!q) return;
    if (q->exec) cudaGraphExecDestroy(q->exec);
    if (q->arena) cudaFree(q->arena);
    if (q->work) cudaFree(q->work);
    if (q->gwork) cudaFree(q->gwork);
    delete q;
    h->seq_state = nullptr;
}

namespace {

// Split A into its densest diagonals (DIA) and an ELL_R part for the rest.
bool build_seq_layout(ffspmv_handle *h, SeqState &q)
{
    const long long n = h->A.nrows;
    const long long *ptr = h->h_ptr.data();
    const int *col = h->h_col.data();
    const u32 *val = h->h_val.data();
    std::vector<long long> cnt((size_t)(2 * n + 1), 0);
    for (long long i = 0; i < n; ++i)
        for (long long k = ptr[i]; k < ptr[i + 1]; ++k) cnt[(size_t)(col[k] - i + n)]++;
    std::vector<std::pair<long long, int>> cand;
    for (size_t t = 0; t < cnt.size(); ++t) {
        long long off = (long long)t - n;
        long long len = n - (off < 0 ? -off : off);
        if (cnt[t] && len * 4 >= n && cnt[t] * 2 >= len) cand.push_back({cnt[t], (int)off});
    }
    std::sort(cand.begin(), cand.end(), [](auto &x, auto &y) { return x.first > y.first; });
    std::vector<int> diag;
    for (size_t i = 0; i < cand.size() && i < 8; ++i) diag.push_back(cand[i].second);
    std::sort(diag.begin(), diag.end());
    const long long ld = (n + 31) / 32 * 32;
    std::vector<unsigned short> dval(diag.size() * ld, 0);
    std::vector<long long> rest(n, 0);
    long long width = 0;
    for (long long i = 0; i < n; ++i) {
        for (long long k = ptr[i]; k < ptr[i + 1]; ++k) {
            long long off = col[k] - i;
            auto it = std::find(diag.begin(), diag.end(), (int)off);
            if (it != diag.end()) {
                size_t idx = (size_t)(it - diag.begin()) * ld + i;
                dval[idx] = (unsigned short)(((u64)dval[idx] + val[k]) % h->m);
            } else {
                rest[i]++;
            }
        }
        width = std::max(width, rest[i]);
    }
    if (width + (long long)diag.size() > kMaxEnt) return false;  // short rows only
    if (n * kS >= (1LL << 31) || width * ld >= (1LL << 31)) return false;  // 32-bit indices
    std::vector<u32> ecol((size_t)(width * ld), 0), rownb(n);
    std::vector<unsigned short> eval((size_t)(width * ld), 0);
    bool uniform = true;
    for (long long i = 0; i < n; ++i) {
        long long j = 0;
        for (long long k = ptr[i]; k < ptr[i + 1]; ++k) {
            long long off = col[k] - i;
            if (std::find(diag.begin(), diag.end(), (int)off) != diag.end()) continue;
            ecol[(size_t)(j * ld + i)] = (u32)col[k];
            eval[(size_t)(j * ld + i)] = (unsigned short)val[k];
            ++j;
        }
        rownb[i] = (u32)j;
        if (j != width) uniform = false;
    }
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t o_doff = 0, o_dval = al(diag.size() * 4 + 4), o_col = o_dval + al(dval.size() * 2 + 2);
    size_t o_val = o_col + al(ecol.size() * 4 + 4), o_nb = o_val + al(eval.size() * 2 + 2);
    size_t total = o_nb + al(rownb.size() * 4 + 4);
    if (cudaMalloc(&q.arena, total) != cudaSuccess) {
        q.arena = nullptr;
        return false;
    }
    char *b = (char *)q.arena;
    cudaMemcpy(b + o_doff, diag.data(), diag.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(b + o_dval, dval.data(), dval.size() * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(b + o_col, ecol.data(), ecol.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(b + o_val, eval.data(), eval.size() * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(b + o_nb, rownb.data(), rownb.size() * 4, cudaMemcpyHostToDevice);
    q.n = n;
    q.ndiag = (int)diag.size();
    q.width = (int)width;
    q.ld = ld;
    q.doff = (const int *)(b + o_doff);
    q.dval = (const unsigned short *)(b + o_dval);
    q.col = (const u32 *)(b + o_col);
    q.val = (const unsigned short *)(b + o_val);
    q.rownb = uniform ? nullptr : (const u32 *)(b + o_nb);
    return cudaGetLastError() == cudaSuccess;
}

ffspmv_status ensure_work(SeqState &q, long long n, int nblocks)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t nq = (size_t)((n + 15) / 16);
    size_t xb = al(nq * 64 * sizeof(uint4));
    size_t vb = al((size_t)n * kS * 2 + 16);
    size_t pb = al((size_t)2 * nblocks * kS * kS * 4);
    size_t need = xb + 2 * vb + pb + 256;
    if (need > q.work_bytes) {
        if (q.work) cudaFree(q.work);
        q.work = nullptr;
        q.work_bytes = 0;
        if (cudaMalloc(&q.work, need) != cudaSuccess) return FFSPMV_ERR_OOM;
        q.work_bytes = need;
    }
    char *b = (char *)q.work;
    q.XF = (uint4 *)b;
    q.V0 = (unsigned short *)(b + xb);
    q.V1 = (unsigned short *)(b + xb + vb);
    q.partial = (u32 *)(b + xb + 2 * vb);
    q.bar = (unsigned *)(b + xb + 2 * vb + pb);
    q.nblocks = nblocks;
    return FFSPMV_OK;
}

ffspmv_status sequence_per_launch(ffspmv_handle *h, SeqState &q, const u32 *X, const u32 *Y,
                                  int s, long long nsteps, u32 *S, u32 *Vnext, cudaStream_t st)
{
    const long long n = h->A.nrows;
    const Mod M = make_mod(h->m, 1, 0);
    size_t vb = ((size_t)n * s * 4 + 255) / 256 * 256 + 256;
    size_t need = 2 * vb + (size_t)s * s * 8 + 256;
    if (need > q.gwork_bytes) {
        if (q.gwork) cudaFree(q.gwork);
        q.gwork = nullptr;
        q.gwork_bytes = 0;
        if (cudaMalloc(&q.gwork, need) != cudaSuccess) return FFSPMV_ERR_OOM;
        q.gwork_bytes = need;
        FF_CUDA(cudaMemset(q.gwork, 0, need));
    }
    u32 *V[2] = {(u32 *)q.gwork, (u32 *)((char *)q.gwork + vb)};
    u64 *Sacc = (u64 *)((char *)q.gwork + 2 * vb);
    if (n > 0) {
        k_reduce_copy<<<(unsigned)((n * s + 255) / 256), 256, 0, st>>>(n * s, Y, V[0], M);
        FF_CUDA(cudaGetLastError());
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned pg = (unsigned)std::max<long long>(1, std::min<long long>(n, (long long)nsm));
    const int outs = s * s;
    const bool wide = (unsigned long long)(h->m - 1) * (h->m - 1) >
                      (~0ull) / (unsigned long long)std::max<long long>(n, 1);
    for (long long i = 0; i < nsteps; ++i) {
        const u32 *Vi = V[i & 1];
        if (n > 0) {
            if (wide)
                k_project<AccWide><<<pg, 256, 0, st>>>(n, s, X, Vi, Sacc, M);
            else
                k_project<AccSmall><<<pg, 256, 0, st>>>(n, s, X, Vi, Sacc, M);
            FF_CUDA(cudaGetLastError());
        }
        k_project_finish<<<(outs + 255) / 256, 256, 0, st>>>(outs, Sacc, S + i * outs, M);
        FF_CUDA(cudaGetLastError());
        if (i + 1 < nsteps || Vnext) {
            ffspmv_status r = run_plan(h->A, Vi, s, V[(i + 1) & 1], s, s, h->m, 1, 0, st);
            if (r != FFSPMV_OK) return r;
        }
    }
    if (Vnext && n > 0) {
        FF_CUDA(cudaMemcpyAsync(Vnext, V[nsteps & 1], (size_t)n * s * 4,
                                cudaMemcpyDeviceToDevice, st));
    }
    FF_CUDA(cudaStreamSynchronize(st));
    return FFSPMV_OK;
}

bool same_key(const SeqArgs &a, const SeqArgs &b)
{
    return memcmp(&a, &b, sizeof(SeqArgs)) == 0;
}

}  // namespace

}  // namespace ff

using namespace ff;

extern "C" ffspmv_status spmv_block_sequence(ffspmv_t h, const uint32_t *d_X, const uint32_t *d_Y,
                                             int32_t s, int64_t start_step, int64_t nsteps,
                                             uint32_t *d_S, uint32_t *d_V_state,
                                             ffspmv_stream_t stream)
{
    if (!h || s < 1 || s > 32 || nsteps < 0 || start_step < 0) return FFSPMV_ERR_ARG;
    if (h->A.nrows != h->A.ncols) return FFSPMV_ERR_ARG;
    const long long n = h->A.nrows;
    // a resumed sequence starts from the state an earlier call left in d_V_state
    if (start_step > 0 && !d_V_state) return FFSPMV_ERR_ARG;
    if (start_step > 0) d_Y = d_V_state;
    uint32_t *d_V_next = d_V_state;
    if (n > 0 && (!d_X || !d_Y)) return FFSPMV_ERR_ARG;
    if (nsteps > 0 && !d_S) return FFSPMV_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!h->seq_state) h->seq_state = new (std::nothrow) SeqState();
    SeqState *q = (SeqState *)h->seq_state;
    if (!q) return FFSPMV_ERR_OOM;

    bool persistent = h->opt.sequence_mode == 0 && h->m <= 65536u && s <= kS && n > 0 && nsteps > 0;
    if (persistent && !q->layout_tried) {
        q->layout_tried = true;
        q->layout_ok = build_seq_layout(h, *q);
    }
    persistent = persistent && q->layout_ok;
    int nblocks = 0;
    if (persistent) {
        int dev = 0, nsm = 0, per_sm = 0, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaFuncSetAttribute(k_sequence, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXfSmemMax);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sequence, kSeqThreads, kXfSmemMax);
        nblocks = nsm * std::min(per_sm, 1);
        if (!coop || per_sm < 1) persistent = false;
        // keep at least one pass of rows per CTA
        long long maxb = std::max<long long>(1, n / 16);
        if (nblocks > maxb) nblocks = (int)maxb;
    }
    if (!persistent) return sequence_per_launch(h, *q, d_X, d_Y, s, nsteps, d_S, d_V_next, st);

    ffspmv_status rs = ensure_work(*q, n, nblocks);
    if (rs != FFSPMV_OK) return rs;
    SeqArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.ndiag = q->ndiag;
    a.width = q->width;
    a.s = s;
    a.ld = q->ld;
    a.nsteps = nsteps;
    a.doff = q->doff;
    a.dval = q->dval;
    a.col = q->col;
    a.val = q->val;
    a.rownb = q->rownb;
    a.XF = q->XF;
    a.V0 = q->V0;
    a.V1 = q->V1;
    a.partial = q->partial;
    a.S = d_S;
    a.Vnext = d_V_next;
    a.bar = q->bar;
    a.status = h->d_status;
    a.spin_limit = h->opt.barrier_spin_limit ? h->opt.barrier_spin_limit : kDefaultSpins;
    a.test_skip = (h->opt.test_hooks & 1) ? 1 : 0;
    // X fragments of the largest CTA slice: 1 KB per 16-row group (+ 2 groups of rounding)
    const size_t xf_bytes = (size_t)((n + nblocks - 1) / nblocks / 16 + 2) * 64 * sizeof(uint4);
    a.xf_smem = xf_bytes <= kXfSmemMax ? 1 : 0;
    // the CTA's matrix rows as well, when they fit beside the X fragments
    a.mrows = (int)(((n + nblocks - 1) / nblocks / 16 + 2) * 16);
    const size_t mat_bytes = ((size_t)q->ndiag * a.mrows * 2 + 15) / 16 * 16 + (size_t)q->width * a.mrows * 4 +
                             ((size_t)q->width * a.mrows * 2 + 15) / 16 * 16 + (q->rownb ? (size_t)a.mrows * 4 : 0);
    a.mat_off = a.xf_smem ? (int)xf_bytes : 0;
    a.mat_smem = (size_t)a.mat_off + mat_bytes <= kXfSmemMax ? 1 : 0;
    const size_t dyn_smem = (size_t)a.mat_off + (a.mat_smem ? mat_bytes : 0);
    a.M = make_mod(h->m, 1, 0);

    // the graph: prepare X/Y, clear barrier + status, run the persistent kernel
    if (!q->exec || !same_key(a, q->key) || q->key_X != d_X || q->key_Y != d_Y) {
        if (q->exec) cudaGraphExecDestroy(q->exec);
        q->exec = nullptr;
        cudaStream_t cs;
        FF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const long long nxf = (n + 15) / 16 * 64;
            k_seq_prepare_x<<<(unsigned)((nxf + 255) / 256), 256, 0, cs>>>(n, s, d_X, q->XF, a.M);
            k_seq_prepare_v<<<(unsigned)((n * kS + 255) / 256), 256, 0, cs>>>(n, s, d_Y, q->V0, a.M);
            cudaMemsetAsync(q->bar, 0, 2 * sizeof(unsigned), cs);
            cudaMemsetAsync(h->d_status, 0, sizeof(int), cs);
            cudaLaunchConfig_t cfg;
            memset(&cfg, 0, sizeof(cfg));
            cfg.gridDim = dim3((unsigned)nblocks);
            cfg.blockDim = dim3(kSeqThreads);
            cfg.dynamicSmemBytes = dyn_smem;
            cfg.stream = cs;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeCooperative;
            at[0].val.cooperative = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            cudaError_t le = cudaLaunchKernelEx(&cfg, k_sequence, a);
            cudaError_t ce = cudaStreamEndCapture(cs, &g);
            ok = le == cudaSuccess && ce == cudaSuccess && g != nullptr;
            if (ok) ok = cudaGraphInstantiate(&q->exec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        cudaStreamDestroy(cs);
        if (!ok) {
            q->exec = nullptr;
            return sequence_per_launch(h, *q, d_X, d_Y, s, nsteps, d_S, d_V_next, st);
        }
        q->key = a;
        q->key_X = d_X;
        q->key_Y = d_Y;
    }
    FF_CUDA(cudaGraphLaunch(q->exec, st));
    int status = 0;
    FF_CUDA(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FF_CUDA(cudaStreamSynchronize(st));
    if (status != 0) {
        cudaMemset(h->d_status, 0, sizeof(int));
        return FFSPMV_ERR_TIMEOUT;
    }
    return FFSPMV_OK;
}

// The projection of one step on its own, for a sequence whose rows are split
// over several processes: each adds its rows' X^T V into a u64 accumulator,
// the accumulators are summed across processes, and the finish reduces them.
extern "C" ffspmv_status spmv_block_project(uint32_t p, int64_t n, int32_t s, const uint32_t *d_X,
                                            const uint32_t *d_V, uint64_t *d_Sacc, ffspmv_stream_t stream)
{
    if (p < 2 || n < 0 || s < 1 || s > 32 || !d_Sacc || (n > 0 && (!d_X || !d_V))) return FFSPMV_ERR_ARG;
    if (n == 0) return FFSPMV_OK;
    const Mod M = make_mod(p, 1, 0);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned pg = (unsigned)std::max<long long>(1, std::min<long long>(n, (long long)std::max(nsm, 1)));
    const bool wide = (unsigned long long)(p - 1) * (p - 1) > (~0ull) / (unsigned long long)n;
    if (wide)
        k_project<AccWide><<<pg, 256, 0, st>>>(n, s, d_X, d_V, (u64 *)d_Sacc, M);
    else
        k_project<AccSmall><<<pg, 256, 0, st>>>(n, s, d_X, d_V, (u64 *)d_Sacc, M);
    FF_CUDA(cudaGetLastError());
    return FFSPMV_OK;
}

extern "C" ffspmv_status spmv_block_project_finish(uint32_t p, int32_t s, uint64_t *d_Sacc, uint32_t *d_S,
                                                   ffspmv_stream_t stream)
{
    if (p < 2 || s < 1 || s > 32 || !d_Sacc || !d_S) return FFSPMV_ERR_ARG;
    const Mod M = make_mod(p, 1, 0);
    const int outs = s * s;
    k_project_finish<<<(outs + 255) / 256, 256, 0, (cudaStream_t)stream>>>(outs, (u64 *)d_Sacc, d_S, M);
    FF_CUDA(cudaGetLastError());
    return FFSPMV_OK;
}
