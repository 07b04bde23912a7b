// The block Wiedemann matrix sequence S_i = X^T A^i Y (mod p), Sec. 3 step 1,
// kept on the device as Sec. 2.5.2 asks.
//
// Persistent path (p <= 2^16, s <= 16, A square and splittable into a few
// dense diagonals plus a narrow ELL_R part): one cooperative kernel runs every
// step.  CTA c owns a contiguous slice of rows; per step it forms its rows of
// V_{i+1} = A V_i (DIA + ELL_R, Sec. 2.4.5), stores them, and projects them on
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
constexpr int kS = 16;                          // block width of the persistent kernel
constexpr int kCPT = 4;                         // components per thread
constexpr int kTPR = kS / kCPT;                 // threads per row
constexpr int kRowsPerPass = kSeqThreads / kTPR;  // 128
constexpr int kKSteps = kRowsPerPass / 16;        // 8 k-steps of 16 rows
constexpr unsigned kDefaultSpins = 1u << 22;      // x ~256 ns sleeps: about a second

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
    const unsigned short *Xh;  // n x 16
    unsigned short *V0, *V1;   // n x 16
    u32 *partial;              // [2][nblocks][256]
    u32 *S;
    u32 *Vnext;
    unsigned *bar;             // [0] arrivals, [1] generation
    int *status;               // [0] timeout flag
    unsigned spin_limit;
    int test_skip;
    Mod M;
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

// Grid barrier with a bounded wait.  Returns false (and sets status[0]) when
// the wait ran out or another CTA already gave up.
__device__ bool grid_barrier(const SeqArgs &a, bool skip)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (!skip) {
            const unsigned gen = ld_acquire(a.bar + 1);
            __threadfence();
            const unsigned arrived = atomicAdd(a.bar, 1u);
            if (arrived == gridDim.x - 1) {
                atomicExch(a.bar, 0u);
                __threadfence();
                atomicAdd(a.bar + 1, 1u);
            } else {
                unsigned it = 0;
                while (ld_acquire(a.bar + 1) == gen) {
                    if (ld_volatile_int(a.status) != 0 || ++it > a.spin_limit) {
                        atomicExch(a.status, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(256);
                }
            }
        } else {
            // test hook: never arrive; wait (bounded) for the others to give up
            unsigned it = 0;
            while (ld_volatile_int(a.status) == 0 && ++it <= a.spin_limit) __nanosleep(256);
            atomicExch(a.status, 1);
            ok = 0;
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ unsigned pack_half2(unsigned lo_elem, unsigned hi_elem)
{
    __half2 h = __halves2half2(__uint2half_rn(lo_elem), __uint2half_rn(hi_elem));
    return *reinterpret_cast<unsigned *>(&h);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&A)[4],
                                         const unsigned (&B)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(A[0]), "r"(A[1]), "r"(A[2]), "r"(A[3]), "r"(B[0]), "r"(B[1]),
          "f"(0.f), "f"(0.f), "f"(0.f), "f"(0.f));
}

struct SeqSmem {
    // limbs of one pass: [limb][row][component], component padded to 18 halves
    unsigned short xs[2][kRowsPerPass][kS + 2];
    unsigned short vs[2][kRowsPerPass][kS + 2];
    unsigned long long acc[kS * kS];
    unsigned long long red[kSeqThreads / 32];
};

// Project the pass tile held in shared memory: warp w takes k-step (w & 7)
// and limb pairs 2*(w>>3), 2*(w>>3)+1 (pair index = 2*x_limb + v_limb).
__device__ __forceinline__ void project_tile(SeqSmem &sm, unsigned long long (&pacc)[2][4])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int ks = w & (kKSteps - 1);
    const int k0 = ks * 16;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int lp = 2 * (w >> 3) + q;
        const int xl = lp >> 1, vl = lp & 1;
        const unsigned long long wgt = (xl ? 256ull : 1ull) * (vl ? 256ull : 1ull);
        unsigned A[4];
        A[0] = pack_half2(sm.xs[xl][k0 + 2 * t][g], sm.xs[xl][k0 + 2 * t + 1][g]);
        A[1] = pack_half2(sm.xs[xl][k0 + 2 * t][g + 8], sm.xs[xl][k0 + 2 * t + 1][g + 8]);
        A[2] = pack_half2(sm.xs[xl][k0 + 2 * t + 8][g], sm.xs[xl][k0 + 2 * t + 9][g]);
        A[3] = pack_half2(sm.xs[xl][k0 + 2 * t + 8][g + 8], sm.xs[xl][k0 + 2 * t + 9][g + 8]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int n = nt * 8 + g;
            unsigned B[2];
            B[0] = pack_half2(sm.vs[vl][k0 + 2 * t][n], sm.vs[vl][k0 + 2 * t + 1][n]);
            B[1] = pack_half2(sm.vs[vl][k0 + 2 * t + 8][n], sm.vs[vl][k0 + 2 * t + 9][n]);
            float d[4];
            mma16816(d, A, B);
#pragma unroll
            for (int e = 0; e < 4; ++e) pacc[nt][e] += wgt * (unsigned long long)__float2uint_rn(d[e]);
        }
    }
}

// V_out rows [r0, r1) = A * V_in, and (if `project`) the partial X^T V_out
// over those rows into sm.acc.
__device__ void spmm_and_project(const SeqArgs &a, SeqSmem &sm, const unsigned short *Vin,
                                 unsigned short *Vout, long long r0, long long r1,
                                 bool compute, bool project)
{
    const int rip = threadIdx.x / kTPR;     // row in pass
    const int c0 = (threadIdx.x % kTPR) * kCPT;
    unsigned long long pacc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    for (long long base = r0; base < r1; base += kRowsPerPass) {
        const long long row = base + rip;
        u32 out[kCPT] = {0, 0, 0, 0};
        if (row < r1) {
            if (compute) {
                unsigned long long acc[kCPT] = {0, 0, 0, 0};
                for (int d = 0; d < a.ndiag; ++d) {
                    const long long j = row + __ldg(a.doff + d);
                    if (j >= 0 && j < a.n) {
                        const u32 v = __ldg(a.dval + (long long)d * a.ld + row);
                        const uint2 q = __ldcg(reinterpret_cast<const uint2 *>(Vin + j * kS + c0));
                        acc[0] += (unsigned long long)v * (q.x & 0xffffu);
                        acc[1] += (unsigned long long)v * (q.x >> 16);
                        acc[2] += (unsigned long long)v * (q.y & 0xffffu);
                        acc[3] += (unsigned long long)v * (q.y >> 16);
                    }
                }
                const int nb = a.rownb ? (int)__ldg(a.rownb + row) : a.width;
                for (int e = 0; e < nb; ++e) {
                    const long long idx = (long long)e * a.ld + row;
                    const long long j = __ldg(a.col + idx);
                    const u32 v = __ldg(a.val + idx);
                    const uint2 q = __ldcg(reinterpret_cast<const uint2 *>(Vin + j * kS + c0));
                    acc[0] += (unsigned long long)v * (q.x & 0xffffu);
                    acc[1] += (unsigned long long)v * (q.x >> 16);
                    acc[2] += (unsigned long long)v * (q.y & 0xffffu);
                    acc[3] += (unsigned long long)v * (q.y >> 16);
                }
#pragma unroll
                for (int v = 0; v < kCPT; ++v) out[v] = red64(acc[v], a.M);
                uint2 st;
                st.x = out[0] | (out[1] << 16);
                st.y = out[2] | (out[3] << 16);
                *reinterpret_cast<uint2 *>(Vout + row * kS + c0) = st;
            } else {
                const uint2 q = __ldcg(reinterpret_cast<const uint2 *>(Vin + row * kS + c0));
                out[0] = q.x & 0xffffu;
                out[1] = q.x >> 16;
                out[2] = q.y & 0xffffu;
                out[3] = q.y >> 16;
            }
        }
        if (!project) continue;
        // stage this pass's limbs
        uint2 xq = make_uint2(0u, 0u);
        if (row < r1) xq = __ldg(reinterpret_cast<const uint2 *>(a.Xh + row * kS + c0));
        const u32 xv[kCPT] = {xq.x & 0xffffu, xq.x >> 16, xq.y & 0xffffu, xq.y >> 16};
#pragma unroll
        for (int v = 0; v < kCPT; ++v) {
            sm.xs[0][rip][c0 + v] = (unsigned short)(xv[v] & 255u);
            sm.xs[1][rip][c0 + v] = (unsigned short)(xv[v] >> 8);
            sm.vs[0][rip][c0 + v] = (unsigned short)(out[v] & 255u);
            sm.vs[1][rip][c0 + v] = (unsigned short)(out[v] >> 8);
        }
        __syncthreads();
        project_tile(sm, pacc);
        __syncthreads();
    }
    if (!project) return;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int b = nt * 8 + 2 * t;
        atomicAdd(&sm.acc[g * kS + b], pacc[nt][0]);
        atomicAdd(&sm.acc[g * kS + b + 1], pacc[nt][1]);
        atomicAdd(&sm.acc[(g + 8) * kS + b], pacc[nt][2]);
        atomicAdd(&sm.acc[(g + 8) * kS + b + 1], pacc[nt][3]);
    }
}

// Write this CTA's partial projection (reduced) and clear the accumulator.
__device__ void publish_partial(const SeqArgs &a, SeqSmem &sm, int buf)
{
    __syncthreads();
    u32 *dst = a.partial + ((size_t)buf * gridDim.x + blockIdx.x) * (kS * kS);
    for (int t = threadIdx.x; t < kS * kS; t += blockDim.x) {
        dst[t] = red64(sm.acc[t], a.M);
        sm.acc[t] = 0;
    }
    __syncthreads();
}

// S_step[o] = sum over CTAs of their partials (mod p), outputs split over CTAs.
__device__ void reduce_step(const SeqArgs &a, SeqSmem &sm, int buf, long long step)
{
    const int nb = gridDim.x;
    const u32 *src = a.partial + (size_t)buf * nb * (kS * kS);
    for (int o = blockIdx.x; o < kS * kS; o += nb) {
        unsigned long long s = 0;
        for (int c = threadIdx.x; c < nb; c += blockDim.x) s += __ldcg(src + (size_t)c * (kS * kS) + o);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += sm.red[i];
            const int ai = o / kS, bi = o % kS;
            if (ai < a.s && bi < a.s) a.S[(step * a.s + ai) * a.s + bi] = red64(tot, a.M);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSeqThreads, 1) k_sequence(const __grid_constant__ SeqArgs a)
{
    __shared__ SeqSmem sm;
    for (int t = threadIdx.x; t < kS * kS; t += blockDim.x) sm.acc[t] = 0;
    const long long nb = gridDim.x;
    const long long r0 = a.n * blockIdx.x / nb, r1 = a.n * (blockIdx.x + 1) / nb;
    if (a.nsteps <= 0 && !a.Vnext) return;
    bool skip = a.test_skip && blockIdx.x == 0;
    // S_0 = X^T Y
    if (a.nsteps > 0) {
        spmm_and_project(a, sm, a.V0, a.V0, r0, r1, false, true);
        publish_partial(a, sm, 0);
        if (!grid_barrier(a, skip)) return;
        reduce_step(a, sm, 0, 0);
    }
    long long done = 0;  // SpMMs done: V_done is current
    for (long long i = 0; i < a.nsteps; ++i) {
        const bool need = (i + 1 < a.nsteps) || a.Vnext;
        if (!need) break;
        const unsigned short *Vin = (i & 1) ? a.V1 : a.V0;
        unsigned short *Vout = (i & 1) ? a.V0 : a.V1;
        const bool proj = i + 1 < a.nsteps;
        spmm_and_project(a, sm, Vin, Vout, r0, r1, true, proj);
        if (proj) publish_partial(a, sm, (int)((i + 1) & 1));
        if (!grid_barrier(a, false)) return;
        done = i + 1;
        if (proj) reduce_step(a, sm, (int)((i + 1) & 1), i + 1);
    }
    if (a.Vnext) {
        const unsigned short *Vf = (done & 1) ? a.V1 : a.V0;
        for (long long t = r0 * a.s + threadIdx.x; t < r1 * a.s; t += blockDim.x) {
            const long long row = t / a.s;
            const int c = (int)(t - row * a.s);
            a.Vnext[t] = __ldcg(Vf + row * kS + c);
        }
    }
}

// X, Y (n x s, u32) -> Xh, V0 (n x 16, u16, zero padded, reduced mod p).
__global__ void k_seq_prepare(long long n, int s, const u32 *__restrict__ X,
                              const u32 *__restrict__ Y, unsigned short *Xh,
                              unsigned short *V0, const Mod M)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * kS) return;
    const long long row = t / kS;
    const int c = (int)(t - row * kS);
    u32 xv = 0, yv = 0;
    if (c < s) {
        xv = red64(X[row * s + c], M);
        yv = red64(Y[row * s + c], M);
    }
    Xh[t] = (unsigned short)xv;
    V0[t] = (unsigned short)yv;
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
    unsigned short *Xh = nullptr, *V0 = nullptr, *V1 = nullptr;
    u32 *partial = nullptr;
    unsigned *bar = nullptr;
    int nblocks = 0;
    // per-launch path buffers
    void *gwork = nullptr;
    size_t gwork_bytes = 0;
    // graph cache
    cudaGraphExec_t exec = nullptr;
    SeqArgs key;
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
    if (width > 64) return false;  // one thread per row: keep rows short
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
    size_t vb = al((size_t)n * kS * 2 + 16);
    size_t pb = al((size_t)2 * nblocks * kS * kS * 4);
    size_t need = 3 * vb + pb + 256;
    if (need > q.work_bytes) {
        if (q.work) cudaFree(q.work);
        q.work = nullptr;
        q.work_bytes = 0;
        if (cudaMalloc(&q.work, need) != cudaSuccess) return FFSPMV_ERR_OOM;
        q.work_bytes = need;
    }
    char *b = (char *)q.work;
    q.Xh = (unsigned short *)b;
    q.V0 = (unsigned short *)(b + vb);
    q.V1 = (unsigned short *)(b + 2 * vb);
    q.partial = (u32 *)(b + 3 * vb);
    q.bar = (unsigned *)(b + 3 * vb + pb);
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
                                             int32_t s, int64_t nsteps, uint32_t *d_S,
                                             uint32_t *d_V_next, ffspmv_stream_t stream)
{
    if (!h || s < 1 || s > 32 || nsteps < 0) return FFSPMV_ERR_ARG;
    if (h->A.nrows != h->A.ncols) return FFSPMV_ERR_ARG;
    const long long n = h->A.nrows;
    if (n > 0 && (!d_X || !d_Y)) return FFSPMV_ERR_ARG;
    if (nsteps > 0 && !d_S) return FFSPMV_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!h->seq_state) h->seq_state = new (std::nothrow) SeqState();
    SeqState *q = (SeqState *)h->seq_state;
    if (!q) return FFSPMV_ERR_OOM;

    bool persistent = h->opt.sequence_mode == 0 && h->m <= 65536u && s <= kS && n > 0;
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sequence, kSeqThreads, 0);
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
    a.Xh = q->Xh;
    a.V0 = q->V0;
    a.V1 = q->V1;
    a.partial = q->partial;
    a.S = d_S;
    a.Vnext = d_V_next;
    a.bar = q->bar;
    a.status = h->d_status;
    a.spin_limit = h->opt.barrier_spin_limit ? h->opt.barrier_spin_limit : kDefaultSpins;
    a.test_skip = (h->opt.test_hooks & 1) ? 1 : 0;
    a.M = make_mod(h->m, 1, 0);

    // the graph: prepare X/Y, clear barrier + status, run the persistent kernel
    if (!q->exec || !same_key(a, q->key)) {
        if (q->exec) cudaGraphExecDestroy(q->exec);
        q->exec = nullptr;
        cudaStream_t cs;
        FF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            k_seq_prepare<<<(unsigned)((n * kS + 255) / 256), 256, 0, cs>>>(n, s, d_X, d_Y, q->Xh, q->V0, a.M);
            cudaMemsetAsync(q->bar, 0, 2 * sizeof(unsigned), cs);
            cudaMemsetAsync(h->d_status, 0, sizeof(int), cs);
            cudaLaunchConfig_t cfg;
            memset(&cfg, 0, sizeof(cfg));
            cfg.gridDim = dim3((unsigned)nblocks);
            cfg.blockDim = dim3(kSeqThreads);
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
