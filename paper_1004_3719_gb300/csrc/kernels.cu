// SpMV / SpMM kernels over Z/mZ for every plan segment format.
//
// One launch runs every segment of a plan phase: CTA b belongs to the segment
// whose CTA range holds b, and runs that segment's device routine.  Each
// routine forms the exact sums of Sec. 2 (y <- alpha*A*x + beta*y, block form
// with NV vectors per launch) in integer accumulators and reduces once per
// output (Sec. 2.2, delayed reduction); +-1 entries flagged in the column
// word add or subtract x instead of multiplying (Sec. 2.4.2).
#include <type_traits>

#include "ff_internal.cuh"

namespace ff {

Mod make_mod(u32 m, u32 alpha, u32 beta)
{
    Mod M;
    unsigned __int128 two64 = (unsigned __int128)1 << 64;
    M.m = m;
    M.mu = (u64)(two64 / m);
    M.c64 = (u32)(two64 % m);
    M.alpha = alpha % m;
    M.beta = beta % m;
    return M;
}

// Matrix words are read once per product: load them without allocating in
// L1, which is left to the gathered rows of x.
__device__ __forceinline__ u32 ld_stream(const u32 *p)
{
    u32 v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ u32 ld_stream(const unsigned short *p)
{
    unsigned short v;
    asm("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ u32 load_val(const void *p, long long i, int vbytes)
{
    if (vbytes == 2) return ld_stream(reinterpret_cast<const unsigned short *>(p) + i);
    return ld_stream(reinterpret_cast<const u32 *>(p) + i);
}

template <int NV>
__device__ __forceinline__ void load_x(const u32 *__restrict__ x, long long j,
                                       long long ldx, u32 (&xv)[NV], bool vec4)
{
    const u32 *p = x + j * ldx;
    if constexpr (NV >= 4) {
        if (vec4) {
#pragma unroll
            for (int i = 0; i < NV / 4; ++i) {
                uint4 t = __ldg(reinterpret_cast<const uint4 *>(p) + i);
                xv[4 * i + 0] = t.x;
                xv[4 * i + 1] = t.y;
                xv[4 * i + 2] = t.z;
                xv[4 * i + 3] = t.w;
            }
            return;
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) xv[v] = __ldg(p + v);
}

template <int NV, class Acc>
__device__ __forceinline__ void apply_entry(Acc (&acc)[NV], u32 cls, u32 val,
                                            const u32 (&xv)[NV], u32 m)
{
    if (cls == 0u) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v].mad(val, xv[v]);
    } else if (cls == kPlus) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v].add(xv[v]);
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v].add(m - xv[v]);
    }
}

template <int NV>
__device__ __forceinline__ void write_row(u32 *__restrict__ y, long long row,
                                          long long ldy, const u64 (&part)[NV],
                                          bool accum, const Mod &M)
{
    u32 *yp = y + row * ldy;
#pragma unroll
    for (int v = 0; v < NV; ++v) yp[v] = combine(red64(part[v], M), yp + v, accum, M);
}

// ---------------------------------------------------------------------------
// Entries k, k + stride, ... below `end` of one CSR row, U at a time: the U
// column words (and values) are loaded first, then the U rows of x, so that
// U independent gathers are in flight per thread.
#ifndef FF_UNROLL1
#define FF_UNROLL1 2
#endif
#ifndef FF_MINB1
#define FF_MINB1 8
#endif

template <int NV>
struct Unroll {
    static constexpr int U = NV == 1 ? FF_UNROLL1 : NV == 2 ? 4 : NV == 4 ? 2 : 1;
};

constexpr u32 kSkip = 3u;  // class of a slot past the end of the row

template <class Acc, int NV>
__device__ __forceinline__ void csr_entries(Acc (&acc)[NV], const SegDesc &S, u32 k, u32 end,
                                            u32 stride, u32 start, u32 vbase,
                                            const u32 *__restrict__ x, long long ldx,
                                            bool vec4, u32 m)
{
    constexpr int U = Unroll<NV>::U;
    for (; k < end; k += U * stride) {
        u32 c[U], a[U], cls[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const u32 kk = k + u * stride;
            c[u] = 0;
            a[u] = 0;
            cls[u] = kSkip;
            if (kk < end) {
                const u32 w = ld_stream(S.col + kk);
                cls[u] = S.pm ? (w >> kClassShift) : 0u;
                c[u] = S.pm ? (w & kColMask) : w;
                if (cls[u] == 0u) a[u] = load_val(S.val, (long long)vbase + (kk - start), S.vbytes);
            }
        }
        u32 xv[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (cls[u] != kSkip) load_x<NV>(x, c[u], ldx, xv[u], vec4);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (cls[u] != kSkip) apply_entry<NV>(acc, cls[u], a[u], xv[u], m);
    }
}

// ---------------------------------------------------------------------------
// CSR, `group` lanes per row (a power of two up to 32).
template <class Acc, int NV>
__device__ void seg_csr(const SegDesc &S, long long lb, const u32 *__restrict__ x,
                        long long ldx, u32 *__restrict__ y, long long ldy,
                        const Mod &M, bool vec4)
{
    const int G = S.group;
    const int gid = threadIdx.x / G;
    const int lane = threadIdx.x & (G - 1);
    const long long r = lb * (kThreads / G) + gid;
    const bool active = r < S.nrows;
    Acc acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v].zero();
    if (active) {
        const u32 start = __ldg(S.ptr + r), end = __ldg(S.ptr + r + 1);
        const u32 vbase = S.vptr ? __ldg(S.vptr + r) : start;
        csr_entries<Acc, NV>(acc, S, start + lane, end, (u32)G, start, vbase, x, ldx, vec4, M.m);
    }
    u64 part[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) part[v] = acc[v].partial(M);
    for (int off = G >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) part[v] += __shfl_xor_sync(0xffffffffu, part[v], off);
    }
    if (active && lane == 0) {
        const long long row = S.rows ? (long long)__ldg(S.rows + r) : S.row0 + r;
        write_row<NV>(y, row, ldy, part, S.accum, M);
    }
}

// Sum of `part` over the CTA, valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(u64 (&part)[NV])
{
    __shared__ u64 red[kThreads / 32][NV];
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) part[v] += __shfl_xor_sync(0xffffffffu, part[v], off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) red[w][v] = part[v];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            u64 t = 0;
            for (int i = 0; i < kThreads / 32; ++i) t += red[i][v];
            part[v] = t;
        }
    }
}

// ---------------------------------------------------------------------------
// CSR, one CTA per row.
template <class Acc, int NV>
__device__ void seg_csrblk(const SegDesc &S, long long lb, const u32 *__restrict__ x,
                           long long ldx, u32 *__restrict__ y, long long ldy,
                           const Mod &M, bool vec4)
{
    const long long r = lb;
    const u32 start = __ldg(S.ptr + r), end = __ldg(S.ptr + r + 1);
    const u32 vbase = S.vptr ? __ldg(S.vptr + r) : start;
    Acc acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v].zero();
    csr_entries<Acc, NV>(acc, S, start + threadIdx.x, end, (u32)kThreads, start, vbase, x, ldx,
                         vec4, M.m);
    u64 part[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) part[v] = acc[v].partial(M);
    block_sum<NV>(part);
    if (threadIdx.x == 0) {
        const long long row = S.rows ? (long long)__ldg(S.rows + r) : S.row0 + r;
        write_row<NV>(y, row, ldy, part, S.accum, M);
    }
}

// ---------------------------------------------------------------------------
// Long rows cut into chunks of at most kSplitChunk entries, one CTA per
// chunk; each CTA adds its reduced partial sum into carry[row] with an exact
// 64-bit atomic and a second launch finishes the rows.  One vector per launch.
template <class Acc>
__device__ void seg_csrsplit(const SegDesc &S, long long lb, const u32 *__restrict__ x,
                             long long ldx, const Mod &M, u64 *__restrict__ carry)
{
    const u32 r = __ldg(S.chunk_row + lb);
    const u32 b = __ldg(S.chunk_beg + lb), e = __ldg(S.chunk_beg + lb + 1);
    const u32 start = __ldg(S.ptr + r);
    const u32 vbase = S.vptr ? __ldg(S.vptr + r) : start;
    Acc acc[1];
    acc[0].zero();
    csr_entries<Acc, 1>(acc, S, b + threadIdx.x, e, (u32)kThreads, start, vbase, x, ldx, false,
                        M.m);
    u64 part[1] = {acc[0].partial(M)};
    block_sum<1>(part);
    if (threadIdx.x == 0) {
        const long long row = S.rows ? (long long)__ldg(S.rows + r) : S.row0 + r;
        atomicAdd(carry + row, (u64)red64(part[0], M));
    }
}

// ---------------------------------------------------------------------------
// One thread per row: DIA diagonals, then ELL_R columns (column-major, Sec.
// 2.1; coalesced on the GPU, Sec. 2.4.3).
template <class Acc, int NV>
__device__ void seg_ellr(const SegDesc &S, long long lb, const u32 *__restrict__ x,
                         long long ldx, u32 *__restrict__ y, long long ldy,
                         const Mod &M, bool vec4)
{
    constexpr int U = Unroll<NV>::U;
    const long long r = lb * kThreads + threadIdx.x;
    if (r >= S.nrows) return;
    const long long row = S.rows ? (long long)__ldg(S.rows + r) : S.row0 + r;
    Acc acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v].zero();
    for (int d = 0; d < S.ndiag; ++d) {
        const long long j = row + __ldg(S.doff + d);
        if (j >= 0 && j < S.ncols) {
            u32 a = load_val(S.dval, (long long)d * S.ld + r, S.dvbytes);
            u32 xv[NV];
            load_x<NV>(x, j, ldx, xv, vec4);
            apply_entry<NV>(acc, 0u, a, xv, M.m);
        }
    }
    const int n = S.rownb ? (int)__ldg(S.rownb + r) : S.width;
    for (int j = 0; j < n; j += U) {
        u32 c[U], a[U], cls[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            c[u] = 0;
            a[u] = 0;
            cls[u] = kSkip;
            if (j + u < n) {
                const long long idx = (long long)(j + u) * S.ld + r;
                const u32 w = ld_stream(S.col + idx);
                cls[u] = S.pm ? (w >> kClassShift) : 0u;
                c[u] = S.pm ? (w & kColMask) : w;
                if (cls[u] == 0u) a[u] = load_val(S.val, idx, S.vbytes);
            }
        }
        u32 xv[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (cls[u] != kSkip) load_x<NV>(x, c[u], ldx, xv[u], vec4);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (cls[u] != kSkip) apply_entry<NV>(acc, cls[u], a[u], xv[u], M.m);
    }
    u64 part[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) part[v] = acc[v].partial(M);
    write_row<NV>(y, row, ldy, part, S.accum, M);
}

// ---------------------------------------------------------------------------
// COO: each warp owns 32*kCooRuns consecutive entries (sorted by row) and
// forms per-row sums by a segmented warp scan of reduced terms.  A row that
// also has entries in another warp's chunk adds its partial sum into
// `carry[row]` with an exact 64-bit atomic; a second launch finishes those
// rows.  One vector per launch.
__device__ __forceinline__ u64 coo_term(u32 cls, u32 a, u32 xv, const Mod &M)
{
    if (cls == 0u) return red64((u64)a * xv, M);
    if (cls == kPlus) return xv;
    return (u64)(M.m - xv);
}

__device__ void seg_coo(const SegDesc &S, long long lb, const u32 *__restrict__ x,
                        long long ldx, u32 *__restrict__ y, long long ldy,
                        const Mod &M, u64 *__restrict__ carry)
{
    const int lane = threadIdx.x & 31;
    const long long w = lb * (kThreads / 32) + (threadIdx.x >> 5);
    const long long cb = w * (32LL * kCooRuns);
    if (cb >= S.nnz) return;
    const long long ce = min(S.nnz, cb + 32LL * kCooRuns);
    const u32 first_row = __ldg(S.rowid + cb);
    const u32 last_row = __ldg(S.rowid + ce - 1);
    const bool started_before = cb > 0 && __ldg(S.rowid + cb - 1) == first_row;
    const bool continues_after = ce < S.nnz && __ldg(S.rowid + ce) == last_row;
    const u32 kNone = 0xffffffffu;

    u32 carry_row = kNone;
    u64 carry_val = 0;

    auto flush = [&](u32 row, u64 s) {
        const bool shared_row = (row == first_row && started_before) ||
                                (row == last_row && continues_after);
        if (shared_row) {
            atomicAdd(carry + row, (u64)red64(s, M));
        } else {
            u32 *yp = y + (long long)row * ldy;
            *yp = combine(red64(s, M), yp, S.accum, M);
        }
    };

    for (long long base = cb; base < ce; base += 32) {
        const long long k = base + lane;
        const bool valid = k < ce;
        u32 row = kNone, cls = 0, a = 0, xv = 0;
        if (valid) {
            row = __ldg(S.rowid + k);
            u32 c = __ldg(S.col + k);
            if (S.pm) {
                cls = c >> kClassShift;
                c &= kColMask;
            }
            if (cls == 0u) a = load_val(S.val, k, S.vbytes);
            xv = __ldg(x + (long long)c * ldx);
        }
        // the run carried from the previous 32 entries ends here unless
        // this run starts with the same row
        const u32 r0 = __shfl_sync(0xffffffffu, row, 0);
        if (carry_row != kNone && r0 != carry_row) {
            if (lane == 0) flush(carry_row, carry_val);
            carry_row = kNone;
            carry_val = 0;
        }
        u32 prev = __shfl_up_sync(0xffffffffu, row, 1);
        if (lane == 0) prev = carry_row;
        u32 next = __shfl_down_sync(0xffffffffu, row, 1);
        const bool tail = valid && (lane == 31 || row != next);
        u64 s = valid ? coo_term(cls, a, xv, M) : 0;
        if (lane == 0 && valid && row == carry_row) s += carry_val;
        bool head = !valid || row != prev;
        // segmented inclusive scan (heads stop the sum)
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            u64 o = __shfl_up_sync(0xffffffffu, s, off);
            int ho = __shfl_up_sync(0xffffffffu, (int)head, off);
            if (lane >= off) {
                if (!head) s += o;
                head = head || ho;
            }
        }
        const bool lane31_valid = __shfl_sync(0xffffffffu, (int)valid, 31);
        if (tail && lane != 31) flush(row, s);
        if (lane31_valid) {
            carry_row = __shfl_sync(0xffffffffu, row, 31);
            u64 cv = __shfl_sync(0xffffffffu, s, 31);
            carry_val = red64(cv, M);
        } else {
            carry_row = kNone;
            carry_val = 0;
        }
    }
    if (lane == 0 && carry_row != kNone) flush(carry_row, carry_val);
}

// ---------------------------------------------------------------------------
// Rows without entries: y <- beta*y (first writer only).
template <int NV>
__device__ void seg_empty(const SegDesc &S, long long lb, u32 *__restrict__ y,
                          long long ldy, const Mod &M)
{
    const long long r = lb * kThreads + threadIdx.x;
    if (r >= S.nrows || S.accum) return;
    const long long row = S.rows ? (long long)__ldg(S.rows + r) : S.row0 + r;
    u32 *yp = y + row * ldy;
#pragma unroll
    for (int v = 0; v < NV; ++v)
        yp[v] = (M.beta == 0u) ? 0u : red64((u64)M.beta * yp[v], M);
}

template <class Acc, int NV>
__global__ void __launch_bounds__(kThreads, NV == 1 ? FF_MINB1 : 2)
k_plan(const __grid_constant__ PlanParams P, const u32 *__restrict__ x,
       long long ldx, u32 *__restrict__ y, long long ldy, const Mod M,
       u64 *__restrict__ carry, int vec4)
{
    // The descriptor of this CTA's segment is copied once into shared memory
    // and from there into registers: indexing the parameter table with a
    // run-time segment number inside the loops would turn every field access
    // into a constant-bank load.
    __shared__ SegDesc sdesc;
    __shared__ int sidx;
    if (threadIdx.x == 0) {
        int lo = 0, hi = P.nseg - 1;
        const long long b = blockIdx.x;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.seg[mid].block0 <= b) lo = mid;
            else hi = mid - 1;
        }
        sidx = lo;
    }
    __syncthreads();
    constexpr int W = (int)(sizeof(SegDesc) / sizeof(u32));
    if (threadIdx.x < W)
        reinterpret_cast<u32 *>(&sdesc)[threadIdx.x] =
            reinterpret_cast<const u32 *>(&P.seg[sidx])[threadIdx.x];
    __syncthreads();
    const SegDesc &S = sdesc;
    const long long lb = (long long)blockIdx.x - S.block0;
    switch (S.kind) {
    case SEG_CSR: seg_csr<Acc, NV>(S, lb, x, ldx, y, ldy, M, vec4 != 0); break;
    case SEG_CSRBLK: seg_csrblk<Acc, NV>(S, lb, x, ldx, y, ldy, M, vec4 != 0); break;
    case SEG_ELLR: seg_ellr<Acc, NV>(S, lb, x, ldx, y, ldy, M, vec4 != 0); break;
    case SEG_COO:
        if constexpr (NV == 1) seg_coo(S, lb, x, ldx, y, ldy, M, carry);
        break;
    case SEG_CSRSPLIT:
        if constexpr (NV == 1) seg_csrsplit<Acc>(S, lb, x, ldx, M, carry);
        break;
    case SEG_EMPTY: seg_empty<NV>(S, lb, y, ldy, M); break;
    default: break;
    }
}

// Rows whose COO entries spanned several warp chunks.
__global__ void k_coo_finish(const u32 *__restrict__ rows, long long n,
                             u64 *__restrict__ carry, u32 *__restrict__ y,
                             long long ldy, const Mod M, int accum)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u32 row = rows[i];
    const u64 c = carry[row];
    carry[row] = 0;
    u32 *yp = y + (long long)row * ldy;
    *yp = combine(red64(c, M), yp, accum != 0, M);
}

template <class Acc, int NV>
static void launch_phase(const PlanParams &pp, const u32 *x, long long ldx,
                         u32 *y, long long ldy, const Mod &M, u64 *carry,
                         bool vec4, cudaStream_t st)
{
    k_plan<Acc, NV><<<(unsigned)pp.total_blocks, kThreads, 0, st>>>(
        pp, x, ldx, y, ldy, M, carry, vec4 ? 1 : 0);
}

template <class Acc>
static void launch_nv(int nv, const PlanParams &pp, const u32 *x, long long ldx,
                      u32 *y, long long ldy, const Mod &M, u64 *carry,
                      bool vec4, cudaStream_t st)
{
    switch (nv) {
    case 16: launch_phase<Acc, 16>(pp, x, ldx, y, ldy, M, carry, vec4, st); break;
    case 8: launch_phase<Acc, 8>(pp, x, ldx, y, ldy, M, carry, vec4, st); break;
    case 4: launch_phase<Acc, 4>(pp, x, ldx, y, ldy, M, carry, vec4, st); break;
    case 2: launch_phase<Acc, 2>(pp, x, ldx, y, ldy, M, carry, vec4, st); break;
    default: launch_phase<Acc, 1>(pp, x, ldx, y, ldy, M, carry, vec4, st); break;
    }
}

static PlanParams params_of(const Phase &ph, int acc_wide)
{
    PlanParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.nseg = (int)ph.segs.size();
    pp.acc_wide = acc_wide;
    long long total = 0;
    for (int i = 0; i < pp.nseg; ++i) {
        pp.seg[i] = ph.segs[i];
        total = pp.seg[i].block0 + pp.seg[i].nblocks;
    }
    pp.total_blocks = total;
    return pp;
}

// ---------------------------------------------------------------------------
// x-panel layout (PanelPart, ff_internal.cuh; the host half is panel.cu).
// u16 / u32 copy of NV x columns, interleaved by vector (xs[i NV + k] =
// x[i ldx + k]), for plans whose CTAs are not all resident at once (their
// panel kernel cannot stage x itself).
template <typename XT, int NV>
__global__ void __launch_bounds__(256) k_x_stage(const u32 *__restrict__ x, long long ldx, long long n,
                                                 XT *__restrict__ xs)
{
    const long long nth = (long long)gridDim.x * blockDim.x;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long done = 0;
    if constexpr (NV > 1) {
        for (long long i = t; i < n; i += nth)
#pragma unroll
            for (int k = 0; k < NV; ++k) xs[i * NV + k] = (XT)__ldg(x + i * ldx + k);
        return;
    }
    if (ldx == 1 && ((uintptr_t)x & 15u) == 0) {
        // contiguous x: 16-byte loads, four elements each
        const long long n4 = n / 4;
        for (long long i = t; i < n4; i += nth) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(x) + i);
            if constexpr (sizeof(XT) == 1) {
                reinterpret_cast<u32 *>(xs)[i] = (v.x & 0xffu) | (v.y & 0xffu) << 8 | (v.z & 0xffu) << 16 | v.w << 24;
            } else if constexpr (sizeof(XT) == 2) {
                uint2 o;
                o.x = (v.x & 0xffffu) | (v.y << 16);
                o.y = (v.z & 0xffffu) | (v.w << 16);
                reinterpret_cast<uint2 *>(xs)[i] = o;
            } else {
                reinterpret_cast<uint4 *>(xs)[i] = v;
            }
        }
        done = n4 * 4;
    }
    for (long long i = done + t; i < n; i += nth) xs[i] = (XT)x[i * ldx];
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The shared::cluster address of `local` in CTA `rank` of the cluster.
template <typename T>
__device__ __forceinline__ u32 map_cluster(const T *local, u32 rank)
{
    u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((u32)__cvta_generic_to_shared(local)), "r"(rank));
    return r;
}

// *addr += v in another CTA's shared memory (posted; ordered by the next cluster barrier).
__device__ __forceinline__ void red_cluster_add(u32 addr, u32 v)
{
    asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void red_cluster_add(u32 addr, u64 v)
{
    asm volatile("red.shared::cluster.add.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

// A value in [0, 2m) congruent to t mod m, for t < 2^32 and mu = floor(2^32 / m):
// the quotient estimate floor(t * mu / 2^32) is floor(t/m) or one less
// (Barrett, 1986); the last conditional subtraction is left to the row sum's
// final reduction.
__device__ __forceinline__ u32 red32_lazy(u32 t, u32 m, u32 mu) { return t - __umulhi(t, mu) * m; }

// v x 2^-32 mod m, in [0, 2m), for odd m < 2^31, v < m and x < 2^32
// (Montgomery, 1985).  With u = (v x mod 2^32)(-1/m) mod 2^32, v x + u m is
// a multiple of 2^32: its low words add up to 0 (v x = 0 mod 2^32) or to
// exactly 2^32, and (v x + u m) / 2^32 < (m 2^32 + 2^32 m) / 2^32 = 2m.
// Values stored as v 2^32 mod m make this v x mod m.
__device__ __forceinline__ u32 mont_red(u32 v, u32 x, u32 m, u32 mneg)
{
    const u32 lo = v * x, hi = __umulhi(v, x);
    const u32 u = lo * mneg;
    return hi + __umulhi(u, m) + (lo != 0u ? 1u : 0u);
}

// -1/m mod 2^32 for odd m: y <- y (2 - m y) doubles the number of correct
// low bits (Newton's iteration for the inverse), starting from y = m, which
// is right to 3 bits (m m = 1 mod 8 for odd m).
__device__ __forceinline__ u32 neg_inv32(u32 m)
{
    u32 y = m;
#pragma unroll
    for (int i = 0; i < 4; ++i) y *= 2u - m * y;
    return 0u - y;
}

// Row sums in shared memory.  A u32 sum takes one reduction.  A 64-bit word
// holds two u32 sums, added as two 32-bit reductions (a 64-bit shared-memory
// atomic add costs far more): for m > 2^16 the sums of the low 16 bits (low
// word) and of the rest (high word) of every value added, the row's sum being
// low + 2^16 high; for two 16-bit-residue vectors, one vector's sum per word.
template <bool SPLIT16>
__device__ __forceinline__ void row_add(u64 *p, u64 c)
{
    u32 *w = reinterpret_cast<u32 *>(p);
    atomicAdd(w, SPLIT16 ? (u32)c & 0xffffu : (u32)c);
    atomicAdd(w + 1, (u32)(c >> (SPLIT16 ? 16 : 32)));
}
template <bool SPLIT16>
__device__ __forceinline__ void row_add(u32 *p, u32 c) { atomicAdd(p, c); }
__device__ __forceinline__ u64 row_total(u64 w) { return (w & 0xffffffffull) + ((w >> 32) << 16); }
__device__ __forceinline__ u64 row_total(u32 w) { return w; }

__device__ __forceinline__ void mbar_init(u32 bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Raise the bytes the current phase of `bar` waits for, without arriving.
__device__ __forceinline__ void mbar_add_tx(u32 bar, u32 bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(u32 bar, u32 bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

// Bulk copy global -> this CTA's shared memory, completing on mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(u32 dst, const void *src, u32 bytes, u32 bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Wait for the phase of `bar` with parity `parity`; false after POLLS polls.
template <unsigned POLLS = kPanelSpin>
__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity)
{
    for (unsigned i = 0; i < POLLS; ++i) {
        u32 done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(u32 bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ u32 ld_acquire_gpu(const u32 *p)
{
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ u32 atom_add_release_gpu(u32 *p, u32 v)
{
    u32 old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_release_gpu(u32 *p, u32 v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Orders this thread's generic-proxy accesses of global memory with later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// The x words of one column: NV interleaved elements of type XT.
template <bool SMALL, int NV>
struct PanelX {
    typedef typename std::conditional<
        (SMALL ? 2 : 4) * NV == 2, unsigned short,
        typename std::conditional<(SMALL ? 2 : 4) * NV == 4, u32,
                                  typename std::conditional<(SMALL ? 2 : 4) * NV == 8, uint2, uint4>::type>::type>::type W;
    // element k of the column
    static __device__ __forceinline__ u32 get(const W &w, int k)
    {
        if constexpr (SMALL) {
            if constexpr (NV == 1) return (u32)w;
            else if constexpr (NV == 2) return k ? w >> 16 : w & 0xffffu;
            else return k == 0 ? w.x & 0xffffu : k == 1 ? w.x >> 16 : k == 2 ? w.y & 0xffffu : w.y >> 16;
        } else {
            if constexpr (NV == 1) return w;
            else return k ? w.y : w.x;
        }
    }
};

// y = alpha A x + beta y for NV vectors at once (x: columns vcol..vcol+NV-1
// of the block, interleaved in the staged copy; row sums [row][NV]).  TINY
// (m <= 256, NV = 1): x and values as u8, terms v x < 2^16 added unreduced.
// MONT (odd 2^16 < m < 2^31): values in Montgomery form, terms v x mod m
// in [0, 2m) by one Montgomery reduction.  For m > 2^16 every row sum is
// a pair of u32 sums (row_add): each row's terms (below 2^32) number at most
// kPanelLong = 2^15, so the low-16-bit sum stays below 2^15 2^16 = 2^31 and
// the high sum below 2^15 2^32 / 2^16 = 2^31, however the terms are grouped
// into pack sums, CTAs and cluster partial sums.
template <bool SMALL, int NV, bool TINY = false, bool MONT = false>
__global__ void __launch_bounds__(kPanelThreads, 1)
k_panel(const PanelPart P, const u32 *__restrict__ x, long long ldx, u32 *__restrict__ y, long long ldy,
        const Mod M, int *status, int skip_stage, int conv)
{
    static_assert(!TINY || (SMALL && NV == 1), "u8 x: one vector, m <= 256");
    static_assert(!MONT || !SMALL, "Montgomery terms: m > 2^16");
    typedef typename std::conditional<TINY, unsigned char,
                                      typename std::conditional<SMALL, unsigned short, u32>::type>::type XT;
    typedef typename std::conditional<SMALL, u32, u64>::type AT;
    // a lane's term: one row sum's (AT), or, for 16-bit residues and NV > 1,
    // two vectors' u32 sums side by side in a u64 (each half stays below
    // 2^32, the bound of a single row sum, so no carry crosses between them)
    typedef typename std::conditional<SMALL && NV == 1, u32, u64>::type LT;
    constexpr int VG = SMALL && NV > 1 ? 2 : 1;  // vectors per term
    typedef PanelX<SMALL, NV> XC;
    typedef typename std::conditional<TINY, XT, typename XC::W>::type XW;
    static_assert(sizeof(XW) == sizeof(XT) * NV, "x word of a column");
    constexpr int VB = TINY ? 1 : SMALL ? 2 : 4;
    constexpr int kWarps = kPanelConsumers / 32;
    extern __shared__ __align__(128) unsigned char panel_smem[];
    const int PX = P.px, EB = P.eb;
    // [x slots][entry buffers][full mbarriers][empty mbarriers][stage descriptors][row sums]
    unsigned char *ebuf = panel_smem + kPanelStages * PX;
    unsigned char *bars = ebuf + kPanelStages * EB;
    uint4 *desc = reinterpret_cast<uint4 *>(bars + kPanelBarBytes);  // (entries, general, packs, x slot)
    u32 &s_gen = *reinterpret_cast<u32 *>(bars + kPanelBarBytes + 16 * kPanelStages);  // grid barrier generation
    AT *acc = reinterpret_cast<AT *>(bars + kPanelBarBytes + kPanelDescBytes);
    const int q = P.q;
    const int cta = blockIdx.x, g = cta / q, rank = cta % q;
    const u32 r0 = __ldg(P.grp_row0 + g), nr = __ldg(P.grp_row0 + g + 1) - r0;
    const u32 s0 = __ldg(P.stage_ptr + cta), ns = __ldg(P.stage_ptr + cta + 1) - s0;
    const u32 sbase = (u32)__cvta_generic_to_shared(panel_smem);
    const u32 full0 = (u32)__cvta_generic_to_shared(bars), empty0 = full0 + 8u * kPanelStages;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    // the grid barrier's generation before this CTA arrives (read early: the
    // load overlaps the conversion below)
    // conv > 0: this launch stages x itself (all its CTAs are resident): conv
    // staged columns (vectors vcol.. of the block, one launch per group of up
    // to four; later launches of the group read the staged copy), or one
    // group of NV interleaved vectors
    const int fused = conv > 0;
    u32 g0 = 0;
    if (fused && t == 0) g0 = ld_acquire_gpu(P.gbar + 1);
    if (fused) {
        // this CTA's share of x, converted into the staged copy that every
        // CTA's bulk copies read
        const long long G = gridDim.x;
        const long long share = ((P.ncols + G - 1) / G + 7) / 8 * 8;
        const long long lo = min(P.ncols, (long long)cta * share) * NV, hi = min(P.ncols, lo / NV + share) * NV;
        XT *xh = reinterpret_cast<XT *>(P.xh);
        long long done = lo;  // lo, hi: elements of the interleaved copy
        if (NV == 1 && conv > 1) {
            // conv vectors at once, one staged column each (P.xstride apart)
            const bool vec = conv == 4 && ldx % 4 == 0 && ((uintptr_t)x & 15u) == 0;
            for (long long i = lo + t; i < hi; i += kPanelThreads) {
                u32 c[4];
                if (vec) {
                    const uint4 w = __ldg(reinterpret_cast<const uint4 *>(x + i * ldx));
                    c[0] = w.x; c[1] = w.y; c[2] = w.z; c[3] = w.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) c[k] = k < conv ? __ldg(x + i * ldx + k) : 0u;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < conv) xh[k * P.xstride + i] = (XT)c[k];
            }
        } else if (ldx == NV && ((uintptr_t)x & 15u) == 0) {
            // the NV columns are contiguous: four 16-byte loads in flight per
            // thread before their stores
            const long long i1 = hi / 4;
            for (long long i0 = lo / 4 + t; i0 < i1; i0 += 4 * kPanelThreads) {
                uint4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + u * kPanelThreads < i1) v[u] = __ldg(reinterpret_cast<const uint4 *>(x) + i0 + u * kPanelThreads);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const long long i = i0 + u * kPanelThreads;
                    if (i >= i1) break;
                    if constexpr (TINY) {
                        reinterpret_cast<u32 *>(xh)[i] =
                            (v[u].x & 0xffu) | (v[u].y & 0xffu) << 8 | (v[u].z & 0xffu) << 16 | v[u].w << 24;
                    } else if constexpr (SMALL) {
                        uint2 o;
                        o.x = (v[u].x & 0xffffu) | (v[u].y << 16);
                        o.y = (v[u].z & 0xffffu) | (v[u].w << 16);
                        reinterpret_cast<uint2 *>(xh)[i] = o;
                    } else {
                        reinterpret_cast<uint4 *>(xh)[i] = v[u];
                    }
                }
            }
            done = max(lo, hi / 4 * 4);
            for (long long i = done + t; i < hi; i += kPanelThreads) xh[i] = (XT)__ldg(x + i);
        } else if (NV > 1 && ldx % NV == 0 && ((uintptr_t)x & (4u * NV - 1u)) == 0) {
            // one 4*NV-byte load per column
            typedef typename std::conditional<NV == 4, uint4, uint2>::type VW;
            for (long long i = lo / NV + t; i < hi / NV; i += kPanelThreads) {
                const VW w = __ldg(reinterpret_cast<const VW *>(x + i * ldx));
                const u32 *c = reinterpret_cast<const u32 *>(&w);
#pragma unroll
                for (int k = 0; k < NV; ++k) xh[i * NV + k] = (XT)c[k];
            }
        } else {
            for (long long i = lo / NV + t; i < hi / NV; i += kPanelThreads)
#pragma unroll
                for (int k = 0; k < NV; ++k) xh[i * NV + k] = (XT)__ldg(x + i * ldx + k);
        }
        fence_proxy_async_global();
    }
    for (u32 r = t; r < nr * NV; r += kPanelThreads) acc[r] = 0;
    __syncthreads();
    if (t == 0) {
        for (int b = 0; b < kPanelStages; ++b) {
            mbar_init(full0 + 8u * b, 1);
            mbar_init(empty0 + 8u * b, kWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n\tfence.proxy.async.shared::cta;" ::: "memory");
        if (fused) {
            // grid barrier: arrivals in gbar[0], generation in gbar[1]; the
            // last CTA to arrive resets the count and moves the generation on.
            // The release of the arrival covers the CTA's conversion stores
            // (ordered before it by the barrier above)
            s_gen = g0;
            if (atom_add_release_gpu(P.gbar, 1u) == gridDim.x - 1) {
                atomicExch(P.gbar, 0u);
                st_release_gpu(P.gbar + 1, g0 + 1);
            }
        }
    }
    __syncthreads();
    bool timed_out = false;
    if (warp >= kWarps) {
        // Copy warps.  Warp kWarps + b fills stage buffer b: stages b,
        // b + kPanelStages, ...  A thread's bulk copies complete one after
        // another, so each stage's copies come from two threads: lane 1 copies
        // the entries and values (they do not depend on x, so the first one
        // starts before the grid barrier) after adding their bytes to the
        // stage's full barrier; lane 0, once x is staged, publishes the stage
        // descriptor, arrives with the x panel's bytes and copies the panel.
        const u32 b = (u32)(warp - kWarps);
        const u32 bar = full0 + 8u * b, ebar = empty0 + 8u * b;
        const u32 d = sbase + kPanelStages * PX + b * EB;
        const unsigned char *xh = reinterpret_cast<const unsigned char *>(P.xh);
        const unsigned char *ev = reinterpret_cast<const unsigned char *>(P.ent);
        const unsigned char *vv = reinterpret_cast<const unsigned char *>(P.val);
        bool xready = !fused;
        for (u32 s = b; s < ns; s += kPanelStages) {
            const PanelStage a = P.stage[s0 + s];
            if (s >= kPanelStages) {
                // stage s - kPanelStages of this buffer must be done with
                u32 ok = 1;
                if (lane == 0) {
                    const u32 ep = (s / kPanelStages - 1) & 1u;
                    ok = (timed_out ? mbar_wait<1>(ebar, ep) : mbar_wait(ebar, ep)) ? 1u : 0u;
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) timed_out = true;
            }
            if ((int)s == skip_stage) continue;  // testing: this stage is never issued
            // values: u8 ones are copied in whole 16-byte blocks (the layout pads them)
            const u32 vbytes = TINY ? (a.ngen + 15u) & ~15u : a.ngen * (u32)VB;
            const u32 dbytes = a.nent * 4u + vbytes;
            if (lane == 1) mbar_add_tx(bar, dbytes);
            __syncwarp();  // the bytes are added before lane 0's arrive
            if (lane == 1) {
                bulk_g2s(d, ev + (size_t)a.k0 * 4, a.nent * 4u, bar);
                if (a.ngen) bulk_g2s(d + 4u * P.pe, vv + (size_t)a.v0 * VB, vbytes, bar);
            }
            if (lane == 0) {
                if (!xready) {
                    // every CTA's share of x is staged before the first panel copy
                    unsigned spin = 0;
                    while (ld_acquire_gpu(P.gbar + 1) == s_gen)
                        if (++spin >= kPanelGridSpin) {
                            timed_out = true;
                            break;
                        }
                    fence_proxy_async_global();
                    xready = true;
                }
                const bool newx = (a.xs & kPanelNewX) != 0;
                desc[b] = make_uint4(a.nent, a.ngen, a.npg | (a.npp << 16), a.xs & kPanelSlotMask);  // published by the arrive
                mbar_expect_tx(bar, newx ? (u32)PX : 0u);
                if (newx) bulk_g2s(sbase + (a.xs & kPanelSlotMask) * PX, xh + (size_t)a.xoff * sizeof(XW), (u32)PX, bar);
            }
            __syncwarp();
        }
    } else {
        const u32 mu32 = (u32)(M.mu >> 32);  // floor(2^32 / m)
        const u32 mneg = MONT ? neg_inv32(M.m) : 0u;
        const u32 rot = ((u32)P.pe / 8u + 31u) / 32u;  // blocks of a full stage
        for (u32 s = 0; s < ns; ++s) {
            const u32 b = s % kPanelStages;
            // after one wait has run out, the others poll once: a CTA whose
            // copies stopped coming ends in bounded time
            const u32 fb = full0 + 8u * b, fp = (s / kPanelStages) & 1u;
            bool released = false;
            if (timed_out ? mbar_wait<1>(fb, fp) : mbar_wait(fb, fp)) {
                const uint4 st = desc[b];
                const u32 nl = st.x >> 3, nlg = st.y >> 3, lpg = (st.z & 0xffffu) >> 3, lpp = (st.z >> 16) >> 3;
                const unsigned char *sb = ebuf + b * EB;
                const unsigned char *vb = sb + 4 * P.pe;
                const unsigned char *xs = panel_smem + st.w * PX;
                // the stage's 32-lane blocks start at a warp that moves on by a
                // full stage's blocks from one stage to the next, so that
                // consecutive stages run on different warps when there are
                // more warps than blocks
                const u32 w0 = ((u32)warp + kWarps - (s * rot) % kWarps) % kWarps;
                for (u32 lb = w0 * 32u; lb < nl; lb += 32u * kWarps) {
                    if constexpr (NV == 1) {
                    // one vector: terms and sums per lane value as u32 (m <= 2^16) or u64
                        const u32 tl = lb + lane, c = min(32u, nl - lb);
                        const bool valid = tl < nl, general = tl < nlg;
                        u32 e[8];
                        AT tm[8];
    #pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            e[u] = 0;
                            tm[u] = 0;
                        }
                        if (valid) {
                            // entries of lane j of this 32-lane block: 4j..4j+3 and 4c+4j..4c+4j+3
                            const uint4 e0 = *reinterpret_cast<const uint4 *>(sb + 4 * (8 * lb + 4 * lane));
                            const uint4 e1 = *reinterpret_cast<const uint4 *>(sb + 4 * (8 * lb + 4 * c + 4 * lane));
                            e[0] = e0.x; e[1] = e0.y; e[2] = e0.z; e[3] = e0.w;
                            e[4] = e1.x; e[5] = e1.y; e[6] = e1.z; e[7] = e1.w;
                            if (general) {
                                u32 v[8];
                                if (TINY) {
                                    const uint2 w = *reinterpret_cast<const uint2 *>(vb + 8 * tl);
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        v[u] = (w.x >> (8 * u)) & 0xffu;
                                        v[u + 4] = (w.y >> (8 * u)) & 0xffu;
                                    }
                                } else if (SMALL) {
                                    const uint4 w = *reinterpret_cast<const uint4 *>(vb + 2 * 8 * tl);
                                    v[0] = w.x & 0xffffu; v[1] = w.x >> 16; v[2] = w.y & 0xffffu; v[3] = w.y >> 16;
                                    v[4] = w.z & 0xffffu; v[5] = w.z >> 16; v[6] = w.w & 0xffffu; v[7] = w.w >> 16;
                                } else {
                                    const u32 cg = min(32u, nlg - lb);
                                    const uint4 w0 = *reinterpret_cast<const uint4 *>(vb + 4 * (8 * lb + 4 * lane));
                                    const uint4 w1 = *reinterpret_cast<const uint4 *>(vb + 4 * (8 * lb + 4 * cg + 4 * lane));
                                    v[0] = w0.x; v[1] = w0.y; v[2] = w0.z; v[3] = w0.w;
                                    v[4] = w1.x; v[5] = w1.y; v[6] = w1.z; v[7] = w1.w;
                                }
    #pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    const u32 xv = *reinterpret_cast<const XT *>(xs + (e[u] & kPanelIdxMask) * sizeof(XT));
                                    tm[u] = TINY ? (AT)(v[u] * xv)
                                                 : SMALL ? (AT)red32_lazy(v[u] * xv, M.m, mu32)
                                                 : MONT ? (AT)mont_red(v[u], xv, M.m, mneg) : (AT)red64((u64)v[u] * xv, M);
                                }
                            } else {
                                // +-1 sections (Sec. 2.4.2): x or m - x, no value
    #pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    const u32 xv = *reinterpret_cast<const XT *>(xs + (e[u] & kPanelIdxMask) * sizeof(XT));
                                    tm[u] = (AT)((e[u] & kPanelNeg) ? M.m - xv : xv);
                                }
                            }
                        }
                        // the warp's last lanes of this stage are in registers (the terms
                        // above read every loaded word): the buffer can be refilled
                        // while the sums go on
                        if (lb + 32u * kWarps >= nl) {
                            __syncwarp();
                            if (lane == 0) mbar_arrive(empty0 + 8u * b);
                            released = true;
                        }
                        const bool pack = valid && (general ? tl < lpg : tl - nlg < lpp);
                        // packs sit in lanes [0, lpg) and [nlg, nlg + lpp): a warp-uniform test
                        if (lb < lpg || (lb + 32u > nlg && lb < nlg + lpp)) {
                            // segmented warp sum over the lanes of one row, then one atomic.
                            // Packs of one row are adjacent within each section; a row
                            // can have packs in both sections, so the +-1 packs get keys
                            // of their own (the runs the sum joins must be contiguous)
                            AT sum = 0;
                            if (pack) sum = ((tm[0] + tm[1]) + (tm[2] + tm[3])) + ((tm[4] + tm[5]) + (tm[6] + tm[7]));
                            const u32 key = pack ? ((e[0] >> 16) | (general ? 0u : 0x20000u)) : (0x10000u + (u32)lane);
    #pragma unroll
                            for (int d = 1; d < 32; d <<= 1) {
                                const AT o = __shfl_down_sync(0xffffffffu, sum, d);
                                const u32 k2 = __shfl_down_sync(0xffffffffu, key, d);
                                if (lane + d < 32 && k2 == key) sum += o;
                            }
                            const u32 kp = __shfl_up_sync(0xffffffffu, key, 1);
                            if (pack && (lane == 0 || kp != key)) row_add<!SMALL>(acc + (key & 0xffffu), sum);
                        }
                        if (valid && !pack) {
    #pragma unroll
                            for (int u = 0; u < 8; ++u) row_add<!SMALL>(acc + (e[u] >> 16), tm[u]);
                        }
                    } else {
                        const u32 tl = lb + lane, c = min(32u, nl - lb);
                        const bool valid = tl < nl, general = tl < nlg;
                        u32 e[8], v[8];
                        XW xw[8];
    #pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            e[u] = 0;
                            v[u] = 0;
                            xw[u] = XW{};
                        }
                        if (valid) {
                            // entries of lane j of this 32-lane block: 4j..4j+3 and 4c+4j..4c+4j+3
                            const uint4 e0 = *reinterpret_cast<const uint4 *>(sb + 4 * (8 * lb + 4 * lane));
                            const uint4 e1 = *reinterpret_cast<const uint4 *>(sb + 4 * (8 * lb + 4 * c + 4 * lane));
                            e[0] = e0.x; e[1] = e0.y; e[2] = e0.z; e[3] = e0.w;
                            e[4] = e1.x; e[5] = e1.y; e[6] = e1.z; e[7] = e1.w;
                            if (general) {
                                if (SMALL) {
                                    const uint4 w = *reinterpret_cast<const uint4 *>(vb + 2 * 8 * tl);
                                    v[0] = w.x & 0xffffu; v[1] = w.x >> 16; v[2] = w.y & 0xffffu; v[3] = w.y >> 16;
                                    v[4] = w.z & 0xffffu; v[5] = w.z >> 16; v[6] = w.w & 0xffffu; v[7] = w.w >> 16;
                                } else {
                                    const u32 cg = min(32u, nlg - lb);
                                    const uint4 w0 = *reinterpret_cast<const uint4 *>(vb + 4 * (8 * lb + 4 * lane));
                                    const uint4 w1 = *reinterpret_cast<const uint4 *>(vb + 4 * (8 * lb + 4 * cg + 4 * lane));
                                    v[0] = w0.x; v[1] = w0.y; v[2] = w0.z; v[3] = w0.w;
                                    v[4] = w1.x; v[5] = w1.y; v[6] = w1.z; v[7] = w1.w;
                                }
                            }
    #pragma unroll
                            for (int u = 0; u < 8; ++u)
                                xw[u] = *reinterpret_cast<const XW *>(xs + (e[u] & kPanelIdxMask) * sizeof(XW));
                        }
                        const bool pack = valid && (general ? tl < lpg : tl - nlg < lpp);
                        // packs sit in lanes [0, lpg) and [nlg, nlg + lpp): a warp-uniform test
                        const bool packwarp = lb < lpg || (lb + 32u > nlg && lb < nlg + lpp);
                        // segmented warp sum over the lanes of one row, then one atomic.
                        // Packs of one row are adjacent within each section; a row
                        // can have packs in both sections, so the +-1 packs get keys
                        // of their own (the runs the sum joins must be contiguous).
                        // Bit i of seg: the lane 2^i further on is in the same run
                        u32 seg = 0;
                        bool head = false;
                        if (packwarp) {
                            const u32 key = pack ? ((e[0] >> 16) | (general ? 0u : 0x20000u)) : (0x10000u + (u32)lane);
    #pragma unroll
                            for (int i = 0; i < 5; ++i) {
                                const u32 k2 = __shfl_down_sync(0xffffffffu, key, 1 << i);
                                if (lane + (1 << i) < 32 && k2 == key) seg |= 1u << i;
                            }
                            const u32 kp = __shfl_up_sync(0xffffffffu, key, 1);
                            head = pack && (lane == 0 || kp != key);
                        }
    #pragma unroll
                        for (int k = 0; k < NV; k += VG) {
                            LT tm[8];
    #pragma unroll
                            for (int u = 0; u < 8; ++u) tm[u] = 0;
                            if (valid) {
    #pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    LT tv = 0;
    #pragma unroll
                                    for (int h = 0; h < VG; ++h) {
                                        const u32 xv = XC::get(xw[u], k + h);
                                        // +-1 sections (Sec. 2.4.2): x or m - x, no value
                                        const LT t1 = general ? (SMALL  ? (LT)red32_lazy(v[u] * xv, M.m, mu32)
                                                                 : MONT ? (LT)mont_red(v[u], xv, M.m, mneg)
                                                                        : (LT)red64((u64)v[u] * xv, M))
                                                              : (LT)((e[u] & kPanelNeg) ? M.m - xv : xv);
                                        tv |= t1 << (32 * h);
                                    }
                                    tm[u] = tv;
                                }
                            }
                            if (k == 0 && lb + 32u * kWarps >= nl) {
                                // the warp's last lanes of this stage are in registers (the
                                // terms above read every loaded word): the buffer can be
                                // refilled while the sums go on
                                __syncwarp();
                                if (lane == 0) mbar_arrive(empty0 + 8u * b);
                                released = true;
                            }
                            if (packwarp) {
                                LT sum = 0;
                                if (pack) sum = ((tm[0] + tm[1]) + (tm[2] + tm[3])) + ((tm[4] + tm[5]) + (tm[6] + tm[7]));
    #pragma unroll
                                for (int i = 0; i < 5; ++i) {
                                    const LT o = __shfl_down_sync(0xffffffffu, sum, 1 << i);
                                    if (seg & (1u << i)) sum += o;
                                }
                                if (head) row_add<!SMALL>(reinterpret_cast<LT *>(acc + (e[0] >> 16) * NV + k), sum);
                            }
                            if (valid && !pack) {
    #pragma unroll
                                for (int u = 0; u < 8; ++u) row_add<!SMALL>(reinterpret_cast<LT *>(acc + (e[u] >> 16) * NV + k), tm[u]);
                            }
                        }
                    }
                }
            } else {
                timed_out = true;
            }
            if (!released) {
                __syncwarp();
                if (lane == 0) mbar_arrive(empty0 + 8u * b);
            }
        }
    }
    if (__syncthreads_or(timed_out)) {
        // a copy, a buffer or the grid barrier never came: report, and give
        // the last copies a bounded chance to land before the CTA leaves
        if (t == 0) {
            if (status) atomicOr(status, 1);
            for (u32 s = ns > kPanelStages ? ns - kPanelStages : 0; s < ns; ++s)
                if ((int)s != skip_stage) mbar_wait(full0 + 8u * (s % kPanelStages), (s / kPanelStages) & 1u);
        }
        __syncthreads();
    }
    // Row sums are taken flat: element f is row f / NV, vector f % NV.  CTA j
    // of the cluster finishes the elements [j share, (j + 1) share): every
    // other CTA adds its partial sums of them into CTA j's with distributed
    // shared-memory reductions, posted as soon as its own stages are done
    // (while slower CTAs still sum), and one cluster barrier makes them
    // final.  A partial sum and the total are both sums of a row's terms, so
    // they stay below the same bound as a single CTA's row sum.
    constexpr u32 G = 16 / sizeof(AT);
    const u32 nf = nr * NV;
    const u32 share = ((nf + q - 1) / q + G - 1) / G * G;
    if (q > 1) {
        for (int j = 0; j < q; ++j) {
            if (j == rank) continue;
            const u32 jb = min(nf, (u32)j * share), je = min(nf, jb + share);
            const u32 base = map_cluster(acc, (u32)j);
            for (u32 f = jb + t; f < je; f += kPanelThreads) {
                const AT v = acc[f];
                // a pair of u32 sums adds word by word (no carry crosses)
                if constexpr (SMALL) {
                    if (v) red_cluster_add(base + f * (u32)sizeof(AT), v);
                } else {
                    if ((u32)v) red_cluster_add(base + f * (u32)sizeof(AT), (u32)v);
                    if ((u32)(v >> 32)) red_cluster_add(base + f * (u32)sizeof(AT) + 4u, (u32)(v >> 32));
                }
            }
        }
        cluster_sync_all();  // every partial sum of this CTA's share has arrived
    }
    const u32 rb = min(nf, rank * share), re = min(nf, rb + share);
    for (u32 f = rb + t; f < re; f += kPanelThreads) {
        u32 *yp = y + (long long)(r0 + f / NV) * ldy + f % NV;
        *yp = combine(red64(row_total(acc[f]), M), yp, false, M);
    }
}

// The panel kernel instance for (16-bit residues, vectors per pass).
typedef void (*PanelKernel)(const PanelPart, const u32 *, long long, u32 *, long long, const Mod, int *, int, int);
static PanelKernel panel_kernel(bool small, int nv, bool tiny = false, bool mont = false)
{
    if (tiny) return k_panel<true, 1, true>;
    if (small) return nv == 4 ? k_panel<true, 4> : nv == 2 ? k_panel<true, 2> : k_panel<true, 1>;
    if (mont) return nv == 2 ? k_panel<false, 2, false, true> : k_panel<false, 1, false, true>;
    return nv == 2 ? k_panel<false, 2> : k_panel<false, 1>;
}

int panel_max_clusters(bool small, int nv, int q, size_t smem, bool tiny)
{
    if (!(nv == 1 || nv == 2 || (nv == 4 && small))) return 0;
    const PanelKernel kf = panel_kernel(small, nv, tiny && small && nv == 1);
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)q, 1, 1);
    cfg.blockDim = dim3(kPanelThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)q;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kf, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// The panel kernel stages x itself when all its CTAs are resident at once
// (one row group per resident cluster); otherwise a staging launch runs first.
static bool panel_fused(const PanelPart &pp) { return pp.ngroup <= pp.resident; }

// One pass of the panel kernel over vectors vcol.. of the block.  conv: for a
// plan whose CTAs are all resident, the staged columns this launch converts
// (0: it reads column xcol that an earlier launch of the group staged).
static ffspmv_status run_panel(const Plan &P, const u32 *x, long long ldx, u32 *y, long long ldy,
                               int vcol, int conv, int xcol, const Mod &M, cudaStream_t st, const PanelCtl *ctl)
{
    PanelPart pp = P.panel;
    const int fused = panel_fused(pp) ? 1 : 0;
    if (fused) pp.xh = (char *)pp.xh + (size_t)xcol * pp.xstride * (pp.tiny ? 1 : pp.small ? 2 : 4);
    else conv = 0;
    if (!fused) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const unsigned sb =
            (unsigned)std::max<long long>(1, std::min<long long>((P.ncols / 4 + 255) / 256, 8LL * std::max(nsm, 1)));
        unsigned short *xs16 = (unsigned short *)pp.xh;
        u32 *xs32 = (u32 *)pp.xh;
        if (pp.tiny) k_x_stage<unsigned char, 1><<<sb, 256, 0, st>>>(x + vcol, ldx, P.ncols, (unsigned char *)pp.xh);
        else if (pp.small && pp.nv == 4) k_x_stage<unsigned short, 4><<<sb, 256, 0, st>>>(x + vcol, ldx, P.ncols, xs16);
        else if (pp.small && pp.nv == 2) k_x_stage<unsigned short, 2><<<sb, 256, 0, st>>>(x + vcol, ldx, P.ncols, xs16);
        else if (pp.small) k_x_stage<unsigned short, 1><<<sb, 256, 0, st>>>(x + vcol, ldx, P.ncols, xs16);
        else if (pp.nv == 2) k_x_stage<u32, 2><<<sb, 256, 0, st>>>(x + vcol, ldx, P.ncols, xs32);
        else k_x_stage<u32, 1><<<sb, 256, 0, st>>>(x + vcol, ldx, P.ncols, xs32);
        FF_CUDA(cudaGetLastError());
    }
    const PanelKernel kf = panel_kernel(pp.small, pp.nv, pp.tiny, pp.mont);
    cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pp.smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(pp.ngroup * pp.q), 1, 1);
    cfg.blockDim = dim3(kPanelThreads, 1, 1);
    cfg.dynamicSmemBytes = pp.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)pp.q;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    u32 *yv = y + vcol;
    const u32 *xv = x + vcol;
    int *status = ctl ? ctl->status : nullptr;
    const int skip = ctl ? ctl->skip_stage : -1;
    FF_CUDA(cudaLaunchKernelEx(&cfg, kf, pp, xv, ldx, yv, ldy, M, status, skip, conv));
    return FFSPMV_OK;
}

static int next_chunk(int left, bool has_atomic)
{
    if (has_atomic) return 1;
    return left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
}

long long count_plan_launches(const Plan &P, int nvec)
{
    if (P.nrows == 0) return 0;
    long long n = P.panel.on ? (P.panel.ngroup <= P.panel.resident ? 1LL : 2LL) * (nvec / P.panel.nv) : 0;
    for (const Phase &ph : P.phases) {
        if (ph.segs.empty()) continue;
        for (int c0 = 0; c0 < nvec; c0 += next_chunk(nvec - c0, ph.has_atomic))
            n += 1 + (ph.nsplit > 0 ? 1 : 0);
    }
    return n;
}

ffspmv_status run_plan(const Plan &P, const u32 *x, long long ldx, u32 *y,
                       long long ldy, int nvec, u32 m, u32 alpha, u32 beta,
                       cudaStream_t st, const PanelCtl *ctl)
{
    const Mod M1 = make_mod(m, alpha, beta);
    if (P.panel.on) {
        // panels first (every row written); the long rows' segments then add
        // in.  A plan for NV vectors per pass takes blocks of a multiple of NV
        if (nvec % P.panel.nv) return FFSPMV_ERR_ARG;
        for (int v = 0; v < nvec; v += P.panel.nv) {
            // one vector per pass: the first launch of each group of
            // P.panel.xcols vectors stages all of them
            const int g = P.panel.xcols, k = (v / P.panel.nv) % g;
            const int conv = k ? 0 : (P.panel.nv == 1 ? std::min(g, nvec - v) : 1);
            ffspmv_status r = run_panel(P, x, ldx, y, ldy, v, conv, k, M1, st, ctl);
            if (r != FFSPMV_OK) return r;
        }
    }
    for (size_t pi = 0; pi < P.phases.size(); ++pi) {
        const Phase &ph = P.phases[pi];
        if (ph.segs.empty()) continue;
        PlanParams pp = params_of(ph, P.acc_wide);
        if (pp.total_blocks <= 0) continue;
        int c0 = 0;
        while (c0 < nvec) {
            int nv = next_chunk(nvec - c0, ph.has_atomic);
            const u32 *xc = x + c0;
            u32 *yc = y + c0;
            bool vec4 = nv >= 4 && (ldx % 4 == 0) && ((uintptr_t)xc % 16 == 0);
            if (P.acc_wide)
                launch_nv<AccWide>(nv, pp, xc, ldx, yc, ldy, M1, P.carry, vec4, st);
            else
                launch_nv<AccSmall>(nv, pp, xc, ldx, yc, ldy, M1, P.carry, vec4, st);
            FF_CUDA(cudaGetLastError());
            if (ph.nsplit > 0) {
                int accum = ph.segs[0].accum;
                unsigned nb = (unsigned)((ph.nsplit + 255) / 256);
                k_coo_finish<<<nb, 256, 0, st>>>(ph.split_rows, ph.nsplit, P.carry, yc, ldy, M1, accum);
                FF_CUDA(cudaGetLastError());
            }
            c0 += nv;
        }
    }
    return FFSPMV_OK;
}

// ---------------------------------------------------------------------------
// A^T * x by scatter: every entry adds its reduced term into the exact 64-bit
// column sum acc[j*nv + v] (integer atomics are order independent, so the
// result is the same as the explicit transposed plan's).
__global__ void k_scatter_T(long long nrows, const long long *__restrict__ ptr,
                            const int *__restrict__ col, const u32 *__restrict__ val,
                            const u32 *__restrict__ x, long long ldx, int nv,
                            u64 *__restrict__ acc, const Mod M)
{
    const int G = 8;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x & (G - 1);
    if (i >= nrows) return;
    const long long s = ptr[i], e = ptr[i + 1];
    for (long long k = s + lane; k < e; k += G) {
        const long long j = col[k];
        const u32 a = val[k];
        for (int v = 0; v < nv; ++v) {
            u32 t = red64((u64)a * __ldg(x + i * ldx + v), M);
            if (t) atomicAdd(acc + j * nv + v, (u64)t);
        }
    }
}

__global__ void k_scatter_finish(long long ncols, int nv, u64 *__restrict__ acc,
                                 u32 *__restrict__ y, long long ldy, const Mod M)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncols * nv) return;
    const long long j = t / nv;
    const int v = (int)(t - j * nv);
    const u64 c = acc[t];
    acc[t] = 0;
    u32 *yp = y + j * ldy + v;
    *yp = combine(red64(c, M), yp, false, M);
}

ffspmv_status run_scatter_transpose(ffspmv_handle *h, const u32 *x,
                                    long long ldx, u32 *y, long long ldy,
                                    int nvec, u32 alpha, u32 beta,
                                    cudaStream_t st)
{
    const long long nrows = h->A.nrows, ncols = h->A.ncols;
    const Mod M = make_mod(h->m, alpha, beta);
    const int chunk = nvec < 16 ? nvec : 16;
    size_t need = (size_t)(ncols > 0 ? ncols : 1) * chunk;
    if (need > h->scatter_elems) {
        if (h->scatter) cudaFree(h->scatter);
        h->scatter = nullptr;
        h->scatter_elems = 0;
        if (cudaMalloc(&h->scatter, need * sizeof(u64)) != cudaSuccess) return FFSPMV_ERR_OOM;
        if (cudaMemset(h->scatter, 0, need * sizeof(u64)) != cudaSuccess) return FFSPMV_ERR_CUDA;
        h->scatter_elems = need;
    }
    for (int c0 = 0; c0 < nvec; c0 += chunk) {
        int nv = nvec - c0 < chunk ? nvec - c0 : chunk;
        if (nrows > 0) {
            long long threads = nrows * 8;
            unsigned nb = (unsigned)((threads + 255) / 256);
            k_scatter_T<<<nb, 256, 0, st>>>(nrows, h->d_rowptr, h->d_col, h->d_val,
                                            x + c0, ldx, nv, h->scatter, M);
            FF_CUDA(cudaGetLastError());
        }
        if (ncols > 0) {
            long long t = ncols * nv;
            k_scatter_finish<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(ncols, nv, h->scatter, y + c0, ldy, M);
            FF_CUDA(cudaGetLastError());
        }
    }
    return FFSPMV_OK;
}

// ---------------------------------------------------------------------------
__global__ void k_check_range(const u32 *__restrict__ x, long long rows,
                              long long ld, int nvec, u32 m, int *flag)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * nvec) return;
    const long long r = t / nvec;
    const int v = (int)(t - r * nvec);
    if (x[r * ld + v] >= m) atomicExch(flag, 1);
}

ffspmv_status check_range(const u32 *x, long long rows, long long ld, int nvec,
                          u32 m, int *d_flag, cudaStream_t st, bool *bad)
{
    *bad = false;
    if (rows == 0) return FFSPMV_OK;
    FF_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    long long t = rows * nvec;
    k_check_range<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(x, rows, ld, nvec, m, d_flag);
    FF_CUDA(cudaGetLastError());
    int hflag = 0;
    FF_CUDA(cudaMemcpyAsync(&hflag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    FF_CUDA(cudaStreamSynchronize(st));
    *bad = hflag != 0;
    return FFSPMV_OK;
}

}  // namespace ff
