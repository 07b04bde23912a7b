// The C ABI: argument checks, plan ownership, and dispatch to the kernels.
#include <cstdio>
#include <cstring>
#include <vector>

#include "ff_internal.cuh"
#include "ff_plan.h"
#include "ff_select.h"
#include "../../include/ffspmv_select.h"

using namespace ff;

namespace {

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
ffspmv_status to_host(const T *p, long long n, std::vector<T> &out, const T *&view)
{
    if (n <= 0) {
        view = p;
        return FFSPMV_OK;
    }
    if (!is_device_ptr(p)) {
        view = p;
        return FFSPMV_OK;
    }
    out.resize((size_t)n);
    FF_CUDA(cudaMemcpy(out.data(), p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost));
    view = out.data();
    return FFSPMV_OK;
}

void destroy_handle(ffspmv_handle *h)
{
    if (!h) return;
    free_plan(h->A);
    free_plan(h->AT);
    for (auto &dir : h->multi)
        for (ff::Plan *&mp : dir) {
            if (mp) free_plan(*mp);
            delete mp;
            mp = nullptr;
        }
    if (h->scatter) cudaFree(h->scatter);
    if (h->csr_arena) cudaFree(h->csr_arena);
    if (h->d_status) cudaFree(h->d_status);
    free_sequence_state(h);
    batch_forget(h);
    free_gf2(h);
    delete h;
}

// FFSPMV_FMT_AUTO (heuristic selector) takes the x-panel layout where it beat
// the binned one on every measured shape: at least 2^21 entries (enough to
// fill the stage pipelines of all SMs) and at least 3 entries per column
// (each column of x streamed through shared memory serves several entries),
// at any modulus (m > 2^16, 8-byte row sums: 61-67 vs 101 us on the 1M
// power-law matrix; 106-158 vs 211-246 us on held-out 34M-entry matrices when
// those sums were still u64 atomics).  Elsewhere AUTO is BINNED.
bool panel_preferred(long long ncols, long long nnz, u32 m)
{
    (void)m;
    return nnz >= (1LL << 21) && nnz >= 3 * ncols;
}

// Mean milliseconds of one Y = A X with plan P for nvec vectors (X = 0, Y
// scratch), after warm-up.
float time_whole_plan(const Plan &P, u32 m, int nvec = 1)
{
    u32 *x = nullptr, *y = nullptr;
    float ms = -1.0f;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t xb = (size_t)std::max<long long>(P.ncols, 1) * 4 * nvec, yb = (size_t)std::max<long long>(P.nrows, 1) * 4 * nvec;
    if (cudaMalloc(&x, xb) == cudaSuccess && cudaMalloc(&y, yb) == cudaSuccess && cudaMemset(x, 0, xb) == cudaSuccess &&
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        const int reps = 5;
        for (int w = 0; w < 2; ++w) run_plan(P, x, nvec, y, nvec, nvec, m, 1, 0, st);
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps; ++k) run_plan(P, x, nvec, y, nvec, nvec, m, 1, 0, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
            ms /= (float)reps;
        else
            ms = -1.0f;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (x) cudaFree(x);
    if (y) cudaFree(y);
    cudaGetLastError();
    return ms;
}

ffspmv_status build_with_selector(Plan &P, long long nrows, long long ncols,
                                  const long long *ptr, const int *col,
                                  const u32 *val, u32 m, const ffspmv_options &o)
{
    const bool exhaustive = o.selector == FFSPMV_SEL_EXHAUSTIVE;
    if (o.priority_format == FFSPMV_FMT_AUTO && !exhaustive && o.selector != FFSPMV_SEL_LEARNED &&
        panel_preferred(ncols, ptr[nrows], m)) {
        ffspmv_options o2 = o;
        o2.priority_format = FFSPMV_FMT_PANEL;
        return build_plan_ex(P, nrows, ncols, ptr, col, val, m, o2, nullptr);
    }
    if (o.priority_format == FFSPMV_FMT_AUTO && exhaustive && ptr[nrows] > 0) {
        // the exhaustive selector also times the whole x-panel plan against
        // the binned plan of its per-bin winners and keeps the faster
        ffspmv_options ob = o;
        ob.priority_format = FFSPMV_FMT_BINNED;
        Plan B, Q;
        ffspmv_status sb = build_with_selector(B, nrows, ncols, ptr, col, val, m, ob);
        if (sb != FFSPMV_OK) return sb;
        ffspmv_options oq = o;
        oq.priority_format = FFSPMV_FMT_PANEL;
        if (build_plan_ex(Q, nrows, ncols, ptr, col, val, m, oq, nullptr) == FFSPMV_OK && Q.panel.on) {
            const float tb = time_whole_plan(B, m), tq = time_whole_plan(Q, m);
            if (tq > 0.0f && (tb < 0.0f || tq < tb)) {
                free_plan(B);
                P = Q;
                return FFSPMV_OK;
            }
        }
        free_plan(Q);
        P = B;
        return FFSPMV_OK;
    }
    if (o.priority_format == FFSPMV_FMT_AUTO && o.selector == FFSPMV_SEL_LEARNED) {
        // the network's matrix-level outputs choose the layout: the x-panel
        // plan, the binned plan with its own per-bin table, or the binned
        // plan with the heuristic table (least predicted whole-plan time);
        // when the best of the other family is predicted within
        // FFSPMV_SEL_VERIFY_MARGIN, both are built and the faster is kept
        BinChoice bins[kBins];
        int layout = -1, alt = -1;
        ffspmv_status st = choose_bins(o.selector, nrows, ncols, ptr, col, val, m, o, bins, &layout, &alt);
        if (st != FFSPMV_OK) return st;
        // no network installed: the exhaustive bins, and the panel rule of AUTO
        if (layout < 0) layout = panel_preferred(ncols, ptr[nrows], m) ? FFSPMV_LAYOUT_PANEL : FFSPMV_LAYOUT_NETBINS;
        auto build_layout = [&](Plan &Q, int lay) -> ffspmv_status {
            ffspmv_options o2 = o;
            if (lay >= FFSPMV_LAYOUT_PANEL_Q1 && ptr[nrows] > 0) {
                o2.priority_format = FFSPMV_FMT_PANEL;
                if (lay <= FFSPMV_LAYOUT_PANEL_Q4) o2.panel_cluster = 1 << (lay - FFSPMV_LAYOUT_PANEL_Q1);
                if (build_plan_ex(Q, nrows, ncols, ptr, col, val, m, o2, nullptr) == FFSPMV_OK && Q.panel.on)
                    return FFSPMV_OK;
                free_plan(Q);
                Q = Plan();
                lay = FFSPMV_LAYOUT_NETBINS;
                o2.panel_cluster = o.panel_cluster;
            }
            o2.priority_format = FFSPMV_FMT_BINNED;
            return build_plan_ex(Q, nrows, ncols, ptr, col, val, m, o2, lay == FFSPMV_LAYOUT_BINNED ? nullptr : bins);
        };
        if ((st = build_layout(P, layout)) != FFSPMV_OK) return st;
        if (alt >= 0) {
            Plan Q;
            if (build_layout(Q, alt) == FFSPMV_OK) {
                const float tp = time_whole_plan(P, m), tq = time_whole_plan(Q, m);
                if (tq > 0.0f && (tp < 0.0f || tq < tp)) std::swap(P, Q);
            }
            free_plan(Q);
        }
        return FFSPMV_OK;
    }
    const bool wants_bins = o.priority_format == FFSPMV_FMT_BINNED ||
                            (o.priority_format == FFSPMV_FMT_AUTO &&
                             (o.selector == FFSPMV_SEL_LEARNED || o.selector == FFSPMV_SEL_EXHAUSTIVE));
    if (wants_bins && (o.selector == FFSPMV_SEL_LEARNED || o.selector == FFSPMV_SEL_EXHAUSTIVE)) {
        BinChoice bins[kBins];
        ffspmv_status st = choose_bins(o.selector, nrows, ncols, ptr, col, val, m, o, bins);
        if (st != FFSPMV_OK) return st;
        ffspmv_options o2 = o;
        o2.priority_format = FFSPMV_FMT_BINNED;
        return build_plan_ex(P, nrows, ncols, ptr, col, val, m, o2, bins);
    }
    ffspmv_options o2 = o;
    if (o2.priority_format == FFSPMV_FMT_AUTO) o2.priority_format = FFSPMV_FMT_BINNED;
    return build_plan_ex(P, nrows, ncols, ptr, col, val, m, o2, nullptr);
}

}  // namespace

namespace ff {
static thread_local char g_last_error[320] = "";

void note_cuda_error(cudaError_t e, const char *file, int line)
{
    const char *base = strrchr(file, '/');
    snprintf(g_last_error, sizeof g_last_error, "%s:%d: %s: %s", base ? base + 1 : file, line,
             cudaGetErrorName(e), cudaGetErrorString(e));
}
}  // namespace ff

extern "C" {

const char *ffspmv_last_error(void) { return ff::g_last_error; }

void ffspmv_options_default(ffspmv_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->selector = FFSPMV_SEL_HEURISTIC;
    o->use_pm1 = -1;
    o->priority_format = FFSPMV_FMT_AUTO;
    o->transpose_mode = FFSPMV_TRANSPOSE_EXPLICIT;
    o->value_check = 0;
    o->group_width = 0;
    o->ell_width = -1;
    o->barrier_spin_limit = 0;
    o->guard_bytes = 0;
    o->sequence_mode = 0;
    o->test_hooks = 0;
    o->panel_cluster = 0;
}

const char *ffspmv_status_string(ffspmv_status s)
{
    switch (s) {
    case FFSPMV_OK: return "ok";
    case FFSPMV_ERR_ARG: return "invalid argument";
    case FFSPMV_ERR_RANGE: return "input residue out of range";
    case FFSPMV_ERR_OOM: return "out of memory";
    case FFSPMV_ERR_CUDA: return "CUDA runtime error";
    case FFSPMV_ERR_UNSUPPORTED: return "unsupported format or size";
    case FFSPMV_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

ffspmv_status spmv_create_hybrid(ffspmv_t *out, int64_t nrows, int64_t ncols,
                                 int64_t nnz, const int64_t *row_ptr,
                                 const int32_t *col, const uint32_t *values,
                                 uint32_t modulus, const ffspmv_options *opt,
                                 ffspmv_stream_t stream)
{
    (void)stream;
    if (!out) return FFSPMV_ERR_ARG;
    *out = nullptr;
    if (nrows < 0 || ncols < 0 || nnz < 0 || modulus < 2u || !row_ptr) return FFSPMV_ERR_ARG;
    if (nrows >= (1LL << 32) - 1 || ncols >= (1LL << 31)) return FFSPMV_ERR_UNSUPPORTED;
    if (nnz > 0 && (!col || !values)) return FFSPMV_ERR_ARG;
    ffspmv_options o;
    ffspmv_options_default(&o);
    if (opt) o = *opt;
    if (o.transpose_mode < 0 || o.transpose_mode > 2) return FFSPMV_ERR_ARG;

    std::vector<long long> hptr;
    std::vector<int> hcol;
    std::vector<u32> hval;
    const long long *ptr = nullptr;
    const int *cidx = nullptr;
    const u32 *vals = nullptr;
    ffspmv_status st;
    if ((st = to_host((const long long *)row_ptr, nrows + 1, hptr, ptr)) != FFSPMV_OK) return st;
    if ((st = to_host((const int *)col, nnz, hcol, cidx)) != FFSPMV_OK) return st;
    if ((st = to_host((const u32 *)values, nnz, hval, vals)) != FFSPMV_OK) return st;
    if (ptr[0] != 0 || ptr[nrows] != nnz) return FFSPMV_ERR_ARG;
    for (long long i = 0; i < nrows; ++i)
        if (ptr[i + 1] < ptr[i]) return FFSPMV_ERR_ARG;
    for (long long k = 0; k < nnz; ++k)
        if (cidx[k] < 0 || cidx[k] >= ncols) return FFSPMV_ERR_ARG;

    ffspmv_handle *h = new (std::nothrow) ffspmv_handle();
    if (!h) return FFSPMV_ERR_OOM;
    h->opt = o;
    h->m = modulus;
    h->transpose_mode = o.transpose_mode;
    cudaGetDevice(&h->device);
    if (cudaMalloc(&h->d_status, 4 * sizeof(int)) != cudaSuccess) {
        h->d_status = nullptr;
        destroy_handle(h);
        return FFSPMV_ERR_OOM;
    }
    cudaMemset(h->d_status, 0, 4 * sizeof(int));
    h->h_ptr.assign(ptr, ptr + nrows + 1);
    h->h_col.assign(cidx, cidx + nnz);
    h->h_val.resize((size_t)nnz);
    for (long long k = 0; k < nnz; ++k) h->h_val[k] = vals[k] % modulus;
    st = build_with_selector(h->A, nrows, ncols, ptr, cidx, vals, modulus, o);
    if (st == FFSPMV_OK && o.transpose_mode == FFSPMV_TRANSPOSE_EXPLICIT) {
        std::vector<long long> tptr;
        std::vector<int> tcol;
        std::vector<u32> tval;
        transpose_csr(nrows, ncols, ptr, cidx, vals, tptr, tcol, tval);
        st = build_with_selector(h->AT, ncols, nrows, tptr.data(), tcol.data(), tval.data(), modulus, o);
        h->has_T = st == FFSPMV_OK;
    }
    if (st == FFSPMV_OK && o.transpose_mode == FFSPMV_TRANSPOSE_ATOMIC) {
        size_t b_ptr = (size_t)(nrows + 1) * 8, b_col = (size_t)nnz * 4, b_val = (size_t)nnz * 4;
        size_t o_col = (b_ptr + 255) / 256 * 256, o_val = o_col + (b_col + 255) / 256 * 256;
        if (cudaMalloc(&h->csr_arena, o_val + b_val + 4) != cudaSuccess) {
            h->csr_arena = nullptr;
            st = FFSPMV_ERR_OOM;
        } else {
            std::vector<u32> red((size_t)nnz);
            for (long long k = 0; k < nnz; ++k) red[k] = vals[k] % modulus;
            char *base = (char *)h->csr_arena;
            cudaMemcpy(base, ptr, b_ptr, cudaMemcpyHostToDevice);
            if (nnz) {
                cudaMemcpy(base + o_col, cidx, b_col, cudaMemcpyHostToDevice);
                cudaMemcpy(base + o_val, red.data(), b_val, cudaMemcpyHostToDevice);
            }
            h->d_rowptr = (const long long *)base;
            h->d_col = (const int *)(base + o_col);
            h->d_val = (const u32 *)(base + o_val);
            h->has_T = true;
            if (cudaGetLastError() != cudaSuccess) st = FFSPMV_ERR_CUDA;
        }
    }
    if (st != FFSPMV_OK) {
        destroy_handle(h);
        return st;
    }
    *out = h;
    return FFSPMV_OK;
}

// The x-panel plan of A (or A^T) for nv = 2 or 4 vectors per pass, built on
// first use from the handle's host copy of the matrix (synchronous).  *out is
// null when that layout does not exist for the matrix (the caller then runs
// one vector per pass).
static ffspmv_status ensure_multi(ffspmv_t h, bool transpose, int nv, const Plan **out)
{
    Plan *&mp = h->multi[transpose ? 1 : 0][nv == 4 ? 1 : 0];
    if (!mp) {
        Plan *np = new (std::nothrow) Plan();
        if (!np) return FFSPMV_ERR_OOM;
        ffspmv_options o = h->opt;
        o.priority_format = FFSPMV_FMT_PANEL;
        o.panel_cluster = (transpose ? h->AT : h->A).panel.q;
        const long long nr = h->A.nrows, nc = h->A.ncols;
        ffspmv_status st;
        if (!transpose) {
            st = build_plan_ex(*np, nr, nc, h->h_ptr.data(), h->h_col.data(), h->h_val.data(), h->m, o, nullptr, nv);
        } else {
            std::vector<long long> tptr;
            std::vector<int> tcol;
            std::vector<u32> tval;
            transpose_csr(nr, nc, h->h_ptr.data(), h->h_col.data(), h->h_val.data(), tptr, tcol, tval);
            st = build_plan_ex(*np, nc, nr, tptr.data(), tcol.data(), tval.data(), h->m, o, nullptr, nv);
        }
        if (st != FFSPMV_OK && st != FFSPMV_ERR_UNSUPPORTED) {
            free_plan(*np);
            delete np;
            return st;
        }
        // kept only where a pass over nv vectors beats nv one-vector passes
        // (measured once, here): wider x words and row sums shrink the panels
        // and row groups, and on matrices with few entries per column of a
        // CTA the extra stages cost more than the shared entry stream saves
        if (st == FFSPMV_OK && np->panel.on && !(h->opt.test_hooks & 4)) {
            const float tm = time_whole_plan(*np, h->m, nv);
            const float t1 = time_whole_plan(transpose ? h->AT : h->A, h->m, nv);
            if (!(tm > 0.0f && t1 > 0.0f && tm < 0.97f * t1)) st = FFSPMV_ERR_UNSUPPORTED;
        }
        if (st != FFSPMV_OK) {
            free_plan(*np);
            *np = Plan();  // no such layout, or not faster: remembered as a plan without panels
        }
        mp = np;
    }
    *out = (mp->panel.on && mp->panel.nv == nv) ? mp : nullptr;
    return FFSPMV_OK;
}

// Vectors in the next pass over a block with `left` vectors still to go.
static int pass_width(const Plan &P, int left)
{
    if (left >= 4 && P.panel.small) return 4;
    return left >= 2 ? 2 : 1;
}

// The next pass over a block with `left` vectors to go: the widest wide
// layout that exists and was kept, else the base plan for all `left` vectors
// (one-vector passes, x staged four vectors at a time).
static ffspmv_status next_pass(ffspmv_t h, bool transpose, const Plan *P, int left, const Plan **Q, int *nv)
{
    *Q = P;
    *nv = left;
    if (h->opt.test_hooks & 8) return FFSPMV_OK;
    for (int w = pass_width(*P, left); w > 1; w /= 2) {
        const Plan *M = nullptr;
        ffspmv_status s = ensure_multi(h, transpose, w, &M);
        if (s != FFSPMV_OK) return s;
        if (M) {
            *Q = M;
            *nv = w;
            return FFSPMV_OK;
        }
    }
    return FFSPMV_OK;
}

static ffspmv_status apply_common(ffspmv_t h, bool transpose, const uint32_t *d_x,
                                  int64_t ldx, uint32_t *d_y, int64_t ldy,
                                  int32_t nvec, uint32_t alpha, uint32_t beta,
                                  ffspmv_stream_t stream)
{
    if (!h || nvec < 1 || ldx < nvec || ldy < nvec) return FFSPMV_ERR_ARG;
    const long long in_rows = transpose ? h->A.nrows : h->A.ncols;
    const long long out_rows = transpose ? h->A.ncols : h->A.nrows;
    if ((in_rows > 0 && !d_x) || (out_rows > 0 && !d_y)) return FFSPMV_ERR_ARG;
    if (transpose && !h->has_T) return FFSPMV_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (h->opt.value_check) {
        bool bad = false;
        ffspmv_status s = check_range(d_x, in_rows, ldx, nvec, h->m, h->d_status + 1, st, &bad);
        if (s != FFSPMV_OK) return s;
        if (bad) return FFSPMV_ERR_RANGE;
    }
    if (out_rows == 0) return FFSPMV_OK;
    if (transpose && h->transpose_mode == FFSPMV_TRANSPOSE_ATOMIC)
        return run_scatter_transpose(h, d_x, ldx, d_y, ldy, nvec, alpha % h->m, beta % h->m, st);
    const Plan *P = transpose ? &h->AT : &h->A;
    PanelCtl ctl;
    ctl.status = h->d_status + 2;
    ctl.skip_stage = (h->opt.test_hooks & 2) ? 1 : -1;
    if (!P->panel.on || nvec == 1)
        return run_plan(*P, d_x, ldx, d_y, ldy, nvec, h->m, alpha % h->m, beta % h->m, st, &ctl);
    // x-panel blocks: passes of 4 or 2 vectors read the matrix once for all
    // of them (Sec. 2.5.1), on layouts built for that width
    for (int c0 = 0; c0 < nvec;) {
        const Plan *Q = P;
        int nv = 1;
        ffspmv_status s = next_pass(h, transpose, P, nvec - c0, &Q, &nv);
        if (s != FFSPMV_OK) return s;
        s = run_plan(*Q, d_x + c0, ldx, d_y + c0, ldy, nv, h->m, alpha % h->m, beta % h->m, st, &ctl);
        if (s != FFSPMV_OK) return s;
        c0 += nv;
    }
    return FFSPMV_OK;
}

ffspmv_status spmv_apply(ffspmv_t h, const uint32_t *d_x, int64_t ldx, uint32_t *d_y,
                         int64_t ldy, int32_t nvec, uint32_t alpha, uint32_t beta,
                         ffspmv_stream_t stream)
{
    return apply_common(h, false, d_x, ldx, d_y, ldy, nvec, alpha, beta, stream);
}

ffspmv_status spmv_apply_transpose(ffspmv_t h, const uint32_t *d_x, int64_t ldx,
                                   uint32_t *d_y, int64_t ldy, int32_t nvec,
                                   uint32_t alpha, uint32_t beta, ffspmv_stream_t stream)
{
    return apply_common(h, true, d_x, ldx, d_y, ldy, nvec, alpha, beta, stream);
}

ffspmv_status spmv_create_binned(ffspmv_t *out, int64_t nrows, int64_t ncols, int64_t nnz,
                                 const int64_t *row_ptr, const int32_t *col, const uint32_t *values,
                                 uint32_t modulus, const int32_t *best, const ffspmv_options *opt,
                                 ffspmv_stream_t stream)
{
    if (!out || !best) return FFSPMV_ERR_ARG;
    *out = nullptr;
    ffspmv_options o;
    ffspmv_options_default(&o);
    if (opt) o = *opt;
    // build through the normal path with the heuristic table, then rebuild A's
    // plan with the given bins (A^T keeps the options' selector)
    ffspmv_options o2 = o;
    o2.priority_format = FFSPMV_FMT_BINNED;
    o2.selector = FFSPMV_SEL_HEURISTIC;
    ffspmv_status st = spmv_create_hybrid(out, nrows, ncols, nnz, row_ptr, col, values, modulus, &o2, stream);
    if (st != FFSPMV_OK) return st;
    ffspmv_handle *h = *out;
    BinChoice bins[kBins];
    for (int b = 0; b < kBins; ++b) {
        const int f = best[3 * b], pm = best[3 * b + 1], valid = best[3 * b + 2];
        bins[b] = (valid && f >= 0 && f < kFormats) ? format_choice(f, pm ? 1 : 0)
                                                   : heuristic_bin_choice(b, 0.0, o.use_pm1);
    }
    free_plan(h->A);
    h->A = Plan();
    st = build_plan_ex(h->A, nrows, ncols, h->h_ptr.data(), h->h_col.data(), h->h_val.data(), modulus, o2, bins);
    if (st != FFSPMV_OK) {
        destroy_handle(h);
        *out = nullptr;
    }
    return st;
}

ffspmv_status spmv_destroy(ffspmv_t h)
{
    destroy_handle(h);
    return FFSPMV_OK;
}

ffspmv_status spmv_describe_plan(ffspmv_t h, char *buf, size_t len)
{
    if (!h || !buf || len == 0) return FFSPMV_ERR_ARG;
    std::string s = "A  " + h->A.summary;
    if (h->has_T && h->transpose_mode == FFSPMV_TRANSPOSE_EXPLICIT) s += "A^T " + h->AT.summary;
    else if (h->transpose_mode == FFSPMV_TRANSPOSE_ATOMIC) s += "A^T by 64-bit atomic scatter\n";
    size_t n = s.size() < len - 1 ? s.size() : len - 1;
    memcpy(buf, s.data(), n);
    buf[n] = '\0';
    return FFSPMV_OK;
}

ffspmv_status spmv_count_launches(ffspmv_t h, int32_t transpose, int32_t nvec, int64_t *launches)
{
    if (!h || !launches || nvec < 1) return FFSPMV_ERR_ARG;
    long long n = 0;
    if (transpose && !h->has_T) return FFSPMV_ERR_UNSUPPORTED;
    if (h->opt.value_check) n += 1;
    if (transpose && h->transpose_mode == FFSPMV_TRANSPOSE_ATOMIC) {
        const int chunk = nvec < 16 ? nvec : 16;
        n += 2LL * ((nvec + chunk - 1) / chunk);
    } else {
        const Plan &P = transpose ? h->AT : h->A;
        if (!P.panel.on || nvec == 1) {
            n += count_plan_launches(P, nvec);
        } else {
            for (int c0 = 0; c0 < nvec;) {
                const Plan *Q = &P;
                int nv = 1;
                ffspmv_status s = next_pass(h, transpose != 0, &P, nvec - c0, &Q, &nv);
                if (s != FFSPMV_OK) return s;
                n += count_plan_launches(*Q, nv);
                c0 += nv;
            }
        }
    }
    *launches = n;
    return FFSPMV_OK;
}

ffspmv_status spmv_get_info(ffspmv_t h, int64_t *nrows, int64_t *ncols, int64_t *nnz,
                            uint32_t *modulus, int64_t *device_bytes)
{
    if (!h) return FFSPMV_ERR_ARG;
    if (nrows) *nrows = h->A.nrows;
    if (ncols) *ncols = h->A.ncols;
    if (nnz) *nnz = h->A.nnz;
    if (modulus) *modulus = h->m;
    if (device_bytes)
        *device_bytes = (int64_t)(h->A.arena_bytes + h->AT.arena_bytes);
    return FFSPMV_OK;
}

ffspmv_status spmv_check_status(ffspmv_t h, ffspmv_stream_t stream)
{
    if (!h || !h->d_status) return FFSPMV_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int word = 0;
    if (cudaMemcpyAsync(&word, h->d_status + 2, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FFSPMV_ERR_CUDA;
    if (word) {
        cudaMemsetAsync(h->d_status + 2, 0, sizeof(int), st);
        return FFSPMV_ERR_TIMEOUT;
    }
    return FFSPMV_OK;
}

}  // extern "C"
