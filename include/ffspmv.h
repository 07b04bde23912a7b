/*
 * ffspmv: exact sparse matrix x dense vector / block products over Z/mZ on
 * GB300 (sm_103a), after Boyer, Dumas and Giorgi, "Exact Sparse
 * Matrix-Vector Multiplication on GPU's and Multicore Architectures".
 *
 * C ABI.  No C++ or PyTorch type appears in a signature.  Pointers named d_*
 * are CUDA device pointers, h_* host pointers; "host or device" pointers are
 * detected with cudaPointerGetAttributes.  Every call is asynchronous with
 * respect to the host and ordered on the `stream` it is given, unless stated
 * otherwise; errors found on the host are returned before anything is
 * enqueued.
 *
 * Residues are uint32 in [0, m).  All results are the exact representatives in
 * [0, m); inputs x must already be in [0, m) (checked when
 * ffspmv_options.value_check = 1, otherwise a larger x gives an unspecified
 * but memory-safe result).
 *
 * Dense blocks of nvec vectors are row-major with a leading dimension:
 * element (k, v) of X is X[k*ldx + v] (ldx >= nvec).  nvec = 1, ldx = 1 is a
 * plain vector.  Sec. 2.5.1 leaves the multi-vector layout open; this is the
 * "one matrix pass, vectors read and written contiguously" form.
 */
#ifndef FFSPMV_H
#define FFSPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ffspmv_stream_t; /* a cudaStream_t; NULL = legacy default stream */
typedef struct ffspmv_handle *ffspmv_t;       /* opaque; owns all device format data */

typedef enum {
    FFSPMV_OK = 0,
    FFSPMV_ERR_ARG = 1,         /* bad argument: null pointer, size, stride, modulus */
    FFSPMV_ERR_RANGE = 2,       /* an input residue x >= m (value_check = 1) */
    FFSPMV_ERR_OOM = 3,         /* device or host allocation failed */
    FFSPMV_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    FFSPMV_ERR_UNSUPPORTED = 5, /* format or size guard refused (e.g. DIA of a random matrix) */
    FFSPMV_ERR_TIMEOUT = 6      /* a bounded device wait expired (grid barrier) */
} ffspmv_status;

/* Storage formats (Sec. 2.1 and 2.4).  FFSPMV_FMT_AUTO, decided separately
 * for A and A^T, by opt.selector:
 *   HEURISTIC (and FIXED): the x-panel layout when nnz >= 2^21 and nnz >=
 *     3 * ncols, else the binned layout with the heuristic table;
 *   LEARNED: the layout of least predicted whole-plan time among x-panel,
 *     binned with the network's per-bin table and binned with the heuristic
 *     table (the network's matrix-level outputs); without installed weights,
 *     the exhaustive bins and the HEURISTIC panel rule;
 *   EXHAUSTIVE: times the x-panel plan and the binned plan of the per-bin
 *     winners on the device and keeps the faster. */
enum {
    FFSPMV_FMT_AUTO = 0,
    FFSPMV_FMT_CSR = 1,     /* plain CSR, one fixed thread-group width per row */
    FFSPMV_FMT_ELLR = 2,    /* ELL_R: column-major ELL + per-row counts (Sec. 2.4.3) */
    FFSPMV_FMT_COO = 3,     /* coordinate triples, element-parallel segmented sums */
    FFSPMV_FMT_COOS = 4,    /* COO_S: CSR over the non-empty rows only (Sec. 2.4.4) */
    FFSPMV_FMT_DIA = 5,     /* diagonals + offsets; refused past a size guard */
    FFSPMV_FMT_HYBRID = 6,  /* paper heuristic: DIA + ELL_R(w) + CSR/COO/COO_S residue (Sec. 2.4.5) */
    FFSPMV_FMT_BINNED = 7,  /* rows binned by length, one format per bin */
    FFSPMV_FMT_PANEL = 8    /* row groups x column groups (CTA clusters), x streamed through
                               shared memory in panels (not in the paper); x staged as u8
                               (m <= 256), u16 (m <= 2^16) or u32 */
};

/* Format selectors (how FFSPMV_FMT_AUTO / FFSPMV_FMT_BINNED pick). */
enum {
    FFSPMV_SEL_HEURISTIC = 0,  /* the paper's chooser, constants of this library */
    FFSPMV_SEL_LEARNED = 1,    /* the selector network (ffspmv_selector_load) */
    FFSPMV_SEL_EXHAUSTIVE = 2, /* time every candidate per bin on the device */
    FFSPMV_SEL_FIXED = 3       /* use priority_format as is */
};

/* Transposed products. */
enum {
    FFSPMV_TRANSPOSE_EXPLICIT = 0, /* build A^T's plan at create time (default) */
    FFSPMV_TRANSPOSE_ATOMIC = 1,   /* scatter with exact 64-bit integer atomics */
    FFSPMV_TRANSPOSE_NONE = 2      /* no transposed product on this handle */
};

typedef struct {
    int32_t selector;          /* FFSPMV_SEL_*; default HEURISTIC */
    int32_t use_pm1;           /* 1: segregate +-1 entries into value-free parts (Sec. 2.4.2); -1 = let the selector decide (default) */
    int32_t priority_format;   /* FFSPMV_FMT_*; default AUTO */
    int32_t transpose_mode;    /* FFSPMV_TRANSPOSE_*; default EXPLICIT */
    int32_t value_check;       /* 1: check x < m on every apply (one extra pass) */
    int32_t group_width;       /* CSR lanes per row (1..32), 0 = from the mean row length */
    int32_t ell_width;         /* ELL_R width for HYBRID, -1 = heuristic */
    uint32_t barrier_spin_limit; /* grid-barrier spins before FFSPMV_ERR_TIMEOUT; 0 = default */
    int64_t guard_bytes;       /* size guard for ELL_R / DIA storage; 0 = default (32 GiB) */
    int32_t sequence_mode;     /* block sequence: 0 = persistent kernel when possible, 1 = one launch per kernel per step */
    int32_t test_hooks;        /* testing only, 0 in normal use: bit 0 = one CTA of the persistent
                                  sequence kernel never arrives at its first grid barrier, so the
                                  bounded wait of every other CTA runs out (FFSPMV_ERR_TIMEOUT);
                                  bit 1 = the x-panel kernel never issues the copies of the second
                                  stage of each CTA, so the waits for it run out (the status word
                                  read by spmv_check_status); bit 2 = x-panel blocks always take
                                  the 2- and 4-vector passes, without the timing that decides it;
                                  bit 3 = x-panel blocks never take them (one-vector passes) */
    int32_t panel_cluster;     /* x-panel layout: CTAs per cluster (column groups); 0 = chosen by
                                  the builder, 1, 2 or 4 to force one */
} ffspmv_options;

/* Fill *opt with the defaults. */
void ffspmv_options_default(ffspmv_options *opt);

/*
 * Build the device plan of an nrows x ncols matrix given in CSR (Sec. 2.1):
 * row i holds entries row_ptr[i] <= k < row_ptr[i+1], A[i, col[k]] = values[k].
 * row_ptr: int64[nrows+1] (row_ptr[0] = 0, non-decreasing); col: int32[nnz]
 * in [0, ncols); values: uint32[nnz], reduced mod m on entry (values >= m are
 * accepted); repeated (i, j) pairs add up.  The three arrays may be host or
 * device memory; they are copied and may be freed on return.
 * modulus: 2 <= m <= 2^32 - 1.  opt: NULL = defaults.  The call is
 * synchronous (it returns once the plan is resident on the current device).
 * Format choice follows Sec. 2.4.4-2.4.5 (hybridisation and the heuristic chooser)
 * or the selector named in opt.  On error *out is NULL and nothing leaks.
 */
ffspmv_status spmv_create_hybrid(ffspmv_t *out, int64_t nrows, int64_t ncols,
                                 int64_t nnz, const int64_t *row_ptr,
                                 const int32_t *col, const uint32_t *values,
                                 uint32_t modulus, const ffspmv_options *opt,
                                 ffspmv_stream_t stream);

/*
 * Y <- alpha*A*X + beta*Y (mod m), Sec. 2 (the operation y <- alpha A x +
 * beta y and its block form).  d_x: ncols x nvec (ldx), d_y: nrows x nvec
 * (ldy); 1 <= nvec; alpha, beta < m (reduced if not).  beta = 0 never reads
 * d_y ("apply": y <- A x).  d_x and d_y must not overlap.  On a handle whose
 * plan is the x-panel layout, a block runs in passes of 4 vectors (m <=
 * 2^16) or 2, then 1: each pass reads the matrix once for all its vectors
 * (Sec. 2.5.1) on an x-panel layout built for that width; the first block
 * that needs a width builds its layout and times one pass of it against the
 * same vectors one at a time (synchronous, host work plus one allocation
 * per handle, direction and width), and keeps it only if it is faster.  Calls on one handle must not
 * overlap on the GPU (the x-panel plans stage x in buffers of the handle).
 */
ffspmv_status spmv_apply(ffspmv_t h, const uint32_t *d_x, int64_t ldx,
                         uint32_t *d_y, int64_t ldy, int32_t nvec,
                         uint32_t alpha, uint32_t beta, ffspmv_stream_t stream);

/*
 * Y <- alpha*A^T*X + beta*Y (mod m): the transpose product (Sec. 1).  d_x:
 * nrows x nvec, d_y: ncols x nvec.  FFSPMV_ERR_UNSUPPORTED when the handle
 * was created with FFSPMV_TRANSPOSE_NONE.
 */
ffspmv_status spmv_apply_transpose(ffspmv_t h, const uint32_t *d_x,
                                   int64_t ldx, uint32_t *d_y, int64_t ldy,
                                   int32_t nvec, uint32_t alpha, uint32_t beta,
                                   ffspmv_stream_t stream);

/*
 * The matrix sequence of block Wiedemann (Sec. 3, step 1, with independent
 * left and right projections): V_0 = Y, V_{i+1} = A*V_i (mod p) and
 * S_i = X^T * V_i (mod p), all kept on the device (Sec. 2.5.2).  This call
 * computes the nsteps blocks S_start_step .. S_{start_step+nsteps-1}.  A must
 * be square; p is the handle's modulus.  d_X, d_Y: n x s row-major (ld = s),
 * 1 <= s <= 32.  d_S: nsteps x s x s, S_{start_step+i}[a][b] at
 * d_S[(i*s + a)*s + b].
 * d_V_state: n x s, in/out, for checkpoint and resume.  With start_step = 0
 * it may be NULL; if given it receives V_nsteps = A^nsteps * Y.  With
 * start_step > 0 it is required: on entry it holds V_start_step (what an
 * earlier call left there), d_Y is not read (may be NULL), and on return it
 * holds V_{start_step+nsteps}.  The steps run as one persistent cooperative
 * kernel captured in a CUDA graph when the grid fits on the device, else as
 * one stream of per-step launches; the graph is kept on the handle and
 * re-captured when s, nsteps, d_X, d_Y (or d_V_state), d_S change.
 * Synchronises `stream` and returns FFSPMV_ERR_TIMEOUT if a bounded
 * grid-barrier wait expired.  FFSPMV_ERR_ARG: start_step < 0, nsteps < 0,
 * s outside [1, 32], A not square, a missing pointer.
 */
ffspmv_status spmv_block_sequence(ffspmv_t h, const uint32_t *d_X,
                                  const uint32_t *d_Y, int32_t s,
                                  int64_t start_step, int64_t nsteps,
                                  uint32_t *d_S, uint32_t *d_V_state,
                                  ffspmv_stream_t stream);

/*
 * One step's projection for a sequence whose rows are split over several
 * processes (each holding rows r0..r1 of A, X and V): d_Sacc[a*s + b] +=
 * sum over the n rows k of X[k][a] * V[k][b], reduced mod p before it is
 * added (d_Sacc: s x s uint64, device, zero before the first call; one call
 * adds at most one value below p per SM to each entry, so the accumulators
 * of many calls and processes stay far below 2^64).  d_X, d_V: n x s row-major (ld = s), residues below p;
 * 1 <= s <= 32, p >= 2.  spmv_block_project_finish then writes S = Sacc mod p
 * (s x s uint32) and zeroes Sacc.  Asynchronous on `stream`; FFSPMV_ERR_ARG
 * on a bad size or a missing pointer.
 */
ffspmv_status spmv_block_project(uint32_t p, int64_t n, int32_t s, const uint32_t *d_X,
                                 const uint32_t *d_V, uint64_t *d_Sacc, ffspmv_stream_t stream);
ffspmv_status spmv_block_project_finish(uint32_t p, int32_t s, uint64_t *d_Sacc, uint32_t *d_S,
                                        ffspmv_stream_t stream);

/*
 * Independent products Y_j = A_j * X_j (mod m_j), j < count, in one launch
 * (not in the paper).  hs: host array of handles (each with its own
 * modulus); d_x / d_y: host arrays of device pointers, X_j: ncols_j x nvec[j]
 * row-major (ld = nvec[j]), Y_j: nrows_j x nvec[j]; 1 <= nvec[j] <= 32.
 * The work list is rebuilt on the host only when the set of handles or nvec
 * changes; that first call also times a few tile shapes (rows per work item,
 * length from which a row gets a whole CTA) on the device and keeps the
 * fastest, writing the outputs several times with the same values.  Not
 * thread-safe: one host thread at a time.
 */
ffspmv_status spmv_batch_apply(int32_t count, const ffspmv_t *hs,
                               const uint32_t *const *d_x,
                               uint32_t *const *d_y, const int32_t *nvec,
                               ffspmv_stream_t stream);

/*
 * Y <- alpha*A^T*X + beta*Y (mod m), like spmv_apply_transpose with
 * FFSPMV_TRANSPOSE_ATOMIC, but without allocating anything: for callers that
 * cannot let a library call cudaMalloc or cudaFree while they run (a serving
 * process whose device memory is all reserved up front for its own pool; a
 * latency-bound caller that cannot take the implicit device-wide
 * synchronisation of cudaFree).  The paper has no counterpart of this call.
 * The exact per-column sums live in one fixed 8 MiB array of 2^20 64-bit
 * words that every device which loads the library holds until the process
 * exits; ncols * min(nvec, 16) must fit in it, so ncols <= 2^20 (larger
 * ncols: FFSPMV_ERR_UNSUPPORTED; wider blocks are done 2^20/ncols vectors at
 * a time).  h must have been created with FFSPMV_TRANSPOSE_ATOMIC (else
 * FFSPMV_ERR_UNSUPPORTED), and h's device must be the current device (else
 * FFSPMV_ERR_ARG).  A handle created with value_check = 1 gets the same
 * input check as spmv_apply_transpose (FFSPMV_ERR_RANGE when some x >= m;
 * that check synchronises `stream`).  The first call on a device, with that device
 * current, looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array and
 * each clears the part it uses: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and give wrong results.
 */
ffspmv_status spmv_apply_transpose_noalloc(ffspmv_t h, const uint32_t *d_x,
                                           int64_t ldx, uint32_t *d_y, int64_t ldy,
                                           int32_t nvec, uint32_t alpha, uint32_t beta,
                                           ffspmv_stream_t stream);

/* Free every device buffer of h.  NULL is accepted. */
ffspmv_status spmv_destroy(ffspmv_t h);

/* Static string naming a status code. */
const char *ffspmv_status_string(ffspmv_status s);

/* The last CUDA runtime failure seen by this host thread ("file:line: name:
 * description"), or "" if none: the detail behind FFSPMV_ERR_CUDA. */
const char *ffspmv_last_error(void);

/* Human-readable summary of the chosen parts, bytes and bins ('\0'-terminated,
 * truncated to len). */
ffspmv_status spmv_describe_plan(ffspmv_t h, char *buf, size_t len);

/* Number of kernel launches that one spmv_apply (transpose = 0) or
 * spmv_apply_transpose (transpose = 1) call with nvec vectors enqueues
 * (nothing is enqueued; on an x-panel handle this builds the layouts for
 * the pass widths the block needs, as spmv_apply does). */
ffspmv_status spmv_count_launches(ffspmv_t h, int32_t transpose, int32_t nvec,
                                  int64_t *launches);

/* Matrix shape, nnz, modulus and device bytes of the plan (A and A^T). */
ffspmv_status spmv_get_info(ffspmv_t h, int64_t *nrows, int64_t *ncols,
                            int64_t *nnz, uint32_t *modulus,
                            int64_t *device_bytes);

/*
 * Products over GF(2) = Z/2Z with bit-packed vectors (Sec. 2 at m = 2: a sum
 * is an exclusive or and an entry counts when its value is odd; packing many
 * vectors into machine words is the binary case the paper's closing remarks
 * point to): Y = A X (transpose = 0) or Y = A^T X (transpose = 1), or, with
 * accumulate = 1, Y ^= A X.  h must have modulus 2 (else
 * FFSPMV_ERR_UNSUPPORTED).  d_X: in_rows x words 64-bit words, row-major,
 * bit b of word k of row j = component 64k + b of x_j (in_rows = ncols, or
 * nrows for A^T); d_Y: out_rows x words; words >= 1.  Repeated (i, j) pairs
 * add up, so an even number of odd copies cancels.  The first call for A (or
 * A^T) builds the pattern of the odd entries on the device (synchronous);
 * later calls are stream-ordered and asynchronous.  d_X and d_Y must not
 * overlap.  Not in the paper as a kernel.
 */
ffspmv_status spmv_apply_gf2(ffspmv_t h, int32_t transpose, const uint64_t *d_X,
                             uint64_t *d_Y, int32_t words, int32_t accumulate,
                             ffspmv_stream_t stream);

/*
 * Synchronises `stream`, then reads and clears h's device status word:
 * FFSPMV_ERR_TIMEOUT if a bounded device wait of an earlier spmv_apply /
 * spmv_apply_transpose on h ran out (the PANEL kernel's wait for a stage's
 * copies; the outputs of that call are then wrong), else FFSPMV_OK.  The
 * apply calls are asynchronous and do not read the word themselves.
 */
ffspmv_status spmv_check_status(ffspmv_t h, ffspmv_stream_t stream);

/*
 * Testing aid for the x-panel layout (FFSPMV_FMT_PANEL); the paper has no
 * counterpart.  Runs only the host half of the layout for the CSR matrix
 * (row_ptr, col, values as in spmv_create_hybrid, host memory) with q CTAs
 * per cluster (1, 2 or 4; 0 = the builder's choice, with clusters / q
 * resident clusters of q, stats[9] telling which), `clusters` resident
 * clusters and nv vectors per
 * pass (1, 2, or 4 when m <= 2^16: the geometry of the layout that a block
 * of that many vectors runs on), then decodes
 * every stored entry back to (row, column, value) and writes the first `cap`
 * of them to out_row / out_col / out_val (host arrays); *out_n = the number
 * decoded.  Padding (value 0) is skipped, so are explicit zeros; rows longer
 * than 32768 entries are not part of the layout.  use_pm1 = 1 puts the +-1
 * entries in value-free sections (decoded as 1 or m - 1).  stats (NULL or
 * double[10]): stages, share of lanes that are packs, mean shared-memory
 * wavefronts of a warp's x gather and of its row-sum atomic per slot (the
 * bank model of the layout), entries in +-1 sections, padding entries, panel
 * bytes, stage capacity, packs that break the kernel's segmented warp sum
 * (entries not all of one row, or lanes of one row and section that are not
 * contiguous within their warp; 0 when the layout is sound), q.  No device
 * call is made.
 */
ffspmv_status ffspmv_panel_decode(int64_t nrows, int64_t ncols, const int64_t *row_ptr,
                                  const int32_t *col, const uint32_t *values, uint32_t m,
                                  int32_t use_pm1, int32_t q, int32_t nv, int32_t clusters,
                                  int64_t cap, int64_t *out_row, int64_t *out_col, uint32_t *out_val,
                                  int64_t *out_n, double *stats);

#ifdef __cplusplus
}
#endif
#endif /* FFSPMV_H */
