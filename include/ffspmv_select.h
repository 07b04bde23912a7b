/*
 * ffspmv format selection: the exhaustive per-bin search, the matrix features
 * and the selector network (a small MLP) that replaces the heuristic chooser
 * of Sec. 2.4.5 ("Heuristic format chooser"), whose parameters the paper
 * leaves to architecture-specific tuning.  The selector only picks storage
 * formats: it has no effect on the arithmetic, so every plan it yields gives
 * the same (exact) results.
 *
 * The binned layout (FFSPMV_FMT_BINNED) puts the empty rows in bin 0 and the
 * rows with 2^(b-2) < length <= 2^(b-1) in bin b (1 <= b <= 16; bin 16 also
 * takes every longer row).  Each non-empty bin gets one candidate format:
 *
 *   0 ELL_R (one thread per row)    5 CSR, 16 lanes per row
 *   1 CSR, 1 lane per row           6 CSR, 32 lanes per row
 *   2 CSR, 2 lanes per row          7 CSR, one CTA per row
 *   3 CSR, 4 lanes per row          8 CSR, long rows cut across CTAs
 *   4 CSR, 8 lanes per row          9 COO (element-parallel)
 *
 * and a +-1 segregation flag (Sec. 2.4.2).
 */
#ifndef FFSPMV_SELECT_H
#define FFSPMV_SELECT_H

#include "ffspmv.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FFSPMV_NUM_BINS 17
#define FFSPMV_NUM_FORMATS 10
#define FFSPMV_NUM_FEATURES 16     /* per matrix */
#define FFSPMV_NUM_BIN_FEATURES 6  /* per bin */
#define FFSPMV_MLP_IN (FFSPMV_NUM_FEATURES + FFSPMV_NUM_BIN_FEATURES)
#define FFSPMV_MLP_HIDDEN 64
/* outputs: the formats' predicted log(t_format / t_best) and log(t_pm / t_nopm)
 * for a (matrix, bin) input; for the matrix-level input (the bin features all
 * FFSPMV_MATRIX_INPUT) the predicted whole-plan log(t / t_binned) of the
 * binned layout with the network's table and of the x-panel layout with
 * clusters of 1, 2 and 4 CTAs, t_binned being the binned layout with the
 * heuristic table */
#define FFSPMV_MLP_OUT (FFSPMV_NUM_FORMATS + 5)
#define FFSPMV_OUT_PM FFSPMV_NUM_FORMATS
#define FFSPMV_OUT_NETBINS (FFSPMV_NUM_FORMATS + 1)
#define FFSPMV_OUT_PANEL (FFSPMV_NUM_FORMATS + 2) /* q = 1; q = 2 and 4 follow */
#define FFSPMV_MATRIX_INPUT (-1.0f) /* value of every bin feature of the matrix-level input */
/* flat parameter vector: W1[H][IN] b1[H] W2[H][H] b2[H] W3[OUT][H] b3[OUT] */
#define FFSPMV_MLP_PARAMS                                                  \
    (FFSPMV_MLP_HIDDEN * FFSPMV_MLP_IN + FFSPMV_MLP_HIDDEN +                \
     FFSPMV_MLP_HIDDEN * FFSPMV_MLP_HIDDEN + FFSPMV_MLP_HIDDEN +            \
     FFSPMV_MLP_OUT * FFSPMV_MLP_HIDDEN + FFSPMV_MLP_OUT)

/*
 * Matrix and bin features, computed on the device from a CSR matrix whose
 * arrays are device memory (row_ptr int64[nrows+1], col int32[nnz], values
 * uint32[nnz], reduced mod m or not).  d_feat: float[16] receives the matrix
 * features, d_binfeat: float[17][6] the per-bin features (their
 * definitions are listed beside k_features_final in csrc/select.cu).
 * Allocates and frees its own scratch; synchronous.
 */
ffspmv_status ffspmv_matrix_features(int64_t nrows, int64_t ncols, const int64_t *d_row_ptr,
                                     const int32_t *d_col, const uint32_t *d_values,
                                     uint32_t modulus, float *d_feat, float *d_binfeat,
                                     ffspmv_stream_t stream);

/*
 * The exhaustive search.  For every non-empty bin, every valid format (and
 * the +-1 flag on the best one) is built over a sample of the bin's rows (at
 * most max_rows rows and about max_nnz entries, evenly spaced) and timed on
 * the device with CUDA events (`reps` timed calls after 2 warm-up calls).
 * Host or device CSR input as for spmv_create_hybrid.  Host outputs:
 * times[17][10]: milliseconds per call per format (NaN: empty bin or invalid
 * format); pm_times[17][2]: the best format without / with +-1 segregation
 * (NaN when the bin has no +-1 entry); sample_nnz[17]: entries in each
 * bin's sample; best[17][3]: (format, +-1 flag, valid) of the argmin.
 */
ffspmv_status ffspmv_tune_bins(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *row_ptr,
                               const int32_t *col, const uint32_t *values, uint32_t modulus,
                               int32_t max_rows, int64_t max_nnz, int32_t reps, float *times,
                               float *pm_times, int64_t *sample_nnz, int32_t *best);

/* Selector network kernels (fp32), on device arrays.  params: float[PARAMS];
 * in: float[batch][IN]; act: float[batch][2*HIDDEN] (post-ReLU activations
 * kept for the backward pass, may be NULL in forward-only use); out:
 * float[batch][OUT]. */
ffspmv_status ffspmv_mlp_forward(const float *d_params, const float *d_in, int32_t batch,
                                 float *d_act, float *d_out, ffspmv_stream_t stream);

/* Masked squared error L = sum(mask*(out-target)^2) / max(1, sum(mask)) and
 * its gradient d_dout = dL/dout; d_loss: float[1]. */
ffspmv_status ffspmv_mlp_loss(const float *d_out, const float *d_target, const float *d_mask,
                              int32_t batch, float *d_dout, float *d_loss,
                              ffspmv_stream_t stream);

/* Gradient of the loss with respect to the parameters (d_grad: float[PARAMS],
 * overwritten), given the forward pass's act and dL/dout. */
ffspmv_status ffspmv_mlp_backward(const float *d_params, const float *d_in, int32_t batch,
                                  const float *d_act, const float *d_dout, float *d_grad,
                                  ffspmv_stream_t stream);

/* One Adam step (Kingma and Ba, 2015) on params, with moment buffers m, v
 * (float[PARAMS], zero at step 1); step counts from 1. */
ffspmv_status ffspmv_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v,
                              int32_t step, float lr, float beta1, float beta2, float eps,
                              ffspmv_stream_t stream);

/* Install the selector weights (host floats, PARAMS of them, copied) used by
 * FFSPMV_SEL_LEARNED; NULL uninstalls them (LEARNED then falls back to the
 * exhaustive search). */
ffspmv_status ffspmv_selector_load(const float *params, int64_t count);

/* The selector's choice for a matrix (host or device CSR): best[17][3] as in
 * ffspmv_tune_bins, from the network's inference kernel on the device, and
 * (layout != NULL) the whole-plan choice of least predicted time:
 * FFSPMV_LAYOUT_BINNED (the binned layout with the heuristic table),
 * FFSPMV_LAYOUT_NETBINS (the binned layout with best[][]) or
 * FFSPMV_LAYOUT_PANEL_Q1/Q2/Q4 (the x-panel layout with clusters of 1, 2 or
 * 4 CTAs) or FFSPMV_LAYOUT_PANEL (x-panel, the builder's cluster size).  A
 * cluster size is named only when its predicted time beats the other two by
 * FFSPMV_SEL_Q_MARGIN (log ratio), and the network's own table only when it
 * beats the heuristic table by FFSPMV_SEL_NET_MARGIN: that output is learned
 * from the exhaustive search's table, which the network's table only
 * approaches.  This is what FFSPMV_SEL_LEARNED builds under FFSPMV_FMT_AUTO
 * (with the timed check of FFSPMV_SEL_VERIFY_MARGIN). */
enum {
    FFSPMV_LAYOUT_BINNED = 0,
    FFSPMV_LAYOUT_NETBINS = 1,
    FFSPMV_LAYOUT_PANEL_Q1 = 2,
    FFSPMV_LAYOUT_PANEL_Q2 = 3,
    FFSPMV_LAYOUT_PANEL_Q4 = 4,
    FFSPMV_LAYOUT_PANEL = 5
};
#define FFSPMV_SEL_Q_MARGIN 0.05f
#define FFSPMV_SEL_NET_MARGIN 0.15f
/* FFSPMV_SEL_LEARNED builds and times the best x-panel and the best binned
 * layout when their predicted times are this close (log ratio), and keeps
 * the faster */
#define FFSPMV_SEL_VERIFY_MARGIN 0.15f
ffspmv_status ffspmv_selector_choose(int64_t nrows, int64_t ncols, int64_t nnz,
                                     const int64_t *row_ptr, const int32_t *col,
                                     const uint32_t *values, uint32_t modulus, int32_t *best,
                                     int32_t *layout);

/* The heuristic table's choice (host CSR: row_ptr, values), best[17][3] as
 * in ffspmv_tune_bins; use_pm1 as in ffspmv_options. */
ffspmv_status ffspmv_heuristic_choose(int64_t nrows, const int64_t *row_ptr, const uint32_t *values,
                                      uint32_t modulus, int32_t use_pm1, int32_t *best);

/* Build a binned plan with the given per-bin choice (best[17][3] as above;
 * entries with valid = 0 fall back to the heuristic table). */
ffspmv_status spmv_create_binned(ffspmv_t *out, int64_t nrows, int64_t ncols, int64_t nnz,
                                 const int64_t *row_ptr, const int32_t *col,
                                 const uint32_t *values, uint32_t modulus,
                                 const int32_t *best, const ffspmv_options *opt,
                                 ffspmv_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* FFSPMV_SELECT_H */
