/*
 * Sigma-bases (minimal approximant bases) over F_p: the second step of block
 * Wiedemann (Sec. 3.2, "Parallelization of the sigma-basis computation"), which
 * turns the matrix sequence S_i = X^T A^i Y into a minimal matrix generator.
 * The algorithm is PM-Basis of Giorgi, Jeannerod and Villard (ISSAC 2003):
 * divide and conquer on the order, reduced to polynomial-matrix products
 * (polymat_mul, the evaluation / pointwise product / interpolation scheme of
 * Sec. 3.2.1), with their iterative M-Basis at small orders, as Sec. 3.2.2
 * recommends.
 *
 * Definitions.  F in F_p[x]^{m x n}, an order d >= 1 and a shift s in Z^m.
 * An order-d sigma-basis of F is an m x m polynomial matrix P whose rows
 * generate every approximant v (a row vector with v F = 0 mod x^d) and have
 * minimal s-shifted degrees; delta_i = s_i + the number of times row i was
 * multiplied by x, and deg P_ij <= delta_i - s_j.  For block Wiedemann,
 * F = [S(x); -I_s] (m = 2s, n = s, zero shift); the s rows of P with the smallest
 * delta (first s columns) give the minimal generator, and deg det - codeg det
 * of that generator (Sec. 3.3) is the rank of a suitably preconditioned A.
 *
 * Layout: polynomial matrices are coefficient-major and row-major inside a
 * coefficient, uint32 residues: F[k][i][j] is the coefficient of x^k in entry
 * (i, j).  The result is the same matrix, bit for bit, as the plain
 * statement of the two algorithms gives: at each order of M-Basis the rows
 * are ordered by (delta_i, i), each column of the order-k residual is
 * eliminated with the first row in that order (not yet a pivot) that is
 * nonzero in it, multiples of the pivot are added only to later non-pivot
 * rows, and the pivot rows are multiplied by x; PM-Basis splits the order as
 * d1 = ceil(d / 2), d - d1 and returns P2 P1.
 */
#ifndef FFSPMV_SIGMA_H
#define FFSPMV_SIGMA_H

#include "ffspmv.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Device workspace (bytes, written to *bytes) that sigma_basis needs for
 * these sizes.  1 <= n <= m <= 32, d >= 1; base = 0 picks the default leaf
 * order (the largest power of two <= 32 whose M-Basis leaf fits in one CTA's
 * shared memory), else 1 <= base <= 32.  FFSPMV_ERR_UNSUPPORTED when the
 * leaf does not fit in shared memory, or the largest product of the
 * recursion (ceil(d/2) + d coefficients) exceeds the 2^15-point transforms
 * of polymat_mul.
 */
ffspmv_status sigma_basis_workspace(int32_t m, int32_t n, int64_t d, int32_t base, int64_t *bytes);

/*
 * Order-d sigma-basis of d_F (device, d x m x n residues; reduced mod p on
 * load) for the shift h_shift (host, m values with |s_i| <= 2^24; NULL =
 * all zero).  p must be a prime, 2 <= p <= 2^31 (FFSPMV_ERR_ARG otherwise).
 * Outputs: d_P (device, (d+1) x m x m, zero above the degree), h_delta
 * (host, m shifted degrees), *h_degree (host, optional): an upper bound on
 * deg P, min(d, max_i delta_i - min_j s_j).  base: as for
 * sigma_basis_workspace (PM-Basis hands orders <= base to M-Basis).  d_work:
 * at least sigma_basis_workspace bytes of device memory, 16-byte aligned,
 * owned by the caller and not used by another call at the same time.
 * Synchronous: the recursion reads each leaf's degrees back to size the next
 * products, so the call returns after the stream has finished the work.
 */
ffspmv_status sigma_basis(uint32_t p, int32_t m, int32_t n, int64_t d, int32_t base,
                          const uint32_t *d_F, const int32_t *h_shift, uint32_t *d_P,
                          int32_t *h_delta, int64_t *h_degree, void *d_work, int64_t work_bytes,
                          ffspmv_stream_t stream);

/*
 * The block-Wiedemann input of sigma_basis: d_F (device, L x 2s x s) =
 * [S(x); -I_s], i.e. F[k][i][j] = S[k][i][j] for i < s, F[0][s+j][j] = p-1,
 * every other entry 0; d_S (device, L x s x s, as spmv_block_sequence writes
 * it).  1 <= s <= 16, L >= 1, 2 <= p <= 2^31.  Stream-ordered, asynchronous.
 */
ffspmv_status sigma_wiedemann_input(uint32_t p, int32_t s, int64_t L, const uint32_t *d_S, uint32_t *d_F,
                                    ffspmv_stream_t stream);

/*
 * deg det U and codeg det U (the multiplicity of x in det U) of the
 * generator of a sigma-basis: U = the n rows of d_P with the least
 * (h_delta_i, i), columns 0..n-1, an n x n polynomial matrix.  For the
 * block-Wiedemann input [S(x); -I_s] (n = s), deg det U - codeg det U is the
 * rank of a suitably preconditioned A (Sec. 3, step 3; Sec. 3.3, determinant
 * co-degree).  d_P: device, (d+1) x m x m as sigma_basis writes it; h_delta:
 * host, the m degrees sigma_basis returns (only their order is used).  p a
 * prime, 2 <= p <= 2^31; 1 <= n <= m <= 32; d >= 0.  Both values are x-adic
 * valuations of determinants (codeg det U = v(det U); deg det U = sum_r D_r -
 * v(det U~), D_r the degree of row r of U and U~ its rows reversed against
 * D_r), each read off Gaussian elimination over F_p[[x]] truncated at x^K
 * with pivots of least valuation, on the device; K starts at 32 and doubles
 * until every pivot is found below the precision, up to max_precision (0 =
 * 4096; at most 65536).  Returns FFSPMV_ERR_UNSUPPORTED when det U = 0 (a
 * zero row, or no pivot below max_precision).  Allocates its working memory
 * (n^2 K words) on the current device, where d_P must live (FFSPMV_ERR_OOM
 * when that fails), and is synchronous (it reads each column's pivot
 * valuations back); results in *h_deg, *h_codeg (host).
 */
ffspmv_status sigma_generator_degrees(uint32_t p, int32_t m, int32_t n, int64_t d, const uint32_t *d_P,
                                      const int32_t *h_delta, int32_t max_precision, int64_t *h_deg,
                                      int64_t *h_codeg, ffspmv_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* FFSPMV_SIGMA_H */
