/*
 * Products of polynomial matrices over Z/pZ: the multiplication that the
 * sigma-basis / PM-Basis step of block Wiedemann is built from, computed by
 * the evaluation / pointwise product / interpolation scheme of Sec. 3
 * (parallel polynomial matrix multiplication).
 * C(x) = A(x) B(x) for s x s matrices whose entries are polynomials over
 * F_p.  Arrays are coefficient-major and row-major inside a coefficient:
 * A[k][i][j] (uint32, < p) is the coefficient of x^k in entry (i, j);
 * A: (da+1) x s x s, B: (db+1) x s x s, C: (da+db+1) x s x s.
 */
#ifndef FFSPMV_POLYMAT_H
#define FFSPMV_POLYMAT_H

#include "ffspmv.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Device workspace that polymat_mul needs for these sizes (bytes, written
 * to *bytes).  1 <= s <= 32, da, db >= 0; FFSPMV_ERR_UNSUPPORTED when
 * da + db + 1 > 2^15 (the transform length is limited by shared memory).
 */
ffspmv_status polymat_mul_workspace(int32_t s, int64_t da, int64_t db, int64_t *bytes);

/*
 * d_C = d_A * d_B mod p (device arrays as above; d_C must not overlap the
 * inputs).  2 <= p <= 2^31; inputs must be below p.  The exact integer
 * coefficients are computed modulo three primes by number-theoretic
 * transforms and recombined by the Chinese remainder theorem, which needs
 * s * (min(da, db) + 1) * (p - 1)^2 < 998244353 * 167772161 * 469762049
 * (about 2^86), else FFSPMV_ERR_UNSUPPORTED.  d_work: device memory of at
 * least polymat_mul_workspace bytes, 16-byte aligned, owned by the caller
 * and not used by another call at the same time.  Stream-ordered and
 * asynchronous.
 */
ffspmv_status polymat_mul(uint32_t p, int32_t s, int64_t da, int64_t db, const uint32_t *d_A,
                          const uint32_t *d_B, uint32_t *d_C, void *d_work, int64_t work_bytes,
                          ffspmv_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* FFSPMV_POLYMAT_H */
