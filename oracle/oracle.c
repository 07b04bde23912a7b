/*
 * CPU oracle for exact sparse products over Z/mZ.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header, table or helper with the CUDA path.
 *
 * Every function is the plain definition, written out: each sum is formed
 * exactly in an unsigned 128-bit integer and reduced once with `%`.  A
 * residue is below 2^32 and a product of two below 2^64, so a sum of fewer
 * than 2^64 products cannot overflow; results are the unique representatives
 * in [0, m).  Nothing is blocked, fused or reordered.
 *
 * Layouts: CSR (Sec. 2.1): row i holds entries row_ptr[i] <= k < row_ptr[i+1]
 * with A[i, col[k]] = val[k]; repeated (i, j) pairs add up.  A block of nvec
 * vectors is row-major with leading dimension ld: element (k, v) is
 * X[k*ld + v].
 *
 * Return value: 0 on success, -1 on a bad argument, -2 when out of memory.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static int bad_common(int64_t nrows, const int64_t *row_ptr, uint32_t m,
                      int64_t ldx, int64_t ldy, int32_t nvec)
{
    return nrows < 0 || row_ptr == 0 || m < 2 || nvec < 1 || ldx < nvec ||
           ldy < nvec;
}

/*
 * y <- alpha*A*x + beta*y  (mod m), block form Y <- alpha*A*X + beta*Y.
 * Sec. 2: the product y <- Ax + y, the general alpha/beta form, the apply
 * operation (beta = 0) and the multi-vector version of the same operation.
 * x: ncols x nvec (ldx), y: nrows x nvec (ldy).
 */
int oracle_spmv(int64_t nrows, int64_t ncols, const int64_t *row_ptr,
                const int32_t *col, const uint32_t *val, uint32_t m,
                const uint32_t *x, int64_t ldx, uint32_t *y, int64_t ldy,
                int32_t nvec, uint32_t alpha, uint32_t beta)
{
    if (bad_common(nrows, row_ptr, m, ldx, ldy, nvec) || ncols < 0)
        return -1;
    for (int64_t i = 0; i < nrows; ++i) {
        for (int32_t v = 0; v < nvec; ++v) {
            u128 acc = 0;
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int64_t j = col[k];
                if (j < 0 || j >= ncols)
                    return -1;
                acc += (u128)val[k] * (u128)x[j * ldx + v];
            }
            u128 r = (u128)alpha * (acc % m) + (u128)beta * y[i * ldy + v];
            y[i * ldy + v] = (uint32_t)(r % m);
        }
    }
    return 0;
}

/*
 * y <- alpha*A^T*x + beta*y  (mod m): the transpose product the library
 * provides next to A*x (Sec. 1).  x: nrows x nvec (ldx), y: ncols x nvec.
 */
int oracle_spmv_transpose(int64_t nrows, int64_t ncols, const int64_t *row_ptr,
                          const int32_t *col, const uint32_t *val, uint32_t m,
                          const uint32_t *x, int64_t ldx, uint32_t *y,
                          int64_t ldy, int32_t nvec, uint32_t alpha,
                          uint32_t beta)
{
    if (bad_common(nrows, row_ptr, m, ldx, ldy, nvec) || ncols < 0)
        return -1;
    u128 *acc = (u128 *)calloc((size_t)(ncols > 0 ? ncols : 1) * nvec,
                               sizeof(u128));
    if (!acc)
        return -2;
    for (int64_t i = 0; i < nrows; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            if (j < 0 || j >= ncols) {
                free(acc);
                return -1;
            }
            for (int32_t v = 0; v < nvec; ++v)
                acc[j * nvec + v] += (u128)val[k] * (u128)x[i * ldx + v];
        }
    }
    for (int64_t j = 0; j < ncols; ++j) {
        for (int32_t v = 0; v < nvec; ++v) {
            u128 r = (u128)alpha * (acc[j * nvec + v] % m) +
                     (u128)beta * y[j * ldy + v];
            y[j * ldy + v] = (uint32_t)(r % m);
        }
    }
    free(acc);
    return 0;
}

/*
 * S_i = X^T * V_i (mod p), one s x s block:  S[a*s + b] = sum_k X[k][a]*V[k][b].
 * X and V: n x s, row-major (leading dimension s).
 */
static void project(int64_t n, uint32_t p, const uint32_t *X,
                    const uint32_t *V, int32_t s, uint32_t *S)
{
    for (int32_t a = 0; a < s; ++a) {
        for (int32_t b = 0; b < s; ++b) {
            u128 acc = 0;
            for (int64_t k = 0; k < n; ++k)
                acc += (u128)X[k * s + a] * (u128)V[k * s + b];
            S[a * s + b] = (uint32_t)(acc % p);
        }
    }
}

/*
 * The matrix sequence of block Wiedemann's first step (Sec. 3, step 1, with
 * independent left and right blocks): V_0 = Y, V_{i+1} = A*V_i (mod p), and
 * S_i = X^T * V_i (mod p) for 0 <= i < nsteps.  S is nsteps x s x s,
 * S[(i*s + a)*s + b].  If V_next is not NULL it receives V_nsteps = A^nsteps*Y,
 * the state a later call continues from.  A must be square (n x n).
 */
int oracle_block_sequence(int64_t n, const int64_t *row_ptr, const int32_t *col,
                          const uint32_t *val, uint32_t p, const uint32_t *X,
                          const uint32_t *Y, int32_t s, int64_t nsteps,
                          uint32_t *S, uint32_t *V_next)
{
    if (n < 0 || row_ptr == 0 || p < 2 || s < 1 || nsteps < 0)
        return -1;
    size_t sz = (size_t)(n > 0 ? n : 1) * (size_t)s;
    uint32_t *V = (uint32_t *)malloc(sz * sizeof(uint32_t));
    uint32_t *W = (uint32_t *)malloc(sz * sizeof(uint32_t));
    if (!V || !W) {
        free(V);
        free(W);
        return -2;
    }
    memcpy(V, Y, (size_t)n * s * sizeof(uint32_t));
    int rc = 0;
    for (int64_t i = 0; i < nsteps && rc == 0; ++i) {
        project(n, p, X, V, s, S + (size_t)i * s * s);
        if (i + 1 < nsteps || V_next) {
            rc = oracle_spmv(n, n, row_ptr, col, val, p, V, s, W, s, s, 1, 0);
            uint32_t *t = V;
            V = W;
            W = t;
        }
    }
    if (rc == 0 && V_next) {
        if (nsteps == 0)
            memcpy(V_next, Y, (size_t)n * s * sizeof(uint32_t));
        else
            memcpy(V_next, V, (size_t)n * s * sizeof(uint32_t));
    }
    free(V);
    free(W);
    return rc;
}

/*
 * The same two products on several host threads, for timing the oracle on
 * all cores.  Rows are split into `nthreads` contiguous blocks (a static row
 * partition); each thread evaluates the plain definition above on its
 * block, unchanged.  For A*x the blocks write disjoint rows of y.  For A^T*x
 * each thread forms the definition's sum over its rows only (its own
 * partial column sums, reduced mod m), and the partial sums are then added
 * exactly and combined with alpha and beta once per output.
 */
struct job {
    int64_t r0, r1, ncols;
    const int64_t *row_ptr;
    const int32_t *col;
    const uint32_t *val;
    uint32_t m;
    const uint32_t *x;
    int64_t ldx;
    uint32_t *y;
    int64_t ldy;
    int32_t nvec;
    uint32_t alpha, beta;
    int transpose, rc;
};

static void *run_job(void *arg)
{
    struct job *j = (struct job *)arg;
    if (j->transpose)
        j->rc = oracle_spmv_transpose(j->r1 - j->r0, j->ncols, j->row_ptr + j->r0, j->col,
                                      j->val, j->m, j->x + j->r0 * j->ldx, j->ldx, j->y,
                                      j->ldy, j->nvec, 1, 0);
    else
        j->rc = oracle_spmv(j->r1 - j->r0, j->ncols, j->row_ptr + j->r0, j->col, j->val,
                            j->m, j->x, j->ldx, j->y + j->r0 * j->ldy, j->ldy, j->nvec,
                            j->alpha, j->beta);
    return 0;
}

static int run_threads(int nthreads, int transpose, int64_t nrows, int64_t ncols,
                       const int64_t *row_ptr, const int32_t *col, const uint32_t *val,
                       uint32_t m, const uint32_t *x, int64_t ldx, uint32_t *y, int64_t ldy,
                       int32_t nvec, uint32_t alpha, uint32_t beta)
{
    if (bad_common(nrows, row_ptr, m, ldx, ldy, nvec) || ncols < 0 || nthreads < 1)
        return -1;
    if (nthreads > 256)
        nthreads = 256;
    struct job jobs[256];
    pthread_t tid[256];
    uint32_t *part = 0;
    if (transpose) {
        part = (uint32_t *)calloc((size_t)nthreads * (size_t)(ncols > 0 ? ncols : 1) * nvec,
                                  sizeof(uint32_t));
        if (!part)
            return -2;
    }
    for (int t = 0; t < nthreads; ++t) {
        struct job *j = &jobs[t];
        j->r0 = nrows * t / nthreads;
        j->r1 = nrows * (t + 1) / nthreads;
        j->ncols = ncols;
        j->row_ptr = row_ptr;
        j->col = col;
        j->val = val;
        j->m = m;
        j->x = x;
        j->ldx = ldx;
        j->y = transpose ? part + (size_t)t * (size_t)ncols * nvec : y;
        j->ldy = transpose ? nvec : ldy;
        j->nvec = nvec;
        j->alpha = alpha;
        j->beta = beta;
        j->transpose = transpose;
        j->rc = 0;
    }
    int started = 0;
    for (; started < nthreads; ++started)
        if (pthread_create(&tid[started], 0, run_job, &jobs[started]) != 0)
            break;
    for (int t = started; t < nthreads; ++t)
        run_job(&jobs[t]);  /* threads that could not start run here */
    for (int t = 0; t < started; ++t)
        pthread_join(tid[t], 0);
    int rc = 0;
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].rc != 0)
            rc = jobs[t].rc;
    if (transpose && rc == 0) {
        for (int64_t jj = 0; jj < ncols; ++jj) {
            for (int32_t v = 0; v < nvec; ++v) {
                u128 acc = 0;
                for (int t = 0; t < nthreads; ++t)
                    acc += part[((size_t)t * ncols + jj) * nvec + v];
                u128 r = (u128)alpha * (acc % m) + (u128)beta * y[jj * ldy + v];
                y[jj * ldy + v] = (uint32_t)(r % m);
            }
        }
    }
    free(part);
    return rc;
}

int oracle_spmv_threads(int32_t nthreads, int64_t nrows, int64_t ncols,
                        const int64_t *row_ptr, const int32_t *col, const uint32_t *val,
                        uint32_t m, const uint32_t *x, int64_t ldx, uint32_t *y,
                        int64_t ldy, int32_t nvec, uint32_t alpha, uint32_t beta)
{
    return run_threads(nthreads, 0, nrows, ncols, row_ptr, col, val, m, x, ldx, y, ldy,
                       nvec, alpha, beta);
}

int oracle_spmv_transpose_threads(int32_t nthreads, int64_t nrows, int64_t ncols,
                                  const int64_t *row_ptr, const int32_t *col,
                                  const uint32_t *val, uint32_t m, const uint32_t *x,
                                  int64_t ldx, uint32_t *y, int64_t ldy, int32_t nvec,
                                  uint32_t alpha, uint32_t beta)
{
    return run_threads(nthreads, 1, nrows, ncols, row_ptr, col, val, m, x, ldx, y, ldy,
                       nvec, alpha, beta);
}
