/*
 * Test infrastructure only: a plain, slow, single-threaded FP64 statement of
 * the block-sparse x dense product of Section 3 (the unnumbered equation
 * Y = (M (.) W) * X with M_ij = Mhat_{floor(i/b), floor(j/b)}).
 *
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no code, header or constant with the CUDA path.
 *
 * The sparse operand is given exactly as a user supplies it: nnzb blocks, block
 * p sitting at block coordinates (brow[p], bcol[p]) with its b*b values stored
 * row-major at vals[p*b*b ...].  Because Section 3 sizes the block mask as
 * ceil(m/b) x ceil(k/b), a block that hangs over the bottom or right edge is
 * truncated: entries with row >= m or column >= k are simply not part of W.
 *
 * Y[i, j] = sum over blocks p with brow[p] == floor(i/b)
 *              sum over l < b with bcol[p]*b + l < k
 *                  vals[p][i - brow[p]*b][l] * X[bcol[p]*b + l, j]
 * Rows of Y not covered by any block are zero (M is zero there).
 */
#include <stdint.h>
#include <string.h>

/* Returns 0 on success, 1 if a block coordinate lies outside the
 * ceil(m/b) x ceil(k/b) block grid (the caller's pattern is then not a block
 * mask of this shape), 2 on bad sizes. */
int oracle_spmm_f64(int64_t m, int64_t k, int64_t n, int64_t b, int64_t nnzb,
                    const int32_t *brow, const int32_t *bcol,
                    const double *vals, const double *X, int64_t ldx,
                    double *Y, int64_t ldy)
{
    if (m < 0 || k < 0 || n < 0 || b <= 0 || nnzb < 0 || ldx < n || ldy < n)
        return 2;
    const int64_t mb = (m + b - 1) / b;
    const int64_t kb = (k + b - 1) / b;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j)
            Y[i * ldy + j] = 0.0;
    for (int64_t p = 0; p < nnzb; ++p) {
        const int64_t r = brow[p], c = bcol[p];
        if (r < 0 || r >= mb || c < 0 || c >= kb)
            return 1;
        const double *blk = vals + p * b * b;
        for (int64_t ii = 0; ii < b; ++ii) {
            const int64_t i = r * b + ii;
            if (i >= m)
                break;
            for (int64_t l = 0; l < b; ++l) {
                const int64_t kk = c * b + l;
                if (kk >= k)
                    break;
                const double w = blk[ii * b + l];
#ifdef ORACLE_MUTANT_TRANSPOSE
                /* planted mistake (mutation tests only): block read transposed */
                const double w_used = blk[l * b + ii];
#elif defined(ORACLE_MUTANT_SIGN)
                /* planted mistake: last block of the list enters with a flipped sign */
                const double w_used = (p == nnzb - 1) ? -w : w;
#else
                const double w_used = w;
#endif
                for (int64_t j = 0; j < n; ++j) {
#ifdef ORACLE_MUTANT_COLSHIFT
                    /* planted mistake: X row index off by one inside a block */
                    const int64_t kx = (l + 1 < b && kk + 1 < k) ? kk + 1 : kk;
                    Y[i * ldy + j] += w_used * X[kx * ldx + j];
#else
                    Y[i * ldy + j] += w_used * X[kk * ldx + j];
#endif
                }
            }
        }
    }
#ifdef ORACLE_MUTANT_DROP_LAST
    /* planted mistake: the last block-row of Y is never written */
    if (m > 0)
        for (int64_t j = 0; j < n; ++j)
            Y[(m - 1) * ldy + j] = 0.0;
#endif
    return 0;
}

/* Decodes FP8 E4M3 ("fn" variant: 1 sign bit, 4 exponent bits with bias 7,
 * 3 mantissa bits, no infinities, S.1111.111 is NaN) into FP64, written from
 * the format's definition: normal numbers (-1)^s * 2^(e-7) * (1 + f/8),
 * subnormals (e == 0) (-1)^s * 2^(-6) * (f/8).  Returns the NaN count. */
int64_t oracle_e4m3_to_f64(const uint8_t *in, int64_t count, double *out)
{
    int64_t nans = 0;
    for (int64_t i = 0; i < count; ++i) {
        const unsigned v = in[i];
        const int s = (v >> 7) & 1;
        const int e = (v >> 3) & 0xF;
        const int f = v & 7;
        double mag;
        if (e == 0xF && f == 7) {
            ++nans;
            mag = 0.0 / 0.0;
        } else if (e == 0) {
            mag = (double)f / 8.0;
            for (int t = 0; t < 6; ++t)
                mag *= 0.5;
        } else {
            mag = 1.0 + (double)f / 8.0;
            int ex = e - 7;
            while (ex > 0) { mag *= 2.0; --ex; }
            while (ex < 0) { mag *= 0.5; ++ex; }
        }
        out[i] = s ? -mag : mag;
    }
    return nans;
}/*
 * The transposed product Z = W^T * Y (the step beside the path in sparse
 * training, Section 1: the same block mask applied to the other operand),
 * written out from its definition over the same user-order blocks:
 *
 * Z[c*b + l, j] = sum over blocks p with bcol[p] == c
 *                    sum over ii < b with brow[p]*b + ii < m
 *                        vals[p][ii][l] * Y[brow[p]*b + ii, j]
 *
 * W is m x k, Y is m x n (ldy), Z is k x n (ldz).  Same return codes as
 * oracle_spmm_f64.
 */
int oracle_spmm_t_f64(int64_t m, int64_t k, int64_t n, int64_t b, int64_t nnzb,
                      const int32_t *brow, const int32_t *bcol, const double *vals,
                      const double *Y, int64_t ldy, double *Z, int64_t ldz)
{
    if (m < 0 || k < 0 || n < 0 || b <= 0 || nnzb < 0 || ldy < n || ldz < n)
        return 2;
    const int64_t mb = (m + b - 1) / b;
    const int64_t kb = (k + b - 1) / b;
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < n; ++j)
            Z[i * ldz + j] = 0.0;
    for (int64_t p = 0; p < nnzb; ++p) {
        const int64_t r = brow[p], c = bcol[p];
        if (r < 0 || r >= mb || c < 0 || c >= kb)
            return 1;
        const double *blk = vals + p * b * b;
        for (int64_t l = 0; l < b; ++l) {
            const int64_t zr = c * b + l;
            if (zr >= k)
                break;
            for (int64_t ii = 0; ii < b; ++ii) {
                const int64_t yr = r * b + ii;
                if (yr >= m)
                    break;
                const double w = blk[ii * b + l];
                for (int64_t j = 0; j < n; ++j)
                    Z[zr * ldz + j] += w * Y[yr * ldy + j];
            }
        }
    }
    return 0;
}

/*
 * The sampled dense-dense product on the block mask (SDDMM): the gradient
 * of Section 3's product with respect to W's stored blocks, as used by the
 * sparse training regimes of Section 1.  For L = sum_ij dY[i,j] * Y[i,j]
 * with Y = (M (.) W) * X, dL/dW[i,l] = M[i,l] * sum_j dY[i,j] * X[l,j], so
 * for every stored block p, written out from that definition:
 *
 * dW[p][ii][l] = sum over j < n of dY[brow[p]*b + ii, j] * X[bcol[p]*b + l, j]
 *
 * for brow[p]*b + ii < m and bcol[p]*b + l < k; entries of a truncated edge
 * block outside the m x k matrix are not part of W and are set to 0.
 * dY is m x n (lddy), X is k x n (ldx); dW holds nnzb blocks of b*b values,
 * row-major, in the order of the pattern.  Same return codes as
 * oracle_spmm_f64.
 */
int oracle_sddmm_f64(int64_t m, int64_t k, int64_t n, int64_t b, int64_t nnzb,
                     const int32_t *brow, const int32_t *bcol,
                     const double *dY, int64_t lddy, const double *X, int64_t ldx,
                     double *dW)
{
    if (m < 0 || k < 0 || n < 0 || b <= 0 || nnzb < 0 || lddy < n || ldx < n)
        return 2;
    const int64_t mb = (m + b - 1) / b;
    const int64_t kb = (k + b - 1) / b;
    for (int64_t p = 0; p < nnzb; ++p) {
        const int64_t r = brow[p], c = bcol[p];
        if (r < 0 || r >= mb || c < 0 || c >= kb)
            return 1;
        double *blk = dW + p * b * b;
        for (int64_t ii = 0; ii < b; ++ii) {
            for (int64_t l = 0; l < b; ++l) {
                const int64_t yr = r * b + ii, xr = c * b + l;
                double acc = 0.0;
#ifdef ORACLE_MUTANT_SDDMM_DROP_TERM
                const int64_t nj = n - 1;       /* planted: the last term is lost */
#else
                const int64_t nj = n;
#endif
                if (yr < m && xr < k)
                    for (int64_t j = 0; j < nj; ++j)
                        acc += dY[yr * lddy + j] * X[xr * ldx + j];
#ifdef ORACLE_MUTANT_SDDMM_TRANSPOSE
                blk[l * b + ii] = acc;          /* planted: block stored transposed */
#else
                blk[ii * b + l] = acc;
#endif
            }
        }
    }
    return 0;
}


