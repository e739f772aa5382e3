/*
 * lnv_oracle.c -- plain, slow FP64 reference for the range-truncated
 * block-sparse LNV path.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg call it; the CUDA library never does,
 * and the two share no code.
 *
 * Every routine is the literal definition it cites, written as nested loops.
 * Matrices are block-CSR over atoms: row_ptr[n+1] (int64), col[nnzb] (int32,
 * sorted ascending inside each row), values nnzb blocks of nsf*nsf doubles,
 * row-major inside a block.  Build with -ffp-contract=off so that no
 * multiply-add is fused (the distance test must round exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* Minimum-image separation along one axis of an orthorhombic periodic cell.
 * The paper does not state its boundary convention; the cell is periodic and
 * each ordered atom pair contributes at most one block (its nearest image). */
static double min_image(double d, double box)
{
    double t = d / box;
    double r = rint(t);
    double m = box * r;
    return d - m;
}

/* Squared minimum-image distance, summed as ((dx*dx)+(dy*dy))+(dz*dz). */
static double dist2(const double *pi, const double *pj, const double *cell)
{
    double dx = min_image(pj[0] - pi[0], cell[0]);
    double dy = min_image(pj[1] - pi[1], cell[1]);
    double dz = min_image(pj[2] - pi[2], cell[2]);
    double xx = dx * dx;
    double yy = dy * dy;
    double zz = dz * dz;
    double s = xx + yy;
    return s + zz;
}

/* Range pattern (Sec. 2: locality is imposed by a distance criterion, L_ij = 0
 * beyond R_L).  Block (i, j) is kept when d_ij^2 < R^2.  Brute force over all
 * pairs.  Fills row_ptr[0..n] and returns nnzb. */
int64_t oracle_pattern_count(const double *pos, int64_t n, const double *cell, double R,
                             int64_t *row_ptr)
{
    double R2 = R * R;
    row_ptr[0] = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (dist2(pos + 3 * i, pos + 3 * j, cell) < R2) ++c;
        row_ptr[i + 1] = c;
    }
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    return row_ptr[n];
}

void oracle_pattern_fill(const double *pos, int64_t n, const double *cell, double R,
                         const int64_t *row_ptr, int32_t *col)
{
    double R2 = R * R;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = row_ptr[i];
        for (int64_t j = 0; j < n; ++j)
            if (dist2(pos + 3 * i, pos + 3 * j, cell) < R2) col[p++] = (int32_t)j;
    }
}

/* Position of block (row, j) in a CSR matrix, or -1 if it is not stored. */
static int64_t find_block(const int64_t *rp, const int32_t *col, int64_t row, int32_t j)
{
    int64_t lo = rp[row], hi = rp[row + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < rp[row + 1] && col[lo] == j) ? lo : -1;
}

/* Range-truncated product C = mask(A B): for every block (i, j) stored in C's
 * pattern, C_ij = sum_k A_ik B_kj over the k with both blocks stored (the
 * paper's K_ij = L_ik S_kl L_lj products, Sec. 2, operation (i)).  Blocks
 * outside C's pattern are not formed.  With a row list, only those rows of C
 * are written. */
void oracle_mprod(int nsf, int64_t n,
                  const int64_t *a_rp, const int32_t *a_col, const double *a_val,
                  const int64_t *b_rp, const int32_t *b_col, const double *b_val,
                  const int64_t *c_rp, const int32_t *c_col, double *c_val,
                  const int64_t *rows /* NULL: every row */, int64_t nrows)
{
    const int64_t bs = (int64_t)nsf * nsf;
    const int64_t m = rows ? nrows : n;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < m; ++r) {
        const int64_t i = rows ? rows[r] : r;
        for (int64_t p = c_rp[i]; p < c_rp[i + 1]; ++p) {
            int32_t j = c_col[p];
            double *c = c_val + p * bs;
            for (int64_t e = 0; e < bs; ++e) c[e] = 0.0;
            for (int64_t q = a_rp[i]; q < a_rp[i + 1]; ++q) {
                int32_t k = a_col[q];
                int64_t pb = find_block(b_rp, b_col, k, j);
                if (pb < 0) continue;
                const double *a = a_val + q * bs;
                const double *b = b_val + pb * bs;
                for (int x = 0; x < nsf; ++x)
                    for (int y = 0; y < nsf; ++y) {
                        double s = c[x * nsf + y];
                        for (int z = 0; z < nsf; ++z) s += a[x * nsf + z] * b[z * nsf + y];
                        c[x * nsf + y] = s;
                    }
            }
        }
    }
}

/* Tr[A B] = sum_i sum_k sum_{x,z} A_ik[x][z] B_ki[z][x]  (used for
 * N_e = 2 Tr[KS], Sec. 2 condition 2, and E = 2 Tr[KH]).  Summed per row
 * in FP64, then over rows in row order.  With a row list, only those rows
 * are summed (a partial trace). */
double oracle_trace(int nsf, int64_t n,
                    const int64_t *a_rp, const int32_t *a_col, const double *a_val,
                    const int64_t *b_rp, const int32_t *b_col, const double *b_val,
                    double *row_part /* n, may be NULL */,
                    const int64_t *rows /* NULL: every row */, int64_t nrows)
{
    const int64_t bs = (int64_t)nsf * nsf;
    const int64_t m = rows ? nrows : n;
    double total = 0.0;
    for (int64_t r = 0; r < m; ++r) {
        const int64_t i = rows ? rows[r] : r;
        double s = 0.0;
        for (int64_t q = a_rp[i]; q < a_rp[i + 1]; ++q) {
            int32_t k = a_col[q];
            int64_t pb = find_block(b_rp, b_col, k, (int32_t)i);
            if (pb < 0) continue;
            const double *a = a_val + q * bs;
            const double *b = b_val + pb * bs;
            for (int x = 0; x < nsf; ++x)
                for (int z = 0; z < nsf; ++z) s += a[x * nsf + z] * b[z * nsf + x];
        }
        if (row_part) row_part[i] = s;
        total += s;
    }
    return total;
}

/* Restriction of M (on pattern m) to pattern c: out_ij = M_ij where stored,
 * else 0.  Used for mask_{R_L}(.) of an already formed matrix. */
void oracle_restrict(int nsf, int64_t n,
                     const int64_t *m_rp, const int32_t *m_col, const double *m_val,
                     const int64_t *c_rp, const int32_t *c_col, double *c_val)
{
    const int64_t bs = (int64_t)nsf * nsf;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = c_rp[i]; p < c_rp[i + 1]; ++p) {
            int64_t r = find_block(m_rp, m_col, i, c_col[p]);
            if (r < 0) memset(c_val + p * bs, 0, sizeof(double) * (size_t)bs);
            else memcpy(c_val + p * bs, m_val + r * bs, sizeof(double) * (size_t)bs);
        }
}

/* Block transpose on a symmetric pattern: out_ij = (M_ji)^T. */
void oracle_transpose(int nsf, int64_t n, const int64_t *rp, const int32_t *col,
                      const double *m_val, double *out_val)
{
    const int64_t bs = (int64_t)nsf * nsf;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int64_t r = find_block(rp, col, col[p], (int32_t)i);
            double *o = out_val + p * bs;
            if (r < 0) { memset(o, 0, sizeof(double) * (size_t)bs); continue; }
            const double *m = m_val + r * bs;
            for (int x = 0; x < nsf; ++x)
                for (int y = 0; y < nsf; ++y) o[x * nsf + y] = m[y * nsf + x];
        }
}

#ifdef _OPENMP
#include <omp.h>
#endif
/* Host threads the parallel loops above will use. */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
