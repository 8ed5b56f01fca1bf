/*
 * cpu_two_vector.c -- multi-threaded CPU two-vector folding (Section 3.1,
 * Algorithm 1, run on a tiled anti-diagonal wavefront as in Section 4), the
 * host-core baseline that the GPU kernels are reported beside.
 *
 * It is a second, independent implementation of the method: it shares no code
 * with the GPU library or with the CPU oracle, and it is not used to check
 * either of them (tests check it against the oracle).  Only bench.py's CPU
 * legs and tests/ load it.
 *
 * Organisation.  The table is cut into B x B tiles, B a multiple of q, so
 * that every column group g (columns gq .. gq+q-1) lies inside one tile
 * column.  Tiles of one anti-diagonal are independent and are shared among
 * OpenMP threads; a barrier separates diagonals.  Inside a tile, rows go
 * bottom-up and columns left to right, so every term of Eq. 1 a cell reads is
 * final: the cell below-left (pair term), the row to its left and the column
 * below it (splits).  Per cell (i,j):
 *   - the pair term b(S_i,S_j) + D(i+1,j-1);
 *   - the residual splits k in [i+1, j] outside every full group (at most
 *     2(q-1) of them), evaluated directly;
 *   - one lookup per full group g (gq >= i, gq + q <= j), Eq. 3:
 *       D(i,gq) + D(gq+1,j) + R[h(i,g)][c(j,g)],
 *     with h the row's difference vector over D(i, gq..gq+q-1) and c the
 *     column's (positive) difference vector over D(gq+1..gq+q, j);
 *   - after the cell, the row vector (i,g) it completes (column gq+q-1 = j)
 *     and the column vector (j,g) it completes (row gq+1 = i) are stored, with
 *     the values D(i,gq) and D(gq+1,j) beside them, so that the group loop of
 *     later cells reads two contiguous arrays.
 * R[(h << (q-1)) | c] is the largest prefix total of (h_p - c_p), p = 1..k,
 * over k = 0..q-1 (Section 3.1's preprocessing), at most 2^18 bytes (q = 10).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n, q, ng, B;
    const uint8_t *s;
    uint16_t mask;
    int16_t *D;       /* n*n row-major, zero below the diagonal */
    int16_t *A;       /* A[i*ng+g] = D(i, g*q)          (row i, group g) */
    uint32_t *H;      /* H[i*ng+g] = h(i,g) << (q-1)                      */
    int16_t *Bv;      /* Bv[j*ng+g] = D(g*q+1, j)        (column j, group g) */
    uint16_t *C;      /* C[j*ng+g] = c(j,g)                               */
    const uint8_t *R;
    int64_t lookups;
} tv_state;

static void build_r(int q, uint8_t *R) {
    const unsigned nv = 1u << (q - 1);
    for (unsigned h = 0; h < nv; ++h)
        for (unsigned c = 0; c < nv; ++c) {
            int run = 0, best = 0;
            for (int p = 1; p <= q - 1; ++p) {
                run += (int)((h >> (p - 1)) & 1u) - (int)((c >> (p - 1)) & 1u);
                if (run > best) best = run;
            }
            R[(h << (q - 1)) | c] = (uint8_t)best;
        }
}

static inline int pairs_with(uint16_t mask, int x, int y) { return (mask >> (4 * x + y)) & 1; }

/* One tile: rows I*B .. I*B+B-1 (bottom-up), columns J*B .. J*B+B-1. */
static int64_t fill_tile(tv_state *st, int I, int J) {
    const int n = st->n, q = st->q, ng = st->ng;
    int16_t *D = st->D;
    const uint8_t *R = st->R;
    int64_t nl = 0;
    const int r0 = I * st->B, r1 = (r0 + st->B < n ? r0 + st->B : n) - 1;
    const int c0 = J * st->B, c1 = (c0 + st->B < n ? c0 + st->B : n) - 1;
    for (int i = r1; i >= r0; --i) {
        const int16_t *rowi = D + (size_t)i * n;
        const int16_t *Ai = st->A + (size_t)i * ng;
        const uint32_t *Hi = st->H + (size_t)i * ng;
        const int g0 = (i + q - 1) / q;                     /* first group with g*q >= i */
        for (int j = (c0 > i + 1 ? c0 : i + 1); j <= c1; ++j) {
            int best = (i + 1 <= j - 1 ? D[(size_t)(i + 1) * n + j - 1] : 0) + pairs_with(st->mask, st->s[i], st->s[j]);
            const int g1 = j >= q ? (j - q) / q : -1;        /* last group with g*q + q <= j */
            int klo_end, khi_begin;                          /* residual: [i+1, klo_end] and [khi_begin, j] */
            if (g0 <= g1) {
                klo_end = g0 * q;
                khi_begin = g1 * q + q + 1;
                const int16_t *Bj = st->Bv + (size_t)j * ng;
                const uint16_t *Cj = st->C + (size_t)j * ng;
                for (int g = g0; g <= g1; ++g) {
                    const int v = Ai[g] + Bj[g] + R[Hi[g] | Cj[g]];
                    best = v > best ? v : best;
                }
                nl += g1 - g0 + 1;
            } else {
                klo_end = j;
                khi_begin = j + 1;
            }
            for (int k = i + 1; k <= klo_end; ++k) {
                const int v = rowi[k - 1] + D[(size_t)k * n + j];
                best = v > best ? v : best;
            }
            for (int k = khi_begin; k <= j; ++k) {
                const int v = rowi[k - 1] + D[(size_t)k * n + j];
                best = v > best ? v : best;
            }
            D[(size_t)i * n + j] = (int16_t)best;
            /* the row vector (i, g) is complete once column g*q+q-1 = j is known */
            if ((j + 1) % q == 0) {
                const int g = (j + 1) / q - 1;
                if (g * q >= i) {
                    unsigned h = 0;
                    for (int p = 1; p <= q - 1; ++p)
                        h |= (unsigned)(rowi[g * q + p] - rowi[g * q + p - 1]) << (p - 1);
                    st->A[(size_t)i * ng + g] = rowi[g * q];
                    st->H[(size_t)i * ng + g] = h << (q - 1);
                }
            }
            /* the column vector (j, g) is complete once row g*q+1 = i is known */
            if (i >= 1 && (i - 1) % q == 0) {
                const int g = (i - 1) / q;
                if (g * q + q <= j) {
                    unsigned c = 0;
                    for (int p = 1; p <= q - 1; ++p)
                        c |= (unsigned)(D[(size_t)(g * q + p) * n + j] - D[(size_t)(g * q + p + 1) * n + j]) << (p - 1);
                    st->Bv[(size_t)j * ng + g] = D[(size_t)(g * q + 1) * n + j];
                    st->C[(size_t)j * ng + g] = (uint16_t)c;
                }
            }
        }
    }
    return nl;
}

/* Folds codes[0..n) (A=0, C=1, G=2, U=3) with vector length q in [2, 10] on
 * `threads` OpenMP threads (<= 0: all).  Returns D(0, n-1) (0 for n <= 1), or
 * -1 for bad arguments and -2 when memory runs out.  If D_out is not NULL it
 * receives the n*n int16 table (row-major, zero below the diagonal).  If
 * lookups is not NULL it receives the number of table lookups made; if
 * threads_used is not NULL, the number of threads that ran. */
int cpu_two_vector(const uint8_t *codes, int n, int q, uint16_t mask, int threads, int16_t *D_out,
                   int64_t *lookups, int *threads_used) {
    if (n < 0 || n > 65535 || q < 2 || q > 10 || (n > 0 && !codes)) return -1;
    if (lookups) *lookups = 0;
    if (threads_used) *threads_used = 1;
    if (n <= 1) {
        if (D_out && n == 1) D_out[0] = 0;
        return 0;
    }
    tv_state st;
    memset(&st, 0, sizeof st);
    st.n = n;
    st.q = q;
    st.ng = n / q + 1;
    st.B = q * ((96 + q - 1) / q);
    st.s = codes;
    st.mask = mask;
    const size_t nn = (size_t)n * n, ngn = (size_t)n * st.ng;
    st.D = D_out ? D_out : (int16_t *)malloc(nn * sizeof(int16_t));
    st.A = (int16_t *)calloc(ngn, sizeof(int16_t));
    st.H = (uint32_t *)calloc(ngn, sizeof(uint32_t));
    st.Bv = (int16_t *)calloc(ngn, sizeof(int16_t));
    st.C = (uint16_t *)calloc(ngn, sizeof(uint16_t));
    uint8_t *R = (uint8_t *)malloc((size_t)1 << (2 * (q - 1)));
    int rc = 0;
    if (!st.D || !st.A || !st.H || !st.Bv || !st.C || !R) {
        rc = -2;
        goto out;
    }
    build_r(q, R);
    st.R = R;
    memset(st.D, 0, nn * sizeof(int16_t));
    const int NT = (n + st.B - 1) / st.B;
    int64_t nl = 0;
#ifdef _OPENMP
    const int nth = threads > 0 ? threads : omp_get_num_procs();
#pragma omp parallel num_threads(nth) reduction(+ : nl)
    {
#pragma omp single
        if (threads_used) *threads_used = omp_get_num_threads();
        for (int d = 0; d < NT; ++d) {
#pragma omp for schedule(dynamic, 1)
            for (int I = 0; I < NT - d; ++I) nl += fill_tile(&st, I, I + d);
        }
    }
#else
    (void)threads;
    for (int d = 0; d < NT; ++d)
        for (int I = 0; I < NT - d; ++I) nl += fill_tile(&st, I, I + d);
#endif
    rc = st.D[n - 1];
    if (lookups) *lookups = nl;
out:
    if (!D_out) free(st.D);
    free(st.A);
    free(st.H);
    free(st.Bv);
    free(st.C);
    free(R);
    return rc;
}
