/*
 * oracle.c -- CPU oracle for the Nussinov base-pair maximisation DP and the
 * two-vector Four-Russians method (Venkatachalam, Gusfield, Frid,
 * "Faster Algorithms for RNA-folding using the Four-Russians method").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * GPU library never includes, links or calls it, and it shares no code with
 * the GPU library.
 *
 * Everything here is plain, slow, single-threaded and obviously correct:
 *
 *   oracle_nussinov     Section 2, Eq. 1: the cubic recurrence written out,
 *                       filled diagonal by diagonal.
 *   oracle_brute        Section 2, problem statement: the largest set of
 *                       disjoint, non-crossing, complementary pairs, found by
 *                       enumerating every matching (no DP).  Tiny n only.
 *   oracle_rtable       Section 3.1, the preprocessing routine (the max-val /
 *                       max-index scan over one vector pair), run for every
 *                       pair of (q-1)-bit difference vectors.
 *   oracle_two_vector   Section 3.1, Algorithm 1: column-wise fill with the
 *                       pair term, the two residual loops, the Four-Russians
 *                       loop of table lookups (Eq. 3), and the vector stores.
 *   oracle_two_vector_sliding
 *                       Section 4: the parallel two-vector algorithm with
 *                       difference vectors at every cell and groups relative
 *                       to i, filled diagonal by diagonal, one column per
 *                       process.
 *   oracle_fg           Section 3.2, the FG algorithm: Algorithm 1's fill with
 *                       a table per row and group (D(i,gq) folded in) built
 *                       when the group completes, instead of one table over
 *                       vector pairs.
 *   oracle_traceback    Section 2, the traceback: the argmax of Eq. 1 (D*)
 *                       re-evaluated at each visited cell of a finished table,
 *                       giving one optimal set of pairs.
 *
 * Conventions (the readings of the paper used throughout):
 *   - positions are 0-based; D(i,j) = 0 for i >= j; answer D(0,n-1);
 *   - bases are coded A=0, C=1, G=2, U=3; b(x,y) = bit (4x+y) of pair_mask,
 *     x the base at the smaller index;
 *   - column groups cover columns g*q .. g*q+q-1 and the matching row groups
 *     cover rows g*q+1 .. g*q+q (Section 3.1: row and column groupings differ
 *     by one); group g is used for cell (i,j) iff g*q >= i and g*q+q <= j;
 *   - a difference vector has q-1 free bits (its first difference is 0 by
 *     definition); bit p-1 holds difference p; the table index is
 *     (h << (q-1)) | c, h the horizontal (row) vector, c the vertical
 *     (column) vector stored as positive bits c_p = D(gq+p,j) - D(gq+p+1,j).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline int pair_b(uint16_t mask, int x, int y) {
    if (x < 0 || x > 3 || y < 0 || y > 3) return 0;
    return (mask >> (4 * x + y)) & 1;
}

/* Section 2, Eq. 1.  D is n*n row-major int32 (caller-owned); D[i*n+j] =
 * D(i,j) for i <= j and 0 below the diagonal.  A transposed copy of the table
 * is kept only so that the inner loop reads both operands contiguously; the
 * arithmetic is exactly Eq. 1. */
int oracle_nussinov(const uint8_t *codes, int n, uint16_t mask, int32_t *D) {
    if (n < 0) return -1;
    if (n == 0) return 0;
    memset(D, 0, sizeof(int32_t) * (size_t)n * (size_t)n);
    int32_t *DT = (int32_t *)calloc((size_t)n * (size_t)n, sizeof(int32_t)); /* DT[j*n+i] = D(i,j) */
    if (!DT) return -2;
    for (int d = 1; d < n; ++d) {
        for (int i = 0; i + d < n; ++i) {
            int j = i + d;
            /* first line of Eq. 1: pair i with j around D(i+1,j-1) (0 when i+1 > j-1) */
            int inner = (i + 1 <= j - 1) ? D[(size_t)(i + 1) * n + (j - 1)] : 0;
            int best = pair_b(mask, codes[i], codes[j]) + inner;
            /* second line of Eq. 1: max over splits i+1 <= k <= j of D(i,k-1) + D(k,j) */
            const int32_t *row = D + (size_t)i * n;   /* row[k-1]   = D(i,k-1) */
            const int32_t *col = DT + (size_t)j * n;  /* col[k]     = D(k,j)   */
            for (int k = i + 1; k <= j; ++k) {
                int v = row[k - 1] + col[k];
                if (v > best) best = v;
            }
            D[(size_t)i * n + j] = best;
            DT[(size_t)j * n + i] = best;
        }
    }
    free(DT);
    return 0;
}

/* Score only: D(0,n-1) from the same recurrence (allocates its own table). */
int oracle_nussinov_score(const uint8_t *codes, int n, uint16_t mask) {
    if (n <= 1) return 0;
    int32_t *D = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
    if (!D) return -2;
    int rc = oracle_nussinov(codes, n, mask, D);
    int s = rc == 0 ? D[n - 1] : rc;
    free(D);
    return s;
}

/* ---- brute force over matchings (Section 2: disjoint, non-crossing pairs) ---- */
typedef struct {
    const uint8_t *s;
    int n;
    uint16_t mask;
    int used[64];
    int pa[32], pb[32];
    int np;
    int best;
} brute_state;

static void brute_rec(brute_state *st, int pos) {
    /* upper bound prune: at most one pair per two remaining free positions */
    int free_left = 0;
    for (int t = pos; t < st->n; ++t) free_left += !st->used[t];
    if (st->np + free_left / 2 <= st->best) return;
    while (pos < st->n && st->used[pos]) ++pos;
    if (pos >= st->n) {
        if (st->np > st->best) st->best = st->np;
        return;
    }
    /* option 1: position pos stays unpaired */
    st->used[pos] = 1;
    brute_rec(st, pos + 1);
    st->used[pos] = 0;
    /* option 2: pair pos with a later free position k */
    for (int k = pos + 1; k < st->n; ++k) {
        if (st->used[k] || !pair_b(st->mask, st->s[pos], st->s[k])) continue;
        /* non-crossing: no existing pair (a,b) with a < pos < b < k (all a < pos here) */
        int ok = 1;
        for (int t = 0; t < st->np; ++t)
            if (st->pa[t] < pos && pos < st->pb[t] && st->pb[t] < k) { ok = 0; break; }
        if (!ok) continue;
        st->used[pos] = st->used[k] = 1;
        st->pa[st->np] = pos;
        st->pb[st->np] = k;
        st->np++;
        brute_rec(st, pos + 1);
        st->np--;
        st->used[pos] = st->used[k] = 0;
    }
}

/* Largest non-crossing matching of codes[0..n) by exhaustive search; n <= 40
 * is accepted but only tiny n finish quickly. */
int oracle_brute(const uint8_t *codes, int n, uint16_t mask) {
    if (n < 0 || n > 40) return -1;
    brute_state st;
    memset(&st, 0, sizeof st);
    st.s = codes;
    st.n = n;
    st.mask = mask;
    brute_rec(&st, 0);
    return st.best;
}

/* Section 3.1 preprocessing routine for one vector pair: scan k = 0..q-1 with
 * running sums of the horizontal differences v_k and vertical differences
 * vbar_k (vbar_k = -c_k), keeping the largest total with a strict '>' test;
 * max-val starts at 0 and max-index at 0.  v_0 = vbar_0 = 0. */
static void preprocess_pair(int q, unsigned h, unsigned c, int *max_val, int *max_index) {
    int mv = 0, mi = 0, sum1 = 0, sum2 = 0;
    for (int k = 0; k < q; ++k) {
        int vk = k == 0 ? 0 : (int)((h >> (k - 1)) & 1u);
        int vbark = k == 0 ? 0 : -(int)((c >> (k - 1)) & 1u);
        sum1 += vk;
        sum2 += vbark;
        if (sum1 + sum2 > mv) {
            mv = sum1 + sum2;
            mi = k;
        }
    }
    *max_val = mv;
    *max_index = mi;
}

/* Exhaustive table: R[(h << (q-1)) | c] = max-val, for q in [1, 12]; if
 * R_index is not NULL it receives max-index.  Returns the entry count. */
long oracle_rtable(int q, uint8_t *R, uint8_t *R_index) {
    if (q < 1 || q > 12) return -1;
    long nv = 1L << (q - 1);
    for (long h = 0; h < nv; ++h)
        for (long c = 0; c < nv; ++c) {
            int mv, mi;
            preprocess_pair(q, (unsigned)h, (unsigned)c, &mv, &mi);
            R[(h << (q - 1)) | c] = (uint8_t)mv;
            if (R_index) R_index[(h << (q - 1)) | c] = (uint8_t)mi;
        }
    return nv * nv;
}

/* Section 3.1, Algorithm 1 (serial two-vector).  Fills D column by column
 * (j ascending, i descending).  Per cell: the pair term, the residual splits
 * before the first full group and after the last one (plain Eq. 1 terms),
 * then one table lookup per full group (Eq. 3), and finally the vector stores
 * for any row or column group that the cell completes.  If lookups is not
 * NULL it receives the number of table lookups made.  D as in oracle_nussinov. */
int oracle_two_vector(const uint8_t *codes, int n, int q, uint16_t mask, int32_t *D, int64_t *lookups) {
    if (n < 0 || q < 1 || q > 12) return -1;
    if (lookups) *lookups = 0;
    if (n == 0) return 0;
    long nent = 1L << (2 * (q - 1));
    uint8_t *R = (uint8_t *)malloc((size_t)nent);
    int ng = n / q + 2;
    /* hv[i*ng+g]: horizontal vector of row i, group g; cv[j*ng+g]: vertical vector of column j, group g */
    uint32_t *hv = (uint32_t *)calloc((size_t)n * ng, sizeof(uint32_t));
    uint32_t *cv = (uint32_t *)calloc((size_t)n * ng, sizeof(uint32_t));
    if (!R || !hv || !cv) { free(R); free(hv); free(cv); return -2; }
    oracle_rtable(q, R, NULL);
    memset(D, 0, sizeof(int32_t) * (size_t)n * (size_t)n);
#define DD(a, b) D[(size_t)(a) * n + (b)]
    int64_t nl = 0;
    for (int j = 0; j < n; ++j) {
        /* D(j,j) = 0 already */
        for (int i = j - 1; i >= 0; --i) {
            int inner = (i + 1 <= j - 1) ? DD(i + 1, j - 1) : 0;
            int best = pair_b(mask, codes[i], codes[j]) + inner;
            int gfirst = (i + q - 1) / q;              /* smallest g with g*q >= i     */
            int glast = j >= q ? (j - q) / q : -1;     /* largest g with g*q + q <= j  */
            if (gfirst <= glast) {
                /* residual splits before the first full group: k in [i+1, gfirst*q] */
                for (int k = i + 1; k <= gfirst * q; ++k) {
                    int v = DD(i, k - 1) + DD(k, j);
                    if (v > best) best = v;
                }
                /* residual splits after the last full group: k in [glast*q+q+1, j] */
                for (int k = glast * q + q + 1; k <= j; ++k) {
                    int v = DD(i, k - 1) + DD(k, j);
                    if (v > best) best = v;
                }
                /* Four-Russians loop: one lookup per full group (Eq. 3) */
                for (int g = gfirst; g <= glast; ++g) {
                    unsigned h = hv[(size_t)i * ng + g], c = cv[(size_t)j * ng + g];
                    int v = DD(i, g * q) + DD(g * q + 1, j) + R[((long)h << (q - 1)) | c];
                    ++nl;
                    if (v > best) best = v;
                }
            } else {
                /* no full group: every split is residual */
                for (int k = i + 1; k <= j; ++k) {
                    int v = DD(i, k - 1) + DD(k, j);
                    if (v > best) best = v;
                }
            }
            DD(i, j) = best;
            /* vertical vector of column j for group g is complete once D(g*q+1, j) is known */
            if (i >= 1 && (i - 1) % q == 0) {
                int g = (i - 1) / q;
                if (g * q + q <= j) {
                    uint32_t c = 0;
                    for (int p = 1; p <= q - 1; ++p)
                        c |= (uint32_t)(DD(g * q + p, j) - DD(g * q + p + 1, j)) << (p - 1);
                    cv[(size_t)j * ng + g] = c;
                }
            }
            /* horizontal vector of row i for group g is complete once D(i, g*q+q-1) is known */
            if ((j + 1) % q == 0) {
                int g = (j + 1) / q - 1;
                if (g * q >= i) {
                    uint32_t h = 0;
                    for (int p = 1; p <= q - 1; ++p)
                        h |= (uint32_t)(DD(i, g * q + p) - DD(i, g * q + p - 1)) << (p - 1);
                    hv[(size_t)i * ng + g] = h;
                }
            }
        }
    }
#undef DD
    if (lookups) *lookups = nl;
    free(R);
    free(hv);
    free(cv);
    return 0;
}

/* Section 4, the parallel two-vector algorithm with difference vectors at
 * every cell (the sliding-window variant).  The fill goes diagonal by diagonal
 * (iteration d = j - i); within an iteration every column j ("process j") fills
 * cell (i, j) = (j - d, j):
 *   1. D(i,j) = D(i+1,j-1) + b(S_i,S_j);
 *   2. groups relative to i: for k' = 0 .. floor((j-i)/q) - 1, k = i + k'q,
 *      D(i,j) = max(D(i,j), D(i,k) + D(k+1,j) + R[dH(i,k)][dV(k+1,j)]);
 *   3. residual splits k = i + floor((j-i)/q)*q .. j-1:
 *      D(i,j) = max(D(i,j), D(i,k) + D(k+1,j));
 *   4. the vectors that cell (i,j) completes are stored: dV(i,j), the vertical
 *      vector of cells D(i..i+q-1, j), and dH(i, j-q+1), the horizontal vector
 *      of cells D(i, j-q+1..j).
 * Vectors (the readings used throughout): dH(i,k) has bit p-1 =
 * D(i,k+p) - D(i,k+p-1) and dV(r,j) has bit p-1 = D(r+p-1,j) - D(r+p,j), for
 * p = 1..q-1, so that D(i,k) + D(k+1,j) + R[dH(i,k)][dV(k+1,j)] is the best of
 * the splits D(i,k+p) + D(k+p+1,j), p = 0..q-1.  The section's loop bounds are
 * garbled in the text; this is the reading in which the groups and the
 * residual together cover every split k in [i, j-1] (in the D(i,k) + D(k+1,j)
 * form) exactly once.  D as in oracle_nussinov; lookups (if not NULL) receives
 * the number of table lookups, sum over cells of floor((j-i)/q). */
int oracle_two_vector_sliding(const uint8_t *codes, int n, int q, uint16_t mask, int32_t *D, int64_t *lookups) {
    if (n < 0 || q < 1 || q > 12) return -1;
    if (lookups) *lookups = 0;
    if (n == 0) return 0;
    long nent = 1L << (2 * (q - 1));
    uint8_t *R = (uint8_t *)malloc((size_t)nent);
    /* dh[i*n+k] = dH(i,k); dv[r*n+j] = dV(r,j) */
    uint32_t *dh = (uint32_t *)calloc((size_t)n * n, sizeof(uint32_t));
    uint32_t *dv = (uint32_t *)calloc((size_t)n * n, sizeof(uint32_t));
    if (!R || !dh || !dv) { free(R); free(dh); free(dv); return -2; }
    oracle_rtable(q, R, NULL);
    memset(D, 0, sizeof(int32_t) * (size_t)n * (size_t)n);
#define DD(a, b) (((a) < n && (b) >= 0 && (a) <= (b)) ? D[(size_t)(a) * n + (b)] : 0)
    int64_t nl = 0;
    for (int d = 1; d < n; ++d) {
        for (int j = d; j < n; ++j) {
            const int i = j - d;
            /* 1. pair term */
            int best = DD(i + 1, j - 1) + pair_b(mask, codes[i], codes[j]);
            /* 2. groups relative to i, one lookup each */
            const int ng = (j - i) / q;
            for (int kp = 0; kp < ng; ++kp) {
                const int k = i + kp * q;
                const unsigned h = dh[(size_t)i * n + k], c = dv[(size_t)(k + 1) * n + j];
                int v = DD(i, k) + DD(k + 1, j) + R[((long)h << (q - 1)) | c];
                ++nl;
                if (v > best) best = v;
            }
            /* 3. residual splits */
            for (int k = i + ng * q; k <= j - 1; ++k) {
                int v = DD(i, k) + DD(k + 1, j);
                if (v > best) best = v;
            }
            D[(size_t)i * n + j] = best;
            /* 4. the vectors this cell completes */
            {
                uint32_t c = 0;
                for (int p = 1; p <= q - 1; ++p) c |= (uint32_t)(DD(i + p - 1, j) - DD(i + p, j)) << (p - 1);
                dv[(size_t)i * n + j] = c;
            }
            if (j - q + 1 >= i) {
                const int k = j - q + 1;
                uint32_t h = 0;
                for (int p = 1; p <= q - 1; ++p) h |= (uint32_t)(DD(i, k + p) - DD(i, k + p - 1)) << (p - 1);
                dh[(size_t)i * n + k] = h;
            }
        }
    }
#undef DD
    if (lookups) *lookups = nl;
    free(R);
    free(dh);
    free(dv);
    return 0;
}

/* Section 3.2, the FG algorithm (Frid and Gusfield).  The fill and the
 * groups are Algorithm 1's (column by column; group g full for cell (i,j) iff
 * g*q >= i and g*q+q <= j; the residual loops before the first and after the
 * last full group), but there is no table over vector pairs: when row i's
 * group g is complete (D(i, g*q+q-1) is known), the preprocessing routine runs
 * for that row's own horizontal vector h against every vertical vector c,
 * D(i, g*q) is added, and the result is tabled per row and group:
 *   FG[i][g][c] = D(i, g*q) + max_{0<=k<=q-1} sum_{p<=k} (h_p - c_p).
 * A cell's group term is FG[i][g][c(g,j)] + D(g*q+1, j).  The text's "added to
 * D(q,j)" is read as D(g*q+1, j), the top of the group's column segment (as
 * in Eq. 3).  If lookups is not NULL it receives the number of table lookups;
 * if tables is not NULL, the number of (row, group) tables built.  D as in
 * oracle_nussinov. */
int oracle_fg(const uint8_t *codes, int n, int q, uint16_t mask, int32_t *D, int64_t *lookups, int64_t *tables) {
    if (n < 0 || q < 1 || q > 12) return -1;
    if (lookups) *lookups = 0;
    if (tables) *tables = 0;
    if (n == 0) return 0;
    const int nb = q - 1, nc = 1 << nb, ng = n / q + 2;
    int32_t *fg = (int32_t *)calloc((size_t)n * ng * nc, sizeof(int32_t));
    uint32_t *cv = (uint32_t *)calloc((size_t)n * ng, sizeof(uint32_t));
    if (!fg || !cv) { free(fg); free(cv); return -2; }
    memset(D, 0, sizeof(int32_t) * (size_t)n * (size_t)n);
#define DD(a, b) D[(size_t)(a) * n + (b)]
    int64_t nl = 0, nt = 0;
    for (int j = 0; j < n; ++j) {
        /* i = j: the diagonal cell, D(j,j) = 0, only completes a group when q = 1 */
        for (int i = j; i >= 0; --i) {
            if (i < j) {
                int inner = (i + 1 <= j - 1) ? DD(i + 1, j - 1) : 0;
                int best = pair_b(mask, codes[i], codes[j]) + inner;
                int gfirst = (i + q - 1) / q;
                int glast = j >= q ? (j - q) / q : -1;
                if (gfirst <= glast) {
                    for (int k = i + 1; k <= gfirst * q; ++k) {
                        int v = DD(i, k - 1) + DD(k, j);
                        if (v > best) best = v;
                    }
                    for (int k = glast * q + q + 1; k <= j; ++k) {
                        int v = DD(i, k - 1) + DD(k, j);
                        if (v > best) best = v;
                    }
                    for (int g = gfirst; g <= glast; ++g) {
                        int v = fg[((size_t)i * ng + g) * nc + cv[(size_t)j * ng + g]] + DD(g * q + 1, j);
                        ++nl;
                        if (v > best) best = v;
                    }
                } else {
                    for (int k = i + 1; k <= j; ++k) {
                        int v = DD(i, k - 1) + DD(k, j);
                        if (v > best) best = v;
                    }
                }
                DD(i, j) = best;
            }
            /* vertical vector of column j, group g, complete once D(g*q+1, j) is known (as in Algorithm 1) */
            if (i >= 1 && (i - 1) % q == 0) {
                int g = (i - 1) / q;
                if (g * q + q <= j) {
                    uint32_t c = 0;
                    for (int p = 1; p <= q - 1; ++p)
                        c |= (uint32_t)(DD(g * q + p, j) - DD(g * q + p + 1, j)) << (p - 1);
                    cv[(size_t)j * ng + g] = c;
                }
            }
            /* row i's group g complete: run the preprocessing for its vector against every c */
            if ((j + 1) % q == 0) {
                int g = (j + 1) / q - 1;
                if (g * q >= i) {
                    uint32_t h = 0;
                    for (int p = 1; p <= q - 1; ++p)
                        h |= (uint32_t)(DD(i, g * q + p) - DD(i, g * q + p - 1)) << (p - 1);
                    for (int c = 0; c < nc; ++c) {
                        int mv, mi;
                        preprocess_pair(q, h, (unsigned)c, &mv, &mi);
                        fg[((size_t)i * ng + g) * nc + c] = DD(i, g * q) + mv;
                    }
                    ++nt;
                }
            }
        }
    }
#undef DD
    if (lookups) *lookups = nl;
    if (tables) *tables = nt;
    free(fg);
    free(cv);
    return 0;
}

/* Section 2: traceback.  The paper keeps D*(i,j), the argmax of Eq. 1, beside
 * D; here the argmax is re-evaluated from D at each cell the traceback visits,
 * with a fixed order of preference so that the result is one definite optimal
 * structure:
 *   1. the split k = i+1 (base i left unpaired), if D(i,j) = D(i+1,j);
 *   2. else the pair (i,j), if b(S_i,S_j) = 1 and D(i,j) = D(i+1,j-1) + 1;
 *   3. else the smallest k in [i+2, j] with D(i,j) = D(i,k-1) + D(k,j).
 * D: the n*n row-major table of oracle_nussinov (D(i,j) = 0 for i >= j).
 * partner[x] = the base paired with x, or -1.  Returns the number of pairs,
 * or -1 if the table admits no argmax somewhere (not a table of Eq. 1). */
int oracle_traceback(const uint8_t *codes, int n, uint16_t mask, const int32_t *D, int32_t *partner) {
    if (n <= 0) return 0;
    for (int x = 0; x < n; ++x) partner[x] = -1;
    int *stack = (int *)malloc(sizeof(int) * 2 * (size_t)(n + 1));
    if (!stack) return -1;
    int top = 0, pairs = 0;
    stack[top++] = 0;
    stack[top++] = n - 1;
#define DV(a, b) ((a) >= (b) ? 0 : D[(size_t)(a) * n + (b)])
    while (top > 0) {
        int j = stack[--top];
        int i = stack[--top];
        while (i < j) {
            const int dij = DV(i, j);
            if (dij == DV(i + 1, j)) {            /* 1: i unpaired */
                ++i;
                continue;
            }
            if (pair_b(mask, codes[i], codes[j]) && dij == DV(i + 1, j - 1) + 1) {   /* 2: pair (i, j) */
                partner[i] = j;
                partner[j] = i;
                ++pairs;
                ++i;
                --j;
                continue;
            }
            int k = i + 2;                          /* 3: the smallest split */
            while (k <= j && DV(i, k - 1) + DV(k, j) != dij) ++k;
            if (k > j) {
                free(stack);
                return -1;
            }
            stack[top++] = k;
            stack[top++] = j;
            j = k - 1;
        }
    }
#undef DV
    free(stack);
    return pairs;
}
