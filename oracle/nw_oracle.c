/*
 * Plain CPU Needleman-Wunsch oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file.  The product path never does; it shares no code with it.
 *
 * What it computes is the textbook global-alignment dynamic programme the
 * paper accelerates, written out cell by cell with no blocking, tiling or
 * reordering:
 *
 *   Grid (Sec. 2.1): H has (m+1) x (n+1) cells; row 0 / column 0 are the
 *   empty label cells, A labels the rows (query, length m), B the columns
 *   (reference, length n).
 *   Initial data (Sec. 2.2): H(0,0) = 0, H(i,0) = i*gap, H(0,j) = j*gap.
 *   Scoring (Sec. 2.3, Eq. 1, read as standard NW -- the printed formula adds
 *   the cell's own score to all three terms, which contradicts the stated gap
 *   penalty; the only reading consistent with both is):
 *       H(i,j) = max( H(i-1,j-1) + s(A_i,B_j),  H(i-1,j) + gap,  H(i,j-1) + gap )
 *       s = match if A_i == B_j else mismatch.
 *   Backtracking (Sec. 2.4) from (m,n) to (0,0): vertical (i-1,j) is a gap in
 *   the row sequence B (op 'I': A_i consumed alone), horizontal (i,j-1) is a
 *   gap in the column sequence A (op 'D': B_j consumed alone), diagonal is a
 *   match '=' or mismatch 'X'.  Where several predecessors tie, the single
 *   path with priority diagonal > vertical > horizontal is taken (the order of
 *   the direction codes 1/2/3 of Sec. 3.1).  On row 0 only horizontal moves
 *   remain, on column 0 only vertical ones.
 *
 * Sequences are arrays of base codes 0..3 (A, C, G, T), one byte per base.
 * All arithmetic is int32 (no rounding anywhere).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NWO_OK 0
#define NWO_ERR_ARG (-1)
#define NWO_ERR_OOM (-2)

static int32_t subst(uint8_t x, uint8_t y, int32_t match, int32_t mismatch) {
    return x == y ? match : mismatch;
}

static int32_t max2(int32_t x, int32_t y) { return x > y ? x : y; }

/* Fill the whole (m+1) x (n+1) score grid H (row-major, stride n+1). */
int nwo_fill(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
             int32_t match, int32_t mismatch, int32_t gap, int32_t *H) {
    if (m < 0 || n < 0 || !H) return NWO_ERR_ARG;
    const int64_t w = n + 1;
    H[0] = 0;                                   /* Sec. 2.2: top-left cell */
    for (int64_t j = 1; j <= n; ++j) H[j] = (int32_t)j * gap;       /* first row */
    for (int64_t i = 1; i <= m; ++i) H[i * w] = (int32_t)i * gap;   /* first column */
    for (int64_t i = 1; i <= m; ++i) {          /* Sec. 2.3: row by row */
        for (int64_t j = 1; j <= n; ++j) {
            int32_t diag = H[(i - 1) * w + (j - 1)] + subst(a[i - 1], b[j - 1], match, mismatch);
            int32_t up = H[(i - 1) * w + j] + gap;
            int32_t left = H[i * w + (j - 1)] + gap;
            H[i * w + j] = max2(diag, max2(up, left));
        }
    }
    return NWO_OK;
}

/* Sec. 2.4 backtracking over a filled grid.  Writes the ops in forward order
 * into ops[0 .. *nops-1] (capacity m+n).  Returns the score H(m,n). */
static int32_t traceback(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                         int32_t match, int32_t mismatch, int32_t gap,
                         const int32_t *H, char *ops, int64_t *nops) {
    const int64_t w = n + 1;
    int64_t i = m, j = n, k = 0;
    while (i > 0 || j > 0) {
        int32_t here = H[i * w + j];
        if (i > 0 && j > 0 &&
            here == H[(i - 1) * w + (j - 1)] + subst(a[i - 1], b[j - 1], match, mismatch)) {
            ops[k++] = (a[i - 1] == b[j - 1]) ? '=' : 'X';
            --i; --j;
        } else if (i > 0 && (j == 0 || here == H[(i - 1) * w + j] + gap)) {
            ops[k++] = 'I';
            --i;
        } else {
            ops[k++] = 'D';
            --j;
        }
    }
    for (int64_t x = 0, y = k - 1; x < y; ++x, --y) {   /* reverse to forward order */
        char t = ops[x]; ops[x] = ops[y]; ops[y] = t;
    }
    *nops = k;
    return H[m * w + n];
}

/* Score plus alignment.  ops needs room for m+n chars.  Materialises the full
 * int32 grid ((m+1)*(n+1)*4 bytes). */
int nwo_align(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
              int32_t match, int32_t mismatch, int32_t gap,
              int32_t *score, char *ops, int64_t *nops) {
    if (m < 0 || n < 0 || !score || !ops || !nops) return NWO_ERR_ARG;
    size_t cells = (size_t)(m + 1) * (size_t)(n + 1);
    int32_t *H = (int32_t *)malloc(cells * sizeof(int32_t));
    if (!H) return NWO_ERR_OOM;
    nwo_fill(a, m, b, n, match, mismatch, gap, H);
    *score = traceback(a, m, b, n, match, mismatch, gap, H, ops, nops);
    free(H);
    return NWO_OK;
}

/* Score only: the same recurrence keeping just the previous row. */
int nwo_score(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
              int32_t match, int32_t mismatch, int32_t gap, int32_t *score) {
    if (m < 0 || n < 0 || !score) return NWO_ERR_ARG;
    int32_t *prev = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return NWO_ERR_OOM; }
    for (int64_t j = 0; j <= n; ++j) prev[j] = (int32_t)j * gap;
    for (int64_t i = 1; i <= m; ++i) {
        cur[0] = (int32_t)i * gap;
        for (int64_t j = 1; j <= n; ++j) {
            int32_t diag = prev[j - 1] + subst(a[i - 1], b[j - 1], match, mismatch);
            int32_t up = prev[j] + gap;
            int32_t left = cur[j - 1] + gap;
            cur[j] = max2(diag, max2(up, left));
        }
        int32_t *t = prev; prev = cur; cur = t;
    }
    *score = prev[n];
    free(prev); free(cur);
    return NWO_OK;
}

/* ------------------------------------------------------------------------
 * Banded variant (not in the paper; the reference for the certified band).
 *
 * With delta = n - m, the band holds the cells whose diagonal d = j - i lies
 * in [min(0,delta) - w, max(0,delta) + w].  Cells outside the band are -inf:
 * they take part in no path.  The boundary cells of row 0 / column 0 keep
 * their Sec. 2.2 values when they are inside the band.
 *
 * Certificate bound U: every path from (0,0) to (m,n) that leaves the band
 * has a first out-of-band cell q = (qi,qj), reached from an in-band cell p by
 * one gap move.  Its score is at most Hb(p) + gap + best(q), where best(q) is
 * the largest score any path from q to (m,n) can collect:
 *     best(q) = match * min(m-qi, n-qj) + gap * |(m-qi) - (n-qj)|
 * (valid when match >= mismatch, match >= 0 and gap <= 0).  U is the max of
 * that over every such exit step (U = -inf when no exit step exists).
 * Hb(p) is the best score over in-band paths to p, so it bounds the in-band
 * prefix of such a path from above; hence U bounds every path that leaves
 * the band.  Writes S_b = Hb(m,n) and U.
 * ---------------------------------------------------------------------- */
#define NWO_NEG_INF (INT32_MIN / 2)

static int in_band(int64_t i, int64_t j, int64_t lo, int64_t hi) {
    int64_t d = j - i;
    return d >= lo && d <= hi;
}

static int32_t rest_bound(int64_t m, int64_t n, int64_t qi, int64_t qj, int32_t match, int32_t gap) {
    int64_t r = m - qi, c = n - qj;
    int64_t mn = r < c ? r : c;
    int64_t diff = r > c ? r - c : c - r;
    return (int32_t)(match * mn + gap * diff);
}

/* The same recurrence restricted to an arbitrary set of cells: row i (1..m)
 * may use columns row_lo[i-1]..row_hi[i-1] (inclusive, 1-based), row 0 the
 * columns 0..row0_hi, column 0 the rows 0..col0_hi; every other cell is
 * -infinity.  The score is H(m,n) (-infinity when unreachable).  Two rolling
 * rows.  This is the plain definition of a DP over a cell subset: any
 * subset containing a band gives a score between the banded and the full
 * one. */
int nwo_region(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
               int32_t match, int32_t mismatch, int32_t gap,
               const int64_t *row_lo, const int64_t *row_hi, int64_t row0_hi, int64_t col0_hi,
               int32_t *score) {
    if (m < 0 || n < 0 || !score || (m > 0 && (!row_lo || !row_hi))) return NWO_ERR_ARG;
    int32_t *prev = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return NWO_ERR_OOM;
    }
    for (int64_t j = 0; j <= n; ++j) prev[j] = j <= row0_hi ? (int32_t)j * gap : NWO_NEG_INF;
    for (int64_t i = 1; i <= m; ++i) {
        cur[0] = i <= col0_hi ? (int32_t)i * gap : NWO_NEG_INF;
        for (int64_t j = 1; j <= n; ++j) {
            if (j < row_lo[i - 1] || j > row_hi[i - 1]) {
                cur[j] = NWO_NEG_INF;
                continue;
            }
            int32_t best = NWO_NEG_INF;
            if (prev[j - 1] > NWO_NEG_INF) best = max2(best, prev[j - 1] + subst(a[i - 1], b[j - 1], match, mismatch));
            if (prev[j] > NWO_NEG_INF) best = max2(best, prev[j] + gap);
            if (cur[j - 1] > NWO_NEG_INF) best = max2(best, cur[j - 1] + gap);
            cur[j] = best;
        }
        int32_t *t = prev;
        prev = cur;
        cur = t;
    }
    *score = prev[n];
    free(prev);
    free(cur);
    return NWO_OK;
}

int nwo_banded(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
               int32_t match, int32_t mismatch, int32_t gap, int64_t w,
               int32_t *score_band, int32_t *bound_out, int32_t *Hout) {
    if (m < 0 || n < 0 || w < 0 || !score_band || !bound_out) return NWO_ERR_ARG;
    const int64_t delta = n - m;
    const int64_t lo = (delta < 0 ? delta : 0) - w;
    const int64_t hi = (delta > 0 ? delta : 0) + w;
    const int64_t W = n + 1;
    size_t cells = (size_t)(m + 1) * (size_t)W;
    int32_t *H = Hout ? Hout : (int32_t *)malloc(cells * sizeof(int32_t));
    if (!H) return NWO_ERR_OOM;
    for (int64_t i = 0; i <= m; ++i) {
        for (int64_t j = 0; j <= n; ++j) {
            int32_t v;
            if (!in_band(i, j, lo, hi)) v = NWO_NEG_INF;
            else if (i == 0) v = (int32_t)j * gap;
            else if (j == 0) v = (int32_t)i * gap;
            else {
                int32_t best = NWO_NEG_INF;
                int32_t dg = H[(i - 1) * W + (j - 1)];
                int32_t up = H[(i - 1) * W + j];
                int32_t lf = H[i * W + (j - 1)];
                if (dg > NWO_NEG_INF) best = max2(best, dg + subst(a[i - 1], b[j - 1], match, mismatch));
                if (up > NWO_NEG_INF) best = max2(best, up + gap);
                if (lf > NWO_NEG_INF) best = max2(best, lf + gap);
                v = best;
            }
            H[i * W + j] = v;
        }
    }
    int32_t U = NWO_NEG_INF;
    for (int64_t i = 0; i <= m; ++i) {
        for (int64_t j = 0; j <= n; ++j) {
            if (!in_band(i, j, lo, hi) || H[i * W + j] <= NWO_NEG_INF) continue;
            /* vertical exit step (i,j) -> (i+1,j) */
            if (i + 1 <= m && !in_band(i + 1, j, lo, hi)) {
                int32_t c = H[i * W + j] + gap + rest_bound(m, n, i + 1, j, match, gap);
                U = max2(U, c);
            }
            /* horizontal exit step (i,j) -> (i,j+1) */
            if (j + 1 <= n && !in_band(i, j + 1, lo, hi)) {
                int32_t c = H[i * W + j] + gap + rest_bound(m, n, i, j + 1, match, gap);
                U = max2(U, c);
            }
        }
    }
    *score_band = H[m * W + n];
    *bound_out = U;
    if (!Hout) free(H);
    return NWO_OK;
}

/* ------------------------------------------------------------------------
 * Local alignment (Smith-Waterman; not in the paper, the same grid with a
 * floor of 0: an alignment may start and end anywhere).
 *
 *   H(i,0) = H(0,j) = 0
 *   H(i,j) = max( 0, H(i-1,j-1) + s(A_i,B_j), H(i-1,j) + gap, H(i,j-1) + gap )
 *
 * The score is the largest H(i,j).  The alignment ends at the first cell in
 * row-major order (smallest i, then smallest j) holding it, and is traced
 * back from there with the priority diagonal > vertical > horizontal of the
 * global walk, stopping at the first cell whose H is 0 (the alignment's
 * start).  A score of 0 gives the empty alignment at (0,0).  Writes the
 * score, the end cell (i_end, j_end) and the start cell (i_start, j_start)
 * -- the alignment covers A[i_start .. i_end) and B[j_start .. j_end),
 * 0-based -- and the ops in forward order.
 * ---------------------------------------------------------------------- */
static int32_t max4(int32_t a, int32_t b, int32_t c, int32_t d) { return max2(max2(a, b), max2(c, d)); }

int nwo_local_fill(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                   int32_t match, int32_t mismatch, int32_t gap, int32_t *H) {
    if (m < 0 || n < 0 || !H) return NWO_ERR_ARG;
    const int64_t w = n + 1;
    for (int64_t j = 0; j <= n; ++j) H[j] = 0;
    for (int64_t i = 1; i <= m; ++i) {
        H[i * w] = 0;
        for (int64_t j = 1; j <= n; ++j) {
            int32_t diag = H[(i - 1) * w + (j - 1)] + subst(a[i - 1], b[j - 1], match, mismatch);
            int32_t up = H[(i - 1) * w + j] + gap;
            int32_t left = H[i * w + (j - 1)] + gap;
            H[i * w + j] = max4(0, diag, up, left);
        }
    }
    return NWO_OK;
}

int nwo_local_align(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    int32_t match, int32_t mismatch, int32_t gap, int32_t *score, int64_t *ends,
                    char *ops, int64_t *nops) {
    if (m < 0 || n < 0 || !score || !ends || !ops || !nops) return NWO_ERR_ARG;
    const int64_t w = n + 1;
    int32_t *H = (int32_t *)malloc((size_t)(m + 1) * (size_t)w * sizeof(int32_t));
    if (!H) return NWO_ERR_OOM;
    nwo_local_fill(a, m, b, n, match, mismatch, gap, H);
    int64_t bi = 0, bj = 0;
    for (int64_t i = 0; i <= m; ++i)           /* row-major: the first maximum */
        for (int64_t j = 0; j <= n; ++j)
            if (H[i * w + j] > H[bi * w + bj]) { bi = i; bj = j; }
    int64_t i = bi, j = bj, k = 0;
    while (H[i * w + j] > 0) {
        int32_t here = H[i * w + j];
        if (here == H[(i - 1) * w + (j - 1)] + subst(a[i - 1], b[j - 1], match, mismatch)) {
            ops[k++] = (a[i - 1] == b[j - 1]) ? '=' : 'X';
            --i; --j;
        } else if (here == H[(i - 1) * w + j] + gap) {
            ops[k++] = 'I';
            --i;
        } else {
            ops[k++] = 'D';
            --j;
        }
    }
    for (int64_t x = 0, y = k - 1; x < y; ++x, --y) {
        char t = ops[x]; ops[x] = ops[y]; ops[y] = t;
    }
    *nops = k;
    *score = H[bi * w + bj];
    ends[0] = i; ends[1] = j; ends[2] = bi; ends[3] = bj;
    free(H);
    return NWO_OK;
}

/* Local score only, two rolling rows. */
int nwo_local_score(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                    int32_t match, int32_t mismatch, int32_t gap, int32_t *score) {
    if (m < 0 || n < 0 || !score) return NWO_ERR_ARG;
    int32_t *prev = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    int32_t *cur = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    if (!prev || !cur) { free(prev); free(cur); return NWO_ERR_OOM; }
    int32_t best = 0;
    for (int64_t i = 1; i <= m; ++i) {
        cur[0] = 0;
        for (int64_t j = 1; j <= n; ++j) {
            int32_t diag = prev[j - 1] + subst(a[i - 1], b[j - 1], match, mismatch);
            int32_t up = prev[j] + gap;
            int32_t left = cur[j - 1] + gap;
            cur[j] = max4(0, diag, up, left);
            best = max2(best, cur[j]);
        }
        int32_t *t = prev; prev = cur; cur = t;
    }
    *score = best;
    free(prev); free(cur);
    return NWO_OK;
}

/* ------------------------------------------------------------------------
 * Affine gaps (Gotoh; not in the paper, whose gap penalty is linear, but the
 * center-star method it cites uses them).  A run of k gap moves of one kind
 * scores go + k*ge (open plus extend, both <= 0).  Three grids:
 *   E(i,j) best score of A[:i] vs B[:j] ending in a horizontal move (B_j alone):
 *          max( E(i,j-1) + ge, H(i,j-1) + go + ge )
 *   F(i,j) ending in a vertical move (A_i alone):
 *          max( F(i-1,j) + ge, H(i-1,j) + go + ge )
 *   H(i,j) best score: max( H(i-1,j-1) + s(A_i,B_j), E(i,j), F(i,j) )
 * Boundary: H(0,0) = 0; H(0,j) = E(0,j) = go + j*ge and F(0,j) = -inf for
 * j >= 1; H(i,0) = F(i,0) = go + i*ge and E(i,0) = -inf for i >= 1.
 * Walk from (m,n) in state H: diagonal if H == H(i-1,j-1) + s, else the
 * vertical gap if H == F, else the horizontal gap; in a gap state the move
 * is emitted and the walk stays in the gap when extending is strictly
 * better than opening (F(i-1,j) + ge > H(i-1,j) + go + ge), else returns to
 * state H at the predecessor -- a tie closes the gap.  On row 0 only
 * horizontal moves remain, on column 0 only vertical ones.  With go = 0
 * this is the linear walk move for move.
 * ---------------------------------------------------------------------- */
#define NWO_AFF_NEG (INT32_MIN / 4)

static int32_t aff_add(int32_t x, int32_t y) { return x <= NWO_AFF_NEG ? NWO_AFF_NEG : x + y; }

int nwo_affine_fill(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, int32_t match, int32_t mismatch,
                    int32_t go, int32_t ge, int32_t *H, int32_t *E, int32_t *F) {
    if (m < 0 || n < 0 || !H || !E || !F) return NWO_ERR_ARG;
    const int64_t w = n + 1;
    H[0] = 0;
    E[0] = F[0] = NWO_AFF_NEG;
    for (int64_t j = 1; j <= n; ++j) {
        H[j] = E[j] = go + (int32_t)j * ge;
        F[j] = NWO_AFF_NEG;
    }
    for (int64_t i = 1; i <= m; ++i) {
        H[i * w] = F[i * w] = go + (int32_t)i * ge;
        E[i * w] = NWO_AFF_NEG;
        for (int64_t j = 1; j <= n; ++j) {
            const int64_t c = i * w + j;
            E[c] = max2(aff_add(E[c - 1], ge), H[c - 1] + go + ge);
            F[c] = max2(aff_add(F[c - w], ge), H[c - w] + go + ge);
            H[c] = max2(H[c - w - 1] + subst(a[i - 1], b[j - 1], match, mismatch), max2(E[c], F[c]));
        }
    }
    return NWO_OK;
}

int nwo_affine_align(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, int32_t match, int32_t mismatch,
                     int32_t go, int32_t ge, int32_t *score, char *ops, int64_t *nops) {
    if (m < 0 || n < 0 || !score || !ops || !nops) return NWO_ERR_ARG;
    const int64_t w = n + 1;
    const size_t cells = (size_t)(m + 1) * (size_t)w;
    int32_t *H = (int32_t *)malloc(cells * sizeof(int32_t));
    int32_t *E = (int32_t *)malloc(cells * sizeof(int32_t));
    int32_t *F = (int32_t *)malloc(cells * sizeof(int32_t));
    if (!H || !E || !F) { free(H); free(E); free(F); return NWO_ERR_OOM; }
    nwo_affine_fill(a, m, b, n, match, mismatch, go, ge, H, E, F);
    int64_t i = m, j = n, k = 0;
    int state = 0;                                   /* 0: H, 1: F (vertical gap), 2: E (horizontal gap) */
    while (i > 0 || j > 0) {
        if (i == 0) { ops[k++] = 'D'; --j; continue; }
        if (j == 0) { ops[k++] = 'I'; --i; continue; }
        const int64_t c = i * w + j;
        if (state == 0) {
            if (H[c] == H[c - w - 1] + subst(a[i - 1], b[j - 1], match, mismatch)) {
                ops[k++] = (a[i - 1] == b[j - 1]) ? '=' : 'X';
                --i; --j;
                continue;
            }
            state = H[c] == F[c] ? 1 : 2;
        }
        if (state == 1) {
            ops[k++] = 'I';
            state = aff_add(F[c - w], ge) > H[c - w] + go + ge ? 1 : 0;
            --i;
        } else {
            ops[k++] = 'D';
            state = aff_add(E[c - 1], ge) > H[c - 1] + go + ge ? 2 : 0;
            --j;
        }
    }
    for (int64_t x = 0, y = k - 1; x < y; ++x, --y) {
        char t = ops[x]; ops[x] = ops[y]; ops[y] = t;
    }
    *nops = k;
    *score = H[m * w + n];
    free(H); free(E); free(F);
    return NWO_OK;
}

/* Affine score only, rolling rows. */
int nwo_affine_score(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, int32_t match, int32_t mismatch,
                     int32_t go, int32_t ge, int32_t *score) {
    if (m < 0 || n < 0 || !score) return NWO_ERR_ARG;
    int32_t *Hp = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *Hc = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *Fp = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *Fc = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    if (!Hp || !Hc || !Fp || !Fc) { free(Hp); free(Hc); free(Fp); free(Fc); return NWO_ERR_OOM; }
    Hp[0] = 0;
    Fp[0] = NWO_AFF_NEG;
    for (int64_t j = 1; j <= n; ++j) { Hp[j] = go + (int32_t)j * ge; Fp[j] = NWO_AFF_NEG; }
    for (int64_t i = 1; i <= m; ++i) {
        Hc[0] = Fc[0] = go + (int32_t)i * ge;
        int32_t e = NWO_AFF_NEG;                      /* E(i,0) */
        for (int64_t j = 1; j <= n; ++j) {
            e = max2(aff_add(e, ge), Hc[j - 1] + go + ge);
            Fc[j] = max2(aff_add(Fp[j], ge), Hp[j] + go + ge);
            Hc[j] = max2(Hp[j - 1] + subst(a[i - 1], b[j - 1], match, mismatch), max2(e, Fc[j]));
        }
        int32_t *t = Hp; Hp = Hc; Hc = t;
        t = Fp; Fp = Fc; Fc = t;
    }
    *score = m == 0 && n == 0 ? 0 : Hp[n];
    free(Hp); free(Hc); free(Fp); free(Fc);
    return NWO_OK;
}
