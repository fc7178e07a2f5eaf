/*
 * nq_oracle.c -- plain, slow, obviously-correct CPU oracle for exact N-Queens
 * solution counting (Yao & Li, "High-Performance N-Queens Solver on GPU:
 * Iterative DFS with Zero Bank Conflicts").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product library
 * never links, loads or calls it, and this file includes no header of the
 * product and shares no helper, table or constant with it.
 *
 * What is computed (problem statement, Section 1): the number of ways to put
 * N mutually non-attacking queens on an N x N board, i.e. the number of
 * permutations s of {0..N-1} with |s(i) - s(j)| != |i - j| for all i != j.
 *
 * Deliberately NOT the paper's method: no bitmasks, no Somers state, no
 * shifting diagonals. A board is three bool arrays indexed by column c,
 * diagonal r + c and anti-diagonal r - c + N - 1, and the search is the
 * textbook row-by-row recursive backtracker.
 *
 * Functions, and what pins each one (tests/test_oracle.py unless noted):
 *   orc_brute_perm          all N! permutations, pairwise attack check (Section
 *                           1's definition written out). Pinned against
 *                           orc_total for N <= 10, which the next pins fix.
 *   orc_total               backtracker over the whole board, no symmetry
 *                           (Section 1). Pinned by an independent Python
 *                           permutation count (N <= 7), orc_brute_perm (N <= 10),
 *                           OEIS A000170 (N <= 13; N <= 16 through the symmetric
 *                           driver), and its node count by brute force over all
 *                           partial placements.
 *   orc_count_constrained   backtracker with some rows' columns fixed (the
 *                           serving extension; not in the paper). Pinned by
 *                           brute force with the queens fixed, the eight board
 *                           symmetries, and k = 0 reducing to orc_total.
 *   orc_prefixes            the symmetric prefix set of Section 1 / Section 2
 *                           (first-row half symmetry and odd-N middle rule) as
 *                           column lists, in the canonical order. Pinned by a
 *                           brute-force prefix set, weights summing to the
 *                           unsymmetric count, and the 27-Queens log's
 *                           453,688,251 subproblems at d = 7 (Section 4.5).
 *   orc_prefix_count        the same set's size, without materialising it.
 *                           Pinned by len(orc_prefixes) and the same log.
 *   orc_prefixes_at_ranks   the prefixes with given canonical indices. Pinned
 *                           by indexing orc_prefixes.
 *   orc_count_prefixes      per-prefix solution and node counts, threaded with
 *                           dynamic pulling of prefixes by the worker threads.
 *                           Pinned by sum of weight x count = Q(N) (OEIS),
 *                           refinement (a prefix's count and nodes are its
 *                           children's sums) and mirror invariance.
 * Parity unpinned: Q(27) (the paper's printed total) is never recomputed.
 *
 * Node: one successful queen placement in a row at or below the prefix depth
 * (rows d..N-1). It does not depend on the order of traversal.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *   - "first half" of row 0 (Section 1) = columns 0 .. floor(N/2)-1, weight 2;
 *   - odd N: the queen in the centre column m = floor(N/2) of row 0 with the
 *     row-1 queen restricted to columns 0 .. m-2 (the footnote's N/2 - 1
 *     positions), weight 2; with d = 1 the centre prefix has weight 1;
 *   - d = 0 is the single empty prefix with weight 1;
 *   - canonical order: depth-first, rows top-down, columns increasing at every
 *     row, the centre branch of row 0 after columns 0 .. m-1.
 *
 * Counts are kept in unsigned __int128 and returned as (lo, hi) halves.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORC_MAXN 31

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ECAP = -3 };

/* ---------------------------------------------------------------------- */
/* Board: columns, diagonals (r + c), anti-diagonals (r - c + N - 1).       */
/* ---------------------------------------------------------------------- */
typedef struct {
    int n;
    unsigned char col[ORC_MAXN];
    unsigned char dg[2 * ORC_MAXN];
    unsigned char ad[2 * ORC_MAXN];
} board_t;

static void board_init(board_t *b, int n)
{
    memset(b, 0, sizeof(*b));
    b->n = n;
}

static int board_free(const board_t *b, int r, int c)
{
    return !b->col[c] && !b->dg[r + c] && !b->ad[r - c + b->n - 1];
}

static void board_set(board_t *b, int r, int c, unsigned char v)
{
    b->col[c] = v;
    b->dg[r + c] = v;
    b->ad[r - c + b->n - 1] = v;
}

/* ---------------------------------------------------------------------- */
/* Brute force: every permutation, then the pairwise attack test.           */
/* fixed[r] >= 0 forces s(r) = fixed[r]; NULL means no constraint.          */
/* ---------------------------------------------------------------------- */
static int perm_ok(const int *s, int n)
{
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            int dc = s[i] - s[j];
            if (dc < 0) dc = -dc;
            if (dc == j - i) return 0;
        }
    return 1;
}

static void perm_rec(int *s, unsigned char *used, int i, int n,
                     const int *fixed, uint64_t *count)
{
    if (i == n) {
        if (perm_ok(s, n)) (*count)++;
        return;
    }
    for (int c = 0; c < n; c++) {
        if (used[c]) continue;
        if (fixed && fixed[i] >= 0 && fixed[i] != c) continue;
        used[c] = 1;
        s[i] = c;
        perm_rec(s, used, i + 1, n, fixed, count);
        used[c] = 0;
    }
}

/* Number of permutations of {0..N-1} with no two entries on a diagonal.
 * N <= 12 (12! = 4.8e8 leaves is the practical ceiling). */
int orc_brute_perm(int n, const int *fixed, uint64_t *count)
{
    if (n < 0 || n > 12 || !count) return ORC_EINVAL;
    int s[ORC_MAXN];
    unsigned char used[ORC_MAXN] = {0};
    *count = 0;
    if (n == 0) {
        *count = 1; /* the empty permutation */
        return ORC_OK;
    }
    perm_rec(s, used, 0, n, fixed, count);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Backtracker: rows top-down, every free column tried in increasing order. */
/* fixed[r] >= 0 means row r may only take column fixed[r].                 */
/* ---------------------------------------------------------------------- */
typedef struct {
    u128 count;
    u128 nodes;
} tally_t;

static void bt(board_t *b, int r, const int *fixed, tally_t *t)
{
    if (r == b->n) {
        t->count++;
        return;
    }
    for (int c = 0; c < b->n; c++) {
        if (fixed && fixed[r] >= 0 && fixed[r] != c) continue;
        if (!board_free(b, r, c)) continue;
        board_set(b, r, c, 1);
        t->nodes++;
        bt(b, r + 1, fixed, t);
        board_set(b, r, c, 0);
    }
}

static void put128(u128 v, uint64_t *out)
{
    if (!out) return;
    out[0] = (uint64_t)v;
    out[1] = (uint64_t)(v >> 64);
}

/* Q(N) with no symmetry reduction; nodes = placements in rows 0..N-1. */
int orc_total(int n, uint64_t *count, uint64_t *nodes)
{
    if (n < 0 || n > ORC_MAXN) return ORC_EINVAL;
    board_t b;
    board_init(&b, n);
    tally_t t = {0, 0};
    bt(&b, 0, NULL, &t);
    put128(t.count, count);
    put128(t.nodes, nodes);
    return ORC_OK;
}

/* Solutions that contain every listed queen (rows[i], cols[i]).
 * A coordinate outside 0..N-1 is an error. The same cell listed twice counts
 * once. Two different cells in one row, or two listed queens that attack each
 * other, give a count of 0 (no solution contains both). nodes counts the
 * placements the backtracker makes in rows 0..N-1, fixed rows included. */
int orc_count_constrained(int n, const int *rows, const int *cols, int k,
                          uint64_t *count, uint64_t *nodes)
{
    if (n < 1 || n > ORC_MAXN || k < 0 || (k > 0 && (!rows || !cols)))
        return ORC_EINVAL;
    int fixed[ORC_MAXN];
    for (int r = 0; r < n; r++) fixed[r] = -1;
    int conflict = 0;
    for (int i = 0; i < k; i++) {
        if (rows[i] < 0 || rows[i] >= n || cols[i] < 0 || cols[i] >= n)
            return ORC_EINVAL;
    }
    for (int i = 0; i < k; i++) {
        int r = rows[i], c = cols[i];
        if (fixed[r] >= 0 && fixed[r] != c) conflict = 1;
        fixed[r] = c;
    }
    /* attacks between listed queens in different rows */
    for (int i = 0; i < n && !conflict; i++) {
        if (fixed[i] < 0) continue;
        for (int j = i + 1; j < n; j++) {
            if (fixed[j] < 0) continue;
            int dc = fixed[i] - fixed[j];
            if (dc < 0) dc = -dc;
            if (dc == 0 || dc == j - i) conflict = 1;
        }
    }
    tally_t t = {0, 0};
    if (!conflict) {
        board_t b;
        board_init(&b, n);
        bt(&b, 0, fixed, &t);
    }
    put128(t.count, count);
    put128(t.nodes, nodes);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Symmetric prefix set (Section 1, Section 2): queens pre-placed in rows   */
/* 0..d-1, first-row half symmetry, odd-N centre rule. Emitted depth-first, */
/* columns increasing at every row.                                         */
/* ---------------------------------------------------------------------- */

/* Columns row r may take in the prefix, given the row-0 column (for the
 * centre rule). Returns [lo, hi). */
static void prefix_row_range(int n, int d, int r, int col0, int *lo, int *hi)
{
    int m = n / 2;
    *lo = 0;
    *hi = n;
    if (r == 0) {
        /* columns 0..m-1, plus the centre column m when N is odd */
        *hi = (n & 1) ? m + 1 : m;
    } else if (r == 1 && (n & 1) && col0 == m && d >= 2) {
        /* centre queen in row 0: row 1 keeps the left side only */
        *hi = m - 1 > 0 ? m - 1 : 0;
    }
}

static int prefix_weight(int n, int d, int col0)
{
    if (d == 0) return 1;
    if ((n & 1) && col0 == n / 2 && d == 1) return 1;
    return 2;
}

typedef struct {
    int n, d;
    int8_t *cols_out;   /* n_out x d, may be NULL (count only) */
    uint8_t *w_out;     /* may be NULL */
    uint64_t cap;
    uint64_t emitted;
    int q[ORC_MAXN];
    board_t b;
} penum_t;

static void penum_rec(penum_t *e, int r)
{
    if (r == e->d) {
        if (e->cols_out && e->emitted < e->cap) {
            for (int i = 0; i < e->d; i++)
                e->cols_out[e->emitted * (uint64_t)e->d + i] = (int8_t)e->q[i];
            if (e->w_out)
                e->w_out[e->emitted] =
                    (uint8_t)prefix_weight(e->n, e->d, e->d ? e->q[0] : -1);
        }
        e->emitted++;
        return;
    }
    int lo, hi;
    prefix_row_range(e->n, e->d, r, r > 0 ? e->q[0] : -1, &lo, &hi);
    for (int c = lo; c < hi; c++) {
        if (!board_free(&e->b, r, c)) continue;
        board_set(&e->b, r, c, 1);
        e->q[r] = c;
        penum_rec(e, r + 1);
        board_set(&e->b, r, c, 0);
    }
}

/* Materialise the prefix set. cols_out: n_out x d int8 column lists (row-major),
 * w_out: weights. If cols_out is NULL only *n_out is set. If more than cap
 * prefixes exist, the first cap are written and ORC_ECAP is returned with the
 * true size in *n_out. */
int orc_prefixes(int n, int d, int8_t *cols_out, uint8_t *w_out, uint64_t cap,
                 uint64_t *n_out)
{
    if (n < 1 || n > ORC_MAXN || d < 0 || d > n || !n_out) return ORC_EINVAL;
    penum_t *e = (penum_t *)calloc(1, sizeof(penum_t));
    if (!e) return ORC_ENOMEM;
    e->n = n;
    e->d = d;
    e->cols_out = cols_out;
    e->w_out = w_out;
    e->cap = cols_out ? cap : 0;
    board_init(&e->b, n);
    penum_rec(e, 0);
    *n_out = e->emitted;
    int rc = (cols_out && e->emitted > cap) ? ORC_ECAP : ORC_OK;
    free(e);
    return rc;
}

/* Size of the prefix set, and the sum of its weights. */
int orc_prefix_count(int n, int d, uint64_t *n_out)
{
    return orc_prefixes(n, d, NULL, NULL, 0, n_out);
}

/* ---------------------------------------------------------------------- */
/* Unranking: the prefixes with given canonical indices.                    */
/*                                                                          */
/* Step 1: enumerate the depth-t nodes of the prefix tree (t = d - 3, or 0) */
/*   in canonical order and, for each, the number of depth-d prefixes below */
/*   it (by enumerating its depth-(d-1) descendants and counting the free   */
/*   cells of row d-1). Running sums of those numbers give the first rank   */
/*   below every depth-t node.                                              */
/* Step 2: for each rank, binary-search the depth-t node that holds it and  */
/*   enumerate that node's depth-d prefixes in order up to the wanted one.  */
/* ---------------------------------------------------------------------- */
typedef struct {
    int n, d, t;
    uint64_t nnodes, cap;
    int8_t *node_cols;   /* nnodes x t */
    uint64_t *first;     /* nnodes + 1 running sums */
    int q[ORC_MAXN];
    board_t b;
} rtab_t;

static void rtab_nodes(rtab_t *x, int r)
{
    if (r == x->t) {
        if (x->node_cols && x->nnodes < x->cap)
            for (int i = 0; i < x->t; i++)
                x->node_cols[x->nnodes * (uint64_t)x->t + i] = (int8_t)x->q[i];
        x->nnodes++;
        return;
    }
    int lo, hi;
    prefix_row_range(x->n, x->d, r, r > 0 ? x->q[0] : -1, &lo, &hi);
    for (int c = lo; c < hi; c++) {
        if (!board_free(&x->b, r, c)) continue;
        board_set(&x->b, r, c, 1);
        x->q[r] = c;
        rtab_nodes(x, r + 1);
        board_set(&x->b, r, c, 0);
    }
}

/* Depth-d prefixes below the placement held in (b, q) rows 0..r-1. When
 * want != NULL, stop at the (*want)-th one (0-based), copy it to q and
 * return 1; otherwise return the count. */
static uint64_t below(int n, int d, board_t *b, int *q, int r, uint64_t *want)
{
    if (r == d) {
        if (want) {
            if (*want == 0) return 1;
            (*want)--;
            return 0;
        }
        return 1;
    }
    uint64_t total = 0;
    int lo, hi;
    prefix_row_range(n, d, r, r > 0 ? q[0] : -1, &lo, &hi);
    for (int c = lo; c < hi; c++) {
        if (!board_free(b, r, c)) continue;
        board_set(b, r, c, 1);
        q[r] = c;
        uint64_t got = below(n, d, b, q, r + 1, want);
        board_set(b, r, c, 0);
        if (want && got) {
            board_set(b, r, c, 1); /* leave the found path placed */
            return 1;
        }
        total += got;
    }
    return want ? 0 : total;
}

typedef struct {
    rtab_t *x;
    uint64_t next;
} rjob_t;

static void *rtab_worker(void *arg)
{
    rjob_t *j = (rjob_t *)arg;
    rtab_t *x = j->x;
    for (;;) {
        uint64_t i = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
        if (i >= x->nnodes) break;
        board_t b;
        int q[ORC_MAXN];
        board_init(&b, x->n);
        for (int r = 0; r < x->t; r++) {
            q[r] = x->node_cols[i * (uint64_t)x->t + r];
            board_set(&b, r, q[r], 1);
        }
        x->first[i + 1] = below(x->n, x->d, &b, q, x->t, NULL);
    }
    return NULL;
}

/* out_cols: k x d. Returns ORC_EINVAL if some rank is not below the size of
 * the prefix set (that row of out_cols is then filled with -1). */
int orc_prefixes_at_ranks(int n, int d, const uint64_t *ranks, uint64_t k,
                          int8_t *out_cols, int threads)
{
    if (n < 1 || n > ORC_MAXN || d < 0 || d > n || (k && (!ranks || !out_cols)))
        return ORC_EINVAL;
    if (threads < 1) threads = 1;
    if (threads > 1024) threads = 1024;
    rtab_t *x = (rtab_t *)calloc(1, sizeof(rtab_t));
    if (!x) return ORC_ENOMEM;
    x->n = n;
    x->d = d;
    x->t = d > 3 ? d - 3 : 0;
    board_init(&x->b, n);
    rtab_nodes(x, 0); /* count */
    x->cap = x->nnodes;
    x->node_cols = (int8_t *)malloc(x->cap * (uint64_t)(x->t ? x->t : 1));
    x->first = (uint64_t *)calloc(x->cap + 1, sizeof(uint64_t));
    if (!x->node_cols || !x->first) {
        free(x->node_cols);
        free(x->first);
        free(x);
        return ORC_ENOMEM;
    }
    x->nnodes = 0;
    board_init(&x->b, n);
    rtab_nodes(x, 0); /* fill */

    rjob_t j = {x, 0};
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    int started = 0;
    for (int t = 1; th && t < threads; t++) {
        if (pthread_create(&th[t], NULL, rtab_worker, &j) != 0) break;
        started++;
    }
    rtab_worker(&j);
    for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
    free(th);
    for (uint64_t i = 0; i < x->nnodes; i++) x->first[i + 1] += x->first[i];

    int rc = ORC_OK;
    for (uint64_t s = 0; s < k; s++) {
        uint64_t rank = ranks[s];
        int8_t *out = out_cols + s * (uint64_t)d;
        if (rank >= x->first[x->nnodes]) {
            for (int i = 0; i < d; i++) out[i] = -1;
            rc = ORC_EINVAL;
            continue;
        }
        /* last node whose first rank is <= rank */
        uint64_t lo = 0, hi = x->nnodes; /* first[lo] <= rank < first[hi] */
        while (hi - lo > 1) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (x->first[mid] <= rank) lo = mid; else hi = mid;
        }
        board_t b;
        int q[ORC_MAXN];
        board_init(&b, n);
        for (int r = 0; r < x->t; r++) {
            q[r] = x->node_cols[lo * (uint64_t)x->t + r];
            board_set(&b, r, q[r], 1);
        }
        uint64_t want = rank - x->first[lo];
        below(n, d, &b, q, x->t, &want);
        for (int i = 0; i < d; i++) out[i] = (int8_t)q[i];
    }
    free(x->node_cols);
    free(x->first);
    free(x);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Per-prefix counts: each prefix's queens are placed on a fresh board and  */
/* the backtracker runs rows d..N-1. Worker threads pull prefix indices     */
/* from a shared atomic counter.                                            */
/* ---------------------------------------------------------------------- */
typedef struct {
    int n, d;
    const int8_t *cols;
    uint64_t np;
    uint64_t *counts;  /* np, may be NULL */
    uint64_t *nodes;   /* np, may be NULL */
    uint64_t next;     /* shared cursor */
    int bad;           /* a prefix whose queens attack each other */
} pjob_t;

static int prefix_place(board_t *b, const int8_t *q, int d)
{
    for (int r = 0; r < d; r++) {
        int c = q[r];
        if (c < 0 || c >= b->n || !board_free(b, r, c)) return 0;
        board_set(b, r, c, 1);
    }
    return 1;
}

static void *pjob_worker(void *arg)
{
    pjob_t *j = (pjob_t *)arg;
    for (;;) {
        uint64_t i = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
        if (i >= j->np) break;
        board_t b;
        board_init(&b, j->n);
        tally_t t = {0, 0};
        if (prefix_place(&b, j->cols + i * (uint64_t)j->d, j->d))
            bt(&b, j->d, NULL, &t);
        else
            __atomic_store_n(&j->bad, 1, __ATOMIC_RELAXED);
        /* a single subtree of N <= 31 stays far below 2^64 leaves for any
           prefix depth the callers use; the caller checks the totals */
        if (j->counts) j->counts[i] = (uint64_t)t.count;
        if (j->nodes) j->nodes[i] = (uint64_t)t.nodes;
    }
    return NULL;
}

/* threads <= 0 means one. Returns ORC_EINVAL if any prefix is not a valid
 * placement (its count is then 0). */
int orc_count_prefixes(int n, int d, const int8_t *cols, uint64_t np,
                       uint64_t *counts, uint64_t *nodes, int threads)
{
    if (n < 1 || n > ORC_MAXN || d < 0 || d > n || (np && !cols))
        return ORC_EINVAL;
    if (threads < 1) threads = 1;
    if (threads > 1024) threads = 1024;
    pjob_t j = {n, d, cols, np, counts, nodes, 0, 0};
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!th) return ORC_ENOMEM;
    int started = 0;
    for (int t = 1; t < threads; t++) {
        if (pthread_create(&th[t], NULL, pjob_worker, &j) != 0) break;
        started++;
    }
    pjob_worker(&j);
    for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
    free(th);
    return j.bad ? ORC_EINVAL : ORC_OK;
}
