/*
 * md_oracle.c -- the CPU oracle for the minimum distance of a binary linear code.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct statement
 * of what the GPU library computes.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it.  It shares no code, header,
 * table or helper with the CUDA library, and includes nothing from it.
 *
 * What it computes (Quintana-Orti, Hernando, Igual, "Parallel implementations for
 * computing the minimum distance of a random linear code on multicomputers"):
 *
 *   - mdo_bruteforce: the definition of Section 2.1: d(C) = min{ wt(xG) : x != 0 },
 *     walking all 2^k - 1 nonzero messages (binary reflected Gray code, so that each step
 *     adds one row of G), with the whole weight distribution as a by-product.
 *   - mdo_info_sets / mdo_gamma: the disjoint information sets S_1..S_m and the
 *     systematic matrices Gamma_j of Section 2.1 (Gamma_j = (I_k | A_j) for a full set,
 *     Gamma_m = [[I_{k_m}, A], [0, B]] for the leftover columns), by greedy pivoting and
 *     Gauss-Jordan elimination.
 *   - mdo_scan: "Process_combination" of Section 2.2.1 (Alg. 2) over a range of
 *     combinations: every g-subset c of the k rows, in colexicographic ("left-
 *     lexicographical", Section 3.1) order, the weight of the full n-bit sum of the rows c.
 *   - mdo_bz: the Brouwer-Zimmermann loop of Alg. 1: for g = 1, 2, ... and for each
 *     Gamma_j, U := min(U, min wt(c Gamma_j) over wt(c) = g); the bounds are checked after
 *     each Gamma matrix (Section 2.2); after each stage L := sum_j max(0, g+1-(k-k_j)).
 *
 * Readings where the paper is silent (the same ones the library documents):
 *   - U starts as "no codeword found" rather than n-k+1, so that a witness always exists;
 *     the run stops when L >= U for the best weight U actually found.
 *   - The witness is the first codeword of weight d in (g, j, colex rank) order.
 *   - Information sets: greedy pivots over the unused columns in ascending order; the
 *     leftover columns form the last, rank-deficient set; Gamma_j is the reduced row
 *     echelon form of G under the column order (S_j ascending, then the others ascending).
 *   - Rows are packed as uint64 words, bit t of word w is column 64w + t.
 *
 * Nothing here is blocked, fused or reordered: each codeword is formed from scratch by
 * adding its g rows, and its weight is the popcount of all n bits.  The optional threads
 * of mdo_scan only split a level into contiguous colex-rank ranges (the shared-memory
 * parallelisation of Section 2.2.2); the lexicographic minimum of (weight, rank) over the
 * ranges equals the sequential result.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define MDO_MAXN 256
#define MDO_MAXW (MDO_MAXN / 64)

enum { MDO_OK = 0, MDO_EINVAL = -1, MDO_ERANK = -2, MDO_ETOOBIG = -3, MDO_ENOMEM = -4 };

static int words_for(int n) { return (n + 63) / 64; }

static int get_bit(const uint64_t *row, int col) { return (int)((row[col / 64] >> (col % 64)) & 1u); }

static int popcount_row(const uint64_t *row, int nw) {
    int w = 0;
    for (int i = 0; i < nw; i++) w += __builtin_popcountll(row[i]);
    return w;
}

static void xor_row(uint64_t *dst, const uint64_t *src, int nw) {
    for (int i = 0; i < nw; i++) dst[i] ^= src[i];
}

/* Binomial coefficient C(a, b), saturating at UINT64_MAX. */
uint64_t mdo_binomial(int a, int b) {
    if (b < 0 || a < 0 || b > a) return 0;
    if (b > a - b) b = a - b;
    unsigned __int128 r = 1;
    for (int i = 1; i <= b; i++) {
        /* after step i, r = C(a - b + i, i): the division is exact; the 128-bit
           product cannot overflow while r itself fits in 64 bits */
        r = r * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
        if (r > (unsigned __int128)UINT64_MAX) return UINT64_MAX;
    }
    return (uint64_t)r;
}

/* ---------------------------------------------------------------- colex order ---- */

/* Colex rank of c[0] < ... < c[g-1]: sum_i C(c[i], i+1). */
uint64_t mdo_colex_rank(const int *c, int g) {
    uint64_t r = 0;
    for (int i = 0; i < g; i++) r += mdo_binomial(c[i], i + 1);
    return r;
}

/* Colex successor inside {0..k-1}: the left-most element moves fastest (Section 3.1).
   Returns 1 and updates c, or 0 if c was the last combination. */
int mdo_colex_next(int *c, int g, int k) {
    for (int i = 0; i < g; i++) {
        int limit = (i + 1 < g) ? c[i + 1] : k;
        if (c[i] + 1 < limit) {
            c[i] += 1;
            for (int t = 0; t < i; t++) c[t] = t;
            return 1;
        }
    }
    return 0;
}

/* Inverse of mdo_colex_rank: the g-subset of {0..k-1} with the given colex rank. */
int mdo_colex_unrank(uint64_t rank, int g, int k, int *c) {
    if (g < 0 || g > k) return MDO_EINVAL;
    if (rank >= mdo_binomial(k, g)) return MDO_EINVAL;
    int top = k - 1;
    for (int i = g; i >= 1; i--) {
        int v = top;
        while (mdo_binomial(v, i) > rank) v--;
        c[i - 1] = v;
        rank -= mdo_binomial(v, i);
        top = v - 1;
    }
    return MDO_OK;
}

/* ------------------------------------------------------------- linear algebra ---- */

/* Rank over F2 of the k x n matrix G. */
int mdo_rank(const uint64_t *G, int n, int k) {
    if (!G || n < 1 || k < 1 || n > MDO_MAXN) return MDO_EINVAL;
    int nw = words_for(n);
    uint64_t *A = (uint64_t *)malloc((size_t)k * nw * sizeof(uint64_t));
    if (!A) return MDO_ENOMEM;
    memcpy(A, G, (size_t)k * nw * sizeof(uint64_t));
    int r = 0;
    for (int col = 0; col < n && r < k; col++) {
        int s = -1;
        for (int t = r; t < k; t++)
            if (get_bit(A + (size_t)t * nw, col)) { s = t; break; }
        if (s < 0) continue;
        for (int w = 0; w < nw; w++) { uint64_t x = A[(size_t)s * nw + w]; A[(size_t)s * nw + w] = A[(size_t)r * nw + w]; A[(size_t)r * nw + w] = x; }
        for (int t = 0; t < k; t++)
            if (t != r && get_bit(A + (size_t)t * nw, col)) xor_row(A + (size_t)t * nw, A + (size_t)r * nw, nw);
        r++;
    }
    free(A);
    return r;
}

/* Gauss-Jordan elimination of G with the columns visited in the given order.
   Writes the reduced row echelon form (columns in their original positions) to Gam
   and returns the number of pivots. */
int mdo_gamma(const uint64_t *G, int n, int k, const int *order, uint64_t *Gam) {
    if (!G || !order || !Gam || n < 1 || k < 1 || n > MDO_MAXN) return MDO_EINVAL;
    int nw = words_for(n);
    memcpy(Gam, G, (size_t)k * nw * sizeof(uint64_t));
    int r = 0;
    for (int p = 0; p < n && r < k; p++) {
        int col = order[p];
        int s = -1;
        for (int t = r; t < k; t++)
            if (get_bit(Gam + (size_t)t * nw, col)) { s = t; break; }
        if (s < 0) continue;
        for (int w = 0; w < nw; w++) { uint64_t x = Gam[(size_t)s * nw + w]; Gam[(size_t)s * nw + w] = Gam[(size_t)r * nw + w]; Gam[(size_t)r * nw + w] = x; }
        for (int t = 0; t < k; t++)
            if (t != r && get_bit(Gam + (size_t)t * nw, col)) xor_row(Gam + (size_t)t * nw, Gam + (size_t)r * nw, nw);
        r++;
    }
    return r;
}

/* Disjoint information sets (Section 2.1).  For j = 0, 1, ...: scan the still-unused
   columns in ascending order and keep each one that raises the rank; if k columns are
   kept they form S_j.  Otherwise the leftover columns, all of them, form the last set,
   whose rank k_m (< k) is the number of kept columns; it is dropped when k_m = 0.
   orders: m rows of n ints, the column order under which Gamma_j is reduced
   (the set's columns ascending, then every other column ascending).
   ranks: k_j per set.  Returns m (>= 1) or an error. */
int mdo_info_sets(const uint64_t *G, int n, int k, int *orders, int *ranks) {
    if (!G || !orders || !ranks || n < 1 || k < 1 || k > n || n > MDO_MAXN) return MDO_EINVAL;
    int nw = words_for(n);
    if (mdo_rank(G, n, k) != k) return MDO_ERANK;
    int used[MDO_MAXN];
    memset(used, 0, sizeof(used));
    uint64_t *A = (uint64_t *)malloc((size_t)k * nw * sizeof(uint64_t));
    if (!A) return MDO_ENOMEM;
    int m = 0;
    for (;;) {
        int remaining[MDO_MAXN], nrem = 0;
        for (int col = 0; col < n; col++) if (!used[col]) remaining[nrem++] = col;
        if (nrem == 0) break;
        memcpy(A, G, (size_t)k * nw * sizeof(uint64_t));
        int kept[MDO_MAXN], r = 0;
        for (int q = 0; q < nrem && r < k; q++) {
            int col = remaining[q];
            int s = -1;
            for (int t = r; t < k; t++)
                if (get_bit(A + (size_t)t * nw, col)) { s = t; break; }
            if (s < 0) continue;
            for (int w = 0; w < nw; w++) { uint64_t x = A[(size_t)s * nw + w]; A[(size_t)s * nw + w] = A[(size_t)r * nw + w]; A[(size_t)r * nw + w] = x; }
            for (int t = 0; t < k; t++)
                if (t != r && get_bit(A + (size_t)t * nw, col)) xor_row(A + (size_t)t * nw, A + (size_t)r * nw, nw);
            kept[r++] = col;
        }
        int *order = orders + (size_t)m * n;
        int in_set[MDO_MAXN];
        memset(in_set, 0, sizeof(in_set));
        int pos = 0;
        if (r == k) {
            for (int q = 0; q < k; q++) { order[pos++] = kept[q]; in_set[kept[q]] = 1; used[kept[q]] = 1; }
            for (int col = 0; col < n; col++) if (!in_set[col]) order[pos++] = col;
            ranks[m++] = k;
            continue;
        }
        if (r > 0) {
            for (int q = 0; q < nrem; q++) { order[pos++] = remaining[q]; in_set[remaining[q]] = 1; }
            for (int col = 0; col < n; col++) if (!in_set[col]) order[pos++] = col;
            ranks[m++] = r;
        }
        break;
    }
    free(A);
    return m;
}

/* ------------------------------------------------------------ brute force ---------- */

typedef struct {
    const uint64_t *G; int n, k, nw;
    uint64_t lo, hi;          /* message indices i in [lo, hi), message = i ^ (i >> 1) */
    uint64_t dist[MDO_MAXN + 1];
} bf_job;

static void *bf_worker(void *arg) {
    bf_job *J = (bf_job *)arg;
    uint64_t acc[MDO_MAXW];
    memset(acc, 0, sizeof(acc));
    uint64_t x = J->lo ^ (J->lo >> 1);
    for (int b = 0; b < J->k; b++)
        if ((x >> b) & 1u) xor_row(acc, J->G + (size_t)b * J->nw, J->nw);
    J->dist[popcount_row(acc, J->nw)] += 1;
    for (uint64_t i = J->lo + 1; i < J->hi; i++) {
        int b = __builtin_ctzll(i);            /* Gray code: message i differs from i-1 in bit b */
        xor_row(acc, J->G + (size_t)b * J->nw, J->nw);
        J->dist[popcount_row(acc, J->nw)] += 1;
    }
    return NULL;
}

/* Weight distribution of all 2^k codewords xG (x = 0 included) into dist[0..n];
   returns d = the least weight of xG over x != 0 (0 if G is rank deficient). */
int mdo_bruteforce(const uint64_t *G, int n, int k, int nthreads, uint64_t *dist) {
    if (!G || !dist || n < 1 || k < 1 || k > 40 || n > MDO_MAXN) return MDO_EINVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int nw = words_for(n);
    uint64_t total = (uint64_t)1 << k;
    if ((uint64_t)nthreads > total) nthreads = (int)total;
    bf_job *jobs = (bf_job *)calloc((size_t)nthreads, sizeof(bf_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return MDO_ENOMEM; }
    for (int t = 0; t < nthreads; t++) {
        jobs[t].G = G; jobs[t].n = n; jobs[t].k = k; jobs[t].nw = nw;
        jobs[t].lo = total / nthreads * t + (t < (int)(total % nthreads) ? t : total % nthreads);
        jobs[t].hi = jobs[t].lo + total / nthreads + (t < (int)(total % nthreads) ? 1 : 0);
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&tid[t], NULL, bf_worker, &jobs[t]);
    bf_worker(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(tid[t], NULL);
    for (int w = 0; w <= n; w++) {
        dist[w] = 0;
        for (int t = 0; t < nthreads; t++) dist[w] += jobs[t].dist[w];
    }
    free(jobs); free(tid);
    /* the zero message gives weight 0; any further weight-0 codeword means rank < k */
    if (dist[0] > 1) return 0;
    for (int w = 1; w <= n; w++) if (dist[w]) return w;
    return 0;
}

/* ------------------------------------------------------- combination scanning ------ */

typedef struct {
    const uint64_t *Gam; int n, k, g, nw;
    uint64_t r0, r1;
    int minw; uint64_t first;
} scan_job;

static void *scan_worker(void *arg) {
    scan_job *J = (scan_job *)arg;
    J->minw = J->n + 1;
    J->first = UINT64_MAX;
    if (J->r0 >= J->r1) return NULL;
    int c[MDO_MAXN];
    mdo_colex_unrank(J->r0, J->g, J->k, c);
    uint64_t rank = J->r0;
    for (;;) {
        /* Process_combination: add the g rows of c, count the weight of the sum */
        uint64_t acc[MDO_MAXW];
        memset(acc, 0, sizeof(acc));
        for (int i = 0; i < J->g; i++) xor_row(acc, J->Gam + (size_t)c[i] * J->nw, J->nw);
        int w = popcount_row(acc, J->nw);
        if (w < J->minw) { J->minw = w; J->first = rank; }
        rank++;
        if (rank >= J->r1) break;
        mdo_colex_next(c, J->g, J->k);
    }
    return NULL;
}

/* Least weight over the colex ranks [r0, r1) of the g-subsets of the k rows of Gam, and
   the first rank reaching it.  Returns MDO_OK; *minw = n + 1 when the range is empty. */
int mdo_scan(const uint64_t *Gam, int n, int k, int g, uint64_t r0, uint64_t r1, int nthreads,
             int *minw, uint64_t *first) {
    if (!Gam || !minw || !first || n < 1 || k < 1 || n > MDO_MAXN || g < 1 || g > k) return MDO_EINVAL;
    uint64_t total = mdo_binomial(k, g);
    if (total == UINT64_MAX) return MDO_ETOOBIG;
    if (r1 > total) r1 = total;
    if (r0 > r1) r0 = r1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    uint64_t span = r1 - r0;
    if ((uint64_t)nthreads > span && span > 0) nthreads = (int)span;
    scan_job *jobs = (scan_job *)calloc((size_t)nthreads, sizeof(scan_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return MDO_ENOMEM; }
    for (int t = 0; t < nthreads; t++) {
        jobs[t].Gam = Gam; jobs[t].n = n; jobs[t].k = k; jobs[t].g = g; jobs[t].nw = words_for(n);
        jobs[t].r0 = r0 + span / nthreads * t + ((uint64_t)t < span % nthreads ? (uint64_t)t : span % nthreads);
        jobs[t].r1 = jobs[t].r0 + span / nthreads + ((uint64_t)t < span % nthreads ? 1 : 0);
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&tid[t], NULL, scan_worker, &jobs[t]);
    scan_worker(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(tid[t], NULL);
    int bw = n + 1; uint64_t br = UINT64_MAX;
    for (int t = 0; t < nthreads; t++)   /* ranges ascend with t: lexicographic min of (w, rank) */
        if (jobs[t].minw < bw) { bw = jobs[t].minw; br = jobs[t].first; }
    *minw = bw; *first = br;
    free(jobs); free(tid);
    return MDO_OK;
}

/* ----------------------------------------------------------- Brouwer-Zimmermann ---- */

/* Indices of the scalar outputs of mdo_bz. */
enum {
    MDO_OUT_D = 0,        /* minimum distance d */
    MDO_OUT_KEY_G,        /* witness key: stage g */
    MDO_OUT_KEY_J,        /* witness key: matrix index j (0-based) */
    MDO_OUT_KEY_RANK,     /* witness key: colex rank of the combination */
    MDO_OUT_L,            /* lower bound L when the loop stopped */
    MDO_OUT_M,            /* number of Gamma matrices */
    MDO_OUT_STOP_G,       /* stage of the last level processed */
    MDO_OUT_STOP_J,       /* matrix of the last level processed */
    MDO_OUT_CODEWORDS,    /* combinations evaluated in total */
    MDO_OUT_NLEVELS,      /* number of levels processed */
    MDO_OUT_COUNT
};

/* Bound from information set j after its combinations of weight <= g are all seen:
   every codeword not seen has at least max(0, g + 1 - (k - k_j)) nonzeros on S_j. */
static int64_t set_bound(int g, int k, int kj) {
    int64_t t = (int64_t)g + 1 - (k - kj);
    return t > 0 ? t : 0;
}

/* Plain Brouwer-Zimmermann (Alg. 1 with the per-matrix check of Section 2.2).
   out: MDO_OUT_COUNT int64 values (see the enum).  witness: nw words.
   levels: per processed level (g, j, min weight, first rank of that weight, count),
   5 int64 each, at most maxlev levels.  stop_after_g > 0 truncates the run after that
   stage (used for bounded samples); 0 runs to the end.
   stop_rule 0: Alg. 1 -- after each Gamma matrix compare with the L of the last complete
   stage, after each stage L := sum_j max(0, g+1-(k-k_j)).  stop_rule 1: the sharper bound
   after matrix j of stage g, sum_{i<=j} bound_i(g) + sum_{i>j} bound_i(g-1) (the matrices
   after j have only completed stage g-1); d and the witness are the same, fewer levels run.
   Returns MDO_OK, or an error if G is invalid or a level exceeds 2^63 combinations. */
int mdo_bz(const uint64_t *G, int n, int k, int nthreads, int stop_after_g, int stop_rule,
           int64_t *out, uint64_t *witness, int64_t *levels, int maxlev) {
    if (!G || !out || !witness || n < 1 || k < 1 || k > n || n > MDO_MAXN) return MDO_EINVAL;
    int nw = words_for(n);
    int *orders = (int *)malloc((size_t)n * n * sizeof(int));
    int ranks[MDO_MAXN];
    if (!orders) return MDO_ENOMEM;
    int m = mdo_info_sets(G, n, k, orders, ranks);
    if (m < 0) { free(orders); return m; }
    uint64_t *Gam = (uint64_t *)malloc((size_t)m * k * nw * sizeof(uint64_t));
    if (!Gam) { free(orders); return MDO_ENOMEM; }
    for (int j = 0; j < m; j++) mdo_gamma(G, n, k, orders + (size_t)j * n, Gam + (size_t)j * k * nw);

    int64_t L = 1;
    int U = n + 1;                 /* n + 1 stands for "no codeword found yet" */
    int key_g = 0, key_j = 0; uint64_t key_rank = 0;
    int nlev = 0, last_g = 0, last_j = 0, stop = 0;
    uint64_t evaluated = 0;
    for (int g = 1; g <= k && !stop; g++) {
        uint64_t count = mdo_binomial(k, g);
        if (count >= ((uint64_t)1 << 63)) { free(orders); free(Gam); return MDO_ETOOBIG; }
        for (int j = 0; j < m; j++) {
            int w; uint64_t first;
            mdo_scan(Gam + (size_t)j * k * nw, n, k, g, 0, count, nthreads, &w, &first);
            evaluated += count;
            if (levels && nlev < maxlev) {
                int64_t *rec = levels + (size_t)nlev * 5;
                rec[0] = g; rec[1] = j; rec[2] = w; rec[3] = (int64_t)first; rec[4] = (int64_t)count;
            }
            nlev++;
            last_g = g; last_j = j;
            if (w < U) { U = w; key_g = g; key_j = j; key_rank = first; }
            if (stop_rule == 1) {                       /* bound after matrix j of stage g */
                L = 0;
                for (int i = 0; i < m; i++) L += set_bound(i <= j ? g : g - 1, k, ranks[i]);
            }
            if (L >= U) { stop = 1; break; }          /* checked after each Gamma matrix */
        }
        if (stop) break;
        L = 0;                                          /* L := sum_j max(0, g+1-(k-k_j)) */
        for (int j = 0; j < m; j++) L += set_bound(g, k, ranks[j]);
        if (L >= U) stop = 1;
        if (stop_after_g > 0 && g >= stop_after_g) break;
    }
    int c[MDO_MAXN];
    memset(witness, 0, (size_t)nw * sizeof(uint64_t));
    if (U <= n) {
        mdo_colex_unrank(key_rank, key_g, k, c);
        for (int i = 0; i < key_g; i++) xor_row(witness, Gam + ((size_t)key_j * k + c[i]) * nw, nw);
    }
    out[MDO_OUT_D] = (U <= n) ? U : -1;
    out[MDO_OUT_KEY_G] = key_g;
    out[MDO_OUT_KEY_J] = key_j;
    out[MDO_OUT_KEY_RANK] = (int64_t)key_rank;
    out[MDO_OUT_L] = L;
    out[MDO_OUT_M] = m;
    out[MDO_OUT_STOP_G] = last_g;
    out[MDO_OUT_STOP_J] = last_j;
    out[MDO_OUT_CODEWORDS] = (int64_t)evaluated;
    out[MDO_OUT_NLEVELS] = nlev;
    free(orders); free(Gam);
    return MDO_OK;
}
