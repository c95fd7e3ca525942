/*
 * Oracle for the exact reset threshold of a synchronizing automaton.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU statement of what the GPU library computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the product
 * path never does.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * Everything is exact integer set work: a subset of Q = {0..n-1} is its
 * characteristic vector, stored as W = ceil(n/64) 64-bit words, state q at
 * bit (q mod 64) of word floor(q/64).
 *
 * Automaton input (all functions): delta is int32 [k][n], letter-major:
 * delta[a*n + q] = delta(q, a)  (paper Section 1, the transition function).
 *
 * Functions and the passages they restate:
 *   oracle_brute           Section 1.3.0 ("checking all words of length
 *                          1, 2, ..., r"): enumerate words by length in
 *                          lexicographic order, return the first reset word.
 *   oracle_forward         Section 1.3.1 (the standard algorithm: a path of
 *                          subsets in the power automaton from Q to a
 *                          singleton), run breadth-first with duplicates
 *                          removed and every visited set kept (equality
 *                          history, Section 2.1).
 *   oracle_level_sizes     sizes of the deduplicated BFS (images of Q) or
 *                          IBFS (preimages of singletons) levels, Section 2.1.
 *   oracle_bidir           Alg. 1 (Section 2.1) with only the duplicate
 *                          deletion (lexicographic sort) and an equality
 *                          history; the meet condition X subset of Y
 *                          (Section 2, the meet of the two searches) checked
 *                          by brute force after every step.
 *   oracle_reduced_level_sizes, oracle_bidir_reduced
 *                          Alg. 1 with its inclusion reductions (Section
 *                          2.1): duplicates removed, then the sets that are
 *                          not minimal (BFS) / maximal (IBFS) in their list
 *                          (MarkProperSupersets), then the supersets (BFS) /
 *                          subsets (IBFS) of every set of an earlier level
 *                          (the history); all by brute force over pairs.
 *   oracle_beam            Section 2.1.3: the heuristic upper bound R from
 *                          an inverse BFS that keeps only the `beam`
 *                          largest preimages of every depth (the cut-off
 *                          inverse BFS the paper cites).
 *   oracle_inverse_dfs_r   Section 2.2: r from the last levels F_i, B_j of a
 *                          bidirectional search (plain or with the
 *                          reductions of Alg. 1 on either side) by the
 *                          inverse DFS phase (a depth-first search over
 *                          preimages from every set of B_j, no history,
 *                          each set reached checked against F_i by brute
 *                          force), deepened one step at a time.
 *   oracle_mark_supersets  Alg. 2 (MarkSupersets / MarkProperSupersets,
 *                          Section 2.1.1): the sets of B that contain some
 *                          set of A, by recursive splitting of the sorted
 *                          list A on one state per level, brute force on
 *                          small intervals.
 *   oracle_is_synchronizing  Section 2, first step: every pair of states can
 *                          be mapped to one state.
 *
 * Readings taken where the paper is silent:
 *   - the word returned is the lexicographically least reset word of length
 *     r (letter 0 < letter 1 < ...);
 *   - level i of a direction is the list of distinct sets first reached at
 *     depth i (duplicates and sets of earlier levels removed), kept in
 *     canonical order: by parent position, then by letter;
 *   - empty preimages are dropped (they contain no nonempty set);
 *   - n = 1 gives r = 0 and the empty word.
 *
 * Return codes: 0 ok, -1 bad arguments, -2 more than max_sets sets would be
 * stored, -3 the automaton is not synchronizing (a search ran dry),
 * -4 the word does not fit in word_cap (r is still written), -5 out of host
 * memory, -6 the brute force found no reset word up to max_len.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ETOOBIG (-2)
#define OR_ENOTSYNC (-3)
#define OR_EWORDCAP (-4)
#define OR_ENOMEM (-5)
#define OR_ENOTFOUND (-6)

/* ------------------------------------------------------------------ */
/* Sets as characteristic vectors                                      */
/* ------------------------------------------------------------------ */

static int words_for(int n) { return (n + 63) / 64; }

static void set_clear(uint64_t *s, int W) {
    for (int w = 0; w < W; w++) s[w] = 0;
}

static void set_add(uint64_t *s, int q) { s[q / 64] |= (uint64_t)1 << (q % 64); }

static int set_has(const uint64_t *s, int q) { return (int)((s[q / 64] >> (q % 64)) & 1u); }

static int set_size(const uint64_t *s, int n) {
    int c = 0;
    for (int q = 0; q < n; q++) c += set_has(s, q);
    return c;
}

static int set_first(const uint64_t *s, int n) {
    for (int q = 0; q < n; q++)
        if (set_has(s, q)) return q;
    return -1;
}

/* X subset of Y: no state of X is missing from Y. */
static int set_subset(const uint64_t *x, const uint64_t *y, int n) {
    for (int q = 0; q < n; q++)
        if (set_has(x, q) && !set_has(y, q)) return 0;
    return 1;
}

/* Lexicographic order of characteristic vectors read from state 0 upwards
 * (the order of the paper's duplicate-removal sort, Section 2.1.1). */
static int set_cmp(const uint64_t *a, const uint64_t *b, int n) {
    for (int q = 0; q < n; q++) {
        int x = set_has(a, q), y = set_has(b, q);
        if (x != y) return x - y;
    }
    return 0;
}

/* Image delta(S, a) = { delta(q, a) : q in S }  (Section 2, definition). */
static void set_image(int n, const int32_t *delta_a, const uint64_t *S, uint64_t *T, int W) {
    set_clear(T, W);
    for (int q = 0; q < n; q++)
        if (set_has(S, q)) set_add(T, delta_a[q]);
}

/* Preimage delta^{-1}(S, a) = { q : delta(q, a) in S }  (Section 2). */
static void set_preimage(int n, const int32_t *delta_a, const uint64_t *S, uint64_t *T, int W) {
    set_clear(T, W);
    for (int q = 0; q < n; q++)
        if (set_has(S, delta_a[q])) set_add(T, q);
}

/* ------------------------------------------------------------------ */
/* Lists of sets (one BFS or IBFS level each)                          */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t count, cap;
    uint64_t *sets;   /* count * W words */
    int64_t *parent;  /* position of the parent in the previous level */
    uint8_t *letter;  /* letter applied to the parent */
} level_t;

static int level_reserve(level_t *L, int64_t cap, int W) {
    if (cap <= L->cap) return 0;
    uint64_t *s = (uint64_t *)realloc(L->sets, (size_t)cap * W * sizeof(uint64_t));
    if (!s) return OR_ENOMEM;
    L->sets = s;
    int64_t *p = (int64_t *)realloc(L->parent, (size_t)cap * sizeof(int64_t));
    if (!p) return OR_ENOMEM;
    L->parent = p;
    uint8_t *l = (uint8_t *)realloc(L->letter, (size_t)cap);
    if (!l) return OR_ENOMEM;
    L->letter = l;
    L->cap = cap;
    return 0;
}

static int level_push(level_t *L, const uint64_t *s, int64_t parent, int letter, int W) {
    if (L->count == L->cap) {
        int rc = level_reserve(L, L->cap ? 2 * L->cap : 16, W);
        if (rc) return rc;
    }
    memcpy(L->sets + L->count * W, s, (size_t)W * sizeof(uint64_t));
    L->parent[L->count] = parent;
    L->letter[L->count] = (uint8_t)letter;
    L->count++;
    return 0;
}

static void level_free(level_t *L) {
    free(L->sets);
    free(L->parent);
    free(L->letter);
    memset(L, 0, sizeof(*L));
}

/* A history: every set visited so far in one direction, kept sorted in the
 * lexicographic order so that membership is a binary search. */
typedef struct {
    int64_t count;
    uint64_t *sets;
} history_t;

static int history_contains(const history_t *H, const uint64_t *s, int n, int W) {
    int64_t lo = 0, hi = H->count;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = set_cmp(H->sets + mid * W, s, n);
        if (c == 0) return 1;
        if (c < 0) lo = mid + 1; else hi = mid;
    }
    return 0;
}

/* Stable merge sort of candidate ids by (set, id); plain bottom-up. */
static int cmp_ids(const uint64_t *cand, int64_t a, int64_t b, int n, int W) {
    int c = set_cmp(cand + a * W, cand + b * W, n);
    if (c) return c;
    return (a > b) - (a < b);
}

static int sort_ids(int64_t *ids, int64_t m, const uint64_t *cand, int n, int W) {
    int64_t *tmp = (int64_t *)malloc((size_t)(m ? m : 1) * sizeof(int64_t));
    if (!tmp) return OR_ENOMEM;
    for (int64_t width = 1; width < m; width *= 2) {
        for (int64_t lo = 0; lo < m; lo += 2 * width) {
            int64_t mid = lo + width < m ? lo + width : m;
            int64_t hi = lo + 2 * width < m ? lo + 2 * width : m;
            int64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi)
                tmp[o++] = cmp_ids(cand, ids[i], ids[j], n, W) <= 0 ? ids[i++] : ids[j++];
            while (i < mid) tmp[o++] = ids[i++];
            while (j < hi) tmp[o++] = ids[j++];
        }
        memcpy(ids, tmp, (size_t)m * sizeof(int64_t));
    }
    free(tmp);
    return 0;
}

/*
 * One BFS (dir = 0, images) or IBFS (dir = 1, preimages) iteration
 * (Alg. 1, CalculateImages / CalculatePreimages, then "delete duplicates
 * (lex. sort)", then the history reduction with equality in place of
 * inclusion).  The candidate of parent p and letter a has id p*k + a; of
 * every distinct set only the candidate with the smallest id is kept, and a
 * set already in H is dropped.  The output keeps the ids' order.  When H is
 * not NULL the kept sets are merged into it.
 */
static int expand(int n, int k, const int32_t *delta, int dir, const level_t *L, history_t *H,
                  level_t *out, int64_t max_sets) {
    int W = words_for(n);
    int64_t m = L->count * (int64_t)k;
    if (m > max_sets) return OR_ETOOBIG;
    uint64_t *cand = (uint64_t *)malloc((size_t)(m ? m : 1) * W * sizeof(uint64_t));
    int64_t *ids = (int64_t *)malloc((size_t)(m ? m : 1) * sizeof(int64_t));
    uint8_t *keep = (uint8_t *)calloc((size_t)(m ? m : 1), 1);
    if (!cand || !ids || !keep) {
        free(cand); free(ids); free(keep);
        return OR_ENOMEM;
    }
    int64_t nvalid = 0;
    for (int64_t p = 0; p < L->count; p++) {
        for (int a = 0; a < k; a++) {
            int64_t id = p * k + a;
            uint64_t *T = cand + id * W;
            if (dir == 0) set_image(n, delta + (size_t)a * n, L->sets + p * W, T, W);
            else set_preimage(n, delta + (size_t)a * n, L->sets + p * W, T, W);
            if (dir == 1 && set_first(T, n) < 0) continue; /* empty preimage */
            ids[nvalid++] = id;
        }
    }
    int rc = sort_ids(ids, nvalid, cand, n, W);
    if (rc) { free(cand); free(ids); free(keep); return rc; }
    /* first of every run of equal sets, unless already visited */
    int64_t nkept = 0;
    for (int64_t i = 0; i < nvalid; i++) {
        const uint64_t *s = cand + ids[i] * W;
        if (i > 0 && set_cmp(cand + ids[i - 1] * W, s, n) == 0) continue;
        if (H && history_contains(H, s, n, W)) continue;
        keep[ids[i]] = 1;
        ids[nkept++] = ids[i]; /* kept ids, still in set order */
    }
    out->count = 0;
    rc = level_reserve(out, nkept ? nkept : 1, W);
    for (int64_t id = 0; !rc && id < m; id++)
        if (keep[id]) rc = level_push(out, cand + id * W, id / k, (int)(id % k), W);
    if (!rc && H && nkept) {
        /* merge the kept sets (sorted) into the sorted history */
        uint64_t *merged = (uint64_t *)malloc((size_t)(H->count + nkept) * W * sizeof(uint64_t));
        if (!merged) rc = OR_ENOMEM;
        else {
            int64_t i = 0, j = 0, o = 0;
            while (i < H->count || j < nkept) {
                const uint64_t *src;
                if (j >= nkept || (i < H->count && set_cmp(H->sets + i * W, cand + ids[j] * W, n) < 0))
                    src = H->sets + (i++) * W;
                else
                    src = cand + ids[j++] * W;
                memcpy(merged + (o++) * W, src, (size_t)W * sizeof(uint64_t));
            }
            free(H->sets);
            H->sets = merged;
            H->count = o;
        }
    }
    free(cand); free(ids); free(keep);
    return rc;
}

/* Start a history with the sets of one level. */
static int history_init(history_t *H, const level_t *L, int n, int W) {
    H->count = 0;
    H->sets = NULL;
    int64_t *ids = (int64_t *)malloc((size_t)(L->count ? L->count : 1) * sizeof(int64_t));
    if (!ids) return OR_ENOMEM;
    for (int64_t i = 0; i < L->count; i++) ids[i] = i;
    int rc = sort_ids(ids, L->count, L->sets, n, W);
    if (!rc) {
        H->sets = (uint64_t *)malloc((size_t)(L->count ? L->count : 1) * W * sizeof(uint64_t));
        if (!H->sets) rc = OR_ENOMEM;
        for (int64_t i = 0; !rc && i < L->count; i++) {
            if (i > 0 && set_cmp(L->sets + ids[i - 1] * W, L->sets + ids[i] * W, n) == 0) continue;
            memcpy(H->sets + H->count * W, L->sets + ids[i] * W, (size_t)W * sizeof(uint64_t));
            H->count++;
        }
    }
    free(ids);
    return rc;
}

static int check_automaton(int n, int k, const int32_t *delta) {
    if (n < 1 || k < 1 || k > 255 || !delta) return OR_EINVAL;
    for (int64_t i = 0; i < (int64_t)n * k; i++)
        if (delta[i] < 0 || delta[i] >= n) return OR_EINVAL;
    return 0;
}

static int level_root_Q(level_t *L, int n, int W) {
    uint64_t *s = (uint64_t *)malloc((size_t)W * sizeof(uint64_t));
    if (!s) return OR_ENOMEM;
    set_clear(s, W);
    for (int q = 0; q < n; q++) set_add(s, q);
    int rc = level_push(L, s, -1, 0, W);
    free(s);
    return rc;
}

static int level_root_singletons(level_t *L, int n, int W) {
    uint64_t *s = (uint64_t *)malloc((size_t)W * sizeof(uint64_t));
    if (!s) return OR_ENOMEM;
    int rc = level_reserve(L, n, W);
    for (int q = 0; !rc && q < n; q++) {
        set_clear(s, W);
        set_add(s, q);
        rc = level_push(L, s, -1, 0, W);
    }
    free(s);
    return rc;
}

/* Word of the set at position pos of level depth: the letters on its chain
 * of parents back to level 0, first letter first. */
static void chain_word(const level_t *levels, int depth, int64_t pos, uint8_t *word) {
    for (int d = depth; d > 0; d--) {
        word[d - 1] = levels[d].letter[pos];
        pos = levels[d].parent[pos];
    }
}

/* ------------------------------------------------------------------ */
/* O0: brute force over words (Section 1.3.0)                          */
/* ------------------------------------------------------------------ */

int oracle_brute(int n, int k, const int32_t *delta, int max_len, int32_t *r_out, uint8_t *word) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    if (max_len < 0 || max_len > 64 || !r_out) return OR_EINVAL;
    int *state = (int *)malloc((size_t)n * sizeof(int));
    int *seen = (int *)malloc((size_t)n * sizeof(int));
    uint8_t w[64];
    if (!state || !seen) { free(state); free(seen); return OR_ENOMEM; }
    rc = OR_ENOTFOUND;
    for (int len = 0; len <= max_len && rc == OR_ENOTFOUND; len++) {
        memset(w, 0, sizeof(w)); /* the lexicographically first word of this length */
        for (;;) {
            /* apply w to every state of Q and count the distinct results */
            for (int q = 0; q < n; q++) {
                int s = q;
                for (int t = 0; t < len; t++) s = delta[(size_t)w[t] * n + s];
                state[q] = s;
            }
            memset(seen, 0, (size_t)n * sizeof(int));
            int distinct = 0;
            for (int q = 0; q < n; q++)
                if (!seen[state[q]]) { seen[state[q]] = 1; distinct++; }
            if (distinct == 1) {
                *r_out = len;
                if (word) memcpy(word, w, (size_t)len);
                rc = OR_OK;
                break;
            }
            /* next word of the same length, lexicographically (odometer) */
            int t = len - 1;
            while (t >= 0 && w[t] == k - 1) w[t--] = 0;
            if (t < 0) break;
            w[t]++;
        }
    }
    free(state);
    free(seen);
    return rc;
}

/* ------------------------------------------------------------------ */
/* O1: forward BFS in the power automaton (Section 1.3.1)              */
/* ------------------------------------------------------------------ */

int oracle_forward(int n, int k, const int32_t *delta, int64_t max_sets, int32_t *r_out,
                   uint8_t *word, int32_t word_cap, int64_t *sizes, int32_t sizes_cap,
                   int32_t *nlevels) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    if (!r_out || n > 1024) return OR_EINVAL;
    int W = words_for(n);
    int cap = 64, depth = 0;
    level_t *lv = (level_t *)calloc((size_t)cap, sizeof(level_t));
    history_t H = {0, NULL};
    if (!lv) return OR_ENOMEM;
    rc = level_root_Q(&lv[0], n, W);
    if (!rc) rc = history_init(&H, &lv[0], n, W);
    int64_t stored = 1;
    int64_t hit = (n == 1) ? 0 : -1;
    while (!rc && hit < 0) {
        if (depth + 1 == cap) {
            level_t *g = (level_t *)realloc(lv, (size_t)cap * 2 * sizeof(level_t));
            if (!g) { rc = OR_ENOMEM; break; }
            lv = g;
            memset(lv + cap, 0, (size_t)cap * sizeof(level_t));
            cap *= 2;
        }
        rc = expand(n, k, delta, 0, &lv[depth], &H, &lv[depth + 1], max_sets - stored);
        if (rc) break;
        depth++;
        stored += lv[depth].count;
        if (stored > max_sets) { rc = OR_ETOOBIG; break; }
        if (lv[depth].count == 0) { rc = OR_ENOTSYNC; break; }
        for (int64_t i = 0; i < lv[depth].count; i++)
            if (set_size(lv[depth].sets + i * W, n) == 1) { hit = i; break; }
    }
    if (!rc) {
        *r_out = depth;
        if (nlevels) *nlevels = depth + 1;
        if (sizes)
            for (int d = 0; d <= depth && d < sizes_cap; d++) sizes[d] = lv[d].count;
        if (word) {
            if (depth <= word_cap) chain_word(lv, depth, hit, word);
            else rc = OR_EWORDCAP;
        }
    }
    for (int d = 0; d < cap; d++) level_free(&lv[d]);
    free(lv);
    free(H.sets);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Level sizes of one direction, to a given depth (Section 2.1)        */
/* ------------------------------------------------------------------ */

int oracle_level_sizes(int n, int k, const int32_t *delta, int dir, int32_t depth,
                       int64_t max_sets, int64_t *sizes) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    if ((dir != 0 && dir != 1) || depth < 0 || !sizes || n > 1024) return OR_EINVAL;
    int W = words_for(n);
    level_t cur = {0}, next = {0};
    history_t H = {0, NULL};
    if (dir == 0) rc = level_root_Q(&cur, n, W);
    else rc = level_root_singletons(&cur, n, W);
    if (!rc) rc = history_init(&H, &cur, n, W);
    int64_t stored = cur.count;
    if (!rc) sizes[0] = cur.count;
    for (int d = 1; !rc && d <= depth; d++) {
        rc = expand(n, k, delta, dir, &cur, &H, &next, max_sets - stored);
        if (rc) break;
        stored += next.count;
        if (stored > max_sets) { rc = OR_ETOOBIG; break; }
        sizes[d] = next.count;
        level_t t = cur; cur = next; next = t;
    }
    level_free(&cur);
    level_free(&next);
    free(H.sets);
    return rc;
}

/* ------------------------------------------------------------------ */
/* O2: bidirectional BFS (Alg. 1 with duplicate deletion only)          */
/* ------------------------------------------------------------------ */

/* Lexicographically least word y of length j with |delta(X, y)| = 1.
 * E_m is the list of all distinct nonempty sets delta^{-1}({q}, y') with
 * |y'| = m (no history): a set S can be mapped to one state by a word of
 * length m exactly when S lies inside one of them.  Choosing at each
 * position the smallest letter that keeps this possible gives the least
 * word. */
static int least_suffix(int n, int k, const int32_t *delta, const uint64_t *X, int j,
                        int64_t max_sets, uint8_t *y) {
    int W = words_for(n);
    if (j == 0) return set_size(X, n) == 1 ? 0 : OR_ENOTSYNC;
    level_t *E = (level_t *)calloc((size_t)j, sizeof(level_t));
    if (!E) return OR_ENOMEM;
    int rc = level_root_singletons(&E[0], n, W);
    for (int m = 1; !rc && m < j; m++)
        rc = expand(n, k, delta, 1, &E[m - 1], NULL, &E[m], max_sets);
    uint64_t S[16], T[16];
    memcpy(S, X, (size_t)W * sizeof(uint64_t));
    for (int t = 0; !rc && t < j; t++) {
        int m = j - 1 - t, chosen = -1;
        for (int a = 0; a < k && chosen < 0; a++) {
            set_image(n, delta + (size_t)a * n, S, T, W);
            for (int64_t e = 0; e < E[m].count; e++)
                if (set_subset(T, E[m].sets + e * W, n)) { chosen = a; break; }
        }
        if (chosen < 0) { rc = OR_ENOTSYNC; break; }
        y[t] = (uint8_t)chosen;
        set_image(n, delta + (size_t)chosen * n, S, T, W);
        memcpy(S, T, (size_t)W * sizeof(uint64_t));
    }
    for (int m = 0; m < j; m++) level_free(&E[m]);
    free(E);
    return rc;
}

/* First position in F (in order) of a set contained in some set of B. */
static int64_t first_meet(const level_t *F, const level_t *B, int n, int W) {
    for (int64_t f = 0; f < F->count; f++)
        for (int64_t b = 0; b < B->count; b++)
            if (set_subset(F->sets + f * W, B->sets + b * W, n)) return f;
    return -1;
}

int oracle_bidir(int n, int k, const int32_t *delta, int64_t max_sets, int32_t *r_out,
                 uint8_t *word, int32_t word_cap, int64_t *fsizes, int32_t *nf, int64_t *bsizes,
                 int32_t *nb, int32_t sizes_cap) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    if (!r_out || n > 1024) return OR_EINVAL;
    int W = words_for(n);
    int cap = 4096; /* levels per direction */
    level_t *F = (level_t *)calloc((size_t)cap, sizeof(level_t));
    level_t *B = (level_t *)calloc((size_t)cap, sizeof(level_t));
    history_t HF = {0, NULL}, HB = {0, NULL};
    if (!F || !B) { free(F); free(B); return OR_ENOMEM; }
    int i = 0, j = 0;
    rc = level_root_Q(&F[0], n, W);
    if (!rc) rc = level_root_singletons(&B[0], n, W);
    if (!rc) rc = history_init(&HF, &F[0], n, W);
    if (!rc) rc = history_init(&HB, &B[0], n, W);
    int64_t stored = F[0].count + B[0].count;
    int64_t hit = rc ? -1 : first_meet(&F[0], &B[0], n, W);
    while (!rc && hit < 0) {
        if (i + 1 >= cap || j + 1 >= cap) { rc = OR_ETOOBIG; break; }
        /* step the side with fewer sets; equal sizes step forward */
        int dir = (F[i].count <= B[j].count) ? 0 : 1;
        if (dir == 0) {
            rc = expand(n, k, delta, 0, &F[i], &HF, &F[i + 1], max_sets - stored);
            if (rc) break;
            i++;
            stored += F[i].count;
            if (F[i].count == 0) { rc = OR_ENOTSYNC; break; }
        } else {
            rc = expand(n, k, delta, 1, &B[j], &HB, &B[j + 1], max_sets - stored);
            if (rc) break;
            j++;
            stored += B[j].count;
            if (B[j].count == 0) { rc = OR_ENOTSYNC; break; }
        }
        if (stored > max_sets) { rc = OR_ETOOBIG; break; }
        hit = first_meet(&F[i], &B[j], n, W);
    }
    if (!rc) {
        int r = i + j;
        *r_out = r;
        if (nf) *nf = i + 1;
        if (nb) *nb = j + 1;
        for (int d = 0; fsizes && d <= i && d < sizes_cap; d++) fsizes[d] = F[d].count;
        for (int d = 0; bsizes && d <= j && d < sizes_cap; d++) bsizes[d] = B[d].count;
        if (word) {
            if (r <= word_cap) {
                chain_word(F, i, hit, word);
                rc = least_suffix(n, k, delta, F[i].sets + hit * W, j, max_sets, word + i);
            } else {
                rc = OR_EWORDCAP;
            }
        }
    }
    for (int d = 0; d < cap; d++) { level_free(&F[d]); level_free(&B[d]); }
    free(F); free(B); free(HF.sets); free(HB.sets);
    return rc;
}

/* ------------------------------------------------------------------ */
/* O3: Alg. 1 with the inclusion reductions (Section 2.1)              */
/* ------------------------------------------------------------------ */

/* X subset of Y, word by word (the same relation as set_subset). */
static int subset_words(const uint64_t *x, const uint64_t *y, int W) {
    for (int w = 0; w < W; w++)
        if (x[w] & ~y[w]) return 0;
    return 1;
}

/*
 * One BFS (dir = 0) or IBFS (dir = 1) iteration with the list reductions of
 * Alg. 1, in the paper's order:
 *   1. CalculateImages / CalculatePreimages (empty preimages dropped);
 *   2. delete duplicates (lexicographic sort; of every set the candidate
 *      with the smallest id p*k + a stays);
 *   3. delete the sets that are not minimal (BFS) / not maximal (IBFS)
 *      with respect to inclusion among the sets of the list
 *      (MarkProperSupersets): every pair is checked;
 *   4. delete the supersets (BFS) / subsets (IBFS) of every set kept at an
 *      earlier level of the same direction (MarkSupersets against the
 *      history H = the union of those levels): every pair is checked.
 * Steps 3 and 4 both test the list as it stands after step 2, so the order
 * in which sets are removed does not matter.  The kept sets leave in
 * candidate-id order (parent position, then letter).  hist: the kept
 * levels 0..nh-1 of this direction.
 */
static int expand_reduced(int n, int k, const int32_t *delta, int dir, const level_t *L,
                          const level_t *hist, int nh, level_t *out, int64_t max_sets) {
    int W = words_for(n);
    int64_t m = L->count * (int64_t)k;
    if (m > max_sets) return OR_ETOOBIG;
    uint64_t *cand = (uint64_t *)malloc((size_t)(m ? m : 1) * W * sizeof(uint64_t));
    int64_t *ids = (int64_t *)malloc((size_t)(m ? m : 1) * sizeof(int64_t));
    uint8_t *keep = (uint8_t *)calloc((size_t)(m ? m : 1), 1);
    if (!cand || !ids || !keep) {
        free(cand); free(ids); free(keep);
        return OR_ENOMEM;
    }
    int64_t nvalid = 0;
    for (int64_t p = 0; p < L->count; p++) {
        for (int a = 0; a < k; a++) {
            int64_t id = p * k + a;
            uint64_t *T = cand + id * W;
            if (dir == 0) set_image(n, delta + (size_t)a * n, L->sets + p * W, T, W);
            else set_preimage(n, delta + (size_t)a * n, L->sets + p * W, T, W);
            if (dir == 1 && set_first(T, n) < 0) continue; /* empty preimage */
            ids[nvalid++] = id;
        }
    }
    int rc = sort_ids(ids, nvalid, cand, n, W);
    if (rc) { free(cand); free(ids); free(keep); return rc; }
    /* 2. the first of every run of equal sets */
    int64_t u = 0;
    for (int64_t i = 0; i < nvalid; i++) {
        if (i > 0 && set_cmp(cand + ids[i - 1] * W, cand + ids[i] * W, n) == 0) continue;
        ids[u++] = ids[i];
    }
    uint8_t *gone = (uint8_t *)calloc((size_t)(u ? u : 1), 1);
    if (!gone) { free(cand); free(ids); free(keep); return OR_ENOMEM; }
    /* 3. self-reduction: the sets are distinct, so inclusion is proper */
    for (int64_t a = 0; a < u; a++) {
        const uint64_t *X = cand + ids[a] * W;
        for (int64_t b = 0; b < u && !gone[a]; b++) {
            if (b == a) continue;
            const uint64_t *Y = cand + ids[b] * W;
            if (dir == 0 ? subset_words(Y, X, W) : subset_words(X, Y, W)) gone[a] = 1;
        }
    }
    /* 4. reduction by the history */
    for (int64_t a = 0; a < u; a++) {
        const uint64_t *X = cand + ids[a] * W;
        for (int h = 0; h < nh && !gone[a]; h++)
            for (int64_t z = 0; z < hist[h].count && !gone[a]; z++) {
                const uint64_t *Z = hist[h].sets + z * W;
                if (dir == 0 ? subset_words(Z, X, W) : subset_words(X, Z, W)) gone[a] = 1;
            }
    }
    int64_t nkept = 0;
    for (int64_t a = 0; a < u; a++)
        if (!gone[a]) { keep[ids[a]] = 1; nkept++; }
    out->count = 0;
    rc = level_reserve(out, nkept ? nkept : 1, W);
    for (int64_t id = 0; !rc && id < m; id++)
        if (keep[id]) rc = level_push(out, cand + id * W, id / k, (int)(id % k), W);
    free(gone); free(cand); free(ids); free(keep);
    return rc;
}

/* Sizes of the reduced levels 0..depth of one direction: dir 0 = images of
 * Q (minimal sets, supersets of earlier levels removed), 1 = preimages of
 * the singletons (maximal sets, subsets of earlier levels removed). */
int oracle_reduced_level_sizes(int n, int k, const int32_t *delta, int dir, int32_t depth,
                               int64_t max_sets, int64_t *sizes) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    if ((dir != 0 && dir != 1) || depth < 0 || !sizes || n > 1024) return OR_EINVAL;
    int W = words_for(n);
    level_t *lv = (level_t *)calloc((size_t)depth + 1, sizeof(level_t));
    if (!lv) return OR_ENOMEM;
    if (dir == 0) rc = level_root_Q(&lv[0], n, W);
    else rc = level_root_singletons(&lv[0], n, W);
    int64_t stored = lv[0].count;
    if (!rc) sizes[0] = lv[0].count;
    for (int d = 1; !rc && d <= depth; d++) {
        rc = expand_reduced(n, k, delta, dir, &lv[d - 1], lv, d, &lv[d], max_sets - stored);
        if (rc) break;
        stored += lv[d].count;
        if (stored > max_sets) { rc = OR_ETOOBIG; break; }
        sizes[d] = lv[d].count;
    }
    for (int d = 0; d <= depth; d++) level_free(&lv[d]);
    free(lv);
    return rc;
}

/*
 * Alg. 1 with the inclusion reductions.  The reduced levels of each side
 * depend on that side alone, and the searches first meet when the depths
 * add up to r whatever the order of the steps; the word does depend on the
 * split.  fwd_depth < 0: the side with fewer sets steps (equal sizes step
 * forward); fwd_depth >= 0: forward steps until the forward depth is
 * fwd_depth, then backward steps (so the first meet is at i = fwd_depth
 * when fwd_depth <= r).  dirs: bit 0 reduces the BFS side, bit 1 the IBFS
 * side; a side that is not reduced keeps duplicate deletion and the
 * equality history (as oracle_bidir).  The word is the parent chain of the
 * first meeting forward set in list order followed by the least suffix
 * (least_suffix).
 */
int oracle_bidir_reduced(int n, int k, const int32_t *delta, int64_t max_sets, int32_t fwd_depth, int32_t dirs,
                         int32_t *r_out, uint8_t *word, int32_t word_cap, int64_t *fsizes, int32_t *nf,
                         int64_t *bsizes, int32_t *nb, int32_t sizes_cap) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    if (!r_out || n > 1024) return OR_EINVAL;
    int W = words_for(n);
    int cap = 4096; /* levels per direction */
    level_t *F = (level_t *)calloc((size_t)cap, sizeof(level_t));
    level_t *B = (level_t *)calloc((size_t)cap, sizeof(level_t));
    if (!F || !B) { free(F); free(B); return OR_ENOMEM; }
    int i = 0, j = 0;
    history_t HF = {0, NULL}, HB = {0, NULL}; /* equality histories of a side that is not reduced */
    rc = level_root_Q(&F[0], n, W);
    if (!rc) rc = level_root_singletons(&B[0], n, W);
    if (!rc && !(dirs & 1)) rc = history_init(&HF, &F[0], n, W);
    if (!rc && !(dirs & 2)) rc = history_init(&HB, &B[0], n, W);
    int64_t stored = F[0].count + B[0].count;
    int64_t hit = rc ? -1 : first_meet(&F[0], &B[0], n, W);
    while (!rc && hit < 0) {
        if (i + 1 >= cap || j + 1 >= cap) { rc = OR_ETOOBIG; break; }
        int dir = fwd_depth >= 0 ? (i < fwd_depth ? 0 : 1) : (F[i].count <= B[j].count ? 0 : 1);
        if (dir == 0) {
            if (dirs & 1) rc = expand_reduced(n, k, delta, 0, &F[i], F, i + 1, &F[i + 1], max_sets - stored);
            else rc = expand(n, k, delta, 0, &F[i], &HF, &F[i + 1], max_sets - stored);
            if (rc) break;
            i++;
            stored += F[i].count;
            if (F[i].count == 0) { rc = OR_ENOTSYNC; break; }
        } else {
            if (dirs & 2) rc = expand_reduced(n, k, delta, 1, &B[j], B, j + 1, &B[j + 1], max_sets - stored);
            else rc = expand(n, k, delta, 1, &B[j], &HB, &B[j + 1], max_sets - stored);
            if (rc) break;
            j++;
            stored += B[j].count;
            if (B[j].count == 0) { rc = OR_ENOTSYNC; break; }
        }
        if (stored > max_sets) { rc = OR_ETOOBIG; break; }
        hit = first_meet(&F[i], &B[j], n, W);
    }
    if (!rc) {
        int r = i + j;
        *r_out = r;
        if (nf) *nf = i + 1;
        if (nb) *nb = j + 1;
        for (int d = 0; fsizes && d <= i && d < sizes_cap; d++) fsizes[d] = F[d].count;
        for (int d = 0; bsizes && d <= j && d < sizes_cap; d++) bsizes[d] = B[d].count;
        if (word) {
            if (r <= word_cap) {
                chain_word(F, i, hit, word);
                rc = least_suffix(n, k, delta, F[i].sets + hit * W, j, max_sets, word + i);
            } else {
                rc = OR_EWORDCAP;
            }
        }
    }
    for (int d = 0; d < cap; d++) { level_free(&F[d]); level_free(&B[d]); }
    free(F); free(B); free(HF.sets); free(HB.sets);
    return rc;
}

/* ------------------------------------------------------------------ */
/* O4: beam upper bound, inverse BFS with a cut-off (Section 2.1.3)    */
/* ------------------------------------------------------------------ */

typedef struct {
    const uint64_t *cand;
    int n, W;
} beam_ctx_t;

/* Order of the beam's cut: larger sets first, then smaller candidate id. */
static int beam_before(const beam_ctx_t *c, int64_t a, int64_t b) {
    int ca = set_size(c->cand + a * c->W, c->n), cb = set_size(c->cand + b * c->W, c->n);
    if (ca != cb) return ca > cb;
    return a < b;
}

/*
 * The beam search that gives the paper's upper bound R (Section 2.1.3, the
 * cut-off inverse BFS it cites): level 0 is the n singletons; level d + 1
 * is made of the preimages delta^{-1}(S, a) of the sets S of level d under
 * every letter a, empty ones dropped and duplicates removed (the smallest
 * candidate id p*k + a of every set stays), of which only the `beam`
 * largest are kept (ties: smaller candidate id first), in candidate-id
 * order.  No history is kept.  The first depth R at which Q itself is a
 * kept set gives the reset word y with delta^{-1}({q}, y) = Q, i.e.
 * delta(Q, y) = {q}: the letters on the chain from that set back to its
 * singleton, last-applied first.  Kept sizes go to sizes[0..R].
 * Returns OR_ENOTFOUND when no level up to max_depth holds Q.
 */
int oracle_beam(int n, int k, const int32_t *delta, int64_t beam, int32_t max_depth, int32_t *R_out,
                uint8_t *word, int32_t word_cap, int64_t *sizes, int32_t sizes_cap, int32_t *nlevels) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    if (!R_out || beam < 1 || max_depth < 0 || n > 8192) return OR_EINVAL;
    int W = words_for(n);
    int cap = max_depth + 1;
    level_t *lv = (level_t *)calloc((size_t)cap, sizeof(level_t));
    if (!lv) return OR_ENOMEM;
    rc = level_root_singletons(&lv[0], n, W);
    int64_t hit = (n == 1) ? 0 : -1;
    int depth = 0;
    while (!rc && hit < 0) {
        if (depth == max_depth) { rc = OR_ENOTFOUND; break; }
        const level_t *L = &lv[depth];
        int64_t m = L->count * (int64_t)k;
        uint64_t *cand = (uint64_t *)malloc((size_t)(m ? m : 1) * W * sizeof(uint64_t));
        int64_t *ids = (int64_t *)malloc((size_t)(m ? m : 1) * sizeof(int64_t));
        uint8_t *keep = (uint8_t *)calloc((size_t)(m ? m : 1), 1);
        if (!cand || !ids || !keep) { free(cand); free(ids); free(keep); rc = OR_ENOMEM; break; }
        int64_t nvalid = 0;
        for (int64_t p = 0; p < L->count; p++)
            for (int a = 0; a < k; a++) {
                int64_t id = p * k + a;
                set_preimage(n, delta + (size_t)a * n, L->sets + p * W, cand + id * W, W);
                if (set_first(cand + id * W, n) >= 0) ids[nvalid++] = id;
            }
        rc = sort_ids(ids, nvalid, cand, n, W);
        int64_t u = 0;
        for (int64_t i = 0; !rc && i < nvalid; i++) {
            if (i > 0 && set_cmp(cand + ids[i - 1] * W, cand + ids[i] * W, n) == 0) continue;
            ids[u++] = ids[i];
        }
        /* the cut: insertion sort would be quadratic; a plain merge sort by
         * (size descending, id ascending) */
        beam_ctx_t ctx = {cand, n, W};
        int64_t *tmp = (int64_t *)malloc((size_t)(u ? u : 1) * sizeof(int64_t));
        if (!rc && !tmp) rc = OR_ENOMEM;
        for (int64_t width = 1; !rc && width < u; width *= 2) {
            for (int64_t lo = 0; lo < u; lo += 2 * width) {
                int64_t mid = lo + width < u ? lo + width : u, hi = lo + 2 * width < u ? lo + 2 * width : u;
                int64_t i = lo, j = mid, o = lo;
                while (i < mid && j < hi) tmp[o++] = beam_before(&ctx, ids[j], ids[i]) ? ids[j++] : ids[i++];
                while (i < mid) tmp[o++] = ids[i++];
                while (j < hi) tmp[o++] = ids[j++];
            }
            memcpy(ids, tmp, (size_t)u * sizeof(int64_t));
        }
        free(tmp);
        int64_t kept = u < beam ? u : beam;
        for (int64_t i = 0; !rc && i < kept; i++) keep[ids[i]] = 1;
        if (!rc) rc = level_reserve(&lv[depth + 1], kept ? kept : 1, W);
        for (int64_t id = 0; !rc && id < m; id++)
            if (keep[id]) rc = level_push(&lv[depth + 1], cand + id * W, id / k, (int)(id % k), W);
        free(cand); free(ids); free(keep);
        if (rc) break;
        depth++;
        if (lv[depth].count == 0) { rc = OR_ENOTSYNC; break; }
        for (int64_t i = 0; i < lv[depth].count && hit < 0; i++)
            if (set_size(lv[depth].sets + i * W, n) == n) hit = i;
    }
    if (!rc) {
        *R_out = depth;
        if (nlevels) *nlevels = depth + 1;
        for (int d = 0; sizes && d <= depth && d < sizes_cap; d++) sizes[d] = lv[d].count;
        if (word) {
            if (depth > word_cap) rc = OR_EWORDCAP;
            else {
                int64_t pos = hit;
                for (int d = depth; d > 0; d--) { /* the set of depth d was made by the (depth - d + 1)-th letter */
                    word[depth - d] = lv[d].letter[pos];
                    pos = lv[d].parent[pos];
                }
            }
        }
    }
    for (int d = 0; d < cap; d++) level_free(&lv[d]);
    free(lv);
    return rc;
}

/* ------------------------------------------------------------------ */
/* O5: the inverse DFS phase (Section 2.2)                              */
/* ------------------------------------------------------------------ */

/* The level of one direction at depth `depth` (distinct sets first reached
 * there, as oracle_level_sizes counts them), left in *out. */
static int level_at(int n, int k, const int32_t *delta, int dir, int depth, int64_t max_sets, level_t *out) {
    int W = words_for(n);
    level_t cur = {0}, next = {0};
    history_t H = {0, NULL};
    int rc = dir == 0 ? level_root_Q(&cur, n, W) : level_root_singletons(&cur, n, W);
    if (!rc) rc = history_init(&H, &cur, n, W);
    int64_t stored = cur.count;
    for (int d = 1; !rc && d <= depth; d++) {
        rc = expand(n, k, delta, dir, &cur, &H, &next, max_sets - stored);
        if (rc) break;
        stored += next.count;
        if (stored > max_sets) rc = OR_ETOOBIG;
        level_t t = cur; cur = next; next = t;
    }
    level_free(&next);
    free(H.sets);
    if (rc) level_free(&cur);
    else *out = cur;
    return rc;
}

/* The reduced level of one direction at depth `depth` (Alg. 1 with its
 * inclusion reductions, as oracle_reduced_level_sizes counts it), left in
 * *out. */
static int reduced_level_at(int n, int k, const int32_t *delta, int dir, int depth, int64_t max_sets,
                            level_t *out) {
    int W = words_for(n);
    level_t *lv = (level_t *)calloc((size_t)depth + 1, sizeof(level_t));
    if (!lv) return OR_ENOMEM;
    int rc = dir == 0 ? level_root_Q(&lv[0], n, W) : level_root_singletons(&lv[0], n, W);
    int64_t stored = lv[0].count;
    for (int d = 1; !rc && d <= depth; d++) {
        rc = expand_reduced(n, k, delta, dir, &lv[d - 1], lv, d, &lv[d], max_sets - stored);
        if (!rc) stored += lv[d].count;
        if (!rc && stored > max_sets) rc = OR_ETOOBIG;
    }
    for (int d = 0; d < depth; d++) level_free(&lv[d]);
    if (rc) level_free(&lv[depth]);
    else *out = lv[depth];
    free(lv);
    return rc;
}

/* Some X of F lies inside Y (brute force over F: the query the paper's
 * static trie answers). */
static int some_subset(const level_t *F, const uint64_t *Y, int n, int W) {
    for (int64_t f = 0; f < F->count; f++)
        if (set_subset(F->sets + f * W, Y, n)) return 1;
    return 0;
}

/* Depth-first over the preimages of Y, d more inverse steps: 1 when a set
 * reached after exactly d steps contains a set of F.  buf holds one set
 * per remaining step. */
static int dfs_reaches(int n, int k, const int32_t *delta, const level_t *F, const uint64_t *Y, int d,
                       uint64_t *buf, int W) {
    if (d == 0) return some_subset(F, Y, n, W);
    uint64_t *P = buf;
    for (int a = 0; a < k; a++) {
        set_preimage(n, delta + (size_t)a * n, Y, P, W);
        if (set_first(P, n) < 0) continue; /* empty preimage */
        if (dfs_reaches(n, k, delta, F, P, d - 1, buf + W, W)) return 1;
    }
    return 0;
}

/*
 * r from the last levels F_i (BFS) and B_j (IBFS) of a bidirectional
 * search, by the memory-bounded inverse phase of Section 2.2: a depth-first
 * inverse search from every set of B_j, without history, checking the sets
 * it reaches against F_i.  D is deepened one step at a time (D = 0, 1, ...,
 * D = 0 being the meet of F_i and B_j themselves); the first D at which some
 * set of B_j reaches, after exactly D inverse steps, a superset of a set of
 * F_i gives r = fwd_depth + bwd_depth + D.  dirs: bit 0 takes F_i from the
 * BFS with the inclusion reductions of Alg. 1, bit 1 takes B_j from the
 * reduced IBFS (otherwise duplicates and the equality history only).
 * Returns OR_ENOTFOUND when no D up to max_depth does.
 */
int oracle_inverse_dfs_r(int n, int k, const int32_t *delta, int32_t fwd_depth, int32_t bwd_depth, int32_t dirs,
                         int32_t max_depth, int64_t max_sets, int32_t *r_out) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    if (fwd_depth < 0 || bwd_depth < 0 || dirs < 0 || dirs > 3 || max_depth < 0 || !r_out || n > 1024)
        return OR_EINVAL;
    int W = words_for(n);
    level_t F = {0}, B = {0};
    rc = (dirs & 1) ? reduced_level_at(n, k, delta, 0, fwd_depth, max_sets, &F)
                    : level_at(n, k, delta, 0, fwd_depth, max_sets, &F);
    if (!rc)
        rc = (dirs & 2) ? reduced_level_at(n, k, delta, 1, bwd_depth, max_sets, &B)
                        : level_at(n, k, delta, 1, bwd_depth, max_sets, &B);
    uint64_t *buf = rc ? NULL : (uint64_t *)malloc((size_t)(max_depth + 1) * W * sizeof(uint64_t));
    if (!rc && !buf) rc = OR_ENOMEM;
    int found = -1;
    for (int D = 0; !rc && found < 0 && D <= max_depth; D++)
        for (int64_t b = 0; found < 0 && b < B.count; b++)
            if (dfs_reaches(n, k, delta, &F, B.sets + b * W, D, buf, W)) found = D;
    if (!rc && found < 0) rc = OR_ENOTFOUND;
    if (!rc) *r_out = fwd_depth + bwd_depth + found;
    free(buf);
    level_free(&F);
    level_free(&B);
    return rc;
}

/* ------------------------------------------------------------------ */
/* O6: MarkSupersets by recursive state splitting (Alg. 2, §2.1.1)     */
/* ------------------------------------------------------------------ */

/* The recursion of Alg. 2 on intervals: A[a0, a1) (indices into the sorted
 * list A, all agreeing on states 0 .. d-1) and the live part bi[b0, b1) of
 * B (indices not marked yet).  A marked B index is swapped to the end of
 * the live part and the interval shrinks, so the live part of every caller
 * stays a prefix of its interval. */
typedef struct {
    const uint64_t *A, *B;
    int n, W, proper, min_brute;
    int64_t *bi;     /* permutation of B's indices */
    uint8_t *mark;   /* mark[b] = 1: B[b] is a (proper) superset of some set of A */
} mark_ctx_t;

static int64_t mark_rec(mark_ctx_t *c, int64_t a0, int64_t a1, int64_t b0, int64_t b1, int d) {
    /* returns the new end of the live part b1 */
    const int W = c->W;
    if (a1 - a0 <= c->min_brute || d >= c->n) {
        for (int64_t p = b0; p < b1;) {
            const uint64_t *Y = c->B + c->bi[p] * W;
            int hit = 0;
            for (int64_t a = a0; a < a1 && !hit; a++) {
                const uint64_t *X = c->A + a * W;
                if (set_subset(X, Y, c->n) && !(c->proper && set_cmp(X, Y, c->n) == 0)) hit = 1;
            }
            if (hit) {
                c->mark[c->bi[p]] = 1;
                int64_t t = c->bi[p];
                c->bi[p] = c->bi[b1 - 1];
                c->bi[b1 - 1] = t;
                b1--;
            } else {
                p++;
            }
        }
        return b1;
    }
    /* A_0 (state d absent) comes first in the sorted interval: find the cut */
    int64_t lo = a0, hi = a1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (set_has(c->A + mid * W, d)) hi = mid;
        else lo = mid + 1;
    }
    const int64_t cut = lo;
    /* A_0 may lie inside any live set of B */
    if (cut > a0) b1 = mark_rec(c, a0, cut, b0, b1, d + 1);
    if (cut < a1) {
        /* a set of A_1 holds state d: only live B sets holding it qualify;
         * order the live part so that they form its suffix */
        int64_t p = b0, q = b1;
        while (p < q) {
            if (set_has(c->B + c->bi[p] * W, d)) {
                q--;
                int64_t t = c->bi[p];
                c->bi[p] = c->bi[q];
                c->bi[q] = t;
            } else {
                p++;
            }
        }
        /* B_1 = bi[q, b1); marks inside it shrink it from its end, so the
         * live part stays bi[b0, b1') with the marked indices after it */
        int64_t e = mark_rec(c, cut, a1, q, b1, d + 1);
        b1 = e;
    }
    return b1;
}

/*
 * Alg. 2 (MarkSupersets, Section 2.1.1): marks every set of B that is a
 * superset (proper = 1: a proper superset, MarkProperSupersets) of some set
 * of A.  A: na sets sorted lexicographically (state 0 first, absent before
 * present) with no repeats; B: nb sets in any order.  A lists of at most
 * min_brute sets is checked against the live part of B pair by pair (the
 * paper's MIN); otherwise A is split by the current state d and the two
 * halves recurse, the half holding d only against the B sets that hold d.
 * mark_out[b] = 1 for the marked sets of B.  Returns the number marked.
 */
int64_t oracle_mark_supersets(int n, const uint64_t *A, int64_t na, const uint64_t *B, int64_t nb, int proper,
                              int32_t min_brute, uint8_t *mark_out) {
    if (n < 1 || n > 4096 || na < 0 || nb < 0 || (na && !A) || (nb && !B) || !mark_out || min_brute < 1)
        return OR_EINVAL;
    const int W = words_for(n);
    for (int64_t a = 1; a < na; a++)
        if (set_cmp(A + (a - 1) * W, A + a * W, n) >= 0) return OR_EINVAL; /* not sorted and unique */
    mark_ctx_t c;
    c.A = A;
    c.B = B;
    c.n = n;
    c.W = W;
    c.proper = proper ? 1 : 0;
    c.min_brute = min_brute;
    c.bi = (int64_t *)malloc((size_t)(nb ? nb : 1) * sizeof(int64_t));
    if (!c.bi) return OR_ENOMEM;
    c.mark = mark_out;
    memset(mark_out, 0, (size_t)nb);
    for (int64_t b = 0; b < nb; b++) c.bi[b] = b;
    int64_t live_end = na ? mark_rec(&c, 0, na, 0, nb, 0) : nb;
    free(c.bi);
    return nb - live_end;
}

/* ------------------------------------------------------------------ */
/* Synchronizability: every pair of states can be merged (Section 2)   */
/* ------------------------------------------------------------------ */

int oracle_is_synchronizing(int n, int k, const int32_t *delta) {
    int rc = check_automaton(n, k, delta);
    if (rc) return rc;
    /* merged[p*n+q] = 1 when some word maps p and q to one state; found by
     * walking backwards from the pairs (s, s) through pairs of preimages.
     * pre[a] lists the states of each preimage delta^{-1}({s}, a) in turn,
     * the states mapped to s starting at start[a*(n+1) + s]. */
    size_t nn = (size_t)n * n;
    uint8_t *merged = (uint8_t *)calloc(nn, 1);
    int64_t *queue = (int64_t *)malloc(nn * sizeof(int64_t));
    int32_t *pre = (int32_t *)malloc((size_t)k * n * sizeof(int32_t));
    int32_t *start = (int32_t *)calloc((size_t)k * (n + 1), sizeof(int32_t));
    if (!merged || !queue || !pre || !start) {
        free(merged); free(queue); free(pre); free(start);
        return OR_ENOMEM;
    }
    for (int a = 0; a < k; a++) {
        int32_t *st = start + (size_t)a * (n + 1);
        for (int q = 0; q < n; q++) st[delta[(size_t)a * n + q] + 1]++;
        for (int s = 0; s < n; s++) st[s + 1] += st[s];
        int32_t *fill = (int32_t *)malloc((size_t)n * sizeof(int32_t));
        if (!fill) { free(merged); free(queue); free(pre); free(start); return OR_ENOMEM; }
        memcpy(fill, st, (size_t)n * sizeof(int32_t));
        for (int q = 0; q < n; q++) pre[(size_t)a * n + fill[delta[(size_t)a * n + q]]++] = q;
        free(fill);
    }
    int64_t head = 0, tail = 0;
    for (int s = 0; s < n; s++) { merged[(size_t)s * n + s] = 1; queue[tail++] = (int64_t)s * n + s; }
    while (head < tail) {
        int64_t st = queue[head++];
        int s = (int)(st / n), t = (int)(st % n);
        for (int a = 0; a < k; a++) {
            const int32_t *sa = start + (size_t)a * (n + 1);
            const int32_t *pa = pre + (size_t)a * n;
            for (int i = sa[s]; i < sa[s + 1]; i++) {
                for (int j = sa[t]; j < sa[t + 1]; j++) {
                    size_t pq = (size_t)pa[i] * n + pa[j];
                    if (!merged[pq]) { merged[pq] = 1; queue[tail++] = (int64_t)pq; }
                }
            }
        }
    }
    int all = 1;
    for (size_t i = 0; i < nn; i++) all &= merged[i];
    free(merged); free(queue); free(pre); free(start);
    return all;
}
