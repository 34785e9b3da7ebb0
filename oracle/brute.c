/*
 * Brute-force local alignment score.  TEST INFRASTRUCTURE ONLY (used by the tests
 * to pin the oracle; never by the library).
 *
 * A local alignment of reads a and b is a global alignment of a substring of a with
 * a substring of b (paper section 2.2 takes the local alignment score of the
 * Smith-Waterman algorithm).  This file finds the best one by listing them all: from
 * every start point (i, j) it walks every path of alignment columns -- a aligned with
 * b (score +match or +mismatch), a against a gap, or b against a gap (score -gap) --
 * and keeps the best running score seen, the empty alignment (score 0) included.
 * The affine variant charges gap_open + gap for the first column of a run of gap
 * columns of one kind and gap for each further one.
 * No table of partial results is kept, so it shares nothing with a dynamic program.
 * Cost grows like the Delannoy numbers; it is meant for reads of length <= 6.
 */
#include <stdint.h>

typedef struct {
    const uint8_t *a, *b;
    int la, lb, match, mismatch, gap, best;
    int gap_open;             /* affine: a run of L gap columns costs gap_open + L * gap */
} walk_t;

static int up(uint8_t c) { return (c >= 'a' && c <= 'z') ? (c - 'a' + 'A') : c; }

static void walk(walk_t *W, int i, int j, int score)
{
    if (score > W->best) W->best = score;
    if (i < W->la && j < W->lb)
        walk(W, i + 1, j + 1, score + (up(W->a[i]) == up(W->b[j]) ? W->match : W->mismatch));
    if (i < W->la) walk(W, i + 1, j, score - W->gap);
    if (j < W->lb) walk(W, i, j + 1, score - W->gap);
}

int brute_local_score(const uint8_t *a, int la, const uint8_t *b, int lb,
                      int match, int mismatch, int gap)
{
    walk_t W = {a, b, la, lb, match, mismatch, gap, 0, 0};
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j) walk(&W, i, j, 0);
    return W.best;
}

/* The same walk, remembering the previous column (0 = aligned pair or start, 1 = a
 * against a gap, 2 = b against a gap): a gap column opens a new gap (gap_open + gap)
 * unless it continues a run of the same kind (gap). */
static void walk_affine(walk_t *W, int i, int j, int score, int prev)
{
    if (score > W->best) W->best = score;
    if (i < W->la && j < W->lb)
        walk_affine(W, i + 1, j + 1, score + (up(W->a[i]) == up(W->b[j]) ? W->match : W->mismatch), 0);
    if (i < W->la) walk_affine(W, i + 1, j, score - W->gap - (prev == 1 ? 0 : W->gap_open), 1);
    if (j < W->lb) walk_affine(W, i, j + 1, score - W->gap - (prev == 2 ? 0 : W->gap_open), 2);
}

int brute_local_score_affine(const uint8_t *a, int la, const uint8_t *b, int lb,
                             int match, int mismatch, int gap_open, int gap)
{
    walk_t W = {a, b, la, lb, match, mismatch, gap, 0, gap_open};
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j) walk_affine(&W, i, j, 0, 0);
    return W.best;
}

/* Every pair of strings over {A,C,G,T} with lengths in [0, maxlen]: out[p] holds the
 * brute-force score of pair p, pairs ordered by (string index of a, string index of b),
 * strings ordered by length, then lexicographically with A < C < G < T. */
static void nth_string(int idx, int maxlen, uint8_t *s, int *len)
{
    static const uint8_t ALPHA[4] = {'A', 'C', 'G', 'T'};
    int L = 0, count = 1;
    while (L <= maxlen && idx >= count) { idx -= count; ++L; count *= 4; }
    for (int k = L - 1; k >= 0; --k) { s[k] = ALPHA[idx & 3]; idx >>= 2; }
    *len = L;
}

int brute_count_strings(int maxlen)
{
    int total = 0, count = 1;
    for (int L = 0; L <= maxlen; ++L) { total += count; count *= 4; }
    return total;
}

void brute_string(int idx, int maxlen, uint8_t *s, int *len) { nth_string(idx, maxlen, s, len); }

void brute_exhaustive(int maxlen, int match, int mismatch, int gap, int gap_open, int32_t *out)
{
    int ns = brute_count_strings(maxlen);
    uint8_t sa[16], sb[16];
    int la, lb;
    for (int x = 0; x < ns; ++x) {
        nth_string(x, maxlen, sa, &la);
        for (int y = 0; y < ns; ++y) {
            nth_string(y, maxlen, sb, &lb);
            out[(int64_t)x * ns + y] =
                gap_open > 0 ? brute_local_score_affine(sa, la, sb, lb, match, mismatch, gap_open, gap)
                             : brute_local_score(sa, la, sb, lb, match, mismatch, gap);
        }
    }
}
