/*
 * CPU oracle for the read-to-read alignment distance.  TEST INFRASTRUCTURE ONLY:
 * it is called by the tests, by the package's smoke check and by the CPU-baseline
 * leg of the benchmark, never by the library's compute path.  It shares no code,
 * header or table with the CUDA library.
 *
 * What it computes (paper section 2.2, "Scalable pairwise distances computation"):
 * the dissimilarity between two reads is derived from their local alignment score,
 * computed with the Smith-Waterman algorithm, for every pair of reads (the m x n
 * matrix D of the program `disseq`, and its all-pairs form with ~5e9 values for
 * 1e5 reads, i.e. the strict upper triangle).
 *
 * The paper fixes neither the scores nor the score-to-distance conversion.  The
 * readings used here (each one an argument, with these defaults):
 *   substitution  s(x,y) = +1 if x == y else -1   (match = 1, mismatch = -1)
 *   gaps          linear, -1 per gapped base      (gap = 1); optionally affine (Gotoh):
 *                 a run of L gapped bases costs gap_open + L * gap  (gap_open = 0: linear)
 *   local score   H(i,0) = H(0,j) = 0,
 *                 H(i,j) = max(0, H(i-1,j-1) + s(a_i,b_j), H(i-1,j) - g, H(i,j-1) - g),
 *                 S = max over all cells of H   (Smith & Waterman 1981, textbook form)
 *   distance      d = max(la, lb) - S           (stored as an unsigned 16-bit integer,
 *                                                 clamped into [0, 65535]); the paper leaves
 *                 the score-to-distance rule open (the authors' own note in section 2.2
 *                 asks whether the dissimilarity is a distance), so three other readings
 *                 are selectable (argument `conversion`):
 *                   1  d = min(la, lb) - S, clamped likewise (0 when one read lies inside
 *                      the other, so not a metric);
 *                   2  the raw score S, clamped likewise;
 *                   3  normalised: d = floor(65535 * (m - S) / m) with m = max(la, lb) and
 *                      m - S clamped into [0, m], i.e. 1 - S/m on a 16-bit fixed-point
 *                      scale; d = 0 when both reads are empty.
 *   all pairs     strict upper triangle, row-major: k(i,j) = i*n - i*(i+1)/2 + (j-i-1)
 *
 * The implementation is the plain definition: the full (la+1) x (lb+1) matrix is
 * allocated and filled row by row.  Bases are compared case-insensitively.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int upper_base(uint8_t c) { return (c >= 'a' && c <= 'z') ? (c - 'a' + 'A') : c; }

static int max2(int x, int y) { return x > y ? x : y; }

/* Smith-Waterman local alignment score S, from the full DP matrix H. */
int oracle_sw_score(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb,
                    int match, int mismatch, int gap)
{
    if (la <= 0 || lb <= 0) return 0;
    int64_t w = lb + 1;
    int *H = (int *)malloc(sizeof(int) * (size_t)(la + 1) * (size_t)w);
    if (!H) return -1;
    for (int64_t j = 0; j <= lb; ++j) H[j] = 0;              /* H(0,j) = 0 */
    int S = 0;
    for (int64_t i = 1; i <= la; ++i) {
        H[i * w] = 0;                                         /* H(i,0) = 0 */
        for (int64_t j = 1; j <= lb; ++j) {
            int s = (upper_base(a[i - 1]) == upper_base(b[j - 1])) ? match : mismatch;
            int h = 0;
            h = max2(h, H[(i - 1) * w + (j - 1)] + s);
            h = max2(h, H[(i - 1) * w + j] - gap);
            h = max2(h, H[i * w + (j - 1)] - gap);
            H[i * w + j] = h;
            S = max2(S, h);
        }
    }
    free(H);
    return S;
}

/* Local score with affine gaps (Gotoh 1982): a run of L gapped bases costs
 * gap_open + L * gap.  Three full matrices: H (best alignment ending at (i, j)), E (ending
 * with b_j against a gap), F (ending with a_i against a gap):
 *   E(i,j) = max(E(i,j-1) - gap, H(i,j-1) - gap_open - gap)
 *   F(i,j) = max(F(i-1,j) - gap, H(i-1,j) - gap_open - gap)
 *   H(i,j) = max(0, H(i-1,j-1) + s(a_i,b_j), E(i,j), F(i,j)),
 * H(i,0) = H(0,j) = 0, E(i,0) = F(0,j) = minus infinity, S = max H. */
int oracle_sw_score_affine(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb,
                           int match, int mismatch, int gap_open, int gap)
{
    if (la <= 0 || lb <= 0) return 0;
    const int NEG = -(1 << 28);
    int64_t w = lb + 1;
    size_t cells = (size_t)(la + 1) * (size_t)w;
    int *H = (int *)malloc(sizeof(int) * cells);
    int *E = (int *)malloc(sizeof(int) * cells);
    int *F = (int *)malloc(sizeof(int) * cells);
    if (!H || !E || !F) { free(H); free(E); free(F); return -1; }
    for (int64_t j = 0; j <= lb; ++j) { H[j] = 0; E[j] = NEG; F[j] = NEG; }
    int S = 0;
    for (int64_t i = 1; i <= la; ++i) {
        H[i * w] = 0; E[i * w] = NEG; F[i * w] = NEG;
        for (int64_t j = 1; j <= lb; ++j) {
            int s = (upper_base(a[i - 1]) == upper_base(b[j - 1])) ? match : mismatch;
            int e = max2(E[i * w + (j - 1)] - gap, H[i * w + (j - 1)] - gap_open - gap);
            int f = max2(F[(i - 1) * w + j] - gap, H[(i - 1) * w + j] - gap_open - gap);
            int h = max2(0, H[(i - 1) * w + (j - 1)] + s);
            h = max2(h, max2(e, f));
            E[i * w + j] = e;
            F[i * w + j] = f;
            H[i * w + j] = h;
            S = max2(S, h);
        }
    }
    free(H); free(E); free(F);
    return S;
}

static int score_of(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb, int match, int mismatch,
                    int gap_open, int gap)
{
    return gap_open > 0 ? oracle_sw_score_affine(a, la, b, lb, match, mismatch, gap_open, gap)
                        : oracle_sw_score(a, la, b, lb, match, mismatch, gap);
}

/* d = max(la, lb) - S, the distance reading of the score, stored as uint16: clamped into
 * [0, 65535].  With the default scores S <= min(la, lb), so d is never negative; a match
 * score above 1 can make S exceed max(la, lb), and d is then 0. */
static int clamp_u16(int64_t d) { return d < 0 ? 0 : (d > 65535 ? 65535 : (int)d); }

/* The score-to-distance rules (conversion codes of the header comment). */
static int convert_score(int64_t S, int64_t la, int64_t lb, int conversion)
{
    int64_t hi = la > lb ? la : lb;
    int64_t lo = la < lb ? la : lb;
    if (conversion == 1) return clamp_u16(lo - S);
    if (conversion == 2) return clamp_u16(S);
    if (conversion == 3) {
        if (hi == 0) return 0;
        int64_t x = hi - S;
        if (x < 0) x = 0;
        if (x > hi) x = hi;
        return (int)((65535 * x) / hi);
    }
    return clamp_u16(hi - S);
}

int oracle_distance(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb,
                    int match, int mismatch, int gap)
{
    int S = oracle_sw_score(a, la, b, lb, match, mismatch, gap);
    return convert_score(S, la, lb, 0);
}

/* Distance under any conversion rule, linear or affine gaps. */
int oracle_distance_conv(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb, int match,
                         int mismatch, int gap, int gap_open, int conversion)
{
    int S = score_of(a, la, b, lb, match, mismatch, gap_open, gap);
    return convert_score(S, la, lb, conversion);
}

/* Position of pair (i, j), i < j, in the row-major strict upper triangle of n reads. */
uint64_t oracle_tri_index(uint64_t i, uint64_t j, uint64_t n)
{
    return i * n - i * (i + 1) / 2 + (j - i - 1);
}

/* ---------------------------------------------------------------- threaded drivers */

typedef struct {
    const uint8_t *seq;
    const uint64_t *off;
    uint64_t n;
    const uint8_t *seqB;      /* rect mode: second read set */
    const uint64_t *offB;
    uint64_t a0, a1, b0, b1, ld;
    const uint64_t *pi, *pj;  /* pairs mode */
    uint64_t npairs;
    uint16_t *out;
    int32_t *out_score;       /* pairs mode: raw scores S instead of distances */
    int match, mismatch, gap, gap_open;
    int conversion;           /* score-to-distance rule (0 = max(la, lb) - S) */
    int mode;                 /* 0 = triangle rows, 1 = pair list, 2 = rectangle rows */
    uint64_t next;            /* shared work counter */
} job_t;

static uint64_t take(job_t *J, uint64_t chunk)
{
    return __atomic_fetch_add(&J->next, chunk, __ATOMIC_RELAXED);
}

static void *worker(void *arg)
{
    job_t *J = (job_t *)arg;
    if (J->mode == 0) {
        for (;;) {
            uint64_t i = take(J, 1);
            if (i >= J->n) break;
            const uint8_t *a = J->seq + J->off[i];
            int64_t la = (int64_t)(J->off[i + 1] - J->off[i]);
            for (uint64_t j = i + 1; j < J->n; ++j) {
                const uint8_t *b = J->seq + J->off[j];
                int64_t lb = (int64_t)(J->off[j + 1] - J->off[j]);
                J->out[oracle_tri_index(i, j, J->n)] = (uint16_t)oracle_distance_conv(
                    a, la, b, lb, J->match, J->mismatch, J->gap, J->gap_open, J->conversion);
            }
        }
    } else if (J->mode == 1) {
        for (;;) {
            uint64_t p0 = take(J, 64);
            if (p0 >= J->npairs) break;
            uint64_t p1 = p0 + 64 < J->npairs ? p0 + 64 : J->npairs;
            for (uint64_t p = p0; p < p1; ++p) {
                uint64_t i = J->pi[p], j = J->pj[p];
                const uint8_t *a = J->seq + J->off[i];
                const uint8_t *b = J->seqB + J->offB[j];
                int64_t la = (int64_t)(J->off[i + 1] - J->off[i]);
                int64_t lb = (int64_t)(J->offB[j + 1] - J->offB[j]);
                if (J->out_score)
                    J->out_score[p] = score_of(a, la, b, lb, J->match, J->mismatch, J->gap_open, J->gap);
                else
                    J->out[p] = (uint16_t)oracle_distance_conv(a, la, b, lb, J->match, J->mismatch, J->gap,
                                                               J->gap_open, J->conversion);
            }
        }
    } else {
        for (;;) {
            uint64_t r = J->a0 + take(J, 1);
            if (r >= J->a1) break;
            const uint8_t *a = J->seq + J->off[r];
            int64_t la = (int64_t)(J->off[r + 1] - J->off[r]);
            for (uint64_t c = J->b0; c < J->b1; ++c) {
                const uint8_t *b = J->seqB + J->offB[c];
                int64_t lb = (int64_t)(J->offB[c + 1] - J->offB[c]);
                J->out[(r - J->a0) * J->ld + (c - J->b0)] = (uint16_t)oracle_distance_conv(
                    a, la, b, lb, J->match, J->mismatch, J->gap, J->gap_open, J->conversion);
            }
        }
    }
    return NULL;
}

static int run(job_t *J, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return -1;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, worker, J) != 0) break;
        ++started;
    }
    if (started == 0) worker(J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    return 0;
}

/* All pairs i < j of one read set into the strict upper triangle out[n(n-1)/2]. */
int oracle_all_pairs(const uint8_t *seq, const uint64_t *off, uint64_t n, uint16_t *out,
                     int match, int mismatch, int gap, int gap_open, int conversion, int nthreads)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.seq = seq; J.off = off; J.n = n; J.out = out;
    J.match = match; J.mismatch = mismatch; J.gap = gap; J.gap_open = gap_open; J.mode = 0;
    J.conversion = conversion;
    return run(&J, nthreads);
}

/* Listed pairs: out[p] = d(A[pi[p]], B[pj[p]]) under the given conversion rule. */
int oracle_pairs(const uint8_t *seqA, const uint64_t *offA, const uint8_t *seqB,
                 const uint64_t *offB, const uint64_t *pi, const uint64_t *pj, uint64_t npairs,
                 uint16_t *out, int match, int mismatch, int gap, int gap_open, int conversion,
                 int nthreads)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.seq = seqA; J.off = offA; J.seqB = seqB; J.offB = offB;
    J.pi = pi; J.pj = pj; J.npairs = npairs; J.out = out;
    J.match = match; J.mismatch = mismatch; J.gap = gap; J.gap_open = gap_open; J.mode = 1;
    J.conversion = conversion;
    return run(&J, nthreads);
}

/* Listed pairs, raw local scores: out[p] = S(A[pi[p]], B[pj[p]]). */
int oracle_pair_scores(const uint8_t *seqA, const uint64_t *offA, const uint8_t *seqB,
                       const uint64_t *offB, const uint64_t *pi, const uint64_t *pj,
                       uint64_t npairs, int32_t *out, int match, int mismatch, int gap,
                       int gap_open, int nthreads)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.seq = seqA; J.off = offA; J.seqB = seqB; J.offB = offB;
    J.pi = pi; J.pj = pj; J.npairs = npairs; J.out_score = out;
    J.match = match; J.mismatch = mismatch; J.gap = gap; J.gap_open = gap_open; J.mode = 1;
    return run(&J, nthreads);
}

/* Rectangle: out[(r-a0)*ld + (c-b0)] = d(A[r], B[c]) for r in [a0,a1), c in [b0,b1). */
int oracle_rect(const uint8_t *seqA, const uint64_t *offA, uint64_t a0, uint64_t a1,
                const uint8_t *seqB, const uint64_t *offB, uint64_t b0, uint64_t b1,
                uint16_t *out, uint64_t ld, int match, int mismatch, int gap, int gap_open,
                int conversion, int nthreads)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.seq = seqA; J.off = offA; J.seqB = seqB; J.offB = offB;
    J.a0 = a0; J.a1 = a1; J.b0 = b0; J.b1 = b1; J.ld = ld; J.out = out;
    J.match = match; J.mismatch = mismatch; J.gap = gap; J.gap_open = gap_open; J.mode = 2;
    J.conversion = conversion;
    return run(&J, nthreads);
}
