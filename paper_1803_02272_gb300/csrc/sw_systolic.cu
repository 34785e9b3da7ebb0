// Warp-systolic int16x2 Smith-Waterman kernel (the hot path).
//
// What it computes: the local alignment score S of section 2.2 (Smith-Waterman,
// match +1, mismatch -1, linear gap 1) for one query read against a stream of
// subject reads, then the distance d = max(la, lb) - S.
//
// Layout of the work (one warp = one work unit = one query vs many subjects):
//  * Lane k owns query rows [kR, kR+R) (R = ceil(la/32) <= 16).  Subjects flow through
//    the warp as a stream of columns; lane k runs 16 steps behind lane k-1, so the value
//    of lane k-1's last row reaches lane k by a warp shuffle, 16-R steps late when R < 16
//    (the sending row keeps its last 16 outputs in registers).  The two 16-bit halves of every register carry two independent
//    subject streams (int16x2 SIMD).
//  * Within a lane, row r at local step u handles stream column u - r, so the R cells a
//    lane updates per step lie on one anti-diagonal and are independent.
//  * Scores are biased by the anti-diagonal: K(i,j) = H(i,j) + i + j + C.  The textbook
//    recurrence H = max(0, H_d + s, H_u - 1, H_l - 1) becomes
//        K = max(f, K_d + s + 2, K_u, K_l),    f = i + j + C  (the "zero" of the local
//    alignment), i.e. one __viaddmax_s16x2 and one __vimax3_s16x2 per two cells.
//  * s + 2 comes from a score profile in shared memory: for each query base q and
//    stream column j, SP[q][j] = (s(q, b_lo[j]) + 2, s(q, b_hi[j]) + 2) as int16x2, or a
//    large negative value where the column is padding.  The profile is a ring of 48
//    chunks of 16 columns, refilled one chunk ahead by the whole warp with one byte
//    permutation per word (the selectors are built once per 16 chunks); each lane reads
//    it with 64-bit loads two steps at a time (a row's column advances by one per step).
//  * Subjects start on 16-column chunk boundaries (a subject's 2-bit packed word = one
//    chunk).  At a subject's first column, a row's left and diagonal inputs are reset to
//    the floor (H(i,0) = 0) with one masked LOP3 per row per chunk.
//  * S = max(K - f) is tracked per step (rows of the current and of the previous column
//    chunk separately), folded per subject, and combined across lanes with a shuffle
//    chain; lane 31 writes the converted distance.
// Values are kept in [~1000, ~10700] by rebasing every 8192 steps, so int16 never
// overflows and 0 acts as minus infinity.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>

#include "gbd_internal.cuh"
#include "sw_systolic.cuh"

namespace gbd {
namespace {

constexpr int LANES = 32;
constexpr int CH = 16;                       // steps per chunk == lane skew
// >= 34 chunks are live at once; 48 chunks of 18 words make the ring 864 words, a
// multiple of the 32 banks, so the lanes' 18-word stride stays conflict-free across the
// ring's wrap.
constexpr int RING_CHUNKS = 48;
constexpr int RING = RING_CHUNKS * CH;       // 768 columns
constexpr int SLOTS = RING + 3 * CH;         // ring index in [-16, RING + 32)
// +2 pad words per 16 columns; arrays start on 32-word (128-byte) boundaries so every
// lane's bank position depends on its column alone
constexpr int PWORDS = (SLOTS + 2 * (SLOTS / 16) + 31) & ~31;
constexpr int NARR = 4;                      // per-warp profiles for A, C, G, T
constexpr int TABLE_WORDS = RING_CHUNKS * 4; // per chunk: 4 words of stream metadata
constexpr int TABLE_OFF = NARR * PWORDS;
// Profile selectors of the 16 chunks described last: per chunk 16 columns x 16 bits
constexpr int SEL_WORDS = 16 * 8;
constexpr int SEL_OFF = TABLE_OFF + TABLE_WORDS;
constexpr int WARP_WORDS = SEL_OFF + SEL_WORDS;
constexpr int WARPS_PER_BLOCK = 2;
constexpr uint32_t NEG2 = 0xC000C000u;       // (-16384, -16384)
constexpr int C0 = 1536;                     // floor offset: f >= ~1000 for every lane
constexpr uint32_t ONE2 = 0x00010001u;
constexpr int REBASE_CHUNKS = 512;           // 8192 steps
constexpr uint32_t REBASE2 = 0x20002000u;    // 8192 in both halves
static_assert(PWORDS % 32 == 0, "profile arrays are 128-byte aligned");
static_assert((REBASE_CHUNKS & (REBASE_CHUNKS - 1)) == 0, "rebase period is a power of two");
static_assert(TABLE_OFF % 4 == 0 && SEL_OFF % 32 == 0 && WARP_WORDS % 32 == 0,
              "table, selector and warp regions stay bank-aligned");
// One never-matching profile per block serves the query rows past a read's end.
constexpr int NEG_OFF = WARPS_PER_BLOCK * WARP_WORDS;
constexpr int BLOCK_WORDS = NEG_OFF + PWORDS;
constexpr int BLOCKS_PER_SM = 6;
static_assert((RING_CHUNKS * 18) % 32 == 0, "ring length is a multiple of the banks");

// padded word index of ring slot rho (rho in [-16, RING + 32))
__host__ __device__ constexpr int pslot(int rho) { return (rho + 16) + 2 * ((rho + 16) >> 4); }
// offset (in words) of relative column e in [-16, 17] from a chunk base P0
__host__ __device__ constexpr int poff(int e) { return e < 0 ? e - 2 : (e < 16 ? e : e + 2); }
__device__ __forceinline__ int chunk_P0(int c)
{
    int m = c % RING_CHUNKS;
    if (m < 0) m += RING_CHUNKS;
    return 18 * m + 18;       // == pslot(16 * m)
}

__device__ __forceinline__ uint32_t vmax3(uint32_t a, uint32_t b, uint32_t c) { return __vimax3_s16x2(a, b, c); }
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) { return __vmaxs2(a, b); }
__device__ __forceinline__ uint32_t vaddmax(uint32_t a, uint32_t b, uint32_t c) { return __viaddmax_s16x2(a, b, c); }
// (v, v) packed as int16x2 for a small signed v; building it as v * 0x00010001 would let
// a negative low half borrow from the high half.
__host__ __device__ constexpr uint32_t pack2(int v) { return ((uint32_t)v & 0xffffu) * 0x00010001u; }

__device__ __forceinline__ uint32_t lop_sel(uint32_t keep, uint32_t repl, uint32_t mask)
{
    return (keep & ~mask) | (repl & mask);
}

// One warp's work: a piece of an entry.
struct SysUnit {
    uint32_t job, q, sub_begin, nsub;
};

// Stream descriptors.  Half h of the stream (h = 0: the low 16 bits of every register,
// h = 1: the high 16 bits) takes the unit's subjects at list positions h, h+2, h+4, ...;
// each subject fills ceil(len/16) chunks of 16 columns (an empty subject one padding
// chunk) and a finished half continues with padding chunks.  Every 16 chunks the warp
// describes the next 16 chunks of both halves at once: lane t of half h (lanes 0-15:
// h = 0, lanes 16-31: h = 1) works out chunk 16b + t of half h from the subject lengths
// by a prefix sum over the half's lanes, writes the chunk's metadata into the table, and
// writes the chunk's profile selectors (below) for the refill.
//
// Profile selectors.  The profile word of query base q and column x is the byte
// permutation of T_q = (bytes c = 0..3: 3 if c == q else 1, i.e. s(q, c) + 2) and
// Y = 0x0000C000 that the column's 16-bit selector picks: per half, a selector byte
// 0x60 | code takes T_q's byte `code` and a zero high byte (s + 2 as int16), and 0x54 (a
// column past the subject's end) takes 0x00 and 0xC0 (the never-matching -16384).  The
// selector bytes of four columns are built at once from the packed word, and the two
// halves of a column are interleaved (low half's byte, then high half's) so that a column's
// selector is one 16-bit word.
struct HalfCursor {
    uint32_t pos;      // list position (within the half) of the subject of chunk 16b
    uint32_t ck;       // chunk of that subject
    uint32_t cnt;      // subjects in the half
};

// Describes chunks [b16, b16 + 16) of this lane's half.  tslot = b16 mod RING_CHUNKS (the
// table slot of chunk b16; b16 is a multiple of 16, so tslot + t never wraps).  Sets C to
// the first chunk where both halves are padding, once such a chunk appears.
__device__ __forceinline__ void describe_chunks(const SysJob &J, const SysUnit &u, int lane, HalfCursor &hc,
                                                uint32_t b16, int tslot, uint32_t *table, uint32_t *sel, int &C)
{
    const uint32_t t = lane & 15, h = lane >> 4;
    // the subject t positions after the current one
    const uint32_t pt = hc.pos + t;
    uint32_t orig = 0, len = 0, nch = 1u << 16;          // past the end: one endless padding run
    if (pt < hc.cnt) {
        const uint32_t li = u.sub_begin + h + 2 * pt;
        orig = J.sub_perm ? __ldg(J.sub_perm + li) : li;
        len = __ldg(J.S.len + orig);
        nch = max(1u, (len + 15u) >> 4);
    }
    // E = chunk (relative to b16) that follows subject pt: inclusive prefix sum of the
    // chunk counts, the current subject's consumed chunks taken off
    uint32_t E = nch - (t == 0 ? hc.ck : 0u);
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, E, d, 16);
        if (t >= (uint32_t)d) E += o;
    }
    // E >= t + 1 for every lane, so the subject of chunk b16 + t is the number of subject
    // ends at relative chunks <= t (never more than t), and it starts at the last of them
    const uint32_t mark = E < 16u ? (1u << (E + 16u * h)) : 0u;
    const uint32_t ends = (__reduce_or_sync(0xffffffffu, mark) >> (16u * h)) & ((2u << t) - 1u);
    const uint32_t si = __popc(ends);
    const uint32_t start = ends ? 31u - __clz(ends) : 0u;
    const uint32_t ckt = t - start + (si == 0 ? hc.ck : 0u);
    const uint32_t slen = __shfl_sync(0xffffffffu, len, (int)si, 16);
    const uint32_t sorig = __shfl_sync(0xffffffffu, orig, (int)si, 16);
    const uint32_t p = hc.pos + si;
    const bool valid = p < hc.cnt;
    const uint32_t rem = slen - 16u * ckt;
    const bool first = valid && ckt == 0;
    const bool last = valid && rem <= 16u;
    const uint32_t nv = valid ? min(16u, rem) : 0u;
    const uint32_t word = valid ? __ldg(J.S.words + (uint64_t)sorig * J.S.stride + ckt) : 0u;
    // selector bytes of this half: byte i of B[j] belongs to column 4j + i
    {
        const uint32_t wm = nv >= 16u ? word : (word & ((1u << (2u * nv)) - 1u));   // past-end codes 0
        const uint32_t nvb = nv * 0x01010101u;
        uint32_t B[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t y = (wm >> (8 * j)) & 0xffu;              // codes of columns 4j..4j+3
            const uint32_t v = (y | (y << 12)) & 0x000f000fu;        // two columns per 16 bits
            const uint32_t c = (v | (v << 6)) & 0x03030303u;         // one column per byte
            // 0x80 + column - nv per byte (no borrow: it stays in [0x70, 0x8f]); bit 7 = past the end
            const uint32_t past = (((0x80808080u + 0x04040404u * (uint32_t)j + 0x03020100u) - nvb) >> 7) & 0x01010101u;
            B[j] = c ^ (past * 0x34u) ^ 0x60606060u;                 // 0x60 | code, or 0x54
        }
        // interleave with the other half's bytes: the low half's lanes keep columns 4j, 4j+1,
        // the high half's 4j+2, 4j+3, as word 2j + h of the chunk's 8 (selector slot t)
        const uint32_t perm = h ? 0x3726u : 0x5140u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t other = __shfl_xor_sync(0xffffffffu, B[j], 16);
            const int wi = 8 * (int)t + 2 * j + (int)h;
            if (bounds_ok((uint64_t)wi, SEL_WORDS, BOUNDS_SYSTOLIC_RING)) sel[wi] = __byte_perm(B[j], other, perm);
        }
    }
    // the table entry of chunk b16 + t joins both halves: exchange with lane t ^ 16
    const uint32_t fa = (first ? 1u : 0u) | (last ? 2u : 0u);
    const uint32_t fb = (valid ? slen : 0u) | (p << 16);
    const uint32_t ga = __shfl_xor_sync(0xffffffffu, fa, 16);
    const uint32_t gb = __shfl_xor_sync(0xffffffffu, fb, 16);
    const uint32_t alo = h ? ga : fa, ahi = h ? fa : ga;
    const uint32_t blo = h ? gb : fb, bhi = h ? fb : gb;
    if (h == 0) {
        uint4 e;
        e.x = ((alo & 1u) ? 0x0000ffffu : 0u) | ((ahi & 1u) ? 0xffff0000u : 0u);
        e.y = ((alo & 2u) ? 0x0000ffffu : 0u) | ((ahi & 2u) ? 0xffff0000u : 0u);
        e.z = (blo & 0xffffu) | (bhi << 16);
        e.w = (blo >> 16) | (bhi & 0xffff0000u);
        if (bounds_ok((uint64_t)(tslot + (int)t), RING_CHUNKS, BOUNDS_SYSTOLIC_RING))
            *reinterpret_cast<uint4 *>(table + 4 * (tslot + (int)t)) = e;
    }
    // state at chunk b16 + 16, from the half's lane 15
    const uint32_t nxt = last ? (p + 1u) : (p | (valid ? (ckt + 1u) << 16 : 0u));
    const uint32_t n15 = __shfl_sync(0xffffffffu, nxt, 15, 16);
    hc.pos = n15 & 0xffffu;
    hc.ck = n15 >> 16;
    // first chunk where both halves are padding
    const uint32_t vb = __ballot_sync(0xffffffffu, valid);
    const uint32_t both = ~(vb | (vb >> 16)) & 0xffffu;
    if (C < 0 && both != 0u) C = (int)b16 + __ffs(both) - 1;
}

// Write chunk X of the two half streams into the warp's profile ring (slot m = X mod
// RING_CHUNKS) from its selectors (selector slot X mod 16): lane x and lane x + 16 take
// column x, the first for bases A and C, the second for G and T.  Ring slot rho = 16m + x
// sits at padded word pslot(rho) = 18(m + 1) + x; slots 0 and 1 are also written one ring
// length on, slot RING_CHUNKS - 1 one ring length back.
__device__ __forceinline__ void fill_chunk(uint32_t *ws, int lane, int m, int slot, const uint32_t (&Tq)[2])
{
    const int x = lane & 15;
    const uint32_t q = (uint32_t)(lane >> 4) * 2u;
    const int si = 16 * slot + x;
    uint32_t sel = 0x5454u;
    if (bounds_ok((uint64_t)si, 2 * SEL_WORDS, BOUNDS_SYSTOLIC_RING))
        sel = reinterpret_cast<const uint16_t *>(ws + SEL_OFF)[si];
    const int w = 18 * m + 18 + x;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const uint32_t v = __byte_perm(Tq[t], 0x0000C000u, sel);
        uint32_t *arr = ws + (q + (uint32_t)t) * PWORDS;
        if (bounds_ok((uint64_t)w, PWORDS, BOUNDS_SYSTOLIC_RING)) arr[w] = v;
        if (m < 2 && bounds_ok((uint64_t)(w + 18 * RING_CHUNKS), PWORDS, BOUNDS_SYSTOLIC_RING))
            arr[w + 18 * RING_CHUNKS] = v;
        if (m == RING_CHUNKS - 1 && bounds_ok((uint64_t)(w - 18 * RING_CHUNKS), PWORDS, BOUNDS_SYSTOLIC_RING))
            arr[w - 18 * RING_CHUNKS] = v;
    }
}
static_assert(pslot(16 * 5 + 7) == 18 * 6 + 7 && pslot(16 * RING_CHUNKS + 15) == 18 * (RING_CHUNKS + 1) + 15 &&
              pslot(-16) == 0 && pslot(16 * 1 + 15 + RING) == 18 * (1 + 1) + 15 + 18 * RING_CHUNKS,
              "ring slot 16m + x sits at padded word 18(m + 1) + x");

__device__ __forceinline__ uint2 lds64(const uint32_t *ws_words, uint32_t byte_off)
{
    return *reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(ws_words) + byte_off);
}

template <int R, bool AFFINE>
__device__ __forceinline__ void run_unit(const SysJob &J, const SysUnit &u, uint32_t *ws, int lane,
                                      int neg_rel, int ws_words, uint32_t *err)
{
    (void)ws_words;                           // the warp region's offset (bounds-checked builds)
    constexpr int D = CH - R;                 // delay steps between lanes
    const int la = J.Q.len[u.q];
    const uint32_t *qwords = J.Q.words + (uint64_t)u.q * J.Q.stride;

    // ---- stream descriptors of chunks 0..15 and the first chunk of the ring
    int C = -1;                                // stream length in chunks, once known
    HalfCursor hc;
    hc.pos = 0;
    hc.ck = 0;
    hc.cnt = (u.nsub + 1 - (uint32_t)(lane >> 4)) >> 1;   // half h: list positions h, h+2, ...
    uint32_t *const table = ws + TABLE_OFF;
    uint32_t *const sel = ws + SEL_OFF;
    int tslot = 0;                             // table slot of the first of the 16 chunks
    // T_q of this lane's two base codes (lanes 0-15: codes 0 and 1; lanes 16-31: 2 and 3)
    const uint32_t Tq[2] = {0x01010101u + (2u << (16u * (uint32_t)(lane >> 4))),
                            0x01010101u + (0x200u << (16u * (uint32_t)(lane >> 4)))};
    // Lane k meets chunks -k..-1 (before the stream reaches it) in table slots 48-k..47;
    // the describes first overwrite those slots after every lane has left them (slots
    // 16..31 when chunk 16 is refilled, 32..47 at chunk 32).  Their entry starts no subject
    // and ends one in both halves, so that each lane's chunk 0 begins with a cleared maximum.
#pragma unroll
    for (int w = 16 * 4 + lane; w < RING_CHUNKS * 4; w += 32) table[w] = ((w & 3) == 1) ? 0xffffffffu : 0u;
    describe_chunks(J, u, lane, hc, 0u, 0, table, sel, C);
    __syncwarp();
    fill_chunk(ws, lane, 0, 0, Tq);
    __syncwarp();

    // ---- per-row profile addresses
    uint32_t addr[R];
    {
        const int P0 = chunk_P0(-lane);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int pos = lane * R + r;
            uint32_t code = 4;
            if (pos < la) code = (__ldg(qwords + (pos >> 4)) >> (2 * (pos & 15))) & 3u;
            addr[r] = ((code < 4 ? (int)code * PWORDS : neg_rel) + P0) * 4u;
        }
    }

    // ---- registers of the systolic state
    const int fk0 = 1 + C0 - lane * D;         // floor of this lane at global step 0
    uint32_t f_prev2 = (uint32_t)(fk0 - 2) * ONE2;
    uint32_t f_prev = (uint32_t)(fk0 - 1) * ONE2;
    uint32_t V0[R], V1[R];                     // V0: even local steps, V1: odd
#pragma unroll
    for (int r = 0; r < R; ++r) { V1[r] = f_prev; V0[r] = f_prev2; }
    // Row R-1 of lane k reaches lane k+1 after 1 + D steps.  With D > 0 the row keeps its
    // outputs of the last 16 steps in hist[step in chunk] (static register names, no
    // copies) and the next lane shuffles the entry it needs directly; with D == 0 the
    // row lives in V0/V1 like the others.
    constexpr bool HIST = D > 0;
    uint32_t hist[HIST ? CH : 1];
#pragma unroll
    for (int i = 0; i < (HIST ? CH : 1); ++i) hist[i] = f_prev;
    // Affine gaps (open `gap_open`, extend 1), in the same bias: Eh = E + f carries a
    // horizontal gap along each row, Fh = F + f a vertical one down the column,
    //   Eh = max(Eh_left, K_left - gap_open), Fh = max(Fh_up, K_up - gap_open),
    //   K = max(f, K_diag + s + 2, Eh, Fh);
    // minus infinity is NEG2.  Fh of a lane's last row reaches the next lane like K does
    // (histF when D > 0).
    constexpr int NA = AFFINE ? R : 1;
    constexpr bool HISTF = AFFINE && HIST;
    uint32_t Eh[NA], Fh[NA];
    uint32_t histF[HISTF ? CH : 1];
#pragma unroll
    for (int r = 0; r < NA; ++r) { Eh[r] = NEG2; Fh[r] = NEG2; }
#pragma unroll
    for (int i = 0; i < (HISTF ? CH : 1); ++i) histF[i] = NEG2;
    const uint32_t ngo = AFFINE ? pack2(-(int)J.gap_open) : 0u;
    uint32_t up0_prev = f_prev2;               // row 0's diagonal input
    uint32_t curRel = 0, prevRel = 0, acc = 0, emit = 0;
    uint32_t Mlast_prev = 0xffffffffu;         // "ends a subject" masks of chunk c-1
    uint32_t lens_prev = 0, pos_prev = 0;
    uint2 sp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e0 = (r & 1) ? -r - 1 : -r;
        sp[r] = lds64(ws, addr[r] + 4 * poff(e0));
    }
    // ring slots (mod RING_CHUNKS) of the chunk being filled and of this lane's chunk
    int m_fill = 1;
    int m_c = (RING_CHUNKS - lane % RING_CHUNKS) % RING_CHUNKS;

    // Linear gaps: two chunks per iteration.  The second one's profile columns lie 18
    // words (72 bytes) after the first one's, so it reads them at immediate offsets, and
    // the loop test, the rebase check and the per-row address advance run once per 32
    // steps.  Reading one chunk past the ring's last slot lands in the copy of slot 0 that
    // every fill of slot 0 also writes.  An extra padding chunk at the end (C + LANES odd)
    // emits nothing.  Affine gaps keep one chunk per iteration: their loop body is twice
    // as long, and doubling it again cost more (registers, instruction fetch) than the
    // loop overhead it saves.
    constexpr int PAIR = AFFINE ? 1 : 2;
    for (int g0 = 0; C < 0 || g0 < C + LANES; g0 += PAIR) {
        // ---- rebase every REBASE_CHUNKS chunks (all lanes at the same global step)
        if (g0 > 0 && (g0 & (REBASE_CHUNKS - 1)) == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) { V0[r] -= REBASE2; V1[r] -= REBASE2; }
#pragma unroll
            for (int i = 0; i < (HIST ? CH : 1); ++i) hist[i] -= REBASE2;
            up0_prev -= REBASE2; f_prev -= REBASE2; f_prev2 -= REBASE2;
            prevRel -= REBASE2;               // curRel is 0 (minus infinity) here
            if (AFFINE) {                     // saturating: minus infinity stays very negative
#pragma unroll
                for (int r = 0; r < NA; ++r) { Eh[r] = __vsubss2(Eh[r], REBASE2); Fh[r] = __vsubss2(Fh[r], REBASE2); }
#pragma unroll
                for (int i = 0; i < (HISTF ? CH : 1); ++i) histF[i] = __vsubss2(histF[i], REBASE2);
            }
        }

        const int m_c1 = (m_c == RING_CHUNKS - 1) ? 0 : m_c + 1;   // table slot of the second chunk
#if GBD_BOUNDS_CHECK
        // the words a row reads in these two chunks: from 18 before its chunk base to 38
        // after it (the second chunk's last 64-bit load); a window leaving the block's shared
        // memory is moved onto the block's padding profile
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (!bounds_ok((uint64_t)(ws_words + (int)(addr[r] / 4u) + 38), BLOCK_WORDS, BOUNDS_SYSTOLIC_RING))
                addr[r] = (uint32_t)((neg_rel + 18) * 4);
#endif
#pragma unroll
        for (int h2 = 0; h2 < PAIR; ++h2) {
            const int g = g0 + h2;
            // ---- refill: chunk g+1 into the ring (describing the next 16 chunks first when
            // g+1 starts them; g+1 is odd for the first chunk of the pair)
            if ((PAIR == 1 || h2 == 1) && ((g + 1) & 15) == 0) {
                tslot = (tslot == RING_CHUNKS - 16) ? 0 : tslot + 16;
                describe_chunks(J, u, lane, hc, (uint32_t)(g + 1), tslot, table, sel, C);
                __syncwarp();
            }
            fill_chunk(ws, lane, m_fill, (g + 1) & 15, Tq);
            m_fill = (m_fill == RING_CHUNKS - 1) ? 0 : m_fill + 1;
            __syncwarp();

            // ---- this lane's chunk c: stream metadata
            const int c = g - lane;
            const uint4 ev = *reinterpret_cast<const uint4 *>(table + 4 * (h2 ? m_c1 : m_c));
            const uint32_t Mfirst = ev.x, Mlast_c = ev.y, lens_c = ev.z, pos_c = ev.w;
            const uint32_t Mend = Mlast_prev;            // chunk c-1 ended a subject (c <= 0: all ones)
            const uint32_t fbase = f_prev + ONE2;         // floor at step 0 of this chunk

            // ---- 16 steps
#pragma unroll
            for (int q = 0; q < CH; ++q) {
                uint32_t *cur = (q & 1) ? V0 : V1;        // V(u-1)
                uint32_t *nxt = (q & 1) ? V1 : V0;        // V(u-2) in, V(u) out
                const uint32_t f = f_prev + ONE2;
                // row R-1 of lane k-1, produced 1 + D steps ago
                uint32_t up0 = __shfl_up_sync(0xffffffffu,
                                              HIST ? hist[(q + CH - 1 - D) & (CH - 1)] : cur[R - 1], 1);
                if (lane == 0) up0 = f_prev;              // top boundary: H(0, j) = 0
                uint32_t fup0 = 0u;
                if (AFFINE) {
                    fup0 = __shfl_up_sync(0xffffffffu, HISTF ? histF[(q + CH - 1 - D) & (CH - 1)] : Fh[R - 1], 1);
                    if (lane == 0) fup0 = NEG2;           // F(0, j) = minus infinity
                }
                uint32_t diag0 = up0_prev;
#pragma unroll
                for (int r = R - 1; r >= 0; --r) {
                    // this row's value one step ago (left input) and its new value
                    uint32_t &left = (HIST && r == R - 1) ? hist[(q + CH - 1) & (CH - 1)] : cur[r];
                    uint32_t &out = (HIST && r == R - 1) ? hist[q] : nxt[r];
                    if (r == q) {
                        // row q reaches a subject's first column: its left input (and, for
                        // row 0, its diagonal) become the floor of column 0.  Rows below
                        // already read the old value as their "up" input this step.
                        left = lop_sel(left, f_prev, Mfirst);
                        if (AFFINE) Eh[r] = lop_sel(Eh[r], NEG2, Mfirst);      // E(i, 0) = -inf
                        if (r == 0) diag0 = lop_sel(diag0, f_prev2, Mfirst);
                    }
                    const uint32_t up = r ? cur[r - 1] : up0;
                    const uint32_t dg = r ? nxt[r - 1] : diag0;
                    const uint32_t s2 = (((q - r) & 1) == 0) ? sp[r].x : sp[r].y;
                    const uint32_t E = vaddmax(dg, s2, f);
                    if (AFFINE) {
                        const uint32_t fu = r ? Fh[r - 1] : fup0;
                        const uint32_t eh = vaddmax(left, ngo, Eh[r]);
                        const uint32_t fh = vaddmax(up, ngo, fu);
                        out = vmax3(E, eh, fh);
                        Eh[r] = eh;
                        if (HISTF && r == R - 1) histF[q] = fh; else Fh[r] = fh;
                    } else {
                        out = vmax3(up, left, E);
                    }
                    if (((q - r) & 1) != 0) sp[r] = lds64(ws, addr[r] + 72u * h2 + 4 * poff(q + 1 - r));
                }
                up0_prev = up0;
                // best: rows <= q are in column chunk c, rows > q in chunk c-1
                {
                    const int nN = (q < R - 1 ? q : R - 1) + 1;
                    auto val = [&](int r) -> uint32_t { return (HIST && r == R - 1) ? hist[q] : nxt[r]; };
                    uint32_t mN = val(0);
#pragma unroll
                    for (int r = 1; r < R; r += 2) {
                        if (r < nN) {
                            if (r + 1 < nN) mN = vmax3(mN, val(r), val(r + 1));
                            else mN = vmax2(mN, val(r));
                        }
                    }
                    curRel = vaddmax(mN, pack2(-q), curRel);
                    if (nN < R) {
                        uint32_t mO = val(nN);
#pragma unroll
                        for (int r = 1; r < R; r += 2) {
                            const int a = nN + r, b = nN + r + 1;
                            if (a < R) {
                                if (b < R) mO = vmax3(mO, val(a), val(b));
                                else mO = vmax2(mO, val(a));
                            }
                        }
                        prevRel = vaddmax(mO, pack2(-q), prevRel);
                    }
                }
                f_prev2 = f_prev;
                f_prev = f;
            }

            // ---- chunk end: fold chunk c-1, pass totals down the lanes, write results
            {
                uint32_t recv = __shfl_up_sync(0xffffffffu, emit, 1);
                if (lane == 0) recv = 0;
                const uint32_t negfb = __vsub2(0u, fbase);                 // -fbase in both halves
                const uint32_t a = vaddmax(prevRel, negfb, acc);       // max(acc, prev - fbase)
                const uint32_t total = vmax2(a, recv);
                emit = lop_sel(emit, total, Mend);
                acc = a & ~Mend;
                prevRel = curRel + 16u * ONE2;
                curRel = 0;
                if (lane == LANES - 1 && c >= 1 && Mend != 0) {
                    const int conv = J.conversion;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if ((Mend >> (16 * h)) & 1u) {
                            const int S = (int)(int16_t)(total >> (16 * h));
                            const uint32_t li = u.sub_begin + h + 2 * ((pos_prev >> (16 * h)) & 0xffffu);
                            const uint32_t so = J.sub_perm ? __ldg(J.sub_perm + li) : li;
                            const int lb = (int)((lens_prev >> (16 * h)) & 0xffffu);
                            uint64_t idx;
                            if (J.mode == OUT_TRI) {
                                const uint64_t i = min((uint64_t)u.q, (uint64_t)so);
                                const uint64_t j = max((uint64_t)u.q, (uint64_t)so);
                                idx = i * J.n - i * (i + 1) / 2 + (j - i - 1) - J.out_base;
                            } else {
                                idx = ((uint64_t)u.q - J.row0) * J.ld + ((uint64_t)so - J.col0);
                            }
                            if (bounds_ok(idx, J.out_len, BOUNDS_SYSTOLIC_OUT))
                            J.out[idx] = score_to_distance(S, la, lb, conv);
                        }
                    }
                }
                Mlast_prev = Mlast_c;
                lens_prev = lens_c;
                pos_prev = pos_c;
            }
        }
        // ---- advance the profile addresses by the chunks of this iteration
        {
            const bool wrap = (m_c >= RING_CHUNKS - PAIR);
            const uint32_t d = wrap ? (uint32_t)(4 * 18 * (PAIR - RING_CHUNKS)) : (uint32_t)(4 * 18 * PAIR);
#pragma unroll
            for (int r = 0; r < R; ++r) addr[r] += d;
            m_c = wrap ? m_c + PAIR - RING_CHUNKS : m_c + PAIR;
        }
        (void)err;
    }
}

template <int R, bool AFFINE>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, (AFFINE && R > 12) ? BLOCKS_PER_SM - 1 : BLOCKS_PER_SM)
sw_systolic_kernel(const SysJob *__restrict__ jobs, const SysEntry *__restrict__ entries,
                   const uint32_t *__restrict__ prefix, uint32_t nentries, uint32_t nunits,
                   uint32_t piece_len, uint32_t *counter, uint32_t *err)
{
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    uint32_t *ws = smem + warp * WARP_WORDS;
    for (int i = threadIdx.x; i < BLOCK_WORDS; i += blockDim.x) smem[i] = NEG2;
    __syncthreads();
    const int neg_rel = NEG_OFF - warp * WARP_WORDS;   // block's padding profile, from ws
    for (;;) {
        uint32_t ui = 0;
        if (lane == 0) ui = atomicAdd(counter, 1u);
        ui = __shfl_sync(0xffffffffu, ui, 0);
        if (ui >= nunits) break;
        // entry e with prefix[e] <= ui < prefix[e+1]
        uint32_t lo = 0, hi = nentries;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(prefix + mid) <= ui) lo = mid; else hi = mid;
        }
        const SysEntry en = entries[lo];
        const uint32_t piece = ui - __ldg(prefix + lo);
        SysUnit u;
        u.job = en.job;
        u.q = en.q;
        u.sub_begin = en.sub_begin + piece * piece_len;
        u.nsub = min(piece_len, en.nsub - piece * piece_len);
        run_unit<R, AFFINE>(jobs[u.job], u, ws, lane, neg_rel, warp * WARP_WORDS, err);
        __syncwarp();
    }
}

// Blocks per SM of each instantiation (set up before any launch or capture).
int g_per_sm[2][17];

template <int R, bool AFFINE>
int prepare_bucket()
{
    const size_t smem = systolic_smem_bytes();
    GBD_CUDA_TRY(cudaFuncSetAttribute(sw_systolic_kernel<R, AFFINE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    int &bps = g_per_sm[AFFINE ? 1 : 0][R];
    GBD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sw_systolic_kernel<R, AFFINE>,
                                                                WARPS_PER_BLOCK * 32, smem));
    if (bps < 1) return fail(GBD_ECUDA, "systolic kernel does not fit on an SM");
    return GBD_OK;
}

template <int R, bool AFFINE>
int launch_bucket(const SysJob *d_jobs, const SysEntry *entries, const uint32_t *prefix,
                  uint32_t nentries, uint32_t nunits, uint32_t piece_len, uint32_t *counter,
                  uint32_t *err, int sm_count, cudaStream_t stream)
{
    const size_t smem = systolic_smem_bytes();
    uint64_t blocks = (uint64_t)sm_count * g_per_sm[AFFINE ? 1 : 0][R];
    const uint64_t need = (nunits + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK;
    if (blocks > need) blocks = need;
    sw_systolic_kernel<R, AFFINE><<<(unsigned)blocks, WARPS_PER_BLOCK * 32, smem, stream>>>(
        d_jobs, entries, prefix, nentries, nunits, piece_len, counter, err);
    note_launches(1);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return cuda_fail(le, "sw_systolic_kernel launch");
    return GBD_OK;
}

}  // namespace

size_t systolic_smem_bytes() { return (size_t)BLOCK_WORDS * sizeof(uint32_t); }

int systolic_prepare()
{
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lk(mu);
    if (done) return GBD_OK;
    int rc = GBD_OK;
#define GBD_CASE(RR) if (rc == GBD_OK) rc = prepare_bucket<RR, false>(); if (rc == GBD_OK) rc = prepare_bucket<RR, true>();
    GBD_CASE(1) GBD_CASE(2) GBD_CASE(3) GBD_CASE(4) GBD_CASE(5) GBD_CASE(6) GBD_CASE(7)
    GBD_CASE(8) GBD_CASE(9) GBD_CASE(10) GBD_CASE(11) GBD_CASE(12) GBD_CASE(13)
    GBD_CASE(14) GBD_CASE(15) GBD_CASE(16)
#undef GBD_CASE
    if (rc == GBD_OK) done = true;
    return rc;
}

// Subjects per work unit for one bucket, from a cost model of the launch: every unit
// pays the systolic pipeline's fill and drain (32 chunks of 16 steps) once, and the
// launch ends with a tail of about half a unit on the slowest warp.  With P pairs in the
// bucket, W resident warps and subjects of mean length L (so a unit of p subjects runs
// p*L/2 steps on two half streams), the time is proportional to
//     P*L/(2W) + (P/p)*512/W + p*L/4,
// minimised at p* = sqrt(2048*P / (W*L)).
uint32_t tuned_piece(uint64_t pairs, double mean_len, int warps)
{
    const double L = mean_len > 16.0 ? mean_len : 16.0;
    double p = std::sqrt(2048.0 * (double)pairs / ((double)std::max(warps, 1) * L));
    p = std::min(4096.0, std::max(64.0, p));
    return ((uint32_t)p + 31u) & ~31u;
}

int build_plan(const std::vector<SysEntry> &entries, const std::vector<uint8_t> &rows,
               SysPlan &plan, bool persistent, cudaStream_t stream, uint32_t piece_len,
               double mean_subject_len, int sm_count, double piece_scale)
{
    plan = SysPlan{};
    plan.piece = piece_len;
    std::vector<std::vector<SysEntry>> by_r(17);
    for (size_t i = 0; i < entries.size(); ++i) {
        if (entries[i].nsub == 0) continue;
        const int R = rows[i];
        if (R < 1 || R > 16) return fail(GBD_EINVAL, "internal: systolic query longer than 512");
        by_r[R].push_back(entries[i]);
    }
    // layout: for each bucket, entries (16 B each) then prefix (nentries + 1 words)
    size_t bytes = 0;
    std::vector<std::vector<uint32_t>> prefixes(17);
    const int warps = systolic_resident_warps(sm_count);
    for (int R = 16; R >= 1; --R) {          // launch order: widest rows first
        if (by_r[R].empty()) continue;
        SysPlan::Bucket b;
        b.R = R;
        b.nentries = (uint32_t)by_r[R].size();
        uint64_t pairs = 0;
        for (const SysEntry &e : by_r[R]) pairs += e.nsub;
        if (piece_len) {
            b.piece = piece_len;
        } else {
            const double p = (double)tuned_piece(pairs, mean_subject_len, warps) * piece_scale;
            b.piece = ((uint32_t)std::min(8192.0, std::max(32.0, p)) + 31u) & ~31u;
        }
        std::vector<uint32_t> &pf = prefixes[R];
        pf.resize(b.nentries + 1);
        uint64_t acc = 0;
        for (uint32_t e = 0; e < b.nentries; ++e) {
            pf[e] = (uint32_t)acc;
            acc += (by_r[R][e].nsub + b.piece - 1) / b.piece;
        }
        if (acc >= 0xffffffffull) return fail(GBD_EINVAL, "too many work units for one launch");
        pf[b.nentries] = (uint32_t)acc;
        b.nunits = (uint32_t)acc;
        b.entry_off = bytes;
        bytes += b.nentries * sizeof(SysEntry);
        b.prefix_off = bytes;
        bytes += (b.nentries + 1) * sizeof(uint32_t);
        bytes = (bytes + 15) & ~size_t(15);
        plan.buckets.push_back(b);
    }
    if (bytes == 0) return GBD_OK;
    std::vector<uint8_t> host(bytes);
    for (const auto &b : plan.buckets) {
        std::memcpy(host.data() + b.entry_off, by_r[b.R].data(), b.nentries * sizeof(SysEntry));
        std::memcpy(host.data() + b.prefix_off, prefixes[b.R].data(), (b.nentries + 1) * sizeof(uint32_t));
    }
    plan.stream_ordered = !persistent;
    if (persistent) {
        GBD_CUDA_TRY(cudaMalloc(&plan.d_buf, bytes));
    } else {
        GBD_CUDA_TRY(cudaMallocAsync(&plan.d_buf, bytes, stream));
    }
    GBD_CUDA_TRY(cudaMemcpyAsync(plan.d_buf, host.data(), bytes, cudaMemcpyHostToDevice, stream));
    if (persistent) GBD_CUDA_TRY(cudaStreamSynchronize(stream));
    return GBD_OK;
}

void free_plan(SysPlan &plan, cudaStream_t stream)
{
    if (plan.d_buf) {
        if (plan.stream_ordered) cudaFreeAsync(plan.d_buf, stream);
        else cudaFree(plan.d_buf);
    }
    plan = SysPlan{};
}

int run_systolic(const SysJob *d_jobs, const SysPlan &plan, int sm_count, cudaStream_t stream,
                 const StreamSet *ss, int naux, bool affine)
{
    if (plan.buckets.empty()) return GBD_OK;
    int prc = systolic_prepare();
    if (prc != GBD_OK) return prc;
    const size_t nb = plan.buckets.size();
    uint32_t *scratch = nullptr;                  // per bucket: work counter, error flags
    GBD_CUDA_TRY(cudaMallocAsync((void **)&scratch, 2 * nb * sizeof(uint32_t), stream));
    GBD_CUDA_TRY(cudaMemsetAsync(scratch, 0, 2 * nb * sizeof(uint32_t), stream));
    // Buckets alternate between `stream` and the aux streams, so the tail of one bucket's
    // launch overlaps the start of the next (a persistent grid starts where the other's
    // blocks have exited).  The streams fork and join on events.
    int extra = (ss == nullptr || nb < 2) ? 0 : std::min(naux, StreamSet::kMaxAux);
    extra = std::min<int>(extra, (int)nb - 1);
    if (extra > 0) {
        GBD_CUDA_TRY(cudaEventRecord(ss->fork, stream));
        for (int k = 0; k < extra; ++k) GBD_CUDA_TRY(cudaStreamWaitEvent(ss->aux[k], ss->fork, 0));
    }
    int rc = GBD_OK;
    for (size_t i = 0; i < nb && rc == GBD_OK; ++i) {
        const SysPlan::Bucket &b = plan.buckets[i];
        const char *base = static_cast<const char *>(plan.d_buf);
        const SysEntry *en = reinterpret_cast<const SysEntry *>(base + b.entry_off);
        const uint32_t *pf = reinterpret_cast<const uint32_t *>(base + b.prefix_off);
        uint32_t *ctr = scratch + 2 * i, *err = scratch + 2 * i + 1;
        const int lane_of = (int)(i % (size_t)(extra + 1));
        cudaStream_t st = lane_of == 0 ? stream : ss->aux[lane_of - 1];
        switch (b.R) {
#define GBD_CASE(RR) case RR: rc = affine ? launch_bucket<RR, true>(d_jobs, en, pf, b.nentries, b.nunits, b.piece, ctr, err, sm_count, st) \
                                         : launch_bucket<RR, false>(d_jobs, en, pf, b.nentries, b.nunits, b.piece, ctr, err, sm_count, st); break;
            GBD_CASE(1) GBD_CASE(2) GBD_CASE(3) GBD_CASE(4) GBD_CASE(5) GBD_CASE(6) GBD_CASE(7)
            GBD_CASE(8) GBD_CASE(9) GBD_CASE(10) GBD_CASE(11) GBD_CASE(12) GBD_CASE(13)
            GBD_CASE(14) GBD_CASE(15) GBD_CASE(16)
#undef GBD_CASE
            default: rc = fail(GBD_EINVAL, "internal: bad rows per lane");
        }
    }
    for (int k = 0; k < extra; ++k) {
        cudaEventRecord(ss->join[k], ss->aux[k]);
        cudaStreamWaitEvent(stream, ss->join[k], 0);
    }
    cudaError_t fe = cudaFreeAsync(scratch, stream);
    if (rc != GBD_OK) return rc;
    if (fe != cudaSuccess) return cuda_fail(fe, "cudaFreeAsync");
    return GBD_OK;
}

}  // namespace gbd

namespace gbd {
uint64_t bounds_take_systolic()
{
#if GBD_BOUNDS_CHECK
    unsigned long long v = ~0ull, reset = ~0ull;
    if (cudaMemcpyFromSymbol(&v, g_bounds_first, sizeof v) != cudaSuccess) v = ~0ull;
    cudaMemcpyToSymbol(g_bounds_first, &reset, sizeof reset);
    return v;
#else
    return ~0ull;
#endif
}

int systolic_resident_warps(int sm_count)
{
    // shared memory bound: BLOCKS_PER_SM blocks of WARPS_PER_BLOCK warps per SM
    return sm_count * BLOCKS_PER_SM * WARPS_PER_BLOCK;
}
}  // namespace gbd
