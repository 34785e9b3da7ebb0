"""Seeded synthetic amplicon reads shaped like the paper's Lake Geneva rbcL samples.

The paper's reads (Material and methods, "A sample from Lake Geneva") are not
available, so every workload here is synthetic: reads are mutated copies of a
small set of ancestral sequences, which gives the clustered structure ("islands
of high density") the paper reports.  This module holds input generation only:
no alignment, scoring or distance arithmetic lives here, so both the CUDA path
and the CPU oracle can be fed from it.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
k-th draw of stream s under seed S is mix64(key(S, s) + k * GAMMA).  Every draw
is addressable, so results do not depend on batch sizes or call order.

Mutation model (per ancestral base, in order):
  * with probability p_sub the base is replaced by a uniformly chosen *other* base;
  * else with probability p_indel an indel happens: half the time a uniform base
    is inserted before it, half the time it is deleted;
  * the mutated copy is then cut to the read's target length (prefix), or
    extended with uniform bases if it is shorter.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
ALPHABET = np.frombuffer(b"ACGT", dtype=np.uint8)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_sequence(seed: int, count: int) -> np.ndarray:
    """The first `count` outputs of a SplitMix64 generator started at `seed`.

    This is the published sequential definition (state += GAMMA, output
    mix64(state)); tests compare it with known reference outputs.
    """
    with np.errstate(over="ignore"):
        states = np.uint64(seed) + GAMMA * (np.arange(1, count + 1, dtype=np.uint64))
    return mix64(states)


class Stream:
    """One addressable stream of uniform 64-bit draws."""

    def __init__(self, seed: int, stream: int):
        with np.errstate(over="ignore"):
            k = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(stream))
        self.key = np.uint64(k)
        self.counter = 0

    def u64(self, shape) -> np.ndarray:
        n = int(np.prod(shape)) if shape != () else 1
        with np.errstate(over="ignore"):
            ctr = np.arange(self.counter, self.counter + n, dtype=np.uint64)
            out = mix64(self.key + ctr * GAMMA)
        self.counter += n
        return out.reshape(shape)

    def uniform(self, shape) -> np.ndarray:
        """Uniform doubles in [0, 1) with 53 random bits."""
        return (self.u64(shape) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, lo: int, hi: int, shape) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return (lo + np.floor(self.uniform(shape) * span)).astype(np.int64)

    def normal(self, shape) -> np.ndarray:
        """Standard normal doubles by the Box-Muller transform of two uniform draws."""
        u1 = self.uniform(shape)
        u2 = self.uniform(shape)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def log_uniform_int(self, lo: int, hi: int, shape) -> np.ndarray:
        """Integers whose logarithm is uniform on [ln lo, ln hi], rounded."""
        u = self.uniform(shape)
        v = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
        return np.clip(np.rint(v), lo, hi).astype(np.int64)


@dataclasses.dataclass
class ReadSet:
    """Reads as concatenated ASCII bytes plus offsets (read r = seq[off[r]:off[r+1]])."""

    seq: np.ndarray        # uint8, ASCII 'A','C','G','T'
    offsets: np.ndarray    # uint64, n+1 entries

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def read(self, r: int) -> bytes:
        return bytes(self.seq[int(self.offsets[r]):int(self.offsets[r + 1])])

    def subset(self, idx) -> "ReadSet":
        return from_strings([self.read(int(i)) for i in idx])

    def total_cells(self) -> int:
        """Sum over i<j of len_i * len_j (the all-pairs DP cell count)."""
        L = self.lengths.astype(np.float64)
        s = L.sum()
        return int(round((s * s - (L * L).sum()) / 2))


def from_strings(reads) -> ReadSet:
    bs = [r.encode() if isinstance(r, str) else bytes(r) for r in reads]
    offs = np.zeros(len(bs) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(b) for b in bs], dtype=np.uint64) if bs else []
    seq = np.frombuffer(b"".join(bs), dtype=np.uint8).copy() if bs else np.zeros(0, np.uint8)
    return ReadSet(seq=seq, offsets=offs)


def random_codes(st: Stream, shape) -> np.ndarray:
    """Uniform base codes 0..3 (A, C, G, T)."""
    return (st.u64(shape) >> np.uint64(62)).astype(np.uint8)


def mutate(st: Stream, parents: np.ndarray, parent_of: np.ndarray, target_len: np.ndarray,
           p_sub, p_indel) -> list[np.ndarray]:
    """Mutated copies of parent code arrays, one per entry of `parent_of`.

    parents: (P, Lp) uint8 codes; parent_of: (m,) indices; target_len: (m,) ints;
    p_sub / p_indel: scalars or (m,) arrays of per-copy rates.
    Returns a list of m uint8 code arrays with the requested lengths.
    """
    m = len(parent_of)
    if m == 0:
        return []
    Lp = parents.shape[1]
    p_sub = np.broadcast_to(np.asarray(p_sub, dtype=np.float64), (m,))[:, None]
    p_indel = np.broadcast_to(np.asarray(p_indel, dtype=np.float64), (m,))[:, None]
    src = parents[parent_of]                        # (m, Lp)
    u_event = st.uniform((m, Lp))
    u_sub = st.u64((m, Lp))
    u_ins = st.u64((m, Lp))
    u_base = random_codes(st, (m, Lp))
    is_sub = u_event < p_sub
    is_indel = (~is_sub) & (u_event < p_sub + p_indel)
    is_ins = is_indel & ((u_ins >> np.uint64(63)) == 1)
    is_del = is_indel & ~is_ins
    # substitution: shift by 1..3 so the new base always differs
    shift = (1 + (u_sub % np.uint64(3))).astype(np.uint8)
    body = np.where(is_sub, (src + shift) & 3, src).astype(np.uint8)
    # two slots per ancestral position: [inserted base, own base]
    slots = np.stack([u_base, body], axis=2).reshape(m, 2 * Lp)
    keep = np.stack([is_ins, ~is_del], axis=2).reshape(m, 2 * Lp)
    mut_len = keep.sum(axis=1)
    width = int(max(int(mut_len.max()), int(np.max(target_len))))
    out = random_codes(st, (m, width))             # tail filler where the copy is short
    pos = np.cumsum(keep, axis=1) - 1
    rows = np.broadcast_to(np.arange(m)[:, None], keep.shape)
    out[rows[keep], pos[keep]] = slots[keep]
    return [out[i, :int(target_len[i])].copy() for i in range(m)]


def _codes_to_readset(codes: list[np.ndarray]) -> ReadSet:
    lens = np.array([len(c) for c in codes], dtype=np.uint64)
    offs = np.zeros(len(codes) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    seq = ALPHABET[np.concatenate(codes)] if codes else np.zeros(0, np.uint8)
    return ReadSet(seq=np.ascontiguousarray(seq, dtype=np.uint8), offsets=offs)


def reads_from_ancestors(st: Stream, ancestors: np.ndarray, n: int, len_lo: int, len_hi: int,
                         p_sub: float, p_indel: float, chunk: int = 8192, return_parents: bool = False):
    """n reads, each a mutated copy of a uniformly chosen ancestor, lengths U[len_lo, len_hi].
    With return_parents, also the ancestor index of every read (a species label)."""
    parent_of = st.integers(0, len(ancestors) - 1, (n,))
    target = st.integers(len_lo, len_hi, (n,))
    codes: list[np.ndarray] = []
    for c0 in range(0, n, chunk):
        sub = Stream(int(st.key), 1000 + c0 // chunk)
        codes += mutate(sub, ancestors, parent_of[c0:c0 + chunk], target[c0:c0 + chunk],
                        p_sub, p_indel)
    rs = _codes_to_readset(codes)
    return (rs, parent_of.astype(np.int32)) if return_parents else rs


def ancestor_tree(st: Stream, length: int, branching=(4, 5, 10), div_lo=0.02, div_hi=0.08,
                  sub_frac=0.8) -> np.ndarray:
    """Leaves of a random tree: a uniform root, each level mutated with divergence U[lo,hi]."""
    level = random_codes(st, (1, length))
    for b in branching:
        P = level.shape[0]
        parent_of = np.repeat(np.arange(P), b)
        delta = div_lo + st.uniform((P * b,)) * (div_hi - div_lo)
        kids = mutate(st, level, parent_of, np.full(P * b, length), delta * sub_frac,
                      delta * (1.0 - sub_frac))
        level = np.stack(kids)
    return level


# --------------------------------------------------------------------------------------
# The five workloads.  Seeds: workload k uses 1000 + k.
# --------------------------------------------------------------------------------------

def workload_plain_small(seed: int = 1001) -> ReadSet:
    """150 reads, lengths U[280,320]; 10 uniform ancestors of length 300; 3 % sub, 1 % indel."""
    st = Stream(seed, 0)
    anc = random_codes(st, (10, 300))
    return reads_from_ancestors(Stream(seed, 1), anc, 150, 280, 320, 0.03, 0.01)


def workload_plain_10k(seed: int = 1002, n: int = 10_000) -> ReadSet:
    """10^4 reads, lengths U[250,450]; 50 ancestors (length 450); 5 % sub, 1.5 % indel."""
    st = Stream(seed, 0)
    anc = random_codes(st, (50, 450))
    return reads_from_ancestors(Stream(seed, 1), anc, n, 250, 450, 0.05, 0.015)


def paper_scale_ancestors(seed: int = 1003) -> np.ndarray:
    """200 ancestors (length 450) from a 4 x 5 x 10 tree, 2-8 % divergence per level."""
    return ancestor_tree(Stream(seed, 0), 450)


def workload_paper_scale(seed: int = 1003, n: int = 100_000, len_lo: int = 250,
                         len_hi: int = 450) -> ReadSet:
    """10^5 reads, lengths U[250,450], from the 200 tree ancestors; 5 % sub, 1.5 % indel."""
    anc = paper_scale_ancestors(seed)
    return reads_from_ancestors(Stream(seed, 1), anc, n, len_lo, len_hi, 0.05, 0.015)


def workload_batched(seed: int = 1004, n_samples: int = 64, n_lo: int = 500,
                     n_hi: int = 20_000) -> list[ReadSet]:
    """64 samples: read counts log-U[500,20000], lengths U[150,500], 5-100 ancestors each."""
    st = Stream(seed, 0)
    counts = st.log_uniform_int(n_lo, n_hi, (n_samples,))
    n_anc = st.integers(5, 100, (n_samples,))
    out = []
    for s in range(n_samples):
        ss = Stream(seed, 100 + s)
        anc = random_codes(ss, (int(n_anc[s]), 500))
        out.append(reads_from_ancestors(Stream(seed, 10_000 + s), anc, int(counts[s]), 150, 500,
                                        0.05, 0.015))
    return out


@dataclasses.dataclass
class QueryRequest:
    arrival_s: float
    reads: ReadSet


def workload_served_queries(n_requests: int, rate_per_s: float, seed: int = 1005,
                            ref_seed: int = 1003, nq_hi: int = 4096) -> list[QueryRequest]:
    """Query batches of log-U[1,4096] reads (lengths U[250,450]) with Poisson arrivals.

    Ancestors: the 200 paper-scale tree ancestors plus 20 novel uniform ones (10 %).
    """
    st = Stream(seed, 0)
    anc = np.concatenate([paper_scale_ancestors(ref_seed), random_codes(st, (20, 450))])
    sizes = st.log_uniform_int(1, nq_hi, (n_requests,))
    gaps = -np.log1p(-st.uniform((n_requests,))) / rate_per_s
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for r in range(n_requests):
        rs = reads_from_ancestors(Stream(seed, 1000 + r), anc, int(sizes[r]), 250, 450,
                                  0.05, 0.015)
        reqs.append(QueryRequest(arrival_s=float(t[r]), reads=rs))
    return reqs
