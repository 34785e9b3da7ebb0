"""CPU oracle for the all-pairs read alignment distance -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may
import this package.  The library's compute path never does, and this package
imports nothing from the library.

It wraps two plain C files, compiled with gcc on first use (or by `build()`):
  * sw_oracle.c -- Smith-Waterman local score from the full DP matrix, the distance
    d = max(la, lb) - S (or one of the other score-to-distance readings: min(la, lb) - S,
    the raw score, or the normalised 1 - S/max(la, lb) on a 16-bit scale), and threaded
    all-pairs / pair-list / rectangle drivers (paper section 2.2);
  * brute.c     -- the local score by listing every alignment of every pair of
    substrings, with no DP table, used to pin sw_oracle.c on tiny reads.
Default scores: match +1, mismatch -1, linear gap -1 (the paper states none); an
optional affine mode (gap_open > 0: a run of L gapped bases costs gap_open + L * gap,
Gotoh's recurrence) pinned by its own brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["sw_oracle.c", "brute.c"]
_lock = threading.Lock()
_lib = None

MATCH, MISMATCH, GAP = 1, -1, 1
# score-to-distance rules (the `conversion` argument of sw_oracle.c)
CONV_MAX, CONV_MIN, CONV_SCORE, CONV_NORM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, portable flags)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-o", tmp] + srcs + ["-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u16p = ctypes.POINTER(ctypes.c_uint16)
            i64 = ctypes.c_int64
            ci = ctypes.c_int
            lib.oracle_sw_score.argtypes = [u8p, i64, u8p, i64, ci, ci, ci]
            lib.oracle_sw_score.restype = ci
            lib.oracle_distance.argtypes = [u8p, i64, u8p, i64, ci, ci, ci]
            lib.oracle_distance.restype = ci
            lib.oracle_tri_index.argtypes = [ctypes.c_uint64] * 3
            lib.oracle_tri_index.restype = ctypes.c_uint64
            lib.oracle_sw_score_affine.argtypes = [u8p, i64, u8p, i64, ci, ci, ci, ci]
            lib.oracle_sw_score_affine.restype = ci
            lib.oracle_distance_conv.argtypes = [u8p, i64, u8p, i64, ci, ci, ci, ci, ci]
            lib.oracle_distance_conv.restype = ci
            lib.oracle_all_pairs.argtypes = [u8p, u64p, ctypes.c_uint64, u16p, ci, ci, ci, ci, ci, ci]
            lib.oracle_pairs.argtypes = [u8p, u64p, u8p, u64p, u64p, u64p, ctypes.c_uint64, u16p,
                                         ci, ci, ci, ci, ci, ci]
            lib.oracle_pair_scores.argtypes = [u8p, u64p, u8p, u64p, u64p, u64p, ctypes.c_uint64,
                                               ctypes.POINTER(ctypes.c_int32), ci, ci, ci, ci, ci]
            lib.oracle_rect.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_uint64, u8p, u64p,
                                        ctypes.c_uint64, ctypes.c_uint64, u16p, ctypes.c_uint64,
                                        ci, ci, ci, ci, ci, ci]
            lib.brute_local_score.argtypes = [u8p, ci, u8p, ci, ci, ci, ci]
            lib.brute_local_score.restype = ci
            lib.brute_local_score_affine.argtypes = [u8p, ci, u8p, ci, ci, ci, ci, ci]
            lib.brute_local_score_affine.restype = ci
            lib.brute_count_strings.argtypes = [ci]
            lib.brute_count_strings.restype = ci
            lib.brute_string.argtypes = [ci, ci, u8p, ctypes.POINTER(ci)]
            lib.brute_exhaustive.argtypes = [ci, ci, ci, ci, ci, ctypes.POINTER(ctypes.c_int32)]
            _lib = lib
    return _lib


def _ptr(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def _bytes(x) -> np.ndarray:
    if isinstance(x, str):
        x = x.encode()
    return np.frombuffer(bytes(x), dtype=np.uint8).copy() if len(x) else np.zeros(1, np.uint8)


def _threads(nthreads):
    return nthreads if nthreads else (os.cpu_count() or 1)


def sw_score(a, b, match=MATCH, mismatch=MISMATCH, gap=GAP) -> int:
    """Smith-Waterman local score S of two reads (full DP matrix)."""
    A, B = _bytes(a), _bytes(b)
    return _load().oracle_sw_score(_ptr(A, ctypes.c_uint8), len(a), _ptr(B, ctypes.c_uint8),
                                   len(b), match, mismatch, gap)


def distance(a, b, match=MATCH, mismatch=MISMATCH, gap=GAP) -> int:
    """d = max(la, lb) - S."""
    A, B = _bytes(a), _bytes(b)
    return _load().oracle_distance(_ptr(A, ctypes.c_uint8), len(a), _ptr(B, ctypes.c_uint8),
                                   len(b), match, mismatch, gap)


def distance_conv(a, b, conversion, match=MATCH, mismatch=MISMATCH, gap=GAP, gap_open=0) -> int:
    """Distance of two reads under a conversion rule (CONV_*), linear or affine gaps."""
    A, B = _bytes(a), _bytes(b)
    return _load().oracle_distance_conv(_ptr(A, ctypes.c_uint8), len(a), _ptr(B, ctypes.c_uint8),
                                        len(b), match, mismatch, gap, gap_open, conversion)


def tri_index(i: int, j: int, n: int) -> int:
    return _load().oracle_tri_index(i, j, n)


def _seq_off(rs):
    seq = np.ascontiguousarray(rs.seq, dtype=np.uint8)
    if seq.size == 0:
        seq = np.zeros(1, np.uint8)
    return seq, np.ascontiguousarray(rs.offsets, dtype=np.uint64)


def all_pairs(rs, match=MATCH, mismatch=MISMATCH, gap=GAP, nthreads=None, gap_open=0,
              conversion=CONV_MAX) -> np.ndarray:
    """Strict upper triangle (row-major, uint16) of all pairwise distances of a ReadSet."""
    n = rs.n
    out = np.zeros(max(n * (n - 1) // 2, 1), dtype=np.uint16)
    seq, off = _seq_off(rs)
    _load().oracle_all_pairs(_ptr(seq, ctypes.c_uint8), _ptr(off, ctypes.c_uint64), n,
                             _ptr(out, ctypes.c_uint16), match, mismatch, gap, gap_open,
                             conversion, _threads(nthreads))
    return out[: n * (n - 1) // 2]


def pairs(rsA, pi, pj, rsB=None, match=MATCH, mismatch=MISMATCH, gap=GAP,
          nthreads=None, gap_open=0, conversion=CONV_MAX) -> np.ndarray:
    """out[p] = d(A[pi[p]], B[pj[p]]) (B defaults to A)."""
    rsB = rsA if rsB is None else rsB
    pi = np.ascontiguousarray(pi, dtype=np.uint64)
    pj = np.ascontiguousarray(pj, dtype=np.uint64)
    out = np.zeros(max(len(pi), 1), dtype=np.uint16)
    sa, oa = _seq_off(rsA)
    sb, ob = _seq_off(rsB)
    _load().oracle_pairs(_ptr(sa, ctypes.c_uint8), _ptr(oa, ctypes.c_uint64),
                         _ptr(sb, ctypes.c_uint8), _ptr(ob, ctypes.c_uint64),
                         _ptr(pi, ctypes.c_uint64), _ptr(pj, ctypes.c_uint64), len(pi),
                         _ptr(out, ctypes.c_uint16), match, mismatch, gap, gap_open,
                         conversion, _threads(nthreads))
    return out[: len(pi)]


def pair_scores(rsA, pi, pj, rsB=None, match=MATCH, mismatch=MISMATCH, gap=GAP,
                nthreads=None, gap_open=0) -> np.ndarray:
    """out[p] = S(A[pi[p]], B[pj[p]]), the raw local alignment score (int32)."""
    rsB = rsA if rsB is None else rsB
    pi = np.ascontiguousarray(pi, dtype=np.uint64)
    pj = np.ascontiguousarray(pj, dtype=np.uint64)
    out = np.zeros(max(len(pi), 1), dtype=np.int32)
    sa, oa = _seq_off(rsA)
    sb, ob = _seq_off(rsB)
    _load().oracle_pair_scores(_ptr(sa, ctypes.c_uint8), _ptr(oa, ctypes.c_uint64),
                               _ptr(sb, ctypes.c_uint8), _ptr(ob, ctypes.c_uint64),
                               _ptr(pi, ctypes.c_uint64), _ptr(pj, ctypes.c_uint64), len(pi),
                               _ptr(out, ctypes.c_int32), match, mismatch, gap, gap_open,
                               _threads(nthreads))
    return out[: len(pi)]


def rect(rsA, a0, a1, rsB, b0, b1, match=MATCH, mismatch=MISMATCH, gap=GAP,
         nthreads=None, gap_open=0, conversion=CONV_MAX) -> np.ndarray:
    """Row-major (a1-a0) x (b1-b0) block of distances d(A[r], B[c])."""
    ld = b1 - b0
    out = np.zeros(max((a1 - a0) * ld, 1), dtype=np.uint16)
    sa, oa = _seq_off(rsA)
    sb, ob = _seq_off(rsB)
    _load().oracle_rect(_ptr(sa, ctypes.c_uint8), _ptr(oa, ctypes.c_uint64), a0, a1,
                        _ptr(sb, ctypes.c_uint8), _ptr(ob, ctypes.c_uint64), b0, b1,
                        _ptr(out, ctypes.c_uint16), ld, match, mismatch, gap, gap_open,
                        conversion, _threads(nthreads))
    return out[: (a1 - a0) * ld].reshape(a1 - a0, ld)


# ------------------------------------------------------------------ brute force (pins)

def brute_score(a, b, match=MATCH, mismatch=MISMATCH, gap=GAP) -> int:
    """Best score over every alignment of every pair of substrings (no DP table)."""
    A, B = _bytes(a), _bytes(b)
    return _load().brute_local_score(_ptr(A, ctypes.c_uint8), len(a), _ptr(B, ctypes.c_uint8),
                                     len(b), match, mismatch, gap)


def sw_score_affine(a, b, gap_open, gap=GAP, match=MATCH, mismatch=MISMATCH) -> int:
    """Local score with affine gaps (Gotoh): a run of L gapped bases costs gap_open + L*gap."""
    A, B = _bytes(a), _bytes(b)
    return _load().oracle_sw_score_affine(_ptr(A, ctypes.c_uint8), len(a), _ptr(B, ctypes.c_uint8),
                                          len(b), match, mismatch, gap_open, gap)


def brute_score_affine(a, b, gap_open, gap=GAP, match=MATCH, mismatch=MISMATCH) -> int:
    """Brute force with affine gap runs (no DP table)."""
    A, B = _bytes(a), _bytes(b)
    return _load().brute_local_score_affine(_ptr(A, ctypes.c_uint8), len(a), _ptr(B, ctypes.c_uint8),
                                            len(b), match, mismatch, gap_open, gap)


def brute_strings(maxlen: int) -> list[bytes]:
    """All strings over ACGT of length <= maxlen, in the order brute_exhaustive uses."""
    lib = _load()
    ns = lib.brute_count_strings(maxlen)
    buf = np.zeros(16, np.uint8)
    L = ctypes.c_int()
    out = []
    for x in range(ns):
        lib.brute_string(x, maxlen, _ptr(buf, ctypes.c_uint8), ctypes.byref(L))
        out.append(bytes(buf[: L.value]))
    return out


def brute_exhaustive(maxlen: int, match=MATCH, mismatch=MISMATCH, gap=GAP, gap_open=0) -> np.ndarray:
    """Matrix of brute-force scores over all string pairs of length <= maxlen."""
    lib = _load()
    ns = lib.brute_count_strings(maxlen)
    out = np.zeros(ns * ns, dtype=np.int32)
    lib.brute_exhaustive(maxlen, match, mismatch, gap, gap_open, _ptr(out, ctypes.c_int32))
    return out.reshape(ns, ns)


def brute_score_py(a: str, b: str, match=MATCH, mismatch=MISMATCH, gap=GAP) -> int:
    """Pure-Python brute force for very small cases: every substring pair, every global
    alignment of it listed explicitly as a column sequence, scored column by column."""
    def alignments(x, y):
        if not x and not y:
            yield []
            return
        if x and y:
            for rest in alignments(x[1:], y[1:]):
                yield [(x[0], y[0])] + rest
        if x:
            for rest in alignments(x[1:], y):
                yield [(x[0], None)] + rest
        if y:
            for rest in alignments(x, y[1:]):
                yield [(None, y[0])] + rest

    best = 0
    subs_a = {a[i:j] for i in range(len(a) + 1) for j in range(i, len(a) + 1)}
    subs_b = {b[i:j] for i in range(len(b) + 1) for j in range(i, len(b) + 1)}
    for x in subs_a:
        for y in subs_b:
            for aln in alignments(x, y):
                sc = 0
                for p, q in aln:
                    if p is None or q is None:
                        sc -= gap
                    elif p.upper() == q.upper():
                        sc += match
                    else:
                        sc += mismatch
                best = max(best, sc)
    return best
