"""CPU oracle for the distance-threshold steps -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may import
this module; the library never does, and this module imports nothing from the library.

What it follows (arxiv 1803.02272):
  * section 4.3 (supervised annotation, the `diagno-syst` step): a sample read is
    compared with every annotated reference read; the references closer than the
    homology gap (classically 97 %) are selected; if they all carry one species the read
    gets that species, if they disagree it is ambiguous (and with no reference in range
    it stays unassigned);
  * section 5 (threshold graph): vertices are the reads, an edge joins i and j when
    d(i, j) <= theta, and the connected components of that graph are the clusters.

Readings where the paper is silent (both are parameters here):
  * "closer than the homology gap": a pair is a hit when d * den <= num * max(la, lb)
    (97 % homology -> num/den = 3/100, the distance as a fraction of the longer read)
    and d <= abs_max; integer arithmetic, so the decision is exact;
  * annotation codes: species ids are integers >= 0; -1 = no hit, -2 = ambiguous;
    references with a negative label do not vote;
  * component labels: each read gets the smallest read index of its component.
Distances come from the distance oracle (oracle.pairs / all_pairs / rect).
"""
from __future__ import annotations

import collections

import numpy as np

NONE, AMBIGUOUS = -1, -2


def is_hit(d, la, lb, num: int, den: int, abs_max: int = 65535):
    """Elementwise hit test: d <= abs_max and d * den <= num * max(la, lb)."""
    d = np.asarray(d, dtype=np.int64)
    L = np.maximum(np.asarray(la, dtype=np.int64), np.asarray(lb, dtype=np.int64))
    return (d <= abs_max) & (d * den <= num * L)


def hits_rect(D, lens_a, lens_b, num: int, den: int, abs_max: int = 65535):
    """Set of (row, col, d) of a distance rectangle D[row][col] that pass the test."""
    D = np.asarray(D)
    la = np.asarray(lens_a)[:, None]
    lb = np.asarray(lens_b)[None, :]
    r, c = np.nonzero(is_hit(D, la, lb, num, den, abs_max))
    return {(int(i), int(j), int(D[i, j])) for i, j in zip(r, c)}


def annotate(D, lens_q, lens_ref, ref_labels, num: int, den: int, abs_max: int = 65535):
    """Section 4.3: per query row, the one species of all its hits, NONE or AMBIGUOUS."""
    D = np.asarray(D)
    out = []
    for i in range(D.shape[0]):
        species = set()
        for j in range(D.shape[1]):
            if ref_labels[j] < 0:
                continue
            if is_hit(D[i, j], lens_q[i], lens_ref[j], num, den, abs_max):
                species.add(int(ref_labels[j]))
        out.append(NONE if not species else (species.pop() if len(species) == 1 else AMBIGUOUS))
    return np.array(out, dtype=np.int32)


def components(n: int, edges):
    """Section 5: connected components of the graph with the given undirected edges, by
    breadth-first search; label = smallest vertex of the component."""
    adj = collections.defaultdict(list)
    for i, j in edges:
        adj[i].append(j)
        adj[j].append(i)
    label = np.full(n, -1, dtype=np.int64)
    for s in range(n):                   # increasing order: s is its component's minimum
        if label[s] >= 0:
            continue
        label[s] = s
        queue = collections.deque([s])
        while queue:
            v = queue.popleft()
            for w in adj[v]:
                if label[w] < 0:
                    label[w] = s
                    queue.append(w)
    return label


def threshold_edges(tri, lens, num: int, den: int, abs_max: int = 65535):
    """Edges (i, j), i < j, of the threshold graph of a strict upper triangle (row-major,
    index k(i, j) = i*n - i*(i+1)/2 + (j-i-1))."""
    lens = np.asarray(lens)
    n = len(lens)
    iu, ju = np.triu_indices(n, 1)
    tri = np.asarray(tri)
    keep = is_hit(tri, lens[iu], lens[ju], num, den, abs_max)
    return list(zip(iu[keep].tolist(), ju[keep].tolist()))
