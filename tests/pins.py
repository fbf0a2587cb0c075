"""Independent pins for the oracle: brute force, closed forms, combinatorial counts.

Nothing here shares code with oracle/ or with the CUDA library.  Each routine
computes the match set or its size from the problem definition (paper Section
2.1) by a different route than the oracle's depth-first search.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np

BIG = np.iinfo(np.int64).max


def edge_order(t):
    """Edge ids: rank by (t, input index)."""
    return sorted(range(len(t)), key=lambda i: (int(t[i]), i))


def brute_force(src, dst, t, edges, delta, gaps=None, elabel=None, nlabel=None,
                edge_labels=None, node_labels=None, anti=None):
    """Every k-subset of edges in id order, tested against conditions 1-6 of the definition
    (6: for each anti-edge (x, y, i, d), no edge other than e_i from phi(x) to phi(y) with
    time in [t(e_i), t(e_i) + d]).

    Returns the sorted list of matches (tuples of edge ids) -- exhaustive, so
    only for tiny graphs (C(m, k) subsets).
    """
    k = len(edges)
    order = edge_order(t)
    S = [int(src[i]) for i in order]
    D = [int(dst[i]) for i in order]
    T = [int(t[i]) for i in order]
    EL = None if edge_labels is None else [int(edge_labels[i]) for i in order]
    gaps = [BIG] * (k - 1) if gaps is None else [BIG if g is None else int(g) for g in gaps]
    out = []
    m = len(order)
    for combo in itertools.combinations(range(m), k):
        ts = [T[e] for e in combo]
        if any(ts[i] >= ts[i + 1] for i in range(k - 1)):
            continue                                     # strictly increasing in time
        if ts[-1] - ts[0] > delta:
            continue                                     # span <= delta
        if any(ts[i + 1] - ts[i] > gaps[i] for i in range(k - 1)):
            continue                                     # per-gap bound
        phi = {}
        ok = True
        for i, e in enumerate(combo):
            x, y = edges[i]
            for mn, gn in ((x, S[e]), (y, D[e])):
                if phi.setdefault(mn, gn) != gn:
                    ok = False
        if not ok or len(set(phi.values())) != len(phi):
            continue                                     # a consistent, injective phi
        if elabel is not None and any(elabel[i] >= 0 and (EL is None or EL[e] != elabel[i])
                                      for i, e in enumerate(combo)):
            continue
        if nlabel is not None and any(nlabel[mn] >= 0 and (node_labels is None or node_labels[gn] != nlabel[mn])
                                      for mn, gn in phi.items()):
            continue
        if anti and any(any(e2 != combo[ai] and S[e2] == phi[ax] and D[e2] == phi[ay]
                            and T[combo[ai]] <= T[e2] <= T[combo[ai]] + ad for e2 in range(m))
                        for ax, ay, ai, ad in anti):
            continue
        out.append(combo)
    return out


# ------------------------------------------------------- two-edge closed forms

def _pairs_in_window(a, b, lim):
    """#{(i, j): a_i < b_j <= a_i + lim} for sorted int64 arrays a, b."""
    if len(a) == 0 or len(b) == 0:
        return 0
    a = np.asarray(a, np.int64); b = np.asarray(b, np.int64)
    hi = np.where(a > BIG - lim, BIG, a + lim)
    return int((np.searchsorted(b, hi, side="right") - np.searchsorted(b, a, side="right")).sum())


def _lists(src, dst, t):
    """Time lists per directed pair, per node (out / in), self-loops dropped."""
    pair, out_t, in_t = {}, {}, {}
    for s, d, tt in zip(src.tolist(), dst.tolist(), t.tolist()):
        if s == d:
            continue
        pair.setdefault((s, d), []).append(tt)
        out_t.setdefault(s, []).append(tt)
        in_t.setdefault(d, []).append(tt)
    f = lambda dct: {k: np.sort(np.asarray(v, np.int64)) for k, v in dct.items()}
    return f(pair), f(out_t), f(in_t)


def two_edge_counts(src, dst, t, delta, gap=BIG):
    """Counts of the five 2-edge motifs from per-pair / per-node sorted time lists.

    With L = min(delta, gap), each motif is a count of ordered edge pairs
    (e1, e2) with t1 < t2 <= t1 + L and the right endpoint pattern:
      pingpong  (a,b),(b,a)   pairs of opposite directions on one node pair
      repeat    (a,b),(a,b)   pairs on one directed pair
      path      (a,b),(b,c)   in-edge then out-edge of b, minus c == a (pingpong)
      outstar   (a,b),(a,c)   out-edge pairs of a, minus b == c (repeat)
      instar    (b,a),(c,a)   in-edge pairs of a, minus b == c (repeat)
    """
    L = min(int(delta), int(gap))
    pair, out_t, in_t = _lists(np.asarray(src), np.asarray(dst), np.asarray(t))
    pingpong = sum(_pairs_in_window(v, pair.get((d, s), ()), L) for (s, d), v in pair.items())
    repeat = sum(_pairs_in_window(v, v, L) for v in pair.values())
    through = sum(_pairs_in_window(in_t.get(b, ()), out_t.get(b, ()), L) for b in set(in_t) | set(out_t))
    fan_out = sum(_pairs_in_window(v, v, L) for v in out_t.values())
    fan_in = sum(_pairs_in_window(v, v, L) for v in in_t.values())
    return {"pingpong": pingpong, "repeat": repeat, "path": through - pingpong,
            "outstar": fan_out - repeat, "instar": fan_in - repeat}


TWO_EDGE_MOTIFS = {"pingpong": [(0, 1), (1, 0)], "repeat": [(0, 1), (0, 1)],
                   "path": [(0, 1), (1, 2)], "outstar": [(0, 1), (0, 2)],
                   "instar": [(1, 0), (2, 0)]}


# ---------------------------------------------------- combinatorial families

def pattern_subsequences(seq, pattern):
    """Number of index-increasing subsequences of seq equal to pattern (DP)."""
    dp = [0] * (len(pattern) + 1)
    dp[0] = 1
    for s in seq:
        for j in range(len(pattern) - 1, -1, -1):
            if pattern[j] == s:
                dp[j + 1] += dp[j]
    return dp[-1]


def triangle_train(n):
    """3n edges cycling a->b, b->c, c->a at t = 1..3n (nodes 0, 1, 2)."""
    kinds = [(0, 1), (1, 2), (2, 0)]
    src = np.array([kinds[i % 3][0] for i in range(3 * n)], np.int32)
    dst = np.array([kinds[i % 3][1] for i in range(3 * n)], np.int32)
    t = np.arange(1, 3 * n + 1, dtype=np.int64)
    return src, dst, t


def triangle_train_count(n):
    """Temporal 3-cycles in triangle_train(n) with unbounded delta: any rotation of the
    edge-type pattern (0,1,2) as a subsequence of the type sequence."""
    seq = [i % 3 for i in range(3 * n)]
    return sum(pattern_subsequences(seq, [r % 3, (r + 1) % 3, (r + 2) % 3]) for r in range(3))


def star_burst(d):
    """d out-edges of node 0 to leaves 1..d at times 1..d."""
    return (np.zeros(d, np.int32), np.arange(1, d + 1, dtype=np.int32), np.arange(1, d + 1, dtype=np.int64))


def star_burst_count(d, k):
    """Out-star with k leaves: any k of the d edges, in time order, has k distinct leaves."""
    return comb(d, k)


# ------------------------------------------------------- search-tree work

def _valid_prefix(combo, S, D, T, EL, edges, delta, gaps, elabel, nlabel, node_labels):
    """phi of a prefix (e_0..e_{i-1}) of the motif's edges if it satisfies conditions 1-5
    restricted to those edges, else None."""
    ts = [T[e] for e in combo]
    if any(ts[j] >= ts[j + 1] for j in range(len(ts) - 1)) or ts[-1] - ts[0] > delta:
        return None
    if any(ts[j + 1] - ts[j] > gaps[j] for j in range(len(ts) - 1)):
        return None
    phi = {}
    for j, e in enumerate(combo):
        x, y = edges[j]
        for mn, gn in ((x, S[e]), (y, D[e])):
            if phi.setdefault(mn, gn) != gn:
                return None
    if len(set(phi.values())) != len(phi):
        return None
    if elabel is not None and any(elabel[j] >= 0 and (EL is None or EL[e] != elabel[j]) for j, e in enumerate(combo)):
        return None
    if nlabel is not None and any(nlabel[mn] >= 0 and (node_labels is None or node_labels[gn] != nlabel[mn])
                                  for mn, gn in phi.items()):
        return None
    return phi


def search_work(src, dst, t, edges, delta, gaps=None, elabel=None, nlabel=None, edge_labels=None,
                node_labels=None, roots=None):
    """Work of Algorithm 1's search tree rooted at every edge, from its definition.

    For each level i = 1..k-1: nodes[i] = the i-edge prefixes (e_0..e_{i-1}) that satisfy the
    match conditions restricted to their own edges (each one locates a candidate list for
    motif edge i); entries[i] = the summed number of list entries with time in
    (t(e_{i-1}), min(t(e_0) + delta, t(e_{i-1}) + gap_{i-1})].  The list is out(phi(x_i)) when
    only x_i is bound, in(phi(y_i)) when only y_i is, all edges when neither is, and when both
    are, out(phi(x_i)) if its length is at most that of in(phi(y_i)), else in(phi(y_i)).
    roots = (r0, r1) keeps only the trees whose root edge id lies in [r0, r1).
    Returns (nodes, entries, list_lengths): list_lengths holds the length of every located list
    (a binary search over a list of length L takes between floor(log2 L) and ceil(log2(L+1))
    probes).
    """
    k = len(edges)
    order = edge_order(t)
    S = [int(src[i]) for i in order]
    D = [int(dst[i]) for i in order]
    T = [int(t[i]) for i in order]
    EL = None if edge_labels is None else [int(edge_labels[i]) for i in order]
    gaps = [BIG] * (k - 1) if gaps is None else [BIG if g is None else int(g) for g in gaps]
    m = len(order)
    out_l = {u: [e for e in range(m) if S[e] == u] for u in set(S)}
    in_l = {v: [e for e in range(m) if D[e] == v] for v in set(D)}
    nodes = [0] * 8
    entries = [0] * 8
    lengths = []
    for i in range(1, k):
        for combo in itertools.combinations(range(m), i):
            if roots is not None and not roots[0] <= combo[0] < roots[1]:
                continue
            phi = _valid_prefix(combo, S, D, T, EL, edges[:i], delta, gaps, elabel, nlabel, node_labels)
            if phi is None:
                continue
            nodes[i] += 1
            x, y = edges[i]
            u, v = phi.get(x), phi.get(y)
            if u is not None and v is not None:
                lst = out_l.get(u, []) if len(out_l.get(u, [])) <= len(in_l.get(v, [])) else in_l.get(v, [])
            elif u is not None:
                lst = out_l.get(u, [])
            elif v is not None:
                lst = in_l.get(v, [])
            else:
                lst = list(range(m))
            tprev, t0 = T[combo[-1]], T[combo[0]]
            lim = min(t0 + delta if t0 <= BIG - delta else BIG,
                      tprev + gaps[i - 1] if tprev <= BIG - gaps[i - 1] else BIG)
            entries[i] += sum(1 for e in lst if tprev < T[e] <= lim)
            lengths.append(len(lst))
    return nodes, entries, lengths
