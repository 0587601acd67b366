"""Exact brute-force tree growth in pure Python, for tiny inputs only.

An independent restatement of greedy CART regression growth (the recursive partitioning of the
random forest the paper fits, Sec. III-B) used to pin the C oracle: every (feature, threshold)
candidate is enumerated by building the left and right row sets explicitly, and the criterion is
evaluated with ``fractions.Fraction``. Random draws (bootstrap multiplicities, tried features) are
inputs, so this file holds no generator.
"""
from __future__ import annotations

from fractions import Fraction


def grow(X, y, w, feats_of, min_node: int, max_depth: int):
    """X: list of F columns (python floats), y: python ints, w: multiplicities.

    feats_of(d, i) -> iterable of features tried at node i of depth d.
    Returns BFS node list of dicts: feature (-1 leaf), thr, left, value, n, S."""
    rows0 = [r for r in range(len(y)) if w[r] > 0]
    nodes = [dict(rows=rows0, depth=0)]
    begin, end = 0, 1
    d = 0
    while begin < end:
        for idx in range(begin, end):
            i = idx - begin
            nd = nodes[idx]
            rows = nd["rows"]
            n = sum(w[r] for r in rows)
            S = sum(w[r] * y[r] for r in rows)
            nd["n"], nd["S"] = n, S
            best = None
            if n > min_node and not (max_depth > 0 and d == max_depth):
                for f in sorted(feats_of(d, i)):
                    values = sorted({X[f][r] for r in rows})
                    for v in values[:-1]:
                        L = [r for r in rows if X[f][r] <= v]
                        R = [r for r in rows if not X[f][r] <= v]
                        nL = sum(w[r] for r in L)
                        nR = sum(w[r] for r in R)
                        SL = sum(w[r] * y[r] for r in L)
                        SR = sum(w[r] * y[r] for r in R)
                        G = Fraction(SL * SL, nL) + Fraction(SR * SR, nR)
                        if best is None or G > best[0]:
                            best = (G, f, v, L, R)
            if best is not None and best[0] > Fraction(S * S, n):
                G, f, v, L, R = best
                nd["feature"], nd["thr"] = f, v + 0.0
                nd["left"] = len(nodes)
                nodes.append(dict(rows=L, depth=d + 1))
                nodes.append(dict(rows=R, depth=d + 1))
                nd["value"] = 0
            else:
                nd["feature"], nd["thr"], nd["left"] = -1, 0.0, -1
                nd["value"] = (2 * S + n) // (2 * n)          # round half up
        begin, end = end, len(nodes)
        d += 1
    return nodes


def leaf_of(nodes, x):
    j = 0
    while nodes[j]["feature"] >= 0:
        j = nodes[j]["left"] + (0 if x[nodes[j]["feature"]] <= nodes[j]["thr"] else 1)
    return j
