"""Pure-Python brute force for tiny systems (test helper, independent of the oracle).

Used to pin the oracle's neighbour sets on N <= 64: plain Python floats and
math.sqrt, one pair at a time, no numpy and no shared code with ``oracle/``.
The neighbour set follows Sec. 3.2 / Sec. 3.3 (vi) of Nitadori & Aarseth 2012:
j != i is a neighbour of i when min(|R|, |R + dtr V|) < h_i (the velocity term
only when a regular step is given).
"""
import math


def neighbour_sets(x, v, act, h, dtr=None):
    """Return, per active particle, the ascending list of its neighbours."""
    out = []
    n = len(x)
    for a, i in enumerate(act):
        i = int(i)
        lst = []
        for j in range(n):
            if j == i:
                continue
            R = [float(x[j][k]) - float(x[i][k]) for k in range(3)]
            V = [float(v[j][k]) - float(v[i][k]) for k in range(3)]
            r = math.sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2])
            if dtr is not None:
                d = float(dtr[a])
                P = [R[k] + d * V[k] for k in range(3)]
                r = min(r, math.sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]))
            if r < float(h[a]):
                lst.append(j)
        out.append(lst)
    return out
