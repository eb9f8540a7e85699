"""Geometry checks shared by the oracle and GPU tests (independent of both)."""
import numpy as np


def tri_tri_intersect(P, T1, T2):
    """Independent FP64 test: does any edge of one triangle cross the other."""
    def orient(a, b, c, d):
        return np.einsum("...i,...i->...", np.cross(b - a, c - a), d - a)

    def seg_tri(p, q, a, b, c):
        s1, s2 = orient(a, b, c, p), orient(a, b, c, q)
        o1, o2, o3 = orient(p, q, a, b), orient(p, q, b, c), orient(p, q, c, a)
        cross = (s1 * s2 <= 0)
        same = ((o1 >= 0) & (o2 >= 0) & (o3 >= 0)) | ((o1 <= 0) & (o2 <= 0) & (o3 <= 0))
        return cross & same

    A = P[T1]
    B = P[T2]
    hit = np.zeros(len(T1), dtype=bool)
    for (i, j) in ((0, 1), (1, 2), (2, 0)):
        hit |= seg_tri(A[:, i], A[:, j], B[:, 0], B[:, 1], B[:, 2])
        hit |= seg_tri(B[:, i], B[:, j], A[:, 0], A[:, 1], A[:, 2])
    return hit
