"""Helpers shared by the GPU tests (no method arithmetic)."""
import numpy as np

TWO32 = 2 ** 32


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def to_dev(torch, *arrays):
    out = []
    for a in arrays:
        out.append(None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda())
    return out


def canon_tris(tri, off):
    """Canonical set of torus triangles: rotate each (p, a, b) so that the
    smallest caller index comes first, offsets re-expressed relative to it."""
    out = set()
    for (p, a, b), (ax, ay, bx, by) in zip(np.asarray(tri).tolist(), np.asarray(off).tolist()):
        v = [(p, 0, 0), (a, ax, ay), (b, bx, by)]
        k = min(range(3), key=lambda i: v[i][0])
        v = v[k:] + v[:k]
        (q0, x0, y0), (q1, x1, y1), (q2, x2, y2) = v
        out.add((q0, q1, x1 - x0, y1 - y0, q2, x2 - x0, y2 - y0))
    return out
