"""Independent simplex quadrature for the oracle pins (collapsed Gauss-Legendre products).

The map from the unit cube to the reference simplex (Duffy / Stroud conical product) turns a
polynomial of degree q into one of degree <= q + d - 1 per coordinate, so g Gauss points per
axis integrate degree q exactly when 2g - 1 >= q + d - 1.  Nothing here uses barycentric
monomial formulas, so it checks the oracle's exact integration from the outside."""
import numpy as np


def reference_rule(d: int, g: int = 6):
    x, w = np.polynomial.legendre.leggauss(g)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    if d == 2:
        a, b = np.meshgrid(x, x, indexing="ij")
        wa, wb = np.meshgrid(w, w, indexing="ij")
        s = a * (1 - b)
        t = b
        jac = 1 - b
        pts = np.stack([s.ravel(), t.ravel()], 1)
        wts = (wa * wb * jac).ravel()
    else:
        a, b, c = np.meshgrid(x, x, x, indexing="ij")
        wa, wb, wc = np.meshgrid(w, w, w, indexing="ij")
        s = a * (1 - b) * (1 - c)
        t = b * (1 - c)
        r = c
        jac = (1 - b) * (1 - c) ** 2
        pts = np.stack([s.ravel(), t.ravel(), r.ravel()], 1)
        wts = (wa * wb * wc * jac).ravel()
    return pts, wts


def simplex_points(verts: np.ndarray, d: int, g: int = 6):
    """Quadrature points (Q, d) and weights (Q,) on the simplex with vertices verts (d+1, d)."""
    pts, wts = reference_rule(d, g)
    b = verts[1:] - verts[0]
    x = verts[0] + pts @ b
    return x, wts * abs(np.linalg.det(b))


def p1_eval(verts: np.ndarray, vals: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Value at points x of the affine function taking vals at verts (solve for its coefficients)."""
    d = verts.shape[1]
    a = np.concatenate([np.ones((d + 1, 1)), verts], 1)
    coef = np.linalg.solve(a, vals)
    return coef[0] + x @ coef[1:]
