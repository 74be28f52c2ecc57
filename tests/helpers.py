"""Shared test helpers: norms on Gauss-Legendre nodes and exact solutions.

Node positions and weights come from the oracle (tests may use it); the
exact solutions are written from the physics of each PDE, not from the
scheme.
"""
import math

import numpy as np

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl


def weights_nd(N, d):
    _, w = orc.gauss_legendre(N)
    W = w
    for _ in range(d - 1):
        W = np.multiply.outer(w, W).reshape(-1)   # axis 0 fastest
    return W


def l2(P, E):
    """Discrete L2 norm over all cells and components, GL quadrature."""
    W = weights_nd(P.N, P.d)
    vol = float(np.prod(P.dx[: P.d]))
    return math.sqrt(vol * float((np.asarray(E) ** 2 * W[None, None, :]).sum()))


def rel_l2(P, A, B):
    return l2(P, np.asarray(A) - np.asarray(B)) / max(l2(P, B), 1e-300)


def coords(P):
    xi, _ = orc.gauss_legendre(P.N)
    return wl.node_coords(P.grid[: P.d], P.dx[: P.d], xi)


def total(P, Q):
    """Integral of every component over the domain (GL quadrature), [m]."""
    W = weights_nd(P.N, P.d)
    return float(np.prod(P.dx[: P.d])) * (np.asarray(Q) * W[None, None, :]).sum(axis=(0, 2))
