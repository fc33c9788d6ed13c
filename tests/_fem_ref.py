"""Independent numpy evaluation of the finite-element building blocks, used
only to pin the CPU oracle: the bases are built here from numpy's Legendre
polynomial routines and exact polynomial arithmetic, not from the oracle."""
import itertools

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def gauss_legendre01(n):
    z, w = npleg.leggauss(n)
    return 0.5 * (z + 1.0), 0.5 * w


def gauss_lobatto01(n):
    """n Gauss-Lobatto nodes on [0,1]: endpoints plus the roots of P_{n-1}'."""
    m = n - 1
    coef = np.zeros(m + 1)
    coef[m] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(coef)))) if m >= 2 else np.array([])
    z = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (z + 1.0)


def lagrange_polys(nodes):
    """Power-series coefficients of the Lagrange polynomials on the nodes."""
    polys = []
    for a, xa in enumerate(nodes):
        others = [xb for b, xb in enumerate(nodes) if b != a]
        c = nppoly.polyfromroots(others) if others else np.array([1.0])
        c = c / nppoly.polyval(xa, c)
        polys.append(c)
    return polys


def tensor_basis(nodes, pts, d):
    """Values and reference gradients of the tensor Lagrange basis on the nodes
    at the tensor points: val[q, i], grad[q, i, m] (lexicographic, first index
    fastest)."""
    P = lagrange_polys(nodes)
    n = len(nodes)
    B = np.array([[nppoly.polyval(t, p) for p in P] for t in pts])          # [q1, a]
    G = np.array([[nppoly.polyval(t, nppoly.polyder(p)) for p in P] for t in pts])
    nq = len(pts)
    qs = list(itertools.product(range(nq), repeat=d))
    qs = [q[::-1] for q in qs]  # make first index fastest
    qs.sort(key=lambda q: sum(q[c] * nq ** c for c in range(d)))
    ids = list(itertools.product(range(n), repeat=d))
    ids = [i[::-1] for i in ids]
    ids.sort(key=lambda i: sum(i[c] * n ** c for c in range(d)))
    val = np.zeros((len(qs), len(ids)))
    grad = np.zeros((len(qs), len(ids), d))
    for qi, q in enumerate(qs):
        for ii, a in enumerate(ids):
            val[qi, ii] = np.prod([B[q[c], a[c]] for c in range(d)])
            for m in range(d):
                grad[qi, ii, m] = np.prod([G[q[c], a[c]] if c == m else B[q[c], a[c]]
                                           for c in range(d)])
    return val, grad


def tensor_weights(w, d):
    nq = len(w)
    out = np.zeros(nq ** d)
    for q in range(nq ** d):
        out[q] = np.prod([w[(q // nq ** c) % nq] for c in range(d)])
    return out


class CartesianMesh:
    """Connectivity of the Cartesian Q_k mesh with the documented layout."""

    def __init__(self, d, n, k):
        self.d, self.n, self.k = d, list(n), k
        self.nn = [m * k + 1 for m in self.n]
        self.nnodes = int(np.prod(self.nn))
        self.nelem = int(np.prod(self.n))

    def conn(self, el):
        d, k = self.d, self.k
        ei = []
        r = el
        for c in range(d):
            ei.append(r % self.n[c])
            r //= self.n[c]
        out = []
        for i in range((k + 1) ** d):
            a = [(i // (k + 1) ** c) % (k + 1) for c in range(d)]
            I = [ei[c] * k + a[c] for c in range(d)]
            idx = 0
            for c in reversed(range(d)):
                idx = idx * self.nn[c] + I[c]
            out.append(idx)
        return np.array(out)
