"""Velocity sets, weights and moment matrices (paper Appendix A).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The lattice speed is c = dx/dt = 1 (lattice units, Table "Units"), so the
diagonal matrix C_d of powers of c is the identity and the natural transform
is M = M0.  The sound speed is c_s^2 = d0 c^2 with the adjustable scale factor
d0 (Sec. 3, below Eq. of f_i^eq).

* D2Q9: weights w0 = (1-d0)^2, w1-4 = (d0-d0^2)/2, w5-8 = d0^2/4 (Appendix A).
  M0 rows are the natural monomials 1, cx, cy, cx^2, cy^2, cx cy, cx cy^2,
  cx^2 cy, cx^2 cy^2, in the order printed; N maps them to the Hermite
  polynomials 1, c, c_a^2 - cs2, cx cy, cx cy^2 - cs2 cx, cx^2 cy - cs2 cy,
  (cx^2 - cs2)(cy^2 - cs2).  The tests compare both with the printed matrices.
* D3Q15: the printed M0 and N_H (Appendix A), kept as printed.
* D3Q19: not in the paper.  Weights are fixed by the same moment conditions the
  D2Q9 / D3Q15 weights satisfy (sum w = 1, sum w c_a^2 = d0, sum w cx^2 cy^2 =
  d0^2): w0 = 1 - 3 d0 + 3 d0^2, w_axis = (d0 - 2 d0^2)/2, w_edge = d0^2/4,
  valid for 0 < d0 < 1/2.  Because the plain Hermite polynomials are not
  w-orthogonal on D3Q19, N is built by w-weighted Gram-Schmidt of the monomial
  rows in the order listed, which is the "row transformation" the paper asks
  for on D3Q15 (end of Appendix A).  Pinned by those moment conditions,
  orthogonality, and the 3D shear-wave decay at nu k^2 along an axis and a
  face diagonal (its second-order rows and their rate groups).  Parity
  unpinned: the third- and fourth-order rows, whose rates are free (1 by
  default) and enter no law the paper states.

The relaxation-rate group of every moment row is returned as ``groups``
(labels "s0", "s1", "s2a", "s2b", "s3", "s4"), matching the printed K.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Lattice:
    name: str
    d: int
    c: np.ndarray          # (Q, d) integer velocities
    w: np.ndarray          # (Q,) weights
    cs2: float             # d0 (c = 1)
    M0: np.ndarray         # (Q, Q) natural moments
    N: np.ndarray          # (Q, Q) unit lower triangular, H = N M0
    groups: list           # rate label of each moment row
    opp: np.ndarray        # index of -c_i

    @property
    def Q(self):
        return len(self.w)

    @property
    def T(self):
        """Hermite transform H = N M (C_d = I)."""
        return self.N @ self.M0


def _opposites(c):
    opp = np.empty(len(c), dtype=int)
    for i, ci in enumerate(c):
        opp[i] = [j for j, cj in enumerate(c) if np.all(cj == -ci)][0]
    return opp


def _monomial_rows(c, exps):
    """Rows of monomials prod_a c_a^e_a evaluated on every velocity."""
    return np.array([[np.prod([float(ci[a]) ** e[a] for a in range(len(e))]) for ci in c] for e in exps])


def w_inner(w, p, q):
    """w-weighted inner product sum_i w_i p_i q_i."""
    return float(np.sum(w * p * q))


def gram_schmidt_N(M0, w):
    """Unit lower-triangular N with rows of N M0 mutually w-orthogonal.

    Row k of H is the monomial row k minus its w-projections on the already
    orthogonalised rows 0..k-1 (classical Gram-Schmidt in the row order).
    """
    Q = M0.shape[0]
    H = np.zeros_like(M0)
    for k in range(Q):
        h = M0[k].copy()
        for j in range(k):
            h -= w_inner(w, M0[k], H[j]) / w_inner(w, H[j], H[j]) * H[j]
        H[k] = h
    return H @ np.linalg.inv(M0)


def d2q9(d0: float) -> Lattice:
    # velocity ordering read off rows 2 and 3 of the printed M0
    c = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
    w = np.array([(1 - d0) ** 2] + [(d0 - d0 ** 2) / 2] * 4 + [d0 ** 2 / 4] * 4)
    exps = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (1, 2), (2, 1), (2, 2)]
    M0 = _monomial_rows(c, exps)
    cs2 = d0
    N = np.eye(9)
    N[3, 0] = -cs2              # cx^2 - cs2
    N[4, 0] = -cs2              # cy^2 - cs2
    N[6, 1] = -cs2              # cx cy^2 - cs2 cx
    N[7, 2] = -cs2              # cx^2 cy - cs2 cy
    N[8, 0] = cs2 * cs2         # (cx^2 - cs2)(cy^2 - cs2)
    N[8, 3] = -cs2
    N[8, 4] = -cs2
    groups = ["s0", "s1", "s1", "s2a", "s2a", "s2b", "s3", "s3", "s4"]
    return Lattice("D2Q9", 2, c, w, cs2, M0, N, groups, _opposites(c))


def d3q19(d0: float) -> Lattice:
    c = [[0, 0, 0],
         [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
         [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
         [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
         [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]]
    c = np.array(c)
    w0 = 1 - 3 * d0 + 3 * d0 ** 2
    wa = (d0 - 2 * d0 ** 2) / 2
    we = d0 ** 2 / 4
    w = np.array([w0] + [wa] * 6 + [we] * 12)
    exps = [(0, 0, 0),
            (1, 0, 0), (0, 1, 0), (0, 0, 1),
            (2, 0, 0), (0, 2, 0), (0, 0, 2),
            (1, 1, 0), (1, 0, 1), (0, 1, 1),
            (2, 1, 0), (2, 0, 1), (1, 2, 0), (0, 2, 1), (1, 0, 2), (0, 1, 2),
            (2, 2, 0), (2, 0, 2), (0, 2, 2)]
    M0 = _monomial_rows(c, exps)
    N = gram_schmidt_N(M0, w)
    groups = ["s0"] + ["s1"] * 3 + ["s2a"] * 3 + ["s2b"] * 3 + ["s3"] * 6 + ["s4"] * 3
    return Lattice("D3Q19", 3, c, w, d0, M0, N, groups, _opposites(c))


def d3q15(d0: float) -> Lattice:
    """D3Q15 with the printed M0 and N_H (Appendix A)."""
    cx = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1]
    cy = [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1]
    cz = [0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1]
    c = np.array([cx, cy, cz]).T
    w = np.array([1 - 3 * d0 + 2 * d0 ** 2] + [(d0 - d0 ** 2) / 2] * 6 + [d0 ** 2 / 8] * 8)
    corner = np.zeros(15)
    corner[7:] = 1.0
    M0 = np.array([
        np.ones(15), c[:, 0], c[:, 1], c[:, 2],
        c[:, 0] ** 2, c[:, 1] ** 2, c[:, 2] ** 2,
        c[:, 0] * c[:, 1], c[:, 1] * c[:, 2], c[:, 0] * c[:, 2],
        corner * c[:, 0], corner * c[:, 1], corner * c[:, 2],
        c[:, 0] * c[:, 1] * c[:, 2], corner,
    ]).astype(float)
    cs2 = d0
    N = np.eye(15)
    for r in (4, 5, 6):
        N[r, 0] = -cs2
    N[10, 1] = -cs2
    N[11, 2] = -cs2
    N[12, 3] = -cs2
    N[14, 0] = 2 * cs2 * cs2
    N[14, 4] = N[14, 5] = N[14, 6] = -cs2
    groups = ["s0"] + ["s1"] * 3 + ["s2a"] * 3 + ["s2b"] * 3 + ["s3"] * 4 + ["s4"]
    return Lattice("D3Q15", 3, c, w, d0, M0, N, groups, _opposites(c))


def make(name: str, d0: float) -> Lattice:
    return {"D2Q9": d2q9, "D3Q19": d3q19, "D3Q15": d3q15}[name](d0)


_ISO_CACHE = {}


def isotropic_stencil(d: int):
    """Velocities and weights of the isotropic central difference stencil.

    The paper computes gradients and Laplacians with second-order isotropic
    central schemes (end of Sec. 3) without printing them.  Reading: the
    standard lattice-weighted forms on D2Q9 (2D) / D3Q19 (3D) with the d0 = 1/3
    weights, for which the fourth-order weight tensor is isotropic:
        grad phi(x)  = sum_i w_i c_i phi(x + c_i) / cs2
        lap  phi(x)  = sum_i 2 w_i (phi(x + c_i) - phi(x)) / cs2,   cs2 = 1/3.
    """
    if d not in _ISO_CACHE:
        lat = d2q9(1.0 / 3.0) if d == 2 else d3q19(1.0 / 3.0)
        _ISO_CACHE[d] = (lat.c, lat.w, 1.0 / 3.0)
    return _ISO_CACHE[d]
