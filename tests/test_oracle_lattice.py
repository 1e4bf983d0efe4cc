"""Pins of the oracle's lattice tables and collision operator (Appendix A)."""
import os

import numpy as np
import pytest

from oracle import lattice as L
from oracle import lbm as olbm

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _printed(name, cs2):
    """Printed matrices of a fixture, with the symbolic sound-speed entries evaluated."""
    mats, cur = {}, None
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("M0", "N"):
            cur = line
            mats[cur] = []
            continue
        vals = {"cs2": cs2, "-cs2": -cs2, "cs4": cs2 * cs2, "2cs4": 2 * cs2 * cs2}
        mats[cur].append([float(vals.get(tok, tok)) if tok in vals else float(tok) for tok in line.split()])
    return np.array(mats["M0"]), np.array(mats["N"])


D0S = (1.0 / 3.0, 0.4, 0.5)


@pytest.mark.parametrize("d0", D0S)
def test_d2q9_matches_printed_appendix(d0):
    lat = L.d2q9(d0)
    M0, N = _printed("d2q9_matrices.txt", d0)
    assert np.array_equal(lat.M0, M0)
    assert np.allclose(lat.N, N, atol=0, rtol=0)


@pytest.mark.parametrize("d0", D0S)
def test_d3q15_matches_printed_appendix(d0):
    lat = L.d3q15(d0)
    M0, N = _printed("d3q15_matrices.txt", d0)
    assert np.array_equal(lat.M0, M0)
    assert np.array_equal(lat.N, N)


@pytest.mark.parametrize("name,d0", [("D2Q9", d) for d in D0S] + [("D3Q15", d) for d in D0S]
                         + [("D3Q19", d) for d in (0.25, 1.0 / 3.0, 0.4)])
def test_weights_and_hermite_orthogonality(name, d0):
    lat = L.make(name, d0)
    w, c = lat.w, lat.c.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.all(w >= 0)   # D3Q15 at d0 = 1/2 has a zero rest weight
    for a in range(lat.d):
        assert abs(np.sum(w * c[:, a])) < 1e-15
        for b in range(lat.d):
            assert abs(np.sum(w * c[:, a] * c[:, b]) - (d0 if a == b else 0.0)) < 1e-15
    if lat.d == 2:
        assert abs(np.sum(w * c[:, 0] ** 2 * c[:, 1] ** 2) - d0 * d0) < 1e-15
    # H = N M0 is w-orthogonal: H diag(w) H^T is diagonal
    H = lat.T
    G = H @ np.diag(w) @ H.T
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-14, np.abs(off).max()
    assert np.all(np.diag(G) >= 0)   # zero norm only where a weight vanishes (D3Q15, d0 = 1/2)
    # N is unit lower triangular
    assert np.allclose(np.triu(lat.N, 1), 0) and np.allclose(np.diag(lat.N), 1)


@pytest.mark.parametrize("d0", D0S)
def test_gram_schmidt_reproduces_printed_d2q9_N(d0):
    # an independent route to N: w-weighted Gram-Schmidt of the printed monomial rows
    lat = L.d2q9(d0)
    assert np.allclose(L.gram_schmidt_N(lat.M0, lat.w), lat.N, atol=1e-14)


def test_d3q19_plain_hermite_is_not_orthogonal():
    # why D3Q19 needs the row transformation: the plain c_x^2 - cs2 row is not
    # orthogonal to (c_y^2 - cs2)(c_z^2 - cs2) on D3Q19
    lat = L.d3q19(1.0 / 3.0)
    c = lat.c.astype(float)
    cs2 = 1.0 / 3.0
    hxx = c[:, 0] ** 2 - cs2
    hyyzz = (c[:, 1] ** 2 - cs2) * (c[:, 2] ** 2 - cs2)
    assert abs(np.sum(lat.w * hxx * hyyzz) + cs2 ** 3) < 1e-15


@pytest.mark.parametrize("name", ["D2Q9", "D3Q19"])
def test_equal_rates_reduce_to_bgk(name):
    # with every rate equal to s, Lambda = M0^-1 N^-1 (s I) N M0 = s I (BGK)
    lat = L.make(name, 1.0 / 3.0)
    coll = olbm.Collision(lat)
    rng = np.random.default_rng(0)
    v = rng.standard_normal((lat.Q, 5, 4))
    s = 1.3
    out = coll.apply(np.full(lat.Q, s), v)
    assert np.allclose(out, s * v, atol=1e-13)


def test_isotropic_stencil_is_the_d0_third_lattice():
    for d in (2, 3):
        c, w, cs2 = L.isotropic_stencil(d)
        assert abs(cs2 - 1.0 / 3.0) < 1e-16
        # fourth-order isotropy: sum w c_a^4 = 3 sum w c_a^2 c_b^2 = 3 cs2^2
        cf = c.astype(float)
        assert abs(np.sum(w * cf[:, 0] ** 4) - 3 * cs2 ** 2) < 1e-15
        assert abs(np.sum(w * cf[:, 0] ** 2 * cf[:, 1] ** 2) - cs2 ** 2) < 1e-15
