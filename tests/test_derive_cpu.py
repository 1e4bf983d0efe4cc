"""The library's host derivation of the model constants against the oracle (CPU, no device call).

lbm_derive returns, in float64, what a context would hand its kernels before
rounding to float32: the wetting closure k(theta, kappa) of Eq. kk, the
spreading coefficients and gamma_T (Sec. 2.2), eta_1 and the CH rate s_1
(Sec. 3), the lattice weights (Appendix A), the viscosity relation of the NS
rates, and the prefactors and K, H constants of the pressure formula (Sec. 3).
The oracle derives each of them independently (oracle/model.py, lattice.py,
lbm.py).  The library takes cs2 = float32(d0) (so that its float32 lattice
identities hold to one rounding); quantities that depend on cs2 therefore agree
to float32 resolution, the rest to float64.
"""
import math

import numpy as np
import pytest

from oracle import lattice as olat
from oracle import lbm as olbm
from oracle import model as omodel

CASES = [
    ("D2Q9", dict(theta_deg=30.0, kappa=0.0, d0=0.5)),
    ("D2Q9", dict(theta_deg=60.0, kappa=0.75, d0=1.0 / 3.0, M_deg=0.05, eta_hat=0.05)),
    ("D2Q9", dict(theta_deg=90.0, kappa=0.2, d0=0.4, sigma=0.02)),
    ("D2Q9", dict(theta_deg=150.0, kappa=0.75, d0=0.5, M_cst=0.01)),
    ("D3Q19", dict(theta_deg=120.0, kappa=0.0, d0=1.0 / 3.0)),
    ("D3Q19", dict(theta_deg=45.0, kappa=0.3, d0=0.3, eta_hat=0.2)),
    ("D3Q15", dict(theta_deg=120.0, kappa=0.0, d0=1.0 / 3.0, eta_hat=0.05)),
    ("D3Q15", dict(theta_deg=70.0, kappa=0.5, d0=0.4)),
]
F32 = 2e-7    # relative: one float32 rounding of d0, propagated


def _lib_params(L, kw):
    return L.lbm_default_params(**kw)


def _oracle_params(L, kw):
    p = _lib_params(L, kw)
    return omodel.Params(W=p.W, M_deg=p.M_deg, M_cst=p.M_cst, theta_deg=p.theta_deg, kappa=p.kappa, sigma=p.sigma,
                         rho=tuple(p.rho), mu=tuple(p.mu), d0=p.d0, eta_hat=p.eta_hat, s_free_ch=p.s_free_ch,
                         s_free_ns=p.s_free_ns)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("name,kw", CASES)
def test_derived_constants_match_the_oracle(lbm_lib, name, kw):
    L = lbm_lib
    lattice = {"D2Q9": L.LBM_D2Q9, "D3Q19": L.LBM_D3Q19, "D3Q15": L.LBM_D3Q15}[name]
    d = L.lbm_derive(lattice, _lib_params(L, kw))
    op = _oracle_params(L, kw)
    c = omodel.constants(op)
    # wetting closure and spreading coefficients: no cs2 involved
    assert _rel(d["k"], c.k) < 1e-13
    for a, b in zip(d["gamma"], c.gamma):
        assert _rel(a, b) < 1e-13
    assert _rel(d["gamma_T"], c.gammaT) < 1e-13
    assert _rel(d["eta"], c.eta) < 1e-13
    # cs2 = float32(d0)
    assert d["cs2"] == float(np.float32(op.d0))
    assert _rel(d["s1_ch"], c.s_ch["s1"]) < F32
    # lattice weights by speed class
    lat = olat.make(name, op.d0)
    c2 = (np.asarray(lat.c) ** 2).sum(axis=1)
    far = 3 if name == "D3Q15" else 2
    w_or = [lat.w[int(np.argmax(c2 == 0))], lat.w[int(np.argmax(c2 == 1))], lat.w[int(np.argmax(c2 == far))]]
    for a, b in zip(d["w"], w_or):
        assert _rel(a, b) < F32
    # viscosity relation: the library's s2a, s2b for a viscosity nu equal the oracle's
    nu = 0.037
    s2a_o, s2b_o = olbm.viscous_rates(lat, 1.0, 0.0, nu)
    for visc, s_o in zip(d["visc"], (s2a_o, s2b_o)):
        assert _rel(1.0 / (0.5 + nu / visc), float(s_o)) < F32
    # pressure formula: prefactors and K, H at arbitrary s0, s2a
    assert _rel(d["p_f"], lat.cs2 / (1.0 - lat.w[0])) < F32
    assert _rel(d["p_w"], lat.w[0] / (1.0 - lat.cs2)) < F32
    for s0, s2a in ((1.0, 1.0), (1.3, 0.7), (0.6, 1.7)):
        K, H = olbm.pressure_constants(lat, op.d0, s0, s2a)
        h = d["p_h"]
        assert _rel(d["p_K"], K) < F32
        assert abs(d["p_K"] * (h[0] / s0 - h[1] / s2a + h[2]) - H) < 1e-6 * max(1.0, abs(H))


def test_invalid_parameters_rejected_with_a_reason(lbm_lib):
    L = lbm_lib
    with pytest.raises(L.LbmError) as e:
        L.lbm_derive(L.LBM_D2Q9, L.lbm_default_params(theta_deg=0.0))
    assert e.value.status == -1 and "theta" in str(e.value)
    with pytest.raises(L.LbmError):
        L.lbm_derive(L.LBM_D3Q19, L.lbm_default_params(d0=0.5))      # w_axis = 0: outside (0, 1/2)
    assert L.library().lbm_derive(L.LBM_D2Q9, None, None) == -1


def test_k_closure_is_eq_kk_at_90_degrees(lbm_lib):
    # at theta = 90 deg the sign term vanishes: k = 9 / (1 + kappa), and gamma_1 = gamma_2 = sigma
    L = lbm_lib
    for kappa in (0.0, 0.75):
        d = L.lbm_derive(L.LBM_D2Q9, L.lbm_default_params(theta_deg=90.0, kappa=kappa, sigma=0.01))
        assert math.isclose(d["k"], 9.0 / (1.0 + kappa), rel_tol=1e-14)
        assert math.isclose(d["gamma"][1], 0.01, rel_tol=1e-13) and math.isclose(d["gamma"][2], 0.01, rel_tol=1e-13)


def test_random_parameter_sets_agree_with_the_oracle(lbm_lib):
    # 300 seeded parameter sets over the whole admissible box: the library accepts exactly the sets whose
    # spreading coefficients the oracle finds positive, and derives the same k, gamma, eta and s_1 for them
    L = lbm_lib
    rng = np.random.default_rng(20231109)
    accepted = rejected = 0
    for _ in range(300):
        name = ("D2Q9", "D3Q19", "D3Q15")[rng.integers(3)]
        # kappa up to 40: gamma_1 = sigma (1 - cos theta) and gamma_2 = sigma (1 + cos theta) are always positive,
        # gamma_0 = sigma (2 k + cos theta - 1) turns negative once k(theta, kappa) is small enough
        kappa = float(rng.uniform(-0.9, 3.0) if rng.random() < 0.6 else rng.uniform(3.0, 40.0))
        kw = dict(theta_deg=float(rng.uniform(1.0, 179.0)), kappa=kappa,
                  sigma=float(10 ** rng.uniform(-3, -1)), M_deg=float(10 ** rng.uniform(-3, 0)),
                  eta_hat=float(10 ** rng.uniform(-2, 0)),
                  d0=float(rng.uniform(0.05, 0.95 if name == "D2Q9" else 0.45)))
        lattice = {"D2Q9": L.LBM_D2Q9, "D3Q19": L.LBM_D3Q19, "D3Q15": L.LBM_D3Q15}[name]
        k, gam = omodel.spreading(math.radians(kw["theta_deg"]), kw["kappa"], kw["sigma"])
        if min(gam) <= 0.0:
            with pytest.raises(L.LbmError):
                L.lbm_derive(lattice, _lib_params(L, kw))
            rejected += 1
            continue
        d = L.lbm_derive(lattice, _lib_params(L, kw))
        c = omodel.constants(_oracle_params(L, kw))
        assert _rel(d["k"], c.k) < 1e-12, kw
        assert max(_rel(a, b) for a, b in zip(d["gamma"], c.gamma)) < 1e-9, kw
        assert _rel(d["eta"], c.eta) < 1e-9, kw
        assert _rel(d["s1_ch"], c.s_ch["s1"]) < F32, kw
        accepted += 1
    assert accepted > 100 and rejected > 10, (accepted, rejected)
