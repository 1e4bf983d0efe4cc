"""Pins of the oracle's velocity inlet and pressure outlet (non-equilibrium
extrapolation, Sec. 4 intro) to the equilibrium moments they must impose and
to plane Poiseuille flow."""
import numpy as np
import pytest

from oracle import lbm, model


def _equilibrium_state(lattice, shape, seed):
    """A state whose streamed populations are exact equilibria of smooth random fields."""
    r = np.random.default_rng(seed)
    prm = model.Params(rho=(1.0, 2.0, 0.5), mu=(0.1, 0.1, 0.1), d0=0.5 if lattice == "D2Q9" else 1.0 / 3.0)
    lat = lbm.L.make(lattice, prm.d0)
    d = lat.d
    phi0 = np.clip(r.uniform(-0.2, 0.4, shape), 0.0, None)
    phi1 = r.uniform(0.0, 1.0, shape) * (1.0 - phi0)
    u = r.normal(0.0, 0.02, (d,) + shape)
    p = r.normal(0.0, 0.01, shape)
    rho = prm.rho[0] * phi0 + prm.rho[1] * phi1 + prm.rho[2] * (1.0 - phi0 - phi1)
    st = lbm.init_state(lattice, phi0, phi1, prm, (False,) + (True,) * (d - 1))
    zero = np.zeros(shape)
    st.f = lbm.f_equilibrium(lat, phi1, zero, u, 0.0)
    st.g = lbm.g_equilibrium(lat, p, rho, u, np.zeros_like(u), prm.rho[0])
    return st, prm, lat, (phi0, phi1, u, p, rho)


def _local_pressure(lat, g, rho, u):
    return lat.cs2 / (1.0 - lat.w[0]) * (g[1:].sum(axis=0) - lat.w[0] * rho * (u ** 2).sum(axis=0) / (1 - lat.cs2))


@pytest.mark.parametrize("lattice,shape", [("D2Q9", (5, 8)), ("D3Q19", (3, 4, 6)), ("D3Q15", (3, 4, 6))])
def test_boundary_nodes_carry_the_imposed_moments(lattice, shape):
    st, prm, lat, (phi0, phi1, u, p, rho) = _equilibrium_state(lattice, shape, 1)
    d = lat.d
    col = shape[:-1]
    u_in = np.random.default_rng(2).normal(0.0, 0.01, (d,) + col)
    st.inout = lbm.InOut(u_in=u_in, phi_in=0.3, p_out=0.004)
    lbm.inout_boundaries(st)
    for xb, xf in ((0, 1), (-1, -2)):
        fb, gb = st.f[..., xb], st.g[..., xb]
        phi_b = fb.sum(axis=0)
        rho_b = prm.rho[0] * phi0[..., xb] + prm.rho[1] * phi_b + prm.rho[2] * (1 - phi0[..., xb] - phi_b)
        j = np.stack([sum(float(ci[a]) * gb[i] for i, ci in enumerate(lat.c)) for a in range(d)])
        ub = j / rho_b
        if xb == 0:
            # inlet: the given phase field and velocity, the neighbour's pressure
            np.testing.assert_allclose(phi_b, 0.3, atol=1e-13)
            np.testing.assert_allclose(ub, u_in, atol=1e-13)
            np.testing.assert_allclose(_local_pressure(lat, gb, rho_b, ub), p[..., xf], atol=1e-13)
            # the CH first moment is the imposed phase flux
            jf = np.stack([sum(float(ci[a]) * fb[i] for i, ci in enumerate(lat.c)) for a in range(d)])
            np.testing.assert_allclose(jf, 0.3 * u_in, atol=1e-13)
        else:
            # outlet: the neighbour's phase field and velocity, the given pressure
            np.testing.assert_allclose(phi_b, phi1[..., xf], atol=1e-13)
            np.testing.assert_allclose(ub, u[..., xf], atol=1e-12)
            np.testing.assert_allclose(_local_pressure(lat, gb, rho_b, ub), 0.004, atol=1e-13)
    # interior columns are untouched
    st2, *_ = _equilibrium_state(lattice, shape, 1)
    np.testing.assert_array_equal(st.f[..., 1:-1], st2.f[..., 1:-1])


def test_neighbour_non_equilibrium_part_is_copied():
    st, prm, lat, _ = _equilibrium_state("D2Q9", (6, 7), 3)
    r = np.random.default_rng(4)
    neq = r.normal(0.0, 1e-3, st.g[..., 1].shape)
    st.g[..., 1] += neq
    g_before = st.g.copy()
    st.inout = lbm.InOut(u_in=(0.01, 0.0), phi_in=None, p_out=None)
    lbm.inout_boundaries(st)
    # the boundary node's populations differ from their equilibrium by the neighbour's perturbation,
    # up to the change of the neighbour's velocity and pressure the perturbation itself causes
    assert np.abs(st.g[..., 0] - g_before[..., 0]).max() > 0
    np.testing.assert_array_equal(st.g[..., -1], g_before[..., -1])   # no outlet: last column untouched


def test_inlet_outlet_need_an_open_x_axis():
    prm = model.Params()
    st = lbm.init_state("D2Q9", np.zeros((4, 6)), np.ones((4, 6)), prm, (True, False))
    st.inout = lbm.InOut(u_in=(0.01, 0.0), p_out=0.0)
    with pytest.raises(ValueError):
        lbm.step(st)


def test_plane_poiseuille_flow():
    """Parabolic inlet, pressure outlet, no-slip walls in y: steady flux, profile and pressure gradient."""
    nx, ny, U, mu = 40, 10, 0.01, 0.1
    prm = model.Params(rho=(1.0, 1.0, 1.0), mu=(mu, mu, mu), d0=0.5)
    st = lbm.init_state("D2Q9", np.zeros((ny, nx)), np.ones((ny, nx)), prm, (False, False))
    y = np.arange(ny) + 0.5                      # half-way walls at y = 0 and y = ny
    prof = 1.5 * U * (1.0 - ((y - ny / 2) / (ny / 2)) ** 2)
    st.inout = lbm.InOut(u_in=np.stack([prof, 0.0 * prof]), phi_in=1.0, p_out=0.0)
    c = model.constants(prm)
    lbm.step(st, c, nsteps=1800)
    u, p = st.macro["u"], st.macro["p"]
    flux = u[0].sum(axis=0) / (ny * U)
    assert np.all(np.abs(flux[1:-1] - 1.0) < 0.01), flux
    mid = u[0][:, nx // 2]
    assert np.abs(mid - prof).max() < 0.02 * U
    dpdx = (p[:, 3 * nx // 4].mean() - p[:, nx // 4].mean()) / (nx / 2)
    assert abs(dpdx / (-12.0 * mu * U / ny ** 2) - 1.0) < 0.01, dpdx
    assert np.abs(u[1]).max() < 0.02 * U
