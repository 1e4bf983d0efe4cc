"""One coupled CH + NS lattice Boltzmann time step of the 2f1s model, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Arrays are indexed ``[y, x]`` (2D) or ``[z, y, x]`` (3D); populations carry a
leading direction axis.  ``periodic`` lists (x, y[, z]); a non-periodic axis
has half-way bounce-back walls half a spacing beyond its first and last node
(Sec. 4, half-way bounce-back for no-flux and no-slip).  dt = dx = c = 1.

State at time n: the post-streaming populations f_i (CH, Sec. 3 first
evolution equation) and g_i (NS, second evolution equation), the frozen solid
indicator phi0, and the previous-step history (phi1, u, S) used by the explicit
Euler time derivatives and by the correction force (readings below).

Per step, in the paper's order (Sec. 2 and 3):
 1. phi1 = sum_i f_i.
 2. Isotropic stencils: grad/Laplacian of phi0 and phi1; phi2 = 1 - phi0 - phi1.
 3. mu_p = df_b/dphi_p - (3D/4) gamma_p lap phi_p  (Sec. 2.1), and
    mubar_1 = gamma_T/3 sum_{q != 1} (mu_1 - mu_q)/gamma_q  (Eq. CHmodel).
 4. grad mubar_1 (stencil).
 5. Degenerate mobility M = M_cst + M_deg phi1 (1-phi1)(1-phi0) (Sec. 4 text).
 6. Flux S, density and viscosity mixtures, F_s = sum_p mu_p grad phi_p,
    F_c = div(S u - u S)/2, F_b; F = F_s + F_b + F_c (Sec. 2.3, Sec. 3).
 7. rho u* = sum c_i g_i + F/2, f = (u_w - u*), u = u* + phi0 f / 2.
 8. Local s2a, s2b from the viscosity relation; K, H; pressure p (Sec. 3).
 9. CH collision  f* = f - L(f - f^eq) + (I - L/2) R,  L = M0^-1 N^-1 K N M0.
10. NS collision  g* = g - L(g - g^eq) + (I - L/2) F_i.
11. Streaming with half-way bounce-back; history <- (phi1, u, S).

Readings where the paper is silent:
* S with frozen phi0 is (rho1 - rho2) M grad(mubar_1) / gamma_1.
* F_c and the Euler derivatives use the stored step n-1 fields; the history
  starts as (phi1^0, u = 0, S = 0).
* d_t(rho u u) ~ u F + F u with F = F_s + F_b + F_c as the paper defines F.
* F_b = (1 - phi0) b with a force density b.
* rho_0 in lambda_0 is a constant (default: the solid density rho_0); the
  dynamics do not depend on it (tests check this).
* 1 - phi0 is evaluated as max(1 - phi0, 2^-24) inside the viscosity relation,
  so that nodes whose solid indicator rounds to exactly 1 get a finite rate.
* The NS rates the paper leaves open: s0 and s4 equal the local s2a, s1 and
  s3 take ``s_free_ns`` (default 1).  Because the pressure is recovered from
  the non-conserved moments H0, tr H2 and H4, a rate set with s0 = s4 = 1 is
  linearly unstable at rest for nu = 0.01 (spectral radius 1.03-1.04 at
  d0 = 1/3 and 1/2); tying s0 and s4 to s2a is stable for every d0 and
  viscosity tested (the tests repeat this check).
* Stencils: see ``lattice.isotropic_stencil``; non-periodic axes use mirror
  ghost nodes (zero normal gradient).
* The initial populations are f = f^eq(phi1, mubar_1, u = 0) and
  g = g^eq(p = 0, u = 0).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import lattice as L
from .model import Params, constants

ONE_MINUS_PHI0_FLOOR = 2.0 ** -24


# --- neighbour access -----------------------------------------------------------

def _axis(a, d):
    """Array axis that holds velocity component a (x is the last axis)."""
    return d - 1 - a


def padded(field, periodic):
    """field with one ghost layer: wrap on periodic axes, mirror on wall axes."""
    d = field.ndim
    out = field
    for a in range(d):
        mode = "wrap" if periodic[a] else "symmetric"
        widths = [(0, 0)] * d
        widths[_axis(a, d)] = (1, 1)
        out = np.pad(out, widths, mode=mode)
    return out


def at_offset(P, ci, shape):
    """Values at x + c_i taken from a 1-padded array P."""
    d = len(shape)
    sl = [None] * d
    for a in range(d):
        ax = _axis(a, d)
        s = 1 + int(ci[a])
        sl[ax] = slice(s, s + shape[ax])
    return P[tuple(sl)]


def grad_lap(field, periodic):
    """Second-order isotropic central gradient and Laplacian (see lattice docstring)."""
    d = field.ndim
    c_iso, w_iso, cs2_iso = L.isotropic_stencil(d)
    P = padded(field, periodic)
    grad = np.zeros((d,) + field.shape)
    lap = np.zeros(field.shape)
    for ci, wi in zip(c_iso, w_iso):
        nb = at_offset(P, ci, field.shape)
        for a in range(d):
            if ci[a] != 0:
                grad[a] += wi * ci[a] * nb / cs2_iso
        lap += 2.0 * wi * (nb - field) / cs2_iso
    return grad, lap


def stream(fstar, lat, periodic):
    """f_i(x + c_i, t+1) = f_i*(x, t); half-way bounce-back on wall axes."""
    d = lat.d
    out = np.empty_like(fstar)
    shape = fstar.shape[1:]
    for i, ci in enumerate(lat.c):
        moved = fstar[i]
        for a in range(d):
            if ci[a] != 0:
                moved = np.roll(moved, int(ci[a]), axis=_axis(a, d))
        # nodes whose upstream node x - c_i lies beyond a wall receive the
        # reflected population of the opposite direction from the same node
        mask = np.zeros(shape, dtype=bool)
        for a in range(d):
            if periodic[a] or ci[a] == 0:
                continue
            idx = [slice(None)] * d
            idx[_axis(a, d)] = 0 if ci[a] > 0 else shape[_axis(a, d)] - 1
            mask[tuple(idx)] = True
        out[i] = np.where(mask, fstar[lat.opp[i]], moved)
    return out


# --- collision operator ----------------------------------------------------------

def _mv(A, v):
    """Matrix times a field of vectors: (Q,Q) x (Q, ...) -> (Q, ...)."""
    return (A @ v.reshape(v.shape[0], -1)).reshape((A.shape[0],) + v.shape[1:])


class Collision:
    """Lambda = (N M0)^-1 K (N M0) = M0^-1 (N^-1 K N) M0 with C_d = I (Sec. 4 intro, Appendix A)."""

    def __init__(self, lat):
        self.lat = lat
        self.T = lat.N @ lat.M0
        self.Tinv = np.linalg.inv(lat.M0) @ np.linalg.inv(lat.N)

    def apply(self, Kdiag, v):
        """Lambda v for a per-node diagonal K given as (Q, ...) or (Q,)."""
        n = _mv(self.T, v)
        K = Kdiag.reshape(Kdiag.shape + (1,) * (v.ndim - Kdiag.ndim)) if Kdiag.ndim < v.ndim else Kdiag
        return _mv(self.Tinv, K * n)

    def step(self, Kdiag, h, heq, src):
        """h - Lambda (h - h^eq) + (I - Lambda/2) src."""
        return h - self.apply(Kdiag, h - heq) + src - 0.5 * self.apply(Kdiag, src)


_COLL_CACHE = {}


def collision_for(lat):
    key = (lat.name, lat.cs2)
    if key not in _COLL_CACHE:
        _COLL_CACHE[key] = Collision(lat)
    return _COLL_CACHE[key]


# --- state -----------------------------------------------------------------------

@dataclasses.dataclass
class State:
    lat: L.Lattice
    params: Params
    periodic: tuple
    f: np.ndarray
    g: np.ndarray
    phi0: np.ndarray
    hist_phi1: np.ndarray
    hist_u: np.ndarray
    hist_S: np.ndarray
    step: int = 0
    macro: dict = dataclasses.field(default_factory=dict)
    macro_cache: dict = dataclasses.field(default_factory=dict)
    inout: "InOut | None" = None

    @property
    def shape(self):
        return self.phi0.shape


def _cdot(ci, v):
    return sum(float(ci[a]) * v[a] for a in range(len(ci)))


def chemical_potentials(phi0, phi1, periodic, consts, W, phi0_stencil=None):
    """mu_p for p = 0, 1, 2 and mubar_1 (Sec. 2.1) plus the stencil results."""
    g0, g1, g2 = consts.gamma
    gT = consts.gammaT
    phi2 = 1.0 - phi0 - phi1
    grad0, lap0 = grad_lap(phi0, periodic) if phi0_stencil is None else phi0_stencil
    grad1, lap1 = grad_lap(phi1, periodic)
    grad2, lap2 = -grad0 - grad1, -lap0 - lap1
    mus = []
    for gam, ph, lp in ((g0, phi0, lap0), (g1, phi1, lap1), (g2, phi2, lap2)):
        # d f_b / d phi_p = (12/D) gamma_p phi_p (1 - phi_p)(1 - 2 phi_p)
        dfb = 12.0 / W * gam * ph * (1.0 - ph) * (1.0 - 2.0 * ph)
        mus.append(dfb - 0.75 * W * gam * lp)
    mu0, mu1, mu2 = mus
    mubar1 = gT / 3.0 * ((mu1 - mu0) / g0 + (mu1 - mu2) / g2)
    return dict(phi2=phi2, grad=(grad0, grad1, grad2), lap=(lap0, lap1, lap2), mu=(mu0, mu1, mu2),
                mubar1=mubar1)


def f_equilibrium(lat, phi1, mubar1, u, eta):
    """CH equilibrium (Sec. 3): f_0 = phi + (w_0 - 1) eta mubar,
    f_i = w_i eta mubar + w_i c_i . phi u / cs2."""
    cs2 = lat.cs2
    feq = np.empty((lat.Q,) + phi1.shape)
    for i, ci in enumerate(lat.c):
        if i == 0:
            feq[i] = phi1 + (lat.w[0] - 1.0) * eta * mubar1
        else:
            feq[i] = lat.w[i] * eta * mubar1 + lat.w[i] * _cdot(ci, phi1 * u) / cs2
    return feq


def g_equilibrium(lat, p, rho, u, S, rho_ref):
    """NS equilibrium (Sec. 3): lambda_i + w_i c.rho u/cs2 + w_i [diagonal + off-diagonal]."""
    cs2 = lat.cs2
    d = lat.d
    geq = np.empty((lat.Q,) + p.shape)
    for i, ci in enumerate(lat.c):
        lam = (lat.w[0] - 1.0) * p / cs2 + rho_ref if i == 0 else lat.w[i] * p / cs2
        diag = sum((ci[a] ** 2 - cs2) * (rho * u[a] * u[a] - S[a] * u[a]) for a in range(d)) / (cs2 - cs2 * cs2)
        off = 0.0
        for a in range(d):
            for b in range(a + 1, d):
                off = off + ci[a] * ci[b] * (rho * u[a] * u[b] - 0.5 * (S[a] * u[b] + u[a] * S[b])) / (cs2 * cs2)
        geq[i] = lam + lat.w[i] * _cdot(ci, rho * u) / cs2 + lat.w[i] * (diag + off)
    return geq


def ns_forcing(lat, u, gradrho, Ft, M2F):
    """F_i = w_i [u.grad rho + c_i.(F + phi0 rho f)/cs2 + diag M2F + off-diag M2F] (Sec. 3)."""
    cs2 = lat.cs2
    d = lat.d
    udg = sum(u[a] * gradrho[a] for a in range(d))
    Fi = np.empty((lat.Q,) + udg.shape)
    for i, ci in enumerate(lat.c):
        diag = sum((ci[a] ** 2 - cs2) * M2F[a][a] for a in range(d)) / (cs2 - cs2 * cs2)
        off = 0.0
        for a in range(d):
            for b in range(a + 1, d):
                off = off + ci[a] * ci[b] * M2F[a][b] / (cs2 * cs2)
        Fi[i] = lat.w[i] * (udg + _cdot(ci, Ft) / cs2 + diag + off)
    return Fi


def pressure_constants(lat, d0, s0, s2a):
    """K and H of the pressure formula (Sec. 3, after the fluid-structure force).

    The 2D constants are the printed D2Q9 ones; the 3D ones are taken as printed
    for D3Q15 and used for D3Q19 too.  H multiplies u . grad rho, which vanishes at
    rest, so the pressure pins (equilibrium pressure, Laplace law) do not reach it:
    parity unpinned for H beyond the oracle-vs-GPU comparison."""
    if lat.d == 2:
        K = 1.0 - d0
        H = K * ((1.0 - d0) / s0 - (2.0 - 4.0 * d0) / s2a + (1.0 - 3.0 * d0) / 2.0)
    else:
        K = 1.0 - 2.0 * d0
        H = K * ((1.0 - d0) / s0 - (3.0 - 7.0 * d0) / s2a + (1.0 - 3.0 * d0))
    return K, H


def viscous_rates(lat, rho, phi0, muv):
    """s2a, s2b from mu/(rho (1-phi0)) = (1/s2a - 1/2)(c^2 - cs2)/2 = (1/s2b - 1/2) cs2."""
    cs2 = lat.cs2
    one_m = np.maximum(1.0 - phi0, ONE_MINUS_PHI0_FLOOR)
    nu_eff = muv / (rho * one_m)
    s2a = 1.0 / (0.5 + nu_eff / ((1.0 - cs2) / 2.0))
    s2b = 1.0 / (0.5 + nu_eff / cs2)
    return s2a, s2b


def macroscopic(st: State, consts, collect=True):
    """Steps 1-8 for every node; returns a dict of fields."""
    lat, prm = st.lat, st.params
    d = lat.d
    cs2 = lat.cs2
    f, g = st.f, st.g
    phi0 = st.phi0
    rho0, rho1, rho2 = prm.rho
    mv0, mv1, mv2 = prm.mu
    g1 = consts.gamma[1]

    phi1 = f.sum(axis=0)
    if "phi0_stencil" not in st.macro_cache:
        st.macro_cache["phi0_stencil"] = grad_lap(phi0, st.periodic)  # phi0 is frozen
    cp = chemical_potentials(phi0, phi1, st.periodic, consts, prm.W, st.macro_cache["phi0_stencil"])
    phi2 = cp["phi2"]
    grad0, grad1, grad2 = cp["grad"]
    mu0, mu1, mu2 = cp["mu"]
    mubar1 = cp["mubar1"]
    gradmu, _ = grad_lap(mubar1, st.periodic)

    fdeg = phi1 * (1.0 - phi1) * (1.0 - phi0)
    M = prm.M_cst + prm.M_deg * fdeg
    S = (rho1 - rho2) * M * gradmu / g1

    rho = rho0 * phi0 + rho1 * phi1 + rho2 * phi2
    gradrho = rho0 * grad0 + rho1 * grad1 + rho2 * grad2
    muv = mv0 * phi0 + mv1 * phi1 + mv2 * phi2

    Fs = mu0 * grad0 + mu1 * grad1 + mu2 * grad2

    # correction force from the stored step n-1 fields: (F_c)_b = 1/2 sum_a d_a (S_a u_b - u_a S_b)
    hu, hS = st.hist_u, st.hist_S
    Fc = np.zeros((d,) + phi0.shape)
    for a in range(d):
        for b in range(d):
            if a == b:
                continue
            grad_ab, _ = grad_lap(hS[a] * hu[b] - hu[a] * hS[b], st.periodic)
            Fc[b] += 0.5 * grad_ab[a]
    Fb = np.stack([(1.0 - phi0) * prm.body_force[a] for a in range(d)])
    F = Fs + Fb + Fc

    mom = np.stack([sum(float(ci[a]) * g[i] for i, ci in enumerate(lat.c)) for a in range(d)])
    ustar = (mom + 0.5 * F) / rho
    ffs = 0.0 - ustar                          # f = (u_w - u*)/dt with u_w = 0
    u = ustar + 0.5 * phi0 * ffs
    Ft = F + phi0 * rho * ffs

    s2a, s2b = viscous_rates(lat, rho, phi0, muv)
    s0n = s2a                                  # NS zeroth-order rate tied to s2a (reading)
    Kc, H = pressure_constants(lat, prm.d0, s0n, s2a)
    udg = sum(u[a] * gradrho[a] for a in range(d))
    q = sum((rho * u[a] - S[a]) * u[a] for a in range(d))
    rho_prev = rho0 * phi0 + rho1 * st.hist_phi1 + rho2 * (1.0 - phi0 - st.hist_phi1)
    q_prev = sum((rho_prev * hu[a] - hS[a]) * hu[a] for a in range(d))
    dq = q - q_prev
    w0 = lat.w[0]
    p = cs2 / (1.0 - w0) * (g[1:].sum(axis=0) + (0.5 + H) * udg - w0 * q / (1.0 - cs2) + Kc * 0.5 * dq)

    return dict(phi0=phi0, phi1=phi1, phi2=phi2, grad0=grad0, grad1=grad1, mu=(mu0, mu1, mu2),
                mubar1=mubar1, gradmu=gradmu, fdeg=fdeg, M=M, S=S, rho=rho, gradrho=gradrho, muv=muv,
                Fs=Fs, Fc=Fc, Fb=Fb, F=F, Ft=Ft, ustar=ustar, u=u, s2a=s2a, s2b=s2b, H=H, Kc=Kc,
                udg=udg, q=q, dq=dq, p=p)


def collide(st: State, consts, m):
    lat, prm = st.lat, st.params
    d = lat.d
    cs2 = lat.cs2
    coll = collision_for(lat)
    phi1, u, S = m["phi1"], m["u"], m["S"]

    # CH: f_eq, R, Hermite MRT
    feq = f_equilibrium(lat, phi1, m["mubar1"], u, consts.eta)
    dt_phiu = phi1 * u - st.hist_phi1 * st.hist_u
    corr = prm.M_deg * (1.0 - m["fdeg"]) / (prm.M_cst + prm.M_deg)
    R = np.empty_like(st.f)
    for i, ci in enumerate(lat.c):
        R[i] = lat.w[i] * (_cdot(ci, dt_phiu) / cs2 + corr * consts.eta * _cdot(ci, m["gradmu"]))
    Kch = np.array([consts.s_ch[gname] for gname in lat.groups])
    fstar = coll.step(Kch, st.f, feq, R)

    # NS: g_eq with the pressure of this step, forcing with M^2F
    rho_ref = prm.rho[0] if prm.rho_ref is None else prm.rho_ref
    geq = g_equilibrium(lat, m["p"], m["rho"], u, S, rho_ref)
    hu, hS = st.hist_u, st.hist_S
    F, Ft, gr = m["F"], m["Ft"], m["gradrho"]
    M2F = [[None] * d for _ in range(d)]
    for a in range(d):
        for b in range(d):
            dSU = 0.5 * (S[a] * u[b] + u[a] * S[b]) - 0.5 * (hS[a] * hu[b] + hu[a] * hS[b])
            val = u[a] * F[b] + F[a] * u[b] - dSU + cs2 * (u[a] * gr[b] + gr[a] * u[b])
            if a == b:
                val = val + (1.0 - 3.0 * cs2) * m["udg"]
            M2F[a][b] = val
    Fi = ns_forcing(lat, u, gr, Ft, M2F)
    # s0 and s4 follow the local s2a, s1 and s3 take the free NS rate (reading)
    rates = {"s0": m["s2a"], "s1": consts.s_ns_free["s1"], "s2a": m["s2a"], "s2b": m["s2b"],
             "s3": consts.s_ns_free["s3"], "s4": m["s2a"]}
    Kns = np.empty((lat.Q,) + phi1.shape)
    for k, gname in enumerate(lat.groups):
        Kns[k] = rates[gname]
    gstar = coll.step(Kns, st.g, geq, Fi)
    return fstar, gstar


@dataclasses.dataclass
class InOut:
    """Velocity inlet at the first x column and pressure outlet at the last
    one, by non-equilibrium extrapolation (Sec. 4 intro: the scheme of Guo,
    Zheng and Shi for velocity or pressure boundaries).  ``u_in``: the inlet
    velocity, a d-tuple (uniform) or an array (d,) + the shape of a column
    ([y] in 2D, [z, y] in 3D); None leaves x = 0 a bounce-back wall, and
    ``p_out`` None the last column; ``phi_in`` None extrapolates phi1 at the
    inlet (zero gradient)."""

    u_in: tuple | None = None
    phi_in: float | None = None
    p_out: float | None = None


def inout_boundaries(st: State):
    """Replace the post-streaming populations of the boundary columns:

    f_i(x_b) = f_i(x_f) + f_i^eq(phi_b, u_b) - f_i^eq(phi_f, u_f)
    g_i(x_b) = g_i(x_f) + g_i^eq(p_b, rho_b, u_b) - g_i^eq(p_f, rho_f, u_f)

    with x_f the neighbouring column.  At x_f: phi_f = sum f_i, rho_f from the
    densities, u_f = sum c_i g_i / rho_f and the local part of the pressure
    formula p_f = cs2/(1 - w_0) (sum_{i != 0} g_i - w_0 rho_f |u_f|^2 / (1 - cs2)).
    The chemical potential and the flux S enter both equilibria alike and
    cancel.  Inlet: u_b = u_in, phi_b = phi_in (or phi_f), p_b = p_f.
    Outlet: u_b = u_f, phi_b = phi_f, p_b = p_out."""
    io = st.inout
    lat, prm = st.lat, st.params
    d, cs2, w0 = lat.d, lat.cs2, lat.w[0]
    rho_ref = prm.rho[0] if prm.rho_ref is None else prm.rho_ref
    nx = st.phi0.shape[-1]
    sides = []
    if io.u_in is not None:
        sides.append((0, 1, "in"))
    if io.p_out is not None:
        sides.append((nx - 1, nx - 2, "out"))
    new_f, new_g = st.f.copy(), st.g.copy()
    for xb, xf, kind in sides:
        ff, gf = st.f[..., xf], st.g[..., xf]
        phi0_f, phi0_b = st.phi0[..., xf], st.phi0[..., xb]
        phi_f = ff.sum(axis=0)
        rho = lambda p0, p1: prm.rho[0] * p0 + prm.rho[1] * p1 + prm.rho[2] * (1.0 - p0 - p1)
        rho_f = rho(phi0_f, phi_f)
        u_f = np.stack([sum(float(ci[a]) * gf[i] for i, ci in enumerate(lat.c)) for a in range(d)]) / rho_f
        p_f = cs2 / (1.0 - w0) * (gf[1:].sum(axis=0) - w0 * rho_f * (u_f ** 2).sum(axis=0) / (1.0 - cs2))
        if kind == "in":
            phi_b = phi_f if io.phi_in is None else np.full_like(phi_f, io.phi_in)
            u_b = np.stack([np.broadcast_to(np.asarray(io.u_in[a], dtype=np.float64), phi_f.shape)
                            for a in range(d)])
            p_b = p_f
        else:
            phi_b, u_b, p_b = phi_f, u_f, np.full_like(phi_f, io.p_out)
        rho_b = rho(phi0_b, phi_b)
        zero = np.zeros_like(phi_f)
        zvec = np.zeros_like(u_f)
        new_f[..., xb] = ff + f_equilibrium(lat, phi_b, zero, u_b, 0.0) - f_equilibrium(lat, phi_f, zero, u_f, 0.0)
        new_g[..., xb] = gf + g_equilibrium(lat, p_b, rho_b, u_b, zvec, rho_ref) - \
            g_equilibrium(lat, p_f, rho_f, u_f, zvec, rho_ref)
    st.f, st.g = new_f, new_g


def step(st: State, consts=None, nsteps=1):
    """Advance the state by ``nsteps`` time steps in place; returns the state."""
    consts = constants(st.params) if consts is None else consts
    if st.inout is not None and st.periodic[0]:
        raise ValueError("inlet / outlet columns need a non-periodic x axis")
    for _ in range(nsteps):
        m = macroscopic(st, consts)
        fstar, gstar = collide(st, consts, m)
        st.f = stream(fstar, st.lat, st.periodic)
        st.g = stream(gstar, st.lat, st.periodic)
        if st.inout is not None:
            inout_boundaries(st)
        st.hist_phi1 = m["phi1"]
        st.hist_u = m["u"]
        st.hist_S = m["S"]
        st.macro = dict(phi1=m["phi1"], u=m["u"], p=m["p"], mubar1=m["mubar1"], S=m["S"], rho=m["rho"])
        st.step += 1
    return st


def init_state(lattice_name, phi0, phi1, params: Params, periodic, consts=None):
    """Equilibrium start: f = f^eq(phi1, mubar_1(phi1), u = 0), g = g^eq(p = 0, u = 0)."""
    lat = L.make(lattice_name, params.d0)
    consts = constants(params) if consts is None else consts
    phi0 = np.asarray(phi0, dtype=np.float64)
    phi1 = np.asarray(phi1, dtype=np.float64)
    d = lat.d
    if phi0.ndim != d:
        raise ValueError("field rank does not match lattice")
    zeros = np.zeros((d,) + phi0.shape)
    cp = chemical_potentials(phi0, phi1, periodic, consts, params.W)
    f = f_equilibrium(lat, phi1, cp["mubar1"], zeros, consts.eta)
    rho_ref = params.rho[0] if params.rho_ref is None else params.rho_ref
    rho = params.rho[0] * phi0 + params.rho[1] * phi1 + params.rho[2] * (1 - phi0 - phi1)
    g = g_equilibrium(lat, np.zeros_like(phi0), rho, zeros, zeros, rho_ref)
    return State(lat, params, tuple(periodic), f, g, phi0.copy(), phi1.copy(), zeros.copy(), zeros.copy())
