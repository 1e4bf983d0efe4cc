"""Writes flat_wall_equilibrium.txt: the FP64 oracle's long-run state of the flat-wall configuration.

Set-up of the droplet-on-a-wall experiment (Sec. 4.2) at 128 x 64: bottom 8
rows a tanh solid of width W = 4, half-disk droplet of radius 25 on the wall
(a 90 deg start for every target angle), sigma 0.01, densities 1, viscosities
0.01, mobility M_deg 0.1, d0 = 1/2, periodic in x, no-flux walls in y; target
contact angles 30, 60, 90, 120 and 150 deg; 60000 steps.  For each angle it
records the contact angle from the droplet height (Sec. 4.2 relation, area
radius R0), the height, the Laplace pressure (bulk means), the phase mass, the
largest velocity, the angle every 2000 steps, and the phase field on the
droplet's symmetry column and on row 12.

Only ``oracle/`` and the input generators are used.  Run from the repository
root:  python tests/golden/make_flat_wall_equilibrium.py  (about 10 minutes
per angle on one core; the angles run in parallel processes).
"""
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

THETAS = (30.0, 60.0, 90.0, 120.0, 150.0)
STEPS, EVERY, ROW = 60000, 2000, 12


def one(theta):
    import numpy as np
    from oracle import lbm, model
    from oracle import observables as ob
    from synthetic.workloads import flat_wall
    wl = flat_wall(theta=theta, d0=0.5)
    phi0 = wl["phi0"][0].astype(np.float64)
    phi1 = wl["phi1"][0].astype(np.float64)
    prm = model.Params(**wl["params"][0])
    c = model.constants(prm)
    st = lbm.init_state("D2Q9", phi0, phi1, prm, (True, False), consts=c)
    trace = []
    for s in range(EVERY, STEPS + 1, EVERY):
        lbm.step(st, c, EVERY)
        trace.append((s, ob.flat_wall_angle(phi0, st.macro["phi1"], 64)[0]))
    th, H, R0 = ob.flat_wall_angle(phi0, st.macro["phi1"], 64)
    u = st.macro["u"]
    return dict(theta_in=theta, steps=STEPS, theta_deg=float(th), height=float(H), R0=float(R0),
                dp=float(ob.laplace_dp(phi0, st.macro["phi1"], st.macro["p"])), mass1=ob.mass(st.macro["phi1"]),
                umax=float(np.sqrt(u[0] ** 2 + u[1] ** 2).max()), trace=[(s, float(t)) for s, t in trace],
                column=st.macro["phi1"][:, 64].tolist(), row=st.macro["phi1"][ROW, :].tolist())


def main():
    with mp.get_context("spawn").Pool(len(THETAS)) as pool:
        res = pool.map(one, THETAS)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flat_wall_equilibrium.txt")
    with open(out, "w") as fh:
        fh.write("# FP64 oracle, flat-wall configuration of Sec. 4.2 at 128 x 64 (see make_flat_wall_equilibrium.py)\n")
        fh.write(f"# steps {STEPS}; probe column 64; row {ROW}\n")
        for r in res:
            fh.write(f"theta_in {r['theta_in']!r}\n")
            for key in ("steps", "theta_deg", "height", "R0", "dp", "mass1", "umax"):
                fh.write(f"{key} {r[key]!r}\n")
            fh.write("trace " + " ".join(f"{s}:{t!r}" for s, t in r["trace"]) + "\n")
            fh.write("column " + " ".join(repr(v) for v in r["column"]) + "\n")
            fh.write("row " + " ".join(repr(v) for v in r["row"]) + "\n")
    print(out)


if __name__ == "__main__":
    main()
