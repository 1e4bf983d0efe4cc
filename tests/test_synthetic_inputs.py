"""Seeded input generators: the block-vectorised forms equal their one-at-a-time definitions."""
import math

import numpy as np

from synthetic import rsa_spheres, spheres_phi0, splitmix64, splitmix64_block


def _rsa_one_at_a_time(n, seed, rmin, rmax, target, max_fail):
    # the definition: draw (r, cx, cy, cz), accept when clear of every accepted sphere
    u = splitmix64(seed * 104729 + 3)
    L = float(n)
    out, vol, fails = [], 0.0, 0
    while vol / L ** 3 < target and fails < max_fail:
        r = rmin + (rmax - rmin) * u()
        c = (L * u(), L * u(), L * u())
        ok = True
        for (qx, qy, qz, qr) in out:
            d2 = 0.0
            for a, b in zip(c, (qx, qy, qz)):
                d = abs(a - b)
                d = min(d, L - d)
                d2 += d * d
            if d2 < (r + qr) ** 2:
                ok = False
                break
        if ok:
            out.append((c[0], c[1], c[2], r))
            vol += 4.0 / 3.0 * math.pi * r ** 3
            fails = 0
        else:
            fails += 1
    return out


def test_splitmix_block_matches_sequential_draws():
    g = splitmix64(12345)
    seq = np.array([g() for _ in range(1000)])
    assert np.array_equal(splitmix64_block(12345, 0, 1000), seq)
    assert np.array_equal(splitmix64_block(12345, 400, 600), seq[400:])


def test_rsa_matches_definition_with_cells():
    # 60 / (2 * 8) -> 3 cells per axis: the cell-list path
    assert rsa_spheres(60, 2, 4.0, 8.0, 0.3) == _rsa_one_at_a_time(60, 2, 4.0, 8.0, 0.3, 1_000_000)


def test_rsa_matches_definition_without_cells_and_fail_stop():
    assert rsa_spheres(40, 3, 3.0, 9.0, 0.35, 2000) == _rsa_one_at_a_time(40, 3, 3.0, 9.0, 0.35, 2000)


def test_rsa_spheres_do_not_overlap_and_reach_target():
    n = 64
    sp = rsa_spheres(n, 1, 4.0, 8.0, 0.3)
    c = np.array([s[:3] for s in sp])
    r = np.array([s[3] for s in sp])
    d = np.abs(c[:, None, :] - c[None, :, :])
    d = np.minimum(d, n - d)
    dist = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(dist, np.inf)
    assert np.all(dist >= r[:, None] + r[None, :])
    assert (4.0 / 3.0 * np.pi * r ** 3).sum() / n ** 3 >= 0.3


def test_spheres_phi0_is_periodic_union_of_profiles():
    n = (12, 14, 16)
    sp = [(1.0, 2.0, 3.0, 3.0), (9.0, 10.0, 8.0, 2.5)]
    phi0 = spheres_phi0(n, sp, 4.0)
    z, y, x = np.meshgrid(*[np.arange(k, dtype=float) for k in n], indexing="ij")
    ref = np.zeros(n)
    for (cx, cy, cz, r) in sp:
        dd = []
        for c, a, m in ((cz, z, n[0]), (cy, y, n[1]), (cx, x, n[2])):
            e = a - c
            dd.append(e - m * np.round(e / m))
        dist = np.sqrt(sum(e * e for e in dd))
        ref = np.maximum(ref, 0.5 + 0.5 * np.tanh(2.0 * (r - dist) / 4.0))
    assert np.allclose(phi0, ref, atol=1e-15)
