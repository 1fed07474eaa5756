"""Pins of the oracle's near field (Sec. 2.4.3), far field (Sec. 2.4.2) and whole method."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------- softened kernel
def _cubic_spline_W(r, h):
    # the standard cubic spline of Monaghan & Lattanzio (1985), support 2h, normalised in 3-D
    q = r / h
    if q < 1:
        w = 1 - 1.5 * q * q + 0.75 * q ** 3
    elif q < 2:
        w = 0.25 * (2 - q) ** 3
    else:
        w = 0.0
    return w / (math.pi * h ** 3)


def test_S_is_the_enclosed_kernel_mass_over_r2():
    # Sec. 2.4.3: F = -m_a m_b eta / r^2 e, eta = 4 pi int_0^r r'^2 W dr', so S = eta / r^2.
    from scipy.integrate import quad
    h = 0.37
    for q in [0.05, 0.3, 0.7, 0.99, 1.0, 1.01, 1.5, 1.9, 2.0, 2.5, 4.0]:
        r = q * h
        pts = [h, 2 * h] if r > 2 * h else ([h] if r > h else None)
        eta, _ = quad(lambda s: 4 * math.pi * s * s * _cubic_spline_W(s, h), 0.0, r, points=pts,
                      epsabs=1e-14, epsrel=1e-13, limit=200)
        assert oracle.kernel_S(r, h) == pytest.approx(eta / r ** 2, rel=1e-10)


def test_S_and_phi_are_continuous_and_consistent():
    h = 0.8
    eps = 1e-12
    for q, S_exp, phi_exp in [(1.0, 19 / 30, -28 / 30), (2.0, 0.25, -0.5)]:
        r = q * h
        for rr in (r * (1 - eps), r, r * (1 + eps)):
            assert oracle.kernel_S(rr, h) * h * h == pytest.approx(S_exp, rel=1e-9)
            assert oracle.kernel_phi(rr, h) * h == pytest.approx(phi_exp, rel=1e-9)
    for q in [0.2, 0.6, 0.95, 1.2, 1.7, 1.99, 2.4, 7.0]:
        r = q * h
        d = 1e-6 * h
        dphi = (oracle.kernel_phi(r + d, h) - oracle.kernel_phi(r - d, h)) / (2 * d)
        assert dphi == pytest.approx(oracle.kernel_S(r, h), rel=1e-7)        # phi' = S
        assert oracle.kernel_S_over_r(r, h) * r == pytest.approx(oracle.kernel_S(r, h), rel=1e-13)
        dsr = (oracle.kernel_S_over_r(r + d, h) - oracle.kernel_S_over_r(r - d, h)) / (2 * d)
        assert oracle.kernel_dSr_over_r(r, h) * r == pytest.approx(dsr, rel=1e-6)
    # Newtonian beyond the support, and a finite force law at r -> 0
    assert oracle.kernel_S(3.0, 1.0) == 1 / 9.0
    assert oracle.kernel_phi(3.0, 1.0) == -1 / 3.0
    assert oracle.kernel_S_over_r(0.0, 1.0) == pytest.approx(4 / 3)


# ---------------------------------------------------------------------------- far field
def test_inverse_r_derivatives_against_finite_differences_and_harmonicity():
    x = np.array([0.7, -1.1, 0.45])
    rng = np.random.default_rng(3)
    assert oracle.dinv_r([], x) == pytest.approx(1 / np.linalg.norm(x), rel=1e-15)
    assert [oracle.dinv_r([i], x) for i in range(3)] == pytest.approx(list(-x / np.linalg.norm(x) ** 3), rel=1e-14)
    for n in range(1, 7):
        for _ in range(6):
            idx = list(rng.integers(0, 3, n))
            last = idx[-1]
            d = 1e-5
            e = np.zeros(3)
            e[last] = d
            fd = (oracle.dinv_r(idx[:-1], x + e) - oracle.dinv_r(idx[:-1], x - e)) / (2 * d)
            assert oracle.dinv_r(idx, x) == pytest.approx(fd, rel=2e-7, abs=1e-9)
            # symmetric in its indices
            assert oracle.dinv_r(idx[::-1], x) == pytest.approx(oracle.dinv_r(idx, x), rel=1e-13)
        if n >= 2:  # 1/r is harmonic: every trace vanishes
            base = list(rng.integers(0, 3, n - 2))
            tr = sum(oracle.dinv_r(base + [i, i], x) for i in range(3))
            assert abs(tr) < 1e-11 * max(1.0, abs(oracle.dinv_r(base + [0, 0], x)))


def _cluster(seed, K=20, H=1.0):
    rng = np.random.default_rng(seed)
    xs = (rng.random((K, 3)) - 0.5) * H
    ms = rng.random(K) + 0.5
    M = ms.sum()
    com = (ms[:, None] * xs).sum(0) / M
    d = xs - com
    Qf = 3 * np.einsum("k,ki,kj->ij", ms, d, d) - np.eye(3) * np.sum(ms * (d * d).sum(1))
    return xs, ms, M, com, np.array([Qf[0, 0], Qf[0, 1], Qf[0, 2], Qf[1, 1], Qf[1, 2], Qf[2, 2]])


def test_quadrupole_expansion_error_falls_as_third_power():
    # Eq. 5: monopole + quadrupole about the COM; the dipole vanishes, so the error is O((H/R)^3).
    xs, ms, M, com, q6 = _cluster(1)
    errs = []
    for R in [4.0, 8.0, 16.0, 32.0]:
        y = com + np.array([R, 0.3 * R, -0.2 * R])
        phi, a = oracle.taylor_eval(oracle.far_coeffs(y - com, M, q6), np.zeros(3))
        rv = y - xs
        r = np.linalg.norm(rv, axis=1)
        ad = -(ms[:, None] * rv / r[:, None] ** 3).sum(0)
        phid = -(ms / r).sum()
        errs.append((abs(phi - phid) / abs(phid), np.linalg.norm(a - ad) / np.linalg.norm(ad)))
    for (p0, a0), (p1, a1) in zip(errs, errs[1:]):
        assert 6.0 < p0 / p1 < 10.5 and 6.0 < a0 / a1 < 10.5


def test_sink_taylor_expansion_orders():
    # Eq. 6: the third-order potential polynomial gives forces with O(|dr|^3) error.
    xs, ms, M, com, q6 = _cluster(2)
    y0 = com + np.array([10.0, 3.0, -2.0])
    C = oracle.far_coeffs(y0 - com, M, q6)
    prev = None
    for s in [1.0, 0.5, 0.25, 0.125]:
        dd = s * np.array([0.3, -0.2, 0.25])
        phi, a = oracle.taylor_eval(C, dd)
        phie, ae = oracle.taylor_eval(oracle.far_coeffs(y0 + dd - com, M, q6), np.zeros(3))
        cur = (abs(phi - phie), np.linalg.norm(a - ae))
        if prev:
            assert 12.0 < prev[0] / cur[0] < 20.0   # potential: 4th order
            assert 6.0 < prev[1] / cur[1] < 10.0    # force: 3rd order
        prev = cur
    # at dr = 0 the force is -grad Phi of Eq. 5 exactly
    phi0, a0 = oracle.taylor_eval(C, np.zeros(3))
    R = y0 - com
    r = np.linalg.norm(R)
    Qf = np.array([[q6[0], q6[1], q6[2]], [q6[1], q6[3], q6[4]], [q6[2], q6[4], q6[5]]])
    assert phi0 == pytest.approx(-M / r - 0.5 * R @ Qf @ R / r ** 5, rel=1e-13)


# ---------------------------------------------------------------------------- whole method
@pytest.fixture(scope="module")
def plummer4096():
    x, m, h = synth.make_particles("plummer", 4096, synth.seed_for(1), "equal")
    return x, m, h, oracle.OracleTree(x, m, h)


def test_theta_zero_is_direct_summation(plummer4096):
    # Sec. 2.4.1: theta = 0 reproduces direct summation.
    x, m, h, T = plummer4096
    T.walk(0.0)
    ls = T.lists()
    nd = T.nodes()
    leaf0 = 1 << T.L
    nonempty = np.flatnonzero(nd["count"][leaf0:] > 0) + leaf0
    assert ls["far_ids"].size == 0
    for j in range(0, T.nleaves, 7):
        if nd["count"][leaf0 + j] == 0:
            continue
        ids = np.sort(ls["near_ids"][ls["near_off"][j]:ls["near_off"][j + 1]])
        assert np.array_equal(ids, nonempty)
    acc, pot = T.gravity()
    ad, pd = oracle.direct(x, m, h)
    rel = np.linalg.norm(acc - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert rel.max() < 1e-12
    assert np.abs(pot - pd).max() < 1e-12 * np.abs(pd).max()


def test_walk_covers_every_particle_exactly_once(plummer4096):
    # For each sink, far nodes and near ll-cells partition the whole particle set; reachable
    # cells are never accepted by the MAC; the sink is in its own near and candidate lists.
    x, m, h, T = plummer4096
    T.walk(0.7)
    ls = T.lists()
    nd = T.nodes()
    leaf0 = 1 << T.L
    for j in range(T.nleaves):
        if nd["count"][leaf0 + j] == 0:
            assert ls["near_off"][j + 1] == ls["near_off"][j]
            continue
        cover = np.zeros(T.N, np.int64)
        near = ls["near_ids"][ls["near_off"][j]:ls["near_off"][j + 1]]
        reach = ls["near_reach"][ls["near_off"][j]:ls["near_off"][j + 1]]
        far = ls["far_ids"][ls["far_off"][j]:ls["far_off"][j + 1]]
        for n in list(near) + list(far):
            cover[nd["first"][n]:nd["first"][n] + nd["count"][n]] += 1
        assert np.all(cover == 1)
        assert (leaf0 + j) in set(near[reach == 1])
        A = leaf0 + j
        for n in far:
            d2 = np.sum((nd["rg"][A] - nd["rg"][n]) ** 2)
            assert d2 >= (nd["hnode"][A] + nd["hint"][n]) ** 2 * (1 - 1e-12)
            R = np.linalg.norm(nd["com"][A] - nd["com"][n])
            assert nd["H"][n] < 0.7 * R * (1 + 1e-12)


def test_mac_only_walk(plummer4096):
    # The Sec. 2.5 variant (no reachability override): theta = 0 is still direct summation; for
    # every sink the far nodes and near cells cover each particle exactly once, every far node
    # passes the MAC, the near cells carry no candidate flag, and they are a subset of the
    # conservative walk's near cells (a leaf whose ancestors all fail the MAC is visited and kept
    # near by both walks).
    x, m, h, T = plummer4096
    T.walk(0.0, mac_only=True)
    acc, _ = T.gravity()
    ad, _ = oracle.direct(x, m, h)
    assert (np.linalg.norm(acc - ad, axis=1) / np.linalg.norm(ad, axis=1)).max() < 1e-12
    T.walk(0.7)
    std = T.lists()
    T.walk(0.7, mac_only=True)
    mac = T.lists()
    nd = T.nodes()
    leaf0 = 1 << T.L
    assert mac["near_ids"].size < std["near_ids"].size
    assert not mac["near_reach"].any()
    for j in range(T.nleaves):
        if nd["count"][leaf0 + j] == 0:
            continue
        near = mac["near_ids"][mac["near_off"][j]:mac["near_off"][j + 1]]
        far = mac["far_ids"][mac["far_off"][j]:mac["far_off"][j + 1]]
        cover = np.zeros(T.N, np.int64)
        for n in list(near) + list(far):
            cover[nd["first"][n]:nd["first"][n] + nd["count"][n]] += 1
        assert np.all(cover == 1)
        A = leaf0 + j
        for n in far:
            R = np.linalg.norm(nd["com"][A] - nd["com"][n])
            assert nd["H"][n] < 0.7 * R * (1 + 1e-12)
        assert set(near.tolist()) <= set(std["near_ids"][std["near_off"][j]:std["near_off"][j + 1]].tolist())


def test_hand_built_two_clusters():
    # two tight clusters 100 apart, 8 particles each: N = 16 gives L = 1 (16/2 < 12); the root
    # splits on x through the COM; each leaf is near to itself and far to the other.
    rng = np.random.default_rng(0)
    a = rng.random((8, 3)) * 0.5
    b = rng.random((8, 3)) * 0.5 + np.array([100.0, 0, 0])
    x = np.concatenate([a, b])
    m = np.ones(16)
    h = np.full(16, 0.01)
    T = oracle.OracleTree(x, m, h)
    assert T.L == 1
    nd = T.nodes()
    assert nd["axis"][1] == 0 and 0.5 < nd["split"][1] < 100
    assert set(T.perm()[:8]) == set(range(8))
    T.walk(0.5)
    ls = T.lists()
    assert list(ls["near_ids"][0:1]) == [2] and list(ls["near_reach"][0:1]) == [1]
    assert list(ls["far_ids"][ls["far_off"][0]:ls["far_off"][1]]) == [3]
    assert list(ls["far_ids"][ls["far_off"][1]:ls["far_off"][2]]) == [2]
    # theta below H/R: no acceptance, the other cell becomes a (non-reachable) near cell
    T.walk(0.001)
    ls = T.lists()
    assert ls["far_ids"].size == 0
    assert list(ls["near_reach"][ls["near_off"][0]:ls["near_off"][1]]) == [1, 0]


@pytest.mark.parametrize("kind,N,mass", [("plummer", 2500, "loguniform10"), ("cube", 3000, "equal"),
                                         ("sphere", 2000, "loguniform10")])
def test_neighbours_equal_brute_force(kind, N, mass):
    # Sec. 2.3: the culled candidate lists are exactly the particles within 2 h_a.
    x, m, h = synth.make_particles(kind, N, synth.seed_for(7, N), mass)
    T = oracle.OracleTree(x, m, h)
    T.walk(0.5)
    off, idx = T.neighbours()
    bo, bi = oracle.brute_neighbours(x, h)
    assert np.array_equal(off, bo) and np.array_equal(idx, bi)


def test_plummer_analytic_acceleration_and_potential():
    # Plummer sphere (M = 1, a = 1, truncated at r_c = 38.7).  For a spherically symmetric
    # distribution the shell theorem gives a(r) = -M(<r) / r^2 and
    # Phi(r) = -M(<r) / r - sum_{r_b > r} m_b / r_b.  Evaluated with the realised radii this
    # removes the coherent Poisson noise of the enclosed mass; only angular noise remains.
    # The analytic profile M(<r) = r^3 / (r^2 + 1)^(3/2) / f is checked against the realised
    # one at the same time.
    N = 16384
    x, m, h = synth.make_particles("plummer", N, synth.seed_for(1, 5), "equal")
    h = 0.1 * h   # softening well below the radii compared, so the point-mass law applies
    T = oracle.OracleTree(x, m, h)
    T.walk(0.5)
    acc, pot = T.gravity()
    r = np.linalg.norm(x, axis=1)
    order = np.argsort(r)
    Menc = np.empty(N)
    Menc[order] = np.cumsum(m[order]) - m[order]                     # mass strictly inside r_i
    outer = np.empty(N)
    inv = (m / r)[order]
    outer[order] = np.cumsum(inv[::-1])[::-1] - inv                   # sum over r_b > r_i
    a_sh = -Menc / r ** 2
    phi_sh = -Menc / r - outer
    f = synth.PLUMMER_XMAX
    M_an = r ** 3 / (r * r + 1) ** 1.5 / f
    assert np.max(np.abs(Menc - M_an)) < 4.0 / math.sqrt(N)           # Kolmogorov-Smirnov scale
    ar = np.einsum("ij,ij->i", acc, x) / r
    edges = [0.3, 0.5, 0.8, 1.2, 2.0, 3.5, 6.0, 12.0]
    for lo, hi in zip(edges, edges[1:]):
        sel = (r >= lo) & (r < hi)
        n = sel.sum()
        ratio = ar[sel] / a_sh[sel]
        assert abs(ratio.mean() - 1) < 4 * ratio.std() / math.sqrt(n) + 2e-3
        pr = pot[sel] / phi_sh[sel]
        assert abs(pr.mean() - 1) < 4 * pr.std() / math.sqrt(n) + 2e-3


# ------------------------------------------------------------------------- SPH density (next-4)
def test_kernel_W_is_the_normalised_cubic_spline():
    from scipy.integrate import quad
    for h in (0.3, 1.0, 2.5):
        for q in (0.0, 0.2, 0.99, 1.0, 1.5, 1.999, 2.0, 3.0):
            assert oracle.kernel_W(q * h, h) == pytest.approx(_cubic_spline_W(q * h, h), rel=1e-14, abs=0.0)
        mass, _ = quad(lambda r: 4 * math.pi * r * r * oracle.kernel_W(r, h), 0.0, 2 * h, points=[h],
                       epsabs=1e-14, epsrel=1e-13)
        assert mass == pytest.approx(1.0, rel=1e-12)


def test_density_over_neighbour_rows_equals_brute_force():
    # rho_a = m_a W(0, h_a) + sum over b != a with r_ab < 2 h_a of m_b W(r_ab, h_a): the oracle's
    # sum over its neighbour CSR against an all-pairs numpy sum
    N = 2000
    x, m, h = synth.make_particles("plummer", N, 91, "loguniform10")
    ref = oracle.OracleTree(x, m, h)
    ref.walk(0.6)
    off, idx = ref.neighbours()
    rho = oracle.density(x, m, h, off, idx)
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    q = d / h[:, None]
    w = np.where(q < 1, 1 - 1.5 * q ** 2 + 0.75 * q ** 3, np.where(q < 2, 0.25 * (2 - q) ** 3, 0.0))
    w /= np.pi * h[:, None] ** 3
    brute = (w * m[None, :]).sum(1)      # includes b = a, the self term m_a W(0, h_a)
    assert np.allclose(rho, brute, rtol=1e-12, atol=0)


def test_density_of_a_uniform_sphere_is_its_mean_density():
    # interior particles of a uniform (uncorrelated) unit sphere of total mass M: the neighbours'
    # part of the sum has expectation (M / (4/3 pi)) times the kernel's integral, 1; the self
    # term m_a W(0, h_a) comes on top (about a fifth of the mean with ~50 neighbours)
    N = 20000
    x, m, h = synth.make_particles("sphere", N, 92, "equal")
    ref = oracle.OracleTree(x, m, h)
    ref.walk(0.7)
    off, idx = ref.neighbours()
    rho = oracle.density(x, m, h, off, idx)
    inner = np.linalg.norm(x, axis=1) < 0.6
    self_term = np.array([m[a] * oracle.kernel_W(0.0, h[a]) for a in range(N)])
    mean = m.sum() / (4.0 / 3.0 * np.pi)
    assert abs(np.mean((rho - self_term)[inner]) / mean - 1.0) < 0.02


def test_median_split_error_tail_does_not_depend_on_theta():
    # Eq. 4 bounds the size of the source cell (H_B < theta R), not the extent of the sink cell about
    # which the field is expanded (Eq. 6).  The median position split makes long, thin sink cells in
    # the sparse outskirts of a Plummer sphere, whose particles sit far from the cell's centre of
    # mass: their third-order Taylor error is the same at any theta, while at theta = 0 (every cell
    # opened) the tree is exact.  The centre-of-mass split of the same set errs less.
    N = 12000
    x, m, h = synth.make_particles("plummer", N, synth.seed_for(9, 7), "loguniform10")
    tg = np.sort(np.random.default_rng(3).choice(N, 600, replace=False))
    ad, _ = oracle.direct(x, m, h, tg)

    def rms(T, th):
        T.walk(th)
        a, _ = T.gravity()
        e = np.linalg.norm(a[tg] - ad, axis=1) / np.linalg.norm(ad, axis=1)
        return float(np.sqrt(np.mean(e * e)))

    med = oracle.OracleTree(x, m, h, split="median")
    r0, r3, r7 = rms(med, 0.0), rms(med, 0.3), rms(med, 0.7)
    assert r0 < 1e-12
    assert r3 > 1e-3 and abs(r7 - r3) < 0.05 * r3, (r3, r7)
    assert rms(oracle.OracleTree(x, m, h), 0.7) < r7


def test_mac_cell_size_readings():
    # Eq. 4's H_B = MAX(S_i,B) read from the tight box of the cell's particles (the repository's
    # reading) and from the cell's bisection box (the root's tight box cut by every ancestor's
    # split plane; Sec. 2.1.5 keeps a corner and a size per node).  The bisection box is never
    # smaller, so it opens more cells: longer near lists always, and on a uniform sphere a clearly
    # smaller error against the direct sum; on a Plummer sphere the error barely moves while the
    # near lists grow several-fold.
    N = 20000
    out = {}
    for kind in ("sphere", "plummer"):
        x, m, h = synth.make_particles(kind, N, synth.seed_for(9, 2), "equal")
        tg = np.sort(np.random.default_rng(4).choice(N, 1500, replace=False))
        ad, _ = oracle.direct(x, m, h, tg)
        for box in ("tight", "bisection"):
            t = oracle.OracleTree(x, m, h)
            t.walk(0.7, mac_box=box)
            a, _ = t.gravity()
            e = np.linalg.norm(a[tg] - ad, axis=1) / np.linalg.norm(ad, axis=1)
            out[kind, box] = (float(e.mean()), float(np.mean(e < 2e-3)), len(t.lists()["near_ids"]))
    print({f"{k[0]}/{k[1]}": v for k, v in out.items()})
    # N = 20000: near entries x1.45 (sphere) and x2.9 (Plummer); mean error x0.70 and x0.99
    assert out["sphere", "bisection"][2] > 1.3 * out["sphere", "tight"][2]
    assert out["sphere", "bisection"][0] < 0.85 * out["sphere", "tight"][0]
    assert out["plummer", "bisection"][2] > 2.5 * out["plummer", "tight"][2]
    assert abs(out["plummer", "bisection"][0] - out["plummer", "tight"][0]) < 0.2 * out["plummer", "tight"][0]
