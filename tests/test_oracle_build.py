"""Pins of the oracle's tree build (Sec. 2.1) against the paper and plain mathematics."""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_depth.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                a, b = line.split()
                rows.append((int(a), int(b)))
    return rows


def test_depth_matches_table1():
    # Sec. 3.2.1, Table 1: N = 500000, the L column for every N_ll.
    for n_ll, L in _table1():
        assert oracle.depth(500000, n_ll) == L


def test_depth_rule_small_and_exact_boundaries():
    assert oracle.depth(1, 12) == 1          # L >= 1 always
    assert oracle.depth(11, 12) == 1
    assert oracle.depth(24, 12) == 2         # 24 / 2 = 12 is not below 12
    assert oracle.depth(23, 12) == 1
    assert oracle.depth(4096, 12) == 9
    assert oracle.depth(4194304, 12) == 19
    assert oracle.depth(100_000_000, 12) == 23


def test_i128_to_double_is_round_to_nearest_even():
    rng = random.Random(5)
    vals = [0, 1, -1, 2**53 + 1, 2**53 + 3, -(2**53 + 1), 2**100 + 2**47, 2**100 + 2**47 + 1,
            -(2**120 + 2**67), 2**126 - 1, -(2**126)]
    for _ in range(2000):
        v = rng.getrandbits(rng.randrange(1, 127))
        vals.append(v if rng.random() < 0.5 else -v)
    for _ in range(500):  # exact ties: 53 significant bits followed by a single half-ulp bit
        shift = rng.randrange(1, 70)
        v = ((rng.getrandbits(52) | (1 << 52)) << shift) | (1 << (shift - 1))
        vals.append(v if rng.random() < 0.5 else -v)
    for v in vals:
        assert oracle.i128_to_double(v) == float(v), v  # Python's int -> float is correctly rounded


@pytest.fixture(scope="module")
def small_tree():
    x, m, h = synth.make_particles("plummer", 3000, synth.seed_for(9, 1), "loguniform10")
    return x, m, h, oracle.OracleTree(x, m, h, n_ll=12)


def test_fixed_point_definition(small_tree):
    x, m, h, T = small_tree
    P = T.fixed()
    p = m[:, None] * x                                   # RN(m * x), float64
    for d in range(3):
        E = math.frexp(float(np.abs(p[:, d]).max()))[1]
        assert E == T.E[d]
        for i in range(0, len(m), 37):
            exact = round(Fraction(float(p[i, d])) * Fraction(2) ** (62 - E))   # half to even
            assert P[i, 1 + d] == exact
    Em = math.frexp(float(m.max()))[1]
    assert Em == T.Em
    for i in range(0, len(m), 37):
        assert P[i, 0] == round(Fraction(float(m[i])) * Fraction(2) ** (62 - Em))


def _i128(pair):
    lo, hi = int(pair[0]), int(pair[1])
    return (hi << 64) + (lo & ((1 << 64) - 1))


def test_sums_compose_and_com_is_exact(small_tree):
    x, m, h, T = small_tree
    nd = T.nodes()
    P = T.fixed()
    perm = T.perm()
    # root sums = sum over all particles
    for k in range(4):
        assert _i128(nd["sums"][1, k]) == int(sum(int(v) for v in P[:, k]))
    for n in range(1, 1 << T.L):
        for k in range(4):
            assert _i128(nd["sums"][n, k]) == _i128(nd["sums"][2 * n, k]) + _i128(nd["sums"][2 * n + 1, k])
    # COM = RN(RN(S) 2^(E-62) / (RN(M) 2^(Em-62))) with Python's correctly rounded int->float
    for n in range(1, 2 << T.L):
        if nd["count"][n] == 0:
            continue
        M = _i128(nd["sums"][n, 0])
        for d in range(3):
            S = _i128(nd["sums"][n, 1 + d])
            com = math.ldexp(float(S), T.E[d] - 62) / math.ldexp(float(M), T.Em - 62)
            assert com == nd["com"][n, d]
        # the cell's particle set sums to its node sums
        f, c = nd["first"][n], nd["count"][n]
        assert _i128(nd["sums"][n, 0]) == int(sum(int(v) for v in P[perm[f:f + c], 0]))


def test_every_split_is_longest_side_through_com(small_tree):
    # Sec. 2.1.3 / 2.1.4 checked by brute force on the particle sets of every cell.
    x, m, h, T = small_tree
    nd = T.nodes()
    perm = T.perm()
    for n in range(1, 1 << T.L):
        f, c = nd["first"][n], nd["count"][n]
        if c == 0:
            assert nd["count"][2 * n] == 0 and nd["count"][2 * n + 1] == 0
            continue
        pts = x[perm[f:f + c]]
        lo, hi = pts.min(0), pts.max(0)
        assert np.array_equal(lo, nd["bmin"][n]) and np.array_equal(hi, nd["bmax"][n])
        ext = hi - lo
        ax = int(np.argmax(ext))                       # first maximum = lowest axis on ties
        assert nd["axis"][n] == ax
        s = nd["split"][n]
        assert s == nd["com"][n, ax]
        fl, cl = nd["first"][2 * n], nd["count"][2 * n]
        fr, cr = nd["first"][2 * n + 1], nd["count"][2 * n + 1]
        assert fl == f and fr == f + cl and cl + cr == c
        assert np.all(x[perm[fl:fl + cl], ax] < s)
        assert np.all(x[perm[fr:fr + cr], ax] >= s)
        assert nd["H"][n] == ext.max()
        assert np.array_equal(nd["rg"][n], 0.5 * (lo + hi))


def test_labelling_identities(small_tree):
    # Sec. 2.1.5: children 2n, 2n+1; level floor(log2 n); level k spans 2^k .. 2^(k+1)-1.
    x, m, h, T = small_tree
    nd = T.nodes()
    L = T.L
    assert nd["first"].shape[0] == 2 << L              # 2^(L+1) - 1 nodes plus the unused 0
    for k in range(L + 1):
        lvl = range(1 << k, 2 << k)
        assert all(int(math.floor(math.log2(n))) == k for n in lvl)
        assert sum(nd["count"][n] for n in lvl) == T.N  # every level covers every particle once
        # 2^p - 2 descendants of a level-k cell, p = number of levels >= k
        p = L + 1 - k
        desc = sum(1 << j for j in range(1, p))
        assert desc == 2**p - 2


def test_quadrupole_eq2_equals_eq1(small_tree):
    # Eq. 2 (shift-up) reproduces Eq. 1 summed directly over all particles of the parent.
    x, m, h, T = small_tree
    nd = T.nodes()
    perm = T.perm()
    for n in range(1, 2 << T.L):
        c = nd["count"][n]
        if c == 0:
            continue
        f = nd["first"][n]
        idx = perm[f:f + c]
        d = x[idx] - nd["com"][n]
        Qf = 3 * np.einsum("k,ki,kj->ij", m[idx], d, d) - np.eye(3) * np.sum(m[idx] * np.einsum("ki,ki->k", d, d))
        q6 = np.array([Qf[0, 0], Qf[0, 1], Qf[0, 2], Qf[1, 1], Qf[1, 2], Qf[2, 2]])
        scale = np.sum(m[idx] * np.einsum("ki,ki->k", d, d)) + 1e-300
        assert np.max(np.abs(nd["Q"][n] - q6)) <= 1e-11 * scale
        assert abs(nd["Q"][n][0] + nd["Q"][n][3] + nd["Q"][n][5]) <= 1e-11 * scale   # traceless


def test_radii(small_tree):
    # Sec. 2.3.1: h_node(A) encloses every kernel of A, h_node_int(B) every particle of B.
    x, m, h, T = small_tree
    nd = T.nodes()
    perm = T.perm()
    leaf0 = 1 << T.L
    for n in range(1, 2 << T.L):
        c = nd["count"][n]
        if c == 0:
            continue
        f = nd["first"][n]
        idx = perm[f:f + c]
        dv = x[idx] - nd["rg"][n]
        dist = np.sqrt((dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1]) + dv[:, 2] * dv[:, 2])
        if n >= leaf0:
            assert nd["hint"][n] == dist.max()
            assert nd["hnode"][n] == np.max(dist + 2.0 * h[idx])
        else:
            assert nd["hint"][n] >= dist.max() * (1 - 1e-15)


def test_input_validation():
    x = np.zeros((4, 3))
    m = np.ones(4)
    h = np.ones(4)
    with pytest.raises(ValueError):
        oracle.OracleTree(np.array([[np.nan, 0, 0]] * 4), m, h)
    with pytest.raises(ValueError):
        oracle.OracleTree(x, -m, h)
    with pytest.raises(ValueError):
        oracle.OracleTree(x, m, 0 * h)
    with pytest.raises(ValueError):
        oracle.OracleTree(x[:0], m[:0], h[:0])


def test_degenerate_inputs_build():
    # single particle, two particles, all particles at one point
    for N in (1, 2, 3):
        x, m, h = synth.make_particles("cube", N, 3, "equal")
        T = oracle.OracleTree(x, m, h)
        assert T.L == 1 and T.nodes()["count"][1] == N
    x = np.ones((50, 3))
    T = oracle.OracleTree(x, np.ones(50), np.ones(50))
    nd = T.nodes()
    assert nd["count"][1] == 50 and nd["H"][1] == 0.0
    leaf0 = 1 << T.L
    assert sum(nd["count"][leaf0:]) == 50


def _route_leaves(nodes, L, x):
    """Leaf number of every position when routed from the root through the stored splits
    (x_axis < split to the left child; into the non-empty child where the other is empty, since
    such a plane separates no particles): an independent statement of the ll-cell membership."""
    n = np.ones(x.shape[0], np.int64)
    cnt = nodes["count"]
    for _ in range(L):
        ax = nodes["axis"][n]
        right = ~(x[np.arange(x.shape[0]), ax] < nodes["split"][n])
        right = np.where(cnt[2 * n] == 0, True, np.where(cnt[2 * n + 1] == 0, False, right))
        n = 2 * n + right.astype(np.int64)
    return n - (1 << L)


@pytest.mark.parametrize("sigma", [0.0, 1e-3, 3e-2])
def test_integrity_check_counts_particles_that_left_their_ll_cell(sigma):
    # Sec. 2.1.8: the update keeps the tree only if no particle crossed its ll-cell's border.  The
    # count must equal the number of particles whose routed leaf differs from their leaf.
    N = 3000
    x, m, h = synth.make_particles("plummer", N, 71, "loguniform10")
    ref = oracle.OracleTree(x, m, h)
    x2 = synth.jitter(x, sigma, 72) if sigma > 0 else x.copy()
    expect = int(np.sum(_route_leaves(ref.nodes(), ref.L, x2) != ref.leaf_of()))
    if sigma == 0.0:
        assert expect == 0
    if sigma == 3e-2:
        assert expect > 100
    before = ref.nodes()
    got = ref.update(x2, m, h)
    assert got == expect
    if got > 0:   # the tree is left as it was
        after = ref.nodes()
        assert np.array_equal(after["com"], before["com"]) and np.array_equal(after["split"], before["split"])


def test_update_inside_equals_refit_with_new_h():
    # every particle still inside: the update is a refit with the new smoothing lengths (radii
    # from the new h), the splits unchanged
    N = 3000
    x, m, h = synth.make_particles("sphere", N, 73, "loguniform10")
    x2 = synth.jitter(x, 1e-9, 74)
    m2 = m * (1.0 + 0.01 * np.random.default_rng(75).random(N))
    h2 = h * (1.0 + 0.05 * np.random.default_rng(76).random(N))
    a = oracle.OracleTree(x, m, h)
    assert a.update(x2, m2, h2) == 0
    b = oracle.OracleTree(x, m, h2)      # same partition (built at x), radii from h2
    b.refit(x2, m2)
    na, nb = a.nodes(), b.nodes()
    for k in ("split", "axis", "com", "bmin", "bmax", "rg", "hint", "hnode", "Q", "mass"):
        assert np.array_equal(na[k], nb[k]), k


def test_unit_weight_splits_are_centres_of_number():
    # the centre-of-number variant (Sec. 2.1.3): with unit weights every split is the cell's mean
    # coordinate along the cut axis (exact rational mean, within one ulp of the fixed-point grid)
    N = 2000
    x, _, h = synth.make_particles("plummer", N, 77, "equal")
    ref = oracle.OracleTree(x, np.ones(N), h)
    nd, perm = ref.nodes(), ref.perm()
    for c in range(1, 1 << ref.L):
        f, n = nd["first"][c], nd["count"][c]
        if n == 0:
            continue
        ax = nd["axis"][c]
        vals = x[perm[f:f + n], ax]
        exact = float(sum(Fraction(v) for v in vals) / n)
        assert abs(nd["split"][c] - exact) <= 2 * np.spacing(abs(exact)), c


def _check_median_cells(x, T, distinct):
    # Sec. 2.1.3, the median position split: every cell is cut along its longest side at the
    # order statistic of rank floor(n/2) of its coordinates, i.e. #(x < s) <= n // 2 < #(x <= s),
    # and s is a coordinate of the cell (the smallest of the right child).  With distinct
    # coordinates the daughters hold exactly floor(n/2) and ceil(n/2) particles.
    nd, perm = T.nodes(), T.perm()
    for n in range(1, 1 << T.L):
        f, c = nd["first"][n], nd["count"][n]
        if c == 0:
            continue
        pts = x[perm[f:f + c]]
        ax = int(np.argmax(pts.max(0) - pts.min(0)))
        assert nd["axis"][n] == ax
        s = nd["split"][n]
        v = pts[:, ax]
        below, upto = int(np.sum(v < s)), int(np.sum(v <= s))
        assert below <= c // 2 < upto, n
        cl, cr = nd["count"][2 * n], nd["count"][2 * n + 1]
        assert cl == below and cl + cr == c
        assert np.all(x[perm[f:f + cl], ax] < s)
        right = x[perm[f + cl:f + c], ax]
        assert np.all(right >= s) and right.min() == s
        if distinct:
            assert cl == c // 2 and cr == c - c // 2


@pytest.mark.parametrize("kind,N", [("plummer", 3000), ("sphere", 2049), ("cube", 13)])
def test_median_split_is_the_order_statistic(kind, N):
    x, m, h = synth.make_particles(kind, N, 78, "loguniform10")
    assert all(len(np.unique(x[:, d])) == N for d in range(3))
    T = oracle.OracleTree(x, m, h, split="median")
    _check_median_cells(x, T, distinct=True)


def test_median_split_with_tied_coordinates():
    # a lattice: many particles share each coordinate; the cut still sits at the order statistic
    g = np.arange(12, dtype=np.float64)
    x = np.stack(np.meshgrid(g, g, g[:9], indexing="ij"), -1).reshape(-1, 3)
    N = x.shape[0]
    T = oracle.OracleTree(x, np.ones(N), np.full(N, 0.7), split="median")
    _check_median_cells(x, T, distinct=False)


def test_median_split_balances_every_leaf():
    # N = 12 * 2^8 particles at N_ll = 12 give L = 9 and 512 ll-cells of exactly 6 particles each
    N = 3072
    x, m, h = synth.make_particles("plummer", N, 79, "loguniform10")
    T = oracle.OracleTree(x, m, h, split="median")
    assert T.L == 9
    nd = T.nodes()
    assert np.all(nd["count"][1 << 9:] == 6)
    # the centre-of-mass split of the same set is not balanced
    assert not np.all(oracle.OracleTree(x, m, h).nodes()["count"][1 << 9:] == 6)


def test_median_split_tree_update_and_refit():
    # the integrity check and the refit use the stored planes, whatever chose them
    N = 3000
    x, m, h = synth.make_particles("sphere", N, 80, "loguniform10")
    a = oracle.OracleTree(x, m, h, split="median")
    before = a.nodes()
    assert a.update(x, m, h) == 0
    after = a.nodes()
    for k in ("split", "axis", "count", "com", "Q"):
        assert np.array_equal(before[k], after[k]), k
    x2 = synth.jitter(x, 3e-2, 81)
    expect = int(np.sum(_route_leaves(a.nodes(), a.L, x2) != a.leaf_of()))
    assert expect > 0 and a.update(x2, m, h) == expect


def test_median_split_tree_gives_direct_sum_and_brute_neighbours():
    # any partition must reproduce the direct sum at theta = 0 (Sec. 2.4.1) and the brute-force
    # neighbour lists (Sec. 2.3): the median tree's moments, radii and lists cover every particle
    N = 1500
    x, m, h = synth.make_particles("plummer", N, 82, "loguniform10")
    T = oracle.OracleTree(x, m, h, split="median")
    T.walk(0.0)
    acc, pot = T.gravity()
    ad, pd = oracle.direct(x, m, h)
    assert np.max(np.linalg.norm(acc - ad, axis=1) / np.linalg.norm(ad, axis=1)) < 1e-12
    assert np.abs(pot - pd).max() < 1e-12 * np.abs(pd).max()
    to, ti = T.neighbours()
    bo, bi = oracle.brute_neighbours(x, h)
    assert np.array_equal(to, bo) and np.array_equal(ti, bi)


def _fixed_exact(x, m):
    """Fixed-point integers of the exact centre of mass, restated from the definition (p = RN(m x),
    E with max|p| < 2^E, P = RN(p 2^(62 - E)), half to even) with Python's exact arithmetic."""
    p = m[:, None] * x
    E = [math.frexp(float(np.abs(p[:, d]).max()))[1] for d in range(3)]
    Em = math.frexp(float(m.max()))[1]
    P = np.empty((len(m), 4), dtype=object)
    for i in range(len(m)):
        P[i, 0] = round(Fraction(float(m[i])) * Fraction(2) ** (62 - Em))
        for d in range(3):
            P[i, 1 + d] = round(Fraction(float(p[i, d])) * Fraction(2) ** (62 - E[d]))
    return P, E, Em


def _check_nodes_against_particles(x, m, h, T):
    """Every node of T against brute force over its own particle set (positions x, masses m and
    smoothing lengths h in original order): exact integer sums, mass and centre of mass, the tight
    box, r_g and H (Sec. 2.1.3, Eq. 4), the quadrupole of Eq. 1 summed directly, and the radii of
    Sec. 2.3.1 (exact for ll-cells, enclosing for internal nodes)."""
    nd, perm = T.nodes(), T.perm()
    P, E, Em = _fixed_exact(x, m)
    leaf0 = 1 << T.L
    for n in range(1, 2 << T.L):
        f, c = nd["first"][n], nd["count"][n]
        if c == 0:
            continue
        idx = perm[f:f + c]
        Ms = int(sum(P[idx, 0]))
        assert _i128(nd["sums"][n, 0]) == Ms, n
        M = math.ldexp(float(Ms), Em - 62)
        assert nd["mass"][n] == M, n
        for d in range(3):
            S = int(sum(P[idx, 1 + d]))
            assert _i128(nd["sums"][n, 1 + d]) == S, n
            assert nd["com"][n, d] == math.ldexp(float(S), E[d] - 62) / M, n
        pts = x[idx]
        lo, hi = pts.min(0), pts.max(0)
        assert np.array_equal(nd["bmin"][n], lo) and np.array_equal(nd["bmax"][n], hi), n
        assert np.array_equal(nd["rg"][n], 0.5 * (lo + hi)), n
        assert nd["H"][n] == (hi - lo).max(), n
        d = pts - nd["com"][n]
        d2 = np.einsum("ki,ki->k", d, d)
        Qf = 3 * np.einsum("k,ki,kj->ij", m[idx], d, d) - np.eye(3) * np.sum(m[idx] * d2)
        q6 = np.array([Qf[0, 0], Qf[0, 1], Qf[0, 2], Qf[1, 1], Qf[1, 2], Qf[2, 2]])
        assert np.max(np.abs(nd["Q"][n] - q6)) <= 1e-11 * (np.sum(m[idx] * d2) + 1e-300), n
        dv = pts - nd["rg"][n]
        dist = np.sqrt((dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1]) + dv[:, 2] * dv[:, 2])
        if n >= leaf0:
            assert nd["hint"][n] == dist.max(), n
            assert nd["hnode"][n] == np.max(dist + 2.0 * h[idx]), n
        else:
            assert nd["hint"][n] >= dist.max() * (1 - 1e-15), n


def test_node_check_holds_on_a_fresh_build(small_tree):
    x, m, h, T = small_tree
    _check_nodes_against_particles(x, m, h, T)


def test_refit_recomputes_every_node_from_the_moved_particles():
    # Sec. 2.1.8 refit with the structure frozen: positions moved far enough that every box,
    # centre, radius and moment changes, masses changed; each node must equal brute force over
    # its (unchanged) particle set at the new positions and masses, as on a fresh build
    N = 2500
    x, m, h = synth.make_particles("plummer", N, 83, "loguniform10")
    T = oracle.OracleTree(x, m, h)
    before = T.nodes()
    x2 = synth.jitter(x, 1e-3, 84)
    m2 = m * (1.0 + 0.5 * np.random.default_rng(85).random(N))
    T.refit(x2, m2)
    after = T.nodes()
    for k in ("bmin", "bmax", "rg", "H", "hint", "hnode", "com", "Q", "mass"):
        assert not np.array_equal(before[k], after[k]), k   # a stale field would pass unnoticed
    assert np.array_equal(before["split"], after["split"]) and np.array_equal(before["count"], after["count"])
    _check_nodes_against_particles(x2, m2, h, T)


def test_update_inside_recomputes_every_node_and_walks_to_exact_results():
    # Sec. 2.1.8 update with every particle still inside its ll-cell: new positions, masses and
    # smoothing lengths; every node equals brute force at the new state, and the tree walked again
    # gives the brute-force neighbour lists (Sec. 2.3) and, at theta = 0, the direct sum (Sec. 2.4.1)
    N = 2500
    x, m, h = synth.make_particles("sphere", N, 86, "loguniform10")
    T = oracle.OracleTree(x, m, h)
    x2 = synth.jitter(x, 1e-9, 87)
    m2 = m * (1.0 + 0.3 * np.random.default_rng(88).random(N))
    h2 = h * (1.0 + 0.2 * np.random.default_rng(89).random(N))
    before = T.nodes()
    assert T.update(x2, m2, h2) == 0
    after = T.nodes()
    for k in ("bmin", "bmax", "hint", "hnode", "com", "Q"):
        assert not np.array_equal(before[k], after[k]), k
    _check_nodes_against_particles(x2, m2, h2, T)
    T.walk(0.0)
    to, ti = T.neighbours()
    bo, bi = oracle.brute_neighbours(x2, h2)
    assert np.array_equal(to, bo) and np.array_equal(ti, bi)
    acc, pot = T.gravity()
    ad, pd = oracle.direct(x2, m2, h2)
    assert np.max(np.linalg.norm(acc - ad, axis=1) / np.linalg.norm(ad, axis=1)) < 1e-12
    assert np.abs(pot - pd).max() < 1e-12 * np.abs(pd).max()
    # and at theta = 0.7 the neighbour lists still equal brute force
    T.walk(0.7)
    to, ti = T.neighbours()
    assert np.array_equal(to, bo) and np.array_equal(ti, bi)
