"""Pins of the CPU oracle to facts the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a
closed form, a library routine, an identity, brute force, or a value printed
in the paper (Mukherjee et al. 2021).
"""
import math
import os

import numpy as np
import pytest
from scipy.special import lpmv

import ics
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def idx(n, m):
    return n * (n + 1) // 2 + m


def full(a, n, m):
    """X_n^m for m < 0 from the m >= 0 storage: X^{-m} = (-1)^m conj(X^m)."""
    if m >= 0:
        return a[idx(n, m)]
    return (-1) ** (-m) * np.conj(a[idx(n, -m)])


# --------------------------------------------------------------- harmonics

@pytest.mark.parametrize("trial", range(6))
def test_harmonics_match_legendre_closed_form(trial):
    """Sec. 2.2 (Dehnen 2014 normalisation): Upsilon = r^n P_n^m e^{im phi}/(n+m)!,
    Theta = (n-m)! P_n^m e^{im phi}/r^{n+1}, P without the Condon-Shortley
    phase; scipy's lpmv includes it, hence the (-1)^m."""
    p = 16
    x, y, z = RNG.normal(size=3) * RNG.uniform(0.3, 3.0)
    r = math.sqrt(x * x + y * y + z * z)
    ct, ph = z / r, math.atan2(y, x)
    U = oracle.regular(p, x, y, z)
    T = oracle.irregular(p, x, y, z)
    for n in range(p + 1):
        for m in range(n + 1):
            pbar = (-1) ** m * lpmv(m, n, ct)
            e = np.exp(1j * m * ph)
            u_ref = r ** n * pbar * e / math.factorial(n + m)
            t_ref = math.factorial(n - m) * pbar * e / r ** (n + 1)
            assert abs(U[idx(n, m)] - u_ref) <= 1e-12 * max(1e-300, abs(u_ref)) + 1e-14 * r ** n / math.factorial(n + m)
            assert abs(T[idx(n, m)] - t_ref) <= 1e-12 * abs(t_ref) + 1e-13 * math.factorial(n - m) / r ** (n + 1)


def test_harmonics_match_paper_p2_list():
    """The explicit p = 2 list printed in Sec. 2.2: each regular harmonic is
    one real constant times (printed re + i printed im)."""
    rows = []
    with open(os.path.join(GOLDEN, "harmonics_p2.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            n, m, re, im = line.split()
            rows.append((int(n), int(m), re, im))
    assert len(rows) == 6  # the 9 printed functions: 1 + 3 + 5 real parts
    pts = RNG.normal(size=(20, 3))
    for n, m, re, im in rows:
        consts = []
        for x, y, z in pts:
            r = math.sqrt(x * x + y * y + z * z)
            env = {"x": x, "y": y, "z": z, "r": r}
            val = eval(re, {}, env) + (1j * eval(im, {}, env) if im != "-" else 0.0)
            u = oracle.regular(2, x, y, z)[idx(n, m)]
            consts.append(u / val)
        consts = np.array(consts)
        assert np.allclose(consts.imag, 0.0, atol=1e-12)
        assert np.allclose(consts.real, consts.real[0], rtol=1e-12)
        assert consts.real[0] != 0.0


@pytest.mark.parametrize("p", [2, 5, 10, 20])
def test_addition_theorem(p):
    """1/|x - y| = sum_{n<=p} sum_m conj(Upsilon_n^m(y)) Theta_n^m(x) up to
    the truncation bound (|y|/|x|)^{p+1} / (|x| - |y|)."""
    for _ in range(20):
        x = RNG.normal(size=3)
        x *= 2.0 / np.linalg.norm(x)
        y = RNG.normal(size=3)
        y *= RNG.uniform(0.1, 1.2) / np.linalg.norm(y)
        U = oracle.regular(p, *y)
        T = oracle.irregular(p, *x)
        s = sum((np.conj(full(U, n, m)) * full(T, n, m)).real for n in range(p + 1) for m in range(-n, n + 1))
        exact = 1.0 / np.linalg.norm(x - y)
        rx, ry = np.linalg.norm(x), np.linalg.norm(y)
        bound = (ry / rx) ** (p + 1) / (rx - ry)
        assert abs(s - exact) <= bound + 1e-14


# ------------------------------------------------------------- translations

def _cluster(n, center, radius, seed):
    g = np.random.default_rng(seed)
    d = g.normal(size=(n, 3))
    d *= (radius * g.uniform(0, 1, n) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    return center + d, g.uniform(0.5, 1.5, n)


def test_m2m_is_exact():
    """P2M at the parent equals M2M of the children's P2M (no truncation)."""
    p = 12
    parent = np.array([0.1, -0.2, 0.3])
    Mp_direct = np.zeros(oracle.NCOEF(p), complex)
    Mp_shift = np.zeros(oracle.NCOEF(p), complex)
    for k in range(4):
        c = parent + RNG.normal(size=3) * 0.3
        pos, m = _cluster(30, c, 0.2, k)
        Mp_direct += oracle.p2m(p, pos, m, parent)
        Mc = oracle.p2m(p, pos, m, c)
        Mp_shift += oracle.m2m(p, Mc, c - parent)
    scale = np.abs(Mp_direct).max()
    assert np.abs(Mp_direct - Mp_shift).max() <= 1e-13 * scale


def test_m2l_l2p_converge_to_direct_potential_and_force():
    """M2L + L2P reproduces the direct potential and acceleration of a distant
    cluster, within an error that falls geometrically with p."""
    za = np.array([3.0, 1.0, -2.0])
    zb = np.array([0.0, 0.0, 0.0])
    pos, m = _cluster(40, za, 0.5, 7)
    x = zb + np.array([0.2, -0.1, 0.15])
    d = pos - x
    r = np.linalg.norm(d, axis=1)
    phi_ref = -(m / r).sum()
    acc_ref = (m[:, None] * d / r[:, None] ** 3).sum(0)
    errs = []
    for p in (2, 4, 6, 8, 10, 12, 14):
        M = oracle.p2m(p, pos, m, za)
        F = oracle.m2l(p, M, za - zb)
        phi, ax, ay, az = oracle.l2p(p, F, x - zb)
        e = max(abs(phi - phi_ref) / abs(phi_ref), np.linalg.norm(np.array([ax, ay, az]) - acc_ref) / np.linalg.norm(acc_ref))
        errs.append(e)
    assert errs[-1] < 1e-9
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_l2l_is_exact_for_the_truncated_expansion():
    """Evaluating a local expansion at x equals evaluating its L2L shift."""
    p = 10
    pos, m = _cluster(20, np.array([4.0, -3.0, 2.0]), 0.7, 3)
    za = pos.T @ m / m.sum()
    zp = np.array([0.1, 0.2, -0.1])
    zc = zp + np.array([0.15, -0.05, 0.1])
    F = oracle.m2l(p, oracle.p2m(p, pos, m, za), za - zp)
    Fc = oracle.l2l(p, F, zc - zp)
    x = zc + np.array([0.05, 0.07, -0.02])
    a = np.array(oracle.l2p(p, F, x - zp))
    b = np.array(oracle.l2p(p, Fc, x - zc))
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_l2p_acceleration_is_minus_gradient_of_potential():
    p = 8
    pos, m = _cluster(25, np.array([2.0, 2.0, 1.0]), 0.5, 11)
    za = pos.T @ m / m.sum()
    F = oracle.m2l(p, oracle.p2m(p, pos, m, za), za)
    x = np.array([0.1, -0.05, 0.08])
    phi, ax, ay, az = oracle.l2p(p, F, x)
    h = 1e-5
    grad = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        grad.append((oracle.l2p(p, F, x + e)[0] - oracle.l2p(p, F, x - e)[0]) / (2 * h))
    assert np.allclose([ax, ay, az], -np.array(grad), rtol=1e-7)


def test_multipole_far_field_potential():
    p = 10
    pos, m = _cluster(50, np.zeros(3), 1.0, 5)
    M = oracle.p2m(p, pos, m, np.zeros(3))
    x = np.array([3.0, -2.5, 4.0])
    ref = -(m / np.linalg.norm(pos - x, axis=1)).sum()
    assert abs(oracle.eval_multipole(p, M, np.zeros(3), x) - ref) < 1e-7 * abs(ref)


# ------------------------------------------------------------------ solves

def test_single_body_and_two_body_exact():
    one = oracle.fmm(np.array([[0.3, -0.2, 0.1]]), np.array([1.0]), p=4)
    assert np.all(one[0] == 0.0) and np.all(one[1] == 0.0)
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0]])
    m = np.array([2.0, 3.0])
    acc, pot = oracle.fmm(pos, m, p=4, G=1.5)
    r = 3.0
    assert np.allclose(acc[0], 1.5 * 3.0 * pos[1] / r ** 3, rtol=1e-15)
    assert np.allclose(acc[1], -1.5 * 2.0 * pos[1] / r ** 3, rtol=1e-15)
    assert np.allclose(pot, [-1.5 * 3.0 / r, -1.5 * 2.0 / r], rtol=1e-15)


def test_direct_sum_obeys_newtons_third_law():
    pos, _, m = ics.plummer(2000, 9)
    m = ics.kroupa_masses(2000, 10)
    acc, _ = oracle.direct(pos, m)
    mom = (m[:, None] * acc).sum(0)
    assert np.abs(mom).max() < 1e-12 * (m[:, None] * np.abs(acc)).sum()


@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 200, 512])
def test_all_direct_when_eps_is_zero(n):
    """With eps = 0 the MAC never accepts, every interaction is P2P and the
    solve equals the direct sum to round-off."""
    pos, _, m = ics.plummer(n, 100 + n)
    run = oracle.OracleRun(pos, m, p=4, eps=0.0, leaf_size=8)
    assert run.status == 0 and run.npairs("m2l") == 0
    acc, pot = run.forces()
    ad, pd = oracle.direct(pos, m)
    if n > 1:
        assert np.abs(acc - ad).max() <= 1e-12 * np.abs(ad).max()
        assert np.abs(pot - pd).max() <= 1e-12 * np.abs(pd).max()
    mom = (m[:, None] * acc).sum(0)
    assert np.abs(mom).max() <= 1e-12 * max(1e-300, (m[:, None] * np.abs(acc)).sum())


def test_error_falls_with_p_at_fixed_geometric_mac():
    """With eps -> infinity the MAC is theta < 1 alone; the error then falls
    monotonically with the expansion order."""
    pos, _, m = ics.plummer(3000, 21)
    ad, _ = oracle.direct(pos, m)
    rms = []
    for p in (1, 2, 4, 6, 8, 10, 12):
        acc, _ = oracle.fmm(pos, m, p=p, eps=1e30, leaf_size=16)
        rms.append(oracle.error_stats(acc, ad)["rms"])
    assert all(b < a for a, b in zip(rms, rms[1:])), rms


def test_median_error_below_eps_and_falls_with_p():
    """Sec. 4.1: the median relative force error is always below the
    tolerance, and at a fixed tolerance it improves as p grows, except where
    the tolerance is small for the order (the paper's lower-left corner:
    there low p opens more cells and is more accurate)."""
    pos, _, m = ics.plummer(8192, 4)
    ad, _ = oracle.direct(pos, m)
    for eps in (1e-3, 1e-4, 1e-6):
        med = []
        for p in (4, 8, 12):
            acc, _ = oracle.fmm(pos, m, p=p, eps=eps)
            med.append(oracle.error_stats(acc, ad)["median"])
        assert all(v < eps for v in med), (eps, med)
        if eps >= 1e-4:
            assert med[2] < med[1] < med[0], (eps, med)


def test_plummer_closed_form_radial_profile():
    """A truncated Plummer sphere has M(<r) = M_P r^3/(r^2+a^2)^{3/2}, so the
    mean radial acceleration in a shell is -G M(<r)/r^2."""
    n = 20000
    pos, _, m = ics.plummer(n, 31, center=False)
    acc, pot = oracle.fmm(pos, m, p=8, eps=1e-6)
    a = ics.PLUMMER_A
    mp = 1.0 / (20.0 ** 3 / (400.0 + a * a) ** 1.5)  # normalisation of the untruncated model
    r = np.linalg.norm(pos, axis=1)
    ar = (acc * pos).sum(1) / r
    edges = np.array([0.2, 0.4, 0.7, 1.0, 1.5, 2.5])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        rr = r[sel]
        model = -mp * rr ** 3 / (rr * rr + a * a) ** 1.5 / rr ** 2
        diff = ar[sel] - model
        # shot noise of N discrete bodies: a few sigma of the shell scatter
        assert abs(diff.mean()) < 4 * diff.std() / math.sqrt(sel.sum()) + 0.02 * abs(model.mean())


def test_plummer_scale_radius_matches_paper():
    vals = {}
    with open(os.path.join(GOLDEN, "plummer.txt")) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            k, v = line.split()
            vals[k] = float(v)
    assert abs(ics.PLUMMER_A - vals["scale_radius_printed"]) < vals["scale_radius_tolerance"]
    assert abs(-3 * math.pi / (64 * ics.PLUMMER_A) - vals["energy"]) < 1e-15


def test_coincident_particles_are_rejected():
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    run = oracle.OracleRun(pos, np.ones(3), p=4)
    assert run.status == -5


# --------------------------------------------------------------- tree, lists

@pytest.mark.parametrize("n,leaf", [(1, 64), (65, 64), (4096, 64), (3000, 8)])
def test_tree_definition(n, leaf):
    pos, _, m = ics.plummer(n, 40 + n)
    run = oracle.OracleRun(pos, m, leaf_size=leaf, stage=oracle.STAGE_TREE)
    t = run.tree()
    keys = t["keys"].astype(np.uint64)
    assert np.all(keys[1:] >= keys[:-1])
    assert np.array_equal(np.sort(t["perm"]), np.arange(n))
    # equal keys keep input order (stable)
    eq = keys[1:] == keys[:-1]
    assert np.all(t["perm"][1:][eq] > t["perm"][:-1][eq])
    lvl, b, e, nch, fc = t["level"], t["begin"], t["end"], t["nchild"], t["first_child"]
    assert np.all(np.diff(lvl) >= 0)  # level-major
    leafcount = np.zeros(n, int)
    for k in range(run.nnodes):
        L = lvl[k]
        shift = np.uint64(3 * (21 - L))
        pre = keys[b[k]:e[k]] >> shift
        assert np.all(pre == pre[0])
        if nch[k] == 0:
            assert e[k] - b[k] <= leaf or L == 21
            leafcount[b[k]:e[k]] += 1
        else:
            assert e[k] - b[k] > leaf and L < 21
            kids = range(fc[k], fc[k] + nch[k])
            assert b[fc[k]] == b[k] and e[fc[k] + nch[k] - 1] == e[k]
            digits = [int((keys[b[c]] >> np.uint64(3 * (20 - L))) & np.uint64(7)) for c in kids]
            assert digits == sorted(set(digits))
            for c in kids:
                assert t["parent"][c] == k and lvl[c] == L + 1
    assert np.all(leafcount == 1)


def _decode_morton(keys, bits):
    """Per-axis integer coordinates (q_x, q_y, q_z) of `bits`-digit Morton
    keys, read with the x bit highest in each 3-bit digit."""
    keys = np.asarray(keys, dtype=np.uint64)
    q = np.zeros((len(keys), 3), dtype=np.int64)
    for b in range(bits):
        digit = ((keys >> np.uint64(3 * (bits - 1 - b))) & np.uint64(7)).astype(np.int64)
        for d in range(3):
            q[:, d] = (q[:, d] << 1) | ((digit >> (2 - d)) & 1)
    return q


def _key_cases():
    g = np.random.default_rng(2024)
    plummer = ics.plummer(3000, 91)[0]
    # extents 10 : 1 : 0.1, so a per-axis (non-cubic) box would differ from the cube
    elongated = g.uniform(0, 1, (2000, 3)) * np.array([10.0, 1.0, 0.1]) + np.array([-3.0, 2.0, 5.0])
    # nearly all bodies inside one octant of the root cube, two at opposite corners
    clustered = np.vstack([g.uniform(0.51, 0.52, (1500, 3)), [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]])
    # bodies on the faces and corners of the bounding box (the top edge is clamped)
    edges = g.uniform(-1, 1, (600, 3))
    edges[:100, 0] = 1.0
    edges[100:200, 1] = -1.0
    edges[200:300, 2] = 1.0
    edges[300] = [1.0, 1.0, 1.0]
    edges[301] = [-1.0, -1.0, -1.0]
    planar = np.column_stack([g.uniform(-2, 2, 800), g.uniform(-1, 1, 800), np.full(800, 0.25)])
    return {"plummer": plummer, "elongated": elongated, "clustered": clustered, "edges": edges,
            "planar": planar}


@pytest.mark.parametrize("case", ["plummer", "elongated", "clustered", "edges", "planar"])
def test_keys_place_every_body_inside_its_cell(case):
    """Reading R1 of the tree of Sec. 2.1 as geometry, not as a formula: the
    root cube has centre (min+max)/2 and half-size max_axis (max-min)/2; a
    body's 21-level key, read x bit first, names the cell of side 2h/2^21
    that contains it (the top face belongs to the last cell); the level-L
    prefix of every node names the cube of side 2h/2^L holding all of its
    bodies. Round instead of floor, a swapped axis order, a per-axis box or
    a missing clamp each put some body outside its cell."""
    pos = _key_cases()[case]
    n = len(pos)
    run = oracle.OracleRun(pos, np.full(n, 1.0 / n), leaf_size=16, stage=oracle.STAGE_TREE)
    assert run.status == 0
    t = run.tree()
    mn, mx = pos.min(0), pos.max(0)
    c, h = 0.5 * (mn + mx), float((0.5 * (mx - mn)).max())
    assert np.array_equal(t["box"][:3], c) and t["box"][3] == h
    lo = c - h
    ps = pos[t["perm"]]
    q = _decode_morton(t["keys"], 21)
    w = 2 * h / 2 ** 21
    tol = 1e-6 * w
    rel = ps - lo
    assert np.all(q >= 0) and np.all(q < 2 ** 21)
    assert np.all(rel >= q * w - tol)
    top = q == 2 ** 21 - 1
    assert np.all((rel < (q + 1) * w + tol) | top)
    assert np.all(rel[top] <= 2 * h + tol)
    # bodies on the top face of the cube are clamped into the last cell
    on_top = np.abs(ps - (c + h)) == 0
    assert np.all(q[on_top] == 2 ** 21 - 1)
    for k in range(run.nnodes):
        L = int(t["level"][k])
        b, e = t["begin"][k], t["end"][k]
        Q = _decode_morton(t["keys"][b:b + 1] >> np.uint64(3 * (21 - L)), L)[0] if L else np.zeros(3, int)
        side = 2 * h / 2 ** L
        r = rel[b:e]
        assert np.all(r >= Q * side - tol) and np.all(r <= (Q + 1) * side + tol)


def _multipole_closed_form(p, pos, m, center):
    """M_n^m = sum_i m_i Upsilon_n^m(x_i - z) with Upsilon from scipy's
    associated Legendre functions (Sec. 2.2, Dehnen's normalisation; scipy
    includes the Condon-Shortley phase, hence the (-1)^m)."""
    d = pos - center
    r = np.linalg.norm(d, axis=1)
    ct = np.where(r > 0, d[:, 2] / np.where(r > 0, r, 1), 1.0)
    ph = np.arctan2(d[:, 1], d[:, 0])
    M = np.zeros(oracle.NCOEF(p), complex)
    for n in range(p + 1):
        for mm in range(n + 1):
            ups = r ** n * (-1) ** mm * lpmv(mm, n, ct) * np.exp(1j * mm * ph) / math.factorial(n + mm)
            M[idx(n, mm)] = (m * ups).sum()
    return M


def test_solve_multipoles_and_degree_norms_follow_their_definitions():
    """The multipoles a solve keeps for every node (P2M at the leaves, M2M
    above) equal the moments sum_i m_i Upsilon_n^m(x_i - z_A) of the node's
    bodies, and the exported degree norms are Sec. 2.3's
    P_n^2 = sum_{m=-n..n} (n-m)!(n+m)! |M_n^m|^2 of those moments. A dropped
    factor 2 on the m >= 1 terms, a wrong factorial or a missing degree
    fails this."""
    p = 8
    pos, _, _ = ics.plummer(1500, 17)
    m = ics.kroupa_masses(1500, 18)
    run = oracle.OracleRun(pos, m, p=p, leaf_size=32, stage=oracle.STAGE_F)
    t, g, mult = run.tree(), run.geometry(), run.multipoles()
    ps, ms = pos[t["perm"]], m[t["perm"]]
    leaves = np.flatnonzero(t["nchild"] == 0)
    inner = np.flatnonzero(t["nchild"] > 0)
    nodes = np.concatenate([[0], inner[:: max(1, len(inner) // 6)], leaves[:: max(1, len(leaves) // 8)]])
    for k in nodes:
        sl = slice(t["begin"][k], t["end"][k])
        ref = _multipole_closed_form(p, ps[sl], ms[sl], g["z"][k])
        scale = ms[sl].sum() * max(g["r"][k], 1e-300) ** np.array([n for n in range(p + 1) for _ in range(n + 1)])
        assert np.all(np.abs(mult[k] - ref) <= 1e-11 * scale + 1e-300), k
        Pn = np.array([math.sqrt(sum(math.factorial(n - mm) * math.factorial(n + mm) * abs(full(ref, n, mm)) ** 2
                                     for mm in range(-n, n + 1))) for n in range(p + 1)])
        assert np.allclose(g["P"][k], Pn, rtol=1e-10, atol=1e-12 * ms[sl].sum() * g["r"][k] ** np.arange(p + 1))
        # P_0 is the mass; P_1 vanishes about the centre of mass (reading R3)
        assert math.isclose(g["P"][k][0], ms[sl].sum(), rel_tol=1e-13)
        assert g["P"][k][1] <= 1e-12 * ms[sl].sum() * max(g["r"][k], 1e-300)
    # every node: the exported norms are those of the exported moments
    for k in range(run.nnodes):
        Pn = [math.sqrt(sum(math.factorial(n - mm) * math.factorial(n + mm) * abs(full(mult[k], n, mm)) ** 2
                            for mm in range(-n, n + 1))) for n in range(p + 1)]
        assert np.allclose(g["P"][k], Pn, rtol=1e-12, atol=0), k


@pytest.mark.parametrize("n,eps,p", [(1200, 1e-4, 4), (1500, 1e-7, 8), (900, 1e30, 3)])
def test_lists_cover_every_particle_pair_exactly_once(n, eps, p):
    """Every ordered pair (i, j), i != j, is handled exactly once: by one M2L
    pair or one P2P pair (the dual-tree walk of Sec. 2.1). Accepted pairs are
    well separated, theta = (r_A + r_B)/r < 1."""
    pos, _, m = ics.plummer(n, 77)
    run = oracle.OracleRun(pos, m, p=p, eps=eps, leaf_size=16, stage=oracle.STAGE_LISTS)
    t, g = run.tree(), run.geometry()
    cover = np.zeros((n, n), int)
    for which in ("m2l", "p2p"):
        for a, b in run.pairs(which):
            ia = np.arange(t["begin"][a], t["end"][a])
            ib = np.arange(t["begin"][b], t["end"][b])
            if a == b:
                cover[np.ix_(ia, ia)] += 1
            else:
                cover[np.ix_(ia, ib)] += 1
                cover[np.ix_(ib, ia)] += 1
            if which == "m2l":
                rr = np.linalg.norm(g["z"][a] - g["z"][b])
                assert g["r"][a] + g["r"][b] < rr
    off = ~np.eye(n, dtype=bool)
    assert np.all(cover[off] == 1)


def test_cell_geometry_definitions():
    pos, _, _ = ics.plummer(3000, 8)
    m = ics.kroupa_masses(3000, 9)
    run = oracle.OracleRun(pos, m, leaf_size=32, stage=oracle.STAGE_F)
    t, g = run.tree(), run.geometry()
    ps = pos[t["perm"]]
    ms = m[t["perm"]]
    for k in range(run.nnodes):
        sl = slice(t["begin"][k], t["end"][k])
        com = (ms[sl, None] * ps[sl]).sum(0) / ms[sl].sum()
        assert np.allclose(g["z"][k], com, rtol=1e-12, atol=1e-13)
        assert math.isclose(g["M"][k], ms[sl].sum(), rel_tol=1e-13)
        rmax = np.linalg.norm(ps[sl] - g["z"][k], axis=1).max()
        assert g["r"][k] >= rmax * (1 - 1e-12)
        if t["nchild"][k] == 0:
            assert math.isclose(g["r"][k], rmax, rel_tol=1e-12)


def test_degree_norms_are_rotation_invariant():
    """P_n of Sec. 2.3 depends only on the multipole's shape: rotating the
    particles about the centre leaves it unchanged."""
    p = 10
    pos, m = _cluster(40, np.zeros(3), 1.0, 2)
    th = 0.7
    rot = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    rot = rot @ np.array([[math.cos(1.1), -math.sin(1.1), 0], [math.sin(1.1), math.cos(1.1), 0], [0, 0, 1]])

    def norms(M):
        return np.array([math.sqrt(sum(math.factorial(n - mm) * math.factorial(n + mm) * abs(full(M, n, mm)) ** 2
                                       for mm in range(-n, n + 1))) for n in range(p + 1)])
    a = norms(oracle.p2m(p, pos, m, np.zeros(3)))
    b = norms(oracle.p2m(p, pos @ rot.T, m, np.zeros(3)))
    assert np.allclose(a, b, rtol=1e-12)


def test_scalar_force_estimate_is_exact_when_all_near():
    """With one leaf (N <= leaf size) the estimate f_i is the exact scalar
    force sum_j m_j/|x_i - x_j|^2 in FP32 (Sec. 2.3)."""
    pos, _, m = ics.plummer(50, 3)
    run = oracle.OracleRun(pos, m, leaf_size=64, stage=oracle.STAGE_F)
    f = run.geometry()["f"]
    ps, ms = pos[run.tree()["perm"]], m[run.tree()["perm"]]
    d = ps[:, None, :] - ps[None, :, :]
    r2 = (d * d).sum(-1)
    np.fill_diagonal(r2, np.inf)
    exact = (ms[None, :] / r2).sum(1)
    assert np.allclose(f, exact, rtol=2e-5)


def test_scalar_force_estimate_tracks_exact():
    pos, _, m = ics.plummer(4096, 6)
    run = oracle.OracleRun(pos, m, leaf_size=64, stage=oracle.STAGE_F)
    f = run.geometry()["f"].astype(np.float64)
    ps, ms = pos[run.tree()["perm"]], m[run.tree()["perm"]]
    exact = np.zeros(len(ms))
    for i in range(0, len(ms), 512):
        d = ps[i:i + 512, None, :] - ps[None, :, :]
        r2 = (d * d).sum(-1)
        r2[r2 == 0] = np.inf
        exact[i:i + 512] = (ms[None, :] / r2).sum(1)
    # theta < 1 lets a monopole stand for a cell seen at up to ~90 degrees, so
    # the estimate is rough; a dropped far term or a wrong power of r would
    # shift the whole distribution by far more than these bounds
    rel = (f - exact) / exact
    assert np.median(np.abs(rel)) < 0.15
    lo, hi = np.percentile(rel, [1, 99])
    assert -0.5 < lo and hi < 1.0 and rel.max() < 2.0


def test_mac_error_estimate_bounds_the_true_m2l_error():
    """E_{A->B} M_A / r^2 (Sec. 2.3) estimates the force error of the
    truncated M2L from A at any particle of B. On the pairs a solve accepts
    it must cover the true error, and not by a wide margin."""
    n, p = 3000, 6
    pos, _, m = ics.plummer(n, 55)
    run = oracle.OracleRun(pos, m, p=p, eps=1e-5, leaf_size=16, stage=oracle.STAGE_LISTS)
    t, g = run.tree(), run.geometry()
    mult = run.multipoles()
    ps, ms = pos[t["perm"]], m[t["perm"]]
    pairs = run.pairs("m2l")
    sel = np.random.default_rng(1).choice(len(pairs), size=min(150, len(pairs)), replace=False)
    worst = 0.0
    ratios = []
    for a, b in pairs[sel]:
        v = run.mac_values(a, b)
        assert v[4] == 1.0 and v[0] < v[2] and v[1] < v[3]
        for src, dst, lhs in ((a, b, v[0]), (b, a, v[1])):
            F = oracle.m2l(p, mult[src], g["z"][src] - g["z"][dst])
            js = np.arange(t["begin"][src], t["end"][src])
            for i in range(t["begin"][dst], t["end"][dst]):
                _, ax, ay, az = oracle.l2p(p, F, ps[i] - g["z"][dst])
                d = ps[js] - ps[i]
                rr = np.linalg.norm(d, axis=1)
                ref = (ms[js, None] * d / rr[:, None] ** 3).sum(0)
                err = np.linalg.norm(np.array([ax, ay, az]) - ref)
                floor = 1e-12 * np.linalg.norm(ref)  # round-off of the reference sum
                if lhs > 1e3 * floor:
                    worst = max(worst, err / lhs)
                    ratios.append(err / lhs)
    q90, q99 = np.percentile(ratios, [90, 99])
    # an estimate, not a strict bound: it covers 99% of particles and is
    # never off by more than 2x; and it is not loose by orders of magnitude
    assert q99 <= 1.0 and worst <= 2.0 and q90 > 0.02, (q90, q99, worst)


# --------------------------------------------------------------- softening

def test_softened_direct_two_body_closed_form():
    """Appendix B: phi(r) = -G m / sqrt(r^2 + soft^2), so a body at d from a
    mass m feels G m d / (|d|^2 + soft^2)^{3/2}."""
    pos = np.array([[0.1, -0.2, 0.3], [0.4, 0.2, -0.1]])
    m = np.array([2.0, 3.0])
    soft, G = 0.07, 1.5
    acc, pot = oracle.direct(pos, m, G=G, soft=soft)
    d = pos[1] - pos[0]
    s2 = d @ d + soft * soft
    assert np.allclose(acc[0], G * 3.0 * d / s2 ** 1.5, rtol=1e-15, atol=0)
    assert np.allclose(acc[1], -G * 2.0 * d / s2 ** 1.5, rtol=1e-15, atol=0)
    assert np.allclose(pot, [-G * 3.0 / math.sqrt(s2), -G * 2.0 / math.sqrt(s2)], rtol=1e-15)


def test_softened_direct_obeys_newtons_third_law_and_tends_to_newton():
    pos, _, m = ics.plummer(1500, 91)
    m = ics.kroupa_masses(1500, 92)
    acc, _ = oracle.direct(pos, m, soft=1e-2)
    mom = (m[:, None] * acc).sum(0)
    assert np.abs(mom).max() < 1e-12 * (m[:, None] * np.abs(acc)).sum()
    # a softening far below every separation changes nothing visible
    a0, p0 = oracle.direct(pos, m)
    a1, p1 = oracle.direct(pos, m, soft=1e-12)
    assert np.allclose(a1, a0, rtol=1e-9) and np.allclose(p1, p0, rtol=1e-12)


@pytest.mark.parametrize("n", [2, 65, 300])
def test_softened_solve_is_the_softened_direct_sum_when_eps_is_zero(n):
    pos, _, m = ics.plummer(n, 200 + n)
    run = oracle.OracleRun(pos, m, p=4, eps=0.0, leaf_size=8, soft=0.03)
    assert run.status == 0 and run.npairs("m2l") == 0
    acc, pot = run.forces()
    ad, pd = oracle.direct(pos, m, soft=0.03)
    assert np.abs(acc - ad).max() <= 1e-12 * np.abs(ad).max()
    assert np.abs(pot - pd).max() <= 1e-12 * np.abs(pd).max()


def test_softening_bound_is_the_leading_term_for_two_bodies():
    """For two single-body cells (r_A = r_B = 0, so d_min = d) the MAC's
    softening term 1.5 M_A soft^2 / d^4 is the leading term of the exact
    difference m/d^2 - m d/(d^2 + soft^2)^{3/2}: their ratio is 1 - O(soft^2/d^2)."""
    pos = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 0.0]])  # d = 0.5
    m = np.array([2.0, 5.0])
    for soft in (5e-4, 5e-3):
        run = oracle.OracleRun(pos, m, p=4, eps=1e-6, leaf_size=1, stage=oracle.STAGE_LISTS, soft=soft)
        t = run.tree()
        leaves = [k for k in range(run.nnodes) if t["nchild"][k] == 0]
        a, b = leaves
        ma, mb = m[t["perm"][t["begin"][a]]], m[t["perm"][t["begin"][b]]]
        v = run.mac_values(a, b)
        d = 0.5
        for mass, bound in ((ma, v[5]), (mb, v[6])):
            exact = mass / d ** 2 - mass * d / (d * d + soft * soft) ** 1.5
            u = soft * soft / (d * d)
            assert 1.0 - 2.0 * u < exact / bound <= 1.0, (soft, exact / bound)


def test_softening_bound_covers_every_accepted_pair():
    """On the pairs a softened solve accepts, the bound covers the exact
    softened-minus-Newtonian acceleration of A's bodies at every body of B."""
    n, soft = 1200, 0.02
    pos, _, m = ics.plummer(n, 93)
    run = oracle.OracleRun(pos, m, p=6, eps=1e-4, leaf_size=16, stage=oracle.STAGE_LISTS, soft=soft)
    t = run.tree()
    ps, ms = pos[t["perm"]], m[t["perm"]]
    pairs = run.pairs("m2l")
    assert len(pairs) > 50
    tight = 0.0
    for a, b in pairs[np.random.default_rng(2).choice(len(pairs), size=min(200, len(pairs)), replace=False)]:
        v = run.mac_values(a, b)
        assert v[4] == 1.0 and v[0] + v[5] < v[2] and v[1] + v[6] < v[3]
        for src, dst, bound in ((a, b, v[5]), (b, a, v[6])):
            js = np.arange(t["begin"][src], t["end"][src])
            for i in range(t["begin"][dst], t["end"][dst]):
                d = ps[js] - ps[i]
                r2 = (d * d).sum(1)
                diff = (ms[js, None] * d * (r2[:, None] ** -1.5 - (r2[:, None] + soft * soft) ** -1.5)).sum(0)
                err = np.linalg.norm(diff)
                assert err <= bound * (1 + 1e-9), (err, bound)
                tight = max(tight, err / bound)
    assert tight > 0.05  # the bound is not loose by orders of magnitude


def test_softened_solve_meets_the_tolerance():
    """With a softening large enough to matter (soft = 0.01 against cell
    separations of ~0.05 in the core), the far field alone would be off by
    ~1.5 (soft/d)^2 ~ 6%; the MAC's softening term keeps the error at the
    tolerance."""
    pos, _, m = ics.plummer(4000, 94)
    soft, eps = 0.01, 1e-6
    ad, _ = oracle.direct(pos, m, soft=soft)
    acc, _ = oracle.fmm(pos, m, p=8, eps=eps, soft=soft)
    st = oracle.error_stats(acc, ad)
    assert st["median"] < eps and st["rms"] < 10 * eps and st["max"] < 1e-3, st


def test_softened_scalar_force_estimate_is_exact_when_all_near():
    """With one leaf the softened estimate is sum_j m_j r_ij / (r_ij^2 + soft^2)^{3/2}
    in FP32."""
    pos, _, m = ics.plummer(50, 3)
    soft = 0.05
    run = oracle.OracleRun(pos, m, leaf_size=64, stage=oracle.STAGE_F, soft=soft)
    f = run.geometry()["f"]
    ps, ms = pos[run.tree()["perm"]], m[run.tree()["perm"]]
    d = ps[:, None, :] - ps[None, :, :]
    r2 = (d * d).sum(-1)
    term = ms[None, :] * np.sqrt(r2) / (r2 + soft * soft) ** 1.5
    np.fill_diagonal(term, 0.0)
    assert np.allclose(f, term.sum(1), rtol=2e-5)


# ------------------------------------------------------------------- jerks

def _fd_regular(p, v, h=1e-6):
    out = []
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        out.append((oracle.regular(p, *(v + e)) - oracle.regular(p, *(v - e))) / (2 * h))
    return out


def test_regular_gradient_matches_finite_differences():
    """The ladder relations d_z U_n^m = U_{n-1}^m, (d_x + i d_y) U_n^m = -U_{n-1}^{m+1},
    (d_x - i d_y) U_n^m = U_{n-1}^{m-1} against central differences of the recurrences."""
    p = 12
    for _ in range(4):
        v = RNG.normal(size=3) * 0.6
        g = oracle.regular_grad(p, *v)
        fd = _fd_regular(p, v)
        for a, b in zip(g, fd):
            assert np.abs(a - b).max() < 1e-8 * max(1.0, np.abs(b).max())


def test_l2p_hessian_is_the_derivative_of_the_l2p_acceleration():
    p = 10
    pos = RNG.normal(size=(40, 3)) * 0.2 + np.array([3.0, -2.0, 1.5])
    m = RNG.uniform(0.5, 1.5, 40)
    F = oracle.m2l(p, oracle.p2m(p, pos, m, pos.mean(0)), pos.mean(0))
    d = np.array([0.11, -0.07, 0.05])
    h = oracle.l2p_hessian(p, F, d)
    H = np.array([[h[0], h[3], h[4]], [h[3], h[1], h[5]], [h[4], h[5], h[2]]])
    e = 1e-5
    for c in range(3):
        dp, dm = d.copy(), d.copy()
        dp[c] += e
        dm[c] -= e
        ap = np.array(oracle.l2p(p, F, dp)[1:])
        am = np.array(oracle.l2p(p, F, dm)[1:])
        assert np.allclose((ap - am) / (2 * e), H[:, c], rtol=1e-6, atol=1e-9 * np.abs(H).max())
    assert abs(h[0] + h[1] + h[2]) < 1e-10 * np.abs(h).max()  # harmonic: traceless


def test_dipole_multipoles_give_the_dipole_far_field():
    """chi(x) = sum_j D_j . grad_x (1/|x_j - x|) = sum_j D_j . (x_j - x)/|x_j - x|^3."""
    p = 14
    c = np.array([0.2, -0.1, 0.3])
    pos = c + RNG.normal(size=(30, 3)) * 0.1
    dip = RNG.normal(size=(30, 3))
    M = oracle.p2m_dipole(p, pos, dip, c)
    assert abs(M[0]) == 0.0  # dipoles carry no monopole
    for x in (np.array([2.0, 1.0, -1.5]), np.array([-3.0, 0.5, 0.2])):
        d = pos - x
        chi = (dip * d).sum(1) @ (1.0 / np.linalg.norm(d, axis=1) ** 3)
        assert np.isclose(-oracle.eval_multipole(p, M, c, x), chi, rtol=1e-10)


def test_direct_jerk_is_the_time_derivative_of_the_acceleration():
    pos, vel, m = ics.plummer(300, 41)
    for soft in (0.0, 0.02):
        j = oracle.direct_jerk(pos, vel, m, G=1.3, soft=soft)
        h = 1e-6
        ap, _ = oracle.direct(pos + h * vel, m, G=1.3, soft=soft)
        am, _ = oracle.direct(pos - h * vel, m, G=1.3, soft=soft)
        fd = (ap - am) / (2 * h)
        assert np.abs(fd - j).max() < 1e-5 * np.abs(j).max()


@pytest.mark.parametrize("soft", [0.0, 0.03])
def test_jerk_is_the_direct_jerk_when_eps_is_zero(soft):
    pos, vel, m = ics.plummer(400, 42)
    run = oracle.OracleRun(pos, m, p=4, eps=0.0, leaf_size=8, soft=soft)
    j = run.jerk(vel)
    jd = oracle.direct_jerk(pos, vel, m, soft=soft)
    assert np.abs(j - jd).max() <= 1e-11 * np.abs(jd).max()


def test_jerk_error_falls_with_eps():
    """The far part (dipole moments, M2M, M2L, L2L, the gradient of chi and
    the Hessian term) converges: as the MAC tolerance falls the jerk error
    falls with it. A wrong sign or index in any far term leaves an O(1)
    error that no tolerance removes. (A purely geometric MAC is no test here:
    pairs at theta near 1 converge like theta^p, slower for the second
    derivatives than for the force.)"""
    pos, vel, m = ics.plummer(3000, 43)
    jd = oracle.direct_jerk(pos, vel, m)
    med = []
    for eps in (1e-3, 1e-5, 1e-7, 1e-9):
        run = oracle.OracleRun(pos, m, p=8, eps=eps, leaf_size=16)
        assert run.npairs("m2l") > 1000
        j = run.jerk(vel)
        d = np.linalg.norm(j - jd, axis=1) / np.linalg.norm(jd, axis=1)
        med.append(np.median(d))
    assert all(b < 0.1 * a for a, b in zip(med, med[1:])), med
    assert med[-1] < 1e-7, med


def test_jerk_meets_a_tolerance_like_the_acceleration():
    pos, vel, m = ics.plummer(4000, 44)
    jd = oracle.direct_jerk(pos, vel, m)
    run = oracle.OracleRun(pos, m, p=10, eps=1e-8, leaf_size=32)
    j = run.jerk(vel)
    d = np.linalg.norm(j - jd, axis=1) / np.linalg.norm(jd, axis=1)
    assert np.median(d) < 1e-6 and np.sqrt(np.mean(d * d)) < 1e-4, (np.median(d), np.sqrt(np.mean(d * d)))


# ---------------------------------------------------------- HOLD (App. A)

def test_pair_step_sizes_and_their_time_derivatives():
    """Free-fall time eta sqrt(r^3 / (G m)) and fly-by time eta r / v; the
    symmetrized step tau / (1 - tau'/2) with tau' checked against central
    differences of tau along the two-body motion."""
    G, mij, eta = 1.3, 0.7, 0.05
    # slow relative motion: the free-fall time is the smaller one
    r, v = np.array([0.3, -0.1, 0.2]), np.array([0.02, 0.05, -0.01])
    rn = np.linalg.norm(r)
    tff = eta * np.sqrt(rn ** 3 / (G * mij))
    assert np.isclose(oracle.tau_pair(r, v, mij, G, eta), tff, rtol=1e-15)
    # fast fly-by: the fly-by time is the smaller one
    vf = np.array([3.0, -2.0, 1.0])
    assert np.isclose(oracle.tau_pair(r, vf, mij, G, eta), eta * rn / np.linalg.norm(vf), rtol=1e-15)
    # circular-like motion (r . v = 0, no radial speed) leaves the free-fall time unchanged
    vc = np.cross(r, [0.0, 0.0, 1.0]) * 0.01
    assert np.isclose(oracle.tau_pair(r, vc, mij, G, eta, sym=True), oracle.tau_pair(r, vc, mij, G, eta), rtol=1e-15)

    def moved(r, v, h):
        a = -G * mij * r / np.linalg.norm(r) ** 3
        return r + h * v + 0.5 * h * h * a, v + h * a

    h = 1e-6
    for rr, vv in ((r, v), (r, vf)):
        t = oracle.tau_pair(rr, vv, mij, G, eta)
        rp, vp = moved(rr, vv, h)
        rm, vm = moved(rr, vv, -h)
        dt = (oracle.tau_pair(rp, vp, mij, G, eta) - oracle.tau_pair(rm, vm, mij, G, eta)) / (2 * h)
        assert np.isclose(oracle.tau_pair(rr, vv, mij, G, eta, sym=True), t / (1 - 0.5 * dt), rtol=1e-7)


def _leapfrog(pos, vel, m, dt, steps):
    pos, vel = pos.copy(), vel.copy()
    for _ in range(steps):
        a, _ = oracle.direct(pos, m)
        vel += 0.5 * dt * a
        pos += dt * vel
        a, _ = oracle.direct(pos, m)
        vel += 0.5 * dt * a
    return pos, vel


def test_hold_is_the_leapfrog_when_no_body_is_fast():
    pos, vel, m = ics.plummer(64, 51)
    p, v, st = oracle.hold(pos, vel, m, dt=1 / 128, nsteps=20, eta=1e6, sym=False)
    lp, lv = _leapfrog(pos, vel, m, 1 / 128, 20)
    assert st["max_depth"] == 0
    assert np.abs(p - lp).max() < 1e-14 and np.abs(v - lv).max() < 1e-13


def test_hold_conserves_momentum_and_angular_momentum():
    """Every kick of V_FS acts on both sets with the same step, drifts are
    straight: both are conserved to round-off across the levels."""
    pos, vel, m = ics.plummer(80, 52)
    m = ics.kroupa_masses(80, 53)
    p, v, st = oracle.hold(pos, vel, m, dt=1 / 32, nsteps=32, eta=0.05, sym=True, dt_min=1e-9)
    assert st["max_depth"] >= 3
    P0, P1 = (m[:, None] * vel).sum(0), (m[:, None] * v).sum(0)
    L0, L1 = (m[:, None] * np.cross(pos, vel)).sum(0), (m[:, None] * np.cross(p, v)).sum(0)
    scale = (m[:, None] * np.abs(v)).sum()
    assert np.abs(P1 - P0).max() < 1e-13 * scale
    assert np.abs(L1 - L0).max() < 1e-12 * (m[:, None] * np.abs(np.cross(p, v))).sum()


@pytest.mark.parametrize("sym", [False, True])
def test_hold_is_second_order(sym):
    """Appendix A: the splitting is second order. Over a quarter time unit the
    positions converge to a small-eta reference with errors falling ~4x per
    halving of eta (the step sizes scale with eta)."""
    pos, vel, m = ics.plummer(100, 7)
    ref, _, _ = oracle.hold(pos, vel, m, dt=1 / 64, nsteps=16, eta=0.0025, sym=sym, dt_min=1e-12)
    err = []
    for eta in (0.04, 0.02, 0.01):
        p, _, _ = oracle.hold(pos, vel, m, dt=1 / 64, nsteps=16, eta=eta, sym=sym, dt_min=1e-12)
        err.append(np.abs(p - ref).max())
    for a, b in zip(err, err[1:]):
        assert 3.0 < a / b < 5.5, err


def test_symmetrized_steps_reduce_the_energy_drift():
    """Appendix A: individual time steps break the leapfrog's time symmetry
    and make the energy drift; the time-symmetrized step removes most of it."""
    errs = {False: [], True: []}
    for seed in (7, 8, 9):
        pos, vel, m = ics.plummer(100, seed)
        E0 = oracle.energy(pos, vel, m)
        for sym in (False, True):
            p, v, _ = oracle.hold(pos, vel, m, dt=1 / 64, nsteps=320, eta=0.05, sym=sym, dt_min=1e-9)
            errs[sym].append(abs(oracle.energy(p, v, m) / E0 - 1))
    assert np.mean(errs[True]) < 0.3 * np.mean(errs[False]), errs


def test_step_sizes_of_a_set_are_the_minimum_over_pairs():
    pos, vel, m = ics.plummer(40, 54)
    t = oracle.taus(pos, vel, m, eta=0.04, sym=True)
    for i in (0, 17, 39):
        ref = min(oracle.tau_pair(pos[j] - pos[i], vel[j] - vel[i], m[i] + m[j], 1.0, 0.04, True)
                  for j in range(40) if j != i)
        assert t[i] == ref


def test_total_energy_two_body_and_against_the_direct_potential():
    """E = sum m v^2 / 2 - G sum_{i<j} m_i m_j / r_ij: the two-body closed form,
    and half the direct sum's potential energy sum m_i phi_i for many bodies."""
    pos = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    vel = np.array([[0.1, 0.0, 0.0], [0.0, -0.2, 0.3]])
    m = np.array([2.0, 3.0])
    e = 0.5 * 2.0 * 0.01 + 0.5 * 3.0 * 0.13 - 1.7 * 6.0 / 0.5
    assert np.isclose(oracle.energy(pos, vel, m, G=1.7), e, rtol=1e-15)
    pos, vel, m = ics.plummer(500, 95)
    _, pot = oracle.direct(pos, m, soft=0.01)
    ref = 0.5 * (m * (vel * vel).sum(1)).sum() + 0.5 * (m * pot).sum()
    assert np.isclose(oracle.energy(pos, vel, m, soft=0.01), ref, rtol=1e-12)
