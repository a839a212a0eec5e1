"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Every test here runs on the CPU (no GPU).  The references are:
  * the gradient of the Ewald short-range potential erfc(r/2x_s)/r
    (Section 2.1.1 "Ewald summation"), differentiated numerically by mpmath;
  * Gauss's law applied to the softening *densities* of Eqs. plummer_shape and
    bspline_shape (integrated by mpmath), rather than the printed force forms;
  * O(N^2) brute force and an explicit sum over the 27 nearest images;
  * Newton's third law, permutation and translation invariance;
  * finite differences of the oracle's forward for its analytic VJP;
  * log2/ceil for Eq. rung, floor() for the subtile ids;
  * the rejection fractions printed in Section 2.1.3 (Monte Carlo).
"""
import math

import numpy as np
import pytest

import oracle
import synth

mp = pytest.importorskip("mpmath")

W = synth.workload("n32k")
XS, XR, EPS, GM = W.x_s, W.x_r, W.eps, W.G_m
EPS_B = 2.8 * EPS


# --------------------------------------------------------------------------
# references
# --------------------------------------------------------------------------

def _ref_newton_part(r, x_s):
    """-(d/dr)[erfc(r/2x_s)/r] / r, the short-range Ewald force per unit displacement."""
    mp.mp.dps = 40
    f = lambda t: mp.erfc(t / (2 * mp.mpf(x_s))) / t
    return -mp.diff(f, mp.mpf(r)) / mp.mpf(r)


def _bspline_density(t, eps_b):
    xb = t / eps_b
    c = 8 / (mp.pi * eps_b ** 3)
    if xb < mp.mpf(1) / 2:
        return c * (1 - 6 * xb ** 2 * (1 - xb))
    if xb < 1:
        return c * 2 * (1 - xb) ** 3
    return mp.mpf(0)


def _plummer_density(t, eps):
    return 3 / (4 * mp.pi * eps ** 3) * (1 + t ** 2 / eps ** 2) ** (-mp.mpf(5) / 2)


def _enclosed_mass(r, softening, eps):
    mp.mp.dps = 40
    r = mp.mpf(r)
    if softening == "bspline":
        eb = mp.mpf(2.8) * mp.mpf(eps)
        pts = [0, min(r, eb / 2), min(r, eb), r]
        pts = sorted(set(pts))
        return mp.quad(lambda t: 4 * mp.pi * t ** 2 * _bspline_density(t, eb), pts)
    if softening == "plummer":
        e = mp.mpf(eps)
        return mp.quad(lambda t: 4 * mp.pi * t ** 2 * _plummer_density(t, e), [0, r])
    return mp.mpf(1)


def _ref_bracket(r, x_s, softening, eps):
    """B(r) from the Ewald potential gradient plus Gauss's law for the shape."""
    rr = mp.mpf(r)
    soft = _enclosed_mass(r, softening, eps) / rr ** 3 - 1 / rr ** 3
    return float(_ref_newton_part(r, x_s) + soft)


# --------------------------------------------------------------------------
# the bracket
# --------------------------------------------------------------------------

@pytest.mark.parametrize("softening", ["none", "plummer", "bspline"])
@pytest.mark.parametrize("frac", [0.1, 0.5, 0.9, 0.999])
def test_bracket_vs_ewald_gradient_and_gauss(softening, frac):
    r = frac * XR
    got = oracle.bracket(r, XS, softening, EPS)[0]
    ref = _ref_bracket(r, XS, softening, EPS)
    assert got == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("softening", ["plummer", "bspline"])
@pytest.mark.parametrize("frac", [1e-4, 0.05, 0.3, 0.5, 0.7, 0.999, 1.001, 1.5])
def test_bracket_inside_softening_length(softening, frac):
    r = frac * EPS_B
    got = oracle.bracket(r, XS, softening, EPS)[0]
    ref = _ref_bracket(r, XS, softening, EPS)
    assert got == pytest.approx(ref, rel=1e-12)


def test_bspline_shape_is_normalised():
    m = _enclosed_mass(EPS_B * 1.0000001, "bspline", EPS)
    assert float(m) == pytest.approx(1.0, abs=1e-15)


def test_newtonian_limit():
    # far inside x_s the short-range force is the Newtonian 1/r^2 (erfc -> 1)
    r = 1e-6 * XS
    b = oracle.bracket(r, XS, "none", 0.0)[0]
    assert b * r ** 3 == pytest.approx(1.0, rel=1e-5)


@pytest.mark.parametrize("point", [0.5, 1.0])
def test_bspline_continuity(point):
    # Eq. bspline_force is continuous at x_B = 1/2 and x_B = 1
    r = point * EPS_B
    lo = oracle.bracket(r * (1 - 1e-12), XS, "bspline", EPS)[0]
    hi = oracle.bracket(r * (1 + 1e-12), XS, "bspline", EPS)[0]
    assert lo == pytest.approx(hi, rel=1e-9)


@pytest.mark.parametrize("softening", ["none", "plummer", "bspline"])
@pytest.mark.parametrize("frac", [0.02, 0.3, 0.8])
def test_bracket_derivative_vs_numeric(softening, frac):
    r = frac * XR if softening == "none" else frac * EPS_B * 3
    got = oracle.bracket_dr(r, XS, softening, EPS)[0]
    mp.mp.dps = 40
    h = r * 1e-5
    # Richardson-extrapolated central difference of the (independently pinned) oracle bracket
    f = lambda t: oracle.bracket(t, XS, softening, EPS)[0]
    d1 = (f(r + h) - f(r - h)) / (2 * h)
    d2 = (f(r + 2 * h) - f(r - 2 * h)) / (4 * h)
    num = (4 * d1 - d2) / 3
    assert got == pytest.approx(num, rel=1e-6)


# --------------------------------------------------------------------------
# sums over particles
# --------------------------------------------------------------------------

def _two_body(x1, x2, softening):
    pos = np.array([x1, x2], dtype=np.float64).T.copy()
    acc, pairs = oracle.sr_accel(pos, XS, XR, GM, softening, EPS)
    return acc, pairs


@pytest.mark.parametrize("softening", ["none", "plummer", "bspline"])
@pytest.mark.parametrize("frac", [0.1, 0.5, 0.9, 0.999])
def test_two_body_acceleration(softening, frac):
    rng = np.random.default_rng(7)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    r = frac * XR
    # place the pair straddling the periodic boundary in x
    x1 = np.array([0.995, 0.5, 0.5])
    x2 = (x1 + r * n) % 1.0
    acc, pairs = _two_body(x1, x2, softening)
    assert pairs == 2
    ref_b = _ref_bracket(r, XS, softening, EPS)
    # a_1 = -G m B(r) x_12 with x_12 = x_1 - x_2 (nearest image) = -r n
    expect = GM * ref_b * r * n
    np.testing.assert_allclose(acc[:, 0], expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())
    np.testing.assert_allclose(acc[:, 1], -expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())


def test_cutoff_is_strict():
    # a pair at distance exactly x_r does not interact (r^2 >= x_r^2 rejected)
    x1 = np.array([0.25, 0.5, 0.5])
    x2 = np.array([0.25 + 0.0625, 0.5, 0.5])  # dyadic: r = 1/16 exactly
    pos = np.array([x1, x2]).T.copy()
    _, pairs = oracle.sr_accel(pos, 0.0625 / 4.5, 0.0625, 1.0, "none", 0.0)
    assert pairs == 0
    _, pairs = oracle.sr_accel(pos, 0.0625 / 4.5, np.nextafter(0.0625, 1.0), 1.0, "none", 0.0)
    assert pairs == 2


def _mixed_positions(n, seed=3):
    full = synth.workload_positions(W)
    rng = np.random.default_rng(seed)
    idx = rng.choice(W.n, size=n, replace=False)
    return np.ascontiguousarray(full[:, idx])


@pytest.mark.parametrize("softening", ["none", "plummer", "bspline"])
def test_cell_list_vs_brute_force(softening):
    pos = _mixed_positions(4096)
    a1, p1 = oracle.sr_accel(pos, XS, XR, GM, softening, EPS)
    a2, p2 = oracle.sr_accel(pos, XS, XR, GM, softening, EPS, brute=True)
    assert p1 == p2
    np.testing.assert_allclose(a1, a2, rtol=0, atol=1e-13 * np.abs(a2).max())


def test_vs_explicit_periodic_images():
    # large cutoff relative to the box so that many pairs cross the boundary
    rng = np.random.default_rng(11)
    n = 300
    pos = rng.random((3, n))
    x_r = 0.2
    x_s = x_r / 4.5
    acc, pairs = oracle.sr_accel(pos, x_s, x_r, 1.0 / n, "bspline", 0.01)
    ref = np.zeros((3, n))
    count = 0
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], float)
    for i in range(n):
        d = pos[:, i][None, :, None] - (pos[None, :, :] + shifts[:, :, None])  # (27, 3, n)
        r2 = (d ** 2).sum(axis=1)
        r2[13, i] = np.inf  # the zero shift of j == i
        k, j = np.nonzero(r2 < x_r ** 2)
        count += len(j)
        r = np.sqrt(r2[k, j])
        b = oracle.bracket(r, x_s, "bspline", 0.01)
        ref[:, i] = -(1.0 / n) * (b[None, :] * d[k, :, j].T).sum(axis=1)
    assert pairs == count
    np.testing.assert_allclose(acc, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_newton_third_law():
    pos = synth.workload_positions(W)
    acc, _ = oracle.sr_accel(pos, XS, XR, GM, "bspline", EPS)
    assert np.abs(acc.sum(axis=1)).max() / np.abs(acc).sum() < 1e-12


def test_permutation_and_translation_invariance():
    pos = _mixed_positions(8192, seed=5)
    pos = np.floor(pos * 2.0 ** 30) / 2.0 ** 30  # dyadic grid: translation + wrap are exact
    acc, pairs = oracle.sr_accel(pos, XS, XR, GM, "bspline", EPS)
    perm = np.random.default_rng(2).permutation(pos.shape[1])
    acc_p, pairs_p = oracle.sr_accel(np.ascontiguousarray(pos[:, perm]), XS, XR, GM, "bspline", EPS)
    shift = np.array([[0.375], [0.8125], [0.0625]])
    acc_t, pairs_t = oracle.sr_accel((pos + shift) % 1.0, XS, XR, GM, "bspline", EPS)
    assert pairs == pairs_p == pairs_t
    scale = np.sqrt((acc ** 2).sum())
    assert np.sqrt(((acc[:, perm] - acc_p) ** 2).sum()) / scale < 1e-13
    assert np.sqrt(((acc - acc_t) ** 2).sum()) / scale < 1e-13


def test_inactive_rows_untouched_and_subset():
    pos = _mixed_positions(3000, seed=8)
    rung = synth.uniform_int8(3000, 99, 0, 8)
    out = np.full((3, 3000), 7.0)
    acc, _ = oracle.sr_accel(pos, XS, XR, GM, "bspline", EPS, rung=rung, rung_min=5, out=out)
    assert np.all(acc[:, rung < 5] == 7.0)
    full, _ = oracle.sr_accel(pos, XS, XR, GM, "bspline", EPS)
    np.testing.assert_array_equal(acc[:, rung >= 5], full[:, rung >= 5])
    recv = np.nonzero(rung >= 5)[0]
    sub, _ = oracle.sr_accel_subset(pos, recv, XS, XR, GM, "bspline", EPS)
    np.testing.assert_array_equal(sub, full[:, recv])


# --------------------------------------------------------------------------
# VJP
# --------------------------------------------------------------------------

@pytest.mark.parametrize("softening", ["none", "bspline"])
@pytest.mark.parametrize("partial", [False, True])
def test_vjp_vs_finite_differences(softening, partial):
    n = 1500
    pos = _mixed_positions(n, seed=21)
    rung = synth.uniform_int8(n, 5, 0, 8) if partial else None
    rmin = 4 if partial else 0
    abar = np.stack([synth.uniform(n, 31, k * n, -1, 1) for k in range(3)])
    xbar = oracle.sr_vjp(pos, abar, XS, XR, GM, softening, EPS, rung=rung, rung_min=rmin)
    # translation invariance: sum_k xbar_k = 0
    assert np.abs(xbar.sum(axis=1)).max() < 1e-10 * np.abs(xbar).sum()

    def loss(p):
        a, pairs = oracle.sr_accel(p, XS, XR, GM, softening, EPS, rung=rung, rung_min=rmin)
        return float((abar * a).sum()), pairs

    _, pairs0 = loss(pos)
    rng = np.random.default_rng(4)
    checked = 0
    for k in rng.choice(n, size=24, replace=False):
        d = int(rng.integers(3))
        h = 1e-7
        vals = {}
        ok = True
        for m in (-2, -1, 1, 2):
            p = pos.copy()
            p[d, k] += m * h
            vals[m], pc = loss(p)
            ok &= pc == pairs0
        if not ok:
            continue  # a pair crossed the cutoff: the loss jumps there
        fd = (8 * (vals[1] - vals[-1]) - (vals[2] - vals[-2])) / (12 * h)
        assert xbar[d, k] == pytest.approx(fd, rel=1e-5, abs=1e-8 * np.abs(xbar).max())
        checked += 1
    assert checked >= 16


# --------------------------------------------------------------------------
# integer decisions
# --------------------------------------------------------------------------

def test_rungs_vs_log2_definition():
    n = 20000
    dt, eta, eps = 0.013, 0.025, EPS
    mag = np.exp(synth.uniform(n, 3, 0, math.log(1e-3), math.log(1e5)))
    dirs = np.stack([synth.uniform(n, 3, (k + 1) * n, -1, 1) for k in range(3)])
    dirs /= np.linalg.norm(dirs, axis=0)
    acc = dirs * mag
    got, bad = oracle.rungs(acc, dt, eta, eps, 8)
    assert bad == 0
    arg = dt * np.sqrt(np.linalg.norm(acc, axis=0) / (2 * eta * eps))
    ref = np.clip(np.ceil(np.log2(arg)), 0, 7).astype(int)
    far = np.abs(np.log2(arg) - np.round(np.log2(arg))) > 1e-9
    assert far.sum() > 0.99 * n
    np.testing.assert_array_equal(got[far], ref[far])
    assert len(set(got.tolist())) == 8


def test_rungs_exact_boundaries():
    # dt = 1, eta = 1/4, eps = 2 give dt^2/(2 eta eps) = 1, so s = |a|^2
    ks = np.arange(0, 7)
    a = 4.0 ** ks  # dt sqrt(|a| / (2 eta eps)) = 2^k exactly  ->  rung k
    acc = np.zeros((3, len(ks) * 2 + 3))
    acc[0, : len(ks)] = a
    acc[0, len(ks): 2 * len(ks)] = np.nextafter(a, np.inf)  # just above -> k + 1
    acc[1, -3] = 0.0
    acc[2, -2] = 1e30
    acc[0, -1] = np.nan
    got, bad = oracle.rungs(acc, 1.0, 0.25, 2.0, 8)
    np.testing.assert_array_equal(got[: len(ks)], ks)
    np.testing.assert_array_equal(got[len(ks): 2 * len(ks)], np.minimum(ks + 1, 7))
    assert got[-3] == 0 and got[-2] == 7 and bad == 1
    got1, _ = oracle.rungs(acc[:, :-1], 1.0, 0.25, 2.0, 1)
    assert np.all(got1 == 0)


def test_subtile_ids():
    n_t, n_s = 11, 2
    m = n_t * n_s
    pos = _mixed_positions(5000, seed=9)
    edge = np.array([[0.0, 1 - 2.0 ** -53, 5 / m, np.nextafter(5 / m, 0)]] * 3)
    pos = np.concatenate([pos, edge], axis=1)
    ids = oracle.subtile_ids(pos, n_t, n_s)
    g = np.minimum(np.floor(pos * m).astype(np.int64), m - 1)
    tile = ((g[0] // n_s) * n_t + g[1] // n_s) * n_t + g[2] // n_s
    sub = ((g[0] % n_s) * n_s + g[1] % n_s) * n_s + g[2] % n_s
    np.testing.assert_array_equal(ids, tile * n_s ** 3 + sub)
    assert ids.min() >= 0 and ids.max() < m ** 3
    assert ids[-3] == ((m - 1) // n_s * n_t * n_t + (m - 1) // n_s * n_t + (m - 1) // n_s) * 8 + 7


# --------------------------------------------------------------------------
# kick / drift
# --------------------------------------------------------------------------

def test_kick_and_drift():
    n = 1000
    rng = np.random.default_rng(1)
    mom = rng.normal(size=(3, n))
    acc = rng.normal(size=(3, n))
    rung = synth.uniform_int8(n, 2, 0, 8)
    kf = 0.1 / 2.0 ** np.arange(8)
    q = oracle.kick(mom, acc, kf, rung=rung, rung_min=3)
    act = rung >= 3
    np.testing.assert_array_equal(q[:, ~act], mom[:, ~act])
    np.testing.assert_array_equal(q[:, act], mom[:, act] + acc[:, act] * kf[rung[act]])
    pos = rng.random((3, n))
    x = oracle.drift(pos, mom, 0.37)
    ref = pos + mom * 0.37
    ref = ref - np.floor(ref)
    np.testing.assert_array_equal(x, ref)
    assert x.min() >= 0 and x.max() < 1


# --------------------------------------------------------------------------
# the paper's printed rejection fractions (Section 2.1.3, "Subtiles")
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case,offset", [("same_tile", (0, 0, 0)), ("face_neighbour", (1, 0, 0)),
                                         ("edge_neighbour", (1, 1, 0)), ("corner_neighbour", (1, 1, 1))])
def test_rejection_fractions(golden, case, offset):
    rng = np.random.default_rng(12345)
    m = 2_000_000
    a = rng.random((m, 3))
    b = rng.random((m, 3)) + np.array(offset)
    rejected = ((a - b) ** 2).sum(axis=1) >= 1.0  # tiles of side x_r = 1
    frac = rejected.mean()
    ref = golden["tile_pair_rejection_fraction"]
    assert abs(frac - ref[case]) <= ref["printed_precision"]


# --------------------------------------------------------------------------
# rung-based leapfrog (Section 2.2.2)
# --------------------------------------------------------------------------

def test_rung_kicks_give_total_impulse_a_dt():
    """With a constant acceleration field, one synchronised global step kicks
    every particle by exactly a * dt, whatever its rung and its rung jumps
    (the kick sizes of the scheme always add up to the step)."""
    n, n_rung = 2000, 4
    dt, eta, eps = 0.1, 0.025, 0.01
    rng = np.random.default_rng(3)
    # accelerations spread over the rung ladder; initial rungs random, so that
    # particles jump up and down during the step
    mag = np.exp(rng.uniform(np.log(1e-2), np.log(1e4), n))
    acc = rng.normal(size=(3, n))
    acc *= mag / np.linalg.norm(acc, axis=0)
    rung = rng.integers(0, n_rung, n).astype(np.int8)
    state = np.zeros(n, dtype=np.int8)
    mom = np.zeros((3, n))
    mom = oracle.kick(mom, acc, [dt / 2.0 ** (l + 1) for l in range(n_rung)], rung=rung, rung_min=0)
    sub = 2 ** (n_rung - 1)
    jumps = 0
    for k in range(1, sub + 1):
        tz = 0
        while tz < n_rung - 1 and (k >> tz) & 1 == 0:
            tz += 1
        before = rung.copy()
        oracle.rung_kick(mom, acc, rung, state, n_rung - 1 - tz, k, n_rung, dt, eta, eps, sync=(k == sub))
        jumps += int((before != rung).sum())
    assert jumps > 100
    np.testing.assert_allclose(mom, acc * dt, rtol=1e-13, atol=0)
    assert np.all(state == 0)


def test_rung_leapfrog_single_rung_is_plain_kdk():
    """With one rung the scheme is the plain kick-drift-kick leapfrog."""
    pos = _mixed_positions(1500, seed=4)
    dt, eta = 0.02, 0.025
    p1, q1, rung, state, _ = oracle.rung_leapfrog(pos, np.zeros_like(pos), XS, XR, GM, "bspline", EPS, dt, eta,
                                                  n_rung=1, n_steps=3)
    # kick-drift-kick with the inner half kicks merged into one kick of dt
    x = pos.copy()
    q = np.zeros_like(pos)
    a, _ = oracle.sr_accel(x, XS, XR, GM, "bspline", EPS)
    q = oracle.kick(q, a, [dt / 2])
    for step in range(3):
        x = oracle.drift(x, q, dt)
        a, _ = oracle.sr_accel(x, XS, XR, GM, "bspline", EPS)
        q = oracle.kick(q, a, [dt if step < 2 else dt / 2])
    np.testing.assert_array_equal(p1, x)
    np.testing.assert_array_equal(q1, q)
    assert np.all(rung == 0)
    # Newton III: all particles on one rung conserve the total momentum
    assert np.abs(q1.sum(axis=1)).max() < 1e-12 * np.abs(q1).sum()


def test_rung_leapfrog_synchronised_every_step_is_unmerged_kdk():
    """Synchronising after every step turns the one-rung scheme into kick
    (dt/2) - drift (dt) - kick (dt/2) with nothing merged."""
    pos = _mixed_positions(1500, seed=6)
    dt, eta = 0.02, 0.025
    p1, q1, _, _, _ = oracle.rung_leapfrog(pos, np.zeros_like(pos), XS, XR, GM, "bspline", EPS, dt, eta,
                                           n_rung=1, n_steps=3, period=1)
    x = pos.copy()
    q = np.zeros_like(pos)
    a, _ = oracle.sr_accel(x, XS, XR, GM, "bspline", EPS)
    for step in range(3):
        q = oracle.kick(q, a, [dt / 2])
        x = oracle.drift(x, q, dt)
        a, _ = oracle.sr_accel(x, XS, XR, GM, "bspline", EPS)
        q = oracle.kick(q, a, [dt / 2])
    np.testing.assert_array_equal(p1, x)
    np.testing.assert_array_equal(q1, q)


def test_rung_leapfrog_with_long_range_is_kdk_of_the_total_force():
    """One rung, synchronised every step, with the mesh force: kick (dt/2) with the
    short- and then the long-range force, drift (dt), kick (dt/2) likewise."""
    from oracle import pm
    pos = _mixed_positions(1500, seed=9)
    dt, eta, n_phi = 0.02, 0.025, 32
    p1, q1, _, _, _ = oracle.rung_leapfrog(pos, np.zeros_like(pos), XS, XR, GM, "bspline", EPS, dt, eta,
                                           n_rung=1, n_steps=2, period=1, n_phi=n_phi)
    x = pos.copy()
    q = np.zeros_like(pos)
    for step in range(2):
        for half in range(2):
            if half == 1:
                x = oracle.drift(x, q, dt)
            a, _ = oracle.sr_accel(x, XS, XR, GM, "bspline", EPS)
            q = oracle.kick(q, a, [dt / 2])
            q = oracle.kick(q, pm.lr_accel(x, n_phi, XS, GM), [dt / 2])
    np.testing.assert_array_equal(p1, x)
    np.testing.assert_array_equal(q1, q)


def test_rung_jump_rules():
    """The time-stepping figure's jump rules: up by one rung at any kick (next kick
    1/2 of the finer rung's), down by one rung only at every other kick of the rung
    (next kick 3/4 of the coarser rung's)."""
    n_rung, dt, eta, eps = 4, 0.1, 0.025, 0.01
    q2 = (dt * dt / (2 * eta * eps)) ** 2
    big = np.sqrt(16.0 ** 3 * 4 / q2)      # Eq. rung gives rung 3 for |a| = big
    for k in range(1, 9):
        tz = 0
        while tz < n_rung - 1 and (k >> tz) & 1 == 0:
            tz += 1
        lmin = n_rung - 1 - tz
        for l in range(lmin, n_rung):
            for a_mag, want_dir in ((0.0, -1), (big, +1)):
                acc = np.zeros((3, 1))
                acc[0, 0] = a_mag
                mom = np.zeros((3, 1))
                rung = np.array([l], np.int8)
                state = np.array([0], np.int8)
                oracle.rung_kick(mom, acc, rung, state, lmin, k, n_rung, dt, eta, eps, False)
                if want_dir < 0:
                    odd = (k >> (n_rung - 1 - l)) & 1
                    if l > 0 and odd:
                        assert rung[0] == l - 1 and state[0] == 2
                    else:
                        assert rung[0] == l and state[0] == 0
                else:
                    if l < n_rung - 1:
                        assert rung[0] == l + 1 and state[0] == 1   # one rung at a time
                    else:
                        assert rung[0] == l and state[0] == 0
                # the kick itself used the rung held before the jump
                assert mom[0, 0] == pytest.approx(a_mag * dt / 2 ** l, rel=1e-15, abs=0)
