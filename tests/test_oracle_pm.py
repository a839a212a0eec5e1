"""Pins of the particle-mesh oracle (oracle/pm.py) against facts that do not
come from the oracle itself: values and identities the paper prints, the
mathematics of interpolation and differencing, conservation laws, and an
independent Ewald summation whose own correctness is pinned by its
independence of the splitting scale."""
import numpy as np
import pytest

import oracle
from oracle import pm


# --------------------------------------------------------------------------
# weight functions (Eqs. W_NGP ... W_PCS, Eq. weight_fourier)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p_i", [1, 2, 3, 4])
def test_weights_at_nodes(golden, p_i):
    g = golden["weight_functions_at_nodes"]
    got = [float(pm.weight_1d(x, p_i)) for x in g["x"]]
    np.testing.assert_allclose(got, g[str(p_i)], rtol=0, atol=1e-15)


@pytest.mark.parametrize("p_i", [1, 2, 3, 4])
def test_weights_partition_of_unity(p_i):
    # the shapes are repeated convolutions of the one-cell top-hat: they sum to 1 over the grid
    s = np.random.default_rng(p_i).random(1000) * 7 - 3
    m = np.arange(-6, 8)
    total = pm.weight_1d(m[None, :] - s[:, None], p_i).sum(axis=1)
    np.testing.assert_allclose(total, 1.0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("p_i", [1, 2, 3, 4])
def test_weight_fourier_transform_is_sinc_power(p_i):
    # Eq. weight_fourier in one dimension: integral W_p(x) e^{-ikx} dx = sinc^p(k/2)
    x = np.linspace(-2.5, 2.5, 400001)
    w = pm.weight_1d(x, p_i)
    for k in (0.3, 1.0, 2.5, 4.0):
        ft = np.trapezoid(w * np.cos(k * x), x)
        # trapezoid rule: O(h) at NGP's jumps, O(h^2) for the continuous shapes
        assert ft == pytest.approx((np.sin(k / 2) / (k / 2)) ** p_i, abs=2e-5 if p_i == 1 else 2e-6)


@pytest.mark.parametrize("p_i", [1, 2, 3, 4])
def test_assignment_conserves_mass_and_cell_centre_cases(p_i):
    rng = np.random.default_rng(5)
    pos = rng.random((3, 500))
    rho = pm.assign(pos, 16, p_i)
    assert rho.sum() == pytest.approx(500.0, rel=1e-13)
    # a particle at a cell centre: the 1-D weights at offsets 0, +-1 (cell units) factorise
    c = np.array([[(5 + 0.5) / 16], [(9 + 0.5) / 16], [(0 + 0.5) / 16]])
    rho = pm.assign(c, 16, p_i)
    w0, w1 = pm.weight_1d(0.0, p_i), pm.weight_1d(1.0, p_i)
    assert rho[5, 9, 0] == pytest.approx(w0 ** 3, abs=1e-15)
    assert rho[6, 9, 0] == pytest.approx(w1 * w0 * w0, abs=1e-15)
    assert rho[5, 9, 15] == pytest.approx(w0 * w0 * w1, abs=1e-15)  # periodic wrap in z


# --------------------------------------------------------------------------
# symmetric differences (Eqs. symmetric_diff_general ... symmetric_diff_8)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p_d", [2, 4, 6, 8])
def test_difference_weights_match_printed(golden, p_d):
    g = golden["symmetric_differences"][str(p_d)]
    c = pm.difference_coefficients(p_d)
    assert c[0] == 0
    for dm, wgt in enumerate(g["weights"], start=1):
        assert c[dm] * g["denominator"] == wgt
        assert c[-dm] == -c[dm]


@pytest.mark.parametrize("p_d", [2, 4, 6, 8])
def test_difference_exact_on_polynomials(p_d):
    # a symmetric p_d-point derivative is exact for polynomials up to degree p_d
    n = 64
    m = np.arange(n, dtype=np.float64)
    for deg in range(p_d + 1):
        f = ((m - 30.3) / 7.0) ** deg
        grid = np.broadcast_to(f[:, None, None], (n, 2, 2)).copy()
        d = pm.difference(grid, p_d, 0)[:, 0, 0]
        exact = deg * ((m - 30.3) / 7.0) ** max(deg - 1, 0) / 7.0 if deg else 0 * m
        inner = slice(p_d, n - p_d)  # away from the periodic seam
        np.testing.assert_allclose(d[inner], np.asarray(exact)[inner], rtol=1e-11, atol=1e-11)
    # and not exact one degree higher
    f = ((m - 30.3) / 7.0) ** (p_d + 1)
    grid = np.broadcast_to(f[:, None, None], (n, 2, 2)).copy()
    d = pm.difference(grid, p_d, 0)[:, 0, 0]
    exact = (p_d + 1) * ((m - 30.3) / 7.0) ** p_d / 7.0
    assert np.abs(d - exact)[p_d:n - p_d].max() > 1e-6


# --------------------------------------------------------------------------
# the independent Ewald reference
# --------------------------------------------------------------------------

def test_ewald_total_force_independent_of_split_scale():
    # short-range (pinned oracle, cut where erfc < 1e-16) + reciprocal sum is the full
    # periodic Newtonian force, whatever x_s: a wrong sign or factor in the reciprocal
    # sum would make the two splits disagree
    rng = np.random.default_rng(2)
    n = 12
    pos = rng.random((3, n))
    tot = []
    for x_s in (0.02, 0.016):
        sr, _ = oracle.sr_accel(pos, x_s, 0.25, 1.0 / n, "none", 0.0)
        tot.append(sr + pm.ewald_lr_exact(pos, x_s, 1.0 / n))
    assert np.abs(tot[0] - tot[1]).max() <= 1e-12 * np.abs(tot[0]).max()


# --------------------------------------------------------------------------
# the PM long-range force
# --------------------------------------------------------------------------

def _rel_rms(a, ref):
    return float(np.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum()))


@pytest.fixture(scope="module")
def lr_case():
    rng = np.random.default_rng(11)
    n = 64
    pos = rng.random((3, n))
    n_phi = 32
    x_s = 1.25 / n_phi  # Eq. p3m_parameters
    return pos, n_phi, x_s, pm.ewald_lr_exact(pos, x_s, 1.0 / n)


@pytest.mark.parametrize("p_i,p_d,tol", [(2, 4, 0.02), (2, 2, 0.05), (3, 4, 0.008), (4, 4, 0.007)])
def test_pm_against_exact_long_range(lr_case, p_i, p_d, tol):
    """At the paper's x_s = 1.25 L_phi the mesh force of the same kernel agrees with
    the exact reciprocal sum to the percent level (the P3M discretisation error;
    without the deconvolutions it is ~6% for CIC)."""
    pos, n_phi, x_s, ex = lr_case
    a = pm.lr_accel(pos, n_phi, x_s, 1.0 / pos.shape[1], p_i=p_i, p_d=p_d)
    assert _rel_rms(a, ex) <= tol


def test_pm_converges_at_second_order(lr_case):
    # fixed x_s, finer mesh: the CIC + D_4 error falls ~4x per halving of L_phi
    pos, n_phi, x_s, ex = lr_case
    errs = [_rel_rms(pm.lr_accel(pos, m, x_s, 1.0 / pos.shape[1]), ex) for m in (32, 64, 128)]
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[2] < 2e-3


def test_pm_momentum_conservation(lr_case):
    # same W for assignment and interpolation, antisymmetric D, even kernel: sum_i a_i = 0
    pos, n_phi, x_s, _ = lr_case
    for p_i, p_d in ((1, 2), (2, 4), (3, 6), (4, 8)):
        a = pm.lr_accel(pos, n_phi, x_s, 1.0 / pos.shape[1], p_i=p_i, p_d=p_d)
        assert np.abs(a.sum(axis=1)).max() <= 1e-13 * np.abs(a).sum()


def test_pm_translation_by_whole_cells(lr_case):
    pos, n_phi, x_s, _ = lr_case
    a = pm.lr_accel(pos, n_phi, x_s, 1.0 / pos.shape[1])
    shifted = (pos + np.array([[3.0], [-5.0], [11.0]]) / n_phi) % 1.0
    b = pm.lr_accel(shifted, n_phi, x_s, 1.0 / pos.shape[1])
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * np.abs(a).max())


def test_pm_poisson_kernel_two_particles_attract():
    # plain PM (x_s = 0, kernel 1/k^2): two particles attract along their separation with
    # equal and opposite accelerations, approaching the periodic (Ewald) force once they
    # are many cells apart (here 20 cells)
    pos = np.array([[0.40, 0.48], [0.5, 0.5], [0.5, 0.5]])
    a = pm.lr_accel(pos, 256, 0.0, 0.5, p_i=2, p_d=2)
    assert a[0, 0] > 0 and a[0, 1] < 0
    assert a[0, 0] == pytest.approx(-a[0, 1], rel=1e-12)
    ew = oracle.sr_accel(pos, 0.02, 0.25, 0.5, "none", 0.0)[0] + pm.ewald_lr_exact(pos, 0.02, 0.5)
    assert a[0, 0] == pytest.approx(ew[0, 0], rel=0.03)


def test_ngp_particle_on_a_cell_face_goes_to_the_upper_cell():
    # reading of Eq. W_NGP's strict inequality: the cell holding x is floor(x / L_phi)
    pos = np.array([[4.0 / 16], [0.5 / 16], [0.5 / 16]])
    rho = pm.assign(pos, 16, 1)
    assert rho.sum() == 1.0 and rho[4, 0, 0] == 1.0


def test_p3m_split_reproduces_the_periodic_force():
    """The two halves of Eq. p3m_gravity together (oracle short-range sum cut at
    x_r = 4.5 x_s, mesh long-range force at x_s = 1.25 L_phi with CIC and D_4)
    give the full periodic force of an Ewald sum to a few tenths of a percent."""
    rng = np.random.default_rng(8)
    n = 128
    pos = rng.random((3, n))
    n_phi = 32
    x_s = 1.25 / n_phi
    sr, _ = oracle.sr_accel(pos, x_s, 4.5 * x_s, 1.0 / n, "none", 0.0)
    lr = pm.lr_accel(pos, n_phi, x_s, 1.0 / n)
    exact = oracle.sr_accel(pos, 0.02, 0.25, 1.0 / n, "none", 0.0)[0] + pm.ewald_lr_exact(pos, 0.02, 1.0 / n)
    assert _rel_rms(sr + lr, exact) <= 5e-3
    # each half alone is far off: the split really is a split
    assert _rel_rms(sr, exact) > 0.05 and _rel_rms(lr, exact) > 0.05
