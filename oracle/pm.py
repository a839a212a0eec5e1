"""CPU oracle for the long-range (particle-mesh) half of the P3M gravity --
TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``: only tests,
``smoke()`` and the benchmark's CPU legs may use it).

Plain FP64 numpy, following the steps of Eq. p3m_gravity (long-range part) in
the paper's order (Sections 2.1.2 and 2.1.3):

  1. particles -> mesh:  rho_m = sum_j W_p((x_m - x_j) / L_phi), cell-centred
     mesh points x_m = L_phi (m + 1/2), W_p from Eqs. W_NGP ... W_PCS;
  2. forward FFT (numpy's unnormalised forward transform);
  3. multiply by the long-range kernel exp(-x_s^2 k^2) / k^2 and by two
     deconvolutions [W_p(L_phi k) / L_phi^3]^-2 = prod_d sinc^(-2p)(L_phi k_d / 2)
     (Eq. weight_fourier); the k = 0 mode is set to zero;
  4. inverse FFT, normalised so that F F^-1 is the identity;
  5. symmetric finite differences D_pd along each dimension, coefficients from
     the Lagrange form of Eq. symmetric_diff_general;
  6. mesh -> particle with the same W_p, and the factor 4 pi G m / L_phi^4
     (accelerations, i.e. the force of Eq. p3m_gravity divided by m).

numpy's FFT is a library primitive used as one step; nothing is fused or
reordered.  Pins (tests/test_oracle_pm.py): partition of unity and mass
conservation of the assignment, exactness of D_pd on polynomials, momentum
conservation, translation by whole cells, and agreement with the exact
reciprocal-space Ewald sum of the same kernel, with second-order convergence
in L_phi.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def weight_1d(x, p_i: int):
    """W_p(x) of Eqs. W_NGP, W_CIC, W_TSC, W_PCS (x in grid units)."""
    a = np.abs(np.asarray(x, dtype=np.float64))
    if p_i == 1:
        return np.where(a < 0.5, 1.0, 0.0)
    if p_i == 2:
        return np.where(a < 1.0, 1.0 - a, 0.0)
    if p_i == 3:
        return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, (2.0 * a - 3.0) ** 2 / 8.0, 0.0))
    if p_i == 4:
        return np.where(a < 1.0, (3.0 * a ** 3 - 6.0 * a * a + 4.0) / 6.0,
                        np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))
    raise ValueError("p_i must be 1, 2, 3 or 4")


def _stencil(pos, n_phi: int, p_i: int, box: float):
    """Per particle and dimension: the 6 candidate cells around it and their weights.

    Cells m with |x_m - x|/L_phi < 2 are floor(s) - 2 ... floor(s) + 3 with
    s = x / L_phi - 1/2; the weight is zero outside W_p's support."""
    L_phi = box / n_phi
    s = np.asarray(pos, dtype=np.float64) / L_phi - 0.5   # (3, n)
    base = np.floor(s).astype(np.int64)
    offs = np.arange(-2, 4)
    cells = base[:, :, None] + offs[None, None, :]          # (3, n, 6)
    if p_i == 1:
        # NGP: the cell holding x.  Eq. W_NGP's strict |x| < 1/2 leaves a particle exactly
        # on a cell face with no cell; it goes to the upper one, floor(s + 1/2).
        w = (cells == np.floor(s + 0.5).astype(np.int64)[:, :, None]).astype(np.float64)
    else:
        w = weight_1d(cells - s[:, :, None], p_i)           # W((x_m - x_j)/L_phi), W even
    return np.mod(cells, n_phi), w


def assign(pos, n_phi: int, p_i: int = 2, box: float = 1.0):
    """Step 1: rho_m = sum_j W_p((x_m - x_j)/L_phi) on an n_phi^3 grid (counts per cell)."""
    cells, w = _stencil(pos, n_phi, p_i, box)
    rho = np.zeros((n_phi, n_phi, n_phi))
    for a in range(6):
        for b in range(6):
            for c in range(6):
                wt = w[0, :, a] * w[1, :, b] * w[2, :, c]
                if not wt.any():
                    continue  # outside W_p's support for every particle
                np.add.at(rho, (cells[0, :, a], cells[1, :, b], cells[2, :, c]), wt)
    return rho


def interpolate(grid, pos, p_i: int = 2, box: float = 1.0):
    """Step 6 (without the prefactor): sum_m W_p((x_i - x_m)/L_phi) grid_m."""
    n_phi = grid.shape[0]
    cells, w = _stencil(pos, n_phi, p_i, box)
    out = np.zeros(cells.shape[1])
    for a in range(6):
        for b in range(6):
            for c in range(6):
                wt = w[0, :, a] * w[1, :, b] * w[2, :, c]
                if not wt.any():
                    continue
                out += wt * grid[cells[0, :, a], cells[1, :, b], cells[2, :, c]]
    return out


def difference_coefficients(p_d: int):
    """Eq. symmetric_diff_general: c[dm] = d/dxi prod_{dm' != dm} (xi - dm')/(dm - dm') at xi = 0,
    for dm = -p_d/2 ... p_d/2 (exact fractions)."""
    if p_d not in (2, 4, 6, 8):
        raise ValueError("p_d must be 2, 4, 6 or 8")
    h = p_d // 2
    pts = list(range(-h, h + 1))
    coef = {}
    for dm in pts:
        others = [q for q in pts if q != dm]
        denom = Fraction(1)
        for q in others:
            denom *= (dm - q)
        # derivative at 0 of prod (xi - q): sum over the dropped factor of prod of the rest at 0
        deriv = Fraction(0)
        for skip in others:
            term = Fraction(1)
            for q in others:
                if q != skip:
                    term *= (0 - q)
            deriv += term
        coef[dm] = deriv / denom
    return coef


def difference(grid, p_d: int, axis: int):
    """Step 5: D_pd along one axis of a periodic grid, in grid units."""
    out = np.zeros_like(grid)
    for dm, c in difference_coefficients(p_d).items():
        if c != 0:
            out += float(c) * np.roll(grid, -dm, axis=axis)   # grid[m + dm]
    return out


def wavenumbers(n_phi: int, box: float = 1.0):
    """k_h = 2 pi h / L for the full (x, y) and half (z) spectrum of a real FFT."""
    h_full = np.fft.fftfreq(n_phi, 1.0 / n_phi)
    h_half = np.fft.rfftfreq(n_phi, 1.0 / n_phi)
    two_pi_L = 2.0 * np.pi / box
    return two_pi_L * h_full, two_pi_L * h_full, two_pi_L * h_half


def potential_mesh(rho, x_s: float, p_i: int = 2, box: float = 1.0):
    """Steps 2-4: phi = F^-1 { [prod sinc^p_i(L_phi k_d/2)]^-2 exp(-x_s^2 k^2)/k^2 F rho }, k = 0 zeroed."""
    n_phi = rho.shape[0]
    L_phi = box / n_phi
    kx, ky, kz = wavenumbers(n_phi, box)
    rho_h = np.fft.rfftn(rho)
    k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2

    def sinc(t):
        return np.where(t == 0.0, 1.0, np.sin(t) / np.where(t == 0.0, 1.0, t))
    w_hat = (sinc(L_phi * kx / 2)[:, None, None] * sinc(L_phi * ky / 2)[None, :, None]
             * sinc(L_phi * kz / 2)[None, None, :]) ** p_i
    with np.errstate(divide="ignore", invalid="ignore"):
        kernel = np.exp(-x_s ** 2 * k2) / k2
    kernel[0, 0, 0] = 0.0
    phi_h = rho_h * kernel / w_hat ** 2
    phi_h[0, 0, 0] = 0.0
    return np.fft.irfftn(phi_h, s=rho.shape, axes=(0, 1, 2))


def lr_accel(pos, n_phi: int, x_s: float, G_m: float, p_i: int = 2, p_d: int = 4, box: float = 1.0):
    """Long-range accelerations of Eq. p3m_gravity (upper half, divided by m): 3 x n."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    L_phi = box / n_phi
    phi = potential_mesh(assign(pos, n_phi, p_i, box), x_s, p_i, box)
    pref = 4.0 * np.pi * G_m / L_phi ** 4
    acc = np.empty_like(pos)
    for d in range(3):
        acc[d] = pref * interpolate(difference(phi, p_d, d), pos, p_i, box)
    return acc


def ewald_lr_exact(pos, x_s: float, G_m: float, box: float = 1.0, k_cut_sigma: float = 7.0, targets=None):
    """Exact long-range force of the same kernel by direct summation over k-vectors:
    a_i = -(4 pi G m / L^3) sum_{k != 0} k exp(-x_s^2 k^2)/k^2 sum_j sin(k . (x_i - x_j)),
    truncated where x_s |k| > k_cut_sigma (relative size exp(-k_cut_sigma^2))."""
    pos = np.asarray(pos, dtype=np.float64)
    idx = np.arange(pos.shape[1]) if targets is None else np.asarray(targets)
    hmax = int(np.ceil(k_cut_sigma * box / (2.0 * np.pi * x_s)))
    hs = np.arange(-hmax, hmax + 1)
    out = np.zeros((3, len(idx)))
    two_pi_L = 2.0 * np.pi / box
    for hx in hs:
        for hy in hs:
            kx, ky = two_pi_L * hx, two_pi_L * hy
            kz = two_pi_L * hs
            k2 = kx * kx + ky * ky + kz * kz
            keep = (k2 > 0) & (x_s * np.sqrt(k2) <= k_cut_sigma)
            if not keep.any():
                continue
            kz, k2 = kz[keep], k2[keep]
            g = np.exp(-x_s ** 2 * k2) / k2                       # (nk,)
            # structure factor sum_j exp(i k.x_j), then sin(k.(x_i - x_j)) summed over j
            phase_j = kx * pos[0][:, None] + ky * pos[1][:, None] + kz[None, :] * pos[2][:, None]
            c, s = np.cos(phase_j).sum(axis=0), np.sin(phase_j).sum(axis=0)
            phase_i = kx * pos[0, idx][:, None] + ky * pos[1, idx][:, None] + kz[None, :] * pos[2, idx][:, None]
            # sum_j sin(k.x_i - k.x_j) = sin(k.x_i) C - cos(k.x_i) S
            t = (np.sin(phase_i) * c - np.cos(phase_i) * s) * g    # (ni, nk)
            out[0] += kx * t.sum(axis=1)
            out[1] += ky * t.sum(axis=1)
            out[2] += (t * kz[None, :]).sum(axis=1)
    return -(4.0 * np.pi * G_m / box ** 3) * out
