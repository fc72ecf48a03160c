"""Pins of the wake-fit diagnostic (the dispersion measurement of Sec. 6,
Fig. 3) on the CPU: an exact sinusoid, and the oracle's linear 1D wake
against the closed form of App. B."""
import numpy as np
import pytest

import oracle as O
from oracle import diagnostics as D


@pytest.mark.parametrize("k0,phi0", [(1.0234, 0.4), (0.8171, -2.9), (1.3303, 1.7)])
def test_fit_recovers_an_exact_sinusoid(k0, phi0):
    dx, zd = 0.02, 30.3
    z = np.arange(2000) * dx
    q = 0.7 * np.cos(k0 * (z - zd) + phi0) + 0.25
    r = D.line_fit(q, dx, zd, -25.0, -5.0, 0.5, 1.5, 201, offset=0.25)
    # the parabola through the grid minimum (step 0.005) leaves ~1e-5 in k
    assert abs(r["k"] - k0) < 1e-5
    assert abs(r["amplitude"] - 0.7) < 1e-5
    assert abs((r["phase"] - phi0 + np.pi) % (2 * np.pi) - np.pi) < 2e-4
    assert r["rms"] < 5e-5 and 1000 <= r["points"] <= 1001


def test_fit_of_the_linear_1d_wake_matches_the_closed_form():
    """1D LEC D = 1, mu = alpha = 1e-3 (App. B in 1D: k_w^2 = 1 / (1 - 1.5 mu),
    E_z amplitude sqrt(2 pi) alpha sigma_z exp(-k_w^2 sigma_z^2 / 2))."""
    cfg = dict(dim=1, n=(2048,), dx=40 / 2048, courant=0.5, tau=0.52, closure="lec", dv=1, mu=1e-3,
               alpha=1e-3, sigma_z=1.0, z0=-5.0, boundary="open")
    o = O.Oracle(cfg)
    N = int(round(39.0625 / o.dt))
    o.step(N)
    E, _ = o.fields()
    r = D.line_fit(E[0], cfg["dx"], cfg["z0"] + (N - 0.5) * o.dt, -25.0, -5.0, 0.5, 1.5, 201)
    kw = 1.0 / np.sqrt(1.0 - 1.5e-3)
    assert abs(r["k"] - kw) < 1e-4
    amp = np.sqrt(2 * np.pi) * 1e-3 * np.exp(-kw ** 2 / 2)
    assert abs(r["amplitude"] / amp - 1) < 3e-3


# ---------------------------------------------------------------------------
# Gauss's law residual on the dual cells (the library's lbpwfa_gauss_residual)
# ---------------------------------------------------------------------------
def _grid(cfg):
    n = (list(cfg["n"]) + [1, 1])[:3]
    nz, nx, ny = n
    dx = cfg["dx"]
    z = np.arange(nz) * dx
    return nz, nx, ny, dx, z


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_gauss_residual_vanishes_for_a_linear_field(dim):
    """E_z = c z (E_x = c' x, E_y = c'' y on their slots) has the discrete
    divergence c + c' + c'' exactly; with n = 1 - (c + c' + c'') and no
    driver the residual is round-off and sum rho^2 = cells (c + c' + c'')^2."""
    cfg = dict(dim=dim, n=(9, 7, 6)[:dim], dx=0.1, courant=0.1, tau=0.53, closure="lec", alpha=0.0, sigma_z=1.0, sigma_r=0.5, z0=0.0)
    nz, nx, ny, dx, z = _grid(cfg)
    c = (0.3, -0.2, 0.15)[:dim]
    shape = (ny, nx, nz)
    kk, jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(nz), indexing="ij")
    E = np.zeros((3,) + shape)
    E[0] = c[0] * ii * dx
    if dim >= 2:
        E[1] = c[1] * jj * dx
    if dim >= 3:
        E[2] = c[2] * kk * dx
    n = np.full(shape, 1.0 - sum(c))
    lo, hi = [0] * dim, [v - 1 for v in cfg["n"]]
    r2, rho2, cells = D.gauss_residual(cfg, n.ravel(), E.reshape(3, -1), 0.0, lo, hi)
    assert cells == np.prod(hi)
    assert r2 <= 1e-26 * cells
    assert abs(rho2 - cells * sum(c) ** 2) <= 1e-12 * rho2


def test_gauss_residual_cylindrical_divergence():
    """Axisymmetric: E_r = c r / 2 on its slots has (1/r) d_r (r E_r) = c
    exactly in the discrete form (r_{j+1}^2 - r_j^2 = 2 r_{j+1/2} dr)."""
    cfg = dict(dim=2, n=(8, 10), dx=0.1, courant=0.1, tau=0.53, closure="lec", alpha=0.0, sigma_z=1.0, sigma_r=0.5, z0=0.0,
               geometry="axisymmetric")
    nz, nx, ny, dx, z = _grid(cfg)
    jj, ii = np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij")
    c, cz = 0.4, -0.1
    E = np.zeros((3, nx, nz))
    E[0] = cz * ii * dx
    E[1] = 0.5 * c * jj * dx
    n = np.full((nx, nz), 1.0 - (c + cz))
    r2, rho2, cells = D.gauss_residual(cfg, n.ravel(), E.reshape(3, -1), 0.0, [0, 0], [nz - 1, nx - 1])
    assert r2 <= 1e-26 * cells
    assert abs(rho2 - cells * (c + cz) ** 2) <= 1e-12 * rho2


def test_gauss_residual_of_a_driven_run():
    """The definition reproduces the driven 2D Gauss check of the oracle
    (300 steps, tau = 0.505): the residual within 2% of |rho|."""
    cfg = dict(dim=2, n=(96, 48), dx=0.1, courant=0.1, tau=0.505, closure="lec", dv=3,
               mu=1e-3, alpha=0.05, sigma_z=0.8, sigma_r=0.6, z0=3.0, boundary="open", init_fields=True)
    o = O.Oracle(cfg)
    o.step(300)
    E, _ = o.fields()
    n = o.moments(1)[0]
    r2, rho2, cells = D.gauss_residual(cfg, n, E, (o.step_count - 0.5) * o.dt, [4, 4], [65, 43])
    assert cells == 61 * 39
    assert np.sqrt(r2 / rho2) < 0.02
