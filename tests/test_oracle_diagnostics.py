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
