"""Pins of the oracle's axisymmetric (r, z) geometry (Sec. 2.2, App. A) and
of the Hankel-transform linear theory of App. B that pins it.

The quadrature of App. B is itself checked against two limits that reduce it
to closed forms: the cold plasma (n_1 separates into the 1D wake times the
bunch's transverse profile) and a bunch much wider than k_p^-1 (the 1D warm
wake with k_w^2 = a_e^2 / (1 - c_s^2)).  The oracle is then compared with
it on the axis and off it, and, for the warm WARMC, whose transverse response
the O(mu) theory does not capture, with the 3D Cartesian oracle (the same
scheme on a Cartesian grid, pinned on its own), which an axisymmetric
problem must reproduce."""
import numpy as np
import pytest

import oracle as O
from oracle import linear_theory as LT

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------------------
# the Hankel quadrature against its closed-form limits
# ---------------------------------------------------------------------------
def test_hankel_cold_limit_separates():
    """c_s = 0, a_e = a_b = 1: every w has K = 1, so n_1(r, xi) = n_1D(xi)
    exp(-r^2 / 2 sigma_r^2); far behind a Gaussian bunch n_1D = -sqrt(2 pi)
    alpha sigma_z exp(-sigma_z^2 / 2) sin(xi_d - xi)."""
    alpha, sz, sr, xd = 1e-3, 0.6, 0.5, 0.0
    xi = np.linspace(xd - 9.0, xd - 5.0, 41)
    r = np.array([0.0, 0.4, 0.8, 1.2])
    got = LT.hankel_n1(r, xi, alpha, sz, sr, xd, 0.0, 1.0, 1.0)
    amp = np.sqrt(2 * np.pi) * alpha * sz * np.exp(-sz ** 2 / 2)
    want = -amp * np.sin(xd - xi)[None, :] * np.exp(-r ** 2 / (2 * sr ** 2))[:, None]
    assert np.abs(got - want).max() <= 2e-4 * amp


def test_hankel_wide_bunch_is_the_1d_warm_wake():
    """sigma_r >> 1: the transform lives at w ~ 1/sigma_r, K(w) -> k_w =
    sqrt(a_e^2 / (1 - c_s^2)) and the axis sees the 1D warm wake
    -a_b^2 / (1 - c_s^2) sqrt(2 pi) alpha sigma_z exp(-k_w^2 sigma_z^2 / 2)
    sin(k_w (xi_d - xi)) / k_w."""
    alpha, sz, sr, xd = 1e-3, 0.6, 40.0, 0.0
    cs2, ae2, ab2 = LT.coefficients("lec", 0.04)
    kw = np.sqrt(ae2 / (1 - cs2))
    xi = np.linspace(xd - 9.0, xd - 5.0, 41)
    got = LT.hankel_n1([0.0], xi, alpha, sz, sr, xd, cs2, ae2, ab2)[0]
    amp = ab2 / (1 - cs2) * np.sqrt(2 * np.pi) * alpha * sz * np.exp(-kw ** 2 * sz ** 2 / 2) / kw
    want = -amp * np.sin(kw * (xd - xi))
    assert np.abs(got - want).max() <= 2e-3 * amp


# ---------------------------------------------------------------------------
# the axisymmetric oracle
# ---------------------------------------------------------------------------
def _axi(closure, mu, n, dx, courant, tau, **kw):
    cfg = dict(dim=2, n=n, dx=dx, courant=courant, tau=tau, closure=closure, dv=3, mu=mu,
               alpha=1e-3, sigma_z=0.6, sigma_r=0.5, z0=3.0, geometry="axisymmetric")
    cfg.update(kw)
    return O.Oracle(cfg)


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_axisymmetric_rest_state_is_a_fixed_point(closure):
    """No driver, no field: every 1/r term of App. A vanishes at rest (u_r =
    0, theta^{rr} = theta^{phi phi}, theta^{rz} = theta^{0r} = 0)."""
    o = _axi(closure, 0.04, (20, 12), 0.1, 0.2, 0.53, alpha=0.0, init_fields=False)
    o.step(30)
    A = o.advected()
    rest = o.rest_advected()
    for k in range(o.K):
        assert np.abs(A[k] - rest[k]).max() <= 1e-14 * max(1.0, abs(rest[k]))
    _, E, B = o.get_state()
    assert not E.any() and not B.any()


def _odd_sets(closure):
    # sets that change sign under r -> -r: n A_r; n lambda u_r, lambda theta^{rz}
    return {2} if closure == "lec" else {3, 7}


_MIRROR = [0, 1, 2, 4, 3, 7, 8, 5, 6]  # D2Q9 (z, r) velocity with r reversed


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_axisymmetric_axis_rules(closure):
    """After any step: the r = 0 node holds node 1's populations (Eq.
    open-bc) for the even sets and their mirror images (Eq. reflective-bc)
    for the odd ones; E_r and B_phi vanish on the axis."""
    nz, nr = 30, 10
    o = _axi(closure, 0.04, (nz, nr), 0.1, 0.2, 0.53, alpha=0.05, z0=1.5)
    o.step(7)
    f, E, B = o.get_state()
    f = f.reshape(o.K, o.Q, nr, nz)
    for k in range(o.K):
        for i in range(o.Q):
            src = _MIRROR[i] if k in _odd_sets(closure) else i
            assert np.array_equal(f[k, i, 0, 1:-1], f[k, src, 1, 1:-1]), (k, i)
    assert not E[1].reshape(nr, nz)[0].any()
    assert not B[2].reshape(nr, nz)[0].any()
    assert np.abs(E[1]).max() > 0 and np.abs(B[2]).max() > 0


def _wake_vs_hankel(o, closure, mu, t_end, window, radii):
    dx = o.cfg["dx"]
    N = int(round(t_end / o.dt))
    o.step(N)
    nr, nz = o.cfg["n"][1], o.cfg["n"][0]
    n1 = o.moments(1)[0].reshape(nr, nz) - 1.0
    xi = np.arange(nz) * dx - N * o.dt
    xd = o.cfg["z0"]
    sel = (xi > xd - window) & (xi < xd + 1.5)
    cs2, ae2, ab2 = LT.coefficients(closure, mu)
    th = LT.hankel_n1(radii, xi[sel], o.cfg["alpha"], o.cfg["sigma_z"], o.cfg["sigma_r"], xd, cs2, ae2, ab2)
    errs = []
    for m, r in enumerate(radii):
        j = int(round(r / dx))
        errs.append(np.linalg.norm(n1[j, sel] - th[m]) / np.linalg.norm(th[m]))
    return np.array(errs)


def test_axisymmetric_cold_lec_wake_matches_hankel():
    """Cold plasma (mu = 0), linear bunch: n - 1 at r = 0.3, 0.6, 1.0 over
    six plasma lengths behind the bunch within 1.5% (relative L2); on the
    axis within 6% (the r = 0 node copies node 1, whose 1/r terms are the
    nearest to the singular ones).  tau = 0.505 and C = 0.5 keep the LB
    diffusion kappa = (tau - 1/2) dx / 3C at 1.7e-4."""
    o = _axi("lec", 0.0, (400, 140), 0.05, 0.5, 0.505)
    e = _wake_vs_hankel(o, "lec", 0.0, 14.0, 6.0, [0.0, 0.3, 0.6, 1.0])
    assert e[1:].max() <= 0.015, e
    assert e[0] <= 0.06, e


def test_axisymmetric_cold_warmc_wake_matches_hankel():
    """The WARMC at mu = 1e-3 (nearly cold) against the same solution:
    within 3.5% off the axis on a grid twice as coarse."""
    o = _axi("warmc", 1e-3, (200, 70), 0.1, 0.5, 0.505)
    cs2 = LT.coefficients("warmc", 1e-3)[0]
    assert cs2 > 0
    e = _wake_vs_hankel(o, "warmc", 1e-3, 14.0, 6.0, [0.0, 0.3, 0.6, 1.0])
    assert e[1:].max() <= 0.035, e
    assert e[0] <= 0.06, e


def test_axisymmetric_warm_lec_wake_matches_hankel():
    """Warm LEC, mu = 0.04 (20 keV; c_s^2 = 5 mu / 3): within 4.5% over one
    plasma wavelength behind the bunch, where the O(mu) coefficients of App.
    B hold (further back their O(mu^2) error shifts the phase)."""
    o = _axi("lec", 0.04, (200, 70), 0.1, 0.15, 0.505)
    e = _wake_vs_hankel(o, "lec", 0.04, 14.0, 4.0, [0.0, 0.3, 0.6, 1.0])
    assert e.max() <= 0.045, e


def test_axisymmetric_warmc_matches_3d_cartesian():
    """Warm WARMC, mu = 0.04: the axisymmetric run against the 3D Cartesian
    oracle on the same spacing, time step and bunch.  The 3D grid puts the
    axis between nodes; its nodes at radius r are compared with the
    axisymmetric profile interpolated linearly in r, over the wake within 3
    plasma lengths of the bunch, for n - 1 and for lambda - lambda_0 (which
    the theta^{0r} / r term of the n lambda equation moves directly): within
    3% at r ~ 0.35, 0.65 and 5% at r ~ 1.05."""
    dx, C, tau, z0, nz, nt, T = 0.1, 0.3, 0.53, 2.5, 80, 36, 5.0
    base = dict(dx=dx, courant=C, tau=tau, closure="warmc", dv=3, mu=0.04, alpha=1e-3, sigma_z=0.6,
                sigma_r=0.5, z0=z0)
    a = O.Oracle(dict(base, dim=2, n=(nz, 24), geometry="axisymmetric"))
    c = O.Oracle(dict(base, dim=3, n=(nz, nt, nt)))
    N = int(round(T / a.dt))
    a.step(N)
    c.step(N)
    lam0 = a.rest_advected()[1]
    xi = np.arange(nz) * dx - N * a.dt
    sel = (xi > z0 - 3.0) & (xi < z0 + 1.5)
    for bit, rest in ((0, 1.0), (9, lam0)):
        na = a.moments(1 << bit)[0].reshape(24, nz) - rest
        n3 = c.moments(1 << bit)[0].reshape(nt, nt, nz) - rest
        iy = nt // 2
        for m, tol in ((3, 0.03), (6, 0.03), (10, 0.05)):
            ix = nt // 2 + m
            x, y = (ix - (nt - 1) / 2) * dx, (iy - (nt - 1) / 2) * dx
            r = np.hypot(x, y)
            j = int(r / dx)
            w = r / dx - j
            prof = (1 - w) * na[j] + w * na[j + 1]
            v3 = n3[iy, ix]
            e = np.linalg.norm(prof[sel] - v3[sel]) / np.linalg.norm(v3[sel])
            assert e <= tol, (bit, r, e)


def test_axisymmetric_uniform_field_drives_a_uniform_oscillation():
    """A uniform E_z in a uniform cold plasma at rest, no bunch: every node,
    the r = 0 node included, feels the same field (the E_z slot below the
    axis mirrors the one above it), u_r stays 0 so no 1/r term acts, and the
    plasma oscillates as a whole.  The outer wall's disturbance moves in by
    at most two nodes per step (one E and one B update), so after 8 steps
    u_z is the same at every node of the 20 rows nearest the axis, to
    round-off."""
    nz, nr = 12, 40
    o = _axi("lec", 0.0, (nz, nr), 0.1, 0.5, 0.53, alpha=0.0, init_fields=False)
    f, E, B = o.get_state()
    E = np.zeros_like(E)
    E[0] = 0.01
    o.set_state(None, E, None)
    o.step(8)
    uz = o.moments(2)[0].reshape(nr, nz)
    inner = uz[: nr - 20, 1:-1]
    assert abs(inner.mean()) > 1e-4
    assert np.abs(inner - inner.mean()).max() <= 1e-12 * abs(inner.mean())


@pytest.mark.parametrize("cs2", [0.02, 0.07, 0.12])
def test_cs2_fit_recovers_the_model_speed(cs2):
    """The c_s^2 fit (Fig. 6 diagnostic) on a map that the Hankel solution
    itself generated, at a_e^2 = 0.9: the generating value to 1e-3."""
    radii = np.arange(0, 16) * 0.1
    xi = np.arange(-6.0, 1.5, 0.1)
    n1 = LT.hankel_n1(radii, xi, 1e-3, 0.47, 0.47, 0.0, cs2, 0.9, 0.9, nw=1500)
    got, mis = LT.fit_cs2(n1, radii, xi, 1e-3, 0.47, 0.47, 0.0, 0.9, 0.9)
    assert abs(got - cs2) <= 1e-3 * cs2 + 2e-5
    assert mis < 1e-3
