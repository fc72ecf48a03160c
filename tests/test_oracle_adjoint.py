"""Pins of the oracle's discrete adjoint against central finite differences
of the forward oracle (itself pinned in test_oracle_pins.py).

J = E_z at one slot after N steps.  Gradients with respect to the driver
parameters (alpha, sigma_z, sigma_r; the sampled-profile values) and, along
random directions, with respect to the whole starting state (f, E, B).  The
finite differences are central with a relative step of 1e-5, whose
truncation and round-off errors sit near 1e-10 relative; the bound is 1e-7.
A dropped term, a wrong sign or a transposed stencil shows up at O(1)."""
import numpy as np
import pytest

import oracle as O
from tests import inputs

N = 12


def _cfg(dim, closure, boundary="open", **kw):
    c = dict(dim=dim, n=[24, 10] if dim == 2 else [40], dx=0.25, courant=0.5, tau=0.6,
             closure=closure, dv=3, mu=0.02, alpha=0.3, sigma_z=0.7, sigma_r=0.6, z0=3.0,
             boundary=boundary, init_fields=dim == 2)
    c.update(kw)
    return c


def _witness(c):
    nz = c["n"][0]
    return nz * (c["n"][1] // 2 - 1 if c["dim"] == 2 else 0) + 8


def _J(c, state=None):
    o = O.Oracle(c)
    if state is not None:
        o.set_state(*state)
    o.step(N)
    _, E, _ = o.get_state()
    return E.flat[_witness(c)]


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-14)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("closure", ["lec", "warmc"])
@pytest.mark.parametrize("boundary", ["open", "periodic"])
def test_adjoint_driver_parameters(dim, closure, boundary):
    c = _cfg(dim, closure, boundary)
    J, g3, _ = O.Oracle(c).adjoint(N, _witness(c))
    assert J == _J(c)
    names = ["alpha", "sigma_z", "sigma_r"][: 3 if dim == 2 else 2]
    for k, name in enumerate(names):
        h = 1e-5 * c[name]
        fd = (_J(dict(c, **{name: c[name] + h})) - _J(dict(c, **{name: c[name] - h}))) / (2 * h)
        assert abs(fd) > 1e-6, name
        assert _rel(g3[k], fd) < 1e-7, (name, g3[k], fd)


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_adjoint_profile_samples(closure):
    prof = 0.3 * np.exp(-0.5 * (np.arange(-12, 13) * 0.25 / 0.7) ** 2)
    c = _cfg(2, closure, profile=prof, profile_dz=0.25)
    J, g3, gp = O.Oracle(c).adjoint(N, _witness(c))
    assert gp.shape == prof.shape
    assert g3[0] == 0.0 and g3[1] == 0.0
    # samples the driver never reaches have zero sensitivity; the others are
    # checked against an absolute bound on the scale of the largest one
    h = 1e-4
    scale = np.max(np.abs(gp))
    assert scale > 1e-3
    for j in range(0, prof.size, 2):
        pp, pm = prof.copy(), prof.copy()
        pp[j] += h
        pm[j] -= h
        fd = (_J(dict(c, profile=pp)) - _J(dict(c, profile=pm))) / (2 * h)
        assert abs(gp[j] - fd) < 1e-7 * scale, (j, gp[j], fd)
    hs = 1e-5 * c["sigma_r"]
    fd = (_J(dict(c, sigma_r=c["sigma_r"] + hs)) - _J(dict(c, sigma_r=c["sigma_r"] - hs))) / (2 * hs)
    assert _rel(g3[2], fd) < 1e-7


def _random_start(o, seed):
    base = o.rest_advected()
    amp = np.abs(base) * 0.05
    dim = o.cfg["dim"]
    if o.cfg["closure"] == "lec":
        amp[1:] = 0.02
    else:
        amp[2:2 + dim] = 0.02
        for j in range(o.K - 2 - dim):
            if base[2 + dim + j] == 0.0:
                amp[2 + dim + j] = 0.05 * o.cfg["mu"]
    f = inputs.random_populations(seed, o.K, o.Q, o.ncell, base, amp)
    E, B = inputs.random_fields(seed + 1, o.ncell, 0.05)
    # the state the oracle actually holds (boundary nodes copy the bulk,
    # wall slots of E are zero)
    o.set_state(f, E, B)
    return o.get_state()


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("closure", ["lec", "warmc"])
@pytest.mark.parametrize("boundary", ["open", "periodic"])
def test_adjoint_starting_state(dim, closure, boundary):
    c = _cfg(dim, closure, boundary)
    o = O.Oracle(c)
    f0, E0, B0 = _random_start(o, 11 + dim)
    J, _, _, (lf, lE, lB) = o.adjoint(N, _witness(c), state_grad=True)
    assert J == _J(c, (f0, E0, B0))
    for seed in (1, 2):
        g = inputs.rng(100 + seed)
        o2 = O.Oracle(c)
        o2.set_state(g.standard_normal(f0.shape) * 1e-2, g.standard_normal(E0.shape) * 1e-2,
                     g.standard_normal(B0.shape) * 1e-2)
        df, dE, dB = o2.get_state()  # a direction the state can take
        h = 1e-5
        Jp = _J(c, (f0 + h * df, E0 + h * dE, B0 + h * dB))
        Jm = _J(c, (f0 - h * df, E0 - h * dE, B0 - h * dB))
        fd = (Jp - Jm) / (2 * h)
        ad = float(np.dot(lf, df.ravel()) + np.sum(lE * dE) + np.sum(lB * dB))
        assert abs(fd) > 1e-8
        assert _rel(ad, fd) < 1e-7, (ad, fd)


def test_adjoint_linear_in_alpha_limit():
    """At alpha -> 0 the plasma response is linear in the driver, so
    J ~ alpha dJ/dalpha (a closed form of the sensitivity's size)."""
    c = _cfg(2, "lec", alpha=1e-6)
    J, g3, _ = O.Oracle(c).adjoint(N, _witness(c))
    assert _rel(c["alpha"] * g3[0], J) < 1e-5
