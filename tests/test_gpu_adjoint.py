"""Discrete adjoint on the GPU (lbpwfa_record / lbpwfa_adjoint_step).

  * FP64: J and dJ/d(alpha, sigma_z, sigma_r, profile) against the oracle's
    FP64 discrete adjoint on the same inputs (1D and 2D, both closures, open
    and periodic, from the driver's initial fields and from a random state),
    grids that span several tiles with a ragged tail.
  * FP64: against central finite differences of the GPU forward.
  * FP32 storage: against central finite differences of the FP64 path
    (bound 1e-4 relative).
  * Checkpointed recomputation gives the same gradient bit for bit as the
    kept tape; the state after the sweep is the end-of-window state.
  * The torch.autograd.Function returns the same gradient.
  * Error paths."""
import numpy as np
import pytest

import oracle as O
from tests import inputs

pytestmark = pytest.mark.gpu

lb = pytest.importorskip("paper_2309_04872_gb300.lbpwfa")


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lb.load_library()


def _cfg(dim, closure, boundary="open", **kw):
    if dim == 1:
        c = dict(dim=1, n=(301,), dx=0.05, courant=0.5, tau=0.53, closure=closure, dv=3, mu=1e-2, alpha=0.2,
                 sigma_z=0.6, z0=5.5, boundary=boundary, init_fields=False)
    else:
        c = dict(dim=2, n=(77, 21), dx=0.1, courant=0.5, tau=0.53, closure=closure, dv=3, mu=1e-2, alpha=0.2,
                 sigma_z=0.6, sigma_r=0.4, z0=4.0, boundary=boundary, init_fields=True)
    c.update(kw)
    return c


def _witness(c):
    # a node just behind the driver's path during the window
    iz = int(round((c["z0"] - 0.6) / c["dx"]))
    return (iz, c["n"][1] // 2 - 1) if c["dim"] == 2 else (iz,)


def _oracle_adjoint(c, N, state=None):
    o = O.Oracle(c)
    if state is not None:
        o.set_state(*state)
    w = _witness(c)
    flat = w[0] + (c["n"][0] * w[1] if c["dim"] == 2 else 0)
    return o.adjoint(N, flat)


def _gpu_adjoint(c, N, precision="fp64", C=0, state=None):
    with lb.Run(c, precision) as run:
        if state is not None:
            run.set_state(*state)
        run.record(N, C)
        run.step(N)
        return run.adjoint(_witness(c))


def _rel(a, b, scale):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / scale


def _random_state(c, seed):
    o = O.Oracle(c)
    base = o.rest_advected()
    amp = np.abs(base) * 0.05
    dim = c["dim"]
    if c["closure"] == "lec":
        amp[1:] = 0.02
    else:
        amp[2:2 + dim] = 0.02
        for j in range(o.K - 2 - dim):
            if base[2 + dim + j] == 0.0:
                amp[2 + dim + j] = 0.05 * c["mu"]
    f = inputs.random_populations(seed, o.K, o.Q, o.ncell, base, amp)
    E, B = inputs.random_fields(seed + 1, o.ncell, 0.02)
    return f, E, B


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("closure", ["lec", "warmc"])
@pytest.mark.parametrize("boundary", ["open", "periodic"])
def test_fp64_adjoint_matches_oracle(dim, closure, boundary):
    c = _cfg(dim, closure, boundary)
    N = 30
    Jo, go, _ = _oracle_adjoint(c, N)
    Jg, gg, _ = _gpu_adjoint(c, N)
    assert abs(Jg - Jo) <= 1e-12 * max(abs(Jo), 1e-3)
    names = 3 if dim == 2 else 2
    scale = np.max(np.abs(go[:names]))
    assert scale > 1e-4
    assert _rel(gg[:names], go[:names], scale) < 1e-9, (gg, go)


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_fp64_adjoint_from_random_state(dim, closure):
    c = _cfg(dim, closure)
    st = _random_state(c, 31 + dim)
    N = 25
    Jo, go, _ = _oracle_adjoint(c, N, st)
    Jg, gg, _ = _gpu_adjoint(c, N, state=st)
    assert abs(Jg - Jo) <= 1e-12 * max(abs(Jo), 1e-3)
    names = 3 if dim == 2 else 2
    scale = np.max(np.abs(go[:names]))
    assert scale > 1e-6
    assert _rel(gg[:names], go[:names], scale) < 1e-9, (gg, go)


# 2D grids at and around the size where the reverse step's gather gives the
# nodes within 3 of an edge their own blocks (both sides at least 7 nodes):
# a band that covers all but one row or column, one whose side columns are a
# single node wide, one just too narrow for it, and a one-tile grid.
SMALL_GRIDS = [(7, 7), (24, 7), (9, 8), (24, 6), (6, 13), (30, 4)]


@pytest.mark.parametrize("n", SMALL_GRIDS)
@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_fp64_adjoint_on_small_grids_matches_oracle(n, closure):
    c = _cfg(2, closure, n=n, z0=0.6 + 0.1 * (n[0] // 2), sigma_z=0.3, sigma_r=0.3)
    st = _random_state(c, 70 + n[0] + n[1])
    N = 12
    Jo, go, _ = _oracle_adjoint(c, N, st)
    Jg, gg, _ = _gpu_adjoint(c, N, state=st)
    assert abs(Jg - Jo) <= 1e-12 * max(abs(Jo), 1e-3)
    scale = np.max(np.abs(go[:3]))
    assert scale > 1e-8
    assert _rel(gg[:3], go[:3], scale) < 1e-9, (gg, go)
    # FP32 storage: the same gather in single precision, against FP64
    _, g32, _ = _gpu_adjoint(c, N, "fp32", state=st)
    assert _rel(g32[:3], gg[:3], scale) < 1e-4, (g32, gg)


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_fp64_profile_gradient_matches_oracle(closure):
    prof = 0.2 * np.exp(-0.5 * (np.arange(-24, 25) * 0.05 / 0.6) ** 2)
    c = _cfg(2, closure, profile=prof, profile_dz=0.05)
    N = 30
    Jo, go, gpo = _oracle_adjoint(c, N)
    Jg, gg, gpg = _gpu_adjoint(c, N)
    assert abs(Jg - Jo) <= 1e-12 * max(abs(Jo), 1e-3)
    scale = np.max(np.abs(gpo))
    assert scale > 1e-4
    assert _rel(gpg, gpo, scale) < 1e-9
    assert gg[0] == 0.0 and gg[1] == 0.0
    assert abs(gg[2] - go[2]) <= 1e-9 * max(abs(go[2]), 1e-12)


def _J_gpu(c, N, precision="fp64"):
    with lb.Run(c, precision) as run:
        run.step(N)
        ez = run.fields(lb.F_EZ)[0]
    w = _witness(c)
    return ez[w[0] + (c["n"][0] * w[1] if c["dim"] == 2 else 0)]


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_fp64_adjoint_matches_finite_differences(closure):
    c = _cfg(2, closure, n=(96, 40))
    N = 60
    _, g, _ = _gpu_adjoint(c, N)
    for k, name in enumerate(["alpha", "sigma_z", "sigma_r"]):
        h = 1e-4 * c[name]
        fd = (_J_gpu(dict(c, **{name: c[name] + h}), N) - _J_gpu(dict(c, **{name: c[name] - h}), N)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * max(abs(fd), 1e-12), (name, g[k], fd)


@pytest.mark.parametrize("prec", ["fp32", "fp32c"])
@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_fp32_adjoint_within_1e4_of_fp64_finite_differences(closure, prec):
    c = _cfg(2, closure, n=(128, 64), dx=0.05, mu=5e-3, alpha=0.1, sigma_z=1.0, sigma_r=0.5, z0=4.0)
    N = 300
    _, g, _ = _gpu_adjoint(c, N, prec, C=50)
    for k, name in enumerate(["alpha", "sigma_z", "sigma_r"]):
        h = 1e-4 * c[name]
        fd = (_J_gpu(dict(c, **{name: c[name] + h}), N) - _J_gpu(dict(c, **{name: c[name] - h}), N)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-4 * abs(fd), (name, g[k], fd)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32c"])
@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_checkpointed_equals_kept_tape(precision, closure):
    prof = 0.2 * np.exp(-0.5 * (np.arange(-24, 25) * 0.05 / 0.6) ** 2)
    c = _cfg(2, closure, profile=prof, profile_dz=0.05)
    N = 47
    J0, g0, p0 = _gpu_adjoint(c, N, precision, C=0)
    for C in (1, 10, 46):
        J1, g1, p1 = _gpu_adjoint(c, N, precision, C=C)
        assert J1 == J0
        assert np.array_equal(g1, g0) and np.array_equal(p1, p0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpointed_window_stepped_short_of_its_end(precision):
    """With checkpoints the forward writes the tape of the window's last two
    segments; a window stepped short of max_steps does not use it and
    recomputes every segment: the gradient is bitwise the kept tape's."""
    c = _cfg(2, "warmc")
    wit = _witness(c)
    with lb.Run(c, precision) as run:
        run.record(25, 0)
        run.step(25)
        J0, g0, _ = run.adjoint(wit)
    for cap, C in ((30, 7), (26, 12), (40, 9), (25, 12)):
        with lb.Run(c, precision) as run:
            run.record(cap, C)
            run.step(25)
            J1, g1, _ = run.adjoint(wit)
        assert J1 == J0 and np.array_equal(g1, g0), (cap, C, g1, g0)


def test_recording_armed_at_create_equals_lbpwfa_record():
    """record_tape / checkpoint_every in the parameters start the window at
    create, as lbpwfa_record does; the gradients are bitwise the same."""
    c = _cfg(2, "warmc")
    N = 23
    J0, g0, _ = _gpu_adjoint(c, N, "fp32", C=10)
    with lb.Run(dict(c, record_tape=N, checkpoint_every=10), "fp32") as run:
        run.step(N)
        wit = (c["n"][0] // 2, c["n"][1] // 2 - 1)
        J1, g1, _ = run.adjoint(wit)
    with lb.Run(c, "fp32") as run:
        run.record(N, 10)
        run.step(N)
        J2, g2, _ = run.adjoint(wit)
    assert J1 == J2 and np.array_equal(g1, g2)


def test_state_after_sweep_is_end_of_window():
    c = _cfg(2, "warmc")
    with lb.Run(c, "fp32") as a, lb.Run(c, "fp32") as b:
        a.record(20, 7)
        a.step(20)
        a.adjoint(_witness(c))
        b.step(20)
        assert a.info().step == 20
        fa, Ea, Ba = a.get_state()
        fb, Eb, Bb = b.get_state()
        assert np.array_equal(fa, fb) and np.array_equal(Ea, Eb) and np.array_equal(Ba, Bb)
        # both continue identically (previous-step values restored too)
        a.step(5)
        b.step(5)
        assert np.array_equal(a.get_state()[0], b.get_state()[0])


def test_recording_leaves_forward_bitwise_unchanged():
    c = _cfg(2, "warmc")
    with lb.Run(c, "fp32") as a, lb.Run(c, "fp32") as b:
        a.record(30, 0)
        a.step(30)
        b.step(30)
        assert np.array_equal(a.get_state()[0], b.get_state()[0])


def test_autograd_function_matches_adjoint():
    import torch

    from paper_2309_04872_gb300.wake_grad import witness_field
    c = _cfg(2, "lec")
    drv = torch.tensor([c["alpha"], c["sigma_z"], c["sigma_r"]], dtype=torch.float64, requires_grad=True)
    J = witness_field(drv, None, c, 30, _witness(c), precision="fp64", checkpoint_every=10)
    (2.0 * J).backward()
    Jg, g, _ = _gpu_adjoint(c, 30)
    assert float(J.detach()) == Jg
    assert np.allclose(drv.grad.numpy(), 2.0 * g, rtol=1e-14, atol=0)


def test_error_paths():
    c3 = dict(dim=3, n=(16, 8, 8), dx=0.1, courant=0.1, tau=0.53, closure="lec", dv=3, mu=1e-2, alpha=0.1,
              sigma_z=1.0, sigma_r=0.5, z0=0.5)
    with lb.Run(c3, "fp32") as r:
        with pytest.raises(lb.LbpwfaError):
            r.record(10)
    c = _cfg(2, "lec")
    with lb.Run(c, "fp16s") as r:
        with pytest.raises(lb.LbpwfaError):
            r.record(10)
    with lb.Run(c, "fp32") as r:
        with pytest.raises(lb.LbpwfaError):
            r.adjoint(_witness(c))           # nothing recorded
        r.record(3)
        r.step(3)
        with pytest.raises(lb.LbpwfaError):
            r.step(1)                        # window full
        with pytest.raises(lb.LbpwfaError):
            r.adjoint((c["n"][0], 0))        # witness outside the grid
        r.record(3)
        r.step(2)
        f, E, B = r.get_state()
        r.set_state(f, E, B)                 # replacing the state ends the recording
        with pytest.raises(lb.LbpwfaError):
            r.adjoint(_witness(c))


def test_adjoint_configuration_gradient_against_finite_differences():
    """The adjoint configuration itself: 2D 512 x 256 WARMC (mu = 5e-3,
    alpha = 0.1, sigma_z = 1, sigma_r = 0.5), 1000 steps recorded in FP32
    with checkpoints every 50; J = E_z on the axis 4 k_p^-1 behind the
    driver centre at the end.  dJ/d(alpha, sigma_z, sigma_r) within 1e-4 of
    FP64 central differences (h = 1e-4 relative)."""
    c = dict(dim=2, n=(512, 256), dx=0.05, courant=0.1, tau=0.53, closure="warmc", dv=3, mu=5e-3, alpha=0.1,
             sigma_z=1.0, sigma_r=0.5, z0=4.0, boundary="open", init_fields=True)
    N = 1000
    dt = 0.1 * 0.05
    w = (int(round((c["z0"] + (N - 0.5) * dt - 4.0) / c["dx"])), c["n"][1] // 2 - 1)

    def J(cfg, prec="fp64"):
        with lb.Run(cfg, prec) as run:
            run.step(N)
            return run.fields(lb.F_EZ)[0][w[0] + cfg["n"][0] * w[1]]

    with lb.Run(c, "fp32") as run:
        run.record(N, 50)
        run.step(N)
        _, g, _ = run.adjoint(w)
    for k, name in enumerate(["alpha", "sigma_z", "sigma_r"]):
        h = 1e-4 * c[name]
        fd = (J(dict(c, **{name: c[name] + h})) - J(dict(c, **{name: c[name] - h}))) / (2 * h)
        assert abs(g[k] - fd) <= 1e-4 * abs(fd), (name, g[k], fd)
