"""Parity of the axisymmetric (z, r) CUDA path with the FP64 oracle (Sec. 2.2
and App. A: the r = 0 boundary node with Eq. open-bc / reflective-bc, the
1/r source terms, the cylindrical Yee curl), through the C ABI, on the same
seeded inputs.  Bounds as in the Cartesian parity tests (tests/parity.py):
FP64 to 1e-12 of the perturbation from rest plus the oracle's own
representation floor, in the L2 norm and element by element; FP32 and FP16S
storage to the unit round-off of the stored deviations times the
field-source amplification."""
import numpy as np
import pytest

import oracle as O
from tests import inputs
from tests import parity as P
from tests.test_gpu_parity import _compare

pytestmark = pytest.mark.gpu

lb = pytest.importorskip("paper_2309_04872_gb300.lbpwfa")


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lb.load_library()


def _cfg(closure, n=(77, 45), **kw):
    cfg = dict(dim=2, n=n, dx=0.05, courant=0.1, tau=0.53, closure=closure, dv=3, mu=1e-2, alpha=0.2,
               sigma_z=0.6, sigma_r=0.3, z0=0.3 * n[0] * 0.05, boundary="open", init_fields=True,
               geometry="axisymmetric")
    cfg.update(kw)
    return cfg


def _random_state(o, seed, mu):
    base = o.rest_advected()
    amp = np.abs(base) * 0.05
    if o.cfg["closure"] == "lec":
        amp[1:] = 0.02
    else:
        amp[2:4] = 0.02
        for j in range(o.K - 4):
            if base[4 + j] == 0.0:
                amp[4 + j] = 0.05 * mu
    f = inputs.random_populations(seed, o.K, o.Q, o.ncell, base, amp)
    E, B = inputs.random_fields(seed + 1, o.ncell, 0.01)
    return f, E, B


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_axi_fp64_random_state_parity(closure):
    """Random state (every set perturbed, odd ones included), 25 steps: the
    advected scalars, fields, populations (the axis node's mirrored sets as
    exported) and every decoded moment to 1e-12."""
    cfg = _cfg(closure)
    orc = O.Oracle(cfg)
    f, E, B = _random_state(orc, 321, cfg["mu"])
    orc.set_state(f, E, B)
    with lb.Run(cfg, "fp64") as run:
        run.set_state(f, E, B)
        assert run.info().kernel_variant == 5
        _compare(run, orc, 0, "t0")
        orc.step(25)
        run.step(25)
        _compare(run, orc, 25, "t25")
        f_g, _, _ = run.get_state()
        f_o, _, _ = orc.get_state()
        P.check_populations64(f_g, f_o, P.rest_populations(O, cfg), 25, orc.Q, "populations", P.rest_scale(orc))
        m_g = run.moments(0x3FFFF)
        m_o = orc.moments(0x3FFFF)
        m_rest = P.rest_moments(O, cfg, 0x3FFFF)
        for b in range(18):
            if np.abs(m_o[b]).max() == 0:
                assert np.abs(m_g[b]).max() == 0, b
                continue
            P.check64(m_g[b], m_o[b], m_rest[b], 25, orc.Q, f"moment bit {b}", P.rest_scale(orc))


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_axi_fp64_driver_from_rest_parity(closure):
    """The driver's initial v -> c field in (z, r) and 150 steps from rest."""
    cfg = _cfg(closure, mu=0.04)
    orc = O.Oracle(cfg)
    with lb.Run(cfg, "fp64") as run:
        _compare(run, orc, 0, "t0")
        orc.step(150)
        run.step(150)
        _compare(run, orc, 150, "t150")


@pytest.mark.parametrize("closure", ["lec", "warmc"])
@pytest.mark.parametrize("prec,tol,floor", [("fp32", 1e-4, 1e-7), ("fp16s", 2e-2, 1e-4)])
def test_axi_reduced_precision_parity(closure, prec, tol, floor):
    cfg = _cfg(closure, mu=0.04)
    orc = O.Oracle(cfg)
    orc.step(100)
    with lb.Run(cfg, prec) as run:
        run.step(100)
        _compare(run, orc, 100, prec, tol=tol, floor=floor)


def test_axi_variant_one_is_the_same_kernel():
    cfg = _cfg("warmc")
    outs = []
    for v in (0, 1):
        with lb.Run(cfg, "fp32", variant=v) as run:
            assert run.info().kernel_variant == 5
            run.step(20)
            outs.append(run.get_state())
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp32", "fp16s", "fp64"])
@pytest.mark.parametrize("n", [(131, 37), (700, 300)])
def test_axi_lec_persistent_and_plain_agree(prec, n):
    """Axisymmetric LEC on the persistent TMA kernel (automatic in FP32 and
    FP16S; variant 3) and on the plain kernel (variant 1): the same step, to
    the storage precision's round-off of the largest deviation from rest
    (700 x 300 has more tiles than persistent CTAs, so boxes are refilled)."""
    cfg = _cfg("lec", n=n, mu=0.04)
    orc = O.Oracle(cfg)
    f, E, B = _random_state(orc, 5 + n[0], cfg["mu"])
    outs = []
    for v in (3, 1):
        with lb.Run(cfg, prec, variant=v) as run:
            assert run.info().kernel_variant == (3 if v == 3 else 5)
            run.set_state(f, E, B)
            run.step(17)
            outs.append((run.advected(), run.get_state()[1]))
    if prec != "fp64":
        with lb.Run(cfg, prec) as run:
            assert run.info().kernel_variant == 3
    rest = orc.rest_advected()
    tol = 1e-12 if prec == "fp64" else 1e-5
    for k in range(orc.K):
        d = np.abs(outs[0][0][k] - outs[1][0][k]).max()
        assert d <= tol * max(np.abs(outs[1][0][k] - rest[k]).max(), 1e-30), k
    dE = np.abs(outs[0][1] - outs[1][1]).max()
    assert dE <= tol * np.abs(outs[1][1]).max()


def test_axi_rejects_the_adjoint():
    cfg = _cfg("lec")
    with lb.Run(cfg, "fp64") as run:
        with pytest.raises(Exception):
            run.record(10)


def test_axi_fp64_paper_grid_matches_oracle():
    """The 3D3V axisymmetric grid of Sec. 6 (L_r = 6, L_z = 30 at dz = dr =
    0.01: 3000 x 600 nodes), WARMC mu = 0.04, sigma_z = sigma_r = 25 um at
    n_i = 1e16 cm^-3 (0.47 k_p^-1), Q~ = 0.5 (Eq. Qtilde with D = 3:
    alpha = Q~ / ((2 pi)^{3/2} sigma_z sigma_r^2)), C = 0.1, tau = 0.53: the
    bench's grid and launch configuration, compared in full after 8 steps."""
    sz, sr = 0.47, 0.47
    alpha = 0.5 / ((2 * np.pi) ** 1.5 * sz * sr * sr)
    cfg = dict(dim=2, n=(3000, 600), dx=0.01, courant=0.1, tau=0.53, closure="warmc", dv=3, mu=0.04,
               alpha=alpha, sigma_z=sz, sigma_r=sr, z0=4.0, boundary="open", init_fields=True,
               geometry="axisymmetric")
    orc = O.Oracle(cfg)
    orc.step(8)
    with lb.Run(cfg, "fp64") as run:
        run.step(8)
        _compare(run, orc, 8, "axi paper grid")


@pytest.mark.parametrize("closure", ["lec", "warmc"])
@pytest.mark.parametrize("n", [(3, 3), (3, 40), (40, 3), (33, 9), (65, 17)])
def test_axi_edge_sizes(closure, n):
    """Grids down to 3 x 3 (every node a boundary node, the axis node's bulk
    node also the outer boundary's), single and ragged tiles, from a random
    state: FP64 parity after 9 steps."""
    cfg = _cfg(closure, n=n)
    orc = O.Oracle(cfg)
    f, E, B = _random_state(orc, 77 + n[0] + n[1], cfg["mu"])
    orc.set_state(f, E, B)
    with lb.Run(cfg, "fp64") as run:
        run.set_state(f, E, B)
        run.step(0)
        orc.step(9)
        run.step(9)
        _compare(run, orc, 9, f"axi {n}")


def test_axi_checkpoint_roundtrip_and_geometry_check(tmp_path):
    cfg = _cfg("warmc")
    path = str(tmp_path / "axi.ckpt")
    with lb.Run(cfg, "fp32") as run:
        run.step(20)
        run.save(path)
        run.step(15)
        want = run.get_state()
    with lb.Run(cfg, "fp32") as run:
        run.load(path)
        run.step(15)
        got = run.get_state()
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    # the same grid in Cartesian geometry refuses the file
    with lb.Run(dict(cfg, geometry="cartesian"), "fp32") as run:
        with pytest.raises(lb.LbpwfaError):
            run.load(path)


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_axi_reduced_precision_wake_after_2000_steps(closure):
    """The precision targets on the axisymmetric path: relative L2 error of
    n - 1 and E_z against the FP64 path after 2000 steps, FP32 storage within
    1e-6, FP16-shifted storage within 1e-3 (600 x 120 nodes, dz = dr = 0.05,
    mu = 0.04, Q~ = 0.5 bunch of sigma_z = sigma_r = 0.47)."""
    alpha = 0.5 / ((2 * np.pi) ** 1.5 * 0.47 ** 3)
    cfg = _cfg(closure, n=(600, 120), mu=0.04, alpha=alpha, sigma_z=0.47, sigma_r=0.47, z0=3.0)
    out = {}
    for prec in ("fp64", "fp32", "fp16s"):
        with lb.Run(cfg, prec) as run:
            run.step(2000)
            out[prec] = (run.moments(lb.M_N)[0] - 1.0, run.fields(lb.F_EZ)[0])
    n_ref, e_ref = out["fp64"]
    for prec, tol in (("fp32", 1e-6), ("fp16s", 1e-3)):
        n1, ez = out[prec]
        en = np.linalg.norm(n1 - n_ref) / np.linalg.norm(n_ref)
        ee = np.linalg.norm(ez - e_ref) / np.linalg.norm(e_ref)
        assert en <= tol and ee <= tol, (prec, en, ee)


@pytest.mark.parametrize("closure,mu,window,tol,C", [("lec", 0.0, 6.0, 0.035, 0.5), ("lec", 0.04, 4.0, 0.045, 0.15),
                                                      ("warmc", 1e-3, 6.0, 0.035, 0.5)])
def test_axi_fp32_wake_matches_the_hankel_solution(closure, mu, window, tol, C):
    """App. B on the GPU path in FP32 storage (LEC on the persistent kernel):
    n - 1 at r = 0.3, 0.6, 1.0 against the order-0 Hankel solution by
    quadrature, with the oracle pins' grid (dz = dr = 0.1, tau = 0.505) and
    bounds."""
    from oracle import linear_theory as LT
    cfg = dict(dim=2, n=(200, 70), dx=0.1, courant=C, tau=0.505, closure=closure, dv=3, mu=mu, alpha=1e-3,
               sigma_z=0.6, sigma_r=0.5, z0=3.0, boundary="open", init_fields=True, geometry="axisymmetric")
    with lb.Run(cfg, "fp32") as run:
        N = int(round(14.0 / run.info().dt))
        run.step(N)
        n1 = run.moments(lb.M_N)[0].reshape(70, 200) - 1.0
        dt = run.info().dt
    xi = np.arange(200) * 0.1 - N * dt
    sel = (xi > 3.0 - window) & (xi < 3.0 + 1.5)
    cs2, ae2, ab2 = LT.coefficients(closure, mu)
    radii = [0.3, 0.6, 1.0]
    th = LT.hankel_n1(radii, xi[sel], 1e-3, 0.6, 0.5, 3.0, cs2, ae2, ab2)
    for m, r in enumerate(radii):
        j = int(round(r / 0.1))
        e = np.linalg.norm(n1[j, sel] - th[m]) / np.linalg.norm(th[m])
        assert e <= tol, (r, e)


def test_axi_fp32_acoustic_speed_against_temperature():
    """Fig. 6 on the GPU path (FP32 storage): c_s^2 fitted from the warm wake
    map (the Hankel solution's c_s^2 that matches the map best, which sets
    the Mach cone, c_s = c sin Theta) at mu = 0.01 and 0.04.  LEC within 12%
    of App. B's 5 mu / 3 (its O(mu) form; the enthalpy factor 1 + 5 mu / 2 is
    the rest), the WARMC faster than the LEC at each temperature (App. B:
    3 mu against 5 mu / 3), c_s^2 growing with mu, misfits below 6%."""
    from oracle import linear_theory as LT
    fitted = {}
    for closure in ("lec", "warmc"):
        for mu in (0.01, 0.04):
            C = 0.15 if closure == "warmc" else 0.2
            cfg = dict(dim=2, n=(160, 50), dx=0.1, courant=C, tau=0.505, closure=closure, dv=3, mu=mu, alpha=1e-3,
                       sigma_z=0.47, sigma_r=0.47, z0=3.0, boundary="open", init_fields=True,
                       geometry="axisymmetric")
            with lb.Run(cfg, "fp32") as run:
                N = int(round(11.0 / run.info().dt))
                run.step(N)
                n1 = run.moments(lb.M_N)[0].reshape(50, 160) - 1.0
                zd = 3.0 + N * run.info().dt
            xi = np.arange(160) * 0.1 - zd
            sel = (xi > -6.0) & (xi < 1.5)
            radii = np.arange(16) * 0.1
            ae2 = 1.0 - 2.5 * mu
            cs2, mis = LT.fit_cs2(n1[:16][:, sel], radii, xi[sel], 1e-3, 0.47, 0.47, 0.0, ae2, ae2)
            assert mis < 0.06, (closure, mu, mis)
            fitted[closure, mu] = cs2
    for mu in (0.01, 0.04):
        lec, warmc = fitted["lec", mu], fitted["warmc", mu]
        assert abs(lec / (5.0 * mu / 3.0) - 1.0) < 0.12, (mu, lec)
        assert 1.4 < warmc / lec < 2.0, (mu, warmc, lec)
    for closure in ("lec", "warmc"):
        assert 3.0 < fitted[closure, 0.04] / fitted[closure, 0.01] < 5.0


def test_axi_fp32_pressure_anisotropy_near_the_bunch():
    """Fig. 7 on the GPU path: WARMC, mu = 0.04, Q~ = 0.5, 25 um bunch,
    (z, r) grid of 30 x 6 k_p^-1 at dz = dr = 0.02, after the bunch has
    travelled 20 k_p^-1.  Ahead of the bunch the plasma is at rest and
    isotropic (P_par = P_perp); within 1.5 k_p^-1 of it |P_par / P_perp - 1|
    is of the order of 10% (5-20%); 8-16 k_p^-1 behind it (away from where
    the bunch started) it is smaller than at the bunch."""
    sz = sr = 0.47
    alpha = 0.5 / ((2 * np.pi) ** 1.5 * sz * sr * sr)
    nz, nr, dx = 1500, 300, 0.02
    cfg = _cfg("warmc", n=(nz, nr), dx=dx, mu=0.04, alpha=alpha, sigma_z=sz, sigma_r=sr, z0=4.0)
    with lb.Run(cfg, "fp32") as run:
        N = int(round(20.0 / run.info().dt))
        run.step(N)
        zd = 4.0 + N * run.info().dt
        ppar, pperp = (v.reshape(nr, nz) for v in run.moments(lb.M_P_PAR | lb.M_P_PERP))
    an = np.abs(ppar / pperp - 1.0)
    xi = np.arange(nz) * dx - zd
    near = an[:, np.abs(xi) < 1.5].max()
    far = an[:, (xi >= -16.0) & (xi < -8.0) & (xi + zd > 9.0)].max()
    ahead = an[:, xi > 2.0].max()
    assert ahead < 1e-5
    assert 0.05 < near < 0.20, near
    assert far < near, (far, near)
