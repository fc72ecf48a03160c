"""The on-device wake fit (lbpwfa_line_fit) against the oracle's definition
of the same fit, and the warm dispersion of Sec. 6 (Fig. 3, Eq.
disp-rel1/2) measured with it on the GPU path."""
import numpy as np
import pytest

import oracle as O
from oracle import diagnostics as D
from tests import paper_values

pytestmark = pytest.mark.gpu

lb = pytest.importorskip("paper_2309_04872_gb300.lbpwfa")


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lb.load_library()


def _cfg1d(mu, closure="lec", dv=1, C=0.5):
    return dict(dim=1, n=(2048,), dx=40 / 2048, courant=C, tau=0.52, closure=closure, dv=dv, mu=mu,
                alpha=1e-3, sigma_z=1.0, z0=-5.0, boundary="open")


def test_line_fit_matches_the_oracle_definition_1d():
    """Same input line (exported from the GPU state): the device fit and the
    oracle's agree to round-off; the FP64 run itself matches the oracle run."""
    cfg = _cfg1d(1e-3)
    with lb.Run(cfg, "fp64") as run:
        N = int(round(39.0625 / run.info().dt))
        run.step(N)
        g = run.line_fit("ez", xi=(-25.0, -5.0), k=(0.5, 1.5, 201))
        ez = run.fields(lb.F_EZ)[0]
        dt = run.info().dt
        gn = run.line_fit("n", xi=(-25.0, -5.0), k=(0.5, 1.5, 201))
        n = run.moments(lb.M_N)[0]
    o = D.line_fit(ez, cfg["dx"], cfg["z0"] + (N - 0.5) * dt, -25.0, -5.0, 0.5, 1.5, 201)
    on = D.line_fit(n, cfg["dx"], cfg["z0"] + N * dt, -25.0, -5.0, 0.5, 1.5, 201, offset=1.0)
    for got, want in ((g, o), (gn, on)):
        assert got["points"] == want["points"]
        for key in ("k", "amplitude", "rms"):
            assert abs(got[key] - want[key]) <= 1e-10 * max(abs(want[key]), 1e-12), key
        assert abs(got["phase"] - want["phase"]) <= 1e-9
    orc = O.Oracle(cfg)
    orc.step(N)
    E, _ = orc.fields()
    ref = D.line_fit(E[0], cfg["dx"], cfg["z0"] + (N - 0.5) * orc.dt, -25.0, -5.0, 0.5, 1.5, 201)
    assert abs(g["k"] - ref["k"]) <= 1e-9 and abs(g["amplitude"] / ref["amplitude"] - 1) <= 1e-9


def test_line_fit_on_the_axis_of_an_axisymmetric_run():
    cfg = dict(dim=2, n=(300, 60), dx=0.05, courant=0.2, tau=0.53, closure="lec", dv=3, mu=0.0, alpha=1e-3,
               sigma_z=0.6, sigma_r=0.5, z0=3.0, boundary="open", init_fields=True, geometry="axisymmetric")
    with lb.Run(cfg, "fp64") as run:
        run.step(800)
        g = run.line_fit("n", line=(0, 0), xi=(-6.0, -1.0), k=(0.5, 1.5, 101))
        n = run.moments(lb.M_N)[0].reshape(60, 300)[0]
        zd = cfg["z0"] + 800 * run.info().dt
    o = D.line_fit(n, cfg["dx"], zd, -6.0, -1.0, 0.5, 1.5, 101, offset=1.0)
    assert g["points"] == o["points"] and abs(g["k"] - o["k"]) <= 1e-10
    assert abs(g["amplitude"] / o["amplitude"] - 1) <= 1e-10


def test_line_fit_rejects_bad_arguments():
    with lb.Run(_cfg1d(1e-3), "fp32") as run:
        for kw in (dict(k=(1.0, 0.5, 11)), dict(k=(0.5, 1.5, 2)), dict(xi=(1.0, -1.0))):
            with pytest.raises(lb.LbpwfaError):
                run.line_fit("ez", **kw)


_COLD = {}


@pytest.mark.parametrize("closure", ["lec", "warmc"])
@pytest.mark.parametrize("mu", [0.01, 0.04])
def test_warm_dispersion_1d3v_on_the_gpu(closure, mu):
    """Fig. 3 on the GPU path (FP32 storage): the warm minus cold shift of
    k_w^2 from the device fit against Eq. disp-rel1/2 (-5 mu / 6 for the
    LEC, +mu / 2 for the WARMC), within 2.5 mu^2 as for the oracle."""
    def kw(m):
        cfg = _cfg1d(m, closure, dv=3, C=0.25)
        with lb.Run(cfg, "fp32") as run:
            run.step(int(round(39.0625 / run.info().dt)))
            return run.line_fit("ez", xi=(-25.0, -5.0), k=(0.5, 1.5, 201))["k"]
    if closure not in _COLD:
        _COLD[closure] = kw(0.0) ** 2
    shift = kw(mu) ** 2 - _COLD[closure]
    paper = float(paper_values.dispersion()[closure][2]) * mu
    assert abs(_COLD[closure] - 1.0) < 2e-4
    assert abs(shift - paper) < 2.5 * mu * mu


@pytest.mark.parametrize("case", ["1d", "2d", "3d", "axi"])
def test_gauss_residual_matches_the_oracle_definition(case):
    """The device reduction against the oracle's definition on the same
    exported density and fields, after a driven FP64 run."""
    cfgs = {
        "1d": dict(dim=1, n=(301,), dx=0.05, courant=0.5, tau=0.53, closure="lec", dv=1, mu=1e-2, alpha=0.1,
                   sigma_z=0.6, z0=3.0, boundary="open"),
        "2d": dict(dim=2, n=(77, 45), dx=0.05, courant=0.1, tau=0.53, closure="warmc", dv=3, mu=1e-2, alpha=0.2,
                   sigma_z=0.6, sigma_r=0.3, z0=1.2, boundary="open", init_fields=True),
        "3d": dict(dim=3, n=(37, 21, 13), dx=0.05, courant=0.08, tau=0.53, closure="lec", dv=3, mu=1e-2,
                   alpha=0.2, sigma_z=0.6, sigma_r=0.3, z0=0.6, boundary="open", init_fields=True),
        "axi": dict(dim=2, n=(77, 45), dx=0.05, courant=0.1, tau=0.53, closure="lec", dv=3, mu=1e-2, alpha=0.2,
                    sigma_z=0.6, sigma_r=0.3, z0=1.2, boundary="open", init_fields=True, geometry="axisymmetric"),
    }
    cfg = cfgs[case]
    dim = cfg["dim"]
    lo = [2, 1, 1][:dim]
    hi = [v - 2 for v in cfg["n"]]
    with lb.Run(cfg, "fp64") as run:
        run.step(40)
        g = run.gauss_residual(lo, hi)
        n = run.moments(lb.M_N)[0]
        E = run.fields(lb.F_EZ | lb.F_EX | lb.F_EY)  # returned in bit order: E_x, E_y, E_z
        E = np.stack([E[2], E[0], E[1]])
        t = (run.info().step - 0.5) * run.info().dt
    r2, rho2, cells = D.gauss_residual(cfg, n, E, t, lo, hi)
    assert g["cells"] == cells
    assert abs(g["res2"] - r2) <= 1e-11 * r2
    assert abs(g["rho2"] - rho2) <= 1e-11 * rho2
    assert g["rho2"] > 0


def test_gauss_law_of_a_driven_run_on_the_gpu():
    """Sec. 6: Gauss's law holds to the LB diffusion (tau = 0.505, 300
    steps, FP32 storage): residual within 2% of |rho|, as for the oracle."""
    cfg = dict(dim=2, n=(96, 48), dx=0.1, courant=0.1, tau=0.505, closure="lec", dv=3,
               mu=1e-3, alpha=0.05, sigma_z=0.8, sigma_r=0.6, z0=3.0, boundary="open", init_fields=True)
    with lb.Run(cfg, "fp32") as run:
        run.step(300)
        g = run.gauss_residual([4, 4], [65, 43])
    assert g["cells"] == 61 * 39
    assert np.sqrt(g["res2"] / g["rho2"]) < 0.02


def test_gauss_residual_rejects_bad_ranges():
    cfg = dict(dim=2, n=(20, 10), dx=0.1, courant=0.1, tau=0.53, closure="lec", dv=3, mu=1e-3, alpha=0.05,
               sigma_z=0.8, sigma_r=0.6, z0=1.0, boundary="open")
    with lb.Run(cfg, "fp32") as run:
        for lo, hi in (([0, 0], [20, 9]), ([3, 3], [3, 5]), ([-1, 0], [5, 5])):
            with pytest.raises(lb.LbpwfaError):
                run.gauss_residual(lo, hi)
