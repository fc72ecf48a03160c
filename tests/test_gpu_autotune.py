"""lbpwfa_autotune: every step kernel a run can take is timed on the run's own
state, the fastest is kept, and the state, step count and results are
exactly those of a run that never tuned.

  * The variants timed are the ones the run can take (2D open LEC: plain, TMA
    box, persistent; periodic: plain only; 3D: tiled and marching;
    axisymmetric LEC: its plain and persistent kernels), and the one kept is
    the fastest of them.
  * After tuning, the run continues bit for bit as a run that loads the same
    state from a checkpoint into the kept kernel.
  * With LBPWFA_TUNE_CACHE set, a second run of the same key reads the choice
    back and times nothing."""
import os

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


def _cfg(**kw):
    c = dict(dim=2, n=(300, 160), dx=0.05, courant=0.1, tau=0.53, closure="lec", dv=3, mu=1e-2, alpha=0.1,
             sigma_z=1.0, sigma_r=0.5, z0=4.0, boundary="open", init_fields=True)
    c.update(kw)
    return c


CASES = {
    "2d_lec_open": (_cfg(), "fp32", {1, 2, 3}),
    "2d_warmc_open": (_cfg(closure="warmc"), "fp32", {1, 2}),
    "2d_lec_periodic": (_cfg(boundary="periodic"), "fp32", {1}),
    "2d_lec_fp16s": (_cfg(), "fp16s", {1, 2, 3}),
    "3d_warmc": (dict(_cfg(closure="warmc", alpha=1.0, sigma_z=0.7, sigma_r=0.3, z0=2.8), dim=3, n=(96, 40, 40)),
                 "fp32", {1, 4}),
    "axi_lec": (_cfg(geometry="axisymmetric", n=(300, 80)), "fp32", {1, 3}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_autotune_keeps_the_fastest_and_the_state(case, tmp_path):
    cfg, prec, allowed = CASES[case]
    orc = O.Oracle(cfg)
    # a perturbed state: the momenta by 0.01, the temperature sets by a
    # twentieth of their rest value or of mu
    base = orc.rest_advected()
    amp = np.abs(base) * 0.05
    dim = cfg["dim"]
    if cfg["closure"] == "lec":
        amp[1:] = 0.01
    else:
        amp[2:2 + dim] = 0.01
        for j in range(orc.K - 2 - dim):
            if base[2 + dim + j] == 0.0:
                amp[2 + dim + j] = 0.05 * cfg["mu"]
    f = inputs.random_populations(41, orc.K, orc.Q, orc.ncell, base, amp)
    E, B = inputs.random_fields(42, orc.ncell, 0.01)
    path = str(tmp_path / "ck.bin")
    with lb.Run(cfg, prec) as a:
        a.set_state(f, E, B)
        a.step(3)
        a.save(path)
        ms, v = a.autotune()
        timed = {k for k, t in ms.items() if t is not None}
        assert timed and timed <= allowed, (timed, allowed)
        kept = 1 if v == 5 else v
        assert kept in timed and ms[kept] == min(ms[k] for k in timed), (ms, v)
        assert a.info().step == 3
        a.step(4)
        A1, F1 = a.advected(), a.fields()
    with lb.Run(cfg, prec, variant=kept) as b:
        assert b.info().kernel_variant == v
        b.load(path)
        b.step(4)
        assert np.array_equal(b.advected(), A1)
        assert np.array_equal(b.fields(), F1)


def test_autotune_cache_is_read_back(tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("LBPWFA_TUNE_CACHE", str(cache))
    cfg = _cfg()
    with lb.Run(cfg, "fp32") as a:
        ms, v = a.autotune()
    assert any(t is not None for t in ms.values())
    assert cache.exists() and '": ' in cache.read_text()
    with lb.Run(cfg, "fp32") as b:
        ms2, v2 = b.autotune()
    assert all(t is None for t in ms2.values())
    assert v2 == v
    # another grid is another key
    with lb.Run(_cfg(n=(256, 160)), "fp32") as c:
        ms3, _ = c.autotune()
    assert any(t is not None for t in ms3.values())
    assert os.path.getsize(cache) > 0
