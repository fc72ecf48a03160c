"""Batched sweeps: many 2D runs of uneven grids and both closures advanced
by one persistent launch per step (CUDA-graph replays of 32 steps plus
single launches for the rest)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from tests import parity as P
from tests import inputs

pytestmark = pytest.mark.gpu

lb = pytest.importorskip("paper_2309_04872_gb300.lbpwfa")


@pytest.fixture(scope="module", autouse=True)
def _library():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lb.load_library()


def _same_to_roundoff(got, ref, rest=None, what=""):
    """Batch and single-run kernels inline the same step; the compiler may
    fuse multiply-adds differently in the two, so FP32 results agree to
    round-off rather than bit for bit: the deviation of every set (or field
    component) within 1e-5 of its own largest deviation after tens of steps
    (FP32 unit round-off 6e-8, grown by the scheme's amplification)."""
    got, ref = np.asarray(got), np.asarray(ref)
    for k in range(ref.shape[0]):
        r0 = 0.0 if rest is None else rest[k]
        # fields: on the scale of all components (E_z of the driver field is
        # a near-cancellation residue of curl B and the driver current)
        scale = np.abs(ref[k] - r0).max() if rest is not None else np.abs(ref).max()
        assert np.abs(got[k] - ref[k]).max() <= 1e-5 * scale + 1e-30, (what, k)


def _runs():
    base = dict(dim=2, dx=0.05, courant=0.1, tau=0.53, dv=3, sigma_r=0.4, boundary="open", init_fields=True)
    return [
        dict(base, n=(96, 40), closure="lec", mu=1e-2, alpha=0.3, sigma_z=0.7, z0=1.5),
        dict(base, n=(131, 37), closure="warmc", mu=5e-3, alpha=0.5, sigma_z=0.5, z0=2.0),
        dict(base, n=(64, 64), closure="warmc", mu=2e-2, alpha=0.1, sigma_z=1.0, z0=1.0),
        dict(base, n=(200, 24), closure="lec", mu=1e-3, alpha=0.8, sigma_z=0.6, z0=3.0),
    ]


@pytest.mark.parametrize("tune", [False, True])
def test_batch_members_match_single_runs(tune):
    runs = _runs()
    nsteps = 70  # two graph replays of 32 steps and 6 single launches
    with lb.Batch(runs, "fp32", tune=tune) as b:
        b.step(nsteps)
        got = [(m.advected(), m.fields()) for m in b.members]
        assert b.info().step == nsteps
    for cfg, (A, F) in zip(runs, got):
        with lb.Run(cfg, "fp32", variant=1) as r:
            r.step(nsteps)
            rest = O.Oracle(cfg).rest_advected()
            _same_to_roundoff(A, r.advected(), rest, "advected")
            _same_to_roundoff(F, r.fields(), None, "fields")


def test_batch_fp64_matches_oracle():
    runs = _runs()[:3]
    with lb.Batch(runs, "fp64", tune=False) as b:
        b.step(40)
        for cfg, m in zip(runs, b.members):
            o = O.Oracle(cfg)
            o.step(40)
            A = m.advected()
            Ao = o.advected()
            rest = o.rest_advected()
            for k in range(o.K):
                P.check64(A[k], Ao[k], rest[k], 40, o.Q, f"batch member A{k}", P.rest_scale(o))


def test_batch_member_state_reset_matches_single_run():
    """Replacing a WARMC member's state restarts its backward time
    differences exactly as lbpwfa_set_state does for a single run."""
    runs = _runs()
    o = O.Oracle(runs[1])
    base = o.rest_advected()
    f = inputs.random_populations(12, o.K, o.Q, o.ncell, base, np.abs(base) * 0.03 + 1e-3)
    with lb.Batch(runs, "fp32", tune=False) as b:
        b.step(5)
        b.members[1].set_state(f)
        b.step(9)
        A = b.members[1].advected()
    with lb.Run(runs[1], "fp32", variant=1) as r:
        r.step(5)
        r.set_state(f)
        r.step(9)
        _same_to_roundoff(A, r.advected(), base, "advected")
    # the batch itself is deterministic
    with lb.Batch(runs, "fp32", tune=False) as b:
        b.step(5)
        b.members[1].set_state(f)
        b.step(9)
        assert np.allclose(b.members[1].advected(), A, rtol=0, atol=0)


def test_batch_member_cannot_step_alone():
    with lb.Batch(_runs()[:2], "fp32", tune=False) as b:
        with pytest.raises(lb.LbpwfaError) as ei:
            b.members[0].step(1)
        assert ei.value.status == -6


def test_batch_autotune_cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("LBPWFA_TUNE_CACHE", str(path))
    runs = _runs()
    closures = {r["closure"] for r in runs}
    assert closures == {"lec", "warmc"}
    with lb.Batch(runs, "fp32", tune=True) as b:
        first = b.info()
        # both closures tuned over the three candidate tiles
        assert all(first.tuned_ms[cl][c] > 0 for cl in range(2) for c in range(3))
        assert all(first.grid[cl] > 0 for cl in range(2))
    entries = json.loads(path.read_text())
    assert len(entries) == 1
    (choice,) = entries.values()
    with lb.Batch(runs, "fp32", tune=True) as b:
        again = b.info()
        assert all(again.tuned_ms[cl][c] < 0 for cl in range(2) for c in range(4))  # read from the cache
        assert [list(t) for t in again.tile] == [list(t) for t in first.tile]
    assert choice // 4 in (0, 1, 2) and choice % 4 in (0, 1, 2)


def test_batch_rejects_exact_sum_storage():
    """FP32C (exact set sums) is a single-run storage mode."""
    with pytest.raises(lb.LbpwfaError) as ei:
        lb.Batch(_runs()[:2], "fp32c", tune=False)
    assert ei.value.status == -1


def test_batch_rejects_mixed_inputs():
    runs = _runs()
    with pytest.raises(lb.LbpwfaError):
        lb.Batch([runs[0], dict(runs[1], dim=3, n=(16, 16, 16))], "fp32")


def test_batch_fp16s_members_match_single_runs():
    """FP16-shifted storage in a batch (Cartesian and axisymmetric runs):
    members agree with the single runs' plain kernels to the storage's
    round-off, 1e-3 of each set's largest deviation after 70 steps (a fused
    multiply-add taken differently can flip one binary16 rounding)."""
    runs = _runs()[:2] + _mixed_geometry_runs()[:2]
    with lb.Batch(runs, "fp16s", tune=False) as b:
        b.step(70)
        got = [m.advected() for m in b.members]
    for cfg, A in zip(runs, got):
        with lb.Run(cfg, "fp16s", variant=1) as r:
            r.step(70)
            ref = r.advected()
        rest = O.Oracle(cfg).rest_advected()
        for k in range(ref.shape[0]):
            scale = np.abs(ref[k] - rest[k]).max()
            assert np.abs(A[k] - ref[k]).max() <= 1e-3 * scale + 1e-30, (cfg["closure"], k)


def _mixed_geometry_runs():
    """Axisymmetric (z, r) runs of both closures beside a Cartesian one."""
    base = dict(dim=2, dx=0.05, courant=0.1, tau=0.53, dv=3, sigma_r=0.3, boundary="open", init_fields=True)
    return [
        dict(base, n=(131, 37), closure="lec", mu=4e-2, alpha=0.3, sigma_z=0.6, z0=2.0, geometry="axisymmetric"),
        dict(base, n=(96, 40), closure="warmc", mu=4e-2, alpha=0.3, sigma_z=0.5, z0=1.5, geometry="axisymmetric"),
        dict(base, n=(77, 45), closure="lec", mu=1e-2, alpha=0.2, sigma_z=0.6, z0=1.2),
    ]


def test_batch_axisymmetric_members_match_single_runs():
    """Axisymmetric and Cartesian runs in one batch (the per-run geometry
    picks the step body): FP32 members agree with the single runs' plain
    kernels to round-off after 70 steps."""
    runs = _mixed_geometry_runs()
    with lb.Batch(runs, "fp32", tune=False) as b:
        b.step(70)
        got = [(m.advected(), m.fields()) for m in b.members]
    for cfg, (A, F) in zip(runs, got):
        with lb.Run(cfg, "fp32", variant=1) as r:
            r.step(70)
            rest = O.Oracle(cfg).rest_advected()
            _same_to_roundoff(A, r.advected(), rest, "advected")
            _same_to_roundoff(F, r.fields(), None, "fields")


def test_batch_axisymmetric_fp64_matches_oracle():
    runs = _mixed_geometry_runs()
    with lb.Batch(runs, "fp64", tune=False) as b:
        b.step(40)
        for cfg, m in zip(runs, b.members):
            o = O.Oracle(cfg)
            o.step(40)
            A = m.advected()
            Ao = o.advected()
            rest = o.rest_advected()
            for k in range(o.K):
                P.check64(A[k], Ao[k], rest[k], 40, o.Q, f"batch member A{k}", P.rest_scale(o))


def test_batched_temperature_sweep_acoustic_speed():
    """Fig. 6 as one batched sweep: six axisymmetric runs (mu = 0.01, 0.02,
    0.04, both closures; FP32) advanced together, c_s^2 fitted from each
    member's wake map with App. B's Hankel solution.  LEC within 12% of
    5 mu / 3 (its O(mu) form), the WARMC faster than the LEC at every mu,
    c_s^2 increasing with mu for both."""
    from oracle import linear_theory as LT
    mus = (0.01, 0.02, 0.04)
    runs = [dict(dim=2, n=(160, 50), dx=0.1, courant=0.15, tau=0.505, closure=cl, dv=3, mu=mu, alpha=1e-3,
                 sigma_z=0.47, sigma_r=0.47, z0=3.0, boundary="open", init_fields=True, geometry="axisymmetric")
            for cl in ("lec", "warmc") for mu in mus]
    N = int(round(11.0 / (0.15 * 0.1)))
    with lb.Batch(runs, "fp32", tune=False) as b:
        b.step(N)
        maps = [m.moments(lb.M_N)[0].reshape(50, 160) - 1.0 for m in b.members]
    xi = np.arange(160) * 0.1 - (3.0 + N * 0.015)
    sel = (xi > -6.0) & (xi < 1.5)
    radii = np.arange(16) * 0.1
    cs2 = {}
    for cfg, n1 in zip(runs, maps):
        ae2 = 1.0 - 2.5 * cfg["mu"]
        c, mis = LT.fit_cs2(n1[:16][:, sel], radii, xi[sel], 1e-3, 0.47, 0.47, 0.0, ae2, ae2)
        assert mis < 0.06, (cfg["closure"], cfg["mu"], mis)
        cs2[cfg["closure"], cfg["mu"]] = c
    for mu in mus:
        assert abs(cs2["lec", mu] / (5.0 * mu / 3.0) - 1.0) < 0.12, (mu, cs2["lec", mu])
        assert cs2["warmc", mu] > 1.3 * cs2["lec", mu], mu
    for cl in ("lec", "warmc"):
        assert cs2[cl, 0.01] < cs2[cl, 0.02] < cs2[cl, 0.04]


def test_full_sweep_fp32_against_fp64():
    """The bench's full batched sweep (64 seeded runs of 256-1024 x 256-512
    nodes, both closures, 15.1 M nodes): after 10 steps every member's
    FP32 n - 1 agrees with the FP64 batch's to 1e-5 (relative L2), and no
    population is non-finite."""
    draws = inputs.batch_draws(64, seed=2309)
    cfgs = [dict(dim=2, n=(d["nz"], d["nx"]), dx=0.05, courant=0.1, tau=0.53, closure=d["closure"], dv=3,
                 mu=d["mu"], alpha=d["alpha"], sigma_z=d["sigma_z"], sigma_r=0.5, z0=4.0 * d["sigma_z"],
                 boundary="open", init_fields=True) for d in draws]
    out = {}
    for prec in ("fp64", "fp32"):
        with lb.Batch(cfgs, prec, tune=False) as b:
            b.step(10)
            out[prec] = [m.moments(lb.M_N)[0] - 1.0 for m in b.members]
            assert all(m.reduce()[2] == 0 for m in b.members)
    for i, (a, r) in enumerate(zip(out["fp32"], out["fp64"])):
        assert np.linalg.norm(a - r) <= 1e-5 * np.linalg.norm(r), i
