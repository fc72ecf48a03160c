"""Failure detection through the C ABI, without a GPU fault.

* Non-finite populations: a NaN planted on the host through lbpwfa_set_state
  is counted by the FP64 reduction, which returns LBPWFA_ERR_NONFINITE; the
  count grows as the step spreads it, and a clean state clears it.
* Bounded waits: the TMA-staged step kernels wait on an mbarrier for each
  tile's population box.  With the poll limit lowered to 0
  (lbpwfa_set_wait_limit) that wait gives up at once; the kernel flags the
  handle's error word, lets the copy in flight land (the drain keeps its long
  limit), and ends the CTA.  The host then reads LBPWFA_ERR_TIMEOUT from
  lbpwfa_synchronize and lbpwfa_reduce until the state is replaced, and the
  context stays usable: the run steps on normally afterwards.
"""
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


def _cfg(closure="lec", n=(200, 90)):
    return dict(dim=2, n=n, dx=0.05, courant=0.1, tau=0.53, closure=closure, dv=3, mu=1e-2, alpha=0.2,
                sigma_z=0.6, sigma_r=0.3, z0=2.0, boundary="open", init_fields=True)


def _state(cfg, seed):
    o = O.Oracle(cfg)
    base = o.rest_advected()
    f = inputs.random_populations(seed, o.K, o.Q, o.ncell, base, np.abs(base) * 0.02 + 1e-3)
    return o, f


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_nonfinite_population_is_reported(prec, closure):
    cfg = _cfg(closure)
    o, f = _state(cfg, 41)
    nz, nx = cfg["n"]
    bad = f.copy()
    node = 50 + nz * 40            # a bulk node, away from every boundary
    bad[0, 3, node] = np.nan
    with lb.Run(cfg, prec) as run:
        run.set_state(f)
        out, st = run.reduce(status=True)
        assert st == 0 and out[2] == 0
        run.set_state(bad)
        out, st = run.reduce(status=True)
        assert st == -4 and out[2] == 1, (st, out)
        run.step(3)
        out, st = run.reduce(status=True)
        assert st == -4 and out[2] > 1, (st, out)
        # a clean state clears it
        run.set_state(f)
        out, st = run.reduce(status=True)
        assert st == 0 and out[2] == 0


@pytest.mark.parametrize("prec,variant,kv", [("fp32", 3, 3), ("fp16s", 3, 3), ("fp64", 2, 2), ("fp32", 2, 2)])
def test_bounded_wait_timeout_is_reported(prec, variant, kv):
    cfg = _cfg("lec", n=(700, 300))   # more tiles than persistent CTAs
    o, f = _state(cfg, 43)
    with lb.Run(cfg, prec, variant=variant) as run:
        assert run.info().kernel_variant == kv
        run.set_state(f)
        _, E0, B0 = run.get_state()
        run.step(2)
        run.synchronize()
        run.set_wait_limit(0)
        run.step(2)
        with pytest.raises(lb.LbpwfaError) as ei:
            run.synchronize()
        assert ei.value.status == -5
        with pytest.raises(lb.LbpwfaError) as ei:
            run.reduce()
        assert ei.value.status == -5
        # sticky until the state is replaced
        with pytest.raises(lb.LbpwfaError) as ei:
            run.synchronize()
        assert ei.value.status == -5
        # the context stays usable: restore the limit and the state, step on
        run.set_wait_limit(1 << 24)
        run.set_state(f, E0, B0)
        run.synchronize()
        run.step(2)
        run.synchronize()
        out, st = run.reduce(status=True)
        assert st == 0 and out[2] == 0
        again = run.advected()
    # the same sequence with four completed steps before the state is replaced
    with lb.Run(cfg, prec, variant=variant) as ref:
        ref.set_state(f)
        ref.step(4)
        ref.set_state(f, E0, B0)
        ref.step(2)
        assert np.array_equal(ref.advected(), again)


def test_plain_kernel_has_no_wait():
    """The global-memory pull kernel waits on nothing: the limit leaves it
    untouched."""
    cfg = _cfg("warmc")
    o, f = _state(cfg, 47)
    with lb.Run(cfg, "fp32") as run:
        assert run.info().kernel_variant == 1
        run.set_state(f)
        run.set_wait_limit(0)
        run.step(3)
        run.synchronize()
        out, st = run.reduce(status=True)
        assert st == 0
