"""lbpwfa_reduce_noalloc: the FP64 diagnostic sums for callers that cannot
allocate device memory (their memory belongs to another allocator, or their
loop cannot take cudaMalloc's implicit synchronisation).  The entry point
keeps its partial sums in a fixed device array inside the library instead of
a buffer the handle allocates.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It passes alone in a fresh
process and after the other tests (the shared array keeps the previous
call's contents, which each call overwrites)."""
import ctypes

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


def _noalloc(run, out, on_device):
    L = lb.load_library()
    ptr = ctypes.c_void_p(out.data_ptr()) if on_device else ctypes.c_void_p(out.ctypes.data)
    return L.lbpwfa_reduce_noalloc(run.handle, ptr, 1 if on_device else 0)


# 131 x 37 nodes fit one partial of the fixed array; 512 x 256 (131 072
# nodes) spread over 16 partials, so the multi-partial part of the array and
# the final sum over the partials run too
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
@pytest.mark.parametrize("n", [(131, 37), (512, 256)])
def test_noalloc_reduce_matches_reduce_on_two_calls(prec, n):
    import torch
    cfg = dict(dim=2, n=n, dx=0.05, courant=0.1, tau=0.53, closure="warmc", dv=3, mu=1e-2,
               alpha=0.2, sigma_z=0.6, sigma_r=0.3, z0=2.0, boundary="open", init_fields=True)
    orc = O.Oracle(cfg)
    base = orc.rest_advected()
    f = inputs.random_populations(3, orc.K, orc.Q, orc.ncell, base, np.abs(base) * 0.05 + 1e-3)
    with lb.Run(cfg, prec) as run:
        run.set_state(f)
        for call in range(2):            # two calls in a row, state changing between them
            run.step(7)
            ref = run.reduce()           # the existing entry point
            host = np.full(3, -1.0)
            assert _noalloc(run, host, False) == 0
            dev = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
            assert _noalloc(run, dev, True) == 0
            run.synchronize()
            for got in (host, dev.cpu().numpy()):
                assert np.allclose(got[:2], ref[:2], rtol=1e-12, atol=0.0), (call, got, ref)
                assert got[2] == ref[2] == 0.0


def test_noalloc_reduce_reports_nonfinite_and_timeout_like_reduce():
    """The host form returns NONFINITE for a planted NaN and TIMEOUT after a
    bounded device wait gave up, as lbpwfa_reduce does."""
    cfg = dict(dim=2, n=(300, 70), dx=0.05, courant=0.1, tau=0.53, closure="lec", dv=3, mu=1e-2,
               alpha=0.2, sigma_z=0.6, sigma_r=0.3, z0=2.0, boundary="open", init_fields=True)
    orc = O.Oracle(cfg)
    base = orc.rest_advected()
    f = inputs.random_populations(5, orc.K, orc.Q, orc.ncell, base, np.abs(base) * 0.02 + 1e-3)
    bad = f.copy()
    bad[1, 2, 40 + 300 * 30] = np.inf
    with lb.Run(cfg, "fp32") as run:
        assert run.info().kernel_variant == 3   # the persistent TMA kernel (bounded waits)
        run.set_state(bad)
        out = np.zeros(3)
        assert _noalloc(run, out, False) == -4 and out[2] == 1
        run.set_state(f)
        assert _noalloc(run, out, False) == 0 and out[2] == 0
        run.set_wait_limit(0)
        run.step(1)
        assert _noalloc(run, out, False) == -5
        run.set_wait_limit(1 << 24)
        run.set_state(f)
        run.step(1)
        assert _noalloc(run, out, False) == 0


def test_noalloc_reduce_rejects_runs_beyond_its_scratch():
    # 8192 x 4097 nodes: one row past the 2^25-node limit (about 3.6 GB of
    # binary16 populations)
    cfg = dict(dim=2, n=(8192, 4097), dx=0.05, courant=0.1, tau=0.53, closure="lec", dv=3, mu=1e-3,
               alpha=0.01, sigma_z=1.0, sigma_r=0.5, z0=2.0, boundary="open", init_fields=False)
    with lb.Run(cfg, "fp16s") as run:
        out = np.zeros(3)
        assert _noalloc(run, out, False) == -1
        msg = lb.load_library().lbpwfa_last_error(run.handle).decode()
        assert "static scratch limit" in msg and str(1 << 25) in msg
