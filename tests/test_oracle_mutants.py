"""The pins catch plausible mistakes in the oracle.

Each mistake below is planted at a PLANTED site of oracle/lbpwfa_oracle.c;
the oracle is rebuilt once per mistake (ORC_PLANT=n, a separate library in
oracle/_build) and the pins named for it must fail in a child pytest run,
while the unplanted oracle passes them in the rest of the suite.  CPU only.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = "tests/test_oracle_pins.py::"
X = "tests/test_oracle_axisymmetric.py::"
J = "tests/test_oracle_adjoint.py::"

# n: (the mistake, the pins that must catch it)
MUTANTS = {
    1: ("equilibrium: second-order Hermite term without its 1/2 (Eq. feq)",
        [P + "test_equilibrium_moments"]),
    2: ("streaming: populations pushed against their velocity instead of pulled (Eq. lbe)",
        [P + "test_streaming_shift"]),
    3: ("Ampere's law: the plasma and bunch current with the wrong sign",
        [P + "test_linear_wake_1d_closed_form"]),
    4: ("Faraday's law: curl E with the wrong sign",
        [X + "test_axisymmetric_cold_lec_wake_matches_hankel"]),
    5: ("LEC source: the magnetic force u x B with the wrong sign (Eq. lb-ade-lec-comps-F)",
        [P + "test_lec_sources_match_appendix_rows"]),
    6: ("WARMC source: one of the two magnetic rotation terms of F_theta dropped (App. A)",
        [P + "test_warmc_sources_match_appendix_rows"]),
    7: ("collision: the source added without its time step (Eq. lsource)",
        [P + "test_linear_wake_1d_closed_form"]),
    8: ("LEC decode: the enthalpy factor 1 + D/2 read as 1 + 2/D (Eq. lb-ade-lec-comps-A)",
        [P + "test_lec_decode_roundtrip"]),
    9: ("axisymmetric Ampere: the Cartesian curl in place of (1/r) d_r (r B_phi)",
        [X + "test_axisymmetric_cold_lec_wake_matches_hankel"]),
    10: ("axisymmetric WARMC: theta^{phi phi} / r with the wrong sign in the n lambda u_r row (App. A)",
         [X + "test_axisymmetric_warmc_matches_3d_cartesian"]),
    11: ("axisymmetric LEC: the -u_r A / r divergence term with the wrong sign",
         [X + "test_axisymmetric_cold_lec_wake_matches_hankel"]),
    12: ("adjoint: the transposed pressure gradient with the wrong sign at the forward neighbour",
         [J + "test_adjoint_driver_parameters", J + "test_adjoint_starting_state"]),
    13: ("adjoint: the electric-field adjoint of the LEC Lorentz force dropped",
         [J + "test_adjoint_driver_parameters", J + "test_adjoint_starting_state"]),
    14: ("driver: the bunch moving towards -z (Eq. bunch-density, zeta = z - z0 - t)",
         [P + "test_driver_normalised_charge"]),
    15: ("WARMC decode: u^a from n lambda u^a divided by n instead of n lambda (Eq. lb-ade-warmc-comps-A)",
         [P + "test_warmc_decode_identities"]),
    16: ("adjoint WARMC decode: an off-diagonal theta pair's adjoint without its transposed entry",
         [J + "test_adjoint_driver_parameters", J + "test_adjoint_starting_state"]),
    17: ("WARMC source: the backward time derivative of theta^{0a} dropped from the n lambda u row",
         [P + "test_warm_dispersion_1d3v"]),
    18: ("3D initial field: an E_x slot taken half a cell low in z (Sec. 6, the v -> c field on the Yee grid)",
         [P + "test_gauss_law_of_the_3d_initial_field"]),
}


def _run(n):
    env = dict(os.environ, ORC_PLANT=str(n), OMP_NUM_THREADS="2")
    # the planted library must build, so that a failing pin is the mistake's
    b = subprocess.run([sys.executable, "-c", "import oracle; oracle.build()"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    if b.returncode != 0:
        return -1, "planted build failed:\n" + b.stdout[-2000:] + b.stderr[-2000:]
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "not gpu", *MUTANTS[n][1]]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def mutant_runs():
    workers = max(1, min(len(MUTANTS), (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        return dict(zip(sorted(MUTANTS), ex.map(_run, sorted(MUTANTS))))


@pytest.mark.parametrize("n", sorted(MUTANTS))
def test_pins_catch_planted_mistake(n, mutant_runs):
    rc, out = mutant_runs[n]
    # 1: the tests ran and at least one failed (-1: the planted build failed;
    # 2 and above: the run itself broke)
    assert rc == 1, f"mistake {n} ({MUTANTS[n][0]}) not caught, rc={rc}\n{out}"
    assert " failed" in out, out
