"""Values the paper prints, read from tests/golden/ (each fixture cites its
section and equations), against the linear theory the oracle is pinned to
and against the workloads the bench and the tests run."""
import math
from fractions import Fraction

import pytest

from oracle import linear_theory as LT
from tests import paper_values as PV


@pytest.mark.parametrize("closure", ["lec", "warmc"])
def test_printed_dispersion_forms_agree(closure):
    """Sec. 6, 1D3V: with the phase velocity at c (omega = k in plasma
    units), 1 + a mu + b mu omega^2 = omega^2 gives omega^2 = (1 + a mu) /
    (1 - b mu) = 1 + (a + b) mu + O(mu^2), which must be Eq. disp-rel1/2's
    1 + c mu: the printed general form and the printed special form agree
    exactly at O(mu)."""
    a, b, c = PV.dispersion()[closure]
    assert a + b == c
    for mu in (Fraction(1, 100), Fraction(1, 25)):
        exact = (1 + a * mu) / (1 - b * mu)
        assert abs(exact - (1 + c * mu)) <= 2 * b * b * mu * mu


@pytest.mark.parametrize("closure", ["lec", "warmc"])
@pytest.mark.parametrize("mu", [1e-3, 1e-2, 4e-2])
def test_linear_theory_coefficients_are_the_printed_ones(closure, mu):
    """App. B's Klein-Gordon model carries the Sec. 6 relation: c_s^2 = b mu,
    a_e^2 = 1 + a mu, and its one-dimensional wavenumber at phase velocity
    c, K(0)^2 = a_e^2 / (1 - c_s^2), is Eq. disp-rel1/2's 1 + c mu to O(mu)."""
    a, b, c = (float(v) for v in PV.dispersion()[closure])
    cs2, ae2, ab2 = LT.coefficients(closure, mu)
    assert cs2 == pytest.approx(b * mu, rel=1e-14)
    assert ae2 == pytest.approx(1 + a * mu, rel=1e-14)
    assert ab2 == ae2
    K0sq = ae2 / (1 - cs2)
    assert abs(K0sq - (1 + c * mu)) <= 2 * b * b * mu * mu


def test_axisymmetric_workload_is_the_papers_setup():
    """The 3000 x 600 axisymmetric workload is the setup of Sec. 6: L_z x L_r
    at dz = dr, the printed time step, the 3D value of tau, the Fig. 4
    temperature and Q~ (Eq. Qtilde with D = 3)."""
    import bench
    s = PV.spatial_setup()
    c = bench.CONFIG_AXI
    assert s["dz"] == s["dr"]
    assert tuple(c["n"]) == (int(s["L_z"] / s["dz"]), int(s["L_r"] / s["dr"]))
    assert Fraction(c["dx"]).limit_denominator(10**6) == s["dz"]
    assert c["courant"] * c["dx"] == pytest.approx(float(s["dt"]), rel=1e-12)
    assert Fraction(c["tau"]).limit_denominator(1000) == s["tau_3d"]
    assert Fraction(c["mu"]).limit_denominator(1000) == s["mu_fig4"]
    Q = (2 * math.pi) ** 1.5 * c["sigma_z"] * c["sigma_r"] ** 2 * c["alpha"]
    assert Q == pytest.approx(float(s["Qtilde_fig4"]), rel=1e-12)
    # mu_i = k_B T / (m_e c^2), m_e c^2 = 510.999 keV: 20 keV is 0.0391
    assert abs(float(s["kT_fig4_keV"]) / 510.999 - float(s["mu_fig4"])) < 1e-3


def test_one_and_three_dimensional_workloads_take_the_printed_tau():
    """Sec. 6: tau = 0.52 in the 1D setups and 0.53 in the 3D ones."""
    import bench
    s = PV.spatial_setup()
    assert Fraction(bench.CONFIG_1D["tau"]).limit_denominator(1000) == s["tau_1d"]
    for c in (bench.CONFIG_3D, bench.CONFIG_AXI):
        assert Fraction(c["tau"]).limit_denominator(1000) == s["tau_3d"]
