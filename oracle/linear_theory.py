"""Warm linear theory of App. B: the axisymmetric linear wake by the order-0
Hankel transform, evaluated by quadrature.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: used by tests/ to pin
the FP64 oracle; the CUDA library never calls it.

The linearised fluid + Maxwell system gives a forced Klein-Gordon equation
for n_1 = n - 1 (App. B, Eq. fhow):

    d_t^2 n_1 - c_s^2 lap n_1 = -a_e^2 n_1 - a_b^2 n_b,

with the closure coefficients of App. B at O(mu).  With every quantity a
function of the co-moving xi = z - t (the driver moves towards +z at c, so
the plasma ahead of it is at rest) and of r, the order-0 Hankel transform
f^(w) = int_0^inf f(r) J_0(w r) r dr turns the transverse Laplacian into -w^2,
and each w obeys a forced oscillator in xi,

    n1^'' = -K(w)^2 n1^ - a_b^2 / (1 - c_s^2) n_b^,
    K(w)^2 = (a_e^2 + w^2 c_s^2) / (1 - c_s^2),

whose causal solution (zero for xi -> +inf) is

    n1^(w, xi) = -a_b^2 / (1 - c_s^2) int_xi^inf n_b^(w, xi') sin(K (xi' - xi)) / K dxi'.

For the Gaussian bunch n_b = L(xi) exp(-r^2 / 2 sigma_r^2) (rms sizes),
n_b^(w, xi) = L(xi) sigma_r^2 exp(-w^2 sigma_r^2 / 2).  n_1 follows from the
inverse transform n_1(r) = int_0^inf n1^(w) J_0(w r) w dw.

Units: k_p^-1, omega_p^-1, c = 1, densities in n_i.
"""
import numpy as np
import scipy.special as sp


def coefficients(closure, mu):
    """(c_s^2, a_e^2, a_b^2) of App. B at O(mu).  For the WARMC the paper
    prints a_b^2 = 1 - mu/2; our own linearisation gives a_b = a_e (the
    bunch enters only through Gauss's law, like n_1), which is what this
    returns."""
    if closure == "lec":
        return 5.0 / 3.0 * mu, 1.0 - 2.5 * mu, 1.0 - 2.5 * mu
    if closure == "warmc":
        return 3.0 * mu, 1.0 - 2.5 * mu, 1.0 - 2.5 * mu
    raise ValueError(closure)


def hankel_n1(r, xi, alpha, sigma_z, sigma_r, xi_d, cs2, ae2, ab2, nw=3000, h=0.005, wmax=None):
    """n_1(r, xi) on the outer product of the radii ``r`` and co-moving
    positions ``xi`` (Gaussian bunch of peak ``alpha`` centred at ``xi_d``).

    Quadrature: midpoint rule in w on [0, wmax] (the transform of the bunch
    falls as exp(-w^2 sigma_r^2 / 2); wmax = 9 / sigma_r), and the trapezoid
    rule in xi' on a grid of step h from below min(xi) to xi_d + 8 sigma_z,
    summed from the front of the bunch backwards (the causal integral for
    every xi at once); values between grid points are linearly
    interpolated."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    wmax = 9.0 / sigma_r if wmax is None else wmax
    dw = wmax / nw
    w = (np.arange(nw) + 0.5) * dw
    K = np.sqrt((ae2 + w * w * cs2) / (1.0 - cs2))
    hi = xi_d + 8.0 * sigma_z
    lo = min(xi.min(), hi) - h
    g = np.arange(lo, hi + h, h)
    L = alpha * np.exp(-(g - xi_d) ** 2 / (2.0 * sigma_z ** 2))
    ph = np.exp(1j * np.outer(K, g))                      # e^{i K xi'}
    f = L[None, :] * ph
    seg = 0.5 * (f[:, 1:] + f[:, :-1]) * h
    F = np.zeros_like(f)                                  # int_{g_m}^{hi} L e^{i K xi'}
    F[:, :-1] = np.cumsum(seg[:, ::-1], axis=1)[:, ::-1]
    S = np.imag(np.conj(ph) * F) / K[:, None]             # int L sin(K (xi' - xi)) / K
    nb_hat = sigma_r ** 2 * np.exp(-0.5 * (w * sigma_r) ** 2)
    n_hat = -(ab2 / (1.0 - cs2)) * nb_hat[:, None] * S    # [w][g]
    n1g = (sp.j0(np.outer(r, w)) * (w * dw)[None, :]) @ n_hat
    return np.stack([np.interp(xi, g, row) for row in n1g])


def fit_cs2(n1, radii, xi, alpha, sigma_z, sigma_r, xi_d, ae2, ab2, bounds=(1e-4, 0.3), nw=1500):
    """The acoustic speed squared c_s^2 that makes the order-0 Hankel
    solution closest (relative L2 over the given radii and co-moving
    positions) to a wake map n1[radius][xi], with a_e^2 and a_b^2 held
    fixed: c_s shapes the Mach cone of the warm wake (Sec. 6, Fig. 6:
    c_s = c sin(Theta)), so the fit measures it from the whole cone rather
    than from one contour of it.  Bounded scalar minimisation (scipy);
    returns (c_s^2, misfit)."""
    from scipy.optimize import minimize_scalar
    n1 = np.asarray(n1, dtype=np.float64)
    scale = np.linalg.norm(n1)

    def misfit(cs2):
        th = hankel_n1(radii, xi, alpha, sigma_z, sigma_r, xi_d, cs2, ae2, ab2, nw=nw)
        return np.linalg.norm(n1 - th) / scale

    r = minimize_scalar(misfit, bounds=bounds, method="bounded", options={"xatol": 1e-5})
    return float(r.x), float(r.fun)
