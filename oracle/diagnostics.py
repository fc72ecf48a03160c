"""Wake diagnostics on oracle (or any FP64) arrays: the least-squares
sinusoid fit along one grid line that measures the wake's wavenumber (the
dispersion measurement of Sec. 6, Fig. 3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

Definition (the same as the library's lbpwfa_line_fit): the values q_j at
xi_j = j dx - z_d inside xi_lo <= xi <= xi_hi are fitted by a cos(k xi) +
b sin(k xi) from the normal equations of the sums of cos^2, cos sin, sin^2,
q cos and q sin; R(k) = sum q^2 - (a sum q cos + b sum q sin).  R is
evaluated on the uniform grid k_lo .. k_hi (nk points); its minimum is
refined by the parabola through it and its neighbours (offset clamped to
half a grid step) and the fit is redone there.  Returns k, A = sqrt(a^2 +
b^2), phi = -atan2(b, a) (so q ~ A cos(k xi + phi)), the rms residual and
the number of points."""
import numpy as np


def _sums(q, xi, k):
    c, s = np.cos(k * xi), np.sin(k * xi)
    return (np.sum(c * c), np.sum(c * s), np.sum(s * s), np.sum(q * c), np.sum(q * s), np.sum(q * q))


def _solve(S):
    cc, cs, ss, qc, qs, qq = S
    det = cc * ss - cs * cs
    if not det > 0:
        return 0.0, 0.0, qq
    a = (qc * ss - qs * cs) / det
    b = (qs * cc - qc * cs) / det
    return a, b, qq - (a * qc + b * qs)


def line_fit(values, dx, zd, xi_lo, xi_hi, k_lo, k_hi, nk, offset=0.0):
    """values: the line's FP64 values along z (index j at z = j dx)."""
    values = np.asarray(values, dtype=np.float64)
    xi_all = np.arange(values.size) * dx - zd
    sel = (xi_all >= xi_lo) & (xi_all <= xi_hi)
    q, xi = values[sel] - offset, xi_all[sel]
    dk = (k_hi - k_lo) / (nk - 1)
    R = np.array([_solve(_sums(q, xi, k_lo + m * dk))[2] for m in range(nk)])
    mb = int(np.argmin(R))
    d = 0.0
    if 0 < mb < nk - 1:
        den = R[mb - 1] - 2 * R[mb] + R[mb + 1]
        if den > 0:
            d = 0.5 * (R[mb - 1] - R[mb + 1]) / den
        d = min(0.5, max(-0.5, d))
    k = k_lo + (mb + d) * dk
    a, b, Rk = _solve(_sums(q, xi, k))
    n = int(q.size)
    return dict(k=k, amplitude=float(np.hypot(a, b)), phase=float(-np.arctan2(b, a)),
                rms=float(np.sqrt(max(Rk, 0.0) / n)) if n else 0.0, points=n)
