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


def gauss_residual(cfg, n, E, t, lo, hi):
    """Gauss's law residual on the dual cells (the definition of the
    library's lbpwfa_gauss_residual): cells (i, j, k) with lo <= index < hi
    per present axis, centred at (z_{i+1/2}, x_{j+1/2}, y_{k+1/2});
    div E from the Yee slots (axisymmetric: (r_{j+1} E_r(j+1) - r_j E_r(j)) /
    (r_{j+1/2} dx)); rho = -(nbar - 1) - n_b(centre, t), nbar the mean of the
    cell's corner densities.  n: [ncell]; E: [3][ncell] (z, x, y); t: the
    time of E.  Returns (sum (div E - rho)^2, sum rho^2, cells)."""
    from oracle import driver_density
    dim = cfg["dim"]
    shape = tuple(reversed((list(cfg["n"]) + [1, 1])[:3]))  # (ny, nx, nz)
    nn = np.asarray(n, dtype=np.float64).reshape(shape)
    Ez, Ex, Ey = (np.asarray(E[a], dtype=np.float64).reshape(shape) for a in range(3))
    dx = cfg["dx"]
    axi = cfg.get("geometry", "cartesian") == "axisymmetric"
    nx, ny = shape[1], shape[0]
    lo = (list(lo) + [0, 0, 0])[:3]
    hi = (list(hi) + [1, 1, 1])[:3]
    for a in range(dim, 3):
        lo[a], hi[a] = 0, 1
    s_res = s_rho = 0.0
    cells = 0
    for k in range(lo[2], hi[2]):
        for j in range(lo[1], hi[1]):
            for i in range(lo[0], hi[0]):
                div = (Ez[k, j, i + 1] - Ez[k, j, i]) / dx
                if dim >= 2:
                    if axi:
                        rl, rh, rm = j * dx, (j + 1) * dx, (j + 0.5) * dx
                        div += (rh * Ex[k, j + 1, i] - rl * Ex[k, j, i]) / (rm * dx)
                    else:
                        div += (Ex[k, j + 1, i] - Ex[k, j, i]) / dx
                if dim >= 3:
                    div += (Ey[k + 1, j, i] - Ey[k, j, i]) / dx
                corners = [nn[k + b, j + a, i + d] for b in range(2 if dim >= 3 else 1)
                           for a in range(2 if dim >= 2 else 1) for d in range(2)]
                nbar = sum(corners) / len(corners)
                zc = (i + 0.5) * dx
                xc = (j + 0.5 - (0.0 if axi else 0.5 * (nx - 1))) * dx
                yc = (k + 0.5 - 0.5 * (ny - 1)) * dx
                nb = driver_density(cfg, zc, xc if dim >= 2 else 0.0, yc if dim >= 3 else 0.0, t=t)
                rho = -(nbar - 1.0) - nb
                s_res += (div - rho) ** 2
                s_rho += rho * rho
                cells += 1
    return s_res, s_rho, cells
