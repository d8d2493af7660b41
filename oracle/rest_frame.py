"""Plain FP64 CPU oracle of the rest-frame analysis of the averaged
energy-momentum tensor (Sec. 4 of Ipp & Mueller, "Progress on 3+1D Glasma
simulations").

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import this module.  The CUDA
library never calls it and shares no code with it.

What it computes:

* The event average <T^{mu nu}>(t, z) of per-event tables (eps, p_L, p_T,
  S_L) sampled at lattice times and z slices (Sec. 4, the 15-event average).
* The local rest frame of the (t, z) block of <T^{mu nu}> (Sec. 4: the
  tensor is diagonalised to give the local rest-frame energy density
  eps_loc): the eigenvalue problem T^mu_nu u^nu = lambda u^mu with metric
  diag(+1, -1) on the block [[eps, S_L], [S_L, p_L]].  The timelike
  eigenvector gives the flow velocity v_z = u^z / u^t and eps_loc = its
  eigenvalue; the spacelike one gives the rest-frame longitudinal pressure
  p_L,loc = -(its eigenvalue).  Computed with LAPACK's general eigensolver
  (numpy.linalg.eig), not with the closed form the CUDA path uses.
* Milne coordinates (Sec. 4): tau = sqrt(t^2 - z^2) and space-time
  rapidity eta_s.  Reading: the paper prints eta_s = ln[(t - z)/(t + z)]/2;
  the standard definition, used here, is eta_s = ln[(t + z)/(t - z)]/2 =
  artanh(z / t), so that z = tau sinh eta_s and t = tau cosh eta_s (the
  printed form is its negative; every profile here is compared through its
  width, which is the same for both).
* Sampling eps_loc(tau, eta_s) from the (t, z) grid by bilinear
  interpolation (scipy's RegularGridInterpolator, linear).
* The Gaussian fit of a rapidity profile (Sec. 4, Fig. 4: the profiles are
  fitted by Gaussians whose widths sigma_eta are quoted): a weighted
  least-squares fit of a parabola to log f over the points with f above a
  fraction of the maximum, weights f on the unsquared residuals
  (numpy.polyfit), giving f = A exp(-(eta - mu)^2 / (2 sigma^2)).
* Free streaming (Sec. 4, Eq. late_time_energy): tau eps_loc(tau, eta_s)
  is independent of tau.
"""
import math

import numpy as np
from scipy.interpolate import RegularGridInterpolator

# columns of a per-slice table, as the simulation returns them
EPS, P_L, P_T, S_L = 0, 1, 2, 3


def collision_origin(nz, a_z, dt, sigma_l, z_offset=0.0):
    """Lab-frame origin of the collision: the nuclei start at z_c -/+ d at
    step 0 and move at the speed of light, so they meet at t_c = d at the
    box centre z_c = nz a_z / 2 (the nucleus placement of the
    initial-condition reading: d = z_offset, else ceil(4 sigma / a_z) + 2
    cells).  Returns (t_c, z_c); slice iz sits at z = iz a_z, step n at
    t = n dt."""
    zc = nz * a_z / 2.0
    d = z_offset if z_offset > 0 else (math.ceil(4 * sigma_l / a_z) + 2) * a_z
    return d, zc


def ensemble_mean(tabs):
    """<T^{mu nu}>: mean over the leading (event) axis of tables
    [events][n_t][nz][4]."""
    return np.mean(np.asarray(tabs, dtype=np.float64), axis=0)


def rest_frame(tab):
    """Local rest frame of every (t, z) entry of a mean table [..., 4].

    Returns a dict of arrays: eps_loc, pl_loc, v (flow velocity u^z / u^t)
    and valid (a timelike eigenvector with real eigenvalues exists)."""
    tab = np.asarray(tab, dtype=np.float64)
    shape = tab.shape[:-1]
    flat = tab.reshape(-1, 4)
    out = {k: np.full(flat.shape[0], np.nan) for k in ("eps_loc", "pl_loc", "v")}
    valid = np.zeros(flat.shape[0], dtype=bool)
    for i, (eps, pl, _, sl) in enumerate(flat):
        if eps == 0.0 and pl == 0.0 and sl == 0.0:
            out["eps_loc"][i] = out["pl_loc"][i] = out["v"][i] = 0.0
            valid[i] = True
            continue
        # mixed tensor T^mu_nu = T^{mu rho} g_{rho nu}, g = diag(1, -1)
        mixed = np.array([[eps, -sl], [sl, -pl]])
        lam, vec = np.linalg.eig(mixed)
        if np.any(np.abs(lam.imag) > 0) or np.any(np.abs(vec.imag) > 0):
            continue
        lam, vec = lam.real, vec.real
        timelike = [k for k in range(2) if abs(vec[0, k]) > abs(vec[1, k])]
        if len(timelike) != 1:
            continue
        k = timelike[0]
        out["eps_loc"][i] = lam[k]
        out["pl_loc"][i] = -lam[1 - k]
        out["v"][i] = vec[1, k] / vec[0, k]
        valid[i] = True
    res = {k: v.reshape(shape) for k, v in out.items()}
    res["valid"] = valid.reshape(shape)
    return res


def milne_to_lab(tau, eta):
    """(tau, eta_s) -> (t, z) relative to the collision origin."""
    tau = np.asarray(tau, dtype=np.float64)
    eta = np.asarray(eta, dtype=np.float64)
    return tau * np.cosh(eta), tau * np.sinh(eta)


def interp_tz(grid, t0, dts, z0, az, t, z):
    """Bilinear interpolation of grid[n_t][nz] (grid point (k, j) at
    t = t0 + k dts, z = z0 + j az) at the points (t, z); NaN outside."""
    grid = np.asarray(grid, dtype=np.float64)
    tk = t0 + dts * np.arange(grid.shape[0])
    zj = z0 + az * np.arange(grid.shape[1])
    f = RegularGridInterpolator((tk, zj), grid, method="linear",
                                bounds_error=False, fill_value=np.nan)
    pts = np.stack(np.broadcast_arrays(np.asarray(t, float),
                                       np.asarray(z, float)), axis=-1)
    return f(pts)


def fit_gaussian(eta, f, frac=0.1):
    """Gaussian fit of a profile: returns (A, mu, sigma) of
    A exp(-(eta - mu)^2 / (2 sigma^2)), fitted as a weighted parabola in
    log f over the points with f > frac * max f."""
    eta = np.asarray(eta, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    ok = np.isfinite(f) & (f > frac * np.nanmax(f))
    c2, c1, c0 = np.polyfit(eta[ok], np.log(f[ok]), 2, w=f[ok])
    if not c2 < 0:
        raise ValueError("profile has no maximum")
    sigma = math.sqrt(-1.0 / (2.0 * c2))
    mu = -c1 / (2.0 * c2)
    amp = math.exp(c0 - c1 * c1 / (4.0 * c2))
    return amp, mu, sigma
