"""Pins of the rest-frame oracle (oracle/rest_frame.py) to facts that do not
come from the oracle itself: Lorentz boosts of known rest-frame tensors,
invariants of the (t, z) block, an exact free-streaming solution of
Sec. 4 Eq. late_time_energy, exact Gaussians and exactly bilinear fields."""
import math

import numpy as np
import pytest

from oracle import rest_frame as RF


def boosted(eps_loc, pl_loc, v):
    """T^{mu nu} (t, z block) of a rest-frame diag(eps_loc, ., ., pl_loc)
    boosted to velocity v: eps_loc u u + pl_loc n n, u = g(1, v),
    n = g(v, 1)."""
    g2 = 1.0 / (1.0 - v * v)
    t00 = g2 * (eps_loc + pl_loc * v * v)
    t03 = g2 * v * (eps_loc + pl_loc)
    t33 = g2 * (eps_loc * v * v + pl_loc)
    return t00, t33, t03


def test_boost_is_undone():
    rng = np.random.default_rng(11)
    n = 400
    eps = rng.uniform(0.1, 3.0, n)
    pl = eps * rng.uniform(-0.45, 0.9, n)
    v = rng.uniform(-0.95, 0.95, n)
    tab = np.zeros((n, 4))
    for i in range(n):
        t00, t33, t03 = boosted(eps[i], pl[i], v[i])
        tab[i] = (t00, t33, 0.5 * (t00 - t33), t03)
    r = RF.rest_frame(tab)
    assert r["valid"].all()
    assert np.max(np.abs(r["eps_loc"] - eps) / eps) < 1e-12
    assert np.max(np.abs(r["pl_loc"] - pl) / eps) < 1e-12
    assert np.max(np.abs(r["v"] - v)) < 1e-12


def test_tensor_at_rest_and_invariants():
    rng = np.random.default_rng(12)
    tab = np.zeros((200, 4))
    tab[:, 0] = rng.uniform(0.5, 2.0, 200)
    tab[:, 1] = rng.uniform(-0.2, 0.5, 200)
    tab[:, 3] = rng.uniform(-0.4, 0.4, 200) * (tab[:, 0] + tab[:, 1])
    tab[:100, 3] = 0.0
    r = RF.rest_frame(tab)
    # no flux: already the rest frame
    assert np.array_equal(r["eps_loc"][:100], tab[:100, 0])
    assert np.array_equal(r["pl_loc"][:100], tab[:100, 1])
    assert np.all(r["v"][:100] == 0.0)
    # trace and determinant of T^mu_nu are frame independent
    e, p, s = tab[:, 0], tab[:, 1], tab[:, 3]
    assert np.allclose(r["eps_loc"] - r["pl_loc"], e - p, rtol=0, atol=1e-13)
    assert np.allclose(r["eps_loc"] * r["pl_loc"], e * p - s * s, rtol=0,
                       atol=1e-13)


def test_spacelike_flux_has_no_rest_frame():
    # |S_L| > (eps + p_L) / 2: no timelike eigenvector
    r = RF.rest_frame(np.array([[1.0, 0.2, 0.4, 0.61], [1.0, 0.2, 0.4, -0.7]]))
    assert not r["valid"].any()
    assert np.isnan(r["eps_loc"]).all()
    r = RF.rest_frame(np.zeros((1, 4)))
    assert r["valid"].all() and r["eps_loc"][0] == 0.0


def test_gaussian_fit_of_an_exact_gaussian():
    eta = np.linspace(-4, 4, 161)
    f = 2.5 * np.exp(-(eta - 0.3) ** 2 / (2 * 1.7 ** 2))
    amp, mu, sigma = RF.fit_gaussian(eta, f, frac=0.05)
    assert abs(amp - 2.5) < 1e-11 and abs(mu - 0.3) < 1e-11
    assert abs(sigma - 1.7) < 1e-11
    with pytest.raises(ValueError):
        RF.fit_gaussian(eta, np.exp(eta ** 2 / 8))


def test_bilinear_fields_are_interpolated_exactly():
    t0, dts, z0, az = -3.0, 0.75, -10.0, 0.5
    tk = t0 + dts * np.arange(9)[:, None]
    zj = z0 + az * np.arange(41)[None, :]
    grid = 1.5 - 0.25 * tk + 0.125 * zj + 0.0625 * tk * zj
    rng = np.random.default_rng(3)
    t = rng.uniform(t0, t0 + 8 * dts, 50)
    z = rng.uniform(z0, z0 + 40 * az, 50)
    got = RF.interp_tz(grid, t0, dts, z0, az, t, z)
    assert np.allclose(got, 1.5 - 0.25 * t + 0.125 * z + 0.0625 * t * z,
                       rtol=0, atol=1e-13)
    out = RF.interp_tz(grid, t0, dts, z0, az, np.array([t0 - 0.1, 0.0]),
                       np.array([0.0, z0 + 40 * az + 0.1]))
    assert np.isnan(out).all()


def free_streaming_table(t, z, amp, sigma):
    """<T^{mu nu}> of free streaming with v_z = z / t and p_L,loc = 0
    (Sec. 4): eps_loc = amp exp(-eta^2 / (2 sigma^2)) / tau, p_T =
    eps_loc / 2; zero outside the forward light cone."""
    T, Z = np.meshgrid(t, z, indexing="ij")
    inside = np.abs(Z) < T
    tau = np.sqrt(np.where(inside, T * T - Z * Z, 1.0))
    eta = np.where(inside, np.arctanh(np.where(inside, Z / T, 0.0)), 0.0)
    e = np.where(inside, amp * np.exp(-eta ** 2 / (2 * sigma ** 2)) / tau, 0)
    tab = np.zeros(T.shape + (4,))
    g2 = np.where(inside, T * T / (tau * tau), 1.0)
    v = np.where(inside, Z / np.where(T > 0, T, 1.0), 0.0)
    tab[..., 0] = g2 * e
    tab[..., 1] = g2 * v * v * e
    tab[..., 2] = 0.5 * e
    tab[..., 3] = g2 * v * e
    return tab, e, v, inside


def test_free_streaming_solution_is_recovered():
    """tau eps_loc is constant along each eta_s (Eq. late_time_energy), the
    flow is z / t, and the Gaussian width in eta_s comes back."""
    dts, az = 0.25, 0.25
    t = 1.0 + dts * np.arange(221)
    z = -48.0 + az * np.arange(385)
    tab, e, v, inside = free_streaming_table(t, z, amp=3.0, sigma=0.9)
    r = RF.rest_frame(tab)
    assert r["valid"].all()
    assert np.allclose(r["eps_loc"][inside], e[inside], rtol=1e-11, atol=0)
    assert np.allclose(r["v"][inside], v[inside], rtol=0, atol=1e-11)
    assert np.max(np.abs(r["pl_loc"][inside])) < 1e-11 * np.max(e)
    eta = np.linspace(-1.2, 1.2, 49)
    prof = {}
    for tau in (12.0, 20.0, 28.0):
        tt, zz = RF.milne_to_lab(tau, eta)
        prof[tau] = RF.interp_tz(r["eps_loc"], t[0], dts, z[0], az, tt, zz)
        assert np.all(np.isfinite(prof[tau]))
        _, mu, sig = RF.fit_gaussian(eta, prof[tau], frac=0.0)
        assert abs(sig - 0.9) < 2e-3 and abs(mu) < 1e-6
    assert np.allclose(12.0 * prof[12.0], 28.0 * prof[28.0], rtol=2e-3)


def test_collision_origin_is_where_the_charges_meet():
    """The charge centroids of the two nuclei of the initial state sit at
    z_c -/+ t_c (they then move at the speed of light), so they meet at
    (t_c, z_c)."""
    import glasma_inputs as gi
    from oracle import glasma_oracle as O
    for kw in (dict(), dict(z_offset=13.0), dict(a_z=0.5, dt=0.25)):
        cfg = gi.small_config(2, nz=64, nx=6, ny=5, **kw)
        p = O.Params.from_dict(cfg)
        st = O.init_mv(p, gi.mv_rho(cfg["seed"], 2, 6, 5, p.g2mu))
        tc, zc = RF.collision_origin(p.nz, p.a_z, p.dt, p.sigma_l,
                                     cfg.get("z_offset", 0.0))
        z = np.arange(p.nz) * p.a_z
        for Q, sign in ((st.QB, -1.0), (st.QA, 1.0)):
            w = np.sum(Q ** 2, axis=(1, 2, 3))
            centroid = np.sum(w * z) / np.sum(w)
            # the profile is sampled on the lattice, hence the cell tolerance
            assert abs(centroid - (zc + sign * tc)) < 0.5 * p.a_z
