"""GPU parity of the rest-frame analysis (Sec. 4): sampled T^{mu nu}
tables, their event mean and local rest frame and the Milne sampling, each
against the FP64 oracle (oracle/rest_frame.py and the simulation oracle) on
the same inputs.  The Gaussian fit is host code, checked on the CPU."""
import numpy as np
import pytest

import glasma_inputs as gi
from oracle import glasma_oracle as O
from oracle import rest_frame as RF

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_02044_gb300 import build as B
    B.build()
    from paper_2009_02044_gb300 import glasma
    glasma.load_library()
    return glasma


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _rest_gpu(G, tabs):
    import torch
    tabs = np.asarray(tabs, dtype=np.float64)
    ne, npt = tabs.shape[0], int(np.prod(tabs.shape[1:-1]))
    d = _dev(tabs.reshape(ne, npt, 4))
    out = torch.empty((npt, 8), dtype=torch.float64, device="cuda")
    G.glasma_rest_frame(d.data_ptr(), ne, npt, out.data_ptr(),
                        torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check_rest(got, tabs, tol=1e-12):
    mean = RF.ensemble_mean(tabs).reshape(-1, 4)
    ref = RF.rest_frame(mean)
    scale = np.max(np.abs(mean))
    assert np.allclose(got[:, :4], mean, rtol=0, atol=1e-15 * scale)
    valid = got[:, 7] == 1.0
    assert np.array_equal(valid, ref["valid"].reshape(-1))
    for col, key in ((4, "eps_loc"), (5, "pl_loc")):
        r = ref[key].reshape(-1)
        assert np.all(np.isnan(got[~valid, col]))
        assert np.max(np.abs(got[valid, col] - r[valid])) <= tol * scale
    rv = ref["v"].reshape(-1)
    assert np.max(np.abs(got[valid, 6] - rv[valid])) <= tol * 10


def test_rest_frame_of_boosted_and_random_tensors(G):
    rng = np.random.default_rng(21)
    ne, n = 3, 5000
    eps = rng.uniform(0.1, 2.0, (ne, n))
    pl = eps * rng.uniform(-0.45, 0.9, (ne, n))
    v = rng.uniform(-0.9, 0.9, (ne, n))
    g2 = 1 / (1 - v * v)
    tabs = np.stack([g2 * (eps + pl * v * v), g2 * (eps * v * v + pl),
                     0.5 * eps, g2 * v * (eps + pl)], axis=-1)
    # special rows: no flux, vacuum, no rest frame, negative eps + p_L
    tabs[:, :50, 3] = 0.0
    tabs[:, 50:60] = 0.0
    tabs[:, 60:70] = [1.0, 0.2, 0.4, 0.7]
    tabs[:, 70:80] = [-1.0, 0.2, 0.4, 0.1]
    _check_rest(_rest_gpu(G, tabs), tabs)


def test_sampling_matches_interpolation(G):
    import torch
    rng = np.random.default_rng(22)
    n_t, nz, stride, comp = 17, 53, 8, 4
    grid = rng.standard_normal((n_t, nz, stride))
    t0, dts, z0, az = -2.0, 0.5, -13.0, 0.5
    t = rng.uniform(t0 - 1, t0 + (n_t - 1) * dts + 1, 3000)
    z = rng.uniform(z0 - 1, z0 + (nz - 1) * az + 1, 3000)
    t[:4] = [t0, t0 + (n_t - 1) * dts, t0, t0 + (n_t - 1) * dts]
    z[:4] = [z0, z0, z0 + (nz - 1) * az, z0 + (nz - 1) * az]
    tau = rng.uniform(0.5, 6.0, 3000)
    eta = rng.uniform(-2.5, 2.5, 3000)
    dg = _dev(grid)
    for coords, (x, y) in (("lab", (t, z)), ("milne", (tau, eta))):
        out = torch.empty(x.size, dtype=torch.float64, device="cuda")
        dx, dy = _dev(x), _dev(y)      # kept alive until the kernel has run
        G.glasma_sample_grid(dg.data_ptr(), n_t, nz, stride, comp, t0, dts,
                             z0, az, dx.data_ptr(), dy.data_ptr(),
                             x.size, out.data_ptr(), coords=coords)
        got = out.cpu().numpy()
        if coords == "milne":
            x, y = RF.milne_to_lab(x, y)
        ref = RF.interp_tz(grid[..., comp], t0, dts, z0, az, x, y)
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        ok = ~np.isnan(ref)
        assert ok.sum() > 1000
        assert np.max(np.abs(got[ok] - ref[ok])) < 1e-13


def test_collision_chain_matches_oracle(G):
    """Three SU(2) FP64 events through the collision: T^{mu nu} sampled on
    the device every 4 steps, its event mean and rest frame, and eps_loc on
    the hyperbola tau = 14 (|eta_s| <= 0.45, clear of the receding nuclei,
    whose truncated profiles reach 8 cells behind the light cone), all
    against the oracle run on the same seeds."""
    import torch
    cfgs = [dict(gi.small_config(2, nz=64, nx=8, ny=6, seed=70 + e))
            for e in range(3)]
    every, n_s = 4, 17
    nz = cfgs[0]["nz"]
    tabs = torch.zeros((3, n_s, nz, 4), dtype=torch.float64, device="cuda")
    ref_tabs = np.zeros((3, n_s, nz, 4))
    for e, c in enumerate(cfgs):
        h = G.glasma_init_mv(c, None)
        p = O.Params.from_dict(c)
        st = O.init_mv(p, gi.mv_rho(c["seed"], 2, p.nx, p.ny, p.g2mu))
        for k in range(n_s):
            if k:
                G.glasma_step(h, every)
                st = O.step(st, every)
            G.glasma_tmunu_device(h, tabs[e, k].data_ptr())
            ref_tabs[e, k] = O.tmunu(st)[0]
    torch.cuda.synchronize()
    got_tabs = tabs.cpu().numpy()
    assert np.max(np.abs(got_tabs - ref_tabs)) <= 1e-11 * np.max(np.abs(ref_tabs))

    out = torch.empty((n_s * nz, 8), dtype=torch.float64, device="cuda")
    G.glasma_rest_frame(tabs.data_ptr(), 3, n_s * nz, out.data_ptr())
    torch.cuda.synchronize()
    rest = out.cpu().numpy()
    mean = RF.ensemble_mean(ref_tabs)
    ref = RF.rest_frame(mean)
    both = (rest[:, 7] == 1.0) & ref["valid"].reshape(-1)
    scale = np.max(np.abs(mean))
    # the rest frame amplifies the 1e-11 table differences near lightlike
    # flow by 1 / (1 - v^2); compare where |v| < 0.9
    slow = both & (np.abs(ref["v"].reshape(-1)) < 0.9)
    assert slow.sum() > 0.3 * both.sum()
    assert np.max(np.abs(rest[slow, 4] - ref["eps_loc"].reshape(-1)[slow])) <= 1e-9 * scale

    p = O.Params.from_dict(cfgs[0])
    tc, zc = RF.collision_origin(p.nz, p.a_z, p.dt, p.sigma_l)
    t0, dts, z0 = -tc, every * p.dt, -zc
    eta = np.linspace(-0.45, 0.45, 37)
    tau = np.full_like(eta, 14.0)
    prof = torch.empty(eta.size, dtype=torch.float64, device="cuda")
    dtau, deta = _dev(tau), _dev(eta)
    G.glasma_sample_grid(out.data_ptr(), n_s, nz, 8, 4, t0, dts, z0, p.a_z,
                         dtau.data_ptr(), deta.data_ptr(), eta.size,
                         prof.data_ptr())
    got_prof = prof.cpu().numpy()
    tt, zz = RF.milne_to_lab(tau, eta)
    ref_prof = RF.interp_tz(ref["eps_loc"], t0, dts, z0, p.a_z, tt, zz)
    assert np.all(np.isfinite(ref_prof))
    assert np.max(np.abs(got_prof - ref_prof)) <= 1e-9 * np.max(ref_prof)


def _profiles(G, m, events, nt, taus, eta):
    """eps_loc(tau, eta_s) of an ensemble of thin-nucleus SU(2) events
    (glasma_inputs.thin_ensemble_configs) through the library's chain:
    batched steps, device T^{mu nu} samples, rest frame, Milne sampling."""
    import math
    import torch
    cfgs = gi.thin_ensemble_configs(m, events, nt=nt)
    c0 = cfgs[0]
    nz, dt, az, every = c0["nz"], c0["dt"], c0["a_z"], 8
    n_s = c0["steps"] // every + 1
    hs = [G.glasma_init_mv(c, None) for c in cfgs]
    tabs = torch.zeros((events, n_s, nz, 4), dtype=torch.float64, device="cuda")
    b = G.glasma_batch_create(hs)
    for k in range(n_s):
        if k:
            G.glasma_batch_step(b, every)
        for e, h in enumerate(hs):
            G.glasma_tmunu_device(h, tabs[e, k].data_ptr())
    torch.cuda.synchronize()
    b.close()
    for h in hs:
        G.glasma_free(h)
    d = (math.ceil(4 * c0["sigma_l"] / az) + 2) * az
    rest = torch.empty((n_s * nz, 8), dtype=torch.float64, device="cuda")
    G.glasma_rest_frame(tabs.data_ptr(), events, n_s * nz, rest.data_ptr(),
                        torch.cuda.current_stream())
    e_d = _dev(eta)
    out = {}
    for tau in taus:
        t_d = _dev(np.full_like(eta, tau))
        o = torch.empty_like(e_d)
        G.glasma_sample_grid(rest.data_ptr(), n_s, nz, 8, 4, -d, every * dt,
                             -nz * az / 2.0, az, t_d.data_ptr(), e_d.data_ptr(),
                             len(eta), o.data_ptr(), coords="milne")
        torch.cuda.synchronize()
        out[tau] = o.cpu().numpy()
    return out


def test_rapidity_profiles_in_the_papers_regime(G):
    """Sec. 4 (Fig. 4, Eq. late_time_energy) on thin SU(2) nuclei: the
    rest-frame energy density is a Gaussian in eta_s centred at 0, it
    narrows as the IR regulator m grows, and tau eps_loc at eta_s = 0 is
    independent of tau (free streaming)."""
    eta = np.linspace(-1.2, 1.2, 25)
    taus = (12.0, 16.0, 20.0)
    sig = {}
    for m in (0.1, 0.4):
        prof = _profiles(G, m, 4, 64, taus, eta)
        amp, mu, s = G.glasma_fit_gaussian(eta, prof[20.0], 0.1)
        assert abs(mu) < 0.15
        sig[m] = s
        te = [tau * prof[tau][12] for tau in taus]
        assert (max(te) - min(te)) / np.mean(te) < 0.05
    assert sig[0.4] < 0.9 * sig[0.1]
