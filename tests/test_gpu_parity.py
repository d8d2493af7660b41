"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle
on the same seeded inputs, element by element.

Tolerances: FP64 path 1e-11 relative to the largest reference entry
(max-norm), as the method's FP64 target states; FP32 path (FP32 links and
fields, FP64 reductions) a bound derived from single-precision rounding
accumulated over the steps taken, written beside each check."""
import numpy as np
import pytest

import glasma_inputs as gi
from oracle import glasma_oracle as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


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


def rel(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def run_both(G, cfg, steps, rho=None):
    p = O.Params.from_dict(cfg)
    if rho is None:
        rho = gi.mv_rho(cfg["seed"], p.nc, p.nx, p.ny, p.g2mu)
    h = G.glasma_init_mv(cfg, rho)
    G.glasma_step(h, steps)
    st = O.step(O.init_mv(p, rho), steps)
    return h, st


def compare_state(G, h, st, tol, what=""):
    U, E, QA, QB, n = G.glasma_get_fields(h)
    assert n == st.n
    errs = dict(U=rel(U, st.U), E=rel(E, st.E), QA=rel(QA, st.QA),
                QB=rel(QB, st.QB))
    tab, H = G.glasma_tmunu(h)
    rtab, rH = O.tmunu(st)
    errs["eps"] = rel(tab[:, 0], rtab[:, 0])
    errs["tmunu"] = rel(tab, rtab)
    errs["H"] = abs(H - rH) / abs(rH)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (what, errs)
    return errs


# ---------------------------------------------------------------------------
# FP64 parity
# ---------------------------------------------------------------------------

def test_su2_init_matches_oracle(G):
    cfg = gi.CONFIGS["su2_128x16x16"]
    h, st = run_both(G, cfg, 0)
    compare_state(G, h, st, TOL64, "init")
    gmax, grms, rmax = G.glasma_gauss_residual(h)
    assert gmax <= 1e-13 * rmax


def test_su2_128x16x16_fp64_100_steps(G):
    """The SU(2) 128 x 16^2 collision, full 100 steps."""
    cfg = gi.CONFIGS["su2_128x16x16"]
    h, st = run_both(G, cfg, cfg["steps"])
    compare_state(G, h, st, TOL64, "su2 100 steps")
    gmax, grms, rmax = G.glasma_gauss_residual(h)
    og = O.gauss_residual(st)
    assert gmax <= 1e-12 * rmax
    assert abs(rmax - og[2]) <= 1e-12 * og[2]


@pytest.mark.parametrize("nc", [2, 3])
def test_small_collision_fp64(G, nc):
    """Ragged 48 x 10 x 12 lattice (no power-of-two extent) through the
    collision: nuclei pass through each other within 40 steps."""
    cfg = gi.small_config(nc)
    h, st = run_both(G, cfg, cfg["steps"])
    compare_state(G, h, st, TOL64, "small nc=%d" % nc)
    gmax, grms, rmax = G.glasma_gauss_residual(h)
    assert gmax <= 1e-12 * rmax


def test_anisotropic_fp64(G):
    """a_z = dt = 0.5 a_t: a hop every step, anisotropic force weights."""
    cfg = gi.small_config(3, nz=64, nx=7, ny=6, a_z=0.5, dt=0.25,
                          sigma_l=1.5, steps=30)
    h, st = run_both(G, cfg, cfg["steps"])
    compare_state(G, h, st, TOL64, "anisotropic")


def test_seed_only_init_matches_host_generator(G):
    """rho drawn on the device from the seed equals the seeded host draw
    (the same Philox4x32-10 counters; Box-Muller via device libm)."""
    cfg = gi.small_config(3, seed=123456789012)
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 3, p.nx, p.ny, p.g2mu)
    h1 = G.glasma_init_mv(cfg, None)
    h2 = G.glasma_init_mv(cfg, rho)
    a = G.glasma_get_fields(h1)
    b = G.glasma_get_fields(h2)
    for x, y in zip(a[:4], b[:4]):
        assert rel(x, y) < 1e-13


def _random_state(nc, nz, ny, nx, seed, charges):
    rng = np.random.default_rng(seed)
    p = O.Params(nc=nc, nz=nz, nx=nx, ny=ny, a_z=0.5, dt=0.25, sigma_l=1.0)
    U = gi.near_identity_su(nc, (3, nz, ny, nx), rng, 0.3)
    U[2][nz - 1] = np.eye(nc)
    na = nc * nc - 1
    E = 0.3 * rng.standard_normal((3, nz, ny, nx, na))
    E[2][nz - 1] = 0.0
    QA = np.zeros((nz, ny, nx, na))
    QB = np.zeros((nz, ny, nx, na))
    if charges:
        QA[nz // 2 + 2: nz - 3] = 0.1 * rng.standard_normal(
            QA[nz // 2 + 2: nz - 3].shape)
        QB[3: nz // 2 - 2] = 0.1 * rng.standard_normal(
            QB[3: nz // 2 - 2].shape)
    return p, O.State(p, U, E, QA, QB, 0, U.copy())


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("shape", [(16, 4, 4), (24, 6, 13)])
def test_random_state_steps(G, nc, shape):
    """Generic (non-MV) links, fields and charges loaded through
    set_fields on 4 x 4 x 16 and a ragged 13 x 6 x 24 lattice: every
    plaquette orientation, both hop directions, T^{mu nu} and Gauss."""
    nz, ny, nx = shape
    p, st = _random_state(nc, nz, ny, nx, 40 + nz, charges=True)
    cfg = dict(nc=nc, nz=nz, nx=nx, ny=ny, a_t=1.0, a_z=0.5, dt=0.25,
               sigma_l=0.25, g2mu=0.0, m_ir=0.2, seed=0, precision="fp64")
    h = G.glasma_init_mv(cfg, None)
    G.glasma_set_fields(h, st.U, st.E, st.QA, st.QB, None, 0)
    G.glasma_step(h, 5)
    ref = O.step(st, 5)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    assert n == 5
    assert rel(U, ref.U) < TOL64
    assert rel(E, ref.E) < TOL64
    assert rel(QA, ref.QA) < TOL64 and rel(QB, ref.QB) < TOL64
    tab, H = G.glasma_tmunu(h)
    rtab, rH = O.tmunu(ref)
    assert rel(tab, rtab) < TOL64
    gm, grms, rm = G.glasma_gauss_residual(h)
    og = O.gauss_residual(ref)
    # random E violates Gauss; the residual itself must match the oracle's
    assert abs(gm - og[0]) <= 1e-12 * og[0]
    assert abs(grms - og[1]) <= 1e-12 * og[1]
    assert abs(rm - og[2]) <= 1e-12 * og[2]


# ---------------------------------------------------------------------------
# FP32 (FP32 links and fields, FP64 reductions)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [2, 3])
def test_small_collision_fp32(G, nc):
    """FP32 state against the FP64 oracle.  Bound: per step the link and
    field updates round at ~6e-8 relative; over 40 steps of a weakly
    nonlinear evolution the accumulated relative error stays below
    40 * 6e-8 * (growth ~10) ~ 3e-5; eps is checked at 1e-5 of its max."""
    cfg = dict(gi.small_config(nc), precision="fp32")
    h, st = run_both(G, cfg, cfg["steps"])
    U, E, QA, QB, n = G.glasma_get_fields(h)
    assert rel(U, st.U) < 3e-5
    assert rel(E, st.E) < 3e-5
    assert rel(QA, st.QA) < 3e-5 and rel(QB, st.QB) < 3e-5
    tab, H = G.glasma_tmunu(h)
    rtab, rH = O.tmunu(st)
    e_eps = np.max(np.abs(tab[:, 0] - rtab[:, 0])) / np.max(rtab[:, 0])
    assert e_eps < 1e-5, e_eps
    gmax, grms, rmax = G.glasma_gauss_residual(h)
    assert gmax < 1e-5 * rmax


# ---------------------------------------------------------------------------
# Full-size workloads, sampled: one step of the oracle at random sites from
# the GPU's own state, in the launch configuration the benchmark times.
# ---------------------------------------------------------------------------

def _sampled_step_check(G, cfg, warm_steps, nsites, tol_e, tol_u, seed=0):
    h = G.glasma_init_mv(cfg, None)
    G.glasma_step(h, warm_steps)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    p = O.Params.from_dict(cfg)
    st = O.State(p, U, E, QA, QB, n)
    rng = np.random.default_rng(seed)
    info = G.glasma_get_info(h)
    zlo = info.window_b[0]
    zhi = info.window_a[0] + info.window_a[1]
    sites = [(int(rng.integers(zlo, zhi)), int(rng.integers(p.ny)),
              int(rng.integers(p.nx))) for _ in range(nsites)]
    sites += [(0, 0, 0), (p.nz - 1, p.ny - 1, p.nx - 1), (p.nz - 2, 1, 2)]
    Eo, Uo = O.step_at_sites(st, sites)
    G.glasma_step(h, 1)
    U2, E2, _, _, _ = G.glasma_get_fields(h)
    for k, (z, y, x) in enumerate(sites):
        assert np.max(np.abs(E2[:, z, y, x] - Eo[k])) <= tol_e, (z, y, x)
        assert np.max(np.abs(U2[:, z, y, x] - Uo[k])) <= tol_u, (z, y, x)
    gmax, grms, rmax = G.glasma_gauss_residual(h)
    nc = p.nc
    uu = np.einsum("...ji,...jk->...ik", np.conj(U2), U2) - np.eye(nc)
    return gmax, rmax, float(np.max(np.abs(uu)))


def test_su3_512x64x64_fp32_sampled(G):
    """The SU(3) 512 x 64^2 event in FP32 (the benchmarked configuration):
    20 steps (10 hops), then one step at 200 sampled sites against the
    oracle evaluated on the GPU's own state.  FP32 bound (absolute): the
    force sums 8 staples of three products of O(1) link entries, each
    rounded at u = 6e-8, weighted by dt * 2/a^2 = 1, so one step's E error
    stays below ~8 * 3 * u ~ 2e-7; the new links round at a few u."""
    cfg = gi.CONFIGS["su3_512x64x64"]
    cfg = dict(cfg, precision="fp32")
    gmax, rmax, udev = _sampled_step_check(G, cfg, 20, 200, 2e-7, 1e-6)
    assert gmax < 1e-4 * rmax
    assert udev < 1e-6


def test_su3_512x64x64_fp64_sampled(G):
    cfg = dict(gi.CONFIGS["su3_512x64x64"], precision="fp64")
    gmax, rmax, udev = _sampled_step_check(G, cfg, 4, 100, 1e-14, 1e-13)
    assert gmax < 1e-12 * rmax
    assert udev < 1e-13


# ---------------------------------------------------------------------------
# Improved (semi-implicit) scheme
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [2, 3])
def test_implicit_fp64_matches_oracle(G, nc):
    """Semi-implicit steps (a_z = 0.5, dt = 0.25, a hop every step) through
    the collision region, FP64, converged to 1e-14 on both sides."""
    cfg = gi.small_config(nc, nz=64, nx=7, ny=6, a_z=0.5, dt=0.25,
                          sigma_l=1.5, steps=10)
    cfg.update(scheme="implicit", implicit_tol=1e-14, implicit_max_iter=60)
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], nc, p.nx, p.ny, p.g2mu)
    h = G.glasma_init_mv(cfg, rho)
    G.glasma_step(h, cfg["steps"])
    st = O.step_implicit(O.init_mv(p, rho), cfg["steps"], tol=1e-14)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    assert rel(U, st.U) < TOL64 and rel(E, st.E) < TOL64
    assert rel(QA, st.QA) < TOL64 and rel(QB, st.QB) < TOL64
    tab, H = G.glasma_tmunu(h)
    # T^{mu nu} uses the leapfrog E(n+1/2) in both implementations
    rtab, rH = O.tmunu(st)
    assert rel(tab, rtab) < TOL64
    gm, _, rm = G.glasma_gauss_residual(h)
    og = O.gauss_residual(st)
    assert abs(gm - og[0]) <= 1e-9 * og[0]
    info = G.glasma_get_info(h)
    assert abs(info.implicit_iters - st.extra["iters"]) <= 1


@pytest.mark.parametrize("nc", [2, 3])
def test_implicit_fp32_matches_oracle(G, nc):
    """FP32 semi-implicit steps against the FP64 oracle (iteration stopped at
    1e-6, far above the FP32 rounding of E ~ 1e-8): relative error bound as
    for the FP32 leapfrog."""
    cfg = gi.small_config(nc, nz=64, nx=7, ny=6, a_z=0.5, dt=0.25,
                          sigma_l=1.5, steps=10)
    cfg.update(scheme="implicit", implicit_tol=1e-7, implicit_max_iter=60,
               precision="fp32")
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], nc, p.nx, p.ny, p.g2mu)
    h = G.glasma_init_mv(cfg, rho)
    G.glasma_step(h, cfg["steps"])
    st = O.step_implicit(O.init_mv(p, rho), cfg["steps"], tol=1e-14)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    assert rel(U, st.U) < 3e-5 and rel(E, st.E) < 3e-5
    tab, H = G.glasma_tmunu(h)
    rtab, rH = O.tmunu(st)
    assert np.max(np.abs(tab[:, 0] - rtab[:, 0])) / np.max(rtab[:, 0]) < 1e-4


@pytest.mark.parametrize("nc", [2, 3])
def test_implicit_fp32_stops_at_its_rounding_level(G, nc):
    """FP32 semi-implicit steps with the default tolerance (1e-14, out of
    FP32's reach): the iteration must stop on its rounding-level rules
    (contraction bound or stagnation) within a few sweeps, and agree with
    the FP64 oracle iterated to 1e-14 as closely as the tolerance-stopped
    FP32 run does."""
    cfg = gi.small_config(nc, nz=64, nx=7, ny=6, a_z=0.5, dt=0.25,
                          sigma_l=1.5, steps=10)
    cfg.update(scheme="implicit", implicit_max_iter=60, precision="fp32")
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], nc, p.nx, p.ny, p.g2mu)
    h = G.glasma_init_mv(cfg, rho)
    iters = []
    for _ in range(cfg["steps"]):
        G.glasma_step(h, 1)
        iters.append(G.glasma_get_info(h).implicit_iters)
    assert max(iters) <= 12, iters
    st = O.step_implicit(O.init_mv(p, rho), cfg["steps"], tol=1e-14)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    assert rel(U, st.U) < 3e-5 and rel(E, st.E) < 3e-5


def test_improved_workload_full_size_properties(G):
    """The benchmarked improved-scheme configuration at full size (SU(3)
    2048 x 128^2, a_z = dt = a_T/4, FP32, the launch configuration of
    bench.py): properties that hold at any size, since the oracle cannot
    hold this lattice.  Every step converges within a few sweeps, the field
    energy is conserved to FP32 rounding over the steps (the nuclei are
    still apart) and the Gauss residual stays small against the charge."""
    cfg = dict(gi.CONFIGS["su3_2048x128x128_improved"])
    h = G.glasma_init_mv(cfg, None)
    _, H0 = G.glasma_tmunu(h)
    iters = []
    for _ in range(6):
        G.glasma_step(h, 1)
        iters.append(G.glasma_get_info(h).implicit_iters)
    _, H1 = G.glasma_tmunu(h)
    gmax, grms, rmax = G.glasma_gauss_residual(h)
    G.glasma_free(h)
    assert all(2 <= k <= 12 for k in iters), iters
    assert abs(H1 / H0 - 1.0) < 1e-5, (H0, H1)
    assert gmax < 1e-3 * rmax, (gmax, rmax)


def test_implicit_not_converged_is_reported(G):
    cfg = gi.small_config(2, nz=64, nx=7, ny=6, a_z=0.5, dt=0.25,
                          sigma_l=1.5, steps=3)
    cfg.update(scheme="implicit", implicit_tol=1e-30, implicit_max_iter=3)
    h = G.glasma_init_mv(cfg, None)
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_step(h, 1)
    assert e.value.code == "NOT_CONVERGED"
    # the step was still taken with the last iterate
    assert G.glasma_get_info(h).step_n == 1


def test_implicit_converges_where_plain_iteration_fails(G):
    """dt = a_T = a_z: the sweep's extreme contraction c = 2 dt^2 / a_T^2 = 2
    would make plain fixed-point iteration diverge; the relaxed sweeps
    contract by c / (2 + c) = 1/2 and converge, and the steps match the
    oracle's relaxed iteration at the FP64 target (both converged to
    1e-13, so the iteration path does not matter)."""
    cfg = gi.small_config(2, nz=48, nx=8, ny=8, a_z=1.0, dt=1.0, sigma_l=1.5,
                          steps=3)
    cfg.update(scheme="implicit", implicit_tol=1e-13, implicit_max_iter=80)
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    h = G.glasma_init_mv(cfg, rho)
    G.glasma_step(h, cfg["steps"])
    st = O.step_implicit(O.init_mv(p, rho), cfg["steps"], tol=1e-13, max_iter=80)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    assert rel(U, st.U) < TOL64 and rel(E, st.E) < TOL64
    assert abs(G.glasma_get_info(h).implicit_iters - st.extra["iters"]) <= 1


def _single_nucleus_energy(G, cfg, steps, every):
    nt = cfg["nx"]
    rho = gi.mv_rho(cfg["seed"], 2, nt, nt, cfg["g2mu"])
    rho[0] = 0.0                                   # nucleus B alone
    h = G.glasma_init_mv(cfg, rho)
    H = [G.glasma_tmunu(h)[1]]
    for _ in range(steps // every):
        G.glasma_step(h, every)
        H.append(G.glasma_tmunu(h)[1])
    return np.array(H)


def test_improved_scheme_is_stable_where_leapfrog_grows(G):
    """A single thin nucleus (sigma_L = 2 a_T = 4 a_z) crossing the box at
    a_z = 0.5 a_T: under the semi-implicit scheme at dt = a_z (dispersion
    free along z, a hop every step) the field energy stays constant; under
    leapfrog at the same a_z with dt = 0.375 (inside its Courant limit
    0.408) numerical Cherenkov radiation makes it grow (FP64 both)."""
    base = dict(nc=2, nz=640, nx=8, ny=8, a_t=1.0, a_z=0.5, sigma_l=2.0,
                g2mu=0.05, m_ir=0.1, seed=77, z_offset=145.0, precision="fp64")
    Hi = _single_nucleus_energy(G, dict(base, scheme="implicit", dt=0.5,
                                        implicit_tol=1e-13, implicit_max_iter=80), 500, 50)
    Hl = _single_nucleus_energy(G, dict(base, scheme="leapfrog", dt=0.375), 666, 66)
    assert np.max(np.abs(Hi / Hi[0] - 1)) < 1e-4
    # leapfrog: compare the same phase of its oscillation early and late
    assert np.max(Hl[-3:]) > 1.05 * np.max(Hl[:3])
    assert np.min(Hl[-3:]) > 1.05 * np.min(Hl[1:4])


# ---------------------------------------------------------------------------
# Longitudinal colour structure: several colour sheets per nucleus
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [2, 3])
def test_colour_sheets_match_oracle(G, nc):
    """Three independent colour sheets per nucleus (path-ordered Wilson
    line), host charges, through the collision in FP64."""
    S = 3
    cfg = dict(gi.small_config(nc, nz=64, nx=7, ny=6, sigma_l=3.0, seed=23), n_sheets=S)
    rho = gi.mv_rho(23, nc, 7, 6, cfg["g2mu"], sheets=S)
    p = O.Params.from_dict(cfg)
    h = G.glasma_init_mv(cfg, rho)
    compare_state(G, h, O.init_mv(p, rho), TOL64, "sheets init")
    G.glasma_step(h, 30)
    compare_state(G, h, O.step(O.init_mv(p, rho), 30), TOL64, "sheets 30 steps")


def test_colour_sheets_seed_only_init(G):
    """The device draw of the sheet charges (counter (x, y, a, N + 2 s))
    equals the host generator's."""
    S = 4
    cfg = dict(gi.small_config(2, nz=64, nx=5, ny=8, sigma_l=3.0, seed=99), n_sheets=S)
    p = O.Params.from_dict(cfg)
    h = G.glasma_init_mv(cfg, None)
    st = O.init_mv(p, gi.mv_rho(99, 2, 5, 8, cfg["g2mu"], sheets=S))
    compare_state(G, h, st, TOL64, "sheets seed init")
