"""GPU checks of the hand-written adjoint (glasma_adjoint_energy): the
gradient of the mid-rapidity energy with respect to the MV charges against
the oracle's autograd adjoint (small lattices, FP64), independence of the
checkpoint spacing, the torch.autograd.Function wrapper, and central finite
differences of the GPU forward on the SU(2) 256 x 32^2, 200-step workload."""
import numpy as np
import pytest

import glasma_inputs as gi
from oracle import adjoint as A
from oracle import glasma_oracle as O

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


SMALL = [
    (gi.small_config(2, nz=40, nx=5, ny=4, seed=3), 24, 8.0),
    (gi.small_config(2, nz=96, nx=4, ny=6, seed=9, a_z=0.5, dt=0.25), 30, 5.0),
    (gi.small_config(2, nz=56, nx=12, ny=10, seed=4), 33, 12.0),
    (gi.small_config(2, nz=40, nx=5, ny=4, seed=3), 0, 8.0),
]


@pytest.mark.parametrize("case", range(len(SMALL)))
def test_adjoint_matches_oracle_autograd(G, case):
    cfg, n, hw = SMALL[case]
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    val, g = G.glasma_adjoint_energy(cfg, rho, n, hw, checkpoint_every=7)
    o_ref, g_ref = A.gradient(p, rho, n, hw)
    assert abs(val - o_ref) <= 1e-11 * abs(o_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-11 * np.max(np.abs(g_ref))


def test_checkpoint_spacing_does_not_change_the_gradient(G):
    cfg, n, hw = SMALL[0]
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    ref = G.glasma_adjoint_energy(cfg, rho, n, hw, checkpoint_every=n)[1]
    for k in (1, 5, 24, 100):
        assert np.array_equal(G.glasma_adjoint_energy(cfg, rho, n, hw, checkpoint_every=k)[1], ref)


def test_autograd_function(G):
    import torch
    cfg, n, hw = SMALL[0]
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    r = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    val = G.mid_rapidity_energy(r, cfg, n, hw)
    (3.0 * val).backward()
    v2, g2 = G.glasma_adjoint_energy(cfg, rho, n, hw)
    assert val.item() == v2
    assert np.array_equal(r.grad.numpy(), 3.0 * g2)


def test_adjoint_rejects_what_it_does_not_cover(G):
    cfg = gi.small_config(3)
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_adjoint_energy(cfg, None, 2, 8.0)
    assert e.value.code == "INVALID_ARG"
    with pytest.raises(G.GlasmaError):
        G.glasma_adjoint_energy(dict(gi.small_config(2), scheme="implicit"), None, 2, 8.0)
    with pytest.raises(G.GlasmaError):
        G.glasma_adjoint_energy(dict(gi.small_config(2), n_sheets=2), None, 2, 8.0)


def test_fp32_forward_gradient_is_close_to_fp64(G):
    """FP32 forward and checkpoints, FP64 reverse pass on the FP32 states:
    the gradient of the FP32 trajectory, within FP32 rounding of the FP64
    gradient (1e-5 relative to its largest entry; 3e-7 measured after 33
    steps), and independent of the checkpoint spacing."""
    cfg, n, hw = SMALL[2]
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    v64, g64 = G.glasma_adjoint_energy(cfg, rho, n, hw, checkpoint_every=7)
    v32, g32 = G.glasma_adjoint_energy(dict(cfg, precision="fp32"), rho, n, hw, checkpoint_every=7)
    assert abs(v32 - v64) <= 1e-5 * v64
    assert np.max(np.abs(g32 - g64)) <= 1e-5 * np.max(np.abs(g64))
    g32b = G.glasma_adjoint_energy(dict(cfg, precision="fp32"), rho, n, hw, checkpoint_every=1)[1]
    assert np.array_equal(g32, g32b)


def test_central_differences_on_the_differentiated_workload(G):
    """SU(2) 256 x 32^2, dt = a/2, sigma_L = 4a, 200 steps, |z - z_c| < 16a:
    the adjoint against central differences (h = 1e-4) of the GPU forward
    at 64 random (nucleus, colour, site) entries, 1e-6 relative."""
    cfg = dict(gi.CONFIGS["su2_256x32x32"], precision="fp64")
    n, hw, h = cfg["steps"], 16.0, 1e-4
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    val, g = G.glasma_adjoint_energy(cfg, rho, n, hw, checkpoint_every=20)
    assert val > 0
    rng = np.random.default_rng(1404)
    errs = []
    for _ in range(64):
        idx = tuple(int(rng.integers(0, s)) for s in rho.shape)
        rp, rm = rho.copy(), rho.copy()
        rp[idx] += h
        rm[idx] -= h
        fp = G.glasma_adjoint_energy(cfg, rp, n, hw, grad=False)[0]
        fm = G.glasma_adjoint_energy(cfg, rm, n, hw, grad=False)[0]
        fd = (fp - fm) / (2 * h)
        errs.append(abs(g[idx] - fd) / max(abs(fd), 1e-3 * np.max(np.abs(g))))
    assert max(errs) <= 1e-6, max(errs)
