"""Pins of the adjoint oracle (oracle/adjoint.py): its torch forward is the
numpy oracle's (so autograd differentiates the pinned computation), its
gradient agrees with central finite differences of the numpy oracle, and
it respects the global colour-rotation invariance of the energy."""
import numpy as np
import pytest

import glasma_inputs as gi
from oracle import adjoint as A
from oracle import glasma_oracle as O

CASES = [  # (config, steps, half width): through the collision, with hops
    (gi.small_config(2, nz=40, nx=5, ny=4, seed=3), 24, 8.0),
    (gi.small_config(2, nz=48, nx=4, ny=6, seed=9, a_z=0.5, dt=0.25), 30, 5.0),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_torch_forward_is_the_numpy_oracle(case):
    cfg, n, hw = CASES[case]
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    o_np = A.observable_numpy(p, rho, n, hw)
    o_t, _ = A.gradient(p, rho, n, hw)
    assert o_np > 0
    assert abs(o_t - o_np) <= 1e-12 * o_np


@pytest.mark.parametrize("case", range(len(CASES)))
def test_gradient_matches_central_differences(case):
    cfg, n, hw = CASES[case]
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    _, g = A.gradient(p, rho, n, hw)
    rng = np.random.default_rng(17 + case)
    h = 1e-4
    for _ in range(5):
        idx = tuple(int(rng.integers(0, s)) for s in rho.shape)
        rp, rm = rho.copy(), rho.copy()
        rp[idx] += h
        rm[idx] -= h
        fd = (A.observable_numpy(p, rp, n, hw)
              - A.observable_numpy(p, rm, n, hw)) / (2 * h)
        assert abs(g[idx] - fd) <= 1e-7 * np.max(np.abs(g)), (idx, g[idx], fd)


def test_gradient_is_orthogonal_to_global_colour_rotations():
    """A global colour rotation of rho rotates every field and leaves the
    energy unchanged, so sum_{N,x} rho(x) x dO/drho(x) = 0 (colour cross
    product), while each term alone is not small."""
    cfg, n, hw = CASES[0]
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 2, p.nx, p.ny, p.g2mu)
    _, g = A.gradient(p, rho, n, hw)
    r = np.moveaxis(rho, 1, -1).reshape(-1, 3)
    gg = np.moveaxis(g, 1, -1).reshape(-1, 3)
    cross = np.cross(r, gg)
    assert np.max(np.abs(cross.sum(axis=0))) <= 1e-10 * np.sum(np.abs(cross))
