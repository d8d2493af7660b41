"""Pin of the oracle's per-site step evaluator (`step_at_sites`) against the
whole-lattice step (`step`).

`step_at_sites` is the checker of the full-size lattices whose complete
evolution the oracle cannot afford: it evaluates Sec. 3 Eq. lattice_1 (force
from the plaquettes U_{i,j} and U_{i,-j}), Eq. lattice_2 (U <- exp(i dt E) U)
and the NGP hop current of Eq. continuity with explicit neighbour indices.
It must agree with `step` (which is itself pinned by the dispersion, finite
difference, plaquette-centric, Gauss, continuity and time-reversal tests) at
every site: on hop and non-hop steps, isotropic and anisotropic spacings, the
open-z boundary slices, and with charges of both nuclei everywhere they may
be.  A flip of the backward-staple conjugation, of the i > j plaquette
orientation or of the A-nucleus transport changes E by O(1) at many sites."""
import itertools

import numpy as np
import pytest

import glasma_inputs as gi
from oracle import glasma_oracle as O


def _random_state(nc, nz, ny, nx, a_z, dt, n, seed):
    rng = np.random.default_rng(seed)
    p = O.Params(nc=nc, nz=nz, nx=nx, ny=ny, a_z=a_z, dt=dt, sigma_l=1.0)
    na = nc * nc - 1
    U = gi.near_identity_su(nc, (3, nz, ny, nx), rng, 0.4)
    U[2][nz - 1] = np.eye(nc)
    E = 0.3 * rng.standard_normal((3, nz, ny, nx, na))
    E[2][nz - 1] = 0.0
    # charges of both nuclei on every slice a hop may start from: B moves
    # +z (none on the last slice), A moves -z (none on the first slice)
    QB = 0.2 * rng.standard_normal((nz, ny, nx, na))
    QB[nz - 1] = 0.0
    QA = 0.2 * rng.standard_normal((nz, ny, nx, na))
    QA[0] = 0.0
    return O.State(p, U, E, QA, QB, n, U.copy())


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("a_z,dt", [(1.0, 0.5), (0.5, 0.25), (0.5, 0.5)])
@pytest.mark.parametrize("hop", [True, False])
def test_step_at_sites_matches_step_everywhere(nc, a_z, dt, hop):
    nz, ny, nx = 7, 4, 5
    pq = O.hop_ratio(O.Params(nc=nc, nz=nz, nx=nx, ny=ny, a_z=a_z, dt=dt))
    if not hop and pq == (1, 1):
        pytest.skip("dt = a_z hops on every step")
    n = next(m for m in range(16) if O.hop_at(m, pq) == hop)
    st = _random_state(nc, nz, ny, nx, a_z, dt, n, seed=100 * nc + 7 * n
                       + int(8 * a_z) + int(16 * dt))
    nxt = O.step(st, 1)
    sites = list(itertools.product(range(nz), range(ny), range(nx)))
    E_s, U_s = O.step_at_sites(st, sites)
    for k, (z, y, x) in enumerate(sites):
        for i in range(3):
            assert np.max(np.abs(E_s[k, i] - nxt.E[i][z, y, x])) <= 1e-14, \
                (z, y, x, i)
            assert np.max(np.abs(U_s[k, i] - nxt.U[i][z, y, x])) <= 1e-14, \
                (z, y, x, i)
    # the hop deposit is present exactly when scheduled, and it reaches the
    # boundary slices z = 0 (A lands there) and z = nz - 2 (B leaves it)
    nohop = O.step(O.State(st.p, st.U, st.E, 0 * st.QA, 0 * st.QB, st.n,
                           st.U), 1)
    dEz = np.abs(nxt.E[2] - nohop.E[2])
    if hop:
        assert np.min(np.max(dEz[0], axis=-1)) > 1e-3
        assert np.min(np.max(dEz[nz - 2], axis=-1)) > 1e-3
    else:
        assert np.max(dEz) == 0.0
    # the last slice has no z link: E_z stays zero, U_z the identity
    assert np.all(E_s[[k for k, s in enumerate(sites) if s[0] == nz - 1],
                      2] == 0.0)


def test_step_at_sites_on_a_collision():
    """Mid-collision MV state (both windows populated, fields everywhere),
    SU(3): every site of every slice."""
    cfg = gi.small_config(3, nz=24, nx=5, ny=4, sigma_l=1.0, steps=12)
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 3, p.nx, p.ny, p.g2mu)
    st = O.step(O.init_mv(p, rho), 6)
    for _ in range(2):          # one hop step and one plain step
        nxt = O.step(st, 1)
        sites = list(itertools.product(range(p.nz), range(p.ny), range(p.nx)))
        E_s, U_s = O.step_at_sites(st, sites)
        Eg = np.stack([nxt.E[i].reshape(-1, p.na) for i in range(3)], 1)
        Ug = np.stack([nxt.U[i].reshape(-1, 3, 3) for i in range(3)], 1)
        assert np.max(np.abs(E_s - Eg)) <= 1e-14
        assert np.max(np.abs(U_s - Ug)) <= 1e-14
        st = nxt
