"""The z-slab decomposition of the leapfrog step (oracle/slab.py) against the
monolithic oracle, bit for bit: every owned slice's links, fields and
charges, the T^{mu nu}(z) rows gathered in rank order, H summed in z order,
and the Gauss residual maximum folded across ranks.  In one process for 2, 3
and 4 ranks (uneven slabs, middle ranks with both halos), and as two gloo
ranks that exchange their halo slices as messages."""
import datetime
import os
import socket

import numpy as np
import pytest

import glasma_inputs as gi
from oracle import glasma_oracle as O
from oracle import slab as S


def _collision(nc, nz=44, nx=5, ny=4, steps=0):
    cfg = gi.small_config(nc, nz=nz, nx=nx, ny=ny, sigma_l=2.0)
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], nc, p.nx, p.ny, p.g2mu)
    return O.init_mv(p, rho)


def _check_against_monolithic(slabs, ref):
    for s in slabs:
        U, E, QA, QB = S.owned(s)
        assert np.array_equal(U, ref.U[:, s.z0:s.z1])
        assert np.array_equal(E, ref.E[:, s.z0:s.z1])
        assert np.array_equal(QA, ref.QA[s.z0:s.z1])
        assert np.array_equal(QB, ref.QB[s.z0:s.z1])
        assert s.st.n == ref.n
    rows = np.concatenate([S.tmunu_rows(s) for s in slabs])
    rtab, rH = O.tmunu(ref)
    assert np.array_equal(rows, rtab)
    assert S.energy_from_rows(ref.p, rows) == rH
    gm = max(S.gauss_partial(s)[0] for s in slabs)
    assert gm == O.gauss_residual(ref)[0]
    # the residual field itself on every owned slice (the divergence at a
    # slab's first slice reads E_z and U_z of the halo below)
    G = O.gauss_divergence(ref.U, ref.E, ref.p) - (ref.QA + ref.QB)
    for s in slabs:
        g = O.gauss_divergence(s.st.U, s.st.E, s.st.p) - (s.st.QA + s.st.QB)
        assert np.array_equal(g[s.lo:s.hi], G[s.z0:s.z1])


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("nranks", [2, 3, 4])
def test_slabs_in_process_match_monolithic(nc, nranks):
    """Through the collision (the nuclei cross slab boundaries in both
    directions, with hops on every other step)."""
    st = _collision(nc)
    steps = 40          # the nuclei meet at step 20; the Glasma then spreads
    slabs = S.run_in_process(st, nranks, steps)
    ref = O.step(st, steps)
    _check_against_monolithic(slabs, ref)
    # both nuclei have crossed a slab boundary
    assert any(np.any(S.owned(s)[3] != 0) for s in slabs[1:])
    assert any(np.any(S.owned(s)[2] != 0) for s in slabs[:-1])


@pytest.mark.parametrize("nc", [2, 3])
def test_slabs_on_a_random_state(nc):
    """Generic links, fields and charges of both nuclei on every slice a hop
    may start from: every part of the halo messages carries O(1) data."""
    rng = np.random.default_rng(11 + nc)
    nz, ny, nx = 17, 3, 4
    p = O.Params(nc=nc, nz=nz, nx=nx, ny=ny, a_z=0.5, dt=0.25, sigma_l=1.0)
    na = nc * nc - 1
    U = gi.near_identity_su(nc, (3, nz, ny, nx), rng, 0.4)
    U[2][nz - 1] = np.eye(nc)
    E = 0.3 * rng.standard_normal((3, nz, ny, nx, na))
    E[2][nz - 1] = 0.0
    QA = 0.2 * rng.standard_normal((nz, ny, nx, na))
    QB = 0.2 * rng.standard_normal((nz, ny, nx, na))
    QA[:3] = 0.0          # room for three hops of A down and B up
    QB[nz - 3:] = 0.0
    st = O.State(p, U, E, QA, QB, 0, U.copy())
    for nranks in (2, 3, 5):
        slabs = S.run_in_process(st, nranks, 5)
        _check_against_monolithic(slabs, O.step(st, 5))


def test_slab_bounds_cover_the_lattice():
    for nz, P in ((44, 3), (7, 7), (100, 8)):
        b = S.slab_bounds(nz, P)
        assert b[0][0] == 0 and b[-1][1] == nz
        assert all(b[k][1] == b[k + 1][0] for k in range(P - 1))
        assert max(z1 - z0 for z0, z1 in b) - min(z1 - z0 for z0, z1 in b) <= 1


# ---------------------------------------------------------------------------
# two gloo ranks, halo slices as messages
# ---------------------------------------------------------------------------

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _send(dist, torch, m, dst):
    for k in sorted(m):
        dist.send(torch.from_numpy(np.ascontiguousarray(m[k])).view(torch.uint8).flatten(), dst)


def _recv(dist, torch, like, src):
    out = {}
    for k in sorted(like):
        buf = torch.empty(like[k].nbytes, dtype=torch.uint8)
        dist.recv(buf, src)
        out[k] = buf.numpy().view(like[k].dtype).reshape(like[k].shape).copy()
    return out


def _gloo_rank(rank, port, nc, steps, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2,
                            timeout=datetime.timedelta(seconds=60))
    st = _collision(nc)
    z0, z1 = S.slab_bounds(st.p.nz, 2)[rank]
    s = S.make_slab(st, z0, z1)
    for _ in range(steps + 1):
        # rank 0 sends up then receives from above; rank 1 the reverse
        if rank == 0:
            _send(dist, torch, S.message_up(s), 1)
            S.receive_from_above(s, _recv(dist, torch, S.message_down(s), 1))
        else:
            S.receive_from_below(s, _recv(dist, torch, S.message_up(s), 0))
            _send(dist, torch, S.message_down(s), 0)
        if _ < steps:
            S.local_step(s)
    rows = S.tmunu_rows(s)
    part = S.gauss_partial(s)
    U, E, QA, QB = S.owned(s)
    if rank == 1:
        _send(dist, torch, dict(U=U, E=E, QA=QA, QB=QB, rows=rows,
                                g=np.array(part[:1])), 0)
    else:
        r1 = S.make_slab(st, *S.slab_bounds(st.p.nz, 2)[1])
        like = dict(zip(("U", "E", "QA", "QB"), S.owned(r1)))
        like.update(rows=np.zeros((r1.hi - r1.lo, 4)), g=np.zeros(1))
        other = _recv(dist, torch, like, 1)
        ref = O.step(st, steps)
        ok = (np.array_equal(U, ref.U[:, :z1]) and np.array_equal(E, ref.E[:, :z1])
              and np.array_equal(QA, ref.QA[:z1]) and np.array_equal(QB, ref.QB[:z1])
              and np.array_equal(other["U"], ref.U[:, z1:])
              and np.array_equal(other["E"], ref.E[:, z1:])
              and np.array_equal(other["QA"], ref.QA[z1:])
              and np.array_equal(other["QB"], ref.QB[z1:]))
        all_rows = np.concatenate([rows, other["rows"]])
        rtab, rH = O.tmunu(ref)
        ok = ok and np.array_equal(all_rows, rtab) and S.energy_from_rows(ref.p, all_rows) == rH
        ok = ok and max(part[0], other["g"][0]) == O.gauss_residual(ref)[0]
        q.put(bool(ok))
    dist.destroy_process_group()


@pytest.mark.parametrize("nc", [2, 3])
def test_two_gloo_ranks_match_monolithic(nc):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, port, nc, 24, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True
