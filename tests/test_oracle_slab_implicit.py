"""The improved scheme (oracle.glasma_oracle.step_implicit) decomposed into
z slabs (oracle/slab.py) against the monolithic oracle, bit for bit: the
step's halo slices (with U(t_{n-1})'s z link of the lower one), each rank
evaluating the iterate's z link of its lower halo slice itself, and the
stopping test on the largest change folded across ranks, so that every
rank takes the same sweeps as the monolithic step.  In one process for 2
to 4 ranks, and as two gloo ranks that exchange their halos as messages
and fold the change with an allreduce."""
import datetime
import os
import socket

import numpy as np
import pytest

import glasma_inputs as gi
from oracle import glasma_oracle as O
from oracle import slab as S


def _collision(nc, nz=28, nx=4, ny=3):
    """a_z = 2 dt (hop every other step); the nuclei (sigma_L = 1) meet
    after 20 steps."""
    cfg = gi.small_config(nc, nz=nz, nx=nx, ny=ny, sigma_l=1.0)
    cfg.update(a_z=0.5, dt=0.25)
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], nc, p.nx, p.ny, p.g2mu)
    return O.init_mv(p, rho)


def _check(slabs, ref):
    for s in slabs:
        U, E, QA, QB = S.owned(s)
        assert np.array_equal(U, ref.U[:, s.z0:s.z1])
        assert np.array_equal(E, ref.E[:, s.z0:s.z1])
        assert np.array_equal(QA, ref.QA[s.z0:s.z1])
        assert np.array_equal(QB, ref.QB[s.z0:s.z1])
        assert np.array_equal(s.st.U_prev[:, s.lo:s.hi], ref.U_prev[:, s.z0:s.z1])
        assert s.st.n == ref.n
        assert s.st.extra["iters"] == ref.extra["iters"]
    rows = np.concatenate([S.tmunu_rows(s) for s in slabs])
    rtab, rH = O.tmunu(ref)
    assert np.array_equal(rows, rtab)
    assert S.energy_from_rows(ref.p, rows) == rH


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("nranks", [2, 4])
def test_implicit_slabs_through_the_collision(nc, nranks):
    st = _collision(nc)
    steps = 24
    slabs = S.run_implicit_in_process(st, nranks, steps, tol=1e-13)
    ref = O.step_implicit(st, steps, tol=1e-13)
    _check(slabs, ref)
    # both nuclei crossed a slab boundary
    assert any(np.any(S.owned(s)[3] != 0) for s in slabs[1:])
    assert any(np.any(S.owned(s)[2] != 0) for s in slabs[:-1])


def _random_state(nc, seed):
    """Generic links, fields, U(t_{n-1}) and charges of both nuclei."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = 13, 3, 4
    p = O.Params(nc=nc, nz=nz, nx=nx, ny=ny, a_z=0.5, dt=0.25, sigma_l=1.0)
    na = nc * nc - 1
    U = gi.near_identity_su(nc, (3, nz, ny, nx), rng, 0.4)
    Up = gi.near_identity_su(nc, (3, nz, ny, nx), rng, 0.4)
    U[2][nz - 1] = np.eye(nc)
    Up[2][nz - 1] = np.eye(nc)
    E = 0.3 * rng.standard_normal((3, nz, ny, nx, na))
    E[2][nz - 1] = 0.0
    QA = 0.2 * rng.standard_normal((nz, ny, nx, na))
    QB = 0.2 * rng.standard_normal((nz, ny, nx, na))
    QA[:2] = 0.0
    QB[nz - 2:] = 0.0
    return O.State(p, U, E, QA, QB, 0, Up)


@pytest.mark.parametrize("nc", [2, 3])
def test_implicit_slabs_on_a_random_state(nc):
    """Every part of the step's halo carries O(1) data."""
    st = _random_state(nc, 21 + nc)
    ref = O.step_implicit(st, 3, tol=1e-12)
    for nranks in (2, 3):
        _check(S.run_implicit_in_process(st, nranks, 3, tol=1e-12), ref)


def test_lower_halo_iterate_equals_the_owners():
    """After every sweep, the z links of the iterate that a rank evaluates
    on its lower halo slice equal, bit for bit, those its lower neighbour
    evaluates on its top owned slice: the sweeps need no messages."""
    st = _collision(3)
    seen = []

    def check(slabs):
        for r in range(1, len(slabs)):
            a = slabs[r].work["X"][2][0]
            b = slabs[r - 1].work["X"][2][slabs[r - 1].hi - 1]
            seen.append(bool(np.array_equal(a, b)))

    S.run_implicit_in_process(st, 3, 22, tol=1e-13, on_sweep=check)
    assert len(seen) > 100 and all(seen)


def test_uprev_halo_is_needed():
    """The t_{n-1} slot reads U(t_{n-1})'s z link of the lower halo slice:
    with the slabs' halos of U_prev left blank (message without it), the
    first step of a state whose z links are not the identity already leaves
    the monolithic result."""
    st = _random_state(2, 5)
    slabs = [S.make_slab(st, z0, z1) for z0, z1 in S.slab_bounds(st.p.nz, 2)]
    ups = [S.message_up(s) for s in slabs]
    downs = [S.message_down(s) for s in slabs]
    ups[0].pop("Uprev_z")
    S.receive_from_below(slabs[1], ups[0])
    S.receive_from_above(slabs[0], downs[1])
    for s in slabs:
        S.implicit_begin(s)
    for it in range(100):
        if max(S.implicit_sweep(s, it) for s in slabs) < 1e-12:
            break
    for s in slabs:
        S.implicit_end(s, it + 1)
    ref = O.step_implicit(st, 1, tol=1e-12)
    assert np.array_equal(S.owned(slabs[0])[1], ref.E[:, :slabs[0].z1])
    assert not np.array_equal(S.owned(slabs[1])[1], ref.E[:, slabs[1].z0:])


# ---------------------------------------------------------------------------
# two gloo ranks
# ---------------------------------------------------------------------------

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _send(dist, torch, a, dst):
    dist.send(torch.from_numpy(np.ascontiguousarray(a)).view(torch.uint8).flatten(), dst)


def _recv(dist, torch, like, src):
    buf = torch.empty(like.nbytes, dtype=torch.uint8)
    dist.recv(buf, src)
    return buf.numpy().view(like.dtype).reshape(like.shape).copy()


def _send_msg(dist, torch, m, dst):
    for k in sorted(m):
        _send(dist, torch, m[k], dst)


def _recv_msg(dist, torch, like, src):
    return {k: _recv(dist, torch, like[k], src) for k in sorted(like)}


def _gloo_rank(rank, port, nc, steps, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2,
                            timeout=datetime.timedelta(seconds=120))
    st = _collision(nc)
    bounds = S.slab_bounds(st.p.nz, 2)
    s = S.make_slab(st, *bounds[rank])

    def halo():
        if rank == 0:
            _send_msg(dist, torch, S.message_up(s), 1)
            S.receive_from_above(s, _recv_msg(dist, torch, S.message_down(s), 1))
        else:
            S.receive_from_below(s, _recv_msg(dist, torch, S.message_up(s), 0))
            _send_msg(dist, torch, S.message_down(s), 0)

    iters = []
    for _ in range(steps):
        halo()
        S.implicit_begin(s)
        for it in range(100):
            d = torch.tensor([S.implicit_sweep(s, it)], dtype=torch.float64)
            dist.all_reduce(d, op=dist.ReduceOp.MAX)
            if float(d[0]) < 1e-13:
                break
        S.implicit_end(s, it + 1)
        iters.append(it + 1)
    halo()
    U, E, QA, QB = S.owned(s)
    if rank == 1:
        for a in (U, E, QA, QB):
            _send(dist, torch, a, 0)
    else:
        r1 = S.make_slab(st, *bounds[1])
        other = [_recv(dist, torch, a, 1) for a in S.owned(r1)]
        ref = O.step_implicit(st, steps, tol=1e-13)
        z1 = bounds[0][1]
        ok = (np.array_equal(U, ref.U[:, :z1]) and np.array_equal(E, ref.E[:, :z1])
              and np.array_equal(QA, ref.QA[:z1]) and np.array_equal(QB, ref.QB[:z1])
              and np.array_equal(other[0], ref.U[:, z1:]) and np.array_equal(other[1], ref.E[:, z1:])
              and np.array_equal(other[2], ref.QA[z1:]) and np.array_equal(other[3], ref.QB[z1:])
              and iters[-1] == ref.extra["iters"])
        q.put(bool(ok))
    dist.destroy_process_group()


def test_two_gloo_ranks_implicit():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, port, 3, 8, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True
