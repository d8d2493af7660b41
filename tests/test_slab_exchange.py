"""Host side of the multi-rank slab path (paper_2009_02044_gb300/slab.py),
on CPU gloo ranks: the halo messages reach the right neighbours, the
whole-lattice charge windows are the union of the ranks' own, the slab
bounds tile the lattice, and a halo message that never arrives ends the
exchange with a TIMEOUT status instead of hanging the rank."""
import datetime
import os
import socket
import time

import pytest

from paper_2009_02044_gb300 import slab as SL


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    return dist


def _deliver(rank, world, port, q):
    import torch
    dist = _init(rank, world, port)
    # message of rank r in direction d: a vector that names them
    send = {d: torch.full((64,), float(10 * rank + (1 if d > 0 else 2)))
            for d in (+1, -1) if 0 <= rank + d < world}
    recv = {d: torch.zeros(64) for d in send}
    SL.exchange_messages(send, recv, rank, world, timeout_s=20.0)
    ok = True
    for d, buf in recv.items():
        peer = rank + d
        # the neighbour above sent its downward message, the one below its
        # upward message
        want = 10 * peer + (2 if d > 0 else 1)
        ok = ok and bool((buf == want).all())
    q.put((rank, ok))
    dist.barrier()
    dist.destroy_process_group()


def test_messages_reach_the_neighbours():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_deliver, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = dict(q.get(timeout=5) for _ in range(3))
    assert res == {0: True, 1: True, 2: True}


def _dropped(rank, port, q):
    import torch
    from paper_2009_02044_gb300 import glasma as G
    dist = _init(rank, 2, port)
    if rank == 0:
        send = {+1: torch.zeros(16)}
        recv = {+1: torch.zeros(16)}
        t = time.time()
        try:
            SL.exchange_messages(send, recv, 0, 2, timeout_s=1.0)
            q.put(("returned", time.time() - t))
        except G.GlasmaError as e:
            q.put((e.code, time.time() - t))
    else:
        # rank 1 drops its message: it receives rank 0's and never sends
        buf = torch.zeros(16)
        dist.recv(buf, 0)
        time.sleep(3.0)
    # the timed-out pair is closed: no further collectives on this group


def test_dropped_halo_message_times_out():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dropped, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    code, waited = q.get(timeout=60)
    for p in procs:
        p.join(timeout=60)
    assert code == "TIMEOUT"
    assert 0.9 <= waited < 10.0


def test_window_union_and_bounds():
    w = [((30, 0), (4, 9)), ((20, 7), (13, 2)), ((27, 9), (0, 0))]
    assert SL.merge_windows(w) == ((20, 16), (4, 11))
    assert SL.merge_windows([((0, 0), (0, 0))]) == ((0, 0), (0, 0))
    for nz, P in ((512, 8), (47, 3), (5, 5)):
        b = SL.slab_bounds(nz, P)
        assert b[0][0] == 0 and b[-1][1] == nz
        assert all(b[k][1] == b[k + 1][0] for k in range(P - 1))


# ---------------------------------------------------------------------------
# the improved step's host loop (slab.implicit_step) with the device calls
# replaced by a scripted sequence of sweep maxima
# ---------------------------------------------------------------------------

class _FakeRank:
    def __init__(self, seq, maxit=10, tol=1e-30, precision="fp32"):
        self.seq = list(seq)
        self.maxit, self.tol, self.precision = maxit, tol, precision
        self.calls = []
        self.h = self


def _patch(monkeypatch):
    from paper_2009_02044_gb300 import glasma as G

    def begin(h):
        h.calls.append("begin")

    def sweep(h):
        h.calls.append("sweep")
        return h.seq.pop(0)

    def end(h):
        h.calls.append("end")

    monkeypatch.setattr(G, "glasma_implicit_begin", begin)
    monkeypatch.setattr(G, "glasma_implicit_sweep", sweep)
    monkeypatch.setattr(G, "glasma_implicit_end", end)
    return G


def test_implicit_step_folds_the_ranks_maxima(monkeypatch):
    """The stopping rule sees the max over ranks: rank 1's slow tail keeps
    both ranks sweeping although rank 0 alone would have stopped."""
    G = _patch(monkeypatch)
    u, emax = 2.0 ** -24, 0.01
    r0 = _FakeRank([(1e6 * u * emax, emax), (1e3 * u * emax, emax), (1.0 * u * emax, emax),
                    (0.5 * u * emax, emax)])
    r1 = _FakeRank([(1e6 * u * emax, emax), (1e5 * u * emax, emax), (1e4 * u * emax, emax),
                    (100 * u * emax, emax)])
    alone = SL.implicit_step([_FakeRank(r0.seq)], SL._fold_max)
    n = SL.implicit_step([r0, r1], SL._fold_max)
    assert alone == 3 and n == 4
    assert r0.calls == ["begin"] + ["sweep"] * 4 + ["end"] == r1.calls


def test_implicit_step_reports_failures(monkeypatch):
    G = _patch(monkeypatch)
    emax = 0.01
    r = _FakeRank([(0.1, emax)] * 3, maxit=3)
    with pytest.raises(G.GlasmaError) as e:       # no convergence: the step
        SL.implicit_step([r], SL._fold_max)       # is still committed
    assert e.value.code == "NOT_CONVERGED" and r.calls[-1] == "end"
    r = _FakeRank([(0.1, emax), (float("inf"), emax)])
    with pytest.raises(G.GlasmaError) as e:       # non-finite: left open
        SL.implicit_step([r], SL._fold_max)
    assert e.value.code == "NONFINITE" and "end" not in r.calls


def _fold_rank(rank, port, q):
    dist = _init(rank, 2, port)
    from paper_2009_02044_gb300 import slab as SLr
    T = SLr.DistTransport.__new__(SLr.DistTransport)
    T.group = None
    q.put((rank, T.fold([(1.0 + rank, 5.0 - rank)])))
    dist.barrier()
    dist.destroy_process_group()


def test_dist_fold_is_the_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fold_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res == {0: (2.0, 5.0), 1: (2.0, 5.0)}
