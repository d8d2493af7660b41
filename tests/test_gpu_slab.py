"""Slab contexts on one GPU (glasma_slab_*), exchanging their halo slices by
device copies (paper_2009_02044_gb300.slab.LocalTransport), against one
context of the whole lattice, bit for bit: the links, fields and charges of
every owned slice, the T^{mu nu}(z) rows, the total energy summed in z
order, and the Gauss residual maximum, through the collision.  The oracle
side of the same decomposition is tests/test_oracle_slab.py."""
import numpy as np
import pytest

import glasma_inputs as gi

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


def _run(G, cfg, nranks, steps, kernel):
    from paper_2009_02044_gb300 import slab as SL
    whole = G.glasma_init_mv(cfg, None)
    G.glasma_set_step_kernel(whole, kernel)
    ranks = [SL.SlabRank(cfg, r, nranks) for r in range(nranks)]
    for r in ranks:
        G.glasma_set_step_kernel(r.h, kernel)
    T = SL.LocalTransport(ranks)
    T.setup()
    for k in range(steps):
        T.step()
        G.glasma_step(whole, 1)
    T.exchange()                       # fresh halos for the observables
    return whole, ranks, T


def _compare(G, cfg, whole, ranks, T):
    from paper_2009_02044_gb300 import slab as SL
    U, E, QA, QB, n = G.glasma_get_fields(whole)
    for r in ranks:
        Ur, Er, QAr, QBr, nr = G.glasma_get_fields(r.h)
        z0, z1, nzl, lo, hi = r.h.slab
        assert nr == n
        assert np.array_equal(Ur[:, lo:hi], U[:, z0:z1]), (r.rank, "U")
        assert np.array_equal(Er[:, lo:hi], E[:, z0:z1]), (r.rank, "E")
        assert np.array_equal(QAr[lo:hi], QA[z0:z1]), (r.rank, "QA")
        assert np.array_equal(QBr[lo:hi], QB[z0:z1]), (r.rank, "QB")
    tab, H = G.glasma_tmunu(whole)
    rows = T.gather_rows()
    assert np.array_equal(rows, tab)
    assert SL.total_energy(cfg, rows) == H
    gw = G.glasma_gauss_residual(whole)
    gs = [G.glasma_gauss_residual(r.h) for r in ranks]
    assert max(g[0] for g in gs) == gw[0]
    assert max(g[2] for g in gs) == gw[2]
    # rms from the partial mean squares (summation order differs)
    nz = cfg["nz"]
    ms = sum(g[1] ** 2 * (r.z1 - r.z0) for g, r in zip(gs, ranks)) / nz
    assert abs(np.sqrt(ms) - gw[1]) <= 1e-12 * gw[1]
    # both nuclei crossed a slab boundary
    assert any(np.any(G.glasma_get_fields(r.h)[3] != 0) for r in ranks[1:])


@pytest.mark.parametrize("nc,precision,kernel", [
    (2, "fp64", "auto"), (3, "fp64", "auto"), (3, "fp64", "staple"),
    (2, "fp32", "staple"), (3, "fp32", "auto"), (3, "fp32", "plaquette")])
@pytest.mark.parametrize("nranks", [2, 3])
def test_slabs_match_the_whole_lattice(G, nc, precision, kernel, nranks):
    """The ragged 47 x 10 x 12 collision (odd nz, uneven slabs) for 44 steps:
    the nuclei meet at step 20 and the Glasma between them crosses the slab
    boundaries."""
    cfg = dict(gi.small_config(nc, nz=47, sigma_l=2.0), precision=precision)
    whole, ranks, T = _run(G, cfg, nranks, 44, kernel)
    _compare(G, cfg, whole, ranks, T)


def test_slabs_with_the_64x64_plane(G):
    """SU(3) FP64 with the 64 x 64 transverse plane (the plaquette kernel's
    blocks of rows with a -y halo) on 3 slabs through the collision."""
    cfg = dict(gi.small_config(3, nz=30, nx=64, ny=64, sigma_l=1.0), precision="fp64")
    whole, ranks, T = _run(G, cfg, 3, 24, "auto")
    _compare(G, cfg, whole, ranks, T)


def test_slab_rows_on_a_long_lattice(G):
    """SU(3) FP32 with 256 slices of 64 x 64 on 2 slabs: each slice's
    T^{mu nu} sums take the same order whatever the number of slices a
    context holds (the whole lattice's 256 against a slab's 129), so the
    gathered rows and H equal the whole lattice's bit for bit."""
    from paper_2009_02044_gb300 import slab as SL
    cfg = dict(gi.CONFIGS["su3_512x64x64"], nz=256, precision="fp32")
    whole, ranks, T = _run(G, cfg, 2, 4, "auto")
    tab, H = G.glasma_tmunu(whole)
    rows = T.gather_rows()
    assert np.array_equal(rows, tab)
    assert SL.total_energy(cfg, rows) == H
    for r in ranks:
        G.glasma_free(r.h)
    G.glasma_free(whole)


def test_slab_calls_reject_bad_use(G):
    from paper_2009_02044_gb300 import slab as SL
    cfg = gi.small_config(2, nz=47)
    r = SL.SlabRank(cfg, 0, 2)
    with pytest.raises(G.GlasmaError):          # windows not set yet
        G.glasma_step(r.h, 1)
    with pytest.raises(G.GlasmaError):          # no rank below rank 0
        G.glasma_slab_pack(r.h, -1, r.buf[("send", +1)].data_ptr())
    with pytest.raises(G.GlasmaError):          # improved scheme: sweep by sweep
        ri = SL.SlabRank(dict(cfg, scheme="implicit"), 0, 2)
        G.glasma_slab_set_windows(ri.h, *SL.merge_windows([ri.windows()]))
        G.glasma_step(ri.h, 1)
    with pytest.raises(G.GlasmaError):          # leapfrog context
        G.glasma_implicit_begin(r.h)
    with pytest.raises(G.GlasmaError):
        G.glasma_slab_init(cfg, 20, 60)
    with pytest.raises(G.GlasmaError):          # checkpoints are whole lattices
        G.glasma_get_state(r.h)
    G.glasma_slab_set_windows(r.h, *SL.merge_windows([r.windows()]))
    with pytest.raises(G.GlasmaError):          # one step per exchange
        G.glasma_step(r.h, 2)


# ---------------------------------------------------------------------------
# The improved scheme on slabs (glasma_implicit_begin / _sweep / _end)
# ---------------------------------------------------------------------------

def _implicit_cfg(nc, precision, nz=47, nx=10, ny=12):
    """a_z = 0.5, dt = 0.25 (a hop every other step); the nuclei meet after
    20 steps and cross the slab boundaries."""
    cfg = gi.small_config(nc, nz=nz, nx=nx, ny=ny, a_z=0.5, dt=0.25, sigma_l=1.0)
    cfg.update(scheme="implicit", implicit_max_iter=60, precision=precision,
               implicit_tol=1e-14 if precision == "fp64" else 1e-7)
    return cfg


@pytest.mark.parametrize("nc,precision", [(2, "fp64"), (3, "fp64"), (2, "fp32"), (3, "fp32")])
@pytest.mark.parametrize("nranks", [2, 3])
def test_implicit_slabs_match_the_whole_lattice(G, nc, precision, nranks):
    """The improved scheme on 2 and 3 slabs of the ragged 47 x 10 x 12
    collision for 30 steps, against one whole-lattice context (glasma_step,
    all sweeps queued at once): the same sweeps every step, and the owned
    slices, the T^{mu nu} rows, H and the Gauss residual maximum bit for
    bit."""
    from paper_2009_02044_gb300 import slab as SL
    cfg = _implicit_cfg(nc, precision)
    whole = G.glasma_init_mv(cfg, None)
    ranks = [SL.SlabRank(cfg, r, nranks) for r in range(nranks)]
    T = SL.LocalTransport(ranks)
    T.setup()
    for _ in range(30):
        sweeps = T.step()
        G.glasma_step(whole, 1)
        assert sweeps == G.glasma_get_info(whole).implicit_iters
        assert all(G.glasma_get_info(r.h).implicit_iters == sweeps for r in ranks)
    T.exchange()
    _compare(G, cfg, whole, ranks, T)
    for r in ranks:
        G.glasma_free(r.h)
    G.glasma_free(whole)


def test_implicit_sweeps_one_by_one_on_a_whole_lattice(G):
    """glasma_implicit_begin / _sweep / _end on an ordinary context equals
    glasma_step bit for bit (the host applies the same stopping rule)."""
    from paper_2009_02044_gb300 import slab as SL
    cfg = _implicit_cfg(3, "fp32", nz=40)
    a = G.glasma_init_mv(cfg, None)
    b = G.glasma_init_mv(cfg, None)
    r = SL.SlabRank.__new__(SL.SlabRank)
    r.h, r.tol, r.maxit, r.precision = b, cfg["implicit_tol"], cfg["implicit_max_iter"], "fp32"
    for _ in range(12):
        G.glasma_step(a, 1)
        assert SL.implicit_step([r], SL._fold_max) == G.glasma_get_info(a).implicit_iters
    fa, fb = G.glasma_get_fields(a), G.glasma_get_fields(b)
    for x, y in zip(fa[:4], fb[:4]):
        assert np.array_equal(x, y)
    with pytest.raises(G.GlasmaError):          # a sweep before begin
        G.glasma_implicit_sweep(b)
    with pytest.raises(G.GlasmaError):          # end without a step
        G.glasma_implicit_end(b)
    G.glasma_implicit_begin(b)
    with pytest.raises(G.GlasmaError):          # glasma_step while one is open
        G.glasma_step(b, 1)
    with pytest.raises(G.GlasmaError):          # observables wait for _end
        G.glasma_tmunu(b)
    with pytest.raises(G.GlasmaError):          # and so do transfers
        G.glasma_get_fields(b)
    with pytest.raises(G.GlasmaError):          # no sweep done yet
        G.glasma_implicit_end(b)
    G.glasma_free(a)
    G.glasma_free(b)


# ---------------------------------------------------------------------------
# Two processes, one slab each, exchanging through torch.distributed (gloo,
# messages staged through host memory; NCCL needs one GPU per rank)
# ---------------------------------------------------------------------------

def _dist_rank(rank, port, cfg, steps, q):
    import datetime
    import os
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2,
                            timeout=datetime.timedelta(seconds=120))
    torch.cuda.set_device(0)
    from paper_2009_02044_gb300 import glasma as G
    from paper_2009_02044_gb300 import slab as SL
    G.load_library()
    r = SL.SlabRank(cfg, rank, 2)
    T = SL.DistTransport(r, timeout_s=60.0)
    T.setup()
    sweeps = [T.step() for _ in range(steps)]
    T.exchange()
    rows = torch.from_numpy(np.ascontiguousarray(r.tmunu_rows()))
    if rank == 1:
        dist.send(rows, 0)
    else:
        n1 = SL.slab_bounds(cfg["nz"], 2)[1]
        other = torch.empty((n1[1] - n1[0], 4), dtype=torch.float64)
        dist.recv(other, 1)
        all_rows = np.concatenate([rows.numpy(), other.numpy()])
        whole = G.glasma_init_mv(cfg, None)
        ws = []
        for _ in range(steps):
            G.glasma_step(whole, 1)
            ws.append(G.glasma_get_info(whole).implicit_iters)
        tab, H = G.glasma_tmunu(whole)
        ok = bool(np.array_equal(all_rows, tab) and SL.total_energy(cfg, all_rows) == H)
        if cfg.get("scheme") == "implicit":
            ok = ok and sweeps == ws
        q.put(ok)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("scheme", ["leapfrog", "implicit"])
def test_two_processes_match_the_whole_lattice(G, scheme):
    """Two processes on the one GPU, each with its slab context, stepping
    through the collision with DistTransport: the gathered T^{mu nu} rows
    and H equal one whole-lattice context's bit for bit (under the improved
    scheme also the sweeps, folded with an allreduce every sweep)."""
    import socket
    import torch.multiprocessing as mp
    if scheme == "implicit":
        cfg = _implicit_cfg(3, "fp32")
    else:
        cfg = dict(gi.small_config(3, nz=47, sigma_l=2.0), precision="fp32")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_dist_rank, args=(r, port, cfg, 30, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True
