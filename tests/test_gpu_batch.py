"""GPU tests of the batched ensemble (glasma_batch_*): several independent
events of uneven lattice size advanced by one kernel per step must give
each event bitwise the state it gets alone from glasma_step with the same
step kernel (the batched graph and persistent modes run the staple kernel's
per-link arithmetic; the per-event mode launches each context's own
kernel), and one batched event must match the FP64 oracle."""
import numpy as np
import pytest

import glasma_inputs as gi
from oracle import glasma_oracle as O

pytestmark = pytest.mark.gpu

# uneven sizes: tails of 0..63 sites against every block shape, different nz
SIZES = [(48, 12, 10), (64, 7, 6), (40, 16, 16), (56, 9, 5), (48, 33, 3)]


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


def _cfgs(nc, precision):
    return [dict(gi.small_config(nc, nz=nz, nx=nx, ny=ny, seed=100 + k),
                 precision=precision)
            for k, (nz, nx, ny) in enumerate(SIZES)]


def _match_kernel(G, hs, mode):
    """Single-event references run the kernel the batch mode runs: the
    staple kernel for the batched graph and persistent modes."""
    for h in hs:
        G.glasma_set_step_kernel(h, "auto" if mode == "per_event" else "staple")


def _same(G, h1, h2):
    a = G.glasma_get_fields(h1)
    b = G.glasma_get_fields(h2)
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert a[4] == b[4]
    assert np.array_equal(G.glasma_tmunu(h1)[0], G.glasma_tmunu(h2)[0])


@pytest.mark.parametrize("mode", ["graph", "persistent", "per_event"])
@pytest.mark.parametrize("nc,precision", [(2, "fp64"), (3, "fp64"),
                                          (2, "fp32"), (3, "fp32")])
def test_batch_is_bitwise_the_single_event_step(G, nc, precision, mode):
    cfgs = _cfgs(nc, precision)
    single = [G.glasma_init_mv(c, None) for c in cfgs]
    batched = [G.glasma_init_mv(c, None) for c in cfgs]
    _match_kernel(G, single, mode)
    b = G.glasma_batch_create(batched)
    G.glasma_batch_set_shape(b, mode, 64)
    G.glasma_batch_step(b, 7)      # two calls: bookkeeping carried over
    G.glasma_batch_step(b, 13)
    G.glasma_batch_step(b, 0)
    for h in single:
        G.glasma_step(h, 20)
    for h1, h2 in zip(single, batched):
        assert G.glasma_get_info(h2).step_n == 20
        _same(G, h1, h2)
    b.close()


@pytest.mark.parametrize("mode", ["graph", "persistent"])
@pytest.mark.parametrize("block_sites", [32, 128])
def test_every_block_shape_is_bitwise(G, mode, block_sites):
    cfgs = _cfgs(3, "fp32")
    single = [G.glasma_init_mv(c, None) for c in cfgs]
    batched = [G.glasma_init_mv(c, None) for c in cfgs]
    _match_kernel(G, single, mode)
    b = G.glasma_batch_create(batched)
    G.glasma_batch_set_shape(b, mode, block_sites)
    G.glasma_batch_step(b, 11)
    for h in single:
        G.glasma_step(h, 11)
    for h1, h2 in zip(single, batched):
        _same(G, h1, h2)


def test_batched_event_matches_oracle(G):
    cfgs = _cfgs(2, "fp64")[:2]
    hs = [G.glasma_init_mv(c, None) for c in cfgs]
    b = G.glasma_batch_create(hs)
    G.glasma_batch_step(b, 16)
    for c, h in zip(cfgs, hs):
        p = O.Params.from_dict(c)
        st = O.step(O.init_mv(p, gi.mv_rho(c["seed"], p.nc, p.nx, p.ny,
                                           p.g2mu)), 16)
        U, E, QA, QB, n = G.glasma_get_fields(h)
        assert n == st.n
        for got, ref in ((U, st.U), (E, st.E), (QA, st.QA), (QB, st.QB)):
            assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tune_keeps_the_state_and_the_result(G, precision):
    cfgs = _cfgs(3, precision)
    single = [G.glasma_init_mv(c, None) for c in cfgs]
    batched = [G.glasma_init_mv(c, None) for c in cfgs]
    for h in single + batched:
        G.glasma_step(h, 3)
    b = G.glasma_batch_create(batched)
    bx, mode = G.glasma_batch_tune(b, 4)
    assert bx in (32, 64, 128) and mode in G.BATCH_MODES
    _match_kernel(G, single, mode)
    for h1, h2 in zip(single, batched):
        _same(G, h1, h2)            # tuning left every event as it was
    G.glasma_batch_step(b, 9)
    for h in single:
        G.glasma_step(h, 9)
    for h1, h2 in zip(single, batched):
        _same(G, h1, h2)


@pytest.mark.parametrize("mode", ["graph", "persistent", "per_event"])
def test_particle_exit_stops_every_event_at_the_same_step(G, mode):
    short = gi.small_config(2, nz=48, steps=0, seed=5)
    long_ = gi.small_config(2, nz=96, nx=6, ny=7, steps=0, seed=6)
    probe = G.glasma_init_mv(short, None)
    with pytest.raises(G.GlasmaError):
        G.glasma_step(probe, 400)
    n_exit = G.glasma_get_info(probe).step_n
    hs = [G.glasma_init_mv(c, None) for c in (short, long_)]
    b = G.glasma_batch_create(hs)
    G.glasma_batch_set_shape(b, mode, 64)
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_batch_step(b, 400)
    assert e.value.code == "PARTICLE_EXIT"
    for c, h in zip((short, long_), hs):
        assert G.glasma_get_info(h).step_n == n_exit
        ref = G.glasma_init_mv(c, None)
        _match_kernel(G, [ref], mode)
        G.glasma_step(ref, n_exit)
        _same(G, ref, h)


def test_batch_rejects_mixed_events(G):
    a = G.glasma_init_mv(gi.small_config(2), None)
    b32 = G.glasma_init_mv(dict(gi.small_config(2), precision="fp32"), None)
    su3 = G.glasma_init_mv(gi.small_config(3), None)
    imp = G.glasma_init_mv(dict(gi.small_config(2), scheme="implicit"), None)
    other_dt = G.glasma_init_mv(gi.small_config(2, dt=0.25), None)
    for bad in ([a, b32], [a, su3], [a, imp], [a, other_dt], [a, a]):
        with pytest.raises(G.GlasmaError) as e:
            G.glasma_batch_create(bad)
        assert e.value.code == "INVALID_ARG"


def test_barrier_wait_that_runs_out_returns_timeout(G):
    """Failure detection of the persistent mode: every barrier waits for one
    block that does not exist, so the first wait runs out after its budget
    (about half a millisecond here); the call returns TIMEOUT, the context
    stays usable and a checkpoint brings the events back."""
    cfgs = _cfgs(2, "fp32")[:3]
    hs = [G.glasma_init_mv(c, None) for c in cfgs]
    blobs = [G.glasma_get_state(h) for h in hs]
    b = G.glasma_batch_create(hs)
    G.glasma_batch_set_shape(b, "persistent", 64)
    G.glasma_batch_set_barrier(b, 1_000_000, extra_arrivals=1)
    G.glasma_batch_step(b, 1)          # one step has no barrier
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_batch_step(b, 3)
    assert e.value.code == "TIMEOUT"
    assert all(G.glasma_get_info(h).step_n == 1 for h in hs)
    G.glasma_batch_set_barrier(b, 2_000_000_000, extra_arrivals=0)
    for h, blob in zip(hs, blobs):
        G.glasma_set_state(h, blob)
    G.glasma_batch_step(b, 5)
    ref = [G.glasma_init_mv(c, None) for c in cfgs]
    _match_kernel(G, ref, "persistent")
    for h1, h2 in zip(ref, hs):
        G.glasma_step(h1, 5)
        _same(G, h1, h2)


def test_persistent_call_longer_than_one_launch(G):
    """150 steps: three cooperative launches of at most 64 steps, the hop
    schedule and the windows carried from one launch to the next."""
    cfgs = [dict(gi.small_config(2, nz=nz, nx=nx, ny=ny, seed=40 + k),
                 precision="fp32")
            for k, (nz, nx, ny) in enumerate([(200, 9, 8), (208, 16, 4)])]
    single = [G.glasma_init_mv(c, None) for c in cfgs]
    batched = [G.glasma_init_mv(c, None) for c in cfgs]
    _match_kernel(G, single, "persistent")
    b = G.glasma_batch_create(batched)
    G.glasma_batch_set_shape(b, "persistent", 64)
    G.glasma_batch_step(b, 150)
    assert G.glasma_get_info(batched[0]).kernel_launches == 3
    for h in single:
        G.glasma_step(h, 150)
    for h1, h2 in zip(single, batched):
        _same(G, h1, h2)
