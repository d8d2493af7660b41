"""GPU tests of the C ABI's checkpoint, error and failure-detection paths.

Failures are made on the host (a corrupted blob, a NaN written through
set_fields, a run that would push a charge off the lattice); no test makes
the GPU fault."""
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


@pytest.mark.parametrize("scheme,precision", [("leapfrog", "fp32"), ("leapfrog", "fp64"),
                                              ("implicit", "fp32")])
def test_checkpoint_resume_is_bitwise(G, scheme, precision):
    cfg = dict(gi.small_config(3, nz=64, nx=7, ny=6, a_z=0.5, dt=0.25, sigma_l=1.5),
               scheme=scheme, precision=precision, implicit_tol=1e-7)
    h = G.glasma_init_mv(cfg, None)
    G.glasma_step(h, 5)
    blob = G.glasma_get_state(h)
    G.glasma_step(h, 7)
    a = G.glasma_get_fields(h)
    ta = G.glasma_tmunu(h)[0]
    h2 = G.glasma_init_mv(cfg, None)
    G.glasma_set_state(h2, blob)
    assert G.glasma_get_info(h2).step_n == 5
    G.glasma_step(h2, 7)
    b = G.glasma_get_fields(h2)
    tb = G.glasma_tmunu(h2)[0]
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert a[4] == b[4] == 12
    assert np.array_equal(ta, tb)


def test_corrupted_checkpoint_is_rejected(G):
    cfg = gi.small_config(2)
    h = G.glasma_init_mv(cfg, None)
    G.glasma_step(h, 3)
    blob = G.glasma_get_state(h)
    bad = blob.copy()
    bad[len(bad) // 2] ^= 0x40
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_set_state(h, bad)
    assert e.value.code == "CHECKSUM"
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_set_state(h, blob[:100])
    assert e.value.code == "INVALID_ARG"
    other = G.glasma_init_mv(gi.small_config(3), None)
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_set_state(other, blob)
    assert e.value.code == "INVALID_ARG"
    G.glasma_set_state(h, blob)           # the intact blob still loads


def test_nonfinite_state_is_detected(G):
    cfg = gi.small_config(2)
    h = G.glasma_init_mv(cfg, None)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    E[0, 10, 3, 4, 1] = np.nan
    G.glasma_set_fields(h, U, E, QA, QB, None, n)
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_gauss_residual(h)
    assert e.value.code == "NONFINITE"
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_tmunu(h)
    assert e.value.code == "NONFINITE"


def test_particle_exit_stops_before_the_offending_step(G):
    cfg = gi.small_config(2, nz=48, steps=0)
    h = G.glasma_init_mv(cfg, None)
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_step(h, 200)
    assert e.value.code == "PARTICLE_EXIT"
    info = G.glasma_get_info(h)
    n = info.step_n
    assert 0 < n < 200
    # the state left behind is the last complete step and is still usable
    gm, _, rm = G.glasma_gauss_residual(h)
    assert gm < 1e-12 * rm
    with pytest.raises(G.GlasmaError):
        G.glasma_step(h, 1)
    assert G.glasma_get_info(h).step_n == n


def test_zero_steps_and_vacuum(G):
    cfg = dict(gi.small_config(3), g2mu=0.0)
    h = G.glasma_init_mv(cfg, None)
    info = G.glasma_get_info(h)
    assert info.window_a[1] == 0 and info.window_b[1] == 0
    U0 = G.glasma_get_fields(h)[0]
    G.glasma_step(h, 0)
    assert G.glasma_get_info(h).step_n == 0
    G.glasma_step(h, 10)
    U1, E1, QA, QB, n = G.glasma_get_fields(h)
    assert np.array_equal(U0, U1) and not np.any(E1) and not np.any(QA)
    tab, H = G.glasma_tmunu(h)
    assert H == 0.0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_device_tmunu_table_equals_host_table(G, precision):
    """glasma_tmunu_device writes the same [nz][4] table as glasma_tmunu,
    bit for bit (SU(3) on a lattice whose site count is not a multiple of
    the 32-site link blocks)."""
    import torch
    cfg = dict(gi.small_config(3, nx=7, ny=5), precision=precision)
    assert (cfg["nz"] * cfg["nx"] * cfg["ny"]) % 32 != 0
    h = G.glasma_init_mv(cfg, None)
    G.glasma_step(h, 30)
    dev = torch.full((cfg["nz"], 4), float("nan"), dtype=torch.float64, device="cuda")
    G.glasma_tmunu_device(h, dev.data_ptr())
    torch.cuda.synchronize()
    tab, H = G.glasma_tmunu(h)
    assert np.array_equal(dev.cpu().numpy(), np.asarray(tab))


def test_allocator_without_16_byte_alignment_is_rejected(G):
    """The state arrays are read with 16-byte vector loads, so an allocator
    whose blocks are only 8-byte aligned is refused by glasma_init_mv,
    which gives every block back before it returns."""
    import ctypes as C
    import torch
    live = {}

    @G._ALLOC_FN
    def alloc(nbytes, stream, user):
        base = torch.cuda.caching_allocator_alloc(int(nbytes) + 16, torch.cuda.current_device())
        live[base + 8] = base
        return base + 8

    @G._FREE_FN
    def free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(live.pop(ptr))

    a = G.glasma_allocator()
    a.alloc, a.free, a.user = alloc, free, None
    p = G.make_params(gi.small_config(2))
    out = C.c_void_p()
    st = G.load_library().glasma_init_mv(C.byref(p), None, C.c_void_p(0), C.byref(a), C.byref(out))
    torch.cuda.synchronize()
    assert G.ERRORS[st] == "INVALID_ARG"
    assert "16-byte" in G.load_library().glasma_last_error_message().decode()
    assert not live and not out.value
