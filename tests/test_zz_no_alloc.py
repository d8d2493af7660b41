"""The allocation-free Gauss residual (glasma_gauss_residual_static).

Some callers cannot allocate device memory: a health check that must run
after the device is out of memory, or code inside a framework whose
allocator owns all device memory.  This entry point takes the caller's own
device fields and uses a fixed scratch array inside the library.  The test
lays out a context's fields in caller-owned device buffers, calls the new
entry point through the C ABI twice in a row (on two different states) and
compares each result with glasma_gauss_residual on the same state.  It
lives in a file of its own that pytest collects last."""
import numpy as np
import pytest

import glasma_inputs as gi

pytestmark = pytest.mark.gpu

TOL = 1e-11   # the FP64 parity tolerance used by the other GPU tests


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


def _device_layout(G, h, dtype):
    """Copy a context's fields (via glasma_get_fields) into caller-owned
    torch device tensors in the library's layout (fields as structure of
    arrays, SU(2) links with the alpha and beta of one link adjacent,
    SU(3) links in blocks of 32 sites with the nine components of a block
    stored one after another); the charge windows cover the whole
    lattice."""
    import torch
    p = h.params
    nc, na = p.nc, p.nc * p.nc - 1
    V = p.nz * p.ny * p.nx
    U, E, QA, QB, n = G.glasma_get_fields(h)
    U = U.reshape(3, V, nc, nc)
    if dtype == torch.float32:      # FP32 links are stored as U - 1
        U = U - np.eye(nc)
    if nc == 2:
        comp = np.stack([U[..., 0, 0], U[..., 0, 1]], axis=-1)  # [3][V][2]
    else:                                                       # [3][C][9][32]
        C = (V + 31) // 32
        pad = np.zeros((3, C * 32, 9), dtype=complex)
        pad[:, :V] = U.reshape(3, V, 9)
        comp = np.moveaxis(pad.reshape(3, C, 32, 9), 3, 2)
    u = np.stack([comp.real, comp.imag], axis=-1)
    e = np.moveaxis(E.reshape(3, V, na), 2, 1)                  # [3][na][V]
    qa = np.moveaxis(QA.reshape(p.nz, p.ny * p.nx, na), 2, 0)   # [na][nz][nxy]
    qb = np.moveaxis(QB.reshape(p.nz, p.ny * p.nx, na), 2, 0)
    dev = [torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)
           for x in (u, e, qa, qb)]
    torch.cuda.synchronize()
    return dev


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nc,nx,ny", [(3, 12, 10), (3, 7, 5), (2, 7, 5)])
def test_static_residual_matches_context_residual(G, precision, nc, nx, ny):
    """(3, 7, 5): the SU(3) link array ends in a padded block of 32 sites."""
    import torch
    cfg = dict(gi.small_config(nc, nx=nx, ny=ny), precision=precision)
    h = G.glasma_init_mv(cfg, None)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    p = h.params
    stream = torch.cuda.current_stream()
    for call in range(2):                 # two calls in a row
        G.glasma_step(h, 7)
        ref = G.glasma_gauss_residual(h)
        u, e, qa, qb = _device_layout(G, h, dtype)
        got = G.glasma_gauss_residual_static(
            p.nc, precision, p.nz, p.ny, p.nx, p.a_t, p.a_z,
            u.data_ptr(), e.data_ptr(), qa.data_ptr(), 0, p.nz,
            qb.data_ptr(), 0, p.nz, stream=stream)
        for g, r in zip(got, ref):
            assert abs(g - r) <= TOL * abs(r), (call, got, ref)
        assert ref[0] > 0 and ref[2] > 0


def _windows_layout(G, h, dtype, with_b=True):
    """The context's own charge windows (first slice and width from
    glasma_get_info), with only those slices copied to the device."""
    import torch
    p = h.params
    na = p.nc * p.nc - 1
    info = G.glasma_get_info(h)
    _, _, QA, QB, _ = G.glasma_get_fields(h)
    out = []
    for Q, (z0, W) in ((QA, info.window_a), (QB, info.window_b)):
        if W == 0 or (Q is QB and not with_b):
            out.append((None, 0, 0))
            continue
        q = np.moveaxis(Q.reshape(p.nz, p.ny * p.nx, na)[z0:z0 + W], 2, 0)
        out.append((torch.from_numpy(np.ascontiguousarray(q)).to("cuda", dtype),
                    z0, W))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_residual_with_context_windows(G, precision):
    """Narrow windows at their own offsets (the ka/kb arithmetic), then a
    state without nucleus B (QB = NULL, WB = 0), each against
    glasma_gauss_residual; the free device memory is the same before and
    after a call."""
    import torch
    cfg = dict(gi.small_config(3, nx=7, ny=5), precision=precision)
    h = G.glasma_init_mv(cfg, None)
    dtype = torch.float64 if precision == "fp64" else torch.float32
    p = h.params
    stream = torch.cuda.current_stream()
    G.glasma_step(h, 9)
    ref = G.glasma_gauss_residual(h)
    u, e, _, _ = _device_layout(G, h, dtype)
    (qa, za, wa), (qb, zb, wb) = _windows_layout(G, h, dtype)
    assert 0 < wa < p.nz and 0 < wb < p.nz and za > 0
    args = (p.nc, precision, p.nz, p.ny, p.nx, p.a_t, p.a_z, u.data_ptr(),
            e.data_ptr(), qa.data_ptr(), za, wa, qb.data_ptr(), zb, wb)
    got = G.glasma_gauss_residual_static(*args, stream=stream)
    for g, r in zip(got, ref):
        assert abs(g - r) <= TOL * abs(r), (got, ref)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got2 = G.glasma_gauss_residual_static(*args, stream=stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert got2 == got
    # drop nucleus B from the context: its residual and the static one
    # (QB = NULL, WB = 0) see the same charge density
    U, E, QA, QB, n = G.glasma_get_fields(h)
    G.glasma_set_fields(h, U, E, QA, np.zeros_like(QB), None, n)
    assert G.glasma_get_info(h).window_b[1] == 0
    ref = G.glasma_gauss_residual(h)
    (qa, za, wa), (qb, zb, wb) = _windows_layout(G, h, dtype, with_b=False)
    assert qb is None and wb == 0
    got = G.glasma_gauss_residual_static(
        p.nc, precision, p.nz, p.ny, p.nx, p.a_t, p.a_z, u.data_ptr(),
        e.data_ptr(), qa.data_ptr(), za, wa, None, 0, 0, stream=stream)
    for g, r in zip(got, ref):
        assert abs(g - r) <= TOL * abs(r), (got, ref)
    assert ref[0] > 1e-6      # the dropped charge violates Gauss's law


def test_static_residual_rejects_oversized_lattice(G):
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_gauss_residual_static(3, "fp64", 8193, 4, 4, 1.0, 1.0, 1, 1)
    assert e.value.code == "INVALID_ARG"
    assert "8192" in str(e.value)
