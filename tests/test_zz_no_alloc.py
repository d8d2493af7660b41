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
    torch device tensors in the library's layout (SU(2) links and all
    fields as structure of arrays, SU(3) links in blocks of 32 sites with
    the nine components of a block stored one after another); the charge
    windows cover the whole lattice."""
    import torch
    p = h.params
    nc, na = p.nc, p.nc * p.nc - 1
    V = p.nz * p.ny * p.nx
    U, E, QA, QB, n = G.glasma_get_fields(h)
    U = U.reshape(3, V, nc, nc)
    if dtype == torch.float32:      # FP32 links are stored as U - 1
        U = U - np.eye(nc)
    if nc == 2:
        comp = np.stack([U[..., 0, 0], U[..., 0, 1]], axis=1)   # [3][2][V]
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


def test_static_residual_rejects_oversized_lattice(G):
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_gauss_residual_static(3, "fp64", 8193, 4, 4, 1.0, 1.0, 1, 1)
    assert e.value.code == "INVALID_ARG"
    assert "8192" in str(e.value)
