"""The leapfrog step kernels (staple form, plaquette-centric form, site
pairs and the staged staple form, glasma_set_step_kernel) against the FP64
oracle and one another, through the C ABI.

The plaquette kernel splits the lattice into blocks of whole transverse rows
with a -y halo row, marching through z in chunks with a warm-up slice; the
cases below cover a block that holds the whole plane (no halo), blocks whose
row count divides ny, a ragged last block (ny prime), the 64 x 64 transverse
plane of the SU(3) 512 x 64^2 workload, chunks of one slice and chunks that
cross the collision, and both block shapes.  Tolerance: the FP64 target,
1e-11 relative to the largest reference entry."""
import numpy as np
import pytest

import glasma_inputs as gi
from oracle import glasma_oracle as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
KERNELS = ["staple", "plaquette", "plaquette_256"]


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


def rel(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def _random_state(nc, nz, ny, nx, seed):
    """Generic links (near the identity, amplitude 0.3), fields and charges
    of both nuclei, so every plaquette orientation and both hop directions
    carry O(1) contributions."""
    rng = np.random.default_rng(seed)
    p = O.Params(nc=nc, nz=nz, nx=nx, ny=ny, a_z=0.5, dt=0.25, sigma_l=1.0)
    na = nc * nc - 1
    U = gi.near_identity_su(nc, (3, nz, ny, nx), rng, 0.3)
    U[2][nz - 1] = np.eye(nc)
    E = 0.3 * rng.standard_normal((3, nz, ny, nx, na))
    E[2][nz - 1] = 0.0
    QA = np.zeros((nz, ny, nx, na))
    QB = np.zeros((nz, ny, nx, na))
    QA[nz // 2 + 1: nz - 2] = 0.1 * rng.standard_normal(QA[nz // 2 + 1: nz - 2].shape)
    QB[2: nz // 2 - 1] = 0.1 * rng.standard_normal(QB[2: nz // 2 - 1].shape)
    return O.State(p, U, E, QA, QB, 0, U.copy())


def _ctx(G, st, precision="fp64"):
    p = st.p
    # a placeholder event (no charge, thin nuclei that fit a short box);
    # set_fields then replaces its whole state
    cfg = dict(nc=p.nc, nz=p.nz, nx=p.nx, ny=p.ny, a_t=1.0, a_z=p.a_z,
               dt=p.dt, sigma_l=0.05, z_offset=0.3, g2mu=0.0, m_ir=0.2,
               seed=0, precision=precision)
    h = G.glasma_init_mv(cfg, None)
    G.glasma_set_fields(h, st.U, st.E, st.QA, st.QB, None, st.n)
    return h


# (nz, ny, nx): whole plane in one block; rows dividing ny; ny prime
# (ragged last block); the 64 x 64 plane of the throughput workload
SHAPES = [(12, 6, 13), (10, 40, 17), (9, 37, 17), (8, 64, 64)]


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kernel", KERNELS)
def test_kernel_matches_oracle_on_random_state(G, nc, shape, kernel):
    nz, ny, nx = shape
    st = _random_state(nc, nz, ny, nx, seed=7 * nz + ny + nc)
    ref = O.step(st, 3)                  # hops at steps 0 and 2
    for zlen in ([0] if kernel == "staple" else [0, 1, 3, nz]):
        h = _ctx(G, st)
        G.glasma_set_step_kernel(h, kernel, zlen)
        G.glasma_step(h, 3)
        U, E, QA, QB, n = G.glasma_get_fields(h)
        assert n == 3
        errs = dict(U=rel(U, ref.U), E=rel(E, ref.E), QA=rel(QA, ref.QA),
                    QB=rel(QB, ref.QB))
        assert all(v <= TOL64 for v in errs.values()), (kernel, zlen, errs)
        G.glasma_free(h)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_plaquette_result_does_not_depend_on_the_chunks(G, precision):
    """Every chunk of z slices starts with a warm-up iteration of the same
    code, so the state is bitwise the same for any chunk length (and for any
    split of the lattice into slabs)."""
    st = _random_state(3, 14, 40, 17, seed=5)
    out = []
    for zlen in (1, 3, 4, 14):
        h = _ctx(G, st, precision)
        G.glasma_set_step_kernel(h, "plaquette", zlen)
        G.glasma_step(h, 3)
        out.append(G.glasma_get_fields(h)[:4])
    for other in out[1:]:
        for x, y in zip(out[0], other):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("shape", [(8, 64, 64), (9, 37, 17), (13, 5, 9)])
@pytest.mark.parametrize("kernel", KERNELS + ["staple_pairs"])
def test_fp32_kernels_match_oracle(G, nc, shape, kernel):
    """FP32 state: each kernel against the FP64 oracle on random states; odd
    nz puts the paired kernel's last lane past the lattice, and its second
    lane meets the open z boundary on its own.  Bound: per step E and U
    round at u = 6e-8 relative to O(1) entries, and the four plaquette
    contributions of a link sum a few such roundings; 3 steps stay below
    3 * 8 * u ~ 1.5e-6 of the largest entry."""
    nz, ny, nx = shape
    st = _random_state(nc, nz, ny, nx, seed=99 + nz)
    ref = O.step(st, 3)
    h = _ctx(G, st, "fp32")
    G.glasma_set_step_kernel(h, kernel)
    G.glasma_step(h, 3)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    errs = dict(U=rel(U, ref.U), E=rel(E, ref.E), QA=rel(QA, ref.QA),
                QB=rel(QB, ref.QB))
    assert all(v < 1.5e-6 for v in errs.values()), errs


@pytest.mark.parametrize("nc", [2, 3])
def test_paired_kernel_through_a_collision_fp32(G, nc):
    """The paired staple kernel on the ragged 47 x 10 x 12
    collision (odd nz) through the crossing, against the FP64 oracle at the
    FP32 bound of the other collision tests, and against the one-site staple
    kernel at the rounding level of 40 steps."""
    cfg = dict(gi.small_config(nc, nz=47, sigma_l=2.0), precision="fp32")
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], nc, p.nx, p.ny, p.g2mu)
    st = O.step(O.init_mv(p, rho), 40)
    got = {}
    for kernel in ("staple_pairs", "staple"):
        h = G.glasma_init_mv(cfg, rho)
        G.glasma_set_step_kernel(h, kernel)
        G.glasma_step(h, 40)
        got[kernel] = G.glasma_get_fields(h)
        tab, H = G.glasma_tmunu(h)
        rtab, rH = O.tmunu(st)
        assert np.max(np.abs(tab[:, 0] - rtab[:, 0])) / np.max(rtab[:, 0]) < 1e-5
        U, E, QA, QB, n = got[kernel]
        assert rel(U, st.U) < 3e-5 and rel(E, st.E) < 3e-5
        assert rel(QA, st.QA) < 3e-5 and rel(QB, st.QB) < 3e-5
        gmax, grms, rmax = G.glasma_gauss_residual(h)
        assert gmax < 1e-5 * rmax
    for a, b in zip(got["staple_pairs"][:4], got["staple"][:4]):
        assert rel(a, b) < 3e-5


def test_su3_64x64_collision_fp64_full_state(G):
    """SU(3) with the 64 x 64 transverse plane of the throughput workload,
    FP64, 20 steps through the collision (sigma_L = a, nuclei meet after 12
    steps), the whole state (U, E, Q_A, Q_B) and eps(z) against the oracle
    at every step count it passes: full 64-site rows and full 32-site link
    blocks are the norm here, not the ragged exception."""
    cfg = gi.small_config(3, nz=28, nx=64, ny=64, sigma_l=1.0, steps=20)
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], 3, p.nx, p.ny, p.g2mu)
    st = O.init_mv(p, rho)
    h = G.glasma_init_mv(cfg, rho)
    for block in (6, 6, 8):
        G.glasma_step(h, block)
        st = O.step(st, block)
        U, E, QA, QB, n = G.glasma_get_fields(h)
        assert n == st.n
        errs = dict(U=rel(U, st.U), E=rel(E, st.E), QA=rel(QA, st.QA),
                    QB=rel(QB, st.QB))
        tab, H = G.glasma_tmunu(h)
        rtab, rH = O.tmunu(st)
        errs["eps"] = rel(tab[:, 0], rtab[:, 0])
        errs["H"] = abs(H - rH) / abs(rH)
        assert all(v <= TOL64 for v in errs.values()), (n, errs)
    # the nuclei have crossed: charge of B beyond the centre
    _, _, zc = O.nucleus_positions(p)
    z = np.arange(p.nz) * p.a_z
    assert np.any(np.abs(st.QB[z > zc]) > 0)
    gmax, grms, rmax = G.glasma_gauss_residual(h)
    assert gmax <= 1e-12 * rmax


def test_set_step_kernel_rejects_bad_arguments(G):
    h = G.glasma_init_mv(gi.small_config(2), None)
    for kernel, zlen in ((7, 0), (1, -1), (2, 10 ** 6)):
        with pytest.raises(G.GlasmaError) as e:
            G._check(G.load_library().glasma_set_step_kernel(h.ptr, kernel, zlen),
                     "glasma_set_step_kernel")
        assert e.value.code == "INVALID_ARG"
    # the paired kernel is FP32 only
    with pytest.raises(G.GlasmaError):
        G.glasma_set_step_kernel(h, "staple_pairs")
    # rows longer than a block take no plaquette kernel
    wide = G.glasma_init_mv(gi.small_config(2, nz=24, nx=400, ny=2, sigma_l=1.0), None)
    with pytest.raises(G.GlasmaError):
        G.glasma_set_step_kernel(wide, "plaquette")
    G.glasma_set_step_kernel(wide, "auto")
    G.glasma_step(wide, 2)            # auto falls back to the staple kernel


# Degenerate transverse planes: one site (every transverse neighbour is the
# site itself, each transverse plaquette of a 1-site direction is trivial),
# one row, one column; the shortest box a placeholder event fits (nz = 5).
DEGENERATE = [(5, 1, 1), (5, 1, 2), (6, 2, 1), (5, 3, 1)]


@pytest.mark.parametrize("nc", [2, 3])
@pytest.mark.parametrize("shape", DEGENERATE)
def test_degenerate_planes_match_oracle(G, nc, shape):
    """Every kernel form in FP64 (1e-11) and FP32 (the bound of the FP32
    random-state test), plus T^{mu nu} and the Gauss residual in FP64."""
    nz, ny, nx = shape
    st = _random_state(nc, nz, ny, nx, seed=3 * nz + 5 * ny + nx + nc)
    st.QA[:] = 0.0
    st.QB[:] = 0.0
    st.QA[3] = 0.1
    st.QB[1] = -0.1
    ref = O.step(st, 3)
    rtab, _ = O.tmunu(ref)
    og = O.gauss_residual(ref)
    for precision, kernels, tol in (("fp64", KERNELS, TOL64),
                                    ("fp32", KERNELS + ["staple_pairs"], 1.5e-6)):
        for kernel in kernels:
            h = _ctx(G, st, precision)
            G.glasma_set_step_kernel(h, kernel)
            G.glasma_step(h, 3)
            U, E, QA, QB, n = G.glasma_get_fields(h)
            errs = dict(U=rel(U, ref.U), E=rel(E, ref.E), QA=rel(QA, ref.QA),
                        QB=rel(QB, ref.QB))
            assert all(v <= tol for v in errs.values()), (precision, kernel, errs)
            if precision == "fp64":
                tab, _ = G.glasma_tmunu(h)
                assert rel(tab, rtab) <= TOL64, kernel
                gm, _, rm = G.glasma_gauss_residual(h)
                assert abs(gm - og[0]) <= 1e-12 * og[0] and abs(rm - og[2]) <= 1e-12 * og[2]
            G.glasma_free(h)


@pytest.mark.parametrize("nc", [2, 3])
def test_longest_lattice_matches_oracle(G, nc):
    """nz = 65535, the most slices a context takes (one grid row per slice
    in the step kernels), on a one-site plane: every kernel form, FP64."""
    nz = 65535
    st = _random_state(nc, nz, 1, 1, seed=11 + nc)
    ref = O.step(st, 3)
    rtab, _ = O.tmunu(ref)
    for kernel in KERNELS:
        h = _ctx(G, st)
        G.glasma_set_step_kernel(h, kernel)
        G.glasma_step(h, 3)
        U, E, QA, QB, n = G.glasma_get_fields(h)
        errs = dict(U=rel(U, ref.U), E=rel(E, ref.E), QA=rel(QA, ref.QA),
                    QB=rel(QB, ref.QB))
        assert all(v <= TOL64 for v in errs.values()), (kernel, errs)
        tab, _ = G.glasma_tmunu(h)
        assert rel(tab, rtab) <= TOL64, kernel
        G.glasma_free(h)
    # and the site-paired FP32 kernel (its grid runs over half the slices)
    h = _ctx(G, st, "fp32")
    G.glasma_set_step_kernel(h, "staple_pairs")
    G.glasma_step(h, 3)
    U, E, QA, QB, n = G.glasma_get_fields(h)
    assert rel(U, ref.U) < 1.5e-6 and rel(E, ref.E) < 1.5e-6
    G.glasma_free(h)


# The staged staple kernel (links of two rows and their halo rows, four z
# slices, in shared memory): rows of 64 sites (two link blocks per row) and
# of 32 (one); a chunk of one slice (nz below the chunk count); a ragged last
# tile (odd ny); fewer rows than the staged image holds, so rows repeat
# (ny = 3, ny = 1).
STAGED_SHAPES = [(8, 64, 64), (23, 7, 64), (40, 64, 64), (30, 3, 32), (5, 1, 64)]


@pytest.mark.parametrize("shape", STAGED_SHAPES)
def test_staged_kernel_is_bitwise_the_staple_kernel(G, shape):
    """The staged kernel performs the staple kernel's arithmetic in the same
    order from shared-memory copies of the same links: after 5 steps (hops
    at 0, 2 and 4, charges of both nuclei) every link, field and charge is
    bitwise the staple kernel's, and within the FP32 bound of the oracle."""
    nz, ny, nx = shape
    st = _random_state(3, nz, ny, nx, seed=31 * nz + ny)
    out = []
    for kernel in ("staple", "staple_staged"):
        h = _ctx(G, st, "fp32")
        G.glasma_set_step_kernel(h, kernel)
        G.glasma_step(h, 5)
        out.append(G.glasma_get_fields(h))
        G.glasma_free(h)
    for x, y in zip(out[0][:4], out[1][:4]):
        assert np.array_equal(x, y)
    assert out[0][4] == out[1][4] == 5
    ref = O.step(st, 5)
    U, E, QA, QB, n = out[1]
    errs = dict(U=rel(U, ref.U), E=rel(E, ref.E), QA=rel(QA, ref.QA), QB=rel(QB, ref.QB))
    assert all(v < 2.5e-6 for v in errs.values()), errs


def test_staged_kernel_through_a_collision(G):
    """Through a collision on 64-site rows: the staged kernel and the
    automatic choice give bitwise the staple kernel's state and table."""
    cfg = dict(gi.small_config(3, nz=48, nx=64, ny=6, sigma_l=2.0), precision="fp32")
    rho = gi.mv_rho(cfg["seed"], 3, cfg["nx"], cfg["ny"], cfg["g2mu"])
    res = []
    for kernel in ("staple", "staple_staged", "auto"):
        h = G.glasma_init_mv(cfg, rho)
        G.glasma_set_step_kernel(h, kernel)
        G.glasma_step(h, 40)
        res.append((G.glasma_get_fields(h)[:4], G.glasma_tmunu(h)[0]))
        G.glasma_free(h)
    for other in res[1:]:
        for x, y in zip(res[0][0], other[0]):
            assert np.array_equal(x, y)
        assert np.array_equal(res[0][1], other[1])


def test_staged_wait_that_runs_out_is_reported(G):
    """A wait of the staged kernel on a barrier that nothing completes (the
    stall switch) runs out after its budget; the block stops, waits for its
    copies in flight, and the next call that returns host values reports
    TIMEOUT once.  No GPU fault: the wait is bounded and the copies land."""
    st = _random_state(3, 8, 64, 64, seed=4)
    h = _ctx(G, st, "fp32")
    G.glasma_set_step_kernel(h, "staple_staged")
    G.glasma_set_staging_wait(h, 1 << 20, stall=True)
    G.glasma_step(h, 1)
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_tmunu(h)
    assert e.value.code == "TIMEOUT"
    G.glasma_set_staging_wait(h, 1 << 31, stall=False)
    G.glasma_step(h, 1)
    tab, H = G.glasma_tmunu(h)   # reported once; the status word is clear again
    assert np.all(np.isfinite(tab))
    G.glasma_free(h)


def test_staged_kernel_rejects_what_it_does_not_stage(G):
    cases = [dict(gi.small_config(3, nx=40), precision="fp32"),      # nx not 32 or 64
             dict(gi.small_config(2, nx=64), precision="fp32"),      # SU(2)
             dict(gi.small_config(3, nx=64), precision="fp64")]      # FP64
    for cfg in cases:
        h = G.glasma_init_mv(cfg, None)
        with pytest.raises(G.GlasmaError) as e:
            G.glasma_set_step_kernel(h, "staple_staged")
        assert e.value.code == "INVALID_ARG"
        for wait, stall in ((0, 0), (1 << 41, 0), (1 << 20, 2)):
            with pytest.raises(G.GlasmaError) as e:
                G._check(G.load_library().glasma_set_staging_wait(h.ptr, wait, stall),
                         "glasma_set_staging_wait")
            assert e.value.code == "INVALID_ARG"
        G.glasma_free(h)
