"""Pins of the FP64 oracle against what the paper and the mathematics fix:
closed-form lattice dispersion, brute-force force and step evaluators,
Gauss-law preservation, continuity of the CPIC current, gauge covariance,
leapfrog energy invariants, time reversal, T^{mu nu} identities, the
Poisson stencil and the structure of the MV initial state."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

import glasma_inputs as gi
from oracle import glasma_oracle as O


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def _small_state(nc, **kw):
    cfg = gi.small_config(nc, **kw)
    p = O.Params.from_dict(cfg)
    rho = gi.mv_rho(cfg["seed"], nc, p.nx, p.ny, p.g2mu)
    return O.init_mv(p, rho)


def _abelian_state(p, phi, e3):
    """SU(2) links exp(i phi t^3) and E along t^3 only (U(1) embedding)."""
    U = np.zeros((3, p.nz, p.ny, p.nx, 2, 2), complex)
    U[..., 0, 0] = np.exp(0.5j * phi)
    U[..., 1, 1] = np.exp(-0.5j * phi)
    E = np.zeros((3, p.nz, p.ny, p.nx, 3))
    E[..., 2] = e3
    z = np.zeros((p.nz, p.ny, p.nx, 3))
    return O.State(p, U, E, z.copy(), z.copy(), 0, U.copy())


def _angle(U):
    return 2.0 * np.angle(U[..., 0, 0])


def _grid(p):
    Z, Y, X = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx),
                          indexing="ij")
    return Z, Y, X


# ---------------------------------------------------------------------------
# P6: dispersion of U(1)-embedded plane waves (sign and weight of the force)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["kz_polx", "kx_polz", "kxkz_poly"])
@pytest.mark.parametrize("aniso", [False, True])
def test_dispersion_closed_form(case, aniso):
    a_z, dt = (0.5, 0.25) if aniso else (1.0, 0.5)
    p = O.Params(nc=2, nz=40, nx=16, ny=4, a_z=a_z, dt=dt, sigma_l=1.0)
    Z, Y, X = _grid(p)
    eps = 1e-5
    kx = 2 * np.pi * 3 / p.nx
    kz = 0.7                      # phase advance per z cell
    phi = np.zeros((3,) + Z.shape)
    if case == "kz_polx":
        pol, ks = 0, (0.0, 0.0, kz)
        phi[0] = eps * np.cos(kz * Z)
    elif case == "kx_polz":
        pol, ks = 2, (kx, 0.0, 0.0)
        phi[2] = eps * np.cos(kx * X)
    else:
        pol, ks = 1, (kx, 0.0, kz)
        phi[1] = eps * np.cos(kx * X + kz * Z)
    phi[2][p.nz - 1] = 0.0
    st = _abelian_state(p, phi, 0.0)
    s1 = O.step(st, 1)
    s2 = O.step(s1, 1)
    f0, f1, f2 = (_angle(s.U[pol]) for s in (st, s1, s2))
    a = p.spacing
    # ks holds the phase advance per cell along x and z
    K = ((4.0 / a[0] ** 2) * math.sin(ks[0] / 2) ** 2
         + (4.0 / a[2] ** 2) * math.sin(ks[2] / 2) ** 2)
    expect = 1.0 - 0.5 * dt * dt * K
    inner = (Z >= 4) & (Z <= p.nz - 6) & (np.abs(f1) > 0.3 * eps)
    est = (f2[inner] + f0[inner]) / (2 * f1[inner])
    assert np.max(np.abs(est - expect)) < 1e-9
    # the wrong sign of the force would give 1 + dt^2 K / 2
    assert abs(expect - (1.0 + 0.5 * dt * dt * K)) > 1e-3


# ---------------------------------------------------------------------------
# P7: force = -dH/dU by finite differences, and a plaquette-centric step
# ---------------------------------------------------------------------------

def _link_ok(p, d, z):
    return 0 <= z <= p.nz - 1 and (d != 2 or z <= p.nz - 2)


def _site(p, x, y, z, d, s=1):
    v = [x, y, z]
    v[d] += s
    return v[0] % p.nx, v[1] % p.ny, v[2]


def _naive_plaq(p, U, i, j, x, y, z):
    """Plaquette at base (x, y, z) in plane (i, j), or None if any of its
    four links is absent."""
    b = (x, y, z)
    bi = _site(p, x, y, z, i)
    bj = _site(p, x, y, z, j)
    links = [(i, b), (j, bi), (i, bj), (j, b)]
    if not all(_link_ok(p, d, s[2]) for d, s in links):
        return None
    g = lambda d, s: U[d][s[2], s[1], s[0]]
    return (g(i, b) @ g(j, bi) @ np.conj(g(i, bj).T) @ np.conj(g(j, b).T))


def _local_action(p, U, i, x, y, z):
    """Sum of 2 (N - Re tr P) / (a_i a_j)^2 over plaquettes containing the
    link (i; x, y, z), times the cell volume."""
    a = p.spacing
    vol = a[0] * a[1] * a[2]
    tot = 0.0
    for j in range(3):
        if j == i:
            continue
        for base in ((x, y, z), _site(p, x, y, z, j, -1)):
            if not (0 <= base[2] <= p.nz - 1):
                continue
            lo, hi = min(i, j), max(i, j)
            P = _naive_plaq(p, U, lo, hi, *base)
            if P is not None:
                tot += vol * 2.0 * (p.nc - np.trace(P).real) / (a[i] * a[j]) ** 2
    return tot


@pytest.mark.parametrize("nc", [2, 3])
def test_force_is_minus_gradient_of_wilson_hamiltonian(nc):
    rng = np.random.default_rng(11 + nc)
    p = O.Params(nc=nc, nz=16, nx=4, ny=4, a_z=0.5, dt=0.25)
    U = gi.near_identity_su(nc, (3, p.nz, p.ny, p.nx), rng, 0.4)
    U[2][p.nz - 1] = np.eye(nc)
    F = O.force(U, p)
    t = O.generators(nc)
    a = p.spacing
    vol = a[0] * a[1] * a[2]
    h = 1e-3
    picks = [(0, 1, 2, 0), (1, 3, 0, 15), (2, 0, 1, 14), (2, 2, 3, 0),
             (0, 0, 0, 15), (1, 2, 2, 7), (2, 1, 1, 6)]
    for i, x, y, z in picks:
        for aa in range(nc * nc - 1):
            vals = []
            for s in (-2, -1, 1, 2):
                Up = U.copy()
                Up[i][z, y, x] = (scipy.linalg.expm(1j * s * h * t[aa])
                                  @ U[i][z, y, x])
                vals.append(_local_action(p, Up, i, x, y, z))
            dW = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h)
            fd = -(a[i] ** 2 / vol) * dW
            assert abs(fd - F[i][z, y, x, aa]) < 1e-9, (i, x, y, z, aa)
    # the absent z link carries no force
    assert np.all(F[2][p.nz - 1] == 0.0)


@pytest.mark.parametrize("nc", [2, 3])
def test_step_matches_plaquette_centric_evaluator(nc):
    rng = np.random.default_rng(21 + nc)
    p = O.Params(nc=nc, nz=16, nx=4, ny=4, a_z=0.5, dt=0.25)
    U = gi.near_identity_su(nc, (3, p.nz, p.ny, p.nx), rng, 0.3)
    U[2][p.nz - 1] = np.eye(nc)
    E = 0.3 * rng.standard_normal((3, p.nz, p.ny, p.nx, nc * nc - 1))
    E[2][p.nz - 1] = 0.0
    z = np.zeros((p.nz, p.ny, p.nx, nc * nc - 1))
    st = O.State(p, U, E, z.copy(), z.copy(), 1, U.copy())   # no hop at n=1
    t = O.generators(nc)
    a = p.spacing
    F = np.zeros_like(E)

    def proj(X):
        return np.array([np.trace(t[c] @ X).imag for c in range(nc * nc - 1)])

    for zz, yy, xx in itertools.product(range(p.nz), range(p.ny), range(p.nx)):
        for i, j in ((0, 1), (0, 2), (1, 2)):
            P = _naive_plaq(p, U, i, j, xx, yy, zz)
            if P is None:
                continue
            b = (xx, yy, zz)
            bi = _site(p, xx, yy, zz, i)
            bj = _site(p, xx, yy, zz, j)
            Ui = U[i][zz, yy, xx]
            Uj = U[j][zz, yy, xx]
            Pd = np.conj(P.T)
            # link (i, b): U_{i,j}(b) = P
            F[i][b[2], b[1], b[0]] -= (2 / a[j] ** 2) * proj(P)
            # link (j, b): U_{j,i}(b) = P^dagger
            F[j][b[2], b[1], b[0]] -= (2 / a[i] ** 2) * proj(Pd)
            # link (i, b+j): U_{i,-j}(b+j) = U_j^dag(b) P^dag U_j(b)
            F[i][bj[2], bj[1], bj[0]] -= (2 / a[j] ** 2) * proj(
                np.conj(Uj.T) @ Pd @ Uj)
            # link (j, b+i): U_{j,-i}(b+i) = U_i^dag(b) P U_i(b)
            F[j][bi[2], bi[1], bi[0]] -= (2 / a[i] ** 2) * proj(
                np.conj(Ui.T) @ P @ Ui)
    En = E + p.dt * F
    nxt = O.step(st, 1)
    assert np.max(np.abs(nxt.E - En)) < 1e-13
    Un = np.empty_like(U)
    for d in range(3):
        for zz, yy, xx in itertools.product(range(p.nz), range(p.ny),
                                            range(p.nx)):
            if _link_ok(p, d, zz):
                H = np.einsum("a,aij->ij", En[d][zz, yy, xx], t)
                Un[d][zz, yy, xx] = (scipy.linalg.expm(1j * p.dt * H)
                                     @ U[d][zz, yy, xx])
            else:
                Un[d][zz, yy, xx] = U[d][zz, yy, xx]
    assert np.max(np.abs(nxt.U - Un)) < 1e-13


# ---------------------------------------------------------------------------
# P1, P2, P9: unitarity, Gauss law through the collision, T^{mu nu} identity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [2, 3])
def test_collision_invariants(nc):
    st = _small_state(nc)
    rho_max0 = O.gauss_residual(st)[2]
    assert rho_max0 > 0.01
    for _ in range(8):
        st = O.step(st, 5)
        gmax, grms, rmax = O.gauss_residual(st)
        assert gmax <= 1e-12 * rmax
        tab, H = O.tmunu(st)
        assert np.max(np.abs(tab[:, 0] - tab[:, 1] - 2 * tab[:, 2])) \
            <= 1e-14 * np.max(np.abs(tab[:, 0]))
        # H against the Hamiltonian evaluated separately
        En, _, _ = O.e_update(st)
        Href = (O.h_mag(st.U, st.p) + 0.5 * (O.h_el(st.E, st.E, st.p)
                                             + O.h_el(En, En, st.p)))
        assert abs(H - Href) <= 1e-13 * abs(Href)
    d1, d2 = O.unitarity_dev(st.U)
    assert d1 < 1e-13 and d2 < 1e-13
    # the nuclei have passed through each other: both carry charge on the
    # far side of the box centre
    _, _, zc = O.nucleus_positions(st.p)
    z = np.arange(st.p.nz) * st.p.a_z
    assert np.any(np.abs(st.QB[z > zc]) > 0) and np.any(
        np.abs(st.QA[z < zc]) > 0)


def test_unitarity_after_100_steps():
    st = _small_state(3, nz=112, nx=4, ny=4, steps=100)
    st = O.step(st, 100)
    d1, d2 = O.unitarity_dev(st.U)
    assert d1 < 1e-13 and d2 < 1e-13


# ---------------------------------------------------------------------------
# P3, P4: charge norm under NGP transport, continuity of the deposit
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [2, 3])
def test_hop_transport_and_continuity(nc):
    st = _small_state(nc)
    st = O.step(st, 3)                     # move to a state with fields
    while not O.hop_at(st.n, O.hop_ratio(st.p)):
        st = O.step(st, 1)
    p = st.p
    QA, QB, djz = O.hop(st)
    # P3: sum_a Q^a Q^a of each particle is unchanged
    for new, old in ((np.sum(QB[1:] ** 2, -1), np.sum(st.QB[:-1] ** 2, -1)),
                     (np.sum(QA[:-1] ** 2, -1), np.sum(st.QA[1:] ** 2, -1))):
        assert np.max(old) > 0
        assert np.all(np.abs(new - old) <= 5e-14 * old + 1e-16 * np.max(old))
    # P4: rho' - rho equals the covariant divergence of dt J, evaluated
    # site by site with explicit loops
    t = O.generators(nc)
    drho = (QA + QB) - (st.QA + st.QB)
    az2 = p.a_z ** 2
    for zz, yy, xx in itertools.product(range(p.nz), range(p.ny), range(p.nx)):
        div = djz[zz, yy, xx] / az2
        if zz >= 1:
            Uz = st.U[2][zz - 1, yy, xx]
            J = np.einsum("a,aij->ij", djz[zz - 1, yy, xx], t)
            back = np.conj(Uz.T) @ J @ Uz
            div = div - np.array([2 * np.trace(t[c] @ back).real
                                  for c in range(nc * nc - 1)]) / az2
        assert np.max(np.abs(drho[zz, yy, xx] - div)) < 1e-15


def test_hop_schedule_tie_rule():
    # dt = a/2: hops at steps 0, 2, 4, ...; dt = a/4: first at step 1, then
    # every 4th; dt = a_z: every step.
    pq = (1, 2)
    assert [n for n in range(9) if O.hop_at(n, pq)] == [0, 2, 4, 6, 8]
    pq = (1, 4)
    assert [n for n in range(13) if O.hop_at(n, pq)] == [1, 5, 9]
    assert all(O.hop_at(n, (1, 1)) for n in range(10))
    # after m steps a charge has moved round(m v dt / a_z) cells, ties up
    for m in range(40):
        assert O.hop_count(m, (1, 2)) == math.floor(m / 2 + 0.5)


# ---------------------------------------------------------------------------
# P5: gauge covariance under a random time-independent gauge transformation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [2, 3])
def test_gauge_covariance(nc):
    st = _small_state(nc, nz=40, nx=6, ny=5)
    rng = np.random.default_rng(5)
    om = gi.haar_su(nc, (st.p.nz, st.p.ny, st.p.nx), rng)
    a = O.step(O.gauge_transform(st, om), 20)
    b = O.gauge_transform(O.step(st, 20), om)
    assert np.max(np.abs(a.U - b.U)) < 1e-12
    assert np.max(np.abs(a.E - b.E)) < 1e-12 * np.max(np.abs(b.E))
    assert np.max(np.abs(a.QA - b.QA)) < 1e-12 * np.max(np.abs(b.QA))
    ta, Ha = O.tmunu(a)
    tb, Hb = O.tmunu(O.step(st, 20))
    # the magnetic terms 2 (N - Re tr U_ij) cancel catastrophically, so the
    # per-plaquette rounding (~1e-15 absolute) sets the scale here
    assert np.max(np.abs(ta - tb)) < 1e-10 * np.max(np.abs(tb))
    assert abs(Ha - Hb) < 1e-10 * abs(Hb)


# ---------------------------------------------------------------------------
# P8: time reversal by the algebraic inverse step
# ---------------------------------------------------------------------------

def _inverse_step(st):
    """(U_{n+1}, E_{n+1/2}, Q_{n+1/2}) -> (U_n, E_{n-1/2}, Q_{n-1/2})."""
    p = st.p
    n = st.n - 1
    Un = np.empty_like(st.U)
    for i in range(3):
        Un[i] = O.mm(O.expi_alg(st.E[i], -p.dt, p.nc), st.U[i])
    Un[2][p.nz - 1] = st.U[2][p.nz - 1]
    QA, QB = st.QA.copy(), st.QB.copy()
    djz = np.zeros_like(QA)
    if O.hop_at(n, O.hop_ratio(p)):
        Uz = Un[2]
        # B moved x -> x+z: old Q_B(x) = U_z(x) Q'(x+z) U_z^dag(x)
        qb = np.zeros_like(QB)
        qn = O.alg_to_mat(QB, p.nc)
        qb[:-1] = O.mat_to_alg(O.mm(Uz[:-1], qn[1:], O.dag(Uz[:-1])), p.nc)
        # A moved x+z -> x: old Q_A(x+z) = U_z^dag(x) Q'(x) U_z(x)
        qa = np.zeros_like(QA)
        qn = O.alg_to_mat(QA, p.nc)
        qa[1:] = O.mat_to_alg(O.mm(O.dag(Uz[:-1]), qn[:-1], Uz[:-1]), p.nc)
        djz = (QA - qb) * p.a_z ** 2
        QA, QB = qa, qb
    F = O.force(Un, p)
    E = st.E - p.dt * F
    E[2] = E[2] - djz
    E[2][p.nz - 1] = 0.0
    return O.State(p, Un, E, QA, QB, n)


def test_time_reversal():
    st0 = _small_state(2)
    st = O.step(st0, 40)
    for _ in range(40):
        st = _inverse_step(st)
    assert st.n == 0
    assert np.max(np.abs(st.U - st0.U)) < 1e-11
    assert np.max(np.abs(st.E - st0.E)) < 1e-11
    assert np.max(np.abs(st.QA - st0.QA)) < 1e-11
    assert np.max(np.abs(st.QB - st0.QB)) < 1e-11


# ---------------------------------------------------------------------------
# P13: energy behaviour
# ---------------------------------------------------------------------------

def test_abelian_leapfrog_invariant():
    p = O.Params(nc=2, nz=12, nx=6, ny=5, a_z=0.5, dt=0.25)
    rng = np.random.default_rng(8)
    phi = 1e-5 * rng.standard_normal((3, p.nz, p.ny, p.nx))
    phi[2][p.nz - 1] = 0.0
    st = _abelian_state(p, phi, 0.0)
    def hmag_abelian(U):
        # 2 (N - Re tr P) = 8 sin^2(theta/4) for P = exp(i theta t^3); the
        # angle form avoids the cancellation of N - Re tr P at small theta
        a = p.spacing
        tot = 0.0
        for (i, j) in ((0, 1), (0, 2), (1, 2)):
            th = _angle(O.plaquette(U, i, j))
            m = O.plaq_mask(i, j, p.nz, p.ny, p.nx)
            tot += np.sum(np.where(m, 8 * np.sin(th / 4) ** 2, 0.0)) \
                / (a[i] * a[j]) ** 2
        return p.a_t * p.a_t * p.a_z * tot

    vals = []
    for _ in range(200):
        En, _, _ = O.e_update(st)
        vals.append(O.h_el(st.E, En, p) + hmag_abelian(st.U))
        st = O.step(st, 1)
    vals = np.array(vals)
    assert np.max(np.abs(vals - vals[0])) <= 1e-9 * abs(vals[0])


def test_nonabelian_energy_error_is_second_order():
    """Free non-abelian fields: the time-averaged energy fluctuates by
    O(dt^2); halving dt shrinks the excursion about four-fold."""
    rng = np.random.default_rng(9)
    base = O.Params(nc=2, nz=10, nx=6, ny=6, a_z=1.0, dt=0.25)
    U = gi.near_identity_su(2, (3, base.nz, base.ny, base.nx), rng, 0.25)
    U[2][base.nz - 1] = np.eye(2)
    dev = []
    for dt in (0.25, 0.125):
        p = O.Params(nc=2, nz=10, nx=6, ny=6, a_z=1.0, dt=dt)
        z = np.zeros((p.nz, p.ny, p.nx, 3))
        st = O.State(p, U.copy(), np.zeros((3, p.nz, p.ny, p.nx, 3)),
                     z.copy(), z.copy(), 0)
        Hs = []
        for _ in range(int(round(4.0 / dt))):
            Hs.append(O.tmunu(st)[1])
            st = O.step(st, 1)
        Hs = np.array(Hs)
        dev.append(np.max(np.abs(Hs - Hs.mean())) / Hs.mean())
    ratio = dev[0] / dev[1]
    assert 3.0 < ratio < 5.5, (dev, ratio)


# ---------------------------------------------------------------------------
# Poynting flux sign and the p_L / p_T split on a light-like wave packet
# ---------------------------------------------------------------------------

def test_poynting_flux_of_forward_wave_packet():
    p = O.Params(nc=2, nz=80, nx=1, ny=1, a_z=1.0, dt=0.25)
    Z = np.arange(p.nz)[:, None, None] * np.ones((1, 1, 1))
    eps, w, z0 = 1e-3, 4.0, 25.0
    prof = lambda t: eps * np.exp(-((Z - z0 - t) ** 2) / (2 * w * w))
    phi = np.zeros((3, p.nz, 1, 1))
    phi[0] = prof(0.0)
    e3 = np.zeros_like(phi)
    e3[0] = (prof(0.0) - prof(-p.dt)) / p.dt
    st = O.step(_abelian_state(p, phi, e3), 8)
    tab, H = O.tmunu(st)
    tot = tab.sum(axis=0)
    assert tot[3] > 0
    assert abs(tot[3] / tot[0] - 1.0) < 0.03      # S_L = eps, light-like
    assert abs(tot[1] / tot[0] - 1.0) < 0.03      # p_L = eps
    assert abs(tot[2]) < 1e-6 * tot[0]            # p_T = 0
    # the packet moved to +z
    zc = np.sum(np.arange(p.nz) * tab[:, 0]) / tot[0]
    assert zc > z0 + 1.0


# ---------------------------------------------------------------------------
# P10, P11: MV initial state
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nc", [2, 3])
def test_init_structure(nc):
    st = _small_state(nc)
    p = st.p
    # Poisson stencil residual
    phi = st.extra["phi"]
    rho = gi.mv_rho(gi.small_config(nc)["seed"], nc, p.nx, p.ny, p.g2mu)
    res = -O.laplacian_t(phi, p.a_t) + p.m_ir ** 2 * phi - rho
    assert np.max(np.abs(res)) <= 1e-12 * np.max(np.abs(rho))
    # transverse plaquettes are 1 at t0: b_xy = 0, p_T = 0, E_z = 0
    b = O.plaquette_terms(st.U, p)
    assert np.max(np.abs(b[(0, 1)])) < 1e-13
    assert np.all(st.E[2] == 0.0)
    assert np.all(st.U[2] == np.eye(nc))
    # the charges have compact, disjoint support and the fields outside the
    # nuclei are static pure gauge: E = 0 exactly there
    zb, za, zc = O.nucleus_positions(p)
    z = np.arange(p.nz) * p.a_z
    outside = ((z < zb - p.dt - 4 * p.sigma_l - 1e-12)
               | (z > za + p.dt + 4 * p.sigma_l + 1e-12)
               | ((z > zb + 4 * p.sigma_l) & (z < za - 4 * p.sigma_l)))
    assert np.all(st.E[:, outside] == 0.0)
    assert np.all(st.QA[z < zc] == 0.0) and np.all(st.QB[z > zc] == 0.0)
    assert np.max(np.abs(st.QA)) > 0 and np.max(np.abs(st.QB)) > 0
    # Gauss law holds exactly at t0 (rho is defined by it)
    assert O.gauss_residual(st)[0] < 1e-15
    # B's field is behind it (low z), A's behind it (high z)
    assert np.max(np.abs(st.U[0][0] - np.eye(nc))) > 1e-3
    assert np.max(np.abs(st.U[0][p.nz - 1] - np.eye(nc))) > 1e-3


@pytest.mark.parametrize("nc", [2, 3])
def test_plaquette_energy_forms_agree(nc):
    """||U_i U_j(x+i) - U_j U_i(x+j)||_F^2 = 2 (N - Re tr U_ij) for unitary
    links: both forms agree to rounding on generic and on weak fields."""
    rng = np.random.default_rng(31)
    p = O.Params(nc=nc, nz=6, nx=4, ny=5, a_z=0.5)
    for amp in (0.5, 1e-3):
        U = gi.near_identity_su(nc, (3, p.nz, p.ny, p.nx), rng, amp)
        U[2][p.nz - 1] = np.eye(nc)
        bf = O.plaquette_terms(U, p)
        bt = O.plaquette_terms_trace(U, p)
        for k in bf:
            assert np.max(np.abs(bf[k] - bt[k])) < 5e-14 / (
                p.spacing[k[0]] * p.spacing[k[1]]) ** 2
        assert np.max(bf[(0, 1)]) > 0


def test_vacuum_stays_vacuum():
    cfg = gi.small_config(3)
    p = O.Params.from_dict(cfg)
    st = O.init_mv(p, np.zeros((2, 8, p.ny, p.nx)))
    assert np.all(st.E == 0) and np.all(st.QA == 0)
    s2 = O.step(st, 6)
    assert np.max(np.abs(s2.U - st.U)) < 1e-15


# ---------------------------------------------------------------------------
# P12: the improved (semi-implicit) scheme
# ---------------------------------------------------------------------------

def test_implicit_with_leapfrog_weights_is_leapfrog_bit_for_bit():
    st = _small_state(3)
    a = O.step(st, 4)
    b = O.step_implicit(st, 4, w=(0.0, 1.0, 0.0))
    assert np.array_equal(a.U, b.U) and np.array_equal(a.E, b.E)
    assert np.array_equal(a.QA, b.QA) and np.array_equal(a.QB, b.QB)


@pytest.mark.parametrize("case", ["kz_polx", "kx_polz", "kxkz_poly"])
def test_implicit_dispersion_closed_form(case):
    """Abelian plane waves under the semi-implicit scheme: the time-averaged
    transverse terms give (a_{n+1} + a_{n-1}) / (2 a_n) =
    (1 - dt^2 K_z/2 - dt^2 K_T/4) / (1 + dt^2 K_T/4), i.e.
    (2/dt)^2 sin^2(w dt/2) = K_z + cos^2(w dt/2) K_T; at dt = a_z and
    k_T = 0 this is w = k_z exactly (no dispersion along z)."""
    a_z = dt = 0.5
    p = O.Params(nc=2, nz=40, nx=16, ny=4, a_z=a_z, dt=dt, sigma_l=1.0)
    Z, Y, X = _grid(p)
    eps = 1e-5
    kx = 2 * np.pi * 3 / p.nx
    kz = 0.7
    phi = np.zeros((3,) + Z.shape)
    if case == "kz_polx":
        pol, KT, Kz = 0, 0.0, (4 / a_z ** 2) * math.sin(kz / 2) ** 2
        phi[0] = eps * np.cos(kz * Z)
    elif case == "kx_polz":
        pol, KT, Kz = 2, 4 * math.sin(kx / 2) ** 2, 0.0
        phi[2] = eps * np.cos(kx * X)
    else:
        pol, KT, Kz = 1, 4 * math.sin(kx / 2) ** 2, (4 / a_z ** 2) * math.sin(kz / 2) ** 2
        phi[1] = eps * np.cos(kx * X + kz * Z)
    phi[2][p.nz - 1] = 0.0
    st = _abelian_state(p, phi, 0.0)
    s1 = O.step_implicit(st, 1)
    s2 = O.step_implicit(s1, 1)
    f0, f1, f2 = (_angle(s.U[pol]) for s in (st, s1, s2))
    expect = (1 - dt * dt * Kz / 2 - dt * dt * KT / 4) / (1 + dt * dt * KT / 4)
    inner = (Z >= 5) & (Z <= p.nz - 7) & (np.abs(f1) > 0.1 * eps)
    assert np.count_nonzero(inner) > 50
    est = (f2[inner] + f0[inner]) / (2 * f1[inner])
    assert np.max(np.abs(est - expect)) < 1e-9
    if case == "kz_polx":
        assert abs(expect - math.cos(kz)) < 1e-14      # w dt = k_z a_z
    # phase velocity along z never below 1: w >= k_z for every mode
    w = math.acos(expect) / dt
    assert w >= (kz / a_z if case != "kx_polz" else 0.0) - 1e-12


def _transverse_mode_state(dt, a_z):
    """U(1)-embedded E_z in the highest transverse mode, k_T = (pi, pi), on
    the unit links: the eigenvector of the sweep's Jacobian with the
    extreme eigenvalue -c, c = 8 w_0 dt^2 / a_T^2 (w_0 = 1/4)."""
    p = O.Params(nc=2, nz=8, nx=4, ny=4, a_z=a_z, dt=dt)
    Z, Y, X = _grid(p)
    e3 = np.zeros((3,) + Z.shape)
    e3[2] = 1e-6 * np.cos(np.pi * (X + Y))
    e3[2][p.nz - 1] = 0.0
    return _abelian_state(p, np.zeros((3,) + Z.shape), e3)


@pytest.mark.parametrize("dt,a_z", [(0.25, 0.5), (0.5, 0.5)])
def test_implicit_sweep_contraction_closed_form(dt, a_z):
    """On the extreme transverse mode the plain iteration's changes shrink
    by exactly c per sweep, the relaxed iteration's (omega = 2 / (2 + c)
    after the first sweep) by c / (2 + c); both reach the same fixed
    point."""
    st = _transverse_mode_state(dt, a_z)
    c = 8 * 0.25 * dt * dt
    assert O.implicit_omega(st.p) == 2.0 / (2.0 + c)
    plain = O.step_implicit(st, 1, tol=1e-19, omega=1.0)
    relaxed = O.step_implicit(st, 1, tol=1e-19)
    dp, dr = plain.extra["deltas"], relaxed.extra["deltas"]
    rp = [dp[k + 1] / dp[k] for k in range(6)]
    rr = [dr[k + 1] / dr[k] for k in range(1, 6)]
    assert np.allclose(rp, c, rtol=1e-6), rp
    assert np.allclose(rr, c / (2 + c), rtol=1e-6), rr
    assert relaxed.extra["iters"] < plain.extra["iters"]
    assert np.max(np.abs(relaxed.E - plain.E)) < 1e-18
    assert np.max(np.abs(relaxed.U - plain.U)) < 1e-18


def test_implicit_relaxed_iteration_converges_where_plain_fails():
    """dt = a_T (c = 2): the plain iteration doubles its changes every sweep
    and never settles; the relaxed one contracts by c / (2 + c) = 1/2."""
    st = _transverse_mode_state(1.0, 1.0)
    with pytest.raises(O.NotConverged):
        O.step_implicit(st, 1, tol=1e-19, omega=1.0, max_iter=40)
    s = O.step_implicit(st, 1, tol=1e-19, max_iter=80)
    d = s.extra["deltas"]
    assert np.allclose([d[k + 1] / d[k] for k in range(1, 6)], 0.5, rtol=1e-6)


def test_implicit_abelian_gauss_is_conserved():
    """In the U(1) embedding each plane keeps one antisymmetric, time-averaged
    field strength, so the abelian Gauss law is conserved exactly."""
    p = O.Params(nc=2, nz=12, nx=6, ny=5, a_z=0.5, dt=0.25)
    rng = np.random.default_rng(12)
    phi = 1e-3 * rng.standard_normal((3, p.nz, p.ny, p.nx))
    phi[2][p.nz - 1] = 0.0
    e3 = 1e-3 * rng.standard_normal((3, p.nz, p.ny, p.nx))
    e3[2][p.nz - 1] = 0.0
    st = _abelian_state(p, phi, e3)
    st.U_prev = st.U.copy()
    g0 = O.gauss_divergence(st.U, st.E, p)
    s = O.step_implicit(st, 6)
    g1 = O.gauss_divergence(s.U, s.E, p)
    assert np.max(np.abs(g1 - g0)) < 1e-14


def test_implicit_gauss_residual_is_bounded():
    """Non-abelian collision: the equal-time Gauss residual of the reading
    adopted is not zero; it stays bounded (reported, not pinned to zero)."""
    st = _small_state(2, nz=64, nx=6, ny=5, a_z=0.5, dt=0.25, sigma_l=1.5)
    res = []
    for _ in range(4):
        st = O.step_implicit(st, 3)
        g = O.gauss_residual(st)
        res.append(g[0] / g[2])
    assert max(res) < 1e-3
    assert res[-1] < 3 * max(res[:2])
