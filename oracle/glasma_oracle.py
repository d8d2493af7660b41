"""Plain FP64 CPU oracle of the 3+1D Glasma CPIC leapfrog step.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import this module.  The CUDA
library never calls it and shares no code with it.

What it computes (Ipp & Mueller, "Progress on 3+1D Glasma simulations"):

* MV initial conditions (Sec. 2 and Sec. 3, Eqs. single_sheet,
  3d_colorfield_1/2): two nuclei with transverse MV charges rho_N(x_T),
  a transverse Poisson solve with IR regulator m, a Gaussian longitudinal
  profile, light-like Wilson lines V_N^dagger = exp(i Lambda_N phi_N) and the
  pure-gauge transverse links of each nucleus, superposed.
* The leapfrog update (Sec. 3, Eqs. lattice_1 and lattice_2) with the
  plaquette of Eq. plaquette, on a lattice periodic in x, y and open in z.
* CPIC with one recoil-less particle per site moving at the speed of light
  (Sec. 3, Eq. continuity and the NGP parallel transport that follows it):
  on a hop the charge is parallel transported along the crossed z link and
  the current that satisfies the discrete continuity equation is deposited.
* The discrete Gauss law with parallel-transported E (Sec. 3, Eq. gauss).
* T^{mu nu} per z slice: eps, p_L, p_T, S_L (Sec. 4, Eq. pT_eL and the
  matrix above it).

Conventions (lattice units, g = 1, a_T = 1):
  SU(N) generators t^a hermitian, tr(t^a t^b) = delta^{ab}/2;
  E_i = E_i^a t^a hermitian, U_i(t + dt) = exp(i dt E_i) U_i(t);
  arrays: U[i][z][y][x][N][N] complex, E[i][z][y][x][a] real,
  i = 0, 1, 2 for x, y, z.
Readings of points the paper leaves open (each restated where used):
  force sign/normalisation from the Wilson Hamiltonian; open z boundary;
  E(t0 - dt/2) from the exact group log; NGP tie rule; current sign.

Every floating-point quantity is float64 / complex128.  The exponential and
logarithm use a hermitian eigen-decomposition (LAPACK via numpy).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np

# ---------------------------------------------------------------------------
# SU(N) algebra (Sec. 2: traceless hermitian generators t^a)
# ---------------------------------------------------------------------------

_GEN = {}


def generators(nc):
    """t^a = sigma^a / 2 for SU(2), lambda^a / 2 (Gell-Mann) for SU(3)."""
    if nc in _GEN:
        return _GEN[nc]
    if nc == 2:
        s = np.zeros((3, 2, 2), complex)
        s[0] = [[0, 1], [1, 0]]
        s[1] = [[0, -1j], [1j, 0]]
        s[2] = [[1, 0], [0, -1]]
        t = s / 2.0
    elif nc == 3:
        l = np.zeros((8, 3, 3), complex)
        l[0][0, 1] = l[0][1, 0] = 1
        l[1][0, 1] = -1j
        l[1][1, 0] = 1j
        l[2][0, 0] = 1
        l[2][1, 1] = -1
        l[3][0, 2] = l[3][2, 0] = 1
        l[4][0, 2] = -1j
        l[4][2, 0] = 1j
        l[5][1, 2] = l[5][2, 1] = 1
        l[6][1, 2] = -1j
        l[6][2, 1] = 1j
        l[7][0, 0] = l[7][1, 1] = 1 / math.sqrt(3)
        l[7][2, 2] = -2 / math.sqrt(3)
        t = l / 2.0
    else:
        raise ValueError("nc must be 2 or 3")
    _GEN[nc] = t
    return t


def dag(x):
    return np.conj(np.swapaxes(x, -1, -2))


def mm(*ms):
    out = ms[0]
    for m in ms[1:]:
        out = np.matmul(out, m)
    return out


def alg_to_mat(v, nc):
    """sum_a v^a t^a for v[..., a]."""
    return np.einsum("...a,aij->...ij", v, generators(nc))


def mat_to_alg(h, nc):
    """Components 2 Re tr(t^a H) of a hermitian matrix H."""
    return 2.0 * np.einsum("aij,...ji->...a", generators(nc), h).real


def im_tr_ta(x, nc):
    """Im tr(t^a X) for every generator a."""
    return np.einsum("aij,...ji->...a", generators(nc), x).imag


def expi_alg(v, c, nc):
    """exp(i c sum_a v^a t^a) from the eigen-decomposition of the hermitian
    matrix sum_a v^a t^a."""
    h = alg_to_mat(v, nc)
    w, q = np.linalg.eigh(h)
    ph = np.exp(1j * c * w)
    return np.einsum("...ik,...k,...jk->...ij", q, ph, np.conj(q))


def logu(w):
    """Hermitian H with exp(i H) = W for unitary W whose eigen-phases lie in
    (-pi/2, pi/2).  The hermitian S = (W - W^dagger)/(2i) has eigenvalues
    sin(theta_k) on W's eigenvectors, so its eigenvectors diagonalise W;
    theta_k = atan2(v^dagger S v, v^dagger C v) with C = (W + W^dagger)/2."""
    s = (w - dag(w)) / 2j
    c = (w + dag(w)) / 2.0
    _, q = np.linalg.eigh(s)
    sv = np.einsum("...ki,...kl,...li->...i", np.conj(q), s, q).real
    cv = np.einsum("...ki,...kl,...li->...i", np.conj(q), c, q).real
    if np.any(cv <= 0.0):
        raise ValueError("logu: eigen-phase outside (-pi/2, pi/2)")
    th = np.arctan2(sv, cv)
    return np.einsum("...ik,...k,...jk->...ij", q, th, np.conj(q))


# ---------------------------------------------------------------------------
# Lattice geometry: periodic x, y; open z (reading: no link U_z at the last
# slice, and plaquettes or staples that leave the z range are absent).
# ---------------------------------------------------------------------------

AXIS = {0: 2, 1: 1, 2: 0}   # direction i -> array axis of [z][y][x]


def shift(f, i, s):
    """f(x + s e_i) with periodic wrap on every axis.  Wrapped values along z
    are never used: every use along z is multiplied by a mask below."""
    return np.roll(f, -s, axis=AXIS[i])


def z_index(nz, ny, nx):
    return np.broadcast_to(np.arange(nz)[:, None, None], (nz, ny, nx))


def link_mask(i, nz, ny, nx):
    """True where link U_i(x) exists (U_z absent on the last z slice)."""
    iz = z_index(nz, ny, nx)
    if i == 2:
        return iz <= nz - 2
    return np.ones((nz, ny, nx), bool)


def plaq_mask(i, j, nz, ny, nx):
    """True where the plaquette based at x in plane (i, j) exists."""
    iz = z_index(nz, ny, nx)
    if 2 in (i, j):
        return iz <= nz - 2
    return np.ones((nz, ny, nx), bool)


def plaquette(U, i, j):
    """U_{i,j}(x) = U_i(x) U_j(x+i) U_i^dagger(x+j) U_j^dagger(x)
    (Sec. 3, Eq. plaquette)."""
    return mm(U[i], shift(U[j], i, 1), dag(shift(U[i], j, 1)), dag(U[j]))


def plaquette_minus(U, i, j):
    """U_{i,-j}(x) = U_i(x) U_j^dagger(x+i-j) U_i^dagger(x-j) U_j(x-j)."""
    return mm(U[i], dag(shift(shift(U[j], i, 1), j, -1)),
              dag(shift(U[i], j, -1)), shift(U[j], j, -1))


# ---------------------------------------------------------------------------
# Parameters and state
# ---------------------------------------------------------------------------

@dataclass
class Params:
    nc: int
    nz: int
    nx: int
    ny: int
    a_t: float = 1.0
    a_z: float = 1.0
    dt: float = 0.5
    sigma_l: float = 4.0
    g2mu: float = 0.1
    m_ir: float = 0.2
    uv_cutoff: float = 0.0
    z_offset: float = 0.0
    seed: int = 0
    n_sheets: int = 1

    @staticmethod
    def from_dict(d):
        keys = Params.__dataclass_fields__.keys()
        return Params(**{k: d[k] for k in keys if k in d})

    @property
    def na(self):
        return self.nc * self.nc - 1

    @property
    def spacing(self):
        return (self.a_t, self.a_t, self.a_z)


@dataclass
class State:
    p: Params
    U: np.ndarray            # [3][z][y][x][N][N] at t_n
    E: np.ndarray            # [3][z][y][x][a] at t_{n-1/2}
    QA: np.ndarray           # [z][y][x][a] at t_{n-1/2}, nucleus A (-z)
    QB: np.ndarray           # [z][y][x][a] at t_{n-1/2}, nucleus B (+z)
    n: int = 0
    U_prev: np.ndarray = None   # U at t_{n-1} (improved scheme)
    extra: dict = field(default_factory=dict)

    def copy(self):
        return State(self.p, self.U.copy(), self.E.copy(), self.QA.copy(),
                     self.QB.copy(), self.n,
                     None if self.U_prev is None else self.U_prev.copy(),
                     dict(self.extra))


class ParticleExit(RuntimeError):
    """A nonzero colour charge would leave the open z range."""


# ---------------------------------------------------------------------------
# Initial conditions (Sec. 2 MV model; Sec. 3 Eqs. single_sheet,
# 3d_colorfield_1, 3d_colorfield_2; Sec. 4 Gaussian profile)
# ---------------------------------------------------------------------------

def poisson(rho, p: Params):
    """phi = (-Delta_T + m^2)^{-1} rho on the periodic transverse lattice
    (Sec. 2: phi(k) = rho(k) / (k_T^2 + m^2), optional UV cutoff Lambda).
    Reading: the lattice Laplacian eigenvalue 4/a^2 sin^2(k a/2) replaces
    k_T^2; the cutoff, if set, removes modes whose eigenvalue exceeds
    Lambda^2.  rho[..., y, x] -> phi[..., y, x]."""
    ny, nx = rho.shape[-2:]
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    k2 = ((4.0 / p.a_t ** 2) * np.sin(ky[:, None] / 2) ** 2
          + (4.0 / p.a_t ** 2) * np.sin(kx[None, :] / 2) ** 2)
    kern = 1.0 / (k2 + p.m_ir ** 2)
    if p.uv_cutoff > 0:
        kern = np.where(k2 > p.uv_cutoff ** 2, 0.0, kern)
    return np.fft.ifft2(np.fft.fft2(rho) * kern).real


def laplacian_t(phi, a_t):
    """Periodic 5-point transverse lattice Laplacian (for the Poisson pin)."""
    return (np.roll(phi, 1, -1) + np.roll(phi, -1, -1) + np.roll(phi, 1, -2)
            + np.roll(phi, -1, -2) - 4 * phi) / a_t ** 2


ERF4 = math.erf(4.0 / math.sqrt(2.0))


def nucleus_positions(p: Params):
    """Centres of B (moving +z) and A (moving -z) at t0.  Reading: centre
    of the box z_c = nz a_z / 2, separation d = ceil(4 sigma/a_z) + 2 cells
    unless z_offset is set; the truncated profiles are then disjoint."""
    zc = p.nz * p.a_z / 2.0
    d = p.z_offset if p.z_offset > 0 else (math.ceil(4 * p.sigma_l / p.a_z)
                                           + 2) * p.a_z
    return zc - d, zc + d, zc


def big_lambda(z, zn, sigma, nucleus):
    """Cumulative longitudinal profile (Sec. 3 Eq. single_sheet with the
    Gaussian lambda of Sec. 4).  Reading: lambda is the Gaussian of standard
    deviation sigma truncated at 4 sigma and renormalised, so Lambda is
    exactly 0 ahead of the nucleus and exactly 1 behind it.
    nucleus 'B' (moving +z): Lambda = int_z^inf lambda(s - zn) ds;
    nucleus 'A' (moving -z): Lambda = int_-inf^z lambda(s - zn) ds."""
    u = (np.asarray(z, float) - zn) / sigma
    uc = np.clip(u, -4.0, 4.0)
    ef = np.array([math.erf(v / math.sqrt(2.0)) for v in np.ravel(uc)])
    ef = ef.reshape(np.shape(uc))
    if nucleus == "B":
        lam = (ERF4 - ef) / (2 * ERF4)
        lam = np.where(u >= 4.0, 0.0, np.where(u <= -4.0, 1.0, lam))
    else:
        lam = (ef + ERF4) / (2 * ERF4)
        lam = np.where(u <= -4.0, 0.0, np.where(u >= 4.0, 1.0, lam))
    return lam


def wilson_line_dag(phi_n, lam_z, nc):
    """V^dagger(z, x_T) = exp(i Lambda(z) phi^a(x_T) t^a) for every z.
    For the single-sheet colour structure all path-ordered factors commute
    (Sec. 2, light-like Wilson lines), so the path ordering is exact.
    phi_n[a][y][x], lam_z[z] -> [z][y][x][N][N]; Lambda = 0 gives 1."""
    nz = lam_z.shape[0]
    ny, nx = phi_n.shape[-2:]
    v = np.moveaxis(phi_n, 0, -1)                      # [y][x][a]
    out = np.broadcast_to(np.eye(nc, dtype=complex),
                          (nz, ny, nx, nc, nc)).copy()
    for iz in range(nz):
        if lam_z[iz] != 0.0:
            out[iz] = expi_alg(v, lam_z[iz], nc)
    return out


def sheet_profiles(lam_z, n_sheets):
    """Cumulative profile of each longitudinal colour sheet (the general
    colour structure rho(x^-, x_T) of Sec. 2 and Sec. 5, one independent
    transverse charge per slab of the profile).  Reading: sheet s holds the
    s-th of n_sheets equal-charge slabs of the Gaussian profile, s = 0 at the
    nucleus' leading edge, so Lambda_s(z) = clip(n Lambda(z) - s, 0, 1) and
    sum_s Lambda_s = n Lambda."""
    s = np.arange(n_sheets)[:, None]
    return np.clip(n_sheets * np.asarray(lam_z)[None, :] - s, 0.0, 1.0)


def wilson_line_dag_sheets(phi_sn, lam_z, nc):
    """Path-ordered V^dagger(z, x_T) = exp(i Lambda_{S-1} phi_{S-1}) ...
    exp(i Lambda_0 phi_0) for sheet fields phi_sn[s][a][y][x] (reading: the
    sheet crossed first, s = 0, acts first, i.e. stands rightmost).  The
    factors no longer commute once the sheets' colour charges differ.
    One sheet gives wilson_line_dag exactly."""
    S = phi_sn.shape[0]
    if S == 1:
        return wilson_line_dag(phi_sn[0], lam_z, nc)
    ls = sheet_profiles(lam_z, S)
    out = None
    for s in range(S):
        f = wilson_line_dag(phi_sn[s], ls[s], nc)
        out = f if out is None else mm(f, out)
    return out


def links_at(p: Params, phi, t_shift):
    """Gauge links of the two superposed nuclei (Sec. 3 Eqs.
    3d_colorfield_1/2) with both nuclei moved by t_shift (0 or -dt) from
    their t0 positions.  Reading of the discretisation of
    A^i = (1/ig) V d^i V^dagger: U_i(x) = V(x) V^dagger(x + i) per nucleus,
    U = U^A U^B, U_z = 1."""
    nc = p.nc
    zb, za, _ = nucleus_positions(p)
    zb = zb + t_shift          # B moves +z: earlier means further back
    za = za - t_shift
    z = np.arange(p.nz) * p.a_z
    lam_a = big_lambda(z, za, p.sigma_l, "A")
    lam_b = big_lambda(z, zb, p.sigma_l, "B")
    ph = phi if phi.ndim == 5 else phi[None]          # [S][N][a][y][x]
    vd_a = wilson_line_dag_sheets(ph[:, 0], lam_a, nc)
    vd_b = wilson_line_dag_sheets(ph[:, 1], lam_b, nc)
    U = np.empty((3, p.nz, p.ny, p.nx, nc, nc), complex)
    for i in (0, 1):
        ua = mm(dag(vd_a), shift(vd_a, i, 1))
        ub = mm(dag(vd_b), shift(vd_b, i, 1))
        U[i] = mm(ua, ub)
    U[2] = np.eye(nc)
    return U


def hop_ratio(p: Params):
    """v dt / a_z = p/q as an exact rational (v = c)."""
    r = Fraction(p.dt) / Fraction(p.a_z)
    if r.denominator > 4096:
        raise ValueError("dt / a_z must be an exact ratio p/q with q <= 4096")
    if r > 1:
        raise ValueError("dt > a_z: a charge would cross several cells")
    return r.numerator, r.denominator


def hop_count(m, pq):
    """Cells travelled after m steps under the nearest-grid-point rule,
    ties rounded up: floor(m p/q + 1/2), in integers."""
    pp, qq = pq
    return (2 * m * pp + qq) // (2 * qq)


def hop_at(n, pq):
    return hop_count(n + 1, pq) > hop_count(n, pq)


def init_mv(p: Params, rho):
    """MV initial state at t0 (U) and t0 - dt/2 (E, charges).

    rho[N][a][y][x]: transverse MV charges of A (N=0) and B (N=1); with
    p.n_sheets = S > 1, rho[s][N][a][y][x]: one independent charge per
    longitudinal colour sheet (wilson_line_dag_sheets).
    Steps: Poisson solve; links at t0 and t0 - dt; E from the exact group
    log of U(t0) U^dagger(t0 - dt) (reading; exactly 0 where the two links
    are bitwise equal); charge density from the discrete Gauss law of
    Sec. 3 Eq. gauss; charges split by the side of the box centre."""
    phi = poisson(rho, p)
    U0 = links_at(p, phi, 0.0)
    Um = links_at(p, phi, -p.dt)
    E = np.zeros((3, p.nz, p.ny, p.nx, p.na))
    for i in (0, 1):
        w = mm(U0[i], dag(Um[i]))
        same = np.all(U0[i] == Um[i], axis=(-1, -2))
        h = np.zeros_like(w)
        idx = ~same
        if np.any(idx):
            h[idx] = logu(w[idx])
        E[i] = mat_to_alg(h, p.nc) / p.dt
    rho3 = gauss_divergence(U0, E, p)
    _, _, zc = nucleus_positions(p)
    z = (np.arange(p.nz) * p.a_z)[:, None, None, None]
    QA = np.where(z > zc, rho3, 0.0)
    QB = np.where(z < zc, rho3, 0.0)
    mid = (z == zc)[..., 0, 0, 0]
    if np.any(rho3[mid] != 0.0):
        raise ValueError("init: charge at the box centre")
    st = State(p, U0, E, QA, QB, 0, Um)
    st.extra["phi"] = phi
    st.extra["rho3"] = rho3
    return st


# ---------------------------------------------------------------------------
# Gauss law (Sec. 3 Eq. gauss) and the force of Eq. lattice_1
# ---------------------------------------------------------------------------

def transport_back(U, F, i):
    """U_i^dagger(x-i) F(x-i) U_i(x-i): an adjoint field at x-i parallel
    transported to x (components F[..., a])."""
    nc = U.shape[-1]
    um = shift(U[i], i, -1)
    fm = shift(alg_to_mat(F, nc), i, -1)
    return mat_to_alg(mm(dag(um), fm, um), nc)


def gauss_divergence(U, E, p: Params):
    """sum_i [E_i(x) - U_i^dag(x-i) E_i(x-i) U_i(x-i)] / a_i^2.
    Reading of the weights: the Hamiltonian normalisation below; for
    a_i = 1 this is the printed Eq. gauss.  Open z: at z = 0 there is no
    link from below, so only E_z(x) enters."""
    a = p.spacing
    iz = z_index(p.nz, p.ny, p.nx)[..., None]
    div = np.zeros(E.shape[1:])
    for i in range(3):
        back = transport_back(U, E[i], i)
        if i == 2:
            back = np.where(iz >= 1, back, 0.0)
        div += (E[i] - back) / a[i] ** 2
    return div


def gauss_residual(st: State):
    """G = div E - rho with rho = Q_A + Q_B; returns (max |G|, rms G,
    max |rho|)."""
    g = gauss_divergence(st.U, st.E, st.p) - (st.QA + st.QB)
    rho = st.QA + st.QB
    return (float(np.max(np.abs(g))), float(np.sqrt(np.mean(g ** 2))),
            float(np.max(np.abs(rho))))


def force(U, p: Params):
    """F_i^a(x) = -sum_{j != i} (2/a_j^2) Im tr[t^a (U_{i,j} + U_{i,-j})].

    Sec. 3 Eq. lattice_1 writes -dt/a_j^2 [U_{i,j} + U_{i,-j}]_ah.  Reading:
    with hermitian E = E^a t^a the generator projection of [X]_ah is
    2 Im tr(t^a X); the sign and weight follow from the Hamiltonian
    H = a_x a_y a_z sum_x [ sum_i E_i^a E_i^a / (2 a_i^2)
                            + sum_{i<j} 2 (N - Re tr U_ij) / (a_i a_j)^2 ],
    i.e. F = -dH/dU, which gives oscillation (the other sign grows).
    Terms whose plaquette leaves the open z range are absent."""
    nz, ny, nx = p.nz, p.ny, p.nx
    a = p.spacing
    nc = p.nc
    F = np.zeros((3, nz, ny, nx, p.na))
    for i in range(3):
        for j in range(3):
            if j == i:
                continue
            fwd = im_tr_ta(plaquette(U, i, j), nc)
            bwd = im_tr_ta(plaquette_minus(U, i, j), nc)
            mf = plaq_mask(i, j, nz, ny, nx)
            mb = shift(plaq_mask(i, j, nz, ny, nx), j, -1)
            if j == 2:
                mb = mb & (z_index(nz, ny, nx) >= 1)
            F[i] -= (2.0 / a[j] ** 2) * (np.where(mf[..., None], fwd, 0.0)
                                         + np.where(mb[..., None], bwd, 0.0))
        F[i] = np.where(link_mask(i, nz, ny, nx)[..., None], F[i], 0.0)
    return F


# ---------------------------------------------------------------------------
# CPIC hop (Sec. 3: NGP parallel transport and Eq. continuity)
# ---------------------------------------------------------------------------

def transport_charge(U, Q, direction):
    """Charges after one NGP hop, and the current on the crossed links.

    direction +1 (nucleus B): Q'(x+z) = U_z^dag(x) Q(x) U_z(x) and
    J_z(x) = -Q(x) a_z^2/dt.  direction -1 (nucleus A):
    Q'(x-z) = U_z(x-z) Q(x) U_z^dag(x-z) and J_z(x-z) = +Q'(x-z) a_z^2/dt.
    Returns (Q', dt*J_z / a_z^2) so the caller scales by a_z^2.
    Reading (sign and weight): the continuity equation
    rho' - rho = dt sum_i [J_i(x) - U_i^dag(x-i) J_i(x-i) U_i(x-i)] / a_i^2,
    consistent with the Gauss weights above and with E += dt J."""
    nc = U.shape[-1]
    nz = Q.shape[0]
    Uz = U[2]
    qm = alg_to_mat(Q, nc)
    if direction > 0:
        if np.any(Q[nz - 1] != 0.0):
            raise ParticleExit("nucleus B reached the upper z boundary")
        moved = mat_to_alg(mm(dag(Uz), qm, Uz), nc)     # at x, to go to x+z
        Qn = np.zeros_like(Q)
        Qn[1:] = moved[:-1]
        dj = -Q.copy()
        dj[nz - 1] = 0.0
        return Qn, dj
    if np.any(Q[0] != 0.0):
        raise ParticleExit("nucleus A reached the lower z boundary")
    qs = np.zeros_like(qm)
    qs[:-1] = qm[1:]                                     # Q(x+z) at x
    moved = mat_to_alg(mm(Uz, qs, dag(Uz)), nc)          # lands on x
    Qn = np.zeros_like(Q)
    Qn[:-1] = moved[:-1]
    dj = Qn.copy()
    return Qn, dj


def hop(st: State):
    """Scheduled NGP hop of both nuclei at step n.  Returns
    (QA', QB', dt*J_z) where dt*J_z already carries a_z^2.  Contributions
    are summed B first, then A."""
    p = st.p
    pq = hop_ratio(p)
    djz = np.zeros_like(st.QA)
    if not hop_at(st.n, pq):
        return st.QA, st.QB, djz
    QBn, djb = transport_charge(st.U, st.QB, +1)
    QAn, dja = transport_charge(st.U, st.QA, -1)
    djz = djz + djb * p.a_z ** 2
    djz = djz + dja * p.a_z ** 2
    return QAn, QBn, djz


# ---------------------------------------------------------------------------
# Leapfrog step (Sec. 3 Eqs. lattice_1 and lattice_2)
# ---------------------------------------------------------------------------

def e_update(st: State):
    """E(t_{n+1/2}) and the hopped charges, without committing them."""
    p = st.p
    QA, QB, djz = hop(st)
    F = force(st.U, p)
    En = st.E + p.dt * F
    En[2] = En[2] + djz
    En[2] = np.where(link_mask(2, p.nz, p.ny, p.nx)[..., None], En[2], 0.0)
    return En, QA, QB


def u_update(U, E, p: Params):
    """U_i(t + dt) = exp(i dt E_i) U_i(t) on every existing link."""
    Un = np.empty_like(U)
    for i in range(3):
        Un[i] = mm(expi_alg(E[i], p.dt, p.nc), U[i])
        if i == 2:
            m = link_mask(2, p.nz, p.ny, p.nx)
            Un[i] = np.where(m[..., None, None], Un[i], U[i])
    return Un


def step(st: State, n_steps=1):
    """Advance the state by n_steps leapfrog steps (returns a new state)."""
    s = st.copy()
    for _ in range(n_steps):
        En, QA, QB = e_update(s)
        Un = u_update(s.U, En, s.p)
        s = State(s.p, Un, En, QA, QB, s.n + 1, s.U, s.extra)
    return s


# ---------------------------------------------------------------------------
# Observables: energy and T^{mu nu} per z slice (Sec. 4)
# ---------------------------------------------------------------------------

def plaquette_terms(U, p: Params):
    """b_ij(x) = 2 (N - Re tr U_ij(x)) / (a_i a_j)^2 for (i,j) in
    (x,y), (x,z), (y,z), zero where the plaquette is absent.

    Evaluated as ||U_i(x) U_j(x+i) - U_j(x) U_i(x+j)||_F^2 / (a_i a_j)^2,
    which equals 2 (N - Re tr U_ij) for unitary links (||A - B||^2 =
    2N - 2 Re tr A B^dagger) and avoids the cancellation of N - Re tr U_ij
    for weak fields (the trace form loses about log10(N / b) digits)."""
    a = p.spacing
    out = {}
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        A = mm(U[i], shift(U[j], i, 1))
        B = mm(U[j], shift(U[i], j, 1))
        f2 = np.sum(np.abs(A - B) ** 2, axis=(-2, -1))
        b = f2 / (a[i] * a[j]) ** 2
        out[(i, j)] = np.where(plaq_mask(i, j, p.nz, p.ny, p.nx), b, 0.0)
    return out


def plaquette_terms_trace(U, p: Params):
    """The same b_ij from the trace form 2 (N - Re tr U_ij) (for checks)."""
    a = p.spacing
    out = {}
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        tr = np.trace(plaquette(U, i, j), axis1=-2, axis2=-1).real
        b = 2.0 * (p.nc - tr) / (a[i] * a[j]) ** 2
        out[(i, j)] = np.where(plaq_mask(i, j, p.nz, p.ny, p.nx), b, 0.0)
    return out


def h_mag(U, p: Params):
    """Magnetic part of the Wilson Hamiltonian (sum over all plaquettes)."""
    vol = p.a_t * p.a_t * p.a_z
    return vol * sum(float(np.sum(b)) for b in plaquette_terms(U, p).values())


def h_el(E1, E2, p: Params):
    """a^3 sum_x sum_i E1_i . E2_i / (2 a_i^2)."""
    vol = p.a_t * p.a_t * p.a_z
    a = p.spacing
    return vol * sum(float(np.sum(E1[i] * E2[i])) / (2 * a[i] ** 2)
                     for i in range(3))


def tmunu(st: State):
    """Per z slice (transverse mean) eps, p_L, p_T, S_L at t_n, and the total
    energy H = a_T^2 a_z nx ny sum_z eps(z).

    Reading (Sec. 4 gives continuum forms only): electric squares are time
    averages e_i^2 = (1/2) sum_a [E_i^a(n-1/2)^2 + E_i^a(n+1/2)^2] / a_i^2
    with E(n+1/2) from a non-committing E update; magnetic terms are the
    single plaquettes at their base site, b_ij above;
      eps = (1/2) sum_i e_i^2 + sum_{i<j} b_ij,
      p_T = (1/2) e_z^2 + b_xy,                      (E_L^2 + B_L^2)/2
      p_L = (1/2)(e_x^2 + e_y^2) + b_xz + b_yz - p_T,  (E_T^2+B_T^2-E_L^2-B_L^2)/2
      S_L = sum_a (Ebar_x^a B_y^a - Ebar_y^a B_x^a),
    Ebar_i = (E_i(n-1/2) + E_i(n+1/2)) / (2 a_i), B_k^a = -2 Im tr(t^a U_ij)
    / (a_i a_j) for cyclic (i, j, k).  The links carry the lower-index field
    (U_i ~ exp(i a A_i)), so the plaquette angle is F_ij = -eps_ijk B^k; the
    minus sign makes S_L the physical Poynting flux, positive for energy
    moving towards +z.  Returns (table[nz][4], H)."""
    p = st.p
    a = p.spacing
    En, _, _ = e_update(st)
    e2 = [0.5 * np.sum(st.E[i] ** 2 + En[i] ** 2, axis=-1) / a[i] ** 2
          for i in range(3)]
    b = plaquette_terms(st.U, p)
    eps = 0.5 * (e2[0] + e2[1] + e2[2]) + b[(0, 1)] + b[(0, 2)] + b[(1, 2)]
    pT = 0.5 * e2[2] + b[(0, 1)]
    pL = 0.5 * (e2[0] + e2[1]) + b[(0, 2)] + b[(1, 2)] - pT
    ebar = [(st.E[i] + En[i]) / (2 * a[i]) for i in range(3)]
    mz = plaq_mask(1, 2, p.nz, p.ny, p.nx)[..., None]
    bx = np.where(mz, -2 * im_tr_ta(plaquette(st.U, 1, 2), p.nc)
                  / (a[1] * a[2]), 0.0)
    by = np.where(mz, -2 * im_tr_ta(plaquette(st.U, 2, 0), p.nc)
                  / (a[2] * a[0]), 0.0)
    sl = np.sum(ebar[0] * by - ebar[1] * bx, axis=-1)
    area = p.nx * p.ny
    tab = np.stack([eps.sum(axis=(1, 2)), pL.sum(axis=(1, 2)),
                    pT.sum(axis=(1, 2)), sl.sum(axis=(1, 2))], axis=1) / area
    H = p.a_t * p.a_t * p.a_z * area * float(np.sum(tab[:, 0]))
    return tab, H


# ---------------------------------------------------------------------------
# Diagnostics
# ---------------------------------------------------------------------------

def unitarity_dev(U):
    """max over links of |U^dag U - 1| and |det U - 1|."""
    nc = U.shape[-1]
    d1 = np.max(np.abs(mm(dag(U), U) - np.eye(nc)))
    d2 = np.max(np.abs(np.linalg.det(U) - 1.0))
    return float(d1), float(d2)


def gauge_transform(st: State, omega):
    """U_i(x) -> Om(x) U_i(x) Om^dag(x+i); adjoint fields E, Q rotated by
    Om(x).  omega[z][y][x][N][N]; the z link at the last slice is absent and
    stays the identity."""
    p = st.p
    s = st.copy()
    for i in range(3):
        s.U[i] = mm(omega, st.U[i], dag(shift(omega, i, 1)))
        s.E[i] = mat_to_alg(mm(omega, alg_to_mat(st.E[i], p.nc),
                               dag(omega)), p.nc)
    last = p.nz - 1
    s.U[2][last] = np.eye(p.nc)
    if st.U_prev is not None:
        for i in range(3):
            s.U_prev[i] = mm(omega, st.U_prev[i], dag(shift(omega, i, 1)))
        s.U_prev[2][last] = np.eye(p.nc)
    for name in ("QA", "QB"):
        q = getattr(st, name)
        setattr(s, name, mat_to_alg(mm(omega, alg_to_mat(q, p.nc),
                                       dag(omega)), p.nc))
    return s


# ---------------------------------------------------------------------------
# One step at selected sites only (for checks of full-size lattices whose
# complete evolution the oracle cannot afford): the same formulas as
# force/hop/u_update, written with explicit neighbour indices.
# ---------------------------------------------------------------------------

def step_at_sites(st: State, sites):
    """E(t_{n+1/2}) and U(t_{n+1}) at the given (iz, iy, ix) sites.
    Returns (E_new[k][3][a], U_new[k][3][N][N]); absent links (U_z on the
    last slice) come back unchanged with E = 0."""
    p = st.p
    nc, na = p.nc, p.na
    a = p.spacing
    U = st.U
    hop_now = hop_at(st.n, hop_ratio(p))

    def link(d, z, y, x):
        return U[d][z, y % p.ny, x % p.nx]

    def exists(d, z):
        return 0 <= z <= p.nz - 1 and (d != 2 or z <= p.nz - 2)

    def plaq(i, j, z, y, x):
        """Plaquette at base (z, y, x) in plane (i, j) or None."""
        off = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]     # (dz, dy, dx) of e_d
        bi = (z + off[i][0], y + off[i][1], x + off[i][2])
        bj = (z + off[j][0], y + off[j][1], x + off[j][2])
        if not (exists(i, z) and exists(j, bi[0]) and exists(i, bj[0])
                and exists(j, z)):
            return None
        return (link(i, z, y, x) @ link(j, *bi) @ dag(link(i, *bj))
                @ dag(link(j, z, y, x)))

    t = generators(nc)
    off = [(0, 0, 1), (0, 1, 0), (1, 0, 0)]
    E_out = np.zeros((len(sites), 3, na))
    U_out = np.zeros((len(sites), 3, nc, nc), complex)
    for k, (z, y, x) in enumerate(sites):
        for i in range(3):
            if not exists(i, z):
                U_out[k, i] = link(i, z, y, x)
                continue
            F = np.zeros(na)
            for j in range(3):
                if j == i:
                    continue
                P = plaq(i, j, z, y, x) if i < j else None
                if i > j:
                    Pj = plaq(j, i, z, y, x)
                    P = None if Pj is None else dag(Pj)
                if P is not None:
                    F -= (2 / a[j] ** 2) * im_tr_ta(P, nc)
                bz, by, bx = z - off[j][0], y - off[j][1], x - off[j][2]
                if 0 <= bz:
                    lo, hi = min(i, j), max(i, j)
                    Pb = plaq(lo, hi, bz, by, bx)
                    if Pb is not None:
                        Uj = link(j, bz, by, bx)
                        # U_{i,-j}(x) = U_j^dag(x-j) U_{j,i}(x-j) U_j(x-j)
                        Pji = Pb if (j, i) == (lo, hi) else dag(Pb)
                        F -= (2 / a[j] ** 2) * im_tr_ta(dag(Uj) @ Pji @ Uj,
                                                        nc)
            e = st.E[i][z, y, x] + p.dt * F
            if i == 2 and hop_now:
                dj = np.zeros(na)
                Uz = link(2, z, y, x)
                dj -= st.QB[z, y, x] * p.a_z ** 2
                if z + 1 <= p.nz - 1:
                    q = alg_to_mat(st.QA[z + 1, y, x], nc)
                    dj += mat_to_alg(Uz @ q @ dag(Uz), nc) * p.a_z ** 2
                e = e + dj
            E_out[k, i] = e
            U_out[k, i] = expi_alg(e, p.dt, nc) @ link(i, z, y, x)
    return E_out, U_out


# ---------------------------------------------------------------------------
# Improved (semi-implicit) scheme against the numerical Cherenkov
# instability (Sec. 3, the paragraph after Eq. gauss and Fig. wilson (b);
# Sec. 5).  The paper gives its properties, not its equations: some spatial
# plaquette terms are replaced by time-averaged plaquette-like terms built
# from links of the past, present and future time slices; the resulting
# semi-implicit system is solved iteratively; propagation along z is free
# of numerical dispersion.
#
# Reading adopted here.  In the force on link i the staple pair of plane
# (i, j) is averaged over time slots m = n+1, n, n-1 with weights
# (1/4, 1/2, 1/4); in a transverse plane (x, y) every link of the loop is
# taken at slot m, in a plane containing z only the z links are taken at
# slot m and the transverse links stay at t_n.  In the abelian,
# small-amplitude limit this gives
#   (2/dt)^2 sin^2(w dt/2) = (2/a_z)^2 sin^2(k_z a_z/2)
#                            + cos^2(w dt/2) sum_T (2/a_T)^2 sin^2(k_T a_T/2),
# exactly dispersion-free along z at dt = a_z, w >= k_z for every mode, and
# transversally unconditionally stable; the abelian Gauss law is conserved
# because each plane keeps one antisymmetric field strength.  Weights
# (0, 1, 0) give back the leapfrog force bit for bit.
# ---------------------------------------------------------------------------

IMPLICIT_WEIGHTS = (0.25, 0.5, 0.25)     # slots: U(t_{n+1}), U(t_n), U(t_{n-1})


def force_implicit(Us, p: Params, w=IMPLICIT_WEIGHTS):
    """Time-averaged force; Us = (U_next, U_now, U_prev)."""
    nz, ny, nx = p.nz, p.ny, p.nx
    a = p.spacing
    nc = p.nc
    F = np.zeros((3, nz, ny, nx, p.na))
    for i in range(3):
        for j in range(3):
            if j == i:
                continue
            zplane = 2 in (i, j)
            mf = plaq_mask(i, j, nz, ny, nx)
            mb = shift(plaq_mask(i, j, nz, ny, nx), j, -1)
            if j == 2:
                mb = mb & (z_index(nz, ny, nx) >= 1)
            for m in range(3):
                if w[m] == 0.0:
                    continue
                L = np.empty_like(Us[1])
                for d in range(3):
                    L[d] = Us[m][d] if (not zplane or d == 2) else Us[1][d]
                fwd = im_tr_ta(plaquette(L, i, j), nc)
                bwd = im_tr_ta(plaquette_minus(L, i, j), nc)
                F[i] -= (2.0 / a[j] ** 2) * w[m] * (
                    np.where(mf[..., None], fwd, 0.0)
                    + np.where(mb[..., None], bwd, 0.0))
        F[i] = np.where(link_mask(i, nz, ny, nx)[..., None], F[i], 0.0)
    return F


class NotConverged(RuntimeError):
    pass


# How the system is iterated (the paper says only that it is solved
# iteratively; reading adopted here).  One sweep maps E to
# G(E) = E(t_{n-1/2}) + dt J + dt F(exp(i dt E) U(t_n), U(t_n), U(t_{n-1})).
# In the small-amplitude abelian limit its Jacobian is -w_0 dt^2 K', with
# w_0 the weight of the slot t_{n+1} and K' the lattice curl-curl acting on
# the links that take that slot: block triangular, with the curl-curl of
# the (x, y) plane and the transverse Laplacian of A_z on its diagonal,
# whose eigenvalues lie in [0, 8 / a_T^2].  So the eigenvalues of the sweep
# lie in [-c, 0] with c = 8 w_0 dt^2 / a_T^2: the plain iteration
# E <- G(E) contracts by c per sweep (c = 1/8 at dt = a_T/4) and diverges
# for c >= 1.  Every sweep after the first is therefore relaxed,
# E <- (1 - omega) E + omega G(E) with omega = 2 / (2 + c), which maps
# [-c, 0] into [-c/(2+c), c/(2+c)]: the contraction is halved at small c
# and stays below 1 for every dt.  The first sweep takes the full step
# G(E(t_{n-1/2})), whose change is the bulk of the update.  The fixed point
# is the same; weights (0, 1, 0) give omega = 1.
def implicit_omega(p: Params, w=IMPLICIT_WEIGHTS):
    """Relaxation of the sweeps after the first."""
    c = 8.0 * w[0] * p.dt * p.dt / (p.a_t * p.a_t)
    return 2.0 / (2.0 + c)


def relax(Ek, G, omega):
    """(1 - omega) Ek + omega G; exactly G when omega = 1."""
    if omega == 1.0:
        return G
    return (1.0 - omega) * Ek + omega * G


def step_implicit(st: State, n_steps=1, w=IMPLICIT_WEIGHTS, tol=1e-14,
                  max_iter=100, omega=None):
    """Semi-implicit steps: fixed-point iteration on E(t_{n+1/2}), starting
    from U(t_{n+1}) = exp(i dt E(t_{n-1/2})) U(t_n), every sweep after the
    first relaxed by omega (implicit_omega unless given), until the largest
    change of any E component is below tol.  The CPIC hop and its current
    are the leapfrog's (they use U(t_n) only).  U_prev must hold
    U(t_{n-1})."""
    s = st.copy()
    p = s.p
    om = implicit_omega(p, w) if omega is None else omega
    for _ in range(n_steps):
        QA, QB, djz = hop(s)
        Ek = s.E
        X = u_update(s.U, Ek, p)
        deltas = []
        for it in range(max_iter):
            F = force_implicit((X, s.U, s.U_prev), p, w)
            G = s.E + p.dt * F
            G[2] = G[2] + djz
            G[2] = np.where(link_mask(2, p.nz, p.ny, p.nx)[..., None],
                            G[2], 0.0)
            En = relax(Ek, G, 1.0 if it == 0 else om)
            delta = float(np.max(np.abs(En - Ek)))
            deltas.append(delta)
            Ek = En
            X = u_update(s.U, En, p)
            if delta < tol:
                break
        else:
            raise NotConverged("implicit step did not converge")
        s.extra["iters"] = it + 1
        s.extra["deltas"] = deltas
        s = State(p, X, Ek, QA, QB, s.n + 1, s.U, s.extra)
    return s
