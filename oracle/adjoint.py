"""Plain FP64 CPU oracle of the gradient of a mid-rapidity energy
observable with respect to the initial MV colour charges (SU(2)).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import this module.  The CUDA
library never calls it and shares no code with it.

What it computes: the same chain as oracle/glasma_oracle.py -- MV initial
conditions from rho_N^a(x_T) (Sec. 2 and Sec. 3 Eqs. single_sheet,
3d_colorfield_1/2, Sec. 4 Gaussian profile), n leapfrog CPIC steps (Sec. 3
Eqs. lattice_1, lattice_2, continuity and the NGP transport) and the energy
density of Sec. 4 -- written again with torch tensors (complex128 matrices,
torch.linalg.matrix_exp for the exponentials, the closed-form SU(2)
logarithm) so that torch's reverse-mode autograd differentiates it.  The
observable is the mid-rapidity integrated energy density

    O = a_z sum_{iz : |iz a_z - z_c| < half_width} eps(iz),

eps the transverse mean of the energy density at the final step (the
T^{00} of glasma_oracle.tmunu), z_c the box centre.  Its gradient with
respect to rho (both nuclei, all colours, every transverse site) is the
"oracle's own adjoint" that the CUDA adjoint is checked against.  The
non-differentiable bookkeeping (profile values, hop schedule, masks) is
taken from glasma_oracle.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import glasma_oracle as O

C128 = torch.complex128
F64 = torch.float64


def _t(nc):
    return torch.as_tensor(O.generators(nc), dtype=C128)


def dag(x):
    return x.conj().transpose(-1, -2)


def alg_to_mat(v, nc):
    return torch.einsum("...a,aij->...ij", v.to(C128), _t(nc))


def mat_to_alg(h, nc):
    return 2.0 * torch.einsum("aij,...ji->...a", _t(nc), h).real


def im_tr_ta(x, nc):
    return torch.einsum("aij,...ji->...a", _t(nc), x).imag


def expi(v, c, nc):
    """exp(i c v^a t^a); c a scalar or an array broadcasting against v[..., 0]."""
    c = torch.as_tensor(c, dtype=F64)
    h = alg_to_mat(v, nc) * c.to(C128)[..., None, None]
    return torch.linalg.matrix_exp(1j * h)


def log_su2(w):
    """h with exp(i h.sigma/2) = W for W = w0 + i w.sigma (SU(2)):
    |h| = 2 atan2(|w|, w0) along w (the principal branch)."""
    w0 = 0.5 * (w[..., 0, 0] + w[..., 1, 1]).real
    wv = torch.stack([w[..., 0, 1].imag, w[..., 0, 1].real, w[..., 0, 0].imag], dim=-1)
    r2 = torch.sum(wv * wv, dim=-1)
    tiny = r2 == 0.0
    r = torch.sqrt(torch.where(tiny, torch.ones_like(r2), r2))
    k = torch.where(tiny, 2.0 / w0, 2.0 * torch.atan2(r, w0) / r)
    return k[..., None] * wv


AXIS = {0: 2, 1: 1, 2: 0}


def shift(f, i, s):
    return torch.roll(f, -s, dims=AXIS[i])


def _m(mask, like):
    return torch.as_tensor(mask).reshape(mask.shape + (1,) * (like.dim() - mask.ndim))


def poisson(rho, p):
    ny, nx = rho.shape[-2:]
    kx = 2 * np.pi * np.fft.fftfreq(nx)
    ky = 2 * np.pi * np.fft.fftfreq(ny)
    k2 = ((4.0 / p.a_t ** 2) * np.sin(ky[:, None] / 2) ** 2
          + (4.0 / p.a_t ** 2) * np.sin(kx[None, :] / 2) ** 2)
    kern = 1.0 / (k2 + p.m_ir ** 2)
    if p.uv_cutoff > 0:
        kern = np.where(k2 > p.uv_cutoff ** 2, 0.0, kern)
    kern = torch.as_tensor(kern, dtype=F64)
    return torch.fft.ifft2(torch.fft.fft2(rho) * kern).real


def links_at(p, phi, t_shift):
    nc = p.nc
    zb, za, _ = O.nucleus_positions(p)
    zb = zb + t_shift
    za = za - t_shift
    z = np.arange(p.nz) * p.a_z
    lam = {"A": O.big_lambda(z, za, p.sigma_l, "A"),
           "B": O.big_lambda(z, zb, p.sigma_l, "B")}
    vd = {}
    for k, N in (("A", 0), ("B", 1)):
        v = torch.movedim(phi[N], 0, -1)                      # [y][x][a]
        c = torch.as_tensor(lam[k], dtype=F64)[:, None, None]  # [z][1][1]
        vd[k] = expi(v[None], c, nc)                          # [z][y][x][N][N]
    U = []
    for i in (0, 1):
        ua = dag(vd["A"]) @ shift(vd["A"], i, 1)
        ub = dag(vd["B"]) @ shift(vd["B"], i, 1)
        U.append(ua @ ub)
    eye = torch.eye(nc, dtype=C128).expand(p.nz, p.ny, p.nx, nc, nc)
    U.append(eye.clone())
    return torch.stack(U)


def transport_back(U, F, i, nc):
    um = shift(U[i], i, -1)
    fm = shift(alg_to_mat(F, nc), i, -1)
    return mat_to_alg(dag(um) @ fm @ um, nc)


def gauss_divergence(U, E, p):
    a = p.spacing
    iz = torch.as_tensor(np.array(O.z_index(p.nz, p.ny, p.nx)))[..., None]
    div = torch.zeros(E.shape[1:], dtype=F64)
    for i in range(3):
        back = transport_back(U, E[i], i, p.nc)
        if i == 2:
            back = torch.where(iz >= 1, back, torch.zeros_like(back))
        div = div + (E[i] - back) / a[i] ** 2
    return div


def init_mv(p, rho):
    """(U, E, QA, QB) at step 0 as differentiable functions of rho."""
    phi = poisson(rho, p)
    U0 = links_at(p, phi, 0.0)
    Um = links_at(p, phi, -p.dt)
    Es = []
    for i in (0, 1):
        same = torch.all(torch.all(U0[i] == Um[i], dim=-1), dim=-1)
        w = U0[i] @ dag(Um[i])
        eye = torch.eye(p.nc, dtype=C128)
        w = torch.where(same[..., None, None], eye, w)
        h = log_su2(w)
        Es.append(torch.where(same[..., None], torch.zeros_like(h), h) / p.dt)
    Es.append(torch.zeros_like(Es[0]))
    E = torch.stack(Es)
    rho3 = gauss_divergence(U0, E, p)
    _, _, zc = O.nucleus_positions(p)
    z = torch.as_tensor(np.arange(p.nz) * p.a_z)[:, None, None, None]
    QA = torch.where(z > zc, rho3, torch.zeros_like(rho3))
    QB = torch.where(z < zc, rho3, torch.zeros_like(rho3))
    return U0, E, QA, QB


def force(U, p):
    nz, ny, nx = p.nz, p.ny, p.nx
    a = p.spacing
    F = []
    for i in range(3):
        Fi = torch.zeros((nz, ny, nx, p.na), dtype=F64)
        for j in range(3):
            if j == i:
                continue
            fwd = im_tr_ta(U[i] @ shift(U[j], i, 1) @ dag(shift(U[i], j, 1))
                           @ dag(U[j]), p.nc)
            bwd = im_tr_ta(U[i] @ dag(shift(shift(U[j], i, 1), j, -1))
                           @ dag(shift(U[i], j, -1)) @ shift(U[j], j, -1), p.nc)
            mf = O.plaq_mask(i, j, nz, ny, nx)
            mb = np.roll(mf, 1, axis=AXIS[j])
            if j == 2:
                mb = mb & (O.z_index(nz, ny, nx) >= 1)
            Fi = Fi - (2.0 / a[j] ** 2) * (
                torch.where(_m(mf, fwd), fwd, torch.zeros_like(fwd))
                + torch.where(_m(mb, bwd), bwd, torch.zeros_like(bwd)))
        lm = O.link_mask(i, nz, ny, nx)
        F.append(torch.where(_m(lm, Fi), Fi, torch.zeros_like(Fi)))
    return torch.stack(F)


def transport_charge(U, Q, direction, nc):
    nz = Q.shape[0]
    Uz = U[2]
    qm = alg_to_mat(Q, nc)
    if direction > 0:
        moved = mat_to_alg(dag(Uz) @ qm @ Uz, nc)
        Qn = torch.cat([torch.zeros_like(moved[:1]), moved[:-1]])
        dj = torch.cat([-Q[:-1], torch.zeros_like(Q[-1:])])
        return Qn, dj
    qs = torch.cat([qm[1:], torch.zeros_like(qm[:1])])
    moved = mat_to_alg(Uz @ qs @ dag(Uz), nc)
    Qn = torch.cat([moved[:-1], torch.zeros_like(moved[-1:])])
    return Qn, Qn


def e_update(U, E, QA, QB, n, p):
    djz = torch.zeros_like(QA)
    if O.hop_at(n, O.hop_ratio(p)):
        QB, djb = transport_charge(U, QB, +1, p.nc)
        QA, dja = transport_charge(U, QA, -1, p.nc)
        djz = djz + djb * p.a_z ** 2
        djz = djz + dja * p.a_z ** 2
    F = force(U, p)
    En = E + p.dt * F
    lm = torch.as_tensor(O.link_mask(2, p.nz, p.ny, p.nx))[..., None]
    ez = torch.where(lm, En[2] + djz, torch.zeros_like(En[2]))
    En = torch.stack([En[0], En[1], ez])
    return En, QA, QB


def u_update(U, E, p):
    out = []
    for i in range(3):
        Ui = expi(E[i], p.dt, p.nc) @ U[i]
        if i == 2:
            lm = torch.as_tensor(O.link_mask(2, p.nz, p.ny, p.nx))[..., None, None]
            Ui = torch.where(lm, Ui, U[i])
        out.append(Ui)
    return torch.stack(out)


def energy_density(U, E, QA, QB, n, p):
    """Transverse mean of eps per z slice at step n (glasma_oracle.tmunu)."""
    a = p.spacing
    En, _, _ = e_update(U, E, QA, QB, n, p)
    eps = torch.zeros((p.nz, p.ny, p.nx), dtype=F64)
    for i in range(3):
        eps = eps + 0.5 * 0.5 * torch.sum(E[i] ** 2 + En[i] ** 2, dim=-1) / a[i] ** 2
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        A = U[i] @ shift(U[j], i, 1)
        B = U[j] @ shift(U[i], j, 1)
        f2 = torch.sum(torch.abs(A - B) ** 2, dim=(-2, -1)) / (a[i] * a[j]) ** 2
        mk = torch.as_tensor(O.plaq_mask(i, j, p.nz, p.ny, p.nx))
        eps = eps + torch.where(mk, f2, torch.zeros_like(f2))
    return eps.mean(dim=(1, 2))


def slice_weights(p, half_width):
    """a_z on the slices with |iz a_z - z_c| < half_width, 0 elsewhere."""
    _, _, zc = O.nucleus_positions(p)
    z = np.arange(p.nz) * p.a_z
    return np.where(np.abs(z - zc) < half_width, p.a_z, 0.0)


def observable(p, rho, n_steps, half_width):
    """O(rho) as a differentiable torch scalar (rho: torch [2][3][ny][nx])."""
    if p.nc != 2:
        raise ValueError("the adjoint oracle covers SU(2)")
    U, E, QA, QB = init_mv(p, rho)
    for n in range(n_steps):
        En, QA, QB = e_update(U, E, QA, QB, n, p)
        U = u_update(U, En, p)
        E = En
    eps = energy_density(U, E, QA, QB, n_steps, p)
    w = torch.as_tensor(slice_weights(p, half_width), dtype=F64)
    return torch.sum(w * eps)


def gradient(p, rho, n_steps, half_width):
    """(O, dO/drho) for rho a numpy [2][3][ny][nx] array."""
    r = torch.tensor(np.asarray(rho, dtype=np.float64), requires_grad=True)
    val = observable(p, r, n_steps, half_width)
    val.backward()
    return float(val.item()), r.grad.numpy().copy()


def observable_numpy(p, rho, n_steps, half_width):
    """The same O evaluated with the numpy oracle (no autograd)."""
    st = O.step(O.init_mv(p, np.asarray(rho, dtype=np.float64)), n_steps)
    tab, _ = O.tmunu(st)
    return float(np.sum(slice_weights(p, half_width) * tab[:, 0]))
