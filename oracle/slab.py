"""Decomposition of the oracle's leapfrog step into z slabs (test
infrastructure, like the rest of oracle/: only tests may use it).

The beam axis is the long axis of the paper's lattices (Sec. 4: 2048 cells
along z against 192^2 transversally), so a run on several devices splits it
into slabs of consecutive z slices, one per rank.  This module states the
decomposition on the oracle, independently of the CUDA library, so that a
multi-rank run can be checked against the monolithic oracle bit for bit.

Rank r owns the slices [z0, z1) and keeps one halo slice on each side that
has a neighbour: z0 - 1 below, z1 above.  Its local lattice is the slab with
its halos, treated by the unmodified oracle step (oracle.glasma_oracle.step)
as a lattice of its own with open ends.  That local step is exact on every
owned slice because Sec. 3 Eq. lattice_1 couples a link only to the slices
z - 1, z and z + 1, and the halos hold exactly what the owner of those
slices holds:

* from the rank below (lower halo, slice z0 - 1): the links of all three
  directions and E_z (the backward z-staples of the transverse links at z0,
  the z-term of the Gauss divergence at z0), and the charge of nucleus B on
  that slice, which the next hop carries into z0 along U_z(z0 - 1);
* from the rank above (upper halo, slice z1): the transverse links (the
  forward z-staples and z-plaquettes of slice z1 - 1) and the charge of
  nucleus A on that slice, which the next hop carries into z1 - 1 along
  U_z(z1 - 1), depositing its current on that owned link.

A charge that leaves the slab is transported and deposited by the owner of
the link it crosses, so each rank drops its charges that have left after the
step (B on the upper halo, A on the lower halo); the halo slices are
refreshed from the neighbours before every step.  Observables: the
T^{mu nu}(z) rows of the owned slices, gathered in rank order and summed in
z order (Sec. 4), and the Gauss residual maxima, folded across ranks.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from oracle import glasma_oracle as O


def slab_bounds(nz, nranks):
    """Contiguous z ranges [z0, z1), sizes differing by at most one slice."""
    base, extra = divmod(nz, nranks)
    out, z = [], 0
    for r in range(nranks):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


@dataclass
class Slab:
    st: O.State          # local lattice: the slab with its halo slices
    z0: int              # first owned global slice
    z1: int              # one past the last owned global slice
    lo: int              # local index of slice z0 (1 with a lower halo)
    hi: int              # local index of slice z1
    nz: int              # global number of slices

    @property
    def has_below(self):
        return self.lo == 1

    @property
    def has_above(self):
        return self.hi < self.st.p.nz


def make_slab(st: O.State, z0, z1):
    """Slab [z0, z1) of a global state.  Its halo slices start blank
    (identity links, zero fields and charges): everything in them comes from
    the neighbours' messages, exchanged before every step."""
    p = st.p
    lo = 1 if z0 > 0 else 0
    hi_halo = 1 if z1 < p.nz else 0
    g0, g1 = z0 - lo, z1 + hi_halo
    pl = O.Params(**{**p.__dict__, "nz": g1 - g0})
    U = st.U[:, g0:g1].copy()
    E = st.E[:, g0:g1].copy()
    QA = st.QA[g0:g1].copy()
    QB = st.QB[g0:g1].copy()
    hi = (g1 - g0) - hi_halo
    for k in list(range(lo)) + list(range(hi, g1 - g0)):
        U[:, k] = np.eye(p.nc)
        E[:, k] = 0.0
    Up = None
    if st.U_prev is not None:
        Up = st.U_prev[:, g0:g1].copy()
        for k in list(range(lo)) + list(range(hi, g1 - g0)):
            Up[:, k] = np.eye(p.nc)
    # charges live only on owned slices; halo charges arrive by exchange
    _clear_halo_charges(QA, QB, lo, hi)
    return Slab(O.State(pl, U, E, QA, QB, st.n, Up), z0, z1, lo, hi, p.nz)


def _clear_halo_charges(QA, QB, lo, hi):
    QA[:lo] = 0.0
    QB[:lo] = 0.0
    QA[hi:] = 0.0
    QB[hi:] = 0.0


def message_up(s: Slab):
    """To the rank above: links (3 directions), E_z and nucleus B's charge of
    the top owned slice; under the improved scheme also its z links at
    t_{n-1} (the t_{n-1} slot's z staples of the slice above)."""
    k = s.hi - 1
    m = dict(U=s.st.U[:, k].copy(), Ez=s.st.E[2][k].copy(), QB=s.st.QB[k].copy())
    if s.st.U_prev is not None:
        m["Uprev_z"] = s.st.U_prev[2][k].copy()
    return m


def message_down(s: Slab):
    """To the rank below: transverse links and nucleus A's charge of the
    bottom owned slice."""
    k = s.lo
    return dict(U=s.st.U[0:2, k].copy(), QA=s.st.QA[k].copy())


def receive_from_below(s: Slab, m):
    s.st.U[:, 0] = m["U"]
    s.st.E[2][0] = m["Ez"]
    s.st.QB[0] = m["QB"]
    if "Uprev_z" in m:
        s.st.U_prev[2][0] = m["Uprev_z"]


def receive_from_above(s: Slab, m):
    k = s.hi
    s.st.U[0:2, k] = m["U"]
    s.st.QA[k] = m["QA"]


def local_step(s: Slab):
    """One oracle step of the local lattice; afterwards the charges that
    left the owned slices (their owners downstream have moved them) are
    dropped."""
    s.st = O.step(s.st, 1)
    _clear_halo_charges(s.st.QA, s.st.QB, s.lo, s.hi)


def owned(s: Slab):
    """(U, E, QA, QB) of the owned slices."""
    a, b = s.lo, s.hi
    return s.st.U[:, a:b], s.st.E[:, a:b], s.st.QA[a:b], s.st.QB[a:b]


def tmunu_rows(s: Slab):
    """T^{mu nu}(z) rows (eps, p_L, p_T, S_L) of the owned slices."""
    tab, _ = O.tmunu(s.st)
    return tab[s.lo:s.hi]


def energy_from_rows(p: O.Params, rows):
    """H from the gathered rows in global z order (the monolithic sum)."""
    return p.a_t * p.a_t * p.a_z * (p.nx * p.ny) * float(np.sum(rows[:, 0]))


def gauss_partial(s: Slab):
    """(max |G|, sum G^2, count, max |rho|) over the owned slices."""
    g = O.gauss_divergence(s.st.U, s.st.E, s.st.p) - (s.st.QA + s.st.QB)
    rho = s.st.QA + s.st.QB
    g = g[s.lo:s.hi]
    return (float(np.max(np.abs(g))), float(np.sum(g ** 2)), g.size,
            float(np.max(np.abs(rho[s.lo:s.hi]))))


def run_in_process(st: O.State, nranks, steps):
    """All slabs of one process, messages passed directly: the reference
    protocol for any number of ranks.  Returns the slabs after `steps`."""
    slabs = [make_slab(st, z0, z1) for z0, z1 in slab_bounds(st.p.nz, nranks)]
    for _ in range(steps):
        exchange_in_process(slabs)
        for s in slabs:
            local_step(s)
    exchange_in_process(slabs)
    return slabs


def exchange_in_process(slabs):
    ups = [message_up(s) for s in slabs]
    downs = [message_down(s) for s in slabs]
    for r, s in enumerate(slabs):
        if s.has_below:
            receive_from_below(s, ups[r - 1])
        if s.has_above:
            receive_from_above(s, downs[r + 1])


# ---------------------------------------------------------------------------
# The improved scheme (oracle.glasma_oracle.step_implicit) on slabs.
#
# Its fixed-point sweeps couple the slices through the iterate U(t_{n+1}),
# but only through z links: in a plane containing z only the z links take
# the time slot, the transverse links stay at t_n.  The force on the z link
# of slice z then reads the z links of slice z at every slot and the
# transverse links of slices z and z + 1 at t_n; so each rank evaluates the
# z link of its lower halo slice itself, every sweep, from what the step's
# halo brings (the links at t_n of both halo slices, E_z and U(t_{n-1})'s z
# link of the lower one, the charges whose hop crosses it), with the same
# arithmetic as its owner, and no sweep needs a message.  What couples the
# ranks is the stopping test: it takes the largest change of E over the
# whole lattice, i.e. each rank's maximum over its owned slices folded with
# max across ranks, so every rank stops after the same sweep as the
# monolithic step.
# ---------------------------------------------------------------------------

def implicit_begin(s: Slab):
    """Hop (the leapfrog's, from U(t_n)) and the first iterate
    U(t_{n+1}) = exp(i dt E(t_{n-1/2})) U(t_n) of the local lattice."""
    st = s.st
    QA, QB, djz = O.hop(st)
    s.work = dict(QA=QA, QB=QB, djz=djz, Ek=st.E, X=O.u_update(st.U, st.E, st.p))


def implicit_sweep(s: Slab, k, w=O.IMPLICIT_WEIGHTS):
    """Sweep k: G = E(t_{n-1/2}) + dt F(X^(k), U(t_n), U(t_{n-1})) + dt J,
    E^(k+1) = G for k = 0 and relaxed towards G after
    (oracle.glasma_oracle.implicit_omega), X^(k+1) = exp(i dt E^(k+1))
    U(t_n).  Returns the largest change of E over the owned slices."""
    st, W = s.st, s.work
    p = st.p
    F = O.force_implicit((W["X"], st.U, st.U_prev), p, w)
    G = st.E + p.dt * F
    G[2] = G[2] + W["djz"]
    G[2] = np.where(O.link_mask(2, p.nz, p.ny, p.nx)[..., None], G[2], 0.0)
    En = O.relax(W["Ek"], G, 1.0 if k == 0 else O.implicit_omega(p, w))
    delta = float(np.max(np.abs(En - W["Ek"])[:, s.lo:s.hi]))
    W["Ek"] = En
    W["X"] = O.u_update(st.U, En, p)
    return delta


def implicit_end(s: Slab, iters):
    """Commit the step: the last iterate and its E; U(t_n) becomes U_prev."""
    W = s.work
    s.st = O.State(s.st.p, W["X"], W["Ek"], W["QA"], W["QB"], s.st.n + 1, s.st.U,
                   dict(s.st.extra, iters=iters))
    _clear_halo_charges(s.st.QA, s.st.QB, s.lo, s.hi)
    s.work = None


def run_implicit_in_process(st: O.State, nranks, steps, w=O.IMPLICIT_WEIGHTS,
                            tol=1e-14, max_iter=100, on_sweep=None):
    """The improved scheme on nranks slabs of one process; every sweep's
    largest change is the max over the ranks' owned slices.  on_sweep(slabs)
    is called after every sweep (for checks).  Returns the slabs after
    `steps`, each with its sweep count in st.extra["iters"]."""
    slabs = [make_slab(st, z0, z1) for z0, z1 in slab_bounds(st.p.nz, nranks)]
    for _ in range(steps):
        exchange_in_process(slabs)
        for s in slabs:
            implicit_begin(s)
        for it in range(max_iter):
            delta = max(implicit_sweep(s, it, w) for s in slabs)
            if on_sweep:
                on_sweep(slabs)
            if delta < tol:
                break
        else:
            raise O.NotConverged("implicit step did not converge")
        for s in slabs:
            implicit_end(s, it + 1)
    exchange_in_process(slabs)
    return slabs
