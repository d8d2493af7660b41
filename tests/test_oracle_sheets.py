"""Pins of the longitudinal colour structure in the oracle (several colour
sheets per nucleus combined in a path-ordered Wilson line): it reduces to
the single-sheet state when the sheets carry the same charge, the order of
the factors matters once they do not commute, the evolution stays
Gauss-law exact and unitary, and the charge density then changes colour
along the beam axis, which a single sheet cannot do."""
import numpy as np
import pytest

import glasma_inputs as gi
from oracle import glasma_oracle as O


def _cfg(nc, S, **kw):
    return dict(gi.small_config(nc, nz=64, nx=6, ny=5, sigma_l=3.0, seed=21, **kw), n_sheets=S)


@pytest.mark.parametrize("nc", [2, 3])
def test_equal_sheets_reproduce_the_single_sheet_state(nc):
    S = 4
    p1 = O.Params.from_dict(_cfg(nc, 1))
    pS = O.Params.from_dict(_cfg(nc, S))
    rho = gi.mv_rho(21, nc, 6, 5, 0.1)
    st1 = O.init_mv(p1, rho)
    stS = O.init_mv(pS, np.broadcast_to(rho / S, (S,) + rho.shape).copy())
    # commuting factors with sum_s Lambda_s = S Lambda
    assert np.max(np.abs(stS.U - st1.U)) < 1e-13
    assert np.max(np.abs(stS.E - st1.E)) < 1e-12 * np.max(np.abs(st1.E))
    assert np.max(np.abs(stS.QA + stS.QB - st1.QA - st1.QB)) < 1e-12 * np.max(np.abs(st1.QA))


def test_sheet_profiles_partition_the_profile():
    lam = np.linspace(0, 1, 101)
    ls = O.sheet_profiles(lam, 5)
    assert np.allclose(ls.sum(axis=0), 5 * lam, rtol=0, atol=1e-15)
    assert np.all((ls >= 0) & (ls <= 1))
    # sheet s is complete before sheet s + 1 starts
    assert np.all(ls[1][ls[0] < 1] == 0)


def test_path_order_matters_and_the_evolution_stays_exact():
    S = 3
    p = O.Params.from_dict(_cfg(2, S))
    rho = gi.mv_rho(21, 2, 6, 5, 0.1, sheets=S)
    st = O.init_mv(p, rho)
    st_rev = O.init_mv(p, rho[::-1].copy())
    assert np.max(np.abs(st.U - st_rev.U)) > 1e-4
    st2 = O.step(st, 24)
    gmax, _, rmax = O.gauss_residual(st2)
    assert gmax <= 1e-12 * rmax
    d1, d2 = O.unitarity_dev(st2.U)
    assert d1 < 1e-13 and d2 < 1e-13


def _colour_cos(Q, z1, z2):
    a, b = Q[z1].reshape(-1, Q.shape[-1]), Q[z2].reshape(-1, Q.shape[-1])
    num = np.sum(a * b, axis=1)
    den = np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1)
    return float(np.mean(np.abs(num / den)))


def test_charge_colour_changes_along_the_beam_only_with_sheets():
    """Nucleus B's charge density at the front and back of its profile, in
    the weak-field (nearly abelian) regime g^2 mu a = 0.02: one sheet gives
    the same colour direction at every z (mean |cos| > 0.98); four
    independent sheets decorrelate front and back (random directions give
    1/2), while neighbouring slices of one sheet stay parallel."""
    out = {}
    for S in (1, 4):
        p = O.Params.from_dict(dict(_cfg(2, S), g2mu=0.02))
        st = O.init_mv(p, gi.mv_rho(21, 2, 6, 5, 0.02, sheets=S))
        w = np.sum(st.QB ** 2, axis=(1, 2, 3))
        zs = np.nonzero(w > 1e-6 * w.max())[0]
        out[S] = (_colour_cos(st.QB, zs[1], zs[-2]), _colour_cos(st.QB, zs[1], zs[2]))
    assert out[1][0] > 0.98
    assert out[4][0] < 0.7
    assert out[4][1] > 0.99
