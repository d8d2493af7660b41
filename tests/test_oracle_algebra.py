"""Pins of the oracle's SU(N) algebra and of the shared input generator
against textbook tables, library routines and published test vectors."""
import os

import numpy as np
import pytest
import scipy.linalg

import glasma_inputs as gi
from oracle import glasma_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _structure_constants(nc):
    t = O.generators(nc)
    na = nc * nc - 1
    f = np.zeros((na, na, na))
    for a in range(na):
        for b in range(na):
            comm = t[a] @ t[b] - t[b] @ t[a]
            # [t^a, t^b] = i f^{abc} t^c  ->  f^{abc} = -2i tr([t^a,t^b] t^c)
            for c in range(na):
                f[a, b, c] = (-2j * np.trace(comm @ t[c])).real
    return f


@pytest.mark.parametrize("nc", [2, 3])
def test_generator_normalisation(nc):
    t = O.generators(nc)
    na = nc * nc - 1
    g = np.einsum("aij,bji->ab", t, t)
    assert np.allclose(g, 0.5 * np.eye(na), atol=1e-15)
    assert np.allclose(np.einsum("aii->a", t), 0, atol=1e-15)
    assert np.allclose(t, np.conj(np.swapaxes(t, -1, -2)), atol=0)


def test_su2_structure_constants_levi_civita():
    f = _structure_constants(2)
    eps = np.zeros((3, 3, 3))
    for (a, b, c), s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1,
                         (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
        eps[a, b, c] = s
    assert np.allclose(f, eps, atol=1e-15)


def test_su3_structure_constants_golden():
    f = _structure_constants(3)
    ref = np.zeros((8, 8, 8))
    for line in open(os.path.join(GOLDEN, "su3_structure_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a, b, c, v = line.split()
        a, b, c, v = int(a) - 1, int(b) - 1, int(c) - 1, float(v)
        for (i, j, k), s in {(a, b, c): 1, (b, c, a): 1, (c, a, b): 1,
                             (b, a, c): -1, (a, c, b): -1,
                             (c, b, a): -1}.items():
            ref[i, j, k] = s * v
    assert np.allclose(f, ref, atol=1e-15)


@pytest.mark.parametrize("nc", [2, 3])
def test_expi_matches_scipy_expm(nc):
    rng = np.random.default_rng(1)
    v = rng.standard_normal((20, nc * nc - 1)) * 2.0
    for c in (0.5, 1e-3, 3.0):
        got = O.expi_alg(v, c, nc)
        for k in range(v.shape[0]):
            ref = scipy.linalg.expm(1j * c * O.alg_to_mat(v[k], nc))
            assert np.max(np.abs(got[k] - ref)) < 1e-13


def test_su2_exp_closed_form():
    rng = np.random.default_rng(2)
    v = rng.standard_normal((50, 3))
    got = O.expi_alg(v, 0.7, 2)
    th = 0.7 * np.linalg.norm(v, axis=1) / 2
    n = v / np.linalg.norm(v, axis=1)[:, None]
    sig = 2 * O.generators(2)
    ref = (np.cos(th)[:, None, None] * np.eye(2)
           + 1j * np.sin(th)[:, None, None]
           * np.einsum("ka,aij->kij", n, sig))
    assert np.max(np.abs(got - ref)) < 1e-14


@pytest.mark.parametrize("nc", [2, 3])
def test_logu_inverts_exp(nc):
    rng = np.random.default_rng(3)
    v = rng.standard_normal((40, nc * nc - 1)) * 0.3
    w = O.expi_alg(v, 1.0, nc)
    h = O.logu(w)
    assert np.max(np.abs(O.mat_to_alg(h, nc) - v)) < 1e-13
    # exp(i log W) = W for a random near-identity unitary
    w2 = gi.near_identity_su(nc, (30,), rng, 0.2)
    h2 = O.logu(w2)
    back = np.stack([scipy.linalg.expm(1j * x) for x in h2])
    assert np.max(np.abs(back - w2)) < 1e-13


def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = gi.philox4x32_10(*w[:6])
        assert [int(x) for x in out] == w[6:]


def test_mv_rho_statistics():
    rho = gi.mv_rho(1002, 3, 64, 64, 0.1)
    assert rho.shape == (2, 8, 64, 64)
    assert abs(rho.mean()) < 0.1 * 0.01
    assert abs(rho.std() / 0.1 - 1.0) < 0.01
    # deterministic in the seed, different between seeds
    assert np.array_equal(rho, gi.mv_rho(1002, 3, 64, 64, 0.1))
    assert not np.array_equal(rho, gi.mv_rho(1003, 3, 64, 64, 0.1))


def test_haar_su_is_special_unitary():
    rng = np.random.default_rng(4)
    for nc in (2, 3):
        u = gi.haar_su(nc, (10,), rng)
        assert np.allclose(u @ np.conj(np.swapaxes(u, -1, -2)), np.eye(nc),
                           atol=1e-14)
        assert np.allclose(np.linalg.det(u), 1.0, atol=1e-14)
