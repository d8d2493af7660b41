"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol that include/glasma.h declares, and rejects bad parameters before
touching the GPU."""
import os
import re

import numpy as np
import pytest

import glasma_inputs as gi
from paper_2009_02044_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2009_02044_gb300 import glasma as G
    return G.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "glasma.h")).read()
    return sorted(set(re.findall(r"GLASMA_API\s+[\w\s\*]+?\b(glasma_\w+)\s*\(",
                                 src)))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("glasma_init_mv", "glasma_step", "glasma_gauss_residual",
                 "glasma_tmunu", "glasma_free"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (glasma_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        getattr(lib, n)


def test_strerror(lib):
    from paper_2009_02044_gb300 import glasma as G
    assert G.glasma_strerror(0) == "ok"
    assert "invalid" in G.glasma_strerror(-1)
    assert G.glasma_strerror(-5).startswith("charge")


@pytest.mark.parametrize("bad", [
    dict(nc=4), dict(nz=1), dict(dt=2.0), dict(dt=0.3, a_z=0.9),
    dict(m_ir=0.0), dict(sigma_l=-1.0), dict(nz=20),
    dict(g2mu=-1.0), dict(z_offset=1.0),
])
def test_invalid_parameters_are_rejected_on_the_host(lib, bad):
    from paper_2009_02044_gb300 import glasma as G
    cfg = gi.small_config(2)
    cfg.update(bad)
    with pytest.raises(G.GlasmaError) as e:
        G.glasma_init_mv(cfg, torch_memory=False)
    assert e.value.code == "INVALID_ARG"


def test_batch_arguments_are_checked_on_the_host(lib):
    import ctypes as C
    from paper_2009_02044_gb300 import glasma as G
    out = C.c_void_p()
    assert lib.glasma_batch_create(None, 1, C.byref(out)) == -1
    arr = (C.c_void_p * 1)(None)
    assert lib.glasma_batch_create(arr, 0, C.byref(out)) == -1
    assert lib.glasma_batch_create(arr, 65, C.byref(out)) == -1
    assert lib.glasma_batch_create(arr, 1, C.byref(out)) == -1
    assert out.value is None
    assert lib.glasma_batch_step(None, 1) == -1
    assert lib.glasma_batch_tune(None, 1, None, None) == -1
    assert lib.glasma_batch_set_shape(None, 0, 64) == -1
    assert lib.glasma_batch_set_barrier(None, 1000, 0) == -1
    lib.glasma_batch_free(None)


def test_host_gaussian_fit_matches_oracle(lib):
    """glasma_fit_gaussian is host code: checked here against the oracle's
    numpy.polyfit fit on exact and on noisy profiles."""
    from oracle import rest_frame as RF
    from paper_2009_02044_gb300 import glasma as G
    eta = np.linspace(-3, 3, 97)
    f = 1.25 * np.exp(-(eta + 0.4) ** 2 / (2 * 0.8 ** 2))
    a, m, s = G.glasma_fit_gaussian(eta, f, 0.02)
    assert abs(a - 1.25) < 1e-11 and abs(m + 0.4) < 1e-11 and abs(s - 0.8) < 1e-11
    rng = np.random.default_rng(5)
    for k in range(20):
        fn = f * (1 + 0.05 * rng.standard_normal(eta.size)) + 0.01 * rng.random()
        frac = (0.05, 0.2, 0.5)[k % 3]
        got = np.array(G.glasma_fit_gaussian(eta, fn, frac))
        ref = np.array(RF.fit_gaussian(eta, fn, frac))
        assert np.allclose(got, ref, rtol=1e-10, atol=0), (got, ref)
    with pytest.raises(G.GlasmaError):
        G.glasma_fit_gaussian(eta, np.exp(eta ** 2 / 8), 0.0)
    with pytest.raises(G.GlasmaError):
        G.glasma_fit_gaussian(eta[:2], f[:2], 0.0)


def test_implicit_stopping_rule_on_measured_sequences(lib):
    """The improved scheme's stopping rule (host code) on the sequences of
    max |dE| measured on the SU(3) 2048 x 128^2 FP32 run, in units of
    u max|E| (u = 2^-24): it stops at the first sweep whose contraction
    bound is below the sweep's rounding noise, not on a first ratio that
    only reflects fast modes, and not while the change stagnates above the
    rounding floor."""
    from paper_2009_02044_gb300 import glasma as G
    u = 2.0 ** -24
    emax = 0.0123

    def stops(seq, **kw):
        d = np.asarray(seq, dtype=float) * u * emax
        return [G.glasma_implicit_converged(d[:k + 1], np.full(k + 1, emax), **kw)
                for k in range(len(seq))]

    # before the collision: the bound after the third sweep, 120 * 0.064 /
    # 0.936 = 8.2, is already below 16 (the next change measured 10)
    assert stops([1.28e6, 1.87e3, 120, 10]) == [False, False, True, True]
    # after it: the floor is higher and the ratios creep up near it
    assert stops([4.52e6, 2.74e5, 2.1e4, 1.82e3, 181, 41]) == [False] * 5 + [True]
    # changes within 64 ulps that no longer halve are the rounding noise
    assert stops([1e6, 1e5, 1e4, 2000, 300, 100, 60]) == [False] * 6 + [True]
    # a change that stops decreasing at the floor is convergence ...
    assert stops([1e6, 1e3, 300, 200, 210]) == [False] * 4 + [True]
    # ... above it, a failing iteration (contraction near or above 1)
    assert not any(stops([1e6, 6e5, 5e5, 5e5, 5.1e5]))
    # the tolerance alone, at any sweep
    assert stops([1.0, 0.5], tol=1.0 * u * emax * 2) == [True, True]
    # FP64 units: the same sequence in FP32 units is far above FP64's floor
    assert not any(stops([1.28e6, 1.87e3, 120, 10], precision="fp64"))
    assert lib.glasma_implicit_converged(None, None, 0, 0.0, 1, None) == -1


def test_static_residual_rejects_unaligned_links_on_the_host(lib):
    """The links are read with 16-byte vector loads: a U address that is
    not 16-byte aligned is refused before any GPU work (the addresses are
    never dereferenced on the host)."""
    from paper_2009_02044_gb300 import glasma as G
    for nc in (2, 3):
        with pytest.raises(G.GlasmaError) as e:
            G.glasma_gauss_residual_static(nc, "fp32", 8, 4, 4, 1.0, 1.0,
                                           0x10008, 0x20000)
        assert e.value.code == "INVALID_ARG"
        assert "16-byte" in str(e.value)


def test_kernel_choices_match_the_header():
    """The binding's kernel names map to the header's GLASMA_KERNEL_* values,
    and bench.py names the CUDA kernel the automatic choice launches."""
    import bench
    from paper_2009_02044_gb300 import glasma as G
    src = open(os.path.join(ROOT, "include", "glasma.h")).read()
    enum = dict((k.lower(), int(v)) for k, v in
                re.findall(r"GLASMA_KERNEL_(\w+)\s*=\s*(\d+)", src))
    assert enum == G.KERNELS
    assert bench.step_kernel_name(3, "fp32", "auto", 64) == "k_step_staged"
    assert bench.step_kernel_name(3, "fp32", "auto", 128) == "k_step_leapfrog"
    assert bench.step_kernel_name(2, "fp32", "auto", 64) == "k_step_leapfrog"
    assert bench.step_kernel_name(3, "fp64", "auto", 64) == "k_step_plaq"
