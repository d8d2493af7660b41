"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

This module holds no arithmetic of the Glasma method itself.  It provides

* the named workloads (lattice sizes, spacings, MV parameters) of the
  synthetic MV-model collisions that stand in for the paper's simulations
  (Ipp & Mueller, Sec. 4: SU(2) collisions with a Gaussian longitudinal
  profile and transverse-constant mu^2);
* the MV colour-charge draw rho_N^a(x_T): i.i.d. Gaussian per
  (nucleus, colour, x, y) with standard deviation g^2 mu a_T (the MV
  functional W[rho] of Sec. 2 on a transverse lattice), generated from a
  Philox4x32-10 counter-based stream (Salmon et al., SC'11) and a
  Box-Muller transform; the CUDA library implements the same generator on
  the device for callers that pass only a seed;
* random SU(N) matrices and small random fields used as test inputs
  (Haar measure via QR of a complex Gaussian matrix).

Array conventions used everywhere in this repository:
  nucleus index 0 = A (moves towards -z), 1 = B (moves towards +z);
  transverse arrays are [ny][nx] with x fastest; 3-D arrays [nz][ny][nx].
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Named workloads.  Units: a_T = 1, g = 1.
# ---------------------------------------------------------------------------

_BASE = dict(a_t=1.0, uv_cutoff=0.0, z_offset=0.0, precision="fp64",
             scheme="leapfrog", implicit_max_iter=50, implicit_tol=1e-14)


def _cfg(**kw):
    d = dict(_BASE)
    d.update(kw)
    return d


CONFIGS = {
    # SU(2) FP64 collision 128 x 16^2, 100 steps (parity workload)
    "su2_128x16x16": _cfg(nc=2, nz=128, nx=16, ny=16, a_z=1.0, dt=0.5,
                          sigma_l=4.0, g2mu=0.1, m_ir=0.2, seed=1001,
                          steps=100),
    # SU(3) single event 512 x 64^2, 400 steps (throughput workload)
    "su3_512x64x64": _cfg(nc=3, nz=512, nx=64, ny=64, a_z=1.0, dt=0.5,
                          sigma_l=8.0, g2mu=0.1, m_ir=0.2, seed=1002,
                          steps=400),
    # SU(2) 256 x 32^2, 200 steps (differentiation workload)
    "su2_256x32x32": _cfg(nc=2, nz=256, nx=32, ny=32, a_z=1.0, dt=0.5,
                          sigma_l=4.0, g2mu=0.1, m_ir=0.2, seed=1004,
                          steps=200, precision="fp32"),
    # SU(2) 1024 x 128^2, FP32: the leapfrog kernel where its arithmetic
    # per byte is low (168 B per site)
    "su2_1024x128x128": _cfg(nc=2, nz=1024, nx=128, ny=128, a_z=1.0, dt=0.5,
                             sigma_l=8.0, g2mu=0.1, m_ir=0.2, seed=1006,
                             steps=200, precision="fp32"),
    # SU(3) 2048 x 128^2 thin nuclei, improved scheme, a_z = dt = 0.25
    "su3_2048x128x128_improved": _cfg(nc=3, nz=2048, nx=128, ny=128,
                                      a_z=0.25, dt=0.25, sigma_l=2.0,
                                      g2mu=0.05, m_ir=0.1, seed=1005,
                                      steps=1000, precision="fp32",
                                      scheme="implicit"),
}


def ensemble_configs():
    """24 independent MV events of uneven transverse size (8 each at 32^2,
    48^2, 64^2), N_L = 256, dt = a/2, sigma_L = 6a, g^2 mu a = 0.1."""
    out = []
    for e in range(24):
        nt = (32, 48, 64)[e // 8]
        out.append(_cfg(nc=3, nz=256, nx=nt, ny=nt, a_z=1.0, dt=0.5,
                        sigma_l=6.0, g2mu=0.1, m_ir=0.2, seed=3000 + e,
                        steps=200, precision="fp32"))
    return out


def thin_ensemble_configs(m_ir, events=8, nc=2, nt=64, nz=768, seed0=5000):
    """Independent MV events in the regime of the paper's rapidity-profile
    study (Sec. 4: SU(2), nuclei thin against the transverse scales, the IR
    regulator well below g^2 mu): a_T = 1, a_z = a_T/8, dt = a_z/2,
    sigma_L = a_T (8 cells), g^2 mu a_T = 0.4, transverse nt^2, N_L = nz
    (96 a_T, so both nuclei stay inside the box until t = 40 a_T after
    the collision)."""
    return [_cfg(nc=nc, nz=nz, nx=nt, ny=nt, a_z=0.125, dt=0.0625,
                 sigma_l=1.0, g2mu=0.4, m_ir=float(m_ir), seed=seed0 + e,
                 steps=704, precision="fp32") for e in range(events)]


def small_config(nc, nz=48, nx=12, ny=10, sigma_l=2.0, steps=40, seed=7,
                 **kw):
    """A small collision whose nuclei meet within `steps` steps: used for
    parity at sizes the oracle finishes in seconds (ragged against any
    power-of-two tile)."""
    return _cfg(nc=nc, nz=nz, nx=nx, ny=ny, a_z=kw.pop("a_z", 1.0),
                dt=kw.pop("dt", 0.5), sigma_l=sigma_l,
                g2mu=kw.pop("g2mu", 0.1), m_ir=kw.pop("m_ir", 0.2),
                seed=seed, steps=steps, **kw)


# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
# easy as 1, 2, 3", SC'11).  Vectorised over numpy uint32 arrays.
# ---------------------------------------------------------------------------

_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on counter (c0..c3) with key (k0, k1); all uint32.

    Each round multiplies c0 and c2 by the two Philox constants (64-bit
    products split into hi/lo words), mixes the high words with c1, c3 and
    the key, and the key is bumped by the Weyl constants between rounds."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = (k0 + _PHILOX_W0).astype(np.uint32)
                k1 = (k1 + _PHILOX_W1).astype(np.uint32)
            p0 = c0.astype(np.uint64) * _PHILOX_M0
            p1 = c2.astype(np.uint64) * _PHILOX_M1
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _u53(hi, lo):
    """Uniform double in the open interval (0, 1) from two 32-bit words:
    27 high bits of `hi` and 26 high bits of `lo`, offset by half an ulp."""
    a = (hi >> np.uint32(5)).astype(np.float64)
    b = (lo >> np.uint32(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) * (1.0 / 9007199254740992.0)


def mv_rho(seed, nc, nx, ny, g2mu, sheets=1):
    """MV colour charges rho[N][a][y][x] (N = 0: nucleus A, 1: nucleus B);
    with sheets = S > 1, rho[s][N][a][y][x] for S independent longitudinal
    colour sheets, each with standard deviation g2mu / sqrt(S) so that the
    charge summed over the sheets keeps the single-sheet variance.

    Counter = (x, y, a, N + 2 s), key = (seed low word, seed high word); the
    four output words give two 53-bit uniforms u1, u2 and one Box-Muller
    normal sqrt(-2 ln u1) cos(2 pi u2), scaled by the standard deviation."""
    na = nc * nc - 1
    if sheets > 1:
        S, N, A, Y, X = np.meshgrid(np.arange(sheets), np.arange(2),
                                    np.arange(na), np.arange(ny),
                                    np.arange(nx), indexing="ij")
        N = N + 2 * S
        g2mu = g2mu / np.sqrt(sheets)
    else:
        N, A, Y, X = np.meshgrid(np.arange(2), np.arange(na), np.arange(ny),
                                 np.arange(nx), indexing="ij")
    seed = int(seed)
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32((seed >> 32) & 0xFFFFFFFF)
    w0, w1, w2, w3 = philox4x32_10(X.astype(np.uint32), Y.astype(np.uint32),
                                   A.astype(np.uint32), N.astype(np.uint32),
                                   k0, k1)
    u1 = _u53(w0, w1)
    u2 = _u53(w2, w3)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return (g2mu * z).astype(np.float64)


# ---------------------------------------------------------------------------
# Random group elements and fields for tests.
# ---------------------------------------------------------------------------

def haar_su(nc, shape, rng):
    """Haar-random SU(nc) matrices of the given batch shape (QR of a complex
    Gaussian matrix with the phases of R's diagonal removed, then the
    determinant divided out)."""
    shape = tuple(shape)
    z = (rng.standard_normal(shape + (nc, nc))
         + 1j * rng.standard_normal(shape + (nc, nc))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / nc))[..., None, None]
    return q


def near_identity_su(nc, shape, rng, amp):
    """SU(nc) matrices close to the identity: the unitary factor of
    1 + amp * (complex Gaussian), with the determinant divided out."""
    shape = tuple(shape)
    z = np.eye(nc) + amp * (rng.standard_normal(shape + (nc, nc))
                            + 1j * rng.standard_normal(shape + (nc, nc)))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / nc))[..., None, None]
    return q
