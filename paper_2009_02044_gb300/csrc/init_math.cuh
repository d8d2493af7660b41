// FP64 helpers of the MV initial state: the group logarithm used for
// E(t0 - dt/2) and the Philox4x32-10 counter-based generator.
#pragma once
#include <stdint.h>

#include "su_n.cuh"

namespace glasma {

// Cyclic complex Jacobi eigen-decomposition of a hermitian 3x3 matrix:
// on return A is diagonal (the eigenvalues) and A_in = V diag V^dagger.
// Each rotation maps the (p,q) pair by D = diag(1, conj(e)) (making the
// off-diagonal element real, e = A_pq / |A_pq|) followed by the real
// Jacobi rotation with t = tan(phi) solving t^2 + 2 zeta t - 1 = 0.
GL_HD void jacobi_herm3(cplx<double>* A, cplx<double>* V) {
  for (int k = 0; k < 9; ++k) V[k] = cplx<double>{k % 4 == 0 ? 1.0 : 0.0, 0.0};
  const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
  for (int sweep = 0; sweep < 32; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int k = 0; k < 3; ++k) {
      cplx<double> x = A[3 * P[k] + Q[k]];
      off += x.re * x.re + x.im * x.im;
      dia += A[4 * k].re * A[4 * k].re;
    }
    if (off == 0.0 || off < 1e-36 * dia) break;
    for (int k = 0; k < 3; ++k) {
      const int p = P[k], q = Q[k];
      cplx<double> apq = A[3 * p + q];
      double r = sqrt(apq.re * apq.re + apq.im * apq.im);
      if (r == 0.0) continue;
      cplx<double> e{apq.re / r, apq.im / r};
      double zeta = (A[4 * q].re - A[4 * p].re) / (2.0 * r);
      double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
      // G = identity except G_pp = c, G_pq = s, G_qp = -s conj(e), G_qq = c conj(e)
      cplx<double> G[9];
      for (int m = 0; m < 9; ++m) G[m] = cplx<double>{m % 4 == 0 ? 1.0 : 0.0, 0.0};
      G[3 * p + p] = cplx<double>{c, 0.0};
      G[3 * p + q] = cplx<double>{s, 0.0};
      G[3 * q + p] = (-s) * cj(e);
      G[3 * q + q] = c * cj(e);
      // A <- G^dag A G ; V <- V G
      cplx<double> T[9], Nw[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          cplx<double> acc{0, 0};
          for (int m = 0; m < 3; ++m) acc = acc + A[3 * i + m] * G[3 * m + j];
          T[3 * i + j] = acc;
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          cplx<double> acc{0, 0};
          for (int m = 0; m < 3; ++m) acc = acc + cj(G[3 * m + i]) * T[3 * m + j];
          Nw[3 * i + j] = acc;
        }
      for (int m = 0; m < 9; ++m) A[m] = Nw[m];
      A[3 * p + q] = cplx<double>{0, 0};
      A[3 * q + p] = cplx<double>{0, 0};
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          cplx<double> acc{0, 0};
          for (int m = 0; m < 3; ++m) acc = acc + V[3 * i + m] * G[3 * m + j];
          T[3 * i + j] = acc;
        }
      for (int m = 0; m < 9; ++m) V[m] = T[m];
    }
  }
}

// Algebra components h^a of the hermitian H with exp(i H) = W (W in SU(3)
// with eigen-phases in (-pi/2, pi/2)).  S = (W - W^+)/(2i) shares W's
// eigenvectors and has eigenvalues sin(theta); theta_k = atan2(v^+ S v,
// v^+ C v) with C = (W + W^+)/2.  Returns false if a phase is outside.
// Close to the identity (|S|_F < 1/4, so every |theta_k| < 0.253) H is
// the arcsine series of S instead, arcsin x = sum_k c_k x^(2k+1) with
// c_k / c_(k-1) = (2k-1)^2 / (2k (2k+1)), summed until a term is below
// 1e-18 |S|: the link changes of one time step at the initial state are
// of this kind, and the series costs a few matrix products where the
// Jacobi sweeps cost many.
GL_HD bool log_su3(const Group<3, double>::M& W, double* h) {
  cplx<double> S[9], C[9], Vm[9];
  double sn2 = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx<double> w = W.m[3 * i + j], wt = cj(W.m[3 * j + i]);
      cplx<double> d = w - wt, s = w + wt;
      S[3 * i + j] = cplx<double>{0.5 * d.im, -0.5 * d.re};  // d / (2i)
      C[3 * i + j] = 0.5 * s;
      sn2 += S[3 * i + j].re * S[3 * i + j].re + S[3 * i + j].im * S[3 * i + j].im;
    }
  if (sn2 < 0.0625) {
    typedef Group<3, double> G;
    G::M Sm, S2, T, H;
    for (int m = 0; m < 9; ++m) Sm.m[m] = S[m];
    S2 = G::mul(Sm, Sm);
    T = Sm;
    H = Sm;
    const double stop = 1e-36 * sn2;
    for (int k = 1; k < 40; ++k) {
      const double r = (double)((2 * k - 1) * (2 * k - 1)) / (double)(2 * k * (2 * k + 1));
      T = G::mul(T, S2);
      double t2 = 0.0;
      for (int m = 0; m < 9; ++m) {
        T.m[m] = r * T.m[m];
        H.m[m] = H.m[m] + T.m[m];
        t2 += T.m[m].re * T.m[m].re + T.m[m].im * T.m[m].im;
      }
      if (t2 <= stop) break;
    }
    G::from_herm(H, h);
    return true;
  }
  cplx<double> A[9];
  for (int m = 0; m < 9; ++m) A[m] = S[m];
  jacobi_herm3(A, Vm);
  double th[3];
  bool ok = true;
  for (int k = 0; k < 3; ++k) {
    cplx<double> sv{0, 0}, cv{0, 0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        cplx<double> vi = cj(Vm[3 * i + k]), vj = Vm[3 * j + k];
        sv = sv + vi * S[3 * i + j] * vj;
        cv = cv + vi * C[3 * i + j] * vj;
      }
    if (!(cv.re > 0.0)) ok = false;
    th[k] = atan2(sv.re, cv.re);
  }
  Group<3, double>::M H;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx<double> acc{0, 0};
      for (int k = 0; k < 3; ++k) acc = acc + th[k] * (Vm[3 * i + k] * cj(Vm[3 * j + k]));
      H.m[3 * i + j] = acc;
    }
  Group<3, double>::from_herm(H, h);
  return ok;
}

// SU(2): W = cos(phi) + i sin(phi) n.sigma, H = phi n.sigma, h^a = 2 phi n^a.
GL_HD bool log_su2(const Group<2, double>::M& W, double* h) {
  double v[3] = {W.b.im, W.b.re, W.a.im};  // sin(phi) n
  double sn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  if (sn == 0.0) {
    h[0] = h[1] = h[2] = 0.0;
    return W.a.re > 0.0;
  }
  double phi = atan2(sn, W.a.re);
  for (int a = 0; a < 3; ++a) h[a] = 2.0 * phi * v[a] / sn;
  return W.a.re > 0.0;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
GL_HD void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Uniform in (0, 1) from 27 + 26 high bits of two words, offset half an ulp.
GL_HD double u53(uint32_t hi, uint32_t lo) {
  return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

}  // namespace glasma
