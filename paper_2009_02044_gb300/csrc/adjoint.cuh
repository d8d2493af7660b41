// Reverse-mode building blocks of the SU(2) adjoint, FP64.
//
// An SU(2) link [[alpha, beta], [-beta*, alpha*]] is the quaternion
// q = (w, x, y, z) with alpha = w + i z, beta = y + i x, i.e.
// U = w 1 + i (x sigma1 + y sigma2 + z sigma3).  Products, daggers and the
// generator projection Im tr(t^a M) = (x, y, z) are polynomials in these
// four reals, so every step of the forward map is a smooth function of the
// link components; the adjoint differentiates those formulas (extended off
// the group by the same expressions).  Because the forward map keeps links
// on the group, the extension does not change the gradient with respect to
// the initial charges.
//
// Adjoint convention: for a real quantity v, vbar = dO/dv; a quaternion's
// adjoint is the 4-vector of partial derivatives of O with respect to its
// components.
#pragma once
#include "glasma_internal.cuh"

namespace glasma {
namespace adj {

struct Q4 {
  double w, x, y, z;
};

GL_HD Q4 q_zero() { return Q4{0.0, 0.0, 0.0, 0.0}; }
GL_HD Q4 q_one() { return Q4{1.0, 0.0, 0.0, 0.0}; }
GL_HD Q4 q_pure(const double* v) { return Q4{0.0, v[0], v[1], v[2]}; }
GL_HD Q4 q_dag(const Q4& a) { return Q4{a.w, -a.x, -a.y, -a.z}; }
GL_HD Q4 q_add(const Q4& a, const Q4& b) { return Q4{a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z}; }
GL_HD Q4 q_sub(const Q4& a, const Q4& b) { return Q4{a.w - b.w, a.x - b.x, a.y - b.y, a.z - b.z}; }
GL_HD Q4 q_scale(const Q4& a, double s) { return Q4{s * a.w, s * a.x, s * a.y, s * a.z}; }
GL_HD void q_acc(Q4& acc, const Q4& a) {
  acc.w += a.w;
  acc.x += a.x;
  acc.y += a.y;
  acc.z += a.z;
}

// (w + i a.s)(v + i b.s) = (w v - a.b) + i (w b + v a - a x b).s
GL_HD Q4 q_mul(const Q4& a, const Q4& b) {
  return Q4{a.w * b.w - (a.x * b.x + a.y * b.y + a.z * b.z),
            a.w * b.x + b.w * a.x - (a.y * b.z - a.z * b.y),
            a.w * b.y + b.w * a.y - (a.z * b.x - a.x * b.z),
            a.w * b.z + b.w * a.z - (a.x * b.y - a.y * b.x)};
}

// reverse of C = A B: abar += dC/dA^T cbar, bbar += dC/dB^T cbar
GL_HD void q_mul_rev(const Q4& a, const Q4& b, const Q4& cb, Q4& ab, Q4& bb) {
  ab.w += b.w * cb.w + b.x * cb.x + b.y * cb.y + b.z * cb.z;
  ab.x += -cb.w * b.x + b.w * cb.x - (b.y * cb.z - b.z * cb.y);
  ab.y += -cb.w * b.y + b.w * cb.y - (b.z * cb.x - b.x * cb.z);
  ab.z += -cb.w * b.z + b.w * cb.z - (b.x * cb.y - b.y * cb.x);
  bb.w += a.w * cb.w + a.x * cb.x + a.y * cb.y + a.z * cb.z;
  bb.x += -cb.w * a.x + a.w * cb.x + (a.y * cb.z - a.z * cb.y);
  bb.y += -cb.w * a.y + a.w * cb.y + (a.z * cb.x - a.x * cb.z);
  bb.z += -cb.w * a.z + a.w * cb.z + (a.x * cb.y - a.y * cb.x);
}

// reverse of D = A^dagger
GL_HD void q_dag_rev(const Q4& db, Q4& ab) {
  ab.w += db.w;
  ab.x -= db.x;
  ab.y -= db.y;
  ab.z -= db.z;
}

GL_HD Q4 q_from(const Group<2, double>::M& m) { return Q4{m.a.re, m.b.im, m.b.re, m.a.im}; }

// link d at site s of an FP64 SU(2) link array ((alpha, beta) as double2)
GL_HD Q4 q_load(const double2* U, int d, int64_t V, int64_t s) {
  const double2 a = U[link_index(2, d, 0, V, s)];
  const double2 b = U[link_index(2, d, 1, V, s)];
  return Q4{a.x, b.y, b.x, a.y};
}

// quaternion adjoints of links: [d][4][V]
GL_HD Q4 qb_load(const double* B, int d, int64_t V, int64_t s) {
  return Q4{B[(int64_t)(d * 4 + 0) * V + s], B[(int64_t)(d * 4 + 1) * V + s], B[(int64_t)(d * 4 + 2) * V + s],
            B[(int64_t)(d * 4 + 3) * V + s]};
}
GL_HD void qb_store(double* B, int d, int64_t V, int64_t s, const Q4& q) {
  B[(int64_t)(d * 4 + 0) * V + s] = q.w;
  B[(int64_t)(d * 4 + 1) * V + s] = q.x;
  B[(int64_t)(d * 4 + 2) * V + s] = q.y;
  B[(int64_t)(d * 4 + 3) * V + s] = q.z;
}

// X = exp(i th.sigma/2) = (cos(r/2), sin(r/2) th / r), r = |th|
GL_HD Q4 q_expi(const double* th) {
  const double r2 = th[0] * th[0] + th[1] * th[1] + th[2] * th[2];
  if (r2 == 0.0) return q_one();
  const double r = sqrt(r2);
  const double s = sin(0.5 * r), c = cos(0.5 * r);
  const double f = s / r;
  return Q4{c, f * th[0], f * th[1], f * th[2]};
}

// thbar += dX/dth^T Xbar for X = q_expi(th):
//   dX0/dth = -(sin(r/2) / (2 r)) th,
//   dXv/dth = g I + (g'(r) / r) th th^T,  g(r) = sin(r/2) / r;
// near r = 0 the Taylor series of the three coefficients is used.
GL_HD void q_expi_rev(const double* th, const Q4& xb, double* thb) {
  const double r2 = th[0] * th[0] + th[1] * th[1] + th[2] * th[2];
  double a0, g, gp;  // sin(r/2)/(2r), g, g'/r
  if (r2 < 1e-6) {
    a0 = 0.25 - r2 / 96.0;
    g = 0.5 - r2 / 48.0;
    gp = -1.0 / 24.0 + r2 / 960.0;
  } else {
    const double r = sqrt(r2);
    const double s = sin(0.5 * r), c = cos(0.5 * r);
    a0 = s / (2.0 * r);
    g = s / r;
    gp = (0.5 * r * c - s) / (r2 * r);
  }
  const double tv = th[0] * xb.x + th[1] * xb.y + th[2] * xb.z;
  thb[0] += -a0 * th[0] * xb.w + g * xb.x + gp * tv * th[0];
  thb[1] += -a0 * th[1] * xb.w + g * xb.y + gp * tv * th[1];
  thb[2] += -a0 * th[2] * xb.w + g * xb.z + gp * tv * th[2];
}

// Reverse of h = kappa(w0, r) wv with kappa = 2 atan2(r, w0) / r (the
// principal SU(2) logarithm, exp(i h.sigma/2) = W):
//   dh/dw0 = -2 wv / (w0^2 + r^2),
//   dh/dwv = kappa I + (dkappa/dr / r) wv wv^T,
//   dkappa/dr / r = 2 [w0 r / (w0^2 + r^2) - atan2(r, w0)] / r^3
// (series -4 / (3 w0^3) + O(r^2) near r = 0).
GL_HD void q_log_rev(const Q4& W, const double* hb, Q4& wb) {
  const double r2 = W.x * W.x + W.y * W.y + W.z * W.z;
  const double n2 = W.w * W.w + r2;
  double kap, kr;
  if (r2 < 1e-12 * W.w * W.w) {
    kap = 2.0 / W.w;
    kr = -4.0 / (3.0 * W.w * W.w * W.w);
  } else {
    const double r = sqrt(r2);
    const double at = atan2(r, W.w);
    kap = 2.0 * at / r;
    kr = 2.0 * (W.w * r / n2 - at) / (r2 * r);
  }
  const double wh = W.x * hb[0] + W.y * hb[1] + W.z * hb[2];
  wb.w += -2.0 * wh / n2;
  wb.x += kap * hb[0] + kr * wh * W.x;
  wb.y += kap * hb[1] + kr * wh * W.y;
  wb.z += kap * hb[2] + kr * wh * W.z;
}

// Reverse of q' = Vec(A (0, q) B) for fixed-shape transports
// (A, B) = (U^dagger, U) or (U, U^dagger): given qbar' returns qbar and
// accumulates the adjoint of U.
GL_HD void transport_rev(const Q4& U, bool dagger_first, const double* q, const double* qpb, double* qb, Q4& ub) {
  const Q4 A = dagger_first ? q_dag(U) : U;
  const Q4 B = dagger_first ? U : q_dag(U);
  const Q4 P = q_pure(q);
  const Q4 p1 = q_mul(A, P);
  const Q4 mb = Q4{0.0, qpb[0], qpb[1], qpb[2]};
  Q4 p1b = q_zero(), bb = q_zero(), ab = q_zero(), pb = q_zero();
  q_mul_rev(p1, B, mb, p1b, bb);
  q_mul_rev(A, P, p1b, ab, pb);
  if (dagger_first) {
    q_dag_rev(ab, ub);
    q_acc(ub, bb);
  } else {
    q_acc(ub, ab);
    q_dag_rev(bb, ub);
  }
  qb[0] = pb.x;
  qb[1] = pb.y;
  qb[2] = pb.z;
}

// Reverse of e . Vec(X1 X2 X3 X4) (coefficient folded into e): the
// adjoints of the four factors.
GL_HD void chain4_rev(const Q4& x1, const Q4& x2, const Q4& x3, const Q4& x4, const double* e, Q4& b1, Q4& b2,
                      Q4& b3, Q4& b4) {
  const Q4 p1 = q_mul(x1, x2);
  const Q4 p2 = q_mul(p1, x3);
  const Q4 mb = Q4{0.0, e[0], e[1], e[2]};
  Q4 p2b = q_zero(), p1b = q_zero();
  q_mul_rev(p2, x4, mb, p2b, b4);
  q_mul_rev(p1, x3, p2b, p1b, b3);
  q_mul_rev(x1, x2, p1b, b1, b2);
}

// ---------------------------------------------------------------------------
// Per-element bodies of the adjoint kernels (host and device, so that the
// same code can be run on the CPU).
// ---------------------------------------------------------------------------

// planes (i, j), i < j: (x, y), (x, z), (y, z)
__host__ __device__ __forceinline__ int plane_i(int pl) { return pl == 2 ? 1 : 0; }
__host__ __device__ __forceinline__ int plane_j(int pl) { return pl == 0 ? 1 : 2; }

// Per base site x and plane (i, j), i < j, with a = U_i(x), b = U_j(x+i),
// c = U_i(x+j), d = U_j(x), the plaquette's share of
//   phi = fs * sum_links Ebar . F   (F of Sec. 3 Eq. lattice_1)
//       + wsl(iz) * |a b - d c|_F^2 / (a_i a_j)^2   (its energy term)
// where the force terms are -w_j Ebar_i(x).Vec(a b c^+ d^+),
// -w_j Ebar_i(x+j).Vec(c b^+ a^+ d), -w_i Ebar_j(x).Vec(d c b^+ a^+) and
// -w_i Ebar_j(x+i).Vec(b c^+ d^+ a).  Writes d phi / d{a,b,c,d} to
// G[((plane*4 + role)*4 + component)*V + s] (zero for absent plaquettes).
GL_HD void plaq_rev_at(const double2* U, const double* Eb, double fs, const double* wsl, double* G, const Geom& g,
                       double wt, double wz, double ia2t, double ia2z, int64_t s) {
  {
    const SiteNbr n = site_nbr(g, s);
    for (int pl = 0; pl < 3; ++pl) {
      const int i = plane_i(pl), j = plane_j(pl);
      Q4 ab = q_zero(), bb = q_zero(), cb = q_zero(), db = q_zero();
      const bool exists = (j != 2) || (n.iz <= g.nz - 2);
      if (exists) {
        const Q4 a = q_load(U, i, g.V, s), b = q_load(U, j, g.V, n.p[i]);
        const Q4 c = q_load(U, i, g.V, n.p[j]), d = q_load(U, j, g.V, s);
        const double wi = i == 2 ? wz : wt, wj = j == 2 ? wz : wt;
        if (fs != 0.0) {
          double e[3];
          Q4 t1 = q_zero(), t2 = q_zero(), t3 = q_zero(), t4 = q_zero();
          // link a: a b c^+ d^+
          for (int k = 0; k < 3; ++k) e[k] = -fs * wj * Eb[(int64_t)(i * 3 + k) * g.V + s];
          t1 = t2 = t3 = t4 = q_zero();
          chain4_rev(a, b, q_dag(c), q_dag(d), e, t1, t2, t3, t4);
          q_acc(ab, t1);
          q_acc(bb, t2);
          q_dag_rev(t3, cb);
          q_dag_rev(t4, db);
          // link c: c b^+ a^+ d
          for (int k = 0; k < 3; ++k) e[k] = -fs * wj * Eb[(int64_t)(i * 3 + k) * g.V + n.p[j]];
          t1 = t2 = t3 = t4 = q_zero();
          chain4_rev(c, q_dag(b), q_dag(a), d, e, t1, t2, t3, t4);
          q_acc(cb, t1);
          q_dag_rev(t2, bb);
          q_dag_rev(t3, ab);
          q_acc(db, t4);
          // link d: d c b^+ a^+
          for (int k = 0; k < 3; ++k) e[k] = -fs * wi * Eb[(int64_t)(j * 3 + k) * g.V + s];
          t1 = t2 = t3 = t4 = q_zero();
          chain4_rev(d, c, q_dag(b), q_dag(a), e, t1, t2, t3, t4);
          q_acc(db, t1);
          q_acc(cb, t2);
          q_dag_rev(t3, bb);
          q_dag_rev(t4, ab);
          // link b: b c^+ d^+ a
          for (int k = 0; k < 3; ++k) e[k] = -fs * wi * Eb[(int64_t)(j * 3 + k) * g.V + n.p[i]];
          t1 = t2 = t3 = t4 = q_zero();
          chain4_rev(b, q_dag(c), q_dag(d), a, e, t1, t2, t3, t4);
          q_acc(bb, t1);
          q_dag_rev(t2, cb);
          q_dag_rev(t3, db);
          q_acc(ab, t4);
        }
        const double ws = wsl ? wsl[n.iz] : 0.0;
        if (ws != 0.0) {
          // |A - B|_F^2 = 2 |A - B|^2 (quaternion norm), A = a b, B = d c
          const double f = ws * (i == 2 || j == 2 ? ia2t * ia2z : ia2t * ia2t);
          const Q4 A = q_mul(a, b), B = q_mul(d, c);
          const Q4 D = q_scale(q_sub(A, B), 4.0 * f);
          q_mul_rev(a, b, D, ab, bb);
          q_mul_rev(d, c, q_scale(D, -1.0), db, cb);
        }
      }
      const Q4 r[4] = {ab, bb, cb, db};
      for (int k = 0; k < 4; ++k) {
        double* gp = G + (int64_t)((pl * 4 + k) * 4) * g.V + s;
        gp[0] = r[k].w;
        gp[g.V] = r[k].x;
        gp[2 * g.V] = r[k].y;
        gp[3 * g.V] = r[k].z;
      }
    }
  }
}

GL_HD void g_add(const double* G, int pl, int role, int64_t V, int64_t s, Q4& acc) {
  const double* gp = G + (int64_t)((pl * 4 + role) * 4) * V + s;
  acc.w += gp[0];
  acc.x += gp[V];
  acc.y += gp[2 * V];
  acc.z += gp[3 * V];
}

// Ubar_d(x) += the parts of the four plaquettes that hold link (x, d):
// as a (base x) and c (base x - j) when d is the plane's first direction,
// as d (base x) and b (base x - i) when it is the second.
GL_HD void gather_at(const double* G, double* Ub, const Geom& g, int64_t s) {
  {
    const SiteNbr n = site_nbr(g, s);
    for (int d = 0; d < 3; ++d) {
      if (d == 2 && n.iz == g.nz - 1) continue;
      Q4 acc = qb_load(Ub, d, g.V, s);
      for (int pl = 0; pl < 3; ++pl) {
        const int i = plane_i(pl), j = plane_j(pl);
        if (d == i) {
          g_add(G, pl, 0, g.V, s, acc);
          if (j != 2 || n.iz >= 1) g_add(G, pl, 2, g.V, n.m[j], acc);
        } else if (d == j) {
          g_add(G, pl, 3, g.V, s, acc);
          g_add(G, pl, 1, g.V, n.m[i], acc);
        }
      }
      qb_store(Ub, d, g.V, s, acc);
    }
  }
}

struct LinkRevArgs {
  const double2* U;   // U_n
  const double* En;   // E_{n+1/2}
  double* Ub;         // in: adjoint of U_{n+1}; out: of U_n (before the force part)
  double* Eb;         // adjoint of E_{n+1/2} (in and out)
  const double* QA;   // charges at step n (before the hop)
  const double* QB;
  double* QAb;        // in: adjoint after the hop; out: before
  double* QBb;
  int hop, zA0, WA, zB0, WB;
  Geom g;
  double dt, az2;
};

// Reverse of U_{n+1} = exp(i dt E_{n+1/2}) U_n per link and, on hop steps,
// of the charge transport and the current on the z links:
//   B: Q'_B = Vec(U^+ (0, Q_B) U) at the slot of x, E_z(x) -= a_z^2 Q_B;
//   A: Q'_A = Vec(U (0, Q_A) U^+) at the slot of x + z, E_z(x) += a_z^2 Q'_A.
GL_HD void link_rev_at(const LinkRevArgs& a, int64_t idx) {
  const Geom& g = a.g;
  do {
    const int d = (int)(idx / g.V);
    const int64_t s = idx - (int64_t)d * g.V;
    const int iz = (int)(s / g.nxy);
    if (d == 2 && iz == g.nz - 1) {  // absent link: unchanged, no field
      for (int k = 0; k < 3; ++k) a.Eb[(int64_t)(6 + k) * g.V + s] = 0.0;
      break;
    }
    const Q4 u = q_load(a.U, d, g.V, s);
    double th[3], thb[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) th[k] = a.dt * a.En[(int64_t)(d * 3 + k) * g.V + s];
    const Q4 X = q_expi(th);
    const Q4 ub1 = qb_load(a.Ub, d, g.V, s);
    Q4 xb = q_zero(), ub = q_zero();
    q_mul_rev(X, u, ub1, xb, ub);
    q_expi_rev(th, xb, thb);
    double eb[3];
    for (int k = 0; k < 3; ++k) {
      eb[k] = a.Eb[(int64_t)(d * 3 + k) * g.V + s] + a.dt * thb[k];
      a.Eb[(int64_t)(d * 3 + k) * g.V + s] = eb[k];
    }
    if (d == 2 && a.hop) {
      const int64_t t = s - (int64_t)iz * g.nxy;
      const int kb = iz - a.zB0;
      if (kb >= 0 && kb < a.WB) {
        double q[3], qpb[3], qb[3];
        for (int k = 0; k < 3; ++k) {
          q[k] = a.QB[((int64_t)k * a.WB + kb) * g.nxy + t];
          qpb[k] = a.QBb[((int64_t)k * a.WB + kb) * g.nxy + t];
        }
        transport_rev(u, true, q, qpb, qb, ub);
        for (int k = 0; k < 3; ++k) a.QBb[((int64_t)k * a.WB + kb) * g.nxy + t] = qb[k] - a.az2 * eb[k];
      }
      const int ka = iz + 1 - a.zA0;
      if (ka >= 0 && ka < a.WA) {
        double q[3], qpb[3], qb[3];
        for (int k = 0; k < 3; ++k) {
          q[k] = a.QA[((int64_t)k * a.WA + ka) * g.nxy + t];
          qpb[k] = a.QAb[((int64_t)k * a.WA + ka) * g.nxy + t] + a.az2 * eb[k];
        }
        transport_rev(u, false, q, qpb, qb, ub);
        for (int k = 0; k < 3; ++k) a.QAb[((int64_t)k * a.WA + ka) * g.nxy + t] = qb[k];
      }
    }
    qb_store(a.Ub, d, g.V, s, ub);
  } while (false);
}

// The current part of the observable's own E update (no transported-charge
// adjoint): E'_z(x) += a_z^2 (Q'_A - Q_B) with adjoint Ebp_z(x).
GL_HD void hop_current_rev_at(const double2* U, const double* Ebp, const double* QA, const double* QB, double* QAb,
                              double* QBb, double* Ub, int zA0, int WA, int zB0, int WB, const Geom& g, double az2,
                              int64_t s) {
  {
    const int iz = (int)(s / g.nxy);
    const int64_t t = s - (int64_t)iz * g.nxy;
    double eb[3];
    for (int k = 0; k < 3; ++k) eb[k] = Ebp[(int64_t)(6 + k) * g.V + s];
    const int kb = iz - zB0;
    if (kb >= 0 && kb < WB)
      for (int k = 0; k < 3; ++k) QBb[((int64_t)k * WB + kb) * g.nxy + t] -= az2 * eb[k];
    const int ka = iz + 1 - zA0;
    if (ka >= 0 && ka < WA) {
      const Q4 u = q_load(U, 2, g.V, s);
      double q[3], qpb[3], qb[3];
      for (int k = 0; k < 3; ++k) {
        q[k] = QA[((int64_t)k * WA + ka) * g.nxy + t];
        qpb[k] = az2 * eb[k];
      }
      Q4 ub = qb_load(Ub, 2, g.V, s);
      transport_rev(u, false, q, qpb, qb, ub);
      qb_store(Ub, 2, g.V, s, ub);
      for (int k = 0; k < 3; ++k) QAb[((int64_t)k * WA + ka) * g.nxy + t] += qb[k];
    }
  }
}

// Direct energy terms of the observable: eps holds (1/4) sum_i (E_i^2 +
// E'_i^2) / a_i^2 per site, E' = E(n+1/2) from the non-committing update:
//   Ebp = w(iz) E' / (2 a_i^2) (adjoint of E'), Eb = w(iz) E / (2 a_i^2) + Ebp
// with w(iz) the slice weight a_z / (nx ny) inside the window.
GL_HD void obs_rev_at(const double* E, const double* Ep, const double* wsl, double* Eb, double* Ebp, const Geom& g,
                      double ia2t, double ia2z, int64_t idx) {
  {
    const int comp = (int)(idx / g.V);
    const int64_t s = idx - (int64_t)comp * g.V;
    const int d = comp / 3;
    const double w = wsl[s / g.nxy] * 0.5 * (d == 2 ? ia2z : ia2t);
    const double bp = w * Ep[idx];
    Ebp[idx] = bp;
    Eb[idx] = w * E[idx] + bp;
  }
}

// Adjoint of the charge density rho(x) = sum_i [E_i(x) - T_i(x)] / a_i^2,
// T_i(x) = Vec(U_i^+(x-i) (0, E_i(x-i)) U_i(x-i)), through the split
// Q_A = rho (z > z_c), Q_B = rho (z < z_c) read from the windows; only the
// transverse links and fields depend on the charges (U_z = 1, E_z = 0).
GL_HD void rho_bar(const double* QAb, const double* QBb, int zA0, int WA, int zB0, int WB,
                                        const Geom& g, int iz, int64_t t, double* out) {
  for (int k = 0; k < 3; ++k) out[k] = 0.0;
  const int ka = iz - zA0, kb = iz - zB0;
  if (ka >= 0 && ka < WA)
    for (int k = 0; k < 3; ++k) out[k] += QAb[((int64_t)k * WA + ka) * g.nxy + t];
  if (kb >= 0 && kb < WB)
    for (int k = 0; k < 3; ++k) out[k] += QBb[((int64_t)k * WB + kb) * g.nxy + t];
}

GL_HD void div_rev_at(const double2* U, const double* E, const double* QAb, const double* QBb, int zA0, int WA,
                      int zB0, int WB, double* Eb, double* Ub, const Geom& g, double ia2t, int64_t s) {
  {
    const SiteNbr n = site_nbr(g, s);
    const int64_t t = s - (int64_t)n.iz * g.nxy;
    double r0[3];
    rho_bar(QAb, QBb, zA0, WA, zB0, WB, g, n.iz, t, r0);
    for (int d = 0; d < 2; ++d) {
      const int64_t sp = n.p[d];
      double r1[3], q[3], qpb[3], qb[3];
      rho_bar(QAb, QBb, zA0, WA, zB0, WB, g, n.iz, sp - (int64_t)n.iz * g.nxy, r1);
      for (int k = 0; k < 3; ++k) {
        q[k] = E[(int64_t)(d * 3 + k) * g.V + s];
        qpb[k] = -ia2t * r1[k];
      }
      Q4 ub = qb_load(Ub, d, g.V, s);
      transport_rev(q_load(U, d, g.V, s), true, q, qpb, qb, ub);
      qb_store(Ub, d, g.V, s, ub);
      for (int k = 0; k < 3; ++k) Eb[(int64_t)(d * 3 + k) * g.V + s] += ia2t * r0[k] + qb[k];
    }
  }
}

// Links of the initial state rebuilt exactly as the forward builds them.
GL_HD Group<2, double>::M vdag_of(const double* phi, int N, int64_t nxy, int64_t t, double lam) {
  typedef Group<2, double> G;
  if (lam == 0.0) return G::ident();
  double v[3];
  for (int a = 0; a < 3; ++a) v[a] = phi[((int64_t)N * 3 + a) * nxy + t];
  return G::expi(v, lam);
}

GL_HD Group<2, double>::M link_of(const double* phi, double la, double lb, int64_t nxy,
                                                        int64_t t0, int64_t t1) {
  typedef Group<2, double> G;
  const G::M ua = G::d_mul(vdag_of(phi, 0, nxy, t0, la), vdag_of(phi, 0, nxy, t1, la));
  const G::M ub = G::d_mul(vdag_of(phi, 1, nxy, t0, lb), vdag_of(phi, 1, nxy, t1, lb));
  return G::mul(ua, ub);
}

// E_i = log(U0 Um^+) / dt on transverse links (zero where the two links are
// bitwise equal, as in the forward): Ub (adjoint of U0) += ..., Umb = ...
GL_HD void log_rev_at(const double* phi, const double* lam, const double* Eb, double* Ub, double* Umb, const Geom& g,
                      double dt, int64_t idx) {
  typedef Group<2, double> G;
  {
    const int d = (int)(idx / g.V);
    const int64_t s = idx - (int64_t)d * g.V;
    const SiteNbr n = site_nbr(g, s);
    const int64_t t0 = s % g.nxy, t1 = n.p[d] % g.nxy;
    const G::M u0 = link_of(phi, lam[0 * g.nz + n.iz], lam[1 * g.nz + n.iz], g.nxy, t0, t1);
    const G::M um = link_of(phi, lam[2 * g.nz + n.iz], lam[3 * g.nz + n.iz], g.nxy, t0, t1);
    Q4 mb = q_zero();
    const bool same = u0.a.re == um.a.re && u0.a.im == um.a.im && u0.b.re == um.b.re && u0.b.im == um.b.im;
    if (!same) {
      const Q4 a = q_from(u0), b = q_dag(q_from(um));
      const Q4 W = q_mul(a, b);
      double hb[3];
      for (int k = 0; k < 3; ++k) hb[k] = Eb[(int64_t)(d * 3 + k) * g.V + s] / dt;
      Q4 wb = q_zero(), a_b = qb_load(Ub, d, g.V, s), bdb = q_zero();
      q_log_rev(W, hb, wb);
      q_mul_rev(a, b, wb, a_b, bdb);
      qb_store(Ub, d, g.V, s, a_b);
      q_dag_rev(bdb, mb);
    }
    qb_store(Umb, d, g.V, s, mb);
  }
}

// For site x and nucleus N: the adjoint of V_N^+(x) at both times from the
// links (x, i) (as V_N(x) = (V_N^+(x))^+) and (x - i, i) (as V_N^+(x)),
// i = x, y, then through V^+ = exp(i Lambda phi.sigma/2):
//   phib_z[(N*3 + a)*V + s] = sum_t Lambda_N(z, t) thbar^a.
GL_HD void links_rev_at(const double* phi, const double* lam, const double* Ub, const double* Umb, double* phib_z,
                        const Geom& g, int64_t s) {
  {
    const SiteNbr n = site_nbr(g, s);
    const int64_t tx = s % g.nxy;
    double acc[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (int tm = 0; tm < 2; ++tm) {
      const double la = lam[(tm * 2 + 0) * g.nz + n.iz], lb = lam[(tm * 2 + 1) * g.nz + n.iz];
      const double* B = tm == 0 ? Ub : Umb;
      const double lamN[2] = {la, lb};
      Q4 vb[2] = {q_zero(), q_zero()};
      for (int i = 0; i < 2; ++i) {
        for (int side = 0; side < 2; ++side) {  // 0: link (x, i); 1: link (x - i, i)
          const int64_t y = side == 0 ? s : n.m[i];
          const int64_t ty = y % g.nxy;
          const SiteNbr ny_ = site_nbr(g, y);
          const int64_t tyi = ny_.p[i] % g.nxy;
          Q4 v0[2], v1[2];
          for (int N = 0; N < 2; ++N) {
            v0[N] = q_from(vdag_of(phi, N, g.nxy, ty, lamN[N]));
            v1[N] = q_from(vdag_of(phi, N, g.nxy, tyi, lamN[N]));
          }
          const Q4 ua = q_mul(q_dag(v0[0]), v1[0]);
          const Q4 ubq = q_mul(q_dag(v0[1]), v1[1]);
          const Q4 lb_ = qb_load(B, i, g.V, y);
          Q4 uab = q_zero(), ubb = q_zero();
          q_mul_rev(ua, ubq, lb_, uab, ubb);
          const Q4 fb[2] = {uab, ubb};
          for (int N = 0; N < 2; ++N) {
            Q4 v0db = q_zero(), v1b = q_zero();
            q_mul_rev(q_dag(v0[N]), v1[N], fb[N], v0db, v1b);
            if (side == 0)
              q_dag_rev(v0db, vb[N]);
            else
              q_acc(vb[N], v1b);
          }
        }
      }
      for (int N = 0; N < 2; ++N) {
        if (lamN[N] == 0.0) continue;
        double th[3], thb[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a) th[a] = lamN[N] * phi[((int64_t)N * 3 + a) * g.nxy + tx];
        q_expi_rev(th, vb[N], thb);
        for (int a = 0; a < 3; ++a) acc[N][a] += lamN[N] * thb[a];
      }
    }
    for (int N = 0; N < 2; ++N)
      for (int a = 0; a < 3; ++a) phib_z[(int64_t)(N * 3 + a) * g.V + s] = acc[N][a];
  }
}

GL_HD void zsum_at(const double* phib_z, double* phib, const Geom& g, int64_t idx) {
  {
    const int64_t f = idx / g.nxy, t = idx - f * g.nxy;
    double acc = 0.0;
    for (int iz = 0; iz < g.nz; ++iz) acc += phib_z[f * g.V + (int64_t)iz * g.nxy + t];
    phib[idx] = acc;
  }
}


}  // namespace adj
}  // namespace glasma
