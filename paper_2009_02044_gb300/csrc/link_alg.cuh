// Arithmetic on stored links.
//
// FP64 links are stored and multiplied as full matrices (Group<NC, double>).
// FP32 links are stored and multiplied as their deviation from the identity,
// d = U - 1.  Links near the identity (weak fields, vacuum, and the slowly
// varying pure-gauge links of the nuclei, |U - 1| <~ 0.1) then carry
// rounding errors of the size u |d| instead of u, in storage and in every
// product, so the force -- a small anti-hermitian difference of O(1)
// products -- keeps about log10(1/|d|) more digits in FP32.
//
// Interface shared by both representations (M = a stored-form link):
//   ident, mul, mul_d (x y^+), d_mul (x^+ y)       products of links
//   Sum, zero_sum, sum_add                          weighted staple sums
//   proj_mul(u, S)                                  Im tr t^a (U S)
//   proj_prod(x, y), proj_prod_d(x, y)              Im tr t^a (x y), (x y^+)
//                                                   of two stored-form links
//   expi(v, c)                                      exp(i c v^a t^a)
//   reunit, adj (U q U^+), adj_dag (U^+ q U)
//
// The FP32 forms are templates over the lane type T: float (one site per
// thread) or f2 (pair.cuh: two sites per thread in the lanes of the packed
// f32x2 instructions).  With T = float every expression is the scalar one.
#pragma once
#include "su_n.cuh"
#ifdef __CUDACC__
#include "pair.cuh"
#endif

namespace glasma {
// fma for the scalar lane types, visible next to the f2 overload of the
// same name (which would otherwise hide the global ones in this namespace)
GL_HD float fma(float a, float b, float c) { return fmaf(a, b, c); }
GL_HD double fma(double a, double b, double c) { return ::fma(a, b, c); }
// lane helpers for T = float (pair.cuh has the f2 forms)
GL_HD bool all_zero_s(float a) { return a == 0.f; }
GL_HD bool any_gt_s(float a, float b) { return a > b; }
GL_HD bool all_abs_lt_s(float a, float b) { return fabsf(a) < b; }
GL_HD float lane_abs_s(float a) { return fabsf(a); }
GL_HD float lane_div_s(float a, float b) { return a / b; }
// a / b, and 0 in a lane where b = 0 (a scalar caller has returned before)
GL_HD float lane_div0_s(float a, float b) { return a / b; }
#ifdef __CUDACC__
__device__ __forceinline__ bool all_zero_s(f2 a) { return all_zero(a); }
__device__ __forceinline__ bool any_gt_s(f2 a, float b) { return any_gt(a, b); }
__device__ __forceinline__ bool all_abs_lt_s(f2 a, float b) { return all_abs_lt(a, b); }
__device__ __forceinline__ f2 lane_abs_s(f2 a) { return lane_abs(a); }
__device__ __forceinline__ f2 lane_div_s(f2 a, f2 b) { return lane_div(a, b); }
__device__ __forceinline__ f2 lane_div0_s(f2 a, f2 b) {
  return f2(b.v.x != 0.f ? a.v.x / b.v.x : 0.f, b.v.y != 0.f ? a.v.y / b.v.y : 0.f);
}
__device__ __forceinline__ f2 gl_sqrt(f2 x) { return lane_sqrt(x); }
__device__ __forceinline__ void gl_sincos(f2 x, f2* s, f2* c) { *s = lane_sincos_s(x, c); }
#endif
}  // namespace glasma

namespace glasma {

template <int NC, typename R> struct LinkAlg;

// ---------------------------------------------------------------------------
// Full matrices (FP64 state).
// ---------------------------------------------------------------------------
template <int NC>
struct LinkAlg<NC, double> : Group<NC, double> {
  typedef Group<NC, double> G;
  typedef typename G::M M;
  static constexpr bool kDelta = false;
  GL_HD static M expi_series(const double* v, double c) { return G::expi(v, c); }
  typedef M Sum;
  GL_HD static M full(const M& u) { return u; }
  GL_HD static Sum zero_sum() { return G::zero(); }
  GL_HD static void sum_add(Sum& s, double w, const M& t) { G::scale_add(s, w, t); }
  GL_HD static void proj_mul_sum(const M& u, const Sum& s, double* out) { G::proj_mul(u, s, out); }
  GL_HD static void proj_prod(const M& x, const M& y, double* out) { G::proj_mul(x, y, out); }
  GL_HD static void proj_prod_d(const M& x, const M& y, double* out) { G::proj_mul(x, G::dag(y), out); }
};

// ---------------------------------------------------------------------------
// SU(3), FP32, deviation form: M holds d = U - 1 (row major).
// ---------------------------------------------------------------------------
template <typename T>
struct LinkAlgDev3 {
  typedef T R;
  typedef Group<3, T> G;
  typedef typename G::M M;
  static constexpr int NA = 8;
  static constexpr bool kDelta = true;

  GL_HD static M ident() { return G::zero(); }
  GL_HD static M full(const M& d) {
    M u = d;
    u.m[0].re += 1.f;
    u.m[4].re += 1.f;
    u.m[8].re += 1.f;
    return u;
  }
  // (1+x)(1+y) - 1 = x (1+y) + y: the products carry the small factor x,
  // so their rounding stays of the size u |x| even though 1+y is O(1).
  GL_HD static M mul(const M& x, const M& y) {
    const M y1 = full(y);
    M r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cplx<R> acc = fma_c(x.m[3 * i], y1.m[j], y.m[3 * i + j]);
        acc = fma_c(x.m[3 * i + 1], y1.m[3 + j], acc);
        acc = fma_c(x.m[3 * i + 2], y1.m[6 + j], acc);
        r.m[3 * i + j] = acc;
      }
    return r;
  }
  // (1+x)(1+y)^+ - 1 = x (1+y)^+ + y^+
  GL_HD static M mul_d(const M& x, const M& y) {
    const M y1 = full(y);
    M r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cplx<R> acc = fma_cj(x.m[3 * i], y1.m[3 * j], cj(y.m[3 * j + i]));
        acc = fma_cj(x.m[3 * i + 1], y1.m[3 * j + 1], acc);
        r.m[3 * i + j] = fma_cj(x.m[3 * i + 2], y1.m[3 * j + 2], acc);
      }
    return r;
  }
  // (1+x)^+(1+y) - 1 = (1+x)^+ y + x^+
  GL_HD static M d_mul(const M& x, const M& y) {
    const M x1 = full(x);
    M r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cplx<R> acc = fma_cj(y.m[j], x1.m[i], cj(x.m[3 * j + i]));
        acc = fma_cj(y.m[3 + j], x1.m[3 + i], acc);
        r.m[3 * i + j] = fma_cj(y.m[6 + j], x1.m[6 + i], acc);
      }
    return r;
  }

  // Staple sums c 1 + d (d a full matrix, c the summed weights).
  struct Sum {
    R c;
    M d;
  };
  GL_HD static Sum zero_sum() { return Sum{0.f, G::zero()}; }
  GL_HD static void sum_add(Sum& s, R w, const M& t) {
    s.c += w;
    G::scale_add(s.d, w, t);
  }
  // Im tr t^a (1+u)(c + d) = Im tr t^a (d + u (c + d)): the identity part
  // projects to zero; only the anti-hermitian part of d + u (c + d) is formed.
  GL_HD static void proj_mul_sum(const M& u, const Sum& s, R* o) {
    M d1 = s.d;
    d1.m[0].re += s.c;
    d1.m[4].re += s.c;
    d1.m[8].re += s.c;
    cplx<R> p[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (i == j) continue;
        cplx<R> acc = fma_c(u.m[3 * i], d1.m[j], s.d.m[3 * i + j]);
        acc = fma_c(u.m[3 * i + 1], d1.m[3 + j], acc);
        p[3 * i + j] = fma_c(u.m[3 * i + 2], d1.m[6 + j], acc);
      }
    R dg[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R acc = s.d.m[4 * i].im;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        acc = fma(u.m[3 * i + k].re, d1.m[3 * k + i].im, acc);
        acc = fma(u.m[3 * i + k].im, d1.m[3 * k + i].re, acc);
      }
      dg[i] = acc;
    }
    o[0] = 0.5f * (p[1].im + p[3].im);
    o[1] = 0.5f * (p[1].re - p[3].re);
    o[2] = 0.5f * (dg[0] - dg[1]);
    o[3] = 0.5f * (p[2].im + p[6].im);
    o[4] = 0.5f * (p[2].re - p[6].re);
    o[5] = 0.5f * (p[5].im + p[7].im);
    o[6] = 0.5f * (p[5].re - p[7].re);
    o[7] = (dg[0] + dg[1] - 2.f * dg[2]) * 0.28867513459481288225f;
  }
  // Same interface for a plain product (1+u) X with X full.
  GL_HD static void proj_mul(const M& u, const M& x, R* o) {
    Sum s{0.f, x};
    proj_mul_sum(u, s, o);
  }
  // Im tr t^a (1+x)(1+y) and Im tr t^a (1+x)(1+y)^+ of two deviations:
  // the staple-sum form with weight 1 and d = y (or y^+), so every
  // rounding stays of the size u |x|, u |y|.
  GL_HD static void proj_prod(const M& x, const M& y, R* o) {
    Sum s{1.f, y};
    proj_mul_sum(x, s, o);
  }
  GL_HD static void proj_prod_d(const M& x, const M& y, R* o) {
    Sum s{1.f, G::dag(y)};
    proj_mul_sum(x, s, o);
  }

  // exp(i c v^a t^a) - 1 by Cayley-Hamilton.  Q = c v^a t^a is hermitian and
  // traceless, so Q^3 = c1 Q + c0 with c1 = tr(Q^2)/2 and c0 = det Q, and
  // every power is Q^n = al_n + be_n Q + ga_n Q^2 with
  //   al_{n+1} = c0 ga_n,  be_{n+1} = al_n + c1 ga_n,  ga_{n+1} = be_n.
  // exp(iQ) - 1 = sum_{n>=1} (i^n/n!) Q^n = f0 + f1 Q + f2 Q^2, summed to
  // n = 9: the remainder is below ||Q||^10/10! < 3e-10 ||Q|| for
  // ||Q||_F <= 1/2.  f0 collects only terms of order ||Q||^3 and up, so
  // nothing of size 1 is formed.  Larger ||Q|| is halved s times first and
  // the result doubled exactly, e_{2h} = 2 e_h + e_h^2.
  GL_HD static M expi(const R* v, R c) {
    R nq2 = 0.f;
#pragma unroll
    for (int a = 0; a < NA; ++a) nq2 += v[a] * v[a];
    R nn = 0.5f * c * c * nq2;  // ||Q||_F^2
    if (all_zero_s(nn)) return G::zero();
    int s = 0;
    R sc = c;
    while (any_gt_s(nn, 0.25f) && s < 40) {
      nn *= 0.25f;
      sc *= 0.5f;
      ++s;
    }
    R cv[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) cv[a] = sc * v[a];
    const M Q = G::herm(cv);
    // Q^2: real diagonal, upper triangle, lower = conjugate
    R d2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R acc = Q.m[4 * i].re * Q.m[4 * i].re;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (k != i) acc = fma(Q.m[3 * i + k].re, Q.m[3 * i + k].re, fma(Q.m[3 * i + k].im, Q.m[3 * i + k].im, acc));
      d2[i] = acc;
    }
    const cplx<R> q01 = fma_c(Q.m[2], Q.m[7], fma_c(Q.m[1], Q.m[4], Q.m[0].re * Q.m[1]));
    const cplx<R> q02 = fma_c(Q.m[1], Q.m[5], fma_c(Q.m[2], Q.m[8], Q.m[0].re * Q.m[2]));
    const cplx<R> q12 = fma_c(Q.m[3], Q.m[2], fma_c(Q.m[5], Q.m[8], Q.m[4].re * Q.m[5]));
    const R c1 = 0.5f * (d2[0] + d2[1] + d2[2]);
    // det Q = q00 q11 q22 + 2 Re(Q01 Q12 Q20) - q00 |Q12|^2 - q11 |Q02|^2 - q22 |Q01|^2
    const cplx<R> t = Q.m[1] * Q.m[5];
    R c0 = Q.m[0].re * Q.m[4].re * Q.m[8].re;
    c0 = fma(2.f * t.re, Q.m[2].re, c0);
    c0 = fma(2.f * t.im, Q.m[2].im, c0);
    c0 = fma(-Q.m[0].re, Q.m[5].re * Q.m[5].re + Q.m[5].im * Q.m[5].im, c0);
    c0 = fma(-Q.m[4].re, Q.m[2].re * Q.m[2].re + Q.m[2].im * Q.m[2].im, c0);
    c0 = fma(-Q.m[8].re, Q.m[1].re * Q.m[1].re + Q.m[1].im * Q.m[1].im, c0);
    // series: n = 1 gives i Q; n >= 2 by the recurrence
    R al = 0.f, be = 1.f, ga = 0.f;
    cplx<R> f0{0.f, 0.f}, f1{0.f, 1.f}, f2{0.f, 0.f};
    const float inv_fact[10] = {1.f, 1.f, 0.5f, 1.f / 6.f, 1.f / 24.f, 1.f / 120.f, 1.f / 720.f, 1.f / 5040.f,
                                1.f / 40320.f, 1.f / 362880.f};
#pragma unroll
    for (int n = 2; n <= 9; ++n) {
      const R nal = c0 * ga, nbe = fma(c1, ga, al);
      ga = be;
      al = nal;
      be = nbe;
      const float k = inv_fact[n];
      // i^n: n mod 4 = 0: +1, 1: +i, 2: -1, 3: -i
      if ((n & 3) == 0) {
        f0.re = fma(k, al, f0.re); f1.re = fma(k, be, f1.re); f2.re = fma(k, ga, f2.re);
      } else if ((n & 3) == 1) {
        f0.im = fma(k, al, f0.im); f1.im = fma(k, be, f1.im); f2.im = fma(k, ga, f2.im);
      } else if ((n & 3) == 2) {
        f0.re = fma(-k, al, f0.re); f1.re = fma(-k, be, f1.re); f2.re = fma(-k, ga, f2.re);
      } else {
        f0.im = fma(-k, al, f0.im); f1.im = fma(-k, be, f1.im); f2.im = fma(-k, ga, f2.im);
      }
    }
    M e;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R qd = Q.m[4 * i].re;
      e.m[4 * i] = cplx<R>{fma(f2.re, d2[i], fma(f1.re, qd, f0.re)), fma(f2.im, d2[i], fma(f1.im, qd, f0.im))};
    }
    e.m[1] = fma_c(f2, q01, f1 * Q.m[1]);
    e.m[2] = fma_c(f2, q02, f1 * Q.m[2]);
    e.m[5] = fma_c(f2, q12, f1 * Q.m[5]);
    e.m[3] = fma_c(f2, cj(q01), f1 * Q.m[3]);
    e.m[6] = fma_c(f2, cj(q02), f1 * Q.m[6]);
    e.m[7] = fma_c(f2, cj(q12), f1 * Q.m[7]);
    for (int k = 0; k < s; ++k) {
      const M e2 = G::mul(e, e);
#pragma unroll
      for (int q = 0; q < 9; ++q) e.m[q] = (R)2 * e.m[q] + e2.m[q];
    }
    return e;
  }

  // The same exponential by a Taylor-Horner series (kept for the implicit
  // sweep, whose register budget suits it better): the series
  // e = iQ (1 + iQ/2 (1 + iQ/3 (1 + iQ/4))) at Q / 2^s with ||Q||_F / 2^s
  // <= 1/32 (truncation below 1e-8 of |e|), then s exact doublings
  // e_{2h} = 2 e_h + e_h^2 (from exp(iQ) = exp(iQ/2)^2).
  GL_HD static M expi_series(const R* v, R c) {
    R nq2 = 0.f;
#pragma unroll
    for (int a = 0; a < NA; ++a) nq2 += v[a] * v[a];
    R nq = lane_abs_s(c) * gl_sqrt(0.5f * nq2);
    if (all_zero_s(nq)) return G::zero();
    int s = 0;
    R sc = c;
    while (any_gt_s(nq, 0.03125f) && s < 40) {
      nq *= 0.5f;
      sc *= 0.5f;
      ++s;
    }
    R cv[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) cv[a] = sc * v[a];
    const M Q = G::herm(cv);
    // Horner: Y <- 1 + (i/k) Q Y for k = 4, 3, 2, then e = i Q Y
    M Y;
#pragma unroll
    for (int k = 0; k < 9; ++k) Y.m[k] = cplx<R>{-0.25f * Q.m[k].im, 0.25f * Q.m[k].re};  // iQ/4
    Y.m[0].re += 1.f;
    Y.m[4].re += 1.f;
    Y.m[8].re += 1.f;
#pragma unroll
    for (int k = 3; k >= 2; --k) {
      const M QY = G::mul(Q, Y);
      const float f = 1.f / (float)k;
#pragma unroll
      for (int q = 0; q < 9; ++q) Y.m[q] = cplx<R>{-f * QY.m[q].im, f * QY.m[q].re};
      Y.m[0].re += 1.f;
      Y.m[4].re += 1.f;
      Y.m[8].re += 1.f;
    }
    M e = G::mul(Q, Y);
#pragma unroll
    for (int q = 0; q < 9; ++q) e.m[q] = cplx<R>{-e.m[q].im, e.m[q].re};  // times i
    for (int k = 0; k < s; ++k) {
      const M e2 = G::mul(e, e);
#pragma unroll
      for (int q = 0; q < 9; ++q) e.m[q] = (R)2 * e.m[q] + e2.m[q];
    }
    return e;
  }

  // Re-unitarisation of 1 + d: rows 0 and 1 by Gram-Schmidt, row 2 =
  // conj(row0 x row1), every step written for the deviation from e_k so
  // that no O(1) quantity is formed.
  GL_HD static R inv_sqrt_m1(R eps) {  // 1/sqrt(1+eps) - 1
    // a link one step from the group has |eps| ~ 1e-7: the binomial series
    // -eps/2 + 3 eps^2/8 - 5 eps^3/16 is exact to 35/128 eps^4 there
    if (all_abs_lt_s(eps, 1e-3f)) return eps * fma(eps, fma(eps, R(-0.3125f), R(0.375f)), R(-0.5f));
    const R r = gl_sqrt(R(1.f) + eps);
    return lane_div_s(-eps, r * (R(1.f) + r));
  }
  GL_HD static M reunit(const M& x) {
    M r;
    const cplx<R>* a = &x.m[0];
    R e0 = 2.f * a[0].re;
#pragma unroll
    for (int k = 0; k < 3; ++k) e0 += a[k].re * a[k].re + a[k].im * a[k].im;
    const R g0 = inv_sqrt_m1(e0), f0 = 1.f + g0;
    cplx<R> ap[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ap[k] = f0 * a[k];
    ap[0].re += g0;
    // row 1 = e1 + b: p = <row0', row1> = b0 + conj(a'_1) + sum conj(a'_k) b_k
    const cplx<R>* b = &x.m[3];
    cplx<R> p = b[0] + cj(ap[1]);
#pragma unroll
    for (int k = 0; k < 3; ++k) p = fma_cj(b[k], ap[k], p);
    cplx<R> bb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) bb[k] = b[k] - p * ap[k];
    bb[0] = bb[0] - p;
    R e1 = 2.f * bb[1].re;
#pragma unroll
    for (int k = 0; k < 3; ++k) e1 += bb[k].re * bb[k].re + bb[k].im * bb[k].im;
    const R g1 = inv_sqrt_m1(e1), f1 = 1.f + g1;
    cplx<R> bp[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) bp[k] = f1 * bb[k];
    bp[1].re += g1;
    // row 2 - e2 = conj(e0 x b' + a' x e1 + a' x b')
    const cplx<R> c0 = ap[1] * bp[2] - ap[2] * bp[1] - ap[2];
    const cplx<R> c1 = ap[2] * bp[0] - ap[0] * bp[2] - bp[2];
    const cplx<R> c2 = ap[0] * bp[1] - ap[1] * bp[0] + bp[1] + ap[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r.m[k] = ap[k];
      r.m[3 + k] = bp[k];
    }
    r.m[6] = cj(c0);
    r.m[7] = cj(c1);
    r.m[8] = cj(c2);
    return r;
  }

  // Adjoint transport of an algebra vector (not a small difference: the full
  // link is used).
  GL_HD static void adj(const M& u, R* q) { G::adj(full(u), q); }
  GL_HD static void adj_dag(const M& u, R* q) { G::adj_dag(full(u), q); }
};

template <>
struct LinkAlg<3, float> : LinkAlgDev3<float> {};

// ---------------------------------------------------------------------------
// SU(2), FP32, deviation form: M = (alpha - 1, beta).
// ---------------------------------------------------------------------------
template <typename T>
struct LinkAlgDev2 {
  typedef T R;
  typedef Group<2, T> G;
  typedef typename G::M M;
  static constexpr int NA = 3;
  static constexpr bool kDelta = true;

  GL_HD static M ident() { return G::zero(); }
  GL_HD static M full(const M& d) { return M{{d.a.re + 1.f, d.a.im}, d.b}; }
  GL_HD static M expi_series(const R* v, R c) { return expi(v, c); }
  GL_HD static M dag(const M& x) { return M{cj(x.a), -x.b}; }
  // alpha = a1 + a2 + a1 a2 - b1 b2*, beta = b1 + b2 + a1 b2 + b1 a2*
  GL_HD static M mul(const M& x, const M& y) {
    return M{x.a + y.a + x.a * y.a - mulc(x.b, y.b), x.b + y.b + x.a * y.b + mulc(x.b, y.a)};
  }
  GL_HD static M mul_d(const M& x, const M& y) { return mul(x, dag(y)); }
  GL_HD static M d_mul(const M& x, const M& y) { return mul(dag(x), y); }

  struct Sum {
    R c;
    M d;
  };
  GL_HD static Sum zero_sum() { return Sum{0.f, G::zero()}; }
  GL_HD static void sum_add(Sum& s, R w, const M& t) {
    s.c += w;
    G::scale_add(s.d, w, t);
  }
  // Im tr t^a (1+u)(c + d) = Im tr t^a (c u + d + u d)
  GL_HD static void proj_mul_sum(const M& u, const Sum& s, R* o) {
    M y{s.c * u.a + s.d.a, s.c * u.b + s.d.b};
    R p[NA], q[NA];
    G::proj(y, p);
    G::proj(G::mul(u, s.d), q);
#pragma unroll
    for (int k = 0; k < NA; ++k) o[k] = p[k] + q[k];
  }
  GL_HD static void proj_mul(const M& u, const M& x, R* o) {
    Sum s{0.f, x};
    proj_mul_sum(u, s, o);
  }
  GL_HD static void proj_prod(const M& x, const M& y, R* o) {
    Sum s{1.f, y};
    proj_mul_sum(x, s, o);
  }
  GL_HD static void proj_prod_d(const M& x, const M& y, R* o) {
    Sum s{1.f, dag(y)};
    proj_mul_sum(x, s, o);
  }
  // exp(i c v.sigma/2) - 1 = (cos th - 1 + i sin th n3, sin th (n2 + i n1)),
  // cos th - 1 = -2 sin^2(th/2)
  GL_HD static M expi(const R* v, R c) {
    const R n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (all_zero_s(n2)) return G::zero();
    const R nrm = gl_sqrt(n2);
    R sh, ch;
    gl_sincos(0.25f * c * nrm, &sh, &ch);  // half of th = c |v| / 2
    // a lane whose field is zero while its partner's is not has nrm = 0
    // and v = 0: its factor is set to 0
    const R s = 2.f * sh * ch, f = lane_div0_s(s, nrm);
    return M{{-2.f * sh * sh, f * v[2]}, {f * v[1], f * v[0]}};
  }
  GL_HD static M reunit(const M& x) {
    const R eps = 2.f * x.a.re + x.a.re * x.a.re + x.a.im * x.a.im + x.b.re * x.b.re + x.b.im * x.b.im;
    const R r = gl_sqrt(R(1.f) + eps), g = lane_div_s(-eps, r * (R(1.f) + r)), f = R(1.f) + g;
    return M{{g + f * x.a.re, f * x.a.im}, f * x.b};
  }
  GL_HD static void adj(const M& u, R* q) { G::adj(full(u), q); }
  GL_HD static void adj_dag(const M& u, R* q) { G::adj_dag(full(u), q); }
};

template <>
struct LinkAlg<2, float> : LinkAlgDev2<float> {};

}  // namespace glasma
