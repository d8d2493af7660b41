// SU(2) and SU(3) arithmetic for the Glasma kernels (host+device).
//
// Conventions (Sec. 2 of Ipp & Mueller: traceless hermitian generators):
//   t^a = sigma^a / 2 (SU(2)) or lambda^a / 2 (SU(3)), tr(t^a t^b) = delta/2;
//   an algebra vector v[a] stands for the hermitian matrix sum_a v^a t^a;
//   proj(X)[a] = Im tr(t^a X), the generator projection of the
//   anti-hermitian traceless part of X used by the leapfrog force
//   (Sec. 3, Eq. lattice_1).
//
// SU(2) elements (and real multiples of them, e.g. sums of plaquettes) are
// stored as the complex pair (alpha, beta) of [[alpha, beta], [-beta*, alpha*]].
// SU(3) elements are 3x3 complex matrices, row major.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#define GL_HD __host__ __device__ __forceinline__

namespace glasma {

template <typename R>
struct cplx {
  R re, im;
};

template <typename R> GL_HD cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <typename R> GL_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> GL_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> GL_HD cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <typename R> GL_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> GL_HD cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> GL_HD cplx<R> cj(cplx<R> a) { return {a.re, -a.im}; }
// a * conj(b)
template <typename R> GL_HD cplx<R> mulc(cplx<R> a, cplx<R> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// acc + a*conj(b), four fused multiply-adds
template <typename R> GL_HD cplx<R> fma_cj(cplx<R> a, cplx<R> b, cplx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.im, b.re, acc.im);
  acc.im = fma(-a.re, b.im, acc.im);
  return acc;
}
// acc + a*b
template <typename R> GL_HD cplx<R> fma_c(cplx<R> a, cplx<R> b, cplx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}

template <typename R> GL_HD R gl_sqrt(R x) { return sqrt(x); }
template <> GL_HD float gl_sqrt<float>(float x) { return sqrtf(x); }
template <typename R> GL_HD void gl_sincos(R x, R* s, R* c) { sincos(x, s, c); }
template <> GL_HD void gl_sincos<float>(float x, float* s, float* c) { sincosf(x, s, c); }

template <int NC, typename R> struct Group;

// ---------------------------------------------------------------------------
// SU(2): (alpha, beta) pair.
// ---------------------------------------------------------------------------
template <typename R>
struct Group<2, R> {
  static constexpr int NA = 3;
  static constexpr int NV = 2;  // complex numbers per stored link
  struct M {
    cplx<R> a, b;
  };
  GL_HD static M ident() { return M{{R(1), R(0)}, {R(0), R(0)}}; }
  GL_HD static M mul(const M& x, const M& y) {
    // [[a1,b1],[-b1*,a1*]] [[a2,b2],[-b2*,a2*]]
    return M{x.a * y.a - mulc(x.b, y.b), x.a * y.b + mulc(x.b, y.a)};
  }
  GL_HD static M dag(const M& x) { return M{cj(x.a), -x.b}; }
  // x * y^dagger
  GL_HD static M mul_d(const M& x, const M& y) { return mul(x, dag(y)); }
  // x^dagger * y
  GL_HD static M d_mul(const M& x, const M& y) { return mul(dag(x), y); }
  GL_HD static void proj(const M& x, R* out) {
    out[0] = x.b.im;  // Im tr(sigma1/2 X)
    out[1] = x.b.re;  // Im tr(sigma2/2 X)
    out[2] = x.a.im;  // Im tr(sigma3/2 X)
  }
  GL_HD static R re_tr(const M& x) { return R(2) * x.a.re; }
  // proj(x y) without forming the unused parts of the product
  GL_HD static void proj_mul(const M& x, const M& y, R* out) { proj(mul(x, y), out); }
  GL_HD static void scale_add(M& acc, R w, const M& x) {
    acc.a = acc.a + w * x.a;
    acc.b = acc.b + w * x.b;
  }
  GL_HD static M zero() { return M{{R(0), R(0)}, {R(0), R(0)}}; }
  // exp(i c sum_a v^a sigma^a/2) = cos(th) + i sin(th) n.sigma, th = c|v|/2
  GL_HD static M expi(const R* v, R c) {
    R n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (n2 == R(0)) return ident();
    R nrm = gl_sqrt(n2);
    R s, co;
    gl_sincos(R(0.5) * c * nrm, &s, &co);
    R f = s / nrm;
    return M{{co, f * v[2]}, {f * v[1], f * v[0]}};
  }
  // i * (q^a sigma^a / 2) in (alpha, beta) form
  GL_HD static M alg_i(const R* q) {
    return M{{R(0), R(0.5) * q[2]}, {R(0.5) * q[1], R(0.5) * q[0]}};
  }
  GL_HD static void from_alg_i(const M& x, R* q) {
    q[0] = R(2) * x.b.im;
    q[1] = R(2) * x.b.re;
    q[2] = R(2) * x.a.im;
  }
  // q <- U^dagger q U
  GL_HD static void adj_dag(const M& u, R* q) {
    M t = mul(d_mul(u, alg_i(q)), u);
    from_alg_i(t, q);
  }
  // q <- U q U^dagger
  GL_HD static void adj(const M& u, R* q) {
    M t = mul_d(mul(u, alg_i(q)), u);
    from_alg_i(t, q);
  }
  GL_HD static M reunit(const M& x) {
    R n2 = x.a.re * x.a.re + x.a.im * x.a.im + x.b.re * x.b.re + x.b.im * x.b.im;
    R f = R(1) / gl_sqrt(n2);
    return M{f * x.a, f * x.b};
  }
  GL_HD static M add(const M& x, const M& y) { return M{x.a + y.a, x.b + y.b}; }
  // squared Frobenius norm of x - y (the 2x2 matrix holds alpha, beta twice)
  GL_HD static R fro2_diff(const M& x, const M& y) {
    cplx<R> da = x.a - y.a, db = x.b - y.b;
    return R(2) * (da.re * da.re + da.im * da.im + db.re * db.re + db.im * db.im);
  }
  // full 2x2 complex matrix element (row r, column c)
  GL_HD static cplx<R> elem(const M& x, int r, int c) {
    if (r == 0) return c == 0 ? x.a : x.b;
    return c == 0 ? -cj(x.b) : cj(x.a);
  }
};

// ---------------------------------------------------------------------------
// SU(3): 3x3 complex, row major.
// ---------------------------------------------------------------------------
template <typename R>
struct Group<3, R> {
  static constexpr int NA = 8;
  static constexpr int NV = 9;
  struct M {
    cplx<R> m[9];
  };
  GL_HD static M ident() {
    M r;
#pragma unroll
    for (int k = 0; k < 9; ++k) r.m[k] = cplx<R>{R(k % 4 == 0 ? 1 : 0), R(0)};
    return r;
  }
  GL_HD static M mul(const M& x, const M& y) {
    M r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cplx<R> acc = x.m[3 * i] * y.m[j];
        acc = fma_c(x.m[3 * i + 1], y.m[3 + j], acc);
        acc = fma_c(x.m[3 * i + 2], y.m[6 + j], acc);
        r.m[3 * i + j] = acc;
      }
    return r;
  }
  // x * y^dagger: (x y^+)_ij = sum_k x_ik conj(y_jk)
  GL_HD static M mul_d(const M& x, const M& y) {
    M r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cplx<R> acc = mulc(x.m[3 * i], y.m[3 * j]);
        acc = fma_cj(x.m[3 * i + 1], y.m[3 * j + 1], acc);
        r.m[3 * i + j] = fma_cj(x.m[3 * i + 2], y.m[3 * j + 2], acc);
      }
    return r;
  }
  // x^dagger * y: sum_k conj(x_ki) y_kj
  GL_HD static M d_mul(const M& x, const M& y) {
    M r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        cplx<R> acc = mulc(y.m[j], x.m[i]);
        acc = fma_cj(y.m[3 + j], x.m[3 + i], acc);
        r.m[3 * i + j] = fma_cj(y.m[6 + j], x.m[6 + i], acc);
      }
    return r;
  }
  GL_HD static M dag(const M& x) {
    M r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) r.m[3 * i + j] = cj(x.m[3 * j + i]);
    return r;
  }
  GL_HD static M add(const M& x, const M& y) {
    M r;
#pragma unroll
    for (int k = 0; k < 9; ++k) r.m[k] = x.m[k] + y.m[k];
    return r;
  }
  GL_HD static R fro2_diff(const M& x, const M& y) {
    R acc = R(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      cplx<R> d = x.m[k] - y.m[k];
      acc += d.re * d.re + d.im * d.im;
    }
    return acc;
  }
  // Im tr(lambda^a/2 X), Gell-Mann basis
  GL_HD static void proj(const M& x, R* o) {
    const cplx<R>* m = x.m;
    o[0] = R(0.5) * (m[1].im + m[3].im);
    o[1] = R(0.5) * (m[1].re - m[3].re);
    o[2] = R(0.5) * (m[0].im - m[4].im);
    o[3] = R(0.5) * (m[2].im + m[6].im);
    o[4] = R(0.5) * (m[2].re - m[6].re);
    o[5] = R(0.5) * (m[5].im + m[7].im);
    o[6] = R(0.5) * (m[5].re - m[7].re);
    o[7] = (m[0].im + m[4].im - R(2) * m[8].im) * R(0.28867513459481288225);  // 1/(2 sqrt 3)
  }
  GL_HD static R re_tr(const M& x) { return x.m[0].re + x.m[4].re + x.m[8].re; }
  GL_HD static M zero() {
    M r;
#pragma unroll
    for (int k = 0; k < 9; ++k) r.m[k] = cplx<R>{R(0), R(0)};
    return r;
  }
  GL_HD static void scale_add(M& acc, R w, const M& x) {
#pragma unroll
    for (int k = 0; k < 9; ++k) acc.m[k] = acc.m[k] + w * x.m[k];
  }
  // (x y)_ij
  GL_HD static cplx<R> prod_elem(const M& x, const M& y, int i, int j) {
    cplx<R> acc = x.m[3 * i] * y.m[j];
    acc = fma_c(x.m[3 * i + 1], y.m[3 + j], acc);
    return fma_c(x.m[3 * i + 2], y.m[6 + j], acc);
  }
  GL_HD static R prod_diag_im(const M& x, const M& y, int i) {
    R acc = x.m[3 * i].re * y.m[i].im + x.m[3 * i].im * y.m[i].re;
    acc = fma(x.m[3 * i + 1].re, y.m[3 + i].im, acc);
    acc = fma(x.m[3 * i + 1].im, y.m[3 + i].re, acc);
    acc = fma(x.m[3 * i + 2].re, y.m[6 + i].im, acc);
    acc = fma(x.m[3 * i + 2].im, y.m[6 + i].re, acc);
    return acc;
  }
  // proj(x y) from the six off-diagonal and three diagonal imaginary parts
  GL_HD static void proj_mul(const M& x, const M& y, R* o) {
    const cplx<R> p01 = prod_elem(x, y, 0, 1), p10 = prod_elem(x, y, 1, 0);
    const cplx<R> p02 = prod_elem(x, y, 0, 2), p20 = prod_elem(x, y, 2, 0);
    const cplx<R> p12 = prod_elem(x, y, 1, 2), p21 = prod_elem(x, y, 2, 1);
    const R d0 = prod_diag_im(x, y, 0), d1 = prod_diag_im(x, y, 1), d2 = prod_diag_im(x, y, 2);
    o[0] = R(0.5) * (p01.im + p10.im);
    o[1] = R(0.5) * (p01.re - p10.re);
    o[2] = R(0.5) * (d0 - d1);
    o[3] = R(0.5) * (p02.im + p20.im);
    o[4] = R(0.5) * (p02.re - p20.re);
    o[5] = R(0.5) * (p12.im + p21.im);
    o[6] = R(0.5) * (p12.re - p21.re);
    o[7] = (d0 + d1 - R(2) * d2) * R(0.28867513459481288225);
  }
  // hermitian H = sum_a v^a lambda^a / 2
  GL_HD static M herm(const R* v) {
    const R r3 = R(0.57735026918962576451);  // 1/sqrt 3
    M h;
    h.m[0] = cplx<R>{R(0.5) * (v[2] + r3 * v[7]), R(0)};
    h.m[4] = cplx<R>{R(0.5) * (-v[2] + r3 * v[7]), R(0)};
    h.m[8] = cplx<R>{-r3 * v[7], R(0)};
    h.m[1] = cplx<R>{R(0.5) * v[0], R(-0.5) * v[1]};
    h.m[3] = cj(h.m[1]);
    h.m[2] = cplx<R>{R(0.5) * v[3], R(-0.5) * v[4]};
    h.m[6] = cj(h.m[2]);
    h.m[5] = cplx<R>{R(0.5) * v[5], R(-0.5) * v[6]};
    h.m[7] = cj(h.m[5]);
    return h;
  }
  // components 2 Re tr(t^a H) = Re tr(lambda^a H) of a hermitian H
  GL_HD static void from_herm(const M& h, R* v) {
    const R r3 = R(0.57735026918962576451);
    v[0] = h.m[1].re + h.m[3].re;
    v[1] = h.m[3].im - h.m[1].im;
    v[2] = h.m[0].re - h.m[4].re;
    v[3] = h.m[2].re + h.m[6].re;
    v[4] = h.m[6].im - h.m[2].im;
    v[5] = h.m[5].re + h.m[7].re;
    v[6] = h.m[7].im - h.m[5].im;
    v[7] = r3 * (h.m[0].re + h.m[4].re - R(2) * h.m[8].re);
  }
  GL_HD static void adj_dag(const M& u, R* q) {
    M t = mul(d_mul(u, herm(q)), u);
    from_herm(t, q);
  }
  GL_HD static void adj(const M& u, R* q) {
    M t = mul_d(mul(u, herm(q)), u);
    from_herm(t, q);
  }

  // exp(i c H) for H = sum v^a t^a by the Cayley-Hamilton form
  //   exp(iQ) = f0 + f1 Q + f2 Q^2,  Q = c H,
  // with f_j from the eigenvalue parametrisation of Morningstar & Peardon,
  // Phys. Rev. D 69 (2004) 054501, Sec. III: c0 = det Q, c1 = tr(Q^2)/2,
  // theta = acos(c0 / c0max), u = sqrt(c1/3) cos(theta/3),
  // w = sqrt(c1) sin(theta/3); negative c0 by f_j(-c0) = (-1)^j conj f_j(c0).
  GL_HD static M expi(const R* v, R c) {
    R cv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) cv[a] = c * v[a];
    M Q = herm(cv);
    M Q2 = mul(Q, Q);
    R c1 = R(0.5) * (Q2.m[0].re + Q2.m[4].re + Q2.m[8].re);
    if (c1 == R(0)) return ident();
    // Small arguments: the series 1 + iQ - Q^2/2 is exact to rounding (its
    // truncation |Q|^3/6 is below the unit roundoff), and the eigenvalue
    // parametrisation below would underflow (c0max = 2 (c1/3)^{3/2} -> 0).
    const R small = sizeof(R) == 4 ? R(1e-8) : R(1e-20);
    if (c1 < small) {
      M r;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        cplx<R> acc{-R(0.5) * Q2.m[k].re - Q.m[k].im, -R(0.5) * Q2.m[k].im + Q.m[k].re};
        if (k % 4 == 0) acc.re += R(1);
        r.m[k] = acc;
      }
      return r;
    }
    // det of the hermitian Q (real)
    cplx<R> d = Q.m[0] * (Q.m[4] * Q.m[8] - Q.m[5] * Q.m[7]) -
                Q.m[1] * (Q.m[3] * Q.m[8] - Q.m[5] * Q.m[6]) +
                Q.m[2] * (Q.m[3] * Q.m[7] - Q.m[4] * Q.m[6]);
    R c0 = d.re;
    bool neg = c0 < R(0);
    if (neg) c0 = -c0;
    R s13 = gl_sqrt(c1 / R(3));
    R c0max = R(2) * s13 * s13 * s13;
    R ratio = c0 / c0max;
    if (ratio > R(1)) ratio = R(1);
    R theta = acos(ratio);
    R st, ct;
    gl_sincos(theta / R(3), &st, &ct);
    R u = s13 * ct;
    R w = gl_sqrt(c1) * st;
    R u2 = u * u, w2 = w * w;
    R xi0;
    if (fabs(w) < R(0.05)) {
      xi0 = R(1) - w2 / R(6) * (R(1) - w2 / R(20) * (R(1) - w2 / R(42)));
    } else {
      R sw, cw_;
      gl_sincos(w, &sw, &cw_);
      xi0 = sw / w;
    }
    R cw, sw_unused;
    gl_sincos(w, &sw_unused, &cw);
    R s2u, c2u, su, cu;
    gl_sincos(R(2) * u, &s2u, &c2u);
    gl_sincos(u, &su, &cu);
    cplx<R> e2iu{c2u, s2u};
    cplx<R> emiu{cu, -su};
    cplx<R> h0 = (u2 - w2) * e2iu +
                 emiu * cplx<R>{R(8) * u2 * cw, R(2) * u * (R(3) * u2 + w2) * xi0};
    cplx<R> h1 = (R(2) * u) * e2iu - emiu * cplx<R>{R(2) * u * cw, -(R(3) * u2 - w2) * xi0};
    cplx<R> h2 = e2iu - emiu * cplx<R>{cw, R(3) * u * xi0};
    R den = R(1) / (R(9) * u2 - w2);
    cplx<R> f0 = den * h0, f1 = den * h1, f2 = den * h2;
    if (neg) {
      f0 = cj(f0);
      f1 = -cj(f1);
      f2 = cj(f2);
    }
    M r;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      cplx<R> acc = f1 * Q.m[k];
      acc = acc + f2 * Q2.m[k];
      if (k % 4 == 0) acc = acc + f0;
      r.m[k] = acc;
    }
    return r;
  }

  // Rows 0, 1 Gram-Schmidt normalised, row 2 = conj(row0 x row1).
  GL_HD static M reunit(const M& x) {
    M r;
    R n0 = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) n0 += x.m[k].re * x.m[k].re + x.m[k].im * x.m[k].im;
    R f0 = R(1) / gl_sqrt(n0);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.m[k] = f0 * x.m[k];
    // project row 1 off row 0: p = <row0, row1> = sum conj(r0k) x1k
    cplx<R> p{R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 3; ++k) p = p + mulc(x.m[3 + k], r.m[k]);
    R n1 = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r.m[3 + k] = x.m[3 + k] - p * r.m[k];
      n1 += r.m[3 + k].re * r.m[3 + k].re + r.m[3 + k].im * r.m[3 + k].im;
    }
    R f1 = R(1) / gl_sqrt(n1);
#pragma unroll
    for (int k = 0; k < 3; ++k) r.m[3 + k] = f1 * r.m[3 + k];
    r.m[6] = cj(r.m[1] * r.m[5] - r.m[2] * r.m[4]);
    r.m[7] = cj(r.m[2] * r.m[3] - r.m[0] * r.m[5]);
    r.m[8] = cj(r.m[0] * r.m[4] - r.m[1] * r.m[3]);
    return r;
  }
  GL_HD static cplx<R> elem(const M& x, int r, int c) { return x.m[3 * r + c]; }
};

}  // namespace glasma
