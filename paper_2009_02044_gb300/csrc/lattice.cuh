// Lattice geometry, structure-of-arrays field access and the staple force
// shared by the step and observable kernels.
//
// Layout in device memory (V = nz*ny*nx sites, site s = (iz*ny + iy)*nx + ix,
// x fastest; x, y periodic, z open):
//   links  complex component k of link d at site s, stored as float2 /
//          double2:
//          SU(2) (k = alpha, beta): U[(d*V + s)*2 + k], so one link is
//          16 contiguous bytes in FP32 (one vector load) and 32 in FP64;
//          SU(3) (k = row-major 3x3 entry), in blocks of 32 sites:
//          U[((d*C + s/32)*9 + k)*32 + s%32] with C = ceil(V/32) blocks per
//          direction, so the components of one link sit 32 entries apart
//          (immediate address offsets) and a warp still reads 32
//          consecutive sites of one component;
//   fields E[(d*NA + a)*V + s]   algebra component a of E_d at site s
//   charges Q[(a*W + w)*nxy + t] component a, window slot w, transverse t
// The z link of the last slice does not exist: it is stored as the identity
// and never updated, and E_z there is zero.
#pragma once
#include <stdint.h>

#include "link_alg.cuh"

namespace glasma {

template <typename R> struct V2T;
template <> struct V2T<float> { typedef float2 T; };
template <> struct V2T<double> { typedef double2 T; };

struct Geom {
  int nx, ny, nz;
  int64_t nxy, V;
};

// Element index of complex component k of link d at site s (see above),
// and the number of complex elements of one link array (SU(3) pads V up to
// whole blocks of 32 sites).
GL_HD int64_t link_index(int nc, int d, int k, int64_t V, int64_t s) {
  if (nc == 2) return ((int64_t)d * V + s) * 2 + k;
  return (((int64_t)d * ((V + 31) >> 5) + (s >> 5)) * 9 + k) * 32 + (s & 31);
}
GL_HD int64_t link_elems(int nc, int64_t V) { return nc == 2 ? 6 * V : 27 * 32 * ((V + 31) >> 5); }

GL_HD int64_t site_index(const Geom& g, int ix, int iy, int iz) {
  return ((int64_t)iz * g.ny + iy) * g.nx + ix;
}

template <int NC, typename R> struct LinkIO;

// FP32 storage holds U - 1 (see link_alg.cuh); loading it as FP64 gives the
// full matrix, storing an FP64 full matrix into it subtracts the identity
// before rounding.  FP64 storage holds U.
template <typename Rs, typename Rc>
struct DeltaConv {
  static constexpr bool to_full = sizeof(Rs) == 4 && sizeof(Rc) == 8;
};

template <typename R>
struct LinkIO<2, R> {
  template <typename Rc>
  GL_HD static typename Group<2, Rc>::M load(const typename V2T<R>::T* U, int d, int64_t V, int64_t s) {
    const typename V2T<R>::T* p = U + link_index(2, d, 0, V, s);
    typename V2T<R>::T a, b;
    if (sizeof(R) == 4) {  // alpha and beta in one 16-byte load
      const float4 v = *reinterpret_cast<const float4*>(p);
      a.x = R(v.x); a.y = R(v.y); b.x = R(v.z); b.y = R(v.w);
    } else {
      a = p[0];
      b = p[1];
    }
    typename Group<2, Rc>::M m{{Rc(a.x), Rc(a.y)}, {Rc(b.x), Rc(b.y)}};
    if (DeltaConv<R, Rc>::to_full) m.a.re += Rc(1);
    return m;
  }
  template <typename Rc>
  GL_HD static void store(typename V2T<R>::T* U, int d, int64_t V, int64_t s, const typename Group<2, Rc>::M& m) {
    typename V2T<R>::T a, b;
    const Rc one = DeltaConv<R, Rc>::to_full ? Rc(1) : Rc(0);
    a.x = R(m.a.re - one); a.y = R(m.a.im);
    b.x = R(m.b.re); b.y = R(m.b.im);
    typename V2T<R>::T* p = U + link_index(2, d, 0, V, s);
    if (sizeof(R) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(float(a.x), float(a.y), float(b.x), float(b.y));
    } else {
      p[0] = a;
      p[1] = b;
    }
  }
};

template <typename R>
struct LinkIO<3, R> {
  template <typename Rc>
  GL_HD static typename Group<3, Rc>::M load(const typename V2T<R>::T* U, int d, int64_t V, int64_t s) {
    typename Group<3, Rc>::M m;
    const typename V2T<R>::T* p = U + link_index(3, d, 0, V, s);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      typename V2T<R>::T v = p[k * 32];
      m.m[k] = cplx<Rc>{Rc(v.x), Rc(v.y)};
    }
    if (DeltaConv<R, Rc>::to_full) {
      m.m[0].re += Rc(1);
      m.m[4].re += Rc(1);
      m.m[8].re += Rc(1);
    }
    return m;
  }
  template <typename Rc>
  GL_HD static void store(typename V2T<R>::T* U, int d, int64_t V, int64_t s, const typename Group<3, Rc>::M& m) {
    const Rc one = DeltaConv<R, Rc>::to_full ? Rc(1) : Rc(0);
    typename V2T<R>::T* p = U + link_index(3, d, 0, V, s);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      typename V2T<R>::T v;
      v.x = R(k % 4 == 0 ? m.m[k].re - one : m.m[k].re);
      v.y = R(m.m[k].im);
      p[k * 32] = v;
    }
  }
};

// Coordinates and neighbour indices of one site.
struct SiteNbr {
  int ix, iy, iz;
  int64_t s;
  int64_t p[3];  // x + e_d
  int64_t m[3];  // x - e_d
};

GL_HD SiteNbr site_nbr(const Geom& g, int64_t s) {
  SiteNbr n;
  n.s = s;
  n.ix = (int)(s % g.nx);
  int64_t t = s / g.nx;
  n.iy = (int)(t % g.ny);
  n.iz = (int)(t / g.ny);
  n.p[0] = n.ix + 1 == g.nx ? s - (g.nx - 1) : s + 1;
  n.m[0] = n.ix == 0 ? s + (g.nx - 1) : s - 1;
  n.p[1] = n.iy + 1 == g.ny ? s - (int64_t)(g.ny - 1) * g.nx : s + g.nx;
  n.m[1] = n.iy == 0 ? s + (int64_t)(g.ny - 1) * g.nx : s - g.nx;
  n.p[2] = s + g.nxy;  // valid for iz <= nz-2
  n.m[2] = s - g.nxy;  // valid for iz >= 1
  return n;
}

// The same from the transverse index t = iy*nx + ix (< 2^31) and the slice
// iz, with 32-bit division only.
GL_HD SiteNbr site_nbr_tz(const Geom& g, uint32_t t, int iz) {
  SiteNbr n;
  const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
  const uint32_t iy = t / nx, ix = t - iy * nx;
  n.ix = (int)ix;
  n.iy = (int)iy;
  n.iz = iz;
  const int64_t base = (int64_t)iz * g.nxy;
  n.s = base + t;
  const uint32_t xp = ix + 1 == nx ? 0 : ix + 1, xm = ix == 0 ? nx - 1 : ix - 1;
  const uint32_t yp = iy + 1 == ny ? 0 : iy + 1, ym = iy == 0 ? ny - 1 : iy - 1;
  n.p[0] = base + iy * nx + xp;
  n.m[0] = base + iy * nx + xm;
  n.p[1] = base + yp * nx + ix;
  n.m[1] = base + ym * nx + ix;
  n.p[2] = n.s + g.nxy;
  n.m[2] = n.s - g.nxy;
  return n;
}

// F^a = -sum_{j != i} w_j [Im tr t^a U_{i,j}(x) + Im tr t^a U_{i,-j}(x)]
// (Sec. 3, Eq. lattice_1 with Eq. plaquette; w_j = 2 / a_j^2), plaquettes
// that leave the open z range omitted, evaluated from the staple sum:
// F = -proj(U_i(x) S) with
// S = sum_j w_j [U_j(x+i) U_i^dag(x+j) U_j^dag(x)
//                + U_j^dag(x+i-j) U_i^dag(x-j) U_j(x-j)],
// since Im tr t^a (U_i S) is linear in S.  Only the anti-hermitian part of
// the last product is formed.
template <int NC, typename Rs, typename Rc>
GL_HD void link_force_staple(const typename V2T<Rs>::T* U, const Geom& g, const SiteNbr& n, int i, const Rc* w,
                             Rc* F) {
  typedef LinkAlg<NC, Rc> G;
  typedef typename G::M M;
  typename G::Sum S = G::zero_sum();
  const Rc wt = w[0], wz = w[2];
  const int64_t pi = n.p[i];
  // one copy of the staple code (fewer instruction-cache misses)
#pragma unroll 1
  for (int j = 0; j < 3; ++j) {
    if (j == i) continue;
    const Rc wj = j == 2 ? wz : wt;
    const bool fwd = (j != 2) || (n.iz <= g.nz - 2);
    const bool bwd = (j != 2) || (n.iz >= 1);
    const int64_t pj = n.p[j], mj = n.m[j];
    if (fwd) {
      M T = G::mul_d(LinkIO<NC, Rs>::template load<Rc>(U, j, g.V, pi),
                     LinkIO<NC, Rs>::template load<Rc>(U, i, g.V, pj));
      T = G::mul_d(T, LinkIO<NC, Rs>::template load<Rc>(U, j, g.V, n.s));
      G::sum_add(S, wj, T);
    }
    if (bwd) {
      // x + e_i - e_j: the periodic wraps of x and y depend only on ix and
      // iy and z has no wrap, so the two offsets add
      M T = G::mul(LinkIO<NC, Rs>::template load<Rc>(U, i, g.V, mj),
                   LinkIO<NC, Rs>::template load<Rc>(U, j, g.V, pi + mj - n.s));
      T = G::d_mul(T, LinkIO<NC, Rs>::template load<Rc>(U, j, g.V, mj));
      G::sum_add(S, wj, T);
    }
  }
  constexpr int NA = G::NA;
  Rc pr[NA];
  // U_i(x) is loaded only here, so it is not live across the staples
  G::proj_mul_sum(LinkIO<NC, Rs>::template load<Rc>(U, i, g.V, n.s), S, pr);
#pragma unroll
  for (int a = 0; a < NA; ++a) F[a] = -pr[a];
}

}  // namespace glasma
