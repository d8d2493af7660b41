// The leapfrog link update of step_link (Sec. 3, Eqs. lattice_1,
// lattice_2, the NGP hop and its current) for two sites at once, in the two
// lanes of the packed FP32 instructions (pair.cuh): lane A is the site
// (t, iz), lane B the site (t, iz + H) with H = ceil(nz / 2).  Both sites
// share their transverse neighbours, so every index of lane B is lane A's
// plus H nxy.  The lanes differ only at the open z boundaries: a staple that
// leaves the z range in one lane gets weight 0 there (its loads read a valid
// site instead), and the z link of the last slice, which does not exist, is
// not written.  FP32 state only.
#pragma once
#include "step_link.cuh"

namespace glasma {

// 32-bit read-only loads that stay separate (two adjacent floats of one
// complex number go to the lanes of two different pairs).  Loading the
// complex number as one 64-bit word and moving its halves into the pairs
// made the SU(3) kernel 24% slower (0.709 against 0.572 ms per
// 512 x 64^2 step).
__device__ __forceinline__ float ldg_f32(const float* p) {
  float r;
  asm("ld.global.nc.f32 %0, [%1];" : "=f"(r) : "l"(p));
  return r;
}

template <int NC> struct PairIO;

template <>
struct PairIO<3> {
  typedef LinkAlgDev3<f2> G;
  typedef G::M M;
  // deviation-form link d at the sites sa (lane A) and sb (lane B)
  __device__ __forceinline__ static M load(const float2* U, int d, int64_t V, int64_t sa, int64_t sb) {
    const float* pa = (const float*)(U + link_index(3, d, 0, V, sa));
    const float* pb = (const float*)(U + link_index(3, d, 0, V, sb));
    M m;
#pragma unroll
    for (int k = 0; k < 9; ++k)
      m.m[k] = cplx<f2>{f2(ldg_f32(pa + 64 * k), ldg_f32(pb + 64 * k)),
                        f2(ldg_f32(pa + 64 * k + 1), ldg_f32(pb + 64 * k + 1))};
    return m;
  }
  __device__ __forceinline__ static void store(float2* U, int d, int64_t V, int64_t sa, int64_t sb, const M& m,
                                               bool wa, bool wb) {
    float2* pa = U + link_index(3, d, 0, V, sa);
    float2* pb = U + link_index(3, d, 0, V, sb);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (wa) pa[32 * k] = make_float2(m.m[k].re.v.x, m.m[k].im.v.x);
      if (wb) pb[32 * k] = make_float2(m.m[k].re.v.y, m.m[k].im.v.y);
    }
  }
};

template <>
struct PairIO<2> {
  typedef LinkAlgDev2<f2> G;
  typedef G::M M;
  // (alpha, beta) of one link are 16 contiguous bytes: one address per lane
  __device__ __forceinline__ static M load(const float2* U, int d, int64_t V, int64_t sa, int64_t sb) {
    const float* pa = (const float*)(U + link_index(2, d, 0, V, sa));
    const float* pb = (const float*)(U + link_index(2, d, 0, V, sb));
    M m;
    m.a = cplx<f2>{f2(ldg_f32(pa), ldg_f32(pb)), f2(ldg_f32(pa + 1), ldg_f32(pb + 1))};
    m.b = cplx<f2>{f2(ldg_f32(pa + 2), ldg_f32(pb + 2)), f2(ldg_f32(pa + 3), ldg_f32(pb + 3))};
    return m;
  }
  __device__ __forceinline__ static void store(float2* U, int d, int64_t V, int64_t sa, int64_t sb, const M& m,
                                               bool wa, bool wb) {
    if (wa)
      *reinterpret_cast<float4*>(U + link_index(2, d, 0, V, sa)) =
          make_float4(m.a.re.v.x, m.a.im.v.x, m.b.re.v.x, m.b.im.v.x);
    if (wb)
      *reinterpret_cast<float4*>(U + link_index(2, d, 0, V, sb)) =
          make_float4(m.a.re.v.y, m.a.im.v.y, m.b.re.v.y, m.b.im.v.y);
  }
};

template <int NC> struct PairAlg;
template <> struct PairAlg<3> { typedef LinkAlgDev3<f2> G; };
template <> struct PairAlg<2> { typedef LinkAlgDev2<f2> G; };

// Geometry of one thread's two sites for one link direction.
struct SitePair {
  SiteNbr n;      // lane A's site and neighbours
  int64_t dB;     // lane B's indices are lane A's plus dB
  int izB;        // lane B's slice
  bool writeB;    // lane B holds a link of the lattice in this direction;
                  // if not, dB = 0 and lane B repeats lane A's work unwritten
};

// Staple force of link i at both sites (link_force_staple with per-lane
// weights; a staple that leaves the open z range in a lane weighs 0 there).
template <int NC>
__device__ __forceinline__ void pair_force(const float2* U, const Geom& g, const SitePair& P, int i, const float* w,
                                           f2* F) {
  typedef typename PairAlg<NC>::G G;
  typedef typename G::M M;
  typename G::Sum S = G::zero_sum();
  const SiteNbr& n = P.n;
  const int64_t pi = n.p[i], dB = P.dB;
#pragma unroll 1
  for (int j = 0; j < 3; ++j) {
    if (j == i) continue;
    const float wj = j == 2 ? w[2] : w[0];
    const int64_t pj = n.p[j], mj = n.m[j];
    // forward staple U_j(x+i) U_i^dag(x+j) U_j^dag(x)
    {
      const bool okA = j != 2 || n.iz <= g.nz - 2, okB = j != 2 || P.izB <= g.nz - 2;
      if (okA || okB) {
        const int64_t cA = okA ? 0 : n.s - pj, cB = okB ? dB : dB + n.s - pj;  // clamp x+j to x
        M T = G::mul_d(PairIO<NC>::load(U, j, g.V, pi, pi + dB), PairIO<NC>::load(U, i, g.V, pj + cA, pj + cB));
        T = G::mul_d(T, PairIO<NC>::load(U, j, g.V, n.s, n.s + dB));
        G::sum_add(S, f2(okA ? wj : 0.f, okB ? wj : 0.f), T);
      }
    }
    // backward staple U_j^dag(x+i-j) U_i^dag(x-j) U_j(x-j)
    {
      const bool okA = j != 2 || n.iz >= 1, okB = j != 2 || P.izB >= 1;
      if (okA || okB) {
        const int64_t cA = okA ? 0 : n.s - mj, cB = okB ? dB : dB + n.s - mj;  // clamp x-j to x
        M T = G::mul(PairIO<NC>::load(U, i, g.V, mj + cA, mj + cB),
                     PairIO<NC>::load(U, j, g.V, pi + mj - n.s + cA, pi + mj - n.s + cB));
        T = G::d_mul(T, PairIO<NC>::load(U, j, g.V, mj + cA, mj + cB));
        G::sum_add(S, f2(okA ? wj : 0.f, okB ? wj : 0.f), T);
      }
    }
  }
  constexpr int NA = G::NA;
  f2 pr[NA];
  G::proj_mul_sum(PairIO<NC>::load(U, i, g.V, n.s, n.s + dB), S, pr);
#pragma unroll
  for (int a = 0; a < NA; ++a) F[a] = -pr[a];
}

// update_link for both lanes: E += dt F (+ the hop current on the z link),
// then exp(i dt E) U re-unitarised; lane B is written only if it exists.
template <int NC>
__device__ __forceinline__ void pair_update(const StepArgs<float>& a, const SitePair& P, int i, uint32_t t,
                                            const f2* F) {
  typedef typename PairAlg<NC>::G G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
  const int64_t sa = P.n.s, sb = sa + P.dB;
  const bool wb = P.writeB;
  const M Ui = PairIO<NC>::load((const float2*)a.U, i, a.g.V, sa, sb);
  f2 e[NA];
#pragma unroll
  for (int c = 0; c < NA; ++c) {
    const float* Ec = a.E + (int64_t)(i * NA + c) * a.g.V;
    e[c] = fma(f2(a.dt), F[c], f2(Ec[sa], Ec[sb]));
  }
  if (i == 2 && a.hop) {
    f2 dj[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) dj[c] = f2(0.f);
    const int nxy = (int)a.g.nxy;
    {
      const int kA = P.n.iz - a.zB0, kB = P.izB - a.zB0;
      const bool inA = kA >= 0 && kA < a.WB, inB = wb && kB >= 0 && kB < a.WB;
      if (inA || inB) {
        const int64_t qa = (int64_t)(inA ? kA : kB) * nxy + t, qb = (int64_t)(inB ? kB : kA) * nxy + t;
        const int64_t cs = (int64_t)a.WB * nxy;
        f2 q[NA];
#pragma unroll
        for (int c = 0; c < NA; ++c) q[c] = f2(a.QB[c * cs + qa], a.QB[c * cs + qb]);
        const f2 wq(inA ? a.az2 : 0.f, inB ? a.az2 : 0.f);
#pragma unroll
        for (int c = 0; c < NA; ++c) dj[c] = fma(-wq, q[c], dj[c]);
        G::adj_dag(Ui, q);
#pragma unroll
        for (int c = 0; c < NA; ++c) {
          if (inA) a.QB[c * cs + qa] = q[c].v.x;
          if (inB) a.QB[c * cs + qb] = q[c].v.y;
        }
      }
    }
    {
      const int kA = P.n.iz + 1 - a.zA0, kB = P.izB + 1 - a.zA0;
      const bool inA = kA >= 0 && kA < a.WA, inB = wb && kB >= 0 && kB < a.WA;
      if (inA || inB) {
        const int64_t qa = (int64_t)(inA ? kA : kB) * nxy + t, qb = (int64_t)(inB ? kB : kA) * nxy + t;
        const int64_t cs = (int64_t)a.WA * nxy;
        f2 q[NA];
#pragma unroll
        for (int c = 0; c < NA; ++c) q[c] = f2(a.QA[c * cs + qa], a.QA[c * cs + qb]);
        G::adj(Ui, q);
        const f2 wq(inA ? a.az2 : 0.f, inB ? a.az2 : 0.f);
#pragma unroll
        for (int c = 0; c < NA; ++c) {
          dj[c] = fma(wq, q[c], dj[c]);
          if (inA) a.QA[c * cs + qa] = q[c].v.x;
          if (inB) a.QA[c * cs + qb] = q[c].v.y;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NA; ++c) e[c] = e[c] + dj[c];
  }
#pragma unroll
  for (int c = 0; c < NA; ++c) {
    float* Ec = a.E + (int64_t)(i * NA + c) * a.g.V;
    Ec[sa] = e[c].v.x;
    if (wb) Ec[sb] = e[c].v.y;
  }
  M un = G::mul(G::expi(e, f2(a.dt)), Ui);
  un = G::reunit(un);
  PairIO<NC>::store(a.Un, i, a.g.V, sa, sb, un, true, wb);
}

// Link i of the two sites (t, iz) and (t, iz + H), 0 <= iz < H.
template <int NC>
__device__ __forceinline__ void step_link_pair(const StepArgs<float>& a, int i, uint32_t t, int iz, int H) {
  constexpr int NA = PairAlg<NC>::G::NA;
  if (t >= (uint32_t)a.g.nxy) return;
  SitePair P;
  P.n = site_nbr_tz(a.g, t, iz);
  P.izB = iz + H;
  // lane B is past the lattice (odd nz) or on the last slice, which has no
  // z link; lane A is never on the last slice (iz < H <= nz - 1)
  P.writeB = P.izB < a.g.nz && !(i == 2 && P.izB == a.g.nz - 1);
  P.dB = P.writeB ? (int64_t)H * a.g.nxy : 0;
  if (!P.writeB) P.izB = iz;
  f2 F[NA];
  pair_force<NC>(a.U, a.g, P, i, a.w, F);
  pair_update<NC>(a, P, i, t, F);
}

}  // namespace glasma
