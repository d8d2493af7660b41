// The leapfrog update of one link (Sec. 3, Eqs. lattice_1, lattice_2, the
// NGP hop and its current), shared by the single-event and the batched step
// kernels.
#pragma once
#include "glasma_internal.cuh"

namespace glasma {

template <typename R>
struct StepArgs {
  const typename V2T<R>::T* U;
  typename V2T<R>::T* Un;
  R* E;
  R* QA;
  R* QB;
  Geom g;
  R dt;
  R w[3];   // 2 / a_j^2
  R az2;    // a_z^2
  int hop;
  int zA0, WA, zB0, WB;
  int zlo;  // first slice the launch updates (the grid covers the owned slices)
};

// Steps (1)-(3) below for link i of the site s = iz*nxy + t, given the
// staple force F (Eq. lattice_1 without the dt):
//   (1) on a hop step, for the z link: transport the charge of B at x to
//       x+z (Q' = U_z^dag Q U_z) and the charge of A at x+z to x
//       (Q' = U_z Q U_z^dag) in their co-moving slots, and deposit
//       dt J_z = a_z^2 (Q'_A - Q_B) (the current of the continuity equation
//       with Gauss weights 1/a_i^2);
//   (2) E += dt F (+ dt J on the z link);
//   (3) write exp(i dt E) U to the other link buffer (re-unitarised in FP32).
// Shared by the staple kernel below, the plaquette kernel (k_step_plaq.cu)
// and the staged kernel (k_step_staged.cu), so all apply the same update
// arithmetic.  update_link_ue takes the link U_i(x) and the field
// E_i(t_{n-1/2}) already loaded (Ui, E0); update_link loads them.
template <int NC, typename R>
__device__ __forceinline__ void update_link_ue(const StepArgs<R>& a, int i, uint32_t t, int iz, int64_t s,
                                               const R* F, const typename LinkAlg<NC, R>::M& Ui, const R* E0) {
  typedef LinkAlg<NC, R> G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
  R e[NA];
#pragma unroll
  for (int c = 0; c < NA; ++c) e[c] = E0[c] + a.dt * F[c];
  if (i == 2 && a.hop) {
    R dj[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) dj[c] = R(0);
    const int kb = iz - a.zB0;
    if (kb >= 0 && kb < a.WB) {
      R q[NA];
#pragma unroll
      for (int c = 0; c < NA; ++c) q[c] = a.QB[((int64_t)c * a.WB + kb) * a.g.nxy + t];
#pragma unroll
      for (int c = 0; c < NA; ++c) dj[c] -= a.az2 * q[c];
      G::adj_dag(Ui, q);
#pragma unroll
      for (int c = 0; c < NA; ++c) a.QB[((int64_t)c * a.WB + kb) * a.g.nxy + t] = q[c];
    }
    const int ka = iz + 1 - a.zA0;
    if (ka >= 0 && ka < a.WA) {
      R q[NA];
#pragma unroll
      for (int c = 0; c < NA; ++c) q[c] = a.QA[((int64_t)c * a.WA + ka) * a.g.nxy + t];
      G::adj(Ui, q);
#pragma unroll
      for (int c = 0; c < NA; ++c) {
        dj[c] += a.az2 * q[c];
        a.QA[((int64_t)c * a.WA + ka) * a.g.nxy + t] = q[c];
      }
    }
#pragma unroll
    for (int c = 0; c < NA; ++c) e[c] += dj[c];
  }
#pragma unroll
  for (int c = 0; c < NA; ++c) a.E[(int64_t)(i * NA + c) * a.g.V + s] = e[c];
  M un = G::mul(G::expi(e, a.dt), Ui);
  if (sizeof(R) == 4) un = G::reunit(un);
  LinkIO<NC, R>::template store<R>(a.Un, i, a.g.V, s, un);
}

template <int NC, typename R>
__device__ __forceinline__ void update_link(const StepArgs<R>& a, int i, uint32_t t, int iz, int64_t s,
                                            const R* F) {
  constexpr int NA = LinkAlg<NC, R>::NA;
  const typename LinkAlg<NC, R>::M Ui = LinkIO<NC, R>::template load<R>(a.U, i, a.g.V, s);
  R E0[NA];
#pragma unroll
  for (int c = 0; c < NA; ++c) E0[c] = a.E[(int64_t)(i * NA + c) * a.g.V + s];
  update_link_ue<NC, R>(a, i, t, iz, s, F, Ui, E0);
}

// Link i of the site with transverse index t on slice iz, its force from
// the four staples (link_force_staple); the z link of the last slice does
// not exist.
template <int NC, typename R>
__device__ __forceinline__ void step_link(const StepArgs<R>& a, int i, uint32_t t, int iz) {
  constexpr int NA = LinkAlg<NC, R>::NA;
  if (t >= (uint32_t)a.g.nxy) return;
  if (i == 2 && iz == a.g.nz - 1) return;  // no z link on the last slice
  const SiteNbr n = site_nbr_tz(a.g, t, iz);
  R F[NA];
  link_force_staple<NC, R, R>(a.U, a.g, n, i, a.w, F);
  update_link<NC, R>(a, i, t, iz, n.s, F);
}

}  // namespace glasma
