// Fused leapfrog step with the CPIC hop (Sec. 3, Eqs. lattice_1, lattice_2,
// continuity and the NGP parallel transport).
//
// One thread per link.  For its link it
//   (1) on a hop step and for the z link: transports the charge of B that
//       sits at x to x+z (Q' = U_z^dag Q U_z) and the charge of A that sits
//       at x+z to x (Q' = U_z Q U_z^dag), and deposits dt J_z =
//       a_z^2 (Q'_A - Q_B) (the current that satisfies the continuity
//       equation with Gauss weights 1/a_i^2);
//   (2) adds dt times the plaquette force to E;
//   (3) writes exp(i dt E) U to the other link buffer (re-unitarised in FP32).
// The charges live in co-moving windows: a hop rewrites each slot in place
// and the host moves the window origin by one slice afterwards, so no slot
// is touched by two threads.
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
};

// One thread per link.  A block is 64 consecutive transverse sites times the
// three directions (threadIdx.y = direction), so the three link updates of a
// site run together and share the neighbour links in L1; blockIdx.y is the
// z slice.  A thread holds the staple sum and one neighbour product at a
// time and reloads its own link after the staples (fewer live registers).
// FP32: 3 blocks of 192 threads per SM; FP64 needs twice the registers.
template <typename R> struct StepOcc { static constexpr int blocks = 3; };
template <> struct StepOcc<double> { static constexpr int blocks = 1; };

template <int NC, typename R>
__global__ void __launch_bounds__(192, StepOcc<R>::blocks) k_step_leapfrog(StepArgs<R> a) {
  typedef LinkAlg<NC, R> G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
  const int i = (int)threadIdx.y;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;  // transverse index
  const int iz = (int)blockIdx.y;
  if (t >= (uint32_t)a.g.nxy) return;
  if (i == 2 && iz == a.g.nz - 1) return;  // no z link on the last slice
  const SiteNbr n = site_nbr_tz(a.g, t, iz);
  const int64_t s = n.s;
  R F[NA];
  link_force_staple<NC, R, R>(a.U, a.g, n, i, a.w, F);
  const M Ui = LinkIO<NC, R>::template load<R>(a.U, i, a.g.V, s);
  R e[NA];
#pragma unroll
  for (int c = 0; c < NA; ++c) e[c] = a.E[(int64_t)(i * NA + c) * a.g.V + s] + a.dt * F[c];
  if (i == 2 && a.hop) {
    R dj[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) dj[c] = R(0);
    const int kb = n.iz - a.zB0;
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
    const int ka = n.iz + 1 - a.zA0;
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
static int launch_t(glasma_ctx* c, bool hop) {
  StepArgs<R> a;
  a.U = (const typename V2T<R>::T*)c->U[c->cur];
  a.Un = (typename V2T<R>::T*)c->U[1 - c->cur];
  a.E = (R*)c->E;
  a.QA = (R*)c->QA;
  a.QB = (R*)c->QB;
  a.g = c->g;
  a.dt = (R)c->p.dt;
  a.w[0] = (R)(2.0 / (c->p.a_t * c->p.a_t));
  a.w[1] = a.w[0];
  a.w[2] = (R)(2.0 / (c->p.a_z * c->p.a_z));
  a.az2 = (R)(c->p.a_z * c->p.a_z);
  a.hop = hop ? 1 : 0;
  a.zA0 = c->zA0;
  a.WA = c->WA;
  a.zB0 = c->zB0;
  a.WB = c->WB;
  const int bs = 64;
  const unsigned ntb = (unsigned)((c->g.nxy + bs - 1) / bs);
  k_step_leapfrog<NC, R><<<dim3(ntb, (unsigned)c->g.nz), dim3(bs, 3), 0, c->stream>>>(a);
  return cuda_check(cudaGetLastError(), "k_step_leapfrog launch");
}

int launch_step_leapfrog(glasma_ctx* c, bool hop) {
  if (c->p.nc == 2) return c->rs == 8 ? launch_t<2, double>(c, hop) : launch_t<2, float>(c, hop);
  return c->rs == 8 ? launch_t<3, double>(c, hop) : launch_t<3, float>(c, hop);
}

}  // namespace glasma
