// Fused leapfrog step with the CPIC hop for one event (the per-link update is
// step_link in step_link.cuh).  The charges live in co-moving windows: a hop
// rewrites each slot in place and the host moves the window origin by one
// slice afterwards, so no slot is touched by two threads.
#include "step_link.cuh"

namespace glasma {

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
  step_link<NC, R>(a, (int)threadIdx.y, blockIdx.x * blockDim.x + threadIdx.x, (int)blockIdx.y);
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
