// Fused leapfrog step with the CPIC hop for one event (the per-link update is
// step_link in step_link.cuh).  The charges live in co-moving windows: a hop
// rewrites each slot in place and the host moves the window origin by one
// slice afterwards, so no slot is touched by two threads.
#include "step_pair.cuh"

namespace glasma {

// One thread per link.  A block is `sites` consecutive transverse sites
// times the three directions (threadIdx.y = direction), so the three link
// updates of a site run together and share the neighbour links in L1;
// blockIdx.y is the z slice.  A thread holds the staple sum and one
// neighbour product at a time and reloads its own link after the staples
// (fewer live registers).  FP32: 6 blocks of 32 sites (96 threads) per SM,
// 18 warps at 96 registers (at most 5 warps on each of the 4 schedulers);
// 15 warps at 126 registers without spills, or 12, were slower.  FP64
// needs twice the registers.
template <typename R> struct StepOcc {
  static constexpr int blocks = 6;
  static constexpr int sites = 32;
};
template <> struct StepOcc<double> {
  static constexpr int blocks = 1;
  static constexpr int sites = 64;
};

template <int NC, typename R>
__global__ void __launch_bounds__(3 * StepOcc<R>::sites, StepOcc<R>::blocks) k_step_leapfrog(StepArgs<R> a) {
  step_link<NC, R>(a, (int)threadIdx.y, blockIdx.x * blockDim.x + threadIdx.x, (int)blockIdx.y + a.zlo);
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
  a.zlo = c->lo;
  const int bs = StepOcc<R>::sites;
  const unsigned ntb = (unsigned)((c->g.nxy + bs - 1) / bs);
  k_step_leapfrog<NC, R><<<dim3(ntb, (unsigned)(c->hi - c->lo)), dim3(bs, 3), 0, c->stream>>>(a);
  return cuda_check(cudaGetLastError(), "k_step_leapfrog launch");
}

// FP32 only: two sites per thread, (t, iz) and (t, iz + H) with
// H = ceil(nz / 2), in the lanes of the packed FP32 instructions; blockIdx.y
// runs over the first H slices.  Two blocks of 192 threads per SM (about
// 170 registers per thread).
template <int NC>
__global__ void __launch_bounds__(192, 2) k_step_pair(StepArgs<float> a, int H) {
  step_link_pair<NC>(a, (int)threadIdx.y, blockIdx.x * blockDim.x + threadIdx.x, (int)blockIdx.y, H);
}

template <int NC>
static int launch_pair_t(glasma_ctx* c, bool hop) {
  StepArgs<float> a;
  a.U = (const float2*)c->U[c->cur];
  a.Un = (float2*)c->U[1 - c->cur];
  a.E = (float*)c->E;
  a.QA = (float*)c->QA;
  a.QB = (float*)c->QB;
  a.g = c->g;
  a.dt = (float)c->p.dt;
  a.w[0] = (float)(2.0 / (c->p.a_t * c->p.a_t));
  a.w[1] = a.w[0];
  a.w[2] = (float)(2.0 / (c->p.a_z * c->p.a_z));
  a.az2 = (float)(c->p.a_z * c->p.a_z);
  a.hop = hop ? 1 : 0;
  a.zA0 = c->zA0;
  a.WA = c->WA;
  a.zB0 = c->zB0;
  a.WB = c->WB;
  a.zlo = 0;
  if (c->slab) return set_error(GLASMA_ERR_INTERNAL, "the paired step kernel does not take slab contexts");
  const int bs = 64;
  const int H = (c->g.nz + 1) / 2;
  const unsigned ntb = (unsigned)((c->g.nxy + bs - 1) / bs);
  k_step_pair<NC><<<dim3(ntb, (unsigned)H), dim3(bs, 3), 0, c->stream>>>(a, H);
  return cuda_check(cudaGetLastError(), "k_step_pair launch");
}

int launch_step_pair(glasma_ctx* c, bool hop) {
  if (c->rs != 4) return set_error(GLASMA_ERR_INTERNAL, "the paired step kernel is FP32 only");
  return c->p.nc == 2 ? launch_pair_t<2>(c, hop) : launch_pair_t<3>(c, hop);
}

int launch_step_leapfrog(glasma_ctx* c, bool hop) {
  if (c->p.nc == 2) return c->rs == 8 ? launch_t<2, double>(c, hop) : launch_t<2, float>(c, hop);
  return c->rs == 8 ? launch_t<3, double>(c, hop) : launch_t<3, float>(c, hop);
}

}  // namespace glasma
