// Gauss-law residual over caller-owned device fields that allocates no
// device memory: its scratch is a fixed array in this file (see
// glasma_gauss_residual_static in glasma.h).
#include "glasma_internal.cuh"

namespace glasma {

// Capacity of the scratch below: one row of partials per z slice.
constexpr int kStaticMaxSlices = 8192;
constexpr int kStaticThreads = 256;

// Per-slice partials (max |G|, sum G^2, max |rho|, non-finite count) and the
// folded result.  Every GPU that loads the library holds these 256 KB until
// the process exits.  Each call overwrites every row it reads back, so no
// part of the array has to start at zero.
static __device__ __align__(256) double g_gauss_scratch[kStaticMaxSlices * 4 + 8];

struct StaticGaussArgs {
  const void* U;
  const void* E;
  const void* QA;
  const void* QB;
  Geom g;
  double ia2[3];
  int zA0, WA, zB0, WB;
  double* scratch;  // device address of g_gauss_scratch
};

__device__ __forceinline__ void static_block_reduce(double (*sh)[kStaticThreads], double* v) {
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) sh[k][t] = v[k];
  __syncthreads();
  for (int w = kStaticThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
      sh[0][t] = fmax(sh[0][t], sh[0][t + w]);
      sh[1][t] = sh[1][t] + sh[1][t + w];
      sh[2][t] = fmax(sh[2][t], sh[2][t + w]);
      sh[3][t] = sh[3][t] + sh[3][t + w];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = sh[k][0];
}

// One block per z slice: residual of Eq. gauss in FP64 for each site of
// the slice, reduced to one row of partials.
template <int NC, typename R>
__global__ void __launch_bounds__(kStaticThreads) k_gauss_static_slices(StaticGaussArgs a) {
  typedef Group<NC, double> G;
  constexpr int NA = G::NA;
  typedef typename V2T<R>::T V2;
  const V2* U = (const V2*)a.U;
  const R* E = (const R*)a.E;
  const R* QA = (const R*)a.QA;
  const R* QB = (const R*)a.QB;
  __shared__ double sh[4][kStaticThreads];
  const int iz = blockIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < a.g.nxy; t += blockDim.x) {
    const int64_t s = (int64_t)iz * a.g.nxy + t;
    SiteNbr n = site_nbr(a.g, s);
    double gv[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) gv[c] = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int c = 0; c < NA; ++c) gv[c] += a.ia2[i] * (double)E[(int64_t)(i * NA + c) * a.g.V + s];
      if (i == 2 && iz == 0) continue;
      double q[NA];
#pragma unroll
      for (int c = 0; c < NA; ++c) q[c] = (double)E[(int64_t)(i * NA + c) * a.g.V + n.m[i]];
      typename G::M um = LinkIO<NC, R>::template load<double>(U, i, a.g.V, n.m[i]);
      G::adj_dag(um, q);
#pragma unroll
      for (int c = 0; c < NA; ++c) gv[c] -= a.ia2[i] * q[c];
    }
    const int ka = iz - a.zA0, kb = iz - a.zB0;
#pragma unroll
    for (int c = 0; c < NA; ++c) {
      double rho = 0.0;
      if (ka >= 0 && ka < a.WA) rho += (double)QA[((int64_t)c * a.WA + ka) * a.g.nxy + t];
      if (kb >= 0 && kb < a.WB) rho += (double)QB[((int64_t)c * a.WB + kb) * a.g.nxy + t];
      const double r = gv[c] - rho;
      if (!isfinite(r)) v[3] += 1.0;
      v[0] = fmax(v[0], fabs(r));
      v[1] += r * r;
      v[2] = fmax(v[2], fabs(rho));
    }
  }
  static_block_reduce(sh, v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) a.scratch[iz * 4 + k] = v[k];
}

// Fold the nz rows in a fixed order into scratch[kStaticMaxSlices*4 ...].
__global__ void __launch_bounds__(kStaticThreads) k_gauss_static_fold(double* scratch, int rows) {
  __shared__ double sh[4][kStaticThreads];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    v[0] = fmax(v[0], scratch[r * 4 + 0]);
    v[1] += scratch[r * 4 + 1];
    v[2] = fmax(v[2], scratch[r * 4 + 2]);
    v[3] += scratch[r * 4 + 3];
  }
  static_block_reduce(sh, v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) scratch[kStaticMaxSlices * 4 + k] = v[k];
}

// Device address of the scratch array on the current device
// (cudaGetSymbolAddress; the name itself is only a host-side stand-in and
// must never be passed to a kernel).  It is looked up on every call, so a
// module reloaded after a device reset is never addressed through a stale
// pointer.  The same call makes sure every kernel of this file is loaded:
// with lazy module loading the first call on a device is the one that loads
// this code and its array, so no later call (of any N_c or precision) loads
// anything.
static int static_scratch(double** out) {
  void* p = nullptr;
  int st = cuda_check(cudaGetSymbolAddress(&p, g_gauss_scratch), "cudaGetSymbolAddress(g_gauss_scratch)");
  if (st) return st;
  const void* fns[5] = {(const void*)k_gauss_static_slices<2, double>, (const void*)k_gauss_static_slices<2, float>,
                        (const void*)k_gauss_static_slices<3, double>, (const void*)k_gauss_static_slices<3, float>,
                        (const void*)k_gauss_static_fold};
  for (int k = 0; k < 5 && !st; ++k) {
    cudaFuncAttributes fa;
    st = cuda_check(cudaFuncGetAttributes(&fa, fns[k]), "cudaFuncGetAttributes (static Gauss kernels)");
  }
  if (st) return st;
  *out = (double*)p;
  return GLASMA_OK;
}

template <int NC, typename R>
static int static_gauss_t(StaticGaussArgs& a, cudaStream_t stream, double* h4) {
  k_gauss_static_slices<NC, R><<<a.g.nz, kStaticThreads, 0, stream>>>(a);
  int st = cuda_check(cudaGetLastError(), "k_gauss_static_slices launch");
  if (st) return st;
  k_gauss_static_fold<<<1, kStaticThreads, 0, stream>>>(a.scratch, a.g.nz);
  st = cuda_check(cudaGetLastError(), "k_gauss_static_fold launch");
  if (st) return st;
  st = cuda_check(cudaMemcpyAsync(h4, a.scratch + kStaticMaxSlices * 4, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                  stream),
                  "static Gauss readback");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(stream), "static Gauss sync");
}

}  // namespace glasma

using namespace glasma;

extern "C" GLASMA_API int glasma_gauss_residual_static(int nc, int precision, int nz, int ny, int nx, double a_t,
                                                       double a_z, const void* U, const void* E, const void* QA,
                                                       int zA0, int WA, const void* QB, int zB0, int WB,
                                                       void* stream, double* max_abs, double* rms,
                                                       double* rho_max) {
  if (nz > kStaticMaxSlices)
    return set_error(GLASMA_ERR_INVALID_ARG,
                     "glasma_gauss_residual_static: nz exceeds the fixed scratch capacity of 8192 z slices");
  if (nc != 2 && nc != 3) return set_error(GLASMA_ERR_INVALID_ARG, "nc must be 2 or 3");
  if (precision != GLASMA_FP64 && precision != GLASMA_FP32)
    return set_error(GLASMA_ERR_INVALID_ARG, "precision must be GLASMA_FP64 or GLASMA_FP32");
  if (nz < 1 || nx < 1 || ny < 1) return set_error(GLASMA_ERR_INVALID_ARG, "need nz, nx, ny >= 1");
  if (!(a_t > 0) || !(a_z > 0)) return set_error(GLASMA_ERR_INVALID_ARG, "a_t, a_z must be positive");
  if (!U || !E) return set_error(GLASMA_ERR_INVALID_ARG, "U and E are required");
  if (((uintptr_t)U & 15) != 0) return set_error(GLASMA_ERR_INVALID_ARG, "U must be 16-byte aligned");
  if (WA < 0 || WB < 0 || (WA > 0 && (!QA || zA0 < 0 || zA0 + WA > nz)) ||
      (WB > 0 && (!QB || zB0 < 0 || zB0 + WB > nz)))
    return set_error(GLASMA_ERR_INVALID_ARG, "charge window outside the lattice or missing");
  double* scratch = nullptr;
  int st = static_scratch(&scratch);
  if (st) return st;
  StaticGaussArgs a;
  a.U = U;
  a.E = E;
  a.QA = QA;
  a.QB = QB;
  a.g.nx = nx;
  a.g.ny = ny;
  a.g.nz = nz;
  a.g.nxy = (int64_t)nx * ny;
  a.g.V = a.g.nxy * nz;
  a.ia2[0] = a.ia2[1] = 1.0 / (a_t * a_t);
  a.ia2[2] = 1.0 / (a_z * a_z);
  a.zA0 = zA0;
  a.WA = WA;
  a.zB0 = zB0;
  a.WB = WB;
  a.scratch = scratch;
  double h[4];
  cudaStream_t s = (cudaStream_t)stream;
  if (nc == 2)
    st = precision == GLASMA_FP64 ? static_gauss_t<2, double>(a, s, h) : static_gauss_t<2, float>(a, s, h);
  else
    st = precision == GLASMA_FP64 ? static_gauss_t<3, double>(a, s, h) : static_gauss_t<3, float>(a, s, h);
  if (st) return st;
  if (max_abs) *max_abs = h[0];
  if (rms) *rms = sqrt(h[1] / ((double)a.g.V * (nc * nc - 1)));
  if (rho_max) *rho_max = h[2];
  if (h[3] != 0.0) return set_error(GLASMA_ERR_NONFINITE, "Gauss residual met a non-finite value");
  return GLASMA_OK;
}
