// Rest-frame analysis of sampled T^{mu nu} tables (Sec. 4): the event
// average, the local rest frame of the (t, z) block, sampling on Milne
// coordinates (tau, eta_s) and the Gaussian fit of a rapidity profile.
#include <math.h>

#include <vector>

#include "glasma_internal.cuh"

namespace glasma {

constexpr int kRestOut = 8;  // <eps>, <p_L>, <p_T>, <S_L>, eps_loc, p_L,loc, v_z, valid

// Local rest frame of the block [[eps, S], [S, p_L]] with metric
// diag(+1, -1): the eigenvalues of T^mu_nu = [[eps, -S], [S, -p_L]] are
//   lambda = ((eps - p_L) +- D) / 2,  D^2 = (eps + p_L)^2 - 4 S^2,
// D^2 evaluated as (a - 2S)(a + 2S), a = eps + p_L, to keep its digits when
// the flow is fast.  The eigenvector of lambda has v = S / (p_L + lambda);
// it is timelike (|v| < 1) for the root whose sign is that of a, which
// gives eps_loc, v = 2S / (a +- D), and p_L,loc = -(the other root).  With
// S = 0 the block is already diagonal; with S != 0 and D^2 <= 0 there is no
// timelike eigenvector and the point is marked invalid (NaN results).
__global__ void k_rest_frame(const double* tabs, int n_events, long long n_points, double* out) {
  const double inv = 1.0 / (double)n_events;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_points;
       i += (long long)gridDim.x * blockDim.x) {
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    for (int e = 0; e < n_events; ++e) {
      const double4 v = *reinterpret_cast<const double4*>(tabs + ((long long)e * n_points + i) * 4);
      m[0] += v.x;
      m[1] += v.y;
      m[2] += v.z;
      m[3] += v.w;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) m[c] *= inv;
    const double eps = m[0], pl = m[1], s = m[3];
    double el, pll, vz, valid;
    if (s == 0.0) {
      el = eps;
      pll = pl;
      vz = 0.0;
      valid = 1.0;
    } else {
      const double a = eps + pl;
      const double d2 = (a - 2.0 * s) * (a + 2.0 * s);
      if (d2 > 0.0) {
        const double d = a >= 0.0 ? sqrt(d2) : -sqrt(d2);
        el = 0.5 * ((eps - pl) + d);
        pll = 0.5 * ((pl - eps) + d);
        vz = 2.0 * s / (a + d);
        valid = 1.0;
      } else {
        el = pll = vz = __longlong_as_double(0x7ff8000000000000LL);
        valid = 0.0;
      }
    }
    double* o = out + i * kRestOut;
    o[0] = m[0];
    o[1] = m[1];
    o[2] = m[2];
    o[3] = m[3];
    o[4] = el;
    o[5] = pll;
    o[6] = vz;
    o[7] = valid;
  }
}

// Bilinear interpolation of component `comp` of grid[n_t][nz][stride]
// (point (k, j) at t = t0 + k dts, z = z0 + j az) at (t, z) = (tau cosh eta,
// tau sinh eta) (coords 0) or at (x, y) = (t, z) directly (coords 1); NaN
// outside the grid.
__global__ void k_sample(const double* grid, int n_t, int nz, int stride, int comp, double t0, double dts,
                         double z0, double az, const double* xs, const double* ys, long long n_pts, int coords,
                         double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pts;
       i += (long long)gridDim.x * blockDim.x) {
    double t = xs[i], z = ys[i];
    if (coords == 0) {
      const double tau = t, eta = z;
      t = tau * cosh(eta);
      z = tau * sinh(eta);
    }
    const double ft = (t - t0) / dts, fz = (z - z0) / az;
    double r = __longlong_as_double(0x7ff8000000000000LL);
    if (ft >= 0.0 && ft <= (double)(n_t - 1) && fz >= 0.0 && fz <= (double)(nz - 1)) {
      int k = (int)floor(ft), j = (int)floor(fz);
      if (k > n_t - 2) k = n_t > 1 ? n_t - 2 : 0;
      if (j > nz - 2) j = nz > 1 ? nz - 2 : 0;
      const double wt = ft - k, wz = fz - j;
      const int k1 = n_t > 1 ? k + 1 : k, j1 = nz > 1 ? j + 1 : j;
      auto g = [&](int kk, int jj) { return grid[((long long)kk * nz + jj) * stride + comp]; };
      r = (1.0 - wt) * ((1.0 - wz) * g(k, j) + wz * g(k, j1)) + wt * ((1.0 - wz) * g(k1, j) + wz * g(k1, j1));
    }
    out[i] = r;
  }
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

}  // namespace glasma

using namespace glasma;

extern "C" {

GLASMA_API int glasma_rest_frame(const double* tabs, int n_events, long long n_points, double* out, void* stream) {
  if (!tabs || !out || n_events < 1 || n_points < 0)
    return set_error(GLASMA_ERR_INVALID_ARG, "tabs, out must be device pointers, n_events >= 1, n_points >= 0");
  if (((uintptr_t)tabs & 31) != 0 || ((uintptr_t)out & 7) != 0)
    return set_error(GLASMA_ERR_INVALID_ARG, "tabs must be 32-byte aligned and out 8-byte aligned");
  if (n_points == 0) return GLASMA_OK;
  k_rest_frame<<<grid_for(n_points), 256, 0, (cudaStream_t)stream>>>(tabs, n_events, n_points, out);
  return cuda_check(cudaGetLastError(), "k_rest_frame launch");
}

GLASMA_API int glasma_sample_grid(const double* grid, int n_t, int nz, int stride, int comp, double t0,
                                  double dts, double z0, double az, const double* x, const double* y,
                                  long long n_pts, int coords, double* out, void* stream) {
  if (!grid || !x || !y || !out || n_t < 1 || nz < 1 || stride < 1 || comp < 0 || comp >= stride ||
      !(dts > 0) || !(az > 0) || n_pts < 0 || (coords != 0 && coords != 1))
    return set_error(GLASMA_ERR_INVALID_ARG, "bad grid, spacing, component or coordinate kind");
  if (n_pts == 0) return GLASMA_OK;
  k_sample<<<grid_for(n_pts), 256, 0, (cudaStream_t)stream>>>(grid, n_t, nz, stride, comp, t0, dts, z0, az, x, y,
                                                              n_pts, coords, out);
  return cuda_check(cudaGetLastError(), "k_sample launch");
}

// Weighted least squares of log f = c0 + c1 u + c2 u^2, u = x - xm (xm the
// weighted mean of x, for conditioning), weights f^2 on the squared
// residuals, over the points with f > frac * max f; the 3 x 3 normal
// equations are solved by Gaussian elimination with partial pivoting.
GLASMA_API int glasma_fit_gaussian(const double* x, const double* f, int n, double frac, double* amp, double* mu,
                                   double* sigma) {
  if (!x || !f || n < 3 || !(frac >= 0.0) || !(frac < 1.0))
    return set_error(GLASMA_ERR_INVALID_ARG, "need n >= 3 points and 0 <= frac < 1");
  double fmax = -INFINITY;
  for (int i = 0; i < n; ++i)
    if (isfinite(f[i]) && f[i] > fmax) fmax = f[i];
  if (!(fmax > 0.0)) return set_error(GLASMA_ERR_INVALID_ARG, "profile has no positive value");
  std::vector<int> use;
  double sw = 0.0, swx = 0.0;
  for (int i = 0; i < n; ++i) {
    if (isfinite(f[i]) && isfinite(x[i]) && f[i] > frac * fmax && f[i] > 0.0) {
      use.push_back(i);
      sw += f[i] * f[i];
      swx += f[i] * f[i] * x[i];
    }
  }
  if (use.size() < 3) return set_error(GLASMA_ERR_INVALID_ARG, "fewer than 3 points above the threshold");
  const double xm = swx / sw;
  double A[3][4] = {{0}};
  for (int i : use) {
    const double w = f[i] * f[i], u = x[i] - xm, y = log(f[i]);
    const double b[3] = {1.0, u, u * u};
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) A[r][c] += w * b[r] * b[c];
      A[r][3] += w * b[r] * y;
    }
  }
  for (int c = 0; c < 3; ++c) {
    int p = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
    if (A[p][c] == 0.0) return set_error(GLASMA_ERR_INVALID_ARG, "singular fit (points on fewer than 3 abscissae)");
    if (p != c)
      for (int k = 0; k < 4; ++k) {
        const double t = A[c][k];
        A[c][k] = A[p][k];
        A[p][k] = t;
      }
    for (int r = c + 1; r < 3; ++r) {
      const double m = A[r][c] / A[c][c];
      for (int k = c; k < 4; ++k) A[r][k] -= m * A[c][k];
    }
  }
  double cf[3];
  for (int r = 2; r >= 0; --r) {
    double s = A[r][3];
    for (int k = r + 1; k < 3; ++k) s -= A[r][k] * cf[k];
    cf[r] = s / A[r][r];
  }
  if (!(cf[2] < 0.0)) return set_error(GLASMA_ERR_INVALID_ARG, "profile has no maximum");
  if (sigma) *sigma = sqrt(-1.0 / (2.0 * cf[2]));
  if (mu) *mu = xm - cf[1] / (2.0 * cf[2]);
  if (amp) *amp = exp(cf[0] - cf[1] * cf[1] / (4.0 * cf[2]));
  return GLASMA_OK;
}

}  // extern "C"
