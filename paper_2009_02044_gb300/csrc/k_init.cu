// MV initial state on the device (Sec. 2 MV model; Sec. 3 Eqs. single_sheet,
// 3d_colorfield_1, 3d_colorfield_2; Sec. 4 Gaussian profile), all in FP64:
//   rho_N^a(x_T)   Philox4x32-10 + Box-Muller, or copied from the host
//   phi_N          (-Delta_T + m^2)^{-1} rho_N by separable DFTs
//   Lambda_N(z,t)  cumulative truncated Gaussian profile (erf)
//   U_i(x; t)      V_A(x) V_A^dag(x+i) V_B(x) V_B^dag(x+i), U_z = 1,
//                  V_N^dag = exp(i Lambda_N phi_N), at t0 and t0 - dt
//   E_i            -i log(U(t0) U^dag(t0 - dt)) / dt, 0 where equal
//   rho(x)         discrete Gauss divergence of the stored state
//   Q_A, Q_B       rho on either side of the box centre, cut to windows
#include <vector>

#include "glasma_internal.cuh"
#include "init_math.cuh"

namespace glasma {

// rho[(s*2 + N)*na + a][y][x] for S sheets; counter (x, y, a, N + 2 s)
__global__ void k_philox_rho(double* rho, int na, int nx, int ny, int S, unsigned long long seed, double g2mu) {
  const int64_t total = (int64_t)2 * S * na * nx * ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    int64_t r = i / nx;
    const int y = (int)(r % ny);
    r /= ny;
    const int a = (int)(r % na);
    const int N = (int)(r / na);  // N + 2 s
    uint32_t c[4] = {(uint32_t)x, (uint32_t)y, (uint32_t)a, (uint32_t)N};
    philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
    const double u1 = u53(c[0], c[1]), u2 = u53(c[2], c[3]);
    rho[i] = g2mu * (sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
  }
}

// One DFT pass along x (axis 0) or y (axis 1) of F complex [ny][nx] fields:
// out_k = sum_m in_m exp(sign 2 pi i k m / n).
__global__ void k_dft(const double2* in, double2* out, int F, int ny, int nx, int axis, int sign) {
  const int64_t total = (int64_t)F * nx * ny;
  const int n = axis == 0 ? nx : ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    int64_t r = i / nx;
    const int y = (int)(r % ny);
    const int64_t f = r / ny;
    const int k = axis == 0 ? x : y;
    double re = 0.0, im = 0.0;
    for (int m = 0; m < n; ++m) {
      const int64_t src = axis == 0 ? (f * ny + y) * nx + m : (f * ny + m) * nx + x;
      const double2 v = in[src];
      const int km = (int)(((int64_t)k * m) % n);
      double s, c;
      sincospi(2.0 * (double)km / (double)n, &s, &c);
      s *= sign;
      re += v.x * c - v.y * s;
      im += v.x * s + v.y * c;
    }
    out[i] = make_double2(re, im);
  }
}

__global__ void k_real_to_cplx(const double* in, double2* out, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_double2(in[i], 0.0);
}

// multiply by 1 / (k^2 + m^2), k^2 = 4/a^2 [sin^2(pi kx/nx) + sin^2(pi ky/ny)]
__global__ void k_poisson_kernel(double2* f, int F, int ny, int nx, double a_t, double m2, double uv2) {
  const int64_t total = (int64_t)F * nx * ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % nx);
    const int ky = (int)((i / nx) % ny);
    const double sx = sinpi((double)kx / nx), sy = sinpi((double)ky / ny);
    const double k2 = 4.0 / (a_t * a_t) * (sy * sy) + 4.0 / (a_t * a_t) * (sx * sx);
    double kern = 1.0 / (k2 + m2);
    if (uv2 > 0.0 && k2 > uv2) kern = 0.0;
    f[i] = make_double2(f[i].x * kern, f[i].y * kern);
  }
}

__global__ void k_cplx_real_scaled(const double2* in, double* out, int64_t total, double scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i].x * scale;
}

// lam[(t*2 + N)*nz + iz], t = 0: t0, 1: t0 - dt; N = 0: A, 1: B
// (iz is local: the slice's global index is iz + zoff)
__global__ void k_profile(double* lam, int nz, int zoff, double a_z, double sigma, double zA0, double zB0,
                          double dt) {
  const double erf4 = erf(2.0 * 1.4142135623730950488);  // erf(4 / sqrt 2)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * nz; i += gridDim.x * blockDim.x) {
    const int iz = i % nz, tn = i / nz, N = tn % 2, t = tn / 2;
    const double z = (iz + zoff) * a_z;
    const double zn = N == 0 ? zA0 + (t ? dt : 0.0) : zB0 - (t ? dt : 0.0);
    const double u = (z - zn) / sigma;
    const double uc = fmin(fmax(u, -4.0), 4.0);
    const double ef = erf(uc / 1.4142135623730950488);
    double L;
    if (N == 1) {  // B, moving +z: 1 behind (low z), 0 ahead
      L = (erf4 - ef) / (2.0 * erf4);
      if (u >= 4.0) L = 0.0;
      if (u <= -4.0) L = 1.0;
    } else {  // A, moving -z: 1 behind (high z), 0 ahead
      L = (ef + erf4) / (2.0 * erf4);
      if (u <= -4.0) L = 0.0;
      if (u >= 4.0) L = 1.0;
    }
    lam[i] = L;
  }
}

// V_N^dagger at transverse site t for the cumulative profile value lam.
// One sheet: exp(i lam phi_N).  S sheets (phi[(s*2 + N)*na + a][t]): the
// path-ordered exp(i L_{S-1} phi_{S-1,N}) ... exp(i L_0 phi_{0,N}) with
// L_s = clip(S lam - s, 0, 1), sheet 0 (the leading slab) acting first.
template <int NC>
GL_HD typename Group<NC, double>::M wilson_dag(const double* phi, int N, int na, int64_t nxy, int64_t t, double lam,
                                               int S = 1, const typename Group<NC, double>::M* full = nullptr) {
  typedef Group<NC, double> G;
  double v[G::NA];
  if (S <= 1) {
    if (lam == 0.0) return G::ident();
    if (lam == 1.0 && full) return full[(int64_t)N * nxy + t];  // behind the nucleus: exp(i phi), tabulated
    for (int a = 0; a < G::NA; ++a) v[a] = phi[((int64_t)N * na + a) * nxy + t];
    return G::expi(v, lam);
  }
  typename G::M m = G::ident();
  bool first = true;
  for (int s = 0; s < S; ++s) {
    double ls = (double)S * lam - (double)s;
    ls = ls < 0.0 ? 0.0 : (ls > 1.0 ? 1.0 : ls);
    typename G::M f;
    if (ls == 0.0) {
      f = G::ident();
    } else {
      for (int a = 0; a < G::NA; ++a) v[a] = phi[((int64_t)(s * 2 + N) * na + a) * nxy + t];
      f = G::expi(v, ls);
    }
    m = first ? f : G::mul(f, m);
    first = false;
  }
  return m;
}

template <int NC>
GL_HD bool group_log(const typename Group<NC, double>::M& W, double* h);
template <>
GL_HD bool group_log<2>(const Group<2, double>::M& W, double* h) { return log_su2(W, h); }
template <>
GL_HD bool group_log<3>(const Group<3, double>::M& W, double* h) { return log_su3(W, h); }

template <int NC>
GL_HD bool same(const typename Group<NC, double>::M& a, const typename Group<NC, double>::M& b) {
  const double* pa = (const double*)&a;
  const double* pb = (const double*)&b;
  for (int k = 0; k < (int)(sizeof(a) / sizeof(double)); ++k)
    if (pa[k] != pb[k]) return false;
  return true;
}

// exp(i phi_N(x_T)) for every transverse site, the Wilson line of all the
// slices a single-sheet nucleus has fully passed (Lambda = 1), computed once.
template <int NC>
__global__ void k_wilson_full(const double* phi, typename Group<NC, double>::M* full, int64_t nxy) {
  typedef Group<NC, double> G;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * nxy; i += (int64_t)gridDim.x * blockDim.x) {
    const int N = (int)(i / nxy);
    const int64_t t = i - (int64_t)N * nxy;
    double v[G::NA];
    for (int a = 0; a < G::NA; ++a) v[a] = phi[((int64_t)N * G::NA + a) * nxy + t];
    full[i] = G::expi(v, 1.0);
  }
}

template <int NC, typename R>
__global__ void k_init_links(const double* phi, const double* lam, typename V2T<R>::T* U0,
                             typename V2T<R>::T* U1, typename V2T<R>::T* Uprev, R* E, Geom g, double dt,
                             int* flag, int S, const typename Group<NC, double>::M* full) {
  typedef Group<NC, double> G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += (int64_t)gridDim.x * blockDim.x) {
    SiteNbr n = site_nbr(g, s);
    const int64_t t0 = s % g.nxy;
    const int64_t tx = n.p[0] % g.nxy, ty = n.p[1] % g.nxy;
    M u[2][2];  // [time][direction]
    // A nucleus whose Lambda is 0 on this slice (ahead of it) contributes
    // the identity, and a slice whose Lambdas are the same at t0 and
    // t0 - dt has the same links at both times (E = 0 there).  Before the
    // collision at most one nucleus has Lambda > 0 on a slice, so most
    // slices need one product per link.
    const double lt[2][2] = {{lam[0 * g.nz + n.iz], lam[1 * g.nz + n.iz]},
                             {lam[2 * g.nz + n.iz], lam[3 * g.nz + n.iz]}};
    const bool moving = lt[0][0] != lt[1][0] || lt[0][1] != lt[1][1];
    for (int t = 0; t < (moving ? 2 : 1); ++t) {
      const double la = lt[t][0], lb = lt[t][1];
      const bool ha = la != 0.0, hb = lb != 0.0;
      M vda = G::ident(), vdb = G::ident();
      if (ha) vda = wilson_dag<NC>(phi, 0, NA, g.nxy, t0, la, S, full);
      if (hb) vdb = wilson_dag<NC>(phi, 1, NA, g.nxy, t0, lb, S, full);
      for (int i = 0; i < 2; ++i) {
        const int64_t tn = i == 0 ? tx : ty;
        M m = G::ident();
        if (ha) m = G::d_mul(vda, wilson_dag<NC>(phi, 0, NA, g.nxy, tn, la, S, full));  // V_A(x) V_A^dag(x+i)
        if (hb) {
          const M ub = G::d_mul(vdb, wilson_dag<NC>(phi, 1, NA, g.nxy, tn, lb, S, full));
          m = ha ? G::mul(m, ub) : ub;
        }
        u[t][i] = m;
      }
    }
    if (!moving) {
      u[1][0] = u[0][0];
      u[1][1] = u[0][1];
    }
    for (int i = 0; i < 2; ++i) {
      double h[NA];
      if (same<NC>(u[0][i], u[1][i])) {
        for (int a = 0; a < NA; ++a) h[a] = 0.0;
      } else {
        M w = G::mul_d(u[0][i], u[1][i]);
        if (!group_log<NC>(w, h)) atomicOr(flag, 1);
      }
      for (int a = 0; a < NA; ++a) E[(int64_t)(i * NA + a) * g.V + s] = (R)(h[a] / dt);
      LinkIO<NC, R>::template store<double>(U0, i, g.V, s, u[0][i]);
      LinkIO<NC, R>::template store<double>(U1, i, g.V, s, u[0][i]);
      if (Uprev) LinkIO<NC, R>::template store<double>(Uprev, i, g.V, s, u[1][i]);
    }
    for (int a = 0; a < NA; ++a) E[(int64_t)(2 * NA + a) * g.V + s] = (R)0;
    M one = G::ident();
    LinkIO<NC, R>::template store<double>(U0, 2, g.V, s, one);
    LinkIO<NC, R>::template store<double>(U1, 2, g.V, s, one);
    if (Uprev) LinkIO<NC, R>::template store<double>(Uprev, 2, g.V, s, one);
  }
}

// rho(x) = sum_i [E_i(x) - U_i^dag(x-i) E_i(x-i) U_i(x-i)] / a_i^2 of the
// stored state, in FP64; one block per z slice also records max |rho|.
template <int NC, typename R>
__global__ void __launch_bounds__(256) k_divergence(const typename V2T<R>::T* U, const R* E, Geom g, double ia2t,
                                                    double ia2z, double* rho3, double* slice_max) {
  typedef Group<NC, double> G;
  constexpr int NA = G::NA;
  __shared__ double sh[256];
  const int iz = blockIdx.x;
  double mx = 0.0;
  for (int t = threadIdx.x; t < g.nxy; t += blockDim.x) {
    const int64_t s = (int64_t)iz * g.nxy + t;
    SiteNbr n = site_nbr(g, s);
    double dv[NA];
    for (int c = 0; c < NA; ++c) dv[c] = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double w = i == 2 ? ia2z : ia2t;
      for (int c = 0; c < NA; ++c) dv[c] += w * (double)E[(int64_t)(i * NA + c) * g.V + s];
      if (i == 2 && iz == 0) continue;
      double q[NA];
      bool nz = false;
      for (int c = 0; c < NA; ++c) {
        q[c] = (double)E[(int64_t)(i * NA + c) * g.V + n.m[i]];
        nz = nz || q[c] != 0.0;
      }
      if (!nz) continue;  // the transported field is zero (E vanishes off the nuclei)
      typename G::M um = LinkIO<NC, R>::template load<double>(U, i, g.V, n.m[i]);
      G::adj_dag(um, q);
      for (int c = 0; c < NA; ++c) dv[c] -= w * q[c];
    }
    for (int c = 0; c < NA; ++c) {
      rho3[(int64_t)c * g.V + s] = dv[c];
      mx = fmax(mx, fabs(dv[c]));
    }
  }
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) slice_max[iz] = sh[0];
}

template <typename R>
__global__ void k_fill_window(const double* rho3, R* Q, int na, int z0, int W, Geom g) {
  const int64_t total = (int64_t)na * W * g.nxy;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i % g.nxy;
    const int64_t r = i / g.nxy;
    const int w = (int)(r % W);
    const int c = (int)(r / W);
    Q[i] = (R)rho3[(int64_t)c * g.V + (int64_t)(z0 + w) * g.nxy + t];
  }
}

static unsigned grid_for(int64_t n, int bs = 256) {
  int64_t nb = (n + bs - 1) / bs;
  if (nb > 152 * 32) nb = 152 * 32;
  if (nb < 1) nb = 1;
  return (unsigned)nb;
}

template <int NC, typename R>
static int init_t(glasma_ctx* c, const double* rho_host) {
  const glasma_params& p = c->p;
  const int na = c->na;
  const int64_t nxy = c->g.nxy, V = c->g.V;
  const int S = p.n_sheets > 1 ? p.n_sheets : 1;
  const int F = 2 * S * na;
  int st;
  // scratch: rho/phi (real), two complex work arrays, lambda table, rho3, slice max, flag
  double* rho = (double*)ctx_alloc(c, sizeof(double) * F * nxy);
  double2* w0 = (double2*)ctx_alloc(c, sizeof(double2) * F * nxy);
  double2* w1 = (double2*)ctx_alloc(c, sizeof(double2) * F * nxy);
  double* lam = (double*)ctx_alloc(c, sizeof(double) * 4 * p.nz);
  double* rho3 = (double*)ctx_alloc(c, sizeof(double) * na * V);
  double* smax = (double*)ctx_alloc(c, sizeof(double) * p.nz);
  if (!rho || !w0 || !w1 || !lam || !rho3 || !smax) return set_error(GLASMA_ERR_OOM, "init scratch allocation failed");
  if (rho_host) {
    st = cuda_check(cudaMemcpyAsync(rho, rho_host, sizeof(double) * F * nxy, cudaMemcpyHostToDevice, c->stream),
                    "rho upload");
    if (st) return st;
  } else {
    k_philox_rho<<<grid_for(F * nxy), 256, 0, c->stream>>>(rho, na, p.nx, p.ny, S, p.seed,
                                                            S > 1 ? p.g2mu / sqrt((double)S) : p.g2mu);
  }
  // Poisson: forward DFT x, y; kernel; inverse y, x; real part / (nx ny)
  k_real_to_cplx<<<grid_for(F * nxy), 256, 0, c->stream>>>(rho, w0, F * nxy);
  k_dft<<<grid_for(F * nxy), 256, 0, c->stream>>>(w0, w1, F, p.ny, p.nx, 0, -1);
  k_dft<<<grid_for(F * nxy), 256, 0, c->stream>>>(w1, w0, F, p.ny, p.nx, 1, -1);
  k_poisson_kernel<<<grid_for(F * nxy), 256, 0, c->stream>>>(w0, F, p.ny, p.nx, p.a_t, p.m_ir * p.m_ir,
                                                               p.uv_cutoff > 0 ? p.uv_cutoff * p.uv_cutoff : 0.0);
  k_dft<<<grid_for(F * nxy), 256, 0, c->stream>>>(w0, w1, F, p.ny, p.nx, 1, +1);
  k_dft<<<grid_for(F * nxy), 256, 0, c->stream>>>(w1, w0, F, p.ny, p.nx, 0, +1);
  k_cplx_real_scaled<<<grid_for(F * nxy), 256, 0, c->stream>>>(w0, rho, F * nxy, 1.0 / (double)nxy);  // rho <- phi
  // nucleus centres at t0 (box centre +- d) in global z (a slab's local
  // slice 0 is global slice zoff)
  const double zc = c->nz_glob * p.a_z / 2.0;
  const double d = p.z_offset > 0 ? p.z_offset : (ceil(4.0 * p.sigma_l / p.a_z) + 2.0) * p.a_z;
  k_profile<<<grid_for(4 * p.nz), 256, 0, c->stream>>>(lam, p.nz, c->zoff, p.a_z, p.sigma_l, zc + d, zc - d, p.dt);
  cudaMemsetAsync(c->dflag, 0, sizeof(int) * 8, c->stream);
  typedef typename Group<NC, double>::M MD;
  MD* full = nullptr;
  if (S <= 1) {
    full = (MD*)ctx_alloc(c, sizeof(MD) * 2 * nxy);
    if (!full) return set_error(GLASMA_ERR_OOM, "init scratch allocation failed");
    k_wilson_full<NC><<<grid_for(2 * nxy), 256, 0, c->stream>>>(rho, full, nxy);
  }
  k_init_links<NC, R><<<grid_for(V, 128), 128, 0, c->stream>>>(
      rho, lam, (typename V2T<R>::T*)c->U[0], (typename V2T<R>::T*)c->U[1], (typename V2T<R>::T*)c->Uprev,
      (R*)c->E, c->g, p.dt, c->dflag, S, full);
  k_divergence<NC, R><<<p.nz, 256, 0, c->stream>>>((const typename V2T<R>::T*)c->U[0], (const R*)c->E, c->g,
                                                  1.0 / (p.a_t * p.a_t), 1.0 / (p.a_z * p.a_z), rho3, smax);
  st = cuda_check(cudaGetLastError(), "init kernels");
  if (st) return st;
  std::vector<double> hmax(p.nz);
  int hflag = 0;
  st = cuda_check(cudaMemcpyAsync(hmax.data(), smax, sizeof(double) * p.nz, cudaMemcpyDeviceToHost, c->stream),
                  "slice max readback");
  if (st) return st;
  st = cuda_check(cudaMemcpyAsync(&hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag");
  if (st) return st;
  st = cuda_check(cudaStreamSynchronize(c->stream), "init sync");
  if (st) return st;
  if (hflag) return set_error(GLASMA_ERR_INVALID_ARG, "init: link change per step too large for the group log");
  // windows: A on slices above the centre, B below; none at the centre
  // (only the owned slices: a slab's halo slices carry no charge of their
  // own, and the divergence of its lower halo lacks the slice below)
  int alo = -1, ahi = -1, blo = -1, bhi = -1;
  for (int iz = c->lo; iz < c->hi; ++iz) {
    if (!(hmax[iz] == hmax[iz])) return set_error(GLASMA_ERR_NONFINITE, "init: non-finite charge density");
    if (hmax[iz] == 0.0) continue;
    const double z = (iz + c->zoff) * p.a_z;
    if (z > zc) {
      if (alo < 0) alo = iz;
      ahi = iz;
    } else if (z < zc) {
      if (blo < 0) blo = iz;
      bhi = iz;
    } else {
      return set_error(GLASMA_ERR_INTERNAL, "init: charge at the box centre");
    }
  }
  c->zA0 = alo < 0 ? 0 : alo;
  c->WA = alo < 0 ? 0 : ahi - alo + 1;
  c->zB0 = blo < 0 ? 0 : blo;
  c->WB = blo < 0 ? 0 : bhi - blo + 1;
  c->QA_cap = (size_t)(c->WA > 0 ? c->WA : 1);
  c->QB_cap = (size_t)(c->WB > 0 ? c->WB : 1);
  c->QA = ctx_alloc(c, c->rs * na * c->QA_cap * nxy);
  c->QB = ctx_alloc(c, c->rs * na * c->QB_cap * nxy);
  if (!c->QA || !c->QB) return set_error(GLASMA_ERR_OOM, "charge window allocation failed");
  if (c->WA > 0)
    k_fill_window<R><<<grid_for((int64_t)na * c->WA * nxy), 256, 0, c->stream>>>(rho3, (R*)c->QA, na, c->zA0,
                                                                                   c->WA, c->g);
  if (c->WB > 0)
    k_fill_window<R><<<grid_for((int64_t)na * c->WB * nxy), 256, 0, c->stream>>>(rho3, (R*)c->QB, na, c->zB0,
                                                                                   c->WB, c->g);
  st = cuda_check(cudaGetLastError(), "window fill");
  if (st) return st;
  if (c->Uit) {  // second iterate buffer of the implicit scheme: identity last-slice z links
    st = cuda_check(cudaMemcpyAsync(c->Uit, c->U[0], link_bytes(c), cudaMemcpyDeviceToDevice,
                                    c->stream),
                    "iterate buffer init");
    if (st) return st;
    c->uprev_valid = true;
  }
  st = cuda_check(cudaStreamSynchronize(c->stream), "init sync 2");
  ctx_free(c, full);
  ctx_free(c, rho);
  ctx_free(c, w0);
  ctx_free(c, w1);
  ctx_free(c, lam);
  ctx_free(c, rho3);
  ctx_free(c, smax);
  return st;
}

// Device helpers shared with the adjoint: the MV draw, the transverse
// Poisson solve of F real [ny][nx] fields (in and out may alias; w0, w1 hold
// F*nx*ny complex values each) and the profile table lam[(t*2 + N)*nz + iz].
int device_philox_rho(const glasma_params& p, int na, double* rho, cudaStream_t s) {
  const int64_t n = (int64_t)2 * na * p.nx * p.ny;
  k_philox_rho<<<grid_for(n), 256, 0, s>>>(rho, na, p.nx, p.ny, 1, p.seed, p.g2mu);
  return cuda_check(cudaGetLastError(), "philox rho");
}

int device_poisson(const glasma_params& p, const double* in, double* out, int F, double2* w0, double2* w1,
                   cudaStream_t s) {
  const int64_t nxy = (int64_t)p.nx * p.ny, n = F * nxy;
  k_real_to_cplx<<<grid_for(n), 256, 0, s>>>(in, w0, n);
  k_dft<<<grid_for(n), 256, 0, s>>>(w0, w1, F, p.ny, p.nx, 0, -1);
  k_dft<<<grid_for(n), 256, 0, s>>>(w1, w0, F, p.ny, p.nx, 1, -1);
  k_poisson_kernel<<<grid_for(n), 256, 0, s>>>(w0, F, p.ny, p.nx, p.a_t, p.m_ir * p.m_ir,
                                                p.uv_cutoff > 0 ? p.uv_cutoff * p.uv_cutoff : 0.0);
  k_dft<<<grid_for(n), 256, 0, s>>>(w0, w1, F, p.ny, p.nx, 1, +1);
  k_dft<<<grid_for(n), 256, 0, s>>>(w1, w0, F, p.ny, p.nx, 0, +1);
  k_cplx_real_scaled<<<grid_for(n), 256, 0, s>>>(w0, out, n, 1.0 / (double)nxy);
  return cuda_check(cudaGetLastError(), "poisson");
}

int device_profile(const glasma_params& p, double* lam, cudaStream_t s) {
  const double zc = p.nz * p.a_z / 2.0;
  const double d = p.z_offset > 0 ? p.z_offset : (ceil(4.0 * p.sigma_l / p.a_z) + 2.0) * p.a_z;
  k_profile<<<grid_for(4 * p.nz), 256, 0, s>>>(lam, p.nz, 0, p.a_z, p.sigma_l, zc + d, zc - d, p.dt);
  return cuda_check(cudaGetLastError(), "profile");
}

int run_init(glasma_ctx* c, const double* rho_host) {
  if (c->p.nc == 2) return c->rs == 8 ? init_t<2, double>(c, rho_host) : init_t<2, float>(c, rho_host);
  return c->rs == 8 ? init_t<3, double>(c, rho_host) : init_t<3, float>(c, rho_host);
}

}  // namespace glasma
