// Observables with FP64 accumulation: the discrete Gauss law residual
// (Sec. 3, Eq. gauss) and the per-slice energy-momentum tensor (Sec. 4).
// Reductions are deterministic: fixed grid, fixed-order tree in shared
// memory, fixed-order final pass over the block partials.
#include "glasma_internal.cuh"

namespace glasma {

constexpr int kRedThreads = 256;

// In-block tree reduction of NV doubles per thread; op 0 = sum, 1 = max.
template <int NV>
__device__ void block_reduce(double (*sh)[kRedThreads], double* v, const int* op) {
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NV; ++k) sh[k][t] = v[k];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
#pragma unroll
      for (int k = 0; k < NV; ++k)
        sh[k][t] = op[k] ? fmax(sh[k][t], sh[k][t + w]) : sh[k][t] + sh[k][t + w];
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = sh[k][0];
}

// ---------------------------------------------------------------------------
// Gauss residual
// ---------------------------------------------------------------------------
template <typename R>
struct GaussArgs {
  const typename V2T<R>::T* U;
  const R* E;
  const R* QA;
  const R* QB;
  Geom g;
  double ia2[3];  // 1 / a_i^2
  int zA0, WA, zB0, WB;
  int64_t s0, s1;  // sites of the owned slices
  double* part;    // [gridDim][4]
};

template <int NC, typename R>
__global__ void __launch_bounds__(kRedThreads) k_gauss(GaussArgs<R> a) {
  typedef Group<NC, double> G;
  constexpr int NA = G::NA;
  __shared__ double sh[4][kRedThreads];
  double gmax = 0, gsum2 = 0, rmax = 0, bad = 0;
  for (int64_t s = a.s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.s1;
       s += (int64_t)gridDim.x * blockDim.x) {
    SiteNbr n = site_nbr(a.g, s);
    double gv[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) gv[c] = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double q[NA];
#pragma unroll
      for (int c = 0; c < NA; ++c) gv[c] += a.ia2[i] * (double)a.E[(int64_t)(i * NA + c) * a.g.V + s];
      if (i == 2 && n.iz == 0) continue;
      const int64_t sm = n.m[i];
#pragma unroll
      for (int c = 0; c < NA; ++c) q[c] = (double)a.E[(int64_t)(i * NA + c) * a.g.V + sm];
      typename G::M um = LinkIO<NC, R>::template load<double>(a.U, i, a.g.V, sm);
      G::adj_dag(um, q);
#pragma unroll
      for (int c = 0; c < NA; ++c) gv[c] -= a.ia2[i] * q[c];
    }
    const int64_t t = s % a.g.nxy;
    double rho[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) rho[c] = 0.0;
    const int ka = n.iz - a.zA0, kb = n.iz - a.zB0;
    if (ka >= 0 && ka < a.WA)
#pragma unroll
      for (int c = 0; c < NA; ++c) rho[c] += (double)a.QA[((int64_t)c * a.WA + ka) * a.g.nxy + t];
    if (kb >= 0 && kb < a.WB)
#pragma unroll
      for (int c = 0; c < NA; ++c) rho[c] += (double)a.QB[((int64_t)c * a.WB + kb) * a.g.nxy + t];
#pragma unroll
    for (int c = 0; c < NA; ++c) {
      double r = gv[c] - rho[c];
      if (!isfinite(r)) bad += 1.0;
      gmax = fmax(gmax, fabs(r));
      gsum2 += r * r;
      rmax = fmax(rmax, fabs(rho[c]));
    }
  }
  double v[4] = {gmax, gsum2, rmax, bad};
  const int op[4] = {1, 0, 1, 0};
  block_reduce<4>(sh, v, op);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) a.part[blockIdx.x * 4 + k] = v[k];
}

// One block folds nb partials of width NV in a fixed order; bit k of MAXMASK
// selects max (else sum) for component k.
template <int NV, int MAXMASK>
__global__ void __launch_bounds__(kRedThreads) k_fold(const double* part, int nb, double* out) {
  __shared__ double sh[NV][kRedThreads];
  int op[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) op[k] = (MAXMASK >> k) & 1;
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nb; b += kRedThreads)
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = op[k] ? fmax(v[k], part[b * NV + k]) : v[k] + part[b * NV + k];
  block_reduce<NV>(sh, v, op);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = v[k];
}

static int reduction_grid(glasma_ctx* c) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  int64_t need = ((int64_t)(c->hi - c->lo) * c->g.nxy + kRedThreads - 1) / kRedThreads;
  int64_t nb = (int64_t)sms * 4;
  return (int)(need < nb ? need : nb);
}

template <int NC, typename R>
static int gauss_t(glasma_ctx* c, double* out3) {
  GaussArgs<R> a;
  a.U = (const typename V2T<R>::T*)c->U[c->cur];
  a.E = (const R*)c->E;
  a.QA = (const R*)c->QA;
  a.QB = (const R*)c->QB;
  a.g = c->g;
  a.ia2[0] = a.ia2[1] = 1.0 / (c->p.a_t * c->p.a_t);
  a.ia2[2] = 1.0 / (c->p.a_z * c->p.a_z);
  a.zA0 = c->zA0;
  a.WA = c->WA;
  a.zB0 = c->zB0;
  a.WB = c->WB;
  a.s0 = (int64_t)c->lo * c->g.nxy;
  a.s1 = (int64_t)c->hi * c->g.nxy;
  const int nb = reduction_grid(c);
  // partials, then the op table and the 4 results, in the context's scratch
  if ((size_t)nb * 4 + 8 > c->red_cap) return set_error(GLASMA_ERR_INTERNAL, "reduction scratch too small");
  a.part = c->red;
  double* res = c->red + (size_t)nb * 4;
  k_gauss<NC, R><<<nb, kRedThreads, 0, c->stream>>>(a);
  int st = cuda_check(cudaGetLastError(), "k_gauss launch");
  if (st) return st;
  k_fold<4, 0x5><<<1, kRedThreads, 0, c->stream>>>(c->red, nb, res);
  st = cuda_check(cudaGetLastError(), "k_fold launch");
  if (st) return st;
  double h[4];
  st = cuda_check(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "gauss readback");
  if (st) return st;
  st = cuda_check(cudaStreamSynchronize(c->stream), "gauss sync");
  if (st) return st;
  out3[0] = h[0];
  out3[1] = sqrt(h[1] / ((double)(a.s1 - a.s0) * (c->na)));
  out3[2] = h[2];
  if (h[3] != 0.0) return set_error(GLASMA_ERR_NONFINITE, "Gauss residual met a non-finite value");
  return GLASMA_OK;
}

int launch_gauss(glasma_ctx* c, double* out3) {
  if (c->p.nc == 2) return c->rs == 8 ? gauss_t<2, double>(c, out3) : gauss_t<2, float>(c, out3);
  return c->rs == 8 ? gauss_t<3, double>(c, out3) : gauss_t<3, float>(c, out3);
}

// ---------------------------------------------------------------------------
// T^{mu nu} per z slice
// ---------------------------------------------------------------------------
template <typename R>
struct TmnArgs {
  const typename V2T<R>::T* U;
  const R* E;
  const R* QA;
  const R* QB;
  Geom g;
  R dt;
  R w[3];
  R az2;
  double a[3];
  // products of reciprocals of the spacings, formed on the host (an FP64
  // division is a long sequence on GB300's narrow FP64 pipe):
  double binv[3];   // 1 / (a_i a_j)^2 of the planes xy, xz, yz
  double hinv2[3];  // 1 / (2 a_i^2)
  double slc[2];    // Poynting weights 1 / (a_x^2 a_z), 1 / (a_y^2 a_z)
  int hop;
  int zA0, WA, zB0, WB;
  int split;     // blocks per z slice
  double* part;  // [nz][split][5] block sums of eps, p_L, p_T, S_L, non-finite count
};

// ||x - y||_F^2 of two links in the state's representation (for FP32 the
// deviations from 1, whose difference is that of the links), in the state's
// precision: a difference of two FP32 entries rounds to within u of itself,
// and the sum of squares has no cancellation, so the FP32 value carries the
// FP32 products' own relative accuracy; it enters the FP64 sums once per
// site.
template <int NC, typename R> struct Fro2;
template <typename R>
struct Fro2<3, R> {
  GL_HD static R diff(const typename Group<3, R>::M& x, const typename Group<3, R>::M& y) {
    R acc = R(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const R dr = x.m[k].re - y.m[k].re, di = x.m[k].im - y.m[k].im;
      acc += dr * dr + di * di;
    }
    return acc;
  }
};
template <typename R>
struct Fro2<2, R> {
  GL_HD static R diff(const typename Group<2, R>::M& x, const typename Group<2, R>::M& y) {
    const R a = x.a.re - y.a.re, b = x.a.im - y.a.im;
    const R c = x.b.re - y.b.re, d = x.b.im - y.b.im;
    return R(2) * (a * a + b * b + c * c + d * d);
  }
};

// Per-site arithmetic in the state's precision R (so E(n+1/2) equals what
// the step kernel would write; FP32 plaquette products in the deviation
// form; the per-site sums of squares and of E B products in R, all of
// positive terms except the Poynting sum), every accumulation over sites in
// FP64.  Block (iz, p) takes the sites
// t = p*256 + threadIdx.x + k*split*256 of slice iz; k_tmunu_fold adds the
// split block sums of a slice in a fixed order.
template <int NC, typename R>
__global__ void __launch_bounds__(kRedThreads) k_tmunu(TmnArgs<R> a) {
  typedef LinkAlg<NC, R> G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
  __shared__ double sh[5][kRedThreads];
  const int iz = blockIdx.x;
  double eps = 0, pl = 0, pt = 0, sl = 0, bad = 0;
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < a.g.nxy; t += a.split * blockDim.x) {
    const int64_t s = (int64_t)iz * a.g.nxy + t;
    SiteNbr n = site_nbr(a.g, s);
    typedef LinkIO<NC, R> IO;
    // magnetic terms from the plaquettes at the base site, with the link
    // products in the state's representation:
    // b_ij = ||U_i(x) U_j(x+i) - U_j(x) U_i(x+j)||_F^2 / (a_i a_j)^2
    // (= 2 (N - Re tr U_ij) for unitary links, without its cancellation),
    // B from Im tr t^a U_ij with U_ij = A B^dagger.  They come first, so that
    // only the projections (in the state's precision) stay live across the
    // three link forces below.
    double bxy, bxz = 0, byz = 0;
    R prx[NA], pry[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) prx[c] = pry[c] = R(0);
    {
      const M A = G::mul(IO::template load<R>(a.U, 0, a.g.V, s), IO::template load<R>(a.U, 1, a.g.V, n.p[0]));
      const M B = G::mul(IO::template load<R>(a.U, 1, a.g.V, s), IO::template load<R>(a.U, 0, a.g.V, n.p[1]));
      bxy = (double)Fro2<NC, R>::diff(A, B) * a.binv[0];
    }
    if (iz <= a.g.nz - 2) {
      M A = G::mul(IO::template load<R>(a.U, 0, a.g.V, s), IO::template load<R>(a.U, 2, a.g.V, n.p[0]));  // U_x U_z(x+x)
      M B = G::mul(IO::template load<R>(a.U, 2, a.g.V, s), IO::template load<R>(a.U, 0, a.g.V, n.p[2]));  // U_z U_x(x+z)
      bxz = (double)Fro2<NC, R>::diff(A, B) * a.binv[1];
      Group<NC, R>::proj(G::mul_d(A, B), pry);  // B_y = -2 Im tr t U_zx / (a_z a_x) = +2 Im tr t U_xz / (a_x a_z)
      A = G::mul(IO::template load<R>(a.U, 1, a.g.V, s), IO::template load<R>(a.U, 2, a.g.V, n.p[1]));  // U_y U_z(x+y)
      B = G::mul(IO::template load<R>(a.U, 2, a.g.V, s), IO::template load<R>(a.U, 1, a.g.V, n.p[2]));  // U_z U_y(x+z)
      byz = (double)Fro2<NC, R>::diff(A, B) * a.binv[2];
      Group<NC, R>::proj(G::mul_d(A, B), prx);  // B_x = -2 Im tr t U_yz / (a_y a_z)
    }
    double e2[3] = {0, 0, 0};
    double s_l = 0;
    const int ilast = (iz == a.g.nz - 1) ? 2 : 3;
    for (int i = 0; i < ilast; ++i) {
      R F[NA];
      link_force_staple<NC, R, R>(a.U, a.g, n, i, a.w, F);
      R en[NA], eo[NA];
#pragma unroll
      for (int c = 0; c < NA; ++c) {
        eo[c] = a.E[(int64_t)(i * NA + c) * a.g.V + s];
        en[c] = eo[c] + a.dt * F[c];
      }
      if (i == 2 && a.hop) {
        R dj[NA];
#pragma unroll
        for (int c = 0; c < NA; ++c) dj[c] = R(0);
        const int kb = iz - a.zB0;
        if (kb >= 0 && kb < a.WB)
#pragma unroll
          for (int c = 0; c < NA; ++c) dj[c] -= a.az2 * a.QB[((int64_t)c * a.WB + kb) * a.g.nxy + t];
        const int ka = iz + 1 - a.zA0;
        if (ka >= 0 && ka < a.WA) {
          R q[NA];
#pragma unroll
          for (int c = 0; c < NA; ++c) q[c] = a.QA[((int64_t)c * a.WA + ka) * a.g.nxy + t];
          G::adj(IO::template load<R>(a.U, 2, a.g.V, s), q);
#pragma unroll
          for (int c = 0; c < NA; ++c) dj[c] += a.az2 * q[c];
        }
#pragma unroll
        for (int c = 0; c < NA; ++c) en[c] += dj[c];
      }
      R acc = R(0), dot = R(0);
#pragma unroll
      for (int c = 0; c < NA; ++c) {
        const R o = eo[c], nn = en[c];
        acc += o * o + nn * nn;
        // S_L = sum_a (Ebar_x B_y - Ebar_y B_x), Ebar the time mean of E / a,
        // B_y = 2 pry / (a_x a_z), B_x = -2 prx / (a_y a_z)
        if (i == 0) dot += (o + nn) * pry[c];
        if (i == 1) dot += (o + nn) * prx[c];
      }
      if (i < 2) s_l += a.slc[i] * (double)dot;
      e2[i] = (double)acc * a.hinv2[i];
    }
    double e = 0.5 * (e2[0] + e2[1] + e2[2]) + bxy + bxz + byz;
    double p_t = 0.5 * e2[2] + bxy;
    double p_l = 0.5 * (e2[0] + e2[1]) + bxz + byz - p_t;
    if (!isfinite(e) || !isfinite(s_l)) bad += 1.0;
    eps += e;
    pl += p_l;
    pt += p_t;
    sl += s_l;
  }
  double v[5] = {eps, pl, pt, sl, bad};
  const int op[5] = {0, 0, 0, 0, 0};
  block_reduce<5>(sh, v, op);
  if (threadIdx.x == 0) {
    double* out = a.part + ((int64_t)iz * a.split + blockIdx.y) * 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) out[k] = v[k];
  }
}

// tab[iz] = (sum over the split blocks of slice iz, in block order) / nxy;
// a slice that met a non-finite value gets a NaN energy density.
__global__ void k_tmunu_fold(const double* part, int split, int nz, double inv, double* tab) {
  const int iz = blockIdx.x * blockDim.x + threadIdx.x;
  if (iz >= nz) return;
  double v[5] = {0, 0, 0, 0, 0};
  for (int p = 0; p < split; ++p)
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += part[((int64_t)iz * split + p) * 5 + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) tab[iz * 4 + k] = v[k] * inv;
  if (v[4] != 0.0) tab[iz * 4 + 0] = __longlong_as_double(0x7ff8000000000000LL);  // NaN marks it
}

template <int NC, typename R>
static int tmunu_t(glasma_ctx* c, bool hop, double* host_tab, double* dev_tab) {
  TmnArgs<R> a;
  a.U = (const typename V2T<R>::T*)c->U[c->cur];
  a.E = (const R*)c->E;
  a.QA = (const R*)c->QA;
  a.QB = (const R*)c->QB;
  a.g = c->g;
  a.dt = (R)c->p.dt;
  a.w[0] = (R)(2.0 / (c->p.a_t * c->p.a_t));
  a.w[1] = a.w[0];
  a.w[2] = (R)(2.0 / (c->p.a_z * c->p.a_z));
  a.az2 = (R)(c->p.a_z * c->p.a_z);
  a.a[0] = a.a[1] = c->p.a_t;
  a.a[2] = c->p.a_z;
  a.binv[0] = 1.0 / (a.a[0] * a.a[1] * a.a[0] * a.a[1]);
  a.binv[1] = 1.0 / (a.a[0] * a.a[2] * a.a[0] * a.a[2]);
  a.binv[2] = 1.0 / (a.a[1] * a.a[2] * a.a[1] * a.a[2]);
  for (int i = 0; i < 3; ++i) a.hinv2[i] = 0.5 / (a.a[i] * a.a[i]);
  a.slc[0] = 1.0 / (a.a[0] * a.a[0] * a.a[2]);
  a.slc[1] = 1.0 / (a.a[1] * a.a[1] * a.a[2]);
  a.hop = hop ? 1 : 0;
  a.zA0 = c->zA0;
  a.WA = c->WA;
  a.zB0 = c->zB0;
  a.WB = c->WB;
  // kTmunuSplit blocks per slice (fewer if the plane has fewer sites than
  // threads): the split, and with it the order of each slice's sums, depends
  // on the transverse plane alone, not on the number of slices or the device,
  // so a z slab's rows equal the whole lattice's bit for bit
  const int64_t per_slice = (c->g.nxy + kRedThreads - 1) / kRedThreads;
  int64_t split = kTmunuSplit;
  if (split > per_slice) split = per_slice;
  if (split < 1) split = 1;
  a.split = (int)split;
  a.part = c->tpart;
  double* tab = dev_tab ? dev_tab : c->tab;
  k_tmunu<NC, R><<<dim3((unsigned)c->g.nz, (unsigned)split), kRedThreads, 0, c->stream>>>(a);
  int st = cuda_check(cudaGetLastError(), "k_tmunu launch");
  if (st) return st;
  k_tmunu_fold<<<(c->g.nz + 127) / 128, 128, 0, c->stream>>>(c->tpart, (int)split, c->g.nz, 1.0 / (double)c->g.nxy,
                                                              tab);
  st = cuda_check(cudaGetLastError(), "k_tmunu_fold launch");
  if (st || !host_tab) return st;
  st = cuda_check(cudaMemcpyAsync(host_tab, c->tab, sizeof(double) * 4 * c->g.nz, cudaMemcpyDeviceToHost,
                                  c->stream),
                  "tmunu readback");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(c->stream), "tmunu sync");
}

int launch_tmunu(glasma_ctx* c, bool hop, double* host_tab, double* dev_tab) {
  if (c->p.nc == 2)
    return c->rs == 8 ? tmunu_t<2, double>(c, hop, host_tab, dev_tab) : tmunu_t<2, float>(c, hop, host_tab, dev_tab);
  return c->rs == 8 ? tmunu_t<3, double>(c, hop, host_tab, dev_tab) : tmunu_t<3, float>(c, hop, host_tab, dev_tab);
}

}  // namespace glasma
