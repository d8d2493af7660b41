// Leapfrog step with the CPIC hop, plaquette-centric form (Sec. 3,
// Eqs. lattice_1, plaquette, lattice_2, continuity).
//
// The staple form (step_link) rebuilds every plaquette once for each of
// its four links.  Here each site x forms the three plaquettes based at it,
// P_ab(x) for (a, b) = (x, y), (x, z), (y, z), once, from two shared
// partial products
//   A = U_b(x+a) U_a^dag(x+b),   B = U_b^dag(x) U_a(x),
// and reads off the loop at each corner where one of its links starts:
//   corner x    (links a and b of x):  P = U_a(x) A U_b^dag(x),
//   corner x+a  (link b of x+a):       U_{b,-a}(x+a) = A B,
//   corner x+b  (link a of x+b):       U_{a,-b}(x+b) = (B A)^dag.
// With F_i = -sum_{j != i} w_j [Im tr t^a U_{i,j} + Im tr t^a U_{i,-j}]
// (w_j = 2/a_j^2) the contributions are
//   F_a(x)   -= w_b p0,   F_b(x)   += w_a p0,
//   F_a(x+b) += w_b pBA,  F_b(x+a) -= w_a pAB,
// with p0 = proj P, pAB = proj AB, pBA = proj BA.  That is 5.5 SU(N)
// products per plaquette (A, B, U_a A, and three projections of 0.83
// products each), 16.5 per site, against 24 for the staples of the same
// three links plus three projections.
//
// Work decomposition: a block owns `rows` full transverse rows (x periodic
// inside the block) and marches through `zlen` consecutive z slices; one
// thread per transverse site.  Contributions to the +x and +y neighbours
// go through shared memory: written, barrier, read by the neighbours,
// barrier (the second one right after the reads, so the link updates and
// the next slice's plaquettes run between barriers).  Those to the +z
// neighbour (the same thread, next slice) wait in the thread's own
// shared-memory slot, read before they are replaced, and so do the y and z
// forces while the x link is updated (fewer live registers).  The row below the block's first row (the -y halo) is
// computed by an extra row of threads that forms only the two partial
// plaquettes the first row needs; the slice before the first one is a
// warm-up that forms only the +z contributions.  A block that holds every
// row of the lattice needs no halo.
//
// Open z (reading R6): no plaquettes in the planes containing z are based
// on the last slice, and there is no z link there.
#include "step_link.cuh"

namespace glasma {

template <typename R>
struct PlaqArgs {
  StepArgs<R> s;
  int rows;      // interior rows per block (== ny: the block holds the plane)
  int halo;      // 1 if the block has a -y halo row
  int zlen;      // slices per block
  int zhi;       // one past the last slice updated (s.zlo is the first)
};

// shared-memory vectors per site: the +x contributions to the y and z
// links and the +y contributions to the x and z links (read by the
// neighbours), the +z contributions to the x and y links and the three
// force partials (read by the thread itself)
enum { kCxY = 0, kCxZ = 1, kCyX = 2, kCyZ = 3, kCzX = 4, kCzY = 5, kF = 6, kVecs = 9 };

template <int NC, typename R>
struct PlaqWork {
  typedef LinkAlg<NC, R> G;
  typedef typename G::M M;
  static constexpr int NA = G::NA;

  // The two partial products of the plaquette in plane (a, b) based at s:
  // A = U_b(x+a) U_a^dag(x+b), B = U_b^dag(x) U_a(x).
  __device__ __forceinline__ static void partials(const typename V2T<R>::T* U, const Geom& g, int a, int b,
                                                  int64_t s, int64_t sa, int64_t sb, M& A, M& B) {
    A = G::mul_d(LinkIO<NC, R>::template load<R>(U, b, g.V, sa), LinkIO<NC, R>::template load<R>(U, a, g.V, sb));
    B = G::d_mul(LinkIO<NC, R>::template load<R>(U, b, g.V, s), LinkIO<NC, R>::template load<R>(U, a, g.V, s));
  }
  // p0 = proj(U_a(x) A U_b^dag(x))
  __device__ __forceinline__ static void corner0(const typename V2T<R>::T* U, const Geom& g, int a, int b,
                                                 int64_t s, const M& A, R* p0) {
    const M C = G::mul(LinkIO<NC, R>::template load<R>(U, a, g.V, s), A);
    G::proj_prod_d(C, LinkIO<NC, R>::template load<R>(U, b, g.V, s), p0);
  }
};

// Block shapes: V = 0 up to 320 threads (96 registers at 2 FP32 blocks per
// SM), V = 1 up to 256 threads (128 registers).  FP64 runs one block per SM.
template <typename R, int V> struct PlaqOcc {
  static constexpr int threads = V == 0 ? 320 : 256, blocks = sizeof(R) == 8 ? 1 : 2;
};

template <int NC, typename R, int V>
__global__ void __launch_bounds__(PlaqOcc<R, V>::threads, PlaqOcc<R, V>::blocks) k_step_plaq(PlaqArgs<R> pa) {
  typedef PlaqWork<NC, R> W;
  typedef typename W::M M;
  constexpr int NA = W::NA;
  const StepArgs<R>& a = pa.s;
  const Geom& g = a.g;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sm = (R*)smem_raw;
  const int nx = g.nx, ny = g.ny;
  const int trows = pa.rows + pa.halo;      // thread rows of the block
  const int TS = trows * nx;                // shared-memory slots per vector
  const int l = threadIdx.x;
  const bool active = l < TS;
  const int r = active ? l / nx : 0;
  const int ix = active ? l - r * nx : 0;
  const int y0 = blockIdx.x * pa.rows;
  const bool halo = pa.halo && r == 0;
  int iy = pa.halo ? y0 + r - 1 : y0 + r;
  if (iy < 0) iy += ny;
  // interior: a site of this block's rows (the last block may be ragged)
  const bool inner = active && !halo && (pa.halo ? y0 + r - 1 : y0 + r) < ny;
  const bool hrow = active && halo;  // a thread of the -y halo row
  const uint32_t t = (uint32_t)iy * nx + ix;
  const uint32_t txp = (uint32_t)iy * nx + (ix + 1 == nx ? 0 : ix + 1);
  const uint32_t typ = (uint32_t)(iy + 1 == ny ? 0 : iy + 1) * nx + ix;
  // shared slots of the -x and -y neighbours
  const int slot_mx = ix == 0 ? l + nx - 1 : l - 1;
  const int slot_my = pa.halo ? l - nx : (r == 0 ? l + (ny - 1) * nx : l - nx);
  const R wt = a.w[0], wz = a.w[2];

  const int z0 = a.zlo + blockIdx.y * pa.zlen;
  const int z1 = min(z0 + pa.zlen, pa.zhi);
  R* cz = sm;
  if (inner && z0 == 0) {
#pragma unroll
    for (int c = 0; c < NA; ++c) cz[(kCzX * NA + c) * TS + l] = cz[(kCzY * NA + c) * TS + l] = R(0);
  }

  // A chunk that starts above slice 0 first runs a warm-up iteration on the
  // slice below it, which only forms the +z contributions (pBA of the
  // (x, z) and (y, z) plaquettes) of that slice: the same instructions as
  // in every other iteration, so the result does not depend on where the
  // chunks (or the slabs of a split lattice) begin.
  for (int iz = z0 > 0 ? z0 - 1 : z0; iz < z1; ++iz) {
    const bool warm = iz < z0;
    R* buf = sm;
    const int64_t s = (int64_t)iz * g.nxy + t;
    const int64_t sxp = s - t + txp, syp = s - t + typ;
    const bool zlink = iz < g.nz - 1;
    if (inner && !warm) {
      // force partials start from the +z contributions of slice iz - 1
#pragma unroll
      for (int c = 0; c < NA; ++c) {
        buf[((kF + 0) * NA + c) * TS + l] = cz[(kCzX * NA + c) * TS + l];
        buf[((kF + 1) * NA + c) * TS + l] = cz[(kCzY * NA + c) * TS + l];
        buf[((kF + 2) * NA + c) * TS + l] = R(0);
      }
    }
    // planes (x, y), (x, z), (y, z); the last slice has only (x, y), the
    // halo row needs pBA of (x, y) and pAB of (y, z) only, the warm-up
    // pBA of (x, z) and (y, z) only
    const int np = zlink ? 3 : 1;
#pragma unroll 1
    for (int pl = warm ? 1 : 0; pl < np; ++pl) {
      const int pa_ = pl == 2 ? 1 : 0, pb = pl == 0 ? 1 : 2;
      // threads of rows past the lattice's last row (a ragged last block)
      // and past the block's rows do nothing
      const bool need_ab = !warm && (inner || (hrow && pl == 2));
      const bool need_ba = inner || (!warm && hrow && pl == 0);
      if (!(need_ab || need_ba)) continue;
      const int64_t sa = pa_ == 0 ? sxp : syp, sb = pb == 1 ? syp : s + g.nxy;
      const R wa = wt, wb = pb == 2 ? wz : wt;  // w_a, w_b = 2 / a^2 of the plane's directions
      // shared vector of pAB (to link b of x+a) and of pBA (to link a of x+b)
      const int vab = pl == 0 ? kCxY : (pl == 1 ? kCxZ : kCyZ);
      const int vba = pl == 0 ? kCyX : (pl == 1 ? kCzX : kCzY);
      M A, B;
      R p[NA];
      W::partials(a.U, g, pa_, pb, s, sa, sb, A, B);
      if (need_ab) {
        LinkAlg<NC, R>::proj_prod(A, B, p);
#pragma unroll
        for (int c = 0; c < NA; ++c) buf[(vab * NA + c) * TS + l] = -wa * p[c];
      }
      if (need_ba) {
        LinkAlg<NC, R>::proj_prod(B, A, p);
#pragma unroll
        for (int c = 0; c < NA; ++c) buf[(vba * NA + c) * TS + l] = wb * p[c];
      }
      if (inner && !warm) {
        W::corner0(a.U, g, pa_, pb, s, A, p);
        R* fa = buf + (kF + pa_) * NA * TS + l;
        R* fb = buf + (kF + pb) * NA * TS + l;
#pragma unroll
        for (int c = 0; c < NA; ++c) {
          fa[c * TS] -= wb * p[c];
          fb[c * TS] += wa * p[c];
        }
      }
    }
    if (warm) continue;  // the same for every thread of the block: no barrier is skipped unevenly
    __syncthreads();
    if (inner) {
#pragma unroll
      for (int c = 0; c < NA; ++c) {
        buf[((kF + 0) * NA + c) * TS + l] += buf[(kCyX * NA + c) * TS + slot_my];
        buf[((kF + 1) * NA + c) * TS + l] += buf[(kCxY * NA + c) * TS + slot_mx];
      }
      if (zlink) {
#pragma unroll
        for (int c = 0; c < NA; ++c)
          buf[((kF + 2) * NA + c) * TS + l] +=
              buf[(kCxZ * NA + c) * TS + slot_mx] + buf[(kCyZ * NA + c) * TS + slot_my];
      }
    }
    __syncthreads();
    if (inner) {
      const int nl = zlink ? 3 : 2;
#pragma unroll 1
      for (int i = 0; i < nl; ++i) {
        R F[NA];
#pragma unroll
        for (int c = 0; c < NA; ++c) F[c] = buf[((kF + i) * NA + c) * TS + l];
        update_link<NC, R>(a, i, t, iz, s, F);
      }
    }
  }
}

// Block shape: the most interior rows (a divisor of ny if one fits) such
// that rows + 1 halo rows of nx threads fit the block; the whole plane in
// one block when it fits without a halo.
static bool plaq_shape(int nx, int ny, int tmax, int* rows, int* halo) {
  if (nx > tmax) return false;
  if (nx * ny <= tmax) {
    *rows = ny;
    *halo = 0;
    return true;
  }
  const int rmax = tmax / nx - 1;
  if (rmax < 1) return false;
  int best = 1;
  for (int r = rmax; r >= 1; --r)
    if (ny % r == 0) {
      best = r;
      break;
    }
  // a divisor below half the maximum wastes more on halos than a ragged
  // last block does
  *rows = best * 2 >= rmax ? best : rmax;
  *halo = 1;
  return true;
}

template <int NC, typename R, int V>
static int launch_plaq_t(glasma_ctx* c, bool hop, int zlen) {
  PlaqArgs<R> pa;
  StepArgs<R>& a = pa.s;
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
  pa.zhi = c->hi;
  constexpr int T = PlaqOcc<R, V>::threads;
  if (!plaq_shape(c->g.nx, c->g.ny, T, &pa.rows, &pa.halo))
    return set_error(GLASMA_ERR_INTERNAL, "plaquette kernel: transverse rows too long");
  pa.zlen = zlen;
  const int TS = (pa.rows + pa.halo) * c->g.nx;
  const size_t smem = (size_t)kVecs * LinkAlg<NC, R>::NA * TS * sizeof(R);
  if (!c->plaq_ready) {
    int st = plaq_prepare(c);
    if (st) return st;
  }
  const unsigned tiles = (unsigned)((c->g.ny + pa.rows - 1) / pa.rows);
  const unsigned chunks = (unsigned)((c->hi - c->lo + zlen - 1) / zlen);
  const unsigned threads = (unsigned)((TS + 31) / 32 * 32);
  k_step_plaq<NC, R, V><<<dim3(tiles, chunks), threads, smem, c->stream>>>(pa);
  return cuda_check(cudaGetLastError(), "k_step_plaq launch");
}

// Block shape variant of the context (0: 320 threads, 1: 256 threads).
static int plaq_variant(const glasma_ctx* c) { return c->step_kernel == GLASMA_KERNEL_PLAQUETTE_256 ? 1 : 0; }

// The dynamic shared-memory limit is a per-device function attribute: set
// it for every instance this context may launch, on the context's device.
template <int NC, typename R>
static int plaq_attrs() {
  int st = cuda_check(cudaFuncSetAttribute(k_step_plaq<NC, R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(kVecs * LinkAlg<NC, R>::NA * PlaqOcc<R, 0>::threads * sizeof(R))),
                      "k_step_plaq attributes");
  if (st) return st;
  return cuda_check(cudaFuncSetAttribute(k_step_plaq<NC, R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kVecs * LinkAlg<NC, R>::NA * PlaqOcc<R, 1>::threads * sizeof(R))),
                    "k_step_plaq attributes");
}

int plaq_prepare(glasma_ctx* c) {
  int st;
  if (c->p.nc == 2)
    st = c->rs == 8 ? plaq_attrs<2, double>() : plaq_attrs<2, float>();
  else
    st = c->rs == 8 ? plaq_attrs<3, double>() : plaq_attrs<3, float>();
  if (!st) c->plaq_ready = true;
  return st;
}

bool plaq_fits(const glasma_ctx* c) {
  int rows, halo;
  return plaq_shape(c->g.nx, c->g.ny, plaq_variant(c) ? 256 : 320, &rows, &halo);
}

// z slices per block: about eight blocks per SM slot in flight over the
// launch, at least 4 slices (the warm-up slice costs a quarter of a slice)
int plaq_default_zlen(const glasma_ctx* c) {
  int rows, halo;
  const int T = plaq_variant(c) ? 256 : 320;
  if (!plaq_shape(c->g.nx, c->g.ny, T, &rows, &halo)) return 16;
  const long long tiles = (c->g.ny + rows - 1) / rows;
  const long long slots = 152LL * (c->rs == 8 ? 1 : 2);
  long long z = tiles * (c->hi - c->lo) / (8 * slots);
  if (z < 4) z = 4;
  if (z > 64) z = 64;
  return (int)z;
}

int launch_step_plaq(glasma_ctx* c, bool hop, int zlen) {
  if (zlen <= 0) zlen = plaq_default_zlen(c);
  const int v = plaq_variant(c);
  if (c->p.nc == 2) {
    if (c->rs == 8) return v ? launch_plaq_t<2, double, 1>(c, hop, zlen) : launch_plaq_t<2, double, 0>(c, hop, zlen);
    return v ? launch_plaq_t<2, float, 1>(c, hop, zlen) : launch_plaq_t<2, float, 0>(c, hop, zlen);
  }
  if (c->rs == 8) return v ? launch_plaq_t<3, double, 1>(c, hop, zlen) : launch_plaq_t<3, double, 0>(c, hop, zlen);
  return v ? launch_plaq_t<3, float, 1>(c, hop, zlen) : launch_plaq_t<3, float, 0>(c, hop, zlen);
}

}  // namespace glasma
