// Semi-implicit step against the numerical Cherenkov instability (Sec. 3,
// the paragraph after Eq. gauss, Fig. wilson (b); Sec. 5).
//
// Each staple pair U_{i,+-j} of Eq. lattice_1 is replaced by its average over
// the time slots m = n+1, n, n-1 with weights (1/4, 1/2, 1/4).  In the
// transverse plane (x, y) every link of the loop is taken at slot m; in a
// plane containing z only the z links are taken at slot m and the transverse
// links stay at t_n.  The system is solved by fixed-point iteration on
// E(t_{n+1/2}) starting from U(t_{n+1}) = exp(i dt E(t_{n-1/2})) U(t_n);
// every sweep after the first is relaxed, E <- (1 - omega) E + omega G(E),
// omega = 2 / (2 + c) with c = 2 dt^2 / a_T^2 the extreme eigenvalue of the
// sweep's Jacobian (dt^2 times the weight 1/4 of the slot t_{n+1} times the
// curl-curl bound 8 / a_T^2): the contraction per sweep drops from c to
// c / (2 + c), below 1 for every dt.
// The CPIC hop and its current are those of the leapfrog step (they use
// U(t_n) only) and are applied once, before the iteration.
//
// Buffers: Uprev = U(t_{n-1}), U[cur] = U(t_n), the other U buffer and Uit
// hold the iterates of U(t_{n+1}); E is iterated in place, Ework keeps
// E(t_{n-1/2}) + dt J + dt times the force of the two fixed slots (t_n and
// t_{n-1}), which the prepare kernel evaluates once per step.  conv[k] is
// the largest |E^(k+1) - E^(k)| of iteration k and conv[maxit + 1 + k] the
// largest |E^(k+1)| (atomicMax on the bit pattern of a non-negative
// double).  The iteration ends when implicit_converged holds: the change is
// below implicit_tol, or it has reached the rounding level of the state's
// precision (always first in FP32).  Every launch after that returns at
// once; if it never holds within implicit_max_iter the step reports
// NOT_CONVERGED.
//
// On a z slab (glasma_slab_init) the step runs in host-driven parts
// (glasma_implicit_begin / _sweep / _end): every sweep's maxima are read
// back, folded across the ranks, and the host applies the stopping test.
// The sweeps need no halo messages: in a plane containing z only the z
// links take the time slot, so the force on a z link reads z links of its
// own slice and transverse links at t_n of its slice and the one above.
// So each part also evaluates the z link of the lower halo slice (one more
// launch over that slice: k_implicit_prep_halo, k_implicit_iter_halo), from
// the step's halo and with its owner's arithmetic, including the hop of the
// charges that cross it; the maxima stay those of the owned slices.
#include <vector>

#include "glasma_internal.cuh"

namespace glasma {

// Iteration k has converged if its largest change d_k = max|dE| is below
// the tolerance; or if the error bound of a contraction, d_k c / (1 - c),
// is at most 16 unit roundoffs of max|E| (the noise that one sweep's
// rounding leaves, 10 to 50 unit roundoffs of max|E| in FP32 depending on
// the fields, so one more sweep cannot improve the iterate), with the rate
// c taken as the larger of the last two observed ratios d_k / d_(k-1) and
// d_(k-1) / d_(k-2) (the first sweeps remove fast modes and contract
// faster than the last ones) and required below 1/2; or if d_k is within
// 64 unit roundoffs of max|E| and no longer falls by half per sweep (the
// changes are then the rounding noise itself); or if d_k no longer
// decreases while already within 1024 unit roundoffs of max|E| (the
// rounding floor).  A change that stops decreasing above that floor is a
// failing iteration (e.g. dt^2 K_T / 4 > 1), not convergence.
GL_HD bool implicit_converged(const double* conv, int maxit, int k, double tol, bool fp32) {
  const double d = conv[k];
  if (d < tol) return true;
  if (k < 1) return false;
  const double u = fp32 ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
  const double emax = conv[maxit + 1 + k];
  if (k >= 2 && conv[k - 1] > 0.0 && conv[k - 2] > 0.0) {
    const double c = fmax(d / conv[k - 1], conv[k - 1] / conv[k - 2]);
    if (c < 0.5 && d * c <= 16.0 * u * emax * (1.0 - c)) return true;
  }
  if (d <= 64.0 * u * emax && d >= 0.5 * conv[k - 1]) return true;
  if (d < conv[k - 1]) return false;
  return d <= 1024.0 * u * emax;
}

template <typename R>
struct ImplArgs {
  typedef typename V2T<R>::T V2;
  const V2* Up;   // U(t_{n-1})
  const V2* Un;   // U(t_n)
  const V2* X;    // current iterate of U(t_{n+1})
  V2* Xn;         // next iterate
  V2* Uout;       // prepare / previous-link kernels: output links
  R* E;
  R* Ework;
  R* QA;
  R* QB;
  double* conv;   // [k]: max |dE| of iteration k; [maxit + 1 + k]: max |E|
  int maxit;
  int k;
  double tol;
  Geom g;
  R dt;
  R w[3];
  R az2;
  int hop;
  int zA0, WA, zB0, WB;
  int zlo, zhi;   // slices of the prepare and sweep kernels: the owned ones
  R omega, omc;   // relaxation of this sweep and 1 - omega (exact)
  int check;      // sweeps return at once after convergence (device test)
};

// Link buffer of slot m for a link of direction d in plane (i, j).
template <typename R>
__device__ __forceinline__ const typename V2T<R>::T* slot_buf(const ImplArgs<R>& a, int m, bool zplane, int d) {
  if (zplane && d != 2) return a.Un;
  return m == 0 ? a.X : (m == 1 ? a.Un : a.Up);
}

// Time-averaged force on link i at x from the time slots m_begin..m_end-1
// (0: the iterate of t_{n+1}, 1: t_n, 2: t_{n-1}); the force is linear in
// the slot terms, so the fixed slots 1 and 2 are summed once per step.
template <int NC, typename R>
__device__ void force_implicit(const ImplArgs<R>& a, const SiteNbr& n, int i, R* F, int m_begin, int m_end) {
  typedef LinkAlg<NC, R> G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
#pragma unroll
  for (int c = 0; c < NA; ++c) F[c] = R(0);
  const int64_t pi = n.p[i];
#pragma unroll 1
  for (int j = 0; j < 3; ++j) {
    if (j == i) continue;
    const bool zplane = (i == 2) || (j == 2);
    const bool fwd = (j != 2) || (n.iz <= a.g.nz - 2);
    const bool bwd = (j != 2) || (n.iz >= 1);
    const int64_t pj = n.p[j], mj = n.m[j];
    const R wj = j == 2 ? a.w[2] : a.w[0];
#pragma unroll 1
    for (int m = m_begin; m < m_end; ++m) {
      const typename V2T<R>::T* Bi = slot_buf(a, m, zplane, i);
      const typename V2T<R>::T* Bj = slot_buf(a, m, zplane, j);
      typename G::Sum S = G::zero_sum();
      if (fwd) {
        M T = G::mul_d(LinkIO<NC, R>::template load<R>(Bj, j, a.g.V, pi),
                       LinkIO<NC, R>::template load<R>(Bi, i, a.g.V, pj));
        T = G::mul_d(T, LinkIO<NC, R>::template load<R>(Bj, j, a.g.V, n.s));
        G::sum_add(S, R(1), T);
      }
      if (bwd) {
        // x + e_i - e_j (the wraps of x and y are independent)
        M T = G::mul(LinkIO<NC, R>::template load<R>(Bi, i, a.g.V, mj),
                     LinkIO<NC, R>::template load<R>(Bj, j, a.g.V, pi + mj - n.s));
        T = G::d_mul(T, LinkIO<NC, R>::template load<R>(Bj, j, a.g.V, mj));
        G::sum_add(S, R(1), T);
      }
      R pr[NA];
      G::proj_mul_sum(LinkIO<NC, R>::template load<R>(Bi, i, a.g.V, n.s), S, pr);
      // slot weights 1/4, 1/2, 1/4 for t_{n+1}, t_n, t_{n-1}
      const R wm = wj * (m == 1 ? R(0.5) : R(0.25));
#pragma unroll
      for (int c = 0; c < NA; ++c) F[c] -= wm * pr[c];
    }
  }
}

// U(t_{n-1}) = exp(-i dt E(t_{n-1/2})) U(t_n), when it is not known.
template <int NC, typename R>
__global__ void __launch_bounds__(192) k_implicit_prev(ImplArgs<R> a) {
  typedef LinkAlg<NC, R> G;
  constexpr int NA = G::NA;
  const int i = (int)threadIdx.y;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const int iz = (int)blockIdx.y;
  if (t >= (uint32_t)a.g.nxy) return;
  if (i == 2 && iz == a.g.nz - 1) return;
  const int64_t s = (int64_t)iz * a.g.nxy + t;
  R e[NA];
#pragma unroll
  for (int c = 0; c < NA; ++c) e[c] = a.E[(int64_t)(i * NA + c) * a.g.V + s];
  typename G::M u = G::mul(G::expi_series(e, -a.dt), LinkIO<NC, R>::template load<R>(a.Un, i, a.g.V, s));
  if (sizeof(R) == 4) u = G::reunit(u);
  LinkIO<NC, R>::template store<R>(a.Uout, i, a.g.V, s, u);
}

// Blocks per SM of the prepare and sweep kernels.  FP32: 4 blocks of 192
// threads (80 registers; the load latency of the staples wants the warps
// more than the spilled registers cost).  FP64 needs the registers of one
// block per SM instead of spilling.
template <typename R> struct ImplOcc { static constexpr int blocks = 4; };
template <> struct ImplOcc<double> { static constexpr int blocks = 1; };

// Hop (charges committed, current into Ework), the first iterate and the
// force of the two fixed time slots.  The first iterate is written before
// the staples, so U_n(x) and E(t_{n-1/2}) are not live across them.
template <int NC, typename R>
__device__ __forceinline__ void prep_link(const ImplArgs<R>& a, int i, uint32_t t, int iz) {
  typedef LinkAlg<NC, R> G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
  if (t >= (uint32_t)a.g.nxy) return;
  if (i == 2 && iz == a.g.nz - 1) return;
  const int64_t s = (int64_t)iz * a.g.nxy + t;
  R ew[NA];
  {
    const M Ui = LinkIO<NC, R>::template load<R>(a.Un, i, a.g.V, s);
    R e[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) ew[c] = e[c] = a.E[(int64_t)(i * NA + c) * a.g.V + s];
    if (i == 2 && a.hop) {
      const int kb = iz - a.zB0;
      R dj[NA];
#pragma unroll
      for (int c = 0; c < NA; ++c) dj[c] = R(0);
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
      for (int c = 0; c < NA; ++c) ew[c] += dj[c];
    }
    // X^(0) = exp(i dt E(t_{n-1/2})) U_n
    M u = G::mul(G::expi_series(e, a.dt), Ui);
    if (sizeof(R) == 4) u = G::reunit(u);
    LinkIO<NC, R>::template store<R>(a.Xn, i, a.g.V, s, u);
  }
  R F[NA];
  force_implicit<NC, R>(a, site_nbr_tz(a.g, t, iz), i, F, 1, 3);
#pragma unroll
  for (int c = 0; c < NA; ++c) a.Ework[(int64_t)(i * NA + c) * a.g.V + s] = ew[c] + a.dt * F[c];
}

// Slices per block of the prepare and sweep kernels.  A block marches
// through kImplZ consecutive z slices of its transverse tile, so the links
// of slice z+1 that it reads as neighbours are in L1 when they become its
// own links (the sweep reads two link arrays in the planes containing z):
// 87 -> 70 ms per step of the SU(3) 2048 x 128^2 workload.
constexpr int kImplZ = 16;

// SLAB: the owned slices start at zlo (a whole lattice's at 0, fixed at
// compile time: the offset costs the 80-register sweep 12 B of spills).
template <int NC, typename R, bool SLAB>
__global__ void __launch_bounds__(192, ImplOcc<R>::blocks) k_implicit_prep(ImplArgs<R> a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const int z0 = (SLAB ? a.zlo : 0) + (int)blockIdx.y * kImplZ;
#pragma unroll 1
  for (int k = 0; k < kImplZ && z0 + k < a.zhi; ++k) prep_link<NC, R>(a, (int)threadIdx.y, t, z0 + k);
}

// The z links of a slab's lower halo slice (zlo - 1), as its owner prepares
// them.
template <int NC, typename R>
__global__ void __launch_bounds__(64) k_implicit_prep_halo(ImplArgs<R> a) {
  prep_link<NC, R>(a, 2, blockIdx.x * blockDim.x + threadIdx.x, a.zlo - 1);
}

// Link i at (t, iz) in one sweep: G = Ework + dt F_0(X), E <- (1 - omega) E
// + omega G (omega = 1: E = G exactly), Xn = exp(i dt E) U_n; the largest
// change and the largest E component go to dmax, emax.
template <int NC, typename R>
__device__ __forceinline__ void sweep_link(const ImplArgs<R>& a, int i, uint32_t t, int iz, R& dmax, R& emax) {
  typedef LinkAlg<NC, R> G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
  const SiteNbr n = site_nbr_tz(a.g, t, iz);
  const int64_t s = n.s;
  R F[NA];
  force_implicit<NC, R>(a, n, i, F, 0, 1);
  R e[NA];
#pragma unroll
  for (int c = 0; c < NA; ++c) {
    const int64_t idx = (int64_t)(i * NA + c) * a.g.V + s;
    const R eo = a.E[idx];
    const R g = a.Ework[idx] + a.dt * F[c];
    e[c] = fma(a.omega, g, a.omc * eo);
    const R d = fabs(e[c] - eo);
    dmax = isfinite(d) ? fmax(dmax, d) : R(INFINITY);
    emax = fmax(emax, fabs(e[c]));
    a.E[idx] = e[c];
  }
  M u = G::mul(G::expi_series(e, a.dt), LinkIO<NC, R>::template load<R>(a.Un, i, a.g.V, s));
  if (sizeof(R) == 4) u = G::reunit(u);
  LinkIO<NC, R>::template store<R>(a.Xn, i, a.g.V, s, u);
}

// One fixed-point sweep: E = Ework + dt F_0(X), Xn = exp(i dt E) U_n, where
// Ework already holds E(t_{n-1/2}) + dt J + dt (F_1(U_n) + F_2(U_{n-1})).
template <int NC, typename R, bool SLAB>
__global__ void __launch_bounds__(192, ImplOcc<R>::blocks) k_implicit_iter(ImplArgs<R> a) {
  typedef LinkAlg<NC, R> G;
  typedef typename G::M M;
  constexpr int NA = G::NA;
  if (a.check && a.k > 0 && implicit_converged(a.conv, a.maxit, a.k - 1, a.tol, sizeof(R) == 4)) return;
  // The maxima are taken in the state's precision (the largest change of
  // an FP32 field, rounded once to FP32, is all the convergence test needs)
  // and converted to FP64 once per block: per-element FP64 arithmetic would
  // occupy GB300's narrow FP64 pipe.
  __shared__ R smax[6], semax[6];
  const int i = (int)threadIdx.y;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  R dmax = R(0), emax = R(0);
  const int z0 = (SLAB ? a.zlo : 0) + (int)blockIdx.y * kImplZ;
#pragma unroll 1
  for (int kz = 0; kz < kImplZ && z0 + kz < a.zhi; ++kz) {
    const int iz = z0 + kz;
    if (t >= (uint32_t)a.g.nxy || (i == 2 && iz == a.g.nz - 1)) continue;
    sweep_link<NC, R>(a, i, t, iz, dmax, emax);
  }
  // block max: warp shuffles, then one value per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31, warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) {
    smax[warp] = dmax;
    semax[warp] = emax;
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    R m = smax[0], me = semax[0];
    for (int w = 1; w < (int)(blockDim.x * blockDim.y) / 32; ++w) {
      m = fmax(m, smax[w]);
      me = fmax(me, semax[w]);
    }
    atomicMax((unsigned long long*)&a.conv[a.k], (unsigned long long)__double_as_longlong((double)m));
    atomicMax((unsigned long long*)&a.conv[a.maxit + 1 + a.k], (unsigned long long)__double_as_longlong((double)me));
  }
}

// The z links of a slab's lower halo slice (zlo - 1) in one sweep, as their
// owner evaluates them; their changes belong to the owner's maxima.
template <int NC, typename R>
__global__ void __launch_bounds__(64) k_implicit_iter_halo(ImplArgs<R> a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (uint32_t)a.g.nxy) return;
  R dmax = R(0), emax = R(0);
  sweep_link<NC, R>(a, 2, t, a.zlo - 1, dmax, emax);
}

// Arguments of the prepare and sweep kernels (the iterate buffers and the
// sweep index are set by the caller).
template <typename R>
static ImplArgs<R> impl_args(glasma_ctx* c, bool hop) {
  typedef typename V2T<R>::T V2;
  ImplArgs<R> a;
  a.E = (R*)c->E;
  a.Ework = (R*)c->Ework;
  a.QA = (R*)c->QA;
  a.QB = (R*)c->QB;
  a.conv = c->conv;
  a.tol = c->p.implicit_tol;
  a.maxit = c->p.implicit_max_iter;
  a.k = 0;
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
  a.Up = (const V2*)c->Uprev;
  a.Un = (const V2*)c->U[c->cur];
  a.X = nullptr;
  a.Xn = nullptr;
  a.Uout = nullptr;
  a.zlo = c->lo;
  a.zhi = c->hi;
  a.check = 1;
  a.omega = R(1);
  a.omc = R(0);
  return a;
}

// Relaxation of sweep k (the first takes the full step).
template <typename R>
static void set_relaxation(const glasma_ctx* c, int k, ImplArgs<R>& a) {
  if (k == 0) {
    a.omega = R(1);
    a.omc = R(0);
    return;
  }
  const double cc = 2.0 * c->p.dt * c->p.dt / (c->p.a_t * c->p.a_t);
  a.omega = (R)(2.0 / (2.0 + cc));
  a.omc = R(1) - a.omega;  // exact: omega lies in (0, 1]
}

// 64 transverse sites x the three directions per block; a row of blocks
// per kImplZ owned slices
static dim3 impl_grid(const glasma_ctx* c) {
  return dim3((unsigned)((c->g.nxy + 63) / 64), (unsigned)((c->hi - c->lo + kImplZ - 1) / kImplZ));
}

// U(t_{n-1}) if unknown, the cleared maxima, and the prepare kernel (hop,
// first iterate into U[1 - cur], work field).
template <int NC, typename R>
static int implicit_prepare(glasma_ctx* c, bool hop) {
  typedef typename V2T<R>::T V2;
  ImplArgs<R> a = impl_args<R>(c, hop);
  const dim3 bs(64, 3);
  int st;
  if (!c->uprev_valid) {
    // every local slice, halos included: a lower halo's z link at t_{n-1}
    // follows from its E_z and U_z, which the step's halo brings
    a.Uout = (V2*)c->Uprev;
    const dim3 grid((unsigned)((c->g.nxy + 63) / 64), (unsigned)c->g.nz);
    k_implicit_prev<NC, R><<<grid, bs, 0, c->stream>>>(a);
    st = cuda_check(cudaGetLastError(), "k_implicit_prev launch");
    if (st) return st;
    c->uprev_valid = true;
  }
  st = cuda_check(cudaMemsetAsync(c->conv, 0, sizeof(double) * 2 * (a.maxit + 1), c->stream), "conv clear");
  if (st) return st;
  a.Xn = (V2*)c->U[1 - c->cur];
  if (c->lo > 0)
    k_implicit_prep<NC, R, true><<<impl_grid(c), bs, 0, c->stream>>>(a);
  else
    k_implicit_prep<NC, R, false><<<impl_grid(c), bs, 0, c->stream>>>(a);
  st = cuda_check(cudaGetLastError(), "k_implicit_prep launch");
  if (st || c->lo == 0) return st;
  k_implicit_prep_halo<NC, R><<<(unsigned)((c->g.nxy + 63) / 64), 64, 0, c->stream>>>(a);
  return cuda_check(cudaGetLastError(), "k_implicit_prep_halo launch");
}

// Iterate buffers of sweep k: it reads xa for even k and xb for odd k
// (xa = U[1 - cur] holds the first iterate, xb = Uit) and writes the other.
template <int NC, typename R>
static int implicit_launch_sweep(glasma_ctx* c, bool hop, int k, bool check) {
  typedef typename V2T<R>::T V2;
  ImplArgs<R> a = impl_args<R>(c, hop);
  void* xa = c->U[1 - c->cur];
  void* xb = c->Uit;
  a.k = k;
  a.check = check ? 1 : 0;
  set_relaxation<R>(c, k, a);
  a.X = (const V2*)(k % 2 == 0 ? xa : xb);
  a.Xn = (V2*)(k % 2 == 0 ? xb : xa);
  if (c->lo > 0)
    k_implicit_iter<NC, R, true><<<impl_grid(c), dim3(64, 3), 0, c->stream>>>(a);
  else
    k_implicit_iter<NC, R, false><<<impl_grid(c), dim3(64, 3), 0, c->stream>>>(a);
  int st = cuda_check(cudaGetLastError(), "k_implicit_iter launch");
  if (st || c->lo == 0) return st;
  k_implicit_iter_halo<NC, R><<<(unsigned)((c->g.nxy + 63) / 64), 64, 0, c->stream>>>(a);
  return cuda_check(cudaGetLastError(), "k_implicit_iter_halo launch");
}

// After `done` sweeps: the last iterate becomes U(t_{n+1}), U(t_n) becomes
// U(t_{n-1}), and the old U(t_{n-1}) and the spare iterate buffer are reused.
void implicit_commit(glasma_ctx* c, int done) {
  void* prev = c->Uprev;
  void* now = c->U[c->cur];
  void* xa = c->U[1 - c->cur];
  void* xb = c->Uit;
  // iteration k writes xb for even k and xa for odd k
  void* fin = ((done - 1) % 2 == 0) ? xb : xa;
  void* spare = fin == xa ? xb : xa;
  c->Uprev = now;
  c->U[c->cur] = fin;
  c->U[1 - c->cur] = prev;
  c->Uit = spare;
}

template <int NC, typename R>
static int implicit_t(glasma_ctx* c, bool hop, int* iters) {
  int st = implicit_prepare<NC, R>(c, hop);
  if (st) return st;
  const int maxit = c->p.implicit_max_iter;
  for (int k = 0; k < maxit; ++k) {
    st = implicit_launch_sweep<NC, R>(c, hop, k, true);
    if (st) return st;
  }
  std::vector<double> conv(2 * (maxit + 1));
  st = cuda_check(cudaMemcpyAsync(conv.data(), c->conv, sizeof(double) * conv.size(), cudaMemcpyDeviceToHost,
                                  c->stream),
                  "conv readback");
  if (st) return st;
  st = cuda_check(cudaStreamSynchronize(c->stream), "implicit sync");
  if (st) return st;
  int done = 0;
  bool converged = false;
  for (int k = 0; k < maxit; ++k) {
    done = k + 1;
    if (!isfinite(conv[k])) return set_error(GLASMA_ERR_NONFINITE, "implicit iteration met a non-finite value");
    if (implicit_converged(conv.data(), maxit, k, c->p.implicit_tol, sizeof(R) == 4)) {
      converged = true;
      break;
    }
  }
  *iters = done;
  implicit_commit(c, done);
  if (!converged)
    return set_error(GLASMA_ERR_NOT_CONVERGED, "implicit iteration did not reach implicit_tol within implicit_max_iter");
  return GLASMA_OK;
}

template <int NC, typename R>
static int implicit_sweep_t(glasma_ctx* c, double* dmax, double* emax) {
  const int k = c->impl_k;
  int st = implicit_launch_sweep<NC, R>(c, c->impl_hop, k, false);
  if (st) return st;
  double h[2];
  const int maxit = c->p.implicit_max_iter;
  st = cuda_check(cudaMemcpyAsync(&h[0], c->conv + k, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                  "sweep maximum readback");
  if (!st)
    st = cuda_check(cudaMemcpyAsync(&h[1], c->conv + maxit + 1 + k, sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream),
                    "sweep maximum readback");
  if (!st) st = cuda_check(cudaStreamSynchronize(c->stream), "sweep sync");
  if (st) return st;
  c->impl_k = k + 1;
  *dmax = h[0];
  *emax = h[1];
  return GLASMA_OK;
}

}  // namespace glasma

extern "C" int glasma_implicit_converged(const double* dmax, const double* emax, int k, double tol, int precision,
                                         int* converged) {
  if (!dmax || !emax || !converged || k < 0 || k > 4096 ||
      (precision != GLASMA_FP32 && precision != GLASMA_FP64))
    return glasma::set_error(GLASMA_ERR_INVALID_ARG, "glasma_implicit_converged: bad arguments");
  std::vector<double> conv(2 * ((size_t)k + 1), 0.0);
  for (int j = 0; j <= k; ++j) {
    conv[j] = dmax[j];
    conv[k + 1 + j] = emax[j];
  }
  *converged = glasma::implicit_converged(conv.data(), k, k, tol, precision == GLASMA_FP32) ? 1 : 0;
  return GLASMA_OK;
}

namespace glasma {

int launch_step_implicit(glasma_ctx* c, bool hop, int* iters) {
  if (c->p.nc == 2) return c->rs == 8 ? implicit_t<2, double>(c, hop, iters) : implicit_t<2, float>(c, hop, iters);
  return c->rs == 8 ? implicit_t<3, double>(c, hop, iters) : implicit_t<3, float>(c, hop, iters);
}

int implicit_begin(glasma_ctx* c, bool hop) {
  if (c->p.nc == 2) return c->rs == 8 ? implicit_prepare<2, double>(c, hop) : implicit_prepare<2, float>(c, hop);
  return c->rs == 8 ? implicit_prepare<3, double>(c, hop) : implicit_prepare<3, float>(c, hop);
}

int implicit_sweep(glasma_ctx* c, double* dmax, double* emax) {
  if (c->p.nc == 2)
    return c->rs == 8 ? implicit_sweep_t<2, double>(c, dmax, emax) : implicit_sweep_t<2, float>(c, dmax, emax);
  return c->rs == 8 ? implicit_sweep_t<3, double>(c, dmax, emax) : implicit_sweep_t<3, float>(c, dmax, emax);
}

}  // namespace glasma
