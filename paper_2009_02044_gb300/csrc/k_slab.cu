// Halo messages of a lattice split into z slabs (the beam axis, Sec. 4's
// long axis), and the hop of the charge that crosses into a slab from below.
//
// A slab context holds its owned slices [lo, hi) and one halo slice on each
// side that has a neighbour (local slice 0 below, local slice hi above).
// Before every step each rank sends
//   up   (dir +1, to the rank above, from slice hi - 1): the links of all
//        three directions, E_z, and nucleus B's charge on that slice;
//   down (dir -1, to the rank below, from slice lo): the transverse links
//        and nucleus A's charge on that slice;
// and writes what it receives into its halo slices.  Message layout (reals
// of the state's precision, x fastest within a slice): the links as
// [direction][complex component][site] (re, im) pairs in their stored form,
// then E_z as [colour][site] (up only), then the charge as [colour][site]
// (zeros when the slice lies outside that nucleus' window).
//
// The charge of B on the lower halo slice moves into the slab at the next
// hop along the halo's z link: k_slab_halo_hop transports it in place with
// the same arithmetic the owner of that link applies (update_link), so the
// slab holds bitwise the charge the whole lattice would.
#include "step_link.cuh"

namespace glasma {

size_t slab_msg_elems(const glasma_ctx* c, int dir) {
  const size_t nxy = (size_t)c->g.nxy;
  const int nv = c->nv, na = c->na;
  return dir > 0 ? (size_t)(3 * 2 * nv + 2 * na) * nxy : (size_t)(2 * 2 * nv + na) * nxy;
}

// One message <-> its slice, in one launch: work item i < nl is a link
// component (V2 units), buf[i] <-> U at link (d, k) of site iz*nxy + t with
// i = (d*nv + k)*nxy + t; the items after it are reals, first the E_z rows
// (up messages), E[c*V + e_off + t], then the charge rows Q[c*q_stride +
// q_off + t].  A charge slice outside the nucleus' window is not present:
// pack writes zeros, unpack skips it.
template <typename R>
struct SlabIOArgs {
  typename V2T<R>::T* U;
  R* E;
  R* Q;
  R* buf;
  int64_t V, nxy, nl, e_off, q_stride, q_off;
  int nc, nv, na, iz;
  int has_e, q_present;
};

template <typename R, bool PACK>
__global__ void k_slab_io(SlabIOArgs<R> a) {
  typedef typename V2T<R>::T V2;
  const int64_t nrows = (int64_t)(a.has_e ? 2 : 1) * a.na * a.nxy;
  const int64_t n = a.nl + nrows;
  V2* lb = (V2*)a.buf;
  R* rb = a.buf + 2 * a.nl;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < a.nl) {
      const int64_t t = i % a.nxy, dk = i / a.nxy;
      const int k = (int)(dk % a.nv), d = (int)(dk / a.nv);
      const int64_t e = link_index(a.nc, d, k, a.V, (int64_t)a.iz * a.nxy + t);
      if (PACK)
        lb[i] = a.U[e];
      else
        a.U[e] = lb[i];
    } else {
      const int64_t j = i - a.nl;
      const int64_t t = j % a.nxy;
      const int64_t c = j / a.nxy;
      if (a.has_e && c < a.na) {
        R* f = a.E + c * a.V + a.e_off + t;
        if (PACK)
          rb[j] = *f;
        else
          *f = rb[j];
      } else {
        const int64_t cq = a.has_e ? c - a.na : c;
        if (PACK)
          rb[j] = a.q_present ? a.Q[cq * a.q_stride + a.q_off + t] : R(0);
        else if (a.q_present)
          a.Q[cq * a.q_stride + a.q_off + t] = rb[j];
      }
    }
  }
}

static unsigned grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

template <typename R>
static int slab_io(glasma_ctx* c, int dir, void* buf, bool pack) {
  SlabIOArgs<R> a;
  a.nxy = c->g.nxy;
  a.V = c->g.V;
  a.na = c->na;
  a.nv = c->nv;
  a.nc = c->p.nc;
  a.U = (typename V2T<R>::T*)c->U[c->cur];
  a.E = (R*)c->E;
  a.buf = (R*)buf;
  // dir +1: my top owned slice (pack) or, unpacking a message from below,
  // my lower halo slice; dir -1 likewise the other side
  const bool up_msg = pack ? dir > 0 : dir < 0;
  a.iz = pack ? (dir > 0 ? c->hi - 1 : c->lo) : (dir < 0 ? 0 : c->hi);
  const int ndir = up_msg ? 3 : 2;
  a.nl = (int64_t)ndir * a.nv * a.nxy;
  a.has_e = up_msg ? 1 : 0;  // E_z of the slice
  a.e_off = (int64_t)2 * a.na * a.V + (int64_t)a.iz * a.nxy;
  // the charge of B (up) or A (down) on the slice, if in the window
  a.Q = (R*)(up_msg ? c->QB : c->QA);
  const int z0 = up_msg ? c->zB0 : c->zA0, W = up_msg ? c->WB : c->WA;
  const int k = a.iz - z0;
  a.q_present = (k >= 0 && k < W) ? 1 : 0;
  a.q_stride = (int64_t)W * a.nxy;
  a.q_off = a.q_present ? (int64_t)k * a.nxy : 0;
  const int64_t n = a.nl + (int64_t)(a.has_e ? 2 : 1) * a.na * a.nxy;
  if (pack)
    k_slab_io<R, true><<<grid_of(n), 256, 0, c->stream>>>(a);
  else
    k_slab_io<R, false><<<grid_of(n), 256, 0, c->stream>>>(a);
  return cuda_check(cudaGetLastError(), pack ? "slab pack" : "slab unpack");
}

int slab_pack(glasma_ctx* c, int dir, void* buf) {
  return c->rs == 8 ? slab_io<double>(c, dir, buf, true) : slab_io<float>(c, dir, buf, true);
}

int slab_unpack(glasma_ctx* c, int dir, const void* buf) {
  return c->rs == 8 ? slab_io<double>(c, dir, (void*)buf, false) : slab_io<float>(c, dir, (void*)buf, false);
}

// Q' = U_z^dag Q U_z for nucleus B's charge on local slice 0, in place
template <int NC, typename R>
__global__ void k_slab_halo_hop(const typename V2T<R>::T* U, R* QB, Geom g, int WB, int kb) {
  typedef LinkAlg<NC, R> G;
  constexpr int NA = G::NA;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.nxy; t += (int64_t)gridDim.x * blockDim.x) {
    const typename G::M Ui = LinkIO<NC, R>::template load<R>(U, 2, g.V, t);
    R q[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) q[c] = QB[((int64_t)c * WB + kb) * g.nxy + t];
    G::adj_dag(Ui, q);
#pragma unroll
    for (int c = 0; c < NA; ++c) QB[((int64_t)c * WB + kb) * g.nxy + t] = q[c];
  }
}

template <int NC, typename R>
static int halo_hop_t(glasma_ctx* c) {
  const int kb = 0 - c->zB0;
  if (kb < 0 || kb >= c->WB) return GLASMA_OK;  // no charge of B there
  k_slab_halo_hop<NC, R><<<grid_of(c->g.nxy), 256, 0, c->stream>>>((const typename V2T<R>::T*)c->U[c->cur],
                                                                  (R*)c->QB, c->g, c->WB, kb);
  return cuda_check(cudaGetLastError(), "slab halo hop");
}

int slab_halo_hop(glasma_ctx* c) {
  if (c->p.nc == 2) return c->rs == 8 ? halo_hop_t<2, double>(c) : halo_hop_t<2, float>(c);
  return c->rs == 8 ? halo_hop_t<3, double>(c) : halo_hop_t<3, float>(c);
}

}  // namespace glasma
