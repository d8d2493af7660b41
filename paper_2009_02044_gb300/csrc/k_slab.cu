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

// links of directions [0, ndir) on slice iz <-> buf[(d*nv + k)*nxy + t]
template <typename V2, bool PACK>
__global__ void k_slab_links(V2* U, int nc, int nv, int64_t V, int64_t nxy, int iz, int ndir, V2* buf) {
  const int64_t n = (int64_t)ndir * nv * nxy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i % nxy, dk = i / nxy;
    const int k = (int)(dk % nv), d = (int)(dk / nv);
    const int64_t e = link_index(nc, d, k, V, (int64_t)iz * nxy + t);
    if (PACK)
      buf[i] = U[e];
    else
      U[e] = buf[i];
  }
}

// comps rows of nxy reals at field[c*stride + off + t] <-> buf[c*nxy + t];
// present = false: the rows do not exist here (pack writes zeros, unpack
// skips)
template <typename R, bool PACK>
__global__ void k_slab_rows(R* field, int comps, int64_t stride, int64_t off, int64_t nxy, bool present, R* buf) {
  const int64_t n = (int64_t)comps * nxy;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i % nxy, c = i / nxy;
    if (PACK)
      buf[i] = present ? field[c * stride + off + t] : R(0);
    else if (present)
      field[c * stride + off + t] = buf[i];
  }
}

static unsigned grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

template <typename R>
static int slab_io(glasma_ctx* c, int dir, void* buf, bool pack) {
  typedef typename V2T<R>::T V2;
  const int64_t nxy = c->g.nxy, V = c->g.V;
  const int na = c->na, nv = c->nv;
  V2* U = (V2*)c->U[c->cur];
  R* b = (R*)buf;
  // dir +1: my top owned slice (pack) or, unpacking a message from below,
  // my lower halo slice; dir -1 likewise the other side
  const bool up_msg = pack ? dir > 0 : dir < 0;
  const int iz = pack ? (dir > 0 ? c->hi - 1 : c->lo) : (dir < 0 ? 0 : c->hi);
  const int ndir = up_msg ? 3 : 2;
  const int64_t nl = (int64_t)ndir * nv * nxy;
  if (pack)
    k_slab_links<V2, true><<<grid_of(nl), 256, 0, c->stream>>>(U, c->p.nc, nv, V, nxy, iz, ndir, (V2*)b);
  else
    k_slab_links<V2, false><<<grid_of(nl), 256, 0, c->stream>>>(U, c->p.nc, nv, V, nxy, iz, ndir, (V2*)b);
  R* rest = b + 2 * nl;
  if (up_msg) {  // E_z of the slice
    const int64_t off = (int64_t)2 * na * V + (int64_t)iz * nxy;
    if (pack)
      k_slab_rows<R, true><<<grid_of(na * nxy), 256, 0, c->stream>>>((R*)c->E, na, V, off, nxy, true, rest);
    else
      k_slab_rows<R, false><<<grid_of(na * nxy), 256, 0, c->stream>>>((R*)c->E, na, V, off, nxy, true, rest);
    rest += (int64_t)na * nxy;
  }
  // the charge of B (up) or A (down) on the slice, if in the window
  R* Q = (R*)(up_msg ? c->QB : c->QA);
  const int z0 = up_msg ? c->zB0 : c->zA0, W = up_msg ? c->WB : c->WA;
  const int k = iz - z0;
  const bool present = k >= 0 && k < W;
  const int64_t stride = (int64_t)W * nxy, off = present ? (int64_t)k * nxy : 0;
  if (pack)
    k_slab_rows<R, true><<<grid_of(na * nxy), 256, 0, c->stream>>>(Q, na, stride, off, nxy, present, rest);
  else
    k_slab_rows<R, false><<<grid_of(na * nxy), 256, 0, c->stream>>>(Q, na, stride, off, nxy, present, rest);
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
