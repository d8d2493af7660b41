// C ABI of the Glasma library: context life cycle, parameter checks, the
// host-side hop schedule and charge-window bookkeeping, field and checkpoint
// transfer.  Every compute step runs in the kernels of k_*.cu.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "glasma_internal.cuh"

namespace glasma {

static thread_local std::string g_last_error;

int set_error(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GLASMA_OK;
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GLASMA_ERR_OOM : GLASMA_ERR_CUDA;
}

void* ctx_alloc(glasma_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (c->has_alloc) {
    p = c->alloc.alloc(bytes, (void*)c->stream, c->alloc.user);
  } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->allocs.push_back({p, bytes});
  return p;
}

void ctx_free(glasma_ctx* c, void* p) {
  if (!p) return;
  for (size_t k = 0; k < c->allocs.size(); ++k) {
    if (c->allocs[k].ptr == p) {
      if (c->has_alloc)
        c->alloc.free(p, c->allocs[k].bytes, (void*)c->stream, c->alloc.user);
      else
        cudaFreeAsync(p, c->stream);
      c->allocs.erase(c->allocs.begin() + k);
      return;
    }
  }
}

uint32_t crc32(const void* data, size_t n, uint32_t crc) {
  static uint32_t table[256];
  static bool ready = false;
  if (!ready) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t r = i;
      for (int k = 0; k < 8; ++k) r = (r & 1) ? (r >> 1) ^ 0xEDB88320u : r >> 1;
      table[i] = r;
    }
    ready = true;
  }
  const unsigned char* b = (const unsigned char*)data;
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = table[(crc ^ b[i]) & 0xFFu] ^ (crc >> 8);
  return ~crc;
}

// dt * q == a_z * p exactly, comparing the doubles' integer mantissas in
// 128-bit arithmetic
static bool exact_ratio(double dt, double a_z, long long p, long long q) {
  int e1, e2;
  const double f1 = frexp(dt, &e1), f2 = frexp(a_z, &e2);
  const long long m1 = (long long)ldexp(f1, 53), m2 = (long long)ldexp(f2, 53);
  __int128 a = (__int128)m1 * q, b = (__int128)m2 * p;
  const int d = e1 - e2;
  if (d > 60 || d < -60) return false;
  if (d > 0) a <<= d;
  if (d < 0) b <<= -d;
  return a == b;
}

// v dt / a_z = p / q exactly, with the smallest q <= 4096
static bool hop_ratio(double dt, double a_z, long long* p, long long* q) {
  for (long long qq = 1; qq <= 4096; ++qq) {
    double pp = nearbyint(dt * (double)qq / a_z);
    if (pp >= 1.0 && exact_ratio(dt, a_z, (long long)pp, qq)) {
      *p = (long long)pp;
      *q = qq;
      return true;
    }
  }
  return false;
}

static int check_params(const glasma_params* p) {
  if (!p) return set_error(GLASMA_ERR_INVALID_ARG, "params is NULL");
  if (p->nc != 2 && p->nc != 3) return set_error(GLASMA_ERR_INVALID_ARG, "nc must be 2 or 3");
  if (p->nz < 2 || p->nx < 1 || p->ny < 1) return set_error(GLASMA_ERR_INVALID_ARG, "need nz >= 2, nx, ny >= 1");
  if ((double)p->nz * p->nx * p->ny > 1.5e9) return set_error(GLASMA_ERR_INVALID_ARG, "lattice too large");
  if (p->nz > 65535) return set_error(GLASMA_ERR_INVALID_ARG, "nz must be <= 65535 (one grid row per slice)");
  if (!(p->a_t > 0) || !(p->a_z > 0) || !(p->dt > 0))
    return set_error(GLASMA_ERR_INVALID_ARG, "a_t, a_z, dt must be positive");
  if (p->dt > p->a_z) return set_error(GLASMA_ERR_INVALID_ARG, "dt > a_z: a charge would cross several cells");
  long long hp, hq;
  if (!hop_ratio(p->dt, p->a_z, &hp, &hq))
    return set_error(GLASMA_ERR_INVALID_ARG, "dt / a_z must be an exact ratio p/q with q <= 4096");
  if (!(p->sigma_l > 0)) return set_error(GLASMA_ERR_INVALID_ARG, "sigma_l must be positive");
  if (!(p->m_ir > 0)) return set_error(GLASMA_ERR_INVALID_ARG, "m_ir must be positive");
  if (!(p->g2mu >= 0)) return set_error(GLASMA_ERR_INVALID_ARG, "g2mu must be >= 0");
  if (!(p->uv_cutoff >= 0) || !(p->z_offset >= 0))
    return set_error(GLASMA_ERR_INVALID_ARG, "uv_cutoff and z_offset must be >= 0");
  if (p->precision != GLASMA_FP64 && p->precision != GLASMA_FP32)
    return set_error(GLASMA_ERR_INVALID_ARG, "precision must be GLASMA_FP64 or GLASMA_FP32");
  if (p->scheme != GLASMA_LEAPFROG && p->scheme != GLASMA_IMPLICIT)
    return set_error(GLASMA_ERR_INVALID_ARG, "scheme must be GLASMA_LEAPFROG or GLASMA_IMPLICIT");
  if (p->n_sheets < 0 || p->n_sheets > 64) return set_error(GLASMA_ERR_INVALID_ARG, "n_sheets must be 0..64");
  if (p->scheme == GLASMA_IMPLICIT && (p->implicit_max_iter < 1 || !(p->implicit_tol > 0)))
    return set_error(GLASMA_ERR_INVALID_ARG, "implicit scheme needs max_iter >= 1 and tol > 0");
  // both truncated profiles (at t0 and t0 - dt) inside the box
  const double zc = p->nz * p->a_z / 2.0;
  const double d = p->z_offset > 0 ? p->z_offset : (ceil(4.0 * p->sigma_l / p->a_z) + 2.0) * p->a_z;
  if (d <= 4.0 * p->sigma_l) return set_error(GLASMA_ERR_INVALID_ARG, "z_offset must exceed 4 sigma_l");
  if (zc - d - p->dt - 4.0 * p->sigma_l < 0.0 || zc + d + p->dt + 4.0 * p->sigma_l > (p->nz - 1) * p->a_z)
    return set_error(GLASMA_ERR_INVALID_ARG, "nuclei do not fit inside the box");
  return GLASMA_OK;
}

// The automatic choice, from CUDA-event timings on GB300: in FP64 the
// plaquette kernel (24% fewer FMAs, and the FP64 pipe bounds the step:
// 12.8 against 15.3 ms per SU(3) 512 x 64^2 step); in FP32 SU(3) with rows
// of 64 sites the staged staple kernel (0.446-0.449 ms against 0.472-0.475
// for the one-site staple kernel, bitwise the same result), else the staple
// kernel (0.469 ms, against 0.521 for the plaquette kernel and 0.572 for
// site pairs, whose 168 registers leave too few warps to hide latency); in
// FP32 SU(2) the staple kernel too (1.10 against 1.39 ms for site pairs per
// 1024 x 128^2 step, once a link's alpha and beta became one 16-byte load:
// the pairs' 32-bit loads then stride 16 bytes).
bool use_plaq_kernel(const glasma_ctx* c) {
  if (c->step_kernel == GLASMA_KERNEL_PLAQUETTE || c->step_kernel == GLASMA_KERNEL_PLAQUETTE_256) return plaq_fits(c);
  return c->step_kernel == GLASMA_KERNEL_AUTO && c->rs == 8 && plaq_fits(c);
}

bool use_pair_kernel(const glasma_ctx* c) {
  if (c->rs != 4 || c->slab) return false;  // the pairs span the whole z range
  return c->step_kernel == GLASMA_KERNEL_STAPLE_PAIRS;
}

bool use_staged_kernel(const glasma_ctx* c) {
  if (c->step_kernel == GLASMA_KERNEL_STAPLE_STAGED) return staged_fits(c);
  return c->step_kernel == GLASMA_KERNEL_AUTO && staged_fits(c) && c->g.nx == 64;
}

int launch_step_chosen(glasma_ctx* c, bool hop) {
  if (use_plaq_kernel(c)) return launch_step_plaq(c, hop, c->step_zlen);
  if (use_pair_kernel(c)) return launch_step_pair(c, hop);
  if (use_staged_kernel(c)) return launch_step_staged(c, hop);
  return launch_step_leapfrog(c, hop);
}

}  // namespace glasma

using namespace glasma;

extern "C" {

const char* glasma_strerror(int status) {
  switch (status) {
    case GLASMA_OK: return "ok";
    case GLASMA_ERR_INVALID_ARG: return "invalid argument";
    case GLASMA_ERR_CUDA: return "CUDA error";
    case GLASMA_ERR_OOM: return "out of device memory";
    case GLASMA_ERR_NONFINITE: return "non-finite value";
    case GLASMA_ERR_PARTICLE_EXIT: return "charge would leave the lattice";
    case GLASMA_ERR_NOT_CONVERGED: return "implicit iteration not converged";
    case GLASMA_ERR_TIMEOUT: return "device wait timed out";
    case GLASMA_ERR_CHECKSUM: return "checkpoint checksum mismatch";
    case GLASMA_ERR_INTERNAL: return "internal error";
    default: return "unknown status";
  }
}

const char* glasma_last_error_message(void) { return g_last_error.c_str(); }

void glasma_free(glasma_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  while (!c->allocs.empty()) ctx_free(c, c->allocs.back().ptr);
  cudaStreamSynchronize(c->stream);
  delete c;
}

}  // extern "C"

// A context over the global slices [z0, z1) of the lattice p describes,
// plus one halo slice on each side that has a neighbour (the whole lattice
// when z0 = 0, z1 = nz).  The context's own lattice is the local one: its
// params carry the local nz, the open-z rules apply at its ends.
static int create_ctx(const glasma_params* p, const double* rho_host, void* stream, const glasma_allocator* alloc,
                      int z0, int z1, glasma_ctx** out) {
  if (!out) return set_error(GLASMA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int st = check_params(p);
  if (st) return st;
  if (z0 < 0 || z1 > p->nz || z1 <= z0) return set_error(GLASMA_ERR_INVALID_ARG, "slab range outside the lattice");
  const int halo_lo = z0 > 0 ? 1 : 0, halo_hi = z1 < p->nz ? 1 : 0;
  const int nz_loc = (z1 - z0) + halo_lo + halo_hi;
  if (nz_loc < 2) return set_error(GLASMA_ERR_INVALID_ARG, "a slab lattice needs at least two slices");
  glasma_ctx* c = new glasma_ctx();
  c->p = *p;
  c->p.nz = nz_loc;
  c->slab = !(z0 == 0 && z1 == p->nz);
  c->zoff = z0 - halo_lo;
  c->lo = halo_lo;
  c->hi = halo_lo + (z1 - z0);
  c->nz_glob = p->nz;
  p = &c->p;
  cudaGetDevice(&c->device);
  c->stream = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  c->na = p->nc * p->nc - 1;
  c->nv = p->nc == 2 ? 2 : 9;
  c->g.nx = p->nx;
  c->g.ny = p->ny;
  c->g.nz = p->nz;
  c->g.nxy = (int64_t)p->nx * p->ny;
  c->g.V = c->g.nxy * p->nz;
  c->rs = p->precision == GLASMA_FP64 ? 8 : 4;
  hop_ratio(p->dt, p->a_z, &c->hop_p, &c->hop_q);
  const size_t ub = link_bytes(c);
  const size_t eb = c->rs * 3 * (size_t)c->na * c->g.V;
  c->U[0] = ctx_alloc(c, ub);
  c->U[1] = ctx_alloc(c, ub);
  c->E = ctx_alloc(c, eb);
  if (p->scheme == GLASMA_IMPLICIT) {
    c->Uprev = ctx_alloc(c, ub);
    c->Uit = ctx_alloc(c, ub);
    c->Ework = ctx_alloc(c, eb);
    c->conv = (double*)ctx_alloc(c, sizeof(double) * 2 * (p->implicit_max_iter + 1));
  }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  c->red_cap = (size_t)sms * 4 * 8 + 64;
  c->red = (double*)ctx_alloc(c, sizeof(double) * c->red_cap);
  c->tab = (double*)ctx_alloc(c, sizeof(double) * 4 * p->nz);
  c->tpart = (double*)ctx_alloc(c, sizeof(double) * 5 * kTmunuSplit * p->nz);
  c->dflag = (int*)ctx_alloc(c, sizeof(int) * 8);
  if (!c->U[0] || !c->U[1] || !c->E || !c->red || !c->tab || !c->tpart || !c->dflag ||
      (p->scheme == GLASMA_IMPLICIT && (!c->Uprev || !c->Uit || !c->Ework || !c->conv))) {
    glasma_free(c);
    return set_error(GLASMA_ERR_OOM, "state allocation failed");
  }
  {
    // vector loads of links and fields need 16-byte aligned buffers
    const void* need[6] = {c->U[0], c->U[1], c->E, c->Uprev, c->Uit, c->Ework};
    for (int k = 0; k < 6; ++k)
      if (((uintptr_t)need[k] & 15) != 0) {
        glasma_free(c);
        return set_error(GLASMA_ERR_INVALID_ARG, "the allocator must return 16-byte aligned memory");
      }
  }
  if (link_elems(p->nc, c->g.V) != (int64_t)3 * c->nv * c->g.V) {
    // SU(3) pads the last block of 32 sites of each direction: zero it, so
    // state blobs hold no uninitialised bytes
    void* lb[4] = {c->U[0], c->U[1], c->Uprev, c->Uit};
    for (int k = 0; k < 4 && !st; ++k)
      if (lb[k]) st = cuda_check(cudaMemsetAsync(lb[k], 0, ub, c->stream), "link padding clear");
    if (st) {
      glasma_free(c);
      return st;
    }
  }
  st = run_init(c, rho_host);
  if (st) {
    std::string keep = g_last_error;
    glasma_free(c);
    g_last_error = keep;
    return st;
  }
  *out = c;
  return GLASMA_OK;
}

extern "C" {

int glasma_init_mv(const glasma_params* p, const double* rho_host, void* stream, const glasma_allocator* alloc,
                   glasma_ctx** out) {
  if (!p) return set_error(GLASMA_ERR_INVALID_ARG, "params is NULL");
  return create_ctx(p, rho_host, stream, alloc, 0, p->nz, out);
}

int glasma_slab_init(const glasma_params* p, const double* rho_host, int z0, int z1, void* stream,
                     const glasma_allocator* alloc, glasma_ctx** out) {
  if (!p) return set_error(GLASMA_ERR_INVALID_ARG, "params is NULL");
  return create_ctx(p, rho_host, stream, alloc, z0, z1, out);
}

int glasma_step(glasma_ctx* c, int n_steps) {
  if (!c || n_steps < 0) return set_error(GLASMA_ERR_INVALID_ARG, "bad context or n_steps");
  if (c->slab && !c->slab_windows)
    return set_error(GLASMA_ERR_INVALID_ARG, "a slab context needs glasma_slab_set_windows before stepping");
  if (c->slab && n_steps > 1)
    return set_error(GLASMA_ERR_INVALID_ARG, "a slab context takes one step per halo exchange");
  if (c->slab && c->p.scheme == GLASMA_IMPLICIT)
    return set_error(GLASMA_ERR_INVALID_ARG,
                     "a slab context takes the improved step sweep by sweep (glasma_implicit_begin/_sweep/_end)");
  if (c->impl_active) return set_error(GLASMA_ERR_INVALID_ARG, "an improved step is in progress (glasma_implicit_end)");
  cudaSetDevice(c->device);
  int launches = 0;
  for (int k = 0; k < n_steps; ++k) {
    const bool hop = hop_at(c->n, c->hop_p, c->hop_q);
    if (hop) {
      // in global slices (a slab's windows are the whole lattice's)
      if (c->WB > 0 && c->zB0 + c->zoff + c->WB - 1 >= c->nz_glob - 1)
        return set_error(GLASMA_ERR_PARTICLE_EXIT, "nucleus B reached the upper z boundary");
      if (c->WA > 0 && c->zA0 + c->zoff <= 0)
        return set_error(GLASMA_ERR_PARTICLE_EXIT, "nucleus A reached the lower z boundary");
    }
    int st;
    if (hop && c->lo > 0) {
      // the charge of B on the lower halo slice crosses into the slab
      st = slab_halo_hop(c);
      if (st) return st;
      launches += 1;
    }
    if (c->p.scheme == GLASMA_IMPLICIT) {
      int iters = 0;
      st = launch_step_implicit(c, hop, &iters);
      c->last_iters = iters;
      launches += iters + 1;
    } else {
      st = launch_step_chosen(c, hop);
      launches += 1;
    }
    // a step that did not converge has still been taken (last iterate kept)
    if (st && st != GLASMA_ERR_NOT_CONVERGED) return st;
    if (c->p.scheme != GLASMA_IMPLICIT) c->cur = 1 - c->cur;  // the implicit launcher rotates its buffers
    if (hop) {
      c->zB0 += 1;
      c->zA0 -= 1;
    }
    c->n += 1;
    if (st) {
      c->last_launches = launches;
      return st;
    }
  }
  c->last_launches = launches;
  return GLASMA_OK;
}

// Between glasma_implicit_begin and _end the fields are mid-iteration (E is
// iterated in place): calls that read or replace the state wait for _end.
static int reject_open_step(const glasma_ctx* c) {
  if (c->impl_active)
    return set_error(GLASMA_ERR_INVALID_ARG, "an improved step is in progress (glasma_implicit_end first)");
  return GLASMA_OK;
}

// exit checks of a hop step, in global slices (a slab's windows are the
// whole lattice's)
static int hop_exit_check(const glasma_ctx* c) {
  if (c->WB > 0 && c->zB0 + c->zoff + c->WB - 1 >= c->nz_glob - 1)
    return set_error(GLASMA_ERR_PARTICLE_EXIT, "nucleus B reached the upper z boundary");
  if (c->WA > 0 && c->zA0 + c->zoff <= 0)
    return set_error(GLASMA_ERR_PARTICLE_EXIT, "nucleus A reached the lower z boundary");
  return GLASMA_OK;
}

int glasma_implicit_begin(glasma_ctx* c) {
  if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "context is NULL");
  if (c->p.scheme != GLASMA_IMPLICIT) return set_error(GLASMA_ERR_INVALID_ARG, "the context runs the leapfrog scheme");
  if (c->impl_active) return set_error(GLASMA_ERR_INVALID_ARG, "an improved step is already in progress");
  if (c->slab && !c->slab_windows)
    return set_error(GLASMA_ERR_INVALID_ARG, "a slab context needs glasma_slab_set_windows before stepping");
  cudaSetDevice(c->device);
  const bool hop = hop_at(c->n, c->hop_p, c->hop_q);
  int st = hop ? hop_exit_check(c) : GLASMA_OK;
  if (!st) st = implicit_begin(c, hop);
  if (st) return st;
  c->impl_active = true;
  c->impl_hop = hop;
  c->impl_k = 0;
  return GLASMA_OK;
}

int glasma_implicit_sweep(glasma_ctx* c, double* dmax, double* emax) {
  if (!c || !dmax || !emax) return set_error(GLASMA_ERR_INVALID_ARG, "bad arguments");
  if (!c->impl_active) return set_error(GLASMA_ERR_INVALID_ARG, "no improved step in progress (glasma_implicit_begin)");
  if (c->impl_k >= c->p.implicit_max_iter)
    return set_error(GLASMA_ERR_NOT_CONVERGED, "implicit_max_iter sweeps already done in this step");
  cudaSetDevice(c->device);
  return implicit_sweep(c, dmax, emax);
}

int glasma_implicit_end(glasma_ctx* c) {
  if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "context is NULL");
  if (!c->impl_active || c->impl_k < 1)
    return set_error(GLASMA_ERR_INVALID_ARG, "no improved step with at least one sweep in progress");
  implicit_commit(c, c->impl_k);
  if (c->impl_hop) {
    c->zB0 += 1;
    c->zA0 -= 1;
  }
  c->n += 1;
  c->last_iters = c->impl_k;
  c->last_launches = c->impl_k + 1;
  c->impl_active = false;
  return GLASMA_OK;
}

int glasma_gauss_residual(glasma_ctx* c, double* max_abs, double* rms, double* rho_max) {
  if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "context is NULL");
  if (reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  double r[3];
  int st = launch_gauss(c, r);
  if (st && st != GLASMA_ERR_NONFINITE) return st;
  if (max_abs) *max_abs = r[0];
  if (rms) *rms = r[1];
  if (rho_max) *rho_max = r[2];
  const int ss = staged_status(c);
  return ss ? ss : st;
}

int glasma_tmunu(glasma_ctx* c, double* out, double* energy_total) {
  if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "context is NULL");
  if (reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  const bool hop = hop_at(c->n, c->hop_p, c->hop_q);
  std::vector<double> tab(4 * (size_t)c->g.nz);
  int st = launch_tmunu(c, hop, tab.data());
  if (st) return st;
  // the owned slices (all of them for a whole lattice)
  double sum = 0.0;
  bool bad = false;
  for (int iz = c->lo; iz < c->hi; ++iz) {
    for (int k = 0; k < 4; ++k)
      if (!isfinite(tab[4 * iz + k])) bad = true;
    sum += tab[4 * iz];
  }
  if (out) memcpy(out, tab.data() + 4 * (size_t)c->lo, sizeof(double) * 4 * (size_t)(c->hi - c->lo));
  if (energy_total) *energy_total = c->p.a_t * c->p.a_t * c->p.a_z * (double)c->g.nxy * sum;
  st = staged_status(c);
  if (st) return st;
  if (bad) return set_error(GLASMA_ERR_NONFINITE, "T^{mu nu} met a non-finite value");
  return GLASMA_OK;
}

int glasma_tmunu_device(glasma_ctx* c, double* dev_out) {
  if (!c || !dev_out) return set_error(GLASMA_ERR_INVALID_ARG, "context or dev_out is NULL");
  if (((uintptr_t)dev_out & 7) != 0) return set_error(GLASMA_ERR_INVALID_ARG, "dev_out must be 8-byte aligned");
  if (reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  return launch_tmunu(c, hop_at(c->n, c->hop_p, c->hop_q), nullptr, dev_out);
}

// ---------------------------------------------------------------------------
// fields in FP64 (host marshalling of the device layout)
// ---------------------------------------------------------------------------

// FP32 storage holds U - 1 (deviation form, see link_alg.cuh): the
// identity is added on the way out and removed (in FP64) on the way in.
static void link_to_matrix(const glasma_ctx* c, const double* comp, double* m) {
  // comp: NV complex (re, im); m: nc x nc complex (re, im)
  const double one = c->rs == 4 ? 1.0 : 0.0;
  if (c->p.nc == 3) {
    memcpy(m, comp, sizeof(double) * 18);
    m[0] += one;
    m[8] += one;
    m[16] += one;
    return;
  }
  const double ar = comp[0] + one, ai = comp[1], br = comp[2], bi = comp[3];
  m[0] = ar;  m[1] = ai;   // alpha
  m[2] = br;  m[3] = bi;   // beta
  m[4] = -br; m[5] = bi;   // -conj(beta)
  m[6] = ar;  m[7] = -ai;  // conj(alpha)
}

static void matrix_to_link(const glasma_ctx* c, const double* m, double* comp) {
  const double one = c->rs == 4 ? 1.0 : 0.0;
  if (c->p.nc == 3) {
    memcpy(comp, m, sizeof(double) * 18);
    comp[0] -= one;
    comp[8] -= one;
    comp[16] -= one;
    return;
  }
  comp[0] = m[0] - one;
  comp[1] = m[1];
  comp[2] = m[2];
  comp[3] = m[3];
}

}  // extern "C"

template <typename T>
static int dl(glasma_ctx* c, std::vector<T>& h, const void* d, size_t count) {
  h.resize(count);
  int st = cuda_check(cudaMemcpyAsync(h.data(), d, sizeof(T) * count, cudaMemcpyDeviceToHost, c->stream), "D2H");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(c->stream), "D2H sync");
}

extern "C" {

// device link array (storage precision) -> host doubles, element for element
// in the device order (see link_index)
static int links_to_host(glasma_ctx* c, const void* dev, std::vector<double>& out) {
  const size_t n = 2 * (size_t)link_elems(c->p.nc, c->g.V);
  out.resize(n);
  if (c->rs == 8) {
    std::vector<double> raw;
    int st = dl(c, raw, dev, n);
    if (st) return st;
    out.swap(raw);
  } else {
    std::vector<float> raw;
    int st = dl(c, raw, dev, n);
    if (st) return st;
    for (size_t i = 0; i < n; ++i) out[i] = raw[i];
  }
  return GLASMA_OK;
}

static int reals_to_host(glasma_ctx* c, const void* dev, size_t n, std::vector<double>& out) {
  out.resize(n);
  if (n == 0) return GLASMA_OK;
  if (c->rs == 8) {
    std::vector<double> raw;
    int st = dl(c, raw, dev, n);
    if (st) return st;
    out.swap(raw);
  } else {
    std::vector<float> raw;
    int st = dl(c, raw, dev, n);
    if (st) return st;
    for (size_t i = 0; i < n; ++i) out[i] = raw[i];
  }
  return GLASMA_OK;
}

static int reals_to_dev(glasma_ctx* c, void* dev, const double* h, size_t n) {
  if (n == 0) return GLASMA_OK;
  int st;
  if (c->rs == 8) {
    st = cuda_check(cudaMemcpyAsync(dev, h, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "H2D");
    if (st) return st;
    return cuda_check(cudaStreamSynchronize(c->stream), "H2D sync");
  }
  std::vector<float> f(n);
  for (size_t i = 0; i < n; ++i) f[i] = (float)h[i];
  st = cuda_check(cudaMemcpyAsync(dev, f.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->stream), "H2D");
  if (st) return st;
  return cuda_check(cudaStreamSynchronize(c->stream), "H2D sync");
}

int glasma_get_fields(glasma_ctx* c, double* U, double* E, double* QA, double* QB, long long* step_n) {
  if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "context is NULL");
  if (reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  const int64_t V = c->g.V, nxy = c->g.nxy;
  const int nc = c->p.nc, na = c->na, nv = c->nv;
  int st;
  if (U) {
    std::vector<double> raw;
    st = links_to_host(c, c->U[c->cur], raw);
    if (st) return st;
    double comp[18];
    for (int d = 0; d < 3; ++d)
      for (int64_t s = 0; s < V; ++s) {
        for (int k = 0; k < nv; ++k) {
          const size_t at = 2 * (size_t)link_index(nc, d, k, V, s);
          comp[2 * k] = raw[at];
          comp[2 * k + 1] = raw[at + 1];
        }
        link_to_matrix(c, comp, U + ((size_t)d * V + s) * nc * nc * 2);
      }
  }
  if (E) {
    std::vector<double> raw;
    st = reals_to_host(c, c->E, 3 * (size_t)na * V, raw);
    if (st) return st;
    for (int d = 0; d < 3; ++d)
      for (int64_t s = 0; s < V; ++s)
        for (int a = 0; a < na; ++a) E[((size_t)d * V + s) * na + a] = raw[((size_t)d * na + a) * V + s];
  }
  const void* qd[2] = {c->QA, c->QB};
  double* qh[2] = {QA, QB};
  const int z0[2] = {c->zA0, c->zB0}, W[2] = {c->WA, c->WB};
  for (int N = 0; N < 2; ++N) {
    if (!qh[N]) continue;
    memset(qh[N], 0, sizeof(double) * (size_t)V * na);
    std::vector<double> raw;
    st = reals_to_host(c, qd[N], (size_t)na * W[N] * nxy, raw);
    if (st) return st;
    for (int a = 0; a < na; ++a)
      for (int w = 0; w < W[N]; ++w) {
        const int iz = z0[N] + w;  // a slab's windows reach past its slices
        if (iz < c->lo || iz >= c->hi) continue;
        for (int64_t t = 0; t < nxy; ++t)
          qh[N][((size_t)iz * nxy + t) * na + a] = raw[((size_t)a * W[N] + w) * nxy + t];
      }
  }
  if (step_n) *step_n = c->n;
  return staged_status(c);
}

static int upload_links(glasma_ctx* c, void* dev, const double* U) {
  const int64_t V = c->g.V;
  const int nc = c->p.nc, nv = c->nv;
  std::vector<double> raw(2 * (size_t)link_elems(nc, V), 0.0);
  double comp[18];
  for (int d = 0; d < 3; ++d)
    for (int64_t s = 0; s < V; ++s) {
      matrix_to_link(c, U + ((size_t)d * V + s) * nc * nc * 2, comp);
      for (int k = 0; k < nv; ++k) {
        const size_t at = 2 * (size_t)link_index(nc, d, k, V, s);
        raw[at] = comp[2 * k];
        raw[at + 1] = comp[2 * k + 1];
      }
    }
  return reals_to_dev(c, dev, raw.data(), raw.size());
}

// nonzero slice range of a full-lattice charge field [V][na]
static void support(const glasma_ctx* c, const double* Q, int* lo, int* W) {
  *lo = 0;
  *W = 0;
  if (!Q) return;
  int first = -1, last = -1;
  const size_t per = (size_t)c->g.nxy * c->na;
  for (int iz = 0; iz < c->g.nz; ++iz) {
    const double* q = Q + (size_t)iz * per;
    bool nz = false;
    for (size_t k = 0; k < per && !nz; ++k) nz = q[k] != 0.0;
    if (nz) {
      if (first < 0) first = iz;
      last = iz;
    }
  }
  if (first >= 0) {
    *lo = first;
    *W = last - first + 1;
  }
}

int glasma_set_fields(glasma_ctx* c, const double* U, const double* E, const double* QA, const double* QB,
                      const double* U_prev, long long step_n) {
  if (!c || !U || !E || step_n < 0) return set_error(GLASMA_ERR_INVALID_ARG, "bad context, U, E or step_n");
  if (c->slab) return set_error(GLASMA_ERR_INVALID_ARG, "set_fields takes a whole lattice, not a slab");
  if (reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  const int64_t V = c->g.V, nxy = c->g.nxy;
  const int na = c->na, nc = c->p.nc;
  // the absent z link of the last slice must be the identity, E_z zero there
  for (int64_t t = 0; t < nxy; ++t) {
    const int64_t s = (int64_t)(c->g.nz - 1) * nxy + t;
    const double* m = U + ((size_t)2 * V + s) * nc * nc * 2;
    for (int r = 0; r < nc; ++r)
      for (int k = 0; k < nc; ++k)
        if (m[2 * (r * nc + k)] != (r == k ? 1.0 : 0.0) || m[2 * (r * nc + k) + 1] != 0.0)
          return set_error(GLASMA_ERR_INVALID_ARG, "U_z on the last slice must be the identity");
    for (int a = 0; a < na; ++a)
      if (E[((size_t)2 * V + s) * na + a] != 0.0)
        return set_error(GLASMA_ERR_INVALID_ARG, "E_z on the last slice must be zero");
  }
  int st = upload_links(c, c->U[0], U);
  if (st) return st;
  st = upload_links(c, c->U[1], U);
  if (st) return st;
  c->cur = 0;
  {
    std::vector<double> raw(3 * (size_t)na * V);
    for (int d = 0; d < 3; ++d)
      for (int64_t s = 0; s < V; ++s)
        for (int a = 0; a < na; ++a) raw[((size_t)d * na + a) * V + s] = E[((size_t)d * V + s) * na + a];
    st = reals_to_dev(c, c->E, raw.data(), raw.size());
    if (st) return st;
  }
  if (c->Uit) {
    st = upload_links(c, c->Uit, U);
    if (st) return st;
  }
  if (c->Uprev) {
    if (U_prev) {
      st = upload_links(c, c->Uprev, U_prev);
      if (st) return st;
      c->uprev_valid = true;
    } else {
      // the first implicit step rebuilds U(t_{n-1}) = exp(-i dt E) U(t_n)
      // on the device
      c->uprev_valid = false;
    }
  }
  const double* qh[2] = {QA, QB};
  int* z0[2] = {&c->zA0, &c->zB0};
  int* W[2] = {&c->WA, &c->WB};
  void** qd[2] = {&c->QA, &c->QB};
  size_t* cap[2] = {&c->QA_cap, &c->QB_cap};
  for (int N = 0; N < 2; ++N) {
    int lo, w;
    support(c, qh[N], &lo, &w);
    if ((size_t)w > *cap[N]) {
      ctx_free(c, *qd[N]);
      *qd[N] = ctx_alloc(c, c->rs * na * (size_t)w * nxy);
      if (!*qd[N]) return set_error(GLASMA_ERR_OOM, "charge window allocation failed");
      *cap[N] = (size_t)w;
    }
    *z0[N] = lo;
    *W[N] = w;
    if (w > 0) {
      std::vector<double> raw((size_t)na * w * nxy);
      for (int a = 0; a < na; ++a)
        for (int k = 0; k < w; ++k)
          for (int64_t t = 0; t < nxy; ++t)
            raw[((size_t)a * w + k) * nxy + t] = qh[N][((size_t)(lo + k) * nxy + t) * na + a];
      st = reals_to_dev(c, *qd[N], raw.data(), raw.size());
      if (st) return st;
    }
  }
  c->n = step_n;
  return GLASMA_OK;
}

// ---------------------------------------------------------------------------
// checkpoint blob: header, then arrays each followed by its CRC-32
// ---------------------------------------------------------------------------

struct StateHeader {
  char magic[8];
  int32_t version, nc, nz, nx, ny, precision, scheme, rs;
  int64_t n;
  int32_t zA0, WA, zB0, WB;
  double a_t, a_z, dt;
  uint32_t header_crc, pad;
};

static size_t blob_arrays(const glasma_ctx* c, size_t sizes[5]) {
  const size_t ub = link_bytes(c);
  sizes[0] = ub;
  sizes[1] = c->rs * 3 * (size_t)c->na * c->g.V;
  sizes[2] = c->rs * (size_t)c->na * c->WA * c->g.nxy;
  sizes[3] = c->rs * (size_t)c->na * c->WB * c->g.nxy;
  sizes[4] = c->Uprev ? ub : 0;
  size_t tot = 0;
  for (int k = 0; k < 5; ++k) tot += sizes[k] + sizeof(uint32_t);
  return tot;
}

int glasma_state_bytes(const glasma_ctx* c, size_t* bytes) {
  if (!c || !bytes) return set_error(GLASMA_ERR_INVALID_ARG, "bad context or bytes");
  size_t sizes[5];
  *bytes = sizeof(StateHeader) + blob_arrays(c, sizes);
  return GLASMA_OK;
}

int glasma_get_state(glasma_ctx* c, void* host_buf, size_t bytes) {
  if (c && c->slab) return set_error(GLASMA_ERR_INVALID_ARG, "checkpoints hold whole lattices, not slabs");
  if (c && reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  size_t need;
  int st = glasma_state_bytes(c, &need);
  if (st) return st;
  if (!host_buf || bytes < need) return set_error(GLASMA_ERR_INVALID_ARG, "state buffer too small");
  cudaSetDevice(c->device);
  StateHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "GLASMA01", 8);
  h.version = 2;  // 2: SU(3) links in blocks of 32 sites
  h.nc = c->p.nc;
  h.nz = c->g.nz;
  h.nx = c->g.nx;
  h.ny = c->g.ny;
  h.precision = c->p.precision;
  h.scheme = c->p.scheme;
  h.rs = (int32_t)c->rs;
  h.n = c->n;
  h.zA0 = c->zA0;
  h.WA = c->WA;
  h.zB0 = c->zB0;
  h.WB = c->WB;
  h.a_t = c->p.a_t;
  h.a_z = c->p.a_z;
  h.dt = c->p.dt;
  h.header_crc = crc32(&h, offsetof(StateHeader, header_crc));
  unsigned char* out = (unsigned char*)host_buf;
  memcpy(out, &h, sizeof(h));
  size_t off = sizeof(h);
  size_t sizes[5];
  blob_arrays(c, sizes);
  const void* src[5] = {c->U[c->cur], c->E, c->QA, c->QB, c->Uprev};
  for (int k = 0; k < 5; ++k) {
    if (sizes[k]) {
      st = cuda_check(cudaMemcpyAsync(out + off, src[k], sizes[k], cudaMemcpyDeviceToHost, c->stream), "state D2H");
      if (st) return st;
    }
    st = cuda_check(cudaStreamSynchronize(c->stream), "state sync");
    if (st) return st;
    uint32_t crc = crc32(out + off, sizes[k]);
    memcpy(out + off + sizes[k], &crc, sizeof(crc));
    off += sizes[k] + sizeof(crc);
  }
  return staged_status(c);
}

int glasma_set_state(glasma_ctx* c, const void* host_buf, size_t bytes) {
  if (!c || !host_buf || bytes < sizeof(StateHeader)) return set_error(GLASMA_ERR_INVALID_ARG, "bad state buffer");
  if (c->slab) return set_error(GLASMA_ERR_INVALID_ARG, "checkpoints hold whole lattices, not slabs");
  if (reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  StateHeader h;
  memcpy(&h, host_buf, sizeof(h));
  if (memcmp(h.magic, "GLASMA01", 8) != 0 || h.version != 2)
    return set_error(GLASMA_ERR_INVALID_ARG, "not a glasma state blob");
  if (crc32(&h, offsetof(StateHeader, header_crc)) != h.header_crc)
    return set_error(GLASMA_ERR_CHECKSUM, "state header checksum mismatch");
  if (h.nc != c->p.nc || h.nz != c->g.nz || h.nx != c->g.nx || h.ny != c->g.ny || h.precision != c->p.precision ||
      h.scheme != c->p.scheme || h.rs != (int32_t)c->rs || h.a_t != c->p.a_t || h.a_z != c->p.a_z || h.dt != c->p.dt)
    return set_error(GLASMA_ERR_INVALID_ARG, "state blob from another configuration");
  const int oldA = c->WA, oldB = c->WB;
  c->WA = h.WA;
  c->WB = h.WB;
  size_t sizes[5];
  size_t need = sizeof(StateHeader) + blob_arrays(c, sizes);
  if (bytes < need) {
    c->WA = oldA;
    c->WB = oldB;
    return set_error(GLASMA_ERR_INVALID_ARG, "state buffer too small");
  }
  const unsigned char* in = (const unsigned char*)host_buf;
  size_t off = sizeof(h);
  for (int k = 0; k < 5; ++k) {
    uint32_t crc;
    memcpy(&crc, in + off + sizes[k], sizeof(crc));
    if (crc32(in + off, sizes[k]) != crc) {
      c->WA = oldA;
      c->WB = oldB;
      return set_error(GLASMA_ERR_CHECKSUM, "state array checksum mismatch");
    }
    off += sizes[k] + sizeof(crc);
  }
  if ((size_t)h.WA > c->QA_cap) {
    ctx_free(c, c->QA);
    c->QA = ctx_alloc(c, sizes[2]);
    c->QA_cap = (size_t)h.WA;
  }
  if ((size_t)h.WB > c->QB_cap) {
    ctx_free(c, c->QB);
    c->QB = ctx_alloc(c, sizes[3]);
    c->QB_cap = (size_t)h.WB;
  }
  if (!c->QA || !c->QB) return set_error(GLASMA_ERR_OOM, "charge window allocation failed");
  c->cur = 0;
  void* dst[5] = {c->U[0], c->E, c->QA, c->QB, c->Uprev};
  off = sizeof(h);
  int st;
  for (int k = 0; k < 5; ++k) {
    if (sizes[k]) {
      st = cuda_check(cudaMemcpyAsync(dst[k], in + off, sizes[k], cudaMemcpyHostToDevice, c->stream), "state H2D");
      if (st) return st;
    }
    off += sizes[k] + sizeof(uint32_t);
  }
  // the other link buffers need the identity z links of the last slice
  st = cuda_check(cudaMemcpyAsync(c->U[1], c->U[0], sizes[0], cudaMemcpyDeviceToDevice, c->stream), "state copy");
  if (st) return st;
  if (c->Uit) {
    st = cuda_check(cudaMemcpyAsync(c->Uit, c->U[0], sizes[0], cudaMemcpyDeviceToDevice, c->stream), "state copy");
    if (st) return st;
    c->uprev_valid = true;
  }
  c->zA0 = h.zA0;
  c->zB0 = h.zB0;
  c->n = h.n;
  return cuda_check(cudaStreamSynchronize(c->stream), "state sync");
}

int glasma_set_step_kernel(glasma_ctx* c, int kernel, int zlen) {
  if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "context is NULL");
  if (kernel != GLASMA_KERNEL_AUTO && kernel != GLASMA_KERNEL_STAPLE && kernel != GLASMA_KERNEL_PLAQUETTE &&
      kernel != GLASMA_KERNEL_PLAQUETTE_256 && kernel != GLASMA_KERNEL_STAPLE_PAIRS &&
      kernel != GLASMA_KERNEL_STAPLE_STAGED)
    return set_error(GLASMA_ERR_INVALID_ARG, "unknown step kernel");
  if (kernel == GLASMA_KERNEL_STAPLE_PAIRS && (c->rs != 4 || c->slab))
    return set_error(GLASMA_ERR_INVALID_ARG, "the paired staple kernel needs FP32 state of a whole lattice");
  if (kernel == GLASMA_KERNEL_STAPLE_STAGED && !staged_fits(c))
    return set_error(GLASMA_ERR_INVALID_ARG,
                     "the staged staple kernel needs FP32 SU(3) state of a whole lattice with nx = 32 or 64");
  if (zlen < 0 || zlen > c->g.nz) return set_error(GLASMA_ERR_INVALID_ARG, "zlen must be in [0, nz]");
  const int old = c->step_kernel;
  c->step_kernel = kernel;
  if ((kernel == GLASMA_KERNEL_PLAQUETTE || kernel == GLASMA_KERNEL_PLAQUETTE_256) && !plaq_fits(c)) {
    c->step_kernel = old;
    return set_error(GLASMA_ERR_INVALID_ARG, "transverse rows too long for the plaquette kernel");
  }
  c->step_zlen = zlen;
  return GLASMA_OK;
}

int glasma_set_staging_wait(glasma_ctx* c, long long wait_cycles, int stall) {
  if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "context is NULL");
  if (wait_cycles < 1 || wait_cycles > (1ll << 40) || (stall != 0 && stall != 1))
    return set_error(GLASMA_ERR_INVALID_ARG, "wait_cycles must be in [1, 2^40] and stall 0 or 1");
  c->staged_wait = wait_cycles;
  c->staged_stall = stall;
  return GLASMA_OK;
}

int glasma_slab_info(const glasma_ctx* c, int* z0, int* z1, int* nz_local, int* lo, int* hi) {
  if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "context is NULL");
  if (z0) *z0 = c->zoff + c->lo;
  if (z1) *z1 = c->zoff + c->hi;
  if (nz_local) *nz_local = c->g.nz;
  if (lo) *lo = c->lo;
  if (hi) *hi = c->hi;
  return GLASMA_OK;
}

int glasma_slab_set_windows(glasma_ctx* c, int zA0, int WA, int zB0, int WB) {
  if (!c || !c->slab) return set_error(GLASMA_ERR_INVALID_ARG, "not a slab context");
  if (WA < 0 || WB < 0 || zA0 < 0 || zB0 < 0 || zA0 + WA > c->nz_glob || zB0 + WB > c->nz_glob)
    return set_error(GLASMA_ERR_INVALID_ARG, "window outside the lattice");
  cudaSetDevice(c->device);
  const int na = c->na;
  const int64_t nxy = c->g.nxy;
  // the new windows (global slices) must hold the slab's own charges
  const int old0[2] = {c->zA0 + c->zoff, c->zB0 + c->zoff}, oldW[2] = {c->WA, c->WB};
  const int new0[2] = {zA0, zB0}, newW[2] = {WA, WB};
  for (int N = 0; N < 2; ++N)
    if (oldW[N] > 0 && (old0[N] < new0[N] || old0[N] + oldW[N] > new0[N] + newW[N]))
      return set_error(GLASMA_ERR_INVALID_ARG, "the windows must contain the slab's own charge windows");
  void** q[2] = {&c->QA, &c->QB};
  size_t* cap[2] = {&c->QA_cap, &c->QB_cap};
  for (int N = 0; N < 2; ++N) {
    const size_t w = (size_t)(newW[N] > 0 ? newW[N] : 1);
    void* nq = ctx_alloc(c, c->rs * na * w * nxy);
    if (!nq) return set_error(GLASMA_ERR_OOM, "charge window allocation failed");
    int st = cuda_check(cudaMemsetAsync(nq, 0, c->rs * na * w * nxy, c->stream), "window clear");
    for (int a = 0; a < na && !st && oldW[N] > 0; ++a) {
      const size_t row = c->rs * (size_t)nxy;
      char* dst = (char*)nq + ((size_t)a * newW[N] + (old0[N] - new0[N])) * row;
      const char* src = (const char*)*q[N] + (size_t)a * oldW[N] * row;
      st = cuda_check(cudaMemcpyAsync(dst, src, row * oldW[N], cudaMemcpyDeviceToDevice, c->stream), "window copy");
    }
    if (st) {
      ctx_free(c, nq);
      return st;
    }
    ctx_free(c, *q[N]);
    *q[N] = nq;
    *cap[N] = w;
  }
  c->zA0 = zA0 - c->zoff;
  c->WA = WA;
  c->zB0 = zB0 - c->zoff;
  c->WB = WB;
  c->slab_windows = true;
  return cuda_check(cudaStreamSynchronize(c->stream), "window sync");
}

int glasma_slab_message_bytes(const glasma_ctx* c, int dir, size_t* bytes) {
  if (!c || !bytes || (dir != 1 && dir != -1)) return set_error(GLASMA_ERR_INVALID_ARG, "bad context, dir or bytes");
  *bytes = c->rs * slab_msg_elems(c, dir);
  return GLASMA_OK;
}

int glasma_slab_pack(glasma_ctx* c, int dir, void* dev_buf) {
  if (!c || !dev_buf || (dir != 1 && dir != -1)) return set_error(GLASMA_ERR_INVALID_ARG, "bad context, dir or buffer");
  if ((dir == 1 && c->hi == c->g.nz) || (dir == -1 && c->lo == 0))
    return set_error(GLASMA_ERR_INVALID_ARG, "no neighbouring slab in that direction");
  if (((uintptr_t)dev_buf & 15) != 0) return set_error(GLASMA_ERR_INVALID_ARG, "message buffer must be 16-byte aligned");
  if (reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  return slab_pack(c, dir, dev_buf);
}

int glasma_slab_unpack(glasma_ctx* c, int dir, const void* dev_buf) {
  if (!c || !dev_buf || (dir != 1 && dir != -1)) return set_error(GLASMA_ERR_INVALID_ARG, "bad context, dir or buffer");
  if ((dir == 1 && c->hi == c->g.nz) || (dir == -1 && c->lo == 0))
    return set_error(GLASMA_ERR_INVALID_ARG, "no neighbouring slab in that direction");
  if (((uintptr_t)dev_buf & 15) != 0) return set_error(GLASMA_ERR_INVALID_ARG, "message buffer must be 16-byte aligned");
  if (reject_open_step(c)) return GLASMA_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  return slab_unpack(c, dir, dev_buf);
}

int glasma_get_info(const glasma_ctx* c, glasma_info* info) {
  if (!c || !info) return set_error(GLASMA_ERR_INVALID_ARG, "bad context or info");
  info->sites = (long long)c->g.V;
  info->step_n = c->n;
  info->nc = c->p.nc;
  info->precision = c->p.precision;
  info->scheme = c->p.scheme;
  info->window_a[0] = c->zA0 + c->zoff;  // global slices
  info->window_a[1] = c->WA;
  info->window_b[0] = c->zB0 + c->zoff;
  info->window_b[1] = c->WB;
  info->state_device_bytes = 2 * link_bytes(c) + c->rs * 3 * (size_t)c->na * c->g.V +
                             c->rs * (size_t)c->na * (c->QA_cap + c->QB_cap) * c->g.nxy;
  info->kernel_launches = c->last_launches;
  info->implicit_iters = c->last_iters;
  return GLASMA_OK;
}

}  // extern "C"
