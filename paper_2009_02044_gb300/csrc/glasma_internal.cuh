// Context object behind the C ABI and the host-side launchers of each kernel
// family.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/glasma.h"
#include "lattice.cuh"

struct glasma_ctx {
  glasma_params p;
  int device = 0;
  cudaStream_t stream = nullptr;
  glasma_allocator alloc{};
  bool has_alloc = false;
  int na = 0, nv = 0;
  glasma::Geom g{};
  size_t rs = 8;              // bytes per real of the state
  void* U[2] = {nullptr, nullptr};
  int cur = 0;                // U[cur] holds U(t_n)
  void* Uprev = nullptr;      // U(t_{n-1}), implicit scheme only
  void* Uit = nullptr;        // implicit scheme: second iterate buffer of U(t_{n+1})
  bool uprev_valid = false;   // Uprev holds U(t_{n-1})
  void* E = nullptr;          // E(t_{n-1/2})
  void* Ework = nullptr;      // implicit scheme: E(t_{n-1/2}) + current, fixed during iteration
  double* conv = nullptr;     // implicit scheme: max |dE| of each iteration
  void* QA = nullptr;         // charge windows (co-moving slots)
  void* QB = nullptr;
  int zA0 = 0, WA = 0, zB0 = 0, WB = 0;  // first slice and slices of each window
  size_t QA_cap = 0, QB_cap = 0;        // allocated slots
  long long n = 0;
  long long hop_p = 1, hop_q = 2;       // v dt / a_z = p / q
  double* red = nullptr;      // reduction partials
  size_t red_cap = 0;         // doubles
  double* tab = nullptr;      // [nz][4] T^{mu nu} table
  double* tpart = nullptr;    // [nz][kTmunuSplit][5] T^{mu nu} block partials
  int* dflag = nullptr;       // device status word(s)
  int last_launches = 0;
  int last_iters = 0;
  int step_kernel = 0;        // GLASMA_KERNEL_* of the leapfrog step
  int step_zlen = 0;          // z slices per block of the plaquette kernel (0 = automatic)
  bool plaq_ready = false;    // the plaquette kernel's attributes are set on this device
  // staged step kernel (k_step_staged.cu): spin budget of one wait on its
  // copies (SM cycles), the timeout test's stall, and whether it has run
  // since its status word (dflag[1]) was last read
  long long staged_wait = 1ll << 31;
  int staged_stall = 0;
  bool staged_launched = false;
  // z slab of a lattice split along the beam axis (glasma_slab_init): the
  // context's lattice is the slab with its halo slices; local slice 0 is
  // global slice zoff; the owned slices are [lo, hi), the others halos.  An
  // ordinary context has zoff = 0, lo = 0, hi = nz, nz_glob = nz.
  bool slab = false;
  bool slab_windows = false;  // the windows hold the whole lattice's extent
  int zoff = 0, lo = 0, hi = 0, nz_glob = 0;
  // improved step driven sweep by sweep from the host (glasma_implicit_*)
  bool impl_active = false;   // between glasma_implicit_begin and _end
  bool impl_hop = false;      // that step is a hop step
  int impl_k = 0;             // sweeps done in it
  struct Alloc {
    void* ptr;
    size_t bytes;
  };
  std::vector<Alloc> allocs;
};

namespace glasma {

// blocks per z slice of the T^{mu nu} kernel, at most
constexpr int kTmunuSplit = 8;

// status helpers (defined in glasma_api.cu)
int set_error(int status, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);
void* ctx_alloc(glasma_ctx* c, size_t bytes);
void ctx_free(glasma_ctx* c, void* p);

// bytes of one link array of the context (all three directions)
inline size_t link_bytes(const glasma_ctx* c) { return 2 * (size_t)c->rs * (size_t)link_elems(c->p.nc, c->g.V); }

// number of hops after m steps: floor(m p/q + 1/2) in integers
GL_HD long long hop_count(long long m, long long p, long long q) {
  return (2 * m * p + q) / (2 * q);
}
GL_HD bool hop_at(long long n, long long p, long long q) {
  return hop_count(n + 1, p, q) > hop_count(n, p, q);
}

// kernel launchers
int launch_step_leapfrog(glasma_ctx* c, bool hop);
// plaquette-centric leapfrog step (k_step_plaq.cu): zlen z slices per block
int launch_step_plaq(glasma_ctx* c, bool hop, int zlen);
bool plaq_fits(const glasma_ctx* c);
// the step kernel glasma_step launches for this context: plaquette, staple
// on site pairs (FP32), staged staple (FP32 SU(3)) or staple
bool use_plaq_kernel(const glasma_ctx* c);
bool use_pair_kernel(const glasma_ctx* c);
bool use_staged_kernel(const glasma_ctx* c);
// staple kernel with the links staged in shared memory by bulk copies
// (FP32 SU(3), rows of 32 or 64 sites, whole lattices)
bool staged_fits(const glasma_ctx* c);
int launch_step_staged(glasma_ctx* c, bool hop);
// TIMEOUT if a staged launch recorded a wait that ran out (synchronises)
int staged_status(glasma_ctx* c);
int launch_step_chosen(glasma_ctx* c, bool hop);
// staple kernel on pairs of sites (t, iz), (t, iz + ceil(nz/2)), FP32 only
int launch_step_pair(glasma_ctx* c, bool hop);
int plaq_default_zlen(const glasma_ctx* c);
// set the plaquette kernel's function attributes for this context (before
// any capture of its launches)
int plaq_prepare(glasma_ctx* c);
int launch_step_implicit(glasma_ctx* c, bool hop, int* iters);
// the same step in host-driven parts (k_implicit.cu): the hop, U(t_{n-1}) if
// needed and the first iterate; one sweep (index c->impl_k) with its
// maxima read back; the commit of the last iterate after `done` sweeps
int implicit_begin(glasma_ctx* c, bool hop);
int implicit_sweep(glasma_ctx* c, double* dmax, double* emax);
void implicit_commit(glasma_ctx* c, int done);
int launch_gauss(glasma_ctx* c, double* out3);  // over the owned slices [lo, hi)
// slab halo messages (k_slab.cu)
size_t slab_msg_elems(const glasma_ctx* c, int dir);
int slab_pack(glasma_ctx* c, int dir, void* buf);
int slab_unpack(glasma_ctx* c, int dir, const void* buf);
int slab_halo_hop(glasma_ctx* c);
// host_tab != NULL: read the table back and synchronise; dev_tab != NULL:
// write the table there instead of the context's own buffer
int launch_tmunu(glasma_ctx* c, bool hop, double* host_tab, double* dev_tab = nullptr);
int run_init(glasma_ctx* c, const double* rho_host);
int device_philox_rho(const glasma_params& p, int na, double* rho, cudaStream_t s);
int device_poisson(const glasma_params& p, const double* in, double* out, int F, double2* w0, double2* w1,
                   cudaStream_t s);
int device_profile(const glasma_params& p, double* lam, cudaStream_t s);

// checkpoint CRC-32 (IEEE 802.3 polynomial, reflected)
uint32_t crc32(const void* data, size_t n, uint32_t crc = 0);

}  // namespace glasma
