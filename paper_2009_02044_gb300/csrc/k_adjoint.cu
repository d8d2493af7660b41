// Hand-written adjoint of the SU(2) FP64 leapfrog CPIC evolution: the
// gradient of the mid-rapidity energy O = a_z sum_{|z - z_c| < w} eps(z) at
// the final step with respect to the initial MV charges rho_N^a(x_T)
// (Sec. 2 MV model, Sec. 3 Eqs. lattice_1, lattice_2, continuity and the
// NGP transport, Sec. 4 energy density).
//
// Reverse pass, per step n (from the adjoints of U_{n+1}, E_{n+1/2} and the
// charges after the step):
//   k_adj_link    U_{n+1} = exp(i dt E_{n+1/2}) U_n    -> Ubar_n, Ebar_{n+1/2}
//                 hop: Q' = Ad(U_z^-+) Q, dt J_z        -> Qbar_n, Ubar_z
//   k_adj_plaq    d/dU_n [dt sum Ebar . F(U_n)], one plaquette at a time
//   k_adj_gather  each link sums its four plaquettes' parts (fixed order)
// The forward states are recomputed per segment from checkpoints taken
// every K steps.  The initial-state adjoint follows the Gauss divergence
// (charges), the group log (E), the link products of the Wilson lines and
// exp(i Lambda phi), then the Poisson solve, which is symmetric.
// No atomics: every adjoint entry has one writer per kernel.
#include <math.h>

#include <vector>

#include "adjoint.cuh"

namespace glasma {
using namespace adj;

namespace {

unsigned grid_of(int64_t n, int bs = 256) {
  int64_t nb = (n + bs - 1) / bs;
  if (nb > 152 * 32) nb = 152 * 32;
  if (nb < 1) nb = 1;
  return (unsigned)nb;
}

#define GRID_STRIDE(var, total) \
  for (int64_t var = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; var < (total); \
       var += (int64_t)gridDim.x * blockDim.x)

__global__ void k_adj_plaq(const double2* U, const double* Eb, double fs, const double* wsl, double* G, Geom g,
                           double wt, double wz, double ia2t, double ia2z) {
  GRID_STRIDE(s, g.V) plaq_rev_at(U, Eb, fs, wsl, G, g, wt, wz, ia2t, ia2z, s);
}

__global__ void k_adj_gather(const double* G, double* Ub, Geom g) { GRID_STRIDE(s, g.V) gather_at(G, Ub, g, s); }

__global__ void k_adj_link(LinkRevArgs a) { GRID_STRIDE(i, 3 * a.g.V) link_rev_at(a, i); }

__global__ void k_adj_hop_current(const double2* U, const double* Ebp, const double* QA, const double* QB,
                                  double* QAb, double* QBb, double* Ub, int zA0, int WA, int zB0, int WB, Geom g,
                                  double az2) {
  GRID_STRIDE(s, (int64_t)(g.nz - 1) * g.nxy)
  hop_current_rev_at(U, Ebp, QA, QB, QAb, QBb, Ub, zA0, WA, zB0, WB, g, az2, s);
}

__global__ void k_adj_obs(const double* E, const double* Ep, const double* wsl, double* Eb, double* Ebp, Geom g,
                          double ia2t, double ia2z) {
  GRID_STRIDE(i, 9 * g.V) obs_rev_at(E, Ep, wsl, Eb, Ebp, g, ia2t, ia2z, i);
}

__global__ void k_adj_div(const double2* U, const double* E, const double* QAb, const double* QBb, int zA0, int WA,
                          int zB0, int WB, double* Eb, double* Ub, Geom g, double ia2t) {
  GRID_STRIDE(s, g.V) div_rev_at(U, E, QAb, QBb, zA0, WA, zB0, WB, Eb, Ub, g, ia2t, s);
}

__global__ void k_adj_log(const double* phi, const double* lam, const double* Eb, double* Ub, double* Umb, Geom g,
                          double dt) {
  GRID_STRIDE(i, 2 * g.V) log_rev_at(phi, lam, Eb, Ub, Umb, g, dt, i);
}

__global__ void k_adj_links(const double* phi, const double* lam, const double* Ub, const double* Umb,
                            double* phib_z, Geom g) {
  GRID_STRIDE(s, g.V) links_rev_at(phi, lam, Ub, Umb, phib_z, g, s);
}

__global__ void k_adj_zsum(const double* phib_z, double* phib, Geom g) {
  GRID_STRIDE(i, 6 * g.nxy) zsum_at(phib_z, phib, g, i);
}

}  // namespace

namespace {

// device allocations of one adjoint call, released (stream-ordered) at exit
struct Scratch {
  glasma_ctx* c;
  std::vector<void*> ptrs;
  bool ok = true;
  explicit Scratch(glasma_ctx* ctx) : c(ctx) {}
  template <typename T>
  T* get(size_t count) {
    void* p = ctx_alloc(c, count * sizeof(T));
    if (!p) ok = false;
    else ptrs.push_back(p);
    return (T*)p;
  }
  ~Scratch() {
    for (void* p : ptrs) ctx_free(c, p);
  }
};

struct StateRef {
  double2* U;
  double* E;
  double* QA;
  double* QB;
  int zA0, zB0;
  long long n;
};

struct Sizes {
  size_t ub, eb, qa, qb;
};

int save_state(glasma_ctx* c, const Sizes& z, StateRef& dst) {
  int st = cuda_check(cudaMemcpyAsync(dst.U, c->U[c->cur], z.ub, cudaMemcpyDeviceToDevice, c->stream), "save U");
  if (!st) st = cuda_check(cudaMemcpyAsync(dst.E, c->E, z.eb, cudaMemcpyDeviceToDevice, c->stream), "save E");
  if (!st && z.qa) st = cuda_check(cudaMemcpyAsync(dst.QA, c->QA, z.qa, cudaMemcpyDeviceToDevice, c->stream), "save QA");
  if (!st && z.qb) st = cuda_check(cudaMemcpyAsync(dst.QB, c->QB, z.qb, cudaMemcpyDeviceToDevice, c->stream), "save QB");
  dst.zA0 = c->zA0;
  dst.zB0 = c->zB0;
  dst.n = c->n;
  return st;
}

int load_state(glasma_ctx* c, const Sizes& z, const StateRef& src) {
  int st = cuda_check(cudaMemcpyAsync(c->U[c->cur], src.U, z.ub, cudaMemcpyDeviceToDevice, c->stream), "load U");
  if (!st) st = cuda_check(cudaMemcpyAsync(c->E, src.E, z.eb, cudaMemcpyDeviceToDevice, c->stream), "load E");
  if (!st && z.qa) st = cuda_check(cudaMemcpyAsync(c->QA, src.QA, z.qa, cudaMemcpyDeviceToDevice, c->stream), "load QA");
  if (!st && z.qb) st = cuda_check(cudaMemcpyAsync(c->QB, src.QB, z.qb, cudaMemcpyDeviceToDevice, c->stream), "load QB");
  c->zA0 = src.zA0;
  c->zB0 = src.zB0;
  c->n = src.n;
  return st;
}

// A state in the context's own precision (raw buffers; the pointer types
// are those of FP64 and are reinterpreted for FP32).
StateRef alloc_state(Scratch& sc, const glasma_ctx* c) {
  StateRef r{};
  const size_t rs = c->rs;
  r.U = (double2*)sc.get<char>(2 * rs * 3 * 2 * (size_t)c->g.V);
  r.E = (double*)sc.get<char>(rs * 9 * (size_t)c->g.V);
  r.QA = (double*)sc.get<char>(rs * 3 * c->QA_cap * (size_t)c->g.nxy);
  r.QB = (double*)sc.get<char>(rs * 3 * c->QB_cap * (size_t)c->g.nxy);
  return r;
}

// FP32 states hold U - 1 (alpha - 1 for SU(2)) and FP32 fields: the reverse
// pass reads them as FP64 full links and fields.
__global__ void k_links_to64(const float2* in, double2* out, int64_t V) {
  GRID_STRIDE(i, 6 * V) {
    const float2 v = in[i];
    const bool alpha = (i & 1) == 0;  // link_index(2, d, k, V, s) = (d V + s) 2 + k
    out[i] = make_double2((double)v.x + (alpha ? 1.0 : 0.0), (double)v.y);
  }
}

__global__ void k_reals_to64(const float* in, double* out, int64_t n) {
  GRID_STRIDE(i, n) out[i] = (double)in[i];
}

// FP64 view of a state: the raw buffers for an FP64 context, converted
// copies in `cv` for an FP32 one.
struct View {
  const double2* U;
  const double* E;
  const double* QA;
  const double* QB;
};

View view64(const StateRef& st, bool f32, const StateRef& cv, const glasma_ctx* c, bool links, bool fields,
            bool charges) {
  if (!f32) return View{st.U, st.E, st.QA, st.QB};
  const Geom& g = c->g;
  cudaStream_t s = c->stream;
  if (links) k_links_to64<<<grid_of(6 * g.V), 256, 0, s>>>((const float2*)st.U, cv.U, g.V);
  if (fields) k_reals_to64<<<grid_of(9 * g.V), 256, 0, s>>>((const float*)st.E, cv.E, 9 * g.V);
  if (charges) {
    const int64_t na = 3 * (int64_t)c->WA * g.nxy, nb = 3 * (int64_t)c->WB * g.nxy;
    if (na) k_reals_to64<<<grid_of(na), 256, 0, s>>>((const float*)st.QA, cv.QA, na);
    if (nb) k_reals_to64<<<grid_of(nb), 256, 0, s>>>((const float*)st.QB, cv.QB, nb);
  }
  return View{cv.U, cv.E, cv.QA, cv.QB};
}

StateRef alloc_state64(Scratch& sc, const glasma_ctx* c) {
  StateRef r{};
  r.U = sc.get<double2>(3 * 2 * (size_t)c->g.V);
  r.E = sc.get<double>(9 * (size_t)c->g.V);
  r.QA = sc.get<double>(3 * c->QA_cap * (size_t)c->g.nxy);
  r.QB = sc.get<double>(3 * c->QB_cap * (size_t)c->g.nxy);
  return r;
}

int adjoint_run(glasma_ctx* c, const double* rho_host, int n_steps, double half_width, int K, double* value,
                double* grad_host) {
  const glasma_params& p = c->p;
  const Geom g = c->g;
  cudaStream_t s = c->stream;
  const size_t rs = c->rs;
  const bool f32 = rs == 4;
  const Sizes z{link_bytes(c), rs * 9 * (size_t)g.V, rs * 3 * (size_t)c->WA * g.nxy,
                rs * 3 * (size_t)c->WB * g.nxy};
  Scratch sc(c);
  const int ncp = n_steps > 0 ? (n_steps + K - 1) / K : 0;
  std::vector<StateRef> ck(ncp);
  for (auto& r : ck) r = alloc_state(sc, c);
  const int seg_len = n_steps > 0 ? (K < n_steps ? K : n_steps) : 0;
  std::vector<StateRef> seg(seg_len + 1);
  for (auto& r : seg) r = alloc_state(sc, c);
  StateRef fin = alloc_state(sc, c);  // the final state before the observable's E update
  // FP64 copies for an FP32 context: state n of a reverse step and E of n+1
  StateRef cva{}, cvb{};
  if (f32) {
    cva = alloc_state64(sc, c);
    cvb.E = sc.get<double>(9 * (size_t)g.V);
  }
  double* Ub = sc.get<double>(12 * (size_t)g.V);
  double* Eb = sc.get<double>(9 * (size_t)g.V);
  double* Ebp = sc.get<double>(9 * (size_t)g.V);
  double* QAb = sc.get<double>(3 * c->QA_cap * (size_t)g.nxy);
  double* QBb = sc.get<double>(3 * c->QB_cap * (size_t)g.nxy);
  double* G = sc.get<double>(48 * (size_t)g.V);
  double* wsl = sc.get<double>(g.nz);
  if (!sc.ok) return set_error(GLASMA_ERR_OOM, "adjoint scratch allocation failed");

  // forward with checkpoints
  int st = GLASMA_OK;
  for (int n = 0; n < n_steps && !st; ++n) {
    if (n % K == 0) st = save_state(c, z, ck[n / K]);
    if (!st) st = glasma_step(c, 1);
  }
  if (st) return st;

  // observable: O = sum_iz w(iz) eps(iz), w = a_z inside |z - z_c| < half_width
  std::vector<double> tab(4 * (size_t)g.nz), w(g.nz);
  st = glasma_tmunu(c, tab.data(), nullptr);
  if (st) return st;
  const double zc = p.nz * p.a_z / 2.0;
  double O = 0.0;
  for (int iz = 0; iz < g.nz; ++iz) {
    w[iz] = fabs(iz * p.a_z - zc) < half_width ? p.a_z : 0.0;
    O += w[iz] * tab[4 * iz];
    w[iz] /= (double)g.nxy;
  }
  if (value) *value = O;
  if (!grad_host) return GLASMA_OK;
  st = cuda_check(cudaMemcpyAsync(wsl, w.data(), sizeof(double) * g.nz, cudaMemcpyHostToDevice, s), "weights");
  if (!st) st = save_state(c, z, fin);
  if (st) return st;
  const double wt = 2.0 / (p.a_t * p.a_t), wz = 2.0 / (p.a_z * p.a_z);
  const double ia2t = 1.0 / (p.a_t * p.a_t), ia2z = 1.0 / (p.a_z * p.a_z), az2 = p.a_z * p.a_z;
  const bool hopN = hop_at(c->n, c->hop_p, c->hop_q);
  st = launch_step_leapfrog(c, hopN);  // E' = E(N + 1/2) in c->E; charges moved in place
  if (st) return st;
  cudaMemsetAsync(Ub, 0, sizeof(double) * 12 * g.V, s);
  // the charge adjoints are FP64 whatever the state's precision
  cudaMemsetAsync(QAb, 0, sizeof(double) * 3 * c->QA_cap * (size_t)g.nxy, s);
  cudaMemsetAsync(QBb, 0, sizeof(double) * 3 * c->QB_cap * (size_t)g.nxy, s);
  const View vf = view64(fin, f32, cva, c, true, true, true);
  const double* Ep = (const double*)c->E;  // E' of the observable's own update
  if (f32) {
    k_reals_to64<<<grid_of(9 * g.V), 256, 0, s>>>((const float*)c->E, cvb.E, 9 * g.V);
    Ep = cvb.E;
  }
  k_adj_obs<<<grid_of(9 * g.V), 256, 0, s>>>(vf.E, Ep, wsl, Eb, Ebp, g, ia2t, ia2z);
  k_adj_plaq<<<grid_of(g.V, 128), 128, 0, s>>>(vf.U, Ebp, p.dt, wsl, G, g, wt, wz, ia2t, ia2z);
  k_adj_gather<<<grid_of(g.V), 256, 0, s>>>(G, Ub, g);
  if (hopN)
    k_adj_hop_current<<<grid_of((int64_t)(g.nz - 1) * g.nxy), 256, 0, s>>>(
        vf.U, Ebp, vf.QA, vf.QB, QAb, QBb, Ub, fin.zA0, c->WA, fin.zB0, c->WB, g, az2);
  st = cuda_check(cudaGetLastError(), "adjoint observable");
  if (st) return st;

  // reverse, one checkpointed segment at a time
  const StateRef* s0 = &fin;
  for (int sg = ncp - 1; sg >= 0 && !st; --sg) {
    const int n0 = sg * K, n1 = n0 + K < n_steps ? n0 + K : n_steps;
    st = load_state(c, z, ck[sg]);
    if (!st) st = save_state(c, z, seg[0]);
    for (int k = 1; k <= n1 - n0 && !st; ++k) {
      st = glasma_step(c, 1);
      if (!st) st = save_state(c, z, seg[k]);
    }
    for (int n = n1 - 1; n >= n0 && !st; --n) {
      const int k = n - n0;
      const View vn = view64(seg[k], f32, cva, c, true, false, true);
      const double* En = seg[k + 1].E;
      if (f32) {
        k_reals_to64<<<grid_of(9 * g.V), 256, 0, s>>>((const float*)seg[k + 1].E, cvb.E, 9 * g.V);
        En = cvb.E;
      }
      LinkRevArgs a;
      a.U = vn.U;
      a.En = En;
      a.Ub = Ub;
      a.Eb = Eb;
      a.QA = vn.QA;
      a.QB = vn.QB;
      a.QAb = QAb;
      a.QBb = QBb;
      a.hop = hop_at(n, c->hop_p, c->hop_q) ? 1 : 0;
      a.zA0 = seg[k].zA0;
      a.WA = c->WA;
      a.zB0 = seg[k].zB0;
      a.WB = c->WB;
      a.g = g;
      a.dt = p.dt;
      a.az2 = az2;
      k_adj_link<<<grid_of(3 * g.V), 256, 0, s>>>(a);
      k_adj_plaq<<<grid_of(g.V, 128), 128, 0, s>>>(vn.U, Eb, p.dt, nullptr, G, g, wt, wz, ia2t, ia2z);
      k_adj_gather<<<grid_of(g.V), 256, 0, s>>>(G, Ub, g);
      st = cuda_check(cudaGetLastError(), "adjoint step");
    }
    s0 = &seg[0];
  }
  if (st) return st;

  // initial state: charges -> E, U0; log -> U0, U(t0 - dt); links -> V^+; exp -> phi; Poisson -> rho
  const int64_t F = 6, nxy = g.nxy;
  double* rho = sc.get<double>(F * nxy);
  double* phi = sc.get<double>(F * nxy);
  double* lam = sc.get<double>(4 * (size_t)g.nz);
  double2* w0 = sc.get<double2>(F * nxy);
  double2* w1 = sc.get<double2>(F * nxy);
  double* Umb = sc.get<double>(8 * (size_t)g.V);
  double* phib_z = sc.get<double>(F * (size_t)g.V);
  double* phib = sc.get<double>(F * nxy);
  if (!sc.ok) return set_error(GLASMA_ERR_OOM, "adjoint scratch allocation failed");
  if (rho_host)
    st = cuda_check(cudaMemcpyAsync(rho, rho_host, sizeof(double) * F * nxy, cudaMemcpyHostToDevice, s), "rho");
  else
    st = device_philox_rho(p, 3, rho, s);
  if (!st) st = device_poisson(p, rho, phi, (int)F, w0, w1, s);
  if (!st) st = device_profile(p, lam, s);
  if (st) return st;
  const View v0 = view64(*s0, f32, cva, c, true, true, false);
  k_adj_div<<<grid_of(g.V), 256, 0, s>>>(v0.U, v0.E, QAb, QBb, s0->zA0, c->WA, s0->zB0, c->WB, Eb, Ub, g, ia2t);
  k_adj_log<<<grid_of(2 * g.V), 256, 0, s>>>(phi, lam, Eb, Ub, Umb, g, p.dt);
  k_adj_links<<<grid_of(g.V, 128), 128, 0, s>>>(phi, lam, Ub, Umb, phib_z, g);
  k_adj_zsum<<<grid_of(F * nxy), 256, 0, s>>>(phib_z, phib, g);
  st = cuda_check(cudaGetLastError(), "adjoint init");
  if (!st) st = device_poisson(p, phib, phib, (int)F, w0, w1, s);
  if (!st)
    st = cuda_check(cudaMemcpyAsync(grad_host, phib, sizeof(double) * F * nxy, cudaMemcpyDeviceToHost, s), "grad");
  if (!st) st = cuda_check(cudaStreamSynchronize(s), "adjoint sync");
  return st;
}

}  // namespace
}  // namespace glasma

using namespace glasma;

extern "C" GLASMA_API int glasma_adjoint_energy(const glasma_params* p, const double* rho_host, int n_steps,
                                                double half_width, int checkpoint_every, void* stream,
                                                const glasma_allocator* alloc, double* value, double* grad_host) {
  if (!p) return set_error(GLASMA_ERR_INVALID_ARG, "params is NULL");
  if (p->nc != 2 || p->scheme != GLASMA_LEAPFROG || p->n_sheets > 1)
    return set_error(GLASMA_ERR_INVALID_ARG, "the adjoint covers SU(2), leapfrog, one colour sheet");
  if (n_steps < 0 || !(half_width > 0.0) || checkpoint_every < 1)
    return set_error(GLASMA_ERR_INVALID_ARG, "need n_steps >= 0, half_width > 0, checkpoint_every >= 1");
  glasma_ctx* c = nullptr;
  int st = glasma_init_mv(p, rho_host, stream, alloc, &c);
  if (st) return st;
  st = adjoint_run(c, rho_host, n_steps, half_width, checkpoint_every, value, grad_host);
  glasma_free(c);
  return st;
}
