// Batched ensemble: independent MV events (the ensemble averages of Sec. 2,
// Eq. ev, and Sec. 4) of uneven lattice size advanced together, with a
// call's steps captured into one CUDA graph.
//
// Graph mode: one launch per time step and geometry class (events of equal
// nx, ny, nz), blockIdx.z the event within the class; it runs the same
// per-link update as the single-event kernel (step_link), so every event's
// result is bitwise the one it would get alone.  Persistent mode: the
// events' blocks are concatenated (event e owns work items [block0_e,
// block0_e + ntb_e * nz_e)); a block finds its event by a binary search
// over the prefix offsets held in the kernel parameters.
//
// Block shape: BX transverse sites x 3 directions; BX in {32, 64, 128} is
// chosen by glasma_batch_tune, which times each shape on the batch itself
// and restores the state afterwards.
#include <string.h>

#include <vector>

#include "step_link.cuh"

namespace glasma {

constexpr int kMaxBatch = 64;  // events per batch: their kernel parameters stay under the 32 KB limit
constexpr int kPersistSteps = 64;  // steps per persistent launch (one hop bit each)

// Graph mode's kernel: the events of one geometry class (equal nx, ny, nz)
// in one launch, blockIdx.z the event within the class, blockIdx.y the z
// slice, blockIdx.x the transverse tile.  The geometry is a parameter of the
// launch, so the per-link update's address arithmetic treats it as the
// single-event kernel does (a constant operand); only the event's pointers,
// windows and hop flag are selected by blockIdx.z.  (With the geometry of
// each event selected per block, the update executed 8.7 % more
// instructions per FMA, mostly uniform-register and integer address work.)
template <typename R>
struct GroupEvent {
  const typename V2T<R>::T* U;
  typename V2T<R>::T* Un;
  R* E;
  R* QA;
  R* QB;
  int zA0, WA, zB0, WB;
  int hop;
};

template <typename R>
struct GroupArgs {
  Geom g;
  R dt;
  R w[3];
  R az2;
  GroupEvent<R> ev[kMaxBatch];  // kernel parameters: 64 x 64 B, under the 32 KB limit
};

template <int BX> struct BatchOcc { static constexpr int blocks = 576 / (3 * BX) > 0 ? 576 / (3 * BX) : 1; };

template <int NC, typename R, int BX>
__global__ void __launch_bounds__(3 * BX, sizeof(R) == 4 ? BatchOcc<BX>::blocks : 1)
    k_step_group(const __grid_constant__ GroupArgs<R> b) {
  const GroupEvent<R>& ev = b.ev[blockIdx.z];
  StepArgs<R> a;
  a.U = ev.U;
  a.Un = ev.Un;
  a.E = ev.E;
  a.QA = ev.QA;
  a.QB = ev.QB;
  a.g = b.g;
  a.dt = b.dt;
  a.w[0] = b.w[0];
  a.w[1] = b.w[1];
  a.w[2] = b.w[2];
  a.az2 = b.az2;
  a.hop = ev.hop;
  a.zA0 = ev.zA0;
  a.WA = ev.WA;
  a.zB0 = ev.zB0;
  a.WB = ev.WB;
  a.zlo = 0;
  step_link<NC, R>(a, (int)threadIdx.y, blockIdx.x * BX + threadIdx.x, (int)blockIdx.y);
}

// Events grouped by geometry, in order of first appearance.
static std::vector<std::vector<int>> geometry_groups(const std::vector<glasma_ctx*>& ev) {
  std::vector<std::vector<int>> out;
  for (int e = 0; e < (int)ev.size(); ++e) {
    bool placed = false;
    for (auto& grp : out) {
      const Geom& g = ev[grp[0]]->g;
      if (g.nx == ev[e]->g.nx && g.ny == ev[e]->g.ny && g.nz == ev[e]->g.nz) {
        grp.push_back(e);
        placed = true;
        break;
      }
    }
    if (!placed) out.push_back(std::vector<int>(1, e));
  }
  return out;
}

// Host-side plan of one step for one geometry class (pointers and windows
// as they will be when that step runs).
template <typename R>
static void plan_group(const std::vector<glasma_ctx*>& ev, const std::vector<int>& grp, const std::vector<int>& cur,
                       const std::vector<long long>& n, const std::vector<int>& zA0, const std::vector<int>& zB0,
                       GroupArgs<R>& b) {
  const glasma_params& p = ev[grp[0]]->p;
  b.g = ev[grp[0]]->g;
  b.dt = (R)p.dt;
  b.w[0] = (R)(2.0 / (p.a_t * p.a_t));
  b.w[1] = b.w[0];
  b.w[2] = (R)(2.0 / (p.a_z * p.a_z));
  b.az2 = (R)(p.a_z * p.a_z);
  for (size_t k = 0; k < grp.size(); ++k) {
    const int e = grp[k];
    glasma_ctx* c = ev[e];
    GroupEvent<R>& d = b.ev[k];
    d.U = (const typename V2T<R>::T*)c->U[cur[e]];
    d.Un = (typename V2T<R>::T*)c->U[1 - cur[e]];
    d.E = (R*)c->E;
    d.QA = (R*)c->QA;
    d.QB = (R*)c->QB;
    d.zA0 = zA0[e];
    d.WA = c->WA;
    d.zB0 = zB0[e];
    d.WB = c->WB;
    d.hop = hop_at(n[e], c->hop_p, c->hop_q) ? 1 : 0;
  }
}

template <int NC, typename R>
static int launch_group(const GroupArgs<R>& b, int nev, int bx, cudaStream_t s) {
  const dim3 grid((unsigned)((b.g.nxy + bx - 1) / bx), (unsigned)b.g.nz, (unsigned)nev);
  if (bx == 32) k_step_group<NC, R, 32><<<grid, dim3(32, 3), 0, s>>>(b);
  else if (bx == 128) k_step_group<NC, R, 128><<<grid, dim3(128, 3), 0, s>>>(b);
  else k_step_group<NC, R, 64><<<grid, dim3(64, 3), 0, s>>>(b);
  return cuda_check(cudaGetLastError(), "k_step_group launch");
}

// ---------------------------------------------------------------------------
// Persistent variant: one cooperative launch runs all steps of a call.  Its
// blocks (as many as fit on the GPU at once) take the work items of a step
// in a grid-stride loop and meet at a grid barrier between steps.  The hop
// schedule and the window origins of step k follow from the event's step
// index at the start of the call, so nothing is read back between steps.
// ---------------------------------------------------------------------------

template <typename R>
struct PersistEvent {
  typename V2T<R>::T* U[2];  // U[0]: links at the launch's first step
  R* E;
  R* QA;
  R* QB;
  Geom g;
  int zA0, WA, zB0, WB;      // windows at the launch's first step
  unsigned long long hops;   // bit k: step k of the launch is a hop step
  uint32_t block0, ntb;
};

template <typename R>
struct PersistArgs {
  int n;
  int steps;             // at most kPersistSteps
  R dt;
  R w[3];
  R az2;
  uint32_t total;        // work items per step
  uint32_t arrivals;     // blocks expected at every barrier
  long long wait_cycles; // spin budget of one barrier wait (SM clock cycles)
  unsigned long long* bar;
  int* err;
  PersistEvent<R> ev[kMaxBatch];
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier on a counter that only grows within a launch: block arrival
// number k waits until the counter reaches k * arrivals.  The wait is
// bounded: after wait_cycles SM cycles, or once another block has given up,
// the block records the failure in *err and the barrier returns false.
__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned long long target, int* err,
                                             long long wait_cycles) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    red_release_add_u64(bar, 1ull);
    const long long t0 = clock64();
    int good = 1;
    while (ld_acquire_u64(bar) < target) {
      if (*(volatile int*)err) {
        good = 0;
        break;
      }
      if (clock64() - t0 > wait_cycles) {
        atomicExch(err, 1);
        good = 0;
        break;
      }
      __nanosleep(32);
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <int BX> struct PersistOcc { static constexpr int blocks = 480 / (3 * BX) > 0 ? 480 / (3 * BX) : 1; };

template <int NC, typename R, int BX>
__global__ void __launch_bounds__(3 * BX, sizeof(R) == 4 ? PersistOcc<BX>::blocks : 1)
    k_step_persistent(const __grid_constant__ PersistArgs<R> a) {
  for (int k = 0; k < a.steps; ++k) {
    for (uint32_t w = blockIdx.x; w < a.total; w += gridDim.x) {
      int lo = 0, hi = a.n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.ev[mid].block0 <= w) lo = mid;
        else hi = mid - 1;
      }
      const PersistEvent<R>& ev = a.ev[lo];
      const uint32_t local = w - ev.block0;
      const unsigned long long below = ev.hops & ((1ull << k) - 1ull);
      const int moved = __popcll(below);
      StepArgs<R> s;
      s.U = ev.U[k & 1];
      s.Un = ev.U[(k & 1) ^ 1];
      s.E = ev.E;
      s.QA = ev.QA;
      s.QB = ev.QB;
      s.g = ev.g;
      s.dt = a.dt;
      s.w[0] = a.w[0];
      s.w[1] = a.w[1];
      s.w[2] = a.w[2];
      s.az2 = a.az2;
      s.hop = (int)((ev.hops >> k) & 1ull);
      s.zA0 = ev.zA0 - moved;
      s.WA = ev.WA;
      s.zB0 = ev.zB0 + moved;
      s.WB = ev.WB;
      s.zlo = 0;
      step_link<NC, R>(s, (int)threadIdx.y, (local % ev.ntb) * BX + threadIdx.x, (int)(local / ev.ntb));
    }
    if (k + 1 < a.steps &&
        !grid_barrier(a.bar, (unsigned long long)(k + 1) * a.arrivals, a.err, a.wait_cycles))
      return;
  }
}

template <int NC, typename R, int BX>
static int persist_launch(PersistArgs<R>& a, int extra_arrivals, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  int st = cuda_check(cudaGetDevice(&dev), "device");
  if (!st) st = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (!st)
    st = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_persistent<NC, R, BX>, 3 * BX, 0),
                    "occupancy");
  if (st) return st;
  if (per_sm < 1) return set_error(GLASMA_ERR_INTERNAL, "persistent step kernel does not fit on an SM");
  uint32_t grid = (uint32_t)sms * (uint32_t)per_sm;
  if (a.total < grid) grid = a.total;
  if (grid < 1) grid = 1;
  a.arrivals = grid + (uint32_t)extra_arrivals;
  void* args[] = {(void*)&a};
  st = cuda_check(cudaLaunchCooperativeKernel((const void*)k_step_persistent<NC, R, BX>, dim3(grid), dim3(BX, 3),
                                              args, 0, s),
                  "k_step_persistent launch");
  return st;
}

template <int NC, typename R>
static int launch_persistent(PersistArgs<R>& a, int bx, int extra_arrivals, cudaStream_t s) {
  if (bx == 32) return persist_launch<NC, R, 32>(a, extra_arrivals, s);
  if (bx == 128) return persist_launch<NC, R, 128>(a, extra_arrivals, s);
  return persist_launch<NC, R, 64>(a, extra_arrivals, s);
}

}  // namespace glasma

struct glasma_batch {
  std::vector<glasma_ctx*> ev;
  int bx = 64;                       // transverse sites per block
  int mode = GLASMA_BATCH_GRAPH;
  int device = 0;
  cudaStream_t stream = nullptr;     // the events' stream
  cudaStream_t capture = nullptr;    // private stream the graph is captured on
  unsigned long long* bar = nullptr; // persistent mode: barrier counter, then the error word
  long long wait_cycles = 2000000000LL;  // about a second at the GB300 SM clock
  int extra_arrivals = 0;
  int last_launches = 0;
};

using namespace glasma;

// Host copy of the per-event bookkeeping that a batched call advances.
struct EventCursor {
  std::vector<int> cur, zA0, zB0;
  std::vector<long long> n;
  explicit EventCursor(const glasma_batch* b) {
    for (const glasma_ctx* c : b->ev) {
      cur.push_back(c->cur);
      zA0.push_back(c->zA0);
      zB0.push_back(c->zB0);
      n.push_back(c->n);
    }
  }
  // true if no charge of any event leaves its lattice in the next step
  bool next_step_fits(const glasma_batch* b) const {
    for (size_t e = 0; e < b->ev.size(); ++e) {
      const glasma_ctx* c = b->ev[e];
      if (!hop_at(n[e], c->hop_p, c->hop_q)) continue;
      if (c->WB > 0 && zB0[e] + c->WB - 1 >= c->g.nz - 1) return false;
      if (c->WA > 0 && zA0[e] <= 0) return false;
    }
    return true;
  }
  void advance(const glasma_batch* b) {
    for (size_t e = 0; e < b->ev.size(); ++e) {
      const glasma_ctx* c = b->ev[e];
      if (hop_at(n[e], c->hop_p, c->hop_q)) {
        zB0[e] += 1;
        zA0[e] -= 1;
      }
      cur[e] = 1 - cur[e];
      n[e] += 1;
    }
  }
  void store(glasma_batch* b, int launches) const {
    for (size_t e = 0; e < b->ev.size(); ++e) {
      glasma_ctx* c = b->ev[e];
      c->cur = cur[e];
      c->zA0 = zA0[e];
      c->zB0 = zB0[e];
      c->n = n[e];
      c->last_launches = launches;
    }
    b->last_launches = launches;
  }
};

// Number of the next n_steps steps that every event can take.
static int steps_allowed(const glasma_batch* b, int n_steps) {
  EventCursor cs(b);
  int k = 0;
  for (; k < n_steps && cs.next_step_fits(b); ++k) cs.advance(b);
  return k;
}

// Graph mode: capture, for every step, one k_step_group launch per
// geometry class on the private stream, launch the graph on the events'
// stream, advance the bookkeeping.
template <int NC, typename R>
static int graph_run(glasma_batch* b, int steps, int bx) {
  if (steps == 0) return GLASMA_OK;
  EventCursor cs(b);
  const std::vector<std::vector<int>> groups = geometry_groups(b->ev);
  int st = cuda_check(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "batch capture begin");
  if (st) return st;
  for (int k = 0; k < steps && !st; ++k) {
    for (size_t q = 0; q < groups.size() && !st; ++q) {
      GroupArgs<R> args;
      plan_group<R>(b->ev, groups[q], cs.cur, cs.n, cs.zA0, cs.zB0, args);
      st = launch_group<NC, R>(args, (int)groups[q].size(), bx, b->capture);
    }
    cs.advance(b);
  }
  cudaGraph_t graph = nullptr;
  const int st_end = cuda_check(cudaStreamEndCapture(b->capture, &graph), "batch capture end");
  if (st || st_end) {
    if (graph) cudaGraphDestroy(graph);
    return st ? st : st_end;
  }
  cudaGraphExec_t exec = nullptr;
  st = cuda_check(cudaGraphInstantiate(&exec, graph, 0), "batch graph instantiate");
  if (!st) st = cuda_check(cudaGraphLaunch(exec, b->stream), "batch graph launch");
  if (exec) cudaGraphExecDestroy(exec);  // freed once the launch completes
  cudaGraphDestroy(graph);
  if (st) return st;
  cs.store(b, steps * (int)groups.size());
  return GLASMA_OK;
}

// Persistent mode: one cooperative launch for all `steps` steps; reads the
// barrier's error word back (synchronises the stream).
template <int NC, typename R>
static int persistent_launch_run(glasma_batch* b, int steps, int bx) {
  const glasma_params& p = b->ev[0]->p;
  PersistArgs<R> a;
  a.n = (int)b->ev.size();
  a.steps = steps;
  a.dt = (R)p.dt;
  a.w[0] = (R)(2.0 / (p.a_t * p.a_t));
  a.w[1] = a.w[0];
  a.w[2] = (R)(2.0 / (p.a_z * p.a_z));
  a.az2 = (R)(p.a_z * p.a_z);
  a.wait_cycles = b->wait_cycles;
  a.bar = b->bar;
  a.err = (int*)(b->bar + 1);
  uint32_t block0 = 0;
  for (size_t e = 0; e < b->ev.size(); ++e) {
    glasma_ctx* c = b->ev[e];
    PersistEvent<R>& d = a.ev[e];
    d.U[0] = (typename V2T<R>::T*)c->U[c->cur];
    d.U[1] = (typename V2T<R>::T*)c->U[1 - c->cur];
    d.E = (R*)c->E;
    d.QA = (R*)c->QA;
    d.QB = (R*)c->QB;
    d.g = c->g;
    d.zA0 = c->zA0;
    d.WA = c->WA;
    d.zB0 = c->zB0;
    d.WB = c->WB;
    d.hops = 0;
    for (int k = 0; k < steps; ++k)
      if (hop_at(c->n + k, c->hop_p, c->hop_q)) d.hops |= 1ull << k;
    d.block0 = block0;
    d.ntb = (uint32_t)((c->g.nxy + bx - 1) / bx);
    block0 += d.ntb * (uint32_t)c->g.nz;
  }
  a.total = block0;
  int st = cuda_check(cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned long long), b->stream), "barrier reset");
  if (!st) st = launch_persistent<NC, R>(a, bx, b->extra_arrivals, b->stream);
  int herr = 0;
  if (!st) st = cuda_check(cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "barrier status");
  if (!st) st = cuda_check(cudaStreamSynchronize(b->stream), "persistent step");
  if (st) return st;
  if (herr)
    return set_error(GLASMA_ERR_TIMEOUT,
                     "a grid barrier wait of the persistent step ran out; the events' states are undefined");
  EventCursor cs(b);
  for (int k = 0; k < steps; ++k) cs.advance(b);
  cs.store(b, 1);
  return GLASMA_OK;
}

template <int NC, typename R>
static int persistent_run(glasma_batch* b, int steps, int bx) {
  int launches = 0;
  for (int done = 0; done < steps; done += kPersistSteps) {
    const int n = steps - done < kPersistSteps ? steps - done : kPersistSteps;
    const int st = persistent_launch_run<NC, R>(b, n, bx);
    if (st) return st;
    ++launches;
  }
  for (glasma_ctx* c : b->ev) c->last_launches = launches;
  b->last_launches = launches;
  return GLASMA_OK;
}

// Per-event mode: the single-event step kernel of every event and step
// (the kernel glasma_step would use for that context), launched step by step
// on the batch's stream; no batched kernel, for events that fill the GPU on
// their own.  Their launches queue far ahead of the GPU, so a graph saves
// nothing here, while capturing and instantiating one per call (steps x
// events nodes) cost 10 % of the ensemble's step time.
static int per_event_run(glasma_batch* b, int steps) {
  if (steps == 0) return GLASMA_OK;
  const size_t ne = b->ev.size();
  EventCursor cs(b);
  int st = GLASMA_OK;
  for (int k = 0; k < steps && !st; ++k) {
    for (size_t e = 0; e < ne && !st; ++e) {
      glasma_ctx* c = b->ev[e];
      c->cur = cs.cur[e];
      c->zA0 = cs.zA0[e];
      c->zB0 = cs.zB0[e];
      st = launch_step_chosen(c, hop_at(cs.n[e], c->hop_p, c->hop_q));
    }
    cs.advance(b);
  }
  if (st) return st;
  cs.store(b, steps * (int)ne);
  return GLASMA_OK;
}

template <int NC, typename R>
static int batch_run(glasma_batch* b, int n_steps, int mode, int bx) {
  const int allowed = steps_allowed(b, n_steps);
  const int st = mode == GLASMA_BATCH_PERSISTENT ? persistent_run<NC, R>(b, allowed, bx)
                 : mode == GLASMA_BATCH_PER_EVENT ? per_event_run(b, allowed)
                                                  : graph_run<NC, R>(b, allowed, bx);
  if (st) return st;
  if (allowed < n_steps)
    return set_error(GLASMA_ERR_PARTICLE_EXIT, "a charge of a batched event would leave its lattice");
  return GLASMA_OK;
}

static int batch_dispatch(glasma_batch* b, int n_steps, int mode, int bx) {
  const glasma_ctx* c = b->ev[0];
  if (c->p.nc == 2)
    return c->rs == 8 ? batch_run<2, double>(b, n_steps, mode, bx) : batch_run<2, float>(b, n_steps, mode, bx);
  return c->rs == 8 ? batch_run<3, double>(b, n_steps, mode, bx) : batch_run<3, float>(b, n_steps, mode, bx);
}

extern "C" {

GLASMA_API int glasma_batch_create(glasma_ctx* const* ctxs, int n, glasma_batch** out) {
  if (!out) return set_error(GLASMA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1 || n > kMaxBatch) return set_error(GLASMA_ERR_INVALID_ARG, "a batch holds 1 to 64 events");
  const glasma_ctx* c0 = ctxs[0];
  for (int e = 0; e < n; ++e) {
    const glasma_ctx* c = ctxs[e];
    if (!c) return set_error(GLASMA_ERR_INVALID_ARG, "NULL context in batch");
    if (c->p.scheme != GLASMA_LEAPFROG) return set_error(GLASMA_ERR_INVALID_ARG, "batched events use the leapfrog scheme");
    if (c->slab) return set_error(GLASMA_ERR_INVALID_ARG, "batched events are whole lattices, not slabs");
    if (c->p.nc != c0->p.nc || c->p.precision != c0->p.precision || c->p.dt != c0->p.dt || c->p.a_t != c0->p.a_t ||
        c->p.a_z != c0->p.a_z || c->device != c0->device || c->stream != c0->stream)
      return set_error(GLASMA_ERR_INVALID_ARG, "batched events must share nc, precision, dt, a_t, a_z, device and stream");
    for (int f = 0; f < e; ++f)
      if (ctxs[f] == c) return set_error(GLASMA_ERR_INVALID_ARG, "an event appears twice in the batch");
  }
  cudaSetDevice(c0->device);
  glasma_batch* b = new glasma_batch();
  b->ev.assign(ctxs, ctxs + n);
  b->device = c0->device;
  b->stream = c0->stream;
  int st = cuda_check(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "batch stream");
  if (!st) {
    b->bar = (unsigned long long*)ctx_alloc(b->ev[0], 2 * sizeof(unsigned long long));
    if (!b->bar) st = set_error(GLASMA_ERR_OOM, "barrier word allocation failed");
  }
  if (!st) st = cuda_check(cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned long long), b->stream), "barrier reset");
  if (st) {
    glasma_batch_free(b);
    return st;
  }
  *out = b;
  return GLASMA_OK;
}

GLASMA_API int glasma_batch_step(glasma_batch* b, int n_steps) {
  if (!b || n_steps < 0) return set_error(GLASMA_ERR_INVALID_ARG, "bad batch or n_steps");
  cudaSetDevice(b->device);
  return batch_dispatch(b, n_steps, b->mode, b->bx);
}

GLASMA_API int glasma_batch_set_shape(glasma_batch* b, int mode, int block_sites) {
  if (!b || mode < GLASMA_BATCH_GRAPH || mode > GLASMA_BATCH_PER_EVENT ||
      (block_sites != 32 && block_sites != 64 && block_sites != 128))
    return set_error(GLASMA_ERR_INVALID_ARG, "unknown mode, or block_sites not 32, 64 or 128");
  b->mode = mode;
  b->bx = block_sites;
  return GLASMA_OK;
}

GLASMA_API int glasma_batch_set_barrier(glasma_batch* b, long long wait_cycles, int extra_arrivals) {
  if (!b || wait_cycles < 1 || extra_arrivals < 0 || extra_arrivals > 1024)
    return set_error(GLASMA_ERR_INVALID_ARG, "wait_cycles must be >= 1 and extra_arrivals in 0..1024");
  b->wait_cycles = wait_cycles;
  b->extra_arrivals = extra_arrivals;
  return GLASMA_OK;
}

GLASMA_API int glasma_batch_tune(glasma_batch* b, int steps, int* block_sites, int* mode) {
  if (!b || steps < 1) return set_error(GLASMA_ERR_INVALID_ARG, "bad batch or steps");
  cudaSetDevice(b->device);
  if (steps_allowed(b, steps + 1) < steps + 1)
    return set_error(GLASMA_ERR_PARTICLE_EXIT, "the trial steps would move a charge off a lattice");
  const size_t ne = b->ev.size();
  // snapshot of the current links, E and charge windows of every event and
  // of the host bookkeeping, restored after each trial
  struct Snap {
    void* buf[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t bytes[4] = {0, 0, 0, 0};
    int cur = 0, zA0 = 0, zB0 = 0;
    long long n = 0;
  };
  std::vector<Snap> snap(ne);
  auto live = [](glasma_ctx* c, int k) -> void* {
    return k == 0 ? c->U[c->cur] : k == 1 ? c->E : k == 2 ? c->QA : c->QB;
  };
  int st = GLASMA_OK;
  for (size_t e = 0; e < ne && !st; ++e) {
    glasma_ctx* c = b->ev[e];
    Snap& s = snap[e];
    s.bytes[0] = link_bytes(c);
    s.bytes[1] = c->rs * 3 * (size_t)c->na * c->g.V;
    s.bytes[2] = c->rs * (size_t)c->na * c->WA * c->g.nxy;
    s.bytes[3] = c->rs * (size_t)c->na * c->WB * c->g.nxy;
    s.cur = c->cur;
    s.zA0 = c->zA0;
    s.zB0 = c->zB0;
    s.n = c->n;
    for (int k = 0; k < 4 && !st; ++k) {
      if (!s.bytes[k]) continue;
      s.buf[k] = ctx_alloc(c, s.bytes[k]);
      if (!s.buf[k]) st = set_error(GLASMA_ERR_OOM, "tuning snapshot allocation failed");
      else st = cuda_check(cudaMemcpyAsync(s.buf[k], live(c, k), s.bytes[k], cudaMemcpyDeviceToDevice, b->stream), "snapshot");
    }
  }
  auto restore = [&]() {
    int r = GLASMA_OK;
    for (size_t e = 0; e < ne && !r; ++e) {
      glasma_ctx* c = b->ev[e];
      const Snap& s = snap[e];
      c->cur = s.cur;
      c->zA0 = s.zA0;
      c->zB0 = s.zB0;
      c->n = s.n;
      for (int k = 0; k < 4 && !r; ++k)
        if (s.bytes[k])
          r = cuda_check(cudaMemcpyAsync(live(c, k), s.buf[k], s.bytes[k], cudaMemcpyDeviceToDevice, b->stream), "restore");
    }
    return r;
  };
  const int shapes[3] = {32, 64, 128};
  float best = -1.f;
  int best_bx = 64, best_mode = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!st) st = cuda_check(cudaEventCreate(&e0), "event");
  if (!st) st = cuda_check(cudaEventCreate(&e1), "event");
  // batched graph and persistent with each block shape, then per-event
  for (int trial = 0; trial < 7 && !st; ++trial) {
    const int mode = trial == 6 ? GLASMA_BATCH_PER_EVENT : trial / 3, bx = trial == 6 ? 64 : shapes[trial % 3];
    st = batch_dispatch(b, 1, mode, bx);  // warm-up: module load, caches
    if (!st) st = cuda_check(cudaEventRecord(e0, b->stream), "event");
    if (!st) st = batch_dispatch(b, steps, mode, bx);
    if (!st) st = cuda_check(cudaEventRecord(e1, b->stream), "event");
    if (!st) st = cuda_check(cudaEventSynchronize(e1), "event sync");
    float ms = 0.f;
    if (!st) st = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event time");
    const int r = restore();
    if (!st) st = r;
    if (!st && (best < 0.f || ms < best)) {
      best = ms;
      best_bx = bx;
      best_mode = mode;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(b->stream);
  for (size_t e = 0; e < ne; ++e)
    for (int k = 0; k < 4; ++k) ctx_free(b->ev[e], snap[e].buf[k]);
  if (st) return st;
  b->bx = best_bx;
  b->mode = best_mode;
  if (block_sites) *block_sites = best_bx;
  if (mode) *mode = best_mode;
  return GLASMA_OK;
}

GLASMA_API void glasma_batch_free(glasma_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->bar) ctx_free(b->ev[0], b->bar);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

}  // extern "C"
