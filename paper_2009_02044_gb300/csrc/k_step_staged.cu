// Leapfrog step with the CPIC hop, staple form with the links staged in
// shared memory by the bulk-copy engine (Sec. 3, Eqs. lattice_1, plaquette,
// lattice_2, continuity).  FP32 SU(3) state, transverse rows of 32 or 64
// sites.
//
// A block owns kStR full transverse rows (x is periodic inside a row) and
// marches through a chunk of z slices.  The links of the rows iy0 - 1 ..
// iy0 + kStR (a one-row halo on each side) of four consecutive slices live
// in shared memory (four slots): the update of slice z reads slices z - 1,
// z and z + 1.  A row of one direction is the contiguous run of its 32-site
// link blocks (the SU(3) layout of lattice.cuh), so the shared image keeps
// the global block layout and a warp reads 32 consecutive sites of one
// component.  One consumer thread per link, all three directions of the
// tile's sites in one block; every link update performs exactly the
// arithmetic of step_link, in the same order, so the result is bitwise that
// of the staple kernel.
//
// One more warp produces: its first lane copies slice s into slot s % 4
// with cp.async.bulk (one copy per row and direction, the bytes counted on
// the slot's full barrier) as soon as every consumer thread has released
// slice s - 4 on the slot's empty barrier.  A consumer releases slice z - 1
// after its update of slice z, the last one that reads it.  No barrier
// spans the block after the start, so warps run up to a slice apart and the
// copies run up to three slices ahead.
//
// Every wait is bounded (staged_wait SM cycles, about a second by default).
// A consumer whose wait runs out stops and raises the block's abort flag;
// the other consumers stop at their next slice; the producer stops issuing,
// waits (bounded) for the copies it has in flight, and, being the last
// thread to use the block's shared memory, exits after them.  The context's
// staged status word is set, and the next call that returns host values
// reports GLASMA_ERR_TIMEOUT.
#include "step_link.cuh"

namespace glasma {

constexpr int kStR = 2;      // interior rows per block
constexpr int kStSlots = 4;  // slices held in shared memory

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sm_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned), completing its bytes on the mbarrier b
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sm_addr(dst)),
               "l"(src), "r"(bytes), "r"(sm_addr(b))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Wait for the completion of phase `parity` of barrier b; false once
// `cycles` SM cycles have passed without it.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long cycles) {
  const long long t0 = clock64();
  while (!mbar_test(b, parity))
    if (clock64() - t0 > cycles) return false;
  return true;
}

// The producer's wait for its copies in flight always allows 2^31 cycles:
// they must land before the block's shared memory is released.
constexpr long long kStDrainCycles = 1ll << 31;

template <int RB>
struct StagedGeo {
  static constexpr int NX = 32 * RB;
  static constexpr int ROWS = kStR + 2;
  static constexpr int DIRB = ROWS * RB * 288;  // float2 per (slot, direction)
  static constexpr int SLOTB = 3 * DIRB;        // float2 per slot
  static constexpr int CONSUMERS = 3 * kStR * NX;
  static constexpr int THREADS = CONSUMERS + 32;  // one producer warp
  // the slots, then a full and an empty barrier per slot and one barrier
  // that nothing completes (the stall test waits on it)
  static constexpr size_t smem =
      (size_t)kStSlots * SLOTB * sizeof(float2) + (2 * kStSlots + 1) * sizeof(unsigned long long);
};

template <int RB>
__device__ __forceinline__ LinkAlg<3, float>::M st_load(const float2* sm, int q, int d, int rr, int ix) {
  typedef StagedGeo<RB> SG;
  const float2* p = sm + (q * 3 + d) * SG::DIRB + (rr * RB + (ix >> 5)) * 288 + (ix & 31);
  LinkAlg<3, float>::M m;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 v = p[k * 32];
    m.m[k] = cplx<float>{v.x, v.y};
  }
  return m;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(b)) : "memory");
}

struct StagedArgs {
  StepArgs<float> s;
  int zhi;
  int zlen;
  long long wait;
  int stall;
  int* status;
};

// Producer warp (lane 0): slice zs goes to slot zs & 3 once the slice four
// before it has been released by every consumer thread (empty barrier).
// Consumers: wait for the slice's full barrier, update, release slice z - 1
// after iteration z (its last reader).
template <int RB>
__global__ void __launch_bounds__(StagedGeo<RB>::THREADS, 1) k_step_staged(StagedArgs sa) {
  typedef StagedGeo<RB> SG;
  typedef LinkAlg<3, float> G;
  typedef G::M M;
  constexpr int NX = SG::NX, ROWS = SG::ROWS;
  extern __shared__ __align__(128) unsigned char st_raw[];
  float2* sm = (float2*)st_raw;
  unsigned long long* full = (unsigned long long*)(st_raw + (size_t)kStSlots * SG::SLOTB * sizeof(float2));
  unsigned long long* empty = full + kStSlots;
  unsigned long long* unarmed = full + 2 * kStSlots;
  __shared__ volatile int abort_flag;
  const StepArgs<float>& a = sa.s;
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int iy0 = blockIdx.x * kStR;
  const int z0 = a.zlo + blockIdx.y * sa.zlen;
  const int z1 = min(z0 + sa.zlen, sa.zhi);
  const int lo_load = max(z0 - 1, 0), hi_load = min(z1, g.nz - 1);
  if (tid == 0) {
    abort_flag = 0;
    for (int q = 0; q < kStSlots; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], SG::CONSUMERS);
    }
    mbar_init(unarmed, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid >= SG::CONSUMERS) {
    // ---- producer ----
    if (tid != SG::CONSUMERS) return;
    const int64_t C = (g.V + 31) >> 5;
    const int64_t bps = g.nxy >> 5;
    const unsigned slice_bytes = 3u * ROWS * RB * 2304u;
    int issued = lo_load - 1;
    bool ok = !(sa.stall && blockIdx.x == 0 && blockIdx.y == 0 && !mbar_wait(unarmed, 0, sa.wait));
    for (int zs = lo_load; zs <= hi_load && ok; ++zs) {
      const int q = zs & (kStSlots - 1);
      const int k = (zs - lo_load) >> 2;  // use of this slot
      if (k > 0) {
        // the slice four before has been released (bounded, and given up
        // if a consumer has aborted)
        const long long t0 = clock64();
        while (!mbar_test(&empty[q], (unsigned)((k - 1) & 1))) {
          if (abort_flag || clock64() - t0 > sa.wait) {
            ok = false;
            break;
          }
        }
        if (!ok) break;
        fence_proxy_async();
      }
      mbar_expect_tx(&full[q], slice_bytes);
      for (int d = 0; d < 3; ++d)
        for (int rr = 0; rr < ROWS; ++rr) {
          const int gy = ((iy0 - 1 + rr) % g.ny + g.ny) % g.ny;
          const float2* src = a.U + (((int64_t)d * C + (int64_t)zs * bps + (int64_t)gy * RB) * 9) * 32;
          bulk_to_smem(sm + (q * 3 + d) * SG::DIRB + rr * RB * 288, src, RB * 2304u, &full[q]);
        }
      issued = zs;
    }
    // the copies still in flight land before this thread (the last user of
    // the block's shared memory) may exit
    for (int zs = max(lo_load, issued - 3); zs <= issued; ++zs)
      mbar_wait(&full[zs & (kStSlots - 1)], (unsigned)(((zs - lo_load) >> 2) & 1), kStDrainCycles);
    if (!ok) {
      abort_flag = 1;
      atomicExch(sa.status, 1);
    }
    return;
  }
  // ---- consumers ----
  const int i = tid / (kStR * NX);
  const int loc = tid - i * (kStR * NX);
  const int r = loc / NX, ix = loc - r * NX;
  const int iy = iy0 + r;
  const bool inner = iy < g.ny;
  const uint32_t t = (uint32_t)(inner ? iy : 0) * NX + ix;
  auto wait_full = [&](int zs) -> bool {
    return mbar_wait(&full[zs & (kStSlots - 1)], (unsigned)(((zs - lo_load) >> 2) & 1), sa.wait);
  };
  bool good = true;
  for (int zs = lo_load; zs <= min(z0, hi_load) && good; ++zs) good = wait_full(zs);
  for (int z = z0; z < z1 && good; ++z) {
    if (abort_flag) break;
    if (z + 1 <= hi_load && !wait_full(z + 1)) {
      good = false;
      break;
    }
    if (inner && !(i == 2 && z == g.nz - 1)) {
      const int q0 = z & 3, qm = (z - 1) & 3, qp = (z + 1) & 3;
      const int rr0 = r + 1;
      const int xp = ix + 1 == NX ? 0 : ix + 1, xm = ix == 0 ? NX - 1 : ix - 1;
      const int64_t s = (int64_t)z * g.nxy + t;
      float E0[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) E0[c] = a.E[(int64_t)(i * 8 + c) * g.V + s];
      auto nb = [&](int d, int sgn, int& q, int& rr, int& cx) {
        q = q0;
        rr = rr0;
        cx = ix;
        if (d == 0) cx = sgn > 0 ? xp : xm;
        else if (d == 1) rr = rr0 + sgn;
        else q = sgn > 0 ? qp : qm;
      };
      G::Sum S = G::zero_sum();
      const float wt = a.w[0], wz = a.w[2];
#pragma unroll 1
      for (int j = 0; j < 3; ++j) {
        if (j == i) continue;
        const float wj = j == 2 ? wz : wt;
        const bool fwd = (j != 2) || (z <= g.nz - 2);
        const bool bwd = (j != 2) || (z >= 1);
        int qi, ri, ci, qj, rj, cj_, qn, rn, cn;
        nb(i, +1, qi, ri, ci);
        nb(j, +1, qj, rj, cj_);
        nb(j, -1, qn, rn, cn);
        if (fwd) {
          M T = G::mul_d(st_load<RB>(sm, qi, j, ri, ci), st_load<RB>(sm, qj, i, rj, cj_));
          T = G::mul_d(T, st_load<RB>(sm, q0, j, rr0, ix));
          G::sum_add(S, wj, T);
        }
        if (bwd) {
          const int qd = i == 2 ? qp : qn, rd = rn + ri - rr0, cd = i == 0 ? ci : cn;
          M T = G::mul(st_load<RB>(sm, qn, i, rn, cn), st_load<RB>(sm, qd, j, rd, cd));
          T = G::d_mul(T, st_load<RB>(sm, qn, j, rn, cn));
          G::sum_add(S, wj, T);
        }
      }
      float pr[8], F[8];
      const M Ui = st_load<RB>(sm, q0, i, rr0, ix);
      G::proj_mul_sum(Ui, S, pr);
#pragma unroll
      for (int c = 0; c < 8; ++c) F[c] = -pr[c];
      update_link_ue<3, float>(a, i, t, z, s, F, Ui, E0);
    }
    // iteration z is the last to read slice z - 1
    if (z - 1 >= lo_load) mbar_arrive(&empty[(z - 1) & (kStSlots - 1)]);
  }
  if (!good) {
    abort_flag = 1;
    atomicExch(sa.status, 1);
  }
}

// Rows of 32 or 64 sites (one or two link blocks), FP32 SU(3), a whole
// lattice (a slab's halo slices are not staged).
bool staged_fits(const glasma_ctx* c) {
  return c->rs == 4 && c->p.nc == 3 && !c->slab && (c->g.nx == 32 || c->g.nx == 64);
}

template <int RB>
static int launch_staged_t(glasma_ctx* c, bool hop) {
  typedef StagedGeo<RB> SG;
  // the shared-memory limit is a per-device function attribute
  static int attr_set[64] = {0};
  if (c->device < 0 || c->device >= 64) return set_error(GLASMA_ERR_INTERNAL, "device ordinal out of range");
  if (!attr_set[c->device]) {
    int st = cuda_check(cudaFuncSetAttribute(k_step_staged<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SG::smem),
                        "k_step_staged attributes");
    if (st) return st;
    attr_set[c->device] = 1;
  }
  StagedArgs sa;
  StepArgs<float>& a = sa.s;
  a.U = (const float2*)c->U[c->cur];
  a.Un = (float2*)c->U[1 - c->cur];
  a.E = (float*)c->E;
  a.QA = (float*)c->QA;
  a.QB = (float*)c->QB;
  a.g = c->g;
  a.dt = (float)c->p.dt;
  a.w[0] = (float)(2.0 / (c->p.a_t * c->p.a_t));
  a.w[1] = a.w[0];
  a.w[2] = (float)(2.0 / (c->p.a_z * c->p.a_z));
  a.az2 = (float)(c->p.a_z * c->p.a_z);
  a.hop = hop ? 1 : 0;
  a.zA0 = c->zA0;
  a.WA = c->WA;
  a.zB0 = c->zB0;
  a.WB = c->WB;
  a.zlo = c->lo;
  sa.zhi = c->hi;
  sa.wait = c->staged_wait;
  sa.stall = c->staged_stall;
  sa.status = c->dflag + 1;
  // about four waves of one block per SM (608 blocks on 152 SMs for the
  // 512 x 64^2 lattice: 32 tiles of 27 slices), measured best among 2 to 8
  const int tiles = (c->g.ny + kStR - 1) / kStR;
  const int nsl = c->hi - c->lo;
  int chunks = (4 * 152 + tiles / 2) / tiles;
  if (chunks < 1) chunks = 1;
  if (chunks > nsl) chunks = nsl;
  sa.zlen = (nsl + chunks - 1) / chunks;
  chunks = (nsl + sa.zlen - 1) / sa.zlen;
  k_step_staged<RB><<<dim3((unsigned)tiles, (unsigned)chunks), SG::THREADS, SG::smem, c->stream>>>(sa);
  c->staged_launched = true;
  return cuda_check(cudaGetLastError(), "k_step_staged launch");
}

int launch_step_staged(glasma_ctx* c, bool hop) {
  if (!staged_fits(c)) return set_error(GLASMA_ERR_INTERNAL, "staged kernel: FP32 SU(3) rows of 32 or 64 sites only");
  return c->g.nx == 64 ? launch_staged_t<2>(c, hop) : launch_staged_t<1>(c, hop);
}

// GLASMA_ERR_TIMEOUT if a staged launch since the last check recorded a
// wait that ran out (the status word is cleared); synchronises the stream.
int staged_status(glasma_ctx* c) {
  if (!c->staged_launched) return GLASMA_OK;
  int h = 0;
  int st = cuda_check(cudaMemcpyAsync(&h, c->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "staged status");
  if (!st) st = cuda_check(cudaStreamSynchronize(c->stream), "staged status sync");
  if (st) return st;
  c->staged_launched = false;
  if (!h) return GLASMA_OK;
  st = cuda_check(cudaMemsetAsync(c->dflag + 1, 0, sizeof(int), c->stream), "staged status reset");
  if (st) return st;
  return set_error(GLASMA_ERR_TIMEOUT,
                   "a shared-memory staging wait of the step kernel ran out; the state after that step is undefined");
}

}  // namespace glasma
