/*
 * glasma.h -- C ABI of the GB300 library for the laboratory-frame 3+1D Glasma
 * time step with colored particle-in-cell (CPIC) charges.
 *
 * Method: D. Mueller and A. Ipp, "Progress on 3+1D Glasma simulations"
 * (arXiv:2009.02044).  Section numbers and equation labels below refer to
 * that paper.
 *
 * Units and conventions: lattice units with g = 1 and a_T = 1 by default;
 * SU(N_c) generators t^a hermitian with tr(t^a t^b) = delta^{ab}/2;
 * E_i = E_i^a t^a hermitian and U_i(t + dt) = exp(i dt E_i) U_i(t).
 * Lattice: N_L = nz sites along the beam axis z (open boundary: there is no
 * z link on the last slice) and nx * ny transverse sites (periodic).
 * Nucleus A moves towards -z, nucleus B towards +z, both at v = c.
 *
 * Memory: a context owns every device buffer it uses.  It allocates them at
 * glasma_init_mv through the optional allocator (or cudaMallocAsync on the
 * given stream) and releases them in glasma_free.  All host pointers passed
 * in are owned by the caller and only read or written during the call.
 *
 * Streams: a context is bound to one CUDA stream and one device.  Calls that
 * return host values (residuals, tables, fields, state) synchronise that
 * stream; glasma_step only enqueues work.
 *
 * Errors: every call returns GLASMA_OK (0) or a negative status; nothing is
 * thrown across the ABI.  glasma_strerror(status) names the status, and
 * glasma_last_error_message() gives the detail of the most recent failure
 * on the calling thread.
 */
#ifndef GLASMA_H
#define GLASMA_H

#include <stddef.h>

#if defined(__GNUC__)
#define GLASMA_API __attribute__((visibility("default")))
#else
#define GLASMA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GLASMA_OK = 0,
  GLASMA_ERR_INVALID_ARG = -1,   /* a parameter or size is out of range */
  GLASMA_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  GLASMA_ERR_OOM = -3,           /* device allocation failed */
  GLASMA_ERR_NONFINITE = -4,     /* a reduction met NaN or Inf */
  GLASMA_ERR_PARTICLE_EXIT = -5, /* a charge would leave the open z range */
  GLASMA_ERR_NOT_CONVERGED = -6, /* implicit iteration hit max_iter */
  GLASMA_ERR_TIMEOUT = -7,       /* a bounded device wait expired */
  GLASMA_ERR_CHECKSUM = -8,      /* a state blob failed its checksum */
  GLASMA_ERR_INTERNAL = -9       /* an internal consistency check failed */
};

enum { GLASMA_FP64 = 0, GLASMA_FP32 = 1 };
enum { GLASMA_LEAPFROG = 0, GLASMA_IMPLICIT = 1 };

typedef struct glasma_ctx glasma_ctx;

/* Parameters of one event (Sec. 3 and 4).  Sizes in units of a_t. */
typedef struct {
  int nc;                   /* gauge group SU(nc): 2 or 3 */
  int nz, nx, ny;           /* N_L (beam axis, open) and transverse sizes */
  double a_t, a_z, dt;      /* transverse and longitudinal spacing, time step */
  double sigma_l;           /* std. dev. of the Gaussian longitudinal profile */
  double g2mu;              /* g^2 mu a_t: std. dev. of rho^a per cell */
  double m_ir;              /* infrared regulator m of the Poisson solve */
  double uv_cutoff;         /* UV cutoff Lambda on k_T; 0 = none */
  double z_offset;          /* initial distance of each nucleus from the box
                               centre; 0 = (ceil(4 sigma_l / a_z) + 2) a_z */
  unsigned long long seed;  /* MV charge seed (used when rho is not given) */
  int precision;            /* GLASMA_FP64 or GLASMA_FP32 (FP32 links and
                               fields; every reduction in FP64) */
  int scheme;               /* GLASMA_LEAPFROG or GLASMA_IMPLICIT */
  int implicit_max_iter;    /* fixed-point iterations of the implicit scheme */
  double implicit_tol;      /* its convergence threshold on max |dE|; the
                               iteration also ends when the contraction
                               bound d c / (1 - c) (d = max |dE|, c the
                               larger of the last two ratios of d, below
                               1/2) is at most 16 unit roundoffs of max |E|,
                               or when max |dE| is within 64 unit
                               roundoffs of max |E| and falls by less than
                               half, or when it stops decreasing within
                               1024 unit roundoffs of max |E| (the
                               precision's rounding floor); see
                               glasma_implicit_converged */
  int n_sheets;             /* longitudinal colour sheets per nucleus
                               (0 or 1: the single-sheet MV charge; S > 1,
                               at most 64: S independent transverse charges,
                               one per equal-charge slab of the profile, each
                               of std. dev. g2mu / sqrt(S), combined in a
                               path-ordered Wilson line) */
} glasma_params;

/* Optional device allocator (e.g. a framework's caching allocator).  Both
 * callbacks are called only from glasma_init_mv / glasma_free /
 * glasma_set_fields on the calling thread.  alloc must return 16-byte
 * aligned memory (the state arrays are read with 16-byte vector loads);
 * glasma_init_mv rejects anything else with GLASMA_ERR_INVALID_ARG. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} glasma_allocator;

/*
 * Build the MV initial state at t0 (links) and t0 - dt/2 (E and charges)
 * (Sec. 2 MV model; Sec. 3 Eqs. single_sheet, 3d_colorfield_1/2; Sec. 4
 * Gaussian longitudinal profile):
 *   rho_N^a(x_T) -> phi_N = (-Delta_T + m^2)^{-1} rho_N (lattice Laplacian,
 *   optional UV cutoff) -> V_N^dagger(z, x_T) = exp(i Lambda_N(z) phi_N)
 *   -> U_i = V_A(x) V_A^dag(x+i) V_B(x) V_B^dag(x+i) for i = x, y, U_z = 1,
 *   at t0 and t0 - dt; E = -i log(U(t0) U^dag(t0 - dt)) / dt (0 where the
 *   two links are equal); charges from the discrete Gauss law (Eq. gauss),
 *   split by the side of the box centre into the two nuclei.
 * p:        parameters (read only).
 * rho_host: NULL to draw rho from p->seed (Philox4x32-10, counter
 *           (x, y, a, N), Box-Muller), or host doubles [2][nc^2-1][ny][nx]
 *           (N = 0: A, N = 1: B) in units of a_t^-2.
 * stream:   cudaStream_t the context will use (NULL = legacy default).
 * alloc:    NULL for cudaMallocAsync, else the callbacks above.
 * out:      receives the new context (NULL on failure).
 * Errors: INVALID_ARG (nc, sizes: nz in [2, 65535], nx, ny >= 1 and at
 * most 1.5e9 sites; dt > a_z, dt/a_z not a ratio p/q with q <= 4096,
 * nuclei not inside the box), OOM, CUDA, INTERNAL.
 */
GLASMA_API int glasma_init_mv(const glasma_params* p, const double* rho_host, void* stream,
                   const glasma_allocator* alloc, glasma_ctx** out);

/*
 * Advance n_steps time steps (n_steps >= 0).  Each step (Sec. 3):
 * (1) if the nearest-grid-point position of the charges changes (hop
 *     counter floor(m v dt / a_z + 1/2)), each charge is parallel
 *     transported along the crossed z link, Q' = U^dag Q U, and the current
 *     that satisfies the discrete continuity equation (Eq. continuity) is
 *     deposited on that link;
 * (2) E_i += -dt sum_j (2/a_j^2) Im tr t^a [U_{i,j} + U_{i,-j}] + dt j_i
 *     (Eq. lattice_1 with Eq. plaquette);
 * (3) U_i <- exp(i dt E_i) U_i (Eq. lattice_2), re-unitarised in FP32.
 * With scheme = GLASMA_IMPLICIT step (2) uses the time-averaged transverse
 * terms of the semi-implicit scheme (Sec. 3, Fig. wilson (b)), iterated.
 * Enqueued on the context's stream; returns before the work completes.
 * Errors: PARTICLE_EXIT (checked on the host before any work of the
 * offending step is enqueued), NOT_CONVERGED, CUDA, INVALID_ARG.  A wait
 * of the staged step kernel that ran out is reported as TIMEOUT by the
 * next glasma_gauss_residual, glasma_tmunu, glasma_get_fields or
 * glasma_get_state.
 */
GLASMA_API int glasma_step(glasma_ctx* c, int n_steps);

/*
 * Discrete Gauss law (Sec. 3, Eq. gauss) with parallel-transported E:
 *   G^a(x) = sum_i [E_i(x) - U_i^dag(x-i) E_i(x-i) U_i(x-i)]^a / a_i^2
 *            - rho^a(x),  rho = Q_A + Q_B,
 * evaluated in FP64 for either precision (at z = 0 no link enters from
 * below).  Outputs (host doubles, any may be NULL): max_{x,a} |G|, the rms
 * of G over all components, and max |rho|.  Synchronises the stream.
 * Errors: NONFINITE, CUDA.
 */
GLASMA_API int glasma_gauss_residual(glasma_ctx* c, double* max_abs, double* rms, double* rho_max);

/*
 * Energy-momentum tensor per z slice at t_n (Sec. 4: eps, p_L, p_T, S_L of
 * <T^{mu nu}>; Eq. pT_eL), transverse means accumulated in FP64:
 *   e_i^2 = (1/2) sum_a [E_i^a(n-1/2)^2 + E_i^a(n+1/2)^2] / a_i^2,
 *   b_ij = 2 (N_c - Re tr U_ij) / (a_i a_j)^2 at the plaquette's base,
 *   eps = (e_x^2+e_y^2+e_z^2)/2 + b_xy + b_xz + b_yz,
 *   p_T = e_z^2/2 + b_xy,  p_L = eps - 2 p_T,
 *   S_L = sum_a (Ebar_x B_y - Ebar_y B_x) (physical Poynting flux,
 *   positive towards +z), Ebar = time mean of E / a_i,
 *   B_k = -2 Im tr(t^a U_ij) / (a_i a_j) for cyclic (i, j, k).
 * E(n+1/2) comes from a non-committing evaluation of the next E update
 * (including the current of a scheduled hop); the state is unchanged.
 * out: host doubles [nz][4] = (eps, p_L, p_T, S_L) per slice, or NULL.
 * energy_total: a_t^2 a_z nx ny sum_z eps(z), or NULL.
 * Synchronises the stream.  Errors: NONFINITE, CUDA.
 */
GLASMA_API int glasma_tmunu(glasma_ctx* c, double* out, double* energy_total);

/*
 * The same table as glasma_tmunu, written to device memory on the context's
 * stream without synchronising, for sampling T^{mu nu}(t, z) during a run.
 * dev_out: device doubles [nz][4] (eps, p_L, p_T, S_L), 8-byte aligned,
 * owned by the caller.  A slice whose sums met a non-finite value gets a
 * NaN eps (no status: nothing is read back).  Errors: INVALID_ARG, CUDA.
 */
GLASMA_API int glasma_tmunu_device(glasma_ctx* c, double* dev_out);

/*
 * Gauss-law residual of fields the caller owns, computed without allocating
 * any device memory.  The paper has no counterpart of this call: it exists
 * for callers that cannot call cudaMalloc -- for example a health check that
 * must still run after the device has run out of memory, or code inside a
 * framework whose allocator owns all device memory and forbids raw
 * allocations (a raw cudaMalloc can also synchronise the device).
 * It computes the same quantity as glasma_gauss_residual.
 * Inputs are device pointers in the library's layout (x fastest, site
 * s = (iz*ny + iy)*nx + ix, V = nz*ny*nx; R = double for GLASMA_FP64,
 * float for GLASMA_FP32):
 *   U  links (16-byte aligned), complex component k of link d at site s
 *      as (re, im) pairs of R.  SU(2): k = 0, 1 for (alpha, beta) of
 *      [[alpha, beta], [-beta*, alpha*]], at U[(d*V + s)*2 + k] (one
 *      link's two pairs are adjacent).
 *      SU(3): k = 0..8 for the row-major 3x3 entries, in blocks of 32
 *      sites: U[((d*C + s/32)*9 + k)*32 + s%32] with C = ceil(V/32)
 *      (the array holds 3*9*32*C pairs; the padding is not read).
 *      In FP32 the stored matrix is U - 1 (alpha - 1 for SU(2)), in FP64
 *      it is U;
 *   E  fields, E[(d*(nc^2-1) + a)*V + s];
 *   QA, QB charge windows of zA0.. zA0+WA-1 and zB0.. zB0+WB-1 (z slices),
 *      Q[(a*W + w)*nx*ny + t]; a pointer may be NULL when its W is 0.
 * Outputs are host doubles (any may be NULL), as in glasma_gauss_residual.
 * Scratch: a fixed device array inside the library, one row of partials
 * per z slice, so nz may be at most 8192; larger nz is rejected with
 * GLASMA_ERR_INVALID_ARG before any GPU work.  Each call looks up the
 * array's device address with the current device (the one that holds the
 * fields).  With CUDA's lazy module loading, the first call on a device
 * loads this entry point's device code and its 256 KB array, which the GPU
 * then keeps until the process exits: make that first call while device
 * memory is still available (for example right after the context is
 * created); later calls allocate nothing.  All calls share the one array,
 * so calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller.  Work runs on `stream` (cudaStream_t,
 * NULL = legacy default); the call synchronises it and copies the result
 * to pageable host memory, so it cannot be recorded into a CUDA graph.
 * Errors: INVALID_ARG (including a U that is not 16-byte aligned),
 * NONFINITE, CUDA.
 */
GLASMA_API int glasma_gauss_residual_static(int nc, int precision, int nz, int ny, int nx, double a_t,
                                            double a_z, const void* U, const void* E, const void* QA,
                                            int zA0, int WA, const void* QB, int zB0, int WB,
                                            void* stream, double* max_abs, double* rms, double* rho_max);

/* Release every device buffer of the context (stream-ordered) and the
 * context itself.  NULL is ignored. */
GLASMA_API void glasma_free(glasma_ctx* c);

/* Static string naming a status code. */
GLASMA_API const char* glasma_strerror(int status);

/* Detail of the most recent failure on this thread (static storage). */
GLASMA_API const char* glasma_last_error_message(void);

/*
 * Fields in FP64, full lattice, for analysis and tests.  Any pointer may be
 * NULL.  Layouts (host doubles, x fastest):
 *   U  [3][nz][ny][nx][nc][nc][2]  (complex matrices, re/im interleaved)
 *   E  [3][nz][ny][nx][nc^2-1]
 *   QA, QB [nz][ny][nx][nc^2-1]    (charges placed at their lattice sites)
 * step_n receives the step index n (U at t_n, E and charges at t_{n-1/2}).
 * Synchronises the stream.
 */
GLASMA_API int glasma_get_fields(glasma_ctx* c, double* U, double* E, double* QA, double* QB,
                      long long* step_n);

/*
 * Replace the state by host FP64 fields in the layouts of glasma_get_fields
 * (U, E required; QA, QB may be NULL for zero charges) at step index
 * step_n.  Values are rounded to the context's precision.  The z link of
 * the last slice must be the identity and E_z there zero.  The charge
 * windows are rebuilt from the nonzero slices of QA and QB.  U_prev (the
 * links at t_{n-1}, used by the implicit scheme) may be NULL, in which case
 * exp(-i dt E) U is used.  Errors: INVALID_ARG, OOM, CUDA.
 */
GLASMA_API int glasma_set_fields(glasma_ctx* c, const double* U, const double* E, const double* QA,
                      const double* QB, const double* U_prev, long long step_n);

/* Size in bytes of the checkpoint blob of glasma_get_state. */
GLASMA_API int glasma_state_bytes(const glasma_ctx* c, size_t* bytes);

/*
 * Checkpoint: the state (links, E, charge windows, step index, parameters)
 * in the context's own precision, with a header and a CRC-32 per array, so
 * that glasma_set_state restores a bitwise identical state.
 * Errors: INVALID_ARG (buffer too small or from another configuration),
 * CHECKSUM, CUDA.
 */
GLASMA_API int glasma_get_state(glasma_ctx* c, void* host_buf, size_t bytes);
GLASMA_API int glasma_set_state(glasma_ctx* c, const void* host_buf, size_t bytes);

/* Introspection for benchmarks: sites, bytes per link/field and device
 * pointers of the current buffers.  Any pointer may be NULL. */
typedef struct {
  long long sites;          /* nz * ny * nx */
  long long step_n;         /* current step index */
  int nc, precision, scheme;
  int window_a[2];          /* charge window of A: first slice, slices */
  int window_b[2];          /* charge window of B */
  size_t state_device_bytes; /* device bytes of U (both buffers), E, charges */
  int kernel_launches;      /* kernels enqueued by the last glasma_step call */
  int implicit_iters;       /* fixed-point iterations of the last implicit step */
} glasma_info;

GLASMA_API int glasma_get_info(const glasma_ctx* c, glasma_info* info);

/*
 * A lattice split into slabs along the beam axis z (Sec. 4: the beam axis
 * is the long one, 2048 cells against 192^2), one context per rank.  The
 * leapfrog step (Sec. 3 Eq. lattice_1) couples a link only to the slices
 * z - 1, z, z + 1, so a slab needs one halo slice from each neighbour,
 * refreshed before every step; the CPIC hop moves a charge across a slab
 * boundary along a link whose owner transports it and deposits its current.
 *
 * glasma_slab_init: context of the global slices [z0, z1) of the event p
 *   describes (p->nz is the whole lattice's; rho_host, stream, alloc as for
 *   glasma_init_mv, every rank passing the same p and charges).  Its local
 *   lattice is the slab plus a halo slice below (if z0 > 0) and above (if
 *   z1 < nz); the initial state of every owned and halo slice equals the
 *   whole lattice's bit for bit.  The leapfrog step kernel is the staple or
 *   plaquette kernel (never the site-paired one); the improved scheme runs
 *   sweep by sweep (glasma_implicit_begin below).  Errors: INVALID_ARG (as
 *   glasma_init_mv; z0 < 0, z1 > nz, z1 <= z0), OOM, CUDA.
 * glasma_slab_info: owned global slices [*z0, *z1), local slices, and the
 *   local indices [*lo, *hi) of the owned slices (any pointer may be NULL).
 * glasma_slab_set_windows: the charge windows of the whole lattice (first
 *   global slice and number of slices of nucleus A and B): the union over
 *   all slabs of the windows glasma_get_info reports after init (global
 *   slices).  Required once before the first step, so that charges keep
 *   their co-moving slots when they cross into a neighbour.  Errors:
 *   INVALID_ARG (not a slab, outside the lattice, not containing the slab's
 *   own windows), OOM, CUDA.
 * glasma_slab_message_bytes: bytes of the message sent in direction dir
 *   (+1: to the rank above, -1: to the rank below).
 * glasma_slab_pack: write that message into dev_buf (device memory of the
 *   caller, 16-byte aligned, message_bytes long), asynchronously on the
 *   context's stream: dir +1 carries the links of all three directions,
 *   E_z and nucleus B's charge of the top owned slice; dir -1 the
 *   transverse links and nucleus A's charge of the bottom owned slice.
 *   Layout: links [direction][complex component][site] as (re, im) reals in
 *   the stored form (FP32: U - 1), E_z [colour][site], charge
 *   [colour][site] (zeros outside the nucleus' window).
 * glasma_slab_unpack: write a received message into the halo: dir -1 a
 *   message from the rank below (its dir +1 message), dir +1 one from the
 *   rank above; asynchronous on the context's stream.
 * Protocol per step: every rank packs its messages, sends them, receives
 *   its neighbours' and unpacks them, then calls glasma_step(c, 1) (a slab
 *   context takes one step per exchange), or under the improved scheme
 *   glasma_implicit_begin, sweeps with the maxima folded across the ranks,
 *   and glasma_implicit_end (below).  glasma_tmunu then returns the
 *   z1 - z0 rows of the owned slices and their partial energy (the whole
 *   lattice's H is the sum of the gathered rows in z order),
 *   glasma_gauss_residual the residual over the owned slices, and
 *   glasma_get_fields the local lattice (charges on owned slices only).
 *   Errors: INVALID_ARG (bad dir, no neighbour that way, unaligned buffer),
 *   CUDA.
 */
GLASMA_API int glasma_slab_init(const glasma_params* p, const double* rho_host, int z0, int z1, void* stream,
                                const glasma_allocator* alloc, glasma_ctx** out);
GLASMA_API int glasma_slab_info(const glasma_ctx* c, int* z0, int* z1, int* nz_local, int* lo, int* hi);
GLASMA_API int glasma_slab_set_windows(glasma_ctx* c, int zA0, int WA, int zB0, int WB);
GLASMA_API int glasma_slab_message_bytes(const glasma_ctx* c, int dir, size_t* bytes);
GLASMA_API int glasma_slab_pack(glasma_ctx* c, int dir, void* dev_buf);
GLASMA_API int glasma_slab_unpack(glasma_ctx* c, int dir, const void* dev_buf);

/* Kernels of the leapfrog step (the same update, Sec. 3 Eqs. lattice_1,
 * plaquette, lattice_2, continuity, in two work decompositions):
 *   GLASMA_KERNEL_STAPLE       one thread per link; each link sums its four
 *                              staples U_{i,+-j} (every plaquette is formed
 *                              once for each of its four links);
 *   GLASMA_KERNEL_PLAQUETTE    one thread per transverse site marching along
 *                              z; each plaquette is formed once and its
 *                              projection, transported to each of its
 *                              corners, goes to the four links it bounds
 *                              (blocks of up to 320 threads);
 *   GLASMA_KERNEL_PLAQUETTE_256  the same with blocks of up to 256 threads
 *                              (more registers per thread);
 *   GLASMA_KERNEL_STAPLE_PAIRS the staple kernel on two sites per thread,
 *                              (x, y, z) and (x, y, z + ceil(nz/2)), in the
 *                              two lanes of the packed FP32 instructions
 *                              (FP32 state only);
 *   GLASMA_KERNEL_STAPLE_STAGED the staple kernel with the links of two
 *                              transverse rows (plus a one-row halo) of four
 *                              consecutive z slices held in shared memory,
 *                              the next slice copied in by the bulk-copy
 *                              engine while the current one is updated; a
 *                              block marches through a chunk of slices.
 *                              Bitwise the staple kernel's result.  FP32
 *                              SU(3) state of a whole lattice (not a slab)
 *                              with nx = 32 or 64 only.  A wait on a copy
 *                              that runs out (glasma_set_staging_wait) is
 *                              reported as TIMEOUT by the next call that
 *                              returns host values;
 *   GLASMA_KERNEL_AUTO         the default, from GB300 timings: for FP64
 *                              state the plaquette kernel where a transverse
 *                              row fits one block (nx <= 320; its 24% fewer
 *                              FMAs win where the FP64 pipe bounds the
 *                              step), else the staple kernel; for FP32 the
 *                              staged staple kernel where it applies with
 *                              nx = 64 (SU(3), whole lattices), else the
 *                              staple kernel. */
enum { GLASMA_KERNEL_AUTO = 0, GLASMA_KERNEL_STAPLE = 1, GLASMA_KERNEL_PLAQUETTE = 2,
       GLASMA_KERNEL_PLAQUETTE_256 = 3, GLASMA_KERNEL_STAPLE_PAIRS = 4, GLASMA_KERNEL_STAPLE_STAGED = 5 };

/*
 * Choose the leapfrog step kernel of a context and, for the plaquette
 * kernel, the number of z slices each block marches through (zlen; 0 =
 * automatic, about eight blocks per resident block slot).  Results of the
 * two kernels agree to rounding (their sums run in different orders); the
 * choice never changes the state's layout, so it may change between steps.
 * Errors: INVALID_ARG (unknown kernel, zlen outside [0, nz], a plaquette
 * kernel asked for on a lattice whose transverse rows do not fit one
 * block, the paired kernel asked for on FP64 state, the staged kernel
 * asked for outside FP32 SU(3) whole lattices with nx = 32 or 64).
 */
GLASMA_API int glasma_set_step_kernel(glasma_ctx* c, int kernel, int zlen);

/*
 * Spin budget of one wait of the staged step kernel on its shared-memory
 * copies, in SM clock cycles (default 2^31, about a second; at most 2^40),
 * and stall (0 or 1, default 0).  stall = 1 makes the first block of every
 * staged launch also wait on a barrier that nothing completes, so that its
 * wait runs out and the launch reports TIMEOUT: it exists to test the
 * timeout path and has no other use.  After a wait runs out the block stops,
 * waits for its copies in flight and records the failure; the state after
 * that step is undefined.  Errors: INVALID_ARG.
 */
GLASMA_API int glasma_set_staging_wait(glasma_ctx* c, long long wait_cycles, int stall);

/*
 * Rest-frame analysis of sampled tables (Sec. 4: the event average of
 * T^{mu nu}, its diagonalisation to the local rest-frame energy density
 * eps_loc, Milne coordinates tau = sqrt(t^2 - z^2), eta_s, and the Gaussian
 * fit of rapidity profiles, Fig. 4).  Device arrays are FP64 and owned by
 * the caller; work runs on `stream` (cudaStream_t, NULL = legacy default)
 * without synchronising.
 *
 * glasma_rest_frame: tabs [n_events][n_points][4] rows (eps, p_L, p_T, S_L)
 *   as glasma_tmunu_device writes them (n_points = samples x nz, 32-byte
 *   aligned); out [n_points][8] = (<eps>, <p_L>, <p_T>, <S_L>, eps_loc,
 *   p_L,loc, v_z, valid) with <.> the mean over events (summed in event
 *   order).  eps_loc and -p_L,loc are the eigenvalues of T^mu_nu on the
 *   (t, z) block (metric diag(+1, -1)) whose eigenvectors are timelike and
 *   spacelike, v_z = u^z / u^t the flow velocity.  A point with S_L != 0
 *   and (eps + p_L)^2 <= 4 S_L^2 has no timelike eigenvector: its eps_loc,
 *   p_L,loc, v_z are NaN and valid is 0 (1 otherwise).
 *   Errors: INVALID_ARG, CUDA.
 * glasma_sample_grid: component comp of grid [n_t][nz][stride] (point
 *   (k, j) at t = t0 + k dts, z = z0 + j az), interpolated bilinearly at
 *   n_pts points given as (tau, eta_s) (coords 0; t = tau cosh eta_s,
 *   z = tau sinh eta_s, eta_s = artanh(z / t)) or as (t, z) (coords 1) in
 *   x[i], y[i]; out[i] is NaN outside the grid.  Errors: INVALID_ARG, CUDA.
 * glasma_fit_gaussian (host arrays, host computation): fits
 *   f = amp exp(-(x - mu)^2 / (2 sigma^2)) by weighted least squares of
 *   log f on a parabola (weights f^2) over the finite points with
 *   f > frac * max f.  Errors: INVALID_ARG (fewer than 3 points, no
 *   maximum).
 */
GLASMA_API int glasma_rest_frame(const double* tabs, int n_events, long long n_points, double* out, void* stream);
GLASMA_API int glasma_sample_grid(const double* grid, int n_t, int nz, int stride, int comp, double t0,
                                  double dts, double z0, double az, const double* x, const double* y,
                                  long long n_pts, int coords, double* out, void* stream);
GLASMA_API int glasma_fit_gaussian(const double* x, const double* f, int n, double frac, double* amp, double* mu,
                                   double* sigma);

/*
 * The stopping rule of the improved scheme's fixed-point iteration, as the
 * library applies it after every sweep (host computation, no GPU):
 * dmax[j] = max |E^(j+1) - E^(j)| and emax[j] = max |E^(j+1)| of sweeps
 * j = 0..k; *converged = 1 if the iteration stops after sweep k, else 0.
 * It stops when dmax[k] < tol; or when the contraction bound
 * dmax[k] c / (1 - c) is at most 16 unit roundoffs of emax[k], with c the
 * larger of dmax[k] / dmax[k-1] and dmax[k-1] / dmax[k-2] (k >= 2) and
 * c < 1/2; or when dmax[k] is within 64 unit roundoffs of emax[k] and at
 * least dmax[k-1] / 2; or when dmax[k] >= dmax[k-1] while dmax[k] is within
 * 1024 unit roundoffs of emax[k] (the precision's rounding floor).  precision:
 * GLASMA_FP32 or GLASMA_FP64 (the state's, which sets the unit roundoff).
 * Errors: INVALID_ARG (NULL pointers, k outside 0..4096, bad precision).
 */
GLASMA_API int glasma_implicit_converged(const double* dmax, const double* emax, int k, double tol, int precision,
                                         int* converged);

/*
 * The improved step (Sec. 3, the paragraph after Eq. gauss; Fig. wilson (b))
 * driven sweep by sweep from the host, the form a lattice split into z
 * slabs needs: the stopping rule takes the largest change of E over the
 * whole lattice, so each rank's sweep maxima are folded (max) across the
 * ranks before the test.  The sweeps need no halo messages (in a plane
 * containing z only the z links take the time slot of the iterate, and the
 * z link of the lower halo slice is evaluated on the slab from the step's
 * halo, with its owner's arithmetic); the step's halo exchange comes before
 * glasma_implicit_begin.  Any context of the improved scheme may use these
 * calls; glasma_step does the same for a whole lattice with every sweep
 * queued at once.
 * glasma_implicit_begin: the CPIC hop, U(t_{n-1}) on the first step, the
 *   first iterate U(t_{n+1}) = exp(i dt E(t_{n-1/2})) U(t_n) and the force
 *   of the time slots t_n and t_{n-1}.  Errors: INVALID_ARG (leapfrog
 *   context, a step already begun, slab windows not set), PARTICLE_EXIT,
 *   CUDA.
 * glasma_implicit_sweep: one sweep (E = E(t_{n-1/2}) + dt J + dt F, the
 *   next iterate), synchronising the stream; *dmax = max |E^(k+1) - E^(k)|
 *   and *emax = max |E^(k+1)| over the owned slices.  The caller folds them
 *   across ranks and applies glasma_implicit_converged to the folded
 *   sequence.  Errors: INVALID_ARG (no step begun, NULL pointers),
 *   NOT_CONVERGED (implicit_max_iter sweeps already done), CUDA.
 * glasma_implicit_end: commit the last sweep's iterate as U(t_{n+1}) and
 *   its E as E(t_{n+1/2}), move the charge windows of a hop step, advance
 *   the step counter (glasma_get_info reports the sweeps).  Errors:
 *   INVALID_ARG (no step begun, no sweep done).
 * Between _begin and _end the fields are mid-iteration: glasma_step, the
 *   observables, field and checkpoint transfers and slab messages return
 *   INVALID_ARG until _end.  A sweep that returns a non-finite maximum
 *   leaves the step open and its state undefined.
 */
GLASMA_API int glasma_implicit_begin(glasma_ctx* c);
GLASMA_API int glasma_implicit_sweep(glasma_ctx* c, double* dmax, double* emax);
GLASMA_API int glasma_implicit_end(glasma_ctx* c);

/*
 * Gradient of the mid-rapidity energy with respect to the initial MV colour
 * charges (SU(2), leapfrog, one colour sheet): the hand-written adjoint of
 * glasma_init_mv followed by n_steps glasma_step calls.  The observable is
 *   O = a_z sum_{iz : |iz a_z - z_c| < half_width} eps(iz)
 * with eps(iz) the energy density of glasma_tmunu at step n_steps (Sec. 4)
 * and z_c = nz a_z / 2.  rho_host: [2][3][ny][nx] charges as for
 * glasma_init_mv (NULL: drawn from p->seed).  The forward run keeps a
 * state every checkpoint_every steps; the reverse pass recomputes each
 * segment from its checkpoint (device memory: (ceil(n_steps / K) +
 * min(K, n_steps) + 2) states plus about 70 doubles per site, through
 * `alloc` as in glasma_init_mv).  Outputs: *value = O (may be NULL) and
 * grad_host[2][3][ny][nx] = dO/drho (NULL: forward only).  With
 * p->precision = GLASMA_FP32 the forward run and its checkpoints are FP32
 * and the reverse pass works in FP64 on those states (converted on the
 * device), i.e. it differentiates the FP32 trajectory; with GLASMA_FP64
 * everything is FP64.  Synchronises the stream.  Errors: INVALID_ARG (not
 * SU(2)/leapfrog, several colour sheets, bad sizes), PARTICLE_EXIT, OOM,
 * CUDA.
 */
GLASMA_API int glasma_adjoint_energy(const glasma_params* p, const double* rho_host, int n_steps,
                                     double half_width, int checkpoint_every, void* stream,
                                     const glasma_allocator* alloc, double* value, double* grad_host);

/*
 * Batched ensemble (the event averages of Sec. 2 and Sec. 4): several
 * independent leapfrog events, possibly of different nz, ny, nx, advanced
 * together.  Each event's result is bitwise the one glasma_step gives it
 * alone (the same per-link arithmetic).  Execution modes:
 *   GLASMA_BATCH_GRAPH (default): per time step, one kernel launch per
 *     geometry class (the events of equal nz, ny, nx together); the
 *     launches of one call are captured on a private stream into one CUDA
 *     graph, launched on the events' stream.  The call does not
 *     synchronise.
 *   GLASMA_BATCH_PERSISTENT: one cooperative launch per 64 steps, its
 *     blocks resident throughout and meeting at a grid barrier between
 *     steps.  Every barrier wait is bounded (glasma_batch_set_barrier); a
 *     wait that runs out makes the call return GLASMA_ERR_TIMEOUT, after
 *     which the events' states are undefined (restore them from a
 *     checkpoint).  The call synchronises the stream to read the barrier's
 *     status after each launch.
 *   GLASMA_BATCH_PER_EVENT: the single-event step kernel of every event and
 *     step captured into one graph (best for events that fill the GPU on
 *     their own).  The call does not synchronise.
 *
 * glasma_batch_create: ctxs[0..n-1], 1 <= n <= 64, distinct contexts that
 *   share nc, precision, dt, a_t, a_z, the device and the stream, all with
 *   the leapfrog scheme.  The batch borrows the contexts (the caller keeps
 *   ownership and must free the batch before any of them; 16 bytes of
 *   barrier state come from the first context's allocator); *out receives
 *   the handle.  Errors: INVALID_ARG, OOM, CUDA.
 * glasma_batch_step: advance every event by n_steps steps.  Before a step in
 *   which a charge of ANY event would leave its lattice, every event stops
 *   after the last complete step and GLASMA_ERR_PARTICLE_EXIT is returned
 *   (glasma_get_info gives each event's step_n).  Do not call it while the
 *   stream is being captured, nor step the batch's contexts from another
 *   thread meanwhile.  Errors: INVALID_ARG, PARTICLE_EXIT, TIMEOUT
 *   (persistent mode), CUDA.
 * glasma_batch_set_shape: the mode and block_sites, the transverse sites
 *   per block of the batched kernels (32, 64 or 128; a block is
 *   block_sites x 3 links; ignored by the per-event mode).
 *   Errors: INVALID_ARG.
 * glasma_batch_tune: time `steps` steps in the graph and persistent modes
 *   with 32, 64 and 128 sites per block and in the per-event mode, on the
 *   batch itself; keep the fastest for later glasma_batch_step calls and
 *   store it in *block_sites and *mode (either may be NULL).  The events'
 *   states are saved before and restored after each trial (temporary device
 *   copies of U, E and the charges, through each context's allocator), so
 *   the call leaves every event as it found it.  Synchronises the stream.
 *   Errors: INVALID_ARG, OOM, PARTICLE_EXIT (steps + 1 trial steps would
 *   move a charge off a lattice), TIMEOUT, CUDA.
 * glasma_batch_set_barrier: spin budget of one grid-barrier wait in SM clock
 *   cycles (default 2e9, about a second) and extra_arrivals (0..1024, default
 *   0), blocks that every barrier waits for in addition to the launched ones.
 *   extra_arrivals > 0 makes every wait run out: it exists to test the
 *   timeout path and has no other use.  Errors: INVALID_ARG.
 * glasma_batch_free: release the batch (not the contexts).  NULL is ignored.
 */
enum { GLASMA_BATCH_GRAPH = 0, GLASMA_BATCH_PERSISTENT = 1, GLASMA_BATCH_PER_EVENT = 2 };
typedef struct glasma_batch glasma_batch;
GLASMA_API int glasma_batch_create(glasma_ctx* const* ctxs, int n, glasma_batch** out);
GLASMA_API int glasma_batch_step(glasma_batch* b, int n_steps);
GLASMA_API int glasma_batch_set_shape(glasma_batch* b, int mode, int block_sites);
GLASMA_API int glasma_batch_tune(glasma_batch* b, int steps, int* block_sites, int* mode);
GLASMA_API int glasma_batch_set_barrier(glasma_batch* b, long long wait_cycles, int extra_arrivals);
GLASMA_API void glasma_batch_free(glasma_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* GLASMA_H */
