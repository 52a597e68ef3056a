/*
 * sdm.h -- C ABI of the GB300 Super-Droplet Method (SDM) coalescence library.
 *
 * The library advances the particle-based warm-rain representation of
 * PySDM v1 (arXiv:2103.17238) by its collision-coalescence dynamic: the SDM
 * Monte-Carlo algorithm of Shima et al. (2009) named in the paper's
 * Introduction.  The calls mirror the paper's statement of the problem (API in
 * brief): a Builder with n_sd super-droplets and a Box(dt, dv) environment,
 * the Coalescence dynamic with a kernel such as Golovin(b), the attributes
 * 'volume' and 'n' (multiplicity), Particulator.run(steps), and the
 * ParticlesVolumeSpectrum product 'dv/dlnr'.
 *
 * Conventions shared by every call
 *   - Every call returns an sdm_status; out-parameters are written only on
 *     SDM_OK.  sdm_last_error() gives a message for the last failure.
 *   - Units are SI: volume in m^3, radius in m, dt in s, dv in m^3,
 *     golovin_b in s^-1.
 *   - The caller keeps ownership of every array it passes; the library copies
 *     what it needs before the call returns (or, for device arrays, orders its
 *     copies on the context's stream before any later work).
 *   - "on_device" flags say whether a pointer is CUDA device memory (1) or
 *     host memory (0).  Host buffers may be pageable or pinned.
 *   - All device work is ordered on the CUDA stream given to sdm_create.
 *     sdm_coalescence_step only enqueues work and returns; calls that hand
 *     results to host memory synchronise that stream first.
 *   - A CUDA error leaves the context unusable: the failing call returns
 *     SDM_ECUDA and every later call on that context SDM_ESTATE.
 *   - Contexts are not thread-safe: one thread at a time per context.
 */
#ifndef SDM_H
#define SDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SDM_OK = 0,
    SDM_EINVAL = 1,   /* an argument or attribute value is out of range */
    SDM_ENOMEM = 2,   /* device or host allocation failed */
    SDM_ECUDA = 3,    /* a CUDA call failed (context now unusable) */
    SDM_ESTATE = 4,   /* call not valid in the context's state */
    SDM_ETIMEOUT = 5, /* a bounded device-side wait gave up */
    SDM_EBUDGET = 6   /* request exceeds the configured memory budget */
} sdm_status;

/* Collision kernels K(j, k) in m^3 s^-1 (paper: Usage examples, Box
 * environment examples -- the Golovin additive kernel, with its analytic
 * solution, and Berry's geometric sweep-out kernel). */
typedef enum {
    SDM_KERNEL_GOLOVIN = 0,   /* K = b (v_j + v_k) */
    SDM_KERNEL_GEOMETRIC = 1, /* K = pi (r_j + r_k)^2 |v_t(r_j) - v_t(r_k)|, E = 1,
                                 v_t from Rogers & Yau (1989), r = (3 v / 4 pi)^(1/3) */
    SDM_KERNEL_LONG = 2       /* the geometric K times Long's (1974) collision
                                 efficiency: with R = max(r_j, r_k), r = min(r_j, r_k),
                                 E = max(4.5e8 R^2 (1 - 3e-6 / r), 1e-3) for R <= 50e-6 m,
                                 E = 1 above (SI form of the published cgs constants) */
} sdm_kernel;

/* Precision of the kernel K and probability p.  Multiplicities are always
 * exact int64 and volumes binary64 in both modes. */
typedef enum {
    SDM_PREC_FP64 = 0, /* K and p in binary64 */
    SDM_PREC_KFP32 = 1 /* K and p in binary32, widened to binary64 for gamma */
} sdm_precision;

/* Device allocator hooks.  alloc returns device memory of at least `bytes`
 * usable on `stream` (or NULL on failure); free releases it.  Both NULL: the
 * library uses cudaMallocAsync / cudaFreeAsync on the context's stream. */
typedef void *(*sdm_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*sdm_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct sdm_config {
    int32_t kernel;    /* sdm_kernel */
    int32_t precision; /* sdm_precision */
    double golovin_b;  /* s^-1 (Golovin only), >= 0 */
    double dt;         /* timestep, s, > 0 */
    double dv;         /* volume of one cell, m^3, > 0 */
    /* Rogers-Yau terminal velocity: k1 r^2 for r < r1, k2 r for r < r2,
     * k3 sqrt(r) otherwise.  sdm_config_default sets k1 = 1.19e8 m^-1 s^-1,
     * k2 = 8e3 s^-1, k3 = 201 m^0.5 s^-1, r1 = 40e-6 m, r2 = 600e-6 m. */
    double ry_k1, ry_k2, ry_k3, ry_r1, ry_r2;
    int32_t n_cells;   /* cells of this run, >= 1 */
    int32_t cell_base; /* index of this run's cell 0 in a larger grid split into pieces (one
                          per context): the random streams use cell_base + c for cell c, and
                          sedimentation counts levels from level cell_base / nx (the pieces of
                          one grid then step exactly as the whole grid would).  0 for a whole
                          grid; cell_base + n_cells < 2^31 */
    uint64_t seed;     /* Philox4x32-10 key of this run's random streams */
    int64_t step0;     /* index of the first step (resume: steps already done) */
    sdm_alloc_fn alloc;
    sdm_free_fn free;
    void *alloc_user;
} sdm_config;

/* Fills *cfg with the paper's worked example: Golovin b = 1500 s^-1,
 * dt = 1 s, dv = 1e6 m^3, one cell, FP64, seed 0, step0 0, the Rogers-Yau
 * defaults, default allocator. */
void sdm_config_default(sdm_config *cfg);

typedef struct sdm_ctx sdm_ctx;     /* one run: its super-droplets and cells */
typedef struct sdm_batch sdm_batch; /* several runs stepped by fused launches */

/* Creates a run (the Builder/Particulator of the paper's API in brief) with
 * room for capacity_sd super-droplets.  cuda_stream is a cudaStream_t (NULL:
 * the legacy default stream).  The context owns its device memory.
 * Errors: SDM_EINVAL (bad config or capacity < 1), SDM_ENOMEM, SDM_ECUDA. */
sdm_status sdm_create(const sdm_config *cfg, int64_t capacity_sd, void *cuda_stream, sdm_ctx **out);

/* Sets the super-droplet attributes (the paper's attributes 'n' and
 * 'volume', plus the cell of each SD).  SD i of the arrays is the SD with
 * id i; within a cell, SDs keep their order of increasing id (the SD's rank,
 * which addresses its random sort key).
 *   xi[n_sd]      int64 multiplicity, >= 0 (0 marks a dead SD)
 *   volume[n_sd]  binary64 volume in m^3, finite, in [1e-30, 1e30]
 *   cell_id[n_sd] int32 cell in [0, n_cells), or -1: outside the domain (an
 *                 SD that has fallen through its bottom; kept, never stepped,
 *                 not counted by sdm_spectrum)
 * n_sd in [1, capacity_sd].  Replaces any earlier state, including positions
 * (sdm_set_positions); the step counter is kept.  Errors: SDM_EINVAL (names
 * the first offending SD), SDM_ECUDA. */
sdm_status sdm_set_attributes(sdm_ctx *ctx, int64_t n_sd, const int64_t *xi, const double *volume,
                              const int32_t *cell_id, int on_device);

/* Enqueues n_steps >= 0 coalescence steps on the context's stream (the
 * paper's Particulator.run(steps) with Coalescence as the only dynamic).
 * Step s, per cell c with n_c live SDs (xi > 0):
 *   1. key_i = Philox4x32-10(key = seed, ctr = (rank_i >> 1, c, s_lo,
 *      s_hi | 0 << 31)), words (0,1) for even rank, (2,3) for odd; the live
 *      SDs are ordered by (key, rank);
 *   2. neighbours form floor(n_c / 2) pairs l, (j, k) with xi_j >= xi_k
 *      (ties: j is the earlier of the two);
 *   3. p = K(j,k) xi_j dt/dv [n_c (n_c - 1) / 2] / floor(n_c / 2);
 *      u = 53-bit uniform from ctr = (l >> 1, c, s_lo, s_hi | 1 << 31);
 *      gamma = min(ceil(p - u), floor(xi_j / xi_k));
 *   4. gamma > 0: xi_j -= gamma xi_k, v_k += gamma v_j; if that leaves
 *      xi_j = 0 the k SD is split: xi_j = floor(xi_k / 2),
 *      xi_k -= floor(xi_k / 2), v_j = v_k = v_k + gamma v_j.
 * Returns without waiting for the GPU.  Errors: SDM_ESTATE (no attributes
 * set), SDM_EINVAL (n_steps < 0), SDM_ECUDA. */
sdm_status sdm_coalescence_step(sdm_ctx *ctx, int32_t n_steps);

/* The ParticlesVolumeSpectrum product dv/dlnr of the paper's API in brief:
 * for radius bins [r_edges[b], r_edges[b+1]) (r = (3 v / 4 pi)^(1/3)), the
 * volume sum(xi v) of live SDs per m^3 of air per unit ln r.
 *   per_cell = 0: out[n_edges - 1], all cells, divided by dv * n_cells;
 *   per_cell = 1: out[n_cells * (n_edges - 1)], cell-major, divided by dv.
 * r_edges: host array, n_edges >= 2, strictly increasing, > 0.  out: caller
 * buffer, host (out_on_device = 0; the call synchronises the stream) or
 * device (ordered on the stream).  Errors: SDM_EINVAL, SDM_ESTATE, SDM_ECUDA. */
sdm_status sdm_spectrum(sdm_ctx *ctx, const double *r_edges, int32_t n_edges, int per_cell, double *out,
                        int out_on_device);

/* Copies the current multiplicities and volumes of all n_sd SDs, in SD-id
 * order (dead SDs included, with xi = 0), into caller buffers xi[n_sd] and
 * volume[n_sd] (either may be NULL).  Host buffers: synchronises the stream.
 * With sdm_set_attributes and sdm_config.step0 this checkpoints and resumes a
 * run bit for bit.  Errors: SDM_ESTATE, SDM_ECUDA. */
sdm_status sdm_get_attributes(sdm_ctx *ctx, int64_t *xi, double *volume, int on_device);

typedef struct sdm_info {
    int64_t n_sd;          /* SDs set by sdm_set_attributes */
    int64_t capacity_sd;   /* room reserved at sdm_create */
    int64_t step;          /* index of the next step */
    int64_t device_bytes;  /* device memory held by the context */
    int32_t n_cells;
    int32_t largest_cell;  /* SDs in the most populated cell */
} sdm_info;

sdm_status sdm_get_info(const sdm_ctx *ctx, sdm_info *out);

/* Device bytes a context with this capacity and cell count holds (the
 * serving loop admits runs by this footprint). */
int64_t sdm_footprint_bytes(int64_t capacity_sd, int32_t n_cells, int32_t largest_cell);

/* Releases the context and its device memory (after the stream's pending
 * work).  NULL is a no-op. */
sdm_status sdm_destroy(sdm_ctx *ctx);

/* Message for the last failed call on ctx, or of the calling thread when
 * ctx is NULL.  Never NULL; valid until the next call on the same object. */
const char *sdm_last_error(const sdm_ctx *ctx);

/* ---- batching: many independent runs (ensemble members, served requests)
 * advanced by fused launches.  A batch refers to its contexts, which must
 * stay alive and keep their attributes while the batch exists; every
 * context keeps its own seed, step counter, kernel, dt and dv, so a batched
 * step gives bit-for-bit the result of stepping each context alone. */

/* use_graph != 0: sdm_batch_step replays a captured CUDA graph of
 * graph_steps launches where it can (graph_steps <= 0: 16). */
sdm_status sdm_batch_create(sdm_ctx *const *ctxs, int32_t n_ctx, void *cuda_stream, int32_t use_graph,
                            int32_t graph_steps, sdm_batch **out);

/* Enqueues n_steps steps of every context in the batch on the batch's
 * stream; the contexts' streams are not used.  Errors: SDM_EINVAL,
 * SDM_ESTATE (also when a context's layout changed since the batch was
 * created: sdm_set_attributes or sdm_sedimentation_step), SDM_ECUDA. */
sdm_status sdm_batch_step(sdm_batch *batch, int32_t n_steps);

sdm_status sdm_batch_destroy(sdm_batch *batch);

const char *sdm_batch_last_error(const sdm_batch *batch);

/* ---- sedimentation (a next step of the method: the paper's "particle
 * displacement" dynamic and the sedimenting drizzle of its 2-D example; the
 * paper prints no formulae).  Cells are levels x columns: cell c lies in
 * level iz = c / nx and column ix = c mod nx, level iz spans heights
 * [iz dz, (iz + 1) dz) above the domain bottom.  Each SD's position is kept
 * as its height zeta above its cell's bottom (binary64).
 *
 * A context with cell_base > 0 is a piece of a larger grid: its levels are
 * levels cell_base / nx and up of that grid (nx must divide cell_base), z
 * is measured from the grid's bottom, and an SD falling below the piece's
 * lowest level continues into the grid's levels below: it leaves this
 * context (sdm_get_heights gives its new cell and height) unless it falls
 * through the grid's bottom (precipitated).
 *
 * One sedimentation step, for every live SD: d = v_t(r) dt in binary32 (the
 * Rogers-Yau speed of the binary32 radius of the binary32 image of the
 * volume, the twin used by SDM_PREC_KFP32, times (float)dt), widened exactly
 * to binary64; zeta -= d; while zeta < 0 the SD enters the level below
 * (zeta += dz).  An SD that goes below level 0 leaves the domain (cell -1)
 * and its xi v is precipitated; if zeta + dz rounds up to dz the SD stays in
 * the level above at zeta = 0.  Dead SDs (xi = 0) leave the domain too.
 * Columns never change.  Afterwards cells hold their SDs in increasing id
 * again, so the next coalescence step sees the new cell membership. */

/* Sets the positions: z[n_sd] (SD-id order, host or device) the height of
 * each SD above the domain bottom, m.  Needs attributes; nx >= 1 divides
 * n_cells; dz > 0 finite.  Each SD's zeta = z - (c / nx) dz (binary64) must
 * lie in [0, dz); SDs outside the domain ignore z.  Errors: SDM_EINVAL (names
 * the first offending SD), SDM_ESTATE (no attributes), SDM_ENOMEM,
 * SDM_ECUDA.  Synchronises the context's stream. */
sdm_status sdm_set_positions(sdm_ctx *ctx, const double *z, int32_t nx, double dz, int on_device);

/* One sedimentation step (asynchronous up to one host read of the new cell
 * offsets; stream-ordered with the coalescence steps).  precipitated
 * (nullable host pointer) receives sum(xi v), m^3, of the SDs that fell
 * through the bottom in this step.  A batch (sdm_batch_create) holding the
 * context must be created again afterwards: its next step fails with
 * SDM_ESTATE.  Errors: SDM_ESTATE (no positions), SDM_ENOMEM, SDM_ECUDA. */
sdm_status sdm_sedimentation_step(sdm_ctx *ctx, double *precipitated);

/* The same as sdm_set_positions, with zeta[n_sd] (SD-id order, host or
 * device) the height of each SD above its cell's bottom, in [0, dz), taken
 * as it is (no subtraction, so heights read by sdm_get_heights come back bit
 * for bit: this is how a piece of a grid receives SDs from the piece above).
 * Errors as sdm_set_positions. */
sdm_status sdm_set_heights(sdm_ctx *ctx, const double *zeta, int32_t nx, double dz, int on_device);

/* Heights and cells for a grid split into pieces (one context per piece of
 * whole levels, sdm_config.cell_base its first cell): per SD in SD-id order,
 * cell[n_sd] (nullable) its cell in the whole grid, cell_base + c, for SDs
 * inside this piece; for an SD that left this piece through its bottom into
 * a level of the grid below it in the last sedimentation step, its new cell
 * there (cell < cell_base); else -1 (fallen through the grid's bottom, dead
 * or outside).  zeta[n_sd] (nullable) the SD's height above the bottom of
 * that cell (0 for -1).  Needs positions.  Host arrays: synchronises;
 * device arrays: stream-ordered.  Errors: SDM_ESTATE, SDM_ENOMEM, SDM_ECUDA. */
sdm_status sdm_get_heights(sdm_ctx *ctx, double *zeta, int32_t *cell, int on_device);

/* Positions in SD-id order: z[n_sd] (nullable; needs positions) the height
 * above the domain bottom, (c / nx) dz + zeta in binary64, 0 for SDs outside
 * the domain; cell[n_sd] (nullable) the SD's cell, -1 outside.  Host
 * arrays: synchronises; device arrays: stream-ordered. */
sdm_status sdm_get_positions(sdm_ctx *ctx, double *z, int32_t *cell, int on_device);

/* ---- condensation (a next step of the method: the paper lists condensation
 * among the dynamics of its framework and prints no formulae).  The large-
 * drop limit of the diffusional growth law, r dr/dt = s G (Rogers & Yau
 * 1989, ch. 7, with the curvature and solute terms dropped): s = S - 1 is
 * the cell's supersaturation and G = 1 / (F_k + F_d) its growth coefficient
 * (m^2 s^-1; F_k, F_d the heat-conduction and vapour-diffusion terms of the
 * ambient temperature and pressure), both held over the step, so r^2 grows
 * by exactly c = 2 G s dt.  An evaporating SD stops at the floor radius
 * r_min, or at its own radius when that is already below r_min.
 *
 * Per live SD inside the domain, with cf = (float)(((2 G) s) dt) of its
 * cell (binary64, rounded once): r = the binary32 radius of (float)v (the
 * KFP32 twin), x = r r, x' = max(x + cf, min(x, (float)(r_min r_min))),
 * d = cf (or that floor - x when the floor acts), a = sqrt(x'), b = sqrt(x),
 * dV = k43 ((d ((x' + a b) + x)) / (a + b)) with k43 = (float)(4 pi / 3),
 * all binary32; v += (double)dV in binary64.  Multiplicities, dead SDs and
 * SDs outside the domain do not change.
 *   G[n_cells], s[n_cells]  host arrays: G >= 0 finite, s in [-1, 1],
 *                           |2 G s dt| <= 1e-6 m^2 (else SDM_EINVAL)
 *   r_min                   floor radius, m, in [1e-9, 1e-3]
 *   condensed               nullable: receives sum(xi dV) of each cell, m^3
 *                           (n_cells values; summed in a fixed order, not
 *                           the oracle's), host (condensed_on_device = 0: the
 *                           call synchronises) or device (stream-ordered)
 * Enqueued on the context's stream.  Errors: SDM_EINVAL, SDM_ESTATE (no
 * attributes), SDM_ENOMEM, SDM_ECUDA. */
sdm_status sdm_condensation_step(sdm_ctx *ctx, const double *G, const double *s, double r_min, double *condensed,
                                 int condensed_on_device);

/* ---- launch tuning.  Which cells are sorted in shared memory (the rest take
 * the multi-pass global path), which run one warp per cell, and how many
 * warps share a block.  Results never depend on it: every setting gives the
 * same state bit for bit.  Process-wide; applies to contexts and batches
 * whose launch plans are built after the call (a context builds its plan at
 * its first sdm_coalescence_step after sdm_set_attributes, a batch at
 * sdm_batch_create).  paper_2103_17238_gb300/autotune.py times candidates
 * and sets the fastest. */
typedef struct sdm_tuning {
    int32_t smem_max_sd;     /* largest cell sorted in shared memory: 512, 1024, 2048 or 4096 (default) */
    int32_t warp_cell_max;   /* largest cell run by one warp: 0, 64, 128, 256 or 512 (default), <= smem_max_sd */
    int32_t warps_per_block; /* warps per block of the warp-per-cell kernel: 1, 2 (default) or 4 */
    int32_t fuse_steps;      /* 2..1024 (default SDM_FUSE_STEPS_DEFAULT): the warp-per-cell kernel
                              * keeps each cell in shared memory for up to fuse_steps consecutive
                              * steps of one sdm_batch_step / sdm_coalescence_step call (the same
                              * state, bit for bit: cells are independent, so a cell may take its
                              * steps apart from the others); cells of other sizes still take one
                              * launch per step, and a one-step call is one launch either way.
                              * 0 or 1: one launch per step for every cell.  A graph captures the
                              * same launches. */
    int32_t mid_max_sd;      /* largest cell above smem_max_sd stepped by one thread-block cluster
                              * (1, 2 or 4 CTAs of up to 16384 SDs each, the whole step in shared
                              * and distributed shared memory); larger cells take the multi-pass
                              * global path.  0: no cluster path.  Default SDM_MID_MAX_SD_DEFAULT. */
} sdm_tuning;

#define SDM_FUSE_STEPS_DEFAULT 64
#define SDM_MID_MAX_SD_DEFAULT 16384

/* NULL restores the defaults.  Errors: SDM_EINVAL. */
sdm_status sdm_set_tuning(const sdm_tuning *tuning);
sdm_status sdm_get_tuning(sdm_tuning *out);

/* ---- allocation-free step of one cell.  This call has no counterpart in
 * the paper; it exists for callers that cannot allocate device memory while
 * they run: a host model that reserves all of its GPU memory up front in its
 * own pool and forbids later allocation, a Fortran/OpenACC code whose runtime
 * owns every device buffer, a latency-bound loop that cannot afford an
 * allocator call.  It allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.  Its scratch is one fixed array of device
 * memory inside the library (about 8.6 MiB for SDM_NOALLOC_MAX_SD SDs), which
 * every GPU that loads the library holds until the process exits.
 *
 * One coalescence step (the same step as sdm_coalescence_step) of ONE cell
 * whose SDs the caller holds, in place:
 *   cfg       kernel, precision, golovin_b, dt, dv, Rogers-Yau coefficients
 *             and seed as for sdm_create; n_cells must be 1; step0 and the
 *             allocator hooks are ignored
 *   step      index of this step (>= 0); the random streams use cell index 0
 *   xi[n_sd]  int64 multiplicities, device (or managed) memory of the
 *             current device, 16-byte aligned, SDs in rank order (the order
 *             that addresses their random keys)
 *   volume[n_sd]  binary64 volumes, the same kind of memory, 16-byte aligned
 *             (both pointers are checked with cudaPointerGetAttributes, which
 *             allocates nothing; a host pointer or another device's memory is
 *             refused with SDM_EINVAL)
 *   n_sd      even, in [2, SDM_NOALLOC_MAX_SD]; pad an odd cell with one dead
 *             SD (xi = 0)
 *   cuda_stream   stream the work is ordered on (NULL: legacy default stream)
 * Values are not validated (they must satisfy sdm_set_attributes' ranges);
 * sizes beyond the maximum are rejected with SDM_EINVAL.  The result equals
 * sdm_coalescence_step on a context with one cell, the same config and
 * step0 = step, bit for bit.  Returns after enqueueing the work.
 *
 * Set-up: the first call on each device (with that device current) looks up
 * the scratch array's device address and configures the kernels; make that
 * first call before any stream capture.  Every call shares the one array and
 * leaves its contents behind, so calls whose work overlaps on the GPU (two
 * streams, two host threads, two devices' calls aimed at one device) race:
 * order them on one stream.  Errors: SDM_EINVAL, SDM_ECUDA (also when a
 * CUDA error from earlier work is pending on the calling thread: it is
 * reported, not cleared, and nothing is launched; message from
 * sdm_last_error(NULL)). */
#define SDM_NOALLOC_MAX_SD 1048576

sdm_status sdm_cell_step_noalloc(const sdm_config *cfg, int64_t step, int64_t *xi, double *volume, int64_t n_sd,
                                 void *cuda_stream);

/* ---- diagnostics.  Not a product of the paper: the sums its coalescence
 * must keep.  Shima's update (the fourth part of the step) moves volume
 * between the two SDs of a pair and never adds multiplicity, so the total
 * water volume sum(xi v) is conserved (up to binary64 rounding) and the
 * total multiplicity sum(xi) never increases. */
typedef struct sdm_diag {
    int64_t live_sd;    /* SDs inside the domain (cell >= 0) with xi > 0 */
    uint64_t sum_xi_lo; /* sum of their xi, exact as a 128-bit integer: low 64 bits */
    uint64_t sum_xi_hi; /*   and high 64 bits */
    double sum_xi_v;    /* sum of their xi v, m^3, in binary64: each product added with one
                           rounding, in a fixed order, so repeated calls give the same bits */
} sdm_diag;

/* The sums over the context's current state, computed on its stream; the
 * call waits for them.  Errors: SDM_EINVAL (NULL out), SDM_ESTATE (no
 * attributes yet, or an unusable context), SDM_ENOMEM, SDM_ECUDA. */
sdm_status sdm_diagnostics(sdm_ctx *ctx, sdm_diag *out);

/* Self-test of failure detection on the device, without a fault.  Every
 * device-side wait of the step (for a bulk copy to arrive) is bounded: a
 * wait that gives up makes the kernel record it in the run's status word and
 * return, and the host reports SDM_ETIMEOUT.  This call runs that path on its
 * own: one block on cuda_stream (NULL: the legacy default stream) waits on a
 * barrier that nothing completes and gives up after max_polls polls (1 ..
 * 2^24).  It returns SDM_ETIMEOUT when the wait gave up as designed (the
 * expected result; the device stays usable), SDM_ESTATE if the barrier
 * completed, SDM_EINVAL for max_polls out of range, SDM_ENOMEM or SDM_ECUDA.
 * Messages from sdm_last_error(NULL). */
sdm_status sdm_selftest_bounded_wait(void *cuda_stream, int64_t max_polls);

#ifdef __cplusplus
}
#endif

#endif /* SDM_H */
