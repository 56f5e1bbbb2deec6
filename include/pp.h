/*
 * pp.h -- C ABI of the GB300 (sm_103a) particle-particle electron-bunch engine.
 *
 * The engine integrates the non-relativistic motion of N macro-electrons of
 * weight w (charge q_e w, mass m_e w, q_e = -e) in open vacuum under their
 * mutual Coulomb repulsion, following arXiv 2502.10640 Sec. 2.1:
 *   - pair force, Eq. A, with r_ij = r_i - r_j;
 *   - field at particle i from all j != i, Eq. B / Eq. E;
 *   - acceleration a_i = (q_e/m_e) E_i, Eq. D / Eq. F (w cancels);
 *   - Velocity Verlet, Eq. G (drift) and Eq. H (kick).
 * An optional Plummer softening eps replaces |r|^2 by |r|^2 + eps^2 (eps = 0
 * is Eq. A exactly).  A pair whose softened squared distance is zero adds
 * nothing.  Pair arithmetic is FP32 on staged positions (re-centred and
 * scaled by a power of two), accumulated per particle in FP64 (or in a
 * compensated FP32 pair); positions, velocities and accelerations are FP64.
 *
 * Units are SI throughout: positions m, velocities m/s, accelerations m/s^2,
 * fields V/m, energies J, momenta kg m/s, times s.
 *
 * Conventions for every call:
 *   - Every call returns a pp_status.  On PP_ERR_ARG, PP_ERR_NOMEM,
 *     PP_ERR_STATE and PP_ERR_TIMEOUT the context stays valid.  After
 *     PP_ERR_CUDA the context must be destroyed.
 *   - pp_last_error() gives a message for the last non-OK status returned
 *     on the calling thread.
 *   - Array arguments are [N][3] row-major doubles (x, y, z of particle i
 *     at 3i, 3i+1, 3i+2).  The on_device argument says where they live
 *     (enum pp_mem): PP_MEM_HOST (0), host memory, pageable or page-locked,
 *     moved by the copy engine through library scratch; PP_MEM_DEVICE (1),
 *     device memory of the context's GPU, read or written in order on the
 *     context's stream; PP_MEM_HOST_MAPPED (2), page-locked host memory that
 *     CUDA maps into the device address space (cudaHostAlloc, cudaMallocHost,
 *     cudaHostRegister, pinned PyTorch tensors), read or written directly by
 *     the library's kernels over the CPU-GPU link with no staging copy.  For
 *     PP_MEM_HOST_MAPPED the whole [N][3] array must lie in one such
 *     allocation; the library checks this on the host before any kernel
 *     touches the buffer and returns PP_ERR_ARG otherwise (pageable memory
 *     included).  The batch calls accept all three kinds and move mapped
 *     memory like PP_MEM_HOST.  Any other value: PP_ERR_ARG.  Inputs are
 *     copied; the caller keeps ownership of every buffer it passes.
 *   - The library owns all device memory it allocates; pp_destroy frees it.
 *   - Calls on one context must not run concurrently from several threads.
 *   - Calls return after the work they enqueue has finished (the stream is
 *     synchronised), so a status reflects device-side errors as well.
 *   - Host-side phases are marked with NVTX ranges named after the call.
 */
#ifndef PP_GB300_H
#define PP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pp_ctx pp_ctx;

/* Where a caller's array lives (the on_device argument of the calls below). */
typedef enum {
    PP_MEM_HOST = 0,         /* host memory, through the copy engine */
    PP_MEM_DEVICE = 1,       /* device memory of the context's GPU */
    PP_MEM_HOST_MAPPED = 2   /* mapped page-locked host memory, accessed by the kernels */
} pp_mem;

typedef enum {
    PP_OK = 0,
    PP_ERR_ARG = -1,      /* invalid argument (size, pointer, non-finite value, option) */
    PP_ERR_NOMEM = -2,    /* device allocation failed or a memory budget is exhausted    */
    PP_ERR_CUDA = -3,     /* CUDA runtime error; destroy the context                      */
    PP_ERR_TIMEOUT = -4,  /* a bounded device-side wait gave up; results of the call void */
    PP_ERR_STATE = -5     /* call out of order (e.g. step before particles are loaded)    */
} pp_status;

/* Force accumulation modes (option PP_OPT_ACC). */
typedef enum {
    PP_ACC_FP64FOLD = 0,  /* FP32 pair math, FP32 tile partials folded into FP64 (default)  */
    PP_ACC_KAHAN = 1,     /* FP32 pair math, tile partials folded into a compensated FP32 pair */
    PP_ACC_FP64_FULL = 2  /* FP64 pair math and accumulation (comparison path, slow)        */
} pp_acc;

/* How staged source positions carry precision into the FP32 pair math
 * (option PP_OPT_POSITIONS).  SINGLE rounds each staged coordinate to one
 * float, so a separation d carries an absolute error of about 2^-24 |r|,
 * i.e. a relative error 2^-24 |r|/|d| that grows for close pairs: the field
 * error of a random bunch is dominated by its few closest pairs (balls of
 * 4e4 or 2^20 particles with nm softening exceed 1e-5 in relative L2).
 * SPLIT stages hi + lo floats (about 48 bits) and forms d = (hi_i - hi_j) +
 * (lo_i - lo_j), exact in its hi part for close pairs, at six more FP32
 * operations per pair (about 30 % slower).
 * GUARDED stages hi/lo but runs the pair loop on the hi parts only, keeping
 * per target and source tile the largest reciprocal softened separation
 * rsqrt(s) (one three-input maximum per two pairs, off the FP32 pipe); a tile
 * holding a source with s < (|p_i| / 256)^2 (p_i: the target's staged position) is
 * summed again for that target with hi/lo separations, and the tile holding
 * the target block itself always is.  From N = 98304 on, each
 * force pass first sorts the staged sources along a Morton curve of their hi
 * positions and replaces the per-pair test by one test per target and tile
 * against the tile's bounding box: a warp sums with hi/lo separations every
 * tile whose box comes closer than |p_i| / 256 to one of its targets (about 60
 * more short launches per pass; the order depends on the positions alone, so
 * results stay bitwise reproducible).  Pairs left to the hi parts then carry a
 * relative error below about 5e-5 each, and the close pairs that dominate the
 * single-staging error get split precision, at nearly single-staging speed.
 * All three work with every FP32 pair path (FP64 fold, compensated fold,
 * per-particle weights); the resident small-N kernel runs SINGLE and SPLIT.
 * AUTO, the default, decides whenever the library picks a staging frame
 * (pp_load_particles, pp_set_weights on a loaded context, pp_set_state
 * without a frame): it computes the fields with hi/lo staging and takes the
 * first of SINGLE, SPLIT (only where the resident small-N kernel would run
 * it), GUARDED, SPLIT whose fields differ from those by at most 5e-6 in
 * relative L2 (half the 1e-5 field tolerance).  That costs two or three
 * extra force passes at those calls only; steps run at the speed of the
 * staging chosen.  pp_get_option(PP_OPT_POSITIONS) reports the staging in
 * force, PP_OPT_POSITIONS_AUTO whether AUTO is on, pp_staging_check the
 * measured differences.  With PP_ACC_FP64_FULL sources are FP64 and the
 * setting has no effect. */
typedef enum {
    PP_POS_SINGLE = 0,
    PP_POS_SPLIT = 1,
    PP_POS_AUTO = 2,      /* default */
    PP_POS_GUARDED = 3
} pp_positions;

/* Option keys for pp_set_option. */
enum {
    PP_OPT_ACC = 1,            /* value: a pp_acc                                              */
    PP_OPT_STREAM = 2,         /* value: cudaStream_t cast to int64 (0 = the context's own)   */
    PP_OPT_SPLIT = 3,          /* value: j-split count S >= 1, or 0 for automatic              */
    PP_OPT_GRAPH_BLOCK = 4,    /* value: steps per captured CUDA graph (0 = plain launches)   */
    PP_OPT_TIMEOUT_NS = 5,     /* value: limit of each device-side wait in ns (default 1e9, or
                                  the environment variable PP_TIMEOUT_NS at creation)        */
    PP_OPT_VARIANT = 6,        /* value: force-kernel variant index (-1 = automatic)          */
    PP_OPT_POSITIONS = 7,      /* value: a pp_positions (FP32 pair paths only)                 */
    PP_OPT_RESIDENT = 8,       /* value: a pp_resident (small-N stepping)                      */
    PP_OPT_RESIDENT_ACTIVE = 9,/* pp_get_option only: 1 if pp_step now runs the resident kernel */
    PP_OPT_POSITIONS_AUTO = 10,/* pp_get_option only: 1 if PP_POS_AUTO decides the staging     */
    PP_OPT_LAUNCHES_PER_PASS = 11,/* pp_get_option only: kernel launches of one per-launch force
                                  pass or step (1, or 1 + the spatial sort's with the tile-box
                                  guard of PP_POS_GUARDED)                                   */
    PP_OPT_TEST_SKIP_COPY = 99 /* value: 1 = the next force launch withholds one tile copy (the
                                  resident kernel: CTA 0's first barrier arrival), so its bounded
                                  waits expire and the call returns PP_ERR_TIMEOUT (tests the
                                  timeout path; no fault, no hang) */
};

/* Resident small-N stepping (PP_OPT_RESIDENT).  The resident kernel runs all
 * steps of a pp_step call in one cooperative launch: every CTA holds the
 * whole staged source array in shared memory, computes the Eq. B sums of its
 * targets (sources split over several threads per target, FP32 partials of at
 * most 512 sources, all partial sums compensated FP32 (TwoSum) in a fixed
 * order, FP64 from each item's final sum on) and the Eq. G/H push, then meets
 * the other CTAs at a grid-wide barrier, after which the next step's staged
 * sources arrive by 1D bulk copies into shared memory (bounded waits:
 * PP_ERR_TIMEOUT on expiry).  It floors
 * s = |d|^2 + eps^2 at 1e-24 in staged units (L0^2), so the self pair adds
 * exactly 0 without a test per pair; for separations the FP32 staging
 * resolves this changes s by less than one FP32 rounding.  Applicable with
 * the FP32 pair paths (PP_ACC_FP64FOLD or PP_ACC_KAHAN, which here fold the
 * same way) and a packed-pair variant (the default, or a PP_OPT_VARIANT
 * override with interleaved staging): with single staging (equal or
 * per-particle weights) for N <= 12288, with hi/lo staging (FP64 fold and
 * equal weights; both parts in shared memory) for N <= 6144.
 * PP_OPT_VARIANT otherwise still chooses the kernel of force passes and of
 * per-launch steps (set PP_RESIDENT_OFF to step with it).
 * Results differ from the per-launch kernels' at the FP32 rounding level
 * (another summation order) and are bitwise reproducible on a given device. */
typedef enum {
    PP_RESIDENT_OFF = 0,   /* always the per-launch kernels */
    PP_RESIDENT_AUTO = 1,  /* default: resident wherever applicable (measured faster than
                              the per-launch kernels at every N up to 12288 on GB300) */
    PP_RESIDENT_ON = 2     /* resident wherever applicable */
} pp_resident;

/*
 * Create a context for N macro-electrons of common weight w (Sec. 2.1 assumes
 * one weight for all macro-particles), time step dt > 0 and softening
 * eps >= 0 (metres).  Allocates the state and staging buffers on the current
 * CUDA device; force passes allocate their workspaces on first use (the j-split
 * partial sums; with guarded staging from N = 98304 on, the spatial-order
 * workspace, 44 to 52 bytes per particle) and return PP_ERR_NOMEM if that
 * fails.  N >= 1 (N = 0 -> PP_ERR_ARG); N <= 2^28.  On success *out receives
 * the context; on failure *out is set to NULL.
 */
pp_status pp_create(int64_t N, double w, double dt, double softening, pp_ctx **out);

/* Set an option (keys above).  Invalid key or value -> PP_ERR_ARG. */
pp_status pp_set_option(pp_ctx *ctx, int key, int64_t value);

/*
 * Read an option's current value: the accumulation mode, the positions mode in
 * force (SINGLE or SPLIT, also after AUTO decided), the split override, the
 * graph block, the wait limit, the stream, or for PP_OPT_VARIANT the index of
 * the force-kernel variant the next step will run.  Unknown key -> PP_ERR_ARG.
 */
pp_status pp_get_option(const pp_ctx *ctx, int key, int64_t *value);

/*
 * Load initial positions (m) and velocities (m/s), both [N][3].  vel may be
 * NULL for a cold bunch (v = 0).  Non-finite entries -> PP_ERR_ARG.
 * Computes the initial acceleration a(r0) (one force pass) so that the
 * first pp_step applies Eq. G with it, and resets the step counter to 0.
 */
pp_status pp_load_particles(pp_ctx *ctx, const double *pos, const double *vel, int on_device);

/*
 * Per-particle weights w_i ([N] doubles, finite and > 0), replacing the common
 * weight of pp_create, which stays the reference weight W: sources enter the
 * sum with w_j (staged as the FP32 ratio w_j / W), and KE, PE and momentum use
 * w_i.  w = NULL returns to equal weights.  If particles are loaded, a is
 * recomputed for the new weights (the state stays at the same time; with
 * PP_POS_AUTO the staging is decided again first).  Needs PP_ACC_FP64FOLD (or
 * PP_ACC_FP64_FULL), else PP_ERR_ARG; either staging of positions.  The paper uses one weight for all macro-particles (Sec. 2.1);
 * this generalises it.
 */
pp_status pp_set_weights(pp_ctx *ctx, const double *w, int on_device);

/*
 * Field E_i (V/m) of Eq. B at every particle's current position, written as
 * [N][3] to E_out.  Does not advance or modify the state.
 */
pp_status pp_compute_fields(pp_ctx *ctx, double *E_out, int on_device);

/*
 * Advance nsteps >= 0 Velocity-Verlet steps (Eq. G then Eq. H), one force
 * pass per step.  Returns after the steps have run.  PP_ERR_STATE if no
 * particles were loaded.
 */
pp_status pp_step(pp_ctx *ctx, int64_t nsteps);

/* Bunch diagnostics; averages <.> are plain means over the N macro-particles. */
typedef struct {
    double t;           /* simulated time, step * dt                          */
    int64_t step;       /* steps taken since the last load                    */
    double rms_radius;  /* sqrt(<|r - <r>|^2>)                                */
    double ke;          /* sum 1/2 m_e w |v|^2                                */
    double pe;          /* 1/2 sum_i sum_{j!=i} k (q_e w)^2 / sqrt(|r_ij|^2+eps^2) */
    double px, py, pz;  /* total momentum sum m_e w v                         */
    double emit_x;      /* Eq. I with raw averages                            */
    double x_rms;       /* sqrt(<x^2>)                                        */
    double x_max;       /* max_i x_i                                          */
    double vx_rms;      /* sqrt(<vx^2>)                                       */
    double vx_max;      /* max_i vx_i                                         */
    double cx, cy, cz;  /* centroid <r>                                       */
} pp_diag;

/*
 * Diagnostics of the current state.  All moments are deterministic FP64
 * reductions; pe needs one O(N^2) pass (FP32 pair math, FP64 fold).
 * with_pe = 0 skips that pass and sets pe to NaN.
 */
pp_status pp_diagnostics(pp_ctx *ctx, pp_diag *out, int with_pe);

/* Copy the current positions and velocities out ([N][3] each; either may be NULL). */
pp_status pp_get_particles(pp_ctx *ctx, double *pos, double *vel, int on_device);

/*
 * Checkpoint / resume.  pp_get_state copies r, v, a ([N][3] each; any may be
 * NULL), the step counter and the staging frame out; pp_set_state restores
 * them exactly (no force pass).  The staging frame is PP_FRAME_LEN = 5 host
 * doubles {cx, cy, cz, L0, staging}: the centre and the power-of-two length
 * about which positions are staged to FP32, and the staging in force
 * (PP_POS_SINGLE or PP_POS_SPLIT).  A context in PP_POS_AUTO adopts the saved
 * staging; a context with an explicit positions mode keeps its own.  Passing
 * the frame saved by pp_get_state makes stepping on from the restored state
 * bitwise identical to stepping on without the round trip; frame = NULL
 * chooses a fresh frame (centroid and RMS radius of pos, and under
 * PP_POS_AUTO a fresh staging decision), which changes results at the FP32
 * rounding level only.  acc must be the acceleration that belongs to pos (as
 * pp_get_state returns it).  Invalid frame (non-finite, L0 <= 0 or not a
 * power of two, staging not 0 or 1) -> PP_ERR_ARG.
 */
#define PP_FRAME_LEN 5
pp_status pp_get_state(pp_ctx *ctx, double *pos, double *vel, double *acc, int64_t *step,
                       double *frame, int on_device);
pp_status pp_set_state(pp_ctx *ctx, const double *pos, const double *vel, const double *acc,
                       int64_t step, const double *frame, int on_device);

/*
 * pp_check_mapped -- the paper has no counterpart; a service call.  PP_OK if
 * the `bytes` bytes at p may be passed as PP_MEM_HOST_MAPPED: page-locked host
 * memory mapped into the device address space, all of it in one allocation.
 * Otherwise PP_ERR_ARG, reason via pp_last_error(NULL).  Host-side only: no
 * kernel runs and the device never touches p.  Every call taking a
 * PP_MEM_HOST_MAPPED buffer makes this check before its kernels run.
 */
pp_status pp_check_mapped(const void *p, int64_t bytes);

/*
 * pp_fields_noalloc -- the paper has no counterpart; this is a service entry
 * point.  Field E_i (V/m) of Eq. B for N macro-electrons of weight w and
 * softening eps at positions pos, written to E_out; both are [N][3] device
 * memory of the current CUDA device, read and written on `stream` (a
 * cudaStream_t, or NULL for the legacy default stream).  No context needed.
 * Sources are staged hi/lo (about 48-bit separations, the PP_POS_SPLIT
 * arithmetic), so the result meets the 1e-5 relative-L2 field tolerance also
 * on inputs with very close pairs.
 *
 * It allocates nothing, for callers that may not call cudaMalloc (code that
 * runs inside a memory arena owned by a host framework, code that must not
 * trigger the allocator's implicit synchronisation, plug-ins restricted to the
 * buffers they are handed).  Every intermediate lives in one fixed device
 * array of 4.09 MB that each GPU loading this library holds until the
 * process exits; N above PP_FIELDS_NOALLOC_MAX_N returns PP_ERR_ARG.
 *
 * All calls on a device share that array and it keeps the last call's
 * contents (the call clears what must start at zero itself).  Calls whose work
 * overlaps on the GPU race on it: serialise them.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress with that
 * device current); make that first call before any stream capture.  The
 * lookup is repeated if the device's context has been recreated since (after
 * cudaDeviceReset, for instance).  The call synchronises `stream` three times
 * before it returns: twice mid-call, to read the centroid and RMS radius that
 * fix the staging frame, and once at the end, to read the error word.
 * Errors: PP_ERR_ARG (size, null pointer, non-finite input), PP_ERR_TIMEOUT,
 * PP_ERR_CUDA; message via pp_last_error(NULL).
 */
#define PP_FIELDS_NOALLOC_MAX_N 16384
pp_status pp_fields_noalloc(int64_t N, double w, double softening, const double *pos,
                            double *E_out, void *stream);

/* Outcome of pp_autotune and pp_batch_autotune. */
typedef struct {
    int variant;         /* chosen force-kernel variant (see pp_variant_name)       */
    int split;           /* chosen j-split count S (j-chunks per block of targets)  */
    double ms_per_pass;  /* measured time of one force pass with that choice, ms    */
    int candidates;      /* number of (variant, split) pairs that were timed        */
} pp_tune_result;

/*
 * ---- Batch contexts: many independent bunches, one persistent launch per step.
 *
 * A batch holds up to 4096 bunches ("slots"), each with its own N, weight,
 * time step, softening and state, and advances all of them together: every
 * time step is one launch of a persistent kernel whose CTAs pull work items
 * (bunch, block of targets, chunk of 8192 sources) from a queue.  Bunches use
 * FP32 pair math with the FP64 fold (PP_ACC_FP64FOLD) and single, hi/lo or
 * guarded staged positions (see pp_positions), chosen per bunch when it is
 * added: option PP_OPT_POSITIONS of the batch (default PP_POS_AUTO, which
 * takes the first of single and guarded staging whose fields differ from the
 * hi/lo-staged ones by at most 5e-6 for the bunch's own positions, else
 * hi/lo; pp_batch_get_option reports a bunch's choice).  A bunch's tiling (512
 * targets per block with single or guarded staging, 256 with hi/lo) depends on
 * its own N and staging only, so its results are bitwise the same alone or in
 * any mix.  Device memory is
 * admitted against the budget given at creation (pp_batch_footprint says what
 * one bunch takes).  Step blocks of PP_OPT_GRAPH_BLOCK steps (even; default
 * 16) replay a captured CUDA graph.  The persistent kernel comes in several
 * compiled shapes (threads per CTA, register budget, unrolling; see
 * pp_batch_shape_name) that all give bitwise the same results;
 * pp_batch_autotune times them on the current bunches.  Options:
 * PP_OPT_STREAM, PP_OPT_GRAPH_BLOCK, PP_OPT_TIMEOUT_NS, PP_OPT_POSITIONS,
 * PP_OPT_VARIANT (a shape index, -1 = the default shape 0),
 * PP_OPT_TEST_SKIP_COPY.
 */
typedef struct pp_batch pp_batch;

/* Device bytes one bunch of N particles takes in a batch (a function of N only). */
pp_status pp_batch_footprint(int64_t N, int64_t *bytes);

/* Create an empty batch on the current device with a device-memory budget in bytes. */
pp_status pp_batch_create(int64_t budget_bytes, pp_batch **out);

pp_status pp_batch_set_option(pp_batch *b, int key, int64_t value);

/*
 * Add a bunch (copies pos and vel, [N][3]; vel may be NULL for v = 0), run its
 * initial force pass, and return its slot index.  PP_ERR_NOMEM if its
 * footprint exceeds the remaining budget (nothing is changed then).
 * Slots of removed bunches are reused.  The bunch joins the next pp_batch_step.
 */
pp_status pp_batch_add(pp_batch *b, int64_t N, double w, double dt, double softening,
                       const double *pos, const double *vel, int on_device, int *slot);

/* Remove a bunch and return its memory to the budget. */
pp_status pp_batch_remove(pp_batch *b, int slot);

/* Advance every bunch in the batch by nsteps Velocity-Verlet steps. */
pp_status pp_batch_step(pp_batch *b, int64_t nsteps);

/* r, v, a ([N][3], any may be NULL) and the step counter of one bunch. */
pp_status pp_batch_get_state(pp_batch *b, int slot, double *pos, double *vel, double *acc,
                             int64_t *step, int on_device);

/* Diagnostics of one bunch, as pp_diagnostics (with_pe = 0 sets pe to NaN). */
pp_status pp_batch_diagnostics(pp_batch *b, int slot, pp_diag *out, int with_pe);

/*
 * Read an option.  slot = -1: the batch's PP_OPT_POSITIONS (for bunches added
 * from now on), PP_OPT_VARIANT (the kernel shape), PP_OPT_GRAPH_BLOCK,
 * PP_OPT_TIMEOUT_NS, PP_OPT_STREAM.  slot >= 0: PP_OPT_POSITIONS of that bunch
 * (PP_POS_SINGLE, PP_POS_SPLIT or PP_POS_GUARDED: the staging it runs with).
 * Else PP_ERR_ARG.
 */
pp_status pp_batch_get_option(pp_batch *b, int slot, int key, int64_t *value);

/* Name of compiled batch-kernel shape `index`, or NULL past the last one. */
const char *pp_batch_shape_name(int index);

/*
 * Batch autotuner: time one force pass (fields of the bunches' pending
 * positions into scratch; states untouched) of every compiled shape on the
 * active bunches and keep the fastest as PP_OPT_VARIANT.  Every shape gives
 * bitwise the same results, so tuning never changes a result.  out->variant is
 * the shape index, out->split 0.  PP_ERR_STATE if the batch is empty.
 */
pp_status pp_batch_autotune(pp_batch *b, pp_tune_result *out);

/* Active bunches, device bytes in use and the budget (any pointer may be NULL). */
pp_status pp_batch_info(pp_batch *b, int64_t *active, int64_t *bytes_used, int64_t *budget);

/* Free the batch and all its bunches.  NULL is accepted. */
pp_status pp_batch_destroy(pp_batch *b);

/*
 * The measurements of the last PP_POS_AUTO decision: relative-L2 difference
 * of the fields with single (and, if it was tried, guarded) staging from the
 * fields with hi/lo staging, at the positions the decision was made on; NaN
 * where not measured.  Either pointer may be NULL.
 */
pp_status pp_staging_check(const pp_ctx *ctx, double *single_rel, double *guarded_rel);

/* Number of particles of the context. */
pp_status pp_get_n(const pp_ctx *ctx, int64_t *n);

/* Free the context and its device memory.  NULL is accepted. */
pp_status pp_destroy(pp_ctx *ctx);

/* Message for the last non-OK status on this thread (ctx may be NULL). */
const char *pp_last_error(const pp_ctx *ctx);

/*
 * Name of compiled force-kernel variant `index` (for PP_OPT_VARIANT and for
 * tuning tools), or NULL past the last one.  Names read
 * "<pairs>.<fold>.t<threads>r<targets per thread>k<tile>", e.g.
 * "f32x2.fold64.t256r4k256": packed FP32x2 pair math, FP64 fold, 256 threads,
 * 4 targets per thread, 256-source tiles.
 */
const char *pp_variant_name(int index);


/*
 * Autotuner: time every compiled force-kernel variant that fits the
 * context's accumulation and positions modes, each with the launch planner's
 * j-split count S and with S/4, S/2 and 2S, on the context's loaded particles, and
 * keep the fastest pair as the context's PP_OPT_VARIANT and PP_OPT_SPLIT.
 * Only force passes run (fields of the current positions into scratch): the
 * particle state and step counter are untouched.  Where steps run on the
 * resident small-N kernel (PP_OPT_RESIDENT), only variants with its staging
 * layout are timed, so the choice keeps the steps resident.  Takes a few
 * hundred force passes at most; PP_ERR_STATE if no particles are loaded.  out
 * may be NULL.
 */
pp_status pp_autotune(pp_ctx *ctx, pp_tune_result *out);

/* Library version string. */
const char *pp_version(void);

/*
 * Pair-interaction count of one step, N*N (the all-pairs convention used for
 * throughput: pair-interactions per second).
 */
double pp_pairs_per_step(int64_t N);

#ifdef __cplusplus
}
#endif

#endif /* PP_GB300_H */
