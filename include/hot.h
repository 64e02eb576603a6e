/*
 * hot.h -- C ABI of the GB300 engine for weighted Gerchberg-Saxton (GSW) holograms by
 * direct superposition (S. Bianchi, R. Di Leonardo, "Real-time optical micro-manipulation
 * using optimized holograms generated on the GPU").
 *
 * The engine computes, for an SLM of W x H pixels (pitch p) and M traps (x_m, y_m, z_m)
 * behind optics of wavelength lambda and effective focal length f:
 *   Eq. 2   Delta_j^m = z_m pi/(lambda f^2) (x_j^2 + y_j^2) + 2 pi/(lambda f) (x_j x_m + y_j y_m)
 *   Eq. 1   V_m = (1/N) sum_j exp(i (phi_j - Delta_j^m))                  (forward field)
 *   Sec. 3  w_m <- w_m <|V|> / |V_m|,  <|V|> = mean over m of |V_m|     (weight update)
 *   Sec. 4  phi_j = arg sum_m w_m (V_m/|V_m|) exp(i Delta_j^m)            (back-projection)
 *   Eq. 4   e = sum_m |V_m|^2,  u = 1 - (max I - min I)/(max I + min I)  (quality)
 *   Sec. 5  8-bit SLM grey levels g_j = rint(phi_j 256/(2 pi)) mod 256
 * Pixel j = iy*W + ix has coordinates x_j = (ix - floor(W/2)) p, y_j = (iy - floor(H/2)) p.
 * Device arithmetic is FP32, except the trap-table set-up (Eq. 2 reduced modulo 2 pi in FP64,
 * once per hot_set_traps) and the sum of the per-sub-tile field sums over the image, which is
 * exact integer arithmetic in 64-bit fixed point.  Every other reduction runs in a fixed
 * order: results are bit-reproducible for a given device, size and precision mode.
 *
 * Conventions shared by every entry point:
 *   - Return value: HOT_OK (0) or a negative hot_status; no call aborts or exits.
 *     hot_last_error() returns a text for the last failure of the calling thread.
 *   - Invalid sizes or pointers give HOT_EINVAL before any device work is queued.
 *   - Work is queued on the context's CUDA stream (given at creation; NULL is the legacy
 *     default stream).  Calls that return data to host memory synchronise that stream.
 *   - Host pointers are read or written before the call returns; device pointers
 *     (on_device = 1) must be valid on the context's device and are used in stream order.
 *   - The library owns every device buffer of a context; hot_destroy frees them.
 *   - A context is not thread-safe: use one context per thread.
 */
#ifndef HOT_H
#define HOT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hot_ctx hot_ctx;

typedef enum {
  HOT_OK = 0,
  HOT_EINVAL = -1,   /* invalid argument (size, pointer, mode) */
  HOT_ENOMEM = -2,   /* device or host allocation failed */
  HOT_ECUDA = -3,    /* a CUDA call failed; see hot_last_error() */
  HOT_ETIMEOUT = -4, /* a bounded device-side wait expired */
  HOT_ESTATE = -5    /* call out of order (e.g. hot_gsw before hot_set_traps) */
} hot_status;

/* Accuracy of the modes against an FP64 evaluation of the method (the parity tests' bounds):
 * |V_m| within 1e-4 relative after one GSW iteration, e and u within 1e-3 after a run, 8-bit
 * output equal except within 1e-4 rad of a level boundary.  HOT_PREC_ACCURATE and
 * HOT_PREC_SEPARABLE meet these bounds on every tested case, up to HOT_MAX_TRAPS traps.
 * HOT_PREC_FAST and HOT_PREC_TENSOR meet them on every tested case except strongly cancelling
 * back-projections: 4096 traps on a 160 x 120 SLM, whose first weight update spreads the weights
 * over a factor ~400, so that the superposition cancels at some pixels and amplifies each term's
 * error.  There the |V_m| error after one iteration is bounded by 2e-4 in the fast mode (1.2e-4
 * measured; accurate 7.6e-5) and by 5e-4 in the tensor mode (3.3e-4 measured).  Measured
 * elsewhere: 512 x 512 px with 100 traps, 2.5e-6 fast, 2.4e-6 accurate (the one-exponential step,
 * hot_set_once; the direct kernels: 4.1e-6, 6.0e-6); 1920 x 1152 px with 1000 traps, 8.8e-6 fast. */
typedef enum {
  HOT_PREC_ACCURATE = 0, /* sincospif on the exactly reduced phase (FP32, ~1 ulp) */
  HOT_PREC_FAST = 1,     /* the direct evaluation on the special-function unit: sin.approx /
                             cos.approx of the reduced phase (arguments pre-scaled by 1 + 8.17e-8
                             against the unit's mean argument shrink); the direct step's forward
                             field rotates the phases of each pixel sub-tile by a fixed
                             pseudo-random angle and its sums back, so that the unit's systematic
                             error does not add up over the pixels (the one-exponential step,
                             M <= 128, forms the forward terms as e^{i phi_j} conj(e^{i Delta}),
                             where a constant error of the unit only meets the small zero-order
                             sum of e^{i phi_j}) */
  HOT_PREC_SEPARABLE = 2, /* Eq. 2 factorised: e^{i Delta} = e^{i X_m(ix)} e^{i Y_m(iy)} from FP32
                             complex tables (FP64 cos/sin once per entry); per pair one complex
                             multiply-add in each step, no transcendental function */
  HOT_PREC_TENSOR = 3      /* EXPERIMENTAL, outside the direct method: the separable form on the
                             tensor cores; each step of a GSW iteration is a complex matrix product
                             (S = P X, T = U X^H) run as tcgen05 FP16 MMAs with every operand split
                             in two FP16 parts (three MMAs per product, FP32 accumulation); the GSW
                             loop only (hot_gsw), other calls run the separable kernels; |V_m|
                             error up to 5e-4 on strongly cancelling back-projections (above) */
} hot_precision;

typedef enum {
  HOT_FMT_F32 = 0, /* float32 radians in (-pi, pi] */
  HOT_FMT_U8 = 1   /* uint8 grey level, rint(phi 256/(2 pi)) mod 256 (Sec. 5) */
} hot_format;

/* Largest trap count a context accepts. */
#define HOT_MAX_TRAPS 4096

/* Creates a context for a W x H SLM (Sec. 3: pixel pitch, wavelength, effective focal
 * length, all in metres) on the current CUDA device, queueing work on cuda_stream
 * (a cudaStream_t, or NULL).  W, H >= 1, W*H < 2^31; pitch, wavelength, focal > 0 and
 * finite.  The initial phase is 0 everywhere and the precision is HOT_PREC_ACCURATE.
 * *out receives the context (set to NULL on failure). */
int hot_create(hot_ctx **out, int width, int height, double pitch_m, double wavelength_m,
               double focal_m, void *cuda_stream);

/* Sets the M traps (Sec. 4 "trap structure"): xyz_m is a host array of M*3 doubles
 * (x_m, y_m, z_m) in metres, row per trap; w0 (host, M doubles > 0, or NULL for all 1) are
 * the initial GSW weights.  1 <= M <= HOT_MAX_TRAPS, coordinates finite.  Builds the
 * per-trap phase tables on the device (Eq. 2 reduced modulo 2 pi in FP64). */
int hot_set_traps(hot_ctx *c, int M, const double *xyz_m, const double *w0);

/* Replaces the GSW weights (host, M doubles > 0).  HOT_ESTATE before hot_set_traps. */
int hot_set_weights(hot_ctx *c, const double *w);

/* Sets the pixel phases phi_j (N = W*H float32 radians, row-major, any range):
 * host memory (on_device = 0) or device memory (on_device = 1). */
int hot_set_phase(hot_ctx *c, const float *phi, int on_device);

/* Selects HOT_PREC_ACCURATE, HOT_PREC_FAST, HOT_PREC_SEPARABLE or HOT_PREC_TENSOR for the
 * following calls (switching between the direct and the separable kernels synchronises and
 * rebuilds the work schedule).  HOT_EINVAL for another value.  In HOT_PREC_TENSOR mode hot_gsw
 * runs three kernels per iteration (weight update and operand P, back-projection GEMM with the
 * phases in its epilogue, forward GEMM with the field sums in its epilogue); its operands
 * (about 4 (2W + 2M)(2M + 2W) + 8 H (W + M) + 8 H M bytes) are built on the first hot_gsw after the
 * traps are set (row-band steps, hot_sharded_*, run the same kernels).  HOT_PREC_TENSOR rejects the
 * persistent form (hot_use_persistent) and hot_autotune with HOT_EINVAL; its batches run each
 * member's own launch sequence (see hot_batch_create). */
int hot_set_precision(hot_ctx *c, int precision);

/* Runs `iters` GSW iterations (Sec. 3, Fig. 2) from the current phases and weights:
 * for k = 1..iters: V = F(phi) (Eq. 1); w_m <- w_m <|V|>/|V_m|; phi = arg of the
 * back-projection with coefficients w_m V_m/|V_m|.  Then V = F(phi) of the final phase and
 * its efficiency e and uniformity u (Eq. 4).  iters = 0 only evaluates F, e and u.
 * Repeated calls continue from the state left by the previous one, so two calls with
 * K1 and K2 iterations give the same phases, weights and fields as one call with K1 + K2.
 * eff_out / unif_out (host, nullable): if either is non-NULL the call synchronises and
 * writes them; otherwise it returns once the work is queued.  Readings where the paper
 * is silent: if |V_m| < 1e-30 the unit field is taken as 1 and w_m is kept; arg(0) = 0.
 * By default each iteration is one kernel launch (three in HOT_PREC_TENSOR), the sequence
 * replayed as a CUDA graph; with hot_use_persistent the iterations run in one cooperative launch
 * whose blocks meet at a grid-wide barrier between iterations.  There a barrier wait longer than
 * the wait limit (hot_set_wait_limit) makes the kernel leave early, and the next synchronising
 * call (this one with eff_out/unif_out, hot_sync, hot_get_fields, hot_get_metrics) returns
 * HOT_ETIMEOUT: the accumulators are reset and the phases are undefined.  The tensor-core
 * kernels bound their pipeline waits by the same limit, with the same outcome.
 * HOT_ESTATE before hot_set_traps; HOT_EINVAL if iters < 0. */
int hot_gsw(hot_ctx *c, int iters, double *eff_out, double *unif_out);

/* Checkpoint / resume: the GSW state is the phases and the weights (float32, exactly as held),
 * so hot_set_state on a context with the same optics and traps continues where hot_get_state
 * left off, bit for bit in the direct, separable and tensor modes.  phi: HOST float32 [H*W];
 * w: HOST float32 [M] (finite, > 0).  Both synchronise; HOT_ESTATE before hot_set_traps.
 * hot_set_state drops the unit phasors below. */
int hot_get_state(hot_ctx *c, float *phi, float *w);
int hot_set_state(hot_ctx *c, const float *phi, const float *w);

/* The one-exponential step (hot_set_once) takes u_j = S_j/|S_j| for the forward field of each
 * iteration and evaluates phi_j = arg S_j only in the last launch of a hot_gsw, where it also
 * keeps u_j; the next hot_gsw of the context starts from those u_j, so that hot_gsw(a) followed by
 * hot_gsw(b) equals hot_gsw(a + b) bit for bit.  They belong to the state of that form:
 * hot_get_phasors copies them out (HOT_ESTATE when the current phases have none: set by the
 * caller, or written by another mode); hot_set_phasors, after hot_set_state with the phases
 * they belong to, restores them, and the resumed run continues bit for bit (without them it
 * starts from e^{i phi_j}, equal to within the phasors' rounding, ~1e-7).  u: HOST float32
 * [H*W][2] (re, im); every value finite with magnitude <= 2, else HOT_EINVAL; HOT_ESTATE when the
 * one-exponential step is not in effect.  Both synchronise.  (No counterpart in the paper.) */
int hot_get_phasors(hot_ctx *c, float *u);
int hot_set_phasors(hot_ctx *c, const float *u);

/* Convergence trace (no counterpart in the paper): with enable != 0, every following hot_gsw
 * records e and u (Eq. 4) of the field each iteration starts from; block 0 of each step
 * computes them from the sums it reads anyway.  hot_get_trace then returns n = iters + 1
 * values of the last call: F(phi^0), ..., F(phi^(iters-1)) and the final F(phi^iters).
 * eff, unif: HOST arrays of n doubles.  HOT_ESTATE without a traced call; HOT_EINVAL for
 * another n.  hot_set_trace synchronises. */
int hot_set_trace(hot_ctx *c, int enable);
int hot_get_trace(hot_ctx *c, double *eff, double *unif, int n);

/* enable != 0: hot_gsw runs as one persistent cooperative launch plus the finalize kernel;
 * 0 (the default): one launch per iteration, replayed as a CUDA graph (hot_use_graphs), whose
 * programmatic dependent launches overlap consecutive iterations.  Both forms use the same
 * schedule and arithmetic and give the same bits. */
int hot_use_persistent(hot_ctx *c, int enable);

/* Longest wait at one grid barrier of the persistent kernel, in seconds (default 2; 0 makes
 * every wait run out at once, which exercises the HOT_ETIMEOUT path).  HOT_EINVAL outside
 * [0, 60]. */
int hot_set_wait_limit(hot_ctx *c, double seconds);

/* Writes the current phases (N pixels, row-major) to dst in format fmt (hot_format):
 * float32 radians in (-pi, pi] or uint8 grey levels (Sec. 5: 256 levels linear in
 * 0..2 pi, level 0 = phase 0, round to nearest).  dst is host (on_device = 0, the call
 * synchronises) or device memory (on_device = 1, queued). */
int hot_phase_out(hot_ctx *c, void *dst, int fmt, int on_device);

/* Copies to host the trap fields V (2*M doubles, interleaved Re, Im) of the last forward
 * evaluation (after hot_gsw: the fields of the final phase) and the current weights w
 * (M doubles).  Either pointer may be NULL.  Synchronises.  HOT_ESTATE if no forward
 * evaluation has run since the traps or phases were set. */
int hot_get_fields(hot_ctx *c, double *V, double *w);

/* Selects how hot_gsw issues its kernels: enable = 1 (default) replays a CUDA graph of the
 * whole iters-iteration sequence, captured on first use for each (iters, precision) and
 * dropped when the trap count changes; enable = 0 launches the kernels one by one.  The
 * results are identical.  While profiling (hot_profile) kernels are always launched one by
 * one. */
int hot_use_graphs(hot_ctx *c, int enable);

/* Back-propagation from the traps with explicit complex coefficients (Sec. 4):
 *   phi_j = arg sum_m c_m exp(i Delta_j^m),
 * which become the context's phases.  With c_m = exp(i theta_m), theta_m random, this is the
 * random superposition (SR) hologram of Eq. 3; GSW can continue from it (hot_gsw), and
 * hot_gsw(c, 0, &e, &u) reports its efficiency and uniformity.  coef: HOST array of 2*M
 * doubles interleaved (Re, Im).  The GSW weights are not changed.  HOT_ESTATE before
 * hot_set_traps. */
int hot_superposition(hot_ctx *c, const double *coef);

/* Trap fields of arbitrary phases (Eq. 1) for the context's traps, without touching its GSW
 * state (phases, weights): V_m = (1/N) sum_j exp(i (phi_j - Delta_j^m)).
 * phi: DEVICE float32 [N] row-major; V: DEVICE float32 [2*M] output, interleaved (Re, Im).
 * Queued on the context's stream.  hot_get_fields afterwards returns these fields.
 * HOT_ESTATE before hot_set_traps. */
int hot_field(hot_ctx *c, const float *phi, float *V);

/* Adjoint of Eq. 1, i.e. the gradient of a real loss L(V) with respect to the phases:
 *   dL/dphi_j = (1/N) Im[ exp(-i phi_j) sum_m G_m exp(i Delta_j^m) ],  G_m = 2 dL/d conj(V_m)
 * (the PyTorch convention for the gradient of a complex tensor).  It is the back-projection
 * superposition of Sec. 4 with coefficients G_m.  phi: DEVICE float32 [N]; G: DEVICE float32
 * [2*M] interleaved; grad: DEVICE float32 [N] output.  Queued on the context's stream; the
 * GSW state is not touched.  HOT_ESTATE before hot_set_traps. */
int hot_field_adjoint(hot_ctx *c, const float *phi, const float *G, float *grad);

/* The trap-intensity loss of the differentiable form and its gradient in one call (no
 * counterpart in the paper; its intensities are those of Eq. 4): with V = F(phi) (Eq. 1) and
 * I_m = |V_m|^2,
 *   L = -sum_m log I_m + beta var_m(I)   (population variance over the traps),
 * and dL/dphi by the adjoint of Eq. 1 with G_m = 2 g_m V_m, g_m = -1/I_m + beta (2/M)(I_m - mean I)
 * (see hot_field_adjoint).  Three kernels on the context's stream (forward field, loss and G in
 * FP64 sums, adjoint), nothing read back: an optimiser step on the phases then costs these
 * kernels and the optimiser's update.  phi: DEVICE float32 [N]; loss: DEVICE float32 [1] output;
 * grad: DEVICE float32 [N] output, or NULL for the loss alone.  The GSW state is not touched;
 * hot_get_fields / hot_get_metrics afterwards report F(phi).  HOT_ESTATE before hot_set_traps;
 * HOT_EINVAL for NULL phi or loss or a non-finite beta. */
int hot_intensity_loss(hot_ctx *c, const float *phi, double beta, float *loss, float *grad);

/* ---- row bands: the sharded form --------------------------------------------------------
 * Eq. 1 is a sum over pixels, so the pixels can be split into row bands, one per GPU: each
 * band computes partial sums of V_m over its rows, the partial sums are added over the bands
 * (one all-reduce of 2M int64 per iteration), and every band then derives the same weights and
 * coefficients (Sec. 3) from the same global sums and back-projects its own rows.  The sums
 * are 64-bit fixed-point integers, so the all-reduce is exact and independent of its order. */

/* Makes the context rows y0 .. y0+height-1 of a width x total_height hologram (its pixel
 * coordinates and the 1/N of Eq. 1 are those of the whole hologram).  total_height = height,
 * y0 = 0 is the plain context.  Rebuilds the phase tables if traps are set; synchronises.
 * HOT_EINVAL if the band does not fit. */
int hot_set_band(hot_ctx *c, int total_height, int y0);

/* The launch sequence of hot_gsw, one launch per call, for a caller that adds the partial
 * sums over the bands between launches (not captured as a graph):
 *   hot_sharded_begin(c)      launch 0: partial sums of V for the current phases;
 *   hot_sharded_sums(c, k, &p, &n) DEVICE pointer to launch k's partial sums, n int64 values
 *                             (copies x [2][M]: Re parts, then Im parts, two's complement; the
 *                             field is their sum over the copies), to be replaced in place, in
 *                             stream order on the context's stream, by their elementwise sum
 *                             over all bands before the next launch;
 *   hot_sharded_step(c, k)    launch k = 1, 2, ...: weight update, back-projection of the band,
 *                             partial sums of the new forward field;
 *   hot_sharded_end(c, K, &e, &u) after launch K: the metrics (Eq. 4) and fields of the summed
 *                             sums, weights home; e, u nullable (synchronises when given).
 * Launches are queued on the context's stream.  HOT_ESTATE for a call out of this order. */
int hot_sharded_begin(hot_ctx *c);
int hot_sharded_step(hot_ctx *c, int k);
int hot_sharded_sums(hot_ctx *c, int k, void **sums_dev, int *count);
int hot_sharded_end(hot_ctx *c, int iters, double *eff_out, double *unif_out);

/* Efficiency e and uniformity u (Eq. 4) of the last forward evaluation (hot_gsw, hot_field or
 * hot_batch_gsw).  Synchronises.  HOT_ESTATE if none has run since the traps or phases changed. */
int hot_get_metrics(hot_ctx *c, double *eff_out, double *unif_out);

/* ---- tiling and autotuning ----------------------------------------------------------------
 * The step kernels give every thread one pixel column of a sub-tile of `rows` rows
 * (1..14: pixels per thread), run `blocks_per_sm` resident blocks of 256 threads per SM
 * (1..4; the grid is one wave of SMs x blocks_per_sm persistent blocks) and stage the trap
 * tables in shared memory `chunk` traps at a time (1..128).  The results do not depend on the
 * tiling beyond FP32 rounding of the per-pixel sums.  Defaults: 14, as many as fit, 128. */

/* Sets the tiling (0 selects a parameter's default) and rebuilds the work schedule.
 * Synchronises the context's stream.  HOT_EINVAL out of range. */
int hot_set_tiling(hot_ctx *c, int rows, int blocks_per_sm, int chunk);

/* The tiling in effect (blocks_per_sm as launched).  Any output pointer may be NULL. */
int hot_get_tiling(const hot_ctx *c, int *rows, int *blocks_per_sm, int *chunk);

/* Block merging of the accurate and fast modes' GSW step (no counterpart in the paper): with
 * 4 schedule blocks per SM (the default count), merge = 4 launches one block of 1024 threads per
 * SM that holds 4 schedule blocks as groups of 256 threads (each with its own shared memory and
 * barrier), merge = 2 two blocks of 512 threads per SM holding 2 each, merge = 1 (default) the
 * schedule's blocks themselves.  Consecutive schedule blocks hold consecutive runs of the image,
 * which add up to their equal share to within one 32-pixel row segment, while independent blocks
 * land on SMs in no fixed order, and an SM may get 4 runs that are each one segment longer than
 * average.  The price of merging is a later start of the next launch's blocks (a launched block's
 * groups must all finish first).  The results are the same bits either way.  hot_autotune
 * searches 1, 2 and 4.  merge: 1, 2 or 4, else HOT_EINVAL.  Rebuilds the schedule; synchronises
 * the context's stream.  hot_get_block_merge reports the setting and the merge in effect (1 where
 * it does not apply: the separable and tensor modes, fewer than 4 blocks per SM). */
int hot_set_block_merge(hot_ctx *c, int merge);
int hot_get_block_merge(const hot_ctx *c, int *requested, int *in_effect);

/* One-exponential step of the accurate and fast modes (no counterpart in the paper's kernel;
 * the same sums, Eq. 1 and Sec. 3): with M <= 128 traps the GSW step evaluates each pixel-trap
 * exponential E = e^{i Delta_j^m} (Eq. 2) once per iteration and keeps it in registers between
 * the back-projection S_j = sum_m c_m E and the forward field N V_m = sum_j u_j conj(E), with
 * u_j = S_j/|S_j| = e^{i phi_j} (phi_j = atan2 S_j is evaluated only in the last launch of a
 * call), which halves the cos/sin work of an iteration.  Its blocks split the M traps among their
 * warps (at most 16 traps per warp, so at most 128 traps) and walk sub-tiles of 2 to 8 rows (fixed
 * by M); its schedule is its own, so the tiling above does not apply to it (it still applies to
 * the adjoint and the superposition, which keep the direct kernels).  A call that continues from
 * the phases of the previous one starts with the forward field of the unit phasors that call's
 * last step kept (hot_get_phasors), in the step's arithmetic, so resumed sequences, CUDA graphs
 * and the persistent form give the same bits; a call that starts from phases the caller set
 * takes their forward field from the separable kernel (complex tables).  Its results differ from
 * the direct kernels' by FP32 rounding.  on: 1 (default) or 0, else HOT_EINVAL; it is in effect
 * where M <= 128 and the mode is HOT_PREC_ACCURATE or HOT_PREC_FAST.  Rebuilds the schedule;
 * synchronises the context's stream.  hot_get_once reports the setting and whether it is in
 * effect. */
int hot_set_once(hot_ctx *c, int on);
int hot_get_once(const hot_ctx *c, int *requested, int *in_effect);

/* Autotuner: times hot_gsw(iters) (CUDA events, best of 3 graph replays) for candidate tilings
 * by coordinate search over rows, blocks_per_sm (with block merging, hot_set_block_merge, as a
 * candidate in the accurate and fast modes) and chunk, keeps the fastest, and reports it
 * with its time per iteration in microseconds (outputs may be NULL).  Where the one-exponential
 * step is requested and applies (hot_set_once), it is timed too and kept if it is faster than
 * the best tiling of the direct kernels; otherwise the setting is turned off (hot_get_once).  The phases and weights
 * are restored afterwards; the fields are stale until the next forward evaluation (HOT_ESTATE
 * from hot_get_fields).  Synchronises.  HOT_ESTATE before hot_set_traps; iters >= 1. */
int hot_autotune(hot_ctx *c, int iters, int *rows, int *blocks_per_sm, int *chunk, double *us_per_iter);

/* ---- batches of holograms ------------------------------------------------------------------
 * A batch runs GSW on several contexts at once -- SLMs of different sizes and trap counts.
 * The holograms are ordered by their work per iteration (N x M pixel-trap pairs, smallest
 * first) and cut into groups of at least `group_pairs` pairs per iteration (and at most 22
 * holograms: their parameters travel in the kernel launch); each group runs
 * its iterations with one kernel launch per iteration that covers all of its holograms (their
 * row segments are dealt out to one wave of blocks in equal shares of pairs), and the groups
 * run one after another, so that small holograms neither leave the GPU idle nor wait for the
 * large ones.  Each hologram keeps its own tables, phases, weights and accumulators (its
 * context's buffers); the iteration is the same as hot_gsw's (Sec. 3). */
typedef struct hot_batch hot_batch;

/* Groups count >= 1 contexts (same device, traps set, same precision mode, not row bands)
 * into a batch
 * queued on cuda_stream (NULL: the legacy stream).  The batch refers to the contexts'
 * buffers: recreate it after hot_set_traps changes a trap count, and destroy it before
 * destroying its contexts.  The contexts must not be used concurrently with the batch.
 * HOT_PREC_TENSOR batches are not packed into shared launches: each member runs exactly the
 * launch sequence of its own hot_gsw (same results, bit for bit), and the members are dealt out
 * to up to 8 chains (largest N M first, each to the least loaded chain) that run concurrently
 * inside the batch's graph, so that the launches of small holograms, which leave most SMs idle,
 * overlap.  Such a batch has no tiling: hot_batch_set_tiling and hot_batch_autotune return
 * HOT_EINVAL, and hot_batch_get_tiling reports the number of chains as its groups. */
int hot_batch_create(hot_batch **out, int count, hot_ctx *const *ctxs, void *cuda_stream);

/* Tiling of the batch's launches (as hot_set_tiling; 0 selects a default) and the minimum
 * work of a group in pixel-trap pairs per iteration (0: 2^26; 1: every hologram its own
 * group; a value above the total: one group, all holograms in lockstep).  Rebuilds the
 * schedule; synchronises the batch's stream. */
int hot_batch_set_tiling(hot_batch *b, int rows, int blocks_per_sm, int chunk, double group_pairs);

/* The batch's tiling, group threshold and number of groups (outputs may be NULL). */
int hot_batch_get_tiling(const hot_batch *b, int *rows, int *blocks_per_sm, int *chunk, double *group_pairs,
                         int *groups);

/* Autotuner of the batch's tiling, as hot_autotune (the group threshold is kept): times
 * hot_batch_gsw(iters) and restores every hologram's phases and weights. */
int hot_batch_autotune(hot_batch *b, int iters, int *rows, int *blocks_per_sm, int *chunk, double *us_per_iter);

/* Runs iters GSW iterations on every hologram of the batch (groups in order, one launch per
 * group and iteration; the whole sequence is one CUDA graph, captured on first use for each
 * iters).  Afterwards each context holds its new phases and weights, and hot_get_fields /
 * hot_get_metrics / hot_phase_out report its final forward field.  Queued; returns at once. */
int hot_batch_gsw(hot_batch *b, int iters);

/* Per-hologram latency of the last hot_batch_gsw: ms[h] = time from the start of its first
 * launch to the completion of hologram h (device %globaltimer stamps, ns resolution of the
 * timer as implemented by the GPU).  ms: HOST array of count doubles, in the order the
 * contexts were given.  Synchronises.  HOT_ESTATE before the first hot_batch_gsw. */
int hot_batch_latency(hot_batch *b, double *ms, int count);

/* Frees the batch (NULL-safe); its contexts are not touched. */
void hot_batch_destroy(hot_batch *b);

/* Waits for all work queued by the context.  HOT_ETIMEOUT if a barrier wait of the persistent
 * kernel ran out since the last check (see hot_gsw). */
int hot_sync(hot_ctx *c);

/* DIAGNOSTIC: number of kernels the context has launched since creation (instrumentation). */
long long hot_kernel_launches(const hot_ctx *c);

/* Kernel classes reported by hot_profile_read. */
typedef enum {
  HOT_KERNEL_STEP = 0,    /* fused back-projection + forward field (one GSW iteration) */
  HOT_KERNEL_FORWARD = 1, /* forward field only (Eq. 1 of the starting phases) */
  HOT_KERNEL_FINISH = 2,  /* FP64 field reduction, weight update, Eq. 4 metrics */
  HOT_KERNEL_OTHER = 3,   /* trap tables, 8-bit encoding */
  HOT_KERNEL_KINDS = 4
} hot_kernel_kind;

/* DIAGNOSTIC (not part of the method's path; for tests and benchmarks).
 * Instrumentation: while enabled (enable = 1), CUDA events are recorded on the context's
 * stream around every kernel the context launches.  hot_profile_read synchronises the
 * stream and writes, per hot_kernel_kind, the summed device time in milliseconds (ms[4])
 * and the number of launches (launches[4]) recorded since the last read, then clears the
 * records.  Either array may be NULL.  Disabling drops unread records. */
int hot_profile(hot_ctx *c, int enable);
int hot_profile_read(hot_ctx *c, double *ms, long long *launches);

/* Frees the context and its device buffers (NULL-safe). */
void hot_destroy(hot_ctx *c);

/* DIAGNOSTIC (not part of the method's path; for benchmarks): a microbenchmark kernel with
 * no counterpart in the paper.  Measures, on the current device, the
 * throughput of the special-function unit that bounds hot_gsw in HOT_PREC_FAST mode, in
 * lane results per clock per SM, with a dependency-free loop of 1024 threads per SM whose
 * arguments change every iteration (clock64-timed).  op: 0 = sin.approx and cos.approx of
 * one argument (the pattern of the GSW kernels), 1 = sin.approx alone, 2 = ex2.approx,
 * 3 = FP32 fused multiply-add (the pipe that bounds HOT_PREC_SEPARABLE).
 * *per_clk_per_sm receives the rate and *sms (nullable) the SM count.  Synchronises the
 * device; takes a few milliseconds. */
int hot_sfu_rate(int op, double *per_clk_per_sm, int *sms);

/* Launch shapes HOT_PREC_TENSOR would use for a width x height hologram with M traps on a GPU
 * with `sms` SMs (host computation only: no device work, no context).  shape (host, 9 ints)
 * receives: [0] tile width of the back-projection GEMM, [1] of the forward GEMM (32, 64, 128 or
 * 256 columns), [2] K splits of the forward GEMM, [3] K slices (64 elements) per split, [4] K of
 * the back-projection GEMM (2M padded to a slice), [5] K of the forward GEMM (2W padded),
 * [6] rows padded to the 128-row tile, [7] 2W and [8] 2M padded to their tile widths. */
int hot_tc_shape(int width, int height, int M, int sms, int *shape);

/* DIAGNOSTIC (not part of the method's path; a test hook): the matrix product of
 * HOT_PREC_TENSOR on its own (no counterpart in the paper):
 * C = A B^T for DEVICE float32 arrays A [rows][K], B [cols][K] (row-major) into C [rows][cols],
 * on the tcgen05 tensor cores with every operand split into two parts (a b ~ a_hi b_hi +
 * a_hi b_lo + a_lo b_hi, FP32 accumulation, each K slice's partial product added in FP32
 * registers), tiles of 128 x tile_n (32, 64, 128 or 256).  operands: HOT_TC_TF32 (two TF32
 * parts, kind::tf32; the FP32 exponent range) or HOT_TC_FP16 (two FP16 parts, kind::f16 at twice
 * the rate; the FP16 range: |x| < 65504, and precision drops for |x| below ~0.25, where the low
 * part is subnormal -- the mode uses it on operands of magnitude ~1).  rows, cols, K >= 1.
 * Allocates its split operands, synchronises cuda_stream (a cudaStream_t or NULL) and frees
 * them before returning.  HOT_ETIMEOUT if a bounded device-side wait ran out. */
#define HOT_TC_TF32 0
#define HOT_TC_FP16 1
int hot_tc_gemm(int rows, int cols, int K, const float *A, const float *B, float *C, int tile_n, int operands,
                void *cuda_stream);

/* Text of the last error on the calling thread ("" if none). */
const char *hot_last_error(void);

/* ---- allocation-free evaluation of the trap fields ---------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers that must not
 * allocate device memory: a real-time hologram loop whose memory is planned once up front,
 * code whose device memory is owned by an external pool or allocator, or hosts that forbid
 * cudaMalloc/cudaFree after start-up.  Every other entry point allocates in its context.
 *
 * hot_field_noalloc computes V_m = (1/N) sum_j exp(i (phi_j - Delta_j^m)) (the same forward
 * field that hot_gsw(c, 0, ...) evaluates for a context) and, if eu is not NULL, e and u of
 * Eq. 4.  It calls no cudaMalloc, cudaFree or other allocating routine: its working memory
 * (trap tables, work schedule, field accumulators, reduction counter) lives in one
 * file-scope __device__ array of HOT_NOALLOC_SCRATCH_BYTES that every GPU which loads the
 * library holds until the process exits.
 *   width, height, pitch_m, wavelength_m, focal_m: as for hot_create.
 *   M, xyz_m: trap count and DEVICE array of M*3 doubles (x_m, y_m, z_m) in metres.
 *   phi: DEVICE array of width*height float32 phases (radians), row-major.
 *   precision: HOT_PREC_ACCURATE or HOT_PREC_FAST.
 *   V: DEVICE output, 2*M doubles interleaved (Re, Im).  eu: DEVICE output of 2 doubles
 *   (e, u) or NULL.  cuda_stream: a cudaStream_t or NULL.
 * Work is queued on cuda_stream; the host reads nothing back.  The working memory is
 *   8 M (W + H) + 88 M + 16 n_sub + 4 (G + 1) bytes, plus at most 2.3 KiB of alignment,
 * where G (at most 4 per SM) is the number of thread blocks and n_sub, about
 * (W/32)(H/14) + 2 G, the number of pixel sub-tiles of the work schedule.  The call computes
 * this need exactly before queueing any device work; sizes whose need exceeds the scratch array
 * are rejected with HOT_EINVAL and a message naming the need and the limit.
 * The first call on each device sets that device up (it must be the current device): it looks
 * up the device address of the scratch array (cudaGetSymbolAddress), raises the forward-field
 * kernels' shared-memory limit and reads their occupancy.  Make that first call before any
 * stream capture.  Every call reuses the same array and leaves its contents behind (each call
 * clears the field accumulators it adds into): calls that overlap on the GPU (on different
 * streams, or from different host threads without ordering) race with each other and give
 * wrong results; serialise them. */
#define HOT_NOALLOC_SCRATCH_BYTES (16u << 20)
int hot_field_noalloc(int width, int height, double pitch_m, double wavelength_m, double focal_m, int M,
                      const double *xyz_m, const float *phi, int precision, double *V, double *eu,
                      void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* HOT_H */
