/*
 * sfseg.h -- C-ABI of the GB300 (sm_103a) SFSeg power-iteration library.
 *
 * SFSeg ("A 3D Convolutional Approach to Spectral Object Segmentation in
 * Space and Time", Burceanu & Leordeanu) segments a video by the principal
 * eigenvector of the pixel-level space-time adjacency matrix
 *
 *     M_ij = sp_i sp_j [1 - alpha (f_i - f_j)^2] G_ij,   sp = S^p     (Eq. 2)
 *
 * where G is a Gaussian over the space-time offset of voxels i and j,
 * truncated to a box of radii (rt, ry, rx).  M is never formed: one power
 * step x <- M x / ||M x|| (Eq. 4, Eq. 8) is evaluated as point-wise products
 * and three separable 3D Gaussian convolutions of the feature volume (Eq. 7).
 *
 * Conventions shared by every entry point
 *   - Volumes are dense, C-contiguous FP32 arrays [nf][h][w] (w fastest) in
 *     DEVICE memory, owned by the caller and only borrowed for the call.
 *   - All work is queued on the caller's CUDA stream (`stream` is a
 *     cudaStream_t; NULL = legacy default stream) and is asynchronous unless
 *     the function says it synchronises.
 *   - Every function returns an sfseg_status; nothing aborts or traps.
 *     sfseg_last_error() gives a message for the last failure on a context.
 *   - A context is not thread-safe: use one context per stream/thread.
 *   - The volume border is zero padding (neighbours outside the volume do
 *     not exist), which keeps M symmetric.  G is the per-axis Gaussian
 *     g(d) = exp(-d^2 / 2 sigma^2) with peak 1, not renormalised.  The
 *     neighbourhood of a voxel contains the voxel itself.
 *   - The operator applied is exactly M of Eq. 2 (Eq. 7 of the paper omits
 *     the overall factor alpha of Eq. 6; eigenvectors are unaffected), so the
 *     Rayleigh quotients reported are eigenvalue estimates of M.
 */
#ifndef SFSEG_H
#define SFSEG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfseg_ctx sfseg_ctx;   /* opaque; owns all device workspace */

typedef enum {
    SFSEG_OK = 0,
    SFSEG_EINVAL = 1,        /* invalid argument (message in sfseg_last_error) */
    SFSEG_ENOMEM = 2,        /* device or host allocation failed */
    SFSEG_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SFSEG_EZERONORM = 4,     /* ||M x|| = 0 at some step (x0 orthogonal to the support) */
    SFSEG_ENONFINITE = 5,    /* NaN/Inf in the inputs or in a norm */
    SFSEG_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
    SFSEG_EUNSUPPORTED = 7,  /* valid request the library does not implement */
    SFSEG_ESTATE = 8         /* call order (e.g. adjoint without a recorded forward) */
} sfseg_status;

typedef enum {
    SFSEG_F32 = 0,           /* FP32 storage of sp, f and the iterate */
    SFSEG_BF16 = 1,          /* BF16 storage, FP32 arithmetic, FP64 reductions */
    SFSEG_F16 = 2            /* FP16 storage (iterate stored scaled to RMS ~ 1) */
} sfseg_dtype;

/* sfseg_params.flags */
enum {
    SFSEG_S_IS_SP = 1,       /* d_s already holds S^p; p is ignored */
    SFSEG_NO_GRAPH = 2,      /* launch the iteration loop eagerly (no CUDA graph) */
    SFSEG_RECORD = 4,        /* record checkpoints during power_iterate for sfseg_adjoint */
    SFSEG_GENERIC = 8,       /* force the generic (any-radius) stencil kernel */
    SFSEG_FUSED = 16,        /* power_iterate runs all its steps in one launch (see below) */
    SFSEG_AUTOTUNE = 32,     /* power_iterate chooses its step path by timing (see below) */
    SFSEG_CLUSTER = 64       /* power_iterate runs in one thread-block cluster (see below) */
};

/* Step paths of sfseg_power_iterate(_batched) (the loop of Algorithm 1, one
 * power step = Eq. 7 + Eq. 8 per iteration):
 *   SFSEG_PATH_FAST     one launch per step of the specialised kernel (radii
 *                       (2,5,5) and (2,4,4)), replayed as a CUDA graph;
 *   SFSEG_PATH_GENERIC  one launch per step of the any-radius kernel;
 *   SFSEG_PATH_FUSED    all K steps in one cooperative launch: per step, the
 *                       y and x passes of every (frame, tile) into an FP32
 *                       scratch of three volumes (12 bytes per voxel, allocated
 *                       by the context on first use), a grid-wide barrier, the
 *                       t-pass, combine, reductions and norm update, a second
 *                       barrier.  Meant for small volumes (whose fixed per-step
 *                       launch cost dominates); one channel only; every
 *                       barrier wait gives up after 1 s with SFSEG_ETIMEOUT.
 *   SFSEG_PATH_CLUSTER  all K steps in one thread-block cluster of up to 16
 *                       CTAs that keeps the whole video (sp, f, the iterate,
 *                       the filtered channels) in shared memory: 16-column
 *                       tiles of all frames per CTA, the neighbours' halo
 *                       read through distributed shared memory, one cluster
 *                       barrier per step, the norm update repeated in every
 *                       CTA from the same records.  One video, one channel,
 *                       radii (3,3,3), (2,5,5) or (2,4,4), at most 16 tiles
 *                       whose frames fit one CTA's shared memory (e.g. a
 *                       64x64 video of 16 frames at (3,3,3)); no internal
 *                       scratch; nothing to time out (no spin-wait).
 * Default: FAST where the radii are specialised, else GENERIC; SFSEG_FUSED
 * selects FUSED (SFSEG_EUNSUPPORTED for nchan > 1, with SFSEG_RECORD, or on a
 * device without cooperative launch); SFSEG_CLUSTER selects CLUSTER
 * (SFSEG_EUNSUPPORTED where the video does not qualify or the device cannot
 * schedule the cluster).  SFSEG_AUTOTUNE: the first
 * power_iterate call on the context times each path it can run (and the fused
 * launch at three grid sizes, when the volume has at most 8 Mi voxels) on the
 * context's own features and x0, keeps the fastest and caches the choice per
 * (video shapes, radii, storage, channels, device) for the process.  That
 * first call synchronises the stream and must not be captured into a graph.
 * Paths differ only in floating-point summation order.  sfseg_rayleigh,
 * sfseg_apply, the binarised and the recorded iteration always run one launch
 * per step (the GENERIC kernel when that path was chosen). */
typedef enum {
    SFSEG_PATH_FAST = 0,
    SFSEG_PATH_GENERIC = 1,
    SFSEG_PATH_FUSED = 2,
    SFSEG_PATH_CLUSTER = 3
} sfseg_path;

typedef struct {
    int32_t nf, h, w;        /* volume: frames x rows x cols, all >= 1 */
    int32_t rt, ry, rx;      /* Gaussian radii (extent 2r+1), 0 <= r <= 16 */
    double sigma_t, sigma_y, sigma_x;  /* Gaussian widths, > 0 */
    double alpha;            /* weight of the pairwise feature term, >= 0 */
    double p;                /* unary exponent: sp = S^p, >= 0 */
    int32_t storage;         /* sfseg_dtype */
    int32_t flags;           /* SFSEG_* flags above; any other bit is rejected (EINVAL) */
    int32_t nchan;           /* pairwise feature channels C (Eq. 9), 1 <= C <= 4; d_f is [C][nf][h][w].
                              * M_ij = sp_i sp_j sum_c [1 - alpha (f_ci - f_cj)^2] G_ij, evaluated
                              * with C + 2 convolutions.  C > 1 runs on the any-radius step kernel;
                              * SFSEG_EUNSUPPORTED when its buffers for the given radii exceed
                              * shared memory, and for the adjoint and the no-alloc entry point
                              * (both C = 1 only). */
    int32_t ckpt_every;      /* adjoint checkpoint interval in steps (0 = 8) */
} sfseg_params;

/* Fill `prm` with defaults for an nf x h x w volume: radii (2, 5, 5),
 * sigma_t = 1.5, sigma_xy = 3, alpha = 1, p = 0.1 (the paper's unsupervised
 * setting, Sec. 5), FP32 storage, one channel. */
void sfseg_default_params(sfseg_params* prm, int32_t nf, int32_t h, int32_t w);

/* Create a context for one volume shape (Sec. 3 defines the operator; the
 * context allocates the device workspace: internal pitched copies of sp, f,
 * the two iterate buffers, reduction partials and the trace).
 * Errors: EINVAL (bad params), ENOMEM, ECUDA.  *out is NULL on failure. */
sfseg_status sfseg_create(const sfseg_params* prm, sfseg_ctx** out);

/* Create one context for a batch of independent videos of uneven shape that
 * share radii/sigmas/alpha/p/storage (`prm`'s nf/h/w are ignored).
 * dims: host array [n_videos][3] of (nf, h, w).  One persistent launch per
 * power step covers every video; each video keeps its own norm, Rayleigh
 * quotient and trace. */
sfseg_status sfseg_create_batched(const sfseg_params* prm, int32_t n_videos,
                                  const int32_t* dims, sfseg_ctx** out);

void sfseg_destroy(sfseg_ctx* ctx);   /* NULL is a no-op; synchronises the device */

/* Load the features into the context: sp = S^p (Eq. 1's unary term; S is
 * taken as-is with SFSEG_S_IS_SP) and f, converted to the storage type.
 * d_s: [nf][h][w] FP32; d_f: [nchan][nf][h][w] FP32 (device).  For a batched
 * context use sfseg_load_features_batched.  Errors: EINVAL, ECUDA. */
sfseg_status sfseg_load_features(sfseg_ctx* ctx, const float* d_s, const float* d_f,
                                 void* stream);

/* Power iteration (Eq. 4 + Eq. 8, Algorithm 1 without binarisation).
 *   d_s, d_f : features as in sfseg_load_features, or both NULL to reuse the
 *              features loaded last;
 *   d_x      : in: x0 (any scale, not all zero); out: x^K, unit L2 norm, FP32;
 *   n_iters  : K >= 0 power steps;
 *   tol      : 0 = exactly K steps; > 0 = stop after the first step k with
 *              rho_k / r_k < tol (r_k Rayleigh quotient, rho_k residual);
 *   iters_done: nullable host pointer; if given, the call synchronises the
 *              stream and stores the number of steps taken.
 * Step k computes y = M x^k, r_k = x^k.y / x^k.x^k, rho_k = ||y - r_k x^k|| /
 * ||x^k||, x^{k+1} = y / ||y||; r_k, rho_k and ||y|| go to the device trace.
 * Errors (reported by this call, or by the next synchronising call when the
 * device detects them): EINVAL, ECUDA, EZERONORM, ENONFINITE. */
sfseg_status sfseg_power_iterate(sfseg_ctx* ctx, const float* d_s, const float* d_f,
                                 float* d_x, int32_t n_iters, double tol,
                                 int32_t* iters_done, void* stream);

/* Batched form: host arrays of n_videos device pointers (x in/out per video). */
sfseg_status sfseg_load_features_batched(sfseg_ctx* ctx, const float* const* d_s,
                                         const float* const* d_f, void* stream);
sfseg_status sfseg_power_iterate_batched(sfseg_ctx* ctx, const float* const* d_s,
                                         const float* const* d_f, float* const* d_x,
                                         int32_t n_iters, void* stream);

/* Binarisation schedule (Alg. 1 Step 3 and Sec. 4 "Binarization - Spectral
 * vs Discrete space"): after a few power steps in the continuous space the
 * iterate is projected through a sigmoid and the next step starts from the
 * projection; after the last step a hard threshold gives the segmentation.
 * The paper gives no values; with u = x / max(x) (x >= 0 by
 * Perron-Frobenius):
 *   after step j (1-based), k0 <= j < n_iters:  x <- p / ||p||,
 *                                      p = 1 / (1 + exp(-beta (u - tau)));
 *   after the last step:              mask = [u >= theta]  (FP32 compare).
 * sfseg_default_binarize: k0 = 3, beta = 10, tau = 0.5, theta = 0.5. */
typedef struct {
    int32_t k0;              /* first step followed by a projection, >= 1 */
    int32_t reserved;        /* 0 */
    double beta;             /* sigmoid steepness, finite, >= 0 */
    double tau;              /* sigmoid centre on u, finite */
    double theta;            /* final threshold on u, finite */
} sfseg_binarize;

void sfseg_default_binarize(sfseg_binarize* b);

/* sfseg_power_iterate with the binarisation schedule (single-video
 * contexts; not with SFSEG_RECORD).  d_x: in x0, out the unit-L2 x^K (FP32);
 * d_mask: nullable device [nf][h][w] bytes (0/1), the hard segmentation of
 * x^K; the trace records r_k, rho_k, ||M x^k|| of every step (x^k being the
 * projected iterate where a projection preceded step k).  Runs step by step
 * (no CUDA graph).  Errors: as sfseg_power_iterate, and EINVAL for bad
 * schedule parameters or a batched context. */
sfseg_status sfseg_power_iterate_binarized(sfseg_ctx* ctx, const float* d_s, const float* d_f,
                                           float* d_x, int32_t n_iters, const sfseg_binarize* b,
                                           uint8_t* d_mask, void* stream);

/* Warnings about the loaded features (bits of *flags):
 *   SFSEG_WARN_NEGATIVE_M: alpha * (max f - min f)^2 > 1 for some video and
 *     channel, so the Taylor affinity 1 - alpha (f_i - f_j)^2 of Eq. 2 can be
 *     negative: M may have negative entries and the Perron-Frobenius argument
 *     of Sec. 3 (a non-negative principal eigenvector) no longer holds.  The
 *     computation itself is unaffected.
 * The range is that of the stored f (after the storage rounding), tracked by
 * the feature load.  Synchronises the device.  No features
 * loaded: *flags = 0.  Errors: EINVAL, ECUDA. */
#define SFSEG_WARN_NEGATIVE_M 1
sfseg_status sfseg_get_warnings(sfseg_ctx* ctx, int32_t* flags);

/* Test aid for failure detection (no counterpart in the paper).  The next
 * n_steps step launches of this context (specialised step kernel only) make
 * the first x-pass warp of every CTA wait on a barrier that nothing arrives
 * on; the wait gives up after its time limit (1 s), the CTA's other waits give
 * up at once, the loads in flight are drained, and the step reports
 * SFSEG_ETIMEOUT through the device status (sfseg_sync_status, or the next
 * synchronising call).  No GPU fault, trap or hang; the context stays usable.
 * Launches with a pending injection run without a CUDA graph.
 * Errors: EINVAL, EUNSUPPORTED (context not on the specialised kernel). */
sfseg_status sfseg_debug_inject_timeout(sfseg_ctx* ctx, int32_t n_steps);

/* Rayleigh quotient lambda = x.Mx / x.x (Eq. 3 read as a Rayleigh quotient)
 * and residual ||Mx - lambda x|| / ||x|| of d_x ([nf][h][w] FP32, device)
 * with the features loaded last.  Synchronises the stream.
 * Errors: EINVAL, ESTATE (no features loaded), ECUDA, ENONFINITE. */
sfseg_status sfseg_rayleigh(sfseg_ctx* ctx, const float* d_x, double* lambda,
                            double* residual, void* stream);

/* One unnormalised application y = M x (Eq. 4 / Eq. 7) with the features
 * loaded last; d_x, d_y: [nf][h][w] FP32 device, may not alias.  Stored
 * operands go through the storage type.  Errors: EINVAL, ESTATE, ECUDA. */
sfseg_status sfseg_apply(sfseg_ctx* ctx, const float* d_x, float* d_y, void* stream);

/* Copy the per-step trace of the last power_iterate of video `video`
 * (0 for a single-video context) to host arrays of capacity `cap`:
 * Rayleigh quotient r_k, residual rho_k, norm ||M x^k||.  Any array may be
 * NULL.  Synchronises the context's last stream.  Returns the number of
 * steps recorded, or -1 on error. */
int32_t sfseg_get_trace(sfseg_ctx* ctx, int32_t video, double* rayleigh,
                        double* residual, double* norms, int32_t cap);

/* Reverse mode of the last power_iterate (which must have run with
 * SFSEG_RECORD): given d_gx = dL/dx^K ([nf][h][w] FP32, device), writes
 *   d_gsp = dL/dsp, d_gf = dL/df (nchan = 1), d_gx0 = dL/dx0
 * (each [nf][h][w] FP32 device, any may be NULL).  M is symmetric, so each
 * backward step is the same stencil plus the normalisation Jacobian
 * u = (g - x (x.g)) / ||y||.  Forward iterates are recomputed from
 * checkpoints kept every `ckpt_every` steps.  Errors: ESTATE, EINVAL, ECUDA. */
sfseg_status sfseg_adjoint(sfseg_ctx* ctx, const float* d_gx, float* d_gsp,
                           float* d_gf, float* d_gx0, void* stream);

/* Wait for the context's last stream and return the device-side status of
 * the last power_iterate/rayleigh/apply: OK, EZERONORM or ENONFINITE. */
sfseg_status sfseg_sync_status(sfseg_ctx* ctx);

/* Power iteration without any device allocation, for callers that cannot
 * call cudaMalloc: code running inside a region captured into a larger CUDA
 * graph, real-time paths with a fixed memory budget (cudaMalloc can stall
 * every stream and can fail under pressure), plug-ins whose host framework
 * owns all device memory.  The paper has no counterpart: this is a packaging
 * of the same computation as sfseg_power_iterate (generic step kernel, exactly
 * n_iters steps, x0 = d_x in, unit-norm x^K out, FP32 [nf][h][w] device
 * buffers owned by the caller).  Its workspace is one fixed 32 MiB device
 * array inside the library, held by every GPU that loads the library until
 * the process exits; volumes needing more (about 2 million voxels in FP32
 * storage) are rejected with SFSEG_EINVAL before any launch.  All calls share
 * that array, so calls that overlap on the GPU race: serialise them on one
 * stream.  The first call on a device looks up the array's address (and the
 * driver may load the library's device code then): make it before any stream
 * capture.  d_trace: nullable device array [min(n_iters,1024)][3] receiving
 * (r_k, rho_k, ||M x^k||).  Device-side statuses (zero norm, non-finite) are
 * not reported; errors of the call itself are, with sfseg_last_error(NULL). */
sfseg_status sfseg_power_iterate_noalloc(const sfseg_params* prm, const float* d_s,
                                         const float* d_f, float* d_x, int32_t n_iters,
                                         double* d_trace, void* stream);

/* ---- One video split along t over several GPUs (one process per GPU).
 * The operator is local (Eq. 7: a separable Gaussian of radii (rt, ry, rx),
 * and "highly parallelizable", Sec. 4), so a video of nf frames cuts into
 * contiguous slabs of frames, one per rank.  A rank owning frames [a, b)
 * keeps the slab [a - rt, b + rt) clipped to the video: its own frames plus
 * up to rt halo frames on each side.  Per power step each rank computes M x
 * on its own frames; the step's four FP64 sums (z.z, x.z, x.x, |z - s x|^2,
 * the inputs of Eq. 3 and Eq. 8) are summed over all ranks (an all-reduce the
 * caller runs, e.g. NCCL) and applied on every rank, so every rank holds the
 * same norm, Rayleigh quotient and trace; then neighbours exchange rt frames
 * of the new stored iterate (the caller moves the bytes, e.g. NCCL send/recv
 * or a peer copy).  One step on R ranks:
 *     sfseg_slab_step(ctx, d_part)          partial sums of the own frames
 *     all-reduce (sum) d_part -> d_sum      4 doubles, over the ranks
 *     sfseg_slab_finish_step(ctx, d_sum)    norm, Rayleigh quotient, residual
 *     halo exchange                          pack (dir 0) own edge frames into
 *                                            send buffers, the caller sends them,
 *                                            unpack (dir 1) received frames
 * The start: sfseg_load_features on the slab's frames, sfseg_slab_start
 * (partial sum of x0^2 of the own frames), all-reduce, sfseg_slab_set_norm.
 * The end: sfseg_slab_output writes the own frames of the unit-norm x^K.
 * Fixed step count (no early stop), one video per context, the per-step
 * kernels.  All device pointers; all calls are stream-ordered, none
 * synchronises.  With one rank (a = 0, b = nf) this is sfseg_power_iterate
 * split into its steps. */

/* prm: the slab's shape (nf = its frame count including the halo frames) and
 * the video's parameters; own frames [own_lo, own_hi) of the slab; the halo
 * on either side has at most rt frames, and a slab with a neighbour owns at
 * least rt frames (a halo then comes from one neighbour); video_voxels: the
 * voxel count of the whole video (it sets the storage gain, the same on
 * every rank).  Errors: EINVAL, EUNSUPPORTED (SFSEG_FUSED, SFSEG_AUTOTUNE,
 * SFSEG_RECORD, SFSEG_CLUSTER), ENOMEM, ECUDA. */
sfseg_status sfseg_create_slab(const sfseg_params* prm, int32_t own_lo, int32_t own_hi,
                               int64_t video_voxels, sfseg_ctx** out);

/* Store x0 (d_x0: the slab's [nf][h][w] FP32 frames, halo frames included)
 * and write the sum of x0^2 over the own frames to d_part[0] (device double).
 * n_iters: the number of steps that will follow (trace capacity; may
 * synchronise the device to grow it).  Errors: EINVAL, ESTATE, ECUDA. */
sfseg_status sfseg_slab_start(sfseg_ctx* ctx, const float* d_x0, int32_t n_iters, double* d_part,
                              void* stream);

/* Start the iteration from d_sumsq[0] = the sum of x0^2 over the whole video
 * (device double, the all-reduced sfseg_slab_start partials).  A zero or
 * non-finite sum sets SFSEG_EZERONORM / SFSEG_ENONFINITE on the device
 * (sfseg_sync_status).  Errors: EINVAL, ESTATE, ECUDA. */
sfseg_status sfseg_slab_set_norm(sfseg_ctx* ctx, const double* d_sumsq, void* stream);

/* One power step on the own frames: y = M x (Eq. 7) stored for the next step,
 * and the four FP64 sums of the own frames written to d_part[0..3] (device):
 * z.z, x.z, x.x and |z - s x|^2 (z the stored step output, x the scaled
 * input, s the previous Rayleigh quotient times the gain).  d_x_final
 * (nullable): this is the last step, and its output goes in FP32 to d_x_final
 * (the own frames, [own_hi - own_lo][h][w], device) instead of the storage
 * type; pass the same buffer to sfseg_slab_output.  At most n_iters steps per
 * sfseg_slab_start.  Errors: EINVAL, ESTATE, ECUDA. */
sfseg_status sfseg_slab_step(sfseg_ctx* ctx, double* d_part, float* d_x_final, void* stream);

/* Apply the step's sums over all ranks (d_sums[0..3], device): Rayleigh
 * quotient, residual and norm into the trace, the next scale and gain
 * (Eq. 3, Eq. 8).  Every rank passes the same sums, so every rank holds the
 * same scalars.  Errors: EINVAL, ESTATE, ECUDA. */
sfseg_status sfseg_slab_finish_step(sfseg_ctx* ctx, const double* d_sums, void* stream);

/* Halo exchange of the stored iterate the next step reads, in the storage
 * type and the library's row layout: frames of [h][pitch] elements, pitch = w
 * rounded up to 8 (pad columns zero).  side 0 = the low-frame end, 1 = the
 * high end; dir 0 packs the rt own frames at that end into d_buf (for the
 * neighbour on that side), dir 1 unpacks d_buf into the halo frames at that
 * end (received from that neighbour).  sfseg_slab_halo_bytes gives the byte
 * count of (side, dir), or -1 for a bad argument; 0 means nothing to move.
 * Errors: EINVAL, ESTATE, ECUDA. */
sfseg_status sfseg_slab_halo(sfseg_ctx* ctx, int32_t side, int32_t dir, void* d_buf, void* stream);
int64_t sfseg_slab_halo_bytes(const sfseg_ctx* ctx, int32_t side, int32_t dir);

/* The own frames of the unit-norm x^K (FP32, [own_hi - own_lo][h][w],
 * device) after the last finish_step: scaled in place when d_x is the buffer
 * the last sfseg_slab_step wrote (FP32 throughout), else read from the stored
 * iterate (rounded to the storage type).  Errors: EINVAL, ESTATE, ECUDA. */
sfseg_status sfseg_slab_output(sfseg_ctx* ctx, float* d_x, void* stream);

/* ---- Bounds-checked build (no counterpart in the paper): the same library
 * compiled with SFSEG_DEBUG (libsfseg_debug.so) checks, inside the kernels,
 * every work item's range (video, frames, tile origin), the TMA box
 * coordinates, the partials and plan slots and the offsets of the stores into
 * the internal pitched workspace and the caller's buffers.  A failed check is
 * counted, the first one's code (1 item range, 2 TMA coordinate, 3 store
 * offset, 4 slot, 5 fused unit) and two values are kept, and the access is
 * skipped: no trap.  sfseg_debug_build returns 1 in that build, 0 otherwise;
 * sfseg_debug_status synchronises the device and returns the violations
 * since its last call (always 0 in the normal build), clearing them. */
int32_t sfseg_debug_build(void);
sfseg_status sfseg_debug_status(int64_t* count, int32_t* code, int64_t* a, int64_t* b);

/* Message of the last failure on ctx (ctx may be NULL: last create failure). */
const char* sfseg_last_error(const sfseg_ctx* ctx);

/* Static name of a status code. */
const char* sfseg_status_string(sfseg_status st);

/* Host-only introspection of the work decomposition of the specialised step
 * kernel (no device needed).  Units are the output frames of every (video,
 * 112x12 tile); n_ctas = min(n_sms, units/8) persistent CTAs.  Per video,
 * while at least n_ctas of its tiles remain, each round gives every CTA one
 * whole tile (CTA c gets that video's tiles c, c + n_ctas, ...); the units of
 * every video's last < n_ctas tiles are laid end to end and split into n_ctas
 * equal contiguous ranges.  dims: [n_videos][3] (nf, h, w).  Writes up
 * to seg_cap segments as [video, x0, y0, t0, t1) rows into `segments` and up
 * to cta_cap entries of `cta_begin` (CTA c owns segments [cta_begin[c],
 * cta_begin[c+1])); either may be NULL.  Returns the number of segments, or
 * -1 (EINVAL, message in sfseg_last_error(NULL)).  The number of CTAs is the
 * number of cta_begin entries minus one (at most n_sms). */
int32_t sfseg_plan_segments(int32_t n_videos, const int32_t* dims, int32_t n_sms,
                            int32_t* segments, int32_t seg_cap, int32_t* cta_begin,
                            int32_t cta_cap);

/* Number of kernel launches this context issued so far (for accounting). */
int64_t sfseg_launch_count(const sfseg_ctx* ctx);

/* The step path power_iterate uses (sfseg_path; with SFSEG_AUTOTUNE, the one
 * chosen by the first call), the CTA count of the fused or cluster launch (0
 * for the per-step paths) and, nullable, us_per_step[4]: the microseconds per
 * step the autotuner measured for each path (index = sfseg_path; -1 where not
 * timed).
 * No device access.  Errors: EINVAL. */
sfseg_status sfseg_get_path(const sfseg_ctx* ctx, int32_t* path, int32_t* fused_ctas,
                            double* us_per_step);

#ifdef __cplusplus
}
#endif

#endif /* SFSEG_H */
