/*
 * spect.h -- C ABI of the GB300 (sm_103a) SPECT projector library.
 *
 * The operator is the rotation-based SPECT system model of Li, Dewaraja &
 * Fessler, "Training end-to-end unrolled iterative neural networks for SPECT
 * image reconstruction" (arXiv 2301.09710), Section II-A:
 *
 *   A  (Algorithm 1): for every view l, rotate the image x and the
 *      attenuation map mu about the axial (z) axis by theta_l with bilinear
 *      interpolation and zero padding; weight the rotated image by the
 *      accumulated attenuation of Eq. (1); blur every depth plane j with
 *      that depth's PSF p(:,:,j,l) (convolution, replicate padding in i and
 *      k); sum over depth.
 *   A' (Algorithm 2): the exact transpose of A, satisfying Eq. (2)
 *      <A x, y> = <x, A' y> up to FP32 rounding.
 *   EM (Eqs. (7)-(8) with beta = 0): x <- x * A'(y / (A x + rbar)) / A'1.
 *
 * All arithmetic is FP32 on the GPU.  Every entry point takes device
 * pointers unless stated otherwise; no entry point allocates on the caller's
 * behalf except spect_plan_create (the plan's own state).
 *
 * ---------------------------------------------------------------- layouts
 * 0-based indices (the paper's are 1-based).  All arrays are dense FP32 with
 * the first index fastest:
 *   image  x, mu : nx*ny*nz,            x(i,j,k)   at i + nx*(j + ny*k)
 *   projections v: nx*nz*nview,         v(i,k,l)   at i + nx*(k + nz*l)
 *   full PSF     : px*pz*ny*nview_psf,  p(a,b,j,l) at a + px*(b + pz*(j + ny*l))
 *   PSF factors  : fx px*ny*nview_psf at a + px*(j + ny*l),
 *                  fz pz*ny*nview_psf at b + pz*(j + ny*l),
 *                  meaning p(a,b,j,l) = fx(a,j,l) * fz(b,j,l).
 * Plane j = ny-1 of the rotated image is the one nearest the detector
 * (Eq. (1)); the PSF depth index j refers to that rotated frame.
 *
 * ---------------------------------------------------------------- geometry
 * Rotation centre c = (nx-1)/2.  Output pixel (i,j) of the rotated slice
 * samples the input at xs = c + cos(t)(i-c) + sin(t)(j-c),
 * ys = c - sin(t)(i-c) + cos(t)(j-c) (the content turns by +t); cosine and
 * sine are exact at multiples of pi/2.  The PSF centre is ((px-1)/2,
 * (pz-1)/2); px and pz must be odd.  Default angles (angles == NULL) are
 * theta_l = 2*pi*l/nview, the paper's 2*pi*(l-1)/nview with 1-based l.
 *
 * ---------------------------------------------------------------- errors
 * Every entry point returns a spect_status.  Argument errors (SPECT_EINVAL)
 * are detected on the host before any work is queued and leave no side
 * effect.  Work is queued on the given stream and is asynchronous; launch
 * failures are reported as SPECT_ECUDA.  spect_last_error() returns a
 * thread-local, human-readable message for the last non-OK status.
 * A plan is not safe for concurrent use from several streams or threads:
 * calls on one plan must be ordered (same stream, or synchronised).
 * Input and output buffers of one call must not overlap.
 */
#ifndef SPECT_H
#define SPECT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* spect_stream;

typedef struct spect_plan_s* spect_plan;

typedef enum {
    SPECT_OK = 0,
    SPECT_EINVAL = 1,       /* bad argument: size, pointer, alignment, flag  */
    SPECT_ENOMEM = 2,       /* device allocation for the plan failed         */
    SPECT_ECUDA = 3,        /* a CUDA call or kernel launch failed           */
    SPECT_ETIMEOUT = 4,     /* reserved: a bounded device wait gave up       */
    SPECT_EUNSUPPORTED = 5  /* valid request this build cannot serve         */
} spect_status;

/* Plan flags. */
enum {
    SPECT_PLAN_DEFAULT = 0u,
    /* Use the separable factors when both a full PSF and factors are given
     * (otherwise the full PSF wins).  Ignored when only one form is given. */
    SPECT_PLAN_PREFER_SEPARABLE = 1u << 0,
    /* Keep device memory O(image + projections): recompute the attenuation
     * per view and stream views through a small work slab, instead of
     * caching the attenuation factors of every view (nview * nx*ny*nz floats)
     * and using the fused kernels. */
    SPECT_PLAN_LOW_MEMORY = 1u << 1,
    /* Rotate the image and the attenuation map by three 1D linear
     * interpolation passes instead of bilinear interpolation (Section II-A
     * implements both): theta = q*pi/2 + phi, q the nearest integer and
     * phi in [-pi/4, pi/4]; the exact quarter turn q, then pull-backs along
     * x at i + tan(phi/2)(j-c), along y at j - sin(phi)(i-c) and along x at
     * i + tan(phi/2)(j-c), each with zero padding, c = (nx-1)/2.  A' is the
     * exact transpose (the passes' transposes in reverse order).  Fused
     * plans only: with SPECT_PLAN_LOW_MEMORY, or when the fused kernels do
     * not fit the geometry, spect_plan_create returns SPECT_EUNSUPPORTED.
     * The three passes run as one eight-tap gather per output inside the
     * rotation kernel (table: nview*ny*16nx floats) and as eight-entry
     * adjacency lists in A'. */
    SPECT_PLAN_ROTATION_3PASS = 1u << 2,
    /* Fused kernels with the attenuation of Eq. (1) recomputed in every
     * projection instead of cached for every view: the views go through the
     * fused kernels in chunks, and before each chunk's rotation (A) or blur
     * adjoint (A') the factors of that chunk's views are computed from the
     * rotated mu-map (the same warp-scan kernel that fills the cache, so A,
     * A' and the EM update are bitwise those of a caching plan).  Device
     * memory then grows with the chunk (work slab and factors of the chunk's
     * views, 512 MiB by default) rather than with nview * nx*ny*nz.  Bilinear
     * rotation on the fused kernels only: with SPECT_PLAN_LOW_MEMORY or
     * SPECT_PLAN_ROTATION_3PASS, or when the fused kernels do not fit the
     * geometry, spect_plan_create returns SPECT_EUNSUPPORTED. */
    SPECT_PLAN_RECOMPUTE_ATTENUATION = 1u << 3
};

/*
 * spect_plan_create -- build the operator A for one geometry (Algorithm 1
 * inputs: attenuation map, 4D PSF, voxel size; Section II-A).
 *
 *   out        receives the plan handle (host pointer, must not be NULL).
 *   nx,ny,nz   image size; nx == ny is required (rotation in the x-y plane);
 *              2 <= nx <= 1024, 1 <= nz <= 4096.
 *   nview      number of views, 1..4096.
 *   mu         device, nx*ny*nz FP32 attenuation coefficients (per unit of
 *              dy), non-negative; may be NULL for no attenuation.
 *   dy         voxel size along the depth direction (Eq. (1) Delta_y), >= 0.
 *   psf        device, full PSF stack (layout above), or NULL.
 *   psf_fx,
 *   psf_fz     device, separable factors (layout above), or both NULL.
 *              At least one of psf / (psf_fx, psf_fz) must be given.
 *   px, pz     PSF size, odd, 1..127.
 *   nview_psf  nview (view-dependent PSF, non-circular orbits) or 1
 *              (the same PSF stack for every view).
 *   angles     HOST, nview angles in radians, or NULL for the defaults.
 *   flags      SPECT_PLAN_* bits.
 *   stream     stream used for the plan's set-up work.
 *
 * The plan copies mu and the PSF into its own device memory and builds its
 * rotation adjacency tables; the call synchronises `stream` before it
 * returns, so the caller may free or reuse its inputs afterwards.
 * Errors: SPECT_EINVAL (sizes, NULL out, misaligned or missing inputs),
 * SPECT_ENOMEM, SPECT_ECUDA.  On error *out is set to NULL.
 */
spect_status spect_plan_create(spect_plan* out, int nx, int ny, int nz, int nview,
                               const float* mu, float dy,
                               const float* psf, const float* psf_fx, const float* psf_fz,
                               int px, int pz, int nview_psf,
                               const double* angles, unsigned flags, spect_stream stream);

/*
 * spect_forward -- v = A x (Algorithm 1).
 *   x  device, nx*ny*nz (image layout), read only.
 *   v  device, nx*nz*nview (projection layout), overwritten.
 * Both 16-byte aligned.  Errors: SPECT_EINVAL (NULL plan/pointer,
 * misalignment), SPECT_ECUDA.
 */
spect_status spect_forward(spect_plan plan, const float* x, float* v, spect_stream stream);

/*
 * spect_back -- x = A' v (Algorithm 2), the exact transpose of
 * spect_forward (Eq. (2)); the adjoint of the rotation is the transpose of
 * the bilinear interpolation, not a rotation by -theta (Section II-A).
 *   v  device, nx*nz*nview, read only.
 *   x  device, nx*ny*nz, overwritten (not accumulated).
 * Errors as spect_forward.
 */
spect_status spect_back(spect_plan plan, const float* v, float* x, spect_stream stream);

/*
 * spect_em_step -- niter MLEM updates (Eqs. (7)-(8) with beta = 0):
 *   x <- x * A'(y / (A x + rbar)) / A'1, in place.
 *   x     device, nx*ny*nz, non-negative; updated in place.
 *   y     device, nx*nz*nview measured counts, read only.
 *   rbar  device, nx*nz*nview background means, or NULL for zero.
 *   niter >= 0 (0 is a no-op).
 * Guards (not stated in the paper): where A x + rbar <= 0 the ratio is 0;
 * where A'1 <= 0 the voxel is set to 0.  The sensitivity A'1 is computed on
 * the first call and cached in the plan.
 * Errors as spect_forward; SPECT_EINVAL for niter < 0.
 */
spect_status spect_em_step(spect_plan plan, float* x, const float* y, const float* rbar,
                           int niter, spect_stream stream);

/*
 * spect_em_step_reg -- niter inner iterations of the regularised EM update,
 * Eqs. (7)-(8):  x <- (-d + sqrt(d^2 + 4 beta x e)) / (2 beta),
 * d = A'1 - beta u, e = A'(y / (A x + rbar)); the non-negative root of the EM
 * surrogate of Eq. (6) with the penalty (beta/2)||x - u||^2.  beta = 0 is the
 * MLEM update of spect_em_step.
 *   u     device, nx*ny*nz regulariser target (u = g_theta(x_k) of Eq. (6)),
 *         read only; may be NULL when beta == 0.
 *   beta  >= 0.
 * The root is evaluated in the cancellation-free form for the sign of d.
 * Errors as spect_em_step; SPECT_EINVAL for beta < 0 or u missing.
 */
spect_status spect_em_step_reg(spect_plan plan, float* x, const float* y, const float* rbar, const float* u,
                               float beta, int niter, spect_stream stream);

/*
 * The element-wise steps of one EM iteration, Eqs. (7)-(8), as separate calls
 * with their gradients, for training through an unrolled reconstruction
 * (Algorithm 3, Section II-B): with spect_forward (A) and spect_back (A') they
 * make up the update x+ = F(x, A'(y / (A x + rbar)), u) that spect_em_step_reg
 * runs fused, in a form an automatic-differentiation system can chain.  All
 * pointers are device, n elements each (rbar and u may be NULL as stated), FP32;
 * work is queued on `stream`.  Element-wise, so any layout works as long as the
 * arrays of one call share it.  Errors: SPECT_EINVAL (NULL pointers, beta < 0 or
 * not finite, u missing with beta > 0), SPECT_ECUDA.
 *
 * spect_em_ratio: ratio = y / (ybar + rbar), 0 where ybar + rbar <= 0 (the
 *   guard of spect_em_step); ybar is A x.
 * spect_em_ratio_backward: g_ybar = dL/dybar from g_ratio = dL/dratio:
 *   g_ybar = -g_ratio * ratio / (ybar + rbar), 0 where the guard applies.
 * spect_em_update: out = the update of spect_em_step_reg from x, e = A'(ratio),
 *   s = A'1 and u (beta = 0: x e / s, u unused); the same arithmetic as the
 *   fused step.
 * spect_em_update_backward: from g_out = dL/dout, g_x = g_out e / q,
 *   g_e = g_out x / q and g_u = g_out beta out / q, q = sqrt(d^2 + 4 beta x e),
 *   d = s - beta u (q = s at beta = 0): the implicit derivative of
 *   beta out^2 + d out - x e = 0; all three are 0 where the forward guard set
 *   out to 0.  Any of g_x, g_e, g_u may be NULL (not computed); g_u is filled
 *   with 0 when beta = 0.
 */
spect_status spect_em_ratio(size_t n, const float* ybar, const float* y, const float* rbar, float* ratio,
                            spect_stream stream);
spect_status spect_em_ratio_backward(size_t n, const float* ybar, const float* y, const float* rbar,
                                     const float* g_ratio, float* g_ybar, spect_stream stream);
spect_status spect_em_update(size_t n, const float* x, const float* e, const float* s, const float* u, float beta,
                             float* out, spect_stream stream);
spect_status spect_em_update_backward(size_t n, const float* x, const float* e, const float* s, const float* u,
                                      float beta, const float* g_out, float* g_x, float* g_e, float* g_u,
                                      spect_stream stream);

/*
 * spect_sensitivity -- copy the plan's sensitivity s = A'1 (the d(0) term
 * of Eq. (8)) into s (device, nx*ny*nz).  Computes and caches it first if
 * needed.  Errors as spect_forward.
 */
spect_status spect_sensitivity(spect_plan plan, float* s, spect_stream stream);

/*
 * spect_plan_info -- describe a plan (host out-pointers; any may be NULL):
 *   separable    1 when the separable-factor kernels are used, else 0.
 *   fused        1 when the fused kernels with the cached attenuation serve
 *                the plan, 0 for the low-memory kernels.
 *   view_chunk   views processed per pass through the work slab.
 *   device_bytes device memory held by the plan (state + work slab).
 */
spect_status spect_plan_info(spect_plan plan, int* separable, int* fused, int* view_chunk, size_t* device_bytes);

/*
 * spect_plan_bytes -- an upper bound of the device memory (bytes, host
 * out-pointer) that spect_plan_create would allocate for this geometry on the
 * current device, without allocating anything: for admission control by a
 * server that holds many plans (the paper has no counterpart).  Arguments as
 * spect_plan_create; separable = 1 when the plan will use the separable
 * factors (psf_fx/psf_fz given, and either no full psf or
 * SPECT_PLAN_PREFER_SEPARABLE).  spect_plan_info reports the exact figure of a
 * created plan, which never exceeds this bound.
 * Errors: SPECT_EINVAL (arguments as spect_plan_create), SPECT_ECUDA.
 */
spect_status spect_plan_bytes(int nx, int ny, int nz, int nview, int px, int pz, int nview_psf, int separable,
                              unsigned flags, size_t* bytes);

/*
 * spect_fp32_peak -- measure the FP32 fused multiply-add throughput of the
 * current device with a register-resident dependent-chain kernel (no memory
 * traffic): tflops_ffma for scalar fmaf, tflops_ffma2 for the packed
 * two-lane form (__ffma2_rn); FLOP = 2 per lane FMA.  Host out-pointers;
 * synchronises `stream`.  A measurement aid for roofline reporting (the
 * paper has no counterpart).
 */
spect_status spect_fp32_peak(double* tflops_ffma, double* tflops_ffma2, spect_stream stream);

/* Kernel classes for spect_profile_read(). */
enum {
    SPECT_K_ROTATE_ATTEN = 0, /* rotate x, mu; Eq. (1) attenuation            */
    SPECT_K_CONV_FWD = 1,     /* PSF blur + depth sum (+ EM ratio)            */
    SPECT_K_CONV_ADJ = 2,     /* PSF blur adjoint + attenuation               */
    SPECT_K_ROTATE_ADJ = 3,   /* adjoint rotation + view sum (+ EM update)    */
    SPECT_K_OTHER = 4,        /* fills and set-up work                        */
    SPECT_K_COUNT = 5
};

/*
 * spect_profile_enable -- when enable != 0, every later kernel launch of the
 * plan is bracketed by a pair of CUDA events recorded on the launch stream,
 * so its device duration can be read back.  Costs two event records per
 * launch; off by default.  Launch counting is always on.
 */
spect_status spect_profile_enable(spect_plan plan, int enable);

/*
 * spect_profile_read -- per kernel class (SPECT_K_*), the number of kernel
 * launches since the last reset (launches[SPECT_K_COUNT], host) and the summed
 * device milliseconds of the launches made while profiling was enabled
 * (ms[SPECT_K_COUNT], host; synchronises on the recorded events).  Either
 * pointer may be NULL.  With reset != 0 the counters restart from zero.
 */
spect_status spect_profile_read(spect_plan plan, long long* launches, double* ms, int reset);

/*
 * spect_plan_check -- synchronise the device and report whether any kernel
 * of the plan gave up a bounded wait since the last check: SPECT_ETIMEOUT if
 * one did (the outputs of the affected calls are not valid), else SPECT_OK.
 * The plan's error word is cleared.  The fused kernels wait on their own
 * bulk copies with a limit of about one second instead of blocking forever.
 */
spect_status spect_plan_check(spect_plan plan);

/*
 * spect_plan_check_stream -- as spect_plan_check, but synchronises only
 * `stream` (the caller has put all of the plan's work on it), so work of
 * other plans on other streams keeps running.  For servers that interleave
 * many plans (the paper has no counterpart).
 */
spect_status spect_plan_check_stream(spect_plan plan, spect_stream stream);

/*
 * spect_plan_selftest_timeout -- exercise the failure path of the bounded
 * device waits without any fault: one thread waits, with the bounded mbarrier
 * wait the fused kernels use on their bulk copies but a limit of spin_clocks
 * SM clocks (0 .. 2^31), on a barrier that nothing completes; the wait runs out
 * and SPECT_ETIMEOUT is recorded in the plan's error word, which the next
 * spect_plan_check reports (and clears).  The plan stays usable.  A test aid
 * (the paper has no counterpart).  Errors: SPECT_EINVAL, SPECT_ECUDA.
 */
spect_status spect_plan_selftest_timeout(spect_plan plan, long long spin_clocks, spect_stream stream);

/* spect_plan_destroy -- release the plan; NULL is accepted and returns OK.
 * Waits for the plan's outstanding work on the device before freeing. */
spect_status spect_plan_destroy(spect_plan plan);

/*
 * spect_plan_release -- release the plan in stream order: its device memory
 * is returned after the work already enqueued on `stream`, and the call does
 * not wait for the device.  The caller guarantees that no work of the plan
 * is pending on any other stream.  The handle is invalid afterwards; NULL is
 * accepted.  Plan memory comes from the device's stream-ordered allocator
 * (cudaMallocAsync on the creation stream) where the device supports it, so
 * creating and releasing plans never synchronises the whole device (the paper
 * has no counterpart).
 */
spect_status spect_plan_release(spect_plan plan, spect_stream stream);

/*
 * Launch-shape tuning of the fused kernels (the paper has no counterpart).
 * fused_J / adj_J: depth planes per block of the forward / adjoint blur
 * kernels (1..32); tiles: column tiles per plane (>= 1; the kernels use the
 * nearest count that divides the plane into whole 16-column runs).  The plan
 * grows its work slab and partial-sum buffer (and, for a plan made with
 * SPECT_PLAN_RECOMPUTE_ATTENUATION, its buffer of one view chunk's
 * attenuation factors) in stream order on `stream` when the shape needs more
 * room.  Results stay within the FP32 tolerance of the
 * oracle for every shape; A' is bitwise independent of the shape, A x depends
 * on fused_J only through the grouping of its depth sum.
 * Errors: SPECT_EINVAL, SPECT_EUNSUPPORTED (low-memory plan, or the shape
 * does not fit shared memory), SPECT_ENOMEM, SPECT_ECUDA.
 */
spect_status spect_plan_set_tuning(spect_plan plan, int fused_J, int adj_J, int tiles, spect_stream stream);
spect_status spect_plan_get_tuning(spect_plan plan, int* fused_J, int* adj_J, int* tiles);

/*
 * spect_plan_autotune -- time the fused kernels' candidate launch shapes
 * (tiles x fused_J for A, tiles x adj_J for A') on this device with CUDA
 * events on `stream` and keep the fastest; the choice is cached per geometry
 * and device for the life of the process, so later plans of the same shape
 * are set without timing.  Overwrites nothing the caller owns; synchronises
 * `stream`.  Low-memory plans are left as they are (SPECT_OK).
 */
spect_status spect_plan_autotune(spect_plan plan, spect_stream stream);

/*
 * Batches: many plans of different sizes, view counts and PSF widths run
 * their EM iterations as ONE CUDA graph launch (the paper has no
 * counterpart).  By default spect_batch_em_step captures, per plan, the
 * kernel sequence spect_em_step would launch (niter iterations, transposes
 * included), each plan on its own branch of the graph, so the plans' kernels
 * overlap on the device.  The executable graph is cached and replayed while
 * niter, the pointer arrays' contents and the mode stay the same (a plan must
 * not be retuned while it is in a batch).
 *   plans        n distinct plans; the batch borrows them (destroy the batch
 *                before its plans, and do not use the plans concurrently with
 *                the batch).
 *   x, y, rbar   HOST arrays of n DEVICE pointers (as spect_em_step; rbar may
 *                be NULL, or hold NULL entries).
 * Each plan's result is bitwise what spect_em_step gives for it alone.
 * spect_batch_set_grouped: with branches >= 1, and when every plan runs the
 * fused separable-PSF kernels (the default for separable PSFs up to 37 taps),
 * each stage of an EM iteration (rotation, blur + depth sums, reduce + ratio,
 * blur adjoint, adjoint rotation + update) is instead ONE grouped launch per
 * kernel variant over the blocks of every plan of a branch (at most 24 plans
 * per launch; the plans split into `branches` branches of about equal work),
 * so an iteration takes a handful of launches per branch whatever the number
 * of plans; each plan still gets bitwise its own values.  For the grouped
 * launches a plan processes every view in one pass: its work slab grows
 * (stream-ordered) to hold every view, and stays so after the batch.  0 (the
 * default) restores a graph branch per plan.  Errors: SPECT_EINVAL.
 * spect_batch_info: plans in the batch and kernels per graph launch (after the
 * first spect_batch_em_step).
 * Errors: SPECT_EINVAL, SPECT_ECUDA (capture or graph failures).
 */
typedef struct spect_batch_s* spect_batch;
spect_status spect_batch_create(spect_batch* out, const spect_plan* plans, int n);
spect_status spect_batch_em_step(spect_batch batch, float* const* x, const float* const* y, const float* const* rbar,
                                 int niter, spect_stream stream);
spect_status spect_batch_set_grouped(spect_batch batch, int branches);
spect_status spect_batch_info(spect_batch batch, int* n_plans, long long* kernels_per_launch);
spect_status spect_batch_destroy(spect_batch batch);

/*
 * spect_forward_static -- v = A x without any device allocation.
 *
 * For callers that cannot allocate device memory: hosts whose device memory
 * is reserved up front and may not grow while they run, and plug-in
 * environments that hand out device buffers but own the allocator, so a
 * library may not take memory behind their back.  No plan is needed: the call takes
 * the same inputs as spect_plan_create (separable PSF factors only) plus x and
 * v, and uses a work slab and rotation constants held in fixed-size static
 * device arrays of the library (the paper has no counterpart).  Nothing is
 * allocated, by this call or by anything it calls.
 *   nx..angles  as spect_plan_create (psf_fx, psf_fz required; mu may be NULL;
 *               angles is a HOST array or NULL).
 *   x           device, nx*ny*nz image; v device, nx*nz*nview, overwritten.
 * Limits: nx*ny*nz <= 8388608 voxels and nview <= 4096, else SPECT_EINVAL.
 * The static arrays (32 MiB + 64 KiB) are held by every device that loads the
 * library until the process exits.  The first call on a device looks up
 * their device addresses (cudaGetSymbolAddress), with that device current.
 * All calls share the arrays: calls that overlap on the
 * GPU (other streams or host threads) race and must be serialised.
 * Errors: SPECT_EINVAL (arguments, sizes beyond the limits), SPECT_EUNSUPPORTED,
 * SPECT_ECUDA.
 */
spect_status spect_forward_static(int nx, int ny, int nz, int nview, const float* x, const float* mu, float dy,
                                  const float* psf_fx, const float* psf_fz, int px, int pz, int nview_psf,
                                  const double* angles, float* v, spect_stream stream);

/* Thread-local message for the last non-OK status returned on this thread
 * ("" if none).  The pointer stays valid until the next call on the thread. */
const char* spect_last_error(void);

/* Library version string, e.g. "spect-gb300 0.1 (sm_103a)". */
const char* spect_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPECT_H */
