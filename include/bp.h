/*
 * bp.h -- C ABI of the GB300 (sm_103a) 2D parallel-beam backprojection library.
 *
 * Operators of Koshev, Helou & Miqueles, "Fast Backprojection Techniques for High
 * Resolution Tomography" (arXiv:1608.03589):
 *   - R*  backprojection, Section 1 eq "B", discretised as Section 2 eq "bp_app";
 *   - the Backprojection-Slice-Theorem (Fourier) form of R*, Section 3 eq "bst",
 *     Section 5.3 Steps 1-4;
 *   - the FBP filter F of Section 3 Remark 1(ii) eq "fbp" and the Tikhonov filter of
 *     Section 6;
 *   - R, the Radon transform of Section 1 eq "P_theta", realised as the exact
 *     (scaled) transpose of each discrete R*, so that the discrete form of the adjoint
 *     identity (Section 1 eq "adjoint") holds.
 *
 * Geometry (Table "tab:symbols", Section 5), shared by every entry point:
 *   image      img[b][iy][ix], N x N float32, row-major, y along rows; pixel centres
 *              x_i = -1 + (i + 1/2) * dx, dx = 2/N, covering [-1, 1]^2.
 *   sinogram   sino[b][k][j], n_theta x n_det, row-major (one projection per row);
 *              detector centres t_j = (j - (n_det - 1)/2) * det_spacing.
 *   angles     theta[k] in radians, any order, any value (taken mod pi for weights).
 *   weights    w_k = half the sum of the two angular gaps around theta_k (mod pi);
 *              w_k = pi / n_theta for theta_k = k pi / n_theta (eq "bp_app").
 *   R*  (direct)   img[p] = sum_k w_k * lerp(sino[k], u_pk),
 *                  u_pk = (x_p . xi_k)/det_spacing + (n_det - 1)/2, zero off-detector.
 *   R   (direct)   sino[k][j] = (dx^2 / det_spacing) * sum_p hat(u_pk - j) * img[p].
 *
 * Conventions for every call:
 *   - Device pointers are caller-owned CUDA device memory on the plan's device,
 *     contiguous, 16-byte aligned; `batch` slices are packed back to back.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All calls are
 *     asynchronous on it unless stated otherwise; the returned status covers argument
 *     validation and launch errors only.
 *   - No call aborts the process.  On error the call returns a non-zero bp_status and
 *     bp_last_error() returns a message (thread-local, valid until the next call on the
 *     same thread).  A plan is not thread-safe: one plan per concurrently used stream.
 *   - The calling thread must have the plan's device current.
 */
#ifndef BP_H
#define BP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bp_plan bp_plan; /* opaque */

typedef enum {
    BP_OK = 0,
    BP_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad enum, misaligned pointer */
    BP_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed */
    BP_ERR_OOM = 3,          /* device or host allocation failed (nothing leaked) */
    BP_ERR_UNSUPPORTED = 4,  /* valid request outside the library's limits */
    BP_ERR_TIMEOUT = 5       /* a bounded device-side wait gave up (batched path) */
} bp_status;

typedef enum { BP_F32 = 0, BP_BF16 = 1, BP_F16 = 2 } bp_dtype;

typedef enum {
    BP_RAMLAK = 0,       /* |nu| band-limited to |nu| <= 1/(2 dt) (eq "fbp") */
    BP_SHEPP_LOGAN = 1,  /* |nu| sinc(nu dt) */
    BP_TIKHONOV = 2      /* |nu| / (1 + param |nu|), Section 6 (nu in cycles per unit t) */
} bp_filter_kind;

/* Limits of the library (BP_ERR_UNSUPPORTED beyond them). */
#define BP_MAX_N 16384
#define BP_MAX_NDET 16384
#define BP_MAX_NTHETA 65536

/*
 * bp_plan_create -- geometry, angle tables and device workspaces for one geometry.
 *   N            image side (pixels), 1..BP_MAX_N.
 *   n_det        detector bins per projection, 1..BP_MAX_NDET.
 *   n_theta      number of projections, 1..BP_MAX_NTHETA.
 *   theta        host array of n_theta angles (radians, finite); copied, caller keeps it.
 *   det_spacing  detector bin width in image units (> 0, finite); 2/n_det covers [-1, 1].
 * Builds in FP64 on the host: the quadrature weights w_k, the per-angle coordinate
 * tables (Section 2, eq "bp_app") and uploads them to the current device.  Fourier-path
 * and filter workspaces are allocated on their first use (make that first call before
 * any CUDA-graph capture).  Returns NULL on error (see bp_last_error()).
 */
bp_plan *bp_plan_create(int N, int n_det, int n_theta, const double *theta, double det_spacing);

/* Release every device and host resource of the plan (NULL is a no-op).  Synchronises
 * the plan's device before freeing. */
void bp_destroy(bp_plan *plan);

/*
 * bp_filter -- FBP row filter, Section 3 Remark 1(ii) eq "fbp" (and Section 6 for
 * BP_TIKHONOV): sino_out[b][k][j] = dt * sum_{i=0}^{n_det-1} h(j - i) * sino_in[b][k][i],
 * a linear (zero-extended, non-circular) convolution with the band-limited spatial
 * kernel h of the chosen frequency response, computed by FFT in float32.
 *   sino_in   device, batch x n_theta x n_det elements of `dtype`.
 *   sino_out  device, batch x n_theta x n_det float32; may equal sino_in only for BP_F32.
 *   param     lambda for BP_TIKHONOV (>= 0), ignored otherwise.
 */
bp_status bp_filter(bp_plan *plan, const void *sino_in, bp_dtype dtype, float *sino_out,
                    bp_filter_kind kind, float param, int batch, void *stream);

/*
 * bp_backproject_direct -- pixel-driven R* with linear interpolation, Section 2 eq
 * "bp_app".  float32 interpolation and accumulation; BF16/F16 sinograms are widened
 * to float32 on load.
 *   sino        device, batch x n_theta x n_det elements of `dtype`.
 *   img         device, batch x N x N float32 (output).
 *   accumulate  0: img = R* sino;  1: img += R* sino.
 */
bp_status bp_backproject_direct(bp_plan *plan, const void *sino, bp_dtype dtype, float *img,
                                int batch, int accumulate, void *stream);

/*
 * bp_backproject_fourier -- the Backprojection Slice Theorem form of R* (Section 3, eq
 * "bst"; Section 5.3 Steps 2.2-4), realised as a type-1 non-uniform FFT: each projection
 * is zero-padded to P = 2^ceil(log2(2 n_det)) and transformed (Step 2.2); its samples
 * on the polar ray are spread onto a 2N x 2N Cartesian frequency grid with a
 * Kaiser-Bessel kernel of width 6 (Step 3; the polar Jacobian |sigma| cancels the
 * BST's 1/sigma, Section 6 eq "reg_fbp"); a 2D inverse FFT (Step 4) and
 * deapodisation give the image.  It computes R* of the band-limited (trigonometric)
 * interpolant of each projection (Nyquist bin dropped), up to the gridding error.
 *   sino, dtype, img, batch as for bp_backproject_direct (img is overwritten).
 * First call allocates the plan's Fourier workspace (about 8 (2N)^2 bytes + 8 n_theta P/2).
 */
bp_status bp_backproject_fourier(bp_plan *plan, const void *sino, bp_dtype dtype, float *img,
                                 int batch, void *stream);

/*
 * bp_backproject_bst -- R* by the paper's own Backprojection-Slice-Theorem algorithm
 * (Section 5.3, Steps 1-4; eq "bst"; eq "kernel"): each projection zero-padded to
 * Pb = radial_oversampling * P points (P = 2^ceil(log2(2 n_det))) and transformed; the
 * transform times K^sigma = 1/|sigma| (1/dsigma at sigma = 0) gives the backprojection's
 * transform on the polar rays theta_k and theta_k + pi; it is interpolated linearly in
 * radius and in angle to the M x M Cartesian frequency grid (M = max(2^ceil(log2(2N)),
 * 64); the origin node takes the mean over the rays), and a 2D inverse FFT (the Riemann sum
 * of the inverse Fourier integral) gives the N x N image.
 * An approximation of R*, cheaper than bp_backproject_fourier and less accurate: linear
 * interpolation of oscillating spectra needs radial_oversampling of 4 or more for errors of
 * a few percent on filtered data, and the value 1/dsigma that K^sigma puts at the origin
 * shifts the mean of unfiltered backprojections.
 *   sino  device [batch][n_theta][n_det] of dtype;  img  device [batch][N][N] float32.
 *   radial_oversampling  1, 2, 4 or 8, with Pb <= 16384, else BP_ERR_INVALID_ARG /
 *   BP_ERR_UNSUPPORTED.  The first call (or one with another oversampling) allocates the
 *   plan's workspace for it (polar values n_theta x Pb/2 complex, besides the Fourier path's
 *   grid).
 */
bp_status bp_backproject_bst(bp_plan *plan, const void *sino, bp_dtype dtype, float *img, int radial_oversampling,
                             int batch, void *stream);

/*
 * bp_backproject_bst_windowed -- the paper's BST algorithm on semi-polar half-lines with the
 * Kaiser-Bessel window (Section 5.3, Steps 1-4 with Step 2.1; eq "w"): each projection becomes
 * the half-lines s >= 0 at theta_k and theta_k + pi, sampled at s_i = i dt (i < ns =
 * floor(n_det/2) + 1) by linear interpolation between detector centres; each half-line is
 * multiplied by w_i = I0(beta sqrt(1 - ((2i - ns + 1)/(ns - 1))^2)) / I0(beta), which tapers
 * both ends of the half-line; the ray at theta carries K^sigma times the transform of the line
 * through its two windowed half-lines (their one-sided transforms, the opposite one
 * conjugated; the sample at s = 0 counted once); then Steps 3-4 as bp_backproject_bst.
 * An accuracy variant, not R*: it is R* of the windowed projections g(t, theta) w(|t|)
 * computed by the BST algorithm; beta = 0 is the identity window (for odd n_det the result
 * is then bp_backproject_bst's; for even n_det the half-line samples lie between detector
 * centres, which averages neighbouring bins).
 *   sino  device [batch][n_theta][n_det] of dtype;  img  device [batch][N][N] float32.
 *   radial_oversampling  1, 2, 4 or 8 (as bp_backproject_bst);  beta  >= 0 and finite,
 *   else BP_ERR_INVALID_ARG.  Besides bp_backproject_bst's workspace the first call
 *   allocates n_theta x (2 ns - 1) floats for the windowed lines.
 */
bp_status bp_backproject_bst_windowed(bp_plan *plan, const void *sino, bp_dtype dtype, float *img,
                                      int radial_oversampling, float beta, int batch, void *stream);

/*
 * bp_backproject_logpolar -- R* by Andersson's log-polar convolution as the paper implements
 * it (Section 5.1 Steps 1-4 with the adaptive rho_0 of Section 5.2; eq "andersson"): the
 * sinogram resampled (linear interpolation) onto a log-polar mesh mu_i = rho_0 + i drho,
 * phi_j = 2 pi j / N_phi with rho_0 = ln(dx/2), the outermost step at most the detector
 * pitch (eq "N_rho") and N_phi = 2^ceil(log2(2 n_theta)); convolved with the kernel
 * delta(1 - e^rho cos theta) (a unit point mass on the mesh, eq "and_kernel") by 2D FFTs
 * (linear in rho, circular in theta); the result interpolated bilinearly at the pixel
 * centres.  An approximation of R*: the lines passing within e^{rho_0} of the origin are
 * missing (the origin problem of Section 5.2), so the error grows toward the image centre
 * (the centre of an odd image takes the mean over the angles at rho_0); away from it the
 * error falls at first order with the resolution.
 *   sino  device [batch][n_theta][n_det] of dtype;  img  device [batch][N][N] float32.
 *   Needs n_det >= 2 and transforms of at most 16384 points (N_rho + N_out, N_phi), i.e.
 *   about N <= 2048 at the default pitch, else BP_ERR_UNSUPPORTED.  The first call builds
 *   the plan's workspace: FP64 interpolation tables (16 bytes per pixel), two N_phi x L
 *   complex arrays (the kernel transform and the work array; 2 x 512 MiB at 2048^2 x 1800).
 */
bp_status bp_backproject_logpolar(bp_plan *plan, const void *sino, bp_dtype dtype, float *img, int batch,
                                  void *stream);

/*
 * bp_backproject_logpolar_partial -- R* by partial (sector) log-polar backprojections
 * (Section 5.2, "Partial Backprojections"; shifting property eq "sh_prop"; per sector the
 * convolution of bp_backproject_logpolar, Section 5.1 Steps 1-4).  The half-line angles
 * phi in [0, pi) (every line once) are split into `sectors` sectors of the mesh phi_j = j pi /
 * n_half (n_half = 2^ceil(log2 n_theta)); sector q moves the origin to -d xi_{phi_c}
 * (phi_c its centre, d = sqrt(2) (1 - a_r) / a_r: the object rescaled to a_r and shifted by
 * 1 - a_r), where every line of the sector lies at s > 0, so its log-polar mesh starts at a
 * finite rho_0 and no line is lost; the shifted sinogram g(s - d cos(phi - phi_c), phi) is
 * resampled (linear), convolved with the point-mass kernel by zero-padded 2D FFTs (linear in
 * rho and angle) and interpolated bilinearly at the pixels; the sectors add up.
 * An approximation of R* (first order in the meshes), free of the origin problem of
 * bp_backproject_logpolar.
 *   sino  device [batch][n_theta][n_det] of dtype;  img  device [batch][N][N] float32.
 *   sectors  a power of two dividing n_half, with the sector narrow enough for the shift
 *   (asin(1/((1 - a_r)/a_r)) + half the sector width + 3 dphi < pi/2), else BP_ERR_INVALID_ARG;
 *   a_r in (0, 1/2).  Transforms of at most 16384 points, else BP_ERR_UNSUPPORTED.  The
 *   first call (or one with other sectors / a_r) builds the plan's workspace: per-sector FP64
 *   pixel tables (16 bytes per pixel and sector) and two complex work arrays.
 */
bp_status bp_backproject_logpolar_partial(bp_plan *plan, const void *sino, bp_dtype dtype, float *img, int sectors,
                                          float a_r, int batch, void *stream);

/*
 * bp_set_fourier_width -- Kaiser-Bessel kernel width W (grid cells) of the gridding in
 * bp_backproject_fourier, bp_fbp_fourier and the Fourier-path R (Section 5.3 Step 3): 6 (the
 * default) or 4.  The gridding error falls roughly as exp(-pi W sqrt(1 - 1/sigma)) with the
 * oversampling sigma = M/N = 2: about 1e-6 relative at W = 6, about 1e-4 at W = 4, which does
 * (36 - 16)/36 less gridding work per sample.  Synchronises the device and releases the
 * Fourier workspace (rebuilt by the next Fourier call) when the width changes.
 * BP_ERR_INVALID_ARG for other widths.
 */
bp_status bp_set_fourier_width(bp_plan *plan, int width);

/*
 * bp_set_direct_workspace -- upper bound (bytes) on the four-image direct R*'s row-table
 * workspace (Section 2 eq "bp_app"; the tables hold each row's weighted samples and their
 * differences, 32 bytes per reachable bin and angle, about 146 MB per 2048^2 x 1800 slice).
 * A batch of one geometry writes the tables of as many slices as the workspace holds with one
 * launch and backprojects them with one persistent launch, chunk after chunk; one slice's
 * tables are always allocated, whatever the bound.  0 (the default) = a quarter of the device
 * memory free when the workspace grows.  Takes effect at the next call that grows or shrinks
 * the workspace: the plan's current tables are released here (after a device
 * synchronisation) when they exceed the new bound.  BP_ERR_INVALID_ARG for a NULL plan.
 */
bp_status bp_set_direct_workspace(bp_plan *plan, unsigned long long bytes);

/*
 * bp_fbp_fourier -- filtered backprojection in the Fourier form: the filter `kind` (param =
 * Tikhonov lambda, else ignored) applied inside the projection transforms of
 * bp_backproject_fourier (Section 3 Remark 1 (ii) eq "fbp" with Section 5.3 Step 2.2: one
 * transform of each projection serves both), saving bp_filter's launch and its round trip
 * of the filtered sinogram through memory.  It performs bp_filter's steps (transform, times
 * the response, inverse transform, cut to the detector) followed by
 * bp_backproject_fourier's, in the same floating-point operations, so the image equals
 * bp_filter followed by bp_backproject_fourier up to rounding (bit for bit when batch is 1
 * or n_theta is even: the two then transform the same pairs of projections together).
 *   sino  device [batch][n_theta][n_det] of dtype (not modified);  img  device [batch][N][N].
 * Limits and errors as bp_filter and bp_backproject_fourier; the first call with a kind
 * (or a new lambda) builds its response, as bp_filter does.
 */
bp_status bp_fbp_fourier(bp_plan *plan, const void *sino, bp_dtype dtype, float *img, bp_filter_kind kind,
                         float param, int batch, void *stream);

/*
 * bp_fbp_direct -- filtered backprojection in the direct form: bp_filter (kind, param =
 * Tikhonov lambda, else ignored; Section 3 Remark 1 (ii) eq "fbp") followed by
 * bp_backproject_direct (Section 2 eq "bp_app"), with the BP_F32 launch shape.  Where
 * bp_backproject_direct takes the four-image form and n_det <= 2048, the filter's last
 * transform writes each filtered row pair straight into that form's per-call row tables (one
 * launch instead of two, and no filtered sinogram in memory); otherwise the filtered slices go
 * to a plan-owned float32 array (batch x n_theta x n_det, allocated or grown on demand after a
 * synchronisation of `stream`, released by bp_destroy) and are backprojected from it.  The
 * filtered values are those of bp_filter (bit for bit when batch is 1 or n_theta is even), so
 * the image equals bp_filter followed by bp_backproject_direct up to the order of the direct
 * form's atomic partial sums.
 *   sino  device [batch][n_theta][n_det] of dtype (not modified);  img  device [batch][N][N]
 *   float32, overwritten.  Limits and errors as bp_filter and bp_backproject_direct.
 */
bp_status bp_fbp_direct(bp_plan *plan, const void *sino, bp_dtype dtype, float *img, bp_filter_kind kind,
                        float param, int batch, void *stream);

/*
 * bp_radon -- R, the forward Radon transform (Section 1 eq "P_theta"), as the scaled
 * exact transpose of a discrete R*:  R = (dx^2/dt) diag(1/w_k) A^T  where A is the
 * matrix of R*.  With fourier_adjoint = 0, A is the direct (linear-interpolation) R*;
 * with fourier_adjoint = 1, A is the Fourier-path R* (band-limited interpolation).
 *   img   device, batch x N x N float32.
 *   sino  device, batch x n_theta x n_det float32 (output, overwritten).
 */
bp_status bp_radon(bp_plan *plan, const float *img, float *sino, int batch, int fourier_adjoint,
                   void *stream);

/*
 * bp_radon_transpose -- img = R^T sino, the exact Euclidean transpose of bp_radon (the
 * gradient of <R f, sino> with respect to f).  Since R = (dx^2/dt) diag(1/w) A^T, this is
 * R* (A) with every quadrature weight w_k replaced by dx^2/dt.  fourier selects the direct
 * or the Fourier-path pair.  sino: device, batch x n_theta x n_det float32; img: device,
 * batch x N x N float32 (overwritten).
 */
bp_status bp_radon_transpose(bp_plan *plan, const float *sino, float *img, int batch, int fourier,
                             void *stream);

/*
 * bp_backproject_transpose -- sino = A^T img, the exact Euclidean transpose of R* (the
 * gradient of <R* g, img> with respect to g): A^T = (dt/dx^2) diag(w_k) R, i.e. R with
 * projection k scaled by w_k instead of dx^2/dt.  fourier selects the direct or the
 * Fourier-path pair.  img: device, batch x N x N float32; sino: device,
 * batch x n_theta x n_det float32 (overwritten).
 */
bp_status bp_backproject_transpose(bp_plan *plan, const float *img, float *sino, int batch, int fourier,
                                   void *stream);

/*
 * bp_fbp_host -- filtered backprojection from HOST memory to HOST memory:
 * for each slice of sino (host, batch x n_theta x n_det float32): copy it to the device,
 * bp_fbp_direct(kind, param), copy the image back into img (host,
 * batch x N x N float32); synchronise before returning.  The slices go through three device
 * slots: slice i + 1 is copied in and slice i - 1 copied out (on two internal streams of the
 * plan) while slice i is filtered and backprojected on `stream`, so with pinned host memory
 * a batch runs at the kernels' rate; pageable memory also works, without the overlap.  The
 * kind and param are checked before any copy is queued (same rules as bp_filter).  Slots,
 * streams and events are owned by the plan, created on the first call and released by
 * bp_destroy.
 */
bp_status bp_fbp_host(bp_plan *plan, const float *sino, float *img, bp_filter_kind kind,
                      float param, int batch, void *stream);

/*
 * bp_backproject_batched -- R* (direct, Section 2 eq "bp_app") of n independent slices with
 * possibly different geometries.  plans[i] gives slice i's geometry (all on the same device);
 * sinos[i] / imgs[i] are device pointers (imgs overwritten), dtypes[i] the sinogram element
 * type.  When every slice takes the four-image form (N even, mirror-symmetric angles, pixels
 * no larger than bins; images 16-byte aligned): one launch writes every slice's row tables and
 * clears the images, then ONE persistent launch backprojects all slices, each in its own
 * geometry (at most 256 slices per launch pair, and as many as the first plan's table budget
 * holds: its bp_set_direct_workspace bound, else a quarter of the free device memory; the
 * tables live in a workspace of the first plan, grown on demand after a synchronisation of
 * `stream`).  Otherwise ONE persistent kernel launch in which CTAs pull (slice, tile) work
 * items from a device counter.  The descriptors travel in the kernel parameters; after one
 * warm-up call with the same slices the call allocates nothing and can be graph-captured.
 */
bp_status bp_backproject_batched(bp_plan *const *plans, const void *const *sinos,
                                 const bp_dtype *dtypes, float *const *imgs, int n, void *stream);

/*
 * bp_fbp_static -- the same filtered backprojection as bp_filter followed by
 * bp_backproject_direct (device pointers, BP_RAMLAK or BP_SHEPP_LOGAN), for callers that
 * cannot allocate device memory when they need it: code inside a framework that owns
 * every device allocation (a fixed pool or memory budget, where a private cudaMalloc may
 * fail or break the budget), or real-time acquisition loops where allocating is not
 * allowed (cudaMalloc can synchronise the device and has no bounded latency).  The paper
 * has no counterpart; it exists only for such callers.
 *   Allocation: none.  Its scratch (one filtered slice) lives in a static device array of
 *   BP_STATIC_SCRATCH_BYTES that every GPU which loads the library holds until the process
 *   exits.  n_theta * n_det floats must fit in it (the 2048-bin x 1800-angle slice does),
 *   else BP_ERR_UNSUPPORTED; batch slices are done one after another through the same
 *   scratch.  The filter response is the plan's own, made in FP64 on the host by
 *   bp_plan_create; the call only reads it.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and keeps it for the life of the
 *   process; make that first call before any stream capture.  The address is not valid
 *   across cudaDeviceReset (nor is any plan).  The plan itself is created beforehand with
 *   bp_plan_create.
 *   Sharing: every call on a device uses the same array and leaves its last contents
 *   there; calls whose work overlaps on the GPU (different streams, or different host
 *   threads without ordering) race on it and must be serialised by the caller.
 *   sino, dtype, img, batch, stream as for bp_backproject_direct.
 */
#define BP_STATIC_SCRATCH_BYTES (16u << 20)
bp_status bp_fbp_static(bp_plan *plan, const void *sino, bp_dtype dtype, float *img, bp_filter_kind kind,
                        int batch, void *stream);

/*
 * bp_check -- synchronise `stream` and report device-side failures of earlier calls on
 * this plan: BP_ERR_TIMEOUT if a kernel's bounded wait on an asynchronous copy gave up
 * (the output of that call is invalid; the flag is cleared), else BP_OK.  Kernels never
 * trap or hang; they record the failure in a plan-owned status word instead.
 */
bp_status bp_check(bp_plan *plan, void *stream);

/*
 * Per-kernel timing (no counterpart in the paper; measurement support for the roofline of
 * each kernel of the path).
 * bp_stage_timing -- on != 0 starts recording, 0 stops; either way earlier records are
 *   dropped.  While it is on, every operator call of this plan records a CUDA event on its
 *   stream when it starts and after each kernel (or memset) it launches.  Off by default;
 *   with it on, do not capture the plan's calls into a CUDA graph.
 * bp_stage_times -- wait for the recorded events, then report per kernel name the summed time
 *   in milliseconds between the event before each launch and the one after it, and the number
 *   of launches; the records are then dropped (recording continues while on).  names[i] point
 *   to static strings of the library.  cap = capacity of names, ms and launches; *count = the
 *   number of distinct names (only the first cap are written).  BP_ERR_UNSUPPORTED when more
 *   than 8192 events were recorded since the last read (the records are dropped).
 */
bp_status bp_stage_timing(bp_plan *plan, int on);
bp_status bp_stage_times(bp_plan *plan, int cap, const char **names, float *ms, int *launches, int *count);

/*
 * Launch shapes and autotuning.  Neither changes what an operator computes, only how its
 * work is split across the GPU (no counterpart in the paper).
 *
 * BP_OP_DIRECT  direct R* (bp_backproject_direct, bp_radon_transpose with fourier = 0,
 *               bp_fbp_host, bp_fbp_static): shape[0] = angles per shared-memory stage
 *               (8, 16 or 32); shape[1] = angle groups (>= 1): each 64 x 64 pixel tile is
 *               backprojected by shape[1] CTAs over disjoint angle ranges whose partial sums
 *               are added atomically (the summation order then varies between runs, within
 *               FP32 rounding).  Geometries with N even, pixels no larger than bins and an
 *               angle set closed under theta -> pi - theta (every uniform set) take the
 *               four-image form instead (one thread serves a pixel block and its three mirror
 *               images; per-call row tables in a plan workspace allocated on first use):
 *               shape[0] = 32 gives each thread two pixel blocks at three CTAs per SM (the
 *               default), 16 one block at three CTAs per SM, 8 two blocks at four CTAs per SM
 *               with 6-angle stages; shape[1] = angle groups of its persistent schedule
 *               (<= 64; default: one per ~96 MB of row tables, so that a group's tables stay
 *               in L2); its partial sums are always added atomically, so its summation order
 *               varies between runs within FP32 rounding.
 *               bp_fbp_static never takes it (it allocates nothing).
 * BP_OP_RADON   direct R (bp_radon and bp_backproject_transpose with the direct form):
 *               shape[0] = angles per CTA (1, 2 or 4); shape[1] = image bands per angle block
 *               (>= 1; partial sinograms added atomically when > 1).  When pixels are no
 *               larger than bins the warps of an angle also fold their tables into the
 *               detector row with shared-memory atomics, so R's summation order varies
 *               between runs within FP32 rounding at every shape.
 *
 * A call (op, dtype, batch) takes the plan's own shape for (op, dtype, batch), else the
 * process-wide tuning cache entry for the plan's geometry (N, n_det, n_theta, window, SM
 * count), else the default rule: the four-image form's default above where it applies, else
 * stage 16 and enough angle groups for about two waves of three CTAs per SM; Radon: 4
 * angles per CTA (2 or 1 when their detector rows exceed 64 KB) and enough bands for four
 * CTAs per SM.  Out-of-range values are clamped at launch
 * (stage lowered when its shared memory does not fit, groups kept <= the number of stages).
 */
typedef enum { BP_OP_DIRECT = 0, BP_OP_RADON = 1 } bp_op;

/*
 * bp_autotune -- time the candidate shapes of `op` for this plan at (dtype, batch) on
 * `stream` with CUDA events (scratch device buffers are allocated, filled with a fixed
 * pattern and freed inside the call; the stream is synchronised) and keep the fastest for
 * the plan and in the process-wide cache (for BP_OP_DIRECT the default shape is kept unless
 * another is more than 1 % faster).  dtype is ignored for BP_OP_RADON.  shape
 * (nullable, 2 ints) receives the chosen shape, ms (nullable) the best time of one call in
 * milliseconds.  Not allowed while `stream` is being captured.
 */
bp_status bp_autotune(bp_plan *plan, bp_op op, bp_dtype dtype, int batch, void *stream, int *shape, float *ms);

/* bp_get_shape -- the shape (2 ints, after clamping) a call (op, dtype, batch) uses now. */
bp_status bp_get_shape(const bp_plan *plan, bp_op op, bp_dtype dtype, int batch, int *shape);

/* bp_set_shape -- fix the shape (2 ints) of calls (op, dtype, batch) on this plan. */
bp_status bp_set_shape(bp_plan *plan, bp_op op, bp_dtype dtype, int batch, const int *shape);

/*
 * bp_tune_cache_save / bp_tune_cache_load -- write / merge the process-wide tuning cache as
 * text, one entry per line: "op dtype batch N n_det n_theta W sm_count shape0 shape1".
 * Loading skips malformed lines; BP_ERR_INVALID_ARG if the file cannot be opened or holds
 * no valid entry.  Both are thread-safe and need no GPU.
 */
bp_status bp_tune_cache_save(const char *path);
bp_status bp_tune_cache_load(const char *path);

/* Last error message of the calling thread ("" if none). */
const char *bp_last_error(void);

/* Library version string, e.g. "bp 0.1 sm_103a". */
const char *bp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BP_H */
