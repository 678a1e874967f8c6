/*
 * sph_filter — double FFT filter for fields on a spherical (r, theta, phi) grid, on one GB300 GPU.
 *
 * The operation is the filter of Ji et al., arXiv:2305.01537, Sec. II.C "Filtering algorithms":
 * every evolved field is first low-passed in theta, on the double-covered great circle made by
 * joining the meridians at phi and phi + pi (with the field's parity sign across the pole), and
 * then low-passed in phi on every (r, theta) ring. Each Fourier mode is multiplied by a filter
 * function f(|l|, l_max) (exponential, Gaussian or spectrally sharp) whose cutoffs
 *     l_max = max(floor, 2 r / dr_min * L),   m_max = max(floor, 2 r / dr_min * sin(theta) * L)
 * depend on the shell radius r and (for phi) on the colatitude theta.
 *
 * Conventions shared by every entry point:
 *  - A state is `nvars * Nr * Ntheta * Nphi` contiguous values in the layout
 *    [var][shell i][theta index j][phi index k], k fastest. theta_j = (j + 1/2) pi / Ntheta
 *    (cell centred), phi_k = 2 pi k / Nphi. Nphi must be even (the phi + pi pairing).
 *  - Device pointers are caller-owned CUDA device memory on the plan's device (memory of another
 *    device is rejected with SPH_EINVAL). `in == out` (in place) is allowed; any other overlap is
 *    rejected with SPH_EALIAS.
 *  - Calls are asynchronous on `stream` (NULL = the legacy default stream) and return after
 *    enqueueing. Argument errors are returned immediately and nothing is enqueued. Errors a
 *    kernel detects on the device are latched in the plan and reported by
 *    sph_filter_plan_sync_status().
 *  - There is no CPU fallback: without a usable CUDA device every call fails with SPH_ECUDA.
 *  - The plan is immutable after creation; concurrent calls on different streams with the same
 *    plan are allowed. (The tensor-core form's single launch per application keeps its work
 *    counters in one of four sets of the plan, taken in turn; a launch waits for the previous user
 *    of its set, except inside a CUDA-graph capture, whose launches are ordered by the graph: do
 *    not run a captured graph of a tensor-core plan concurrently with other calls of that plan.)
 *  - A plan with shells whose theta pass is the identity (see sph_filter_plan_launches) runs part
 *    of an FP64 call on a stream it owns: the call forks that stream from `stream` with an event
 *    and joins it back with another before returning, so work enqueued on `stream` afterwards
 *    sees the whole result, as with any call. The calls of one plan share that stream, so their
 *    forked parts run one after the other. A CUDA-graph capture records the fork and the join as
 *    graph dependencies.
 */
#ifndef SPH_FILTER_H
#define SPH_FILTER_H

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* A cudaStream_t. */
typedef struct CUstream_st* sph_stream_t;

/* Opaque plan, created by sph_filter_plan_create and owned by the library until destroyed. */
typedef struct sph_filter_plan_s* sph_filter_plan;

typedef enum {
  SPH_OK = 0,
  SPH_EINVAL = 1,       /* invalid argument (sizes, parity, kind, cutoff parameters, NULL) */
  SPH_ENOMEM = 2,       /* device or host allocation failed */
  SPH_ECUDA = 3,        /* a CUDA runtime call failed (no device, launch failure, ...) */
  SPH_EUNSUPPORTED = 4, /* valid request this build cannot run (e.g. a shell too large) */
  SPH_ETIMEOUT = 5,     /* a bounded device-side wait gave up (latched by the device) */
  SPH_EALIAS = 6,       /* input and output partially overlap */
  SPH_EDEVICE = 7       /* a kernel latched an internal consistency error */
} sph_status;

/* Filter functions (Sec. II.C):
 *  SPH_FILTER_EXP    Eq. (exp_filter): 1 for |l| <= l_max, exp(-(|l| - l_max)) above.
 *  SPH_FILTER_GAUSS  Eq. (gaussian_filter): exp(log(0.9) (l / (l_max + 1))^2) for every l.
 *  SPH_FILTER_SHARP  the spectrally sharp low-pass: 1 for |l| <= l_max, 0 above.
 *  SPH_FILTER_HYBRID the hybrid filter of Sec. II.C: each theta circle and each phi ring takes
 *                    the Gaussian filter if Jameson's shock detector fires in one of its cells,
 *                    else the exponential filter. For a cell u_i with neighbours u_{i-1}, u_{i+1}
 *                    along the circle (across the poles with the parity sign) or the ring,
 *                      sigma = |(u_{i-1} + u_{i+1}) - 2 u_i| / (((|u_{i-1}| + |u_{i+1}|) + 2 |u_i|) + eps)
 *                    and the detector fires if sigma >= 0.95. Both detectors read the filter's
 *                    input; the decision is that of this expression evaluated in FP64 with IEEE
 *                    round-to-nearest, in this order. The switch makes the filter nonlinear, so
 *                    plans with hybrid fields run only sph_filter_apply and its FP32-storage,
 *                    host-buffer and batch forms (the adjoint and tanh calls return
 *                    SPH_EUNSUPPORTED), with the FP64 or compensated-FP32 precision and the
 *                    staged shell kernels (one CTA per shell, or a CTA pair for shells such as
 *                    128 x 256); plans that need the chunked FP64 kernel (lengths with prime
 *                    factors above 3) or the tensor-core form fail to create with
 *                    SPH_EUNSUPPORTED. */
typedef enum { SPH_FILTER_EXP = 0, SPH_FILTER_GAUSS = 1, SPH_FILTER_SHARP = 2, SPH_FILTER_HYBRID = 3 } sph_kind;

/* Arithmetic of the plan's kernels. Inputs and outputs are FP64 for every choice.
 *  SPH_PREC_F64     plain form: FFTs in FP64 arithmetic.
 *  SPH_PREC_F32X2   plain form with FFTs in compensated FP32-pair arithmetic (about 48-bit
 *                   significands).
 *  SPH_PREC_SPLIT_TC split-precision tensor-core form.
 *  SPH_PREC_SPECTRAL the same filter in its spectral form, FP64: the theta pass is diagonal in
 *                   the azimuthal mode m (shifting phi by pi multiplies mode m by (-1)^m), so a
 *                   shell with a theta pass is filtered as one phi transform per ring, per mode m
 *                   the theta filter of the even or odd extension over the Ntheta values (a
 *                   cosine or sine transform pair, through a complex FFT of length Ntheta), the
 *                   phi multiply, and one inverse phi transform; shells without a theta pass take
 *                   the phi pass alone, as in SPH_PREC_F64. Requires Ntheta even and a shell that
 *                   one CTA stages (Ntheta (Nphi + 2) 8 bytes plus scratch within the shared
 *                   memory of one SM); plans with hybrid fields or other shapes fail to create
 *                   with SPH_EUNSUPPORTED. */
typedef enum { SPH_PREC_F64 = 0, SPH_PREC_SPLIT_TC = 1, SPH_PREC_F32X2 = 2, SPH_PREC_SPECTRAL = 3 } sph_precision;

/* Cutoff parameters (Sec. II.C, cutoff equations), copied into the plan at creation. */
typedef struct {
  const double* r;  /* [Nr] physical radius of each shell (any radial map already applied), >= 0 */
  double dr_min;    /* smallest radial spacing of the grid, > 0 */
  const double* L;  /* [nvars] the calligraphic-L factor per field, > 0 (paper: 3 metric, 12 matter) */
  const int* kind;  /* [nvars] sph_kind per field */
  double floor;     /* lower bound of l_max and m_max; the paper's value is 2; >= 0 */
  int precision;    /* sph_precision */
  double eps;       /* epsilon of Jameson's detector (SPH_FILTER_HYBRID fields), finite, >= 0;
                       ignored when no field is hybrid */
} sph_cutoff_params;

/* Create a plan for states of nvars fields on an Nr x Ntheta x Nphi grid, on the current CUDA
 * device. parity[v] in {0, 1} is the axis parity exponent a of field v in the double covering
 * X(vartheta) = (-1)^a X(2 pi - vartheta, phi + pi) (Sec. II.C). Builds the cutoff tables
 * (l_max per shell and field class, m_max per ring and class) and the twiddle tables in FP64 on
 * the host and copies them to the device. *out is set to NULL on failure.
 * Errors: SPH_EINVAL (Nr, Ntheta, nvars < 1; Nphi < 2 or odd; parity not 0/1; kind unknown;
 * dr_min <= 0; r < 0; L <= 0; floor < 0; precision unknown; eps < 0 or not finite with a hybrid
 * field; NULL pointer), SPH_EUNSUPPORTED (a hybrid field in a plan that cannot run it, see
 * SPH_FILTER_HYBRID), SPH_ENOMEM, SPH_ECUDA. */
sph_status sph_filter_plan_create(sph_filter_plan* out, int Nr, int Ntheta, int Nphi, int nvars,
                                  const int* parity, const sph_cutoff_params* params);

/* Release the plan and its device tables. Synchronises the plan's device first. NULL is a no-op. */
void sph_filter_plan_destroy(sph_filter_plan plan);

/* out = F in: the double filter (theta pass on the double-covered circles, then the phi pass on
 * the rings), Sec. II.C. in/out: device FP64 states in the layout above. */
sph_status sph_filter_apply(sph_filter_plan plan, const double* in, double* out, sph_stream_t stream);

/* out = F^T in: the transpose of the filter, i.e. the phi pass followed by the theta pass (each
 * pass is a real symmetric operator: a circulant with an even real multiplier, conjugated by the
 * signed doubling permutation). Used for reverse-mode differentiation. */
sph_status sph_filter_apply_adjoint(sph_filter_plan plan, const double* in, double* out,
                                    sph_stream_t stream);

/* Pointwise maps fused into the filter for a chain x_{k+1} = F(tanh(x_k)) (Sec. II.C's filter
 * composed with an elementwise nonlinearity):
 *   sph_filter_apply_tanh:          out = F(tanh(z))
 *   sph_filter_apply_adjoint_tanh:  out = (1 - tanh(z)^2) * F^T(g)    (chain rule through tanh)
 * z, g, out are device FP64 states; out may alias g (not z). tanh is evaluated in the plan's
 * arithmetic: FP64 for SPH_PREC_F64 and SPH_PREC_SPECTRAL, compensated FP32 pairs (relative error
 * below 2^-45) for SPH_PREC_F32X2; the tensor-core form returns SPH_EUNSUPPORTED. */
sph_status sph_filter_apply_tanh(sph_filter_plan plan, const double* z, double* out,
                                 sph_stream_t stream);
sph_status sph_filter_apply_adjoint_tanh(sph_filter_plan plan, const double* g, const double* z,
                                         double* out, sph_stream_t stream);

/* FP32 storage variants of the four calls above: in, out, z and g are FP32 device states; the
 * values are widened on load and rounded once on store, and the arithmetic in between is the
 * plan's precision. */
sph_status sph_filter_apply_f32(sph_filter_plan plan, const float* in, float* out, sph_stream_t stream);
sph_status sph_filter_apply_adjoint_f32(sph_filter_plan plan, const float* in, float* out,
                                        sph_stream_t stream);
sph_status sph_filter_apply_tanh_f32(sph_filter_plan plan, const float* z, float* out,
                                     sph_stream_t stream);
sph_status sph_filter_apply_adjoint_tanh_f32(sph_filter_plan plan, const float* g, const float* z,
                                             float* out, sph_stream_t stream);

/* End-to-end variant for host-resident states: copies host_in to the device, filters, copies
 * the result to host_out, ordered on `stream` (the work starts after what `stream` already holds and
 * `stream` continues after the last copy out), and returns after enqueueing. Internally the state
 * moves in chunks of whole fields: the copies in on one stream of the plan, each chunk's kernels on
 * one of several compute streams, the copies out on another stream, so both copy directions and
 * the kernels overlap. host_in/host_out should be page-locked for the copies to overlap. The device staging buffers are allocated by the plan
 * on first use and kept until the plan is destroyed (for the tensor-core form also the work lists
 * of the field chunks the call filters one at a time); calls of this function on one plan share
 * them, so order such calls (one stream, or a synchronisation between them). Synchronise the
 * stream before reading host_out. Errors as sph_filter_apply, plus SPH_ENOMEM. */
sph_status sph_filter_apply_host(sph_filter_plan plan, const double* host_in, double* host_out,
                                 sph_stream_t stream);

/* Same as sph_filter_apply_host, but allocates no device memory: the device copies of the input
 * and the output live in a fixed array inside the library (32 MiB on every GPU where this call has
 * run, held until the process exits). The paper has no counterpart; this is for callers that cannot
 * let a library allocate device memory, e.g. a framework whose own allocator has reserved the
 * whole device at start-up, or code that must not risk the device synchronisation that
 * cudaMalloc/cudaFree may cause. No cudaMalloc, cudaFree or allocating library routine is called.
 * Limits and behaviour:
 *  - The state may have at most 2,097,152 points (nvars * Nr * Ntheta * Nphi); larger states are
 *    rejected with SPH_EINVAL before anything is enqueued.
 *  - The array's device memory is committed on a device by the first call there (the code holding
 *    the array is loaded lazily, at that call), and that first call may synchronise the device.
 *    A caller whose allocator reserves the whole device should make one call (a small plan will
 *    do) before reserving it, and every caller should make the first call before any stream
 *    capture. Each call looks up the array's address on the current device again, so a
 *    cudaDeviceReset between calls does not leave a stale address.
 *  - Every call uses the same array, and nothing in it needs to start at zero (each call overwrites
 *    what it reads). Calls whose work overlaps on the GPU (e.g. on two streams) race on the array;
 *    order them on one stream or synchronise between them.
 *  - host_in/host_out as in sph_filter_apply_host; asynchronous on `stream`. */
sph_status sph_filter_apply_host_noalloc(sph_filter_plan plan, const double* host_in, double* host_out,
                                         sph_stream_t stream);

/* Wait for all work on the plan's device and return the first error a kernel latched for this
 * plan (SPH_OK if none), then clear it. */
sph_status sph_filter_plan_sync_status(sph_filter_plan plan);

/* Number of filtered points per application: nvars * Nr * Ntheta * Nphi (0 for NULL). */
long long sph_filter_plan_points(sph_filter_plan plan);

/* Number of kernel launches one out-of-place sph_filter_apply enqueues for this plan. A plan whose
 * shells include some with an identity theta pass (exponential or sharp filter with l_max >=
 * Ntheta) runs three: a copy of those shells, the shell kernel over the others and a kernel over
 * their active phi ring pairs. In-place, FP32 and mapped calls may enqueue fewer; see
 * sph_filter_plan_launch_count for the exact number. 0 for NULL. */
int sph_filter_plan_launches(sph_filter_plan plan);

/* Kernel launches this plan has enqueued so far, over all its calls and streams (a launch captured
 * into a CUDA graph counts once, when it is captured; replays do not add to it). 0 for NULL. */
long long sph_filter_plan_launch_count(sph_filter_plan plan);

/* Algebraic constraints applied after filtering (Sec. II.C, "Filtering spacetime fields in the
 * presence of BHs": the constraints det(gamma_bar) = det(gamma_hat) and gamma_bar^{ij} A_bar_ij = 0
 * and the substitutions that enforce them), in place on a state, point by point:
 *  - standard form: with m = delta + h, the metric becomes det(m)^(-1/3) m (so det = 1) and A loses
 *    m tr / 3, tr = sum_ab (m^-1)_ab A_ab (its trace in the metric);
 *  - modified form, at points of shells flagged in theta_filtered whose lapse is below alpha_bh
 *    (strictly): h_11 is solved from det(m) = 1 with the other components kept, A is kept.
 * Components are orthonormal-basis components of the conformal metric perturbation h and of the
 * conformal extrinsic curvature A (gamma_bar_ij = R_i R_j (delta_ij + h_ij) for the spherical
 * scale factors R = (1, r, r sin theta), which cancel from both constraints).
 * Arguments:
 *  - state: device FP64 state [nvars][Nr][Ntheta][Nphi] (layout of the filter calls), modified in
 *    place; fields other than the 13 named below are not touched.
 *  - h_vars, a_vars: host arrays of 6 field indices each, in the order 11, 12, 13, 22, 23, 33;
 *    alpha_var: the lapse field. All 13 must be distinct and in [0, nvars).
 *  - theta_filtered: device array of Nr bytes, nonzero for the shells where the theta filter is
 *    active (e.g. l_max < Ntheta for the metric fields' filter), or NULL for none (standard form
 *    everywhere). alpha_bh: the lapse threshold of the modified form (0.3 in the paper).
 * Returns SPH_EINVAL for a NULL or host state, a state or flag array on a device other than the
 * current one, bad sizes, indices out of range or repeated, or a
 * non-finite alpha_bh (nothing is enqueued); SPH_ECUDA if the launch fails. Asynchronous on
 * `stream`. A point whose det(m) is not positive gives non-finite values (no physical metric). */
sph_status sph_enforce_constraints(double* state, int nvars, int Nr, int Ntheta, int Nphi, const int* h_vars,
                                   const int* a_vars, int alpha_var, const unsigned char* theta_filtered,
                                   double alpha_bh, sph_stream_t stream);

/* Static description of a status code. */
const char* sph_filter_status_string(sph_status status);

/* ---- several grids at once (uneven shapes, e.g. the levels of a multi-grid evolution) ---- */

/* Opaque batch of plans, one per grid; owned by the library until destroyed. */
typedef struct sph_filter_batch_s* sph_filter_batch;

/* Group nplans plans (created on the same device) so that one call filters all their grids. The
 * kernels of different grids run concurrently on internal streams forked from the caller's
 * stream and joined back into it. The plans must outlive the batch. *out is NULL on failure.
 * Errors: SPH_EINVAL (nplans < 1, NULL plan, plans on different devices), SPH_ENOMEM, SPH_ECUDA. */
sph_status sph_filter_batch_create(sph_filter_batch* out, int nplans, const sph_filter_plan* plans);

/* Release the batch (its streams, events and graph). Synchronises first. NULL is a no-op. */
void sph_filter_batch_destroy(sph_filter_batch batch);

/* out[g] = F_g in[g] for every grid g (Sec. II.C double filter): in and out are host arrays of
 * nplans device pointers to FP64 states of the plans' shapes. Asynchronous on `stream`. Errors as
 * sph_filter_apply. */
sph_status sph_filter_batch_apply(sph_filter_batch batch, const double* const* in, double* const* out,
                                  sph_stream_t stream);

/* Record napply consecutive applications into a CUDA graph kept by the batch: the first filters
 * in -> out, the others filter out in place (one filter application per Runge-Kutta substep).
 * The pointers are baked into the graph; capture again to change them. Must not be called while
 * `stream` is itself being captured. Errors: SPH_EINVAL (napply < 1), SPH_ECUDA. */
sph_status sph_filter_batch_capture(sph_filter_batch batch, const double* const* in, double* const* out,
                                    int napply, sph_stream_t stream);

/* Replay the captured graph on `stream` (one graph launch). SPH_EINVAL if nothing was captured. */
sph_status sph_filter_batch_launch(sph_filter_batch batch, sph_stream_t stream);

/* Autotuner: time every valid choice of threads per CTA and FFT batch size for this plan on the
 * caller's in/out device buffers (FP64, the plan's shape; out is overwritten) and keep the
 * fastest. Synchronous. Must not run concurrently with other calls on the same plan. *best_ms
 * (may be NULL) receives the fastest time of one application. */
sph_status sph_filter_plan_autotune(sph_filter_plan plan, const double* in, double* out, sph_stream_t stream,
                                    double* best_ms);

#ifdef __cplusplus
}
#endif

#endif /* SPH_FILTER_H */
