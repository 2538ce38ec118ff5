/*
 * lrvol.h -- C ABI of liblrvol: direct volume ray casting of trivariate
 * LR-splines on one GPU (sm_103a).
 *
 * Method: Fuchs, Barrowclough, Hjelmervik, Dahl, "Direct interactive
 * visualization of locally refined spline volumes for scalar and vector
 * fields".  An LR-spline f = sum_i c_i gamma_i N_i (Eq. 2) is converted once
 * to one Bezier block per element (Sec. 3.2.3), elements are found through a
 * k-d forest (Sec. 3.2.1, Alg. 1), and each pixel ray is sampled at a fixed
 * step or at the adaptive distance of Eq. 4, mapped through a 1D transfer
 * function and composited front to back (Alg. 2).
 *
 * Conventions for every function:
 *   - returns an lrvol_status (0 = LRVOL_OK); no C++ exception and no exit()
 *     crosses this boundary; lrvol_last_error() describes the last failure
 *     of the calling thread;
 *   - pointers named *_dev are device pointers on the handle's device, owned
 *     by the caller; host pointers are read during the call only;
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); calls
 *     that take one are asynchronous on it, except where stated;
 *   - one handle may be used by one stream at a time;
 *   - element ids are positions in the caller's element array (0-based);
 *     0xFFFFFFFF marks "no element" (a point outside [0,1]^3).
 *
 * Boxes are half open, [lo, hi); the upper domain face x = 1 belongs to the
 * element whose hi is 1.  Ties at a split plane go to the ">=" side, as in
 * Alg. 1.
 */
#ifndef LRVOL_H
#define LRVOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrvol_s *lrvol_t; /* opaque; owns all device copies of one volume */

typedef enum {
  LRVOL_OK = 0,
  LRVOL_ERR_ARG = -1,         /* invalid argument (null pointer, bad size, bad enum) */
  LRVOL_ERR_OOM = -2,         /* device or host allocation failed */
  LRVOL_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  LRVOL_ERR_STATE = -4,       /* call out of order (e.g. render before to_bezier/build_accel) */
  LRVOL_ERR_BOUNDS = -5,      /* a kernel's bounds check tripped (index outside its buffer) */
  LRVOL_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up */
  LRVOL_ERR_UNSUPPORTED = -7  /* valid but not supported by this build (e.g. degree > 3 in render) */
} lrvol_status;

enum { LRVOL_ORTHO = 0, LRVOL_PERSP = 1 };
enum { LRVOL_STEP_FIXED = 0, LRVOL_STEP_HEURISTIC = 1, LRVOL_STEP_LEARNED = 2 };
enum { LRVOL_FIELD_SCALAR = 0, LRVOL_FIELD_MAGNITUDE = 1, LRVOL_FIELD_COMPONENT = 2 };
enum { LRVOL_STORE_F32 = 0, LRVOL_STORE_F16 = 1, LRVOL_STORE_BF16 = 2 };
enum { LRVOL_SHADE_NONE = 0, LRVOL_SHADE_GRADIENT = 1 };

/* Camera.  Ray of pixel (i, j), row j = 0 at the top, in FP32 with this exact
 * order of operations (fmaf = fused multiply-add, all other ops IEEE-rounded):
 *   FP64, once: F = normalize(target - eye), R = normalize(cross(F, up)),
 *     U = cross(R, F); ty = tan(fovy/2) (persp) or extent/2 (ortho);
 *     tx = ty*width/height; sxs = (float)(2*tx/width), sxo = (float)(-tx),
 *     sys = (float)(-2*ty/height), syo = (float)ty; E,F,R,U rounded to float.
 *   a = fmaf(i + 0.5f, sxs, sxo); b = fmaf(j + 0.5f, sys, syo)
 *   persp: d_c = fmaf(a, R_c, fmaf(b, U_c, F_c)); n = sqrtf(fmaf(dx,dx, fmaf(dy,dy, dz*dz)));
 *          d_c = d_c / n; o = E
 *   ortho: o_c = fmaf(a, R_c, fmaf(b, U_c, E_c)); d = F
 *   slab test against [0,1]^3 from t = 0 gives [t_in, t_out); a miss writes 0.
 * Rows [row_begin, row_end) are rendered (both 0: all rows); other rows of
 * the output are left untouched.  With band_count = n > 1 those rows are cut
 * into bands of LRVOL_BAND_ROWS rows (the last one may be shorter) and only
 * the bands b with b mod n == band_index are rendered (0 <= band_index < n),
 * so n ranks with band_index 0..n-1 interleave their bands over the frame.
 * These are the screen-space sharding hooks (Sec. 4's rays are independent). */
#define LRVOL_BAND_ROWS 8
typedef struct {
  int32_t projection; /* LRVOL_ORTHO | LRVOL_PERSP */
  int32_t width, height;
  double eye[3], target[3], up[3];
  double fovy;   /* persp: full vertical field of view, radians */
  double extent; /* ortho: full height of the view window, world units */
  int32_t row_begin, row_end;
  int32_t band_count, band_index; /* interleaved bands (0 or 1: every band) */
} lrvol_camera;

/* Transfer function: 256 RGBA entries spanning [vmin, vmax]; value v maps to
 * x = clamp((v - vmin)/(vmax - vmin), 0, 1) * 255 and the entries floor(x)
 * and floor(x)+1 are linearly interpolated (colour not premultiplied).
 * Copied during the call. */
typedef struct {
  float rgba[256][4];
  double vmin, vmax;
} lrvol_tf;

/* Sampling and compositing (Sec. 4.2, Alg. 2, Eq. 4).
 *   FIXED:     t_k = fmaf((float)k, h, t_in)
 *   HEURISTIC: t_{k+1} = t_k + ds(e_k), ds(e) = (float)(2^-d * min side of e),
 *              d = max(p1,p2,p3), e_k the element holding sample k (Eq. 4)
 *   LEARNED:   t_{k+1} = t_k + ds(e_k) * mult[e_k] (one FP32 product), with
 *              mult a caller-owned device array of one multiplier per element
 *              (e.g. from lrvol_features and lrvol_mlp_infer); Eq. 4 when all are 1
 * Sample k sits at p_k = clamp(fmaf(t_k, d, o), 0, 1); its segment is
 * min(t_{k+1}, t_out) - t_k; T = (1 - alpha_src)^(segment/xi);
 * C += (1-T)(1-alpha) C_src; alpha += (1-T)(1-alpha); the ray stops at
 * t_out or once alpha >= alpha_stop.  Output is premultiplied RGBA.
 * Gradient shading (Sec. 4.1, scalar fields): C_src is multiplied by
 * I = max(0.4, |l . n|), with n = grad f / max(|grad f|, eps) at the sample,
 * eps = 1e-3 (vmax - vmin) (a gradient below eps counts as none, and I
 * tends to 0.4 continuously), and l the unit vector towards the light:
 * `light` normalised, or -d (a light at the eye) when `light` is all zero.
 * Trimming (Sec. 4.1): with `trim` set, a pixel's [t_in, t_out] is cut to
 * [t_front, t_back]; a pixel with neither hit is transparent, one with only
 * back-face hits (the eye inside the mesh) keeps [t_in, t_back], one with
 * only front-face hits (an open mesh) keeps [t_front, t_out]. */
typedef struct {
  int32_t mode;      /* LRVOL_STEP_FIXED | LRVOL_STEP_HEURISTIC | LRVOL_STEP_LEARNED */
  int32_t field;     /* LRVOL_FIELD_SCALAR | _MAGNITUDE (|v| of a 3-vector) | _COMPONENT */
  int32_t component; /* for LRVOL_FIELD_COMPONENT */
  double h;          /* fixed step (FIXED only) */
  double xi;         /* reference length xi of Alg. 2 (T = (1 - alpha)^(segment / xi)) */
  double alpha_stop; /* early ray termination threshold; 1.0 = only when fully opaque */
  const float *mult; /* LEARNED: n_elem step multipliers (device), read during the render */
  int32_t shading;   /* LRVOL_SHADE_NONE | LRVOL_SHADE_GRADIENT (scalar fields only) */
  double light[3];   /* GRADIENT: direction towards the light (any length); all zero = -ray direction */
  const float *trim; /* NULL, or per pixel (t_front, t_back) from lrvol_trim (device, height x width x 2
                        floats, row major), read during the render */
} lrvol_step;

/* Diagnostics; the depth rows match the paper's tables (Sec. 4.3). */
typedef struct {
  int64_t n_elem, n_basis, n_nodes;
  int32_t blocks[3];
  int32_t depth_min, depth_max; /* tree depth per forest block (0: the head names the element) */
  double depth_mean, depth_var;
  int64_t incidence_entries;    /* element-to-B-spline pairs used by the change of basis */
  int64_t bytes_device;         /* device memory held by the handle */
  int64_t samples, lookups, rays_hit; /* counters of the last render call */
} lrvol_stats_t;

/* Create a volume from an LR-spline (Eq. 2).  Synchronous.
 * deg[3]     tri-degree p, each in 1..4 (render needs all equal, 1..3)
 * ncomp      1 (scalar) or 3 (vector field)
 * elem_box   n_elem x 6 doubles: lo x,y,z then hi x,y,z; a box partition of [0,1]^3
 * knots      n_basis x (p1+2 + p2+2 + p3+2) doubles: each LR B-spline's local
 *            knot vectors, x then y then z, non-decreasing
 * coef       n_basis x ncomp doubles (c_i); weight: n_basis doubles (gamma_i)
 * The inputs are copied to the current device; the caller keeps ownership.
 * Errors: LRVOL_ERR_ARG for null pointers, sizes < 1, degrees out of range,
 * boxes outside [0,1] or empty, decreasing knots; LRVOL_ERR_OOM; LRVOL_ERR_CUDA. */
int lrvol_create(const int32_t deg[3], int32_t ncomp, int64_t n_elem, const double *elem_box,
                 int64_t n_basis, const double *knots, const double *coef, const double *weight,
                 lrvol_t *out);

/* Build the k-d forest (Sec. 3.2.1): blocks[0] x blocks[1] x blocks[2]
 * regular blocks (each a power of two, at most 1024), one depth-balanced k-d
 * tree per block over the elements meeting it; split planes are element
 * faces rounded up to FP32 so that FP32 queries decide exactly as in FP64.
 * The tree is built on the host and uploaded on `stream`.
 * Errors: LRVOL_ERR_ARG (blocks not powers of two), LRVOL_ERR_OOM, LRVOL_ERR_CUDA. */
int lrvol_build_accel(lrvol_t vol, const int32_t blocks[3], void *stream);

/* The same forest with a choice of split rule inside each block:
 *   LRVOL_SPLIT_BALANCED  the depth-balanced trees of lrvol_build_accel;
 *   LRVOL_SPLIT_MIDPOINT  octree-style trees: each node splits its region at
 *                         the midpoint, on x, y and z in turn (three binary
 *                         levels are one octree level of the paper's octree
 *                         look-up, Sec. 3.2); with blocks at the finest
 *                         element size and no trees the forest is the
 *                         paper's look-up texture.
 * Element ids are the same whichever rule builds the forest.  Midpoint splits
 * reach element faces only at dyadic coordinates: a mesh with other faces
 * returns LRVOL_ERR_UNSUPPORTED.  Errors otherwise as lrvol_build_accel. */
#define LRVOL_SPLIT_BALANCED 0
#define LRVOL_SPLIT_MIDPOINT 1
int lrvol_build_accel_split(lrvol_t vol, const int32_t blocks[3], int32_t split, void *stream);

/* Change of basis to Bezier blocks (Sec. 3.2.3), FP64 on the GPU by blossoming
 * each incident B-spline's univariate factors over the element (exact up to
 * rounding); kept in FP64 for lrvol_get_bezier, and stored for rendering as
 *   LRVOL_STORE_F32   FP32 coefficients;
 *   LRVOL_STORE_F16 / LRVOL_STORE_BF16   16-bit values with a per-element,
 *     per-component FP32 offset o = (max+min)/2 and scale s = (max-min)/2:
 *     a sample differs from the FP32-storage value by at most s*u,
 *     u = 2^-11 (FP16) or 2^-8 (BF16); accumulation stays FP32.  With FP16
 *     blocks the render, the streamline tracer and the tube colouring keep
 *     the 16-bit values in registers and multiply them with the x monomials
 *     rounded to FP16 (mixed-precision FMAs, exact products, FP32 sums):
 *     their values differ from the FP32-storage value by at most 2*s*u
 *     (lrvol_eval, lrvol_eval_grad: s*u).
 * Errors: LRVOL_ERR_ARG (bad storage), LRVOL_ERR_OOM, LRVOL_ERR_CUDA. */
int lrvol_to_bezier(lrvol_t vol, int32_t storage, void *stream);

/* Render one image into rgba_dev (height x width x 4 floats, row major,
 * premultiplied RGBA, caller-owned device buffer).  Needs build_accel and
 * to_bezier first (else LRVOL_ERR_STATE).  Asynchronous on `stream`.
 * Errors: LRVOL_ERR_ARG (bad camera/step, null), LRVOL_ERR_STATE,
 * LRVOL_ERR_UNSUPPORTED (non-isotropic degree or degree > 3), LRVOL_ERR_CUDA. */
int lrvol_render(lrvol_t vol, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                 float *rgba_dev, void *stream);

/* Trace of the render kernel's own samples for a list of pixels: the parity
 * hook that compares the march of lrvol_render, sample by sample, with an
 * independent implementation of Sec. 4 (ray setup), Alg. 1 (element look-up),
 * Sec. 3.2.3 (Bezier evaluation), Eq. 4 (step) and Alg. 2 (compositing).  It
 * runs the same kernel template as lrvol_render, with a compile-time trace
 * flag that is off in every lrvol_render launch; every per-ray decision and
 * value is the same as in lrvol_render's image (one thread per listed pixel
 * instead of per tile position; a ray's work does not depend on its
 * neighbours).
 *   pix_dev      n_pix x 2 int32 (i, j) pixel coordinates (device); the
 *                camera's row range is ignored.  A pixel outside the image
 *                gets count 0, RGBA 0 and sets the status word (LRVOL_ERR_BOUNDS
 *                at the next lrvol_stats).
 *   trace_dev    n_pix x max_samples x 4 floats (device): for composited
 *                sample k < max_samples of pixel q, at [q][k]:
 *                (t_k, element id as the bits of a uint32, the field value
 *                before the transfer function -- scalar, |v| or the chosen
 *                component --, segment length min(t_{k+1}, t_out) - t_k).
 *                Entries past a pixel's count are unspecified (the sample
 *                evaluated after the last composited one may be written).
 *   count_dev    n_pix int32 (device): samples composited for the pixel (may
 *                exceed max_samples; only the first max_samples are written).
 *   rgba_dev     n_pix x 4 floats (device): the pixel's premultiplied RGBA,
 *                equal to lrvol_render's for that pixel.
 * lrvol_stats then reports this call's samples, look-ups and rays hit.
 * Asynchronous on `stream`.  n_pix = 0 launches nothing.
 * Errors: LRVOL_ERR_ARG (negative sizes, null pointers with n_pix > 0, bad
 * camera/step as lrvol_render), LRVOL_ERR_STATE, LRVOL_ERR_UNSUPPORTED,
 * LRVOL_ERR_CUDA. */
int lrvol_render_trace(lrvol_t vol, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                       const int32_t *pix_dev, int64_t n_pix, int32_t max_samples, float *trace_dev,
                       int32_t *count_dev, float *rgba_dev, void *stream);

/* lrvol_render for callers that may not allocate device memory.  Some
 * callers cannot call cudaMalloc: a host application that owns every byte of
 * device memory through its own pool and forbids libraries to allocate, or a
 * long-running service whose device footprint must not change once it has
 * started.  This call allocates nothing (no cudaMalloc, no cudaFree, no
 * allocating library routine) and does not touch the handle's scratch: the
 * kernel's scratch (sample/look-up/ray counters and the status word)
 * is a file-scope static device array of 256 bytes, which every GPU that
 * loads the library holds until the process exits.  The paper has no
 * counterpart; it is an integration variant of lrvol_render.
 *
 * The caller passes the inputs (a handle whose build_accel and to_bezier are
 * done, camera, TF, step) and the outputs: rgba_dev as for lrvol_render, and
 * optionally counters_dev (4 uint64 on the device, or NULL) receiving samples,
 * look-ups, rays hit and the device status word (0 ok, 1 bounds, 2 timeout).
 * The first call on each device looks up the array's device address with
 * that device current (make that first call before any stream capture); the
 * address is kept for the life of the process, so a caller that resets the
 * device (cudaDeviceReset) must not call this function afterwards.
 * Each call clears the scratch on `stream` first; all calls share the one
 * array and it keeps the last call's contents, so calls that overlap on the
 * GPU (other streams, other threads) race on it.  An empty row band
 * (row_begin == row_end != 0) launches no kernel and reports zero counters.
 * Sizes: one call uses 72 of the 256 bytes (8 counter slots and the status
 * word), whatever the image size; the maximum image is 32768 x 32768 (as for
 * lrvol_render), larger ones are rejected with LRVOL_ERR_ARG.  Other errors:
 * as lrvol_render. */
int lrvol_render_noalloc(lrvol_t vol, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                         float *rgba_dev, uint64_t *counters_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Learned step sizes.  The paper's Eq. 4 step is multiplied per element by
 * m = 2^clamp(y, ymin, ymax), y the output of a small network run once per
 * element and frame on 16 block-local features; LRVOL_STEP_LEARNED renders
 * with these multipliers (ymin < 0 lets the network refine below Eq. 4 where
 * Eq. 4 is too coarse for the transfer function, ymax > 0 lets it stretch).  Network: 16 -> 64 -> 64 -> 64 -> 1, ReLU on the
 * hidden layers.  FP32 master parameters (LRVOL_MLP_PARAMS floats) are laid
 * out W1[16][64], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4
 * (W[in][out], row major).  The paper has no learned component; Eq. 4 stays
 * the fallback (all multipliers 1).
 * ------------------------------------------------------------------------- */
#define LRVOL_MLP_IN 16
#define LRVOL_MLP_HIDDEN 64
#define LRVOL_MLP_PARAMS 9473
#define LRVOL_MLP_PACKED 10120 /* uint16 entries: BF16 tensor-core operands, BF16 w4, FP32 biases */

/* Features of every element for a camera and transfer function, n_elem x 16
 * floats into feat_dev (device).  With w the element's sides, [cmin, cmax] the
 * range of the rendered field on the element (from its Bezier block: the
 * coefficient range for a component, bounds of |v| for the magnitude) and x =
 * (c - vmin)/(vmax - vmin) the TF coordinate:
 *   0..2  log2(64 w_a)
 *   3, 4  x(cmin), x(cmax);  5  x(cmax) - x(cmin)
 *   6, 7  max and mean TF alpha over the entries floor(255 x(cmin)) ..
 *         ceil(255 x(cmax)) (coordinates clamped to [0, 1])
 *   8     255 * max |alpha[i+1] - alpha[i]| over those entries
 *   9     max over R, G, B of (max - min) over those entries
 *   10..12  unit direction from the eye to the element centre
 *   13    log2(2048 ds), ds the element's Eq. 4 step
 *   14    (|d_x| w_x + |d_y| w_y + |d_z| w_z) / (8 ds), d the direction above
 *   15    log2(1 + 255 (x(cmax) - x(cmin)))
 * Needs to_bezier.  Field and component come from `step`. */
int lrvol_features(lrvol_t vol, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                   float *feat_dev, void *stream);

/* Pack FP32 master parameters (device, LRVOL_MLP_PARAMS floats) into the
 * layout lrvol_mlp_infer reads (device, LRVOL_MLP_PACKED uint16,
 * caller-owned): W1..W3 as BF16 tensor-core B operands in shared-memory
 * order, w4 in BF16, the biases in FP32.  The layout is private to the
 * library; treat the buffer as opaque. */
int lrvol_mlp_pack(const float *params_dev, uint16_t *packed_dev, void *stream);

/* Network forward for n feature rows (device, n x 16); writes out_dev[n] =
 * 2^clamp(y, ymin, ymax).  The three hidden layers run on the 5th-generation
 * tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32 accumulators in
 * tensor memory, 128 rows per tile); the features and hidden activations are
 * rounded to BF16 as MMA operands, biases are added in FP32, and the 64 -> 1
 * output layer is an FP32 dot product of the BF16 activations and BF16 w4.
 * ymin in [-8, 0], ymax in [0, 8]; packed_dev 16-byte aligned (it is read in
 * 16-byte words).
 * The kernel's waits for the tensor cores are bounded: if one runs out (not
 * expected), the rows of the tiles it leaves get multiplier 1 (the Eq. 4
 * step) and the library's network status records it for lrvol_mlp_check. */
int lrvol_mlp_infer(const float *feat_dev, int64_t n, const uint16_t *packed_dev, float ymin, float ymax,
                    float *out_dev, void *stream);

/* Synchronises the device and reports the network status of every
 * lrvol_mlp_infer since the last check: LRVOL_OK, or LRVOL_ERR_TIMEOUT if a
 * tensor-core wait ran out (the status is then cleared). */
int lrvol_mlp_check(void);

/* Diagnostic of the timeout path: lrvol_mlp_infer with no MMAs issued, so
 * every tile's bounded wait runs out (after at most 0.1 s per wait) and
 * out_dev[0..n) becomes 1; lrvol_mlp_check then reports LRVOL_ERR_TIMEOUT.
 * n in 1 .. 2^20. */
int lrvol_mlp_infer_timeout_test(const float *feat_dev, int64_t n, const uint16_t *packed_dev, float ymin,
                                 float ymax, float *out_dev, void *stream);

/* FP32 training step of the network on a batch (device): loss = mean over
 * rows of (y - target)^2 / 2.  lrvol_mlp_grad writes the gradient
 * (LRVOL_MLP_PARAMS floats) and the loss (1 float); lrvol_mlp_train_step then
 * applies Adam (beta1 0.9, beta2 0.999, eps 1e-8, step count t >= 1) to params
 * with moment buffers m, v (LRVOL_MLP_PARAMS floats each, zero at t = 1).
 * scratch_dev must hold lrvol_mlp_scratch_floats(n) floats (activations, their
 * gradients and one gradient vector).  Batch n in 1 .. 2^20. */
int64_t lrvol_mlp_scratch_floats(int64_t n);
int lrvol_mlp_grad(const float *x_dev, const float *target_dev, int64_t n, const float *params_dev, float *grad_dev,
                   float *loss_dev, float *scratch_dev, void *stream);
int lrvol_mlp_train_step(const float *x_dev, const float *target_dev, int64_t n, float *params_dev, float *m_dev,
                         float *v_dev, int64_t t, float lr, float *loss_dev, float *scratch_dev, void *stream);

/* Training labels from fine-step samples (scalar volumes).  Every ray of the
 * camera is marched with Eq. 4 steps; a visit of element e starts at the
 * first heuristic sample in e, t_a, and ends at the first one past it, t_b.
 * Candidate i marches from t_a with the step s_i = cand[i]*ds(e) (FP32
 * product), samples fmaf(k, s_i, t_a), until its first sample outside e (or
 * the ray's exit), t_i.  Over [t_a, t_i) Alg. 2 is run from transparent with
 * the step s_i and with the fixed fine step h_fine (reference), every sample
 * evaluated in the element that holds it; the error of candidate i is
 * T_front * max(|dC_r|, |dC_g|, |dC_b|, |d alpha|), T_front the reference
 * transmittance of the ray in front of t_a (fine-step composites of the
 * earlier visits [t_a, t_b)).  For every visited element, label_dev[e]
 * becomes min(label_dev[e], the largest i such that candidates 1..i all have
 * error <= tau), so the caller initialises label_dev (n_elem int32) to
 * n_cand.  Needs to_bezier with LRVOL_STORE_F32 and build_accel.  cand_dev:
 * 1..16 increasing multipliers on the device (read back during the call);
 * cand[0], the smallest, is always accepted (1 keeps every step at least the
 * Eq. 4 step; a value below 1 lets labels ask for finer steps than Eq. 4).
 * A ray stops when its reference transmittance is <= 1 - step->alpha_stop. */
int lrvol_labels(lrvol_t vol, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step, double h_fine,
                 double tau, const float *cand_dev, int32_t n_cand, int32_t *label_dev, void *stream);

/* Element look-up through the forest (Alg. 1) for n FP32 points (n x 3,
 * device) into elem_dev (n uint32, device).  Needs build_accel. */
int lrvol_lookup(lrvol_t vol, const float *pts_dev, int64_t n, uint32_t *elem_dev, void *stream);

/* Field values (Eq. 2 through the Bezier blocks, FP32) at n FP32 points into
 * val_dev (n x ncomp floats, device).  Needs build_accel and to_bezier. */
int lrvol_eval(lrvol_t vol, const float *pts_dev, int64_t n, float *val_dev, void *stream);

/* Value and gradient of a scalar volume at n points (device, n x 3 floats):
 * val_grad_dev n x 4 floats (f, df/dx, df/dy, df/dz), evaluated from the
 * element's render block as the renderer's gradient shading does (the
 * derivative of the Bezier tensor polynomial, scaled by 1/(hi - lo) per
 * axis).  Points outside [0,1]^3 give zeros.  LRVOL_ERR_UNSUPPORTED for
 * vector volumes. */
int lrvol_eval_grad(lrvol_t vol, const float *pts_dev, int64_t n, float *val_grad_dev, void *stream);

/* Copy the FP64 Bezier blocks to host_out: n_elem x ncomp x (p3+1) x (p2+1)
 * x (p1+1) doubles, x index fastest.  Synchronous. */
int lrvol_get_bezier(lrvol_t vol, double *host_out);

/* ---------------------------------------------------------------------------
 * Trimming by a boundary mesh (Sec. 4.1), the two depth buffers of a
 * z-prepass computed by ray casting: for every pixel ray (as lrvol_render
 * generates it), t_front = the nearest hit on a front face (+inf if none)
 * and t_back = the farthest hit on a back face (0 if none), hits at t <= 0
 * ignored.  Triangles are counter-clockwise seen from outside; a face is
 * front-facing when the ray sees that winding.  Hits are decided by the
 * watertight ray/triangle test of Woop, Benthin and Wald (JCGT 2013) in FP32,
 * retrying an edge function that is exactly 0 in FP64, so rays through
 * shared edges and vertices are not lost.  A warp sets up 32 triangles, one
 * per lane, and tests the pixel rays of their conservative screen boxes
 * (pixel centres within 1/4 pixel of the projected box) 32 at a time.
 * tri_dev: n_tri x 9 floats (device); trim_dev: height x width x 2 floats
 * (device, overwritten).  The camera's row range is ignored.
 * ------------------------------------------------------------------------- */
int lrvol_trim(const lrvol_camera *cam, const float *tri_dev, int64_t n_tri, float *trim_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Streamlines of a 3-vector volume (Sec. 5): dx/dt = f(x) from each seed by
 * an explicit Runge-Kutta method (Eq. 5).  The outer loop accumulates x in
 * more than FP32 precision (an unevaluated pair of floats, about 48
 * significant bits) and t in FP64; f is evaluated in FP32 at the FP32
 * rounding of each stage point (the paper's mixed precision, Sec. 5.5).
 * Steps: FIXED h; HEURISTIC h times the Eq. 4 step of the element holding
 * the FP32 rounding of x_n (Sec. 5.2; h is the base factor); ADAPTIVE (the
 * embedded pairs only): the step after an accepted or rejected attempt is
 * h * clamp(0.9 (tol/err)^(1/(q+1)), 0.2, 5), err = |h sum (b_i - b^_i) k_i|,
 * q the lower order, accept when err <= tol, first step h (0 = Eq. 4), at
 * most 64 attempts per step.  The last step is clipped to end at t_end.
 * A streamline stops at t_end (status 0), when a stage point or the next
 * point leaves [0,1]^3 (status 1; the point before is the last sample),
 * after max_samples samples (2), or when the step control gives up (3).
 * One thread traces one line at a time; a grid that fits on the GPU at once
 * takes the seeds from a counter in the handle, so concurrent streamline
 * calls on one handle are not allowed (as for every call on a handle).
 * With fewer seeds than the GPU holds warps, each warp traces fewer than 32
 * lines (down to one), so a small rake is not slowed by warp-mates' element
 * look-ups; the samples are the same whatever the number of seeds.  The
 * call returns when its kernels are queued; samples, counts and statuses are
 * valid once the stream reaches that point.
 * ------------------------------------------------------------------------- */
enum {
  LRVOL_RK1 = 0,   /* explicit Euler */
  LRVOL_RK2 = 1,   /* explicit midpoint */
  LRVOL_RK3 = 2,   /* Kutta's third-order method */
  LRVOL_RK4 = 3,   /* classic fourth order */
  LRVOL_RK38 = 4,  /* 3/8 rule */
  LRVOL_RKF5 = 5,  /* Fehlberg's fifth-order solution */
  LRVOL_HE = 6,    /* Heun-Euler 2(1), second order propagated */
  LRVOL_BS = 7,    /* Bogacki-Shampine 3(2), third order propagated */
  LRVOL_RKF45 = 8  /* Fehlberg 4(5), fifth order propagated */
};
enum { LRVOL_SL_FIXED = 0, LRVOL_SL_HEURISTIC = 1, LRVOL_SL_ADAPTIVE = 2 };

typedef struct {
  int32_t method;      /* LRVOL_RK1 .. LRVOL_RKF45 */
  int32_t step_rule;   /* LRVOL_SL_* */
  double h;            /* FIXED: step (> 0); HEURISTIC: factor on Eq. 4 (> 0); ADAPTIVE: first step, 0 = Eq. 4 */
  double t_end;        /* > 0 */
  double tol;          /* ADAPTIVE: local error tolerance (> 0, parameter-space units) */
  int32_t max_samples; /* >= 1, per streamline, the seed included */
} lrvol_streamline_params;

/* n seeds (device, n x 3 doubles) -> samples_dev (n x max_samples x 4
 * doubles: x, y, z, t; the seed first at t = 0), count_dev (n int32:
 * samples written), status_dev (n int32).  Needs build_accel and to_bezier,
 * ncomp 3, equal degrees 1..3; any block storage.  Seeds outside [0,1]^3
 * give count 0 and status 1. */
int lrvol_streamlines(lrvol_t vol, const lrvol_streamline_params *params, const double *seeds_dev, int64_t n,
                      double *samples_dev, int32_t *count_dev, int32_t *status_dev, void *stream);

/* Streamline tubes (Sec. 5.3): every segment of the polylines that
 * lrvol_streamlines wrote (samples_dev, count_dev; max_samples per line) is
 * drawn as a capsule of the given radius around the segment (endpoints
 * rounded to FP32).  Visibility is decided in FP32: per pixel the hit with
 * the smallest t wins, ties going to the earlier segment (line by line, in
 * order).  The pixel then takes the colour map's RGB at the speed |f| of the
 * volume at the closest point on the winning segment's axis, times
 * I = max(0.4, |n . d|), n the capsule normal at the hit; alpha 1; pixels
 * without a hit are (0, 0, 0, 0).  A warp walks a line's segments 32 at a
 * time, one per lane, and tests the pixel rays of their conservative screen
 * boxes 32 at a time; hits merge by a 64-bit atomic minimum of
 * (t bits, segment index) in vis_dev (height x width uint64 scratch,
 * caller-owned), then one thread per pixel shades the winner into rgba_dev
 * (height x width x 4 floats).  Needs a 3-vector volume (build_accel,
 * to_bezier); n_lines * (max_samples - 1) < 2^32. */
int lrvol_tubes(lrvol_t vol, const lrvol_camera *cam, const double *samples_dev, const int32_t *count_dev,
                int64_t n_lines, int32_t max_samples, float radius, const lrvol_tf *cmap, uint64_t *vis_dev,
                float *rgba_dev, void *stream);

/* Eq. 7 per streamline (device): sums_dev[j] = sum over the approximation's
 * samples i >= 1 of (t_i - t_{i-1}) |x_j(t_i) - y_j(t_i)|_2, the reference
 * x_j linear between its samples; samples past the reference's last time
 * are left out.  Layouts as lrvol_streamlines writes them (ref_max and
 * app_max samples per line).  The metric E is the maximum of the sums. */
int lrvol_streamline_error(const double *ref_dev, const int32_t *ref_count_dev, int32_t ref_max,
                           const double *app_dev, const int32_t *app_count_dev, int32_t app_max, int64_t n,
                           double *sums_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Host-side arena bookkeeping (first fit, coalescing): offsets into a range
 * of `bytes`, every block aligned to `align` (a power of two).  The frame
 * server below carves its output images from one device allocation with it;
 * the functions touch no device memory.  Not thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct lrvol_arena_s *lrvol_arena_t;
int lrvol_arena_create(int64_t bytes, int64_t align, lrvol_arena_t *out);
/* Offset of a free block of at least `bytes` (the lowest that fits), or -1. */
int64_t lrvol_arena_alloc(lrvol_arena_t a, int64_t bytes);
/* Return a block by the offset lrvol_arena_alloc gave; LRVOL_ERR_ARG if none. */
int lrvol_arena_free(lrvol_arena_t a, int64_t offset);
/* Bytes in use (rounded up to the alignment) and the largest free block. */
int64_t lrvol_arena_used(lrvol_arena_t a);
int64_t lrvol_arena_largest_free(lrvol_arena_t a);
void lrvol_arena_destroy(lrvol_arena_t a);

/* ---------------------------------------------------------------------------
 * Frame server: continuous batching of frame requests over resident volumes
 * (the paper renders one interactive view; it has no counterpart).
 *
 * A server owns `slots` slots (each three CUDA streams of different
 * priority, two events and statistics counters) and one device arena of `arena_bytes`
 * for output images (and, for learned steps, per-frame features and
 * multipliers).  lrvol_server_submit queues a request and returns at once.
 * lrvol_server_progress, called from the host loop, first retires the
 * frames whose work has finished, then admits waiting requests while a slot
 * is free and the arena holds the request's memory, launching each on its
 * slot's stream: frames of different requests run concurrently on the
 * device.  Admission is FIFO.  With size tiers on (see
 * lrvol_server_set_priority_pixels) it is FIFO within each tier, smaller
 * tiers are served first, and the tier of the largest frames holds at most
 * slots - max(1, slots/4) slots; a request that does not fit waits at the
 * head of its tier while smaller tiers may go ahead.  Results are
 * identical to lrvol_render of the same request alone: the same kernel with
 * the same parameters, and statistics counters of its own.
 *
 * All calls on one server must come from one host thread.  Volumes must stay
 * alive while requests on them are queued or running.
 * ------------------------------------------------------------------------- */
typedef struct lrvol_server_s *lrvol_server_t;

enum { LRVOL_REQ_QUEUED = 0, LRVOL_REQ_RUNNING = 1, LRVOL_REQ_DONE = 2, LRVOL_REQ_FAILED = 3 };

typedef struct {
  int32_t state;                 /* LRVOL_REQ_* */
  int32_t status;                /* LRVOL_OK, or the error of a failed request */
  const float *rgba_dev;         /* DONE: the image (height x width x 4) in the arena, until released;
                                    NULL once released or when the request copied to host_out */
  double t_submit, t_admit, t_done; /* lrvol_server_clock() at submission, launch, and when progress
                                    saw the frame finished (0 while not reached) */
  float device_ms;               /* between events recorded before and after the frame's work */
  float dev_start_ms, dev_end_ms; /* those events relative to one recorded at server creation: frames
                                    whose [start, end] intervals intersect ran concurrently */
  int64_t samples, lookups, rays_hit; /* counters of this frame's render */
  int64_t bytes;                 /* arena bytes the request holds while admitted */
} lrvol_frame_info;

typedef struct {
  int64_t submitted, queued, running, done, failed;
  int64_t arena_bytes, arena_used, arena_high_water;
  int32_t slots, max_running;    /* max_running: most frames in flight at once so far */
} lrvol_server_stats;

/* slots 1..64, arena_bytes >= 1 MiB (allocated here, once).  The arena and
 * the slot streams live until lrvol_server_destroy. */
int lrvol_server_create(int32_t slots, int64_t arena_bytes, lrvol_server_t *out);
/* Attach a learned step model for requests with mode LRVOL_STEP_LEARNED and
 * mult == NULL: the server then runs lrvol_features and lrvol_mlp_infer for
 * the request's volume and camera before its render, on the same stream, with
 * the features and multipliers in the arena.  packed_dev (LRVOL_MLP_PACKED
 * uint16, 16-byte aligned) stays caller-owned and must outlive the server;
 * ymin and ymax as for lrvol_mlp_infer. */
int lrvol_server_set_step_model(lrvol_server_t s, const uint16_t *packed_dev, float ymin, float ymax);
/* Stream priority tiers by frame size: frames of at most max_pixels pixels
 * run at the device's greatest stream priority, frames of at most
 * 4 * max_pixels at a middle one, larger frames at the least, so the block
 * scheduler dispatches the CTAs of smaller frames ahead of those of larger
 * frames already running.  0 (the default) puts every frame in the last
 * tier.  Each slot holds one stream per tier (3 x slots streams): a process
 * that serves should set CUDA_DEVICE_MAX_CONNECTIONS to at least that many
 * (at most 32) before its CUDA context exists, or streams share hardware
 * queues and a small frame can wait behind a large one. */
int lrvol_server_set_priority_pixels(lrvol_server_t s, int64_t max_pixels);
/* With size tiers on: at most max_in_flight frames of the largest tier run at
 * once (0, the default: slots - max(1, slots/4)).  Large frames each fill
 * the GPU; running fewer of them side by side shortens each one's latency
 * without lowering throughput. */
int lrvol_server_set_large_cap(lrvol_server_t s, int32_t max_in_flight);
/* Queue one frame.  cam, tf and step are copied.  host_out: NULL, or a host
 * buffer (pinned for an asynchronous copy) of height x width x 4 floats that
 * receives the image as part of the frame's work; the arena memory is then
 * returned when the frame retires.  Without host_out the image stays in the
 * arena until lrvol_server_release.  Errors: LRVOL_ERR_ARG for requests that
 * fail lrvol_render's checks or that need more memory than the whole arena. */
int lrvol_server_submit(lrvol_server_t s, lrvol_t vol, const lrvol_camera *cam, const lrvol_tf *tf,
                        const lrvol_step *step, float *host_out, int64_t *ticket);
/* Retire finished frames, then admit and launch waiting requests.  Never
 * waits for the device.  n_retired (may be NULL) receives the number of
 * frames retired by this call. */
int lrvol_server_progress(lrvol_server_t s, int32_t *n_retired);
/* Block until every submitted request is done or failed (progress in a loop;
 * waits on the oldest running frame's event between rounds). */
int lrvol_server_drain(lrvol_server_t s);
/* Tickets of requests that became done or failed since the previous call, in
 * the order they were retired (at most max_n; the rest stay for the next
 * call).  *n receives the count. */
int lrvol_server_poll(lrvol_server_t s, int64_t *tickets, int32_t max_n, int32_t *n);
int lrvol_server_info(lrvol_server_t s, int64_t ticket, lrvol_frame_info *info);
/* Forget a finished request and return its arena memory (LRVOL_ERR_STATE while
 * it is queued or running). */
int lrvol_server_release(lrvol_server_t s, int64_t ticket);
int lrvol_server_get_stats(lrvol_server_t s, lrvol_server_stats *out);
/* The host clock of the t_* fields: seconds of a monotonic clock. */
double lrvol_server_clock(void);
/* Synchronises the slot streams, then frees the arena, streams and events. */
void lrvol_server_destroy(lrvol_server_t s);

/* Statistics of the forest and of the last render.  Synchronous; also
 * reports a pending device-side status (LRVOL_ERR_BOUNDS / _TIMEOUT). */
int lrvol_stats(lrvol_t vol, lrvol_stats_t *out);

const char *lrvol_status_string(int status);
const char *lrvol_last_error(void);

/* Release all device memory of the handle (synchronises the device first). */
void lrvol_destroy(lrvol_t vol);

#ifdef __cplusplus
}
#endif
#endif /* LRVOL_H */
