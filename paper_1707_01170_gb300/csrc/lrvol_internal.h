// Internal declarations of liblrvol (host code and kernels).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "lrvol.h"

namespace lrvol {

constexpr uint32_t kLeaf = 0x80000000u;   // forest reference: bit 31 set = element id in bits 0..30
constexpr uint32_t kNone = 0xFFFFFFFFu;   // "no element"
constexpr int kMaxDepth = 96;             // traversal bound: a deeper tree is reported as LRVOL_ERR_BOUNDS
constexpr int kMaxDeg = 4;
constexpr int kMaxSamplesPerRay = 1 << 24;  // a longer ray stops with LRVOL_ERR_TIMEOUT

// Device status word values (first error wins).
enum : uint32_t { kStatusOk = 0, kStatusBounds = 1, kStatusTimeout = 2 };

// Counters written by render (one slot each).
enum { kCntSamples = 0, kCntLookups = 1, kCntRays = 2, kCntQueue = 3, kNumCounters = 8 };

// Static scratch of lrvol_render_noalloc: kNumCounters counters, then the
// status word (in a 64-bit slot); 32 words = 256 bytes per device.  One call
// uses kNumCounters + 1 words (72 bytes), whatever the image size.
constexpr int kStaticScratchWords = 32;
constexpr int kStaticScratchBytesPerCall = (kNumCounters + 1) * 8;
static_assert(kNumCounters + 1 <= kStaticScratchWords, "static scratch too small for one render");
static_assert(kStaticScratchBytesPerCall == 72 && kStaticScratchWords * 8 == 256,
              "lrvol.h states 72 of 256 bytes per lrvol_render_noalloc call");
constexpr int kMaxImageSide = 32768;  // largest width or height a render accepts

// Element record, 4 x float4 = 64 bytes:
//   a = {lo_ru.x, lo_ru.y, lo_ru.z, ds}   lower corner rounded up to FP32 (membership), Eq. 4 step
//   b = {hi_ru.x, hi_ru.y, hi_ru.z, 0}    upper corner rounded up (+inf where hi = 1)
//   c = {off.x, off.y, off.z, 0}          (float)((lo_ru - lo) / (hi - lo)) >= 0, from FP64
//   d = {iw.x, iw.y, iw.z, 0}             (float)(1 / (hi - lo))
// Local coordinate u = fma(p - lo_ru, iw, off).
struct ElemRec {
  float4 a, b, c, d;
};

// Forest node, 16 bytes: split value (FP32, rounded up), axis, child refs for
// p[axis] < split and p[axis] >= split.  A ref with kLeaf set names an element.
struct Node {
  uint32_t split_bits;
  uint32_t axis;
  uint32_t child[2];
};

struct ForestView {
  const uint32_t *head;  // blocks[2] x blocks[1] x blocks[0], x fastest
  const uint4 *nodes;
  int64_t n_nodes;
  int bx, by, bz;        // block counts (powers of two)
  float fbx, fby, fbz;
};

struct RayConsts {
  float E[3], F[3], R[3], U[3];
  float sxs, sxo, sys, syo;
  int persp;
};

// Render layout of one element's Bezier block (binomials folded in),
// arranged for packed two-lane FP32 arithmetic (fma.rn.f32x2) and 256-bit
// loads.  Values sit in "slots":
//   Scalar volumes (nc = 1): rows r = k*(p1+1) + j of (p0+1) values, stored
//     in pairs: value i of rows 2m and 2m+1 side by side,
//     slot(r, i) = (r >> 1) * 2*(p0+1) + 2*i + (r & 1).
//   Vector volumes (nc = 3): with q = r*(p0+1) + i, components 0 and 1
//     interleaved, slot(q, c) = 2q + c (c = 0, 1), then component 2 at
//     pair_slots + q, pair_slots = roundup8(2*nb).  These volumes also keep
//     a plain copy for component renders: component c at c*roundup8(nb) + q.
// Storage: FP32 slots (4 bytes each); or FP16/BF16 slots (2 bytes each) after
// a 32-byte header of FP32 offsets o[3] and scales s[3], holding
// q' = (c' - binomial*o)/s, so a component's value is o + s * contraction(q').
// Element strides are multiples of 32 bytes.
__host__ __device__ inline int roundup8(int x) { return (x + 7) & ~7; }
__host__ __device__ inline int roundup32(int x) { return (x + 31) & ~31; }
__host__ __device__ inline int render_pair_slots(int nb) { return roundup8(2 * nb); }
__host__ __device__ inline int render_slots(int nc, int n0, int n1, int n2) {
  const int nb = n0 * n1 * n2;
  if (nc == 1) return roundup8(((n1 * n2 + 1) / 2) * 2 * n0);
  return render_pair_slots(nb) + roundup8(nb);
}
__host__ __device__ inline int render_slot(int nc, int n0, int nb, int r, int i, int c) {
  if (nc == 1) return (r >> 1) * 2 * n0 + 2 * i + (r & 1);
  const int q = r * n0 + i;
  return c < 2 ? 2 * q + c : render_pair_slots(nb) + q;
}
constexpr int kHeaderBytes = 32;  // FP32 o[3], s[3], 2 unused (16-bit storage only)
__host__ __device__ inline int slot_bytes(int storage) { return storage == LRVOL_STORE_F32 ? 4 : 2; }
__host__ __device__ inline int header_bytes(int storage) { return storage == LRVOL_STORE_F32 ? 0 : kHeaderBytes; }
__host__ __device__ inline int elem_bytes(int storage, int slots) {
  return roundup32(header_bytes(storage) + slot_bytes(storage) * slots);
}

// Field code of launch_render for a scalar volume rendered with gradient
// shading (the public LRVOL_FIELD_* codes are 0..2).
constexpr int kFieldShaded = 3;

struct RenderParams {
  const ElemRec *elem;
  int64_t n_elem;
  const unsigned char *bez;   // render blocks (layout above)
  int elem_bytes;             // bytes per element
  const unsigned char *bezc;  // vector volumes: plain per-component copy
  int elemc_bytes;            // bytes per element of bezc
  int comp;               // component evaluated (FIELD_COMPONENT)
  ForestView forest;
  float *out;
  int width, height, row_begin, row_end;
  int band_count, band_index;  // interleaved LRVOL_BAND_ROWS-row bands (count >= 1)
  RayConsts ray;
  int mode;               // LRVOL_STEP_*
  const float *mult;      // LEARNED: per-element step multipliers
  float h, inv_xi, alpha_stop;
  float tf_scale, tf_bias; // x = v * tf_scale + tf_bias, clamped to [0, 255]
  const float2 *trim;     // NULL or per pixel (t_front, t_back), row major over the full image
  int light_set;          // shading: 1 = light[] (unit), 0 = towards the eye along the ray
  float light[3];
  float grad_eps;         // shading: gradients below this count as none (1e-3 (vmax - vmin))
  unsigned long long *counters;
  uint32_t *status;
  // lrvol_render_trace only (null / 0 in every product launch)
  const int32_t *trace_pix;  // trace_n (i, j) pixel pairs
  int64_t trace_n;
  int trace_max;             // records kept per pixel
  float4 *trace_rec;         // trace_n x trace_max (t, element id bits, value, segment)
  int32_t *trace_count;      // per pixel: samples composited
  float4 *trace_rgba;        // per pixel: the composited RGBA
  float4 tf[256];
};

struct Volume;

}  // namespace lrvol

struct lrvol_s {
  int device = 0;
  int p[3] = {0, 0, 0};
  int nc = 1;
  int64_t n_elem = 0, n_basis = 0;
  int kw = 0;  // knots per B-spline
  std::vector<double> box, knots, coef, weight;

  // device copies of the spline
  double *d_box = nullptr, *d_knots = nullptr, *d_coef = nullptr, *d_weight = nullptr;
  // change of basis
  int64_t *d_inc_ptr = nullptr;
  int32_t *d_inc_idx = nullptr;
  int64_t inc_entries = 0;
  double *d_bez64 = nullptr;
  unsigned char *d_bez = nullptr;   // render blocks in `storage`
  unsigned char *d_bezc = nullptr;  // vector volumes: plain per-component copy
  int elem_bytes = 0, elemc_bytes = 0;
  int storage = -1;
  float2 *d_range = nullptr;  // per element and component: coefficient min, max
  lrvol::ElemRec *d_elem = nullptr;
  bool have_bezier = false;
  // forest
  uint32_t *d_head = nullptr;
  uint4 *d_nodes = nullptr;
  int64_t n_nodes = 0;
  int blocks[3] = {0, 0, 0};
  int depth_min = 0, depth_max = 0;
  double depth_mean = 0, depth_var = 0;
  bool have_accel = false;
  // scratch
  unsigned long long *d_counters = nullptr;
  uint32_t *d_status = nullptr;
  int64_t bytes_device = 0;                                 // sum of the live allocations below
  std::unordered_map<const void *, int64_t> alloc_bytes;    // size of each live device allocation
};

namespace lrvol {

// kernels.cu
cudaError_t launch_to_bezier(const lrvol_s *v, cudaStream_t s);
cudaError_t launch_pack(const lrvol_s *v, cudaStream_t s);
cudaError_t launch_elem_records(const lrvol_s *v, cudaStream_t s);
cudaError_t launch_lookup(const lrvol_s *v, const float *pts, int64_t n, uint32_t *out, cudaStream_t s);
cudaError_t launch_eval_grad(const lrvol_s *v, const float *pts, int64_t n, float *out, cudaStream_t s);
cudaError_t launch_eval(const lrvol_s *v, const float *pts, int64_t n, float *out, cudaStream_t s);
cudaError_t launch_render(const RenderParams &prm, int degree, int field, int storage, cudaStream_t s);
cudaError_t launch_render_trace(const RenderParams &prm, int degree, int field, int storage, cudaStream_t s);
cudaError_t launch_render_static(RenderParams prm, int degree, int field, int storage, cudaStream_t s,
                                 unsigned long long *counters_out);

// host.cpp
void camera_consts(const lrvol_camera *c, RayConsts *k);
ForestView forest_view(const lrvol_s *v);

}  // namespace lrvol

namespace lrvol {

// Learned step sizes (lrvol.h): parameter offsets of the FP32 master vector
constexpr int kIn = 16, kHid = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kIn * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid, kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kHid,
              kParams = kOffB4 + 1;
// Packed weights (uint16 offsets).  W1, W2, W3 as BF16 tensor-core B operands
// (N = 64 rows of K, K-major, in the canonical no-swizzle layout of 8-row x
// 16-byte core matrices, see tc_off), then w4 as 64 BF16 values, then the FP32
// biases b1, b2, b3, b4 as pairs of uint16 (low half first), zero padding to
// the ABI size.
constexpr int kTcW1 = 0, kTcW2 = kTcW1 + kHid * kIn, kTcW3 = kTcW2 + kHid * kHid, kTcW4 = kTcW3 + kHid * kHid,
              kTcBias = kTcW4 + kHid, kTcEnd = kTcBias + 2 * (3 * kHid + 1), kPacked = 10120;
static_assert(kParams == 9473, "parameter count");
static_assert(kTcEnd <= kPacked && (kTcBias * 2) % 4 == 0, "packed layout");

// Byte offset of element (r, k) of a K-major BF16 operand with K columns in the
// canonical no-swizzle layout: 8x8 core matrices (8 rows of 16 bytes, 128
// contiguous bytes); core matrices adjacent in K are 128 B apart (the
// descriptor's leading byte offset), 8-row groups K * 16 B apart (its stride
// byte offset).
__host__ __device__ constexpr int tc_off(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
static_assert(tc_off(1, 0, 64) == 16 && tc_off(0, 1, 64) == 2 && tc_off(0, 8, 64) == 128 && tc_off(8, 0, 64) == 1024 &&
                  tc_off(127, 63, 64) == 128 * 64 * 2 - 2 && tc_off(127, 15, 16) == 128 * 16 * 2 - 2,
              "canonical operand layout");

struct FeatureParams {
  const double *box;
  const ElemRec *elem;
  const float2 *range;  // per element and component: coefficient min, max (rounded outward)
  int64_t n_elem;
  int nc, field, comp;
  float eye[3];
  float tf_scale, tf_bias;  // x = v * scale + bias in TF entries (0..255)
  float4 tf[256];
};

cudaError_t launch_features(const FeatureParams &fp, float *out, cudaStream_t s);

// Trimming (Sec. 4.1)
cudaError_t launch_trim(const RayConsts &ray, int width, int height, const float *tri, int64_t n_tri, float *out,
                        cudaStream_t s);

// Streamlines (Sec. 5)
struct SLParams {
  const ElemRec *elem;
  int64_t n_elem;
  const unsigned char *bez;
  int elem_bytes;
  ForestView forest;
  uint32_t *status;   // device status word (bounds)
  unsigned long long *queue;  // streamlines: next seed to trace (zeroed per call)
  int method, rule, max_samples;
  double h, t_end;
  float tol_f;
  bool pair_out;      // streamlines: store float pairs, widened to FP64 by a second pass
};
cudaError_t launch_streamlines(const SLParams &sp, int degree, int storage, const double *seeds, int64_t n,
                               double *out, int32_t *count, int32_t *status, cudaStream_t s);
struct TubeParams {
  SLParams field;          // volume access for the speed at the axis point
  RayConsts ray;
  int width, height;
  float radius;
  const double *samples;   // n_lines x max_samples x 4
  const int32_t *count;
  int64_t n_lines;
  int max_samples;
  unsigned long long *vis; // height x width
  float *out;              // height x width x 4
  float tf_scale, tf_bias;
  float4 cmap[256];
};
cudaError_t launch_tubes(const TubeParams &tp, int degree, int storage, cudaStream_t s);
cudaError_t launch_streamline_error(const double *ref, const int32_t *rc, int rmax, const double *app,
                                    const int32_t *ac, int amax, int64_t n, double *sums, cudaStream_t s);

// host.cpp: error reporting (sets the thread's last error, returns the status)
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
// host.cpp: the checks and kernel parameters of lrvol_render (scratch
// pointers left null) and of lrvol_features
int prepare_render(const lrvol_s *v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                   float *rgba_dev, RenderParams *prm, int *field_out);
int prepare_features(const lrvol_s *v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                     FeatureParams *fp);

#define CU(call, what)                                        \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::lrvol::cuda_fail(_e, what); \
  } while (0)
cudaError_t launch_mlp_pack(const float *params, uint16_t *packed, cudaStream_t s);
// status: device word that records LRVOL_ERR_TIMEOUT-class failures (kStatusTimeout) of the kernel's bounded waits
// no_mma: diagnostic of the timeout path (no MMAs issued, every wait runs out)
cudaError_t launch_mlp_infer(const float *x, int64_t n, const uint16_t *packed, float ymin, float ymax, float *out,
                             uint32_t *status, cudaStream_t s, bool no_mma = false);
// the library's status word for lrvol_mlp_infer calls (device address)
uint32_t *mlp_status_word();
cudaError_t launch_mlp_grad(const float *x, const float *target, int64_t n, const float *params, float *grad,
                            float *loss, float *scratch, cudaStream_t s);
cudaError_t launch_adam(float *params, const float *grad, float *m, float *v, int64_t t, float lr, cudaStream_t s);
cudaError_t launch_labels(const RenderParams &prm, int degree, float h_fine, float tau, const float *cand, int n_cand,
                          int32_t *label, cudaStream_t s);

}  // namespace lrvol
