// liblrvol host side: the C ABI of lrvol.h, input validation, the
// element-to-B-spline incidence used by the change of basis, and the k-d
// forest build (Sec. 3.2.1).  Every per-sample computation runs in kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "lrvol_internal.h"

using namespace lrvol;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace lrvol {

int fail(int status, const std::string &msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? LRVOL_ERR_OOM : LRVOL_ERR_CUDA;
}

}  // namespace lrvol

namespace {

template <class T>
int dev_alloc(lrvol_s *v, T **p, size_t count, const char *what) {
  if (*p) {   // a rebuild replaces the buffer
    auto it = v->alloc_bytes.find(*p);
    if (it != v->alloc_bytes.end()) {
      v->bytes_device -= it->second;
      v->alloc_bytes.erase(it);
    }
    cudaFree(*p);
    *p = nullptr;
  }
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, what);
  }
  v->bytes_device += (int64_t)(count * sizeof(T));
  v->alloc_bytes[*p] = (int64_t)(count * sizeof(T));
  return LRVOL_OK;
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// ----------------------------------------------------------------------------
// element -> B-spline incidence: B-splines whose support contains the element
// ----------------------------------------------------------------------------
int build_incidence(lrvol_s *v, std::vector<int64_t> &ptr, std::vector<int32_t> &idx) {
  const int64_t N = v->n_elem, M = v->n_basis;
  // bucket elements by centre on an R^3 grid
  int R = (int)std::cbrt((double)N / 4.0);
  R = std::max(1, std::min(R, 96));
  std::vector<int64_t> cell_ptr((size_t)R * R * R + 1, 0);
  std::vector<int32_t> cell_of(N);
  auto cell_coord = [&](double x) { return std::min(R - 1, std::max(0, (int)(x * R))); };
  for (int64_t e = 0; e < N; ++e) {
    const double *b = &v->box[6 * e];
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = cell_coord(0.5 * (b[a] + b[3 + a]));
    cell_of[e] = (c[2] * R + c[1]) * R + c[0];
    cell_ptr[cell_of[e] + 1]++;
  }
  for (size_t i = 1; i < cell_ptr.size(); ++i) cell_ptr[i] += cell_ptr[i - 1];
  std::vector<int32_t> cell_el(N);
  {
    std::vector<int64_t> fill(cell_ptr.begin(), cell_ptr.end() - 1);
    for (int64_t e = 0; e < N; ++e) cell_el[fill[cell_of[e]]++] = (int32_t)e;
  }
  // pairs (element, bspline), bspline-major
  std::vector<int64_t> count(N + 1, 0);
  std::vector<std::pair<int32_t, int32_t>> pairs;
  pairs.reserve((size_t)N * 64);
  const int off[3] = {0, v->p[0] + 2, v->p[0] + v->p[1] + 4};
  for (int64_t i = 0; i < M; ++i) {
    const double *k = &v->knots[(size_t)i * v->kw];
    double lo[3], hi[3];
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = k[off[a]];
      hi[a] = k[off[a] + v->p[a] + 1];
      c0[a] = cell_coord(lo[a]);
      c1[a] = cell_coord(hi[a]);
    }
    for (int cz = c0[2]; cz <= c1[2]; ++cz)
      for (int cy = c0[1]; cy <= c1[1]; ++cy)
        for (int cx = c0[0]; cx <= c1[0]; ++cx) {
          int cell = (cz * R + cy) * R + cx;
          for (int64_t q = cell_ptr[cell]; q < cell_ptr[cell + 1]; ++q) {
            int32_t e = cell_el[q];
            const double *b = &v->box[6 * (size_t)e];
            bool in = true;
            for (int a = 0; a < 3 && in; ++a) in = lo[a] <= b[a] && b[3 + a] <= hi[a];
            if (in) {
              pairs.push_back({e, (int32_t)i});
              count[e + 1]++;
            }
          }
        }
  }
  for (int64_t e = 0; e < N; ++e) {
    if (count[e + 1] == 0) return fail(LRVOL_ERR_ARG, "an element lies in no B-spline support");
    count[e + 1] += count[e];
  }
  ptr.assign(count.begin(), count.end());
  idx.resize(pairs.size());
  std::vector<int64_t> fill(count.begin(), count.end() - 1);
  for (auto &pr : pairs) idx[fill[pr.first]++] = pr.second;  // B-spline order kept per element
  return LRVOL_OK;
}

// ----------------------------------------------------------------------------
// k-d forest (Sec. 3.2.1).  Split rule (the paper balances depth by counting,
// per direction, the elements on either side of a mean split plane): candidates are the
// element faces strictly inside the node region; per axis the candidate
// nearest to the mean of the candidates; score = max(#left, #right) with
// straddling elements counted on both sides; lowest score wins, ties x<y<z.
// ----------------------------------------------------------------------------
float round_up_f32(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, INFINITY);
  return f;
}

struct ForestBuilder {
  const lrvol_s *v;
  std::vector<Node> nodes;
  std::vector<uint32_t> head;
  std::vector<int32_t> depth;  // per block
  int B[3];
  bool midpoint = false;       // octree-style splits (LRVOL_SPLIT_MIDPOINT)
  bool unresolved = false;     // a midpoint tree reached kMaxDepth

  const double *box(int32_t e) const { return &v->box[6 * (size_t)e]; }

  // Build a tree over `els` inside region [rlo, rhi); returns a reference.
  uint32_t build(std::vector<int32_t> &els, const double *rlo, const double *rhi, int d, int *maxd) {
    *maxd = std::max(*maxd, d);
    if (els.size() == 1) return kLeaf | (uint32_t)els[0];
    if (midpoint) return build_mid(els, rlo, rhi, d, maxd);
    int best_axis = -1;
    double best_t = 0;
    size_t best_score = SIZE_MAX;
    std::vector<double> cand;
    for (int a = 0; a < 3; ++a) {
      cand.clear();
      for (int32_t e : els) {
        const double *b = box(e);
        if (b[a] > rlo[a] && b[a] < rhi[a]) cand.push_back(b[a]);
        if (b[3 + a] > rlo[a] && b[3 + a] < rhi[a]) cand.push_back(b[3 + a]);
      }
      if (cand.empty()) continue;
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      double mean = 0;
      for (double c : cand) mean += c;
      mean /= (double)cand.size();
      double t = cand[0];
      for (double c : cand)
        if (std::fabs(c - mean) < std::fabs(t - mean)) t = c;
      size_t nl = 0, nr = 0;
      for (int32_t e : els) {
        const double *b = box(e);
        nl += b[a] < t;
        nr += b[3 + a] > t;
      }
      size_t score = std::max(nl, nr);
      if (score < best_score) {
        best_score = score;
        best_axis = a;
        best_t = t;
      }
    }
    if (best_axis < 0) return kNone;  // cannot happen for a valid box partition
    std::vector<int32_t> L, R;
    for (int32_t e : els) {
      const double *b = box(e);
      if (b[best_axis] < best_t) L.push_back(e);
      if (b[3 + best_axis] > best_t) R.push_back(e);
    }
    if (L.size() >= els.size() || R.size() >= els.size() || L.empty() || R.empty()) return kNone;
    uint32_t me = (uint32_t)nodes.size();
    nodes.push_back(Node{0, 0, {0, 0}});
    Node nd;
    float s = round_up_f32(best_t);
    std::memcpy(&nd.split_bits, &s, 4);
    nd.axis = (uint32_t)best_axis;
    double llo[3], lhi[3], hlo[3], hhi[3];
    for (int a = 0; a < 3; ++a) {
      llo[a] = hlo[a] = rlo[a];
      lhi[a] = hhi[a] = rhi[a];
    }
    lhi[best_axis] = best_t;
    hlo[best_axis] = best_t;
    els.clear();
    els.shrink_to_fit();
    nd.child[0] = build(L, llo, lhi, d + 1, maxd);
    nd.child[1] = build(R, hlo, hhi, d + 1, maxd);
    if (nd.child[0] == kNone || nd.child[1] == kNone) return kNone;
    nodes[me] = nd;
    return me;
  }

  // Octree-style tree: the region's midpoint on axes x, y, z in turn (three
  // binary levels make one octree level).  An element straddling the plane
  // goes to both sides; a leaf is a region that one element covers.  Dyadic
  // faces are reached exactly (midpoints of dyadic regions are dyadic, and
  // exact in FP32 down to 2^-149); a face at a non-dyadic coordinate never
  // is, and the tree is abandoned at kMaxDepth.
  uint32_t build_mid(std::vector<int32_t> &els, const double *rlo, const double *rhi, int d, int *maxd) {
    if (d >= kMaxDepth - 1) {
      unresolved = true;
      return kNone;
    }
    const int a = d % 3;
    const double t = 0.5 * (rlo[a] + rhi[a]);
    std::vector<int32_t> L, R;
    for (int32_t e : els) {
      const double *b = box(e);
      if (b[a] < t) L.push_back(e);
      if (b[3 + a] > t) R.push_back(e);
    }
    if (L.empty() || R.empty()) return kNone;   // not a box partition
    uint32_t me = (uint32_t)nodes.size();
    nodes.push_back(Node{0, 0, {0, 0}});
    Node nd;
    float s = round_up_f32(t);
    std::memcpy(&nd.split_bits, &s, 4);
    nd.axis = (uint32_t)a;
    double llo[3], lhi[3], hlo[3], hhi[3];
    for (int c = 0; c < 3; ++c) {
      llo[c] = hlo[c] = rlo[c];
      lhi[c] = hhi[c] = rhi[c];
    }
    lhi[a] = t;
    hlo[a] = t;
    els.clear();
    els.shrink_to_fit();
    nd.child[0] = build(L, llo, lhi, d + 1, maxd);
    if (nd.child[0] == kNone) return kNone;
    nd.child[1] = build(R, hlo, hhi, d + 1, maxd);
    if (nd.child[1] == kNone) return kNone;
    nodes[me] = nd;
    return me;
  }

  // Recursive region subdivision over blocks [b0, b1) with the elements meeting it.
  bool region(std::vector<int32_t> &els, const int *b0, const int *b1) {
    if (els.empty()) return false;
    if (els.size() == 1) {
      for (int z = b0[2]; z < b1[2]; ++z)
        for (int y = b0[1]; y < b1[1]; ++y)
          for (int x = b0[0]; x < b1[0]; ++x) {
            size_t q = ((size_t)z * B[1] + y) * B[0] + x;
            head[q] = kLeaf | (uint32_t)els[0];
            depth[q] = 0;
          }
      return true;
    }
    int ext[3] = {b1[0] - b0[0], b1[1] - b0[1], b1[2] - b0[2]};
    if (ext[0] == 1 && ext[1] == 1 && ext[2] == 1) {
      double lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        lo[a] = (double)b0[a] / B[a];
        hi[a] = (double)b1[a] / B[a];
      }
      int maxd = 0;
      uint32_t r = build(els, lo, hi, 0, &maxd);
      if (r == kNone) return false;
      size_t q = ((size_t)b0[2] * B[1] + b0[1]) * B[0] + b0[0];
      head[q] = r;
      depth[q] = maxd;
      return true;
    }
    int a = 0;
    for (int c = 1; c < 3; ++c)
      if (ext[c] > ext[a]) a = c;
    int mid = b0[a] + ext[a] / 2;
    double m = (double)mid / B[a];
    std::vector<int32_t> L, R;
    for (int32_t e : els) {
      const double *b = box(e);
      if (b[a] < m) L.push_back(e);
      if (b[3 + a] > m) R.push_back(e);
    }
    els.clear();
    els.shrink_to_fit();
    int l1[3] = {b1[0], b1[1], b1[2]}, r0[3] = {b0[0], b0[1], b0[2]};
    l1[a] = mid;
    r0[a] = mid;
    return region(L, b0, l1) && region(R, r0, b1);
  }
};

}  // namespace

namespace lrvol {

void camera_consts(const lrvol_camera *c, RayConsts *k) {
  // FP64 camera algebra rounded once to FP32; the order of operations is part
  // of the ray definition in lrvol.h.
  double F[3], R[3], U[3], n;
  for (int a = 0; a < 3; ++a) F[a] = c->target[a] - c->eye[a];
  n = std::sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  for (int a = 0; a < 3; ++a) F[a] = F[a] / n;
  R[0] = F[1] * c->up[2] - F[2] * c->up[1];
  R[1] = F[2] * c->up[0] - F[0] * c->up[2];
  R[2] = F[0] * c->up[1] - F[1] * c->up[0];
  n = std::sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
  for (int a = 0; a < 3; ++a) R[a] = R[a] / n;
  U[0] = R[1] * F[2] - R[2] * F[1];
  U[1] = R[2] * F[0] - R[0] * F[2];
  U[2] = R[0] * F[1] - R[1] * F[0];
  double ty = c->projection == LRVOL_PERSP ? std::tan(0.5 * c->fovy) : 0.5 * c->extent;
  double tx = ty * (double)c->width / (double)c->height;
  for (int a = 0; a < 3; ++a) {
    k->E[a] = (float)c->eye[a];
    k->F[a] = (float)F[a];
    k->R[a] = (float)R[a];
    k->U[a] = (float)U[a];
  }
  k->sxs = (float)(2.0 * tx / (double)c->width);
  k->sxo = (float)(-tx);
  k->sys = (float)(-2.0 * ty / (double)c->height);
  k->syo = (float)ty;
  k->persp = c->projection == LRVOL_PERSP;
}

ForestView forest_view(const lrvol_s *v) {
  ForestView f;
  f.head = v->d_head;
  f.nodes = v->d_nodes;
  f.n_nodes = v->n_nodes;
  f.bx = v->blocks[0];
  f.by = v->blocks[1];
  f.bz = v->blocks[2];
  f.fbx = (float)v->blocks[0];
  f.fby = (float)v->blocks[1];
  f.fbz = (float)v->blocks[2];
  return f;
}

}  // namespace lrvol

namespace lrvol {

// Checks of lrvol_render and the kernel parameters of a frame, except the
// scratch pointers (counters, status), which the caller sets.
int prepare_render(const lrvol_s *v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                   float *rgba_dev, RenderParams *prm, int *field_out) {
  if (!v || !cam || !tf || !step || !rgba_dev) return fail(LRVOL_ERR_ARG, "null pointer");
  if (!v->have_bezier || !v->have_accel) return fail(LRVOL_ERR_STATE, "render needs to_bezier and build_accel");
  if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
    return fail(LRVOL_ERR_ARG, "bad image size");
  if (cam->projection != LRVOL_ORTHO && cam->projection != LRVOL_PERSP) return fail(LRVOL_ERR_ARG, "bad projection");
  int r0 = cam->row_begin, r1 = cam->row_end;
  if (r0 == 0 && r1 == 0) r1 = cam->height;
  if (r0 < 0 || r1 > cam->height || r0 > r1) return fail(LRVOL_ERR_ARG, "bad row range");
  const int nb = cam->band_count < 1 ? 1 : cam->band_count;
  if (cam->band_count < 0 || cam->band_index < 0 || cam->band_index >= nb)
    return fail(LRVOL_ERR_ARG, "bad interleaved band (need 0 <= band_index < band_count)");
  // rows of this call's first band to the end: none when band_index is past the last band
  const int n_bands = (r1 - r0 + LRVOL_BAND_ROWS - 1) / LRVOL_BAND_ROWS;
  if (cam->band_index >= n_bands) r1 = r0;
  if (step->mode != LRVOL_STEP_FIXED && step->mode != LRVOL_STEP_HEURISTIC && step->mode != LRVOL_STEP_LEARNED)
    return fail(LRVOL_ERR_ARG, "bad step mode");
  if (step->mode == LRVOL_STEP_LEARNED && !step->mult) return fail(LRVOL_ERR_ARG, "learned steps need multipliers");
  if (step->mode == LRVOL_STEP_FIXED && !(step->h > 0)) return fail(LRVOL_ERR_ARG, "fixed step must be > 0");
  if (!(step->xi > 0) || !(tf->vmax > tf->vmin)) return fail(LRVOL_ERR_ARG, "xi and vmax - vmin must be > 0");
  int field = step->field;
  if (field == LRVOL_FIELD_SCALAR && v->nc != 1) return fail(LRVOL_ERR_ARG, "scalar field needs ncomp = 1");
  if (field == LRVOL_FIELD_MAGNITUDE && v->nc != 3) return fail(LRVOL_ERR_ARG, "magnitude needs ncomp = 3");
  if (field == LRVOL_FIELD_COMPONENT && (step->component < 0 || step->component >= v->nc))
    return fail(LRVOL_ERR_ARG, "bad component");
  if (field < 0 || field > 2) return fail(LRVOL_ERR_ARG, "bad field");
  if (v->p[0] != v->p[1] || v->p[0] != v->p[2] || v->p[0] > 3)
    return fail(LRVOL_ERR_UNSUPPORTED, "render needs equal degrees 1..3");
  if (step->shading != LRVOL_SHADE_NONE && step->shading != LRVOL_SHADE_GRADIENT)
    return fail(LRVOL_ERR_ARG, "bad shading");
  if (step->shading == LRVOL_SHADE_GRADIENT && field != LRVOL_FIELD_SCALAR)
    return fail(LRVOL_ERR_UNSUPPORTED, "gradient shading needs a scalar field");
  const double ll = step->light[0] * step->light[0] + step->light[1] * step->light[1] +
                    step->light[2] * step->light[2];
  if (!(ll < INFINITY)) return fail(LRVOL_ERR_ARG, "light must be finite");
  std::memset(prm, 0, sizeof(*prm));
  prm->elem = v->d_elem;
  prm->n_elem = v->n_elem;
  prm->bez = v->d_bez;
  prm->elem_bytes = v->elem_bytes;
  prm->bezc = v->d_bezc;
  prm->elemc_bytes = v->elemc_bytes;
  prm->comp = field == LRVOL_FIELD_COMPONENT ? step->component : 0;
  prm->forest = forest_view(v);
  prm->out = rgba_dev;
  prm->width = cam->width;
  prm->height = cam->height;
  prm->row_begin = r0;
  prm->row_end = r1;
  prm->band_count = nb;
  prm->band_index = r1 > r0 ? cam->band_index : 0;
  camera_consts(cam, &prm->ray);
  prm->mode = step->mode;
  prm->mult = step->mult;
  prm->h = (float)step->h;
  prm->inv_xi = (float)(1.0 / step->xi);
  prm->alpha_stop = (float)step->alpha_stop;
  prm->tf_scale = (float)(255.0 / (tf->vmax - tf->vmin));
  prm->tf_bias = (float)(-tf->vmin * 255.0 / (tf->vmax - tf->vmin));
  for (int q = 0; q < 256; ++q) prm->tf[q] = make_float4(tf->rgba[q][0], tf->rgba[q][1], tf->rgba[q][2], tf->rgba[q][3]);
  prm->trim = reinterpret_cast<const float2 *>(step->trim);
  if (step->shading == LRVOL_SHADE_GRADIENT) {
    field = kFieldShaded;
    prm->light_set = ll > 0.0;
    for (int a = 0; a < 3; ++a) prm->light[a] = ll > 0.0 ? (float)(step->light[a] / std::sqrt(ll)) : 0.f;
    prm->grad_eps = (float)(1e-3 * (tf->vmax - tf->vmin));
  }
  *field_out = field;
  return LRVOL_OK;
}

// Checks of lrvol_features and its kernel parameters.
int prepare_features(const lrvol_s *v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                     FeatureParams *fp) {
  if (!v || !cam || !tf || !step) return fail(LRVOL_ERR_ARG, "null pointer");
  if (!v->have_bezier) return fail(LRVOL_ERR_STATE, "features need to_bezier");
  if (!(tf->vmax > tf->vmin)) return fail(LRVOL_ERR_ARG, "vmax - vmin must be > 0");
  const int field = step->field;
  if (field < 0 || field > 2 || (field == LRVOL_FIELD_SCALAR && v->nc != 1) ||
      (field == LRVOL_FIELD_MAGNITUDE && v->nc != 3) ||
      (field == LRVOL_FIELD_COMPONENT && (step->component < 0 || step->component >= v->nc)))
    return fail(LRVOL_ERR_ARG, "bad field/component for this volume");
  std::memset(fp, 0, sizeof(*fp));
  fp->box = v->d_box;
  fp->elem = v->d_elem;
  fp->range = v->d_range;
  fp->n_elem = v->n_elem;
  fp->nc = v->nc;
  fp->field = field;
  fp->comp = step->component;
  for (int a = 0; a < 3; ++a) fp->eye[a] = (float)cam->eye[a];
  fp->tf_scale = (float)(255.0 / (tf->vmax - tf->vmin));
  fp->tf_bias = (float)(-tf->vmin * 255.0 / (tf->vmax - tf->vmin));
  for (int q = 0; q < 256; ++q) fp->tf[q] = make_float4(tf->rgba[q][0], tf->rgba[q][1], tf->rgba[q][2], tf->rgba[q][3]);
  return LRVOL_OK;
}

}  // namespace lrvol

extern "C" {

const char *lrvol_status_string(int s) {
  switch (s) {
    case LRVOL_OK: return "ok";
    case LRVOL_ERR_ARG: return "invalid argument";
    case LRVOL_ERR_OOM: return "out of memory";
    case LRVOL_ERR_CUDA: return "CUDA error";
    case LRVOL_ERR_STATE: return "call out of order";
    case LRVOL_ERR_BOUNDS: return "device bounds check failed";
    case LRVOL_ERR_TIMEOUT: return "device wait timed out";
    case LRVOL_ERR_UNSUPPORTED: return "unsupported by this build";
    default: return "unknown status";
  }
}

const char *lrvol_last_error(void) { return g_last_error.c_str(); }

int lrvol_create(const int32_t deg[3], int32_t ncomp, int64_t n_elem, const double *elem_box,
                 int64_t n_basis, const double *knots, const double *coef, const double *weight,
                 lrvol_t *out) {
  if (!deg || !elem_box || !knots || !coef || !weight || !out) return fail(LRVOL_ERR_ARG, "null pointer");
  *out = nullptr;
  if (ncomp != 1 && ncomp != 3) return fail(LRVOL_ERR_ARG, "ncomp must be 1 or 3");
  if (n_elem < 1 || n_elem >= (int64_t)kLeaf || n_basis < 1 || n_basis >= (int64_t)INT32_MAX)
    return fail(LRVOL_ERR_ARG, "bad element or basis count");
  for (int a = 0; a < 3; ++a)
    if (deg[a] < 1 || deg[a] > kMaxDeg) return fail(LRVOL_ERR_ARG, "degree out of range 1..4");
  int kw = deg[0] + deg[1] + deg[2] + 6;
  for (int64_t e = 0; e < n_elem; ++e)
    for (int a = 0; a < 3; ++a) {
      double lo = elem_box[6 * e + a], hi = elem_box[6 * e + 3 + a];
      if (!(lo >= 0.0 && hi <= 1.0 && lo < hi)) return fail(LRVOL_ERR_ARG, "element box outside [0,1] or empty");
    }
  for (int64_t i = 0; i < n_basis; ++i) {
    const double *k = knots + i * kw;
    for (int j = 1; j < kw; ++j) {
      bool axis_start = (j == deg[0] + 2) || (j == deg[0] + deg[1] + 4);
      if (!axis_start && !(k[j] >= k[j - 1])) return fail(LRVOL_ERR_ARG, "knots must be non-decreasing");
    }
    if (!std::isfinite(weight[i])) return fail(LRVOL_ERR_ARG, "non-finite weight");
  }
  int dev = 0;
  CU(cudaGetDevice(&dev), "cudaGetDevice");
  lrvol_s *v = new lrvol_s();
  v->device = dev;
  for (int a = 0; a < 3; ++a) v->p[a] = deg[a];
  v->nc = ncomp;
  v->n_elem = n_elem;
  v->n_basis = n_basis;
  v->kw = kw;
  v->box.assign(elem_box, elem_box + 6 * n_elem);
  v->knots.assign(knots, knots + kw * n_basis);
  v->coef.assign(coef, coef + ncomp * n_basis);
  v->weight.assign(weight, weight + n_basis);
  int rc;
  if ((rc = dev_alloc(v, &v->d_box, 6 * n_elem, "alloc boxes")) ||
      (rc = dev_alloc(v, &v->d_knots, (size_t)kw * n_basis, "alloc knots")) ||
      (rc = dev_alloc(v, &v->d_coef, (size_t)ncomp * n_basis, "alloc coef")) ||
      (rc = dev_alloc(v, &v->d_weight, n_basis, "alloc weight")) ||
      (rc = dev_alloc(v, &v->d_counters, kNumCounters, "alloc counters")) ||
      (rc = dev_alloc(v, &v->d_status, 1, "alloc status"))) {
    lrvol_destroy(v);
    return rc;
  }
  cudaError_t e = cudaSuccess;
  if (!e) e = cudaMemcpy(v->d_box, elem_box, sizeof(double) * 6 * n_elem, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(v->d_knots, knots, sizeof(double) * kw * n_basis, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(v->d_coef, coef, sizeof(double) * ncomp * n_basis, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(v->d_weight, weight, sizeof(double) * n_basis, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemset(v->d_counters, 0, sizeof(unsigned long long) * kNumCounters);
  if (!e) e = cudaMemset(v->d_status, 0, sizeof(uint32_t));
  if (e) {
    lrvol_destroy(v);
    return cuda_fail(e, "upload volume");
  }
  *out = v;
  return LRVOL_OK;
}

int lrvol_build_accel(lrvol_t v, const int32_t blocks[3], void *stream) {
  return lrvol_build_accel_split(v, blocks, LRVOL_SPLIT_BALANCED, stream);
}

int lrvol_build_accel_split(lrvol_t v, const int32_t blocks[3], int32_t split, void *stream) {
  if (!v || !blocks) return fail(LRVOL_ERR_ARG, "null pointer");
  if (split != LRVOL_SPLIT_BALANCED && split != LRVOL_SPLIT_MIDPOINT) return fail(LRVOL_ERR_ARG, "bad split rule");
  for (int a = 0; a < 3; ++a)
    if (!is_pow2(blocks[a]) || blocks[a] > 1024) return fail(LRVOL_ERR_ARG, "blocks must be powers of two <= 1024");
  if ((int64_t)blocks[0] * blocks[1] * blocks[2] > (int64_t)1 << 28) return fail(LRVOL_ERR_ARG, "too many blocks");
  ForestBuilder fb;
  fb.v = v;
  fb.midpoint = split == LRVOL_SPLIT_MIDPOINT;
  for (int a = 0; a < 3; ++a) fb.B[a] = blocks[a];
  size_t nblk = (size_t)blocks[0] * blocks[1] * blocks[2];
  fb.head.assign(nblk, kNone);
  fb.depth.assign(nblk, 0);
  std::vector<int32_t> all(v->n_elem);
  std::iota(all.begin(), all.end(), 0);
  int b0[3] = {0, 0, 0}, b1[3] = {blocks[0], blocks[1], blocks[2]};
  if (!fb.region(all, b0, b1)) {
    if (fb.unresolved)
      return fail(LRVOL_ERR_UNSUPPORTED, "midpoint splits do not resolve this mesh (faces at non-dyadic coordinates)");
    return fail(LRVOL_ERR_ARG, "elements do not form a box partition of [0,1]^3");
  }
  for (uint32_t h : fb.head)
    if (h == kNone) return fail(LRVOL_ERR_ARG, "a forest block holds no element");
  if (fb.nodes.size() >= kLeaf) return fail(LRVOL_ERR_ARG, "forest too large");
  // depth statistics over blocks
  double s = 0, s2 = 0;
  int dmin = INT32_MAX, dmax = 0;
  for (int32_t d : fb.depth) {
    s += d;
    s2 += (double)d * d;
    dmin = std::min(dmin, d);
    dmax = std::max(dmax, d);
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  // from here the previous forest is replaced: until the new one is complete
  // the handle has none (a failed host build above left the previous one)
  v->have_accel = false;
  if ((rc = dev_alloc(v, &v->d_head, nblk, "alloc forest head")) ||
      (rc = dev_alloc(v, &v->d_nodes, fb.nodes.size(), "alloc forest nodes")))
    return rc;
  CU(cudaMemcpyAsync(v->d_head, fb.head.data(), sizeof(uint32_t) * nblk, cudaMemcpyHostToDevice, st), "upload head");
  if (!fb.nodes.empty())
    CU(cudaMemcpyAsync(v->d_nodes, fb.nodes.data(), sizeof(Node) * fb.nodes.size(), cudaMemcpyHostToDevice, st),
       "upload nodes");
  CU(cudaStreamSynchronize(st), "build_accel sync");  // host vectors go out of scope
  v->n_nodes = (int64_t)fb.nodes.size();
  for (int a = 0; a < 3; ++a) v->blocks[a] = blocks[a];
  v->depth_min = dmin;
  v->depth_max = dmax;
  v->depth_mean = s / (double)nblk;
  v->depth_var = std::max(0.0, s2 / (double)nblk - v->depth_mean * v->depth_mean);
  v->have_accel = true;
  return LRVOL_OK;
}

int lrvol_to_bezier(lrvol_t v, int32_t storage, void *stream) {
  if (!v) return fail(LRVOL_ERR_ARG, "null handle");
  if (storage != LRVOL_STORE_F32 && storage != LRVOL_STORE_F16 && storage != LRVOL_STORE_BF16)
    return fail(LRVOL_ERR_ARG, "bad storage");
  std::vector<int64_t> ptr;
  std::vector<int32_t> idx;
  int rc = build_incidence(v, ptr, idx);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int n0 = v->p[0] + 1, n1 = v->p[1] + 1, n2 = v->p[2] + 1, nb = n0 * n1 * n2;
  v->have_bezier = false;   // the blocks are replaced: none until the new ones are complete
  v->storage = storage;
  v->elem_bytes = elem_bytes(storage, render_slots(v->nc, n0, n1, n2));
  v->elemc_bytes = v->nc == 3 ? elem_bytes(storage, 3 * roundup8(nb)) : 0;
  if ((rc = dev_alloc(v, &v->d_inc_ptr, ptr.size(), "alloc incidence ptr")) ||
      (rc = dev_alloc(v, &v->d_inc_idx, idx.size(), "alloc incidence")) ||
      (rc = dev_alloc(v, &v->d_bez64, (size_t)v->n_elem * v->nc * nb, "alloc bezier64")) ||
      (rc = dev_alloc(v, &v->d_bez, (size_t)v->n_elem * v->elem_bytes, "alloc render blocks")) ||
      (v->nc == 3 && (rc = dev_alloc(v, &v->d_bezc, (size_t)v->n_elem * v->elemc_bytes, "alloc render copy"))) ||
      (rc = dev_alloc(v, &v->d_elem, (size_t)v->n_elem, "alloc element records")) ||
      (rc = dev_alloc(v, &v->d_range, (size_t)v->n_elem * v->nc, "alloc coefficient ranges")))
    return rc;
  CU(cudaMemcpyAsync(v->d_inc_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice, st),
     "upload incidence ptr");
  CU(cudaMemcpyAsync(v->d_inc_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice, st),
     "upload incidence");
  CU(cudaMemsetAsync(v->d_bez, 0, (size_t)v->n_elem * v->elem_bytes, st), "clear render blocks");
  if (v->d_bezc) CU(cudaMemsetAsync(v->d_bezc, 0, (size_t)v->n_elem * v->elemc_bytes, st), "clear render copy");
  CU(launch_to_bezier(v, st), "to_bezier kernel");
  CU(launch_pack(v, st), "pack kernel");
  CU(launch_elem_records(v, st), "element record kernel");
  CU(cudaStreamSynchronize(st), "to_bezier sync");  // host incidence goes out of scope
  v->inc_entries = (int64_t)idx.size();
  v->have_bezier = true;
  return LRVOL_OK;
}

int lrvol_render(lrvol_t v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                 float *rgba_dev, void *stream) {
  RenderParams prm;
  int field = 0;
  int rc = prepare_render(v, cam, tf, step, rgba_dev, &prm, &field);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  prm.counters = v->d_counters;
  prm.status = v->d_status;
  CU(cudaMemsetAsync(v->d_counters, 0, sizeof(unsigned long long) * kNumCounters, st), "clear counters");
  if (prm.row_end > prm.row_begin) CU(launch_render(prm, v->p[0], field, v->storage, st), "render kernel");
  return LRVOL_OK;
}

// The render kernel's own samples for a list of pixels (parity diagnostic):
// same checks and kernel template as lrvol_render, with the trace compiled in.
int lrvol_render_trace(lrvol_t v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                       const int32_t *pix_dev, int64_t n_pix, int32_t max_samples, float *trace_dev,
                       int32_t *count_dev, float *rgba_dev, void *stream) {
  if (n_pix < 0 || max_samples < 0) return fail(LRVOL_ERR_ARG, "n_pix and max_samples must be >= 0");
  if (n_pix > ((int64_t)1 << 37)) return fail(LRVOL_ERR_ARG, "more than 2^37 pixels");
  if (n_pix > 0 && (!pix_dev || !count_dev || !rgba_dev || (max_samples > 0 && !trace_dev)))
    return fail(LRVOL_ERR_ARG, "null pointer");
  RenderParams prm;
  int field = 0;
  float unused = 0.f;   // prepare_render wants an image pointer; the traced kernel writes none
  int rc = prepare_render(v, cam, tf, step, &unused, &prm, &field);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  prm.counters = v->d_counters;
  prm.status = v->d_status;
  prm.out = nullptr;
  prm.trace_pix = pix_dev;
  prm.trace_n = n_pix;
  prm.trace_max = max_samples;
  prm.trace_rec = reinterpret_cast<float4 *>(trace_dev);
  prm.trace_count = count_dev;
  prm.trace_rgba = reinterpret_cast<float4 *>(rgba_dev);
  CU(cudaMemsetAsync(v->d_counters, 0, sizeof(unsigned long long) * kNumCounters, st), "clear counters");
  CU(launch_render_trace(prm, v->p[0], field, v->storage, st), "render trace kernel");
  return LRVOL_OK;
}

// The allocation-free render: same checks and kernel as lrvol_render, but the
// kernel's scratch (statistics counters, status word) is the library's
// static device array instead of memory of the handle, and nothing is allocated.
int lrvol_render_noalloc(lrvol_t v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step,
                         float *rgba_dev, uint64_t *counters_dev, void *stream) {
  if (cam && (cam->width > kMaxImageSide || cam->height > kMaxImageSide))
    return fail(LRVOL_ERR_ARG, "image size outside 1..32768 x 1..32768, the maximum of lrvol_render_noalloc");
  RenderParams prm;
  int field = 0;
  int rc = prepare_render(v, cam, tf, step, rgba_dev, &prm, &field);
  if (rc) return rc;
  cudaError_t e = launch_render_static(prm, v->p[0], field, v->storage, (cudaStream_t)stream,
                                       reinterpret_cast<unsigned long long *>(counters_dev));
  if (e != cudaSuccess) return cuda_fail(e, "render_noalloc");
  return LRVOL_OK;
}

// ---- learned step sizes ----------------------------------------------------

int lrvol_features(lrvol_t v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step, float *feat,
                   void *stream) {
  if (!feat) return fail(LRVOL_ERR_ARG, "null pointer");
  FeatureParams fp;
  int rc = prepare_features(v, cam, tf, step, &fp);
  if (rc) return rc;
  CU(launch_features(fp, feat, (cudaStream_t)stream), "features kernel");
  return LRVOL_OK;
}

int lrvol_mlp_pack(const float *params, uint16_t *packed, void *stream) {
  if (!params || !packed) return fail(LRVOL_ERR_ARG, "null pointer");
  CU(launch_mlp_pack(params, packed, (cudaStream_t)stream), "mlp pack kernel");
  return LRVOL_OK;
}

int lrvol_mlp_infer(const float *x, int64_t n, const uint16_t *packed, float ymin, float ymax, float *out,
                    void *stream) {
  if (n < 0 || (n > 0 && (!x || !packed || !out))) return fail(LRVOL_ERR_ARG, "bad arguments");
  if (!(ymax >= 0.f && ymax <= 8.f)) return fail(LRVOL_ERR_ARG, "ymax must be in [0, 8]");
  if (!(ymin >= -8.f && ymin <= 0.f)) return fail(LRVOL_ERR_ARG, "ymin must be in [-8, 0]");
  if (n == 0) return LRVOL_OK;
  if (reinterpret_cast<uintptr_t>(packed) & 15) return fail(LRVOL_ERR_ARG, "packed weights must be 16-byte aligned");
  uint32_t *status = mlp_status_word();
  if (!status) return fail(LRVOL_ERR_CUDA, "network status word unavailable");
  CU(launch_mlp_infer(x, n, packed, ymin, ymax, out, status, (cudaStream_t)stream), "mlp infer kernel");
  return LRVOL_OK;
}

int lrvol_mlp_infer_timeout_test(const float *x, int64_t n, const uint16_t *packed, float ymin, float ymax,
                                 float *out, void *stream) {
  if (n < 1 || n > ((int64_t)1 << 20) || !x || !packed || !out) return fail(LRVOL_ERR_ARG, "bad arguments");
  if (!(ymax >= 0.f && ymax <= 8.f)) return fail(LRVOL_ERR_ARG, "ymax must be in [0, 8]");
  if (!(ymin >= -8.f && ymin <= 0.f)) return fail(LRVOL_ERR_ARG, "ymin must be in [-8, 0]");
  if (reinterpret_cast<uintptr_t>(packed) & 15) return fail(LRVOL_ERR_ARG, "packed weights must be 16-byte aligned");
  uint32_t *status = mlp_status_word();
  if (!status) return fail(LRVOL_ERR_CUDA, "network status word unavailable");
  CU(launch_mlp_infer(x, n, packed, ymin, ymax, out, status, (cudaStream_t)stream, true),
     "mlp infer kernel (timeout test)");
  return LRVOL_OK;
}

int lrvol_mlp_check(void) {
  uint32_t *status = mlp_status_word();
  if (!status) return fail(LRVOL_ERR_CUDA, "network status word unavailable");
  uint32_t h = 0;
  CU(cudaDeviceSynchronize(), "synchronise before the network status");
  CU(cudaMemcpy(&h, status, sizeof h, cudaMemcpyDeviceToHost), "read the network status");
  if (h == 0) return LRVOL_OK;
  CU(cudaMemset(status, 0, sizeof h), "clear the network status");
  return fail(LRVOL_ERR_TIMEOUT, "a tensor-core wait of lrvol_mlp_infer ran out; its rows got multiplier 1");
}

// activations and their gradients (n x (6*64 + 2)), then one gradient vector
int64_t lrvol_mlp_scratch_floats(int64_t n) { return n < 0 ? 0 : n * (6 * (int64_t)kHid + 2) + kParams; }

int lrvol_mlp_grad(const float *x, const float *target, int64_t n, const float *params, float *grad, float *loss,
                   float *scratch, void *stream) {
  if (!x || !target || !params || !grad || !scratch) return fail(LRVOL_ERR_ARG, "null pointer");
  if (n < 1 || n > ((int64_t)1 << 20)) return fail(LRVOL_ERR_ARG, "batch must be 1 .. 2^20 rows");
  CU(launch_mlp_grad(x, target, n, params, grad, loss, scratch, (cudaStream_t)stream), "mlp grad kernels");
  return LRVOL_OK;
}

int lrvol_mlp_train_step(const float *x, const float *target, int64_t n, float *params, float *m, float *vv,
                         int64_t t, float lr, float *loss, float *scratch, void *stream) {
  if (!m || !vv || t < 1 || !(lr > 0.f)) return fail(LRVOL_ERR_ARG, "bad optimiser arguments");
  // the gradient lands in the last kParams floats of the scratch
  float *grad = scratch + lrvol_mlp_scratch_floats(n) - kParams;
  int rc = lrvol_mlp_grad(x, target, n, params, grad, loss, scratch, stream);
  if (rc) return rc;
  CU(launch_adam(params, grad, m, vv, t, lr, (cudaStream_t)stream), "adam kernel");
  return LRVOL_OK;
}

int lrvol_labels(lrvol_t v, const lrvol_camera *cam, const lrvol_tf *tf, const lrvol_step *step, double h_fine,
                 double tau, const float *cand, int32_t n_cand, int32_t *label, void *stream) {
  if (!v || !cam || !tf || !step || !cand || !label) return fail(LRVOL_ERR_ARG, "null pointer");
  if (!v->have_bezier || !v->have_accel) return fail(LRVOL_ERR_STATE, "labels need to_bezier and build_accel");
  if (v->nc != 1 || v->storage != LRVOL_STORE_F32) return fail(LRVOL_ERR_UNSUPPORTED, "labels need a scalar FP32 volume");
  if (v->p[0] != v->p[1] || v->p[0] != v->p[2] || v->p[0] > 3)
    return fail(LRVOL_ERR_UNSUPPORTED, "labels need equal degrees 1..3");
  if (n_cand < 1 || n_cand > 16 || !(h_fine > 0) || !(tau >= 0)) return fail(LRVOL_ERR_ARG, "bad label arguments");
  if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
    return fail(LRVOL_ERR_ARG, "bad image size");
  if (!(step->xi > 0) || !(tf->vmax > tf->vmin)) return fail(LRVOL_ERR_ARG, "xi and vmax - vmin must be > 0");
  float hc[16];
  static_assert(sizeof(hc) / sizeof(hc[0]) >= 16, "room for the largest candidate list");
  CU(cudaMemcpy(hc, cand, sizeof(float) * n_cand, cudaMemcpyDeviceToHost), "read candidates");
  if (!(hc[0] > 0.f)) return fail(LRVOL_ERR_ARG, "candidates must be positive");
  for (int q = 1; q < n_cand; ++q)
    if (!(hc[q] > hc[q - 1])) return fail(LRVOL_ERR_ARG, "candidates must increase");
  RenderParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.elem = v->d_elem;
  prm.n_elem = v->n_elem;
  prm.bez = v->d_bez;
  prm.elem_bytes = v->elem_bytes;
  prm.forest = forest_view(v);
  prm.width = cam->width;
  prm.height = cam->height;
  prm.row_begin = 0;
  prm.row_end = cam->height;
  prm.band_count = 1;
  prm.band_index = 0;
  camera_consts(cam, &prm.ray);
  prm.mode = LRVOL_STEP_HEURISTIC;
  prm.inv_xi = (float)(1.0 / step->xi);
  prm.alpha_stop = (float)step->alpha_stop;
  prm.tf_scale = (float)(255.0 / (tf->vmax - tf->vmin));
  prm.tf_bias = (float)(-tf->vmin * 255.0 / (tf->vmax - tf->vmin));
  prm.counters = v->d_counters;
  prm.status = v->d_status;
  for (int q = 0; q < 256; ++q) prm.tf[q] = make_float4(tf->rgba[q][0], tf->rgba[q][1], tf->rgba[q][2], tf->rgba[q][3]);
  CU(launch_labels(prm, v->p[0], (float)h_fine, (float)tau, cand, n_cand, label, (cudaStream_t)stream),
     "labels kernel");
  return LRVOL_OK;
}

int lrvol_lookup(lrvol_t v, const float *pts, int64_t n, uint32_t *elem, void *stream) {
  if (!v || (n > 0 && (!pts || !elem)) || n < 0) return fail(LRVOL_ERR_ARG, "bad arguments");
  if (!v->have_accel) return fail(LRVOL_ERR_STATE, "lookup needs build_accel");
  if (n == 0) return LRVOL_OK;
  CU(launch_lookup(v, pts, n, elem, (cudaStream_t)stream), "lookup kernel");
  return LRVOL_OK;
}

int lrvol_eval(lrvol_t v, const float *pts, int64_t n, float *val, void *stream) {
  if (!v || (n > 0 && (!pts || !val)) || n < 0) return fail(LRVOL_ERR_ARG, "bad arguments");
  if (!v->have_accel || !v->have_bezier) return fail(LRVOL_ERR_STATE, "eval needs build_accel and to_bezier");
  if (n == 0) return LRVOL_OK;
  CU(launch_eval(v, pts, n, val, (cudaStream_t)stream), "eval kernel");
  return LRVOL_OK;
}

int lrvol_eval_grad(lrvol_t v, const float *pts, int64_t n, float *out, void *stream) {
  if (!v || (n > 0 && (!pts || !out)) || n < 0) return fail(LRVOL_ERR_ARG, "bad arguments");
  if (!v->have_bezier || !v->have_accel) return fail(LRVOL_ERR_STATE, "eval_grad needs to_bezier and build_accel");
  if (v->nc != 1) return fail(LRVOL_ERR_UNSUPPORTED, "eval_grad needs a scalar volume");
  if (n == 0) return LRVOL_OK;
  CU(launch_eval_grad(v, pts, n, out, (cudaStream_t)stream), "eval_grad kernel");
  return LRVOL_OK;
}

int lrvol_trim(const lrvol_camera *cam, const float *tri, int64_t n_tri, float *out, void *stream) {
  if (!cam || !out || n_tri < 0 || (n_tri > 0 && !tri)) return fail(LRVOL_ERR_ARG, "bad arguments");
  if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
    return fail(LRVOL_ERR_ARG, "bad image size");
  if (cam->projection != LRVOL_ORTHO && cam->projection != LRVOL_PERSP) return fail(LRVOL_ERR_ARG, "bad projection");
  RayConsts K;
  camera_consts(cam, &K);
  CU(launch_trim(K, cam->width, cam->height, tri, n_tri, out, (cudaStream_t)stream), "trim kernels");
  return LRVOL_OK;
}

int lrvol_streamlines(lrvol_t v, const lrvol_streamline_params *P, const double *seeds, int64_t n, double *out,
                      int32_t *count, int32_t *status, void *stream) {
  if (!v || !P || n < 0 || (n > 0 && (!seeds || !out || !count || !status))) return fail(LRVOL_ERR_ARG, "bad arguments");
  if (!v->have_bezier || !v->have_accel) return fail(LRVOL_ERR_STATE, "streamlines need to_bezier and build_accel");
  if (v->nc != 3) return fail(LRVOL_ERR_UNSUPPORTED, "streamlines need a 3-vector volume");
  if (v->p[0] != v->p[1] || v->p[0] != v->p[2] || v->p[0] > 3)
    return fail(LRVOL_ERR_UNSUPPORTED, "streamlines need equal degrees 1..3");
  if (P->method < LRVOL_RK1 || P->method > LRVOL_RKF45) return fail(LRVOL_ERR_ARG, "bad method");
  if (P->step_rule < LRVOL_SL_FIXED || P->step_rule > LRVOL_SL_ADAPTIVE) return fail(LRVOL_ERR_ARG, "bad step rule");
  if (P->step_rule == LRVOL_SL_ADAPTIVE && P->method < LRVOL_HE)
    return fail(LRVOL_ERR_ARG, "adaptive steps need an embedded pair (HE, BS, RKF45)");
  if (P->step_rule != LRVOL_SL_ADAPTIVE ? !(P->h > 0) : !(P->h >= 0)) return fail(LRVOL_ERR_ARG, "bad step");
  if (!(P->t_end > 0 && P->t_end < INFINITY)) return fail(LRVOL_ERR_ARG, "t_end must be positive and finite");
  if (P->step_rule == LRVOL_SL_ADAPTIVE && !(P->tol > 0)) return fail(LRVOL_ERR_ARG, "tol must be > 0");
  if (P->max_samples < 1) return fail(LRVOL_ERR_ARG, "max_samples must be >= 1");
  if (n == 0) return LRVOL_OK;
  SLParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.elem = v->d_elem;
  sp.n_elem = v->n_elem;
  sp.bez = v->d_bez;
  sp.elem_bytes = v->elem_bytes;
  sp.forest = forest_view(v);
  sp.status = v->d_status;
  sp.queue = v->d_counters + kCntQueue;
  sp.method = P->method;
  sp.rule = P->step_rule;
  sp.max_samples = P->max_samples;
  sp.h = P->h;
  sp.t_end = P->t_end;
  sp.tol_f = (float)P->tol;
  CU(launch_streamlines(sp, v->p[0], v->storage, seeds, n, out, count, status, (cudaStream_t)stream),
     "streamline kernel");
  return LRVOL_OK;
}

int lrvol_tubes(lrvol_t v, const lrvol_camera *cam, const double *samples, const int32_t *count, int64_t n_lines,
                int32_t max_samples, float radius, const lrvol_tf *cmap, uint64_t *vis, float *rgba, void *stream) {
  if (!v || !cam || !cmap || !vis || !rgba || n_lines < 0 || (n_lines > 0 && (!samples || !count)))
    return fail(LRVOL_ERR_ARG, "bad arguments");
  if (!v->have_bezier || !v->have_accel) return fail(LRVOL_ERR_STATE, "tubes need to_bezier and build_accel");
  if (v->nc != 3) return fail(LRVOL_ERR_UNSUPPORTED, "tubes need a 3-vector volume (speed colouring)");
  if (v->p[0] != v->p[1] || v->p[0] != v->p[2] || v->p[0] > 3)
    return fail(LRVOL_ERR_UNSUPPORTED, "tubes need equal degrees 1..3");
  if (max_samples < 2 || !(radius > 0.f && radius < INFINITY)) return fail(LRVOL_ERR_ARG, "bad max_samples or radius");
  if (n_lines * (int64_t)(max_samples - 1) >= ((int64_t)1 << 32)) return fail(LRVOL_ERR_ARG, "too many segments");
  if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
    return fail(LRVOL_ERR_ARG, "bad image size");
  if (cam->projection != LRVOL_ORTHO && cam->projection != LRVOL_PERSP) return fail(LRVOL_ERR_ARG, "bad projection");
  if (!(cmap->vmax > cmap->vmin)) return fail(LRVOL_ERR_ARG, "colour map needs vmax > vmin");
  TubeParams tp;
  std::memset(&tp, 0, sizeof(tp));
  tp.field.elem = v->d_elem;
  tp.field.n_elem = v->n_elem;
  tp.field.bez = v->d_bez;
  tp.field.elem_bytes = v->elem_bytes;
  tp.field.forest = forest_view(v);
  tp.field.status = v->d_status;
  camera_consts(cam, &tp.ray);
  tp.width = cam->width;
  tp.height = cam->height;
  tp.radius = radius;
  tp.samples = samples;
  tp.count = count;
  tp.n_lines = n_lines;
  tp.max_samples = max_samples;
  tp.vis = reinterpret_cast<unsigned long long *>(vis);
  tp.out = rgba;
  tp.tf_scale = (float)(255.0 / (cmap->vmax - cmap->vmin));
  tp.tf_bias = (float)(-cmap->vmin * 255.0 / (cmap->vmax - cmap->vmin));
  for (int q = 0; q < 256; ++q)
    tp.cmap[q] = make_float4(cmap->rgba[q][0], cmap->rgba[q][1], cmap->rgba[q][2], cmap->rgba[q][3]);
  CU(launch_tubes(tp, v->p[0], v->storage, (cudaStream_t)stream), "tube kernels");
  return LRVOL_OK;
}

int lrvol_streamline_error(const double *ref, const int32_t *rc, int32_t rmax, const double *app, const int32_t *ac,
                           int32_t amax, int64_t n, double *sums, void *stream) {
  if (n < 0 || rmax < 1 || amax < 1 || (n > 0 && (!ref || !rc || !app || !ac || !sums)))
    return fail(LRVOL_ERR_ARG, "bad arguments");
  if (n == 0) return LRVOL_OK;
  CU(launch_streamline_error(ref, rc, rmax, app, ac, amax, n, sums, (cudaStream_t)stream), "streamline error kernel");
  return LRVOL_OK;
}

int lrvol_get_bezier(lrvol_t v, double *host_out) {
  if (!v || !host_out) return fail(LRVOL_ERR_ARG, "null pointer");
  if (!v->have_bezier) return fail(LRVOL_ERR_STATE, "get_bezier needs to_bezier");
  size_t nb = (size_t)(v->p[0] + 1) * (v->p[1] + 1) * (v->p[2] + 1);
  CU(cudaDeviceSynchronize(), "sync");
  CU(cudaMemcpy(host_out, v->d_bez64, sizeof(double) * nb * v->nc * v->n_elem, cudaMemcpyDeviceToHost),
     "download bezier");
  return LRVOL_OK;
}

int lrvol_stats(lrvol_t v, lrvol_stats_t *out) {
  if (!v || !out) return fail(LRVOL_ERR_ARG, "null pointer");
  std::memset(out, 0, sizeof(*out));
  out->n_elem = v->n_elem;
  out->n_basis = v->n_basis;
  out->n_nodes = v->n_nodes;
  for (int a = 0; a < 3; ++a) out->blocks[a] = v->blocks[a];
  out->depth_min = v->depth_min;
  out->depth_max = v->depth_max;
  out->depth_mean = v->depth_mean;
  out->depth_var = v->depth_var;
  out->incidence_entries = v->inc_entries;
  out->bytes_device = v->bytes_device;
  CU(cudaDeviceSynchronize(), "sync");
  unsigned long long c[kNumCounters];
  uint32_t status = 0;
  CU(cudaMemcpy(c, v->d_counters, sizeof(c), cudaMemcpyDeviceToHost), "read counters");
  CU(cudaMemcpy(&status, v->d_status, sizeof(status), cudaMemcpyDeviceToHost), "read status");
  out->samples = (int64_t)c[kCntSamples];
  out->lookups = (int64_t)c[kCntLookups];
  out->rays_hit = (int64_t)c[kCntRays];
  if (status == kStatusBounds) return fail(LRVOL_ERR_BOUNDS, "a kernel bounds check tripped");
  if (status == kStatusTimeout) return fail(LRVOL_ERR_TIMEOUT, "a device wait timed out");
  return LRVOL_OK;
}

void lrvol_destroy(lrvol_t v) {
  if (!v) return;
  cudaDeviceSynchronize();
  void *ptrs[] = {v->d_box,   v->d_knots, v->d_coef,  v->d_weight, v->d_inc_ptr,  v->d_inc_idx, v->d_bez64,
                  v->d_bez,   v->d_bezc,  v->d_elem,  v->d_head,  v->d_nodes, v->d_counters, v->d_status,
                  v->d_range};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete v;
}

}  // extern "C"
