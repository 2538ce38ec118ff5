// liblrvol kernels for sm_103a.
//
//   k_to_bezier    Sec. 3.2.3 change of basis, FP64: per element, the Bernstein
//                  coefficients of every incident B-spline's univariate factors
//                  over the element, by blossoming, accumulated with gamma*c.
//   k_elem_records element boxes -> FP32 records (rounded-up corners, Eq. 4 step).
//   k_lookup       Alg. 1 element look-up through the k-d forest.
//   k_eval         look-up + Bezier block evaluation at points.
//   (k_render, the per-pixel ray casting of Sec. 4, is in render.cu; the
//   device helpers both files use are in device_common.cuh.)
//   k_features, k_mlp_infer, k_labels, k_dense_*, k_adam
//                  learned step multipliers (not in the paper; Eq. 4 stays the
//                  base): per-element features, the network on the tcgen05
//                  tensor cores, training labels and FP32 training.
//   k_streamlines, k_streamline_error, k_tube_*
//                  Sec. 5 streamlines (Eq. 4 steps), the Eq. 7 error, tubes.
//   k_trim_raster  Sec. 4.1 trimming: per-pixel interval of a boundary mesh.
#include <algorithm>

#include "device_common.cuh"

namespace lrvol {
namespace {

// ----------------------------------------------------------------------------
// change of basis (FP64)
// ----------------------------------------------------------------------------

// Bernstein coefficients over [a, b] of the univariate B-spline on knots
// xi[0..p+1], where [a, b] lies in one knot span.  beta_j is the blossom
// B(a,..,a, b,..,b) with j arguments b, evaluated by the de Boor triangle of
// the span restricted to its non-zero entries (only the B-spline itself has
// coefficient 1), so every denominator is a positive knot difference.
__device__ void bernstein_of_bspline(const double *xi, int p, double a, double b, double *beta) {
  int m = 0;
  for (int q = 1; q <= p; ++q)
    if (xi[q] <= a) m = q;
  // the triangle's denominators depend on (r, k) only: one FP64 division
  // each (FP64 division is a long instruction sequence on GB300), reused for
  // all p + 1 blossoms
  double inv[kMaxDeg + 1][kMaxDeg + 1];
  for (int r = 1; r <= p; ++r) {
    const int khi = m < r ? m : r;
    const int klo = (m - p + r) > 0 ? (m - p + r) : 0;
    for (int k = khi; k >= klo; --k) inv[r][k] = 1.0 / (xi[k + p + 1 - r] - xi[k]);
  }
  for (int j = 0; j <= p; ++j) {
    double D[kMaxDeg + 1];
    D[0] = 1.0;
    for (int q = 1; q <= p; ++q) D[q] = 0.0;
    for (int r = 1; r <= p; ++r) {
      const double t = (r <= p - j) ? a : b;
      const int khi = m < r ? m : r;
      const int klo = (m - p + r) > 0 ? (m - p + r) : 0;
      for (int k = khi; k >= klo; --k) {
        const double alpha = (t - xi[k]) * inv[r][k];
        const double prev = k > 0 ? D[k - 1] : 0.0;
        D[k] = (1.0 - alpha) * prev + alpha * D[k];
      }
    }
    beta[j] = D[m];
  }
}

// C(n, k) in integer arithmetic (each partial product is itself a binomial,
// so every division is exact)
__device__ __forceinline__ int binomial(int n, int k) {
  int b = 1;
  for (int i = 1; i <= k; ++i) b = b * (n - k + i) / i;
  return b;
}

constexpr int kBezWarps = 4;
constexpr int kChunk = 32;

// One warp per element; lane l owns coefficients q = l, l+32, ... of the
// (p0+1)(p1+1)(p2+1) block, for every component.
__global__ void __launch_bounds__(32 * kBezWarps) k_to_bezier(
    const double *__restrict__ box, const double *__restrict__ knots, const double *__restrict__ coef,
    const double *__restrict__ weight, const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_idx,
    int p0, int p1, int p2, int nc, int kw, int64_t n_elem, double *__restrict__ out64) {
  __shared__ double sb[kBezWarps][kChunk][3 * (kMaxDeg + 1)];
  __shared__ double sg[kBezWarps][kChunk][3];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * kBezWarps + w;
  if (e >= n_elem) return;
  const int n0 = p0 + 1, n1 = p1 + 1, n2 = p2 + 1;
  const int nb = n0 * n1 * n2;
  const int deg[3] = {p0, p1, p2};
  const int off[3] = {0, p0 + 2, p0 + p1 + 4};
  double acc[4][3];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 3; ++c) acc[r][c] = 0.0;
  const double *eb = box + 6 * e;
  const int64_t beg = inc_ptr[e], end = inc_ptr[e + 1];
  for (int64_t base = beg; base < end; base += kChunk) {
    const int cnt = (int)min((int64_t)kChunk, end - base);
    if (lane < cnt) {
      const int32_t i = inc_idx[base + lane];
      for (int a = 0; a < 3; ++a) {
        double xi[kMaxDeg + 2];
        for (int q = 0; q <= deg[a] + 1; ++q) xi[q] = knots[(int64_t)i * kw + off[a] + q];
        bernstein_of_bspline(xi, deg[a], eb[a], eb[3 + a], &sb[w][lane][a * (kMaxDeg + 1)]);
      }
      for (int c = 0; c < nc; ++c) sg[w][lane][c] = weight[i] * coef[(int64_t)i * nc + c];
    }
    __syncwarp();
    for (int s = 0; s < cnt; ++s) {
      const double *bs = sb[w][s];
      for (int r = 0; r < 4; ++r) {
        const int q = lane + 32 * r;
        if (q < nb) {
          const int ix = q % n0, iy = (q / n0) % n1, iz = q / (n0 * n1);
          const double prod = bs[ix] * bs[(kMaxDeg + 1) + iy] * bs[2 * (kMaxDeg + 1) + iz];
          for (int c = 0; c < nc; ++c) acc[r][c] += sg[w][s][c] * prod;
        }
      }
    }
    __syncwarp();
  }
  for (int r = 0; r < 4; ++r) {
    const int q = lane + 32 * r;
    if (q < nb)
      for (int c = 0; c < nc; ++c) out64[(e * nc + c) * nb + q] = acc[r][c];
  }
}

// Render copy of the FP64 blocks (layout and storage in lrvol_internal.h):
// binomials folded in; for 16-bit storage a per-element, per-component offset
// o = (max+min)/2 and scale s = (max-min)/2 of the FP64 coefficients, and
// q' = binomial*(c - o)/s rounded once from FP64.  One warp per element.
__device__ __forceinline__ void store_slot(unsigned char *base, int storage, int slot, double x) {
  if (storage == LRVOL_STORE_F32) {
    reinterpret_cast<float *>(base)[slot] = (float)x;
  } else if (storage == LRVOL_STORE_F16) {
    reinterpret_cast<__half *>(base + kHeaderBytes)[slot] = __double2half(x);
  } else {
    reinterpret_cast<__nv_bfloat16 *>(base + kHeaderBytes)[slot] = __double2bfloat16(x);
  }
}

__global__ void __launch_bounds__(32 * kBezWarps) k_pack(const double *__restrict__ b64, int p0, int p1, int p2, int nc,
                                                        int64_t n_elem, int storage, unsigned char *__restrict__ out,
                                                        int ebytes, unsigned char *__restrict__ outc, int ecbytes,
                                                        float2 *__restrict__ range) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * kBezWarps + w;
  if (e >= n_elem) return;
  const int n0 = p0 + 1, n1 = p1 + 1, nb = n0 * n1 * (p2 + 1);
  const double *be = b64 + e * nc * nb;
  double o[3] = {0.0, 0.0, 0.0}, sc[3] = {1.0, 1.0, 1.0};
  for (int c = 0; c < nc; ++c) {
    // coefficient range (the block's convex hull bounds the field on the element)
    double mn = __longlong_as_double(0x7ff0000000000000ll), mx = -mn;
    for (int q = lane; q < nb; q += 32) {
      mn = fmin(mn, be[c * nb + q]);
      mx = fmax(mx, be[c * nb + q]);
    }
    for (int off = 16; off > 0; off >>= 1) {
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, off));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if (lane == 0) range[e * nc + c] = make_float2(__double2float_rd(mn), __double2float_ru(mx));
    if (storage != LRVOL_STORE_F32) {
      o[c] = 0.5 * (mx + mn);
      sc[c] = 0.5 * (mx - mn);
      if (!(sc[c] > 0.0)) sc[c] = 1.0;
    }
  }
  if (storage != LRVOL_STORE_F32) {
    if (lane < 8) {
      const float hv = lane < 3 ? (float)o[lane] : (lane < 6 ? (float)sc[lane - 3] : 0.f);
      reinterpret_cast<float *>(out + e * ebytes)[lane] = hv;
      if (outc) reinterpret_cast<float *>(outc + e * ecbytes)[lane] = hv;
    }
  }
  for (int q = lane; q < nb; q += 32) {
    const int ix = q % n0, iy = (q / n0) % n1, iz = q / (n0 * n1);
    const double binom = (double)(binomial(p0, ix) * binomial(p1, iy) * binomial(p2, iz));
    for (int c = 0; c < nc; ++c) {
      const double d = be[c * nb + q] - o[c];   // o = 0 and s = 1 for FP32 storage
      const double x = storage == LRVOL_STORE_F32 ? binom * d : binom * d / sc[c];
      store_slot(out + e * ebytes, storage, render_slot(nc, n0, nb, iz * n1 + iy, ix, c), x);
      if (outc) store_slot(outc + e * ecbytes, storage, c * roundup8(nb) + q, x);
    }
  }
}

__global__ void k_elem_records(const double *__restrict__ box, int64_t n_elem, int d, ElemRec *__restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  const double *b = box + 6 * e;
  float lo[3], hi[3], off[3], iw[3];
  double m = b[3] - b[0];
  if (b[4] - b[1] < m) m = b[4] - b[1];
  if (b[5] - b[2] < m) m = b[5] - b[2];
  for (int a = 0; a < 3; ++a) {
    lo[a] = __double2float_ru(b[a]);
    hi[a] = b[3 + a] == 1.0 ? __int_as_float(0x7f800000) : __double2float_ru(b[3 + a]);
    const double inv = 1.0 / (b[3 + a] - b[a]);
    off[a] = (float)(((double)lo[a] - b[a]) * inv);   // (lo_RU - lo) / (hi - lo), in FP64
    iw[a] = (float)inv;
  }
  ElemRec r;
  r.a = make_float4(lo[0], lo[1], lo[2], __double2float_rn(ldexp(m, -d)));
  r.b = make_float4(hi[0], hi[1], hi[2], 0.f);
  r.c = make_float4(off[0], off[1], off[2], 0.f);
  r.d = make_float4(iw[0], iw[1], iw[2], 0.f);
  out[e] = r;
}


__global__ void k_lookup(ForestView f, int64_t n_elem, const float *__restrict__ pts, int64_t n,
                         uint32_t *__restrict__ out, uint32_t *status) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float x = pts[3 * q], y = pts[3 * q + 1], z = pts[3 * q + 2];
  uint32_t e = kNone;
  if (x >= 0.f && x <= 1.f && y >= 0.f && y <= 1.f && z >= 0.f && z <= 1.f) {
    e = forest_lookup(f, x, y, z, status);
    if (e != kNone && (int64_t)e >= n_elem) {
      set_status(status, kStatusBounds);
      e = kNone;
    }
  }
  out[q] = e;
}


// Generic-degree evaluation for the point kernel (any p0,p1,p2 <= 4).
__device__ float eval_generic(const float *c, const int *deg, float ux, float uy, float uz) {
  float b[3][kMaxDeg + 1];
  const float u[3] = {ux, uy, uz};
  for (int a = 0; a < 3; ++a) {
    const int p = deg[a];
    const float v = 1.f - u[a];
    for (int i = 0; i <= p; ++i) {
      float m = 1.f;
      for (int q = 0; q < i; ++q) m *= u[a];
      for (int q = i; q < p; ++q) m *= v;
      b[a][i] = m;
    }
  }
  const int n0 = deg[0] + 1, n1 = deg[1] + 1, n2 = deg[2] + 1;
  float f = 0.f;
  for (int k = 0; k < n2; ++k) {
    float t = 0.f;
    for (int j = 0; j < n1; ++j) {
      float s = 0.f;
      for (int i = 0; i < n0; ++i) s = fmaf(c[(k * n1 + j) * n0 + i], b[0][i], s);
      t = fmaf(s, b[1][j], t);
    }
    f = fmaf(t, b[2][k], f);
  }
  return f;
}

// Value and derivatives in local coordinates (d/du, d/dv, d/dw) of the same block.
__device__ float eval_generic_grad(const float *c, const int *deg, float ux, float uy, float uz, float *g) {
  float b[3][kMaxDeg + 1], db[3][kMaxDeg + 1];
  const float u[3] = {ux, uy, uz};
  for (int a = 0; a < 3; ++a) {
    const int p = deg[a];
    const float v = 1.f - u[a];
    for (int i = 0; i <= p; ++i) {
      float m = 1.f, d1 = 0.f, d2 = 0.f;
      for (int q = 0; q < i; ++q) m *= u[a];
      for (int q = i; q < p; ++q) m *= v;
      if (i > 0) {  // i u^(i-1) v^(p-i)
        d1 = (float)i;
        for (int q = 0; q < i - 1; ++q) d1 *= u[a];
        for (int q = i; q < p; ++q) d1 *= v;
      }
      if (i < p) {  // (p-i) u^i v^(p-i-1)
        d2 = (float)(p - i);
        for (int q = 0; q < i; ++q) d2 *= u[a];
        for (int q = i + 1; q < p; ++q) d2 *= v;
      }
      b[a][i] = m;
      db[a][i] = d1 - d2;
    }
  }
  const int n0 = deg[0] + 1, n1 = deg[1] + 1, n2 = deg[2] + 1;
  float f = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
  for (int k = 0; k < n2; ++k) {
    float t = 0.f, tx = 0.f, ty = 0.f;
    for (int j = 0; j < n1; ++j) {
      float s = 0.f, sx = 0.f;
      for (int i = 0; i < n0; ++i) {
        const float cc = c[(k * n1 + j) * n0 + i];
        s = fmaf(cc, b[0][i], s);
        sx = fmaf(cc, db[0][i], sx);
      }
      t = fmaf(s, b[1][j], t);
      tx = fmaf(sx, b[1][j], tx);
      ty = fmaf(s, db[1][j], ty);
    }
    f = fmaf(t, b[2][k], f);
    gx = fmaf(tx, b[2][k], gx);
    gy = fmaf(ty, b[2][k], gy);
    gz = fmaf(t, db[2][k], gz);
  }
  g[0] = gx;
  g[1] = gy;
  g[2] = gz;
  return f;
}

__device__ __forceinline__ float load_slot(const unsigned char *eb, int storage, int slot) {
  if (storage == LRVOL_STORE_F32) return __ldg(reinterpret_cast<const float *>(eb) + slot);
  const unsigned short h = __ldg(reinterpret_cast<const unsigned short *>(eb + kHeaderBytes) + slot);
  if (storage == LRVOL_STORE_F16) return __half2float(__ushort_as_half(h));
  return __uint_as_float((unsigned)h << 16);
}

__global__ void k_eval(ForestView f, const ElemRec *__restrict__ elem, int64_t n_elem,
                       const unsigned char *__restrict__ bez, int ebytes, int storage, int p0, int p1, int p2, int nc,
                       const float *__restrict__ pts, int64_t n, float *__restrict__ out, uint32_t *status) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float x = pts[3 * q], y = pts[3 * q + 1], z = pts[3 * q + 2];
  uint32_t e = kNone;
  if (x >= 0.f && x <= 1.f && y >= 0.f && y <= 1.f && z >= 0.f && z <= 1.f) e = forest_lookup(f, x, y, z, status);
  if (e == kNone || (int64_t)e >= n_elem) {
    for (int c = 0; c < nc; ++c) out[q * nc + c] = 0.f;
    return;
  }
  const ElemRec r = elem[e];
  const float ux = local_u(x, r.a.x, r.c.x, r.d.x);
  const float uy = local_u(y, r.a.y, r.c.y, r.d.y);
  const float uz = local_u(z, r.a.z, r.c.z, r.d.z);
  const int deg[3] = {p0, p1, p2};
  const int n0 = p0 + 1, n1 = p1 + 1, nb = n0 * n1 * (p2 + 1);
  const unsigned char *eb = bez + (int64_t)e * ebytes;
  for (int c = 0; c < nc; ++c) {
    float cl[(kMaxDeg + 1) * (kMaxDeg + 1) * (kMaxDeg + 1)];
    for (int t = 0; t < nb; ++t) cl[t] = load_slot(eb, storage, render_slot(nc, n0, nb, t / n0, t % n0, c));
    const float v = eval_generic(cl, deg, ux, uy, uz);
    if (storage == LRVOL_STORE_F32) {
      out[q * nc + c] = v;
    } else {
      const float *hdr = reinterpret_cast<const float *>(eb);
      out[q * nc + c] = fmaf(__ldg(hdr + 3 + c), v, __ldg(hdr + c));
    }
  }
}

// Value and world-space gradient of a scalar volume at points (n x 4 out).
__global__ void k_eval_grad(ForestView f, const ElemRec *__restrict__ elem, int64_t n_elem,
                            const unsigned char *__restrict__ bez, int ebytes, int storage, int p0, int p1, int p2,
                            const float *__restrict__ pts, int64_t n, float *__restrict__ out, uint32_t *status) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float x = pts[3 * q], y = pts[3 * q + 1], z = pts[3 * q + 2];
  uint32_t e = kNone;
  if (x >= 0.f && x <= 1.f && y >= 0.f && y <= 1.f && z >= 0.f && z <= 1.f) e = forest_lookup(f, x, y, z, status);
  float4 *o = reinterpret_cast<float4 *>(out) + q;
  if (e == kNone || (int64_t)e >= n_elem) {
    *o = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const ElemRec r = elem[e];
  const int deg[3] = {p0, p1, p2};
  const int n0 = p0 + 1, nb = n0 * (p1 + 1) * (p2 + 1);
  const unsigned char *eb = bez + (int64_t)e * ebytes;
  float cl[(kMaxDeg + 1) * (kMaxDeg + 1) * (kMaxDeg + 1)];
  for (int t = 0; t < nb; ++t) cl[t] = load_slot(eb, storage, render_slot(1, n0, nb, t / n0, t % n0, 0));
  float g[3];
  float v = eval_generic_grad(cl, deg, local_u(x, r.a.x, r.c.x, r.d.x), local_u(y, r.a.y, r.c.y, r.d.y),
                              local_u(z, r.a.z, r.c.z, r.d.z), g);
  float sc = 1.f;
  if (storage != LRVOL_STORE_F32) {
    const float *hdr = reinterpret_cast<const float *>(eb);
    sc = __ldg(hdr + 3);
    v = fmaf(sc, v, __ldg(hdr));
  }
  *o = make_float4(v, sc * g[0] * r.d.x, sc * g[1] * r.d.y, sc * g[2] * r.d.z);
}


}  // namespace

cudaError_t launch_to_bezier(const lrvol_s *v, cudaStream_t s) {
  const int64_t blocks = (v->n_elem + kBezWarps - 1) / kBezWarps;
  k_to_bezier<<<(unsigned)blocks, 32 * kBezWarps, 0, s>>>(v->d_box, v->d_knots, v->d_coef, v->d_weight, v->d_inc_ptr,
                                                         v->d_inc_idx, v->p[0], v->p[1], v->p[2], v->nc, v->kw,
                                                         v->n_elem, v->d_bez64);
  return cudaGetLastError();
}

cudaError_t launch_pack(const lrvol_s *v, cudaStream_t s) {
  const int64_t blocks = (v->n_elem + kBezWarps - 1) / kBezWarps;
  k_pack<<<(unsigned)blocks, 32 * kBezWarps, 0, s>>>(v->d_bez64, v->p[0], v->p[1], v->p[2], v->nc, v->n_elem,
                                                    v->storage, v->d_bez, v->elem_bytes, v->d_bezc, v->elemc_bytes,
                                                    v->d_range);
  return cudaGetLastError();
}

cudaError_t launch_elem_records(const lrvol_s *v, cudaStream_t s) {
  int d = v->p[0];
  if (v->p[1] > d) d = v->p[1];
  if (v->p[2] > d) d = v->p[2];
  k_elem_records<<<(unsigned)((v->n_elem + 255) / 256), 256, 0, s>>>(v->d_box, v->n_elem, d, v->d_elem);
  return cudaGetLastError();
}

cudaError_t launch_lookup(const lrvol_s *v, const float *pts, int64_t n, uint32_t *out, cudaStream_t s) {
  k_lookup<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(forest_view(v), v->n_elem, pts, n, out, v->d_status);
  return cudaGetLastError();
}

cudaError_t launch_eval(const lrvol_s *v, const float *pts, int64_t n, float *out, cudaStream_t s) {
  k_eval<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(forest_view(v), v->d_elem, v->n_elem, v->d_bez,
                                                    v->elem_bytes, v->storage, v->p[0], v->p[1], v->p[2],
                                                    v->nc, pts, n, out, v->d_status);
  return cudaGetLastError();
}

cudaError_t launch_eval_grad(const lrvol_s *v, const float *pts, int64_t n, float *out, cudaStream_t s) {
  k_eval_grad<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(forest_view(v), v->d_elem, v->n_elem, v->d_bez,
                                                         v->elem_bytes, v->storage, v->p[0], v->p[1], v->p[2], pts,
                                                         n, out, v->d_status);
  return cudaGetLastError();
}


// ----------------------------------------------------------------------------
// Learned step sizes: features, BF16 tensor-core inference, FP32 training,
// fine-step labels.  The network is 16 -> 64 -> 64 -> 64 -> 1 (ReLU).
// ----------------------------------------------------------------------------
namespace {

// Range of the rendered field on an element: a component's coefficient range
// (convex hull of the Bezier block), or bounds of |v| from the three ranges.
__device__ __forceinline__ void field_range(const FeatureParams &fp, int64_t e, float &lo, float &hi) {
  if (fp.field == LRVOL_FIELD_MAGNITUDE) {
    float s_lo = 0.f, s_hi = 0.f;
    for (int c = 0; c < 3; ++c) {
      const float2 r = fp.range[e * fp.nc + c];
      const float m = fmaxf(fabsf(r.x), fabsf(r.y));
      const float d = r.x > 0.f ? r.x : (r.y < 0.f ? -r.y : 0.f);   // distance of 0 to [r.x, r.y]
      s_hi = fmaf(m, m, s_hi);
      s_lo = fmaf(d, d, s_lo);
    }
    lo = sqrtf(s_lo);
    hi = sqrtf(s_hi);
  } else {
    const float2 r = fp.range[e * fp.nc + (fp.field == LRVOL_FIELD_COMPONENT ? fp.comp : 0)];
    lo = r.x;
    hi = r.y;
  }
}

// The TF in shared memory with aggregates over blocks of kTfBlock bins (the
// largest opacity, the opacity sum, the largest opacity step to the next bin,
// the RGB range), so that an element's bin range [i0, i1] costs at most
// 2 (kTfBlock - 1) single bins plus whole blocks instead of up to 256 bins:
// one element straddling a sharp TF band would otherwise hold its whole warp.
// Maxima and minima are exact in any order; only the opacity sum is added in
// another order.
constexpr int kTfBlock = 16, kTfBlocks = 256 / kTfBlock;

__global__ void k_features(const __grid_constant__ FeatureParams fp, float *__restrict__ out) {
  __shared__ float4 tfs[256];
  __shared__ float b_amax[kTfBlocks], b_asum[kTfBlocks], b_slope[kTfBlocks];
  __shared__ float b_cmin[3][kTfBlocks], b_cmax[3][kTfBlocks];
  for (int q = threadIdx.x; q < 256; q += blockDim.x) tfs[q] = fp.tf[q];
  __syncthreads();
  if (threadIdx.x < kTfBlocks) {
    const int q = threadIdx.x;
    float am = 0.f, as = 0.f, sl = 0.f;
    float mn[3] = {1e30f, 1e30f, 1e30f}, mx[3] = {-1e30f, -1e30f, -1e30f};
    for (int i = q * kTfBlock; i < (q + 1) * kTfBlock; ++i) {
      const float4 t = tfs[i];
      am = fmaxf(am, t.w);
      as += t.w;
      if (i < 255) sl = fmaxf(sl, fabsf(tfs[i + 1].w - t.w));   // the step from bin i to bin i + 1
      mn[0] = fminf(mn[0], t.x); mx[0] = fmaxf(mx[0], t.x);
      mn[1] = fminf(mn[1], t.y); mx[1] = fmaxf(mx[1], t.y);
      mn[2] = fminf(mn[2], t.z); mx[2] = fmaxf(mx[2], t.z);
    }
    b_amax[q] = am;
    b_asum[q] = as;
    b_slope[q] = sl;
    for (int c = 0; c < 3; ++c) {
      b_cmin[c][q] = mn[c];
      b_cmax[c][q] = mx[c];
    }
  }
  __syncthreads();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= fp.n_elem) return;
  {
    // the box as three 16-byte loads (48 bytes per element, so 16-byte aligned)
    const double2 *b2 = reinterpret_cast<const double2 *>(fp.box + 6 * e);
    const double2 q0 = __ldg(b2), q1 = __ldg(b2 + 1), q2 = __ldg(b2 + 2);
    const double b[6] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y};
    float w[3], ctr[3];
    for (int a = 0; a < 3; ++a) {
      w[a] = (float)(b[3 + a] - b[a]);
      ctr[a] = (float)(0.5 * (b[a] + b[3 + a]));
    }
    const float ds = __ldg(&fp.elem[e].a.w);
    float lo, hi;
    field_range(fp, e, lo, hi);
    const float xlo = fmaf(lo, fp.tf_scale, fp.tf_bias) * (1.f / 255.f);
    const float xhi = fmaf(hi, fp.tf_scale, fp.tf_bias) * (1.f / 255.f);
    const int i0 = (int)floorf(255.f * fminf(fmaxf(xlo, 0.f), 1.f));
    const int i1 = min(255, (int)ceilf(255.f * fminf(fmaxf(xhi, 0.f), 1.f)));
    float amax = 0.f, asum = 0.f, slope = 0.f;
    float cmin[3] = {1e30f, 1e30f, 1e30f}, cmax[3] = {-1e30f, -1e30f, -1e30f};
    auto bin = [&](int i) {
      const float4 t = tfs[i];
      amax = fmaxf(amax, t.w);
      asum += t.w;
      cmin[0] = fminf(cmin[0], t.x); cmax[0] = fmaxf(cmax[0], t.x);
      cmin[1] = fminf(cmin[1], t.y); cmax[1] = fmaxf(cmax[1], t.y);
      cmin[2] = fminf(cmin[2], t.z); cmax[2] = fmaxf(cmax[2], t.z);
    };
    int i = i0;   // bins i0 .. i1: head to a block boundary, whole blocks, tail
    for (; i <= i1 && (i % kTfBlock) != 0; ++i) bin(i);
    for (; i + kTfBlock - 1 <= i1; i += kTfBlock) {
      const int q = i / kTfBlock;
      amax = fmaxf(amax, b_amax[q]);
      asum += b_asum[q];
      for (int c = 0; c < 3; ++c) {
        cmin[c] = fminf(cmin[c], b_cmin[c][q]);
        cmax[c] = fmaxf(cmax[c], b_cmax[c][q]);
      }
    }
    for (; i <= i1; ++i) bin(i);
    // the largest opacity step between neighbouring bins of the range: steps i -> i + 1 for i0 <= i < i1
    for (i = i0; i < i1 && (i % kTfBlock) != 0; ++i) slope = fmaxf(slope, fabsf(tfs[i + 1].w - tfs[i].w));
    for (; i + kTfBlock - 1 < i1; i += kTfBlock) slope = fmaxf(slope, b_slope[i / kTfBlock]);
    for (; i < i1; ++i) slope = fmaxf(slope, fabsf(tfs[i + 1].w - tfs[i].w));
    float dir[3];
    float nn = 0.f;
    for (int a = 0; a < 3; ++a) {
      dir[a] = ctr[a] - fp.eye[a];
      nn = fmaf(dir[a], dir[a], nn);
    }
    nn = rsqrtf(fmaxf(nn, 1e-30f));
    float proj = 0.f;
    for (int a = 0; a < 3; ++a) {
      dir[a] *= nn;
      proj = fmaf(fabsf(dir[a]), w[a], proj);
    }
    const float f[kIn] = {log2f(64.f * w[0]), log2f(64.f * w[1]), log2f(64.f * w[2]), xlo,
                          xhi, xhi - xlo, amax, asum / (float)(i1 - i0 + 1),
                          255.f * slope, fmaxf(cmax[0] - cmin[0], fmaxf(cmax[1] - cmin[1], cmax[2] - cmin[2])),
                          dir[0], dir[1],
                          dir[2], log2f(2048.f * ds), proj / (8.f * ds), log2f(1.f + 255.f * (xhi - xlo))};
    float *o = out + e * kIn;
    if ((reinterpret_cast<uintptr_t>(out) & 15) == 0) {   // one 64-byte row, four 16-byte stores
      float4 *o4 = reinterpret_cast<float4 *>(o);
#pragma unroll
      for (int c = 0; c < kIn / 4; ++c) o4[c] = make_float4(f[4 * c], f[4 * c + 1], f[4 * c + 2], f[4 * c + 3]);
    } else {                                               // a caller's buffer not 16-byte aligned
#pragma unroll
      for (int c = 0; c < kIn; ++c) o[c] = f[c];
    }
  }
}

// ---- the step network on the 5th-generation tensor cores (tcgen05) ----
// Pack: W1, W2, W3 into the canonical K-major layout of tc_off (B[n][k] =
// W[k][n]), w4 as BF16, biases as FP32.
__global__ void k_mlp_pack(const float *__restrict__ p, uint16_t *__restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kPacked) return;
  if (q < kTcW4) {
    const int K = q < kTcW2 ? kIn : kHid;
    const int base = q < kTcW2 ? kTcW1 : (q < kTcW3 ? kTcW2 : kTcW3);
    const int woff = q < kTcW2 ? kOffW1 : (q < kTcW3 ? kOffW2 : kOffW3);
    const int byte = 2 * (q - base), grp = byte / (K * 16), rem = byte % (K * 16);
    const int n = grp * 8 + (rem % 128) / 16, k = (rem / 128) * 8 + (rem % 16) / 2;
    out[q] = __bfloat16_as_ushort(__float2bfloat16_rn(p[woff + k * kHid + n]));
    return;
  }
  if (q < kTcBias) {
    out[q] = __bfloat16_as_ushort(__float2bfloat16_rn(p[kOffW4 + (q - kTcW4)]));
    return;
  }
  const int r = q - kTcBias, f = r >> 1;
  float bv = 0.f;
  if (f < kHid) bv = p[kOffB1 + f];
  else if (f < 2 * kHid) bv = p[kOffB2 + f - kHid];
  else if (f < 3 * kHid) bv = p[kOffB3 + f - 2 * kHid];
  else if (f == 3 * kHid) bv = p[kOffB4];
  const unsigned bits = __float_as_uint(bv);
  out[q] = q >= kTcEnd ? (uint16_t)0 : ((r & 1) ? (uint16_t)(bits >> 16) : (uint16_t)(bits & 0xffffu));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (K-adjacent core matrices) and stride byte offset (8-row groups), all
// in 16-byte units; descriptor version 1 at bit 46; no swizzling (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
constexpr uint32_t kTcM = 128, kTcN = 64;
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kTcN >> 3) << 17) | ((kTcM >> 4) << 24);
constexpr int kTcSpin = 1 << 20;                 // bound on mbarrier polls per wait ...
constexpr uint64_t kTcWaitNs = 100000000ull;     // ... and on its duration (100 ms)

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :: "r"(tmem), "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane; the wait is in the
// same statement, so the registers are complete when it returns.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\ttcgen05.wait::ld.sync.aligned;"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the mbarrier phase with the given parity; false after kTcSpin polls
// or kTcWaitNs nanoseconds, whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  if (mbar_try_wait(mbar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int it = 0; it < kTcSpin; ++it) {
    if (mbar_try_wait(mbar, parity)) return true;
    if (global_ns() - t0 > kTcWaitNs) return false;
  }
  return false;
}

// Synchronisation of the 128 threads of warpgroup g (named barrier 1 + g;
// immediate ids, so only barriers 0-2 are reserved), and the AND of v over them.
__device__ __forceinline__ void wg_sync(int g) {
  if (g == 0) asm volatile("bar.sync 1, 128;" ::: "memory");
  else asm volatile("bar.sync 2, 128;" ::: "memory");
}
__device__ __forceinline__ bool wg_sync_and(int g, bool v) {
  uint32_t r;
  if (g == 0)
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, 1, 128, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v) : "memory");
  else
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, 2, 128, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((uint32_t)v) : "memory");
  return r != 0;
}

// Two BF16 values (round to nearest even) in one word, the first in the low half.
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

constexpr int kTcGroups = 2;                                   // warpgroups (row pipelines) per CTA
constexpr int kTcSmemBytes = 2 * kTcW4 + kTcGroups * 2 * (int)kTcM * kHid;   // weights + operand tiles

// A CTA holds the weights once in shared memory and runs two independent
// pipelines, one per warpgroup, each taking tiles of 128 rows.  Per hidden
// layer the warpgroup's first thread issues the MMAs (M = 128, N = 64, K = 16
// per instruction) from the warpgroup's operand tile and the layer's weights
// into its own 128 x 64 FP32 accumulator in tensor memory, and commits them
// to the warpgroup's mbarrier; every warp then reads its 32 rows back
// (tcgen05.ld), adds the bias, applies ReLU and writes the BF16 activations as
// the next layer's operand tile.  The 64 -> 1 output layer runs on the CUDA
// cores in FP32 on the BF16-rounded operands.  Waits are bounded: a tile
// whose MMAs do not complete gets multiplier 1 (the Eq. 4 step) for its rows
// and for every later tile of that pipeline, and the status word records
// kStatusTimeout.  no_mma (a diagnostic of that path) issues no MMAs and no
// commits, so every pipeline's first wait runs out.
__global__ void __launch_bounds__(128 * kTcGroups, 4) k_mlp_infer(const float *__restrict__ x, int64_t n,
                                                               const uint16_t *__restrict__ packed, float ymin,
                                                               float ymax,
                                                               float *__restrict__ out, uint32_t *__restrict__ status,
                                                               bool no_mma) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  uint16_t *sw = reinterpret_cast<uint16_t *>(tc_smem);                         // W1, W2, W3 (18,432 B)
  __shared__ float sb[3 * kHid + 1], sw4[kHid];
  __shared__ __align__(8) unsigned long long mbar[kTcGroups];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, g = tid >> 7, gt = tid & 127;
  for (int q = tid; q < kTcW4 / 8; q += blockDim.x)
    reinterpret_cast<uint4 *>(sw)[q] = __ldg(reinterpret_cast<const uint4 *>(packed) + q);
  for (int q = tid; q < kHid; q += blockDim.x) sw4[q] = __bfloat162float(__ushort_as_bfloat16(packed[kTcW4 + q]));
  for (int q = tid; q < 3 * kHid + 1; q += blockDim.x)
    sb[q] = __uint_as_float((unsigned)packed[kTcBias + 2 * q] | ((unsigned)packed[kTcBias + 2 * q + 1] << 16));
  if (tid < kTcGroups) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[tid])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tmem_slot)),
                 "r"(kTcN * kTcGroups) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot + kTcN * g;                               // this pipeline's accumulator
  const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);    // this warp's 32 TMEM lanes
  unsigned char *sa = tc_smem + 2 * kTcW4 + g * 2 * kTcM * kHid;            // this pipeline's operand tile
  const uint32_t a_addr = smem_u32(sa), w_addr = smem_u32(sw), mb = smem_u32(&mbar[g]);
  const bool vec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  uint32_t phase = 0;
  bool ok = true;
  const int64_t tiles = (n + kTcM - 1) / kTcM;
  int64_t tile = (int64_t)blockIdx.x * kTcGroups + g;
  for (; tile < tiles; tile += (int64_t)gridDim.x * kTcGroups) {
    const int64_t row = tile * kTcM + gt;
    {  // layer-1 operand: this thread's feature row in BF16 (K = 16)
      float f[kIn];
      if (row < n && vec) {
        const float4 *xr = reinterpret_cast<const float4 *>(x + row * kIn);
#pragma unroll
        for (int c = 0; c < kIn / 4; ++c) {
          const float4 v = __ldg(xr + c);
          f[4 * c] = v.x; f[4 * c + 1] = v.y; f[4 * c + 2] = v.z; f[4 * c + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int c = 0; c < kIn; ++c) f[c] = row < n ? __ldg(x + row * kIn + c) : 0.f;
      }
      unsigned char *dst = sa + tc_off(gt, 0, kIn);
      *reinterpret_cast<uint4 *>(dst) = make_uint4(bf16x2(f[0], f[1]), bf16x2(f[2], f[3]), bf16x2(f[4], f[5]), bf16x2(f[6], f[7]));
      *reinterpret_cast<uint4 *>(dst + 128) =
          make_uint4(bf16x2(f[8], f[9]), bf16x2(f[10], f[11]), bf16x2(f[12], f[13]), bf16x2(f[14], f[15]));
    }
    float y = sb[3 * kHid];
    for (int layer = 0; layer < 3; ++layer) {
      const int K = layer == 0 ? kIn : kHid;
      fence_async_smem();   // the operand tile's generic-proxy stores, visible to the tensor core
      tc_fence_before();
      wg_sync(g);
      if (gt == 0 && !no_mma) {
        tc_fence_after();
        const uint32_t wl = w_addr + 2u * (layer == 0 ? kTcW1 : (layer == 1 ? kTcW2 : kTcW3));
        for (int ks = 0; ks < K / 16; ++ks)
          tc_mma(tmem, tc_desc(a_addr + 256u * ks, 128u, 16u * K), tc_desc(wl + 256u * ks, 128u, 16u * K), ks > 0);
        tc_commit(mb);
      }
      ok = wg_sync_and(g, mbar_wait_bounded(mb, phase));
      phase ^= 1u;
      if (!ok) break;
      tc_fence_after();
      const float *bl = sb + layer * kHid;
      unsigned char *dst = sa + tc_off(gt, 0, kHid);
      float h[16];
#pragma unroll
      for (int c = 0; c < kHid / 8; ++c) {
        if ((c & 1) == 0) tc_ld16(lane_addr + 8 * c, h);   // columns 8c .. 8c + 15
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 8 * c + 2 * q, i = 8 * (c & 1) + 2 * q;
          w[q] = bf16x2(fmaxf(h[i] + bl[j], 0.f), fmaxf(h[i + 1] + bl[j + 1], 0.f));
        }
        if (layer < 2) {
          *reinterpret_cast<uint4 *>(dst + 128 * c) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = 8 * c + 2 * q;
            y = fmaf(__uint_as_float(w[q] << 16), sw4[j], y);
            y = fmaf(__uint_as_float(w[q] & 0xffff0000u), sw4[j + 1], y);
          }
        }
      }
    }
    if (!ok) break;
    if (row < n) out[row] = exp2f(fminf(fmaxf(y, ymin), ymax));
  }
  if (!ok) {
    if (gt == 0) set_status(status, kStatusTimeout);
    for (; tile < tiles; tile += (int64_t)gridDim.x * kTcGroups)
      if (tile * kTcM + gt < n) out[tile * kTcM + gt] = 1.f;
    // one more bounded wait for the MMAs in flight before the accumulator is freed
    if (!no_mma) mbar_wait_bounded(mb, phase ^ 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem_slot), "r"(kTcN * kTcGroups)
                 : "memory");
  }
}

// ---- FP32 training (plain CUDA-core kernels; batch up to 2^20 rows) ----
// out[b][j] = act(sum_k in[b][k] W[k][j] + bias[j])
__global__ void k_dense_fwd(const float *__restrict__ in, int K, const float *__restrict__ W,
                            const float *__restrict__ bias, int N, int64_t n, bool relu, float *__restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * N) return;
  const int64_t b = q / N;
  const int j = (int)(q % N);
  float acc = bias[j];
  for (int k = 0; k < K; ++k) acc = fmaf(in[b * K + k], W[k * N + j], acc);
  out[q] = relu ? fmaxf(acc, 0.f) : acc;
}

// dy[b] = (y[b] - t[b]) / n and the loss (one CTA, fixed order)
__global__ void k_loss(const float *__restrict__ y, const float *__restrict__ tgt, int64_t n, float *__restrict__ dy,
                       float *__restrict__ loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t b = threadIdx.x; b < n; b += blockDim.x) {
    const float r = y[b] - tgt[b];
    dy[b] = r / (float)n;
    acc += 0.5 * (double)r * (double)r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
    if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = (float)(red[0] / (double)n);
}

// gW[k][j] = sum_b in[b][k] d[b][j];  gb[j] = sum_b d[b][j]   (thread per (k, j), fixed order)
__global__ void k_dense_wgrad(const float *__restrict__ in, int K, const float *__restrict__ d, int N, int64_t n,
                              float *__restrict__ gW, float *__restrict__ gb) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (K + 1) * N) return;
  const int k = q / N, j = q % N;
  float acc = 0.f;
  if (k < K) {
    for (int64_t b = 0; b < n; ++b) acc = fmaf(in[b * K + k], d[b * N + j], acc);
    gW[k * N + j] = acc;
  } else {
    for (int64_t b = 0; b < n; ++b) acc += d[b * N + j];
    gb[j] = acc;
  }
}

// din[b][k] = (sum_j d[b][j] W[k][j]) * (in[b][k] > 0)   (in = post-ReLU activations)
__global__ void k_dense_dgrad(const float *__restrict__ d, int N, const float *__restrict__ W,
                              const float *__restrict__ in, int K, int64_t n, float *__restrict__ din) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * K) return;
  const int64_t b = q / K;
  const int k = (int)(q % K);
  float acc = 0.f;
  for (int j = 0; j < N; ++j) acc = fmaf(d[b * N + j], W[k * N + j], acc);
  din[q] = in[q] > 0.f ? acc : 0.f;
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int count, float lr, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const float mq = 0.9f * m[q] + 0.1f * g[q];
  const float vq = 0.999f * v[q] + 0.001f * g[q] * g[q];
  m[q] = mq;
  v[q] = vq;
  p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + 1e-8f);
}

// ---- fine-step labels (scalar volumes, FP32 storage) ----
struct SegState {
  uint32_t e;
  float4 ra, rb, rc, rd;
};

template <int P>
__device__ __forceinline__ bool seg_locate(const RenderParams &prm, SegState &st, Block<P, 0, LRVOL_STORE_F32> &blk,
                                           float px, float py, float pz) {
  const bool inside = st.e != kNone && px >= st.ra.x && py >= st.ra.y && pz >= st.ra.z && px < st.rb.x &&
                      py < st.rb.y && pz < st.rb.z;
  if (inside) return true;
  const uint32_t e = forest_lookup(prm.forest, px, py, pz, prm.status);
  if (e == kNone || (int64_t)e >= prm.n_elem) {
    set_status(prm.status, kStatusBounds);
    return false;
  }
  st.e = e;
  load_record(prm.elem + e, st.ra, st.rb, st.rc, st.rd);
  blk.load(prm.bez + (int64_t)e * prm.elem_bytes, 0);
  return true;
}

// Alg. 2 from transparent over [ta, tb) with samples ta + k*h (each in its element).
template <int P>
__device__ void seg_composite(const RenderParams &prm, const Ray &ray, const float4 *tfb, const float4 *tfd,
                              float ta, float tb, float h, SegState &st, Block<P, 0, LRVOL_STORE_F32> &blk,
                              float &C0, float &C1, float &C2, float &Tr) {
  constexpr int N = P + 1;
  C0 = C1 = C2 = 0.f;
  Tr = 1.f;
  for (int k = 0; k < kMaxSamplesPerRay; ++k) {
    const float t = __fmaf_rn((float)k, h, ta);
    if (!(t < tb)) break;
    const float px = fminf(fmaxf(__fmaf_rn(t, ray.d[0], ray.o[0]), 0.f), 1.f);
    const float py = fminf(fmaxf(__fmaf_rn(t, ray.d[1], ray.o[1]), 0.f), 1.f);
    const float pz = fminf(fmaxf(__fmaf_rn(t, ray.d[2], ray.o[2]), 0.f), 1.f);
    if (!seg_locate<P>(prm, st, blk, px, py, pz)) return;
    float bx[N], by[N], bz[N];
    monomials<P>(local_u(px, st.ra.x, st.rc.x, st.rd.x), bx);
    monomials<P>(local_u(py, st.ra.y, st.rc.y, st.rd.y), by);
    monomials<P>(local_u(pz, st.ra.z, st.rc.z, st.rd.z), bz);
    const float v = blk.eval(bx, by, bz);
    const float tn = __fmaf_rn((float)(k + 1), h, ta);
    composite(tfb, tfd, v, __fsub_rn(fminf(tn, tb), t), prm, C0, C1, C2, Tr);
  }
}

template <int P>
__global__ void __launch_bounds__(128) k_labels(const __grid_constant__ RenderParams prm, float h_fine, float tau,
                                                const float *__restrict__ cand, int n_cand,
                                                int32_t *__restrict__ label) {
  __shared__ float4 tfb[256], tfd[256];
  for (int q = threadIdx.x; q < 256; q += blockDim.x) {
    const float4 e0 = prm.tf[q], e1 = prm.tf[q < 255 ? q + 1 : 255];
    tfb[q] = e0;
    tfd[q] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
  const int j = prm.row_begin + blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
  if (i >= prm.width || j >= prm.row_end) return;
  Ray ray;
  if (!make_ray(prm.ray, i, j, ray)) return;
  Block<P, 0, LRVOL_STORE_F32> blk;
  SegState st;
  st.e = kNone;
  const float tr_stop = 1.f - prm.alpha_stop;
  float Tfront = 1.f;
  float t = ray.tin;
  for (int visit = 0; visit < kMaxSamplesPerRay && t < ray.tout && Tfront > tr_stop; ++visit) {
    // the visit: element of the heuristic sample at t, up to the first heuristic sample past it
    float px = fminf(fmaxf(__fmaf_rn(t, ray.d[0], ray.o[0]), 0.f), 1.f);
    float py = fminf(fmaxf(__fmaf_rn(t, ray.d[1], ray.o[1]), 0.f), 1.f);
    float pz = fminf(fmaxf(__fmaf_rn(t, ray.d[2], ray.o[2]), 0.f), 1.f);
    if (!seg_locate<P>(prm, st, blk, px, py, pz)) return;
    const uint32_t e = st.e;
    const float4 ra = st.ra, rb = st.rb;
    const float ds = ra.w;
    float tb = t;
    for (int q = 0; q < kMaxSamplesPerRay; ++q) {
      tb = __fadd_rn(tb, ds);
      if (!(tb < ray.tout)) break;
      px = fminf(fmaxf(__fmaf_rn(tb, ray.d[0], ray.o[0]), 0.f), 1.f);
      py = fminf(fmaxf(__fmaf_rn(tb, ray.d[1], ray.o[1]), 0.f), 1.f);
      pz = fminf(fmaxf(__fmaf_rn(tb, ray.d[2], ray.o[2]), 0.f), 1.f);
      if (!(px >= ra.x && py >= ra.y && pz >= ra.z && px < rb.x && py < rb.y && pz < rb.z)) break;
    }
    tb = fminf(tb, ray.tout);
    float R0, R1, R2, RT;
    seg_composite<P>(prm, ray, tfb, tfd, t, tb, h_fine, st, blk, R0, R1, R2, RT);
    int best = 0;
    for (int c = 1; c < n_cand; ++c) {
      // the candidate's first sample outside e (or the ray's exit)
      const float sc = __fmul_rn(ds, cand[c]);
      float tc = t;
      for (int k = 1; k < kMaxSamplesPerRay; ++k) {
        tc = __fmaf_rn((float)k, sc, t);
        if (!(tc < ray.tout)) break;
        px = fminf(fmaxf(__fmaf_rn(tc, ray.d[0], ray.o[0]), 0.f), 1.f);
        py = fminf(fmaxf(__fmaf_rn(tc, ray.d[1], ray.o[1]), 0.f), 1.f);
        pz = fminf(fmaxf(__fmaf_rn(tc, ray.d[2], ray.o[2]), 0.f), 1.f);
        if (!(px >= ra.x && py >= ra.y && pz >= ra.z && px < rb.x && py < rb.y && pz < rb.z)) break;
      }
      tc = fminf(tc, ray.tout);
      float F0, F1, F2, FT, A0, A1, A2, AT;
      seg_composite<P>(prm, ray, tfb, tfd, t, tc, h_fine, st, blk, F0, F1, F2, FT);
      seg_composite<P>(prm, ray, tfb, tfd, t, tc, sc, st, blk, A0, A1, A2, AT);
      const float err = Tfront * fmaxf(fmaxf(fabsf(A0 - F0), fabsf(A1 - F1)), fmaxf(fabsf(A2 - F2), fabsf(AT - FT)));
      if (!(err <= tau)) break;
      best = c;
    }
    atomicMin(label + e, best);
    Tfront *= RT;
    t = tb;
  }
}

}  // namespace

cudaError_t launch_features(const FeatureParams &fp, float *out, cudaStream_t s) {
  if (fp.n_elem == 0) return cudaSuccess;
  k_features<<<(unsigned)((fp.n_elem + 127) / 128), 128, 0, s>>>(fp, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float *params, uint16_t *packed, cudaStream_t s) {
  k_mlp_pack<<<(kPacked + 255) / 256, 256, 0, s>>>(params, packed);
  return cudaGetLastError();
}

__device__ uint32_t g_mlp_status;

uint32_t *mlp_status_word() {
  void *p = nullptr;
  return cudaGetSymbolAddress(&p, g_mlp_status) == cudaSuccess ? static_cast<uint32_t *>(p) : nullptr;
}

cudaError_t launch_mlp_infer(const float *x, int64_t n, const uint16_t *packed, float ymin, float ymax, float *out,
                             uint32_t *status, cudaStream_t s, bool no_mma) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  static bool smem_set = false;
  if (!smem_set) {
    const cudaError_t e = cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
    if (e != cudaSuccess) return e;
    smem_set = true;
  }
  // Shared memory (about 52 KB per CTA) allows at most 4 CTAs per SM, so their
  // tensor memory (128 columns each) never exceeds the SM's 512 columns.
  const int64_t tiles = (n + kTcM - 1) / kTcM;
  const int64_t blocks = std::min<int64_t>((tiles + kTcGroups - 1) / kTcGroups, 4 * (int64_t)sms);
  k_mlp_infer<<<(unsigned)std::max<int64_t>(blocks, 1), 128 * kTcGroups, kTcSmemBytes, s>>>(x, n, packed, ymin, ymax,
                                                                                           out, status, no_mma);
  return cudaGetLastError();
}

// Scratch layout (floats): h1, h2, h3 (n x 64 each), y (n), dy (n), d3, d2, d1 (n x 64 each)
cudaError_t launch_mlp_grad(const float *x, const float *target, int64_t n, const float *p, float *grad,
                            float *loss, float *scratch, cudaStream_t s) {
  float *h1 = scratch, *h2 = h1 + n * kHid, *h3 = h2 + n * kHid, *y = h3 + n * kHid, *dy = y + n;
  float *d3 = dy + n, *d2 = d3 + n * kHid, *d1 = d2 + n * kHid;
  const unsigned thr = 256;
  auto blocks = [&](int64_t c) { return (unsigned)((c + thr - 1) / thr); };
  k_dense_fwd<<<blocks(n * kHid), thr, 0, s>>>(x, kIn, p + kOffW1, p + kOffB1, kHid, n, true, h1);
  k_dense_fwd<<<blocks(n * kHid), thr, 0, s>>>(h1, kHid, p + kOffW2, p + kOffB2, kHid, n, true, h2);
  k_dense_fwd<<<blocks(n * kHid), thr, 0, s>>>(h2, kHid, p + kOffW3, p + kOffB3, kHid, n, true, h3);
  k_dense_fwd<<<blocks(n), thr, 0, s>>>(h3, kHid, p + kOffW4, p + kOffB4, 1, n, false, y);
  k_loss<<<1, 256, 0, s>>>(y, target, n, dy, loss);
  k_dense_wgrad<<<blocks((kHid + 1) * 1), thr, 0, s>>>(h3, kHid, dy, 1, n, grad + kOffW4, grad + kOffB4);
  k_dense_dgrad<<<blocks(n * kHid), thr, 0, s>>>(dy, 1, p + kOffW4, h3, kHid, n, d3);
  k_dense_wgrad<<<blocks((kHid + 1) * kHid), thr, 0, s>>>(h2, kHid, d3, kHid, n, grad + kOffW3, grad + kOffB3);
  k_dense_dgrad<<<blocks(n * kHid), thr, 0, s>>>(d3, kHid, p + kOffW3, h2, kHid, n, d2);
  k_dense_wgrad<<<blocks((kHid + 1) * kHid), thr, 0, s>>>(h1, kHid, d2, kHid, n, grad + kOffW2, grad + kOffB2);
  k_dense_dgrad<<<blocks(n * kHid), thr, 0, s>>>(d2, kHid, p + kOffW2, h1, kHid, n, d1);
  k_dense_wgrad<<<blocks((kIn + 1) * kHid), thr, 0, s>>>(x, kIn, d1, kHid, n, grad + kOffW1, grad + kOffB1);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *params, const float *grad, float *m, float *v, int64_t t, float lr, cudaStream_t s) {
  const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
  k_adam<<<(kParams + 255) / 256, 256, 0, s>>>(params, grad, m, v, kParams, lr, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_labels(const RenderParams &prm, int degree, float h_fine, float tau, const float *cand, int n_cand,
                          int32_t *label, cudaStream_t s) {
  const dim3 grid((unsigned)((prm.width + 15) / 16), (unsigned)((prm.row_end - prm.row_begin + 7) / 8));
  switch (degree) {
    case 1: k_labels<1><<<grid, 128, 0, s>>>(prm, h_fine, tau, cand, n_cand, label); break;
    case 2: k_labels<2><<<grid, 128, 0, s>>>(prm, h_fine, tau, cand, n_cand, label); break;
    case 3: k_labels<3><<<grid, 128, 0, s>>>(prm, h_fine, tau, cand, n_cand, label); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Trimming (Sec. 4.1).  The paper's z-prepass rasterises the boundary mesh's
// front and back faces into two depth buffers; here each triangle is one
// warp that tests the rays of the pixels in its conservative screen box
// (watertight test, FP32, in the oracle's order of operations) and keeps
// the nearest front-face and farthest back-face distances with atomics on
// the float bits (t > 0, so bit order is value order).
// ----------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float pick3(int k, float x, float y, float z) { return k == 0 ? x : (k == 1 ? y : z); }

// Watertight ray/triangle test (Woop, Benthin and Wald, JCGT 2013), FP32,
// with the oracle's order of operations; component selection by value so
// that nothing goes to local memory.
// v: the triangle's 9 coordinates, in global memory or in registers (plain loads).
__device__ __forceinline__ bool tri_hit(const Ray &ray, const float *__restrict__ v, float &t, bool &front) {
  const float d0 = ray.d[0], d1 = ray.d[1], d2 = ray.d[2];
  int kz = 0;
  if (fabsf(d1) > fabsf(pick3(kz, d0, d1, d2))) kz = 1;
  if (fabsf(d2) > fabsf(pick3(kz, d0, d1, d2))) kz = 2;
  int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
  const float dz = pick3(kz, d0, d1, d2);
  if (dz < 0.f) {
    const int w = kx;
    kx = ky;
    ky = w;
  }
  const float Sx = __fdiv_rn(pick3(kx, d0, d1, d2), dz), Sy = __fdiv_rn(pick3(ky, d0, d1, d2), dz);
  const float Sz = __fdiv_rn(1.f, dz);
  const float a0 = __fsub_rn(v[0], ray.o[0]), a1 = __fsub_rn(v[1], ray.o[1]);
  const float a2 = __fsub_rn(v[2], ray.o[2]);
  const float b0 = __fsub_rn(v[3], ray.o[0]), b1 = __fsub_rn(v[4], ray.o[1]);
  const float b2 = __fsub_rn(v[5], ray.o[2]);
  const float c0 = __fsub_rn(v[6], ray.o[0]), c1 = __fsub_rn(v[7], ray.o[1]);
  const float c2 = __fsub_rn(v[8], ray.o[2]);
  const float Akz = pick3(kz, a0, a1, a2), Bkz = pick3(kz, b0, b1, b2), Ckz = pick3(kz, c0, c1, c2);
  const float Ax = __fsub_rn(pick3(kx, a0, a1, a2), __fmul_rn(Sx, Akz));
  const float Ay = __fsub_rn(pick3(ky, a0, a1, a2), __fmul_rn(Sy, Akz));
  const float Bx = __fsub_rn(pick3(kx, b0, b1, b2), __fmul_rn(Sx, Bkz));
  const float By = __fsub_rn(pick3(ky, b0, b1, b2), __fmul_rn(Sy, Bkz));
  const float Cx = __fsub_rn(pick3(kx, c0, c1, c2), __fmul_rn(Sx, Ckz));
  const float Cy = __fsub_rn(pick3(ky, c0, c1, c2), __fmul_rn(Sy, Ckz));
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.f || V == 0.f || W == 0.f) {
    U = __double2float_rn(__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx)));
    V = __double2float_rn(__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx)));
    W = __double2float_rn(__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax)));
  }
  if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
  const float det = __fadd_rn(__fadd_rn(U, V), W);
  if (det == 0.f) return false;
  const float Az = __fmul_rn(Sz, Akz), Bz = __fmul_rn(Sz, Bkz), Cz = __fmul_rn(Sz, Ckz);
  const float T = __fadd_rn(__fadd_rn(__fmul_rn(U, Az), __fmul_rn(V, Bz)), __fmul_rn(W, Cz));
  if (det > 0.f ? !(T > 0.f) : !(T < 0.f)) return false;
  t = __fdiv_rn(T, det);
  front = det > 0.f;
  return true;
}

// The pixels whose centres (i + 1/2, j + 1/2) project into the image-plane
// box [amin, amax] x [bmin, bmax], widened by a margin: 1/4 pixel plus 1e-5
// of the box's coordinates in pixels.  The FP32 projection of a primitive's
// vertices and the FP32 pixel rays of make_ray are each within a few ulps of
// exact, a few thousandths of a pixel even for narrow fields of view, so
// every pixel whose ray can hit the primitive is in the box.  False if the
// box holds no pixel centre.
__device__ __forceinline__ bool pixel_box(const RayConsts &K, int width, int height, float amin, float amax,
                                          float bmin, float bmax, int &i0, int &i1, int &j0, int &j1) {
  const float ia = (amin - K.sxo) / K.sxs - 0.5f, ib = (amax - K.sxo) / K.sxs - 0.5f;
  const float ja = (bmin - K.syo) / K.sys - 0.5f, jb = (bmax - K.syo) / K.sys - 0.5f;
  const float mi = 0.25f + 1e-5f * (fabsf(amin) + fabsf(amax) + 1.f) / fabsf(K.sxs);
  const float mj = 0.25f + 1e-5f * (fabsf(bmin) + fabsf(bmax) + 1.f) / fabsf(K.sys);
  // clamp before converting (NaN widens to the whole image)
  const float lo_i = fmaxf(fminf(ia, ib) - mi, -1.f), hi_i = fminf(fmaxf(ia, ib) + mi, (float)width);
  const float lo_j = fmaxf(fminf(ja, jb) - mj, -1.f), hi_j = fminf(fmaxf(ja, jb) + mj, (float)height);
  i0 = max(0, (int)ceilf(lo_i));
  i1 = min(width - 1, (int)floorf(hi_i));
  j0 = max(0, (int)ceilf(lo_j));
  j1 = min(height - 1, (int)floorf(hi_j));
  return i0 <= i1 && j0 <= j1;
}

__global__ void k_trim_init(float2 *__restrict__ out, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = make_float2(__int_as_float(0x7f800000), 0.f);
}

// One warp takes 32 consecutive triangles: lane l projects triangle l of the
// group and finds its pixel box, then the warp walks the group's (triangle,
// pixel) pairs 32 at a time, each lane finding its pair's triangle by a
// search over the lanes' prefix sums and fetching that triangle by shuffles.
// Small triangles (most of a fine mesh covers a pixel centre or none) then
// cost one lane's set-up instead of a warp's.  `split` warps share a group,
// each taking a contiguous part of its pairs, so a coarse mesh of large
// triangles still spreads over the GPU.
__global__ void __launch_bounds__(128) k_trim_raster(const RayConsts K, int width, int height,
                                                     const float *__restrict__ tri, int64_t n_tri, int split,
                                                     float2 *__restrict__ out) {
  const unsigned full_mask = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t wid = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int64_t group = wid / split;
  const int part = (int)(wid - group * split);
  if (group * 32 >= n_tri) return;   // whole warp
  const int64_t tr = group * 32 + lane;
  float v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = 0.f;
  int i0 = 0, j0 = 0, bw = 1, cnt = 0;
  if (tr < n_tri) {
#pragma unroll
    for (int c = 0; c < 9; ++c) v[c] = __ldg(tri + 9 * tr + c);
    // conservative pixel box of the projected triangle (whole image when a
    // vertex is at or behind the eye plane; nothing when all three are)
    float amin = __int_as_float(0x7f800000), amax = -amin, bmin = amin, bmax = -amin;
    bool full = false;
    int behind = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float X = v[3 * q] - K.E[0], Y = v[3 * q + 1] - K.E[1], Z = v[3 * q + 2] - K.E[2];
      const float r = X * K.R[0] + Y * K.R[1] + Z * K.R[2];
      const float u = X * K.U[0] + Y * K.U[1] + Z * K.U[2];
      float a = r, b = u;
      if (K.persp) {
        const float z = X * K.F[0] + Y * K.F[1] + Z * K.F[2];
        if (!(z > 1e-6f)) {
          full = true;
          ++behind;
          continue;
        }
        a = r / z;
        b = u / z;
      }
      amin = fminf(amin, a);
      amax = fmaxf(amax, a);
      bmin = fminf(bmin, b);
      bmax = fmaxf(bmax, b);
    }
    int i1 = width - 1, j1 = height - 1;
    if (behind < 3 && (full || pixel_box(K, width, height, amin, amax, bmin, bmax, i0, i1, j0, j1))) {
      if (full) {
        i0 = 0;
        j0 = 0;
        i1 = width - 1;
        j1 = height - 1;
      }
      bw = i1 - i0 + 1;
      cnt = bw * (j1 - j0 + 1);   // <= 32768^2 < 2^31
    }
  }
  // prefix sums of the lanes' pair counts
  long long inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(full_mask, inc, o);
    if (lane >= o) inc += y;
  }
  const long long total = __shfl_sync(full_mask, inc, 31), exc = inc - cnt;
  const long long chunk = (((total + split - 1) / split) + 31) & ~31ll;
  const long long w0 = (long long)part * chunk, w1 = w0 + chunk < total ? w0 + chunk : total;
  for (long long base = w0; base < w1; base += 32) {
    const long long w = base + lane;
    int q = 0;   // the last lane whose pairs start at or before w (its count is then > 0)
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const long long e = __shfl_sync(full_mask, exc, q + step);
      if (e <= w) q += step;
    }
    const long long eq = __shfl_sync(full_mask, exc, q);
    const int qi0 = __shfl_sync(full_mask, i0, q), qj0 = __shfl_sync(full_mask, j0, q);
    const int qbw = __shfl_sync(full_mask, bw, q);
    float tv[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) tv[c] = __shfl_sync(full_mask, v[c], q);
    if (w >= w1) continue;
    const unsigned pix = (unsigned)(w - eq);
    const int i = qi0 + (int)(pix % (unsigned)qbw), j = qj0 + (int)(pix / (unsigned)qbw);
    Ray ray;
    make_ray(K, i, j, ray);   // origin and direction; the unit-cube interval is not needed here
    float t;
    bool front;
    if (!tri_hit(ray, tv, t, front)) continue;
    unsigned *slot = reinterpret_cast<unsigned *>(out + (int64_t)j * width + i);
    if (front)
      atomicMin(slot, __float_as_uint(t));
    else
      atomicMax(slot + 1, __float_as_uint(t));
  }
}

}  // namespace

cudaError_t launch_trim(const RayConsts &ray, int width, int height, const float *tri, int64_t n_tri, float *out,
                        cudaStream_t s) {
  const int64_t npix = (int64_t)width * height;
  float2 *o = reinterpret_cast<float2 *>(out);
  k_trim_init<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(o, npix);
  if (n_tri > 0) {
    // warps per group of 32 triangles: about 512 pairs per warp when the
    // mesh covers the image twice, 1 for fine meshes, at most 256
    const int64_t groups = (n_tri + 31) / 32;
    int64_t split = (2 * npix + groups * 512 - 1) / (groups * 512);
    split = split < 1 ? 1 : (split > 256 ? 256 : split);
    const int64_t warps = groups * split;
    k_trim_raster<<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(ray, width, height, tri, n_tri, (int)split, o);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Streamlines (Sec. 5): dx/dt = f(x) by explicit Runge-Kutta methods (Eq. 5),
// one thread per seed.  The outer loop keeps x as an unevaluated float pair
// (hi + lo, about 48 significant bits) and t in FP64: on GB300 FP64
// arithmetic runs at a small fraction of the FP32 rate, and compensated
// FP32 sums keep the accumulation exact enough that the steps are not lost
// to rounding (the reason for the paper's double-precision outer loop,
// Sec. 5.5).  Stage increments h * sum a_ij k_j are formed in FP32 (they
// are small against x) and added exactly; the field is evaluated in FP32
// at the FP32 rounding of the stage point, reusing the element (box and
// block in registers) while consecutive points stay in it.
// ----------------------------------------------------------------------------
namespace {

struct __align__(32) SLSample {
  double x, y, z, t;
};

// A sample x = (double)x_hi + (double)x_lo.  With fewer than 32 lines per
// warp the tracing kernel stores the float pairs (x_hi, x_lo, y_hi, y_lo,
// z_hi, z_lo) and t in the same 32 bytes instead, and a second pass widens
// them in place with all 32 lanes of a warp on one line's samples: FP64
// instructions cost the same per warp whatever the number of active lanes.
// With full warps the extra pass over the samples costs more than it saves.
__device__ __forceinline__ void store_sample(SLSample *o, const float *xh, const float *xl, double t, bool pairs) {
  if (pairs) {
    float4 *o4 = reinterpret_cast<float4 *>(o);
    o4[0] = make_float4(xh[0], xl[0], xh[1], xl[1]);
    o4[1] = make_float4(xh[2], xl[2], __int_as_float(__double2loint(t)), __int_as_float(__double2hiint(t)));
  } else {
    *o = SLSample{(double)xh[0] + (double)xl[0], (double)xh[1] + (double)xl[1], (double)xh[2] + (double)xl[2], t};
  }
}

struct SLTab {
  int s, embedded, q_low;
  float a[6][6], b[6], bh[6];
};

// Butcher tableaus in the order of LRVOL_RK1 .. LRVOL_RKF45 (coefficients in FP32).
__constant__ SLTab c_sl_tab[9] = {
    {1, 0, 0, {}, {1.f}, {}},
    {2, 0, 0, {{0.f}, {0.5f}}, {0.f, 1.f}, {}},
    {3, 0, 0, {{0.f}, {0.5f}, {-1.f, 2.f}}, {1.f / 6, 2.f / 3, 1.f / 6}, {}},
    {4, 0, 0, {{0.f}, {0.5f}, {0.f, 0.5f}, {0.f, 0.f, 1.f}}, {1.f / 6, 1.f / 3, 1.f / 3, 1.f / 6}, {}},
    {4, 0, 0, {{0.f}, {1.f / 3}, {-1.f / 3, 1.f}, {1.f, -1.f, 1.f}}, {0.125f, 0.375f, 0.375f, 0.125f}, {}},
    {6, 0, 4,
     {{0.f},
      {0.25f},
      {3.f / 32, 9.f / 32},
      {1932.f / 2197, -7200.f / 2197, 7296.f / 2197},
      {439.f / 216, -8.f, 3680.f / 513, -845.f / 4104},
      {-8.f / 27, 2.f, -3544.f / 2565, 1859.f / 4104, -11.f / 40}},
     {16.f / 135, 0.f, 6656.f / 12825, 28561.f / 56430, -9.f / 50, 2.f / 55},
     {25.f / 216, 0.f, 1408.f / 2565, 2197.f / 4104, -0.2f, 0.f}},
    {2, 1, 1, {{0.f}, {1.f}}, {0.5f, 0.5f}, {1.f, 0.f}},
    {4, 1, 2, {{0.f}, {0.5f}, {0.f, 0.75f}, {2.f / 9, 1.f / 3, 4.f / 9}}, {2.f / 9, 1.f / 3, 4.f / 9, 0.f},
     {7.f / 24, 0.25f, 1.f / 3, 0.125f}},
    {6, 1, 4,
     {{0.f},
      {0.25f},
      {3.f / 32, 9.f / 32},
      {1932.f / 2197, -7200.f / 2197, 7296.f / 2197},
      {439.f / 216, -8.f, 3680.f / 513, -845.f / 4104},
      {-8.f / 27, 2.f, -3544.f / 2565, 1859.f / 4104, -11.f / 40}},
     {16.f / 135, 0.f, 6656.f / 12825, 28561.f / 56430, -9.f / 50, 2.f / 55},
     {25.f / 216, 0.f, 1408.f / 2565, 2197.f / 4104, -0.2f, 0.f}},
};

// x + d for x = hi + lo and a float d, renormalised (two-sum, then fast two-sum)
__device__ __forceinline__ void ff_add(float &hi, float &lo, float d) {
  const float s = __fadd_rn(hi, d);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
  const float t = __fadd_rn(e, lo);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

template <int P, int STORE>
struct SLField {
  static constexpr int N = P + 1;
  float4 ra, rb, rc, rd;
  uint32_t cur;
  Block<P, 1, STORE> blk;

  // f at the FP32 point p; false outside [0,1]^3 (or on a failed look-up)
  __device__ __forceinline__ bool eval(const SLParams &sp, float px, float py, float pz, float &v0, float &v1,
                                       float &v2) {
    if (!(px >= 0.f && px <= 1.f && py >= 0.f && py <= 1.f && pz >= 0.f && pz <= 1.f)) return false;
    if (!locate(sp, px, py, pz)) return false;
    float bx[N], by[N], bz[N];
    monomials<P>(local_u(px, ra.x, rc.x, rd.x), bx);
    monomials<P>(local_u(py, ra.y, rc.y, rd.y), by);
    monomials<P>(local_u(pz, ra.z, rc.z, rd.z), bz);
    blk.components(bx, by, bz, v0, v1, v2);
    return true;
  }

  __device__ __forceinline__ bool locate(const SLParams &sp, float px, float py, float pz) {
    if (cur != kNone && px >= ra.x && py >= ra.y && pz >= ra.z && px < rb.x && py < rb.y && pz < rb.z) return true;
    const uint32_t e = forest_lookup(sp.forest, px, py, pz, sp.status);
    if (e == kNone || (int64_t)e >= sp.n_elem) {
      set_status(sp.status, kStatusBounds);
      return false;
    }
    cur = e;
    load_record(sp.elem + e, ra, rb, rc, rd);
    blk.load(sp.bez + (int64_t)e * sp.elem_bytes, 0);
    return true;
  }
};

// One streamline, seed q.
template <int P, int STORE>
__device__ __forceinline__ void trace_line(const SLParams &sp, const double *__restrict__ seeds, int64_t q,
                                           SLSample *__restrict__ out, int32_t *__restrict__ count,
                                           int32_t *__restrict__ status) {
  const SLTab &T = c_sl_tab[sp.method];
  SLField<P, STORE> F;
  F.cur = kNone;
  float xh[3], xl[3];
  for (int a = 0; a < 3; ++a) {
    const double s = seeds[3 * q + a];
    xh[a] = __double2float_rn(s);
    xl[a] = __double2float_rn(s - (double)xh[a]);
  }
  SLSample *o = out + q * (int64_t)sp.max_samples;
  int nout = 0, st = 0;
  float v0, v1, v2;
  if (!(xh[0] >= 0.f && xh[0] <= 1.f && xh[1] >= 0.f && xh[1] <= 1.f && xh[2] >= 0.f && xh[2] <= 1.f) ||
      !F.locate(sp, xh[0], xh[1], xh[2])) {
    count[q] = 0;
    status[q] = 1;
    return;
  }
  store_sample(o, xh, xl, 0.0, sp.pair_out);
  nout = 1;
  // FP64 runs at a small fraction of the FP32 rate on GB300, so the time
  // bookkeeping keeps to one FP64 add per step: h and fl32(h) change only
  // with the element (Eq. 4 rule) or the controller (adaptive rule); the
  // comparisons with t_end compare bit patterns (t, t_end >= 0 order like
  // their bits); the loop ends on a flag set with the step that reaches t_end.
  double t = 0.0;
  float dsn = F.ra.w;  // Eq. 4 step of the element holding x_n
  double h = sp.rule == 0 ? sp.h : (sp.rule == 1 ? sp.h * (double)dsn : (sp.h > 0.0 ? sp.h : (double)dsn));
  float hf_h = __double2float_rn(h), ds_h = dsn;   // fl32(h); the Eq. 4 step h was formed from
  const long long t_end_bits = __double_as_longlong(sp.t_end);
  bool done = false;   // t >= t_end (t_end > 0 is checked on the host)
  for (;;) {
    if (done) {
      st = 0;
      break;
    }
    if (nout >= sp.max_samples) {
      st = 2;
      break;
    }
    if (sp.rule == 1 && dsn != ds_h) {
      h = sp.h * (double)dsn;
      hf_h = __double2float_rn(h);
      ds_h = dsn;
    }
    bool taken = false, left = false;
    float nh[3], nl[3];
    for (int tries = 0; tries < 64 && !taken; ++tries) {
      const double tn = t + h;
      const bool last = __double_as_longlong(tn) > t_end_bits;
      double hs = h;
      float hf = hf_h;
      if (last) {
        hs = sp.t_end - t;
        hf = __double2float_rn(hs);
      }
      float k[6][3];
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i < T.s) {
          float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
          for (int j = 0; j < i; ++j) {
            const float a = T.a[i][j];
            d0 = fmaf(a, k[j][0], d0);
            d1 = fmaf(a, k[j][1], d1);
            d2 = fmaf(a, k[j][2], d2);
          }
          float yh0 = xh[0], yl0 = xl[0], yh1 = xh[1], yl1 = xl[1], yh2 = xh[2], yl2 = xl[2];
          if (i > 0) {
            ff_add(yh0, yl0, hf * d0);
            ff_add(yh1, yl1, hf * d1);
            ff_add(yh2, yl2, hf * d2);
          }
          if (!left && !F.eval(sp, yh0, yh1, yh2, v0, v1, v2)) left = true;
          k[i][0] = v0;
          k[i][1] = v1;
          k[i][2] = v2;
        }
      }
      if (left) break;
      float D0 = 0.f, D1 = 0.f, D2 = 0.f, E0 = 0.f, E1 = 0.f, E2 = 0.f;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (i < T.s) {
          const float b = T.b[i], e = T.b[i] - T.bh[i];
          D0 = fmaf(b, k[i][0], D0);
          D1 = fmaf(b, k[i][1], D1);
          D2 = fmaf(b, k[i][2], D2);
          E0 = fmaf(e, k[i][0], E0);
          E1 = fmaf(e, k[i][1], E1);
          E2 = fmaf(e, k[i][2], E2);
        }
      }
      if (sp.rule == 2) {
        const float err = hf * sqrtf(fmaf(E0, E0, fmaf(E1, E1, E2 * E2)));
        float fac = err > 0.f ? 0.9f * powf(sp.tol_f / err, 1.f / (float)(T.q_low + 1)) : 5.f;
        fac = fminf(fmaxf(fac, 0.2f), 5.f);
        if (err > sp.tol_f) {
          h = hs * (double)fac;
          hf_h = __double2float_rn(h);
          continue;
        }
        if (!last) {
          h = hs * (double)fac;
          hf_h = __double2float_rn(h);
        }
      }
      for (int a = 0; a < 3; ++a) {
        nh[a] = xh[a];
        nl[a] = xl[a];
      }
      ff_add(nh[0], nl[0], hf * D0);
      ff_add(nh[1], nl[1], hf * D1);
      ff_add(nh[2], nl[2], hf * D2);
      if (!(nh[0] >= 0.f && nh[0] <= 1.f && nh[1] >= 0.f && nh[1] <= 1.f && nh[2] >= 0.f && nh[2] <= 1.f) ||
          !F.locate(sp, nh[0], nh[1], nh[2])) {
        left = true;
        break;
      }
      dsn = F.ra.w;
      t = last ? sp.t_end : tn;
      done = last || __double_as_longlong(tn) == t_end_bits;
      taken = true;
    }
    if (left) {
      st = 1;
      break;
    }
    if (!taken) {
      st = 3;
      break;
    }
    for (int a = 0; a < 3; ++a) {
      xh[a] = nh[a];
      xl[a] = nl[a];
    }
    store_sample(o + nout++, xh, xl, t, sp.pair_out);
  }
  count[q] = nout;
  status[q] = st;
}

// Persistent threads: a grid that fits on the GPU at once takes lines from
// a counter until none is left, so lines of very different lengths do not
// leave a partial last wave idle behind the longest one.  Only the first
// `lanes` lanes of each warp trace lines: with fewer lines than the GPU has
// warp slots, one line per warp keeps a line from waiting on its warp-mates'
// element look-ups (a line's steps are a sequential chain, so its latency is
// what a small rake of seeds waits for).
template <int P, int STORE>
__global__ void __launch_bounds__(128) k_streamlines(const __grid_constant__ SLParams sp,
                                                     const double *__restrict__ seeds, int64_t n, int lanes,
                                                     SLSample *__restrict__ out, int32_t *__restrict__ count,
                                                     int32_t *__restrict__ status) {
  if ((int)(threadIdx.x & 31) >= lanes) return;
  for (;;) {
    const int64_t q = (int64_t)atomicAdd(sp.queue, 1ull);
    if (q >= n) return;
    trace_line<P, STORE>(sp, seeds, q, out, count, status);
  }
}

// The FP64 samples x = (double)x_hi + (double)x_lo, in place; one warp per line.
__global__ void __launch_bounds__(128) k_sl_widen(SLSample *__restrict__ out, const int32_t *__restrict__ count,
                                                  int64_t n, int max_samples) {
  const int64_t q = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (q >= n) return;
  SLSample *o = out + q * (int64_t)max_samples;
  const int c = count[q];
  for (int i = threadIdx.x & 31; i < c; i += 32) {
    const float4 *p4 = reinterpret_cast<const float4 *>(o + i);
    const float4 a = p4[0], b = p4[1];
    o[i] = SLSample{(double)a.x + (double)a.y, (double)a.z + (double)a.w, (double)b.x + (double)b.y,
                    __hiloint2double(__float_as_int(b.w), __float_as_int(b.z))};
  }
}

// Eq. 7 per streamline: sum over the approximation's samples i >= 1 of
// (t_i - t_{i-1}) * |x_ref(t_i) - y_i|, x_ref linear between its samples.
__global__ void __launch_bounds__(128) k_streamline_error(const SLSample *__restrict__ ref,
                                                          const int32_t *__restrict__ rc, int rmax,
                                                          const SLSample *__restrict__ app,
                                                          const int32_t *__restrict__ ac, int amax, int64_t n,
                                                          double *__restrict__ sums) {
  // one warp per line; lane l takes the approximation's samples l+1, l+33, ...
  const int64_t q = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (q >= n) return;
  const int lane = threadIdx.x & 31;
  const SLSample *r = ref + q * (int64_t)rmax, *y = app + q * (int64_t)amax;
  const int nr = rc[q], na = ac[q];
  double acc = 0.0;
  if (nr >= 2 && na >= 2) {
    const double tlast = r[nr - 1].t;
    for (int i = 1 + lane; i < na; i += 32) {
      const SLSample p = y[i];
      if (!(p.t <= tlast)) break;   // the samples after it are later still
      // reference segment [j, j+1]: j = #{m in [1, nr-2] : t_m < t_i}, the
      // first segment that ends at or after t_i (reference times increase)
      int lo = 1, hi = nr - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (r[mid].t < p.t)
          lo = mid + 1;
        else
          hi = mid;
      }
      const SLSample r0 = r[lo - 1], r1 = r[lo];
      const double dt = r1.t - r0.t;
      const double f = dt > 0.0 ? (p.t - r0.t) / dt : 0.0;
      const double ex = fma(f, r1.x - r0.x, r0.x) - p.x;
      const double ey = fma(f, r1.y - r0.y, r0.y) - p.y;
      const double ez = fma(f, r1.z - r0.z, r0.z) - p.z;
      acc = fma(p.t - y[i - 1].t, sqrt(fma(ex, ex, fma(ey, ey, ez * ez))), acc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) sums[q] = acc;
}

}  // namespace

template <int P, int STORE>
cudaError_t launch_sl(const SLParams &sp, const double *seeds, int64_t n, SLSample *o, int32_t *count,
                      int32_t *status, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_streamlines<P, STORE>, 128, 0)) != cudaSuccess)
    return e;
  const int64_t fit = (int64_t)sms * (per_sm > 0 ? per_sm : 1);   // resident CTAs of 4 warps
  int64_t lanes = (n + 4 * fit - 1) / (4 * fit);                      // lines per warp, 1..32
  lanes = lanes < 1 ? 1 : (lanes > 32 ? 32 : lanes);
  const int64_t need = (n + 4 * lanes - 1) / (4 * lanes);
  SLParams spl = sp;
  spl.pair_out = lanes < 32;
  if ((e = cudaMemsetAsync(sp.queue, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  k_streamlines<P, STORE><<<(unsigned)(need < fit ? need : fit), 128, 0, s>>>(spl, seeds, n, (int)lanes, o, count,
                                                                             status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (spl.pair_out) k_sl_widen<<<(unsigned)((n + 3) / 4), 128, 0, s>>>(o, count, n, sp.max_samples);
  return cudaGetLastError();
}

cudaError_t launch_streamlines(const SLParams &sp, int degree, int storage, const double *seeds, int64_t n,
                               double *out, int32_t *count, int32_t *status, cudaStream_t s) {
  SLSample *o = reinterpret_cast<SLSample *>(out);
#define LRVOL_SL_CASE(P_, S_) return launch_sl<P_, S_>(sp, seeds, n, o, count, status, s)
  switch (degree * 3 + storage) {
    case 3: LRVOL_SL_CASE(1, LRVOL_STORE_F32); break;
    case 4: LRVOL_SL_CASE(1, LRVOL_STORE_F16); break;
    case 5: LRVOL_SL_CASE(1, LRVOL_STORE_BF16); break;
    case 6: LRVOL_SL_CASE(2, LRVOL_STORE_F32); break;
    case 7: LRVOL_SL_CASE(2, LRVOL_STORE_F16); break;
    case 8: LRVOL_SL_CASE(2, LRVOL_STORE_BF16); break;
    case 9: LRVOL_SL_CASE(3, LRVOL_STORE_F32); break;
    case 10: LRVOL_SL_CASE(3, LRVOL_STORE_F16); break;
    case 11: LRVOL_SL_CASE(3, LRVOL_STORE_BF16); break;
    default: return cudaErrorInvalidValue;
  }
#undef LRVOL_SL_CASE
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Streamline tubes (Sec. 5.3): capsules around the polyline segments,
// visibility by a 64-bit atomic minimum of (t bits, segment index) per pixel,
// then one thread per pixel shades the winner.
// ----------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float dot3r(float x0, float x1, float x2, float y0, float y1, float y2) {
  return __fadd_rn(__fadd_rn(__fmul_rn(x0, y0), __fmul_rn(x1, y1)), __fmul_rn(x2, y2));
}

// Ray/capsule hit in FP32 with the oracle's order of operations; t > 0 only.
__device__ __forceinline__ bool capsule_hit(const Ray &ray, const float *a, const float *b, float r, float &t) {
  const float ba0 = __fsub_rn(b[0], a[0]), ba1 = __fsub_rn(b[1], a[1]), ba2 = __fsub_rn(b[2], a[2]);
  const float oa0 = __fsub_rn(ray.o[0], a[0]), oa1 = __fsub_rn(ray.o[1], a[1]), oa2 = __fsub_rn(ray.o[2], a[2]);
  const float ob0 = __fsub_rn(ray.o[0], b[0]), ob1 = __fsub_rn(ray.o[1], b[1]), ob2 = __fsub_rn(ray.o[2], b[2]);
  const float d0 = ray.d[0], d1 = ray.d[1], d2 = ray.d[2];
  const float baba = dot3r(ba0, ba1, ba2, ba0, ba1, ba2), bard = dot3r(ba0, ba1, ba2, d0, d1, d2);
  const float baoa = dot3r(ba0, ba1, ba2, oa0, oa1, oa2), rdoa = dot3r(d0, d1, d2, oa0, oa1, oa2);
  const float oaoa = dot3r(oa0, oa1, oa2, oa0, oa1, oa2), rr = __fmul_rn(r, r);
  const float A = __fsub_rn(baba, __fmul_rn(bard, bard));
  if (A > 0.f) {
    const float B = __fsub_rn(__fmul_rn(baba, rdoa), __fmul_rn(baoa, bard));
    const float C = __fsub_rn(__fsub_rn(__fmul_rn(baba, oaoa), __fmul_rn(baoa, baoa)), __fmul_rn(rr, baba));
    const float H = __fsub_rn(__fmul_rn(B, B), __fmul_rn(A, C));
    if (H >= 0.f) {
      const float tb = __fdiv_rn(__fsub_rn(-B, __fsqrt_rn(H)), A);
      const float y = __fadd_rn(baoa, __fmul_rn(tb, bard));
      if (y > 0.f && y < baba) {
        if (tb > 0.f) {
          t = tb;
          return true;
        }
        return false;
      }
    }
  }
  float best = __int_as_float(0x7f800000);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float c0 = k == 0 ? oa0 : ob0, c1 = k == 0 ? oa1 : ob1, c2 = k == 0 ? oa2 : ob2;
    const float bb = dot3r(d0, d1, d2, c0, c1, c2), cc = __fsub_rn(dot3r(c0, c1, c2, c0, c1, c2), rr);
    const float h = __fsub_rn(__fmul_rn(bb, bb), cc);
    if (h > 0.f) {
      const float tc = __fsub_rn(-bb, __fsqrt_rn(h));
      if (tc > 0.f && tc < best) best = tc;
    }
  }
  if (best < __int_as_float(0x7f800000)) {
    t = best;
    return true;
  }
  return false;
}

__device__ __forceinline__ bool tube_segment(const TubeParams &tp, int64_t s, float *a, float *b) {
  const int per = tp.max_samples - 1;
  const int64_t j = s / per;
  const int k = (int)(s % per);
  if (k >= tp.count[j] - 1) return false;
  const double *p = tp.samples + (j * tp.max_samples + k) * 4;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a[c] = __double2float_rn(p[c]);
    b[c] = __double2float_rn(p[4 + c]);
  }
  return true;
}

__global__ void k_vis_init(unsigned long long *__restrict__ vis, int64_t n) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) vis[q] = ~0ull;
}

__device__ __forceinline__ void tube_group(const TubeParams &tp, int64_t line, int k0, int nseg, int split, int part,
                                           int lane);

// One warp per line (times `split`) walks the line's segments in groups of
// 32: lane l bounds segment l of the group on the screen, then the warp walks
// the group's (segment, pixel) pairs 32 at a time, as the trimming raster
// does.  `split` warps share a line, each taking a contiguous part of every
// group's pairs, when few long segments could cover much of the image.
__global__ void __launch_bounds__(128) k_tube_raster(const __grid_constant__ TubeParams tp, int split) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int64_t line = wid / split;
  const int part = (int)(wid - line * split);
  if (line >= tp.n_lines) return;                      // whole warp
  const int nseg = tp.count[line] - 1;
  for (int k0 = 0; k0 < nseg; k0 += 32) tube_group(tp, line, k0, nseg, split, part, lane);
}

// One group of 32 segment slots of a line (see k_tube_raster).
__device__ __forceinline__ void tube_group(const TubeParams &tp, int64_t line, int k0, int nseg, int split, int part,
                                           int lane) {
  const unsigned full_mask = 0xffffffffu;
  const int per = tp.max_samples - 1;                  // segment slots per line
  const RayConsts &K = tp.ray;
  float a[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f};
  int i0 = 0, j0 = 0, bw = 1, cnt = 0;
  if (k0 + lane < nseg && tube_segment(tp, line * per + k0 + lane, a, b)) {
    // conservative pixel box of the capsule's bounding box
    float amin = __int_as_float(0x7f800000), amax = -amin, bmin = amin, bmax = -amin;
    bool full = false;
    int behind = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float cx = ((q & 1) ? fmaxf(a[0], b[0]) + tp.radius : fminf(a[0], b[0]) - tp.radius) - K.E[0];
      const float cy = ((q & 2) ? fmaxf(a[1], b[1]) + tp.radius : fminf(a[1], b[1]) - tp.radius) - K.E[1];
      const float cz = ((q & 4) ? fmaxf(a[2], b[2]) + tp.radius : fminf(a[2], b[2]) - tp.radius) - K.E[2];
      const float r = cx * K.R[0] + cy * K.R[1] + cz * K.R[2];
      const float u = cx * K.U[0] + cy * K.U[1] + cz * K.U[2];
      float x = r, y = u;
      if (K.persp) {
        const float z = cx * K.F[0] + cy * K.F[1] + cz * K.F[2];
        if (!(z > 1e-6f)) {
          full = true;
          ++behind;
          continue;
        }
        x = r / z;
        y = u / z;
      }
      amin = fminf(amin, x);
      amax = fmaxf(amax, x);
      bmin = fminf(bmin, y);
      bmax = fmaxf(bmax, y);
    }
    int i1 = tp.width - 1, j1 = tp.height - 1;
    if (behind < 8 && (full || pixel_box(K, tp.width, tp.height, amin, amax, bmin, bmax, i0, i1, j0, j1))) {
      if (full) {
        i0 = 0;
        j0 = 0;
        i1 = tp.width - 1;
        j1 = tp.height - 1;
      }
      bw = i1 - i0 + 1;
      cnt = bw * (j1 - j0 + 1);   // <= 32768^2 < 2^31
    }
  }
  long long inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(full_mask, inc, o);
    if (lane >= o) inc += y;
  }
  const long long total = __shfl_sync(full_mask, inc, 31), exc = inc - cnt;
  const long long chunk = (((total + split - 1) / split) + 31) & ~31ll;
  const long long w0 = (long long)part * chunk, w1 = w0 + chunk < total ? w0 + chunk : total;
  for (long long base = w0; base < w1; base += 32) {
    const long long w = base + lane;
    int q = 0;   // the last lane whose pairs start at or before w (its count is then > 0)
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const long long e = __shfl_sync(full_mask, exc, q + step);
      if (e <= w) q += step;
    }
    const long long eq = __shfl_sync(full_mask, exc, q);
    const int qi0 = __shfl_sync(full_mask, i0, q), qj0 = __shfl_sync(full_mask, j0, q);
    const int qbw = __shfl_sync(full_mask, bw, q);
    float qa[3], qb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      qa[c] = __shfl_sync(full_mask, a[c], q);
      qb[c] = __shfl_sync(full_mask, b[c], q);
    }
    if (w >= w1) continue;
    const unsigned pix = (unsigned)(w - eq);
    const int i = qi0 + (int)(pix % (unsigned)qbw), j = qj0 + (int)(pix / (unsigned)qbw);
    Ray ray;
    make_ray(K, i, j, ray);
    float t;
    if (!capsule_hit(ray, qa, qb, tp.radius, t)) continue;
    const uint32_t sid = (uint32_t)(line * per + k0 + q);
    const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | (unsigned long long)sid;
    atomicMin(tp.vis + (int64_t)j * tp.width + i, key);
  }
}

template <int P, int STORE>
__global__ void __launch_bounds__(128) k_tube_resolve(const __grid_constant__ TubeParams tp) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)tp.width * tp.height) return;
  float4 *o = reinterpret_cast<float4 *>(tp.out) + q;
  const unsigned long long key = tp.vis[q];
  if (key == ~0ull) {
    *o = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int64_t s = (int64_t)(key & 0xffffffffull);
  const float t = __uint_as_float((unsigned)(key >> 32));
  float a[3], b[3];
  tube_segment(tp, s, a, b);
  Ray ray;
  make_ray(tp.ray, (int)(q % tp.width), (int)(q / tp.width), ray);
  float p[3], ba[3], pa[3], qa[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p[c] = __fadd_rn(ray.o[c], __fmul_rn(t, ray.d[c]));
    ba[c] = __fsub_rn(b[c], a[c]);
    pa[c] = __fsub_rn(p[c], a[c]);
  }
  const float baba = dot3r(ba[0], ba[1], ba[2], ba[0], ba[1], ba[2]);
  float hcl = baba > 0.f ? __fdiv_rn(dot3r(pa[0], pa[1], pa[2], ba[0], ba[1], ba[2]), baba) : 0.f;
  hcl = fminf(fmaxf(hcl, 0.f), 1.f);
#pragma unroll
  for (int c = 0; c < 3; ++c) qa[c] = __fadd_rn(a[c], __fmul_rn(hcl, ba[c]));
  SLField<P, STORE> F;
  F.cur = kNone;
  float v0 = 0.f, v1 = 0.f, v2 = 0.f;
  F.eval(tp.field, qa[0], qa[1], qa[2], v0, v1, v2);
  const float speed = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
  const float x = fminf(fmaxf(fmaf(speed, tp.tf_scale, tp.tf_bias), 0.f), 255.f);
  const int k = min((int)x, 254);
  const float fr = x - (float)k;
  const float4 e0 = tp.cmap[k], e1 = tp.cmap[k + 1];
  const float n0 = p[0] - qa[0], n1 = p[1] - qa[1], n2 = p[2] - qa[2];
  const float nn = fmaf(n0, n0, fmaf(n1, n1, n2 * n2));
  float I = nn > 0.f ? fabsf(fmaf(n0, ray.d[0], fmaf(n1, ray.d[1], n2 * ray.d[2]))) * rsqrtf(nn) : 1.f;
  I = fmaxf(I, 0.4f);
  *o = make_float4(I * fmaf(fr, e1.x - e0.x, e0.x), I * fmaf(fr, e1.y - e0.y, e0.y), I * fmaf(fr, e1.z - e0.z, e0.z),
                   1.f);
}

}  // namespace

cudaError_t launch_tubes(const TubeParams &tp, int degree, int storage, cudaStream_t s) {
  const int64_t npix = (int64_t)tp.width * tp.height;
  const int64_t nseg = tp.n_lines * (int64_t)(tp.max_samples - 1);
  k_vis_init<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(tp.vis, npix);
  if (nseg > 0) {
    // warps per line: about 512 pairs per warp and group when the lines'
    // first groups cover the image twice, 1 for many lines, at most 256
    const int64_t lines = tp.n_lines;
    int64_t split = (2 * npix + lines * 512 - 1) / (lines * 512);
    split = split < 1 ? 1 : (split > 256 ? 256 : split);
    const int64_t warps = lines * split;
    k_tube_raster<<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(tp, (int)split);
  }
  const unsigned blocks = (unsigned)((npix + 127) / 128);
#define LRVOL_TUBE_CASE(P_, S_) k_tube_resolve<P_, S_><<<blocks, 128, 0, s>>>(tp)
  switch (degree * 3 + storage) {
    case 3: LRVOL_TUBE_CASE(1, LRVOL_STORE_F32); break;
    case 4: LRVOL_TUBE_CASE(1, LRVOL_STORE_F16); break;
    case 5: LRVOL_TUBE_CASE(1, LRVOL_STORE_BF16); break;
    case 6: LRVOL_TUBE_CASE(2, LRVOL_STORE_F32); break;
    case 7: LRVOL_TUBE_CASE(2, LRVOL_STORE_F16); break;
    case 8: LRVOL_TUBE_CASE(2, LRVOL_STORE_BF16); break;
    case 9: LRVOL_TUBE_CASE(3, LRVOL_STORE_F32); break;
    case 10: LRVOL_TUBE_CASE(3, LRVOL_STORE_F16); break;
    case 11: LRVOL_TUBE_CASE(3, LRVOL_STORE_BF16); break;
    default: return cudaErrorInvalidValue;
  }
#undef LRVOL_TUBE_CASE
  return cudaGetLastError();
}

cudaError_t launch_streamline_error(const double *ref, const int32_t *rc, int rmax, const double *app,
                                    const int32_t *ac, int amax, int64_t n, double *sums, cudaStream_t s) {
  k_streamline_error<<<(unsigned)((n + 3) / 4), 128, 0, s>>>(reinterpret_cast<const SLSample *>(ref), rc, rmax,
                                                             reinterpret_cast<const SLSample *>(app), ac, amax, n,
                                                             sums);
  return cudaGetLastError();
}

}  // namespace lrvol
