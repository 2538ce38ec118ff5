// liblrvol kernels for sm_103a.
//
//   k_to_bezier    Sec. 3.2.3 change of basis, FP64: per element, the Bernstein
//                  coefficients of every incident B-spline's univariate factors
//                  over the element, by blossoming, accumulated with gamma*c.
//   k_elem_records element boxes -> FP32 records (rounded-up corners, Eq. 4 step).
//   k_lookup       Alg. 1 element look-up through the k-d forest.
//   k_eval         look-up + Bezier block evaluation at points.
//   k_render       Sec. 4: per-pixel ray casting with element reuse, Eq. 4
//                  steps, transfer function and Alg. 2 compositing.
#include <cuda_runtime.h>

#include <cstdint>

#include "lrvol_internal.h"

namespace lrvol {
namespace {

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t code) { atomicCAS(status, 0u, code); }

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
  for (int j = 0; j <= p; ++j) {
    double D[kMaxDeg + 1];
    D[0] = 1.0;
    for (int q = 1; q <= p; ++q) D[q] = 0.0;
    for (int r = 1; r <= p; ++r) {
      const double t = (r <= p - j) ? a : b;
      const int khi = m < r ? m : r;
      const int klo = (m - p + r) > 0 ? (m - p + r) : 0;
      for (int k = khi; k >= klo; --k) {
        const double alpha = (t - xi[k]) / (xi[k + p + 1 - r] - xi[k]);
        const double prev = k > 0 ? D[k - 1] : 0.0;
        D[k] = (1.0 - alpha) * prev + alpha * D[k];
      }
    }
    beta[j] = D[m];
  }
}

constexpr int kBezWarps = 4;
constexpr int kChunk = 32;

// One warp per element; lane l owns coefficients q = l, l+32, ... of the
// (p0+1)(p1+1)(p2+1) block, for every component.
__global__ void __launch_bounds__(32 * kBezWarps) k_to_bezier(
    const double *__restrict__ box, const double *__restrict__ knots, const double *__restrict__ coef,
    const double *__restrict__ weight, const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc_idx,
    int p0, int p1, int p2, int nc, int kw, int64_t n_elem, double *__restrict__ out64, float *__restrict__ out32,
    int comp_stride, int elem_stride) {
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
      for (int c = 0; c < nc; ++c) {
        out64[(e * nc + c) * nb + q] = acc[r][c];
        out32[e * elem_stride + c * comp_stride + q] = (float)acc[r][c];
      }
  }
}

__global__ void k_elem_records(const double *__restrict__ box, int64_t n_elem, int d, ElemRec *__restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  const double *b = box + 6 * e;
  float lo[3], hi[3], dlo[3], iw[3];
  double m = b[3] - b[0];
  if (b[4] - b[1] < m) m = b[4] - b[1];
  if (b[5] - b[2] < m) m = b[5] - b[2];
  for (int a = 0; a < 3; ++a) {
    lo[a] = __double2float_ru(b[a]);
    hi[a] = b[3 + a] == 1.0 ? __int_as_float(0x7f800000) : __double2float_ru(b[3 + a]);
    dlo[a] = (float)((double)lo[a] - b[a]);
    iw[a] = (float)(1.0 / (b[3 + a] - b[a]));
  }
  ElemRec r;
  r.a = make_float4(lo[0], lo[1], lo[2], __double2float_rn(ldexp(m, -d)));
  r.b = make_float4(hi[0], hi[1], hi[2], 0.f);
  r.c = make_float4(dlo[0], dlo[1], dlo[2], 0.f);
  r.d = make_float4(iw[0], iw[1], iw[2], 0.f);
  out[e] = r;
}

// ----------------------------------------------------------------------------
// look-up (Alg. 1)
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint32_t forest_lookup(const ForestView &f, float x, float y, float z, uint32_t *status) {
  const int bx = min((int)(x * f.fbx), f.bx - 1);
  const int by = min((int)(y * f.fby), f.by - 1);
  const int bz = min((int)(z * f.fbz), f.bz - 1);
  uint32_t w = __ldg(f.head + ((int64_t)bz * f.by + by) * f.bx + bx);
  for (int depth = 0; !(w & kLeaf); ++depth) {
    if ((int64_t)w >= f.n_nodes || depth >= kMaxDepth) {
      set_status(status, kStatusBounds);
      return kNone;
    }
    const uint4 n = __ldg(f.nodes + w);
    const float pa = n.y == 0 ? x : (n.y == 1 ? y : z);
    w = pa < __uint_as_float(n.x) ? n.z : n.w;
  }
  return w & ~kLeaf;
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

// ----------------------------------------------------------------------------
// Bezier evaluation
// ----------------------------------------------------------------------------

template <int P>
__device__ __forceinline__ void bernstein(float u, float *b) {
  const float v = 1.f - u;
  if constexpr (P == 1) {
    b[0] = v;
    b[1] = u;
  } else if constexpr (P == 2) {
    b[0] = v * v;
    b[1] = 2.f * u * v;
    b[2] = u * u;
  } else {
    const float u2 = u * u, v2 = v * v;
    b[0] = v2 * v;
    b[1] = 3.f * u * v2;
    b[2] = 3.f * u2 * v;
    b[3] = u2 * u;
  }
}

// sum_{k,j,i} c[k][j][i] bx[i] by[j] bz[k], x fastest
template <int P>
__device__ __forceinline__ float contract(const float *c, const float *bx, const float *by, const float *bz) {
  constexpr int N = P + 1;
  float f = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i) s = fmaf(c[(k * N + j) * N + i], bx[i], s);
      t = fmaf(s, by[j], t);
    }
    f = fmaf(t, bz[k], f);
  }
  return f;
}

__device__ __forceinline__ float local_u(float p, float lo, float dlo, float iw) { return ((p - lo) + dlo) * iw; }

// Generic-degree evaluation for the point kernel (any p0,p1,p2 <= 4).
__device__ float eval_generic(const float *c, const int *deg, float ux, float uy, float uz) {
  float b[3][kMaxDeg + 1];
  const float u[3] = {ux, uy, uz};
  for (int a = 0; a < 3; ++a) {
    const int p = deg[a];
    const float v = 1.f - u[a];
    // Bernstein values by the triangular recurrence B^r_j = v B^{r-1}_j + u B^{r-1}_{j-1}
    b[a][0] = 1.f;
    for (int r = 1; r <= p; ++r) {
      b[a][r] = u[a] * b[a][r - 1];
      for (int j = r - 1; j >= 1; --j) b[a][j] = v * b[a][j] + u[a] * b[a][j - 1];
      b[a][0] = v * b[a][0];
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

__global__ void k_eval(ForestView f, const ElemRec *__restrict__ elem, int64_t n_elem, const float *__restrict__ bez,
                       int elem_stride, int comp_stride, int p0, int p1, int p2, int nc,
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
  for (int c = 0; c < nc; ++c) {
    const float *cb = bez + (int64_t)e * elem_stride + c * comp_stride;
    float cl[(kMaxDeg + 1) * (kMaxDeg + 1) * (kMaxDeg + 1)];
    const int nb = (p0 + 1) * (p1 + 1) * (p2 + 1);
    for (int t = 0; t < nb; ++t) cl[t] = __ldg(cb + t);
    out[q * nc + c] = eval_generic(cl, deg, ux, uy, uz);
  }
}

// ----------------------------------------------------------------------------
// render (Sec. 4, Alg. 2, Eq. 4)
// ----------------------------------------------------------------------------

// FIELD: 0 = one component (scalar or chosen), 1 = magnitude of 3 components
template <int P, int FIELD>
__global__ void __launch_bounds__(128) k_render(const __grid_constant__ RenderParams prm) {
  constexpr int N = P + 1;
  constexpr int NB = N * N * N;
  constexpr int CS = (NB + 3) & ~3;
  constexpr int NCE = FIELD == 1 ? 3 : 1;
  __shared__ float4 tf[256];
  for (int q = threadIdx.x; q < 256; q += blockDim.x) tf[q] = prm.tf[q];
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
  const int j = prm.row_begin + blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
  const bool active = i < prm.width && j < prm.row_end;
  unsigned long long nsamp = 0, nlook = 0, nhit = 0;
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);

  if (active) {
    const RayConsts &K = prm.ray;
    const float a = __fmaf_rn(__fadd_rn((float)i, 0.5f), K.sxs, K.sxo);
    const float b = __fmaf_rn(__fadd_rn((float)j, 0.5f), K.sys, K.syo);
    float o[3], d[3];
    if (K.persp) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        d[c] = __fmaf_rn(a, K.R[c], __fmaf_rn(b, K.U[c], K.F[c]));
        o[c] = K.E[c];
      }
      const float n = __fsqrt_rn(__fmaf_rn(d[0], d[0], __fmaf_rn(d[1], d[1], __fmul_rn(d[2], d[2]))));
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] = __fdiv_rn(d[c], n);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c] = __fmaf_rn(a, K.R[c], __fmaf_rn(b, K.U[c], K.E[c]));
        d[c] = K.F[c];
      }
    }
    float tin = 0.f, tout = __int_as_float(0x7f800000);
    bool hit = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (d[c] == 0.f) {
        if (o[c] < 0.f || o[c] > 1.f) hit = false;
      } else {
        const float inv = __fdiv_rn(1.f, d[c]);
        const float ta = __fmul_rn(__fsub_rn(0.f, o[c]), inv);
        const float tb = __fmul_rn(__fsub_rn(1.f, o[c]), inv);
        tin = fmaxf(tin, fminf(ta, tb));
        tout = fminf(tout, fmaxf(ta, tb));
      }
    }
    hit = hit && tin < tout;
    if (hit) {
      nhit = 1;
      float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
      uint32_t cur = kNone;
      float4 ra = make_float4(0, 0, 0, 0), rb = ra, rc = ra, rd = ra;
      float cf[NCE][CS];
      float t = tin;
      int k = 0;
      while (t < tout) {
        const float px = fminf(fmaxf(__fmaf_rn(t, d[0], o[0]), 0.f), 1.f);
        const float py = fminf(fmaxf(__fmaf_rn(t, d[1], o[1]), 0.f), 1.f);
        const float pz = fminf(fmaxf(__fmaf_rn(t, d[2], o[2]), 0.f), 1.f);
        const bool inside = cur != kNone && px >= ra.x && py >= ra.y && pz >= ra.z && px < rb.x && py < rb.y &&
                            pz < rb.z;
        if (!inside) {
          cur = forest_lookup(prm.forest, px, py, pz, prm.status);
          if (cur == kNone || (int64_t)cur >= prm.n_elem) {
            set_status(prm.status, kStatusBounds);
            break;
          }
          ++nlook;
          const ElemRec *er = prm.elem + cur;
          ra = __ldg(&er->a);
          rb = __ldg(&er->b);
          rc = __ldg(&er->c);
          rd = __ldg(&er->d);
          const float4 *cb = reinterpret_cast<const float4 *>(prm.bez + (int64_t)cur * prm.elem_stride +
                                                              (FIELD == 1 ? 0 : prm.comp * prm.comp_stride));
#pragma unroll
          for (int c = 0; c < NCE; ++c)
#pragma unroll
            for (int q = 0; q < CS / 4; ++q) {
              const float4 v = __ldg(cb + c * (prm.comp_stride / 4) + q);
              cf[c][4 * q] = v.x;
              cf[c][4 * q + 1] = v.y;
              cf[c][4 * q + 2] = v.z;
              cf[c][4 * q + 3] = v.w;
            }
        }
        float tn = prm.mode == LRVOL_STEP_HEURISTIC ? __fadd_rn(t, ra.w) : __fmaf_rn((float)(k + 1), prm.h, tin);
        if (!(tn > t)) tn = nextafterf(t, __int_as_float(0x7f800000));
        const float seg = __fsub_rn(fminf(tn, tout), t);
        float bx[N], by[N], bz[N];
        bernstein<P>(local_u(px, ra.x, rc.x, rd.x), bx);
        bernstein<P>(local_u(py, ra.y, rc.y, rd.y), by);
        bernstein<P>(local_u(pz, ra.z, rc.z, rd.z), bz);
        float v;
        if constexpr (FIELD == 1) {
          const float v0 = contract<P>(cf[0], bx, by, bz);
          const float v1 = contract<P>(cf[NCE > 1 ? 1 : 0], bx, by, bz);
          const float v2 = contract<P>(cf[NCE > 2 ? 2 : 0], bx, by, bz);
          v = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
        } else {
          v = contract<P>(cf[0], bx, by, bz);
        }
        // transfer function
        const float x = fminf(fmaxf((v - prm.tf_off) * prm.tf_scale, 0.f), 255.f);
        const int i0 = min((int)x, 254);
        const float fr = x - (float)i0;
        const float4 e0 = tf[i0], e1 = tf[i0 + 1];
        const float sr = fmaf(fr, e1.x - e0.x, e0.x);
        const float sg = fmaf(fr, e1.y - e0.y, e0.y);
        const float sb = fmaf(fr, e1.z - e0.z, e0.z);
        const float sa = fmaf(fr, e1.w - e0.w, e0.w);
        // Alg. 2
        const float T = exp2f(__log2f(fmaxf(1.f - sa, 0.f)) * (seg * prm.inv_xi));
        const float wgt = (1.f - T) * (1.f - A);
        C0 = fmaf(wgt, sr, C0);
        C1 = fmaf(wgt, sg, C1);
        C2 = fmaf(wgt, sb, C2);
        A += wgt;
        ++nsamp;
        ++k;
        t = tn;
        if (A >= prm.alpha_stop) break;
        if (k >= kMaxSamplesPerRay) {
          set_status(prm.status, kStatusTimeout);
          break;
        }
      }
      out = make_float4(C0, C1, C2, A);
    }
    reinterpret_cast<float4 *>(prm.out)[(int64_t)j * prm.width + i] = out;
  }
  // per-warp counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nsamp += __shfl_down_sync(0xffffffffu, nsamp, o);
    nlook += __shfl_down_sync(0xffffffffu, nlook, o);
    nhit += __shfl_down_sync(0xffffffffu, nhit, o);
  }
  if (lane == 0) {
    atomicAdd(prm.counters + kCntSamples, nsamp);
    atomicAdd(prm.counters + kCntLookups, nlook);
    atomicAdd(prm.counters + kCntRays, nhit);
  }
}

}  // namespace

cudaError_t launch_to_bezier(const lrvol_s *v, cudaStream_t s) {
  const int64_t blocks = (v->n_elem + kBezWarps - 1) / kBezWarps;
  k_to_bezier<<<(unsigned)blocks, 32 * kBezWarps, 0, s>>>(v->d_box, v->d_knots, v->d_coef, v->d_weight, v->d_inc_ptr,
                                                         v->d_inc_idx, v->p[0], v->p[1], v->p[2], v->nc, v->kw,
                                                         v->n_elem, v->d_bez64, v->d_bez32, v->comp_stride,
                                                         v->elem_stride);
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
  k_eval<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(forest_view(v), v->d_elem, v->n_elem, v->d_bez32,
                                                    v->elem_stride, v->comp_stride, v->p[0], v->p[1], v->p[2],
                                                    v->nc, pts, n, out, v->d_status);
  return cudaGetLastError();
}

cudaError_t launch_render(const RenderParams &prm, int degree, int field, cudaStream_t s) {
  dim3 block(128);
  dim3 grid((unsigned)((prm.width + 15) / 16), (unsigned)((prm.row_end - prm.row_begin + 7) / 8));
  const bool mag = field == LRVOL_FIELD_MAGNITUDE;
  switch (degree * 2 + (mag ? 1 : 0)) {
    case 2: k_render<1, 0><<<grid, block, 0, s>>>(prm); break;
    case 3: k_render<1, 1><<<grid, block, 0, s>>>(prm); break;
    case 4: k_render<2, 0><<<grid, block, 0, s>>>(prm); break;
    case 5: k_render<2, 1><<<grid, block, 0, s>>>(prm); break;
    case 6: k_render<3, 0><<<grid, block, 0, s>>>(prm); break;
    case 7: k_render<3, 1><<<grid, block, 0, s>>>(prm); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lrvol
