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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

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

__device__ __forceinline__ double binomial(int n, int k) {
  double b = 1.0;
  for (int i = 1; i <= k; ++i) b = b * (double)(n - k + i) / (double)i;
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
                                                        int ebytes, unsigned char *__restrict__ outc, int ecbytes) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * kBezWarps + w;
  if (e >= n_elem) return;
  const int n0 = p0 + 1, n1 = p1 + 1, nb = n0 * n1 * (p2 + 1);
  const double *be = b64 + e * nc * nb;
  double o[3] = {0.0, 0.0, 0.0}, sc[3] = {1.0, 1.0, 1.0};
  if (storage != LRVOL_STORE_F32) {
    for (int c = 0; c < nc; ++c) {
      double mn = __longlong_as_double(0x7ff0000000000000ll), mx = -mn;
      for (int q = lane; q < nb; q += 32) {
        mn = fmin(mn, be[c * nb + q]);
        mx = fmax(mx, be[c * nb + q]);
      }
      for (int off = 16; off > 0; off >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
      }
      o[c] = 0.5 * (mx + mn);
      sc[c] = 0.5 * (mx - mn);
      if (!(sc[c] > 0.0)) sc[c] = 1.0;
    }
    if (lane < 8) {
      const float hv = lane < 3 ? (float)o[lane] : (lane < 6 ? (float)sc[lane - 3] : 0.f);
      reinterpret_cast<float *>(out + e * ebytes)[lane] = hv;
      if (outc) reinterpret_cast<float *>(outc + e * ecbytes)[lane] = hv;
    }
  }
  for (int q = lane; q < nb; q += 32) {
    const int ix = q % n0, iy = (q / n0) % n1, iz = q / (n0 * n1);
    const double binom = binomial(p0, ix) * binomial(p1, iy) * binomial(p2, iz);
    for (int c = 0; c < nc; ++c) {
      const double x = binom * (be[c * nb + q] - o[c]) / sc[c];
      store_slot(out + e * ebytes, storage, render_slot(nc, n0, nb, iz * n1 + iy, ix, c), x);
      if (outc) store_slot(outc + e * ecbytes, storage, c * roundup8(nb) + q, x);
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
// Bezier evaluation.  Render blocks hold binomially scaled coefficients, so a
// block is evaluated as sum c'_ijk m_i(u) m_j(v) m_k(w) with monomials
// m_i(u) = u^i (1-u)^(p-i).
// ----------------------------------------------------------------------------

template <int P>
__device__ __forceinline__ void monomials(float u, float *m) {
  const float v = 1.f - u;
  if constexpr (P == 1) {
    m[0] = v;
    m[1] = u;
  } else if constexpr (P == 2) {
    m[0] = v * v;
    m[1] = u * v;
    m[2] = u * u;
  } else {
    const float u2 = u * u, v2 = v * v;
    m[0] = v2 * v;
    m[1] = u * v2;
    m[2] = u2 * v;
    m[3] = u2 * u;
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

// ----------------------------------------------------------------------------
// render (Sec. 4, Alg. 2, Eq. 4)
// ----------------------------------------------------------------------------

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct Ray {
  float o[3], d[3], tin, tout;
};

// FP32 ray of pixel (i, j) and its interval in the unit cube (order of
// operations as stated in lrvol.h).  Returns false on a miss.
__device__ __forceinline__ bool make_ray(const RayConsts &K, int i, int j, Ray &r) {
  const float a = __fmaf_rn(__fadd_rn((float)i, 0.5f), K.sxs, K.sxo);
  const float b = __fmaf_rn(__fadd_rn((float)j, 0.5f), K.sys, K.syo);
  if (K.persp) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r.d[c] = __fmaf_rn(a, K.R[c], __fmaf_rn(b, K.U[c], K.F[c]));
      r.o[c] = K.E[c];
    }
    const float n = __fsqrt_rn(__fmaf_rn(r.d[0], r.d[0], __fmaf_rn(r.d[1], r.d[1], __fmul_rn(r.d[2], r.d[2]))));
#pragma unroll
    for (int c = 0; c < 3; ++c) r.d[c] = __fdiv_rn(r.d[c], n);
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r.o[c] = __fmaf_rn(a, K.R[c], __fmaf_rn(b, K.U[c], K.E[c]));
      r.d[c] = K.F[c];
    }
  }
  float tin = 0.f, tout = __int_as_float(0x7f800000);
  bool hit = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (r.d[c] == 0.f) {
      if (r.o[c] < 0.f || r.o[c] > 1.f) hit = false;
    } else {
      const float inv = __fdiv_rn(1.f, r.d[c]);
      const float ta = __fmul_rn(__fsub_rn(0.f, r.o[c]), inv);
      const float tb = __fmul_rn(__fsub_rn(1.f, r.o[c]), inv);
      tin = fmaxf(tin, fminf(ta, tb));
      tout = fminf(tout, fmaxf(ta, tb));
    }
  }
  r.tin = tin;
  r.tout = tout;
  return hit && tin < tout;
}

// Transfer function lookup and one Alg. 2 update in transmittance form
// (Tr = 1 - alpha_dst): w = (1 - T) Tr, C += w C_src, Tr *= T.
__device__ __forceinline__ void composite(const float4 *tfb, const float4 *tfd, float v, float seg,
                                          const RenderParams &prm, float &C0, float &C1, float &C2, float &Tr) {
  const float x = fminf(fmaxf(fmaf(v, prm.tf_scale, prm.tf_bias), 0.f), 255.f);
  const int q = min((int)x, 254);
  const float fr = x - (float)q;
  const float4 e0 = tfb[q], de = tfd[q];
  const float sa = fmaf(fr, de.w, e0.w);
  const float T = ex2_approx(lg2_approx(fmaxf(1.f - sa, 0.f)) * (seg * prm.inv_xi));
  const float w = fmaf(-Tr, T, Tr);
  C0 = fmaf(w, fmaf(fr, de.x, e0.x), C0);
  C1 = fmaf(w, fmaf(fr, de.y, e0.y), C1);
  C2 = fmaf(w, fmaf(fr, de.z, e0.z), C2);
  Tr *= T;
}

// ---- packed two-lane FP32 (fma.rn.f32x2 and friends; lane "lo" first) ----
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(f2 a, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// 256-bit read-only load (32-byte aligned address)
__device__ __forceinline__ void ld256(const void *p, f2 &a, f2 &b, f2 &c, f2 &d) {
  asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}
__device__ __forceinline__ float4 f2x2_to_float4(f2 a, f2 b) {
  float4 r;
  f2_unpack(a, r.x, r.y);
  f2_unpack(b, r.z, r.w);
  return r;
}

// Element record: two 256-bit loads.
__device__ __forceinline__ void load_record(const ElemRec *er, float4 &ra, float4 &rb, float4 &rc, float4 &rd) {
  f2 w0, w1, w2, w3, w4, w5, w6, w7;
  ld256(er, w0, w1, w2, w3);
  ld256(reinterpret_cast<const char *>(er) + 32, w4, w5, w6, w7);
  ra = f2x2_to_float4(w0, w1);
  rb = f2x2_to_float4(w2, w3);
  rc = f2x2_to_float4(w4, w5);
  rd = f2x2_to_float4(w6, w7);
}

// 16-bit storage: two values of one 32-bit word -> FP32 pair (lo = low half).
template <int STORE>
__device__ __forceinline__ float h_to_f(unsigned h) {
  if constexpr (STORE == LRVOL_STORE_F16) return __half2float(__ushort_as_half((unsigned short)h));
  return __uint_as_float(h << 16);
}
template <int STORE>
__device__ __forceinline__ f2 word_to_f2(unsigned w) {
  if constexpr (STORE == LRVOL_STORE_BF16) {
    return ((f2)(w & 0xffff0000u) << 32) | (f2)(w << 16);
  } else {
    return f2_pack(h_to_f<STORE>(w & 0xffffu), h_to_f<STORE>(w >> 16));
  }
}

// One element's block in registers and its evaluation at monomials bx, by, bz.
//   FIELD 0: scalar volume; 1: |v| of a 3-vector; 2: one component of a
//   3-vector, read from the plain per-component copy.
//   STORE: LRVOL_STORE_F32, or F16/BF16 values converted to FP32 when the
//   element is entered, with the value of component c = o_c + s_c * contraction.
template <int P, int FIELD, int STORE>
struct Block {
  static constexpr int N = P + 1;
  static constexpr int NB = N * N * N;
  static constexpr bool ROWPAIR = FIELD == 0 && P == 3;   // scalar tricubic: packed row pairs
  static constexpr bool SCALAR_GENERIC = FIELD == 0 && P != 3;
  static constexpr bool PAIRS = FIELD == 1;                // components 0 and 1 packed
  static constexpr bool COMP2 = FIELD == 1 || FIELD == 2;  // one component as plain floats
  static constexpr bool F32 = STORE == LRVOL_STORE_F32;
  static constexpr int SGF = ((N * N + 1) / 2) * 2 * N;    // scalar generic: slots used (<= stride)
  static constexpr int PAIRF = (2 * NB + 7) & ~7;          // slots of the component pair block
  static constexpr int C2F = (NB + 7) & ~7;                // slots of one plain component

  f2 rp[ROWPAIR ? 8 : 1][4];                 // row pairs (2m, 2m+1), value i
  float sg[SCALAR_GENERIC ? ((SGF + 7) & ~7) : 1];
  f2 cp[PAIRS ? PAIRF / 2 : 1];              // (c0, c1) per q
  float c2[COMP2 ? C2F : 1];
  float oa, sa, ob, sb, oc, sc;              // affine map of 16-bit storage (component a/b/c)

  __device__ __forceinline__ void load(const unsigned char *eb, int comp) {
    if constexpr (F32) {
      const float *fb = reinterpret_cast<const float *>(eb);
      if constexpr (ROWPAIR) {
#pragma unroll
        for (int m = 0; m < 8; ++m) ld256(fb + 8 * m, rp[m][0], rp[m][1], rp[m][2], rp[m][3]);
      }
      if constexpr (SCALAR_GENERIC) {
        const float4 *b4 = reinterpret_cast<const float4 *>(fb);
#pragma unroll
        for (int q = 0; q < (SGF + 3) / 4; ++q) {
          const float4 v = __ldg(b4 + q);
          sg[4 * q] = v.x;
          sg[4 * q + 1] = v.y;
          sg[4 * q + 2] = v.z;
          sg[4 * q + 3] = v.w;
        }
      }
      if constexpr (PAIRS) {
#pragma unroll
        for (int q = 0; q < PAIRF / 8; ++q) ld256(fb + 8 * q, cp[4 * q], cp[4 * q + 1], cp[4 * q + 2], cp[4 * q + 3]);
      }
      if constexpr (COMP2) {
        const float4 *b4 = reinterpret_cast<const float4 *>(FIELD == 1 ? fb + PAIRF : fb + comp * C2F);
#pragma unroll
        for (int q = 0; q < C2F / 4; ++q) {
          const float4 v = __ldg(b4 + q);
          c2[4 * q] = v.x;
          c2[4 * q + 1] = v.y;
          c2[4 * q + 2] = v.z;
          c2[4 * q + 3] = v.w;
        }
      }
    } else {
      const float4 *hdr = reinterpret_cast<const float4 *>(eb);
      const float4 h0 = __ldg(hdr), h1 = __ldg(hdr + 1);   // o0 o1 o2 s0 | s1 s2 - -
      const uint4 *d = reinterpret_cast<const uint4 *>(eb + kHeaderBytes);   // 8 slots per chunk
      if constexpr (ROWPAIR) {
        oa = h0.x;
        sa = h0.w;
#pragma unroll
        for (int m = 0; m < 8; ++m) {   // chunk m holds words 4m+i = (row 2m, row 2m+1) value i
          const uint4 w = __ldg(d + m);
          rp[m][0] = word_to_f2<STORE>(w.x);
          rp[m][1] = word_to_f2<STORE>(w.y);
          rp[m][2] = word_to_f2<STORE>(w.z);
          rp[m][3] = word_to_f2<STORE>(w.w);
        }
      }
      if constexpr (SCALAR_GENERIC) {
        oa = h0.x;
        sa = h0.w;
#pragma unroll
        for (int q = 0; q < (SGF + 7) / 8; ++q) {
          const uint4 w = __ldg(d + q);
          const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            sg[8 * q + 2 * t] = h_to_f<STORE>(ws[t] & 0xffffu);
            sg[8 * q + 2 * t + 1] = h_to_f<STORE>(ws[t] >> 16);
          }
        }
      }
      if constexpr (PAIRS) {
        oa = h0.x;
        ob = h0.y;
        sa = h0.w;
        sb = h1.x;
#pragma unroll
        for (int q = 0; q < PAIRF / 8; ++q) {
          const uint4 w = __ldg(d + q);
          cp[4 * q] = word_to_f2<STORE>(w.x);
          cp[4 * q + 1] = word_to_f2<STORE>(w.y);
          cp[4 * q + 2] = word_to_f2<STORE>(w.z);
          cp[4 * q + 3] = word_to_f2<STORE>(w.w);
        }
      }
      if constexpr (COMP2) {
        if constexpr (FIELD == 1) {
          oc = h0.z;
          sc = h1.y;
        } else {
          oc = comp == 0 ? h0.x : (comp == 1 ? h0.y : h0.z);
          sc = comp == 0 ? h0.w : (comp == 1 ? h1.x : h1.y);
        }
        const uint4 *dc = d + (FIELD == 1 ? PAIRF : comp * C2F) / 8;
#pragma unroll
        for (int q = 0; q < C2F / 8; ++q) {
          const uint4 w = __ldg(dc + q);
          const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            c2[8 * q + 2 * t] = h_to_f<STORE>(ws[t] & 0xffffu);
            c2[8 * q + 2 * t + 1] = h_to_f<STORE>(ws[t] >> 16);
          }
        }
      }
    }
  }

  __device__ __forceinline__ float eval(const float *bx, const float *by, const float *bz) const {
    if constexpr (ROWPAIR) {
      // rows r = k*4 + j; pair m = 2k + (j >> 1) holds (row 2m, row 2m+1)
      const f2 X0 = f2_pack(bx[0], bx[0]), X1 = f2_pack(bx[1], bx[1]);
      const f2 X2 = f2_pack(bx[2], bx[2]), X3 = f2_pack(bx[3], bx[3]);
      const f2 Y01 = f2_pack(by[0], by[1]), Y23 = f2_pack(by[2], by[3]);
      f2 F = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const f2 *a = rp[2 * k], *b = rp[2 * k + 1];
        const f2 S0 = f2_fma(a[3], X3, f2_fma(a[2], X2, f2_fma(a[1], X1, f2_mul(a[0], X0))));
        const f2 S1 = f2_fma(b[3], X3, f2_fma(b[2], X2, f2_fma(b[1], X1, f2_mul(b[0], X0))));
        const f2 T = f2_fma(S1, Y23, f2_mul(S0, Y01));   // (t_k over j even, t_k over j odd)
        const f2 Z = f2_pack(bz[k], bz[k]);
        F = k == 0 ? f2_mul(T, Z) : f2_fma(T, Z, F);
      }
      float lo, hi;
      f2_unpack(F, lo, hi);
      return F32 ? lo + hi : fmaf(sa, lo + hi, oa);
    } else if constexpr (SCALAR_GENERIC) {
      float f = 0.f;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        float t = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int r = k * N + j;
          float sx = 0.f;
#pragma unroll
          for (int i = 0; i < N; ++i) sx = fmaf(sg[(r >> 1) * 2 * N + 2 * i + (r & 1)], bx[i], sx);
          t = fmaf(sx, by[j], t);
        }
        f = fmaf(t, bz[k], f);
      }
      return F32 ? f : fmaf(sa, f, oa);
    } else {
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      if constexpr (PAIRS) {
        f2 X[N], Y[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          X[i] = f2_pack(bx[i], bx[i]);
          Y[i] = f2_pack(by[i], by[i]);
        }
        f2 V = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          f2 T = 0;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const f2 *c = &cp[(k * N + j) * N];
            f2 S = f2_mul(c[0], X[0]);
#pragma unroll
            for (int i = 1; i < N; ++i) S = f2_fma(c[i], X[i], S);
            T = j == 0 ? f2_mul(S, Y[0]) : f2_fma(S, Y[j], T);
          }
          const f2 Z = f2_pack(bz[k], bz[k]);
          V = k == 0 ? f2_mul(T, Z) : f2_fma(T, Z, V);
        }
        f2_unpack(V, v0, v1);
        if constexpr (!F32) {
          v0 = fmaf(sa, v0, oa);
          v1 = fmaf(sb, v1, ob);
        }
      }
      if constexpr (COMP2) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
          float t = 0.f;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            float sx = 0.f;
#pragma unroll
            for (int i = 0; i < N; ++i) sx = fmaf(c2[(k * N + j) * N + i], bx[i], sx);
            t = fmaf(sx, by[j], t);
          }
          v2 = fmaf(t, bz[k], v2);
        }
        if constexpr (!F32) v2 = fmaf(sc, v2, oc);
      }
      if constexpr (FIELD == 1) return sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
      return v2;
    }
  }
};

// One CTA of 4 warps renders a 16x8-pixel tile (each warp an 8x4 patch), so
// the warps sharing an SM's L1 march through neighbouring elements; one lane
// traces one ray.  The element-change branch (look-up and block loads) is kept
// minimal: a warp runs it whenever any of its lanes changes element, which
// happens almost every iteration.
//
// In the sample loop the Alg. 2 update of sample k is issued together with
// the evaluation of sample k+1 (they are independent), so the scheduler can
// overlap their latencies; a ray that terminates after sample k discards the
// already evaluated sample k+1.
template <int P, int FIELD, int STORE>
__global__ void __launch_bounds__(128, 4) k_render(const __grid_constant__ RenderParams prm) {
  constexpr int N = P + 1;
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
  unsigned nsamp = 0, nlook = 0, nhit = 0;
  const float inf = __int_as_float(0x7f800000);

  Ray ray;
  if (i < prm.width && j < prm.row_end) {
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.f;
    if (make_ray(prm.ray, i, j, ray)) {
      ++nhit;
      const float tr_stop = 1.f - prm.alpha_stop;
      float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra, rd = ra;
      Block<P, FIELD, STORE> blk;
      float t = ray.tin;
      int k = 0;
      bool pend = false;     // a sample evaluated but not yet composited
      float pv = 0.f, pseg = 0.f;
      for (;;) {
        if (!(t < ray.tout)) {
          if (pend) {
            composite(tfb, tfd, pv, pseg, prm, C0, C1, C2, Tr);
            ++nsamp;
          }
          break;
        }
        const float px = fminf(fmaxf(__fmaf_rn(t, ray.d[0], ray.o[0]), 0.f), 1.f);
        const float py = fminf(fmaxf(__fmaf_rn(t, ray.d[1], ray.o[1]), 0.f), 1.f);
        const float pz = fminf(fmaxf(__fmaf_rn(t, ray.d[2], ray.o[2]), 0.f), 1.f);
        const bool inside = px >= ra.x && py >= ra.y && pz >= ra.z && px < rb.x && py < rb.y && pz < rb.z;
        if (!inside) {
          const uint32_t cur = forest_lookup(prm.forest, px, py, pz, prm.status);
          if (cur == kNone || (int64_t)cur >= prm.n_elem) {
            set_status(prm.status, kStatusBounds);
            break;
          }
          ++nlook;
          load_record(prm.elem + cur, ra, rb, rc, rd);
          if constexpr (FIELD == 2)
            blk.load(prm.bezc + (int64_t)cur * prm.elemc_bytes, prm.comp);
          else
            blk.load(prm.bez + (int64_t)cur * prm.elem_bytes, 0);
        }
        float tn = prm.mode == LRVOL_STEP_HEURISTIC ? __fadd_rn(t, ra.w) : __fmaf_rn((float)(k + 1), prm.h, ray.tin);
        if (!(tn > t)) tn = nextafterf(t, inf);
        const float seg = __fsub_rn(fminf(tn, ray.tout), t);
        // evaluate sample k ...
        float bx[N], by[N], bz[N];
        monomials<P>(local_u(px, ra.x, rc.x, rd.x), bx);
        monomials<P>(local_u(py, ra.y, rc.y, rd.y), by);
        monomials<P>(local_u(pz, ra.z, rc.z, rd.z), bz);
        const float v = blk.eval(bx, by, bz);
        // ... while compositing sample k-1
        if (pend) {
          composite(tfb, tfd, pv, pseg, prm, C0, C1, C2, Tr);
          ++nsamp;
          if (Tr <= tr_stop) break;
        }
        pend = true;
        pv = v;
        pseg = seg;
        t = tn;
        if (++k >= kMaxSamplesPerRay) {
          set_status(prm.status, kStatusTimeout);
          break;
        }
      }
    }
    reinterpret_cast<float4 *>(prm.out)[(int64_t)j * prm.width + i] = make_float4(C0, C1, C2, 1.f - Tr);
  }
  // per-warp counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nsamp += __shfl_down_sync(0xffffffffu, nsamp, o);
    nlook += __shfl_down_sync(0xffffffffu, nlook, o);
    nhit += __shfl_down_sync(0xffffffffu, nhit, o);
  }
  if (lane == 0) {
    atomicAdd(prm.counters + kCntSamples, (unsigned long long)nsamp);
    atomicAdd(prm.counters + kCntLookups, (unsigned long long)nlook);
    atomicAdd(prm.counters + kCntRays, (unsigned long long)nhit);
  }
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
                                                    v->storage, v->d_bez, v->elem_bytes, v->d_bezc, v->elemc_bytes);
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

template <int P, int FIELD, int STORE>
cudaError_t launch_render_t(const RenderParams &prm, cudaStream_t s) {
  const dim3 grid((unsigned)((prm.width + 15) / 16), (unsigned)((prm.row_end - prm.row_begin + 7) / 8));
  k_render<P, FIELD, STORE><<<grid, 128, 0, s>>>(prm);
  return cudaGetLastError();
}

template <int STORE>
cudaError_t launch_render_s(const RenderParams &prm, int degree, int f, cudaStream_t s) {
  switch (degree * 3 + f) {
    case 3: return launch_render_t<1, 0, STORE>(prm, s);
    case 4: return launch_render_t<1, 1, STORE>(prm, s);
    case 5: return launch_render_t<1, 2, STORE>(prm, s);
    case 6: return launch_render_t<2, 0, STORE>(prm, s);
    case 7: return launch_render_t<2, 1, STORE>(prm, s);
    case 8: return launch_render_t<2, 2, STORE>(prm, s);
    case 9: return launch_render_t<3, 0, STORE>(prm, s);
    case 10: return launch_render_t<3, 1, STORE>(prm, s);
    case 11: return launch_render_t<3, 2, STORE>(prm, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_render(const RenderParams &prm, int degree, int field, int storage, cudaStream_t s) {
  const int f = field == LRVOL_FIELD_MAGNITUDE ? 1 : (field == LRVOL_FIELD_COMPONENT ? 2 : 0);
  switch (storage) {
    case LRVOL_STORE_F32: return launch_render_s<LRVOL_STORE_F32>(prm, degree, f, s);
    case LRVOL_STORE_F16: return launch_render_s<LRVOL_STORE_F16>(prm, degree, f, s);
    case LRVOL_STORE_BF16: return launch_render_s<LRVOL_STORE_BF16>(prm, degree, f, s);
    default: return cudaErrorInvalidValue;
  }
}

// ----------------------------------------------------------------------------
// Scratch for lrvol_render_noalloc.  The render kernel needs a little global
// memory beyond its inputs and outputs: three statistics counters and a status
// word.  lrvol_render takes them from the handle; lrvol_render_noalloc takes
// them from this file-scope array, so that the call itself allocates nothing.
// Every GPU that loads the library holds these 256 bytes until the process
// exits.  Host code must not pass the symbol itself to a kernel (on the host it
// names a stand-in, not device memory): its device address is looked up once
// per device below.
// ----------------------------------------------------------------------------
}  // namespace lrvol

static __device__ __align__(256) unsigned long long g_render_scratch[lrvol::kStaticScratchWords];

namespace lrvol {

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_scratch_mutex;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};
}  // namespace

// Device address of g_render_scratch on the current device; resolved on the
// first call for that device, with that device current.
cudaError_t static_scratch(unsigned long long **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_render_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned long long *>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Same kernel as launch_render, with the counters and the status word in the
// static scratch (cleared on the stream before the launch).
cudaError_t launch_render_static(RenderParams prm, int degree, int field, int storage, cudaStream_t s,
                                 unsigned long long *counters_out) {
  unsigned long long *scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * kStaticScratchWords, s);
  if (e != cudaSuccess) return e;
  prm.counters = scratch;
  prm.status = reinterpret_cast<uint32_t *>(scratch + kNumCounters);
  e = launch_render(prm, degree, field, storage, s);
  if (e != cudaSuccess) return e;
  if (counters_out) {
    // samples, lookups, rays hit, then the status word widened to 64 bits
    e = cudaMemcpyAsync(counters_out, scratch + kCntSamples, sizeof(unsigned long long) * 3,
                        cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(counters_out + 3, scratch + kNumCounters, sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, s);
  }
  return e;
}

}  // namespace lrvol
