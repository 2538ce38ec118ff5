// Device helpers shared by the render kernel (render.cu) and the other
// kernels (kernels.cu): status word, forest look-up (Alg. 1), monomial
// basis and local coordinates of Bezier blocks (Sec. 3.2.3), FP32 rays,
// the transfer function and Alg. 2 compositing, packed FP32 pairs and
// the per-element block held in registers.  Each translation unit gets
// its own internal-linkage copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lrvol_internal.h"

namespace lrvol {
namespace {

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t code) { atomicCAS(status, 0u, code); }

// ----------------------------------------------------------------------------
// look-up (Alg. 1)
// ----------------------------------------------------------------------------

// Element holding the FP32 point (x, y, z), each coordinate in [0, 1] (every
// caller clamps or checks first): head word of its block, then the tree walk.
__device__ __forceinline__ uint32_t forest_lookup(const ForestView &f, float x, float y, float z, uint32_t *status) {
  // block index floor(p * blocks) (0 <= p <= 1, blocks <= 1024) as 2^23 + floor
  // by a round-down add, without a float-int conversion
  const int bx = min(__float_as_int(__fadd_rd(x * f.fbx, 8388608.f)) - 0x4b000000, f.bx - 1);
  const int by = min(__float_as_int(__fadd_rd(y * f.fby, 8388608.f)) - 0x4b000000, f.by - 1);
  const int bz = min(__float_as_int(__fadd_rd(z * f.fbz, 8388608.f)) - 0x4b000000, f.bz - 1);
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

// Derivatives d m_i / du = i u^(i-1) (1-u)^(p-i) - (p-i) u^i (1-u)^(p-i-1).
template <int P>
__device__ __forceinline__ void dmonomials(float u, float *d) {
  const float v = 1.f - u;
  if constexpr (P == 1) {
    d[0] = -1.f;
    d[1] = 1.f;
  } else if constexpr (P == 2) {
    d[0] = -2.f * v;
    d[1] = v - u;
    d[2] = 2.f * u;
  } else {
    const float uv = u * v;
    d[0] = -3.f * (v * v);
    d[1] = fmaf(-2.f, uv, v * v);
    d[2] = fmaf(2.f, uv, -(u * u));
    d[3] = 3.f * (u * u);
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

// u = (p - lo) / (hi - lo) as (p - lo_RU) * iw + (lo_RU - lo) * iw: one fused rounding after
// the subtraction, which is exact when p is near lo_RU (the offset term is tiny).
__device__ __forceinline__ float local_u(float p, float lo_ru, float off, float iw) {
  return __fmaf_rn(__fsub_rn(p, lo_ru), iw, off);
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
  // floor(x) without a float-int conversion (those issue on the narrow XU
  // pipe): adding 2^23 rounding down leaves 2^23 + floor(x) exactly
  const float r = __fadd_rd(x, 8388608.f);
  const int q = min(__float_as_int(r) - 0x4b000000, 254);
  const float fr = x - fminf(__fsub_rn(r, 8388608.f), 254.f);
  const float4 e0 = tfb[q], de = tfd[q];
  const float sa = fmaf(fr, de.w, e0.w);
  const float T = ex2_approx(lg2_approx(fmaxf(1.f - sa, 0.f)) * (seg * prm.inv_xi));
  const float w = fmaf(-Tr, T, Tr);
  C0 = fmaf(w, fmaf(fr, de.x, e0.x), C0);
  C1 = fmaf(w, fmaf(fr, de.y, e0.y), C1);
  C2 = fmaf(w, fmaf(fr, de.z, e0.z), C2);
  Tr *= T;
}

// Alg. 2 with C_src multiplied by the shading intensity sh (Sec. 4.1).
__device__ __forceinline__ void composite_shaded(const float4 *tfb, const float4 *tfd, float v, float seg, float sh,
                                                 const RenderParams &prm, float &C0, float &C1, float &C2,
                                                 float &Tr) {
  const float x = fminf(fmaxf(fmaf(v, prm.tf_scale, prm.tf_bias), 0.f), 255.f);
  // floor(x) without a float-int conversion (those issue on the narrow XU
  // pipe): adding 2^23 rounding down leaves 2^23 + floor(x) exactly
  const float r = __fadd_rd(x, 8388608.f);
  const int q = min(__float_as_int(r) - 0x4b000000, 254);
  const float fr = x - fminf(__fsub_rn(r, 8388608.f), 254.f);
  const float4 e0 = tfb[q], de = tfd[q];
  const float sa = fmaf(fr, de.w, e0.w);
  const float T = ex2_approx(lg2_approx(fmaxf(1.f - sa, 0.f)) * (seg * prm.inv_xi));
  const float w = fmaf(-Tr, T, Tr) * sh;
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

// A pixel's ray interval cut by its trimming interval (Sec. 4.1): no hit
// hides the pixel; only back faces (the eye inside the mesh) keep
// [t_in, t_back]; only front faces keep [t_front, t_out].
__device__ __forceinline__ bool trim_cut(float2 tr, float &tin, float &tout) {
  const float inf = __int_as_float(0x7f800000);
  if (tr.x == inf && tr.y == 0.f) return false;
  if (tr.x != inf && tr.x > tin) tin = tr.x;
  if (tr.y != 0.f && tr.y < tout) tout = tr.y;
  return tin < tout;
}

// Mixed-precision FMA d = a * b + c with FP16 a, b (exact product) and FP32 c, d.
__device__ __forceinline__ float fma_f16(unsigned short a, unsigned short b, float c) {
  float d;
  asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
  return d;
}
__device__ __forceinline__ unsigned short f16_bits(float x) { return __half_as_ushort(__float2half_rn(x)); }

// One element's block in registers and its evaluation at monomials bx, by, bz.
//   FIELD 0: scalar volume; 1: |v| of a 3-vector; 2: one component of a
//   3-vector, read from the plain per-component copy.
//   STORE: LRVOL_STORE_F32, or F16/BF16 values converted to FP32 when the
//   element is entered, with the value of component c = o_c + s_c * contraction.
//   FP16 blocks (MIXED) stay as 16-bit pairs in registers (half the registers
//   of FP32 values), and the first contraction stage multiplies them with the
//   x monomials rounded to FP16 in mixed-precision FMAs (exact products, FP32
//   sums); the later stages run in FP32 as for the other storages.
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

  static constexpr bool MIXED = STORE == LRVOL_STORE_F16;
  f2 rp[ROWPAIR && !MIXED ? 8 : 1][4];       // row pairs (2m, 2m+1), value i
  unsigned rh[ROWPAIR && MIXED ? 8 : 1][4];  // MIXED: FP16 words (row 2m, row 2m+1), value i
  float sg[SCALAR_GENERIC && !MIXED ? ((SGF + 7) & ~7) : 1];
  unsigned sgh[SCALAR_GENERIC && MIXED ? ((SGF + 7) & ~7) / 2 : 1];   // MIXED: slots (2w, 2w+1)
  f2 cp[PAIRS && !MIXED ? PAIRF / 2 : 1];    // (c0, c1) per q
  unsigned cph[PAIRS && MIXED ? PAIRF / 2 : 1];   // MIXED: FP16 (c0, c1) per q
  float c2[COMP2 && !MIXED ? C2F : 1];
  unsigned c2h[COMP2 && MIXED ? C2F / 2 : 1];     // MIXED: slots (2w, 2w+1)

  // half h (0: low) of a word of FP16 pairs
  __device__ __forceinline__ static unsigned short half_of(unsigned w, int h) {
    unsigned short lo, hi;
    asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(w));
    return h ? hi : lo;
  }
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
        // chunk m holds words 4m+i = (row 2m, row 2m+1) value i
        if constexpr (MIXED) {   // chunks m and m + 1 by one 256-bit load (the data start 32-byte aligned)
#pragma unroll
          for (int m = 0; m < 8; m += 2) {
            f2 a, b, c, e;
            ld256(d + m, a, b, c, e);
            rh[m][0] = (unsigned)a;
            rh[m][1] = (unsigned)(a >> 32);
            rh[m][2] = (unsigned)b;
            rh[m][3] = (unsigned)(b >> 32);
            rh[m + 1][0] = (unsigned)c;
            rh[m + 1][1] = (unsigned)(c >> 32);
            rh[m + 1][2] = (unsigned)e;
            rh[m + 1][3] = (unsigned)(e >> 32);
          }
        } else {
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const uint4 w = __ldg(d + m);
            rp[m][0] = word_to_f2<STORE>(w.x);
            rp[m][1] = word_to_f2<STORE>(w.y);
            rp[m][2] = word_to_f2<STORE>(w.z);
            rp[m][3] = word_to_f2<STORE>(w.w);
          }
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
            if constexpr (MIXED) {
              sgh[4 * q + t] = ws[t];
            } else {
              sg[8 * q + 2 * t] = h_to_f<STORE>(ws[t] & 0xffffu);
              sg[8 * q + 2 * t + 1] = h_to_f<STORE>(ws[t] >> 16);
            }
          }
        }
      }
      constexpr bool V256 = MIXED && (PAIRS || COMP2) && (FIELD == 1 || (C2F / 8) % 2 == 0);
      if constexpr (V256) {
        // this field's 16-bit words ((c0, c1) pairs then component 2, or one
        // component) by 256-bit loads from a 32-byte aligned start, a 128-bit tail
        constexpr int NP = PAIRS ? PAIRF / 8 : 0, NCH = NP + C2F / 8;
        const uint4 *src = FIELD == 1 ? d : d + comp * (C2F / 8);
        unsigned wv[4 * NCH];
#pragma unroll
        for (int q = 0; q + 1 < NCH; q += 2) {
          f2 a, b, c, e;
          ld256(src + q, a, b, c, e);
          wv[4 * q] = (unsigned)a;
          wv[4 * q + 1] = (unsigned)(a >> 32);
          wv[4 * q + 2] = (unsigned)b;
          wv[4 * q + 3] = (unsigned)(b >> 32);
          wv[4 * q + 4] = (unsigned)c;
          wv[4 * q + 5] = (unsigned)(c >> 32);
          wv[4 * q + 6] = (unsigned)e;
          wv[4 * q + 7] = (unsigned)(e >> 32);
        }
        if constexpr (NCH % 2 == 1) {
          const uint4 w = __ldg(src + NCH - 1);
          wv[4 * NCH - 4] = w.x;
          wv[4 * NCH - 3] = w.y;
          wv[4 * NCH - 2] = w.z;
          wv[4 * NCH - 1] = w.w;
        }
        if constexpr (PAIRS) {
#pragma unroll
          for (int q = 0; q < 4 * NP; ++q) cph[q] = wv[q];
        }
#pragma unroll
        for (int q = 0; q < C2F / 2; ++q) c2h[q] = wv[4 * NP + q];
      }
      if constexpr (PAIRS) {
        oa = h0.x;
        ob = h0.y;
        sa = h0.w;
        sb = h1.x;
#pragma unroll
        for (int q = 0; q < (V256 ? 0 : PAIRF / 8); ++q) {
          const uint4 w = __ldg(d + q);
          if constexpr (MIXED) {
            cph[4 * q] = w.x;
            cph[4 * q + 1] = w.y;
            cph[4 * q + 2] = w.z;
            cph[4 * q + 3] = w.w;
          } else {
            cp[4 * q] = word_to_f2<STORE>(w.x);
            cp[4 * q + 1] = word_to_f2<STORE>(w.y);
            cp[4 * q + 2] = word_to_f2<STORE>(w.z);
            cp[4 * q + 3] = word_to_f2<STORE>(w.w);
          }
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
        for (int q = 0; q < (V256 ? 0 : C2F / 8); ++q) {
          const uint4 w = __ldg(dc + q);
          const unsigned ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if constexpr (MIXED) {
              c2h[4 * q + t] = ws[t];
            } else {
              c2[8 * q + 2 * t] = h_to_f<STORE>(ws[t] & 0xffffu);
              c2[8 * q + 2 * t + 1] = h_to_f<STORE>(ws[t] >> 16);
            }
          }
        }
      }
    }
  }

  // MIXED: the x sums of rows 4k .. 4k+3 against FP16 monomials xh, as the
  // pairs (rows 4k, 4k+1) and (rows 4k+2, 4k+3).
  __device__ __forceinline__ void row_sums(int k, const unsigned short *xh, f2 &S0, f2 &S1) const {
    float s[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float se = 0.f, so = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        unsigned short lo, hi;
        asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(rh[2 * k + h][i]));
        se = fma_f16(lo, xh[i], se);
        so = fma_f16(hi, xh[i], so);
      }
      s[2 * h] = se;
      s[2 * h + 1] = so;
    }
    S0 = f2_pack(s[0], s[1]);
    S1 = f2_pack(s[2], s[3]);
  }

  // Scalar blocks: value and derivatives in local coordinates (d/du, d/dv, d/dw)
  // at monomials b* and their derivatives d*, reusing the partial sums of the value.
  __device__ __forceinline__ float eval_grad(const float *bx, const float *by, const float *bz, const float *dx,
                                             const float *dy, const float *dz, float &gu, float &gv,
                                             float &gw) const {
    static_assert(FIELD == 0, "gradients of scalar blocks only");
    if constexpr (ROWPAIR && MIXED) {
      unsigned short xh[4], dh[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xh[i] = f16_bits(bx[i]);
        dh[i] = f16_bits(dx[i]);
      }
      const f2 Y01 = f2_pack(by[0], by[1]), Y23 = f2_pack(by[2], by[3]);
      const f2 E01 = f2_pack(dy[0], dy[1]), E23 = f2_pack(dy[2], dy[3]);
      f2 F = 0, FX = 0, FY = 0, FZ = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        f2 S0, S1, R0, R1;
        row_sums(k, xh, S0, S1);
        row_sums(k, dh, R0, R1);
        const f2 T = f2_fma(S1, Y23, f2_mul(S0, Y01));
        const f2 TX = f2_fma(R1, Y23, f2_mul(R0, Y01));
        const f2 TY = f2_fma(S1, E23, f2_mul(S0, E01));
        const f2 Z = f2_pack(bz[k], bz[k]), DZ = f2_pack(dz[k], dz[k]);
        F = k == 0 ? f2_mul(T, Z) : f2_fma(T, Z, F);
        FX = k == 0 ? f2_mul(TX, Z) : f2_fma(TX, Z, FX);
        FY = k == 0 ? f2_mul(TY, Z) : f2_fma(TY, Z, FY);
        FZ = k == 0 ? f2_mul(T, DZ) : f2_fma(T, DZ, FZ);
      }
      float lo, hi;
      f2_unpack(FX, lo, hi);
      gu = sa * (lo + hi);
      f2_unpack(FY, lo, hi);
      gv = sa * (lo + hi);
      f2_unpack(FZ, lo, hi);
      gw = sa * (lo + hi);
      f2_unpack(F, lo, hi);
      return fmaf(sa, lo + hi, oa);
    } else if constexpr (ROWPAIR) {
      const f2 X0 = f2_pack(bx[0], bx[0]), X1 = f2_pack(bx[1], bx[1]);
      const f2 X2 = f2_pack(bx[2], bx[2]), X3 = f2_pack(bx[3], bx[3]);
      const f2 D0 = f2_pack(dx[0], dx[0]), D1 = f2_pack(dx[1], dx[1]);
      const f2 D2 = f2_pack(dx[2], dx[2]), D3 = f2_pack(dx[3], dx[3]);
      const f2 Y01 = f2_pack(by[0], by[1]), Y23 = f2_pack(by[2], by[3]);
      const f2 E01 = f2_pack(dy[0], dy[1]), E23 = f2_pack(dy[2], dy[3]);
      f2 F = 0, FX = 0, FY = 0, FZ = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const f2 *a = rp[2 * k], *b = rp[2 * k + 1];
        const f2 S0 = f2_fma(a[3], X3, f2_fma(a[2], X2, f2_fma(a[1], X1, f2_mul(a[0], X0))));
        const f2 S1 = f2_fma(b[3], X3, f2_fma(b[2], X2, f2_fma(b[1], X1, f2_mul(b[0], X0))));
        const f2 R0 = f2_fma(a[3], D3, f2_fma(a[2], D2, f2_fma(a[1], D1, f2_mul(a[0], D0))));
        const f2 R1 = f2_fma(b[3], D3, f2_fma(b[2], D2, f2_fma(b[1], D1, f2_mul(b[0], D0))));
        const f2 T = f2_fma(S1, Y23, f2_mul(S0, Y01));
        const f2 TX = f2_fma(R1, Y23, f2_mul(R0, Y01));
        const f2 TY = f2_fma(S1, E23, f2_mul(S0, E01));
        const f2 Z = f2_pack(bz[k], bz[k]), DZ = f2_pack(dz[k], dz[k]);
        F = k == 0 ? f2_mul(T, Z) : f2_fma(T, Z, F);
        FX = k == 0 ? f2_mul(TX, Z) : f2_fma(TX, Z, FX);
        FY = k == 0 ? f2_mul(TY, Z) : f2_fma(TY, Z, FY);
        FZ = k == 0 ? f2_mul(T, DZ) : f2_fma(T, DZ, FZ);
      }
      float lo, hi;
      f2_unpack(FX, lo, hi);
      gu = F32 ? lo + hi : sa * (lo + hi);
      f2_unpack(FY, lo, hi);
      gv = F32 ? lo + hi : sa * (lo + hi);
      f2_unpack(FZ, lo, hi);
      gw = F32 ? lo + hi : sa * (lo + hi);
      f2_unpack(F, lo, hi);
      return F32 ? lo + hi : fmaf(sa, lo + hi, oa);
    } else {
      unsigned short xh[N], dh[N];
      if constexpr (MIXED) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          xh[i] = f16_bits(bx[i]);
          dh[i] = f16_bits(dx[i]);
        }
      }
      float f = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        float t = 0.f, tx = 0.f, ty = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int r = k * N + j;
          float sx = 0.f, rx = 0.f;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            if constexpr (MIXED) {
              const unsigned short c = half_of(sgh[(r >> 1) * N + i], r & 1);
              sx = fma_f16(c, xh[i], sx);
              rx = fma_f16(c, dh[i], rx);
            } else {
              const float c = sg[(r >> 1) * 2 * N + 2 * i + (r & 1)];
              sx = fmaf(c, bx[i], sx);
              rx = fmaf(c, dx[i], rx);
            }
          }
          t = fmaf(sx, by[j], t);
          tx = fmaf(rx, by[j], tx);
          ty = fmaf(sx, dy[j], ty);
        }
        f = fmaf(t, bz[k], f);
        fx = fmaf(tx, bz[k], fx);
        fy = fmaf(ty, bz[k], fy);
        fz = fmaf(t, dz[k], fz);
      }
      gu = F32 ? fx : sa * fx;
      gv = F32 ? fy : sa * fy;
      gw = F32 ? fz : sa * fz;
      return F32 ? f : fmaf(sa, f, oa);
    }
  }

  __device__ __forceinline__ float eval(const float *bx, const float *by, const float *bz) const {
    if constexpr (ROWPAIR && MIXED) {
      unsigned short xh[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xh[i] = f16_bits(bx[i]);
      const f2 Y01 = f2_pack(by[0], by[1]), Y23 = f2_pack(by[2], by[3]);
      f2 F = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        f2 S0, S1;
        row_sums(k, xh, S0, S1);
        const f2 T = f2_fma(S1, Y23, f2_mul(S0, Y01));
        const f2 Z = f2_pack(bz[k], bz[k]);
        F = k == 0 ? f2_mul(T, Z) : f2_fma(T, Z, F);
      }
      float lo, hi;
      f2_unpack(F, lo, hi);
      return fmaf(sa, lo + hi, oa);
    } else if constexpr (ROWPAIR) {
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
      unsigned short xh[N];
      if constexpr (MIXED) {
#pragma unroll
        for (int i = 0; i < N; ++i) xh[i] = f16_bits(bx[i]);
      }
      float f = 0.f;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        float t = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int r = k * N + j;
          float sx = 0.f;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            if constexpr (MIXED)
              sx = fma_f16(half_of(sgh[(r >> 1) * N + i], r & 1), xh[i], sx);
            else
              sx = fmaf(sg[(r >> 1) * 2 * N + 2 * i + (r & 1)], bx[i], sx);
          }
          t = fmaf(sx, by[j], t);
        }
        f = fmaf(t, bz[k], f);
      }
      return F32 ? f : fmaf(sa, f, oa);
    } else {
      float v0, v1, v2;
      components(bx, by, bz, v0, v1, v2);
      if constexpr (FIELD == 1) return sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
      return v2;
    }
  }

  // Vector blocks: the components as evaluated (FIELD 1: all three; FIELD 2:
  // the chosen component in v2).
  __device__ __forceinline__ void components(const float *bx, const float *by, const float *bz, float &v0,
                                             float &v1, float &v2) const {
    v0 = 0.f;
    v1 = 0.f;
    v2 = 0.f;
    unsigned short xh[N];
    if constexpr (MIXED) {
#pragma unroll
      for (int i = 0; i < N; ++i) xh[i] = f16_bits(bx[i]);
    }
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
          f2 S;
          if constexpr (MIXED) {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const unsigned w = cph[(k * N + j) * N + i];
              s0 = fma_f16(half_of(w, 0), xh[i], s0);
              s1 = fma_f16(half_of(w, 1), xh[i], s1);
            }
            S = f2_pack(s0, s1);
          } else {
            const f2 *c = &cp[(k * N + j) * N];
            S = f2_mul(c[0], X[0]);
#pragma unroll
            for (int i = 1; i < N; ++i) S = f2_fma(c[i], X[i], S);
          }
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
          for (int i = 0; i < N; ++i) {
            const int q = (k * N + j) * N + i;
            if constexpr (MIXED)
              sx = fma_f16(half_of(c2h[q >> 1], q & 1), xh[i], sx);
            else
              sx = fmaf(c2[q], bx[i], sx);
          }
          t = fmaf(sx, by[j], t);
        }
        v2 = fmaf(t, bz[k], v2);
      }
      if constexpr (!F32) v2 = fmaf(sc, v2, oc);
    }
  }
};

}  // namespace
}  // namespace lrvol
