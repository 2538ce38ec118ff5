// liblrvol render kernel for sm_103a (Sec. 4, Alg. 2, Eq. 4).
//
//   k_render<P, FIELD, STORE, TRACE>
//       per-pixel ray casting with element reuse, Eq. 4 (or fixed, or learned)
//       steps, transfer function and Alg. 2 compositing, and gradient shading
//       (Sec. 4.1).  TRACE = false is the product kernel; TRACE = true is the
//       same template over a pixel list, writing every sample it composites.
//   launch_render, launch_render_trace, launch_render_static
//       the launches of lrvol_render, lrvol_render_trace and
//       lrvol_render_noalloc (the last with the library's static scratch).
#include <mutex>

#include "device_common.cuh"

static_assert(LRVOL_BAND_ROWS == 8, "a CTA renders 8 rows: one interleaved band");

namespace lrvol {
namespace {

// One CTA of 4 warps renders a 16x8-pixel tile, so the warps sharing an SM's
// L1 march through neighbouring elements; one lane traces one ray.  A warp
// covers an 8x4 patch for scalar fields and a 4x8 patch for 3-vector fields
// (the shapes that measured fastest for each).  The element-change branch (look-up and block loads) is kept
// minimal: a warp runs it whenever any of its lanes changes element, which
// happens almost every iteration.
//
// In the sample loop the Alg. 2 update of sample k is issued together with
// the evaluation of sample k+1 (they are independent), so the scheduler can
// overlap their latencies; a ray that terminates after sample k discards the
// already evaluated sample k+1.
//
// TRACE (a compile-time flag; false in every product launch, where the trace
// code compiles out) runs the same march for a list of pixels, one thread per
// listed pixel, and also writes each sample's (t, element id, field value,
// segment length), the composited sample count and the pixel's RGBA.  It is
// the parity hook that compares this kernel's own samples with the oracle.
//
// FIELD 3 renders a scalar volume with gradient shading (Sec. 4.1): each
// sample also evaluates the block's gradient, and C_src is scaled by
// I = max(0.4, |l . g| / max(|g|, eps)).
// CTAs per SM the register budget allows: the tricubic FP32/BF16 block takes
// 64 registers a lane (4 CTAs of 128 threads), 16-bit pairs of an FP16 block
// 32 (5 CTAs); the triquadratic 3-vector FP16 block (42 registers instead of
// 83) also fits 5.  The shaded tricubic kernel keeps the gradient's partial
// sums too: at 4 CTAs it spills 88 bytes and still beats 3 CTAs without
// spills by 5 % (measured); forcing 5 CTAs on the FP32 kernels spills
// inside the sample loop and costs 37-51 %.
template <int P, int FIELD, int STORE>
constexpr int render_min_ctas() {
  if (STORE == LRVOL_STORE_F16) {
    if (P == 3 && FIELD == 0) return 5;
    if (P == 2 && (FIELD == 1 || FIELD == 2)) return 5;
  }
  return 4;
}

template <int P, int FIELD, int STORE, bool TRACE>
__global__ void __launch_bounds__(128, (render_min_ctas<P, FIELD, STORE>())) k_render(const __grid_constant__ RenderParams prm) {
  constexpr int N = P + 1;
  constexpr bool SHADE = FIELD == 3;
  constexpr int BF = SHADE ? 0 : FIELD;
  __shared__ float4 tfb[256], tfd[256];
  for (int q = threadIdx.x; q < 256; q += blockDim.x) {
    const float4 e0 = prm.tf[q], e1 = prm.tf[q < 255 ? q + 1 : 255];
    tfb[q] = e0;
    tfd[q] = make_float4(e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w);
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int i, j;
  bool active;
  int64_t g = 0;               // TRACE: position in the pixel list
  uint32_t cur_e = kNone;      // TRACE: element of the current sample
  if constexpr (TRACE) {
    g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    active = g < prm.trace_n;
    i = active ? __ldg(prm.trace_pix + 2 * g) : 0;
    j = active ? __ldg(prm.trace_pix + 2 * g + 1) : 0;
    if (active && (i < 0 || i >= prm.width || j < 0 || j >= prm.height)) {
      set_status(prm.status, kStatusBounds);
      prm.trace_count[g] = 0;
      prm.trace_rgba[g] = make_float4(0.f, 0.f, 0.f, 0.f);
      active = false;
    }
  } else {
    if constexpr (BF == 1 || BF == 2) {   // 3-vector fields: four 4x8 patches side by side
      i = blockIdx.x * 16 + warp * 4 + (lane & 3);
      j = prm.row_begin + (blockIdx.y * prm.band_count + prm.band_index) * 8 + (lane >> 2);
    } else {                              // scalar fields: 2x2 patches of 8x4
      i = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
      j = prm.row_begin + (blockIdx.y * prm.band_count + prm.band_index) * 8 + (warp >> 1) * 4 + (lane >> 3);
    }
    active = i < prm.width && j < prm.row_end;
  }
  unsigned nsamp = 0, nlook = 0, nhit = 0;
  const float inf = __int_as_float(0x7f800000);

  Ray ray;
  if (active) {
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, Tr = 1.f;
    if (make_ray(prm.ray, i, j, ray) &&
        (prm.trim == nullptr || trim_cut(__ldg(prm.trim + (int64_t)j * prm.width + i), ray.tin, ray.tout))) {
      ++nhit;
      const float tr_stop = 1.f - prm.alpha_stop;
      float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra, rc = ra, rd = ra;
      float dsv = 0.f;       // step inside the current element (Eq. 4, or Eq. 4 x learned multiplier)
      Block<P, BF, STORE> blk;
      float t = ray.tin;
      int k = 0;
      bool pend = false;     // a sample evaluated but not yet composited
      float pv = 0.f, pseg = 0.f, psh = 1.f;
      float lx = 0.f, ly = 0.f, lz = 0.f;   // towards the light (shading)
      if constexpr (SHADE) {
        lx = prm.light_set ? prm.light[0] : -ray.d[0];
        ly = prm.light_set ? prm.light[1] : -ray.d[1];
        lz = prm.light_set ? prm.light[2] : -ray.d[2];
      }
      for (;;) {
        if (!(t < ray.tout)) {
          if (pend) {
            if constexpr (SHADE)
              composite_shaded(tfb, tfd, pv, pseg, psh, prm, C0, C1, C2, Tr);
            else
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
          if constexpr (TRACE) cur_e = cur;
          load_record(prm.elem + cur, ra, rb, rc, rd);
          dsv = prm.mode == LRVOL_STEP_LEARNED ? __fmul_rn(ra.w, __ldg(prm.mult + cur)) : ra.w;
          if constexpr (BF == 2)
            blk.load(prm.bezc + (int64_t)cur * prm.elemc_bytes, prm.comp);
          else
            blk.load(prm.bez + (int64_t)cur * prm.elem_bytes, 0);
        }
        float tn = prm.mode == LRVOL_STEP_FIXED ? __fmaf_rn((float)(k + 1), prm.h, ray.tin) : __fadd_rn(t, dsv);
        if (!(tn > t)) tn = nextafterf(t, inf);
        const float seg = __fsub_rn(fminf(tn, ray.tout), t);
        // evaluate sample k ...
        float bx[N], by[N], bz[N];
        const float ux = local_u(px, ra.x, rc.x, rd.x);
        const float uy = local_u(py, ra.y, rc.y, rd.y);
        const float uz = local_u(pz, ra.z, rc.z, rd.z);
        monomials<P>(ux, bx);
        monomials<P>(uy, by);
        monomials<P>(uz, bz);
        float v, sh = 1.f;
        if constexpr (SHADE) {
          float dx[N], dy[N], dz[N], gu, gv, gw;
          dmonomials<P>(ux, dx);
          dmonomials<P>(uy, dy);
          dmonomials<P>(uz, dz);
          v = blk.eval_grad(bx, by, bz, dx, dy, dz, gu, gv, gw);
          const float gx = gu * rd.x, gy = gv * rd.y, gz = gw * rd.z;   // world gradient: d/dx = iw d/du
          const float gl = fmaf(gx, lx, fmaf(gy, ly, gz * lz));
          const float gn = fmaxf(sqrtf(fmaf(gx, gx, fmaf(gy, gy, gz * gz))), prm.grad_eps);
          sh = fmaxf(0.4f, fabsf(gl) / gn);
        } else {
          v = blk.eval(bx, by, bz);
        }
        if constexpr (TRACE) {
          if (k < prm.trace_max) prm.trace_rec[g * prm.trace_max + k] = make_float4(t, __uint_as_float(cur_e), v, seg);
        }
        // ... while compositing sample k-1
        if (pend) {
          if constexpr (SHADE)
            composite_shaded(tfb, tfd, pv, pseg, psh, prm, C0, C1, C2, Tr);
          else
            composite(tfb, tfd, pv, pseg, prm, C0, C1, C2, Tr);
          ++nsamp;
          if (Tr <= tr_stop) break;
        }
        pend = true;
        pv = v;
        psh = sh;
        pseg = seg;
        t = tn;
        if (++k >= kMaxSamplesPerRay) {
          set_status(prm.status, kStatusTimeout);
          break;
        }
      }
    }
    if constexpr (TRACE) {
      prm.trace_rgba[g] = make_float4(C0, C1, C2, 1.f - Tr);
      prm.trace_count[g] = (int32_t)nsamp;
    } else {
      reinterpret_cast<float4 *>(prm.out)[(int64_t)j * prm.width + i] = make_float4(C0, C1, C2, 1.f - Tr);
    }
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

template <int P, int FIELD, int STORE, bool TRACE>
cudaError_t launch_render_t(const RenderParams &prm, cudaStream_t s) {
  if constexpr (TRACE) {
    k_render<P, FIELD, STORE, true><<<(unsigned)((prm.trace_n + 127) / 128), 128, 0, s>>>(prm);
  } else {
    // this call's bands: band_index, band_index + band_count, ... of the 8-row bands
    const int n_bands = (prm.row_end - prm.row_begin + 7) / 8;
    const int mine = (n_bands - prm.band_index + prm.band_count - 1) / prm.band_count;
    const dim3 grid((unsigned)((prm.width + 15) / 16), (unsigned)mine);
    k_render<P, FIELD, STORE, false><<<grid, 128, 0, s>>>(prm);
  }
  return cudaGetLastError();
}

template <int STORE, bool TRACE>
cudaError_t launch_render_s(const RenderParams &prm, int degree, int f, cudaStream_t s) {
  if (f == 3) {  // scalar with gradient shading
    switch (degree) {
      case 1: return launch_render_t<1, 3, STORE, TRACE>(prm, s);
      case 2: return launch_render_t<2, 3, STORE, TRACE>(prm, s);
      case 3: return launch_render_t<3, 3, STORE, TRACE>(prm, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (degree * 3 + f) {
    case 3: return launch_render_t<1, 0, STORE, TRACE>(prm, s);
    case 4: return launch_render_t<1, 1, STORE, TRACE>(prm, s);
    case 5: return launch_render_t<1, 2, STORE, TRACE>(prm, s);
    case 6: return launch_render_t<2, 0, STORE, TRACE>(prm, s);
    case 7: return launch_render_t<2, 1, STORE, TRACE>(prm, s);
    case 8: return launch_render_t<2, 2, STORE, TRACE>(prm, s);
    case 9: return launch_render_t<3, 0, STORE, TRACE>(prm, s);
    case 10: return launch_render_t<3, 1, STORE, TRACE>(prm, s);
    case 11: return launch_render_t<3, 2, STORE, TRACE>(prm, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool TRACE>
cudaError_t launch_render_any(const RenderParams &prm, int degree, int field, int storage, cudaStream_t s) {
  const int f = field == kFieldShaded ? 3 : (field == LRVOL_FIELD_MAGNITUDE ? 1 : (field == LRVOL_FIELD_COMPONENT ? 2 : 0));
  switch (storage) {
    case LRVOL_STORE_F32: return launch_render_s<LRVOL_STORE_F32, TRACE>(prm, degree, f, s);
    case LRVOL_STORE_F16: return launch_render_s<LRVOL_STORE_F16, TRACE>(prm, degree, f, s);
    case LRVOL_STORE_BF16: return launch_render_s<LRVOL_STORE_BF16, TRACE>(prm, degree, f, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_render(const RenderParams &prm, int degree, int field, int storage, cudaStream_t s) {
  return launch_render_any<false>(prm, degree, field, storage, s);
}

// The same kernel template with the trace compiled in, over the pixel list in
// prm.trace_pix (prm.trace_n entries).
cudaError_t launch_render_trace(const RenderParams &prm, int degree, int field, int storage, cudaStream_t s) {
  if (prm.trace_n == 0) return cudaSuccess;
  return launch_render_any<true>(prm, degree, field, storage, s);
}

// ----------------------------------------------------------------------------
// Scratch for lrvol_render_noalloc.  The render kernel needs a little global
// memory beyond its inputs and outputs: the kNumCounters statistics slots (the
// kernel adds to the first three) and a status word in a 64-bit slot, 72 bytes
// in all.  lrvol_render takes them from the handle; lrvol_render_noalloc takes
// them from this file-scope array, so that the call itself allocates nothing.
// Every GPU that loads the library holds these 256 bytes until the process
// exits.  Host code must not pass the symbol itself to a kernel (on the host it
// names a stand-in, not device memory): its device address is looked up once
// per device below and cached for the life of the process (a device reset by
// the caller invalidates it).
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
  if (prm.row_end > prm.row_begin) {   // an empty row band launches nothing, as in lrvol_render
    e = launch_render(prm, degree, field, storage, s);
    if (e != cudaSuccess) return e;
  }
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

