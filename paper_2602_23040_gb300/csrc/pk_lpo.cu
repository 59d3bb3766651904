// Low-precision proxy (Sec. 4.2 "Low Precision Optimization", Supp. "Video
// Coding"): per-channel min/max normalisation over the live texels of every
// frame and the 8-bit plane layout (position as two bytes).  The gather
// that reads the proxy lives with the other gathers.
//
// Both kernels stream the planar FP32 atlas once, four consecutive texels
// per thread, one block row per (frame, channel) plane.
#include "pk_common.cuh"

using namespace pk;

namespace {

constexpr int kLpoThreads = 256;

// Order-preserving map of a float onto uint32 (NaN excluded by the caller).
__device__ __forceinline__ uint32_t ordered(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unordered(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_minmax_init(uint32_t *keys, int D) {
  const int i = threadIdx.x;
  if (i < 2 * D) keys[i] = (i & 1) ? 0u : 0xffffffffu;
}

// Planes fc = f * D + c from blockIdx.y in steps of gridDim.y; each thread
// folds up to 4 texels per stride step.
__global__ __launch_bounds__(kLpoThreads) void k_minmax(const float *__restrict__ atlas,
                                                        const uint32_t *__restrict__ occ, int W, int H, int D,
                                                        int64_t planes, uint32_t *keys) {
  const int Wq = (W + 3) >> 2, Wp = (W + 31) >> 5;
  const int64_t nq = (int64_t)Wq * H, plane = (int64_t)W * H;
  const bool vec = (W & 3) == 0;   // 16-byte aligned rows of four texels
  for (int64_t fc = blockIdx.y; fc < planes; fc += gridDim.y) {
    const int c = (int)(fc % D);
    const float *src = atlas + fc * plane;
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int64_t qi = (int64_t)blockIdx.x * kLpoThreads + threadIdx.x; qi < nq;
         qi += (int64_t)gridDim.x * kLpoThreads) {
      const int y = (int)(qi / Wq), x0 = (int)(qi - (int64_t)y * Wq) * 4;
      // the four texels share one occupancy word (x0 is a multiple of 4)
      const uint32_t word = __ldg(occ + (int64_t)y * Wp + (x0 >> 5)) >> (x0 & 31);
      if (!(word & 15u)) continue;
      float v4[4];
      if (vec) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(src + (int64_t)y * W + x0));
        v4[0] = q.x; v4[1] = q.y; v4[2] = q.z; v4[3] = q.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) v4[i] = x0 + i < W ? __ldg(src + (int64_t)y * W + x0 + i) : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float v = v4[i];
        if (x0 + i >= W || !((word >> i) & 1u) || v != v) continue;
        const uint32_t k = ordered(v);
        lo = min(lo, k);
        hi = max(hi, k);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
      if (lo != 0xffffffffu) atomicMin(&keys[2 * c], lo);
      if (hi != 0u) atomicMax(&keys[2 * c + 1], hi);
    }
  }
}

__global__ void k_minmax_final(uint32_t *keys, int D) {
  const int c = threadIdx.x;
  if (c >= D) return;
  const uint32_t lo = keys[2 * c], hi = keys[2 * c + 1];
  float *out = reinterpret_cast<float *>(keys);
  const bool none = lo == 0xffffffffu;
  out[2 * c] = none ? 0.0f : unordered(lo);
  out[2 * c + 1] = none ? 0.0f : unordered(hi);
}

__device__ __forceinline__ uint32_t lpo_code(float x, float lo, float delta, float L) {
  const float u = floorf(__fadd_rn(__fdiv_rn(__fsub_rn(x, lo), delta), 0.5f));
  if (!(u >= 0.0f)) return 0u;
  if (u >= L) return (uint32_t)L;
  return (uint32_t)u;
}

__device__ __forceinline__ void encode_plane(const float *__restrict__ atlas, const uint32_t *__restrict__ occ,
                                             const float *__restrict__ lohi, int W, int H, int D, int64_t fc,
                                             uint8_t *__restrict__ codes) {
  const int f = (int)(fc / D), c = (int)(fc - (int64_t)f * D);
  const int Wq = (W + 3) >> 2, Wp = (W + 31) >> 5;
  const int64_t nq = (int64_t)Wq * H, plane = (int64_t)W * H;
  const float L = c < 3 ? 65535.0f : 255.0f;
  const float lo = __ldg(lohi + 2 * c);
  const float delta = __fdiv_rn(__fsub_rn(__ldg(lohi + 2 * c + 1), lo), L);
  const float *src = atlas + fc * plane;
  uint8_t *p0 = codes + ((int64_t)f * (D + 3) + (c < 3 ? 2 * c : c + 3)) * plane;
  uint8_t *p1 = c < 3 ? p0 + plane : nullptr;
  const bool vec = (W & 3) == 0;
  for (int64_t qi = (int64_t)blockIdx.x * kLpoThreads + threadIdx.x; qi < nq;
       qi += (int64_t)gridDim.x * kLpoThreads) {
    const int y = (int)(qi / Wq), x0 = (int)(qi - (int64_t)y * Wq) * 4;
    const int64_t at0 = (int64_t)y * W + x0;
    const uint32_t word = __ldg(occ + (int64_t)y * Wp + (x0 >> 5)) >> (x0 & 31);
    float v4[4] = {0.f, 0.f, 0.f, 0.f};
    if (word & 15u) {
      if (vec) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(src + at0));
        v4[0] = q.x; v4[1] = q.y; v4[2] = q.z; v4[3] = q.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) v4[i] = x0 + i < W ? __ldg(src + at0 + i) : 0.f;
      }
    }
    uint32_t b0 = 0, b1 = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int x = x0 + i;
      if (x >= W || !((word >> i) & 1u)) continue;
      const uint32_t q = lpo_code(v4[i], lo, delta, L);
      if (c < 3) {
        b0 |= (q >> 8) << (8 * i);
        b1 |= (q & 255u) << (8 * i);
      } else {
        b0 |= q << (8 * i);
      }
    }
    if (vec) {
      *reinterpret_cast<uint32_t *>(p0 + at0) = b0;
      if (p1) *reinterpret_cast<uint32_t *>(p1 + at0) = b1;
    } else {
      for (int i = 0; i < 4 && x0 + i < W; ++i) {
        p0[at0 + i] = (uint8_t)(b0 >> (8 * i));
        if (p1) p1[at0 + i] = (uint8_t)(b1 >> (8 * i));
      }
    }
  }
}

// Planes fc = f * D + c as in k_minmax; four texels per thread, written as
// one 4-byte group per code plane when the width allows.
__global__ __launch_bounds__(kLpoThreads) void k_encode(const float *__restrict__ atlas,
                                                        const uint32_t *__restrict__ occ,
                                                        const float *__restrict__ lohi, int W, int H, int D,
                                                        int64_t planes, uint8_t *__restrict__ codes) {
  for (int64_t fc = blockIdx.y; fc < planes; fc += gridDim.y) encode_plane(atlas, occ, lohi, W, H, D, fc, codes);
}

dim3 plane_grid(const pk_plan *p, int64_t planes) {
  const int W = p->desc.atlas_w, H = p->desc.atlas_h;
  const int64_t nq = (int64_t)((W + 3) / 4) * H;
  int64_t bx = (nq + kLpoThreads - 1) / kLpoThreads;
  // about 8 resident blocks per SM over all planes
  const int64_t cap = (152 * 8 + planes - 1) / planes;
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, (unsigned)(planes < 65535 ? planes : 65535));
}

}  // namespace

extern "C" pk_status pk_lpo_minmax(const pk_plan *p, const float *atlas, const uint32_t *occ, float *lohi, void *ws,
                                   pk_stream_t stream) {
  if (!p || !atlas || !occ || !lohi || !ws) return PK_ERR_ARG;
  if (!aligned16(atlas) || !aligned16(lohi)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t *keys = reinterpret_cast<uint32_t *>(lohi);
  k_minmax_init<<<1, 128, 0, st>>>(keys, p->D);
  k_minmax<<<plane_grid(p, (int64_t)p->F * p->D), kLpoThreads, 0, st>>>(atlas, occ, p->desc.atlas_w,
                                                                        p->desc.atlas_h, p->D,
                                                                        (int64_t)p->F * p->D, keys);
  k_minmax_final<<<1, 64, 0, st>>>(keys, p->D);
  return check_launch();
}

extern "C" pk_status pk_lpo_encode(const pk_plan *p, const float *atlas, const uint32_t *occ, const float *lohi,
                                   uint8_t *codes, void *ws, pk_stream_t stream) {
  if (!p || !atlas || !occ || !lohi || !codes || !ws) return PK_ERR_ARG;
  if (!aligned16(atlas) || !aligned16(codes)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_encode<<<plane_grid(p, (int64_t)p->F * p->D), kLpoThreads, 0, st>>>(atlas, occ, lohi, p->desc.atlas_w,
                                                                        p->desc.atlas_h, p->D,
                                                                        (int64_t)p->F * p->D, codes);
  return check_launch();
}
