// a1 -- atlas gather (Sec. 4.2 "Fitting UV Maps Directly"; FP16 proxy of
// "Low Precision Optimization").  Live texels of the occupancy mask, in
// row-major order, become the Gaussians 0..N-1 of every frame.
//
// Two kernels: a single-block scan of per-word popcounts (the mask is at
// most a few hundred thousand words), then one thread per group of four
// texels that reads each channel with one 16-byte (FP32) or 8-byte (FP16)
// load and writes the live ones to the channel-major SoA.
#include <cuda_fp16.h>

#include "pk_common.cuh"

using namespace pk;

namespace {

constexpr int kScanThreads = 1024;

// woff[i] = number of live texels in mask words [0, i); woff[nwords] = total.
// One block: each pass covers kScanThreads * kRun consecutive words, a run
// of kRun per thread (popcounts summed in the thread, one block-wide scan of
// the run totals, then the run's prefixes written back), so a 1024^2 mask
// takes one pass instead of 32 barrier-separated steps.
constexpr int kRun = 32;
__global__ __launch_bounds__(kScanThreads) void k_word_scan(const uint32_t *__restrict__ occ, int64_t nwords,
                                                            uint32_t *__restrict__ woff,
                                                            pk_device_status *status, int64_t N) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nwords; base += (int64_t)kScanThreads * kRun) {
    const int64_t w0 = base + (int64_t)tid * kRun;
    uint32_t c[kRun];
    uint32_t tot = 0;
    if (w0 + kRun <= nwords && (reinterpret_cast<uintptr_t>(occ) & 15u) == 0) {
      // a whole run: 16-byte loads (the run starts on a 128-byte boundary)
      const uint4 *q = reinterpret_cast<const uint4 *>(occ + w0);
#pragma unroll
      for (int k = 0; k < kRun / 4; ++k) {
        const uint4 v = __ldg(q + k);
        c[4 * k] = __popc(v.x);
        c[4 * k + 1] = __popc(v.y);
        c[4 * k + 2] = __popc(v.z);
        c[4 * k + 3] = __popc(v.w);
      }
    } else {
#pragma unroll
      for (int k = 0; k < kRun; ++k) c[k] = w0 + k < nwords ? __popc(__ldg(occ + w0 + k)) : 0u;
    }
#pragma unroll
    for (int k = 0; k < kRun; ++k) tot += c[k];
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t carry = s_carry;
    uint32_t run = carry + (warp ? s_warp[warp - 1] : 0u) + x - tot;
    if (w0 + kRun <= nwords && (reinterpret_cast<uintptr_t>(woff) & 15u) == 0) {
      // a whole run: 16-byte stores, a quarter of the store instructions
      uint4 *o4 = reinterpret_cast<uint4 *>(woff + w0);
#pragma unroll
      for (int k = 0; k < kRun / 4; ++k) {
        uint4 v;
        v.x = run;
        v.y = v.x + c[4 * k];
        v.z = v.y + c[4 * k + 1];
        v.w = v.z + c[4 * k + 2];
        run = v.w + c[4 * k + 3];
        o4[k] = v;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kRun; ++k) {
        if (w0 + k < nwords) woff[w0 + k] = run;
        run += c[k];
      }
    }
    __syncthreads();
    if (tid == 0) s_carry = carry + s_warp[31];
    __syncthreads();
  }
  if (tid == 0) {
    woff[nwords] = s_carry;
    status->live_seen = s_carry;
    status->nonfinite = 0;   // counted by the gather kernel that follows
    if ((int64_t)s_carry != N) atomicOr(&status->flags, PK_DEV_LIVE_MISMATCH);
  }
}

template <typename Tex>
struct Quad;
template <>
struct Quad<float> {
  using V = float4;
  __device__ static float get(const V &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
  __device__ static float one(const float *p) { return *p; }
};
template <>
struct Quad<__half> {
  using V = uint2;
  __device__ static float get(const V &v, int i) {
    uint32_t w = (i < 2) ? v.x : v.y;
    unsigned short h = (i & 1) ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xffffu);
    return __half2float(__ushort_as_half(h));
  }
  __device__ static float one(const __half *p) { return __half2float(*p); }
};

// Live bits and Gaussian indices of the (up to) four texels x0 .. x0 + 3
// of row y; writes their texel ids and dynamic flags.  False if none is live.
__device__ __forceinline__ bool quad_live(const uint32_t *__restrict__ occ, const uint32_t *__restrict__ dyn,
                                          const uint32_t *__restrict__ woff, int W, int y, int x0, int64_t N,
                                          uint32_t *__restrict__ texel, uint8_t *__restrict__ dynflag,
                                          bool live[4], int64_t gidx[4]) {
  const int Wp = (W + 31) / 32;
  bool any = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int x = x0 + i;
    live[i] = false;
    gidx[i] = 0;
    if (x < W) {
      uint32_t word = occ[(int64_t)y * Wp + (x >> 5)];
      uint32_t bit = 1u << (x & 31);
      if (word & bit) {
        int64_t g = woff[(int64_t)y * Wp + (x >> 5)] + __popc(word & (bit - 1u));
        if (g < N) {
          live[i] = true;
          gidx[i] = g;
          any = true;
          texel[g] = (uint32_t)((int64_t)y * W + x);
          dynflag[g] = dyn ? (uint8_t)((dyn[(int64_t)y * Wp + (x >> 5)] >> (x & 31)) & 1u) : (uint8_t)1;
        }
      }
    }
  }
  return any;
}

// One thread per 4 consecutive texels of a row.
template <typename Tex, bool kVec>
__global__ __launch_bounds__(256) void k_gather(const Tex *__restrict__ atlas, const uint32_t *__restrict__ occ,
                                                const uint32_t *__restrict__ dyn, const uint32_t *__restrict__ woff,
                                                int W, int H, int F, int D, int64_t N,
                                                float *__restrict__ soa, uint32_t *__restrict__ texel,
                                                uint8_t *__restrict__ dynflag, pk_device_status *status) {
  const int Wq = (W + 3) / 4;
  uint32_t nbad = 0;   // (frame, Gaussian) pairs of this thread with a non-finite texel value
  const int64_t nq = (int64_t)Wq * H;
  const int64_t plane = (int64_t)W * H;
  const int64_t G = (int64_t)F * N;
  for (int64_t qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qi < nq; qi += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(qi / Wq), x0 = (int)(qi % Wq) * 4;
    int64_t gidx[4];
    bool live[4];
    if (!quad_live(occ, dyn, woff, W, y, x0, N, texel, dynflag, live, gidx)) continue;
    const int64_t pix = (int64_t)y * W + x0;
    for (int f = 0; f < F; ++f) {
      uint32_t bad = 0;   // bit i: texel i has a non-finite value in some channel of frame f
#pragma unroll 4
      for (int c = 0; c < D; ++c) {
        const Tex *src = atlas + ((int64_t)f * D + c) * plane + pix;
        float* dst = soa + (int64_t)c * G + (int64_t)f * N;
        if (kVec) {
          typename Quad<Tex>::V v = __ldg(reinterpret_cast<const typename Quad<Tex>::V *>(src));
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (live[i]) {
              const float x = Quad<Tex>::get(v, i);
              dst[gidx[i]] = x;
              bad |= (uint32_t)!isfinite(x) << i;
            }
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (live[i]) {
              const float x = Quad<Tex>::one(src + i);
              dst[gidx[i]] = x;
              bad |= (uint32_t)!isfinite(x) << i;
            }
        }
      }
      nbad += __popc(bad);
    }
  }
  // one atomic per warp
  const uint32_t wbad = __reduce_add_sync(0xffffffffu, nbad);
  if ((threadIdx.x & 31) == 0 && wbad) atomicAdd(reinterpret_cast<unsigned long long *>(&status->nonfinite), wbad);
}

// Low-precision proxy (Sec. 4.2 "Low Precision Optimization"): channel c
// quantised to 16 (position) or 8 bits over [lo_c, hi_c], read either as
// codes ([F][D + 3][H][W] bytes, position as high and low byte planes) or
// by fake-quantising the FP32 masters on the fly.  FP32 steps in the order
// packuv.h states, without fused multiply-adds.
__device__ __forceinline__ float lpo_proxy(uint32_t q, float lo, float delta) {
  return __fadd_rn(lo, __fmul_rn((float)q, delta));
}

__device__ __forceinline__ uint32_t lpo_code(float x, float lo, float delta, float L) {
  const float u = floorf(__fadd_rn(__fdiv_rn(__fsub_rn(x, lo), delta), 0.5f));
  if (!(u >= 0.0f)) return 0u;
  if (u >= L) return (uint32_t)L;
  return (uint32_t)u;
}

template <bool kCodes>
__global__ __launch_bounds__(256) void k_gather_lpo(const void *__restrict__ src, const float *__restrict__ lohi,
                                                    const uint32_t *__restrict__ occ,
                                                    const uint32_t *__restrict__ dyn,
                                                    const uint32_t *__restrict__ woff, int W, int H, int F, int D,
                                                    int64_t N, float *__restrict__ soa,
                                                    uint32_t *__restrict__ texel, uint8_t *__restrict__ dynflag) {
  __shared__ float s_lo[PK_MAX_CHANNELS], s_delta[PK_MAX_CHANNELS];
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    const float L = c < 3 ? 65535.0f : 255.0f;
    s_lo[c] = lohi[2 * c];
    s_delta[c] = __fdiv_rn(__fsub_rn(lohi[2 * c + 1], lohi[2 * c]), L);
  }
  __syncthreads();
  const int Wq = (W + 3) / 4;
  const int64_t nq = (int64_t)Wq * H;
  const int64_t plane = (int64_t)W * H;
  const int64_t G = (int64_t)F * N;
  for (int64_t qi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qi < nq; qi += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(qi / Wq), x0 = (int)(qi % Wq) * 4;
    int64_t gidx[4];
    bool live[4];
    if (!quad_live(occ, dyn, woff, W, y, x0, N, texel, dynflag, live, gidx)) continue;
    const int64_t pix = (int64_t)y * W + x0;
    for (int f = 0; f < F; ++f) {
      for (int c = 0; c < D; ++c) {
        const float lo = s_lo[c], delta = s_delta[c];
        float *dst = soa + (int64_t)c * G + (int64_t)f * N;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!live[i]) continue;
          uint32_t q;
          if (kCodes) {
            const uint8_t *cb = reinterpret_cast<const uint8_t *>(src) + (int64_t)f * (D + 3) * plane + pix + i;
            q = c < 3 ? ((uint32_t)__ldg(cb + (2 * c) * plane) << 8) | __ldg(cb + (2 * c + 1) * plane)
                      : (uint32_t)__ldg(cb + (c + 3) * plane);
          } else {
            const float x = __ldg(reinterpret_cast<const float *>(src) + ((int64_t)f * D + c) * plane + pix + i);
            q = lpo_code(x, lo, delta, c < 3 ? 65535.0f : 255.0f);
          }
          dst[gidx[i]] = lpo_proxy(q, lo, delta);
        }
      }
    }
  }
}

}  // namespace

extern "C" pk_status pk_atlas_gather_lpo(const pk_plan *p, const void *src, int32_t src_kind, const float *lohi,
                                         const uint32_t *occ, const uint32_t *dyn, float *soa, uint32_t *texel,
                                         uint8_t *dynflag, void *ws, pk_stream_t stream) {
  if (!p || !src || !lohi || !occ || !soa || !texel || !dynflag || !ws) return PK_ERR_ARG;
  if (src_kind != PK_LPO_CODES && src_kind != PK_LPO_MASTERS) return PK_ERR_ARG;
  if (!aligned16(soa)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int W = p->desc.atlas_w, H = p->desc.atlas_h;
  const int64_t nwords = (int64_t)((W + 31) / 32) * H;
  uint32_t *woff = at<uint32_t>(ws, p->ws.woff);
  pk_device_status *status = at<pk_device_status>(ws, p->ws.status);
  k_word_scan<<<1, kScanThreads, 0, st>>>(occ, nwords, woff, status, p->N);
  const int64_t nq = (int64_t)((W + 3) / 4) * H;
  int blocks = (int)((nq + 255) / 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  if (src_kind == PK_LPO_CODES)
    k_gather_lpo<true><<<blocks, 256, 0, st>>>(src, lohi, occ, dyn, woff, W, H, p->F, p->D, p->N, soa, texel,
                                               dynflag);
  else
    k_gather_lpo<false><<<blocks, 256, 0, st>>>(src, lohi, occ, dyn, woff, W, H, p->F, p->D, p->N, soa, texel,
                                                dynflag);
  return check_launch();
}

extern "C" pk_status pk_atlas_gather(const pk_plan *p, const void *atlas, const uint32_t *occ, const uint32_t *dyn,
                                     float *soa, uint32_t *texel, uint8_t *dynflag, void *ws, pk_stream_t stream) {
  if (!p || !atlas || !occ || !soa || !texel || !dynflag || !ws) return PK_ERR_ARG;
  if (!aligned16(atlas) || !aligned16(soa)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int W = p->desc.atlas_w, H = p->desc.atlas_h;
  const int64_t nwords = (int64_t)((W + 31) / 32) * H;
  uint32_t *woff = at<uint32_t>(ws, p->ws.woff);
  pk_device_status *status = at<pk_device_status>(ws, p->ws.status);
  k_word_scan<<<1, kScanThreads, 0, st>>>(occ, nwords, woff, status, p->N);
  const int64_t nq = (int64_t)((W + 3) / 4) * H;
  int blocks = (int)((nq + 255) / 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  const bool vec = (W % 4) == 0;
  if (p->desc.texel_type == PK_TEXEL_F16) {
    auto a = reinterpret_cast<const __half *>(atlas);
    if (vec)
      k_gather<__half, true><<<blocks, 256, 0, st>>>(a, occ, dyn, woff, W, H, p->F, p->D, p->N, soa, texel, dynflag, status);
    else
      k_gather<__half, false><<<blocks, 256, 0, st>>>(a, occ, dyn, woff, W, H, p->F, p->D, p->N, soa, texel, dynflag,
                                                      status);
  } else {
    auto a = reinterpret_cast<const float *>(atlas);
    if (vec)
      k_gather<float, true><<<blocks, 256, 0, st>>>(a, occ, dyn, woff, W, H, p->F, p->D, p->N, soa, texel, dynflag,
                                                    status);
    else
      k_gather<float, false><<<blocks, 256, 0, st>>>(a, occ, dyn, woff, W, H, p->F, p->D, p->N, soa, texel, dynflag,
                                                     status);
  }
  return check_launch();
}
