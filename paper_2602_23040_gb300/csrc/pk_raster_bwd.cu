// a5 -- adjoint of the compositing (Sec. 4.2 "Objective").  Each pixel
// walks its tile's list backwards from its last blended splat, recovering
// T_i = T_{i+1} / (1 - alpha_i) from the stored final transmittance, so no
// per-step state of the forward is kept.  Per splat the 9 gradients of a
// warp's 32 pixels are summed by a reduce-scatter over the lanes (12
// shuffles instead of 45 for nine full butterfly sums), after which nine
// lanes each hold one complete sum and add it to the splat's gradient
// record with one coalesced atomic instruction.
#include "pk_raster.cuh"

using namespace pk;

namespace {

// Reduce-scatter of v[0..8] over the 32 lanes.  Level xor-16 splits the
// nine values 5 | 4, xor-8 splits each half 3 | 2, xor-4 2 | 1, xor-2 1 | 1
// and xor-1 adds the last pair.  Returns the complete sum held by this lane
// and its value index in *idx (-1 for lanes left holding padding).
__device__ __forceinline__ float warp_reduce_scatter9(const float (&v)[9], int lane, int *idx) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float w[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const float lo = v[j], hi = (5 + j < 9) ? v[5 + j] : 0.f;
    const float r = __shfl_xor_sync(0xffffffffu, b4 ? lo : hi, 16);
    w[j] = (b4 ? hi : lo) + r;
  }
  float x[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float lo = w[j], hi = (3 + j < 5) ? w[3 + j] : 0.f;
    const float r = __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 8);
    x[j] = (b3 ? hi : lo) + r;
  }
  float y[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float lo = x[j], hi = (2 + j < 3) ? x[2 + j] : 0.f;
    const float r = __shfl_xor_sync(0xffffffffu, b2 ? lo : hi, 4);
    y[j] = (b2 ? hi : lo) + r;
  }
  float z;
  {
    const float r = __shfl_xor_sync(0xffffffffu, b1 ? y[0] : y[1], 2);
    z = (b1 ? y[1] : y[0]) + r;
  }
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  // value index held: level sets [0..4 | 5..8], slots [0,1,2 | 3,4], [0,1 | 2], [0 | 1]
  const int s2 = b2 ? (b1 ? -1 : 2) : (b1 ? 1 : 0);         // slot in x
  const int s3 = s2 < 0 ? -1 : (b3 ? (s2 < 2 ? 3 + s2 : -1) : s2);  // slot in w
  const int s4 = s3 < 0 ? -1 : (b4 ? (s3 < 4 ? 5 + s3 : -1) : s3);  // value index
  *idx = (lane & 1) ? -1 : s4;
  return z;
}

__global__ __launch_bounds__(kRasterThreads) void k_raster_bwd(
    const float *__restrict__ rec, const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
    const DevView *__restrict__ views, const uint32_t *__restrict__ toff, int V, uint32_t n_tiles, float bg0,
    float bg1, float bg2, const float *__restrict__ Tfin, const uint32_t *__restrict__ ncontrib,
    const float *__restrict__ dimg, float *__restrict__ grad2d, uint32_t *queue, unsigned long long *evals_out) {
  __shared__ float4 s_a[kBatch], s_b[kBatch], s_c[kBatch], s_box[kBatch], s_q[kBatch];
  __shared__ uint32_t s_tile;
  __shared__ int s_view;
  __shared__ uint32_t s_wmax[kRasterThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Staged st{s_a, s_b, s_c, s_box, s_q};
  int ox, oy;
  pixel_of(tid, ox, oy);
  unsigned long long evals = 0;
  for (;;) {
    if (tid == 0) {
      const uint32_t t = atomicAdd(queue, 1u);
      s_tile = t;
      s_view = t < n_tiles ? view_of_tile(toff, V, t) : -1;
    }
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= n_tiles) break;
    const DevView &view = views[s_view];
    const int W = view.width, H = view.height;
    const uint32_t local = t - (uint32_t)view.tile_off;
    const int ty = (int)(local / (uint32_t)view.tiles_x), tx = (int)(local - (uint32_t)ty * view.tiles_x);
    const int x = tx * kTileSide + ox, y = ty * kTileSide + oy;
    const bool inside = x < W && y < H;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    const float wx0 = (float)(tx * kTileSide + (ox & ~7)) + 0.5f, wx1 = wx0 + 7.f;
    const float wy0 = (float)(ty * kTileSide + (oy & ~3)) + 0.5f, wy1 = wy0 + 3.f;
    const uint32_t s = __ldg(ranges + 2 * (size_t)t);
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t nc = 0;
    if (inside) {
      const size_t pix = (size_t)view.pix_off + (size_t)y * W + x;
      const size_t plane = (size_t)W * H;
      const float *gi = dimg + 3 * (size_t)view.pix_off + (size_t)y * W + x;
      T = Tfin[pix];
      nc = ncontrib[pix];
      g0 = gi[0];
      g1 = gi[plane];
      g2 = gi[2 * plane];
    }
    // colour composited behind the current splat, background included
    float S0 = T * bg0, S1 = T * bg1, S2 = T * bg2;
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, nc);
    if (lane == 0) s_wmax[warp] = wmax;
    __syncthreads();
    uint32_t tmax = 0;
#pragma unroll
    for (int w = 0; w < kRasterThreads / 32; ++w) tmax = max(tmax, s_wmax[w]);
    for (uint32_t end = tmax; end > 0;) {
      const uint32_t beg = end > (uint32_t)kBatch ? end - kBatch : 0u;
      const int nb = (int)(end - beg);
      __syncthreads();
      if (tid < nb) stage_splat(rec, __ldg(vals + s + beg + tid), st, tid);
      __syncthreads();
      // splats that can reach this warp's block and that some pixel of the
      // warp blended or skipped before stopping (list position < wmax)
      uint32_t hits[kBatch / 32];
#pragma unroll
      for (int k = 0; k < kBatch / 32; ++k) {
        const int j = 32 * k + lane;
        hits[k] = __ballot_sync(0xffffffffu, j < nb && beg + (uint32_t)j < wmax &&
                                                 block_may_hit(s_box[j], s_q[j], s_a[j].x, s_a[j].y, wx0, wx1, wy0, wy1));
      }
#pragma unroll
      for (int k = kBatch / 32 - 1; k >= 0; --k) {
       uint32_t m = hits[k];
       while (m) {
        const int bit = 31 - __clz(m);
        m &= ~(1u << bit);
        const int j = 32 * k + bit;
        const uint32_t pos = beg + (uint32_t)j;       // 0-based list position
        const float4 a = s_a[j], b = s_b[j];
        Hit h;
        bool act = false;
        float dmx = 0.f, dmy = 0.f, dca = 0.f, dcb = 0.f, dcc = 0.f, dop = 0.f, dr = 0.f, dg = 0.f, db = 0.f;
        const float4 c4 = s_c[j];
        if (pos < nc) {
          ++evals;
          act = splat_alpha(a, b, c4.z, px, py, h);
        }
        if (act) {
          const float cb_ = c4.x;
          const float om = __fsub_rn(1.f, h.alpha);
          const float inv = 1.f / om;
          const float Ti = T * inv;
          const float wT = h.alpha * Ti;
          const float da = g0 * (Ti * b.z - S0 * inv) + g1 * (Ti * b.w - S1 * inv) + g2 * (Ti * cb_ - S2 * inv);
          S0 = fmaf(wT, b.z, S0);
          S1 = fmaf(wT, b.w, S1);
          S2 = fmaf(wT, cb_, S2);
          T = Ti;
          dr = wT * g0;
          dg = wT * g1;
          db = wT * g2;
          if (!h.clamped) {
            // alpha = o 2^power, power = k q: dL/dq = -alpha dL/dalpha / 2
            dop = da * h.G;
            const float dq = -0.5f * h.alpha * da;
            const float dx = h.dx, dy = h.dy;
            dca = dq * dx * dx;
            dcb = dq * 2.f * dx * dy;
            dcc = dq * dy * dy;
            // dq/dm = -2 conic d = -(2 A dx + B dy, B dx + 2 C dy) / k
            const float s2 = dq * kInvExpScale;
            dmx = -s2 * (2.f * a.z * dx + a.w * dy);
            dmy = -s2 * (a.w * dx + 2.f * b.x * dy);
          }
        }
        if (__any_sync(0xffffffffu, act)) {
          const float v9[9] = {dmx, dmy, dca, dcb, dcc, dop, dr, dg, db};
          int idx;
          const float sum = warp_reduce_scatter9(v9, lane, &idx);
          if (idx >= 0) {
            const uint32_t pid = __float_as_uint(c4.y);
            atomicAdd(grad2d + (size_t)pid * kG2d + idx, sum);
          }
        }
       }
      }
      end = beg;
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if (lane == 0 && evals) atomicAdd(evals_out, evals);
}

}  // namespace

extern "C" pk_status pk_rasterize_bwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                                      const uint32_t *tile_ranges, const float *T_final, const uint32_t *n_contrib,
                                      const float *dL_dimage, float *grad2d, void *ws, pk_stream_t stream) {
  if (!p || !records || !sorted_vals || !tile_ranges || !T_final || !n_contrib || !dL_dimage || !grad2d || !ws)
    return PK_ERR_ARG;
  if (!aligned16(records) || !aligned16(grad2d)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevCounters *ctr = at<DevCounters>(ws, p->ws.counters);
  pk_device_status *status = at<pk_device_status>(ws, p->ws.status);
  if (cudaMemsetAsync(grad2d, 0, sizeof(float) * kG2d * (size_t)p->pairs, st) != cudaSuccess) return PK_ERR_CUDA;
  if (cudaMemsetAsync(&ctr->tile_queue[1], 0, sizeof(uint32_t), st) != cudaSuccess) return PK_ERR_CUDA;
  if (cudaMemsetAsync(&status->evals_bwd, 0, sizeof(uint64_t), st) != cudaSuccess) return PK_ERR_CUDA;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_bwd, kRasterThreads, 0);
  if (sms < 1) sms = 1;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > p->n_tiles) grid = p->n_tiles;
  if (grid < 1) grid = 1;
  k_raster_bwd<<<(int)grid, kRasterThreads, 0, st>>>(
      records, sorted_vals, tile_ranges, at<DevView>(ws, p->ws.views), at<uint32_t>(ws, p->ws.toff), p->V,
      (uint32_t)p->n_tiles, p->opts.bg[0], p->opts.bg[1], p->opts.bg[2], T_final, n_contrib, dL_dimage, grad2d,
      &ctr->tile_queue[1], reinterpret_cast<unsigned long long *>(&status->evals_bwd));
  return check_launch();
}
