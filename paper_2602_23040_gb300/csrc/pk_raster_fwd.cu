// a4 -- front-to-back compositing (Supp. "Viewer": C = sum_i T_i a_i c_i,
// T_i = prod_{j<i} (1 - a_j)) over the depth-sorted list of each tile.
//
// One persistent launch covers the tiles of every view: each CTA takes the
// next tile from a device counter, stages the tile's splats batch by
// batch into shared memory and composites two pixels per thread.  Warps
// cover 8 x 8 pixel blocks and skip, as a whole, every splat whose
// contributing ellipse misses their block.  The CTA leaves a tile as soon
// as every pixel has stopped (transmittance cutoff) or the list ends.
#include "pk_raster.cuh"
#include "pk_tma.cuh"

using namespace pk;

namespace {

// kTma: the records of the next batch are fetched into shared memory by
// bulk copies (one 48-byte copy per splat, completed on an mbarrier) while
// the current batch is composited; the derived per-splat values are then
// computed from shared memory.
template <int kBatch, bool kTma>
__global__ __launch_bounds__(kRasterThreads) void k_raster_fwd(
    const float *__restrict__ rec, const uint32_t *__restrict__ vals, const uint32_t *__restrict__ ranges,
    const DevView *__restrict__ views, const uint32_t *__restrict__ toff, int V, uint32_t n_tiles, float bg0,
    float bg1, float bg2, float *__restrict__ image, float *__restrict__ Tout, uint32_t *__restrict__ ncontrib,
    uint32_t *queue, unsigned long long *evals_out, pk_device_status *status) {
  __shared__ float4 s_a[kBatch], s_b[kBatch], s_c[kBatch], s_box[kBatch], s_q[kBatch];
  __shared__ __align__(16) float4 s_raw[kTma ? 3 * kBatch : 1];
  __shared__ uint32_t s_pid[kTma ? kBatch : 1];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tile;
  __shared__ int s_view;
  const int tid = threadIdx.x, lane = tid & 31;
  const Staged st{s_a, s_b, s_c, s_box, s_q};
  int ox, oy;
  pixel_of(tid, ox, oy);
  uint32_t evals = 0;   // per thread: far below 2^32
  uint32_t phase = 0;
  bool timed_out = false;
  if (kTma) {
    if (tid == 0) {
      mbar_init(&s_bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  // bulk copies of the records of list entries [b, b + nb) into s_raw
  // (expect_tx is set by thread 0 before the block barrier that precedes this)
  auto fetch = [&](uint32_t b, int nb) {
    for (int j = tid; j < nb; j += kRasterThreads) {
      const uint32_t pid = __ldg(vals + b + j);
      s_pid[j] = pid;
      tma_load_1d(&s_raw[3 * j], rec + (size_t)pid * kRec, 3 * sizeof(float4), &s_bar);
    }
  };
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
    const int x = tx * kTileSide + ox, y0 = ty * kTileSide + oy, y1 = y0 + 4;
    const bool in0 = x < W && y0 < H, in1 = x < W && y1 < H;
    const float px = (float)x + 0.5f, py0 = (float)y0 + 0.5f, py1 = (float)y1 + 0.5f;
    // pixel-centre bounds of this warp's 8 x 8 block
    const float wx0 = (float)(tx * kTileSide + (ox & ~7)) + 0.5f, wx1 = wx0 + 7.f;
    const float wy0 = (float)(ty * kTileSide + (oy & ~7)) + 0.5f, wy1 = wy0 + 7.f;
    const uint32_t s = __ldg(ranges + 2 * (size_t)t), e = __ldg(ranges + 2 * (size_t)t + 1);
    float T0 = 1.f, T1 = 1.f, c00 = 0.f, c01 = 0.f, c02 = 0.f, c10 = 0.f, c11 = 0.f, c12 = 0.f;
    uint32_t last0 = 0, last1 = 0;
    bool done0 = !in0, done1 = !in1;
    bool pending = false;   // a fetch is in flight (uniform over the block)
    if (kTma && s < e) {
      if (tid == 0) mbar_expect_tx(&s_bar, (uint32_t)min((uint32_t)kBatch, e - s) * 3u * sizeof(float4));
      __syncthreads();
      fetch(s, (int)min((uint32_t)kBatch, e - s));
      pending = true;
    }
    for (uint32_t base = s; base < e; base += kBatch) {
      const int nb = (int)min((uint32_t)kBatch, e - base);
      if (kTma) {
        if (!mbar_wait_bounded(&s_bar, phase)) {
          timed_out = true;
          mbar_wait_bounded(&s_bar, phase);   // let this batch's copies land before leaving
        }
        phase ^= 1u;
        pending = false;
#pragma unroll
        for (int j = tid; j < kBatch; j += kRasterThreads)
          if (j < nb) stage_from(s_raw[3 * j], s_raw[3 * j + 1], s_raw[3 * j + 2], s_pid[j], st, j);
        fence_proxy_async();   // these reads of s_raw before the next bulk writes into it
        const uint32_t nxt = base + kBatch;
        const int nbn = nxt < e ? (int)min((uint32_t)kBatch, e - nxt) : 0;
        if (tid == 0 && nbn > 0) mbar_expect_tx(&s_bar, (uint32_t)nbn * 3u * sizeof(float4));
        if (__syncthreads_or(timed_out)) {
          timed_out = true;
          break;
        }
        if (nbn > 0) {
          fetch(nxt, nbn);
          pending = true;
        }
      } else {
        __syncthreads();
#pragma unroll
        for (int j = tid; j < kBatch; j += kRasterThreads)
          if (j < nb) stage_splat(rec, __ldg(vals + base + j), st, j);
        __syncthreads();
      }
      if (!__all_sync(0xffffffffu, done0 && done1)) {
        // which staged splats can reach this warp's block: 8 tests per lane,
        // one ballot per 32 splats, then only the hits are visited
        uint32_t hits[kBatch / 32];
#pragma unroll
        for (int k = 0; k < kBatch / 32; ++k) {
          const int j = 32 * k + lane;
          hits[k] = __ballot_sync(0xffffffffu, j < nb && block_may_hit(s_box[j], s_q[j], s_a[j].x, s_a[j].y,
                                                                       wx0, wx1, wy0, wy1));
        }
        bool all_done = false;
#pragma unroll
        for (int k = 0; k < kBatch / 32; ++k) {
          uint32_t m = hits[k];
          while (m && !all_done) {
            const int j = 32 * k + __ffs(m) - 1;
            m &= m - 1;
            const float4 a = s_a[j], b = s_b[j], c = s_c[j];
            const float dx = __fsub_rn(px, a.x), zx = __fmul_rn(a.z, dx);
            const uint32_t pos1 = base - s + (uint32_t)j + 1u;
            Hit h;
            if (!done0) {
              ++evals;
              if (splat_alpha(a, b, c.z, dx, zx, py0, h)) {
                const float Tn = __fmul_rn(T0, __fsub_rn(1.f, h.alpha));
                if (Tn < kTMin) {
                  done0 = true;
                } else {
                  const float w = __fmul_rn(h.alpha, T0);
                  c00 = __fmaf_rn(w, b.z, c00);
                  c01 = __fmaf_rn(w, b.w, c01);
                  c02 = __fmaf_rn(w, c.x, c02);
                  T0 = Tn;
                  last0 = pos1;
                }
              }
            }
            if (!done1) {
              ++evals;
              if (splat_alpha(a, b, c.z, dx, zx, py1, h)) {
                const float Tn = __fmul_rn(T1, __fsub_rn(1.f, h.alpha));
                if (Tn < kTMin) {
                  done1 = true;
                } else {
                  const float w = __fmul_rn(h.alpha, T1);
                  c10 = __fmaf_rn(w, b.z, c10);
                  c11 = __fmaf_rn(w, b.w, c11);
                  c12 = __fmaf_rn(w, c.x, c12);
                  T1 = Tn;
                  last1 = pos1;
                }
              }
            }
            all_done = __all_sync(0xffffffffu, done0 && done1);
          }
        }
      }
      if (__syncthreads_count(!(done0 && done1)) == 0) break;
    }
    if (kTma) {
      // a tile that stopped early may still have its next batch in flight
      if (pending) {
        if (!mbar_wait_bounded(&s_bar, phase)) {
          timed_out = true;
          mbar_wait_bounded(&s_bar, phase);
        }
        phase ^= 1u;
      }
      if (__syncthreads_or(timed_out)) {
        if (tid == 0) atomicOr(&status->flags, PK_DEV_TIMEOUT);
        break;
      }
    }
    const size_t plane = (size_t)W * H;
    if (in0) {
      const size_t pix = (size_t)view.pix_off + (size_t)y0 * W + x;
      float *img = image + 3 * (size_t)view.pix_off + (size_t)y0 * W + x;
      img[0] = __fmaf_rn(T0, bg0, c00);
      img[plane] = __fmaf_rn(T0, bg1, c01);
      img[2 * plane] = __fmaf_rn(T0, bg2, c02);
      Tout[pix] = T0;
      ncontrib[pix] = last0;
    }
    if (in1) {
      const size_t pix = (size_t)view.pix_off + (size_t)y1 * W + x;
      float *img = image + 3 * (size_t)view.pix_off + (size_t)y1 * W + x;
      img[0] = __fmaf_rn(T1, bg0, c10);
      img[plane] = __fmaf_rn(T1, bg1, c11);
      img[2 * plane] = __fmaf_rn(T1, bg2, c12);
      Tout[pix] = T1;
      ncontrib[pix] = last1;
    }
    __syncthreads();   // everyone has read s_tile / s_view before the next fetch
  }
  // one atomic per warp for the evaluation counter
  unsigned long long ev = evals;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
  if (lane == 0 && ev) atomicAdd(evals_out, ev);
}

// One persistent launch: as many CTAs as fit on the GPU, at most one per tile.
template <int kBatch, bool kFwdTma>
pk_status launch_fwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                     const uint32_t *tile_ranges, float *image, float *T_final, uint32_t *n_contrib, void *ws,
                     DevCounters *ctr, pk_device_status *status, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_fwd<kBatch, kFwdTma>, kRasterThreads, 0);
  if (sms < 1) sms = 1;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > p->n_tiles) grid = p->n_tiles;
  if (grid < 1) grid = 1;
  k_raster_fwd<kBatch, kFwdTma><<<(int)grid, kRasterThreads, 0, st>>>(
      records, sorted_vals, tile_ranges, at<DevView>(ws, p->ws.views), at<uint32_t>(ws, p->ws.toff), p->V,
      (uint32_t)p->n_tiles, p->opts.bg[0], p->opts.bg[1], p->opts.bg[2], image, T_final, n_contrib,
      &ctr->tile_queue[0], reinterpret_cast<unsigned long long *>(&status->evals_fwd), status);
  return check_launch();
}

}  // namespace

extern "C" pk_status pk_rasterize_fwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                                      const uint32_t *tile_ranges, float *image, float *T_final, uint32_t *n_contrib,
                                      void *ws, pk_stream_t stream) {
  if (!p || !records || !sorted_vals || !tile_ranges || !image || !T_final || !n_contrib || !ws) return PK_ERR_ARG;
  if (!aligned16(records)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevCounters *ctr = at<DevCounters>(ws, p->ws.counters);
  pk_device_status *status = at<pk_device_status>(ws, p->ws.status);
  if (cudaMemsetAsync(&ctr->tile_queue[0], 0, sizeof(uint32_t), st) != cudaSuccess) return PK_ERR_CUDA;
  if (cudaMemsetAsync(&status->evals_fwd, 0, sizeof(uint64_t), st) != cudaSuccess) return PK_ERR_CUDA;
#define PK_FWD(B, M) \
  return launch_fwd<B, M>(p, records, sorted_vals, tile_ranges, image, T_final, n_contrib, ws, ctr, status, st)
  const bool tma = p->opts.stage_fwd == PK_STAGE_BULK;
  switch (p->opts.batch) {
    case 64:
      if (tma) PK_FWD(64, true);
      PK_FWD(64, false);
    case 128:
      if (tma) PK_FWD(128, true);
      PK_FWD(128, false);
    default:
      if (tma) PK_FWD(256, true);
      PK_FWD(256, false);
  }
#undef PK_FWD
}
