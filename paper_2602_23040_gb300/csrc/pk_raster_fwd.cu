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
// computed from shared memory.  kPx: pixels per thread (Geo).
// At 2 pixels per thread the kernel is held to 48 registers (a few
// spilled) for 10 resident CTAs per SM instead of 9.
// kT: side of the tiles the lists were binned for (16 or 32); each CTA
// composites a 16 x 16 quadrant of one, walking the whole list of its tile
// (its warps' block tests skip what misses them), so a pixel still stops
// as soon as its own 16 x 16 block is done.
// With a target (not null) the epilogue also takes the L1 term of the
// objective: dL/dimage = sign(image - target) * scale and the sum of
// |image - target| (FP32 per thread, FP64 across warps) into loss_acc.
// kCount: count the (pixel, splat) evaluations into evals_out (a
// measurement; the variant without it carries no counter in its loop).
// clr (may be null): clr_n4 float4 set to zero along the way, clr_per of
// them per work item -- the backward's gradient records, cleared by stores
// that ride along with the compositing instead of a pass of their own.
template <int kBatch, bool kTma, int kPx, int kT, bool kCount>
__global__ __launch_bounds__(Geo<kPx>::kThreads, (kPx == 2 ? 10 : 1)) void k_raster_fwd(
    const float *__restrict__ rec, const uint32_t *__restrict__ vals, const uint64_t *__restrict__ ranges,
    const DevView *__restrict__ views, const uint32_t *__restrict__ toff, int V, uint32_t n_items, float bg0,
    float bg1, float bg2, float *__restrict__ image, float *__restrict__ Tout, uint32_t *__restrict__ ncontrib,
    uint32_t *queue, unsigned long long *evals_out, pk_device_status *status, const float *__restrict__ target,
    float *__restrict__ dimg, float scale, double *loss_acc, uint32_t first_polls, uint32_t npairs,
    float4 *__restrict__ clr, uint64_t clr_n4, uint64_t clr_per) {
  using G = Geo<kPx>;
  constexpr uint32_t kQuads = (kT / kTileSide) * (kT / kTileSide);   // CTAs per list tile
  __shared__ float4 s_a[kBatch], s_b[kBatch], s_c[kBatch], s_box[kBatch], s_q[kBatch];
  __shared__ __align__(16) float4 s_raw[kTma ? 3 * kBatch : 1];
  __shared__ uint32_t s_pid[kTma ? kBatch : 1];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tile;
  __shared__ int s_view;
  const int tid = threadIdx.x, lane = tid & 31;
  const Staged st{s_a, s_b, s_c, s_box, s_q};
  int ox, oy, bx, by;
  pixel_of<kPx>(tid, ox, oy, bx, by);
  uint32_t evals = 0;   // per thread: far below 2^32
  uint32_t phase = 0;
  bool timed_out = false;
  float lsum = 0.f;     // sum of |image - target| over this thread's pixels
  if (kTma) {
    if (tid == 0) {
      mbar_init(&s_bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
  }
  // bulk copies of the records of list entries [b, b + nb) into s_raw
  // (expect_tx is set by thread 0 before the block barrier that precedes this)
  auto fetch = [&](uint64_t b, int nb) {
    for (int j = tid; j < nb; j += G::kThreads) {
      const uint32_t pid = __ldg(vals + b + j);
      const bool named = pid < npairs;   // else record 0 is fetched in its place and not used
      s_pid[j] = named ? pid : kNoPair;
      tma_load_1d(&s_raw[3 * j], rec + (size_t)(named ? pid : 0u) * kRec, 3 * sizeof(float4), &s_bar);
    }
  };
  for (;;) {
    // work item: (list tile t, 16 x 16 quadrant q of it)
    if (tid == 0) {
      const uint32_t w = atomicAdd(queue, 1u);
      s_tile = w;
      s_view = w < n_items ? view_of_tile(toff, V, w / kQuads) : -1;
    }
    __syncthreads();
    const uint32_t w = s_tile;
    if (w >= n_items) break;
    if (clr) {   // this work item's share of the buffer to clear (every item takes one, so all of it is)
      const uint64_t c0 = (uint64_t)w * clr_per, c1 = min(clr_n4, c0 + clr_per);
      for (uint64_t i = c0 + tid; i < c1; i += G::kThreads) clr[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const uint32_t t = w / kQuads, q = w - t * kQuads;
    const DevView &view = views[s_view];
    const int W = view.width, H = view.height;
    const uint32_t local = t - (uint32_t)view.tile_off;
    const int ty = (int)(local / (uint32_t)view.tiles_x), tx = (int)(local - (uint32_t)ty * view.tiles_x);
    const int X0 = tx * kT + (int)(q % (kT / kTileSide)) * kTileSide;
    const int Y0 = ty * kT + (int)(q / (kT / kTileSide)) * kTileSide;
    if (X0 >= W || Y0 >= H) {   // a quadrant past the view's edge
      __syncthreads();
      continue;
    }
    const int x = X0 + ox, y0 = Y0 + oy;
    const float px = (float)x + 0.5f, py0 = (float)y0 + 0.5f;
    // pixel-centre bounds of this warp's block
    const float wx0 = (float)(X0 + bx) + 0.5f, wx1 = wx0 + (float)(G::kBW - 1);
    const float wy0 = (float)(Y0 + by) + 0.5f, wy1 = wy0 + (float)(G::kBH - 1);
    const uint64_t s = __ldg(ranges + 2 * (size_t)t), e = __ldg(ranges + 2 * (size_t)t + 1);
    float T[kPx], c0[kPx], c1[kPx], c2[kPx];
    uint32_t last[kPx];
    uint32_t live = 0;   // bit k: pixel k is inside the view and still compositing
#pragma unroll
    for (int k = 0; k < kPx; ++k) {
      T[k] = 1.f;
      c0[k] = c1[k] = c2[k] = 0.f;
      last[k] = 0;
      if (x < W && y0 + k * G::kRowStep < H) live |= 1u << k;
    }
    bool pending = false;   // a fetch is in flight (uniform over the block)
    if (kTma && s < e) {
      if (tid == 0) mbar_expect_tx(&s_bar, (uint32_t)min((uint64_t)kBatch, e - s) * 3u * sizeof(float4));
      __syncthreads();
      fetch(s, (int)min((uint64_t)kBatch, e - s));
      pending = true;
    }
    // plain loads: each thread's list entries of the next batch are read a
    // batch ahead, so staging waits for one load (the record) instead of two
    constexpr int kPer = (kBatch + G::kThreads - 1) / G::kThreads;
    uint32_t npid[kPer];
    if (!kTma) {
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int j = tid + u * G::kThreads;
        npid[u] = j < kBatch && s + j < e ? __ldg(vals + s + j) : 0u;
      }
    }
    for (uint64_t base = s; base < e; base += kBatch) {
      const int nb = (int)min((uint64_t)kBatch, e - base);
      if (kTma) {
        if (!mbar_wait_bounded(&s_bar, phase, first_polls)) {
          timed_out = true;
          mbar_wait_bounded(&s_bar, phase);   // let this batch's copies land before leaving
        }
        phase ^= 1u;
        pending = false;
#pragma unroll
        for (int j = tid; j < kBatch; j += G::kThreads)
          if (j < nb) {
            if (s_pid[j] == kNoPair) {
              stage_none(st, j);
              atomicOr(&status->flags, PK_DEV_BOUNDS);
            } else {
              stage_from(s_raw[3 * j], s_raw[3 * j + 1], s_raw[3 * j + 2], s_pid[j], st, j);
            }
          }
        fence_proxy_async();   // these reads of s_raw before the next bulk writes into it
        const uint64_t nxt = base + kBatch;
        const int nbn = nxt < e ? (int)min((uint64_t)kBatch, e - nxt) : 0;
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
        for (int u = 0; u < kPer; ++u) {
          const int j = tid + u * G::kThreads;
          if (j < nb) stage_splat(rec, npid[u], npairs, st, j, status);
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int j = tid + u * G::kThreads;
          const uint64_t nx = base + kBatch + (uint64_t)j;
          npid[u] = j < kBatch && nx < e ? __ldg(vals + nx) : 0u;
        }
        __syncthreads();
      }
      if (__any_sync(0xffffffffu, live != 0)) {
        // which staged splats can reach this warp's block: one ballot per
        // 32 splats, then only the hits are visited
        uint32_t hits[kBatch / 32];
#pragma unroll
        for (int k = 0; k < kBatch / 32; ++k) {
          const int j = 32 * k + lane;
          hits[k] = __ballot_sync(0xffffffffu, j < nb && block_may_hit(s_box[j], s_q[j], s_a[j].x, s_a[j].y,
                                                                       wx0, wx1, wy0, wy1));
        }
        bool any_live = true;
#pragma unroll
        for (int k = 0; k < kBatch / 32; ++k) {
          uint32_t m = hits[k];
          while (m && any_live) {
            const int j = 32 * k + __ffs(m) - 1;
            m &= m - 1;
            const float4 a = s_a[j], b = s_b[j], c = s_c[j];
            const float dx = __fsub_rn(px, a.x);
            const float zxdx = __fmul_rn(__fmul_rn(a.z, dx), dx), bdx = __fmul_rn(a.w, dx);
            const uint32_t pos1 = (uint32_t)(base - s) + (uint32_t)j + 1u;   // within the tile's list
            if (kCount) evals += __popc(live);   // evaluated at every live pixel of the thread
#pragma unroll
            for (int q = 0; q < kPx; ++q) {
              // one test per pixel: still compositing, and power >= pcut (both
              // q <= 9 and alpha >= 1/255); alpha = min(0.99, o 2^power)
              const float power = splat_power(a, b, bdx, zxdx, py0 + (float)(q * G::kRowStep));
              if (((live >> q) & 1u) && power >= c.z) {
                const float araw = __fmul_rn(-b.y, ex2_approx(power));   // staged opacity is negated
                const float alpha = araw > kAlphaMax ? kAlphaMax : araw;
                const float Tn = __fmul_rn(T[q], __fsub_rn(1.f, alpha));
                if (Tn < kTMin) {
                  live &= ~(1u << q);
                } else {
                  const float w = __fmul_rn(alpha, T[q]);
                  c0[q] = __fmaf_rn(w, b.z, c0[q]);
                  c1[q] = __fmaf_rn(w, b.w, c1[q]);
                  c2[q] = __fmaf_rn(w, c.x, c2[q]);
                  T[q] = Tn;
                  last[q] = pos1;
                }
              }
            }
            any_live = __any_sync(0xffffffffu, live != 0);
          }
        }
      }
      if (__syncthreads_count(live != 0) == 0) break;
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
#pragma unroll
    for (int q = 0; q < kPx; ++q) {
      const int y = y0 + q * G::kRowStep;
      if (x < W && y < H) {
        const size_t pix = (size_t)view.pix_off + (size_t)y * W + x;
        const size_t at0 = 3 * (size_t)view.pix_off + (size_t)y * W + x;
        const float v0 = __fmaf_rn(T[q], bg0, c0[q]), v1 = __fmaf_rn(T[q], bg1, c1[q]);
        const float v2 = __fmaf_rn(T[q], bg2, c2[q]);
        image[at0] = v0;
        image[at0 + plane] = v1;
        image[at0 + 2 * plane] = v2;
        Tout[pix] = T[q];
        ncontrib[pix] = last[q];
        if (target) {
          const float vs[3] = {v0, v1, v2};
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float d = vs[c] - __ldcs(target + at0 + c * plane);
            lsum += fabsf(d);
            __stcs(dimg + at0 + c * plane, d > 0.f ? scale : (d < 0.f ? -scale : 0.f));
          }
        }
      }
    }
    __syncthreads();   // everyone has read s_tile / s_view before the next fetch
  }
  // one atomic per warp for the evaluation counter (and the loss)
  if (kCount) {
    unsigned long long ev = evals;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if (lane == 0 && ev) atomicAdd(evals_out, ev);
  }
  if (target) {
    double dl = (double)lsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dl += __shfl_xor_sync(0xffffffffu, dl, o);
    if (lane == 0 && dl != 0.0) atomicAdd(loss_acc, dl);
  }
}

// One persistent launch: as many CTAs as fit on the GPU, at most one per tile.
template <int kBatch, bool kFwdTma, int kT, bool kCount>
pk_status launch_fwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                     const uint64_t *tile_ranges, float *image, float *T_final, uint32_t *n_contrib, void *ws,
                     DevCounters *ctr, pk_device_status *status, const float *target, float *dimg, float *clear,
                     uint64_t clear_floats, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_fwd<kBatch, kFwdTma, kFwdPx, kT, kCount>,
                                                Geo<kFwdPx>::kThreads, 0);
  if (sms < 1) sms = 1;
  if (per_sm < 1) per_sm = 1;
  const int64_t items = p->n_tiles * (kT / kTileSide) * (kT / kTileSide);
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > items) grid = items;
  if (grid < 1) grid = 1;
  const uint64_t clr_n4 = clear ? clear_floats / 4 : 0;
  const uint64_t clr_per = items > 0 ? (clr_n4 + (uint64_t)items - 1) / (uint64_t)items : 0;
  k_raster_fwd<kBatch, kFwdTma, kFwdPx, kT, kCount><<<(int)grid, Geo<kFwdPx>::kThreads, 0, st>>>(
      records, sorted_vals, tile_ranges, at<DevView>(ws, p->ws.views), at<uint32_t>(ws, p->ws.toff), p->V,
      (uint32_t)items, p->opts.bg[0], p->opts.bg[1], p->opts.bg[2], image, T_final, n_contrib,
      &ctr->tile_queue[0], reinterpret_cast<unsigned long long *>(&status->evals_fwd), status, target, dimg,
      (float)(1.0 / (3.0 * (double)std::max<int64_t>(1, p->P))), &ctr->loss_acc, p->first_polls, (uint32_t)p->pairs,
      reinterpret_cast<float4 *>(clr_n4 ? clear : nullptr), clr_n4, clr_per);
  return check_launch();
}

pk_status rasterize_fwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                        const uint64_t *tile_ranges, const float *target, float *image, float *T_final,
                        uint32_t *n_contrib, float *dimg, float *clear, uint64_t clear_floats, void *ws,
                        cudaStream_t st) {
  DevCounters *ctr = at<DevCounters>(ws, p->ws.counters);
  pk_device_status *status = at<pk_device_status>(ws, p->ws.status);
  // the tile queue, the evaluation counter and, with a target, loss_acc,
  // ssim_acc and ssim_lambda (0: the loss is L1 alone)
  pk_status ze = zero_async({{&ctr->tile_queue[0], sizeof(uint32_t)},
                             {&status->evals_fwd, sizeof(uint64_t)},
                             {&ctr->loss_acc, target ? 2 * sizeof(double) + sizeof(float) : 0}},
                            st);
  if (ze != PK_OK) return ze;
#define PK_FWD_T(B, M, C)                                                                                     \
  return p->T == 32 ? launch_fwd<B, M, 32, C>(p, records, sorted_vals, tile_ranges, image, T_final, n_contrib, \
                                              ws, ctr, status, target, dimg, clear, clear_floats, st)           \
                    : launch_fwd<B, M, 16, C>(p, records, sorted_vals, tile_ranges, image, T_final, n_contrib, \
                                              ws, ctr, status, target, dimg, clear, clear_floats, st)
#define PK_FWD(B, M)            \
  {                             \
    if (p->opts.count_evals) {  \
      PK_FWD_T(B, M, true);     \
    }                           \
    PK_FWD_T(B, M, false);      \
  }
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
#undef PK_FWD_T
}

}  // namespace

extern "C" pk_status pk_rasterize_fwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                                      const uint64_t *tile_ranges, float *image, float *T_final, uint32_t *n_contrib,
                                      void *ws, pk_stream_t stream) {
  if (!p || !records || !sorted_vals || !tile_ranges || !image || !T_final || !n_contrib || !ws) return PK_ERR_ARG;
  if (!aligned16(records) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7u)) return PK_ERR_ARG;
  return rasterize_fwd(p, records, sorted_vals, tile_ranges, nullptr, image, T_final, n_contrib, nullptr, nullptr, 0,
                       ws, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" pk_status pk_rasterize_fwd_l1(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                                         const uint64_t *tile_ranges, const float *target, float *image,
                                         float *T_final, uint32_t *n_contrib, float *dL_dimage, void *ws,
                                         pk_stream_t stream) {
  if (!p || !records || !sorted_vals || !tile_ranges || !target || !image || !T_final || !n_contrib ||
      !dL_dimage || !ws)
    return PK_ERR_ARG;
  if (!aligned16(records) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7u)) return PK_ERR_ARG;
  return rasterize_fwd(p, records, sorted_vals, tile_ranges, target, image, T_final, n_contrib, dL_dimage, nullptr,
                       0, ws, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" pk_status pk_rasterize_fwd_l1_clear(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                                               const uint64_t *tile_ranges, const float *target, float *image,
                                               float *T_final, uint32_t *n_contrib, float *dL_dimage,
                                               float *grad2d, void *ws, pk_stream_t stream) {
  if (!p || !records || !sorted_vals || !tile_ranges || !target || !image || !T_final || !n_contrib ||
      !dL_dimage || !grad2d || !ws)
    return PK_ERR_ARG;
  if (!aligned16(records) || !aligned16(grad2d) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7u))
    return PK_ERR_ARG;
  return rasterize_fwd(p, records, sorted_vals, tile_ranges, target, image, T_final, n_contrib, dL_dimage, grad2d,
                       (uint64_t)kG2d * (uint64_t)p->pairs, ws, reinterpret_cast<cudaStream_t>(stream));
}
