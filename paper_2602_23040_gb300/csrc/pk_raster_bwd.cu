// a5 -- adjoint of the compositing (Sec. 4.2 "Objective").  Each pixel
// walks its tile's list backwards from its last blended splat, recovering
// T_i = T_{i+1} / (1 - alpha_i) from the stored final transmittance, so no
// per-step state of the forward is kept.  Each thread holds four pixels
// (two packed pairs); per splat the 9 gradients of a warp's 128 pixels are
// summed over the lanes (eight by a reduce-scatter, the ninth by a
// butterfly: 14 shuffles instead of 45 for nine full butterfly sums),
// after which nine lanes each hold one complete sum and add it to the
// splat's gradient record with one coalesced atomic instruction.
#include "pk_raster.cuh"
#include "pk_tma.cuh"

using namespace pk;

namespace {

// Sum over the 32 lanes of nine values per lane, eight of them by a
// reduce-scatter and the ninth by a plain butterfly: xor-16 splits v[0..7]
// 4 | 4, xor-8 each half 2 | 2, xor-4 1 | 1 (one select pair, shuffle and
// add per value and level), then xor-2 and xor-1 add the last value
// outright.  Lane l then holds the complete sum of v[4 (l & 16) / 16 + 2
// (l & 8) / 8 + (l & 4) / 4] in *s8 and every lane the sum of v[8] in *s9
// -- 9 + 5 shuffles and 14 selects, against 12 shuffles and 24 selects for
// a reduce-scatter of all nine.
__device__ __forceinline__ int reduce_scatter8_index(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

__device__ __forceinline__ void warp_reduce_9(const float (&v)[9], int lane, float &s8, float &s9) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float lo = v[j], hi = v[4 + j];
    const float r = __shfl_xor_sync(0xffffffffu, b4 ? lo : hi, 16);
    w[j] = (b4 ? hi : lo) + r;
  }
  float x[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float lo = w[j], hi = w[2 + j];
    const float r = __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 8);
    x[j] = (b3 ? hi : lo) + r;
  }
  float z;
  {
    const float r = __shfl_xor_sync(0xffffffffu, b2 ? x[0] : x[1], 4);
    z = (b2 ? x[1] : x[0]) + r;
  }
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  s8 = z;
  float t = v[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  s9 = t;
}

// Per-splat sums of a thread's pixels, kept as two packed lanes (the two
// pixels of a pair) and added lane to lane once per splat.
struct AdjSums {
  f32x2 a5, a6, a7, a8, q1, qy, qyy;
};

// Two pixels' shares of the adjoint of a blended splat, pixels h and h + 1
// of a thread side by side in the packed FP32 lanes, from their exponents
// pw and row offsets dy (splat_power2); ok0 / ok1: the pixel blended or
// skipped this splat in the forward and passes its footprint test.  Per pixel, T
// (transmittance after the splat) becomes T before it; GS = dL/dC . S, S
// being the colour composited behind (background included), takes the
// splat's own term (only that dot product enters dL/dalpha); the colour and
// opacity gradients go to the sums a5..a8.  The conic and mean gradients
// are linear in dq = dL/dq, so a pixel only adds dq, dq dy and dq dy^2 to
// q1, qy, qyy (dx is common to a thread's pixels) and the caller forms them
// once per splat.  A pixel that skips the splat (ok false: outside the
// footprint, or past its last blended entry) takes alpha 0, which leaves
// its T and GS unchanged and adds 0 to every sum, so the pair runs without
// a branch.  GS is kept negated (NGS = -dL/dC . S) and alpha as nal =
// -alpha (the staged opacity is negated), which turns dL/dalpha into one
// fused multiply-add.  kFirst: this pair starts the sums instead of adding
// to them.
template <bool kFirst>
__device__ __forceinline__ void pixel_adjoint2(const float4 &a, const float4 &b, const float4 &c4, f32x2 pw, f32x2 dy,
                                               bool ok0, bool ok1, f32x2 g0, f32x2 g1, f32x2 g2, float &T0,
                                               float &T1, float &NGS0, float &NGS1, AdjSums &s) {
  float p0, p1;
  unpack2(pw, p0, p1);
  // power <= 0 for the positive-definite conics of pk_project_and_sh: G in
  // [0, 1] at every pixel, and a skipping pixel's zero alpha zeroes its terms
  const float G0 = ex2_approx(p0), G1 = ex2_approx(p1);
  // 1 + nal, nal Ti and the sums below are exactly the negations of the
  // alpha forms
  float r0, r1;
  unpack2(mul2(dup2(b.y), pack2(G0, G1)), r0, r1);
  const bool cl0 = r0 < -kAlphaMax, cl1 = r1 < -kAlphaMax;
  const float nal0 = ok0 ? (cl0 ? -kAlphaMax : r0) : 0.f;
  const float nal1 = ok1 ? (cl1 ? -kAlphaMax : r1) : 0.f;
  const f32x2 nal = pack2(nal0, nal1);
  float om0, om1;
  unpack2(add2(dup2(1.f), nal), om0, om1);
  const f32x2 inv = pack2(rcp_approx(om0), rcp_approx(om1));
  const f32x2 Tv = pack2(T0, T1);
  float ti0, ti1;
  const f32x2 Ti = mul2(Tv, inv);
  unpack2(Ti, ti0, ti1);
  const f32x2 nwT = mul2(nal, Ti);
  // dL/dalpha = (T g.rgb - g.S) / (1 - alpha), with NGS = -g.S
  const f32x2 gr = fma2(g2, dup2(c4.x), fma2(g1, dup2(b.w), mul2(g0, dup2(b.z))));
  const f32x2 NGSv = pack2(NGS0, NGS1);
  float da0, da1;
  unpack2(mul2(fma2(Tv, gr, NGSv), inv), da0, da1);
  unpack2(fma2(nwT, gr, NGSv), NGS0, NGS1);
  // a skipping pixel has alpha 0: 1 / (1 - 0) = 1 exactly, T stays
  T0 = ti0;
  T1 = ti1;
  // the first pair of a thread starts the sums, the others add to them
  s.a6 = kFirst ? mul2(nwT, g0) : fma2(nwT, g0, s.a6);
  s.a7 = kFirst ? mul2(nwT, g1) : fma2(nwT, g1, s.a7);
  s.a8 = kFirst ? mul2(nwT, g2) : fma2(nwT, g2, s.a8);
  // alpha = o 2^power, power = k q: dL/dq = -alpha dL/dalpha / 2 (unclamped pixels only)
  const f32x2 dav = pack2(ok0 && !cl0 ? da0 : 0.f, ok1 && !cl1 ? da1 : 0.f);
  s.a5 = kFirst ? mul2(dav, pack2(G0, G1)) : fma2(dav, pack2(G0, G1), s.a5);
  const f32x2 dq = mul2(mul2(dup2(0.5f), nal), dav);
  const f32x2 t = mul2(dq, dy);
  s.q1 = kFirst ? dq : add2(s.q1, dq);
  s.qy = kFirst ? t : add2(s.qy, t);
  s.qyy = kFirst ? mul2(t, dy) : fma2(t, dy, s.qyy);
}

__device__ __forceinline__ float lane_sum(f32x2 v) {
  float lo, hi;
  unpack2(v, lo, hi);
  return lo + hi;
}

// Conic and mean gradients of a splat from the pixel sums q1 = sum dq,
// qy = sum dq dy, qyy = sum dq dy^2 (common dx): d/dconic = dq (dx^2,
// 2 dx dy, dy^2), dq/dm = -2 conic d = -(2 A dx + B dy, B dx + 2 C dy) / k.
__device__ __forceinline__ void conic_mean_grads(const float4 &a, const float4 &b, float dx, float q1, float qy,
                                                 float qyy, float (&acc)[9]) {
  const float dq1 = dx * q1;
  acc[2] = dx * dq1;
  acc[3] = 2.f * dx * qy;
  acc[4] = qyy;
  acc[0] = -kInvExpScale * (2.f * a.z * dq1 + a.w * qy);
  acc[1] = -kInvExpScale * (a.w * dq1 + 2.f * b.x * qy);
}

// kTma: the records of the next (earlier) batch are fetched into shared
// memory by bulk copies (one 48-byte copy per splat, completed on an
// mbarrier) while the current batch is processed.  kPx: pixels per thread.
// At 4 pixels per thread the kernel is held to 64 registers (no spills) for
// 16 resident CTAs per SM (72 registers and 14 CTAs: 1 % slower).
// kT: side of the tiles the lists were binned for; each CTA takes a 16 x 16
// quadrant of one, as in the forward.  kCount: count the evaluations (a
// measurement; the variant without it carries no counter in its loop).
template <int kBatch, bool kTma, int kPx, int kT, bool kCount>
__global__ __launch_bounds__(Geo<kPx>::kThreads, (kPx == 4 ? 16 : 1)) void k_raster_bwd(
    const float *__restrict__ rec, const uint32_t *__restrict__ vals, const uint64_t *__restrict__ ranges,
    const DevView *__restrict__ views, const uint32_t *__restrict__ toff, int V, uint32_t n_items, float bg0,
    float bg1, float bg2, const float *__restrict__ Tfin, const uint32_t *__restrict__ ncontrib,
    const float *__restrict__ dimg, float *__restrict__ grad2d, uint32_t *queue, unsigned long long *evals_out,
    pk_device_status *status, uint32_t first_polls, uint32_t npairs) {
  using G = Geo<kPx>;
  constexpr uint32_t kQuads = (kT / kTileSide) * (kT / kTileSide);   // CTAs per list tile
  __shared__ float4 s_a[kBatch], s_b[kBatch], s_c[kBatch], s_box[kBatch], s_q[kBatch];
  __shared__ __align__(16) float4 s_raw[kTma ? 3 * kBatch : 1];
  __shared__ uint32_t s_pid[kTma ? kBatch : 1];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_tile;
  __shared__ int s_view;
  __shared__ uint32_t s_wmax[G::kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Staged st{s_a, s_b, s_c, s_box, s_q};
  int ox, oy, bx, by;
  pixel_of<kPx>(tid, ox, oy, bx, by);
  // the lane that adds each of the nine sums: lanes 0, 4, ..., 28 the
  // scattered eight, lane 1 the ninth (-1: none)
  const int my_idx = (lane & 3) == 0 ? reduce_scatter8_index(lane) : (lane == 1 ? 8 : -1);
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
    const float wx0 = (float)(X0 + bx) + 0.5f, wx1 = wx0 + (float)(G::kBW - 1);
    const float wy0 = (float)(Y0 + by) + 0.5f, wy1 = wy0 + (float)(G::kBH - 1);
    // list start, and its length (one tile's list names each of its
    // view's pairs at most once: below 2^32)
    const uint64_t s = __ldg(ranges + 2 * (size_t)t);
    const uint32_t len = (uint32_t)(__ldg(ranges + 2 * (size_t)t + 1) - s);
    const size_t plane = (size_t)W * H;
    float T[kPx], NGS[kPx], g0[kPx], g1[kPx], g2[kPx], pyq[kPx];
    uint32_t nc[kPx];
    uint32_t ncmax = 0;
#pragma unroll
    for (int q = 0; q < kPx; ++q) {
      const int y = y0 + q * G::kRowStep;
      pyq[q] = py0 + (float)(q * G::kRowStep);
      T[q] = 1.f;
      g0[q] = g1[q] = g2[q] = 0.f;
      nc[q] = 0;
      if (x < W && y < H) {
        const size_t pix = (size_t)view.pix_off + (size_t)y * W + x;
        const float *gi = dimg + 3 * (size_t)view.pix_off + (size_t)y * W + x;
        T[q] = Tfin[pix];
        // a count past the tile's list (n_contrib not written by the forward
        // of these lists) reads no entry beyond it
        nc[q] = min(ncontrib[pix], len);
        g0[q] = gi[0];
        g1[q] = gi[plane];
        g2[q] = gi[2 * plane];
      }
      // -dL/dC . (colour composited behind the current splat, background included)
      NGS[q] = -(T[q] * fmaf(g2[q], bg2, fmaf(g1[q], bg1, g0[q] * bg0)));
      ncmax = max(ncmax, nc[q]);
    }
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, ncmax);
    if (lane == 0) s_wmax[warp] = wmax;
    __syncthreads();
    uint32_t tmax = 0;
#pragma unroll
    for (int w = 0; w < G::kWarps; ++w) tmax = max(tmax, s_wmax[w]);
    if (kTma && tmax > 0) {
      const uint32_t b0 = tmax > (uint32_t)kBatch ? tmax - kBatch : 0u;
      if (tid == 0) mbar_expect_tx(&s_bar, (tmax - b0) * 3u * (uint32_t)sizeof(float4));
      __syncthreads();
      fetch(s + b0, (int)(tmax - b0));
    }
    // plain loads: each thread's list entries of the next (earlier) batch
    // are read a batch ahead, so staging waits for one load (the record)
    // instead of two
    constexpr int kPer = (kBatch + G::kThreads - 1) / G::kThreads;
    uint32_t npid[kPer];
    if (!kTma) {
      const uint32_t b0 = tmax > (uint32_t)kBatch ? tmax - kBatch : 0u;
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int j = tid + u * G::kThreads;
        npid[u] = j < kBatch && b0 + (uint32_t)j < tmax ? __ldg(vals + s + b0 + j) : 0u;
      }
    }
    for (uint32_t end = tmax; end > 0;) {
      const uint32_t beg = end > (uint32_t)kBatch ? end - kBatch : 0u;
      const int nb = (int)(end - beg);
      if (kTma) {
        if (!mbar_wait_bounded(&s_bar, phase, first_polls)) {
          timed_out = true;
          mbar_wait_bounded(&s_bar, phase);   // let this batch's copies land before leaving
        }
        phase ^= 1u;
        __syncthreads();   // every warp is done with the previous batch's staged values
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
        const uint32_t nbeg = beg > (uint32_t)kBatch ? beg - kBatch : 0u;
        if (tid == 0 && beg > 0) mbar_expect_tx(&s_bar, (beg - nbeg) * 3u * (uint32_t)sizeof(float4));
        if (__syncthreads_or(timed_out)) {
          timed_out = true;
          break;
        }
        if (beg > 0) fetch(s + nbeg, (int)(beg - nbeg));
      } else {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int j = tid + u * G::kThreads;
          if (j < nb) stage_splat(rec, npid[u], npairs, st, j, status);
        }
        const uint32_t nbeg = beg > (uint32_t)kBatch ? beg - kBatch : 0u;
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int j = tid + u * G::kThreads;
          npid[u] = j < kBatch && nbeg + (uint32_t)j < beg ? __ldg(vals + s + nbeg + j) : 0u;
        }
        __syncthreads();
      }
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
          const uint32_t pos = beg + (uint32_t)j;   // 0-based list position
          const float4 a = s_a[j], b = s_b[j], c4 = s_c[j];
          const float dx = __fsub_rn(px, a.x);
          const float zxdx = __fmul_rn(__fmul_rn(a.z, dx), dx), bdx = __fmul_rn(a.w, dx);
          // the exponent at the thread's pixels, and which of them blended
          // or skipped this splat in the forward and pass its footprint
          // test; a splat that no pixel of the warp takes is left at once
          f32x2 pw[kPx / 2], dyv[kPx / 2];
          bool ok[kPx];
          bool any = false;
#pragma unroll
          for (int h = 0; h < kPx; h += 2) {
            const bool e0 = pos < nc[h], e1 = pos < nc[h + 1];
            if (kCount) evals += (uint32_t)e0 + (uint32_t)e1;
            pw[h / 2] = splat_power2(a, b, bdx, zxdx, pack2(pyq[h], pyq[h + 1]), dyv[h / 2]);
            float p0, p1;
            unpack2(pw[h / 2], p0, p1);
            ok[h] = e0 && p0 >= c4.z;
            ok[h + 1] = e1 && p1 >= c4.z;
            any = any || ok[h] || ok[h + 1];
          }
          if (!__any_sync(0xffffffffu, any)) continue;
          AdjSums sums;   // started by the first pair
#pragma unroll
          for (int h = 0; h < kPx; h += 2) {
            if (h == 0)
              pixel_adjoint2<true>(a, b, c4, pw[h / 2], dyv[h / 2], ok[h], ok[h + 1], pack2(g0[h], g0[h + 1]),
                                   pack2(g1[h], g1[h + 1]), pack2(g2[h], g2[h + 1]), T[h], T[h + 1], NGS[h],
                                   NGS[h + 1], sums);
            else
              pixel_adjoint2<false>(a, b, c4, pw[h / 2], dyv[h / 2], ok[h], ok[h + 1], pack2(g0[h], g0[h + 1]),
                                    pack2(g1[h], g1[h + 1]), pack2(g2[h], g2[h + 1]), T[h], T[h + 1], NGS[h],
                                    NGS[h + 1], sums);
          }
          {
            float acc[9];
            acc[5] = lane_sum(sums.a5);
            acc[6] = -lane_sum(sums.a6);   // the colour sums hold -alpha T dL/dC
            acc[7] = -lane_sum(sums.a7);
            acc[8] = -lane_sum(sums.a8);
            conic_mean_grads(a, b, dx, lane_sum(sums.q1), lane_sum(sums.qy), lane_sum(sums.qyy), acc);
            float s8, s9;
            warp_reduce_9(acc, lane, s8, s9);
            if (my_idx >= 0) atomicAdd(grad2d + (size_t)__float_as_uint(c4.y) * kG2d + my_idx, lane == 1 ? s9 : s8);
          }
        }
      }
      end = beg;
    }
    if (kTma && timed_out) {
      if (tid == 0) atomicOr(&status->flags, PK_DEV_TIMEOUT);
      break;
    }
    __syncthreads();
  }
  if (kCount) {
    unsigned long long ev = evals;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if (lane == 0 && ev) atomicAdd(evals_out, ev);
  }
}

// One persistent launch: as many CTAs as fit on the GPU, at most one per tile.
template <int kBatch, bool kBwdTma, int kT, bool kCount>
pk_status launch_bwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                     const uint64_t *tile_ranges, const float *T_final, const uint32_t *n_contrib,
                     const float *dL_dimage, float *grad2d, void *ws, DevCounters *ctr, pk_device_status *status,
                     cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_bwd<kBatch, kBwdTma, kBwdPx, kT, kCount>,
                                                Geo<kBwdPx>::kThreads, 0);
  if (sms < 1) sms = 1;
  if (per_sm < 1) per_sm = 1;
  const int64_t items = p->n_tiles * (kT / kTileSide) * (kT / kTileSide);
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > items) grid = items;
  if (grid < 1) grid = 1;
  k_raster_bwd<kBatch, kBwdTma, kBwdPx, kT, kCount><<<(int)grid, Geo<kBwdPx>::kThreads, 0, st>>>(
      records, sorted_vals, tile_ranges, at<DevView>(ws, p->ws.views), at<uint32_t>(ws, p->ws.toff), p->V,
      (uint32_t)items, p->opts.bg[0], p->opts.bg[1], p->opts.bg[2], T_final, n_contrib, dL_dimage, grad2d,
      &ctr->tile_queue[1], reinterpret_cast<unsigned long long *>(&status->evals_bwd), status, p->first_polls, (uint32_t)p->pairs);
  return check_launch();
}

}  // namespace

namespace {

// zero_grad2d: clear the gradient records first (pk_rasterize_bwd), or add
// to what they hold (pk_rasterize_bwd_accumulate).
pk_status rasterize_bwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                        const uint64_t *tile_ranges, const float *T_final, const uint32_t *n_contrib,
                        const float *dL_dimage, float *grad2d, void *ws, bool zero_grad2d, cudaStream_t st) {
  if (!p || !records || !sorted_vals || !tile_ranges || !T_final || !n_contrib || !dL_dimage || !grad2d || !ws)
    return PK_ERR_ARG;
  if (!aligned16(records) || !aligned16(grad2d) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7u))
    return PK_ERR_ARG;
  DevCounters *ctr = at<DevCounters>(ws, p->ws.counters);
  pk_device_status *status = at<pk_device_status>(ws, p->ws.status);
  pk_status ze = zero_async({{grad2d, zero_grad2d ? sizeof(float) * kG2d * (size_t)p->pairs : 0},
                             {&ctr->tile_queue[1], sizeof(uint32_t)},
                             {&status->evals_bwd, sizeof(uint64_t)}},
                            st);
  if (ze != PK_OK) return ze;
#define PK_BWD_T(B, M, C)                                                                                   \
  return p->T == 32 ? launch_bwd<B, M, 32, C>(p, records, sorted_vals, tile_ranges, T_final, n_contrib,       \
                                              dL_dimage, grad2d, ws, ctr, status, st)                         \
                    : launch_bwd<B, M, 16, C>(p, records, sorted_vals, tile_ranges, T_final, n_contrib,       \
                                              dL_dimage, grad2d, ws, ctr, status, st)
#define PK_BWD(B, M)            \
  {                             \
    if (p->opts.count_evals) {  \
      PK_BWD_T(B, M, true);     \
    }                           \
    PK_BWD_T(B, M, false);      \
  }
  const bool tma = p->opts.stage_bwd == PK_STAGE_BULK;
  switch (p->opts.batch_bwd) {
    case 64:
      if (tma) PK_BWD(64, true);
      PK_BWD(64, false);
    case 128:
      if (tma) PK_BWD(128, true);
      PK_BWD(128, false);
    default:
      if (tma) PK_BWD(256, true);
      PK_BWD(256, false);
  }
#undef PK_BWD
#undef PK_BWD_T
}

}  // namespace

extern "C" pk_status pk_rasterize_bwd(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                                      const uint64_t *tile_ranges, const float *T_final, const uint32_t *n_contrib,
                                      const float *dL_dimage, float *grad2d, void *ws, pk_stream_t stream) {
  return rasterize_bwd(p, records, sorted_vals, tile_ranges, T_final, n_contrib, dL_dimage, grad2d, ws, true,
                       reinterpret_cast<cudaStream_t>(stream));
}

extern "C" pk_status pk_rasterize_bwd_accumulate(const pk_plan *p, const float *records, const uint32_t *sorted_vals,
                                                 const uint64_t *tile_ranges, const float *T_final,
                                                 const uint32_t *n_contrib, const float *dL_dimage, float *grad2d,
                                                 void *ws, pk_stream_t stream) {
  return rasterize_bwd(p, records, sorted_vals, tile_ranges, T_final, n_contrib, dL_dimage, grad2d, ws, false,
                       reinterpret_cast<cudaStream_t>(stream));
}
