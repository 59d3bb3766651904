// Motion masks and the covariance-aware dynamic mask (Sec. 4.2 "Optical
// Flow and Binary Motion Masks", "Covariance-Aware Gaussian Masking",
// Alg. 1).
//
// Motion masks are bit rows (32 pixels per word, the layout of the atlas
// occupancy mask) for every view at once: a threshold kernel (a warp per
// four mask words, coalesced flow reads, one ballot per word) and a separable
// square dilation, a horizontal pass on 64-bit word pairs with logarithmic
// bit smearing and a vertical pass of (2r + 1) coalesced word loads.
//
// The dynamic mask takes one lane per Gaussian; a warp visits the views in
// order and a Gaussian stops at its first hit, so the OR over cameras
// happens on the device and a dynamic Gaussian usually costs one view.
// Per view the pair's projected record gives mean, conic and radius; a
// block mask (one bit per 32 x 32 pixels) rules out most pairs on the
// lane that owns them, and the rest are scanned by the whole warp, one
// row per lane: the word mask skips motion-free 32-pixel runs, and only
// pixels whose mask bit is set are tested against the ellipse.
#include "pk_common.cuh"

using namespace pk;

namespace {

constexpr int kMaskThreads = 256;

// One warp per 4 consecutive mask words (loads of all four in flight before
// the ballots): bit `lane` of word (view, y, wx) is pixel x = 32 wx + lane
// of row y.
constexpr int kWordsPerWarp = 4;
__global__ __launch_bounds__(kMaskThreads) void k_motion_threshold(const float *__restrict__ flow,
                                                                    const DevView *__restrict__ views, float tau,
                                                                    uint32_t *__restrict__ bits) {
  const DevView &view = views[blockIdx.y];
  const int W = view.width, H = view.height, wpr = (W + 31) >> 5;
  const int64_t nwords = (int64_t)H * wpr, plane = (int64_t)W * H;
  const int64_t wbase = (((int64_t)blockIdx.x * kMaskThreads + threadIdx.x) >> 5) * kWordsPerWarp;
  const int lane = threadIdx.x & 31;
  if (wbase >= nwords) return;   // uniform over the warp
  const float *f = flow + 2 * view.pix_off;
  float fx[kWordsPerWarp], fy[kWordsPerWarp];
  bool in[kWordsPerWarp];
#pragma unroll
  for (int k = 0; k < kWordsPerWarp; ++k) {
    const int64_t w = wbase + k;
    const int y = (int)(w / wpr), x = 32 * (int)(w - (int64_t)y * wpr) + lane;
    in[k] = w < nwords && x < W;
    const int64_t i = (int64_t)y * W + x;
    fx[k] = in[k] ? __ldg(f + i) : 0.0f;
    fy[k] = in[k] ? __ldg(f + plane + i) : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < kWordsPerWarp; ++k) {
    const bool on = in[k] && __fsqrt_rn(__fadd_rn(__fmul_rn(fx[k], fx[k]), __fmul_rn(fy[k], fy[k]))) > tau;
    const uint32_t word = __ballot_sync(0xffffffffu, on);
    if (lane == 0 && wbase + k < nwords) bits[view.mask_off + wbase + k] = word;
  }
}

// OR of v >> k over k = 0 .. n (0 <= n < 64): v covers [0, m], a shift by
// m + 1 doubles the cover, a last shift by n - m <= m + 1 closes the gap.
__device__ __forceinline__ uint64_t smear_right(uint64_t v, int n) {
  int m = 0;
  while (2 * m + 1 <= n) {
    v |= v >> (m + 1);
    m = 2 * m + 1;
  }
  if (m < n) v |= v >> (n - m);
  return v;
}

// Horizontal dilation: output bit x is set iff a source bit lies in
// [x - r, x + r].  The source bit offsets sb = 32 wx + s, s in [-r, r],
// are taken in runs that share one pair of source words.
__global__ __launch_bounds__(kMaskThreads) void k_dilate_rows(const uint32_t *__restrict__ src,
                                                               const DevView *__restrict__ views, int r,
                                                               uint32_t *__restrict__ dst) {
  const DevView &view = views[blockIdx.y];
  const int W = view.width, H = view.height, wpr = (W + 31) >> 5;
  const int64_t w = (int64_t)blockIdx.x * kMaskThreads + threadIdx.x;
  if (w >= (int64_t)H * wpr) return;
  const int y = (int)(w / wpr), wx = (int)(w - (int64_t)y * wpr);
  const uint32_t *row = src + view.mask_off + (int64_t)y * wpr;
  auto word = [&](int64_t j) -> uint32_t { return (j >= 0 && j < wpr) ? __ldg(row + j) : 0u; };
  uint32_t out = 0;
  const int64_t sb1 = 32 * (int64_t)wx + r;
  for (int64_t sb = 32 * (int64_t)wx - r; sb <= sb1;) {
    const int64_t j = sb >= 0 ? sb >> 5 : -((31 - sb) >> 5);   // floor(sb / 32)
    const int64_t end = min(sb1, 32 * j + 31);
    const uint64_t v = ((uint64_t)word(j + 1) << 32) | word(j);
    const int o0 = (int)(sb - 32 * j), n = (int)(end - sb);
    out |= (uint32_t)smear_right(v >> o0, n);
    sb = end + 1;
  }
  if (wx == wpr - 1 && (W & 31)) out &= (1u << (W & 31)) - 1u;
  dst[view.mask_off + w] = out;
}

// Vertical dilation: OR of the words of rows y - r .. y + r (inside the image).
__global__ __launch_bounds__(kMaskThreads) void k_dilate_cols(const uint32_t *__restrict__ src,
                                                               const DevView *__restrict__ views, int r,
                                                               uint32_t *__restrict__ dst) {
  const DevView &view = views[blockIdx.y];
  const int W = view.width, H = view.height, wpr = (W + 31) >> 5;
  const int64_t w = (int64_t)blockIdx.x * kMaskThreads + threadIdx.x;
  if (w >= (int64_t)H * wpr) return;
  const int y = (int)(w / wpr), wx = (int)(w - (int64_t)y * wpr);
  const uint32_t *col = src + view.mask_off + wx;
  const int y0 = max(0, y - r), y1 = min(H - 1, y + r);
  uint32_t out = 0;
  for (int yy = y0; yy <= y1; ++yy) out |= __ldg(col + (int64_t)yy * wpr);
  dst[view.mask_off + w] = out;
}

// Block mask: bit wx & 31 of word (cy, wx >> 5) is set iff the 32 x 32
// pixel block of mask rows 32 cy .. 32 cy + 31 and word column wx holds a
// moving pixel.  One warp per block-mask word, lane = word column.
__global__ __launch_bounds__(kMaskThreads) void k_mask_coarse(const uint32_t *__restrict__ mask,
                                                               const DevView *__restrict__ views,
                                                               uint32_t *__restrict__ coarse) {
  const DevView &view = views[blockIdx.y];
  const int W = view.width, H = view.height, wpr = (W + 31) >> 5;
  const int cpr = (wpr + 31) >> 5, ch = (H + 31) >> 5;
  const int64_t w = ((int64_t)blockIdx.x * kMaskThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)ch * cpr) return;   // uniform over the warp
  const int cy = (int)(w / cpr), cx = (int)(w - (int64_t)cy * cpr);
  const int wx = 32 * cx + lane;
  uint32_t any = 0;
  if (wx < wpr) {
    const uint32_t *col = mask + view.mask_off + wx;
    const int y1 = min(H, 32 * cy + 32);
    for (int y = 32 * cy; y < y1; ++y) any |= __ldg(col + (int64_t)y * wpr);
  }
  const uint32_t word = __ballot_sync(0xffffffffu, any != 0u);
  if (lane == 0) coarse[view.coarse_off + w] = word;
}

// Does the ellipse q <= 9 of a pair cover a moving pixel of its rectangle
// [x0, x1] x [y0, y1]?  Called by a whole warp with the same pair: lane l
// takes rows y0 + l, y0 + l + 32, ...; per row a conservative filter keeps
// the x interval of {q <= 9} (widened far beyond FP32 error: it never
// decides a pixel, it only skips ones that cannot pass), the block mask
// skips 32-pixel words of blocks without motion, the word mask pixels
// without motion, and each moving pixel left takes the decision: d^2 in
// FP32 without fused multiply-adds, in the order stated in packuv.h.
__device__ bool warp_pair_hits(float mx, float my, float a, float b, float c, int x0, int x1, int y0, int y1, int W,
                               int wpr, int cpr, const uint32_t *__restrict__ vmask,
                               const uint32_t *__restrict__ vcoarse, int lane) {
  const float ax = __fsub_rn(mx, 0.5f);
  const float det = a * c - b * b;
  const bool filt = a > 0.0f && c > 0.0f && det > 0.0f && isfinite(det);
  const float b2 = __fmul_rn(2.0f, b);
  const float ra = filt ? 1.0f / a : 0.0f, pad = filt ? 9e-4f * a : 0.0f;
  for (int yb = y0; yb <= y1; yb += 32) {
    const int y = yb + lane;
    bool h = false;
    if (y <= y1) {
      const uint32_t *crow = vcoarse + (int64_t)(y >> 5) * cpr;
      const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), my);
      int xa = x0, xb = x1;
      if (filt) {
        const float disc = 9.0f * a - dy * dy * det;
        const float half = sqrtf(fmaxf(disc, 0.0f) + pad) * ra + 1.0f;
        const float xc = ax - b * dy * ra;
        xa = max(xa, (int)fmaxf(ceilf(xc - half), 0.0f));
        xb = min(xb, (int)fminf(floorf(xc + half), (float)(W - 1)));
      }
      if (xa <= xb) {
        const float cyy = __fmul_rn(__fmul_rn(c, dy), dy), bdy = __fmul_rn(b2, dy);
        const int wa = xa >> 5, wb = xb >> 5;
        for (int wx = wa; wx <= wb && !h; ++wx) {
          if (!((__ldg(crow + (wx >> 5)) >> (wx & 31)) & 1u)) continue;
          uint32_t m = __ldg(vmask + (int64_t)y * wpr + wx);
          if (wx == wa) m &= ~0u << (xa & 31);
          if (wx == wb) m &= ~0u >> (31 - (xb & 31));
          while (m) {
            const int x = 32 * wx + __ffs(m) - 1;
            m &= m - 1u;
            const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), mx);
            const float q = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(a, dx), dx), cyy), __fmul_rn(bdy, dx));
            if (q <= kQMax) {
              h = true;
              break;
            }
          }
        }
      }
    }
    if (__any_sync(0xffffffffu, h)) return true;
  }
  return false;
}

// Alg. 1 step 5 and the OR over views.  A warp holds 32 Gaussians and
// walks the views together.  Per view each lane does the cheap part for
// its own pair: the square of radius r around the mean, the conservative
// extent filter (rows within 3 sqrt(a / det) of the mean, columns within
// 3 sqrt(c / det), widened) and the block mask over that rectangle.  The
// pairs whose rectangle reaches a moving block are then scanned one after
// the other by the whole warp (warp_pair_hits), so that a long scan near
// the motion does not run on one lane while the others wait.  A Gaussian
// is marked at its first hit and takes no further views.
__global__ __launch_bounds__(kMaskThreads) void k_dynamic_mask(const float *__restrict__ rec,
                                                                const uint32_t *__restrict__ texel,
                                                                const uint32_t *__restrict__ mask,
                                                                const uint32_t *__restrict__ coarse,
                                                                const DevView *__restrict__ views, int V,
                                                                int64_t N, int atlas_w, int atlas_h, float r_max,
                                                                uint32_t *dyn) {
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kMaskThreads + threadIdx.x;
  uint32_t t = 0;
  bool live = g < N;
  if (live) {
    t = __ldg(texel + g);
    // texel ids past the atlas (unwritten after a live-count mismatch) are skipped
    live = t < (uint32_t)atlas_w * (uint32_t)atlas_h;
  }
  for (int v = 0; v < V; ++v) {
    if (!__any_sync(0xffffffffu, live)) break;
    const DevView &view = views[v];
    const int W = view.width, H = view.height, wpr = (W + 31) >> 5, cpr = (wpr + 31) >> 5;
    const uint32_t *vmask = mask + view.mask_off;
    const uint32_t *vcoarse = coarse + view.coarse_off;
    float mx = 0.0f, my = 0.0f, a = 0.0f, b = 0.0f, c = 0.0f;
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    bool need = false;
    if (live) {
      const size_t pr = ((size_t)v * N + g) * kRec;
      const float4 r0 = __ldg(reinterpret_cast<const float4 *>(rec + pr));
      const float2 r1 = __ldg(reinterpret_cast<const float2 *>(rec + pr + 4));
      float rad = __ldg(rec + pr + 7);
      mx = r0.x;
      my = r0.y;
      a = r0.z;
      b = r0.w;
      c = r1.x;
      if (r_max > 0.0f && rad > r_max) rad = r_max;
      if (rad > 0.0f && isfinite(mx) && isfinite(my)) {
        const float ax = __fsub_rn(mx, 0.5f), ay = __fsub_rn(my, 0.5f);
        const float lox = fmaxf(ceilf(__fsub_rn(ax, rad)), 0.0f),
                    hix = fminf(floorf(__fadd_rn(ax, rad)), (float)(W - 1));
        const float loy = fmaxf(ceilf(__fsub_rn(ay, rad)), 0.0f),
                    hiy = fminf(floorf(__fadd_rn(ay, rad)), (float)(H - 1));
        if (lox <= hix && loy <= hiy) {
          x0 = (int)lox;
          x1 = (int)hix;
          y0 = (int)loy;
          y1 = (int)hiy;
          const float det = a * c - b * b;
          if (a > 0.0f && c > 0.0f && det > 0.0f && isfinite(det)) {
            const float ey = 3.0f * sqrtf(a / det) * 1.001f + 1.0f, ex = 3.0f * sqrtf(c / det) * 1.001f + 1.0f;
            y0 = max(y0, (int)fmaxf(ceilf(ay - ey), 0.0f));
            y1 = min(y1, (int)fminf(floorf(ay + ey), (float)(H - 1)));
            x0 = max(x0, (int)fmaxf(ceilf(ax - ex), 0.0f));
            x1 = min(x1, (int)fminf(floorf(ax + ex), (float)(W - 1)));
          }
          // does a block of the rectangle move?
          const int w0 = x0 >> 5, w1 = x1 >> 5;
          for (int cy = y0 >> 5; y0 <= y1 && x0 <= x1 && cy <= (y1 >> 5) && !need; ++cy) {
            const uint32_t *crow = vcoarse + (int64_t)cy * cpr;
            for (int cw = w0 >> 5; cw <= (w1 >> 5) && !need; ++cw) {
              uint32_t cm = __ldg(crow + cw);
              if (cw == (w0 >> 5)) cm &= ~0u << (w0 & 31);
              if (cw == (w1 >> 5)) cm &= ~0u >> (31 - (w1 & 31));
              need = cm != 0u;
            }
          }
        }
      }
    }
    uint32_t todo = __ballot_sync(0xffffffffu, need);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1u;
      const float smx = __shfl_sync(0xffffffffu, mx, src), smy = __shfl_sync(0xffffffffu, my, src);
      const float sa = __shfl_sync(0xffffffffu, a, src), sb = __shfl_sync(0xffffffffu, b, src);
      const float sc = __shfl_sync(0xffffffffu, c, src);
      const int sx0 = __shfl_sync(0xffffffffu, x0, src), sx1 = __shfl_sync(0xffffffffu, x1, src);
      const int sy0 = __shfl_sync(0xffffffffu, y0, src), sy1 = __shfl_sync(0xffffffffu, y1, src);
      if (warp_pair_hits(smx, smy, sa, sb, sc, sx0, sx1, sy0, sy1, W, wpr, cpr, vmask, vcoarse, lane) &&
          lane == src) {
        const uint32_t ty = t / (uint32_t)atlas_w, tx = t - ty * (uint32_t)atlas_w;
        atomicOr(dyn + (size_t)ty * (((uint32_t)atlas_w + 31u) >> 5) + (tx >> 5), 1u << (tx & 31u));
        live = false;
      }
    }
  }
}

int64_t max_view_words(const pk_plan *p) {
  int64_t m = 0;
  for (int v = 0; v < p->V; ++v) {
    const DevView &d = p->h_views[v];
    m = max(m, (int64_t)d.height * ((d.width + 31) / 32));
  }
  return m;
}

int64_t max_view_coarse_words(const pk_plan *p) {
  int64_t m = 0;
  for (int v = 0; v < p->V; ++v) {
    const DevView &d = p->h_views[v];
    m = max(m, (int64_t)((d.height + 31) / 32) * ((((d.width + 31) / 32) + 31) / 32));
  }
  return m;
}

}  // namespace

extern "C" pk_status pk_motion_mask(const pk_plan *p, const float *flow, float tau, int32_t dilate_r,
                                    uint32_t *mask_bits, void *ws, pk_stream_t stream) {
  if (!p || !flow || !mask_bits || !ws) return PK_ERR_ARG;
  if (tau != tau || dilate_r < 0 || dilate_r > 4096) return PK_ERR_ARG;
  if (!aligned16(flow) || !aligned16(mask_bits)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const DevView *views = at<DevView>(ws, p->ws.views);
  uint32_t *tmp = at<uint32_t>(ws, p->ws.mask_tmp);
  const int64_t words = max_view_words(p);
  const int64_t warps = (words + kWordsPerWarp - 1) / kWordsPerWarp;
  const dim3 warp_grid((unsigned)((warps * 32 + kMaskThreads - 1) / kMaskThreads), (unsigned)p->V);
  const dim3 word_grid((unsigned)((words + kMaskThreads - 1) / kMaskThreads), (unsigned)p->V);
  k_motion_threshold<<<warp_grid, kMaskThreads, 0, st>>>(flow, views, tau, mask_bits);
  if (dilate_r > 0) {
    k_dilate_rows<<<word_grid, kMaskThreads, 0, st>>>(mask_bits, views, dilate_r, tmp);
    k_dilate_cols<<<word_grid, kMaskThreads, 0, st>>>(tmp, views, dilate_r, mask_bits);
  }
  return check_launch();
}

extern "C" pk_status pk_dynamic_mask(const pk_plan *p, const float *records, const uint32_t *texel,
                                     const uint32_t *mask_bits, float r_max, uint32_t *dyn, int32_t accumulate,
                                     void *ws, pk_stream_t stream) {
  if (!p || !records || !texel || !mask_bits || !dyn || !ws) return PK_ERR_ARG;
  if (r_max != r_max || (accumulate != 0 && accumulate != 1)) return PK_ERR_ARG;
  if (!aligned16(records)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int aw = p->desc.atlas_w, ah = p->desc.atlas_h;
  if (!accumulate) {
    const pk_status ze = zero_async({{dyn, sizeof(uint32_t) * (size_t)ah * (size_t)((aw + 31) / 32)}}, st);
    if (ze != PK_OK) return ze;
  }
  if (p->N == 0) return PK_OK;
  const DevView *views = at<DevView>(ws, p->ws.views);
  uint32_t *coarse = at<uint32_t>(ws, p->ws.mask_coarse);
  const int64_t cwords = max_view_coarse_words(p);
  const dim3 cgrid((unsigned)((cwords * 32 + kMaskThreads - 1) / kMaskThreads), (unsigned)p->V);
  k_mask_coarse<<<cgrid, kMaskThreads, 0, st>>>(mask_bits, views, coarse);
  const unsigned grid = (unsigned)((p->N + kMaskThreads - 1) / kMaskThreads);
  k_dynamic_mask<<<grid, kMaskThreads, 0, st>>>(records, texel, mask_bits, coarse, views, p->V, p->N, aw, ah, r_max,
                                                dyn);
  return check_launch();
}
