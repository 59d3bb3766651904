// Shared pieces of the forward (a4) and backward (a5) compositing kernels:
// tile -> view lookup, batch staging of a tile's splats into shared memory,
// and the per-pixel alpha evaluation.  The evaluation is written with
// explicit round-to-nearest intrinsics so that both kernels take exactly
// the same skip / clamp decisions for the same (pixel, splat).
#pragma once

#include "pk_common.cuh"
#include "pk_f32x2.cuh"

namespace pk {

constexpr int kTileSide = 16;   // side of the pixel block of one compositing CTA
// Splats staged per batch: a template parameter of the compositing
// kernels (64, 128 or 256; pk_options.batch, chosen by pk_autotune).
constexpr int kBatchMax = 256;

// One CTA per 16 x 16 pixel block with kPx pixels per thread (2, 4 or 8).
// A warp covers a kBW x kBH block (8 x 8 for 2 pixels, 16 x 8 for 4, the
// whole 16 x 16 for 8) and skips as a whole every splat that misses its
// block; a lane holds one column of it, kPx pixels kRowStep rows apart.
// More pixels per lane spread the per-splat work of a warp (shared-memory
// loads, the block test, the gradient reduction) over more pixels, at the
// price of a coarser block test and more registers.
template <int kPx>
struct Geo {
  static_assert(kPx == 2 || kPx == 4 || kPx == 8, "2, 4 or 8 pixels per thread");
  static constexpr int kThreads = kTileSide * kTileSide / kPx;   // 128, 64 or 32
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kBW = kPx == 2 ? 8 : 16;
  static constexpr int kBH = kPx == 8 ? 16 : 8;
  static constexpr int kRowStep = kBH / kPx;                      // 4, 2 or 2
  static constexpr int kBlocksX = kTileSide / kBW;                // warp blocks per row
  static_assert(kBW * kBH == 32 * kPx, "a warp's block holds its lanes' pixels");
};

// Pixels per thread: the forward keeps 2 (its per-splat work is small, and
// 8 x 8 blocks skip more), the backward 4 (its per-splat reduction of nine
// gradients is spread over twice the pixels); measured at the 52-view rig.
constexpr int kFwdPx = 2, kBwdPx = 4;

// Lane's column ox and first row oy in the tile; (bx, by) = its warp block's corner.
template <int kPx>
__device__ __forceinline__ void pixel_of(int tid, int &ox, int &oy, int &bx, int &by) {
  using G = Geo<kPx>;
  const int w = tid >> 5, l = tid & 31;
  bx = (w % G::kBlocksX) * G::kBW;
  by = (w / G::kBlocksX) * G::kBH;
  ox = bx + (l % G::kBW);
  oy = by + l / G::kBW;
}

// View that owns global tile t (binary search over tile offsets).
__device__ __forceinline__ int view_of_tile(const uint32_t *__restrict__ toff, int V, uint32_t t) {
  int lo = 0, hi = V - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(toff + mid) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct Staged {
  float4 *a;     // m_x, m_y, A = k conic_a, B = 2 k conic_b      (k = -log2(e) / 2)
  float4 *b;     // C = k conic_c, -opacity, red, green
  float4 *c;     // blue, pair index (bits), pcut, 0
  float4 *box;   // conservative pixel-centre box of the contributing ellipse
  float4 *q;     // conic_a, conic_b, conic_c, qlim = min(9, 2 ln(255 o)) for the block test
};

// 2^x on the MUFU unit (one instruction; relative error below 2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1 / x and sqrt(x) on the MUFU unit (one instruction each, relative error
// near 2^-22): used only for the culling box, whose margins are far wider.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Stage one splat.  The exponent of the Gaussian is evaluated directly as
// power = k q = A dx^2 + B dx dy + C dy^2, so alpha = o 2^power; a pixel is
// skipped unless power >= pcut = max(9 k, -log2(255 o)), i.e. unless both
// q <= 9 and o e^{-q/2} >= 1/255 hold.  The box bounds every pixel where
// q <= min(9, 2 ln(255 o)), widened by a relative 1e-3 and 0.01 px so that
// rounding can never put a passing pixel outside; it only lets whole warps
// skip, the per-pixel test still decides.
__device__ __forceinline__ void stage_from(const float4 r0, const float4 r1, const float4 r2, uint32_t pid,
                                           const Staged &s, int j) {
  const float ca = r0.z, cb = r0.w, cc = r1.x, o = r1.y;
  s.a[j] = make_float4(r0.x, r0.y, __fmul_rn(kExpScale, ca), __fmul_rn(2.f * kExpScale, cb));
  s.b[j] = make_float4(__fmul_rn(kExpScale, cc), -o, r2.x, r2.y);
  const float pcut = fmaxf(9.f * kExpScale, -__log2f(255.f * o));
  s.c[j] = make_float4(r2.z, __uint_as_float(pid), pcut, 0.f);
  const float qlim = fminf(kQMax, 2.f * __logf(255.f * o));
  s.q[j] = make_float4(ca, cb, cc, qlim);
  const float detq = ca * cc - cb * cb;
  float4 box;
  if (!(qlim >= 0.f)) {
    box = make_float4(1.f, -1.f, 1.f, -1.f);    // can never pass the alpha test
  } else if (detq > 0.f && isfinite(detq)) {
    const float rd = qlim * rcp_approx(detq);
    const float hx = sqrt_approx(rd * cc) * 1.001f + 0.01f;
    const float hy = sqrt_approx(rd * ca) * 1.001f + 0.01f;
    box = make_float4(r0.x - hx, r0.x + hx, r0.y - hy, r0.y + hy);
  } else {
    box = make_float4(-INFINITY, INFINITY, -INFINITY, INFINITY);
  }
  s.box[j] = box;
}

// A list entry that names no pair of the plan (a list that pk_bin_and_sort
// did not write for this plan): staged as a splat that reaches no pixel.
constexpr uint32_t kNoPair = 0xffffffffu;   // never a pair index (pairs < 2^32 - 1)
__device__ __forceinline__ void stage_none(const Staged &s, int j) {
  s.a[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  s.b[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  s.c[j] = make_float4(0.f, __uint_as_float(kNoPair), INFINITY, 0.f);
  s.q[j] = make_float4(0.f, 0.f, 0.f, -1.f);
  s.box[j] = make_float4(1.f, -1.f, 1.f, -1.f);   // misses every block
}

__device__ __forceinline__ void stage_splat(const float *__restrict__ rec, uint32_t pid, uint32_t npairs,
                                            const Staged &s, int j, pk_device_status *status) {
  if (pid >= npairs) {
    stage_none(s, j);
    atomicOr(&status->flags, PK_DEV_BOUNDS);
    return;
  }
  const float4 *r = reinterpret_cast<const float4 *>(rec + (size_t)pid * kRec);
  stage_from(__ldg(r), __ldg(r + 1), __ldg(r + 2), pid, s, j);
}

// The exponent power = k q = A dx^2 + B dx dy + C dy^2 of a staged splat at
// two pixel centres of one column, two lanes at a time, from the per-splat
// terms zxdx = (A dx) dx and bdx = B dx of the column: power = (C dy + bdx)
// dy + zxdx, dy = py - m_y, each step rounded to nearest in this order,
// exactly the steps of splat_power below (the forward's scalar form), so the
// two kernels take identical skip and clamp decisions.  A pixel skips the
// splat unless power >= pcut; then alpha = min(0.99, o 2^power).
__device__ __forceinline__ f32x2 splat_power2(const float4 &a, const float4 &b, float bdx, float zxdx, f32x2 py,
                                              f32x2 &dy) {
  dy = sub2(py, dup2(a.y));
  return fma2(fma2(dup2(b.x), dy, dup2(bdx)), dy, dup2(zxdx));
}

// The same exponent at one pixel centre (the forward's scalar form): the
// steps and rounding of splat_power2, so the two kernels take identical
// skip and clamp decisions.
__device__ __forceinline__ float splat_power(const float4 &a, const float4 &b, float bdx, float zxdx, float py) {
  const float dy = __fsub_rn(py, a.y);
  return __fmaf_rn(__fmaf_rn(b.x, dy, bdx), dy, zxdx);
}

__device__ __forceinline__ bool box_misses(const float4 &box, float x0, float x1, float y0, float y1) {
  return box.x > x1 || box.y < x0 || box.z > y1 || box.w < y0;
}

// Can the staged splat pass both skip tests anywhere in the pixel-centre
// rectangle [x0, x1] x [y0, y1] of a warp's block?  First the box, then the
// least q over the rectangle (0 with the mean inside, else on an edge facing
// the mean, at the clamped 1-D minimiser) against qlim, with a relative
// 1e-3 + 1e-3 margin so rounding can only keep a splat, never drop one.
__device__ __forceinline__ bool block_may_hit(const float4 &box, const float4 &q, float mx, float my, float x0,
                                              float x1, float y0, float y1) {
  if (box_misses(box, x0, x1, y0, y1)) return false;
  const float a = q.x, b = q.y, c = q.z;
  if (!(a > 0.f) || !(c > 0.f)) return true;
  const bool inx = mx >= x0 && mx <= x1, iny = my >= y0 && my <= y1;
  if (inx && iny) return true;
  const float lx = x0 - mx, hx = x1 - mx, ly = y0 - my, hy = y1 - my;
  float best = INFINITY;
  if (!inx) {
    const float dx = mx < x0 ? lx : hx;
    const float dy = fminf(fmaxf(-__fdividef(b * dx, c), ly), hy);
    best = fminf(best, (a * dx + 2.f * b * dy) * dx + c * dy * dy);
  }
  if (!iny) {
    const float dy = my < y0 ? ly : hy;
    const float dx = fminf(fmaxf(-__fdividef(b * dy, a), lx), hx);
    best = fminf(best, (a * dx + 2.f * b * dy) * dx + c * dy * dy);
  }
  return best <= q.w * 1.001f + 1e-3f;
}

}  // namespace pk
