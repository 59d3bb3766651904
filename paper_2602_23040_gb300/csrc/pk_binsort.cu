// a3 -- duplicate-key tile binning and a stable device radix sort
// (Sec. 3 tile-based rasteriser; Supp. "Viewer": per-camera depth order).
//
// Contract: entries ordered by (global tile id, bits(z), pair index).
// Instead of sorting (tile << 32 | bits(z)) keys over all entries, which
// costs about 7 radix passes over every (pair, tile) entry, the pairs are
// first sorted by depth alone (4 passes over pairs, ~15x fewer than
// entries), entries are emitted in that depth order, and a stable sort on
// the tile id alone (ceil(log2 tiles) bits, 2-3 passes) finishes the job:
// inside one tile every entry comes from the same view, so the stable
// tile sort leaves them in (bits(z), pair) order, exactly the contract.
//
// Every kernel runs on a fixed grid and reads its element count from
// device memory, so the whole step can be captured in a CUDA graph while
// the counts change from iteration to iteration.
#include <algorithm>

#include "pk_common.cuh"
#include "pk_tma.cuh"

using namespace pk;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;     // 2048

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Tile rectangle of a splat in FP32, in the contract's order, no FMA.
__device__ __forceinline__ bool bin_rect(float mx, float my, float r, int W, int H, int T, int &tx0, int &ty0,
                                         int &tx1, int &ty1) {
  if (!(r > 0.f)) return false;
  if (!isfinite(mx) || !isfinite(my)) return false;
  const float ax = __fsub_rn(mx, 0.5f), ay = __fsub_rn(my, 0.5f);
  const float lox = fmaxf(ceilf(__fsub_rn(ax, r)), 0.f);
  const float hix = fminf(floorf(__fadd_rn(ax, r)), (float)(W - 1));
  const float loy = fmaxf(ceilf(__fsub_rn(ay, r)), 0.f);
  const float hiy = fminf(floorf(__fadd_rn(ay, r)), (float)(H - 1));
  if (!(lox <= hix) || !(loy <= hiy)) return false;
  tx0 = (int)lox / T;
  ty0 = (int)loy / T;
  tx1 = (int)hix / T;
  ty1 = (int)hiy / T;
  return true;
}

// A splat's footprint for the ellipse rule, with the per-splat reciprocals
// hoisted (the same values a per-tile evaluation would produce).
struct Foot {
  float mx, my, a, b, c, ra, rc, b2;
};

__device__ __forceinline__ Foot make_foot(float mx, float my, float a, float b, float c) {
  Foot f;
  f.mx = mx;
  f.my = my;
  f.a = a;
  f.b = b;
  f.c = c;
  f.ra = __fdiv_rn(1.f, a);
  f.rc = __fdiv_rn(1.f, c);
  f.b2 = __fadd_rn(b, b);
  return f;
}

// Ellipse rule: does q = d^T conic d <= 9 (1 + 2^-12) reach the rectangle
// [x0, x1] x [y0, y1] of a tile's pixel centres?  Minimum of the convex q
// over the rectangle: 0 with the mean inside, else on an edge facing the
// mean, where the 1-D minimiser is clamped to the edge.  FP32 in exactly
// this order, no FMA.
__device__ __forceinline__ bool ellipse_hits_rect(const Foot &f, float x0, float x1, float y0, float y1) {
  const float qmax = 9.0f * (1.0f + 1.0f / 4096.0f);
  if (!(f.a > 0.f) || !(f.c > 0.f)) return true;
  const bool inx = f.mx >= x0 && f.mx <= x1, iny = f.my >= y0 && f.my <= y1;
  if (inx && iny) return true;
  const float lx = __fsub_rn(x0, f.mx), hx = __fsub_rn(x1, f.mx), ly = __fsub_rn(y0, f.my), hy = __fsub_rn(y1, f.my);
  float best = INFINITY;
  if (!inx) {
    const float dx = f.mx < x0 ? lx : hx;
    const float t = __fmul_rn(__fmul_rn(f.b, dx), f.rc);
    const float dy = fminf(fmaxf(-t, ly), hy);
    float q = __fmul_rn(__fmul_rn(f.a, dx), dx);
    q = __fadd_rn(q, __fmul_rn(__fmul_rn(f.b2, dx), dy));
    q = __fadd_rn(q, __fmul_rn(__fmul_rn(f.c, dy), dy));
    best = fminf(best, q);
  }
  if (!iny) {
    const float dy = f.my < y0 ? ly : hy;
    const float t = __fmul_rn(__fmul_rn(f.b, dy), f.ra);
    const float dx = fminf(fmaxf(-t, lx), hx);
    float q = __fmul_rn(__fmul_rn(f.a, dx), dx);
    q = __fadd_rn(q, __fmul_rn(__fmul_rn(f.b2, dx), dy));
    q = __fadd_rn(q, __fmul_rn(__fmul_rn(f.c, dy), dy));
    best = fminf(best, q);
  }
  return best <= qmax;
}

// local = q * w + r for a candidate index below 2^24: quotient from a float
// reciprocal, then corrected by one step, so the result is exact.
__device__ __forceinline__ void divmod_small(uint32_t local, uint32_t w, float rw, uint32_t &q, uint32_t &r) {
  q = __float2uint_rz(__fmul_rn(__uint2float_rn(local), rw));
  int rr = (int)local - (int)(q * w);
  if (rr < 0) {
    --q;
    rr += (int)w;
  } else if (rr >= (int)w) {
    ++q;
    rr -= (int)w;
  }
  r = (uint32_t)rr;
}

// Ellipse mode: the candidate tiles need only cover the footprint's
// bounding box |dx| <= 3 sqrt(Sigma_xx), |dy| <= 3 sqrt(Sigma_yy) (Sigma =
// conic^-1) rather than the whole r-square.  The box is widened by 1 % and
// one pixel, far beyond FP32 rounding, so every tile the exact test accepts
// stays a candidate and the entries are unchanged; it only skips tiles
// that the test would reject.
__device__ __forceinline__ void shrink_to_footprint(float mx, float my, float a, float b, float c, int T, int &tx0,
                                                    int &ty0, int &tx1, int &ty1) {
  const float det = a * c - b * b;
  if (!(a > 0.f) || !(c > 0.f) || !(det > 0.f) || !isfinite(det)) return;
  // MUFU reciprocal and square root (relative error near 2^-22): the 1 %
  // and one-pixel widening dwarfs it, so the box still holds every tile
  // the exact test accepts
  float idet, sx, sy;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(idet) : "f"(det));
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sx) : "f"(c * idet));
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sy) : "f"(a * idet));
  const float ex = 3.f * sx * 1.01f + 1.f, ey = 3.f * sy * 1.01f + 1.f;
  // tile tx holds pixel centres [tx T + 0.5, tx T + T - 0.5]
  const float rT = 1.f / (float)T;   // T is a power of two: x * rT == x / T exactly
  const float fx0 = floorf((mx - ex - 0.5f) * rT), fx1 = floorf((mx + ex - 0.5f) * rT);
  const float fy0 = floorf((my - ey - 0.5f) * rT), fy1 = floorf((my + ey - 0.5f) * rT);
  if (fx0 > (float)tx0) tx0 = (int)fminf(fx0, (float)tx1);
  if (fx1 < (float)tx1) tx1 = (int)fmaxf(fx1, (float)tx0);
  if (fy0 > (float)ty0) ty0 = (int)fminf(fy0, (float)ty1);
  if (fy1 < (float)ty1) ty1 = (int)fmaxf(fy1, (float)ty0);
}

__device__ __forceinline__ bool tile_hit(const Foot &f, int tx, int ty, int W, int H, int T) {
  const float x0 = (float)(tx * T) + 0.5f, y0 = (float)(ty * T) + 0.5f;
  const float x1 = (float)min((tx + 1) * T, W) - 0.5f, y1 = (float)min((ty + 1) * T, H) - 0.5f;
  return ellipse_hits_rect(f, x0, x1, y0, y1);
}

// Two 16-bit tile coordinates (or extents) in one word.
__device__ __forceinline__ uint32_t pack_rect(int a, int b) { return (uint32_t)a | ((uint32_t)b << 16); }

// A pair with at most this many candidate tiles keeps a bit mask of its
// receiving candidates from the count pass, so the emission need not test
// them again.
constexpr uint32_t kMaskBits = 64;

// Per-warp staging of 32 splats' candidate rectangles for the cooperative
// walk over their candidate tiles (one candidate per lane per step).
struct WarpSplat {
  float4 g0;   // mx, my, a, b
  float4 g1;   // c, ra, rc, b2
  int4 r0;     // tx0, ty0, wt, W
  int4 r1;     // H, tile base (tile_off + ty0 * tiles_x + tx0), tiles_x, ncand
};

// Owner of candidate e: number of lanes whose inclusive count is <= e.
__device__ __forceinline__ int candidate_owner(uint32_t incl, uint32_t e) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const uint32_t c = __shfl_sync(0xffffffffu, incl, pos + s - 1);
    if (c <= e) pos += s;
  }
  return pos;
}

// Contiguous chunk [begin, end) of block b when n items are split over nb
// blocks in whole tiles of `tile` items.
__device__ __forceinline__ void chunk_of(uint64_t n, int nb, int b, int tile, uint64_t &begin, uint64_t &end) {
  uint64_t per = (n + nb - 1) / nb;
  per = (per + tile - 1) / tile * tile;
  begin = per * b;
  end = begin + per;
  if (begin > n) begin = n;
  if (end > n) end = n;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// the block total.  s must hold kWarps + 1 elements.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T &total, T *s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = warp_incl_scan(v);
  if (lane == 31) s[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < kWarps ? s[lane] : T(0);
    T wi = warp_incl_scan(w);
    if (lane < kWarps) s[lane] = wi - w;
    if (lane == kWarps - 1) s[kWarps] = wi;
  }
  __syncthreads();
  T r = s[warp] + incl - v;
  total = s[kWarps];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Per-pair tile counts
// ---------------------------------------------------------------------------

// Receiving tiles per pair.  Rectangle mode: the size of the r-square.
// Ellipse mode: a warp walks the candidate tiles of its 32 pairs together,
// one candidate per lane, so long and short pairs share the work; each pair
// also keeps a bit mask of its receiving candidates when it has <= 64 of
// them, so the emission need not test them again.
__global__ __launch_bounds__(kThreads) void k_pair_count(const float *__restrict__ rec, int64_t pairs, int64_t N,
                                                         const DevView *__restrict__ views, int T, int mode,
                                                         uint32_t *__restrict__ cnt, uint4 *__restrict__ pinfo,
                                                         uint32_t *__restrict__ zbits) {
  constexpr uint32_t kBalChunks = 64;   // a walk of up to 2,048 candidates keeps its ballots
  __shared__ WarpSplat s_ws[kWarps][32];
  __shared__ uint32_t s_bal[kWarps][kBalChunks];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t nwarps = (uint64_t)gridDim.x * kWarps;
  for (uint64_t w = blockIdx.x * (uint64_t)kWarps + warp; w * 32 < (uint64_t)pairs; w += nwarps) {
    const uint64_t p = w * 32 + lane;
    uint32_t ncand = 0;
    WarpSplat ws;
    ws.g0 = make_float4(0.f, 0.f, 0.f, 0.f);
    ws.g1 = ws.g0;
    ws.r0 = make_int4(0, 0, 1, 1);
    ws.r1 = make_int4(1, 0, 1, 0);
    if (p < (uint64_t)pairs) {
      const float4 a = __ldg(reinterpret_cast<const float4 *>(rec + p * kRec));
      const float4 b = __ldg(reinterpret_cast<const float4 *>(rec + p * kRec) + 1);
      zbits[p] = __float_as_uint(b.z);   // the depth key, for the compaction
      const DevView &v = views[(uint32_t)p / (uint32_t)N];   // pairs < 2^32 (checked by the plan)
      int x0, y0, x1, y1;
      if (bin_rect(a.x, a.y, b.w, v.width, v.height, T, x0, y0, x1, y1)) {
        if (mode != PK_BIN_RECT) shrink_to_footprint(a.x, a.y, a.z, a.w, b.x, T, x0, y0, x1, y1);
        const int wt = x1 - x0 + 1;
        ncand = (uint32_t)(wt * (y1 - y0 + 1));
        const Foot f = make_foot(a.x, a.y, a.z, a.w, b.x);
        ws.g0 = make_float4(f.mx, f.my, f.a, f.b);
        ws.g1 = make_float4(f.c, f.ra, f.rc, f.b2);
        ws.r0 = make_int4(x0, y0, wt, v.width);
        ws.r1 = make_int4(v.height, 0, 0, (int)ncand);
      }
    }
    if (mode == PK_BIN_RECT) {
      if (p < (uint64_t)pairs) {
        cnt[p] = ncand;
        pinfo[p] = make_uint4(0u, 0u, pack_rect(ws.r0.x, ws.r0.y), pack_rect(ws.r0.z, ncand ? (int)ncand / ws.r0.z : 0));
      }
      continue;
    }
    const uint32_t incl = warp_incl_scan(ncand);
    const uint32_t excl = incl - ncand;
    // the owner's walk offset and 1 / width ride in the record, so a lane
    // reads its candidate's owner from shared memory alone
    ws.r1.y = (int)excl;
    ws.r1.z = __float_as_int(__frcp_rn((float)ws.r0.z));   // for the candidate -> (row, column) split
    s_ws[warp][lane] = ws;
    __syncwarp();
    const uint32_t E = __shfl_sync(0xffffffffu, incl, 31);
    // Each lane's own candidates [excl, incl) are read off the walk's
    // ballots: after the walk from the kept ballots (a lane visits only
    // the 1-3 steps its pair spans), or, for a longer walk, step by step.
    const bool keep = E <= 32 * kBalChunks;
    uint32_t mine = 0;
    uint64_t mask = 0;
    auto take_bits = [&](uint32_t e0, uint32_t bal) {
      const uint32_t lo = max(excl, e0), hi = min(incl, e0 + 32);
      if (lo < hi) {
        const uint32_t span = hi - lo;
        const uint32_t bits = (bal >> (lo - e0)) & (span >= 32 ? 0xffffffffu : ((1u << span) - 1u));
        mine += __popc(bits);
        if (ncand <= kMaskBits) mask |= (uint64_t)bits << (lo - excl);
      }
    };
    for (uint32_t e0 = 0; e0 < E; e0 += 32) {
      const uint32_t e = e0 + lane;
      const uint32_t ee = e < E ? e : E - 1;
      const int o = candidate_owner(incl, ee);
      const WarpSplat &os = s_ws[warp][o];
      const int4 r0 = os.r0, r1 = os.r1;
      const uint32_t local = ee - (uint32_t)r1.y;
      uint32_t lyq, lxr;
      divmod_small(local, (uint32_t)r0.z, __int_as_float(r1.z), lyq, lxr);
      const int ty = r0.y + (int)lyq, tx = r0.x + (int)lxr;
      bool hit = false;
      if (e < E) {
        const float4 g0 = os.g0, g1 = os.g1;
        const Foot f{g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
        hit = tile_hit(f, tx, ty, r0.w, r1.x, T);
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, hit);
      if (keep) {
        if (lane == 0) s_bal[warp][e0 >> 5] = bal;
      } else {
        take_bits(e0, bal);
      }
    }
    if (keep) {
      __syncwarp();   // lane 0's ballots visible to every lane
      if (ncand)
        for (uint32_t c = excl >> 5; 32 * c < incl; ++c) take_bits(32 * c, s_bal[warp][c]);
    }
    if (p < (uint64_t)pairs) {
      cnt[p] = mine;
      pinfo[p] = make_uint4((uint32_t)mask, (uint32_t)(mask >> 32), pack_rect(ws.r0.x, ws.r0.y),
                            pack_rect(ws.r0.z, ncand ? (int)ncand / ws.r0.z : 0));
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Chunked reduce-then-scan.  Item i of the scanned sequence is src(i).
// ---------------------------------------------------------------------------

struct SrcValid {      // 1 if pair i touches a tile
  const uint32_t *cnt;
  __device__ uint32_t operator()(uint64_t i) const { return cnt[i] > 0u ? 1u : 0u; }
};
__device__ __forceinline__ uint64_t load_n(const uint64_t *n_dev, uint64_t n_host) {
  return n_dev ? *n_dev : n_host;
}

template <typename Src>
__global__ __launch_bounds__(kThreads) void k_scan_reduce(Src src, const uint64_t *n_dev, uint64_t n_host,
                                                          uint64_t *__restrict__ bsum) {
  __shared__ uint64_t s[kWarps + 1];
  const uint64_t n = load_n(n_dev, n_host);
  uint64_t b0, b1;
  chunk_of(n, gridDim.x, blockIdx.x, kScanTile, b0, b1);
  uint64_t acc = 0;
  for (uint64_t i = b0 + threadIdx.x; i < b1; i += kThreads) acc += src(i);
  uint64_t tot;
  block_excl_scan<uint64_t>(acc, tot, s);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Exclusive scan of the block sums (one block of 1024 threads, up to 4096
// sums: kScanBlocks).  mode 0: compaction (total
// = valid pairs); mode 1: emission offsets (total = entries, checked
// against the capacity).
__global__ __launch_bounds__(1024) void k_scan_top(uint64_t *__restrict__ bsum, int nb, int mode,
                                                   uint64_t max_dups, DevCounters *ctr, pk_device_status *status) {
  __shared__ uint64_t s[33];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // four consecutive block sums per thread (nb <= 4096)
  uint64_t q[4], v = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    q[j] = 4 * tid + j < nb ? bsum[4 * tid + j] : 0;
    v += q[j];
  }
  uint64_t incl = warp_incl_scan(v);
  if (lane == 31) s[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = s[lane];
    uint64_t wi = warp_incl_scan(w);
    s[lane] = wi - w;
    if (lane == 31) s[32] = wi;
  }
  __syncthreads();
  uint64_t run = s[warp] + incl - v;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (4 * tid + j < nb) bsum[4 * tid + j] = run;
    run += q[j];
  }
  if (tid == 0) {
    const uint64_t total = s[32];
    ctr->scan_total = total;
    if (mode == 0) {
      ctr->n_valid = total;
      status->valid_pairs = total;
    } else {
      status->dups_needed = total;
      if (ctr->sort_abort) {   // a depth pass gave up: emit nothing
        ctr->dups = 0;
        status->dups = 0;
      } else if (total > max_dups) {
        ctr->dups = 0;
        status->dups = 0;
        atomicOr(&status->flags, PK_DEV_CAPACITY);
      } else {
        ctr->dups = total;
        status->dups = total;
      }
    }
  }
}

// Eight consecutive items of a u32 array from item i0 (a multiple of 8): two
// 16-byte loads where all eight lie below b1, else one by one (0 past b1).
__device__ __forceinline__ void load8(const uint32_t *__restrict__ a, uint64_t i0, uint64_t b1, uint32_t (&v)[8]) {
  if (i0 + 7 < b1) {
    const uint4 x = __ldg(reinterpret_cast<const uint4 *>(a + i0));
    const uint4 y = __ldg(reinterpret_cast<const uint4 *>(a + i0) + 1);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = i0 + j < b1 ? __ldg(a + i0 + j) : 0u;
  }
}
static_assert(kScanItems == 8, "load8 takes a thread's scan items");

// Down-sweep of the compaction: writes (bits(z), pair) of every valid pair
// in pair order.  A tile's outputs go through shared memory so that the
// writes are contiguous.
__global__ __launch_bounds__(kThreads) void k_compact_down(const uint32_t *__restrict__ cnt,
                                                           const uint32_t *__restrict__ zbits, uint64_t n,
                                                           const uint64_t *__restrict__ bsum,
                                                           uint32_t *__restrict__ zkey, uint32_t *__restrict__ pval) {
  __shared__ uint32_t s[kWarps + 1];
  __shared__ uint32_t s_z[kScanTile], s_p[kScanTile];
  uint64_t b0, b1;
  chunk_of(n, gridDim.x, blockIdx.x, kScanTile, b0, b1);
  uint32_t run = (uint32_t)bsum[blockIdx.x];   // valid pairs < 2^32
  for (uint64_t base = b0; base < b1; base += kScanTile) {
    const uint64_t i0 = base + (uint64_t)threadIdx.x * kScanItems;
    uint32_t cv[8], zv[8], c = 0;
    load8(cnt, i0, b1, cv);
    load8(zbits, i0, b1, zv);
#pragma unroll
    for (int j = 0; j < 8; ++j) c += cv[j] > 0u ? 1u : 0u;
    uint32_t tot;
    uint32_t pre = block_excl_scan<uint32_t>(c, tot, s);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (cv[j] > 0u) {
        s_z[pre] = zv[j];
        s_p[pre] = (uint32_t)(i0 + j);
        ++pre;
      }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < tot; k += kThreads) {
      zkey[run + k] = s_z[k];
      pval[run + k] = s_p[k];
    }
    __syncthreads();   // before the next tile's outputs reuse s_z, s_p
    run += tot;
  }
}

// Tile counts of the pairs in depth order, gathered once: csorted[i] =
// cnt[pval[i]] (0 for a pair index past the pairs, which a depth pass that
// gave up can leave), and each block's sum for the offset scan.
__global__ __launch_bounds__(kThreads) void k_reduce_sorted(const uint32_t *__restrict__ cnt,
                                                            const uint32_t *__restrict__ pval, uint64_t pairs,
                                                            const uint64_t *n_dev, uint32_t *__restrict__ csorted,
                                                            uint64_t *__restrict__ bsum) {
  __shared__ uint64_t s[kWarps + 1];
  const uint64_t n = *n_dev;
  uint64_t b0, b1;
  chunk_of(n, gridDim.x, blockIdx.x, kScanTile, b0, b1);
  uint64_t acc = 0;
  for (uint64_t base = b0; base < b1; base += kScanTile) {
    const uint64_t i0 = base + (uint64_t)threadIdx.x * kScanItems;
    uint32_t pv[8], v[8];
    load8(pval, i0, b1, pv);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = i0 + j < b1 && pv[j] < pairs ? __ldg(cnt + pv[j]) : 0u;
      acc += v[j];
    }
    if (i0 + 7 < b1) {
      reinterpret_cast<uint4 *>(csorted + i0)[0] = make_uint4(v[0], v[1], v[2], v[3]);
      reinterpret_cast<uint4 *>(csorted + i0)[1] = make_uint4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (i0 + j < b1) csorted[i0 + j] = v[j];
    }
  }
  uint64_t tot;
  block_excl_scan<uint64_t>(acc, tot, s);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Down-sweep of the emission-offset scan: offs[i] = entries before pair i
// (64-bit: the entries of a launch may pass 2^32), from the gathered counts.
__global__ __launch_bounds__(kThreads) void k_offsets_down(const uint32_t *__restrict__ csorted,
                                                           const uint64_t *n_dev, const uint64_t *__restrict__ bsum,
                                                           const DevCounters *ctr, uint64_t *__restrict__ offs) {
  __shared__ uint64_t s[kWarps + 1];
  if (ctr->dups == 0) return;   // overflow (or nothing): nothing will be emitted
  const uint64_t n = *n_dev;
  uint64_t b0, b1;
  chunk_of(n, gridDim.x, blockIdx.x, kScanTile, b0, b1);
  uint64_t run = bsum[blockIdx.x];
  for (uint64_t base = b0; base < b1; base += kScanTile) {
    const uint64_t i0 = base + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[8];
    load8(csorted, i0, b1, v);
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) c += v[j];
    uint64_t tot;
    uint64_t pre = block_excl_scan<uint64_t>(c, tot, s) + run;
    uint64_t o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      o[j] = pre;
      pre += v[j];
    }
    if (i0 + 7 < b1) {
#pragma unroll
      for (int j = 0; j < 8; j += 2) reinterpret_cast<ulonglong2 *>(offs + i0)[j / 2] = make_ulonglong2(o[j], o[j + 1]);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (i0 + j < b1) offs[i0 + j] = o[j];
    }
    run += tot;
  }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, one pass = upsweep + scan + downsweep, digits of
// up to RB bits.
// ---------------------------------------------------------------------------

// Where a radix block works.  Global mode (tab == nullptr): the whole
// array [0, n) split over the grid, histogram counter of digit d at
// d * gridDim.x + blockIdx.x.  Segmented mode: block b belongs to segment
// tab[b].x (a view's entries [seg[v], seg[v + 1])), as part tab[b].y of
// tab[b].z parts, counters at tab[b].w + d * tab[b].z + tab[b].y, so the
// one scan of the histogram keeps every segment in place and sorts within
// it.
struct SegSpec {
  const int4 *tab;
  const uint64_t *seg;
};

__device__ __forceinline__ void radix_chunk(const SegSpec &sp, uint64_t n, int tile, uint64_t &b0, uint64_t &b1,
                                            uint32_t &hbase, uint32_t &hstride) {
  if (!sp.tab) {
    chunk_of(n, gridDim.x, blockIdx.x, tile, b0, b1);
    hbase = blockIdx.x;
    hstride = gridDim.x;
    return;
  }
  const int4 t = sp.tab[blockIdx.x];
  const uint64_t s0 = sp.seg[t.x], s1 = sp.seg[t.x + 1];
  chunk_of(s1 - s0, t.z, t.y, tile, b0, b1);
  b0 += s0;
  b1 += s0;
  hbase = (uint32_t)(t.w + t.y);
  hstride = (uint32_t)t.z;
}

// RB-bit digits, IT keys per thread and tile.  More keys per thread give
// longer runs per bucket in the scatter; fewer give more resident blocks.
// The pair passes (33 M keys at C3, random low digits) take 12 at 3 blocks
// per SM, the entry passes (410 M keys) 8 at 4 blocks per SM.
template <int RB, int IT>
struct Radix {
  static constexpr int kR = 1 << RB;                       // buckets
  static constexpr int kItems = IT;                        // keys per thread and tile
  static constexpr int kTile = kThreads * kItems;          // a multiple of 4
  static constexpr int kCopies = RB <= 8 ? kWarps : 2;     // private histograms in the upsweep
  static constexpr int kPerThread = kR / kThreads;         // buckets per thread in the digit scan
  // resident per SM (downsweep): 8-bit digits by registers, 11-bit digits by
  // shared memory (per-warp counters and the double buffer, ~82-98 KB)
  static constexpr int kMinBlocks = RB > 8 ? 2 : (IT >= 12 ? 3 : (IT >= 8 ? 4 : 5));
};
constexpr int kPairItems = 12, kEntryItems = 8;

template <int RB, int IT>
__global__ __launch_bounds__(kThreads) void k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                            const uint64_t *n_dev, uint64_t n_host, int shift,
                                                            uint32_t mask, uint64_t *__restrict__ hist, SegSpec sp) {
  using C = Radix<RB, IT>;
  __shared__ uint32_t s_cnt[C::kCopies][C::kR];   // private digit counts
  for (int i = threadIdx.x; i < C::kCopies * C::kR; i += kThreads) (&s_cnt[0][0])[i] = 0;
  __syncthreads();
  const uint64_t n = load_n(n_dev, n_host);
  uint64_t b0, b1;
  uint32_t hbase, hstride;
  radix_chunk(sp, n, C::kTile, b0, b1, hbase, hstride);
  uint32_t *cw = s_cnt[(threadIdx.x >> 5) % C::kCopies];
  // up to 3 keys before the first 16-byte boundary (segments start anywhere)
  const uint64_t a0 = min(b1, (b0 + 3) & ~uint64_t(3));
  if (threadIdx.x < a0 - b0) atomicAdd(&cw[(__ldg(keys + b0 + threadIdx.x) >> shift) & mask], 1u);
  // 16-byte vector loads, four in flight per thread
  const uint4 *k4 = reinterpret_cast<const uint4 *>(keys + a0);
  const uint64_t n4 = (b1 - a0) / 4;
  for (uint64_t t0 = 0; t0 < n4; t0 += 4 * kThreads) {
    uint4 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t i = t0 + (uint64_t)u * kThreads + threadIdx.x;
      q[u] = i < n4 ? __ldg(k4 + i) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (t0 + (uint64_t)u * kThreads + threadIdx.x >= n4) break;
      atomicAdd(&cw[(q[u].x >> shift) & mask], 1u);
      atomicAdd(&cw[(q[u].y >> shift) & mask], 1u);
      atomicAdd(&cw[(q[u].z >> shift) & mask], 1u);
      atomicAdd(&cw[(q[u].w >> shift) & mask], 1u);
    }
  }
  for (uint64_t i = a0 + 4 * n4 + threadIdx.x; i < b1; i += kThreads)
    atomicAdd(&cw[(__ldg(keys + i) >> shift) & mask], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < C::kR; d += kThreads) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < C::kCopies; ++w) t += s_cnt[w][d];
    hist[hbase + (size_t)d * hstride] = t;
  }
}

// Exclusive scan of hist in [digit][block] order.  The counters are
// 64-bit: after the scan they are output positions, and the entries of a
// launch may pass 2^32.  Each block of 1024 threads takes a chunk of 4096
// consecutive counters: k_radix_chunk_sums writes each chunk's total,
// k_radix_scan_chunks adds the totals of the chunks before its own (at most
// a few hundred) and scans its chunk in place -- two short launches instead
// of one block walking every chunk in turn (63 us a pass at the 52-view
// rig).  The chunk totals use the binning's block-sum buffer, idle while
// the radix passes run.
constexpr int kHistChunk = 4096;
__global__ __launch_bounds__(1024) void k_radix_chunk_sums(const uint64_t *__restrict__ hist, int count,
                                                           uint64_t *__restrict__ csum) {
  __shared__ uint64_t s[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = blockIdx.x * kHistChunk + 4 * tid;
  uint64_t t = 0;
  if (i + 3 < count) {
    const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(hist + i);
    const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(hist + i + 2);
    t = a.x + a.y + b.x + b.y;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) t += i + j < count ? hist[i + j] : 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) s[warp] = t;
  __syncthreads();
  if (warp == 0) {
    t = s[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) csum[blockIdx.x] = t;
  }
}

__global__ __launch_bounds__(1024) void k_radix_scan_chunks(uint64_t *__restrict__ hist, int count,
                                                            const uint64_t *__restrict__ csum) {
  __shared__ uint64_t s[33];
  __shared__ uint64_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  // counters of the chunks before this one
  uint64_t c = 0;
  for (int k = tid; k < b; k += 1024) c += csum[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) s[warp] = c;
  __syncthreads();
  if (warp == 0) {
    c = s[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) s_carry = c;
  }
  __syncthreads();
  const int i = b * kHistChunk + 4 * tid;
  uint64_t q[4];
  if (i + 3 < count) {
    const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(hist + i);
    const ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(hist + i + 2);
    q[0] = x.x; q[1] = x.y; q[2] = y.x; q[3] = y.y;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) q[j] = i + j < count ? hist[i + j] : 0ull;
  }
  const uint64_t sum = q[0] + q[1] + q[2] + q[3];
  const uint64_t incl = warp_incl_scan(sum);
  if (lane == 31) s[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint64_t w = s[lane];
    const uint64_t wi = warp_incl_scan(w);
    s[lane] = wi - w;
  }
  __syncthreads();
  uint64_t e = s_carry + s[warp] + incl - sum;
  uint64_t o[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    o[j] = e;
    e += q[j];
  }
  if (i + 3 < count) {
    *reinterpret_cast<ulonglong2 *>(hist + i) = make_ulonglong2(o[0], o[1]);
    *reinterpret_cast<ulonglong2 *>(hist + i + 2) = make_ulonglong2(o[2], o[3]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (i + j < count) hist[i + j] = o[j];
  }
}

// Downsweep with the next tile's keys and values prefetched by TMA into the
// other half of a double buffer while the current tile is ranked and
// scattered; the ranking permutes the current tile in place.
template <int RB, int IT>
struct Down {
  static constexpr int kTile = Radix<RB, IT>::kTile;
  static constexpr int kSpan = kTile + 4;                         // a tile plus up to 3 keys of misalignment
  static constexpr size_t kBuf = 2 * sizeof(uint32_t) * kSpan;    // keys + values of one tile
  static constexpr size_t kSmem = 2 * kBuf + sizeof(uint16_t) * kWarps * Radix<RB, IT>::kR +
                                  (sizeof(uint32_t) + sizeof(uint64_t)) * Radix<RB, IT>::kR +
                                  sizeof(uint32_t) * (kWarps + 1) + 2 * sizeof(uint64_t) + 16;
};

// The last pass over packed entries (one word: tile id above pair index)
// writes no words: it writes each entry's pair index into vout and folds
// the tile ranges in with atomics (start as the largest ~position, end as
// the largest position + 1, on ranges zeroed beforehand; k_range_fix turns
// them into [start, end)).  In a segmented sort both ids are local to the
// block's view.
struct Unpack {
  uint64_t *ranges;
  const uint32_t *toff;   // [V + 1] first global tile of each view
  uint32_t N;             // pairs per view
  int pbits;              // pair-index bits below the tile id
  uint32_t n_tiles;
  uint64_t npairs;
};

// kMode 0: values travel with the keys (vin/vout); 1: keys only (packed
// entries); 2: keys only, the last pass (pair indices and tile ranges out).
template <int RB, int IT, int kMode>
__global__ __launch_bounds__(kThreads, (Radix<RB, IT>::kMinBlocks)) void k_radix_downsweep(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint64_t *n_dev, uint64_t n_host, int shift, uint32_t mask,
    const uint64_t *__restrict__ hist, pk_device_status *status, SegSpec sp, uint32_t *abort_flag,
    uint32_t first_polls, bool try_single, Unpack up) {
  using C = Radix<RB, IT>;
  constexpr bool kV = kMode == 0, kLast = kMode == 2;
  constexpr int kTile = C::kTile;
  constexpr int kSpan = Down<RB, IT>::kSpan;
  extern __shared__ __align__(16) unsigned char s_raw[];
  uint32_t *buf[2] = {reinterpret_cast<uint32_t *>(s_raw), reinterpret_cast<uint32_t *>(s_raw + Down<RB, IT>::kBuf)};
  uint16_t *s_wcnt = reinterpret_cast<uint16_t *>(s_raw + 2 * Down<RB, IT>::kBuf);       // [kWarps][kR]
  uint32_t *s_start = reinterpret_cast<uint32_t *>(s_wcnt + kWarps * C::kR);         // [kR]
  uint64_t *s_gbase = reinterpret_cast<uint64_t *>(s_start + C::kR);                // [kR] output positions
  uint32_t *s_scan = reinterpret_cast<uint32_t *>(s_gbase + C::kR);                 // [kWarps + 1]
  uint64_t *s_bar = reinterpret_cast<uint64_t *>(
      (reinterpret_cast<uintptr_t>(s_scan + kWarps + 1) + 7) & ~uintptr_t(7));      // [2]
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t n = load_n(n_dev, n_host);
  uint64_t b0, b1;
  uint32_t hbase, hstride;
  radix_chunk(sp, n, kTile, b0, b1, hbase, hstride);
  if (b1 - b0 > 0xffffffffull) {   // a block's digit counts are 32-bit: give the call up
    if (tid == 0) {
      atomicOr(&status->flags, PK_DEV_BOUNDS);
      *abort_flag = 1u;
    }
    return;
  }
  for (int d = tid; d < C::kR; d += kThreads) s_gbase[d] = hist[hbase + (size_t)d * hstride];
  const int ntile = (int)((b1 - b0 + kTile - 1) / kTile);
  // last packed pass: the block's view (segmented) turns local ids global
  uint32_t tile0 = 0, tile1 = up.n_tiles;
  uint64_t pid0 = 0;
  if (kLast && sp.tab) {
    const int vw = sp.tab[blockIdx.x].x;
    tile0 = __ldg(up.toff + vw);
    tile1 = __ldg(up.toff + vw + 1);
    pid0 = (uint64_t)vw * up.N;
  }
  // Every tile of this chunk starts mis = b0 mod 4 keys past a 16-byte
  // boundary: the bulk copy starts at that boundary and takes whole
  // 16-byte groups; tile key li lands at buf[mis + li].
  const uint32_t mis = (uint32_t)(b0 & 3);
  auto issue = [&](int t) {
    const uint64_t base = b0 + (uint64_t)t * kTile;
    const uint32_t valid = (uint32_t)min((uint64_t)kTile, b1 - base);
    const uint32_t bytes = ((mis + valid) & ~3u) * 4u;
    uint32_t *dst = buf[t & 1];
    mbar_expect_tx(&s_bar[t & 1], (kV ? 2u : 1u) * bytes);
    if (bytes) {
      tma_load_1d(dst, kin + (base - mis), bytes, &s_bar[t & 1]);
      if (kV) tma_load_1d(dst + kSpan, vin + (base - mis), bytes, &s_bar[t & 1]);
    }
  };
  if (tid == 0) {
    s_abort = 0;
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (ntile > 0) issue(0);
  }
  __syncthreads();
  const uint32_t lt = lanemask_lt();
  uint16_t *wc = s_wcnt + warp * C::kR;
  uint32_t parity[2] = {0u, 0u};
  for (int t = 0; t < ntile; ++t) {
    const int cur = t & 1;
    const uint64_t base = b0 + (uint64_t)t * kTile;
    const uint32_t valid = (uint32_t)min((uint64_t)kTile, b1 - base);
    uint32_t *bk = buf[cur] + mis, *bv = buf[cur] + kSpan + mis;
    // the other buffer was last written (by this block's scatter) before the
    // fence and barrier that ended the previous tile
    if (tid == 0 && t + 1 < ntile) issue(t + 1);
    const bool ok = mbar_wait_bounded(&s_bar[cur], parity[cur], first_polls);
    // keys past the last whole 16-byte group come by plain loads; a tile
    // that ends before the first group boundary (mis + valid < 4: nothing
    // was copied) loads all its keys that way.  The start stays unsigned
    // and in [0, valid]: (whole - mis) alone would wrap below zero there.
    const uint32_t whole = (mis + valid) & ~3u;
    const uint32_t tail0 = whole ? whole - mis : 0u;
    if (tid < (int)(valid - tail0)) {
      bk[tail0 + tid] = __ldg(kin + base + tail0 + tid);
      if (kV) bv[tail0 + tid] = __ldg(vin + base + tail0 + tid);
    }
    for (int i = tid; i < kWarps * C::kR / 2; i += kThreads) reinterpret_cast<uint32_t *>(s_wcnt)[i] = 0;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        s_abort = 1;
        // copies in flight: tile t (not yet arrived) and tile t + 1 if issued
        mbar_wait_bounded(&s_bar[cur], parity[cur]);
        if (t + 1 < ntile) mbar_wait_bounded(&s_bar[cur ^ 1], parity[cur ^ 1]);
      }
      break;
    }
    parity[cur] ^= 1u;
    uint32_t key[C::kItems], rank[C::kItems];
    // a tile whose keys all share one digit keeps its order: its run goes
    // out as it is (tried only where that is likely -- the top byte of the
    // depths, which all lie within a binade or two -- since the check costs
    // a pass over the tile)
    if (!kLast && try_single) {
      const uint32_t d0 = (bk[0] >> shift) & mask;   // valid >= 1 here
      bool same = true;
#pragma unroll
      for (int j = 0; j < C::kItems; ++j) {
        const uint32_t li = (uint32_t)(warp * 32 * C::kItems + j * 32 + lane);
        if (li < valid) same = same && ((bk[li] >> shift) & mask) == d0;
      }
      if (__syncthreads_and(same)) {
        const uint64_t o0 = s_gbase[d0];
        bool bad = false;
        for (uint32_t i = tid; i < valid; i += kThreads) {
          const uint64_t o = (uint64_t)o0 + i;
          if (o >= n) {   // a histogram out of step with the keys: never write past the items
            bad = true;
            continue;
          }
          kout[o] = bk[i];
          if (kV) vout[o] = bv[i];
        }
        if (bad) {
          atomicOr(&status->flags, PK_DEV_BOUNDS);
          *abort_flag = 1u;
        }
        __syncthreads();
        if (tid == 0) s_gbase[d0] = o0 + valid;
        fence_proxy_async();   // this buffer's generic reads before the next TMA into it
        __syncthreads();
        continue;
      }
    }
    // stable warp-level ranking: items in (warp, item, lane) order
#pragma unroll
    for (int j = 0; j < C::kItems; ++j) {
      const uint32_t li = (uint32_t)(warp * 32 * C::kItems + j * 32 + lane);
      const bool in = li < valid;
      key[j] = in ? bk[li] : 0xffffffffu;
      const uint32_t d = in ? ((key[j] >> shift) & mask) : (uint32_t)(C::kR - 1);
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t before = __popc(peers & lt);
      const uint32_t c = wc[d];
      rank[j] = c + before;
      __syncwarp();
      if (before == 0) wc[d] = (uint16_t)(c + __popc(peers));
      __syncwarp();
    }
    __syncthreads();
    // per digit: prefix over warps (in place), then over digits
    uint32_t dcount[C::kPerThread];
    uint32_t tsum = 0;
#pragma unroll
    for (int u = 0; u < C::kPerThread; ++u) {
      const int d = tid * C::kPerThread + u;
      uint32_t sum = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_wcnt[w * C::kR + d];
        s_wcnt[w * C::kR + d] = (uint16_t)sum;
        sum += c;
      }
      dcount[u] = sum;
      tsum += sum;
    }
    uint32_t tot;
    uint32_t run = block_excl_scan<uint32_t>(tsum, tot, s_scan);
#pragma unroll
    for (int u = 0; u < C::kPerThread; ++u) {
      s_start[tid * C::kPerThread + u] = run;
      run += dcount[u];
    }
    // values of this thread's items, read before the in-place permutation
    uint32_t val[C::kItems];
#pragma unroll
    for (int j = 0; j < C::kItems; ++j) {
      const uint32_t li = (uint32_t)(warp * 32 * C::kItems + j * 32 + lane);
      val[j] = kV && li < valid ? bv[li] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < C::kItems; ++j) {
      const uint32_t li = (uint32_t)(warp * 32 * C::kItems + j * 32 + lane);
      const bool in = li < valid;
      const uint32_t d = in ? ((key[j] >> shift) & mask) : (uint32_t)(C::kR - 1);
      const uint32_t r = s_start[d] + wc[d] + rank[j];
      bk[r] = key[j];
      if (kV) bv[r] = val[j];
    }
    __syncthreads();
    for (uint32_t i = tid; i < valid; i += kThreads) {
      const uint32_t k = bk[i];
      const uint32_t d = (k >> shift) & mask;
      const uint64_t o = s_gbase[d] + (i - s_start[d]);
      if (o >= n) {   // a histogram out of step with the keys: never write past the items
        atomicOr(&status->flags, PK_DEV_BOUNDS);
        *abort_flag = 1u;
        continue;
      }
      if (kLast) {
        // a tile's entries are one run here (same digit, and the earlier
        // passes left them together), so its first and last write the range
        const uint32_t lt = k >> up.pbits;
        const uint64_t tile = (uint64_t)tile0 + lt, gp = pid0 + (k & ((1u << up.pbits) - 1u));
        if (tile >= tile1 || gp >= up.npairs) {   // a word that names no tile or pair
          atomicOr(&status->flags, PK_DEV_BOUNDS);
          *abort_flag = 1u;
          continue;
        }
        vout[o] = (uint32_t)gp;
        if (i == 0 || (bk[i - 1] >> up.pbits) != lt)
          atomicMax(reinterpret_cast<unsigned long long *>(up.ranges + 2 * tile), (unsigned long long)~o);
        if (i + 1 == valid || (bk[i + 1] >> up.pbits) != lt)
          atomicMax(reinterpret_cast<unsigned long long *>(up.ranges + 2 * tile + 1), (unsigned long long)(o + 1));
      } else {
        kout[o] = k;
        if (kV) vout[o] = bv[i];
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < C::kPerThread; ++u) s_gbase[tid * C::kPerThread + u] += dcount[u];
    fence_proxy_async();   // this buffer's generic writes before the next TMA into it
    __syncthreads();
  }
  if (s_abort && tid == 0) {
    atomicOr(&status->flags, PK_DEV_TIMEOUT);
    *abort_flag = 1u;
  }
}

// ---------------------------------------------------------------------------
// Emission: one (tile, pair) entry per touched tile, warp-cooperative so
// that the stores of a warp are contiguous.
// ---------------------------------------------------------------------------

// What a lane of the emission walk reads of the pair that owns its
// candidate: everything it needs comes from shared memory in two 16-byte
// loads (three more for a footprint of more than 64 candidates), instead of
// one shuffle per value.
struct EmitPair {
  int4 c;      // key of the first candidate tile, tiles per view row (bit 31: > 64 candidates), width w, 1/w bits
  uint4 e;     // first candidate's index in the warp's walk, value, receiving mask (low, high)
};
struct EmitFoot {
  float4 g0, g1;   // the footprint (mx, my, a, b), (c, 1/a, 1/c, 2b)
  int4 r;          // first candidate tile (x, y), view width and height
};

__global__ __launch_bounds__(kThreads) void k_emit(const float *__restrict__ rec, const uint32_t *__restrict__ pval,
                                                   const uint64_t *__restrict__ offs, const uint4 *__restrict__ pinfo,
                                                   DevCounters *ctr, const DevView *__restrict__ views,
                                                   int64_t N, int64_t pairs, int T, int mode, int local_bits,
                                                   int pbits, uint32_t *__restrict__ keys,
                                                   uint32_t *__restrict__ vals, pk_device_status *status) {
  __shared__ EmitPair s_ep[kWarps][32];
  __shared__ EmitFoot s_ef[kWarps][32];
  const uint64_t dups = ctr->dups;
  if (dups == 0) return;
  const uint64_t n = ctr->n_valid;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt = lanemask_lt();
  const uint64_t nwarps = (uint64_t)gridDim.x * kWarps;
  for (uint64_t w = blockIdx.x * (uint64_t)kWarps + warp; w * 32 < n; w += nwarps) {
    const uint64_t k = w * 32 + lane;
    uint32_t ncand = 0;
    EmitPair ep;
    ep.c = make_int4(0, 0, 1, __float_as_int(1.f));
    ep.e = make_uint4(0u, 0u, 0u, 0u);
    if (k < n) {
      // the count pass left the candidate rectangle and, for up to 64
      // candidates, the mask of the receiving ones: the record is read
      // again only for a larger footprint
      uint32_t p = pval[k];
      if ((uint64_t)p >= (uint64_t)pairs) {   // never index past the pairs
        atomicOr(&status->flags, PK_DEV_BOUNDS);
        ctr->sort_abort = 1u;
        p = 0;
      }
      const uint4 info = __ldg(pinfo + p);
      const int x0 = (int)(info.z & 0xffffu), y0 = (int)(info.z >> 16);
      const int wt = (int)(info.w & 0xffffu), ht = (int)(info.w >> 16);
      ncand = (uint32_t)(wt * ht);
      if (ncand) {
        const uint32_t vi = p / (uint32_t)N;
        const DevView &v = views[vi];
        const bool large = mode != PK_BIN_RECT && ncand > kMaskBits;
        if (large) {
          const float4 a = __ldg(reinterpret_cast<const float4 *>(rec + (uint64_t)p * kRec));
          const float4 b = __ldg(reinterpret_cast<const float4 *>(rec + (uint64_t)p * kRec) + 1);
          const Foot f = make_foot(a.x, a.y, a.z, a.w, b.x);
          EmitFoot ef;
          ef.g0 = make_float4(f.mx, f.my, f.a, f.b);
          ef.g1 = make_float4(f.c, f.ra, f.rc, f.b2);
          ef.r = make_int4(x0, y0, v.width, v.height);
          s_ef[warp][lane] = ef;
        }
        // key: the global tile id, or (segmented sort) the view above the
        // local tile id, whose low local_bits bits alone are sorted.
        // Packed (pbits > 0): one word, the tile id (local to the view in a
        // segmented sort) above the pair index (local to the view there too)
        const uint32_t kbase = pbits ? (local_bits ? 0u : (uint32_t)v.tile_off)
                                     : (local_bits ? (vi << local_bits) : (uint32_t)v.tile_off);
        const uint32_t pw = pbits && local_bits ? p - vi * (uint32_t)N : p;
        ep.c = make_int4((int)(kbase + (uint32_t)y0 * v.tiles_x + (uint32_t)x0),
                         v.tiles_x | (large ? (int)0x80000000u : 0), wt, __float_as_int(__frcp_rn((float)wt)));
        ep.e = make_uint4(0u, pw, info.x, info.y);
      }
    }
    uint64_t off0 = 0;
    if (lane == 0) off0 = offs[w * 32];
    off0 = __shfl_sync(0xffffffffu, off0, 0);
    const uint32_t incl = warp_incl_scan(ncand);
    ep.e.x = incl - ncand;
    s_ep[warp][lane] = ep;
    __syncwarp();
    const uint32_t E = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t written = 0;
    for (uint32_t e0 = 0; e0 < E; e0 += 32) {
      const uint32_t e = e0 + lane;
      const uint32_t ee = e < E ? e : E - 1;
      const int o = candidate_owner(incl, ee);
      const int4 c = s_ep[warp][o].c;
      const uint4 oe = s_ep[warp][o].e;
      const uint32_t local = ee - oe.x;
      uint32_t ly, lx;
      divmod_small(local, (uint32_t)c.z, __int_as_float(c.w), ly, lx);
      bool take = e < E;
      const bool large = c.y < 0;
      if (take && mode != PK_BIN_RECT) {
        if (!large) {
          take = ((local < 32 ? oe.z >> local : oe.w >> (local - 32)) & 1u) != 0u;
        } else {
          const EmitFoot &ef = s_ef[warp][o];
          const float4 g0 = ef.g0, g1 = ef.g1;
          const int4 r = ef.r;
          const Foot f{g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
          take = tile_hit(f, r.x + (int)lx, r.y + (int)ly, r.z, r.w, T);
        }
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, take);
      if (take) {
        const uint64_t at = off0 + written + __popc(bal & lt);
        if (at < dups) {
          const uint32_t key = (uint32_t)c.x + ly * (uint32_t)(c.y & 0x7fffffff) + lx;
          if (pbits) {
            keys[at] = (key << pbits) | oe.y;
          } else {
            keys[at] = key;
            vals[at] = oe.y;
          }
        } else {   // more receiving tiles than counted: never write past the entries
          atomicOr(&status->flags, PK_DEV_BOUNDS);
          ctr->sort_abort = 1u;
        }
      }
      written += __popc(bal);
    }
    __syncwarp();
  }
}

// Tile ranges from the sorted tile ids; four entries per thread.
// Per-tile [start, end) of the sorted entries (64-bit positions).  Keys
// are global tile ids, or (local_bits > 0) the view above a per-view local
// tile id: then the view's tile_off is added to the local id.
__global__ __launch_bounds__(kThreads) void k_ranges(const uint32_t *__restrict__ keys, int local_bits,
                                                     const uint32_t *__restrict__ toff, const DevCounters *ctr,
                                                     uint64_t *__restrict__ ranges, int V, uint32_t n_tiles,
                                                     pk_device_status *status) {
  const uint64_t n = ctr->sort_abort ? 0u : ctr->dups;   // a pass gave up: every range stays empty
  const uint64_t nq = (n + 3) / 4;
  const uint32_t lmask = (1u << local_bits) - 1u;
  for (uint64_t q = blockIdx.x * (uint64_t)kThreads + threadIdx.x; q < nq; q += (uint64_t)gridDim.x * kThreads) {
    const uint64_t i0 = 4 * q;
    uint32_t k[6];   // tile ids of entries i0 - 1 .. i0 + 4
    k[0] = i0 ? __ldg(keys + i0 - 1) : 0xffffffffu;
    if (i0 + 3 < n) {
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(keys + i0));
      k[1] = v.x; k[2] = v.y; k[3] = v.z; k[4] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) k[1 + j] = i0 + j < n ? __ldg(keys + i0 + j) : 0xffffffffu;
    }
    k[5] = i0 + 4 < n ? __ldg(keys + i0 + 4) : 0xffffffffu;
    bool bad = false;
    if (local_bits) {
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if (k[j] != 0xffffffffu) {
          const uint32_t v = k[j] >> local_bits;
          bad |= v >= (uint32_t)V;
          k[j] = v < (uint32_t)V ? __ldg(toff + v) + (k[j] & lmask) : 0xffffffffu;
        }
    }
#pragma unroll
    for (int j = 1; j < 5; ++j) bad |= i0 + j - 1 < n && k[j] >= n_tiles;
    if (bad) {   // a key that names no tile: record it, write nothing
      atomicOr(&status->flags, PK_DEV_BOUNDS);
      continue;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t i = i0 + j;
      if (i >= n) break;
      const uint32_t t = k[1 + j];
      if (i == 0 || k[j] != t) ranges[2 * (size_t)t] = i;
      if (i + 1 == n || k[2 + j] != t) ranges[2 * (size_t)t + 1] = i + 1;
    }
  }
}

// Tile ranges after the last packed pass, which left start as the largest
// ~position (0: no entry) and end as the largest position + 1.  A call
// that gave up leaves every range empty.
__global__ __launch_bounds__(kThreads) void k_range_fix(uint64_t *__restrict__ ranges, uint32_t n_tiles,
                                                        const DevCounters *ctr) {
  const bool gave_up = ctr->sort_abort != 0;
  for (uint32_t t = blockIdx.x * kThreads + threadIdx.x; t < n_tiles; t += gridDim.x * kThreads) {
    const uint64_t a = ranges[2 * (size_t)t];
    if (gave_up || a == 0ull) {
      ranges[2 * (size_t)t] = 0ull;
      ranges[2 * (size_t)t + 1] = 0ull;
    } else {
      ranges[2 * (size_t)t] = ~a;
    }
  }
}

// Where every view's items start, the pairs being grouped by view (pair
// pid belongs to view pid / N): one thread per view finds the first pair
// with pid >= v N by binary search.  kEntries: seg[v] = offs of that pair
// (the total number of entries where no such pair is left), else seg[v] =
// its index (n where none is left); seg[V] = the total.
template <bool kEntries>
__global__ __launch_bounds__(kThreads) void k_view_segments(const uint32_t *__restrict__ pval,
                                                            const uint64_t *__restrict__ offs,
                                                            const DevCounters *ctr, uint32_t N, int V,
                                                            uint64_t *__restrict__ seg) {
  const uint32_t n = (uint32_t)ctr->n_valid;   // valid pairs < 2^32 (pair indices are 32-bit)
  const uint64_t total = kEntries ? ctr->dups : n;
  for (int v = blockIdx.x * kThreads + threadIdx.x; v <= V; v += gridDim.x * kThreads) {
    if (n == 0 || total == 0) {
      seg[v] = 0;
      continue;
    }
    const uint64_t first = (uint64_t)v * N;
    uint32_t lo = 0, hi = n;   // first index with pval >= first
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo) / 2;
      if ((uint64_t)pval[mid] < first) lo = mid + 1; else hi = mid;
    }
    seg[v] = lo == n ? total : (kEntries ? offs[lo] : lo);
  }
}

template <int RB, int IT, int kMode>
pk_status radix_pass_rb(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                        const uint64_t *n_dev, uint64_t n_host, int shift, int bits, uint64_t *hist, int nblocks,
                        uint64_t *csum, pk_device_status *status, SegSpec sp, uint32_t *abort_flag,
                        uint32_t first_polls, bool try_single, const Unpack &up, cudaStream_t st) {
  using C = Radix<RB, IT>;
  if (cudaFuncSetAttribute(k_radix_downsweep<RB, IT, kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)Down<RB, IT>::kSmem) != cudaSuccess)
    return PK_ERR_CUDA;
  const uint32_t mask = (1u << bits) - 1u;
  k_radix_upsweep<RB, IT><<<nblocks, kThreads, 0, st>>>(kin, n_dev, n_host, shift, mask, hist, sp);
  const int count = C::kR * nblocks, nchunks = (count + kHistChunk - 1) / kHistChunk;
  k_radix_chunk_sums<<<nchunks, 1024, 0, st>>>(hist, count, csum);
  k_radix_scan_chunks<<<nchunks, 1024, 0, st>>>(hist, count, csum);
  k_radix_downsweep<RB, IT, kMode><<<nblocks, kThreads, Down<RB, IT>::kSmem, st>>>(
      kin, vin, kout, vout, n_dev, n_host, shift, mask, hist, status, sp, abort_flag, first_polls, try_single, up);
  return check_launch();
}

// One stable pass over key bits [shift, shift + bits), bits <= 8, over the
// depth-sorted pairs (pair_blocks() blocks) or over the entries
// (sort_blocks() blocks, or the segmented table's), with digits of up to
// rb = 8 or 11 bits (pk_options.sort_bits_*: wider digits take fewer passes
// but run fewer blocks per SM and scatter into more runs).  vin == nullptr:
// packed entries, keys only; then up.ranges != nullptr marks the last pass.
pk_status radix_pass(bool entries, int rb, const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                     const uint64_t *n_dev, uint64_t n_host, int shift, int bits, uint64_t *hist, int nblocks,
                     uint64_t *csum, pk_device_status *status, uint32_t *abort_flag, uint32_t first_polls,
                     bool try_single, cudaStream_t st, SegSpec sp = SegSpec{nullptr, nullptr},
                     Unpack up = Unpack{}) {
#define PK_PASS(RB, IT, M)                                                                                        \
  return radix_pass_rb<RB, IT, M>(kin, vin, kout, vout, n_dev, n_host, shift, bits, hist, nblocks, csum, status, \
                                  sp, abort_flag, first_polls, try_single, up, st)
  if (entries) {
    if (!vin && up.ranges) {
      if (rb > 8) PK_PASS(11, kEntryItems, 2);
      PK_PASS(8, kEntryItems, 2);
    }
    if (!vin) {
      if (rb > 8) PK_PASS(11, kEntryItems, 1);
      PK_PASS(8, kEntryItems, 1);
    }
    if (rb > 8) PK_PASS(11, kEntryItems, 0);
    PK_PASS(8, kEntryItems, 0);
  }
  if (rb > 8) PK_PASS(11, kPairItems, 0);
  PK_PASS(8, kPairItems, 0);
#undef PK_PASS
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, sms);
}

// Blocks of the pair passes: resident ones, within the histogram.
int pair_blocks(int rb) {
  const int per_sm = rb > 8 ? Radix<11, kPairItems>::kMinBlocks : Radix<8, kPairItems>::kMinBlocks;
  return std::max(1, std::min(kSortBlocks, per_sm * sm_count()));
}

}  // namespace

// Blocks of the entry passes on this device.
int pk::sort_blocks(int rb) {
  // the entry passes' resident blocks, leaving the histogram room for the
  // segmented table's one extra block per view
  const int per_sm = rb > 8 ? Radix<11, kEntryItems>::kMinBlocks : Radix<8, kEntryItems>::kMinBlocks;
  return std::max(1, std::min(kSortBlocks - 128, per_sm * sm_count()));
}

namespace {

// Block table of a segmented sort: per view a share of `nblocks`
// proportional to weight(v) (at least one), each {view, part, parts, first
// histogram counter}.  Returns the number of blocks, or 0 when the views do
// not fit the histogram.
template <typename Weight>
int share_blocks(int V, int nblocks, int rb, const Weight &weight, int4 *tab) {
  int64_t total = 0;
  for (int v = 0; v < V; ++v) total += weight(v);
  int nb = 0;
  for (int v = 0; v < V; ++v) {
    const int parts = std::max<int>(1, (int)((int64_t)nblocks * weight(v) / std::max<int64_t>(1, total)));
    if (nb + parts > kSortBlocks) return 0;
    for (int j = 0; j < parts; ++j) tab[nb + j] = make_int4(v, j, parts, (1 << rb) * nb);
    nb += parts;
  }
  return nb;
}

}  // namespace

// The tile passes' table (shares by tiles) and the depth passes' (equal
// shares: every view has N pairs at most); false when the plan sorts
// unsegmented (one view, or too many views for the histogram).
bool pk::seg_tables(const pk_plan *p, int4 *tab, int *ntile, int *npair) {
  *ntile = *npair = 0;
  if (p->V < 2) return false;
  const int rt = p->opts.sort_bits_tile, rd = p->opts.sort_bits_depth;
  const int nt = share_blocks(p->V, sort_blocks(rt), rt,
                              [&](int v) { return (int64_t)p->h_views[v].tiles_x * p->h_views[v].tiles_y; },
                              tab);
  const int np = share_blocks(p->V, pair_blocks(rd), rd, [](int) { return int64_t(1); }, tab + kSortBlocks);
  if (nt == 0 || np == 0) return false;
  *ntile = nt;
  *npair = np;
  return true;
}

namespace {

// Digit widths for a key of `bits` bits: as few passes of <= maxw bits as
// possible, split evenly.
int radix_plan(int bits, int maxw, int *widths) {
  const int npass = (bits + maxw - 1) / maxw;
  for (int i = 0, left = bits; i < npass; ++i) {
    widths[i] = (left + (npass - i) - 1) / (npass - i);
    left -= widths[i];
  }
  return npass;
}

// Bits of the largest per-view tile id (the digits of the segmented sort).
int local_tile_bits(const pk_plan *p) {
  int64_t most = 1;
  for (int v = 0; v < p->V; ++v)
    most = std::max<int64_t>(most, (int64_t)p->h_views[v].tiles_x * p->h_views[v].tiles_y);
  int bits = 1;
  while ((int64_t(1) << bits) < most) ++bits;
  return bits;
}

// The whole binning + sort on one workspace layout (shared by the two
// entry points below).
pk_status bin_and_sort_impl(const pk_plan *p, const WsLayout &L, void *ws, const float *records,
                            uint32_t *sorted_vals, uint64_t *tile_ranges, uint64_t maxd, cudaStream_t st) {
  const DevView *views = at<DevView>(ws, L.views);
  DevCounters *ctr = at<DevCounters>(ws, L.counters);
  pk_device_status *status = at<pk_device_status>(ws, L.status);
  uint32_t *cnt = at<uint32_t>(ws, L.pair_cnt);
  uint32_t *zk[2] = {at<uint32_t>(ws, L.zkey0), at<uint32_t>(ws, L.zkey1)};
  uint32_t *pv[2] = {at<uint32_t>(ws, L.pval0), at<uint32_t>(ws, L.pval1)};
  uint64_t *offs = at<uint64_t>(ws, L.offs);
  uint4 *pinfo = at<uint4>(ws, L.rmask);
  uint64_t *bsum = at<uint64_t>(ws, L.blocksums);
  uint64_t *hist = at<uint64_t>(ws, L.hist);
  uint32_t *dk0 = at<uint32_t>(ws, L.dkey0), *dk1 = at<uint32_t>(ws, L.dkey1);
  uint32_t *dv = at<uint32_t>(ws, L.dval);
  const uint64_t *n_valid = &ctr->n_valid;
  const uint64_t pairs = (uint64_t)p->pairs;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // segmented sorts (V >= 2): the depth passes sort each view's pairs in
  // place, the tile passes each view's entries on per-view local tile ids
  int4 tab_host[2 * kSortBlocks];
  int nseg = 0, npseg = 0;
  const bool seg = seg_tables(p, tab_host, &nseg, &npseg);
  const int4 *tab = at<int4>(ws, L.sblk);
  uint64_t *vseg = at<uint64_t>(ws, L.vseg), *pseg = vseg + (p->V + 1);

  pk_status ze = zero_async({{tile_ranges, sizeof(uint64_t) * 2 * (size_t)p->n_tiles},
                             {ctr, pairs == 0 ? sizeof(DevCounters) : 0},
                             {&ctr->sort_abort, pairs == 0 ? 0 : sizeof(uint32_t)}},
                            st);
  if (ze != PK_OK || pairs == 0) return ze;
  const int cblocks = (int)std::min<uint64_t>((pairs + kThreads - 1) / kThreads, 152 * 16);
  k_pair_count<<<cblocks, kThreads, 0, st>>>(records, p->pairs, p->N, views, p->T, p->opts.bin_mode, cnt, pinfo,
                                              zk[1]);
  // compaction of the pairs that touch a tile, keyed by depth bits
  k_scan_reduce<SrcValid><<<kScanBlocks, kThreads, 0, st>>>(SrcValid{cnt}, nullptr, pairs, bsum);
  k_scan_top<<<1, 1024, 0, st>>>(bsum, kScanBlocks, 0, maxd, ctr, status);
  k_compact_down<<<kScanBlocks, kThreads, 0, st>>>(cnt, zk[1], pairs, bsum, zk[0], pv[0]);
  // depth sort of the pairs: stable passes over the 32 bits of z; the
  // compaction kept the (view, Gaussian) order, so sorting inside each
  // view's segment leaves the pairs in (view, depth) order
  SegSpec psp{nullptr, nullptr};
  if (seg) {
    k_view_segments<false><<<(p->V + kThreads) / kThreads, kThreads, 0, st>>>(pv[0], nullptr, ctr, (uint32_t)p->N,
                                                                            p->V, pseg);
    psp = SegSpec{tab + kSortBlocks, pseg};
  }
  pk_status e;
  int widths[8];
  const int rd = p->opts.sort_bits_depth, rt = p->opts.sort_bits_tile;
  int np = radix_plan(32, rd, widths), shift = 0;
  for (int pass = 0; pass < np; ++pass) {
    const int a = pass & 1, b = a ^ 1;
    if ((e = radix_pass(false, rd, zk[a], pv[a], zk[b], pv[b], n_valid, 0, shift, widths[pass], hist,
                        seg ? npseg : pair_blocks(rd), bsum, status, &ctr->sort_abort, p->first_polls,
                        pass == np - 1, st, psp)) != PK_OK)
      return e;
    shift += widths[pass];
  }
  const uint32_t *pval = pv[np & 1];
  // emission offsets in (view,) depth order, capacity check
  uint32_t *csorted = zk[1];   // the depth keys are spent: their buffer takes the gathered counts
  k_reduce_sorted<<<kScanBlocks, kThreads, 0, st>>>(cnt, pval, pairs, n_valid, csorted, bsum);
  k_scan_top<<<1, 1024, 0, st>>>(bsum, kScanBlocks, 1, maxd, ctr, status);
  k_offsets_down<<<kScanBlocks, kThreads, 0, st>>>(csorted, n_valid, bsum, ctr, offs);
  // emission and the stable tile sort; the last pass lands in sorted_vals
  int key_bits = p->tile_bits;
  SegSpec sp{nullptr, nullptr};
  int nblocks = sort_blocks(rt);
  if (seg) {
    key_bits = local_tile_bits(p);
    k_view_segments<true><<<(p->V + kThreads) / kThreads, kThreads, 0, st>>>(pval, offs, ctr, (uint32_t)p->N, p->V,
                                                                          vseg);
    sp = SegSpec{tab, vseg};
    nblocks = nseg;
  }
  // Packed entries when the tile id and the pair index fit one word
  // together (both local to the view in a segmented sort; at the 52-view
  // rig 11 + 20 bits): the tile passes then move 4 bytes per entry
  // instead of 8, and the last one writes the pair indices and folds the
  // tile ranges in (no pass over the sorted keys).
  const uint64_t pid_end = seg ? (uint64_t)p->N : pairs;
  int pbits = 1;
  while ((uint64_t(1) << pbits) < pid_end) ++pbits;
  const bool packed = key_bits + pbits <= 32;
  np = radix_plan(key_bits, rt, widths);
  uint32_t *vbuf[2] = {(np & 1) ? dv : sorted_vals, (np & 1) ? sorted_vals : dv};
  uint32_t *kbuf[2] = {dk0, dk1};
  k_emit<<<std::max(1, sms) * 32, kThreads, 0, st>>>(records, pval, offs, pinfo, ctr, views, p->N, p->pairs, p->T,
                                                      p->opts.bin_mode, seg ? key_bits : 0, packed ? pbits : 0,
                                                      kbuf[0], vbuf[0], status);
  // Digits from the top down: each tile's entries still end up contiguous
  // and in emission order, and the first pass, whose input holds each
  // splat's tiles side by side, ranks on tile-row bands that the 32 entries
  // of a warp rarely differ in (ranking slows with the distinct digits of
  // a warp).  The tiles follow one another by (low digit, high digit)
  // instead of by id.
  shift = (packed ? pbits : 0) + key_bits;
  const Unpack up{tile_ranges, at<uint32_t>(ws, L.toff), (uint32_t)p->N, pbits, (uint32_t)p->n_tiles, pairs};
  for (int pass = 0; pass < np; ++pass) {
    const int a = pass & 1, b = a ^ 1;
    const bool last = pass + 1 == np;
    shift -= widths[pass];
    if (packed)
      e = radix_pass(true, rt, kbuf[a], nullptr, last ? nullptr : kbuf[b], last ? sorted_vals : nullptr, &ctr->dups,
                     0, shift, widths[pass], hist, nblocks, bsum, status, &ctr->sort_abort, p->first_polls, false,
                     st, sp, last ? up : Unpack{});
    else
      e = radix_pass(true, rt, kbuf[a], vbuf[a], kbuf[b], vbuf[b], &ctr->dups, 0, shift, widths[pass], hist, nblocks,
                     bsum, status, &ctr->sort_abort, p->first_polls, false, st, sp);
    if (e != PK_OK) return e;
  }
  if (packed)
    k_range_fix<<<std::max(1, sms) * 4, kThreads, 0, st>>>(tile_ranges, (uint32_t)p->n_tiles, ctr);
  else
    k_ranges<<<std::max(1, sms) * 16, kThreads, 0, st>>>(kbuf[np & 1], seg ? key_bits : 0,
                                                          at<uint32_t>(ws, L.toff), ctr, tile_ranges, p->V,
                                                          (uint32_t)p->n_tiles, status);
  return check_launch();
}

}  // namespace

// Mirrors the launches of bin_and_sort_impl: zeroing, count, scan (2),
// compaction, [pair segments], the depth passes, offsets (3), [entry
// segments], emission, the tile passes, ranges; 4 kernels per radix pass.
int pk::bin_kernel_count(const pk_plan *p) {
  if (!p) return 0;
  if (p->pairs == 0) return 1;
  int4 tab[2 * kSortBlocks];
  int nt = 0, np = 0;
  const bool seg = seg_tables(p, tab, &nt, &np);
  int widths[8];
  int passes = radix_plan(32, p->opts.sort_bits_depth, widths);
  int kernels = 1 + 4 + 3 + 1 + 1;
  if (seg) kernels += 2;   // the pairs' and the entries' view segments
  passes += radix_plan(seg ? local_tile_bits(p) : p->tile_bits, p->opts.sort_bits_tile, widths);
  return kernels + 4 * passes;
}

extern "C" pk_status pk_bin_and_sort(const pk_plan *p, const float *records, uint32_t *sorted_vals,
                                     uint64_t *tile_ranges, void *ws, pk_stream_t stream) {
  if (!p || !records || !sorted_vals || !tile_ranges || !ws) return PK_ERR_ARG;
  if (!aligned16(records) || !aligned16(sorted_vals) || (reinterpret_cast<uintptr_t>(ws) & 255u) ||
      (reinterpret_cast<uintptr_t>(tile_ranges) & 7u))
    return PK_ERR_ARG;
  return bin_and_sort_impl(p, p->ws, ws, records, sorted_vals, tile_ranges, p->max_dups,
                           reinterpret_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// Allocation-free variant of pk_bin_and_sort.
//
// Some callers cannot hand the library a workspace: a host application that
// drives the renderer from inside another framework's frame callback, where
// that framework owns every device allocation and allocating would stall
// the frame, or a small tool with no device allocator of its own.  This
// entry point keeps its scratch in one file-scope device array instead,
// sized once for every process that loads the library.
// ---------------------------------------------------------------------------

#include <cstring>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB, held by every GPU that loads the library
constexpr int kMaxDevices = 64;
__device__ __align__(256) unsigned char g_bin_scratch[kStaticScratchBytes];

std::mutex g_bin_scratch_mu;
void *g_bin_scratch_addr[kMaxDevices] = {};

// Device address of g_bin_scratch on the current device (looked up once per
// device; the host-side symbol itself is only a stand-in and must never be
// passed to a kernel).
pk_status static_scratch(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PK_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_bin_scratch_mu);
  if (!g_bin_scratch_addr[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_bin_scratch) != cudaSuccess || !ptr) return PK_ERR_CUDA;
    g_bin_scratch_addr[dev] = ptr;
  }
  *out = g_bin_scratch_addr[dev];
  return PK_OK;
}

// The call's outcome in one word: the entries, or a sentinel -- the status
// block lives in the static array, where the caller's pk_read_status cannot
// reach it.
__global__ void k_report_entries(const DevCounters *ctr, const pk_device_status *status, uint32_t *n_entries) {
  const uint32_t f = status->flags;
  *n_entries = (f & PK_DEV_CAPACITY) ? 0xffffffffu
                                     : ((f & (PK_DEV_TIMEOUT | PK_DEV_BOUNDS)) || ctr->sort_abort) ? 0xfffffffeu
                                                                                                    : (uint32_t)ctr->dups;
}

// The plan's host tables reach the static array as kernel arguments, which
// the launch itself copies: no host buffer has to stay pinned or alive
// after the call, and no copy engine is involved.  Chunks of 960 words keep
// each launch's arguments inside the 4 KB parameter space.
constexpr uint32_t kChunkWords = 960;
struct WordChunk {
  uint32_t n;
  uint32_t w[kChunkWords];
};
__global__ void k_put_words(const WordChunk c, uint32_t *__restrict__ dst) {
  for (uint32_t i = threadIdx.x; i < c.n; i += blockDim.x) dst[i] = c.w[i];
}
pk_status put_words(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  const uint32_t *s = static_cast<const uint32_t *>(src);
  uint32_t *d = static_cast<uint32_t *>(dst);
  const size_t words = bytes / 4;
  WordChunk c;
  for (size_t off = 0; off < words; off += kChunkWords) {
    c.n = (uint32_t)std::min<size_t>(kChunkWords, words - off);
    std::memcpy(c.w, s + off, sizeof(uint32_t) * c.n);
    k_put_words<<<1, 256, 0, st>>>(c, d + off);
    const pk_status e = check_launch();
    if (e != PK_OK) return e;
  }
  return PK_OK;
}

}  // namespace

extern "C" pk_status pk_bin_and_sort_noalloc(const pk_plan *p, const float *records, uint32_t *sorted_vals,
                                             uint64_t *tile_ranges, uint32_t *n_entries, pk_stream_t stream) {
  if (!p || !records || !sorted_vals || !tile_ranges || !n_entries) return PK_ERR_ARG;
  if (!aligned16(records) || !aligned16(sorted_vals) || (reinterpret_cast<uintptr_t>(tile_ranges) & 7u))
    return PK_ERR_ARG;
  // layout of this plan's scratch inside the static array
  const uint64_t pairs = (uint64_t)p->pairs, maxd = p->max_dups;
  WsLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at_ = off;
    off = (off + bytes + 255) & ~size_t(255);
    return at_;
  };
  L.status = take(sizeof(pk_device_status));
  L.counters = take(sizeof(DevCounters));
  L.views = take(sizeof(DevView) * p->V);
  L.toff = take(sizeof(uint32_t) * (p->V + 1));
  L.sblk = take(sizeof(int4) * 2 * kSortBlocks);
  L.vseg = take(sizeof(uint64_t) * 2 * (p->V + 1));
  L.pair_cnt = take(sizeof(uint32_t) * pairs);
  L.zkey0 = take(sizeof(uint32_t) * pairs);
  L.zkey1 = take(sizeof(uint32_t) * pairs);
  L.pval0 = take(sizeof(uint32_t) * pairs);
  L.pval1 = take(sizeof(uint32_t) * pairs);
  L.offs = take(sizeof(uint64_t) * pairs);
  L.rmask = take(sizeof(uint4) * pairs);
  L.blocksums = take(sizeof(uint64_t) * (kScanBlocks + 1));
  // digit counters of the widest radix pass of the plan's two sorts
  L.hist = take(sizeof(uint64_t) * (size_t(1) << std::max(p->opts.sort_bits_tile, p->opts.sort_bits_depth)) *
                kSortBlocks);
  L.dkey0 = take(sizeof(uint32_t) * maxd);
  L.dkey1 = take(sizeof(uint32_t) * maxd);
  L.dval = take(sizeof(uint32_t) * maxd);
  if (off > kStaticScratchBytes) return PK_ERR_TOO_LARGE;
  void *ws = nullptr;
  pk_status e = static_scratch(&ws);
  if (e != PK_OK) return e;

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: reset the status and
  // counters, refresh this plan's view table
  if ((e = zero_async({{at<char>(ws, L.status), L.views - L.status}}, st)) != PK_OK) return e;
  if ((e = put_words(at<char>(ws, L.views), p->h_views, sizeof(DevView) * p->V, st)) != PK_OK) return e;
  if ((e = put_words(at<char>(ws, L.toff), p->h_toff, sizeof(uint32_t) * (p->V + 1), st)) != PK_OK) return e;
  int4 tab[2 * kSortBlocks] = {};
  int nt = 0, np = 0;
  if (seg_tables(p, tab, &nt, &np) && (e = put_words(at<char>(ws, L.sblk), tab, sizeof(tab), st)) != PK_OK)
    return e;
  if ((e = bin_and_sort_impl(p, L, ws, records, sorted_vals, tile_ranges, maxd, st)) != PK_OK) return e;
  const DevCounters *ctr = at<DevCounters>(ws, L.counters);
  const pk_device_status *status = at<pk_device_status>(ws, L.status);
  k_report_entries<<<1, 1, 0, st>>>(ctr, status, n_entries);
  return check_launch();
}
