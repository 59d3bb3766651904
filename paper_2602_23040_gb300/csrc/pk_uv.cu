// UV cells (eq. uvgs2) and Max-K UV pruning (Sec. 4.2 "UV-Based Pruning").
//
// Five launches over n candidate Gaussians and an M x N map: cell and
// in-cell slot per Gaussian (one atomic per valid Gaussian on the cell's
// counter), an exclusive scan of the per-cell counts, a scatter of the
// Gaussian indices into per-cell buckets, and the rank of every Gaussian
// within its bucket by opacity (higher first, then lower index): the
// buckets hold a handful of Gaussians, so each Gaussian counts the members
// that beat it.  The cell is taken in FP64 (atan2, acos), where a
// neighbouring cell is only chosen within ~1e-15 of a cell boundary.
#include "pk_common.cuh"

using namespace pk;

namespace {

constexpr int kUvThreads = 256;
constexpr int kUvScanItems = 2048;   // counts per scan block (8 per thread)
constexpr uint32_t kInvalid = 0xFFFFFFFFu;

struct UvScratch {
  size_t slot, offs, bsum, bucket, total;
};

UvScratch uv_layout(int64_t n, int64_t cells) {
  UvScratch L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at_ = off;
    off = (off + bytes + 255) & ~size_t(255);
    return at_;
  };
  const int64_t blocks = (cells + kUvScanItems - 1) / kUvScanItems;
  L.slot = take(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  L.offs = take(sizeof(uint32_t) * (size_t)cells);
  L.bsum = take(sizeof(uint32_t) * (size_t)(blocks + 1));
  L.bucket = take(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  L.total = off;
  return L;
}

__global__ __launch_bounds__(kUvThreads) void k_uv_cell(const float *__restrict__ soa, int64_t n, int64_t stride,
                                                         int M, int N, uint32_t *__restrict__ cell,
                                                         uint32_t *__restrict__ slot, uint32_t *count) {
  const int64_t i = (int64_t)blockIdx.x * kUvThreads + threadIdx.x;
  if (i >= n) return;
  const double x = __ldg(soa + i), y = __ldg(soa + stride + i), z = __ldg(soa + 2 * stride + i);
  const float lg = __ldg(soa + 10 * stride + i);
  uint32_t c = kInvalid;
  const double rho = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
  if (rho > 0.0 && isfinite(rho) && lg == lg) {
    const double kPi = 3.14159265358979323846;
    const double su = (kPi + atan2(y, x)) / (2.0 * kPi) * M, sv = acos(z / rho) / kPi * N;
    const double u = floor(su), v = floor(sv);
    if (u >= 0.0 && u < M && v >= 0.0 && v < N) c = (uint32_t)v * (uint32_t)M + (uint32_t)u;
  }
  cell[i] = c;
  if (c != kInvalid) slot[i] = atomicAdd(count + c, 1u);
}

// Exclusive scan of counts: per-block totals, a one-block scan of those,
// then each block scans its counts from its base.
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t x, uint32_t &total, uint32_t *s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kUvThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kUvThreads / 32) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[kUvThreads / 32 - 1];
  const uint32_t excl = (warp ? s_warp[warp - 1] : 0u) + inc - x;
  __syncthreads();
  return excl;
}

__global__ __launch_bounds__(kUvThreads) void k_uv_block_sums(const uint32_t *__restrict__ count, int64_t cells,
                                                               uint32_t *__restrict__ bsum) {
  __shared__ uint32_t s_warp[32];
  constexpr int kPer = kUvScanItems / kUvThreads;
  const int64_t base = (int64_t)blockIdx.x * kUvScanItems + (int64_t)threadIdx.x * kPer;
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k)
    if (base + k < cells) acc += __ldg(count + base + k);
  uint32_t tot;
  block_scan_excl(acc, tot, s_warp);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ __launch_bounds__(kUvThreads) void k_uv_scan_sums(uint32_t *bsum, int64_t blocks) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < blocks; b0 += kUvThreads) {
    const int64_t i = b0 + threadIdx.x;
    const uint32_t x = i < blocks ? bsum[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_scan_excl(x, tot, s_warp);
    const uint32_t carry = s_carry;
    if (i < blocks) bsum[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blocks] = s_carry;
}

__global__ __launch_bounds__(kUvThreads) void k_uv_offsets(const uint32_t *__restrict__ count, int64_t cells,
                                                            const uint32_t *__restrict__ bsum,
                                                            uint32_t *__restrict__ offs) {
  __shared__ uint32_t s_warp[32];
  constexpr int kPer = kUvScanItems / kUvThreads;
  const int64_t base = (int64_t)blockIdx.x * kUvScanItems + (int64_t)threadIdx.x * kPer;
  uint32_t v[kPer], acc = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    v[k] = base + k < cells ? __ldg(count + base + k) : 0u;
    acc += v[k];
  }
  uint32_t tot;
  uint32_t run = bsum[blockIdx.x] + block_scan_excl(acc, tot, s_warp);
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (base + k < cells) offs[base + k] = run;
    run += v[k];
  }
}

__global__ __launch_bounds__(kUvThreads) void k_uv_bucket(const uint32_t *__restrict__ cell,
                                                           const uint32_t *__restrict__ slot,
                                                           const uint32_t *__restrict__ offs, int64_t n,
                                                           uint32_t *__restrict__ bucket) {
  const int64_t i = (int64_t)blockIdx.x * kUvThreads + threadIdx.x;
  if (i >= n) return;
  const uint32_t c = cell[i];
  if (c != kInvalid) bucket[offs[c] + slot[i]] = (uint32_t)i;
}

// Rank of Gaussian i among the Gaussians of its cell: those with a higher
// opacity logit, or an equal logit and a lower index, come first.
__global__ __launch_bounds__(kUvThreads) void k_uv_rank(const float *__restrict__ soa, int64_t stride,
                                                         const uint32_t *__restrict__ cell,
                                                         const uint32_t *__restrict__ offs,
                                                         const uint32_t *__restrict__ count,
                                                         const uint32_t *__restrict__ bucket, int64_t n, int K,
                                                         uint32_t *__restrict__ rank, uint8_t *__restrict__ keep) {
  const int64_t i = (int64_t)blockIdx.x * kUvThreads + threadIdx.x;
  if (i >= n) return;
  const uint32_t c = cell[i];
  if (c == kInvalid) {
    rank[i] = kInvalid;
    keep[i] = 0;
    return;
  }
  const float* logit = soa + 10 * stride;
  const float li = __ldg(logit + i);
  const uint32_t beg = offs[c], cnt = count[c];
  uint32_t r = 0;
  for (uint32_t k = 0; k < cnt; ++k) {
    const uint32_t j = __ldg(bucket + beg + k);
    const float lj = __ldg(logit + j);
    r += (lj > li || (lj == li && j < (uint32_t)i)) ? 1u : 0u;
  }
  rank[i] = r;
  keep[i] = r < (uint32_t)K ? 1 : 0;
}

}  // namespace

extern "C" uint64_t pk_uv_max_k_scratch_bytes(int64_t n, int32_t M, int32_t N) {
  if (n < 0 || M < 1 || N < 1) return 0;
  return uv_layout(n, (int64_t)M * N).total;
}

extern "C" pk_status pk_uv_max_k(const float *soa, int64_t n, int64_t stride, int32_t M, int32_t N, int32_t K,
                                 uint32_t *cell, uint32_t *rank, uint8_t *keep, uint32_t *count, void *scratch,
                                 pk_stream_t stream) {
  if (n < 0 || M < 1 || N < 1 || K < 0 || stride < n) return PK_ERR_ARG;
  const int64_t cells = (int64_t)M * N;
  if (cells >= (int64_t)kInvalid || n >= (int64_t)kInvalid) return PK_ERR_ARG;
  if (!count || !scratch || (n > 0 && (!soa || !cell || !rank || !keep))) return PK_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(scratch) & 255u) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const UvScratch L = uv_layout(n, cells);
  uint32_t *slot = at<uint32_t>(scratch, L.slot), *offs = at<uint32_t>(scratch, L.offs);
  uint32_t *bsum = at<uint32_t>(scratch, L.bsum), *bucket = at<uint32_t>(scratch, L.bucket);
  pk_status ze = zero_async({{count, sizeof(uint32_t) * (size_t)cells}}, st);
  if (ze != PK_OK) return ze;
  if (n == 0) return PK_OK;
  const unsigned gn = (unsigned)((n + kUvThreads - 1) / kUvThreads);
  const int64_t blocks = (cells + kUvScanItems - 1) / kUvScanItems;
  k_uv_cell<<<gn, kUvThreads, 0, st>>>(soa, n, stride, M, N, cell, slot, count);
  k_uv_block_sums<<<(unsigned)blocks, kUvThreads, 0, st>>>(count, cells, bsum);
  k_uv_scan_sums<<<1, kUvThreads, 0, st>>>(bsum, blocks);
  k_uv_offsets<<<(unsigned)blocks, kUvThreads, 0, st>>>(count, cells, bsum, offs);
  k_uv_bucket<<<gn, kUvThreads, 0, st>>>(cell, slot, offs, n, bucket);
  k_uv_rank<<<gn, kUvThreads, 0, st>>>(soa, stride, cell, offs, count, bucket, n, K, rank, keep);
  return check_launch();
}
