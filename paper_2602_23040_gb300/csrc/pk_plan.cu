// Host side of the C ABI: atlas layout, plan validation, workspace layout,
// status read-back, and the one zeroing kernel the other calls share.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "pk_common.cuh"
#include "pk_tma.cuh"

using namespace pk;

namespace pk {

pk_status check_launch() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PK_OK : PK_ERR_CUDA;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

namespace {

struct ZeroSpans {
  uint32_t *p[4];
  uint64_t n[4];   // 32-bit words
  int k;
};

// Zeroes up to four word ranges: 16-byte stores over each range's aligned
// body, single words at its ends.
__global__ __launch_bounds__(256) void k_zero(ZeroSpans z) {
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  for (int s = 0; s < z.k; ++s) {
    uint32_t *p = z.p[s];
    const uint64_t n = z.n[s];
    const uint64_t head = std::min<uint64_t>(n, ((16u - (reinterpret_cast<uintptr_t>(p) & 15u)) & 15u) / 4u);
    const uint64_t n4 = (n - head) / 4;
    if (tid < head) p[tid] = 0u;
    uint4 *q = reinterpret_cast<uint4 *>(p + head);
    for (uint64_t i = tid; i < n4; i += nt) q[i] = make_uint4(0u, 0u, 0u, 0u);
    const uint64_t tail = head + 4 * n4;
    if (tid < n - tail) p[tail + tid] = 0u;
  }
}

// Status block and counters -> host memory mapped into the device: one
// block's stores, no copy engine.  (A device-to-host copy can queue on a
// copy engine behind the caller's unrelated host-to-device copies of
// another stream -- the next iteration's inputs -- and wait for them.)
__global__ void k_status_out(const uint32_t *__restrict__ st, int nst, const uint32_t *__restrict__ ctr, int nctr,
                             uint32_t *host_st, uint32_t *host_ctr) {
  for (int i = threadIdx.x; i < nst; i += blockDim.x) host_st[i] = st[i];
  for (int i = threadIdx.x; i < nctr; i += blockDim.x) host_ctr[i] = ctr[i];
}

}  // namespace

// One kernel instead of cudaMemsetAsync: inside a CUDA graph a memset node
// may be run by a copy engine, where it queues behind (and is delayed by)
// unrelated host <-> device copies of other streams.
pk_status zero_async(std::initializer_list<std::pair<void *, size_t>> spans, cudaStream_t st) {
  ZeroSpans z{};
  uint64_t most = 0;
  for (const auto &sp : spans) {
    if (z.k == 4 || (reinterpret_cast<uintptr_t>(sp.first) & 3u) || (sp.second & 3u)) return PK_ERR_ARG;
    if (sp.second == 0) continue;
    z.p[z.k] = static_cast<uint32_t *>(sp.first);
    z.n[z.k] = sp.second / 4;
    most = std::max<uint64_t>(most, z.n[z.k]);
    ++z.k;
  }
  if (z.k == 0) return PK_OK;
  const uint64_t blocks = std::min<uint64_t>(std::max<uint64_t>(1, (most / 4 + 255) / 256), 152 * 8);
  k_zero<<<(unsigned)blocks, 256, 0, st>>>(z);
  return check_launch();
}

}  // namespace pk

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

extern "C" int32_t pk_version(void) { return PK_VERSION; }

extern "C" const char *pk_status_string(pk_status s) {
  switch (s) {
    case PK_OK: return "ok";
    case PK_ERR_ARG: return "invalid argument";
    case PK_ERR_DESC: return "invalid atlas descriptor or view table";
    case PK_ERR_CAPACITY: return "device capacity exceeded";
    case PK_ERR_TIMEOUT: return "device wait timed out";
    case PK_ERR_CUDA: return "CUDA runtime error";
    case PK_ERR_UNSUPPORTED: return "unsupported option";
    case PK_ERR_TOO_LARGE: return "problem larger than the fixed scratch of the allocation-free call";
  }
  return "unknown status";
}

// Sec. 4.1: level k of the pyramid has (M_k, N_k) = (M_{k-1}, N_{k-1}/2) for
// odd k and (M_{k-1}/2, N_{k-1}) for even k; native width M_k (along u),
// height N_k (along v).  Packing: L0 at the right, L1 turned CCW in the
// left column, L2 under it, deeper levels in the strip under L0 from the
// right edge of L2 on, odd ones turned.
extern "C" pk_status pk_atlas_layout(int32_t S, int32_t K, pk_atlas_desc *d) {
  if (!d || S < 2 || K < 1 || K > PK_MAX_LEVELS) return PK_ERR_ARG;
  int32_t M[PK_MAX_LEVELS], N[PK_MAX_LEVELS];
  M[0] = S;
  N[0] = S;
  for (int k = 1; k < K; ++k) {
    M[k] = (k & 1) ? M[k - 1] : M[k - 1] / 2;
    N[k] = (k & 1) ? N[k - 1] / 2 : N[k - 1];
    if (M[k] < 1 || N[k] < 1) return PK_ERR_ARG;
  }
  int32_t W = 0, H = 0, strip_x = 0;
  for (int k = 0; k < K; ++k) {
    pk_level &l = d->level[k];
    bool turned = (k & 1) != 0;
    l.rotated = turned ? 1 : 0;
    l.w = turned ? N[k] : M[k];
    l.h = turned ? M[k] : N[k];
    if (K == 1) {
      l.x0 = 0;
      l.y0 = 0;
    } else if (k == 0) {
      l.x0 = N[1];   // right of the left column (width of the turned L1)
      l.y0 = 0;
    } else if (k == 1) {
      l.x0 = 0;
      l.y0 = 0;
    } else if (k == 2) {
      l.x0 = 0;
      l.y0 = M[1];
      strip_x = l.w;
    } else {
      l.x0 = strip_x;
      l.y0 = M[1];
      strip_x += l.w;
    }
    if (l.x0 + l.w > W) W = l.x0 + l.w;
    if (l.y0 + l.h > H) H = l.y0 + l.h;
  }
  for (int k = K; k < PK_MAX_LEVELS; ++k) d->level[k] = pk_level{0, 0, 0, 0, 0};
  d->num_levels = K;
  d->atlas_w = W;
  d->atlas_h = H;
  return PK_OK;
}

static bool finite_view(const pk_view &v) {
  for (int i = 0; i < 9; ++i)
    if (!isfinite(v.R[i])) return false;
  for (int i = 0; i < 3; ++i)
    if (!isfinite(v.t[i])) return false;
  return isfinite(v.fx) && isfinite(v.fy) && isfinite(v.cx) && isfinite(v.cy) && v.fx > 0 && v.fy > 0;
}

extern "C" pk_status pk_plan_create(const pk_atlas_desc *desc, const pk_view *views, int32_t n_views,
                                    int64_t n_live, const pk_options *opts, pk_plan **out) {
  if (!out) return PK_ERR_ARG;
  *out = nullptr;
  if (!desc || !views || n_views < 1 || n_views > PK_MAX_VIEWS || n_live < 0) return PK_ERR_ARG;
  const pk_atlas_desc &d = *desc;
  if (d.atlas_w < 1 || d.atlas_h < 1 || d.atlas_w > 65536 || d.atlas_h > 65536) return PK_ERR_DESC;
  if (d.num_levels < 1 || d.num_levels > PK_MAX_LEVELS) return PK_ERR_DESC;
  if (d.sh_degree < 0 || d.sh_degree > 3 || d.frames < 1 || d.frames > 4096) return PK_ERR_DESC;
  if (d.texel_type != PK_TEXEL_F32 && d.texel_type != PK_TEXEL_F16) return PK_ERR_DESC;
  for (int k = 0; k < d.num_levels; ++k) {
    const pk_level &a = d.level[k];
    if (a.w < 1 || a.h < 1 || a.x0 < 0 || a.y0 < 0 || a.x0 + a.w > d.atlas_w || a.y0 + a.h > d.atlas_h)
      return PK_ERR_DESC;
    for (int j = 0; j < k; ++j) {
      const pk_level &b = d.level[j];
      bool apart = a.x0 >= b.x0 + b.w || b.x0 >= a.x0 + a.w || a.y0 >= b.y0 + b.h || b.y0 >= a.y0 + a.h;
      if (!apart) return PK_ERR_DESC;
    }
  }
  if (n_live > (int64_t)d.atlas_w * d.atlas_h) return PK_ERR_ARG;
  pk_options o;
  o.tile = 32;
  o.znear = 0.01f;
  o.bg[0] = o.bg[1] = o.bg[2] = 0.0f;
  o.max_dups = 0;
  o.bin_mode = PK_BIN_ELLIPSE;
  o.batch = 128;
  o.stage_fwd = PK_STAGE_LOADS;
  o.stage_bwd = PK_STAGE_LOADS;
  o.batch_bwd = 128;
  o.sort_bits_tile = 8;
  o.sort_bits_depth = 8;
  o.count_evals = 0;
  o.first_wait_polls = 0;
  if (opts) o = *opts;
  if (o.count_evals != 0 && o.count_evals != 1) return PK_ERR_ARG;
  if (o.first_wait_polls < -1) return PK_ERR_ARG;
  if (o.sort_bits_tile == 0) o.sort_bits_tile = 8;
  if (o.sort_bits_depth == 0) o.sort_bits_depth = 8;
  for (const int32_t b : {o.sort_bits_tile, o.sort_bits_depth})
    if (b != 8 && b != 11) return PK_ERR_ARG;
  if (o.bin_mode != PK_BIN_RECT && o.bin_mode != PK_BIN_ELLIPSE) return PK_ERR_ARG;
  if (o.batch == 0) o.batch = 128;
  if (o.batch_bwd == 0) o.batch_bwd = 128;
  for (const int32_t b : {o.batch, o.batch_bwd})
    if (b != 64 && b != 128 && b != 256) return PK_ERR_ARG;
  if ((o.stage_fwd != PK_STAGE_LOADS && o.stage_fwd != PK_STAGE_BULK) ||
      (o.stage_bwd != PK_STAGE_LOADS && o.stage_bwd != PK_STAGE_BULK))
    return PK_ERR_ARG;
  if (o.tile == 0) o.tile = 32;
  if (o.tile != 16 && o.tile != 32) return PK_ERR_UNSUPPORTED;
  if (!(o.znear > 0.0f) || !isfinite(o.znear)) return PK_ERR_ARG;
  for (int c = 0; c < 3; ++c)
    if (!isfinite(o.bg[c])) return PK_ERR_ARG;
  const int64_t N = n_live, F = d.frames, V = n_views;
  if (F * N >= (int64_t(1) << 31) || V * N >= (int64_t(1) << 32) - 1) return PK_ERR_ARG;
  int64_t P = 0, tiles = 0;
  for (int v = 0; v < n_views; ++v) {
    const pk_view &w = views[v];
    if (w.width < 1 || w.height < 1 || w.width > 32768 || w.height > 32768) return PK_ERR_DESC;
    if (w.frame < 0 || w.frame >= d.frames || !finite_view(w)) return PK_ERR_DESC;
    P += (int64_t)w.width * w.height;
    tiles += (int64_t)((w.width + o.tile - 1) / o.tile) * ((w.height + o.tile - 1) / o.tile);
  }
  if (tiles >= (int64_t(1) << 31) || 3 * P >= (int64_t(1) << 40)) return PK_ERR_ARG;
  uint64_t pairs = (uint64_t)(V * N);
  if (pairs > 0xFFFFFFFFull) return PK_ERR_ARG;   // pair indices are 32-bit
  uint64_t maxd = o.max_dups ? o.max_dups : 32 * pairs;
  if (maxd < 1024) maxd = 1024;
  // entry positions are 64-bit; 2^35 entries (412 GB of lists and sort
  // buffers) is beyond any one GPU's memory
  if (maxd > kMaxEntries) maxd = kMaxEntries;
  o.max_dups = maxd;

  pk_plan *p = new (std::nothrow) pk_plan;
  if (!p) return PK_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->desc = d;
  p->opts = o;
  p->V = n_views;
  p->F = d.frames;
  p->L = d.sh_degree;
  p->D = 11 + 3 * (d.sh_degree + 1) * (d.sh_degree + 1);
  p->T = o.tile;
  p->N = N;
  p->G = F * N;
  p->pairs = (int64_t)pairs;
  p->P = P;
  p->n_tiles = tiles;
  p->max_dups = maxd;
  p->first_polls = o.first_wait_polls == 0 ? kWaitPolls : (o.first_wait_polls < 0 ? 0u : (uint32_t)o.first_wait_polls);
  int bits = 1;
  while ((int64_t(1) << bits) < tiles) ++bits;
  p->tile_bits = bits;

  p->h_views = new DevView[V];
  p->h_toff = new uint32_t[V + 1];
  p->h_fview_off = new int32_t[F + 1];
  p->h_fview_idx = new int32_t[V];
  int64_t po = 0, to = 0, mo = 0, co = 0;
  for (int v = 0; v < n_views; ++v) {
    const pk_view &w = views[v];
    DevView &dv = p->h_views[v];
    memset(&dv, 0, sizeof(dv));
    memcpy(dv.R, w.R, sizeof(dv.R));
    memcpy(dv.t, w.t, sizeof(dv.t));
    dv.fx = w.fx;
    dv.fy = w.fy;
    dv.cx = w.cx;
    dv.cy = w.cy;
    for (int a = 0; a < 3; ++a)
      dv.campos[a] = -(w.R[a] * w.t[0] + w.R[3 + a] * w.t[1] + w.R[6 + a] * w.t[2]);
    dv.width = w.width;
    dv.height = w.height;
    dv.frame = w.frame;
    dv.tiles_x = (w.width + o.tile - 1) / o.tile;
    dv.tiles_y = (w.height + o.tile - 1) / o.tile;
    dv.pix_off = po;
    dv.tile_off = to;
    dv.mask_off = mo;
    dv.coarse_off = co;
    p->h_toff[v] = (uint32_t)to;
    po += (int64_t)w.width * w.height;
    to += (int64_t)dv.tiles_x * dv.tiles_y;
    const int64_t wpr = (w.width + 31) / 32;
    mo += (int64_t)w.height * wpr;
    co += (int64_t)((w.height + 31) / 32) * ((wpr + 31) / 32);
  }
  p->mask_words = mo;
  p->coarse_words = co;
  p->h_toff[V] = (uint32_t)to;
  // views grouped by frame (CSR), keeping view order inside a frame
  int32_t k = 0;
  for (int f = 0; f < d.frames; ++f) {
    p->h_fview_off[f] = k;
    for (int v = 0; v < n_views; ++v)
      if (views[v].frame == f) p->h_fview_idx[k++] = v;
  }
  p->h_fview_off[F] = k;

  // workspace layout
  WsLayout &L = p->ws;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t Wp = (size_t)(d.atlas_w + 31) / 32;
  L.status = take(sizeof(pk_device_status));
  L.counters = take(sizeof(DevCounters));
  L.views = take(sizeof(DevView) * V);
  L.toff = take(sizeof(uint32_t) * (V + 1));
  L.fview_off = take(sizeof(int32_t) * (F + 1));
  L.fview_idx = take(sizeof(int32_t) * V);
  L.woff = take(sizeof(uint32_t) * (Wp * d.atlas_h + 1));
  L.pair_cnt = take(sizeof(uint32_t) * pairs);
  L.zkey0 = take(sizeof(uint32_t) * pairs);
  L.zkey1 = take(sizeof(uint32_t) * pairs);
  L.pval0 = take(sizeof(uint32_t) * pairs);
  L.pval1 = take(sizeof(uint32_t) * pairs);
  L.offs = take(sizeof(uint64_t) * pairs);
  L.rmask = take(sizeof(uint4) * pairs);
  L.blocksums = take(sizeof(uint64_t) * (kScanBlocks + 1));
  // digit counters of the widest radix pass (room for 11-bit digits, so
  // that pk_autotune may pick them)
  L.hist = take(sizeof(uint64_t) * (size_t(1) << kMaxRadixBits) * kSortBlocks);
  L.dkey0 = take(sizeof(uint32_t) * maxd);
  L.dkey1 = take(sizeof(uint32_t) * maxd);
  L.dval = take(sizeof(uint32_t) * maxd);
  L.sblk = take(sizeof(int4) * 2 * kSortBlocks);
  L.vseg = take(sizeof(uint64_t) * 2 * (V + 1));
  L.mask_tmp = take(sizeof(uint32_t) * (size_t)p->mask_words);
  L.mask_coarse = take(sizeof(uint32_t) * (size_t)p->coarse_words);
  L.total = off;
  *out = p;
  return PK_OK;
}

extern "C" pk_status pk_plan_sizes(const pk_plan *p, pk_sizes *s) {
  if (!p || !s) return PK_ERR_ARG;
  s->n_live = p->N;
  s->n_gauss = p->G;
  s->channels = p->D;
  s->n_views = p->V;
  s->n_pairs = p->pairs;
  s->n_pixels = p->P;
  s->n_tiles = p->n_tiles;
  s->max_dups = p->max_dups;
  s->workspace_bytes = p->ws.total;
  s->mask_words = p->mask_words;
  s->bin_kernels = bin_kernel_count(p);
  return PK_OK;
}

extern "C" pk_status pk_plan_options(const pk_plan *p, pk_options *out) {
  if (!p || !out) return PK_ERR_ARG;
  *out = p->opts;
  return PK_OK;
}

extern "C" void pk_plan_destroy(pk_plan *p) {
  if (!p) return;
  delete[] p->h_views;
  delete[] p->h_toff;
  delete[] p->h_fview_off;
  delete[] p->h_fview_idx;
  if (p->h_status) cudaFreeHost(p->h_status);
  delete p;
}

extern "C" pk_status pk_workspace_init(const pk_plan *p, void *ws, pk_stream_t stream) {
  if (!p || !ws || (reinterpret_cast<uintptr_t>(ws) & 255u)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const WsLayout &L = p->ws;
  if (cudaMemsetAsync(at<char>(ws, L.status), 0, L.views - L.status, st) != cudaSuccess) return PK_ERR_CUDA;
  if (cudaMemcpyAsync(at<char>(ws, L.views), p->h_views, sizeof(DevView) * p->V, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return PK_ERR_CUDA;
  if (cudaMemcpyAsync(at<char>(ws, L.toff), p->h_toff, sizeof(uint32_t) * (p->V + 1), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return PK_ERR_CUDA;
  if (cudaMemcpyAsync(at<char>(ws, L.fview_off), p->h_fview_off, sizeof(int32_t) * (p->F + 1),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PK_ERR_CUDA;
  if (cudaMemcpyAsync(at<char>(ws, L.fview_idx), p->h_fview_idx, sizeof(int32_t) * p->V, cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return PK_ERR_CUDA;
  // block tables of the segmented sorts (for this device's SM count)
  int4 *tab = const_cast<pk_plan *>(p)->h_segtab;
  int nt = 0, np = 0;
  if (seg_tables(p, tab, &nt, &np) &&
      cudaMemcpyAsync(at<char>(ws, L.sblk), tab, sizeof(p->h_segtab), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PK_ERR_CUDA;
  // pageable sources: make sure the copies are done before the plan may go away
  if (cudaStreamSynchronize(st) != cudaSuccess) return PK_ERR_CUDA;
  return PK_OK;
}

extern "C" pk_status pk_read_status(const pk_plan *p, const void *ws, pk_stream_t stream, pk_device_status *out) {
  if (!p || !ws || !out) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // both blocks land in a small mapped pinned buffer of the plan (allocated
  // on first use), written by one small kernel on `stream`
  constexpr size_t kCtrOff = (sizeof(pk_device_status) + 15) & ~size_t(15);
  pk_plan *pm = const_cast<pk_plan *>(p);
  if (!pm->h_status) {
    if (cudaHostAlloc(&pm->h_status, kCtrOff + sizeof(DevCounters), cudaHostAllocMapped) != cudaSuccess) {
      pm->h_status = nullptr;
      return PK_ERR_CUDA;
    }
  }
  void *dmap = nullptr;
  if (cudaHostGetDevicePointer(&dmap, pm->h_status, 0) != cudaSuccess || !dmap) return PK_ERR_CUDA;
  char *hb = static_cast<char *>(pm->h_status);
  static_assert(sizeof(pk_device_status) % 4 == 0 && sizeof(DevCounters) % 4 == 0, "status words");
  k_status_out<<<1, 64, 0, st>>>(at<uint32_t>(const_cast<void *>(ws), p->ws.status), (int)(sizeof(*out) / 4),
                                 at<uint32_t>(const_cast<void *>(ws), p->ws.counters), (int)(sizeof(DevCounters) / 4),
                                 static_cast<uint32_t *>(dmap), reinterpret_cast<uint32_t *>(static_cast<char *>(dmap) + kCtrOff));
  if (check_launch() != PK_OK) return PK_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PK_ERR_CUDA;
  DevCounters c;
  memcpy(out, hb, sizeof(*out));
  memcpy(&c, hb + kCtrOff, sizeof(c));
  const double n = 3.0 * (double)p->P, lam = c.ssim_lambda;
  out->ssim = c.ssim_acc / n;
  out->loss = (1.0 - lam) * c.loss_acc / n + (lam > 0.0 ? lam * (1.0 - out->ssim) : 0.0);
  if (out->flags & PK_DEV_CAPACITY) return PK_ERR_CAPACITY;
  if (out->flags & PK_DEV_TIMEOUT) return PK_ERR_TIMEOUT;
  return PK_OK;
}

namespace {

// Milliseconds of `reps` runs of fn after one warm-up, on stream st.
template <typename Fn>
pk_status time_runs(Fn fn, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps, float *ms) {
  pk_status e = fn();
  if (e != PK_OK) return e;
  if (cudaEventRecord(e0, st) != cudaSuccess) return PK_ERR_CUDA;
  for (int r = 0; r < reps && e == PK_OK; ++r) e = fn();
  if (e != PK_OK) return e;
  if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
    return PK_ERR_CUDA;
  return PK_OK;
}

}  // namespace

extern "C" pk_status pk_autotune(pk_plan *p, const float *records, uint32_t *sorted_vals, uint64_t *tile_ranges,
                                 float *image, float *T_final, uint32_t *n_contrib,
                                 const float *dL_dimage, float *grad2d, void *ws, pk_stream_t stream,
                                 int32_t *chosen_batch) {
  if (!p) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PK_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PK_ERR_CUDA;
  }
  const pk_options keep = p->opts;
  auto fwd = [&]() { return pk_rasterize_fwd(p, records, sorted_vals, tile_ranges, image, T_final, n_contrib, ws, stream); };
  auto bwd = [&]() {
    return pk_rasterize_bwd(p, records, sorted_vals, tile_ranges, T_final, n_contrib, dL_dimage, grad2d, ws, stream);
  };
  auto both = [&]() {
    pk_status e = fwd();
    return e == PK_OK ? bwd() : e;
  };
  pk_status e = PK_OK;
  // each kernel's batch, with plain loads (the backward reads the
  // forward's outputs, which no batch changes); another choice than the
  // default (128, loads) must win by more than 2 %, so timing noise does not
  // flip it
  const float kMargin = 0.98f;
  const int32_t cands[3] = {128, 256, 64};
  p->opts.stage_fwd = p->opts.stage_bwd = PK_STAGE_LOADS;
  p->opts.batch = p->opts.batch_bwd = 128;
  e = fwd();
  for (int k = 0; k < 2 && e == PK_OK; ++k) {
    int32_t *batch = k == 0 ? &p->opts.batch : &p->opts.batch_bwd;
    int32_t best = 128;
    float best_ms = 0.f;
    for (int i = 0; i < 3 && e == PK_OK; ++i) {
      *batch = cands[i];
      float ms = 0.f;
      e = k == 0 ? time_runs(fwd, st, e0, e1, 2, &ms) : time_runs(bwd, st, e0, e1, 2, &ms);
      if (e == PK_OK && (i == 0 || ms < kMargin * best_ms)) {
        best_ms = ms;
        best = cands[i];
      }
    }
    *batch = best;
  }
  // the staging mode of each kernel
  for (int k = 0; k < 2 && e == PK_OK; ++k) {
    int32_t *mode = k == 0 ? &p->opts.stage_fwd : &p->opts.stage_bwd;
    float ms_loads = 0.f, ms_bulk = 0.f;
    *mode = PK_STAGE_LOADS;
    e = k == 0 ? time_runs(fwd, st, e0, e1, 2, &ms_loads) : time_runs(bwd, st, e0, e1, 2, &ms_loads);
    if (e != PK_OK) break;
    *mode = PK_STAGE_BULK;
    e = k == 0 ? time_runs(fwd, st, e0, e1, 2, &ms_bulk) : time_runs(bwd, st, e0, e1, 2, &ms_bulk);
    if (e == PK_OK) *mode = ms_bulk < kMargin * ms_loads ? PK_STAGE_BULK : PK_STAGE_LOADS;
  }
  // the digit widths of the two radix sorts of pk_bin_and_sort (8 or 11
  // bits): the depth sort's first, then the tile sort's, each timed over the
  // whole call; the lists do not depend on them.  The segmented sorts'
  // block tables depend on the widths and are uploaded again.
  auto upload_tables = [&]() -> pk_status {
    int nt = 0, np = 0;
    if (seg_tables(p, p->h_segtab, &nt, &np) &&
        cudaMemcpyAsync(at<char>(ws, p->ws.sblk), p->h_segtab, sizeof(p->h_segtab), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
      return PK_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? PK_OK : PK_ERR_CUDA;
  };
  auto sort = [&]() { return pk_bin_and_sort(p, records, sorted_vals, tile_ranges, ws, stream); };
  for (int k = 0; k < 2 && e == PK_OK; ++k) {
    int32_t *bits = k == 0 ? &p->opts.sort_bits_depth : &p->opts.sort_bits_tile;
    float ms8 = 0.f, ms11 = 0.f;
    *bits = 8;
    if ((e = upload_tables()) != PK_OK || (e = time_runs(sort, st, e0, e1, 2, &ms8)) != PK_OK) break;
    *bits = 11;
    if ((e = upload_tables()) != PK_OK || (e = time_runs(sort, st, e0, e1, 2, &ms11)) != PK_OK) break;
    *bits = ms11 < kMargin * ms8 ? 11 : 8;
    e = upload_tables();
  }
  if (e != PK_OK) {
    p->opts = keep;
    upload_tables();
  } else {
    e = sort();
    if (e == PK_OK) e = both();
  }
  if (e == PK_OK && cudaStreamSynchronize(st) != cudaSuccess) e = PK_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (chosen_batch) *chosen_batch = p->opts.batch;
  return e;
}
