// Internal definitions shared by the kernels and the host side of the
// library.  Not part of the public ABI (include/packuv.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <initializer_list>
#include <utility>

#include "../../include/packuv.h"

namespace pk {

constexpr int kRec = PK_RECORD_FLOATS;   // floats per projected record
constexpr int kG2d = PK_GRAD2D_FLOATS;   // floats per 2D gradient record

// Compositing constants (see packuv.h): alpha clamp, skip threshold,
// transmittance cutoff, footprint d^2 <= 9.
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kQMax = 9.0f;
constexpr float kLowPass = 0.3f;
constexpr float kDetMin = 1e-7f;
// exp(-q/2) = exp2(q * kExpScale), kExpScale = -log2(e) / 2
constexpr float kExpScale = -0.72134752044448170f;
constexpr float kInvExpScale = -1.38629436111989061f;   // 1 / kExpScale = -2 ln 2

// Fixed grid sizes of the device-count-driven kernels (scan, radix sort).
constexpr int kScanBlocks = 4096;
constexpr int kSortBlocks = 768;      // most radix blocks of one pass (histogram capacity)
constexpr int kMaxRadixBits = 11;     // widest radix digit (pk_options.sort_bits_*: 8 or 11)
constexpr uint64_t kMaxEntries = uint64_t(1) << 35;   // most (pair, tile) entries of a plan

// Per-view constants on the device, 144 bytes.
struct alignas(16) DevView {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float campos[3];    // -R^T t
  int32_t width, height, frame;
  int32_t tiles_x, tiles_y;
  int32_t pad0;
  int64_t pix_off;    // first pixel of this view in the concatenated images
  int64_t tile_off;   // first global tile id of this view
  int64_t mask_off;   // first word of this view's motion-mask rows
  int64_t coarse_off; // first word of this view's 32 x 32-pixel block mask
};
static_assert(sizeof(DevView) % 16 == 0, "DevView layout");

// Internal device scalars kept after the public status block.
struct DevCounters {
  uint64_t n_valid;        // pairs with >= 1 tile (after the compaction scan)
  uint64_t dups;           // entries emitted (0 on overflow); 64-bit, as are entry positions
  uint32_t tile_queue[4];  // persistent-kernel work counters
  uint64_t scan_total;     // total of the last scan
  double loss_acc;         // sum of |image - target| of the last loss call
  double ssim_acc;         // sum of the SSIM map of the last photometric loss call
  float ssim_lambda;       // its lambda (0 after pk_l1_loss_grad)
  uint32_t sort_abort;     // this bin_and_sort call gave up (a wait timed out or an index check
                           // failed): it emits nothing; cleared at the start of each call
};

// Byte offsets of every region inside the workspace.
struct WsLayout {
  size_t status, counters, views, toff, fview_off, fview_idx, woff;
  size_t pair_cnt, zkey0, zkey1, pval0, pval1, offs, rmask;   // rmask: per pair {mask (2 words), rectangle (2)}
  size_t blocksums, hist;
  size_t dkey0, dkey1, dval;
  size_t sblk, vseg;       // segmented sorts: block tables [2][kSortBlocks] int4 (tile passes, depth
                           // passes), view starts [2][V + 1] (entries, pairs)
  size_t mask_tmp;         // one motion mask's worth of words (dilation scratch)
  size_t mask_coarse;      // per view, one bit per 32 x 32-pixel block: any moving pixel
  size_t total;
};

}  // namespace pk

// Host-side plan (opaque to C callers).
struct pk_plan {
  pk_atlas_desc desc;
  pk_options opts;
  int32_t V, F, D, T, L;
  int64_t N, G, pairs, P, n_tiles, mask_words, coarse_words;
  uint64_t max_dups;
  int32_t tile_bits;       // bits needed for a global tile id
  int32_t num_sms;
  uint32_t first_polls;    // polls of the first bounded wait on a bulk-copied batch
  pk::WsLayout ws;
  pk::DevView *h_views;    // host copies uploaded by pk_workspace_init
  uint32_t *h_toff;        // [V+1] tile offsets (global tile id -> view)
  int32_t *h_fview_off;    // [F+1]
  int32_t *h_fview_idx;    // [V]
  int4 h_segtab[2 * pk::kSortBlocks];   // block tables of the segmented sorts (copied to the device)
  void *h_status;          // mapped pinned host copy of the status block and counters (first pk_read_status)
};

namespace pk {

template <typename T>
__host__ __device__ inline T *at(void *base, size_t off) {
  return reinterpret_cast<T *>(reinterpret_cast<char *>(base) + off);
}

// Host-side launch helpers (implemented in pk_plan.cu).
pk_status check_launch();
bool aligned16(const void *p);
// Zero up to four (pointer, bytes) ranges with one kernel (4-byte aligned
// pointers, sizes multiples of 4 bytes).
pk_status zero_async(std::initializer_list<std::pair<void *, size_t>> spans, cudaStream_t st);
// Radix blocks of the entry passes on the current device, and the block
// tables of the segmented (per-view) sorts: tab[0, kSortBlocks) for the
// tile passes, tab[kSortBlocks, 2 kSortBlocks) for the depth passes
// (pk_binsort.cu); false = the plan sorts unsegmented.
int sort_blocks(int rb);
bool seg_tables(const pk_plan *p, int4 *tab, int *ntile, int *npair);
// Kernels one pk_bin_and_sort call launches for this plan on this device.
int bin_kernel_count(const pk_plan *p);

}  // namespace pk
