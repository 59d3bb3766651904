// Photometric objective of Sec. 4.2 "Objective": (1 - lambda) L1 +
// lambda (1 - SSIM), loss and gradient in one pass over every view.
//
// One CTA per 32 x 32 output tile of one channel of one view.  It stages
// the 52 x 52 input window of image and target (halo 2 x 5) in shared
// memory, forms the five window sums (X, Y, XX, YY, XY) on the 42 x 42
// region (halo 5) by a horizontal then a vertical 11-tap pass, turns them
// into the SSIM value and its partial derivatives in place, and sums those
// back onto the 32 x 32 tile with the same separable window (the adjoint of
// the window sums).  Image and target are read once per tile (plus halo)
// and the gradient written once; the arithmetic (about 400 FP32 operations
// per value) bounds the kernel.
#include "pk_common.cuh"

using namespace pk;

namespace {

constexpr int kR = 5;                 // window radius (11 taps)
constexpr int kT = 32;                // output tile side
constexpr int kM = kT + 2 * kR;       // 42: window-sum region
constexpr int kI = kT + 4 * kR;       // 52: input region
constexpr int kSsimThreads = 256;
constexpr float kC1 = 0.0001f, kC2 = 0.0009f;

// 1-D Gaussian weights (standard deviation 1.5 over -5..5, sum 1), set by
// the host in double precision and rounded once.
__constant__ float c_w[2 * kR + 1];

struct SsimSmem {
  float x[kI][kI], y[kI][kI];         // inputs, 0 outside the image
  float h[5][kI][kM];                 // horizontal sums; later [3][kM][kT] backward sums
  float m[5][kM][kM];                 // window sums; later the three partial maps
};

__global__ __launch_bounds__(kSsimThreads, 2) void k_photo(const float *__restrict__ img,
                                                           const float *__restrict__ tgt,
                                                           const DevView *__restrict__ views, float lambda,
                                                           float inv_n, float *__restrict__ grad, double *l1_acc,
                                                           double *ssim_acc, float *lambda_out) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  SsimSmem &S = *reinterpret_cast<SsimSmem *>(s_raw);
  __shared__ float s_red[2][kSsimThreads / 32];
  const int v = blockIdx.z / 3, c = blockIdx.z - 3 * v;
  const DevView &view = views[v];
  const int W = view.width, H = view.height;
  const int tx0 = blockIdx.x * kT, ty0 = blockIdx.y * kT;
  if (tx0 >= W || ty0 >= H) return;   // uniform over the block
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) *lambda_out = lambda;
  const int64_t plane = (int64_t)W * H;
  const float *X = img + 3 * view.pix_off + c * plane, *Y = tgt + 3 * view.pix_off + c * plane;
  const int tid = threadIdx.x;

  // inputs over [ty0 - 10, ty0 + 42) x [tx0 - 10, tx0 + 42)
  for (int i = tid; i < kI * kI; i += kSsimThreads) {
    const int r = i / kI, q = i - r * kI;
    const int yy = ty0 - 2 * kR + r, xx = tx0 - 2 * kR + q;
    const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
    S.x[r][q] = in ? __ldg(X + (int64_t)yy * W + xx) : 0.0f;
    S.y[r][q] = in ? __ldg(Y + (int64_t)yy * W + xx) : 0.0f;
  }
  __syncthreads();
  // horizontal window sums: every input row, the 42 window-sum columns
  for (int i = tid; i < kI * kM; i += kSsimThreads) {
    const int r = i / kM, q = i - r * kM;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
    for (int j = 0; j <= 2 * kR; ++j) {
      const float w = c_w[j], xv = S.x[r][q + j], yv = S.y[r][q + j];
      a0 = fmaf(w, xv, a0);
      a1 = fmaf(w, yv, a1);
      a2 = fmaf(w, xv * xv, a2);
      a3 = fmaf(w, yv * yv, a3);
      a4 = fmaf(w, xv * yv, a4);
    }
    S.h[0][r][q] = a0;
    S.h[1][r][q] = a1;
    S.h[2][r][q] = a2;
    S.h[3][r][q] = a3;
    S.h[4][r][q] = a4;
  }
  __syncthreads();
  // vertical window sums, then the SSIM value and its partial derivatives
  // with respect to m1 = G*X, e11 = G*XX, e12 = G*XY (0 outside the image)
  float ssim_sum = 0.f;
  for (int i = tid; i < kM * kM; i += kSsimThreads) {
    const int r = i / kM, q = i - r * kM;
    float m1 = 0.f, m2 = 0.f, e11 = 0.f, e22 = 0.f, e12 = 0.f;
#pragma unroll
    for (int j = 0; j <= 2 * kR; ++j) {
      const float w = c_w[j];
      m1 = fmaf(w, S.h[0][r + j][q], m1);
      m2 = fmaf(w, S.h[1][r + j][q], m2);
      e11 = fmaf(w, S.h[2][r + j][q], e11);
      e22 = fmaf(w, S.h[3][r + j][q], e22);
      e12 = fmaf(w, S.h[4][r + j][q], e12);
    }
    const int yy = ty0 - kR + r, xx = tx0 - kR + q;
    float d1 = 0.f, d11 = 0.f, d12 = 0.f;
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
      const float A1 = 2.f * m1 * m2 + kC1, A2 = 2.f * (e12 - m1 * m2) + kC2;
      const float B1 = m1 * m1 + m2 * m2 + kC1, B2 = (e11 - m1 * m1) + (e22 - m2 * m2) + kC2;
      // approximate reciprocals (2 ulp): far inside the FP32 tolerance of the loss
      const float iA1 = __fdividef(1.f, A1), iA2 = __fdividef(1.f, A2), iB1 = __fdividef(1.f, B1),
                  iB2 = __fdividef(1.f, B2);
      const float s = A1 * A2 * iB1 * iB2;
      d1 = 2.f * s * (m2 * (iA1 - iA2) + m1 * (iB2 - iB1));
      d11 = -s * iB2;
      d12 = 2.f * s * iA2;
      if (r >= kR && r < kR + kT && q >= kR && q < kR + kT) ssim_sum += s;
    }
    S.m[0][r][q] = d1;
    S.m[1][r][q] = d11;
    S.m[2][r][q] = d12;
  }
  __syncthreads();
  // backward horizontal sums of the three maps: rows of the 42 region,
  // the 32 tile columns (into the h buffer, as [3][kM][kT])
  float(*hb)[kM][kT] = reinterpret_cast<float(*)[kM][kT]>(&S.h[0][0][0]);
  for (int i = tid; i < kM * kT; i += kSsimThreads) {
    const int r = i / kT, q = i - r * kT;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int j = 0; j <= 2 * kR; ++j) {
      const float w = c_w[j];
      a0 = fmaf(w, S.m[0][r][q + j], a0);
      a1 = fmaf(w, S.m[1][r][q + j], a1);
      a2 = fmaf(w, S.m[2][r][q + j], a2);
    }
    hb[0][r][q] = a0;
    hb[1][r][q] = a1;
    hb[2][r][q] = a2;
  }
  __syncthreads();
  // vertical sums onto the tile, combined with X, Y and the L1 term
  float l1_sum = 0.f;
  const float gl1 = (1.f - lambda) * inv_n, gs = lambda * inv_n;
  for (int i = tid; i < kT * kT; i += kSsimThreads) {
    const int r = i / kT, q = i - r * kT;
    const int yy = ty0 + r, xx = tx0 + q;
    if (yy >= H || xx >= W) continue;
    float t1 = 0.f, t11 = 0.f, t12 = 0.f;
#pragma unroll
    for (int j = 0; j <= 2 * kR; ++j) {
      const float w = c_w[j];
      t1 = fmaf(w, hb[0][r + j][q], t1);
      t11 = fmaf(w, hb[1][r + j][q], t11);
      t12 = fmaf(w, hb[2][r + j][q], t12);
    }
    const float xv = S.x[r + 2 * kR][q + 2 * kR], yv = S.y[r + 2 * kR][q + 2 * kR];
    const float dS = t1 + 2.f * xv * t11 + yv * t12;
    const float d = xv - yv;
    l1_sum += fabsf(d);
    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    grad[3 * view.pix_off + c * plane + (int64_t)yy * W + xx] = gl1 * sg - gs * dS;
  }
  // block sums of L1 and SSIM, one double atomic each
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l1_sum += __shfl_xor_sync(0xffffffffu, l1_sum, o);
    ssim_sum += __shfl_xor_sync(0xffffffffu, ssim_sum, o);
  }
  if ((tid & 31) == 0) {
    s_red[0][tid >> 5] = l1_sum;
    s_red[1][tid >> 5] = ssim_sum;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kSsimThreads / 32; ++w) {
      a += s_red[0][w];
      b += s_red[1][w];
    }
    atomicAdd(l1_acc, a);
    atomicAdd(ssim_acc, b);
  }
}

bool g_weights_set[64] = {};

}  // namespace

extern "C" pk_status pk_photo_loss_grad(const pk_plan *p, const float *image, const float *target, float lambda,
                                        float *dL_dimage, void *ws, pk_stream_t stream) {
  if (!p || !image || !target || !dL_dimage || !ws) return PK_ERR_ARG;
  if (!(lambda >= 0.0f && lambda <= 1.0f)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PK_ERR_CUDA;
  if (dev < 0 || dev >= 64) return PK_ERR_UNSUPPORTED;
  if (!g_weights_set[dev]) {
    // window weights, computed once per device (outside any capture: the
    // first call on a device must not be captured)
    double w[2 * kR + 1], s = 0.0;
    for (int k = -kR; k <= kR; ++k) s += (w[k + kR] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)));
    float wf[2 * kR + 1];
    for (int k = 0; k <= 2 * kR; ++k) wf[k] = (float)(w[k] / s);
    if (cudaMemcpyToSymbol(c_w, wf, sizeof(wf)) != cudaSuccess) return PK_ERR_CUDA;
    if (cudaFuncSetAttribute(k_photo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SsimSmem)) !=
        cudaSuccess)
      return PK_ERR_CUDA;
    g_weights_set[dev] = true;
  }
  DevCounters *ctr = at<DevCounters>(ws, p->ws.counters);
  if (cudaMemsetAsync(&ctr->loss_acc, 0, 2 * sizeof(double) + sizeof(float), st) != cudaSuccess) return PK_ERR_CUDA;
  int maxw = 1, maxh = 1;
  for (int v = 0; v < p->V; ++v) {
    maxw = max(maxw, p->h_views[v].width);
    maxh = max(maxh, p->h_views[v].height);
  }
  const dim3 grid((unsigned)((maxw + kT - 1) / kT), (unsigned)((maxh + kT - 1) / kT), (unsigned)(3 * p->V));
  k_photo<<<grid, kSsimThreads, sizeof(SsimSmem), st>>>(image, target, at<DevView>(ws, p->ws.views), lambda,
                                                        (float)(1.0 / (3.0 * (double)p->P)), dL_dimage,
                                                        &ctr->loss_acc, &ctr->ssim_acc, &ctr->ssim_lambda);
  return check_launch();
}
