// Photometric objective of Sec. 4.2 "Objective": (1 - lambda) L1 +
// lambda (1 - SSIM), loss and gradient in one pass over every view.
//
// One CTA per 32 x 32 output tile of one channel of one view.  It stages
// the 52 x 52 input window of image and target (halo 2 x 5) in shared
// memory, forms the five window sums (X, Y, XX, YY, XY) on the 42 x 42
// region (halo 5) by a horizontal then a vertical 11-tap pass, turns them
// into the SSIM value and its partial derivatives, and sums those back onto
// the 32 x 32 tile with the same separable window (the adjoint of the
// window sums).  Every pass is register-tiled: a thread produces 4 to 8
// consecutive outputs of one row or column from one sliding read of the
// inputs, so shared-memory reads are about 1/4 of the multiply-adds.  The
// sums travel in pairs -- (X, Y), (XX, YY) and, backwards, (d1, d11) -- so
// each tap is one packed FP32 multiply-add per pair (two round-to-nearest
// results, each the scalar one) plus one scalar for the fifth sum.
// Image and target are read once per tile (plus halo) and the gradient
// written once; the arithmetic (about 400 FP32 operations per value)
// bounds the kernel.  The five barrier-separated stages each leave some
// threads idle, so the SM is kept busy by CTAs at different stages: the
// derivative maps reuse the shared memory of the input window (the last
// stage reads its centre values again from global memory, where they are
// still cached), which brings a CTA to 67 KB and three CTAs onto an SM.
#include "pk_common.cuh"
#include "pk_f32x2.cuh"

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

// Row strides padded to odd lengths so that threads walking down a column
// hit distinct banks.
constexpr int kIP = kI + 1, kMP = kM + 1, kTP = kT + 1;
constexpr int kGB = 6;   // stage B: window-sum columns per item (42 = 7 x 6)
constexpr int kGC = 7;   // stage C: window-sum rows per item (42 = 6 x 7)
constexpr int kGD = 8;   // stage D: tile columns per item (32 = 4 x 8)
constexpr int kGE = 4;   // stage E: tile rows per item (32 = 8 x 4)

struct SsimSmem {
  union {
    struct {
      float x[kI][kIP], y[kI][kIP];   // inputs, 0 outside the image (read by the horizontal sums only)
    };
    struct {
      f32x2 d01[kM][kMP];             // then: partial derivatives of the SSIM map, (d1, d11) and d12
      float d2[kM][kMP];
    };
  };
  f32x2 h01[kI][kMP], h23[kI][kMP];   // horizontal sums (X, Y), (XX, YY); later the backward
  float h4[kI][kMP];                  //   sums ((d1, d11) pairs, d12) on [kM][kTP]; XY
};
static_assert(sizeof(float) * 2 * kM * kMP + sizeof(float) * kM * kMP <= sizeof(float) * 2 * kI * kIP,
              "the derivative maps fit in the input tiles they replace");

__global__ __launch_bounds__(kSsimThreads, 3) void k_photo(const float *__restrict__ img,
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
  float w[2 * kR + 1];
  f32x2 wd[2 * kR + 1];   // each weight twice, for the packed pairs
#pragma unroll
  for (int j = 0; j <= 2 * kR; ++j) {
    w[j] = c_w[j];
    wd[j] = dup2(w[j]);
  }
  const f32x2 z2 = dup2(0.f);

  // A: inputs over [ty0 - 10, ty0 + 42) x [tx0 - 10, tx0 + 42), every load
  // of a thread issued before the first store
  {
    constexpr int kLoads = (kI * kI + kSsimThreads - 1) / kSsimThreads;
    float xv[kLoads], yv[kLoads];
#pragma unroll
    for (int k = 0; k < kLoads; ++k) {
      const int i = tid + k * kSsimThreads;
      const int r = i / kI, q = i - r * kI;
      const int yy = ty0 - 2 * kR + r, xx = tx0 - 2 * kR + q;
      const bool in = i < kI * kI && yy >= 0 && yy < H && xx >= 0 && xx < W;
      xv[k] = in ? __ldg(X + (int64_t)yy * W + xx) : 0.0f;
      yv[k] = in ? __ldg(Y + (int64_t)yy * W + xx) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kLoads; ++k) {
      const int i = tid + k * kSsimThreads;
      if (i < kI * kI) {
        const int r = i / kI, q = i - r * kI;
        S.x[r][q] = xv[k];
        S.y[r][q] = yv[k];
      }
    }
  }
  __syncthreads();
  // B: horizontal window sums of X, Y, XX, YY, XY: each item one input row
  // and kGB consecutive window-sum columns (threads walk down the rows)
  for (int it = tid; it < kI * (kM / kGB); it += kSsimThreads) {
    const int g = it / kI, r = it - g * kI, q0 = g * kGB;
    f32x2 a01[kGB], a23[kGB];
    float a4[kGB];
#pragma unroll
    for (int o = 0; o < kGB; ++o) {
      a01[o] = z2;
      a23[o] = z2;
      a4[o] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < kGB + 2 * kR; ++t) {
      const float xv = S.x[r][q0 + t], yv = S.y[r][q0 + t];
      const f32x2 v = pack2(xv, yv);
      const f32x2 sq = mul2(v, v);
      const float xy = xv * yv;
#pragma unroll
      for (int o = 0; o < kGB; ++o) {
        const int j = t - o;
        if (j < 0 || j > 2 * kR) continue;
        a01[o] = fma2(wd[j], v, a01[o]);
        a23[o] = fma2(wd[j], sq, a23[o]);
        a4[o] = fmaf(w[j], xy, a4[o]);
      }
    }
#pragma unroll
    for (int o = 0; o < kGB; ++o) {
      S.h01[r][q0 + o] = a01[o];
      S.h23[r][q0 + o] = a23[o];
      S.h4[r][q0 + o] = a4[o];
    }
  }
  __syncthreads();
  // C: vertical window sums on kGC consecutive rows of one column, then the
  // SSIM value and its partial derivatives with respect to m1 = G*X,
  // e11 = G*XX, e12 = G*XY (0 outside the image)
  float ssim_sum = 0.f;
  for (int it = tid; it < kM * (kM / kGC); it += kSsimThreads) {
    const int g = it / kM, q = it - g * kM, r0 = g * kGC;
    f32x2 a01[kGC], a23[kGC];
    float a4[kGC];
#pragma unroll
    for (int o = 0; o < kGC; ++o) {
      a01[o] = z2;
      a23[o] = z2;
      a4[o] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < kGC + 2 * kR; ++t) {
      const f32x2 h01 = S.h01[r0 + t][q], h23 = S.h23[r0 + t][q];
      const float h4 = S.h4[r0 + t][q];
#pragma unroll
      for (int o = 0; o < kGC; ++o) {
        const int j = t - o;
        if (j < 0 || j > 2 * kR) continue;
        a01[o] = fma2(wd[j], h01, a01[o]);
        a23[o] = fma2(wd[j], h23, a23[o]);
        a4[o] = fmaf(w[j], h4, a4[o]);
      }
    }
    const int xx = tx0 - kR + q;
#pragma unroll
    for (int o = 0; o < kGC; ++o) {
      const int r = r0 + o, yy = ty0 - kR + r;
      float d1 = 0.f, d11 = 0.f, d12 = 0.f;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
        float m1, m2, e11, e22;
        unpack2(a01[o], m1, m2);
        unpack2(a23[o], e11, e22);
        const float e12 = a4[o];
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
      S.d01[r][q] = pack2(d1, d11);
      S.d2[r][q] = d12;
    }
  }
  __syncthreads();
  // D: backward horizontal sums of the three maps: one row of the 42 region,
  // kGD consecutive tile columns (into the h buffers, as [kM][kTP])
  f32x2(*hb01)[kTP] = reinterpret_cast<f32x2(*)[kTP]>(&S.h01[0][0]);
  float(*hb2)[kTP] = reinterpret_cast<float(*)[kTP]>(&S.h4[0][0]);
  for (int it = tid; it < kM * (kT / kGD); it += kSsimThreads) {
    const int g = it / kM, r = it - g * kM, q0 = g * kGD;
    f32x2 b01[kGD];
    float b2[kGD];
#pragma unroll
    for (int o = 0; o < kGD; ++o) {
      b01[o] = z2;
      b2[o] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < kGD + 2 * kR; ++t) {
      const f32x2 d01 = S.d01[r][q0 + t];
      const float d2 = S.d2[r][q0 + t];
#pragma unroll
      for (int o = 0; o < kGD; ++o) {
        const int j = t - o;
        if (j < 0 || j > 2 * kR) continue;
        b01[o] = fma2(wd[j], d01, b01[o]);
        b2[o] = fmaf(w[j], d2, b2[o]);
      }
    }
#pragma unroll
    for (int o = 0; o < kGD; ++o) {
      hb01[r][q0 + o] = b01[o];
      hb2[r][q0 + o] = b2[o];
    }
  }
  __syncthreads();
  // E: vertical sums onto kGE rows of one tile column, combined with X, Y
  // (read again from global memory: their shared copy now holds the
  // derivative maps) and the L1 term
  float l1_sum = 0.f;
  const float gl1 = (1.f - lambda) * inv_n, gs = lambda * inv_n;
  for (int it = tid; it < kT * (kT / kGE); it += kSsimThreads) {
    const int g = it / kT, q = it - g * kT, r0 = g * kGE;
    const int xx = tx0 + q;
    if (xx >= W) continue;
    f32x2 c01[kGE];
    float c2[kGE];
#pragma unroll
    for (int o = 0; o < kGE; ++o) {
      c01[o] = z2;
      c2[o] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < kGE + 2 * kR; ++t) {
      const f32x2 v01 = hb01[r0 + t][q];
      const float v2 = hb2[r0 + t][q];
#pragma unroll
      for (int o = 0; o < kGE; ++o) {
        const int j = t - o;
        if (j < 0 || j > 2 * kR) continue;
        c01[o] = fma2(wd[j], v01, c01[o]);
        c2[o] = fmaf(w[j], v2, c2[o]);
      }
    }
#pragma unroll
    for (int o = 0; o < kGE; ++o) {
      const int r = r0 + o, yy = ty0 + r;
      if (yy >= H) break;
      const float xv = __ldg(X + (int64_t)yy * W + xx), yv = __ldg(Y + (int64_t)yy * W + xx);
      float s0, s1;
      unpack2(c01[o], s0, s1);
      const float dS = s0 + 2.f * xv * s1 + yv * c2[o];
      const float dd = xv - yv;
      l1_sum += fabsf(dd);
      const float sg = dd > 0.f ? 1.f : (dd < 0.f ? -1.f : 0.f);
      grad[3 * view.pix_off + c * plane + (int64_t)yy * W + xx] = gl1 * sg - gs * dS;
    }
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
    for (int k = 0; k < kSsimThreads / 32; ++k) {
      a += s_red[0][k];
      b += s_red[1][k];
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
  pk_status ze = zero_async({{&ctr->loss_acc, 2 * sizeof(double) + sizeof(float)}}, st);
  if (ze != PK_OK) return ze;
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
