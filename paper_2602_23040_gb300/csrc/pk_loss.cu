// Photometric L1 term of the fitting objective (Sec. 4.2 "Objective"):
// loss = mean |image - target|, dL/dimage = sign(image - target) / (3 P).
// The loss sum is accumulated per thread in FP32 and across threads in
// FP64, in the workspace.
#include "pk_common.cuh"

using namespace pk;

namespace {

// Four values per thread and step (16-byte loads and stores when the
// arrays allow), FP32 partial sums per thread (a few thousand values each),
// then FP64 across threads.
__global__ __launch_bounds__(256) void k_l1(const float *__restrict__ img, const float *__restrict__ tgt, int64_t n,
                                            float scale, float *__restrict__ grad, double *acc) {
  __shared__ double s[8];
  float local = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = n / 4;
  const float4 *i4 = reinterpret_cast<const float4 *>(img);
  const float4 *t4 = reinterpret_cast<const float4 *>(tgt);
  float4 *g4 = reinterpret_cast<float4 *>(grad);
  auto sgn = [&](float d) { return d > 0.f ? scale : (d < 0.f ? -scale : 0.f); };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 a = __ldcs(i4 + i), b = __ldcs(t4 + i);
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
    local += (fabsf(dx) + fabsf(dy)) + (fabsf(dz) + fabsf(dw));
    __stcs(g4 + i, make_float4(sgn(dx), sgn(dy), sgn(dz), sgn(dw)));
  }
  for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const float d = img[i] - tgt[i];
    local += fabsf(d);
    grad[i] = sgn(d);
  }
  double dl = (double)local;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dl += __shfl_xor_sync(0xffffffffu, dl, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = dl;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s[w];
    atomicAdd(acc, t);
  }
}

}  // namespace

extern "C" pk_status pk_l1_loss_grad(const pk_plan *p, const float *image, const float *target, float *dL_dimage,
                                     void *ws, pk_stream_t stream) {
  if (!p || !image || !target || !dL_dimage || !ws) return PK_ERR_ARG;
  if (!aligned16(image) || !aligned16(target) || !aligned16(dL_dimage)) return PK_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevCounters *ctr = at<DevCounters>(ws, p->ws.counters);
  // loss_acc, ssim_acc and ssim_lambda (0: the loss is L1 alone)
  pk_status ze = zero_async({{&ctr->loss_acc, 2 * sizeof(double) + sizeof(float)}}, st);
  if (ze != PK_OK) return ze;
  const int64_t n = 3 * p->P;
  if (n == 0) return PK_OK;
  int64_t blocks = (n / 4 + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_l1<<<(int)blocks, 256, 0, st>>>(image, target, n, (float)(1.0 / (double)n), dL_dimage, &ctr->loss_acc);
  return check_launch();
}
