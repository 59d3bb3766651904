// Photometric L1 term of the fitting objective (Sec. 4.2 "Objective"):
// loss = mean |image - target|, dL/dimage = sign(image - target) / (3 P).
// The loss sum is accumulated in double precision in the workspace.
#include "pk_common.cuh"

using namespace pk;

namespace {

__global__ __launch_bounds__(256) void k_l1(const float *__restrict__ img, const float *__restrict__ tgt, int64_t n,
                                            float scale, float *__restrict__ grad, double *acc) {
  __shared__ double s[8];
  double local = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[i] - tgt[i];
    local += fabs((double)d);
    grad[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = local;
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
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevCounters *ctr = at<DevCounters>(ws, p->ws.counters);
  // loss_acc, ssim_acc and ssim_lambda (0: the loss is L1 alone)
  if (cudaMemsetAsync(&ctr->loss_acc, 0, 2 * sizeof(double) + sizeof(float), st) != cudaSuccess) return PK_ERR_CUDA;
  const int64_t n = 3 * p->P;
  if (n == 0) return PK_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_l1<<<(int)blocks, 256, 0, st>>>(image, target, n, (float)(1.0 / (double)n), dL_dimage, &ctr->loss_acc);
  return check_launch();
}
