// a2 -- per (view, Gaussian) EWA projection and SH colour.
//
// One thread per Gaussian of every frame: its D attributes are read once
// (coalesced, channel-major SoA), activated once, and then projected into
// every view of its frame; each view's record is one coalesced 48-byte
// store.  The atlas is therefore read once per launch however many views
// the launch holds.
#include "pk_proj_math.cuh"

using namespace pk;

namespace {

constexpr int kProjThreads = 256;

// The SH coefficients of a thread's Gaussian live in shared memory, column
// tid of s_k[3 NB][kProjThreads] (each thread reads only its own column, so
// no barrier is needed); in registers they would cap the occupancy.
template <int L>
__global__ __launch_bounds__(kProjThreads) void k_project(const float *__restrict__ soa, int64_t G, int64_t N,
                                                          const DevView *__restrict__ views,
                                                          const int32_t *__restrict__ fview_off,
                                                          const int32_t *__restrict__ fview_idx, float znear,
                                                          float *__restrict__ rec) {
  constexpr int NB = (L + 1) * (L + 1);
  extern __shared__ float s_k[];   // [3 NB][kProjThreads]
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < G; gi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = gi / N, g = gi - f * N;
    auto attr = [&](int c) { return __ldg(soa + (int64_t)c * G + gi); };
    Act a;
    activate(attr, a);
    auto k = [&](int j, int c) -> float & { return s_k[(3 * j + c) * kProjThreads + threadIdx.x]; };
    bool finite = a.finite;   // a Gaussian with a non-finite texel value is culled in every view
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float kv = attr(11 + 3 * j + c);
        k(j, c) = kv;
        finite = finite && isfinite(kv);
      }
    const int vb = __ldg(fview_off + f), ve = __ldg(fview_off + f + 1);
    for (int vi = vb; vi < ve; ++vi) {
      const int v = __ldg(fview_idx + vi);
      const DevView &view = views[v];
      float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
      Proj p;
      bool ok = finite && project(a, view, znear, p);
      if (ok) {
        float d[3], len;
        view_dir(a, view, d, len);
        float Y[NB];
        sh_basis<L>(d[0], d[1], d[2], Y);
        float rgb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float acc = 0.5f;
#pragma unroll
          for (int j = 0; j < NB; ++j) acc = fmaf(k(j, c), Y[j], acc);
          rgb[c] = fmaxf(acc, 0.f);
        }
        ok = isfinite(rgb[0]) && isfinite(rgb[1]) && isfinite(rgb[2]) && isfinite(a.o);
        if (ok) {
          r0 = make_float4(p.m[0], p.m[1], p.conic[0], p.conic[1]);
          r1 = make_float4(p.conic[2], a.o, p.X[2], p.radius);
          r2 = make_float4(rgb[0], rgb[1], rgb[2], 0.f);
        }
      }
      float4 *dst = reinterpret_cast<float4 *>(rec + ((int64_t)v * N + g) * kRec);
      dst[0] = r0;
      dst[1] = r1;
      dst[2] = r2;
    }
  }
}

}  // namespace

extern "C" pk_status pk_project_and_sh(const pk_plan *p, const float *soa, float *records, void *ws,
                                       pk_stream_t stream) {
  if (!p || !soa || !records || !ws) return PK_ERR_ARG;
  if (!aligned16(records)) return PK_ERR_ARG;
  if (p->G == 0) return PK_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const DevView *views = at<DevView>(ws, p->ws.views);
  const int32_t *fo = at<int32_t>(ws, p->ws.fview_off), *fi = at<int32_t>(ws, p->ws.fview_idx);
  int64_t blocks = (p->G + kProjThreads - 1) / kProjThreads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  const float zn = p->opts.znear;
  const size_t smem = sizeof(float) * 3 * (p->L + 1) * (p->L + 1) * kProjThreads;
  switch (p->L) {
    case 0: k_project<0><<<(int)blocks, kProjThreads, smem, st>>>(soa, p->G, p->N, views, fo, fi, zn, records); break;
    case 1: k_project<1><<<(int)blocks, kProjThreads, smem, st>>>(soa, p->G, p->N, views, fo, fi, zn, records); break;
    case 2: k_project<2><<<(int)blocks, kProjThreads, smem, st>>>(soa, p->G, p->N, views, fo, fi, zn, records); break;
    default: k_project<3><<<(int)blocks, kProjThreads, smem, st>>>(soa, p->G, p->N, views, fo, fi, zn, records); break;
  }
  return check_launch();
}
