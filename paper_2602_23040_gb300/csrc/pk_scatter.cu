// a6 -- chain the per-view 2D gradients back to the texel attributes, sum
// over the views of the Gaussian's frame, apply the freeze mask D_i
// (Sec. 4.2 "Gradient Freezing") and write the texel gradients (straight
// through the FP16 proxy, Sec. 4.2 "Low Precision Optimization").
//
// One thread per Gaussian: everything view-independent (the Sigma3D ->
// scale/rotation chain, the opacity sigmoid) is applied once after the
// loop over views; per view only the projection and the colour adjoints
// run.  Sums stay in registers, so no atomics are needed.
#include "pk_proj_math.cuh"

using namespace pk;

namespace {

constexpr int kScatterThreads = 128;
// 4 resident blocks per SM (at most 128 registers, a few spilled): latency
// of the per-view gradient loads, not arithmetic, bounds this kernel.

template <int L>
__global__ __launch_bounds__(kScatterThreads, 4) void k_scatter(const float *__restrict__ soa, int64_t G, int64_t N,
                                                 const DevView *__restrict__ views,
                                                 const int32_t *__restrict__ fview_off,
                                                 const int32_t *__restrict__ fview_idx, float znear,
                                                 const float *__restrict__ grad2d,
                                                 const uint8_t *__restrict__ dynflag,
                                                 const uint32_t *__restrict__ texel, int64_t plane, int D,
                                                 float *__restrict__ out, int accumulate) {
  constexpr int NB = (L + 1) * (L + 1);
  extern __shared__ float s_k[];   // [2 * 3 NB][kScatterThreads]: coefficients, then their gradients
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < G; gi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = gi / N, g = gi - f * N;
    float *dst = out + (int64_t)f * D * plane + __ldg(texel + g);
    if (dynflag && !__ldg(dynflag + g)) {
      if (!accumulate)
        for (int c = 0; c < D; ++c) dst[(int64_t)c * plane] = 0.f;
      continue;
    }
    auto attr = [&](int c) { return __ldg(soa + (int64_t)c * G + gi); };
    Act a;
    activate(attr, a);
    // SH coefficients and their gradient sums in shared memory, column tid
    // of s_k / s_dk (each thread touches only its own column)
    auto k = [&](int j, int c) -> float & { return s_k[(3 * j + c) * kScatterThreads + threadIdx.x]; };
    auto dk = [&](int j, int c) -> float & { return s_k[(3 * (NB + j) + c) * kScatterThreads + threadIdx.x]; };
    bool finite = a.finite;
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float kv = attr(11 + 3 * j + c);
        k(j, c) = kv;
        dk(j, c) = 0.f;
        finite = finite && isfinite(kv);
      }
    if (!finite) {   // culled in every view by the projection: a zero gradient
      if (!accumulate)
        for (int c = 0; c < D; ++c) dst[(int64_t)c * plane] = 0.f;
      continue;
    }
    float dmu[3] = {0.f, 0.f, 0.f};
    float dS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma3D entries xx xy xz yy yz zz
    float dop = 0.f;
    const int vb = __ldg(fview_off + f), ve = __ldg(fview_off + f + 1);
    // the next view's 2D gradient record is loaded while this view's is
    // chained, so two loads per thread are in flight instead of one
    auto load_g = [&](int vi, int &v, float4 &x0, float4 &x1, float4 &x2) {
      v = __ldg(fview_idx + vi);
      const float4 *gsrc = reinterpret_cast<const float4 *>(grad2d + ((int64_t)v * N + g) * kG2d);
      x0 = __ldg(gsrc);
      x1 = __ldg(gsrc + 1);
      x2 = __ldg(gsrc + 2);
    };
    int nv = 0;
    float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0, n2 = n0;
    if (vb < ve) load_g(vb, nv, n0, n1, n2);
    for (int vi = vb; vi < ve; ++vi) {
      const int v = nv;
      const float4 g0 = n0, g1 = n1, g2 = n2;
      if (vi + 1 < ve) load_g(vi + 1, nv, n0, n1, n2);
      if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f &&
          g1.z == 0.f && g1.w == 0.f && g2.x == 0.f)
        continue;
      const DevView &view = views[v];
      Proj p;
      if (!project(a, view, znear, p)) continue;
      // colour: rgb = max(0, sum_j k_j Y_j(dir) + 0.5)
      {
        float d[3], len;
        view_dir(a, view, d, len);
        float Y[NB];
        sh_basis<L>(d[0], d[1], d[2], Y);
        const float grgb[3] = {g1.z, g1.w, g2.x};
        float gcs[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float pre = 0.5f;
#pragma unroll
          for (int j = 0; j < NB; ++j) pre = fmaf(k(j, c), Y[j], pre);
          gcs[c] = pre >= 0.f ? grgb[c] : 0.f;
        }
        // d rgb_c / d dir = sum_j k_jc grad Y_j: contract the channels first
        float K[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
          float kj = 0.f;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float kc = k(j, c);
            dk(j, c) = fmaf(gcs[c], Y[j], dk(j, c));
            kj = fmaf(gcs[c], kc, kj);
          }
          K[j] = kj;
        }
        float ddir[3];
        sh_grad_dot<L>(d[0], d[1], d[2], K, ddir);
        const float dd = ddir[0] * d[0] + ddir[1] * d[1] + ddir[2] * d[2];
        const float il = 1.f / len;
#pragma unroll
        for (int c = 0; c < 3; ++c) dmu[c] += (ddir[c] - d[c] * dd) * il;
      }
      dop += g1.y;
      // conic = Sigma2D^-1  ->  dL/dSigma2D = -Q G_Q Q
      const float ca = p.conic[0], cb = p.conic[1], cc = p.conic[2];
      const float ga = g0.z, gb = 0.5f * g0.w, gc = g1.x;
      const float m00 = ga * ca + gb * cb, m01 = ga * cb + gb * cc;
      const float m10 = gb * ca + gc * cb, m11 = gb * cb + gc * cc;
      const float S00 = -(ca * m00 + cb * m10), S01 = -(ca * m01 + cb * m11), S11 = -(cb * m01 + cc * m11);
      // Sigma2D = T Sigma3D T^T + 0.3 I,  T rows t0, t1
      const float *t0 = p.t0, *t1 = p.t1;
      dS[0] += S00 * t0[0] * t0[0] + 2.f * S01 * t0[0] * t1[0] + S11 * t1[0] * t1[0];
      dS[1] += S00 * t0[0] * t0[1] + S01 * (t0[0] * t1[1] + t1[0] * t0[1]) + S11 * t1[0] * t1[1];
      dS[2] += S00 * t0[0] * t0[2] + S01 * (t0[0] * t1[2] + t1[0] * t0[2]) + S11 * t1[0] * t1[2];
      dS[3] += S00 * t0[1] * t0[1] + 2.f * S01 * t0[1] * t1[1] + S11 * t1[1] * t1[1];
      dS[4] += S00 * t0[1] * t0[2] + S01 * (t0[1] * t1[2] + t1[1] * t0[2]) + S11 * t1[1] * t1[2];
      dS[5] += S00 * t0[2] * t0[2] + 2.f * S01 * t0[2] * t1[2] + S11 * t1[2] * t1[2];
      const float *S = a.S;
      float u0[3], u1[3];
      u0[0] = S[0] * t0[0] + S[1] * t0[1] + S[2] * t0[2];
      u0[1] = S[1] * t0[0] + S[3] * t0[1] + S[4] * t0[2];
      u0[2] = S[2] * t0[0] + S[4] * t0[1] + S[5] * t0[2];
      u1[0] = S[0] * t1[0] + S[1] * t1[1] + S[2] * t1[2];
      u1[1] = S[1] * t1[0] + S[3] * t1[1] + S[4] * t1[2];
      u1[2] = S[2] * t1[0] + S[4] * t1[1] + S[5] * t1[2];
      float dT0[3], dT1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dT0[c] = 2.f * (S00 * u0[c] + S01 * u1[c]);
        dT1[c] = 2.f * (S01 * u0[c] + S11 * u1[c]);
      }
      // T = J W  ->  dJ = dT W^T (only the non-zero entries of J)
      const float *W = view.R;
      const float dJ00 = W[0] * dT0[0] + W[1] * dT0[1] + W[2] * dT0[2];
      const float dJ02 = W[6] * dT0[0] + W[7] * dT0[1] + W[8] * dT0[2];
      const float dJ11 = W[3] * dT1[0] + W[4] * dT1[1] + W[5] * dT1[2];
      const float dJ12 = W[6] * dT1[0] + W[7] * dT1[1] + W[8] * dT1[2];
      const float x = p.X[0], y = p.X[1], iz = p.iz, iz2 = iz * iz, iz3 = iz2 * iz;
      const float fx = view.fx, fy = view.fy;
      const float gmx = g0.x, gmy = g0.y;
      float dX0 = gmx * fx * iz - dJ02 * fx * iz2;
      float dX1 = gmy * fy * iz - dJ12 * fy * iz2;
      float dX2 = -gmx * fx * x * iz2 - gmy * fy * y * iz2 - dJ00 * fx * iz2 + 2.f * dJ02 * fx * x * iz3 -
                  dJ11 * fy * iz2 + 2.f * dJ12 * fy * y * iz3;
      dmu[0] += W[0] * dX0 + W[3] * dX1 + W[6] * dX2;
      dmu[1] += W[1] * dX0 + W[4] * dX1 + W[7] * dX2;
      dmu[2] += W[2] * dX0 + W[5] * dX1 + W[8] * dX2;
    }
    // Sigma3D = M M^T, M = R diag(s):  dM = 2 dSigma M
    const float *R = a.R;
    const float G3[9] = {dS[0], dS[1], dS[2], dS[1], dS[3], dS[4], dS[2], dS[4], dS[5]};
    float dR[9], dls[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      float ds = 0.f;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float dM = 2.f * (G3[3 * r] * R[kk] + G3[3 * r + 1] * R[3 + kk] + G3[3 * r + 2] * R[6 + kk]) * a.s[kk];
        ds += R[3 * r + kk] * dM;
        dR[3 * r + kk] = dM * a.s[kk];
      }
      dls[kk] = ds * a.s[kk];
    }
    const float qw = a.qn[0], qx = a.qn[1], qy = a.qn[2], qz = a.qn[3];
    float dq[4];
    dq[0] = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
    dq[1] = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - qw * dR[5] + qz * dR[6] + qw * dR[7] -
                   2.f * qx * dR[8]);
    dq[2] = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + qw * dR[2] + qx * dR[3] + qz * dR[5] - qw * dR[6] +
                   qz * dR[7] - 2.f * qy * dR[8]);
    dq[3] = 2.f * (-2.f * qz * dR[0] - qw * dR[1] + qx * dR[2] + qw * dR[3] - 2.f * qz * dR[4] + qy * dR[5] +
                   qx * dR[6] + qy * dR[7]);
    const float dot = dq[0] * qw + dq[1] * qx + dq[2] * qy + dq[3] * qz;
    float outv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) outv[i] = (dq[i] - a.qn[i] * dot) * a.qinv;
    const float dlogit = dop * a.o * (1.f - a.o);
    auto put = [&](int c, float val) {
      float *q = dst + (int64_t)c * plane;
      *q = accumulate ? *q + val : val;
    };
    put(0, dmu[0]);
    put(1, dmu[1]);
    put(2, dmu[2]);
    put(3, dls[0]);
    put(4, dls[1]);
    put(5, dls[2]);
    put(6, outv[0]);
    put(7, outv[1]);
    put(8, outv[2]);
    put(9, outv[3]);
    put(10, dlogit);
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) put(11 + 3 * j + c, dk(j, c));
  }
}

}  // namespace

extern "C" pk_status pk_atlas_scatter_grad(const pk_plan *p, const float *soa, const float *grad2d,
                                           const uint8_t *dynflag, const uint32_t *texel, float *grad_atlas,
                                           int32_t accumulate, void *ws, pk_stream_t stream) {
  if (!p || !soa || !grad2d || !texel || !grad_atlas || !ws) return PK_ERR_ARG;
  if (!aligned16(grad2d)) return PK_ERR_ARG;
  if (p->G == 0) return PK_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const DevView *views = at<DevView>(ws, p->ws.views);
  const int32_t *fo = at<int32_t>(ws, p->ws.fview_off), *fi = at<int32_t>(ws, p->ws.fview_idx);
  const int64_t plane = (int64_t)p->desc.atlas_w * p->desc.atlas_h;
  int64_t blocks = (p->G + kScatterThreads - 1) / kScatterThreads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  const float zn = p->opts.znear;
  const int acc = accumulate ? 1 : 0;
  const size_t smem = sizeof(float) * 6 * (p->L + 1) * (p->L + 1) * kScatterThreads;
#define PK_SCATTER(LL)                                                                                     \
  k_scatter<LL><<<(int)blocks, kScatterThreads, smem, st>>>(soa, p->G, p->N, views, fo, fi, zn, grad2d,   \
                                                            dynflag, texel, plane, p->D, grad_atlas, acc)
  switch (p->L) {
    case 0: PK_SCATTER(0); break;
    case 1: PK_SCATTER(1); break;
    case 2: PK_SCATTER(2); break;
    default: PK_SCATTER(3); break;
  }
#undef PK_SCATTER
  return check_launch();
}
