// FP32 activation, EWA projection and SH colour, forward and adjoint, shared
// by the projection kernel (a2) and the gradient scatter kernel (a6) so the
// scatter recomputes exactly the forward's intermediates.
//
// Passages: Sec. 4.2 "Covariance-Aware Gaussian Masking" and Alg. 1 steps
// 1-4 (Sigma3D = R(q) diag(s^2) R(q)^T, Sigma_cam = W Sigma3D W^T,
// Sigma2D = J Sigma_cam J^T + 0.3 I with J the pinhole Jacobian at the
// camera-space mean, det <= 1e-7 invalid, lambda_max, r = ceil(3
// sqrt(lambda_max))); Supp. "Viewer" (X_c = R X + t, perspective division).
#pragma once

#include "pk_common.cuh"

namespace pk {

// Real SH basis (Condon-Shortley phase), index j = l^2 + l + m, as
// homogeneous polynomials of the unit direction.  Constants are the
// closed-form normalisations:
//   c0 = 1/(2 sqrt(pi))          c1 = sqrt(3/(4 pi))
//   c2a = sqrt(15/pi)/2          c2c = sqrt(5/pi)/4       c2e = sqrt(15/pi)/4
//   c3a = sqrt(35/(32 pi))       c3b = sqrt(105/pi)/2     c3c = sqrt(42/pi)/8
//   c3d = sqrt(7/pi)/4           c3f = sqrt(105/pi)/4
constexpr float kC0 = 0.28209479177387814f;
constexpr float kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2c = 0.31539156525252005f;
constexpr float kC2e = 0.5462742152960396f;
constexpr float kC3a = 0.5900435899266435f;
constexpr float kC3b = 2.890611442640554f;
constexpr float kC3c = 0.4570457994644658f;
constexpr float kC3d = 0.3731763325901154f;
constexpr float kC3f = 1.445305721320277f;

template <int L>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
  Y[0] = kC0;
  if (L >= 1) {
    Y[1] = -kC1 * y;
    Y[2] = kC1 * z;
    Y[3] = -kC1 * x;
  }
  if (L >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y;
    Y[5] = -kC2a * y * z;
    Y[6] = kC2c * (2.f * zz - xx - yy);
    Y[7] = -kC2a * x * z;
    Y[8] = kC2e * (xx - yy);
    if (L >= 3) {
      Y[9] = -kC3a * y * (3.f * xx - yy);
      Y[10] = kC3b * x * y * z;
      Y[11] = -kC3c * y * (4.f * zz - xx - yy);
      Y[12] = kC3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -kC3c * x * (4.f * zz - xx - yy);
      Y[14] = kC3f * z * (xx - yy);
      Y[15] = -kC3a * x * (xx - 3.f * yy);
    }
  }
}

// sum_j K_j grad Y_j(x, y, z) for the polynomials above (their gradient
// with respect to (x, y, z), contracted with the weights K without forming
// the 3 x (L+1)^2 gradient table).
template <int L>
__device__ __forceinline__ void sh_grad_dot(float x, float y, float z, const float *K, float *g) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (L >= 1) {
    gx = -kC1 * K[3];
    gy = -kC1 * K[1];
    gz = kC1 * K[2];
  }
  if (L >= 2) {
    const float a4 = kC2a * K[4], a5 = kC2a * K[5], a7 = kC2a * K[7];
    const float c6 = 2.f * kC2c * K[6], e8 = 2.f * kC2e * K[8];
    gx += a4 * y - a7 * z - c6 * x + e8 * x;
    gy += a4 * x - a5 * z - c6 * y - e8 * y;
    gz += -a5 * y + 2.f * c6 * z - a7 * x;
    if (L >= 3) {
      const float xx = x * x, yy = y * y, zz = z * z;
      const float k9 = kC3a * K[9], k10 = kC3b * K[10], k11 = kC3c * K[11], k12 = kC3d * K[12];
      const float k13 = kC3c * K[13], k14 = kC3f * K[14], k15 = kC3a * K[15];
      // Y9 = -a y (3x^2 - y^2): (-6a x y, -3a (x^2 - y^2), 0)
      gx += -6.f * k9 * x * y;
      gy += -3.f * k9 * (xx - yy);
      // Y10 = b x y z
      gx += k10 * y * z;
      gy += k10 * x * z;
      gz += k10 * x * y;
      // Y11 = -c y (4z^2 - x^2 - y^2): (2c x y, -c (4z^2 - x^2 - 3y^2), -8c y z)
      gx += 2.f * k11 * x * y;
      gy += -k11 * (4.f * zz - xx - 3.f * yy);
      gz += -8.f * k11 * y * z;
      // Y12 = d z (2z^2 - 3x^2 - 3y^2): (-6d x z, -6d y z, d (6z^2 - 3x^2 - 3y^2))
      gx += -6.f * k12 * x * z;
      gy += -6.f * k12 * y * z;
      gz += k12 * (6.f * zz - 3.f * xx - 3.f * yy);
      // Y13 = -c x (4z^2 - x^2 - y^2): (-c (4z^2 - 3x^2 - y^2), 2c x y, -8c x z)
      gx += -k13 * (4.f * zz - 3.f * xx - yy);
      gy += 2.f * k13 * x * y;
      gz += -8.f * k13 * x * z;
      // Y14 = f z (x^2 - y^2): (2f x z, -2f y z, f (x^2 - y^2))
      gx += 2.f * k14 * x * z;
      gy += -2.f * k14 * y * z;
      gz += k14 * (xx - yy);
      // Y15 = -a x (x^2 - 3y^2): (-3a (x^2 - y^2), 6a x y, 0)
      gx += -3.f * k15 * (xx - yy);
      gy += 6.f * k15 * x * y;
    }
  }
  g[0] = gx;
  g[1] = gy;
  g[2] = gz;
}

// View-independent activation of one Gaussian.
struct Act {
  float mu[3];
  float s[3];      // exp(log-scale)
  float qn[4];     // q / |q|  (w, x, y, z)
  float qinv;      // 1 / |q|
  float R[9];      // rotation of qn, row-major
  float S[6];      // Sigma3D: xx, xy, xz, yy, yz, zz
  float o;         // sigmoid(logit)
  bool finite;     // channels 0..10 (position, log-scale, quaternion, opacity logit) all finite
};

// attr(c) reads channel c of this Gaussian.
template <typename Get>
__device__ __forceinline__ void activate(const Get &attr, Act &a) {
  a.mu[0] = attr(0);
  a.mu[1] = attr(1);
  a.mu[2] = attr(2);
  const float l0 = attr(3), l1 = attr(4), l2 = attr(5), logit = attr(10);
  a.s[0] = expf(l0);
  a.s[1] = expf(l1);
  a.s[2] = expf(l2);
  float qw = attr(6), qx = attr(7), qy = attr(8), qz = attr(9);
  a.finite = isfinite(a.mu[0]) && isfinite(a.mu[1]) && isfinite(a.mu[2]) && isfinite(l0) && isfinite(l1) &&
             isfinite(l2) && isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) && isfinite(logit);
  float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
  a.qinv = rsqrtf(n2);
  qw *= a.qinv; qx *= a.qinv; qy *= a.qinv; qz *= a.qinv;
  a.qn[0] = qw; a.qn[1] = qx; a.qn[2] = qy; a.qn[3] = qz;
  float *R = a.R;
  R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
  R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
  R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
  const float s0 = a.s[0] * a.s[0], s1 = a.s[1] * a.s[1], s2 = a.s[2] * a.s[2];
  // Sigma = R diag(s^2) R^T
  a.S[0] = R[0] * R[0] * s0 + R[1] * R[1] * s1 + R[2] * R[2] * s2;
  a.S[1] = R[0] * R[3] * s0 + R[1] * R[4] * s1 + R[2] * R[5] * s2;
  a.S[2] = R[0] * R[6] * s0 + R[1] * R[7] * s1 + R[2] * R[8] * s2;
  a.S[3] = R[3] * R[3] * s0 + R[4] * R[4] * s1 + R[5] * R[5] * s2;
  a.S[4] = R[3] * R[6] * s0 + R[4] * R[7] * s1 + R[5] * R[8] * s2;
  a.S[5] = R[6] * R[6] * s0 + R[7] * R[7] * s1 + R[8] * R[8] * s2;
  a.o = 1.f / (1.f + expf(-logit));
}

// Per-view projection of one activated Gaussian.
struct Proj {
  float X[3];      // camera-space mean
  float iz;
  float t0[3], t1[3];  // rows of T = J W
  float A, B, C;   // Sigma2D incl. low-pass
  float det;
  float conic[3];
  float m[2];
  float radius;
};

__device__ __forceinline__ bool project(const Act &a, const DevView &v, float znear, Proj &p) {
  const float *W = v.R;
  p.X[0] = W[0] * a.mu[0] + W[1] * a.mu[1] + W[2] * a.mu[2] + v.t[0];
  p.X[1] = W[3] * a.mu[0] + W[4] * a.mu[1] + W[5] * a.mu[2] + v.t[1];
  p.X[2] = W[6] * a.mu[0] + W[7] * a.mu[1] + W[8] * a.mu[2] + v.t[2];
  const float z = p.X[2];
  if (!(z > znear)) return false;
  const float iz = 1.f / z;
  p.iz = iz;
  const float j00 = v.fx * iz, j02 = -v.fx * p.X[0] * iz * iz;
  const float j11 = v.fy * iz, j12 = -v.fy * p.X[1] * iz * iz;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p.t0[k] = j00 * W[k] + j02 * W[6 + k];
    p.t1[k] = j11 * W[3 + k] + j12 * W[6 + k];
  }
  const float *S = a.S;
  float u0[3], u1[3];  // Sigma3D t0, Sigma3D t1
  u0[0] = S[0] * p.t0[0] + S[1] * p.t0[1] + S[2] * p.t0[2];
  u0[1] = S[1] * p.t0[0] + S[3] * p.t0[1] + S[4] * p.t0[2];
  u0[2] = S[2] * p.t0[0] + S[4] * p.t0[1] + S[5] * p.t0[2];
  u1[0] = S[0] * p.t1[0] + S[1] * p.t1[1] + S[2] * p.t1[2];
  u1[1] = S[1] * p.t1[0] + S[3] * p.t1[1] + S[4] * p.t1[2];
  u1[2] = S[2] * p.t1[0] + S[4] * p.t1[1] + S[5] * p.t1[2];
  p.A = p.t0[0] * u0[0] + p.t0[1] * u0[1] + p.t0[2] * u0[2] + kLowPass;
  p.B = p.t1[0] * u0[0] + p.t1[1] * u0[1] + p.t1[2] * u0[2];
  p.C = p.t1[0] * u1[0] + p.t1[1] * u1[1] + p.t1[2] * u1[2] + kLowPass;
  p.det = p.A * p.C - p.B * p.B;
  if (!(p.det > kDetMin)) return false;
  const float idet = 1.f / p.det;
  p.conic[0] = p.C * idet;
  p.conic[1] = -p.B * idet;
  p.conic[2] = p.A * idet;
  p.m[0] = v.fx * p.X[0] * iz + v.cx;
  p.m[1] = v.fy * p.X[1] * iz + v.cy;
  const float tr = p.A + p.C;
  const float lam = 0.5f * (tr + sqrtf(fmaxf(0.f, tr * tr - 4.f * p.det)));
  p.radius = ceilf(3.f * sqrtf(lam));
  return isfinite(p.m[0]) && isfinite(p.m[1]) && isfinite(p.conic[0]) && isfinite(p.conic[1]) &&
         isfinite(p.conic[2]) && isfinite(p.radius);
}

// Unit viewing direction and its length.
__device__ __forceinline__ void view_dir(const Act &a, const DevView &v, float *d, float &len) {
  float u0 = a.mu[0] - v.campos[0], u1 = a.mu[1] - v.campos[1], u2 = a.mu[2] - v.campos[2];
  len = sqrtf(u0 * u0 + u1 * u1 + u2 * u2);
  const float il = 1.f / len;
  d[0] = u0 * il;
  d[1] = u1 * il;
  d[2] = u2 * il;
}

}  // namespace pk
