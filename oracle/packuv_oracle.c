/*
 * PackUV-GS render step -- plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal definition of
 * what the GPU library computes.  Only the test-suite, the package smoke
 * check and the CPU-baseline leg of the benchmark load it.  It includes no
 * header of the CUDA library and the CUDA library includes nothing from
 * here; the two share no code.
 *
 * Passages of PackUV (arXiv 2602.23040) followed, by function:
 *   or_pyramid_sizes   Sec. 4.1 "Pyramid UV Mapping", the unnumbered
 *                      equation for (M_k, N_k)
 *   or_atlas_layout    Sec. 4.1 "UV Atlas Layout" (L0 right, L1 rotated 90
 *                      deg CCW and L2 on the left, deeper levels rightward of
 *                      L2, odd rotated / even horizontal; 88.5 % efficiency)
 *   or_gather          Sec. 4.2 "Fitting UV Maps Directly" (U[u,v,k] = g_i)
 *                      and "Low Precision Optimization" (the renderer reads a
 *                      low-precision proxy; FP16 texels decoded here)
 *   or_project         Sec. 4.2 "Covariance-Aware Gaussian Masking" and
 *                      Alg. 1 steps 1-4 (Sigma3D = R diag(s^2) R^T, EWA
 *                      Jacobian J, +0.3 low-pass, det check, lambda_max,
 *                      r = ceil(3 sqrt(lambda_max))); Supp. "Viewer" for the
 *                      pinhole projection X_c = R X + t; Sec. 3 (3DGS:
 *                      opacity, SH colour)
 *   or_bin_sort        Sec. 3 (tile-based rasterizer) and Supp. "Viewer"
 *                      (Gaussians depth-sorted per camera); a tile receives
 *                      a splat if its 3-sigma footprint (Sec. 4.2, d^2 <= 9)
 *                      reaches the tile (or, in the rectangle mode, if the
 *                      tile meets the r = ceil(3 sqrt(lambda_max)) square)
 *   or_render          Supp. "Viewer" compositing C = sum T_i a_i c_i,
 *                      T_i = prod_{j<i} (1 - a_j); footprint d^2 <= 9 of
 *                      Sec. 4.2 / Alg. 1 step 5
 *   or_render_bwd,     the analytic adjoint of the above (Sec. 4.2
 *   or_scatter_grad    "Objective": gradients of the photometric loss flow
 *                      to every attribute) and gradient freezing
 *                      grad_i <- D_i grad_i (Sec. 4.2 "Gradient Freezing")
 *   or_motion_mask     Sec. 4.2 "Optical Flow and Binary Motion Masks"
 *                      (flow magnitude above tau, then dilation)
 *   or_dynamic_mask,   Sec. 4.2 "Covariance-Aware Gaussian Masking" and
 *   or_dynamic_mask32  Alg. 1 step 5: a Gaussian is dynamic if a masked
 *                      pixel of some view lies in its d^2 <= 9 ellipse,
 *                      OR-ed over the views
 *   or_lpo_minmax,     Sec. 4.2 "Low Precision Optimization" and Supp.
 *   or_lpo_encode,     "Video Coding": per-channel min/max normalisation,
 *   or_lpo_decode      uniform 16-bit (position, as two 8-bit planes) and
 *                      8-bit (all other channels) quantisation, proxy
 *                      lo + q Delta
 *   or_uv_cell,        Sec. 3 "UV-based Point-to-Image Transformation"
 *   or_uv_max_k        (eq. uvgs2) and Sec. 4.2 "UV-Based Pruning": valid
 *                      UV projection, top-K Gaussians per cell by opacity
 *   or_photo_loss      Sec. 4.2 "Objective": (1 - lambda) L1 +
 *                      lambda (1 - SSIM) and its gradient
 *
 * Where the paper is silent the readings are: 3DGS conventions for the
 * opacity sigmoid, the +0.5 SH offset and the clamp of colour at 0; alpha
 * clamp 0.99, skip below 1/255, stop (excluding the Gaussian) when the
 * transmittance would fall below 1e-4; real SH with the Condon-Shortley
 * phase, coefficient j = l^2 + l + m; pixel centres at (i + 0.5, j + 0.5).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_VS 20   /* doubles per view: R[9] t[3] fx fy cx cy width height frame pad */
#define OR_REC 12  /* doubles per projected record */
#define OR_G2D 9   /* doubles per per-view 2D gradient */

enum {
  R_MX = 0, R_MY, R_CA, R_CB, R_CC, R_OP, R_Z, R_RAD, R_RED, R_GRN, R_BLU, R_FLAGS
};

/* record flag bits */
#define F_CULL_NEAR 1u   /* z or det within 1e-5 (relative) of its culling cutoff */
#define F_CLAMP_NEAR 2u  /* a pre-clamp colour channel within 1e-6 of 0 */

/* pixel borderline bits */
#define B_Q 1u        /* d^2 near 9 */
#define B_ALPHA 2u    /* alpha near 1/255 */
#define B_STOP 4u     /* transmittance near 1e-4 */
#define B_DEPTH 8u    /* two contributors with (nearly) equal FP32 depth */
#define B_CULL 16u    /* a contributor was near a culling cutoff */
#define B_CLAMP 32u   /* a contributor has alpha near the 0.99 clamp (gradient only) */

static const double ALPHA_MAX = 0.99;
static const double ALPHA_MIN = 1.0 / 255.0;
static const double T_MIN = 1e-4;
static const double Q_MAX = 9.0;
static const double LOWPASS = 0.3;
static const double DET_MIN = 1e-7;

/* ------------------------------------------------------------------------ */
/* Pyramid and atlas layout                                                 */
/* ------------------------------------------------------------------------ */

/* (M_0, N_0) = base; odd k halves N, even k halves M. */
int or_pyramid_sizes(int M0, int N0, int K, int32_t *M, int32_t *N) {
  if (K < 1 || K > 16 || M0 < 1 || N0 < 1) return -1;
  M[0] = M0;
  N[0] = N0;
  for (int k = 1; k < K; ++k) {
    if (k % 2 == 1) {
      M[k] = M[k - 1];
      N[k] = N[k - 1] / 2;
    } else {
      M[k] = M[k - 1] / 2;
      N[k] = N[k - 1];
    }
    if (M[k] < 1 || N[k] < 1) return -1;
  }
  return 0;
}

/*
 * Packed layout of K pyramid levels of a square base S x S.  Native level k
 * is M_k texels wide (along u) and N_k high (along v).  Output per level:
 * stored width, stored height, x0, y0, rotated.  Reading of the text: L0
 * right; L1 rotated CCW in the left column above L2; levels >= 3 left to
 * right in the strip below L0 starting right of L2, odd ones rotated.
 */
int or_atlas_layout(int S, int K, int32_t *lv, int32_t *WH) {
  int32_t M[16], N[16];
  if (or_pyramid_sizes(S, S, K, M, N)) return -1;
  int W = 0, H = 0;
  for (int k = 0; k < K; ++k) {
    int w, h, x0, y0, rot = 0;
    if (K == 1) {
      w = M[0]; h = N[0]; x0 = 0; y0 = 0;
    } else if (k == 0) {
      w = M[0]; h = N[0]; x0 = N[1]; y0 = 0;
    } else if (k == 1) {
      w = N[1]; h = M[1]; x0 = 0; y0 = 0; rot = 1;
    } else if (k == 2) {
      w = M[2]; h = N[2]; x0 = 0; y0 = M[1];
    } else {
      int x = M[2];
      for (int j = 3; j < k; ++j) x += (j % 2 == 1) ? N[j] : M[j];
      rot = (k % 2 == 1);
      w = rot ? N[k] : M[k];
      h = rot ? M[k] : N[k];
      x0 = x; y0 = M[1];
    }
    lv[5 * k + 0] = w; lv[5 * k + 1] = h; lv[5 * k + 2] = x0; lv[5 * k + 3] = y0; lv[5 * k + 4] = rot;
    if (x0 + w > W) W = x0 + w;
    if (y0 + h > H) H = y0 + h;
  }
  WH[0] = W;
  WH[1] = H;
  return 0;
}

/* Atlas texel (x, y) -> (level, u, v); returns -1 if in no level. */
int or_texel_to_uv(const int32_t *lv, int K, int x, int y, int32_t *out) {
  for (int k = 0; k < K; ++k) {
    int w = lv[5 * k], h = lv[5 * k + 1], x0 = lv[5 * k + 2], y0 = lv[5 * k + 3], rot = lv[5 * k + 4];
    if (x < x0 || x >= x0 + w || y < y0 || y >= y0 + h) continue;
    out[0] = k;
    if (rot) {            /* stored h x w of a native (h wide, w high) level */
      out[1] = h - 1 - (y - y0);
      out[2] = x - x0;
    } else {
      out[1] = x - x0;
      out[2] = y - y0;
    }
    return 0;
  }
  return -1;
}

int or_uv_to_texel(const int32_t *lv, int K, int k, int u, int v, int32_t *xy) {
  if (k < 0 || k >= K) return -1;
  int w = lv[5 * k], h = lv[5 * k + 1], x0 = lv[5 * k + 2], y0 = lv[5 * k + 3], rot = lv[5 * k + 4];
  if (rot) {
    if (u < 0 || u >= h || v < 0 || v >= w) return -1;
    xy[0] = x0 + v;
    xy[1] = y0 + (h - 1 - u);
  } else {
    if (u < 0 || u >= w || v < 0 || v >= h) return -1;
    xy[0] = x0 + u;
    xy[1] = y0 + v;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Gather                                                                    */
/* ------------------------------------------------------------------------ */

/* IEEE 754 binary16 -> double, from the format definition. */
double or_half_to_double(uint16_t h) {
  int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0)
    v = ldexp((double)m, -24);
  else if (e == 31)
    v = m ? NAN : INFINITY;
  else
    v = ldexp((double)(1024 + m), e - 25);
  return s ? -v : v;
}

static int bit_at(const uint32_t *bits, int Wp, int x, int y) {
  return (int)((bits[(int64_t)y * Wp + (x >> 5)] >> (x & 31)) & 1u);
}

int64_t or_count_live(const uint32_t *occ, int H, int W) {
  int Wp = (W + 31) / 32;
  int64_t n = 0;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) n += bit_at(occ, Wp, x, y);
  return n;
}

/*
 * Live texels in row-major atlas order become Gaussians 0..N-1 of every
 * frame; attribute c of Gaussian g of frame f lands at soa[c][f*N + g].
 * dtype 0 = float32 texels, 1 = IEEE half texels.  Returns N, or -1 if the
 * occupancy holds a different number of live texels than N.
 */
int64_t or_gather(const void *atlas, int dtype, int F, int D, int H, int W,
                  const uint32_t *occ, const uint32_t *dyn, int64_t N,
                  double *soa, uint32_t *texel, uint8_t *dynflag) {
  int Wp = (W + 31) / 32;
  if (or_count_live(occ, H, W) != N) return -1;
  int64_t G = (int64_t)F * N, g = 0;
  for (int y = 0; y < H; ++y) {
    for (int x = 0; x < W; ++x) {
      if (!bit_at(occ, Wp, x, y)) continue;
      texel[g] = (uint32_t)(y * W + x);
      dynflag[g] = dyn ? (uint8_t)bit_at(dyn, Wp, x, y) : 1;
      for (int f = 0; f < F; ++f) {
        for (int c = 0; c < D; ++c) {
          int64_t off = (((int64_t)f * D + c) * H + y) * W + x;
          double val = dtype == 1 ? or_half_to_double(((const uint16_t *)atlas)[off])
                                  : (double)((const float *)atlas)[off];
          soa[(int64_t)c * G + (int64_t)f * N + g] = val;
        }
      }
      ++g;
    }
  }
  return N;
}

/* ------------------------------------------------------------------------ */
/* Rotation and spherical harmonics                                         */
/* ------------------------------------------------------------------------ */

/* Rotation matrix (row-major) of a unit quaternion (w, x, y, z). */
void or_quat_rot(const double *q, double *R) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR[e][i] = d R_e / d q_i for the formula above. */
static void quat_rot_jac(const double *q, double dR[9][4]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double t[9][4] = {
      {0, 0, -4 * y, -4 * z},
      {-2 * z, 2 * y, 2 * x, -2 * w},
      {2 * y, 2 * z, 2 * w, 2 * x},
      {2 * z, 2 * y, 2 * x, 2 * w},
      {0, -4 * x, 0, -4 * z},
      {-2 * x, -2 * w, 2 * z, 2 * y},
      {-2 * y, 2 * z, -2 * w, 2 * x},
      {2 * x, 2 * w, 2 * z, 2 * y},
      {0, -4 * x, -4 * y, 0},
  };
  memcpy(dR, t, sizeof(t));
}

static double factorial(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

/* Normalisation K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!). */
static double sh_norm(int l, int m) {
  return sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
}

/* Coefficients (ascending powers of z) of the Legendre polynomial P_l, by
   Bonnet's recursion (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1}. */
static void legendre(int l, double c[8]) {
  double p0[8] = {1}, p1[8] = {0, 1}, p2[8];
  if (l == 0) { memcpy(c, p0, sizeof(p0)); return; }
  for (int n = 1; n < l; ++n) {
    memset(p2, 0, sizeof(p2));
    for (int i = 0; i < 7; ++i) p2[i + 1] += (2.0 * n + 1.0) * p1[i];
    for (int i = 0; i < 8; ++i) p2[i] -= n * p0[i];
    for (int i = 0; i < 8; ++i) p2[i] /= (n + 1.0);
    memcpy(p0, p1, sizeof(p1));
    memcpy(p1, p2, sizeof(p2));
  }
  memcpy(c, p1, sizeof(p1));
}

/* k-th derivative of the polynomial c, evaluated at z. */
static double poly_deriv_eval(const double c[8], int k, double z) {
  double s = 0.0, zp = 1.0;
  for (int i = k; i < 8; ++i) {
    double f = 1.0;
    for (int j = 0; j < k; ++j) f *= (i - j);
    s += c[i] * f * zp;
    zp *= z;
  }
  return s;
}

/*
 * Real spherical harmonics up to degree deg at unit direction d, and their
 * gradient (of the polynomial extension in x, y, z).  Y_lm for m > 0 is
 * sqrt(2) K_lm P_l^m(z) cos(m phi), for m < 0 sqrt(2) K_l|m| P_l^|m|(z)
 * sin(|m| phi), for m = 0 K_l0 P_l(z), with the Condon-Shortley phase in
 * P_l^m.  With P_l^m(z) = (-1)^m (1 - z^2)^(m/2) d^m P_l/dz^m and
 * sin^m(theta) e^{i m phi} = (x + i y)^m this is a polynomial in x, y, z.
 */
void or_sh_basis(int deg, const double *d, double *Y, double *dY /* [16][3] or NULL */) {
  double x = d[0], y = d[1], z = d[2];
  for (int l = 0; l <= deg; ++l) {
    double P[8];
    legendre(l, P);
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      int j = l * l + l + m;
      /* w^am and w^(am-1), w = x + i y */
      double re = 1, im = 0, re1 = 0, im1 = 0;
      for (int i = 0; i < am; ++i) {
        re1 = re; im1 = im;
        double nr = re * x - im * y, ni = re * y + im * x;
        re = nr; im = ni;
      }
      double c = (m == 0) ? sh_norm(l, 0) : sqrt(2.0) * sh_norm(l, am) * ((am % 2) ? -1.0 : 1.0);
      double Pm = poly_deriv_eval(P, am, z), Pm1 = poly_deriv_eval(P, am + 1, z);
      double W = (m == 0) ? 1.0 : (m > 0 ? re : im);
      double Wx = 0, Wy = 0;
      if (m > 0) { Wx = am * re1; Wy = -am * im1; }
      if (m < 0) { Wx = am * im1; Wy = am * re1; }
      Y[j] = c * Pm * W;
      if (dY) {
        dY[3 * j + 0] = c * Pm * Wx;
        dY[3 * j + 1] = c * Pm * Wy;
        dY[3 * j + 2] = c * Pm1 * W;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Projection (activation, EWA, colour)                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  double mu[3], s[3], qraw[4], qn[4], qnorm, R[9], S3[9];
  double X[3], J[6], T[6], A, B, C, det, conic[3], m[2], lam, radius, o, logit;
  double u[3], unorm, dir[3], Y[16], dY[48], vpre[3], rgb[3];
  int valid, flags, nb;
} proj_t;

static int near_rel(double a, double cut, double rel) {
  return fabs(a - cut) <= rel * fabs(cut);
}

/* attr points at the D attributes of one Gaussian, with stride `stride`. */
static void project_one(const double *attr, int64_t stride, int sh_deg, const double *cv,
                        double znear, proj_t *P) {
  memset(P, 0, sizeof(*P));
  /* a Gaussian with a non-finite texel value (any of its D channels) is
     culled in every view (reading of the contract's "non-finite" cull) */
  const int D = 11 + 3 * (sh_deg + 1) * (sh_deg + 1);
  for (int ch = 0; ch < D; ++ch)
    if (!isfinite(attr[ch * stride])) return;
  const double *Rc = cv, *tc = cv + 9;
  double fx = cv[12], fy = cv[13], cx = cv[14], cy = cv[15];
  for (int i = 0; i < 3; ++i) P->mu[i] = attr[i * stride];
  for (int i = 0; i < 3; ++i) P->s[i] = exp(attr[(3 + i) * stride]);
  for (int i = 0; i < 4; ++i) P->qraw[i] = attr[(6 + i) * stride];
  P->logit = attr[10 * stride];
  P->qnorm = sqrt(P->qraw[0] * P->qraw[0] + P->qraw[1] * P->qraw[1] + P->qraw[2] * P->qraw[2] +
                  P->qraw[3] * P->qraw[3]);
  for (int i = 0; i < 4; ++i) P->qn[i] = P->qraw[i] / P->qnorm;
  or_quat_rot(P->qn, P->R);
  /* Sigma3D = R diag(s^2) R^T */
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += P->R[3 * a + k] * P->s[k] * P->s[k] * P->R[3 * b + k];
      P->S3[3 * a + b] = acc;
    }
  /* camera-space mean */
  for (int a = 0; a < 3; ++a)
    P->X[a] = Rc[3 * a] * P->mu[0] + Rc[3 * a + 1] * P->mu[1] + Rc[3 * a + 2] * P->mu[2] + tc[a];
  double x = P->X[0], y = P->X[1], z = P->X[2];
  if (near_rel(z, znear, 1e-5)) P->flags |= F_CULL_NEAR;
  if (!(z > znear)) return;
  /* EWA Jacobian of (fx x/z + cx, fy y/z + cy) */
  P->J[0] = fx / z; P->J[1] = 0;       P->J[2] = -fx * x / (z * z);
  P->J[3] = 0;      P->J[4] = fy / z;  P->J[5] = -fy * y / (z * z);
  /* T = J Rc (2x3) */
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b)
      P->T[3 * a + b] = P->J[3 * a] * Rc[b] + P->J[3 * a + 1] * Rc[3 + b] + P->J[3 * a + 2] * Rc[6 + b];
  /* Sigma2D = T Sigma3D T^T + 0.3 I */
  double S2[4];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double acc = 0;
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) acc += P->T[3 * a + i] * P->S3[3 * i + k] * P->T[3 * b + k];
      S2[2 * a + b] = acc;
    }
  P->A = S2[0] + LOWPASS;
  P->B = 0.5 * (S2[1] + S2[2]);
  P->C = S2[3] + LOWPASS;
  P->det = P->A * P->C - P->B * P->B;
  if (near_rel(P->det, DET_MIN, 1e-5)) P->flags |= F_CULL_NEAR;
  if (!(P->det > DET_MIN)) return;
  P->conic[0] = P->C / P->det;
  P->conic[1] = -P->B / P->det;
  P->conic[2] = P->A / P->det;
  P->m[0] = fx * x / z + cx;
  P->m[1] = fy * y / z + cy;
  double tr = P->A + P->C;
  P->lam = 0.5 * (tr + sqrt(fmax(0.0, tr * tr - 4.0 * P->det)));
  P->radius = ceil(3.0 * sqrt(P->lam));
  P->o = 1.0 / (1.0 + exp(-P->logit));
  /* colour from SH along the viewing direction */
  double cp[3];
  for (int a = 0; a < 3; ++a) cp[a] = -(Rc[a] * tc[0] + Rc[3 + a] * tc[1] + Rc[6 + a] * tc[2]);
  for (int a = 0; a < 3; ++a) P->u[a] = P->mu[a] - cp[a];
  P->unorm = sqrt(P->u[0] * P->u[0] + P->u[1] * P->u[1] + P->u[2] * P->u[2]);
  for (int a = 0; a < 3; ++a) P->dir[a] = P->u[a] / P->unorm;
  P->nb = (sh_deg + 1) * (sh_deg + 1);
  or_sh_basis(sh_deg, P->dir, P->Y, P->dY);
  for (int c = 0; c < 3; ++c) {
    double acc = 0;
    for (int j = 0; j < P->nb; ++j) acc += attr[(11 + 3 * j + c) * stride] * P->Y[j];
    P->vpre[c] = acc + 0.5;
    P->rgb[c] = P->vpre[c] > 0 ? P->vpre[c] : 0.0;
    if (fabs(P->vpre[c]) <= 1e-6) P->flags |= F_CLAMP_NEAR;
  }
  int finite = isfinite(P->m[0]) && isfinite(P->m[1]) && isfinite(P->conic[0]) &&
               isfinite(P->conic[1]) && isfinite(P->conic[2]) && isfinite(P->o) &&
               isfinite(P->rgb[0]) && isfinite(P->rgb[1]) && isfinite(P->rgb[2]) &&
               isfinite(P->radius);
  P->valid = finite;
}

/*
 * Per (view, Gaussian) records, rec[(v*N + g)*12 + field]; view v renders
 * Gaussians f*N .. f*N+N-1 of its frame f.  A culled pair has radius 0.
 */
void or_project(const double *soa, int64_t G, int64_t N, int D, int sh_deg,
                const double *views, int V, double znear, double *rec) {
  (void)D;
  for (int v = 0; v < V; ++v) {
    const double *cv = views + (int64_t)v * OR_VS;
    int64_t f = (int64_t)cv[18];
    for (int64_t g = 0; g < N; ++g) {
      proj_t P;
      project_one(soa + f * N + g, G, sh_deg, cv, znear, &P);
      double *r = rec + ((int64_t)v * N + g) * OR_REC;
      memset(r, 0, sizeof(double) * OR_REC);
      r[R_FLAGS] = P.flags;
      if (!P.valid) continue;
      r[R_MX] = P.m[0]; r[R_MY] = P.m[1];
      r[R_CA] = P.conic[0]; r[R_CB] = P.conic[1]; r[R_CC] = P.conic[2];
      r[R_OP] = P.o; r[R_Z] = P.X[2]; r[R_RAD] = P.radius;
      r[R_RED] = P.rgb[0]; r[R_GRN] = P.rgb[1]; r[R_BLU] = P.rgb[2];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Binning and depth sort (FP32 integer stage)                               */
/* ------------------------------------------------------------------------ */

/* Tile rectangle of one splat, evaluated in FP32 in exactly this order. */
static int bin_rect32(float mx, float my, float r, int W, int H, int T, int *t) {
  if (!(r > 0.0f)) return 0;
  if (!isfinite(mx) || !isfinite(my)) return 0;
  float ax = mx - 0.5f, ay = my - 0.5f;
  float lox = fmaxf(ceilf(ax - r), 0.0f), hix = fminf(floorf(ax + r), (float)(W - 1));
  float loy = fmaxf(ceilf(ay - r), 0.0f), hiy = fminf(floorf(ay + r), (float)(H - 1));
  if (!(lox <= hix) || !(loy <= hiy)) return 0;
  t[0] = (int)lox / T; t[1] = (int)loy / T; t[2] = (int)hix / T; t[3] = (int)hiy / T;
  return 1;
}

/*
 * Ellipse binning rule: does the footprint q = d^T conic d <= 9 (times
 * 1 + 2^-12, so FP32 per-pixel tests can never accept a pixel outside it)
 * reach the rectangle [x0, x1] x [y0, y1] of a tile's pixel centres?  The
 * minimum of the convex q over the rectangle is 0 if the mean is inside;
 * else it lies on an edge that faces the mean (x = x0 if m_x < x0, x = x1
 * if m_x > x1, likewise in y): a segment from any point of the rectangle
 * towards the mean lowers q and leaves the rectangle through such an edge.
 * On x = const the minimiser is dy = -(b dx)/c clamped to the edge,
 * likewise on y = const.  FP32, in exactly this order, no FMA.
 */
static int ellipse_hits_rect32(float mx, float my, float a, float b, float c, float x0, float x1, float y0,
                               float y1) {
  const float qmax = 9.0f * (1.0f + 1.0f / 4096.0f);
  if (!(a > 0.0f) || !(c > 0.0f)) return 1;
  const int inx = mx >= x0 && mx <= x1, iny = my >= y0 && my <= y1;
  if (inx && iny) return 1;
  const float ra = 1.0f / a, rc = 1.0f / c, b2 = b + b;
  const float lx = x0 - mx, hx = x1 - mx, ly = y0 - my, hy = y1 - my;
  float best = INFINITY;
  if (!inx) {
    float dx = mx < x0 ? lx : hx;
    float t = b * dx;
    t = t * rc;
    float dy = fminf(fmaxf(-t, ly), hy);
    float q = (a * dx) * dx;
    q = q + (b2 * dx) * dy;
    q = q + (c * dy) * dy;
    best = fminf(best, q);
  }
  if (!iny) {
    float dy = my < y0 ? ly : hy;
    float t = b * dy;
    t = t * ra;
    float dx = fminf(fmaxf(-t, lx), hx);
    float q = (a * dx) * dx;
    q = q + (b2 * dx) * dy;
    q = q + (c * dy) * dy;
    best = fminf(best, q);
  }
  return best <= qmax;
}

typedef struct {
  uint64_t key, idx;
  uint32_t val;
} entry_t;

static int cmp_entry(const void *pa, const void *pb) {
  const entry_t *a = (const entry_t *)pa, *b = (const entry_t *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
  return 0;
}

static uint32_t f32_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

int64_t or_tiles_total(int V, const int32_t *vw, const int32_t *vh, int T, int64_t *toff) {
  int64_t t = 0;
  for (int v = 0; v < V; ++v) {
    if (toff) toff[v] = t;
    t += (int64_t)((vw[v] + T - 1) / T) * ((vh[v] + T - 1) / T);
  }
  return t;
}

/* Does tile (tx, ty) of a W x H view receive the splat?  mode 0: every
   tile of the rectangle does; mode 1: only tiles the ellipse reaches. */
static int tile_receives(int mode, const float *ca, const float *cb, const float *cc, int64_t p, float mx,
                         float my, int tx, int ty, int W, int H, int T) {
  if (mode == 0) return 1;
  const float x0 = (float)(tx * T) + 0.5f, y0 = (float)(ty * T) + 0.5f;
  const float x1 = (float)((tx + 1) * T < W ? (tx + 1) * T : W) - 0.5f;
  const float y1 = (float)((ty + 1) * T < H ? (ty + 1) * T : H) - 0.5f;
  return ellipse_hits_rect32(mx, my, ca[p], cb[p], cc[p], x0, x1, y0, y1);
}

/*
 * Emit one (key, value) per receiving tile of the splat's rectangle, in
 * order view, Gaussian, tile row-major; key = (global tile id << 32) |
 * bits(z), value = v*N + g; sort ascending by (key, emission index).
 * ranges[2t], ranges[2t+1] = [start, end) of tile t.  mode 0 = every tile
 * of the rectangle, 1 = tiles the 3-sigma ellipse reaches (ca, cb, cc are
 * the conic entries; unused in mode 0).  Returns the number of entries, or
 * -1 if above cap; with vals == NULL only counts them.
 */
int64_t or_bin_sort(const float *mx, const float *my, const float *rad, const float *z, const float *ca,
                    const float *cb, const float *cc, int mode, int V, int64_t N, const int32_t *vw,
                    const int32_t *vh, int T, uint32_t *vals, int64_t cap, uint32_t *ranges) {
  int64_t *toff = (int64_t *)malloc(sizeof(int64_t) * (V + 1));
  int64_t ntiles = or_tiles_total(V, vw, vh, T, toff);
  int64_t n = 0;
  for (int v = 0; v < V; ++v)
    for (int64_t g = 0; g < N; ++g) {
      int64_t p = (int64_t)v * N + g;
      int t[4];
      if (!bin_rect32(mx[p], my[p], rad[p], vw[v], vh[v], T, t)) continue;
      for (int ty = t[1]; ty <= t[3]; ++ty)
        for (int tx = t[0]; tx <= t[2]; ++tx)
          n += tile_receives(mode, ca, cb, cc, p, mx[p], my[p], tx, ty, vw[v], vh[v], T);
    }
  memset(ranges, 0, sizeof(uint32_t) * 2 * ntiles);
  if (!vals || n > cap) { /* count only, or not enough room */
    free(toff);
    return vals ? -1 : n;
  }
  entry_t *e = (entry_t *)malloc(sizeof(entry_t) * (n > 0 ? n : 1));
  int64_t k = 0;
  for (int v = 0; v < V; ++v) {
    int tx_n = (vw[v] + T - 1) / T;
    for (int64_t g = 0; g < N; ++g) {
      int64_t p = (int64_t)v * N + g;
      int t[4];
      if (!bin_rect32(mx[p], my[p], rad[p], vw[v], vh[v], T, t)) continue;
      for (int ty = t[1]; ty <= t[3]; ++ty)
        for (int tx = t[0]; tx <= t[2]; ++tx) {
          if (!tile_receives(mode, ca, cb, cc, p, mx[p], my[p], tx, ty, vw[v], vh[v], T)) continue;
          uint64_t tile = (uint64_t)(toff[v] + (int64_t)ty * tx_n + tx);
          e[k].key = (tile << 32) | f32_bits(z[p]);
          e[k].idx = (uint64_t)k;
          e[k].val = (uint32_t)p;
          ++k;
        }
    }
  }
  qsort(e, (size_t)n, sizeof(entry_t), cmp_entry);
  for (int64_t i = 0; i < n; ++i) {
    vals[i] = e[i].val;
    uint64_t tile = e[i].key >> 32;
    if (i == 0 || (e[i - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)i;
    ranges[2 * tile + 1] = (uint32_t)(i + 1);
  }
  free(e);
  free(toff);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Compositing                                                              */
/* ------------------------------------------------------------------------ */

static uint64_t fnv(uint64_t h, uint64_t x) {
  for (int i = 0; i < 8; ++i) {
    h ^= (x >> (8 * i)) & 0xffu;
    h *= 1099511628211ull;
  }
  return h;
}

typedef struct {
  uint32_t p;      /* record index */
  int64_t pos;     /* position in the tile list */
  double T, alpha, G, dx, dy;
  int clamped;
} contrib_t;

/*
 * Tolerances of the borderline rule.  A decision of the compositing (q vs 9,
 * alpha vs 1/255, T' vs 1e-4, the depth order of two contributors, a cull)
 * is borderline when an FP32 evaluation of the same step could take the
 * other side:
 *   - q is off by at most dq = |grad_m q| m_tol + (q_rel + cond_rel cond)
 *     (|a| dx^2 + 2 |b dx dy| + |c| dy^2), m_tol bounding the error of the
 *     projected mean (per record in mtol[], else m_fixed), q_rel the
 *     rounding of the quadratic form, cond = (|a c| + b^2) / (a c - b^2)
 *     the condition of the conic (its error grows with it);
 *   - ln alpha is off by dq / 2 + 1e-5 (alpha's own rounding);
 *   - T' relative 1e-4, and any decision after a flip whose change of T
 *     could move the stop;
 *   - two contributors' depths closer than ztol[] of both plus one FP32 ulp
 *     (else 4 FP32 ulps).
 * mtol / ztol are NULL when both sides composite identical FP32 records.
 */
typedef struct {
  const double *mtol, *ztol;
  double m_fixed, q_rel, cond_rel, bg_max;
} tol_t;

static const double U32 = 5.9604644775390625e-08;   /* 2^-24, FP32 unit roundoff */

/*
 * Front-to-back compositing of one pixel over list positions [s, e).
 * Records contributors in c (if non-NULL, capacity e - s); returns their
 * count and sets *Tout, rgb, *last (1-based list position of the last
 * blended entry, 0 if none), *flags (borderline bits), *hash.
 * bnd (if non-NULL) receives the pixel's flip bound: bnd[0] bounds the
 * change of any colour channel, bnd[1] that of T_final, if every
 * borderline decision went the other way.  A flipped splat k changes the
 * colour by T_k a_k (c_k - B / (1 - a_k)), B the colour behind, so by at
 * most T_k a_k cmax (cmax: the largest colour of the tile's list or the
 * background); a swap of two adjacent contributors by T a_1 a_2 cmax; a
 * flipped stop by T cmax.  A flip changes T behind it by a factor (1 -
 * a_k)^(+-1), and a stop that such a change could move is a flip too.
 */
static int composite_pixel(const double *rec, const uint32_t *vals, int64_t s, int64_t e,
                           double px, double py, const tol_t *tol, double *rgb, double *Tout,
                           int64_t *last, uint32_t *flags, uint64_t *hash, contrib_t *c,
                           double *bnd) {
  double T = 1.0;
  int n = 0;
  uint32_t prev_zb = 0;
  double prev_z = 0.0, prev_m[2] = {0.0, 0.0}, prev_T = 0.0, prev_a = 0.0, prev_zt = 0.0;
  int have_prev = 0;
  double cmax = tol->bg_max, bI = 0.0, bT = 0.0;
  double rho = 1.0;   /* T of the other side lies within [T rho^-1, T rho] */
  if (bnd)
    for (int64_t k = s; k < e; ++k) {
      const double *r = rec + (int64_t)vals[k] * OR_REC;
      for (int ch = 0; ch < 3; ++ch)
        if (r[R_RED + ch] > cmax) cmax = r[R_RED + ch];
    }
  rgb[0] = rgb[1] = rgb[2] = 0.0;
  *last = 0;
  for (int64_t k = s; k < e; ++k) {
    const double *r = rec + (int64_t)vals[k] * OR_REC;
    double dx = px - r[R_MX], dy = py - r[R_MY];
    double q = r[R_CA] * dx * dx + 2.0 * r[R_CB] * dx * dy + r[R_CC] * dy * dy;
    /* error bound of q: an m_tol shift of the mean (|grad_m q| m_tol) plus
       the rounding of the form and of the conic */
    double gq = 2.0 * sqrt((r[R_CA] * dx + r[R_CB] * dy) * (r[R_CA] * dx + r[R_CB] * dy) +
                           (r[R_CB] * dx + r[R_CC] * dy) * (r[R_CB] * dx + r[R_CC] * dy));
    double sabs = fabs(r[R_CA]) * dx * dx + 2.0 * fabs(r[R_CB] * dx * dy) + fabs(r[R_CC]) * dy * dy;
    double detc = r[R_CA] * r[R_CC] - r[R_CB] * r[R_CB];
    double cond = detc > 0 ? (fabs(r[R_CA] * r[R_CC]) + r[R_CB] * r[R_CB]) / detc : 1e30;
    double mt = tol->mtol ? tol->mtol[vals[k]] : tol->m_fixed;
    double dq = gq * mt + (tol->q_rel + tol->cond_rel * cond) * sabs;
    int nearq = fabs(q - Q_MAX) <= dq;
    double araw = r[R_OP] * exp(-0.5 * q);
    int neara = araw > 0 && fabs(log(araw) - log(ALPHA_MIN)) <= 0.5 * dq + 1e-5;
    if (nearq) *flags |= B_Q;
    if (neara) *flags |= B_ALPHA;
    /* the other side may blend a splat skipped here, or skip one blended
       here: possible when each test either passes or is borderline */
    if ((nearq || neara) && (q <= Q_MAX || nearq) && (araw >= ALPHA_MIN || neara)) {
      double af = araw > ALPHA_MAX ? ALPHA_MAX : (araw < ALPHA_MIN ? ALPHA_MIN : araw);
      bI += T * rho * af * cmax;
      bT += T * rho * af;
      rho /= (1.0 - af);
    }
    if (q > Q_MAX) {
      *hash = fnv(*hash, ((uint64_t)k << 2) | 0);
      continue;
    }
    double Gv = exp(-0.5 * q);
    double alpha = araw > ALPHA_MAX ? ALPHA_MAX : araw;
    if (alpha < ALPHA_MIN) {
      *hash = fnv(*hash, ((uint64_t)k << 2) | 1);
      continue;
    }
    double Tn = T * (1.0 - alpha);
    /* an FP32 depth order can differ from this one between two depths
       closer than their FP32 errors -- exact FP64 ties included, since FP32
       rounding can split them -- unless the two splats sit at the same
       place (same depth and mean), which every precision computes alike.
       Tested before the stop: swapping the pair can move the stop into it
       (this splat first could already end the pixel, or ends it here). */
    uint32_t zb = f32_bits((float)r[R_Z]);
    double zt = tol->ztol ? tol->ztol[vals[k]] : 0.0;
    int zclose = tol->ztol ? fabs(r[R_Z] - prev_z) <= zt + prev_zt + 2.0 * U32 * fabs(r[R_Z])
                           : (zb - prev_zb) <= 4u;
    if (have_prev && zclose && !(r[R_Z] == prev_z && r[R_MX] == prev_m[0] && r[R_MY] == prev_m[1])) {
      *flags |= B_DEPTH;
      double lim = T_MIN * (1.0 + 1e-4) * rho;
      int stop_moves = Tn < lim || prev_T * (1.0 - alpha) < lim;
      bI += prev_T * rho * (stop_moves ? 1.0 : prev_a * alpha) * cmax;
      if (stop_moves) bT += prev_T * rho;
    }
    /* a stop the other side could take differently: near the cutoff, or
       within the spread of T that earlier flips allow */
    if (near_rel(Tn, T_MIN, 1e-4) || (Tn * rho >= T_MIN && Tn / rho < T_MIN)) {
      *flags |= B_STOP;
      bI += T * rho * cmax;
      bT += T * rho;
    }
    if (Tn < T_MIN) {
      *hash = fnv(*hash, ((uint64_t)k << 2) | 3);
      break;
    }
    if (((uint32_t)r[R_FLAGS]) & F_CULL_NEAR) {
      *flags |= B_CULL;
      bI += T * rho * alpha * cmax;
      bT += T * rho * alpha;
      rho /= (1.0 - alpha);
    }
    if (fabs(araw - ALPHA_MAX) <= 1e-4) *flags |= B_CLAMP;
    prev_zb = zb;
    prev_z = r[R_Z];
    prev_zt = zt;
    prev_m[0] = r[R_MX];
    prev_m[1] = r[R_MY];
    prev_T = T;
    prev_a = alpha;
    have_prev = 1;
    rgb[0] += T * alpha * r[R_RED];
    rgb[1] += T * alpha * r[R_GRN];
    rgb[2] += T * alpha * r[R_BLU];
    if (c) {
      c[n].p = vals[k]; c[n].pos = k; c[n].T = T; c[n].alpha = alpha; c[n].G = Gv;
      c[n].dx = dx; c[n].dy = dy; c[n].clamped = araw > ALPHA_MAX;
    }
    ++n;
    T = Tn;
    *last = k - s + 1;
    *hash = fnv(*hash, ((uint64_t)k << 2) | 2);
  }
  *Tout = T;
  if (bnd) {
    bnd[0] = bI;
    bnd[1] = bT;
  }
  return n;
}

/*
 * Bounds on the FP32 error of each record's projected mean and depth, as
 * the library computes them from FP32 texels and an FP32 camera: X = R mu +
 * t (four roundings over terms of size at most sqrt(3) |mu| + |t_i|), then
 * m = fx X_x / X_z + cx (three roundings and the final add), to first
 * order: dm = fx (dX_x + |x/z| dX_z) / z + 3u fx |x/z| + u |m|, and alike
 * in y; dz = dX_z.  |mu| = |X - t| since R is a rotation.  Culled records
 * get 0.
 */
static void mean_error_bounds(const double *rec, int V, int64_t N, const double *views, double *mtol,
                              double *ztol) {
  for (int v = 0; v < V; ++v) {
    const double *cv = views + (int64_t)v * OR_VS;
    const double *tc = cv + 9;
    double fx = cv[12], fy = cv[13], cx = cv[14], cy = cv[15];
    for (int64_t g = 0; g < N; ++g) {
      int64_t p = (int64_t)v * N + g;
      const double *r = rec + p * OR_REC;
      mtol[p] = ztol[p] = 0.0;
      if (!(r[R_RAD] > 0)) continue;
      double z = r[R_Z], xz = (r[R_MX] - cx) / fx, yz = (r[R_MY] - cy) / fy;
      double X[3] = {xz * z, yz * z, z};
      double mu = sqrt((X[0] - tc[0]) * (X[0] - tc[0]) + (X[1] - tc[1]) * (X[1] - tc[1]) +
                       (X[2] - tc[2]) * (X[2] - tc[2]));
      double dX[3];
      for (int a = 0; a < 3; ++a) dX[a] = 4.0 * U32 * (sqrt(3.0) * mu + fabs(tc[a]));
      double dmx = fx * (dX[0] + fabs(xz) * dX[2]) / z + 3.0 * U32 * fx * fabs(xz) + U32 * fabs(r[R_MX]);
      double dmy = fy * (dX[1] + fabs(yz) * dX[2]) / z + 3.0 * U32 * fy * fabs(yz) + U32 * fabs(r[R_MY]);
      mtol[p] = dmx > dmy ? dmx : dmy;
      ztol[p] = dX[2];
    }
  }
}

void or_mean_error_bounds(const double *rec, int V, int64_t N, const double *views, double *mtol,
                          double *ztol) {
  mean_error_bounds(rec, V, N, views, mtol, ztol);
}

/* The rule's tolerances: m_tol < 0 derives the per-record bounds above
   (records of the oracle's own FP64 projection), m_tol >= 0 is a fixed
   mean tolerance in pixels (0: identical FP32 records on both sides). */
static void make_tol(tol_t *tol, const double *rec, int V, int64_t N, const double *views, double m_tol,
                     double q_rel, const double *bg, double **mt, double **zt) {
  memset(tol, 0, sizeof(*tol));
  *mt = *zt = NULL;
  tol->q_rel = q_rel;
  for (int c = 0; c < 3; ++c)
    if (bg && bg[c] > tol->bg_max) tol->bg_max = bg[c];
  if (m_tol < 0) {
    *mt = (double *)malloc(sizeof(double) * (size_t)(V * N > 0 ? V * N : 1));
    *zt = (double *)malloc(sizeof(double) * (size_t)(V * N > 0 ? V * N : 1));
    mean_error_bounds(rec, V, N, views, *mt, *zt);
    tol->mtol = *mt;
    tol->ztol = *zt;
    tol->cond_rel = 8.0 * U32;
  } else {
    tol->m_fixed = m_tol;
  }
}

static void view_offsets(const double *views, int V, int T, int64_t *poff, int64_t *toff) {
  int64_t p = 0, t = 0;
  for (int v = 0; v < V; ++v) {
    int W = (int)views[(int64_t)v * OR_VS + 16], H = (int)views[(int64_t)v * OR_VS + 17];
    poff[v] = p;
    toff[v] = t;
    p += (int64_t)W * H;
    t += (int64_t)((W + T - 1) / T) * ((H + T - 1) / T);
  }
  poff[V] = p;
  toff[V] = t;
}

/*
 * Render all views.  img is planar per view, [V][3][H][W] concatenated;
 * Tfin, last and border are [V][H][W] concatenated.  Returns a hash of
 * every per-pixel decision (used to reject finite-difference samples whose
 * discrete decisions changed).
 */
uint64_t or_render(const double *rec, int V, int64_t N, const double *views, int T,
                   const uint32_t *vals, const uint32_t *ranges, const double *bg, double m_tol,
                   double q_rel, double *img, double *Tfin, uint32_t *last, uint8_t *border,
                   double *bnd) {
  tol_t tol;
  double *mt, *zt;
  make_tol(&tol, rec, V, N, views, m_tol, q_rel, bg, &mt, &zt);
  int64_t *poff = (int64_t *)malloc(sizeof(int64_t) * (V + 1));
  int64_t *toff = (int64_t *)malloc(sizeof(int64_t) * (V + 1));
  view_offsets(views, V, T, poff, toff);
  uint64_t hash = 1469598103934665603ull;
  for (int v = 0; v < V; ++v) {
    int W = (int)views[(int64_t)v * OR_VS + 16], H = (int)views[(int64_t)v * OR_VS + 17];
    int tx_n = (W + T - 1) / T;
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int64_t tile = toff[v] + (int64_t)(y / T) * tx_n + x / T;
        int64_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
        double rgb[3], Tv;
        int64_t lst;
        uint32_t fl = 0;
        hash = fnv(hash, (uint64_t)(poff[v] + (int64_t)y * W + x));
        int64_t pix = poff[v] + (int64_t)y * W + x;
        composite_pixel(rec, vals, s, e, x + 0.5, y + 0.5, &tol, rgb, &Tv, &lst, &fl, &hash, NULL,
                        bnd ? bnd + 2 * pix : NULL);
        for (int c = 0; c < 3; ++c)
          img[3 * poff[v] + (int64_t)c * W * H + (int64_t)y * W + x] = rgb[c] + Tv * bg[c];
        Tfin[pix] = Tv;
        last[pix] = (uint32_t)lst;
        border[pix] = (uint8_t)fl;
      }
  }
  free(poff);
  free(toff);
  free(mt);
  free(zt);
  return hash;
}

/*
 * Reverse-mode adjoint of or_render for dL/dimage dimg (same layout as img).
 * grad2d[(v*N+g)*9 + i] accumulates dL/d(m_x, m_y, conic_a, conic_b,
 * conic_c, opacity, red, green, blue) of each projected splat.  conic_b is
 * the off-diagonal entry (it appears twice in d^T conic d).
 */
void or_render_bwd(const double *rec, int V, int64_t N, const double *views, int T,
                   const uint32_t *vals, const uint32_t *ranges, const double *bg,
                   const double *dimg, double *grad2d) {
  int64_t *poff = (int64_t *)malloc(sizeof(int64_t) * (V + 1));
  int64_t *toff = (int64_t *)malloc(sizeof(int64_t) * (V + 1));
  view_offsets(views, V, T, poff, toff);
  memset(grad2d, 0, sizeof(double) * OR_G2D * (size_t)V * (size_t)N);
  int64_t maxlist = 1;
  for (int64_t t = 0; t < toff[V]; ++t)
    if ((int64_t)ranges[2 * t + 1] - ranges[2 * t] > maxlist) maxlist = ranges[2 * t + 1] - ranges[2 * t];
  contrib_t *cb = (contrib_t *)malloc(sizeof(contrib_t) * maxlist);
  tol_t tol0;
  memset(&tol0, 0, sizeof(tol0));
  for (int v = 0; v < V; ++v) {
    int W = (int)views[(int64_t)v * OR_VS + 16], H = (int)views[(int64_t)v * OR_VS + 17];
    int tx_n = (W + T - 1) / T;
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int64_t tile = toff[v] + (int64_t)(y / T) * tx_n + x / T;
        int64_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
        double rgb[3], Tf;
        int64_t lst;
        uint32_t fl = 0;
        uint64_t h = 0;
        int n = composite_pixel(rec, vals, s, e, x + 0.5, y + 0.5, &tol0, rgb, &Tf, &lst, &fl, &h, cb, NULL);
        double gC[3];
        for (int c = 0; c < 3; ++c) gC[c] = dimg[3 * poff[v] + (int64_t)c * W * H + (int64_t)y * W + x];
        /* S = colour composited behind contributor i (incl. background) */
        double S[3] = {Tf * bg[0], Tf * bg[1], Tf * bg[2]};
        for (int i = n - 1; i >= 0; --i) {
          const contrib_t *ci = &cb[i];
          const double *r = rec + (int64_t)ci->p * OR_REC;
          double col[3] = {r[R_RED], r[R_GRN], r[R_BLU]};
          double *g2 = grad2d + (int64_t)ci->p * OR_G2D;
          double dalpha = 0;
          for (int c = 0; c < 3; ++c) {
            g2[6 + c] += ci->T * ci->alpha * gC[c];
            dalpha += gC[c] * (ci->T * col[c] - S[c] / (1.0 - ci->alpha));
          }
          for (int c = 0; c < 3; ++c) S[c] += ci->T * ci->alpha * col[c];
          if (ci->clamped) continue;           /* alpha = 0.99 is constant */
          /* alpha = o exp(-q/2) */
          g2[5] += dalpha * ci->G;
          double dq = -0.5 * ci->alpha * dalpha;
          double dx = ci->dx, dy = ci->dy;
          g2[2] += dq * dx * dx;
          g2[3] += dq * 2.0 * dx * dy;
          g2[4] += dq * dy * dy;
          /* d = p - m, dq/dm = -2 conic d */
          g2[0] += -dq * 2.0 * (r[R_CA] * dx + r[R_CB] * dy);
          g2[1] += -dq * 2.0 * (r[R_CB] * dx + r[R_CC] * dy);
        }
      }
  }
  free(cb);
  free(poff);
  free(toff);
}

/*
 * Chain the per-view 2D gradients back to the Gaussian attributes, sum over
 * the views of each Gaussian's frame and apply the freeze mask D_i
 * (dynflag, NULL = all dynamic).  out[c*G + gi], G = F*N, zeroed first.
 */
void or_scatter_grad(const double *soa, int64_t G, int64_t N, int D, int sh_deg,
                     const double *views, int V, double znear, const double *grad2d,
                     const uint8_t *dynflag, double *out) {
  memset(out, 0, sizeof(double) * (size_t)D * (size_t)G);
  for (int v = 0; v < V; ++v) {
    const double *cv = views + (int64_t)v * OR_VS;
    const double *Rc = cv;
    double fx = cv[12], fy = cv[13];
    int64_t f = (int64_t)cv[18];
    for (int64_t g = 0; g < N; ++g) {
      int64_t gi = f * N + g;
      if (dynflag && !dynflag[g]) continue;
      const double *g2 = grad2d + ((int64_t)v * N + g) * OR_G2D;
      proj_t P;
      project_one(soa + gi, G, sh_deg, cv, znear, &P);
      if (!P.valid) continue;
      double dmu[3] = {0, 0, 0};
      /* opacity */
      out[10 * G + gi] += g2[5] * P.o * (1.0 - P.o);
      /* colour: rgb = max(0, sum_j k_j Y_j(dir) + 0.5) */
      double ddir[3] = {0, 0, 0};
      for (int c = 0; c < 3; ++c) {
        if (P.vpre[c] < 0) continue;
        double gc = g2[6 + c];
        for (int j = 0; j < P.nb; ++j) {
          out[(int64_t)(11 + 3 * j + c) * G + gi] += gc * P.Y[j];
          double k = soa[(int64_t)(11 + 3 * j + c) * G + gi];
          for (int a = 0; a < 3; ++a) ddir[a] += gc * k * P.dY[3 * j + a];
        }
      }
      double dd = ddir[0] * P.dir[0] + ddir[1] * P.dir[1] + ddir[2] * P.dir[2];
      for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - P.dir[a] * dd) / P.unorm;
      /* conic = Sigma2D^-1: dL/dSigma = -Q G_Q Q with symmetric G_Q */
      double Q[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
      double GQ[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};
      double tmp[4], GS[4];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) tmp[2 * a + b] = GQ[2 * a] * Q[b] + GQ[2 * a + 1] * Q[2 + b];
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) GS[2 * a + b] = -(Q[2 * a] * tmp[b] + Q[2 * a + 1] * tmp[2 + b]);
      /* Sigma2D = T Sigma3D T^T + 0.3 I */
      double G3[9], dT[6];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double acc = 0;
          for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 2; ++k) acc += P.T[3 * i + a] * GS[2 * i + k] * P.T[3 * k + b];
          G3[3 * a + b] = acc;
        }
      for (int i = 0; i < 2; ++i)
        for (int b = 0; b < 3; ++b) {
          double acc = 0;
          for (int k = 0; k < 2; ++k)
            for (int c = 0; c < 3; ++c) acc += GS[2 * i + k] * P.T[3 * k + c] * P.S3[3 * c + b];
          dT[3 * i + b] = 2.0 * acc;
        }
      /* T = J Rc  ->  dJ = dT Rc^T */
      double dJ[6];
      for (int i = 0; i < 2; ++i)
        for (int a = 0; a < 3; ++a)
          dJ[3 * i + a] = dT[3 * i] * Rc[3 * a] + dT[3 * i + 1] * Rc[3 * a + 1] + dT[3 * i + 2] * Rc[3 * a + 2];
      double x = P.X[0], y = P.X[1], z = P.X[2];
      double dX[3];
      dX[0] = g2[0] * fx / z;
      dX[1] = g2[1] * fy / z;
      dX[2] = -g2[0] * fx * x / (z * z) - g2[1] * fy * y / (z * z);
      dX[2] += dJ[0] * (-fx / (z * z));
      dX[0] += dJ[2] * (-fx / (z * z));
      dX[2] += dJ[2] * (2.0 * fx * x / (z * z * z));
      dX[2] += dJ[4] * (-fy / (z * z));
      dX[1] += dJ[5] * (-fy / (z * z));
      dX[2] += dJ[5] * (2.0 * fy * y / (z * z * z));
      for (int a = 0; a < 3; ++a) dmu[a] += Rc[a] * dX[0] + Rc[3 + a] * dX[1] + Rc[6 + a] * dX[2];
      for (int a = 0; a < 3; ++a) out[(int64_t)a * G + gi] += dmu[a];
      /* Sigma3D = M M^T, M = R diag(s) */
      double M[9], dM[9];
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) M[3 * a + k] = P.R[3 * a + k] * P.s[k];
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) {
          double acc = 0;
          for (int b = 0; b < 3; ++b) acc += G3[3 * a + b] * M[3 * b + k];
          dM[3 * a + k] = 2.0 * acc;
        }
      double dR[9];
      for (int k = 0; k < 3; ++k) {
        double ds = 0;
        for (int a = 0; a < 3; ++a) ds += P.R[3 * a + k] * dM[3 * a + k];
        out[(int64_t)(3 + k) * G + gi] += ds * P.s[k];
      }
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 3; ++k) dR[3 * a + k] = dM[3 * a + k] * P.s[k];
      double jq[9][4], dqn[4] = {0, 0, 0, 0};
      quat_rot_jac(P.qn, jq);
      for (int e = 0; e < 9; ++e)
        for (int i = 0; i < 4; ++i) dqn[i] += dR[e] * jq[e][i];
      double dot = dqn[0] * P.qn[0] + dqn[1] * P.qn[1] + dqn[2] * P.qn[2] + dqn[3] * P.qn[3];
      for (int i = 0; i < 4; ++i) out[(int64_t)(6 + i) * G + gi] += (dqn[i] - P.qn[i] * dot) / P.qnorm;
    }
  }
  (void)D;
}

/*
 * Sampled pixels of a large scene, by brute force over every splat of the
 * pixel's view: candidates are the splats whose FP32 tile rectangle holds
 * the pixel, in (FP32 depth bits, index) order, composited as or_render
 * does.  pix[3*i..] = (view, x, y).  rgb[3*i..] and Tout[i] are written.
 */
void or_render_pixels(const double *rec, int V, int64_t N, const double *views, int T,
                      const double *bg, double m_tol, double q_rel, int64_t npix, const int32_t *pix,
                      double *rgb_out, double *Tout, uint8_t *border, double *bnd) {
  tol_t tol;
  double *mt, *zt;
  make_tol(&tol, rec, V, N, views, m_tol, q_rel, bg, &mt, &zt);
  entry_t *e = (entry_t *)malloc(sizeof(entry_t) * (N > 0 ? N : 1));
  uint32_t *vals = (uint32_t *)malloc(sizeof(uint32_t) * (N > 0 ? N : 1));
  for (int64_t i = 0; i < npix; ++i) {
    int v = pix[3 * i], x = pix[3 * i + 1], y = pix[3 * i + 2];
    int W = (int)views[(int64_t)v * OR_VS + 16], H = (int)views[(int64_t)v * OR_VS + 17];
    int64_t n = 0;
    for (int64_t g = 0; g < N; ++g) {
      int64_t p = (int64_t)v * N + g;
      const double *r = rec + p * OR_REC;
      int t[4];
      if (!bin_rect32((float)r[R_MX], (float)r[R_MY], (float)r[R_RAD], W, H, T, t)) continue;
      if (x / T < t[0] || x / T > t[2] || y / T < t[1] || y / T > t[3]) continue;
      e[n].key = f32_bits((float)r[R_Z]);
      e[n].idx = (uint64_t)g;
      e[n].val = (uint32_t)p;
      ++n;
    }
    qsort(e, (size_t)n, sizeof(entry_t), cmp_entry);
    for (int64_t k = 0; k < n; ++k) vals[k] = e[k].val;
    double rgb[3], Tv;
    int64_t lst;
    uint32_t fl = 0;
    uint64_t h = 0;
    composite_pixel(rec, vals, 0, n, x + 0.5, y + 0.5, &tol, rgb, &Tv, &lst, &fl, &h, NULL,
                    bnd ? bnd + 2 * i : NULL);
    for (int c = 0; c < 3; ++c) rgb_out[3 * i + c] = rgb[c] + Tv * bg[c];
    Tout[i] = Tv;
    border[i] = (uint8_t)fl;
  }
  free(e);
  free(vals);
  free(mt);
  free(zt);
}

/* ------------------------------------------------------------------------ */
/* Motion masks and the covariance-aware dynamic mask                        */
/* ------------------------------------------------------------------------ */

/*
 * Binary motion mask of one view (Sec. 4.2 "Optical Flow and Binary Motion
 * Masks"): a pixel is moving when the magnitude of its flow vector exceeds
 * tau; the mask is then dilated with radius r.  Readings: the magnitude and
 * the comparison are taken in FP32, the flow's own precision, as
 * sqrtf(fx * fx + fy * fy) > tau; the dilation's structuring element is the
 * (2r+1) x (2r+1) square and pixels outside the image count as still.
 * flow: [2][H][W] (x component plane, then y); M: out [H][W], 0 or 1.
 */
void or_motion_mask(const float *flow, int W, int H, float tau, int r, uint8_t *M) {
  const int64_t plane = (int64_t)W * H;
  uint8_t *raw = (uint8_t *)malloc(plane > 0 ? (size_t)plane : 1);
  for (int64_t i = 0; i < plane; ++i) {
    float fx = flow[i], fy = flow[plane + i];
    float mag = sqrtf(fx * fx + fy * fy);
    raw[i] = mag > tau;
  }
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int on = 0;
      for (int dy = -r; dy <= r && !on; ++dy) {
        int yy = y + dy;
        if (yy < 0 || yy >= H) continue;
        for (int dx = -r; dx <= r; ++dx) {
          int xx = x + dx;
          if (xx >= 0 && xx < W && raw[(int64_t)yy * W + xx]) {
            on = 1;
            break;
          }
        }
      }
      M[(int64_t)y * W + x] = (uint8_t)on;
    }
  free(raw);
}

/*
 * Dynamic mask from FP32 projected records (Alg. 1 step 5 and the OR over
 * cameras of Sec. 4.2 "Covariance-Aware Gaussian Masking").  rec: [V*N][12]
 * float records {m_x, m_y, a, b, c, opacity, z, radius, ...} with conic
 * [[a, b], [b, c]] and radius 0 for a culled pair; M: the views' motion
 * masks concatenated, [sum_v H_v W_v] bytes.  D_g = 1 iff in some view v a
 * pixel (x, y) of the square |centre - m|_inf <= r, r = min(r_max, radius)
 * (r_max <= 0: no clamp), lies in the image, has M_v = 1 and
 * d^2 = (p - m)^T conic (p - m) <= 9 at its centre p = (x + 0.5, y + 0.5).
 * Square and d^2 in FP32, in exactly this order, no fused multiply-add:
 *   x_lo = ceil((m_x - 0.5) - r), x_hi = floor((m_x - 0.5) + r) (same in y),
 *   clamped to the image;
 *   d^2 = ((a dx) dx + (c dy) dy) + ((2 b) dy) dx, dx = (x + 0.5) - m_x.
 */
void or_dynamic_mask32(const float *rec, int V, int64_t N, const int32_t *vw, const int32_t *vh,
                       const uint8_t *M, float r_max, uint8_t *D) {
  memset(D, 0, (size_t)(N > 0 ? N : 0));
  int64_t poff = 0;
  for (int v = 0; v < V; ++v) {
    const int W = vw[v], H = vh[v];
    const uint8_t *Mv = M + poff;
    for (int64_t g = 0; g < N; ++g) {
      if (D[g]) continue;
      const float *r = rec + ((int64_t)v * N + g) * OR_REC;
      float rad = r[R_RAD];
      if (!(rad > 0.0f)) continue;
      if (r_max > 0.0f && rad > r_max) rad = r_max;
      float mx = r[R_MX], my = r[R_MY], a = r[R_CA], b = r[R_CB], c = r[R_CC];
      if (!isfinite(mx) || !isfinite(my)) continue;
      float ax = mx - 0.5f, ay = my - 0.5f;
      float lox = fmaxf(ceilf(ax - rad), 0.0f), hix = fminf(floorf(ax + rad), (float)(W - 1));
      float loy = fmaxf(ceilf(ay - rad), 0.0f), hiy = fminf(floorf(ay + rad), (float)(H - 1));
      if (!(lox <= hix) || !(loy <= hiy)) continue;
      const float b2 = 2.0f * b;
      for (int y = (int)loy; y <= (int)hiy && !D[g]; ++y) {
        float dy = ((float)y + 0.5f) - my;
        float cyy = (c * dy) * dy;
        float bdy = b2 * dy;
        for (int x = (int)lox; x <= (int)hix; ++x) {
          if (!Mv[(int64_t)y * W + x]) continue;
          float dx = ((float)x + 0.5f) - mx;
          float q = ((a * dx) * dx + cyy) + bdy * dx;
          if (q <= 9.0f) {
            D[g] = 1;
            break;
          }
        }
      }
    }
    poff += (int64_t)W * H;
  }
}

/*
 * The same mask in FP64 from the oracle's own records (or_project), taking
 * Alg. 1 step 5 literally.  border[g] = 1 when a finite-precision
 * evaluation could decide D_g differently: D_g is an OR, so that needs a
 * shaky pixel -- a masked pixel whose d^2 lies within the error bound of 9
 * (the bound of the compositing rule: a shift of the mean by m_tol pixels,
 * plus relative 1e-5), a masked footprint pixel within 1e-3 px of the
 * clamped square's edge, or any masked footprint pixel of a pair near a
 * culling cutoff -- and no firm hit anywhere else (a masked pixel clear of
 * all three, inside the footprint).
 */
void or_dynamic_mask(const double *rec, int V, int64_t N, const int32_t *vw, const int32_t *vh,
                     const uint8_t *M, double r_max, double m_tol, uint8_t *D, uint8_t *border) {
  uint8_t *firm = (uint8_t *)calloc((size_t)(N > 0 ? N : 1), 1);
  memset(D, 0, (size_t)(N > 0 ? N : 0));
  memset(border, 0, (size_t)(N > 0 ? N : 0));
  int64_t poff = 0;
  for (int v = 0; v < V; ++v) {
    const int W = vw[v], H = vh[v];
    const uint8_t *Mv = M + poff;
    for (int64_t g = 0; g < N; ++g) {
      const double *r = rec + ((int64_t)v * N + g) * OR_REC;
      const int near_cull = (((uint32_t)r[R_FLAGS]) & F_CULL_NEAR) != 0;
      double rad = r[R_RAD];
      if (!(rad > 0.0)) {
        /* culled here, possibly valid in FP32: any masked pixel may count */
        if (near_cull) border[g] = 1;
        continue;
      }
      int clamp = r_max > 0.0 && rad > r_max;
      if (clamp) rad = r_max;
      double mx = r[R_MX], my = r[R_MY], a = r[R_CA], b = r[R_CB], c = r[R_CC];
      /* scan one pixel beyond the square when clamped, for the edge rule */
      double grow = clamp ? 1.0 : 0.0;
      double lox = fmax(ceil(mx - 0.5 - rad - grow), 0.0), hix = fmin(floor(mx - 0.5 + rad + grow), W - 1.0);
      double loy = fmax(ceil(my - 0.5 - rad - grow), 0.0), hiy = fmin(floor(my - 0.5 + rad + grow), H - 1.0);
      for (int y = (int)loy; y <= (int)hiy; ++y)
        for (int x = (int)lox; x <= (int)hix; ++x) {
          if (!Mv[(int64_t)y * W + x]) continue;
          double dx = x + 0.5 - mx, dy = y + 0.5 - my;
          double q = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy;
          double gq = 2.0 * sqrt((a * dx + b * dy) * (a * dx + b * dy) + (b * dx + c * dy) * (b * dx + c * dy));
          double dq = gq * m_tol + 1e-5 * fabs(q) + 1e-6;
          int inside = fabs(dx) <= rad && fabs(dy) <= rad;
          int shaky = fabs(q - Q_MAX) <= dq;
          if (clamp && q <= Q_MAX + dq && (fabs(fabs(dx) - rad) <= 1e-3 || fabs(fabs(dy) - rad) <= 1e-3))
            shaky = 1;
          if (near_cull && q <= Q_MAX + dq) shaky = 1;
          if (shaky) border[g] = 1;
          if (inside && q <= Q_MAX) {
            D[g] = 1;
            if (!shaky) firm[g] = 1;
          }
        }
    }
    poff += (int64_t)W * H;
  }
  for (int64_t g = 0; g < N; ++g)
    if (firm[g]) border[g] = 0;
  free(firm);
}

/* ------------------------------------------------------------------------ */
/* Low-precision proxy (LPO) and the 8-bit plane layout                      */
/* ------------------------------------------------------------------------ */

/*
 * Sec. 4.2 "Low Precision Optimization" and Supp. "Video Coding": every
 * attribute channel is normalised by its min/max over the live texels of
 * all frames and quantised uniformly to K bits with scale
 * Delta = (hi - lo) / (2^K - 1); K = 16 for the three position channels,
 * each kept as two 8-bit planes (high byte, then low byte), and K = 8 for
 * scale, rotation, opacity and colour.  The renderer reads the proxy
 * lo + q Delta.  Readings: q = floor((x - lo) / Delta + 0.5) clamped to
 * [0, 2^K - 1], and q = 0 when that is not a number (hi == lo, or x NaN);
 * min/max skip NaN texels and are 0 when no texel is live; every step in
 * FP32, IEEE-rounded, in exactly this order.  Plane p of a frame holds
 * channel p / 2's high (p even) or low byte for p < 6, channel p - 3
 * otherwise: D + 3 planes per frame, [F][D + 3][H][W] bytes, 0 at texels
 * that are not live.
 */
static int lpo_bits(int c) { return c < 3 ? 16 : 8; }

void or_lpo_minmax(const float *atlas, int F, int D, int H, int W, const uint32_t *occ, float *lohi) {
  const int Wp = (W + 31) / 32;
  for (int c = 0; c < D; ++c) {
    int any = 0;
    float lo = 0.0f, hi = 0.0f;
    for (int f = 0; f < F; ++f)
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
          if (!bit_at(occ, Wp, x, y)) continue;
          float v = atlas[(((int64_t)f * D + c) * H + y) * W + x];
          if (v != v) continue;
          if (!any || v < lo) lo = v;
          if (!any || v > hi) hi = v;
          any = 1;
        }
    lohi[2 * c] = lo;
    lohi[2 * c + 1] = hi;
  }
}

static float lpo_delta(const float *lohi, int c) {
  const float L = (float)((1u << lpo_bits(c)) - 1u);
  return (lohi[2 * c + 1] - lohi[2 * c]) / L;
}

static uint32_t lpo_code(float x, float lo, float delta, int bits) {
  const float L = (float)((1u << bits) - 1u);
  float t = (x - lo) / delta;
  float u = floorf(t + 0.5f);
  if (!(u >= 0.0f)) return 0u;
  if (u >= L) return (uint32_t)L;
  return (uint32_t)u;
}

void or_lpo_encode(const float *atlas, int F, int D, int H, int W, const uint32_t *occ, const float *lohi,
                   uint8_t *codes) {
  const int Wp = (W + 31) / 32, NP = D + 3;
  const int64_t plane = (int64_t)W * H;
  memset(codes, 0, (size_t)((int64_t)F * NP * plane));
  for (int f = 0; f < F; ++f)
    for (int c = 0; c < D; ++c) {
      const float lo = lohi[2 * c], delta = lpo_delta(lohi, c);
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
          if (!bit_at(occ, Wp, x, y)) continue;
          const int64_t px = (int64_t)y * W + x;
          uint32_t q = lpo_code(atlas[((int64_t)f * D + c) * plane + px], lo, delta, lpo_bits(c));
          if (c < 3) {
            codes[((int64_t)f * NP + 2 * c) * plane + px] = (uint8_t)(q >> 8);
            codes[((int64_t)f * NP + 2 * c + 1) * plane + px] = (uint8_t)(q & 255u);
          } else {
            codes[((int64_t)f * NP + c + 3) * plane + px] = (uint8_t)q;
          }
        }
    }
}

/* Codes back to the proxy atlas [F][D][H][W] float32 (0 where not live). */
void or_lpo_decode(const uint8_t *codes, int F, int D, int H, int W, const uint32_t *occ, const float *lohi,
                   float *proxy) {
  const int Wp = (W + 31) / 32, NP = D + 3;
  const int64_t plane = (int64_t)W * H;
  memset(proxy, 0, sizeof(float) * (size_t)((int64_t)F * D * plane));
  for (int f = 0; f < F; ++f)
    for (int c = 0; c < D; ++c) {
      const float lo = lohi[2 * c], delta = lpo_delta(lohi, c);
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
          if (!bit_at(occ, Wp, x, y)) continue;
          const int64_t px = (int64_t)y * W + x;
          uint32_t q;
          if (c < 3)
            q = ((uint32_t)codes[((int64_t)f * NP + 2 * c) * plane + px] << 8) |
                codes[((int64_t)f * NP + 2 * c + 1) * plane + px];
          else
            q = codes[((int64_t)f * NP + c + 3) * plane + px];
          proxy[((int64_t)f * D + c) * plane + px] = lo + (float)q * delta;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* UV cells (eq. uvgs2) and Max-K UV pruning                                */
/* ------------------------------------------------------------------------ */

/*
 * UV cell of a position (Sec. 3 "UV-based Point-to-Image Transformation",
 * eq. uvgs2): rho = |mu|, theta = atan2(y, x), phi = acos(z / rho),
 * u = floor((pi + theta) / (2 pi) M), v = floor(phi / pi N).  The cell is
 * valid (Sec. 4.2 "Valid UV Projection Pruning") iff rho is positive and
 * finite and 0 <= u < M, 0 <= v < N; its id is v M + u (u along the width
 * M, the reading of eq. uvgs2).  *border = 1 when either scaled coordinate
 * lies within 1e-9 (relative to the map size) of an integer, where another
 * precision could pick the neighbouring cell.  Returns the id or
 * 0xFFFFFFFF.
 */
uint32_t or_uv_cell(double x, double y, double z, int M, int N, int *border) {
  double rho = sqrt(x * x + y * y + z * z);
  *border = 0;
  if (!(rho > 0.0) || !isfinite(rho)) return 0xFFFFFFFFu;
  double theta = atan2(y, x), phi = acos(z / rho);
  double su = (M_PI + theta) / (2.0 * M_PI) * M, sv = phi / M_PI * N;
  if (fabs(su - nearbyint(su)) <= 1e-9 * M || fabs(sv - nearbyint(sv)) <= 1e-9 * N) *border = 1;
  double u = floor(su), v = floor(sv);
  if (!(u >= 0.0 && u < M && v >= 0.0 && v < N)) return 0xFFFFFFFFu;
  return (uint32_t)v * (uint32_t)M + (uint32_t)u;
}

typedef struct {
  uint32_t cell;
  double logit;
  int64_t idx;
} uvk_t;

static int cmp_uvk(const void *pa, const void *pb) {
  const uvk_t *a = (const uvk_t *)pa, *b = (const uvk_t *)pb;
  if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
  if (a->logit != b->logit) return a->logit > b->logit ? -1 : 1;   /* higher opacity first */
  return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

/*
 * Max-K UV pruning (Sec. 4.2 "Max-K UV Pruning", UVGS layers ordered by
 * opacity): of the valid Gaussians of each cell, the K of highest opacity
 * are kept; rank = 0-based position in that order (ties: lower index
 * first).  Opacity o = sigmoid(logit) is increasing, so logits are
 * compared; a NaN logit makes a Gaussian invalid.  soa: channel-major
 * [D][stride], Gaussian i in column i (position channels 0..2, logit 10).
 * Outputs per Gaussian: cell (0xFFFFFFFF if invalid), rank (0xFFFFFFFF if
 * invalid), keep; count [M N] = valid Gaussians per cell; border as in
 * or_uv_cell, spread to every Gaussian of a cell that holds one.
 */
void or_uv_max_k(const double *soa, int64_t n, int64_t stride, int M, int N, int K, uint32_t *cell,
                 uint32_t *rank, uint8_t *keep, uint32_t *count, uint8_t *border) {
  uvk_t *e = (uvk_t *)malloc(sizeof(uvk_t) * (size_t)(n > 0 ? n : 1));
  uint8_t *cb = (uint8_t *)calloc((size_t)M * (size_t)N, 1);
  memset(count, 0, sizeof(uint32_t) * (size_t)M * (size_t)N);
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    int b = 0;
    double lg = soa[10 * stride + i];
    uint32_t c = or_uv_cell(soa[i], soa[stride + i], soa[2 * stride + i], M, N, &b);
    if (lg != lg) c = 0xFFFFFFFFu;
    cell[i] = c;
    rank[i] = 0xFFFFFFFFu;
    keep[i] = 0;
    border[i] = (uint8_t)b;
    if (c == 0xFFFFFFFFu) continue;
    if (b) cb[c] = 1;
    e[m].cell = c;
    e[m].logit = lg;
    e[m].idx = i;
    ++m;
  }
  qsort(e, (size_t)m, sizeof(uvk_t), cmp_uvk);
  for (int64_t j = 0; j < m; ++j) {
    uint32_t r = count[e[j].cell]++;
    rank[e[j].idx] = r;
    keep[e[j].idx] = r < (uint32_t)K;
  }
  for (int64_t i = 0; i < n; ++i)
    if (cell[i] != 0xFFFFFFFFu && cb[cell[i]]) border[i] = 1;
  free(e);
  free(cb);
}

/* ------------------------------------------------------------------------ */
/* Photometric objective: L1 + D-SSIM                                        */
/* ------------------------------------------------------------------------ */

#define SSIM_R 5          /* 11 x 11 window */
static const double SSIM_SIGMA = 1.5, SSIM_C1 = 0.0001, SSIM_C2 = 0.0009;

/* 1-D Gaussian weights of standard deviation 1.5 over -5..5, summing to 1;
 * the 2-D window is their outer product. */
static void ssim_weights(double w[2 * SSIM_R + 1]) {
  double s = 0.0;
  for (int k = -SSIM_R; k <= SSIM_R; ++k) s += (w[k + SSIM_R] = exp(-(double)(k * k) / (2.0 * SSIM_SIGMA * SSIM_SIGMA)));
  for (int k = 0; k <= 2 * SSIM_R; ++k) w[k] /= s;
}

/*
 * Photometric objective of Sec. 4.2 "Objective":
 *   L = (1 - lambda) ||I^ - I||_1 + lambda (1 - SSIM(I^, I)).
 * Readings (the paper gives neither constants nor normalisation): the L1
 * term is the mean of |I^ - I| over the 3 P values; SSIM is the mean over
 * the 3 P values of the per-channel SSIM map of Wang et al. with the 11 x 11
 * Gaussian window (standard deviation 1.5, weights summing to 1), pixels
 * outside the image counting as 0 in every window sum, C1 = 0.01^2 and
 * C2 = 0.03^2 (the 3DGS convention); lambda = 0.2 by default.  Per pixel
 * with window sums m1 = G*X, m2 = G*Y, e11 = G*(X X), e22 = G*(Y Y),
 * e12 = G*(X Y):
 *   s = (2 m1 m2 + C1)(2 (e12 - m1 m2) + C2) /
 *       ((m1^2 + m2^2 + C1)((e11 - m1^2) + (e22 - m2^2) + C2)).
 * img, tgt: [3P] planar per view as the images of the render step.
 * grad: out dL/dimg [3P] (or NULL) -- the L1 part is sign(X - Y) / (3P),
 * 0 where equal; the SSIM part is the adjoint of every window sum.
 * ssim_map: out [3P] (or NULL).  Returns L; *ssim = mean SSIM.
 */
double or_photo_loss(const double *img, const double *tgt, int V, const int32_t *vw, const int32_t *vh,
                     double lambda, double *grad, double *ssim_map, double *ssim) {
  double w[2 * SSIM_R + 1];
  ssim_weights(w);
  int64_t P = 0;
  for (int v = 0; v < V; ++v) P += (int64_t)vw[v] * vh[v];
  const double n = 3.0 * (double)P;
  double l1 = 0.0, ssum = 0.0;
  int64_t off = 0;
  for (int v = 0; v < V; ++v) {
    const int W = vw[v], H = vh[v];
    const int64_t plane = (int64_t)W * H;
    double *ds1 = (double *)malloc(sizeof(double) * (size_t)plane);
    double *ds11 = (double *)malloc(sizeof(double) * (size_t)plane);
    double *ds12 = (double *)malloc(sizeof(double) * (size_t)plane);
    for (int c = 0; c < 3; ++c) {
      const double *X = img + 3 * off + c * plane, *Y = tgt + 3 * off + c * plane;
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
          double m1 = 0, m2 = 0, e11 = 0, e22 = 0, e12 = 0;
          for (int i = -SSIM_R; i <= SSIM_R; ++i)
            for (int j = -SSIM_R; j <= SSIM_R; ++j) {
              int yy = y + i, xx = x + j;
              if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
              double g = w[i + SSIM_R] * w[j + SSIM_R], a = X[(int64_t)yy * W + xx], b = Y[(int64_t)yy * W + xx];
              m1 += g * a;
              m2 += g * b;
              e11 += g * a * a;
              e22 += g * b * b;
              e12 += g * a * b;
            }
          double A1 = 2.0 * m1 * m2 + SSIM_C1, A2 = 2.0 * (e12 - m1 * m2) + SSIM_C2;
          double B1 = m1 * m1 + m2 * m2 + SSIM_C1, B2 = (e11 - m1 * m1) + (e22 - m2 * m2) + SSIM_C2;
          double s = (A1 * A2) / (B1 * B2);
          const int64_t p = (int64_t)y * W + x;
          ssum += s;
          if (ssim_map) ssim_map[3 * off + c * plane + p] = s;
          /* partial derivatives of s with respect to m1, e11, e12 */
          ds1[p] = s * (2.0 * m2 / A1 - 2.0 * m2 / A2 - 2.0 * m1 / B1 + 2.0 * m1 / B2);
          ds11[p] = -s / B2;
          ds12[p] = 2.0 * s / A2;
          double d = X[p] - Y[p];
          l1 += fabs(d);
        }
      if (grad) {
        for (int y = 0; y < H; ++y)
          for (int x = 0; x < W; ++x) {
            const int64_t p = (int64_t)y * W + x;
            /* d(sum_q s(q)) / dX(p): every window sum at q that contains p */
            double t1 = 0, t11 = 0, t12 = 0;
            for (int i = -SSIM_R; i <= SSIM_R; ++i)
              for (int j = -SSIM_R; j <= SSIM_R; ++j) {
                int yy = y + i, xx = x + j;
                if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                double g = w[i + SSIM_R] * w[j + SSIM_R];
                int64_t q = (int64_t)yy * W + xx;
                t1 += g * ds1[q];
                t11 += g * ds11[q];
                t12 += g * ds12[q];
              }
            double dS = t1 + 2.0 * X[p] * t11 + Y[p] * t12;
            double d = X[p] - Y[p];
            double sg = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
            grad[3 * off + c * plane + p] = (1.0 - lambda) * sg / n - lambda * dS / n;
          }
      }
    }
    free(ds1);
    free(ds11);
    free(ds12);
    off += plane;
  }
  *ssim = ssum / n;
  return (1.0 - lambda) * l1 / n + lambda * (1.0 - ssum / n);
}
