/*
 * FP64 CPU oracle of the differentiable 3D Gaussian splatting rasterizer of
 * Gaussian-LIC2 (arxiv 2507.04004).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library; the two sides meet only through the seeded input generator.
 *
 * What it computes, and where the paper defines it:
 *   - projection of a Gaussian (Sec. "3D Gaussian Splatting Representation",
 *     the equations for mu', mu_hat and Sigma' that precede Eq. alpha);
 *   - the per-pixel weight alpha (Eq. alpha);
 *   - front-to-back compositing of colour, depth and opacity
 *     (Eq. rendered_rgb, Eq. rendered_depth, Eq. rendered_opacity);
 *   - view-dependent colour from spherical harmonics (the text after
 *     Eq. rendered_opacity);
 *   - the tile list of a Gaussian under the 1/255 tile culling rule
 *     (Sec. "Fast Tile-based Culling");
 *   - the depth-regularised loss (Eq. depth_loss; L1 photometric and
 *     opacity-normalised sparse depth terms);
 *   - gradients w.r.t. the Gaussian parameters and the right-perturbation
 *     derivative w.r.t. the camera pose (Eq. 3dgs_jacobi and the manifold
 *     derivative defined after it).
 *
 * Readings where the paper defers to 3DGS (kerbl20233d) or is silent; every
 * one is a named field of ocl_config or a fixed convention stated here:
 *   - alpha is clamped at alpha_max (0.99); a Gaussian with alpha below
 *     alpha_min (1/255) at a pixel is skipped; compositing stops before a
 *     Gaussian whose blending would drop the transmittance below t_min (1e-4);
 *   - pixel (i, j) is sampled at (i + 0.5, j + 0.5);
 *   - the depth key used for ordering and for the near-plane cut is the FP32
 *     value fmaf(R20, x, fmaf(R21, y, fmaf(R22, z, t2))) on the FP32-rounded
 *     inputs; ties are broken by Gaussian index;
 *   - Sigma' carries a dilation of 0.3 px^2 on the diagonal, and the
 *     normalised camera coordinates inside the affine Jacobian are clamped to
 *     fov_clamp (1.3) times the half field of view; the clamp is differentiated
 *     exactly (zero slope for a clamped coordinate);
 *   - colour = max(0, sum_k SH_k Y_k(dir) + 0.5) with dir the unit vector from
 *     the camera centre c_w = -R^T t to the Gaussian mean;
 *   - the real spherical-harmonic basis carries the Condon-Shortley phase and
 *     is ordered m = -l..l inside each degree l; it is built here from the
 *     Legendre polynomials, not from a table of constants;
 *   - the L1 norms of Eq. depth_loss are means: the colour term over 3HW, the
 *     depth term over |M_d| = #(D_s > 0); a pixel that no Gaussian reaches
 *     (O = 0) contributes nothing to the depth term; sign(0) = 0;
 *   - the pose derivative uses the right perturbation T Exp(xi) of the
 *     world-to-camera transform, xi = (rho, theta), translation first.
 *
 * Derivatives: the per-pixel compositing adjoint is written out by hand in
 * reverse mode; the per-Gaussian projection chain is differentiated by forward
 * mode with dual numbers (exact derivatives of the same FP64 forward code),
 * and so are the per-pixel pose Jacobian rows.
 */
#include <omp.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" {

typedef struct {
  int64_t n;
  int32_t sh_degree;            /* 0..3 */
  const double* mean;           /* [3][n] */
  const double* log_scale;      /* [3][n] */
  const double* quat;           /* [4][n], (w, x, y, z), not necessarily unit */
  const double* logit_opacity;  /* [n] */
  const double* sh_dc;          /* [3][n] */
  const double* sh_rest;        /* [(K-1)][3][n], K = (deg+1)^2; may be null if deg == 0 */
} ocl_map;

typedef struct {
  double R[9];  /* world-to-camera rotation, row-major */
  double t[3];  /* world-to-camera translation */
  double fx, fy, cx, cy;
  int32_t width, height;
} ocl_camera;

typedef struct {
  double alpha_min, alpha_max, t_min, near_z, dilation, fov_clamp;
  double bg[3];
} ocl_config;

}  // extern "C"

namespace {

constexpr double kPi = 3.14159265358979323846;

/* ---------------- dual numbers (forward-mode derivatives) ---------------- */

template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0) { std::fill(d, d + N, 0.0); }
  Dual(double x) : v(x) { std::fill(d, d + N, 0.0); }  // NOLINT: implicit on purpose
};

template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v; for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }

template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r; r.v = std::sqrt(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}
template <int N> inline Dual<N> exp(const Dual<N>& a) {
  Dual<N> r; r.v = std::exp(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * r.v;
  return r;
}
inline double val(double x) { return x; }
template <int N> inline double val(const Dual<N>& x) { return x.v; }
using std::exp;
using std::sqrt;

/* ---------------- real spherical harmonics ---------------- */

/* Coefficients of the Legendre polynomials P_0..P_3 in powers of z. */
const double kLegendre[4][4] = {
    {1.0, 0.0, 0.0, 0.0},
    {0.0, 1.0, 0.0, 0.0},
    {-0.5, 0.0, 1.5, 0.0},
    {0.0, -1.5, 0.0, 2.5},
};

double factorial(int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; }

/* Real SH basis of degree <= deg at (x, y, z), |.| = 1 expected.
 * Y_l^m = K_lm * d^m P_l/dz^m (z) * Re (x + i y)^m   (m > 0)
 * Y_l^-m = K_lm * d^m P_l/dz^m (z) * Im (x + i y)^m  (m > 0)
 * K_lm = (-1)^m sqrt(2)^[m>0] sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
 * On the unit sphere this is sqrt(2) N_lm P_l^m(cos th) {cos, sin}(m phi) with
 * the Condon-Shortley phase, i.e. the textbook real basis. */
template <class S>
void sh_basis(int deg, const S& x, const S& y, const S& z, S* Y) {
  S re[4], im[4];
  re[0] = S(1.0); im[0] = S(0.0);
  for (int m = 1; m <= 3; ++m) {
    re[m] = re[m - 1] * x - im[m - 1] * y;
    im[m] = re[m - 1] * y + im[m - 1] * x;
  }
  for (int l = 0; l <= deg; ++l) {
    for (int m = 0; m <= l; ++m) {
      /* m-th derivative of P_l, evaluated by Horner at z */
      double dc[4] = {0, 0, 0, 0};
      for (int k = 0; k <= 3; ++k) dc[k] = kLegendre[l][k];
      for (int r = 0; r < m; ++r) {
        double nd[4] = {0, 0, 0, 0};
        for (int k = 1; k <= 3; ++k) nd[k - 1] = dc[k] * k;
        std::memcpy(dc, nd, sizeof(dc));
      }
      S q = S(dc[3]);
      for (int k = 2; k >= 0; --k) q = q * z + dc[k];
      double K = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - m) / factorial(l + m));
      if (m > 0) K *= std::sqrt(2.0);
      if (m % 2 == 1) K = -K;
      Y[l * l + l + m] = K * q * re[m];
      if (m > 0) Y[l * l + l - m] = K * q * im[m];
    }
  }
}

/* ---------------- per-Gaussian projection ---------------- */

template <class S>
struct Proj {
  bool valid = false;
  float depth32 = 0.f;
  S mx, my;        /* mean2d, pixels */
  S A, B, C;       /* Sigma' (dilated), symmetric 2x2 */
  S ca, cb, cc;    /* conic = inverse of Sigma': q = ca dx^2 + 2 cb dx dy + cc dy^2 */
  S o;             /* opacity */
  S col[3];        /* colour after the clamp at 0 */
  double raw[3];   /* colour before the clamp (values only) */
  S depth;         /* camera-frame depth */
  bool clamp_x = false, clamp_y = false;
};

template <class S>
struct GaussIn {
  S mean[3], log_scale[3], quat[4], logit;
  S sh[16][3];
};

/* FP32 depth key of a Gaussian (the ordering and near-cut quantity). */
float depth_key(const double R[9], const double t[3], double x, double y, double z) {
  return std::fmaf((float)R[6], (float)x,
                   std::fmaf((float)R[7], (float)y, std::fmaf((float)R[8], (float)z, (float)t[2])));
}

template <class S>
Proj<S> project_one(const GaussIn<S>& g, int deg, const S W[9], const S t[3], const ocl_camera& cam,
                    const ocl_config& cfg, float depth32) {
  Proj<S> p;
  p.depth32 = depth32;
  if (!(depth32 > (float)cfg.near_z)) return p;
  /* mu_hat = R mu + t */
  S mh[3];
  for (int i = 0; i < 3; ++i) mh[i] = W[3 * i] * g.mean[0] + W[3 * i + 1] * g.mean[1] + W[3 * i + 2] * g.mean[2] + t[i];
  S z = mh[2];
  p.depth = z;
  p.mx = cam.fx * mh[0] / z + cam.cx;
  p.my = cam.fy * mh[1] / z + cam.cy;
  /* affine Jacobian of the perspective projection, with clamped x/z, y/z */
  double limx = cfg.fov_clamp * 0.5 * cam.width / cam.fx;
  double limy = cfg.fov_clamp * 0.5 * cam.height / cam.fy;
  S tx = mh[0] / z, ty = mh[1] / z;
  if (val(tx) > limx) { tx = S(limx); p.clamp_x = true; }
  if (val(tx) < -limx) { tx = S(-limx); p.clamp_x = true; }
  if (val(ty) > limy) { ty = S(limy); p.clamp_y = true; }
  if (val(ty) < -limy) { ty = S(-limy); p.clamp_y = true; }
  S J[2][3];
  J[0][0] = cam.fx / z; J[0][1] = S(0.0); J[0][2] = -(cam.fx * tx) / z;
  J[1][0] = S(0.0); J[1][1] = cam.fy / z; J[1][2] = -(cam.fy * ty) / z;
  /* M = J R (2x3) */
  S M[2][3];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) M[r][c] = J[r][0] * W[c] + J[r][1] * W[3 + c] + J[r][2] * W[6 + c];
  /* rotation of the Gaussian from its normalised quaternion (w, x, y, z) */
  S qn = sqrt(g.quat[0] * g.quat[0] + g.quat[1] * g.quat[1] + g.quat[2] * g.quat[2] + g.quat[3] * g.quat[3]);
  S qw = g.quat[0] / qn, qx = g.quat[1] / qn, qy = g.quat[2] / qn, qz = g.quat[3] / qn;
  S Rg[3][3];
  Rg[0][0] = 1.0 - 2.0 * (qy * qy + qz * qz); Rg[0][1] = 2.0 * (qx * qy - qw * qz); Rg[0][2] = 2.0 * (qx * qz + qw * qy);
  Rg[1][0] = 2.0 * (qx * qy + qw * qz); Rg[1][1] = 1.0 - 2.0 * (qx * qx + qz * qz); Rg[1][2] = 2.0 * (qy * qz - qw * qx);
  Rg[2][0] = 2.0 * (qx * qz - qw * qy); Rg[2][1] = 2.0 * (qy * qz + qw * qx); Rg[2][2] = 1.0 - 2.0 * (qx * qx + qy * qy);
  /* Sigma = R_g S S^T R_g^T */
  S s2[3];
  for (int k = 0; k < 3; ++k) { S s = exp(g.log_scale[k]); s2[k] = s * s; }
  S Sig[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Sig[i][j] = Rg[i][0] * s2[0] * Rg[j][0] + Rg[i][1] * s2[1] * Rg[j][1] + Rg[i][2] * s2[2] * Rg[j][2];
  /* Sigma' = M Sigma M^T + dilation I */
  S MS[2][3];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c) MS[r][c] = M[r][0] * Sig[0][c] + M[r][1] * Sig[1][c] + M[r][2] * Sig[2][c];
  p.A = MS[0][0] * M[0][0] + MS[0][1] * M[0][1] + MS[0][2] * M[0][2] + cfg.dilation;
  p.B = MS[0][0] * M[1][0] + MS[0][1] * M[1][1] + MS[0][2] * M[1][2];
  p.C = MS[1][0] * M[1][0] + MS[1][1] * M[1][1] + MS[1][2] * M[1][2] + cfg.dilation;
  S det = p.A * p.C - p.B * p.B;
  if (!(val(det) > 0.0)) return p;
  p.ca = p.C / det; p.cb = -p.B / det; p.cc = p.A / det;
  p.o = 1.0 / (1.0 + exp(-g.logit));
  /* view-dependent colour; camera centre c_w = -R^T t */
  S cw[3];
  for (int i = 0; i < 3; ++i) cw[i] = -(W[i] * t[0] + W[3 + i] * t[1] + W[6 + i] * t[2]);
  S v[3] = {g.mean[0] - cw[0], g.mean[1] - cw[1], g.mean[2] - cw[2]};
  S vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  S Y[16];
  sh_basis(deg, v[0] / vn, v[1] / vn, v[2] / vn, Y);
  int K = (deg + 1) * (deg + 1);
  for (int ch = 0; ch < 3; ++ch) {
    S acc = S(0.5);
    for (int k = 0; k < K; ++k) acc = acc + g.sh[k][ch] * Y[k];
    p.raw[ch] = val(acc);
    p.col[ch] = val(acc) > 0.0 ? acc : S(0.0);
  }
  p.valid = true;
  return p;
}

template <class S>
GaussIn<S> load_gauss(const ocl_map& m, int64_t i) {
  GaussIn<S> g;
  const int64_t n = m.n;
  for (int k = 0; k < 3; ++k) { g.mean[k] = S(m.mean[k * n + i]); g.log_scale[k] = S(m.log_scale[k * n + i]); }
  for (int k = 0; k < 4; ++k) g.quat[k] = S(m.quat[k * n + i]);
  g.logit = S(m.logit_opacity[i]);
  int K = (m.sh_degree + 1) * (m.sh_degree + 1);
  for (int k = 0; k < 16; ++k)
    for (int ch = 0; ch < 3; ++ch) g.sh[k][ch] = S(0.0);
  for (int ch = 0; ch < 3; ++ch) g.sh[0][ch] = S(m.sh_dc[ch * n + i]);
  for (int k = 1; k < K; ++k)
    for (int ch = 0; ch < 3; ++ch) g.sh[k][ch] = S(m.sh_rest[((int64_t)(k - 1) * 3 + ch) * n + i]);
  return g;
}

float key_of(const ocl_map& m, const ocl_camera& cam, int64_t i) {
  const int64_t n = m.n;
  return depth_key(cam.R, cam.t, m.mean[i], m.mean[n + i], m.mean[2 * n + i]);
}

Proj<double> project_plain(const ocl_map& m, const ocl_camera& cam, const ocl_config& cfg, int64_t i) {
  GaussIn<double> g = load_gauss<double>(m, i);
  return project_one<double>(g, m.sh_degree, cam.R, cam.t, cam, cfg, key_of(m, cam, i));
}

/* ---------------- SE(3) exponential, right perturbation ---------------- */

/* T Exp(xi) for dual-number xi whose value is exactly zero: the series
 * R = I + [th]x + [th]x^2 / 2, V = I + [th]x / 2 + [th]x^2 / 6 is exact in
 * value and first derivative there. */
template <class S>
void perturb_pose(const double R[9], const double t[3], const S xi[6], S Wp[9], S tp[3]) {
  const S* rho = xi;
  const S* th = xi + 3;
  S K[3][3] = {{S(0.0), -th[2], th[1]}, {th[2], S(0.0), -th[0]}, {-th[1], th[0], S(0.0)}};
  S K2[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[i][j] = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
  S Re[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double I = (i == j) ? 1.0 : 0.0;
      Re[i][j] = I + K[i][j] + 0.5 * K2[i][j];
      V[i][j] = I + 0.5 * K[i][j] + K2[i][j] / 6.0;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Wp[3 * i + j] = R[3 * i] * Re[0][j] + R[3 * i + 1] * Re[1][j] + R[3 * i + 2] * Re[2][j];
  S Vr[3];
  for (int i = 0; i < 3; ++i) Vr[i] = V[i][0] * rho[0] + V[i][1] * rho[1] + V[i][2] * rho[2];
  for (int i = 0; i < 3; ++i) tp[i] = R[3 * i] * Vr[0] + R[3 * i + 1] * Vr[1] + R[3 * i + 2] * Vr[2] + t[i];
}

/* ---------------- per-pixel candidate lists ---------------- */

struct Cand {
  float key;
  int32_t gid;
};

/* Exact pixel box containing every pixel centre where o exp(-q/2) >= a_lo.
 * The ellipse {d : d^T Sigma'^-1 d <= r} spans |dx| <= sqrt(r Sigma'_xx),
 * |dy| <= sqrt(r Sigma'_yy).  One pixel of slack on each side; the caller
 * tests every pixel of the box exactly. */
bool footprint(const Proj<double>& p, double a_lo, int W, int H, int* x0, int* x1, int* y0, int* y1) {
  if (!p.valid) return false;
  if (!(p.o >= a_lo)) return false;
  double r = 2.0 * std::log(p.o / a_lo);
  double hx = std::sqrt(r * p.A), hy = std::sqrt(r * p.C);
  *x0 = std::max(0, (int)std::floor(p.mx - hx - 0.5) - 1);
  *x1 = std::min(W - 1, (int)std::ceil(p.mx + hx - 0.5) + 1);
  *y0 = std::max(0, (int)std::floor(p.my - hy - 0.5) - 1);
  *y1 = std::min(H - 1, (int)std::ceil(p.my + hy - 0.5) + 1);
  return *x0 <= *x1 && *y0 <= *y1;
}

inline double quad_form(const Proj<double>& p, double px, double py) {
  double dx = px - p.mx, dy = py - p.my;
  return p.ca * dx * dx + 2.0 * p.cb * dx * dy + p.cc * dy * dy;
}

enum { FLAG_SKIP = 1, FLAG_STOP = 2, FLAG_CLAMP = 4 };

/* Projected map of one view plus, per image row, the Gaussians whose
 * footprint box meets that row. */
struct ViewCache {
  std::vector<Proj<double>> proj;
  std::vector<std::vector<int32_t>> rows;
  std::vector<int> bx0, bx1;
};

/* Only the pixel rectangle [rx0, rx0+rw) x [ry0, ry0+rh) is filled in. */
void build_view(const ocl_map& m, const ocl_camera& cam, const ocl_config& cfg, double margin_eps, bool brute,
                int rx0, int ry0, int rw, int rh, ViewCache* vc) {
  const int64_t n = m.n;
  vc->proj.resize(n);
  vc->bx0.assign(n, 0);
  vc->bx1.assign(n, -1);
  vc->rows.assign(cam.height, {});
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) vc->proj[i] = project_plain(m, cam, cfg, i);
  double a_lo = cfg.alpha_min * (1.0 - margin_eps);
  for (int64_t i = 0; i < n; ++i) {
    int x0, x1, y0, y1;
    bool hit;
    if (brute) {
      hit = vc->proj[i].valid;
      x0 = 0; x1 = cam.width - 1; y0 = 0; y1 = cam.height - 1;
    } else {
      hit = footprint(vc->proj[i], a_lo, cam.width, cam.height, &x0, &x1, &y0, &y1);
    }
    if (!hit) continue;
    if (x1 < rx0 || x0 >= rx0 + rw) continue;
    vc->bx0[i] = x0; vc->bx1[i] = x1;
    for (int y = std::max(y0, ry0); y <= std::min(y1, ry0 + rh - 1); ++y) vc->rows[y].push_back((int32_t)i);
  }
}

/* Contributors of one pixel, in compositing order. */
struct PixelState {
  std::vector<int32_t> gid;
  std::vector<double> alpha, T, G;
  std::vector<char> clamped;
  double T_final = 1.0;
  int flags = 0;
};

/* Candidates are the Gaussians with o exp(-q/2) >= alpha_min in depth-key
 * order; ones just below the threshold (within margin_eps) are walked too, only
 * to flag the pixel when such a near-threshold decision comes before the stop. */
void composite_pixel(const ViewCache& vc, const ocl_config& cfg, int px, int py, double margin_eps, PixelState* st) {
  std::vector<Cand> cand;
  const double cxp = px + 0.5, cyp = py + 0.5;
  const double a_lo = cfg.alpha_min * (1.0 - margin_eps);
  for (int32_t i : vc.rows[py]) {
    if (px < vc.bx0[i] || px > vc.bx1[i]) continue;
    const Proj<double>& p = vc.proj[i];
    double q = quad_form(p, cxp, cyp);
    double a = p.o * std::exp(-0.5 * q);
    if (a >= a_lo) cand.push_back({p.depth32, i});
  }
  std::sort(cand.begin(), cand.end(), [](const Cand& u, const Cand& v) {
    return u.key < v.key || (u.key == v.key && u.gid < v.gid);
  });
  double T = 1.0;
  for (const Cand& c : cand) {
    const Proj<double>& p = vc.proj[c.gid];
    double q = quad_form(p, cxp, cyp);
    double G = std::exp(-0.5 * q);
    double a_raw = p.o * G;
    if (std::fabs(a_raw / cfg.alpha_min - 1.0) <= margin_eps) st->flags |= FLAG_SKIP;
    if (!(a_raw >= cfg.alpha_min)) continue;
    bool clamped = a_raw > cfg.alpha_max;
    if (std::fabs(a_raw / cfg.alpha_max - 1.0) <= margin_eps) st->flags |= FLAG_CLAMP;
    double a = clamped ? cfg.alpha_max : a_raw;
    double Tn = T * (1.0 - a);
    if (std::fabs(Tn / cfg.t_min - 1.0) <= margin_eps) st->flags |= FLAG_STOP;
    if (Tn < cfg.t_min) break;
    st->gid.push_back(c.gid);
    st->alpha.push_back(a);
    st->T.push_back(T);
    st->G.push_back(G);
    st->clamped.push_back(clamped);
    T = Tn;
  }
  st->T_final = T;
}

/* Per-Gaussian 2D adjoint: d/d(mx, my, ca, cb, cc, o, r, g, b, depth). */
constexpr int kAdj = 10;

}  // namespace

extern "C" {

/* Real SH basis values Y[0..(deg+1)^2) at a unit direction. */
void ocl_sh_basis(int32_t deg, const double* dir, double* Y) {
  for (int k = 0; k < 16; ++k) Y[k] = 0.0;
  sh_basis<double>(deg, dir[0], dir[1], dir[2], Y);
}

/* Projection of every Gaussian into one view. Arrays are planar [c][n]. */
int32_t ocl_project(const ocl_map* m, const ocl_camera* cam, const ocl_config* cfg, int32_t* valid,
                    double* mean2d, double* cov2d, double* conic, double* opacity, double* rgb, double* depth,
                    float* depth32, int32_t* clamp_flags) {
  const int64_t n = m->n;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    Proj<double> p = project_plain(*m, *cam, *cfg, i);
    valid[i] = p.valid ? 1 : 0;
    depth32[i] = p.depth32;
    clamp_flags[i] = (p.clamp_x ? 1 : 0) | (p.clamp_y ? 2 : 0);
    if (!p.valid) continue;
    mean2d[i] = p.mx; mean2d[n + i] = p.my;
    cov2d[i] = p.A; cov2d[n + i] = p.B; cov2d[2 * n + i] = p.C;
    conic[i] = p.ca; conic[n + i] = p.cb; conic[2 * n + i] = p.cc;
    opacity[i] = p.o;
    for (int c = 0; c < 3; ++c) rgb[c * n + i] = p.col[c];
    depth[i] = p.depth;
    for (int c = 0; c < 3; ++c)
      if (p.raw[c] <= 0.0) clamp_flags[i] |= 4 << c;
  }
  return 0;
}

/* Tile lists (16x16 tiles): every (tile, Gaussian) pair whose tile holds a
 * pixel centre with o exp(-q/2) >= alpha_min, found by testing every pixel of
 * every tile the footprint box meets (brute = every tile of the image).
 * Pairs are written sorted by (tile, depth key, Gaussian index).  margin[k] is
 * 1 when the pair's decision lies within a relative margin_eps of the
 * threshold in q.  Returns the pair count, or -(count) if cap is too small. */
int64_t ocl_tiles(const ocl_map* m, const ocl_camera* cam, const ocl_config* cfg, int32_t brute, double margin_eps,
                  int64_t cap, int32_t* tile, int32_t* gid, int32_t* margin) {
  const int64_t n = m->n;
  const int W = cam->width, H = cam->height;
  const int tw = (W + 15) / 16;
  struct Pair { int32_t tile; float key; int32_t gid; int32_t margin; };
  std::vector<std::vector<Pair>> per(n);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    Proj<double> p = project_plain(*m, *cam, *cfg, i);
    int x0, x1, y0, y1;
    if (!p.valid) continue;
    if (brute) { x0 = 0; x1 = W - 1; y0 = 0; y1 = H - 1; }
    else if (!footprint(p, cfg->alpha_min * (1.0 - margin_eps), W, H, &x0, &x1, &y0, &y1)) continue;
    if (!(p.o > 0.0)) continue;
    double q_thr = 2.0 * std::log(p.o / cfg->alpha_min);
    for (int ty = y0 / 16; ty <= y1 / 16; ++ty)
      for (int tx = x0 / 16; tx <= x1 / 16; ++tx) {
        double qmin = INFINITY;
        for (int y = ty * 16; y < std::min(H, ty * 16 + 16); ++y)
          for (int x = tx * 16; x < std::min(W, tx * 16 + 16); ++x) qmin = std::min(qmin, quad_form(p, x + 0.5, y + 0.5));
        bool near_thr = std::fabs(qmin - q_thr) <= margin_eps * std::max(1.0, std::fabs(q_thr));
        bool pass = p.o * std::exp(-0.5 * qmin) >= cfg->alpha_min;
        /* margin: 0 = clean pass, 1 = pass near the threshold,
         * 2 = fail near the threshold (not part of the exact list) */
        if (pass || near_thr) per[i].push_back({ty * tw + tx, p.depth32, (int32_t)i, near_thr ? (pass ? 1 : 2) : 0});
      }
  }
  std::vector<Pair> all;
  for (int64_t i = 0; i < n; ++i) all.insert(all.end(), per[i].begin(), per[i].end());
  std::sort(all.begin(), all.end(), [](const Pair& a, const Pair& b) {
    if (a.tile != b.tile) return a.tile < b.tile;
    if (a.key != b.key) return a.key < b.key;
    return a.gid < b.gid;
  });
  int64_t np = (int64_t)all.size();
  if (np > cap) return -np;
  for (int64_t k = 0; k < np; ++k) { tile[k] = all[k].tile; gid[k] = all[k].gid; margin[k] = all[k].margin; }
  return np;
}

/* Render the pixel rectangle [x0, x0+w) x [y0, y0+h) of one view.  Outputs
 * are planar over the rectangle: rgb [3][h][w], the rest [h][w].  n_contrib
 * counts the Gaussians blended at a pixel, last_gid is the last one (or -1),
 * flags marks pixels with a decision within margin_eps of a threshold.
 * brute = 1 tests every Gaussian at every pixel. */
int32_t ocl_render(const ocl_map* m, const ocl_camera* cam, const ocl_config* cfg, int32_t x0, int32_t y0, int32_t w,
                   int32_t h, int32_t brute, double margin_eps, double* rgb, double* depth, double* opac,
                   double* t_final, int32_t* n_contrib, int32_t* last_gid, int32_t* flags) {
  ViewCache vc;
  build_view(*m, *cam, *cfg, margin_eps, brute != 0, x0, y0, w, h, &vc);
  const int64_t hw = (int64_t)w * h;
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < h; ++j) {
    for (int i = 0; i < w; ++i) {
      PixelState st;
      composite_pixel(vc, *cfg, x0 + i, y0 + j, margin_eps, &st);
      double C[3] = {0, 0, 0}, D = 0, O = 0;
      for (size_t k = 0; k < st.gid.size(); ++k) {
        const Proj<double>& p = vc.proj[st.gid[k]];
        double wgt = st.alpha[k] * st.T[k];
        for (int c = 0; c < 3; ++c) C[c] += p.col[c] * wgt;
        D += p.depth * wgt;
        O += wgt;
      }
      for (int c = 0; c < 3; ++c) C[c] += st.T_final * cfg->bg[c];
      int64_t o = (int64_t)j * w + i;
      for (int c = 0; c < 3; ++c) rgb[c * hw + o] = C[c];
      depth[o] = D; opac[o] = O; t_final[o] = st.T_final;
      n_contrib[o] = (int32_t)st.gid.size();
      last_gid[o] = st.gid.empty() ? -1 : st.gid.back();
      flags[o] = st.flags;
    }
  }
  return 0;
}

/* Gradients of a loss through every view.  Per view v the pixel adjoints are
 *   fused loss (tgt_rgb != null): L_v = w_rgb mean_{3HW} |C^ - C|
 *        + w_depth / |M_d| sum_{D_s>0, O^>0} |D^/O^ - D_s|, |M_d| = #(D_s > 0);
 *   external (tgt_rgb == null): dL/dC^, dL/dD^, dL/dO^ read from ext_* arrays.
 * Only pixels inside the rectangle [x0,x0+w) x [y0,y0+h) are back-propagated
 * (the full image gives the exact gradient).  Gradients are written (not
 * accumulated) to the g_* arrays, which mirror the map layout; g_pose is
 * [V][6] = dL/d(rho, theta) for T_v Exp(xi); loss is [V].  Returns 0. */
int32_t ocl_backward(const ocl_map* m, int32_t n_views, const ocl_camera* cams, const ocl_config* cfg,
                     const double* tgt_rgb, const double* tgt_depth, double w_rgb, double w_depth,
                     const double* ext_rgb, const double* ext_depth, const double* ext_opac, int32_t x0, int32_t y0,
                     int32_t w, int32_t h, double* loss, double* g_mean, double* g_log_scale, double* g_quat,
                     double* g_logit, double* g_sh_dc, double* g_sh_rest, double* g_pose) {
  const int64_t n = m->n;
  const int deg = m->sh_degree;
  const int K = (deg + 1) * (deg + 1);
  std::fill(g_mean, g_mean + 3 * n, 0.0);
  std::fill(g_log_scale, g_log_scale + 3 * n, 0.0);
  std::fill(g_quat, g_quat + 4 * n, 0.0);
  std::fill(g_logit, g_logit + n, 0.0);
  std::fill(g_sh_dc, g_sh_dc + 3 * n, 0.0);
  if (K > 1 && g_sh_rest) std::fill(g_sh_rest, g_sh_rest + (int64_t)(K - 1) * 3 * n, 0.0);
  for (int v = 0; v < n_views; ++v) {
    const ocl_camera& cam = cams[v];
    const int W = cam.width, H = cam.height;
    const int64_t HW = (int64_t)W * H;
    ViewCache vc;
    build_view(*m, cam, *cfg, 0.0, false, x0, y0, w, h, &vc);
    std::vector<double> adj((size_t)n * kAdj, 0.0);
    double n_depth = 0.0;
    if (tgt_rgb && tgt_depth)
      for (int64_t k = 0; k < HW; ++k) n_depth += tgt_depth[v * HW + k] > 0.0 ? 1.0 : 0.0;
    double loss_v = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : loss_v)
    for (int j = y0; j < y0 + h; ++j) {
      for (int i = x0; i < x0 + w; ++i) {
        PixelState st;
        composite_pixel(vc, *cfg, i, j, 0.0, &st);
        const size_t nc = st.gid.size();
        double C[3] = {0, 0, 0}, D = 0, O = 0;
        for (size_t k = 0; k < nc; ++k) {
          const Proj<double>& p = vc.proj[st.gid[k]];
          double wgt = st.alpha[k] * st.T[k];
          for (int c = 0; c < 3; ++c) C[c] += p.col[c] * wgt;
          D += p.depth * wgt;
          O += wgt;
        }
        for (int c = 0; c < 3; ++c) C[c] += st.T_final * cfg->bg[c];
        const int64_t pix = (int64_t)j * W + i;
        double gC[3], gD, gO;
        if (tgt_rgb) {
          for (int c = 0; c < 3; ++c) {
            double r = C[c] - tgt_rgb[(v * 3 + c) * HW + pix];
            loss_v += w_rgb * std::fabs(r) / (3.0 * HW);
            gC[c] = w_rgb * ((r > 0) - (r < 0)) / (3.0 * HW);
          }
          gD = 0.0; gO = 0.0;
          double ds = tgt_depth ? tgt_depth[v * HW + pix] : 0.0;
          if (ds > 0.0 && O > 0.0 && n_depth > 0.0) {
            double r = D / O - ds;
            double s = (double)((r > 0) - (r < 0));
            loss_v += w_depth * std::fabs(r) / n_depth;
            gD = w_depth * s / (O * n_depth);
            gO = -w_depth * s * D / (O * O * n_depth);
          }
        } else {
          for (int c = 0; c < 3; ++c) gC[c] = ext_rgb ? ext_rgb[(v * 3 + c) * HW + pix] : 0.0;
          gD = ext_depth ? ext_depth[v * HW + pix] : 0.0;
          gO = ext_opac ? ext_opac[v * HW + pix] : 0.0;
        }
        /* Suffix sums behind each contributor: Sx_k = sum_{k' > k} x_k' a_k' T_k' */
        std::vector<double> SC(3 * nc + 3, 0.0), SD(nc + 1, 0.0), SO(nc + 1, 0.0);
        for (size_t kk = nc; kk-- > 0;) {
          const Proj<double>& p = vc.proj[st.gid[kk]];
          double wgt = st.alpha[kk] * st.T[kk];
          for (int c = 0; c < 3; ++c) SC[3 * kk + c] = SC[3 * (kk + 1) + c] + p.col[c] * wgt;
          SD[kk] = SD[kk + 1] + p.depth * wgt;
          SO[kk] = SO[kk + 1] + wgt;
        }
        const double cxp = i + 0.5, cyp = j + 0.5;
        for (size_t k = 0; k < nc; ++k) {
          const int32_t g = st.gid[k];
          const Proj<double>& p = vc.proj[g];
          const double a = st.alpha[k], T = st.T[k], Tn = T * (1.0 - a);
          /* what lies behind k, normalised by the transmittance after k */
          double dLda = 0.0;
          for (int c = 0; c < 3; ++c) {
            double behind = (SC[3 * (k + 1) + c] + st.T_final * cfg->bg[c]) / Tn;
            dLda += gC[c] * T * (p.col[c] - behind);
          }
          dLda += gD * T * (p.depth - SD[k + 1] / Tn);
          dLda += gO * T * (1.0 - SO[k + 1] / Tn);
          double* A = &adj[(size_t)g * kAdj];
          double dL_do = 0.0, dL_dq = 0.0;
          if (!st.clamped[k]) {
            dL_do = dLda * st.G[k];
            dL_dq = -0.5 * dLda * p.o * st.G[k];
          }
          double dx = cxp - p.mx, dy = cyp - p.my;
          double contrib[kAdj];
          contrib[0] = dL_dq * (-2.0) * (p.ca * dx + p.cb * dy);
          contrib[1] = dL_dq * (-2.0) * (p.cb * dx + p.cc * dy);
          contrib[2] = dL_dq * dx * dx;
          contrib[3] = dL_dq * 2.0 * dx * dy;
          contrib[4] = dL_dq * dy * dy;
          contrib[5] = dL_do;
          for (int c = 0; c < 3; ++c) contrib[6 + c] = gC[c] * a * T;
          contrib[9] = gD * a * T;
          for (int q = 0; q < kAdj; ++q) {
#pragma omp atomic
            A[q] += contrib[q];
          }
        }
      }
    }
    loss[v] = loss_v;
    /* Chain the 2D adjoints through the projection by forward-mode
     * derivatives: parameters (59 tangents) and pose (6 tangents). */
    constexpr int NP = 3 + 3 + 4 + 1 + 48;
    double pose_acc[6] = {0, 0, 0, 0, 0, 0};
    std::vector<double> pose_part((size_t)n * 6, 0.0);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t gi = 0; gi < n; ++gi) {
      const double* A = &adj[(size_t)gi * kAdj];
      bool any = false;
      for (int q = 0; q < kAdj; ++q) any |= A[q] != 0.0;
      if (!any) continue;
      const float key = key_of(*m, cam, gi);
      {
        GaussIn<Dual<NP>> g = load_gauss<Dual<NP>>(*m, gi);
        int s = 0;
        for (int k = 0; k < 3; ++k) g.mean[k].d[s++] = 1.0;
        for (int k = 0; k < 3; ++k) g.log_scale[k].d[s++] = 1.0;
        for (int k = 0; k < 4; ++k) g.quat[k].d[s++] = 1.0;
        g.logit.d[s++] = 1.0;
        for (int k = 0; k < 16; ++k)
          for (int ch = 0; ch < 3; ++ch) g.sh[k][ch].d[s++] = 1.0;
        Dual<NP> Wd[9], td[3];
        for (int k = 0; k < 9; ++k) Wd[k] = Dual<NP>(cam.R[k]);
        for (int k = 0; k < 3; ++k) td[k] = Dual<NP>(cam.t[k]);
        Proj<Dual<NP>> p = project_one<Dual<NP>>(g, deg, Wd, td, cam, *cfg, key);
        const Dual<NP>* outs[kAdj] = {&p.mx, &p.my, &p.ca, &p.cb, &p.cc, &p.o, &p.col[0], &p.col[1], &p.col[2], &p.depth};
        double gp[NP];
        for (int d = 0; d < NP; ++d) {
          double acc = 0.0;
          for (int q = 0; q < kAdj; ++q) acc += A[q] * outs[q]->d[d];
          gp[d] = acc;
        }
        int s2 = 0;
        for (int k = 0; k < 3; ++k) g_mean[k * n + gi] += gp[s2++];
        for (int k = 0; k < 3; ++k) g_log_scale[k * n + gi] += gp[s2++];
        for (int k = 0; k < 4; ++k) g_quat[k * n + gi] += gp[s2++];
        g_logit[gi] += gp[s2++];
        for (int k = 0; k < 16; ++k)
          for (int ch = 0; ch < 3; ++ch, ++s2) {
            if (k >= K) continue;
            if (k == 0) g_sh_dc[ch * n + gi] += gp[s2];
            else g_sh_rest[((int64_t)(k - 1) * 3 + ch) * n + gi] += gp[s2];
          }
      }
      {
        GaussIn<Dual<6>> g = load_gauss<Dual<6>>(*m, gi);
        Dual<6> xi[6], Wd[9], td[3];
        for (int k = 0; k < 6; ++k) { xi[k] = Dual<6>(0.0); xi[k].d[k] = 1.0; }
        perturb_pose<Dual<6>>(cam.R, cam.t, xi, Wd, td);
        Proj<Dual<6>> p = project_one<Dual<6>>(g, deg, Wd, td, cam, *cfg, key);
        const Dual<6>* outs[kAdj] = {&p.mx, &p.my, &p.ca, &p.cb, &p.cc, &p.o, &p.col[0], &p.col[1], &p.col[2], &p.depth};
        for (int d = 0; d < 6; ++d) {
          double acc = 0.0;
          for (int q = 0; q < kAdj; ++q) acc += A[q] * outs[q]->d[d];
          pose_part[(size_t)gi * 6 + d] = acc;
        }
      }
    }
    for (int64_t gi = 0; gi < n; ++gi)
      for (int d = 0; d < 6; ++d) pose_acc[d] += pose_part[(size_t)gi * 6 + d];
    for (int d = 0; d < 6; ++d) g_pose[v * 6 + d] = pose_acc[d];
  }
  return 0;
}

/* Pose Jacobian rows: for each listed pixel (linear index y*W + x) of one
 * view, J[p][c][k] = d C^_c / d xi_k under T Exp(xi) at xi = 0, by
 * forward-mode derivatives through projection and compositing; rgb[p][c] is
 * the rendered colour.  Returns 0. */
int32_t ocl_pose_jacobian(const ocl_map* m, const ocl_camera* cam, const ocl_config* cfg, const int32_t* pix,
                          int32_t n_pix, double* J, double* rgb) {
  const int64_t n = m->n;
  ViewCache vc;
  build_view(*m, *cam, *cfg, 0.0, false, 0, 0, cam->width, cam->height, &vc);
  // dual-number projections only for the Gaussians that contribute to a listed pixel
  std::vector<PixelState> states(n_pix);
#pragma omp parallel for schedule(dynamic, 16)
  for (int32_t k = 0; k < n_pix; ++k)
    composite_pixel(vc, *cfg, pix[k] % cam->width, pix[k] / cam->width, 0.0, &states[k]);
  std::vector<int32_t> slot(n, -1), used;
  for (int32_t k = 0; k < n_pix; ++k)
    for (int32_t g : states[k].gid)
      if (slot[g] < 0) { slot[g] = (int32_t)used.size(); used.push_back(g); }
  std::vector<Proj<Dual<6>>> pd(used.size());
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t u = 0; u < (int64_t)used.size(); ++u) {
    const int64_t gi = used[u];
    GaussIn<Dual<6>> g = load_gauss<Dual<6>>(*m, gi);
    Dual<6> xi[6], Wd[9], td[3];
    for (int k = 0; k < 6; ++k) { xi[k] = Dual<6>(0.0); xi[k].d[k] = 1.0; }
    perturb_pose<Dual<6>>(cam->R, cam->t, xi, Wd, td);
    pd[u] = project_one<Dual<6>>(g, m->sh_degree, Wd, td, *cam, *cfg, key_of(*m, *cam, gi));
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int32_t k = 0; k < n_pix; ++k) {
    const int px = pix[k] % cam->width, py = pix[k] / cam->width;
    const PixelState& st = states[k];
    Dual<6> C[3] = {Dual<6>(0.0), Dual<6>(0.0), Dual<6>(0.0)};
    Dual<6> T(1.0);
    const double cxp = px + 0.5, cyp = py + 0.5;
    for (size_t c = 0; c < st.gid.size(); ++c) {
      const Proj<Dual<6>>& p = pd[slot[st.gid[c]]];
      Dual<6> dx = cxp - p.mx, dy = cyp - p.my;
      Dual<6> q = p.ca * dx * dx + 2.0 * p.cb * dx * dy + p.cc * dy * dy;
      Dual<6> a = st.clamped[c] ? Dual<6>(cfg->alpha_max) : p.o * exp(-0.5 * q);
      for (int ch = 0; ch < 3; ++ch) C[ch] = C[ch] + p.col[ch] * a * T;
      T = T * (1.0 - a);
    }
    for (int ch = 0; ch < 3; ++ch) {
      C[ch] = C[ch] + T * cfg->bg[ch];
      rgb[k * 3 + ch] = C[ch].v;
      for (int d = 0; d < 6; ++d) J[(k * 3 + ch) * 6 + d] = C[ch].d[d];
    }
  }
  return 0;
}

/* Worker threads of the parallel loops (timing on a given number of cores). */
void ocl_set_threads(int32_t n) { omp_set_num_threads(n > 0 ? n : 1); }
int32_t ocl_get_threads() { return (int32_t)omp_get_max_threads(); }

/* FP32 depth keys of every Gaussian in one view (ordering quantity). */
void ocl_depth_keys(const ocl_map* m, const ocl_camera* cam, float* keys) {
  for (int64_t i = 0; i < m->n; ++i) keys[i] = key_of(*m, *cam, i);
}

}  // extern "C"
