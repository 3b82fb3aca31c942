// FP64 CPU oracle for the 4D-GS render path.  TEST INFRASTRUCTURE ONLY: see
// fs4d_oracle.h for what it is, which passage each function follows, and who may
// call it.  Plain loops, no blocking or fusion, so it can be checked by eye
// against the paper.
#include "fs4d_oracle.h"

#include <algorithm>
#include <array>
#include <map>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// The six planes of the HexPlane, as (first axis, second axis); axis 3 is time
// (Sec. 4.2: (x,y), (x,z), (y,z), (x,t), (y,t), (z,t)).
const int kPlaneAxes[6][2] = {{0, 1}, {0, 2}, {1, 2}, {0, 3}, {1, 3}, {2, 3}};
const int kHeadOut[3] = {3, 4, 3};

int plane_res(const orc_scene* s, int level, int axis) {
  return axis < 3 ? s->res_spatial[level] : s->res_time;
}

// Start (in floats) of plane (level, p) inside the packed plane buffer.
int64_t plane_offset(const orc_scene* s, int level, int p) {
  int64_t off = 0;
  for (int l = 0; l < s->n_levels; ++l)
    for (int q = 0; q < 6; ++q) {
      if (l == level && q == p) return off;
      off += (int64_t)plane_res(s, l, kPlaneAxes[q][0]) * plane_res(s, l, kPlaneAxes[q][1]) * s->feat_dim;
    }
  return off;
}


// Bilinear-interpolation setup along one axis of resolution R, for a coordinate
// u normalised to [-1, 1].  Vertex k sits at u = -1 + 2k/(R-1) (corner-aligned);
// coordinates outside the box are clamped to its border.
void axis_setup(double u, int R, int* i0, double* f, double* dgdu) {
  double uc = std::min(1.0, std::max(-1.0, u));
  double g = (uc + 1.0) * 0.5 * (R - 1);
  int i = (int)std::floor(g);
  if (i > R - 2) i = R - 2;
  if (i < 0) i = 0;
  *i0 = i;
  *f = g - i;
  // d g / d u, zero where the coordinate is clamped.
  *dgdu = (u > -1.0 && u < 1.0) ? 0.5 * (R - 1) : 0.0;
}

// Layer (out, in) shapes d1 d2 x1 x2 r1 r2 s1 s2 and the float offset of each.
// With colour heads (App. B) four more layers follow: c1 (W -> W), c2 (W -> 3K),
// a1 (W -> W), a2 (W -> 1).
struct MlpLayout {
  int out[12], in[12];
  int64_t w[12], b[12];
  int n_layers;
  int64_t total;
};

MlpLayout mlp_layout(const orc_scene* s) {
  MlpLayout L;
  int W = s->mlp_width, hin = s->feat_dim * s->n_levels;
  const int K3 = 3 * (s->sh_degree + 1) * (s->sh_degree + 1);
  L.out[0] = W; L.in[0] = hin;
  L.out[1] = W; L.in[1] = W;
  for (int h = 0; h < 3; ++h) {
    L.out[2 + 2 * h] = W; L.in[2 + 2 * h] = W;
    L.out[3 + 2 * h] = kHeadOut[h]; L.in[3 + 2 * h] = W;
  }
  L.n_layers = s->color_heads ? 12 : 8;
  L.out[8] = W; L.in[8] = W;
  L.out[9] = K3; L.in[9] = W;
  L.out[10] = W; L.in[10] = W;
  L.out[11] = 1; L.in[11] = W;
  int64_t off = 0;
  for (int k = 0; k < L.n_layers; ++k) {
    L.w[k] = off; off += (int64_t)L.out[k] * L.in[k];
    L.b[k] = off; off += L.out[k];
  }
  L.total = off;
  return L;
}

// y = W x + b for layer k of the packed MLP.
void linear(const orc_scene* s, const MlpLayout& L, int k, const double* x, double* y) {
  for (int o = 0; o < L.out[k]; ++o) {
    double acc = s->mlp[L.b[k] + o];
    for (int i = 0; i < L.in[k]; ++i) acc += (double)s->mlp[L.w[k] + (int64_t)o * L.in[k] + i] * x[i];
    y[o] = acc;
  }
}

double relu(double v) { return v > 0.0 ? v : 0.0; }

// Normalised 4-D coordinate (x, y, z, t) in [-1, 1]: the scene box maps to the
// grid (Sec. 4.2, "bounding plane voxels"), t in [0, 1] maps to [-1, 1].
void normalise(const orc_scene* s, const double* xyz, double t, double c[4]) {
  for (int a = 0; a < 3; ++a) c[a] = 2.0 * (xyz[a] - s->aabb_min[a]) / (s->aabb_max[a] - s->aabb_min[a]) - 1.0;
  c[3] = 2.0 * t - 1.0;
}

// Real spherical harmonics up to degree 3 (textbook real basis, no Condon-Shortley
// phase), ordered by degree then m = -l..l.
void sh_basis(int degree, const double d[3], double* Y) {
  const double x = d[0], y = d[1], z = d[2];
  const double PI = 3.14159265358979323846;
  Y[0] = 0.5 * std::sqrt(1.0 / PI);
  if (degree < 1) return;
  const double c1 = std::sqrt(3.0 / (4.0 * PI));
  Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
  if (degree < 2) return;
  Y[4] = 0.5 * std::sqrt(15.0 / PI) * x * y;
  Y[5] = 0.5 * std::sqrt(15.0 / PI) * y * z;
  Y[6] = 0.25 * std::sqrt(5.0 / PI) * (3.0 * z * z - 1.0);
  Y[7] = 0.5 * std::sqrt(15.0 / PI) * x * z;
  Y[8] = 0.25 * std::sqrt(15.0 / PI) * (x * x - y * y);
  if (degree < 3) return;
  Y[9] = 0.25 * std::sqrt(35.0 / (2.0 * PI)) * y * (3.0 * x * x - y * y);
  Y[10] = 0.5 * std::sqrt(105.0 / PI) * x * y * z;
  Y[11] = 0.25 * std::sqrt(21.0 / (2.0 * PI)) * y * (5.0 * z * z - 1.0);
  Y[12] = 0.25 * std::sqrt(7.0 / PI) * z * (5.0 * z * z - 3.0);
  Y[13] = 0.25 * std::sqrt(21.0 / (2.0 * PI)) * x * (5.0 * z * z - 1.0);
  Y[14] = 0.25 * std::sqrt(105.0 / PI) * z * (x * x - y * y);
  Y[15] = 0.25 * std::sqrt(35.0 / (2.0 * PI)) * x * (x * x - 3.0 * y * y);
}

// Rotation matrix of a unit quaternion (w, x, y, z).
void quat_to_rot(const double q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

double frac_margin(double v) {  // distance (in v's units) to the nearest integer
  return std::fabs(v - std::floor(v + 0.5));
}

const double kAlphaMax = 0.99;
const double kAlphaMin = 1.0 / 255.0;
const double kTMin = 1e-4;
const double kDilation = 0.3;
const double kGuard = 1.3;

}  // namespace

extern "C" {

void orc_set_threads(int32_t n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

// Eq. 5 "interp": bilinear interpolation of the 4 grid vertices around (ua, ub).
void orc_plane_sample(const orc_scene* s, int32_t level, int32_t p, double ua, double ub, double* out) {
  const int h = s->feat_dim;
  const int Ra = plane_res(s, level, kPlaneAxes[p][0]);
  const int Rb = plane_res(s, level, kPlaneAxes[p][1]);
  const float* P = s->planes + plane_offset(s, level, p);
  int i0, j0;
  double fa, fb, da, db;
  axis_setup(ua, Ra, &i0, &fa, &da);
  axis_setup(ub, Rb, &j0, &fb, &db);
  for (int c = 0; c < h; ++c) {
    double v00 = P[((int64_t)j0 * Ra + i0) * h + c];
    double v10 = P[((int64_t)j0 * Ra + i0 + 1) * h + c];
    double v01 = P[((int64_t)(j0 + 1) * Ra + i0) * h + c];
    double v11 = P[((int64_t)(j0 + 1) * Ra + i0 + 1) * h + c];
    out[c] = (1 - fa) * (1 - fb) * v00 + fa * (1 - fb) * v10 + (1 - fa) * fb * v01 + fa * fb * v11;
  }
}

// Eq. 5: f_h = concat over levels of the Hadamard product over the six planes.
void orc_features(const orc_scene* s, const double* xyz, int32_t n, double t, double* fh) {
  const int h = s->feat_dim, L = s->n_levels;
#pragma omp parallel for schedule(static)
  for (int g = 0; g < n; ++g) {
    double c[4];
    normalise(s, xyz + 3 * (int64_t)g, t, c);
    std::vector<double> v(h);
    for (int l = 0; l < L; ++l) {
      double* f = fh + (int64_t)g * h * L + (int64_t)l * h;
      for (int k = 0; k < h; ++k) f[k] = 1.0;
      for (int p = 0; p < 6; ++p) {
        orc_plane_sample(s, l, p, c[kPlaneAxes[p][0]], c[kPlaneAxes[p][1]], v.data());
        for (int k = 0; k < h; ++k) f[k] *= v[k];
      }
    }
  }
}

// Sec. 4.2: f_d = phi_d(f_h); dX = phi_x(f_d), dr = phi_r(f_d), ds = phi_s(f_d).
// delta is [n][10] = (dX 3, dr 4, ds 3).
void orc_mlp(const orc_scene* s, const double* fh, int32_t n, double* delta) {
  const MlpLayout Lo = mlp_layout(s);
  const int W = s->mlp_width, hin = s->feat_dim * s->n_levels;
#pragma omp parallel for schedule(static)
  for (int g = 0; g < n; ++g) {
    std::vector<double> a1(W), fd(W), hid(W), out(4);
    linear(s, Lo, 0, fh + (int64_t)g * hin, a1.data());
    for (auto& v : a1) v = relu(v);
    linear(s, Lo, 1, a1.data(), fd.data());
    for (auto& v : fd) v = relu(v);
    int col = 0;
    for (int head = 0; head < 3; ++head) {
      linear(s, Lo, 2 + 2 * head, fd.data(), hid.data());
      for (auto& v : hid) v = relu(v);
      linear(s, Lo, 3 + 2 * head, hid.data(), out.data());
      for (int o = 0; o < kHeadOut[head]; ++o) delta[(int64_t)g * 10 + col + o] = out[o];
      col += kHeadOut[head];
    }
  }
}

// Eq. 6: (X', r', s') = (X + dX, r + dr, s + ds); opacity and SH are unchanged.
void orc_deform(const orc_scene* s, double t, double* means, double* quats, double* log_scales) {
  const int n = s->n, hin = s->feat_dim * s->n_levels;
  std::vector<double> xyz(3 * (int64_t)n), fh((int64_t)n * hin), delta((int64_t)n * 10);
  for (int64_t i = 0; i < 3 * (int64_t)n; ++i) xyz[i] = s->means[i];
  orc_features(s, xyz.data(), n, t, fh.data());
  orc_mlp(s, fh.data(), n, delta.data());
  for (int64_t g = 0; g < n; ++g) {
    for (int a = 0; a < 3; ++a) means[3 * g + a] = (double)s->means[3 * g + a] + delta[10 * g + a];
    for (int a = 0; a < 4; ++a) quats[4 * g + a] = (double)s->quats[4 * g + a] + delta[10 * g + 3 + a];
    for (int a = 0; a < 3; ++a) log_scales[3 * g + a] = (double)s->log_scales[3 * g + a] + delta[10 * g + 7 + a];
  }
}

// App. B: dC = phi_C(f_d), dalpha = phi_alpha(f_d), each head Lin(W->W), ReLU,
// Lin(W->out) like the others; C' = C + dC over every SH coefficient, and the
// opacity deformation is read as an addition to the stored logit.
void orc_appearance(const orc_scene* s, double t, double* sh, double* opacity_logits) {
  const int n = s->n, hin = s->feat_dim * s->n_levels, W = s->mlp_width;
  const int K3 = 3 * (s->sh_degree + 1) * (s->sh_degree + 1);
  for (int64_t i = 0; i < (int64_t)n * K3; ++i) sh[i] = s->sh[i];
  for (int g = 0; g < n; ++g) opacity_logits[g] = s->opacity_logits[g];
  if (!s->color_heads) return;
  const MlpLayout Lo = mlp_layout(s);
  std::vector<double> xyz(3 * (int64_t)n), fh((int64_t)n * hin);
  for (int64_t i = 0; i < 3 * (int64_t)n; ++i) xyz[i] = s->means[i];
  orc_features(s, xyz.data(), n, t, fh.data());
#pragma omp parallel for schedule(static)
  for (int g = 0; g < n; ++g) {
    std::vector<double> a1(W), fd(W), hid(W), dc(K3), da(1);
    linear(s, Lo, 0, fh.data() + (int64_t)g * hin, a1.data());
    for (auto& v : a1) v = relu(v);
    linear(s, Lo, 1, a1.data(), fd.data());
    for (auto& v : fd) v = relu(v);
    linear(s, Lo, 8, fd.data(), hid.data());
    for (auto& v : hid) v = relu(v);
    linear(s, Lo, 9, hid.data(), dc.data());
    for (int j = 0; j < K3; ++j) sh[(int64_t)g * K3 + j] += dc[j];
    linear(s, Lo, 10, fd.data(), hid.data());
    for (auto& v : hid) v = relu(v);
    linear(s, Lo, 11, hid.data(), da.data());
    opacity_logits[g] += da[0];
  }
}

void orc_sh_basis(int32_t degree, const double* dir, double* basis) { sh_basis(degree, dir, basis); }

// Eq. 2 and Eq. 3 (EWA splatting), colour from SH, screen-space tile rectangle.
void orc_project(const orc_scene* s, const double* means, const double* quats, const double* log_scales,
                 const orc_camera* cam, int32_t tile, orc_projected* out) {
  orc_project_appearance(s, means, quats, log_scales, nullptr, nullptr, cam, tile, out);
}

void orc_project_appearance(const orc_scene* s, const double* means, const double* quats,
                            const double* log_scales, const double* shd, const double* lgd,
                            const orc_camera* cam, int32_t tile, orc_projected* out) {
  const int n = s->n;
  const int K = (s->sh_degree + 1) * (s->sh_degree + 1);
  const int tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
  const double* M = cam->world_to_cam;
  double Rc[3][3], tc[3], campos[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) Rc[r][c] = M[4 * r + c];
    tc[r] = M[4 * r + 3];
  }
  for (int c = 0; c < 3; ++c) campos[c] = -(Rc[0][c] * tc[0] + Rc[1][c] * tc[1] + Rc[2][c] * tc[2]);
  const double limx = kGuard * cam->width / (2.0 * cam->fx), limy = kGuard * cam->height / (2.0 * cam->fy);

#pragma omp parallel for schedule(static)
  for (int g = 0; g < n; ++g) {
    const double* X = means + 3 * (int64_t)g;
    out->radius[g] = 0;
    for (int k = 0; k < 4; ++k) out->rect[4 * (int64_t)g + k] = 0;
    out->margin[g] = 1e30;
    double p[3];
    for (int r = 0; r < 3; ++r) p[r] = Rc[r][0] * X[0] + Rc[r][1] * X[1] + Rc[r][2] * X[2] + tc[r];
    out->depth[g] = p[2];
    const double logit = lgd ? lgd[g] : (double)s->opacity_logits[g];
    out->opacity[g] = 1.0 / (1.0 + std::exp(-logit));
    out->margin[g] = std::min(out->margin[g], std::fabs(p[2] - cam->znear));
    if (!(p[2] > cam->znear)) continue;
    // Sigma = R S S^T R^T with R from the normalised quaternion, S = diag(exp(s')).
    double q[4], qn = 0;
    for (int k = 0; k < 4; ++k) { q[k] = quats[4 * (int64_t)g + k]; qn += q[k] * q[k]; }
    qn = std::sqrt(qn);
    for (int k = 0; k < 4; ++k) q[k] /= qn;
    double R[3][3];
    quat_to_rot(q, R);
    double S[3];
    for (int k = 0; k < 3; ++k) S[k] = std::exp(log_scales[3 * (int64_t)g + k]);
    double Sig[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int k = 0; k < 3; ++k) acc += R[i][k] * S[k] * S[k] * R[j][k];
        Sig[i][j] = acc;
      }
    // Jacobian of the perspective map at the mean (guard-band clamped).
    double txz = std::min(limx, std::max(-limx, p[0] / p[2])) * p[2];
    double tyz = std::min(limy, std::max(-limy, p[1] / p[2])) * p[2];
    double J[2][3] = {{cam->fx / p[2], 0.0, -cam->fx * txz / (p[2] * p[2])},
                      {0.0, cam->fy / p[2], -cam->fy * tyz / (p[2] * p[2])}};
    double T[2][3];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) T[i][j] = J[i][0] * Rc[0][j] + J[i][1] * Rc[1][j] + J[i][2] * Rc[2][j];
    double C2[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double acc = 0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) acc += T[i][a] * Sig[a][b] * T[j][b];
        C2[i][j] = acc;
      }
    double a = C2[0][0] + kDilation, b = C2[0][1], c = C2[1][1] + kDilation;
    out->cov2d[3 * (int64_t)g + 0] = a;
    out->cov2d[3 * (int64_t)g + 1] = b;
    out->cov2d[3 * (int64_t)g + 2] = c;
    double det = a * c - b * b;
    if (!(det > 0.0)) continue;
    out->conic[3 * (int64_t)g + 0] = c / det;
    out->conic[3 * (int64_t)g + 1] = -b / det;
    out->conic[3 * (int64_t)g + 2] = a / det;
    double mid = 0.5 * (a + c);
    double lmax = mid + std::sqrt(std::max(0.0, mid * mid - det));
    double r3 = 3.0 * std::sqrt(lmax);
    int radius = (int)std::ceil(r3);
    double u = cam->fx * p[0] / p[2] + cam->cx, v = cam->fy * p[1] / p[2] + cam->cy;
    out->xy[2 * (int64_t)g + 0] = u;
    out->xy[2 * (int64_t)g + 1] = v;
    double mg = frac_margin(r3);
    int x0 = (int)std::floor((u - radius) / tile), x1 = (int)std::floor((u + radius) / tile) + 1;
    int y0 = (int)std::floor((v - radius) / tile), y1 = (int)std::floor((v + radius) / tile) + 1;
    mg = std::min(mg, tile * std::min(frac_margin((u - radius) / tile), frac_margin((u + radius) / tile)));
    mg = std::min(mg, tile * std::min(frac_margin((v - radius) / tile), frac_margin((v + radius) / tile)));
    out->margin[g] = std::min(out->margin[g], mg);
    x0 = std::min(tiles_x, std::max(0, x0)); x1 = std::min(tiles_x, std::max(0, x1));
    y0 = std::min(tiles_y, std::max(0, y0)); y1 = std::min(tiles_y, std::max(0, y1));
    if (x1 <= x0 || y1 <= y0) continue;
    out->radius[g] = radius;
    int32_t* rc = out->rect + 4 * (int64_t)g;
    rc[0] = x0; rc[1] = y0; rc[2] = x1; rc[3] = y1;
    // Colour: SH evaluated along the viewing direction, offset by 0.5, clamped at 0.
    double dir[3], dn = 0;
    for (int k = 0; k < 3; ++k) { dir[k] = X[k] - campos[k]; dn += dir[k] * dir[k]; }
    dn = std::sqrt(dn);
    for (int k = 0; k < 3; ++k) dir[k] /= dn;
    double Y[16];
    sh_basis(s->sh_degree, dir, Y);
    for (int ch = 0; ch < 3; ++ch) {
      double acc = 0.5;
      for (int k = 0; k < K; ++k) {
        const int64_t e = ((int64_t)g * K + k) * 3 + ch;
        acc += Y[k] * (shd ? shd[e] : (double)s->sh[e]);
      }
      out->rgb[3 * (int64_t)g + ch] = std::max(0.0, acc);
    }
  }
}

// One (tile, depth) key per Gaussian and touched tile, emitted in Gaussian order
// and, within a Gaussian, in row-major tile order; then a stable sort on the key
// (so equal keys stay in Gaussian-index order) and per-tile [start, end) ranges.
int64_t orc_bin_sort(int32_t n, const uint32_t* depth_bits, const int32_t* rect, int32_t tiles_x,
                     int32_t tiles_y, int64_t capacity, uint64_t* keys, uint32_t* values, uint32_t* ranges) {
  std::vector<std::pair<uint64_t, uint32_t>> pairs;
  for (int g = 0; g < n; ++g) {
    const int32_t* rc = rect + 4 * (int64_t)g;
    for (int ty = rc[1]; ty < rc[3]; ++ty)
      for (int tx = rc[0]; tx < rc[2]; ++tx) {
        uint64_t tile_id = (uint64_t)ty * tiles_x + tx;
        pairs.push_back({(tile_id << 32) | depth_bits[g], (uint32_t)g});
      }
  }
  std::stable_sort(pairs.begin(), pairs.end(),
                   [](const std::pair<uint64_t, uint32_t>& a, const std::pair<uint64_t, uint32_t>& b) {
                     return a.first < b.first;
                   });
  const int64_t K = (int64_t)pairs.size();
  for (int64_t i = 0; i < std::min(K, capacity); ++i) {
    keys[i] = pairs[i].first;
    values[i] = pairs[i].second;
  }
  if (ranges) {
    std::memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)tiles_x * tiles_y);
    for (int64_t i = 0; i < K; ++i) {
      uint32_t tile_id = (uint32_t)(pairs[i].first >> 32);
      if (i == 0 || (uint32_t)(pairs[i - 1].first >> 32) != tile_id) ranges[2 * tile_id] = (uint32_t)i;
      if (i == K - 1 || (uint32_t)(pairs[i + 1].first >> 32) != tile_id) ranges[2 * tile_id + 1] = (uint32_t)(i + 1);
    }
  }
  return K;
}

// Eq. 4 with Eq. 1: per pixel, front to back over its tile's sorted list,
// C = sum_i c_i a_i prod_{j<i} (1 - a_j), a_i = min(0.99, o_i exp(-d^T conic d / 2)).
// Terms with a_i < 1/255 are skipped; the loop stops before the term that would
// take the transmittance below 1e-4.  Pixel (x, y) is evaluated at its centre
// (x + 0.5, y + 0.5); the background is black.
void orc_composite(int32_t width, int32_t height, int32_t tile, const uint32_t* ranges, const uint32_t* values,
                   const double* xy, const double* conic, const double* opacity, const double* rgb,
                   const double* depth, double* image, double* t_final, int32_t* n_contrib, double* margin) {
  const int tiles_x = (width + tile - 1) / tile;
#pragma omp parallel for schedule(dynamic, 16)
  for (int pix = 0; pix < width * height; ++pix) {
    const int px = pix % width, py = pix / width;
    const int tid = (py / tile) * tiles_x + (px / tile);
    const uint32_t start = ranges[2 * tid], end = ranges[2 * tid + 1];
    double T = 1.0, C[3] = {0, 0, 0}, mg = 1e30, prev_depth = -1.0;
    int last = 0;
    const double cx = px + 0.5, cy = py + 0.5;
    for (uint32_t k = start; k < end; ++k) {
      const uint32_t g = values[k];
      const double dx = xy[2 * g] - cx, dy = xy[2 * g + 1] - cy;
      const double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
      if (power > 0.0) continue;
      const double a_raw = opacity[g] * std::exp(power);
      const double alpha = std::min(kAlphaMax, a_raw);
      mg = std::min(mg, std::fabs(alpha - kAlphaMin) / kAlphaMin);
      if (alpha < kAlphaMin) continue;
      // Two blended terms whose depths tie to within float32 rounding may be
      // ordered differently by a float32 implementation: record the relative gap
      // (weighted x100, so one threshold of 5e-5 flags alpha/T decisions within
      // 5e-5 and depth gaps within 5e-7, ~8 float32 ulps, relative).
      if (prev_depth > 0.0) mg = std::min(mg, 100.0 * std::fabs(depth[g] - prev_depth) / std::fabs(depth[g]));
      prev_depth = depth[g];
      const double Tn = T * (1.0 - alpha);
      mg = std::min(mg, std::fabs(Tn - kTMin) / kTMin);
      if (Tn < kTMin) break;
      for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
      T = Tn;
      last = (int)(k - start) + 1;
    }
    for (int ch = 0; ch < 3; ++ch) image[3 * (int64_t)pix + ch] = C[ch];
    if (t_final) t_final[pix] = T;
    if (n_contrib) n_contrib[pix] = last;
    if (margin) margin[pix] = mg;
  }
}

// The blend of Eq. 4 for ONE pixel over a given list, with chosen decisions
// taken the other way.  A float32 implementation may legitimately decide a
// comparison differently from this float64 code when the compared quantities
// lie within rounding of each other; the outcomes below are every result such
// an implementation can produce (test support for parity checks, not part of
// the method).  Decisions of the pass over the list:
//   skip  -- alpha_i < 1/255 drops term i;
//   stop  -- T (1 - alpha_i) < 1e-4 ends the blend before term i;
//   order -- two blended terms whose depths tie to within rounding may swap.
// flip_kind/flip_gid name the decisions to invert (kind 0 skip, 1 stop, 2 order
// with the term that follows flip_gid in the list as blended).  Terms whose
// projected attributes (position, conic, opacity, colour) are identical -- copies
// made by densification -- take every decision alike in any implementation (the
// same inputs through the same arithmetic) and are interchangeable in order: they
// share one skip decision and never form an order decision with each other.
namespace {
struct Decision { int kind; uint32_t gid; };

// One pass; records the decisions within tolerance when `found` is non-null.
void blend_pixel(int len, const uint32_t* list, double px, double py, const double* xy, const double* conic,
                 const double* opacity, const double* rgb, const double* depth, const Decision* flips, int n_flips,
                 double rel_tol, double depth_tol, double C[5], std::vector<Decision>* found) {
  std::vector<uint32_t> order(list, list + len);
  // order flips first: swap the named term with the next term that blends at this pixel
  auto blends = [&](uint32_t g) {
    const double dx = xy[2 * g] - px, dy = xy[2 * g + 1] - py;
    const double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
    return power <= 0.0 && std::min(kAlphaMax, opacity[g] * std::exp(power)) >= kAlphaMin;
  };
  for (int f = 0; f < n_flips; ++f) {
    if (flips[f].kind != 2) continue;
    for (int k = 0; k < len; ++k) {
      if (order[k] != flips[f].gid) continue;
      for (int j = k + 1; j < len; ++j)
        if (blends(order[j])) { std::swap(order[k], order[j]); break; }
      break;
    }
  }
  auto flipped = [&](int kind, uint32_t g) {
    for (int f = 0; f < n_flips; ++f)
      if (flips[f].kind == kind && flips[f].gid == g) return true;
    return false;
  };
  // the first term of the list with the same projected attributes as each term
  std::map<std::array<double, 9>, uint32_t> first;
  std::map<uint32_t, uint32_t> rep;
  for (int k = 0; k < len; ++k) {
    const uint32_t g = order[k];
    const std::array<double, 9> key = {xy[2 * g], xy[2 * g + 1], conic[3 * g], conic[3 * g + 1], conic[3 * g + 2],
                                       opacity[g], rgb[3 * g], rgb[3 * g + 1], rgb[3 * g + 2]};
    rep[g] = first.emplace(key, g).first->second;
  }
  double T = 1.0, prev_depth = -1.0;
  uint32_t prev = 0;
  int last = 0;
  C[0] = C[1] = C[2] = 0.0;
  for (int k = 0; k < len; ++k) {
    const uint32_t g = order[k];
    const double dx = xy[2 * g] - px, dy = xy[2 * g + 1] - py;
    const double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
    if (power > 0.0) continue;
    const double alpha = std::min(kAlphaMax, opacity[g] * std::exp(power));
    const uint32_t r = rep[g];
    if (found && r == g && std::fabs(alpha - kAlphaMin) / kAlphaMin < rel_tol) found->push_back({0, g});
    if ((alpha < kAlphaMin) != flipped(0, r)) continue;
    if (found && prev_depth > 0.0 && rep[prev] != r &&
        std::fabs(depth[g] - prev_depth) / std::fabs(depth[g]) < depth_tol)
      found->push_back({2, prev});
    prev_depth = depth[g];
    prev = g;
    const double Tn = T * (1.0 - alpha);
    if (found && std::fabs(Tn - kTMin) / kTMin < rel_tol) found->push_back({1, g});
    if ((Tn < kTMin) != flipped(1, g)) break;
    for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
    T = Tn;
    last = k + 1;
  }
  C[3] = T;
  C[4] = last;
}
}  // namespace

int32_t orc_pixel_outcomes(int32_t len, const uint32_t* list, double px, double py, const double* xy,
                           const double* conic, const double* opacity, const double* rgb, const double* depth,
                           double rel_tol, double depth_tol, int32_t max_flip, int32_t max_out, double* out) {
  std::vector<Decision> found;
  double C[5];
  blend_pixel(len, list, px, py, xy, conic, opacity, rgb, depth, nullptr, 0, rel_tol, depth_tol, C, &found);
  if (max_out < 1) return -1;
  for (int ch = 0; ch < 5; ++ch) out[ch] = C[ch];
  const int m = (int)found.size();
  if (m > max_flip || (1 << m) > max_out) return -1;
  std::vector<Decision> sel;
  for (int mask = 1; mask < (1 << m); ++mask) {
    sel.clear();
    for (int b = 0; b < m; ++b)
      if (mask & (1 << b)) sel.push_back(found[b]);
    blend_pixel(len, list, px, py, xy, conic, opacity, rgb, depth, sel.data(), (int)sel.size(), rel_tol,
                depth_tol, C, nullptr);
    for (int ch = 0; ch < 5; ++ch) out[5 * mask + ch] = C[ch];
  }
  return 1 << m;
}

// The same blend without tiling: every pixel walks all visible Gaussians in
// (float32 depth, index) order and keeps those whose tile rectangle holds the
// pixel's tile.
void orc_composite_bruteforce(int32_t n, int32_t width, int32_t height, int32_t tile, const int32_t* radius,
                              const int32_t* rect, const double* xy, const double* conic,
                              const double* opacity, const double* rgb, const double* depth,
                              double* image, double* t_final) {
  std::vector<int> order;
  for (int g = 0; g < n; ++g)
    if (radius[g] > 0) order.push_back(g);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (float)depth[a] < (float)depth[b];
  });
#pragma omp parallel for schedule(dynamic, 16)
  for (int pix = 0; pix < width * height; ++pix) {
    const int px = pix % width, py = pix / width, tx = px / tile, ty = py / tile;
    double T = 1.0, C[3] = {0, 0, 0};
    const double cx = px + 0.5, cy = py + 0.5;
    for (int g : order) {
      const int32_t* rc = rect + 4 * (int64_t)g;
      if (tx < rc[0] || tx >= rc[2] || ty < rc[1] || ty >= rc[3]) continue;
      const double dx = xy[2 * g] - cx, dy = xy[2 * g + 1] - cy;
      const double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
      if (power > 0.0) continue;
      const double alpha = std::min(kAlphaMax, opacity[g] * std::exp(power));
      if (alpha < kAlphaMin) continue;
      const double Tn = T * (1.0 - alpha);
      if (Tn < kTMin) break;
      for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
      T = Tn;
    }
    for (int ch = 0; ch < 3; ++ch) image[3 * (int64_t)pix + ch] = C[ch];
    if (t_final) t_final[pix] = T;
  }
}

// Full frame: deform (or not, for the static 3D-GS special case), project, bin,
// sort and composite.  Returns the number of (tile, Gaussian) pairs.
int64_t orc_render(const orc_scene* s, const orc_camera* cam, double t, int32_t deform, int32_t tile,
                   double* image, double* t_final, int32_t* n_contrib, double* margin) {
  const int n = s->n;
  std::vector<double> X(3 * (int64_t)n), Q(4 * (int64_t)n), Sc(3 * (int64_t)n);
  if (deform) {
    orc_deform(s, t, X.data(), Q.data(), Sc.data());
  } else {
    for (int64_t i = 0; i < 3 * (int64_t)n; ++i) { X[i] = s->means[i]; Sc[i] = s->log_scales[i]; }
    for (int64_t i = 0; i < 4 * (int64_t)n; ++i) Q[i] = s->quats[i];
  }
  std::vector<double> xy(2 * (int64_t)n), conic(3 * (int64_t)n, 0.0), cov(3 * (int64_t)n, 0.0), op(n),
      rgb(3 * (int64_t)n, 0.0), depth(n), mg(n);
  std::vector<int32_t> radius(n), rect(4 * (int64_t)n);
  orc_projected P{xy.data(), conic.data(), cov.data(), op.data(), rgb.data(), depth.data(), radius.data(),
                  rect.data(), mg.data()};
  if (deform && s->color_heads) {  // App. B: the colour and opacity deformation
    const int K3 = 3 * (s->sh_degree + 1) * (s->sh_degree + 1);
    std::vector<double> shd((int64_t)n * K3), lgd(n);
    orc_appearance(s, t, shd.data(), lgd.data());
    orc_project_appearance(s, X.data(), Q.data(), Sc.data(), shd.data(), lgd.data(), cam, tile, &P);
  } else {
    orc_project(s, X.data(), Q.data(), Sc.data(), cam, tile, &P);
  }
  const int tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
  std::vector<uint32_t> dbits(n);
  for (int g = 0; g < n; ++g) {
    float f = (float)depth[g];
    std::memcpy(&dbits[g], &f, 4);
  }
  int64_t K = 0;
  for (int g = 0; g < n; ++g) K += (int64_t)(rect[4 * g + 2] - rect[4 * g]) * (rect[4 * g + 3] - rect[4 * g + 1]);
  std::vector<uint64_t> keys(K);
  std::vector<uint32_t> values(K), ranges(2 * (size_t)tiles_x * tiles_y);
  orc_bin_sort(n, dbits.data(), rect.data(), tiles_x, tiles_y, K, keys.data(), values.data(), ranges.data());
  orc_composite(cam->width, cam->height, tile, ranges.data(), values.data(), xy.data(), conic.data(), op.data(),
                rgb.data(), depth.data(), image, t_final, n_contrib, margin);
  return K;
}

}  // extern "C"

// ============================================================================
// Backward: the chain rule of every step above, in double precision, written
// step by step in reverse order (training, Sec. 4.3).  The loss is
// L = sum(dl_dimage * image); non-differentiable decisions (culling, tile
// rectangles, the 1/255 skip, the transmittance stop, the 0.99 clamp, ReLU and
// border clamps at their kinks) are held fixed.
// ============================================================================
namespace {

// Derivative of the real SH basis with respect to the direction components
// (x, y, z), differentiating each basis formula exactly as written above.
void sh_basis_grad(int degree, const double d[3], double dY[16][3]) {
  const double x = d[0], y = d[1], z = d[2];
  const double PI = 3.14159265358979323846;
  for (int k = 0; k < 16; ++k) dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
  if (degree < 1) return;
  const double c1 = std::sqrt(3.0 / (4.0 * PI));
  dY[1][1] = c1; dY[2][2] = c1; dY[3][0] = c1;
  if (degree < 2) return;
  const double a = 0.5 * std::sqrt(15.0 / PI), b = 0.25 * std::sqrt(5.0 / PI), dd = 0.25 * std::sqrt(15.0 / PI);
  dY[4][0] = a * y; dY[4][1] = a * x;
  dY[5][1] = a * z; dY[5][2] = a * y;
  dY[6][2] = 6.0 * b * z;
  dY[7][0] = a * z; dY[7][2] = a * x;
  dY[8][0] = 2.0 * dd * x; dY[8][1] = -2.0 * dd * y;
  if (degree < 3) return;
  const double e = 0.25 * std::sqrt(35.0 / (2.0 * PI)), f = 0.5 * std::sqrt(105.0 / PI);
  const double g = 0.25 * std::sqrt(21.0 / (2.0 * PI)), h = 0.25 * std::sqrt(7.0 / PI), m = 0.25 * std::sqrt(105.0 / PI);
  dY[9][0] = 6.0 * e * x * y; dY[9][1] = e * (3.0 * x * x - 3.0 * y * y);
  dY[10][0] = f * y * z; dY[10][1] = f * x * z; dY[10][2] = f * x * y;
  dY[11][1] = g * (5.0 * z * z - 1.0); dY[11][2] = 10.0 * g * y * z;
  dY[12][2] = h * (15.0 * z * z - 3.0);
  dY[13][0] = g * (5.0 * z * z - 1.0); dY[13][2] = 10.0 * g * x * z;
  dY[14][0] = 2.0 * m * x * z; dY[14][1] = -2.0 * m * y * z; dY[14][2] = m * (x * x - y * y);
  dY[15][0] = e * (3.0 * x * x - 3.0 * y * y); dY[15][1] = -6.0 * e * x * y;
}

// d R(q) / d q for the rotation matrix of quat_to_rot, q = (w, x, y, z).
void quat_rot_grad(const double q[4], double dR[4][3][3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  const double Rw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
  const double Rx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
  const double Ry[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
  const double Rz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      dR[0][i][j] = Rw[i][j]; dR[1][i][j] = Rx[i][j]; dR[2][i][j] = Ry[i][j]; dR[3][i][j] = Rz[i][j];
    }
}

}  // namespace

extern "C" int32_t orc_render_backward(const orc_scene* s, const orc_camera* cam, double t, int32_t deform,
                                       int32_t tile, const double* dl_dimage, orc_grads* G) {
  if (s->color_heads) return 3;  // the backward through the colour and opacity heads is not written
  const int n = s->n, W = s->mlp_width, L = s->n_levels, h = s->feat_dim, hin = h * L;
  const int K = (s->sh_degree + 1) * (s->sh_degree + 1);
  const MlpLayout Lo = mlp_layout(s);
  // ---------------------------------------------------------------- forward, keeping what the backward needs
  std::vector<double> X(3 * (int64_t)n), Q(4 * (int64_t)n), Sc(3 * (int64_t)n);
  std::vector<double> fh((int64_t)n * hin, 0.0), a1((int64_t)n * W), fd((int64_t)n * W), hid((int64_t)n * 3 * W);
  std::vector<double> xyz(3 * (int64_t)n);
  for (int64_t i = 0; i < 3 * (int64_t)n; ++i) xyz[i] = s->means[i];
  if (deform) {
    orc_features(s, xyz.data(), n, t, fh.data());
    for (int g = 0; g < n; ++g) {
      double* A1 = &a1[(int64_t)g * W];
      double* FD = &fd[(int64_t)g * W];
      linear(s, Lo, 0, &fh[(int64_t)g * hin], A1);
      for (int o = 0; o < W; ++o) A1[o] = relu(A1[o]);
      linear(s, Lo, 1, A1, FD);
      for (int o = 0; o < W; ++o) FD[o] = relu(FD[o]);
      double out[4];
      int col = 0;
      for (int hd = 0; hd < 3; ++hd) {
        double* HID = &hid[((int64_t)g * 3 + hd) * W];
        linear(s, Lo, 2 + 2 * hd, FD, HID);
        for (int o = 0; o < W; ++o) HID[o] = relu(HID[o]);
        linear(s, Lo, 3 + 2 * hd, HID, out);
        for (int o = 0; o < kHeadOut[hd]; ++o) {
          double base = col + o < 3 ? s->means[3 * (int64_t)g + col + o]
                        : col + o < 7 ? s->quats[4 * (int64_t)g + col + o - 3]
                                      : s->log_scales[3 * (int64_t)g + col + o - 7];
          double* dst = col + o < 3 ? &X[3 * (int64_t)g + col + o]
                        : col + o < 7 ? &Q[4 * (int64_t)g + col + o - 3]
                                      : &Sc[3 * (int64_t)g + col + o - 7];
          *dst = base + out[o];
        }
        col += kHeadOut[hd];
      }
    }
  } else {
    for (int64_t i = 0; i < 3 * (int64_t)n; ++i) { X[i] = s->means[i]; Sc[i] = s->log_scales[i]; }
    for (int64_t i = 0; i < 4 * (int64_t)n; ++i) Q[i] = s->quats[i];
  }
  std::vector<double> xy(2 * (int64_t)n, 0.0), conic(3 * (int64_t)n, 0.0), cov(3 * (int64_t)n, 0.0), op(n),
      rgb(3 * (int64_t)n, 0.0), depth(n), mg(n);
  std::vector<int32_t> radius(n), rect(4 * (int64_t)n);
  orc_projected P{xy.data(), conic.data(), cov.data(), op.data(), rgb.data(), depth.data(), radius.data(),
                  rect.data(), mg.data()};
  orc_project(s, X.data(), Q.data(), Sc.data(), cam, tile, &P);
  const int tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
  std::vector<uint32_t> dbits(n);
  int64_t KP = 0;
  for (int g = 0; g < n; ++g) {
    float f = (float)depth[g];
    std::memcpy(&dbits[g], &f, 4);
    KP += (int64_t)(rect[4 * g + 2] - rect[4 * g]) * (rect[4 * g + 3] - rect[4 * g + 1]);
  }
  std::vector<uint64_t> keys(std::max<int64_t>(KP, 1));
  std::vector<uint32_t> values(std::max<int64_t>(KP, 1)), ranges(2 * (size_t)tiles_x * tiles_y);
  orc_bin_sort(n, dbits.data(), rect.data(), tiles_x, tiles_y, KP, keys.data(), values.data(), ranges.data());
  const int npix = cam->width * cam->height;
  std::vector<double> img(3 * (size_t)npix), Tfin(npix), marg(npix);
  std::vector<int32_t> ncon(npix);
  orc_composite(cam->width, cam->height, tile, ranges.data(), values.data(), xy.data(), conic.data(), op.data(),
                rgb.data(), depth.data(), img.data(), Tfin.data(), ncon.data(), marg.data());

  // ---------------------------------------------------------------- Eq. 4 backward, per pixel, back to front
  std::vector<double> g_xy(2 * (int64_t)n, 0.0), g_conic(3 * (int64_t)n, 0.0), g_op(n, 0.0),
      g_rgb(3 * (int64_t)n, 0.0);
  for (int pix = 0; pix < npix; ++pix) {
    const int px = pix % cam->width, py = pix / cam->width;
    const int tid = (py / tile) * tiles_x + (px / tile);
    const uint32_t start = ranges[2 * tid];
    const double cx = px + 0.5, cy = py + 0.5;
    const double* dC = dl_dimage + 3 * (int64_t)pix;
    double T = Tfin[pix];          // transmittance after the last blended term
    double behind[3] = {0, 0, 0};  // sum of c_j a_j T_j over the terms behind the current one
    for (int k = ncon[pix] - 1; k >= 0; --k) {
      const uint32_t g = values[start + k];
      const double dx = xy[2 * g] - cx, dy = xy[2 * g + 1] - cy;
      const double A = conic[3 * g], B = conic[3 * g + 1], Cc = conic[3 * g + 2];
      const double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
      if (power > 0.0) continue;
      const double Gv = std::exp(power);
      const double a_raw = op[g] * Gv;
      const double alpha = std::min(kAlphaMax, a_raw);
      if (alpha < kAlphaMin) continue;
      const double Ti = T / (1.0 - alpha);  // transmittance in front of this term
      double dL_dalpha = 0.0;
      for (int ch = 0; ch < 3; ++ch) {
        g_rgb[3 * g + ch] += dC[ch] * alpha * Ti;
        dL_dalpha += dC[ch] * (rgb[3 * g + ch] * Ti - behind[ch] / (1.0 - alpha));
      }
      for (int ch = 0; ch < 3; ++ch) behind[ch] += rgb[3 * g + ch] * alpha * Ti;
      T = Ti;
      if (a_raw > kAlphaMax) continue;  // clamped: no gradient to opacity or shape
      g_op[g] += dL_dalpha * Gv;
      const double dpow = dL_dalpha * op[g] * Gv;
      g_xy[2 * g] += dpow * (-(A * dx + B * dy));
      g_xy[2 * g + 1] += dpow * (-(Cc * dy + B * dx));
      g_conic[3 * g] += dpow * (-0.5 * dx * dx);
      g_conic[3 * g + 1] += dpow * (-dx * dy);
      g_conic[3 * g + 2] += dpow * (-0.5 * dy * dy);
    }
  }

  if (G->xy)
    for (int64_t i = 0; i < 2 * (int64_t)n; ++i) G->xy[i] += g_xy[i];

  // ---------------------------------------------------------------- Eq. 2 / Eq. 3 / SH backward, per Gaussian
  const double* M = cam->world_to_cam;
  double Rc[3][3], tc[3], campos[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) Rc[r][c] = M[4 * r + c];
    tc[r] = M[4 * r + 3];
  }
  for (int c = 0; c < 3; ++c) campos[c] = -(Rc[0][c] * tc[0] + Rc[1][c] * tc[1] + Rc[2][c] * tc[2]);
  const double limx = kGuard * cam->width / (2.0 * cam->fx), limy = kGuard * cam->height / (2.0 * cam->fy);
  std::vector<double> gX(3 * (int64_t)n, 0.0), gQ(4 * (int64_t)n, 0.0), gS(3 * (int64_t)n, 0.0);
  for (int g = 0; g < n; ++g) {
    if (G->opacity_logits) G->opacity_logits[g] += g_op[g] * op[g] * (1.0 - op[g]);
    if (radius[g] == 0) continue;
    const double* Xg = &X[3 * (int64_t)g];
    // colour
    double v[3], vn = 0;
    for (int k = 0; k < 3; ++k) { v[k] = Xg[k] - campos[k]; vn += v[k] * v[k]; }
    vn = std::sqrt(vn);
    double dir[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
    double Y[16], dY[16][3];
    sh_basis(s->sh_degree, dir, Y);
    sh_basis_grad(s->sh_degree, dir, dY);
    double g_dir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
      double raw = 0.5;
      for (int k = 0; k < K; ++k) raw += Y[k] * (double)s->sh[((int64_t)g * K + k) * 3 + ch];
      if (!(raw > 0.0)) continue;  // clamped at 0
      const double gr = g_rgb[3 * g + ch];
      for (int k = 0; k < K; ++k) {
        if (G->sh) G->sh[((int64_t)g * K + k) * 3 + ch] += gr * Y[k];
        for (int a = 0; a < 3; ++a) g_dir[a] += gr * (double)s->sh[((int64_t)g * K + k) * 3 + ch] * dY[k][a];
      }
    }
    const double dd = dir[0] * g_dir[0] + dir[1] * g_dir[1] + dir[2] * g_dir[2];
    for (int a = 0; a < 3; ++a) gX[3 * (int64_t)g + a] += (g_dir[a] - dir[a] * dd) / vn;
    // camera-space mean
    double p[3];
    for (int r = 0; r < 3; ++r) p[r] = Rc[r][0] * Xg[0] + Rc[r][1] * Xg[1] + Rc[r][2] * Xg[2] + tc[r];
    double gp[3] = {0, 0, 0};
    // mean2D: u = fx px/pz + cx, v = fy py/pz + cy
    gp[0] += g_xy[2 * g] * cam->fx / p[2];
    gp[1] += g_xy[2 * g + 1] * cam->fy / p[2];
    gp[2] += -g_xy[2 * g] * cam->fx * p[0] / (p[2] * p[2]) - g_xy[2 * g + 1] * cam->fy * p[1] / (p[2] * p[2]);
    // conic = Sigma2D^-1: dL/dSigma2D = -K G_K K with G_K the symmetric gradient of K
    const double ka = conic[3 * g], kb = conic[3 * g + 1], kc = conic[3 * g + 2];
    const double Km[2][2] = {{ka, kb}, {kb, kc}};
    const double GK[2][2] = {{g_conic[3 * g], 0.5 * g_conic[3 * g + 1]}, {0.5 * g_conic[3 * g + 1], g_conic[3 * g + 2]}};
    double GS2[2][2];  // dL/dSigma2D (symmetric matrix gradient)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double acc = 0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) acc += Km[i][a] * GK[a][b] * Km[b][j];
        GS2[i][j] = -acc;
      }
    // Sigma2D = T Sigma T^T + 0.3 I, T = J W, Sigma = (R S)(R S)^T
    double qv[4], qn = 0;
    for (int k = 0; k < 4; ++k) { qv[k] = Q[4 * (int64_t)g + k]; qn += qv[k] * qv[k]; }
    qn = std::sqrt(qn);
    double qh[4] = {qv[0] / qn, qv[1] / qn, qv[2] / qn, qv[3] / qn};
    double R[3][3];
    quat_to_rot(qh, R);
    double sc[3];
    for (int k = 0; k < 3; ++k) sc[k] = std::exp(Sc[3 * (int64_t)g + k]);
    double RS[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) RS[i][j] = R[i][j] * sc[j];
    const bool clx = std::fabs(p[0] / p[2]) > limx, cly = std::fabs(p[1] / p[2]) > limy;
    const double rx = std::min(limx, std::max(-limx, p[0] / p[2])), ry = std::min(limy, std::max(-limy, p[1] / p[2]));
    double J[2][3] = {{cam->fx / p[2], 0.0, -cam->fx * rx / p[2]}, {0.0, cam->fy / p[2], -cam->fy * ry / p[2]}};
    double T[2][3];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) T[i][j] = J[i][0] * Rc[0][j] + J[i][1] * Rc[1][j] + J[i][2] * Rc[2][j];
    double Am[2][3];  // A = T R S
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) Am[i][j] = T[i][0] * RS[0][j] + T[i][1] * RS[1][j] + T[i][2] * RS[2][j];
    double gA[2][3];  // dL/dA = (GS2 + GS2^T) A = 2 GS2 A
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) gA[i][j] = 2.0 * (GS2[i][0] * Am[0][j] + GS2[i][1] * Am[1][j]);
    double gT[2][3], gRS[3][3];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) gT[i][j] = gA[i][0] * RS[j][0] + gA[i][1] * RS[j][1] + gA[i][2] * RS[j][2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gRS[i][j] = T[0][i] * gA[0][j] + T[1][i] * gA[1][j];
    double gR[3][3], gsc[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        gR[i][j] = gRS[i][j] * sc[j];
        gsc[j] += gRS[i][j] * R[i][j];
      }
    for (int k = 0; k < 3; ++k) gS[3 * (int64_t)g + k] += gsc[k] * sc[k];
    double dR[4][3][3], gqh[4] = {0, 0, 0, 0};
    quat_rot_grad(qh, dR);
    for (int c = 0; c < 4; ++c)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) gqh[c] += gR[i][j] * dR[c][i][j];
    const double qd = qh[0] * gqh[0] + qh[1] * gqh[1] + qh[2] * gqh[2] + qh[3] * gqh[3];
    for (int c = 0; c < 4; ++c) gQ[4 * (int64_t)g + c] += (gqh[c] - qh[c] * qd) / qn;
    // T = J W: dL/dJ = dL/dT W^T
    double gJ[2][3];
    for (int i = 0; i < 2; ++i)
      for (int a = 0; a < 3; ++a) gJ[i][a] = gT[i][0] * Rc[a][0] + gT[i][1] * Rc[a][1] + gT[i][2] * Rc[a][2];
    const double pz = p[2], pz2 = pz * pz;
    gp[2] += gJ[0][0] * (-cam->fx / pz2) + gJ[1][1] * (-cam->fy / pz2);
    if (!clx) {  // J02 = -fx px / pz^2
      gp[0] += gJ[0][2] * (-cam->fx / pz2);
      gp[2] += gJ[0][2] * (2.0 * cam->fx * p[0] / (pz2 * pz));
    } else {     // J02 = -fx rx / pz with rx held at the guard band
      gp[2] += gJ[0][2] * (cam->fx * rx / pz2);
    }
    if (!cly) {
      gp[1] += gJ[1][2] * (-cam->fy / pz2);
      gp[2] += gJ[1][2] * (2.0 * cam->fy * p[1] / (pz2 * pz));
    } else {
      gp[2] += gJ[1][2] * (cam->fy * ry / pz2);
    }
    // p = W X' + t
    for (int a = 0; a < 3; ++a) gX[3 * (int64_t)g + a] += Rc[0][a] * gp[0] + Rc[1][a] * gp[1] + Rc[2][a] * gp[2];
  }

  // ---------------------------------------------------------------- Eq. 6: X' = X + dX, r' = r + dr, s' = s + ds
  for (int64_t i = 0; i < 3 * (int64_t)n; ++i) {
    if (G->means) G->means[i] += gX[i];
    if (G->log_scales) G->log_scales[i] += gS[i];
  }
  for (int64_t i = 0; i < 4 * (int64_t)n; ++i)
    if (G->quats) G->quats[i] += gQ[i];
  if (!deform) return 0;

  // ---------------------------------------------------------------- heads, phi_d and Eq. 5 backward
  for (int g = 0; g < n; ++g) {
    const double* FD = &fd[(int64_t)g * W];
    const double* A1 = &a1[(int64_t)g * W];
    std::vector<double> gfd(W, 0.0), ga1(W, 0.0), gfh(hin, 0.0);
    int col = 0;
    for (int hd = 0; hd < 3; ++hd) {
      const double* HID = &hid[((int64_t)g * 3 + hd) * W];
      const int ko = 3 + 2 * hd, kh = 2 + 2 * hd;
      std::vector<double> ghid(W, 0.0);
      for (int o = 0; o < kHeadOut[hd]; ++o) {
        const double gout = col + o < 3 ? gX[3 * (int64_t)g + col + o]
                            : col + o < 7 ? gQ[4 * (int64_t)g + col + o - 3]
                                          : gS[3 * (int64_t)g + col + o - 7];
        if (G->mlp) {
          G->mlp[Lo.b[ko] + o] += gout;
          for (int i = 0; i < W; ++i) G->mlp[Lo.w[ko] + (int64_t)o * W + i] += gout * HID[i];
        }
        for (int i = 0; i < W; ++i) ghid[i] += gout * (double)s->mlp[Lo.w[ko] + (int64_t)o * W + i];
      }
      col += kHeadOut[hd];
      for (int o = 0; o < W; ++o) {
        const double gpre = HID[o] > 0.0 ? ghid[o] : 0.0;
        if (G->mlp) {
          G->mlp[Lo.b[kh] + o] += gpre;
          for (int i = 0; i < W; ++i) G->mlp[Lo.w[kh] + (int64_t)o * W + i] += gpre * FD[i];
        }
        for (int i = 0; i < W; ++i) gfd[i] += gpre * (double)s->mlp[Lo.w[kh] + (int64_t)o * W + i];
      }
    }
    for (int o = 0; o < W; ++o) {
      const double gpre = FD[o] > 0.0 ? gfd[o] : 0.0;
      if (G->mlp) {
        G->mlp[Lo.b[1] + o] += gpre;
        for (int i = 0; i < W; ++i) G->mlp[Lo.w[1] + (int64_t)o * W + i] += gpre * A1[i];
      }
      for (int i = 0; i < W; ++i) ga1[i] += gpre * (double)s->mlp[Lo.w[1] + (int64_t)o * W + i];
    }
    const double* FH = &fh[(int64_t)g * hin];
    for (int o = 0; o < W; ++o) {
      const double gpre = A1[o] > 0.0 ? ga1[o] : 0.0;
      if (G->mlp) {
        G->mlp[Lo.b[0] + o] += gpre;
        for (int i = 0; i < hin; ++i) G->mlp[Lo.w[0] + (int64_t)o * hin + i] += gpre * FH[i];
      }
      for (int i = 0; i < hin; ++i) gfh[i] += gpre * (double)s->mlp[Lo.w[0] + (int64_t)o * hin + i];
    }
    // Test support: |J|^T 1, the sensitivity of f_h's gradient to a unit error in each of
    // this Gaussian's ten output gradients (dX', dr', ds'), through |W| with the same
    // ReLU masks; propagated to the planes below as planes_sens.
    std::vector<double> sfh;
    if (G->planes_sens) {
      std::vector<double> sfd(W, 0.0), sa1(W, 0.0);
      sfh.assign(hin, 0.0);
      for (int hd = 0; hd < 3; ++hd) {
        const double* HID = &hid[((int64_t)g * 3 + hd) * W];
        const int ko = 3 + 2 * hd, kh = 2 + 2 * hd;
        std::vector<double> shid(W, 0.0);
        for (int o = 0; o < kHeadOut[hd]; ++o)
          for (int i = 0; i < W; ++i) shid[i] += std::fabs((double)s->mlp[Lo.w[ko] + (int64_t)o * W + i]);
        for (int o = 0; o < W; ++o)
          if (HID[o] > 0.0)
            for (int i = 0; i < W; ++i) sfd[i] += shid[o] * std::fabs((double)s->mlp[Lo.w[kh] + (int64_t)o * W + i]);
      }
      for (int o = 0; o < W; ++o)
        if (FD[o] > 0.0)
          for (int i = 0; i < W; ++i) sa1[i] += sfd[o] * std::fabs((double)s->mlp[Lo.w[1] + (int64_t)o * W + i]);
      for (int o = 0; o < W; ++o)
        if (A1[o] > 0.0)
          for (int i = 0; i < hin; ++i) sfh[i] += sa1[o] * std::fabs((double)s->mlp[Lo.w[0] + (int64_t)o * hin + i]);
    }
    // Eq. 5: f_l[c] = prod_p v_p[c]; v_p = bilinear(R_{l,p}) at (c_a, c_b)
    double c4[4];
    normalise(s, &xyz[3 * (int64_t)g], t, c4);
    for (int l = 0; l < L; ++l) {
      std::vector<std::vector<double>> vp(6, std::vector<double>(h));
      int i0[6], j0[6], Ra[6], Rb[6];
      double fa[6], fb[6], da[6], db[6];
      for (int p = 0; p < 6; ++p) {
        Ra[p] = plane_res(s, l, kPlaneAxes[p][0]);
        Rb[p] = plane_res(s, l, kPlaneAxes[p][1]);
        axis_setup(c4[kPlaneAxes[p][0]], Ra[p], &i0[p], &fa[p], &da[p]);
        axis_setup(c4[kPlaneAxes[p][1]], Rb[p], &j0[p], &fb[p], &db[p]);
        orc_plane_sample(s, l, p, c4[kPlaneAxes[p][0]], c4[kPlaneAxes[p][1]], vp[p].data());
      }
      for (int p = 0; p < 6; ++p) {
        const int64_t off = plane_offset(s, l, p);
        const float* Pl = s->planes + off;
        for (int c = 0; c < h; ++c) {
          double others = 1.0;
          for (int q = 0; q < 6; ++q)
            if (q != p) others *= vp[q][c];
          const double gv = gfh[l * h + c] * others;
          const int64_t e00 = ((int64_t)j0[p] * Ra[p] + i0[p]) * h + c, e10 = e00 + h;
          const int64_t e01 = e00 + (int64_t)Ra[p] * h, e11 = e01 + h;
          if (G->planes) {
            G->planes[off + e00] += gv * (1 - fa[p]) * (1 - fb[p]);
            G->planes[off + e10] += gv * fa[p] * (1 - fb[p]);
            G->planes[off + e01] += gv * (1 - fa[p]) * fb[p];
            G->planes[off + e11] += gv * fa[p] * fb[p];
          }
          if (G->planes_sens) {
            const double sv = sfh[l * h + c] * std::fabs(others);
            G->planes_sens[off + e00] += sv * (1 - fa[p]) * (1 - fb[p]);
            G->planes_sens[off + e10] += sv * fa[p] * (1 - fb[p]);
            G->planes_sens[off + e01] += sv * (1 - fa[p]) * fb[p];
            G->planes_sens[off + e11] += sv * fa[p] * fb[p];
          }
          if (G->planes_abs) {  // magnitudes of the same terms (test support: conditioning of the sums)
            G->planes_abs[off + e00] += std::fabs(gv * (1 - fa[p]) * (1 - fb[p]));
            G->planes_abs[off + e10] += std::fabs(gv * fa[p] * (1 - fb[p]));
            G->planes_abs[off + e01] += std::fabs(gv * (1 - fa[p]) * fb[p]);
            G->planes_abs[off + e11] += std::fabs(gv * fa[p] * fb[p]);
          }
          const double dv_dfa = (1 - fb[p]) * ((double)Pl[e10] - Pl[e00]) + fb[p] * ((double)Pl[e11] - Pl[e01]);
          const double dv_dfb = (1 - fa[p]) * ((double)Pl[e01] - Pl[e00]) + fa[p] * ((double)Pl[e11] - Pl[e10]);
          const int a = kPlaneAxes[p][0], b = kPlaneAxes[p][1];
          // the canonical mean moves the sampling point (time has no gradient)
          if (G->means && a < 3)
            G->means[3 * (int64_t)g + a] += gv * dv_dfa * da[p] * 2.0 / (s->aabb_max[a] - s->aabb_min[a]);
          if (G->means && b < 3)
            G->means[3 * (int64_t)g + b] += gv * dv_dfb * db[p] * 2.0 / (s->aabb_max[b] - s->aabb_min[b]);
        }
      }
    }
  }
  return 0;
}

// ============================================================================
// Training step (Sec. 4.3, App. A): the loss L = |I^ - I| + L_tv and one Adam
// update of the parameters with learning rates decayed over the training run.
// ============================================================================
extern "C" {

// L1 colour loss: the mean absolute difference over every pixel and channel
// (reading of |I^ - I|), and its gradient sign(I^ - I) / count (0 where equal).
double orc_l1_loss(int64_t count, const double* image, const double* target, double* grad) {
  double sum = 0.0;
  for (int64_t i = 0; i < count; ++i) {
    const double d = image[i] - target[i];
    sum += std::fabs(d);
    if (grad) grad[i] = d > 0.0 ? 1.0 / (double)count : (d < 0.0 ? -1.0 / (double)count : 0.0);
  }
  return count > 0 ? sum / (double)count : 0.0;
}

// Grid total-variation loss over the HexPlane (reading of L_tv, which the paper
// names without a formula): for every level and every one of the six planes, the
// mean over all neighbouring cell pairs along each of the plane's two axes of the
// squared feature difference (every channel), the two axes' means added, summed
// over planes and levels, times `weight`.  grad (if non-null) receives the
// gradient with respect to every plane value (planes layout).  Returns the loss.
double orc_tv_loss(const orc_scene* s, double weight, double* grad) {
  const int h = s->feat_dim;
  double total = 0.0;
  for (int l = 0; l < s->n_levels; ++l) {
    for (int p = 0; p < 6; ++p) {
      const int Ra = plane_res(s, l, kPlaneAxes[p][0]);
      const int Rb = plane_res(s, l, kPlaneAxes[p][1]);
      const int64_t off = plane_offset(s, l, p);
      const float* P = s->planes + off;
      auto at = [&](int b, int a, int c) { return (double)P[((int64_t)b * Ra + a) * h + c]; };
      const double na = (double)Rb * (Ra - 1) * h, nb = (double)(Rb - 1) * Ra * h;
      double sa = 0.0, sb = 0.0;
      for (int b = 0; b < Rb; ++b)
        for (int a = 0; a < Ra; ++a)
          for (int c = 0; c < h; ++c) {
            if (a + 1 < Ra) {
              const double d = at(b, a + 1, c) - at(b, a, c);
              sa += d * d;
              if (grad) {
                grad[off + ((int64_t)b * Ra + a + 1) * h + c] += weight * 2.0 * d / na;
                grad[off + ((int64_t)b * Ra + a) * h + c] -= weight * 2.0 * d / na;
              }
            }
            if (b + 1 < Rb) {
              const double d = at(b + 1, a, c) - at(b, a, c);
              sb += d * d;
              if (grad) {
                grad[off + ((int64_t)(b + 1) * Ra + a) * h + c] += weight * 2.0 * d / nb;
                grad[off + ((int64_t)b * Ra + a) * h + c] -= weight * 2.0 * d / nb;
              }
            }
          }
      total += sa / na + sb / nb;
    }
  }
  return weight * total;
}

// Learning rate of step k (0-based) of a run of `total` steps, decayed from lr0 to
// lr1 (App. A: "decayed to ... at the end of training"); reading: log-linear
// (exponential) interpolation, lr1 from step `total` on.
double orc_lr(double lr0, double lr1, int64_t k, int64_t total) {
  if (total <= 0 || lr0 <= 0.0 || lr1 <= 0.0) return lr0;
  const double f = std::min(1.0, (double)k / (double)total);
  return std::exp((1.0 - f) * std::log(lr0) + f * std::log(lr1));
}

// One Adam step (bias-corrected first and second moments; step = 1 for the first
// update) of `count` parameters with gradient g at learning rate lr.
void orc_adam_step(int64_t count, double* param, const double* g, double* m, double* v, double lr, double beta1,
                   double beta2, double eps, int64_t step) {
  const double c1 = 1.0 - std::pow(beta1, (double)step), c2 = 1.0 - std::pow(beta2, (double)step);
  for (int64_t i = 0; i < count; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    param[i] -= lr * mh / (std::sqrt(vh) + eps);
  }
}

// Adaptive density control (App. A keeps the densification and pruning of 3D
// Gaussian splatting and stops the growth late in training).  Written out as
// its definition: the Gaussians whose mean view-space gradient is at least the
// threshold are densified -- copied when small (largest log-scale at or below
// split_log_scale), replaced by two children drawn from N(mu, Sigma) with the
// scales divided by 1.6 when large -- and every Gaussian whose opacity logit is
// below prune_logit is removed together with whatever it would have produced.
// The three decisions are taken in float32 on the float32 inputs.
// Output order: the kept Gaussians, the copies, the first children, the second
// children, each in source order; src/kind give each output's source Gaussian
// and 0 kept, 1 copy, 2 first child, 3 second child.
int64_t orc_densify(const orc_scene* s, const float* grad_sum, const float* visible, const float* normals,
                    float grad_threshold, float split_log_scale, float prune_logit, int64_t cap, int64_t* src,
                    int32_t* kind, double* means, double* log_scales, double* quats, double* opacity_logits,
                    double* sh) {
  const int64_t n = s->n, K = (int64_t)(s->sh_degree + 1) * (s->sh_degree + 1);
  std::vector<int> cls(n);  // 0 removed, 1 kept, 2 kept and copied, 3 split
  for (int64_t i = 0; i < n; ++i) {
    const float avg = visible[i] > 0.f ? grad_sum[i] / visible[i] : 0.f;
    const bool selected = avg >= grad_threshold;
    float smax = s->log_scales[3 * i];
    for (int k = 1; k < 3; ++k) smax = std::max(smax, s->log_scales[3 * i + k]);
    const bool large = smax > split_log_scale;
    if (s->opacity_logits[i] < prune_logit) cls[i] = 0;
    else if (!selected) cls[i] = 1;
    else cls[i] = large ? 3 : 2;
  }
  std::vector<std::pair<int64_t, int>> out;
  for (int64_t i = 0; i < n; ++i)
    if (cls[i] == 1 || cls[i] == 2) out.push_back({i, 0});
  for (int64_t i = 0; i < n; ++i)
    if (cls[i] == 2) out.push_back({i, 1});
  for (int c = 0; c < 2; ++c)
    for (int64_t i = 0; i < n; ++i)
      if (cls[i] == 3) out.push_back({i, 2 + c});
  if ((int64_t)out.size() > cap) return -1;
  const double shrink = std::log(1.6);
  for (size_t o = 0; o < out.size(); ++o) {
    const int64_t i = out[o].first;
    const int kd = out[o].second;
    src[o] = i;
    kind[o] = kd;
    for (int k = 0; k < 3; ++k) {
      means[3 * o + k] = s->means[3 * i + k];
      log_scales[3 * o + k] = s->log_scales[3 * i + k];
    }
    for (int k = 0; k < 4; ++k) quats[4 * o + k] = s->quats[4 * i + k];
    opacity_logits[o] = s->opacity_logits[i];
    for (int64_t k = 0; k < 3 * K; ++k) sh[3 * K * o + k] = s->sh[3 * K * i + k];
    if (kd >= 2) {
      // child = mu + R S z, z ~ N(0, I): a draw from N(mu, R S S^T R^T) (Eq. 2)
      double q[4], qn = 0.0, R[3][3];
      for (int k = 0; k < 4; ++k) { q[k] = s->quats[4 * i + k]; qn += q[k] * q[k]; }
      qn = std::sqrt(qn);
      for (int k = 0; k < 4; ++k) q[k] /= qn;
      quat_to_rot(q, R);
      const float* z = normals + 6 * i + 3 * (kd - 2);
      double sz[3];
      for (int k = 0; k < 3; ++k) sz[k] = std::exp((double)s->log_scales[3 * i + k]) * (double)z[k];
      for (int r = 0; r < 3; ++r) means[3 * o + r] += R[r][0] * sz[0] + R[r][1] * sz[1] + R[r][2] * sz[2];
      for (int k = 0; k < 3; ++k) log_scales[3 * o + k] -= shrink;
    }
  }
  return (int64_t)out.size();
}

}  // extern "C"
