// gs2d oracle -- plain, slow, FP64 CPU reference of the differentiable
// 2D Gaussian surfel rasterizer of 2DGS-SLAM (Sec. III-A and III-B).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file;
// only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
// It shares no code, header or constant with the CUDA implementation.
//
// What it computes, per pixel p with centre (x, y) = (i + 0.5, j + 0.5):
//   * the ray  z * r(p),  r = ((x - cx)/fx, (y - cy)/fy, 1)   (Eq. homo: the
//     pixel ray x = (xz, yz, z, 1) hits the splat at camera depth z);
//   * for every surfel, the camera-space splat H_c = T_cw H (Eq. hc), i.e.
//     columns s_u t_uc, s_v t_vc and centre mu_c;
//   * the ray/splat intersection (u, v, z) from
//         mu_c + u (s_u t_uc) + v (s_v t_vc) = z r
//     solved by Cramer's rule (the literal ray-plane intersection that
//     Sec. III-A describes; the CUDA side uses a different formulation);
//   * G(u, v) = exp(-(u^2 + v^2) / 2) (Sec. III-A), a = alpha G;
//   * front-to-back alpha blending of colour, depth z, normal t_nc and
//     opacity (Eq. alpha_blending), surfels ordered by (centre depth, id).
// Readings of points the paper leaves open:
//   * a = min(alpha G, alpha_max); a surfel is skipped if a < alpha_min or
//     u^2+v^2 > cutoff_r2; blending stops before the surfel whose inclusion
//     would drive the transmittance below t_min.  "exact" mode disables the
//     clamp, the skip, the cutoff and the stop (used for identities and FD).
//   * intersections need z > near and the surfel centre mu_c.z > near;
//     a singular Cramer system (ray parallel to the splat plane) is skipped.
//   * depth output is the literal blended D = sum w z, opacity O = sum w.
// Backward: reverse-mode derivative of the above, by hand, to the surfel
// parameters (mu, raw quaternion, scales, opacity, colour) and to the pose
// tangent tau = (rho, theta) of the left perturbation Exp(tau) o T_cw
// (Eq. derivatives and the manifold derivative of Sec. III-B).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct V3 {
  double x, y, z;
};
inline V3 mk(double x, double y, double z) { return V3{x, y, z}; }
inline V3 operator+(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
inline V3 operator-(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
inline V3 operator*(double s, V3 a) { return mk(s * a.x, s * a.y, s * a.z); }
inline V3 operator-(V3 a) { return mk(-a.x, -a.y, -a.z); }
inline V3& operator+=(V3& a, V3 b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  return a;
}
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// determinant of the 3x3 matrix with columns a, b, c
inline double det3(V3 a, V3 b, V3 c) { return dot(a, cross(b, c)); }

struct Cam {
  double fx, fy, cx, cy, near_z;
  int W, H;
};
struct Rule {
  double alpha_min, alpha_max, t_min, cutoff_r2;
  int exact;
};

// rotation matrix of a unit quaternion (w, x, y, z); R[r][c]
void quat_matrix(const double q[4], double R[3][3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z);
  R[0][1] = 2 * (x * y - w * z);
  R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);
  R[1][1] = 1 - 2 * (x * x + z * z);
  R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);
  R[2][1] = 2 * (y * z + w * x);
  R[2][2] = 1 - 2 * (x * x + y * y);
}

// d R[r][c] / d q_k for the unit-quaternion matrix above
void quat_matrix_jac(const double q[4], double J[3][3][4]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  const double t[3][3][4] = {
      {{0, 0, -4 * y, -4 * z}, {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x}},
      {{2 * z, 2 * y, 2 * x, 2 * w}, {0, -4 * x, 0, -4 * z}, {-2 * x, -2 * w, 2 * z, 2 * y}},
      {{-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y}, {0, -4 * x, -4 * y, 0}}};
  std::memcpy(J, t, sizeof(t));
}

V3 matvec(const double M[9], V3 v) {
  return mk(M[0] * v.x + M[1] * v.y + M[2] * v.z, M[3] * v.x + M[4] * v.y + M[5] * v.z,
            M[6] * v.x + M[7] * v.y + M[8] * v.z);
}
V3 matTvec(const double M[9], V3 v) {
  return mk(M[0] * v.x + M[3] * v.y + M[6] * v.z, M[1] * v.x + M[4] * v.y + M[7] * v.z,
            M[2] * v.x + M[5] * v.y + M[8] * v.z);
}

// One surfel expressed in camera space (Eq. hc).
struct CamSurfel {
  double qn[4], qlen;   // normalised quaternion and the raw quaternion's length
  V3 tu, tv, tn;        // world-space columns of R
  V3 mu_c, tu_c, tv_c, tn_c;
  V3 m_u, m_v;          // s_u t_uc, s_v t_vc
  double su, sv, alpha;
  V3 col;
};

CamSurfel make_cam_surfel(int i, const double* mu, const double* quat, const double* scale,
                          const double* opacity, const double* rgb, const double* Rcw,
                          const double* tcw) {
  CamSurfel s;
  const double* q = quat + 4 * i;
  s.qlen = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) s.qn[k] = q[k] / s.qlen;
  double R[3][3];
  quat_matrix(s.qn, R);
  s.tu = mk(R[0][0], R[1][0], R[2][0]);
  s.tv = mk(R[0][1], R[1][1], R[2][1]);
  s.tn = mk(R[0][2], R[1][2], R[2][2]);
  const V3 muw = mk(mu[3 * i], mu[3 * i + 1], mu[3 * i + 2]);
  s.mu_c = matvec(Rcw, muw) + mk(tcw[0], tcw[1], tcw[2]);
  s.tu_c = matvec(Rcw, s.tu);
  s.tv_c = matvec(Rcw, s.tv);
  s.tn_c = matvec(Rcw, s.tn);
  s.su = scale[2 * i];
  s.sv = scale[2 * i + 1];
  s.m_u = s.su * s.tu_c;
  s.m_v = s.sv * s.tv_c;
  s.alpha = opacity[i];
  s.col = mk(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
  return s;
}

// Cramer solve of  u m_u + v m_v - z r = -mu_c.
struct Hit {
  bool ok;
  double u, v, z, det0;
  V3 nr;  // -r (third column)
};
Hit intersect(const CamSurfel& s, V3 r) {
  Hit h;
  h.nr = -r;
  const V3 rhs = -s.mu_c;
  h.det0 = det3(s.m_u, s.m_v, h.nr);
  if (h.det0 == 0.0 || !std::isfinite(h.det0)) {
    h.ok = false;
    return h;
  }
  h.u = det3(rhs, s.m_v, h.nr) / h.det0;
  h.v = det3(s.m_u, rhs, h.nr) / h.det0;
  h.z = det3(s.m_u, s.m_v, rhs) / h.det0;
  h.ok = std::isfinite(h.u) && std::isfinite(h.v) && std::isfinite(h.z);
  return h;
}

struct Item {
  double depth_c;   // centre depth mu_c.z: the sort key
  int id;
  double u, v, z, G, a;
  bool clamped;
};

// All surfels that the pixel keeps, in blending order (centre depth, id).
void pixel_items(const std::vector<CamSurfel>& S, const Cam& cam, const Rule& rule, double x,
                 double y, std::vector<Item>& items) {
  items.clear();
  const V3 r = mk((x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0);
  for (int i = 0; i < (int)S.size(); ++i) {
    const CamSurfel& s = S[i];
    if (!(s.mu_c.z > cam.near_z)) continue;
    Hit h = intersect(s, r);
    if (!h.ok) continue;
    if (!(h.z > cam.near_z)) continue;
    const double r2 = h.u * h.u + h.v * h.v;
    if (!rule.exact && r2 > rule.cutoff_r2) continue;
    const double G = std::exp(-0.5 * r2);
    double a = s.alpha * G;
    bool clamped = false;
    if (!rule.exact) {
      if (a > rule.alpha_max) {
        a = rule.alpha_max;
        clamped = true;
      }
      if (a < rule.alpha_min) continue;
    }
    items.push_back(Item{s.mu_c.z, i, h.u, h.v, h.z, G, a, clamped});
  }
  std::sort(items.begin(), items.end(), [](const Item& p, const Item& q) {
    if (p.depth_c != q.depth_c) return p.depth_c < q.depth_c;
    return p.id < q.id;
  });
}

// Keep only the blended prefix: blending stops before the item whose
// inclusion would take the transmittance below t_min.
int blended_count(const std::vector<Item>& items, const Rule& rule) {
  if (rule.exact) return (int)items.size();
  double T = 1.0;
  for (int k = 0; k < (int)items.size(); ++k) {
    const double Tn = T * (1.0 - items[k].a);
    if (Tn < rule.t_min) return k;
    T = Tn;
  }
  return (int)items.size();
}

std::vector<CamSurfel> camera_surfels(int n, const double* mu, const double* quat,
                                      const double* scale, const double* opacity,
                                      const double* rgb, const double* Rcw, const double* tcw) {
  std::vector<CamSurfel> S(n);
  for (int i = 0; i < n; ++i) S[i] = make_cam_surfel(i, mu, quat, scale, opacity, rgb, Rcw, tcw);
  return S;
}

void pixel_coord(int k, int n_pix, const int* pix, int W, double& x, double& y) {
  (void)n_pix;
  int px, py;
  if (pix) {
    px = pix[2 * k];
    py = pix[2 * k + 1];
  } else {
    px = k % W;
    py = k / W;
  }
  x = px + 0.5;
  y = py + 0.5;
}

int n_threads_or_default(int n_threads) {
#ifdef _OPENMP
  return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
  (void)n_threads;
  return 1;
#endif
}

struct Cand {
  double depth_c;
  int id;
  bool on_edge;
};

// Relative margins of the threshold diagnostics: an intersection whose
// u^2 + v^2, alpha G or depth lies within kTight (relative) of the cutoff,
// alpha_min or the near plane, or a stop test whose transmittance lies within
// kLooseT (relative) of t_min, may be decided otherwise by an FP32
// evaluation of the same pixel.
constexpr double kTight = 2e-5, kLooseT = 1e-4;

// Diagnostic of the parity tests (no computed value depends on it): fills
// cand with the pixel's candidates in blending order -- surfels whose
// intersection passes the near, cutoff and alpha_min tests within kTight --
// and returns true if the pixel holds a decision that FP32 may take
// otherwise: a candidate within kTight of a threshold at or before the
// position where blending stops, or a stop test (of a blended item or of the
// first item not blended) within kLooseT of t_min.  Such a decision changes
// the pixel's weights from that position on, and through the transmittance
// and the suffix sums of the backward pass the gradients of every item the
// pixel blends.  Exact mode has none of these thresholds: false.
bool pixel_threshold_ambiguous(const std::vector<CamSurfel>& S, const Cam& cam, const Rule& rule,
                               V3 r, const std::vector<Item>& items, int nb,
                               std::vector<Cand>& cand) {
  cand.clear();
  if (rule.exact) return false;
  for (int i = 0; i < (int)S.size(); ++i) {
    const CamSurfel& s = S[i];
    if (!(s.mu_c.z > cam.near_z)) continue;
    Hit h = intersect(s, r);
    if (!h.ok || !(h.z > cam.near_z * (1.0 - kTight))) continue;
    const double r2 = h.u * h.u + h.v * h.v;
    if (r2 > rule.cutoff_r2 * (1.0 + kTight)) continue;
    const double a = s.alpha * std::exp(-0.5 * r2);
    if (a < rule.alpha_min * (1.0 - kTight)) continue;
    const bool on_edge = std::fabs(r2 - rule.cutoff_r2) <= kTight * rule.cutoff_r2 ||
                         std::fabs(a - rule.alpha_min) <= kTight * rule.alpha_min ||
                         std::fabs(h.z - cam.near_z) <= kTight * cam.near_z;
    cand.push_back(Cand{s.mu_c.z, i, on_edge});
  }
  std::sort(cand.begin(), cand.end(), [](const Cand& p, const Cand& q) {
    if (p.depth_c != q.depth_c) return p.depth_c < q.depth_c;
    return p.id < q.id;
  });
  int p_stop = (int)cand.size();
  if (nb < (int)items.size())
    for (int c = 0; c < (int)cand.size(); ++c)
      if (cand[c].id == items[nb].id) {
        p_stop = c;
        break;
      }
  for (int c = 0; c <= p_stop && c < (int)cand.size(); ++c)
    if (cand[c].on_edge) return true;
  double T = 1.0;
  for (int m = 0; m < (int)items.size() && m <= nb; ++m) {
    const double Tn = T * (1.0 - items[m].a);
    if (std::fabs(Tn - rule.t_min) <= kLooseT * rule.t_min) return true;
    T = Tn;
  }
  return false;
}

}  // namespace

extern "C" {

// Forward render of the listed pixels (all W*H pixels, row-major, if pix is
// NULL).  cam5 = (fx, fy, cx, cy, near); rule4 = (alpha_min, alpha_max,
// t_min, cutoff_r2); R9 row-major world->camera rotation, t3 translation.
// Outputs per listed pixel: rgb[3], depth, normal[3], opacity, T_final, the
// number of blended surfels and (if out_mincos is non-NULL) the smallest
// |cos| between the ray and a blended surfel's normal -- near zero when a
// surfel is seen edge-on, where the intersection is ill-conditioned -- and
// (if out_amb is non-NULL) 1 where pixel_threshold_ambiguous holds.
int orc_render(int n, const double* mu, const double* quat, const double* scale,
               const double* opacity, const double* rgb, const double* cam5, int W, int H,
               const double* R9, const double* t3, const double* rule4, int exact, int n_pix,
               const int* pix, double* out_rgb, double* out_depth, double* out_normal,
               double* out_opacity, double* out_tfinal, int* out_count, double* out_mincos,
               int* out_amb, int n_threads) {
  const Cam cam{cam5[0], cam5[1], cam5[2], cam5[3], cam5[4], W, H};
  const Rule rule{rule4[0], rule4[1], rule4[2], rule4[3], exact};
  const std::vector<CamSurfel> S = camera_surfels(n, mu, quat, scale, opacity, rgb, R9, t3);
  const int np = pix ? n_pix : W * H;
#pragma omp parallel num_threads(n_threads_or_default(n_threads))
  {
    std::vector<Item> items;
    std::vector<Cand> cand;
#pragma omp for schedule(dynamic, 16)
    for (int k = 0; k < np; ++k) {
      double x, y;
      pixel_coord(k, np, pix, W, x, y);
      pixel_items(S, cam, rule, x, y, items);
      const int nb = blended_count(items, rule);
      double T = 1.0, D = 0.0, mincos = 1.0;
      V3 C = mk(0, 0, 0), N = mk(0, 0, 0);
      const V3 rr = mk((x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0);
      for (int m = 0; m < nb; ++m) {
        const Item& it = items[m];
        const CamSurfel& s = S[it.id];
        mincos = std::min(mincos, std::fabs(dot(rr, s.tn_c)) / std::sqrt(dot(rr, rr)));
        const double w = it.a * T;
        C += w * s.col;
        D += w * it.z;
        N += w * s.tn_c;
        T *= (1.0 - it.a);
      }
      out_rgb[3 * k] = C.x;
      out_rgb[3 * k + 1] = C.y;
      out_rgb[3 * k + 2] = C.z;
      out_depth[k] = D;
      out_normal[3 * k] = N.x;
      out_normal[3 * k + 1] = N.y;
      out_normal[3 * k + 2] = N.z;
      out_opacity[k] = 1.0 - T;
      out_tfinal[k] = T;
      out_count[k] = nb;
      if (out_mincos) out_mincos[k] = mincos;
      if (out_amb) out_amb[k] = pixel_threshold_ambiguous(S, cam, rule, rr, items, nb, cand) ? 1 : 0;
    }
  }
  return 0;
}

// Per-surfel contribution (Sec. III-D, Eq. weight and Eq. contribution):
// out_contrib[i] = sum over the listed pixels of w_i(p) = a_i T_i, the
// blending weight of surfel i in pixel p (the same items and stop rule as
// orc_render).  Diagnostics for the parity tests, per surfel:
//   out_flag[i]  = 1 if, at some pixel, i is a candidate (a valid
//                  intersection in front of the near plane, inside or near
//                  the cutoff and alpha_min bounds) at or after the first
//                  candidate in blending order whose evaluation sits within
//                  a small relative margin of a threshold (cutoff radius,
//                  alpha_min, near plane, or the stop test on T) and that
//                  the pixel reaches (an FP32 evaluation may legitimately
//                  decide that one otherwise, which changes the weights
//                  from there on), or the item whose stop test sits within
//                  a small margin of t_min, or the item after it;
//   out_bbox[4i..4i+3] = x0, y0, x1, y1 of the listed pixels where i is a
//                  candidate (x0 = -1 if none);
//   out_mincos[i] = smallest |cos| between a ray it blends into and its
//                  normal (1 if none).
int orc_contrib(int n, const double* mu, const double* quat, const double* scale,
                const double* opacity, const double* rgb, const double* cam5, int W, int H,
                const double* R9, const double* t3, const double* rule4, int exact, int n_pix,
                const int* pix, double* out_contrib, int* out_flag, int* out_bbox,
                double* out_mincos, int n_threads) {
  const Cam cam{cam5[0], cam5[1], cam5[2], cam5[3], cam5[4], W, H};
  const Rule rule{rule4[0], rule4[1], rule4[2], rule4[3], exact};
  const std::vector<CamSurfel> S = camera_surfels(n, mu, quat, scale, opacity, rgb, R9, t3);
  const int np = pix ? n_pix : W * H;
  const double tight = 2e-5, loose_t = 1e-4;
  const int nt = n_threads_or_default(n_threads);
  std::vector<std::vector<double>> acc(nt), mc(nt);
  std::vector<std::vector<int>> flag(nt), box(nt);
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    const int tid = omp_get_thread_num();
#else
    const int tid = 0;
#endif
    acc[tid].assign(n, 0.0);
    mc[tid].assign(n, 1.0);
    flag[tid].assign(n, 0);
    box[tid].assign(4 * (size_t)n, -1);
    std::vector<Item> items;
    std::vector<Cand> cand;
#pragma omp for schedule(dynamic, 16)
    for (int k = 0; k < np; ++k) {
      double x, y;
      pixel_coord(k, np, pix, W, x, y);
      const int px = (int)std::floor(x), py = (int)std::floor(y);
      const V3 r = mk((x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0);
      // candidates (loose bounds) in blending order, each with its margin flag
      cand.clear();
      for (int i = 0; i < n; ++i) {
        const CamSurfel& s = S[i];
        if (!(s.mu_c.z > cam.near_z)) continue;
        Hit h = intersect(s, r);
        if (!h.ok || !(h.z > cam.near_z * (1.0 - tight))) continue;
        const double r2 = h.u * h.u + h.v * h.v;
        if (r2 > rule.cutoff_r2 * (1.0 + tight)) continue;
        const double a = s.alpha * std::exp(-0.5 * r2);
        if (a < rule.alpha_min * (1.0 - tight)) continue;
        const bool on_edge = std::fabs(r2 - rule.cutoff_r2) <= tight * rule.cutoff_r2 ||
                             std::fabs(a - rule.alpha_min) <= tight * rule.alpha_min ||
                             std::fabs(h.z - cam.near_z) <= tight * cam.near_z;
        cand.push_back(Cand{s.mu_c.z, i, on_edge});
      }
      std::sort(cand.begin(), cand.end(), [](const Cand& p, const Cand& q) {
        if (p.depth_c != q.depth_c) return p.depth_c < q.depth_c;
        return p.id < q.id;
      });
      auto pos_of = [&](int id) {
        for (int c = 0; c < (int)cand.size(); ++c)
          if (cand[c].id == id) return c;
        return (int)cand.size();
      };
      pixel_items(S, cam, rule, x, y, items);
      const int nb = blended_count(items, rule);
      // a decision taken otherwise at candidate position m changes the
      // weights from m on; positions after the stop are reached by neither
      // side unless the stop itself moves
      const int p_stop = nb < (int)items.size() ? pos_of(items[nb].id) : (int)cand.size();
      int first = (int)cand.size();
      for (int c = 0; c <= p_stop && c < (int)cand.size(); ++c)
        if (cand[c].on_edge) {
          first = c;
          break;
        }
      // the stop test near t_min moves the stop by one item: only that item
      // and the next one can change weight (by about t_min a / (1 - a))
      double T = 1.0;
      for (int m = 0; m < (int)items.size() && m <= nb; ++m) {
        const double Tn = T * (1.0 - items[m].a);
        if (!rule.exact && std::fabs(Tn - rule.t_min) <= loose_t * rule.t_min) {
          flag[tid][items[m].id] = 1;
          if (m + 1 < (int)items.size()) flag[tid][items[m + 1].id] = 1;
        }
        if (m == nb) break;
        const Item& it = items[m];
        const CamSurfel& s = S[it.id];
        acc[tid][it.id] += it.a * T;
        mc[tid][it.id] = std::min(mc[tid][it.id],
                                  std::fabs(dot(r, s.tn_c)) / std::sqrt(dot(r, r)));
        T = Tn;
      }
      for (int c = first; c < (int)cand.size(); ++c) flag[tid][cand[c].id] = 1;
      for (const Cand& cd : cand) {
        const int i = cd.id;
        int* b = &box[tid][4 * (size_t)i];
        if (b[0] < 0) {
          b[0] = b[2] = px;
          b[1] = b[3] = py;
        } else {
          b[0] = std::min(b[0], px);
          b[1] = std::min(b[1], py);
          b[2] = std::max(b[2], px);
          b[3] = std::max(b[3], py);
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    double c = 0.0, m = 1.0;
    int f = 0, b0 = -1, b1 = -1, b2 = -1, b3 = -1;
    for (int t = 0; t < nt; ++t) {
      c += acc[t][i];
      m = std::min(m, mc[t][i]);
      f |= flag[t][i];
      const int* b = &box[t][4 * (size_t)i];
      if (b[0] < 0) continue;
      if (b0 < 0) {
        b0 = b[0], b1 = b[1], b2 = b[2], b3 = b[3];
      } else {
        b0 = std::min(b0, b[0]), b1 = std::min(b1, b[1]);
        b2 = std::max(b2, b[2]), b3 = std::max(b3, b[3]);
      }
    }
    out_contrib[i] = c;
    if (out_flag) out_flag[i] = f;
    if (out_bbox) {
      out_bbox[4 * i] = b0, out_bbox[4 * i + 1] = b1, out_bbox[4 * i + 2] = b2,
      out_bbox[4 * i + 3] = b3;
    }
    if (out_mincos) out_mincos[i] = m;
  }
  return 0;
}

// Reverse mode of orc_render.  g_* are dL/d(rgb, depth, normal, opacity) per
// listed pixel.  Writes dL/d(mu, quat (raw), scale, opacity, rgb) per surfel
// and dL/dtau, tau = (rho, theta), for the left perturbation of T_cw; and, if
// d_mincos is non-NULL, per surfel the smallest |cos| between a pixel ray it
// blends into and its normal (1 if it blends into none): near zero marks a
// surfel seen edge-on, whose intersection is ill-conditioned; and, if d_amb
// is non-NULL, per surfel 1 if it is a candidate (pixel_threshold_ambiguous's
// list) of a listed pixel for which pixel_threshold_ambiguous holds -- an
// FP32 evaluation may legitimately give that surfel other gradient terms.
int orc_render_bwd(int n, const double* mu, const double* quat, const double* scale,
                   const double* opacity, const double* rgb, const double* cam5, int W, int H,
                   const double* R9, const double* t3, const double* rule4, int exact, int n_pix,
                   const int* pix, const double* g_rgb, const double* g_depth,
                   const double* g_normal, const double* g_opac, double* d_mu, double* d_quat,
                   double* d_scale, double* d_opacity, double* d_rgb, double* d_pose6,
                   double* d_mincos, int* d_amb, int n_threads) {
  const Cam cam{cam5[0], cam5[1], cam5[2], cam5[3], cam5[4], W, H};
  const Rule rule{rule4[0], rule4[1], rule4[2], rule4[3], exact};
  const std::vector<CamSurfel> S = camera_surfels(n, mu, quat, scale, opacity, rgb, R9, t3);
  const int np = pix ? n_pix : W * H;
  int nt = n_threads_or_default(n_threads);
  // bound the per-thread accumulators to about 2 GB
  const long long per_thread = (long long)n * 128;
  if (per_thread > 0 && nt > 1 && per_thread * nt > (2LL << 30))
    nt = std::max(1, (int)((2LL << 30) / per_thread));
  // camera-space gradients per surfel, one buffer per thread, summed in
  // thread order afterwards (deterministic for a fixed thread count)
  struct Acc {
    V3 g_mu_c, g_mu, g_mv, g_tn_c, g_col;
    double g_alpha;
    double mincos;  // smallest |cos(ray, normal)| over the pixels it blends into
  };
  std::vector<std::vector<Acc>> acc(nt, std::vector<Acc>(n, Acc{mk(0, 0, 0), mk(0, 0, 0), mk(0, 0, 0),
                                                                 mk(0, 0, 0), mk(0, 0, 0), 0.0, 1.0}));
  std::vector<std::vector<char>> amb(nt);
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    const int tid = omp_get_thread_num();
#else
    const int tid = 0;
#endif
    std::vector<Acc>& A = acc[tid];
    if (d_amb) amb[tid].assign(n, 0);
    std::vector<Item> items;
    std::vector<Cand> cand;
    std::vector<double> Tb;  // transmittance before each blended item
#pragma omp for schedule(dynamic, 16)
    for (int k = 0; k < np; ++k) {
      double x, y;
      pixel_coord(k, np, pix, W, x, y);
      const V3 r = mk((x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0);
      pixel_items(S, cam, rule, x, y, items);
      const int nb = blended_count(items, rule);
      if (d_amb && pixel_threshold_ambiguous(S, cam, rule, r, items, nb, cand))
        for (const Cand& cd : cand) amb[tid][cd.id] = 1;
      Tb.assign(nb + 1, 1.0);
      for (int m = 0; m < nb; ++m) Tb[m + 1] = Tb[m] * (1.0 - items[m].a);
      const V3 gC = mk(g_rgb[3 * k], g_rgb[3 * k + 1], g_rgb[3 * k + 2]);
      const double gD = g_depth[k];
      const V3 gN = mk(g_normal[3 * k], g_normal[3 * k + 1], g_normal[3 * k + 2]);
      // O = 1 - T_final
      double gT = -g_opac[k];
      for (int m = nb - 1; m >= 0; --m) {
        const Item& it = items[m];
        const CamSurfel& s = S[it.id];
        const double T = Tb[m];
        const double w = it.a * T;
        // T_{m+1} = T_m (1 - a_m)
        double g_a = -gT * T;
        double g_Tm = gT * (1.0 - it.a);
        // w_m = a_m T_m feeds C, D, N
        const double g_w = dot(gC, s.col) + gD * it.z + dot(gN, s.tn_c);
        g_a += g_w * T;
        g_Tm += g_w * it.a;
        gT = g_Tm;
        Acc& a = A[it.id];
        a.mincos = std::min(a.mincos, std::fabs(dot(r, s.tn_c)) / std::sqrt(dot(r, r)));
        a.g_col += w * gC;
        a.g_tn_c += w * gN;
        double g_z = w * gD;
        // a = alpha G (unless clamped)
        double g_G = 0.0;
        if (!it.clamped) {
          a.g_alpha += it.G * g_a;
          g_G = s.alpha * g_a;
        }
        const double g_r2 = -0.5 * it.G * g_G;
        const double g_u = 2.0 * it.u * g_r2;
        const double g_v = 2.0 * it.v * g_r2;
        // Cramer: u = det[rhs,m_v,nr]/d0, v = det[m_u,rhs,nr]/d0,
        //         z = det[m_u,m_v,rhs]/d0, d0 = det[m_u,m_v,nr], rhs = -mu_c
        const Hit h = intersect(s, r);
        const V3 rhs = -s.mu_c;
        const double gNu = g_u / h.det0, gNv = g_v / h.det0, gNz = g_z / h.det0;
        const double gd0 = -(g_u * it.u + g_v * it.v + g_z * it.z) / h.det0;
        // d det[a,b,c]: da = b x c, db = c x a, dc = a x b
        V3 g_rhs = gNu * cross(s.m_v, h.nr) + gNv * cross(h.nr, s.m_u) + gNz * cross(s.m_u, s.m_v);
        V3 g_mu = gNv * cross(rhs, h.nr) + gNz * cross(s.m_v, rhs) + gd0 * cross(s.m_v, h.nr);
        V3 g_mv = gNu * cross(h.nr, rhs) + gNz * cross(rhs, s.m_u) + gd0 * cross(h.nr, s.m_u);
        a.g_mu_c += -g_rhs;
        a.g_mu += g_mu;
        a.g_mv += g_mv;
      }
    }
  }
  // fixed-order reduction over threads, then per-surfel chain rule
  V3 g_rho = mk(0, 0, 0), g_theta = mk(0, 0, 0);
  for (int i = 0; i < n; ++i) {
    Acc t{};
    t.mincos = 1.0;
    for (int th = 0; th < nt; ++th) {
      const Acc& a = acc[th][i];
      t.mincos = std::min(t.mincos, a.mincos);
      t.g_mu_c += a.g_mu_c;
      t.g_mu += a.g_mu;
      t.g_mv += a.g_mv;
      t.g_tn_c += a.g_tn_c;
      t.g_col += a.g_col;
      t.g_alpha += a.g_alpha;
    }
    const CamSurfel& s = S[i];
    // m_u = s_u t_uc, m_v = s_v t_vc
    const V3 g_tu_c = s.su * t.g_mu, g_tv_c = s.sv * t.g_mv, g_tn_c = t.g_tn_c;
    d_scale[2 * i] = dot(s.tu_c, t.g_mu);
    d_scale[2 * i + 1] = dot(s.tv_c, t.g_mv);
    // pose: mu_c and the columns of R_c move with the left perturbation
    g_rho += t.g_mu_c;
    g_theta += cross(s.mu_c, t.g_mu_c) + cross(s.tu_c, g_tu_c) + cross(s.tv_c, g_tv_c) +
               cross(s.tn_c, g_tn_c);
    // camera -> world
    const V3 gmu = matTvec(R9, t.g_mu_c);
    const V3 gtu = matTvec(R9, g_tu_c), gtv = matTvec(R9, g_tv_c), gtn = matTvec(R9, g_tn_c);
    d_mu[3 * i] = gmu.x;
    d_mu[3 * i + 1] = gmu.y;
    d_mu[3 * i + 2] = gmu.z;
    // R(q_hat) columns -> normalised quaternion -> raw quaternion
    double J[3][3][4];
    quat_matrix_jac(s.qn, J);
    const double gR[3][3] = {{gtu.x, gtv.x, gtn.x}, {gtu.y, gtv.y, gtn.y}, {gtu.z, gtv.z, gtn.z}};
    double gq[4] = {0, 0, 0, 0};
    for (int rr = 0; rr < 3; ++rr)
      for (int cc = 0; cc < 3; ++cc)
        for (int k = 0; k < 4; ++k) gq[k] += gR[rr][cc] * J[rr][cc][k];
    const double qd = s.qn[0] * gq[0] + s.qn[1] * gq[1] + s.qn[2] * gq[2] + s.qn[3] * gq[3];
    for (int k = 0; k < 4; ++k) d_quat[4 * i + k] = (gq[k] - s.qn[k] * qd) / s.qlen;
    d_opacity[i] = t.g_alpha;
    if (d_mincos) d_mincos[i] = t.mincos;
    if (d_amb) {
      int f = 0;
      for (int th = 0; th < nt; ++th) f |= amb[th][i];
      d_amb[i] = f;
    }
    d_rgb[3 * i] = t.g_col.x;
    d_rgb[3 * i + 1] = t.g_col.y;
    d_rgb[3 * i + 2] = t.g_col.z;
  }
  d_pose6[0] = g_rho.x;
  d_pose6[1] = g_rho.y;
  d_pose6[2] = g_rho.z;
  d_pose6[3] = g_theta.x;
  d_pose6[4] = g_theta.y;
  d_pose6[5] = g_theta.z;
  return 0;
}

// Unit vectors (c, s) with A c + B s = rhs: rhs / |(A, B)| clamped to
// [-1, 1] unless exact (then |rhs| must not exceed |(A, B)|).
static int unit_solutions(double A, double B, double rhs, bool exact, double cs[2][2]) {
  const double R = std::sqrt(A * A + B * B);
  if (!(R > 0.0)) return 0;
  double t = rhs / R;
  if (exact && std::fabs(t) > 1.0) return 0;
  t = std::max(-1.0, std::min(1.0, t));
  const double q = std::sqrt(std::max(1.0 - t * t, 0.0));
  const double hx = A / R, hy = B / R;
  cs[0][0] = t * hx - q * hy;
  cs[0][1] = t * hy + q * hx;
  cs[1][0] = t * hx + q * hy;
  cs[1][1] = t * hy - q * hx;
  return 2;
}

// Conservative tile rectangle of each surfel's footprint, in FP64.
// A pixel can only pass the cutoff and alpha tests inside the disc
// u^2 + v^2 <= rho^2, rho^2 = 1.01 min(cutoff_r2, 2 ln(alpha / alpha_min)),
// and only where its hit depth is beyond the near plane; the footprint is the
// image of that disc clipped to camera depth z >= 0.99 near.  Its boundary is
// the circle P(c, s) = mu_c + rho (c m_u + s m_v) (c^2 + s^2 = 1) and the
// chord where the circle meets z = 0.99 near.  The image coordinate
// x = fx P_x / P_z + cx has its extremes over the (convex) clipped disc at
// stationary points on the circle -- d/dt (P_x / P_z) = 0, which works out to
//   c (m_vx mu_z - mu_x m_vz) + s (mu_x m_uz - m_ux mu_z) = rho (m_ux m_vz - m_vx m_uz)
// -- when they lie in front of the clip plane, or at the chord's ends.  y
// alike.  Pixels with centres inside [xmin, xmax] are ceil(xmin - 0.5) ..
// floor(xmax - 0.5); tiles are those pixels // tile size.
// rect = (tx0, ty0, tx1, ty1), or (1, 1, 0, 0) for a culled surfel.
int orc_tile_rects(int n, const double* mu, const double* quat, const double* scale,
                   const double* opacity, const double* cam5, int W, int H, const double* R9,
                   const double* t3, const double* rule4, int tile_w, int tile_h, int* rect_out,
                   double* depth_out) {
  const Cam cam{cam5[0], cam5[1], cam5[2], cam5[3], cam5[4], W, H};
  std::vector<double> rgb0(3 * (size_t)n, 0.0);
  const std::vector<CamSurfel> S = camera_surfels(n, mu, quat, scale, opacity, rgb0.data(), R9, t3);
  const double amin = rule4[0], cutoff = rule4[3];
  const double zmin = 0.99 * cam.near_z;
  for (int i = 0; i < n; ++i) {
    const CamSurfel& s = S[i];
    int* rc = rect_out + 4 * i;
    depth_out[i] = s.mu_c.z;
    rc[0] = 1;
    rc[1] = 1;
    rc[2] = 0;
    rc[3] = 0;
    if (!(s.mu_c.z > cam.near_z) || !(s.alpha >= amin)) continue;
    const double rho2 = 1.01 * std::min(cutoff, 2.0 * std::log(s.alpha / amin));
    if (!(rho2 > 0.0)) continue;
    const double rho = std::sqrt(rho2);
    const V3 a = s.m_u, b = s.m_v, m = s.mu_c;
    double cand[6][2];
    int nc = 0;
    double cs[2][2];
    int k = unit_solutions(b.x * m.z - m.x * b.z, m.x * a.z - a.x * m.z, rho * (a.x * b.z - b.x * a.z),
                           false, cs);
    for (int j = 0; j < k; ++j) { cand[nc][0] = cs[j][0]; cand[nc][1] = cs[j][1]; ++nc; }
    const bool open_x = k == 0;
    k = unit_solutions(b.y * m.z - m.y * b.z, m.y * a.z - a.y * m.z, rho * (a.y * b.z - b.y * a.z),
                       false, cs);
    for (int j = 0; j < k; ++j) { cand[nc][0] = cs[j][0]; cand[nc][1] = cs[j][1]; ++nc; }
    const bool open_y = k == 0;
    k = unit_solutions(a.z, b.z, (zmin - m.z) / rho, true, cs);
    for (int j = 0; j < k; ++j) { cand[nc][0] = cs[j][0]; cand[nc][1] = cs[j][1]; ++nc; }
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    bool any = false;
    for (int j = 0; j < nc; ++j) {
      const V3 P = m + rho * (cand[j][0] * a + cand[j][1] * b);
      if (!(P.z >= zmin * (1.0 - 1e-9))) continue;
      const double x = cam.fx * P.x / P.z + cam.cx, y = cam.fy * P.y / P.z + cam.cy;
      x0 = std::min(x0, x);
      x1 = std::max(x1, x);
      y0 = std::min(y0, y);
      y1 = std::max(y1, y);
      any = true;
    }
    if (!any) continue;
    if (open_x) {
      x0 = -1e300;
      x1 = 1e300;
    }
    if (open_y) {
      y0 = -1e300;
      y1 = 1e300;
    }
    const double i0 = std::max(std::ceil(x0 - 0.5), 0.0), i1 = std::min(std::floor(x1 - 0.5), W - 1.0);
    const double j0 = std::max(std::ceil(y0 - 0.5), 0.0), j1 = std::min(std::floor(y1 - 0.5), H - 1.0);
    if (i0 > i1 || j0 > j1) continue;
    rc[0] = (int)i0 / tile_w;
    rc[1] = (int)j0 / tile_h;
    rc[2] = (int)i1 / tile_w;
    rc[3] = (int)j1 / tile_h;
  }
  return 0;
}

// Tile binning and depth ordering as a plain library sort: every surfel with
// a non-empty rectangle emits one (tile, depth) pair per covered tile, row by
// row; the pairs are stable-sorted by key = tile << 32 | depth_bits, so equal
// keys keep surfel-id order (the depth ordering of Sec. III-A).  Returns the
// number of pairs, or -1 if it exceeds cap.  ranges[2t], ranges[2t+1] are the
// [start, end) of tile t (0, 0 for an empty tile).
long long orc_bin_sort(int n, const int* rect, const uint32_t* depth_bits, int tiles_x,
                       int tiles_y, uint64_t* keys, uint32_t* vals, long long cap, int* ranges) {
  std::vector<std::pair<uint64_t, uint32_t>> kv;
  for (int i = 0; i < n; ++i) {
    const int* rc = rect + 4 * i;
    for (int ty = rc[1]; ty <= rc[3]; ++ty)
      for (int tx = rc[0]; tx <= rc[2]; ++tx) {
        const uint64_t tile = (uint64_t)ty * tiles_x + tx;
        kv.emplace_back((tile << 32) | depth_bits[i], (uint32_t)i);
      }
  }
  std::stable_sort(kv.begin(), kv.end(),
                   [](const std::pair<uint64_t, uint32_t>& a,
                      const std::pair<uint64_t, uint32_t>& b) { return a.first < b.first; });
  if ((long long)kv.size() > cap) return -1;
  const int nt = tiles_x * tiles_y;
  for (int t = 0; t < 2 * nt; ++t) ranges[t] = 0;
  for (size_t k = 0; k < kv.size(); ++k) {
    keys[k] = kv[k].first;
    vals[k] = kv[k].second;
    const int t = (int)(kv[k].first >> 32);
    if (k == 0 || (int)(kv[k - 1].first >> 32) != t) ranges[2 * t] = (int)k;
    if (k + 1 == kv.size() || (int)(kv[k + 1].first >> 32) != t) ranges[2 * t + 1] = (int)k + 1;
  }
  return (long long)kv.size();
}

}  // extern "C"
