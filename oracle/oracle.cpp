// FP64 CPU oracle for the sharp-interface VOF phase-change hot path — TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, obviously correct restatement of what the method computes, used to check the CUDA
// library. It shares no code with the library. Only the tests, the smoke check and the benchmark's
// CPU-baseline leg may load it.
//
// Steps (paper: "Interface capturing method" Sec. 2.1, Eq. (edge_intersection); "Energy specific
// terms" Sec. 2.3 Eqs. (mass_transfer), (front_interpolation), (extrapolation), (latent_source),
// (interface_htc); Appendix B least squares):
//   R0  interface cells: eps < alpha < 1 - eps
//   R1  vertex field: inverse-distance (or plain) average of the alpha of the cells around a vertex
//   R2  liquid sub-volume V_L(c) of a cell: the cell split into tetrahedra of its own vertices
//       (faces fanned from their lowest-id vertex, the cell fanned from its lowest-id vertex),
//       phi linear on each; the wet part of each tetrahedron by clipping with the plane phi = c
//       through the cuts of Eq. edge_intersection
//   R3  isovalue by bisection on V_L(c)/V - alpha; or by the interval cubic (bisection over the
//       sorted vertex values, then the cubic V_L has between two of them, solved on its own)
//   R4  crossing point x_f on faces with (alpha_P - 1/2)(alpha_Q - 1/2) < 0
//   R5  per-side gradients: own phase from the modified LSQ gradient, other phase from one upwind
//       sweep over the neighbours on that side; or from the full
//       pseudo-time solve of Eq. (extrapolation), first-order upwind, per side and component
//   R6  q_l, q_v, mdot, Q_phase
//   R7  interface-modified least squares gradient (Appendix B), explicit symmetric inverse
//   R8  totals by a fixed pairwise tree
//   S   stencil variants of R7 for the stencil-anisotropy study:
//       standard (unmodified) stencil, inverse-distance weights, vertex neighbours; cond(G_P)
//
// Pinned only in special cases: R5, a reading of the extrapolation step (closed forms when the
// neighbour gradients are equal; its weights also enter the pseudo-time solve, whose first step at a
// Courant number of 1 reproduces it). R1 (inverse distances to cells of different sizes) and R4's
// choice between two different planes are pinned by cases worked by hand.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

extern "C" {

struct OrcMesh {
  int64_t n_cells, n_faces, n_verts;
  const double *vx, *vy, *vz;
  const int64_t* face_vert_off;
  const int32_t* face_vert;
  const int32_t *face_owner, *face_neigh;
  const int64_t* cell_face_off;
  const int32_t* cell_face;
};

struct OrcProps {
  double k_l, k_v, h_lv, T_sat;
};

// Options of the pseudo-time extrapolation; iters[] returns the iterations each of the six
// solves took (liquid side x, y, z, then vapour side x, y, z).
struct OrcExtrap {
  int max_iter;
  double tol;   // K/m, absolute, on the largest change of one iteration
  double dtau;  // pseudo-time step; <= 0: the mesh's min_f |d_f|
  int32_t iters[6];
};

}  // extern "C"

namespace {

// status bits (same meaning as the library's)
constexpr int ST_DEGENERATE = 1;
constexpr int ST_NOT_CONVERGED = 2;
constexpr int ST_SINGULAR_LSQ = 8;
constexpr int ST_NO_SIDE = 16;

using V3 = std::array<double, 3>;
V3 sub(const V3& a, const V3& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
V3 add(const V3& a, const V3& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
V3 mul(const V3& a, double s) { return {a[0] * s, a[1] * s, a[2] * s}; }
double dot(const V3& a, const V3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
V3 cross(const V3& a, const V3& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
double norm(const V3& a) { return std::sqrt(dot(a, a)); }

V3 vert(const OrcMesh& m, int32_t v) { return {m.vx[v], m.vy[v], m.vz[v]}; }

// Vertex loop of face f as seen from cell c (outward from c).
std::vector<int32_t> loop_of(const OrcMesh& m, int32_t face_entry) {
  const int32_t f = face_entry & 0x7fffffff;
  std::vector<int32_t> L(m.face_vert + m.face_vert_off[f], m.face_vert + m.face_vert_off[f + 1]);
  if (face_entry < 0) std::reverse(L.begin(), L.end());
  return L;
}

std::vector<int32_t> cell_vertices(const OrcMesh& m, int64_t c) {
  std::vector<int32_t> vs;
  for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
    const int32_t f = m.cell_face[k] & 0x7fffffff;
    for (int64_t j = m.face_vert_off[f]; j < m.face_vert_off[f + 1]; ++j) vs.push_back(m.face_vert[j]);
  }
  std::sort(vs.begin(), vs.end());
  vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
  return vs;
}

V3 mean_point(const OrcMesh& m, const std::vector<int32_t>& vs) {
  V3 s = {0, 0, 0};
  for (int32_t v : vs) s = add(s, vert(m, v));
  return mul(s, 1.0 / (double)vs.size());
}

// Signed volume of the tetrahedron (x0, a, b, c); positive when (a, b, c) is counter-clockwise
// seen from outside, x0 inside.
double tet_vol(const V3& x0, const V3& a, const V3& b, const V3& c) {
  return dot(sub(a, x0), cross(sub(b, x0), sub(c, x0))) / 6.0;
}

// Signed volume enclosed (with apex x0) by a polygon fanned about the point m.
double fan_volume(const std::vector<V3>& P, const V3& m, const V3& x0) {
  if (P.size() < 3) return 0.0;
  double v = 0;
  for (size_t i = 0; i < P.size(); ++i) v += tet_vol(x0, m, P[i], P[(i + 1) % P.size()]);
  return v;
}

V3 vertex_mean(const std::vector<V3>& P) {
  V3 m = {0, 0, 0};
  for (const V3& p : P) m = add(m, p);
  return mul(m, 1.0 / (double)P.size());
}

// ------------------------------------------------------------------------------ geometry
// Face vector area and centroid: fan of triangles about the face's vertex mean. Cell volume and
// centroid: fan tetrahedra from the cell's vertex mean to each face triangle.
void geometry(const OrcMesh& m, double* face_area, double* face_cen, double* cell_vol, double* cell_cen) {
  for (int64_t f = 0; f < m.n_faces; ++f) {
    std::vector<int32_t> L(m.face_vert + m.face_vert_off[f], m.face_vert + m.face_vert_off[f + 1]);
    const V3 a = mean_point(m, L);
    V3 A = {0, 0, 0}, cs = {0, 0, 0};
    double at = 0;
    for (size_t i = 0; i < L.size(); ++i) {
      const V3 p = vert(m, L[i]), q = vert(m, L[(i + 1) % L.size()]);
      const V3 t = mul(cross(sub(p, a), sub(q, a)), 0.5);
      A = add(A, t);
      const double ar = norm(t);
      cs = add(cs, mul(add(add(a, p), q), ar / 3.0));
      at += ar;
    }
    for (int k = 0; k < 3; ++k) {
      face_area[3 * f + k] = A[k];
      face_cen[3 * f + k] = at > 0 ? cs[k] / at : a[k];
    }
  }
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const V3 x0 = mean_point(m, cell_vertices(m, c));
    double vol = 0;
    V3 cs = {0, 0, 0};
    for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
      const std::vector<int32_t> L = loop_of(m, m.cell_face[k]);
      const V3 fm = mean_point(m, L);
      for (size_t i = 0; i < L.size(); ++i) {
        const V3 p = vert(m, L[i]), q = vert(m, L[(i + 1) % L.size()]);
        const double v = tet_vol(x0, fm, p, q);
        vol += v;
        cs = add(cs, mul(add(add(x0, fm), add(p, q)), v / 4.0));
      }
    }
    cell_vol[c] = vol;
    for (int k = 0; k < 3; ++k) cell_cen[3 * c + k] = cs[k] / vol;
  }
}

// ------------------------------------------------------------------------------ R2
struct IsoGeom {
  double VL = 0;
  double area = 0;           // area of the iso-surface
  V3 vec_area = {0, 0, 0};   // outward from the liquid (points to the vapour)
  V3 centroid = {0, 0, 0};   // area-weighted centroid of the iso-surface
};

struct VPt {
  V3 x;
  double phi;
};

// Wet part {phi >= c} of a tetrahedron on which phi is linear (values at its corners), by
// clipping: each triangular face keeps its corners with phi >= c and the cuts of Eq.
// edge_intersection on edges that straddle c; the cut section closes the wet polyhedron. Adds its
// volume (signed tetrahedra from the reference point x0) and the section's area, vector area and
// area moment to g.
void clip_tet(const VPt* T, double c, const V3& x0, IsoGeom& g, V3& moment) {
  static const int F[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
  // orient the faces outward
  const double s = dot(sub(T[1].x, T[0].x), cross(sub(T[2].x, T[0].x), sub(T[3].x, T[0].x)));
  auto cut = [&](int i, int j) {
    const double lam = (c - T[i].phi) / (T[j].phi - T[i].phi);
    return add(T[i].x, mul(sub(T[j].x, T[i].x), lam));
  };
  std::vector<V3> sec;  // section points
  std::vector<std::pair<int, int>> sec_edge;
  for (int f = 0; f < 4; ++f) {
    int v[3] = {F[f][0], F[f][1], F[f][2]};
    if (s < 0) std::swap(v[1], v[2]);
    std::vector<V3> W;
    // wet corners are those strictly above c: {phi > c} has the volume of {phi >= c}, and a corner
    // at exactly c then enters the wet polygons and the section as the cut of its edges to wet
    // corners (lambda = 1), so the wet surface stays closed when c equals a vertex value
    for (int k = 0; k < 3; ++k) {
      const int i = v[k], j = v[(k + 1) % 3];
      if (T[i].phi > c) W.push_back(T[i].x);
      if ((T[i].phi > c) != (T[j].phi > c)) {
        W.push_back(cut(i, j));
        const std::pair<int, int> e = {std::min(i, j), std::max(i, j)};
        if (std::find(sec_edge.begin(), sec_edge.end(), e) == sec_edge.end()) {
          sec_edge.push_back(e);
          sec.push_back(cut(e.first, e.second));
        }
      }
    }
    if (W.size() >= 3) g.VL += fan_volume(W, vertex_mean(W), x0);
  }
  if (sec.size() < 3) return;
  // the section is planar and convex: order its points by angle about their mean, oriented
  // along the direction of decreasing phi (outward from the liquid)
  V3 grad_dir;  // -grad phi direction of the linear field, from the corner values
  {
    const V3 e1 = sub(T[1].x, T[0].x), e2 = sub(T[2].x, T[0].x), e3 = sub(T[3].x, T[0].x);
    const double d1 = T[1].phi - T[0].phi, d2 = T[2].phi - T[0].phi, d3 = T[3].phi - T[0].phi;
    const V3 c23 = cross(e2, e3), c31 = cross(e3, e1), c12 = cross(e1, e2);
    const double det = dot(e1, c23);
    const V3 grad = mul(add(add(mul(c23, d1), mul(c31, d2)), mul(c12, d3)), 1.0 / det);
    grad_dir = mul(grad, -1.0);
  }
  const V3 m = vertex_mean(sec);
  V3 u = sub(sec[0], m);
  const V3 w = cross(grad_dir, u);
  std::vector<std::pair<double, V3>> ord;
  for (const V3& p : sec) ord.push_back({std::atan2(dot(sub(p, m), w), dot(sub(p, m), u)), p});
  std::sort(ord.begin(), ord.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<V3> P;
  for (auto& o : ord) P.push_back(o.second);
  // the wet polyhedron's cap: seen from the dry side the loop is counter-clockwise
  g.VL += fan_volume(P, m, x0);
  for (size_t k = 0; k < P.size(); ++k) {
    const V3 tv = mul(cross(sub(P[k], m), sub(P[(k + 1) % P.size()], m)), 0.5);
    const double ar = norm(tv);
    g.area += ar;
    g.vec_area = add(g.vec_area, tv);
    moment = add(moment, mul(add(add(m, P[k]), P[(k + 1) % P.size()]), ar / 3.0));
  }
}

// R2. The cell is split into tetrahedra using only its own vertices: each face is fanned from
// its lowest-id vertex, and the cell is fanned from its lowest-id vertex (the apex) over every
// face triangle that does not contain the apex (a convex cell is star-shaped from any vertex).
// phi is linear on each tetrahedron, so its iso-surface there is planar and passes through the cuts
// of Eq. edge_intersection on the tetrahedron's edges, the cell's own edges included. V_L(c) is the
// volume of the wet parts: continuous and non-increasing in c, exact for a linear field, and the
// faces whose four crossings are ambiguous for straight chords (saddle faces) are resolved.
IsoGeom liquid_volume(const OrcMesh& m, int64_t cell, const double* phi, double c, const V3* x0_in) {
  const std::vector<int32_t> vs = cell_vertices(m, cell);
  const int32_t apex = vs[0];
  const V3 x0 = x0_in ? *x0_in : mean_point(m, vs);
  IsoGeom g;
  V3 moment = {0, 0, 0};
  for (int64_t k = m.cell_face_off[cell]; k < m.cell_face_off[cell + 1]; ++k) {
    const std::vector<int32_t> L = loop_of(m, m.cell_face[k]);
    const size_t n = L.size();
    const size_t s = std::min_element(L.begin(), L.end()) - L.begin();
    for (size_t i = 1; i + 1 < n; ++i) {
      const int32_t t0 = L[s], t1 = L[(s + i) % n], t2 = L[(s + i + 1) % n];
      if (t0 == apex || t1 == apex || t2 == apex) continue;
      const VPt T[4] = {{vert(m, apex), phi[apex]}, {vert(m, t0), phi[t0]}, {vert(m, t1), phi[t1]}, {vert(m, t2), phi[t2]}};
      clip_tet(T, c, x0, g, moment);
    }
  }
  if (g.area > 0) g.centroid = mul(moment, 1.0 / g.area);
  return g;
}

// ------------------------------------------------------------------------------ R3
struct RootResult {
  double c = 0;
  int status = 0;
  int evals = 0;
};

RootResult bisect(const OrcMesh& m, int64_t cell, const double* phi, double alpha, double V, double tol,
                  int max_iter) {
  const std::vector<int32_t> vs = cell_vertices(m, cell);
  double lo = phi[vs[0]], hi = phi[vs[0]];
  for (int32_t v : vs) { lo = std::min(lo, phi[v]); hi = std::max(hi, phi[v]); }
  RootResult r;
  if (hi - lo < 1e-14) { r.c = lo; r.status = ST_DEGENERATE; return r; }
  // f(lo) = 1 - alpha (every vertex wet), f(hi) = -alpha (nothing strictly above)
  double best_c = (1 - alpha) <= alpha ? lo : hi, best_f = std::min(1 - alpha, alpha);
  const V3 x0 = mean_point(m, vs);
  for (int it = 0; it < max_iter; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double f = liquid_volume(m, cell, phi, mid, &x0).VL / V - alpha;
    r.evals++;
    if (std::fabs(f) < best_f) { best_f = std::fabs(f); best_c = mid; }
    if (std::fabs(f) <= tol) break;
    if (f > 0) lo = mid; else hi = mid;
    const double scale = std::max(std::fabs(lo), std::fabs(hi));
    if (hi - lo <= 4 * (std::nextafter(scale, 2 * scale + 1) - scale)) break;
  }
  r.c = best_c;
  if (best_f > tol) r.status = ST_NOT_CONVERGED;
  return r;
}

// R3, interval cubic (an alternative to bisection): between two consecutive distinct
// vertex values of the cell no tetrahedron changes its number of wet corners, so V_L(c) is one
// cubic polynomial there (R2 is exact for a linear field on each tetrahedron). Steps: sort the
// cell's distinct vertex values u_0 < ... < u_m; bisect over that list (one evaluation per probe)
// for the pair u_k < u_k+1 with f(u_k) > 0 >= f(u_k+1), where f = V_L/V - alpha, f(u_0) = 1 - alpha
// and f(u_m) = -alpha; interpolate the cubic through f at u_k, u_k + h/3, u_k + 2h/3 and u_k+1
// (h = u_k+1 - u_k, Newton's divided differences on those four points); solve it on the interval
// by bisection on the polynomial, without further cut-volume evaluations; one last evaluation at
// the root checks |f| <= tol.
RootResult interval_cubic(const OrcMesh& m, int64_t cell, const double* phi, double alpha, double V, double tol,
                          int max_iter) {
  const std::vector<int32_t> vs = cell_vertices(m, cell);
  std::vector<double> u;
  for (int32_t v : vs) u.push_back(phi[v]);
  std::sort(u.begin(), u.end());
  u.erase(std::unique(u.begin(), u.end()), u.end());
  RootResult r;
  if (u.back() - u.front() < 1e-14) { r.c = u.front(); r.status = ST_DEGENERATE; return r; }
  const V3 x0 = mean_point(m, vs);
  auto f = [&](double c) {
    r.evals++;
    return liquid_volume(m, cell, phi, c, &x0).VL / V - alpha;
  };
  size_t lo = 0, hi = u.size() - 1;
  double f_lo = 1 - alpha, f_hi = -alpha;
  while (hi - lo > 1) {
    const size_t mid = (lo + hi) / 2;
    const double fm = f(u[mid]);
    if (fm == 0) { r.c = u[mid]; return r; }
    if (fm > 0) { lo = mid; f_lo = fm; } else { hi = mid; f_hi = fm; }
  }
  const double x[4] = {u[lo], u[lo] + (u[hi] - u[lo]) / 3, u[lo] + 2 * (u[hi] - u[lo]) / 3, u[hi]};
  double d[4] = {f_lo, f(x[1]), f(x[2]), f_hi};
  for (int j = 1; j < 4; ++j)  // divided differences, in place
    for (int i = 3; i >= j; --i) d[i] = (d[i] - d[i - 1]) / (x[i] - x[i - j]);
  auto p = [&](double c) { return d[0] + (c - x[0]) * (d[1] + (c - x[1]) * (d[2] + (c - x[2]) * d[3])); };
  double a = x[0], b = x[3];  // p(a) > 0 >= p(b)
  for (int it = 0; it < max_iter; ++it) {
    const double mid = 0.5 * (a + b);
    if (mid <= a || mid >= b) break;
    if (p(mid) > 0) a = mid; else b = mid;
  }
  const double fa = std::fabs(p(a)), fb = std::fabs(p(b));
  r.c = fa <= fb ? a : b;
  if (std::fabs(f(r.c)) > tol) r.status = ST_NOT_CONVERGED;
  return r;
}

// R3, fixed isovalue (the paper's own choice, Sec. 2.1: the iso-surface at a prescribed
// alpha_iso, typically 0.5): no volume matching, c = alpha_iso. A
// cell whose vertex values all lie on one side of it has no interface there (its area is 0).
RootResult fixed_iso(const OrcMesh& m, int64_t cell, const double* phi, double iso) {
  const std::vector<int32_t> vs = cell_vertices(m, cell);
  double lo = phi[vs[0]], hi = phi[vs[0]];
  for (int32_t v : vs) { lo = std::min(lo, phi[v]); hi = std::max(hi, phi[v]); }
  RootResult r;
  if (hi - lo < 1e-14) { r.c = lo; r.status = ST_DEGENERATE; return r; }
  r.c = iso;
  return r;
}

double pairwise_sum(std::vector<double> a) {
  if (a.empty()) return 0.0;
  size_t n = 1;
  while (n < a.size()) n <<= 1;
  a.resize(n, 0.0);
  while (n > 1) {
    for (size_t i = 0; i < n / 2; ++i) a[i] = a[2 * i] + a[2 * i + 1];
    n /= 2;
  }
  return a[0];
}

// ------------------------------------------------------------------------------ S (study)
// Eigenvalues of a symmetric 3x3 matrix by the cyclic Jacobi method (plane rotations that zero
// one off-diagonal entry at a time, swept until the off-diagonal part is negligible).
std::array<double, 3> sym3_eigenvalues(double A[3][3]) {
  double a[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) a[i][j] = A[i][j];
  for (int sweep = 0; sweep < 100; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-34 * dia) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0) continue;
        // rotation angle that zeroes a[p][q]: tan(2 phi) = 2 a_pq / (a_qq - a_pp)
        const double theta = (a[q][q] - a[p][p]) / (2 * a[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        const double c = 1 / std::sqrt(t * t + 1), sn = t * c;
        double b[3][3];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) b[i][j] = a[i][j];
        for (int k = 0; k < 3; ++k) {  // columns p, q of A R
          b[k][p] = c * a[k][p] - sn * a[k][q];
          b[k][q] = sn * a[k][p] + c * a[k][q];
        }
        for (int k = 0; k < 3; ++k) {  // rows p, q of R^T (A R)
          a[p][k] = c * b[p][k] - sn * b[q][k];
          a[q][k] = sn * b[p][k] + c * b[q][k];
          if (k != p && k != q) {
            a[k][p] = b[k][p];
            a[k][q] = b[k][q];
          }
        }
        a[p][q] = a[q][p] = 0;
      }
  }
  std::array<double, 3> e = {a[0][0], a[1][1], a[2][2]};
  std::sort(e.begin(), e.end());
  return e;
}

// R7 with the study's variants (bits of `variant`): 1 the standard stencil (neighbours across the
// interface enter with their own centroid and temperature), 2 inverse-distance weights w = 1/|r|^2
// on every stencil entry, 4 the stencil of every cell sharing a vertex (boundary faces as in R7);
// in the modified stencil a vertex-only neighbour across the interface enters at the linear
// interpolation of alpha along the centroid connection (t = (alpha_P - 1/2)/(alpha_P - alpha_Q)),
// a face neighbour at the face's x_f. cond receives lambda_max / lambda_min of G_P (inf when
// lambda_min <= 0); grad and the singular flag as R7.
void lsq_study(const OrcMesh& m, const double* face_cen, const double* cell_cen, const double* alpha, const double* T,
               const double* T_bnd, double T_sat, const uint8_t* crossing, const double* x_f, const uint8_t* in_band,
               int variant, double* grad, double* cond, int32_t* status) {
  const bool standard = variant & 1, idw = variant & 2, ext = variant & 4;
  const int64_t nc = m.n_cells;
  std::vector<std::vector<int32_t>> cells_of(ext ? m.n_verts : 0);
  if (ext)
    for (int64_t c = 0; c < nc; ++c)
      for (int32_t v : cell_vertices(m, c)) cells_of[v].push_back((int32_t)c);
  for (int64_t c = 0; c < nc; ++c) {
    grad[3 * c] = grad[3 * c + 1] = grad[3 * c + 2] = 0;
    cond[c] = 0;
    if (!in_band[c]) continue;
    const V3 xP = {cell_cen[3 * c], cell_cen[3 * c + 1], cell_cen[3 * c + 2]};
    double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0};
    auto add_entry = [&](const V3& r, double dT) {
      const double w = idw ? 1.0 / dot(r, r) : 1.0;
      for (int i = 0; i < 3; ++i) {
        b[i] += w * r[i] * dT;
        for (int j = 0; j < 3; ++j) G[i][j] += w * r[i] * r[j];
      }
    };
    std::map<int32_t, int32_t> face_to;  // face neighbour -> face
    for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
      const int32_t f = m.cell_face[k] & 0x7fffffff;
      const int32_t q = m.face_owner[f] == c ? m.face_neigh[f] : m.face_owner[f];
      if (q < 0) {
        if (T_bnd) add_entry(sub({face_cen[3 * f], face_cen[3 * f + 1], face_cen[3 * f + 2]}, xP), T_bnd[f] - T[c]);
        continue;
      }
      face_to[q] = f;
    }
    std::vector<int32_t> nbrs;
    if (ext) {
      std::vector<int32_t> all;
      for (int32_t v : cell_vertices(m, c))
        for (int32_t q : cells_of[v])
          if (q != c) all.push_back(q);
      std::sort(all.begin(), all.end());
      all.erase(std::unique(all.begin(), all.end()), all.end());
      nbrs = all;
    } else {
      for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
        const int32_t f = m.cell_face[k] & 0x7fffffff;
        const int32_t q = m.face_owner[f] == c ? m.face_neigh[f] : m.face_owner[f];
        if (q >= 0) nbrs.push_back(q);
      }
    }
    for (int32_t q : nbrs) {
      const V3 xQ = {cell_cen[3 * q], cell_cen[3 * q + 1], cell_cen[3 * q + 2]};
      const bool across = (alpha[c] - 0.5) * (alpha[q] - 0.5) < 0;
      if (standard || !across) {
        add_entry(sub(xQ, xP), T[q] - T[c]);
        continue;
      }
      const auto it = face_to.find(q);
      V3 xs;
      if (it != face_to.end() && crossing[it->second]) {
        const int32_t f = it->second;
        xs = {x_f[3 * f], x_f[3 * f + 1], x_f[3 * f + 2]};
      } else {
        const double t = (alpha[c] - 0.5) / (alpha[c] - alpha[q]);
        xs = add(xP, mul(sub(xQ, xP), t));
      }
      add_entry(sub(xs, xP), T_sat - T[c]);
    }
    const auto ev = sym3_eigenvalues(G);
    cond[c] = ev[0] > 0 ? ev[2] / ev[0] : INFINITY;
    const double det = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                       G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                       G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    const double tr = (G[0][0] + G[1][1] + G[2][2]) / 3.0;
    if (!(det > 1e-12 * tr * tr * tr)) {
      status[c] |= ST_SINGULAR_LSQ;
      continue;
    }
    double Gi[3][3];
    Gi[0][0] = (G[1][1] * G[2][2] - G[1][2] * G[2][1]) / det;
    Gi[0][1] = (G[0][2] * G[2][1] - G[0][1] * G[2][2]) / det;
    Gi[0][2] = (G[0][1] * G[1][2] - G[0][2] * G[1][1]) / det;
    Gi[1][1] = (G[0][0] * G[2][2] - G[0][2] * G[2][0]) / det;
    Gi[1][2] = (G[0][2] * G[1][0] - G[0][0] * G[1][2]) / det;
    Gi[2][2] = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) / det;
    Gi[1][0] = Gi[0][1];
    Gi[2][0] = Gi[0][2];
    Gi[2][1] = Gi[1][2];
    for (int i = 0; i < 3; ++i) grad[3 * c + i] = Gi[i][0] * b[0] + Gi[i][1] * b[1] + Gi[i][2] * b[2];
  }
}

}  // namespace

extern "C" {

int orc_version() { return 1; }

void orc_geometry(const OrcMesh* m, double* face_area, double* face_cen, double* cell_vol, double* cell_cen) {
  geometry(*m, face_area, face_cen, cell_vol, cell_cen);
}

// R1: phi_v = sum_c w alpha_c / sum_c w over the cells around v; w = 1/|x_v - x_c| (mode 0) or 1 (mode 1).
void orc_vertex_field(const OrcMesh* mp, const double* cell_cen, const double* alpha, int mode, double* phi) {
  const OrcMesh& m = *mp;
  std::vector<double> num(m.n_verts, 0.0), den(m.n_verts, 0.0);
  for (int64_t c = 0; c < m.n_cells; ++c) {
    const V3 xc = {cell_cen[3 * c], cell_cen[3 * c + 1], cell_cen[3 * c + 2]};
    for (int32_t v : cell_vertices(m, c)) {
      const double w = mode == 0 ? 1.0 / norm(sub(vert(m, v), xc)) : 1.0;
      num[v] += w * alpha[c];
      den[v] += w;
    }
  }
  for (int64_t v = 0; v < m.n_verts; ++v) phi[v] = den[v] > 0 ? num[v] / den[v] : 0.0;
}

// R2 for one cell. out[0..8] = V_L, area, vec_area(3), centroid(3), nloops. x0 may be null
// (vertex mean of the cell).
void orc_liquid_volume(const OrcMesh* m, int64_t cell, const double* phi, double c, const double* x0, double* out) {
  V3 p;
  if (x0) p = {x0[0], x0[1], x0[2]};
  const IsoGeom g = liquid_volume(*m, cell, phi, c, x0 ? &p : nullptr);
  out[0] = g.VL;
  out[1] = g.area;
  for (int k = 0; k < 3; ++k) { out[2 + k] = g.vec_area[k]; out[5 + k] = g.centroid[k]; }
  out[8] = 0;
}

// R0 + R3 + geometry at the root for every cell with eps < alpha < 1 - eps (other cells get
// iso = nan, status 0, evals 0, zero geometry). Arrays are [n_cells] or [3 n_cells].
// `cells`, when non-null, restricts the work to the listed cells (n_list of them).
// method 0: bisection (R3); 1: interval cubic (R3); 2: fixed isovalue iso_fixed.
void orc_reconstruct_m(const OrcMesh* mp, const double* alpha, const double* phi, const double* cell_vol, double eps,
                       double tol, int max_iter, const int64_t* cells, int64_t n_list, int method, double iso_fixed,
                       double* iso,
                       int32_t* status, int32_t* evals, double* A_int, double* n_int, double* x_gamma, int32_t* nloops) {
  const OrcMesh& m = *mp;
  std::vector<int64_t> todo;
  if (cells) {
    todo.assign(cells, cells + n_list);
  } else {
    for (int64_t c = 0; c < m.n_cells; ++c)
      if (alpha[c] > eps && alpha[c] < 1 - eps) todo.push_back(c);
  }
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < (int64_t)todo.size(); ++t) {
    const int64_t c = todo[t];
    const RootResult r = method == 1   ? interval_cubic(m, c, phi, alpha[c], cell_vol[c], tol, max_iter)
                         : method == 2 ? fixed_iso(m, c, phi, iso_fixed)
                                       : bisect(m, c, phi, alpha[c], cell_vol[c], tol, max_iter);
    iso[c] = r.c;
    status[c] = r.status;
    evals[c] = r.evals;
    IsoGeom g;
    if (!(r.status & ST_DEGENERATE)) g = liquid_volume(m, c, phi, r.c, nullptr);
    A_int[c] = g.area;
    const double vn = norm(g.vec_area);
    for (int k = 0; k < 3; ++k) {
      n_int[3 * c + k] = vn > 0 ? -g.vec_area[k] / vn : 0.0;  // vapour -> liquid
      x_gamma[3 * c + k] = g.centroid[k];
    }
    nloops[c] = 0;
  }
}

void orc_reconstruct(const OrcMesh* mp, const double* alpha, const double* phi, const double* cell_vol, double eps,
                     double tol, int max_iter, const int64_t* cells, int64_t n_list, double* iso, int32_t* status,
                     int32_t* evals, double* A_int, double* n_int, double* x_gamma, int32_t* nloops) {
  orc_reconstruct_m(mp, alpha, phi, cell_vol, eps, tol, max_iter, cells, n_list, 0, 0.5, iso, status, evals, A_int,
                    n_int, x_gamma, nloops);
}

// R4: crossing point of face f (owner o, neighbour n); returns t along x_o -> x_n, and the cell
// whose interface plane gave it (-1 for the alpha-interpolated fallback).
//   xf_mode 0 RECON: intersection with the interface plane (x_gamma, n_int) of an interface cell
//           (the one nearest the face centroid when both qualify), t in [0, 1]; else mode 1.
//   xf_mode 1 LINEAR: t = (alpha_o - 1/2)/(alpha_o - alpha_n).
//   xf_mode 2 AS PRINTED in Eq. front_interpolation: t = |alpha_n - 1/2| / |alpha_o - alpha_n|.
double crossing_t(const OrcMesh& m, int64_t f, const double* alpha, const double* cell_cen, const double* face_cen,
                  const uint8_t* is_iface, const double* n_int, const double* x_gamma, int xf_mode, int32_t* src) {
  const int32_t o = m.face_owner[f], n = m.face_neigh[f];
  *src = -1;
  if (xf_mode == 2) return std::fabs(alpha[n] - 0.5) / std::fabs(alpha[o] - alpha[n]);
  const double t_lin = (alpha[o] - 0.5) / (alpha[o] - alpha[n]);
  if (xf_mode == 1) return t_lin;
  const V3 xo = {cell_cen[3 * o], cell_cen[3 * o + 1], cell_cen[3 * o + 2]};
  const V3 xn = {cell_cen[3 * n], cell_cen[3 * n + 1], cell_cen[3 * n + 2]};
  const V3 xfc = {face_cen[3 * f], face_cen[3 * f + 1], face_cen[3 * f + 2]};
  double best_t = 0, best_d = 0;
  for (int32_t c : {o, n}) {
    if (!is_iface[c]) continue;
    const V3 nn = {n_int[3 * c], n_int[3 * c + 1], n_int[3 * c + 2]};
    const V3 xg = {x_gamma[3 * c], x_gamma[3 * c + 1], x_gamma[3 * c + 2]};
    const double den = dot(nn, sub(xn, xo));
    if (den == 0) continue;
    const double t = dot(nn, sub(xg, xo)) / den;
    if (!(t >= 0 && t <= 1)) continue;
    // nearest by squared distance: the same order as the distance, without a square root
    const V3 r = sub(add(xo, mul(sub(xn, xo), t)), xfc);
    const double d = dot(r, r);
    if (*src < 0 || d < best_d) { best_t = t; best_d = d; *src = c; }
  }
  return *src >= 0 ? best_t : t_lin;
}

// Pseudo-time step of Eq. (extrapolation): the smallest |d_f| over the mesh's faces, d_f the vector
// from a face's owner centroid to its neighbour centroid (to the face centroid on a boundary face,
// where the boundary value sits).
double extrap_dtau(const OrcMesh& m, const double* cell_cen, const double* face_cen) {
  double d = INFINITY;
  for (int64_t f = 0; f < m.n_faces; ++f) {
    const int32_t o = m.face_owner[f], n = m.face_neigh[f];
    const V3 xo = {cell_cen[3 * o], cell_cen[3 * o + 1], cell_cen[3 * o + 2]};
    const V3 xn = n >= 0 ? V3{cell_cen[3 * n], cell_cen[3 * n + 1], cell_cen[3 * n + 2]}
                         : V3{face_cen[3 * f], face_cen[3 * f + 1], face_cen[3 * f + 2]};
    d = std::min(d, norm(sub(xn, xo)));
  }
  return d;
}

// Eq. (extrapolation) in pseudo-time, once per side and per gradient component. The field phi
// starts as the modified LSQ gradient component of every cell. Information travels from the bulk
// of a side towards and across the interface (the text's direction): the liquid side moves along
// -n_int, the vapour side along +n_int. The unknowns of a side are the interface cells (A_int > 0)
// of the other phase; every cell of the side itself keeps its gradient. First-order upwind: at an
// unknown P the inflow faces are those whose outward area A_f has w = sigma n_P . A_f > 0
// (sigma = +1 for the liquid side, -1 for the vapour side), and a face counts when its neighbour
// is a cell of the side (known) or an unknown of the same solve; others carry no value of this
// side and are left out. One explicit step (Jacobi: every unknown from the previous iterate):
//   phi_P <- phi_P + (dtau_P / V_P) sum_f w_f (phi_Q - phi_P),
// dtau_P = min(dtau, V_P / sum_f w_f): the global step, limited where it would exceed the cell's
// upwind Courant limit, so that each step is a convex combination. The solve stops after the
// iteration whose largest change over its unknowns is below tol, or after max_iter. An unknown
// with no counted inflow face keeps its initial value and is flagged ST_NO_SIDE.
void extrapolate(const OrcMesh& m, const double* face_area, const double* cell_vol, const double* alpha,
                 const uint8_t* iface, const double* n_int, const double* grad, double dtau, int max_iter, double tol,
                 double* g_other, int32_t* iters, int32_t* status) {
  const int64_t nc = m.n_cells;
  for (int side = 0; side < 2; ++side) {  // 0 liquid, 1 vapour
    const double sigma = side == 0 ? 1.0 : -1.0;
    auto of_side = [&](int64_t c) { return (alpha[c] > 0.5) == (side == 0); };
    std::vector<uint8_t> unknown(nc, 0);
    for (int64_t c = 0; c < nc; ++c) unknown[c] = iface[c] && !of_side(c);
    for (int j = 0; j < 3; ++j) {
      std::vector<double> phi(nc);
      for (int64_t c = 0; c < nc; ++c) phi[c] = grad[3 * c + j];
      int k = 1;
      for (;; ++k) {
        std::vector<double> next = phi;
        double change = 0;
        for (int64_t P = 0; P < nc; ++P) {
          if (!unknown[P]) continue;
          const V3 nn = {n_int[3 * P], n_int[3 * P + 1], n_int[3 * P + 2]};
          std::vector<std::pair<double, int32_t>> in;  // (w_f, Q) of the counted inflow faces
          double wsum = 0;
          for (int64_t e = m.cell_face_off[P]; e < m.cell_face_off[P + 1]; ++e) {
            const int32_t fe = m.cell_face[e];
            const int32_t f = fe & 0x7fffffff;
            const int32_t Q = m.face_owner[f] == P ? m.face_neigh[f] : m.face_owner[f];
            if (Q < 0) continue;
            V3 Af = {face_area[3 * f], face_area[3 * f + 1], face_area[3 * f + 2]};
            if (fe < 0) Af = mul(Af, -1.0);  // outward from P
            const double w = sigma * dot(nn, Af);
            if (!(w > 0)) continue;
            if (!of_side(Q) && !unknown[Q]) continue;
            in.push_back({w, Q});
            wsum += w;
          }
          if (wsum == 0) {
            if (j == 0 && k == 1) status[P] |= ST_NO_SIDE;
            continue;
          }
          const double dtau_P = std::min(dtau, cell_vol[P] / wsum);
          double s = 0;
          for (const auto& [w, Q] : in) s += w * (phi[Q] - phi[P]);
          next[P] = phi[P] + dtau_P / cell_vol[P] * s;
          change = std::max(change, std::fabs(next[P] - phi[P]));
        }
        phi.swap(next);
        if (change < tol || k >= max_iter) break;
      }
      iters[3 * side + j] = k;
      for (int64_t c = 0; c < nc; ++c)
        if (unknown[c]) g_other[3 * c + j] = phi[c];
    }
  }
}

// R4-R8. Inputs: geometry (from orc_geometry), alpha, reconstruction (iso/status/A_int/n_int/
// x_gamma arrays from orc_reconstruct), T at cells, T at boundary faces (may be null: boundary
// faces then stay out of the stencil), properties; ex = null for R5's single sweep, else the
// options of the pseudo-time solve, whose iteration counts it returns.
// Outputs ([n_cells] or [3 n_cells]): band flag, grad (modified LSQ) on band cells, grad_l,
// grad_v, q_l, q_v, mdot, Q on interface cells, status bits (ORed into `status`);
// per face: crossing flag, x_f, d_own, d_neigh, A_int_f; totals[0..1] = sum mdot V, sum Q V.
void orc_phase_change(const OrcMesh* mp, const double* face_area, const double* face_cen, const double* cell_vol,
                      const double* cell_cen, const double* alpha, double eps, const double* A_int, const double* n_int,
                      const double* x_gamma, const double* T, const double* T_bnd, const OrcProps* pr, int xf_mode,
                      uint8_t* in_band, double* grad, double* grad_l, double* grad_v, double* q_l, double* q_v,
                      double* mdot, double* Qph, int32_t* status, uint8_t* crossing, double* x_f, double* d_own,
                      double* d_neigh, double* A_int_f, double* totals, OrcExtrap* ex) {
  const OrcMesh& m = *mp;
  const int64_t nc = m.n_cells;
  std::vector<uint8_t> iface(nc, 0);
  for (int64_t c = 0; c < nc; ++c) iface[c] = alpha[c] > eps && alpha[c] < 1 - eps && A_int[c] > 0;
  std::vector<uint8_t> in_I(nc, 0);
  for (int64_t c = 0; c < nc; ++c) in_I[c] = alpha[c] > eps && alpha[c] < 1 - eps;
  // band = interface cells and their face neighbours
  std::memset(in_band, 0, nc);
  for (int64_t c = 0; c < nc; ++c) {
    if (!in_I[c]) continue;
    in_band[c] = 1;
    for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
      const int32_t f = m.cell_face[k] & 0x7fffffff;
      const int32_t q = m.face_owner[f] == c ? m.face_neigh[f] : m.face_owner[f];
      if (q >= 0) in_band[q] = 1;
    }
  }
  // R4 on every crossing face
  auto is_crossing = [&](int64_t f) {
    const int32_t o = m.face_owner[f], n = m.face_neigh[f];
    return n >= 0 && (alpha[o] - 0.5) * (alpha[n] - 0.5) < 0;
  };
  for (int64_t f = 0; f < m.n_faces; ++f) {
    crossing[f] = is_crossing(f);
    x_f[3 * f] = x_f[3 * f + 1] = x_f[3 * f + 2] = 0;
    d_own[f] = d_neigh[f] = A_int_f[f] = 0;
    if (!crossing[f]) continue;
    const int32_t o = m.face_owner[f], n = m.face_neigh[f];
    int32_t src;
    const double t = crossing_t(m, f, alpha, cell_cen, face_cen, iface.data(), n_int, x_gamma, xf_mode, &src);
    const V3 xo = {cell_cen[3 * o], cell_cen[3 * o + 1], cell_cen[3 * o + 2]};
    const V3 xn = {cell_cen[3 * n], cell_cen[3 * n + 1], cell_cen[3 * n + 2]};
    const V3 x = add(xo, mul(sub(xn, xo), t));
    for (int k = 0; k < 3; ++k) x_f[3 * f + k] = x[k];
    d_own[f] = norm(sub(x, xo));
    d_neigh[f] = norm(sub(x, xn));
    // interface area projected onto the face (Eq. interface_htc): |A_int n_int . n_f|
    int32_t a = src >= 0 ? src : (iface[o] ? o : (iface[n] ? n : -1));
    if (a >= 0) {
      const V3 Af = {face_area[3 * f], face_area[3 * f + 1], face_area[3 * f + 2]};
      const V3 nn = {n_int[3 * a], n_int[3 * a + 1], n_int[3 * a + 2]};
      A_int_f[f] = std::fabs(A_int[a] * dot(nn, Af) / norm(Af));
    }
  }
  // R7: interface-modified least squares on band cells
  for (int64_t c = 0; c < nc; ++c) {
    grad[3 * c] = grad[3 * c + 1] = grad[3 * c + 2] = 0;
    if (!in_band[c]) continue;
    const V3 xP = {cell_cen[3 * c], cell_cen[3 * c + 1], cell_cen[3 * c + 2]};
    double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0};
    for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
      const int32_t f = m.cell_face[k] & 0x7fffffff;
      const int32_t q = m.face_owner[f] == c ? m.face_neigh[f] : m.face_owner[f];
      V3 r;
      double dT;
      if (q >= 0) {
        if (crossing[f]) {
          r = sub({x_f[3 * f], x_f[3 * f + 1], x_f[3 * f + 2]}, xP);
          dT = pr->T_sat - T[c];
        } else {
          r = sub({cell_cen[3 * q], cell_cen[3 * q + 1], cell_cen[3 * q + 2]}, xP);
          dT = T[q] - T[c];
        }
      } else {
        if (!T_bnd) continue;
        r = sub({face_cen[3 * f], face_cen[3 * f + 1], face_cen[3 * f + 2]}, xP);
        dT = T_bnd[f] - T[c];
      }
      for (int i = 0; i < 3; ++i) {
        b[i] += r[i] * dT;
        for (int j = 0; j < 3; ++j) G[i][j] += r[i] * r[j];
      }
    }
    const double det = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                       G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                       G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    const double tr = (G[0][0] + G[1][1] + G[2][2]) / 3.0;
    if (!(det > 1e-12 * tr * tr * tr)) {
      status[c] |= ST_SINGULAR_LSQ;
      continue;
    }
    // explicit symmetric inverse (cofactors / det)
    double Gi[3][3];
    Gi[0][0] = (G[1][1] * G[2][2] - G[1][2] * G[2][1]) / det;
    Gi[0][1] = (G[0][2] * G[2][1] - G[0][1] * G[2][2]) / det;
    Gi[0][2] = (G[0][1] * G[1][2] - G[0][2] * G[1][1]) / det;
    Gi[1][1] = (G[0][0] * G[2][2] - G[0][2] * G[2][0]) / det;
    Gi[1][2] = (G[0][2] * G[1][0] - G[0][0] * G[1][2]) / det;
    Gi[2][2] = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) / det;
    Gi[1][0] = Gi[0][1];
    Gi[2][0] = Gi[0][2];
    Gi[2][1] = Gi[1][2];
    for (int i = 0; i < 3; ++i) grad[3 * c + i] = Gi[i][0] * b[0] + Gi[i][1] * b[1] + Gi[i][2] * b[2];
  }
  // the pseudo-time solve (when asked): the other side's gradient of every interface cell from the pseudo-time solve
  std::vector<double> g_n2;
  if (ex) {
    g_n2.assign(3 * nc, 0.0);
    const double dtau = ex->dtau > 0 ? ex->dtau : extrap_dtau(m, cell_cen, face_cen);
    extrapolate(m, face_area, cell_vol, alpha, iface.data(), n_int, grad, dtau, ex->max_iter, ex->tol, g_n2.data(),
                ex->iters, status);
  }
  // R5 + R6 on interface cells
  std::vector<double> mv, qv;
  for (int64_t c = 0; c < nc; ++c) {
    for (int k = 0; k < 3; ++k) grad_l[3 * c + k] = grad_v[3 * c + k] = 0;
    q_l[c] = q_v[c] = mdot[c] = Qph[c] = 0;
    if (!in_I[c]) continue;
    if (iface[c]) {
      const V3 nn = {n_int[3 * c], n_int[3 * c + 1], n_int[3 * c + 2]};
      const bool P_liquid = alpha[c] > 0.5;
      const double sigma = P_liquid ? -1.0 : 1.0;  // other side: vapour (-1) or liquid (+1)
      V3 acc = {0, 0, 0};
      double wsum = 0;
      for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
        const int32_t fe = m.cell_face[k];
        const int32_t f = fe & 0x7fffffff;
        const int32_t q = m.face_owner[f] == c ? m.face_neigh[f] : m.face_owner[f];
        if (q < 0) continue;
        if ((alpha[q] > 0.5) == P_liquid) continue;  // same phase as P
        V3 Af = {face_area[3 * f], face_area[3 * f + 1], face_area[3 * f + 2]};
        if (fe < 0) Af = mul(Af, -1.0);  // outward from P
        const double w = std::max(0.0, sigma * dot(nn, Af));
        acc = add(acc, mul({grad[3 * q], grad[3 * q + 1], grad[3 * q + 2]}, w));
        wsum += w;
      }
      V3 g_other = {0, 0, 0};
      if (ex) g_other = {g_n2[3 * c], g_n2[3 * c + 1], g_n2[3 * c + 2]};
      else if (wsum > 0) g_other = mul(acc, 1.0 / wsum);
      else status[c] |= ST_NO_SIDE;
      const V3 g_own = {grad[3 * c], grad[3 * c + 1], grad[3 * c + 2]};
      const V3 gl = P_liquid ? g_own : g_other;
      const V3 gv = P_liquid ? g_other : g_own;
      for (int k = 0; k < 3; ++k) { grad_l[3 * c + k] = gl[k]; grad_v[3 * c + k] = gv[k]; }
      q_l[c] = pr->k_l * dot(gl, nn) * A_int[c];
      q_v[c] = -pr->k_v * dot(gv, nn) * A_int[c];
      mdot[c] = (q_l[c] + q_v[c]) / (pr->h_lv * cell_vol[c]);
      Qph[c] = -mdot[c] * pr->h_lv;
    }
    mv.push_back(mdot[c] * cell_vol[c]);
    qv.push_back(Qph[c] * cell_vol[c]);
  }
  totals[0] = pairwise_sum(mv);
  totals[1] = pairwise_sum(qv);
}

// Eq. interface_htc: on each side of a crossing face the interface
// heat-transfer coefficient a_f = k_phi A_int,f / d_f, k_phi the conductivity of the phase the cell
// resides in (liquid when alpha > 1/2) and d_f the cell centre's distance to the crossing point;
// 0 on other faces. The cell adds a_f to its energy-matrix diagonal and a_f T_sat to its
// right-hand side (the face itself is detached from the diffusive coupling).
void orc_interface_htc(const OrcMesh* mp, const double* alpha, const uint8_t* crossing, const double* A_int_f,
                       const double* d_own, const double* d_neigh, double k_l, double k_v, double* a_own,
                       double* a_neigh) {
  const OrcMesh& m = *mp;
  for (int64_t f = 0; f < m.n_faces; ++f) {
    a_own[f] = a_neigh[f] = 0;
    if (!crossing[f]) continue;
    const double ko = alpha[m.face_owner[f]] > 0.5 ? k_l : k_v;
    const double kn = alpha[m.face_neigh[f]] > 0.5 ? k_l : k_v;
    if (d_own[f] > 0) a_own[f] = ko * A_int_f[f] / d_own[f];
    if (d_neigh[f] > 0) a_neigh[f] = kn * A_int_f[f] / d_neigh[f];
  }
}

// Eq. interface_htc's place in the energy equation: a cell whose face f is detached
// from the diffusive coupling by the interface adds a_f to its matrix diagonal and a_f T_sat to its
// right-hand side. Per cell, over its faces in the cell's face order: diag = sum a_f, rhs =
// sum a_f T_sat, with a_f the coefficient of the cell's own side of the face.
void orc_htc_cell_sums(const OrcMesh* mp, const uint8_t* crossing, const double* a_own, const double* a_neigh,
                       double T_sat, double* diag, double* rhs) {
  const OrcMesh& m = *mp;
  for (int64_t c = 0; c < m.n_cells; ++c) {
    double d = 0, r = 0;
    for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
      const int32_t f = m.cell_face[k] & 0x7fffffff;
      if (!crossing[f]) continue;
      const double a = m.face_owner[f] == c ? a_own[f] : a_neigh[f];
      d += a;
      r += a * T_sat;
    }
    diag[c] = d;
    rhs[c] = r;
  }
}

// The pseudo-time solve alone, on a given gradient field: g_other [3 n_cells] receives the other side's gradient of
// every interface cell (iface[c] != 0; its phase: liquid when alpha > 1/2), iters[6] the counts.
void orc_extrapolate(const OrcMesh* m, const double* face_area, const double* cell_vol, const double* alpha,
                     const uint8_t* iface, const double* n_int, const double* grad, double dtau, int max_iter,
                     double tol, double* g_other, int32_t* iters, int32_t* status) {
  extrapolate(*m, face_area, cell_vol, alpha, iface, n_int, grad, dtau, max_iter, tol, g_other, iters, status);
}

// S: the study's least-squares variants on the band (see lsq_study).
void orc_lsq_study(const OrcMesh* m, const double* face_cen, const double* cell_cen, const double* alpha,
                   const double* T, const double* T_bnd, double T_sat, const uint8_t* crossing, const double* x_f,
                   const uint8_t* in_band, int variant, double* grad, double* cond, int32_t* status) {
  lsq_study(*m, face_cen, cell_cen, alpha, T, T_bnd, T_sat, crossing, x_f, in_band, variant, grad, cond, status);
}

void orc_sym3_eigenvalues(const double* A9, double* out3) {
  double A[3][3];
  for (int i = 0; i < 9; ++i) A[i / 3][i % 3] = A9[i];
  const auto e = sym3_eigenvalues(A);
  for (int i = 0; i < 3; ++i) out3[i] = e[i];
}

void orc_extrap_dtau(const OrcMesh* m, const double* cell_cen, const double* face_cen, double* out) {
  *out = extrap_dtau(*m, cell_cen, face_cen);
}

void orc_pairwise_sum(const double* a, int64_t n, double* out) { *out = pairwise_sum(std::vector<double>(a, a + n)); }

}  // extern "C"
