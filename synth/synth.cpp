// Seeded synthetic inputs: polyhedral meshes and the alpha / temperature fields that are laid on
// them. This module produces inputs only. It holds none of the reconstruction, gradient or
// phase-change arithmetic; the oracle and the CUDA library each derive their own geometry
// (volumes, centroids, face areas) from the primitive arrays written here.
//
// Mesh format (shared by every consumer):
//   vertices  vx, vy, vz                 float64 [n_verts]
//   faces     face_vert_off [n_faces+1]  int64, face_vert int32: vertex loop, counter-clockwise
//             seen from outside the owner cell (i.e. oriented outward from the owner)
//             face_owner, face_neigh     int32 (neigh = -1 on the domain boundary)
//   cells     cell_face_off [n_cells+1]  int64, cell_face int32: face id, bit 31 set when the
//             face loop is inward for this cell (the cell is the face's neighbour)
//
// Meshes: uniform hex, 6-tet (Kuhn) split hex, 2-prism split hex, jittered-BCC Voronoi clipped to
// a box, and an extruded jittered 2D Voronoi disk (pipe). Voronoi vertices are identified by the
// sorted set of the four generators (sites or box planes) that define them and their coordinates
// are computed once from that key, so neighbouring cells share vertices bit for bit.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <random>
#include <string_view>
#include <unordered_map>
#include <vector>

namespace {

struct Mesh {
  std::vector<double> vx, vy, vz;
  std::vector<int64_t> face_vert_off{0};
  std::vector<int32_t> face_vert, face_owner, face_neigh;
  std::vector<int64_t> cell_face_off{0};
  std::vector<int32_t> cell_face;
  int64_t n_cells = 0;
  int64_t conform_errors = 0;  // faces whose two cells disagree on the vertex loop
  std::string_view kind;
};

constexpr double kPi = 3.14159265358979323846;
constexpr int32_t REV = int32_t(0x80000000u);

// Builds cell_face from owner/neigh (faces listed in face-id order per cell).
void build_cell_faces(Mesh& m) {
  const int64_t nf = (int64_t)m.face_owner.size();
  std::vector<int64_t> cnt(m.n_cells + 1, 0);
  for (int64_t f = 0; f < nf; ++f) {
    cnt[m.face_owner[f] + 1]++;
    if (m.face_neigh[f] >= 0) cnt[m.face_neigh[f] + 1]++;
  }
  for (int64_t c = 0; c < m.n_cells; ++c) cnt[c + 1] += cnt[c];
  m.cell_face_off = cnt;
  m.cell_face.assign(cnt[m.n_cells], 0);
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  for (int64_t f = 0; f < nf; ++f) {
    m.cell_face[pos[m.face_owner[f]]++] = (int32_t)f;
    if (m.face_neigh[f] >= 0) m.cell_face[pos[m.face_neigh[f]]++] = (int32_t)f | REV;
  }
}

void add_face(Mesh& m, const int32_t* v, int n, int32_t owner, int32_t neigh) {
  for (int i = 0; i < n; ++i) m.face_vert.push_back(v[i]);
  m.face_vert_off.push_back((int64_t)m.face_vert.size());
  m.face_owner.push_back(owner);
  m.face_neigh.push_back(neigh);
}

// ---------------------------------------------------------------- structured hex-based meshes
struct Grid {
  int nx, ny, nz;
  double lo[3], hi[3];
  int32_t vid(int i, int j, int k) const { return (int32_t)((int64_t)(k * (ny + 1) + j) * (nx + 1) + i); }
  void fill_vertices(Mesh& m) const {
    for (int k = 0; k <= nz; ++k)
      for (int j = 0; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
          m.vx.push_back(lo[0] + (hi[0] - lo[0]) * i / nx);
          m.vy.push_back(lo[1] + (hi[1] - lo[1]) * j / ny);
          m.vz.push_back(lo[2] + (hi[2] - lo[2]) * k / nz);
        }
  }
};

// Generic conforming assembly: every cell is given as a list of faces (vertex loops oriented
// outward from that cell). Interior faces are matched through their sorted vertex set.
struct Assembler {
  Mesh& m;
  std::map<std::vector<int32_t>, int64_t> open;  // sorted verts -> face id waiting for a partner
  explicit Assembler(Mesh& mm) : m(mm) {}
  void cell_face(int32_t cell, std::vector<int32_t> loop) {
    std::vector<int32_t> key = loop;
    std::sort(key.begin(), key.end());
    auto it = open.find(key);
    if (it == open.end()) {
      open.emplace(std::move(key), (int64_t)m.face_owner.size());
      add_face(m, loop.data(), (int)loop.size(), cell, -1);
    } else {
      const int64_t f = it->second;
      // the partner must traverse the loop in the opposite direction
      const int64_t o = m.face_vert_off[f];
      const int n = (int)(m.face_vert_off[f + 1] - o);
      bool ok = (n == (int)loop.size());
      if (ok) {
        int s = -1;
        for (int i = 0; i < n; ++i)
          if (m.face_vert[o + i] == loop[0]) s = i;
        ok = s >= 0;
        for (int i = 0; ok && i < n; ++i)
          ok = m.face_vert[o + ((s - i) % n + n) % n] == loop[i];
      }
      if (!ok) m.conform_errors++;
      m.face_neigh[f] = cell;
      open.erase(it);
    }
  }
};

Mesh* make_hex(int nx, int ny, int nz, const double* lo, const double* hi) {
  auto* m = new Mesh;
  m->kind = "hex";
  Grid g{nx, ny, nz, {lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}};
  g.fill_vertices(*m);
  m->n_cells = (int64_t)nx * ny * nz;
  auto cid = [&](int i, int j, int k) { return (int32_t)((int64_t)(k * ny + j) * nx + i); };
  // x-faces
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        int32_t v[4] = {g.vid(i, j, k), g.vid(i, j + 1, k), g.vid(i, j + 1, k + 1), g.vid(i, j, k + 1)};
        if (i == 0) {  // boundary, owner is cell (0,j,k), outward = -x
          int32_t r[4] = {v[0], v[3], v[2], v[1]};
          add_face(*m, r, 4, cid(0, j, k), -1);
        } else {  // owner (i-1), outward +x: loop CCW seen from +x
          add_face(*m, v, 4, cid(i - 1, j, k), i < nx ? cid(i, j, k) : -1);
        }
      }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int32_t v[4] = {g.vid(i, j, k), g.vid(i, j, k + 1), g.vid(i + 1, j, k + 1), g.vid(i + 1, j, k)};
        if (j == 0) {
          int32_t r[4] = {v[0], v[3], v[2], v[1]};
          add_face(*m, r, 4, cid(i, 0, k), -1);
        } else {
          add_face(*m, v, 4, cid(i, j - 1, k), j < ny ? cid(i, j, k) : -1);
        }
      }
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int32_t v[4] = {g.vid(i, j, k), g.vid(i + 1, j, k), g.vid(i + 1, j + 1, k), g.vid(i, j + 1, k)};
        if (k == 0) {
          int32_t r[4] = {v[0], v[3], v[2], v[1]};
          add_face(*m, r, 4, cid(i, j, 0), -1);
        } else {
          add_face(*m, v, 4, cid(i, j, k - 1), k < nz ? cid(i, j, k) : -1);
        }
      }
  build_cell_faces(*m);
  return m;
}

// Orients a triangle (a,b,c) outward from a cell whose interior contains point q.
void tri_out(const Mesh& m, int32_t* t, const double* q) {
  const double ax = m.vx[t[0]], ay = m.vy[t[0]], az = m.vz[t[0]];
  const double ux = m.vx[t[1]] - ax, uy = m.vy[t[1]] - ay, uz = m.vz[t[1]] - az;
  const double wx = m.vx[t[2]] - ax, wy = m.vy[t[2]] - ay, wz = m.vz[t[2]] - az;
  const double nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
  if (nx * (ax - q[0]) + ny * (ay - q[1]) + nz * (az - q[2]) < 0) std::swap(t[1], t[2]);
}
void quad_out(const Mesh& m, int32_t* v, const double* q) {
  int32_t t[3] = {v[0], v[1], v[2]};
  tri_out(m, t, q);
  if (t[1] != v[1]) std::swap(v[1], v[3]);
}

// Kuhn (Freudenthal) split of each hex into 6 tets sharing the main diagonal; conforming.
Mesh* make_tet(int nx, int ny, int nz, const double* lo, const double* hi) {
  auto* m = new Mesh;
  m->kind = "tet";
  Grid g{nx, ny, nz, {lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}};
  g.fill_vertices(*m);
  Assembler as(*m);
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int32_t cell = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        for (int p = 0; p < 6; ++p) {
          int c[3] = {i, j, k};
          int32_t tv[4];
          tv[0] = g.vid(c[0], c[1], c[2]);
          for (int s = 0; s < 3; ++s) {
            c[perms[p][s]]++;
            tv[s + 1] = g.vid(c[0], c[1], c[2]);
          }
          double q[3] = {0, 0, 0};
          for (int a = 0; a < 4; ++a) {
            q[0] += 0.25 * m->vx[tv[a]];
            q[1] += 0.25 * m->vy[tv[a]];
            q[2] += 0.25 * m->vz[tv[a]];
          }
          static const int fidx[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
          for (int f = 0; f < 4; ++f) {
            int32_t t[3] = {tv[fidx[f][0]], tv[fidx[f][1]], tv[fidx[f][2]]};
            tri_out(*m, t, q);
            as.cell_face(cell, {t[0], t[1], t[2]});
          }
          cell++;
        }
  m->n_cells = cell;
  build_cell_faces(*m);
  return m;
}

// Each hex split into two triangular prisms along the diagonal (i,j)-(i+1,j+1); conforming.
Mesh* make_prism(int nx, int ny, int nz, const double* lo, const double* hi) {
  auto* m = new Mesh;
  m->kind = "prism";
  Grid g{nx, ny, nz, {lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}};
  g.fill_vertices(*m);
  Assembler as(*m);
  int32_t cell = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        for (int h = 0; h < 2; ++h) {
          // triangle in xy: (i,j),(i+1,j),(i+1,j+1) or (i,j),(i+1,j+1),(i,j+1)
          int tri[3][2] = {{i, j}, {i + 1, j}, {i + 1, j + 1}};
          if (h == 1) {
            tri[1][0] = i + 1; tri[1][1] = j + 1;
            tri[2][0] = i;     tri[2][1] = j + 1;
          }
          int32_t b[3], t[3];
          double q[3] = {0, 0, 0};
          for (int a = 0; a < 3; ++a) {
            b[a] = g.vid(tri[a][0], tri[a][1], k);
            t[a] = g.vid(tri[a][0], tri[a][1], k + 1);
            q[0] += (m->vx[b[a]] + m->vx[t[a]]) / 6.0;
            q[1] += (m->vy[b[a]] + m->vy[t[a]]) / 6.0;
            q[2] += (m->vz[b[a]] + m->vz[t[a]]) / 6.0;
          }
          int32_t f0[3] = {b[0], b[1], b[2]};
          tri_out(*m, f0, q);
          as.cell_face(cell, {f0[0], f0[1], f0[2]});
          int32_t f1[3] = {t[0], t[1], t[2]};
          tri_out(*m, f1, q);
          as.cell_face(cell, {f1[0], f1[1], f1[2]});
          for (int a = 0; a < 3; ++a) {
            int32_t qd[4] = {b[a], b[(a + 1) % 3], t[(a + 1) % 3], t[a]};
            quad_out(*m, qd, q);
            as.cell_face(cell, {qd[0], qd[1], qd[2], qd[3]});
          }
          cell++;
        }
  m->n_cells = cell;
  build_cell_faces(*m);
  return m;
}

// ---------------------------------------------------------------- Voronoi (3D, clipped to a box)
// Generators: sites have ids >= 0; the six box planes have ids -1..-6 (x-lo, x-hi, y-lo, ...).
struct CVert {
  double x[3];
  std::array<int32_t, 3> planes;  // sorted ids of the three generators (besides the site)
};
struct CFace {
  int32_t plane;
  std::vector<int> v;  // local vertex loop, CCW from outside
};
struct CPoly {
  std::vector<CVert> verts;
  std::vector<CFace> faces;
};

CPoly box_poly(const double* lo, const double* hi) {
  CPoly p;
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 2; ++i) {
        CVert v;
        v.x[0] = i ? hi[0] : lo[0];
        v.x[1] = j ? hi[1] : lo[1];
        v.x[2] = k ? hi[2] : lo[2];
        std::array<int32_t, 3> pl = {-(1 + i), -(3 + j), -(5 + k)};
        std::sort(pl.begin(), pl.end());
        v.planes = pl;
        p.verts.push_back(v);
      }
  auto id = [](int i, int j, int k) { return i + 2 * j + 4 * k; };
  p.faces.push_back({-1, {id(0, 0, 0), id(0, 0, 1), id(0, 1, 1), id(0, 1, 0)}});
  p.faces.push_back({-2, {id(1, 0, 0), id(1, 1, 0), id(1, 1, 1), id(1, 0, 1)}});
  p.faces.push_back({-3, {id(0, 0, 0), id(1, 0, 0), id(1, 0, 1), id(0, 0, 1)}});
  p.faces.push_back({-4, {id(0, 1, 0), id(0, 1, 1), id(1, 1, 1), id(1, 1, 0)}});
  p.faces.push_back({-5, {id(0, 0, 0), id(0, 1, 0), id(1, 1, 0), id(1, 0, 0)}});
  p.faces.push_back({-6, {id(0, 0, 1), id(1, 0, 1), id(1, 1, 1), id(0, 1, 1)}});
  return p;
}

// Keeps the part of the polyhedron with n.x <= d. Returns false if nothing was cut.
bool clip(CPoly& p, const double* n, double d, int32_t plane_id) {
  const int nv = (int)p.verts.size();
  std::vector<double> s(nv);
  bool any_out = false, any_in = false;
  for (int i = 0; i < nv; ++i) {
    s[i] = n[0] * p.verts[i].x[0] + n[1] * p.verts[i].x[1] + n[2] * p.verts[i].x[2] - d;
    if (s[i] > 0) any_out = true; else any_in = true;
  }
  if (!any_out) return false;
  if (!any_in) { p.verts.clear(); p.faces.clear(); return true; }
  std::map<std::pair<int, int>, int> cut;  // edge -> new vertex
  std::vector<int> remap(nv, -1);
  CPoly q;
  for (int i = 0; i < nv; ++i)
    if (s[i] <= 0) { remap[i] = (int)q.verts.size(); q.verts.push_back(p.verts[i]); }
  auto cut_vertex = [&](int a, int b) {
    auto key = std::make_pair(std::min(a, b), std::max(a, b));
    auto it = cut.find(key);
    if (it != cut.end()) return it->second;
    const double t = s[a] / (s[a] - s[b]);
    CVert v;
    for (int k = 0; k < 3; ++k) v.x[k] = p.verts[a].x[k] + t * (p.verts[b].x[k] - p.verts[a].x[k]);
    // the edge lies on the two generators shared by its endpoints
    int32_t common[3] = {0, 0, 0}, nc = 0;
    for (int32_t x : p.verts[a].planes)
      for (int32_t y : p.verts[b].planes)
        if (x == y && nc < 2) common[nc++] = x;
    std::array<int32_t, 3> pl = {common[0], nc > 1 ? common[1] : common[0], plane_id};
    std::sort(pl.begin(), pl.end());
    v.planes = pl;
    const int id = (int)q.verts.size();
    q.verts.push_back(v);
    cut.emplace(key, id);
    return id;
  };
  std::map<int, int> cap_next;  // cap loop: entry vertex -> exit vertex
  for (const CFace& f : p.faces) {
    CFace g;
    g.plane = f.plane;
    const int m = (int)f.v.size();
    int exit_v = -1;
    for (int k = 0; k < m; ++k) {
      const int a = f.v[k], b = f.v[(k + 1) % m];
      if (s[a] <= 0) g.v.push_back(remap[a]);
      if ((s[a] <= 0) != (s[b] <= 0)) {
        const int c = cut_vertex(a, b);
        g.v.push_back(c);
        if (s[a] <= 0) exit_v = c;                 // leaving the kept side
        else if (exit_v >= 0) { cap_next[c] = exit_v; exit_v = -1; }
        else cap_next[c] = -2 - k;                  // resolved after the loop
      }
    }
    // wrap-around: an entry seen before its exit in this loop
    for (auto& kv : cap_next)
      if (kv.second <= -2 && exit_v >= 0) { kv.second = exit_v; exit_v = -1; }
    if (g.v.size() >= 3) q.faces.push_back(std::move(g));
  }
  // cap face: traverse the clipped faces' new edges backwards
  if (!cap_next.empty()) {
    CFace cap;
    cap.plane = plane_id;
    const int start = cap_next.begin()->first;
    int v = start;
    for (size_t guard = 0; guard <= cap_next.size(); ++guard) {
      cap.v.push_back(v);
      auto it = cap_next.find(v);
      if (it == cap_next.end() || it->second < 0) break;
      v = it->second;
      if (v == start) break;
    }
    if (cap.v.size() >= 3) q.faces.push_back(std::move(cap));
  }
  p = std::move(q);
  return true;
}

// Canonical vertex position from its four generators (sorted ids). Sites give bisector planes
// relative to the lowest site id; box planes fix one coordinate.
void key_point(const std::array<int32_t, 4>& key, const std::vector<double>& S, const double* lo,
               const double* hi, double* out) {
  double A[3][3], b[3];
  int row = 0;
  int first = -1;
  for (int32_t g : key)
    if (g >= 0) { first = g; break; }
  const double* s0 = &S[3 * (size_t)first];
  for (int32_t g : key) {
    if (row == 3) break;
    if (g < 0) {
      const int ax = (-g - 1) / 2;
      const double val = ((-g - 1) % 2) ? hi[ax] : lo[ax];
      A[row][0] = A[row][1] = A[row][2] = 0;
      A[row][ax] = 1;
      b[row] = val - s0[ax];
      row++;
    } else if (g != first) {
      const double* s = &S[3 * (size_t)g];
      double r[3] = {s[0] - s0[0], s[1] - s0[1], s[2] - s0[2]};
      A[row][0] = 2 * r[0]; A[row][1] = 2 * r[1]; A[row][2] = 2 * r[2];
      b[row] = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      row++;
    }
  }
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  double y[3];
  for (int c = 0; c < 3; ++c) {
    double M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] = (j == c) ? b[i] : A[i][j];
    y[c] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
            M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
            M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
  }
  for (int k = 0; k < 3; ++k) out[k] = s0[k] + y[k];
}

struct KeyHash {
  size_t operator()(const std::array<int32_t, 4>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int32_t x : k) { h ^= (uint32_t)x; h *= 1099511628211ull; }
    return (size_t)h;
  }
};

// Uniform double in [0,1) from a 64-bit draw (same on every platform).
inline double u01(std::mt19937_64& g) { return (double)(g() >> 11) * (1.0 / 9007199254740992.0); }

Mesh* voronoi_from_sites(const std::vector<double>& S, const double* lo, const double* hi, double h) {
  const int64_t ns = (int64_t)S.size() / 3;
  auto* m = new Mesh;
  m->kind = "voronoi";
  // bucket grid of cell size h
  int gn[3];
  for (int k = 0; k < 3; ++k) gn[k] = std::max(1, (int)std::floor((hi[k] - lo[k]) / h));
  auto bucket = [&](const double* x, int* b) {
    for (int k = 0; k < 3; ++k) {
      int v = (int)std::floor((x[k] - lo[k]) / (hi[k] - lo[k]) * gn[k]);
      b[k] = std::min(std::max(v, 0), gn[k] - 1);
    }
  };
  std::vector<int64_t> boff((size_t)gn[0] * gn[1] * gn[2] + 1, 0);
  std::vector<int32_t> bsite(ns);
  for (int64_t s = 0; s < ns; ++s) {
    int b[3];
    bucket(&S[3 * s], b);
    boff[((size_t)b[2] * gn[1] + b[1]) * gn[0] + b[0] + 1]++;
  }
  for (size_t i = 1; i < boff.size(); ++i) boff[i] += boff[i - 1];
  {
    std::vector<int64_t> pos(boff.begin(), boff.end() - 1);
    for (int64_t s = 0; s < ns; ++s) {
      int b[3];
      bucket(&S[3 * s], b);
      bsite[pos[((size_t)b[2] * gn[1] + b[1]) * gn[0] + b[0]]++] = (int32_t)s;
    }
  }
  const double bw = std::min({(hi[0] - lo[0]) / gn[0], (hi[1] - lo[1]) / gn[1], (hi[2] - lo[2]) / gn[2]});
  std::vector<CPoly> cells(ns);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t s = 0; s < ns; ++s) {
    const double* x = &S[3 * s];
    int b[3];
    bucket(x, b);
    CPoly p = box_poly(lo, hi);
    for (int rad = 2;; ++rad) {
      std::vector<std::pair<double, int32_t>> cand;
      for (int k = b[2] - rad; k <= b[2] + rad; ++k)
        for (int j = b[1] - rad; j <= b[1] + rad; ++j)
          for (int i = b[0] - rad; i <= b[0] + rad; ++i) {
            if (i < 0 || j < 0 || k < 0 || i >= gn[0] || j >= gn[1] || k >= gn[2]) continue;
            const size_t bi = ((size_t)k * gn[1] + j) * gn[0] + i;
            for (int64_t t = boff[bi]; t < boff[bi + 1]; ++t) {
              const int32_t o = bsite[t];
              if (o == s) continue;
              const double* y = &S[3 * (size_t)o];
              const double d2 = (y[0] - x[0]) * (y[0] - x[0]) + (y[1] - x[1]) * (y[1] - x[1]) + (y[2] - x[2]) * (y[2] - x[2]);
              cand.emplace_back(d2, o);
            }
          }
      std::sort(cand.begin(), cand.end());
      p = box_poly(lo, hi);
      double rmax2 = 0;
      bool done = false;
      for (auto& c : cand) {
        rmax2 = 0;
        for (auto& v : p.verts) {
          const double d2 = (v.x[0] - x[0]) * (v.x[0] - x[0]) + (v.x[1] - x[1]) * (v.x[1] - x[1]) + (v.x[2] - x[2]) * (v.x[2] - x[2]);
          rmax2 = std::max(rmax2, d2);
        }
        if (c.first > 4 * rmax2) { done = true; break; }
        const double* y = &S[3 * (size_t)c.second];
        double n[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
        const double d = 0.5 * (n[0] * (x[0] + y[0]) + n[1] * (x[1] + y[1]) + n[2] * (x[2] + y[2]));
        clip(p, n, d, c.second);
      }
      if (!done) {
        rmax2 = 0;
        for (auto& v : p.verts) {
          const double d2 = (v.x[0] - x[0]) * (v.x[0] - x[0]) + (v.x[1] - x[1]) * (v.x[1] - x[1]) + (v.x[2] - x[2]) * (v.x[2] - x[2]);
          rmax2 = std::max(rmax2, d2);
        }
        // everything within the searched radius has been used: the cell is final if its
        // security sphere lies inside the searched block
        if (2 * std::sqrt(rmax2) <= rad * bw) done = true;
      }
      if (done) break;
    }
    cells[s] = std::move(p);
  }
  // Global vertices from canonical keys. Entry q = (cell s, local vertex i), numbered in cell
  // order; a vertex takes its id in the order of its first entry. The entries are hashed into
  // buckets (a stable counting sort), each bucket finds the first entry of every key on its own,
  // and one pass in entry order hands out the ids.
  std::vector<int64_t> voff(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) voff[s + 1] = voff[s] + (int64_t)cells[s].verts.size();
  const int64_t nq = voff[ns];
  constexpr int kBuckets = 4096;
  std::vector<std::array<int32_t, 4>> key(nq);
  std::vector<uint32_t> kb(nq);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < ns; ++s)
    for (size_t i = 0; i < cells[s].verts.size(); ++i) {
      const auto& pl = cells[s].verts[i].planes;
      std::array<int32_t, 4> k = {pl[0], pl[1], pl[2], (int32_t)s};
      std::sort(k.begin(), k.end());
      key[voff[s] + i] = k;
      kb[voff[s] + i] = (uint32_t)(KeyHash()(k) % kBuckets);
    }
  std::vector<int64_t> bstart(kBuckets + 1, 0), order(nq);
  for (int64_t q = 0; q < nq; ++q) bstart[kb[q] + 1]++;
  for (int b = 0; b < kBuckets; ++b) bstart[b + 1] += bstart[b];
  {
    std::vector<int64_t> pos(bstart.begin(), bstart.end() - 1);
    for (int64_t q = 0; q < nq; ++q) order[pos[kb[q]]++] = q;
  }
  std::vector<int64_t> rep(nq);
#pragma omp parallel for schedule(dynamic, 16)
  for (int b = 0; b < kBuckets; ++b) {
    std::unordered_map<std::array<int32_t, 4>, int64_t, KeyHash> first;
    first.reserve((size_t)(bstart[b + 1] - bstart[b]));
    for (int64_t t = bstart[b]; t < bstart[b + 1]; ++t) {
      const int64_t q = order[t];  // increasing within the bucket
      rep[q] = first.emplace(key[q], q).first->second;
    }
  }
  std::vector<int32_t> vid(nq);
  int32_t nv = 0;
  for (int64_t q = 0; q < nq; ++q) vid[q] = rep[q] == q ? nv++ : vid[rep[q]];
  m->vx.resize(nv);
  m->vy.resize(nv);
  m->vz.resize(nv);
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < nq; ++q)
    if (rep[q] == q) {
      double y[3];
      key_point(key[q], S, lo, hi, y);
      m->vx[vid[q]] = y[0];
      m->vy[vid[q]] = y[1];
      m->vz[vid[q]] = y[2];
    }
  // Faces, in cell order: cell s emits its box faces and its faces toward higher sites (owner =
  // lower site id); a face toward a lower site p must match the loop p emitted, reversed.
  std::vector<int64_t> fcount(ns + 1, 0), fvcount(ns + 1, 0);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < ns; ++s)
    for (const CFace& f : cells[s].faces)
      if (f.plane < 0 || f.plane > s) { fcount[s + 1]++; fvcount[s + 1] += (int64_t)f.v.size(); }
  for (int64_t s = 0; s < ns; ++s) { fcount[s + 1] += fcount[s]; fvcount[s + 1] += fvcount[s]; }
  const int64_t nf = fcount[ns];
  m->face_vert_off.assign(nf + 1, 0);
  m->face_vert.resize(fvcount[ns]);
  m->face_owner.resize(nf);
  m->face_neigh.resize(nf);
  std::vector<uint8_t> matched(nf, 0);
  int64_t errors = 0;
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < ns; ++s) {
    int64_t fi = fcount[s], vo = fvcount[s];
    for (const CFace& f : cells[s].faces) {
      if (!(f.plane < 0 || f.plane > s)) continue;
      for (int v : f.v) m->face_vert[vo++] = vid[voff[s] + v];
      m->face_vert_off[fi + 1] = vo;
      m->face_owner[fi] = (int32_t)s;
      m->face_neigh[fi] = f.plane < 0 ? -1 : f.plane;
      fi++;
    }
  }
#pragma omp parallel for schedule(static) reduction(+ : errors)
  for (int64_t s = 0; s < ns; ++s) {
    for (const CFace& f : cells[s].faces) {
      if (f.plane < 0 || f.plane > s) continue;
      // the face that the lower site p = f.plane emitted toward s
      const int64_t p = f.plane;
      int64_t fi = fcount[p];
      bool found = false;
      for (const CFace& g : cells[p].faces) {
        if (!(g.plane < 0 || g.plane > p)) continue;
        if (g.plane == s) { found = true; break; }
        fi++;
      }
      if (!found) { errors++; continue; }
      matched[fi] = 1;
      const int64_t o = m->face_vert_off[fi];
      const int n = (int)(m->face_vert_off[fi + 1] - o);
      bool ok = n == (int)f.v.size();
      int st = -1;
      for (int i = 0; ok && i < n; ++i)
        if (m->face_vert[o + i] == vid[voff[s] + f.v[0]]) st = i;
      ok = ok && st >= 0;
      for (int i = 0; ok && i < n; ++i) ok = m->face_vert[o + ((st - i) % n + n) % n] == vid[voff[s] + f.v[i]];
      if (!ok) errors++;
    }
  }
  // faces never matched by the other cell
  for (int64_t fi = 0; fi < nf; ++fi)
    if (m->face_neigh[fi] >= 0 && !matched[fi]) { errors++; m->face_neigh[fi] = -1; }
  m->conform_errors += errors;
  m->n_cells = ns;
  build_cell_faces(*m);
  return m;
}

Mesh* make_voronoi_bcc(int n, double jitter, uint64_t seed, const double* lo, const double* hi) {
  // BCC lattice of cubic spacing h = L/n: sites at ((i+1/4)h, ...) and ((i+3/4)h, ...),
  // i = 0..n-1, so that a jitter of up to h/4 per axis keeps every site inside the box.
  const double h = (hi[0] - lo[0]) / n;
  std::mt19937_64 rng(seed);
  std::vector<double> S;
  S.reserve((size_t)6 * n * n * n);
  for (int sub = 0; sub < 2; ++sub) {
    const double off = sub ? 0.75 : 0.25;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const double base[3] = {lo[0] + (i + off) * (hi[0] - lo[0]) / n, lo[1] + (j + off) * (hi[1] - lo[1]) / n,
                                  lo[2] + (k + off) * (hi[2] - lo[2]) / n};
          for (int a = 0; a < 3; ++a) S.push_back(base[a] + jitter * h * (2 * u01(rng) - 1));
        }
  }
  return voronoi_from_sites(S, lo, hi, h);
}

// ---------------------------------------------------------------- extruded 2D Voronoi disk (pipe)
struct C2Vert { double x[2]; std::array<int32_t, 2> gens; };
struct C2Poly { std::vector<C2Vert> v; std::vector<int32_t> edge_gen; };  // edge k: v[k] -> v[k+1]

void clip2(C2Poly& p, const double* n, double d, int32_t gen) {
  const int m = (int)p.v.size();
  std::vector<double> s(m);
  bool out = false;
  for (int i = 0; i < m; ++i) { s[i] = n[0] * p.v[i].x[0] + n[1] * p.v[i].x[1] - d; out |= s[i] > 0; }
  if (!out) return;
  C2Poly q;
  for (int k = 0; k < m; ++k) {
    const int a = k, b = (k + 1) % m;
    if (s[a] <= 0) { q.v.push_back(p.v[a]); q.edge_gen.push_back(p.edge_gen[k]); }
    if ((s[a] <= 0) != (s[b] <= 0)) {
      const double t = s[a] / (s[a] - s[b]);
      C2Vert c;
      c.x[0] = p.v[a].x[0] + t * (p.v[b].x[0] - p.v[a].x[0]);
      c.x[1] = p.v[a].x[1] + t * (p.v[b].x[1] - p.v[a].x[1]);
      std::array<int32_t, 2> g = {p.edge_gen[k], gen};
      std::sort(g.begin(), g.end());
      c.gens = g;
      q.v.push_back(c);
      q.edge_gen.push_back(s[a] <= 0 ? gen : p.edge_gen[k]);
    }
  }
  p = std::move(q);
}

Mesh* make_pipe(double spacing, int layers, double radius, double length, double jitter, uint64_t seed) {
  auto* m = new Mesh;
  m->kind = "pipe";
  std::mt19937_64 rng(seed);
  // jittered square lattice inside the disk, mirrored across the circle near the wall
  std::vector<double> S;
  const int nl = (int)std::ceil(radius / spacing) + 1;
  for (int j = -nl; j <= nl; ++j)
    for (int i = -nl; i <= nl; ++i) {
      const double x = (i + 0.5) * spacing + jitter * spacing * (2 * u01(rng) - 1);
      const double y = (j + 0.5) * spacing + jitter * spacing * (2 * u01(rng) - 1);
      const double r = std::sqrt(x * x + y * y);
      if (r < radius - 0.3 * spacing) { S.push_back(x); S.push_back(y); }
    }
  const int64_t nreal = (int64_t)S.size() / 2;
  for (int64_t s = 0; s < nreal; ++s) {
    const double x = S[2 * s], y = S[2 * s + 1], r = std::sqrt(x * x + y * y);
    if (r > radius - 3 * spacing) {
      const double f = (2 * radius - r) / r;
      S.push_back(x * f); S.push_back(y * f);
    }
  }
  const int64_t nall = (int64_t)S.size() / 2;
  // bucket grid
  const int gn = (int)std::ceil(2 * (radius + 3 * spacing) / spacing);
  const double g0 = -(radius + 3 * spacing), gw = 2 * (radius + 3 * spacing) / gn;
  std::vector<std::vector<int32_t>> bk((size_t)gn * gn);
  auto bix = [&](double v) { return std::min(std::max((int)std::floor((v - g0) / gw), 0), gn - 1); };
  for (int64_t s = 0; s < nall; ++s) bk[(size_t)bix(S[2 * s + 1]) * gn + bix(S[2 * s])].push_back((int32_t)s);
  std::vector<C2Poly> cells(nreal);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t s = 0; s < nreal; ++s) {
    const double x = S[2 * s], y = S[2 * s + 1];
    C2Poly p;
    const double B = 4 * spacing;
    const double box[4][2] = {{x - B, y - B}, {x + B, y - B}, {x + B, y + B}, {x - B, y + B}};
    for (int k = 0; k < 4; ++k) {
      C2Vert v;
      v.x[0] = box[k][0]; v.x[1] = box[k][1];
      v.gens = {-1 - ((k + 3) % 4), -1 - k};
      p.v.push_back(v);
      p.edge_gen.push_back(-1 - k);
    }
    std::vector<std::pair<double, int32_t>> cand;
    const int bx = bix(x), by = bix(y);
    for (int j = by - 3; j <= by + 3; ++j)
      for (int i = bx - 3; i <= bx + 3; ++i) {
        if (i < 0 || j < 0 || i >= gn || j >= gn) continue;
        for (int32_t o : bk[(size_t)j * gn + i]) {
          if (o == s) continue;
          const double dx = S[2 * o] - x, dy = S[2 * o + 1] - y;
          cand.emplace_back(dx * dx + dy * dy, o);
        }
      }
    std::sort(cand.begin(), cand.end());
    for (auto& c : cand) {
      double rmax2 = 0;
      for (auto& v : p.v) rmax2 = std::max(rmax2, (v.x[0] - x) * (v.x[0] - x) + (v.x[1] - y) * (v.x[1] - y));
      if (c.first > 4 * rmax2) break;
      const double ox = S[2 * c.second], oy = S[2 * c.second + 1];
      double n[2] = {ox - x, oy - y};
      clip2(p, n, 0.5 * (n[0] * (x + ox) + n[1] * (y + oy)), c.second);
    }
    cells[s] = std::move(p);
  }
  // 2D vertices by key (three generators), canonical circumcentres
  struct K3H { size_t operator()(const std::array<int32_t, 3>& k) const { return (size_t)(((uint64_t)k[0] * 73856093u) ^ ((uint64_t)k[1] * 19349663u) ^ ((uint64_t)k[2] * 83492791u)); } };
  std::unordered_map<std::array<int32_t, 3>, int32_t, K3H> vmap;
  std::vector<double> V2;
  std::vector<std::vector<int32_t>> gid(nreal);
  for (int64_t s = 0; s < nreal; ++s) {
    for (auto& v : cells[s].v) {
      std::array<int32_t, 3> key = {v.gens[0], v.gens[1], (int32_t)s};
      std::sort(key.begin(), key.end());
      auto it = vmap.find(key);
      int32_t id;
      if (it == vmap.end() && key[0] < 0) {
        // a helper-box edge survived: the cell was not closed by real or mirror sites
        m->conform_errors++;
        id = (int32_t)(V2.size() / 2);
        V2.push_back(v.x[0]);
        V2.push_back(v.x[1]);
        vmap.emplace(key, id);
      } else if (it == vmap.end()) {
        const double* a = &S[2 * (size_t)key[0]];
        const double* b = &S[2 * (size_t)key[1]];
        const double* c = &S[2 * (size_t)key[2]];
        const double bx2 = b[0] - a[0], by2 = b[1] - a[1], cx2 = c[0] - a[0], cy2 = c[1] - a[1];
        const double D = 2 * (bx2 * cy2 - by2 * cx2);
        const double b2 = bx2 * bx2 + by2 * by2, c2 = cx2 * cx2 + cy2 * cy2;
        id = (int32_t)(V2.size() / 2);
        V2.push_back(a[0] + (cy2 * b2 - by2 * c2) / D);
        V2.push_back(a[1] + (bx2 * c2 - cx2 * b2) / D);
        vmap.emplace(key, id);
      } else {
        id = it->second;
      }
      gid[s].push_back(id);
    }
  }
  const int64_t nv2 = (int64_t)V2.size() / 2;
  for (int l = 0; l <= layers; ++l)
    for (int64_t v = 0; v < nv2; ++v) {
      m->vx.push_back(V2[2 * v]);
      m->vy.push_back(V2[2 * v + 1]);
      m->vz.push_back(length * l / layers);
    }
  auto v3 = [&](int32_t v, int l) { return (int32_t)((int64_t)l * nv2 + v); };
  // 2D edges: owner = lower site; edges toward a mirror site or the helper box are the wall
  std::unordered_map<uint64_t, int> seen;
  for (int64_t s = 0; s < nreal; ++s) {
    const auto& p = cells[s];
    const int n = (int)p.v.size();
    for (int k = 0; k < n; ++k) {
      const int32_t g = p.edge_gen[k];
      const bool wall = g < 0 || g >= nreal;
      if (!wall && g < s) continue;  // emitted by the lower site
      const int32_t a = gid[s][k], b = gid[s][(k + 1) % n];
      for (int l = 0; l < layers; ++l) {
        const int32_t own = (int32_t)(l * nreal + s);
        const int32_t nb = wall ? -1 : (int32_t)(l * nreal + g);
        // 2D polygon is CCW, so edge a->b has the cell on its left; outward quad loop:
        int32_t q[4] = {v3(a, l), v3(b, l), v3(b, l + 1), v3(a, l + 1)};
        add_face(*m, q, 4, own, nb);
      }
    }
  }
  // caps
  for (int l = 0; l <= layers; ++l)
    for (int64_t s = 0; s < nreal; ++s) {
      std::vector<int32_t> loop;
      const int n = (int)gid[s].size();
      if (l == layers || l == 0) {
        // bottom cap faces -z: reverse of CCW; top cap +z: CCW
        for (int k = 0; k < n; ++k) loop.push_back(v3(gid[s][l == 0 ? (n - k) % n : k], l));
        add_face(*m, loop.data(), n, (int32_t)((l == 0 ? 0 : layers - 1) * nreal + s), -1);
      } else {
        for (int k = 0; k < n; ++k) loop.push_back(v3(gid[s][k], l));
        add_face(*m, loop.data(), n, (int32_t)((l - 1) * nreal + s), (int32_t)(l * nreal + s));
      }
    }
  m->n_cells = (int64_t)layers * nreal;
  build_cell_faces(*m);
  return m;
}

// ---------------------------------------------------------------- fields
// Liquid indicator: g(x) > 0 is liquid. Types: 0 plane n.x < d; 1 spheres (vapour inside);
// 2 wavy film z < z0 + a sin(2 pi x / lx) sin(2 pi y / ly); 3 pipe film r > r0 - a sin(2 pi (z - t)/lam).
struct Region {
  int type;
  const double* p;
  int np;
  double g(const double* x) const {
    switch (type) {
      case 0: return p[3] - (p[0] * x[0] + p[1] * x[1] + p[2] * x[2]);
      case 1: {
        double best = 1e300;
        for (int s = 0; s < np / 4; ++s) {
          const double* q = p + 4 * s;
          const double r = std::sqrt((x[0] - q[0]) * (x[0] - q[0]) + (x[1] - q[1]) * (x[1] - q[1]) + (x[2] - q[2]) * (x[2] - q[2]));
          best = std::min(best, r - q[3]);
        }
        return best;
      }
      case 2: return p[0] + p[1] * std::sin(2 * kPi * x[0] / p[2]) * std::sin(2 * kPi * x[1] / p[3]) - x[2];
      case 3: {
        const double r = std::sqrt(x[0] * x[0] + x[1] * x[1]);
        return r - (p[0] - p[1] * std::sin(2 * kPi * (x[2] - p[3]) / p[2]));
      }
    }
    return 0;
  }
  // Lipschitz bound of g, used to skip cells that the interface cannot reach
  double lip() const {
    switch (type) {
      case 0: return std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
      case 1: return 1.0;
      case 2: return std::sqrt(1 + 2 * std::pow(2 * kPi * p[1] / std::min(p[2], p[3]), 2));
      case 3: return std::sqrt(1 + std::pow(2 * kPi * p[1] / p[2], 2));
    }
    return 1;
  }
};

struct CellTets {
  // fan tetrahedra (apex = vertex mean of the cell, face fans about the face vertex mean)
  std::vector<std::array<double, 12>> tets;
  double vol = 0, cen[3] = {0, 0, 0}, apex[3] = {0, 0, 0}, rad = 0;
};

void cell_tets(const Mesh& m, int64_t c, CellTets& ct) {
  ct.tets.clear();
  std::vector<int32_t> vs;
  for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
    const int32_t f = m.cell_face[k] & 0x7fffffff;
    for (int64_t j = m.face_vert_off[f]; j < m.face_vert_off[f + 1]; ++j) vs.push_back(m.face_vert[j]);
  }
  std::sort(vs.begin(), vs.end());
  vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
  double a[3] = {0, 0, 0};
  for (int32_t v : vs) { a[0] += m.vx[v]; a[1] += m.vy[v]; a[2] += m.vz[v]; }
  for (int k = 0; k < 3; ++k) a[k] /= (double)vs.size();
  ct.rad = 0;
  for (int32_t v : vs) {
    const double d2 = (m.vx[v] - a[0]) * (m.vx[v] - a[0]) + (m.vy[v] - a[1]) * (m.vy[v] - a[1]) + (m.vz[v] - a[2]) * (m.vz[v] - a[2]);
    ct.rad = std::max(ct.rad, std::sqrt(d2));
  }
  for (int k = 0; k < 3; ++k) ct.apex[k] = a[k];
  ct.vol = 0;
  double cs[3] = {0, 0, 0};
  for (int64_t k = m.cell_face_off[c]; k < m.cell_face_off[c + 1]; ++k) {
    const int32_t fe = m.cell_face[k];
    const int32_t f = fe & 0x7fffffff;
    const bool rev = fe < 0;
    const int64_t o = m.face_vert_off[f];
    const int n = (int)(m.face_vert_off[f + 1] - o);
    double fm[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) { const int32_t v = m.face_vert[o + i]; fm[0] += m.vx[v]; fm[1] += m.vy[v]; fm[2] += m.vz[v]; }
    for (int q = 0; q < 3; ++q) fm[q] /= n;
    for (int i = 0; i < n; ++i) {
      int32_t v0 = m.face_vert[o + i], v1 = m.face_vert[o + (i + 1) % n];
      if (rev) std::swap(v0, v1);
      std::array<double, 12> t = {a[0], a[1], a[2], fm[0], fm[1], fm[2], m.vx[v0], m.vy[v0], m.vz[v0], m.vx[v1], m.vy[v1], m.vz[v1]};
      const double ux = t[3] - a[0], uy = t[4] - a[1], uz = t[5] - a[2];
      const double vx = t[6] - a[0], vy = t[7] - a[1], vz = t[8] - a[2];
      const double wx = t[9] - a[0], wy = t[10] - a[1], wz = t[11] - a[2];
      const double vol = (ux * (vy * wz - vz * wy) - uy * (vx * wz - vz * wx) + uz * (vx * wy - vy * wx)) / 6.0;
      ct.vol += vol;
      for (int q = 0; q < 3; ++q) cs[q] += vol * (t[q] + t[3 + q] + t[6 + q] + t[9 + q]) / 4.0;
      ct.tets.push_back(t);
    }
  }
  for (int q = 0; q < 3; ++q) ct.cen[q] = cs[q] / ct.vol;
}

// Recursive red refinement of a tet (8 children of equal volume); at depth 0 the indicator is
// sampled at the child's centroid.
double tet_fraction(const double* P, int depth, const Region& R) {
  if (depth == 0) {
    double c[3];
    for (int k = 0; k < 3; ++k) c[k] = 0.25 * (P[k] + P[3 + k] + P[6 + k] + P[9 + k]);
    return R.g(c) > 0 ? 1.0 : 0.0;
  }
  double M[6][3];
  static const int e[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  for (int i = 0; i < 6; ++i)
    for (int k = 0; k < 3; ++k) M[i][k] = 0.5 * (P[3 * e[i][0] + k] + P[3 * e[i][1] + k]);
  const double* v0 = P; const double* v1 = P + 3; const double* v2 = P + 6; const double* v3 = P + 9;
  const double* m01 = M[0]; const double* m02 = M[1]; const double* m03 = M[2];
  const double* m12 = M[3]; const double* m13 = M[4]; const double* m23 = M[5];
  const double* ch[8][4] = {{v0, m01, m02, m03}, {m01, v1, m12, m13}, {m02, m12, v2, m23}, {m03, m13, m23, v3},
                            {m01, m02, m03, m13}, {m01, m02, m12, m13}, {m02, m03, m13, m23}, {m02, m12, m13, m23}};
  double s = 0;
  for (int c = 0; c < 8; ++c) {
    double Q[12];
    for (int i = 0; i < 4; ++i)
      for (int k = 0; k < 3; ++k) Q[3 * i + k] = ch[c][i][k];
    s += tet_fraction(Q, depth - 1, R);
  }
  return s / 8.0;
}

}  // namespace

extern "C" {

void* synth_hex(int nx, int ny, int nz, const double* lo, const double* hi) { return make_hex(nx, ny, nz, lo, hi); }
void* synth_tet(int nx, int ny, int nz, const double* lo, const double* hi) { return make_tet(nx, ny, nz, lo, hi); }
void* synth_prism(int nx, int ny, int nz, const double* lo, const double* hi) { return make_prism(nx, ny, nz, lo, hi); }
void* synth_voronoi_bcc(int n, double jitter, uint64_t seed, const double* lo, const double* hi) {
  return make_voronoi_bcc(n, jitter, seed, lo, hi);
}
void* synth_voronoi_sites(const double* sites, int64_t ns, double h, const double* lo, const double* hi) {
  std::vector<double> S(sites, sites + 3 * ns);
  return voronoi_from_sites(S, lo, hi, h);
}
void* synth_pipe(double spacing, int layers, double radius, double length, double jitter, uint64_t seed) {
  return make_pipe(spacing, layers, radius, length, jitter, seed);
}

// sizes: n_cells, n_faces, n_verts, n_face_vert, n_cell_face, conform_errors
void synth_sizes(void* h, int64_t* out) {
  auto* m = (Mesh*)h;
  out[0] = m->n_cells;
  out[1] = (int64_t)m->face_owner.size();
  out[2] = (int64_t)m->vx.size();
  out[3] = (int64_t)m->face_vert.size();
  out[4] = (int64_t)m->cell_face.size();
  out[5] = m->conform_errors;
}

void synth_copy(void* h, double* vx, double* vy, double* vz, int64_t* fvo, int32_t* fv, int32_t* own, int32_t* nei,
                int64_t* cfo, int32_t* cf) {
  auto* m = (Mesh*)h;
  std::memcpy(vx, m->vx.data(), 8 * m->vx.size());
  std::memcpy(vy, m->vy.data(), 8 * m->vy.size());
  std::memcpy(vz, m->vz.data(), 8 * m->vz.size());
  std::memcpy(fvo, m->face_vert_off.data(), 8 * m->face_vert_off.size());
  std::memcpy(fv, m->face_vert.data(), 4 * m->face_vert.size());
  std::memcpy(own, m->face_owner.data(), 4 * m->face_owner.size());
  std::memcpy(nei, m->face_neigh.data(), 4 * m->face_neigh.size());
  std::memcpy(cfo, m->cell_face_off.data(), 8 * m->cell_face_off.size());
  std::memcpy(cf, m->cell_face.data(), 4 * m->cell_face.size());
}

void synth_free(void* h) { delete (Mesh*)h; }

// Builds a temporary view on caller-owned arrays (used by the field generators).
static Mesh view(int64_t nc, const double* vx, const double* vy, const double* vz, int64_t nv, const int64_t* fvo,
                 const int32_t* fv, int64_t nf, const int64_t* cfo, const int32_t* cf) {
  Mesh m;
  m.n_cells = nc;
  m.vx.assign(vx, vx + nv); m.vy.assign(vy, vy + nv); m.vz.assign(vz, vz + nv);
  m.face_vert_off.assign(fvo, fvo + nf + 1);
  m.face_vert.assign(fv, fv + fvo[nf]);
  m.cell_face_off.assign(cfo, cfo + nc + 1);
  m.cell_face.assign(cf, cf + cfo[nc]);
  return m;
}

// Liquid volume fraction per cell by sampling the region indicator.
//   mode 0: fan tets of the cell, each refined `level` times (8^level sub-tets, centroid samples)
//   mode 1: axis-aligned box cells, (2^level)^3 midpoint samples of the bounding box
// Cells that the interface cannot reach (|g(apex)| > lip * radius) get exactly 0 or 1.
void synth_alpha(int64_t nc, const double* vx, const double* vy, const double* vz, int64_t nv, const int64_t* fvo,
                 const int32_t* fv, int64_t nf, const int64_t* cfo, const int32_t* cf, int type, const double* p, int np,
                 int mode, int level, double* alpha) {
  Mesh m = view(nc, vx, vy, vz, nv, fvo, fv, nf, cfo, cf);
  Region R{type, p, np};
  const double L = R.lip();
#pragma omp parallel
  {
    CellTets ct;
    std::vector<double> near;
#pragma omp for schedule(dynamic, 512)
    for (int64_t c = 0; c < nc; ++c) {
      cell_tets(m, c, ct);
      const double g0 = R.g(ct.apex);
      if (std::fabs(g0) > L * ct.rad * 1.0001 + 1e-12) { alpha[c] = g0 > 0 ? 1.0 : 0.0; continue; }
      Region Rc = R;
      if (R.type == 1 && R.np > 32) {
        // Every sample lies within Rb of the apex (2 rad covers the bounding box too), where sphere
        // s contributes a term in [d_s - R_s - Rb, d_s - R_s + Rb]. A sphere whose lowest term is
        // above the smallest highest term can never be the minimum, so g is unchanged without it.
        const double Rb = 2 * ct.rad * 1.0001 + 1e-12;
        auto dist = [&](const double* q) {
          return std::sqrt((ct.apex[0] - q[0]) * (ct.apex[0] - q[0]) + (ct.apex[1] - q[1]) * (ct.apex[1] - q[1]) +
                           (ct.apex[2] - q[2]) * (ct.apex[2] - q[2]));
        };
        double mu = 1e300;
        for (int k = 0; k + 4 <= R.np; k += 4) mu = std::min(mu, dist(R.p + k) - R.p[k + 3] + Rb);
        const double tol = 1e-9 * (1 + std::fabs(mu));
        near.clear();
        for (int k = 0; k + 4 <= R.np; k += 4)
          if (dist(R.p + k) - R.p[k + 3] - Rb <= mu + tol) near.insert(near.end(), R.p + k, R.p + k + 4);
        Rc = Region{1, near.data(), (int)near.size()};
      }
      if (mode == 1) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (auto& t : ct.tets)
          for (int i = 1; i < 4; ++i)
            for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], t[3 * i + k]); hi[k] = std::max(hi[k], t[3 * i + k]); }
        const int n = 1 << level;
        int64_t in = 0;
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              const double x[3] = {lo[0] + (hi[0] - lo[0]) * (i + 0.5) / n, lo[1] + (hi[1] - lo[1]) * (j + 0.5) / n,
                                   lo[2] + (hi[2] - lo[2]) * (k + 0.5) / n};
              in += Rc.g(x) > 0;
            }
        alpha[c] = (double)in / ((double)n * n * n);
      } else {
        double s = 0, vt = 0;
        for (auto& t : ct.tets) {
          const double ux = t[3] - t[0], uy = t[4] - t[1], uz = t[5] - t[2];
          const double vx2 = t[6] - t[0], vy2 = t[7] - t[1], vz2 = t[8] - t[2];
          const double wx = t[9] - t[0], wy = t[10] - t[1], wz = t[11] - t[2];
          const double vol = std::fabs(ux * (vy2 * wz - vz2 * wy) - uy * (vx2 * wz - vz2 * wx) + uz * (vx2 * wy - vy2 * wx)) / 6.0;
          s += vol * tet_fraction(t.data(), level, Rc);
          vt += vol;
        }
        alpha[c] = std::min(1.0, std::max(0.0, s / vt));
      }
    }
  }
}

// Cell centroids (fan-tet, volume weighted) and boundary-face centroids (fan about the vertex
// mean, area weighted), for evaluating analytic temperature profiles.
void synth_points(int64_t nc, const double* vx, const double* vy, const double* vz, int64_t nv, const int64_t* fvo,
                  const int32_t* fv, int64_t nf, const int64_t* cfo, const int32_t* cf, double* cell_xyz, double* face_xyz) {
  Mesh m = view(nc, vx, vy, vz, nv, fvo, fv, nf, cfo, cf);
#pragma omp parallel
  {
    CellTets ct;
#pragma omp for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
      cell_tets(m, c, ct);
      for (int k = 0; k < 3; ++k) cell_xyz[3 * c + k] = ct.cen[k];
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < nf; ++f) {
    const int64_t o = fvo[f];
    const int n = (int)(fvo[f + 1] - o);
    double a[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) { a[0] += vx[fv[o + i]]; a[1] += vy[fv[o + i]]; a[2] += vz[fv[o + i]]; }
    for (int k = 0; k < 3; ++k) a[k] /= n;
    double cs[3] = {0, 0, 0}, at = 0;
    for (int i = 0; i < n; ++i) {
      const int32_t v0 = fv[o + i], v1 = fv[o + (i + 1) % n];
      const double ux = vx[v0] - a[0], uy = vy[v0] - a[1], uz = vz[v0] - a[2];
      const double wx = vx[v1] - a[0], wy = vy[v1] - a[1], wz = vz[v1] - a[2];
      const double cx = uy * wz - uz * wy, cy = uz * wx - ux * wz, cz = ux * wy - uy * wx;
      const double ar = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
      cs[0] += ar * (a[0] + vx[v0] + vx[v1]) / 3; cs[1] += ar * (a[1] + vy[v0] + vy[v1]) / 3; cs[2] += ar * (a[2] + vz[v0] + vz[v1]) / 3;
      at += ar;
    }
    for (int k = 0; k < 3; ++k) face_xyz[3 * f + k] = at > 0 ? cs[k] / at : a[k];
  }
}

}  // extern "C"
