// Host-side feeders: voxel mesh + SWG face table, KD cluster tree, quadrature rules.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace vie {

// Kuhn tetrahedra [v0, v0+e_p0, v0+e_p0+e_p1, v0+(1,1,1)] for the 6 axis
// permutations p in lexicographic order (Sec. II mesh; voxel mesh reading).
const int kKuhn[6][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {1, 1, 1}},  // (0,1,2)
    {{0, 0, 0}, {1, 0, 0}, {1, 0, 1}, {1, 1, 1}},  // (0,2,1)
    {{0, 0, 0}, {0, 1, 0}, {1, 1, 0}, {1, 1, 1}},  // (1,0,2)
    {{0, 0, 0}, {0, 1, 0}, {0, 1, 1}, {1, 1, 1}},  // (1,2,0)
    {{0, 0, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}},  // (2,0,1)
    {{0, 0, 0}, {0, 0, 1}, {0, 1, 1}, {1, 1, 1}},  // (2,1,0)
};

static inline uint64_t pack_lattice(int64_t i, int64_t j, int64_t k) {
  const int64_t B = int64_t(1) << 20;
  return (uint64_t(i + B) << 42) | (uint64_t(j + B) << 21) | uint64_t(k + B);
}

static void make_face_table(Mesh& m);

void build_mesh(const vie_voxels& body, Mesh& m) {
  m.h = body.h;
  m.nvox = body.nvox;
  m.vox.assign(body.ijk, body.ijk + 3 * body.nvox);
  m.eps.assign(body.eps, body.eps + 2 * body.nvox);
  for (int64_t i = 0; i < 3 * body.nvox; ++i)
    VIE_REQUIRE(std::abs(body.ijk[i]) < (1 << 19), VIE_EINVAL, "voxel index out of range (|i| < 2^19)");
  for (int64_t v = 0; v < body.nvox; ++v)  // kappa = (eps_r - 1) / eps_r needs a finite, nonzero eps_r
    VIE_REQUIRE(std::isfinite(m.eps[2 * v]) && std::isfinite(m.eps[2 * v + 1]) &&
                    (m.eps[2 * v] != 0.0 || m.eps[2 * v + 1] != 0.0),
                VIE_EINVAL, "eps_r must be finite and nonzero");
  m.nt = 6 * m.nvox;
  // vertices: unique lattice points, lexicographic (i, j, k)
  std::vector<uint64_t> keys(4 * m.nt);
  for (int64_t v = 0; v < m.nvox; ++v)
    for (int p = 0; p < 6; ++p)
      for (int a = 0; a < 4; ++a) {
        const int32_t* c = &m.vox[3 * v];
        keys[(6 * v + p) * 4 + a] =
            pack_lattice(c[0] + kKuhn[p][a][0], c[1] + kKuhn[p][a][1], c[2] + kKuhn[p][a][2]);
      }
  std::vector<uint64_t> uniq(keys);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  m.nv = (int64_t)uniq.size();
  m.vlat.resize(3 * m.nv);
  const int64_t B = int64_t(1) << 20, M21 = (int64_t(1) << 21) - 1;
  for (int64_t i = 0; i < m.nv; ++i) {
    m.vlat[3 * i + 0] = int32_t(int64_t(uniq[i] >> 42) - B);
    m.vlat[3 * i + 1] = int32_t(int64_t((uniq[i] >> 21) & M21) - B);
    m.vlat[3 * i + 2] = int32_t(int64_t(uniq[i] & M21) - B);
  }
  m.tets.resize(4 * m.nt);
  for (int64_t i = 0; i < 4 * m.nt; ++i)
    m.tets[i] = int32_t(std::lower_bound(uniq.begin(), uniq.end(), keys[i]) - uniq.begin());
  make_face_table(m);
}

// faces: local face a is opposite local vertex a; unique sorted triples, lexicographic;
// T+ = the lower tet id holding the face
static void make_face_table(Mesh& m) {
  struct Rec { std::array<int32_t, 3> v; int32_t t; int32_t a; };
  std::vector<Rec> recs(4 * m.nt);
  static const int loc[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  for (int64_t t = 0; t < m.nt; ++t)
    for (int a = 0; a < 4; ++a) {
      std::array<int32_t, 3> v = {m.tets[4 * t + loc[a][0]], m.tets[4 * t + loc[a][1]], m.tets[4 * t + loc[a][2]]};
      std::sort(v.begin(), v.end());
      recs[4 * t + a] = Rec{v, int32_t(t), a};
    }
  std::sort(recs.begin(), recs.end(), [](const Rec& x, const Rec& y) {
    if (x.v != y.v) return x.v < y.v;
    return x.t < y.t;
  });
  m.faces.clear(); m.tp.clear(); m.tm.clear(); m.lp.clear(); m.lm.clear();
  m.tet_faces.assign(4 * m.nt, -1);
  for (size_t i = 0; i < recs.size();) {
    size_t j = i + 1;
    while (j < recs.size() && recs[j].v == recs[i].v) ++j;
    VIE_REQUIRE(j - i <= 2, VIE_EINVAL, "non-manifold face (shared by more than two tets)");
    int32_t f = (int32_t)m.tp.size();
    m.faces.insert(m.faces.end(), recs[i].v.begin(), recs[i].v.end());
    m.tp.push_back(recs[i].t); m.lp.push_back(recs[i].a);
    m.tet_faces[4 * recs[i].t + recs[i].a] = f;
    if (j - i == 2) {
      m.tm.push_back(recs[i + 1].t); m.lm.push_back(recs[i + 1].a);
      m.tet_faces[4 * recs[i + 1].t + recs[i + 1].a] = f;
    } else {
      m.tm.push_back(-1); m.lm.push_back(-1);
    }
    i = j;
  }
  m.nf = (int64_t)m.tp.size();
}

// General tetrahedral mesh (Sec. II): vertices and tets as given, the face table as for
// voxel meshes, and the tier cells of the quadrature rule: the cell pitch is the mean
// (in tet order) of each tet's shortest edge, a tet's cell is floor(centroid / pitch).
// On a voxel/Kuhn mesh the cells are the voxels.  Every step uses +, -, *, / and sqrt
// in a fixed order, so the cells do not depend on the machine.
void build_mesh_general(const vie_mesh& mm, Mesh& m) {
  VIE_REQUIRE(mm.nv >= 4 && mm.nt >= 1 && mm.xyz && mm.tet && mm.eps_r, VIE_EINVAL, "empty or invalid tet mesh");
  VIE_REQUIRE(mm.nv < (int64_t(1) << 31) && mm.nt < (int64_t(1) << 29), VIE_EINVAL, "tet mesh too large");
  m.general = true;
  m.nv = mm.nv;
  m.nt = mm.nt;
  m.nvox = 0;
  m.xyz.assign(mm.xyz, mm.xyz + 3 * mm.nv);
  m.tets.assign(mm.tet, mm.tet + 4 * mm.nt);
  m.eps.assign(mm.eps_r, mm.eps_r + 2 * mm.nt);
  for (double v : m.xyz) VIE_REQUIRE(std::isfinite(v), VIE_EINVAL, "vertex coordinate not finite");
  for (int64_t t = 0; t < m.nt; ++t) {
    const int32_t* T = &m.tets[4 * t];
    for (int a = 0; a < 4; ++a) {
      VIE_REQUIRE(T[a] >= 0 && T[a] < m.nv, VIE_EINVAL, "tet vertex id out of range");
      for (int b = 0; b < a; ++b) VIE_REQUIRE(T[a] != T[b], VIE_EINVAL, "tet with a repeated vertex");
    }
    const double* P0 = &m.xyz[3 * T[0]];
    double e[3][3];
    for (int a = 0; a < 3; ++a)
      for (int d = 0; d < 3; ++d) e[a][d] = m.xyz[3 * T[a + 1] + d] - P0[d];
    const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                       e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                       e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    VIE_REQUIRE(std::abs(det) > 0.0 && std::isfinite(det), VIE_EINVAL, "degenerate tet (zero volume)");
    VIE_REQUIRE(std::isfinite(m.eps[2 * t]) && std::isfinite(m.eps[2 * t + 1]) &&
                    (m.eps[2 * t] != 0.0 || m.eps[2 * t + 1] != 0.0),
                VIE_EINVAL, "eps_r must be finite and nonzero");
  }
  double sum = 0.0;
  for (int64_t t = 0; t < m.nt; ++t) {
    const int32_t* T = &m.tets[4 * t];
    double emin = INFINITY;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        const double dx = m.xyz[3 * T[b]] - m.xyz[3 * T[a]];
        const double dy = m.xyz[3 * T[b] + 1] - m.xyz[3 * T[a] + 1];
        const double dz = m.xyz[3 * T[b] + 2] - m.xyz[3 * T[a] + 2];
        emin = std::min(emin, std::sqrt((dx * dx + dy * dy) + dz * dz));
      }
    sum += emin;
  }
  m.h = sum / double(m.nt);
  m.cells.resize(3 * m.nt);
  for (int64_t t = 0; t < m.nt; ++t) {
    const int32_t* T = &m.tets[4 * t];
    for (int d = 0; d < 3; ++d) {
      const double c = (((m.xyz[3 * T[0] + d] + m.xyz[3 * T[1] + d]) + m.xyz[3 * T[2] + d]) + m.xyz[3 * T[3] + d]) * 0.25;
      const double q = std::floor(c / m.h);
      VIE_REQUIRE(std::abs(q) < double(1 << 30), VIE_EINVAL, "tet far from the origin for its size");
      m.cells[3 * t + d] = (int32_t)q;
    }
  }
  make_face_table(m);
}

std::vector<double> face_centroids(const Mesh& m) {
  std::vector<double> pts(3 * m.nf);
  for (int64_t f = 0; f < m.nf; ++f)
    for (int d = 0; d < 3; ++d) {
      double a, b, c;
      if (m.general) {
        a = m.xyz[3 * m.faces[3 * f] + d];
        b = m.xyz[3 * m.faces[3 * f + 1] + d];
        c = m.xyz[3 * m.faces[3 * f + 2] + d];
      } else {
        a = double(m.vlat[3 * m.faces[3 * f] + d]) * m.h;
        b = double(m.vlat[3 * m.faces[3 * f + 1] + d]) * m.h;
        c = double(m.vlat[3 * m.faces[3 * f + 2] + d]) * m.h;
      }
      pts[3 * f + d] = ((a + b) + c) / 3.0;
    }
  return pts;
}

// ---------------------------------------------------------------------------
// KD cluster tree (Sec. III-A): split along the longest bounding-box axis
// (ties: lowest axis), order by coordinate (ties: face id), left = ceil(n/2).
// ---------------------------------------------------------------------------
void build_tree(const std::vector<double>& pts, int leaf, Tree& t) {
  const int64_t n = (int64_t)pts.size() / 3;
  t.levels = n <= leaf ? 0 : (int)std::ceil(std::log2(double(n) / double(leaf)));
  t.perm.resize(n);
  std::iota(t.perm.begin(), t.perm.end(), 0);
  t.bounds.assign(1, std::vector<int64_t>{0, n});
  t.bbox.clear();
  auto node_bbox = [&](int64_t a, int64_t b, double* bb) {
    for (int d = 0; d < 3; ++d) { bb[d] = INFINITY; bb[3 + d] = -INFINITY; }
    for (int64_t i = a; i < b; ++i)
      for (int d = 0; d < 3; ++d) {
        double x = pts[3 * t.perm[i] + d];
        bb[d] = std::min(bb[d], x);
        bb[3 + d] = std::max(bb[3 + d], x);
      }
  };
  for (int l = 0; l <= t.levels; ++l) {
    const auto& b = t.bounds[l];
    const int64_t nn = (int64_t)b.size() - 1;
    std::vector<double> bb(6 * nn);
    for (int64_t i = 0; i < nn; ++i) node_bbox(b[i], b[i + 1], &bb[6 * i]);
    t.bbox.push_back(bb);
    if (l == t.levels) break;
    std::vector<int64_t> nxt{0};
    for (int64_t i = 0; i < nn; ++i) {
      const int64_t a = b[i], e = b[i + 1];
      int ax = 0;
      double ext[3];
      for (int d = 0; d < 3; ++d) ext[d] = e > a ? bb[6 * i + 3 + d] - bb[6 * i + d] : 0.0;
      for (int d = 1; d < 3; ++d)
        if (ext[d] > ext[ax]) ax = d;
      std::sort(t.perm.begin() + a, t.perm.begin() + e, [&](int32_t x, int32_t y) {
        double cx = pts[3 * x + ax], cy = pts[3 * y + ax];
        if (cx != cy) return cx < cy;
        return x < y;
      });
      nxt.push_back(a + (e - a + 1) / 2);
      nxt.push_back(e);
    }
    t.bounds.push_back(nxt);
  }
}

// ---------------------------------------------------------------------------
// Quadrature: symmetric degree-2 rules and Stroud conical product rules.
// Gauss-Jacobi nodes from the Golub-Welsch eigenproblem of the Jacobi matrix
// of the weight (1-x)^alpha on [-1, 1] (cyclic Jacobi eigenvalue iteration).
// ---------------------------------------------------------------------------
static void gauss_jacobi01(int n, int alpha, std::vector<double>& x, std::vector<double>& w) {
  const double al = alpha, be = 0.0;
  std::vector<double> A(n * n, 0.0), Vv(n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    double s = 2.0 * k + al + be;
    A[k * n + k] = (k == 0) ? (be - al) / (al + be + 2.0) : (be * be - al * al) / (s * (s + 2.0));
    if (k >= 1) {
      double num = 4.0 * k * (k + al) * (k + be) * (k + al + be);
      double den = s * s * (s + 1.0) * (s - 1.0);
      A[k * n + k - 1] = A[(k - 1) * n + k] = std::sqrt(num / den);
    }
    Vv[k * n + k] = 1.0;
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-32) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::abs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double tt = (theta >= 0 ? 1.0 : -1.0) / (std::abs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < n; ++k) {  // A <- J^T A J
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = Vv[k * n + p], vkq = Vv[k * n + q];
          Vv[k * n + p] = c * vkp - s * vkq;
          Vv[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  const double mu0 = alpha == 0 ? 2.0 : (alpha == 1 ? 2.0 : 8.0 / 3.0);
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[a * n + a] < A[b * n + b]; });
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    int k = idx[i];
    x[i] = 0.5 * (1.0 + A[k * n + k]);
    w[i] = mu0 * Vv[0 * n + k] * Vv[0 * n + k] / std::pow(2.0, alpha + 1);
  }
}

Rule rule_tet4() {
  Rule r;
  r.n = 4;
  const double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
  for (int q = 0; q < 4; ++q) {
    for (int k = 0; k < 4; ++k) r.lam.push_back(q == k ? a : b);
    r.w.push_back(0.25);
  }
  return r;
}

Rule rule_tri3() {
  Rule r;
  r.n = 3;
  for (int q = 0; q < 3; ++q) {
    for (int k = 0; k < 3; ++k) r.lam.push_back(q == k ? 2.0 / 3.0 : 1.0 / 6.0);
    r.w.push_back(1.0 / 3.0);
  }
  return r;
}

Rule rule_tet_conical(int n) {
  std::vector<double> u, wu, v, wv, s, ws;
  gauss_jacobi01(n, 2, u, wu);
  gauss_jacobi01(n, 1, v, wv);
  gauss_jacobi01(n, 0, s, ws);
  Rule r;
  r.n = n * n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        double x = u[i], y = (1.0 - u[i]) * v[j], z = (1.0 - u[i]) * (1.0 - v[j]) * s[k];
        r.lam.insert(r.lam.end(), {1.0 - x - y - z, x, y, z});
        r.w.push_back(6.0 * wu[i] * wv[j] * ws[k]);
      }
  return r;
}

Rule rule_tri_conical(int n) {
  std::vector<double> u, wu, v, wv;
  gauss_jacobi01(n, 1, u, wu);
  gauss_jacobi01(n, 0, v, wv);
  Rule r;
  r.n = n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double x = u[i], y = (1.0 - u[i]) * v[j];
      r.lam.insert(r.lam.end(), {1.0 - x - y, x, y});
      r.w.push_back(2.0 * wu[i] * wv[j]);
    }
  return r;
}

}  // namespace vie
