// Galerkin SWG entries of the D-VIE on the GPU (FP64), Eqs. (1)-(5).
//
//   Z(m,n) =   int f_m.f_n/eps_r
//            - k0^2 int int f_m(r).kappa(r') f_n(r') g
//            + int int (div f_m)(r) (div' kappa f_n)(r') g,   g = exp(-j k0 R)/(4 pi R)
//
// with distributional divergences: the test side carries -1 on a boundary
// (half-SWG) face, the source side kappa(T-) - kappa(T+) on face n.
//
// GB300 design: the mesh is a voxel lattice, so the interaction integrals of a
// pair of elements (a tetrahedron or one of its faces) depend only on the two
// Kuhn types and on the voxel offset.  Every pair within Chebyshev voxel
// distance 2 (the near and mid quadrature tiers) is integrated once into a
// small table of geometric moments (M0, M1, M1', M2 for volume pairs, the
// scalar integral for every element pair); an entry is then a handful of
// table reads combined with the SWG coefficients and the kappa's.  Far pairs
// (distance >= 3) are integrated on the fly with the 4-point rules.
// Quadrature specification (the paper is silent on it):
//   far : tet4 x tet4, tri3 x tri3 on the full kernel
//   mid : conical(2) x conical(2) on the full kernel
//   near: 1/(4 pi R) integrated in closed form over the source element (flat
//         triangle potential; a tetrahedron reduced to its faces), conical(3)
//         over the observer; smooth remainder (exp(-j k0 R) - 1)/(4 pi R) with
//         conical(2) on both sides.
#include <math.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace vie {

struct Tab {               // one (type p, type q, voxel offset) entry
  double2 S[5][5];         // element pairs: 0 = volume, 1 + a = local face a
  double2 M1[3], M1p[3], M2;
  double2 pad;
};

__constant__ double c_area[6][4];        // face areas of the Kuhn tets (pitch h)
__constant__ double c_nrm[6][4][3];      // outward unit normals
__constant__ double c_tet4[4][5];        // lam[4], w
__constant__ double c_tri3[3][4];        // lam[3], w
__constant__ double c_tetc2[8][5];
__constant__ double c_tetc3[27][5];
__constant__ double c_tric2[4][4];
__constant__ double c_tric3[9][4];
__constant__ int c_kuhn[6][4][3];
__constant__ int c_loc[4][3];

static constexpr double kPi = 3.14159265358979323846;
static constexpr double kInv4Pi = 0.079577471545947667884;  // 1/(4 pi)

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

struct V3 { double x, y, z; };
__device__ __forceinline__ V3 v3(double x, double y, double z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double norm(V3 a) { return sqrt(dot(a, a)); }

__device__ __forceinline__ double2 green(double R, double k0) {
  double s, c;
  sincos(k0 * R, &s, &c);
  double f = kInv4Pi / R;
  return make_double2(c * f, -s * f);
}

__device__ __forceinline__ double2 green_smooth(double R, double k0) {
  if (R <= 0.0) return make_double2(0.0, -k0 * kInv4Pi);
  double s, c, sh, ch;
  sincos(k0 * R, &s, &c);
  sincos(0.5 * k0 * R, &sh, &ch);
  double f = kInv4Pi / R;
  return make_double2(-2.0 * sh * sh * f, -s * f);
}

// vertices of a Kuhn tet of type p at voxel offset (dx,dy,dz), relative to the origin voxel corner
__device__ __forceinline__ V3 kuhn_vertex(int p, int a, int dx, int dy, int dz, double h) {
  return v3(double(dx + c_kuhn[p][a][0]) * h, double(dy + c_kuhn[p][a][1]) * h, double(dz + c_kuhn[p][a][2]) * h);
}

// int_T 1/|r-r'| ds' and int_T |r-r'| ds' over the flat triangle ABC (closed form,
// Wilton et al. 1984 / Graglia 1993): per edge, the in-plane distance to the edge line
// and the two edge-end distances give the log and arctan terms of both potentials.
__device__ void tri_pot(V3 r, V3 A, V3 B, V3 C, double& Im1, double& I1) {
  V3 n = cross(B - A, C - A);
  n = (1.0 / norm(n)) * n;
  double d = dot(r - A, n), ad = fabs(d);
  V3 rho = r - d * n;
  double im1 = 0.0, s1 = 0.0;
  V3 P[3] = {A, B, C};
  for (int e = 0; e < 3; ++e) {
    V3 P1 = P[e], P2 = P[(e + 1) % 3];
    V3 ed = P2 - P1;
    V3 lh = (1.0 / norm(ed)) * ed;
    V3 uh = cross(lh, n);
    double t0 = dot(P1 - rho, uh);
    double lp = dot(P2 - rho, lh), lm = dot(P1 - rho, lh);
    double R02 = t0 * t0 + d * d;
    double Rp = sqrt(lp * lp + R02), Rm = sqrt(lm * lm + R02);
    double tiny = 1e-30 + 1e-24 * (lp * lp + lm * lm);
    if (R02 > tiny) {
      double num = lp >= 0 ? Rp + lp : R02 / (Rp - lp);
      double den = lm >= 0 ? Rm + lm : R02 / (Rm - lm);
      double f = log(num / den);
      double beta = atan2(t0 * lp, R02 + ad * Rp) - atan2(t0 * lm, R02 + ad * Rm);
      im1 += t0 * f - ad * beta;
      s1 += t0 * (R02 * f + lp * Rp - lm * Rm);
    } else {
      s1 += t0 * (lp * Rp - lm * Rm);
    }
  }
  Im1 = im1;
  I1 = (d * d * im1 + 0.5 * s1) / 3.0;
}

// U = int_T 1/R dv', W = int_T (r'-r)/R dv' for the tet (type q, voxel offset off)
__device__ void tet_pot(V3 r, int q, int ox, int oy, int oz, double h, double& U, V3& W) {
  U = 0.0;
  W = v3(0, 0, 0);
  for (int f = 0; f < 4; ++f) {
    V3 A = kuhn_vertex(q, c_loc[f][0], ox, oy, oz, h);
    V3 B = kuhn_vertex(q, c_loc[f][1], ox, oy, oz, h);
    V3 C = kuhn_vertex(q, c_loc[f][2], ox, oy, oz, h);
    V3 nf = v3(c_nrm[q][f][0], c_nrm[q][f][1], c_nrm[q][f][2]);
    double hf = dot(A - r, nf);
    double im1, i1;
    tri_pot(r, A, B, C, im1, i1);
    if (fabs(hf) > 0.0) U += 0.5 * hf * im1;
    W = W + i1 * nf;
  }
}

// quadrature points of an element (tet or local face) of type p at offset o
struct Elem {
  int p, face;  // face = -1: volume
  int ox, oy, oz;
};

__device__ __forceinline__ int rule_size(int face, int level) {
  // level 0 far (tet4 / tri3), 2 conical(2), 3 conical(3)
  if (face < 0) return level == 0 ? 4 : (level == 2 ? 8 : 27);
  return level == 0 ? 3 : (level == 2 ? 4 : 9);
}

__device__ V3 rule_point(const Elem& e, int level, int i, double h, double& w) {
  const double vol = h * h * h / 6.0;
  if (e.face < 0) {
    const double* row = level == 0 ? c_tet4[i] : (level == 2 ? c_tetc2[i] : c_tetc3[i]);
    V3 r = v3(0, 0, 0);
    for (int a = 0; a < 4; ++a) r = r + row[a] * kuhn_vertex(e.p, a, e.ox, e.oy, e.oz, h);
    w = row[4] * vol;
    return r;
  }
  const double* row = level == 0 ? c_tri3[i] : (level == 2 ? c_tric2[i] : c_tric3[i]);
  V3 r = v3(0, 0, 0);
  for (int a = 0; a < 3; ++a) r = r + row[a] * kuhn_vertex(e.p, c_loc[e.face][a], e.ox, e.oy, e.oz, h);
  w = row[3] * c_area[e.p][e.face] * h * h;
  return r;
}

// ---------------------------------------------------------------------------
// table kernel: one CTA per (p, q, offset), thread t < 25 -> S[t/5][t%5];
// thread 0 also the vector moments of the volume pair.
// ---------------------------------------------------------------------------
__global__ void table_kernel(Tab* tab, double h, double k0) {
  const int idx = blockIdx.x;
  const int p = idx / (6 * 125), q = (idx / 125) % 6, o = idx % 125;
  const int ox = o / 25 - 2, oy = (o / 5) % 5 - 2, oz = o % 5 - 2;
  const int t = threadIdx.x;
  if (t >= 25) return;
  const int eo = t / 5 - 1, es = t % 5 - 1;
  const int tier = max(abs(ox), max(abs(oy), abs(oz)));
  Elem A{p, eo, 0, 0, 0}, B{q, es, ox, oy, oz};
  double2 S = make_double2(0, 0), M1[3], M1p[3], M2 = make_double2(0, 0);
  for (int d = 0; d < 3; ++d) M1[d] = M1p[d] = make_double2(0, 0);
  const bool vv = (eo < 0 && es < 0);
  if (tier == 2) {
    for (int i = 0; i < rule_size(eo, 2); ++i) {
      double wi;
      V3 ri = rule_point(A, 2, i, h, wi);
      for (int j = 0; j < rule_size(es, 2); ++j) {
        double wj;
        V3 rj = rule_point(B, 2, j, h, wj);
        double2 g = cscale(green(norm(ri - rj), k0), wi * wj);
        S = cadd(S, g);
        if (vv) {
          M1[0] = cadd(M1[0], cscale(g, ri.x)); M1[1] = cadd(M1[1], cscale(g, ri.y)); M1[2] = cadd(M1[2], cscale(g, ri.z));
          M1p[0] = cadd(M1p[0], cscale(g, rj.x)); M1p[1] = cadd(M1p[1], cscale(g, rj.y)); M1p[2] = cadd(M1p[2], cscale(g, rj.z));
          M2 = cadd(M2, cscale(g, dot(ri, rj)));
        }
      }
    }
  } else if (tier <= 1) {
    // static part: closed form over the source, conical(3) over the observer
    for (int i = 0; i < rule_size(eo, 3); ++i) {
      double wi;
      V3 ri = rule_point(A, 3, i, h, wi);
      if (es < 0) {
        double U;
        V3 W;
        tet_pot(ri, q, ox, oy, oz, h, U, W);
        double u = wi * U * kInv4Pi;
        S.x += u;
        if (vv) {
          V3 inner = W + U * ri;  // int rho'/R over the source
          M1[0].x += u * ri.x; M1[1].x += u * ri.y; M1[2].x += u * ri.z;
          double c = wi * kInv4Pi;
          M1p[0].x += c * inner.x; M1p[1].x += c * inner.y; M1p[2].x += c * inner.z;
          M2.x += c * dot(ri, inner);
        }
      } else {
        V3 Av = kuhn_vertex(q, c_loc[es][0], ox, oy, oz, h);
        V3 Bv = kuhn_vertex(q, c_loc[es][1], ox, oy, oz, h);
        V3 Cv = kuhn_vertex(q, c_loc[es][2], ox, oy, oz, h);
        double im1, i1;
        tri_pot(ri, Av, Bv, Cv, im1, i1);
        S.x += wi * im1 * kInv4Pi;
      }
    }
    // smooth remainder: conical(2) on both sides
    for (int i = 0; i < rule_size(eo, 2); ++i) {
      double wi;
      V3 ri = rule_point(A, 2, i, h, wi);
      for (int j = 0; j < rule_size(es, 2); ++j) {
        double wj;
        V3 rj = rule_point(B, 2, j, h, wj);
        double2 g = cscale(green_smooth(norm(ri - rj), k0), wi * wj);
        S = cadd(S, g);
        if (vv) {
          M1[0] = cadd(M1[0], cscale(g, ri.x)); M1[1] = cadd(M1[1], cscale(g, ri.y)); M1[2] = cadd(M1[2], cscale(g, ri.z));
          M1p[0] = cadd(M1p[0], cscale(g, rj.x)); M1p[1] = cadd(M1p[1], cscale(g, rj.y)); M1p[2] = cadd(M1p[2], cscale(g, rj.z));
          M2 = cadd(M2, cscale(g, dot(ri, rj)));
        }
      }
    }
  }
  Tab& T = tab[idx];
  T.S[eo + 1][es + 1] = S;
  if (vv) {
    for (int d = 0; d < 3; ++d) { T.M1[d] = M1[d]; T.M1p[d] = M1p[d]; }
    T.M2 = M2;
  }
}

// ---------------------------------------------------------------------------
// entry evaluation
// ---------------------------------------------------------------------------
struct EntryCtx {
  const FaceDev* faces;
  const TetDev* tets;   // general meshes: vx, vy, vz hold the tet's tier cell
  const Tab* tab;       // voxel meshes only
  const TetGeo* geo;    // general meshes only
  double h, k0;
  int general;
};

__device__ __forceinline__ const Tab* tab_lookup(const EntryCtx& c, int p, int q, int dx, int dy, int dz) {
  return &c.tab[(p * 6 + q) * 125 + (dx + 2) * 25 + (dy + 2) * 5 + (dz + 2)];
}

__device__ __forceinline__ double2 ld2(const double2* p) { return __ldg(p); }

// far tier: int int over two elements with the 4-point / 3-point rules
__device__ double2 far_scalar(const EntryCtx& c, const Elem& A, const Elem& B) {
  double2 s = make_double2(0, 0);
  for (int i = 0; i < rule_size(A.face, 0); ++i) {
    double wi;
    V3 ri = rule_point(A, 0, i, c.h, wi);
    for (int j = 0; j < rule_size(B.face, 0); ++j) {
      double wj;
      V3 rj = rule_point(B, 0, j, c.h, wj);
      s = cadd(s, cscale(green(norm(ri - rj), c.k0), wi * wj));
    }
  }
  return s;
}

// far tier in FP32 (used by the HOD-BF builder): the 4-point rules of both tets, relative
// coordinates, FP32 kernel evaluations; the result is accurate to ~1e-6 relative.
struct F3 { float x, y, z; };
__device__ __forceinline__ F3 f3_point(int p, int i, int ox, int oy, int oz, float h) {
  F3 r{0.f, 0.f, 0.f};
  for (int a = 0; a < 4; ++a) {
    const float l = (float)c_tet4[i][a];
    r.x += l * (float)(ox + c_kuhn[p][a][0]) * h;
    r.y += l * (float)(oy + c_kuhn[p][a][1]) * h;
    r.z += l * (float)(oz + c_kuhn[p][a][2]) * h;
  }
  return r;
}

__device__ void far_tet_pair_f32(const EntryCtx& c, int pa, int pb, int dx, int dy, int dz, V3 qa, V3 qb,
                                 double2& sum, double2& sumv) {
  const float h = (float)c.h, k0 = (float)c.k0, w = (float)(0.25 * c.h * c.h * c.h / 6.0);
  float sr = 0.f, si = 0.f, vr = 0.f, vi = 0.f;
  F3 rj[4];
  for (int j = 0; j < 4; ++j) rj[j] = f3_point(pb, j, dx, dy, dz, h);
  for (int i = 0; i < 4; ++i) {
    const F3 ri = f3_point(pa, i, 0, 0, 0, h);
    const float ax = ri.x - (float)qa.x, ay = ri.y - (float)qa.y, az = ri.z - (float)qa.z;
    for (int j = 0; j < 4; ++j) {
      const float ex = ri.x - rj[j].x, ey = ri.y - rj[j].y, ez = ri.z - rj[j].z;
      const float R = sqrtf(ex * ex + ey * ey + ez * ez);
      float sn, cs;
      sincosf(k0 * R, &sn, &cs);
      const float f = (float)kInv4Pi * w * w / R;
      const float gr = cs * f, gi = -sn * f;
      sr += gr;
      si += gi;
      const float d = ax * (rj[j].x - (float)qb.x) + ay * (rj[j].y - (float)qb.y) + az * (rj[j].z - (float)qb.z);
      vr += gr * d;
      vi += gi * d;
    }
  }
  sum = make_double2(sr, si);
  sumv = make_double2(vr, vi);
}

// contribution of the tet pair (T, a) x (T', b) to Z(m, n)
template <bool FAR32>
__device__ double2 tet_pair(const EntryCtx& c, int T, int a, double sa, int Tp, int b, double sb) {
  const TetDev tA = c.tets[T], tB = c.tets[Tp];
  const int dx = tB.vx - tA.vx, dy = tB.vy - tA.vy, dz = tB.vz - tA.vz;
  const double h = c.h, vol = h * h * h / 6.0;
  const double ca = sa * c_area[tA.type][a] * h * h / (3.0 * vol);
  const double cb = sb * c_area[tB.type][b] * h * h / (3.0 * vol);
  const double diva = 3.0 * ca, divb = 3.0 * cb;
  const V3 qa = kuhn_vertex(tA.type, a, 0, 0, 0, h);
  const V3 qb = kuhn_vertex(tB.type, b, dx, dy, dz, h);
  double2 Avec, Phi;
  const int tier = max(abs(dx), max(abs(dy), abs(dz)));
  if (tier <= 2) {
    const Tab* e = tab_lookup(c, tA.type, tB.type, dx, dy, dz);
    double2 M0 = ld2(&e->S[0][0]);
    double2 m1[3] = {ld2(&e->M1[0]), ld2(&e->M1[1]), ld2(&e->M1[2])};
    double2 m1p[3] = {ld2(&e->M1p[0]), ld2(&e->M1p[1]), ld2(&e->M1p[2])};
    double2 M2 = ld2(&e->M2);
    double2 qbM1 = cadd(cadd(cscale(m1[0], qb.x), cscale(m1[1], qb.y)), cscale(m1[2], qb.z));
    double2 qaM1p = cadd(cadd(cscale(m1p[0], qa.x), cscale(m1p[1], qa.y)), cscale(m1p[2], qa.z));
    double2 I = make_double2(M2.x - qbM1.x - qaM1p.x + dot(qa, qb) * M0.x,
                             M2.y - qbM1.y - qaM1p.y + dot(qa, qb) * M0.y);
    Avec = cscale(I, ca * cb);
    Phi = M0;
  } else if (FAR32) {
    double2 s, sv;
    far_tet_pair_f32(c, tA.type, tB.type, dx, dy, dz, qa, qb, s, sv);
    Avec = cscale(sv, ca * cb);
    Phi = s;
  } else {
    Elem EA{tA.type, -1, 0, 0, 0}, EB{tB.type, -1, dx, dy, dz};
    double2 s = make_double2(0, 0), sv = make_double2(0, 0);
    for (int i = 0; i < 4; ++i) {
      double wi;
      V3 ri = rule_point(EA, 0, i, h, wi);
      for (int j = 0; j < 4; ++j) {
        double wj;
        V3 rj = rule_point(EB, 0, j, h, wj);
        double2 g = cscale(green(norm(ri - rj), c.k0), wi * wj);
        s = cadd(s, g);
        sv = cadd(sv, cscale(g, dot(ri - qa, rj - qb)));
      }
    }
    Avec = cscale(sv, ca * cb);
    Phi = s;
  }
  const double2 kap = make_double2(tB.kap_re, tB.kap_im);
  const double k2 = c.k0 * c.k0;
  double2 z = cmul(kap, make_double2(-k2 * Avec.x + diva * divb * Phi.x, -k2 * Avec.y + diva * divb * Phi.y));
  if (T == Tp) {  // Gram term, tet4 (exact for the quadratic integrand)
    Elem EA{tA.type, -1, 0, 0, 0};
    double g = 0.0;
    for (int i = 0; i < 4; ++i) {
      double wi;
      V3 ri = rule_point(EA, 0, i, h, wi);
      g += wi * dot(ri - qa, ri - qb);
    }
    z = cadd(z, cscale(make_double2(tA.inveps_re, tA.inveps_im), g * ca * cb));
  }
  return z;
}

// scalar int int g between two elements attached to tets T (obs) and Tp (src)
__device__ double2 pair_scalar(const EntryCtx& c, int T, int fa, int Tp, int fb) {
  const TetDev tA = c.tets[T], tB = c.tets[Tp];
  const int dx = tB.vx - tA.vx, dy = tB.vy - tA.vy, dz = tB.vz - tA.vz;
  const int tier = max(abs(dx), max(abs(dy), abs(dz)));
  if (tier <= 2) return ld2(&tab_lookup(c, tA.type, tB.type, dx, dy, dz)->S[fa + 1][fb + 1]);
  return far_scalar(c, Elem{tA.type, fa, 0, 0, 0}, Elem{tB.type, fb, dx, dy, dz});
}

template <bool FAR32>
__device__ double2 entry(const EntryCtx& c, int m, int n) {
  const FaceDev Fm = c.faces[m], Fn = c.faces[n];
  const double h = c.h, vol = h * h * h / 6.0;
  double2 z = make_double2(0, 0);
  const int Tm[2] = {Fm.tp, Fm.tm}, Am[2] = {Fm.lp, Fm.lm};
  const int Tn[2] = {Fn.tp, Fn.tm}, Bn[2] = {Fn.lp, Fn.lm};
  for (int i = 0; i < 2; ++i) {
    if (Tm[i] < 0) continue;
    for (int j = 0; j < 2; ++j) {
      if (Tn[j] < 0) continue;
      z = cadd(z, tet_pair<FAR32>(c, Tm[i], Am[i], i == 0 ? 1.0 : -1.0, Tn[j], Bn[j], j == 0 ? 1.0 : -1.0));
    }
  }
  const double2 jump = make_double2(Fn.jump_re, Fn.jump_im);
  const bool has_jump = (jump.x != 0.0 || jump.y != 0.0);
  if (Fm.boundary) {
    // test surface (density -1 on face m, owned by T+ of m) x source volume kappa div f_n
    for (int j = 0; j < 2; ++j) {
      if (Tn[j] < 0) continue;
      const TetDev tB = c.tets[Tn[j]];
      double divb = (j == 0 ? 1.0 : -1.0) * c_area[tB.type][Bn[j]] * h * h / vol;
      double2 s = pair_scalar(c, Fm.tp, Fm.lp, Tn[j], -1);
      z = cadd(z, cscale(cmul(make_double2(tB.kap_re, tB.kap_im), s), -divb));
    }
  }
  if (has_jump) {
    // test volume div f_m x source surface (density jump on face n, owned by T+ of n)
    for (int i = 0; i < 2; ++i) {
      if (Tm[i] < 0) continue;
      const TetDev tA = c.tets[Tm[i]];
      double diva = (i == 0 ? 1.0 : -1.0) * c_area[tA.type][Am[i]] * h * h / vol;
      double2 s = pair_scalar(c, Tm[i], -1, Fn.tp, Fn.lp);
      z = cadd(z, cscale(cmul(jump, s), diva));
    }
    if (Fm.boundary) {
      double2 s = pair_scalar(c, Fm.tp, Fm.lp, Fn.tp, Fn.lp);
      z = cadd(z, cscale(cmul(jump, s), -1.0));
    }
  }
  return z;
}

// ---------------------------------------------------------------------------
// general tetrahedral meshes: every element pair integrated on the fly with the
// same quadrature specification as the lattice tables (tiers from the tets'
// cells), the vertices taken from the tet's own geometry record
// ---------------------------------------------------------------------------
__device__ __forceinline__ V3 gvert(const TetGeo& g, int a) { return v3(g.P[a][0], g.P[a][1], g.P[a][2]); }

// point i of the level-`level` rule over the tet (face < 0) or its local face `face`;
// face rules run over the face's vertices in increasing global vertex id
__device__ V3 grule_point(const TetGeo& g, int face, int level, int i, double& w) {
  V3 r = v3(0, 0, 0);
  if (face < 0) {
    const double* row = level == 0 ? c_tet4[i] : (level == 2 ? c_tetc2[i] : c_tetc3[i]);
    for (int a = 0; a < 4; ++a) r = r + row[a] * gvert(g, a);
    w = row[4] * g.vol;
    return r;
  }
  const double* row = level == 0 ? c_tri3[i] : (level == 2 ? c_tric2[i] : c_tric3[i]);
  for (int a = 0; a < 3; ++a) r = r + row[a] * gvert(g, g.fv[face][a]);
  w = row[3] * g.area[face];
  return r;
}

// U = int_T 1/R dv', W = int_T (r'-r)/R dv' over a general tet
__device__ void gtet_pot(V3 r, const TetGeo& g, double& U, V3& W) {
  U = 0.0;
  W = v3(0, 0, 0);
  for (int f = 0; f < 4; ++f) {
    const V3 A = gvert(g, g.fv[f][0]), B = gvert(g, g.fv[f][1]), C = gvert(g, g.fv[f][2]);
    const V3 nf = v3(g.nrm[f][0], g.nrm[f][1], g.nrm[f][2]);
    const double hf = dot(A - r, nf);
    double im1, i1;
    tri_pot(r, A, B, C, im1, i1);
    if (fabs(hf) > 0.0) U += 0.5 * hf * im1;
    W = W + i1 * nf;
  }
}

// tier of two elements held by tets T and Tp: Chebyshev distance of the tets' cells,
// at most 1 (near) when the tets share a vertex
__device__ __forceinline__ int gtier(const EntryCtx& c, int T, int Tp) {
  const TetDev a = c.tets[T], b = c.tets[Tp];
  int tier = max(abs(b.vx - a.vx), max(abs(b.vy - a.vy), abs(b.vz - a.vz)));
  if (tier > 1) {
    const TetGeo& ga = c.geo[T];
    const TetGeo& gb = c.geo[Tp];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if (ga.vid[i] == gb.vid[j]) tier = 1;
  }
  return tier;
}

// far tier in FP32 for the builder: tet4 x tet4, coordinates relative to the observer
// tet's first vertex (formed in FP64), FP32 kernel evaluations
__device__ void gfar_tet_pair_f32(const TetGeo& gA, const TetGeo& gB, V3 qa, V3 qb, double k0, double2& sum,
                                  double2& sumv) {
  const V3 o = gvert(gA, 0);
  float sr = 0.f, si = 0.f, vr = 0.f, vi = 0.f;
  F3 rj[4];
  float wj[4];
  for (int j = 0; j < 4; ++j) {
    V3 r = v3(0, 0, 0);
    for (int a = 0; a < 4; ++a) r = r + c_tet4[j][a] * (gvert(gB, a) - o);
    rj[j] = F3{(float)r.x, (float)r.y, (float)r.z};
    wj[j] = (float)(c_tet4[j][4] * gB.vol);
  }
  const V3 qar = qa - o, qbr = qb - o;
  for (int i = 0; i < 4; ++i) {
    V3 r = v3(0, 0, 0);
    for (int a = 0; a < 4; ++a) r = r + c_tet4[i][a] * (gvert(gA, a) - o);
    const F3 ri{(float)r.x, (float)r.y, (float)r.z};
    const float wi = (float)(c_tet4[i][4] * gA.vol);
    const float ax = ri.x - (float)qar.x, ay = ri.y - (float)qar.y, az = ri.z - (float)qar.z;
    for (int j = 0; j < 4; ++j) {
      const float ex = ri.x - rj[j].x, ey = ri.y - rj[j].y, ez = ri.z - rj[j].z;
      const float R = sqrtf(ex * ex + ey * ey + ez * ez);
      float sn, cs;
      sincosf((float)k0 * R, &sn, &cs);
      const float f = (float)kInv4Pi * wi * wj[j] / R;
      const float gr = cs * f, gi = -sn * f;
      sr += gr;
      si += gi;
      const float d = ax * (rj[j].x - (float)qbr.x) + ay * (rj[j].y - (float)qbr.y) + az * (rj[j].z - (float)qbr.z);
      vr += gr * d;
      vi += gi * d;
    }
  }
  sum = make_double2(sr, si);
  sumv = make_double2(vr, vi);
}

// contribution of the tet pair (T, a) x (T', b) to Z(m, n) on a general mesh:
// A = int int g (r - q_a).(r' - q_b), Phi = int int g
template <bool FAR32>
__device__ double2 gtet_pair(const EntryCtx& c, int T, int a, double sa, int Tp, int b, double sb) {
  const TetDev tA = c.tets[T], tB = c.tets[Tp];
  const TetGeo& gA = c.geo[T];
  const TetGeo& gB = c.geo[Tp];
  const double ca = sa * gA.area[a] / (3.0 * gA.vol), cb = sb * gB.area[b] / (3.0 * gB.vol);
  const double diva = 3.0 * ca, divb = 3.0 * cb;
  const V3 qa = gvert(gA, a), qb = gvert(gB, b);
  const int tier = gtier(c, T, Tp);
  double2 A = make_double2(0, 0), Phi = make_double2(0, 0);
  if (tier <= 1) {
    // 1/(4 pi R): closed form over the source tet, conical(3) over the observer
    for (int i = 0; i < 27; ++i) {
      double wi;
      const V3 ri = grule_point(gA, -1, 3, i, wi);
      double U;
      V3 W;
      gtet_pot(ri, gB, U, W);
      const double cw = wi * kInv4Pi;
      Phi.x += cw * U;
      A.x += cw * dot(ri - qa, W + U * (ri - qb));  // int (r' - q_b)/R = W + U (r - q_b)
    }
    // smooth remainder: conical(2) on both sides
    for (int i = 0; i < 8; ++i) {
      double wi;
      const V3 ri = grule_point(gA, -1, 2, i, wi);
      for (int j = 0; j < 8; ++j) {
        double wj;
        const V3 rj = grule_point(gB, -1, 2, j, wj);
        const double2 g = cscale(green_smooth(norm(ri - rj), c.k0), wi * wj);
        Phi = cadd(Phi, g);
        A = cadd(A, cscale(g, dot(ri - qa, rj - qb)));
      }
    }
  } else if (tier == 2) {
    for (int i = 0; i < 8; ++i) {
      double wi;
      const V3 ri = grule_point(gA, -1, 2, i, wi);
      for (int j = 0; j < 8; ++j) {
        double wj;
        const V3 rj = grule_point(gB, -1, 2, j, wj);
        const double2 g = cscale(green(norm(ri - rj), c.k0), wi * wj);
        Phi = cadd(Phi, g);
        A = cadd(A, cscale(g, dot(ri - qa, rj - qb)));
      }
    }
  } else if (FAR32) {
    gfar_tet_pair_f32(gA, gB, qa, qb, c.k0, Phi, A);
  } else {
    for (int i = 0; i < 4; ++i) {
      double wi;
      const V3 ri = grule_point(gA, -1, 0, i, wi);
      for (int j = 0; j < 4; ++j) {
        double wj;
        const V3 rj = grule_point(gB, -1, 0, j, wj);
        const double2 g = cscale(green(norm(ri - rj), c.k0), wi * wj);
        Phi = cadd(Phi, g);
        A = cadd(A, cscale(g, dot(ri - qa, rj - qb)));
      }
    }
  }
  const double2 kap = make_double2(tB.kap_re, tB.kap_im);
  const double k2 = c.k0 * c.k0, cab = ca * cb;
  double2 z = cmul(kap, make_double2(-k2 * cab * A.x + diva * divb * Phi.x, -k2 * cab * A.y + diva * divb * Phi.y));
  if (T == Tp) {  // Gram term, tet4 (exact for the quadratic integrand)
    double g = 0.0;
    for (int i = 0; i < 4; ++i) {
      double wi;
      const V3 ri = grule_point(gA, -1, 0, i, wi);
      g += wi * dot(ri - qa, ri - qb);
    }
    z = cadd(z, cscale(make_double2(tA.inveps_re, tA.inveps_im), g * cab));
  }
  return z;
}

// scalar int int g between element fa of tet T (observer) and element fb of tet Tp
__device__ double2 gpair_scalar(const EntryCtx& c, int T, int fa, int Tp, int fb) {
  const TetGeo& gA = c.geo[T];
  const TetGeo& gB = c.geo[Tp];
  const int tier = gtier(c, T, Tp);
  const int nA2 = fa < 0 ? 8 : 4, nB2 = fb < 0 ? 8 : 4;
  double2 S = make_double2(0, 0);
  if (tier <= 1) {
    for (int i = 0; i < (fa < 0 ? 27 : 9); ++i) {
      double wi;
      const V3 ri = grule_point(gA, fa, 3, i, wi);
      double pot;
      if (fb < 0) {
        V3 W;
        gtet_pot(ri, gB, pot, W);
      } else {
        double i1;
        tri_pot(ri, gvert(gB, gB.fv[fb][0]), gvert(gB, gB.fv[fb][1]), gvert(gB, gB.fv[fb][2]), pot, i1);
      }
      S.x += wi * pot * kInv4Pi;
    }
    for (int i = 0; i < nA2; ++i) {
      double wi;
      const V3 ri = grule_point(gA, fa, 2, i, wi);
      for (int j = 0; j < nB2; ++j) {
        double wj;
        const V3 rj = grule_point(gB, fb, 2, j, wj);
        S = cadd(S, cscale(green_smooth(norm(ri - rj), c.k0), wi * wj));
      }
    }
    return S;
  }
  const int lvl = tier == 2 ? 2 : 0;
  const int nA = rule_size(fa, lvl), nB = rule_size(fb, lvl);
  for (int i = 0; i < nA; ++i) {
    double wi;
    const V3 ri = grule_point(gA, fa, lvl, i, wi);
    for (int j = 0; j < nB; ++j) {
      double wj;
      const V3 rj = grule_point(gB, fb, lvl, j, wj);
      S = cadd(S, cscale(green(norm(ri - rj), c.k0), wi * wj));
    }
  }
  return S;
}

template <bool FAR32>
__device__ double2 gentry(const EntryCtx& c, int m, int n) {
  const FaceDev Fm = c.faces[m], Fn = c.faces[n];
  double2 z = make_double2(0, 0);
  const int Tm[2] = {Fm.tp, Fm.tm}, Am[2] = {Fm.lp, Fm.lm};
  const int Tn[2] = {Fn.tp, Fn.tm}, Bn[2] = {Fn.lp, Fn.lm};
  for (int i = 0; i < 2; ++i) {
    if (Tm[i] < 0) continue;
    for (int j = 0; j < 2; ++j) {
      if (Tn[j] < 0) continue;
      z = cadd(z, gtet_pair<FAR32>(c, Tm[i], Am[i], i == 0 ? 1.0 : -1.0, Tn[j], Bn[j], j == 0 ? 1.0 : -1.0));
    }
  }
  const double2 jump = make_double2(Fn.jump_re, Fn.jump_im);
  const bool has_jump = (jump.x != 0.0 || jump.y != 0.0);
  if (Fm.boundary) {
    for (int j = 0; j < 2; ++j) {
      if (Tn[j] < 0) continue;
      const TetDev tB = c.tets[Tn[j]];
      const double divb = (j == 0 ? 1.0 : -1.0) * c.geo[Tn[j]].area[Bn[j]] / c.geo[Tn[j]].vol;
      const double2 s = gpair_scalar(c, Fm.tp, Fm.lp, Tn[j], -1);
      z = cadd(z, cscale(cmul(make_double2(tB.kap_re, tB.kap_im), s), -divb));
    }
  }
  if (has_jump) {
    for (int i = 0; i < 2; ++i) {
      if (Tm[i] < 0) continue;
      const double diva = (i == 0 ? 1.0 : -1.0) * c.geo[Tm[i]].area[Am[i]] / c.geo[Tm[i]].vol;
      const double2 s = gpair_scalar(c, Tm[i], -1, Fn.tp, Fn.lp);
      z = cadd(z, cscale(cmul(jump, s), diva));
    }
    if (Fm.boundary) {
      const double2 s = gpair_scalar(c, Fm.tp, Fm.lp, Fn.tp, Fn.lp);
      z = cadd(z, cscale(cmul(jump, s), -1.0));
    }
  }
  return z;
}

template <bool FAR32>
__global__ void entries_pairs_kernel(EntryCtx c, const int32_t* rows, const int32_t* cols, int64_t count,
                                     double2* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = c.general ? gentry<FAR32>(c, rows[i], cols[i]) : entry<FAR32>(c, rows[i], cols[i]);
}

template <bool FAR32>
__global__ void entries_blocks_kernel(EntryCtx c, const EntryBlock* blocks, const int64_t* prefix, int nblocks,
                                      int64_t total, const int32_t* rows, const int32_t* cols, double2* out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nblocks - 1;  // last block with prefix <= g
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const EntryBlock b = blocks[lo];
    int64_t k = g - prefix[lo];
    int i = int(k % b.m), j = int(k / b.m);
    const int m = rows[b.row_off + i], n = cols[b.col_off + j];
    out[b.out_off + k] = c.general ? gentry<FAR32>(c, m, n) : entry<FAR32>(c, m, n);
  }
}

// ---------------------------------------------------------------------------
// right-hand side and far field
// ---------------------------------------------------------------------------
__global__ void rhs_kernel(EntryCtx c, int64_t n, const double* khat, const double* pol, int nrhs, double2* V) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n * nrhs; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = g % n;
    const int r = int(g / n);
    const FaceDev F = c.faces[m];
    V3 kh = v3(khat[3 * r], khat[3 * r + 1], khat[3 * r + 2]);
    V3 pl = v3(pol[3 * r], pol[3 * r + 1], pol[3 * r + 2]);
    double2 acc = make_double2(0, 0);
    const int T[2] = {F.tp, F.tm}, A[2] = {F.lp, F.lm};
    for (int s = 0; s < 2; ++s) {
      if (T[s] < 0) continue;
      if (c.general) {  // conical(3) over the tet, absolute coordinates
        const TetGeo& G = c.geo[T[s]];
        const double ca = (s == 0 ? 1.0 : -1.0) * G.area[A[s]] / (3.0 * G.vol);
        const V3 qa = gvert(G, A[s]);
        for (int i = 0; i < 27; ++i) {
          double w;
          const V3 r = grule_point(G, -1, 3, i, w);
          double sn, cs;
          sincos(-c.k0 * dot(kh, r), &sn, &cs);
          const double f = w * ca * dot(r - qa, pl);
          acc.x += f * cs;
          acc.y += f * sn;
        }
        continue;
      }
      const TetDev t = c.tets[T[s]];
      const double h = c.h, vol = h * h * h / 6.0;
      const double ca = (s == 0 ? 1.0 : -1.0) * c_area[t.type][A[s]] * h * h / (3.0 * vol);
      Elem E{t.type, -1, 0, 0, 0};
      V3 qa = kuhn_vertex(t.type, A[s], 0, 0, 0, h);
      for (int i = 0; i < 27; ++i) {
        double w;
        V3 rl = rule_point(E, 3, i, h, w);
        V3 r = v3(double(t.vx) * h, double(t.vy) * h, double(t.vz) * h) + rl;
        double sn, cs;
        sincos(-c.k0 * dot(kh, r), &sn, &cs);
        double f = w * ca * dot(rl - qa, pl);
        acc.x += f * cs;
        acc.y += f * sn;
      }
    }
    V[m + (int64_t)r * n] = acc;
  }
}

__global__ void farfield_kernel(EntryCtx c, int64_t nt, const int32_t* tet_faces, const double2* I, int64_t n,
                                const double* dirs, double2* F /* (ndir*nrhs) x 3 */, int nrhs) {
  const int dirr = blockIdx.x;  // one CTA per (direction, rhs)
  const int dd = dirr / nrhs, r = dirr % nrhs;
  V3 u = v3(dirs[3 * dd], dirs[3 * dd + 1], dirs[3 * dd + 2]);
  double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  const double h = c.h, vol = h * h * h / 6.0;
  for (int64_t T = threadIdx.x; T < nt; T += blockDim.x) {
    const TetDev t = c.tets[T];
    if (c.general) {
      const TetGeo& G = c.geo[T];
      double2 coef[4];
      double ca[4];
      for (int a = 0; a < 4; ++a) {
        const int f = tet_faces[4 * T + a];
        coef[a] = I[f + (int64_t)r * n];
        ca[a] = (c.faces[f].tp == T ? 1.0 : -1.0) * G.area[a] / (3.0 * G.vol);
      }
      for (int i = 0; i < 27; ++i) {
        double w;
        const V3 rg = grule_point(G, -1, 3, i, w);
        double2 d[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
        for (int a = 0; a < 4; ++a) {
          const V3 f = ca[a] * (rg - gvert(G, a));
          d[0] = cadd(d[0], cscale(coef[a], f.x));
          d[1] = cadd(d[1], cscale(coef[a], f.y));
          d[2] = cadd(d[2], cscale(coef[a], f.z));
        }
        double sn, cs;
        sincos(c.k0 * dot(u, rg), &sn, &cs);
        const double2 ph = cmul(make_double2(cs, sn), make_double2(t.kap_re * w, t.kap_im * w));
        for (int k = 0; k < 3; ++k) acc[k] = cadd(acc[k], cmul(ph, d[k]));
      }
      continue;
    }
    Elem E{t.type, -1, 0, 0, 0};
    double2 coef[4];
    V3 qa[4];
    double ca[4];
    for (int a = 0; a < 4; ++a) {
      int f = tet_faces[4 * T + a];
      coef[a] = I[f + (int64_t)r * n];
      FaceDev F = c.faces[f];
      double s = (F.tp == T) ? 1.0 : -1.0;
      ca[a] = s * c_area[t.type][a] * h * h / (3.0 * vol);
      qa[a] = kuhn_vertex(t.type, a, 0, 0, 0, h);
    }
    for (int i = 0; i < 27; ++i) {
      double w;
      V3 rl = rule_point(E, 3, i, h, w);
      V3 rg = v3(double(t.vx) * h, double(t.vy) * h, double(t.vz) * h) + rl;
      double2 d[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
      for (int a = 0; a < 4; ++a) {
        V3 f = ca[a] * (rl - qa[a]);
        d[0] = cadd(d[0], cscale(coef[a], f.x));
        d[1] = cadd(d[1], cscale(coef[a], f.y));
        d[2] = cadd(d[2], cscale(coef[a], f.z));
      }
      double sn, cs;
      sincos(c.k0 * dot(u, rg), &sn, &cs);
      double2 ph = cmul(make_double2(cs, sn), make_double2(t.kap_re * w, t.kap_im * w));
      for (int k = 0; k < 3; ++k) acc[k] = cadd(acc[k], cmul(ph, d[k]));
    }
  }
  __shared__ double2 red[3][256];
  for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = cadd(red[k][threadIdx.x], red[k][threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) F[3 * (int64_t)dirr + k] = red[k][0];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static void upload_constants() {
  if (done_on_device((const void*)&upload_constants)) return;
  double area[6][4], nrm[6][4][3];
  static const int loc[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  for (int p = 0; p < 6; ++p)
    for (int a = 0; a < 4; ++a) {
      double P[4][3];
      for (int v = 0; v < 4; ++v)
        for (int d = 0; d < 3; ++d) P[v][d] = kKuhn[p][v][d];
      const double* A = P[loc[a][0]];
      const double* B = P[loc[a][1]];
      const double* C = P[loc[a][2]];
      double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
      double ln = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      double s = (n[0] * (A[0] - P[a][0]) + n[1] * (A[1] - P[a][1]) + n[2] * (A[2] - P[a][2])) > 0 ? 1.0 : -1.0;
      for (int d = 0; d < 3; ++d) nrm[p][a][d] = s * n[d] / ln;
      area[p][a] = 0.5 * ln;  // in units of h^2
    }
  VIE_CUDA(cudaMemcpyToSymbol(c_area, area, sizeof(area)));
  VIE_CUDA(cudaMemcpyToSymbol(c_nrm, nrm, sizeof(nrm)));
  VIE_CUDA(cudaMemcpyToSymbol(c_kuhn, kKuhn, sizeof(kKuhn)));
  VIE_CUDA(cudaMemcpyToSymbol(c_loc, loc, sizeof(loc)));
  auto put = [](const Rule& r, int dim, void* dst, size_t bytes, const void* sym) {
    std::vector<double> buf;
    for (int q = 0; q < r.n; ++q) {
      for (int k = 0; k < dim; ++k) buf.push_back(r.lam[q * dim + k]);
      buf.push_back(r.w[q]);
    }
    VIE_REQUIRE(buf.size() * sizeof(double) == bytes, VIE_EINVAL, "rule size");
    (void)dst;
    VIE_CUDA(cudaMemcpyToSymbol(sym, buf.data(), bytes));
  };
  put(rule_tet4(), 4, nullptr, sizeof(double) * 4 * 5, c_tet4);
  put(rule_tri3(), 3, nullptr, sizeof(double) * 3 * 4, c_tri3);
  put(rule_tet_conical(2), 4, nullptr, sizeof(double) * 8 * 5, c_tetc2);
  put(rule_tet_conical(3), 4, nullptr, sizeof(double) * 27 * 5, c_tetc3);
  put(rule_tri_conical(2), 3, nullptr, sizeof(double) * 4 * 4, c_tric2);
  put(rule_tri_conical(3), 3, nullptr, sizeof(double) * 9 * 4, c_tric3);
  mark_on_device((const void*)&upload_constants);
}

void geometry_upload(const Mesh& m, double k0, Geometry& g, cudaStream_t s) {
  upload_constants();
  g.n = m.nf;
  g.nt = m.nt;
  g.h = m.h;
  g.k0 = k0;
  g.general = m.general;
  std::vector<TetDev> tets(m.nt);
  for (int64_t t = 0; t < m.nt; ++t) {
    const int64_t v = m.general ? t : t / 6;  // row of eps: the voxel, or the tet itself
    TetDev d;
    if (m.general) {
      d.vx = m.cells[3 * t]; d.vy = m.cells[3 * t + 1]; d.vz = m.cells[3 * t + 2];
      d.type = -1;
    } else {
      d.vx = m.vox[3 * v]; d.vy = m.vox[3 * v + 1]; d.vz = m.vox[3 * v + 2];
      d.type = int(t % 6);
    }
    double er = m.eps[2 * v], ei = m.eps[2 * v + 1];
    double den = er * er + ei * ei;
    d.inveps_re = er / den;
    d.inveps_im = -ei / den;
    d.kap_re = 1.0 - d.inveps_re;  // kappa = 1 - 1/eps_r
    d.kap_im = -d.inveps_im;
    tets[t] = d;
  }
  std::vector<FaceDev> faces(m.nf);
  for (int64_t f = 0; f < m.nf; ++f) {
    FaceDev d{};
    d.tp = m.tp[f]; d.tm = m.tm[f];
    d.lp = (int8_t)m.lp[f]; d.lm = (int8_t)(m.tm[f] >= 0 ? m.lm[f] : 0);
    d.boundary = m.tm[f] < 0;
    double kpr = tets[d.tp].kap_re, kpi = tets[d.tp].kap_im;
    double kmr = d.tm >= 0 ? tets[d.tm].kap_re : 0.0, kmi = d.tm >= 0 ? tets[d.tm].kap_im : 0.0;
    d.jump_re = kmr - kpr;
    d.jump_im = kmi - kpi;
    faces[f] = d;
  }
  if (m.general) {  // per-tet geometry records: vertices, volume, face areas and outward normals
    static const int loc[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
    std::vector<TetGeo> geo(m.nt);
    for (int64_t t = 0; t < m.nt; ++t) {
      TetGeo G{};
      const int32_t* T = &m.tets[4 * t];
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) G.P[a][d] = m.xyz[3 * T[a] + d];
      double e[3][3];
      for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) e[a][d] = G.P[a + 1][d] - G.P[0][d];
      const double cx = e[0][1] * e[1][2] - e[0][2] * e[1][1], cy = e[0][2] * e[1][0] - e[0][0] * e[1][2],
                   cz = e[0][0] * e[1][1] - e[0][1] * e[1][0];
      G.vol = std::abs(cx * e[2][0] + cy * e[2][1] + cz * e[2][2]) / 6.0;
      for (int a = 0; a < 4; ++a) {
        const double* A = G.P[loc[a][0]];
        const double* B = G.P[loc[a][1]];
        const double* C = G.P[loc[a][2]];
        const double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double ln = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        const double sg =
            (n[0] * (A[0] - G.P[a][0]) + n[1] * (A[1] - G.P[a][1]) + n[2] * (A[2] - G.P[a][2])) > 0 ? 1.0 : -1.0;
        for (int d = 0; d < 3; ++d) G.nrm[a][d] = sg * n[d] / ln;
        G.area[a] = 0.5 * ln;
        int lv[3] = {loc[a][0], loc[a][1], loc[a][2]};
        std::sort(lv, lv + 3, [&](int x, int y) { return T[x] < T[y]; });
        for (int k = 0; k < 3; ++k) G.fv[a][k] = (int8_t)lv[k];
        G.vid[a] = T[a];
      }
      geo[t] = G;
    }
    g.geo.alloc(sizeof(TetGeo) * m.nt);
    VIE_CUDA(cudaMemcpyAsync(g.geo.p, geo.data(), sizeof(TetGeo) * m.nt, cudaMemcpyHostToDevice, s));
    VIE_CUDA(cudaStreamSynchronize(s));
  }
  g.tets.alloc(sizeof(TetDev) * m.nt);
  g.faces.alloc(sizeof(FaceDev) * m.nf);
  VIE_CUDA(cudaMemcpyAsync(g.tets.p, tets.data(), sizeof(TetDev) * m.nt, cudaMemcpyHostToDevice, s));
  VIE_CUDA(cudaMemcpyAsync(g.faces.p, faces.data(), sizeof(FaceDev) * m.nf, cudaMemcpyHostToDevice, s));
  VIE_CUDA(cudaStreamSynchronize(s));
}

void geometry_table(Geometry& g, cudaStream_t s) {
  g.table.alloc(sizeof(Tab) * 6 * 6 * 125);
  VIE_CUDA(cudaMemsetAsync(g.table.p, 0, g.table.bytes, s));
  table_kernel<<<6 * 6 * 125, 32, 0, s>>>(g.table.as<Tab>(), g.h, g.k0);
  VIE_CUDA(cudaGetLastError());
}

static EntryCtx ctx(const Geometry& g) {
  return EntryCtx{g.faces.as<FaceDev>(), g.tets.as<TetDev>(), g.table.as<Tab>(), g.geo.as<TetGeo>(),
                  g.h,               g.k0,                   g.general ? 1 : 0};
}

void entries_pairs(const Geometry& g, const int32_t* rows, const int32_t* cols, int64_t count, double2* out,
                   cudaStream_t s, bool far32) {
  if (count <= 0) return;
  int grid = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
  if (far32) entries_pairs_kernel<true><<<grid, 256, 0, s>>>(ctx(g), rows, cols, count, out);
  else entries_pairs_kernel<false><<<grid, 256, 0, s>>>(ctx(g), rows, cols, count, out);
  VIE_CUDA(cudaGetLastError());
}

void entries_blocks(const Geometry& g, const EntryBlock* d_blocks, const int64_t* d_prefix, int nblocks,
                    int64_t total, const int32_t* d_rows, const int32_t* d_cols, double2* d_out, cudaStream_t s) {
  if (total <= 0 || nblocks <= 0) return;
  int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
  // the builder evaluates far-tier volume pairs in FP32 (near/mid tables and surface terms stay FP64)
  entries_blocks_kernel<true><<<grid, 256, 0, s>>>(ctx(g), d_blocks, d_prefix, nblocks, total, d_rows, d_cols, d_out);
  VIE_CUDA(cudaGetLastError());
}

void rhs_planewave(const Geometry& g, const double* khat, const double* pol, int nrhs, double2* V, cudaStream_t s) {
  DevBuf dk, dp;
  dk.alloc(sizeof(double) * 3 * nrhs);
  dp.alloc(sizeof(double) * 3 * nrhs);
  VIE_CUDA(cudaMemcpyAsync(dk.p, khat, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, s));
  VIE_CUDA(cudaMemcpyAsync(dp.p, pol, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, s));
  int64_t tot = g.n * nrhs;
  int grid = (int)std::min<int64_t>((tot + 255) / 256, 152 * 16);
  rhs_kernel<<<grid, 256, 0, s>>>(ctx(g), g.n, dk.as<double>(), dp.as<double>(), nrhs, V);
  VIE_CUDA(cudaGetLastError());
  VIE_CUDA(cudaStreamSynchronize(s));
}

}  // namespace vie

// far field needs the tet -> face map; kept with the operator
namespace vie {
void farfield_impl(const Geometry& g, const int32_t* d_tet_faces, const double2* I, int nrhs, const double* dirs,
                   int ndir, double* rcs, cudaStream_t s) {
  DevBuf dd, dF;
  dd.alloc(sizeof(double) * 3 * ndir);
  dF.alloc(sizeof(double2) * 3 * (size_t)ndir * nrhs);
  VIE_CUDA(cudaMemcpyAsync(dd.p, dirs, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, s));
  farfield_kernel<<<ndir * nrhs, 256, 0, s>>>(ctx(g), g.nt, d_tet_faces, I, g.n, dd.as<double>(), dF.as<double2>(),
                                              nrhs);
  VIE_CUDA(cudaGetLastError());
  std::vector<double2> F(3 * (size_t)ndir * nrhs);
  VIE_CUDA(cudaMemcpyAsync(F.data(), dF.p, F.size() * sizeof(double2), cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  const double k0 = g.k0;
  for (int d = 0; d < ndir; ++d)
    for (int r = 0; r < nrhs; ++r) {
      const double2* f = &F[3 * ((size_t)d * nrhs + r)];
      double u[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
      double2 ur = make_double2(u[0] * f[0].x + u[1] * f[1].x + u[2] * f[2].x, u[0] * f[0].y + u[1] * f[1].y + u[2] * f[2].y);
      double s2 = 0;
      for (int k = 0; k < 3; ++k) {
        double re = f[k].x - ur.x * u[k], im = f[k].y - ur.y * u[k];
        s2 += re * re + im * im;
      }
      rcs[(size_t)r * ndir + d] = k0 * k0 * k0 * k0 / (4.0 * kPi) * s2;
    }
}
}  // namespace vie
