// HOD-BF inverse from matrix-vector products only (Sec. III-B, Algorithms 1-2,
// BF_random_matvec), on the GPU.
//
// Algorithm 1 inverts level by level, from the leaves up.  With the inverses of
// the two children of tau known (the inverse program built so far, block
// diagonal over the level below), line 7 recompresses
//   B'_taui = D_taui^-1 B_taui            (products: Z's butterflies of that level, then the inverse so far)
// as a butterfly from products with it and its adjoint, and line 8 computes
//   E_tau = [I, B'_tau1; B'_tau2, I]^-1 - I
// by BF_SMW (Algorithm 2): split into quadrants over the children, invert the
// (2,2) quadrant recursively, recompress the Schur complement from products,
// invert it recursively, and recompress the whole inverse from products with
// its block LDU factors.  Every "recompress from products" is BF_random_matvec,
// built here in the two-sided form of a butterfly (an equivalent form, Sec. III-A):
//   * column side, levels 0 .. h = floor(L/2): Gaussian blocks supported on one
//     row node of level l give the row sketches G^H A(tau, :) of every column at
//     once (products with A^H); the ID of each candidate column set (a column
//     leaf, else the two children's skeletons) gives the V^0 / W^l factors;
//   * row side, steps t = 0 .. L - h: Gaussian blocks supported on one column
//     node of level t give A(:, nu) G (products with A); the ID of the transposed
//     sketch over each candidate row set gives skeleton rows and the
//     interpolation A(cand, nu) ~ U A(I, nu);
//   * middle, at (row level h, column level L - h): M from A(I, nu) G = M (C G),
//     C the column chain, by least squares (Householder QR, FP64).
// The apply of the result is a program like every other: column chain, middle,
// row chain (each output block of a row step sums the two parent blocks of one
// column pair, so every output has one owner), row leaves.
//
// Batching: the nodes of one tree level are independent, so all of them are
// built at once.  Vectors are full length (N rows, tree order, right-hand sides
// fastest); a random block for "row node i" has entries on row node i of every
// node of the level, and the operator's block structure keeps them apart.  All
// products are multi-column applies of programs (tensor cores from 16 columns);
// the least squares run in FP64 (lsq_kernel), the IDs in FP32 arithmetic on FP64 data when
// chi_fact >= 1e-3 (id_batched), FP64 below.
// The recursion bottom (nodes of at most kDenseSmw unknowns, or L <= 2) forms
// the node's block from products with unit vectors and inverts it densely.
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <memory>

#include "internal.h"

namespace vie {

namespace {

#define VIE_CUSOLVER2(call)                                                                     \
  do {                                                                                          \
    cusolverStatus_t st_ = (call);                                                              \
    if (st_ != CUSOLVER_STATUS_SUCCESS) throw Error{VIE_ECUDA, std::string(#call) + " failed"}; \
  } while (0)

constexpr int kDenseSmw = 512;   // BF_SMW recursion bottom: dense inverse of the node block
constexpr int kProdCols = 256;   // right-hand sides per product call (two tensor-core M tiles)

int gridn(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// VIE_INV_TRACE=1 in the environment: one line per butterfly built from products (stderr),
// with a device synchronization after every product so that a failure names its phase.
bool trace() {
  static const bool on = std::getenv("VIE_INV_TRACE") != nullptr;
  return on;
}

// ---------------------------------------------------------------------------
// row-range sets and vector kernels (full-length N x k blocks, k = row stride)
// ---------------------------------------------------------------------------
struct RangeDev {
  int64_t lo, hi, pre;  // rows [lo, hi); pre = rows of the ranges before this one
};

struct Ranges {
  std::vector<RangeDev> r;
  DevBuf d;
  int64_t rows = 0;
  void set(const std::vector<std::pair<int64_t, int64_t>>& v, cudaStream_t s) {
    r.clear();
    rows = 0;
    for (auto& p : v)
      if (p.second > p.first) { r.push_back(RangeDev{p.first, p.second, rows}); rows += p.second - p.first; }
    d.alloc(sizeof(RangeDev) * std::max<size_t>(1, r.size()));
    if (!r.empty()) VIE_CUDA(cudaMemcpyAsync(d.p, r.data(), sizeof(RangeDev) * r.size(), cudaMemcpyHostToDevice, s));
  }
};

__device__ __forceinline__ int64_t range_row(const RangeDev* r, int n, int64_t local) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (r[mid].pre <= local) lo = mid; else hi = mid - 1;
  }
  return r[lo].lo + (local - r[lo].pre);
}

enum { V_ZERO = 0, V_COPY = 1, V_ADD = 2, V_SUB = 3, V_RSUB = 4 };  // y=0, y=x, y+=x, y-=x, y=x-y

__global__ void rows_kernel(int op, float2* y, const float2* x, int k, const RangeDev* r, int n, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = range_row(r, n, e / k);
    const int64_t i = row * k + e % k;
    if (op == V_ZERO) {
      y[i] = make_float2(0.f, 0.f);
      continue;
    }
    float2 v = x[i];
    if (op == V_ADD) { float2 w = y[i]; v = make_float2(w.x + v.x, w.y + v.y); }
    else if (op == V_SUB) { float2 w = y[i]; v = make_float2(w.x - v.x, w.y - v.y); }
    else if (op == V_RSUB) { float2 w = y[i]; v = make_float2(v.x - w.x, v.y - w.y); }
    y[i] = v;
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Complex unit-variance Gaussian entries G[row, col0 + c] for rows in the ranges, c < ncols:
// splitmix64 of (seed, row, hcol0 + c) gives two uniforms, the Box-Muller transform the pair
// (the sample's own column index hcol0 + c, so that a block drawn in pieces is the same block).
__global__ void gauss_rows_kernel(float2* g, int ld, int col0, int hcol0, int ncols, const RangeDev* r, int n,
                                  int64_t total, uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total * ncols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = range_row(r, n, e / ncols);
    const int c = int(e % ncols);
    const uint64_t hsh = mix64(seed ^ mix64((uint64_t)row * 0x100000001B3ull + (uint64_t)(hcol0 + c)));
    const float u1 = ((uint32_t)(hsh >> 40) + 1u) * (1.0f / 16777217.0f);
    const float u2 = (uint32_t)(hsh & 0xFFFFFFu) * (1.0f / 16777216.0f);
    const float rad = sqrtf(-logf(u1));
    float sn, cs;
    sincosf(6.28318530717958647692f * u2, &sn, &cs);
    g[row * ld + col0 + c] = make_float2(rad * cs, rad * sn);
  }
}

// unit vectors: for every range (a node) and c < ncols, G[lo + q0 + c, c] = 1 when inside the node
__global__ void unit_rows_kernel(float2* g, int ld, int q0, int ncols, const RangeDev* r, int n) {
  const RangeDev rg = r[blockIdx.x];
  for (int c = threadIdx.x; c < ncols; c += blockDim.x)
    if (rg.lo + q0 + c < rg.hi) g[(rg.lo + q0 + c) * ld + c] = make_float2(1.f, 0.f);
}

// sketch gather into an FP64 ID pool, one piece of sample rows at a time:
// out[off + row0 + q + c m] = (conj) V[idx[c] * ld + q0 + q] for q < mq, c < n (m x n column-major)
struct GatherJob {
  int64_t out_off, idx_off;
  int32_t n, m, q0, conj, row0, mq;
};

__global__ void sketch_gather_kernel(const GatherJob* jobs, const int32_t* idx, const float2* V, int ld, double2* out) {
  const GatherJob j = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)j.mq * j.n; e += blockDim.x) {
    const int q = int(e % j.mq), c = int(e / j.mq);
    const float2 v = V[(int64_t)idx[j.idx_off + c] * ld + j.q0 + q];
    out[j.out_off + j.row0 + q + (int64_t)c * j.m] = make_double2(v.x, j.conj ? -v.y : v.y);
  }
}

// coefficient gather for the middle level: out[off + row0 + q + c m] = conj(C[(coff + c) * ld + q0 + q])
struct CoefJob {
  int64_t out_off, coff;
  int32_t rows, m, q0, row0, mq, pad;
};

__global__ void coef_gather_kernel(const CoefJob* jobs, const float2* C, int ld, double2* out) {
  const CoefJob j = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)j.mq * j.rows; e += blockDim.x) {
    const int q = int(e % j.mq), c = int(e / j.mq);
    const float2 v = C[(j.coff + c) * ld + j.q0 + q];
    out[j.out_off + j.row0 + q + (int64_t)c * j.m] = make_double2(v.x, -v.y);
  }
}

// [A | B] of one least-squares job: A (m x nc) copied from the column-chain pool, B (m x nr)
// = conj of the sample rows of the chosen skeleton rows, read from a copy of the ID pool
struct AssembleJob {
  int64_t ab_off, cg_off, x_off, piv_off;
  int32_t m, nc, nr, pad;
};

__global__ void lsq_assemble_kernel(const AssembleJob* jobs, const double2* cg, const double2* xs,
                                    const int32_t* piv, double2* ab) {
  const AssembleJob j = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)j.m * (j.nc + j.nr); e += blockDim.x) {
    const int q = int(e % j.m), c = int(e / j.m);
    double2 v;
    if (c < j.nc) v = cg[j.cg_off + e];
    else {
      v = xs[j.x_off + q + (int64_t)piv[j.piv_off + c - j.nc] * j.m];
      v.y = -v.y;
    }
    ab[j.ab_off + e] = v;
  }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zcmul(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Batched least squares min_Z || A Z - B ||_F with [A | B] one m x (nc + nr) column-major
// block (FP64): Householder QR of A (no pivoting) applied to B, back substitution,
// output M = Z^H (nr x nc, row-major).  Directions with |R_kk| <= 1e-12 |R_00| are dropped.
struct LsqJob {
  int64_t ab_off, out_off;
  int32_t m, nc, nr, pad;
};

template <int NT>
__global__ void __launch_bounds__(NT) lsq_kernel(const LsqJob* jobs, double2* pool, double2* out) {
  const LsqJob J = jobs[blockIdx.x];
  const int m = J.m, nc = J.nc, nr = J.nr, nt = nc + nr;
  double2* a = pool + J.ab_off;
  __shared__ double s_nrm, s_vn2;
  __shared__ double2 s_diag[1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT / 32;
  double r00 = 0.0;
  const int kmax = min(m, nc);
  for (int i = 0; i < kmax; ++i) {
    if (warp == 0) {
      double s = 0.0;
      for (int k = i + lane; k < m; k += 32) s += zabs2(a[k + (int64_t)i * m]);
      s = wsum(s);
      if (lane == 0) s_nrm = sqrt(s);
    }
    __syncthreads();
    const double nrm = s_nrm;
    if (i == 0) r00 = nrm;
    if (tid == 0) {
      const double2 x0 = a[i + (int64_t)i * m];
      const double ax0 = sqrt(zabs2(x0));
      const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
      const double2 alpha = make_double2(-ph.x * nrm, -ph.y * nrm);
      s_diag[0] = alpha;
      a[i + (int64_t)i * m] = make_double2(x0.x - alpha.x, x0.y - alpha.y);
      s_vn2 = 2.0 * nrm * nrm + 2.0 * nrm * ax0;
    }
    __syncthreads();
    const double inv = s_vn2 > 0.0 ? 2.0 / s_vn2 : 0.0;
    const double2* v = a + (int64_t)i * m;
    for (int j = i + 1 + warp; j < nt; j += nw) {
      double2* col = a + (int64_t)j * m;
      double wr = 0.0, wi = 0.0;
      for (int k = i + lane; k < m; k += 32) {
        const double2 t = zcmul(v[k], col[k]);
        wr += t.x; wi += t.y;
      }
      wr = wsum(wr);
      wi = wsum(wi);
      const double2 f = make_double2(wr * inv, wi * inv);
      for (int k = i + lane; k < m; k += 32) {
        const double2 t = zmul(v[k], f);
        col[k].x -= t.x;
        col[k].y -= t.y;
      }
    }
    __syncthreads();
    // the reflector is no longer needed: keep R_ii in its place
    if (tid == 0) a[i + (int64_t)i * m] = s_diag[0];
    __syncthreads();
  }
  // back substitution R Z = (Q^H B)(0:nc, :), one thread per right-hand column of B
  for (int c = tid; c < nr; c += NT) {
    double2* b = a + (int64_t)(nc + c) * m;
    for (int k = kmax - 1; k >= 0; --k) {
      double2 t = b[k];
      for (int l = k + 1; l < kmax; ++l) {
        const double2 u = zmul(a[k + (int64_t)l * m], b[l]);
        t.x -= u.x; t.y -= u.y;
      }
      const double2 d = a[k + (int64_t)k * m];
      const double dd = zabs2(d);
      b[k] = (sqrt(dd) > 1e-12 * r00 && dd > 0.0)
                 ? make_double2((t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd)
                 : make_double2(0.0, 0.0);
    }
    // M = Z^H: row c of M is conj(Z(:, c))
    for (int k = 0; k < nc; ++k) {
      const double2 z = k < kmax ? b[k] : make_double2(0.0, 0.0);
      out[J.out_off + (int64_t)c * nc + k] = make_double2(z.x, -z.y);
    }
  }
}

// Row-step factor packing, one column block at a time: dst[m * ld + col0 + c] = V[c][row0 + m]
// for m < M, c < r (V row-major r x ncand): the transposed interpolation matrix U = V^T, rows
// row0 .. row0 + M - 1 of it (one child's rows of the candidate set).
struct RowPackJob {
  int64_t v, dst;
  int32_t r, ncand, row0, M, ld, col0;
};

__global__ void rowpack_kernel(const RowPackJob* jobs, const double2* pool, float2* dst) {
  const RowPackJob j = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)j.M * j.r; e += blockDim.x) {
    const int m = int(e / j.r), c = int(e % j.r);
    const double2 v = pool[j.v + (int64_t)c * j.ncand + j.row0 + m];
    dst[j.dst + (int64_t)m * j.ld + j.col0 + c] = make_float2((float)v.x, (float)v.y);
  }
}

// Generic row-major packing from an FP64 pool: dst (M x K, ld) = src (M x K, row-major, sld)
struct PackJob {
  int64_t src, dst;
  int32_t M, K, sld, ld;
};

__global__ void pack_rm_kernel(const PackJob* jobs, const double2* pool, float2* dst) {
  const PackJob j = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)j.M * j.ld; e += blockDim.x) {
    const int m = int(e / j.ld), c = int(e % j.ld);
    const double2 v = c < j.K ? pool[j.src + (int64_t)m * j.sld + c] : make_double2(0.0, 0.0);
    dst[j.dst + e] = make_float2((float)v.x, (float)v.y);
  }
}

// dense blocks of the recursion bottom: D[b] (n_b x n_b column-major, c64) <- Y[lo_b + r, q] for q < ncols
struct DenseJob {
  int64_t lo, off;
  int32_t n, pad;
};

__global__ void dense_extract_kernel(const DenseJob* jobs, const float2* Y, int ld, int q0, int ncols, float2* D) {
  const DenseJob j = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)j.n * ncols; e += blockDim.x) {
    const int r = int(e % j.n), q = int(e / j.n);
    if (q0 + q < j.n) D[j.off + r + (int64_t)(q0 + q) * j.n] = Y[(j.lo + r) * ld + q];
  }
}

__global__ void add_identity_kernel(float2* D, int64_t n, float sgn) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    D[i + i * n].x += sgn;
}

__global__ void identity_kernel(float2* D, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x)
    D[e] = make_float2((e % n) == (e / n) ? 1.f : 0.f, 0.f);
}

// column-major c64 n x n -> row-major padded (ld = n rounded up to even)
__global__ void cm_to_rm_kernel(const float2* src, int n, int ld, float2* dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * ld; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = int(e / ld), c = int(e % ld);
    dst[e] = c < n ? src[r + (int64_t)c * n] : make_float2(0.f, 0.f);
  }
}

template <class J>
void upload_vec(DevBuf& b, const std::vector<J>& v, cudaStream_t s) {
  b.alloc(sizeof(J) * std::max<size_t>(1, v.size()));
  if (!v.empty()) VIE_CUDA(cudaMemcpyAsync(b.p, v.data(), sizeof(J) * v.size(), cudaMemcpyHostToDevice, s));
}

// ---------------------------------------------------------------------------
// construction context: tree, stream, workspaces, counters
// ---------------------------------------------------------------------------
struct Ctx {
  vie_op* h;
  cudaStream_t s;
  const Tree& t;
  int64_t N;
  int p;          // oversampling of every random block
  double tol;     // chi_fact
  uint64_t seed;
  int64_t products = 0;  // columns multiplied by an operator or its adjoint
  double t_id = 0, t_prod = 0;
  DevBuf coef;
  // reusable N x k vectors
  std::vector<std::unique_ptr<DevBuf>> pool;
  std::vector<bool> busy;

  Ctx(vie_op* hh, cudaStream_t ss, double tl)
      : h(hh), s(ss), t(hh->tree), N(hh->mesh.nf), p(std::max(hh->cfg.oversample, 4)), tol(tl),
        seed(hh->cfg.seed ^ 0xC2B2AE3D27D4EB4Full) {}

  float2* coef_ws(int64_t ncoef, int k) {
    const size_t need = sizeof(float2) * (size_t)std::max<int64_t>(ncoef, 1) * (size_t)k;
    if (coef.bytes < need) coef.alloc(need);
    return coef.as<float2>();
  }
  int64_t node_lo(int lev, int64_t i) const { return t.bounds[lev][i]; }
  int64_t node_hi(int lev, int64_t i) const { return t.bounds[lev][i + 1]; }
};

// A leased N x k vector from the context's pool.
struct Vec {
  Ctx* c = nullptr;
  int slot = -1;
  float2* p = nullptr;
  Vec(Ctx& ctx, int k) : c(&ctx) {
    const size_t need = sizeof(float2) * (size_t)ctx.N * (size_t)k;
    for (size_t i = 0; i < ctx.pool.size(); ++i)
      if (!ctx.busy[i] && ctx.pool[i]->bytes >= need) { slot = (int)i; break; }
    if (slot < 0) {
      for (size_t i = 0; i < ctx.pool.size(); ++i)
        if (!ctx.busy[i]) { slot = (int)i; break; }
      if (slot < 0) {
        ctx.pool.emplace_back(new DevBuf());
        ctx.busy.push_back(false);
        slot = (int)ctx.pool.size() - 1;
      }
      ctx.pool[slot]->alloc(need);
    }
    ctx.busy[slot] = true;
    p = ctx.pool[slot]->as<float2>();
  }
  ~Vec() { if (c && slot >= 0) c->busy[slot] = false; }
  Vec(const Vec&) = delete;
  Vec& operator=(const Vec&) = delete;
};

void rows_op(Ctx& c, int op, float2* y, const float2* x, int k, const Ranges& r) {
  if (r.rows == 0) return;
  rows_kernel<<<gridn(r.rows * k), 256, 0, c.s>>>(op, y, x, k, r.d.as<RangeDev>(), (int)r.r.size(), r.rows);
  VIE_CUDA(cudaGetLastError());
}

Ranges node_ranges(Ctx& c, int lev, const std::vector<int64_t>& nodes) {
  std::vector<std::pair<int64_t, int64_t>> v;
  for (int64_t i : nodes) v.push_back({c.node_lo(lev, i), c.node_hi(lev, i)});
  std::sort(v.begin(), v.end());
  Ranges r;
  r.set(v, c.s);
  return r;
}

// ---------------------------------------------------------------------------
// operators given by products: y(rows) = A x(cols); y(cols) = A^H x(rows)
// ---------------------------------------------------------------------------
struct LinOp {
  virtual ~LinOp() = default;
  virtual void mv(const float2* x, float2* y, int k) = 0;
  virtual void rmv(const float2* x, float2* y, int k) = 0;
};

// A program applied on tree-ordered vectors.  `accumulates`: the program adds into Y
// (zero it first); `inplace`: the program reads Y (its adjoint adds into its input).
struct ProgOp : LinOp {
  Ctx& c;
  Program own, adj;
  Program* fwd = &own;  // the forward program (its own, or one owned elsewhere)
  bool adj_ready = false, accumulates = false, inplace = false;
  bool dense = false;   // one stage of dense node blocks (the recursion bottom)
  const Ranges* rows = nullptr;  // where mv writes (zeroed first when accumulates)
  const Ranges* cols = nullptr;  // where rmv writes
  Ranges own_rows, own_cols;
  explicit ProgOp(Ctx& cc) : c(cc) {}
  void run(Program& p, int64_t ncoef_zero, float2* xt, float2* yt, int k) {
    if (k >= p.tc_min_rhs) program_prepare_tc(p, c.s);
    float2* cf = c.coef_ws(p.ncoef, k);
    if (ncoef_zero) VIE_CUDA(cudaMemsetAsync(cf, 0, sizeof(float2) * (size_t)p.ncoef * k, c.s));
    program_run(p, k, VIE_C64, xt, yt, cf, c.s);
    if (trace()) VIE_CUDA(cudaStreamSynchronize(c.s));
  }
  void mv(const float2* x, float2* y, int k) override {
    if (accumulates) rows_op(c, V_ZERO, y, nullptr, k, *rows);
    run(*fwd, 0, const_cast<float2*>(x), y, k);
    c.products += k;
  }
  void rmv(const float2* x, float2* y, int k) override {
    if (!adj_ready) { program_adjoint(*fwd, adj, c.s); adj_ready = true; }
    rows_op(c, V_ZERO, y, nullptr, k, *cols);
    if (inplace) {  // the adjoint adds into its input: work on a copy
      Vec t(c, k);
      rows_op(c, V_COPY, t.p, x, k, *rows);
      run(adj, 1, y, t.p, k);
    } else {
      run(adj, 1, y, const_cast<float2*>(x), k);
    }
    c.products += k;
  }
};

struct Compose : LinOp {  // A B
  Ctx& c;
  LinOp &a, &b;
  Compose(Ctx& cc, LinOp& aa, LinOp& bb) : c(cc), a(aa), b(bb) {}
  void mv(const float2* x, float2* y, int k) override {
    Vec t(c, k);
    b.mv(x, t.p, k);
    a.mv(t.p, y, k);
  }
  void rmv(const float2* x, float2* y, int k) override {
    Vec t(c, k);
    a.rmv(x, t.p, k);
    b.rmv(t.p, y, k);
  }
};

// ---------------------------------------------------------------------------
// BF_random_matvec: a batch of butterflies A(o_b, s_b), o_b and s_b nodes of level lam
// ---------------------------------------------------------------------------
struct VRef {   // an ID output in a chunk pool: V (r x n, row-major) at off
  int pool = -1;
  int64_t off = 0;
  int32_t r = 0, n = 0;
};

std::unique_ptr<ProgOp> rbf_build(Ctx& c, LinOp& A, int lam, const std::vector<int64_t>& onodes,
                                  const std::vector<int64_t>& snodes, int L, uint64_t seed) {
  const auto tm0 = std::chrono::steady_clock::now();
  const int B = (int)onodes.size();
  const int h = L / 2;
  const int p = c.p;
  std::vector<std::unique_ptr<DevBuf>> pools;  // FP64 V / M pools kept until packing
  auto out = std::make_unique<ProgOp>(c);
  Ranges& orows = out->own_rows;
  Ranges& scols = out->own_cols;
  orows = node_ranges(c, lam, onodes);
  scols = node_ranges(c, lam, snodes);
  out->rows = &orows;
  out->cols = &scols;
  // per level of the column side: V refs and skeletons, index (b * ni + i) * nj + j
  std::vector<std::vector<VRef>> colV(h + 1);
  std::vector<std::vector<int32_t>> cskel;  // current level's skeleton columns (tree positions)

  // run the ID jobs of one chunk; jobs: (pool offset of the m x n sketch, m, n); returns V refs
  auto run_ids = [&](DevBuf& A64, const std::vector<std::pair<int64_t, std::pair<int, int>>>& jobs,
                     std::vector<VRef>& refs, std::vector<std::vector<int32_t>>& piv_out) {
    std::vector<IdJob> ij;
    int64_t voff = 0, poff = 0;
    int maxn = 1;
    for (auto& jb : jobs) {
      const int m = jb.second.first, n = jb.second.second;
      ij.push_back(IdJob{jb.first, voff, poff, m, n, 0.0});
      voff += (int64_t)std::min(m, n) * n;
      poff += n;
      maxn = std::max(maxn, n);
    }
    pools.emplace_back(new DevBuf());
    DevBuf& dV = *pools.back();
    DevBuf dij, dpiv, drank;
    dV.alloc(sizeof(double2) * std::max<int64_t>(1, voff));
    dpiv.alloc(sizeof(int32_t) * std::max<int64_t>(1, poff));
    drank.alloc(sizeof(int32_t) * std::max<size_t>(1, ij.size()));
    upload_vec(dij, ij, c.s);
    const auto t0 = std::chrono::steady_clock::now();
    // FP32 arithmetic when chi_fact >= 1e-3 (the sketches carry BF16x3 products anyway)
    id_batched(dij.as<IdJob>(), (int)ij.size(), maxn, A64.as<double2>(), dV.as<double2>(), dpiv.as<int32_t>(),
               drank.as<int32_t>(), c.tol, c.s, /*single=*/c.tol >= 1e-3);
    std::vector<int32_t> piv(poff), rk(ij.size());
    VIE_CUDA(cudaMemcpyAsync(piv.data(), dpiv.p, sizeof(int32_t) * poff, cudaMemcpyDeviceToHost, c.s));
    VIE_CUDA(cudaMemcpyAsync(rk.data(), drank.p, sizeof(int32_t) * ij.size(), cudaMemcpyDeviceToHost, c.s));
    VIE_CUDA(cudaStreamSynchronize(c.s));
    c.t_id += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    refs.resize(ij.size());
    piv_out.resize(ij.size());
    for (size_t q = 0; q < ij.size(); ++q) {
      refs[q] = VRef{(int)pools.size() - 1, ij[q].v_off, rk[q], ij[q].n};
      piv_out[q].assign(piv.begin() + ij[q].p_off, piv.begin() + ij[q].p_off + rk[q]);
    }
  };

  // ---- column side ----
  for (int l = 0; l <= h; ++l) {
    const int64_t ni = int64_t(1) << l, nj = int64_t(1) << (L - l);
    std::vector<std::vector<int32_t>> cand((size_t)B * ni * nj);
    int kl = 0;
    for (int b = 0; b < B; ++b)
      for (int64_t i = 0; i < ni; ++i)
        for (int64_t j = 0; j < nj; ++j) {
          auto& cd = cand[((size_t)b * ni + i) * nj + j];
          if (l == 0) {
            const int lev = lam + L;
            const int64_t g = snodes[b] * nj + j;
            for (int64_t q = c.node_lo(lev, g); q < c.node_hi(lev, g); ++q) cd.push_back((int32_t)q);
          } else {
            const int64_t pi = i / 2, pnj = nj * 2;
            const auto& s1 = cskel[((size_t)b * (ni / 2) + pi) * pnj + 2 * j];
            const auto& s2 = cskel[((size_t)b * (ni / 2) + pi) * pnj + 2 * j + 1];
            cd.insert(cd.end(), s1.begin(), s1.end());
            cd.insert(cd.end(), s2.begin(), s2.end());
          }
          kl = std::max(kl, (int)cd.size());
        }
    const int k = std::max(kl + p, 16);
    colV[l].resize(cand.size());
    std::vector<std::vector<int32_t>> nskel(cand.size());
    // batches of whole row blocks i (one block when its samples alone exceed a product); the
    // k samples of a block are drawn in pieces of at most kProdCols columns
    const int per = std::max(1, kProdCols / k);
    const int qstep = std::min(k, kProdCols);
    for (int64_t i0 = 0; i0 < ni; i0 += per) {
      const int64_t i1 = std::min<int64_t>(ni, i0 + per);
      std::vector<GatherJob> gj;
      std::vector<int64_t> gi;  // block i of each job
      std::vector<int32_t> idx;
      std::vector<std::pair<int64_t, std::pair<int, int>>> jobs;
      std::vector<size_t> jq;
      int64_t aoff = 0;
      for (int b = 0; b < B; ++b)
        for (int64_t i = i0; i < i1; ++i)
          for (int64_t j = 0; j < nj; ++j) {
            const size_t q = ((size_t)b * ni + i) * nj + j;
            const auto& cd = cand[q];
            if (cd.empty()) continue;
            gj.push_back(GatherJob{aoff, (int64_t)idx.size(), (int32_t)cd.size(), k, 0, 1, 0, 0});
            gi.push_back(i);
            idx.insert(idx.end(), cd.begin(), cd.end());
            jobs.push_back({aoff, {k, (int)cd.size()}});
            jq.push_back(q);
            aoff += (int64_t)k * cd.size();
          }
      if (jobs.empty()) continue;
      DevBuf A64, dgj, didx;
      A64.alloc(sizeof(double2) * aoff);
      upload_vec(didx, idx, c.s);
      for (int q0 = 0; q0 < k; q0 += qstep) {
        const int kq = std::min(qstep, k - q0);
        const int kc = (int)(i1 - i0) * kq;
        Vec G(c, kc), S(c, kc);
        rows_op(c, V_ZERO, G.p, nullptr, kc, orows);
        for (int64_t i = i0; i < i1; ++i) {
          std::vector<std::pair<int64_t, int64_t>> rv;
          for (int b = 0; b < B; ++b) {
            const int64_t g = onodes[b] * ni + i;
            rv.push_back({c.node_lo(lam + l, g), c.node_hi(lam + l, g)});
          }
          Ranges rr;
          rr.set(rv, c.s);
          if (rr.rows)
            gauss_rows_kernel<<<gridn(rr.rows * kq), 256, 0, c.s>>>(
                G.p, kc, (int)(i - i0) * kq, q0, kq, rr.d.as<RangeDev>(), (int)rr.r.size(), rr.rows,
                seed ^ (0xA5A5ull << 32) ^ ((uint64_t)l << 48) ^ (uint64_t)i);
          VIE_CUDA(cudaGetLastError());
          VIE_CUDA(cudaStreamSynchronize(c.s));  // rr is released at the end of this iteration
        }
        A.rmv(G.p, S.p, kc);
        // job (b, i, j): rows q0 .. q0 + kq of its k x |cand| row sketch
        for (size_t u = 0; u < gj.size(); ++u) {
          gj[u].q0 = (int32_t)((gi[u] - i0) * kq);
          gj[u].row0 = q0;
          gj[u].mq = kq;
        }
        upload_vec(dgj, gj, c.s);
        sketch_gather_kernel<<<(int)gj.size(), 256, 0, c.s>>>(dgj.as<GatherJob>(), didx.as<int32_t>(), S.p, kc,
                                                              A64.as<double2>());
        VIE_CUDA(cudaGetLastError());
        VIE_CUDA(cudaStreamSynchronize(c.s));
      }
      std::vector<VRef> refs;
      std::vector<std::vector<int32_t>> piv;
      run_ids(A64, jobs, refs, piv);
      for (size_t u = 0; u < jq.size(); ++u) {
        colV[l][jq[u]] = refs[u];
        auto& sk = nskel[jq[u]];
        for (int32_t pv : piv[u]) sk.push_back(cand[jq[u]][pv]);
      }
    }
    cskel = std::move(nskel);
  }
  // coefficient layout of the column side: level-major, then (b, i, j)
  int64_t ncoef = 0;
  std::vector<std::vector<int64_t>> coff(h + 1);
  for (int l = 0; l <= h; ++l) {
    coff[l].resize(colV[l].size());
    for (size_t q = 0; q < colV[l].size(); ++q) { coff[l][q] = ncoef; ncoef += colV[l][q].r; }
  }
  // column-chain stages (V^0 reads X) -> out->fwd
  Program& P = out->own;
  P.n = c.N;
  P.factor_dtype = VIE_C64;
  // builds one stage from ops whose matrices come from (pool, PackJob) lists
  auto make_stage = [&](std::vector<OpDesc> ops, const std::vector<std::pair<int, PackJob>>& pj,
                        const std::vector<std::pair<int, RowPackJob>>& rj) {
    int64_t total = 0;
    for (auto& o : ops) total = std::max<int64_t>(total, o.mat_off + (int64_t)o.M * o.ld);
    DevBuf mats;
    mats.alloc(sizeof(float2) * std::max<int64_t>(total, 2));
    VIE_CUDA(cudaMemsetAsync(mats.p, 0, sizeof(float2) * std::max<int64_t>(total, 2), c.s));  // padding columns
    // one launch per source pool
    for (size_t pi = 0; pi < pools.size(); ++pi) {
      std::vector<PackJob> a;
      for (auto& x : pj) if (x.first == (int)pi) a.push_back(x.second);
      std::vector<RowPackJob> r;
      for (auto& x : rj) if (x.first == (int)pi) r.push_back(x.second);
      if (!a.empty()) {
        DevBuf d;
        upload_vec(d, a, c.s);
        pack_rm_kernel<<<(int)a.size(), 256, 0, c.s>>>(d.as<PackJob>(), pools[pi]->as<double2>(), mats.as<float2>());
        VIE_CUDA(cudaGetLastError());
        VIE_CUDA(cudaStreamSynchronize(c.s));
      }
      if (!r.empty()) {
        DevBuf d;
        upload_vec(d, r, c.s);
        rowpack_kernel<<<(int)r.size(), 256, 0, c.s>>>(d.as<RowPackJob>(), pools[pi]->as<double2>(), mats.as<float2>());
        VIE_CUDA(cudaGetLastError());
        VIE_CUDA(cudaStreamSynchronize(c.s));
      }
    }
    P.stages.emplace_back();
    stage_set(P.stages.back(), std::move(ops), std::move(mats), total, 8, c.s);
  };
  for (int l = 0; l <= h; ++l) {
    const int64_t ni = int64_t(1) << l, nj = int64_t(1) << (L - l);
    std::vector<OpDesc> ops;
    std::vector<std::pair<int, PackJob>> pj;
    int64_t moff = 0;
    for (int b = 0; b < B; ++b)
      for (int64_t i = 0; i < ni; ++i)
        for (int64_t j = 0; j < nj; ++j) {
          const size_t q = ((size_t)b * ni + i) * nj + j;
          const VRef& v = colV[l][q];
          if (v.r == 0) continue;
          OpDesc o{};
          o.M = v.r;
          o.K = v.n;
          o.ld = (v.n + 1) & ~1;
          o.mat_off = moff;
          o.out_space = SP_C;
          o.out_off = coff[l][q];
          o.accumulate = 0;
          if (l == 0) {
            o.in_space = SP_X;
            o.in_off = c.node_lo(lam + L, snodes[b] * nj + j);
          } else {
            o.in_space = SP_C;
            o.in_off = coff[l - 1][((size_t)b * (ni / 2) + i / 2) * (nj * 2) + 2 * j];
          }
          pj.push_back({v.pool, PackJob{v.off, moff, v.r, v.n, v.n, o.ld}});
          moff += (int64_t)o.M * o.ld;
          moff = (moff + 1) & ~int64_t(1);
          ops.push_back(o);
        }
    make_stage(std::move(ops), pj, {});
  }
  P.ncoef = ncoef;
  // ---- row side: steps t = 0 .. L - h; the middle at the last step ----
  std::vector<std::vector<VRef>> rowV(L - h + 1);
  std::vector<std::vector<int32_t>> rsk;  // (b, i, j) at the current step
  std::vector<std::pair<int, int>> mid_ref;  // (pool, pair index) per middle pair
  std::vector<VRef> midV;   // middle blocks (r_r x r_c) per (b, i, j) at row level h
  for (int t = 0; t <= L - h; ++t) {
    const int64_t ni = int64_t(1) << (L - t), nj = int64_t(1) << t;
    std::vector<std::vector<int32_t>> cand((size_t)B * ni * nj);
    int kl = 0;
    for (int b = 0; b < B; ++b)
      for (int64_t i = 0; i < ni; ++i)
        for (int64_t j = 0; j < nj; ++j) {
          auto& cd = cand[((size_t)b * ni + i) * nj + j];
          if (t == 0) {
            const int lev = lam + L;
            const int64_t g = onodes[b] * ni + i;
            for (int64_t q = c.node_lo(lev, g); q < c.node_hi(lev, g); ++q) cd.push_back((int32_t)q);
          } else {
            const int64_t pnj = nj / 2;
            const auto& s1 = rsk[((size_t)b * (ni * 2) + 2 * i) * pnj + j / 2];
            const auto& s2 = rsk[((size_t)b * (ni * 2) + 2 * i + 1) * pnj + j / 2];
            cd.insert(cd.end(), s1.begin(), s1.end());
            cd.insert(cd.end(), s2.begin(), s2.end());
          }
          kl = std::max(kl, (int)cd.size());
        }
    const bool last = t == L - h;
    int k = std::max(kl + p, 16);
    if (last) {  // the least squares of the middle needs at least r_c + p samples
      int rc = 0;
      for (auto& v : colV[h]) rc = std::max(rc, (int)v.r);
      k = std::max(k, rc + p);
    }
    rowV[t].resize(cand.size());
    std::vector<std::vector<int32_t>> nsk(cand.size());
    if (last) midV.resize((size_t)B * (int64_t(1) << h) * nj);
    const int per = std::max(1, kProdCols / k);
    const int qstep = std::min(k, kProdCols);
    const int64_t nih = int64_t(1) << h;
    for (int64_t j0 = 0; j0 < nj; j0 += per) {
      const int64_t j1 = std::min<int64_t>(nj, j0 + per);
      std::vector<GatherJob> gj;
      std::vector<int64_t> gjj;  // column block j of each job
      std::vector<int32_t> idx;
      std::vector<std::pair<int64_t, std::pair<int, int>>> jobs;
      std::vector<size_t> jq;
      int64_t aoff = 0;
      for (int b = 0; b < B; ++b)
        for (int64_t i = 0; i < ni; ++i)
          for (int64_t j = j0; j < j1; ++j) {
            const size_t q = ((size_t)b * ni + i) * nj + j;
            const auto& cd = cand[q];
            if (cd.empty()) continue;
            gj.push_back(GatherJob{aoff, (int64_t)idx.size(), (int32_t)cd.size(), k, 0, 0, 0, 0});
            gjj.push_back(j);
            idx.insert(idx.end(), cd.begin(), cd.end());
            jobs.push_back({aoff, {k, (int)cd.size()}});
            jq.push_back(q);
            aoff += (int64_t)k * cd.size();
          }
      // middle (last step): the column chain of the same random blocks, C G_j, per pair (b, i, j)
      std::vector<CoefJob> cj;
      std::vector<int64_t> cjj, cgoff;
      std::vector<size_t> cq;
      int64_t cgn = 0;
      if (last)
        for (int b = 0; b < B; ++b)
          for (int64_t i = 0; i < nih; ++i)
            for (int64_t j = j0; j < j1; ++j) {
              const size_t qc = ((size_t)b * nih + i) * nj + j;
              const int rc = colV[h][qc].r;
              if (rc == 0) continue;
              cj.push_back(CoefJob{cgn, coff[h][qc], rc, k, 0, 0, 0, 0});
              cjj.push_back(j);
              cq.push_back(qc);
              cgoff.push_back(cgn);
              cgn += (int64_t)k * rc;
            }
      if (jobs.empty() && cj.empty()) continue;
      DevBuf A64, dgj, didx, CG, dcj;
      A64.alloc(sizeof(double2) * std::max<int64_t>(1, aoff));
      if (cgn) CG.alloc(sizeof(double2) * cgn);
      upload_vec(didx, idx, c.s);
      for (int q0 = 0; q0 < k; q0 += qstep) {
        const int kq = std::min(qstep, k - q0);
        const int kc = (int)(j1 - j0) * kq;
        Vec G(c, kc), X(c, kc);
        rows_op(c, V_ZERO, G.p, nullptr, kc, scols);
        for (int64_t j = j0; j < j1; ++j) {
          std::vector<std::pair<int64_t, int64_t>> rv;
          for (int b = 0; b < B; ++b) {
            const int64_t g = snodes[b] * nj + j;
            rv.push_back({c.node_lo(lam + t, g), c.node_hi(lam + t, g)});
          }
          Ranges rr;
          rr.set(rv, c.s);
          if (rr.rows)
            gauss_rows_kernel<<<gridn(rr.rows * kq), 256, 0, c.s>>>(
                G.p, kc, (int)(j - j0) * kq, q0, kq, rr.d.as<RangeDev>(), (int)rr.r.size(), rr.rows,
                seed ^ (0x5A5Aull << 32) ^ ((uint64_t)t << 48) ^ (uint64_t)j);
          VIE_CUDA(cudaGetLastError());
          VIE_CUDA(cudaStreamSynchronize(c.s));
        }
        A.mv(G.p, X.p, kc);
        if (!gj.empty()) {
          for (size_t u = 0; u < gj.size(); ++u) {
            gj[u].q0 = (int32_t)((gjj[u] - j0) * kq);
            gj[u].row0 = q0;
            gj[u].mq = kq;
          }
          upload_vec(dgj, gj, c.s);
          sketch_gather_kernel<<<(int)gj.size(), 256, 0, c.s>>>(dgj.as<GatherJob>(), didx.as<int32_t>(), X.p, kc,
                                                                A64.as<double2>());
          VIE_CUDA(cudaGetLastError());
        }
        if (!cj.empty()) {  // the column chain only writes C
          Vec dummyY(c, kc);
          if (kc >= P.tc_min_rhs) program_prepare_tc(P, c.s);
          float2* cf = c.coef_ws(P.ncoef, kc);
          program_run(P, kc, VIE_C64, G.p, dummyY.p, cf, c.s);
          for (size_t u = 0; u < cj.size(); ++u) {
            cj[u].q0 = (int32_t)((cjj[u] - j0) * kq);
            cj[u].row0 = q0;
            cj[u].mq = kq;
          }
          upload_vec(dcj, cj, c.s);
          coef_gather_kernel<<<(int)cj.size(), 256, 0, c.s>>>(dcj.as<CoefJob>(), cf, kc, CG.as<double2>());
          VIE_CUDA(cudaGetLastError());
        }
        VIE_CUDA(cudaStreamSynchronize(c.s));
      }
      // the row IDs destroy their pool: keep a copy of the samples for the middle
      DevBuf Xs;
      if (last && !jobs.empty()) {
        Xs.alloc(sizeof(double2) * aoff);
        VIE_CUDA(cudaMemcpyAsync(Xs.p, A64.p, sizeof(double2) * aoff, cudaMemcpyDeviceToDevice, c.s));
      }
      std::vector<VRef> refs;
      std::vector<std::vector<int32_t>> piv;
      std::vector<int64_t> job_of(cand.size(), -1);
      if (!jobs.empty()) {
        run_ids(A64, jobs, refs, piv);
        for (size_t u = 0; u < jq.size(); ++u) {
          rowV[t][jq[u]] = refs[u];
          job_of[jq[u]] = (int64_t)u;
          auto& sk = nsk[jq[u]];
          for (int32_t pv : piv[u]) sk.push_back(cand[jq[u]][pv]);
        }
      }
      if (!last || cj.empty() || jobs.empty()) continue;
      // ---- middle for the pairs (b, i < 2^h, j in this batch): M (C G_j) = X_j(I, :)
      std::vector<AssembleJob> aj;
      std::vector<int32_t> pvs;
      std::vector<LsqJob> lj;
      std::vector<size_t> lq;
      int64_t off2 = 0, moff2 = 0;
      for (size_t u = 0; u < cq.size(); ++u) {
        const size_t qc = cq[u];  // row-side job of the same pair (row level h = L - t)
        const int64_t jb = job_of[qc];
        if (jb < 0 || piv[jb].empty()) continue;
        const int rc = colV[h][qc].r, rr = (int)piv[jb].size();
        aj.push_back(AssembleJob{off2, cgoff[u], jobs[jb].first, (int64_t)pvs.size(), k, rc, rr, 0});
        pvs.insert(pvs.end(), piv[jb].begin(), piv[jb].end());
        lj.push_back(LsqJob{off2, moff2, k, rc, rr, 0});
        lq.push_back(qc);
        off2 += (int64_t)k * (rc + rr);
        moff2 += (int64_t)rr * rc;
      }
      if (lj.empty()) continue;
      DevBuf AB, daj, dpv, dlj;
      pools.emplace_back(new DevBuf());
      DevBuf& Mp = *pools.back();
      AB.alloc(sizeof(double2) * off2);
      Mp.alloc(sizeof(double2) * std::max<int64_t>(1, moff2));
      upload_vec(daj, aj, c.s);
      upload_vec(dpv, pvs, c.s);
      upload_vec(dlj, lj, c.s);
      lsq_assemble_kernel<<<(int)aj.size(), 256, 0, c.s>>>(daj.as<AssembleJob>(), CG.as<double2>(), Xs.as<double2>(),
                                                           dpv.as<int32_t>(), AB.as<double2>());
      VIE_CUDA(cudaGetLastError());
      lsq_kernel<256><<<(int)lj.size(), 256, 0, c.s>>>(dlj.as<LsqJob>(), AB.as<double2>(), Mp.as<double2>());
      VIE_CUDA(cudaGetLastError());
      VIE_CUDA(cudaStreamSynchronize(c.s));
      for (size_t u = 0; u < lq.size(); ++u)
        midV[lq[u]] = VRef{(int)pools.size() - 1, lj[u].out_off, lj[u].nr, lj[u].nc};
    }
    rsk = std::move(nsk);
    if (!last) continue;
  }
  // ---- remaining stages: middle, row chain, row leaves ----
  // row-side coefficient blocks dd[t][(b, i, j)], size = |row skeleton|, t = L - h .. 0
  std::vector<std::vector<int64_t>> doff(L - h + 1);
  for (int t = L - h; t >= 0; --t) {
    doff[t].resize(rowV[t].size());
    for (size_t q = 0; q < rowV[t].size(); ++q) { doff[t][q] = ncoef; ncoef += rowV[t][q].r; }
  }
  {  // middle: cc[h] -> dd[L - h]
    const int64_t nih = int64_t(1) << h, nj = int64_t(1) << (L - h);
    std::vector<OpDesc> ops;
    std::vector<std::pair<int, PackJob>> pj;
    int64_t moff = 0;
    for (int b = 0; b < B; ++b)
      for (int64_t i = 0; i < nih; ++i)
        for (int64_t j = 0; j < nj; ++j) {
          const size_t q = ((size_t)b * nih + i) * nj + j;
          const int rr = rowV[L - h][q].r, rc = colV[h][q].r;
          if (rr == 0) continue;
          OpDesc o{};
          o.M = rr;
          o.K = midV[q].pool >= 0 ? rc : 0;
          o.ld = (o.K + 1) & ~1;
          o.mat_off = moff;
          o.in_space = SP_C;
          o.in_off = coff[h][q];
          o.out_space = SP_C;
          o.out_off = doff[L - h][q];
          o.accumulate = 0;
          if (o.K > 0) pj.push_back({midV[q].pool, PackJob{midV[q].off, moff, rr, rc, rc, o.ld}});
          moff += (int64_t)o.M * o.ld;
          moff = (moff + 1) & ~int64_t(1);
          ops.push_back(o);
        }
    make_stage(std::move(ops), pj, {});
  }
  for (int t = L - h; t >= 1; --t) {  // dd[t] -> dd[t - 1]
    const int64_t ni = int64_t(1) << (L - t), nj = int64_t(1) << t;
    std::vector<OpDesc> ops;
    std::vector<std::pair<int, RowPackJob>> rj;
    int64_t moff = 0;
    for (int b = 0; b < B; ++b)
      for (int64_t i = 0; i < ni; ++i)
        for (int64_t jp = 0; jp < nj / 2; ++jp)
          for (int ch = 0; ch < 2; ++ch) {
            const size_t qa = ((size_t)b * ni + i) * nj + 2 * jp, qb = qa + 1;
            const size_t qo = ((size_t)b * (ni * 2) + 2 * i + ch) * (nj / 2) + jp;
            const int M = rowV[t - 1][qo].r;
            if (M == 0) continue;
            const VRef &va = rowV[t][qa], &vb = rowV[t][qb];
            const int n0 = rowV[t - 1][((size_t)b * (ni * 2) + 2 * i) * (nj / 2) + jp].r;  // rows of child 0
            OpDesc o{};
            o.M = M;
            o.K = va.r + vb.r;
            o.ld = (o.K + 1) & ~1;
            o.mat_off = moff;
            o.in_space = SP_C;
            o.in_off = doff[t][qa];
            o.out_space = SP_C;
            o.out_off = doff[t - 1][qo];
            o.accumulate = 0;
            if (o.K > 0) {
              // [U(i, 2j')(child rows), U(i, 2j'+1)(child rows)]; the two parts may sit in different pools
              if (va.r) rj.push_back({va.pool, RowPackJob{va.off, moff, va.r, va.n, ch ? n0 : 0, M, o.ld, 0}});
              if (vb.r) rj.push_back({vb.pool, RowPackJob{vb.off, moff, vb.r, vb.n, ch ? n0 : 0, M, o.ld, va.r}});
            }
            moff += (int64_t)o.M * o.ld;
            moff = (moff + 1) & ~int64_t(1);
            ops.push_back(o);
          }
    make_stage(std::move(ops), {}, rj);
  }
  {  // row leaves: y(leaf) = U0 dd[0]
    const int64_t ni = int64_t(1) << L;
    std::vector<OpDesc> ops;
    std::vector<std::pair<int, RowPackJob>> rj;
    int64_t moff = 0;
    for (int b = 0; b < B; ++b)
      for (int64_t i = 0; i < ni; ++i) {
        const size_t q = (size_t)b * ni + i;
        const int64_t g = onodes[b] * ni + i;
        const int M = (int)(c.node_hi(lam + L, g) - c.node_lo(lam + L, g));
        if (M == 0) continue;
        const VRef& v = rowV[0][q];
        OpDesc o{};
        o.M = M;
        o.K = v.r;
        o.ld = (o.K + 1) & ~1;
        o.mat_off = moff;
        o.in_space = SP_C;
        o.in_off = doff[0][q];
        o.out_space = SP_Y;
        o.out_off = c.node_lo(lam + L, g);
        o.accumulate = 0;
        if (v.r) rj.push_back({v.pool, RowPackJob{v.off, moff, v.r, v.n, 0, M, o.ld, 0}});
        moff += (int64_t)o.M * o.ld;
        moff = (moff + 1) & ~int64_t(1);
        ops.push_back(o);
      }
    make_stage(std::move(ops), {}, rj);
  }
  P.ncoef = ncoef;
  program_totals(P);
  program_check(P);
  program_compact_coef(P, c.s);
  VIE_REQUIRE(program_finite(P, c.s), VIE_ENAN,
              "non-finite factor in a butterfly built from products (the inverse construction diverged)");
  P.tc_ready = false;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - tm0).count();
  c.t_prod += secs;
  if (trace())
    std::fprintf(stderr,
                 "[inverse] butterfly level %d, %d blocks, L %d: %lld entries, %lld coefficients, %.2f s "
                 "(IDs %.2f s so far), %lld products so far\n",
                 lam, B, L, (long long)P.entries, (long long)P.ncoef, secs, c.t_id, (long long)c.products);
  return out;
}

// ---------------------------------------------------------------------------
// dense inverse at the recursion bottom: E_b = (I + M_b)^-1 - I, M_b = (A - I) over node b
// ---------------------------------------------------------------------------
std::unique_ptr<ProgOp> dense_smw(Ctx& c, LinOp& A, int lam, const std::vector<int64_t>& nodes, const Ranges& rg) {
  std::vector<DenseJob> dj;
  int nmax = 0;
  int64_t off = 0;
  for (int64_t nd : nodes) {
    const int n = (int)(c.node_hi(lam, nd) - c.node_lo(lam, nd));
    dj.push_back(DenseJob{c.node_lo(lam, nd), off, n, 0});
    off += (int64_t)n * n;
    nmax = std::max(nmax, n);
  }
  DevBuf D, djb;
  D.alloc(sizeof(float2) * std::max<int64_t>(1, off));
  upload_vec(djb, dj, c.s);
  for (int q0 = 0; q0 < nmax; q0 += kProdCols) {
    const int kc = std::min(kProdCols, nmax - q0);
    const int k = std::max(kc, 16);
    Vec G(c, k), Y(c, k);
    rows_op(c, V_ZERO, G.p, nullptr, k, rg);
    if (!rg.r.empty())
      unit_rows_kernel<<<(int)rg.r.size(), 128, 0, c.s>>>(G.p, k, q0, kc, rg.d.as<RangeDev>(), (int)rg.r.size());
    VIE_CUDA(cudaGetLastError());
    A.mv(G.p, Y.p, k);
    dense_extract_kernel<<<(int)dj.size(), 256, 0, c.s>>>(djb.as<DenseJob>(), Y.p, k, q0, kc, D.as<float2>());
    VIE_CUDA(cudaGetLastError());
    VIE_CUDA(cudaStreamSynchronize(c.s));
  }
  cusolverDnHandle_t sol = nullptr;
  VIE_CUSOLVER2(cusolverDnCreate(&sol));
  struct H { cusolverDnHandle_t s; ~H() { if (s) cusolverDnDestroy(s); } } hd{sol};
  VIE_CUSOLVER2(cusolverDnSetStream(sol, c.s));
  auto out = std::make_unique<ProgOp>(c);
  out->dense = true;
  out->own_rows = node_ranges(c, lam, nodes);
  out->own_cols = node_ranges(c, lam, nodes);
  out->rows = &out->own_rows;
  out->cols = &out->own_cols;
  std::vector<OpDesc> ops;
  int64_t total = 0;
  for (auto& j : dj) total += (int64_t)j.n * ((j.n + 1) & ~1);
  DevBuf mats;
  mats.alloc(sizeof(float2) * std::max<int64_t>(2, total));
  int64_t moff = 0;
  for (auto& j : dj) {
    const int n = j.n;
    if (n == 0) continue;
    float2* Mb = D.as<float2>() + j.off;
    add_identity_kernel<<<gridn(n), 256, 0, c.s>>>(Mb, n, 1.f);  // I + M
    DevBuf inv, work, ipiv, info;
    inv.alloc(sizeof(float2) * (size_t)n * n);
    int lwork = 0;
    VIE_CUSOLVER2(cusolverDnCgetrf_bufferSize(sol, n, n, (cuComplex*)Mb, n, &lwork));
    work.alloc(sizeof(cuComplex) * std::max(lwork, 1));
    ipiv.alloc(sizeof(int) * n);
    info.alloc(sizeof(int));
    VIE_CUSOLVER2(cusolverDnCgetrf(sol, n, n, (cuComplex*)Mb, n, work.as<cuComplex>(), ipiv.as<int>(), info.as<int>()));
    identity_kernel<<<gridn((int64_t)n * n), 256, 0, c.s>>>(inv.as<float2>(), n);
    VIE_CUSOLVER2(cusolverDnCgetrs(sol, CUBLAS_OP_N, n, n, (const cuComplex*)Mb, n, ipiv.as<int>(),
                                   (cuComplex*)inv.p, n, info.as<int>()));
    int hinfo = 0;
    VIE_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, c.s));
    VIE_CUDA(cudaStreamSynchronize(c.s));
    VIE_REQUIRE(hinfo == 0, VIE_ENAN, "singular block at the bottom of the inverse recursion");
    add_identity_kernel<<<gridn(n), 256, 0, c.s>>>(inv.as<float2>(), n, -1.f);  // (I + M)^-1 - I
    const int ld = (n + 1) & ~1;
    cm_to_rm_kernel<<<gridn((int64_t)n * ld), 256, 0, c.s>>>(inv.as<float2>(), n, ld, mats.as<float2>() + moff);
    VIE_CUDA(cudaGetLastError());
    VIE_CUDA(cudaStreamSynchronize(c.s));
    OpDesc o{};
    o.M = n;
    o.K = n;
    o.ld = ld;
    o.mat_off = moff;
    o.in_space = SP_X;
    o.in_off = j.lo;
    o.out_space = SP_Y;
    o.out_off = j.lo;
    o.accumulate = 0;
    ops.push_back(o);
    moff += (int64_t)n * ld;
  }
  Program& P = out->own;
  P.n = c.N;
  P.factor_dtype = VIE_C64;
  P.ncoef = 0;
  P.stages.emplace_back();
  stage_set(P.stages.back(), std::move(ops), std::move(mats), moff, 8, c.s);
  program_totals(P);
  program_check(P);
  VIE_REQUIRE(program_finite(P, c.s), VIE_ENAN, "non-finite dense block at the bottom of the inverse recursion");
  return out;
}

// ---------------------------------------------------------------------------
// BF_SMW (Algorithm 2): E = A^-1 - I over the nodes of level lam, from products with A - I
// ---------------------------------------------------------------------------
std::unique_ptr<ProgOp> bf_smw(Ctx& c, LinOp& A, int lam, const std::vector<int64_t>& nodes, int L, bool zero_diag,
                               uint64_t seed) {
  Ranges rg = node_ranges(c, lam, nodes);
  int nmax = 0;
  for (int64_t nd : nodes) nmax = std::max<int>(nmax, (int)(c.node_hi(lam, nd) - c.node_lo(lam, nd)));
  if (L <= 2 || nmax <= kDenseSmw || lam + 1 > c.t.levels) return dense_smw(c, A, lam, nodes, rg);
  std::vector<int64_t> n1, n2;
  for (int64_t nd : nodes) { n1.push_back(2 * nd); n2.push_back(2 * nd + 1); }
  Ranges r1 = node_ranges(c, lam + 1, n1), r2 = node_ranges(c, lam + 1, n2);
  // (2,2) quadrant and its inverse (zero when A - I has no diagonal quadrants)
  struct Quad : LinOp {
    Ctx& c; LinOp& A; const Ranges &all, &in, &outr;
    Quad(Ctx& cc, LinOp& a, const Ranges& al, const Ranges& i, const Ranges& o) : c(cc), A(a), all(al), in(i), outr(o) {}
    void mv(const float2* x, float2* y, int k) override {
      Vec xa(c, k), t(c, k);
      rows_op(c, V_ZERO, xa.p, nullptr, k, all);
      rows_op(c, V_COPY, xa.p, x, k, in);
      A.mv(xa.p, t.p, k);
      rows_op(c, V_COPY, y, t.p, k, outr);
    }
    void rmv(const float2* x, float2* y, int k) override {
      Vec xa(c, k), t(c, k);
      rows_op(c, V_ZERO, xa.p, nullptr, k, all);
      rows_op(c, V_COPY, xa.p, x, k, outr);
      A.rmv(xa.p, t.p, k);
      rows_op(c, V_COPY, y, t.p, k, in);
    }
  };
  std::unique_ptr<ProgOp> R22;
  if (!zero_diag) {
    Quad A22(c, A, rg, r2, r2);
    R22 = bf_smw(c, A22, lam + 1, n2, L - 2, false, seed * 31 + 1);
  }
  // y2 <- y2 + R22 y2 (or its adjoint) on the second children
  auto inv22 = [&](float2* v, int k, bool adjoint) {
    if (!R22) return;
    Vec w(c, k);
    if (adjoint) R22->rmv(v, w.p, k); else R22->mv(v, w.p, k);
    rows_op(c, V_ADD, v, w.p, k, r2);
  };
  // Schur complement S - I = A11 - A12 (I + R22) A21 (- I) on the first children
  struct Schur : LinOp {
    Ctx& c; LinOp& A; const Ranges &all, &r1, &r2;
    std::function<void(float2*, int, bool)> inv22;
    Schur(Ctx& cc, LinOp& a, const Ranges& al, const Ranges& x1, const Ranges& x2, std::function<void(float2*, int, bool)> f)
        : c(cc), A(a), all(al), r1(x1), r2(x2), inv22(std::move(f)) {}
    void apply(const float2* x, float2* y, int k, bool adj) {
      Vec xa(c, k), t(c, k), ub(c, k), v(c, k);
      rows_op(c, V_ZERO, xa.p, nullptr, k, all);
      rows_op(c, V_COPY, xa.p, x, k, r1);
      if (adj) A.rmv(xa.p, t.p, k); else A.mv(xa.p, t.p, k);      // t1 = A11 x1, t2 = A21 x1 (adjoint: A11^H, A12^H)
      rows_op(c, V_ZERO, ub.p, nullptr, k, all);
      rows_op(c, V_COPY, ub.p, t.p, k, r2);
      inv22(ub.p, k, adj);
      if (adj) A.rmv(ub.p, v.p, k); else A.mv(ub.p, v.p, k);      // v1 = A12 u2 (adjoint: A21^H u2)
      rows_op(c, V_COPY, y, t.p, k, r1);
      rows_op(c, V_SUB, y, v.p, k, r1);
    }
    void mv(const float2* x, float2* y, int k) override { apply(x, y, k, false); }
    void rmv(const float2* x, float2* y, int k) override { apply(x, y, k, true); }
  };
  Schur S(c, A, rg, r1, r2, inv22);
  std::unique_ptr<ProgOp> Sb = rbf_build(c, S, lam + 1, n1, n1, L - 2, seed * 31 + 2);
  std::unique_ptr<ProgOp> R11 = bf_smw(c, *Sb, lam + 1, n1, L - 2, false, seed * 31 + 3);
  Sb.reset();
  // A^-1 - I through the block LDU factors
  struct Full : LinOp {
    Ctx& c; LinOp& A; ProgOp& R11; const Ranges &all, &r1, &r2;
    std::function<void(float2*, int, bool)> inv22;
    Full(Ctx& cc, LinOp& a, ProgOp& r, const Ranges& al, const Ranges& x1, const Ranges& x2,
         std::function<void(float2*, int, bool)> f)
        : c(cc), A(a), R11(r), all(al), r1(x1), r2(x2), inv22(std::move(f)) {}
    // forward:  i2 = inv22 x2; u1 = x1 - A12 i2; v1 = (I + R11) u1; w2 = i2 - inv22 A21 v1
    // adjoint:  j2 = inv22^H y2; a1 = y1 - A21^H j2; b1 = (I + R11)^H a1; c2 = j2 - inv22^H A12^H b1
    void apply(const float2* x, float2* y, int k, bool adj) {
      Vec i2(c, k), t(c, k), u1(c, k), w(c, k);
      rows_op(c, V_ZERO, i2.p, nullptr, k, all);
      rows_op(c, V_COPY, i2.p, x, k, r2);
      inv22(i2.p, k, adj);
      if (adj) A.rmv(i2.p, t.p, k); else A.mv(i2.p, t.p, k);      // t1 = A12 i2 (adjoint: A21^H j2)
      rows_op(c, V_COPY, u1.p, x, k, r1);
      rows_op(c, V_SUB, u1.p, t.p, k, r1);
      {
        Vec q(c, k);
        if (adj) R11.rmv(u1.p, q.p, k); else R11.mv(u1.p, q.p, k);
        rows_op(c, V_ADD, u1.p, q.p, k, r1);                      // u1 <- v1
      }
      rows_op(c, V_ZERO, t.p, nullptr, k, all);
      rows_op(c, V_COPY, t.p, u1.p, k, r1);
      if (adj) A.rmv(t.p, w.p, k); else A.mv(t.p, w.p, k);        // w2 = A21 v1 (adjoint: A12^H b1)
      rows_op(c, V_ZERO, t.p, nullptr, k, all);
      rows_op(c, V_COPY, t.p, w.p, k, r2);
      inv22(t.p, k, adj);
      rows_op(c, V_SUB, i2.p, t.p, k, r2);                        // i2 <- w2
      rows_op(c, V_COPY, y, u1.p, k, r1);
      rows_op(c, V_SUB, y, x, k, r1);
      rows_op(c, V_COPY, y, i2.p, k, r2);
      rows_op(c, V_SUB, y, x, k, r2);
    }
    void mv(const float2* x, float2* y, int k) override { apply(x, y, k, false); }
    void rmv(const float2* x, float2* y, int k) override { apply(x, y, k, true); }
  };
  Full F(c, A, *R11, rg, r1, r2, inv22);
  return rbf_build(c, F, lam, nodes, nodes, L, seed * 31 + 4);
}

}  // namespace

// Algorithm 1 from products, for the levels l = l_top .. 0 whose diagonal blocks are
// not formed densely; h->zinv holds the inverse of every level below l_top already.
void build_inverse_products(vie_op* h, int l_top, double tol, cudaStream_t s, InverseProductStats& st) {
  if (l_top < 0) return;
  VIE_REQUIRE(h->cfg.factor_dtype == VIE_C64, VIE_ENOTSUP, "the product-built inverse needs complex FP32 factors");
  Trace tr("vie:build/Zinv/products");
  Ctx c(h, s, tol);
  const int LH = c.t.levels;
  const auto t0 = std::chrono::steady_clock::now();
  Program& Zinv = h->zinv;
  // the inverse built so far as an operator, with its adjoint kept up to date as levels are added
  Ranges all;
  all.set({{0, c.N}}, s);
  ProgOp Zi(c);
  Zi.fwd = &Zinv;
  Zi.rows = Zi.cols = &all;
  Zi.inplace = true;
  program_adjoint(Zinv, Zi.adj, s);
  Zi.adj_ready = true;
  for (int l = l_top; l >= 0; --l) {
    const int L = LH - l;
    // Z's butterflies between the two children of every node of level l
    ProgOp Zoff(c);
    program_filter(h->z, l + 1, Zoff.own, s);
    Zoff.rows = Zoff.cols = &all;
    Zoff.accumulates = true;
    Compose F(c, Zi, Zoff);  // [0, B'1; B'2, 0] = diag(D_tau1^-1, D_tau2^-1) [0, B1; B2, 0]
    std::vector<int64_t> ch, sib, nodes;
    for (int64_t i = 0; i < (int64_t(1) << (l + 1)); ++i) { ch.push_back(i); sib.push_back(i ^ 1); }
    for (int64_t i = 0; i < (int64_t(1) << l); ++i) nodes.push_back(i);
    // Algorithm 1, line 7: B'_taui recompressed from products with it and its adjoint
    std::unique_ptr<ProgOp> Bp = rbf_build(c, F, l + 1, ch, sib, L - 1, c.seed ^ (0x1000ull * (l + 1)));
    Zoff.own.stages.clear();
    Zoff.adj.stages.clear();
    // line 8: E_tau = BF_SMW([I, B'1; B'2, I]) - I from products with the recompressed B'
    std::unique_ptr<ProgOp> E = bf_smw(c, *Bp, l, nodes, L, /*zero_diag=*/true, c.seed ^ (0x2000ull * (l + 1)));
    Bp.reset();
    if (E->dense)  // a dense node block cannot update y in place in one stage: recompress it as a butterfly
      E = rbf_build(c, *E, l, nodes, nodes, L, c.seed ^ (0x3000ull * (l + 1)));
    // in-place form for the inverse program: y_tau <- y_tau + E_tau y_tau
    Program& Ep = E->own;
    for (OpDesc& o : Ep.stages.front().host_ops)
      if (o.in_space == SP_X) o.in_space = SP_Y;
    for (OpDesc& o : Ep.stages.back().host_ops)
      if (o.out_space == SP_Y) o.accumulate = 1;
    for (Stage* stp : {&Ep.stages.front(), &Ep.stages.back()})
      VIE_CUDA(cudaMemcpyAsync(stp->ops.p, stp->host_ops.data(), sizeof(OpDesc) * stp->host_ops.size(),
                               cudaMemcpyHostToDevice, s));
    program_relocate_coef(Ep, Zinv.ncoef, s);  // drops any tensor-core preparation; ncoef = base + own
    for (Stage& x : Ep.stages) Zinv.stages.push_back(std::move(x));
    Zinv.ncoef = Ep.ncoef;
    Ep.stages.clear();
    E.reset();
    program_totals(Zinv);
    program_compact_coef(Zinv, s);  // the levels run one after another: their coefficients share memory
    if (l > 0) {  // the adjoint of the grown inverse, for the next level's products
      Zi.adj.stages.clear();
      program_adjoint(Zinv, Zi.adj, s);
    }
    program_check(Zinv);
    c.pool.clear();  // work vectors and coefficients are sized per level
    c.busy.clear();
    c.coef.release();
    ++st.levels;
  }
  st.products = c.products;
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  st.id_seconds = c.t_id;
}

}  // namespace vie
