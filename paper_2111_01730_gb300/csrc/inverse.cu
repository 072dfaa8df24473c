// HOD-BF approximate inverse Zinv (Sec. III-B, Algorithm 1), built on the GPU.
//
// Algorithm 1 writes the inverse of every diagonal block recursively as
//   D_tau^-1 = (I + E_tau) diag(D_tau1^-1, D_tau2^-1),
//   E_tau    = [I, B'_tau1; B'_tau2, I]^-1 - I,   B'_taui = D_taui^-1 B_taui,
// and compresses each E_tau (a tau x tau block) as a butterfly at chi_fact.
// Applying Zinv is then: y = D_leaf^-1 x on the leaves, followed, level by
// level from the leaves to the root, by y_tau <- y_tau + E_tau y_tau.
//
// Construction here: for each node tau, E_tau is formed densely in complex
// FP32 from its plain definition, E_tau = D_tau^-1 diag(D_tau1, D_tau2) - I
// (the same matrix as above), with D_tau = Z(tau, tau) from the entry
// evaluator: an LU factorization of D_tau and a two-sided triangular solve
// with diag(D_tau1, D_tau2) as right-hand sides (two n x n matrices per node).
// It is then compressed by the same level-by-level ID construction as Z
// (Eqs. 7-10), except that each ID reads a Gaussian row sketch G^H E_tau(tau', :)
// of its row node tau' (products of E_tau^H with random vectors supported on
// tau', as the randomized construction of Sec. III-B does) instead of sampled
// rows; the B^L blocks read exact entries.  This replaces the randomized
// recompression from black-box products (BF_random_matvec inside BF_SMW,
// Algorithm 2) and
// is limited by the dense blocks: a level joins the inverse when its largest
// node fits twice in the free device memory and holds at most
// kDenseInverseLimit unknowns; above the first level that does not, the
// inverse is block diagonal.  Nodes of a level are compressed in batches
// whose dense E_tau fit in memory together.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <chrono>
#include <map>
#include <tuple>

#include "internal.h"

namespace vie {

#define VIE_CUBLAS(call)                                                                      \
  do {                                                                                        \
    cublasStatus_t st_ = (call);                                                              \
    if (st_ != CUBLAS_STATUS_SUCCESS) throw Error{VIE_ECUDA, std::string(#call) + " failed"}; \
  } while (0)
#define VIE_CUSOLVER(call)                                                                      \
  do {                                                                                          \
    cusolverStatus_t st_ = (call);                                                              \
    if (st_ != CUSOLVER_STATUS_SUCCESS) throw Error{VIE_ECUDA, std::string(#call) + " failed"}; \
  } while (0)

namespace {

__global__ void c128_to_c64(const double2* a, float2* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void set_identity(float2* a, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x)
    a[e] = make_float2((e % n) == (e / n) ? 1.f : 0.f, 0.f);
}

__global__ void sub_identity(float2* a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i + i * n].x -= 1.f;
}

struct DenseRef {
  const float2* p;
  int64_t base;  // tree position of row/column 0
  int64_t ld;
};

// out[block] (c128 col-major) = M_src[rows - base, cols - base]
__global__ void gather_dense(const DenseRef* mats, const EntryBlock* blocks, const int64_t* prefix, const int32_t* src,
                             int nblocks, int64_t total, const int32_t* rows, const int32_t* cols, double2* out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nblocks - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const EntryBlock b = blocks[lo];
    const DenseRef M = mats[src[lo]];
    int64_t k = g - prefix[lo];
    int i = int(k % b.m), j = int(k / b.m);
    float2 v = M.p[(rows[b.row_off + i] - M.base) + (cols[b.col_off + j] - M.base) * M.ld];
    out[b.out_off + k] = make_double2(v.x, v.y);
  }
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

// Complex Gaussian entries (unit variance) from a counter-based hash: splitmix64 of
// (seed, index) gives two uniforms, the Box-Muller transform two normals.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gaussian_fill(float2* g, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64(seed ^ mix64((uint64_t)i));
    const float u1 = ((uint32_t)(h >> 40) + 1u) * (1.0f / 16777217.0f);  // (0, 1]
    const float u2 = (uint32_t)(h & 0xFFFFFFu) * (1.0f / 16777216.0f);
    const float r = sqrtf(-logf(u1));  // |z|^2 / 2 of a unit complex normal
    float sn, cs;
    sincosf(6.28318530717958647692f * u2, &sn, &cs);
    g[i] = make_float2(r * cs, r * sn);
  }
}

struct SketchJob {
  int64_t out_off, col_off;  // block output offset, first column in the column pool
  int32_t m, n;              // sketch rows used, columns
  int64_t s_off;             // the group's sketch S (K x ld, column-major)
  int32_t K, pad;
  int64_t base;              // tree position of column 0 of S
};

// dA[out_off + i + c m] = S[i + (col_c - base) K] for every sketched ID job
__global__ void sketch_gather(const SketchJob* jobs, int nj, const int32_t* cols, const float2* S, double2* dA) {
  const SketchJob j = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < (int64_t)j.m * j.n; e += blockDim.x) {
    const int i = int(e % j.m), c = int(e / j.m);
    const float2 v = S[j.s_off + i + (int64_t)(cols[j.col_off + c] - j.base) * j.K];
    dA[j.out_off + e] = make_double2(v.x, v.y);
  }
}

struct DenseSource : EntrySource {
  std::vector<DenseRef> refs;
  std::vector<int64_t> lo, hi;  // row node of each ID job of the next eval
  bool sketch = false;          // ID jobs read G^H E(tau, :) instead of sampled rows of E
  uint64_t seed = 1;
  cublasHandle_t blas = nullptr;
  ~DenseSource() override { if (blas) cublasDestroy(blas); }
  void set_row_ranges(const std::vector<int64_t>& l, const std::vector<int64_t>& h) override { lo = l; hi = h; }
  void eval(const std::vector<EntryBlock>& eb, const std::vector<int64_t>& prefix, const std::vector<int32_t>& rows,
            const std::vector<int32_t>& cols, const std::vector<int32_t>& srcs, int64_t total, double2* dA,
            cudaStream_t s) override {
    const int nj = (int)eb.size();
    DevBuf dref, deb, dpre, dsrc, drows, dcols;
    dref.alloc(sizeof(DenseRef) * refs.size());
    deb.alloc(sizeof(EntryBlock) * nj);
    dpre.alloc(sizeof(int64_t) * nj);
    dsrc.alloc(sizeof(int32_t) * nj);
    drows.alloc(sizeof(int32_t) * std::max<size_t>(1, rows.size()));
    dcols.alloc(sizeof(int32_t) * std::max<size_t>(1, cols.size()));
    VIE_CUDA(cudaMemcpyAsync(dref.p, refs.data(), sizeof(DenseRef) * refs.size(), cudaMemcpyHostToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(deb.p, eb.data(), sizeof(EntryBlock) * nj, cudaMemcpyHostToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(dpre.p, prefix.data(), sizeof(int64_t) * nj, cudaMemcpyHostToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(dsrc.p, srcs.data(), sizeof(int32_t) * nj, cudaMemcpyHostToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(drows.p, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(dcols.p, cols.data(), sizeof(int32_t) * cols.size(), cudaMemcpyHostToDevice, s));
    if (total > 0)
      gather_dense<<<grid_for(total), 256, 0, s>>>(dref.as<DenseRef>(), deb.as<EntryBlock>(), dpre.as<int64_t>(),
                                                   dsrc.as<int32_t>(), nj, total, drows.as<int32_t>(),
                                                   dcols.as<int32_t>(), dA);
    VIE_CUDA(cudaGetLastError());
    if (sketch) sketch_jobs(eb, cols, srcs, dA, s);
    VIE_CUDA(cudaStreamSynchronize(s));
  }

  // ID jobs whose rows are a sample of their row node tau get, in place of those m rows,
  // the first m rows of S = G^H E(tau, :), G a complex Gaussian |tau| x K block (K the
  // largest m of the jobs sharing tau): products of E^H with random vectors supported on
  // tau, the row sketch the randomized construction uses (Sec. III-B).
  void sketch_jobs(const std::vector<EntryBlock>& eb, const std::vector<int32_t>& cols,
                   const std::vector<int32_t>& srcs, double2* dA, cudaStream_t s) {
    if (lo.size() != eb.size()) return;
    std::map<std::tuple<int32_t, int64_t, int64_t>, std::vector<int>> groups;
    for (int q = 0; q < (int)eb.size(); ++q)
      if (lo[q] >= 0 && eb[q].m < hi[q] - lo[q]) groups[{srcs[q], lo[q], hi[q]}].push_back(q);
    if (groups.empty()) return;
    if (!blas) VIE_CUBLAS(cublasCreate(&blas));
    VIE_CUBLAS(cublasSetStream(blas, s));
    DevBuf dcols;
    dcols.alloc(sizeof(int32_t) * std::max<size_t>(1, cols.size()));
    VIE_CUDA(cudaMemcpyAsync(dcols.p, cols.data(), sizeof(int32_t) * cols.size(), cudaMemcpyHostToDevice, s));
    for (auto& kv : groups) {
      const DenseRef& R = refs[std::get<0>(kv.first)];
      const int64_t a = std::get<1>(kv.first), b = std::get<2>(kv.first), rows = b - a, n = R.ld;
      int K = 0;
      for (int q : kv.second) K = std::max(K, eb[q].m);
      DevBuf G, S, dj;
      G.alloc(sizeof(float2) * rows * K);
      S.alloc(sizeof(float2) * (int64_t)K * n);
      const uint64_t gseed = seed ^ ((uint64_t)std::get<0>(kv.first) << 48) ^ ((uint64_t)a << 24) ^ (uint64_t)b;
      gaussian_fill<<<grid_for(rows * K), 256, 0, s>>>(G.as<float2>(), rows * K, gseed);
      VIE_CUDA(cudaGetLastError());
      const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f);
      // S (K x n) = G^H (K x rows) E(a:b, :) (rows x n); E column-major with ld = n
      VIE_CUBLAS(cublasCgemm(blas, CUBLAS_OP_C, CUBLAS_OP_N, K, (int)n, (int)rows, &one, (const cuComplex*)G.p,
                             (int)rows, (const cuComplex*)(R.p + (a - R.base)), (int)n, &zero, (cuComplex*)S.p, K));
      std::vector<SketchJob> js;
      for (int q : kv.second)
        js.push_back(SketchJob{eb[q].out_off, eb[q].col_off, eb[q].m, eb[q].n, 0, K, 0, R.base});  // s_off 0: one S
      dj.alloc(sizeof(SketchJob) * js.size());
      VIE_CUDA(cudaMemcpyAsync(dj.p, js.data(), sizeof(SketchJob) * js.size(), cudaMemcpyHostToDevice, s));
      sketch_gather<<<(int)js.size(), 256, 0, s>>>(dj.as<SketchJob>(), (int)js.size(), dcols.as<int32_t>(),
                                                   S.as<float2>(), dA);
      VIE_CUDA(cudaGetLastError());
      VIE_CUDA(cudaStreamSynchronize(s));  // G, S, dj are released at the end of this iteration
    }
  }
};

// D = Z(tau, tau) in complex FP32, column-major n x n (tree order within tau)
void dense_block(vie_op* h, int64_t a, int64_t n, float2* D, cudaStream_t s) {
  const auto& perm = h->tree.perm;
  DevBuf rows, cols, tmp;
  std::vector<int32_t> r(n);
  for (int64_t i = 0; i < n; ++i) r[i] = perm[a + i];
  rows.alloc(sizeof(int32_t) * n);
  VIE_CUDA(cudaMemcpyAsync(rows.p, r.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
  const int64_t panel = std::max<int64_t>(1, (int64_t(1) << 26) / n);  // columns per panel
  tmp.alloc(sizeof(double2) * n * std::min(panel, n));
  cols.alloc(sizeof(int32_t) * n * std::min(panel, n));
  DevBuf prow;
  prow.alloc(sizeof(int32_t) * n * std::min(panel, n));
  for (int64_t c0 = 0; c0 < n; c0 += panel) {
    const int64_t nc = std::min(panel, n - c0);
    std::vector<int32_t> pr(n * nc), pc(n * nc);
    for (int64_t j = 0; j < nc; ++j)
      for (int64_t i = 0; i < n; ++i) { pr[j * n + i] = r[i]; pc[j * n + i] = r[c0 + j]; }
    VIE_CUDA(cudaMemcpyAsync(prow.p, pr.data(), sizeof(int32_t) * n * nc, cudaMemcpyHostToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(cols.p, pc.data(), sizeof(int32_t) * n * nc, cudaMemcpyHostToDevice, s));
    entries_pairs(h->geo, prow.as<int32_t>(), cols.as<int32_t>(), n * nc, tmp.as<double2>(), s, /*far32=*/true);
    c128_to_c64<<<grid_for(n * nc), 256, 0, s>>>(tmp.as<double2>(), D + c0 * n, n * nc);
    VIE_CUDA(cudaGetLastError());
    VIE_CUDA(cudaStreamSynchronize(s));
  }
}

// Dinv = D^-1 (D is overwritten by its LU factors)
void dense_inverse(cusolverDnHandle_t sol, float2* D, float2* Dinv, int64_t n, cudaStream_t s) {
  int lwork = 0;
  VIE_CUSOLVER(cusolverDnCgetrf_bufferSize(sol, (int)n, (int)n, (cuComplex*)D, (int)n, &lwork));
  DevBuf work, ipiv, info;
  work.alloc(sizeof(cuComplex) * std::max(lwork, 1));
  ipiv.alloc(sizeof(int) * n);
  info.alloc(sizeof(int));
  VIE_CUSOLVER(cusolverDnCgetrf(sol, (int)n, (int)n, (cuComplex*)D, (int)n, work.as<cuComplex>(), ipiv.as<int>(),
                                info.as<int>()));
  set_identity<<<grid_for(n * n), 256, 0, s>>>(Dinv, n);
  VIE_CUSOLVER(cusolverDnCgetrs(sol, CUBLAS_OP_N, (int)n, (int)n, (const cuComplex*)D, (int)n, ipiv.as<int>(),
                                (cuComplex*)Dinv, (int)n, info.as<int>()));
  int hinfo = 0;
  VIE_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  VIE_REQUIRE(hinfo == 0, VIE_ENAN, "singular diagonal block in the inverse construction");
}

}  // namespace

void build_inverse(vie_op* h, cudaStream_t s, BuildResult& res) {
  const Tree& t = h->tree;
  const int LH = t.levels;
  size_t free_b = 0, total_b = 0;
  VIE_CUDA(cudaMemGetInfo(&free_b, &total_b));
  // room for the dense matrices: what is free now, less a margin for the ID
  // builder's scratch, the solver workspace and the factors being built
  const int64_t margin = int64_t(24) << 30;
  const int64_t room = std::max<int64_t>(0, (int64_t)free_b - margin);
  auto level_max = [&](int l) {
    int64_t big = 0;
    for (size_t i = 0; i + 1 < t.bounds[l].size(); ++i) big = std::max<int64_t>(big, t.bounds[l][i + 1] - t.bounds[l][i]);
    return big;
  };
  const int64_t limit = h->cfg.inv_dense_max > 0 ? h->cfg.inv_dense_max : kDenseInverseLimit;
  int l_min = 0;
  while (l_min < LH) {
    const int64_t big = level_max(l_min);
    if (big <= limit && 2 * big * big * (int64_t)sizeof(float2) <= room) break;
    ++l_min;
  }
  h->zinv_top_level = l_min;
  cusolverDnHandle_t sol = nullptr;
  VIE_CUSOLVER(cusolverDnCreate(&sol));
  struct Handle {
    cusolverDnHandle_t s;
    ~Handle() { if (s) cusolverDnDestroy(s); }
  } hd{sol};
  VIE_CUSOLVER(cusolverDnSetStream(sol, s));
  Program& P = h->zinv;
  P.stages.clear();
  P.ncoef = 0;
  // leaves: dense inverses (stage 0: y = D_leaf^-1 x)
  {
    const auto& b = t.bounds[LH];
    const int64_t nl = (int64_t)b.size() - 1;
    std::vector<DevBuf> inv(nl);
    DenseSource src;
    for (int64_t i = 0; i < nl; ++i) {
      const int64_t a = b[i], n = b[i + 1] - b[i];
      DevBuf D;
      D.alloc(sizeof(float2) * n * n);
      inv[i].alloc(sizeof(float2) * n * n);
      dense_block(h, a, n, D.as<float2>(), s);
      dense_inverse(sol, D.as<float2>(), inv[i].as<float2>(), n, s);
      src.refs.push_back(DenseRef{inv[i].as<float2>(), a, n});
    }
    build_program(h, {}, src, h->cfg.tol_fact, P, /*leaf_blocks=*/true, SP_X, s, res);
  }
  // levels L_H - 1 .. l_min: E_tau = D_tau^-1 diag(D_tau1, D_tau2) - I, compressed at chi_fact
  for (int l = LH - 1; l >= l_min; --l) {
    const auto& b = t.bounds[l];
    const auto& bc = t.bounds[l + 1];
    const int64_t nn = (int64_t)b.size() - 1;
    const int64_t big = level_max(l);
    // E_tau of a batch stay resident until the batch is compressed; one D_tau at a time
    const int64_t batch_room = room - big * big * (int64_t)sizeof(float2);
    for (int64_t i0 = 0; i0 < nn;) {
      std::vector<DevBuf> E;
      DenseSource src;
      src.sketch = true;  // IDs of E_tau from Gaussian row sketches (products with E_tau^H)
      src.seed = h->cfg.seed ^ (0x5851F42D4C957F2Dull * (uint64_t)(l + 1));
      std::vector<BfSpec> specs;
      int64_t used = 0;
      int64_t i = i0;
      for (; i < nn; ++i) {
        const int64_t a = b[i], n = b[i + 1] - b[i];
        const int64_t bytes = n * n * (int64_t)sizeof(float2);
        if (i > i0 && used + bytes > batch_room) break;
        const int64_t n1 = bc[2 * i + 1] - bc[2 * i], n2 = n - n1;
        DevBuf D, ipiv, info, work;
        D.alloc(bytes);
        E.emplace_back();
        E.back().alloc(bytes);
        used += bytes;
        float2* Dp = D.as<float2>();
        float2* Ep = E.back().as<float2>();
        dense_block(h, a, n, Dp, s);
        // E = diag(D_tau1, D_tau2) before D is factored in place
        VIE_CUDA(cudaMemsetAsync(Ep, 0, bytes, s));
        VIE_CUDA(cudaMemcpy2DAsync(Ep, sizeof(float2) * n, Dp, sizeof(float2) * n, sizeof(float2) * n1, n1,
                                   cudaMemcpyDeviceToDevice, s));
        VIE_CUDA(cudaMemcpy2DAsync(Ep + n1 * n + n1, sizeof(float2) * n, Dp + n1 * n + n1, sizeof(float2) * n,
                                   sizeof(float2) * n2, n2, cudaMemcpyDeviceToDevice, s));
        int lwork = 0;
        VIE_CUSOLVER(cusolverDnCgetrf_bufferSize(sol, (int)n, (int)n, (cuComplex*)Dp, (int)n, &lwork));
        work.alloc(sizeof(cuComplex) * std::max(lwork, 1));
        ipiv.alloc(sizeof(int) * n);
        info.alloc(sizeof(int));
        VIE_CUSOLVER(cusolverDnCgetrf(sol, (int)n, (int)n, (cuComplex*)Dp, (int)n, work.as<cuComplex>(),
                                      ipiv.as<int>(), info.as<int>()));
        VIE_CUSOLVER(cusolverDnCgetrs(sol, CUBLAS_OP_N, (int)n, (int)n, (const cuComplex*)Dp, (int)n, ipiv.as<int>(),
                                      (cuComplex*)Ep, (int)n, info.as<int>()));
        int hinfo = 0;
        VIE_CUDA(cudaMemcpyAsync(&hinfo, info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        VIE_CUDA(cudaStreamSynchronize(s));
        VIE_REQUIRE(hinfo == 0, VIE_ENAN, "singular diagonal block in the inverse construction");
        sub_identity<<<grid_for(n), 256, 0, s>>>(Ep, n);
        VIE_CUDA(cudaGetLastError());
        src.refs.push_back(DenseRef{Ep, a, n});
        specs.push_back(BfSpec{l, i, i, (int)(i - i0)});
      }
      VIE_CUDA(cudaStreamSynchronize(s));
      build_program(h, specs, src, h->cfg.tol_fact, P, /*leaf_blocks=*/false, SP_Y, s, res);
      i0 = i;
    }
  }
  program_compact_coef(P, s);
  // levels above: from products only (Algorithm 1 line 7, Algorithm 2), no dense E_tau
  if (l_min > 0 && h->cfg.factor_dtype == VIE_C64) {
    InverseProductStats ps;
    build_inverse_products(h, l_min - 1, h->cfg.tol_fact, s, ps);
    h->zinv_top_level = 0;
    h->stats.zinv_product_levels = ps.levels;
    h->stats.inverse_products = ps.products;
    h->stats.invert_product_seconds = ps.seconds;
  }
  h->has_zinv = true;
}

}  // namespace vie
