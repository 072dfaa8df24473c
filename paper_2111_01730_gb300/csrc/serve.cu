// Serving: continuous batching of plane-wave solves against resident operators.
//
// Requests (one operator, nrhs right-hand sides, rtol) are admitted while the
// device memory their Krylov state needs fits the budget, and leave as soon as
// they are done, so requests that arrive while others are on the GPU join the
// next step.  A step advances every admitted request by one Arnoldi iteration
// of right-preconditioned GMRES (the same method as vie_solve): the current
// basis vectors of all active columns of one operator are packed into one
// multi-column block, and the blocks of all operators pass through Zinv and Z
// in one grouped sequence of launches (one per stage depth, a work list over
// operators, blocks and tiles; tensor-core items for blocks of 16 or more
// columns), replayed from a CUDA graph while the mix of operators and column
// counts stays the same; then every column is orthogonalized (classical
// Gram-Schmidt twice, FP64) by batched kernels over all requests.
// Restart cycles end with x += M V y and an FP64 refinement residual
// r = b - Z x, which also decides convergence; the Krylov state stays on the
// device for the whole life of the request.
#include <chrono>
#include <cmath>
#include <cstring>
#include <complex>
#include <deque>
#include <map>
#include <memory>

#include "internal.h"

namespace vie {

namespace {

using cd = std::complex<double>;

struct ColDesc {      // one right-hand side column of one request
  double2* V;         // basis vector j of this column at V + j * n
  double2* w;         // work vector
  double2* h;         // dot products (ldh entries)
  int64_t n;
  int32_t k;          // vectors to orthogonalize against
  int32_t pad;
};

struct OpPack {       // the packed columns of one operator in a step
  const int32_t* perm; // cluster-tree permutation of the operator
  float2* t;           // tree-ordered c64 block, n x ncol, columns fastest
  int64_t n;
  int32_t ncol, col0;  // its columns, and the first of them in the column-pointer table
};

__global__ void k_dots(const ColDesc* cols, int ncols, int kmax) {
  const int c = blockIdx.x / kmax, i = blockIdx.x % kmax;
  const ColDesc d = cols[c];
  if (i >= d.k) return;
  const double2* v = d.V + (int64_t)i * d.n;
  double re = 0, im = 0;
  for (int64_t t = threadIdx.x; t < d.n; t += blockDim.x) {
    double2 a = v[t], b = d.w[t];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  __shared__ double sr[256], si[256];
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) { sr[threadIdx.x] += sr[threadIdx.x + s]; si[threadIdx.x] += si[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) d.h[i] = make_double2(sr[0], si[0]);
}

__global__ void k_update(const ColDesc* cols, int ncols, int chunks) {
  const int c = blockIdx.x / chunks, part = blockIdx.x % chunks;
  const ColDesc d = cols[c];
  for (int64_t t = part * (int64_t)blockDim.x + threadIdx.x; t < d.n; t += (int64_t)chunks * blockDim.x) {
    double2 acc = d.w[t];
    for (int i = 0; i < d.k; ++i) {
      double2 a = d.V[(int64_t)i * d.n + t], b = d.h[i];
      acc.x -= a.x * b.x - a.y * b.y;
      acc.y -= a.x * b.y + a.y * b.x;
    }
    d.w[t] = acc;
  }
}

__global__ void k_norm(const ColDesc* cols, int ncols, double* out) {
  const ColDesc d = cols[blockIdx.x];
  double s = 0;
  for (int64_t t = threadIdx.x; t < d.n; t += blockDim.x) s += d.w[t].x * d.w[t].x + d.w[t].y * d.w[t].y;
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// V_{k} = w * scale  (k = d.k)
__global__ void k_store(const ColDesc* cols, int ncols, const double* scale, int chunks) {
  const int c = blockIdx.x / chunks, part = blockIdx.x % chunks;
  const ColDesc d = cols[c];
  const double s = scale[c];
  for (int64_t t = part * (int64_t)blockDim.x + threadIdx.x; t < d.n; t += (int64_t)chunks * blockDim.x) {
    double2 v = d.w[t];
    d.V[(int64_t)d.k * d.n + t] = make_double2(v.x * s, v.y * s);
  }
}

// t[i * ncol + j] = (c64) V_j[perm[i]]: the columns of each operator into its tree-ordered block
__global__ void k_pack_gather(const OpPack* ops, const double2* const* cols) {
  const OpPack d = ops[blockIdx.y];
  const int64_t tot = d.n * d.ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d.ncol;
    const int j = int(e % d.ncol);
    const double2 v = cols[d.col0 + j][d.perm[i]];
    d.t[e] = make_float2((float)v.x, (float)v.y);
  }
}

// W_j[perm[i]] = (c128) t[i * ncol + j]: each operator's result block back to its columns
__global__ void k_scatter_unpack(const OpPack* ops, double2* const* cols) {
  const OpPack d = ops[blockIdx.y];
  const int64_t tot = d.n * d.ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d.ncol;
    const int j = int(e % d.ncol);
    const float2 v = d.t[e];
    cols[d.col0 + j][d.perm[i]] = make_double2(v.x, v.y);
  }
}

// out(:, c) = sum_{i<k} V_i(c) y[c * ldh + i], columns of one request
__global__ void k_combine(const double2* V, int64_t n, int ldb, int k, const double2* y, int ldh, int nrhs,
                          float2* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = int(e / n);
    const int64_t t = e % n;
    double2 acc = make_double2(0, 0);
    for (int i = 0; i < k; ++i) {
      double2 a = V[((int64_t)c * ldb + i) * n + t], b = y[(int64_t)c * ldh + i];
      acc.x += a.x * b.x - a.y * b.y;
      acc.y += a.x * b.y + a.y * b.x;
    }
    out[e] = make_float2((float)acc.x, (float)acc.y);
  }
}

__global__ void k_add_c64(double2* x, const float2* d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i].x += d[i].x;
    x[i].y += d[i].y;
  }
}

__global__ void k_sub(const double2* a, const double2* b, double2* z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

__global__ void k_colnorm(const double2* w, int64_t n, double* out) {
  const double2* x = w + (int64_t)blockIdx.x * n;
  double s = 0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) s += x[t].x * x[t].x + x[t].y * x[t].y;
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

int gsz(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 8); }

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum ReqState { PENDING, RESIDUAL, ITERATING, DONE };

struct Req {
  int64_t id = 0;
  int op = 0;
  int nrhs = 0;
  double rtol = 0;
  ReqState state = PENDING;
  std::vector<double2> b_host;
  DevBuf b, x, r, V, w, h, t64a, t64b;
  int k = 0;           // Krylov dimension of the current cycle
  std::vector<int> its, live;
  std::vector<double> bn, rel, target;
  std::vector<std::vector<cd>> H, sn, g;
  std::vector<std::vector<double>> cs;
  double t_submit = 0, t_done = 0;
  size_t bytes = 0;
};

}  // namespace

struct Server {
  std::vector<vie_op*> ops;
  int m = 30, max_iter = 300;
  size_t budget = 0, used = 0;
  int64_t next_id = 1;
  std::deque<std::unique_ptr<Req>> pending;
  std::map<int64_t, std::unique_ptr<Req>> active, done;
  cudaStream_t s = nullptr;
  DevBuf cols, packs, nrm, scale, blk_a, blk_b, hall;
  int64_t steps = 0;
  // the grouped matvec of a step: per operator a tree-ordered block pair and a
  // coefficient block (grown as needed), a descriptor table, and CUDA graphs of the
  // launch sequence keyed by the operators, their column counts and the buffers
  std::vector<DevBuf> op_a, op_b, op_c;
  DevBuf table;
  struct StepGraph {
    std::vector<int64_t> key;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
  };
  std::vector<StepGraph> graphs;
  uint64_t graph_clock = 0;
  cudaStream_t capture = nullptr;
  ~Server() {
    for (auto& g : graphs) if (g.exec) cudaGraphExecDestroy(g.exec);
    if (capture) cudaStreamDestroy(capture);
  }
};

static size_t req_bytes(int64_t n, int nrhs, int m) {
  return (size_t)n * nrhs * 16 * (size_t)(m + 1 + 4) + (size_t)n * nrhs * 16 + 4096;
}

static void admit(Server& S) {
  while (!S.pending.empty()) {
    Req& q = *S.pending.front();
    const int64_t n = S.ops[q.op]->mesh.nf;
    const size_t need = req_bytes(n, q.nrhs, S.m);
    if (!S.active.empty() && S.used + need > S.budget) break;  // Krylov-basis memory admission
    std::unique_ptr<Req> r = std::move(S.pending.front());
    S.pending.pop_front();
    const int64_t nb = n * r->nrhs;
    r->b.alloc(sizeof(double2) * nb);
    r->x.alloc(sizeof(double2) * nb);
    r->r.alloc(sizeof(double2) * nb);
    r->w.alloc(sizeof(double2) * nb);
    r->V.alloc(sizeof(double2) * nb * (S.m + 1));
    r->h.alloc(sizeof(double2) * r->nrhs * (S.m + 1));
    r->t64a.alloc(sizeof(float2) * nb);
    r->t64b.alloc(sizeof(float2) * nb);
    VIE_CUDA(cudaMemcpyAsync(r->b.p, r->b_host.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, S.s));
    VIE_CUDA(cudaMemsetAsync(r->x.p, 0, sizeof(double2) * nb, S.s));
    VIE_CUDA(cudaMemsetAsync(r->V.p, 0, sizeof(double2) * nb * (S.m + 1), S.s));
    r->b_host.clear();
    r->b_host.shrink_to_fit();
    std::vector<double> bn2(r->nrhs);
    DevBuf tmp;
    tmp.alloc(sizeof(double) * r->nrhs);
    k_colnorm<<<r->nrhs, 256, 0, S.s>>>(r->b.as<double2>(), n, tmp.as<double>());
    VIE_CUDA(cudaMemcpyAsync(bn2.data(), tmp.p, sizeof(double) * r->nrhs, cudaMemcpyDeviceToHost, S.s));
    VIE_CUDA(cudaStreamSynchronize(S.s));
    r->bn.resize(r->nrhs);
    for (int c = 0; c < r->nrhs; ++c) r->bn[c] = std::sqrt(bn2[c]);
    r->its.assign(r->nrhs, 0);
    r->rel.assign(r->nrhs, 1.0);
    r->live.assign(r->nrhs, 0);
    r->state = RESIDUAL;
    r->bytes = need;
    S.used += need;
    const int64_t id = r->id;
    S.active[id] = std::move(r);
  }
}

// FP64 residual r = b - Z x; starts a cycle or finishes the request
static void start_cycle(Server& S, Req& q) {
  vie_op* h = S.ops[q.op];
  const int64_t n = h->mesh.nf, nb = n * q.nrhs;
  op_apply(h, VIE_OP_Z, q.x.p, q.r.p, q.nrhs, VIE_C128, S.s);
  k_sub<<<gsz(nb), 256, 0, S.s>>>(q.b.as<double2>(), q.r.as<double2>(), q.r.as<double2>(), nb);
  DevBuf tmp;
  tmp.alloc(sizeof(double) * q.nrhs);
  k_colnorm<<<q.nrhs, 256, 0, S.s>>>(q.r.as<double2>(), n, tmp.as<double>());
  std::vector<double> rn2(q.nrhs);
  VIE_CUDA(cudaMemcpyAsync(rn2.data(), tmp.p, sizeof(double) * q.nrhs, cudaMemcpyDeviceToHost, S.s));
  VIE_CUDA(cudaStreamSynchronize(S.s));
  bool any = false;
  std::vector<double> scale(q.nrhs, 0.0);
  q.H.assign(q.nrhs, std::vector<cd>((size_t)(S.m + 1) * S.m, cd(0)));
  q.cs.assign(q.nrhs, std::vector<double>(S.m, 0.0));
  q.sn.assign(q.nrhs, std::vector<cd>(S.m, cd(0)));
  q.g.assign(q.nrhs, std::vector<cd>(S.m + 1, cd(0)));
  q.target.assign(q.nrhs, 0.0);
  for (int c = 0; c < q.nrhs; ++c) {
    const double beta = std::sqrt(rn2[c]);
    q.rel[c] = q.bn[c] > 0 ? beta / q.bn[c] : 0.0;
    q.live[c] = q.rel[c] > q.rtol && q.its[c] < S.max_iter;
    any |= q.live[c] != 0;
    q.g[c][0] = beta;
    scale[c] = (q.live[c] && beta > 0) ? 1.0 / beta : 0.0;
    q.target[c] = std::max(q.rtol * q.bn[c], 1e-5 * beta);
  }
  q.k = 0;
  if (!any) {
    q.state = DONE;
    q.t_done = now_s();
    return;
  }
  // V_0 = r / beta (columns: V + c * (m+1) * n)
  std::vector<ColDesc> cds(q.nrhs);
  for (int c = 0; c < q.nrhs; ++c)
    cds[c] = ColDesc{q.V.as<double2>() + (int64_t)c * (S.m + 1) * n, q.r.as<double2>() + (int64_t)c * n,
                     q.h.as<double2>() + (int64_t)c * (S.m + 1), n, 0, 0};
  DevBuf dc, ds;
  dc.alloc(sizeof(ColDesc) * q.nrhs);
  ds.alloc(sizeof(double) * q.nrhs);
  VIE_CUDA(cudaMemcpyAsync(dc.p, cds.data(), sizeof(ColDesc) * q.nrhs, cudaMemcpyHostToDevice, S.s));
  VIE_CUDA(cudaMemcpyAsync(ds.p, scale.data(), sizeof(double) * q.nrhs, cudaMemcpyHostToDevice, S.s));
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, n / 4096));
  k_store<<<q.nrhs * chunks, 256, 0, S.s>>>(dc.as<ColDesc>(), q.nrhs, ds.as<double>(), chunks);
  VIE_CUDA(cudaStreamSynchronize(S.s));
  q.state = ITERATING;
}

// x += M (V y) for the columns of the cycle
static void end_cycle(Server& S, Req& q) {
  vie_op* h = S.ops[q.op];
  const int64_t n = h->mesh.nf, nb = n * q.nrhs;
  const int ldh = S.m + 1;
  std::vector<double2> yv((size_t)q.nrhs * ldh, make_double2(0, 0));
  for (int c = 0; c < q.nrhs; ++c) {
    const int k = q.k;
    std::vector<cd> yy(k);
    for (int i = k - 1; i >= 0; --i) {
      cd t = q.g[c][i];
      for (int j = i + 1; j < k; ++j) t -= q.H[c][(size_t)j * ldh + i] * yy[j];
      yy[i] = q.H[c][(size_t)i * ldh + i] != cd(0) ? t / q.H[c][(size_t)i * ldh + i] : cd(0);
    }
    for (int i = 0; i < k; ++i) yv[(size_t)c * ldh + i] = make_double2(yy[i].real(), yy[i].imag());
  }
  DevBuf dy;
  dy.alloc(sizeof(double2) * yv.size());
  VIE_CUDA(cudaMemcpyAsync(dy.p, yv.data(), sizeof(double2) * yv.size(), cudaMemcpyHostToDevice, S.s));
  k_combine<<<gsz(nb), 256, 0, S.s>>>(q.V.as<double2>(), n, S.m + 1, q.k, dy.as<double2>(), ldh, q.nrhs,
                                       q.t64a.as<float2>());
  if (h->has_zinv) {
    op_apply(h, VIE_OP_ZINV, q.t64a.p, q.t64b.p, q.nrhs, VIE_C64, S.s);
    k_add_c64<<<gsz(nb), 256, 0, S.s>>>(q.x.as<double2>(), q.t64b.as<float2>(), nb);
  } else {
    k_add_c64<<<gsz(nb), 256, 0, S.s>>>(q.x.as<double2>(), q.t64a.as<float2>(), nb);
  }
  VIE_CUDA(cudaStreamSynchronize(S.s));
  q.state = RESIDUAL;
}

static void arnoldi_step(Server& S) {
  // columns of all iterating requests, grouped by operator
  std::vector<Req*> reqs;
  for (auto& kv : S.active)
    if (kv.second->state == ITERATING) reqs.push_back(kv.second.get());
  if (reqs.empty()) return;
  std::map<int, std::vector<Req*>> by_op;
  for (Req* q : reqs) by_op[q->op].push_back(q);
  // Z (Zinv v) for the current basis vector of every column: the columns of each operator
  // packed into one tree-ordered block, all operators' blocks in one grouped launch sequence
  if (S.op_a.empty()) { S.op_a.resize(S.ops.size()); S.op_b.resize(S.ops.size()); S.op_c.resize(S.ops.size()); }
  const int nop = (int)by_op.size();
  std::vector<OpPack> pin, pout;
  std::vector<const double2*> cin;
  std::vector<double2*> cout;
  std::vector<GroupJob> jinv, jz;
  std::vector<int64_t> key;
  int64_t nmax_blk = 1;
  for (auto& kv : by_op) {
    const int oi = kv.first;
    vie_op* h = S.ops[oi];
    const int64_t n = h->mesh.nf;
    int ncol = 0;
    for (Req* q : kv.second)
      for (int c = 0; c < q->nrhs; ++c) {
        cin.push_back(q->V.as<double2>() + ((int64_t)c * (S.m + 1) + q->k) * n);
        cout.push_back(q->w.as<double2>() + (int64_t)c * n);
        ++ncol;
      }
    Program& pz = h->z;
    Program* pinv = h->has_zinv ? &h->zinv : nullptr;
    for (Program* p : {&pz, pinv}) {
      if (!p) continue;
      VIE_REQUIRE(p->factor_dtype == VIE_C64, VIE_EINVAL, "serving needs c64 factors");
      if (ncol >= p->tc_min_rhs) program_prepare_tc(*p, S.s);
    }
    const size_t vec = sizeof(float2) * (size_t)n * ncol;
    const size_t cbytes = sizeof(float2) * (size_t)std::max(pz.ncoef, pinv ? pinv->ncoef : 0) * ncol;
    if (S.op_a[oi].bytes < vec) { S.op_a[oi].alloc(vec); S.op_b[oi].alloc(vec); }
    if (S.op_c[oi].bytes < std::max<size_t>(cbytes, 8)) S.op_c[oi].alloc(std::max<size_t>(cbytes, 8));
    float2 *A = S.op_a[oi].as<float2>(), *B = S.op_b[oi].as<float2>(), *C = S.op_c[oi].as<float2>();
    const int col0 = (int)cin.size() - ncol;
    // Zinv: A -> B, then Z: B -> A; without an inverse Z: A -> B
    pin.push_back(OpPack{h->perm.as<int32_t>(), A, n, ncol, col0});
    pout.push_back(OpPack{h->perm.as<int32_t>(), pinv ? A : B, n, ncol, col0});
    if (pinv) {
      jinv.push_back(GroupJob{pinv, ncol, A, B, C});
      jz.push_back(GroupJob{&pz, ncol, B, A, C});
    } else {
      jz.push_back(GroupJob{&pz, ncol, A, B, C});
    }
    nmax_blk = std::max<int64_t>(nmax_blk, n * ncol);
    for (int64_t v : {(int64_t)oi, (int64_t)ncol, (int64_t)(uintptr_t)A, (int64_t)(uintptr_t)B, (int64_t)(uintptr_t)C})
      key.push_back(v);
  }
  // descriptor table: [pack-in x nop][pack-out x nop][column pointers in][column pointers out]
  const int ncol_all = (int)cin.size();
  const size_t tab_bytes = sizeof(OpPack) * 2 * nop + sizeof(void*) * 2 * (size_t)ncol_all;
  if (S.table.bytes < tab_bytes) S.table.alloc(tab_bytes * 2);
  std::vector<uint8_t> tab(tab_bytes);
  std::memcpy(tab.data(), pin.data(), sizeof(OpPack) * nop);
  std::memcpy(tab.data() + sizeof(OpPack) * nop, pout.data(), sizeof(OpPack) * nop);
  std::memcpy(tab.data() + sizeof(OpPack) * 2 * nop, cin.data(), sizeof(void*) * ncol_all);
  std::memcpy(tab.data() + sizeof(OpPack) * 2 * nop + sizeof(void*) * ncol_all, cout.data(), sizeof(void*) * ncol_all);
  VIE_CUDA(cudaMemcpyAsync(S.table.p, tab.data(), tab_bytes, cudaMemcpyHostToDevice, S.s));
  key.push_back((int64_t)(uintptr_t)S.table.p);
  key.push_back(ncol_all);
  Server::StepGraph* hit = nullptr;
  for (auto& g : S.graphs)
    if (g.exec && g.key == key) hit = &g;
  if (!hit) {
    if (S.graphs.size() < kGraphCache) {
      S.graphs.emplace_back();
      hit = &S.graphs.back();
    } else {
      hit = &S.graphs[0];
      for (auto& g : S.graphs)
        if (g.used < hit->used) hit = &g;
      if (hit->exec) { cudaGraphExecDestroy(hit->exec); hit->exec = nullptr; }
    }
    if (!S.capture) VIE_CUDA(cudaStreamCreateWithFlags(&S.capture, cudaStreamNonBlocking));
    uint8_t* T = S.table.as<uint8_t>();
    const OpPack* d_in = reinterpret_cast<const OpPack*>(T);
    const OpPack* d_out = reinterpret_cast<const OpPack*>(T + sizeof(OpPack) * nop);
    const double2* const* d_cin = reinterpret_cast<const double2* const*>(T + sizeof(OpPack) * 2 * nop);
    double2* const* d_cout =
        reinterpret_cast<double2* const*>(T + sizeof(OpPack) * 2 * nop + sizeof(void*) * ncol_all);
    const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(256, (nmax_blk + 255) / 256)), (unsigned)nop);
    cudaGraph_t g = nullptr;
    VIE_CUDA(cudaStreamBeginCapture(S.capture, cudaStreamCaptureModeThreadLocal));
    try {
      k_pack_gather<<<grid, 256, 0, S.capture>>>(d_in, d_cin);
      VIE_CUDA(cudaGetLastError());
      group_run_stages(jinv, S.capture);
      group_run_stages(jz, S.capture);
      k_scatter_unpack<<<grid, 256, 0, S.capture>>>(d_out, d_cout);
      VIE_CUDA(cudaGetLastError());
    } catch (...) {
      cudaStreamEndCapture(S.capture, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    VIE_CUDA(cudaStreamEndCapture(S.capture, &g));
    cudaError_t ie = cudaGraphInstantiate(&hit->exec, g, 0);
    cudaGraphDestroy(g);
    VIE_CUDA(ie);
    hit->key = key;
  }
  hit->used = ++S.graph_clock;
  VIE_CUDA(cudaGraphLaunch(hit->exec, S.s));

  // batched CGS2 over every column of every iterating request
  std::vector<ColDesc> cds;
  std::vector<std::pair<Req*, int>> who;
  int kmax = 1;
  int64_t nmax = 1;
  int ncols = 0;
  for (Req* q : reqs) ncols += q->nrhs;
  const int ldh0 = S.m + 1;
  if (S.hall.bytes < sizeof(double2) * (size_t)ncols * ldh0) S.hall.alloc(sizeof(double2) * (size_t)ncols * ldh0 * 2);
  for (Req* q : reqs) {
    const int64_t n = S.ops[q->op]->mesh.nf;
    for (int c = 0; c < q->nrhs; ++c) {
      // dot products of all columns land in one contiguous buffer: one copy to the host per pass
      cds.push_back(ColDesc{q->V.as<double2>() + (int64_t)c * (S.m + 1) * n, q->w.as<double2>() + (int64_t)c * n,
                            S.hall.as<double2>() + (int64_t)cds.size() * ldh0, n, q->k + 1, 0});
      who.push_back({q, c});
    }
    kmax = std::max(kmax, q->k + 1);
    nmax = std::max(nmax, n);
  }
  const int nc = (int)cds.size();
  if (S.cols.bytes < sizeof(ColDesc) * nc) S.cols.alloc(sizeof(ColDesc) * nc * 2);
  if (S.nrm.bytes < sizeof(double) * nc) { S.nrm.alloc(sizeof(double) * nc * 2); S.scale.alloc(sizeof(double) * nc * 2); }
  VIE_CUDA(cudaMemcpyAsync(S.cols.p, cds.data(), sizeof(ColDesc) * nc, cudaMemcpyHostToDevice, S.s));
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(64, nmax / 4096));
  std::vector<std::vector<double2>> hv(2);
  const int ldh = S.m + 1;
  std::vector<double2> hbuf((size_t)nc * ldh);
  std::vector<std::vector<cd>> hsum(nc, std::vector<cd>(kmax, cd(0)));
  for (int pass = 0; pass < 2; ++pass) {
    k_dots<<<nc * kmax, 256, 0, S.s>>>(S.cols.as<ColDesc>(), nc, kmax);
    k_update<<<nc * chunks, 256, 0, S.s>>>(S.cols.as<ColDesc>(), nc, chunks);
    VIE_CUDA(cudaMemcpyAsync(hbuf.data(), S.hall.p, sizeof(double2) * (size_t)nc * ldh, cudaMemcpyDeviceToHost, S.s));
    VIE_CUDA(cudaStreamSynchronize(S.s));
    for (int i = 0; i < nc; ++i)
      for (int j = 0; j < cds[i].k; ++j) hsum[i][j] += cd(hbuf[(size_t)i * ldh + j].x, hbuf[(size_t)i * ldh + j].y);
  }
  k_norm<<<nc, 256, 0, S.s>>>(S.cols.as<ColDesc>(), nc, S.nrm.as<double>());
  std::vector<double> hn(nc), scale(nc);
  VIE_CUDA(cudaMemcpyAsync(hn.data(), S.nrm.p, sizeof(double) * nc, cudaMemcpyDeviceToHost, S.s));
  VIE_CUDA(cudaStreamSynchronize(S.s));
  for (int i = 0; i < nc; ++i) {
    hn[i] = std::sqrt(hn[i]);
    Req* q = who[i].first;
    const int c = who[i].second;
    scale[i] = (q->live[c] && hn[i] > 0) ? 1.0 / hn[i] : 0.0;
  }
  // store V_{k+1}: the descriptors' k = q->k + 1 is the index of the new vector
  VIE_CUDA(cudaMemcpyAsync(S.scale.p, scale.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, S.s));
  k_store<<<nc * chunks, 256, 0, S.s>>>(S.cols.as<ColDesc>(), nc, S.scale.as<double>(), chunks);
  // Givens rotations per live column
  for (int i = 0; i < nc; ++i) {
    Req* q = who[i].first;
    const int c = who[i].second, k = q->k;
    if (!q->live[c]) continue;
    auto& Hc = q->H[c];
    for (int j = 0; j <= k; ++j) Hc[(size_t)k * ldh + j] = hsum[i][j];
    Hc[(size_t)k * ldh + k + 1] = hn[i];
    for (int j = 0; j < k; ++j) {
      cd t = q->cs[c][j] * Hc[(size_t)k * ldh + j] + q->sn[c][j] * Hc[(size_t)k * ldh + j + 1];
      Hc[(size_t)k * ldh + j + 1] = -std::conj(q->sn[c][j]) * Hc[(size_t)k * ldh + j] + q->cs[c][j] * Hc[(size_t)k * ldh + j + 1];
      Hc[(size_t)k * ldh + j] = t;
    }
    cd a = Hc[(size_t)k * ldh + k], bb = Hc[(size_t)k * ldh + k + 1];
    double den = std::sqrt(std::norm(a) + std::norm(bb));
    if (std::abs(a) == 0.0) { q->cs[c][k] = 0.0; q->sn[c][k] = 1.0; }
    else { q->cs[c][k] = std::abs(a) / den; q->sn[c][k] = (a / std::abs(a)) * std::conj(bb) / den; }
    Hc[(size_t)k * ldh + k] = q->cs[c][k] * a + q->sn[c][k] * bb;
    Hc[(size_t)k * ldh + k + 1] = 0.0;
    q->g[c][k + 1] = -std::conj(q->sn[c][k]) * q->g[c][k];
    q->g[c][k] = q->cs[c][k] * q->g[c][k];
    q->its[c] += 1;
    if (std::abs(q->g[c][k + 1]) <= q->target[c] || q->its[c] >= S.max_iter || hn[i] == 0.0) q->live[c] = 0;
  }
  VIE_CUDA(cudaStreamSynchronize(S.s));
  for (Req* q : reqs) {
    q->k += 1;
    bool any = false;
    for (int c = 0; c < q->nrhs; ++c) any |= q->live[c] != 0;
    if (!any || q->k == S.m) end_cycle(S, *q);
  }
}

}  // namespace vie

using namespace vie;

struct vie_server {
  Server S;
};

template <class F>
static vie_status guarded_s(F&& f) {
  try {
    f();
    return VIE_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return VIE_ENOMEM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return VIE_EINVAL;
  }
}

extern "C" {

vie_status vie_server_create(vie_op* const* ops, int32_t nops, int32_t restart, int32_t max_iter, int64_t mem_budget,
                             void* stream, vie_server** out) {
  return guarded_s([&] {
    VIE_REQUIRE(ops && nops >= 1 && out && restart >= 1 && max_iter >= 1 && mem_budget > 0, VIE_EINVAL,
                "bad server arguments");
    for (int i = 0; i < nops; ++i) {
      VIE_REQUIRE(ops[i] != nullptr, VIE_EINVAL, "null operator");
      VIE_REQUIRE(ops[i]->z.factor_dtype == VIE_C64, VIE_EINVAL, "serving needs operators with c64 factors");
    }
    auto* sv = new vie_server();
    sv->S.ops.assign(ops, ops + nops);
    sv->S.m = restart;
    sv->S.max_iter = max_iter;
    sv->S.budget = (size_t)mem_budget;
    sv->S.s = (cudaStream_t)stream;
    *out = sv;
  });
}

vie_status vie_server_submit(vie_server* sv, int32_t op, const void* V_host, int64_t nrhs, double rtol, int64_t* id) {
  return guarded_s([&] {
    VIE_REQUIRE(sv && V_host && id && nrhs >= 1 && nrhs <= (1 << 20) && rtol > 0, VIE_EINVAL, "bad request");
    Server& S = sv->S;
    VIE_REQUIRE(op >= 0 && op < (int)S.ops.size(), VIE_EINVAL, "operator index out of range");
    const int64_t n = S.ops[op]->mesh.nf;
    VIE_REQUIRE(req_bytes(n, (int)nrhs, S.m) <= S.budget, VIE_ENOMEM, "request needs more memory than the budget");
    auto r = std::make_unique<Req>();
    r->id = S.next_id++;
    r->op = op;
    r->nrhs = (int)nrhs;
    r->rtol = rtol;
    const double2* src = static_cast<const double2*>(V_host);
    for (int64_t i = 0; i < n * nrhs; ++i)
      VIE_REQUIRE(std::isfinite(src[i].x) && std::isfinite(src[i].y), VIE_ENAN, "right-hand side holds NaN or Inf");
    r->b_host.assign(src, src + n * nrhs);
    r->t_submit = now_s();
    *id = r->id;
    S.pending.push_back(std::move(r));
  });
}

vie_status vie_server_step(vie_server* sv, int32_t* active, int32_t* pending) {
  return guarded_s([&] {
    VIE_REQUIRE(sv, VIE_EINVAL, "null server");
    Trace tr("vie:server_step");
    Server& S = sv->S;
    admit(S);
    for (auto& kv : S.active)
      if (kv.second->state == RESIDUAL) start_cycle(S, *kv.second);
    arnoldi_step(S);
    // retire finished requests (their memory returns to the budget)
    for (auto it = S.active.begin(); it != S.active.end();) {
      if (it->second->state == RESIDUAL) start_cycle(S, *it->second);
      if (it->second->state == DONE) {
        Req& q = *it->second;
        q.V.release(); q.w.release(); q.r.release(); q.h.release(); q.t64a.release(); q.t64b.release(); q.b.release();
        S.used -= q.bytes;
        S.done[it->first] = std::move(it->second);
        it = S.active.erase(it);
      } else {
        ++it;
      }
    }
    ++S.steps;
    if (active) *active = (int32_t)S.active.size();
    if (pending) *pending = (int32_t)S.pending.size();
  });
}

vie_status vie_server_result(vie_server* sv, int64_t id, void* I_host, int32_t* iters, double* relres,
                             double* latency_s) {
  vie_status st = guarded_s([&] {
    VIE_REQUIRE(sv, VIE_EINVAL, "null server");
    Server& S = sv->S;
    auto it = S.done.find(id);
    if (it == S.done.end()) {
      bool known = S.active.count(id) > 0;
      for (auto& p : S.pending) known |= p->id == id;
      VIE_REQUIRE(known, VIE_EINVAL, "unknown request id");
      throw Error{VIE_ENOTCONV, "request not finished yet"};
    }
    Req& q = *it->second;
    const int64_t n = S.ops[q.op]->mesh.nf;
    if (I_host)
      VIE_CUDA(cudaMemcpy(I_host, q.x.p, sizeof(double2) * n * q.nrhs, cudaMemcpyDeviceToHost));
    for (int c = 0; c < q.nrhs; ++c) {
      if (iters) iters[c] = q.its[c];
      if (relres) relres[c] = q.rel[c];
    }
    if (latency_s) *latency_s = q.t_done - q.t_submit;
    S.done.erase(it);
  });
  return st;
}

vie_status vie_server_cancel(vie_server* sv, int64_t id) {
  return guarded_s([&] {
    VIE_REQUIRE(sv, VIE_EINVAL, "null server");
    Server& S = sv->S;
    for (auto it = S.pending.begin(); it != S.pending.end(); ++it)
      if ((*it)->id == id) {
        S.pending.erase(it);
        return;
      }
    auto a = S.active.find(id);
    if (a != S.active.end()) {
      // between steps nothing on the stream reads the request's buffers (every step ends
      // synchronized), and the next step's descriptor table no longer lists its columns
      VIE_CUDA(cudaStreamSynchronize(S.s));
      S.used -= a->second->bytes;
      S.active.erase(a);  // frees its device buffers
      return;
    }
    auto d = S.done.find(id);
    VIE_REQUIRE(d != S.done.end(), VIE_EINVAL, "unknown request id");
    S.done.erase(d);
  });
}

vie_status vie_server_memory(const vie_server* sv, int64_t* used, int64_t* budget) {
  return guarded_s([&] {
    VIE_REQUIRE(sv, VIE_EINVAL, "null server");
    if (used) *used = (int64_t)sv->S.used;
    if (budget) *budget = (int64_t)sv->S.budget;
  });
}

void vie_server_destroy(vie_server* sv) { delete sv; }

}  // extern "C"
