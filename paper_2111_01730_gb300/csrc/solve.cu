// Solve driver: right-preconditioned restarted GMRES inside FP64 iterative refinement.
//
// The paper solves the preconditioned system (Eq. 6) with TFQMR; the reading
// used here is right preconditioning, Z M u = r, x = M u, with M = Zinv when
// the operator carries one, so that the stopping test is on the true residual.
// Precision split: every application of Z or Zinv inside the Krylov loop runs
// on complex FP32 vectors (C32 factors, FP32 accumulation) -- or on FP64
// vectors when the operator stores FP64 factors (the plain FP64 solver); the Arnoldi basis,
// its classical Gram-Schmidt (applied twice) orthogonalization and the Givens
// least squares are FP64; the outer refinement residual r = b - Z x applies
// the same C32 factors with FP64 vectors and accumulation.
//
// Every right-hand side column runs its own Krylov space; the applies of all
// columns are batched into one multi-column apply.
#include <cmath>
#include <complex>

#include "internal.h"

namespace vie {

namespace {

using cd = std::complex<double>;

__global__ void to_c64(const double2* src, float2* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

__global__ void to_c128(const float2* src, double2* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = make_double2(src[i].x, src[i].y);
}

// v_j of column c lives at V + (c * ldb + j) * n
__global__ void gather_basis(const double2* V, int64_t n, int ldb, int j, int nrhs, double2* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    int c = int(e / n);
    int64_t i = e % n;
    out[e] = V[((int64_t)c * ldb + j) * n + i];
  }
}

// h[c * ldh + i] = V_i(c)^H w(c) for i < k  (one CTA per (i, c))
__global__ void dots(const double2* V, int64_t n, int ldb, const double2* w, int k, double2* h, int ldh) {
  const int i = blockIdx.x % k, c = blockIdx.x / k;
  const double2* v = V + ((int64_t)c * ldb + i) * n;
  const double2* x = w + (int64_t)c * n;
  double re = 0, im = 0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    double2 a = v[t], b = x[t];
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
  if (threadIdx.x == 0) h[(int64_t)c * ldh + i] = make_double2(sr[0], si[0]);
}

// w(c) -= sum_{i<k} V_i(c) h[c*ldh + i]
__global__ void orth_update(const double2* V, int64_t n, int ldb, double2* w, int k, const double2* h, int ldh,
                            int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    int c = int(e / n);
    int64_t t = e % n;
    double2 acc = w[e];
    for (int i = 0; i < k; ++i) {
      double2 a = V[((int64_t)c * ldb + i) * n + t], b = h[(int64_t)c * ldh + i];
      acc.x -= a.x * b.x - a.y * b.y;
      acc.y -= a.x * b.y + a.y * b.x;
    }
    w[e] = acc;
  }
}

__global__ void col_norm2(const double2* w, int64_t n, double* out) {
  const int c = blockIdx.x;
  const double2* x = w + (int64_t)c * n;
  double s = 0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) s += x[t].x * x[t].x + x[t].y * x[t].y;
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = sh[0];
}

// V_j(c) = w(c) * scale[c]
__global__ void store_basis(double2* V, int64_t n, int ldb, int j, const double2* w, const double* scale, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    int c = int(e / n);
    int64_t t = e % n;
    double s = scale[c];
    double2 v = w[e];
    V[((int64_t)c * ldb + j) * n + t] = make_double2(v.x * s, v.y * s);
  }
}

// out(c) = sum_{i<k} V_i(c) y[c*ldh + i]
__global__ void combine(const double2* V, int64_t n, int ldb, int k, const double2* y, int ldh, int nrhs, double2* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    int c = int(e / n);
    int64_t t = e % n;
    double2 acc = make_double2(0, 0);
    for (int i = 0; i < k; ++i) {
      double2 a = V[((int64_t)c * ldb + i) * n + t], b = y[(int64_t)c * ldh + i];
      acc.x += a.x * b.x - a.y * b.y;
      acc.y += a.x * b.y + a.y * b.x;
    }
    out[e] = acc;
  }
}

// z = a - b (elementwise)
__global__ void sub(const double2* a, const double2* b, double2* z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

// x += d for the columns with mask[c] != 0
__global__ void add_masked(double2* x, const double2* d, int64_t n, int nrhs, const int* mask) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[e / n]) continue;
    x[e].x += d[e].x;
    x[e].y += d[e].y;
  }
}

__global__ void has_nonfinite(const double2* a, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[i].x) || !isfinite(a[i].y)) *flag = 1;
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 8); }

}  // namespace

struct SolveWs {
  DevBuf V, w, t64a, t64b, h, y, nrm, scale, mask, flag, r, x, d, tmp;
};

// Y = op(X) on c64 or c128 device vectors (column-major, ld = n)
void op_apply(vie_op* h, int which, const void* X, void* Y, int64_t nrhs, int dtype, cudaStream_t s);

void solve_gmres(vie_op* h, const double2* b, double2* x_out, int64_t nrhs, double rtol, int restart, int max_iter,
                 int32_t* iters_out, double* relres_out, cudaStream_t s, bool& converged_all) {
  const int64_t n = h->mesh.nf;
  const int m = std::max(1, restart);
  const int ldb = m + 1, ldh = m + 1;
  const int64_t nb = n * nrhs;
  SolveWs ws;
  ws.V.alloc(sizeof(double2) * nb * ldb);
  VIE_CUDA(cudaMemsetAsync(ws.V.p, 0, sizeof(double2) * nb * ldb, s));
  ws.w.alloc(sizeof(double2) * nb);
  // operators with FP64 factors solve in FP64 throughout (the plain FP64 path)
  const bool fp64 = h->cfg.factor_dtype == VIE_C128;
  ws.t64a.alloc((fp64 ? sizeof(double2) : sizeof(float2)) * nb);
  ws.t64b.alloc((fp64 ? sizeof(double2) : sizeof(float2)) * nb);
  ws.h.alloc(sizeof(double2) * nrhs * ldh);
  ws.y.alloc(sizeof(double2) * nrhs * ldh);
  ws.nrm.alloc(sizeof(double) * nrhs);
  ws.scale.alloc(sizeof(double) * nrhs);
  ws.mask.alloc(sizeof(int) * nrhs);
  ws.flag.alloc(sizeof(int));
  ws.r.alloc(sizeof(double2) * nb);
  ws.x.alloc(sizeof(double2) * nb);
  ws.d.alloc(sizeof(double2) * nb);
  ws.tmp.alloc(sizeof(double2) * nb);
  const int G = grid_for(nb);
  double2* V = ws.V.as<double2>();
  double2* w = ws.w.as<double2>();
  float2* va = ws.t64a.as<float2>();
  float2* vb = ws.t64b.as<float2>();
  // NaN / Inf in the right-hand side is an input error
  VIE_CUDA(cudaMemsetAsync(ws.flag.p, 0, sizeof(int), s));
  has_nonfinite<<<G, 256, 0, s>>>(b, nb, ws.flag.as<int>());
  int flag = 0;
  VIE_CUDA(cudaMemcpyAsync(&flag, ws.flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  VIE_REQUIRE(!flag, VIE_ENAN, "right-hand side holds NaN or Inf");

  std::vector<double> bn2(nrhs), rn2(nrhs);
  col_norm2<<<(int)nrhs, 256, 0, s>>>(b, n, ws.nrm.as<double>());
  VIE_CUDA(cudaMemcpyAsync(bn2.data(), ws.nrm.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaMemsetAsync(ws.x.p, 0, sizeof(double2) * nb, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  std::vector<int> its(nrhs, 0);
  std::vector<double> rel(nrhs, 1.0);
  std::vector<int> active(nrhs, 1);
  const bool pre = h->has_zinv;
  const int max_outer = 1000;  // refinement steps; columns stop at rtol or max_iter
  for (int outer = 0; outer < max_outer; ++outer) {
    // r = b - Z x   (C32 factors, FP64 vectors and accumulation)
    op_apply(h, VIE_OP_Z, ws.x.p, ws.tmp.p, nrhs, VIE_C128, s);
    sub<<<G, 256, 0, s>>>(b, ws.tmp.as<double2>(), ws.r.as<double2>(), nb);
    col_norm2<<<(int)nrhs, 256, 0, s>>>(ws.r.as<double2>(), n, ws.nrm.as<double>());
    VIE_CUDA(cudaMemcpyAsync(rn2.data(), ws.nrm.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    for (int c = 0; c < nrhs; ++c) {
      rel[c] = bn2[c] > 0 ? std::sqrt(rn2[c] / bn2[c]) : 0.0;
      active[c] = rel[c] > rtol && its[c] < max_iter;
      any |= active[c] != 0;
    }
    if (!any) break;
    // inner GMRES(m) on Z M u = r, started from u = 0, one cycle per refinement step
    std::vector<double> beta(nrhs), scale(nrhs);
    for (int c = 0; c < nrhs; ++c) {
      beta[c] = std::sqrt(rn2[c]);
      scale[c] = beta[c] > 0 ? 1.0 / beta[c] : 0.0;
    }
    VIE_CUDA(cudaMemcpyAsync(ws.scale.p, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    store_basis<<<G, 256, 0, s>>>(V, n, ldb, 0, ws.r.as<double2>(), ws.scale.as<double>(), (int)nrhs);
    std::vector<std::vector<cd>> H(nrhs, std::vector<cd>((size_t)ldh * m, cd(0)));
    std::vector<std::vector<double>> cs(nrhs, std::vector<double>(m));
    std::vector<std::vector<cd>> sn(nrhs, std::vector<cd>(m)), g(nrhs, std::vector<cd>(m + 1, cd(0)));
    for (int c = 0; c < nrhs; ++c) g[c][0] = beta[c];
    std::vector<int> kused(nrhs, 0), live(active);
    // the inner solve aims at the outer tolerance or 1e-5 relative, whichever is looser
    std::vector<double> target(nrhs);
    for (int c = 0; c < nrhs; ++c)
      target[c] = std::max(rtol * std::sqrt(bn2[c]), 1e-5 * beta[c]);
    std::vector<double2> hv((size_t)nrhs * ldh), hv2((size_t)nrhs * ldh);
    std::vector<double> hn(nrhs);
    for (int k = 0; k < m; ++k) {
      bool any_live = false;
      for (int c = 0; c < nrhs; ++c) any_live |= live[c] != 0;
      if (!any_live) break;
      // w = Z M v_k
      if (fp64) {
        double2* da = ws.t64a.as<double2>();
        double2* db = ws.t64b.as<double2>();
        gather_basis<<<G, 256, 0, s>>>(V, n, ldb, k, (int)nrhs, da);
        if (pre) {
          op_apply(h, VIE_OP_ZINV, da, db, nrhs, VIE_C128, s);
          op_apply(h, VIE_OP_Z, db, w, nrhs, VIE_C128, s);
        } else {
          op_apply(h, VIE_OP_Z, da, w, nrhs, VIE_C128, s);
        }
      } else {
        gather_basis<<<G, 256, 0, s>>>(V, n, ldb, k, (int)nrhs, ws.tmp.as<double2>());
        to_c64<<<G, 256, 0, s>>>(ws.tmp.as<double2>(), va, nb);
        if (pre) {
          op_apply(h, VIE_OP_ZINV, va, vb, nrhs, VIE_C64, s);
          op_apply(h, VIE_OP_Z, vb, va, nrhs, VIE_C64, s);
        } else {
          op_apply(h, VIE_OP_Z, va, vb, nrhs, VIE_C64, s);
          std::swap(va, vb);
        }
        to_c128<<<G, 256, 0, s>>>(va, w, nb);
      }
      // classical Gram-Schmidt, twice
      for (int pass = 0; pass < 2; ++pass) {
        dots<<<(int)nrhs * (k + 1), 256, 0, s>>>(V, n, ldb, w, k + 1, ws.h.as<double2>(), ldh);
        orth_update<<<G, 256, 0, s>>>(V, n, ldb, w, k + 1, ws.h.as<double2>(), ldh, (int)nrhs);
        VIE_CUDA(cudaMemcpyAsync(pass == 0 ? hv.data() : hv2.data(), ws.h.p, sizeof(double2) * nrhs * ldh,
                                 cudaMemcpyDeviceToHost, s));
      }
      col_norm2<<<(int)nrhs, 256, 0, s>>>(w, n, ws.nrm.as<double>());
      VIE_CUDA(cudaMemcpyAsync(hn.data(), ws.nrm.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
      VIE_CUDA(cudaStreamSynchronize(s));
      for (int c = 0; c < nrhs; ++c) {
        hn[c] = std::sqrt(hn[c]);
        scale[c] = (live[c] && hn[c] > 0) ? 1.0 / hn[c] : 0.0;
      }
      VIE_CUDA(cudaMemcpyAsync(ws.scale.p, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
      store_basis<<<G, 256, 0, s>>>(V, n, ldb, k + 1, w, ws.scale.as<double>(), (int)nrhs);
      for (int c = 0; c < nrhs; ++c) {
        if (!live[c]) continue;
        auto& Hc = H[c];
        for (int i = 0; i <= k; ++i) {
          double2 a = hv[(size_t)c * ldh + i], b2 = hv2[(size_t)c * ldh + i];
          Hc[(size_t)k * ldh + i] = cd(a.x + b2.x, a.y + b2.y);
        }
        Hc[(size_t)k * ldh + k + 1] = hn[c];
        for (int i = 0; i < k; ++i) {  // previous rotations [c, s; -conj(s), c]
          cd t = cs[c][i] * Hc[(size_t)k * ldh + i] + sn[c][i] * Hc[(size_t)k * ldh + i + 1];
          Hc[(size_t)k * ldh + i + 1] = -std::conj(sn[c][i]) * Hc[(size_t)k * ldh + i] + cs[c][i] * Hc[(size_t)k * ldh + i + 1];
          Hc[(size_t)k * ldh + i] = t;
        }
        cd a = Hc[(size_t)k * ldh + k], bb = Hc[(size_t)k * ldh + k + 1];
        double den = std::sqrt(std::norm(a) + std::norm(bb));
        if (std::abs(a) == 0.0) { cs[c][k] = 0.0; sn[c][k] = 1.0; }
        else { cs[c][k] = std::abs(a) / den; sn[c][k] = (a / std::abs(a)) * std::conj(bb) / den; }
        Hc[(size_t)k * ldh + k] = cs[c][k] * a + sn[c][k] * bb;
        Hc[(size_t)k * ldh + k + 1] = 0.0;
        g[c][k + 1] = -std::conj(sn[c][k]) * g[c][k];
        g[c][k] = cs[c][k] * g[c][k];
        kused[c] = k + 1;
        its[c] += 1;
        if (std::abs(g[c][k + 1]) <= target[c] || its[c] >= max_iter || hn[c] == 0.0) live[c] = 0;
      }
    }
    // y = H^-1 g (upper triangular), d = M (V y), x += d
    std::vector<double2> yv((size_t)nrhs * ldh, make_double2(0, 0));
    for (int c = 0; c < nrhs; ++c) {
      if (!active[c]) continue;
      const int k = kused[c];
      std::vector<cd> yy(k);
      for (int i = k - 1; i >= 0; --i) {
        cd t = g[c][i];
        for (int j = i + 1; j < k; ++j) t -= H[c][(size_t)j * ldh + i] * yy[j];
        yy[i] = t / H[c][(size_t)i * ldh + i];
      }
      for (int i = 0; i < k; ++i) yv[(size_t)c * ldh + i] = make_double2(yy[i].real(), yy[i].imag());
    }
    VIE_CUDA(cudaMemcpyAsync(ws.y.p, yv.data(), sizeof(double2) * nrhs * ldh, cudaMemcpyHostToDevice, s));
    combine<<<G, 256, 0, s>>>(V, n, ldb, m, ws.y.as<double2>(), ldh, (int)nrhs, ws.d.as<double2>());
    if (pre && fp64) {
      op_apply(h, VIE_OP_ZINV, ws.d.p, ws.tmp.p, nrhs, VIE_C128, s);
      VIE_CUDA(cudaMemcpyAsync(ws.d.p, ws.tmp.p, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, s));
    } else if (pre) {
      to_c64<<<G, 256, 0, s>>>(ws.d.as<double2>(), va, nb);
      op_apply(h, VIE_OP_ZINV, va, vb, nrhs, VIE_C64, s);
      to_c128<<<G, 256, 0, s>>>(vb, ws.d.as<double2>(), nb);
    }
    std::vector<int> mask(active);
    VIE_CUDA(cudaMemcpyAsync(ws.mask.p, mask.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
    add_masked<<<G, 256, 0, s>>>(ws.x.as<double2>(), ws.d.as<double2>(), n, (int)nrhs, ws.mask.as<int>());
    VIE_CUDA(cudaStreamSynchronize(s));
  }
  converged_all = true;
  for (int c = 0; c < nrhs; ++c) {
    if (iters_out) iters_out[c] = its[c];
    if (relres_out) relres_out[c] = rel[c];
    converged_all &= rel[c] <= rtol;
  }
  VIE_CUDA(cudaMemcpyAsync(x_out, ws.x.p, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, s));
  VIE_CUDA(cudaStreamSynchronize(s));
}

}  // namespace vie
