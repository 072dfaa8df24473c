// Solve drivers: right-preconditioned restarted GMRES inside FP64 iterative
// refinement, and the paper's left-preconditioned TFQMR.
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

// out[c] = a(c)^H b(c), one CTA per column
__global__ void coldot(const double2* a, const double2* b, int64_t n, double2* out) {
  const int c = blockIdx.x;
  const double2* x = a + (int64_t)c * n;
  const double2* y = b + (int64_t)c * n;
  double re = 0, im = 0;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    re += x[t].x * y[t].x + x[t].y * y[t].y;
    im += x[t].x * y[t].y - x[t].y * y[t].x;
  }
  __shared__ double sr[256], si[256];
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) { sr[threadIdx.x] += sr[threadIdx.x + k]; si[threadIdx.x] += si[threadIdx.x + k]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = make_double2(sr[0], si[0]);
}

// out(c) = a(c) + cb[c] * b(c)   (out may alias a or b)
__global__ void axpby_col(const double2* a, const double2* b, const double2* cb, double2* out, int64_t n, int nrhs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 k = cb[e / n], u = a[e], v = b[e];
    out[e] = make_double2(u.x + k.x * v.x - k.y * v.y, u.y + k.x * v.y + k.y * v.x);
  }
}

}  // namespace

struct SolveWs {
  DevBuf V, w, t64a, t64b, h, y, nrm, scale, mask, flag, r, x, d, tmp;
};

// Y = op(X) on c64 or c128 device vectors (column-major, ld = n)
void op_apply(vie_op* h, int which, const void* X, void* Y, int64_t nrhs, int dtype, cudaStream_t s);

void solve_gmres(vie_op* h, const double2* b, double2* x_out, int64_t nrhs, double rtol, int restart, int max_iter,
                 int32_t* iters_out, double* relres_out, cudaStream_t s, bool& converged_all) {
  Trace tr("vie:solve/gmres");
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

// Left-preconditioned TFQMR (Freund 1993) on M Z I = M V (Eq. 6), M = Zinv
// when the operator carries one.  Per iteration: y2 = y1 - alpha v, two
// quasi-residual half-steps (w -= alpha A y; theta = ||w|| / tau;
// c = 1 / sqrt(1 + theta^2); tau *= theta c; d = y + theta_prev^2 eta_prev /
// alpha d; eta = c^2 alpha; x += eta d), then beta = rho_new / rho,
// y1 = w + beta y2 and v = A y1 + beta (A y2 + beta v): two applications of
// A = M Z.  A column stops when tau sqrt(m + 1) <= rtol ||M V|| (m = half-steps),
// and the true preconditioned residual, applied with FP64 vectors, decides
// whether it restarts from its iterate.  Inside the recurrence the applies of
// a C32 operator run on complex FP32 vectors; vectors and scalars are FP64.
// All columns step together through batched multi-column applies; a stopped
// column gets zero coefficients so that its iterate stays fixed.
void solve_tfqmr(vie_op* h, const double2* b, double2* x_out, int64_t nrhs, double rtol, int max_iter,
                 int32_t* iters_out, double* relres_out, cudaStream_t s, bool& converged_all) {
  Trace tr("vie:solve/tfqmr");
  const int64_t n = h->mesh.nf;
  const int64_t nb = n * nrhs;
  const bool fp64 = h->cfg.factor_dtype == VIE_C128;
  const bool pre = h->has_zinv;
  DevBuf bx, bmb, brt, bw, by1, by2, bay1, bay2, bv, bd, bt, bt2, bva, bvb, bcoef, bdot, bnrm, bflag;
  for (DevBuf* p : {&bx, &bmb, &brt, &bw, &by1, &by2, &bay1, &bay2, &bv, &bd, &bt, &bt2}) p->alloc(sizeof(double2) * nb);
  bva.alloc((fp64 ? sizeof(double2) : sizeof(float2)) * nb);
  bvb.alloc((fp64 ? sizeof(double2) : sizeof(float2)) * nb);
  bcoef.alloc(sizeof(double2) * nrhs);
  bdot.alloc(sizeof(double2) * nrhs);
  bnrm.alloc(sizeof(double) * nrhs);
  bflag.alloc(sizeof(int));
  const int G = grid_for(nb);
  double2 *x = bx.as<double2>(), *mb = bmb.as<double2>(), *rt = brt.as<double2>(), *w = bw.as<double2>();
  double2 *y1 = by1.as<double2>(), *y2 = by2.as<double2>(), *Ay1 = bay1.as<double2>(), *Ay2 = bay2.as<double2>();
  double2 *v = bv.as<double2>(), *d = bd.as<double2>(), *t = bt.as<double2>(), *t2 = bt2.as<double2>();
  double2* coef = bcoef.as<double2>();
  VIE_CUDA(cudaMemsetAsync(bflag.p, 0, sizeof(int), s));
  has_nonfinite<<<G, 256, 0, s>>>(b, nb, bflag.as<int>());
  int flag = 0;
  VIE_CUDA(cudaMemcpyAsync(&flag, bflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  VIE_REQUIRE(!flag, VIE_ENAN, "right-hand side holds NaN or Inf");

  // out = A u inside the recurrence (C32 applies for a C32 operator)
  auto applyA = [&](const double2* u, double2* out) {
    if (fp64) {
      if (pre) {
        op_apply(h, VIE_OP_Z, u, bva.p, nrhs, VIE_C128, s);
        op_apply(h, VIE_OP_ZINV, bva.p, out, nrhs, VIE_C128, s);
      } else {
        op_apply(h, VIE_OP_Z, u, out, nrhs, VIE_C128, s);
      }
    } else {
      to_c64<<<G, 256, 0, s>>>(u, bva.as<float2>(), nb);
      op_apply(h, VIE_OP_Z, bva.p, bvb.p, nrhs, VIE_C64, s);
      float2* r = bvb.as<float2>();
      if (pre) {
        op_apply(h, VIE_OP_ZINV, bvb.p, bva.p, nrhs, VIE_C64, s);
        r = bva.as<float2>();
      }
      to_c128<<<G, 256, 0, s>>>(r, out, nb);
    }
  };
  // out = M u with FP64 vectors (C32 or FP64 factors)
  auto applyM = [&](const double2* u, double2* out) {
    if (pre) op_apply(h, VIE_OP_ZINV, u, out, nrhs, VIE_C128, s);
    else VIE_CUDA(cudaMemcpyAsync(out, u, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, s));
  };
  auto norms = [&](const double2* a, std::vector<double>& out) {
    col_norm2<<<(int)nrhs, 256, 0, s>>>(a, n, bnrm.as<double>());
    VIE_CUDA(cudaMemcpyAsync(out.data(), bnrm.p, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    for (double& q : out) q = std::sqrt(q);
  };
  auto dotc = [&](const double2* a, const double2* bb, std::vector<cd>& out) {
    coldot<<<(int)nrhs, 256, 0, s>>>(a, bb, n, bdot.as<double2>());
    std::vector<double2> hv(nrhs);
    VIE_CUDA(cudaMemcpyAsync(hv.data(), bdot.p, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    for (int64_t c = 0; c < nrhs; ++c) out[c] = cd(hv[c].x, hv[c].y);
  };
  // out = a + k[c] b
  auto axpby = [&](const double2* a, const std::vector<cd>& k, const double2* bb, double2* out) {
    std::vector<double2> hk(nrhs);
    for (int64_t c = 0; c < nrhs; ++c) hk[c] = make_double2(k[c].real(), k[c].imag());
    VIE_CUDA(cudaMemcpyAsync(coef, hk.data(), sizeof(double2) * nrhs, cudaMemcpyHostToDevice, s));
    axpby_col<<<G, 256, 0, s>>>(a, bb, coef, out, n, (int)nrhs);
    VIE_CUDA(cudaStreamSynchronize(s));  // hk goes out of scope
  };
  // preconditioned residual r = M (b - Z x) into `out` (FP64 vectors)
  auto pres = [&](double2* out) {
    op_apply(h, VIE_OP_Z, x, t2, nrhs, VIE_C128, s);
    sub<<<G, 256, 0, s>>>(b, t2, t2, nb);
    applyM(t2, out);
  };

  VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * nb, s));
  applyM(b, mb);
  std::vector<double> nmb(nrhs), nr(nrhs), nw(nrhs);
  norms(mb, nmb);
  std::vector<int> its(nrhs, 0), want(nrhs, 0);
  std::vector<double> prel(nrhs, 1.0);
  for (int cycle = 0; cycle < 64; ++cycle) {
    pres(t);  // r0 = M (b - Z x)
    norms(t, nr);
    bool any = false;
    for (int64_t c = 0; c < nrhs; ++c) {
      prel[c] = nmb[c] > 0 ? nr[c] / nmb[c] : 0.0;
      want[c] = prel[c] > rtol && its[c] < max_iter;
      any |= want[c] != 0;
    }
    if (!any) break;
    const std::vector<int> its0(its);
    std::vector<int> live(want);
    VIE_CUDA(cudaMemcpyAsync(rt, t, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(w, t, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, s));
    VIE_CUDA(cudaMemcpyAsync(y1, t, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, s));
    VIE_CUDA(cudaMemsetAsync(d, 0, sizeof(double2) * nb, s));
    applyA(y1, Ay1);
    VIE_CUDA(cudaMemcpyAsync(v, Ay1, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, s));
    std::vector<double> tau(nr), theta(nrhs, 0.0);
    std::vector<cd> rho(nrhs), alpha(nrhs), sigma(nrhs), beta(nrhs), eta(nrhs, cd(0)), kd(nrhs), kx(nrhs), ka(nrhs);
    std::vector<int> m(nrhs, 0);
    for (int64_t c = 0; c < nrhs; ++c) rho[c] = cd(nr[c] * nr[c], 0.0);  // r~0 = r0
    for (;;) {
      dotc(rt, v, sigma);
      bool alive = false;
      for (int64_t c = 0; c < nrhs; ++c) {
        if (live[c] && (std::abs(sigma[c]) == 0.0 || std::abs(rho[c]) == 0.0)) live[c] = 0;  // breakdown
        alpha[c] = live[c] ? rho[c] / sigma[c] : cd(0);
        ka[c] = -alpha[c];
        alive |= live[c] != 0;
      }
      if (!alive) break;
      axpby(y1, ka, v, y2);  // y2 = y1 - alpha v
      applyA(y2, Ay2);
      for (int64_t c = 0; c < nrhs; ++c) its[c] += live[c];
      for (int half = 0; half < 2; ++half) {
        const double2* y = half == 0 ? y1 : y2;
        const double2* Ay = half == 0 ? Ay1 : Ay2;
        axpby(w, ka, Ay, w);  // w -= alpha A y
        norms(w, nw);
        for (int64_t c = 0; c < nrhs; ++c) {
          kd[c] = kx[c] = cd(0);
          if (!live[c]) continue;
          m[c] += 1;
          const double th_prev = theta[c];
          const cd eta_prev = eta[c];
          theta[c] = tau[c] > 0 ? nw[c] / tau[c] : 0.0;
          const double cc = 1.0 / std::sqrt(1.0 + theta[c] * theta[c]);
          tau[c] = tau[c] * theta[c] * cc;
          kd[c] = th_prev * th_prev * eta_prev / alpha[c];
          eta[c] = cc * cc * alpha[c];
          kx[c] = eta[c];
          if (tau[c] * std::sqrt((double)m[c] + 1.0) <= rtol * nmb[c]) live[c] = 0;
        }
        axpby(y, kd, d, d);  // d = y + (theta_prev^2 eta_prev / alpha) d
        axpby(x, kx, d, x);  // x += eta d
        for (int64_t c = 0; c < nrhs; ++c) ka[c] = live[c] ? -alpha[c] : cd(0);
      }
      bool more = false;
      for (int64_t c = 0; c < nrhs; ++c) {
        if (its[c] >= max_iter) live[c] = 0;
        more |= live[c] != 0;
      }
      if (!more) break;
      std::vector<cd> rho_new(nrhs);
      dotc(rt, w, rho_new);
      for (int64_t c = 0; c < nrhs; ++c) {
        beta[c] = live[c] ? rho_new[c] / rho[c] : cd(0);
        if (live[c]) rho[c] = rho_new[c];
      }
      axpby(w, beta, y2, y1);  // y1 = w + beta y2
      applyA(y1, Ay1);
      axpby(Ay2, beta, v, t);  // t = A y2 + beta v
      axpby(Ay1, beta, t, v);  // v = A y1 + beta t
    }
    bool progressed = false;
    for (int64_t c = 0; c < nrhs; ++c) progressed |= its[c] > its0[c];
    if (!progressed) break;  // breakdown before any step
  }
  pres(t);
  norms(t, nr);
  converged_all = true;
  for (int64_t c = 0; c < nrhs; ++c) {
    prel[c] = nmb[c] > 0 ? nr[c] / nmb[c] : 0.0;
    converged_all &= prel[c] <= rtol;
  }
  if (relres_out) {  // true residual ||b - Z x|| / ||b||
    std::vector<double> nbv(nrhs);
    norms(b, nbv);
    op_apply(h, VIE_OP_Z, x, t2, nrhs, VIE_C128, s);
    sub<<<G, 256, 0, s>>>(b, t2, t2, nb);
    norms(t2, nr);
    for (int64_t c = 0; c < nrhs; ++c) relres_out[c] = nbv[c] > 0 ? nr[c] / nbv[c] : 0.0;
  }
  if (iters_out)
    for (int64_t c = 0; c < nrhs; ++c) iters_out[c] = its[c];
  VIE_CUDA(cudaMemcpyAsync(x_out, x, sizeof(double2) * nb, cudaMemcpyDeviceToDevice, s));
  VIE_CUDA(cudaStreamSynchronize(s));
}

}  // namespace vie
