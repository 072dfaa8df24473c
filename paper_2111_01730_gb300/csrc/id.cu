// Batched interpolative decomposition (Eq. 7) by column-pivoted Householder QR, FP64
// (or FP32 arithmetic on the FP64 pools, for the inverse's sketches at chi_fact).
//
// For each job, the m x n column-major block A (complex) is factored as
// A P = Q R with Businger-Golub column pivoting; the rank r is the number of
// pivots with |R_kk| > tol |R_11| (reading of "O(chi_con)").  The output is the
// pivot order (the first r entries are the skeleton columns) and the
// interpolation matrix V = [I, R11^-1 R12] P^T (r x n, row-major), so that
// A ~ A(:, skeleton) V.
//
// One CTA per job.  Column norms are downdated after every reflection and
// recomputed from the remaining rows when cancellation has eaten most of them.
#include "internal.h"

namespace vie {

template <class R> struct RC2 { R x, y; };

template <class R> __device__ __forceinline__ RC2<R> ld(const double2& a) { return RC2<R>{R(a.x), R(a.y)}; }
template <class R> __device__ __forceinline__ double2 st(RC2<R> a) { return make_double2(double(a.x), double(a.y)); }
template <class R> __device__ __forceinline__ RC2<R> cmul(RC2<R> a, RC2<R> b) {
  return RC2<R>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class R> __device__ __forceinline__ RC2<R> cconjmul(RC2<R> a, RC2<R> b) {  // conj(a) * b
  return RC2<R>{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <class R> __device__ __forceinline__ R abs2(RC2<R> a) { return a.x * a.x + a.y * a.y; }

template <class R> __device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// R: the arithmetic (double, or float for the sketches of the inverse built at chi_fact,
// six orders of magnitude above FP32 rounding); the pools stay complex FP64.
template <int NT, class R>
__global__ void __launch_bounds__(NT) id_kernel(const IdJob* jobs, double2* Apool, double2* Vpool, int32_t* pivpool,
                                                int32_t* rank_out, double tol_batch) {
  extern __shared__ double smem[];
  const IdJob J = jobs[blockIdx.x];
  const int m = J.m, n = J.n;
  const R tol = R(J.tol > 0.0 ? J.tol : tol_batch);
  const int kmax = min(m, n);
  // layout (bytes, the same for both precisions): norms 2 n x 8, reflector heads kmax x 16, pivots n x 4
  R* cn = reinterpret_cast<R*>(smem);                                          // n
  R* cref = cn + n;                                                            // n
  RC2<R>* rd = reinterpret_cast<RC2<R>*>(smem + 2 * n);                        // kmax
  int* pv = reinterpret_cast<int*>(reinterpret_cast<double2*>(smem + 2 * n) + kmax);  // n
  __shared__ R s_wv[NT / 32];
  __shared__ int s_wi[NT / 32];
  __shared__ R s_nrm, s_vn2;
  __shared__ int s_p;
  double2* a = Apool + J.a_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT / 32;

  for (int j = warp; j < n; j += nw) {
    R s = 0;
    for (int i = lane; i < m; i += 32) s += abs2(ld<R>(a[i + (int64_t)j * m]));
    s = warp_sum(s);
    if (!isfinite(s)) s = R(-1);  // a non-finite column is never a pivot (and ends the ID below)
    if (lane == 0) { cn[j] = s; cref[j] = s; pv[j] = j; }
  }
  __syncthreads();
  int r = kmax;
  R R00 = 0;
  for (int i = 0; i < kmax; ++i) {
    // pivot: largest remaining column norm (ties: lowest index)
    R bv = R(-1);
    int bi = n;
    for (int j = i + tid; j < n; j += NT)
      if (cn[j] > bv) { bv = cn[j]; bi = j; }
    for (int o = 16; o > 0; o >>= 1) {
      R ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_wv[warp] = bv; s_wi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      R v = s_wv[0];
      int k = s_wi[0];
      for (int w = 1; w < nw; ++w)
        if (s_wv[w] > v || (s_wv[w] == v && s_wi[w] < k)) { v = s_wv[w]; k = s_wi[w]; }
      s_p = k;
    }
    __syncthreads();
    const int p = s_p;
    if (p >= n || !(cn[p] >= R(0))) { r = i; break; }  // no valid pivot left (non-finite input)
    // exact norm of the pivot column over rows i..m-1
    if (warp == 0) {
      R s = 0;
      for (int k = i + lane; k < m; k += 32) s += abs2(ld<R>(a[k + (int64_t)p * m]));
      s = warp_sum(s);
      if (lane == 0) s_nrm = sqrt(s);
    }
    __syncthreads();
    const R nrm = s_nrm;
    if (i == 0) R00 = nrm;
    if (!(nrm > tol * R00) || nrm == R(0) || !isfinite(nrm)) { r = i; break; }
    // swap columns i and p
    if (p != i) {
      for (int k = tid; k < m; k += NT) {
        double2 t = a[k + (int64_t)i * m];
        a[k + (int64_t)i * m] = a[k + (int64_t)p * m];
        a[k + (int64_t)p * m] = t;
      }
      if (tid == 0) {
        R t = cn[i]; cn[i] = cn[p]; cn[p] = t;
        t = cref[i]; cref[i] = cref[p]; cref[p] = t;
        int q = pv[i]; pv[i] = pv[p]; pv[p] = q;
      }
    }
    __syncthreads();
    // Householder reflector for column i: H x = alpha e1, alpha = -exp(j arg x0) |x|
    if (tid == 0) {
      const RC2<R> x0 = ld<R>(a[i + (int64_t)i * m]);
      const R ax0 = sqrt(abs2(x0));
      const RC2<R> ph = ax0 > R(0) ? RC2<R>{x0.x / ax0, x0.y / ax0} : RC2<R>{R(1), R(0)};
      const RC2<R> alpha{-ph.x * nrm, -ph.y * nrm};
      rd[i] = alpha;
      s_vn2 = R(2) * nrm * nrm + R(2) * nrm * ax0;  // v^H v
      a[i + (int64_t)i * m] = st<R>(RC2<R>{x0.x - alpha.x, x0.y - alpha.y});
    }
    __syncthreads();
    const R inv = s_vn2 > R(0) ? R(2) / s_vn2 : R(0);
    const double2* v = a + (int64_t)i * m;
    for (int j = i + 1 + warp; j < n; j += nw) {
      double2* col = a + (int64_t)j * m;
      R wr = 0, wi = 0;
      for (int k = i + lane; k < m; k += 32) {
        const RC2<R> t = cconjmul(ld<R>(v[k]), ld<R>(col[k]));
        wr += t.x; wi += t.y;
      }
      wr = warp_sum(wr);
      wi = warp_sum(wi);
      const RC2<R> f{wr * inv, wi * inv};
      for (int k = i + lane; k < m; k += 32) {
        const RC2<R> t = cmul(ld<R>(v[k]), f);
        RC2<R> c = ld<R>(col[k]);
        c.x -= t.x;
        c.y -= t.y;
        col[k] = st<R>(c);
      }
      __syncwarp();
      // downdate the norm of the remaining rows i+1..m-1
      R nn = cn[j] - abs2(ld<R>(col[i]));
      if (nn <= R(1e-4) * cref[j]) {
        R s = 0;
        for (int k = i + 1 + lane; k < m; k += 32) s += abs2(ld<R>(col[k]));
        nn = warp_sum(s);
        if (lane == 0) cref[j] = nn;
      }
      if (lane == 0) cn[j] = fmax(nn, R(0));
      __syncwarp();
    }
    __syncthreads();
  }
  // T = R11^-1 R12, in place in rows 0..r-1 of columns r..n-1
  for (int c = r + tid; c < n; c += NT) {
    double2* col = a + (int64_t)c * m;
    for (int k = r - 1; k >= 0; --k) {
      RC2<R> t = ld<R>(col[k]);
      for (int l = k + 1; l < r; ++l) {
        const RC2<R> u = cmul(ld<R>(a[k + (int64_t)l * m]), ld<R>(col[l]));
        t.x -= u.x; t.y -= u.y;
      }
      const RC2<R> d = rd[k];
      const R dd = abs2(d);
      col[k] = st<R>(RC2<R>{(t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd});
    }
  }
  __syncthreads();
  double2* V = Vpool + J.v_off;
  for (int64_t e = tid; e < (int64_t)r * n; e += NT) {
    int k = int(e / n), c = int(e % n);
    V[(int64_t)k * n + pv[c]] = c < r ? make_double2(c == k ? 1.0 : 0.0, 0.0) : a[k + (int64_t)c * m];
  }
  int32_t* po = pivpool + J.p_off;
  for (int c = tid; c < n; c += NT) po[c] = pv[c];
  if (tid == 0) rank_out[blockIdx.x] = r;
}

void id_batched(const IdJob* d_jobs, int njobs, int max_n, double2* d_a, double2* d_v, int32_t* d_piv,
                int32_t* d_rank, double tol, cudaStream_t s, bool single) {
  if (njobs <= 0) return;
  constexpr int NT = 256;
  // shared memory: 2 n reals (norms) within n doubles, kmax <= n complex reflector heads, n ints
  size_t smem = sizeof(double) * 2 * max_n + sizeof(double2) * max_n + sizeof(int) * max_n + 64;
  VIE_REQUIRE(smem <= 200 * 1024, VIE_ENOTSUP, "ID block too wide for shared memory");
  if (single) {
    VIE_CUDA(cudaFuncSetAttribute((const void*)id_kernel<NT, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    id_kernel<NT, float><<<njobs, NT, smem, s>>>(d_jobs, d_a, d_v, d_piv, d_rank, tol);
  } else {
    VIE_CUDA(cudaFuncSetAttribute((const void*)id_kernel<NT, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    id_kernel<NT, double><<<njobs, NT, smem, s>>>(d_jobs, d_a, d_v, d_piv, d_rank, tol);
  }
  VIE_CUDA(cudaGetLastError());
}

}  // namespace vie
