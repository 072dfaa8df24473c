// HOD-BF apply: batched block-sparse complex products, one launch per stage.
//
// A HOD-BF operator (Sec. III-A, Fig. 1) applied to x in cluster-tree order is
//   y_tau = D_tau x_tau + sum over levels of B_tau x_sibling,
// and every butterfly B = B^L W^L ... W^1 V^0 (Eq. 9) is a chain of
// block-diagonal factors whose blocks are small dense matrices of uneven
// sizes (the butterfly ranks).  The apply therefore is a short sequence of
// stages; stage k multiplies, for every butterfly at once, all its factor-k
// blocks with slices of the previous stage's coefficient vectors.  All blocks
// of a stage are independent, so one launch per stage streams that stage's
// factor bytes once from HBM:
//   * blocks are stored row-major, rows padded to 16 bytes, in one buffer per stage;
//   * work is cut into warp tiles of rows of one block; g lanes (a power of two)
//     share a row, each lane streaming 16-byte vectors (two c64 or one c128
//     entries) with coalesced loads; the g partial sums meet by warp shuffles
//     and one lane writes the output (no atomics: every output row belongs to
//     exactly one tile per stage, so results are deterministic);
//   * coefficient vectors (small, L2 resident) are read through the read-only path.
#include "internal.h"

namespace vie {

template <class T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

// Accumulate row . x for a row of K entries starting at A (row-major), lanes li..g.
template <class TM, class TV, int NR>
__device__ __forceinline__ void row_dot(const typename C2<TM>::type* __restrict__ A, int K, int li, int g,
                                        const typename C2<TV>::type* __restrict__ x, int nrhs,
                                        TV (&acc_re)[NR], TV (&acc_im)[NR]);

template <>
__device__ __forceinline__ void row_dot<float, float, 1>(const float2* __restrict__ A, int K, int li, int g,
                                                          const float2* __restrict__ x, int nrhs,
                                                          float (&re)[1], float (&im)[1]) {
  // four independent 16-byte loads in flight per lane (memory-level parallelism)
  const float4* A4 = reinterpret_cast<const float4*>(A);
  constexpr int U = 4;
  for (int k0 = 2 * li; k0 < K; k0 += 2 * g * U) {
    float4 a[U];
    float2 x0[U], x1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + 2 * g * u;
      if (k < K) {
        a[u] = __ldcs(A4 + (k >> 1));
        x0[u] = __ldg(x + k);
        x1[u] = (k + 1 < K) ? __ldg(x + k + 1) : make_float2(0.f, 0.f);
      } else {
        a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        x0[u] = x1[u] = make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      re[0] = fmaf(a[u].x, x0[u].x, re[0]); re[0] = fmaf(-a[u].y, x0[u].y, re[0]);
      im[0] = fmaf(a[u].x, x0[u].y, im[0]); im[0] = fmaf(a[u].y, x0[u].x, im[0]);
      re[0] = fmaf(a[u].z, x1[u].x, re[0]); re[0] = fmaf(-a[u].w, x1[u].y, re[0]);
      im[0] = fmaf(a[u].z, x1[u].y, im[0]); im[0] = fmaf(a[u].w, x1[u].x, im[0]);
    }
  }
}

template <int NR>
__device__ __forceinline__ void row_dot_c64_multi(const float2* __restrict__ A, int K, int li, int g,
                                                  const float2* __restrict__ x, int nrhs, float (&re)[NR],
                                                  float (&im)[NR]) {
  const float4* A4 = reinterpret_cast<const float4*>(A);
  for (int k = 2 * li; k < K; k += 2 * g) {
    float4 a = __ldcs(A4 + (k >> 1));
    const float2* x0 = x + (int64_t)k * nrhs;
    const bool two = k + 1 < K;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      float2 u = __ldg(x0 + j);
      float2 v = two ? __ldg(x0 + nrhs + j) : make_float2(0.f, 0.f);
      re[j] = fmaf(a.x, u.x, re[j]); re[j] = fmaf(-a.y, u.y, re[j]);
      im[j] = fmaf(a.x, u.y, im[j]); im[j] = fmaf(a.y, u.x, im[j]);
      re[j] = fmaf(a.z, v.x, re[j]); re[j] = fmaf(-a.w, v.y, re[j]);
      im[j] = fmaf(a.z, v.y, im[j]); im[j] = fmaf(a.w, v.x, im[j]);
    }
  }
}

// generic (any factor / vector precision, any rhs chunk): one complex entry per step
template <class TM, class TV, int NR>
__device__ __forceinline__ void row_dot_generic(const typename C2<TM>::type* __restrict__ A, int K, int li, int g,
                                                const typename C2<TV>::type* __restrict__ x, int nrhs,
                                                TV (&re)[NR], TV (&im)[NR]) {
  for (int k = li; k < K; k += g) {
    typename C2<TM>::type a = A[k];
    const TV ar = TV(a.x), ai = TV(a.y);
    const typename C2<TV>::type* xk = x + (int64_t)k * nrhs;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      typename C2<TV>::type u = __ldg(xk + j);
      re[j] += ar * u.x - ai * u.y;
      im[j] += ar * u.y + ai * u.x;
    }
  }
}

// Single right-hand side, c64 factors and vectors: the bandwidth-bound hot path.
// U = 16-byte factor loads a lane keeps in flight (4, or 8 at lower occupancy).
template <int U>
__global__ void __launch_bounds__(256, U == 4 ? 5 : 3) stage1_kernel(const OpDesc* __restrict__ ops,
                                                                     const Tile* __restrict__ tiles, int64_t ntiles,
                                                                     const float2* __restrict__ mats, const float2* xt,
                                                                     float2* yt, float2* coef) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp0; t < ntiles; t += nwarps) {
    const Tile tl = tiles[t];
    const OpDesc& op = ops[tl.op];
    const int K = op.K, M = op.M, ld = op.ld;
    const int g = tl.g, rp = 32 / g;
    const int li = lane & (g - 1);
    const float2* x = (op.in_space == SP_X ? xt : (op.in_space == SP_Y ? (const float2*)yt : coef)) + op.in_off;
    float2* y = (op.out_space == SP_Y ? yt : (op.out_space == SP_X ? const_cast<float2*>(xt) : coef)) + op.out_off;
    const float4* A4 = reinterpret_cast<const float4*>(mats + op.mat_off);
    const bool acc_mode = op.accumulate != 0;
    for (int r = tl.r0 + lane / g; r < tl.r0 + tl.nr; r += rp) {
      float re = 0.f, im = 0.f;
      if (r < M) {
        const float4* row = A4 + ((int64_t)r * ld >> 1);
        for (int k0 = 2 * li; k0 < K; k0 += 2 * U * g) {
          float4 a[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int k = k0 + 2 * g * u;
            a[u] = k < K ? __ldcs(row + (k >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int k = k0 + 2 * g * u;
            if (k < K) {
              const float2 x0 = __ldg(x + k);
              const float2 x1 = (k + 1 < K) ? __ldg(x + k + 1) : make_float2(0.f, 0.f);
              re = fmaf(a[u].x, x0.x, re); re = fmaf(-a[u].y, x0.y, re);
              im = fmaf(a[u].x, x0.y, im); im = fmaf(a[u].y, x0.x, im);
              re = fmaf(a[u].z, x1.x, re); re = fmaf(-a[u].w, x1.y, re);
              im = fmaf(a[u].z, x1.y, im); im = fmaf(a[u].w, x1.x, im);
            }
          }
        }
      }
      for (int o = g >> 1; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (r < M && li == 0) {
        if (acc_mode) {
          float2 v = y[r];
          y[r] = make_float2(v.x + re, v.y + im);
        } else {
          y[r] = make_float2(re, im);
        }
      }
    }
  }
}

// Single right-hand side, c64, with the factor tiles staged in shared memory:
// each CTA walks its tiles through a ring of kBulkSlots slots, one bulk
// asynchronous copy (cp.async.bulk, completion counted on the slot's mbarrier)
// per tile, issued kBulkSlots tiles ahead.  Every SM then keeps about
// 2 x 96 KB of factor reads in flight regardless of how many warps are busy
// with arithmetic, and 16 warps per CTA read their rows from shared memory
// with four coefficient-pair loads in flight per lane.  Same tiles, lanes per
// row and output ownership as stage1_kernel (a tile's rows are contiguous in
// the stage buffer, at most kBulkSlotBytes long).  Waits are bounded: a CTA
// that gives up sets *err, waits (bounded) for its copies in flight and
// returns.
constexpr int kBulkSlots = 3;
constexpr int kBulkSlotBytes = 32768;
constexpr int kBulkThreads = 512;
constexpr uint32_t kBulkSpin = 1u << 24;

__device__ __forceinline__ uint32_t bulk_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bulk_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kBulkSpin; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(kBulkThreads, 2) stage1_bulk_kernel(const OpDesc* __restrict__ ops,
                                                                      const Tile* __restrict__ tiles, int64_t ntiles,
                                                                      const float2* __restrict__ mats,
                                                                      const float2* xt, float2* yt, float2* coef,
                                                                      int* err) {
  extern __shared__ __align__(128) uint8_t bulk_smem[];
  __shared__ __align__(8) uint64_t full[kBulkSlots];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int q = 0; q < kBulkSlots; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bulk_smem_u32(&full[q])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  auto issue = [&](int64_t i) {  // thread 0: copy the rows of this CTA's i-th tile into slot i % kBulkSlots
    const int64_t t = blockIdx.x + i * gridDim.x;
    if (t >= ntiles) return;
    const Tile tl = tiles[t];
    const OpDesc& op = ops[tl.op];
    const int rows = min(tl.nr, op.M - tl.r0);
    const uint32_t bytes = (uint32_t)rows * (uint32_t)op.ld * 8u;
    const float2* src = mats + op.mat_off + (int64_t)tl.r0 * op.ld;
    const int slot = (int)(i % kBulkSlots);
    const uint32_t bar = bulk_smem_u32(&full[slot]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(bulk_smem_u32(bulk_smem + slot * kBulkSlotBytes)), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
  };
  if (tid == 0)
    for (int q = 0; q < kBulkSlots; ++q) issue(q);
  bool ok = true;
  int64_t i = 0;
  for (;; ++i) {
    const int64_t t = blockIdx.x + i * gridDim.x;
    if (t >= ntiles) break;
    const int slot = (int)(i % kBulkSlots);
    ok = __syncthreads_and(bulk_wait(bulk_smem_u32(&full[slot]), (uint32_t)((i / kBulkSlots) & 1)) ? 1 : 0) != 0;
    if (!ok) break;
    const Tile tl = tiles[t];
    const OpDesc& op = ops[tl.op];
    const int K = op.K, ld = op.ld;
    const int rows = min(tl.nr, op.M - tl.r0);
    const int g = tl.g, rp = 32 / g;
    const int li = lane & (g - 1);
    const float2* x = (op.in_space == SP_X ? xt : (op.in_space == SP_Y ? (const float2*)yt : coef)) + op.in_off;
    float2* y = (op.out_space == SP_Y ? yt : (op.out_space == SP_X ? const_cast<float2*>(xt) : coef)) + op.out_off +
                tl.r0;
    const bool acc_mode = op.accumulate != 0;
    const float4* A4 = reinterpret_cast<const float4*>(bulk_smem + slot * kBulkSlotBytes);
    constexpr int nwarps = kBulkThreads / 32;
    for (int rb = warp * rp; rb < rows; rb += nwarps * rp) {  // warp-uniform bound: every lane joins the shuffles
      const int r = rb + lane / g;
      float re = 0.f, im = 0.f;
      if (r < rows) {
        const float4* row = A4 + (int64_t)r * (ld >> 1);
        for (int k0 = 2 * li; k0 < K; k0 += 8 * g) {  // four coefficient pairs in flight per lane
          float2 x0[4], x1[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = k0 + 2 * g * u;
            x0[u] = k < K ? __ldg(x + k) : make_float2(0.f, 0.f);
            x1[u] = k + 1 < K ? __ldg(x + k + 1) : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int k = k0 + 2 * g * u;
            if (k < K) {
              const float4 a = row[k >> 1];
              re = fmaf(a.x, x0[u].x, re); re = fmaf(-a.y, x0[u].y, re);
              im = fmaf(a.x, x0[u].y, im); im = fmaf(a.y, x0[u].x, im);
              re = fmaf(a.z, x1[u].x, re); re = fmaf(-a.w, x1[u].y, re);
              im = fmaf(a.z, x1[u].y, im); im = fmaf(a.w, x1[u].x, im);
            }
          }
        }
      }
      for (int o = g >> 1; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (r < rows && li == 0) {
        if (acc_mode) {
          const float2 v = y[r];
          y[r] = make_float2(v.x + re, v.y + im);
        } else {
          y[r] = make_float2(re, im);
        }
      }
    }
    __syncthreads();  // the slot is consumed
    if (tid == 0) issue(i + kBulkSlots);
  }
  if (!ok && tid == 0) {  // let the copies in flight land before the CTA exits
    for (int64_t q = i; q < i + kBulkSlots; ++q)
      if (blockIdx.x + q * gridDim.x < ntiles)
        bulk_wait(bulk_smem_u32(&full[q % kBulkSlots]), (uint32_t)((q / kBulkSlots) & 1));
    atomicExch(err, 1);
  }
}

// The bulk kernel's tiles must each fit one slot and start on 16 bytes.
bool bulk_tiles_fit(const std::vector<OpDesc>& ops, const std::vector<Tile>& tiles) {
  for (const Tile& t : tiles) {
    const OpDesc& o = ops[t.op];
    const int64_t rows = std::min(t.nr, o.M - t.r0);
    if (rows * (int64_t)o.ld * 8 > kBulkSlotBytes || (o.ld & 1) || (o.mat_off & 1)) return false;
    if (rows * (int64_t)o.ld == 0) return false;  // blocks with no columns (zero rows of a product-built factor)
  }
  return true;
}

void launch_bulk(const Stage& st, const Tile* tiles, int64_t ntiles, const void* xt, void* yt, void* coef, int* err,
                 cudaStream_t s) {
  ensure_smem_attr((const void*)stage1_bulk_kernel, kBulkSlots * kBulkSlotBytes);
  const int grid = (int)std::min<int64_t>(ntiles, 152 * 2);
  stage1_bulk_kernel<<<grid, kBulkThreads, kBulkSlots * kBulkSlotBytes, s>>>(
      st.ops.as<OpDesc>(), tiles, ntiles, st.mats.as<float2>(), (const float2*)xt, (float2*)yt, (float2*)coef, err);
  VIE_CUDA(cudaGetLastError());
}

template <class TM, class TV, int NR>
__global__ void __launch_bounds__(256) stage_kernel(const OpDesc* __restrict__ ops, const Tile* __restrict__ tiles,
                                                    int64_t ntiles, const typename C2<TM>::type* __restrict__ mats,
                                                    const typename C2<TV>::type* xt, typename C2<TV>::type* yt,
                                                    typename C2<TV>::type* coef, int nrhs, int rhs0) {
  using V2 = typename C2<TV>::type;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp0; t < ntiles; t += nwarps) {
    const Tile tl = tiles[t];
    const OpDesc op = ops[tl.op];
    const int g = tl.g, rp = 32 / g;
    const int li = lane & (g - 1);
    const V2* xin = (op.in_space == SP_X ? xt : (op.in_space == SP_Y ? (const V2*)yt : coef)) + op.in_off * nrhs + rhs0;
    V2* yout = (op.out_space == SP_Y ? yt : (op.out_space == SP_X ? const_cast<V2*>(xt) : coef)) + op.out_off * nrhs +
               rhs0;
    for (int r = tl.r0 + lane / g; r < tl.r0 + tl.nr; r += rp) {
      const bool active = r < op.M;
      TV re[NR], im[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) { re[j] = TV(0); im[j] = TV(0); }
      if (active) {
        const typename C2<TM>::type* A = mats + op.mat_off + (int64_t)r * op.ld;
        if constexpr (sizeof(TM) == 4 && sizeof(TV) == 4) {
          if constexpr (NR == 1) {
            if (nrhs == 1) row_dot<float, float, 1>(A, op.K, li, g, xin, nrhs, re, im);
            else row_dot_c64_multi<1>(A, op.K, li, g, xin, nrhs, re, im);
          } else {
            row_dot_c64_multi<NR>(A, op.K, li, g, xin, nrhs, re, im);
          }
        } else {
          row_dot_generic<TM, TV, NR>(A, op.K, li, g, xin, nrhs, re, im);
        }
      }
#pragma unroll
      for (int j = 0; j < NR; ++j)
        for (int o = g >> 1; o > 0; o >>= 1) {
          re[j] += __shfl_xor_sync(0xffffffffu, re[j], o);
          im[j] += __shfl_xor_sync(0xffffffffu, im[j], o);
        }
      if (active && li == 0) {
        V2* yr = yout + (int64_t)r * nrhs;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (op.accumulate) {
            V2 v = yr[j];
            v.x += re[j];
            v.y += im[j];
            yr[j] = v;
          } else {
            V2 v;
            v.x = re[j];
            v.y = im[j];
            yr[j] = v;
          }
        }
      }
    }
  }
}

// Grouped SIMT stage: the tiles of one stage of several operators (SimtGroup), any
// column count, in chunks of eight columns with the last chunk masked.  Per column
// the arithmetic is that of stage1_kernel / stage_kernel on the same tiles (same
// lanes per row, the same sequence of fused multiply-adds over k, the same shuffle
// tree), so a grouped apply returns the bits of the per-operator applies.
__global__ void __launch_bounds__(256) group_simt_kernel(const __grid_constant__ SimtGroup grp) {
  constexpr int NR = 8, U = 4;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp0; t < grp.total; t += nwarps) {
    int si = 0;  // the segment (operator) of tile t
    while (si + 1 < grp.n && grp.s[si + 1].begin <= t) ++si;
    const SimtSeg& sg = grp.s[si];
    const Tile tl = sg.tiles[t - sg.begin];
    const OpDesc op = sg.ops[tl.op];
    const int nrhs = sg.nrhs, K = op.K;
    const int g = tl.g, rp = 32 / g;
    const int li = lane & (g - 1);
    const float2* xin = (op.in_space == SP_X ? sg.xt : (op.in_space == SP_Y ? (const float2*)sg.yt : sg.coef)) +
                        op.in_off * nrhs;
    float2* yout = (op.out_space == SP_Y ? sg.yt : (op.out_space == SP_X ? const_cast<float2*>(sg.xt) : sg.coef)) +
                   op.out_off * nrhs;
    for (int c0 = 0; c0 < nrhs; c0 += NR) {
      const int nc = min(NR, nrhs - c0);  // uniform across the warp
      for (int r = tl.r0 + lane / g; r < tl.r0 + tl.nr; r += rp) {
        const bool active = r < op.M;
        float re[NR], im[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) { re[j] = 0.f; im[j] = 0.f; }
        if (active) {
          const float4* row = reinterpret_cast<const float4*>(sg.mats + op.mat_off + (int64_t)r * op.ld);
          for (int k0 = 2 * li; k0 < K; k0 += 2 * U * g) {
            float4 a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int k = k0 + 2 * g * u;
              a[u] = k < K ? __ldcs(row + (k >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int k = k0 + 2 * g * u;
              if (k < K) {
                const float2* x0 = xin + (int64_t)k * nrhs + c0;
                const bool two = k + 1 < K;
#pragma unroll
                for (int j = 0; j < NR; ++j) {
                  if (j < nc) {
                    const float2 v0 = __ldg(x0 + j);
                    const float2 v1 = two ? __ldg(x0 + nrhs + j) : make_float2(0.f, 0.f);
                    re[j] = fmaf(a[u].x, v0.x, re[j]); re[j] = fmaf(-a[u].y, v0.y, re[j]);
                    im[j] = fmaf(a[u].x, v0.y, im[j]); im[j] = fmaf(a[u].y, v0.x, im[j]);
                    re[j] = fmaf(a[u].z, v1.x, re[j]); re[j] = fmaf(-a[u].w, v1.y, re[j]);
                    im[j] = fmaf(a[u].z, v1.y, im[j]); im[j] = fmaf(a[u].w, v1.x, im[j]);
                  }
                }
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < NR; ++j)
          if (j < nc)
            for (int o = g >> 1; o > 0; o >>= 1) {
              re[j] += __shfl_xor_sync(0xffffffffu, re[j], o);
              im[j] += __shfl_xor_sync(0xffffffffu, im[j], o);
            }
        if (active && li == 0) {
          float2* yr = yout + (int64_t)r * nrhs + c0;
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            if (j < nc) {
              if (op.accumulate) {
                const float2 v = yr[j];
                yr[j] = make_float2(v.x + re[j], v.y + im[j]);
              } else {
                yr[j] = make_float2(re[j], im[j]);
              }
            }
          }
        }
      }
    }
  }
}

void simt_launch_group(const SimtGroup& g, cudaStream_t s) {
  if (g.total == 0) return;
  const int grid = (int)std::min<int64_t>((g.total + 7) / 8, 152 * 16);
  group_simt_kernel<<<grid, 256, 0, s>>>(g);
  VIE_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// permutation gather / scatter (cluster-tree order <-> original face order)
// ---------------------------------------------------------------------------
template <class TV>
__global__ void gather_kernel(const int32_t* perm, int64_t n, int nrhs, const typename C2<TV>::type* X, int64_t ldx,
                              typename C2<TV>::type* xt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / nrhs;
    int j = int(e % nrhs);
    xt[e] = X[perm[i] + (int64_t)j * ldx];
  }
}

template <class TV>
__global__ void scatter_kernel(const int32_t* perm, int64_t n, int nrhs, const typename C2<TV>::type* yt,
                               typename C2<TV>::type* Y, int64_t ldy) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / nrhs;
    int j = int(e % nrhs);
    Y[perm[i] + (int64_t)j * ldy] = yt[e];
  }
}

// ---------------------------------------------------------------------------
// matrix packing: c128 source (row- or column-major) -> row-major padded c64/c128
// ---------------------------------------------------------------------------
template <class TM>
__global__ void pack_kernel(const double2* src, const int64_t* src_off, const int32_t* src_ld, const int32_t* colmajor,
                            const int64_t* dst_off, const int32_t* M, const int32_t* K, const int32_t* ld,
                            typename C2<TM>::type* dst) {
  const int i = blockIdx.x;
  const int m = M[i], k = K[i], l = ld[i], sl = src_ld[i];
  const bool cm = colmajor[i] != 0;
  const double2* s = src + src_off[i];
  typename C2<TM>::type* d = dst + dst_off[i];
  for (int64_t e = threadIdx.x; e < (int64_t)m * l; e += blockDim.x) {
    int r = int(e / l), c = int(e % l);
    double2 v = make_double2(0.0, 0.0);
    if (c < k) v = cm ? s[r + (int64_t)c * sl] : s[(int64_t)r * sl + c];
    typename C2<TM>::type o;
    o.x = TM(v.x);
    o.y = TM(v.y);
    d[e] = o;
  }
}

void pack_matrices(const double2* src, const int64_t* d_src_off, const int32_t* d_src_ld, const int32_t* d_src_colmajor,
                   const int64_t* d_dst_off, const int32_t* d_M, const int32_t* d_K, const int32_t* d_ld, int nmat,
                   void* dst, int dst_dtype, cudaStream_t s) {
  if (nmat <= 0) return;
  if (dst_dtype == VIE_C64)
    pack_kernel<float><<<nmat, 256, 0, s>>>(src, d_src_off, d_src_ld, d_src_colmajor, d_dst_off, d_M, d_K, d_ld,
                                            static_cast<float2*>(dst));
  else
    pack_kernel<double><<<nmat, 256, 0, s>>>(src, d_src_off, d_src_ld, d_src_colmajor, d_dst_off, d_M, d_K, d_ld,
                                             static_cast<double2*>(dst));
  VIE_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// tiles: rows of one op per warp tile, about 16 KB of factor data per tile
// ---------------------------------------------------------------------------
void make_tiles(const std::vector<OpDesc>& ops, std::vector<Tile>& tiles) { make_tiles(ops, tiles, 16384, 4); }

void make_tiles(const std::vector<OpDesc>& ops, std::vector<Tile>& tiles, int64_t max_tile_bytes, int vec_target) {
  // g lanes share a row so that each lane streams about `vec_target` 16-byte
  // vectors of the row (fewer shuffle rounds per byte, several loads in flight).
  // Tiles hold up to max_tile_bytes of factor data, less for small stages so that
  // the launch still has enough warps (152 SMs x 48 warps) to keep HBM busy.
  tiles.clear();
  int64_t stage_bytes = 0;
  for (const OpDesc& o : ops) stage_bytes += (int64_t)o.M * o.ld * 8;
  const int64_t tile_bytes = std::max<int64_t>(2048, std::min<int64_t>(max_tile_bytes, stage_bytes / (152 * 48)));
  for (size_t i = 0; i < ops.size(); ++i) {
    const OpDesc& o = ops[i];
    if (o.M <= 0) continue;
    const int per = (o.K + 1) / 2;  // 16-byte vectors per row for c64
    int g = 1;
    while (g < 32 && vec_target * g < per) g <<= 1;
    const int rp = 32 / g;
    const int64_t row_bytes = (int64_t)o.ld * 8;
    const int64_t passes = std::max<int64_t>(1, tile_bytes / std::max<int64_t>(1, row_bytes * rp));
    const int nr = int(std::min<int64_t>(passes * rp, (int64_t)((o.M + rp - 1) / rp) * rp));
    for (int r0 = 0; r0 < o.M; r0 += nr)
      tiles.push_back(Tile{int32_t(i), r0, (std::min(nr, o.M - r0) + rp - 1) / rp * rp, g});
  }
}

template <class TM, class TV>
static void launch_tiles(const Stage& st, const OpDesc* ops, const Tile* tiles, int64_t ntiles, const void* xt,
                         void* yt, void* coef, int nrhs, cudaStream_t s);

template <class TM, class TV>
static void launch_stage(const Stage& st, const void* xt, void* yt, void* coef, int nrhs, int* err, cudaStream_t s) {
  if constexpr (sizeof(TM) == 4 && sizeof(TV) == 4) {
    if (nrhs == 1 && st.kernel == kKernelBulk && st.ntiles > 0) {
      launch_bulk(st, st.tiles.as<Tile>(), st.ntiles, xt, yt, coef, err, s);
      return;
    }
  }
  launch_tiles<TM, TV>(st, st.ops.as<OpDesc>(), st.tiles.as<Tile>(), st.ntiles, xt, yt, coef, nrhs, s);
}

template <class TM, class TV>
static void launch_tiles(const Stage& st, const OpDesc* ops, const Tile* tiles, int64_t ntiles, const void* xt,
                         void* yt, void* coef, int nrhs, cudaStream_t s) {
  using V2 = typename C2<TV>::type;
  if (ntiles == 0) return;
  int64_t blocks = (ntiles + 7) / 8;
  int grid = (int)std::min<int64_t>(blocks, 152 * 16);
  const typename C2<TM>::type* mats = st.mats.as<typename C2<TM>::type>();
  if constexpr (sizeof(TM) == 4 && sizeof(TV) == 4) {
    if (nrhs == 1) {
      if (st.kernel == kKernelPlain8)
        stage1_kernel<8><<<grid, 256, 0, s>>>(ops, tiles, ntiles, (const float2*)mats, (const float2*)xt, (float2*)yt,
                                              (float2*)coef);
      else
        stage1_kernel<4><<<grid, 256, 0, s>>>(ops, tiles, ntiles, (const float2*)mats, (const float2*)xt, (float2*)yt,
                                              (float2*)coef);
      VIE_CUDA(cudaGetLastError());
      return;
    }
  }
  for (int r0 = 0; r0 < nrhs;) {
    int left = nrhs - r0;
    if (left >= 8) {
      stage_kernel<TM, TV, 8><<<grid, 256, 0, s>>>(ops, tiles, ntiles, mats, (const V2*)xt, (V2*)yt, (V2*)coef, nrhs, r0);
      r0 += 8;
    } else if (left >= 4) {
      stage_kernel<TM, TV, 4><<<grid, 256, 0, s>>>(ops, tiles, ntiles, mats, (const V2*)xt, (V2*)yt, (V2*)coef, nrhs, r0);
      r0 += 4;
    } else if (left >= 2) {
      stage_kernel<TM, TV, 2><<<grid, 256, 0, s>>>(ops, tiles, ntiles, mats, (const V2*)xt, (V2*)yt, (V2*)coef, nrhs, r0);
      r0 += 2;
    } else {
      stage_kernel<TM, TV, 1><<<grid, 256, 0, s>>>(ops, tiles, ntiles, mats, (const V2*)xt, (V2*)yt, (V2*)coef, nrhs, r0);
      r0 += 1;
    }
    VIE_CUDA(cudaGetLastError());
  }
}

template <class TV>
static void run_stages(const Program& p, int64_t nrhs, void* xt, void* yt, void* coef, cudaStream_t s,
                       cudaEvent_t* ev, int& e);

template <class TV>
static void run_program(const Program& p, const int32_t* perm, const void* X, void* Y, int64_t nrhs, int64_t ldx,
                        int64_t ldy, void* xt, void* yt, void* coef, cudaStream_t s, cudaEvent_t* ev,
                        cudaGraphExec_t graph = nullptr) {
  using V2 = typename C2<TV>::type;
  const int64_t tot = p.n * nrhs;
  const int grid = (int)std::min<int64_t>((tot + 255) / 256, 152 * 8);
  int e = 0;
  if (ev) VIE_CUDA(cudaEventRecord(ev[e++], s));
  gather_kernel<TV><<<grid, 256, 0, s>>>(perm, p.n, (int)nrhs, (const V2*)X, ldx, (V2*)xt);
  VIE_CUDA(cudaGetLastError());
  if (ev) VIE_CUDA(cudaEventRecord(ev[e++], s));
  if (graph) VIE_CUDA(cudaGraphLaunch(graph, s));
  else run_stages<TV>(p, nrhs, xt, yt, coef, s, ev, e);
  scatter_kernel<TV><<<grid, 256, 0, s>>>(perm, p.n, (int)nrhs, (const V2*)yt, (V2*)Y, ldy);
  VIE_CUDA(cudaGetLastError());
  if (ev) VIE_CUDA(cudaEventRecord(ev[e++], s));
}

template <class TV>
static void run_stages(const Program& p, int64_t nrhs, void* xt, void* yt, void* coef, cudaStream_t s,
                       cudaEvent_t* ev, int& e) {
  const bool tc = p.tc_ready && sizeof(TV) == 4 && p.factor_dtype == VIE_C64 && nrhs >= p.tc_min_rhs;
  for (const Stage& st : p.stages) {
    if (tc) {
      // dense blocks on the tensor cores, the small ones on the SIMT kernel
      tc_launch(st, xt, yt, coef, (int)nrhs, p.err.as<int>(), s);
      launch_tiles<float, TV>(st, st.rest_ops.as<OpDesc>(), st.rest_tiles.as<Tile>(), st.rest_ntiles, xt, yt, coef,
                              (int)nrhs, s);
    } else if (p.factor_dtype == VIE_C64) {
      launch_stage<float, TV>(st, xt, yt, coef, (int)nrhs, p.err.as<int>(), s);
    } else {
      launch_stage<double, TV>(st, xt, yt, coef, (int)nrhs, p.err.as<int>(), s);
    }
    if (ev) VIE_CUDA(cudaEventRecord(ev[e++], s));
  }
}

void program_apply_graph(Program& p, const int32_t* d_perm, const void* X, void* Y, int64_t nrhs, int64_t ldx,
                         int64_t ldy, int dtype, void* d_xt, void* d_yt, void* d_c, cudaStream_t s) {
  const bool tc = p.tc_ready && dtype == VIE_C64 && p.factor_dtype == VIE_C64 && nrhs >= p.tc_min_rhs;
  Program::GraphEntry* hit = nullptr;
  for (auto& g : p.graphs)
    if (g.exec && g.nrhs == nrhs && g.dtype == dtype && g.tc == tc && g.xt == d_xt && g.yt == d_yt && g.coef == d_c)
      hit = &g;
  if (!hit) {
    if (p.graphs.size() < kGraphCache) {
      p.graphs.emplace_back();
      hit = &p.graphs.back();
    } else {
      hit = &p.graphs[0];
      for (auto& g : p.graphs)
        if (g.used < hit->used) hit = &g;
      if (hit->exec) { cudaGraphExecDestroy(hit->exec); hit->exec = nullptr; }
    }
    if (!p.capture_stream) VIE_CUDA(cudaStreamCreateWithFlags(&p.capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    VIE_CUDA(cudaStreamBeginCapture(p.capture_stream, cudaStreamCaptureModeThreadLocal));
    int e = 0;
    try {
      if (dtype == VIE_C64) run_stages<float>(p, nrhs, d_xt, d_yt, d_c, p.capture_stream, nullptr, e);
      else run_stages<double>(p, nrhs, d_xt, d_yt, d_c, p.capture_stream, nullptr, e);
    } catch (...) {
      cudaStreamEndCapture(p.capture_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    VIE_CUDA(cudaStreamEndCapture(p.capture_stream, &g));
    cudaError_t ie = cudaGraphInstantiate(&hit->exec, g, 0);
    cudaGraphDestroy(g);
    VIE_CUDA(ie);
    hit->nrhs = nrhs; hit->dtype = dtype; hit->tc = tc; hit->xt = d_xt; hit->yt = d_yt; hit->coef = d_c;
  }
  hit->used = ++p.graph_clock;
  if (dtype == VIE_C64) run_program<float>(p, d_perm, X, Y, nrhs, ldx, ldy, d_xt, d_yt, d_c, s, nullptr, hit->exec);
  else run_program<double>(p, d_perm, X, Y, nrhs, ldx, ldy, d_xt, d_yt, d_c, s, nullptr, hit->exec);
}

// Adjoint apply with an adjoint program (program_adjoint): the input goes to the Y
// space, the X space and the coefficients start at zero, the result is read from X.
void program_apply_adjoint(const Program& adj, const int32_t* d_perm, const void* X, void* Y, int64_t nrhs,
                           int64_t ldx, int64_t ldy, int dtype, void* d_xt, void* d_yt, void* d_c, cudaStream_t s) {
  const int64_t tot = adj.n * nrhs;
  const int grid = (int)std::min<int64_t>((tot + 255) / 256, 152 * 8);
  const size_t es = dtype == VIE_C64 ? 8 : 16;
  VIE_CUDA(cudaMemsetAsync(d_xt, 0, es * (size_t)tot, s));
  if (adj.ncoef) VIE_CUDA(cudaMemsetAsync(d_c, 0, es * (size_t)adj.ncoef * nrhs, s));
  int e = 0;
  if (dtype == VIE_C64) {
    gather_kernel<float><<<grid, 256, 0, s>>>(d_perm, adj.n, (int)nrhs, (const float2*)X, ldx, (float2*)d_yt);
    VIE_CUDA(cudaGetLastError());
    run_stages<float>(adj, nrhs, d_xt, d_yt, d_c, s, nullptr, e);
    scatter_kernel<float><<<grid, 256, 0, s>>>(d_perm, adj.n, (int)nrhs, (const float2*)d_xt, (float2*)Y, ldy);
  } else {
    gather_kernel<double><<<grid, 256, 0, s>>>(d_perm, adj.n, (int)nrhs, (const double2*)X, ldx, (double2*)d_yt);
    VIE_CUDA(cudaGetLastError());
    run_stages<double>(adj, nrhs, d_xt, d_yt, d_c, s, nullptr, e);
    scatter_kernel<double><<<grid, 256, 0, s>>>(d_perm, adj.n, (int)nrhs, (const double2*)d_xt, (double2*)Y, ldy);
  }
  VIE_CUDA(cudaGetLastError());
}

void program_run(const Program& p, int64_t nrhs, int dtype, void* xt, void* yt, void* coef, cudaStream_t s) {
  int e = 0;
  if (dtype == VIE_C64) run_stages<float>(p, nrhs, xt, yt, coef, s, nullptr, e);
  else run_stages<double>(p, nrhs, xt, yt, coef, s, nullptr, e);
}

void program_apply(const Program& p, const int32_t* d_perm, const void* X, void* Y, int64_t nrhs, int64_t ldx,
                   int64_t ldy, int dtype, void* d_xt, void* d_yt, void* d_c, cudaStream_t s, cudaEvent_t* ev) {
  if (dtype == VIE_C64) run_program<float>(p, d_perm, X, Y, nrhs, ldx, ldy, d_xt, d_yt, d_c, s, ev);
  else run_program<double>(p, d_perm, X, Y, nrhs, ldx, ldy, d_xt, d_yt, d_c, s, ev);
}

// Single-RHS candidates of the autotuner: 0-8 stage1_kernel<4> with a maximum
// tile of {4, 16, 64} KB x {2, 4, 8} 16-byte vectors per lane (tile index * 3 +
// vector index); 9-11 stage1_bulk_kernel (32 KB tiles) x {2, 4, 8};
// 12-20 stage1_kernel<8> with the tiles of 0-8.
constexpr int kCandidates = 21;

static void candidate(int c, int& kernel, int64_t& tile, int& vec) {
  static const int64_t kTileCand[] = {4096, 16384, 65536};
  static const int kVecCand[] = {2, 4, 8};
  if (c < 9) { kernel = kKernelPlain4; tile = kTileCand[c / 3]; vec = kVecCand[c % 3]; }
  else if (c < 12) { kernel = kKernelBulk; tile = kBulkSlotBytes; vec = kVecCand[c - 9]; }
  else { kernel = kKernelPlain8; tile = kTileCand[(c - 12) / 3]; vec = kVecCand[(c - 12) % 3]; }
}

static void launch_single(const Stage& st, int kernel, const Tile* tiles, int64_t nt, void* xt, void* yt, void* coef,
                          int* err, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((nt + 7) / 8, 152 * 16);
  if (kernel == kKernelBulk) {
    launch_bulk(st, tiles, nt, xt, yt, coef, err, s);
    return;
  }
  if (kernel == kKernelPlain8)
    stage1_kernel<8><<<grid, 256, 0, s>>>(st.ops.as<OpDesc>(), tiles, nt, st.mats.as<float2>(), (const float2*)xt,
                                          (float2*)yt, (float2*)coef);
  else
    stage1_kernel<4><<<grid, 256, 0, s>>>(st.ops.as<OpDesc>(), tiles, nt, st.mats.as<float2>(), (const float2*)xt,
                                          (float2*)yt, (float2*)coef);
  VIE_CUDA(cudaGetLastError());
}

static void ensure_err(Program& p, cudaStream_t s) {
  if (!p.err.p) {
    p.err.alloc(sizeof(int));
    VIE_CUDA(cudaMemsetAsync(p.err.p, 0, sizeof(int), s));
  }
}

// Autotuner of the single-RHS apply: per stage, time every candidate with CUDA
// events (best of two after one warm-up launch) and keep the fastest.
int program_autotune(Program& p, void* xt, void* yt, void* coef, cudaStream_t s, int32_t* choice) {
  if (p.factor_dtype != VIE_C64) return 0;
  ensure_err(p, s);
  cudaEvent_t e0, e1;
  VIE_CUDA(cudaEventCreate(&e0));
  VIE_CUDA(cudaEventCreate(&e1));
  int nst = 0;
  for (Stage& st : p.stages) {
    if (st.host_ops.empty()) { ++nst; continue; }
    float best = 1e30f;
    std::vector<Tile> best_tiles;
    int best_c = 0, best_kernel = kKernelPlain4;
    for (int c = 0; c < kCandidates; ++c) {
      int kernel, vec;
      int64_t tb;
      candidate(c, kernel, tb, vec);
      std::vector<Tile> tiles;
      make_tiles(st.host_ops, tiles, tb, vec);
      if (kernel == kKernelBulk && !bulk_tiles_fit(st.host_ops, tiles)) continue;
      DevBuf dt;
      dt.alloc(sizeof(Tile) * std::max<size_t>(1, tiles.size()));
      VIE_CUDA(cudaMemcpyAsync(dt.p, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, s));
      float tmin = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        VIE_CUDA(cudaEventRecord(e0, s));
        launch_single(st, kernel, dt.as<Tile>(), (int64_t)tiles.size(), xt, yt, coef, p.err.as<int>(), s);
        VIE_CUDA(cudaEventRecord(e1, s));
        VIE_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        VIE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) tmin = std::min(tmin, ms);
      }
      if (tmin < best) { best = tmin; best_tiles = tiles; best_c = c; best_kernel = kernel; }
    }
    st.tiles.alloc(sizeof(Tile) * std::max<size_t>(1, best_tiles.size()));
    VIE_CUDA(cudaMemcpyAsync(st.tiles.p, best_tiles.data(), sizeof(Tile) * best_tiles.size(), cudaMemcpyHostToDevice, s));
    st.ntiles = (int64_t)best_tiles.size();
    st.kernel = best_kernel;
    if (choice) choice[nst] = best_c;
    ++nst;
  }
  VIE_CUDA(cudaStreamSynchronize(s));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (auto& g : p.graphs)  // tiles changed
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
  return nst;
}

// Set the single-RHS kernel and tiling of every stage to a given candidate.
void program_set_tiling(Program& p, const int32_t* choice, int n, cudaStream_t s) {
  VIE_REQUIRE(p.factor_dtype == VIE_C64, VIE_EINVAL, "tiling choices apply to c64 factors");
  VIE_REQUIRE(n == (int)p.stages.size(), VIE_EINVAL, "one choice per stage");
  for (int i = 0; i < n; ++i) VIE_REQUIRE(choice[i] >= 0 && choice[i] < kCandidates, VIE_EINVAL, "choice out of range");
  ensure_err(p, s);
  for (int i = 0; i < n; ++i) {
    Stage& st = p.stages[i];
    if (st.host_ops.empty()) continue;
    int kernel, vec;
    int64_t tb;
    candidate(choice[i], kernel, tb, vec);
    std::vector<Tile> tiles;
    make_tiles(st.host_ops, tiles, tb, vec);
    VIE_REQUIRE(kernel != kKernelBulk || bulk_tiles_fit(st.host_ops, tiles), VIE_EINVAL,
                "a tile does not fit the bulk kernel's slot");
    st.tiles.alloc(sizeof(Tile) * std::max<size_t>(1, tiles.size()));
    VIE_CUDA(cudaMemcpyAsync(st.tiles.p, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, s));
    st.ntiles = (int64_t)tiles.size();
    st.kernel = kernel;
  }
  VIE_CUDA(cudaStreamSynchronize(s));
  for (auto& g : p.graphs)
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
}

void program_prepare_tc(Program& p, cudaStream_t s) {
  if (p.tc_ready || p.factor_dtype != VIE_C64) return;
  // keep an existing flag: graphs captured earlier (single-RHS bulk stages) hold its address
  ensure_err(p, s);
  for (Stage& st : p.stages) tc_prepare_stage(st, st.host_ops, p.tc_tf32, s);
  p.tc_ready = true;
}

void program_set_tc_variant(Program& p, bool tf32) {
  if (p.tc_tf32 == tf32) return;
  VIE_CUDA(cudaDeviceSynchronize());  // nothing in flight may still read the tiles
  for (auto& g : p.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  p.graphs.clear();
  for (Stage& st : p.stages) {
    st.tc_tiles.release(); st.tc_ops.release(); st.rest_ops.release(); st.rest_tiles.release();
    st.tc_items = st.tc_bytes = st.rest_ntiles = 0;
  }
  p.tc_ready = false;
  p.tc_tf32 = tf32;
}

int64_t program_launches(const Program& p, int64_t nrhs, int dtype) {
  const bool c64 = dtype == VIE_C64 && p.factor_dtype == VIE_C64;
  const bool tc = p.tc_ready && c64 && nrhs >= p.tc_min_rhs;
  int64_t chunks = 0;
  for (int64_t r = 0; r < nrhs;) {
    int64_t left = nrhs - r;
    r += left >= 8 ? 8 : (left >= 4 ? 4 : (left >= 2 ? 2 : 1));
    ++chunks;
  }
  int64_t n = 2;  // gather, scatter
  for (const Stage& st : p.stages) {
    if (tc) n += (st.tc_items ? 1 : 0) + (st.rest_ntiles ? chunks : 0);
    else n += st.ntiles ? chunks : 0;
  }
  return n;
}

// Crossover between the two multi-RHS paths: time the stages of one apply with
// 2, 4, 8 and 16 columns on the SIMT kernel and on the tensor cores (CUDA
// events, best of two after a warm-up) and keep the smallest column count from
// which the tensor cores are faster for it and every larger candidate.
int program_tune_rhs(Program& p, void* xt, void* yt, void* coef, cudaStream_t s) {
  if (p.factor_dtype != VIE_C64) return p.tc_min_rhs;
  program_prepare_tc(p, s);
  static const int kCand[] = {2, 4, 8, 16};
  constexpr int nc = 4;
  float t_simt[nc], t_tc[nc];
  cudaEvent_t e0, e1;
  VIE_CUDA(cudaEventCreate(&e0));
  VIE_CUDA(cudaEventCreate(&e1));
  const int saved = p.tc_min_rhs;
  try {
    for (int i = 0; i < nc; ++i)
      for (int mode = 0; mode < 2; ++mode) {
        p.tc_min_rhs = mode ? 1 : (1 << 30);
        float tmin = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          int e = 0;
          VIE_CUDA(cudaEventRecord(e0, s));
          run_stages<float>(p, kCand[i], xt, yt, coef, s, nullptr, e);
          VIE_CUDA(cudaEventRecord(e1, s));
          VIE_CUDA(cudaEventSynchronize(e1));
          float ms = 0;
          VIE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (rep > 0) tmin = std::min(tmin, ms);
        }
        (mode ? t_tc : t_simt)[i] = tmin;
      }
  } catch (...) {
    p.tc_min_rhs = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int pick = 2 * kCand[nc - 1];  // the tensor cores never won: only from 32 columns
  for (int i = nc - 1; i >= 0 && t_tc[i] < t_simt[i]; --i) pick = kCand[i];
  p.tc_min_rhs = pick;
  return pick;
}

}  // namespace vie
