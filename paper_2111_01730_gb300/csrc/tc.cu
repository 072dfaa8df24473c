// Multi-RHS HOD-BF apply on the 5th-generation tensor cores (tcgen05, TMEM).
//
// With many right-hand sides every stage block Y_blk = A X_blk (A: M x K complex)
// is a dense contraction.  It runs transposed, Y^T (nrhs x M) = X^T (nrhs x K) A^T,
// so that the MMA's M dimension (128) is the right-hand-side count and the
// butterfly rank M only sets the MMA's N (a multiple of 16).  The complex
// product is split into four real products (the 4M form),
//   Yr^T = Xr^T Ar^T - Xi^T Ai^T,   Yi^T = Xr^T Ai^T + Xi^T Ar^T,
// with the minus sign carried by the instruction's negate-A bit, and each real
// product runs as three BF16 products with FP32 accumulation in TMEM
// (a = a_hi + a_lo, a_hi b_hi + a_hi b_lo + a_lo b_hi), which keeps about 16
// mantissa bits of the FP32 factors.
//
// Data movement: the factor blocks of the operator are packed once into
// per-(block, 128-row chunk, 32-column chunk) tiles of [Ar_hi|Ar_lo|Ai_hi|Ai_lo]
// bf16 in the canonical no-swizzle K-major core-matrix layout and copied into
// shared memory with one bulk asynchronous copy (cp.async.bulk, completion on an
// mbarrier) per k-chunk; the coefficient vectors X are converted to the same
// layout by the CTA's threads.  Four CTAs per SM (49 KB of shared memory and
// 128 TMEM columns each) overlap one another's copies, conversions and MMAs.
// One thread issues the MMAs; eight warps drain TMEM with tcgen05.ld.
// Blocks too small to fill a tile stay on the SIMT path (stage_kernel).
//
// TF32 variant (VIE_P_TC_TF32): the same tiles hold [Ar | Ai] and [Xr | Xi] as
// FP32 values rounded to TF32 (10 mantissa bits, round to nearest), in the same
// core-matrix layout with 4-byte elements, and each real product is one
// kind::tf32 MMA (K = 8 per instruction): 4 MMAs per 8 columns of K instead of
// 12 per 16, at half the BF16 rate, so about 1.5x less tensor time for about
// 11 instead of 16 mantissa bits.
//
// Every wait on an mbarrier is bounded; a CTA that gives up records the event in
// an error flag that the host reads after the apply.
#include <cuda_bf16.h>

#include <map>
#include <tuple>

#include "internal.h"

namespace vie {

namespace {

constexpr int kKc = 32;        // complex columns (K) per chunk
constexpr int kRows = 128;     // right-hand sides per MMA (M of the instruction)
constexpr int kMaxN = 64;      // output rows per work item (N of the instruction)
constexpr int kTmemCols = 2 * kMaxN;  // D_r and D_i
constexpr int kThreads = 256;  // eight warps; warp w drains TMEM lane quarter w % 4
constexpr int kTileA = 4 * kRows * kKc * 2;   // bytes: Xr_hi, Xr_lo, Xi_hi, Xi_lo (32 KB)
constexpr int kTileBMax = 4 * kMaxN * kKc * 2;  // 16 KB
constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// canonical K-major no-swizzle layout: element (r, k) of an R x 32 tile; a core
// matrix is 8 rows x 16 bytes (8 bf16 or 4 tf32), core matrices run along K first
__device__ __forceinline__ int cm_index(int r, int k) { return ((r >> 3) * (kKc / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }
__device__ __forceinline__ int cm_index32(int r, int k) { return ((r >> 3) * (kKc / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

template <bool TF32>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // start address, leading byte offset (next core matrix along K) = 128 B, stride byte
  // offset (next 8-row group) = the core matrices of one 32-column row: 4 x 128 B for
  // bf16, 8 x 128 B for tf32; version 1, no swizzle
  constexpr uint32_t sbo = TF32 ? 1024 : 512;
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(sbo >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

template <bool TF32>
__device__ __forceinline__ uint32_t instr_desc(int n, int neg_a) {
  constexpr uint32_t fmt = TF32 ? 2u : 1u;  // operand format: BF16 (kind::f16) or TF32 (kind::tf32)
  uint32_t d = 0;
  d |= 1u << 4;     // accumulate in F32
  d |= fmt << 7;    // A
  d |= fmt << 10;   // B
  d |= (uint32_t)neg_a << 13;
  d |= (uint32_t)(n >> 3) << 17;
  d |= (uint32_t)(kRows >> 4) << 24;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t taddr, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               :: "r"(taddr), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_tf32(uint32_t taddr, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
               :: "r"(taddr), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// FP32 -> TF32 bit pattern, round to nearest (ties away from zero)
__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
  return u;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

}  // namespace

// ---------------------------------------------------------------------------
// packing: c64 row-major block rows [m0, m0+Mc) -> bf16 tiles per 32-column chunk
// ---------------------------------------------------------------------------
__device__ __forceinline__ int seg_of(const TcItem& it, int m) {
  int sgi = 0;
  for (int q = 1; q < it.nseg; ++q)
    if (m >= it.seg[q].start) sgi = q;
  return sgi;
}

// TF32 tiles: [Ar | Ai] per k-chunk, FP32 rounded to TF32, 4-byte core-matrix layout
__global__ void tc_pack_tf32_kernel(const TcItem* items, int nitems, const float2* mats, uint32_t* out) {
  const TcItem& it = items[blockIdx.x];
  const int nk = (it.K + kKc - 1) / kKc;
  const int64_t tile = (int64_t)2 * it.n * kKc;  // 4-byte elements per k-chunk tile
  for (int64_t e = threadIdx.x; e < (int64_t)nk * it.n * kKc; e += blockDim.x) {
    const int kc = int(e / (it.n * kKc));
    const int rem = int(e % (it.n * kKc));
    const int r = rem / kKc, k = rem % kKc;
    const int kk = kc * kKc + k;
    float2 a = make_float2(0.f, 0.f);
    if (r < it.mc && kk < it.K) {
      const TcSeg& sg = it.seg[seg_of(it, r)];
      a = mats[sg.mat_off + (int64_t)(sg.row0 + r - sg.start) * sg.ld + kk];
    }
    uint32_t* t = out + it.b_off / 4 + kc * tile;
    const int ci = cm_index32(r, k);
    t[ci] = to_tf32(a.x);
    t[(int64_t)it.n * kKc + ci] = to_tf32(a.y);
  }
}

__global__ void tc_pack_kernel(const TcItem* items, int nitems, const float2* mats, __nv_bfloat16* out) {
  const TcItem& it = items[blockIdx.x];
  const int nk = (it.K + kKc - 1) / kKc;
  const int64_t tile = (int64_t)4 * it.n * kKc;  // bf16 elements per k-chunk tile
  for (int64_t e = threadIdx.x; e < (int64_t)nk * it.n * kKc; e += blockDim.x) {
    const int kc = int(e / (it.n * kKc));
    const int rem = int(e % (it.n * kKc));
    const int r = rem / kKc, k = rem % kKc;
    const int kk = kc * kKc + k;
    float2 a = make_float2(0.f, 0.f);
    if (r < it.mc && kk < it.K) {
      const TcSeg& sg = it.seg[seg_of(it, r)];
      a = mats[sg.mat_off + (int64_t)(sg.row0 + r - sg.start) * sg.ld + kk];
    }
    __nv_bfloat16 rh, rl, ih, il;
    split_bf16(a.x, rh, rl);
    split_bf16(a.y, ih, il);
    __nv_bfloat16* t = out + it.b_off / 2 + kc * tile;
    const int ci = cm_index(r, k);
    const int64_t part = (int64_t)it.n * kKc;
    t[ci] = rh;
    t[part + ci] = rl;
    t[2 * part + ci] = ih;
    t[3 * part + ci] = il;
  }
}

// ---------------------------------------------------------------------------
// the tensor-core stage kernel (persistent over work items; several CTAs per SM
// interleave their copy / convert / MMA phases)
// ---------------------------------------------------------------------------
template <bool TF32>
__global__ void __launch_bounds__(kThreads, 4) tc_stage_kernel(const __grid_constant__ TcGroup grp) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sA = smem;
  uint8_t* sB = smem + kTileA;
  __shared__ __align__(8) uint64_t load_bar, mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ float2* s_dst[kMaxN];   // output row base (row m of the item, right-hand side 0)
  __shared__ int s_acc[kMaxN];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&load_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mma_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;  // D_r: columns [0, kMaxN), D_i: [kMaxN, 2 kMaxN)
  uint32_t load_phase = 0, mma_phase = 0;
  bool ok = true;
  int* err = grp.s[0].err;
  for (int64_t w = blockIdx.x; w < grp.total && ok; w += gridDim.x) {
    int si = 0;  // the segment (operator) of work index w
    while (si + 1 < grp.n && grp.s[si + 1].begin <= w) ++si;
    const TcSeg2& sgm = grp.s[si];
    err = sgm.err;
    const uint8_t* __restrict__ btiles = sgm.btiles;
    const float2* xt = sgm.xt;
    float2* yt = sgm.yt;
    float2* coef = sgm.coef;
    const int nrhs = sgm.nrhs;
    const int nrc = (nrhs + kRows - 1) / kRows;
    const int64_t lw = w - sgm.begin;
    const TcItem& it = sgm.items[lw / nrc];
    const int r0 = int(lw % nrc) * kRows;
    const int nk = (it.K + kKc - 1) / kKc;
    const float2* x = (it.in_space == SP_X ? xt : (it.in_space == SP_Y ? (const float2*)yt : coef)) +
                      (int64_t)it.in_off * nrhs;
    const uint32_t tile_bytes = 4u * it.n * kKc * 2u;
    if (tid < it.mc) {  // output row pointers of the item, resolved once
      const TcSeg& sg = it.seg[seg_of(it, tid)];
      s_dst[tid] = (sg.out_space == SP_Y ? yt : (sg.out_space == SP_X ? const_cast<float2*>(xt) : coef)) +
                   (sg.out_off + sg.row0 + tid - sg.start) * nrhs;
      s_acc[tid] = sg.accumulate;
    }
    for (int kc = 0; kc < nk && ok; ++kc) {
      if (kc > 0) {  // single buffer: the previous chunk's MMAs must have read it
        ok = mbar_wait(smem_u32(&mma_bar), mma_phase);
        mma_phase ^= 1;
      }
      if (tid == 0 && ok) {
        const uint32_t bar = smem_u32(&load_bar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(tile_bytes) : "memory");
        const uint8_t* src = btiles + it.b_off + (int64_t)kc * tile_bytes;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(sB)), "l"(src), "r"(tile_bytes), "r"(bar) : "memory");
      }
      const int kvalid = min(kKc, it.K - kc * kKc);
      if constexpr (TF32) {
        // X chunk -> [Xr | Xi] TF32 planes: a thread owns (rhs r, 4 consecutive k) and
        // writes one 16-byte row segment of a core matrix per plane
        constexpr int part = kRows * kKc;
        constexpr int groups = kRows * (kKc / 4);
#pragma unroll
        for (int gi = tid; gi < groups; gi += kThreads) {
          const int r = gi % kRows, kg = gi / kRows;
          const int rr = r0 + r;
          float2 v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int k = kg * 4 + j;
            v[j] = (k < kvalid && rr < nrhs) ? __ldg(x + (int64_t)(kc * kKc + k) * nrhs + rr) : make_float2(0.f, 0.f);
          }
          const int ci = cm_index32(r, kg * 4);
          uint4* a4 = reinterpret_cast<uint4*>(sA);
          a4[ci / 4] = make_uint4(to_tf32(v[0].x), to_tf32(v[1].x), to_tf32(v[2].x), to_tf32(v[3].x));
          a4[(part + ci) / 4] = make_uint4(to_tf32(v[0].y), to_tf32(v[1].y), to_tf32(v[2].y), to_tf32(v[3].y));
        }
      } else {
        // X chunk -> bf16 hi/lo tiles (rows = right-hand sides, columns = k).  A thread
        // owns (rhs r, 8 consecutive k): it issues its 8 global loads first, then writes
        // one 16-byte row segment of a core matrix per plane (bank-conflict free).
        constexpr int part = kRows * kKc;  // bf16 elements per plane
        constexpr int groups = kRows * (kKc / 8);  // (rhs, k-group) pairs per chunk
#pragma unroll
        for (int gi = tid; gi < groups; gi += kThreads) {
          const int r = gi % kRows, kg = gi / kRows;  // consecutive threads: consecutive rhs
          const int rr = r0 + r;
          float2 v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int k = kg * 8 + j;
            v[j] = (k < kvalid && rr < nrhs) ? __ldg(x + (int64_t)(kc * kKc + k) * nrhs + rr) : make_float2(0.f, 0.f);
          }
          uint32_t rh[4], rl[4], ih[4], il[4];  // bf16 pairs
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(v[j].x, h0, l0);
            split_bf16(v[j + 1].x, h1, l1);
            rh[j / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            rl[j / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            split_bf16(v[j].y, h0, l0);
            split_bf16(v[j + 1].y, h1, l1);
            ih[j / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            il[j / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
          }
          const int ci = cm_index(r, kg * 8);  // start of the 16-byte row segment
          uint4* a4 = reinterpret_cast<uint4*>(sA);
          a4[ci / 8] = make_uint4(rh[0], rh[1], rh[2], rh[3]);
          a4[(part + ci) / 8] = make_uint4(rl[0], rl[1], rl[2], rl[3]);
          a4[(2 * part + ci) / 8] = make_uint4(ih[0], ih[1], ih[2], ih[3]);
          a4[(3 * part + ci) / 8] = make_uint4(il[0], il[1], il[2], il[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0 && ok) {
        ok = mbar_wait(smem_u32(&load_bar), load_phase);
        load_phase ^= 1;
        if (ok) {
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t A0 = smem_u32(sA), B0 = smem_u32(sB);
          const uint32_t idp = instr_desc<TF32>(it.n, 0), idm = instr_desc<TF32>(it.n, 1);
          const uint32_t Dr = tmem, Di = tmem + kMaxN;
          if constexpr (TF32) {
            const uint32_t pa = (uint32_t)kRows * kKc * 4u, pb = (uint32_t)it.n * kKc * 4u;  // bytes per plane
            const uint32_t Xr = A0, Xi = A0 + pa, Ar = B0, Ai = B0 + pb;
            for (int ks = 0; ks < kKc / 8; ++ks) {
              const uint32_t o = ks * 256;  // two core matrices along K
              const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
              // Dr += Xr Ar - Xi Ai ; Di += Xr Ai + Xi Ar
              mma_tf32(Dr, smem_desc<true>(Xr + o), smem_desc<true>(Ar + o), idp, acc0);
              mma_tf32(Dr, smem_desc<true>(Xi + o), smem_desc<true>(Ai + o), idm, 1);
              mma_tf32(Di, smem_desc<true>(Xr + o), smem_desc<true>(Ai + o), idp, acc0);
              mma_tf32(Di, smem_desc<true>(Xi + o), smem_desc<true>(Ar + o), idp, 1);
            }
          } else {
            const uint32_t pa = (uint32_t)kRows * kKc * 2u, pb = (uint32_t)it.n * kKc * 2u;  // bytes per hi/lo plane
            const uint32_t Xrh = A0, Xrl = A0 + pa, Xih = A0 + 2 * pa, Xil = A0 + 3 * pa;
            const uint32_t Arh = B0, Arl = B0 + pb, Aih = B0 + 2 * pb, Ail = B0 + 3 * pb;
            for (int ks = 0; ks < kKc / 16; ++ks) {
              const uint32_t o = ks * 256;  // two core matrices along K
              const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
              // Dr += Xr Ar - Xi Ai ; Di += Xr Ai + Xi Ar  (each as hi*hi + hi*lo + lo*hi)
              mma_bf16(Dr, smem_desc<false>(Xrh + o), smem_desc<false>(Arh + o), idp, acc0);
              mma_bf16(Dr, smem_desc<false>(Xrh + o), smem_desc<false>(Arl + o), idp, 1);
              mma_bf16(Dr, smem_desc<false>(Xrl + o), smem_desc<false>(Arh + o), idp, 1);
              mma_bf16(Dr, smem_desc<false>(Xih + o), smem_desc<false>(Aih + o), idm, 1);
              mma_bf16(Dr, smem_desc<false>(Xih + o), smem_desc<false>(Ail + o), idm, 1);
              mma_bf16(Dr, smem_desc<false>(Xil + o), smem_desc<false>(Aih + o), idm, 1);
              mma_bf16(Di, smem_desc<false>(Xrh + o), smem_desc<false>(Aih + o), idp, acc0);
              mma_bf16(Di, smem_desc<false>(Xrh + o), smem_desc<false>(Ail + o), idp, 1);
              mma_bf16(Di, smem_desc<false>(Xrl + o), smem_desc<false>(Aih + o), idp, 1);
              mma_bf16(Di, smem_desc<false>(Xih + o), smem_desc<false>(Arh + o), idp, 1);
              mma_bf16(Di, smem_desc<false>(Xih + o), smem_desc<false>(Arl + o), idp, 1);
              mma_bf16(Di, smem_desc<false>(Xil + o), smem_desc<false>(Arh + o), idp, 1);
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       :: "r"(smem_u32(&mma_bar)) : "memory");
        }
      }
      ok = __syncthreads_and(ok ? 1 : 0) != 0;
    }
    if (ok) {  // the last commit covers every MMA of the item
      ok = mbar_wait(smem_u32(&mma_bar), mma_phase);
      mma_phase ^= 1;
    }
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w drains TMEM lanes (right-hand sides) 32 (w % 4) .. +31,
    // warps 0-3 the first half of the output rows, warps 4-7 the second half
    const int rr = r0 + (warp & 3) * 32 + lane;
    const int half = it.n / 2;
    const int cbeg = (warp >> 2) * half;
    for (int c0 = cbeg; c0 < cbeg + half; c0 += 8) {
      uint32_t vr[8], vi[8];
      const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + c0;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]), "=r"(vr[7])
                   : "r"(lane_addr));
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]), "=r"(vi[7])
                   : "r"(lane_addr + kMaxN));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (rr < nrhs) {
        float2 old[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // all reads in flight before the writes
          const int m = c0 + j;
          old[j] = (m < it.mc && s_acc[m]) ? s_dst[m][rr] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int m = c0 + j;
          if (m < it.mc) s_dst[m][rr] = make_float2(old[j].x + __uint_as_float(vr[j]), old[j].y + __uint_as_float(vi[j]));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// failure-path check of the bounded mbarrier wait: wait on a barrier that
// nothing arrives on, with a short spin limit, and report the timeout
// ---------------------------------------------------------------------------
__global__ void wait_timeout_kernel(uint32_t spins, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  uint32_t done = 0;
  for (uint32_t it = 0; it < spins && !done; ++it)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(smem_u32(&bar)), "r"(0) : "memory");
  if (threadIdx.x == 0) *status = done ? 0 : 1;
}

void wait_timeout_check(uint32_t spins, int* d_status, cudaStream_t s) {
  wait_timeout_kernel<<<1, 32, 0, s>>>(spins, d_status);
  VIE_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t tc_smem_bytes() { return (size_t)kTileA + (size_t)kTileBMax + 1024; }

bool tc_eligible(const OpDesc& o) { return o.M >= 16 && o.K >= 32; }

void tc_prepare_stage(Stage& st, const std::vector<OpDesc>& ops, bool tf32, cudaStream_t s) {
  // the shared-memory attribute of both variants, set here (outside any stream capture)
  ensure_smem_attr((const void*)tc_stage_kernel<false>, (int)tc_smem_bytes());
  ensure_smem_attr((const void*)tc_stage_kernel<true>, (int)tc_smem_bytes());
  // Eligible blocks that read the same input slice (the V0 blocks and the leaf block
  // of one leaf; the two W blocks of the children of one node) share work items of
  // up to 64 rows, so each input chunk is converted once for all of them.
  std::map<std::tuple<int, int64_t, int>, std::vector<size_t>> groups;
  for (size_t i = 0; i < ops.size(); ++i)
    if (tc_eligible(ops[i])) groups[{ops[i].in_space, ops[i].in_off, ops[i].K}].push_back(i);
  std::vector<TcItem> items;
  int64_t off = 0;
  for (auto& kv : groups) {
    TcItem t{};
    auto flush = [&]() {
      if (t.mc == 0) return;
      t.n = (t.mc + 15) / 16 * 16;
      t.b_off = off;
      off += (int64_t)((t.K + kKc - 1) / kKc) * 4 * t.n * kKc * 2;  // bf16: 4 planes x 2 B; tf32: 2 planes x 4 B
      items.push_back(t);
      TcItem z{};
      z.in_space = t.in_space; z.in_off = t.in_off; z.K = t.K;
      t = z;
    };
    t.in_space = (int16_t)std::get<0>(kv.first);
    t.in_off = std::get<1>(kv.first);
    t.K = std::get<2>(kv.first);
    for (size_t i : kv.second) {
      const OpDesc& o = ops[i];
      for (int r = 0; r < o.M;) {
        if (t.mc == kMaxN || t.nseg == kTcMaxSeg) flush();
        const int take = std::min(o.M - r, kMaxN - t.mc);
        TcSeg& sg = t.seg[t.nseg++];
        sg.mat_off = o.mat_off; sg.out_off = o.out_off; sg.ld = o.ld; sg.row0 = r; sg.rows = take;
        sg.start = t.mc; sg.out_space = o.out_space; sg.accumulate = (int16_t)o.accumulate;
        t.mc += take;
        r += take;
      }
    }
    flush();
  }
  st.tc_items = (int64_t)items.size();
  st.tc_bytes = off;
  st.tc_tf32 = tf32;
  if (!items.empty()) {
    st.tc_tiles.alloc(off);
    st.tc_ops.alloc(sizeof(TcItem) * items.size());
    VIE_CUDA(cudaMemcpyAsync(st.tc_ops.p, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice, s));
    if (tf32)
      tc_pack_tf32_kernel<<<(int)items.size(), 256, 0, s>>>(st.tc_ops.as<TcItem>(), (int)items.size(),
                                                            st.mats.as<float2>(), st.tc_tiles.as<uint32_t>());
    else
      tc_pack_kernel<<<(int)items.size(), 256, 0, s>>>(st.tc_ops.as<TcItem>(), (int)items.size(), st.mats.as<float2>(),
                                                       st.tc_tiles.as<__nv_bfloat16>());
    VIE_CUDA(cudaGetLastError());
  }
  // the SIMT remainder: ops that are not eligible (a stage may have no eligible op at all)
  std::vector<OpDesc> rest;
  for (const OpDesc& o : ops)
    if (!tc_eligible(o)) rest.push_back(o);
  std::vector<Tile> tiles;
  make_tiles(rest, tiles);
  st.rest_ops.alloc(sizeof(OpDesc) * std::max<size_t>(1, rest.size()));
  st.rest_tiles.alloc(sizeof(Tile) * std::max<size_t>(1, tiles.size()));
  if (!rest.empty())
    VIE_CUDA(cudaMemcpyAsync(st.rest_ops.p, rest.data(), sizeof(OpDesc) * rest.size(), cudaMemcpyHostToDevice, s));
  if (!tiles.empty())
    VIE_CUDA(cudaMemcpyAsync(st.rest_tiles.p, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, s));
  st.rest_ntiles = (int64_t)tiles.size();
  VIE_CUDA(cudaStreamSynchronize(s));
}

void tc_launch_group(const TcGroup& g, cudaStream_t s) {
  if (g.total == 0) return;
  const int grid = (int)std::min<int64_t>(g.total, 152 * 4);  // four CTAs per SM (smem 49 KB, TMEM 128 columns each)
  if (g.tf32) {
    ensure_smem_attr((const void*)tc_stage_kernel<true>, (int)tc_smem_bytes());
    tc_stage_kernel<true><<<grid, kThreads, tc_smem_bytes(), s>>>(g);
  } else {
    ensure_smem_attr((const void*)tc_stage_kernel<false>, (int)tc_smem_bytes());
    tc_stage_kernel<false><<<grid, kThreads, tc_smem_bytes(), s>>>(g);
  }
  VIE_CUDA(cudaGetLastError());
}

int64_t tc_work_units(int64_t items, int nrhs) { return items * ((nrhs + kRows - 1) / kRows); }

void tc_launch(const Stage& st, const void* xt, void* yt, void* coef, int nrhs, int* d_err, cudaStream_t s) {
  if (st.tc_items == 0) return;
  TcGroup g{};
  g.n = 1;
  g.tf32 = st.tc_tf32 ? 1 : 0;
  g.s[0] = TcSeg2{st.tc_ops.as<TcItem>(), st.tc_tiles.as<uint8_t>(), (const float2*)xt, (float2*)yt, (float2*)coef,
                  d_err, 0, (int32_t)st.tc_items, nrhs};
  g.total = tc_work_units(st.tc_items, nrhs);
  tc_launch_group(g, s);
}

}  // namespace vie
