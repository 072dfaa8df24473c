// Sharded apply by subtrees (Sec. III-D): with P GPUs, rank r owns the rows of node r
// at tree level log2 P (a contiguous range of tree positions) and the blocks of the
// apply program those rows depend on.  For Z that is the leaf blocks and butterflies
// rooted in the rank's subtree plus the row-side parts of the upper butterflies that
// end in its rows; their column sides read X anywhere, so every rank takes the whole
// of X (one all-gather across ranks, done by the caller) and writes only its rows of Y.
// The rank's blocks are the dependency closure of its output rows in the program
// (program_restrict_rows), selected on first use and kept with the operator.
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace vie {

namespace {

template <class T>
__global__ void gather_all(const int32_t* perm, int64_t n, int nrhs, const T* X, int64_t ldx, T* xt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * nrhs; e += (int64_t)gridDim.x * blockDim.x)
    xt[e] = X[perm[e / nrhs] + (e % nrhs) * ldx];
}

template <class T>
__global__ void scatter_range(const int32_t* perm, int64_t lo, int64_t hi, int nrhs, const T* yt, T* Y, int64_t ldy) {
  const int64_t cnt = (hi - lo) * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = lo + e / nrhs;
    const int j = int(e % nrhs);
    Y[perm[i] + j * ldy] = yt[i * nrhs + j];
  }
}

}  // namespace

struct ShardCache {
  std::mutex mu;
  std::map<std::tuple<int, int, int>, std::unique_ptr<Program>> progs;
};

static std::mutex g_shard_mu;
static std::map<const vie_op*, std::unique_ptr<ShardCache>> g_shards;

void shard_forget(const vie_op* h) {
  std::lock_guard<std::mutex> lock(g_shard_mu);
  g_shards.erase(h);
}

static void shard_range(const vie_op* h, int rank, int nranks, int64_t& lo, int64_t& hi) {
  VIE_REQUIRE(nranks >= 1 && nranks <= (1 << 20), VIE_EINVAL, "nranks out of range [1, 2^20]");
  int lev = 0;
  while ((1 << lev) < nranks) ++lev;
  VIE_REQUIRE((1 << lev) == nranks, VIE_EINVAL, "nranks must be a power of two");
  VIE_REQUIRE(lev <= h->tree.levels, VIE_EINVAL, "more ranks than leaves of the cluster tree");
  VIE_REQUIRE(rank >= 0 && rank < nranks, VIE_EINVAL, "rank out of range");
  lo = h->tree.bounds[lev][rank];
  hi = h->tree.bounds[lev][rank + 1];
}

}  // namespace vie

using namespace vie;

extern "C" vie_status vie_shard_range(const vie_op* h, int32_t rank, int32_t nranks, int64_t* lo, int64_t* hi) {
  try {
    VIE_REQUIRE(h && lo && hi, VIE_EINVAL, "null argument");
    shard_range(h, rank, nranks, *lo, *hi);
    return VIE_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {  // no exception leaves the C ABI
    set_error(e.what());
    return VIE_EINVAL;
  }
}

extern "C" vie_status vie_apply_shard(vie_op* h, int32_t which, int32_t rank, int32_t nranks, const void* X, void* Y,
                                      int64_t nrhs, int64_t ldx, int64_t ldy, int32_t dtype, void* stream) {
  try {
    VIE_REQUIRE(h && X && Y, VIE_EINVAL, "null argument");
    VIE_REQUIRE(nrhs >= 1 && ldx >= h->mesh.nf && ldy >= h->mesh.nf, VIE_EINVAL, "bad nrhs or leading dimension");
    VIE_REQUIRE(dtype == VIE_C64 || dtype == VIE_C128, VIE_EINVAL, "bad dtype");
    VIE_REQUIRE(which == VIE_OP_Z || which == VIE_OP_ZINV, VIE_EINVAL, "bad operator kind");
    VIE_REQUIRE(which == VIE_OP_Z || h->has_zinv, VIE_ENOTSUP, "operator has no inverse (tol_fact <= 0)");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t lo, hi;
    shard_range(h, rank, nranks, lo, hi);
    ShardCache* cache;
    {
      std::lock_guard<std::mutex> lock(g_shard_mu);
      auto& c = g_shards[h];
      if (!c) c.reset(new ShardCache());
      cache = c.get();
    }
    std::lock_guard<std::mutex> lock(cache->mu);
    auto& slot = cache->progs[{which, rank, nranks}];
    if (!slot) {
      slot.reset(new Program());
      program_restrict_rows(which == VIE_OP_Z ? h->z : h->zinv, lo, hi, *slot, s);
    }
    Program& p = *slot;
    if (nrhs >= p.tc_min_rhs && dtype == VIE_C64) program_prepare_tc(p, s);
    ensure_ws(h, p, nrhs, dtype);
    const int64_t n = h->mesh.nf;
    const int grid = (int)std::min<int64_t>((n * nrhs + 255) / 256, 152 * 8);
    const int gsc = (int)std::max<int64_t>(1, std::min<int64_t>(((hi - lo) * nrhs + 255) / 256, 152 * 8));
    if (dtype == VIE_C64) {
      gather_all<float2><<<grid, 256, 0, s>>>(h->perm.as<int32_t>(), n, (int)nrhs, (const float2*)X, ldx,
                                             h->xt.as<float2>());
      VIE_CUDA(cudaGetLastError());
      program_run(p, nrhs, dtype, h->xt.p, h->yt.p, h->coef.p, s);
      scatter_range<float2><<<gsc, 256, 0, s>>>(h->perm.as<int32_t>(), lo, hi, (int)nrhs, h->yt.as<float2>(),
                                                (float2*)Y, ldy);
    } else {
      gather_all<double2><<<grid, 256, 0, s>>>(h->perm.as<int32_t>(), n, (int)nrhs, (const double2*)X, ldx,
                                              h->xt.as<double2>());
      VIE_CUDA(cudaGetLastError());
      program_run(p, nrhs, dtype, h->xt.p, h->yt.p, h->coef.p, s);
      scatter_range<double2><<<gsc, 256, 0, s>>>(h->perm.as<int32_t>(), lo, hi, (int)nrhs, h->yt.as<double2>(),
                                                 (double2*)Y, ldy);
    }
    VIE_CUDA(cudaGetLastError());
    return VIE_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    set_error(e.what());
    return VIE_EINVAL;
  }
}
