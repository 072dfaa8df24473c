// vie_apply_noalloc: the HOD-BF apply without any device allocation.
//
// vie_apply keeps its work vectors (the tree-ordered copies of X and Y and the
// butterfly coefficient vectors) in device buffers that it allocates and grows
// on demand.  Some callers cannot let a library call cudaMalloc: cudaMalloc may
// synchronize the whole device, which stalls every stream of a latency-bound
// serving loop, and processes whose device memory is owned by another
// framework's caching allocator have no headroom for allocations made behind
// its back.  This entry point runs the same kernels with its work vectors in
// one fixed, statically sized device array instead.
//
// The array is a file-scope __device__ variable of kNoAllocScratchBytes bytes;
// every GPU that loads the library holds it until the process exits.  Host
// code cannot use the array's name as a device address (on the host it only
// names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and caches
// it; make that first call before any stream capture.  All calls on a device
// share the array: calls whose work overlaps on the GPU (different streams,
// or different threads) race on it and must be ordered by the caller.  The
// array keeps the last call's contents; nothing in it has to start at zero,
// because every work vector element is written by the apply before it is
// read (the leaf stage assigns all of Y's tree-ordered copy, and each
// coefficient block is assigned by the stage that produces it).
#include <mutex>

#include "internal.h"

namespace vie {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256] = {};

static void* noalloc_scratch() {
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  VIE_REQUIRE(dev >= 0 && dev < 256, VIE_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error{VIE_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

static size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace vie

using namespace vie;

extern "C" vie_status vie_apply_noalloc(vie_op* h, int32_t which, const void* X, void* Y, int64_t nrhs, int64_t ldx,
                                        int64_t ldy, int32_t dtype, void* stream) {
  try {
    VIE_REQUIRE(h && X && Y, VIE_EINVAL, "null argument");
    VIE_REQUIRE(nrhs >= 1 && ldx >= h->mesh.nf && ldy >= h->mesh.nf, VIE_EINVAL, "bad nrhs or leading dimension");
    VIE_REQUIRE(dtype == VIE_C64 || dtype == VIE_C128, VIE_EINVAL, "bad dtype");
    VIE_REQUIRE(which == VIE_OP_Z || which == VIE_OP_ZINV, VIE_EINVAL, "bad operator kind");
    VIE_REQUIRE(which == VIE_OP_Z || h->has_zinv, VIE_ENOTSUP, "operator has no inverse (tol_fact <= 0)");
    const Program& p = which == VIE_OP_Z ? h->z : h->zinv;
    const size_t es = dtype == VIE_C64 ? 8 : 16;
    const size_t vec = align256(es * (size_t)nrhs * (size_t)std::max<int64_t>(p.n, 1));
    const size_t cof = align256(es * (size_t)nrhs * (size_t)std::max<int64_t>(p.ncoef, 1));
    const size_t need = 2 * vec + cof;
    if (need > kNoAllocScratchBytes)
      throw Error{VIE_EINVAL, "vie_apply_noalloc: work vectors need " + std::to_string(need) +
                                  " bytes, more than the fixed scratch of " + std::to_string(kNoAllocScratchBytes) +
                                  " bytes (use vie_apply, or fewer right-hand sides)"};
    char* base = static_cast<char*>(noalloc_scratch());
    program_apply(p, h->perm.as<int32_t>(), X, Y, nrhs, ldx, ldy, dtype, base, base + vec, base + 2 * vec,
                  (cudaStream_t)stream);
    return VIE_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    set_error(e.what());
    return VIE_EINVAL;
  }
}
