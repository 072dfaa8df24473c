// Grouped applies: several operators, each with its own right-hand sides, in one
// sequence of launches.
//
// The applies of different HOD-BF operators are independent, and every one is a
// short chain of stages (Sec. III-A: leaf blocks, then the butterfly factors level
// by level).  A grouped apply walks the stage depth d = 0, 1, ... once for all
// operators: launch d holds stage d of every operator that has one, as a work
// list over (operator, block, row tile) for the SIMT kernel and over (operator,
// tensor-core item, 128-column chunk) for the tensor-core kernel.  The launch
// count is the deepest program's stage count, not the sum over operators, and
// operators too small to fill the GPU alone share its SMs.  The tree-order
// gather and scatter of all operators are one launch each.
#include "internal.h"

namespace vie {

namespace {

struct PermSeg {          // one operator's columns: tree order <-> original order
  const int32_t* perm;
  const float2* src;
  float2* dst;
  int64_t n, ld, begin;   // begin: first global element index (n * nrhs per segment)
  int32_t nrhs, pad;
};
struct PermGroup {
  PermSeg s[kGroupMax];
  int64_t total;
  int32_t n, pad;
};

// dst (tree order, rhs fastest) <- src (original order, column-major, ld)
__global__ void group_gather_kernel(const __grid_constant__ PermGroup g) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.total; e += (int64_t)gridDim.x * blockDim.x) {
    int si = 0;
    while (si + 1 < g.n && g.s[si + 1].begin <= e) ++si;
    const PermSeg& sg = g.s[si];
    const int64_t l = e - sg.begin, i = l / sg.nrhs;
    const int j = int(l % sg.nrhs);
    sg.dst[l] = sg.src[sg.perm[i] + (int64_t)j * sg.ld];
  }
}

// dst (original order, column-major, ld) <- src (tree order, rhs fastest)
__global__ void group_scatter_kernel(const __grid_constant__ PermGroup g) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.total; e += (int64_t)gridDim.x * blockDim.x) {
    int si = 0;
    while (si + 1 < g.n && g.s[si + 1].begin <= e) ++si;
    const PermSeg& sg = g.s[si];
    const int64_t l = e - sg.begin, i = l / sg.nrhs;
    const int j = int(l % sg.nrhs);
    sg.dst[sg.perm[i] + (int64_t)j * sg.ld] = sg.src[l];
  }
}

void launch_perm(const PermGroup& g, bool gather, cudaStream_t s) {
  if (g.total == 0) return;
  const int grid = (int)std::min<int64_t>((g.total + 255) / 256, 152 * 8);
  if (gather) group_gather_kernel<<<grid, 256, 0, s>>>(g);
  else group_scatter_kernel<<<grid, 256, 0, s>>>(g);
  VIE_CUDA(cudaGetLastError());
}

}  // namespace

void group_run_stages(const std::vector<GroupJob>& jobs, cudaStream_t s) {
  size_t depth = 0;
  for (const GroupJob& j : jobs) {
    VIE_REQUIRE(j.p->factor_dtype == VIE_C64, VIE_EINVAL, "grouped applies need c64 factors");
    depth = std::max(depth, j.p->stages.size());
  }
  for (size_t d = 0; d < depth; ++d) {
    SimtGroup sg{};
    TcGroup tgv[2]{};  // BF16x3 and TF32 tiles launch separately
    tgv[1].tf32 = 1;
    auto add_simt = [&](const OpDesc* ops, const Tile* tiles, int64_t nt, const Stage& st, const GroupJob& j) {
      if (nt == 0) return;
      if (sg.n == kGroupMax) { simt_launch_group(sg, s); sg = SimtGroup{}; }
      sg.s[sg.n++] = SimtSeg{ops, tiles, st.mats.as<float2>(), j.xt, j.yt, j.coef, sg.total, (int32_t)j.nrhs, 0};
      sg.total += nt;
    };
    for (const GroupJob& j : jobs) {
      const Program& p = *j.p;
      if (d >= p.stages.size()) continue;
      const Stage& st = p.stages[d];
      const bool tc = p.tc_ready && j.nrhs >= p.tc_min_rhs;
      if (tc) {
        if (st.tc_items > 0) {
          TcGroup& tg = tgv[st.tc_tf32 ? 1 : 0];
          if (tg.n == kGroupMax) {
            tc_launch_group(tg, s);
            const int32_t v = tg.tf32;
            tg = TcGroup{};
            tg.tf32 = v;
          }
          tg.s[tg.n++] = TcSeg2{st.tc_ops.as<TcItem>(), st.tc_tiles.as<uint8_t>(), j.xt, j.yt, j.coef,
                                p.err.as<int>(), tg.total, (int32_t)st.tc_items, (int32_t)j.nrhs};
          tg.total += tc_work_units(st.tc_items, (int)j.nrhs);
        }
        add_simt(st.rest_ops.as<OpDesc>(), st.rest_tiles.as<Tile>(), st.rest_ntiles, st, j);
      } else {
        add_simt(st.ops.as<OpDesc>(), st.tiles.as<Tile>(), st.ntiles, st, j);
      }
    }
    for (const TcGroup& tg : tgv)
      if (tg.n) tc_launch_group(tg, s);
    if (sg.n) simt_launch_group(sg, s);
  }
}

}  // namespace vie

using namespace vie;

extern "C" {

vie_status vie_apply_group(vie_op* const* ops, const int32_t* which, const void* const* X, void* const* Y,
                           const int64_t* nrhs, int32_t count, void* stream) {
  try {
    VIE_REQUIRE(count >= 0 && (count == 0 || (ops && which && X && Y && nrhs)), VIE_EINVAL, "null argument");
    Trace tr("vie:apply_group");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<GroupJob> jobs;
    for (int i = 0; i < count; ++i) {
      vie_op* h = ops[i];
      VIE_REQUIRE(h && X[i] && Y[i] && nrhs[i] >= 1, VIE_EINVAL, "null operator or vector, or nrhs < 1");
      VIE_REQUIRE(which[i] == VIE_OP_Z || which[i] == VIE_OP_ZINV, VIE_EINVAL, "grouped applies take Z or Zinv");
      VIE_REQUIRE(which[i] == VIE_OP_Z || h->has_zinv, VIE_ENOTSUP, "operator has no inverse (tol_fact <= 0)");
      for (int k = 0; k < i; ++k)
        VIE_REQUIRE(ops[k] != h, VIE_EINVAL, "an operator appears twice in one group (its workspaces are shared)");
      Program& p = which[i] == VIE_OP_Z ? h->z : h->zinv;
      VIE_REQUIRE(p.factor_dtype == VIE_C64, VIE_EINVAL, "grouped applies need c64 factors");
      if (nrhs[i] >= p.tc_min_rhs) program_prepare_tc(p, s);
      ensure_ws(h, p, nrhs[i], VIE_C64);
      jobs.push_back(GroupJob{&p, nrhs[i], h->xt.as<float2>(), h->yt.as<float2>(), h->coef.as<float2>()});
    }
    // gathers, the stage launches, scatters; at most kGroupMax operators per permutation launch
    for (int pass = 0; pass < 2; ++pass) {
      PermGroup g{};
      for (int i = 0; i < count; ++i) {
        if (g.n == kGroupMax) { launch_perm(g, pass == 0, s); g = PermGroup{}; }
        vie_op* h = ops[i];
        const int64_t n = h->mesh.nf;
        g.s[g.n++] = pass == 0 ? PermSeg{h->perm.as<int32_t>(), (const float2*)X[i], h->xt.as<float2>(), n, n,
                                         g.total, (int32_t)nrhs[i], 0}
                               : PermSeg{h->perm.as<int32_t>(), h->yt.as<float2>(), (float2*)Y[i], n, n, g.total,
                                         (int32_t)nrhs[i], 0};
        g.total += n * nrhs[i];
      }
      if (g.n) launch_perm(g, pass == 0, s);
      if (pass == 0) group_run_stages(jobs, s);
    }
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

}  // extern "C"
