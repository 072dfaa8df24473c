// Construction helpers for apply programs: stages from packed ops, the adjoint
// program, the sub-program of one tree level's butterflies, and relocation of
// the coefficient space when programs are concatenated.
//
// An apply program is a list of stages; each stage is a set of independent
// block products  y[out] (=|+=) A x[in]  over three vector spaces (X: input,
// Y: output, C: butterfly coefficients).  The adjoint of a program runs the
// conjugate-transposed blocks in reverse stage order, every block accumulating
// into what was its input:  x[in] += A^H y[out].  Within one forward stage two
// blocks may read the same input slice (the two children of a node read the
// same pair of coefficient blocks in a butterfly transfer level, Eq. 10), so
// their adjoints write the same slice; such blocks are split into sub-stages
// (greedy colouring of the output intervals) so that every output element still
// has one writer per launch and the result stays deterministic.
//
// Conditions for the adjoint to be exact (all programs built here meet them):
// every C slice is written by one forward block (assign), X is never written,
// and a forward block that assigns Y is not preceded by one that writes the same
// rows.  The adjoint program reads its input in Y and accumulates into X and C,
// which the caller sets to zero first; it also accumulates into Y when the
// forward program reads Y (in-place updates y <- y + E y).
#include <algorithm>
#include <map>
#include <set>

#include "internal.h"

namespace vie {

namespace {

struct CopyJob {
  int64_t src, dst, count;  // elements
};

template <class T>
__global__ void copy_jobs_kernel(const CopyJob* jobs, const T* src, T* dst) {
  const CopyJob j = jobs[blockIdx.x];
  for (int64_t e = threadIdx.x; e < j.count; e += blockDim.x) dst[j.dst + e] = src[j.src + e];
}

struct AdjJob {
  int64_t src, dst;  // element offsets of the forward block (M x K, ld) and of its adjoint (K x M, ld')
  int32_t M, K, ld, ldt;
};

template <class T>
__global__ void adjoint_pack_kernel(const AdjJob* jobs, const T* src, T* dst) {
  const AdjJob j = jobs[blockIdx.x];
  // dst row c (c < K) holds conj(A(:, c)); columns M .. ldt-1 are zero padding
  for (int64_t e = threadIdx.x; e < (int64_t)j.K * j.ldt; e += blockDim.x) {
    const int c = int(e / j.ldt), r = int(e % j.ldt);
    T v;
    if (r < j.M) {
      v = src[j.src + (int64_t)r * j.ld + c];
      v.y = -v.y;
    } else {
      v.x = 0;
      v.y = 0;
    }
    dst[j.dst + e] = v;
  }
}

template <class J>
void upload(DevBuf& b, const std::vector<J>& v, cudaStream_t s) {
  b.alloc(sizeof(J) * std::max<size_t>(1, v.size()));
  if (!v.empty()) VIE_CUDA(cudaMemcpyAsync(b.p, v.data(), sizeof(J) * v.size(), cudaMemcpyHostToDevice, s));
}

int elem_bytes_of(const Program& p) { return p.factor_dtype == VIE_C64 ? 8 : 16; }

}  // namespace

void stage_set(Stage& st, std::vector<OpDesc> ops, DevBuf&& mats, int64_t elems, int elem_bytes, cudaStream_t s) {
  st.mats = std::move(mats);
  if (!st.mats.p) st.mats.alloc(2 * elem_bytes);
  std::vector<Tile> tiles;
  make_tiles(ops, tiles);
  st.nops = (int64_t)ops.size();
  st.ntiles = (int64_t)tiles.size();
  upload(st.ops, ops, s);
  upload(st.tiles, tiles, s);
  st.entries = 0;
  for (const OpDesc& o : ops) st.entries += (int64_t)o.M * o.K;
  st.bytes = elems * elem_bytes;
  st.kernel = kKernelPlain4;
  st.host_ops = std::move(ops);
  if (st.host_tag.size() != st.host_ops.size()) st.host_tag.assign(st.host_ops.size(), -1);
  st.tc_items = st.tc_bytes = st.rest_ntiles = 0;
  VIE_CUDA(cudaStreamSynchronize(s));
}

void program_totals(Program& p) {
  p.entries = p.bytes = 0;
  for (const Stage& st : p.stages) { p.entries += st.entries; p.bytes += st.bytes; }
}

void program_adjoint(const Program& fwd, Program& adj, cudaStream_t s) {
  const int eb = elem_bytes_of(fwd);
  adj.stages.clear();
  adj.n = fwd.n;
  adj.ncoef = fwd.ncoef;
  adj.factor_dtype = fwd.factor_dtype;
  adj.tc_ready = false;
  for (int k = (int)fwd.stages.size() - 1; k >= 0; --k) {
    const Stage& st = fwd.stages[k];
    const auto& ops = st.host_ops;
    if (ops.empty()) continue;
    // colour: sub-stage g holds ops whose outputs (the forward inputs) do not overlap
    std::vector<std::map<std::pair<int, int64_t>, int64_t>> used;  // (space, lo) -> hi
    std::vector<int> colour(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
      const OpDesc& o = ops[i];
      const int sp = o.in_space;
      const int64_t lo = o.in_off, hi = o.in_off + o.K;
      size_t g = 0;
      for (; g < used.size(); ++g) {
        auto& m = used[g];
        auto it = m.lower_bound({sp, lo});
        bool clash = false;
        if (it != m.end() && it->first.first == sp && it->first.second < hi) clash = true;
        if (!clash && it != m.begin()) {
          auto pv = std::prev(it);
          if (pv->first.first == sp && pv->second > lo) clash = true;
        }
        if (!clash) break;
      }
      if (g == used.size()) used.emplace_back();
      used[g][{sp, lo}] = hi;
      colour[i] = (int)g;
    }
    for (size_t g = 0; g < used.size(); ++g) {
      std::vector<OpDesc> aops;
      std::vector<int32_t> atags;
      std::vector<AdjJob> jobs;
      int64_t off = 0;
      for (size_t i = 0; i < ops.size(); ++i) {
        if (colour[i] != (int)g) continue;
        const OpDesc& o = ops[i];
        OpDesc a{};
        a.M = o.K;
        a.K = o.M;
        a.ld = (o.M + 1) & ~1;
        a.mat_off = off;
        a.in_space = o.out_space;
        a.in_off = o.out_off;
        a.out_space = o.in_space;
        a.out_off = o.in_off;
        a.accumulate = 1;
        jobs.push_back(AdjJob{o.mat_off, off, o.M, o.K, o.ld, a.ld});
        off += (int64_t)a.M * a.ld;
        off = (off + 1) & ~int64_t(1);
        aops.push_back(a);
        atags.push_back(i < st.host_tag.size() ? st.host_tag[i] : -1);
      }
      DevBuf mats, dj;
      mats.alloc(std::max<int64_t>(off, 2) * eb);
      upload(dj, jobs, s);
      if (eb == 8)
        adjoint_pack_kernel<float2><<<(int)jobs.size(), 256, 0, s>>>(dj.as<AdjJob>(), st.mats.as<float2>(),
                                                                     mats.as<float2>());
      else
        adjoint_pack_kernel<double2><<<(int)jobs.size(), 256, 0, s>>>(dj.as<AdjJob>(), st.mats.as<double2>(),
                                                                      mats.as<double2>());
      VIE_CUDA(cudaGetLastError());
      adj.stages.emplace_back();
      adj.stages.back().host_tag = atags;
      stage_set(adj.stages.back(), std::move(aops), std::move(mats), off, eb, s);
    }
  }
  program_totals(adj);
}

void program_filter(const Program& src, int32_t tag, Program& out, cudaStream_t s) {
  const int eb = elem_bytes_of(src);
  out.stages.clear();
  out.n = src.n;
  out.factor_dtype = src.factor_dtype;
  out.tc_ready = false;
  // coefficient runs written by the kept ops, merged, in order: compact offsets
  std::vector<std::pair<int64_t, int64_t>> iv;
  for (const Stage& st : src.stages)
    for (size_t i = 0; i < st.host_ops.size(); ++i)
      if (i < st.host_tag.size() && st.host_tag[i] == tag && st.host_ops[i].out_space == SP_C)
        iv.push_back({st.host_ops[i].out_off, st.host_ops[i].out_off + st.host_ops[i].M});
  std::sort(iv.begin(), iv.end());
  std::vector<std::pair<int64_t, int64_t>> runs;  // merged [lo, hi)
  for (auto& p : iv) {
    if (!runs.empty() && p.first <= runs.back().second) runs.back().second = std::max(runs.back().second, p.second);
    else runs.push_back(p);
  }
  std::vector<int64_t> base(runs.size());
  int64_t nc = 0;
  for (size_t r = 0; r < runs.size(); ++r) { base[r] = nc; nc += runs[r].second - runs[r].first; }
  auto remap = [&](int64_t off, int64_t len) {
    auto it = std::upper_bound(runs.begin(), runs.end(), std::make_pair(off, INT64_MAX));
    VIE_REQUIRE(it != runs.begin(), VIE_EINVAL, "sub-program reads coefficients it does not write");
    --it;
    VIE_REQUIRE(off >= it->first && off + len <= it->second, VIE_EINVAL,
                "sub-program reads coefficients it does not write");
    return base[it - runs.begin()] + (off - it->first);
  };
  for (const Stage& st : src.stages) {
    std::vector<OpDesc> ops;
    std::vector<int32_t> tags;
    std::vector<CopyJob> jobs;
    int64_t off = 0;
    for (size_t i = 0; i < st.host_ops.size(); ++i) {
      if (i >= st.host_tag.size() || st.host_tag[i] != tag) continue;
      OpDesc o = st.host_ops[i];
      const int64_t cnt = (int64_t)o.M * o.ld;
      jobs.push_back(CopyJob{o.mat_off, off, cnt});
      o.mat_off = off;
      off += cnt;
      off = (off + 1) & ~int64_t(1);
      if (o.out_space == SP_C) o.out_off = remap(o.out_off, o.M);
      if (o.in_space == SP_C) o.in_off = remap(o.in_off, o.K);
      ops.push_back(o);
      tags.push_back(tag);
    }
    if (ops.empty()) continue;
    DevBuf mats, dj;
    mats.alloc(std::max<int64_t>(off, 2) * eb);
    upload(dj, jobs, s);
    if (eb == 8)
      copy_jobs_kernel<float2><<<(int)jobs.size(), 256, 0, s>>>(dj.as<CopyJob>(), st.mats.as<float2>(), mats.as<float2>());
    else
      copy_jobs_kernel<double2><<<(int)jobs.size(), 256, 0, s>>>(dj.as<CopyJob>(), st.mats.as<double2>(),
                                                                 mats.as<double2>());
    VIE_CUDA(cudaGetLastError());
    out.stages.emplace_back();
    out.stages.back().host_tag = tags;
    stage_set(out.stages.back(), std::move(ops), std::move(mats), off, eb, s);
  }
  out.ncoef = nc;
  program_totals(out);
}

void program_relocate_coef(Program& p, int64_t shift, cudaStream_t s) {
  if (shift == 0) return;
  for (Stage& st : p.stages) {
    for (OpDesc& o : st.host_ops) {
      if (o.in_space == SP_C) o.in_off += shift;
      if (o.out_space == SP_C) o.out_off += shift;
    }
    if (!st.host_ops.empty())
      VIE_CUDA(cudaMemcpyAsync(st.ops.p, st.host_ops.data(), sizeof(OpDesc) * st.host_ops.size(),
                               cudaMemcpyHostToDevice, s));
    // the tensor-core items hold the old offsets: drop them (prepared again on first use)
    st.tc_tiles.release(); st.tc_ops.release(); st.rest_ops.release(); st.rest_tiles.release();
    st.tc_items = st.tc_bytes = st.rest_ntiles = 0;
  }
  p.tc_ready = false;
  p.ncoef += shift;
  VIE_CUDA(cudaStreamSynchronize(s));
}

void program_append(Program& dst, Program&& src, cudaStream_t s) {
  VIE_REQUIRE(dst.factor_dtype == src.factor_dtype, VIE_EINVAL, "appending programs of different factor types");
  const int64_t base = dst.ncoef;
  program_relocate_coef(src, base, s);  // src.ncoef becomes base + its own count
  for (Stage& st : src.stages) dst.stages.push_back(std::move(st));
  dst.ncoef = src.ncoef;
  src.stages.clear();
  program_totals(dst);
  dst.tc_ready = false;
  for (auto& g : dst.graphs)
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
}

void program_prepend(Program& dst, Program&& src) {
  // both programs index one shared coefficient space (the adjoint of a program built by appends)
  std::vector<Stage> st;
  st.reserve(src.stages.size() + dst.stages.size());
  for (Stage& x : src.stages) st.push_back(std::move(x));
  for (Stage& x : dst.stages) st.push_back(std::move(x));
  dst.stages = std::move(st);
  dst.ncoef = std::max(dst.ncoef, src.ncoef);
  src.stages.clear();
  program_totals(dst);
  dst.tc_ready = false;
  for (auto& g : dst.graphs)
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
}

}  // namespace vie
