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

__global__ void nonfinite_kernel(const float* v, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) { *flag = 1; return; }
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

void program_check(const Program& p) {
  const int64_t eb = elem_bytes_of(p);
  for (size_t k = 0; k < p.stages.size(); ++k) {
    const Stage& st = p.stages[k];
    const int64_t elems = (int64_t)st.mats.bytes / eb;
    for (const OpDesc& o : st.host_ops) {
      auto fits = [&](int sp, int64_t off, int64_t len) {
        const int64_t lim = sp == SP_C ? p.ncoef : p.n;
        return (sp == SP_X || sp == SP_Y || sp == SP_C) && off >= 0 && len >= 0 && off + len <= lim;
      };
      const bool ok = o.M >= 0 && o.K >= 0 && o.ld >= o.K && (o.ld & 1) == 0 && (o.mat_off & 1) == 0 &&
                      o.mat_off >= 0 && o.mat_off + (int64_t)o.M * o.ld <= elems && fits(o.in_space, o.in_off, o.K) &&
                      fits(o.out_space, o.out_off, o.M);
      VIE_REQUIRE(ok, VIE_EINVAL, "apply program block out of range (stage " + std::to_string(k) + ")");
    }
  }
}

bool program_finite(const Program& p, cudaStream_t s) {
  DevBuf flag;
  flag.alloc(sizeof(int));
  VIE_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), s));
  for (const Stage& st : p.stages) {
    const int64_t n = (int64_t)(st.mats.bytes / sizeof(float));
    if (n) nonfinite_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(st.mats.as<float>(), n,
                                                                                             flag.as<int>());
  }
  VIE_CUDA(cudaGetLastError());
  int h = 0;
  VIE_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  VIE_CUDA(cudaStreamSynchronize(s));
  return h == 0;
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
  // The first adjoint block writing a coefficient interval assigns instead of adding: the
  // coefficients then need no zero from the caller and their memory can be shared by
  // lifetime (the forward program may already share it).  In execution order, a write is the
  // first of its interval when no write to that interval is pending, a pending write being
  // one that no block has read since; the second child of a pair then adds to the first.
  {
    std::map<int64_t, int64_t> pending;  // written, not yet read: lo -> hi
    for (Stage& st : adj.stages) {
      for (const OpDesc& o : st.host_ops)  // reads of this launch consume pending writes
        if (o.in_space == SP_C && o.K > 0) {
          const int64_t a = o.in_off, b = o.in_off + o.K;
          auto it = pending.upper_bound(a);
          if (it != pending.begin() && std::prev(it)->second > a) --it;
          while (it != pending.end() && it->first < b) it = pending.erase(it);
        }
      bool changed = false;
      for (OpDesc& o : st.host_ops) {
        if (o.out_space != SP_C || o.M <= 0) continue;
        const int64_t a = o.out_off, b = o.out_off + o.M;
        auto it = pending.find(a);
        if (it != pending.end() && it->second == b) continue;  // adds to the pending write
        auto nx = pending.upper_bound(a);
        const bool clash = (nx != pending.end() && nx->first < b) ||
                           (nx != pending.begin() && std::prev(nx)->second > a);
        VIE_REQUIRE(!clash, VIE_EINVAL, "adjoint program: overlapping coefficient writes of different extent");
        pending[a] = b;
        o.accumulate = 0;
        changed = true;
      }
      if (changed)
        VIE_CUDA(cudaMemcpyAsync(st.ops.p, st.host_ops.data(), sizeof(OpDesc) * st.host_ops.size(),
                                 cudaMemcpyHostToDevice, s));
    }
    VIE_CUDA(cudaStreamSynchronize(s));
  }
  program_totals(adj);
  program_check(adj);
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
  program_check(out);
}

// Coefficient space by lifetimes.  A unit is a maximal run of coefficients that
// some block reads or writes as part of one interval.  A unit whose first access
// (in stage order) is a set of assigning writes covering all of it, and that some
// block reads later, carries nothing in from before; it is live from that stage to
// its last access and may share memory with units whose lives end earlier.  Any
// other unit keeps memory of its own (it relies on the zero the caller sets before
// the run).  The adjoint program of a compacted program keeps these offsets: its
// lifetimes are the same intervals reversed, and program_adjoint makes the first
// write of every unit an assignment.  Units with the
// same (first, last) stages are packed together in their original order, which
// keeps every interval a block reads across adjacent units contiguous.
void program_compact_coef(Program& p, cudaStream_t s) {
  struct Acc { int64_t lo, hi; int stage; bool write, assign; };
  std::vector<Acc> acc;
  for (size_t k = 0; k < p.stages.size(); ++k)
    for (const OpDesc& o : p.stages[k].host_ops) {
      if (o.in_space == SP_C && o.K > 0) acc.push_back(Acc{o.in_off, o.in_off + o.K, (int)k, false, false});
      if (o.out_space == SP_C && o.M > 0) acc.push_back(Acc{o.out_off, o.out_off + o.M, (int)k, true, o.accumulate == 0});
    }
  if (acc.empty()) { p.ncoef = 0; return; }
  std::vector<size_t> ord(acc.size());
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return acc[a].lo < acc[b].lo; });
  struct Unit { int64_t lo, hi; int first = 1 << 30, last = -1; bool init = false, read = false; int64_t base = 0; };
  std::vector<Unit> units;
  std::vector<int> unit_of(acc.size());
  for (size_t q : ord) {
    if (units.empty() || acc[q].lo >= units.back().hi) units.push_back(Unit{acc[q].lo, acc[q].hi});
    else units.back().hi = std::max(units.back().hi, acc[q].hi);
    unit_of[q] = (int)units.size() - 1;
  }
  for (size_t q = 0; q < acc.size(); ++q) {
    Unit& u = units[unit_of[q]];
    u.first = std::min(u.first, acc[q].stage);
    u.last = std::max(u.last, acc[q].stage);
    if (!acc[q].write) u.read = true;
  }
  {  // self-initializing: the accesses of the first stage are assigning writes covering the unit
    std::vector<std::vector<std::pair<int64_t, int64_t>>> cover(units.size());
    std::vector<char> bad(units.size(), 0);
    for (size_t q = 0; q < acc.size(); ++q) {
      const int ui = unit_of[q];
      if (acc[q].stage != units[ui].first) continue;
      if (!acc[q].write || !acc[q].assign) bad[ui] = 1;
      else cover[ui].push_back({acc[q].lo, acc[q].hi});
    }
    for (size_t ui = 0; ui < units.size(); ++ui) {
      if (bad[ui]) continue;
      auto& cv = cover[ui];
      std::sort(cv.begin(), cv.end());
      int64_t reach = units[ui].lo;
      for (auto& c : cv) {
        if (c.first > reach) break;
        reach = std::max(reach, c.second);
      }
      // a unit no block reads is read first in the adjoint program (which takes its offsets
      // from this one) and must hold the zero the caller sets: it keeps memory of its own
      units[ui].init = reach >= units[ui].hi && units[ui].read;
    }
  }
  // exclusive memory first, then lifetime groups placed first-fit over freed regions
  int64_t top = 0;
  for (Unit& u : units)
    if (!u.init) { u.base = top; top += u.hi - u.lo; }
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (size_t ui = 0; ui < units.size(); ++ui)
    if (units[ui].init) groups[{units[ui].first, units[ui].last}].push_back((int)ui);
  struct Region { int64_t addr, size; int last; };
  std::vector<Region> busy;
  std::vector<std::pair<int64_t, int64_t>> freel;  // (addr, size)
  for (auto& g : groups) {  // ordered by first stage
    const int first = g.first.first, last = g.first.second;
    for (size_t i = 0; i < busy.size();) {
      if (busy[i].last < first) { freel.push_back({busy[i].addr, busy[i].size}); busy.erase(busy.begin() + i); }
      else ++i;
    }
    std::sort(freel.begin(), freel.end());
    std::vector<std::pair<int64_t, int64_t>> merged;
    for (auto& f : freel) {
      if (!merged.empty() && merged.back().first + merged.back().second == f.first) merged.back().second += f.second;
      else merged.push_back(f);
    }
    freel = merged;
    int64_t need = 0;
    for (int ui : g.second) need += units[ui].hi - units[ui].lo;
    int64_t addr = -1;
    for (size_t i = 0; i < freel.size(); ++i)
      if (freel[i].second >= need) {
        addr = freel[i].first;
        freel[i].first += need;
        freel[i].second -= need;
        if (freel[i].second == 0) freel.erase(freel.begin() + i);
        break;
      }
    if (addr < 0) { addr = top; top += need; }
    int64_t off = addr;
    for (int ui : g.second) { units[ui].base = off; off += units[ui].hi - units[ui].lo; }
    busy.push_back(Region{addr, need, last});
  }
  auto remap = [&](int64_t lo) {
    auto it = std::upper_bound(units.begin(), units.end(), lo, [](int64_t v, const Unit& u) { return v < u.lo; });
    --it;
    return it->base + (lo - it->lo);
  };
  for (Stage& st : p.stages) {
    bool changed = false;
    for (OpDesc& o : st.host_ops) {
      if (o.in_space == SP_C && o.K > 0) { o.in_off = remap(o.in_off); changed = true; }
      if (o.out_space == SP_C && o.M > 0) { o.out_off = remap(o.out_off); changed = true; }
      if (o.in_space == SP_C && o.K == 0) o.in_off = 0;
    }
    if (changed && !st.host_ops.empty())
      VIE_CUDA(cudaMemcpyAsync(st.ops.p, st.host_ops.data(), sizeof(OpDesc) * st.host_ops.size(),
                               cudaMemcpyHostToDevice, s));
    st.tc_tiles.release(); st.tc_ops.release(); st.rest_ops.release(); st.rest_tiles.release();
    st.tc_items = st.tc_bytes = st.rest_ntiles = 0;
  }
  p.tc_ready = false;
  for (auto& g : p.graphs)
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
  p.ncoef = top;
  VIE_CUDA(cudaStreamSynchronize(s));
  program_check(p);
}

// The blocks of a program that the output rows [lo, hi) of Y depend on (their dependency
// closure, found backwards through the stages), copied with their matrices into `out`;
// coefficient offsets are kept (out.ncoef = p.ncoef).  For Z the closure writes Y only
// on [lo, hi); a program that reads Y (the in-place levels of Zinv) may also need, and
// then writes, other rows of Y, which the caller discards.  The restricted program reads
// X wherever the kept blocks read it (the caller provides the whole of X).
void program_restrict_rows(const Program& p, int64_t lo, int64_t hi, Program& out, cudaStream_t s) {
  const int eb = elem_bytes_of(p);
  // needed intervals per space (C, Y): map lo -> hi, disjoint and merged
  std::map<int64_t, int64_t> need[3];
  auto overlaps = [&](int sp, int64_t a, int64_t b) {
    auto& m = need[sp];
    auto it = m.upper_bound(a);
    if (it != m.begin()) { auto pv = std::prev(it); if (pv->second > a) return true; }
    return it != m.end() && it->first < b;
  };
  auto add = [&](int sp, int64_t a, int64_t b) {
    if (b <= a) return;
    auto& m = need[sp];
    auto it = m.upper_bound(a);
    if (it != m.begin()) {
      auto pv = std::prev(it);
      if (pv->second >= a) { a = pv->first; b = std::max(b, pv->second); it = m.erase(pv); }
    }
    while (it != m.end() && it->first <= b) { b = std::max(b, it->second); it = m.erase(it); }
    m[a] = b;
  };
  add(SP_Y, lo, hi);
  std::vector<std::vector<char>> keep(p.stages.size());
  for (int k = (int)p.stages.size() - 1; k >= 0; --k) {
    const auto& ops = p.stages[k].host_ops;
    keep[k].assign(ops.size(), 0);
    std::vector<size_t> kept;
    for (size_t i = 0; i < ops.size(); ++i) {
      const OpDesc& o = ops[i];
      if (o.M <= 0) continue;
      if (o.out_space != SP_X && overlaps(o.out_space, o.out_off, o.out_off + o.M)) { keep[k][i] = 1; kept.push_back(i); }
    }
    for (size_t i : kept) {  // inputs of this stage's kept blocks are needed from earlier stages
      const OpDesc& o = ops[i];
      if (o.in_space != SP_X && o.K > 0) add(o.in_space, o.in_off, o.in_off + o.K);
    }
  }
  out.stages.clear();
  out.n = p.n;
  out.ncoef = p.ncoef;
  out.factor_dtype = p.factor_dtype;
  out.tc_ready = false;
  for (size_t k = 0; k < p.stages.size(); ++k) {
    const Stage& st = p.stages[k];
    std::vector<OpDesc> ops;
    std::vector<int32_t> tags;
    std::vector<CopyJob> jobs;
    int64_t off = 0;
    for (size_t i = 0; i < st.host_ops.size(); ++i) {
      if (!keep[k][i]) continue;
      OpDesc o = st.host_ops[i];
      const int64_t cnt = (int64_t)o.M * o.ld;
      jobs.push_back(CopyJob{o.mat_off, off, cnt});
      o.mat_off = off;
      off += cnt;
      off = (off + 1) & ~int64_t(1);
      ops.push_back(o);
      tags.push_back(i < st.host_tag.size() ? st.host_tag[i] : -1);
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
  program_totals(out);
  program_check(out);
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
