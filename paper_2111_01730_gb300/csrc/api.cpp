// C ABI of libvie (declared in include/vie.h).
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <utility>

#include "internal.h"

namespace vie {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

static std::mutex g_attr_mu;
static std::set<std::pair<int, const void*>> g_attr_done;

bool done_on_device(const void* key) {
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_attr_mu);
  return g_attr_done.count({dev, key}) != 0;
}

void mark_on_device(const void* key) {
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_attr_mu);
  g_attr_done.insert({dev, key});
}

void ensure_smem_attr(const void* kernel, int bytes) {
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (g_attr_done.count({dev, kernel})) return;
  VIE_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  g_attr_done.insert({dev, kernel});
}

void DevBuf::alloc(size_t n) {
  release();
  if (n == 0) n = 16;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    throw Error{VIE_ENOMEM, std::string("cudaMalloc(") + std::to_string(n) + "): " + cudaGetErrorString(e)};
  }
  bytes = n;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

void ensure_ws(vie_op* h, const Program& p, int64_t nrhs, int dtype) {
  size_t es = dtype == VIE_C64 ? 8 : 16;
  size_t need = es * (size_t)nrhs * (size_t)std::max<int64_t>(p.n, 1);
  size_t needc = es * (size_t)nrhs * (size_t)std::max<int64_t>(p.ncoef, 1);
  if (h->xt.bytes < need) { h->xt.alloc(need); h->yt.alloc(need); }
  if (h->coef.bytes < needc) h->coef.alloc(needc);
}

void op_apply(vie_op* h, int which, const void* X, void* Y, int64_t nrhs, int dtype, cudaStream_t s) {
  Program& p = which == VIE_OP_Z ? h->z : h->zinv;
  if (nrhs >= p.tc_min_rhs && dtype == VIE_C64) program_prepare_tc(p, s);
  ensure_ws(h, p, nrhs, dtype);
  program_apply_graph(p, h->perm.as<int32_t>(), X, Y, nrhs, h->mesh.nf, h->mesh.nf, dtype, h->xt.p, h->yt.p,
                      h->coef.p, s);
}

}  // namespace vie

using namespace vie;

template <class F>
static vie_status guarded(F&& f) {
  try {
    f();
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

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

extern "C" {

const char* vie_last_error(void) { return g_err.c_str(); }

static void check_config(const vie_config* cfg, double k0) {
  VIE_REQUIRE(cfg->leaf >= 4 && cfg->tol_con > 0 && k0 > 0, VIE_EINVAL, "invalid configuration");
  VIE_REQUIRE(cfg->factor_dtype == VIE_C64 || cfg->factor_dtype == VIE_C128, VIE_EINVAL, "factor dtype");
  VIE_REQUIRE(cfg->prec >= VIE_P_AUTO && cfg->prec <= VIE_P_TC_TF32, VIE_EINVAL, "bad precision");
}

// everything after the mesh: geometry, cluster tree, Z (Sec. III-A), Zinv (Sec. III-B)
static void build_operator(vie_op* h, double k0, const vie_config* cfg, cudaStream_t s, double t0) {
  Trace tr("vie:build");
  h->cfg = *cfg;
  if (h->cfg.oversample <= 0) h->cfg.oversample = 10;
  if (cfg->prec == VIE_P_FP64) h->cfg.factor_dtype = VIE_C128;
  if (cfg->prec == VIE_P_C32 || cfg->prec == VIE_P_TC_BF16X3 || cfg->prec == VIE_P_TC_TF32)
    h->cfg.factor_dtype = VIE_C64;
  geometry_upload(h->mesh, k0, h->geo, s);
  if (!h->mesh.general) geometry_table(h->geo, s);
  const int64_t N = h->mesh.nf;
  build_tree(face_centroids(h->mesh), cfg->leaf, h->tree);
  h->perm.alloc(sizeof(int32_t) * N);
  VIE_CUDA(cudaMemcpyAsync(h->perm.p, h->tree.perm.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
  h->tet_faces.alloc(sizeof(int32_t) * 4 * h->mesh.nt);
  VIE_CUDA(cudaMemcpyAsync(h->tet_faces.p, h->mesh.tet_faces.data(), sizeof(int32_t) * 4 * h->mesh.nt,
                           cudaMemcpyHostToDevice, s));
  BuildResult br;
  {
    Trace tz("vie:build/Z");
    build_hodbf(h, s, br);
  }
  const int never = 1 << 30;
  h->z.tc_min_rhs = h->zinv.tc_min_rhs = cfg->prec == VIE_P_C32 ? never : kTcMinRhs;
  VIE_CUDA(cudaStreamSynchronize(s));
  h->stats.n = N;
  h->stats.ntets = h->mesh.nt;
  h->stats.levels = h->tree.levels;
  h->stats.max_rank = br.max_rank;
  h->stats.entries_z = h->z.entries;
  h->stats.bytes_z = h->z.bytes;
  h->stats.entries_evaluated = br.entries_evaluated;
  h->stats.apply_stages_z = (int32_t)h->z.stages.size();
  h->stats.build_entries_seconds = br.t_entries;
  h->stats.build_id_seconds = br.t_id;
  h->stats.build_host_seconds = br.t_host;
  h->stats.build_seconds = now_s() - t0;
  if (cfg->tol_fact > 0) {
    double t1 = now_s();
    BuildResult bi;
    Trace ti("vie:build/Zinv");
    build_inverse(h, s, bi);
    VIE_CUDA(cudaStreamSynchronize(s));
    h->stats.entries_zinv = h->zinv.entries;
    h->stats.bytes_zinv = h->zinv.bytes;
    h->stats.apply_stages_zinv = (int32_t)h->zinv.stages.size();
    h->stats.max_rank = std::max(h->stats.max_rank, bi.max_rank);
    h->stats.invert_seconds = now_s() - t1;
    h->stats.zinv_top_level = h->zinv_top_level;
  }
  // the TF32 variant serves the caller's applies; the construction above ran its
  // products with the BF16x3 split
  if (cfg->prec == VIE_P_TC_TF32) {
    program_set_tc_variant(h->z, true);
    program_set_tc_variant(h->zinv, true);
  }
}

vie_status vie_build(const vie_voxels* body, double k0, const vie_config* cfg, void* stream, vie_op** out) {
  return guarded([&] {
    VIE_REQUIRE(body && cfg && out, VIE_EINVAL, "null argument");
    VIE_REQUIRE(body->nvox > 0 && body->ijk && body->eps && body->h > 0, VIE_EINVAL, "empty or invalid voxel body");
    check_config(cfg, k0);
    *out = nullptr;
    const double t0 = now_s();
    vie_op* h = new vie_op();
    try {
      build_mesh(*body, h->mesh);
      build_operator(h, k0, cfg, (cudaStream_t)stream, t0);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

vie_status vie_build_mesh(const vie_mesh* mesh, double k0, const vie_config* cfg, void* stream, vie_op** out) {
  return guarded([&] {
    VIE_REQUIRE(mesh && cfg && out, VIE_EINVAL, "null argument");
    check_config(cfg, k0);
    *out = nullptr;
    const double t0 = now_s();
    vie_op* h = new vie_op();
    try {
      build_mesh_general(*mesh, h->mesh);
      build_operator(h, k0, cfg, (cudaStream_t)stream, t0);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

void vie_destroy(vie_op* op) {
  if (op) shard_forget(op);
  delete op;
}

vie_status vie_apply(vie_op* h, int32_t which, const void* X, void* Y, int64_t nrhs, int64_t ldx, int64_t ldy,
                     int32_t dtype, void* stream) {
  return guarded([&] {
    VIE_REQUIRE(h && X && Y, VIE_EINVAL, "null argument");
    VIE_REQUIRE(nrhs >= 1 && ldx >= h->mesh.nf && ldy >= h->mesh.nf, VIE_EINVAL, "bad nrhs or leading dimension");
    VIE_REQUIRE(dtype == VIE_C64 || dtype == VIE_C128, VIE_EINVAL, "bad dtype");
    VIE_REQUIRE(which >= VIE_OP_Z && which <= VIE_OP_ZINVH, VIE_EINVAL, "bad operator kind");
    Trace tr(which == VIE_OP_Z ? "vie:apply/Z" : which == VIE_OP_ZINV ? "vie:apply/Zinv" : "vie:apply/adjoint");
    VIE_REQUIRE(which == VIE_OP_Z || which == VIE_OP_ZH || h->has_zinv, VIE_ENOTSUP,
                "operator has no inverse (tol_fact <= 0)");
    cudaStream_t s = (cudaStream_t)stream;
    if (which == VIE_OP_ZH || which == VIE_OP_ZINVH) {
      const bool inv = which == VIE_OP_ZINVH;
      Program& a = inv ? h->zinvh : h->zh;
      bool& ready = inv ? h->zinvh_ready : h->zh_ready;
      if (!ready) {
        program_adjoint(inv ? h->zinv : h->z, a, s);
        program_set_tc_variant(a, (inv ? h->zinv : h->z).tc_tf32);
        ready = true;
      }
      if (nrhs >= a.tc_min_rhs && dtype == VIE_C64) program_prepare_tc(a, s);
      ensure_ws(h, a, nrhs, dtype);
      program_apply_adjoint(a, h->perm.as<int32_t>(), X, Y, nrhs, ldx, ldy, dtype, h->xt.p, h->yt.p, h->coef.p, s);
      return;
    }
    Program& p = which == VIE_OP_Z ? h->z : h->zinv;
    if (nrhs >= p.tc_min_rhs && dtype == VIE_C64) program_prepare_tc(p, s);
    ensure_ws(h, p, nrhs, dtype);
    program_apply_graph(p, h->perm.as<int32_t>(), X, Y, nrhs, ldx, ldy, dtype, h->xt.p, h->yt.p, h->coef.p, s);
  });
}

vie_status vie_apply_profile(vie_op* h, int32_t which, const void* X, void* Y, int64_t nrhs, int64_t ldx,
                             int64_t ldy, int32_t dtype, void* stream, double* ms, int64_t* launches, int32_t cap) {
  return guarded([&] {
    VIE_REQUIRE(h && X && Y && ms, VIE_EINVAL, "null argument");
    VIE_REQUIRE(nrhs >= 1 && ldx >= h->mesh.nf && ldy >= h->mesh.nf, VIE_EINVAL, "bad nrhs or leading dimension");
    VIE_REQUIRE(dtype == VIE_C64 || dtype == VIE_C128, VIE_EINVAL, "bad dtype");
    VIE_REQUIRE(which == VIE_OP_Z || (which == VIE_OP_ZINV && h->has_zinv), VIE_ENOTSUP, "no such operator");
    Program& p = which == VIE_OP_Z ? h->z : h->zinv;
    if (nrhs >= p.tc_min_rhs && dtype == VIE_C64) program_prepare_tc(p, (cudaStream_t)stream);
    const int ns = (int)p.stages.size() + 2;
    VIE_REQUIRE(cap >= ns, VIE_EINVAL, "ms array too short (stages + 2 needed)");
    ensure_ws(h, p, nrhs, dtype);
    std::vector<cudaEvent_t> ev(ns + 1);
    for (auto& e : ev) VIE_CUDA(cudaEventCreate(&e));
    cudaStream_t s = (cudaStream_t)stream;
    try {
      program_apply(p, h->perm.as<int32_t>(), X, Y, nrhs, ldx, ldy, dtype, h->xt.p, h->yt.p, h->coef.p, s, ev.data());
      VIE_CUDA(cudaEventSynchronize(ev[ns]));
      for (int i = 0; i < ns; ++i) {
        float t = 0;
        VIE_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
        ms[i] = t;
      }
      if (launches) *launches = program_launches(p, nrhs, dtype);
    } catch (...) {
      for (auto& e : ev) cudaEventDestroy(e);
      throw;
    }
    for (auto& e : ev) cudaEventDestroy(e);
  });
}

vie_status vie_program_info(const vie_op* h, int32_t which, int64_t* entries, int64_t* bytes, int64_t* launches,
                            int32_t cap, int32_t* nstages) {
  return guarded([&] {
    VIE_REQUIRE(h && nstages, VIE_EINVAL, "null argument");
    VIE_REQUIRE(which == VIE_OP_Z || (which == VIE_OP_ZINV && h->has_zinv), VIE_ENOTSUP, "no such operator");
    const Program& p = which == VIE_OP_Z ? h->z : h->zinv;
    *nstages = (int32_t)p.stages.size();
    for (int i = 0; i < (int)p.stages.size() && i < cap; ++i) {
      if (entries) entries[i] = p.stages[i].entries;
      if (bytes) bytes[i] = p.stages[i].bytes;
      if (launches) launches[i] = p.stages[i].ntiles;
    }
  });
}

vie_status vie_program_blocks(const vie_op* h, int32_t which, int32_t stage, int32_t* M, int32_t* K, int64_t cap,
                              int64_t* count) {
  return guarded([&] {
    VIE_REQUIRE(h && count, VIE_EINVAL, "null argument");
    VIE_REQUIRE(which == VIE_OP_Z || (which == VIE_OP_ZINV && h->has_zinv), VIE_ENOTSUP, "no such operator");
    const Program& p = which == VIE_OP_Z ? h->z : h->zinv;
    VIE_REQUIRE(stage >= 0 && stage < (int)p.stages.size(), VIE_EINVAL, "stage out of range");
    const auto& ops = p.stages[stage].host_ops;
    *count = (int64_t)ops.size();
    for (int64_t i = 0; i < (int64_t)ops.size() && i < cap; ++i) {
      if (M) M[i] = ops[i].M;
      if (K) K[i] = ops[i].K;
    }
  });
}

vie_status vie_autotune(vie_op* h, int32_t which, int32_t* choice, int32_t cap, void* stream) {
  return guarded([&] {
    VIE_REQUIRE(h, VIE_EINVAL, "null operator");
    VIE_REQUIRE(which == VIE_OP_Z || (which == VIE_OP_ZINV && h->has_zinv), VIE_ENOTSUP, "no such operator");
    Program& p = which == VIE_OP_Z ? h->z : h->zinv;
    VIE_REQUIRE(!choice || cap >= (int32_t)p.stages.size(), VIE_EINVAL, "choice array too short");
    ensure_ws(h, p, 1, VIE_C64);
    VIE_CUDA(cudaMemsetAsync(h->xt.p, 0, h->xt.bytes, (cudaStream_t)stream));
    VIE_CUDA(cudaMemsetAsync(h->yt.p, 0, h->yt.bytes, (cudaStream_t)stream));
    VIE_CUDA(cudaMemsetAsync(h->coef.p, 0, h->coef.bytes, (cudaStream_t)stream));
    program_autotune(p, h->xt.p, h->yt.p, h->coef.p, (cudaStream_t)stream, choice);
  });
}

vie_status vie_autotune_rhs(vie_op* h, int32_t which, int32_t* tc_min_rhs, void* stream) {
  return guarded([&] {
    if (h && (h->cfg.prec == VIE_P_C32 || h->cfg.prec == VIE_P_TC_BF16X3 ||
              h->cfg.prec == VIE_P_TC_TF32)) {  // the precision fixes the path
      Program& p = which == VIE_OP_ZINV ? h->zinv : h->z;
      if (tc_min_rhs) *tc_min_rhs = p.tc_min_rhs;
      return;
    }
    VIE_REQUIRE(h, VIE_EINVAL, "null operator");
    VIE_REQUIRE(which == VIE_OP_Z || (which == VIE_OP_ZINV && h->has_zinv), VIE_ENOTSUP, "no such operator");
    Program& p = which == VIE_OP_Z ? h->z : h->zinv;
    ensure_ws(h, p, 16, VIE_C64);
    VIE_CUDA(cudaMemsetAsync(h->xt.p, 0, h->xt.bytes, (cudaStream_t)stream));
    VIE_CUDA(cudaMemsetAsync(h->yt.p, 0, h->yt.bytes, (cudaStream_t)stream));
    VIE_CUDA(cudaMemsetAsync(h->coef.p, 0, h->coef.bytes, (cudaStream_t)stream));
    const int m = program_tune_rhs(p, h->xt.p, h->yt.p, h->coef.p, (cudaStream_t)stream);
    if (tc_min_rhs) *tc_min_rhs = m;
  });
}

vie_status vie_set_prec(vie_op* h, int32_t prec) {
  return guarded([&] {
    VIE_REQUIRE(h, VIE_EINVAL, "null operator");
    VIE_REQUIRE(prec == VIE_P_C32 || prec == VIE_P_TC_BF16X3 || prec == VIE_P_TC_TF32, VIE_EINVAL,
                "prec must be VIE_P_C32, VIE_P_TC_BF16X3 or VIE_P_TC_TF32");
    VIE_REQUIRE(h->z.factor_dtype == VIE_C64, VIE_EINVAL, "the operator has complex FP64 factors");
    const int never = 1 << 30;
    for (Program* p : {&h->z, &h->zinv, &h->zh, &h->zinvh}) {
      program_set_tc_variant(*p, prec == VIE_P_TC_TF32);
      p->tc_min_rhs = prec == VIE_P_C32 ? never : kTcMinRhs;
    }
    h->cfg.prec = prec;
  });
}

vie_status vie_set_tiling(vie_op* h, int32_t which, const int32_t* choice, int32_t n, void* stream) {
  return guarded([&] {
    VIE_REQUIRE(h && choice, VIE_EINVAL, "null argument");
    VIE_REQUIRE(which == VIE_OP_Z || (which == VIE_OP_ZINV && h->has_zinv), VIE_ENOTSUP, "no such operator");
    Program& p = which == VIE_OP_Z ? h->z : h->zinv;
    program_set_tiling(p, choice, n, (cudaStream_t)stream);
  });
}

vie_status vie_entries(vie_op* h, const int32_t* rows, const int32_t* cols, int64_t count, void* out, void* stream) {
  return guarded([&] {
    VIE_REQUIRE(h && (count == 0 || (rows && cols && out)), VIE_EINVAL, "null argument");
    VIE_REQUIRE(count >= 0, VIE_EINVAL, "negative count");
    entries_pairs(h->geo, rows, cols, count, (double2*)out, (cudaStream_t)stream);
  });
}

vie_status vie_rhs_planewave(vie_op* h, const double* khat, const double* pol, int64_t nrhs, void* V, void* stream) {
  return guarded([&] {
    VIE_REQUIRE(h && khat && pol && V && nrhs >= 1, VIE_EINVAL, "bad argument");
    rhs_planewave(h->geo, khat, pol, (int)nrhs, (double2*)V, (cudaStream_t)stream);
  });
}

vie_status vie_farfield(vie_op* h, const void* I, int64_t nrhs, const double* dirs, int64_t ndir, double* rcs,
                        void* stream) {
  return guarded([&] {
    VIE_REQUIRE(h && I && dirs && rcs && nrhs >= 1 && ndir >= 1, VIE_EINVAL, "bad argument");
    farfield_impl(h->geo, h->tet_faces.as<int32_t>(), (const double2*)I, (int)nrhs, dirs, (int)ndir, rcs,
                  (cudaStream_t)stream);
  });
}

vie_status vie_mesh_faces(const vie_op* h, int32_t* faces, int32_t* tp, int32_t* tm) {
  return guarded([&] {
    VIE_REQUIRE(h, VIE_EINVAL, "null operator");
    const int64_t n = h->mesh.nf;
    if (faces) std::memcpy(faces, h->mesh.faces.data(), sizeof(int32_t) * 3 * n);
    if (tp) std::memcpy(tp, h->mesh.tp.data(), sizeof(int32_t) * n);
    if (tm) std::memcpy(tm, h->mesh.tm.data(), sizeof(int32_t) * n);
  });
}

vie_status vie_mesh_host(const vie_voxels* body, int32_t leaf, int64_t* n, int32_t* faces, int32_t* tp, int32_t* tm,
                         int32_t* perm, int32_t* levels) {
  return guarded([&] {
    VIE_REQUIRE(body && n, VIE_EINVAL, "null argument");
    VIE_REQUIRE(body->nvox > 0 && body->ijk && body->eps && body->h > 0 && leaf >= 4, VIE_EINVAL, "invalid body");
    Mesh m;
    build_mesh(*body, m);
    *n = m.nf;
    if (faces) std::memcpy(faces, m.faces.data(), sizeof(int32_t) * 3 * m.nf);
    if (tp) std::memcpy(tp, m.tp.data(), sizeof(int32_t) * m.nf);
    if (tm) std::memcpy(tm, m.tm.data(), sizeof(int32_t) * m.nf);
    if (perm || levels) {
      const std::vector<double> pts = face_centroids(m);
      Tree t;
      build_tree(pts, leaf, t);
      if (perm) std::memcpy(perm, t.perm.data(), sizeof(int32_t) * m.nf);
      if (levels) *levels = t.levels;
    }
  });
}

vie_status vie_mesh_host_tets(const vie_mesh* mesh, int32_t leaf, int64_t* n, int32_t* faces, int32_t* tp,
                              int32_t* tm, int32_t* perm, int32_t* levels, int32_t* cells, double* cell_pitch) {
  return guarded([&] {
    VIE_REQUIRE(mesh && n && leaf >= 4, VIE_EINVAL, "null argument or leaf < 4");
    Mesh m;
    build_mesh_general(*mesh, m);
    *n = m.nf;
    if (faces) std::memcpy(faces, m.faces.data(), sizeof(int32_t) * 3 * m.nf);
    if (tp) std::memcpy(tp, m.tp.data(), sizeof(int32_t) * m.nf);
    if (tm) std::memcpy(tm, m.tm.data(), sizeof(int32_t) * m.nf);
    if (cells) std::memcpy(cells, m.cells.data(), sizeof(int32_t) * 3 * m.nt);
    if (cell_pitch) *cell_pitch = m.h;
    if (perm || levels) {
      Tree t;
      build_tree(face_centroids(m), leaf, t);
      if (perm) std::memcpy(perm, t.perm.data(), sizeof(int32_t) * m.nf);
      if (levels) *levels = t.levels;
    }
  });
}

vie_status vie_tree_perm(const vie_op* h, int32_t* perm) {
  return guarded([&] {
    VIE_REQUIRE(h && perm, VIE_EINVAL, "null argument");
    std::memcpy(perm, h->tree.perm.data(), sizeof(int32_t) * h->mesh.nf);
  });
}

vie_status vie_check(vie_op* h, void* stream) {
  return guarded([&] {
    VIE_REQUIRE(h, VIE_EINVAL, "null operator");
    for (Program* p : {&h->z, &h->zinv}) {
      if (!p->err.p) continue;
      int e = 0;
      VIE_CUDA(cudaMemcpyAsync(&e, p->err.p, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
      VIE_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
      if (e) {
        VIE_CUDA(cudaMemsetAsync(p->err.p, 0, sizeof(int), (cudaStream_t)stream));
        throw Error{VIE_ETIMEOUT, "a bounded wait in an apply kernel ran out; its output is invalid"};
      }
    }
  });
}

vie_status vie_wait_selftest(int32_t spins, void* stream) {
  return guarded([&] {
    VIE_REQUIRE(spins >= 1 && spins <= (1 << 20), VIE_EINVAL, "spins out of range [1, 2^20]");
    DevBuf st;
    st.alloc(sizeof(int));
    VIE_CUDA(cudaMemsetAsync(st.p, 0, sizeof(int), (cudaStream_t)stream));
    wait_timeout_check((uint32_t)spins, st.as<int>(), (cudaStream_t)stream);
    int h = 0;
    VIE_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    VIE_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (h) throw Error{VIE_ETIMEOUT, "bounded device wait ran out (expected in this self-test)"};
  });
}

vie_status vie_stats(const vie_op* h, vie_stats_t* out) {
  return guarded([&] {
    VIE_REQUIRE(h && out, VIE_EINVAL, "null argument");
    *out = h->stats;
  });
}

vie_status vie_solve(vie_op* h, const void* V, void* I, int64_t nrhs, double rtol, int32_t restart, int32_t max_iter,
                     int32_t* iters, double* relres, void* stream) {
  bool conv = true;
  vie_status st = guarded([&] {
    VIE_REQUIRE(h && V && I && nrhs >= 1, VIE_EINVAL, "bad argument");
    VIE_REQUIRE(rtol > 0 && restart >= 1 && max_iter >= 1, VIE_EINVAL, "bad tolerance or iteration limits");
    solve_gmres(h, (const double2*)V, (double2*)I, nrhs, rtol, restart, max_iter, iters, relres,
                (cudaStream_t)stream, conv);
  });
  if (st == VIE_OK && !conv) {
    set_error("GMRES stopped before reaching rtol");
    return VIE_ENOTCONV;
  }
  return st;
}

vie_status vie_solve_tfqmr(vie_op* h, const void* V, void* I, int64_t nrhs, double rtol, int32_t max_iter,
                           int32_t* iters, double* relres, void* stream) {
  bool conv = true;
  vie_status st = guarded([&] {
    VIE_REQUIRE(h && V && I && nrhs >= 1, VIE_EINVAL, "bad argument");
    VIE_REQUIRE(rtol > 0 && max_iter >= 1, VIE_EINVAL, "bad tolerance or iteration limit");
    solve_tfqmr(h, (const double2*)V, (double2*)I, nrhs, rtol, max_iter, iters, relres, (cudaStream_t)stream, conv);
  });
  if (st == VIE_OK && !conv) {
    set_error("TFQMR stopped before reaching rtol");
    return VIE_ENOTCONV;
  }
  return st;
}

}  // extern "C"
