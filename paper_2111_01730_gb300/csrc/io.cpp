// Checkpoint of a built operator: vie_save / vie_load.
//
// A build (entries, IDs, the inverse from products) costs minutes at the
// workload sizes; the apply programs it produces are plain data.  The file
// holds the inputs the host needs to remake the mesh, tree and interaction
// tables (voxel lattice, permittivities, k0, configuration), the statistics,
// and every stage of the Z and Zinv programs exactly as the apply runs them:
// block descriptors, tags, warp tiles with the single-RHS kernel choice, and
// the packed factor bytes.  Loading re-uploads them, so applies of a loaded
// operator are bit-identical to applies of the saved one.
//
// Layout (little-endian, native struct layout of this library):
//   "VIEOPv1\0", vie_config, double k0, double h, then the body: int64 nvox,
//   int32 ijk[3 nvox], double eps[2 nvox] (voxels), or int64 -1, int64 nv,
//   double xyz[3 nv], int64 nt, int32 tet[4 nt], double eps[2 nt] (a tet mesh);
//   vie_stats_t, int32 has_zinv, int32 zinv_top_level,
//   int32 tc_min_rhs(Z), int32 tc_min_rhs(Zinv), then each program:
//   int64 n, ncoef, entries, bytes; int32 factor_dtype, nstages; per stage:
//   int64 nops, ntiles, mats_bytes, entries, bytes; int32 kernel, pad;
//   OpDesc[nops], int32 tag[nops], Tile[ntiles], mats bytes.
#include <cstdio>
#include <cstring>
#include <memory>

#include "internal.h"

namespace vie {

namespace {

constexpr char kMagic[8] = {'V', 'I', 'E', 'O', 'P', 'v', '1', '\0'};
constexpr size_t kChunk = size_t(256) << 20;  // host staging for factor bytes

struct File {
  FILE* f = nullptr;
  ~File() { if (f) std::fclose(f); }
};

void wr(FILE* f, const void* p, size_t n) {
  if (n && std::fwrite(p, 1, n, f) != n) throw Error{VIE_EINVAL, "vie_save: write failed"};
}
void rd(FILE* f, void* p, size_t n) {
  if (n && std::fread(p, 1, n, f) != n) throw Error{VIE_EINVAL, "vie_load: truncated or unreadable file"};
}
template <class T> void wrv(FILE* f, const T& v) { wr(f, &v, sizeof(T)); }
template <class T> T rdv(FILE* f) { T v; rd(f, &v, sizeof(T)); return v; }

void save_program(FILE* f, const Program& p, cudaStream_t s) {
  wrv(f, p.n); wrv(f, p.ncoef); wrv(f, p.entries); wrv(f, p.bytes);
  wrv<int32_t>(f, p.factor_dtype);
  wrv<int32_t>(f, (int32_t)p.stages.size());
  std::unique_ptr<char[]> buf(new char[kChunk]);
  for (const Stage& st : p.stages) {
    wrv<int64_t>(f, (int64_t)st.host_ops.size());
    wrv<int64_t>(f, st.ntiles);
    wrv<int64_t>(f, (int64_t)st.mats.bytes);
    wrv(f, st.entries); wrv(f, st.bytes);
    wrv<int32_t>(f, st.kernel); wrv<int32_t>(f, 0);
    wr(f, st.host_ops.data(), sizeof(OpDesc) * st.host_ops.size());
    std::vector<int32_t> tag(st.host_ops.size(), -1);
    for (size_t i = 0; i < tag.size() && i < st.host_tag.size(); ++i) tag[i] = st.host_tag[i];
    wr(f, tag.data(), sizeof(int32_t) * tag.size());
    std::vector<Tile> tiles((size_t)st.ntiles);
    if (st.ntiles)
      VIE_CUDA(cudaMemcpyAsync(tiles.data(), st.tiles.p, sizeof(Tile) * tiles.size(), cudaMemcpyDeviceToHost, s));
    VIE_CUDA(cudaStreamSynchronize(s));
    wr(f, tiles.data(), sizeof(Tile) * tiles.size());
    for (size_t off = 0; off < st.mats.bytes; off += kChunk) {
      const size_t n = std::min(kChunk, st.mats.bytes - off);
      VIE_CUDA(cudaMemcpyAsync(buf.get(), (const char*)st.mats.p + off, n, cudaMemcpyDeviceToHost, s));
      VIE_CUDA(cudaStreamSynchronize(s));
      wr(f, buf.get(), n);
    }
  }
}

void load_program(FILE* f, Program& p, cudaStream_t s) {
  p.stages.clear();
  p.n = rdv<int64_t>(f); p.ncoef = rdv<int64_t>(f); p.entries = rdv<int64_t>(f); p.bytes = rdv<int64_t>(f);
  p.factor_dtype = rdv<int32_t>(f);
  const int32_t ns = rdv<int32_t>(f);
  VIE_REQUIRE(p.factor_dtype == VIE_C64 || p.factor_dtype == VIE_C128, VIE_EINVAL, "vie_load: bad factor type");
  VIE_REQUIRE(ns >= 0 && ns < 1 << 16, VIE_EINVAL, "vie_load: bad stage count");
  std::unique_ptr<char[]> buf(new char[kChunk]);
  p.stages.resize(ns);
  for (Stage& st : p.stages) {
    const int64_t nops = rdv<int64_t>(f), ntiles = rdv<int64_t>(f), mb = rdv<int64_t>(f);
    st.entries = rdv<int64_t>(f); st.bytes = rdv<int64_t>(f);
    st.kernel = rdv<int32_t>(f); (void)rdv<int32_t>(f);
    VIE_REQUIRE(nops >= 0 && ntiles >= 0 && mb >= 0, VIE_EINVAL, "vie_load: bad stage header");
    st.host_ops.resize(nops);
    rd(f, st.host_ops.data(), sizeof(OpDesc) * nops);
    st.host_tag.resize(nops);
    rd(f, st.host_tag.data(), sizeof(int32_t) * nops);
    std::vector<Tile> tiles(ntiles);
    rd(f, tiles.data(), sizeof(Tile) * ntiles);
    st.nops = nops;
    st.ntiles = ntiles;
    st.ops.alloc(sizeof(OpDesc) * std::max<int64_t>(1, nops));
    st.tiles.alloc(sizeof(Tile) * std::max<int64_t>(1, ntiles));
    if (nops) VIE_CUDA(cudaMemcpyAsync(st.ops.p, st.host_ops.data(), sizeof(OpDesc) * nops, cudaMemcpyHostToDevice, s));
    if (ntiles) VIE_CUDA(cudaMemcpyAsync(st.tiles.p, tiles.data(), sizeof(Tile) * ntiles, cudaMemcpyHostToDevice, s));
    st.mats.alloc((size_t)std::max<int64_t>(mb, 16));
    for (int64_t off = 0; off < mb; off += (int64_t)kChunk) {
      const size_t n = (size_t)std::min<int64_t>((int64_t)kChunk, mb - off);
      rd(f, buf.get(), n);
      VIE_CUDA(cudaMemcpyAsync((char*)st.mats.p + off, buf.get(), n, cudaMemcpyHostToDevice, s));
      VIE_CUDA(cudaStreamSynchronize(s));
    }
  }
  program_check(p);
}

}  // namespace

}  // namespace vie

using namespace vie;

extern "C" vie_status vie_save(const vie_op* h, const char* path, void* stream) {
  try {
    VIE_REQUIRE(h && path, VIE_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    File F;
    F.f = std::fopen(path, "wb");
    VIE_REQUIRE(F.f, VIE_EINVAL, std::string("vie_save: cannot open ") + path);
    FILE* f = F.f;
    wr(f, kMagic, sizeof(kMagic));
    wrv(f, h->cfg);
    wrv(f, h->geo.k0);
    wrv(f, h->mesh.h);
    if (h->mesh.general) {  // body: -1, then the tet mesh as given
      wrv<int64_t>(f, -1);
      wrv(f, h->mesh.nv);
      wr(f, h->mesh.xyz.data(), sizeof(double) * h->mesh.xyz.size());
      wrv(f, h->mesh.nt);
      wr(f, h->mesh.tets.data(), sizeof(int32_t) * h->mesh.tets.size());
      wr(f, h->mesh.eps.data(), sizeof(double) * h->mesh.eps.size());
    } else {
      wrv(f, h->mesh.nvox);
      wr(f, h->mesh.vox.data(), sizeof(int32_t) * h->mesh.vox.size());
      wr(f, h->mesh.eps.data(), sizeof(double) * h->mesh.eps.size());
    }
    wrv(f, h->stats);
    wrv<int32_t>(f, h->has_zinv ? 1 : 0);
    wrv<int32_t>(f, h->zinv_top_level);
    wrv<int32_t>(f, h->z.tc_min_rhs);
    wrv<int32_t>(f, h->zinv.tc_min_rhs);
    save_program(f, h->z, s);
    if (h->has_zinv) save_program(f, h->zinv, s);
    VIE_REQUIRE(std::fflush(f) == 0, VIE_EINVAL, "vie_save: write failed");
    return VIE_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    set_error(e.what());
    return VIE_EINVAL;
  }
}

extern "C" vie_status vie_load(const char* path, void* stream, vie_op** out) {
  vie_op* h = nullptr;
  try {
    VIE_REQUIRE(path && out, VIE_EINVAL, "null argument");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    File F;
    F.f = std::fopen(path, "rb");
    VIE_REQUIRE(F.f, VIE_EINVAL, std::string("vie_load: cannot open ") + path);
    FILE* f = F.f;
    char magic[8];
    rd(f, magic, sizeof(magic));
    VIE_REQUIRE(std::memcmp(magic, kMagic, sizeof(kMagic)) == 0, VIE_EINVAL, "vie_load: not an operator file");
    h = new vie_op();
    h->cfg = rdv<vie_config>(f);
    VIE_REQUIRE(h->cfg.leaf >= 4 && h->cfg.tol_con > 0 &&
                    (h->cfg.factor_dtype == VIE_C64 || h->cfg.factor_dtype == VIE_C128) &&
                    h->cfg.prec >= VIE_P_AUTO && h->cfg.prec <= VIE_P_TC_TF32,
                VIE_EINVAL, "vie_load: bad configuration");
    const double k0 = rdv<double>(f), hh = rdv<double>(f);
    const int64_t nvox = rdv<int64_t>(f);
    VIE_REQUIRE((nvox > 0 || nvox == -1) && nvox < (int64_t(1) << 34) && hh > 0 && k0 > 0, VIE_EINVAL,
                "vie_load: bad body header");
    // mesh, tree and interaction tables remade from the inputs (deterministic host code)
    if (nvox == -1) {
      const int64_t nv = rdv<int64_t>(f);
      VIE_REQUIRE(nv >= 4 && nv < (int64_t(1) << 31), VIE_EINVAL, "vie_load: bad vertex count");
      std::vector<double> xyz(3 * nv);
      rd(f, xyz.data(), sizeof(double) * xyz.size());
      const int64_t nt = rdv<int64_t>(f);
      VIE_REQUIRE(nt >= 1 && nt < (int64_t(1) << 29), VIE_EINVAL, "vie_load: bad tet count");
      std::vector<int32_t> tet(4 * nt);
      std::vector<double> eps(2 * nt);
      rd(f, tet.data(), sizeof(int32_t) * tet.size());
      rd(f, eps.data(), sizeof(double) * eps.size());
      const vie_mesh mm{nv, xyz.data(), nt, tet.data(), eps.data()};
      build_mesh_general(mm, h->mesh);
      geometry_upload(h->mesh, k0, h->geo, s);
    } else {
      std::vector<int32_t> ijk(3 * nvox);
      std::vector<double> eps(2 * nvox);
      rd(f, ijk.data(), sizeof(int32_t) * ijk.size());
      rd(f, eps.data(), sizeof(double) * eps.size());
      const vie_voxels body{nvox, ijk.data(), eps.data(), hh};
      build_mesh(body, h->mesh);
      geometry_upload(h->mesh, k0, h->geo, s);
      geometry_table(h->geo, s);
    }
    const int64_t N = h->mesh.nf;
    const std::vector<double> pts = face_centroids(h->mesh);
    build_tree(pts, h->cfg.leaf, h->tree);
    h->perm.alloc(sizeof(int32_t) * N);
    VIE_CUDA(cudaMemcpyAsync(h->perm.p, h->tree.perm.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
    h->tet_faces.alloc(sizeof(int32_t) * 4 * h->mesh.nt);
    VIE_CUDA(cudaMemcpyAsync(h->tet_faces.p, h->mesh.tet_faces.data(), sizeof(int32_t) * 4 * h->mesh.nt,
                             cudaMemcpyHostToDevice, s));
    h->stats = rdv<vie_stats_t>(f);
    VIE_REQUIRE(h->stats.n == N, VIE_EINVAL, "vie_load: the file's operator does not match its mesh");
    h->has_zinv = rdv<int32_t>(f) != 0;
    h->zinv_top_level = rdv<int32_t>(f);
    const int32_t tcz = rdv<int32_t>(f), tci = rdv<int32_t>(f);
    load_program(f, h->z, s);
    h->z.tc_min_rhs = tcz;
    VIE_REQUIRE(h->z.n == N, VIE_EINVAL, "vie_load: program size does not match the mesh");
    if (h->has_zinv) {
      load_program(f, h->zinv, s);
      h->zinv.tc_min_rhs = tci;
    }
    for (Program* pp : {&h->z, &h->zinv}) {  // the wait flag of the bounded-wait kernels
      pp->err.alloc(sizeof(int));
      VIE_CUDA(cudaMemsetAsync(pp->err.p, 0, sizeof(int), s));
      pp->tc_tf32 = h->cfg.prec == VIE_P_TC_TF32;
    }
    VIE_CUDA(cudaStreamSynchronize(s));
    *out = h;
    return VIE_OK;
  } catch (const Error& e) {
    delete h;
    set_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    delete h;
    set_error("vie_load: host allocation failed (corrupt file?)");
    return VIE_ENOMEM;
  } catch (const std::exception& e) {
    delete h;
    set_error(e.what());
    return VIE_EINVAL;
  }
}
