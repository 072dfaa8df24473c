// Internal declarations shared by the translation units of libvie.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vie.h"

namespace vie {

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

// Tracing: an NVTX range for the lifetime of the object ("vie:<phase>"), shown by
// Nsight Systems and other NVTX tools; without a tool attached the calls do nothing.
struct Trace {
  explicit Trace(const char* name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace&) = delete;
  Trace& operator=(const Trace&) = delete;
};

struct Error {
  vie_status status;
  std::string msg;
};

#define VIE_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw ::vie::Error{VIE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define VIE_REQUIRE(cond, status, msg)                   \
  do {                                                   \
    if (!(cond)) throw ::vie::Error{(status), (msg)};    \
  } while (0)

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current device,
// once per (device, kernel); thread safe.  cudaFuncSetAttribute acts per device,
// so a process-wide flag would leave a second device at the default limit.
void ensure_smem_attr(const void* kernel, int bytes);
// Per-device one-time set-up flags keyed by an address: done_on_device asks,
// mark_on_device records (current device); thread safe.
bool done_on_device(const void* key);
void mark_on_device(const void* key);

// ---------------------------------------------------------------------------
// device memory owned by the operator
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t n);
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------------------
// mesh (host): voxels -> Kuhn tets -> faces (SWG table), Sec. II / Eq. (3)
// ---------------------------------------------------------------------------
struct Mesh {
  double h = 0;                    // voxel pitch; general meshes: the tier-cell pitch
  int64_t nvox = 0, nt = 0, nf = 0, nv = 0;
  bool general = false;            // built from a vie_mesh (vertex coordinates, any tets)
  std::vector<int32_t> vox;        // 3*nvox
  std::vector<double> eps;         // 2*nvox (voxel meshes) or 2*nt (general meshes)
  std::vector<int32_t> tets;       // 4*nt vertex ids
  std::vector<int32_t> vlat;       // 3*nv lattice coordinates of the vertices (voxel meshes)
  std::vector<double> xyz;         // 3*nv vertex coordinates (general meshes)
  std::vector<int32_t> cells;      // 3*nt tier cells of the tets (general meshes)
  std::vector<int32_t> faces;      // 3*nf sorted vertex ids
  std::vector<int32_t> tp, tm, lp, lm;  // nf: T+, T-, local face index in T+ / T-
  std::vector<int32_t> tet_faces;  // 4*nt
};
void build_mesh(const vie_voxels& body, Mesh& m);
void build_mesh_general(const vie_mesh& mesh, Mesh& m);
std::vector<double> face_centroids(const Mesh& m);  // 3*nf, ((a + b) + c) / 3 per coordinate

// Kuhn tetrahedra: offsets of the 4 vertices of the 6 types from the voxel corner.
extern const int kKuhn[6][4][3];

// ---------------------------------------------------------------------------
// cluster tree (host), Sec. III-A
// ---------------------------------------------------------------------------
struct Tree {
  int levels = 0;                       // L_H
  std::vector<int32_t> perm;            // tree position -> original face
  std::vector<std::vector<int64_t>> bounds;  // bounds[l]: 2^l + 1 offsets
  std::vector<std::vector<double>> bbox;     // bbox[l]: 6 doubles per node (lo xyz, hi xyz)
};
void build_tree(const std::vector<double>& pts /*3n*/, int leaf, Tree& t);

// ---------------------------------------------------------------------------
// quadrature rules (host), barycentric with weights summing to 1
// ---------------------------------------------------------------------------
struct Rule {
  int n = 0;
  std::vector<double> lam;  // n * (4 or 3)
  std::vector<double> w;
};
Rule rule_tet4();
Rule rule_tri3();
Rule rule_tet_conical(int n);
Rule rule_tri_conical(int n);

// ---------------------------------------------------------------------------
// device geometry + entry evaluator (entries.cu)
// ---------------------------------------------------------------------------
struct FaceDev {
  int32_t tp, tm;      // owner tets (tm = -1 on the boundary)
  int8_t lp, lm;       // local face indices
  int8_t boundary;     // half-SWG: test surface density -1
  int8_t pad;
  double jump_re, jump_im;  // source surface density kappa(T-) - kappa(T+)
};

struct TetDev {
  int32_t vx, vy, vz;  // voxel (general meshes: the tier cell)
  int32_t type;        // Kuhn type 0..5 (general meshes: -1)
  double kap_re, kap_im;      // kappa
  double inveps_re, inveps_im;
};

struct TetGeo {        // a tet of a general mesh
  double P[4][3];      // vertices in the mesh's order
  double vol;
  double area[4];      // area of local face a (opposite vertex a)
  double nrm[4][3];    // outward unit normal of local face a
  int8_t fv[4][3];     // local vertices of face a in increasing global vertex id
  int8_t pad[4];
  int32_t vid[4];      // global vertex ids (tets sharing one are near)
};

struct Geometry {
  int64_t n = 0, nt = 0;
  double h = 0, k0 = 0;
  bool general = false;
  DevBuf faces;   // FaceDev[n]
  DevBuf tets;    // TetDev[nt]
  DevBuf table;   // near / mid tier interaction table (FP64), voxel meshes
  DevBuf geo;     // TetGeo[nt], general meshes
};
void geometry_upload(const Mesh& m, double k0, Geometry& g, cudaStream_t s);
void geometry_table(Geometry& g, cudaStream_t s);   // computes the near/mid table

// One dense block of Z to evaluate: out[i + j*ld] = Z(rows[i], cols[j]) (col-major, c128).
struct EntryBlock {
  int64_t out_off;   // element offset into the output pool
  int64_t row_off;   // offset into the row index pool
  int64_t col_off;   // offset into the col index pool
  int32_t m, n;      // rows, cols
};
void entries_blocks(const Geometry& g, const EntryBlock* d_blocks, const int64_t* d_prefix,
                    int nblocks, int64_t total, const int32_t* d_rows, const int32_t* d_cols,
                    double2* d_out, cudaStream_t s);
void entries_pairs(const Geometry& g, const int32_t* rows, const int32_t* cols, int64_t count,
                   double2* out, cudaStream_t s, bool far32 = false);
void rhs_planewave(const Geometry& g, const double* khat, const double* pol, int nrhs, double2* V,
                   cudaStream_t s);

// ---------------------------------------------------------------------------
// batched interpolative decomposition (id.cu), Eq. (7)
// ---------------------------------------------------------------------------
struct IdJob {
  int64_t a_off;   // col-major m x n input (destroyed), c128
  int64_t v_off;   // row-major r x n output V = [I T] P^T, c128 (space min(m,n)*n)
  int64_t p_off;   // n ints: pivot order (first r = skeleton)
  int32_t m, n;
  double tol;      // truncation |R_kk| <= tol |R_11| of this job (<= 0: the batch's tolerance)
};
void id_batched(const IdJob* d_jobs, int njobs, int max_n, double2* d_a, double2* d_v, int32_t* d_piv,
                int32_t* d_rank, double tol, cudaStream_t s, bool single = false);

// ---------------------------------------------------------------------------
// apply program (apply.cu)
// ---------------------------------------------------------------------------
enum Space : int32_t { SP_X = 0, SP_Y = 1, SP_C = 2 };

struct OpDesc {          // y[out] (=|+=) A (M x K, row-major, ld) * x[in]
  int64_t mat_off;       // element offset of A in the stage's matrix buffer
  int64_t in_off, out_off;
  int32_t M, K, ld;
  int16_t in_space, out_space;
  int32_t accumulate;    // 0: assign, 1: add
  int32_t pad;
};

struct Tile {            // a warp's unit of work: rows [r0, r0 + nr) of op `op`
  int32_t op, r0, nr, g; // g = lanes per row (power of two)
};

// A tensor-core work item: up to 64 output rows taken from up to kTcMaxSeg
// blocks of one stage that read the same input slice (so the slice is converted
// once for all of them).
constexpr int kTcMaxSeg = 8;
struct TcSeg {
  int64_t mat_off, out_off;  // c64 matrix offset, output row offset of the block
  int32_t ld, row0;          // block row stride; first block row in this item
  int32_t rows, start;       // rows taken; first item row they occupy
  int16_t out_space, accumulate;
  int32_t pad;
};
struct TcItem {
  int64_t b_off, in_off;     // bf16 tile byte offset; input row offset
  int32_t K, n, mc, nseg;    // K columns, n = mc rounded up to 16 (the MMA's N), mc rows
  int16_t in_space, pad16;
  int32_t pad;
  TcSeg seg[kTcMaxSeg];
};

constexpr int kTcMinRhs = 16;  // default smallest right-hand-side count on the tensor cores

// single-RHS stage kernels the autotuner chooses from
constexpr int kKernelPlain4 = 0;  // stage1_kernel<4>: streaming loads, four 16-byte loads in flight per lane
constexpr int kKernelBulk = 1;    // stage1_bulk_kernel: tiles staged in shared memory by bulk copies
constexpr int kKernelPlain8 = 2;  // stage1_kernel<8>: eight loads in flight per lane, lower occupancy

struct Stage {
  DevBuf mats;           // packed factor matrices (c64 or c128)
  DevBuf ops;            // OpDesc[nops]
  DevBuf tiles;          // Tile[ntiles]
  int64_t nops = 0, ntiles = 0, entries = 0, bytes = 0;
  int kernel = 0;        // single RHS c64: kKernelPlain4, kKernelBulk or kKernelPlain8
  std::vector<OpDesc> host_ops;  // kept for the tensor-core preparation
  std::vector<int32_t> host_tag; // per op: tree level of its butterfly's row node (-1: leaf block)
  // tensor-core (multi-RHS) form, prepared on first use
  DevBuf tc_tiles, tc_ops, rest_ops, rest_tiles;
  int64_t tc_items = 0, tc_bytes = 0, rest_ntiles = 0;
  bool tc_tf32 = false;  // tiles packed for the TF32 variant (else BF16x3)
};

struct Program {         // one operator's apply: gather, stages, scatter
  std::vector<Stage> stages;
  int64_t n = 0, ncoef = 0;
  int factor_dtype = VIE_C64;
  int64_t entries = 0, bytes = 0;
  bool tc_ready = false;
  int tc_min_rhs = kTcMinRhs;  // applies with at least this many columns use the tensor cores
  bool tc_tf32 = false;        // tensor-core variant: TF32 (VIE_P_TC_TF32) or BF16x3
  DevBuf err;            // device int: a bounded wait in a tensor-core kernel ran out
  // CUDA graphs of the stage launches (the gather and scatter stay outside: they
  // touch the caller's X and Y), one per (nrhs, dtype, path, workspaces), least
  // recently used evicted beyond kGraphCache
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t nrhs = -1;
    int dtype = -1;
    bool tc = false;
    const void *xt = nullptr, *yt = nullptr, *coef = nullptr;
    uint64_t used = 0;
  };
  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;
  cudaStream_t capture_stream = nullptr;
  Program() = default;
  Program(const Program&) = delete;
  Program& operator=(const Program&) = delete;
  ~Program() {
    for (auto& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    if (capture_stream) cudaStreamDestroy(capture_stream);
  }
};

// Grouped launches (group.cu): one launch runs the work of one stage of up to
// kGroupMax operators, each with its own factors, vectors and column count.  The
// segment table travels in the kernel's parameters (no upload, graph-capturable);
// a work index finds its segment by a scan over the segments' first indices.
constexpr int kGroupMax = 16;
struct SimtSeg {         // SIMT tiles of one operator's stage
  const OpDesc* ops;
  const Tile* tiles;
  const float2* mats;
  const float2* xt;
  float2* yt;
  float2* coef;
  int64_t begin;         // first global tile index of the segment
  int32_t nrhs, pad;
};
struct SimtGroup {
  SimtSeg s[kGroupMax];
  int64_t total;         // tiles of all segments
  int32_t n, pad;
};
struct TcSeg2 {          // tensor-core items of one operator's stage
  const TcItem* items;
  const uint8_t* btiles;
  const float2* xt;
  float2* yt;
  float2* coef;
  int* err;              // set when a bounded wait of this segment's work ran out
  int64_t begin;         // first global work index (items x 128-column chunks)
  int32_t nitems, nrhs;
};
struct TcGroup {
  TcSeg2 s[kGroupMax];
  int64_t total;
  int32_t n, tf32;       // every segment of a launch has tiles of the same variant
};
void simt_launch_group(const SimtGroup& g, cudaStream_t s);
struct Program;
struct GroupJob {        // one operator's stages in a grouped apply, on tree-ordered work vectors
  const Program* p;
  int64_t nrhs;
  float2* xt;
  float2* yt;
  float2* coef;
};
// stage d of every job in launch d (c64 factors and vectors); tensor-core items for
// jobs with at least the program's tensor-core column count (prepared beforehand)
void group_run_stages(const std::vector<GroupJob>& jobs, cudaStream_t s);

// tensor-core multi-RHS path (tc.cu)
bool tc_eligible(const OpDesc& o);
void tc_prepare_stage(Stage& st, const std::vector<OpDesc>& ops, bool tf32, cudaStream_t s);
void tc_launch(const Stage& st, const void* xt, void* yt, void* coef, int nrhs, int* d_err, cudaStream_t s);
void tc_launch_group(const TcGroup& g, cudaStream_t s);
int64_t tc_work_units(int64_t items, int nrhs);  // work indices of a segment: items x 128-column chunks
size_t tc_smem_bytes();
void wait_timeout_check(uint32_t spins, int* d_status, cudaStream_t s);
constexpr size_t kGraphCache = 8;
constexpr int64_t kDenseInverseLimit = 65536;  // largest diagonal block formed densely by the inverse builder

void make_tiles(const std::vector<OpDesc>& ops, std::vector<Tile>& tiles);
void make_tiles(const std::vector<OpDesc>& ops, std::vector<Tile>& tiles, int64_t max_tile_bytes, int vec_target);
void program_apply(const Program& p, const int32_t* d_perm, const void* X, void* Y, int64_t nrhs,
                   int64_t ldx, int64_t ldy, int dtype, void* d_xt, void* d_yt, void* d_c,
                   cudaStream_t s, cudaEvent_t* events = nullptr);
void program_apply_adjoint(const Program& adj, const int32_t* d_perm, const void* X, void* Y, int64_t nrhs,
                           int64_t ldx, int64_t ldy, int dtype, void* d_xt, void* d_yt, void* d_c, cudaStream_t s);
// the stages alone on tree-ordered work vectors (rows x nrhs, rhs fastest): no permutation
void program_run(const Program& p, int64_t nrhs, int dtype, void* xt, void* yt, void* coef, cudaStream_t s);
// program construction helpers (program.cu)
void stage_set(Stage& st, std::vector<OpDesc> ops, DevBuf&& mats, int64_t elems, int elem_bytes, cudaStream_t s);
void program_totals(Program& p);
void program_check(const Program& p);
bool program_finite(const Program& p, cudaStream_t s);  // every stored factor entry finite  // every block inside its vector spaces and matrix buffer (host)
void program_adjoint(const Program& fwd, Program& adj, cudaStream_t s);
void program_filter(const Program& src, int32_t tag, Program& out, cudaStream_t s);
void program_relocate_coef(Program& p, int64_t shift, cudaStream_t s);
void program_compact_coef(Program& p, cudaStream_t s);  // coefficient memory shared by lifetime
void program_restrict_rows(const Program& p, int64_t lo, int64_t hi, Program& out, cudaStream_t s);
void program_append(Program& dst, Program&& src, cudaStream_t s);
void program_prepend(Program& dst, Program&& src);
// same, with the stage launches replayed from a cached CUDA graph
void program_apply_graph(Program& p, const int32_t* d_perm, const void* X, void* Y, int64_t nrhs, int64_t ldx,
                         int64_t ldy, int dtype, void* d_xt, void* d_yt, void* d_c, cudaStream_t s);
int64_t program_launches(const Program& p, int64_t nrhs, int dtype);
void program_prepare_tc(Program& p, cudaStream_t s);
// switch the tensor-core variant; drops the prepared tiles and the captured graphs
void program_set_tc_variant(Program& p, bool tf32);
int program_autotune(Program& p, void* xt, void* yt, void* coef, cudaStream_t s, int32_t* choice);
void program_set_tiling(Program& p, const int32_t* choice, int n, cudaStream_t s);
int program_tune_rhs(Program& p, void* xt, void* yt, void* coef, cudaStream_t s);
void pack_matrices(const double2* src, const int64_t* d_src_off, const int32_t* d_src_ld,
                   const int32_t* d_src_colmajor, const int64_t* d_dst_off, const int32_t* d_M,
                   const int32_t* d_K, const int32_t* d_ld, int nmat, void* dst, int dst_dtype,
                   cudaStream_t s);

struct BuildResult {
  int64_t entries_evaluated = 0;
  int64_t leaf_entries = 0;
  int max_rank = 0;
  double t_entries = 0, t_id = 0, t_host = 0;  // seconds (entries incl. transfers, batched IDs, host sampling)
};

// Where the builder takes matrix entries from (tree positions in, c128 col-major blocks out).
struct EntrySource {
  virtual ~EntrySource() = default;
  // Row ranges [row_lo[q], row_hi[q]) of the row node of each job of the next eval (ID jobs
  // only; -1 for the others).  A source may return, for an ID job whose m rows are a sample
  // of that range, m other rows with the same column geometry (e.g. a Gaussian sketch).
  virtual void set_row_ranges(const std::vector<int64_t>& /*row_lo*/, const std::vector<int64_t>& /*row_hi*/) {}
  virtual void eval(const std::vector<EntryBlock>& eb, const std::vector<int64_t>& prefix,
                    const std::vector<int32_t>& rows, const std::vector<int32_t>& cols,
                    const std::vector<int32_t>& srcs, int64_t total, double2* dA, cudaStream_t s) = 0;
};

// One butterfly to build: row node o and column node s at tree level `level`.
struct BfSpec {
  int level;
  int64_t o, s;
  int src;
};

}  // namespace vie

struct vie_op;
namespace vie {
struct ZEntrySource : EntrySource {
  vie_op* h;
  explicit ZEntrySource(vie_op* hh) : h(hh) {}
  void eval(const std::vector<EntryBlock>& eb, const std::vector<int64_t>& prefix, const std::vector<int32_t>& rows,
            const std::vector<int32_t>& cols, const std::vector<int32_t>& srcs, int64_t total, double2* dA,
            cudaStream_t s) override;
};
void build_hodbf(vie_op* h, cudaStream_t s, BuildResult& res);
void build_program(vie_op* h, const std::vector<BfSpec>& specs, EntrySource& src, double tol, Program& P,
                   bool leaf_blocks, int v0_space, cudaStream_t s, BuildResult& res);
void build_inverse(vie_op* h, cudaStream_t s, BuildResult& res);
void shard_forget(const vie_op* h);  // drop the operator's sharded sub-programs
struct InverseProductStats {
  int levels = 0;         // Algorithm 1 levels built from products
  int64_t products = 0;   // columns multiplied by an operator or its adjoint
  double seconds = 0, id_seconds = 0;
};
void build_inverse_products(vie_op* h, int l_top, double tol, cudaStream_t s, InverseProductStats& st);
void ensure_ws(vie_op* h, const Program& p, int64_t nrhs, int dtype);
void op_apply(vie_op* h, int which, const void* X, void* Y, int64_t nrhs, int dtype, cudaStream_t s);
void solve_gmres(vie_op* h, const double2* b, double2* x_out, int64_t nrhs, double rtol, int restart, int max_iter,
                 int32_t* iters_out, double* relres_out, cudaStream_t s, bool& converged_all);
void solve_tfqmr(vie_op* h, const double2* b, double2* x_out, int64_t nrhs, double rtol, int max_iter,
                 int32_t* iters_out, double* relres_out, cudaStream_t s, bool& converged_all);
void farfield_impl(const Geometry& g, const int32_t* d_tet_faces, const double2* I, int nrhs, const double* dirs,
                   int ndir, double* rcs, cudaStream_t s);
}  // namespace vie

// The operator handle
struct vie_op {
  vie::Mesh mesh;
  vie::Tree tree;
  vie::Geometry geo;
  vie::DevBuf perm;      // int32 tree -> original
  vie::DevBuf tet_faces; // int32 4*nt
  vie::Program z, zinv;
  vie::Program zh, zinvh;   // adjoint programs, built on the first adjoint apply
  bool zh_ready = false, zinvh_ready = false;
  bool has_zinv = false;
  int zinv_top_level = 0;   // Algorithm 1 levels l >= this are in Zinv
  vie::DevBuf xt, yt, coef;  // apply workspaces (grown on demand)
  size_t ws_bytes = 0;
  vie_config cfg{};
  vie_stats_t stats{};
};
