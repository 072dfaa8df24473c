/*
 * vie.h — C ABI of the GB300 butterfly-accelerated VIE library.
 *
 * The library applies the HOD-BF compressed Galerkin system matrix Z of the
 * D-VIE and its HOD-BF approximate inverse Zinv to blocks of vectors, and
 * builds both on one GPU (sm_103a).
 *
 *   Problem (Sec. II, Eqs. 1-5): D/eps - j w eta0 L[kappa D] = E_inc in V,
 *   discretized with one SWG function per face of a tetrahedral mesh and
 *   Galerkin testing, Z I = V.  Preconditioned solve (Eq. 6).
 *   HOD-BF (Sec. III-A, Eqs. 7-10): dense leaf blocks D_tau plus butterfly
 *   factorizations of every sibling off-diagonal block B_tau.
 *   Inverse (Sec. III-B, Algorithms 1-2).
 *
 * Units: lambda0 = 1 (k0 = 2 pi for the paper's normalization is passed
 * explicitly), time convention exp(+j w t), so lossy media have Im eps_r < 0.
 * Complex numbers are interleaved (re, im) pairs: c64 = 2 x float,
 * c128 = 2 x double.  Vectors are column-major N x nrhs blocks in the
 * ORIGINAL face order of the mesh (faces numbered as described at
 * vie_mesh_faces).
 *
 * Ownership: the caller owns every array it passes; the library owns the
 * operator (vie_op) and its device memory until vie_destroy.  Device pointers
 * must be on the current CUDA device.  All calls taking a `stream` are
 * stream-ordered (cudaStream_t passed as void*, NULL = legacy default stream)
 * and return without synchronizing unless they write a host out-parameter.
 *
 * Errors: every call returns a vie_status; VIE_OK = 0.  No call aborts the
 * process.  vie_last_error() returns a thread-local message for the last
 * failing call on the calling thread.
 */
#ifndef VIE_H
#define VIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vie_op vie_op; /* opaque */

typedef enum {
  VIE_OK = 0,
  VIE_EINVAL = -1,    /* invalid argument (null pointer, bad size, bad enum)     */
  VIE_ENOMEM = -2,    /* device or host allocation failed                       */
  VIE_ENOTCONV = -3,  /* iterative solve stopped before reaching the tolerance  */
  VIE_ETIMEOUT = -4,  /* a bounded device wait ran out                          */
  VIE_ENAN = -5,      /* NaN or Inf found in an input or a result               */
  VIE_ECUDA = -6,     /* a CUDA runtime call failed                             */
  VIE_ENOTSUP = -7    /* the operator lacks what the call needs (e.g. no Zinv)  */
} vie_status;

typedef enum { VIE_OP_Z = 0, VIE_OP_ZINV = 1, VIE_OP_ZH = 2, VIE_OP_ZINVH = 3 } vie_opkind;
typedef enum { VIE_C64 = 0, VIE_C128 = 1 } vie_dtype;

/* Arithmetic of the stored factors and of the multi-RHS applies:
 *   VIE_P_AUTO       factor_dtype decides; complex FP32 factors apply on the tensor cores from
 *                    16 columns (or the count vie_autotune_rhs chose);
 *   VIE_P_FP64       the plain FP64 method: complex FP64 factors, FP64 applies;
 *   VIE_P_C32        complex FP32 factors and applies, never the tensor cores;
 *   VIE_P_TC_BF16X3  complex FP32 factors, tensor cores (BF16x3 split products, FP32
 *                    accumulation) from 16 columns, crossover fixed;
 *   VIE_P_TC_TF32    complex FP32 factors, tensor cores from 16 columns with one TF32
 *                    product per real product (operands rounded to TF32, 10 mantissa
 *                    bits; FP32 accumulation): about 1.5x less tensor time than BF16x3
 *                    at about 5e-4 relative accuracy per product; crossover fixed.
 *                    The construction of Zinv still runs its products in BF16x3. */
typedef enum { VIE_P_AUTO = 0, VIE_P_FP64 = 1, VIE_P_C32 = 2, VIE_P_TC_BF16X3 = 3, VIE_P_TC_TF32 = 4 } vie_prec;

/* A scatterer on a cubic voxel lattice of pitch h: voxel (i, j, k) is the cube
 * [i h, (i+1) h] x [j h, (j+1) h] x [k h, (k+1) h].  Each voxel is split into
 * the 6 Kuhn tetrahedra (Sec. II mesh, reading of the voxel mesh rule).
 * ijk: host, 3*nvox int32, no duplicates; eps: host, 2*nvox doubles
 * (re, im) relative permittivity per voxel. */
typedef struct {
  int64_t nvox;
  const int32_t* ijk;
  const double* eps;
  double h;
} vie_voxels;

/* A general tetrahedral mesh (Sec. II: the scatterer discretized by tets, one SWG
 * function per face, Eq. 3).  xyz: host, 3*nv vertex coordinates (lambda0 units);
 * tet: host, 4*nt vertex ids per tet in any orientation; eps_r: host, 2*nt
 * (re, im) relative permittivity per tet (finite, nonzero).  Faces are numbered
 * as the unique sorted vertex-id triples in lexicographic order, T+ of a face is
 * the lower tet id holding it.  The quadrature tiers of the entries use cells of
 * pitch h_c = the mean (in tet order) of each tet's shortest edge: a tet's cell
 * is floor(centroid / h_c), the tier of two elements the Chebyshev distance of
 * their tets' cells (on a voxel mesh, the voxel rule).  Meant for quasi-uniform
 * meshes, like those of the paper. */
typedef struct {
  int64_t nv;
  const double* xyz;
  int64_t nt;
  const int32_t* tet;
  const double* eps_r;
} vie_mesh;

typedef struct {
  double tol_con;      /* chi_con: ID truncation |R_kk| <= tol |R_11| (Eq. 7) */
  double tol_fact;     /* chi_fact of the inverse (Sec. III-B); <= 0: no Zinv  */
  int32_t leaf;        /* max unknowns per leaf of the cluster tree (64)        */
  int32_t factor_dtype;/* vie_dtype of the stored factors (VIE_C64 default)     */
  uint64_t seed;       /* seed of the row sampling in the IDs                   */
  int32_t oversample;  /* extra random rows per ID beyond the candidate count   */
  int32_t id_tol_div;  /* each ID truncates at tol / id_tol_div (<= 1: at tol)  */
  int32_t inv_dense_max; /* inverse: largest diagonal block (unknowns) whose E_tau is
                            formed densely; the levels above are built from products
                            only (Algorithms 1-2 with BF_random_matvec).  0: 65,536.
                            Complex FP64 factors keep the dense construction only.  */
  int32_t prec;          /* a vie_prec value; 0 = VIE_P_AUTO                           */
} vie_config;

typedef struct {
  int64_t n;              /* unknowns = faces of the mesh                       */
  int64_t ntets;
  int32_t levels;         /* L_H                                                */
  int32_t max_rank;       /* max butterfly rank over all blocks                 */
  int64_t entries_z;      /* complex entries stored for Z (leaf + butterflies)  */
  int64_t entries_zinv;   /* complex entries stored for Zinv (0 if none)        */
  int64_t bytes_z;        /* bytes of the stored Z factors (incl. padding)      */
  int64_t bytes_zinv;
  int64_t entries_evaluated; /* matrix entries evaluated during the build       */
  double build_seconds;
  double invert_seconds;
  int32_t apply_stages_z; /* kernel stages of one Z apply                       */
  int32_t apply_stages_zinv;
  double build_entries_seconds;  /* of build_seconds: matrix entries on the GPU   */
  double build_id_seconds;       /* of build_seconds: batched IDs on the GPU      */
  double build_host_seconds;     /* of build_seconds: row sampling on the host    */
  int32_t zinv_top_level;        /* Zinv holds Algorithm 1's levels l >= this one (0 = all);
                                    with complex FP64 factors, nodes larger than 65,536
                                    unknowns are not inverted                            */
  int32_t zinv_product_levels;   /* Algorithm 1 levels built from products only          */
  int64_t inverse_products;      /* columns multiplied by an operator or its adjoint there */
  double invert_product_seconds; /* of invert_seconds: the product-built levels           */
} vie_stats_t;

/* Build Z (and Zinv when cfg->tol_fact > 0) for the voxel body at wavenumber
 * k0 (Sec. III-A construction; Sec. III-B inversion).  Mesh, SWG table and
 * cluster tree are made on the host; entries, IDs and factors on the GPU.
 * Returns VIE_EINVAL for nvox <= 0, h <= 0, leaf < 4, tol_con <= 0, a voxel
 * index with |i| >= 2^19, a voxel listed twice, or an eps_r that is zero or not
 * finite. */
vie_status vie_build(const vie_voxels* body, double k0, const vie_config* cfg,
                     void* stream, vie_op** out);

/* vie_build for a general tetrahedral mesh.  The entries are evaluated per element
 * pair on the fly (no lattice tables): closed-form potentials over the source and
 * conical rules over the observer in the near tier, conical rules in the mid tier,
 * 4-point rules in the far tier.  VIE_EINVAL for an empty mesh, a vertex id out of
 * range, a repeated vertex in a tet, a zero-volume tet, a face shared by more than
 * two tets, a non-finite coordinate or eps_r, and the configuration errors of
 * vie_build. */
vie_status vie_build_mesh(const vie_mesh* mesh, double k0, const vie_config* cfg,
                          void* stream, vie_op** out);

/* Y = op(X) for op = Z, Zinv, or their adjoints Z^H, Zinv^H (VIE_OP_ZH,
 * VIE_OP_ZINVH: the conjugate-transposed factors in reverse order, the products
 * the randomized construction of Sec. III-B needs; the adjoint factors are
 * formed on the first such call, about the size of the operator's factors),
 * X and Y device arrays, N x nrhs column-major
 * with leading dimensions ldx, ldy >= N (in elements), dtype VIE_C64 or
 * VIE_C128 for both.  The factors keep their stored type; accumulation runs
 * in the vector type (c128 vectors give the FP64-accumulated apply used for
 * refinement residuals).  X and Y must not overlap.  (Sec. III-A: the
 * apply of the compressed operator costs O(N log N); Algorithm 1 for Zinv.) */
vie_status vie_apply(vie_op* op, int32_t which, const void* X, void* Y, int64_t nrhs,
                     int64_t ldx, int64_t ldy, int32_t dtype, void* stream);

/* Grouped apply: Y[i] = op_i(X[i]) for count operators at once, op_i = Z
 * (which[i] = VIE_OP_Z) or Zinv (VIE_OP_ZINV) of ops[i], each X[i], Y[i] a
 * device array of complex FP32 (VIE_C64), N_i x nrhs[i] column-major with
 * leading dimension N_i.  The independent stage chains of the operators (Sec.
 * III-A; Algorithm 1 for Zinv) run as one launch per stage depth, each a work
 * list over (operator, factor block, row tile) and, for nrhs[i] at or above the
 * operator's tensor-core column count, (operator, tensor-core item, 128-column
 * chunk); the results are bit-identical to count separate vie_apply calls.
 * Operators need c64 factors, and each may appear once per call (its
 * workspaces hold that operator's vectors).  Stream-ordered on `stream`.
 * VIE_EINVAL: null pointers, nrhs < 1, a repeated operator, c128 factors, a
 * kind other than Z / Zinv; VIE_ENOTSUP: Zinv of an operator without one. */
vie_status vie_apply_group(vie_op* const* ops, const int32_t* which, const void* const* X,
                           void* const* Y, const int64_t* nrhs, int32_t count, void* stream);

/* vie_apply that also times each kernel of the apply with CUDA events on
 * `stream` and waits for it: ms (host, cap >= stages + 2) receives the
 * milliseconds of [gather, stage 0 .. stage S-1, scatter]; *launches (may be
 * NULL) the number of kernel launches of one apply.  Metrics/profiling aid;
 * same arguments and errors as vie_apply, plus VIE_EINVAL if cap is short. */
vie_status vie_apply_profile(vie_op* op, int32_t which, const void* X, void* Y, int64_t nrhs,
                             int64_t ldx, int64_t ldy, int32_t dtype, void* stream, double* ms,
                             int64_t* launches, int32_t cap);

/* Per-stage layout of an operator's apply program: *nstages receives the
 * stage count S; entries[i] (complex entries of the factor blocks of stage i,
 * the algorithmic count), bytes[i] (stored bytes incl. row padding) and
 * tiles[i] (warp tiles) are written for i < min(S, cap).  Host arrays; any
 * of them may be NULL. */
vie_status vie_program_info(const vie_op* op, int32_t which, int64_t* entries, int64_t* bytes,
                            int64_t* tiles, int32_t cap, int32_t* nstages);

/* vie_apply without any device allocation (the paper has no counterpart:
 * this serves callers that cannot allocate device memory).  cudaMalloc may
 * synchronize the whole device, which stalls every stream of a latency-bound
 * serving loop, and a process whose device memory is owned by another
 * framework's caching allocator has no headroom for allocations made behind
 * its back.  Same arguments, layout and errors as vie_apply; the work vectors
 * (tree-ordered X and Y and the butterfly coefficients, 2 N nrhs + C nrhs
 * complex elements of `dtype`, C the operator's coefficient count) live in one
 * fixed 64 MiB device array inside the library, held by every GPU that loads
 * the library until the process exits.  Returns VIE_EINVAL, allocating
 * nothing, when they do not fit.  The first call on each device looks the
 * array's device address up (with that device current) and caches it: make
 * that first call before any stream capture.  All calls on a device share the
 * array, so calls that overlap on the GPU race on it; order them.  The array
 * keeps the last call's contents, and no element needs to start at zero. */
vie_status vie_apply_noalloc(vie_op* op, int32_t which, const void* X, void* Y, int64_t nrhs,
                             int64_t ldx, int64_t ldy, int32_t dtype, void* stream);

/* Autotune the single-RHS apply (c64 factors): for every stage, time each
 * candidate with CUDA events on `stream` and keep the fastest.  Candidates
 * 0-8: the streaming kernel (four 16-byte loads in flight per lane) with a
 * maximum tile of 4, 16 or 64 KB of factor data x 2, 4 or 8 16-byte vectors
 * per lane and row (index = tile-size index * 3 + vector index); 9-11: the
 * kernel that stages 32 KB tiles in shared memory by bulk asynchronous
 * copies, with 2, 4 or 8 vectors per lane; 12-20: the streaming kernel with
 * eight loads in flight per lane, tiles as in 0-8.  choice (host, cap >=
 * stages, may be NULL) receives the chosen index per stage.  Results of
 * later applies are unchanged (tiling and staging only move work between
 * warps and memories; each output row keeps one owner). */
vie_status vie_autotune(vie_op* op, int32_t which, int32_t* choice, int32_t cap, void* stream);

/* Set the single-RHS kernel and tiling of every stage to the autotuner
 * candidate choice[i] (host, n = the program's stage count; indices as in
 * vie_autotune), e.g. to restore a saved tuning.  VIE_EINVAL for a wrong
 * count, an index outside 0-20, c128 factors, or a bulk candidate whose tile
 * does not fit its 32 KB slot. */
vie_status vie_set_tiling(vie_op* op, int32_t which, const int32_t* choice, int32_t n, void* stream);

/* Choose where multi-RHS applies (c64 vectors, c64 factors) switch from the
 * SIMT kernel to the tensor cores: the stages of one apply are timed with 2,
 * 4, 8 and 16 columns on both paths (CUDA events on `stream`), and later
 * applies with at least *tc_min_rhs columns (host, may be NULL; the smallest
 * count from which the tensor cores won at every larger candidate, else 32)
 * use the tensor cores; the default before this call is 16.  Packs the
 * tensor-core tiles if that has not happened yet (device memory about the
 * size of the factors).  Results stay within the tensor-core tolerance of the
 * SIMT path (BF16x3 split products, FP32 accumulation). */
vie_status vie_autotune_rhs(vie_op* op, int32_t which, int32_t* tc_min_rhs, void* stream);

/* Switch the multi-RHS arithmetic of a built operator with complex FP32 factors:
 * prec = VIE_P_C32 (SIMT only), VIE_P_TC_BF16X3 or VIE_P_TC_TF32 (tensor cores
 * from 16 columns).  Waits for the device, drops the packed tensor-core tiles and
 * captured graphs of Z and Zinv (repacked on the next multi-RHS apply) and sets
 * vie_config.prec.  Not while a server (vie_server_create) holds the operator:
 * its captured steps keep the old tiles.  VIE_EINVAL: null op, another prec
 * value, complex FP64 factors. */
vie_status vie_set_prec(vie_op* op, int32_t prec);

/* Block shapes of one stage of an apply program (introspection for profiling):
 * *count receives the number of blocks; M[i], K[i] (host, may be NULL) their
 * rows and columns for i < min(count, cap). */
vie_status vie_program_blocks(const vie_op* op, int32_t which, int32_t stage, int32_t* M, int32_t* K,
                              int64_t cap, int64_t* count);

/* out[i] = Z(rows[i], cols[i]) for i < count, evaluated on the GPU in FP64
 * from Eq. (5) (entries of the uncompressed matrix).  rows, cols: device int32
 * face indices in [0, N); out: device c128. */
vie_status vie_entries(vie_op* op, const int32_t* rows, const int32_t* cols, int64_t count,
                       void* out, void* stream);

/* V(:, j) = <f_m, pol_j exp(-j k0 khat_j . r)> (Eq. 5) for j < nrhs.
 * khat, pol: host, 3*nrhs doubles; V: device c128, N x nrhs (ld = N). */
vie_status vie_rhs_planewave(vie_op* op, const double* khat, const double* pol, int64_t nrhs,
                             void* V, void* stream);

/* Solve Z I = V with right-preconditioned restarted GMRES (Zinv as the
 * preconditioner when present, Eq. 6) inside FP64 iterative refinement.
 * V, I: device c128 N x nrhs (ld = N).  iters, relres: host arrays of nrhs
 * (may be NULL).  Returns VIE_ENOTCONV (I holds the best iterate) when a
 * column misses rtol within max_iter inner iterations. */
vie_status vie_solve(vie_op* op, const void* V, void* I, int64_t nrhs, double rtol,
                     int32_t restart, int32_t max_iter, int32_t* iters, double* relres,
                     void* stream);

/* Solve the left-preconditioned system Zinv Z I = Zinv V (Eq. 6; M = I when
 * the operator has no Zinv) with TFQMR (the paper's solver, Sec. II).  A
 * column stops when the quasi-residual bound tau sqrt(m + 1) (m half-steps)
 * falls below rtol ||M V|| and the true preconditioned residual
 * ||M (V - Z I)|| / ||M V|| confirms rtol; otherwise it restarts from its
 * iterate.  V, I: device c128 N x nrhs (ld = N).  iters (host, may be NULL):
 * TFQMR iterations per column (two applications of Zinv Z each).  relres
 * (host, may be NULL): the unpreconditioned ||V - Z I|| / ||V||.  Returns
 * VIE_ENOTCONV (I holds the last iterate) when a column misses rtol within
 * max_iter iterations, VIE_ENAN for a non-finite V. */
vie_status vie_solve_tfqmr(vie_op* op, const void* V, void* I, int64_t nrhs, double rtol,
                           int32_t max_iter, int32_t* iters, double* relres, void* stream);

/* Bistatic RCS sigma(dir_k) for each column of I (device c128 N x nrhs) and
 * each unit direction dirs (host 3*ndir): rcs (host, ndir x nrhs, column
 * major), in lambda0^2, sigma = k0^4/(4 pi) |(I - rr) . F|^2,
 * F = int kappa d exp(j k0 rhat . r) dv. */
vie_status vie_farfield(vie_op* op, const void* I, int64_t nrhs, const double* dirs, int64_t ndir,
                        double* rcs, void* stream);

/* Face table of the mesh: faces (host 3*N int32, sorted vertex ids, faces
 * sorted lexicographically), tp / tm (host N int32: the lower / higher tet
 * id holding the face, tm = -1 on the boundary).  Voxel bodies: vertices are
 * the lattice points sorted lexicographically by (i, j, k); tets are
 * voxel-major, then the 6 axis permutations in lexicographic order.  General
 * meshes: vertices and tets as given.  Any pointer may be NULL. */
vie_status vie_mesh_faces(const vie_op* op, int32_t* faces, int32_t* tp, int32_t* tm);

/* Host only (no GPU needed): the mesh and cluster tree that vie_build would
 * make for `body`.  *n receives N; when non-NULL, faces (3*N), tp, tm (N) are
 * filled as in vie_mesh_faces, perm (N) as in vie_tree_perm and *levels with
 * L_H.  Call once with NULL arrays to size them. */
vie_status vie_mesh_host(const vie_voxels* body, int32_t leaf, int64_t* n, int32_t* faces, int32_t* tp,
                         int32_t* tm, int32_t* perm, int32_t* levels);

/* vie_mesh_host for a general tet mesh (vie_build_mesh's mesh, cells and tree):
 * additionally cells (host 3*nt int32, NULL allowed) receives the tier cell of
 * every tet and *cell_pitch (NULL allowed) the cell pitch h_c.  Faces and tree as
 * in vie_mesh_host (vertex ids as given).  Errors as in vie_build_mesh. */
vie_status vie_mesh_host_tets(const vie_mesh* mesh, int32_t leaf, int64_t* n, int32_t* faces,
                              int32_t* tp, int32_t* tm, int32_t* perm, int32_t* levels,
                              int32_t* cells, double* cell_pitch);

/* perm (host, N int32): original face index at each position of the cluster
 * tree order (Sec. III-A: KD bisection to a complete tree of L_H levels). */
vie_status vie_tree_perm(const vie_op* op, int32_t* perm);

vie_status vie_stats(const vie_op* op, vie_stats_t* out);

/* Sharded apply across GPUs by subtrees (Sec. III-D: processors assigned by the cluster
 * tree).  With nranks GPUs (a power of two, at most 2^L_H) rank r owns the faces at tree
 * positions [lo, hi) of node r at level log2(nranks) (vie_shard_range; vie_tree_perm maps
 * tree positions to faces).  vie_apply_shard writes exactly the rank's rows of Y (original
 * face order; other rows untouched) from the whole of X, which every rank supplies (one
 * all-gather of X across ranks, done by the caller with its own collective library), so
 * that the ranks' rows together equal vie_apply.  The blocks the rank's rows depend on
 * (leaf blocks and butterflies of its subtree, the row sides of the upper butterflies
 * ending in its rows and the column sides feeding them) are selected on the first call
 * per (which, rank, nranks) and kept until vie_destroy (device memory up to the
 * operator's own).  For Zinv the upper levels update rows of several ranks in place, so
 * a rank's closure includes other ranks' leaves (computed redundantly, results
 * discarded).  Arguments, layout and errors as vie_apply, plus VIE_EINVAL for a bad
 * rank or rank count. */
vie_status vie_shard_range(const vie_op* op, int32_t rank, int32_t nranks, int64_t* lo, int64_t* hi);
vie_status vie_apply_shard(vie_op* op, int32_t which, int32_t rank, int32_t nranks, const void* X, void* Y,
                           int64_t nrhs, int64_t ldx, int64_t ldy, int32_t dtype, void* stream);

/* Checkpoint of a built operator (the paper has no file format; a build costs
 * minutes at the workload sizes).  vie_save writes the voxel body, k0, the
 * configuration, the statistics and every stage of the Z and Zinv apply
 * programs (block descriptors, warp tiles and single-RHS kernel choices, packed
 * factor bytes) to `path`; the factors are read back from the device in 256 MiB
 * pieces on `stream`.  vie_load reads such a file, remakes the mesh, tree and
 * interaction tables on the host and the device, and re-uploads the programs
 * into a new operator (*out, owned by the caller until vie_destroy): its
 * applies are bit-identical to the saved operator's.  Both return VIE_EINVAL
 * for an unopenable, foreign, truncated or inconsistent file (nothing is
 * returned in *out then), VIE_ENOMEM when the device or host runs out. */
vie_status vie_save(const vie_op* op, const char* path, void* stream);
vie_status vie_load(const char* path, void* stream, vie_op** out);

/* Waits for `stream` and reports device-side failures of earlier applies:
 * VIE_ETIMEOUT when a bounded wait inside a tensor-core kernel or the
 * bulk-staged single-RHS kernel ran out (the outputs of that apply are
 * invalid; the flag is cleared), else VIE_OK.
 * Applies with nrhs >= 16 (or the count vie_autotune_rhs chose) on c64
 * vectors and c64 factors run on the tensor
 * cores (tcgen05, BF16x3 split products, FP32 accumulation); the first such
 * apply packs the factor tiles (device memory about the size of the factors). */
vie_status vie_check(vie_op* op, void* stream);

/* Failure-path self-test of the bounded device waits used by the tensor-core
 * kernels: a kernel waits `spins` (1 .. 2^20) polls on an mbarrier that nothing
 * arrives on and gives up; returns VIE_ETIMEOUT (the expected outcome), with the
 * context still usable.  VIE_EINVAL for spins out of range. */
vie_status vie_wait_selftest(int32_t spins, void* stream);

/* ---- serving: continuous batching of solves against resident operators ----
 * (the paper has no serving layer; each request is the solve phase of Eq. 6 with Zinv.)
 * A server holds up to `nops` built operators (not owned).  Requests are
 * admitted while the device memory of their Krylov state (about
 * N nrhs (restart + 6) 16 bytes) fits `mem_budget`; each vie_server_step
 * admits what fits, advances every admitted request by one preconditioned
 * GMRES iteration (the columns of each operator packed into one block, the
 * blocks of all operators applied in one grouped launch sequence as in
 * vie_apply_group, tensor cores for a block of 16 columns or the count
 * vie_autotune_rhs chose, replayed from a CUDA graph while the operators and
 * column counts of the step repeat), ends restart cycles with an FP64
 * refinement residual, and retires finished requests.  The operators need c64
 * factors (VIE_EINVAL otherwise).
 * Requests submitted between steps join at the next step.  All work runs on
 * `stream`; every call is synchronous with respect to the host. */
typedef struct vie_server vie_server;

vie_status vie_server_create(vie_op* const* ops, int32_t nops, int32_t restart, int32_t max_iter,
                             int64_t mem_budget, void* stream, vie_server** out);

/* Queue a request: V_host is a host c128 N_op x nrhs column-major block (copied
 * now); *id receives the request id.  VIE_EINVAL for nrhs outside [1, 2^20] or
 * rtol <= 0, VIE_ENAN for NaN/Inf input, VIE_ENOMEM when one request alone
 * exceeds the budget. */
vie_status vie_server_submit(vie_server* srv, int32_t op, const void* V_host, int64_t nrhs, double rtol,
                             int64_t* id);

/* One step; *active / *pending (may be NULL) receive the request counts after it. */
vie_status vie_server_step(vie_server* srv, int32_t* active, int32_t* pending);

/* Result of a finished request: I_host (host c128 N x nrhs, may be NULL), iters
 * and relres per column (may be NULL), latency_s = seconds from submit to done.
 * Returns VIE_ENOTCONV while the request is still queued or running (nothing
 * written), VIE_EINVAL for an unknown id; a fetched result is released. */
vie_status vie_server_result(vie_server* srv, int64_t id, void* I_host, int32_t* iters, double* relres,
                             double* latency_s);

/* Cancel request `id` between steps: a pending request is dropped, an admitted one
 * leaves the batch and its Krylov state is freed (its memory returns to the
 * budget), a finished one discards its result.  The other requests continue
 * unchanged.  VIE_EINVAL: null server or unknown id. */
vie_status vie_server_cancel(vie_server* srv, int64_t id);

/* Device bytes the admitted requests' Krylov state holds against the budget (host
 * out-parameters, either may be NULL). */
vie_status vie_server_memory(const vie_server* srv, int64_t* used, int64_t* budget);

void vie_server_destroy(vie_server* srv);

void vie_destroy(vie_op* op);
const char* vie_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VIE_H */
