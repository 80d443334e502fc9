/*
 * gmg.h -- C ABI of the GB300 local-smoothing geometric multigrid solver.
 *
 * The library solves  -div(a grad u) = f  in a Cartesian brick with u = 0 on
 * the boundary, discretised by continuous Q_k elements (k = 1, 2) on an
 * adaptively refined, 2:1-balanced hexahedral (quadrilateral in 2D) forest,
 * with a conjugate-gradient solver preconditioned by one geometric multigrid
 * V-cycle with local smoothing.  Method: Clevenger, Heister, Kanschat,
 * Kronbichler, "A flexible, parallel, adaptive geometric multigrid method
 * for FEM", ACM TOMS 47(1), 2021 (arXiv 1904.03317):
 *   - weak form a(u,v) = f(v)                                   Sec. 2.1
 *   - mesh hierarchy, level spaces, transfer P and R = P^T       Sec. 2.2
 *   - V-cycle                                                    Algorithm 2
 *   - local smoothing on V_l^S, edge matrices A^SI / A^IS        Sec. 2.3
 *   - Chebyshev-Jacobi smoother, eigenvalue estimate, FP32 cycle Sec. 4.1
 *   - outer CG on the leaf mesh with hanging-node elimination    Sec. 1, 4.1
 *
 * Conventions shared by every entry point:
 *   - Every call returns a gmg_status; nothing throws across the ABI.  On
 *     failure gmg_last_error() returns a message for the calling thread.
 *   - Host arrays passed in are owned by the caller and copied during the
 *     call.  Objects created by gmg_*_create / gmg_hier_build are owned by
 *     the library until the matching destroy call.
 *   - "Device pointer" arguments are CUDA device addresses on the context's
 *     device (for example the data_ptr() of a torch tensor); the caller owns
 *     them.  All device work is enqueued on the context's stream; calls return
 *     without synchronising unless stated otherwise.
 *   - Active vectors (right-hand side, solution, residual) are FP64, one
 *     entry per unknown, in canonical order: unknowns sorted by node key.
 *   - Node key: the node's integer coordinates (x, y, z) on the node lattice
 *     of the finest level Lf of the hierarchy (spacing h_Lf / k), packed as
 *     (z << 42) | (y << 21) | x.  Sorting by key is lexicographic (z, y, x).
 */
#ifndef GMG_H
#define GMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gmg_status {
  GMG_OK = 0,
  GMG_EINVAL = 1,      /* invalid argument (null pointer, size, range, state) */
  GMG_ENOMEM = 2,      /* host or device allocation failed */
  GMG_ECUDA = 3,       /* a CUDA runtime call failed */
  GMG_ENOTCONV = 4,    /* CG hit max_iter; x holds the last iterate, stats filled */
  GMG_EBREAKDOWN = 5,  /* CG breakdown: p.Ap <= 0 (operator not SPD) */
  GMG_ENAN = 6,        /* NaN or Inf in a CG scalar */
  GMG_ETIMEOUT = 7,    /* a bounded device wait gave up */
  GMG_EUNSUPPORTED = 8 /* valid request this build does not implement */
} gmg_status;

typedef struct gmg_ctx gmg_ctx;
typedef struct gmg_mesh gmg_mesh;
typedef struct gmg_hier gmg_hier;

/* Coarse mesh: the brick [lo, hi] split into n0[0] x n0[1] (x n0[2]) equal
 * cells (Sec. 2.2: the coarse mesh T_0).  dim is 2 or 3; for dim 2 the third
 * entries are ignored.  present: NULL, or one byte per coarse cell in
 * lexicographic order (x fastest), nonzero if the cell belongs to the
 * domain; the domain is the union of the present cells (for instance the
 * Fichera corner of Sec. 4.3, a brick with one octant removed), u = 0 on its
 * whole boundary.  The array is copied when the mesh is created; at least one
 * cell must be present. */
typedef struct gmg_coarse_mesh {
  int dim;
  int n0[3];
  double lo[3];
  double hi[3];
  const uint8_t* present;
} gmg_coarse_mesh;

typedef enum gmg_precision { GMG_PREC_FP64 = 0, GMG_PREC_FP32 = 1 } gmg_precision;

/* Solver parameters (defaults from Sec. 4.1 of the paper). */
/* smoothers and coarse solvers (gmg_params.smoother, .coarse_solver) */
#define GMG_SMOOTHER_CHEBYSHEV 0
#define GMG_SMOOTHER_JACOBI 1
#define GMG_COARSE_CHOLESKY 0
#define GMG_COARSE_CHEBYSHEV 1
#define GMG_COARSE_CG 2

typedef struct gmg_params {
  int cheb_degree;            /* m: Chebyshev updates per smoothing (Sec. 4.1 uses 5); >= 1 */
  double eig_lo;              /* damping range [eig_lo, eig_hi] x lambda_max: 0.08 */
  double eig_hi;              /*                                              1.2  */
  int eig_iters;              /* CG steps of the eigenvalue estimate: 10 */
  int vcycle_prec;            /* gmg_precision of the whole V-cycle; CG is always FP64 */
  const double* fixed_lambda; /* optional host array, one value per level (index 0
                                 unused): use these lambda_max instead of estimating.
                                 NULL = estimate. Copied during gmg_hier_build. */
  int smoother;               /* GMG_SMOOTHER_CHEBYSHEV (default; Sec. 4.1) or GMG_SMOOTHER_JACOBI:
                                 cheb_degree undamped Jacobi steps x += D^-1 (g - A x), the
                                 "MF" setting of Sec. 4.3 with cheb_degree = 1 */
  int coarse_solver;          /* GMG_COARSE_CHOLESKY (default; "direct solver", Sec. 2.2),
                                 GMG_COARSE_CHEBYSHEV (Sec. 4.1: Chebyshev-Jacobi over
                                 [lmin, 1.2 lmax] of D^-1 A_0 from a Jacobi-PCG run to the
                                 relative residual coarse_tol, degree from the a-priori bound
                                 2 ((sqrt k - 1)/(sqrt k + 1))^m <= coarse_tol; at most 2048
                                 coarse unknowns) or GMG_COARSE_CG (Sec. 4.3: unpreconditioned
                                 CG from zero to the relative residual coarse_tol, on one
                                 thread block; at most 4096 coarse unknowns) */
  double coarse_tol;          /* default 1e-3 */
  int solve_graph;            /* 1 (default): gmg_solve runs the whole CG loop as one CUDA
                                 graph whose loop is controlled on the device (a conditional
                                 WHILE node): one launch and one synchronisation per solve.
                                 The graph is captured by the first such solve, which also
                                 allocates its iterate (n_unknowns doubles).  0, or profile
                                 timing on (gmg_profile_reset): one stream launch per kernel
                                 and one host check per iteration.  Both modes perform the
                                 same operations in the same order (identical results). */
  int deterministic;          /* 0 (default): the leaf-mesh operator and the restriction add the
                                 contributions of neighbouring elements to shared nodes with
                                 atomics, so two runs agree to rounding.  1: they add them
                                 without atomics, one colour of elements per launch (elements
                                 of one colour share no node) in a fixed colour order, so a
                                 solve gives bitwise the same result every time (and a
                                 problem gives the same bits alone and in a batch).  Costs a
                                 few more launches per operator application. */
  int brick_min_members;      /* tile shape of the 3D smoother: a 2x2x2 position of sibling
                                 groups that is not a full brick becomes a partial brick when
                                 at least this many of its groups can be smoothed together
                                 (2..8; 8 = full bricks only; 0 = the default, 4); the other
                                 groups take the single-group kernel */
} gmg_params;

#define GMG_MAX_LEVELS 24

typedef struct gmg_info {
  int dim, degree, n_levels;  /* levels 0 .. n_levels-1 */
  int vcycle_prec;
  uint64_t n_unknowns;        /* active unknowns (length of active vectors) */
  uint64_t n_leaves;
  uint64_t n_hanging;         /* constrained (hanging) nodes of the leaf mesh */
  uint64_t n_leaf_nodes;      /* all distinct nodes of leaf cells (incl. boundary) */
  uint64_t cells[GMG_MAX_LEVELS];       /* cells of each level, leaves or not */
  uint64_t leaves[GMG_MAX_LEVELS];      /* leaf cells of each level */
  uint64_t groups[GMG_MAX_LEVELS];      /* sibling groups (refined parents) of level l >= 1 */
  uint64_t ghosts[GMG_MAX_LEVELS];      /* storage blocks for refinement-edge nodes */
  uint64_t slots[GMG_MAX_LEVELS];       /* level vector length (entries) */
  uint64_t n_S[GMG_MAX_LEVELS];         /* S nodes of each level (Sec. 2.3) */
  uint64_t n_I[GMG_MAX_LEVELS];         /* I (refinement-edge) nodes of each level */
  uint64_t n_home[GMG_MAX_LEVELS];      /* unknowns whose home level is l */
  uint64_t bricks[GMG_MAX_LEVELS];      /* full 2x2x2 bricks of uniform groups (3D tiles) */
  uint64_t groups_jump[GMG_MAX_LEVELS]; /* groups next to a coefficient jump (general kernel) */
  double lambda_max[GMG_MAX_LEVELS];    /* estimated (or fixed) lambda_max of D^-1 A_l^S */
  uint64_t device_bytes;                /* device memory held by the hierarchy */
  double setup_host_s, setup_device_s;  /* wall time of the two setup phases */
  /* how the leaf-mesh operator covers the leaf cells: patches of 4^d cells
   * (the grandchildren of one cell, all leaves), full sibling groups of 2^d
   * leaf cells, and single cells */
  uint64_t leaf_patches, leaf_groups, leaf_single_cells;
  /* Chebyshev coarse solver: degree and eigenvalue range [lmin, 1.2 lmax] */
  int coarse_degree;
  double coarse_range[2];
  /* host setup phases (s): level blocks and classes, leaf nodes, node classes
   * and numbering, hanging constraints, leaf cell tables, leaf patches and
   * groups, home slots, coarse matrix */
  double setup_phase_s[8];
  /* partial bricks of each level (3D smoother tiles with 4 to 7 member
   * groups; the other positions are read as halo only) */
  uint64_t bricks_partial[GMG_MAX_LEVELS];
} gmg_info;

typedef struct gmg_stats {
  int iterations;         /* completed CG updates of x */
  int converged;          /* 1 if ||r|| <= tol ||b|| was reached */
  double rel_residual;    /* ||r_final|| / ||b|| (recursively updated residual) */
  double norm_b;          /* ||b||_2 */
} gmg_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, enqueueing all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * device = -1 creates a host-only context: meshes and hierarchies can be
 * built and exported (for testing the host logic), but every call that
 * needs the GPU returns GMG_EINVAL. */
gmg_status gmg_create(int device, void* cuda_stream, gmg_ctx** out);
void gmg_destroy(gmg_ctx* ctx);
/* Message of the last failing call on this thread ("" if none). */
const char* gmg_last_error(void);
/* *has_sm103a = 1 if the library was compiled with device code for sm_103a;
 * *version = ABI version (2: gmg_coarse_mesh.present, the seed of gmg_assemble_rhs). */
gmg_status gmg_build_info(int* has_sm103a, int* version);

/* ------------------------------------------------------------------- mesh */

/* Forest of the coarse brick (Sec. 2.3: one tree per coarse cell). */
gmg_status gmg_mesh_create(const gmg_coarse_mesh* cm, gmg_mesh** out);
void gmg_mesh_destroy(gmg_mesh* mesh);
/* Number of leaf cells (the leaf mesh T_L, Sec. 2.3). */
gmg_status gmg_mesh_num_leaves(const gmg_mesh* mesh, uint64_t* n);
/* Number of levels 0 .. L that hold cells. */
gmg_status gmg_mesh_num_levels(const gmg_mesh* mesh, int* n);
/* Leaf cells in canonical order: coarse cells lexicographically (x fastest),
 * and within each coarse cell in Morton (z-curve) order.  level[i] is the
 * cell's level l, coords[3i..3i+2] its lattice coordinates on the level-l
 * lattice of n0[d] * 2^l cells per direction (unused dimension: 0).  Both
 * arrays are caller-allocated with room for num_leaves entries (x3). */
gmg_status gmg_mesh_leaves(const gmg_mesh* mesh, int32_t* level, int32_t* coords);
/* Refine every leaf i with flags[i] != 0 into 2^dim children (isotropic
 * refinement, Sec. 2.2), then restore the 2:1 closure: leaves whose closures
 * touch differ by at most one level (Sec. 3.5; for continuous elements the
 * one-irregularity of Sec. 1).  The closure adds the minimal set of further
 * refinements.  flags follows gmg_mesh_leaves order; n_flags must equal the
 * current number of leaves. */
gmg_status gmg_mesh_refine(gmg_mesh* mesh, const uint8_t* flags, uint64_t n_flags);

/* Partitioning efficiency model of Sec. 3.4 (Eq. for W and E): every cell of
 * every level of the hierarchy is one unit of work.  The leaves, in
 * gmg_mesh_leaves order (the space-filling curve), are split into n_parts
 * contiguous pieces, part p taking leaves [p N / n_parts, (p+1) N / n_parts)
 * in integer division; a refined cell belongs to the part that owns its
 * first child, recursively (the first-child rule, Sec. 3.3).  With N_l the
 * cells of level l and N_{l,p} those of part p:
 *   w_opt = sum_l N_l / n_parts,  w_sync = sum_l ceil(N_l / n_parts),
 *   w = sum_l max_p N_{l,p},      efficiency = w_opt / w.
 * Level 0 stands for the coarse solve at one unit per coarse cell, as in the
 * paper's worked example.  On one GPU, n_parts read as the number of
 * resident cell batches makes w_sync / w_opt the predicted occupancy of a
 * level-synchronous V-cycle.  Host only; n_parts in [1, 2^31).  Errors:
 * GMG_EINVAL on a null argument or n_parts out of range. */
typedef struct gmg_partition_model {
  int n_levels;
  double n_cells[GMG_MAX_LEVELS];  /* N_l */
  double w_level[GMG_MAX_LEVELS];  /* max_p N_{l,p} */
  double w_opt, w_sync, w, efficiency;
} gmg_partition_model;
gmg_status gmg_mesh_partition_model(const gmg_mesh* mesh, int64_t n_parts, gmg_partition_model* out);

/* -------------------------------------------------------------- hierarchy */

void gmg_params_default(gmg_params* p);

/* Build the multigrid hierarchy of `mesh` for degree k (1 or 2): level
 * meshes (all cells of level l, Sec. 2.3), their S/I node splitting, the
 * leaf-mesh unknowns with hanging-node constraints, the active<->level copy
 * maps, and, for a device context, all device data: inverse diagonals, the
 * eigenvalue estimates of Sec. 4.1 and the factorised coarse matrix A_0.
 * coarse_coeff: the coefficient a (> 0) of each coarse cell, x fastest, or
 * NULL for a = 1; descendants inherit it.  p may be NULL for the defaults.
 * Synchronises the context stream before returning. */
gmg_status gmg_hier_build(gmg_ctx* ctx, const gmg_mesh* mesh, int degree,
                          const double* coarse_coeff, const gmg_params* p, gmg_hier** out);
void gmg_hier_destroy(gmg_hier* h);
gmg_status gmg_hier_info(const gmg_hier* h, gmg_info* info);

/* Flags of one refinement round (Sec. 3.5: a round refines the flagged
 * leaves, then the closure restores 2:1 balance).  Called with the current
 * leaves in gmg_mesh_leaves order (level[i], coords[3i..3i+2], n_leaves
 * entries, valid for the call only); writes flags[i] != 0 for each leaf to
 * refine (the library zero-fills flags first).  Returns 0 to go on; any
 * other value stops the build, which then fails with GMG_EINVAL. */
typedef int (*gmg_refine_fn)(void* user, int round, uint64_t n_leaves, const int32_t* level,
                             const int32_t* coords, uint8_t* flags);

/* The hierarchy in one call, as the paper states the problem (Sec. 2.3 and
 * Sec. 3.5): the forest of the coarse brick `cm`, n_rounds >= 0 refinement
 * rounds whose flags `refine` computes on the leaves of the mesh as it
 * stands (closure after each), then gmg_hier_build with degree,
 * coarse_coeff and p as there.  The mesh is internal and released before
 * returning (use the gmg_mesh_* calls to keep it).  Errors: those of
 * gmg_mesh_create, gmg_mesh_refine and gmg_hier_build; GMG_EINVAL for a null
 * argument, n_rounds < 0, refine NULL with n_rounds > 0, or a callback that
 * stops the build.  *out is NULL on failure. */
gmg_status gmg_build_hierarchy(gmg_ctx* ctx, const gmg_coarse_mesh* cm, int n_rounds, gmg_refine_fn refine,
                               void* user, int degree, const double* coarse_coeff, const gmg_params* p,
                               gmg_hier** out);

/* What gmg_hier_export writes (host buffers; *count in/out = entries). */
typedef enum gmg_export_what {
  GMG_EXPORT_UNKNOWN_KEYS = 0,  /* int64 node key per unknown (canonical order) */
  GMG_EXPORT_HOME_LEVEL = 1,    /* int32 home level per unknown: the coarsest level of
                                   the leaves containing it, where it is an S node */
  GMG_EXPORT_HANGING = 2,       /* records {int64 hanging key, int64 master key,
                                   double weight}; Dirichlet masters omitted */
  GMG_EXPORT_LEVEL_KEYS = 3,    /* int64 node key per slot of level `level`, -1 unused */
  GMG_EXPORT_LEVEL_CLASS = 4,   /* int8 per slot: 0 unused, 1 S, 2 I, 3 Dirichlet */
  GMG_EXPORT_HOME_SLOT = 5      /* int64 slot of each unknown in its home level */
} gmg_export_what;

/* Copy a table out of the hierarchy.  If buf is NULL only *count is set to
 * the number of entries (records for GMG_EXPORT_HANGING).  Otherwise *count
 * holds the capacity of buf in entries on entry and the number written on
 * return (GMG_EINVAL if too small).  `level` is used by the LEVEL_* items. */
gmg_status gmg_hier_export(const gmg_hier* h, int what, int level, void* buf, uint64_t* count);

/* ------------------------------------------------------------ solve path */

/* Right-hand sides (gmg_assemble_rhs kind). */
#define GMG_RHS_SINE 0   /* b = C^T (int f phi_i) over the leaf cells with the (k+1)^d-point
                            Gauss-Legendre rule, f = d pi^2 prod sin(pi x_i): the manufactured
                            solution u = prod sin(pi x_i) on [0,1]^d (seed unused) */
#define GMG_RHS_ONE 2    /* b = C^T (int f phi_i) with f = 1, the same quadrature as
                            GMG_RHS_SINE (the Laplace example of Sec. 4.3; seed unused) */
#define GMG_RHS_RANDOM 1 /* b_i uniform in [-1, 1) per unknown i in canonical order: with the
                            SplitMix64 output function s (Steele, Lea, Flood, OOPSLA 2014),
                            b_i = 2 (s(seed xor (i * 0xD1B54A32D192ED03)) >> 11) 2^-53 - 1
                            (64-bit wrapping arithmetic); the random right-hand sides of the
                            variable-coefficient, batched and served workloads */

/* Right-hand side of kind GMG_RHS_SINE, GMG_RHS_ONE or GMG_RHS_RANDOM (with `seed`).
 * d_b: device pointer, n_unknowns FP64, overwritten.  GMG_EINVAL for another
 * kind. */
gmg_status gmg_assemble_rhs(gmg_hier* h, int kind, uint64_t seed, double* d_b);

/* y = A x with the leaf-mesh operator A = C^T A_leaf C (hanging nodes
 * eliminated, Dirichlet rows removed).  d_x, d_y: device, n_unknowns FP64;
 * they must not overlap. */
gmg_status gmg_apply(gmg_hier* h, const double* d_x, double* d_y);

/* z = B r: one local-smoothing V-cycle (Algorithm 2 in the form of Sec. 2.3)
 * in the hierarchy's V-cycle precision; r and z are FP64 active vectors
 * (device pointers, must not overlap). */
gmg_status gmg_vcycle(gmg_hier* h, const double* d_r, double* d_z);

/* Preconditioned CG from x = 0 (Sec. 4.1): stop when ||r||_2 <= tol ||b||_2
 * or after max_iter updates; if fixed_iterations > 0, run exactly that many
 * updates and ignore tol.  d_b, d_x: device FP64 active vectors.  The
 * stopping test runs on the device in graph mode (gmg_params.solve_graph) and
 * on the host in stream mode; either way the call returns after the stream
 * has been synchronised.  The first graph-mode solve captures the graph on a
 * private stream: it must not itself be called while a stream capture of
 * the calling thread is in progress.
 * Returns GMG_ENOTCONV when max_iter is hit without convergence (x holds the
 * last iterate), GMG_EBREAKDOWN / GMG_ENAN on a bad CG scalar. */
gmg_status gmg_solve(gmg_hier* h, const double* d_b, double* d_x, double tol, int max_iter,
                     int fixed_iterations, gmg_stats* stats);

/* Asynchronous solve for request loops: enqueue the graph-mode solve of
 * gmg_solve (x0 = 0, tol, max_iter) on the context stream and return at
 * once; d_b must stay valid and d_x untouched until gmg_solve_poll reports
 * the solve ready.  One pending solve per hierarchy.  Needs solve_graph = 1
 * and per-launch timing off.  Hierarchies on different contexts (streams)
 * overlap on the device.  No counterpart in the paper. */
gmg_status gmg_solve_async(gmg_hier* h, const double* d_b, double* d_x, double tol, int max_iter);
/* Completion of the pending asynchronous solve: *ready = 0 while it runs
 * (wait = 0 never blocks; wait = 1 blocks until it ends); once ready,
 * stats (optional) and *status are those gmg_solve would have returned.
 * GMG_EINVAL if no solve is pending. */
gmg_status gmg_solve_poll(gmg_hier* h, int wait, int* ready, gmg_stats* stats, gmg_status* status);

/* Independent solves at once (batched): problem i solves hs[i] x = b with
 * d_b[i], d_x[i] as in gmg_solve (graph mode, x0 = 0, tol, max_iter).  The
 * problems' solve graphs are launched round-robin on n_streams streams of a
 * pool owned by the library, so small problems fill the GPU together; the
 * call returns after all have finished.  Each problem first waits for the
 * work already queued on its hierarchy's context stream.  stats (optional)
 * and status receive one entry per problem (status as gmg_solve's return);
 * the return value is GMG_OK, or the first error met while launching.  All
 * hierarchies must live on one device, be built with solve_graph = 1, appear
 * once, and have per-launch timing off.  Serialised against other batched
 * calls (the stream pool is shared).  The paper solves one problem at a time;
 * this is the GPU's way to batch many small ones. */
gmg_status gmg_solve_batch(gmg_hier* const* hs, const double* const* d_b, double* const* d_x, int n, double tol,
                           int max_iter, int n_streams, gmg_stats* stats, gmg_status* status);

/* ----------------------------------------------- level operations (tests)
 * These expose the individual V-cycle steps on device level vectors in the
 * hierarchy's V-cycle precision (float for FP32, double for FP64), laid out
 * by slot (see GMG_EXPORT_LEVEL_KEYS / _CLASS; level 0 slots are the coarse
 * node lattice).  Level l is in 1 .. n_levels-1 unless stated otherwise. */

/* y = A_l x on the S slots of level l, where A_l is the operator of the
 * level-l cells (Sec. 2.3) and x is read on S and I slots (so y^S =
 * A^S x^S + A^SI x^I).  Slots that are not S are left untouched. */
gmg_status gmg_level_apply(gmg_hier* h, int level, const void* d_x, void* d_y);
/* d_gc += R_{l-1} t on level l-1 with t = g - A_l u on the S and I slots of
 * level l, evaluated as sum over sibling groups of the group's cells
 * (t^I = g^I - A^IS u^S when u^I = 0; Sec. 2.3, restriction R = P^T). */
gmg_status gmg_level_residual_restrict(gmg_hier* h, int level, const void* d_u, const void* d_g,
                                       void* d_gc);
/* d_u += P_{l-1} d_uc on the S slots, and the I slots of both d_u and d_u2
 * are set to P_{l-1} d_uc (the interface values the smoother keeps fixed).
 * d_u2 may equal d_u. */
gmg_status gmg_level_prolongate(gmg_hier* h, int level, const void* d_uc, void* d_u, void* d_u2);
/* One Chebyshev-Jacobi smoothing of `cheb_degree` updates (Sec. 4.1) on the
 * S slots of level l, right-hand side d_g, starting from d_u (from_zero=0)
 * or from 0 (from_zero=1, d_u is then overwritten); I slots of d_u are kept.
 * d_tmp: second level vector used by the recurrence (contents destroyed).
 * The result ends in d_u.  d_g, d_u and d_tmp must be three distinct
 * buffers (GMG_EINVAL otherwise: the updates write d_u and d_tmp while later
 * updates still read d_g). */
gmg_status gmg_level_smooth(gmg_hier* h, int level, const void* d_g, void* d_u, void* d_tmp,
                            int from_zero);
/* Same smoothing as gmg_level_smooth, but the recurrence's second level
 * vector is kept in a static device array inside the library, so this call
 * allocates no memory and needs no d_tmp.  For callers that cannot call
 * cudaMalloc while they run: processes whose device memory belongs to another
 * allocator (a framework's caching allocator or a fixed memory budget), and
 * latency-critical loops that cannot pay the device-wide synchronisation of
 * cudaMalloc/cudaFree.  The paper has no counterpart to this entry point.
 * Limit: the level vector (its slot count times 4 bytes for an FP32 V-cycle,
 * 8 for FP64) must fit in the 8 MiB array, else GMG_EINVAL; d_g and d_u must
 * not alias (GMG_EINVAL).  The array is held by every GPU that loads the
 * library until the process exits, and is shared by all calls: calls whose
 * work overlaps on the GPU (other streams, other hierarchies on the same
 * device) race on it.  gmg_hier_build on a device context looks up the
 * array's device address (cudaGetSymbolAddress, with the device current),
 * which loads the part of the library that holds it, so the array's 8 MiB are
 * allocated during that build (once per device and process) and never during
 * this call; the address is kept with the hierarchy and is valid as long as
 * the hierarchy's own device memory is.  The contents of d_u are as after
 * gmg_level_smooth; the array's contents afterwards are unspecified. */
gmg_status gmg_level_smooth_noalloc(gmg_hier* h, int level, const void* d_g, void* d_u, int from_zero);
/* Inverse diagonal of A_l^S on S slots, 0 elsewhere (level >= 1). */
gmg_status gmg_level_inv_diag(gmg_hier* h, int level, void* d_out);
/* u_0 = A_0^{-1} g_0 on the coarse lattice (interior slots; boundary slots 0). */
gmg_status gmg_coarse_solve(gmg_hier* h, const void* d_g0, void* d_u0);

/* ------------------------------------------------------ launch accounting
 * The library counts every kernel it launches, by kind, together with the
 * algorithmic bytes (vectors read and written, plus per-cell index data for
 * the leaf-mesh operator) and floating-point operations of each launch.
 * With timing enabled it also brackets each launch with CUDA events on the
 * context stream and accumulates the durations. */
enum gmg_kernel_kind {
  GMG_K_CHEB = 0,          /* level operator + Chebyshev update (or apply) */
  GMG_K_SMOOTH_FIRST = 1,  /* first smoothing update from zero (x = D^-1 g / theta) */
  GMG_K_RESTRICT = 2,      /* residual on S u I + restriction R = P^T */
  GMG_K_PROLONG = 3,       /* prolongation P */
  GMG_K_COARSE = 4,        /* coarse solve */
  GMG_K_COPY_TO = 5,       /* active residual -> level right-hand sides (gmg_vcycle); in
                              gmg_solve: r = b with b.b and the first level right-hand sides */
  GMG_K_COPY_FROM = 6,     /* level solutions -> active z with r.z (gmg_vcycle); in gmg_solve:
                              r.z with z read from the level solutions (z is not stored) */
  GMG_K_ACTIVE = 7,        /* leaf-mesh operator with hanging nodes, fused p.Ap */
  GMG_K_CG_XR = 8,         /* x += alpha p, r -= alpha Ap, fused r.r and the next V-cycle's
                              level right-hand sides */
  GMG_K_CG_P = 9,          /* p = z + beta p with z read from the level solutions, Ap = 0 */
  GMG_K_OTHER = 10,        /* dot products, setup kernels */
  GMG_NUM_KERNEL_KINDS = 11
};

typedef struct gmg_kernel_stats {
  uint64_t launches[GMG_NUM_KERNEL_KINDS];
  double ms[GMG_NUM_KERNEL_KINDS];     /* summed event time (0 unless timing enabled) */
  double bytes[GMG_NUM_KERNEL_KINDS];  /* summed algorithmic bytes */
  double flops[GMG_NUM_KERNEL_KINDS];  /* summed floating-point operations */
} gmg_kernel_stats;

/* Reset the counters of h; enable_timing != 0 also records CUDA events
 * around each launch from now on (adds a small host cost per launch). */
gmg_status gmg_profile_reset(gmg_hier* h, int enable_timing);
/* Synchronise the context stream and return the counters since the reset. */
gmg_status gmg_profile_read(gmg_hier* h, gmg_kernel_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* GMG_H */
