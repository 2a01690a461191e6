/*
 * hb.h - C ABI of the GB300 Hadamard-Babich (HB) volume integrator.
 *
 * The library applies the discretised HB integrator of arXiv 2210.02698,
 *     U = K^{v2v} I,   I_j = s(r_j) h^2            (Sec. 3.1, Eq. m_v2v)
 * over the N_v = nx*ny cell centres of a regular 2D grid, with
 *     K_ij = g(r_i, r_j) = v0 f0(w, tau) + v1 f1(w, tau)   (i != j, Eq. babich, N = 1)
 *     f0 = i sqrt(pi)/2 H0(w tau),  f1 = -i sqrt(pi)/2 (2 tau / w) H1(w tau)   (Eq. termf)
 * where tau^2, v0, v1 are Chebyshev-interpolated from tables at node pairs
 * (Sec. 4.1, Eq. chebinterp) and K_ii is the cell-integrated self term of
 * Appendix A (Eq. HankelIntegral2dlemma) divided by h^2.  The operator is
 * applied densely (matrix free, FP64) or in HODBF / butterfly-compressed form
 * (Sec. 4.2, Eq. butterfly_mat), in FP64 or with factors and vectors stored as
 * split-BF16 pairs (hi + lo) and three BF16 tensor-core products per complex
 * multiply-add, accumulated in FP32.
 *
 * Conventions shared by every entry point:
 *  - Cells are in natural order: index = b*nx + a, a the x index (fastest),
 *    centroid (x0 + (a+1/2) h, y0 + (b+1/2) h).
 *  - Vectors s and u are caller-owned DEVICE buffers of complex128 values
 *    (interleaved re, im), N_v x nrhs, column-major (one right-hand side
 *    contiguous), natural order, unless a function says otherwise.
 *  - hb_apply*(s -> u) computes u = K (h^2 s); hb_apply*_adjoint(u -> s)
 *    computes its exact adjoint s = h^2 K^H u (conjugate transpose).
 *  - Work is enqueued on the given cudaStream_t (passed as void*, NULL = the
 *    legacy default stream) and is asynchronous unless stated.
 *  - No exception crosses the ABI.  Every call returns an hb_status; the
 *    message of the last failure is kept per handle (hb_last_error) or, for
 *    calls without a handle, per thread (hb_last_error(NULL)).
 *  - A handle is not thread-safe: use it from one host thread and one stream
 *    at a time.  Calls on a handle serialise through its internal buffers.
 *  - There is no CPU fallback: without a CUDA device every compute call
 *    returns HB_ERR_CUDA.
 */
#ifndef HB_H_
#define HB_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hb_ctx* hb_handle;

typedef enum {
  HB_OK = 0,
  HB_ERR_ARG = 1,          /* invalid argument (null pointer, size, option)   */
  HB_ERR_CUDA = 2,         /* a CUDA runtime call or kernel failed            */
  HB_ERR_OOM = 3,          /* device or host allocation failed                */
  HB_ERR_TIMEOUT = 4,      /* a bounded device wait gave up                   */
  HB_ERR_STATE = 5,        /* call not valid in the handle's state            */
  HB_ERR_UNSUPPORTED = 6   /* valid request the library does not implement    */
} hb_status;

enum { HB_FP64 = 0, HB_MIXED_BF16X3 = 1 };

/* Regular cell-centred 2D grid (Sec. 3.1): nx*ny cells of size h. */
typedef struct {
  int nx, ny;
  double x0, y0, h;
} hb_grid;

/* Tabulated HB ingredients (Sec. 4.1).  All HOST pointers, copied by
 * hb_create.  nodes_x / nodes_y: the n_I Chebyshev nodes per dimension in
 * domain coordinates.  tau2, v0, v1: N_I x N_I row-major (N_I = n_I^2),
 * row = observation node i, column = source node j, node index
 * i = i2*n_I + i1 (x index fastest), i.e. F^c_ij = f(r^c_i, r^c_j) of
 * Eq. chebinterp.  n_cells: n(r) at the N_v centroids, natural order
 * (used by the self term, Appendix A). */
typedef struct {
  int n_I;
  const double* nodes_x;
  const double* nodes_y;
  const double* tau2;
  const double* v0;
  const double* v1;
  const double* n_cells;
} hb_tables;

/* Construction options (Sec. 4.2).  eps: relative tolerance of the ID
 * (Eq. ID); leaf: maximum cluster-tree leaf size; chi: oversampling of the
 * uniform proxy rows and nbr_radius_h: neighbour radius in units of h
 * (Eq. proxyv2v); precision: HB_FP64 or HB_MIXED_BF16X3 for hb_apply /
 * hb_apply_adjoint; workspace_mb: device workspace bound for the build
 * (0 = default); barrier_cycles: spin budget (SM clock cycles, counted from
 * the start of each kernel) of the bounded device waits of the mixed apply
 * (0 = default, 2^31).  A wait that runs out sets a mapped error word; the
 * kernel then lets its copies in flight land (waiting at least 2^31 cycles
 * for them) and stops; a later hb_apply / hb_apply_adjoint on the handle,
 * called once the device has run the apply that ran out, returns
 * HB_ERR_TIMEOUT (the outputs of the apply that ran out are undefined).
 * autotune: 0 = the default launch shape of the mixed apply (a gather and
 * one launch per dependency depth, 16 KB items); 1 = the first
 * mixed apply of each direction and m-tile count (16 right-hand sides per
 * m-tile) times every candidate shape on the caller's stream (one launch per
 * dependency depth at 16 KB or 8 KB items, with or without the cone launch
 * of the first butterfly levels, fused level pairs and the tcgen05 leaf
 * kernel; every depth in one launch with grid barriers; one persistent
 * dataflow launch at 16 KB or
 * 8 KB items, placement slack 16, 48 or 128 cost units, 1 or 4 chains per
 * flag publication; each a full apply, best of three) and keeps the fastest
 * (hb_launch_shape reports it).  That first apply then blocks the host for
 * the tuning (milliseconds to seconds, growing with N_v); under stream
 * capture no tuning happens and the default shape is used.  2 = always the
 * persistent dataflow launch (16 KB items, slack 48, one chain per
 * publication).  3 = one launch per dependency depth with the leaf outputs
 * on the 5th-generation tensor cores (tcgen05.mma, accumulators in tensor
 * memory; the autotuner's candidates include this shape too).  4 = the
 * first four butterfly levels of every butterfly as "cones" in one launch
 * (a CTA takes whole cones - forward: one column group, adjoint: one row
 * group, closed under the dependencies of those levels - and separates their
 * levels with bounded CTA barriers), then one launch per remaining depth.
 * 5 = the transfer depths fused in pairs (2P, 2P + 1), one launch per pair:
 * each producer / consumer component of a pair runs on one CTA, its chains
 * spread over the CTA's warps; a consumer waits (bounded) on a shared-memory
 * count of its component's unfinished producer chains and copies its
 * inputs (other warps' outputs, still in L2) with cp.async.  6 = every
 * dependency depth in one cooperative launch (after the gather), the
 * depths separated by bounded grid barriers: the warps of a CTA meet on a
 * shared-memory barrier, one thread publishes the CTA's stores at gpu scope
 * and counts the CTA in, and the next depth's input runs go out once every
 * CTA has arrived (its factor runs are fetched before). */
typedef struct {
  double eps;
  int leaf;
  double chi;
  double nbr_radius_h;
  int precision;
  int workspace_mb;
  long long barrier_cycles;
  int autotune;
} hb_options;

/* Statistics filled by hb_info. */
typedef struct {
  long long n_v;
  int levels;                 /* L_v of the cluster tree                    */
  int max_rank;               /* largest butterfly rank r_{tau,nu}          */
  long long factor_entries;   /* complex entries of all factors + leaves    */
  long long factor_bytes_fp64;
  long long factor_bytes_mixed; /* one direction's split-BF16 arena (8-row
                                   tiles, rows padded to multiples of 8)   */
  long long id_blocks;        /* interpolative decompositions computed      */
  long long sampled_entries;  /* matrix entries evaluated by the build      */
  double build_ms;
  int built;
  int apply_launches;         /* kernels launched by one mixed-precision
                                 hb_apply of up to 32 right-hand sides in
                                 the default launch shape (the gather and
                                 one launch per dependency depth;
                                 hb_launch_shape says which shape an apply
                                 actually used)                            */
  long long skeleton_rows;    /* sum of all ranks: rows of skeleton vectors */
} hb_stats;

/* hb_create: validate and copy the grid, tables and options; upload the
 * tables; precompute the Lagrange interpolants at the cell coordinates and
 * the self terms K_ii (Appendix A).  Synchronous.  On success *out owns
 * device memory until hb_destroy.  Errors: HB_ERR_ARG for invalid input
 * (non-positive sizes, n_I < 2, omega <= 0, eps <= 0, leaf < 1),
 * HB_ERR_UNSUPPORTED for n_I > 16, HB_ERR_OOM, HB_ERR_CUDA. */
hb_status hb_create(const hb_grid* grid, const hb_tables* tables, double omega,
                    const hb_options* opts, hb_handle* out);

/* hb_build: construct the HODBF representation (Sec. 4.2): K-D cluster tree,
 * per butterfly level proxy rows (Eq. proxyv2v, host), sampled blocks
 * (device, Eq. chebinterpblock + Eq. babich), batched CPQR interpolative
 * decompositions (device, Eq. ID / Eq. proxy), skeleton factors K^L and
 * dense leaf blocks; packs the factors for the FP64 and mixed applies.
 * Synchronous.  Errors: HB_ERR_OOM, HB_ERR_CUDA, HB_ERR_STATE if built. */
hb_status hb_build(hb_handle h);

/* hb_set_omega: move the handle to another angular frequency omega > 0
 * (Sec. 4.1: tau^2, v0 and v1 - the tables - do not depend on omega, so one
 * table set serves every frequency).  Keeps the uploaded tables, their
 * interpolation data, the cluster tree and the options; recomputes the
 * omega-dependent self terms; frees the factors, plans and apply scratch of
 * a previous hb_build (the handle is then unbuilt: call hb_build again
 * before hb_apply) and assembles a curve set with hb_curve_set again at the
 * new frequency (its compressed operators of hb_curve_compress are dropped).  The result equals a handle created at omega with the same
 * tables.  Synchronous.  Errors: HB_ERR_ARG (null handle, omega <= 0 or not
 * finite), HB_ERR_OOM, HB_ERR_CUDA. */
hb_status hb_set_omega(hb_handle h, double omega);

/* hb_apply: u = K (h^2 s) with the compressed operator (Eq. butterfly_mat
 * summed over the HODBF, plus the dense leaf blocks), in the precision of
 * opts.precision (see hb_set_precision).  s, u: device, complex128,
 * N_v x nrhs column-major, must not overlap.  1 <= nrhs <= 1024.
 * Errors: HB_ERR_STATE before hb_build, HB_ERR_ARG, HB_ERR_CUDA. */
hb_status hb_apply(hb_handle h, const void* s, void* u, int nrhs, void* stream);

/* hb_apply_adjoint: s = h^2 K~^H u, the exact adjoint of hb_apply's
 * compressed operator K~ (reversed factor order, conjugate-transposed
 * blocks).  Same layout, limits and errors as hb_apply. */
hb_status hb_apply_adjoint(hb_handle h, const void* u, void* s, int nrhs, void* stream);

/* hb_save: write the built operator to a file: the creation inputs (grid,
 * omega, options, tables, n_cells), the cluster tree, the FP64 factor arena
 * and the factor index; hb_load reads it back into a new, built handle (the
 * tree is rebuilt from the grid and must agree with the file).  The file is
 * little-endian with every integer int64 and every real double:
 *   "HBFACT01" | nx ny | x0 y0 h omega | eps chi nbr_radius_h |
 *   leaf precision workspace_mb barrier_cycles | n_I | nodes_x[n_I]
 *   nodes_y[n_I] | tau2, v0, v1 [N_I^2 each] | n_cells[N_v] | L_v |
 *   perm[N_v] (tree position -> natural index) | bounds of tree levels
 *   l = 0..L_v (2^l + 1 tree positions each) | n_factor |
 *   arena[n_factor] (complex128, re then im) | leaf_off[2^L_v] |
 *   n_butterfly | per butterfly (levels l = 1..L_v, sibling pairs p,
 *   (oi, si) = (2p, 2p + 1) then (2p + 1, 2p)): l oi si L, then (rank,
 *   f_off) of every block (i, j) of every level k = 0..L in the order
 *   k, i 2^(L-k) + j, then kl_off[2^L].
 * Blocks are column-major at their arena offset: dense leaf t |t| x |t|;
 * V^0 block j rank x |leaf si 2^L + j|; W^k block (i, j) rank x (r1 + r2)
 * with r1, r2 the ranks of level k-1 blocks (i/2) 2^(L-k+1) + 2j and + 1;
 * K^L block i |leaf oi 2^L + i| x rank of level-L block i (Sec. 4.2.1,
 * Eq. butterfly_mat; Sec. 4.2 HODBF; the paper has no file format).
 * Synchronous.  Errors: HB_ERR_STATE (hb_save before hb_build), HB_ERR_ARG
 * (unwritable path, unreadable, truncated or inconsistent file), HB_ERR_OOM,
 * HB_ERR_CUDA. */
hb_status hb_save(hb_handle h, const char* path);
hb_status hb_load(const char* path, hb_handle* out);

/* Shards of the apply for several devices (Sec. 4.2: each off-diagonal
 * butterfly K(o, s) of the HODBF writes only the rows of o, so the rows
 * split by cluster-tree subtree).  Rank `rank` of `nranks` (a power of two,
 * at most 2^L_v) owns node `rank` of level log2(nranks) of the cluster tree:
 * the tree positions [*lo, *hi) (hb_shard_rows; their natural indices are
 * hb_tree_perm's entries lo .. hi - 1).
 * hb_apply_shard: s is the whole input (every rank's cells, natural order,
 * as after an all-gather); computes every task whose rows meet the rank's
 * and writes u on the rank's cells only (other cells of u untouched).  Its
 * values there equal hb_apply's bit for bit.
 * hb_apply_shard_adjoint: u holds the rank's cells (its other cells are
 * ignored, read as zero); computes the tasks whose rows meet the rank's
 * with the other ranks' skeleton vectors zero and writes the rank's share
 * of s = h^2 K^H u on every cell; the shares of all ranks add up to
 * hb_apply_adjoint's result (a reduce-scatter or all-reduce across ranks).
 * Both run with the handle's precision, one launch per dependency depth in
 * the mixed path.  Errors as hb_apply; HB_ERR_ARG for a bad nranks / rank. */
hb_status hb_shard_rows(hb_handle h, int nranks, int rank, long long* lo, long long* hi);
hb_status hb_apply_shard(hb_handle h, const void* s, void* u, int nrhs, int nranks, int rank, void* stream);
hb_status hb_apply_shard_adjoint(hb_handle h, const void* u, void* s, int nrhs, int nranks, int rank,
                                 void* stream);
/* hb_host_shard_rows: hb_shard_rows for an nx x ny grid and leaf size,
 * without a handle or a device. */
hb_status hb_host_shard_rows(int nx, int ny, int leaf, int nranks, int rank, long long* lo, long long* hi);

/* hb_set_precision: HB_FP64 or HB_MIXED_BF16X3 for later applies. */
hb_status hb_set_precision(hb_handle h, int precision);

/* hb_set_wait_selftest: failure-detection self-test of the mixed apply (no
 * counterpart in the paper).  When on != 0, the first warp of every step
 * launch of later mixed applies also waits - with the same bounded wait as
 * the data waits and the handle's barrier_cycles budget - on an mbarrier
 * that nothing completes; the wait runs out and sets the mapped error word,
 * and the apply otherwise completes normally, so a later hb_apply /
 * hb_apply_adjoint (called after the device has run it) returns
 * HB_ERR_TIMEOUT.  No fault or hang is involved;
 * each launch spends about barrier_cycles SM cycles in the wait.
 * Errors: HB_ERR_ARG for a null handle. */
hb_status hb_set_wait_selftest(hb_handle h, int on);

/* hb_device_alloc_cap: test hook for the out-of-memory paths.  Every device
 * allocation of the library is counted; with cap_bytes > 0 an allocation
 * that would take the live total above cap_bytes fails as a real
 * out-of-memory does (HB_ERR_OOM from the call that needed it); 0 removes
 * the cap, a negative value leaves it unchanged.  *live_bytes (if not NULL)
 * receives the bytes the library holds now.  Process-wide, not tied to a
 * handle; no device work.  A build that fails for lack of memory frees what
 * it allocated and leaves the handle unbuilt (hb_build may be called
 * again); an apply that fails for lack of scratch may be repeated. */
hb_status hb_device_alloc_cap(long long cap_bytes, long long* live_bytes);

/* hb_apply_dense / hb_apply_dense_adjoint: the same sums (Eq. m_v2v) and
 * their adjoint, matrix free, every entry evaluated in FP64 on the fly
 * (Eq. chebinterpblock, Eq. babich, Appendix A).  Needs no hb_build.
 * Same layout and limits as hb_apply.  On grids with fewer than eight
 * 64-cell output segments per SM the source lines are split over CTAs and
 * the first such call allocates the per-share partial sums (owned by the
 * handle, freed by hb_destroy): make that first call outside a CUDA graph
 * capture.  Results do not depend on the split being taken or not beyond
 * the order of the FP64 additions. */
hb_status hb_apply_dense(hb_handle h, const void* s, void* u, int nrhs, void* stream);
hb_status hb_apply_dense_adjoint(hb_handle h, const void* u, void* s, int nrhs, void* stream);

/* hb_entries: K[rows, cols] for index lists (natural order, int64, HOST
 * arrays), written as an m x n complex128 column-major DEVICE array `out`
 * (Eq. chebinterpblock + Eq. babich; diagonal pairs rows[a] == cols[b] give
 * the self term of Appendix A).  Synchronous.  Errors: HB_ERR_ARG for
 * m, n < 1 or an index outside [0, N_v). */
hb_status hb_entries(hb_handle h, const long long* rows, int m, const long long* cols,
                     int n, void* out, void* stream);

/* Scattering by a curve inclusion (Sec. 3.2).  The curve is given as ns
 * straight segments: centers (ns x 2, row-major (x, z) pairs), lengths w_i
 * and the refractive index n_i at each centre, all HOST arrays.  With
 * g = v0 f0 + v1 f1 interpolated at the points from the handle's tables:
 *   K^{s2s}_ij = -g(r^s_i, r^s_j) w_j for i != j (Eq. s2s), and on the
 *     diagonal -(i w_i/4)(1 + (2i/pi)(ln(gamma omega n_i w_i / 4) - 1)),
 *     gamma = e^{Euler's constant}: minus the integral of (i/4) H0(omega n_i |t|)
 *     over the segment in its small-argument form;
 *   K^{v2s}_ij = g(r^s_i, r_j) (Eq. m_v2s),  K^{s2v}_ij = g(r_i, r^s_j) w_j
 *     (Eq. m_s2v), r_j the cell centres.
 * The total field vanishes on the curve (Eq. sie; Eq. m_sie: K^{s2s} P = U^inc).
 *
 * hb_curve_set: evaluates the three operators densely on the device and
 * factors K^{s2s} (LU with partial pivoting) and keeps its inverse (N_s^2
 * more complex values); replaces an earlier curve.
 * Synchronous.  Device memory: (2 ns N_v + 2 ns^2) x 16 bytes plus 2 ns x
 * nrhs x 16 bytes at the first hb_apply_inclusion, owned by the handle until the
 * next hb_curve_set or hb_destroy.  Errors: HB_ERR_ARG for ns outside
 * [1, 16384], a non-finite centre, a length or n that is not positive, or a
 * singular K^{s2s} (the handle then has no curve); HB_ERR_OOM. */
hb_status hb_curve_set(hb_handle h, const double* centers, const double* lengths, const double* n_seg,
                       long long ns);

/* hb_curve_operators: K^{s2s} (ns x ns), K^{v2s} (ns x N_v) and K^{s2v}
 * (N_v x ns) of the curve, evaluated again into caller-owned DEVICE
 * complex128 column-major buffers (any of them NULL to skip it).
 * Asynchronous on `stream`.  Errors: HB_ERR_STATE without a curve. */
hb_status hb_curve_operators(hb_handle h, void* k_s2s, void* k_v2s, void* k_s2v, void* stream);

/* hb_apply_inclusion: the total field with the inclusion (Eq. m_v2v_inclu),
 *   u = (K^{v2v} + K^{s2v} (K^{s2s})^{-1} K^{v2s}) (h^2 s),
 * s, u as for hb_apply.  K^{v2v} is applied matrix free in FP64 when
 * v2v_dense != 0 (no hb_build needed), else by the compressed operator in
 * the handle's precision (needs hb_build); the surface part runs in FP64.
 * The first call with more right-hand sides than before allocates the
 * surface vectors: make it outside a CUDA graph capture.  Errors:
 * HB_ERR_STATE without a curve, or v2v_dense == 0 before hb_build. */
hb_status hb_apply_inclusion(hb_handle h, const void* s, void* u, int nrhs, int v2v_dense, void* stream);

/* hb_curve_compress: K^{v2s} and K^{s2v} of the curve set with hb_curve_set
 * as butterflies (Sec. 4.2, the K^{v2s} / K^{s2v} items; Sec. 4.2.1): one
 * each between the cells' cluster tree and a K-D tree over the segment
 * centres with leaves of at most leaf_s segments, both cut at L = min(L_v,
 * L_s) levels; proxy rows by Eq. proxyv2v with the other set's points as
 * seeds (the handle's chi and nbr_radius_h), IDs at the handle's eps.  The
 * dense K^{v2s} / K^{s2v} are freed; hb_apply_inclusion then applies the
 * butterflies (FP64) around the inverse of K^{s2s}.  A later hb_curve_set
 * or hb_set_omega drops them.  Synchronous.  Errors: HB_ERR_STATE without
 * a curve, HB_ERR_ARG (leaf_s < 1), HB_ERR_UNSUPPORTED (an empty tree node),
 * HB_ERR_OOM, HB_ERR_CUDA.
 * hb_curve_info: of the compressed K^{v2s} (which = 0) or K^{s2v} (1): its
 * levels L, largest rank and stored complex entries.  HB_ERR_STATE before
 * hb_curve_compress. */
hb_status hb_curve_compress(hb_handle h, int leaf_s);
hb_status hb_curve_info(hb_handle h, int which, int* levels, int* max_rank, long long* entries);

/* Table builder for media without closed-form ingredients (Sec. 2.3 and
 * Sec. 4.1): the tables hb_create takes, computed on the device.
 *
 * hb_sweep_taylor: the near-source Taylor numbers of ns source points from
 * the series of n^2 about each (Sec. 2.2, d = 2: Eq. recursiveT, Eq.
 * recursiveB, Eq. C0, Eq. C1, Eq. recursiveC).  s2: HOST ns x 15, row k =
 * S_0..S_4 of n(r_k + (X, Z))^2 = sum_j S_j(X, Z), piece j = j + 1
 * coefficients of X^(j-m) Z^m, m = 0..j; S_0 = n(r_k)^2 > 0.  taylor: HOST
 * ns x 46 out, row k = T_2..T_6, B_0..B_4, C_0..C_2 (the pieces of the
 * expansions Eq. expansionT, Eq. expansionV0, Eq. expansionV1 in the same
 * layout).  Errors: HB_ERR_ARG (null array, ns < 0, S_0 <= 0).
 *
 * hb_sweep_tables: per source node, the factored eikonal (Eq. faceik) on
 * the mesh x_i = lo + i h, z_j = lo + j h (i, j < M) and the transports of
 * v0 and v1 (Eq. equVs) on its window [w0, w1]^2 (region of interest
 * [roi0, roi1]^2 in window indices) by Lax-Friedrichs WENO5 Gauss-Seidel
 * sweeping (four orderings per iteration, until the largest update over the
 * window - resp. the region of interest - is below tol, at most max_iter
 * iterations), the points within 5 h (eikonal), 3 h (v0) and 1 h (v1) of
 * the source fixed at their Taylor values, then 4 x 4 local cubic
 * interpolation to the NI observation points.  n_mesh: HOST M x M, n at
 * (x_i, z_j) in [j][i].  px, pz: HOST NI point coordinates (the tensor
 * Chebyshev nodes of hb_tables, x fastest).  src: HOST ns node indices of
 * the sources, taylor: HOST ns x 46 (hb_sweep_taylor).  Out (HOST, NI x ns
 * row-major, [observation][source]): tau2, v0, v1 - the tables' columns
 * src[k] (at a source's own node tau2 is 0, v0 = B_0 and v1 = C_0 by
 * Eq. expansionT..V1: set those entries, which the interpolation only
 * approximates); info: HOST ns x 6, the iterations and the last largest
 * update of the three solves.  One CTA per source; each anti-diagonal of a
 * sweep is updated in parallel, which gives the row-by-row Gauss-Seidel
 * iterates bit for bit.  Device memory: ns x (5 M^2 + 7 (w1 - w0 + 1)^2) x
 * 8 bytes.  Synchronous.  Errors: HB_ERR_ARG (null array, bad mesh - M < 8,
 * h <= 0, window outside the mesh or under 8 points, region of interest
 * outside the window - node index out of range, S_0 <= 0), HB_ERR_OOM,
 * HB_ERR_CUDA. */
hb_status hb_sweep_taylor(int ns, const double* s2, double* taylor);
hb_status hb_sweep_tables(int M, double lo, double h, int w0, int w1, int roi0, int roi1, const double* n_mesh,
                          int NI, const double* px, const double* pz, int ns, const int* src, const double* taylor,
                          int max_iter, double tol, double* tau2, double* v0, double* v1, double* info);

/* hb_id_batch: batched column-pivoted QR interpolative decompositions
 * (Eq. ID) of `count` complex128 matrices, with the same rules as the build:
 * pivot on the largest recomputed trailing column norm (lowest index on exact
 * ties), rank = first k >= 1 with |R_kk| <= eps |R_00|, V = [I | R11^-1 R12] P^T.
 * A: DEVICE, matrix b is m[b] x n[b] column-major at element offset a_off[b];
 * it is overwritten.  m, n, a_off: HOST arrays of length count.
 * Outputs (DEVICE): rank[b]; skel + sum_{c<b} n[c]: the rank[b] skeleton
 * column indices in pivot order; V + sum_{c<b} n[c]^2: the rank x n[b]
 * matrix V, column-major with leading dimension n[b].  Synchronous. */
hb_status hb_id_batch(int count, const int* m, const int* n, const long long* a_off,
                      void* A, double eps, int* rank, int* skel, void* V);

/* hb_id_batch_noalloc: the decompositions of hb_id_batch, with the same
 * arguments, layouts and results (skel receives the full pivot order of each
 * matrix, its first rank[b] entries being the skeleton), for callers that
 * cannot allocate device memory: code running under another framework's
 * memory manager, which has reserved the device memory for its own pool (a
 * raw cudaMalloc can then fail, or stall every stream with its implicit
 * synchronisation), and latency-critical paths that must not take that
 * synchronisation.  The paper has no counterpart: this is a library
 * interface concern, not part of the method.
 * It calls no cudaMalloc / cudaFree and no allocating library routine: the
 * per-matrix sizes and offsets the kernels read on the device go to a 2 MiB
 * static device array that every GPU loading the library keeps until the
 * process exits.  Limit: count <= 65536 matrices (larger counts return
 * HB_ERR_ARG with a message; nothing is launched).
 * Asynchronous on `stream` (NULL = legacy default stream).  The host arrays
 * m, n, a_off, pageable or page-locked, may be reused or freed on return:
 * the call copies them into a static host array (pageable memory) before it
 * enqueues the host-to-device copy, which has then consumed its source.
 * Host threads calling this entry point serialise on a mutex for the
 * duration of the call's enqueueing.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) for that device: make
 * that first call before any stream capture.  All calls share the array,
 * whose contents after a call are that call's metadata; each call writes
 * everything it reads, so nothing must start at zero, but calls that
 * overlap on the GPU (other streams or host threads without a
 * synchronisation in between) race on it. */
hb_status hb_id_batch_noalloc(int count, const int* m, const int* n, const long long* a_off,
                              void* A, double eps, int* rank, int* skel, void* V, void* stream);

/* hb_fp64_fma_peak: the measured FP64 rate of the current device in
 * TFLOP/s (2 flops per fused multiply-add), from a kernel of independent
 * FMA recurrences filling every SM, timed with CUDA events on `stream`
 * (best of three after a warm-up run; synchronous, ~milliseconds).  The
 * denominator of the FP64 rooflines (the paper's method has no counterpart:
 * a measurement utility).  Errors: HB_ERR_ARG, HB_ERR_CUDA. */
hb_status hb_fp64_fma_peak(double* tflops, void* stream);

/* hb_launch_shape: the launch shape the mixed apply uses for one direction
 * (adjoint 0 or 1) and m-tile count (mtiles 1: up to 16 right-hand sides
 * per pass, 2: up to 32): *mode = 0 for a gather plus one launch per
 * dependency depth, 1 for one persistent dataflow launch (the gather
 * inside), 2 for a gather plus one launch per depth with the leaf outputs
 * on the tcgen05 tensor-core kernel, 3 for the cone launch then one launch
 * per remaining depth, 4 for that with the tcgen05 leaf kernel, 5 for the
 * fused level pairs, 6 for those with the tcgen05 leaf kernel, 7 for every
 * depth in one launch with grid barriers, -1 if no
 * apply has run yet at that m-tile count; *item_bytes the
 * item size the accumulation chains are cut to, *stages the shared-memory
 * ring stages per warp, *pub_batch the chains a dataflow warp publishes
 * together, *slack the dataflow placement's margin between a producer's
 * simulated finish and its consumers (cost units: one per 512-byte factor
 * tile, four per item), *tuned_ms the autotuner's time for the chosen shape
 * (0 when it did not run) and *candidates the shapes it timed.
 * HB_ERR_STATE before hb_build. */
hb_status hb_launch_shape(hb_handle h, int adjoint, int mtiles, int* mode, int* item_bytes, int* stages,
                          int* pub_batch, int* slack, double* tuned_ms, int* candidates);

/* hb_record_id_blocks / hb_recorded_id_count / hb_recorded_id_block: keep,
 * for a check of the interpolative decomposition (Sec. 4.2.1, Eq. ID, on the
 * blocks of Eq. proxy), copies of the sampled blocks that hb_build hands to
 * its ID.  Call hb_record_id_blocks before hb_build (HB_ERR_STATE after):
 * at every butterfly level k the build then keeps up to per_level of that
 * level's blocks, every (blocks / per_level)-th one in the build's job order
 * (0 = keep none, the default).  Each kept record holds the level k, the
 * proxy rows and the column set as natural indices (m and n of them), the
 * sampled m x n block as the ID received it (complex128, column-major), the
 * rank the ID chose and its full pivot order (n positions in the column
 * set; the first rank of them are the skeleton).  hb_recorded_id_block
 * copies record `index` into HOST arrays: level, m, n and rank always;
 * rows (m), cols (n), A (m*n complex128) and pivots (n) unless NULL, so a
 * first call with NULL arrays returns the sizes.  Records live until the
 * handle is destroyed.  Errors: HB_ERR_ARG (index out of range). */
hb_status hb_record_id_blocks(hb_handle h, int per_level);
hb_status hb_recorded_id_count(hb_handle h, int* count);
hb_status hb_recorded_id_block(hb_handle h, int index, int* level, int* m, int* n, long long* rows,
                               long long* cols, void* A, int* rank, int* pivots);

/* hb_tree_perm: copy the cluster-tree permutation (tree position ->
 * natural index, N_v int64) to a HOST array.  Valid after hb_create. */
hb_status hb_tree_perm(hb_handle h, long long* perm_out);

/* hb_host_cluster_tree / hb_host_proxy_rows: the host rules of hb_create and
 * hb_build without a handle or a device, for an nx x ny grid: the K-D
 * cluster tree (split the longer side of the node's bounding box in cells,
 * order by (coordinate, natural index), first child ceil(n/2); L_v = the
 * smallest L with ceil(N_v / 2^L) <= leaf; leaves in natural order) and the
 * proxy rows of Eq. proxyv2v (as hb_proxy_rows, with chi and the neighbour
 * radius in cells given here).  HOST arrays: perm_out N_v int64 (NULL to
 * skip), bounds_out the node boundaries of levels 0..L_v concatenated
 * (2^l + 1 per level; NULL to skip), *levels = L_v.  Errors: HB_ERR_ARG. */
hb_status hb_host_cluster_tree(int nx, int ny, int leaf, long long* perm_out, long long* bounds_out, int* levels);
hb_status hb_host_proxy_rows(int nx, int ny, int leaf, double chi, double nbr_radius_h, long long t0, long long t1,
                             const long long* seeds, int nseeds, long long* out, long long* count);

/* hb_host_segment_tree: the K-D tree T_{H_s} over ns curve segment centres
 * (centers: HOST ns x 2 (x, z) pairs) by the cluster tree's rule on real
 * coordinates (split the longer side of the node's bounding box, order by
 * (coordinate, segment index), first child ceil(n/2); leaves in index
 * order), the column tree of the compressed surface operators (Sec. 4.2,
 * the K^{s2v} and K^{s2s} items).  Outputs as hb_host_cluster_tree.
 * Errors: HB_ERR_ARG. */
hb_status hb_host_segment_tree(const double* centers, long long ns, int leaf, long long* perm_out,
                               long long* bounds_out, int* levels);

/* hb_host_point_proxy_rows: Eq. proxyv2v between two point sets, the rule of
 * the compressed surface operators (rows: cells or segment centres in tree
 * order; seeds: points of the other set): m = min(t1 - t0, ceil(chi nseeds))
 * rows of [t0, t1) at positions t0 + floor(k (t1 - t0) / m), plus every row
 * of [t0, t1) within `radius` (domain units) of a seed.  rows_xz: HOST
 * nrows x 2, seeds_xz: HOST nseeds x 2; out: HOST, capacity t1 - t0, sorted
 * positions; *count their number.  Errors: HB_ERR_ARG. */
hb_status hb_host_point_proxy_rows(const double* rows_xz, long long nrows, long long t0, long long t1,
                                   const double* seeds_xz, int nseeds, double chi, double radius, long long* out,
                                   long long* count);

/* hb_proxy_rows: the proxy-row rule Eq. proxyv2v for the row node
 * tau = tree positions [t0, t1) and seed columns `seeds` (tree positions,
 * HOST).  Writes the sorted proxy tree positions to the HOST array out
 * (capacity t1 - t0) and their number to *count. */
hb_status hb_proxy_rows(hb_handle h, long long t0, long long t1, const long long* seeds,
                        int nseeds, long long* out, long long* count);

hb_status hb_info(hb_handle h, hb_stats* stats);

/* hb_rank_profile: the ranks r_{tau,nu} of the built HODBF by HODBF level l
 * (the 2^l butterflies between sibling clusters of level l, l = 1..L_v) and
 * butterfly level k (k = 0: V^0; k = 1..L_v - l: W^k, the last also giving
 * K^L's columns).  max_rank (int) and mean_rank (double) are HOST arrays of
 * (L_v + 1) x (L_v + 1) entries, row-major [l][k]; entries without blocks
 * (l = 0, k > L_v - l) are 0.  Sec. 4.2.2 relates them to the cluster sizes:
 * bounded away from the middle level, growing near it.  Synchronous (host
 * data only).  Errors: HB_ERR_STATE before hb_build. */
hb_status hb_rank_profile(hb_handle h, int* max_rank, double* mean_rank);

/* hb_kernel_times: enable (1) / disable (0) CUDA-event timing of every
 * kernel launched by hb_apply / hb_apply_adjoint on the launch stream, and
 * read back the accumulated per-kernel-group totals: names, total ms and
 * launch counts for up to `cap` groups (HOST arrays); *ngroups receives the
 * number of groups.  Reading resets the totals.  Synchronous. */
hb_status hb_set_kernel_timing(hb_handle h, int enable);
hb_status hb_kernel_times(hb_handle h, int cap, char (*names)[32], double* total_ms,
                          long long* launches, int* ngroups);

const char* hb_last_error(hb_handle h);
void hb_destroy(hb_handle h);

#ifdef __cplusplus
}
#endif
#endif /* HB_H_ */
