/*
 * dh2.h - C ABI of the GB300 hybrid DH^2 library.
 *
 * Hybrid compression of the Galerkin matrix of the Helmholtz single layer
 * operator (Boerm & Boerst, "Hybrid matrix compression for high-frequency
 * problems"): directional Chebyshev interpolation (Section 2) followed by
 * algebraic recompression (Section 3.2), and the matrix-vector product of the
 * resulting DH^2 matrix.
 *
 * Conventions for every entry point:
 *   - The return value is a dh2_status: 0 (DH2_OK) or a negative error code.
 *     No C++ exception crosses this boundary.  dh2_last_error() returns a
 *     thread-local, NUL-terminated description of the last failure.
 *   - Handles (dh2_tree, dh2_matrix) are opaque and owned by the library;
 *     release them with dh2_free_tree / dh2_free_matrix.  A matrix keeps a
 *     reference to nothing but its own copies: the tree may be freed first.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device pointers must be valid on the current CUDA device.
 *   - Device memory of the library comes from the device's default memory
 *     pool, allocated and freed in stream order on the call's stream.  The
 *     library sets the pool's release threshold to a quarter of the device's
 *     memory: up to that much freed memory stays mapped for reuse.
 *   - Invalid arguments are rejected with DH2_EINVAL before any GPU work.
 *   - Complex vectors are interleaved (re, im) pairs: DH2_C64 = 2 x float,
 *     DH2_C128 = 2 x double.
 *   - All index arrays are int32 and 0-based.
 */
#ifndef DH2_H
#define DH2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DH2_OK = 0,
    DH2_EINVAL = -1,        /* invalid argument (detected on the host, no GPU work done) */
    DH2_ENOMEM = -2,        /* device or host allocation failed */
    DH2_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed */
    DH2_ETIMEOUT = -4,      /* a bounded device-side wait gave up */
    DH2_ENUMERIC = -5,      /* NaN/Inf or a non-converged factorisation */
    DH2_EUNSUPPORTED = -6   /* valid but not supported by the library (e.g. k too large) */
} dh2_status;

enum { DH2_FP64 = 0, DH2_MIXED = 1 };                 /* dh2_options.precision */
enum { DH2_C64 = 1, DH2_C128 = 2 };                   /* vector dtypes */
enum { DH2_RANK_BLOCKREL = 0, DH2_RANK_GLOBAL = 1, DH2_RANK_SPECTRAL = 2 };  /* dh2_options.rank_rule */
enum { DH2_FAULT_NONE = 0, DH2_FAULT_TIMEOUT = 1, DH2_FAULT_NONFINITE = 2, DH2_FAULT_ALLOC = 3 };  /* dh2_options.fault */
enum { DH2_SINGLE_LAYER = 0, DH2_DOUBLE_LAYER = 1 };  /* dh2_options.layer */

typedef struct dh2_tree_s* dh2_tree;
typedef struct dh2_matrix_s* dh2_matrix;
typedef struct dh2_model_s* dh2_model;   /* learned order/rank model, see below */

typedef struct {
    double eta1;            /* direction parameter eta_1 of Eq. (3a)/(4); paper: 10 (Section 5) */
    int32_t leaf_max;       /* clusters with at most leaf_max elements are leaves; paper: 32 */
    int32_t precision;      /* DH2_FP64: complex FP64 everywhere.  DH2_MIXED: complex FP32
                               kernel evaluation, coupling and projection GEMMs (3xTF32 on the
                               tensor cores) and matvec storage; the weight QRs and the SVD
                               truncation in FP64 (qr_fp64 = svd_fp64 = 1, the defaults) or,
                               with both set to 0, in FP32 (the all-FP32 variant) */
    int32_t rank_rule;      /* DH2_RANK_BLOCKREL: sum_{i>k} sigma_i^2 <= eps^2 with every block
                               weighted by 1/|G_b|_F (blockwise relative Frobenius, Section 5);
                               DH2_RANK_GLOBAL: <= eps^2 sum_i sigma_i^2, unweighted;
                               DH2_RANK_SPECTRAL: sigma_{k+1} <= eps with the block weights
                               of DH2_RANK_BLOCKREL (error control in the spectral norm,
                               Section 5) */
    int32_t qr_fp64;        /* weight QRs (R, Z-hat) and the orthogonalisation of the leaf bases:
                               1 (default) = FP64 Cholesky QR: the FP64 Gram matrix Z^* Z of the
                               stack and its pivoted Cholesky factor R (R^* R = Z^* Z; pivots below
                               16 u_64 max diag(Z^* Z) are dropped as rounding noise), FP64 Jacobi
                               for the leaves; 2 = FP64 Householder; 0 = FP32 Householder and FP32
                               one-sided Jacobi (DH2_MIXED only; the FP64 form treats 0 as 1) */
    int32_t qr_group_rows;  /* stacks taller than this are factored in row groups whose R
                               factors are stacked and factored again (0 = 1024 rows; never
                               below twice the stack's columns) */
    int64_t workspace_bytes;/* cap on the stacked weight workspace per level (0 = 16 GiB) */
    int32_t tensor_cores;   /* DH2_MIXED with m <= 5: 1 (default) = coupling products of the
                               total weights on the tcgen05 tensor cores in 3xTF32 (FP32-level
                               accuracy); 0 = FP32 CUDA-core products */
    int32_t kb_store;       /* with the tensor-core path: 0 (default) = keep the block products
                               K_b = R_t S_b R_s^* for the column pass and the projection of leaf
                               pairs when they take at most a quarter of the free device memory,
                               recompute them otherwise; 1 = always keep; 2 = always recompute */
    int32_t learned;        /* 1 = choose the interpolation order and cap the truncation ranks
                               with `model` (see "Learned order and rank" below); the m argument
                               of the build is then ignored.  0 (default) = the plain fixed-order
                               method */
    int32_t svd_fp64;       /* DH2_MIXED only: 1 (default) = SVD truncation through the FP64 Gram
                               matrix and an FP64 Hermitian Jacobi eigensolver; 0 = FP32
                               one-sided Jacobi on the rows of A */
    dh2_model model;        /* the model used when learned = 1 (not owned) */
    int32_t qr_tpc[3];      /* FP32 weight QRs of at most 32, 64 and 128 columns: threads per
                               column of the column-parallel kernel, which sets the rows per
                               chunk (16 x threads); 0 = the defaults 8, 4, 2; allowed
                               1, 2, 4, 8 with threads x class width <= 256 (dh2_autotune
                               picks them) */
    int32_t fault;          /* test hook, 0 in normal use: DH2_FAULT_TIMEOUT / DH2_FAULT_NONFINITE
                               make the host find that device error bit set after the projection
                               stage (the build then fails as it would after a real device-side
                               timeout or non-finite value); DH2_FAULT_ALLOC makes the first
                               device allocation of the build fail.  Nothing is injected on the
                               GPU itself */
    int32_t symmetry;       /* 1 (default): use the complex symmetry G^T = G of the Galerkin
                               matrix (Eq. 1, 2) with the point-symmetric direction sets D_l = -D_l
                               (Remark "construction of directions"): the basis weights of (t, -c)
                               and the column-pass total weights, truncated bases and basis-change
                               matrices of (t, c) are the complex conjugates of the row pass at
                               (t, -c), so they are copied instead of computed.  Used only when the
                               host finds the directions, son maps, block tree and sizes symmetric
                               (dh2_matrix_info.symmetric); 0 = compute both passes */
    int32_t direct;         /* 1 = direct recompression during the set-up (Section 5, the low-memory
                               variant of the Boeing run): the leaf bases of each tree level are
                               evaluated and orthogonalised at once and never held for the whole
                               tree, and the intermediates of the recompression (basis weights R,
                               leaf factors P, total weights, transfers, block products K_b) are
                               released as soon as the last stage that reads them is done; the
                               stacked-weight workspace per level defaults to 2 GiB.  The matrix and
                               its products are those of direct = 0; dh2_export_pair of R, P and
                               the total weights then reports DH2_EUNSUPPORTED.  0 (default) =
                               keep them for inspection */
    int32_t layer;          /* DH2_SINGLE_LAYER (default): the single layer operator, kernel g of
                               Eq. (1).  DH2_DOUBLE_LAYER: the double layer operator of the paper's
                               second experiment (Section 5), kernel d/dn_y g(x, y) =
                               exp(i kappa r)(1 - i kappa r) <x - y, n_y> / (4 pi r^3) with the unit
                               normal n_y = (v1 - v0) x (v2 - v0) / |.| of the y element (vertex
                               order); the nearfield by the 3 x 3 interior rule (0 on the diagonal,
                               where x - y lies in the element's plane); rows interpolated as for the
                               single layer (V), columns with the normal derivative of the modified
                               Lagrange polynomials, W_sc = int phi_j d/dn_y [exp(i kappa <y, c>)
                               L_{s,mu}(y)], and separate basis weights for V and W (Section 3.2 with
                               W != V).  The matrix is not symmetric: both passes are computed */
    int32_t gram_tc;        /* DH2_MIXED with qr_fp64 = 1: 1 (default) = the Gram matrices Z^* Z of
                               weight stacks wider than 32 columns from exact integer products on
                               the tensor cores: each real column, scaled by a power of two, is
                               split into 8 signed base-64 digits (BF16), the digit products of
                               one weight summed exactly in FP32 (at most 2048 rows per sum) and
                               combined in FP64; error at most about 2^-43 max|z_m| max|z_n| per
                               row.  0 = FP64 FMAs on the CUDA cores */
} dh2_options;

typedef struct {
    int64_t n;              /* number of elements (triangles) */
    int32_t nclusters;
    int32_t depth;          /* p_I: levels are 0..depth */
} dh2_tree_info;

typedef struct {
    int64_t n;
    int32_t depth;
    int32_t m, k;           /* Chebyshev points per axis, k = m^3 */
    int64_t nadm;           /* admissible leaves of the block tree */
    int64_t nnear;          /* nearfield (inadmissible) leaves */
    int64_t npairs;         /* pairs (t, c), c in D_level(t) */
    int64_t nactive;        /* pairs visited by the recompression */
    int64_t near_entries;   /* stored nearfield coefficients */
    int64_t coupling_entries; /* stored recompressed coupling coefficients */
    int64_t basis_entries;  /* stored leaf bases Q and transfers F, rows + columns */
    int64_t matvec_bytes;   /* algorithmic bytes one matvec streams (matrix + vectors) */
    int32_t max_rank_row, max_rank_col;
    double mean_rank_row, mean_rank_col;
    double stage_ms[16];    /* device time per build stage (see dh2_stage_name) */
    double kernel_ms[16];   /* summed CUDA-event duration per kernel (see dh2_kernel_name):
                               build kernels always, matvec kernels while timing is on */
    int64_t kernel_launches[16]; /* number of timed launches per kernel */
    double kernel_work[16]; /* algorithmic work of each kernel in one build (build kernels) or
                               one matvec (matvec kernels), in the unit of kernel_work_kind */
    int32_t kernel_work_kind[16]; /* 0 none, 1 FP32 flop, 2 FP64 flop, 3 bytes moved,
                                   4 BF16 tensor-core flop */
    int32_t learned_m;      /* the order the learned model chose (0 for a plain build) */
    int32_t rank_cap_retries; /* truncation passes redone because a rank exceeded its learned cap */
    int64_t truncation_bytes; /* device bytes of the truncated bases of both passes as allocated
                               (Q / F, C, U', singular values), which the learned rank caps size */
    int32_t symmetric;      /* 1 when the build derived the column pass from the row pass
                               (dh2_options.symmetry) */
    int32_t direct;         /* 1 for a build with dh2_options.direct */
    int64_t peak_pool_bytes;  /* high-water mark of the device memory the library's stream-ordered
                               pool had handed out during the build (process-wide: concurrent
                               builds count together) */
} dh2_matrix_info;

/* Fills *opt with the paper's parameters: eta1 = 10, leaf_max = 32, DH2_MIXED with FP64
 * weight QRs and FP64 SVD truncation, blockwise relative rank rule, default workspace. */
dh2_status dh2_options_default(dh2_options* opt);

/*
 * Cluster tree (Def. "cluster tree"; Section 5: binary space partitioning to
 * at most leaf_max elements per leaf) and bounding boxes B_t (Section 2).
 * vertices: HOST, FP64 [nv][3].  triangles: HOST, int32 [nt][3], vertex ids in
 * [0, nv); both are copied, the caller keeps ownership.  triangles == NULL
 * selects point mode: every vertex is one element (used by interpolation
 * tests).  The tree is built by GPU kernels on `stream`; the call returns
 * after the tree is complete.  Errors: DH2_EINVAL for nv <= 0, nt < 0, an
 * out-of-range vertex id or NULL pointers; DH2_ENOMEM; DH2_ECUDA.
 */
dh2_status dh2_build_tree(const double* vertices, int64_t nv, const int32_t* triangles,
                          int64_t nt, const dh2_options* opt, void* stream, dh2_tree* out);

/*
 * Builds the recompressed DH^2 matrix for the Helmholtz kernel
 * g(x,y) = exp(i kappa |x-y|)/(4 pi |x-y|) (Eq. 1) with piecewise-constant
 * Galerkin discretisation (Eq. 2):
 *   directions D_l and son maps (Remark "construction of directions"),
 *   block tree with eta = eta_2 of Eq. (3b),(3c) (Def. "block tree"),
 *   nearfield blocks, leaf bases and transfers of the directional Chebyshev
 *   interpolation with m points per axis (k = m^3; Eq. matrix_apx,
 *   nested_apx), then Section 3.2: basis weights, total weights, truncation
 *   at tolerance eps, projection of the couplings (Lemma "Projections").
 * The couplings S_b of the interpolation are never stored: they are evaluated
 * where they are used.  Blocks until the matrix is complete.
 * Errors: DH2_EINVAL for kappa < 0, m not in [1, 8], eta <= 0, eps <= 0;
 * DH2_ENOMEM when a level's workspace exceeds opt->workspace_bytes or the
 * device is full; DH2_ECUDA; DH2_ENUMERIC for NaN/Inf in a factorisation.
 */
dh2_status dh2_build_dh2(dh2_tree tree, double kappa, int32_t m, double eta, double eps,
                         const dh2_options* opt, void* stream, dh2_matrix* out);

/*
 * Batched build (the paper has no counterpart; it builds one matrix at a time):
 * out[i] = dh2_build_dh2(trees[i], kappas[i], m, eta, eps, opt) for i < count.
 * The builds run concurrently: `nstreams` host worker threads (0 = min(count, 8)),
 * each with its own non-blocking CUDA stream on the calling thread's current
 * device, take the meshes largest first from a shared queue, so the kernels of
 * small meshes fill the SMs that the small launches of other meshes leave idle.
 * Each matrix is identical to the one dh2_build_dh2 gives for the same arguments
 * (up to floating-point summation order).  Blocks until all are built.  trees,
 * kappas, out: host arrays of `count` entries; the trees stay owned by the caller.
 * Errors: every argument is checked first (as for dh2_build_dh2, plus count < 0,
 * nstreams < 0, NULL arrays: DH2_EINVAL before any GPU work).  If any build fails,
 * every matrix of the batch is freed, out[] is all NULL and the first failure's
 * status is returned.
 */
dh2_status dh2_build_dh2_batch(const dh2_tree* trees, int32_t count, const double* kappas, int32_t m,
                               double eta, double eps, const dh2_options* opt, int32_t nstreams,
                               dh2_matrix* out);

/*
 * y = G~ x with the recompressed DH^2 matrix: forward transform with the
 * column basis, couplings, backward transform with the row basis, nearfield
 * (derived from Eq. nested and Eq. vsw).  x, y: DEVICE buffers of n complex
 * values of type `dtype` (DH2_C64 or DH2_C128) in the ORIGINAL element order,
 * caller-owned, not aliased.  Asynchronous on `stream`; the library's
 * internal scratch is per matrix, so concurrent matvecs with one matrix on
 * different streams race.  Errors: DH2_EINVAL (bad dtype, NULL), DH2_ECUDA.
 */
dh2_status dh2_matvec(dh2_matrix mat, const void* x, void* y, int32_t dtype, void* stream);

/*
 * Batched product (no counterpart in the paper): y[i] = G~_i x[i] for count
 * distinct matrices, with x[i], y[i] device buffers as in dh2_matvec.  The
 * products are issued on up to eight internal non-blocking streams that wait
 * for `stream` and that `stream` then waits for, so they overlap on the GPU and
 * the call is asynchronous on `stream` like dh2_matvec.  mats, x, y: host arrays
 * of `count` entries.  Errors: DH2_EINVAL for NULL entries, aliased x[i]/y[i],
 * a bad dtype or a matrix that appears twice (its work buffers would be shared);
 * DH2_ECUDA.
 */
dh2_status dh2_matvec_batch(const dh2_matrix* mats, int32_t count, const void* const* x, void* const* y,
                            int32_t dtype, void* stream);

/*
 * Allocation-free variant of dh2_matvec (the paper has no counterpart; this is
 * an interface for callers that cannot call cudaMalloc when they need the
 * product: code recording into a CUDA graph while another framework owns all
 * device memory, real-time host loops where an allocator call may block, or
 * runtimes that give this library a fixed memory budget).  Same arguments,
 * results and stream semantics as dh2_matvec, but the scratch of the product
 * (permuted input, forward/backward basis coefficients) lives in one fixed
 * 16 MiB device array that the library holds on every GPU it is loaded on until
 * the process exits; the call itself allocates nothing.  The first call on a
 * device looks the array's device address up (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents (every kernel writes
 * its scratch before reading it); calls that overlap on the GPU race and must
 * be serialised by the caller.  Errors: DH2_EINVAL when the matrix needs more
 * than 16 MiB of scratch (n complex values of the matrix precision plus the
 * basis coefficients of both transforms, each rounded up to 256 bytes), bad
 * dtype or NULL pointers; DH2_ECUDA.
 */
dh2_status dh2_matvec_noalloc(dh2_matrix mat, const void* x, void* y, int32_t dtype, void* stream);

/*
 * End-to-end matvec from HOST memory: copies x (n complex128, original order)
 * to the device, runs dh2_matvec in the matrix precision, copies y back to
 * the host buffer.  Synchronous.  Pinned host memory gives the fastest copies.
 */
dh2_status dh2_matvec_host(dh2_matrix mat, const double* x_host, double* y_host, void* stream);

/* Reference rows of the Galerkin matrix (Eq. 2) times x, in FP64 on the GPU, for the
 * error of the compressed product on sampled rows: out[i] = sum_j g_{rows[i], j} x_j
 * with the entries of the nearfield (3 x 3 interior Gauss points off the diagonal, the
 * 7-point degree-5 rule against the 3-point rule on it), every column evaluated.
 * rows: HOST int32 [count], original element ids; x: DEVICE complex128 [n], original
 * order; out: HOST complex128 [count].  Blocks until done.  Errors: DH2_EINVAL for NULL
 * pointers, count < 0, a point-mode tree, a row out of range or kappa < 0; DH2_ECUDA. */
dh2_status dh2_dense_rows(dh2_tree tree, double kappa, const int32_t* rows, int32_t count, const double* x,
                          double* out, void* stream);

/* The Gram matrix G = Z^* Z of a complex FP32 matrix, formed as the weight factorisations of
 * the mixed form form it (the first step of their Cholesky QR, Section 3.2's QR of the stacked
 * weights): the real and imaginary parts of Z in FP64 FMAs (gram_tc = 0), or, for more than
 * 32 columns with gram_tc = 1, from exact integer digit products on the tensor cores (see
 * dh2_options.gram_tc), in both cases summed over row groups in FP64.  Exposed so that the
 * product can be checked on its own.
 * z: DEVICE complex64 [rows x ld], row-major (column j of row i at i * ld + j), read only;
 * g: DEVICE complex128 [cols x cols], row-major, written (both triangles; G(i, j) =
 * conj(G(j, i)) exactly).  Blocks until done.  Errors: DH2_EINVAL for NULL pointers, rows
 * outside [1, 2^31), cols outside [1, 512], ld < cols or gram_tc not 0/1; DH2_ENUMERIC if z
 * holds a non-finite value (g is then unspecified); DH2_ETIMEOUT if a bounded tensor-core
 * wait gives up; DH2_ENOMEM; DH2_ECUDA. */
dh2_status dh2_gram(const void* z, int64_t rows, int32_t cols, int64_t ld, int32_t gram_tc, void* g, void* stream);

/* Turns per-launch CUDA-event timing of the matvec kernels on (1) or off (0);
 * the sums are reported in dh2_matrix_info.kernel_ms / kernel_launches (matvec
 * entries are reset by this call).  Timing synchronises the stream per launch. */
dh2_status dh2_set_timing(dh2_matrix mat, int32_t on);

/* Number of kernels this library has launched in this process so far (all
 * devices, all streams).  Library-internal device-wide scans and sorts are not
 * counted. */
int64_t dh2_kernel_launches(void);

/* Waits for `stream` and reports deferred device errors. */
dh2_status dh2_sync(void* stream);

/* Waits for the current device, then returns the freed device memory that the library's
 * stream-ordered pool keeps for reuse to the driver (the pool keeps up to a quarter of the
 * device otherwise).  For processes that also allocate through another allocator (e.g.
 * PyTorch's caching allocator), which cannot use memory the pool holds.  A device
 * allocation of the library that fails does the same once and retries before it reports
 * DH2_ENOMEM.  Errors: DH2_ECUDA. */
dh2_status dh2_release_cached(void);

/*
 * Autotuner (no counterpart in the paper): picks the tile shapes of the FP32 weight
 * QRs (the dominant kernels of a build) for a workload by timing complete builds of
 * it on `stream`.  Coordinate search starting from *base: for the column classes of
 * at most 32, 64 and 128 columns in turn, the threads per column (qr_tpc: 16 x
 * threads rows per chunk), then the row-group size of tall stacks (qr_group_rows in
 * {512, 1024, 2048, 4096}); each candidate is scored by the summed CUDA-event time of
 * the QR kernels over `reps` builds, after one warm-up build.  *tuned = *base with the
 * chosen qr_tpc and qr_group_rows; *tuned_ms and *base_ms (may be NULL) receive the
 * QR time per build of the choice and of *base.  The builds are discarded.  Blocks.
 * Errors: as dh2_build_dh2, and reps < 1 or NULL tuned (DH2_EINVAL).
 */
dh2_status dh2_autotune(dh2_tree tree, double kappa, int32_t m, double eta, double eps, const dh2_options* base,
                        int32_t reps, void* stream, dh2_options* tuned, double* tuned_ms, double* base_ms);

/* ---- Learned order and rank (no counterpart in the paper) ----
 *
 * The paper uses one interpolation order m for the whole matrix (Section 5) and
 * finds every rank k_tc by SVD truncation (Section 3.2).  A dh2_model is a small
 * MLP, 8 -> 128 -> 128 -> 2 with ReLU hidden layers and a linear output, BF16
 * weights and FP32 biases, accumulation in FP32, that maps 8 geometric features of
 * a pair (t, c) to (m_tc / 8, k_tc / 64): the order its interpolation needs and its
 * truncation rank.  A build with opt->learned = 1 computes the features of every
 * pair from the block structure, evaluates the model, builds with the 99th
 * percentile of the orders predicted for the active pairs, rounded down and clamped
 * to [3, 8] (the transfer matrices E of Eq. nested tie the orders of a cluster and
 * its sons, so one order serves the matrix; the training calibrates the order
 * unit's offset so that this reaches the order the training meshes need) and sizes
 * the truncated bases by the predicted ranks (1.25 x + 4 columns per pair) on the
 * levels with D_l = {0}, the kind of pair the training meshes provide; directional
 * pairs keep the structural bound.  The
 * SVD truncation still decides every rank: a pass in which one exceeds its cap is
 * redone with the structural bounds (dh2_matrix_info.rank_cap_retries).
 *
 * Features per pair (t, c), t on level l (FP32, [npairs][8]):
 *   f0 = kappa diam(B_t) / eta1; f1 = atan(sqrt(2) / m_l) / pi, 1 when D_l = {0};
 *   f2 = l / depth; f3 >= f4 >= f5 = extents of B_t / diam(B_t);
 *   f6 = log2(#t) / 16; f7 = max over the admissible blocks (t, s, c) of
 *   diam(B_t) / dist(B_t, B_s) (0 without blocks).
 * Labels come from the method itself: dh2_learned_probe gives the interpolation
 * error of each pair at m = 3..8 (the order label is the smallest m whose error is
 * <= eps / 2), and dh2_export_ranks of a plain build gives the ranks.
 *
 * Parameters are packed FP32: W1 [128][8], b1 [128], W2 [128][128], b2 [128],
 * W3 [2][128], b3 [2] (DH2_MLP_NPARAMS values).  All device arrays are row-major.
 */
enum { DH2_MLP_IN = 8, DH2_MLP_HIDDEN = 128, DH2_MLP_OUT = 2, DH2_MLP_NPARAMS = 17922, DH2_PROBE_ORDERS = 6 };

/* Creates a model on the current device from HOST parameters (copied).  Errors:
 * DH2_EINVAL for NULL pointers or non-finite parameters; DH2_ENOMEM; DH2_ECUDA. */
dh2_status dh2_model_create(const float* params, void* stream, dh2_model* out);
/* Copies the FP32 master parameters to HOST memory (DH2_MLP_NPARAMS floats). */
dh2_status dh2_model_get_params(dh2_model model, float* params);
/* Y = MLP(X): X DEVICE FP32 [n][8], Y DEVICE FP32 [n][2]; asynchronous on `stream`.
 * n = 0 does nothing.  Errors: DH2_EINVAL (NULL, n < 0), DH2_ECUDA. */
dh2_status dh2_model_forward(dh2_model model, const float* X, int64_t n, float* Y, void* stream);
/* Loss L = sum_{s,o} (y_so - t_so)^2 / (2n) and its gradient with respect to the
 * parameters (the BF16 weights' gradient is taken as the master weights'), into
 * DEVICE buffers grad [DH2_MLP_NPARAMS] and loss [1].  X, T: DEVICE FP32 [n][8] and
 * [n][2].  Asynchronous.  Errors: DH2_EINVAL (NULL, n <= 0), DH2_ECUDA. */
dh2_status dh2_model_grad(dh2_model model, const float* X, const float* T, int64_t n, float* grad, float* loss,
                          void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the loss of
 * the batch X, T (as dh2_model_grad); loss (DEVICE, may be NULL) receives the batch
 * loss before the step.  Asynchronous.  Errors: as dh2_model_grad, and lr <= 0. */
dh2_status dh2_model_train_step(dh2_model model, const float* X, const float* T, int64_t n, float lr, float* loss,
                                void* stream);
void dh2_free_model(dh2_model model);

/* Features of every pair (t, c) of the block structure for (tree, kappa, eta,
 * opt->eta1), in pair order tc: features DEVICE FP32 [cap][8]; *npairs receives the
 * number of pairs; with features == NULL only *npairs is computed.  active (HOST
 * int8 [cap], may be NULL) marks the pairs the recompression visits.  Blocks until
 * done.  Errors: as dh2_build_dh2 for the arguments; DH2_EINVAL when cap < npairs
 * (nothing is written then but *npairs). */
dh2_status dh2_learned_features(dh2_tree tree, double kappa, double eta, const dh2_options* opt, void* stream,
                                float* features, int64_t cap, int64_t* npairs, int8_t* active);
/* Interpolation error of every pair at m = 3..8 (HOST FP64 [cap][6], pair order; NULL
 * computes only *npairs; cap < npairs is DH2_EINVAL): for the first 8
 * admissible blocks (t, s, c) of row(t, c), the Chebyshev interpolant of g_c(., y)
 * on the padded box of t (Section 2) against g_c at the 3-point quadrature nodes of
 * up to 8 elements of t and of s; the largest error over the samples divided by the
 * largest |g_c|, maximised over the blocks; 0 for pairs without blocks.  Blocks. */
dh2_status dh2_learned_probe(dh2_tree tree, double kappa, double eta, const dh2_options* opt, void* stream,
                             double* err, int64_t cap, int64_t* npairs);

/* ---- inspection and parity exports (host copies; caller-allocated buffers) ---- */

dh2_status dh2_tree_get_info(dh2_tree tree, dh2_tree_info* out);

/* perm[n]: element index of the i-th position in cluster order.  Cluster
 * arrays of length nclusters: offset, size, parent (-1 at the root), son0 and
 * son1 (-1 at leaves), level.  lo, hi: FP64 [nclusters][3] bounding boxes.
 * Any pointer may be NULL to skip that array. */
dh2_status dh2_tree_export(dh2_tree tree, int32_t* perm, int32_t* offset, int32_t* size,
                           int32_t* parent, int32_t* son0, int32_t* son1, int32_t* level,
                           double* lo, double* hi);

dh2_status dh2_matrix_get_info(dh2_matrix mat, dh2_matrix_info* out);

/* Directions of level l: *count = |D_l|; msplit = m_l (0 if D_l = {0});
 * dirs FP64 [count][3] and sd int32 [count] (index into D_{l+1}; zeros on the
 * last level) if non-NULL. */
dh2_status dh2_export_directions(dh2_matrix mat, int32_t level, int32_t* count, int32_t* msplit,
                                 double* dirs, int32_t* sd);

/* adm int32 [nadm][3] = (t, s, c), near int32 [nnear][2] = (t, s), in the
 * breadth-first order of the block-tree recursion; active int8 [npairs]. */
dh2_status dh2_export_blocks(dh2_matrix mat, int32_t* adm, int32_t* near, int8_t* active);

enum {
    DH2_X_R = 0,        /* basis weight R_tc, rows x k */
    DH2_X_ZROW = 1,     /* total weight Z-hat_tc of the row pass (r_z x k); for a leaf pair in the
                           coordinates of its orthonormal basis P (r_z x r_t, Z' with
                           Z'^* Z' = R Z-hat^* Z-hat R^*) */
    DH2_X_ZCOL = 2,     /* total weight of the column pass (same conventions) */
    DH2_X_SROW = 3,     /* singular values of the row truncation (1 x count) */
    DH2_X_SCOL = 4,
    DH2_X_QROW = 5,     /* leaf: Q_tc (#t x k_tc); non-leaf: [F_t1c; F_t2c] */
    DH2_X_QCOL = 6,
    DH2_X_CROW = 7,     /* basis change C_tc = Q_tc^* V_tc, k_tc x k */
    DH2_X_CCOL = 8,
    DH2_X_P = 9,        /* leaf pair: orthonormal P with V_tc = P R_tc (#t x r_t) */
    DH2_X_RW = 10,      /* column basis weight R_W,tc (double layer; equals DH2_X_R otherwise) */
    DH2_X_PW = 11       /* leaf pair: orthonormal P_W with W_tc = P_W R_W,tc (double layer) */
};
/* Copies one per-pair matrix as complex128 (interleaved, row-major) into out
 * (capacity `cap` complex values; singular values are stored as (sigma, 0)).
 * *rows, *cols receive the shape; a pair that is not active gives 0 x 0. */
dh2_status dh2_export_pair(dh2_matrix mat, int32_t which, int64_t tc, double* out, int64_t cap,
                           int32_t* rows, int32_t* cols);

/* Ranks k_tc of the row and column bases, int32 [npairs] (-1 if inactive). */
dh2_status dh2_export_ranks(dh2_matrix mat, int32_t* rank_row, int32_t* rank_col);

/* Name of build stage i for dh2_matrix_info.stage_ms (NULL past the end). */
const char* dh2_stage_name(int32_t i);

/* Name of kernel i for dh2_matrix_info.kernel_ms (NULL past the end). */
const char* dh2_kernel_name(int32_t i);

/* Release a handle (NULL is ignored).  Both wait for the device first, since
 * work queued on any stream may still read the object; the memory returns to
 * the device's default pool. */
void dh2_free_tree(dh2_tree tree);
void dh2_free_matrix(dh2_matrix mat);
const char* dh2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DH2_H */
