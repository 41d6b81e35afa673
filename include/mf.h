/*
 * mf.h -- C ABI of the GB300 butterfly-compressed multifrontal solver.
 *
 * The solver factors a sparse complex matrix A (N x N, CSR) by the
 * multifrontal method in nested-dissection order (paper Sec. 2, Alg. 1) and
 * compresses the large fronts in the hierarchically off-diagonal butterfly
 * format (Sec. 4-5, Alg. 5), then solves A x = b to a relative residual
 * ||b - A x|| / ||b|| <= rtol with FP64 GMRES(30) or iterative refinement
 * preconditioned by the factorization (Sec. 6).
 *
 * Conventions
 *  - Complex numbers are interleaved pairs of doubles (re, im) at this ABI.
 *  - Right-hand sides and solutions are column-major N x nrhs with leading
 *    dimension ld (in complex elements, ld >= N).
 *  - Every call returns MF_OK (0) or a negative MF_ERR_* code; the message of
 *    the last failure is available from mf_last_error().  A failed call
 *    leaves the handle valid for mf_destroy().
 *  - The caller owns every input array; the library copies what it keeps.
 *    The handle owns all device memory it allocates and frees it in
 *    mf_destroy().
 *  - One handle is used by one host thread at a time; different handles may
 *    be used concurrently on different CUDA streams.
 */
#ifndef MF_H_
#define MF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MF_OK = 0,
  MF_ERR_ARG = -1,            /* invalid argument                                        */
  MF_ERR_STATE = -2,          /* call out of order (e.g. solve before factor)            */
  MF_ERR_UNSUPPORTED = -3,    /* input outside what the ordering rule handles            */
  MF_ERR_OOM = -4,            /* device or host allocation failed                        */
  MF_ERR_SINGULAR = -5,       /* zero pivot in a front (front id in the message)         */
  MF_ERR_NO_CONVERGENCE = -6, /* refinement stopped above rtol; x and info still written */
  MF_ERR_TIMEOUT = -7,        /* a bounded device wait expired                           */
  MF_ERR_CUDA = -8            /* CUDA runtime error                                      */
};

enum { MF_LATTICE_NODE = 0, MF_LATTICE_EDGE = 1 };
enum { MF_PREC_C64 = 0 /* complex64 factors + FP64 refinement */, MF_PREC_C128 = 1 /* all complex128 */ };
enum { MF_REFINE_NONE = 0, MF_REFINE_GMRES = 1, MF_REFINE_IR = 2 };

#define MF_OPTIONS_V1 1   /* the options up to coords */
#define MF_OPTIONS_V2 2   /* adds ordering; mf_options_init fills version 2 */

/* Nested-dissection ordering (mf_options.ordering):
 *   MF_ORDER_AUTO: planar separators when coords are given, graph nested dissection otherwise;
 *   MF_ORDER_HYBRID: planar separators while they are compressed (|I^s| >= nmin_sep); a box
 *     whose planar separator would be smaller (a dense front) is ordered by graph nested
 *     dissection of its unknowns, which leaves less fill in the dense fronts (needs coords);
 *   MF_ORDER_GRAPH: graph nested dissection even when coords are given. */
enum { MF_ORDER_AUTO = 0, MF_ORDER_HYBRID = 1, MF_ORDER_GRAPH = 2 };

/* Options.  mf_options_init() fills the defaults given in brackets. */
typedef struct {
  int32_t version;        /* MF_OPTIONS_V2 (MF_OPTIONS_V1: the fields up to coords)             */
  int32_t leaf_size;      /* [64]   nested-dissection leaf (unknowns per leaf front)            */
  int32_t nmin_sep;       /* [1024] fronts with |I^s| >= nmin_sep are HOD-BF compressed (Alg. 5) */
  int32_t hodbf_leaf;     /* [64]   leaf size of the HOD-BF and butterfly cluster trees          */
  int32_t max_rank;       /* [0]    cap on every ID rank, 0 = none                               */
  int32_t alpha;          /* [2]    uniform proxy oversampling (Sec. 3.1)                        */
  int32_t knn;            /* [8]    graph nearest neighbours per point (Sec. 5.2)                */
  int32_t precision;      /* [MF_PREC_C64]                                                      */
  int32_t refine;         /* [MF_REFINE_GMRES]                                                  */
  int32_t gmres_restart;  /* [30]                                                               */
  int32_t max_iters;      /* [300]  cap on Krylov iterations (or refinement steps) per column   */
  int32_t lattice;        /* [MF_LATTICE_NODE] how coords are read (see mf_analyze)             */
  double rtol;            /* [1e-8] target ||b - A x|| / ||b||                                  */
  uint64_t seed;          /* [1]    seed of the random sketches                                 */
  const int32_t* coords;  /* [NULL] N x 3 integer lattice coordinates; NULL: graph ordering    */
  int32_t ordering;       /* [MF_ORDER_AUTO] MF_ORDER_*                                         */
  int32_t parallel_levels;/* [0] the planar rule cuts the top parallel_levels levels along the root
                           * separator's axis (while a box extends >= 3 units along it): parallel
                           * instead of crossing separators there (the remedy of the remark in
                           * Sec. 5.3 for F12 / F21 ranks between crossing separators)            */
} mf_options;

typedef struct {
  int32_t iters;          /* Krylov iterations (or refinement steps), max over columns */
  int32_t converged;      /* 1 if every column met rtol                                 */
  double max_rel_residual;/* max over columns of ||b - A x|| / ||b|| (FP64, true residual) */
} mf_solve_info;

typedef struct {
  int64_t n;              /* N                                                        */
  int64_t nfronts;        /* fronts in the assembly tree                              */
  int64_t ncompressed;    /* fronts factored in HOD-BF form                           */
  int32_t tree_levels;    /* depth of the assembly tree + 1                           */
  int32_t max_rank;       /* largest ID rank met in the factorization                 */
  double factor_flops;    /* real floating-point operations of the numeric factorization */
  double factor_bytes;    /* device bytes holding the factors                          */
  double factor_seconds;  /* wall time of the last mf_factor                           */
  int32_t precision;      /* MF_PREC_*                                                 */
  int32_t gpu_launches_factor;  /* kernel launches of one factorization                */
  int32_t gpu_launches_solve;   /* kernel launches of one preconditioner application   */
  int32_t reserved;
  double arena_peak_bytes;      /* compressed fronts: peak use of the device arenas (factors + work) */
  double arena_capacity_bytes;  /* compressed fronts: device memory reserved for those arenas      */
} mf_stats_t;

typedef struct mf_handle mf_handle;

/* Fill *opt with the defaults.  Returns MF_OK or MF_ERR_ARG (opt == NULL). */
int mf_options_init(mf_options* opt);

/*
 * Symbolic analysis (the ordering and symbolic steps of Alg. 1 and Alg. 5; Sec. 2, 5.1, 5.2).
 *   n, rowptr[n+1] (int64), colind[nnz] (int32, 0-based), vals[2*nnz] (re, im):
 *     the CSR matrix A; the pattern must be structurally symmetric.
 *   opt->coords (N x 3 int32, optional): lattice coordinates of the unknowns.
 *     MF_LATTICE_NODE: grid indices (separator planes are layers of unknowns);
 *     MF_LATTICE_EDGE: doubled coordinates of a Yee edge lattice (an edge at
 *     (i+1/2, j, k) is (2i+1, 2j, 2k)); separators are node planes.
 *     NULL: general CSR input, ordered by graph nested dissection (breadth-first
 *     level structures from a pseudo-peripheral vertex; separator = the level
 *     where half of the reached vertices are passed; a compressed separator's
 *     HOD-BF tree comes from recursive bisection of its two-hop graph).
 *   cuda_stream: the CUDA stream all device work of this handle runs on (NULL = default).
 * Computes the nested-dissection ordering (planar, hybrid or graph: opt->ordering), the assembly tree, the
 * update sets, the HOD-BF cluster trees and the neighbour lists on the host;
 * no device memory is touched until mf_factor.  *out receives a new handle.
 * Errors: MF_ERR_ARG (bad pointers/sizes/CSR, an unknown ordering, MF_ORDER_HYBRID without
 * coords), MF_ERR_UNSUPPORTED (a box with
 * an empty separator), MF_ERR_OOM.
 */
int mf_analyze(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* vals,
               const mf_options* opt, void* cuda_stream, mf_handle** out);

/*
 * Numeric factorization on the GPU (Alg. 1 for fronts with |I^s| < nmin_sep,
 * Alg. 5 otherwise).  tol is the ID tolerance epsilon of the butterfly
 * constructions (Sec. 6.1); it is ignored by dense fronts.  May be called
 * again (refactorization with the same pattern).  Blocks until done.
 * Errors: MF_ERR_STATE (no analysis), MF_ERR_SINGULAR, MF_ERR_OOM, MF_ERR_CUDA.
 */
int mf_factor(mf_handle* h, double tol);

/*
 * Solve A X = B for nrhs columns with host buffers (b: N x nrhs, ldb; x: N x
 * nrhs, ldx; x may equal b).  The copies to and from the device are part of
 * the call.  Uses the refinement of opt->refine.  info may be NULL.
 * Errors: MF_ERR_STATE (not factored), MF_ERR_ARG, MF_ERR_NO_CONVERGENCE
 * (x and info written), MF_ERR_CUDA.
 */
int mf_solve(mf_handle* h, int32_t nrhs, const double* b, int64_t ldb, double* x, int64_t ldx,
             mf_solve_info* info);

/* Same as mf_solve with device buffers (interleaved complex128, column-major, ld = N). */
int mf_solve_device(mf_handle* h, int32_t nrhs, const void* d_b, void* d_x, mf_solve_info* info);

/*
 * Per-column results of the last mf_solve / mf_solve_device on h (Sec. 6: every
 * right-hand side runs its own Krylov iteration, so each column has its own
 * count and residual, independent of the other columns solved with it).
 * nrhs must equal the last solve's; any output pointer may be NULL:
 *   iters[c]        Krylov iterations (or refinement steps) of column c
 *   converged[c]    1 if column c met rtol
 *   rel_residual[c] ||b_c - A x_c|| / ||b_c|| (FP64, true residual)
 * Errors: MF_ERR_ARG (h NULL, nrhs mismatch), MF_ERR_STATE (no solve yet).
 */
int mf_solve_columns(const mf_handle* h, int32_t nrhs, int32_t* iters, int32_t* converged, double* rel_residual);

/* Counters of the analysis and of the last factorization. */
int mf_stats(const mf_handle* h, mf_stats_t* out);

/* Message of the last failure on h (h == NULL: of the calling thread). Never NULL. */
const char* mf_last_error(const mf_handle* h);

/* CUDA-event timing of two kernel families, for roofline figures (sampled).
 * mf_profile(h, N) with N > 0 enables it and clears the counters (0 disables it);
 * while it is on, one launch in N of each family gets a start and a stop event on
 * the stream it runs on, and one replay in N of each solve graph runs a copy of
 * the graph with those events as graph nodes (N = 1: every launch):
 *   MF_PROF_NARROW_GEMM: the narrow GEMM (n <= 128: the solve's front products
 *     with the right-hand sides and the butterfly level products) in mf_factor
 *     and mf_solve*;
 *   MF_PROF_FRONT_GEMM: the dense fronts' Schur-update GEMMs in mf_factor.
 * mf_profile_read returns for one family the timed launches, their summed device
 * time, algorithmic flops (8 m n k per complex product) and algorithmic bytes
 * (A and B read once, C written, and read when beta != 0; planar complex). */
enum { MF_PROF_NARROW_GEMM = 0, MF_PROF_FRONT_GEMM = 1 };
typedef struct {
  int64_t launches;
  double ms;
  double flops;
  double bytes;
} mf_kernel_profile_t;
int mf_profile(mf_handle* h, int32_t enable);
int mf_profile_read(mf_handle* h, int32_t kernel, mf_kernel_profile_t* out);

/*
 * Component entry point of the front-update GEMM kernels (the Schur update
 * C = F22 - F21 F12 of Sec. 2 step 4 and the triangular products before it).
 * One planar complex64 product on device memory:
 *   C = alpha * A * B^T + beta * C,  A: m x k, B: n x k, C: m x n, all row-major,
 *   each matrix given by its real plane (device pointer), leading dimension ld and
 *   the element offset pl of its imaginary plane (im = re + pl).
 * engine 0: SIMT FP32 kernel; engine 1: tcgen05 kind::tf32 tensor-core kernel, one
 * TF32 pass; engine 2: the same kernel in split precision (three TF32 passes,
 * hi*hi + hi*lo + lo*hi), the form used by mf_factor.  Engines 1 and 2 require
 * lda, ldb, pla, plb multiples of 4 and 16-byte aligned planes.
 * Runs on `stream` and waits for it.  Errors: MF_ERR_ARG, MF_ERR_TIMEOUT, MF_ERR_CUDA.
 */
int mf_gemm_c64(int32_t engine, int32_t m, int32_t n, int32_t k, const float* A, int64_t lda, int64_t pla,
                const float* B, int64_t ldb, int64_t plb, float* C, int64_t ldc, int64_t plc, float alpha, float beta,
                void* stream);

/*
 * Component entry point of the narrow GEMM kernel of the solve (Alg. 1, last line:
 * the front products with the block of right-hand sides) and of the butterfly level
 * products with blocks of vectors (Sec. 3).  One planar complex64 product on device
 * memory:
 *   C = alpha * op(A) * B + beta * C,  op(A) = A (trans_a = 0, A: m x k) or A^T
 *   (trans_a = 1, A stored k x m), B: k x n, C: m x n, all row-major, n <= 128,
 *   each matrix given by its real plane, leading dimension and imaginary-plane offset.
 * ksplit: number of CTAs of a thread-block cluster sharing one 32-row tile's K range
 * (1, 2, 4 or 8), 0 = the library's choice, or -1 for the tensor-core kernel (n <= 64:
 * tcgen05 kind::tf32, three split-precision passes; the kernel the library uses for
 * complex64 butterfly level products with at most 64 vectors).  No alignment requirements.
 * Runs on `stream` and waits for it.  Errors: MF_ERR_ARG, MF_ERR_TIMEOUT (a bounded wait of
 * the tensor-core kernel expired), MF_ERR_CUDA.
 */
int mf_gemm_nrhs_c64(int32_t trans_a, int32_t m, int32_t n, int32_t k, const float* A, int64_t lda, int64_t pla,
                     const float* B, int64_t ldb, int64_t plb, float* C, int64_t ldc, int64_t plc, float alpha,
                     float beta, int32_t ksplit, void* stream);

/*
 * Component entry point of the batched row interpolative decomposition (Sec. 3):
 * for each of nmat complex64 matrices M_q (m x n), a column-pivoted Householder
 * QR of M_q^T truncated at the first k with |R_{k+1,k+1}| <= tol |R_11| (at most
 * kmax = min(m, n, max_rank > 0 ? max_rank : n) steps) gives the skeleton rows
 * I_q (|I_q| = rank_q) and U_q with M_q ~= U_q M_q(I_q, :) and U_q(I_q, :) = I.
 * Device buffers:
 *   M     nmat matrices back to back, each a real m x n row-major plane followed by
 *         its imaginary plane (2 m n floats per matrix); not modified
 *   U     out, nmat blocks of 2 m kmax floats (real then imaginary m x kmax row-major;
 *         columns >= rank_q are unspecified)
 *   sk    out, nmat x kmax int32 (first rank_q entries valid), rank out, nmat int32.
 * Matrices with m, n <= 128 keep their rows in registers (1024 threads each); otherwise
 * the QR work matrix (2 m n floats per matrix) lives in shared memory when it fits
 * (2 m n + 2 n + 2 m floats <= 200 KiB), else in scratch allocated by the call, each such
 * matrix shared by a cluster of 8 thread blocks (same results as one block per matrix).
 * Runs on `stream` and waits for it.  Errors: MF_ERR_ARG (sizes: n <= 8192, m <= 2048),
 * MF_ERR_OOM, MF_ERR_CUDA.
 */
int mf_row_id_c64(int32_t nmat, int32_t m, int32_t n, const float* M, double tol, int32_t max_rank, float* U,
                  int32_t* sk, int32_t* rank, void* stream);

/*
 * mf_row_id_c64 without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory where
 * they need the decomposition -- applications whose own pool allocator reserves
 * the GPU's memory up front and owns every buffer (a library cudaMalloc would
 * fail or take memory the pool counts on), and latency-sensitive loops that may
 * not call cudaMalloc / cudaFree, which can synchronize the whole device and
 * stall other streams.  Same arguments, layouts and results as
 * mf_row_id_c64; the QR work matrix lives in a fixed array inside the library
 * (8 MiB per GPU, held by every GPU that loads the library until the process
 * exits) instead of a per-call allocation.
 *  - Limit: 2 * m * n * nmat <= 2^21 floats (e.g. 16 matrices of 128 x 512);
 *    larger batches return MF_ERR_ARG and do nothing.
 *  - The first call on a device looks up the array's device address (with that
 *    device current) and sets the kernel's shared-memory limit; make that first
 *    call before any stream capture.
 *  - All calls share the one array and the work matrix is fully rewritten by
 *    every call, so calls that overlap on the GPU (different streams or
 *    threads without ordering) race and give wrong results.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine.  Waits for `stream`.
 * Errors: MF_ERR_ARG, MF_ERR_CUDA.
 */
int mf_row_id_c64_noalloc(int32_t nmat, int32_t m, int32_t n, const float* M, double tol, int32_t max_rank,
                          float* U, int32_t* sk, int32_t* rank, void* stream);

/* ---------------- serving: continuous batching over resident factorizations ---------------- */

/*
 * A solve server over nproblems resident factorizations (handles already
 * factored; each should have its own CUDA stream).  One worker thread per
 * handle batches every request waiting for that handle when its previous batch
 * ends (requests that arrive during a solve join the next batch), admits
 * requests (up to max_batch_rhs columns; a wider request runs alone, in slices of
 * max_batch_rhs columns) while the batch's device workspace, estimated as 40 * N * nrhs * 16
 * bytes, fits together with the other batches in flight both mf_server_create's
 * mem_budget_bytes and the device's free memory less 1 GiB (cudaMemGetInfo, read
 * when the batch is formed), and runs the batch as one mf_solve.  Each request
 * reports its own columns (mf_solve_columns): its status, iterations, converged
 * flag and residual are those it would get if solved alone.  The handles must
 * be on the device that is current at mf_server_create; they stay owned by the
 * caller and must not be used elsewhere while the server lives.
 */
typedef struct mf_server mf_server;
typedef struct {
  int64_t id;
  int32_t problem, nrhs;
  int32_t iters, converged;  /* max over the request's columns; 1 if all its columns met rtol */
  int32_t batch_rhs;          /* right-hand sides of the batch the request ran in */
  int32_t reserved;
  double max_rel_residual;    /* max over the request's columns */
  double t_arrival, t_start, t_done;   /* seconds since the server was created */
} mf_request_info;

int mf_server_create(int32_t nproblems, mf_handle* const* handles, int32_t max_batch_rhs, int64_t mem_budget_bytes,
                     mf_server** out);
/* Queue nrhs right-hand sides b (host, N x nrhs column-major, interleaved) for problem `problem`;
 * x (host, same shape) is written when the request completes; *id identifies it.  b and x must
 * stay valid until mf_server_wait returns.  MF_ERR_OOM if the request alone exceeds the budget. */
int mf_server_submit(mf_server* s, int32_t problem, int32_t nrhs, const double* b, double* x, int64_t* id);
/* Block until request id is done and fill *info.  Returns MF_OK if every column of the request
 * met rtol, MF_ERR_NO_CONVERGENCE if one did not (x still written), or the batch's mf_solve
 * error (MF_ERR_CUDA, ...). */
int mf_server_wait(mf_server* s, int64_t id, mf_request_info* info);
/* Finish queued requests and stop the workers. */
void mf_server_destroy(mf_server* s);

/* ---------------- butterfly component: Green's-function block sets ---------------- */

/*
 * HOD-BF compression of nblk blocks of the 3-D Helmholtz Green's function
 * G(x, y) = exp(i k |x - y|) / (4 pi |x - y|) (Sec. 3.1) between two parallel
 * m_b x m_b point grids of spacing h, at z = 0 and z = h.  Each block is an
 * m_b^2 x m_b^2 HOD-BF matrix (Sec. 4) over a uniform-depth geometric bisection
 * of the plane with leaves of at most `leaf` points; its off-diagonal blocks
 * are butterflies built by entry evaluation (Alg. 2, ID tolerance tol, rank cap
 * max_rank (0 = none), alpha uniform + knn nearest proxies), complex64, on the
 * GPU.  Rows of block b occupy [off_b, off_b + m_b^2) of the set, points in the
 * set's order (see mf_green_points).  *out receives the set (owns its memory).
 */
typedef struct mf_bfset mf_bfset;
int mf_green_build(int32_t nblk, const int32_t* m, double k, double h, double tol, int32_t leaf, int32_t max_rank,
                   int32_t alpha, int32_t knn, void* stream, mf_bfset** out);
/* rows of the set, stored complex entries, largest ID rank, build wall time */
int mf_green_info(const mf_bfset* s, int64_t* rows, double* storage_entries, int32_t* max_rank,
                  double* build_seconds);
/* Work of one mf_green_apply with nrhs vectors (after a first call with that nrhs): real flops
 * (8 m n k per complex block product) and the bytes its block products move when each level's
 * vectors go through device memory (factor blocks + input + output vectors of every product);
 * MF_ERR_STATE before the first call. */
int mf_green_apply_counts(const mf_bfset* s, int32_t nrhs, double* flops, double* bytes);
/* host copies of the source (z = 0) and target (z = h) points, rows x 3 each, in the set's row order */
int mf_green_points(const mf_bfset* s, double* P, double* Q);
/*
 * y_b = H_b x_b for every block (the butterfly apply of Sec. 3.1, level by level).
 * x, y: device, planar complex64 rows x nrhs row-major (real plane, then the
 * imaginary plane at offset rows * nrhs).  Waits for the set's stream.  The launch
 * sequence for one (nrhs, x, y) runs eagerly on its first call, is captured into a
 * CUDA graph on the second and replayed by later calls (x and y must stay allocated
 * while the set uses them).
 */
int mf_green_apply(mf_bfset* s, int32_t nrhs, const float* x, float* y);
void mf_green_destroy(mf_bfset* s);

/* Kernel launches issued by the library since it was loaded (all handles, all streams). */
int64_t mf_launch_counter(void);

/* Frees everything owned by h (NULL is ignored). */
void mf_destroy(mf_handle* h);

/* ---------------- inspection of the analysis (host only, no GPU needed) ---------------- */

typedef struct {
  int64_t n;
  int64_t nfronts;
  int64_t upd_total;      /* sum of |I^u| over fronts */
  int64_t tree_total;     /* sum over compressed fronts of the ranges of both cluster trees */
  int64_t nn_total;       /* sum over compressed fronts of the lengths of the four neighbour lists */
} mf_analysis_sizes_t;

int mf_analysis_sizes(const mf_handle* h, mf_analysis_sizes_t* out);

/*
 * Copies the analysis into caller buffers (sizes from mf_analysis_sizes):
 *   perm[n]                 perm[new] = old
 *   front_parent[nfronts]   parent front id (-1 for the root), fronts in post-order
 *   front_sep[2*nfronts]    [sep_begin, sep_end) in the new numbering
 *   front_flags[nfronts]    bit 0: compressed
 *   upd_ptr[nfronts+1], upd_idx[upd_total]   I^u of every front (sorted new indices)
 * Any pointer may be NULL to skip that array.
 */
int mf_analysis_export(const mf_handle* h, int64_t* perm, int64_t* front_parent, int64_t* front_sep,
                       int32_t* front_flags, int64_t* upd_ptr, int64_t* upd_idx);

/*
 * Failure detection of the tensor-core kernels: every mbarrier wait in them polls at most
 * `spins` times (0 restores the default, 2^26) before the kernel records an expired wait, stops
 * issuing work, waits for its committed MMAs (always with the default limit), frees its tensor
 * memory and returns; the call that launched it then returns MF_ERR_TIMEOUT and the CUDA context
 * stays usable.  Process-wide; meant for tests of that path.  Errors: MF_ERR_ARG (spins < 0).
 */
int mf_set_wait_limit(int64_t spins);

/*
 * Apply one operator of compressed front f (Alg. 5) to nrhs host vectors, for inspection
 * (for example the per-front compression error against a dense assembly of the same block):
 *   which = MF_OP_F11 (0): the HOD-BF F11 (Sec. 4.1), s x s
 *           MF_OP_F11_INV (1): its Alg. 4 inverse, s x s
 *           MF_OP_F12 (2): the butterfly F12 (Alg. 2), s x u
 *           MF_OP_F21 (3): the butterfly F21, u x s
 *           MF_OP_C (4): the HOD-BF contribution block C = F22 - F21 F11^-1 F12 (kept for the
 *                        parent; absent at the root), u x u
 * s = |I^s|, u = |I^u| of front f; rows and columns in the new numbering's order of
 * [sep_begin, sep_end) and of I^u (see mf_analysis_export).  x: in x nrhs, y: out x nrhs,
 * host, column-major, interleaved complex128.  Synchronous; allocates device staging.
 * Errors: MF_ERR_ARG (not a compressed front, no such operator), MF_ERR_STATE (not factored).
 */
#define MF_OP_F11 0
#define MF_OP_F11_INV 1
#define MF_OP_F12 2
#define MF_OP_F21 3
#define MF_OP_C 4
int mf_front_apply(mf_handle* h, int64_t f, int32_t which, int32_t nrhs, const double* x, double* y);

/*
 * Cluster trees of front f (Sec. 5.1).  nlev[0], nlev[1] receive the number of
 * levels (depth + 1) of the HOD-BF tree T_H of F11 and of the F22 tree (0 for a
 * dense front).  If ranges != NULL it receives, for T_H then the F22 tree,
 * level by level, the 2^l ranges (a, b) of level l as int64 pairs; its length
 * is 2 * (2^nlev[0] - 1) + 2 * (2^nlev[1] - 1) values.
 */
int mf_front_trees(const mf_handle* h, int64_t f, int64_t* nlev, int64_t* ranges);

/*
 * Graph nearest-neighbour lists of front f (Sec. 5.2) with knn neighbours:
 * nn11 (rows I^s, within the graph of A(I^s,I^s), outside the row's T_H leaf),
 * nn22 (rows I^u, graph A(I^u,I^u), outside the row's F22 leaf),
 * nn12 (rows I^s, nearest vertices of I^u) and nn21 (rows I^u, nearest of I^s),
 * breadth-first, level by level, increasing vertex order within a level.
 * counts[4] receives the total entries of each list.  If ptr != NULL it receives
 * the four CSR row-pointer arrays back to back (lengths s+1, u+1, s+1, u+1) and
 * idx the entries (new indices) back to back.
 */
int mf_front_neighbours(const mf_handle* h, int64_t f, int32_t knn, int64_t* counts, int64_t* ptr, int64_t* idx);

#ifdef __cplusplus
}
#endif

#endif /* MF_H_ */
