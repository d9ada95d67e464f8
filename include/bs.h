/*
 * bs.h -- C ABI of libbs: the Benchmark Streaming operations (BS1-BS7) and
 * the conjugate-gradient solve of Chalmers & Warburton, "Portable high-order
 * finite element kernels I: Streaming Operations" (arXiv 2009.10917), built
 * for NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Vectors are caller-owned DEVICE pointers on the current CUDA device,
 *    contiguous, element i at ptr[i].  FP64 unless the name ends in _f32.
 *    16-byte alignment enables the 128-bit path; other alignments are
 *    accepted and take a scalar path.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *    call is asynchronous on that stream unless stated otherwise; results
 *    written to device scalars are valid once the stream reaches them.
 *  - Opaque objects (bs_workspace, bs_map, bs_problem) are owned by the
 *    library, created on the current device and freed by *_destroy.  Host
 *    arrays passed to *_create are copied; the caller keeps ownership.
 *  - One bs_workspace may serve one stream at a time: reductions that share
 *    a workspace must not overlap on the GPU.
 *  - Every function returns a bs_status.  No C++ exception crosses the ABI.
 *    bs_last_error() gives a thread-local description of the last failure.
 *    Arguments are validated before any launch; on BS_ERR_ARG nothing was
 *    enqueued.
 *  - Sizes are int64_t counts of elements; n == 0 is valid and enqueues
 *    nothing except the zero results of reductions.
 */
#ifndef BS_H_
#define BS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */

typedef enum {
  BS_OK = 0,
  BS_ERR_ARG = 1,            /* invalid argument; nothing enqueued          */
  BS_ERR_CUDA = 2,           /* a CUDA runtime call failed                  */
  BS_ERR_TIMEOUT = 3,        /* a bounded device-side wait ran out          */
  BS_ERR_BREAKDOWN = 4,      /* CG breakdown: p.Ap <= 0 or not finite       */
  BS_ERR_NOT_CONVERGED = 5,  /* iteration limit reached before tolerance    */
  BS_ERR_DEVICE_CHECK = 6,   /* a device-side validity check failed         */
  BS_ERR_ALLOC = 7           /* device or host allocation failed            */
} bs_status;

/* Static description of a status code. */
const char *bs_error_string(int status);
/* Thread-local detail of the most recent failing call on this thread. */
const char *bs_last_error(void);
/* Library version as 10000*major + 100*minor + patch. */
int bs_version(void);

/* Checked build (the library compiled with -DBS_CHECK=1; no counterpart in
 * the paper: a stand-in for a memory checker).  Every kernel then tests each
 * index it reads from memory -- map entries against N_G, CSR row bounds and
 * columns against nnz and N_L, gather tiles, the pipelined gather's chunk
 * ids and staged offsets, the batched solver's items -- before using it; a
 * failing test records a code (BS_CHK_* in the library's csrc/bs_check_pred.h)
 * and skips the access (a load reads 0, a store is dropped), so results are
 * then meaningless but no memory outside the buffers is touched.
 * bs_check_enabled: 1 in a checked build, 0 otherwise.
 * bs_check_device: synchronises the current device, collects and clears the
 * recorded codes; BS_OK when none was recorded (always, in the default
 * build), BS_ERR_DEVICE_CHECK naming the first code otherwise, BS_ERR_CUDA
 * when the device cannot be read.  Call it between library calls, not while
 * another thread is inside one. */
int bs_check_enabled(void);
int bs_check_device(void);

/* ------------------------------------------------------------ workspace */

/* Scratch for single-launch reductions: per-block partial sums, an arrival
 * counter and result slots (a few KB of device memory, cudaMalloc'd on the
 * current device).  The counter is left at zero after every reduction. */
typedef struct bs_workspace bs_workspace;
int bs_workspace_create(bs_workspace **ws);
int bs_workspace_destroy(bs_workspace *ws);

/* ------------------------------------------------------------ BS1-BS5 */

/* BS1, vector copy (Table 1; Listing 1): y[i] = x[i], i < n.  Bitwise. */
int bs_copy(int64_t n, const double *x, double *y, void *stream);

/* BS2, vector AXPY (Table 1; Listing 2): y[i] = fma(alpha, x[i], beta*y[i]),
 * i.e. alpha*x + beta*y with the product beta*y rounded on its own and one
 * fused multiply-add.  Bitwise reproducible; x and y must not overlap. */
int bs_axpy(int64_t n, double alpha, const double *x, double beta, double *y,
            void *stream);

/* BS3, vector norm (Table 1; Listing 3): d_out[0] = x.x, d_out[1] =
 * sqrt(x.x), written to DEVICE memory (2 doubles) in one launch.  The
 * summation order is fixed by n and the device, so repeated calls are
 * bitwise identical. */
int bs_norm(int64_t n, const double *x, double *d_out, bs_workspace *ws,
            void *stream);

/* BS4, inner product (Table 1): d_out[0] = x.y (DEVICE, 1 double), one
 * launch, deterministic as bs_norm. */
int bs_dot(int64_t n, const double *x, const double *y, double *d_out,
           bs_workspace *ws, void *stream);

/* BS5, fused CG update (Table 1; Algorithm 1 steps 8-10 fused):
 *   x[i] = fma(alpha, p[i], x[i]);  r[i] = fma(-alpha, Ap[i], r[i]);
 *   d_rr[0] = sum of the updated r[i]^2   (DEVICE, 1 double)
 * in one pass: x and r are read and written once, p and Ap read once. */
int bs_cg_update(int64_t n, double alpha, const double *p, const double *Ap,
                 double *x, double *r, double *d_rr, bs_workspace *ws,
                 void *stream);

/* FP32-storage twins (vectors of float).  Products and sums inside the
 * reductions are carried as unevaluated pairs of floats (about 44 bits);
 * the per-block partials are combined in double, and results are doubles. */
int bs_copy_f32(int64_t n, const float *x, float *y, void *stream);
int bs_axpy_f32(int64_t n, float alpha, const float *x, float beta, float *y,
                void *stream);
int bs_norm_f32(int64_t n, const float *x, double *d_out, bs_workspace *ws,
                void *stream);
int bs_dot_f32(int64_t n, const float *x, const float *y, double *d_out,
               bs_workspace *ws, void *stream);
int bs_cg_update_f32(int64_t n, float alpha, const float *p, const float *Ap,
                     float *x, float *r, double *d_rr, bs_workspace *ws,
                     void *stream);

/* ------------------------------------------------------------ BS6, BS7 */

/* The scatter operator Z (eq. scatter_def): an N_L x N_G Boolean matrix with
 * one unit entry per row, given by the int32 local-to-global map
 * h_l2g[l], l < N_L = E*(N+1)^3 (Sec. 5: "scatterIds").  h_l2g[l] < 0 masks
 * local node l (Sec. 5: boundary conditions).  Every h_l2g[l] must be < NG.
 * bs_map_create copies the map to the device and builds the CSR form of Z^T
 * (Sec. 5, Listing 4): rowStarts[NG+1] and colIds[nnz], the local indices of
 * each global node in ascending order, and the gather's per-tile re-encoding
 * of it (the distinct chunks of two q_L values each tile reads, uint16
 * offsets, row starts and summing order: about 4 more bytes of device memory
 * per local node and 4 per global node).  Host-side, synchronous. */
typedef struct bs_map bs_map;
int bs_map_create(int32_t E, int32_t N, int64_t NG, const int32_t *h_l2g,
                  bs_map **map);
int bs_map_destroy(bs_map *map);
/* N_L, N_G and the number of unmasked local nodes (nnz of Z). */
int bs_map_info(const bs_map *map, int64_t *NL, int64_t *NG, int64_t *nnz);
/* Copy the CSR of Z^T back to host arrays rowStarts[NG+1], colIds[nnz]
 * (synchronous; for verification). */
int bs_map_export(const bs_map *map, int32_t *h_row_starts, int32_t *h_col_ids);
/* Device valence diag(Z^T Z) into d_val[NG] (int32). */
int bs_map_valence(const bs_map *map, int32_t *d_val, void *stream);

/* BS7, scatter q_L = Z q_G (Table 1; Listing 5): qL[l] = qG[l2g[l]] for
 * l2g[l] >= 0; masked entries of qL are left untouched.  Bitwise. */
int bs_scatter(const bs_map *map, const double *qG, double *qL, void *stream);

/* BS6, gather q_G = Z^T q_L (Table 1; Listing 4): qG[g] = sum of qL[l] over
 * the local copies l of g, accumulated from +0.0 in ascending l (no atomics,
 * bitwise reproducible).  A global node with no copies gets 0. */
int bs_gather(const bs_map *map, const double *qL, double *qG, void *stream);

int bs_scatter_f32(const bs_map *map, const float *qG, float *qL, void *stream);
int bs_gather_f32(const bs_map *map, const float *qL, float *qG, void *stream);

/* ------------------------------------------------------------ BS6 over several ranks */

/* The device steps of a gather whose elements are split over ranks (Sec. 3
 * leaves the multi-rank gather/scatter aside as the non-trivial parallel
 * implementation; the exchange plan and the messages are host-side, in the
 * Python package's dist module).  Each rank owns a contiguous range of the
 * element storage order and a bs_map of its elements onto the global nodes
 * they touch (numbered rank-locally).  A node held by several ranks is summed
 * as a chain in rank order: the first holder's ordinary bs_gather, then each
 * later holder continues the serial sum from the partial it receives
 * (bs_gather_rows with `start`), so the last holder gets bitwise the
 * single-domain BS6 value (ascending local index), and sends it back.
 *
 * bs_rows: a set of `nrows` distinct rows (rank-local global-node indices in
 * [0, NG)) of a map's Z^T, in the order of a message.  Host array copied;
 * the map must outlive the row set.  Errors: BS_ERR_ARG (NULL, out of range,
 * repeated row), BS_ERR_CUDA. */
typedef struct bs_rows bs_rows;
int bs_rows_create(const bs_map *map, int64_t nrows, const int32_t *h_rows,
                   bs_rows **out);
int bs_rows_destroy(bs_rows *rows);
/* For i < nrows, g = rows[i]: qG[g] = start[i] + qL[l_1] + qL[l_2] + ...
 * over g's local copies in ascending l, added one at a time; with start ==
 * NULL the sum begins from +0.0 exactly as bs_gather does.  Other entries of
 * qG are untouched.  start (DEVICE, nrows doubles) may be NULL. */
int bs_gather_rows(const bs_rows *rows, const double *qL, const double *start,
                   double *qG, void *stream);
/* buf[i] = qG[rows[i]] (pack) and qG[rows[i]] = buf[i] (unpack); buf is a
 * DEVICE array of nrows doubles.  Bitwise moves. */
int bs_rows_pack(const bs_rows *rows, const double *qG, double *buf, void *stream);
int bs_rows_unpack(const bs_rows *rows, const double *buf, double *qG, void *stream);

/* ------------------------------------------------------------ operator */

/* The Helmholtz operator A = Z^T (S_L + lambda M_L) Z of eqs. global_system,
 * assembled_stiff and assembled_mass, discretised with degree-N GLL
 * Lagrange bases on affine cube elements of side h (Sec. 2, eq. basis),
 * collocated GLL quadrature (lumped mass):
 *   (A_e u)_ijk = c_e (h/2) [ (K x W x W) + (W x K x W) + (W x W x K) ] u
 *               + lambda (h/2)^3 w_i w_j w_k u_ijk,   K = D^T W D,
 * with c_e = h_coef[e] (or 1 when h_coef is NULL).  Local node (i,j,k) of
 * element e is l = e*(N+1)^3 + i + (N+1)(j + (N+1)k).  The problem keeps a
 * reference to `map` (which must outlive it) and owns its device scratch
 * (two N_L and six N_G vectors).  Host-side, synchronous. */
typedef struct bs_problem bs_problem;
int bs_problem_create(const bs_map *map, double h, double lambda,
                      const double *h_coef, bs_problem **prob);
int bs_problem_destroy(bs_problem *prob);

/* The same operator on general hexahedra (the non-affine geometric factors
 * Sec. 5 allows for): element e is the trilinear image of [-1,1]^3 with
 * corner v = vx + 2 (vy + 2 vz) (vx, vy, vz in {0,1}; vertex v sits at
 * reference point (2vx-1, 2vy-1, 2vz-1)) at h_verts[24 e + 3 v + d],
 * d = x, y, z (HOST, copied; E*24 doubles).  With J = dx/dr at each GLL node,
 *   (A_e u)_n = c_e sum_q grad_r l_n(q)^T G_q grad_r u(q) + lambda M_n u_n,
 *   G_q = w_q det J J^-1 J^-T,  M_n = w_n det J,
 * G and M are computed here in FP64 and kept on the device (7 doubles per
 * local node).  N <= 11.  BS_ERR_ARG if some element has det J <= 0 at a
 * node.  Such a problem serves bs_apply_A, bs_apply_local, bs_diag_A,
 * bs_apply_A_ff and bs_cg_solve (FP64 or float-float element kernel, the
 * latter splitting the factors into float pairs on the fly; Jacobi, graphs,
 * scattered storage); the FP32 refined, batched and learned solvers return
 * BS_ERR_ARG for it. */
int bs_problem_create_geo(const bs_map *map, double lambda, const double *h_coef,
                          const double *h_verts, bs_problem **prob);

/* Ap = A p (N_G vectors). */
int bs_apply_A(const bs_problem *prob, const double *p, double *Ap,
               void *stream);
/* Element-local A_L uL (N_L vectors; no Z, no Z^T). */
int bs_apply_local(const bs_problem *prob, const double *uL, double *AuL,
                   void *stream);
/* diag(A) = Z^T diag(A_L) into d_diag[NG]. */
int bs_diag_A(const bs_problem *prob, double *d_diag, void *stream);

/* bs_apply_A with the element operator in float-float arithmetic (no
 * counterpart in the paper): GB300 executes FP64 at about 1/64 of its FP32
 * rate, so each input is split exactly into a pair of floats by integer
 * operations, the contractions accumulate error-free products of the high
 * parts with TwoSum on the FP32 pipes, and only the final combination of a
 * node is FP64.  Error per node: a few units of 2^-46 times sum |K| |u|
 * (about 64 times the FP64 operator's); inputs below 2^-102 in magnitude
 * count as zero (scale b so that the entries that matter lie above that)
 * and inputs of 2^127 or more become infinite.  On a problem with geometric
 * factors the six entries of w det J J^-1 J^-T and lambda w det J are split
 * the same way, so the same window applies to them: they scale as L and
 * lambda L^3 with the mesh's length scale L, and below 2^-102 they count as
 * zero -- keep L above about 2^-28 (lambda of order 1) for the accuracy
 * stated here.  The gather is the same as bs_apply_A's. */
int bs_apply_A_ff(const bs_problem *prob, const double *p, double *Ap, void *stream);

/* How A p is formed, process-wide, by bs_apply_A, bs_apply_local,
 * bs_apply_A_ff and every solver (the batched one reads BS_OP_DIRECT when a
 * batch is set up, and never fuses); mode is a set of bits
 * (0, the default, is the fastest measured form):
 *  BS_OP_FUSED: a global node with a single local copy (an element
 *   interior, a face on the natural boundary) needs no gather, so the
 *   element kernel writes its value into Ap itself and adds its term of p.Ap
 *   in the same pass; only nodes with several copies go through the N_L
 *   buffer and a gather over their rows alone.  Without it the element
 *   kernel writes every local value and the gather (BS6) sums every row.  Ap
 *   is bitwise the same either way (a one-copy row sums to +0 + v); p.Ap
 *   differs only by summation order.  Measured slower on GB300
 *   (partial-sector writes into Ap; N = 7 on 48^3: 1.37 vs 1.24 ms per
 *   float-float A p).
 *  BS_OP_DIRECT: the element kernels (FP64, FP32, float-float) contract
 *   with the full 1-D stiffness K = D^T W D (3 (N+1) multiply-adds per
 *   node).  Without it, for odd N <= 9, they use the even-odd form of the
 *   centrosymmetric W^-1 K (Solomonoff's decomposition; half-length
 *   contractions, about a quarter fewer operations per node); results
 *   differ by rounding only.
 * Problems with geometric factors (bs_problem_create_geo) always use their
 * own unfused FP64 kernel.  Returns the previous mode; a negative value only
 * queries it.  Not thread-safe against solves in flight. */
enum { BS_OP_FUSED = 1, BS_OP_DIRECT = 2 };
int bs_operator_mode(int32_t mode);

/* ------------------------------------------------------------ CG */

enum {
  BS_CG_FIXED_ITERS = 1, /* run exactly maxit iterations                   */
  BS_CG_JACOBI = 2,      /* Jacobi preconditioner z = diag(A)^-1 r         */
  BS_CG_GRAPH = 4,       /* replay the iteration as a captured CUDA graph  */
  BS_CG_X0 = 8,          /* x holds the initial guess (else x0 = 0)        */
  BS_CG_REFINED_F32 = 32, /* batched: FP32 inner CG, FP64 refinement       */
  BS_CG_FF_OPERATOR = 256, /* the float-float operator of bs_apply_A_ff     */
  BS_CG_SCATTERED = 512,    /* bs_cg_solve: vectors in scattered storage    */
  BS_CG_BLOCK_JACOBI = 1024 /* bs_cg_solve: element-interior block Jacobi   */
};

typedef struct {
  int32_t iterations;   /* CG iterations performed                        */
  int32_t status;       /* bs_status of the solve                         */
  int32_t outer;        /* refinement steps (bs_cg_solve_refined_f32)     */
  int32_t fallbacks;    /* learned FPCG: corrections replaced by Jacobi   */
  double rr;            /* final r.r (recursive residual)                 */
  double bb;            /* b.b                                            */
  double rel_residual;  /* sqrt(rr / bb); FP64 true residual when refined */
  double seconds;       /* wall time of the solve on the host             */
} bs_cg_info;

/* Algorithm 1 on A x = b (N_G vectors b, x).  Stops when r.r <= tol^2 b.b or
 * after maxit iterations; the convergence flag is computed on the device and
 * read back every few iterations.  d_hist (DEVICE, may be NULL) receives
 * 3*(maxit+1) doubles: alpha_j at [3j], beta_j at [3j+1], r_{j+1}.r_{j+1} at
 * [3j+2].  flags: BS_CG_FIXED_ITERS, BS_CG_JACOBI, BS_CG_GRAPH, BS_CG_X0,
 * BS_CG_FF_OPERATOR (every A p with the float-float element operator of
 * bs_apply_A_ff; vectors, reductions and updates stay FP64; the solve runs
 * on the system scaled by the power of two that brings the RMS of b near 1,
 * exactly undone on x, so the operator's 2^-102 floor is relative to b;
 * d_hist then holds the scaled r.r), BS_CG_SCATTERED (the scattered form
 * that Sec. 3 sets against global storage: Z applied to both sides, every
 * CG vector kept as its N_L-sized scattered copy v_L = Z v_G, A p formed as
 * Z Z^T A_L p_L -- element kernel on contiguous local data, gather (BS6),
 * scatter (BS7) -- and each inner product summed over one copy of every
 * global node, the lowest local index, so that it equals the global one
 * term for term; b and x stay N_G vectors at the boundary; 122 N_L + 20 N_G
 * bytes per iteration against 24 N_L + 100 N_G in global storage, 1.5 times
 * as many at N = 7), BS_CG_BLOCK_JACOBI (the preconditioned Algorithm 1
 * with z = D^-1 r except on element interiors, where z_I = A_II^-1 r_I
 * solves the interior block of the element matrix exactly -- on every
 * element whose interior nodes are unmasked and held by that element alone;
 * no counterpart in the paper: it is the exact form of the map the learned
 * preconditioner imitates.  A_II^-1 is applied by fast diagonalisation, the
 * 1-D generalised eigenvectors of the interior stiffness and mass blocks, in
 * FP32 on per-element power-of-two-normalised values; affine elements of
 * degree 2..9 in global storage only).  Synchronises
 * `stream` before returning; info (host) may be NULL.  Returns
 * BS_ERR_NOT_CONVERGED if maxit is reached without BS_CG_FIXED_ITERS,
 * BS_ERR_BREAKDOWN on p.Ap <= 0. */
int bs_cg_solve(const bs_problem *prob, const double *b, double *x, double tol,
                int32_t maxit, int32_t flags, double *d_hist,
                bs_cg_info *info, void *stream);

/* CG with FP32 vectors inside FP64 iterative refinement (the mixed-precision
 * form of Algorithm 1; no counterpart in the paper, which studies FP64 only).
 * Outer loop in FP64: r = b - A x; stop when ||r|| <= tol ||b|| (the FP64
 * TRUE residual); else solve A d = r by Algorithm 1 with every vector and the
 * operator in FP32 (dot products carried as float pairs, alpha and beta in
 * double) to ||r_d|| <= inner_tol ||r|| from d_0 = 0, then x = x + d in FP64.
 * maxit caps the total inner iterations, outer_maxit the refinement steps.
 * flags: BS_CG_GRAPH (inner iterations replayed as a CUDA graph), BS_CG_X0.
 * info->iterations = inner iterations, info->outer = refinement steps,
 * info->rel_residual = ||b - A x|| / ||b|| in FP64.  Synchronises `stream`.
 * The problem owns the FP32 scratch (four N_G float vectors, allocated on
 * the first call).  Returns BS_ERR_NOT_CONVERGED or BS_ERR_BREAKDOWN as
 * bs_cg_solve does. */
int bs_cg_solve_refined_f32(const bs_problem *prob, const double *b, double *x,
                            double tol, int32_t maxit, double inner_tol,
                            int32_t outer_maxit, int32_t flags, bs_cg_info *info,
                            void *stream);

/* bs_cg_solve_batched: nsolves independent solves A_s x_s = b_s (Algorithm 1
 * on each; no counterpart in the paper, which runs one problem at a time),
 * advanced together.  Each CG iteration of all still-running solves is ONE
 * cooperative launch: fused scatter + element operator, gather with p.Ap,
 * fused update with r.r and the search-direction update, separated by grid
 * barriers; alpha, beta and the stop flag of every solve are formed on the
 * device from per-item partial sums taken in a fixed order (deterministic).
 * Solves that have stopped drop out of the work lists at no cost.
 *  - probs[s] must be distinct problems on the current device (each lends its
 *    scratch), of degree N <= 8; b[s], x[s] are DEVICE vectors of its N_G;
 *    x0 = 0.
 *  - Stop: r.r <= tol^2 b.b per solve, or maxit iterations.
 *  - flags: BS_CG_GRAPH (iterations replayed as a CUDA graph),
 *    BS_CG_REFINED_F32 (FP32-storage inner CG of every solve inside an FP64
 *    iterative refinement done for all solves together; inner tolerance 1e-4,
 *    at most 50 refinement steps; then tol is met by the FP64 TRUE residual
 *    and maxit caps each solve's total inner iterations), or
 *    BS_CG_FF_OPERATOR (FP64 form with the float-float element operator of
 *    bs_apply_A_ff).
 *  - infos[s] (host, may be NULL) receives each solve's iterations, outer
 *    steps, final r.r, b.b, relative residual, status; seconds is the whole
 *    batch's wall time.  Synchronises `stream`.
 *  - Grid barrier waits are bounded (about 2 s); on expiry the call returns
 *    BS_ERR_TIMEOUT.  Returns the first failing solve's status otherwise. */
int bs_cg_solve_batched(int32_t nsolves, const bs_problem *const *probs,
                        const double *const *b, double *const *x, double tol,
                        int32_t maxit, int32_t flags, bs_cg_info *infos,
                        void *stream);

/* Launch configuration of the batched solver.  Every field 0 = default.
 *  chunk: vector entries per work item of the update phases (a power of two
 *         in [1024, 65536]; default 4096);
 *  blocks_per_sm: cooperative grid = SMs x this, capped by occupancy
 *         (default: the occupancy maximum);
 *  unroll: vector entries each thread carries per sweep of the update
 *         phases, all loads issued together (1, 2, 4 or 8; default 4).
 * The block size (256 threads) is fixed by the element operator's mapping.
 * chunk and unroll change the order of the per-solve sums (results differ in
 * rounding, not in convergence); blocks_per_sm does not.  A given
 * configuration is deterministic. */
typedef struct {
  int32_t chunk;
  int32_t blocks_per_sm;
  int32_t unroll;
} bs_batched_config;

/* bs_cg_solve_batched with an explicit configuration (cfg may be NULL). */
int bs_cg_solve_batched_ex(int32_t nsolves, const bs_problem *const *probs,
                           const double *const *b, double *const *x, double tol,
                           int32_t maxit, int32_t flags, const bs_batched_config *cfg,
                           bs_cg_info *infos, void *stream);

/* Autotuner: times `iters` batched iterations (after one untimed) of these
 * solves under each candidate configuration -- chunk in {2048, 4096, 8192,
 * 16384} x unroll in {2, 4, 8} x blocks_per_sm in {1, occupancy maximum} --
 * from x = 0 into scratch solution vectors it allocates (the problems'
 * scratch is overwritten), with the given flags (BS_CG_REFINED_F32 times the
 * FP32 inner iteration, BS_CG_FF_OPERATOR the float-float one), and writes
 * the fastest to *best and its time per iteration (ms) to
 * *ms_per_iteration (may be NULL).  Synchronises `stream`. */
int bs_cg_batched_autotune(int32_t nsolves, const bs_problem *const *probs,
                           const double *const *b, int32_t flags, int32_t iters,
                           bs_batched_config *best, double *ms_per_iteration,
                           void *stream);

/* bs_set_wait_budget: the limit, in SM clock cycles, on every grid-barrier
 * wait of the batched solver's cooperative kernel, on the CURRENT device.
 * The paper has no counterpart: the bound is part of this library's failure
 * handling (a device-side wait that could spin forever gives up instead).
 * When a wait exceeds the budget the kernel records BS_ERR_TIMEOUT, every
 * block returns (a block that passed the barrier meets the next one and gives
 * up in turn), and bs_cg_solve_batched / bs_cg_batched_autotune return
 * BS_ERR_TIMEOUT with the solves' results undefined; the next call starts
 * from fresh barrier state.  cycles <= 0 restores the default, 2^32 cycles
 * (about 2 s at 2 GHz; cooperative launches keep every block resident, so a
 * healthy barrier never comes near it).  The old budget goes to *previous
 * (may be NULL).  Synchronous; call it while no batched solve is running on
 * the device.  The tcgen05 GEMM's mbarrier waits keep their own fixed limit.
 * Errors: BS_ERR_CUDA. */
int bs_set_wait_budget(int64_t cycles, int64_t *previous);

/* ------------------------------------------------------------ learned preconditioner */

/* A per-element network for a flexible PCG preconditioner.  The paper has no
 * learned part; everything in this section is this library's own definition.
 *
 * Network: y = W2 relu(W1 x), W1 [H x D], W2 [D x H] row-major FP32 masters,
 * no biases, D = (N+1)^3 values of one element.  Products run on the BF16
 * tensor cores with FP32 accumulation: in BF16 mode weights and activations
 * are single bf16 values; with BS_MLP_BF16X3 each is carried as hi + lo
 * (hi = bf16(v), lo = bf16(v - hi)) and a product is ahi bhi + ahi blo +
 * alo bhi, about 2^-16 relative instead of 2^-8.  Training is Adam on the
 * mean squared error, all in the library's kernels.
 *
 * Odd part: for a bias-free ReLU network, (f(x) - f(-x)) / 2 = W2 W1 x / 2
 * (relu(a) - relu(-a) = a) -- a LINEAR map.  BS_MLP_ODD / BS_FPCG_ODD
 * evaluate that instead of f; a Krylov method needs its preconditioner to be
 * (near) linear, and training on sign-symmetric pairs drives f's even part
 * W2 |W1 x| / 2 towards zero anyway. */
typedef struct bs_mlp bs_mlp;

enum {
  BS_MLP_BF16X3 = 1, /* bs_mlp_create: hi + lo bf16 operands (three products) */
  BS_MLP_ODD = 2,    /* bs_mlp_forward: the odd part W2 W1 x / 2              */
  BS_FPCG_ODD = 64,       /* bs_fpcg_learned: precondition with the odd part  */
  BS_FPCG_NO_JUDGE = 128  /* bs_fpcg_learned: never switch to Jacobi for good */
};

/* Engine of the network's GEMMs, process-wide: 0 (the default) runs every
 * GEMM on mma.sync (bf16 -> fp32); 1 runs them on the tcgen05 tensor cores
 * (accumulator in tensor memory, operands staged by cp.async in the
 * canonical K-major layout) wherever the shape allows -- K a multiple of 8,
 * 16-byte aligned operands, any epilogue but the relu' mask of the backward
 * pass.  Both give bitwise identical results; at the learned
 * preconditioner's shapes the mma.sync kernel is measured faster (97 vs
 * 137 us for the interior GEMM at N = 5 on 48^3).  Returns the previous
 * engine; any other value only queries it. */
int bs_gemm_engine(int32_t engine);

/* Create a network from HOST weights h_W1 [H x D], h_W2 [D x H] (copied).
 * 1 <= D <= 4096; H a multiple of 32 in [32, 4096].  flags: 0 or
 * BS_MLP_BF16X3.  Synchronous.  Adam state starts at zero. */
int bs_mlp_create(int32_t D, int32_t H, const float *h_W1, const float *h_W2,
                  int32_t flags, bs_mlp **out);
int bs_mlp_destroy(bs_mlp *mlp);
/* Copy the FP32 master weights to HOST h_W1 [H x D], h_W2 [D x H] (either
 * may be NULL).  Synchronous. */
int bs_mlp_get_weights(const bs_mlp *mlp, float *h_W1, float *h_W2);
/* Checkpointing the training state (the paper has no learned part; this is
 * the library's own): the FP32 master weights, both layers' Adam moments and
 * the Adam step count, as one host image of bs_mlp_state_bytes() bytes (a
 * header with the shape and the step, then the device arrays as stored).
 * Loading it into a network of the same D, H and precision mode and training
 * on continues bitwise as if training had never stopped.  Both calls
 * synchronise the device.  Errors: BS_ERR_ARG (short buffer, not an image,
 * shape or mode mismatch), BS_ERR_CUDA.  bs_mlp_state_bytes returns -1 for a
 * NULL network. */
int64_t bs_mlp_state_bytes(const bs_mlp *mlp);
int bs_mlp_save_state(const bs_mlp *mlp, void *h_buf, int64_t nbytes);
int bs_mlp_load_state(bs_mlp *mlp, const void *h_buf, int64_t nbytes);
/* d_Y [B x D] = f(d_X [B x D]) (DEVICE float), or the odd part with
 * BS_MLP_ODD.  Scratch for B rows is allocated on first use and kept. */
int bs_mlp_forward(bs_mlp *mlp, int64_t B, const float *d_X, float *d_Y,
                   int32_t flags, void *stream);
/* Mean squared error L = sum (f(x) - t)^2 / (B D) over a batch d_X, d_T
 * [B x D] into d_loss[0] (DEVICE double), and dL/dW1 [H x D], dL/dW2
 * [D x H] into d_gW1, d_gW2 (DEVICE float, may be NULL).  B a positive
 * multiple of 32.  The backward products use bf16 (hi) operands. */
int bs_mlp_loss_grad(bs_mlp *mlp, int64_t B, const float *d_X, const float *d_T,
                     double *d_loss, float *d_gW1, float *d_gW2, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr > 0)
 * on the batch; d_loss[0] receives the batch loss before the step. */
int bs_mlp_train_step(bs_mlp *mlp, int64_t B, const float *d_X, const float *d_T,
                      float lr, double *d_loss, void *stream);

/* Training pairs from a global residual d_r [N_G] (DEVICE): for pair q and
 * element e = d_elems[q] (DEVICE int32), with u = diag(A)^-1 r on the
 * element's (N+1)^3 nodes and rms = sqrt(mean u^2):
 *   d_X[q] = s u / rms,   d_T[q] = s (e_I - u_I) / rms on interior nodes
 *   (1 <= i,j,k <= N-1), 0 on the others,
 * where e_I solves A_II e_I = r_I, A_II the interior block of
 * c_e S_e + lambda M_e: the element-interior error, i.e. the correction
 * that zeroes the residual on the element's interior with its other nodes
 * held.  e_I comes from Jacobi-preconditioned CG on that element, run by one
 * thread block to a relative residual of 1e-13 (at most 4 (N-1)^3
 * iterations).  s = -1 for odd q when negate_odd (the pair (-r, -e) is as
 * valid as (r, e)), else 1; rms = 0 gives zero rows.  d_X, d_T are DEVICE
 * float [count x (N+1)^3].  Degrees 2..8. */
int bs_mlp_pairs(const bs_problem *prob, const double *d_r, int64_t count,
                 const int32_t *d_elems, int32_t negate_odd, float *d_X, float *d_T,
                 void *stream);

/* Flexible PCG with the learned correction, x0 = 0:
 *   z = M(r) = D^-1 r + corr,  corr_g = rms_e g(u_e / rms_e)_l at each
 *   element-interior node g (local index l of element e, 1 <= i,j,k <= N-1),
 *   0 at every other node, u = Z D^-1 r, rms_e = sqrt(mean u_e^2),
 * with g = f, or its odd part with BS_FPCG_ODD.  The training targets (the
 * element-interior error of bs_mlp_pairs) vanish off the interior, so only
 * interior outputs are used; each interior node belongs to one element.
 * alpha = r.z / p.Ap; x += alpha p; r -= alpha Ap; beta = r.(z' - z) /
 * (r.z)_old (Polak-Ribiere); p = z' + beta p.  mlp == NULL gives Jacobi-PCG.
 * Jacobi is the fallback and the judge: an iteration whose r.z' <= 0 (or not
 * finite) uses z' = D^-1 r (counted in info->fallbacks), and if r.r has not
 * fallen by 4 within max(1024, 16 N_G^(1/3)) iterations (a stall guard: r.r
 * is not monotone, and Jacobi-PCG itself has gone 7.5 N_G^(1/3) iterations
 * without halving it on these operators) the solve restarts from the current x
 * with Jacobi for good (info->outer = the iteration of that switch, 0 if
 * none).  Stop: r.r <= tol^2 b.b or maxit.  flags: BS_CG_GRAPH,
 * BS_FPCG_ODD, BS_FPCG_NO_JUDGE, BS_CG_FF_OPERATOR.  The network's input size must be (N+1)^3,
 * 2 <= N <= 9.  Synchronises `stream`.  Returns BS_ERR_NOT_CONVERGED or
 * BS_ERR_BREAKDOWN as bs_cg_solve does. */
int bs_fpcg_learned(const bs_problem *prob, bs_mlp *mlp, const double *b, double *x,
                    double tol, int32_t maxit, int32_t flags, bs_cg_info *info,
                    void *stream);

/* ------------------------------------------------------------ no allocation */

/* Largest number of per-block partial sums bs_dot_noalloc can hold. */
#define BS_NOALLOC_MAX_PARTIALS 2048

/* bs_dot_noalloc: the inner product x.y of bs_dot, written to d_out[0]
 * (DEVICE), for callers that must not allocate device memory -- code running
 * inside a host application that owns every device allocation through its
 * own pool, or a latency-critical loop where the implicit device
 * synchronisation of cudaMalloc/cudaFree is not acceptable.  The paper has
 * no counterpart to this entry point.
 *
 * Instead of a bs_workspace it uses scratch compiled into the library: a
 * static device array of BS_NOALLOC_MAX_PARTIALS doubles plus an arrival
 * counter (about 16 KiB), present on every GPU that loads libbs and held
 * until the process exits.  The call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine); the caller passes the inputs and
 * the output.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it; make
 *    that first call before any stream capture begins.
 *  - Every call shares the one array, which keeps the previous call's
 *    contents; the counter is cleared on `stream` at the start of each call.
 *    Calls that overlap on the GPU (on different streams, or from several
 *    threads) race on the array and give wrong results: serialise them.
 *  - The grid never exceeds BS_NOALLOC_MAX_PARTIALS blocks (the kernel is
 *    grid-stride, so any n fits); on a device with fewer resident blocks than
 *    that the result is bitwise the one of bs_dot.
 *  - Returns BS_ERR_ARG on the argument errors of bs_dot (n < 0, NULL output,
 *    NULL vectors with n > 0). */
int bs_dot_noalloc(int64_t n, const double *x, const double *y, double *d_out,
                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BS_H_ */
