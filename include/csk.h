/*
 * csk.h -- C ABI of the GB300 (sm_103a) Count Sketch Kaczmarz library.
 *
 * Method: Zhang & Li, "A Count Sketch Kaczmarz Method For Solving Large
 * Overdetermined Linear Systems" (arXiv 2004.02480).  The problem is the
 * consistent system A x = b with A m x n, m >> n (Section 1, eq. (1)).
 * Algorithm 1 takes A, b, the sketch size d and x0 and returns x: it forms
 * At = S A and bt = S b with the count sketch S = Phi D of Definition 1,
 * then repeats the maximal-weighted-residual step
 *     i_k = argmax_j |bt_j - At_j x_k| / ||At_j||,
 *     x_{k+1} = x_k + (bt_{i_k} - At_{i_k} x_k) / ||At_{i_k}||^2 * At_{i_k}^T
 * until RES = ||x_k - x*||^2 / ||x*||^2 <= 1e-6 or the step cap (Section 3).
 *
 * Conventions shared by every entry point
 *  - Matrices are row-major.  A has leading dimension lda >= n (elements).
 *    Indices are 0-based (the paper's [m], [d] are 1-based).
 *  - Every pointer named *_dev, and every array argument not marked "host",
 *    is CUDA device memory on the current device, allocated and owned by the
 *    caller.  The library never allocates or frees memory on these paths; the
 *    caller passes a workspace of at least the size the matching
 *    *_workspace_size function returns, 256-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work is enqueued on it; the call returns without
 *    synchronising.  Calls on different streams must use different
 *    workspaces and outputs.
 *  - Errors in the arguments are detected on the host and returned at once
 *    (CSK_EINVAL, CSK_EUNSUPPORTED); nothing is enqueued then.  A CUDA launch
 *    error is returned as CSK_ECUDA.  The outcome of the iteration (converged,
 *    cap reached, numerical failure, wait timeout) is written to the csk_info
 *    record in device memory when the stream reaches it; the return value
 *    CSK_OK then means "enqueued".
 *  - Randomness: the sketch of row i is drawn from the SplitMix64 output
 *    u_i = mix64(seed + (i+1) * 0x9E3779B97F4A7C15) (Steele, Lea & Flood
 *    2014): bucket h(i) = ((u_i >> 32) * d) >> 32, sign D_ii = -1 if bit 0 of
 *    u_i is set, else +1.  Same seed, same sketch, on every device.
 */
#ifndef CSK_H
#define CSK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CSK_OK = 0,            /* converged (in csk_info) / enqueued (return)   */
    CSK_MAXITER = 1,       /* step cap reached before the tolerance         */
    CSK_INPROGRESS = 2,    /* csk_batched_iterate: the unit's step budget of
                              this call ran out; call again to continue      */
    CSK_EINVAL = -1,       /* invalid argument (sizes, NULL, workspace)     */
    CSK_ENOMEM = -2,       /* a size overflows the supported index range    */
    CSK_ETIMEOUT = -3,     /* an inter-CTA wait exceeded its poll limit     */
    CSK_ENUMERIC = -4,     /* NaN/Inf residual, or At has no non-zero row   */
    CSK_ECUDA = -5,        /* a CUDA runtime call failed                    */
    CSK_EUNSUPPORTED = -6  /* valid request this library does not support   */
} csk_status;

typedef enum { CSK_F32 = 0, CSK_F64 = 1 } csk_dtype;

/* Residual path of the iteration.
 *  GEMV: r = bt - At x recomputed every step (Algorithm 1 as printed).
 *  GRAM: r_{k+1} = r_k - alpha_k G[:, i_k] with G = At At^T formed once on
 *        the tensor cores in split BF16 (hi*hi + hi*lo + lo*hi, FP32
 *        accumulation), r_{i_k} set to 0 exactly, and an FP64 recomputation
 *        of r every refresh_every steps.  Equal to GEMV in exact arithmetic.
 *  AUTO: the library picks (GEMV when the sketch fits on chip).
 *  UPDATE: the residual-update form of Remark 1: the loop keeps r and sets
 *        r_{k+1} = r_k - alpha_k At At_{i_k}^T (a GEMV of At against the
 *        chosen row, same bytes per step as GEMV), r_{i_k} = 0 exactly, with
 *        r recomputed as bt - At x at the first step and every refresh_every
 *        steps.  Runs the streamed loop (n a multiple of 16 bytes, n <= 1024
 *        FP32 / 512 FP64); equal to GEMV in exact arithmetic. */
typedef enum {
    CSK_RESID_GEMV = 0,
    CSK_RESID_GRAM = 1,
    CSK_RESID_AUTO = 2,
    CSK_RESID_UPDATE = 3
} csk_resid;

typedef struct {
    int64_t d;              /* sketch rows; 0 = no sketch (MWRK on A, Remark 1) */
    uint64_t seed;          /* sketch seed (Definition 1)                       */
    double tol;             /* RES tolerance, default 1e-6 (Section 3)           */
    int64_t max_iter;       /* step cap, default 20000 (Section 3)               */
    int32_t refresh_every;  /* GRAM: FP64 residual refresh period; UPDATE: period
                               of the recomputation bt - At x; 0 = off          */
    int32_t path;           /* csk_resid                                         */
    int64_t spin_limit;     /* polls per inter-CTA wait before CSK_ETIMEOUT,
                               0 = default (about a second)                      */
    int32_t *ik_log;        /* device, nullable: i_k of step k, k < ik_log_len   */
    int64_t ik_log_len;
    int32_t grid;           /* CTAs of the persistent kernel, 0 = library choice */
    int32_t fault_inject;   /* test hook: 1 = CTA 0 never publishes, so every
                               wait runs out and the solve ends CSK_ETIMEOUT     */
    void *x_log;            /* device, nullable: x_k (n elements of the dtype) of
                               step k < x_log_len, row k of an x_log_len x n
                               array -- the iterate step k selects from          */
    int64_t x_log_len;
    int32_t threads;        /* csk_solve_batched: threads per CTA, 0 = choice    */
    int32_t gemv_variant;   /* GEMV loop: 0 = library choice, 1 = rows of At in
                               shared memory (or read from global memory when
                               they do not fit), 2 = rows of At in registers
                               (FP32, n <= 512, n % 4 == 0, few rows per CTA),
                               3 = rows streamed every step through a shared-
                               memory ring of bulk copies (n a multiple of 16
                               bytes, n <= 1024 FP32 / 512 FP64; the choice
                               when rows fit neither registers nor shared
                               memory)                                          */
    void *stage_events[5];  /* optional cudaEvent_t handles (caller-owned), each
                               recorded on the stream when non-NULL: [0] before
                               the sketch, [1] after sketch and row norms, [2]
                               before the iteration (after the Gram matrix),
                               [3] after the iteration, [4] after the check     */
    int32_t log_system;     /* csk_solve_batched: ik_log / x_log record the
                               (system log_system, right-hand side log_rhs)
                               pair -- indices into the caller's array and
                               the system's columns; ignored by csk_solve   */
    int32_t log_rhs;
    int32_t fused;          /* csk_solve: 1 = form the sketch inside the loop's
                               cooperative kernel (each CTA sketches the rows
                               it owns in the loop; one launch for the sort,
                               the sums, the norms and the loop): GEMV path,
                               d <= 65535, at most 1024 rows per CTA, the
                               shared-memory loop or the register loop with
                               rows of 257..512 columns; CSK_EUNSUPPORTED
                               otherwise.  0 = separate
                               launches.  Stage events [1] and [2] are then
                               recorded before the loop, which includes the
                               sketch                                        */
    int32_t reserved_;
} csk_params;

/* Outcome of one solve, written by the device (64 bytes). */
typedef struct {
    int32_t status;         /* csk_status of the solve                          */
    int32_t path;           /* residual path used (csk_resid)                   */
    int64_t iters;          /* updates performed (IT of Section 3)              */
    double rse;             /* ||x - x*||^2 / ||x*||^2 in FP64 (NaN without x*) */
    double resid;           /* ||bt - At x|| / ||bt|| in FP64                    */
    int32_t rows;           /* rows iterated on (d, or m without sketch)        */
    int32_t empty_rows;     /* rows of At with zero norm (excluded, no 0/0)     */
    int32_t grid;           /* CTAs of the persistent kernel                    */
    int32_t reserved0;
    double reserved1;
    double reserved2;
} csk_info;

/* Defaults of Section 3: tol 1e-6, max_iter 20000, d = 0 (caller sets it),
 * seed 0, GEMV path, no refresh, default poll limit, no log. */
void csk_params_default(csk_params *p);

/* Human-readable name of a status code (static string). */
const char *csk_strerror(int status);

/* ABI version of this header (major * 10000 + minor * 100 + patch). */
int csk_version(void);

/* Number of CUDA kernels this library has enqueued in this process so far
 * (all devices and threads).  Lets a caller count the library's launches in
 * a region by differencing two reads. */
int64_t csk_kernel_launches(void);

/* ----------------------------------------------------------------------
 * csk_info_sync -- read a solve's outcome on the host.
 *
 * Algorithm 1's OUTPUT is x; its outcome under the Section 3 stopping rule
 * (converged at RES <= tol, step cap, failure) and IT are written by the
 * device into a csk_info record when the stream reaches the end of the
 * solve.  This copies the record info_dev (device, 64 bytes) into info_host
 * (host memory; page-locked or pageable) after the work queued on `stream`
 * so far, waits for the stream, and returns info_host->status (a csk_status:
 * CSK_OK, CSK_MAXITER, CSK_ENUMERIC, CSK_ETIMEOUT, ...).  Returns CSK_EINVAL
 * for a NULL pointer and CSK_ECUDA if the copy or the wait fails (the host
 * record is then unspecified).
 * -------------------------------------------------------------------- */
int csk_info_sync(const csk_info *info_dev, csk_info *info_host, void *stream);

/* ----------------------------------------------------------------------
 * csk_workspace_size -- one workspace size for every device entry point on
 * a problem of this shape.
 *
 * Algorithm 1's INPUT is A (m x n), b (here nrhs right-hand sides), the
 * sketch size d and x0; the residual path `resid` (csk_resid) selects
 * how r is updated.  Returns the largest of the workspaces that
 * csk_sketch(m, d), csk_solve(m, n, dtype, {d, resid}) and -- for FP32 with
 * d >= 1 and nrhs >= 1 -- csk_solve_batched of the one system (m, n, d,
 * nrhs) need, so a caller can size one buffer up front.  0 for invalid
 * sizes (m, n < 1, d < 0, nrhs < 0, bad dtype or path).
 * -------------------------------------------------------------------- */
size_t csk_workspace_size(int64_t m, int64_t n, int64_t d, int32_t nrhs, int32_t dtype,
                          int32_t resid);

/* ----------------------------------------------------------------------
 * csk_exchange_floor -- the latency floor of one step of the persistent
 * loop (no counterpart in the paper: a measurement aid).
 *
 * Every step of csk_solve's single-system loop ends with one exchange among
 * its CTAs: each CTA reduces its candidate for i_k across its warps, then
 * publishes it to every other CTA and waits for all of theirs.  This
 * enqueues one cooperative launch of `grid` CTAs (1 <= grid <= 320) that
 * runs `rounds` such exchanges (CTA reduction + mailbox round trip) and
 * nothing else, so (event time) / rounds is the per-step time of the loop
 * with its arithmetic taken away -- the floor a step cannot go below with
 * this exchange.  ws: csk_exchange_floor_workspace_size(grid) bytes (the
 * mailboxes and a status record).  Returns CSK_EINVAL for bad arguments,
 * CSK_ECUDA if the launch fails.
 * -------------------------------------------------------------------- */
size_t csk_exchange_floor_workspace_size(int32_t grid);

int csk_exchange_floor(int32_t grid, int64_t rounds, void *ws, size_t ws_bytes, void *stream);

/* ----------------------------------------------------------------------
 * csk_sketch -- Algorithm 1, "Initialize": At = S A and Bt = S B.
 *
 * A     m x n (lda >= n), dtype elements.  B m x nrhs (ldb >= nrhs), may be
 *       NULL when nrhs == 0.
 * At    out, d x n, leading dimension n.  Row j is the signed sum of the rows
 *       i with h(i) = j, added in ascending i (fixed order: an FP32 result
 *       is reproducible bit for bit).  Bt out, d x nrhs (ld nrhs), nullable.
 * norms2_out  out, nullable: d doubles, ||At_j||^2 accumulated in FP64.
 * perm_out    out, nullable: m int32, the rows sorted by (h(i), i).
 * off_out     out, nullable: d+1 int32, bucket j is perm[off[j] .. off[j+1]).
 * ws          scratch of csk_sketch_workspace_size(m, d) bytes.
 * Limits: 1 <= m, n, d <= 2^31 - 1; m * max(n, nrhs) elements addressable.
 * d >= m is accepted (rows of At may then be zero).
 * The library picks one of three ways to form the sums, all with the same
 * additions in the same order and so the same bits: a counting sort of the
 * rows by bucket followed by a segmented sum with a warp per bucket (FP32,
 * up to 128 rows per bucket on average) or a CTA per bucket, or, for FP32
 * problems of at most 32M elements, a pass in which each CTA owns a range
 * of buckets and orders their rows itself.  The environment variable
 * CSK_SKETCH_PATH = sort | own | warp | cta, read once per process, forces
 * a way where it applies (a test and measurement aid).
 * -------------------------------------------------------------------- */
size_t csk_sketch_workspace_size(int64_t m, int64_t d);

int csk_sketch(const void *A, int64_t m, int64_t n, int64_t lda,
               const void *B, int64_t ldb, int32_t nrhs, int32_t dtype,
               int64_t d, uint64_t seed,
               void *At, void *Bt, double *norms2_out,
               int32_t *perm_out, int32_t *off_out,
               void *ws, size_t ws_bytes, void *stream);

/* ----------------------------------------------------------------------
 * csk_sketch_noalloc -- csk_sketch without a workspace argument.
 *
 * The paper has no counterpart: this is a packaging variant for callers
 * that cannot allocate device memory -- code handed only input and output
 * pointers by a host application that owns all device memory (a plugin or
 * callback with no allocator in its interface), or latency-critical code
 * that must not call cudaMalloc because it can synchronise the device and
 * take driver-wide locks.  Arguments and results are those of csk_sketch;
 * the counting-sort scratch lives instead in one static device array of
 * about 10 MB, which every GPU that loads the library holds until the
 * process exits.  The call allocates nothing.
 * Limits: m <= 1,048,576 rows and d <= 262,144 buckets; larger sizes return
 * CSK_ENOMEM before anything is enqueued.
 * The first call on a device looks up the array's device address for that
 * device (a one-time host-side set-up); make that first call before any
 * stream capture.  The address is kept for the life of the process, so the
 * entry point must not be used on a device after cudaDeviceReset (a lookup
 * that failed is not kept: the next call tries again).  The stream must
 * belong to the current device (CSK_EINVAL otherwise, nothing enqueued).
 * Every call shares the one array (it keeps the last
 * call's contents; what must start at zero is cleared by each call), so
 * calls whose GPU work overlaps -- on different streams, or from different
 * host threads -- race and give wrong results.  Serialise them.
 * -------------------------------------------------------------------- */
int csk_sketch_noalloc(const void *A, int64_t m, int64_t n, int64_t lda,
                       const void *B, int64_t ldb, int32_t nrhs, int32_t dtype,
                       int64_t d, uint64_t seed,
                       void *At, void *Bt, double *norms2_out,
                       int32_t *perm_out, int32_t *off_out, void *stream);

/* ----------------------------------------------------------------------
 * csk_gram -- G = At At^T (d x d, FP32) on the tensor cores, split BF16.
 *
 * The residual of Algorithm 1 after the projection onto row i_k changes by
 * -alpha_k At At_{i_k}^T (from x_{k+1} = x_k + alpha_k At_{i_k}^T), so with G
 * the per-step residual update costs O(d) instead of O(dn).  G is formed as
 * hi hi^T + hi lo^T + lo hi^T with hi = bf16(At), lo = bf16(At - hi) (FP32
 * accumulation; about 2^-16 relative error per product).  Only tiles on or
 * above the diagonal are computed and mirrored, so G is exactly symmetric.
 * At     d x n FP32, leading dimension n.
 * norms2 nullable: d doubles; when given, G_jj is set to fl32(norms2_j).
 * G      out, d x d with leading dimension ldg >= d (ldg % 4 == 0 is fastest).
 * info   nullable device csk_info: status CSK_ETIMEOUT if a wait ran out.
 * ws     scratch of csk_gram_workspace_size(d, n) bytes (the BF16 operands).
 * -------------------------------------------------------------------- */
size_t csk_gram_workspace_size(int64_t d, int64_t n);

int csk_gram(const float *At, int64_t d, int64_t n, const double *norms2,
             float *G, int64_t ldg, csk_info *info, void *ws, size_t ws_bytes,
             void *stream);

/* ----------------------------------------------------------------------
 * csk_solve -- Algorithm 1 end to end for one right-hand side.
 *
 * A m x n (lda), b m-vector, dtype CSK_F32 or CSK_F64.  FP32 inputs iterate
 * in FP32 with FP64 row norms, FP64 refresh and FP64 final check; FP64
 * inputs iterate in FP64.
 * params  host pointer; params->d == 0 runs MWRK on A itself (Remark 1).
 * x0      nullable (x0 = 0); x_star nullable.  With x_star the step loop stops
 *         when RES <= tol (tested before every step, Section 3); without it
 *         when ||bt - At x||^2 / ||bt||^2 <= tol.
 * x_out   out, n elements of dtype.
 * info    out, device csk_info.
 * ws      scratch of csk_solve_workspace_size(m, n, dtype, params) bytes.
 * -------------------------------------------------------------------- */
size_t csk_solve_workspace_size(int64_t m, int64_t n, int32_t dtype,
                                const csk_params *params);

int csk_solve(const void *A, int64_t m, int64_t n, int64_t lda,
              const void *b, int32_t dtype, const csk_params *params,
              const void *x0, const void *x_star, void *x_out,
              csk_info *info, void *ws, size_t ws_bytes, void *stream);

/* ----------------------------------------------------------------------
 * csk_solve_host -- csk_solve with the problem and the results in HOST
 * memory: A, b, x0, x_star are copied to the device inside the call, x and
 * the csk_info record are copied back, and the call returns after the
 * stream has finished (the host buffers are then valid).  Page-locked host
 * buffers make the copies asynchronous DMA; pageable ones also work.
 * ws is DEVICE scratch of csk_solve_host_workspace_size(...) bytes: the
 * device copies of the inputs plus the workspace of csk_solve.
 * Return value: the csk_status of the solve itself (CSK_OK, CSK_MAXITER, ...)
 * once it has finished, or an argument / CUDA error.
 * -------------------------------------------------------------------- */
size_t csk_solve_host_workspace_size(int64_t m, int64_t n, int32_t dtype,
                                     const csk_params *params);

int csk_solve_host(const void *A_host, int64_t m, int64_t n, int64_t lda,
                   const void *b_host, int32_t dtype, const csk_params *params,
                   const void *x0_host, const void *x_star_host,
                   void *x_out_host, csk_info *info_host,
                   void *ws, size_t ws_bytes, void *stream);

/* ----------------------------------------------------------------------
 * csk_solve_host_many -- a sequence of csk_solve_host problems, solved one
 * after another on `stream`, with the host-to-device copies of problem k+1
 * (on a copy stream the library creates once per device, with its events,
 * and reuses in later calls) overlapping the solve of problem k.  Every problem is an independent run of Algorithm 1 with the
 * same params (one sketch seed, d, tolerance, path); overlapping the copies
 * changes no arithmetic.  This is the pipelining a solver service applies
 * to a stream of systems arriving in host memory (the paper has no
 * counterpart: it concerns one solve).
 * probs   host array of `count` problems; every pointer in it is HOST memory
 *         (page-locked for the copies to overlap; pageable works but
 *         serialises more); A m x n with leading dimension lda, x0 / x_star
 *         nullable, x_out n elements, info one record.  The results of
 *         problem k are queued after the input copies of problem k+1.
 * ws      DEVICE scratch of csk_solve_host_many_workspace_size(...) bytes:
 *         two staging areas (the largest problem's device copies) that
 *         alternate, plus one csk_solve workspace shared by the solves.
 * Returns after every queued solve has finished: CSK_OK, the first
 * non-OK solve status in problem order (each info record holds its own),
 * or an argument / CUDA error.  The argument checks of every problem run
 * before any copy is queued; count == 0 does nothing.
 * -------------------------------------------------------------------- */
typedef struct {
    const void *A;        /* m x n, leading dimension lda (host)                */
    int64_t m, n, lda;
    const void *b;        /* m (host)                                           */
    const void *x0;       /* nullable, n (host)                                 */
    const void *x_star;   /* nullable, n (host)                                 */
    void *x_out;          /* out, n (host)                                      */
    csk_info *info;       /* out, one record (host)                             */
} csk_host_problem;

size_t csk_solve_host_many_workspace_size(const csk_host_problem *probs, int32_t count,
                                          int32_t dtype, const csk_params *params);

int csk_solve_host_many(const csk_host_problem *probs, int32_t count, int32_t dtype,
                        const csk_params *params, void *ws, size_t ws_bytes, void *stream);

/* ----------------------------------------------------------------------
 * csk_solve_batched -- many independent systems, each with several
 * right-hand sides, in one persistent launch (FP32, GRAM residual path).
 *
 * Each (system, right-hand side) pair is one run of Algorithm 1 with the
 * system's own count sketch (d, seed) and the Section 3 stopping rule; the
 * sketch and split-BF16 Gram matrix of a system are formed once and shared
 * by its right-hand sides.  A CTA runs one pair at a time to completion,
 * pairs ordered by decreasing d*n; CTAs never wait for each other.
 * Every array in csk_system is device memory; B, X0, Xstar and Xout hold one
 * column per right-hand side (row-major, leading dimensions ldb / nrhs).
 * info: nrhs csk_info records per system (device), written when the pair
 * finishes; rse is FP64, resid uses a compensated FP32 dot product.
 * params: tol, max_iter, refresh_every (FP64 residual recomputation period,
 * 0 = never), grid and threads; d/seed/path ignored.  With threads = grid = 0
 * the call uses the launch shape installed for this batch's signature by
 * csk_solve_batched_set_plan (an autotuner's pick), else the library's
 * default (256 threads, as many CTAs as stay resident).  ik_log / x_log (with
 * log_system, log_rhs) record i_k and x_k of one pair, as in csk_solve.
 * The host array `sys` is read during the call only, and nothing in the call
 * synchronises, so the sequence can be captured in a CUDA graph.
 * ws: csk_solve_batched_workspace_size(sys, nsys) bytes (sketches, Gram
 * matrices and descriptors of every system, and the scratch of the prepare
 * lanes described under csk_batched_prepare).
 * -------------------------------------------------------------------- */
typedef struct {
    const void *A;        /* m x n FP32, leading dimension lda                  */
    int64_t m, n, lda;
    const void *B;        /* m x nrhs FP32, leading dimension ldb               */
    int64_t ldb;
    int32_t nrhs;
    int32_t reserved_;
    int64_t d;            /* sketch rows of this system                         */
    uint64_t seed;        /* sketch seed of this system                         */
    const void *X0;       /* nullable, n x nrhs                                 */
    const void *Xstar;    /* nullable, n x nrhs                                 */
    void *Xout;           /* n x nrhs                                           */
    csk_info *info;       /* nrhs records                                       */
    void *area;           /* nullable: the system's resident area (256-byte
                             aligned, csk_batched_area_size bytes: its sketch,
                             Gram matrix and unit states); NULL = carved from
                             the workspace (csk_solve_batched only)           */
} csk_system;

size_t csk_solve_batched_workspace_size(const csk_system *sys, int32_t nsys);

/* ----------------------------------------------------------------------
 * Step-chunked batched solves (continuous batching): the two halves of
 * csk_solve_batched, for a caller that keeps each system's sketch and Gram
 * matrix resident and runs its units a chunk of steps at a time, so that
 * systems arriving later join the next chunk's launch.
 *
 * csk_batched_area_size: bytes of one system's resident area.
 * csk_batched_prepare: Algorithm 1's Initialize for every system (its
 *   sketch At, Bt, the FP64 row norms and the split-BF16 Gram matrix, as in
 *   csk_solve_batched) into sys[i].area (required), and resets its units.
 *   ws: csk_batched_prepare_workspace_size(sys, nsys) bytes of scratch (one
 *   sort and one Gram scratch per lane: the systems are prepared on up to
 *   four streams forked from `stream` and joined back to it before the call's
 *   later work on `stream`; while `stream` is being captured into a CUDA
 *   graph and no lane streams exist yet, on `stream` alone).  Each system's
 *   results do not depend on the lane it ran on.
 * csk_batched_iterate: one persistent launch running every unfinished unit
 *   of the prepared systems for at most step_budget more steps (0 = to the
 *   end), resuming it where the previous call left it (r, x and the pending
 *   projection are saved in the area).  A unit that finishes writes Xout and
 *   its info as csk_solve_batched does; one that does not reports
 *   CSK_INPROGRESS with iters = steps so far.  Units already finished cost
 *   nothing.  A unit's arithmetic does not depend on the budget: the same
 *   steps in the same order, whatever the chunking.  params as for
 *   csk_solve_batched (the same tol, max_iter, refresh_every on every call
 *   of a system); ws: csk_batched_iterate_workspace_size(nsys) bytes.
 * Both return CSK_EINVAL for bad arguments (a NULL area included) and do not
 * synchronise.
 * -------------------------------------------------------------------- */
size_t csk_batched_area_size(int64_t n, int64_t d, int32_t nrhs);
size_t csk_batched_prepare_workspace_size(const csk_system *sys, int32_t nsys);
size_t csk_batched_iterate_workspace_size(const csk_system *sys, int32_t nsys);
int csk_batched_prepare(const csk_system *sys, int32_t nsys, void *ws, size_t ws_bytes,
                        void *stream);
int csk_batched_iterate(const csk_system *sys, int32_t nsys, const csk_params *params,
                        int64_t step_budget, void *ws, size_t ws_bytes, void *stream);

int csk_solve_batched(const csk_system *sys, int32_t nsys, const csk_params *params,
                      void *ws, size_t ws_bytes, void *stream);

/* Install the launch shape (threads per CTA: 64..512, a multiple of 32; CTAs
 * >= 1) that csk_solve_batched uses for batches of this signature when called
 * with threads = grid = 0, on the current device; threads = grid = 0 removes
 * it.  The signature (csk_solve_batched_signature) is the number of
 * right-hand sides per (floor(log2 d), floor(log2 n)) bin, so batches with
 * the same shape distribution share a plan.  An autotuner times candidate
 * shapes with explicit threads / grid and installs the fastest; the shape
 * changes only how pairs are scheduled, not any pair's arithmetic at a given
 * thread count.  Host-only (the table lives in the process); thread-safe.
 * Returns CSK_EINVAL for bad arguments. */
int csk_solve_batched_set_plan(const csk_system *sys, int32_t nsys, int32_t threads,
                               int32_t grid);
uint64_t csk_solve_batched_signature(const csk_system *sys, int32_t nsys);

/* ----------------------------------------------------------------------
 * csk_synth_systems -- seeded Gaussian test systems generated on the device
 * (no counterpart in the paper: the stand-in for systems that arrive with
 * their data, used by the serving harness).
 *
 * For each system: A (m x n, row-major, leading dimension n) and X (n x nrhs,
 * row-major) get iid N(0,1) entries, each a pure function of (seed, matrix,
 * element index) -- a SplitMix64 counter hash and Box-Muller -- so a system's
 * data do not depend on the other systems of the call; then B = A X
 * (m x nrhs) accumulated in FP32 in a fixed order.  All pointers are DEVICE
 * memory owned by the caller; nrhs <= 16.  Two launches per 32 systems; no
 * synchronisation.  Returns CSK_EINVAL / CSK_ENOMEM on bad sizes (nothing
 * enqueued), CSK_ECUDA if a launch fails.
 * -------------------------------------------------------------------- */
typedef struct {
    int64_t m, n;
    int32_t nrhs;
    int32_t reserved_;
    uint64_t seed;
    void *A;              /* out, m x n FP32                                    */
    void *X;              /* out, n x nrhs FP32                                 */
    void *B;              /* out, m x nrhs FP32                                 */
} csk_synth_system;

int csk_synth_systems(const csk_synth_system *sys, int32_t count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CSK_H */
