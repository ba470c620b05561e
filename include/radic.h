/*
 * radic.h -- C ABI of the GB300 (sm_103a) library for Radic's determinant of
 * a non-square matrix.
 *
 * Definition (Definition 3, Eq. (1) of Abdollahi, Jafari, Bayat, Amiri and
 * Fathy, "An efficient parallel algorithm for computing determinant of
 * non-square matrices based on Radic's definition", arXiv 1508.01326):
 * for an m x n matrix A with m <= n,
 *
 *     det_R(A) = sum over 1 <= j1 < ... < jm <= n of
 *                (-1)^(r+s) * det(A[:, j1..jm]),
 *     r = 1 + 2 + ... + m,   s = j1 + ... + jm,
 *
 * and det_R(A) = 0 when m > n.  The C(n,m) column sequences are numbered
 * 0 .. C(n,m)-1 in dictionary order (Definition 2, Table 2); each one is
 * produced directly from its number (Section 4, Theorem 2), so every minor is
 * independent of every other one and the GPU processes contiguous runs of
 * numbers (Section 5).
 *
 * Conventions for every entry point below:
 *  - Matrices are row-major: element (i, j) of A is A[i * lda + j], lda >= n.
 *  - "device" pointers are CUDA device memory on the current device and are
 *    owned by the caller; the library never frees them.  "host" pointers are
 *    ordinary host memory.  Except where stated (batch plans and graphs),
 *    the library allocates no memory: scratch memory is the caller's
 *    `workspace` of at least the size that the matching *_workspace_bytes
 *    function returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it and return without waiting; results
 *    are valid once the stream reaches that point.
 *  - The return value reports host-side validation and launch errors only
 *    (RADIC_OK, RADIC_EINVAL, ...).  Errors found on the device are written
 *    to the `status` field of the device-resident result.
 *  - Limits: 1 <= m <= RADIC_MAX_M, 1 <= n <= RADIC_MAX_N.  m > n is valid
 *    and gives 0 (Definition 3).  With n <= 64 every rank fits in 63 bits.
 */
#ifndef RADIC_H
#define RADIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RADIC_MAX_M 32
#define RADIC_MAX_N 64
#define RADIC_MAX_PRIMES 4
#define RADIC_WIDE_MAX_PRIMES 32
#define RADIC_WIDE_LIMBS 32

/* Status codes (return values and radic_result.status). */
enum {
  RADIC_OK = 0,
  RADIC_EINVAL = 1,      /* bad argument: size, pointer, dtype, mode, lda     */
  RADIC_EOVERFLOW = 2,   /* exact result may need more than the prime budget  */
  RADIC_ECUDA = 3,       /* a CUDA runtime call failed                         */
  RADIC_ETIMEOUT = 4,    /* a bounded device-side wait gave up                 */
  RADIC_EWORKSPACE = 5,  /* workspace pointer null/misaligned or too small     */
  RADIC_EUNSUPPORTED = 6 /* valid request the library does not implement       */
};

/* Element type of A. */
enum { RADIC_I8 = 0, RADIC_I32 = 1, RADIC_F32 = 2, RADIC_F64 = 3 };

/* Arithmetic of the minor determinants.
 *  FP64  -- binary64 partial-pivot LU per minor, binary64 compensated sum.
 *  MIXED -- binary32 partial-pivot LU per minor; minors whose pivot growth
 *           exceeds the threshold, whose result is not finite, or one of
 *           whose dividing pivots is not bounded away from zero by its
 *           error radius, are recomputed in binary64; sums are compensated
 *           (float-float per run of ranks, then binary64 two-sum across
 *           runs and blocks).
 *  EXACT -- LU modulo 31-bit primes (as many as a Hadamard bound needs, at
 *           most RADIC_MAX_PRIMES) and Chinese remaindering to a signed
 *           128-bit integer, bit-exact.  Integer inputs directly; binary32
 *           and binary64 inputs (radic_det only) as the dyadic rationals they
 *           are: row i is scaled by 2^-e_i, e_i the exponent of the lowest
 *           set bit among its nonzero entries, to an integer row, and the
 *           result is the integer times 2^exact_exp, exact_exp = sum_i e_i.
 *           Inputs with many significant bits per row (for instance random
 *           binary64 values) exceed the prime budget: status
 *           RADIC_EOVERFLOW; radic_det_exact_wide takes up to
 *           RADIC_WIDE_MAX_PRIMES primes for them.  A non-finite entry:
 *           status RADIC_EINVAL.
 *  PAIR  -- the MIXED scheme with the leaves carried out in pairs of
 *           binary32 numbers (hi + lo, about 48 significant bits, on the
 *           binary32 pipe) and the prefix factorisations in binary64:
 *           PREFIX mapping, 3 <= m <= 10; flagged prefixes are recomputed
 *           in binary64.  Also the value of a batched result's `tier`
 *           field for matrices routed to pairs. */
enum { RADIC_MODE_FP64 = 0, RADIC_MODE_MIXED = 1, RADIC_MODE_EXACT = 2, RADIC_MODE_PAIR = 3 };

/* Minor-to-thread mapping.
 *  THREAD -- one thread factors one minor in registers (m <= 8 for FP64,
 *            m <= 12 for MIXED and EXACT).
 *  GROUP  -- a group of `group_width` lanes of one warp (16 or 32) factors
 *            one minor, one row per lane, pivot rows shared by warp shuffles.
 *  PREFIX -- 3 <= m <= n, m <= 10 (FP64, PAIR) or 12 (MIXED, EXACT): one
 *            thread factors the m x (m-D) matrix of an ascending
 *            (m-D)-column prefix once (D = 2 or 3, the prefix depth;
 *            partial pivoting, or in EXACT mode the first nonzero pivot of
 *            a non-dividing elimination mod p); every minor of that
 *            prefix's lexicographic subtree then costs one D x D
 *            determinant of Schur-complement entries (for D = 3 a scalar
 *            triple product).  Same pivots and elimination steps as
 *            per-minor LU, shared by the subtree.
 *  AUTO   -- PREFIX when 3 <= m <= n within its limit, else THREAD when
 *            m <= 8 (12 for EXACT), else GROUP. */
enum { RADIC_MAP_AUTO = 0, RADIC_MAP_THREAD = 1, RADIC_MAP_GROUP = 2, RADIC_MAP_PREFIX = 3 };

/* Launch and precision options.  Pass NULL for the defaults; a zero field
 * also means "default". */
typedef struct radic_options {
  int32_t mapping;          /* RADIC_MAP_*                                    */
  int32_t group_width;      /* GROUP mapping: 16 or 32 lanes per minor        */
  int32_t ranks_per_task;   /* consecutive ranks per task (default 64)        */
  int32_t threads_per_block;/* 32..256 (EXACT: ..128), multiple of 32 (128)   */
  int32_t blocks;           /* grid size (default: SMs x resident blocks)     */
  int32_t flag_capacity;    /* MIXED: flagged ranks kept per warp (default 32)*/
  double growth_threshold;  /* MIXED: flag when max|pivot| > t * max|a| (64)  */
  void* kernel_events;      /* optional: two cudaEvent_t recorded on the
                               stream right before and right after the main
                               per-minor kernel (profiling hook)             */
  int32_t prefix_depth;     /* PREFIX mapping: trailing columns per leaf, 2 or
                               3 (0: 3 when m >= 7 and n - m <= 3.5m, else 2) */
  int32_t lanes_per_prefix; /* PREFIX mapping: lanes of a warp that share the
                               leaves of one prefix (1, 2, 4, ..., 32; 0:
                               per prefix group, from the plan's cost model) */
  int32_t deterministic;    /* PREFIX mapping, floating-point modes: 0
                               (default) = after its first task a warp draws
                               the next from a counter, which evens out the
                               warps' work; which warp sums which prefixes then
                               varies, so repeated calls can differ in the last
                               bits of value and abs_sum (far below err_bound).
                               1 = every warp takes a fixed share of the
                               tasks: repeated calls give identical bits.
                               The exact mode is exact either way. */
  int32_t reserved32;
  int64_t reserved[1];
} radic_options;

/* Device-resident result of one determinant (16 eight-byte words). */
typedef struct radic_result {
  double value;     /* det_R(A) rounded to binary64 (EXACT: from exact value)  */
  double abs_sum;   /* sum over J of |det(A[:, J])| in the mode's arithmetic   */
  double err_bound; /* floating-point modes: an upper bound on
                       |value - det_R(A)| for A as given (it also covers
                       the final rounding of value to binary64), from
                       running error analysis of the eliminations actually
                       performed (midpoint-radius enclosures of every
                       quantity; a pivot whose enclosure reaches zero gets
                       its minor or prefix redone in binary64, or in
                       binary64 is bounded by Hadamard's inequality on the
                       enclosure of the remaining Schur complement) and of
                       the summations; +inf or NaN when no bound could be
                       formed.  Entries below about 2^-100 (binary32,
                       pairs) or 2^-70 (binary64) of their row's largest are
                       not covered.  EXACT: 0.                             */
  int64_t exact_lo; /* EXACT: low 64 bits of det_R(A), two's complement int128 */
  int64_t exact_hi; /* EXACT: high 64 bits                                     */
  int64_t minors;   /* C(n, m), or 0 when m > n                                */
  int64_t flagged;  /* MIXED: minors recomputed in binary64                    */
  int64_t status;   /* RADIC_OK, RADIC_EOVERFLOW, RADIC_ETIMEOUT ...           */
  int64_t n_primes; /* EXACT: primes used                                      */
  int64_t tier;     /* mode that produced value (batched router decision)      */
  int64_t exact_exp;/* EXACT: det_R(A) = (exact_hi:exact_lo) * 2^exact_exp
                       (0 for integer inputs; see RADIC_MODE_EXACT)            */
  int64_t reserved[5];
} radic_result;

/* Device-resident result of radic_det_exact_wide (192 bytes). */
typedef struct radic_wide_result {
  double value;      /* det_R(A) rounded to binary64 (within one unit in the
                        last place; +-inf beyond binary64's range)          */
  int64_t status;    /* RADIC_OK, RADIC_EOVERFLOW (the bound needs more than
                        RADIC_WIDE_MAX_PRIMES primes), RADIC_EINVAL (an
                        entry is not finite)                                 */
  int64_t n_primes;  /* primes used                                          */
  int64_t exact_exp; /* det_R(A) = sign * magnitude * 2^exact_exp            */
  int64_t sign;      /* -1, 0 or +1                                          */
  int64_t n_limbs;   /* limbs holding the magnitude (the others are 0)       */
  int64_t minors;    /* C(n, m), or 0 when m > n                             */
  int64_t reserved;
  uint32_t limbs[RADIC_WIDE_LIMBS]; /* magnitude = sum_i limbs[i] 2^(32 i)   */
} radic_wide_result;

/* ---- general ------------------------------------------------------------ */

/* Human-readable name of a status code (static string, never NULL). */
const char* radic_status_string(int status);

/* Library version as 10000*major + 100*minor + patch. */
int radic_version(void);

/* The 31-bit primes of the EXACT mode, in the order they are used.
 * primes: host array of at least max_count entries.  Returns how many
 * primes were written (at most RADIC_MAX_PRIMES). */
int radic_primes(uint32_t* primes, int max_count);

/* ---- one matrix --------------------------------------------------------- */

/* Bytes of workspace radic_det needs for this shape, mode and options
 * (a multiple of 256; the workspace must be 256-byte aligned).  Returns 0
 * for invalid arguments. */
size_t radic_workspace_bytes(int m, int n, int mode, const radic_options* opts);

/* The launch plan radic_det would use for this shape, mode and options,
 * written to the first `count` (<= RADIC_PLAN_INFO_COUNT) entries of host
 * array info: [0] mapping (RADIC_MAP_THREAD, _GROUP or _PREFIX), [1] prefix
 * depth (0 unless PREFIX), [2] group width (0 unless GROUP), [3] threads per
 * block, [4] blocks of the main kernel, [5] ranks per processor run (THREAD,
 * GROUP) or warp tasks (PREFIX), [6] dynamic shared memory bytes of the main
 * kernel, [7] workspace bytes.  Same errors as radic_det's planning. */
#define RADIC_PLAN_INFO_COUNT 8
int radic_plan_info(int m, int n, int mode, const radic_options* opts, int64_t* info, int count);

/* Host-only view of the prefix mapping's task table (the Section 5 split of
 * the minors into contiguous runs, here runs of prefixes grouped by their
 * last column v), planned for `sms` SMs with `blocks_per_sm` resident blocks
 * instead of the current device: no GPU is touched.  opts->mapping is taken
 * as RADIC_MAP_PREFIX.  info (host, count >= 8 + 4n int64): [0] prefix depth
 * D, [1] warp tasks, [2] blocks, [3] v_lo, [4] v_hi, [5] 1 when warps draw
 * tasks from the counter, [6..7] 0; then for every v four entries at
 * 8 + 4v: prefixes whose last column is v (C(v, m-D-1)), prefixes per lane
 * group in one task, lanes per prefix, first task of the group (0 outside
 * v_lo..v_hi).  Errors: RADIC_EINVAL, RADIC_EUNSUPPORTED as radic_det's
 * planning. */
int radic_prefix_plan_host(int m, int n, int mode, const radic_options* opts, int sms, int blocks_per_sm,
                           int64_t* info, int count);

/* det_R(A) of one m x n matrix (Eq. (1)).
 * A:        device, m x n, row-major with leading dimension lda, type dtype.
 * out:      device, one radic_result, fully overwritten.
 * workspace:device scratch, >= radic_workspace_bytes(m, n, mode, opts).
 * The hot path per minor: unrank its dictionary-order number with a binomial
 * table staged in shared memory (Section 4), step to the next numbers with
 * the dictionary successor (Section 5), gather the m x m minor from shared
 * memory, factor it (LU with partial pivoting, or modular elimination),
 * apply the sign (-1)^(r+s), and accumulate; per-block partial sums are
 * combined in a fixed order by the last block (tree sum of Section 6).
 * Calls on different streams need separate workspaces.
 * Errors: RADIC_EINVAL (m or n out of range, lda < n, NULL A or out,
 * unknown dtype/mode), RADIC_EWORKSPACE, RADIC_ECUDA.  Device:
 * out->status = RADIC_EOVERFLOW when the exact value could exceed the prime
 * budget, RADIC_EINVAL when EXACT meets a non-finite real entry. */
int radic_det(const void* A, int m, int n, int64_t lda, int dtype, int mode,
              const radic_options* opts, radic_result* out, void* workspace,
              size_t workspace_bytes, void* stream);

/* EXACT det_R(A) (Definition 3, Eq. (1)) beyond the 128-bit range of
 * radic_det: the same modular elimination and row scaling as RADIC_MODE_EXACT
 * (integer inputs, and binary32/binary64 inputs as the dyadic rationals
 * they are), with as many 31-bit primes as the Hadamard bound of the scaled
 * integer rows needs, up to RADIC_WIDE_MAX_PRIMES (about 990 bits).  The
 * primes are taken RADIC_MAX_PRIMES per pass of the EXACT kernels (passes
 * whose primes the bound does not need return at once), and a last kernel
 * rebuilds the integer by mixed-radix (Garner) reconstruction into base-2^32
 * limbs.  Not a computation of the paper: its extension of the exact mode to
 * inputs whose value does not fit 128 bits.
 * A: device, row-major m x n, leading dimension lda; out: device;
 * workspace: device, 256-byte aligned, radic_wide_workspace_bytes(m, n,
 * opts) bytes.  Options as radic_det's (mapping, threads, prefix depth).
 * Errors: RADIC_EINVAL (m or n out of range, lda < n, NULL pointers, unknown
 * dtype), RADIC_EWORKSPACE, RADIC_ECUDA; device: out->status. */
size_t radic_wide_workspace_bytes(int m, int n, const radic_options* opts);
int radic_det_exact_wide(const void* A, int m, int n, int64_t lda, int dtype, const radic_options* opts,
                         radic_wide_result* out, void* workspace, size_t workspace_bytes, void* stream);

/* The signed terms (-1)^(r+s) det(A[:, J_q]) of Eq. (1) for the consecutive
 * dictionary ranks q = q0 .. q0+count-1 (all < C(n,m)), computed by the same
 * per-minor device code as radic_det with the same options.
 * terms: device.  FP64: count doubles.  MIXED: count doubles holding the
 *        binary32 results (flagged minors are not recomputed here; a NaN
 *        marks each flagged minor).  EXACT: RADIC_MAX_PRIMES x count uint32
 *        residues in [0, p), prime-major in the order of radic_primes; only
 *        the first K rows are written, K being the number of primes
 *        radic_det uses for this A (radic_result.n_primes).
 * No workspace.  Errors: RADIC_EINVAL (as radic_det, EXACT with a real
 * dtype, or a rank outside [0, C(n,m))), RADIC_ECUDA. */
int radic_terms(const void* A, int m, int n, int64_t lda, int dtype, int mode,
                const radic_options* opts, uint64_t q0, uint64_t count,
                void* terms, void* stream);

/* Column sequences of the dictionary ranks q0 .. q0+count-1 (Section 4 and
 * the successor of Section 5), as the device computes them.
 * cols: device, count x m bytes, 0-based column indices.
 * Errors: RADIC_EINVAL (bad sizes or a rank outside [0, C(n,m))),
 * RADIC_ECUDA. */
int radic_unrank(int n, int m, uint64_t q0, uint64_t count, uint8_t* cols,
                 const radic_options* opts, void* stream);

/* A captured CUDA graph of one radic_det call on fixed buffers (opaque). */
typedef struct radic_graph radic_graph;

/* Captures one radic_det call with these arguments into a CUDA graph owned
 * by the library; radic_graph_launch replays it on any stream (same
 * kernels, without the per-call planning and launch latency), and
 * radic_graph_destroy frees it.  The buffers must stay valid while the graph
 * is used.  Errors: those of radic_det, and RADIC_ECUDA if capture fails. */
int radic_graph_create(const void* A, int m, int n, int64_t lda, int dtype, int mode, const radic_options* opts,
                       radic_result* out, void* workspace, size_t workspace_bytes, radic_graph** graph);
int radic_graph_launch(radic_graph* graph, void* stream);
int radic_graph_destroy(radic_graph* graph);

/* ---- batches of matrices of uneven shape ------------------------------- */

/* Host-side plan (opaque) of one batch layout, and a captured CUDA graph of
 * one batched call. */
typedef struct radic_batch_plan radic_batch_plan;
typedef struct radic_batch_graph radic_batch_graph;

/* Per-m tuning of the batched path (written by the autotuner; zero fields
 * mean "default").  kind[m]: RADIC_MAP_PREFIX or RADIC_MAP_THREAD (per-minor,
 * m <= 8).  task_cost[m]: target work per lane and task, in the plan's cost
 * units (default 30000; smaller = more, shorter tasks). */
typedef struct radic_batch_tuning {
  int32_t kind[RADIC_MAX_M + 1];
  double task_cost[RADIC_MAX_M + 1];
  double tol;              /* MIXED: target |err| / sum|terms| (default 1e-10) */
  double growth_threshold; /* MIXED: growth flag threshold (default 64)         */
  int32_t blocks_per_sm;   /* cap on resident blocks per SM (0: occupancy)     */
  int32_t prefix_depth[RADIC_MAX_M + 1]; /* 2, 3, or 0 for the default rule */
  int32_t tiers;           /* MIXED: allowed low tiers, bit 0 binary32, bit 1
                              pairs (0: both); binary64 is always allowed  */
  int32_t head_sharing;    /* prefix tasks with m - D - 1 >= 5: factor each
                              head (first m-D-1 columns) once for all its
                              prefixes (0: on, -1: off)                      */
  int32_t reserved[5];
  void* kernel_events;     /* optional: two cudaEvent_t recorded on the call's
                              stream right before and right after the launch
                              of the plan's dominant kernel, the low-tier
                              kernel with the most estimated work (profiling
                              hook; see radic_batch_plan_info [12..14])       */
} radic_batch_tuning;

/* Builds the plan of `batch` matrices: matrix b is m[b] x n[b], row-major
 * with leading dimension n[b], starting offsets[b] elements into one packed
 * buffer (all three arrays are host memory).  mode is RADIC_MODE_FP64 or
 * RADIC_MODE_MIXED.  In MIXED mode each matrix is routed to the cheapest
 * allowed tier whose expected error relative to sum|terms| meets
 * tuning->tol: binary32 elimination when 2.5e-6 / sqrt(C(n,m)) meets it,
 * else pairs of binary32 (m >= 3) when 1e-11 / sqrt(C(n,m)) meets it, else
 * binary64 (the constants are envelopes of measured errors on random
 * inputs).  Binary32 and pair tasks that meet a growth flag are redone in
 * binary64.  The result's `tier` field holds RADIC_MODE_MIXED (binary32),
 * RADIC_MODE_PAIR or RADIC_MODE_FP64.  The work of every matrix is cut into warp tasks
 * (runs of prefixes or of dictionary ranks, per the tuning) for persistent
 * kernels with atomic work queues, one per tier and m, followed by a
 * per-matrix fixed-order reduction.  Limits: 1 <= m <= 10, n <= 64.
 * The plan is host memory owned by the library until
 * radic_batch_plan_destroy.  Errors: RADIC_EINVAL, RADIC_EUNSUPPORTED
 * (EXACT mode, m > 10), RADIC_ECUDA. */
int radic_batch_plan_create(const int32_t* m, const int32_t* n, const int64_t* offsets, int batch, int mode,
                            const radic_batch_tuning* tuning, radic_batch_plan** plan);
int radic_batch_plan_destroy(radic_batch_plan* plan);

/* Host-only view of the tasks radic_batch_plan_create would make for the
 * same arguments (routing, task split and task order), without a GPU: the
 * Section 5 split of each matrix's ranks into contiguous runs, one run per
 * lane, 32 lanes per task.  tasks (host, capacity rows of
 * RADIC_BATCH_TASK_FIELDS int64): matrix b, tier (RADIC_MODE_MIXED for
 * binary32, _PAIR, _FP64), kind (0: per minor, else the prefix depth D),
 * shared (1: units are heads, the first m-D-1 prefix columns), group (last
 * prefix or head column; 0 per minor), r0 (first unit of lane 0), run (units
 * per lane), lim (end of the unit range: C(v, m-D-1) prefixes, C(u, m-D-2)
 * heads or C(n,m) ranks), then for head-shared tasks the segment of each
 * head's last prefix columns the task covers, vlo and vhi (last columns in
 * [vlo, vhi]); zeros otherwise.  Lane l of a task takes units
 * [r0 + l*run, min(r0 + (l+1)*run, lim)).  *n_tasks receives the total; rows
 * past capacity are not written.  Errors as radic_batch_plan_create's
 * planning (RADIC_EINVAL, RADIC_EUNSUPPORTED). */
#define RADIC_BATCH_TASK_FIELDS 10
int radic_batch_plan_tasks_host(const int32_t* m, const int32_t* n, const int64_t* offsets, int batch, int mode,
                                const radic_batch_tuning* tuning, int64_t* tasks, int64_t capacity,
                                int64_t* n_tasks);

/* Workspace bytes the plan needs (256-byte aligned device memory). */
size_t radic_batch_workspace_bytes(const radic_batch_plan* plan);

/* Writes the first `count` (<= RADIC_BATCH_INFO_COUNT) entries of the plan
 * summary to host array info: [0] tasks binary32, [1] tasks binary64,
 * [2] matrices binary32, [3] matrices binary64, [4] minors binary32,
 * [5] minors binary64, [6] largest persistent grid binary32, [7] same for
 * binary64, [8] tasks pairs, [9] matrices pairs, [10] minors pairs,
 * [11] largest persistent grid pairs, [12] kernel launches per call,
 * [13] m and [14] task path of the dominant kernel (0 per minor, 1 prefix
 * depth 2, 2 prefix depth 3, 3 and 4 the same with head sharing) and [15]
 * its tier (RADIC_MODE_MIXED for binary32, RADIC_MODE_PAIR, or -1 when the
 * plan has no low-tier work).  RADIC_EINVAL on a null pointer or a count
 * outside 0..RADIC_BATCH_INFO_COUNT. */
#define RADIC_BATCH_INFO_COUNT 16
int radic_batch_plan_info(const radic_batch_plan* plan, int64_t* info, int count);

/* Copies the plan's task tables into `workspace` (once per workspace, before
 * the first batched call or graph capture).  Waits for the copies. */
int radic_batch_upload(const radic_batch_plan* plan, void* workspace, size_t workspace_bytes, void* stream);

/* det_R of every matrix of the batch.  A: device, packed matrices of type
 * dtype; out: device, `batch` radic_result; workspace: uploaded with
 * radic_batch_upload.  Calls on the same workspace must not overlap.  The
 * per-group kernels of each phase run concurrently on `stream` and two
 * streams the plan owns (joined back into `stream` before the call's later
 * work); calls with one plan must therefore be issued from one host thread
 * at a time.  Stream capture records the same fork and join. */
int radic_det_batched(const radic_batch_plan* plan, const void* A, int dtype, radic_result* out, void* workspace,
                      size_t workspace_bytes, void* stream);

/* Captures one radic_det_batched call on these buffers into a CUDA graph
 * owned by the library (the one allocation it makes); launch it any number
 * of times with radic_batch_graph_launch, free it with
 * radic_batch_graph_destroy. */
int radic_batch_graph_create(const radic_batch_plan* plan, const void* A, int dtype, radic_result* out,
                             void* workspace, size_t workspace_bytes, radic_batch_graph** graph);
int radic_batch_graph_launch(radic_batch_graph* graph, void* stream);
int radic_batch_graph_destroy(radic_batch_graph* graph);

/* ---- differentiation ------------------------------------------------------ */

/* Workspace bytes of radic_det_backward (0 for unsupported shapes). */
size_t radic_backward_workspace_bytes(int batch, int m, int n);

/* Gradient of sum_b grad_out[b] * det_R(A_b) with respect to every A_b, in
 * binary64.  d det_R / d A[:, J] = (-1)^(r+s) adj(A[:, J])^T for every
 * column sequence J of Eq. (1): each minor's signed cofactors
 * det(M) inv(M)^T are scatter-added into the gradient columns J.  For
 * m >= 3 the cofactors of all minors of one (m-2)-column prefix are summed
 * in closed form from the prefix's partial-pivot LU (block inverse of the
 * minor); for m <= 2, and for prefixes with an exactly zero pivot, from
 * each minor's own LU.  A: device, batch matrices m x n, row-major with
 * leading dimension lda, matrix b at A + b * stride.  grad_out: device,
 * batch values.  grad_A: device, same layout as A, overwritten.  1 <= m <= 8
 * (m > n gives a zero gradient).  Errors: RADIC_EINVAL, RADIC_EUNSUPPORTED
 * (m > 8), RADIC_EWORKSPACE, RADIC_ECUDA. */
int radic_det_backward(const double* A, int batch, int m, int n, int64_t lda, int64_t stride,
                       const double* grad_out, double* grad_A, void* workspace, size_t workspace_bytes,
                       void* stream);

/* radic_det_backward with the arithmetic of the per-prefix eliminations
 * chosen by mode: RADIC_MODE_FP64 (as radic_det_backward) or RADIC_MODE_PAIR
 * (pairs of binary32, about 48 significant bits, on the binary32 pipe; the
 * cofactor sums are still accumulated in binary64).  m <= 2 and singular
 * prefixes use binary64 in both modes.  Same workspace and errors, plus
 * RADIC_EINVAL for another mode. */
int radic_det_backward_mode(const double* A, int batch, int m, int n, int64_t lda, int64_t stride,
                            const double* grad_out, double* grad_A, void* workspace, size_t workspace_bytes,
                            int mode, void* stream);

/* ---- allocation-free variant ------------------------------------------- */

/* Capacity in bytes of the library's own static scratch array. */
#define RADIC_NOALLOC_SCRATCH_BYTES 131072

/* det_R(A) in RADIC_MODE_FP64 without any caller workspace.  The paper has
 * no counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc when they need a determinant -- for example code whose device
 * memory is entirely owned by another allocator or a fixed pool, or a loop
 * that cannot afford the device synchronisation an allocation may cause.
 * Such callers still provide A and `out`, but no workspace.
 *
 * Scratch lives in one file-scope __device__ array of
 * RADIC_NOALLOC_SCRATCH_BYTES bytes inside libradic.so; every GPU that loads
 * the library holds it until the process exits.  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress, with
 * that device current) and caches it; make that first call before any
 * stream capture.  The call itself allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.  The cached address lives as long
 * as the device's primary context: after cudaDeviceReset on a device, do not
 * call radic_det_noalloc on that device again in the same process.
 *
 * All calls on one device share the array and it keeps the last call's
 * contents; each call clears the part that must start at zero.  Calls that
 * overlap on the GPU (other streams, other host threads) race on the array
 * and give wrong results: serialise them.
 *
 * Arguments are those of radic_det with mode RADIC_MODE_FP64.  Errors:
 * as radic_det; RADIC_EWORKSPACE when the launch plan for these options
 * needs more than RADIC_NOALLOC_SCRATCH_BYTES of scratch (the default
 * options fit on GPUs with up to 255 SMs; GB300 has 152); RADIC_ECUDA when the
 * symbol lookup fails. */
int radic_det_noalloc(const void* A, int m, int n, int64_t lda, int dtype,
                      const radic_options* opts, radic_result* out,
                      void* stream);

#ifdef __cplusplus
} /* extern "C" */
#endif

#endif /* RADIC_H */
