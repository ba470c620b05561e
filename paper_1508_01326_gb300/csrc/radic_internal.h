// Internal declarations shared by the host launchers and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/radic.h"

namespace radic {

// dtype / mode / mapping codes (same values as the C enums)
enum : int { kI8 = RADIC_I8, kI32 = RADIC_I32, kF32 = RADIC_F32, kF64 = RADIC_F64 };
enum : int {
  kModeFp64 = RADIC_MODE_FP64,
  kModeMixed = RADIC_MODE_MIXED,
  kModeExact = RADIC_MODE_EXACT,
  kModePair = RADIC_MODE_PAIR
};

constexpr int kMaxM = RADIC_MAX_M;
constexpr int kMaxN = RADIC_MAX_N;
constexpr int kMaxPrimes = RADIC_MAX_PRIMES;
constexpr int kThreadMaxMFp64 = 8;   // thread mapping limits (register budget)
constexpr int kThreadMaxMFp32 = 12;
constexpr int kThreadMaxMModp = 12;
constexpr int kPrefixMaxMFp64 = 10;  // prefix mapping limits
constexpr int kPrefixMaxMFp32 = 12;
constexpr int kPrefixMaxMPair = 10;
constexpr int kPrefixMaxMModp = 12;

// 31-bit primes of the exact mode: the largest primes below 2^31, in
// descending order.  radic_det uses the first RADIC_MAX_PRIMES; the wide
// exact entry point up to RADIC_WIDE_MAX_PRIMES, RADIC_MAX_PRIMES per pass.
constexpr int kWidePrimes = RADIC_WIDE_MAX_PRIMES;
constexpr uint32_t kPrimeTable[kWidePrimes] = {
    2147483647u, 2147483629u, 2147483587u, 2147483579u, 2147483563u, 2147483549u, 2147483543u, 2147483497u,
    2147483489u, 2147483477u, 2147483423u, 2147483399u, 2147483353u, 2147483323u, 2147483269u, 2147483249u,
    2147483237u, 2147483179u, 2147483171u, 2147483137u, 2147483123u, 2147483077u, 2147483069u, 2147483059u,
    2147483053u, 2147483033u, 2147483029u, 2147482951u, 2147482949u, 2147482943u, 2147482937u, 2147482921u};
constexpr uint32_t kPrime0 = kPrimeTable[0], kPrime1 = kPrimeTable[1], kPrime2 = kPrimeTable[2],
                   kPrime3 = kPrimeTable[3];
constexpr uint32_t kPrimes[kMaxPrimes] = {kPrime0, kPrime1, kPrime2, kPrime3};  // host use

// Header at the start of every workspace (zeroed by the launcher).
struct WsHeader {
  unsigned int ticket[4];   // last-block tickets of up to four kernels
  int overflow;             // MIXED: some warp's flag list overflowed
  int status;               // device-side status
  double main_hi, main_lo;  // MIXED: binary32 kernel total (scaled rows), two-sum form
  double main_abs;          // MIXED: its sum of |terms|
  double main_bnd;          // MIXED: its error bound (scaled rows)
  long long flag_total;     // MIXED: flagged minors or prefixes seen by the main kernel
  int escale;               // exponent of the row scaling
  int pad;
  unsigned long long next_task;  // prefix kernels: tasks handed out after each warp's first
};
static_assert(sizeof(WsHeader) <= 256, "header must fit its slot");

// Per-block partial of the floating-point kernels: two-sum total of the
// signed minors, sum of their magnitudes, a count, and the error bound of
// the block's share (scaled rows).
struct FpPartial {
  double hi, lo, abs_sum;
  long long count;
  double bound;
  double pad;
};

// Per-block partial of the binary32-elimination prefix kernel: float-float
// totals of the signed minors and of their magnitudes, stored in the same
// workspace slots as FpPartial.
struct FfPartial {
  float hi, lo, abs_hi, abs_lo;
  long long count;
  double bound;
  long long pad[2];
};
static_assert(sizeof(FfPartial) == sizeof(FpPartial), "partials share their slots");

// Per-group task table of the prefix mapping, passed by value to the kernel.
// Group v holds the prefixes whose last column is v; a warp task covers 32
// runs of run[v] consecutive prefixes of one group.
struct PrefixTable {
  int v_lo, v_hi;                          // groups v_lo .. v_hi
  unsigned long long total_tasks;          // warp tasks over all groups
  unsigned long long count[kMaxN];         // prefixes in group v: C(v, m-D-1)
  unsigned long long run[kMaxN];           // prefixes per lane group in one task
  unsigned long long task_start[kMaxN];    // first task index of group v
  int lanes[kMaxN];                        // lanes sharing one prefix in group v (1..32, power of 2)
  int dynamic;                             // warps draw later tasks from the header counter
};

// Launch plan of one single-matrix call (computed identically by
// radic_workspace_bytes and radic_det).
struct SinglePlan {
  int mode = 0, m = 0, n = 0;
  int mapping = RADIC_MAP_THREAD;  // resolved mapping
  int group = 0;                   // lanes per minor for the group mapping
  PrefixTable ptab{};              // prefix mapping only
  int depth = 2;                   // prefix mapping: trailing columns per leaf
  int threads = 128;
  int blocks = 1;
  unsigned long long ranks_per_task = 64;
  int flag_cap = 32;
  double growth = 64.0;
  unsigned long long total = 0;    // C(n, m)
  unsigned long long tasks = 0;
  size_t smem = 0;
  void* events = nullptr;          // optional cudaEvent_t[2] around the main kernel
  // workspace layout (byte offsets)
  size_t off_partials = 0, off_partials2 = 0, off_flag_count = 0, off_flag_ranks = 0, off_modp = 0;
  int blocks2 = 0;                 // MIXED fix-up kernel grid
  size_t ws_bytes = 0;
};

// Arguments passed by value to every single-matrix kernel.
struct SingleArgs {
  const void* A;
  long long lda;
  int dtype, m, n;
  unsigned long long ranks_per_task;
  unsigned long long total, tasks;
  double growth;
  int flag_cap;
  int flag_prefix;  // 0: flag lists hold ranks; P > 0: they hold P-column prefixes
  int n_warps;      // warps in the main grid (flag lists)
  WsHeader* hdr;
  FpPartial* partials;
  FpPartial* partials2;
  int* flag_count;
  unsigned long long* flag_ranks;
  uint32_t* modp_partials;  // blocks x kMaxPrimes residues
  int prime_base;           // EXACT: first prime of this pass (wide entry point; 0 otherwise)
  uint32_t* wide;           // EXACT wide passes: residues by prime index, then needed, exponent, status
  radic_result* out;
  // terms mode
  unsigned long long q0, count;
  void* terms;
};

unsigned long long binom_host(int n, int k);  // exact C(n, k) for n <= 64 (0 if k > n)
int device_sm_count();

// Launchers (return a RADIC_* code).  When `args.terms` is non-null the
// kernel writes per-rank terms instead of reducing.
int launch_fp64(const SinglePlan& p, const SingleArgs& a, cudaStream_t s);
int launch_mixed(const SinglePlan& p, const SingleArgs& a, cudaStream_t s);
int launch_pair(const SinglePlan& p, const SingleArgs& a, cudaStream_t s);
int launch_modp(const SinglePlan& p, const SingleArgs& a, cudaStream_t s);
// Wide exact result from the residues of the passes (total 0: a zero result).
int launch_wide_crt(const uint32_t* wide, radic_wide_result* out, unsigned long long total, cudaStream_t s);
int launch_unrank(int n, int m, unsigned long long q0, unsigned long long count, uint8_t* cols,
                  int ranks_per_task, cudaStream_t s);

// Occupancy helpers filled in by the arithmetic files.
int blocks_per_sm_fp64(const SinglePlan& p);
int blocks_per_sm_mixed(const SinglePlan& p);
int blocks_per_sm_pair(const SinglePlan& p);
int blocks_per_sm_modp(const SinglePlan& p);
size_t smem_fp64(const SinglePlan& p);
size_t smem_mixed(const SinglePlan& p);
size_t smem_pair(const SinglePlan& p);
size_t smem_modp(const SinglePlan& p);

// Persistent batched kernels per m and task path (argument: the batched
// path's BatchArgs): binary32 tier, pair tier (m >= 3), binary64 tier;
// nullptr outside 1..10 or for a path that does not apply to m.
const void* batch_kernel_f32(int m, int path);
const void* batch_kernel_pair(int m, int path);
const void* batch_kernel_f64(int m, int path);

// Prefix kernel of the EXACT mode for (m, depth) (arguments: SingleArgs,
// PrefixTable), or nullptr.
const void* modp_prefix_kernel(int m, int depth, bool terms);

// Binary64 fix-up kernel of the MIXED and PAIR modes (arguments: SingleArgs,
// int main_blocks, int tier) and its dynamic shared memory.
const void* mixed_fixup_kernel(int m);
size_t mixed_fixup_smem(const SinglePlan& p);

// Cost model of the prefix mapping (instruction units): P = m - D prefix
// columns, D = 2 or 3 trailing columns per leaf; a prefix with k candidate
// columns costs its factorisation m P^2, m + 2 D P per candidate column,
// 8 per column pair (D = 3) and 6 per leaf.  Group v (last prefix column)
// holds C(v, P-1) prefixes with k = n-1-v.
inline double prefix_cost(int m, int D, int k) {
  const int P = m - D;
  double c = (double)m * P * P + (double)k * (m + 2.0 * D * P) + 6.0 * (double)binom_host(k, D);
  if (D == 3) c += 8.0 * (double)binom_host(k, 2);
  return c;
}

// The part of prefix_cost that every lane sharing one prefix repeats: the
// factorisation (depth 3 lanes split the k column reductions as well as the
// leaves; depth 2 does not split prefixes).
inline double prefix_cost_shared(int m, int D, int k) {
  const int P = m - D;
  return (double)m * P * P + (D == 3 ? 0.0 : (double)k * (m + 2.0 * D * P));
}

// Default prefix depth for an m x n matrix.  Depth 3 divides the number of
// prefix factorisations by about (n - m + 3) / (m - 2) but holds three
// Schur-complement entries per candidate column, up to n - m + 3 columns per
// lane, in shared memory, and its leaves grow like C(k, 3).  Measured on
// GB300 in all three floating-point modes (single 5x60, 6x24, 6x40, 7x30,
// 8x24, 8x32, 9x28, 10x20, 10x30, 12x28 matrices; batched m = 3..10 sets
// with n - m <= 20): depth 3 wins while n - m <= 3.5m, from m = 7 on for
// single matrices and from m = 6 on in the batched path.
inline int prefix_auto_depth(int m, int n, bool batched) {
  if (m < (batched ? 6 : 7)) return 2;
  return 2 * (n - m) <= 7 * m ? 3 : 2;
}

inline int ceil_div(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace radic
