// Device side of the batched path: task and argument layouts, per-warp
// staging, the per-task work (per-minor, prefix and head-shared prefix
// tasks) and the persistent kernel template k_batch.  The host plan lives
// in radic_batched.cu; each tier's kernels are instantiated in their own
// file (radic_batched_k32.cu, _kpair.cu, _k64.cu).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "radic_prefix.cuh"

namespace radic {

namespace {

constexpr int kBatchMaxM = 10;      // prefix mapping covers 3..10, per-minor 1..8
constexpr int kBatchThreads = 128;  // four warps per block
constexpr int kKindMinor = 0;       // otherwise: prefix depth (2 or 3)

// Task paths, each compiled into kernels of its own (one path per kernel
// keeps the register allocation and code size of that path alone): 0 per
// minor, 1 prefix depth 2, 2 prefix depth 3, 3 head-shared depth 2, 4
// head-shared depth 3.  A group is one (m, path) pair.
constexpr int kPaths = 5;
constexpr int kGroups = (kBatchMaxM + 1) * kPaths;
__host__ __device__ inline int path_of(int kind, int shared) {
  return kind == kKindMinor ? 0 : (shared ? kind + 1 : kind - 1);
}
__host__ __device__ inline int group_of(int m, int path) { return m * kPaths + path; }
// Head sharing is used for heads of five or more columns (m - D - 1 >= 5).
__host__ __device__ constexpr bool path_valid(int m, int path, bool pairs) {
  return path == 0 ? (m <= 8 && !pairs)
         : path == 1 ? m >= 3
         : path == 2 ? m >= 4
         : path == 3 ? m >= 8
                     : m >= 9;
}
// First-tier routing constants: envelopes of err_bound / sum|terms| measured
// on random matrices (the device check decides per matrix).
constexpr double kBinary32BoundK = 1e-4;
constexpr double kPairBoundK = 2e-11;

struct BatchTask {
  long long offset;         // element offset of the matrix in the packed buffer
  unsigned long long r0;    // first prefix (prefix kind) or first rank (minor kind) of lane 0
  unsigned long long run;   // prefixes or ranks per lane
  unsigned long long lim;   // prefixes in the group, or C(n,m): end of the range
  int b, m, n, v;           // matrix, shape, prefix group
  int kind, tier;           // kKindMinor or the prefix depth; kModeMixed, kModePair or kModeFp64
  int shared;               // prefix kind: units are heads (first m-D-1 columns, v = their last column)
  int vlo, vhi;             // head sharing: last prefix columns in [max(v+1, vlo), vhi] (a segment
                            // of each head's subtree)
  unsigned long long per_unit;  // minors under one unit (prefix, group segment or rank)
};

struct BatchHeader {
  unsigned int queue[3][kGroups];  // work-queue counters: binary32, pair, binary64 kernels of each group
  unsigned int nflag[kGroups];     // binary32 and pair tasks of each group sent to binary64
  int status;
};
constexpr size_t kBatchHeaderBytes = 1024;  // zeroed before every call
static_assert(sizeof(BatchHeader) <= kBatchHeaderBytes, "header slot");

struct BatchArgs {
  const void* A;
  int dtype;
  double tol;               // MIXED: target err_bound / sum|terms| of a matrix
  int flag_base_g[kGroups]; // first entry of each group's region of `flagged`
  int* rerouted;            // per matrix: 1 when its low-tier result missed tol
  int group;                // this launch's group (m, path)
  int queue;                // this launch's queue: 0 binary32, 1 pairs, 2 binary64
  int begin32, end32;       // low-tier launch: its tasks [begin32, end32) of tasks32
  int begin64, end64;       // this group's binary64 tasks
  int flag_base;            // first entry of this group's region of `flagged`
  int n_tasks32;            // slot index of the first binary64 task
  const BatchTask* tasks32; // binary32 and pair tasks (per m: binary32 first)
  const BatchTask* tasks64;
  FpPartial* slots;         // n_tasks32 + n_tasks64
  int* flagged;             // ids of flagged binary32 and pair tasks, per m
  int* escale;              // per matrix
  BatchHeader* hdr;
  double growth;
  int slice_bytes;          // shared memory per warp
};

struct ReduceArgs {
  const int* csr_ptr;       // batch + 1
  const int* csr_idx;       // task ids (binary32 ids first, then binary64 ids)
  const int* tier;          // per matrix: kModeMixed, kModePair or kModeFp64
  const int* rerouted;      // per matrix: redone in binary64 after the bound check
  const int* shape;         // per matrix: m, n
  const FpPartial* slots;
  const int* escale;
  radic_result* out;
  int batch;
};

template <typename T>
struct WarpSlice {
  uint64_t* binom;
  T* As;
  double* As64;  // pairs only: binary64 copy (their prefixes are factored in binary64)
  Rad<T>* colnorm;
  unsigned char* zbuf;
};

// Per-warp slice layout: binom (n+1)(m+1) | As n x cs | (pairs: binary64
// copy n x cs64) | column norms n x 8 bytes | column buffer.
__host__ __device__ inline size_t slice_bytes_before_zbuf(int n, int m, int cs, int elem, bool dbl) {
  size_t off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
  off += ((size_t)n * cs * elem + 31) / 32 * 32;
  if (dbl) off += ((size_t)n * ((m + 1) / 2 * 2) * 8 + 31) / 32 * 32;
  off += ((size_t)n * 8 + 31) / 32 * 32;
  return off;
}
template <typename T>
__device__ WarpSlice<T> carve_slice(unsigned char* base, int n, int m, int cs) {
  constexpr bool kDbl = std::is_same<T, ff>::value;
  WarpSlice<T> w;
  size_t off = 0;
  w.binom = reinterpret_cast<uint64_t*>(base);
  off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
  w.As = reinterpret_cast<T*>(base + off);
  off += ((size_t)n * cs * sizeof(T) + 31) / 32 * 32;
  w.As64 = kDbl ? reinterpret_cast<double*>(base + off) : nullptr;
  if (kDbl) off += ((size_t)n * ((m + 1) / 2 * 2) * 8 + 31) / 32 * 32;
  w.colnorm = reinterpret_cast<Rad<T>*>(base + off);
  off += ((size_t)n * 8 + 31) / 32 * 32;
  w.zbuf = base + off;
  return w;
}

// Warp-cooperative staging of one matrix: binomial table and row-scaled copy.
// Returns the exponent sum of the row scaling in every lane.
template <typename T>
__device__ int stage_warp(const BatchArgs& a, const BatchTask& t, int cs, const WarpSlice<T>& w, bool& exact) {
  const int lane = threadIdx.x & 31;
  const int m = t.m, n = t.n, stride = m + 1;
  for (int idx = lane; idx < (n + 1) * stride; idx += 32) {
    const int vv = idx / stride, k = idx - vv * stride;
    w.binom[idx] = __ldg(&c_binom.v[vv][k]);
  }
  const void* A = a.A;
  int esum = 0;
  bool ex = true;
  for (int i = 0; i < m; ++i) {
    uint32_t h = 0u;
    for (int j = lane; j < n; j += 32) h = max(h, hi_abs(load_elem(A, a.dtype, t.offset + (long long)i * n + j)));
    h = __reduce_max_sync(kFull, h);
    const int e = row_exponent_bits(h);  // the same in every lane
    esum += e;
    for (int j = lane; j < n; j += 32) {
      const double x = scale_pow2(load_elem(A, a.dtype, t.offset + (long long)i * n + j), e);
      const T v = to_elem<T>(x);
      w.As[j * cs + i] = v;
      ex &= as_double(v) == x;
    }
  }
  exact = __all_sync(kFull, ex) != 0;
  for (int idx = lane; idx < (cs - m) * n; idx += 32) {
    const int j = idx / (cs - m), i = m + (idx - j * (cs - m));
    w.As[j * cs + i] = T(0);
  }
  __syncwarp();
  column_norms<T>(w.As, cs, m, n, w.colnorm, lane, 32);
  if constexpr (std::is_same<T, ff>::value) stage_double_copy(w.As, cs, m, n, w.As64, (m + 1) / 2 * 2, lane, 32);
  __syncwarp();
  return esum;
}

// Lane accumulator of a task: float-float for binary32, two-sum for binary64.
template <typename T>
struct TaskAcc;
template <>
struct TaskAcc<double> {
  PrefixAcc<double> p;
  __device__ void minor(double d, float b) {
    p.add_column(d, fabs(d));
    p.add_bound(static_cast<double>(b));
  }
};
template <>
struct TaskAcc<float> {
  PrefixAcc<float> p;
  __device__ void minor(float d, float b) {
    p.add_column(d, fabsf(d));
    p.add_bound(b);
    p.end_prefix();
  }
};

template <>
struct TaskAcc<ff> {  // pair tasks are prefix tasks only
  PrefixAcc<ff> p;
};

template <typename T, int M, int D, bool kFlag>
__device__ bool run_prefix(const BatchArgs& a, const BatchTask& t, const WarpSlice<T>& w, TaskAcc<T>& acc,
                           unsigned long long first, unsigned long long last, float uin) {
  constexpr int CS = ColStride<T, M>::value;
  constexpr int P = M - D;
  constexpr int H = P > 1 ? P - 1 : 1;
  const int lane = threadIdx.x & 31;
  const T thr = static_cast<T>(a.growth);
  bool flagged = false;
  int head[H];
  if constexpr (P > 1) unrank<P - 1>(first < t.lim ? first : 0ull, t.v, w.binom, M + 1, head);
  TermsSink ts{nullptr, 0, 0, 0, 0};
  const ZBuf<T, D> zb(w.zbuf, lane, 32, t.n - M + D);
  for (unsigned long long it = 0; it < t.run; ++it) {
    const bool act = first + it < last;
    int c[P];
#pragma unroll
    for (int j = 0; j < P - 1; ++j) c[j] = head[j];
    c[P - 1] = t.v;
    const bool f =
        prefix_one<T, M, D, CS, false, kFlag>(w.As, w.binom, t.n, t.v, c, zb, thr, act, 0, 1, acc.p, ts, uin, w.As64);
    if (kFlag && act && f) flagged = true;
    acc.p.end_prefix();
    if constexpr (P > 1) {
      if (first + it + 1 < last) successor<P - 1>(head, t.v);
    }
  }
  return flagged;
}

// Head-shared prefix task: each lane takes a run of heads (the first
// H = m-D-1 prefix columns, H-1 of them from {0..u-1} plus u = t.v), factors
// each head once and appends every last column v of the task's segment
// [max(u+1, vlo), vhi] in turn (one elimination step each).  The segment
// bounds the work of one unit (a head's whole subtree can hold over ten
// thousand minors, and the longest unit sets the kernel's critical path);
// its trip count is the same in every lane.
template <typename T, int M, int D, bool kFlag>
__device__ bool run_prefix_heads(const BatchArgs& a, const BatchTask& t, const WarpSlice<T>& w, TaskAcc<T>& acc,
                                 unsigned long long first, unsigned long long last, float uin) {
  constexpr int CS = ColStride<T, M>::value;
  constexpr int P = M - D, H = P - 1;
  static_assert(H >= 2, "head sharing needs a head of two or more columns");
  const int lane = threadIdx.x & 31;
  const int u = t.v;
  const T thr = static_cast<T>(a.growth);
  bool flagged = false;
  int hc[H - 1];  // first H-1 head columns, an (H-1)-subset of {0..u-1}
  unrank<H - 1>(first < t.lim ? first : 0ull, u, w.binom, M + 1, hc);
  TermsSink ts{nullptr, 0, 0, 0, 0};
  const ZBuf<T, D> zb(w.zbuf, lane, 32, t.n - M + D);
  // the head and its extensions are factored in FT: binary64 for pairs,
  // from the binary64 copy (prefix_extend_pair), the element type otherwise
  constexpr bool kPair = std::is_same<T, ff>::value;
  using FT = typename std::conditional<kPair, double, T>::type;
  constexpr int CSF = ColStride<FT, M>::value;
  const FT* AsF;
  if constexpr (kPair) AsF = w.As64;
  else AsF = w.As;
  for (unsigned long long it = 0; it < t.run; ++it) {
    const bool act = first + it < last;
    int c[P];
#pragma unroll
    for (int j = 0; j < H - 1; ++j) c[j] = hc[j];
    c[H - 1] = u;
    FT W1[D + 1][H];
    Rad<T> rW1[D + 1][H], k1[D + 1];
    int idx1[M];
    FT prod1, gmax1;
    bool neg1, bad1;
    Rad<T> rel1;
    {
      int ch[H];
#pragma unroll
      for (int j = 0; j < H; ++j) ch[j] = c[j];
      prefix_factor_b<FT, M, D + 1, CSF, FT>(AsF, ch, W1, rW1, idx1, prod1, gmax1, neg1, rel1, bad1, uin);
    }
    head_kappas<FT, D + 1, H, FT>(W1, rW1, k1, uin);
    for (int v = max(u + 1, t.vlo); v <= t.vhi; ++v) {
      c[P - 1] = v;
      T W[D][P];
      Rad<T> rW[D][P];
      int idx[M];
      T prod, gmax;
      bool neg;
      PrefixErr<Rad<T>> pe;
      if constexpr (kPair) {
        prefix_extend_pair<M, D, CSF>(AsF, v, w.colnorm[v], W1, rW1, k1, idx1, prod1, gmax1, neg1, rel1, bad1, W, rW,
                                      idx, prod, gmax, neg, pe.rel_alpha, pe.bad);
      } else {
        prefix_extend_b<T, M, D, CS>(w.As, v, w.colnorm[v], W1, rW1, k1, idx1, prod1, gmax1, neg1, rel1, bad1, W, rW,
                                     idx, prod, gmax, neg, pe.rel_alpha, pe.bad);
      }
      pe.kappa = 0.0f;
      const bool f = prefix_leaves<T, M, D, CS, false, kFlag>(w.As, w.binom, t.n, v, c, W, idx, prod, gmax, neg, zb,
                                                              thr, act, 0, 1, acc.p, ts, pe, rW, uin);
      if (kFlag && act && f) flagged = true;
      acc.p.end_prefix();
    }
    if (first + it + 1 < last) successor<H - 1>(hc, u);
  }
  return flagged;
}

// Works one task of path PATH in the warp; returns (in every lane) whether
// a lane flagged.
template <typename T, int M, int PATH, bool kFlag>
__device__ bool run_task(const BatchArgs& a, const BatchTask& t, const WarpSlice<T>& w, TaskAcc<T>& acc, float uin) {
  constexpr int CS = ColStride<T, M>::value;
  const int lane = threadIdx.x & 31;
  const T thr = static_cast<T>(a.growth);
  bool flagged = false;
  const unsigned long long first = t.r0 + (unsigned long long)lane * t.run;
  const unsigned long long last = min(first + t.run, t.lim);
  if constexpr (PATH == 3) {
    if constexpr (M >= 5) flagged = run_prefix_heads<T, M, 2, kFlag>(a, t, w, acc, first, last, uin);
  } else if constexpr (PATH == 4) {
    if constexpr (M >= 6) flagged = run_prefix_heads<T, M, 3, kFlag>(a, t, w, acc, first, last, uin);
  } else if constexpr (PATH == 1) {
    if constexpr (M >= 3) flagged = run_prefix<T, M, 2, kFlag>(a, t, w, acc, first, last, uin);
  } else if constexpr (PATH == 2) {
    if constexpr (M >= 4) flagged = run_prefix<T, M, 3, kFlag>(a, t, w, acc, first, last, uin);
  } else {
    // per-minor mapping, m <= 8: binary32 tasks, binary64 tasks of m <= 2 and
    // the binary64 redo of flagged binary32 tasks; never pairs
    if constexpr (!std::is_same<T, ff>::value && M <= 8) {
      int c[M];
      unrank<M>(first < t.lim ? first : 0ull, t.n, w.binom, M + 1, c);
      for (unsigned long long it = 0; it < t.run; ++it) {
        const bool act = first + it < last;
        T mm[M][M];
        gather<T, M, CS>(w.As, c, mm);
        T gmax;
        float b;
        bool bad;
        T det = lu_det_b<T, M>(mm, gmax, b, bad, uin);
        if (sign_negative<M>(c)) det = -det;
        if (act) acc.minor(det, b);
        if (kFlag && act && (mixed_flag<T>(det, gmax, thr) || bad)) flagged = true;
        if (first + it + 1 < last) successor<M>(c, t.n);
      }
    }
  }
  return __any_sync(kFull, flagged);
}

template <typename T>
__device__ __forceinline__ void warp_sum(TaskAcc<T>& acc, Dd& d, double& ab, double& bnd) {
  if constexpr (!std::is_same<T, float>::value) acc.p.finish();  // adds the lane total's own bound
  bnd = static_cast<double>(acc.p.bnd);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) bnd += __shfl_xor_sync(kFull, bnd, off);
  if constexpr (std::is_same<T, float>::value) {
    // float-float tree on the binary32 pipe, widened once
    Ff t = acc.p.tot, ta = acc.p.tot_abs;
    warp_reduce_ff(t, ta);
    d = Dd();
    d.add(static_cast<double>(t.hi));
    d.add(static_cast<double>(t.lo));
    ab = static_cast<double>(ta.hi) + static_cast<double>(ta.lo);
    return;
  }
  d = acc.p.acc;
  ab = acc.p.abs_sum;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Dd o;
    o.hi = __shfl_xor_sync(kFull, d.hi, off);
    o.lo = __shfl_xor_sync(kFull, d.lo, off);
    d.merge(o);
    ab += __shfl_xor_sync(kFull, ab, off);
  }
}

template <typename T, int M, int PATH, bool kFlag>
__device__ void do_task(const BatchArgs& a, const BatchTask& t, unsigned char* slice, int task_id, int slot_id) {
  constexpr int CS = ColStride<T, M>::value;
  const int lane = threadIdx.x & 31;
  TaskAcc<T> acc;
  const WarpSlice<T> w = carve_slice<T>(slice, t.n, M, CS);
  bool exact_in;
  const int esc = stage_warp<T>(a, t, CS, w, exact_in);
  const float uin = exact_in ? 0.0f : static_cast<float>(BoundTraits<T>::u_in);
  const bool flagged = run_task<T, M, PATH, kFlag>(a, t, w, acc, uin);
  Dd d;
  double ab, bnd;
  warp_sum<T>(acc, d, ab, bnd);
  __syncwarp();
  if (lane == 0) {
    a.escale[t.b] = esc;
    if (kFlag && flagged) {
      const unsigned int pos = atomicAdd(&a.hdr->nflag[a.group], 1u);
      a.flagged[a.flag_base + pos] = task_id;
      a.slots[slot_id] = FpPartial{0.0, 0.0, 0.0, -1ll, 0.0, 0.0};  // marked: redone in binary64
    } else {
      // count: minors of a binary32 or pair task recomputed here in binary64
      long long redone = 0;
      if (!kFlag && t.tier != kModeFp64) {
        const unsigned long long units = min(32ull * t.run, t.lim - t.r0);
        redone = (long long)(units * t.per_unit);
      }
      a.slots[slot_id] = FpPartial{d.hi, d.lo, ab, redone, bnd, 0.0};
    }
  }
}

// Persistent kernel of one tier and one group (m, path).  Binary32 (T =
// float) and pair (T = ff) tiers: queue over this group's tasks of that tier.
// Binary64 tier: queue over this group's binary64 tasks, then over its
// binary32 and pair tasks that were flagged or rerouted (their slots are
// overwritten with binary64 sums).
template <typename T, bool kMixedTier, int M, int PATH>
__global__ void __launch_bounds__(kBatchThreads) k_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* slice = smem_raw + (size_t)warp * a.slice_bytes;
  const int own = kMixedTier ? a.end32 - a.begin32 : a.end64 - a.begin64;
  const int total = kMixedTier ? own : own + (int)__ldcg(&a.hdr->nflag[a.group]);
  unsigned int* counter = &a.hdr->queue[a.queue][a.group];
  for (;;) {
    unsigned int i = 0;
    if (lane == 0) i = atomicAdd(counter, 1u);
    i = __shfl_sync(kFull, i, 0);
    if ((int)i >= total) break;
    if (kMixedTier) {
      const int id = a.begin32 + (int)i;
      do_task<T, M, PATH, true>(a, a.tasks32[id], slice, id, id);
    } else if ((int)i < own) {
      const int id = a.begin64 + (int)i;
      do_task<T, M, PATH, false>(a, a.tasks64[id], slice, id, a.n_tasks32 + id);
    } else {
      const int id = __ldcg(&a.flagged[a.flag_base + (int)i - own]);
      BatchTask t = a.tasks32[id];
      do_task<T, M, PATH, false>(a, t, slice, id, id);
    }
  }
}

// A-posteriori check of the routing (MIXED): one warp per matrix of a low
// tier adds the error bounds and magnitude sums of its tasks that were not
// already sent to binary64; when margin * bound exceeds tol * sum|terms| the
// matrix's remaining low-tier tasks are appended to the binary64 redo lists,
// so that its result comes from binary64 instead.  The routing constants only
// choose the first tier; this check decides.
__global__ void __launch_bounds__(128) k_batch_check(BatchArgs a, ReduceArgs r) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= r.batch || r.tier[b] == kModeFp64) return;
  const int p0 = r.csr_ptr[b], p1 = r.csr_ptr[b + 1];
  double ab = 0.0, bnd = 0.0;
  int kept = 0;
  for (int p = p0 + lane; p < p1; p += 32) {
    const int id = r.csr_idx[p];
    if (id >= a.n_tasks32) continue;
    const FpPartial s = r.slots[id];
    if (s.count < 0) continue;
    ab += s.abs_sum;
    bnd += s.bound;
    ++kept;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ab += __shfl_xor_sync(kFull, ab, off);
    bnd += __shfl_xor_sync(kFull, bnd, off);
  }
  // a matrix none of whose low-tier tasks survived is computed in binary64
  // already (its flagged tasks are queued) and is reported as such
  if (__ballot_sync(kFull, kept > 0) == 0u) {
    if (lane == 0 && p1 > p0) a.rerouted[b] = 1;
    return;
  }
  const bool fail = !(kBoundMargin * bnd <= a.tol * ab);
  if (!fail) return;
  if (lane == 0) a.rerouted[b] = 1;
  for (int p = p0 + lane; p < p1; p += 32) {
    const int id = r.csr_idx[p];
    if (id >= a.n_tasks32 || r.slots[id].count < 0) continue;
    const BatchTask& t = a.tasks32[id];
    const int g = group_of(t.m, path_of(t.kind, t.shared));
    const unsigned int pos = atomicAdd(&a.hdr->nflag[g], 1u);
    a.flagged[a.flag_base_g[g] + pos] = id;
  }
}

// One warp per matrix: adds its slots in task order and writes the result.
__global__ void __launch_bounds__(128) k_batch_reduce(ReduceArgs r) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= r.batch) return;
  const int p0 = r.csr_ptr[b], p1 = r.csr_ptr[b + 1];
  Dd d;
  double ab = 0.0, bnd = 0.0;
  long long redone = 0;
  for (int p = p0 + lane; p < p1; p += 32) {
    const FpPartial s = r.slots[r.csr_idx[p]];
    Dd o;
    o.hi = s.hi;
    o.lo = s.lo;
    d.merge(o);
    ab += s.abs_sum;
    bnd += s.bound;
    redone += s.count;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Dd o;
    o.hi = __shfl_xor_sync(kFull, d.hi, off);
    o.lo = __shfl_xor_sync(kFull, d.lo, off);
    d.merge(o);
    ab += __shfl_xor_sync(kFull, ab, off);
    bnd += __shfl_xor_sync(kFull, bnd, off);
    redone += __shfl_xor_sync(kFull, redone, off);
  }
  if (lane == 0) {
    const int m = r.shape[2 * b], n = r.shape[2 * b + 1];
    const unsigned long long total = (m <= n) ? c_binom.v[n][m] : 0ull;
    const int tier = r.rerouted[b] ? kModeFp64 : r.tier[b];
    if (total == 0) {
      Dd z;
      write_fp_result(&r.out[b], z, 0.0, 0.0, 0, m, 0, 0, RADIC_OK, r.tier[b]);
    } else {
      write_fp_result(&r.out[b], d, ab, bnd, r.escale[b], m, total, redone, RADIC_OK, tier);
    }
  }
}

template <typename T, bool kMixed, int M, int PATH>
const void* batch_kernel_mp() {
  if constexpr (!path_valid(M, PATH, std::is_same<T, ff>::value)) return nullptr;
  else return reinterpret_cast<const void*>(&k_batch<T, kMixed, M, PATH>);
}

template <typename T, bool kMixed, int M>
const void* batch_kernel_m(int path) {
  switch (path) {
    case 0: return batch_kernel_mp<T, kMixed, M, 0>();
    case 1: return batch_kernel_mp<T, kMixed, M, 1>();
    case 2: return batch_kernel_mp<T, kMixed, M, 2>();
    case 3: return batch_kernel_mp<T, kMixed, M, 3>();
    case 4: return batch_kernel_mp<T, kMixed, M, 4>();
    default: return nullptr;
  }
}

// Kernel of one tier for group (m, path), or nullptr where the path does not
// apply (path_valid).
template <typename T, bool kMixed>
const void* batch_kernel(int m, int path) {
  switch (m) {
    case 1: return batch_kernel_m<T, kMixed, 1>(path);
    case 2: return batch_kernel_m<T, kMixed, 2>(path);
    case 3: return batch_kernel_m<T, kMixed, 3>(path);
    case 4: return batch_kernel_m<T, kMixed, 4>(path);
    case 5: return batch_kernel_m<T, kMixed, 5>(path);
    case 6: return batch_kernel_m<T, kMixed, 6>(path);
    case 7: return batch_kernel_m<T, kMixed, 7>(path);
    case 8: return batch_kernel_m<T, kMixed, 8>(path);
    case 9: return batch_kernel_m<T, kMixed, 9>(path);
    case 10: return batch_kernel_m<T, kMixed, 10>(path);
    default: return nullptr;
  }
}

}  // namespace
}  // namespace radic
