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
constexpr double kBinary32ErrorK = 2.5e-6;  // error model constants of the router
constexpr double kPairErrorK = 1e-11;

struct BatchTask {
  long long offset;         // element offset of the matrix in the packed buffer
  unsigned long long r0;    // first prefix (prefix kind) or first rank (minor kind) of lane 0
  unsigned long long run;   // prefixes or ranks per lane
  unsigned long long lim;   // prefixes in the group, or C(n,m): end of the range
  int b, m, n, v;           // matrix, shape, prefix group
  int kind, tier;           // kKindMinor or the prefix depth; kModeMixed, kModePair or kModeFp64
  int shared;               // prefix kind: units are heads (first m-D-1 columns, v = their last column)
};

struct BatchHeader {
  unsigned int q32[kBatchMaxM + 1];    // work-queue counters, binary32 tier, per m
  unsigned int qpair[kBatchMaxM + 1];  // work-queue counters, pair tier, per m
  unsigned int q64[kBatchMaxM + 1];    // work-queue counters, binary64 tier, per m
  unsigned int nflag[kBatchMaxM + 1];  // binary32 and pair tasks of each m sent to binary64
  int status;
};
static_assert(sizeof(BatchHeader) <= 256, "header slot");

struct BatchArgs {
  const void* A;
  int dtype;
  int begin32, end32;       // low-tier launch: its tasks [begin32, end32) of tasks32
  int begin64, end64;       // this m's binary64 tasks
  int flag_base;            // first entry of this m's region of `flagged`
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
  unsigned char* zbuf;
};

// Per-warp slice layout: binom (n+1)(m+1) | As n x cs | column buffer.
template <typename T>
__device__ WarpSlice<T> carve_slice(unsigned char* base, int n, int m, int cs) {
  WarpSlice<T> w;
  size_t off = 0;
  w.binom = reinterpret_cast<uint64_t*>(base);
  off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
  w.As = reinterpret_cast<T*>(base + off);
  off += ((size_t)n * cs * sizeof(T) + 31) / 32 * 32;
  w.zbuf = base + off;
  return w;
}

// Warp-cooperative staging of one matrix: binomial table and row-scaled copy.
// Returns the exponent sum of the row scaling in every lane.
template <typename T>
__device__ int stage_warp(const BatchArgs& a, const BatchTask& t, int cs, const WarpSlice<T>& w) {
  const int lane = threadIdx.x & 31;
  const int m = t.m, n = t.n, stride = m + 1;
  for (int idx = lane; idx < (n + 1) * stride; idx += 32) {
    const int vv = idx / stride, k = idx - vv * stride;
    w.binom[idx] = __ldg(&c_binom.v[vv][k]);
  }
  const void* A = a.A;
  int esum = 0;
  for (int i = 0; i < m; ++i) {
    uint32_t h = 0u;
    for (int j = lane; j < n; j += 32) h = max(h, hi_abs(load_elem(A, a.dtype, t.offset + (long long)i * n + j)));
    h = __reduce_max_sync(kFull, h);
    const int e = row_exponent_bits(h);  // the same in every lane
    esum += e;
    for (int j = lane; j < n; j += 32)
      w.As[j * cs + i] = to_elem<T>(scale_pow2(load_elem(A, a.dtype, t.offset + (long long)i * n + j), e));
  }
  for (int idx = lane; idx < (cs - m) * n; idx += 32) {
    const int j = idx / (cs - m), i = m + (idx - j * (cs - m));
    w.As[j * cs + i] = T(0);
  }
  __syncwarp();
  return esum;
}

// Lane accumulator of a task: float-float for binary32, two-sum for binary64.
template <typename T>
struct TaskAcc;
template <>
struct TaskAcc<double> {
  PrefixAcc<double> p;
  __device__ void minor(double d) { p.add_column(d, fabs(d)); }
};
template <>
struct TaskAcc<float> {
  PrefixAcc<float> p;
  __device__ void minor(float d) {
    p.add_column(d, fabsf(d));
    p.end_prefix();
  }
};

template <>
struct TaskAcc<ff> {  // pair tasks are prefix tasks only
  PrefixAcc<ff> p;
};

template <typename T, int M, int D, bool kFlag>
__device__ bool run_prefix(const BatchArgs& a, const BatchTask& t, const WarpSlice<T>& w, TaskAcc<T>& acc,
                           unsigned long long first, unsigned long long last) {
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
    const bool f = prefix_one<T, M, D, CS, false>(w.As, w.binom, t.n, t.v, c, zb, thr, act, 0, 1, acc.p, ts);
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
// each head once and appends every last column v = u+1 .. n-1-D in turn.
template <typename T, int M, int D, bool kFlag>
__device__ bool run_prefix_heads(const BatchArgs& a, const BatchTask& t, const WarpSlice<T>& w, TaskAcc<T>& acc,
                                 unsigned long long first, unsigned long long last) {
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
  for (unsigned long long it = 0; it < t.run; ++it) {
    const bool act = first + it < last;
    int c[P];
#pragma unroll
    for (int j = 0; j < H - 1; ++j) c[j] = hc[j];
    c[H - 1] = u;
    T W1[D + 1][H];
    int idx1[M];
    T prod1, gmax1;
    bool neg1;
    {
      int ch[H];
#pragma unroll
      for (int j = 0; j < H; ++j) ch[j] = c[j];
      prefix_factor<T, M, D + 1, CS>(w.As, ch, W1, idx1, prod1, gmax1, neg1);
    }
    for (int v = u + 1; v <= t.n - 1 - D; ++v) {
      c[P - 1] = v;
      T W[D][P];
      int idx[M];
      T prod, gmax;
      bool neg;
      prefix_extend<T, M, D, CS>(w.As, v, W1, idx1, prod1, gmax1, neg1, W, idx, prod, gmax, neg);
      const bool f = prefix_leaves<T, M, D, CS, false>(w.As, w.binom, t.n, v, c, W, idx, prod, gmax, neg, zb, thr, act,
                                                       0, 1, acc.p, ts);
      if (kFlag && act && f) flagged = true;
      acc.p.end_prefix();
    }
    if (first + it + 1 < last) successor<H - 1>(hc, u);
  }
  return flagged;
}

// Works one task in the warp; returns (in every lane) whether a lane flagged.
template <typename T, int M, bool kFlag>
__device__ bool run_task(const BatchArgs& a, const BatchTask& t, const WarpSlice<T>& w, TaskAcc<T>& acc) {
  constexpr int CS = ColStride<T, M>::value;
  const int lane = threadIdx.x & 31;
  const T thr = static_cast<T>(a.growth);
  bool flagged = false;
  const unsigned long long first = t.r0 + (unsigned long long)lane * t.run;
  const unsigned long long last = min(first + t.run, t.lim);
  if (t.kind == 2 && t.shared) {
    if constexpr (M >= 5) flagged = run_prefix_heads<T, M, 2, kFlag>(a, t, w, acc, first, last);
  } else if (t.kind == 3 && t.shared) {
    if constexpr (M >= 6) flagged = run_prefix_heads<T, M, 3, kFlag>(a, t, w, acc, first, last);
  } else if (t.kind == 2) {
    if constexpr (M >= 3) flagged = run_prefix<T, M, 2, kFlag>(a, t, w, acc, first, last);
  } else if (t.kind == 3) {
    if constexpr (M >= 4) flagged = run_prefix<T, M, 3, kFlag>(a, t, w, acc, first, last);
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
        T det = lu_det<T, M>(mm, gmax);
        if (sign_negative<M>(c)) det = -det;
        if (act) acc.minor(det);
        if (kFlag && act && mixed_flag<T>(det, gmax, thr)) flagged = true;
        if (first + it + 1 < last) successor<M>(c, t.n);
      }
    }
  }
  return __any_sync(kFull, flagged);
}

template <typename T>
__device__ __forceinline__ void warp_sum(TaskAcc<T>& acc, Dd& d, double& ab) {
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
  acc.p.finish();
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

template <typename T, int M, bool kFlag>
__device__ void do_task(const BatchArgs& a, const BatchTask& t, unsigned char* slice, int task_id, int slot_id) {
  constexpr int CS = ColStride<T, M>::value;
  const int lane = threadIdx.x & 31;
  TaskAcc<T> acc;
  const WarpSlice<T> w = carve_slice<T>(slice, t.n, M, CS);
  const int esc = stage_warp<T>(a, t, CS, w);
  const bool flagged = run_task<T, M, kFlag>(a, t, w, acc);
  Dd d;
  double ab;
  warp_sum<T>(acc, d, ab);
  __syncwarp();
  if (lane == 0) {
    a.escale[t.b] = esc;
    if (kFlag && flagged) {
      const unsigned int pos = atomicAdd(&a.hdr->nflag[M], 1u);
      a.flagged[a.flag_base + pos] = task_id;
    } else {
      // count: minors of a binary32 or pair task recomputed here in binary64
      long long redone = 0;
      if (!kFlag && t.tier != kModeFp64) {
        const unsigned long long units = min(32ull * t.run, t.lim - t.r0);
        const int D = t.kind;
        redone = (long long)(D == kKindMinor ? units
                             : t.shared     ? units * c_binom.v[t.n - 1 - t.v][D + 1]
                                            : units * c_binom.v[t.n - 1 - t.v][D]);
      }
      a.slots[slot_id] = FpPartial{d.hi, d.lo, ab, redone};
    }
  }
}

// Persistent kernel of one tier and one m.  Binary32 (T = float) and pair
// (T = ff) tiers: queue over this m's tasks of that tier.  Binary64 tier:
// queue over this m's binary64 tasks, then over this m's binary32 and pair
// tasks that were flagged (their slots are overwritten with binary64 sums).
template <typename T, bool kMixedTier, int M>
__global__ void __launch_bounds__(kBatchThreads) k_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* slice = smem_raw + (size_t)warp * a.slice_bytes;
  const int own = kMixedTier ? a.end32 - a.begin32 : a.end64 - a.begin64;
  const int total = kMixedTier ? own : own + (int)__ldcg(&a.hdr->nflag[M]);
  unsigned int* counter =
      kMixedTier ? (std::is_same<T, ff>::value ? &a.hdr->qpair[M] : &a.hdr->q32[M]) : &a.hdr->q64[M];
  for (;;) {
    unsigned int i = 0;
    if (lane == 0) i = atomicAdd(counter, 1u);
    i = __shfl_sync(kFull, i, 0);
    if ((int)i >= total) break;
    if (kMixedTier) {
      const int id = a.begin32 + (int)i;
      do_task<T, M, true>(a, a.tasks32[id], slice, id, id);
    } else if ((int)i < own) {
      const int id = a.begin64 + (int)i;
      do_task<T, M, false>(a, a.tasks64[id], slice, id, a.n_tasks32 + id);
    } else {
      const int id = __ldcg(&a.flagged[a.flag_base + (int)i - own]);
      BatchTask t = a.tasks32[id];
      do_task<T, M, false>(a, t, slice, id, id);
    }
  }
}

// One warp per matrix: adds its slots in task order and writes the result.
__global__ void __launch_bounds__(128) k_batch_reduce(ReduceArgs r) {
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= r.batch) return;
  const int p0 = r.csr_ptr[b], p1 = r.csr_ptr[b + 1];
  Dd d;
  double ab = 0.0;
  long long redone = 0;
  for (int p = p0 + lane; p < p1; p += 32) {
    const FpPartial s = r.slots[r.csr_idx[p]];
    Dd o;
    o.hi = s.hi;
    o.lo = s.lo;
    d.merge(o);
    ab += s.abs_sum;
    redone += s.count;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Dd o;
    o.hi = __shfl_xor_sync(kFull, d.hi, off);
    o.lo = __shfl_xor_sync(kFull, d.lo, off);
    d.merge(o);
    ab += __shfl_xor_sync(kFull, ab, off);
    redone += __shfl_xor_sync(kFull, redone, off);
  }
  if (lane == 0) {
    const int m = r.shape[2 * b], n = r.shape[2 * b + 1];
    const unsigned long long total = (m <= n) ? c_binom.v[n][m] : 0ull;
    if (total == 0) {
      Dd z;
      write_fp_result(&r.out[b], z, 0.0, 0, m, 0, 0, RADIC_OK, r.tier[b]);
    } else {
      write_fp_result(&r.out[b], d, ab, r.escale[b], m, total, redone, RADIC_OK, r.tier[b]);
    }
  }
}

template <typename T, bool kMixed, int M>
const void* batch_kernel_m() {
  if constexpr (std::is_same<T, ff>::value && M < 3) return nullptr;  // pairs: prefix tasks, m >= 3
  else return reinterpret_cast<const void*>(&k_batch<T, kMixed, M>);
}

template <typename T, bool kMixed>
const void* batch_kernel(int m) {
  switch (m) {
    case 1: return batch_kernel_m<T, kMixed, 1>();
    case 2: return batch_kernel_m<T, kMixed, 2>();
    case 3: return batch_kernel_m<T, kMixed, 3>();
    case 4: return batch_kernel_m<T, kMixed, 4>();
    case 5: return batch_kernel_m<T, kMixed, 5>();
    case 6: return batch_kernel_m<T, kMixed, 6>();
    case 7: return batch_kernel_m<T, kMixed, 7>();
    case 8: return batch_kernel_m<T, kMixed, 8>();
    case 9: return batch_kernel_m<T, kMixed, 9>();
    case 10: return batch_kernel_m<T, kMixed, 10>();
    default: return nullptr;
  }
}

}  // namespace
}  // namespace radic
