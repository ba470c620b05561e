// C-ABI entry points of the single-matrix path: argument validation, launch
// planning (mapping, grid, workspace layout) and launches.  Validation happens
// entirely on the host before anything is enqueued.
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>

#include "radic_device.cuh"

namespace radic {

unsigned long long binom_host(int n, int k) {
  if (k < 0 || k > n) return 0ull;
  unsigned long long c[kMaxN + 1] = {1ull};
  for (int v = 1; v <= n; ++v)
    for (int j = (v < k ? v : k); j >= 1; --j) c[j] += c[j - 1];
  return c[k];
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

namespace {

bool valid_dtype(int d) { return d == kI8 || d == kI32 || d == kF32 || d == kF64; }
bool valid_mode(int md) { return md == kModeFp64 || md == kModeMixed || md == kModeExact || md == kModePair; }

int thread_limit(int mode) {
  if (mode == kModePair) return 0;  // prefix mapping only
  return mode == kModeFp64 ? kThreadMaxMFp64 : (mode == kModeMixed ? kThreadMaxMFp32 : kThreadMaxMModp);
}

int blocks_per_sm(const SinglePlan& p) {
  switch (p.mode) {
    case kModeFp64: return blocks_per_sm_fp64(p);
    case kModeMixed: return blocks_per_sm_mixed(p);
    case kModePair: return blocks_per_sm_pair(p);
    default: return blocks_per_sm_modp(p);
  }
}

size_t smem_of(const SinglePlan& p) {
  switch (p.mode) {
    case kModeFp64: return smem_fp64(p);
    case kModeMixed: return smem_mixed(p);
    case kModePair: return smem_pair(p);
    default: return smem_modp(p);
  }
}

void layout_workspace(SinglePlan& pl);


int plan_prefix(SinglePlan pl, const radic_options& d, int sms, int per_sm, unsigned long long units,
                SinglePlan* out) {
  const int m = pl.m, n = pl.n, D = pl.depth, P = m - D;
  PrefixTable& t = pl.ptab;
  t.v_lo = P - 1;
  t.v_hi = n - 1 - D;
  t.dynamic = d.deterministic ? 0 : 1;
  double total_cost = 0.0;
  double cost[kMaxN] = {0};
  for (int v = t.v_lo; v <= t.v_hi; ++v) {
    t.count[v] = binom_host(v, P - 1);
    cost[v] = prefix_cost(m, D, n - 1 - v);
    total_cost += cost[v] * (double)t.count[v];
  }
  const unsigned long long lanes = (unsigned long long)sms * per_sm * pl.threads;
  const double per_lane = total_cost / (double)lanes / 4.0;  // about four tasks per warp
  unsigned long long start = 0;
  for (int v = t.v_lo; v <= t.v_hi; ++v) {
    // Lanes per prefix: a prefix with many candidate columns costs far more
    // than a lane's share of the launch (the leaves grow like C(k, D)), so
    // its column reductions and leaves are split over LP lanes of the warp,
    // each of which repeats the factorisation.  LP is the smallest power of
    // two that brings a lane's cost down to a target near the mean per-lane
    // work.
    int lp = 1;
    if (d.lanes_per_prefix > 0) {
      lp = d.lanes_per_prefix;
    } else if (D == 3) {
      // Only depth 3 (its leaves grow like C(k, 3); splitting depth-2
      // prefixes measured slower).  Target with binary32 elimination: 1.4
      // times the mean lane work when that is large, three times when the
      // launch is small and the repeated factorisations would dominate.
      // Binary64 and pair leaves keep their pipes busy, so there the balance
      // of the warps' shares matters more than the repeated work: the mean
      // itself.  (Measured on the shapes of prefix_auto_depth, warps drawing
      // tasks from the shared counter.)
      const double mean = 4.0 * per_lane;
      const double tf = (pl.mode == kModeMixed) ? (mean >= 1000.0 ? 1.4 : 3.0) : 1.0;
      const double target = tf * mean;
      const double red = prefix_cost_shared(m, D, n - 1 - v), split = cost[v] - red;
      while (lp < 32 && red + split / lp > target) lp *= 2;
    }
    const unsigned long long groups = 32 / lp;  // lane groups per warp
    double r = per_lane * lp / cost[v];
    unsigned long long run = r < 1.0 ? 1ull : (unsigned long long)r;
    if (d.ranks_per_task > 0) run = (unsigned long long)d.ranks_per_task;
    const unsigned long long maxrun = (t.count[v] + groups - 1) / groups;
    if (run > maxrun) run = maxrun > 0 ? maxrun : 1;
    t.lanes[v] = lp;
    t.run[v] = run;
    t.task_start[v] = start;
    start += (t.count[v] + groups * run - 1) / (groups * run);
  }
  if (t.v_hi + 1 < kMaxN) t.task_start[t.v_hi + 1] = start;
  if (t.v_hi < t.v_lo) start = 0;
  t.total_tasks = start;
  const unsigned long long warps_per_block = pl.threads / 32;
  const unsigned long long need = (start + warps_per_block - 1) / warps_per_block;
  const unsigned long long cap = (unsigned long long)sms * per_sm;
  unsigned long long blocks = need < cap ? need : cap;
  if (d.blocks > 0) blocks = (unsigned long long)d.blocks;
  if (blocks < 1) blocks = 1;
  if (blocks > (1ull << 20)) return RADIC_EINVAL;
  pl.blocks = (int)blocks;
  pl.blocks2 = sms;
  // per-minor split used by the binary64 fall-back pass of the mixed mode
  const unsigned long long procs = (unsigned long long)pl.blocks2 * 128;
  pl.ranks_per_task = (units + procs - 1) / procs;
  if (pl.ranks_per_task < 1) pl.ranks_per_task = 1;
  pl.tasks = (units + pl.ranks_per_task - 1) / pl.ranks_per_task;
  layout_workspace(pl);
  *out = pl;
  return RADIC_OK;
}

// Plans a launch over `units` ranks (C(n,m) for radic_det, `count` for
// radic_terms).  Returns a RADIC_* code.
int make_plan_uncached(int m, int n, int mode, const radic_options* o, unsigned long long units, SinglePlan* p,
                       int sms_given = 0, int per_sm_given = 0);

// Plans are pure functions of (device, shape, mode, options, units); repeated
// calls on one shape (the common case when serving) reuse the plan instead of
// repeating the occupancy queries.  The kernel_events pointer is not part of
// the plan and is filled in per call.
int make_plan(int m, int n, int mode, const radic_options* o, unsigned long long units, SinglePlan* p) {
  int dev = 0;
  // without a device the uncached planner still reports argument errors first
  if (cudaGetDevice(&dev) != cudaSuccess) return make_plan_uncached(m, n, mode, o, units, p);
  radic_options key_opts;
  std::memset(&key_opts, 0, sizeof(key_opts));
  if (o) key_opts = *o;
  key_opts.kernel_events = nullptr;
  const int head[4] = {dev, m, n, mode};
  std::string key(reinterpret_cast<const char*>(head), sizeof(head));
  key.append(reinterpret_cast<const char*>(&units), sizeof(units));
  key.append(reinterpret_cast<const char*>(&key_opts), sizeof(key_opts));
  static std::mutex mu;
  static std::unordered_map<std::string, SinglePlan> cache;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *p = it->second;
      p->events = o ? o->kernel_events : nullptr;
      return RADIC_OK;
    }
  }
  const int rc = make_plan_uncached(m, n, mode, o, units, p);
  if (rc == RADIC_OK) {
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() >= 4096) cache.clear();
    cache.emplace(key, *p);
  }
  return rc;
}

// sms_given / per_sm_given > 0 replace the device's SM count and the
// occupancy query (host-only planning).
int make_plan_uncached(int m, int n, int mode, const radic_options* o, unsigned long long units, SinglePlan* p,
                       int sms_given, int per_sm_given) {
  if (m < 1 || m > kMaxM || n < 1 || n > kMaxN || !valid_mode(mode)) return RADIC_EINVAL;
  radic_options d;
  std::memset(&d, 0, sizeof(d));
  if (o) d = *o;
  SinglePlan pl;
  pl.mode = mode;
  pl.m = m;
  pl.n = n;
  pl.total = (m <= n) ? binom_host(n, m) : 0ull;
  const int auto_limit = (mode == kModeExact) ? kThreadMaxMModp : 8;
  const int prefix_limit = (mode == kModeFp64)    ? kPrefixMaxMFp64
                           : (mode == kModeMixed) ? kPrefixMaxMFp32
                           : (mode == kModePair)  ? kPrefixMaxMPair
                                                  : kPrefixMaxMModp;
  int mapping = d.mapping;
  if (mapping == RADIC_MAP_AUTO) {
    if (m >= 3 && m <= prefix_limit && m <= n) mapping = RADIC_MAP_PREFIX;
    else mapping = (m <= auto_limit ? RADIC_MAP_THREAD : RADIC_MAP_GROUP);
  }
  if (mapping != RADIC_MAP_THREAD && mapping != RADIC_MAP_GROUP && mapping != RADIC_MAP_PREFIX) return RADIC_EINVAL;
  if (mode == kModePair && mapping != RADIC_MAP_PREFIX) return RADIC_EUNSUPPORTED;
  if (mapping == RADIC_MAP_THREAD && m > thread_limit(mode)) return RADIC_EUNSUPPORTED;
  if (mapping == RADIC_MAP_PREFIX && (m < 3 || m > prefix_limit || m > n)) return RADIC_EUNSUPPORTED;
  pl.mapping = mapping;
  if (mapping == RADIC_MAP_PREFIX) {
    if (d.prefix_depth != 0 && d.prefix_depth != 2 && d.prefix_depth != 3) return RADIC_EINVAL;
    const int lp = d.lanes_per_prefix;
    if (lp < 0 || lp > 32 || (lp & (lp - 1)) != 0) return RADIC_EINVAL;
    if (d.prefix_depth == 3 && m < 4) return RADIC_EUNSUPPORTED;
    pl.depth = d.prefix_depth ? d.prefix_depth : prefix_auto_depth(m, n, false);
  }
  if (mapping == RADIC_MAP_GROUP) {
    const int gw = d.group_width ? d.group_width : (m <= 16 ? 16 : 32);
    if ((gw != 16 && gw != 32) || gw < m) return RADIC_EINVAL;
    pl.group = gw;
  }
  const int max_threads = (mode == kModeExact || mapping == RADIC_MAP_PREFIX) ? 128 : 256;
  pl.threads = d.threads_per_block ? d.threads_per_block : 128;
  if (pl.threads < 32 || pl.threads > max_threads || pl.threads % 32) return RADIC_EINVAL;
  if (d.ranks_per_task < 0 || d.ranks_per_task > (1 << 30)) return RADIC_EINVAL;
  pl.flag_cap = d.flag_capacity ? d.flag_capacity : 32;
  if (pl.flag_cap < 1 || pl.flag_cap > (1 << 16)) return RADIC_EINVAL;
  pl.growth = d.growth_threshold > 0.0 ? d.growth_threshold : 64.0;
  pl.events = d.kernel_events;
  pl.smem = smem_of(pl);

  const int sms = sms_given > 0 ? sms_given : device_sm_count();
  const int per_sm = per_sm_given > 0 ? per_sm_given : blocks_per_sm(pl);
  if (sms <= 0) return RADIC_ECUDA;
  if (per_sm <= 0) return RADIC_EUNSUPPORTED;
  // Work split of Section 5: K processors (threads, or lane groups) each take
  // one contiguous run of about C(n,m)/K ranks.  K is the number of resident
  // processors of a full-occupancy grid, so every processor gets one task and
  // no SM waits on a tail; an explicit ranks_per_task overrides the run length.
  const unsigned long long cap = (unsigned long long)sms * per_sm;
  if (mapping == RADIC_MAP_PREFIX) return plan_prefix(pl, d, sms, per_sm, units, p);
  const unsigned long long per_block =
      (mapping == RADIC_MAP_THREAD) ? (unsigned long long)pl.threads : (unsigned long long)(pl.threads / pl.group);
  unsigned long long L = (unsigned long long)d.ranks_per_task;
  if (L == 0) {
    const unsigned long long procs = cap * per_block;
    L = (units + procs - 1) / procs;
    if (L < 1) L = 1;
  }
  pl.ranks_per_task = L;
  pl.tasks = (units + L - 1) / L;
  const unsigned long long need = (pl.tasks + per_block - 1) / per_block;
  unsigned long long blocks = need < cap ? need : cap;
  if (d.blocks > 0) blocks = (unsigned long long)d.blocks;
  if (blocks < 1) blocks = 1;
  if (blocks > (1ull << 20)) return RADIC_EINVAL;
  pl.blocks = (int)blocks;
  pl.blocks2 = sms;
  layout_workspace(pl);
  *p = pl;
  return RADIC_OK;
}

void layout_workspace(SinglePlan& pl) {
  const int mode = pl.mode;
  const int n_warps = pl.blocks * pl.threads / 32;
  size_t off = 256;
  pl.off_partials = off;
  off = align_up(off + (size_t)pl.blocks * sizeof(FpPartial), 256);
  if (mode == kModeMixed || mode == kModePair) {
    pl.off_partials2 = off;
    off = align_up(off + (size_t)pl.blocks2 * sizeof(FpPartial), 256);
    pl.off_flag_count = off;
    off = align_up(off + (size_t)n_warps * sizeof(int), 256);
    pl.off_flag_ranks = off;
    off = align_up(off + (size_t)n_warps * pl.flag_cap * sizeof(unsigned long long), 256);
  }
  if (mode == kModeExact) {
    pl.off_modp = off;
    off = align_up(off + (size_t)pl.blocks * kMaxPrimes * sizeof(uint32_t), 256);
  }
  pl.ws_bytes = off;
}

__global__ void k_zero_result(radic_result* out, int tier) {
  out->value = 0.0;
  out->abs_sum = 0.0;
  out->err_bound = 0.0;
  out->exact_lo = 0;
  out->exact_hi = 0;
  out->minors = 0;
  out->flagged = 0;
  out->status = RADIC_OK;
  out->n_primes = (tier == kModeExact) ? 1 : 0;
  out->tier = tier;
  out->exact_exp = 0;
  for (int i = 0; i < 5; ++i) out->reserved[i] = 0;
}

template <int M>
__global__ void k_unrank(int n, unsigned long long q0, unsigned long long count, int L, uint8_t* cols) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* binom = reinterpret_cast<uint64_t*>(smem_raw);
  build_binom(binom, n, M);
  const unsigned long long tasks = (count + L - 1) / L;
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < tasks; t += nthreads) {
    unsigned long long q = q0 + t * L;
    const unsigned long long q1 = min(q + L, q0 + count);
    int c[M];
    unrank<M>(q, n, binom, M + 1, c);
    for (; q < q1; ++q) {
#pragma unroll
      for (int i = 0; i < M; ++i) cols[(q - q0) * M + i] = static_cast<uint8_t>(c[i]);
      if (q + 1 < q1) successor<M>(c, n);
    }
  }
}

template <int G>
__global__ void k_unrank_dyn(int n, int m, unsigned long long q0, unsigned long long count, int L, uint8_t* cols) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* binom = reinterpret_cast<uint64_t*>(smem_raw);
  build_binom(binom, n, m);
  const unsigned long long tasks = (count + L - 1) / L;
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < tasks; t += nthreads) {
    unsigned long long q = q0 + t * L;
    const unsigned long long q1 = min(q + L, q0 + count);
    int c[G];
    unrank_dyn<G>(q, n, m, binom, m + 1, c);
    for (; q < q1; ++q) {
#pragma unroll
      for (int i = 0; i < G; ++i)
        if (i < m) cols[(q - q0) * m + i] = static_cast<uint8_t>(c[i]);
      if (q + 1 < q1) successor_dyn<G>(c, n, m);
    }
  }
}

const void* unrank_kernel(int m) {
  switch (m) {
    case 1: return reinterpret_cast<const void*>(&k_unrank<1>);
    case 2: return reinterpret_cast<const void*>(&k_unrank<2>);
    case 3: return reinterpret_cast<const void*>(&k_unrank<3>);
    case 4: return reinterpret_cast<const void*>(&k_unrank<4>);
    case 5: return reinterpret_cast<const void*>(&k_unrank<5>);
    case 6: return reinterpret_cast<const void*>(&k_unrank<6>);
    case 7: return reinterpret_cast<const void*>(&k_unrank<7>);
    case 8: return reinterpret_cast<const void*>(&k_unrank<8>);
    case 9: return reinterpret_cast<const void*>(&k_unrank<9>);
    case 10: return reinterpret_cast<const void*>(&k_unrank<10>);
    case 11: return reinterpret_cast<const void*>(&k_unrank<11>);
    case 12: return reinterpret_cast<const void*>(&k_unrank<12>);
    default: return nullptr;
  }
}

}  // namespace

int launch_unrank(int n, int m, unsigned long long q0, unsigned long long count, uint8_t* cols, int L,
                  cudaStream_t s) {
  const int sms = device_sm_count();
  if (sms <= 0) return RADIC_ECUDA;
  const unsigned long long tasks = (count + L - 1) / L;
  unsigned long long blocks = (tasks + 127) / 128;
  if (blocks > (unsigned long long)sms * 8) blocks = (unsigned long long)sms * 8;
  if (blocks < 1) blocks = 1;
  const size_t smem = (size_t)(n + 1) * (m + 1) * 8;
  unsigned long long qq = q0, cc = count;
  int nn = n, mm = m, ll = L;
  cudaError_t e;
  if (const void* k = unrank_kernel(m)) {
    void* params[] = {&nn, &qq, &cc, &ll, &cols};
    e = cudaLaunchKernel(k, dim3((unsigned)blocks), dim3(128), params, smem, s);
  } else {
    void* params[] = {&nn, &mm, &qq, &cc, &ll, &cols};
    const void* k2 = (m <= 16) ? reinterpret_cast<const void*>(&k_unrank_dyn<16>)
                               : reinterpret_cast<const void*>(&k_unrank_dyn<32>);
    e = cudaLaunchKernel(k2, dim3((unsigned)blocks), dim3(128), params, smem, s);
  }
  return e == cudaSuccess ? RADIC_OK : RADIC_ECUDA;
}

}  // namespace radic

using namespace radic;

extern "C" {

const char* radic_status_string(int status) {
  switch (status) {
    case RADIC_OK: return "ok";
    case RADIC_EINVAL: return "invalid argument";
    case RADIC_EOVERFLOW: return "exact value may exceed the prime budget";
    case RADIC_ECUDA: return "CUDA runtime error";
    case RADIC_ETIMEOUT: return "device-side wait timed out";
    case RADIC_EWORKSPACE: return "workspace missing, misaligned or too small";
    case RADIC_EUNSUPPORTED: return "unsupported combination of arguments";
    default: return "unknown status";
  }
}

int radic_version(void) { return 10000; }

int radic_primes(uint32_t* primes, int max_count) {
  if (!primes || max_count <= 0) return 0;
  const int k = max_count < kMaxPrimes ? max_count : kMaxPrimes;
  for (int i = 0; i < k; ++i) primes[i] = kPrimes[i];
  return k;
}

size_t radic_workspace_bytes(int m, int n, int mode, const radic_options* opts) {
  SinglePlan p;
  if (make_plan(m, n, mode, opts, (m <= n && n <= kMaxN && m >= 1) ? binom_host(n, m) : 0ull, &p) != RADIC_OK)
    return 0;
  return p.ws_bytes;
}

int radic_plan_info(int m, int n, int mode, const radic_options* opts, int64_t* info, int count) {
  if ((!info && count > 0) || count < 0 || count > RADIC_PLAN_INFO_COUNT) return RADIC_EINVAL;
  SinglePlan p;
  const int rc =
      make_plan(m, n, mode, opts, (m <= n && n <= kMaxN && m >= 1 && n >= 1) ? binom_host(n, m) : 0ull, &p);
  if (rc != RADIC_OK) return rc;
  int64_t v[RADIC_PLAN_INFO_COUNT];
  v[0] = p.mapping;
  v[1] = (p.mapping == RADIC_MAP_PREFIX) ? p.depth : 0;
  v[2] = (p.mapping == RADIC_MAP_GROUP) ? p.group : 0;
  v[3] = p.threads;
  v[4] = p.blocks;
  v[5] = (p.mapping == RADIC_MAP_PREFIX) ? (int64_t)p.ptab.total_tasks : (int64_t)p.ranks_per_task;
  v[6] = (int64_t)p.smem;
  v[7] = (int64_t)p.ws_bytes;
  for (int i = 0; i < count; ++i) info[i] = v[i];
  return RADIC_OK;
}

int radic_prefix_plan_host(int m, int n, int mode, const radic_options* opts, int sms, int blocks_per_sm,
                           int64_t* info, int count) {
  if (!info || sms < 1 || blocks_per_sm < 1 || count < 8 + 4 * n) return RADIC_EINVAL;
  if (m < 1 || n < 1 || n > kMaxN || m > n) return RADIC_EINVAL;
  radic_options d;
  std::memset(&d, 0, sizeof(d));
  if (opts) d = *opts;
  d.mapping = RADIC_MAP_PREFIX;
  SinglePlan p;
  const int rc = make_plan_uncached(m, n, mode, &d, binom_host(n, m), &p, sms, blocks_per_sm);
  if (rc != RADIC_OK) return rc;
  const PrefixTable& t = p.ptab;
  for (int i = 0; i < count; ++i) info[i] = 0;
  info[0] = p.depth;
  info[1] = static_cast<int64_t>(t.total_tasks);
  info[2] = p.blocks;
  info[3] = t.v_lo;
  info[4] = t.v_hi;
  info[5] = t.dynamic;
  for (int v = t.v_lo; v <= t.v_hi; ++v) {
    info[8 + 4 * v + 0] = static_cast<int64_t>(t.count[v]);
    info[8 + 4 * v + 1] = static_cast<int64_t>(t.run[v]);
    info[8 + 4 * v + 2] = t.lanes[v];
    info[8 + 4 * v + 3] = static_cast<int64_t>(t.task_start[v]);
  }
  return RADIC_OK;
}

int radic_det(const void* A, int m, int n, int64_t lda, int dtype, int mode, const radic_options* opts,
              radic_result* out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!A || !out || lda < n || !valid_dtype(dtype)) return RADIC_EINVAL;
  SinglePlan p;
  const unsigned long long total = (m >= 1 && n >= 1 && m <= n && n <= kMaxN) ? binom_host(n, m) : 0ull;
  const int rc = make_plan(m, n, mode, opts, total, &p);
  if (rc != RADIC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.total == 0) {
    k_zero_result<<<1, 1, 0, s>>>(out, mode);
    return cudaGetLastError() == cudaSuccess ? RADIC_OK : RADIC_ECUDA;
  }
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < p.ws_bytes)
    return RADIC_EWORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (cudaMemsetAsync(ws, 0, 256, s) != cudaSuccess) return RADIC_ECUDA;
  SingleArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = A;
  a.lda = lda;
  a.dtype = dtype;
  a.m = m;
  a.n = n;
  a.ranks_per_task = p.ranks_per_task;
  a.total = p.total;
  a.tasks = p.tasks;
  a.growth = p.growth;
  a.flag_cap = p.flag_cap;
  a.flag_prefix = (p.mapping == RADIC_MAP_PREFIX) ? m - p.depth : 0;
  a.n_warps = p.blocks * p.threads / 32;
  a.hdr = reinterpret_cast<WsHeader*>(ws);
  a.partials = reinterpret_cast<FpPartial*>(ws + p.off_partials);
  a.partials2 = reinterpret_cast<FpPartial*>(ws + p.off_partials2);
  a.flag_count = reinterpret_cast<int*>(ws + p.off_flag_count);
  a.flag_ranks = reinterpret_cast<unsigned long long*>(ws + p.off_flag_ranks);
  a.modp_partials = reinterpret_cast<uint32_t*>(ws + p.off_modp);
  a.out = out;
  int r;
  switch (mode) {
    case kModeFp64: r = launch_fp64(p, a, s); break;
    case kModeMixed: r = launch_mixed(p, a, s); break;
    case kModePair: r = launch_pair(p, a, s); break;
    default: r = launch_modp(p, a, s); break;
  }
  return r;
}

size_t radic_wide_workspace_bytes(int m, int n, const radic_options* opts) {
  SinglePlan p;
  const unsigned long long total = (m >= 1 && n >= 1 && m <= n && n <= kMaxN) ? binom_host(n, m) : 0ull;
  if (make_plan(m, n, kModeExact, opts, total, &p) != RADIC_OK) return 0;
  // the EXACT workspace, then the residues of every pass (kWidePrimes words,
  // then needed, exponent and status)
  return align_up(p.ws_bytes, 256) + 256;
}

int radic_det_exact_wide(const void* A, int m, int n, int64_t lda, int dtype, const radic_options* opts,
                         radic_wide_result* out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!A || !out || lda < n || !valid_dtype(dtype)) return RADIC_EINVAL;
  SinglePlan p;
  const unsigned long long total = (m >= 1 && n >= 1 && m <= n && n <= kMaxN) ? binom_host(n, m) : 0ull;
  const int rc = make_plan(m, n, kModeExact, opts, total, &p);
  if (rc != RADIC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.total == 0) return launch_wide_crt(nullptr, out, 0ull, s);
  const size_t off_wide = align_up(p.ws_bytes, 256);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < off_wide + 256)
    return RADIC_EWORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  uint32_t* wide = reinterpret_cast<uint32_t*>(ws + off_wide);
  for (int base = 0; base < kWidePrimes; base += kMaxPrimes) {
    if (cudaMemsetAsync(ws, 0, 256, s) != cudaSuccess) return RADIC_ECUDA;
    SingleArgs a;
    std::memset(&a, 0, sizeof(a));
    a.A = A;
    a.lda = lda;
    a.dtype = dtype;
    a.m = m;
    a.n = n;
    a.ranks_per_task = p.ranks_per_task;
    a.total = p.total;
    a.tasks = p.tasks;
    a.growth = p.growth;
    a.n_warps = p.blocks * p.threads / 32;
    a.hdr = reinterpret_cast<WsHeader*>(ws);
    a.modp_partials = reinterpret_cast<uint32_t*>(ws + p.off_modp);
    a.prime_base = base;
    a.wide = wide;
    const int r = launch_modp(p, a, s);
    if (r != RADIC_OK) return r;
  }
  return launch_wide_crt(wide, out, p.total, s);
}

int radic_terms(const void* A, int m, int n, int64_t lda, int dtype, int mode, const radic_options* opts,
                uint64_t q0, uint64_t count, void* terms, void* stream) {
  if (!A || !terms || lda < n || !valid_dtype(dtype)) return RADIC_EINVAL;
  if (mode == kModeExact && (dtype == kF32 || dtype == kF64)) return RADIC_EINVAL;
  if (m < 1 || n < 1 || m > n || n > kMaxN || m > kMaxM) return RADIC_EINVAL;
  const unsigned long long total = binom_host(n, m);
  if (q0 >= total || count > total - q0) return RADIC_EINVAL;
  if (count == 0) return RADIC_OK;
  SinglePlan p;
  const int rc = make_plan(m, n, mode, opts, count, &p);
  if (rc != RADIC_OK) return rc;
  SingleArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = A;
  a.lda = lda;
  a.dtype = dtype;
  a.m = m;
  a.n = n;
  a.ranks_per_task = p.ranks_per_task;
  a.total = total;
  a.tasks = p.tasks;
  a.growth = p.growth;
  a.flag_cap = p.flag_cap;
  a.q0 = q0;
  a.count = count;
  a.terms = terms;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (mode) {
    case kModeFp64: return launch_fp64(p, a, s);
    case kModeMixed: return launch_mixed(p, a, s);
    case kModePair: return launch_pair(p, a, s);
    default: return launch_modp(p, a, s);
  }
}

int radic_unrank(int n, int m, uint64_t q0, uint64_t count, uint8_t* cols, const radic_options* opts,
                 void* stream) {
  if (!cols || m < 1 || n < 1 || m > n || n > kMaxN || m > kMaxM) return RADIC_EINVAL;
  const unsigned long long total = binom_host(n, m);
  if (q0 >= total || count > total - q0) return RADIC_EINVAL;
  if (count == 0) return RADIC_OK;
  const int L = (opts && opts->ranks_per_task > 0) ? opts->ranks_per_task : 64;
  return launch_unrank(n, m, q0, count, cols, L, static_cast<cudaStream_t>(stream));
}

struct radic_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

int radic_graph_create(const void* A, int m, int n, int64_t lda, int dtype, int mode, const radic_options* opts,
                       radic_result* out, void* workspace, size_t workspace_bytes, radic_graph** graph) {
  if (!graph) return RADIC_EINVAL;
  *graph = nullptr;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return RADIC_ECUDA;
  radic_graph* g = new (std::nothrow) radic_graph;
  int rc = g ? RADIC_OK : RADIC_EINVAL;
  if (rc == RADIC_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = RADIC_ECUDA;
  if (rc == RADIC_OK) {
    const int r = radic_det(A, m, n, lda, dtype, mode, opts, out, workspace, workspace_bytes, cs);
    const cudaError_t e = cudaStreamEndCapture(cs, &g->graph);
    if (r != RADIC_OK) rc = r;
    else if (e != cudaSuccess) rc = RADIC_ECUDA;
  }
  if (rc == RADIC_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = RADIC_ECUDA;
  cudaStreamDestroy(cs);
  if (rc != RADIC_OK) {
    if (g) {
      if (g->exec) cudaGraphExecDestroy(g->exec);
      if (g->graph) cudaGraphDestroy(g->graph);
      delete g;
    }
    return rc;
  }
  *graph = g;
  return RADIC_OK;
}

int radic_graph_launch(radic_graph* graph, void* stream) {
  if (!graph || !graph->exec) return RADIC_EINVAL;
  return cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RADIC_OK : RADIC_ECUDA;
}

int radic_graph_destroy(radic_graph* graph) {
  if (!graph) return RADIC_OK;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  delete graph;
  return RADIC_OK;
}

}  // extern "C"
