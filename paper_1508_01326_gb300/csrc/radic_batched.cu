// Batched Radic determinants: many matrices of uneven m and n in one pass.
//
// The host plan routes every matrix to a tier (binary32 elimination with
// binary64 sums, elimination in pairs of binary32 with binary64 sums, or
// binary64) and cuts its work into warp tasks: runs of
// (m-2)-column prefixes of one group (prefix mapping) or runs of dictionary
// ranks (per-minor mapping), each with about the same estimated cost.  Tasks
// are sorted by cost, largest first.  One persistent kernel per tier pulls
// tasks from an atomic work queue; a warp stages its task's matrix and
// binomial table in its own slice of shared memory, works the task (every
// lane one contiguous run, as in the split of Section 5) and writes the
// task's partial sum into the task's own slot.  Binary32 and pair tasks that
// meet a flag are appended to a list and recomputed in binary64 by the
// binary64 kernel into the same slot, so the result does not depend on which
// warp ran which task.  A last kernel adds each matrix's slots in task order.
#include "radic_batched.cuh"


// ---------------------------------------------------------------------------
// Host plan and C ABI
// ---------------------------------------------------------------------------
using namespace radic;

struct radic_batch_plan {
  int batch = 0, mode = 0;
  std::vector<int> shape;            // m, n per matrix
  std::vector<long long> offset;
  std::vector<int> tier;
  // t32: binary32 and pair tasks, t64: binary64 tasks; both sorted by group
  // (m, task path), then tier (binary32 before pairs), then cost (largest first)
  std::vector<BatchTask> t32, t64;
  int g32[kGroups + 1] = {0}, g64[kGroups + 1] = {0};  // task ranges per group
  int gpair[kGroups] = {0};  // first pair task of the group in t32 (binary32 tasks before it)
  std::vector<int> csr_ptr, csr_idx;
  int max_n = 1, max_m = 1;
  // persistent grid of each group's kernel per queue (0 binary32, 1 pairs, 2 binary64)
  int blocks[3][kGroups] = {{0}};
  int slice32[kBatchMaxM + 1] = {0}, slice64[kBatchMaxM + 1] = {0}, slicep[kBatchMaxM + 1] = {0};  // per warp
  double tol = 1e-10, growth = 64.0;
  int tiers = 3;  // allowed low tiers: bit 0 binary32, bit 1 pairs
  // workspace layout
  size_t off_t32 = 0, off_t64 = 0, off_slots = 0, off_flagged = 0, off_escale = 0, off_csr_ptr = 0,
         off_csr_idx = 0, off_tier = 0, off_shape = 0, off_rerouted = 0, ws_bytes = 0;
  long long n_fp32_matrices = 0, n_fp64_matrices = 0, n_pair_matrices = 0;
  unsigned long long minors32 = 0, minors64 = 0, minors_pair = 0;
  int tasks_pair = 0;
  int launches = 0;                      // kernel launches per call
  int dom_queue = -1, dom_group = -1;    // the low-tier kernel with the most estimated work
  void* events = nullptr;                // optional cudaEvent_t[2] around it
  // launch order of the per-group kernels, most estimated work first:
  // (queue, group) of the low tiers, groups of the binary64 kernels
  std::vector<std::pair<int, int>> order_low;
  std::vector<int> order64;
  // the per-group kernels of one phase run concurrently on the caller's
  // stream and kAux more (fork and join by events), so that a kernel's tail,
  // when its work queue runs dry, is filled by the next kernel's blocks
  static constexpr int kAux = 2;
  cudaStream_t aux[kAux] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[kAux] = {nullptr, nullptr};
  ~radic_batch_plan() {
    for (int i = 0; i < kAux; ++i) {
      if (aux[i]) cudaStreamDestroy(aux[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

struct radic_batch_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

double cost_minor(int m) { return 10.0 * m * m * m / 3.0 + 40.0; }

// Cost of one head (H = m-D-1 columns) whose last prefix columns run over
// [v0, v1]: its factorisation, then per appended column v one elimination
// step and the prefix's leaves.
double head_cost(int m, int D, int n, int v0, int v1) {
  const int H = m - D - 1, P = m - D;
  double c = (double)m * H * H;
  for (int v = v0; v <= v1; ++v) c += m + 4.0 * (D + 1) * H + prefix_cost(m, D, n - 1 - v) - (double)m * P * P;
  return c;
}

// Minors one lane works for one unit of a head-shared task at most (a single
// prefix, up to C(n-m+D, D) minors, is never split): a head's whole subtree
// holds up to C(n-m+1, D+1) minors, and the longest unit sets the kernel's
// critical path.
constexpr unsigned long long kSegmentMinors = 4096;

// Splits the last columns v = u+1 .. n-1-D of the heads with last column u
// into consecutive ranges of at most kSegmentMinors minors.
std::vector<std::pair<int, int>> head_segments(int n, int D, int u) {
  std::vector<std::pair<int, int>> out;
  const int ve = n - 1 - D;
  int v = u + 1;
  while (v <= ve) {
    int v1 = v;
    unsigned long long sm = binom_host(n - 1 - v, D);
    while (v1 + 1 <= ve && sm + binom_host(n - 2 - v1, D) <= kSegmentMinors) sm += binom_host(n - 1 - ++v1, D);
    out.push_back({v, v1});
    v = v1 + 1;
  }
  return out;
}

int make_tasks(radic_batch_plan& pl, int b, int tier, const radic_batch_tuning* tun) {
  const int m = pl.shape[2 * b], n = pl.shape[2 * b + 1];
  std::vector<BatchTask>& out = (tier == kModeFp64) ? pl.t64 : pl.t32;
  if (m > n) return RADIC_OK;
  int kind = (m >= 3) ? prefix_auto_depth(m, n, true) : kKindMinor;
  if (tun && tun->kind[m] == RADIC_MAP_THREAD && m <= 8 && tier == kModeMixed) kind = kKindMinor;
  if (tun && tun->kind[m] == RADIC_MAP_PREFIX && m >= 3) kind = prefix_auto_depth(m, n, true);
  if (kind != kKindMinor && tun && (tun->prefix_depth[m] == 2 || (tun->prefix_depth[m] == 3 && m >= 4)))
    kind = tun->prefix_depth[m];
  const double lane_cost = (tun && tun->task_cost[m] > 0.0) ? tun->task_cost[m] : 30000.0;
  BatchTask t;
  std::memset(&t, 0, sizeof(t));
  t.offset = pl.offset[b];
  t.b = b;
  t.m = m;
  t.n = n;
  t.kind = kind;
  t.tier = tier;
  // Head sharing pays from heads of five columns on (measured on the batched
  // m = 5..10 sets: 25% faster at m = 10, depth 3; slower below four head
  // columns, where heads are few and their work uneven).
  const bool share = kind != kKindMinor && m - kind - 1 >= 5 && !(tun && tun->head_sharing < 0);
  if (share) {
    // head-shared tasks: group u = last head column, C(u, H-1) heads each,
    // one task list per segment of the heads' last columns
    const int D = kind, H = m - D - 1;
    t.shared = 1;
    for (int u = H - 1; u <= n - 2 - D; ++u) {
      const unsigned long long cnt = binom_host(u, H - 1);
      for (const auto& sg : head_segments(n, D, u)) {
        const double c = head_cost(m, D, n, sg.first, sg.second);
        unsigned long long run = (unsigned long long)std::max(1.0, std::floor(lane_cost / c));
        run = std::min(run, (cnt + 31) / 32);
        if (run < 1) run = 1;
        t.vlo = sg.first;
        t.vhi = sg.second;
        t.per_unit = 0;
        for (int v = sg.first; v <= sg.second; ++v) t.per_unit += binom_host(n - 1 - v, D);
        for (unsigned long long r0 = 0; r0 < cnt; r0 += 32 * run) {
          t.v = u;
          t.r0 = r0;
          t.run = run;
          t.lim = cnt;
          out.push_back(t);
        }
      }
    }
  } else if (kind != kKindMinor) {
    const int D = kind, P = m - D;
    for (int v = P - 1; v <= n - 1 - D; ++v) {
      const unsigned long long cnt = binom_host(v, P - 1);
      const double c = prefix_cost(m, D, n - 1 - v);
      unsigned long long run = (unsigned long long)std::max(1.0, std::floor(lane_cost / c));
      run = std::min(run, (cnt + 31) / 32);
      if (run < 1) run = 1;
      t.per_unit = binom_host(n - 1 - v, D);
      for (unsigned long long r0 = 0; r0 < cnt; r0 += 32 * run) {
        t.v = v;
        t.r0 = r0;
        t.run = run;
        t.lim = cnt;
        out.push_back(t);
      }
    }
  } else {
    const unsigned long long total = binom_host(n, m);
    unsigned long long run = (unsigned long long)std::max(1.0, std::floor(lane_cost / cost_minor(m)));
    run = std::min(run, (total + 31) / 32);
    if (run < 1) run = 1;
    t.per_unit = 1;
    for (unsigned long long r0 = 0; r0 < total; r0 += 32 * run) {
      t.v = 0;
      t.r0 = r0;
      t.run = run;
      t.lim = total;
      out.push_back(t);
    }
  }
  return RADIC_OK;
}

double task_cost(const BatchTask& t) {
  if (t.kind != kKindMinor && t.shared) return (double)t.run * head_cost(t.m, t.kind, t.n, t.vlo, t.vhi);
  if (t.kind != kKindMinor) return (double)t.run * prefix_cost(t.m, t.kind, t.n - 1 - t.v);
  return (double)t.run * cost_minor(t.m);
}

int persistent_blocks(const void* k, int slice_bytes, int sms) {
  const size_t smem = (size_t)slice_bytes * (kBatchThreads / 32);
  if (!k || !allow_smem(k, smem)) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kBatchThreads, smem) != cudaSuccess) return 0;
  return nb * sms;
}

const void* group_kernel(int queue, int g) {
  const int m = g / kPaths, path = g % kPaths;
  return queue == 0 ? batch_kernel_f32(m, path) : queue == 1 ? batch_kernel_pair(m, path) : batch_kernel_f64(m, path);
}

int enqueue(const radic_batch_plan* pl, const void* A, int dtype, radic_result* out, void* workspace, cudaStream_t s) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (cudaMemsetAsync(ws, 0, kBatchHeaderBytes, s) != cudaSuccess) return RADIC_ECUDA;
  if (cudaMemsetAsync(ws + pl->off_rerouted, 0, (size_t)pl->batch * sizeof(int), s) != cudaSuccess)
    return RADIC_ECUDA;
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.A = A;
  a.dtype = dtype;
  a.tol = pl->tol;
  for (int g = 0; g < kGroups; ++g) a.flag_base_g[g] = pl->g32[g];
  a.rerouted = reinterpret_cast<int*>(ws + pl->off_rerouted);
  a.n_tasks32 = (int)pl->t32.size();
  a.tasks32 = reinterpret_cast<const BatchTask*>(ws + pl->off_t32);
  a.tasks64 = reinterpret_cast<const BatchTask*>(ws + pl->off_t64);
  a.slots = reinterpret_cast<FpPartial*>(ws + pl->off_slots);
  a.flagged = reinterpret_cast<int*>(ws + pl->off_flagged);
  a.escale = reinterpret_cast<int*>(ws + pl->off_escale);
  a.hdr = reinterpret_cast<BatchHeader*>(ws);
  a.growth = pl->growth;
  cudaEvent_t* ev = static_cast<cudaEvent_t*>(pl->events);
  // inside a stream capture the events become event-record nodes of the graph
  // (recorded at every replay) only with the external flag
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (ev && cudaStreamIsCapturing(s, &cap) != cudaSuccess) return RADIC_ECUDA;
  const unsigned ev_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
  // the caller's stream and the plan's auxiliary streams; kernel i of a
  // phase goes to stream i mod (kAux + 1)
  cudaStream_t lanes[radic_batch_plan::kAux + 1] = {s, pl->aux[0], pl->aux[1]};
  const int nl = pl->fork ? radic_batch_plan::kAux + 1 : 1;
  auto fork = [&]() {
    if (nl == 1) return true;
    if (cudaEventRecord(pl->fork, s) != cudaSuccess) return false;
    for (int i = 1; i < nl; ++i)
      if (cudaStreamWaitEvent(lanes[i], pl->fork, 0) != cudaSuccess) return false;
    return true;
  };
  auto join = [&]() {
    for (int i = 1; i < nl; ++i) {
      if (cudaEventRecord(pl->join[i - 1], lanes[i]) != cudaSuccess) return false;
      if (cudaStreamWaitEvent(s, pl->join[i - 1], 0) != cudaSuccess) return false;
    }
    return true;
  };
  auto launch = [&](int queue, int g, int slice, cudaStream_t st) {
    a.group = g;
    a.queue = queue;
    a.slice_bytes = slice;
    void* params[] = {&a};
    const bool dom = ev && queue == pl->dom_queue && g == pl->dom_group;
    if (dom && cudaEventRecordWithFlags(ev[0], st, ev_flags) != cudaSuccess) return false;
    if (cudaLaunchKernel(group_kernel(queue, g), dim3(pl->blocks[queue][g]), dim3(kBatchThreads), params,
                         (size_t)slice * (kBatchThreads / 32), st) != cudaSuccess)
      return false;
    return !dom || cudaEventRecordWithFlags(ev[1], st, ev_flags) == cudaSuccess;
  };
  // binary32 and pair tiers, one persistent kernel per tier and group
  // present, most work first
  if (!fork()) return RADIC_ECUDA;
  int li = 0;
  for (const auto& qg : pl->order_low) {
    const int queue = qg.first, g = qg.second, m = g / kPaths;
    a.flag_base = pl->g32[g];
    a.begin64 = pl->g64[g];
    a.end64 = pl->g64[g + 1];
    a.begin32 = queue == 0 ? pl->g32[g] : pl->gpair[g];
    a.end32 = queue == 0 ? pl->gpair[g] : pl->g32[g + 1];
    if (!launch(queue, g, queue == 0 ? pl->slice32[m] : pl->slicep[m], lanes[li++ % nl])) return RADIC_ECUDA;
  }
  if (!join()) return RADIC_ECUDA;
  ReduceArgs r;
  r.csr_ptr = reinterpret_cast<const int*>(ws + pl->off_csr_ptr);
  r.csr_idx = reinterpret_cast<const int*>(ws + pl->off_csr_idx);
  r.tier = reinterpret_cast<const int*>(ws + pl->off_tier);
  r.rerouted = a.rerouted;
  r.shape = reinterpret_cast<const int*>(ws + pl->off_shape);
  r.slots = a.slots;
  r.escale = a.escale;
  r.out = out;
  r.batch = pl->batch;
  const unsigned blocks = (unsigned)((pl->batch * 32 + 127) / 128);
  // a-posteriori check of the low tiers: matrices whose error bound misses
  // tol are redone by the binary64 kernels below
  if (!pl->t32.empty()) {
    void* cparams[] = {&a, &r};
    if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_batch_check), dim3(blocks > 0 ? blocks : 1), dim3(128),
                         cparams, 0, s) != cudaSuccess)
      return RADIC_ECUDA;
  }
  // binary64 tier (and the flagged or rerouted binary32 and pair tasks), one
  // kernel per group present, most binary64 work first
  if (!fork()) return RADIC_ECUDA;
  li = 0;
  for (const int g : pl->order64) {
    a.flag_base = pl->g32[g];
    a.begin32 = pl->g32[g];
    a.end32 = pl->g32[g + 1];
    a.begin64 = pl->g64[g];
    a.end64 = pl->g64[g + 1];
    if (!launch(2, g, pl->slice64[g / kPaths], lanes[li++ % nl])) return RADIC_ECUDA;
  }
  if (!join()) return RADIC_ECUDA;
  void* rparams[] = {&r};
  if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_batch_reduce), dim3(blocks > 0 ? blocks : 1), dim3(128),
                       rparams, 0, s) != cudaSuccess)
    return RADIC_ECUDA;
  return RADIC_OK;
}

}  // namespace

namespace {
// Host part of the plan: routing of every matrix to a tier, its tasks, and
// their order.  Returns a RADIC_* code; `pl` is filled on success.
int plan_tasks(radic_batch_plan* pl, const int32_t* m, const int32_t* n, const int64_t* offsets, int batch, int mode,
               const radic_batch_tuning* tuning) {
  pl->batch = batch;
  pl->mode = mode;
  if (tuning && tuning->tol > 0.0) pl->tol = tuning->tol;
  if (tuning && tuning->growth_threshold > 0.0) pl->growth = tuning->growth_threshold;
  if (tuning && tuning->tiers != 0) pl->tiers = tuning->tiers & 3;
  pl->shape.resize(2 * (size_t)batch);
  pl->offset.resize(batch);
  pl->tier.resize(batch);
  for (int b = 0; b < batch; ++b) {
    if (m[b] < 1 || n[b] < 1 || m[b] > kBatchMaxM || n[b] > kMaxN || offsets[b] < 0)
      return m[b] > kBatchMaxM && m[b] <= kMaxM ? RADIC_EUNSUPPORTED : RADIC_EINVAL;
    pl->shape[2 * b] = m[b];
    pl->shape[2 * b + 1] = n[b];
    pl->offset[b] = offsets[b];
    pl->max_n = std::max(pl->max_n, (int)n[b]);
    pl->max_m = std::max(pl->max_m, (int)m[b]);
    const unsigned long long c = (m[b] <= n[b]) ? binom_host(n[b], m[b]) : 0ull;
    // Routing: the first tier of a matrix is the cheapest whose error bound
    // relative to sum|terms| usually meets the target: binary32 elimination
    // when kBinary32BoundK <= tol, else pairs (m >= 3) when kPairBoundK <=
    // tol, else binary64.  The constants are envelopes of the bounds measured
    // on random matrices; the device then checks every matrix's own bound
    // (k_batch_check) and redoes in binary64 those that miss tol.
    int tier = kModeFp64;
    if (mode == RADIC_MODE_MIXED && c > 0) {
      if ((pl->tiers & 1) && kBinary32BoundK <= pl->tol) tier = kModeMixed;
      else if ((pl->tiers & 2) && m[b] >= 3 && kPairBoundK <= pl->tol) tier = kModePair;
    }
    pl->tier[b] = tier;
    if (tier == kModeMixed) {
      pl->n_fp32_matrices++;
      pl->minors32 += c;
    } else if (tier == kModePair) {
      pl->n_pair_matrices++;
      pl->minors_pair += c;
    } else {
      pl->n_fp64_matrices++;
      pl->minors64 += c;
    }
    make_tasks(*pl, b, tier, tuning);
  }
  // per group (m, task path) and tier (binary32 before pairs), largest tasks
  // first (longest-processing-time order for each queue)
  auto gid = [](const BatchTask& t) { return group_of(t.m, path_of(t.kind, t.shared)); };
  auto order = [&](const BatchTask& x, const BatchTask& y) {
    if (gid(x) != gid(y)) return gid(x) < gid(y);
    if (x.tier != y.tier) return x.tier == kModeMixed;
    return task_cost(x) > task_cost(y);
  };
  std::stable_sort(pl->t32.begin(), pl->t32.end(), order);
  std::stable_sort(pl->t64.begin(), pl->t64.end(), order);
  for (int g = 0; g <= kGroups; ++g) {
    pl->g32[g] = (int)(std::lower_bound(pl->t32.begin(), pl->t32.end(), g,
                                        [&](const BatchTask& t, int gg) { return gid(t) < gg; }) -
                       pl->t32.begin());
    pl->g64[g] = (int)(std::lower_bound(pl->t64.begin(), pl->t64.end(), g,
                                        [&](const BatchTask& t, int gg) { return gid(t) < gg; }) -
                       pl->t64.begin());
  }
  for (int g = 0; g < kGroups; ++g) {
    int i = pl->g32[g];
    while (i < pl->g32[g + 1] && pl->t32[i].tier == kModeMixed) ++i;
    pl->gpair[g] = i;
  }
  for (const BatchTask& t : pl->t32) pl->tasks_pair += (t.tier == kModePair);
  return RADIC_OK;
}
}  // namespace

extern "C" {


int radic_batch_plan_create(const int32_t* m, const int32_t* n, const int64_t* offsets, int batch, int mode,
                            const radic_batch_tuning* tuning, radic_batch_plan** plan) {
  if (!plan || batch < 1 || !m || !n || !offsets) return RADIC_EINVAL;
  if (mode != RADIC_MODE_FP64 && mode != RADIC_MODE_MIXED) return RADIC_EUNSUPPORTED;
  *plan = nullptr;
  radic_batch_plan* pl = new (std::nothrow) radic_batch_plan;
  if (!pl) return RADIC_EINVAL;
  {
    const int rc = plan_tasks(pl, m, n, offsets, batch, mode, tuning);
    if (rc != RADIC_OK) {
      delete pl;
      return rc;
    }
  }
  // per-matrix task lists in task order (fixed summation order)
  std::vector<std::vector<int>> per(batch);
  for (size_t i = 0; i < pl->t32.size(); ++i) per[pl->t32[i].b].push_back((int)i);
  for (size_t i = 0; i < pl->t64.size(); ++i) per[pl->t64[i].b].push_back((int)(pl->t32.size() + i));
  pl->csr_ptr.assign(batch + 1, 0);
  for (int b = 0; b < batch; ++b) {
    pl->csr_ptr[b + 1] = pl->csr_ptr[b] + (int)per[b].size();
    for (int id : per[b]) pl->csr_idx.push_back(id);
  }
  if (pl->csr_idx.empty()) pl->csr_idx.push_back(0);
  // per-warp shared-memory slices of each m's kernels: binomial table and
  // staged matrix for the largest n of that m, column buffer for the most
  // candidate columns and the deepest prefix among that kernel's tasks (the
  // binary64 kernel of m also redoes flagged binary32 tasks of m)
  {
    int n32[kBatchMaxM + 1] = {0}, d32[kBatchMaxM + 1] = {0}, n64[kBatchMaxM + 1] = {0}, d64[kBatchMaxM + 1] = {0};
    int np[kBatchMaxM + 1] = {0}, dp[kBatchMaxM + 1] = {0};
    for (const BatchTask& t : pl->t32) {
      int* nn = (t.tier == kModePair) ? np : n32;
      int* dd = (t.tier == kModePair) ? dp : d32;
      nn[t.m] = std::max(nn[t.m], t.n);
      if (t.kind != kKindMinor) dd[t.m] = std::max(dd[t.m], t.kind);
    }
    for (const BatchTask& t : pl->t64) {
      n64[t.m] = std::max(n64[t.m], t.n);
      if (t.kind != kKindMinor) d64[t.m] = std::max(d64[t.m], t.kind);
    }
    auto slice = [](int m, int n, int depth, int cs, int elem, bool dbl) {
      size_t b = slice_bytes_before_zbuf(n, m, cs, elem, dbl);
      if (depth > 0) b += zbuf_bytes(n - m + depth, 32, depth, elem);
      return (int)align_up(b, 32);
    };
    for (int m = 1; m <= kBatchMaxM; ++m) {
      n64[m] = std::max(n64[m], std::max(n32[m], np[m]));
      d64[m] = std::max(d64[m], std::max(d32[m], dp[m]));
      if (n32[m] > 0) pl->slice32[m] = slice(m, n32[m], d32[m], ((m + 3) / 4) * 4, 4, false);
      if (np[m] > 0) pl->slicep[m] = slice(m, np[m], dp[m], ((m + 1) / 2) * 2, 8, true);
      if (n64[m] > 0) pl->slice64[m] = slice(m, n64[m], d64[m], ((m + 1) / 2) * 2, 8, false);
    }
  }
  const int sms = device_sm_count();
  if (sms <= 0) {
    delete pl;
    return RADIC_ECUDA;
  }
  const int occ = (tuning && tuning->blocks_per_sm > 0) ? tuning->blocks_per_sm : 0;
  for (int g = 0; g < kGroups; ++g) {
    const int m = g / kPaths;
    const bool has32 = pl->gpair[g] > pl->g32[g];
    const bool hasp = pl->g32[g + 1] > pl->gpair[g];
    const bool has64 = pl->g64[g + 1] > pl->g64[g] || has32 || hasp;
    const bool need[3] = {has32, hasp, has64};
    const int slice[3] = {pl->slice32[m], pl->slicep[m], pl->slice64[m]};
    for (int q = 0; q < 3; ++q) {
      if (!need[q]) continue;
      pl->blocks[q][g] = persistent_blocks(group_kernel(q, g), slice[q], sms);
      if (occ > 0) pl->blocks[q][g] = std::min(pl->blocks[q][g], occ * sms);
      if (pl->blocks[q][g] <= 0) {
        delete pl;
        return RADIC_EUNSUPPORTED;
      }
    }
  }
  // launches per call, their order (most estimated work first), and the
  // dominant low-tier kernel
  {
    std::vector<std::pair<double, std::pair<int, int>>> low;
    std::vector<std::pair<double, int>> hi;
    for (int g = 0; g < kGroups; ++g) {
      const int ranges[2][2] = {{pl->g32[g], pl->gpair[g]}, {pl->gpair[g], pl->g32[g + 1]}};
      for (int q = 0; q < 2; ++q) {
        if (ranges[q][1] <= ranges[q][0]) continue;
        double c = 0.0;
        for (int i = ranges[q][0]; i < ranges[q][1]; ++i) c += task_cost(pl->t32[i]);
        low.push_back({c, {q, g}});
      }
      if (pl->g64[g + 1] > pl->g64[g] || pl->g32[g + 1] > pl->g32[g]) {
        double c = 0.0;
        for (int i = pl->g64[g]; i < pl->g64[g + 1]; ++i) c += task_cost(pl->t64[i]);
        hi.push_back({c, g});
      }
    }
    // stable order: most work first, ties by (queue, group)
    std::stable_sort(low.begin(), low.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::stable_sort(hi.begin(), hi.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (const auto& e : low) pl->order_low.push_back(e.second);
    for (const auto& e : hi) pl->order64.push_back(e.second);
    if (!low.empty()) {
      pl->dom_queue = low[0].second.first;
      pl->dom_group = low[0].second.second;
    }
    pl->launches = (int)(low.size() + hi.size()) + 1 + (pl->t32.empty() ? 0 : 1);  // + reduce, check
    if (tuning) pl->events = tuning->kernel_events;
  }
  // auxiliary streams and fork/join events of the concurrent phases
  for (int i = 0; i < radic_batch_plan::kAux; ++i) {
    if (cudaStreamCreateWithFlags(&pl->aux[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->join[i], cudaEventDisableTiming) != cudaSuccess) {
      delete pl;
      return RADIC_ECUDA;
    }
  }
  if (cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete pl;
    return RADIC_ECUDA;
  }
  // workspace layout
  size_t off = kBatchHeaderBytes;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  pl->off_t32 = take(std::max<size_t>(1, pl->t32.size()) * sizeof(BatchTask));
  pl->off_t64 = take(std::max<size_t>(1, pl->t64.size()) * sizeof(BatchTask));
  pl->off_slots = take((pl->t32.size() + pl->t64.size() + 1) * sizeof(FpPartial));
  pl->off_flagged = take((pl->t32.size() + 1) * sizeof(int));
  pl->off_escale = take((size_t)batch * sizeof(int));
  pl->off_csr_ptr = take((size_t)(batch + 1) * sizeof(int));
  pl->off_csr_idx = take(pl->csr_idx.size() * sizeof(int));
  pl->off_tier = take((size_t)batch * sizeof(int));
  pl->off_shape = take((size_t)2 * batch * sizeof(int));
  pl->off_rerouted = take((size_t)batch * sizeof(int));
  pl->ws_bytes = off;
  *plan = pl;
  return RADIC_OK;
}

constexpr int kTaskRow = RADIC_BATCH_TASK_FIELDS;

int radic_batch_plan_tasks_host(const int32_t* m, const int32_t* n, const int64_t* offsets, int batch, int mode,
                                const radic_batch_tuning* tuning, int64_t* tasks, int64_t capacity,
                                int64_t* n_tasks) {
  if (batch < 1 || !m || !n || !offsets || !n_tasks || capacity < 0 || (capacity > 0 && !tasks)) return RADIC_EINVAL;
  if (mode != RADIC_MODE_FP64 && mode != RADIC_MODE_MIXED) return RADIC_EUNSUPPORTED;
  radic_batch_plan pl;
  const int rc = plan_tasks(&pl, m, n, offsets, batch, mode, tuning);
  if (rc != RADIC_OK) return rc;
  *n_tasks = (int64_t)(pl.t32.size() + pl.t64.size());
  int64_t i = 0;
  for (const std::vector<BatchTask>* list : {&pl.t32, &pl.t64}) {
    for (const BatchTask& t : *list) {
      if (i >= capacity) return RADIC_OK;
      int64_t* r = tasks + kTaskRow * i;
      r[0] = t.b;
      r[1] = t.tier;
      r[2] = t.kind;
      r[3] = t.shared;
      r[4] = t.v;
      r[5] = (int64_t)t.r0;
      r[6] = (int64_t)t.run;
      r[7] = (int64_t)t.lim;
      r[8] = t.vlo;
      r[9] = t.vhi;
      ++i;
    }
  }
  return RADIC_OK;
}

int radic_batch_plan_destroy(radic_batch_plan* plan) {
  delete plan;
  return RADIC_OK;
}

size_t radic_batch_workspace_bytes(const radic_batch_plan* plan) { return plan ? plan->ws_bytes : 0; }

int radic_batch_plan_info(const radic_batch_plan* plan, int64_t* info, int count) {
  if (!plan || (!info && count > 0) || count < 0 || count > RADIC_BATCH_INFO_COUNT) return RADIC_EINVAL;
  int64_t v[RADIC_BATCH_INFO_COUNT];
  v[0] = (int64_t)plan->t32.size() - plan->tasks_pair;
  v[1] = (int64_t)plan->t64.size();
  v[2] = plan->n_fp32_matrices;
  v[3] = plan->n_fp64_matrices;
  v[4] = (int64_t)plan->minors32;
  v[5] = (int64_t)plan->minors64;
  int64_t b32 = 0, b64 = 0, bp = 0;
  for (int g = 0; g < kGroups; ++g) {
    b32 = std::max<int64_t>(b32, plan->blocks[0][g]);
    bp = std::max<int64_t>(bp, plan->blocks[1][g]);
    b64 = std::max<int64_t>(b64, plan->blocks[2][g]);
  }
  v[6] = b32;
  v[7] = b64;
  v[8] = plan->tasks_pair;
  v[9] = plan->n_pair_matrices;
  v[10] = (int64_t)plan->minors_pair;
  v[11] = bp;
  v[12] = plan->launches;
  v[13] = plan->dom_group >= 0 ? plan->dom_group / kPaths : 0;
  v[14] = plan->dom_group >= 0 ? plan->dom_group % kPaths : 0;
  v[15] = plan->dom_queue < 0 ? -1 : (plan->dom_queue == 0 ? RADIC_MODE_MIXED : RADIC_MODE_PAIR);
  for (int i = 0; i < count; ++i) info[i] = v[i];
  return RADIC_OK;
}

int radic_batch_upload(const radic_batch_plan* plan, void* workspace, size_t workspace_bytes, void* stream) {
  if (!plan || !workspace) return RADIC_EINVAL;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < plan->ws_bytes) return RADIC_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  auto put = [&](size_t off, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(ws + off, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
  };
  bool ok = put(plan->off_t32, plan->t32.data(), plan->t32.size() * sizeof(BatchTask)) &&
            put(plan->off_t64, plan->t64.data(), plan->t64.size() * sizeof(BatchTask)) &&
            put(plan->off_csr_ptr, plan->csr_ptr.data(), plan->csr_ptr.size() * sizeof(int)) &&
            put(plan->off_csr_idx, plan->csr_idx.data(), plan->csr_idx.size() * sizeof(int)) &&
            put(plan->off_tier, plan->tier.data(), plan->tier.size() * sizeof(int)) &&
            put(plan->off_shape, plan->shape.data(), plan->shape.size() * sizeof(int));
  if (!ok) return RADIC_ECUDA;
  // the host vectors are pageable: wait until the copies have been consumed
  return cudaStreamSynchronize(s) == cudaSuccess ? RADIC_OK : RADIC_ECUDA;
}

int radic_det_batched(const radic_batch_plan* plan, const void* A, int dtype, radic_result* out, void* workspace,
                      size_t workspace_bytes, void* stream) {
  if (!plan || !A || !out || !workspace) return RADIC_EINVAL;
  if (dtype != RADIC_I8 && dtype != RADIC_I32 && dtype != RADIC_F32 && dtype != RADIC_F64) return RADIC_EINVAL;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < plan->ws_bytes) return RADIC_EWORKSPACE;
  return enqueue(plan, A, dtype, out, workspace, static_cast<cudaStream_t>(stream));
}

int radic_batch_graph_create(const radic_batch_plan* plan, const void* A, int dtype, radic_result* out,
                             void* workspace, size_t workspace_bytes, radic_batch_graph** graph) {
  if (!plan || !A || !out || !workspace || !graph) return RADIC_EINVAL;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < plan->ws_bytes) return RADIC_EWORKSPACE;
  *graph = nullptr;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return RADIC_ECUDA;
  radic_batch_graph* g = new (std::nothrow) radic_batch_graph;
  int rc = g ? RADIC_OK : RADIC_EINVAL;
  if (rc == RADIC_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = RADIC_ECUDA;
  if (rc == RADIC_OK) {
    const int r = enqueue(plan, A, dtype, out, workspace, cs);
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

int radic_batch_graph_launch(radic_batch_graph* graph, void* stream) {
  if (!graph || !graph->exec) return RADIC_EINVAL;
  return cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RADIC_OK : RADIC_ECUDA;
}

int radic_batch_graph_destroy(radic_batch_graph* graph) {
  if (!graph) return RADIC_OK;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  delete graph;
  return RADIC_OK;
}

}  // extern "C"
