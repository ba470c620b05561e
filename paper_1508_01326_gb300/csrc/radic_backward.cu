// Gradient of Radic's determinant with respect to the matrix entries.
//
// d det_R / d A[:, J] = sign(J) * adj(A[:, J])^T, the cofactor matrix of each
// minor, so the gradient of det_R(A) scatter-adds every minor's signed
// cofactors into the columns J of the gradient.  Per minor (one thread, in
// registers): partial-pivot LU P M = L U with the row order tracked in
// idx[], B = U^{-1} L^{-1} = M^{-1} P^T, and cofactor(idx[s], j) =
// det(M) * B[j][s].  A block owns one run of dictionary ranks of one matrix
// and adds its cofactors into a shared-memory copy of that matrix's gradient
// (shared-memory atomics); blocks write their tiles to per-block slots and a
// second kernel adds a matrix's slots in block order and scales by the
// incoming gradient.  Binary64 throughout.  A minor with an exactly zero
// pivot (singular) takes a slow path that forms its cofactors from
// (m-1) x (m-1) determinants.
//
// For 3 <= m the default kernel shares the work per (m-2)-column prefix, as
// the forward prefix kernels do, in binary64 or in pairs of binary32.  With the prefix rows T (pivot order) and B
// (the other two), A = A_TT, W = -A_BT A^{-1}, the Schur complement of a leaf
// (x, y) is S = [z(x) z(y)], z = x_B + W x_T, det(N) = det(A) det(S) for the
// row-permuted minor N, and by the block inverse
//   det(N) N^{-1} = det(A) [[det(S) A^{-1} - A^{-1} X_T adj(S) W, -A^{-1} X_T adj(S)],
//                           [adj(S) W,                            adj(S)]].
// Summed over the leaves of the prefix with their signs (column parities
// folded into z~ = (-1)^col z), every candidate column q receives
//   alpha (-1)^q [W^T; I] g_q,   g_q = rot(Z_>q - Z_<q),   rot(h) = (h1, -h0),
// where Z_<q and Z_>q are the sums of z~ over the columns before and after
// q, and the prefix columns receive alpha [s A^{-1} - A^{-1} Q W | -A^{-1} Q]^T
// with s = sum over leaves of det[z~_x z~_y] and
// Q = sum_q (-1)^q x_T(q) g_q^T.  A prefix thus costs O(m^2 (m-2) + k m)
// operations for its k candidate columns and its C(k, 2) leaves, and scatters
// m (m - 2 + k) gradient entries.  A prefix with an exactly zero pivot falls
// back to the per-minor cofactors for its leaves.
//
// Gathering those entries: each warp adds into its own gradient tile in
// shared memory (binary64 or pairs, as the kernel computes), without
// atomics, and the block adds its warps' tiles in warp order at the end.  The
// 32 lanes of a warp task hold prefixes with the same last column v, so they
// share the candidate columns and v: those columns are summed over the warp in
// registers (a reduce-scatter of the m rows, one lane per entry), v's entries
// first per lane over the lane's run.  Of the other prefix columns, the ones
// that change slowly in dictionary order are summed per lane in shared memory
// and added when the column moves on; the fastest one is added per prefix,
// lanes with the same column taking turns.  (Atomic binary64 additions to
// shared memory retry under contention; adding every entry that way, with 32
// lanes on one column, made them the bulk of the kernel.)
//
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "radic_prefix.cuh"

namespace radic {
namespace {

constexpr int kBwdThreads = 128;
constexpr int kBwdMaxM = 8;

struct BwdArgs {
  const double* A;
  long long lda, stride;  // row stride, matrix stride (elements)
  int batch, m, n;
  int chunks;             // blocks per matrix
  unsigned long long total;
  double* slots;          // batch x chunks x m x n
};

// Full partial-pivot LU with multipliers stored below the diagonal; idx[s] is
// the original row in slot s.  Returns det(M) and whether a pivot was zero.
template <int M>
__device__ __forceinline__ double lu_full(double (&a)[M][M], int (&idx)[M], bool& zero_pivot) {
  double det = 1.0;
  bool neg = false;
  zero_pivot = false;
#pragma unroll
  for (int i = 0; i < M; ++i) idx[i] = i;
#pragma unroll
  for (int k = 0; k < M; ++k) {
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const bool sw = mag_key(a[i][k]) > mag_key(a[k][k]);
#pragma unroll
      for (int j = 0; j < M; ++j) {
        const double x = a[k][j], y = a[i][j];
        a[k][j] = sw ? y : x;
        a[i][j] = sw ? x : y;
      }
      const int ik = idx[k], ii = idx[i];
      idx[k] = sw ? ii : ik;
      idx[i] = sw ? ik : ii;
      neg ^= sw;
    }
    const double piv = a[k][k];
    zero_pivot |= (piv == 0.0);
    det *= piv;
    const double r = rcp_f64(piv);
#pragma unroll
    for (int i = k + 1; i < M; ++i) {
      const double l = a[i][k] * r;
      a[i][k] = l;
#pragma unroll
      for (int j = k + 1; j < M; ++j) a[i][j] = fma(-l, a[k][j], a[i][j]);
    }
  }
  return neg ? -det : det;
}

// X = U^{-1} L^{-1} from the packed factors in a (L unit lower, U upper):
// first X = L^{-1} column by column (forward substitution), then, in place,
// X = U^{-1} X (back substitution).
template <int M, typename T = double>
__device__ __forceinline__ void inverse_factors(const T (&a)[M][M], T (&X)[M][M]) {
#pragma unroll
  for (int j = 0; j < M; ++j) {
#pragma unroll
    for (int i = 0; i < M; ++i) {
      if (i < j) X[i][j] = T(0);
      else if (i == j) X[i][j] = T(1);
      else {
        T s = -a[i][j];
#pragma unroll
        for (int k = j + 1; k < i; ++k) s = fma(-a[i][k], X[k][j], s);
        X[i][j] = s;
      }
    }
  }
  T rinv[M];
#pragma unroll
  for (int i = 0; i < M; ++i) rinv[i] = rcp_t(a[i][i]);
#pragma unroll
  for (int j = 0; j < M; ++j) {
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
      T s = X[i][j];
#pragma unroll
      for (int k = i + 1; k < M; ++k) s = fma(-a[i][k], X[k][j], s);
      X[i][j] = s * rinv[i];
    }
  }
}

// Slow path for a singular minor: cofactor(i, j) = (-1)^(i+j) det of M
// without row i and column j, by LU of each (m-1) x (m-1) submatrix.
template <int M>
__device__ __noinline__ void cofactors_slow(const double* As, int cs, const int (&c)[M], double (&cof)[M][M]) {
  for (int i = 0; i < M; ++i) {
    for (int j = 0; j < M; ++j) {
      double sub[M > 1 ? M - 1 : 1][M > 1 ? M - 1 : 1];
      int rr = 0;
      for (int r = 0; r < M; ++r) {
        if (r == i) continue;
        int cc = 0;
        for (int q = 0; q < M; ++q) {
          if (q == j) continue;
          sub[rr][cc++] = As[c[q] * cs + r];
        }
        ++rr;
      }
      double det = 1.0;
      bool neg = false;
      const int S = M - 1;
      for (int k = 0; k < S; ++k) {
        int p = k;
        for (int r = k + 1; r < S; ++r)
          if (fabs(sub[r][k]) > fabs(sub[p][k])) p = r;
        if (p != k) {
          for (int q = 0; q < S; ++q) {
            const double t = sub[k][q];
            sub[k][q] = sub[p][q];
            sub[p][q] = t;
          }
          neg = !neg;
        }
        const double piv = sub[k][k];
        det *= piv;
        if (piv == 0.0) break;
        for (int r = k + 1; r < S; ++r) {
          const double l = sub[r][k] / piv;
          for (int q = k + 1; q < S; ++q) sub[r][q] -= l * sub[k][q];
        }
      }
      if (neg) det = -det;
      cof[i][j] = ((i + j) & 1) ? -det : det;
    }
  }
}

template <int M>
__global__ void __launch_bounds__(kBwdThreads) k_backward(BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CS = ColStride<double, M>::value;
  const int n = a.n;
  const int b = blockIdx.y;
  const int chunk = blockIdx.x;
  uint64_t* binom = reinterpret_cast<uint64_t*>(smem_raw);
  size_t off = ((size_t)(n + 1) * (M + 1) * 8 + 15) / 16 * 16;
  double* As = reinterpret_cast<double*>(smem_raw + off);
  off += ((size_t)n * CS * 8 + 15) / 16 * 16;
  double* G = reinterpret_cast<double*>(smem_raw + off);  // M x n gradient tile
  build_binom(binom, n, M);
  const double* Ab = a.A + (long long)b * a.stride;
  for (int idx = threadIdx.x; idx < n * CS; idx += blockDim.x) {
    const int j = idx / CS, i = idx - j * CS;
    As[idx] = (i < M) ? Ab[(long long)i * a.lda + j] : 0.0;
  }
  for (int idx = threadIdx.x; idx < M * n; idx += blockDim.x) G[idx] = 0.0;
  __syncthreads();

  // this block's run of ranks, split evenly over its threads
  const unsigned long long per_chunk = (a.total + a.chunks - 1) / a.chunks;
  const unsigned long long c0 = (unsigned long long)chunk * per_chunk;
  const unsigned long long c1 = min(c0 + per_chunk, a.total);
  if (c0 < c1) {
    const unsigned long long per_thread = (c1 - c0 + blockDim.x - 1) / blockDim.x;
    const unsigned long long q0 = c0 + threadIdx.x * per_thread;
    const unsigned long long q1 = min(q0 + per_thread, c1);
    if (q0 < q1) {
      int c[M];
      unrank<M>(q0, n, binom, M + 1, c);
      for (unsigned long long q = q0; q < q1; ++q) {
        double mm[M][M];
        gather<double, M, CS>(As, c, mm);
        int idx[M];
        bool zp;
        const double det = lu_full<M>(mm, idx, zp);
        const double sgn = sign_negative<M>(c) ? -1.0 : 1.0;
        if (!zp) {
          double B[M][M];
          inverse_factors<M>(mm, B);
          const double s = sgn * det;
#pragma unroll
          for (int sl = 0; sl < M; ++sl) {
            double* grow = G + idx[sl] * n;
#pragma unroll
            for (int j = 0; j < M; ++j) atomicAdd(grow + c[j], s * B[j][sl]);
          }
        } else {
          double cof[M][M];
          cofactors_slow<M>(As, CS, c, cof);
          for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) atomicAdd(G + i * n + c[j], sgn * cof[i][j]);
        }
        if (q + 1 < q1) successor<M>(c, n);
      }
    }
  }
  __syncthreads();
  double* slot = a.slots + ((size_t)b * a.chunks + chunk) * (size_t)M * n;
  for (int idx = threadIdx.x; idx < M * n; idx += blockDim.x) slot[idx] = G[idx];
}

// Signed cofactors of one minor read from the binary64 matrix in global
// memory (row stride lda), added into the gradient tile G.
template <int M>
__device__ __noinline__ void minor_cofactors_scatter_global(const double* Ab, long long lda, const int (&c)[M],
                                                            double* G, int n) {
  constexpr int CSG = ColStride<double, M>::value;
  double col[M * CSG];
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < CSG; ++i) col[j * CSG + i] = (i < M) ? Ab[(long long)i * lda + c[j]] : 0.0;
  int cl[M];
  for (int j = 0; j < M; ++j) cl[j] = j;
  double mm[M][M];
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) mm[i][j] = col[j * CSG + i];
  int idx[M];
  bool zp;
  const double det = lu_full<M>(mm, idx, zp);
  const double sgn = sign_negative<M>(c) ? -1.0 : 1.0;
  if (!zp) {
    double B[M][M];
    inverse_factors<M>(mm, B);
    const double s = sgn * det;
    for (int sl = 0; sl < M; ++sl)
      for (int j = 0; j < M; ++j) atomicAdd(G + idx[sl] * n + c[j], s * B[j][sl]);
  } else {
    double cof[M][M];
    cofactors_slow<M>(col, CSG, cl, cof);
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) atomicAdd(G + i * n + c[j], sgn * cof[i][j]);
  }
}

__device__ __forceinline__ bool pivot_greater(double x, double y) { return mag_key(x) > mag_key(y); }
__device__ __forceinline__ bool pivot_greater(ff x, ff y) { return fabsf(x.hi) > fabsf(y.hi); }
__device__ __forceinline__ bool is_zero(double x) { return x == 0.0; }
__device__ __forceinline__ bool is_zero(ff x) { return x.hi == 0.0f; }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(ff x) { return static_cast<double>(x); }

__device__ __forceinline__ double shfl_x(double x, int off) { return __shfl_xor_sync(kFull, x, off); }
__device__ __forceinline__ ff shfl_x(ff x, int off) {
  return ff(__shfl_xor_sync(kFull, x.hi, off), __shfl_xor_sync(kFull, x.lo, off));
}

// Adds the sum over the warp's 32 lanes of v[0..M-1] (one value per row of
// the matrix) to column `tcol` of the warp's gradient tile.  Three exchange
// steps on lane bits 4, 3 and 2 halve the vector each time (a
// reduce-scatter), so each group of four lanes ends with one row summed over
// eight lanes; two butterfly steps on bits 1 and 0 finish the sum, and the
// group's first lane adds it in: one lane per entry, so no atomics.  Nine
// additions and nine exchanges per lane.  Every lane of the warp must call it.
template <typename T, int M>
__device__ __forceinline__ void warp_add_column(const T (&v)[M], T* tcol, int n, int lane) {
  static_assert(M <= 8, "rows are spread over lane bits 4..2");
  T p[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) p[j] = T(0);
#pragma unroll
  for (int j = 0; j < M; ++j) p[j] = v[j];
  const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
  T w4[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T keep = b4 ? p[j + 4] : p[j], send = b4 ? p[j] : p[j + 4];
    w4[j] = keep + shfl_x(send, 16);
  }
  T w2[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T keep = b3 ? w4[j + 2] : w4[j], send = b3 ? w4[j] : w4[j + 2];
    w2[j] = keep + shfl_x(send, 8);
  }
  T w = (b2 ? w2[1] : w2[0]) + shfl_x(b2 ? w2[0] : w2[1], 4);
  w = w + shfl_x(w, 2);
  w = w + shfl_x(w, 1);
  const int row = (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0);
  if ((lane & 3) == 0 && row < M) tcol[row * n] += w;
  __syncwarp();
}

// The same for two adjacent columns at once: lane bit 4 picks the column and
// bits 3..1 the row, so the five exchange steps serve both columns (at most
// fourteen additions per lane for m <= 8) and lanes with bit 0 clear add the
// sums.  `second` (the same on every lane) says whether column tcol + 1 exists.
template <typename T, int M>
__device__ __forceinline__ void warp_add_columns2(const T (&va)[M], const T (&vb)[M], T* tcol, int n, int lane,
                                                  bool second) {
  static_assert(M <= 8, "rows are spread over lane bits 3..1");
  const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0, b1 = (lane & 2) != 0;
  T w8[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) w8[j] = T(0);
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const T keep = b4 ? vb[j] : va[j], send = b4 ? va[j] : vb[j];
    w8[j] = keep + shfl_x(send, 16);
  }
  T w4[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T keep = b3 ? w8[j + 4] : w8[j], send = b3 ? w8[j] : w8[j + 4];
    w4[j] = keep + shfl_x(send, 8);
  }
  T w2[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T keep = b2 ? w4[j + 2] : w4[j], send = b2 ? w4[j] : w4[j + 2];
    w2[j] = keep + shfl_x(send, 4);
  }
  T w = (b1 ? w2[1] : w2[0]) + shfl_x(b1 ? w2[0] : w2[1], 2);
  w = w + shfl_x(w, 1);
  const int row = (b3 ? 4 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0);
  if ((lane & 1) == 0 && row < M && (!b4 || second)) tcol[(b4 ? 1 : 0) + row * n] += w;
  __syncwarp();
}

// Adds u[0..M-1] to rows 0..M-1 of column `key` of the warp's tile for the
// lanes with key >= 0.  Lanes with the same column take turns, in lane order,
// one round per lane of the largest such group, so no two lanes write one
// entry in the same round.  Every lane of the warp must call it.
template <typename T, int M>
__device__ __forceinline__ void warp_tile_add(T* tile, int n, int key, const T (&u)[M], int lane) {
  const unsigned grp = __match_any_sync(kFull, key);
  const unsigned rank = __popc(grp & ((1u << lane) - 1u));
  const unsigned rounds = __reduce_max_sync(kFull, key >= 0 ? (unsigned)__popc(grp) : 0u);
  for (unsigned it = 0; it < rounds; ++it) {
    if (key >= 0 && rank == it) {
#pragma unroll
      for (int i = 0; i < M; ++i) tile[i * n + key] += u[i];
    }
    __syncwarp();
  }
}

// u[rho] = x[r] for the slot r with idx[r] == rho: values in pivot order back
// to the matrix's row order (selects only, no indexed registers).
template <typename T, int M>
__device__ __forceinline__ void unpermute(const T (&x)[M], const int (&idx)[M], T (&u)[M]) {
#pragma unroll
  for (int rho = 0; rho < M; ++rho) {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < M; ++r) s = (idx[r] == rho) ? x[r] : s;
    u[rho] = s;
  }
}

template <typename T, int M>
__global__ void __launch_bounds__(kBwdThreads) k_backward_prefix(BwdArgs a, PrefixTable tab) {
  constexpr int D = 2, P = M - D;
  // head positions 0 .. P-3 change slowly in dictionary order and are summed
  // per lane in shared memory (NS of them); position P-2 changes with every
  // prefix and is added directly; column v is the same for the whole warp
  constexpr int NS = P > 2 ? P - 2 : 0;
  constexpr int CS = ColStride<T, M>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n;
  const int b = blockIdx.y, chunk = blockIdx.x;
  uint64_t* binom = reinterpret_cast<uint64_t*>(smem_raw);
  size_t off = ((size_t)(n + 1) * (M + 1) * 8 + 15) / 16 * 16;
  T* As = reinterpret_cast<T*>(smem_raw + off);
  off += ((size_t)n * CS * sizeof(T) + 15) / 16 * 16;
  double* G = reinterpret_cast<double*>(smem_raw + off);  // M x n tile of the singular-prefix path
  off += ((size_t)M * n * 8 + 15) / 16 * 16;
  const ZBuf<T, D> zb(smem_raw + off, threadIdx.x, blockDim.x, n - M + D);
  off += (zbuf_bytes(n - M + D, blockDim.x, D, 8) + 15) / 16 * 16;
  T* Hacc = reinterpret_cast<T*>(smem_raw + off) + threadIdx.x;  // [NS][M] per lane, lane-strided
  off += (size_t)NS * M * blockDim.x * sizeof(T);
  T* Gall = reinterpret_cast<T*>(smem_raw + off);  // one M x n tile per warp
  build_binom(binom, n, M);
  const double* Ab = a.A + (long long)b * a.stride;
  for (int idx = threadIdx.x; idx < n * CS; idx += blockDim.x) {
    const int j = idx / CS, i = idx - j * CS;
    As[idx] = (i < M) ? to_elem<T>(Ab[(long long)i * a.lda + j]) : T(0);
  }
  for (int idx = threadIdx.x; idx < M * n; idx += blockDim.x) G[idx] = 0.0;
  for (int idx = threadIdx.x; idx < (int)(blockDim.x >> 5) * M * n; idx += blockDim.x) Gall[idx] = T(0);
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int bs = M + 1;
  const int hs = blockDim.x;
  T* Gw = Gall + (size_t)warp * M * n;  // stride between a lane's accumulator entries
  for (unsigned long long t = (unsigned long long)chunk * wpb + warp; t < tab.total_tasks;
       t += (unsigned long long)a.chunks * wpb) {
    // everything up to the step loop is the same for the 32 lanes of the task
    int v = tab.v_lo;
    while (v < tab.v_hi && t >= tab.task_start[v + 1]) ++v;
    const unsigned long long runlen = tab.run[v], cnt = tab.count[v];
    const unsigned long long r0 = (t - tab.task_start[v]) * 32ull * runlen + (unsigned long long)lane * runlen;
    const unsigned long long r1 = min(r0 + runlen, cnt);
    const bool ever = r0 < r1;  // true for lane 0: a task starts below cnt
    constexpr int H = P > 1 ? P - 1 : 1;
    int head[H];
    if constexpr (P > 1) unrank<P - 1>(ever ? r0 : cnt - 1, v, binom, bs, head);
    const int k = n - 1 - v;
    T vacc[M];
#pragma unroll
    for (int i = 0; i < M; ++i) vacc[i] = T(0);
    int hcol[NS > 0 ? NS : 1];
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      hcol[p] = head[p];
#pragma unroll
      for (int i = 0; i < M; ++i) Hacc[(p * M + i) * hs] = T(0);
    }
    // lanes past their run repeat their last prefix with zero weight, so that
    // the whole warp takes every step (the column sums exchange registers)
    for (unsigned long long st = 0; st < runlen; ++st) {
      const unsigned long long r = r0 + st;
      const bool live = r < r1;
      int c[P];
#pragma unroll
      for (int j = 0; j < P - 1; ++j) c[j] = head[j];
      c[P - 1] = v;
      // factor the M x P prefix: partial pivoting, L \ U packed in fa
      T fa[M][P];
#pragma unroll
      for (int j = 0; j < P; ++j)
#pragma unroll
        for (int i = 0; i < M; ++i) fa[i][j] = As[c[j] * CS + i];
      int idx[M];
#pragma unroll
      for (int i = 0; i < M; ++i) idx[i] = i;
      bool neg = false, zp = false;
      T prod = T(1);
#pragma unroll
      for (int kk = 0; kk < P; ++kk) {
#pragma unroll
        for (int i = kk + 1; i < M; ++i) {
          const bool sw = pivot_greater(fa[i][kk], fa[kk][kk]);
#pragma unroll
          for (int j = 0; j < P; ++j) {
            const T x = fa[kk][j], y = fa[i][j];
            fa[kk][j] = sw ? y : x;
            fa[i][j] = sw ? x : y;
          }
          const int ik = idx[kk], ii = idx[i];
          idx[kk] = sw ? ii : ik;
          idx[i] = sw ? ik : ii;
          neg ^= sw;
        }
        const T piv = fa[kk][kk];
        zp |= is_zero(piv);
        prod *= piv;
        const T rr = rcp_t(piv);
#pragma unroll
        for (int i = kk + 1; i < M; ++i) {
          const T l = fa[i][kk] * rr;
          fa[i][kk] = l;
#pragma unroll
          for (int j = kk + 1; j < P; ++j) fa[i][j] = fma(-l, fa[kk][j], fa[i][j]);
        }
      }
      if (live && zp) {  // singular prefix: per-minor cofactors of its leaves
        for (int x = v + 1; x < n; ++x)
          for (int y = x + 1; y < n; ++y) {
            int cm[M];
            for (int j = 0; j < P; ++j) cm[j] = c[j];
            cm[P] = x;
            cm[P + 1] = y;
            minor_cofactors_scatter_global<M>(Ab, a.lda, cm, G, n);
          }
      }
      // below, a singular or repeated prefix runs with non-finite or unwanted
      // values that `use` replaces by zeros
      const bool use = live && !zp;
      // W = -L21 L11^{-1} (D x P) and Ainv = U11^{-1} L11^{-1} (P x P)
      T W[D][P];
#pragma unroll
      for (int d = 0; d < D; ++d) {
#pragma unroll
        for (int j = P - 1; j >= 0; --j) {
          T sum = -fa[P + d][j];
#pragma unroll
          for (int i = j + 1; i < P; ++i) sum = fma(-W[d][i], fa[i][j], sum);
          W[d][j] = sum;
        }
      }
      T Ai[P][P];
      {
        T top[P][P];
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
          for (int j = 0; j < P; ++j) top[i][j] = fa[i][j];
        inverse_factors<P, T>(top, Ai);
      }
      int sp = M * (M + 1) / 2 + D;
#pragma unroll
      for (int j = 0; j < P; ++j) sp += c[j] + 1;
      const T alpha = ((sp & 1) != neg) ? -prod : prod;
      // pass 1: z~ of every candidate column, their sum, and s
      T zt0 = T(0), zt1 = T(0), ssum = T(0);
      for (int q = 0; q < k; ++q) {
        const int col = v + 1 + q;
        T z[D];
        prefix_column<T, M, D>(As + col * CS, W, idx, z);
        if (col & 1) {
          z[0] = -z[0];
          z[1] = -z[1];
        }
        ssum = fma(zt0, z[1], fma(-zt1, z[0], ssum));  // det[Z_<q, z~_q]
        zt0 += z[0];
        zt1 += z[1];
        zb.put(q, z);
      }
      // the gradient of candidate column q at pivot slot r is
      // (-1)^q alpha ([W^T; I] g_q)[r]; Ca, Cb hold [W^T; I] in row order
      T Ca[M], Cb[M];
      {
        T ca[M], cb[M];
#pragma unroll
        for (int r = 0; r < M; ++r) {
          ca[r] = r < P ? W[0][r < P ? r : 0] : (r == P ? T(1) : T(0));
          cb[r] = r < P ? W[1][r < P ? r : 0] : (r == P + 1 ? T(1) : T(0));
        }
        unpermute<T, M>(ca, idx, Ca);
        unpermute<T, M>(cb, idx, Cb);
      }
      // pass 2: candidate-column gradients (summed over the warp) and Q
      T Q[P][D];
#pragma unroll
      for (int i = 0; i < P; ++i) Q[i][0] = Q[i][1] = T(0);
      T zp0 = T(0), zp1 = T(0);
      auto column = [&](int q, T (&val)[M]) {
        const int col = v + 1 + q;
        T z[D];
        zb.get(q, z);
        const T h0 = zt0 - (zp0 + zp0) - z[0], h1 = zt1 - (zp1 + zp1) - z[1];
        const T g0 = h1, g1 = -h0;  // rot(Z_>q - Z_<q)
        zp0 += z[0];
        zp1 += z[1];
        const T sc = (col & 1) ? -alpha : alpha;
#pragma unroll
        for (int i = 0; i < M; ++i) val[i] = use ? sc * fma(Ca[i], g0, Cb[i] * g1) : T(0);
        const T* xc = As + col * CS;
#pragma unroll
        for (int i = 0; i < P; ++i) {
          const T xt = (col & 1) ? -xc[idx[i]] : xc[idx[i]];
          Q[i][0] = fma(xt, g0, Q[i][0]);
          Q[i][1] = fma(xt, g1, Q[i][1]);
        }
      };
      if constexpr (std::is_same<T, ff>::value) {
        // pairs: one column per warp sum (the column body is long; inlining
        // it twice measured slower, with instruction-fetch stalls)
        for (int q = 0; q < k; ++q) {
          T va[M];
          column(q, va);
          warp_add_column<T, M>(va, Gw + v + 1 + q, n, lane);
        }
      } else {
        for (int q = 0; q < k; q += 2) {  // binary64: two columns per warp sum
          const bool two = q + 1 < k;
          T va[M], vb[M];
          column(q, va);
          if (two) {
            column(q + 1, vb);
          } else {
#pragma unroll
            for (int i = 0; i < M; ++i) vb[i] = T(0);
          }
          warp_add_columns2<T, M>(va, vb, Gw + v + 1 + q, n, lane, two);
        }
      }
      // prefix columns: alpha [s Ainv - Ainv Q W | -Ainv Q]^T, formed in row
      // order: with a = (Ainv row tt, 0, 0) in pivot order, row idx[r] of
      // column c[tt] receives alpha (s a[r] - (Ainv Q)[tt] . [W^T; I][r])
#pragma unroll
      for (int tt = 0; tt < P; ++tt) {
        T R0 = T(0), R1 = T(0);  // (Ainv Q)[tt][:]
#pragma unroll
        for (int u = 0; u < P; ++u) {
          R0 = fma(Ai[tt][u], Q[u][0], R0);
          R1 = fma(Ai[tt][u], Q[u][1], R1);
        }
        T ai[M], air[M];
#pragma unroll
        for (int r = 0; r < M; ++r) ai[r] = r < P ? Ai[tt][r < P ? r : 0] : T(0);
        unpermute<T, M>(ai, idx, air);
        T u[M];
#pragma unroll
        for (int i = 0; i < M; ++i) u[i] = alpha * (ssum * air[i] - fma(R0, Ca[i], R1 * Cb[i]));
        if (tt == P - 1) {
#pragma unroll
          for (int i = 0; i < M; ++i) vacc[i] += use ? u[i] : T(0);
        } else if (tt < NS) {
#pragma unroll
          for (int i = 0; i < M; ++i) {
            T& h = Hacc[(tt * M + i) * hs];
            h += use ? u[i] : T(0);
          }
        } else {
          warp_tile_add<T, M>(Gw, n, use ? c[tt] : -1, u, lane);
        }
      }
      if constexpr (P > 1) {
        const bool adv = r + 1 < r1;
        if (adv) successor<P - 1>(head, v);
#pragma unroll
        for (int p = 0; p < NS; ++p) {
          const bool moved = adv && head[p] != hcol[p];
          if (__any_sync(kFull, moved)) {  // a slow head column moved on: add its sum
            T u[M];
#pragma unroll
            for (int i = 0; i < M; ++i) u[i] = Hacc[(p * M + i) * hs];
            warp_tile_add<T, M>(Gw, n, moved ? hcol[p] : -1, u, lane);
            if (moved) {
#pragma unroll
              for (int i = 0; i < M; ++i) Hacc[(p * M + i) * hs] = T(0);
              hcol[p] = head[p];
            }
          }
        }
      }
    }
    // the task's sums of column v and of the slow head columns
    warp_add_column<T, M>(vacc, Gw + v, n, lane);
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      T u[M];
#pragma unroll
      for (int i = 0; i < M; ++i) u[i] = Hacc[(p * M + i) * hs];
      const int c0 = __shfl_sync(kFull, hcol[p], 0);
      if (__all_sync(kFull, !ever || hcol[p] == c0)) {
        warp_add_column<T, M>(u, Gw + c0, n, lane);
      } else {
        warp_tile_add<T, M>(Gw, n, ever ? hcol[p] : -1, u, lane);
      }
    }
  }
  __syncthreads();
  // the block's tile: the singular-prefix entries plus the warps' tiles in
  // warp order
  double* slot = a.slots + ((size_t)b * a.chunks + chunk) * (size_t)M * n;
  for (int idx = threadIdx.x; idx < M * n; idx += blockDim.x) {
    double sum = G[idx];
    for (int w = 0; w < wpb; ++w) sum += to_double(Gall[(size_t)w * M * n + idx]);
    slot[idx] = sum;
  }
}

// grad_A[b] = grad_out[b] * sum over chunks (in order) of the tiles.
__global__ void k_backward_reduce(const double* slots, int batch, int m, int n, int chunks, const double* grad_out,
                                  double* grad, long long lda, long long stride) {
  const long long total = (long long)batch * m * n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / (m * n));
    const int e = (int)(t - (long long)b * m * n);
    const int i = e / n, j = e - i * n;
    double s = 0.0;
    for (int k = 0; k < chunks; ++k) s += slots[((size_t)b * chunks + k) * (size_t)m * n + e];
    grad[(long long)b * stride + (long long)i * lda + j] = s * grad_out[b];
  }
}

const void* bwd_kernel(int m) {
  switch (m) {
    case 1: return reinterpret_cast<const void*>(&k_backward<1>);
    case 2: return reinterpret_cast<const void*>(&k_backward<2>);
    case 3: return reinterpret_cast<const void*>(&k_backward<3>);
    case 4: return reinterpret_cast<const void*>(&k_backward<4>);
    case 5: return reinterpret_cast<const void*>(&k_backward<5>);
    case 6: return reinterpret_cast<const void*>(&k_backward<6>);
    case 7: return reinterpret_cast<const void*>(&k_backward<7>);
    case 8: return reinterpret_cast<const void*>(&k_backward<8>);
    default: return nullptr;
  }
}

template <typename T, int M>
const void* bwd_prefix_kernel_m() {
  if constexpr (M >= 3) return reinterpret_cast<const void*>(&k_backward_prefix<T, M>);
  else return nullptr;
}

template <typename T>
const void* bwd_prefix_kernel(int m) {
  switch (m) {
    case 3: return bwd_prefix_kernel_m<T, 3>();
    case 4: return bwd_prefix_kernel_m<T, 4>();
    case 5: return bwd_prefix_kernel_m<T, 5>();
    case 6: return bwd_prefix_kernel_m<T, 6>();
    case 7: return bwd_prefix_kernel_m<T, 7>();
    case 8: return bwd_prefix_kernel_m<T, 8>();
    default: return nullptr;
  }
}

// Work split of the prefix backward: prefixes grouped by their last column v
// (k = n-1-v candidate columns), warp tasks of 32 lanes x a run of prefixes,
// run lengths from a cost model (factorisation m P^2 + P^3, per candidate
// column m + 4P and 2(m + P) gradient entries), `chunks` blocks per matrix.
void bwd_prefix_plan(int batch, int m, int n, int sms, int* chunks, PrefixTable* tab) {
  const int P = m - 2;
  PrefixTable t;
  std::memset(&t, 0, sizeof(t));
  t.v_lo = P - 1;
  t.v_hi = n - 3;
  double cost[kMaxN] = {0}, total = 0.0;
  for (int v = t.v_lo; v <= t.v_hi; ++v) {
    const int k = n - 1 - v;
    t.count[v] = binom_host(v, P - 1);
    cost[v] = (double)m * P * P + (double)P * P * P + (double)k * (3.0 * m + 6.0 * P);
    total += cost[v] * (double)t.count[v];
  }
  const long long want = (long long)(sms > 0 ? sms : 1) * 16;  // about 16 blocks per SM in all
  long long ch = (want + batch - 1) / batch;
  if (ch > 65535) ch = 65535;
  if (ch < 1) ch = 1;
  const double per_lane = total / ((double)ch * kBwdThreads) / 2.0;  // about two tasks per warp
  unsigned long long start = 0;
  for (int v = t.v_lo; v <= t.v_hi; ++v) {
    double r = per_lane / cost[v];
    unsigned long long run = r < 1.0 ? 1ull : (unsigned long long)r;
    const unsigned long long maxrun = (t.count[v] + 31) / 32;
    if (run > maxrun) run = maxrun > 0 ? maxrun : 1;
    t.lanes[v] = 1;
    t.run[v] = run;
    t.task_start[v] = start;
    start += (t.count[v] + 32 * run - 1) / (32 * run);
  }
  if (t.v_hi + 1 < kMaxN) t.task_start[t.v_hi + 1] = start;
  t.total_tasks = start;
  *chunks = (int)ch;
  *tab = t;
}

size_t bwd_prefix_smem(int m, int n) {  // binary64 and pair elements are both 8 bytes
  const int cs = ((m + 1) / 2) * 2;
  size_t off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
  off += ((size_t)n * cs * 8 + 15) / 16 * 16;
  off += ((size_t)m * n * 8 + 15) / 16 * 16;
  off += (zbuf_bytes(n - m + 2, kBwdThreads, 2, 8) + 15) / 16 * 16;
  const int ns = m - 2 > 2 ? m - 4 : 0;  // per-lane sums of the slow head columns
  off += (size_t)ns * m * kBwdThreads * 8;
  off += (size_t)(kBwdThreads / 32) * m * n * 8;  // the warps' gradient tiles
  return off;
}

int bwd_chunks(int batch, unsigned long long total) {
  const int sms = device_sm_count();
  const long long want = (long long)(sms > 0 ? sms : 1) * 16;  // about 16 blocks per SM in all
  long long ch = (want + batch - 1) / batch;
  const long long by_work = (long long)((total + 4095) / 4096);  // at least ~32 minors per thread
  if (ch > by_work) ch = by_work;
  if (ch < 1) ch = 1;
  if (ch > 65535) ch = 65535;
  return (int)ch;
}

size_t bwd_smem(int m, int n) {
  const int cs = ((m + 1) / 2) * 2;
  size_t off = ((size_t)(n + 1) * (m + 1) * 8 + 15) / 16 * 16;
  off += ((size_t)n * cs * 8 + 15) / 16 * 16;
  off += (size_t)m * n * 8;
  return off;
}

}  // namespace
}  // namespace radic

using namespace radic;

extern "C" {

size_t radic_backward_workspace_bytes(int batch, int m, int n) {
  if (batch < 1 || m < 1 || m > kBwdMaxM || n < 1 || n > kMaxN) return 0;
  const unsigned long long total = (m <= n) ? binom_host(n, m) : 0ull;
  int chunks = bwd_chunks(batch, total);
  if (m >= 3 && m <= n) {
    PrefixTable tab;
    bwd_prefix_plan(batch, m, n, device_sm_count(), &chunks, &tab);
  }
  return align_up((size_t)batch * chunks * m * n * sizeof(double), 256) + 256;
}

int radic_det_backward(const double* A, int batch, int m, int n, int64_t lda, int64_t stride, const double* grad_out,
                       double* grad_A, void* workspace, size_t workspace_bytes, void* stream) {
  return radic_det_backward_mode(A, batch, m, n, lda, stride, grad_out, grad_A, workspace, workspace_bytes,
                                 RADIC_MODE_FP64, stream);
}

int radic_det_backward_mode(const double* A, int batch, int m, int n, int64_t lda, int64_t stride,
                            const double* grad_out, double* grad_A, void* workspace, size_t workspace_bytes, int mode,
                            void* stream) {
  if (!A || !grad_out || !grad_A || batch < 1 || m < 1 || n < 1 || n > kMaxN || lda < n || stride < (int64_t)m * lda)
    return RADIC_EINVAL;
  if (mode != RADIC_MODE_FP64 && mode != RADIC_MODE_PAIR) return RADIC_EINVAL;
  if (m > kBwdMaxM) return RADIC_EUNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (m > n) {  // det_R is identically zero: zero gradient
    for (int b = 0; b < batch; ++b)
      if (cudaMemset2DAsync(grad_A + (long long)b * stride, lda * sizeof(double), 0, n * sizeof(double), m, s) !=
          cudaSuccess)
        return RADIC_ECUDA;
    return RADIC_OK;
  }
  const size_t need = radic_backward_workspace_bytes(batch, m, n);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u) || workspace_bytes < need) return RADIC_EWORKSPACE;
  BwdArgs a;
  a.A = A;
  a.lda = lda;
  a.stride = stride;
  a.batch = batch;
  a.m = m;
  a.n = n;
  a.total = binom_host(n, m);
  a.chunks = bwd_chunks(batch, a.total);
  a.slots = static_cast<double*>(workspace);
  PrefixTable tab;
  const void* k;
  size_t smem;
  if (m >= 3) {  // prefix-shared backward
    bwd_prefix_plan(batch, m, n, device_sm_count(), &a.chunks, &tab);
    k = (mode == RADIC_MODE_PAIR) ? bwd_prefix_kernel<ff>(m) : bwd_prefix_kernel<double>(m);
    smem = bwd_prefix_smem(m, n);
  } else {
    k = bwd_kernel(m);
    smem = bwd_smem(m, n);
  }
  if (!k || !allow_smem(k, smem)) return RADIC_EUNSUPPORTED;
  void* params[] = {&a, &tab};
  if (cudaLaunchKernel(k, dim3(a.chunks, batch), dim3(kBwdThreads), params, smem, s) != cudaSuccess)
    return RADIC_ECUDA;
  const long long total = (long long)batch * m * n;
  const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 65535);
  const double* slots = a.slots;
  int bb = batch, mm = m, nn = n, ch = a.chunks;
  long long l = lda, st = stride;
  void* rparams[] = {&slots, &bb, &mm, &nn, &ch, &grad_out, &grad_A, &l, &st};
  if (cudaLaunchKernel(reinterpret_cast<const void*>(&k_backward_reduce), dim3(blocks), dim3(256), rparams, 0, s) !=
      cudaSuccess)
    return RADIC_ECUDA;
  return RADIC_OK;
}

}  // extern "C"
