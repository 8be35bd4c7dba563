// Batched persistent solve of many independent scenes (serving-style batches of uneven size).
//
// One persistent launch walks a work queue of scenes in descending size order; each CTA takes
// the next scene and runs the whole Riemannian staircase for it on the chip (Alg. 1 with
// RTR-tCG of Sec. 3.2, the Thm. 1 certificate, the Thm. 2 escape, the Sec. 2.2 rounding) with
// block-level reductions instead of grid-wide ones: no host round trip and no inter-CTA
// synchronisation.  Per-scene Q (n_s <= a few thousand) is kept dense and full in FP32 (all the
// bulk sweeps, HVPs and certificate products) and FP64 (polish gradients, objective, rounding),
// row-major with the row length padded to a multiple of 4.  The sweep is a block-row product:
// each warp owns RPW consecutive rows per step, lanes stride over 16-byte column chunks, Y is
// staged in shared memory.  RPW is chosen per scene-size class by an autotuner that times the
// candidates on the batch itself (xm_batch_autotune).
//
// The mixed-precision schedule matches xm_solve's XM_FP32_BULK mode: FP32 RTR-tCG to the bulk
// tolerance, a 30-step quick certificate, an FP64-gradient polish with FP32 HVPs, then the
// Lanczos certificate with FP64 vectors and Ritz values and the FP64 stationarity check.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "xm_internal.cuh"
#include "xm_ops.cuh"

namespace xm {
namespace bat {

constexpr int NT = 256;            // threads per CTA
constexpr int NW = NT / 32;
// Krylov steps of the quick certificate before the polish: it only looks for a strongly negative
// direction to escape along (lambda_min < -1e-4 |lambda_max|), which Lanczos finds among its
// first Ritz values; the full certificate after the polish decides (60 steps had cost ~5 % more)
constexpr int KQUICK = 30;
// Automatic team sizes (xm_batch_cluster cs = 0, n_min = 0), in units of the smallest n whose
// n^2 outweighs one SM's share of the batch's sum of n^2: scenes from QUAD_FACTOR times that on
// 4-CTA clusters when at least two reach it (at most one SM in 16 per quad scene), pairs from
// PAIR_FACTOR times it beside them.  Chosen by a list-scheduling model on the measured per-scene
// times of the 256-scene batch for 1, 2 and 4 CTAs (47 ms against 52 ms for pairs alone).
constexpr double QUAD_FACTOR = 1.8;
constexpr double PAIR_FACTOR = 1.3;
constexpr int NVEC = 17;           // per-slot vectors of NM x 8 doubles
constexpr int NCLASS = 4;          // scene-size classes of the tiling table
constexpr int XM_BATCH_KMAX = 400;       // Krylov cap of the batched certificate (shared memory)
constexpr int XM_BATCH_HANDOVER = 100;   // internal status: continued by the rank-8 kernel

__host__ __device__ inline int size_class(int n) { return n <= 150 ? 0 : (n <= 450 ? 1 : (n <= 900 ? 2 : 3)); }

struct Desc {                      // one scene (device table, in queue order)
  int N, n, ldq, scene;            // cameras, 3N, padded row length, index in the caller's order
  int64_t q32, q64;                // element offsets of the dense Q copies
  int64_t cam0;                    // first camera of the scene in the per-camera outputs
  int64_t spill;                   // offset of the scene's hand-over area (n x 8 + n doubles)
};

struct Params {
  const Desc* desc;
  int S;
  const float* Q32;
  const double* Q64;
  double* slots;                   // per-CTA scratch
  int64_t slot_doubles;
  int NM;                          // max ldq over the batch
  int kmax;                        // Krylov cap of the final certificate
  double* spill;                   // per-scene hand-over from the rank-4 to the rank-8 kernel
  double* R_out;                   // sum N x 9
  double* s_out;                   // sum N
  xm_batch_info* out;              // S entries, indexed by the caller's scene order
  unsigned* queue;                 // work-queue counter
  int tile[NCLASS];                // sweep tiling variant per size class
  xm_opts o;
  double mu;                       // App. D weight
  unsigned long long time_limit_ns;  // per-scene wall-clock cap (0: none)
  int team_min_n;                  // scenes with n >= this run on a whole cluster
  int pf_dist;                     // L2 prefetch distance of the sweeps (rounds; 0: none)
  int slot_base;                   // first per-CTA slot of this launch (launches side by side)
  // after this launch's own queue (desc[0..S)): its CTAs continue one by one on a second queue
  // shared with the launch beside it (null: none)
  unsigned* queue2;
  const Desc* desc2;
  int S2;
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------------ CTA reductions
// Deterministic CTA sum of K values: warp butterflies, then the warp partials in warp order;
// every thread returns the totals.  red: NW * K doubles of shared memory.
// CTA sum of K values per thread, the same on every thread: warp sums, then thread k adds the
// NW warp sums of value k in warp order and publishes it (one warp's FP64 adds instead of every
// thread's: B300's FP64 pipe is narrow).  K <= 64.
__shared__ double s_bsum[64];
template <int K>
__device__ __forceinline__ void bsum(double (&v)[K], double* red) {
  static_assert(K <= 64, "bsum: K <= 64");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double x = warp_sum(v[k]);
    if (lane == 0) red[wid * K + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += red[w * K + threadIdx.x];
    s_bsum[threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = s_bsum[k];
}

// ------------------------------------------------------------------ thread-block clusters
// A large scene may run on a team of CS CTAs, one thread-block cluster (xm_batch_cluster): every
// CTA of the team executes the same solver on the same data (identical arithmetic, hence
// identical branches), each computes a contiguous share of the rows of every Q product and
// stores it into all the team's copies of the product (distributed shared memory), between two
// cluster barriers.  Only rank 0 claims work, reads the clock for the time limit and writes
// results.  The queue is ordered by size; at the first scene below the team threshold the
// cluster splits up for good and its CTAs claim scenes one by one (no cluster barrier or
// distributed-shared-memory access after that point).
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// CTAs working on the current scene: the cluster size until the cluster splits up, then 1
__shared__ int s_team;
__device__ __forceinline__ int team() { return s_team; }
// this CTA writes the scene's results (alone, or rank 0 of its team)
__device__ __forceinline__ bool team_lead() { return s_team == 1 || cl_rank() == 0; }
// all threads of every CTA of the cluster; orders the shared::cluster stores before it
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void* p, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void cl_st(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void cl_st(uint32_t a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void cl_st(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
// rows [r0, r1) of this CTA's share of an n-row product (multiples of 8 rows)
__device__ __forceinline__ void cl_rows(int n, int& r0, int& r1) {
  const int cs = team(), per = ((n + cs - 1) / cs + 7) & ~7;
  r0 = min(n, (int)cl_rank() * per);
  r1 = min(n, r0 + per);
}
// copy rows [r0, r1) of ws (R values a row) into the other CTAs' ws, then a cluster barrier
template <typename T, int R>
__device__ __forceinline__ void cl_share_rows(T* ws, int r0, int r1) {
  const unsigned cs = (unsigned)team(), me = cl_rank();
  __syncthreads();
  for (unsigned k = 1; k < cs; ++k) {
    const unsigned peer = (me + k) % cs;
    const uint32_t base = cl_map(ws, peer);
    for (int e = r0 * R + threadIdx.x; e < r1 * R; e += NT) cl_st(base + (uint32_t)(e * sizeof(T)), ws[e]);
  }
  cl_sync();
}

// ------------------------------------------------------------------ block-row sweeps
// L2 prefetch distance of the sweeps, in rounds of NW x RPW rows (set at kernel start)
__shared__ int s_pfd;
// bulk prefetch of `bytes` at p into L2 (TMA engine; no completion to wait for).  p 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// lane 0 of each warp: prefetch its row group `pf` rounds ahead (rows rb + pf NW RPW ...)
template <typename T, int RPW>
__device__ __forceinline__ void prefetch_rows(const T* Q, int rb, int n, int ldq, int pf) {
  const int nx = rb + pf * NW * RPW;
  if (nx < n) l2_prefetch(Q + (size_t)nx * ldq, (uint32_t)(min(RPW, n - nx) * ldq * (int)sizeof(T)));
}
// ws (n x R, row-major) = Q xs with Q dense row-major (ld ldq, rows padded with zeros) and xs
// in shared memory column by column (column j at xs + j ldq, zero beyond row n: a lane's
// 16-byte loads of consecutive chunks fall in distinct banks).  Warp w takes rows [w RPW, w RPW + RPW), then strides
// by NW RPW; lane l reads the 16-byte chunks l, l + 32, ... of each row, U chunks per step with
// all RPW x U loads issued before the FMAs (memory-level parallelism: one CTA streams a whole
// scene's Q).
template <int R, int RPW, int U>
__device__ __forceinline__ void sweep32_t(const float* __restrict__ Q, int r0, int n, int ldq,
                                          const float* __restrict__ xs, float* __restrict__ ws) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nc = ldq >> 2;
  const int pfd = s_pfd;
  if (lane == 0)
    for (int d = 1; d < pfd; ++d) prefetch_rows<float, RPW>(Q, r0 + wid * RPW, n, ldq, d);
  for (int rb = r0 + wid * RPW; rb < n; rb += NW * RPW) {
    if (lane == 0 && pfd > 0) prefetch_rows<float, RPW>(Q, rb, n, ldq, pfd);
    float acc[RPW][R];
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[q][j] = 0.f;
    for (int c0 = lane; c0 < nc; c0 += 32 * U) {
      float4 a[RPW][U];
#pragma unroll
      for (int q = 0; q < RPW; ++q)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = c0 + 32 * u;
          a[q][u] = (rb + q < n && c < nc)
                        ? __ldg(reinterpret_cast<const float4*>(Q + (size_t)(rb + q) * ldq) + c)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = c0 + 32 * u;
        if (c < nc) {
          float y[4][R];
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const float4 t = *reinterpret_cast<const float4*>(xs + (size_t)j * ldq + 4 * c);
            y[0][j] = t.x; y[1][j] = t.y; y[2][j] = t.z; y[3][j] = t.w;
          }
#pragma unroll
          for (int q = 0; q < RPW; ++q)
#pragma unroll
            for (int j = 0; j < R; ++j)
              acc[q][j] = fmaf(a[q][u].x, y[0][j], fmaf(a[q][u].y, y[1][j],
                          fmaf(a[q][u].z, y[2][j], fmaf(a[q][u].w, y[3][j], acc[q][j]))));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        float x = acc[q][j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        acc[q][j] = x;
      }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < RPW; ++q)
        if (rb + q < n)
#pragma unroll
          for (int j = 0; j < R; ++j) ws[(rb + q) * R + j] = acc[q][j];
    }
  }
}

// Tiling variants of the FP32 sweep (rows per warp, column chunks per step); the autotuner
// picks one per scene-size class.
constexpr int NTILE = 6;
__host__ __device__ inline int tile_rpw(int v) { const int t[NTILE] = {2, 4, 4, 4, 8, 8}; return t[v]; }
__host__ __device__ inline int tile_u(int v) { const int t[NTILE] = {4, 1, 2, 4, 1, 2}; return t[v]; }

template <int R, int RPW>
__device__ __forceinline__ void sweep64_t(const double* __restrict__ Q, int r0, int n, int ldq,
                                          const double* __restrict__ xs, double* __restrict__ ws) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nc = ldq >> 1;
  const int pfd = s_pfd;
  if (lane == 0)
    for (int d = 1; d < pfd; ++d) prefetch_rows<double, RPW>(Q, r0 + wid * RPW, n, ldq, d);
  for (int rb = r0 + wid * RPW; rb < n; rb += NW * RPW) {
    if (lane == 0 && pfd > 0) prefetch_rows<double, RPW>(Q, rb, n, ldq, pfd);
    double acc[RPW][R];
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[q][j] = 0.0;
    for (int c = lane; c < nc; c += 32) {
      double y[2][R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const double2 t = *reinterpret_cast<const double2*>(xs + (size_t)j * ldq + 2 * c);
        y[0][j] = t.x; y[1][j] = t.y;
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (rb + q < n) {
          const double2 a = __ldg(reinterpret_cast<const double2*>(Q + (size_t)(rb + q) * ldq) + c);
#pragma unroll
          for (int j = 0; j < R; ++j) acc[q][j] = fma(a.x, y[0][j], fma(a.y, y[1][j], acc[q][j]));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[q][j] = warp_sum(acc[q][j]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < RPW; ++q)
        if (rb + q < n)
#pragma unroll
          for (int j = 0; j < R; ++j) ws[(rb + q) * R + j] = acc[q][j];
    }
  }
}

// Out of line on purpose: one copy of the tiling variants per R instead of one per call site
// keeps the solver kernel's instruction footprint small.
// In a cluster: a barrier first (every CTA has finished reading the previous product from its ws,
// which the peers are about to write), this CTA's rows, then the exchange.  Each row is still
// one warp's fixed-order sum, so the product is bit-identical to the one-CTA sweep.
template <int R>
__device__ __noinline__ void sweep32(int tile, const float* Q, int n, int ldq, const float* xs, float* ws) {
  int r0 = 0, r1 = n;
  const bool clu = team() > 1;
  if (clu) {
    cl_sync();
    cl_rows(n, r0, r1);
  }
  switch (tile) {
    case 0: sweep32_t<R, 2, 4>(Q, r0, r1, ldq, xs, ws); break;
    case 1: sweep32_t<R, 4, 1>(Q, r0, r1, ldq, xs, ws); break;
    case 2: sweep32_t<R, 4, 2>(Q, r0, r1, ldq, xs, ws); break;
    case 3: sweep32_t<R, 4, 4>(Q, r0, r1, ldq, xs, ws); break;
    case 4: sweep32_t<R, 8, 1>(Q, r0, r1, ldq, xs, ws); break;
    default: sweep32_t<R, 8, 2>(Q, r0, r1, ldq, xs, ws); break;
  }
  if (clu) cl_share_rows<float, R>(ws, r0, r1);
  else __syncthreads();
}

template <int R>
__device__ __noinline__ void sweep64(const double* Q, int n, int ldq, const double* xs, double* ws) {
  int r0 = 0, r1 = n;
  const bool clu = team() > 1;
  if (clu) {
    cl_sync();
    cl_rows(n, r0, r1);
  }
  sweep64_t<R, 2>(Q, r0, r1, ldq, xs, ws);
  if (clu) cl_share_rows<double, R>(ws, r0, r1);
  else __syncthreads();
}

// xs (R columns of ldq, type Td) <- v (n x R row-major, type Ts), zero below row n
template <typename Ts, typename Td, int R>
__device__ __forceinline__ void stage(const Ts* __restrict__ v, int n, int ldq, Td* __restrict__ xs) {
  constexpr int B = 4;   // elements a thread loads before it stores
  for (int e0 = threadIdx.x; e0 < ldq * R; e0 += B * NT) {
    Ts t[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int e = e0 + u * NT, j = e / ldq, i = e - j * ldq;
      t[u] = (e < ldq * R && i < n) ? v[(size_t)i * R + j] : Ts(0);
    }
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (e0 + u * NT < ldq * R) xs[e0 + u * NT] = Td(t[u]);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ serial small algebra
// (run by one thread; m <= 8, Krylov dimension <= a few hundred)

// cyclic Jacobi, eigenvalues in descending order, eigenvectors as columns of V (m x m row-major)
__device__ void dev_sym_eig_desc(int m, double* A, double* w, double* V) {
  for (int i = 0; i < m * m; ++i) V[i] = 0.0;
  for (int i = 0; i < m; ++i) V[i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q) {
        const double a = A[p * m + q];
        tot += a * a;
        if (p != q) off += a * a;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[p * m + q];
        if (fabs(apq) < 1e-300) continue;
        const double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = A[k * m + p], akq = A[k * m + q];
          A[k * m + p] = c * akp - s * akq;
          A[k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = A[p * m + k], aqk = A[q * m + k];
          A[p * m + k] = c * apk - s * aqk;
          A[q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[k * m + p], vkq = V[k * m + q];
          V[k * m + p] = c * vkp - s * vkq;
          V[k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < m; ++i) w[i] = A[i * m + i];
  // selection sort, descending, carrying the columns of V
  for (int i = 0; i < m; ++i) {
    int b = i;
    for (int j = i + 1; j < m; ++j) if (w[j] > w[b]) b = j;
    if (b != i) {
      const double t = w[i]; w[i] = w[b]; w[b] = t;
      for (int k = 0; k < m; ++k) { const double u = V[k * m + i]; V[k * m + i] = V[k * m + b]; V[k * m + b] = u; }
    }
  }
}

__device__ int dev_sturm(int k, const double* a, const double* b, double x) {
  int c = 0;
  double q = a[0] - x;
  if (q < 0) ++c;
  for (int i = 1; i < k; ++i) {
    const double qq = (q == 0.0) ? 1e-300 : q;
    q = a[i] - x - b[i - 1] * b[i - 1] / qq;
    if (q < 0) ++c;
  }
  return c;
}

// j-th smallest eigenvalue of the tridiagonal (a[0..k), b[0..k-1)) by bisection
__device__ double dev_tri_eig(int k, const double* a, const double* b, int j) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  const double span = fmax(fabs(lo), fabs(hi)) + 1e-300;
  for (int it = 0; it < 200 && hi - lo > 1e-16 * span; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (dev_sturm(k, a, b, mid) > j) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// eigenvector of the tridiagonal for th by inverse iteration on T - sigma I with a pivoted LU;
// work: 5 k doubles + k chars
__device__ void dev_tri_eigvec(int k, const double* a, const double* b, double th, double* s,
                               double* work, char* piv) {
  if (k == 1) { s[0] = 1.0; return; }
  double* d = work;
  double* du = work + k;
  double* du2 = work + 2 * k;
  double* l = work + 3 * k;
  double* dl = work + 4 * k;
  double scale = 0.0;
  for (int i = 0; i < k; ++i) scale = fmax(scale, fabs(a[i]) + (i < k - 1 ? fabs(b[i]) : 0.0));
  const double sigma = th - 1e-13 * (scale + 1e-300);
  for (int i = 0; i < k; ++i) { d[i] = a[i] - sigma; du[i] = i < k - 1 ? b[i] : 0.0; du2[i] = 0.0; piv[i] = 0; }
  for (int i = 0; i < k - 1; ++i) dl[i] = b[i];
  for (int i = 0; i < k - 1; ++i) {
    if (fabs(d[i]) >= fabs(dl[i])) {
      const double f = d[i] != 0.0 ? dl[i] / d[i] : 0.0;
      l[i] = f;
      d[i + 1] -= f * du[i];
    } else {
      const double f = d[i] / dl[i];
      l[i] = f;
      piv[i] = 1;
      const double t = du[i];
      d[i] = dl[i];
      du[i] = d[i + 1];
      d[i + 1] = t - f * d[i + 1];
      if (i < k - 2) { du2[i] = du[i + 1]; du[i + 1] = -f * du[i + 1]; }
    }
  }
  for (int i = 0; i < k; ++i) d[i] = 1.0 / (d[i] == 0.0 ? 1e-300 : d[i]);   // reciprocals
  for (int i = 0; i < k; ++i) s[i] = 1.0 / sqrt((double)k) * ((i % 3) ? 1.0 : -0.7);
  for (int it = 0; it < 4; ++it) {
    for (int i = 0; i < k - 1; ++i) {
      if (piv[i]) { const double t = s[i]; s[i] = s[i + 1]; s[i + 1] = t - l[i] * s[i + 1]; }
      else s[i + 1] -= l[i] * s[i];
    }
    s[k - 1] *= d[k - 1];
    if (k > 1) s[k - 2] = (s[k - 2] - du[k - 2] * s[k - 1]) * d[k - 2];
    for (int i = k - 3; i >= 0; --i) s[i] = (s[i] - du[i] * s[i + 1] - du2[i] * s[i + 2]) * d[i];
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += s[i] * s[i];
    const double inv = 1.0 / sqrt(nrm);
    for (int i = 0; i < k; ++i) s[i] *= inv;
  }
}

// Number of eigenvalues of the symmetric tridiagonal (a[0..k), b[0..k-1)) below x: sign
// changes of the Sturm sequence p_0 = 1, p_i = (a_i - x) p_{i-1} - b_{i-1}^2 p_{i-2}, without
// divisions (B300's FP64 division is slow).  Three FP64 operations a step (a_i - x, b^2 p_{i-2}
// and one FMA); the sign and the range tests read the exponent and sign bits with integer
// operations, off the narrow FP64 pipe.  The pair (p_{i-1}, p_i) is rescaled by an exact power
// of two (which changes no sign) when |p_i| >= 2^501, or when both are below 2^-500.  A zero
// p_i takes the sign opposite to p_{i-1}.
__device__ __forceinline__ int sturm_nodiv(int k, const double* __restrict__ a, const double* __restrict__ b2,
                                           double x) {
  double pm = 1.0, p = a[0] - x;
  int c = 0;
  bool neg_prev = false;                       // sign of p_0 = +1
  int ex_prev = 1023;                          // biased exponent of p_0
  for (int i = 0;;) {
    const int hi = __double2hiint(p);
    const bool zero = ((hi & 0x7fffffff) | __double2loint(p)) == 0;
    const bool neg = zero ? !neg_prev : hi < 0;
    c += neg != neg_prev;
    neg_prev = neg;
    if (++i >= k) break;
    const int ex = (hi >> 20) & 0x7ff;
    if (ex > 1023 + 500 || (ex < 1023 - 500 && ex_prev < 1023 - 500)) {
      const double sc = ex > 1023 + 500 ? 0x1p-500 : 0x1p500;
      p *= sc;
      pm *= sc;
    }
    ex_prev = (__double2hiint(p) >> 20) & 0x7ff;
    const double pn = fma(a[i] - x, p, -(b2[i - 1] * pm));
    pm = p;
    p = pn;
  }
  return c;
}

// Smallest and largest eigenvalues of the tridiagonal by multisection: each round warps 0-1
// evaluate Sturm counts at 64 interior points of the bracket of the smallest (65 equal parts),
// warps 2-3 of the largest, one warp per SM partition; 10 rounds shrink each bracket by
// 65^10 > 2^60, to FP64 resolution.  (More points a round cost FP64 issue slots, of which B300
// has few: fewer, longer rounds are cheaper.)  a, b2 (= b^2) and the scratch `cnt` (NT ints)
// in shared memory.
__device__ __noinline__ void tri_extremes(int k, const double* a, const double* b, double* b2, int* cnt, double* brk,
                             double& tmin, double& tmax) {
  constexpr int PTS = 64;
  for (int i = threadIdx.x; i < k - 1; i += NT) b2[i] = b[i] * b[i];
  if (threadIdx.x == 0) {
    double lo = a[0], hi = a[0];
    for (int i = 0; i < k; ++i) {
      const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
      lo = fmin(lo, a[i] - r);
      hi = fmax(hi, a[i] + r);
    }
    const double pad = 1e-12 * (fabs(lo) + fabs(hi)) + 1e-300;
    brk[0] = lo - pad; brk[1] = hi + pad;   // bracket of the smallest
    brk[2] = lo - pad; brk[3] = hi + pad;   // bracket of the largest
  }
  __syncthreads();
  const bool active = threadIdx.x < 2 * PTS;
  const bool upper = threadIdx.x >= PTS;
  const int t = threadIdx.x % PTS;
  for (int round = 0; round < 10; ++round) {
    if (active) {
      const double lo = brk[upper ? 2 : 0], hi = brk[upper ? 3 : 1];
      const double x = lo + (hi - lo) * (double)(t + 1) / (double)(PTS + 1);
      cnt[threadIdx.x] = sturm_nodiv(k, a, b2, x);
    }
    __syncthreads();
    if (threadIdx.x == 0 || threadIdx.x == PTS) {
      // first point whose count reaches the target: the eigenvalue lies in (x_{u-1}, x_u]; none
      // does: in (x_{PTS-1}, hi]
      const double lo = brk[upper ? 2 : 0], hi = brk[upper ? 3 : 1];
      const int target = upper ? k : 1;
      const int base = upper ? PTS : 0;
      int first = PTS;
      for (int u = 0; u < PTS; ++u)
        if (cnt[base + u] >= target) { first = u; break; }
      const double nlo = first == 0 ? lo : lo + (hi - lo) * (double)first / (double)(PTS + 1);
      const double nhi = first == PTS ? hi : lo + (hi - lo) * (double)(first + 1) / (double)(PTS + 1);
      brk[upper ? 2 : 0] = nlo;
      brk[upper ? 3 : 1] = nhi;
    }
    __syncthreads();
  }
  tmin = 0.5 * (brk[0] + brk[1]);
  tmax = 0.5 * (brk[2] + brk[3]);
  __syncthreads();
}

// ------------------------------------------------------------------ the per-CTA solver
struct Smem {
  void* xs;                        // sweep input staging, ldq x R (float or double)
  void* ws;                        // sweep output, n x R
  double* red;                     // NW x 64
  double* small;                   // 320 doubles: Gram, eigenvectors, rotation, O0, scalars
  double* ha;                      // Krylov alpha (kmax + 1)
  double* hb;                      // Krylov beta (kmax + 1)
  double* hs;                      // Ritz coefficients (kmax + 1)
  double* cv;                      // reorthogonalisation coefficients (kmax + 16)
  double* work;                    // 5 (kmax + 1)
  double* b2;                      // squared Krylov beta (kmax + 1)
  double* brk;                     // multisection brackets (4)
  int* cnt;                        // Sturm counts (NT)
  char* piv;                       // kmax + 1
};

__host__ __device__ inline size_t smem_bytes(int NM, int R, int kmax) {
  const size_t k1 = (size_t)kmax + 1;
  return 2 * (size_t)NM * R * sizeof(double) + (size_t)NW * 64 * sizeof(double) + 320 * sizeof(double) +
         (3 * k1 + (kmax + 16) + 5 * k1 + k1 + 4) * sizeof(double) + NT * sizeof(int) + ((k1 + 15) / 16) * 16;
}

__device__ inline Smem carve(char* base, int NM, int R, int kmax) {
  Smem s;
  const size_t k1 = (size_t)kmax + 1;
  double* p = reinterpret_cast<double*>(base);
  s.xs = p; p += (size_t)NM * R;
  s.ws = p; p += (size_t)NM * R;
  s.red = p; p += NW * 64;
  s.small = p; p += 320;
  s.ha = p; p += k1;
  s.hb = p; p += k1;
  s.hs = p; p += k1;
  s.cv = p; p += kmax + 16;
  s.work = p; p += 5 * k1;
  s.b2 = p; p += k1;
  s.brk = p; p += 4;
  s.cnt = reinterpret_cast<int*>(p);
  s.piv = reinterpret_cast<char*>(s.cnt + NT);
  return s;
}

template <int R>
struct Cta {
  const Params* P;
  Desc d;
  int N, n, ldq, tile;
  const float* Q32;
  const double* Q64;
  Smem sm;
  double* slot;
  // vectors (each NM x 8 doubles of the slot); the pointers move when RTR accepts a step
  double *y64, *yc64, *g64, *gc64, *yh, *xi, *lam, *lamc;
  float *yf, *ycf, *gf, *gcf;
  double *t0, *t1, *t2, *t3, *t4;   // tCG vectors, used as float or double
  double *V, *lw, *lritz;
  xm_batch_info info;
  double ref_g, cur_g2, f_cur;
  bool timed_out;

  __device__ void setup(const Params* p, const Desc& dd, char* smem_base) {
    P = p; d = dd; N = dd.N; n = dd.n; ldq = dd.ldq;
    tile = p->tile[size_class(n)];
    Q32 = p->Q32 + dd.q32;
    Q64 = p->Q64 + dd.q64;
    sm = carve(smem_base, p->NM, R, p->kmax);
    slot = p->slots + (size_t)(blockIdx.x + p->slot_base) * p->slot_doubles;
    const size_t VS = (size_t)p->NM * 8;
    double* v[NVEC];
    for (int k = 0; k < NVEC; ++k) v[k] = slot + k * VS;
    y64 = v[0]; yc64 = v[1]; g64 = v[2]; gc64 = v[3]; yh = v[4]; xi = v[5];
    yf = (float*)v[6]; ycf = (float*)v[7]; gf = (float*)v[8]; gcf = (float*)v[9];
    t0 = v[10]; t1 = v[11]; t2 = v[12]; t3 = v[13]; t4 = v[14]; lam = v[15]; lamc = v[16];
    V = slot + NVEC * VS;
    lw = V + (size_t)p->NM * (XM_MAX_RANK + p->kmax + 1);
    lritz = lw + p->NM;
    ref_g = -1.0; cur_g2 = 0.0; f_cur = 0.0; timed_out = false;
  }

  // CTA-uniform: thread 0 reads the clock and broadcasts, so every thread takes the same branch
  // In a team, rank 0's clock decides for every CTA (the branches must stay identical); a CTA
  // working alone decides for itself, whatever its rank in the cluster it split from.
  __device__ bool over_time() {
    if (!P->time_limit_ns) return timed_out;
    __shared__ int s_late;
    const unsigned cs = (unsigned)team();
    if (cs > 1) cl_sync();               // every CTA has read the previous decision
    if (threadIdx.x == 0 && team_lead()) {
      const int late = gtimer() > info.t_begin_ns + P->time_limit_ns ? 1 : 0;
      s_late = late;
      for (unsigned k = 1; k < cs; ++k) cl_st(cl_map(&s_late, k), late);
    }
    if (cs > 1) cl_sync();
    else __syncthreads();
    if (s_late) timed_out = true;
    __syncthreads();
    return timed_out;
  }

  // W = Q Y in the sweep precision of To, then the gradient epilogue
  template <typename To>
  __device__ void grad_at(const To* Y, To* G, double* Lam, double& f, double& g2, double& y2) {
    if (sizeof(To) == 4) {
      stage<To, float, R>(Y, n, ldq, (float*)sm.xs);
      sweep32<R>(tile, Q32, n, ldq, (const float*)sm.xs, (float*)sm.ws);
    } else {
      stage<To, double, R>(Y, n, ldq, (double*)sm.xs);
      sweep64<R>(Q64, n, ldq, (const double*)sm.xs, (double*)sm.ws);
      ++info.n_sweeps_fp64;
    }
    ++info.n_sweeps;
    double v[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < N; i += NT) {
      double vi[3];
      grad_block<To, R, To>(i, N, Y, (To*)sm.ws, G, Lam, P->mu, vi);
      v[0] += vi[0]; v[1] += vi[1]; v[2] += vi[2];
    }
    bsum<3>(v, sm.red);
    f = v[0]; g2 = v[1]; y2 = v[2];
  }

  // Hd = Hess[d] at Yin (Ti precision sweep); returns <d, Hd>
  template <typename Ti>
  __device__ double hvp(const Ti* Yin, const Ti* dv, Ti* Hd, const double* Lam) {
    if (sizeof(Ti) == 4) {
      stage<Ti, float, R>(dv, n, ldq, (float*)sm.xs);
      sweep32<R>(tile, Q32, n, ldq, (const float*)sm.xs, (float*)sm.ws);
    } else {
      stage<Ti, double, R>(dv, n, ldq, (double*)sm.xs);
      sweep64<R>(Q64, n, ldq, (const double*)sm.xs, (double*)sm.ws);
      ++info.n_sweeps_fp64;
    }
    ++info.n_sweeps;
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < N; i += NT)
      v[0] += hvp_block<Ti, R, Ti>(i, N, Yin, (Ti*)sm.ws, dv, Hd, Lam, P->mu);
    bsum<1>(v, sm.red);
    return v[0];
  }

  __device__ double dot(const double* a, const double* b, int len) {
    double v[1] = {0.0};
    for (int e0 = threadIdx.x; e0 < len; e0 += EB * NT) {
      double x[EB], y[EB];
#pragma unroll
      for (int u = 0; u < EB; ++u) {
        const int e = e0 + u * NT;
        x[u] = e < len ? a[e] : 0.0; y[u] = e < len ? b[e] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < EB; ++u)
        if (e0 + u * NT < len) v[0] += x[u] * y[u];
    }
    bsum<1>(v, sm.red);
    return v[0];
  }

  // Riemannian trust region (Absil et al. 2008, Alg. 10) with Steihaug-Toint tCG (Alg. 11);
  // constants as in xm_solve.  To: iterate / gradient type, Ti: tCG type.  Y, G, Lam and their
  // candidates are the member pointers of that precision (swapped on acceptance).
  // The per-element loops below give thread t the elements t, t + NT, t + 2 NT, ... (the order
  // of its partial sums) and take EB of them at a time with every load issued before any store:
  // the vectors may alias as far as the compiler knows, so a load after a store would wait one
  // memory round trip per element.  The per-camera loops load a camera's blocks before storing.
  static constexpr int EB = 4;
  // tCG iterations per step of the FP32 bulk phase (at most max_tcg), as xm_solve: truncated
  // inner solves far from the optimum; the polish keeps max_tcg
  static constexpr int BULK_TCG_CAP = 60;
  static constexpr int NMAX_LZ = 4 * NT;   // Lanczos rows a CTA keeps in registers across a step
  template <typename To, typename Ti>
  __device__ void rtr(double tol_rel, int max_outer, bool bulk) {
    To*& Y = *reinterpret_cast<To**>(sizeof(To) == 4 ? (void*)&yf : (void*)&y64);
    To*& Yc = *reinterpret_cast<To**>(sizeof(To) == 4 ? (void*)&ycf : (void*)&yc64);
    To*& G = *reinterpret_cast<To**>(sizeof(To) == 4 ? (void*)&gf : (void*)&g64);
    To*& Gc = *reinterpret_cast<To**>(sizeof(To) == 4 ? (void*)&gcf : (void*)&gc64);
    Ti* eta = (Ti*)t0;
    Ti* Heta = (Ti*)t1;
    Ti* rv = (Ti*)t2;
    Ti* dv = (Ti*)t3;
    Ti* Hd = (Ti*)t4;
    const int nR = n * R;
    double f, g2, y2;
    grad_at<To>(Y, G, lam, f, g2, y2);
    if (ref_g <= 0) ref_g = sqrt(g2);
    const double tol_abs = tol_rel * ref_g;
    const double Delta_bar = sqrt(fmax(y2, 1e-300));
    double Delta = Delta_bar / 8.0;
    const double eps_reg = sizeof(To) == 4 ? 1e2 * 1.1920929e-07 : 1e3 * 2.220446049250313e-16;
    // the tCG's copy of Y when its precision differs (FP64 polish with FP32 HVPs)
    const Ti* Yin;
    int rejects = 0;
    constexpr int STALL_W = 5;   // bulk-phase stagnation window (as xm_solve)
    double f_hist[STALL_W + 1];
    int n_hist = 0;
    for (int k = 0; k < max_outer; ++k) {
      if (!(sqrt(g2) > tol_abs) || over_time()) break;
      if (sizeof(To) != sizeof(Ti)) {
        for (int e0 = threadIdx.x; e0 < nR; e0 += EB * NT) {
          To v[EB];
#pragma unroll
          for (int u = 0; u < EB; ++u) v[u] = e0 + u * NT < nR ? Y[e0 + u * NT] : To(0);
#pragma unroll
          for (int u = 0; u < EB; ++u)
            if (e0 + u * NT < nR) ((Ti*)yf)[e0 + u * NT] = Ti(v[u]);
        }
        Yin = (const Ti*)yf;
      } else {
        Yin = (const Ti*)Y;
      }
      // ---- tCG
      for (int e0 = threadIdx.x; e0 < nR; e0 += EB * NT) {
        Ti g[EB];
#pragma unroll
        for (int u = 0; u < EB; ++u) g[u] = e0 + u * NT < nR ? Ti(G[e0 + u * NT]) : Ti(0);
#pragma unroll
        for (int u = 0; u < EB; ++u) {
          const int e = e0 + u * NT;
          if (e < nR) { eta[e] = Ti(0); Heta[e] = Ti(0); rv[e] = g[u]; dv[e] = -g[u]; }
        }
      }
      __syncthreads();
      double rr = g2, ee = 0.0, ed = 0.0, dd = g2;
      const double r0 = sqrt(g2);
      // The FP64 polish's Hessian products are FP32 (relative error ~1e-5 on these scenes): a
      // residual below 1e-4 of r0 buys nothing but iterations (the target r0^2 had run every
      // polish step to the max_tcg cap).  An inexact Newton step with this forcing term still
      // converges to the same gradient tolerance, checked by the outer loop in FP64.
      const double floor_rel = (!bulk && sizeof(Ti) < sizeof(To)) ? 1e-4 : 0.0;
      int iters = 0;
      const int tcg_cap = bulk ? min(P->o.max_tcg, BULK_TCG_CAP) : P->o.max_tcg;
      for (int j = 0; j < tcg_cap; ++j) {
        const double kap = hvp<Ti>(Yin, dv, Hd, lam);
        ++iters;
        const double D2 = Delta * Delta;
        const double a = kap > 0.0 ? rr / kap : 0.0;
        if (!(kap > 0.0) || ee + 2.0 * a * ed + a * a * dd >= D2) {
          const double disc = ed * ed + dd * (D2 - ee);
          const double tau = (-ed + sqrt(disc > 0.0 ? disc : 0.0)) / dd;
          for (int e0 = threadIdx.x; e0 < nR; e0 += EB * NT) {
            Ti x[EB], h[EB], d[EB], hd[EB];
#pragma unroll
            for (int u = 0; u < EB; ++u) {
              const int e = e0 + u * NT;
              const bool ok = e < nR;
              x[u] = ok ? eta[e] : Ti(0); h[u] = ok ? Heta[e] : Ti(0);
              d[u] = ok ? dv[e] : Ti(0); hd[u] = ok ? Hd[e] : Ti(0);
            }
#pragma unroll
            for (int u = 0; u < EB; ++u) {
              const int e = e0 + u * NT;
              if (e < nR) {
                eta[e] = Ti(double(x[u]) + tau * double(d[u]));
                Heta[e] = Ti(double(h[u]) + tau * double(hd[u]));
              }
            }
          }
          __syncthreads();
          break;
        }
        // eta += a d, Heta += a Hd, r += a Hd re-projected onto the tangent space (tCG
        // arithmetic in the tCG's precision; per-thread partial sums, CTA sum in FP64)
        Ti part = Ti(0);
        const Ti at = Ti(a);
        for (int i = threadIdx.x; i < N; i += NT) {
          Ti y[3][R], r3[3][R];
          if constexpr (R <= 4) {
            Ti hd[3][R], et[3][R], he[3][R], db[3][R];
            load_block<Ti, Ti, R>(Hd, i, hd);
            load_block<Ti, Ti, R>(eta, i, et);
            load_block<Ti, Ti, R>(Heta, i, he);
            load_block<Ti, Ti, R>(dv, i, db);
            load_block<Ti, Ti, R>(rv, i, r3);
            load_block<Ti, Ti, R>(Yin, i, y);
#pragma unroll
            for (int aa = 0; aa < 3; ++aa)
#pragma unroll
              for (int jj = 0; jj < R; ++jj) {
                et[aa][jj] = et[aa][jj] + at * db[aa][jj];
                he[aa][jj] = he[aa][jj] + at * hd[aa][jj];
                r3[aa][jj] = r3[aa][jj] + at * hd[aa][jj];
              }
            store_block<Ti, Ti, R>(eta, i, et);
            store_block<Ti, Ti, R>(Heta, i, he);
          } else {   // rank 8: element by element (the blocks would not fit in registers)
            load_block<Ti, Ti, R>(Yin, i, y);
#pragma unroll
            for (int aa = 0; aa < 3; ++aa)
#pragma unroll
              for (int jj = 0; jj < R; ++jj) {
                const size_t e = (size_t)(3 * i + aa) * R + jj;
                const Ti hd = Hd[e];
                eta[e] = eta[e] + at * dv[e];
                Heta[e] = Heta[e] + at * hd;
                r3[aa][jj] = rv[e] + at * hd;
              }
          }
          Ti S[3][3], al;
          dual_block<Ti, R>(r3, y, i == 0, S, al);
#pragma unroll
          for (int aa = 0; aa < 3; ++aa)
#pragma unroll
            for (int jj = 0; jj < R; ++jj) {
              r3[aa][jj] -= S[aa][0] * y[0][jj] + S[aa][1] * y[1][jj] + S[aa][2] * y[2][jj];
              part += r3[aa][jj] * r3[aa][jj];
            }
          store_block<Ti, Ti, R>(rv, i, r3);
        }
        double v[1] = {double(part)};
        bsum<1>(v, sm.red);
        const double rr_new = v[0];
        if (sqrt(rr_new) <= r0 * fmax(fmin(pow(r0, 1.0), 0.1), floor_rel)) break;
        const double beta = rr_new / rr;
        rr = rr_new;
        Ti p3[3] = {Ti(0), Ti(0), Ti(0)};
        const Ti bt = Ti(beta);
        for (int e0 = threadIdx.x; e0 < nR; e0 += EB * NT) {
          Ti rq[EB], dq[EB], tq[EB];
#pragma unroll
          for (int u = 0; u < EB; ++u) {
            const int e = e0 + u * NT;
            const bool ok = e < nR;
            rq[u] = ok ? rv[e] : Ti(0); dq[u] = ok ? dv[e] : Ti(0); tq[u] = ok ? eta[e] : Ti(0);
          }
#pragma unroll
          for (int u = 0; u < EB; ++u) {
            const int e = e0 + u * NT;
            if (e < nR) {
              const Ti de = -rq[u] + bt * dq[u];
              dv[e] = de;
              const Ti et = tq[u];
              p3[0] += et * et; p3[1] += et * de; p3[2] += de * de;
            }
          }
        }
        double w3[3] = {double(p3[0]), double(p3[1]), double(p3[2])};
        bsum<3>(w3, sm.red);
        ee = w3[0]; ed = w3[1]; dd = w3[2];
      }
      info.n_tcg += iters;
      // ---- model decrease, candidate, ratio test
      double m3[3] = {0.0, 0.0, 0.0};
      for (int e0 = threadIdx.x; e0 < nR; e0 += EB * NT) {
        To gq[EB];
        Ti xq[EB], hq[EB];
#pragma unroll
        for (int u = 0; u < EB; ++u) {
          const int e = e0 + u * NT;
          const bool ok = e < nR;
          gq[u] = ok ? G[e] : To(0); xq[u] = ok ? eta[e] : Ti(0); hq[u] = ok ? Heta[e] : Ti(0);
        }
#pragma unroll
        for (int u = 0; u < EB; ++u)
          if (e0 + u * NT < nR) {
            const double g = double(gq[u]), x = double(xq[u]), h = double(hq[u]);
            m3[0] += g * x; m3[1] += x * h; m3[2] += x * x;
          }
      }
      bsum<3>(m3, sm.red);
      for (int i = threadIdx.x; i < N; i += NT) retract_block<To, Ti, R, To>(i, Y, eta, 1.0, Yc);
      __syncthreads();
      double fc, gc2, yc2;
      grad_at<To>(Yc, Gc, lamc, fc, gc2, yc2);
      ++info.n_outer;
      const double model_dec = -(m3[0] + 0.5 * m3[1]);
      const double reg = fmax(1.0, fabs(f)) * eps_reg;
      const double rho = (f - fc + reg) / (model_dec + reg);
      const double en = sqrt(m3[2]);
      if (!isfinite(fc) || rho < 0.25) Delta *= 0.25;
      else if (rho > 0.75 && en >= Delta * (1.0 - 1e-6)) Delta = fmin(2.0 * Delta, Delta_bar);
      const bool accept = isfinite(fc) && rho > 0.1 && fc <= f + reg;
      if (accept) {
        To* t = Y; Y = Yc; Yc = t;
        t = G; G = Gc; Gc = t;
        double* u = lam; lam = lamc; lamc = u;
        f = fc; g2 = gc2;
        rejects = 0;
      } else {
        ++rejects;
      }
      if (Delta < 1e-12 * Delta_bar) break;
      if (bulk && (rejects >= 6 || Delta < 1e-7 * Delta_bar)) break;
      // A step rejected at the FP32 floor (||rgrad|| <= 1e-6 of the start): the FP32 objective
      // can no longer rank the candidates, and every further bulk step (each a tCG run to the
      // trust-region boundary, then rejected) is lost work; the FP64-gradient polish takes over.
      if (bulk && !accept && sqrt(g2) <= 1e-6 * ref_g) break;
      if (bulk) {
        // near the FP32 floor (||rgrad|| <= 1e-6 of the start) and f no longer improving beyond
        // its own noise (reg) over STALL_W steps: hand over to the FP64-gradient polish.  This
        // bounds the bulk work of the many small scenes of a batch; xm_solve keeps iterating
        // to the bulk tolerance (its large scenes lean on the longer FP32 phase).
        f_hist[n_hist % (STALL_W + 1)] = f;
        ++n_hist;
        if (n_hist > STALL_W && f_hist[(n_hist - 1 - STALL_W) % (STALL_W + 1)] - f < reg &&
            sqrt(g2) <= 1e-6 * ref_g)
          break;
      }
    }
    f_cur = f;
    cur_g2 = g2;
  }

  // Gram Y^T Y (R x R) of the FP64 iterate, then thread 0: eigen-decomposition of its leading
  // m x m block, eigenvalues (descending) into small[0..m), eigenvectors (columns, m x m
  // row-major) into small[64..)
  __device__ void gram_eig(int m) {
    double v[R * R];
#pragma unroll
    for (int k = 0; k < R * R; ++k) v[k] = 0.0;
    for (int e = threadIdx.x; e < n; e += NT) {
      double y[R];
#pragma unroll
      for (int a = 0; a < R; ++a) y[a] = y64[(size_t)e * R + a];
#pragma unroll
      for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) v[a * R + b] += y[a] * y[b];
    }
    bsum<R * R>(v, sm.red);
    if (threadIdx.x == 0) {
      double A[R * R];
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) A[a * m + b] = v[a * R + b];
      dev_sym_eig_desc(m, A, sm.small, sm.small + 64);
    }
    __syncthreads();
  }

  // The Lanczos basis is kept in FP32 (column stride NM): the Z products are FP32 sweeps, so
  // FP32 orthogonality (~1e-7) matches their accuracy; the working vector lw, the recurrence
  // coefficients, the Ritz values and the decision stay FP64.
  __device__ float* Vf() const { return reinterpret_cast<float*>(V); }

  // w -= V c with c = V^T w over the first m columns of V: one pass of classical Gram-Schmidt in
  // FP32 arithmetic (FP64 w, converted once per pass: float <-> double conversions share B300's
  // narrow FP64 pipe).  Each c_j is one warp's sum over the 16-byte chunks of column j (lane l
  // takes chunks l, l + 32, ...), each (V c)_e one thread's sum over j in order, so neither
  // depends on which warp or CTA computes it: a team splits the columns of c and the rows of V c
  // between its CTAs and exchanges them through distributed shared memory, bit-identical to one
  // CTA.  Every load of V is 16 bytes with several in flight per thread (the basis streams from
  // L2 at the SM's bandwidth rather than its latency).  Columns of V are zero in rows [n, ldq).
  static constexpr int RO_COLS = 4;      // columns of c per warp and pass
  static constexpr int RO_U = 2;         // 16-byte chunks per lane and column in flight
  static constexpr int RO_J = 8;         // columns of V per thread in flight in V c
  __device__ void reorth(double* w, int m) {
    if (m <= 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int NM4 = P->NM >> 2, n4 = ldq >> 2;
    const float4* V4 = reinterpret_cast<const float4*>(Vf());
    float* wf = (float*)sm.ws;             // FP32 w, ldq entries (free between Z products)
    float* tf = (float*)sm.xs;             // V c, ldq entries
    float* cf = (float*)sm.cv;             // c, m entries
    const int cs = team();
    const unsigned me = cs > 1 ? cl_rank() : 0u;
    for (int e0 = threadIdx.x; e0 < ldq; e0 += EB * NT) {
      double x[EB];
#pragma unroll
      for (int u = 0; u < EB; ++u) x[u] = e0 + u * NT < n ? w[e0 + u * NT] : 0.0;
#pragma unroll
      for (int u = 0; u < EB; ++u)
        if (e0 + u * NT < ldq) wf[e0 + u * NT] = float(x[u]);
    }
    __syncthreads();
    {  // c_j for j in [j0, j1)
      const int per = (m + cs - 1) / cs;
      const int j0 = min(m, (int)me * per), j1 = min(m, j0 + per);
      const float4* w4 = reinterpret_cast<const float4*>(wf);
      for (int jb = j0 + RO_COLS * wid; jb < j1; jb += RO_COLS * NW) {
        float acc[RO_COLS];
#pragma unroll
        for (int q = 0; q < RO_COLS; ++q) acc[q] = 0.f;
        for (int c0 = lane; c0 < n4; c0 += 32 * RO_U) {
          float4 a[RO_COLS][RO_U];
#pragma unroll
          for (int q = 0; q < RO_COLS; ++q)
#pragma unroll
            for (int u = 0; u < RO_U; ++u) {
              const int c = c0 + 32 * u;
              a[q][u] = (jb + q < j1 && c < n4) ? V4[(size_t)(jb + q) * NM4 + c] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
          for (int u = 0; u < RO_U; ++u) {
            const int c = c0 + 32 * u;
            if (c < n4) {
              const float4 y = w4[c];
#pragma unroll
              for (int q = 0; q < RO_COLS; ++q)
                acc[q] = fmaf(a[q][u].x, y.x, fmaf(a[q][u].y, y.y, fmaf(a[q][u].z, y.z, fmaf(a[q][u].w, y.w, acc[q]))));
            }
          }
        }
#pragma unroll
        for (int q = 0; q < RO_COLS; ++q) {
          float x = acc[q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
          if (lane == q && jb + q < j1) {
            cf[jb + q] = x;
            for (int k = 1; k < cs; ++k) cl_st(cl_map(cf + jb + q, (me + k) % cs), x);
          }
        }
      }
    }
    if (cs > 1) cl_sync();
    else __syncthreads();
    {  // (V c)_e for the rows [r0, r1), 4 rows (one 16-byte chunk) a thread, two chunks at a time
      int r0 = 0, r1 = n;
      if (cs > 1) cl_rows(n, r0, r1);
      const int cb0 = r0 >> 2, cb1 = r0 < r1 ? (r1 + 3) >> 2 : cb0;
      float4* t4 = reinterpret_cast<float4*>(tf);
      for (int c = cb0 + threadIdx.x; c < cb1; c += 2 * NT) {
        const int c2 = c + NT;
        const bool two = c2 < cb1;
        float4 s1 = make_float4(0.f, 0.f, 0.f, 0.f), s2 = s1;
        int j = 0;
        for (; j + RO_J <= m; j += RO_J) {
          float4 a1[RO_J], a2[RO_J];
#pragma unroll
          for (int u = 0; u < RO_J; ++u) {
            a1[u] = V4[(size_t)(j + u) * NM4 + c];
            a2[u] = two ? V4[(size_t)(j + u) * NM4 + c2] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < RO_J; ++u) {
            const float cj = cf[j + u];
            s1.x = fmaf(a1[u].x, cj, s1.x); s1.y = fmaf(a1[u].y, cj, s1.y);
            s1.z = fmaf(a1[u].z, cj, s1.z); s1.w = fmaf(a1[u].w, cj, s1.w);
            s2.x = fmaf(a2[u].x, cj, s2.x); s2.y = fmaf(a2[u].y, cj, s2.y);
            s2.z = fmaf(a2[u].z, cj, s2.z); s2.w = fmaf(a2[u].w, cj, s2.w);
          }
        }
        for (; j < m; ++j) {
          const float cj = cf[j];
          const float4 a = V4[(size_t)j * NM4 + c];
          s1.x = fmaf(a.x, cj, s1.x); s1.y = fmaf(a.y, cj, s1.y);
          s1.z = fmaf(a.z, cj, s1.z); s1.w = fmaf(a.w, cj, s1.w);
          if (two) {
            const float4 b = V4[(size_t)j * NM4 + c2];
            s2.x = fmaf(b.x, cj, s2.x); s2.y = fmaf(b.y, cj, s2.y);
            s2.z = fmaf(b.z, cj, s2.z); s2.w = fmaf(b.w, cj, s2.w);
          }
        }
        t4[c] = s1;
        if (two) t4[c2] = s2;
        for (int k = 1; k < cs; ++k) {
          const unsigned peer = (me + k) % cs;
          cl_st(cl_map(t4 + c, peer), s1);
          if (two) cl_st(cl_map(t4 + c2, peer), s2);
        }
      }
    }
    if (cs > 1) cl_sync();
    else __syncthreads();
    for (int e0 = threadIdx.x; e0 < n; e0 += EB * NT) {
      double x[EB];
      float t[EB];
#pragma unroll
      for (int u = 0; u < EB; ++u) {
        const int e = e0 + u * NT;
        x[u] = e < n ? w[e] : 0.0; t[u] = e < n ? tf[e] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < EB; ++u)
        if (e0 + u * NT < n) w[e0 + u * NT] = x[u] - double(t[u]);
    }
    __syncthreads();
  }

  // w = Z v for an FP32 basis vector v
  __device__ void zmul_f(const float* v, double* w) {
    stage<float, float, 1>(v, n, ldq, (float*)sm.xs);
    sweep32<1>(tile, Q32, n, ldq, (const float*)sm.xs, (float*)sm.ws);
    ++info.n_sweeps;
    const float* ws = (const float*)sm.ws;
    for (int i = threadIdx.x; i < N; i += NT) {
      const double x0 = v[3 * i], x1 = v[3 * i + 1], x2 = v[3 * i + 2];
      const double* L = lam + 9 * (size_t)i;
      const double dreg = lam[(size_t)9 * N + i];
      w[3 * i] = double(ws[3 * i]) - (L[0] * x0 + L[1] * x1 + L[2] * x2);
      w[3 * i + 1] = double(ws[3 * i + 1]) - (L[3] * x0 + L[4] * x1 + L[5] * x2);
      w[3 * i + 2] = double(ws[3 * i + 2]) - (L[6] * x0 + L[7] * x1 + L[8] * x2) + dreg * x2;
    }
    __syncthreads();
  }

  __device__ void certify(int r, int kcap_steps, double& lam_def, double& lam_max, double& lam_range) {
    const unsigned long long tc0 = threadIdx.x == 0 ? gtimer() : 0ull;
    certify_body(r, kcap_steps, lam_def, lam_max, lam_range);
    if (threadIdx.x == 0) info.t_cert_ns += gtimer() - tc0;
  }

  // Lanczos on Z restricted to range(Y)^perp (Thm. 1), as Solver::certify: deflation basis from
  // the Gram matrix, Rayleigh quotients of Z on range(Y), full reorthogonalisation (twice), Ritz
  // values by multisection at K = 10, 20, 30, 45, 65, ... (about x1.45), Ritz vector of the
  // smallest into lritz.
  __device__ void certify_body(int r, int kcap_steps, double& lam_def, double& lam_max, double& lam_range) {
    const int NMc = P->NM;
    const int kmax = P->kmax;
    float* Vb = Vf();
    gram_eig(r);
    // rotation: column j = E_j / sqrt(w_j) for the retained directions
    __shared__ int s_nd;
    if (threadIdx.x == 0) {
      const double* w = sm.small;
      const double* E = sm.small + 64;
      double* rot = sm.small + 128;
      int nd = 0;
      for (int k = 0; k < R * R; ++k) rot[k] = 0.0;
      for (int j = 0; j < r; ++j)
        if (w[j] > 1e-10 * w[0]) {
          for (int a = 0; a < r; ++a) rot[a * R + nd] = E[a * r + j] / sqrt(w[j]);
          ++nd;
        }
      s_nd = nd;
    }
    __syncthreads();
    const int nd = s_nd;
    const double* rot = sm.small + 128;
    for (int e = threadIdx.x; e < ldq; e += NT)
      for (int j = 0; j < nd; ++j) {
        double t = 0.0;
        if (e < n)
          for (int a = 0; a < R; ++a) t += y64[(size_t)e * R + a] * rot[a * R + j];
        Vb[(size_t)j * NMc + e] = float(t);
      }
    __syncthreads();
    // Rayleigh quotients V_d^T Z V_d (nd x nd) -> smallest eigenvalue lam_range
    __shared__ double zr[XM_MAX_RANK * XM_MAX_RANK];
    for (int j = 0; j < nd; ++j) {
      zmul_f(Vb + (size_t)j * NMc, lw);
      for (int l = 0; l < nd; ++l) {
        double v[1] = {0.0};
        for (int e = threadIdx.x; e < n; e += NT) v[0] += double(Vb[(size_t)l * NMc + e]) * lw[e];
        bsum<1>(v, sm.red);
        if (threadIdx.x == 0) zr[j * nd + l] = v[0];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (nd > 0) {
        double A[XM_MAX_RANK * XM_MAX_RANK], w[XM_MAX_RANK], E[XM_MAX_RANK * XM_MAX_RANK];
        for (int a = 0; a < nd; ++a)
          for (int b = 0; b < nd; ++b) A[a * nd + b] = 0.5 * (zr[a * nd + b] + zr[b * nd + a]);
        dev_sym_eig_desc(nd, A, w, E);
        sm.small[300] = w[nd - 1];
      } else {
        sm.small[300] = 0.0;
      }
    }
    __syncthreads();
    lam_range = sm.small[300];
    // start vector: splitmix64 uniform(-1, 1) keyed by (seed, index), as xm_solve
    for (int e = threadIdx.x; e < n; e += NT) {
      uint64_t z = P->o.seed + 0x9E3779B97F4A7C15ull * (uint64_t)(e + 1);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      lw[e] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    __syncthreads();
    reorth(lw, nd);
    {
      const double nrm = sqrt(dot(lw, lw, n));
      const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
      float* v0 = Vb + (size_t)nd * NMc;
      for (int e = threadIdx.x; e < ldq; e += NT) v0[e] = e < n ? float(lw[e] * inv) : 0.f;
      __syncthreads();
    }
    int K = 0;
    double th_min = 0.0, th_max = 0.0;
    const int kcap = min(kcap_steps > 0 ? min(kcap_steps, kmax) : kmax, n - nd);
    __shared__ int s_conv;
    int next_check = 10;
    for (int k = 0; k < kcap; ++k) {
      const float* vk = Vb + (size_t)(nd + k) * NMc;
      const float* vkm1 = k > 0 ? Vb + (size_t)(nd + k - 1) * NMc : nullptr;
      zmul_f(vk, lw);
      // a thread's EB elements of v_k, v_{k-1} and w stay in registers between the two loops
      float vq[(NMAX_LZ + NT - 1) / NT], vmq[(NMAX_LZ + NT - 1) / NT];
      double wq[(NMAX_LZ + NT - 1) / NT];
      double av[1] = {0.0};
#pragma unroll
      for (int u = 0; u < (NMAX_LZ + NT - 1) / NT; ++u) {
        const int e = threadIdx.x + u * NT;
        const bool ok = e < n;
        vq[u] = ok ? vk[e] : 0.f; vmq[u] = (ok && vkm1) ? vkm1[e] : 0.f; wq[u] = ok ? lw[e] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < (NMAX_LZ + NT - 1) / NT; ++u)
        if (threadIdx.x + u * NT < n) av[0] += double(vq[u]) * wq[u];
      for (int e = threadIdx.x + NMAX_LZ; e < n; e += NT) av[0] += double(vk[e]) * lw[e];
      bsum<1>(av, sm.red);
      const double a = av[0];
      const double b = k > 0 ? sm.hb[k - 1] : 0.0;
#pragma unroll
      for (int u = 0; u < (NMAX_LZ + NT - 1) / NT; ++u)
        if (threadIdx.x + u * NT < n)
          lw[threadIdx.x + u * NT] = wq[u] - (a * double(vq[u]) + (vkm1 ? b * double(vmq[u]) : 0.0));
      for (int e = threadIdx.x + NMAX_LZ; e < n; e += NT) lw[e] -= a * double(vk[e]) + (vkm1 ? b * double(vkm1[e]) : 0.0);
      __syncthreads();
      reorth(lw, nd + k + 1);
      reorth(lw, nd + k + 1);
      const double bn = sqrt(dot(lw, lw, n));
      const double inv = bn > 0.0 ? 1.0 / bn : 0.0;
      float* vk1 = Vb + (size_t)(nd + k + 1) * NMc;
      for (int e0 = threadIdx.x; e0 < ldq; e0 += EB * NT) {
        double x[EB];
#pragma unroll
        for (int u = 0; u < EB; ++u) x[u] = e0 + u * NT < n ? lw[e0 + u * NT] : 0.0;
#pragma unroll
        for (int u = 0; u < EB; ++u)
          if (e0 + u * NT < ldq) vk1[e0 + u * NT] = e0 + u * NT < n ? float(x[u] * inv) : 0.f;
      }
      if (threadIdx.x == 0) { sm.ha[k] = a; sm.hb[k] = bn; }
      __syncthreads();
      ++info.n_lanczos;
      K = k + 1;
      if (K == next_check || K == kcap) {
        next_check = max(next_check + 10, (next_check * 29) / 20);
        tri_extremes(K, sm.ha, sm.hb, sm.b2, sm.cnt, sm.brk, th_min, th_max);
        if (threadIdx.x == 0) {
          dev_tri_eigvec(K, sm.ha, sm.hb, th_min, sm.hs, sm.work, sm.piv);
          const double res = fabs(sm.hb[K - 1] * sm.hs[K - 1]);
          const double scale = fmax(fabs(th_max), fabs(th_min)) + 1e-300;
          s_conv = (res <= P->o.lanczos_tol * scale || sm.hb[K - 1] <= 1e-14 * scale || K == kcap) ? 1 : 0;
        }
        __syncthreads();
        if (s_conv) break;
      }
    }
    // Ritz vector of th_min (FP32 combination of the FP32 basis)
    float* hsf = (float*)sm.cv;
    for (int j = threadIdx.x; j < K; j += NT) hsf[j] = float(sm.hs[j]);
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += NT) {
      float t = 0.f;
      for (int j = 0; j < K; ++j) t = fmaf(Vb[(size_t)(nd + j) * NMc + e], hsf[j], t);
      lritz[e] = double(t);
    }
    __syncthreads();
    lam_def = th_min;
    lam_max = th_max;
  }

  // F(X) - <grad F(X), X> at the FP64 iterate (App. E dual value; 0 without regulariser)
  __device__ double reg_dual() {
    if (P->mu == 0.0) return 0.0;
    double v[2] = {0.0, 0.0};
    for (int i = threadIdx.x + 0; i < N; i += NT) {
      if (i == 0) continue;
      double x2 = 0.0;
      for (int j = 0; j < R; ++j) { const double t = y64[(size_t)(3 * i + 2) * R + j]; x2 += t * t; }
      v[0] += P->mu * (x2 - 1.0) * (x2 - 1.0);
      v[1] += 2.0 * P->mu * (x2 - 1.0) * x2;
    }
    bsum<2>(v, sm.red);
    return v[0] - v[1];
  }

  // rounding (Sec. 2.2) into the scene's R and s; returns rho_hat = f(Yhat) in FP64 (+ F)
  __device__ double round_and_eval(int r) {
    gram_eig(r);
    const double* E = sm.small + 64;
    for (int e = threadIdx.x; e < n; e += NT) {
      for (int j = 0; j < 3; ++j) {
        double t = 0.0;
        for (int a = 0; a < r; ++a) t += y64[(size_t)e * R + a] * (j < r ? E[a * r + j] : 0.0);
        yh[(size_t)e * 4 + j] = t;
      }
      yh[(size_t)e * 4 + 3] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // O0 = polar factor of Ubar_0 = Yh_0^T
      double Ub[9], UtU[9], w3[3], V3[9];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Ub[a * 3 + b] = yh[b * 4 + a];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double t = 0.0;
          for (int k = 0; k < 3; ++k) t += Ub[k * 3 + a] * Ub[k * 3 + b];
          UtU[a * 3 + b] = t;
        }
      dev_sym_eig_desc(3, UtU, w3, V3);
      double* O0 = sm.small + 200;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double t = 0.0;
          for (int k = 0; k < 3; ++k) {
            const double sig = sqrt(fmax(w3[k], 1e-300));
            double uk = 0.0;
            for (int m = 0; m < 3; ++m) uk += Ub[a * 3 + m] * V3[m * 3 + k];
            t += uk / sig * V3[b * 3 + k];
          }
          O0[a * 3 + b] = t;
        }
    }
    __syncthreads();
    double* Yhat = xi;   // n x 4
    // the results go out from the team's lead; the other CTAs write the same values to t0
    const bool lead = team_lead();
    double* Rdst = lead ? P->R_out + 9 * d.cam0 : t0;
    double* sdst = lead ? P->s_out + d.cam0 : t0 + 9 * (size_t)N;
    for (int i = threadIdx.x; i < N; i += NT) round_block(i, yh, sm.small + 200, Rdst, sdst, Yhat);
    __syncthreads();
    stage<double, double, 4>(Yhat, n, ldq, (double*)sm.xs);
    sweep64<4>(Q64, n, ldq, (const double*)sm.xs, (double*)sm.ws);
    ++info.n_sweeps; ++info.n_sweeps_fp64;
    const double* ws = (const double*)sm.ws;
    double v[1] = {0.0};
    for (int e = threadIdx.x; e < n * 4; e += NT) v[0] += Yhat[e] * ws[e];
    if (P->mu != 0.0)
      for (int i = threadIdx.x; i < N; i += NT)
        if (i > 0) {
          double x2 = 0.0;
          for (int j = 0; j < 4; ++j) { const double t = Yhat[(size_t)(3 * i + 2) * 4 + j]; x2 += t * t; }
          v[0] += P->mu * (x2 - 1.0) * (x2 - 1.0);
        }
    bsum<1>(v, sm.red);
    return v[0];
  }

  // f at the FP64-retracted point Y + a Xi, evaluated with FP32 sweeps (the mixed mode's line
  // search); the retracted point is left in yh
  __device__ double f_at(double a) {
    for (int i = threadIdx.x; i < N; i += NT) retract_block<double, double, R>(i, y64, xi, a, yh);
    __syncthreads();
    for (int e = threadIdx.x; e < n * R; e += NT) ycf[e] = float(yh[e]);
    __syncthreads();
    double f, g2, y2;
    grad_at<float>(ycf, gcf, lamc, f, g2, y2);
    return f;
  }

  __device__ void copy64(const double* s, double* t, int len) {
    for (int e = threadIdx.x; e < len; e += NT) t[e] = s[e];
    __syncthreads();
  }

  // The staircase for one scene (Alg. 1 with xm_solve's FP32-bulk schedule).  Returns false
  // when the scene needs rank > R and was handed over (rank-4 kernel only).
  __device__ bool run(bool resume) {
    const xm_opts& o = P->o;
    const size_t nR = (size_t)n * R;
    int r = o.r0;
    bool pending_escape = false;
    double* spill = P->spill + d.spill;
    if (!resume) {
      for (int i = threadIdx.x; i < N; i += NT) init_block(i, R, r, o.init_jitter, o.seed, y64);
      __syncthreads();
      if (o.init_jitter != 0.0 && r > 3) {   // make the jittered start feasible
        for (int e = threadIdx.x; e < (int)nR; e += NT) xi[e] = 0.0;
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += NT) retract_block<double, double, R>(i, y64, xi, 0.0, yc64);
        __syncthreads();
        double* t = y64; y64 = yc64; yc64 = t;
      }
    } else {
      // hand-over from the rank-4 kernel: [ref_g, r, Y (n x 4), Ritz vector (n)]
      ref_g = spill[0];
      const int r_old = (int)spill[1];
      for (int e = threadIdx.x; e < n; e += NT)
        for (int j = 0; j < R; ++j) {
          y64[(size_t)e * R + j] = j < 4 ? spill[2 + (size_t)e * 4 + j] : 0.0;
          xi[(size_t)e * R + j] = j == r_old ? spill[2 + (size_t)n * 4 + e] : 0.0;
        }
      __syncthreads();
      r = r_old + 1;
      pending_escape = true;
    }
    double lam_def = 0.0, lam_max = 0.0, lam_range = 0.0;
    bool certified = false;
    int status = XM_OK;
    for (;;) {
      if (!pending_escape) {
        // ---- FP32 bulk
        for (int e = threadIdx.x; e < (int)nR; e += NT) yf[e] = float(y64[e]);
        __syncthreads();
        rtr<float, float>(o.bulk_tol_rel, o.max_outer, true);
        for (int e = threadIdx.x; e < (int)nR; e += NT) y64[e] = double(yf[e]);
        __syncthreads();
        bool quick_escape = false;
        if (r < o.r_max) {
          certify(r, KQUICK, lam_def, lam_max, lam_range);
          quick_escape = lam_def < -1e-4 * fabs(lam_max);
        }
        double gap = 0.0;
        bool stationary = false;
        if (!quick_escape) {
          // FP64 polish from the FP64-projected iterate
          for (int e = threadIdx.x; e < (int)nR; e += NT) xi[e] = 0.0;
          __syncthreads();
          for (int i = threadIdx.x; i < N; i += NT) retract_block<double, double, R>(i, y64, xi, 0.0, yc64);
          __syncthreads();
          { double* t = y64; y64 = yc64; yc64 = t; }
          const unsigned long long tp0 = threadIdx.x == 0 ? gtimer() : 0ull;
          rtr<double, float>(o.grad_tol_rel, o.max_polish, false);
          if (threadIdx.x == 0) info.t_polish_ns += gtimer() - tp0;
          certify(r, 0, lam_def, lam_max, lam_range);
          const double regd = reg_dual();
          gap = f_cur - (lam[0] + lam[4] + lam[8] + regd);
          stationary = fabs(gap) <= 1e-6 * (1.0 + fabs(f_cur));
        }
        const double tau = o.cert_tau_rel * fmax(fabs(lam_max), 1e-300);
        certified = !quick_escape && lam_def >= -tau && stationary;
        if (certified) break;
        if (timed_out || (!quick_escape && lam_def >= -tau && !stationary)) { status = XM_ENOCONV; break; }
        if (r >= o.r_max) { status = XM_ENOTCERT; break; }
        // ---- escape (Thm. 2): into a null column of Y if one exists, else one rank up
        gram_eig(r);
        int col;
        if (sm.small[r - 1] < 1e-12 * sm.small[0]) {
          const double* E = sm.small + 64;
          for (int e = threadIdx.x; e < n; e += NT) {
            double y[R], t[R];
            for (int a = 0; a < R; ++a) y[a] = y64[(size_t)e * R + a];
            for (int b = 0; b < R; ++b) {
              double acc = 0.0;
              for (int a = 0; a < R; ++a)
                acc += y[a] * ((a < r && b < r) ? E[a * r + b] : (a == b ? 1.0 : 0.0));
              t[b] = acc;
            }
            for (int b = 0; b < R; ++b) y64[(size_t)e * R + b] = t[b];
          }
          __syncthreads();
          col = r - 1;
        } else if (r + 1 > R) {
          // hand the scene to the rank-8 kernel
          if (team_lead()) {
            if (threadIdx.x == 0) { spill[0] = ref_g; spill[1] = r; }
            for (int e = threadIdx.x; e < n; e += NT) {
              for (int j = 0; j < 4; ++j) spill[2 + (size_t)e * 4 + j] = y64[(size_t)e * R + j];
              spill[2 + (size_t)n * 4 + e] = lritz[e];
            }
          }
          __syncthreads();
          return false;
        } else {
          col = r;
          r += 1;
        }
        for (int e = threadIdx.x; e < n; e += NT)
          for (int j = 0; j < R; ++j) xi[(size_t)e * R + j] = j == col ? lritz[e] : 0.0;
        __syncthreads();
      }
      pending_escape = false;
      // ---- line search along the escape direction
      const double f0 = f_at(0.0);
      bool moved = false;
      double alpha = 1.0;
      for (int h = 0; h <= 30; ++h, alpha *= 0.5) {
        const double fa = f_at(alpha);
        if (fa < f0) {
          copy64(yh, y64, n * R);
          moved = true;
          break;
        }
      }
      ++info.n_escapes;
      if (!moved) { status = XM_ENOTCERT; break; }
      // every escape strictly lowers f; the cap bounds the work of a pathological scene
      if (info.n_escapes >= 4 * XM_MAX_RANK) { status = XM_ENOTCERT; break; }
    }
    // ---- rounding and the reported numbers
    const double rho_hat = round_and_eval(r);
    double yy[1] = {0.0};
    for (int e = threadIdx.x; e < (int)nR; e += NT) yy[0] += y64[e] * y64[e];
    bsum<1>(yy, sm.red);
    const double regd = reg_dual();
    const double dual = lam[0] + lam[4] + lam[8] + regd;
    const double lmin = fmin(lam_def, lam_range);
    info.f = f_cur;
    info.grad_norm = sqrt(cur_g2);
    info.lambda_min_deflated = lam_def;
    info.lambda_min = lmin;
    info.lambda_max = lam_max;
    info.dual = dual;
    info.rho_hat = rho_hat;
    info.eta = (rho_hat - f_cur) / (1.0 + fabs(rho_hat) + fabs(f_cur));
    const double lower = dual + fmin(0.0, lmin) * yy[0];
    info.eta_robust = (rho_hat - lower) / (1.0 + fabs(rho_hat) + fabs(lower));
    info.rank = r;
    info.certified = certified ? 1 : 0;
    info.status = status;
    return true;
  }
};

// ------------------------------------------------------------------ kernels
// Persistent batched solve: CTA-per-scene work queue (scenes in descending size order).  The
// rank-4 kernel runs every scene; a scene that needs rank > 4 is handed to the rank-8 kernel
// (launched right after it, which only takes the handed-over scenes).
template <int R>
__global__ void __launch_bounds__(NT, 1) k_batched(Params p) {
  extern __shared__ __align__(16) char smem_base[];
  __shared__ int s_job;
  if (threadIdx.x == 0) { s_team = (int)cl_size(); s_pfd = p.pf_dist; }
  __syncthreads();
  const Desc* descs = p.desc;
  int S = p.S;
  unsigned* queue = p.queue;
  bool second = false;
  for (;;) {
    // a team's rank 0 claims the next scene for the whole team
    const int tm = team();
    if (tm > 1) cl_sync();               // every CTA has read the previous claim
    if (threadIdx.x == 0 && cl_rank() == 0) {
      const int job = (int)atomicAdd(queue, 1u);
      s_job = job;
      for (int k = 1; k < tm; ++k) cl_st(cl_map(&s_job, (unsigned)k), job);
    } else if (threadIdx.x == 0 && tm == 1) {
      s_job = (int)atomicAdd(queue, 1u);
    }
    if (tm > 1) cl_sync();
    else __syncthreads();
    const int job = s_job;
    __syncthreads();
    if (job >= S) {
      // this launch's own scenes are all claimed: its CTAs go on one by one with the queue it
      // shares with the launch beside it (every CTA of a team saw the same claim)
      if (!second && p.queue2) {
        second = true;
        descs = p.desc2;
        S = p.S2;
        queue = p.queue2;
        if (threadIdx.x == 0) s_team = 1;
        __syncthreads();
        continue;
      }
      break;
    }
    const Desc d = descs[job];
    if (tm > 1 && d.n < p.team_min_n) {
      // below the team threshold: the cluster splits up, rank 0 keeps this scene alone and the
      // others go back to the queue
      if (threadIdx.x == 0) s_team = 1;
      __syncthreads();
      if (cl_rank() != 0) continue;
    }
    xm_batch_info* out = p.out + d.scene;
    if (R == 8 && out->status != XM_BATCH_HANDOVER) continue;
    Cta<R> c;
    c.setup(&p, d, smem_base);
    const bool resume = (R == 8);
    if (resume) {
      c.info = *out;
    } else {
      c.info = xm_batch_info{};
      c.info.N = d.N;
      c.info.t_begin_ns = gtimer();
    }
    __syncthreads();
    const bool finished = c.run(resume);
    __syncthreads();
    if (threadIdx.x == 0 && team_lead()) {
      if (!finished) c.info.status = XM_BATCH_HANDOVER;
      c.info.t_end_ns = gtimer();
      *out = c.info;
    }
    __syncthreads();
  }
}

// Autotuner probe: persistent CTAs (one per SM, as the solver) each run `reps` FP32 sweeps
// (r = 4) of their scenes with one tiling variant and record the clock cycles per scene.
template <int RPW, int U>
__global__ void __launch_bounds__(NT, 1) k_tune_sweep(const Desc* desc, const float* Q32, int S, int NM, int reps,
                                                     int pfd, long long* cycles) {
  extern __shared__ __align__(16) char smem_base[];
  if (threadIdx.x == 0) s_pfd = pfd;
  __syncthreads();
  for (int j = blockIdx.x; j < S; j += gridDim.x) {
    const Desc d = desc[j];
    float* xs = reinterpret_cast<float*>(smem_base);
    float* ws = xs + (size_t)NM * 4;
    for (int e = threadIdx.x; e < d.ldq * 4; e += NT) xs[e] = e % d.ldq < d.n ? 1.0f / (1 + (e % 7)) : 0.0f;
    __syncthreads();
    const long long t0 = clock64();
    for (int k = 0; k < reps; ++k) {
      sweep32_t<4, RPW, U>(Q32 + d.q32, 0, d.n, d.ldq, xs, ws);
      __syncthreads();
    }
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[j] = t1 - t0;
    __syncthreads();
  }
}

}  // namespace bat
}  // namespace xm

// ====================================================================================== host
namespace xm {
xm_status unpack_dense(xm_ctx* ctx, const DeviceQ& q, double* Qd);

// dense n x n FP64 -> row-padded (n x ldq) FP64 and FP32 copies, zero padding
__global__ void k_pack_batch_scene(const double* __restrict__ Qd, int n, int ldq, double* __restrict__ q64,
                                   float* __restrict__ q32) {
  const int64_t total = (int64_t)n * ldq;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / ldq), col = (int)(e % ldq);
    const double v = col < n ? Qd[(size_t)row * n + col] : 0.0;
    q64[e] = v;
    q32[e] = float(v);
  }
}
}  // namespace xm

struct xm_batch {
  int S = 0, NM = 0, n_max = 0;
  int64_t total_cams = 0;
  std::vector<xm::bat::Desc> desc_h;       // queue order
  xm::bat::Desc* desc = nullptr;
  float* Q32 = nullptr;
  double* Q64 = nullptr;
  double* spill = nullptr;
  xm_batch_info* out = nullptr;
  unsigned* queue = nullptr;
  int tile[xm::bat::NCLASS] = {1, 2, 2, 3};
  bool tuned = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaStream_t stream2 = nullptr;           // the 4-CTA launch beside the pairs (captured fork)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* slots = nullptr;
  size_t slots_doubles = 0;
  // graph cache
  cudaGraphExec_t gexec = nullptr;
  xm_opts gopts{};
  double* gR = nullptr;
  double* gs = nullptr;
  int gkmax = 0;
  int cluster = 0;                          // CTAs per large scene (0: automatic)
  int team_n = 0;                           // rows from which a scene is large (0: automatic)
  int gcs = 0, gteam = 0;                   // the captured graph's cluster size and threshold
  int gquad = -1;                           // and its number of scenes on 4-CTA clusters
  int glaunches = 0;                        // kernel launches per replay of the graph
  int pf = 1, gpf = -1;                     // sweep L2 prefetch distance (and the graph's): one
                                            // round measured best on the 256-scene batch (2 and 3
                                            // evict rows still in use)
};

using namespace xm;

namespace {

void batch_release(xm_batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  void* ps[] = {b->desc, b->Q32, b->Q64, b->spill, b->out, b->queue, b->slots};
  for (void* p : ps) if (p) cudaFree(p);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->stream) cudaStreamDestroy(b->stream);
  if (b->stream2) cudaStreamDestroy(b->stream2);
  delete b;
}

}  // namespace

extern "C" xm_status xm_batch_create(xm_ctx* c, int S, const xm_qmat* const* qs, xm_batch** out) {
  if (!c || !qs || !out || S < 1) return set_error(XM_EINVAL, "xm_batch_create: bad arguments");
  *out = nullptr;
  XM_CUDA_TRY(cudaSetDevice(c->device));
  std::vector<int> order(S);
  for (int j = 0; j < S; ++j) {
    if (!qs[j]) return set_error(XM_EINVAL, "xm_batch_create: scene %d has no Q", j);
    if (!qs[j]->d.q64) return set_error(XM_EINVAL, "xm_batch_create: scene %d's Q has no FP64 copy", j);
    order[j] = j;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return qs[a]->d.n > qs[b]->d.n; });
  xm_batch* b = new xm_batch();
  b->S = S;
  std::vector<int64_t> cam0(S);
  int64_t cams = 0;
  for (int j = 0; j < S; ++j) { cam0[j] = cams; cams += qs[j]->d.N; }
  b->total_cams = cams;
  int64_t o64 = 0, osp = 0;
  for (int k = 0; k < S; ++k) {
    const int j = order[k];
    bat::Desc d{};
    d.N = qs[j]->d.N;
    d.n = qs[j]->d.n;
    d.ldq = (d.n + 3) & ~3;
    d.scene = j;
    d.q32 = o64;
    d.q64 = o64;
    d.cam0 = cam0[j];
    d.spill = osp;
    o64 += (int64_t)d.n * d.ldq;
    osp += 2 + 5 * (int64_t)d.n;
    b->NM = std::max(b->NM, d.ldq);
    b->n_max = std::max(b->n_max, d.n);
    b->desc_h.push_back(d);
  }
  auto fail = [&](xm_status st) { batch_release(b); return st; };
#define XB_TRY(...)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (__VA_ARGS__);                                                        \
    if (e_ != cudaSuccess)                                                                 \
      return fail(set_error(e_ == cudaErrorMemoryAllocation ? XM_ENOMEM : XM_ECUDA,        \
                            "%s failed: %s", #__VA_ARGS__, cudaGetErrorString(e_)));       \
  } while (0)
  XB_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  XB_TRY(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
  XB_TRY(cudaStreamCreateWithFlags(&b->stream2, cudaStreamNonBlocking));
  XB_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  XB_TRY(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
  XB_TRY(cudaMalloc(&b->desc, sizeof(bat::Desc) * S));
  XB_TRY(cudaMalloc(&b->Q32, sizeof(float) * (size_t)o64));
  XB_TRY(cudaMalloc(&b->Q64, sizeof(double) * (size_t)o64));
  XB_TRY(cudaMalloc(&b->spill, sizeof(double) * (size_t)osp));
  XB_TRY(cudaMalloc(&b->out, sizeof(xm_batch_info) * S));
  XB_TRY(cudaMalloc(&b->queue, sizeof(unsigned) * 4));
  XB_TRY(cudaMemcpyAsync(b->desc, b->desc_h.data(), sizeof(bat::Desc) * S, cudaMemcpyHostToDevice, c->stream));
  double* tmp = nullptr;
  XB_TRY(cudaMalloc(&tmp, sizeof(double) * (size_t)b->n_max * b->n_max));
  for (int k = 0; k < S; ++k) {
    const bat::Desc& d = b->desc_h[k];
    xm_status st = unpack_dense(c, qs[d.scene]->d, tmp);
    if (st != XM_OK) { cudaFree(tmp); return fail(st); }
    const int64_t total = (int64_t)d.n * d.ldq;
    const int g = (int)std::min<int64_t>((total + 255) / 256, (int64_t)c->num_sms * 8);
    k_pack_batch_scene<<<std::max(g, 1), 256, 0, c->stream>>>(tmp, d.n, d.ldq, b->Q64 + d.q64, b->Q32 + d.q32);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { cudaFree(tmp); return fail(set_error(XM_ECUDA, "pack: %s", cudaGetErrorString(e))); }
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(set_error(XM_ECUDA, "xm_batch_create: %s", cudaGetErrorString(e)));
#undef XB_TRY
  *out = b;
  return XM_OK;
}

extern "C" xm_status xm_batch_free(xm_ctx* c, xm_batch* b) {
  if (!b) return XM_OK;
  if (c) cudaSetDevice(c->device);
  batch_release(b);
  return XM_OK;
}

extern "C" xm_status xm_batch_launches(xm_ctx* c, const xm_batch* b, int* launches, int* quad_scenes) {
  if (!c || !b) return set_error(XM_EINVAL, "xm_batch_launches: NULL argument");
  if (!b->gexec) return set_error(XM_EINVAL, "xm_batch_launches: no batched solve yet");
  if (launches) *launches = b->glaunches;
  if (quad_scenes) *quad_scenes = b->gquad;
  return XM_OK;
}

extern "C" xm_status xm_batch_cluster(xm_ctx* c, xm_batch* b, int cs, int n_min) {
  if (!c || !b) return set_error(XM_EINVAL, "xm_batch_cluster: NULL argument");
  if (cs != 0 && cs != 1 && cs != 2 && cs != 4)
    return set_error(XM_EINVAL, "xm_batch_cluster: cs = %d not in {0, 1, 2, 4}", cs);
  if (n_min < 0) return set_error(XM_EINVAL, "xm_batch_cluster: n_min = %d < 0", n_min);
  b->cluster = cs;
  b->team_n = n_min;
  return XM_OK;
}

extern "C" xm_status xm_batch_autotune(xm_ctx* c, xm_batch* b, int reps, int* tile_out) {
  if (!c || !b) return set_error(XM_EINVAL, "xm_batch_autotune: NULL argument");
  if (reps < 1) reps = 1;
  XM_CUDA_TRY(cudaSetDevice(c->device));
  const int S = b->S;
  long long* dcyc = nullptr;
  XM_CUDA_TRY(cudaMalloc(&dcyc, sizeof(long long) * S));
  // the solver's own shared-memory footprint, so that one CTA per SM runs, as in the solve
  const size_t smem = std::max((size_t)b->NM * 4 * sizeof(float) * 2,
                               bat::smem_bytes(b->NM, 4, std::max(10, std::min(400, b->n_max))));
  const int grid = std::min(c->num_sms, S);
  double tot[bat::NTILE][bat::NCLASS] = {};
  std::vector<long long> cyc(S);
  xm_status st = XM_OK;
  for (int v = 0; v < bat::NTILE && st == XM_OK; ++v) {
    cudaError_t e = cudaSuccess;
#define XB_TUNE(RP, UU)                                                                           \
  e = cudaFuncSetAttribute(bat::k_tune_sweep<RP, UU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
  if (e == cudaSuccess) bat::k_tune_sweep<RP, UU><<<grid, bat::NT, smem, b->stream>>>(b->desc, b->Q32, S, b->NM, reps, b->pf, dcyc);
    switch (v) {
      case 0: XB_TUNE(2, 4) break;
      case 1: XB_TUNE(4, 1) break;
      case 2: XB_TUNE(4, 2) break;
      case 3: XB_TUNE(4, 4) break;
      case 4: XB_TUNE(8, 1) break;
      default: XB_TUNE(8, 2) break;
    }
#undef XB_TUNE
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(cyc.data(), dcyc, sizeof(long long) * S, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { st = set_error(XM_ECUDA, "xm_batch_autotune: %s", cudaGetErrorString(e)); break; }
    for (int k = 0; k < S; ++k) tot[v][bat::size_class(b->desc_h[k].n)] += (double)cyc[k];
  }
  cudaFree(dcyc);
  if (st != XM_OK) return st;
  for (int cl = 0; cl < bat::NCLASS; ++cl) {
    int best = -1;
    for (int v = 0; v < bat::NTILE; ++v)
      if (tot[v][cl] > 0 && (best < 0 || tot[v][cl] < tot[best][cl])) best = v;
    if (best >= 0) b->tile[cl] = best;
  }
  b->tuned = true;
  if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  if (tile_out)
    for (int cl = 0; cl < bat::NCLASS; ++cl) {
      tile_out[2 * cl] = bat::tile_rpw(b->tile[cl]);
      tile_out[2 * cl + 1] = bat::tile_u(b->tile[cl]);
    }
  return XM_OK;
}

extern "C" xm_status xm_solve_batched(xm_ctx* c, xm_batch* b, const xm_opts* opts, double* R_out,
                                      double* s_out, xm_batch_info* info) {
  if (!c || !b || !opts || !R_out || !s_out) return set_error(XM_EINVAL, "xm_solve_batched: NULL argument");
  const xm_opts& o = *opts;
  if (o.r0 < 3 || o.r0 > 4 || o.r_max < o.r0 || o.r_max > XM_MAX_RANK)
    return set_error(XM_EINVAL, "xm_solve_batched: need 3 <= r0 <= 4 and r0 <= r_max <= %d", XM_MAX_RANK);
  if (o.max_outer < 1 || o.max_tcg < 1 || o.lanczos_max < 1)
    return set_error(XM_EINVAL, "xm_solve_batched: iteration caps must be positive");
  if (!(o.scale_reg >= 0.0) || !std::isfinite(o.scale_reg))
    return set_error(XM_EINVAL, "xm_solve_batched: scale_reg must be finite and >= 0");
  XM_CUDA_TRY(cudaSetDevice(c->device));
  // The Krylov recurrence lives in shared memory beside the scene's sweep buffers, so the batched
  // certificate caps its dimension at XM_BATCH_KMAX whatever lanczos_max asks for.
  const int kmax = std::max(10, std::min(std::min(o.lanczos_max, xm::bat::XM_BATCH_KMAX), b->n_max));
  const size_t smem4 = bat::smem_bytes(b->NM, 4, kmax);
  const size_t smem8 = bat::smem_bytes(b->NM, 8, kmax);
  cudaFuncAttributes fa4{}, fa8{};
  XM_CUDA_TRY(cudaFuncGetAttributes(&fa4, bat::k_batched<4>));
  XM_CUDA_TRY(cudaFuncGetAttributes(&fa8, bat::k_batched<8>));
  if (smem4 + fa4.sharedSizeBytes > c->smem_optin || smem8 + fa8.sharedSizeBytes > c->smem_optin)
    return set_error(XM_EINVAL, "xm_solve_batched: largest scene (3N = %d) needs %zu bytes of shared "
                     "memory, above %zu", b->n_max, smem8 + fa8.sharedSizeBytes, c->smem_optin);
  XM_CUDA_TRY(cudaFuncSetAttribute(bat::k_batched<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem4));
  XM_CUDA_TRY(cudaFuncSetAttribute(bat::k_batched<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem8));
  // Teams: a scene whose solve alone would outlast the average load of a CTA sets the batch's
  // makespan, so it runs on a cluster of cs CTAs (its solve is mostly Q products, which the
  // cluster splits by rows).  Cost model: n^2 per scene (the products' bytes), spread over one
  // CTA per SM.  Without such a scene the launch has no clusters.  The automatic setting also
  // looks for scenes of QUAD_FACTOR times that size: when at least two exist they run on 4-CTA
  // clusters in a launch beside the pairs (two branches of the graph, disjoint slots), the
  // pairs then starting at PAIR_FACTOR times it; both launches go on with single CTAs from one
  // shared queue once their team scenes are claimed.
  auto max_clusters = [&](int csz, int* out) -> xm_status {
    int ncl = 0;
    for (int pass = 0; pass < 2; ++pass) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(csz * std::max(1, c->num_sms / csz));
      cfg.blockDim = dim3(bat::NT);
      cfg.dynamicSmemBytes = pass == 0 ? smem4 : smem8;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = csz;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int k = 0;
      XM_CUDA_TRY(cudaOccupancyMaxActiveClusters(&k, pass == 0 ? (const void*)bat::k_batched<4>
                                                                : (const void*)bat::k_batched<8>, &cfg));
      ncl = pass == 0 ? k : std::min(ncl, k);
    }
    *out = ncl;
    return XM_OK;
  };
  int cs = b->cluster > 0 ? b->cluster : 2;
  int team_n = b->team_n;
  int nquad = 0;
  if (cs > 1 && team_n == 0) {
    double w = 0.0;
    for (const bat::Desc& d : b->desc_h) w += (double)d.n * d.n;
    const double base = std::sqrt(w / c->num_sms);
    team_n = (int)std::ceil(base);
    if (b->cluster == 0) {
      const int quad_n = (int)std::ceil(bat::QUAD_FACTOR * base);
      for (const bat::Desc& d : b->desc_h) nquad += d.n >= quad_n;
      nquad = std::min(nquad, c->num_sms / 16);
      if (nquad >= 2) team_n = (int)std::ceil(bat::PAIR_FACTOR * base);
      else nquad = 0;
    }
  }
  if (b->n_max < team_n) { cs = 1; nquad = 0; }
  if (cs == 1) team_n = 0;
  int grid = std::min(c->num_sms, b->S);   // the single launch, and the rank-8 launch
  int gridA = 0, gridB = 0;                 // the 4-CTA launch and the pairs beside it
  if (cs > 1) {
    int ncl = 0;
    XM_TRY(max_clusters(cs, &ncl));
    if (ncl < 1) return set_error(XM_EINVAL, "xm_solve_batched: no cluster of %d CTAs fits on this device", cs);
    int big = 0;
    for (const bat::Desc& d : b->desc_h) big += d.n >= team_n;
    grid = cs * std::min(ncl, big + (b->S - big + cs - 1) / cs);   // teams, then single CTAs
    if (nquad > 0) {
      int ncl4 = 0;
      XM_TRY(max_clusters(4, &ncl4));
      nquad = std::min(nquad, ncl4);
      if (nquad >= 2) {
        gridA = 4 * nquad;
        const int SB = b->S - nquad;
        int bigB = 0;
        for (int j = nquad; j < b->S; ++j) bigB += b->desc_h[j].n >= team_n;
        const int avail = (c->num_sms - gridA) / 2;
        gridB = 2 * std::max(1, std::min(std::min(ncl, avail), bigB + (SB - bigB + 1) / 2));
      } else {
        nquad = 0;
      }
    }
  }
  const int nslots = std::max(grid, gridA + gridB);
  const size_t slot_doubles = ((size_t)bat::NVEC * b->NM * 8 + (size_t)b->NM * (XM_MAX_RANK + kmax + 1) +
                               2 * (size_t)b->NM + 31) & ~size_t(31);
  if (!b->slots || b->slots_doubles < slot_doubles * nslots) {
    if (b->slots) cudaFree(b->slots);
    b->slots = nullptr;
    b->slots_doubles = 0;
    XM_CUDA_TRY(cudaMalloc(&b->slots, sizeof(double) * slot_doubles * nslots));
    b->slots_doubles = slot_doubles * nslots;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
  }
  if (!b->tuned) XM_TRY(xm_batch_autotune(c, b, 8, nullptr));
  // order after the caller's work on the context stream
  XM_CUDA_TRY(cudaEventRecord(b->ev, c->stream));
  XM_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev, 0));
  const bool same = b->gexec && b->gR == R_out && b->gs == s_out && b->gkmax == kmax && b->gcs == cs && b->gteam == team_n && b->gquad == nquad && b->gpf == b->pf &&
                    std::memcmp(&b->gopts, &o, sizeof(xm_opts)) == 0;
  if (!same) {
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    bat::Params p{};
    p.desc = b->desc;
    p.S = b->S;
    p.Q32 = b->Q32;
    p.Q64 = b->Q64;
    p.slots = b->slots;
    p.slot_doubles = (int64_t)slot_doubles;
    p.NM = b->NM;
    p.kmax = kmax;
    p.spill = b->spill;
    p.R_out = R_out;
    p.s_out = s_out;
    p.out = b->out;
    for (int cl = 0; cl < bat::NCLASS; ++cl) p.tile[cl] = b->tile[cl];
    p.o = o;
    p.mu = o.scale_reg;
    p.time_limit_ns = o.time_limit_s > 0 ? (unsigned long long)(o.time_limit_s * 1e9) : 0ull;
    p.team_min_n = team_n;
    p.pf_dist = b->pf;
    p.slot_base = 0;
    p.queue2 = nullptr;
    p.desc2 = nullptr;
    p.S2 = 0;
    bat::Params p8 = p;
    p.queue = b->queue;
    p8.queue = b->queue + 1;
    // queues: [0] the pairs (or the single launch), [1] the rank-8 launch, [2] the 4-CTA launch
    bat::Params pA = p, pB = p;
    if (nquad > 0) {
      pA.S = nquad;
      pA.queue = b->queue + 2;
      pA.team_min_n = 0;
      pA.queue2 = b->queue;
      pA.desc2 = b->desc + nquad;
      pA.S2 = b->S - nquad;
      pB.desc = b->desc + nquad;
      pB.S = b->S - nquad;
      pB.slot_base = gridA;
    }
    auto launch = [&](cudaStream_t stv, int g, int csz, size_t smem, bool r8, const bat::Params& pp) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(g);
      cfg.blockDim = dim3(bat::NT);
      cfg.stream = stv;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = csz;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cfg.dynamicSmemBytes = smem;
      if (r8) cudaLaunchKernelEx(&cfg, bat::k_batched<8>, pp);
      else cudaLaunchKernelEx(&cfg, bat::k_batched<4>, pp);
    };
    cudaGraph_t graph = nullptr;
    XM_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(b->queue, 0, sizeof(unsigned) * 4, b->stream);
    if (nquad > 0) {
      cudaEventRecord(b->ev_fork, b->stream);
      cudaStreamWaitEvent(b->stream2, b->ev_fork, 0);
      launch(b->stream2, gridA, 4, smem4, false, pA);
      launch(b->stream, gridB, 2, smem4, false, pB);
      cudaEventRecord(b->ev_join, b->stream2);
      cudaStreamWaitEvent(b->stream, b->ev_join, 0);
    } else {
      launch(b->stream, grid, cs, smem4, false, p);
    }
    if (o.r_max > 4) launch(b->stream, grid, cs, smem8, true, p8);
    const cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
    if (ec != cudaSuccess) return set_error(XM_ECUDA, "xm_solve_batched: capture failed: %s", cudaGetErrorString(ec));
    const cudaError_t ei = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      b->gexec = nullptr;
      return set_error(XM_ECUDA, "xm_solve_batched: graph instantiate failed: %s", cudaGetErrorString(ei));
    }
    b->gR = R_out;
    b->gs = s_out;
    b->gkmax = kmax;
    b->gcs = cs;
    b->gteam = team_n;
    b->gquad = nquad;
    b->glaunches = (nquad > 0 ? 2 : 1) + (o.r_max > 4 ? 1 : 0);
    b->gpf = b->pf;
    b->gopts = o;
  }
  XM_CUDA_TRY(cudaGraphLaunch(b->gexec, b->stream));
  XM_CUDA_TRY(cudaStreamSynchronize(b->stream));
  g_last_launches = o.r_max > 4 ? 2 : 1;
  std::vector<xm_batch_info> h(b->S);
  XM_CUDA_TRY(cudaMemcpy(h.data(), b->out, sizeof(xm_batch_info) * b->S, cudaMemcpyDeviceToHost));
  long sweeps = 0;
  int worst = XM_OK;
  for (const auto& x : h) {
    sweeps += x.n_sweeps;
    if (x.status == XM_ENOCONV) worst = XM_ENOCONV;
    else if (x.status != XM_OK && worst == XM_OK) worst = x.status;
  }
  g_last_sweeps = sweeps;
  if (info) std::memcpy(info, h.data(), sizeof(xm_batch_info) * b->S);
  if (worst == XM_ENOTCERT) return set_error(XM_ENOTCERT, "xm_solve_batched: some scenes stopped at r_max without a certificate");
  if (worst == XM_ENOCONV) return set_error(XM_ENOCONV, "xm_solve_batched: some scenes hit the time limit or iteration caps");
  if (worst != XM_OK) return set_error((xm_status)worst, "xm_solve_batched: scene status %d", worst);
  return XM_OK;
}
