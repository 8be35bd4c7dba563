// Construction of the reduced data matrix Q (Prop. 1, App. A) on the device, in FP64.
//
//   1. validate observations, accumulate per camera Q1 blocks (sum w u u^T), V1 (sum w u) and
//      Q2 (sum w), per landmark Q3 (d_k = sum w);
//   2. landmark elimination: for every landmark the camera pairs (a, b) of its observers get
//      P_ab -= w_a w_b u_a u_b^T / d_k, B_ab -= w_a w_b u_a / d_k, S_ab -= w_a w_b / d_k
//      (P = Q1 - V2 D^-1 V2^T, B = V1 - V2 D^-1 V3^T, S = Q2 - V3 D^-1 V3^T with D = Q3);
//   3. translation elimination with the anchor t_0 = 0: Sbar = L L^T (Cholesky), C = L^-1 Bbar^T
//      (dense FP64 factor and triangular solve from cuSOLVER / cuBLAS: the paper's "large dense
//      matrix multiplications"), then Q = P - C^T C: either cuSOLVER DPOTRF + cuBLAS DTRSM + DSYRK
//      (FP64 units) or, with XM_BUILD_SPLIT_BF16, the blocked Cholesky factor, blocked triangular
//      solve and rank-k update of xm_ozaki.cu with their dense products on the BF16 tensor
//      cores (digit splitting, FP64-accurate);
//   4. pack the upper triangle into the tile layout of the sweep kernel (FP64 / FP32 / BF16);
//      the tensor-core update writes the packed tiles itself.
// Connectivity of the view graph (rank N+M-1 of the Laplacian Q_tp, App. A lemma) is checked
// with a union-find over the camera-landmark edges before any elimination.

#include <algorithm>
#include <chrono>

#include "xm_internal.cuh"

namespace xm {

// ------------------------------------------------------------------ validation / sums
__global__ void k_validate(int64_t E, int N, int M, const int32_t* cam, const int32_t* lmk,
                           const double* ukp, const double* w, int* err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = cam[e], k = lmk[e];
    if (i < 0 || i >= N || k < 0 || k >= M) atomicOr(err, DEV_BAD_INDEX);
    const double ww = w[e];
    const double u0 = ukp[3 * e], u1 = ukp[3 * e + 1], u2 = ukp[3 * e + 2];
    if (!(ww > 0.0) || !isfinite(ww) || !isfinite(u0) || !isfinite(u1) || !isfinite(u2))
      atomicOr(err, DEV_BAD_VALUE);
  }
}

// union-find over vertices 0..N-1 (cameras) and N..N+M-1 (landmarks).  Links always point from
// a larger to a smaller index, so every parent chain strictly decreases and find() terminates.
__device__ int uf_find(int* parent, int x) {
  while (true) {
    const int p = parent[x];
    if (p == x) return x;
    const int gp = parent[p];
    if (gp != p) atomicCAS(&parent[x], p, gp);   // path halving (benign race)
    x = p;
  }
}
__global__ void k_uf_init(int* parent, int nv) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x)
    parent[v] = v;
}
__global__ void k_uf_union(int64_t E, int N, const int32_t* cam, const int32_t* lmk, int* parent) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a = cam[e], b = N + lmk[e];
    for (int guard = 0; guard < (1 << 20); ++guard) {
      int ra = uf_find(parent, a), rb = uf_find(parent, b);
      if (ra == rb) break;
      if (ra < rb) { const int t = ra; ra = rb; rb = t; }
      if (atomicCAS(&parent[ra], ra, rb) == ra) break;   // link the larger root under the smaller
    }
  }
}
// every camera and every observed landmark must share camera 0's root
__global__ void k_uf_check(int64_t E, int N, const int32_t* cam, const int32_t* lmk, int* parent,
                           int* disconnected) {
  const int r0 = uf_find(parent, 0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E + N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int v = e < E ? N + lmk[e] : (int)(e - E);
    if (uf_find(parent, v) != r0) *disconnected = 1;
  }
}

// per-observation terms on the camera diagonal: Q1 block (upper entries), V1 column, Q2;
// and the landmark weight sums d_k and counts.
__global__ void k_camera_terms(int64_t E, int n, int N, const int32_t* cam, const int32_t* lmk,
                               const double* ukp, const double* w, double* P, double* B,
                               double* S, double* d, int* cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = cam[e], k = lmk[e];
    const double ww = w[e];
    const double u[3] = {ukp[3 * e], ukp[3 * e + 1], ukp[3 * e + 2]};
    for (int p = 0; p < 3; ++p) {
      for (int q = p; q < 3; ++q) atomicAdd(&P[(size_t)(3 * i + p) * n + 3 * i + q], ww * u[p] * u[q]);
      atomicAdd(&B[(size_t)(3 * i + p) * N + i], ww * u[p]);
    }
    atomicAdd(&S[(size_t)i * N + i], ww);
    atomicAdd(&d[k], ww);
    atomicAdd(&cnt[k], 1);
  }
}

// ------------------------------------------------------------------ landmark CSR
// exclusive scan of cnt[0..M) into off[0..M] (blocks of 1024, two levels)
__global__ void k_scan_blocks(const int* in, int64_t* out, int64_t* bsum, int M) {
  __shared__ int64_t sh[1024];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  int64_t v = i < M ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < M) out[i] = sh[threadIdx.x] - v;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = sh[1023];
}
__global__ void k_scan_sums(int64_t* bsum, int nb) {   // one thread: nb is small (M / 1024)
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t run = 0;
    for (int b = 0; b < nb; ++b) { const int64_t t = bsum[b]; bsum[b] = run; run += t; }
    bsum[nb] = run;
  }
}
__global__ void k_scan_add(int64_t* out, const int64_t* bsum, int M) {
  const int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < M) out[i] += bsum[blockIdx.x];
  if (i == 0) out[M] = bsum[(M + 1023) / 1024];
}
__global__ void k_csr_fill(int64_t E, const int32_t* lmk, const int64_t* off, int* cursor,
                           int64_t* idx) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = lmk[e];
    const int pos = atomicAdd(&cursor[k], 1);
    idx[off[k] + pos] = e;
  }
}
// Deterministic order within each group (landmark or camera): its observation indices ascending.
// Groups of at most CSR_SMALL entries (the landmarks' tracks) are sorted by one thread each;
// larger ones (a camera's observations) are queued for k_csr_sort_big.
constexpr int CSR_SMALL = 16;
constexpr int CSR_BIG_THREADS = 512;
constexpr int CSR_OWN = 16;                          // entries per thread in k_csr_sort_big
constexpr int CSR_BIG_MAX = CSR_BIG_THREADS * CSR_OWN;
constexpr int CSR_CHUNK = 4096;                      // entries staged in shared memory at a time
__global__ void k_csr_sort(int M, const int64_t* off, int64_t* idx, int* big, int* nbig) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    const int64_t a = off[k], b = off[k + 1];
    if (b - a > CSR_SMALL) {
      big[atomicAdd(nbig, 1)] = k;
      continue;
    }
    for (int64_t x = a + 1; x < b; ++x) {
      const int64_t v = idx[x];
      int64_t y = x - 1;
      while (y >= a && idx[y] > v) { idx[y + 1] = idx[y]; --y; }
      idx[y + 1] = v;
    }
  }
}
// One block per queued group: the entries are distinct, so entry v goes to position
// #{entries < v} (counted against chunks of the group staged in shared memory), written to tmp
// and copied back.  Groups beyond CSR_BIG_MAX entries fall back to one thread's insertion sort
// (correct, slow).
__global__ void __launch_bounds__(CSR_BIG_THREADS) k_csr_sort_big(const int64_t* off, int64_t* idx,
                                                                 int64_t* tmp, const int* big,
                                                                 const int* nbig) {
  __shared__ int64_t sv[CSR_CHUNK];
  const int t = threadIdx.x;
  const int ng = *nbig;
  for (int g = blockIdx.x; g < ng; g += gridDim.x) {
    const int key = big[g];
    const int64_t a = off[key], b = off[key + 1], k = b - a;
    if (k > CSR_BIG_MAX) {
      if (t == 0)
        for (int64_t x = a + 1; x < b; ++x) {
          const int64_t v = idx[x];
          int64_t y = x - 1;
          while (y >= a && idx[y] > v) { idx[y + 1] = idx[y]; --y; }
          idx[y + 1] = v;
        }
      __syncthreads();
      continue;
    }
    int64_t val[CSR_OWN];
    int cnt[CSR_OWN];
#pragma unroll
    for (int m = 0; m < CSR_OWN; ++m) {
      const int64_t j = a + t + (int64_t)CSR_BIG_THREADS * m;
      val[m] = j < b ? idx[j] : INT64_MAX;
      cnt[m] = 0;
    }
    for (int64_t c0 = a; c0 < b; c0 += CSR_CHUNK) {
      const int ch = (int)min((int64_t)CSR_CHUNK, b - c0);
      __syncthreads();
      for (int q = t; q < ch; q += CSR_BIG_THREADS) sv[q] = idx[c0 + q];
      __syncthreads();
      for (int q = 0; q < ch; ++q) {
        const int64_t x = sv[q];
#pragma unroll
        for (int m = 0; m < CSR_OWN; ++m) cnt[m] += x < val[m] ? 1 : 0;
      }
    }
#pragma unroll
    for (int m = 0; m < CSR_OWN; ++m)
      if (a + t + (int64_t)CSR_BIG_THREADS * m < b) tmp[a + cnt[m]] = val[m];
    __syncthreads();
    for (int64_t q = t; q < k; q += CSR_BIG_THREADS) idx[a + q] = tmp[a + q];
    __syncthreads();
  }
}

// landmark elimination: one thread per landmark, all ordered observer pairs
__global__ void k_landmark_schur(int M, int n, int N, const int64_t* off, const int64_t* idx,
                                 const int32_t* cam, const double* ukp, const double* w,
                                 const double* d, double* P, double* B, double* S) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    const int64_t a0 = off[k], a1 = off[k + 1];
    if (a1 - a0 < 1 || !(d[k] > 0.0)) continue;
    const double dinv = 1.0 / d[k];
    for (int64_t x = a0; x < a1; ++x) {
      const int64_t ea = idx[x];
      const int i = cam[ea];
      const double wa = w[ea] * dinv;
      const double ua[3] = {ukp[3 * ea], ukp[3 * ea + 1], ukp[3 * ea + 2]};
      for (int64_t y = a0; y < a1; ++y) {
        const int64_t eb = idx[y];
        const int j = cam[eb];
        const double c = wa * w[eb];
        const double ub[3] = {ukp[3 * eb], ukp[3 * eb + 1], ukp[3 * eb + 2]};
        for (int p = 0; p < 3; ++p) atomicAdd(&B[(size_t)(3 * i + p) * N + j], -c * ua[p]);
        if (i < j) {
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q)
              atomicAdd(&P[(size_t)(3 * i + p) * n + 3 * j + q], -c * ua[p] * ub[q]);
          atomicAdd(&S[(size_t)i * N + j], -c);
        } else if (i == j) {
          for (int p = 0; p < 3; ++p)
            for (int q = p; q < 3; ++q)
              atomicAdd(&P[(size_t)(3 * i + p) * n + 3 * i + q], -c * ua[p] * ub[q]);
          atomicAdd(&S[(size_t)i * N + i], -c);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ tile packing
// Reads the upper triangle (row <= col) of a row-major n x n matrix (equivalently the lower
// triangle of a column-major one); one block per tile.
template <typename TI>
__global__ void k_pack_tiles(const TI* __restrict__ Qd, int n, int nt, int64_t ntiles,
                             double* q64, float* q32, __nv_bfloat16* q16) {
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // tile coordinates from the linear index (row-major upper triangle)
    int I = (int)(((2.0f * nt + 1.0f) -
                   sqrtf((2.0f * nt + 1.0f) * (2.0f * nt + 1.0f) - 8.0f * (float)t)) * 0.5f);
    if (I < 0) I = 0;
    if (I > nt - 1) I = nt - 1;
    while (I > 0 && tile_index(nt, I, I) > t) --I;
    while (I + 1 < nt && tile_index(nt, I + 1, I + 1) <= t) ++I;
    const int J = I + (int)(t - tile_index(nt, I, I));
    const int64_t g0 = t * TILE * TILE;
    for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
      const int a = e / TILE, b = e % TILE;
      const int row = I * TILE + a, col = J * TILE + b;
      double v = 0.0;
      if (row < n && col < n) {
        if (I < J || a < b) v = (double)Qd[(size_t)row * n + col];
        else if (a == b) v = 0.5 * (double)Qd[(size_t)row * n + col];
      }
      if (q64) q64[g0 + e] = v;
      if (q32) q32[g0 + e] = (float)v;
      if (q16) q16[g0 + bf16_tile_off(a, b)] = __double2bfloat16(v);
    }
  }
}

// dense symmetric n x n from FP64 tiles
__global__ void k_unpack_tiles(const double* __restrict__ q64, int n, int nt, double* Qd) {
  const int64_t total = (int64_t)n * n;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int row = (int)(g / n), col = (int)(g % n);
    if (row > col) { const int t = row; row = col; col = t; }
    const int I = row / TILE, J = col / TILE, a = row % TILE, b = col % TILE;
    double v = q64[tile_index(nt, I, J) * TILE * TILE + (int64_t)a * TILE + b];
    if (I == J && a == b) v *= 2.0;
    Qd[g] = v;
  }
}

static int grid_for(int64_t work, int threads, int num_sms) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

xm_status alloc_tiles(xm_ctx* ctx, DeviceQ& q, int N, unsigned mask) {
  (void)ctx;
  q.N = N;
  q.n = 3 * N;
  q.nt = (q.n + TILE - 1) / TILE;
  q.n_pad = q.nt * TILE;
  q.ntiles = tile_count(q.nt);
  q.mask = mask;
  const size_t elems = (size_t)q.ntiles * TILE * TILE;
  if (mask & XM_STORE_FP64) XM_CUDA_TRY(cudaMalloc(&q.q64, elems * sizeof(double)));
  if (mask & XM_STORE_FP32) XM_CUDA_TRY(cudaMalloc(&q.q32, elems * sizeof(float)));
  if (mask & XM_STORE_BF16) {
    XM_CUDA_TRY(cudaMalloc(&q.q16, elems * sizeof(__nv_bfloat16)));
    XM_CUDA_TRY(cudaMalloc(&q.ydig, (size_t)32 * q.n_pad * sizeof(__nv_bfloat16)));
  }
  return XM_OK;
}

void free_tiles(DeviceQ& q) {
  if (q.fact) {
    qfact_release(*q.fact);
    delete q.fact;
    q.fact = nullptr;
  }
  if (q.q64) cudaFree(q.q64);
  if (q.q32) cudaFree(q.q32);
  if (q.q16) cudaFree(q.q16);
  if (q.ydig) cudaFree(q.ydig);
  q.q64 = nullptr; q.q32 = nullptr; q.q16 = nullptr; q.ydig = nullptr;
}

xm_status pack_dense(xm_ctx* ctx, DeviceQ& q, const double* Qd) {
  const int grid = (int)(q.ntiles < (int64_t)ctx->num_sms * 16 ? q.ntiles : (int64_t)ctx->num_sms * 16);
  k_pack_tiles<double><<<grid, 256, 0, ctx->stream>>>(Qd, q.n, q.nt, q.ntiles, q.q64, q.q32, q.q16);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

xm_status pack_dense_f32(xm_ctx* ctx, DeviceQ& q, const float* A) {
  const int grid = (int)(q.ntiles < (int64_t)ctx->num_sms * 16 ? q.ntiles : (int64_t)ctx->num_sms * 16);
  k_pack_tiles<float><<<grid, 256, 0, ctx->stream>>>(A, q.n, q.nt, q.ntiles, q.q64, q.q32, q.q16);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

xm_status unpack_dense(xm_ctx* ctx, const DeviceQ& q, double* Qd) {
  if (!q.q64) return set_error(XM_EINVAL, "Q has no FP64 copy to unpack");
  const int64_t total = (int64_t)q.n * q.n;
  k_unpack_tiles<<<grid_for(total, 256, ctx->num_sms), 256, 0, ctx->stream>>>(q.q64, q.n, q.nt, Qd);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

namespace {
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  template <typename T> T* as() { return static_cast<T*>(p); }
};
}  // namespace

// XM_EDISCONNECTED unless every camera and every observed landmark lie in one component of the
// camera-landmark view graph (App. A lemma: Q_tp has rank N + M - 1 exactly then).
xm_status check_connected(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk) {
  cudaStream_t st = ctx->stream;
  const int threads = 256;
  DevBuf parent, flag;
  XM_CUDA_TRY(cudaMalloc(&parent.p, sizeof(int) * (size_t)(N + M)));
  XM_CUDA_TRY(cudaMalloc(&flag.p, sizeof(int)));
  XM_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
  k_uf_init<<<grid_for(N + M, threads, ctx->num_sms), threads, 0, st>>>(parent.as<int>(), N + M);
  if (E > 0)
    k_uf_union<<<grid_for(E, threads, ctx->num_sms), threads, 0, st>>>(E, N, cam, lmk, parent.as<int>());
  k_uf_check<<<grid_for(E + N, threads, ctx->num_sms), threads, 0, st>>>(E, N, cam, lmk, parent.as<int>(),
                                                                         flag.as<int>());
  XM_CUDA_TRY(cudaGetLastError());
  int h = 0;
  XM_CUDA_TRY(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  if (h) return set_error(XM_EDISCONNECTED, "view graph is not connected (N=%d, M=%d)", N, M);
  return XM_OK;
}

// Ascending observation indices within each of the K groups of idx (CSR offsets off): short
// groups by one thread each, the rest one block each (k_csr_sort_big).  Synchronous: its scratch
// (the queue of large groups and an E-entry copy buffer) is freed on return.
static xm_status csr_sort(xm_ctx* ctx, int K, int64_t E, const int64_t* off, int64_t* idx) {
  if (K <= 0 || E <= 0) return XM_OK;
  cudaStream_t st = ctx->stream;
  DevBuf big, nbig, tmp;
  XM_CUDA_TRY(cudaMalloc(&big.p, sizeof(int) * (size_t)K));
  XM_CUDA_TRY(cudaMalloc(&nbig.p, sizeof(int)));
  XM_CUDA_TRY(cudaMalloc(&tmp.p, sizeof(int64_t) * (size_t)E));
  XM_CUDA_TRY(cudaMemsetAsync(nbig.p, 0, sizeof(int), st));
  k_csr_sort<<<grid_for(K, 256, ctx->num_sms), 256, 0, st>>>(K, off, idx, big.as<int>(), nbig.as<int>());
  k_csr_sort_big<<<ctx->num_sms * 4, CSR_BIG_THREADS, 0, st>>>(off, idx, tmp.as<int64_t>(), big.as<int>(),
                                                              nbig.as<int>());
  XM_CUDA_TRY(cudaGetLastError());
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  return XM_OK;
}

xm_status build_Q(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                  const double* ukp, const double* w, unsigned mask, DeviceQ& out,
                  double* t_build) {
  auto tic = std::chrono::steady_clock::now();
  cudaStream_t st = ctx->stream;
  const int n = 3 * N;
  const int threads = 256;
  XM_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  if (E > 0) {
    k_validate<<<grid_for(E, threads, ctx->num_sms), threads, 0, st>>>(E, N, M, cam, lmk, ukp, w,
                                                                       ctx->d_err);
    XM_CUDA_TRY(cudaGetLastError());
  }
  XM_TRY(check_device_error(ctx, "observation validation"));

  // ---- connectivity (App. A lemma: rank N + M - 1 iff the view graph is connected)
  XM_TRY(check_connected(ctx, N, M, E, cam, lmk));

  // ---- the factored operator (XM_STORE_FACTORED), with or without dense copies
  if (mask & XM_STORE_FACTORED) {
    out.fact = new QFact();
    const xm_status sf = qfact_build(ctx, N, M, E, cam, lmk, ukp, w, *out.fact);
    if (sf != XM_OK) {
      qfact_release(*out.fact);
      delete out.fact;
      out.fact = nullptr;
      return sf;
    }
    if (!(mask & XM_STORE_ALL)) {     // no dense copy: Q itself is never formed
      XM_TRY(alloc_tiles(ctx, out, N, 0));
      out.mask = mask;
      if (t_build)
        *t_build = std::chrono::duration<double>(std::chrono::steady_clock::now() - tic).count();
      return XM_OK;
    }
  }

  DevBuf P, B, S, d, cnt, off, bsum, cursor, idx;
  XM_CUDA_TRY(cudaMalloc(&P.p, sizeof(double) * (size_t)n * n));
  XM_CUDA_TRY(cudaMalloc(&B.p, sizeof(double) * (size_t)n * N));
  XM_CUDA_TRY(cudaMalloc(&S.p, sizeof(double) * (size_t)N * N));
  XM_CUDA_TRY(cudaMalloc(&d.p, sizeof(double) * (size_t)(M > 0 ? M : 1)));
  XM_CUDA_TRY(cudaMalloc(&cnt.p, sizeof(int) * (size_t)(M > 0 ? M : 1)));
  XM_CUDA_TRY(cudaMemsetAsync(P.p, 0, sizeof(double) * (size_t)n * n, st));
  XM_CUDA_TRY(cudaMemsetAsync(B.p, 0, sizeof(double) * (size_t)n * N, st));
  XM_CUDA_TRY(cudaMemsetAsync(S.p, 0, sizeof(double) * (size_t)N * N, st));
  XM_CUDA_TRY(cudaMemsetAsync(d.p, 0, sizeof(double) * (size_t)(M > 0 ? M : 1), st));
  XM_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (size_t)(M > 0 ? M : 1), st));
  if (E > 0) {
    k_camera_terms<<<grid_for(E, threads, ctx->num_sms), threads, 0, st>>>(
        E, n, N, cam, lmk, ukp, w, P.as<double>(), B.as<double>(), S.as<double>(), d.as<double>(),
        cnt.as<int>());
    XM_CUDA_TRY(cudaGetLastError());
  }
  if (M > 0 && E > 0) {
    const int nb = (M + 1023) / 1024;
    XM_CUDA_TRY(cudaMalloc(&off.p, sizeof(int64_t) * (size_t)(M + 1)));
    XM_CUDA_TRY(cudaMalloc(&bsum.p, sizeof(int64_t) * (size_t)(nb + 1)));
    XM_CUDA_TRY(cudaMalloc(&cursor.p, sizeof(int) * (size_t)M));
    XM_CUDA_TRY(cudaMalloc(&idx.p, sizeof(int64_t) * (size_t)E));
    XM_CUDA_TRY(cudaMemsetAsync(cursor.p, 0, sizeof(int) * (size_t)M, st));
    k_scan_blocks<<<nb, 1024, 0, st>>>(cnt.as<int>(), off.as<int64_t>(), bsum.as<int64_t>(), M);
    k_scan_sums<<<1, 32, 0, st>>>(bsum.as<int64_t>(), nb);
    k_scan_add<<<nb, 1024, 0, st>>>(off.as<int64_t>(), bsum.as<int64_t>(), M);
    k_csr_fill<<<grid_for(E, threads, ctx->num_sms), threads, 0, st>>>(
        E, lmk, off.as<int64_t>(), cursor.as<int>(), idx.as<int64_t>());
    XM_TRY(csr_sort(ctx, M, E, off.as<int64_t>(), idx.as<int64_t>()));
    k_landmark_schur<<<grid_for(M, 128, ctx->num_sms), 128, 0, st>>>(
        M, n, N, off.as<int64_t>(), idx.as<int64_t>(), cam, ukp, w, d.as<double>(),
        P.as<double>(), B.as<double>(), S.as<double>());
    XM_CUDA_TRY(cudaGetLastError());
  }

  // ---- translation elimination (dense FP64, own kernels: no vendor library on this path)
  if (N > 1) {
    const int m = N - 1;
    // rows/cols 1..N-1 of S, ld N: the row-major upper triangle is the column-major lower one
    double* Sbar = S.as<double>() + N + 1;
    double* BbarT = B.as<double>() + 1;          // column-major (N-1) x n, ld N
    bool split = false;
    if (ctx->build_mode == XM_BUILD_SPLIT_BF16) {
      if (!split_update_fits(m, n))
        return set_error(XM_EINVAL, "split-BF16 build: N - 1 = %d outside its range", m);
      split = true;
    } else if (ctx->build_mode == XM_BUILD_AUTO) {
      split = N >= XM_BUILD_SPLIT_MIN_N && split_update_fits(m, n);
    }
    // Cholesky factor, C = L^{-1} Bbar^T and Q = P - C^T C, timed together (device events)
    cudaEvent_t e0, e1;
    XM_CUDA_TRY(cudaEventCreate(&e0));
    XM_CUDA_TRY(cudaEventCreate(&e1));
    XM_CUDA_TRY(cudaEventRecord(e0, st));
    int hinfo = 0;
    DevBuf fail;
    XM_CUDA_TRY(cudaMalloc(&fail.p, sizeof(int)));
    XM_CUDA_TRY(cudaMemsetAsync(fail.p, 0, sizeof(int), st));
    if (split) {
      XM_TRY(split_potrf(ctx, Sbar, N, m, &hinfo));
    } else {
      XM_TRY(dense_potrf(ctx, Sbar, N, m, fail.as<int>(), &hinfo));
    }
    if (hinfo != 0) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return set_error(XM_EDISCONNECTED,
                       "translation Schur block not positive definite (leading minor %d)", hinfo);
    }
    xm_status stu = XM_OK;
    if (split) {
      // both on the tensor cores; the rank-k update writes the packed tiles itself
      stu = split_trsm(ctx, Sbar, N, BbarT, N, m, n);
      if (stu == XM_OK) stu = alloc_tiles(ctx, out, N, mask);
      DevBuf acc;
      double* acc64 = out.q64;
      if (stu == XM_OK && !acc64) {
        if (cudaMalloc(&acc.p, sizeof(double) * (size_t)out.ntiles * TILE * TILE) != cudaSuccess) {
          (void)cudaGetLastError();
          stu = set_error(XM_ENOMEM, "split-BF16 build: FP64 tile scratch");
        }
        acc64 = acc.as<double>();
      }
      if (stu == XM_OK) stu = split_update_pack(ctx, BbarT, N, m, P.as<double>(), out, acc64);
      out.build_path = XM_BUILD_SPLIT_BF16;
    } else {
      // C = L^{-1} Bbar^T (blocked substitution), then P -= C^T C on the lower triangle of the
      // column-major P (its row-major upper triangle, which the packing reads)
      stu = dense_trsm_left_lower(ctx, Sbar, N, BbarT, N, m, n, nullptr);
      if (stu == XM_OK)
        stu = dense_gemm(ctx, true, false, true, n, n, m, -1.0, BbarT, N, BbarT, N, 1.0, P.as<double>(), n,
                         nullptr);
      if (stu == XM_OK) stu = alloc_tiles(ctx, out, N, mask);
      if (stu == XM_OK) stu = pack_dense(ctx, out, P.as<double>());
      out.build_path = XM_BUILD_FP64;
    }
    float ms = 0.f;
    if (stu == XM_OK && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess)
      cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    XM_TRY(stu);
    out.t_update_s = ms * 1e-3;
  } else {
    XM_TRY(alloc_tiles(ctx, out, N, mask));
    XM_TRY(pack_dense(ctx, out, P.as<double>()));
  }

  XM_CUDA_TRY(cudaStreamSynchronize(st));
  XM_TRY(check_device_error(ctx, "Q construction"));
  if (t_build)
    *t_build = std::chrono::duration<double>(std::chrono::steady_clock::now() - tic).count();
  return XM_OK;
}

}  // namespace xm

// ------------------------------------------------------------------ adjoint support
namespace xm {

// Index and value checks of the observation arrays (DEV_BAD_INDEX / DEV_BAD_VALUE).
xm_status validate_obs(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                       const double* ukp, const double* w) {
  cudaStream_t st = ctx->stream;
  XM_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), st));
  if (E > 0) {
    k_validate<<<grid_for(E, 256, ctx->num_sms), 256, 0, st>>>(E, N, M, cam, lmk, ukp, w, ctx->d_err);
    XM_CUDA_TRY(cudaGetLastError());
  }
  return check_device_error(ctx, "observation validation");
}

__global__ void k_count_keys(int64_t E, const int32_t* key, int* cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[key[e]], 1);
}

// Observations grouped by key (landmark or camera): off (K+1) and idx (E), both allocated by the
// caller; within a group the observation indices are ascending, so that every per-group sum
// taken in idx order is deterministic.
xm_status obs_csr(xm_ctx* ctx, int64_t E, const int32_t* key, int K, int64_t* off, int64_t* idx) {
  cudaStream_t st = ctx->stream;
  const int threads = 256;
  if (K <= 0) return XM_OK;
  if (E <= 0) {
    XM_CUDA_TRY(cudaMemsetAsync(off, 0, sizeof(int64_t) * (size_t)(K + 1), st));
    return XM_OK;
  }
  DevBuf cnt, bsum, cursor;
  const int nb = (K + 1023) / 1024;
  XM_CUDA_TRY(cudaMalloc(&cnt.p, sizeof(int) * (size_t)K));
  XM_CUDA_TRY(cudaMalloc(&bsum.p, sizeof(int64_t) * (size_t)(nb + 1)));
  XM_CUDA_TRY(cudaMalloc(&cursor.p, sizeof(int) * (size_t)K));
  XM_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (size_t)K, st));
  XM_CUDA_TRY(cudaMemsetAsync(cursor.p, 0, sizeof(int) * (size_t)K, st));
  k_count_keys<<<grid_for(E, threads, ctx->num_sms), threads, 0, st>>>(E, key, cnt.as<int>());
  k_scan_blocks<<<nb, 1024, 0, st>>>(cnt.as<int>(), off, bsum.as<int64_t>(), K);
  k_scan_sums<<<1, 32, 0, st>>>(bsum.as<int64_t>(), nb);
  k_scan_add<<<nb, 1024, 0, st>>>(off, bsum.as<int64_t>(), K);
  k_csr_fill<<<grid_for(E, threads, ctx->num_sms), threads, 0, st>>>(E, key, off, cursor.as<int>(), idx);
  XM_TRY(csr_sort(ctx, K, E, off, idx));
  XM_CUDA_TRY(cudaGetLastError());
  XM_CUDA_TRY(cudaStreamSynchronize(st));   // the scratch above is freed on return
  return XM_OK;
}

// d_k = sum of the weights of landmark k; S (row-major upper triangle) gets the camera
// diagonal sum_e w_e, one thread per camera group so that the sums are deterministic
__global__ void k_S_diag(int N, int M, const int64_t* coff, const int64_t* cidx,
                         const int64_t* loff, const int64_t* lidx, const double* w, double* S,
                         double* d) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = tid; j < N; j += stride) {
    double s = 0.0;
    for (int64_t x = coff[j]; x < coff[j + 1]; ++x) s += w[cidx[x]];
    S[(size_t)j * N + j] = s;
  }
  for (int64_t k = tid; k < M; k += stride) {
    double s = 0.0;
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) s += w[lidx[x]];
    d[k] = s;
  }
}

// S_ij -= w_a w_b / d_k over the ordered observer pairs (a, b) of every landmark k with
// cam_a <= cam_b (row-major upper triangle == column-major lower triangle)
__global__ void k_landmark_S(int M, int N, const int64_t* off, const int64_t* idx,
                             const int32_t* cam, const double* w, const double* d, double* S) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    const int64_t a0 = off[k], a1 = off[k + 1];
    if (a1 <= a0 || !(d[k] > 0.0)) continue;
    const double dinv = 1.0 / d[k];
    for (int64_t x = a0; x < a1; ++x) {
      const int i = cam[idx[x]];
      const double wa = w[idx[x]] * dinv;
      for (int64_t y = a0; y < a1; ++y) {
        const int j = cam[idx[y]];
        if (i <= j) atomicAdd(&S[(size_t)i * N + j], -wa * w[idx[y]]);
      }
    }
  }
}

// b (N x c column-major) <- -b
__global__ void k_negate_cols(int N, int c, double* b) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * c; e += gridDim.x * blockDim.x) b[e] = -b[e];
}

// The camera block S = diag(sum w) - sum_k (w w^T)/d_k that remains after the landmarks are
// eliminated (App. A), and the Cholesky factor of Sbar (camera 0 anchored, t_0 = 0).  S (N x N)
// and d (M) are allocated by the caller; on return the column-major lower triangle of rows and
// columns 1..N-1 of S (leading dimension N) holds the factor.
xm_status schur_S_factor(xm_ctx* ctx, int N, int M, const int32_t* cam, const double* w,
                         const int64_t* coff, const int64_t* cidx, const int64_t* loff,
                         const int64_t* lidx, double* S, double* d) {
  cudaStream_t st = ctx->stream;
  XM_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(double) * (size_t)N * N, st));
  const int g = grid_for(std::max(N, M), 128, ctx->num_sms);
  k_S_diag<<<g, 128, 0, st>>>(N, M, coff, cidx, loff, lidx, w, S, d);
  if (M > 0)
    k_landmark_S<<<grid_for(M, 128, ctx->num_sms), 128, 0, st>>>(M, N, loff, lidx, cam, w, d, S);
  XM_CUDA_TRY(cudaGetLastError());
  if (N > 1) {
    // Cholesky factor of Sbar: tensor-core trailing updates from XM_BUILD_SPLIT_MIN_N rows (the
    // build's own factorisation), the FP64 blocked factor below
    const int m = N - 1;
    double* Sbar = S + N + 1;
    int hinfo = 0;
    if (m >= XM_BUILD_SPLIT_MIN_N) {
      XM_TRY(split_potrf(ctx, Sbar, N, m, &hinfo));
    } else {
      DevBuf fail;
      XM_CUDA_TRY(cudaMalloc(&fail.p, sizeof(int)));
      XM_CUDA_TRY(cudaMemsetAsync(fail.p, 0, sizeof(int), st));
      XM_TRY(dense_potrf(ctx, Sbar, N, m, fail.as<int>(), &hinfo));
    }
    if (hinfo != 0)
      return set_error(XM_EDISCONNECTED, "translation Schur block not positive definite (minor %d)", hinfo);
  }
  return XM_OK;
}

// b (N x c, column-major, leading dimension N) <- t with Sbar tbar = -bbar and t_0 = 0, using
// the factor left in S by schur_S_factor.
xm_status schur_S_solve(xm_ctx* ctx, int N, const double* S, double* b, int c) {
  cudaStream_t st = ctx->stream;
  if (N > 1 && c > 0) {
    const double* Sbar = S + N + 1;
    // tbar = -Sbar^{-1} bbar = -L^{-T} L^{-1} bbar
    XM_TRY(dense_trsm_left_lower(ctx, Sbar, N, b + 1, N, N - 1, c, nullptr));
    XM_TRY(dense_trsm_left_lower_t(ctx, Sbar, N, b + 1, N, N - 1, c, nullptr));
    k_negate_cols<<<std::max(1, std::min(c * N / 256 + 1, 1024)), 256, 0, st>>>(N, c, b);
    XM_CUDA_TRY(cudaGetLastError());
  }
  if (c > 0) XM_CUDA_TRY(cudaMemset2DAsync(b, sizeof(double) * N, 0, sizeof(double), c, st));
  return XM_OK;
}

}  // namespace xm
