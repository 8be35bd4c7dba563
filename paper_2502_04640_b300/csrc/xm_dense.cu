// FP64 dense kernels of the translation elimination (App. A: the Cholesky factor of the anchored
// camera block, triangular solves with it, and the symmetric product that forms Q), written for
// this library so that building Q loads no vendor linear-algebra library.
//
//   k_trsv_units  forward substitution L x = a (L lower, non-unit diagonal) for many right-hand
//                 sides ("units") at once: unit u's k-th entry lives at X[u su + k sk].  One warp
//                 owns UPW units held in shared memory and walks the columns of L (column-oriented:
//                 x_j = a_j / L_jj, then a_i -= L_ij x_j for i > j), so every step reads one
//                 contiguous column of L and shares it between its units.  Covers X L^T = A (units
//                 = rows of A) and L X = B (units = columns of B).
//   k_potf_small  Cholesky factor of a block of at most 64 rows in one CTA (shared memory), with
//                 the first failing leading minor reported.
//   k_dgemm       C = alpha op(A) op(B) + beta C, column-major, 64 x 64 tiles, optionally only the
//                 tiles that meet the lower triangle.
// Host drivers: dense_potrf (right-looking, 64-column panels), dense_trsm_right_lower_t (panels of
// the blocked Cholesky), dense_trsm_left_lower (blocked, 256-row steps), dense_gemm.
#include <algorithm>
#include <mutex>

#include "xm_internal.cuh"

namespace xm {

constexpr int TRSV_UPW = 4;          // units per warp
constexpr int TRSV_WARPS = 8;        // warps per CTA
constexpr int TRSV_MAX_B = 512;      // largest system one launch solves (shared memory)
constexpr int POTF_NB = 64;          // panel width of dense_potrf
constexpr int TRSM_NB = 256;         // row block of dense_trsm_left_lower

template <int UPW>
__global__ void __launch_bounds__(32 * TRSV_WARPS)
k_trsv_units(int nunits, int b, const double* __restrict__ L, int ldl, double* __restrict__ X,
             int64_t su, int64_t sk, const int* __restrict__ fail) {
  extern __shared__ double trsv_sm[];
  if (fail && *fail) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* xs = trsv_sm + (size_t)warp * UPW * b;
  const int u0 = (blockIdx.x * TRSV_WARPS + warp) * UPW;
  if (u0 >= nunits) return;
  const int nu = min(UPW, nunits - u0);
  for (int u = 0; u < nu; ++u)
    for (int k = lane; k < b; k += 32) xs[u * b + k] = X[(int64_t)(u0 + u) * su + (int64_t)k * sk];
  __syncwarp();
  for (int j = 0; j < b; ++j) {
    const double* Lj = L + (size_t)j * ldl;
    const double inv = 1.0 / Lj[j];
    double xj[UPW];
#pragma unroll
    for (int u = 0; u < UPW; ++u) xj[u] = u < nu ? xs[u * b + j] * inv : 0.0;
    for (int i = j + 1 + lane; i < b; i += 32) {
      const double l = Lj[i];
#pragma unroll
      for (int u = 0; u < UPW; ++u)
        if (u < nu) xs[u * b + i] -= l * xj[u];
    }
    __syncwarp();
    if (lane == 0)
#pragma unroll
      for (int u = 0; u < UPW; ++u)
        if (u < nu) xs[u * b + j] = xj[u];
  }
  __syncwarp();
  for (int u = 0; u < nu; ++u)
    for (int k = lane; k < b; k += 32) X[(int64_t)(u0 + u) * su + (int64_t)k * sk] = xs[u * b + k];
}

// Backward substitution with the transpose, L^T x = y (L lower, non-unit diagonal), one warp per
// unit (few right-hand sides): x_j = (y_j - sum_{l > j} L_lj x_l) / L_jj for j = b-1 .. 0, the sum
// over the contiguous column j of L below its diagonal, reduced across the warp.
__global__ void __launch_bounds__(32 * TRSV_WARPS)
k_trsv_t_units(int nunits, int b, const double* __restrict__ L, int ldl, double* __restrict__ X,
               int64_t su, int64_t sk, const int* __restrict__ fail) {
  extern __shared__ double trsv_sm[];
  if (fail && *fail) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int u = blockIdx.x * TRSV_WARPS + warp;
  if (u >= nunits) return;
  double* xs = trsv_sm + (size_t)warp * b;
  for (int k = lane; k < b; k += 32) xs[k] = X[(int64_t)u * su + (int64_t)k * sk];
  __syncwarp();
  for (int j = b - 1; j >= 0; --j) {
    const double* Lj = L + (size_t)j * ldl;
    double acc = 0.0;
    for (int l = j + 1 + lane; l < b; l += 32) acc += Lj[l] * xs[l];
    acc = warp_sum(acc);
    const double xj = (xs[j] - acc) / Lj[j];
    __syncwarp();
    if (lane == 0) xs[j] = xj;
    __syncwarp();
  }
  for (int k = lane; k < b; k += 32) X[(int64_t)u * su + (int64_t)k * sk] = xs[k];
}

// Cholesky factor (lower, in place) of the nb x nb block at A (column-major, ld lda), nb <= 64.
// On a non-positive or non-finite pivot *fail = base + j + 1 (the failing leading minor of the
// whole matrix) and the block is left as it is.
__global__ void __launch_bounds__(256) k_potf_small(double* __restrict__ A, int lda, int nb, int base,
                                                    int* __restrict__ fail) {
  __shared__ double s[POTF_NB][POTF_NB + 1];
  __shared__ int bad;
  if (*fail) return;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, k = e / nb;
    s[i][k] = A[i + (size_t)k * lda];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = s[j][j];
      if (!(d > 0.0) || !isfinite(d)) bad = j + 1;
      else s[j][j] = sqrt(d);
    }
    __syncthreads();
    if (bad) break;
    const double ljj = s[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) s[i][j] /= ljj;
    __syncthreads();
    // trailing update of the lower triangle: s[i][k] -= s[i][j] s[k][j], j < k <= i
    const int rem = nb - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e % rem, k = j + 1 + e / rem;
      if (k <= i) s[i][k] -= s[i][j] * s[k][j];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicCAS(fail, 0, base + bad);
    return;
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, k = e / nb;
    if (k <= i) A[i + (size_t)k * lda] = s[i][k];
  }
}

// C (m x n) = alpha op(A) op(B) + beta C, all column-major.  op(A) is m x k (A, or A^T when TA);
// op(B) is k x n.  256 threads compute a 64 x 64 tile, each a 4 x 4 set of entries strided by
// 16 (conflict-free shared-memory reads).  LOWER: only tiles with a row >= some column.
constexpr int GM_T = 64, GM_K = 16;
template <bool TA, bool TB, bool LOWER>
__global__ void __launch_bounds__(256)
k_dgemm(int m, int n, int k, double alpha, const double* __restrict__ A, int lda,
        const double* __restrict__ B, int ldb, double beta, double* __restrict__ C, int ldc,
        const int* __restrict__ fail) {
  __shared__ double As[GM_K][GM_T + 1];
  __shared__ double Bs[GM_K][GM_T + 1];
  if (fail && *fail) return;
  const int i0 = blockIdx.x * GM_T, j0 = blockIdx.y * GM_T;
  if (LOWER && j0 > i0 + GM_T - 1) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
  for (int k0 = 0; k0 < k; k0 += GM_K) {
    // op(A)[i0 + r][k0 + c] -> As[c][r]; op(B)[k0 + c][j0 + r] -> Bs[c][r]
    for (int e = threadIdx.x; e < GM_T * GM_K; e += 256) {
      int r, c;
      if (!TA) { r = e % GM_T; c = e / GM_T; } else { c = e % GM_K; r = e / GM_K; }
      const int gi = i0 + r, gk = k0 + c;
      double v = 0.0;
      if (gi < m && gk < k) v = TA ? A[gk + (size_t)gi * lda] : A[gi + (size_t)gk * lda];
      As[c][r] = v;
    }
    for (int e = threadIdx.x; e < GM_T * GM_K; e += 256) {
      int r, c;
      if (TB) { r = e % GM_T; c = e / GM_T; } else { c = e % GM_K; r = e / GM_K; }
      const int gj = j0 + r, gk = k0 + c;
      double v = 0.0;
      if (gj < n && gk < k) v = TB ? B[gj + (size_t)gk * ldb] : B[gk + (size_t)gj * ldb];
      Bs[c][r] = v;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < GM_K; ++c) {
      double a[4], bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[c][ty + 16 * q]; bv[q] = Bs[c][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], bv[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gi = i0 + ty + 16 * p, gj = j0 + tx + 16 * q;
      if (gi < m && gj < n && (!LOWER || gj <= gi)) {
        double* c = C + gi + (size_t)gj * ldc;
        *c = beta == 0.0 ? alpha * acc[p][q] : fma(alpha, acc[p][q], beta * *c);
      }
    }
}

// ------------------------------------------------------------------ host drivers
xm_status dense_gemm(xm_ctx* ctx, bool ta, bool tb, bool lower, int m, int n, int k, double alpha,
                     const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                     const int* fail) {
  if (m <= 0 || n <= 0) return XM_OK;
  const dim3 grid((m + GM_T - 1) / GM_T, (n + GM_T - 1) / GM_T);
  cudaStream_t st = ctx->stream;
#define XM_GEMM_CASE(TA_, TB_, LO_)                                                                  \
  if (ta == TA_ && tb == TB_ && lower == LO_)                                                        \
    k_dgemm<TA_, TB_, LO_><<<grid, 256, 0, st>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, fail);
  XM_GEMM_CASE(false, false, false)
  XM_GEMM_CASE(false, true, false)
  XM_GEMM_CASE(true, false, false)
  XM_GEMM_CASE(false, true, true)
  XM_GEMM_CASE(true, false, true)
#undef XM_GEMM_CASE
  if ((ta && tb) || (lower && ta == tb))
    return set_error(XM_EINVAL, "dense_gemm: unsupported operand form");
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

// the substitution kernels' shared-memory opt-in, once per device
static xm_status trsv_configure(xm_ctx* ctx) {
  constexpr int MAX_DEVICES = 64;
  static std::mutex mu;
  static bool configured[MAX_DEVICES] = {};
  if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
    return set_error(XM_EINVAL, "triangular solve: device %d out of range", ctx->device);
  std::lock_guard<std::mutex> lock(mu);
  if (!configured[ctx->device]) {
    XM_CUDA_TRY(cudaFuncSetAttribute(k_trsv_units<TRSV_UPW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(double) * TRSV_WARPS * TRSV_UPW * TRSV_MAX_B)));
    configured[ctx->device] = true;
  }
  return XM_OK;
}

static xm_status trsv_units(xm_ctx* ctx, int nunits, int b, const double* L, int ldl, double* X,
                            int64_t su, int64_t sk, const int* fail) {
  if (nunits <= 0 || b <= 0) return XM_OK;
  if (b > TRSV_MAX_B) return set_error(XM_EINVAL, "triangular solve: block %d above %d", b, TRSV_MAX_B);
  XM_TRY(trsv_configure(ctx));
  const size_t smem = sizeof(double) * (size_t)TRSV_WARPS * TRSV_UPW * b;
  const int per_cta = TRSV_WARPS * TRSV_UPW;
  k_trsv_units<TRSV_UPW><<<(nunits + per_cta - 1) / per_cta, 32 * TRSV_WARPS, smem, ctx->stream>>>(
      nunits, b, L, ldl, X, su, sk, fail);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

// X <- L^{-T} X for X column-major m x n (ld ldx, few columns), L lower m x m (ld ldl): 256-row
// steps from the bottom, each a backward substitution on its diagonal block and a product update
// of the rows above it.
xm_status dense_trsm_left_lower_t(xm_ctx* ctx, const double* L, int ldl, double* X, int ldx, int m, int n,
                                  const int* fail) {
  const int nblk = (m + TRSM_NB - 1) / TRSM_NB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int j0 = bi * TRSM_NB, bj = std::min(TRSM_NB, m - j0);
    const double* Ljj = L + j0 + (size_t)j0 * ldl;
    const size_t smem = sizeof(double) * (size_t)TRSV_WARPS * bj;
    k_trsv_t_units<<<(n + TRSV_WARPS - 1) / TRSV_WARPS, 32 * TRSV_WARPS, smem, ctx->stream>>>(
        n, bj, Ljj, ldl, X + j0, ldx, 1, fail);
    XM_CUDA_TRY(cudaGetLastError());
    if (j0 > 0)   // X[0:j0] -= L[j0:j0+bj, 0:j0]^T X[j0:j0+bj]
      XM_TRY(dense_gemm(ctx, true, false, false, j0, n, bj, -1.0, L + j0, ldl, X + j0, ldx, 1.0, X, ldx,
                        fail));
  }
  return XM_OK;
}

// A <- A L^{-T} for A column-major rows x b (ld lda), L lower b x b (ld ldl), b <= 512: every row
// of A is a unit of L x = a.
xm_status dense_trsm_right_lower_t(xm_ctx* ctx, const double* L, int ldl, double* A, int lda, int rows,
                                   int b, const int* fail) {
  return trsv_units(ctx, rows, b, L, ldl, A, 1, lda, fail);
}

// X <- L^{-1} X for X column-major m x n (ld ldx), L lower m x m (ld ldl): 256-row steps, each a
// substitution on its diagonal block (units = the n columns) and a product update of the rows
// below it.
xm_status dense_trsm_left_lower(xm_ctx* ctx, const double* L, int ldl, double* X, int ldx, int m, int n,
                                const int* fail) {
  for (int j0 = 0; j0 < m; j0 += TRSM_NB) {
    const int bj = std::min(TRSM_NB, m - j0);
    const double* Ljj = L + j0 + (size_t)j0 * ldl;
    XM_TRY(trsv_units(ctx, n, bj, Ljj, ldl, X + j0, ldx, 1, fail));
    const int rest = m - j0 - bj;
    if (rest > 0)
      XM_TRY(dense_gemm(ctx, false, false, false, rest, n, bj, -1.0, L + j0 + bj + (size_t)j0 * ldl, ldl,
                        X + j0, ldx, 1.0, X + j0 + bj, ldx, fail));
  }
  return XM_OK;
}

// In-place Cholesky factor (lower) of the SPD m x m A (column-major, ld lda): 64-column panels,
// each factored in one CTA, its rows below solved by substitution and the trailing lower
// triangle updated by a product.  *minor = first failing leading minor (0: success).
// fail_dev: a device int the caller zeroed (shared by the launches, so work after a failure is
// skipped).  Synchronous (reads the result back).
xm_status dense_potrf(xm_ctx* ctx, double* A, int lda, int m, int* fail_dev, int* minor) {
  cudaStream_t st = ctx->stream;
  for (int k0 = 0; k0 < m; k0 += POTF_NB) {
    const int bk = std::min(POTF_NB, m - k0);
    double* Akk = A + k0 + (size_t)k0 * lda;
    k_potf_small<<<1, 256, 0, st>>>(Akk, lda, bk, k0, fail_dev);
    XM_CUDA_TRY(cudaGetLastError());
    const int rest = m - k0 - bk;
    if (rest == 0) break;
    double* P = Akk + bk;
    XM_TRY(dense_trsm_right_lower_t(ctx, Akk, lda, P, lda, rest, bk, fail_dev));
    XM_TRY(dense_gemm(ctx, false, true, true, rest, rest, bk, -1.0, P, lda, P, lda, 1.0,
                      P + (size_t)bk * lda, lda, fail_dev));
  }
  int h = 0;
  XM_CUDA_TRY(cudaMemcpyAsync(&h, fail_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  *minor = h;
  return XM_OK;
}

}  // namespace xm
