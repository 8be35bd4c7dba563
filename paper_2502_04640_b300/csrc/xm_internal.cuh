// Internal declarations shared by the libxm translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/xm.h"

namespace xm {

// ------------------------------------------------------------------ errors (host side)
xm_status set_error(xm_status st, const char* fmt, ...);
// On failure the runtime's last-error slot is read and cleared as well, so that a non-sticky
// error reported here is not picked up again by the next, unrelated cudaGetLastError().
#define XM_CUDA_TRY(...)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (__VA_ARGS__);                                                        \
    if (e_ != cudaSuccess) {                                                               \
      (void)cudaGetLastError();                                                            \
      return ::xm::set_error(e_ == cudaErrorMemoryAllocation ? XM_ENOMEM : XM_ECUDA,       \
                             "%s failed: %s (%s:%d)", #__VA_ARGS__, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                          \
    }                                                                                      \
  } while (0)
#define XM_TRY(...)                                                                        \
  do {                                                                                     \
    xm_status s_ = (__VA_ARGS__);                                                          \
    if (s_ != XM_OK) return s_;                                                            \
  } while (0)

// Device error word values (ctx->d_err); host maps them to xm_status.
enum DevErr : int {
  DEV_OK = 0,
  DEV_TIMEOUT = 1,        // bounded mbarrier / flag wait gave up
  DEV_BAD_INDEX = 2,      // observation index out of range
  DEV_BAD_VALUE = 4,      // w <= 0 or non-finite input
  DEV_NUMERIC = 8,        // NaN / Inf produced
};

// ------------------------------------------------------------------ Q storage
// Packed symmetric layout: n is padded to n_pad = nt * TILE; the upper-triangle tiles (I <= J)
// are stored one after another in row-major tile order, each tile a contiguous TILE x TILE
// row-major block.  Off-diagonal tile (I, J) holds Q[I*T + a][J*T + b]; a diagonal tile holds
// the upper triangle of its block with the diagonal halved and zeros below, so that every
// tile T contributes T Y_J to W_I and T^T Y_I to W_J (the diagonal block is T + T^T).
constexpr int TILE = 128;
constexpr int XM_BUILD_SPLIT_MIN_N = 512;   // XM_BUILD_AUTO: tensor-core update from this N
constexpr int SLAB_BYTES = 16384;   // unit of one bulk async copy

__host__ __device__ inline int64_t tile_count(int nt) { return (int64_t)nt * (nt + 1) / 2; }
// Element offset of entry (a, b) of a packed 128 x 128 BF16 tile, stored in the tensor cores'
// operand layout: two 64-column halves of 16 KB, rows of 128 bytes, the 16-byte chunks of each
// row permuted by the 128-byte swizzle (chunk c of row a at position c xor (a mod 8)).  One
// contiguous bulk copy then lands a tile in shared memory ready for tcgen05.mma.
__host__ __device__ inline int bf16_tile_off(int a, int b) {
  return (b >> 6) * (128 * 64) + a * 64 + ((((b & 63) >> 3) ^ (a & 7)) << 3) + (b & 7);
}
__host__ __device__ inline int64_t tile_index(int nt, int I, int J) {
  return (int64_t)I * nt - (int64_t)I * (I - 1) / 2 + (J - I);
}

struct QFact;

struct DeviceQ {
  int N = 0, n = 0, n_pad = 0, nt = 0;
  int64_t ntiles = 0;
  unsigned mask = 0;
  double* q64 = nullptr;            // packed FP64 tiles
  float* q32 = nullptr;             // packed FP32 tiles
  __nv_bfloat16* q16 = nullptr;     // packed BF16 tiles
  __nv_bfloat16* ydig = nullptr;    // with q16: the tensor-core sweep's BF16 digit rows of Y
                                    // (32 x n_pad; one sweep of this Q at a time)
  int build_path = 0;               // XM_BUILD_* of the rank-(N-1) update that built it
  double t_update_s = 0.0;          // device time of that update (digit split + tensor cores)
  QFact* fact = nullptr;            // factored operator (XM_STORE_FACTORED): FP64 products
                                    // when there is no FP64 tile copy
};

// Factored Q operator (xm_factored.cu): observations in landmark- and camera-major order, the
// landmark weight sums and the packed FP64 tiles of -Sbar^{-1}.
struct QFact {
  int N = 0, M = 0;
  int64_t E = 0;
  int64_t *loff = nullptr, *coff = nullptr;        // landmark / camera CSR offsets (M+1, N+1)
  double *lu = nullptr, *lw = nullptr;             // landmark-major u (E x 3) and w (E)
  int32_t* lc = nullptr;                           // camera of each landmark-major observation
  double *cu = nullptr, *cw = nullptr;             // camera-major u (E x 3) and w (E)
  int32_t* cl = nullptr;                           // landmark of each camera-major observation
  double* dinv = nullptr;                          // 1 / d_k (0 for a landmark without observations)
  DeviceQ sinv;                                    // packed tiles of -Sbar^{-1} (n = N - 1), FP64
  double *mk = nullptr, *tbk = nullptr;            // landmark means (M x 8)
  double *bb = nullptr, *tt = nullptr;             // sweep input / output (sinv.n_pad x 8)
  size_t bytes = 0;
  double t_setup_s = 0.0;
};
xm_status qfact_build(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                      const double* ukp, const double* w, QFact& f);
void qfact_release(QFact& f);
// W += Q Y (FP64; first r columns of rows of ld doubles; skip as for qy_launch)
xm_status qfact_apply(xm_ctx* ctx, const QFact& f, int r, int ld, const double* Y, double* W,
                      const int* skip, cudaStream_t st);

}  // namespace xm

struct xm_qmat {
  xm::DeviceQ d;
  double t_build_s = 0.0;
};

struct xm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  size_t smem_optin = 0;
  int* d_err = nullptr;           // device error word
  int* h_err = nullptr;           // pinned mirror
  // reduction scratch: per-block partials and a completion counter
  double* d_partials = nullptr;
  size_t partials_cap = 0;        // doubles
  unsigned* d_counter = nullptr;
  int build_mode = 0;             // XM_BUILD_* for xm_build_Q's dense update
};

namespace xm {

xm_status check_device_error(xm_ctx* ctx, const char* where);
extern long g_last_launches;   // kernel launches of the last solve / certify call
extern long g_last_sweeps;
xm_status ensure_partials(xm_ctx* ctx, size_t ndoubles);

// ------------------------------------------------------------------ sweep (xm_qy.cu)
// W = Q Y (n_pad x R, row-major, zero-initialised by the caller: the kernel accumulates).
// skip: optional device flag; when non-zero the launch does nothing (early-exit of loops).
// packed tiles (alloc_tiles/free_tiles in the build); pack_dense_f32 packs the lower triangle of
// a column-major n x n FP32 symmetric matrix into the copies q's mask holds
xm_status alloc_tiles(xm_ctx* ctx, DeviceQ& q, int N, unsigned mask);
void free_tiles(DeviceQ& q);
xm_status pack_dense_f32(xm_ctx* ctx, DeviceQ& q, const float* A);
xm_status qy_launch(xm_ctx* ctx, const DeviceQ& q, int prec, int R, const void* Y, void* W,
                    const int* skip, cudaStream_t st);
// the BF16-stored Q's sweep on the tensor cores (xm_qy_tc.cu): FP32 Y (n_pad x R, R in
// {1, 4, 8}) in three BF16 digits, FP32 W accumulated
xm_status qy_tc_launch(xm_ctx* ctx, const DeviceQ& q, int R, const float* Y, float* W,
                       const int* skip, cudaStream_t st);

// ------------------------------------------------------------------ split-BF16 update (xm_ozaki.cu)
// Whether the tensor-core rank-K update handles K = N - 1 and n = 3N.
bool split_update_fits(int K, int n);
// Packed tiles of Q = P - C^T C (C column-major K x n, leading dimension ldc; P row-major n x n,
// upper triangle) written into q's copies; acc64 is q.q64 or an FP64 tile scratch of that size.
xm_status split_update_pack(xm_ctx* ctx, const double* C, int ldc, int K, const double* P,
                            DeviceQ& q, double* acc64);
// X <- L^{-1} X (L lower triangular m x m, X m x n, both column-major): blocked forward
// substitution with FP64-formed diagonal-block inverses and tensor-core block updates.
xm_status split_trsm(xm_ctx* ctx, const double* L, int ldl, double* X, int ldx, int m, int n);
// In-place Cholesky factor (lower) of the SPD m x m A (column-major): blocked, FP64 diagonal
// blocks and panels (dense_*), tensor-core trailing updates; *minor = first failing leading
// minor or 0.
xm_status split_potrf(xm_ctx* ctx, double* A, int lda, int m, int* minor);

// ------------------------------------------------------------------ SPD inverse (xm_spdinv.cu)
// In-place inverse of the SPD n x n FP32 matrix A (column-major, lda >= n, both triangles set):
// Schur-complement recursion with BF16-digit tensor-core products.  Synchronous; XM_ENUMERIC
// if A is not numerically positive definite (A then undefined).  *gflop (optional): the
// products' FP32-equivalent GFLOP.
xm_status spd_inverse_f32(xm_ctx* ctx, float* A, int lda, int n, double* gflop);
// ------------------------------------------------------------------ FP64 dense kernels (xm_dense.cu)
// All column-major.  fail: optional device flag; when non-zero the launches do nothing.
// C = alpha op(A) op(B) + beta C (op = transpose when ta / tb; lower: only C's lower triangle;
// supported: NN, NT, TN and the lower NT / TN forms).
xm_status dense_gemm(xm_ctx* ctx, bool ta, bool tb, bool lower, int m, int n, int k, double alpha,
                     const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                     const int* fail);
// In-place Cholesky factor (lower) of an SPD m x m A; fail_dev a zeroed device int; *minor =
// first failing leading minor (0: success).  Synchronous.
xm_status dense_potrf(xm_ctx* ctx, double* A, int lda, int m, int* fail_dev, int* minor);
// A <- A L^{-T} (A rows x b, L lower b x b, b <= 512).
xm_status dense_trsm_right_lower_t(xm_ctx* ctx, const double* L, int ldl, double* A, int lda, int rows,
                                   int b, const int* fail);
// X <- L^{-1} X and X <- L^{-T} X (X m x n, L lower m x m).
xm_status dense_trsm_left_lower(xm_ctx* ctx, const double* L, int ldl, double* X, int ldx, int m, int n,
                                const int* fail);
xm_status dense_trsm_left_lower_t(xm_ctx* ctx, const double* L, int ldl, double* X, int ldx, int m, int n,
                                  const int* fail);

// ------------------------------------------------------------------ adjoint support (xm_build.cu)
// Index and value checks of the observation arrays (synchronous; XM_EINVAL on a bad entry).
xm_status validate_obs(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                       const double* ukp, const double* w);
// XM_EDISCONNECTED unless the camera-landmark view graph is connected (App. A lemma).
xm_status check_connected(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk);
// Observations grouped by key (ascending observation index within a group); off (K+1), idx (E)
// are allocated by the caller.
xm_status obs_csr(xm_ctx* ctx, int64_t E, const int32_t* key, int K, int64_t* off, int64_t* idx);
// Camera block S left after landmark elimination and the Cholesky factor of Sbar (camera 0
// anchored); S (N x N) and d (M, landmark weight sums) are allocated by the caller.
xm_status schur_S_factor(xm_ctx* ctx, int N, int M, const int32_t* cam, const double* w,
                         const int64_t* coff, const int64_t* cidx, const int64_t* loff,
                         const int64_t* lidx, double* S, double* d);
// b (N x c column-major) <- t with Sbar tbar = -bbar, t_0 = 0.
xm_status schur_S_solve(xm_ctx* ctx, int N, const double* S, double* b, int c);

// ------------------------------------------------------------------ device helpers
#ifdef __CUDACC__
constexpr long long WAIT_LIMIT = 1ll << 24;   // try_wait polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Bounded wait for the completion of the phase with the given parity.  Returns false after
// `limit` polls (WAIT_LIMIT unless a self-check passes a smaller one); the caller records
// DEV_TIMEOUT and stops waiting.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = WAIT_LIMIT) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk async copy global -> shared, completion signalled on an mbarrier (TMA engine).
// Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Entry (r, c) of Q from the packed tiles (upper-triangle tiles, halved diagonal).
template <typename TQ>
__device__ __forceinline__ double q_entry(const TQ* __restrict__ tiles, int nt, int r, int c) {
  if (r > c) { const int t = r; r = c; c = t; }
  const int I = r / TILE, J = c / TILE, a = r % TILE, b = c % TILE;
  const double v = double(tiles[tile_index(nt, I, J) * TILE * TILE + (int64_t)a * TILE + b]);
  return (I == J && a == b) ? 2.0 * v : v;
}

// Traversal order of the tiles: tile rows 0, nt-1, 1, nt-2, ... (a long row, then the short row
// that completes it to nt + 1 tiles), each row from its diagonal tile outwards.  Every CTA takes a
// contiguous range of this order, so each crosses one to three row boundaries (a row change costs
// a flush of the row partials and a Y_I reload), where row-major order left the CTA holding the
// last, shortest rows with a dozen or more.
__device__ __forceinline__ void pair_order_start(int nt, int64_t v, int& I, int& J) {
  const int64_t P = (int64_t)nt + 1;
  const int p = (int)(v / P), rem = (int)(v % P);
  if (rem < nt - p) { I = p; J = p + rem; }
  else { I = nt - 1 - p; J = I + (rem - (nt - p)); }
}
__device__ __forceinline__ void pair_order_next(int nt, int& I, int& J) {
  if (++J < nt) return;
  I = (2 * I < nt - 1) ? nt - 1 - I : nt - I;   // long row p -> short row nt-1-p -> long row p+1
  J = I;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
#endif

}  // namespace xm
