// The dense rank-(N-1) update of the Q build on the BF16 tensor cores (tcgen05), FP64-accurate.
//
// Translation elimination (App. A, Prop. 1) ends with Q = P - C^T C, C = L^{-1} Bbar^T an
// (N-1) x n matrix (L the Cholesky factor of the anchored translation block Sbar).  C^T C is
// the one truly dense contraction of the method: n = 30465, K = N - 1 = 10154 at 10155 cameras,
// 9.4 TFLOP in FP64, about 9 s at B300's FP64 rate.  It is computed here by the error-free
// splitting of Ozaki, Ogita, Oishi and Rump (2012) on the BF16 tensor cores:
//
//   * every column c of C is written as 2^{e_c} sum_{s<8} d_{s,c} 2^{-7(s+1)} with integer
//     digits |d| <= 127 (exact in BF16); the 8 digits hold every entry to within 2^{-56} of the
//     largest entry of its column;
//   * (C^T C)_{ij} = 2^{e_i+e_j} sum_{m<8} 2^{-7(m+2)} L_m(i,j), L_m = sum_{a+b=m} d_a,i . d_b,j,
//     dropping digit products of order m >= 8 (below 2^{-56} K max|c_i| max|c_j|): normwise as
//     accurate as an FP64 rank-k update;
//   * each level L_m is a BF16 GEMM over the concatenated K' = (m+1) K.  Its FP32 accumulation
//     in tensor memory is exact when at most 1024 products (each < 2^14) are summed, so the
//     accumulation restarts every 16 k-blocks of 64 and the epilogue adds each chunk, as an
//     integer, to int32 registers (|L_m| < 2^31 for K <= 16640);
//   * a finished level is scaled by an exact power of two and added in FP64 into the packed
//     FP64 tile; after the last level the tile gets P added and is written in the sweep's
//     packed layout (halved diagonal, zero lower triangle) in FP64, FP32 and BF16.
//
// Kernel: persistent, one CTA per SM, 128 x 128 output tiles of the upper triangle in a
// block-row order that lets concurrent CTAs share operand k-blocks in L2.  Warp 0 streams the
// two 128 x 64 BF16 operand boxes of each k-block with TMA (128-byte swizzle) into a 6-stage
// mbarrier ring; one thread of warp 1 issues tcgen05.mma (M = 128, N = 128, K = 16) into one of
// two TMEM accumulators; warps 2..9 read finished chunks with tcgen05.ld (two warps per TMEM lane
// quarter, 64 columns each) while the next chunk accumulates in the other buffer.  Every wait is
// bounded; a stalled pipeline raises DEV_TIMEOUT, drains its copies and frees tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "xm_internal.cuh"

namespace xm {
namespace {

constexpr int OZ_BM = 128;                 // tile rows (MMA M)
constexpr int OZ_BN = 128;                 // tile columns (MMA N)
constexpr int OZ_BK = 64;                  // k-block: one 128-byte swizzled row of BF16
constexpr int OZ_BITS = 7;                 // digit magnitude bits
constexpr int OZ_SLICES = 8;               // digits per entry = levels
constexpr int OZ_CHUNK = 16;               // k-blocks per exact FP32 accumulation (1024 products)
constexpr int OZ_STAGES = 6;
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 32 * (2 + OZ_EPI_WARPS);
constexpr int OZ_EPI_COLS = OZ_BN / 2;     // columns per epilogue warp
constexpr uint32_t OZ_A_BYTES = OZ_BM * OZ_BK * 2;
constexpr uint32_t OZ_B_BYTES = OZ_BN * OZ_BK * 2;
constexpr uint32_t OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;
constexpr uint32_t OZ_TMEM_COLS = 2 * OZ_BN;   // two FP32 accumulators
constexpr size_t OZ_SMEM = 1024 + (size_t)OZ_STAGES * OZ_STAGE_BYTES + 1024 +
                           (size_t)OZ_EPI_WARPS * OZ_EPI_COLS * sizeof(double);
constexpr int64_t OZ_MAX_K = 16640;        // int32 level sums: 8 K 127^2 < 2^31

// instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both K-major,
// N = 128 (bits 17..22 hold N / 8), M = 128 (bits 24..28 hold M / 16)
constexpr uint32_t OZ_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
                              ((uint32_t)(OZ_BM >> 4) << 24);

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 bytes,
// 8-row groups 1024 bytes apart (the layout a 64-wide BF16 TMA box with 128-byte swizzle
// writes); base 1024-byte aligned
__device__ __forceinline__ uint64_t sm_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;                  // descriptor version of sm_100 and later
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive (once) on the mbarrier when every tcgen05.mma issued so far by this thread is complete
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// ------------------------------------------------------------------ digit split
// One warp per output index c (a column of C, K entries at C + c * ldc).  Writes the 8 digit
// slices S[s][c][0..K_pad) (BF16, zero beyond K and for c >= n) and scale[c] = 2^{e_c} with
// max_k |C[k][c]| < 2^{e_c}.
__global__ void k_oz_split(const double* __restrict__ C, int ldc, int K, int n, int n_pad,
                           int K_pad, __nv_bfloat16* __restrict__ S, size_t slice_stride,
                           double* __restrict__ scale) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < n_pad; c += gridDim.x * wpb) {
    const double* col = C + (size_t)c * ldc;
    double mx = 0.0;
    if (c < n)
      for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(col[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) (void)frexp(mx, &e);     // mx = f 2^e, f in [0.5, 1)
    if (lane == 0) scale[c] = mx > 0.0 ? ldexp(1.0, e) : 0.0;
    __nv_bfloat16* dst = S + (size_t)c * K_pad;
    for (int k = lane; k < K_pad; k += 32) {
      double x = (c < n && k < K && mx > 0.0) ? ldexp(col[k], -e) : 0.0;   // |x| < 1
#pragma unroll
      for (int s = 0; s < OZ_SLICES; ++s) {
        const double t = x * (double)(1 << OZ_BITS);
        const double d = trunc(t);          // |d| <= 127, exact in BF16
        x = t - d;                          // exact
        dst[(size_t)s * slice_stride + k] = __double2bfloat16(d);
      }
    }
  }
}

// ------------------------------------------------------------------ rank-k update + pack
struct OzArgs {
  const int2* tiles;        // (I, J) per work item, I <= J
  int ntiles;
  int KB;                   // k-blocks per digit slice
  int n, nt;
  const double* scale;      // 2^{e_c}, n_pad entries
  const double* P;          // row-major n x n, upper triangle valid
  double* acc64;            // packed FP64 tiles (accumulator, then result)
  float* q32;               // packed FP32 tiles or null
  __nv_bfloat16* q16;       // packed BF16 tiles or null
  int* err;
};

__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_syrk(const __grid_constant__ CUtensorMap tmap, OzArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* stages = base;                                   // 1024-byte aligned
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + (size_t)OZ_STAGES * OZ_STAGE_BYTES);
  uint64_t* full = bars;                       // [OZ_STAGES]
  uint64_t* empty = full + OZ_STAGES;          // [OZ_STAGES]
  uint64_t* accfull = empty + OZ_STAGES;       // [2]
  uint64_t* accempty = accfull + 2;            // [2]
  uint64_t* done = accempty + 2;               // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  double* colscale = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(bars) + 1024);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], OZ_EPI_WARPS);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int KB = args.KB;

  if (warp == 0) {
    // ---------------- producer: operand boxes of every k-block, in MMA order
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int64_t issued = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < args.ntiles && ok; w += gridDim.x) {
        const int2 tj = args.tiles[w];
        for (int m = 0; m < OZ_SLICES && ok; ++m)
          for (int a = 0; a <= m && ok; ++a)
            for (int kb = 0; kb < KB; ++kb) {
              if (!mbar_wait(&empty[stage], phase ^ 1u)) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
              mbar_arrive_expect_tx(&full[stage], OZ_STAGE_BYTES);
              unsigned char* sa = stages + (size_t)stage * OZ_STAGE_BYTES;
              tma_load_3d(sa, &tmap, kb * OZ_BK, tj.x * OZ_BM, a, &full[stage]);
              tma_load_3d(sa + OZ_A_BYTES, &tmap, kb * OZ_BK, tj.y * OZ_BN, m - a, &full[stage]);
              ++issued;
              if (++stage == OZ_STAGES) { stage = 0; phase ^= 1u; }
            }
      }
      // do not leave while copies into this CTA's shared memory are in flight
      for (int64_t k = issued > OZ_STAGES ? issued - OZ_STAGES : 0; k < issued; ++k)
        if (!mbar_wait(&full[k % OZ_STAGES], (uint32_t)((k / OZ_STAGES) & 1))) { atomicOr(args.err, DEV_TIMEOUT); break; }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int64_t chunk = 0;
      bool ok = true;
      const uint32_t sbase = smem_u32(stages);
      for (int w = blockIdx.x; w < args.ntiles && ok; w += gridDim.x) {
        for (int m = 0; m < OZ_SLICES && ok; ++m) {
          const int total = (m + 1) * KB;
          for (int g = 0; g < total; ++g) {
            const int buf = (int)(chunk & 1);
            if (g % OZ_CHUNK == 0) {
              if (!mbar_wait(&accempty[buf], (uint32_t)(((chunk >> 1) & 1) ^ 1))) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
              tc_fence_after();
            }
            if (!mbar_wait(&full[stage], phase)) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
            tc_fence_after();
            const uint32_t sa = sbase + (uint32_t)stage * OZ_STAGE_BYTES;
            const uint64_t da = sm_desc(sa), db = sm_desc(sa + OZ_A_BYTES);
#pragma unroll
            for (int j = 0; j < OZ_BK / 16; ++j)   // K = 16 per MMA: 32 bytes along the row
              tc_mma(tmem + (uint32_t)(buf * OZ_BN), da + 2 * j, db + 2 * j, OZ_IDESC,
                     (g % OZ_CHUNK != 0 || j > 0) ? 1u : 0u);
            tc_commit(&empty[stage]);
            if (++stage == OZ_STAGES) { stage = 0; phase ^= 1u; }
            if ((g + 1) % OZ_CHUNK == 0 || g + 1 == total) {
              tc_commit(&accfull[buf]);
              ++chunk;
            }
          }
        }
      }
      // every issued MMA complete before tensor memory is freed
      tc_commit(done);
      if (!mbar_wait(done, 0)) atomicOr(args.err, DEV_TIMEOUT);
    }
  } else {
    // ---------------- epilogue: warps 2..9
    const int ew = warp - 2;
    const int quarter = warp & 3;            // TMEM lanes 32q .. 32q+31
    const int c0 = (ew >> 2) * OZ_EPI_COLS;  // first tile column of this warp
    const int a_loc = 32 * quarter + lane;   // tile row of this thread
    double* cs = colscale + (size_t)ew * OZ_EPI_COLS;
    int64_t chunk = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < args.ntiles && ok; w += gridDim.x) {
      const int2 tj = args.tiles[w];
      const int I = tj.x, J = tj.y;
      const int row = I * OZ_BM + a_loc;
      const double rs = args.scale[row];
      __syncwarp();
      for (int c = lane; c < OZ_EPI_COLS; c += 32) cs[c] = args.scale[J * OZ_BN + c0 + c];
      __syncwarp();
      const int64_t t = tile_index(args.nt, I, J);
      double* dst = args.acc64 + (size_t)t * TILE * TILE + (size_t)a_loc * TILE + c0;
      for (int m = 0; m < OZ_SLICES && ok; ++m) {
        int acc[OZ_EPI_COLS];
#pragma unroll
        for (int c = 0; c < OZ_EPI_COLS; ++c) acc[c] = 0;
        const int nchunk = ((m + 1) * KB + OZ_CHUNK - 1) / OZ_CHUNK;
        for (int q = 0; q < nchunk; ++q) {
          const int buf = (int)(chunk & 1);
          if (!mbar_wait(&accfull[buf], (uint32_t)((chunk >> 1) & 1))) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
          tc_fence_after();
          const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * OZ_BN + c0);
#pragma unroll
          for (int p = 0; p < OZ_EPI_COLS / 16; ++p) {
            float v[16];
            tc_ld16(ta + 16 * p, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[16 * p + i] += __float2int_rn(v[i]);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&accempty[buf]);
          ++chunk;
        }
        if (!ok) break;
        // level m: tile -= 2^{e_row + e_col - 7(m+2)} L_m (exact scaling, FP64 sum)
        const double f = ldexp(rs, -OZ_BITS * (m + 2));
#pragma unroll
        for (int c = 0; c < OZ_EPI_COLS; c += 2) {
          double2 cur = m == 0 ? make_double2(0.0, 0.0) : *reinterpret_cast<const double2*>(dst + c);
          cur.x -= (double)acc[c] * (f * cs[c]);
          cur.y -= (double)acc[c + 1] * (f * cs[c + 1]);
          *reinterpret_cast<double2*>(dst + c) = cur;
        }
      }
      if (!ok) break;
      // Q = P - C^T C in the packed layout: upper triangle, halved diagonal, zero padding
      const int n = args.n;
      const size_t g0 = (size_t)t * TILE * TILE + (size_t)a_loc * TILE + c0;
      for (int c = 0; c < OZ_EPI_COLS; ++c) {
        const int b_loc = c0 + c;
        const int col = J * OZ_BN + b_loc;
        double v = 0.0;
        if (row < n && col < n && (I < J || a_loc <= b_loc)) {
          v = args.P[(size_t)row * n + col] + dst[c];
          if (I == J && a_loc == b_loc) v *= 0.5;
        }
        dst[c] = v;
        if (args.q32) args.q32[g0 + c] = (float)v;
        if (args.q16) args.q16[g0 + c] = __double2bfloat16(v);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

struct DevMem {
  void* p = nullptr;
  ~DevMem() { if (p) cudaFree(p); }
};

}  // namespace

bool split_update_fits(int K, int n) { return K >= 1 && K <= OZ_MAX_K && n >= 1; }

// Q tiles <- pack(P - C^T C); C column-major K x n with leading dimension ldc (device), P
// row-major n x n (upper triangle valid).  q's tiles are allocated; acc64 is q.q64 or an FP64
// tile scratch of the same size.
xm_status split_update_pack(xm_ctx* ctx, const double* C, int ldc, int K, const double* P,
                            DeviceQ& q, double* acc64, double* t_update) {
  if (!split_update_fits(K, q.n))
    return set_error(XM_EINVAL, "split-BF16 update: K = %d outside [1, %lld]", K, (long long)OZ_MAX_K);
  cudaStream_t st = ctx->stream;
  const int KB = (K + OZ_BK - 1) / OZ_BK;
  const int K_pad = KB * OZ_BK;
  const int n_pad = q.n_pad;
  const size_t slice_stride = (size_t)n_pad * K_pad;
  DevMem S, scale, tl;
  XM_CUDA_TRY(cudaMalloc(&S.p, sizeof(__nv_bfloat16) * slice_stride * OZ_SLICES));
  XM_CUDA_TRY(cudaMalloc(&scale.p, sizeof(double) * (size_t)n_pad));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (t_update) {
    XM_CUDA_TRY(cudaEventCreate(&e0));
    XM_CUDA_TRY(cudaEventCreate(&e1));
    XM_CUDA_TRY(cudaEventRecord(e0, st));
  }
  {
    const int threads = 256;
    int grid = (n_pad + threads / 32 - 1) / (threads / 32);
    grid = std::min(grid, ctx->num_sms * 16);
    k_oz_split<<<grid, threads, 0, st>>>(C, ldc, K, q.n, n_pad, K_pad,
                                         static_cast<__nv_bfloat16*>(S.p), slice_stride,
                                         static_cast<double*>(scale.p));
    XM_CUDA_TRY(cudaGetLastError());
  }
  // work list: block rows of 8 tile rows, column by column, so that the CTAs running at one
  // time share the operand k-blocks of a few tile rows and columns in L2
  const int nt = q.nt;
  std::vector<int2> order;
  order.reserve((size_t)q.ntiles);
  for (int I0 = 0; I0 < nt; I0 += 8)
    for (int J = I0; J < nt; ++J)
      for (int I = I0; I < std::min(I0 + 8, J + 1); ++I) order.push_back(make_int2(I, J));
  XM_CUDA_TRY(cudaMalloc(&tl.p, sizeof(int2) * order.size()));
  XM_CUDA_TRY(cudaMemcpyAsync(tl.p, order.data(), sizeof(int2) * order.size(),
                              cudaMemcpyHostToDevice, st));

  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return set_error(XM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  CUtensorMap map;
  const cuuint64_t gdim[3] = {(cuuint64_t)K_pad, (cuuint64_t)n_pad, (cuuint64_t)OZ_SLICES};
  const cuuint64_t gstride[2] = {(cuuint64_t)K_pad * 2, (cuuint64_t)slice_stride * 2};
  const cuuint32_t box[3] = {OZ_BK, OZ_BM, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, S.p, gdim, gstride, box,
                          estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return set_error(XM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);

  static int configured_dev = -1;
  if (configured_dev != ctx->device) {
    XM_CUDA_TRY(cudaFuncSetAttribute(k_oz_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)OZ_SMEM));
    configured_dev = ctx->device;
  }
  OzArgs a;
  a.tiles = static_cast<const int2*>(tl.p);
  a.ntiles = (int)order.size();
  a.KB = KB;
  a.n = q.n;
  a.nt = nt;
  a.scale = static_cast<const double*>(scale.p);
  a.P = P;
  a.acc64 = acc64;
  a.q32 = q.q32;
  a.q16 = q.q16;
  a.err = ctx->d_err;
  const int grid = std::min(ctx->num_sms, a.ntiles);
  k_oz_syrk<<<grid, OZ_THREADS, OZ_SMEM, st>>>(map, a);
  XM_CUDA_TRY(cudaGetLastError());
  if (t_update) {
    XM_CUDA_TRY(cudaEventRecord(e1, st));
    XM_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    XM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *t_update = ms * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  return check_device_error(ctx, "split-BF16 rank-k update");
}

}  // namespace xm
