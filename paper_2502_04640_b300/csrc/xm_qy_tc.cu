// Q.Y sweep of the BF16-stored Q on the fifth-generation tensor cores (the Hessian-vector
// product of Sec. 3.2 in the mixed-precision bulk phase; BF16 storage of Q is this
// implementation's choice, App. A fixes only the matrix).
//
// Each packed upper-triangle tile T = Q_IJ (128 x 128 BF16) is read from HBM once and used
// twice, as in the SIMT sweep: W_I += T Y_J and W_J += T^T Y_I.  Both products are one
// tcgen05.mma chain on the same shared-memory copy of T: the row product reads T K-major, the
// column product reads it MN-major (the transpose costs nothing: the operand descriptor walks
// 64-element MN blocks LBO = 16 KB apart and 8-row K groups SBO = 1 KB apart).  Y is FP32; it
// enters the MMA as three BF16 digits y = d0 + d1 + d2 (each the round-to-nearest BF16 of what
// the previous ones left, so |y - d0 - d1 - d2| <= 2^-27 |y|), laid side by side as the MMA's N
// columns (3R of NP = 16 or 32); BF16 x BF16 products are exact and accumulate in FP32 in
// tensor memory, and the epilogue adds the three digit columns of each output.
//
//   * persistent grid, one CTA per SM, contiguous ranges of the tile list in the SIMT sweep's
//     paired row order (a long tile row, then the short one that completes it);
//   * warp 0: one thread streams each tile with the digit tiles of Y_J and Y_I into a 5-stage
//     (4 at r = 8) mbarrier ring, each a contiguous bulk copy (cp.async.bulk, the TMA engine): the BF16
//     tiles are stored in the operand layout itself (two 64-column halves, 128-byte swizzle,
//     bf16_tile_off) and the digit rows of Y are written per 128-row tile in the same layout;
//   * warps 1 and 6: one thread each issues the 8 MMAs (K = 16) of one product per tile into
//     tensor memory: warp 1 into the row accumulator of the current tile row (NP columns,
//     flushed once per row), warp 6 into four rotating column accumulators (flushed every tile;
//     the MMAs of a tile wait only for the epilogue of the tile four back);
//   * warps 2-5: read the accumulators with tcgen05.ld (one TMEM lane quarter each), add the
//     digit columns and add the results to W with vector reductions in L2.
// Every wait is bounded: a stalled pipeline raises DEV_TIMEOUT, drains its copies, waits for
// its MMAs and frees tensor memory.
#include <algorithm>
#include <mutex>

#include "xm_internal.cuh"

namespace xm {

namespace {

constexpr int TC_EPI_WARPS = 4;
constexpr int TC_NCOL = 4;                                  // column accumulators in flight
constexpr int TC_COL_WARP = 2 + TC_EPI_WARPS;               // issuer of the column products
constexpr int TC_THREADS = 32 * (3 + TC_EPI_WARPS);
constexpr uint32_t TC_Q_BYTES = TILE * TILE * 2;          // one BF16 tile, two 16 KB boxes
constexpr uint32_t TC_QBOX = TC_Q_BYTES / 2;                 // one 64-column half
constexpr int TC_DIGITS = 3;

template <int NP>
struct TcCfg {
  static constexpr uint32_t YBOX = NP * 128;                 // NP rows x 64 BF16 (128 bytes)
  static constexpr uint32_t YTILE = 2 * YBOX;                // all digit columns of 128 rows
  static constexpr uint32_t STAGE = TC_Q_BYTES + 2 * YTILE;  // T, Y_J digits, Y_I digits
  static constexpr int STAGES = NP == 16 ? 5 : 4;            // as many as shared memory holds
  static constexpr uint32_t TMEM_COLS = NP == 16 ? 128 : 256; // row + TC_NCOL column accumulators
  // kind::f16 instruction descriptor: D FP32, A and B BF16, M = 128, N = NP; bit 15 reads A
  // MN-major (the column product's T^T)
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NP >> 3) << 17) |
                                    ((uint32_t)(128 >> 4) << 24);
  static constexpr uint32_t IDESC_T = IDESC | (1u << 15);
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256;
};

// shared-memory operand descriptor (sm_100 form): start, leading and stride byte offsets in
// 16-byte units, 128-byte swizzle; atoms of 8 rows x 128 bytes, 1024-byte aligned
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
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
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
template <int NP>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&v)[NP]) {
  static_assert(NP == 16 || NP == 32, "NP");
  uint32_t r[16];
#pragma unroll
  for (int h = 0; h < NP / 16; ++h) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr + 16 * h));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[16 * h + i] = __uint_as_float(r[i]);
  }
}
// W rows += the digit sums of one accumulator row (R outputs; v holds digit d of output j at
// column d R + j)
template <int R, int NP>
__device__ __forceinline__ void add_row(float* w, const float (&v)[NP]) {
  float o[R];
#pragma unroll
  for (int j = 0; j < R; ++j) o[j] = (v[j] + v[R + j]) + v[2 * R + j];
  if constexpr (R == 1) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(w), "f"(o[0]) : "memory");
  } else {
#pragma unroll
    for (int j = 0; j < R; j += 4)
      asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(w + j), "f"(o[j]),
                   "f"(o[j + 1]), "f"(o[j + 2]), "f"(o[j + 3])
                   : "memory");
  }
}

// Yd: per 128-row tile of Y, the NP x 128 BF16 digit block in the operand layout (two 64-row
// halves of NP x 128 bytes, chunk c of digit row m at position c xor (m mod 8)); digit row
// d R + j holds digit d of column j, rows >= 3R are zero.
template <int R, int NP>
__global__ void k_y_digits(int n_pad, const float* __restrict__ Y, __nv_bfloat16* __restrict__ Yd,
                           const int* skip) {
  if (skip != nullptr && *skip != 0) return;
  const int64_t total = (int64_t)NP * n_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    // e enumerates (tile, half, digit row, k within the half) in storage order
    const int64_t tile = e / (NP * TILE);
    const int rem = (int)(e - tile * (NP * TILE));
    const int half = rem / (NP * 64), m = (rem / 64) % NP, pos = rem % 64;
    const int kk = ((((pos >> 3) ^ (m & 7)) << 3) | (pos & 7));   // the swizzle is an involution
    const int64_t k = tile * TILE + half * 64 + kk;
    float out = 0.f;
    if (m < TC_DIGITS * R) {
      const int d = m / R, j = m - d * R;
      float r = Y[(size_t)k * R + j];
      for (int s = 0; s < d; ++s) r -= __bfloat162float(__float2bfloat16_rn(r));
      out = r;
    }
    Yd[e] = __float2bfloat16_rn(out);
  }
}

template <int R, int NP>
__global__ void __launch_bounds__(TC_THREADS, 1)
qy_tc_kernel(int nt, int64_t ntiles, const __nv_bfloat16* __restrict__ tiles,
             const __nv_bfloat16* __restrict__ Yd, float* __restrict__ W, int* err, const int* skip) {
  using C = TcCfg<NP>;
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* stages = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(stages + (size_t)C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* colfull = empty + C::STAGES;   // [TC_NCOL]
  uint64_t* colempty = colfull + TC_NCOL;  // [TC_NCOL]
  uint64_t* rowfull = colempty + TC_NCOL;
  uint64_t* rowempty = rowfull + 1;
  uint64_t* done = rowempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x;
  const int64_t t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 2);      // both issuers' MMAs have read the stage
    }
    for (int b = 0; b < TC_NCOL; ++b) {
      mbar_init(&colfull[b], 1);
      mbar_init(&colempty[b], TC_EPI_WARPS);
    }
    mbar_init(rowfull, 1);
    mbar_init(rowempty, TC_EPI_WARPS);
    mbar_init(done, 2);
    fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int I0, J0;
  pair_order_start(nt, t0, I0, J0);

  if (warp == 0) {
    // ---------------- producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int64_t issued = 0;
      int I = I0, J = J0;
      for (int64_t t = t0; t < t1; ++t) {
        if (!mbar_wait(&empty[stage], phase ^ 1u)) { atomicOr(err, DEV_TIMEOUT); break; }
        mbar_arrive_expect_tx(&full[stage], C::STAGE);
        unsigned char* s = stages + (size_t)stage * C::STAGE;
        const unsigned char* yd = reinterpret_cast<const unsigned char*>(Yd);
        bulk_g2s(s, tiles + (size_t)tile_index(nt, I, J) * TILE * TILE, TC_Q_BYTES, &full[stage]);
        bulk_g2s(s + TC_Q_BYTES, yd + (size_t)J * C::YTILE, C::YTILE, &full[stage]);
        bulk_g2s(s + TC_Q_BYTES + C::YTILE, yd + (size_t)I * C::YTILE, C::YTILE, &full[stage]);
        ++issued;
        if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
        pair_order_next(nt, I, J);
      }
      // do not leave while copies into this CTA's shared memory are in flight
      for (int64_t k = issued > C::STAGES ? issued - C::STAGES : 0; k < issued; ++k)
        if (!mbar_wait(&full[k % C::STAGES], (uint32_t)((k / C::STAGES) & 1))) { atomicOr(err, DEV_TIMEOUT); break; }
    }
  } else if (warp == 1 || warp == TC_COL_WARP) {
    // ---------------- MMA issuers: warp 1 the row products, the last warp the column products
    // (two issuing threads: the tensor core takes a small MMA about as fast as one thread can
    // issue it, so splitting the two independent chains doubles the rate)
    if (lane == 0) {
      const bool rows = warp == 1;
      int stage = 0;
      uint32_t phase = 0;
      int I = I0, J = J0;
      int64_t rows_done = 0;      // tile rows whose accumulator was handed to the epilogue
      bool ok = true;
      const uint32_t sbase = smem_u32(stages);
      for (int64_t t = t0; t < t1 && ok; ++t) {
        const int64_t k = t - t0;
        const bool newrow = (t == t0) || J == I;   // a tile row starts at its diagonal (or at t0)
        const int cb = (int)(k % TC_NCOL);
        if (rows && newrow && rows_done > 0) {
          if (!mbar_wait(rowempty, (uint32_t)((rows_done - 1) & 1))) { atomicOr(err, DEV_TIMEOUT); ok = false; break; }
        }
        if (!rows && k >= TC_NCOL) {
          if (!mbar_wait(&colempty[cb], (uint32_t)(((k - TC_NCOL) / TC_NCOL) & 1))) { atomicOr(err, DEV_TIMEOUT); ok = false; break; }
        }
        if (!mbar_wait(&full[stage], phase)) { atomicOr(err, DEV_TIMEOUT); ok = false; break; }
        tc_fence_after();
        const uint32_t qa = sbase + (uint32_t)stage * C::STAGE;
        const uint32_t yj = qa + TC_Q_BYTES, yi = yj + C::YTILE;
        if (rows) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {   // W_I += T Y_J: T K-major, K = columns of the tile
            const uint64_t a = tc_desc(qa + (j >> 2) * TC_QBOX + 32 * (j & 3), 16, 1024);
            const uint64_t b = tc_desc(yj + (j >> 2) * C::YBOX + 32 * (j & 3), 16, 1024);
            tc_mma(tmem, a, b, C::IDESC, (newrow && j == 0) ? 0u : 1u);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {   // W_J += T^T Y_I: T MN-major, K = rows of the tile
            const uint64_t a = tc_desc(qa + 2048 * j, TC_QBOX, 1024);
            const uint64_t b = tc_desc(yi + (j >> 2) * C::YBOX + 32 * (j & 3), 16, 1024);
            tc_mma(tmem + (uint32_t)(NP * (1 + cb)), a, b, C::IDESC_T, j > 0 ? 1u : 0u);
          }
        }
        tc_commit(&empty[stage]);
        if (!rows) tc_commit(&colfull[cb]);
        if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
        int In = I, Jn = J;
        pair_order_next(nt, In, Jn);
        if (rows && (t + 1 == t1 || In != I)) {
          tc_commit(rowfull);
          ++rows_done;
        }
        I = In; J = Jn;
      }
      // every issued MMA complete before tensor memory is freed
      tc_commit(done);
      if (!mbar_wait(done, 0)) atomicOr(err, DEV_TIMEOUT);
    }
  } else {
    // ---------------- epilogue: warps 2..5, TMEM lane quarter warp % 4
    const int quarter = warp & 3;
    const int r_loc = 32 * quarter + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    int I = I0, J = J0;
    int64_t rows_done = 0;
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t k = t - t0;
      const int cb = (int)(k % TC_NCOL);
      if (!mbar_wait(&colfull[cb], (uint32_t)((k / TC_NCOL) & 1))) { atomicOr(err, DEV_TIMEOUT); break; }
      tc_fence_after();
      float v[NP];
      tc_ld<NP>(lane_base + (uint32_t)(NP * (1 + cb)), v);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&colempty[cb]);
      add_row<R, NP>(W + ((size_t)J * TILE + r_loc) * R, v);
      int In = I, Jn = J;
      pair_order_next(nt, In, Jn);
      if (t + 1 == t1 || In != I) {
        if (!mbar_wait(rowfull, (uint32_t)(rows_done & 1))) { atomicOr(err, DEV_TIMEOUT); break; }
        tc_fence_after();
        float u[NP];
        tc_ld<NP>(lane_base, u);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(rowempty);
        add_row<R, NP>(W + ((size_t)I * TILE + r_loc) * R, u);
        ++rows_done;
      }
      I = In; J = Jn;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
}

template <int R, int NP>
xm_status launch_tc(xm_ctx* ctx, const DeviceQ& q, const float* Y, float* W, const int* skip,
                    cudaStream_t st) {
  using C = TcCfg<NP>;
  constexpr int MAX_DEVICES = 64;
  static std::mutex mu;
  static bool configured[MAX_DEVICES] = {};
  if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
    return set_error(XM_EINVAL, "sweep: device %d out of range", ctx->device);
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!configured[ctx->device]) {
      if (C::SMEM > ctx->smem_optin)
        return set_error(XM_ECUDA, "tensor-core sweep: needs %zu bytes of shared memory", C::SMEM);
      XM_CUDA_TRY(cudaFuncSetAttribute(qy_tc_kernel<R, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::SMEM));
      configured[ctx->device] = true;
    }
  }
  const int64_t total = (int64_t)NP * q.n_pad;
  const int gd = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 4);
  k_y_digits<R, NP><<<gd, 256, 0, st>>>(q.n_pad, Y, q.ydig, skip);
  int grid = ctx->num_sms;
  if ((int64_t)grid > q.ntiles) grid = (int)q.ntiles;
  qy_tc_kernel<R, NP><<<grid, TC_THREADS, C::SMEM, st>>>(q.nt, q.ntiles, q.q16, q.ydig, W, ctx->d_err, skip);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

}  // namespace

xm_status qy_tc_launch(xm_ctx* ctx, const DeviceQ& q, int R, const float* Y, float* W,
                       const int* skip, cudaStream_t st) {
  if (!q.q16 || !q.ydig) return set_error(XM_EINVAL, "sweep: Q has no BF16 copy");
  switch (R) {
    case 1: return launch_tc<1, 16>(ctx, q, Y, W, skip, st);
    case 4: return launch_tc<4, 16>(ctx, q, Y, W, skip, st);
    case 8: return launch_tc<8, 32>(ctx, q, Y, W, skip, st);
    default: return set_error(XM_EINVAL, "sweep: padded width %d not in {1,4,8}", R);
  }
}

}  // namespace xm
