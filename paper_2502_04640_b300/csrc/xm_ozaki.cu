// The dense FP64 contractions of the Q build on the BF16 tensor cores (tcgen05), FP64-accurate.
//
// Translation elimination (App. A, Prop. 1) forms C = L^{-1} Bbar^T, an (N-1) x n matrix (L the
// Cholesky factor of the anchored translation block Sbar), and Q = P - C^T C.  The triangular
// solve (3 N^3 flops) and the symmetric rank-(N-1) product (9 N^3 flops: 9.4 TFLOP at 10155
// cameras) are the method's dense contractions; at B300's FP64 rate (about 1 TFLOP/s) they take
// 12 s.  Both run here as products on the BF16 tensor cores by the error-free splitting of
// Ozaki, Ogita, Oishi and Rump (2012):
//
//   * every operand vector v (a column of C or of a block of C, a row of a block of L) is written
//     as 2^{e_v} sum_{s<8} d_s 2^{-7(s+1)} with integer digits |d_s| <= 127 (exact in BF16); the
//     8 digits hold every entry to within 2^{-56} of the largest entry of its vector;
//   * (u . v) = 2^{e_u+e_v} sum_{m<8} 2^{-7(m+2)} L_m, L_m = sum_{a+b=m} d_a(u) . d_b(v), dropping
//     digit products of order m >= 8 (below 2^{-56} K max|u| max|v|): normwise as accurate as FP64;
//   * each level L_m is a BF16 GEMM over the concatenated K' = (m+1) K whose FP32 accumulation
//     in tensor memory is exact as long as at most 1024 products (each < 2^14) are summed: the
//     accumulator restarts every 16 k-blocks of 64 and the epilogue adds each chunk, as an
//     integer, to int32 registers (|L_m| < 2^31 for K <= 16640);
//   * a finished level is scaled by an exact power of two and subtracted in FP64 from the output.
//
// Two uses of one kernel (template MODE):
//   OZ_SYRK  Q = P - C^T C into the packed upper-triangle tiles of the sweep (FP64 accumulator
//            tile, then P added, diagonal halved, lower triangle and padding zeroed, FP32 and
//            BF16 copies written);
//   OZ_GEMM  out -= A B^T into a column-major FP64 matrix: the steps X_i = 0 - (-L_ii^{-1}) X_i and
//            the block updates X_rest -= L_rest,i X_i of a right-looking blocked triangular solve
//            (the 1024 x 1024 diagonal-block inverses formed in FP64 by cuBLAS), and the trailing
//            updates S_rest -= L_k L_k^T of a right-looking blocked Cholesky factorisation
//            (diagonal blocks by cuSOLVER, panels by DTRSM, FP64; only tiles meeting the lower
//            triangle).
//
// Kernel: persistent, one CTA per SM, 128 x 256 output tiles (MMA M = 128, N = 256) in an order
// that lets concurrent CTAs share operand k-blocks in L2.  Warp 0 streams the 128 x 64 and
// 256 x 64 BF16 operand boxes of each k-block with TMA (128-byte swizzle) into a 4-stage
// mbarrier ring; one thread of warp 1 issues tcgen05.mma (K = 16) into one of two 256-column
// TMEM accumulators (all 512 columns); warps 2..17 read finished chunks with tcgen05.ld (four
// warps per TMEM lane quarter, 64 columns each) while the next chunk accumulates.  Every wait is
// bounded; a stalled pipeline raises DEV_TIMEOUT, drains its copies and frees tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "xm_internal.cuh"

namespace xm {

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query: no libcuda
// link); null when the driver lacks it
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {

constexpr int OZ_BM = 128;                 // tile rows (MMA M)
constexpr int OZ_BN = 256;                 // tile columns (MMA N)
constexpr int OZ_BK = 64;                  // k-block: one 128-byte swizzled row of BF16
constexpr int OZ_BITS = 7;                 // digit magnitude bits
constexpr int OZ_SLICES = 8;               // digits per entry = levels
constexpr int OZ_CHUNK = 16;               // k-blocks per exact FP32 accumulation (1024 products)
constexpr int OZ_STAGES = 4;
constexpr int OZ_ACC = 2;                  // TMEM accumulators (2 x 256 columns = all 512)
constexpr int OZ_EPI_WARPS = 16;
constexpr int OZ_THREADS = 32 * (2 + OZ_EPI_WARPS);
constexpr int OZ_EPI_COLS = 64;            // columns per epilogue warp
constexpr uint32_t OZ_A_BYTES = OZ_BM * OZ_BK * 2;
constexpr uint32_t OZ_B_BYTES = OZ_BN * OZ_BK * 2;
constexpr uint32_t OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;
constexpr uint32_t OZ_TMEM_COLS = OZ_ACC * OZ_BN;
constexpr size_t OZ_SMEM = 1024 + (size_t)OZ_STAGES * OZ_STAGE_BYTES + 256;
constexpr int64_t OZ_MAX_K = 16640;        // int32 level sums: 8 K 127^2 < 2^31
constexpr int OZ_TRSM_BLOCK = 1024;        // diagonal block of the blocked triangular solve
constexpr int OZ_CHOL_BLOCK = 256;         // diagonal block of the blocked Cholesky factorisation

enum { OZ_SYRK = 0, OZ_GEMM = 1 };

// instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both K-major,
// N = 256 (bits 17..22 hold N / 8), M = 128 (bits 24..28 hold M / 16)
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

// 8 digits of x = v 2^{-e} (|v| < 2^e): d_s = trunc(2^7 r_s), r_0 = x, r_{s+1} = 2^7 r_s - d_s.
// Each step truncates toward zero, so d_s carries the sign of x and |d_s| is digit s (most
// significant first) of the base-128 expansion of floor(|x| 2^56).  That integer is read off the
// bits of v: |v| = m 2^{ex} with m the 53-bit significand, floor(|x| 2^56) = floor(m 2^{ex+56-e})
// (< 2^56 since |x| < 1).  Integer operations only: B300's FP64 pipe is 1/64 of its FP32 rate.
__device__ __forceinline__ void digits8(double v, int e, int (&d)[OZ_SLICES]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((bits >> 52) & 0x7FFu);
  unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
  int ex = -1074;                                    // subnormal (or zero) v
  if (E != 0) { m |= 1ull << 52; ex = E - 1075; }
  const int sh = ex + 56 - e;                        // <= 3 because |v| < 2^e
  unsigned long long U = 0;
  if (sh >= 0) U = m << sh;
  else if (sh > -64) U = m >> (-sh);
  const bool neg = (bits >> 63) != 0;
#pragma unroll
  for (int s = 0; s < OZ_SLICES; ++s) {
    const int g = (int)((U >> (OZ_BITS * (OZ_SLICES - 1 - s))) & 127u);
    d[s] = neg ? -g : g;
  }
}

// the BF16 pair (lo, hi) of two digits (|d| <= 127: exact) as one 32-bit word
__device__ __forceinline__ uint32_t bf16_pair(int lo, int hi) {
  const __nv_bfloat162 p = __halves2bfloat162(__float2bfloat16_rn((float)lo), __float2bfloat16_rn((float)hi));
  return *reinterpret_cast<const uint32_t*>(&p);
}

// |v| as an ordered integer key (sign cleared: the order of non-negative doubles)
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// scale exponent of a vector with largest magnitude mx: mx = f 2^e, f in [0.5, 1); 0 if mx == 0
__device__ __forceinline__ int scale_exp(double mx) {
  int e = 0;
  if (mx > 0.0) (void)frexp(mx, &e);
  return e;
}

// ------------------------------------------------------------------ digit split
// Columns of a column-major matrix: one warp per vector c (K entries at V + c * ldv, c < nv);
// lane l takes entries 8l .. 8l+7 of every 256 and writes each digit slice 16 bytes at a time.
// Writes the digit slices S[s][c][0..K_pad) (BF16, zero beyond K and for nv <= c < rows) and
// the scale exponent sexp[c] = e_c with max_k |V[k][c]| < 2^{e_c} (0 for a zero vector).
__global__ void k_oz_split_cols(const double* __restrict__ V, int ldv, int K, int nv, int rows,
                                int K_pad, __nv_bfloat16* __restrict__ S, size_t slice_stride,
                                int* __restrict__ sexp) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < rows; c += gridDim.x * wpb) {
    const double* col = V + (size_t)c * ldv;
    const bool valid = c < nv;
    unsigned long long mk = 0;
    if (valid)
      for (int k = lane; k < K; k += 32) mk = max(mk, abs_key(col[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
    const double mx = __longlong_as_double((long long)mk);
    const int e = scale_exp(mx);
    if (lane == 0) sexp[c] = e;
    __nv_bfloat16* dst = S + (size_t)c * K_pad;
    for (int k0 = 8 * lane; k0 < K_pad; k0 += 256) {
      uint32_t w[OZ_SLICES][4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        int d0[OZ_SLICES], d1[OZ_SLICES];
        const int k = k0 + j;
        digits8((valid && k < K) ? col[k] : 0.0, e, d0);
        digits8((valid && k + 1 < K) ? col[k + 1] : 0.0, e, d1);
#pragma unroll
        for (int s = 0; s < OZ_SLICES; ++s) w[s][j / 2] = bf16_pair(d0[s], d1[s]);
      }
#pragma unroll
      for (int s = 0; s < OZ_SLICES; ++s)
        *reinterpret_cast<uint4*>(dst + (size_t)s * slice_stride + k0) =
            make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
  }
}

// Rows of a column-major block: one thread per vector r (entries A[r + k * lda], k < K, r < nv);
// same outputs as k_oz_split_cols, written 8 digits (16 bytes) at a time.
__global__ void k_oz_split_rows(const double* __restrict__ A, int lda, int K, int nv, int rows,
                                int K_pad, __nv_bfloat16* __restrict__ S, size_t slice_stride,
                                int* __restrict__ sexp) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const bool valid = r < nv;
    unsigned long long mk = 0;
    if (valid)
      for (int k = 0; k < K; ++k) mk = max(mk, abs_key(A[r + (size_t)k * lda]));
    const double mx = __longlong_as_double((long long)mk);
    const int e = scale_exp(mx);
    sexp[r] = e;
    for (int k0 = 0; k0 < K_pad; k0 += 8) {
      uint32_t w[OZ_SLICES][4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        int d0[OZ_SLICES], d1[OZ_SLICES];
        const int k = k0 + j;
        digits8((valid && k < K) ? A[r + (size_t)k * lda] : 0.0, e, d0);
        digits8((valid && k + 1 < K) ? A[r + (size_t)(k + 1) * lda] : 0.0, e, d1);
#pragma unroll
        for (int s = 0; s < OZ_SLICES; ++s) w[s][j / 2] = bf16_pair(d0[s], d1[s]);
      }
#pragma unroll
      for (int s = 0; s < OZ_SLICES; ++s)
        *reinterpret_cast<uint4*>(S + (size_t)s * slice_stride + (size_t)r * K_pad + k0) =
            make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
  }
}

// 2^E a as a double (a an int32), exact whenever it is a normal double: the leading bit, the
// significand and the exponent field are set with integer operations (no branch, no FP64
// instruction), so that a level fold costs one FP64 operation (the subtraction) instead of three
// (conversion, scaling, subtraction) on B300's slow FP64 pipe.  Below the normal range the
// result is 0 (a level term under 2^-1022, far below the rounding of the FP64 output); above it,
// +-inf.
__device__ __forceinline__ double i2d_pow2(int a, int E) {
  const unsigned u = a < 0 ? 0u - (unsigned)a : (unsigned)a;
  const int p = 31 - __clz(u | 1u);                  // 2^p <= u < 2^{p+1} (u > 0)
  const int be = p + E + 1023;
  const unsigned long long sign = a < 0 ? (1ull << 63) : 0ull;
  const unsigned long long mant = ((unsigned long long)u << (52 - p)) & 0xFFFFFFFFFFFFFull;
  unsigned long long bits = sign | ((unsigned long long)(be > 0 ? be : 0) << 52) | mant;
  bits = be >= 2047 ? (sign | 0x7FF0000000000000ull) : bits;
  bits = (u == 0u || be <= 0) ? 0ull : bits;
  return __longlong_as_double((long long)bits);
}

// ------------------------------------------------------------------ digit-product kernel
struct OzArgs {
  const int2* tiles;        // (I, J) per work item: rows I*128.., columns J*256..
  int ntiles;
  int KB;                   // k-blocks per digit slice
  const int* expA;          // scale exponents e of the A vectors (rows of the output)
  const int* expB;          // scale exponents e of the B vectors (columns of the output)
  // OZ_SYRK
  int n, nt;                // Q order, 128-tiles per side
  const double* P;          // row-major n x n, upper triangle valid
  double* acc64;            // packed FP64 tiles (accumulator, then result)
  float* q32;               // packed FP32 tiles or null
  __nv_bfloat16* q16;       // packed BF16 tiles or null
  // OZ_GEMM
  double* out;              // column-major, out[row + col * ldo] -= product
  int ldo, M, ncols;
  int* err;
};

template <int MODE>
__global__ void __launch_bounds__(OZ_THREADS, 1)
k_oz_mma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
         OzArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* stages = base;                                   // 1024-byte aligned
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + (size_t)OZ_STAGES * OZ_STAGE_BYTES);
  uint64_t* full = bars;                       // [OZ_STAGES]
  uint64_t* empty = full + OZ_STAGES;          // [OZ_STAGES]
  uint64_t* accfull = empty + OZ_STAGES;       // [OZ_ACC]
  uint64_t* accempty = accfull + OZ_ACC;       // [OZ_ACC]
  uint64_t* done = accempty + OZ_ACC;          // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < OZ_ACC; ++b) {
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
              tma_load_3d(sa, &mapA, kb * OZ_BK, tj.x * OZ_BM, a, &full[stage]);
              tma_load_3d(sa + OZ_A_BYTES, &mapB, kb * OZ_BK, tj.y * OZ_BN, m - a, &full[stage]);
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
            const int buf = (int)(chunk % OZ_ACC);
            if (g % OZ_CHUNK == 0) {
              if (!mbar_wait(&accempty[buf], (uint32_t)(((chunk / OZ_ACC) & 1) ^ 1))) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
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
    // ---------------- epilogue: warps 2..17
    const int quarter = warp & 3;             // TMEM lanes 32q .. 32q+31
    const int grp = (warp - 2) >> 2;          // 64-column group of the 256-column tile
    const int a_loc = 32 * quarter + lane;    // tile row of this thread
    int64_t chunk = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < args.ntiles && ok; w += gridDim.x) {
      const int2 tj = args.tiles[w];
      const int row = tj.x * OZ_BM + a_loc;
      const int col0 = tj.y * OZ_BN + grp * OZ_EPI_COLS;       // first output column
      const int er = args.expA[row];
      const int* ce = args.expB + col0;                          // uniform across the warp
      // OZ_SYRK: the packed 128 x 128 tile this warp's columns fall in
      const int I = tj.x, J = 2 * tj.y + (grp >> 1);
      const bool live = MODE == OZ_GEMM || (J >= I && J < args.nt);
      const int64_t t = (MODE == OZ_SYRK && live) ? tile_index(args.nt, I, J) : 0;
      double* dst = MODE == OZ_SYRK
                        ? args.acc64 + (size_t)t * TILE * TILE + (size_t)a_loc * TILE + (grp & 1) * OZ_EPI_COLS
                        : nullptr;
      for (int m = 0; m < OZ_SLICES && ok; ++m) {
        int acc[OZ_EPI_COLS];
#pragma unroll
        for (int c = 0; c < OZ_EPI_COLS; ++c) acc[c] = 0;
        const int nchunk = ((m + 1) * KB + OZ_CHUNK - 1) / OZ_CHUNK;
        for (int q = 0; q < nchunk; ++q) {
          const int buf = (int)(chunk % OZ_ACC);
          if (!mbar_wait(&accfull[buf], (uint32_t)((chunk / OZ_ACC) & 1))) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
          tc_fence_after();
          if (live) {
            const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) +
                                (uint32_t)(buf * OZ_BN + grp * OZ_EPI_COLS);
#pragma unroll
            for (int p = 0; p < OZ_EPI_COLS / 16; ++p) {
              float v[16];
              tc_ld16(ta + 16 * p, v);
#pragma unroll
              for (int i = 0; i < 16; ++i) acc[16 * p + i] += __float2int_rn(v[i]);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&accempty[buf]);
          ++chunk;
        }
        if (!ok || !live) continue;
        // level m: output -= 2^{e_row + e_col - 7(m+2)} L_m (exact scaling, FP64 subtraction)
        const int Em = er - OZ_BITS * (m + 2);
        if constexpr (MODE == OZ_SYRK) {
#pragma unroll
          for (int c = 0; c < OZ_EPI_COLS; c += 2) {
            double2 cur = m == 0 ? make_double2(0.0, 0.0) : *reinterpret_cast<const double2*>(dst + c);
            cur.x -= i2d_pow2(acc[c], Em + ce[c]);
            cur.y -= i2d_pow2(acc[c + 1], Em + ce[c + 1]);
            *reinterpret_cast<double2*>(dst + c) = cur;
          }
        } else {
          if (row < args.M) {
#pragma unroll
            for (int c = 0; c < OZ_EPI_COLS; ++c) {
              const int col = col0 + c;
              if (col < args.ncols) {
                double* o = args.out + (size_t)col * args.ldo + row;   // coalesced along rows
                *o -= i2d_pow2(acc[c], Em + ce[c]);
              }
            }
          }
        }
      }
      if (!ok) break;
      if constexpr (MODE == OZ_SYRK) {
        if (!live) continue;
        // Q = P - C^T C in the packed layout: upper triangle, halved diagonal, zero padding
        const int n = args.n;
        const size_t g0 = (size_t)t * TILE * TILE + (size_t)a_loc * TILE + (grp & 1) * OZ_EPI_COLS;
        for (int c = 0; c < OZ_EPI_COLS; ++c) {
          const int b_loc = (grp & 1) * OZ_EPI_COLS + c;
          const int col = J * TILE + b_loc;
          double v = 0.0;
          if (row < n && col < n && (I < J || a_loc <= b_loc)) {
            v = args.P[(size_t)row * n + col] + dst[c];
            if (I == J && a_loc == b_loc) v *= 0.5;
          }
          dst[c] = v;
          if (args.q32) args.q32[g0 + c] = (float)v;
          if (args.q16) args.q16[(size_t)t * TILE * TILE + bf16_tile_off(a_loc, b_loc)] = __double2bfloat16(v);
        }
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

// 3-D map of digit slices S[8][rows][K_pad] (BF16), box of 64 k x box_rows rows x 1 slice
xm_status slice_map(CUtensorMap* map, void* S, int K_pad, int rows, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return set_error(XM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t gdim[3] = {(cuuint64_t)K_pad, (cuuint64_t)rows, (cuuint64_t)OZ_SLICES};
  const cuuint64_t gstride[2] = {(cuuint64_t)K_pad * 2, (cuuint64_t)K_pad * 2 * (cuuint64_t)rows};
  const cuuint32_t box[3] = {OZ_BK, box_rows, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, S, gdim, gstride, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return set_error(XM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  return XM_OK;
}

template <int MODE>
xm_status launch_mma(xm_ctx* ctx, const CUtensorMap& ma, const CUtensorMap& mb, OzArgs a) {
  static int configured_dev = -1;
  if (configured_dev != ctx->device) {
    XM_CUDA_TRY(cudaFuncSetAttribute(k_oz_mma<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)OZ_SMEM));
    configured_dev = ctx->device;
  }
  const int grid = std::min(ctx->num_sms, a.ntiles);
  if (grid < 1) return XM_OK;
  k_oz_mma<MODE><<<grid, OZ_THREADS, OZ_SMEM, ctx->stream>>>(ma, mb, a);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

int split_grid(xm_ctx* ctx, int work, int per_block);

// (I, J) work items: groups of 8 tile rows, column by column, so that the CTAs running at one
// time share the operand k-blocks of a few tile rows and columns in L2.  keep(I, J) filters.
template <typename F>
std::vector<int2> tile_order(int nI, int nJ, F keep) {
  std::vector<int2> order;
  for (int I0 = 0; I0 < nI; I0 += 8)
    for (int J = 0; J < nJ; ++J)
      for (int I = I0; I < std::min(I0 + 8, nI); ++I)
        if (keep(I, J)) order.push_back(make_int2(I, J));
  return order;
}

struct DevMem {
  void* p = nullptr;
  ~DevMem() { if (p) cudaFree(p); }
  template <typename T> T* as() { return static_cast<T*>(p); }
};

int split_grid(xm_ctx* ctx, int work, int per_block) {
  int g = (work + per_block - 1) / per_block;  // grid-stride kernels: at most 16 blocks per SM
  return std::max(1, std::min(g, ctx->num_sms * 16));
}

}  // namespace

bool split_update_fits(int K, int n) { return K >= 1 && K <= OZ_MAX_K && n >= 1; }

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

// Q tiles <- pack(P - C^T C); C column-major K x n with leading dimension ldc (device), P
// row-major n x n (upper triangle valid).  q's tiles are allocated; acc64 is q.q64 or an FP64
// tile scratch of the same size.
xm_status split_update_pack(xm_ctx* ctx, const double* C, int ldc, int K, const double* P,
                            DeviceQ& q, double* acc64) {
  if (!split_update_fits(K, q.n))
    return set_error(XM_EINVAL, "split-BF16 update: K = %d outside [1, %lld]", K, (long long)OZ_MAX_K);
  cudaStream_t st = ctx->stream;
  const int KB = (K + OZ_BK - 1) / OZ_BK;
  const int K_pad = KB * OZ_BK;
  const int nt = q.nt;
  const int nt2 = (nt + 1) / 2;                   // 256-column tiles
  const int rows = nt2 * OZ_BN;                   // slice rows: a multiple of 128 and 256
  const size_t slice_stride = (size_t)rows * K_pad;
  DevMem S, sexp, tl;
  XM_CUDA_TRY(cudaMalloc(&S.p, sizeof(__nv_bfloat16) * slice_stride * OZ_SLICES));
  XM_CUDA_TRY(cudaMalloc(&sexp.p, sizeof(int) * (size_t)rows));
  k_oz_split_cols<<<split_grid(ctx, rows, 8), 256, 0, st>>>(C, ldc, K, q.n, rows, K_pad,
                                                            S.as<__nv_bfloat16>(), slice_stride,
                                                            sexp.as<int>());
  XM_CUDA_TRY(cudaGetLastError());
  // 128 x 256 tiles meeting the upper triangle: packed tile (I, 2J) or (I, 2J+1) with J >= I
  std::vector<int2> order = tile_order(nt, nt2, [](int I, int J) { return 2 * J + 1 >= I; });
  XM_CUDA_TRY(cudaMalloc(&tl.p, sizeof(int2) * order.size()));
  XM_CUDA_TRY(cudaMemcpyAsync(tl.p, order.data(), sizeof(int2) * order.size(),
                              cudaMemcpyHostToDevice, st));
  CUtensorMap ma, mb;
  XM_TRY(slice_map(&ma, S.p, K_pad, rows, OZ_BM));
  XM_TRY(slice_map(&mb, S.p, K_pad, rows, OZ_BN));
  OzArgs a{};
  a.tiles = tl.as<int2>();
  a.ntiles = (int)order.size();
  a.KB = KB;
  a.expA = sexp.as<int>();
  a.expB = sexp.as<int>();
  a.n = q.n;
  a.nt = nt;
  a.P = P;
  a.acc64 = acc64;
  a.q32 = q.q32;
  a.q16 = q.q16;
  a.err = ctx->d_err;
  XM_TRY(launch_mma<OZ_SYRK>(ctx, ma, mb, a));
  XM_CUDA_TRY(cudaStreamSynchronize(st));       // the order vector and buffers die here
  return check_device_error(ctx, "split-BF16 rank-k update");
}

// Inverses of the 128 x 128 diagonal leaves of a lower-triangular m x m matrix L (column-major,
// leading dimension ldl; leaf g covers rows and columns [128 g, 128 g + h), h = min(128, m - 128 g)),
// written into the diagonal blocks of Li: block j (b x b, column-major, leading dimension b, b a
// multiple of 128) holds rows and columns [j b, j b + b).  Thread c forward-substitutes
// L_leaf x = e_c for column c of the inverse, keeping the column in shared memory; the loop over
// l is the same for every thread (entries above the diagonal are zero), so all threads read the
// same entry of L at a time.
constexpr int OZ_LEAF = 128;
__global__ void __launch_bounds__(OZ_LEAF) k_oz_trinv_leaf(const double* __restrict__ L, int ldl,
                                                          double* __restrict__ Li, int b, int m) {
  extern __shared__ double xs[];                        // [OZ_LEAF rows][OZ_LEAF columns]
  const int j0 = blockIdx.x * OZ_LEAF, h = min(OZ_LEAF, m - j0);
  const int c = threadIdx.x;
  for (int k = 0; k < h; ++k) {
    const double* Lk = L + (size_t)(j0 + k) + (size_t)j0 * ldl;   // L[j0 + k, j0 + l] = Lk[l ldl]
    double s = k == c ? 1.0 : 0.0;
    for (int l = 0; l < k; ++l) s -= Lk[(size_t)l * ldl] * xs[l * OZ_LEAF + c];
    xs[k * OZ_LEAF + c] = k < c ? 0.0 : s / Lk[(size_t)k * ldl];
  }
  const int blk = j0 / b, off = j0 - blk * b;
  double* dst = Li + (size_t)blk * b * b + off + (size_t)off * b;
  if (c < h)
    for (int k = 0; k < h; ++k) dst[k + (size_t)c * b] = xs[k * OZ_LEAF + c];
}

__global__ void k_oz_negate(double* __restrict__ v, size_t count) {
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < count;
       g += (size_t)gridDim.x * blockDim.x)
    v[g] = -v[g];
}

// -L_jj^{-1} of the diagonal blocks of the lower-triangular m x m matrix L (blocks of b rows, b a
// multiple of 128; the last one m - (nb - 1) b) into Li (nb blocks of b x b, column-major,
// leading dimension b, zeros above the diagonal).  The 128 x 128 leaves are inverted by
// k_oz_trinv_leaf; then, leaf row by leaf row, X_ik = -L_ii^{-1} sum_{k <= l < i} L_il X_lk
// (FP64 cuBLAS products, 7 GFLOP at 10 blocks of 1024).  The batched library triangular solve
// this replaces cost 0.9-1.5 s at its first call in a process on a fresh B300 machine.
static xm_status tri_inverse_blocks(xm_ctx* ctx, const double* L, int ldl, int m, int b, double* Li) {
  cudaStream_t st = ctx->stream;
  const int nb = (m + b - 1) / b;
  {
    constexpr int MAX_DEVICES = 64;
    static std::mutex mu;
    static bool configured[MAX_DEVICES] = {};
    if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
      return set_error(XM_EINVAL, "triangular inverse: device %d out of range", ctx->device);
    std::lock_guard<std::mutex> lock(mu);
    if (!configured[ctx->device]) {
      XM_CUDA_TRY(cudaFuncSetAttribute(k_oz_trinv_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * OZ_LEAF * OZ_LEAF)));
      configured[ctx->device] = true;
    }
  }
  XM_CUDA_TRY(cudaMemsetAsync(Li, 0, sizeof(double) * (size_t)nb * b * b, st));
  k_oz_trinv_leaf<<<(m + OZ_LEAF - 1) / OZ_LEAF, OZ_LEAF, sizeof(double) * OZ_LEAF * OZ_LEAF, st>>>(
      L, ldl, Li, b, m);
  XM_CUDA_TRY(cudaGetLastError());
  DevMem T;
  XM_CUDA_TRY(cudaMalloc(&T.p, sizeof(double) * (size_t)OZ_LEAF * b));
  for (int j = 0; j < nb; ++j) {
    const int o = j * b, bj = std::min(b, m - o);
    const double* Ljj = L + (size_t)o + (size_t)o * ldl;
    double* X = Li + (size_t)j * b * b;
    for (int r0 = OZ_LEAF; r0 < bj; r0 += OZ_LEAF) {
      const int hi = std::min(OZ_LEAF, bj - r0);
      // T = L[r0:r0+hi, 0:r0] X[0:r0, 0:r0]; X[r0:r0+hi, 0:r0] = -X[r0:, r0:] T
      XM_TRY(dense_gemm(ctx, false, false, false, hi, r0, r0, 1.0, Ljj + r0, ldl, X, b, 0.0,
                        T.as<double>(), OZ_LEAF, nullptr));
      XM_TRY(dense_gemm(ctx, false, false, false, hi, r0, hi, -1.0, X + r0 + (size_t)r0 * b, b,
                        T.as<double>(), OZ_LEAF, 0.0, X + r0, b, nullptr));
    }
  }
  k_oz_negate<<<ctx->num_sms * 4, 256, 0, st>>>(Li, (size_t)nb * b * b);
  XM_CUDA_TRY(cudaGetLastError());
  // T is freed on return: the products above must have read it
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  return XM_OK;
}

// X <- L^{-1} X for L lower triangular m x m (column-major, leading dimension ldl) and X m x n
// (column-major, leading dimension ldx): right-looking blocked forward substitution in blocks of
// 1024 rows, every product on the tensor cores.  The inverses -L_ii^{-1} of the diagonal blocks
// are formed first in FP64 (tri_inverse_blocks: 7 GFLOP at m = 10154, where solving the n
// right-hand sides by substitution costs m 1024 n = 320 GFLOP at the FP64 rate); each step is then X_i <- L_ii^{-1} X_i as X_i = 0 - (-L_ii^{-1}) X_i (its digits taken
// before X_i is cleared) and the block update X_rest -= L_rest,i X_i.  Multiplying by a
// triangular inverse formed by substitution has the componentwise error bound of substitution.
// Blocks of 1024 rather than 512 halve the FP64 level folds per tensor-core flop of the block
// updates (10154 x 30465: 0.70 -> 0.63 s for the whole update; 2048 is no faster and its
// difference from the FP64 build is 3x larger).
xm_status split_trsm(xm_ctx* ctx, const double* L, int ldl, double* X, int ldx, int m, int n) {
  cudaStream_t st = ctx->stream;
  const int b = OZ_TRSM_BLOCK;                               // a multiple of OZ_BM and OZ_BK
  const int K_pad = b;
  const int nb = (m + b - 1) / b;
  const int nJ = (n + OZ_BN - 1) / OZ_BN;
  const int rowsB = nJ * OZ_BN;
  const int rowsA_max = ((std::max(m - b, b) + OZ_BM - 1) / OZ_BM) * OZ_BM;
  DevMem SA, SB, scA, scB, tl, tld, Li;
  XM_CUDA_TRY(cudaMalloc(&SA.p, sizeof(__nv_bfloat16) * (size_t)OZ_SLICES * rowsA_max * K_pad));
  XM_CUDA_TRY(cudaMalloc(&SB.p, sizeof(__nv_bfloat16) * (size_t)OZ_SLICES * rowsB * K_pad));
  XM_CUDA_TRY(cudaMalloc(&scA.p, sizeof(int) * (size_t)rowsA_max));
  XM_CUDA_TRY(cudaMalloc(&scB.p, sizeof(int) * (size_t)rowsB));
  const int nI_max = rowsA_max / OZ_BM;
  XM_CUDA_TRY(cudaMalloc(&tl.p, sizeof(int2) * (size_t)nI_max * nJ));
  XM_CUDA_TRY(cudaMalloc(&tld.p, sizeof(int2) * (size_t)(b / OZ_BM) * nJ));

  // -L_jj^{-1} for every diagonal block (FP64, column-major b x b each)
  XM_CUDA_TRY(cudaMalloc(&Li.p, sizeof(double) * (size_t)nb * b * b));
  XM_TRY(tri_inverse_blocks(ctx, L, ldl, m, b, Li.as<double>()));

  auto gemm = [&](const int2* tiles, const std::vector<int2>& order, int rowsA, int KB,
                  double* out, int M) -> xm_status {
    CUtensorMap ma, mb;
    XM_TRY(slice_map(&ma, SA.p, K_pad, rowsA, OZ_BM));
    XM_TRY(slice_map(&mb, SB.p, K_pad, rowsB, OZ_BN));
    OzArgs a{};
    a.tiles = tiles;
    a.ntiles = (int)order.size();
    a.KB = KB;
    a.expA = scA.as<int>();
    a.expB = scB.as<int>();
    a.out = out;
    a.ldo = ldx;
    a.M = M;
    a.ncols = n;
    a.err = ctx->d_err;
    return launch_mma<OZ_GEMM>(ctx, ma, mb, a);
  };
  std::vector<int2> order_d, order;
  for (int i0 = 0, blk = 0; i0 < m; i0 += b, ++blk) {
    const int bi = std::min(b, m - i0);
    const int KB = (bi + OZ_BK - 1) / OZ_BK;
    const size_t strideB = (size_t)rowsB * K_pad;
    // X_i <- L_ii^{-1} X_i: digits of the rows of -L_ii^{-1} and of the columns of X_i, X_i
    // cleared, then X_i -= (-L_ii^{-1}) X_i
    const int rowsD = ((bi + OZ_BM - 1) / OZ_BM) * OZ_BM;
    k_oz_split_rows<<<split_grid(ctx, rowsD, 128), 128, 0, st>>>(
        Li.as<double>() + (size_t)blk * b * b, b, bi, bi, rowsD, K_pad, SA.as<__nv_bfloat16>(),
        (size_t)rowsD * K_pad, scA.as<int>());
    k_oz_split_cols<<<split_grid(ctx, rowsB, 8), 256, 0, st>>>(
        X + i0, ldx, bi, n, rowsB, K_pad, SB.as<__nv_bfloat16>(), strideB, scB.as<int>());
    XM_CUDA_TRY(cudaGetLastError());
    XM_CUDA_TRY(cudaMemset2DAsync(X + i0, sizeof(double) * (size_t)ldx, 0, sizeof(double) * (size_t)bi,
                                  (size_t)n, st));
    order_d = tile_order(rowsD / OZ_BM, nJ, [](int, int) { return true; });
    XM_CUDA_TRY(cudaMemcpyAsync(tld.p, order_d.data(), sizeof(int2) * order_d.size(),
                                cudaMemcpyHostToDevice, st));
    XM_TRY(gemm(tld.as<int2>(), order_d, rowsD, KB, X + i0, bi));
    const int rest = m - i0 - bi;
    if (rest == 0) break;
    // X_rest -= L_rest,i X_i
    const int rowsA = ((rest + OZ_BM - 1) / OZ_BM) * OZ_BM;
    k_oz_split_rows<<<split_grid(ctx, rowsA, 128), 128, 0, st>>>(
        L + (i0 + bi) + (size_t)i0 * ldl, ldl, bi, rest, rowsA, K_pad, SA.as<__nv_bfloat16>(),
        (size_t)rowsA * K_pad, scA.as<int>());
    k_oz_split_cols<<<split_grid(ctx, rowsB, 8), 256, 0, st>>>(
        X + i0, ldx, bi, n, rowsB, K_pad, SB.as<__nv_bfloat16>(), strideB, scB.as<int>());
    XM_CUDA_TRY(cudaGetLastError());
    order = tile_order(rowsA / OZ_BM, nJ, [](int, int) { return true; });
    XM_CUDA_TRY(cudaMemcpyAsync(tl.p, order.data(), sizeof(int2) * order.size(),
                                cudaMemcpyHostToDevice, st));
    XM_TRY(gemm(tl.as<int2>(), order, rowsA, KB, X + i0 + bi, rest));
    // the host order vectors are reused next step: their copies must have been consumed
    XM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return check_device_error(ctx, "split-BF16 triangular solve");
}

}  // namespace xm

namespace xm {

// In-place Cholesky factor of the m x m SPD matrix A (column-major, leading dimension lda, lower
// triangle used and overwritten by L): right-looking, blocks of OZ_CHOL_BLOCK (256); the
// diagonal blocks by dense_potrf and the panels by substitution (dense_trsm_right_lower_t), both
// this library's FP64 kernels, the trailing updates A_rest -= L_k L_k^T on the tensor cores (only
// the tiles that meet the lower triangle).  (Panels as products with explicit inverses of the
// diagonal blocks doubled the build's difference from the FP64 build at 1500 cameras, to 2.1e-11
// of max |Q|.  256-row blocks halve the panels' substitution work and chains against 512 for a
// few more level folds of the updates: 10155-camera build 0.667 -> 0.648 s.)
// *minor = 0 on success, else the 1-based order of the first non-positive leading minor.
xm_status split_potrf(xm_ctx* ctx, double* A, int lda, int m, int* minor) {
  cudaStream_t st = ctx->stream;
  const int b = OZ_CHOL_BLOCK;
  const int K_pad = b;
  *minor = 0;
  const int rows_max = ((std::max(m - b, 1) + OZ_BN - 1) / OZ_BN) * OZ_BN;   // boxes of 128 and 256 rows
  DevMem fail, S, sc, tl;
  XM_CUDA_TRY(cudaMalloc(&fail.p, sizeof(int)));
  XM_CUDA_TRY(cudaMemsetAsync(fail.p, 0, sizeof(int), st));
  XM_CUDA_TRY(cudaMalloc(&S.p, sizeof(__nv_bfloat16) * (size_t)OZ_SLICES * rows_max * K_pad));
  XM_CUDA_TRY(cudaMalloc(&sc.p, sizeof(int) * (size_t)rows_max));
  XM_CUDA_TRY(cudaMalloc(&tl.p, sizeof(int2) * (size_t)(rows_max / OZ_BM) * (rows_max / OZ_BN)));
  std::vector<int2> order;
  for (int k0 = 0; k0 < m; k0 += b) {
    const int bk = std::min(b, m - k0);
    double* Akk = A + k0 + (size_t)k0 * lda;
    // FP64 diagonal block (own blocked factor) and its panel (own substitution)
    int h = 0;
    XM_TRY(dense_potrf(ctx, Akk, lda, bk, fail.as<int>(), &h));
    if (h != 0) { *minor = h + k0; return XM_OK; }
    const int rest = m - k0 - bk;
    if (rest == 0) break;
    double* P = A + (k0 + bk) + (size_t)k0 * lda;              // panel, rest x bk
    XM_TRY(dense_trsm_right_lower_t(ctx, Akk, lda, P, lda, rest, bk, nullptr));
    const int rows = ((rest + OZ_BN - 1) / OZ_BN) * OZ_BN;
    const size_t stride = (size_t)rows * K_pad;
    const int nI = (rest + OZ_BM - 1) / OZ_BM, nJ = (rest + OZ_BN - 1) / OZ_BN;
    k_oz_split_rows<<<split_grid(ctx, rows, 128), 128, 0, st>>>(P, lda, bk, rest, rows, K_pad,
                                                               S.as<__nv_bfloat16>(), stride,
                                                               sc.as<int>());
    XM_CUDA_TRY(cudaGetLastError());
    // 128 x 256 tiles with some column <= some row (they meet the lower triangle)
    order = tile_order(nI, nJ, [](int I, int J) { return J * OZ_BN <= I * OZ_BM + OZ_BM - 1; });
    XM_CUDA_TRY(cudaMemcpyAsync(tl.p, order.data(), sizeof(int2) * order.size(),
                                cudaMemcpyHostToDevice, st));
    CUtensorMap ma, mb;
    XM_TRY(slice_map(&ma, S.p, K_pad, rows, OZ_BM));
    XM_TRY(slice_map(&mb, S.p, K_pad, rows, OZ_BN));
    OzArgs a{};
    a.tiles = tl.as<int2>();
    a.ntiles = (int)order.size();
    a.KB = (bk + OZ_BK - 1) / OZ_BK;
    a.expA = sc.as<int>();
    a.expB = sc.as<int>();
    a.out = A + (k0 + bk) + (size_t)(k0 + bk) * lda;
    a.ldo = lda;
    a.M = rest;
    a.ncols = rest;
    a.err = ctx->d_err;
    XM_TRY(launch_mma<OZ_GEMM>(ctx, ma, mb, a));
    // the host order vectors are reused next step
    XM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return check_device_error(ctx, "split-BF16 Cholesky factor");
}

}  // namespace xm
