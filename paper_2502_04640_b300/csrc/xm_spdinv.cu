// Inverse of a dense symmetric positive definite FP32 matrix, with every O(n^3) step on the BF16
// tensor cores (tcgen05).  Used for the adjoint's preconditioner (Z + gamma Pi_Y)^{-1}, whose
// explicit inverse is applied by the packed Q.Y sweep once per CG step; exported as
// xm_spd_inverse.
//
// Algorithm: block inversion by Schur complements.  With A = [A11 A21^T; A21 A22] (A11 k x k,
// k a multiple of 128 near n / 2):
//   X = A11^{-1} (recursively), T = A21 X, S = A22 - T A21^T, Y = S^{-1} (recursively),
//   U = -Y T = (A^{-1})_21,  (A^{-1})_11 = X - T^T U,  (A^{-1})_12 = U^T.
// Every Schur complement of an SPD matrix is SPD, so no pivoting is needed.  The recursion ends
// at blocks of at most 128 rows, inverted in shared memory by Gauss–Jordan elimination (one CTA
// per block).  Flops: n^3 / 2 multiply-adds with the symmetric products computed on
// their lower triangle only, the same count as a Cholesky factorisation followed by the inverse
// of its factor.
//
// The four products per level are GEMMs C = alpha L R + beta C on FP32 data.  Each operand entry
// x is split into three BF16 digits x = d0 + d1 + d2 + e (each digit the round-to-nearest BF16 of
// what the previous ones left, |e| <= 2^-27 |x|); the products d_a(l) d_b(r) with a + b <= 2
// (six of nine) are exact in FP32 and accumulate in FP32 in tensor memory, so a product entry
// carries an error of about 3 * 2^-27 sum |l||r| beside the FP32 accumulation's own rounding:
// the accuracy of an FP32 GEMM.
//
// GEMM kernel: persistent, one CTA per SM, 128 x 256 output tiles (MMA M = 128, N = 256), tiles
// in groups of 8 tile rows taken column by column (concurrent CTAs share operand k-blocks in L2).
// Warp 0 streams, per k-block of 64, the three digit boxes of the 128-row A block (one 48 KB
// unit, 2-slot ring) and the three 256-row B digit boxes (32 KB each, 4-slot ring) with TMA;
// one thread of warp 1 issues the six digit products (4 MMAs of K = 16 each) into one of two
// 256-column TMEM accumulators, releasing each B digit after its last use (B0 after A0, A1,
// A2; B1 after A0, A1; B2 after A0) and the A unit after all; warps 2..17 read a finished tile
// with tcgen05.ld and write alpha acc + beta C (FP32, column-major).  Every wait is bounded; a
// stalled pipeline raises DEV_TIMEOUT, drains its copies and frees tensor memory.
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <mutex>

#include "xm_internal.cuh"
#include "xm_tc.cuh"

namespace xm {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {

constexpr int SI_BM = 128;                   // tile rows (MMA M)
constexpr int SI_BN = 256;                   // tile columns (MMA N)
constexpr int SI_BK = 64;                    // k-block: one 128-byte swizzled row of BF16
constexpr int SI_DIG = 3;                    // BF16 digits per FP32 entry
constexpr int SI_ASTAGES = 2;                // A units (three digit boxes each) in flight
constexpr int SI_BSTAGES = 4;                // B digit boxes in flight
constexpr int SI_ACC = 2;                    // TMEM accumulators (2 x 256 columns)
constexpr int SI_EPI_WARPS = 16;
constexpr int SI_THREADS = 32 * (2 + SI_EPI_WARPS);
constexpr int SI_EPI_COLS = 64;              // accumulator columns per epilogue warp
constexpr uint32_t SI_A_BYTES = SI_BM * SI_BK * 2;              // one A digit box, 16 KB
constexpr uint32_t SI_AUNIT = SI_DIG * SI_A_BYTES;              // 48 KB
constexpr uint32_t SI_B_BYTES = SI_BN * SI_BK * 2;              // one B digit box, 32 KB
constexpr uint32_t SI_TMEM_COLS = SI_ACC * SI_BN;
constexpr size_t SI_SMEM = 1024 + (size_t)SI_ASTAGES * SI_AUNIT + (size_t)SI_BSTAGES * SI_B_BYTES + 256;
constexpr int SI_LEAF = 128;                 // largest block inverted directly
constexpr int SI_LEAF_LD = SI_LEAF + 4;      // shared-memory row stride of the leaf (floats)
constexpr size_t SI_LEAF_SMEM =              // block, column panel, row panel, D times it, D
    sizeof(float) * ((size_t)SI_LEAF * SI_LEAF_LD + SI_LEAF * 17 + 2 * 16 * SI_LEAF_LD + 16 * 20);
constexpr int SI_LEAF_THREADS = 512;

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, N = 256, M = 128
constexpr uint32_t SI_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(SI_BN >> 3) << 17) |
                              ((uint32_t)(SI_BM >> 4) << 24);

struct SiArgs {
  float* C;                 // output, column-major, C[row + col * ldc]
  int ldc, M, N;            // C is M x N
  float alpha, beta;        // C = alpha L R + beta C (beta == 0: C is not read)
  int KB;                   // k-blocks of 64
  int nI, nJ;               // 128-row and 256-column tile counts
  int lower;                // only tiles that meet the lower triangle (row >= col)
  int* err;
};

// work item w -> tile (I, J): groups of 8 tile rows, column by column within a group
__device__ __forceinline__ bool si_tile(const SiArgs& a, int w, int& I, int& J) {
  const int g = w / (8 * a.nJ);
  const int rem = w - g * 8 * a.nJ;
  const int gsz = min(8, a.nI - 8 * g);
  J = rem / gsz;
  I = 8 * g + (rem - J * gsz);
  return !a.lower || J * SI_BN <= I * SI_BM + SI_BM - 1;
}

__global__ void __launch_bounds__(SI_THREADS, 1)
k_si_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
          SiArgs args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sa_base = base;                                            // A units
  unsigned char* sb_base = base + (size_t)SI_ASTAGES * SI_AUNIT;            // B digit boxes
  uint64_t* bars = reinterpret_cast<uint64_t*>(sb_base + (size_t)SI_BSTAGES * SI_B_BYTES);
  uint64_t* afull = bars;                      // [SI_ASTAGES]
  uint64_t* aempty = afull + SI_ASTAGES;       // [SI_ASTAGES]
  uint64_t* bfull = aempty + SI_ASTAGES;       // [SI_BSTAGES]
  uint64_t* bempty = bfull + SI_BSTAGES;       // [SI_BSTAGES]
  uint64_t* accfull = bempty + SI_BSTAGES;     // [SI_ACC]
  uint64_t* accempty = accfull + SI_ACC;       // [SI_ACC]
  uint64_t* done = accempty + SI_ACC;          // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = args.nI * args.nJ;
  if (threadIdx.x == 0) {
    for (int s = 0; s < SI_ASTAGES; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&aempty[s], 1);
    }
    for (int s = 0; s < SI_BSTAGES; ++s) {
      mbar_init(&bfull[s], 1);
      mbar_init(&bempty[s], 1);
    }
    for (int b = 0; b < SI_ACC; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], SI_EPI_WARPS);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 1) tc::alloc(tmem_slot, SI_TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  const int KB = args.KB;

  if (warp == 0) {
    // ---------------- producer
    if (lane == 0) {
      int as = 0, bs = 0;
      uint32_t aph = 0, bph = 0;
      int64_t a_issued = 0, b_issued = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < total && ok; w += gridDim.x) {
        int I, J;
        if (!si_tile(args, w, I, J)) continue;
        for (int kb = 0; kb < KB && ok; ++kb) {
          if (!mbar_wait(&aempty[as], aph ^ 1u)) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
          mbar_arrive_expect_tx(&afull[as], SI_AUNIT);
          unsigned char* sa = sa_base + (size_t)as * SI_AUNIT;
#pragma unroll
          for (int d = 0; d < SI_DIG; ++d)
            tc::tma_load_3d(sa + d * SI_A_BYTES, &mapA, kb * SI_BK, I * SI_BM, d, &afull[as]);
          ++a_issued;
          if (++as == SI_ASTAGES) { as = 0; aph ^= 1u; }
          for (int d = 0; d < SI_DIG; ++d) {
            if (!mbar_wait(&bempty[bs], bph ^ 1u)) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
            mbar_arrive_expect_tx(&bfull[bs], SI_B_BYTES);
            tc::tma_load_3d(sb_base + (size_t)bs * SI_B_BYTES, &mapB, kb * SI_BK, J * SI_BN, d, &bfull[bs]);
            ++b_issued;
            if (++bs == SI_BSTAGES) { bs = 0; bph ^= 1u; }
          }
        }
      }
      // do not leave while copies into this CTA's shared memory are in flight
      for (int64_t k = a_issued > SI_ASTAGES ? a_issued - SI_ASTAGES : 0; k < a_issued; ++k)
        if (!mbar_wait(&afull[k % SI_ASTAGES], (uint32_t)((k / SI_ASTAGES) & 1))) { atomicOr(args.err, DEV_TIMEOUT); break; }
      for (int64_t k = b_issued > SI_BSTAGES ? b_issued - SI_BSTAGES : 0; k < b_issued; ++k)
        if (!mbar_wait(&bfull[k % SI_BSTAGES], (uint32_t)((k / SI_BSTAGES) & 1))) { atomicOr(args.err, DEV_TIMEOUT); break; }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int as = 0, bs = 0;
      uint32_t aph = 0, bph = 0;
      int64_t tcount = 0;
      bool ok = true;
      const uint32_t sa0 = smem_u32(sa_base), sb0 = smem_u32(sb_base);
      for (int w = blockIdx.x; w < total && ok; w += gridDim.x) {
        int I, J;
        if (!si_tile(args, w, I, J)) continue;
        const int buf = (int)(tcount & 1);
        if (!mbar_wait(&accempty[buf], (uint32_t)(((tcount >> 1) & 1) ^ 1))) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
        tc::fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * SI_BN);
        for (int kb = 0; kb < KB && ok; ++kb) {
          if (!mbar_wait(&afull[as], aph)) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
          tc::fence_after();
          const uint32_t sa = sa0 + (uint32_t)as * SI_AUNIT;
          for (int b = 0; b < SI_DIG; ++b) {
            if (!mbar_wait(&bfull[bs], bph)) { atomicOr(args.err, DEV_TIMEOUT); ok = false; break; }
            tc::fence_after();
            const uint64_t db = tc::kmajor_desc(sb0 + (uint32_t)bs * SI_B_BYTES);
            for (int a = 0; a + b < SI_DIG; ++a) {   // digit products of order a + b <= 2
              const uint64_t da = tc::kmajor_desc(sa + (uint32_t)a * SI_A_BYTES);
#pragma unroll
              for (int j = 0; j < SI_BK / 16; ++j)   // K = 16 per MMA: 32 bytes along the row
                tc::mma_f16(dt, da + 2 * j, db + 2 * j, SI_IDESC,
                            (kb > 0 || b > 0 || a > 0 || j > 0) ? 1u : 0u);
            }
            tc::commit(&bempty[bs]);
            if (++bs == SI_BSTAGES) { bs = 0; bph ^= 1u; }
          }
          tc::commit(&aempty[as]);
          if (++as == SI_ASTAGES) { as = 0; aph ^= 1u; }
        }
        if (!ok) break;
        tc::commit(&accfull[buf]);
        ++tcount;
      }
      // every issued MMA complete before tensor memory is freed
      tc::commit(done);
      if (!mbar_wait(done, 0)) atomicOr(args.err, DEV_TIMEOUT);
    }
  } else {
    // ---------------- epilogue: warps 2..17, TMEM lane quarter warp % 4, 64 columns each
    const int quarter = warp & 3;
    const int grp = (warp - 2) >> 2;
    const int a_loc = 32 * quarter + lane;
    int64_t tcount = 0;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
      int I, J;
      if (!si_tile(args, w, I, J)) continue;
      const int buf = (int)(tcount & 1);
      if (!mbar_wait(&accfull[buf], (uint32_t)((tcount >> 1) & 1))) { atomicOr(args.err, DEV_TIMEOUT); break; }
      tc::fence_after();
      float v[SI_EPI_COLS];
      const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * SI_BN + grp * SI_EPI_COLS);
#pragma unroll
      for (int p = 0; p < SI_EPI_COLS / 16; ++p) {
        float u[16];
        tc::ld16(ta + 16 * p, u);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[16 * p + i] = u[i];
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[buf]);
      ++tcount;
      const int row = I * SI_BM + a_loc;
      const int col0 = J * SI_BN + grp * SI_EPI_COLS;
      if (row < args.M) {
        const float al = args.alpha, be = args.beta;
#pragma unroll
        for (int c = 0; c < SI_EPI_COLS; ++c) {
          const int col = col0 + c;
          if (col < args.N) {
            float* o = args.C + (size_t)col * args.ldc + row;   // coalesced along rows
            *o = be != 0.f ? fmaf(al, v[c], be * *o) : al * v[c];
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 1) tc::dealloc(tmem, SI_TMEM_COLS);
}

// ------------------------------------------------------------------ digit split
// three BF16 digits of x: d0 = bf16(x), d1 = bf16(x - d0), d2 = bf16(x - d0 - d1) (the
// differences are exact in FP32)
__device__ __forceinline__ void digits3(float x, float (&d)[SI_DIG]) {
  float r = x;
#pragma unroll
  for (int s = 0; s < SI_DIG; ++s) {
    d[s] = __bfloat162float(__float2bfloat16_rn(r));
    r -= d[s];
  }
}
__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
  const __nv_bfloat162 p = __halves2bfloat162(__float2bfloat16_rn(lo), __float2bfloat16_rn(hi));
  return *reinterpret_cast<const uint32_t*>(&p);
}

// S[d][v][k] (d < 3, v < rows, k < K_pad; BF16, K-major) = digit d of X(v, k) = src[v vs + k ks]
// for v < nv and k < K, zero elsewhere.  A block transposes a 64 x 64 tile through shared memory
// so that the reads are coalesced along whichever of v and k has unit stride.
__global__ void __launch_bounds__(256) k_si_split(const float* __restrict__ src, int64_t vs, int64_t ks,
                                                   int nv, int K, int K_pad, size_t slice,
                                                   __nv_bfloat16* __restrict__ S) {
  __shared__ float t[64][65];
  const int v0 = blockIdx.x * 64, k0 = blockIdx.y * 64;
  const bool kfast = ks == 1;
  for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
    const int vl = kfast ? (idx >> 6) : (idx & 63);
    const int kl = kfast ? (idx & 63) : (idx >> 6);
    const int v = v0 + vl, k = k0 + kl;
    t[vl][kl] = (v < nv && k < K) ? src[(int64_t)v * vs + (int64_t)k * ks] : 0.f;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 64 * 8; idx += 256) {
    const int vl = idx >> 3, c = idx & 7;
    uint32_t w[SI_DIG][4];
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      float a[SI_DIG], b[SI_DIG];
      digits3(t[vl][8 * c + j], a);
      digits3(t[vl][8 * c + j + 1], b);
#pragma unroll
      for (int s = 0; s < SI_DIG; ++s) w[s][j / 2] = bf16_pair(a[s], b[s]);
    }
    const size_t off = (size_t)(v0 + vl) * K_pad + k0 + 8 * c;
#pragma unroll
    for (int s = 0; s < SI_DIG; ++s)
      *reinterpret_cast<uint4*>(S + (size_t)s * slice + off) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  }
}

// ------------------------------------------------------------------ leaves and transposes
// In-place inverse of an SPD m x m block (m <= 128; column-major FP32, leading dimension lda,
// both triangles valid) by blocked Gauss–Jordan elimination in FP32 in shared memory, without
// pivoting (every pivot block is a diagonal block of a Schur complement of the SPD matrix,
// hence SPD).  The block is padded to 128 x 128 with the identity.  Eliminating the 16 pivots of
// block K at once, with D = A_KK^{-1}:
//   A_KK <- D,  A_KR <- D A_KR,  A_RK <- -A_RK D,  A_RR <- A_RR - A_RK (D A_KR)
// (R: every index outside K; the single-pivot step is the case |K| = 1).  D comes from
// single-pivot steps on the 16 x 16 block by one warp; the rank-16 update runs on all threads,
// thread t owning rows 4 (t / 16) .. + 3 and columns 8 (t % 16) .. + 7 (one 4-row group and one
// 8-column group lie wholly inside or outside K).  FP32 like the products around it (an FP64
// version took 2 ms per block on B300's FP64 units, the unblocked FP32 one 0.45 ms).  A pivot
// of D that is not positive and finite sets *fail and leaves the block unfinished.
constexpr int SI_LB = 16;                     // pivots eliminated together
constexpr int SI_DLD = 20;                    // row stride of D (16-byte aligned rows)
static_assert(SI_LEAF_SMEM == sizeof(float) * ((size_t)SI_LEAF * SI_LEAF_LD + SI_LEAF * (SI_LB + 1) +
                                               2 * SI_LB * SI_LEAF_LD + SI_LB * SI_DLD),
              "leaf shared-memory layout");
__global__ void __launch_bounds__(SI_LEAF_THREADS) k_si_leaf(float* __restrict__ A, int lda, int m,
                                                             int* __restrict__ fail) {
  extern __shared__ float4 sm4[];
  float* s = reinterpret_cast<float*>(sm4);               // [128][SI_LEAF_LD]
  float* Cp = s + SI_LEAF * SI_LEAF_LD;                   // [128][SI_LB + 1]: old column panel
  float* Rp = Cp + SI_LEAF * (SI_LB + 1);                 // [SI_LB][SI_LEAF_LD]: old row panel
  float* Pp = Rp + SI_LB * SI_LEAF_LD;                    // [SI_LB][SI_LEAF_LD]: D times Rp
  float* Dm = Pp + SI_LB * SI_LEAF_LD;                    // [SI_LB][SI_DLD]
  __shared__ int bad;
  const int t = threadIdx.x;
  for (int e = t; e < SI_LEAF * SI_LEAF; e += blockDim.x) {
    const int i = e & (SI_LEAF - 1), j = e >> 7;         // coalesced along i
    s[i * SI_LEAF_LD + j] = (i < m && j < m) ? A[i + (size_t)j * lda] : (i == j ? 1.f : 0.f);
  }
  if (t == 0) bad = 0;
  __syncthreads();
  const int i0 = 4 * (t >> 4), j0 = 8 * (t & 15);
  for (int p0 = 0; p0 < SI_LEAF; p0 += SI_LB) {
    // old panels: columns K of every row, rows K of every column
    for (int e = t; e < SI_LEAF * SI_LB; e += blockDim.x) {
      const int i = e >> 4, l = e & (SI_LB - 1);
      Cp[i * (SI_LB + 1) + l] = s[i * SI_LEAF_LD + p0 + l];
      const int l2 = e >> 7, j = e & (SI_LEAF - 1);
      Rp[l2 * SI_LEAF_LD + j] = s[(p0 + l2) * SI_LEAF_LD + j];
    }
    __syncthreads();
    if (t < 32) {
      // D = A_KK^{-1}: lane t owns row t / 2, columns 8 (t % 2) .. + 7
      const int a = t >> 1, b0 = 8 * (t & 1);
      for (int k = 0; k < 8; ++k) Dm[a * SI_DLD + b0 + k] = Rp[a * SI_LEAF_LD + p0 + b0 + k];
      __syncwarp();
      for (int q = 0; q < SI_LB; ++q) {
        const float piv = Dm[q * SI_DLD + q];
        if (!(piv > 0.f && piv < 3.0e38f)) {           // the same decision in every lane
          if (t == 0) bad = 1;
          break;
        }
        const float inv = 1.f / piv;
        const float cq = Dm[a * SI_DLD + q];
        float rq[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) rq[k] = Dm[q * SI_DLD + b0 + k];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int b = b0 + k;
          float v;
          if (a == q) v = b == q ? inv : rq[k] * inv;
          else if (b == q) v = -cq * inv;
          else v = fmaf(-cq, rq[k] * inv, Dm[a * SI_DLD + b]);
          Dm[a * SI_DLD + b] = v;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (bad) {
      if (t == 0) atomicOr(fail, 1);
      return;
    }
    // P = D Rp (16 x 128)
    for (int e = t; e < SI_LB * SI_LEAF; e += blockDim.x) {
      const int a = e >> 7, j = e & (SI_LEAF - 1);
      float acc = 0.f;
#pragma unroll
      for (int l = 0; l < SI_LB; ++l) acc = fmaf(Dm[a * SI_DLD + l], Rp[l * SI_LEAF_LD + j], acc);
      Pp[a * SI_LEAF_LD + j] = acc;
    }
    __syncthreads();
    // rank-16 update of this thread's 4 x 8 block
    const bool iK = i0 >= p0 && i0 < p0 + SI_LB, jK = j0 >= p0 && j0 < p0 + SI_LB;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + r;
      float acc[8];
      float4* dst = reinterpret_cast<float4*>(s + i * SI_LEAF_LD + j0);
      if (iK) {
        const float* src = jK ? Dm + (i - p0) * SI_DLD + (j0 - p0) : Pp + (i - p0) * SI_LEAF_LD + j0;
        const float4 u0 = *reinterpret_cast<const float4*>(src);
        const float4 u1 = *reinterpret_cast<const float4*>(src + 4);
        acc[0] = u0.x; acc[1] = u0.y; acc[2] = u0.z; acc[3] = u0.w;
        acc[4] = u1.x; acc[5] = u1.y; acc[6] = u1.z; acc[7] = u1.w;
      } else {
        if (jK) {
#pragma unroll
          for (int k = 0; k < 8; ++k) acc[k] = 0.f;
        } else {
          const float4 u0 = dst[0], u1 = dst[1];
          acc[0] = u0.x; acc[1] = u0.y; acc[2] = u0.z; acc[3] = u0.w;
          acc[4] = u1.x; acc[5] = u1.y; acc[6] = u1.z; acc[7] = u1.w;
        }
        const float* srow = jK ? Dm + (j0 - p0) : Pp + j0;
        const int sld = jK ? SI_DLD : SI_LEAF_LD;
#pragma unroll
        for (int l = 0; l < SI_LB; ++l) {
          const float c = Cp[i * (SI_LB + 1) + l];
          const float4 u0 = *reinterpret_cast<const float4*>(srow + l * sld);
          const float4 u1 = *reinterpret_cast<const float4*>(srow + l * sld + 4);
          acc[0] = fmaf(-c, u0.x, acc[0]); acc[1] = fmaf(-c, u0.y, acc[1]);
          acc[2] = fmaf(-c, u0.z, acc[2]); acc[3] = fmaf(-c, u0.w, acc[3]);
          acc[4] = fmaf(-c, u1.x, acc[4]); acc[5] = fmaf(-c, u1.y, acc[5]);
          acc[6] = fmaf(-c, u1.z, acc[6]); acc[7] = fmaf(-c, u1.w, acc[7]);
        }
      }
      dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
    __syncthreads();
  }
  // both triangles from the computed lower triangle (the elimination's rounding is not
  // symmetric; the inverse is)
  for (int e = t; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;
    A[r + (size_t)c * lda] = r >= c ? s[r * SI_LEAF_LD + c] : s[c * SI_LEAF_LD + r];
  }
}

// dst(j, i) = src(i, j) for i < m, j < n (column-major; dst = src^T).  strict_lower: only the
// entries with i > j, so that src == dst (a square block) copies its lower triangle onto its
// upper triangle.  32 x 32 tiles through shared memory.
__global__ void __launch_bounds__(256) k_si_transpose(const float* src, int lds, float* dst, int ldd,
                                                      int m, int n, int strict_lower) {
  __shared__ float t[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  if (strict_lower && i0 + 31 <= j0) return;          // no entry with i > j
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + tx, j = j0 + r;
    if (i < m && j < n) t[r][tx] = src[i + (size_t)j * lds];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + tx, i = i0 + r;
    if (i < m && j < n && (!strict_lower || i > j)) dst[j + (size_t)i * ldd] = t[tx][r];
  }
}

// ------------------------------------------------------------------ host side
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// 3-D map of digit slices S[3][rows][K_pad] (BF16), box of 64 k x box_rows rows x 1 digit
xm_status si_slice_map(CUtensorMap* map, void* S, int K_pad, int rows, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return set_error(XM_ECUDA, "cuTensorMapEncodeTiled unavailable");
  const cuuint64_t gdim[3] = {(cuuint64_t)K_pad, (cuuint64_t)rows, (cuuint64_t)SI_DIG};
  const cuuint64_t gstride[2] = {(cuuint64_t)K_pad * 2, (cuuint64_t)K_pad * 2 * (cuuint64_t)rows};
  const cuuint32_t box[3] = {SI_BK, box_rows, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, S, gdim, gstride, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return set_error(XM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  return XM_OK;
}

// one operand of a product: vector v, entry k at p[v vs + k ks]
struct Opnd {
  const float* p;
  int64_t vs, ks;
};

// Scratch of one inversion: the digit slices of the two operands of the current product and a
// stack of T blocks (T of a level stays live across the inversion of its Schur complement).
struct SiWork {
  __nv_bfloat16* SA = nullptr;
  __nv_bfloat16* SB = nullptr;
  size_t capA = 0, capB = 0;     // BF16 elements
  float* Tstack = nullptr;
  size_t capT = 0;               // floats
  int* fail = nullptr;
  long launches = 0;
  double flops = 0.0;            // FP32-equivalent multiply-add flops of the products (2 per MAC)
};

std::mutex g_si_mu;
bool g_si_configured[64] = {};

xm_status si_configure(xm_ctx* ctx) {
  if (ctx->device < 0 || ctx->device >= 64)
    return set_error(XM_EINVAL, "spd inverse: device %d out of range", ctx->device);
  std::lock_guard<std::mutex> lock(g_si_mu);
  if (g_si_configured[ctx->device]) return XM_OK;
  if (SI_SMEM > ctx->smem_optin)
    return set_error(XM_ECUDA, "spd inverse: needs %zu bytes of shared memory", SI_SMEM);
  XM_CUDA_TRY(cudaFuncSetAttribute(k_si_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SI_SMEM));
  XM_CUDA_TRY(cudaFuncSetAttribute(k_si_leaf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)SI_LEAF_SMEM));
  g_si_configured[ctx->device] = true;
  return XM_OK;
}

// C (M x N, column-major, ldc) = alpha L R + beta C with L's rows and R's columns given as
// operand vectors of length K; lower: only the tiles that meet C's lower triangle.
xm_status si_gemm(xm_ctx* ctx, SiWork& W, Opnd L, Opnd R, int M, int N, int K, float alpha, float beta,
                  float* C, int ldc, bool lower) {
  if (M <= 0 || N <= 0) return XM_OK;
  cudaStream_t st = ctx->stream;
  const int K_pad = (int)round_up(std::max(K, 1), SI_BK);
  const int rowsA = (int)round_up(M, SI_BM), rowsB = (int)round_up(N, SI_BN);
  const size_t sliceA = (size_t)rowsA * K_pad, sliceB = (size_t)rowsB * K_pad;
  if (SI_DIG * sliceA > W.capA || SI_DIG * sliceB > W.capB)
    return set_error(XM_ECUDA, "spd inverse: digit scratch too small (internal)");
  k_si_split<<<dim3(rowsA / 64, K_pad / 64), 256, 0, st>>>(L.p, L.vs, L.ks, M, K, K_pad, sliceA, W.SA);
  k_si_split<<<dim3(rowsB / 64, K_pad / 64), 256, 0, st>>>(R.p, R.vs, R.ks, N, K, K_pad, sliceB, W.SB);
  CUtensorMap ma, mb;
  XM_TRY(si_slice_map(&ma, W.SA, K_pad, rowsA, SI_BM));
  XM_TRY(si_slice_map(&mb, W.SB, K_pad, rowsB, SI_BN));
  SiArgs a{};
  a.C = C;
  a.ldc = ldc;
  a.M = M;
  a.N = N;
  a.alpha = alpha;
  a.beta = beta;
  a.KB = K_pad / SI_BK;
  a.nI = rowsA / SI_BM;
  a.nJ = rowsB / SI_BN;
  a.lower = lower ? 1 : 0;
  a.err = ctx->d_err;
  const int grid = std::min(ctx->num_sms, a.nI * a.nJ);
  k_si_gemm<<<grid, SI_THREADS, SI_SMEM, st>>>(ma, mb, a);
  XM_CUDA_TRY(cudaGetLastError());
  W.launches += 3;
  W.flops += 2.0 * M * (double)N * K * (lower ? 0.5 : 1.0);
  return XM_OK;
}

xm_status si_transpose(xm_ctx* ctx, SiWork& W, const float* src, int lds, float* dst, int ldd, int m, int n,
                       bool strict_lower) {
  if (m <= 0 || n <= 0) return XM_OK;
  k_si_transpose<<<dim3((m + 31) / 32, (n + 31) / 32), 256, 0, ctx->stream>>>(src, lds, dst, ldd, m, n,
                                                                               strict_lower ? 1 : 0);
  XM_CUDA_TRY(cudaGetLastError());
  ++W.launches;
  return XM_OK;
}

// split point of an n-row block: a multiple of 128 near n / 2
inline int si_split_point(int n) { return SI_LEAF * std::max(1, n / (2 * SI_LEAF)); }

// A (n x n, column-major, lda, both triangles) <- A^{-1}; T: this call's part of the T stack
xm_status si_inverse(xm_ctx* ctx, SiWork& W, float* A, int lda, int n, float* T) {
  if (n <= SI_LEAF) {
    k_si_leaf<<<1, SI_LEAF_THREADS, SI_LEAF_SMEM, ctx->stream>>>(A, lda, n, W.fail);
    XM_CUDA_TRY(cudaGetLastError());
    ++W.launches;
    return XM_OK;
  }
  const int k = si_split_point(n), m2 = n - k;
  float* A11 = A;
  float* A21 = A + k;
  float* A12 = A + (size_t)k * lda;
  float* A22 = A + k + (size_t)k * lda;
  if (T + (size_t)m2 * k > W.Tstack + W.capT) return set_error(XM_ECUDA, "spd inverse: T stack too small (internal)");
  const int ldt = m2;
  XM_TRY(si_inverse(ctx, W, A11, lda, k, T));                                   // X = A11^{-1}
  // T = A21 X
  XM_TRY(si_gemm(ctx, W, Opnd{A21, 1, lda}, Opnd{A11, lda, 1}, m2, k, k, 1.f, 0.f, T, ldt, false));
  // S = A22 - T A21^T (lower triangle), then its upper triangle
  XM_TRY(si_gemm(ctx, W, Opnd{T, 1, ldt}, Opnd{A21, 1, lda}, m2, m2, k, -1.f, 1.f, A22, lda, true));
  XM_TRY(si_transpose(ctx, W, A22, lda, A22, lda, m2, m2, true));
  XM_TRY(si_inverse(ctx, W, A22, lda, m2, T + (size_t)m2 * k));                 // Y = S^{-1}
  // (A^{-1})_21 = U = -Y T
  XM_TRY(si_gemm(ctx, W, Opnd{A22, 1, lda}, Opnd{T, ldt, 1}, m2, k, m2, -1.f, 0.f, A21, lda, false));
  // (A^{-1})_11 = X - T^T U (lower triangle), its upper triangle, (A^{-1})_12 = U^T
  XM_TRY(si_gemm(ctx, W, Opnd{T, ldt, 1}, Opnd{A21, lda, 1}, k, k, m2, -1.f, 1.f, A11, lda, true));
  XM_TRY(si_transpose(ctx, W, A11, lda, A11, lda, k, k, true));
  XM_TRY(si_transpose(ctx, W, A21, lda, A12, lda, m2, k, false));
  return XM_OK;
}

// T stack needed below an n-row block: this level's T (live while its Schur complement is
// inverted) on top of what that inversion needs, or what the inversion of A11 needs (before T
// exists), whichever is larger
size_t si_tstack(int n) {
  if (n <= SI_LEAF) return 0;
  const int k = si_split_point(n), m2 = n - k;
  return std::max(si_tstack(k), (size_t)m2 * k + si_tstack(m2));
}

struct Mem {
  void* p = nullptr;
  ~Mem() { if (p) cudaFree(p); }
};

}  // namespace

// In-place inverse of the SPD n x n FP32 matrix A (column-major, lda >= n, both triangles set).
// Synchronous.  XM_ENUMERIC when a leaf pivot is not positive (A not numerically positive
// definite); A is then undefined.  *gflop (optional): FP32-equivalent GFLOP of the products.
xm_status spd_inverse_f32(xm_ctx* ctx, float* A, int lda, int n, double* gflop) {
  if (n <= 0) return XM_OK;
  XM_TRY(si_configure(ctx));
  cudaStream_t st = ctx->stream;
  SiWork W;
  Mem mA, mB, mT, mF;
  if (n > SI_LEAF) {
    // the largest operands are those of the top level (the Schur branch is the larger half)
    const int k = si_split_point(n), m2 = n - k;
    const int64_t big = std::max(k, m2);
    W.capA = (size_t)SI_DIG * round_up(big, SI_BM) * round_up(big, SI_BK);
    W.capB = (size_t)SI_DIG * round_up(big, SI_BN) * round_up(big, SI_BK);
    W.capT = si_tstack(n);
    XM_CUDA_TRY(cudaMalloc(&mA.p, sizeof(__nv_bfloat16) * W.capA));
    XM_CUDA_TRY(cudaMalloc(&mB.p, sizeof(__nv_bfloat16) * W.capB));
    XM_CUDA_TRY(cudaMalloc(&mT.p, sizeof(float) * W.capT));
    W.SA = static_cast<__nv_bfloat16*>(mA.p);
    W.SB = static_cast<__nv_bfloat16*>(mB.p);
    W.Tstack = static_cast<float*>(mT.p);
  }
  XM_CUDA_TRY(cudaMalloc(&mF.p, sizeof(int)));
  W.fail = static_cast<int*>(mF.p);
  XM_CUDA_TRY(cudaMemsetAsync(W.fail, 0, sizeof(int), st));
  XM_TRY(si_inverse(ctx, W, A, lda, n, W.Tstack));
  int hfail = 0;
  XM_CUDA_TRY(cudaMemcpyAsync(&hfail, W.fail, sizeof(int), cudaMemcpyDeviceToHost, st));
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  XM_TRY(check_device_error(ctx, "spd inverse"));
  if (gflop) *gflop = W.flops * 1e-9;
  g_last_launches = W.launches;
  if (hfail) return set_error(XM_ENUMERIC, "spd inverse: matrix not numerically positive definite");
  return XM_OK;
}

}  // namespace xm

extern "C" xm_status xm_spd_inverse(xm_ctx* ctx, int n, float* A, int lda) {
  if (!ctx) return xm::set_error(XM_EINVAL, "xm_spd_inverse: null context");
  if (n < 0 || (n > 0 && (!A || lda < n)))
    return xm::set_error(XM_EINVAL, "xm_spd_inverse: bad arguments (n = %d, lda = %d)", n, lda);
  XM_CUDA_TRY(cudaSetDevice(ctx->device));
  return xm::spd_inverse_f32(ctx, A, lda, n, nullptr);
}
