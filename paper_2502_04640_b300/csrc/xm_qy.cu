// Q.Y sweep on the packed symmetric tile layout (the Euclidean Hessian-vector product of
// Sec. 3.2: "matrix-vector multiplication"; one sweep also gives the gradient 2QY and the
// objective tr(Y^T Q Y) of Eq. 17).
//
// B300 design: Q is dense (a Schur complement through the inverse of a connected Laplacian,
// App. A), so each unique entry must be read once per sweep and the kernel is HBM-bound for
// FP32/BF16 storage.  Storing only the upper-triangle tiles halves the bytes; every tile is
// then used twice, T Y_J -> W_I (row contribution) and T^T Y_I -> W_J (column contribution).
//   * persistent grid, one CTA per SM, contiguous ranges of the tile list per CTA;
//   * one producer thread streams 16 KB slabs with cp.async.bulk (TMA engine) into a ring of
//     mbarrier-guarded stages (bounded waits: a stall sets DEV_TIMEOUT, no wait is endless);
//   * NW consumer warps: lane l owns columns 4l..4l+3 of the tile, keeps Y_J for them in
//     registers and accumulates the column contribution; the row contribution of each slab
//     row is reduced across lanes with a transpose-reduce butterfly and accumulated per
//     tile row in registers;
//   * the producer also bulk-copies Y_J of every tile into a 4-slot ring, so no consumer waits
//     on a global load; each warp adds its column partials to W_J with vector reductions (no
//     barrier between warps inside a tile row); row partials are kept per tile row in registers
//     (FP32/BF16, R = 4) and reduced across lanes once per tile row.
#include <cuda.h>
#include <cstring>
#include <mutex>
#include <cudaTypedefs.h>

#include "xm_internal.cuh"

namespace xm {

template <typename TQ> struct QT;
template <> struct QT<float> {
  using A = float;
  static constexpr int ROWS = SLAB_BYTES / (TILE * 4);   // 32 rows per slab
};
template <> struct QT<double> {
  using A = double;
  static constexpr int ROWS = SLAB_BYTES / (TILE * 8);   // 16
};

// four consecutive stored Q values of a slab row -> accumulation type
__device__ __forceinline__ void load4(const float* p, float (&q)[4]) {
  float4 v = *reinterpret_cast<const float4*>(p);
  q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double (&q)[4]) {
  double2 a = *reinterpret_cast<const double2*>(p);
  double2 b = *reinterpret_cast<const double2*>(p + 2);
  q[0] = a.x; q[1] = a.y; q[2] = b.x; q[3] = b.y;
}

// Packed FP32 pair arithmetic (fma.rn.f32x2, sm_100 and later): two FMAs per instruction.
__device__ __forceinline__ unsigned long long pk(float x, float y) {
  unsigned long long u;
  asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(x), "f"(y));
  return u;
}
__device__ __forceinline__ void upk(unsigned long long u, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(u));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// 2-D tensor copy global -> shared (TMA), completion on an mbarrier; x must be 16-byte aligned
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// W[0..3] += (a, b, c, d) with one vector reduction (16-byte aligned address)
__device__ __forceinline__ void red_add4(float* w, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(w), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}
__device__ __forceinline__ void red_add4(double*, double, double, double, double) {}

// Butterfly transpose-reduce of V <= 32 per-lane values: afterwards lane l holds the
// warp-wide sum of value index l * V / 32 (lanes sharing that index hold the same sum).
template <int V, typename T>
__device__ __forceinline__ T transpose_reduce(T (&v)[V], int lane) {
  static_assert(V >= 1 && V <= 32 && (V & (V - 1)) == 0, "V must be a power of two <= 32");
  int o = 16;
#pragma unroll
  for (int h = V / 2; h >= 1; h >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    o >>= 1;
  }
  T x = v[0];
#pragma unroll
  for (; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <typename TQ, int R, int NW, bool SW>
struct SweepCfg {
  using A = typename QT<TQ>::A;
  static constexpr int ROWS = QT<TQ>::ROWS;           // rows per slab
  static constexpr int SLABS = TILE / ROWS;           // slabs per tile
  static constexpr int RPW = ROWS / NW;               // slab rows per consumer warp
  static_assert(RPW >= 1 && RPW * NW == ROWS, "slab rows must split evenly over warps");
  static constexpr int CHUNK = (RPW * R <= 32) ? RPW : (32 / R);   // rows per butterfly
  static constexpr int NCHUNK = RPW / CHUNK;
  static constexpr int V = CHUNK * R;
  // FP32 accumulation with R >= 2 uses packed pairs; Y_I is then staged as duplicated pairs
  static constexpr bool PAIR = sizeof(A) == 4 && R >= 2;
  // CRED: the consumer warps hand their column partials of each tile to a reducer warp through
  // NPB shared-memory buffers; it adds the NW copies and issues one set of vector reductions
  // into W_J per tile (NW sets otherwise: the dominant L2 traffic of the FP32 sweep after Q)
  static constexpr bool CRED = PAIR;
  static constexpr int NPB = 2;
  static constexpr size_t PART_BYTES = CRED ? (size_t)NW * TILE * R * sizeof(A) : 0;
  static constexpr int THREADS = 32 * (NW + 1 + (CRED ? 1 : 0));
  // row partials kept per tile row (reduced across lanes once per tile row) when they fit
  static constexpr bool DEFER = PAIR && SLABS * RPW * R <= 64;
  static constexpr size_t YSM_BYTES = sizeof(A) * TILE * R * (PAIR ? 2 : 1);
  static constexpr int YJ_SLOTS = 4;                       // ring of Y_J tiles
  static constexpr uint32_t YJ_BYTES = sizeof(A) * TILE * R;
  // SW: Y_J arrives by a 2-D tensor copy with the 128-byte swizzle (Y viewed as rows of 32
  // floats); lane l then reads its 4 rows (R = 4: 64 bytes, R = 8: 128 bytes) with 16-byte loads
  // that hit distinct banks.  A contiguous copy would put the lanes 64 (128) bytes apart: a
  // 16-way bank conflict at the start of every tile, in all consumer warps at once.
  static_assert(!SW || (sizeof(A) == 4 && (R == 4 || R == 8)), "swizzled Y_J: FP32, R = 4 or 8");
  static constexpr int YV_ROWS = TILE * R / 32;            // 32-float rows of one Y_J tile
  static size_t smem_bytes(int nstage) {
    return 1024 + (size_t)nstage * SLAB_BYTES + YSM_BYTES + (size_t)YJ_SLOTS * YJ_BYTES +
           (size_t)NPB * PART_BYTES + 16 * (size_t)(nstage + YJ_SLOTS + (CRED ? NPB : 0));
  }
};

template <typename TQ, int R, int NW, bool SW>
__global__ void __launch_bounds__(SweepCfg<TQ, R, NW, SW>::THREADS, 1)
qy_packed_kernel(const TQ* __restrict__ tiles, int nt, int64_t ntiles, int nstage,
                 const typename QT<TQ>::A* __restrict__ Y, typename QT<TQ>::A* __restrict__ W,
                 int* err, const int* skip, const __grid_constant__ CUtensorMap ymap) {
  using C = SweepCfg<TQ, R, NW, SW>;
  using A = typename C::A;
  if (skip != nullptr && *skip != 0) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  // 1024-byte alignment (the swizzle pattern of a Y_J slot) as an offset into the shared array
  // (an integer round trip of the pointer would hide its address space and turn every shared
  // load into a generic load); slabs and Y_I staging are multiples of 1024 bytes
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* stages = base;
  A* ysm = reinterpret_cast<A*>(stages + (size_t)nstage * SLAB_BYTES);
  A* yjs = reinterpret_cast<A*>(reinterpret_cast<unsigned char*>(ysm) + C::YSM_BYTES);
  A* part = reinterpret_cast<A*>(reinterpret_cast<unsigned char*>(yjs) + (size_t)C::YJ_SLOTS * C::YJ_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(part) +
                                               (size_t)C::NPB * C::PART_BYTES);
  uint64_t* empty = full + nstage;
  uint64_t* fully = empty + nstage;
  uint64_t* emptyy = fully + C::YJ_SLOTS;
  uint64_t* pfull = emptyy + C::YJ_SLOTS;    // [NPB] (CRED): partials of every consumer warp written
  uint64_t* pempty = pfull + C::NPB;         // [NPB] (CRED): the reducer has read the buffer

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x;
  const int64_t t1 = ntiles * (blockIdx.x + 1) / gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstage; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NW);
    }
    for (int s = 0; s < C::YJ_SLOTS; ++s) {
      mbar_init(&fully[s], 1);
      mbar_init(&emptyy[s], NW);
    }
    if constexpr (C::CRED)
      for (int b = 0; b < C::NPB; ++b) {
        mbar_init(&pfull[b], NW);
        mbar_init(&pempty[b], 1);
      }
    fence_mbar_init();
  }
  __syncthreads();
  if (t0 >= t1) return;

  // first tile coordinates of this CTA's range (in the paired row order)
  int I0, J0;
  pair_order_start(nt, t0, I0, J0);

  if (warp == NW) {
    // ---------------- producer: one thread streams, per tile, Y_J then the tile's slabs
    if (lane == 0) {
      const unsigned char* qsrc = reinterpret_cast<const unsigned char*>(tiles);
      const unsigned char* ysrc = reinterpret_cast<const unsigned char*>(Y);
      int stage = 0, ys = 0;
      uint32_t phase = 0, yphase = 0;
      int64_t issued = 0, yissued = 0;
      int Jp = J0, Ip = I0;
      bool good = true;
      for (int64_t t = t0; t < t1 && good; ++t) {
        if (!mbar_wait(&emptyy[ys], yphase ^ 1u)) { atomicOr(err, DEV_TIMEOUT); break; }
        mbar_arrive_expect_tx(&fully[ys], C::YJ_BYTES);
        if constexpr (SW)
          tma_load_2d(reinterpret_cast<unsigned char*>(yjs) + (size_t)ys * C::YJ_BYTES, &ymap, 0,
                      Jp * C::YV_ROWS, &fully[ys]);
        else
          bulk_g2s(reinterpret_cast<unsigned char*>(yjs) + (size_t)ys * C::YJ_BYTES,
                   ysrc + (size_t)Jp * C::YJ_BYTES, C::YJ_BYTES, &fully[ys]);
        ++yissued;
        if (++ys == C::YJ_SLOTS) { ys = 0; yphase ^= 1u; }
        const unsigned char* src = qsrc + (size_t)tile_index(nt, Ip, Jp) * C::SLABS * SLAB_BYTES;
        for (int sl = 0; sl < C::SLABS; ++sl, ++issued) {
          if (!mbar_wait(&empty[stage], phase ^ 1u)) { atomicOr(err, DEV_TIMEOUT); good = false; break; }
          mbar_arrive_expect_tx(&full[stage], SLAB_BYTES);
          bulk_g2s(stages + (size_t)stage * SLAB_BYTES, src + (size_t)sl * SLAB_BYTES, SLAB_BYTES,
                   &full[stage]);
          if (++stage == nstage) { stage = 0; phase ^= 1u; }
        }
        pair_order_next(nt, Ip, Jp);
      }
      // Drain: do not leave while copies into this CTA's shared memory are in flight.
      for (int64_t k = issued > nstage ? issued - nstage : 0; k < issued; ++k) {
        if (!mbar_wait(&full[k % nstage], (uint32_t)((k / nstage) & 1))) { atomicOr(err, DEV_TIMEOUT); break; }
      }
      for (int64_t k = yissued > C::YJ_SLOTS ? yissued - C::YJ_SLOTS : 0; k < yissued; ++k) {
        if (!mbar_wait(&fully[k % C::YJ_SLOTS], (uint32_t)((k / C::YJ_SLOTS) & 1))) { atomicOr(err, DEV_TIMEOUT); break; }
      }
    }
    return;
  }

  if constexpr (C::CRED) {
    if (warp == NW + 1) {
      // ---------------- reducer: per tile, the NW warps' column partials (buffer layout
      // [warp][column 4l + cc as (cc, l)][R]) summed in warp order, one vector reduction per
      // 4 outputs into W_J
      constexpr int F4 = TILE * R / 4;          // float4 groups of one warp's partials
      int I = I0, J = J0;
      for (int64_t t = t0; t < t1; ++t) {
        const int64_t k = t - t0;
        const int b = (int)(k % C::NPB);
        const uint32_t par = (uint32_t)((k / C::NPB) & 1);
        if (!mbar_wait(&pfull[b], par)) { atomicOr(err, DEV_TIMEOUT); break; }
        const float4* pb = reinterpret_cast<const float4*>(part + (size_t)b * (C::PART_BYTES / sizeof(A)));
#pragma unroll
        for (int qd = 0; qd < F4 / 32; ++qd) {
          const int m = qd * 32 + lane;          // float4 index within one warp's partials
          float4 acc = pb[m];
#pragma unroll
          for (int w = 1; w < NW; ++w) {
            const float4 u = pb[(size_t)w * F4 + m];
            acc.x += u.x; acc.y += u.y; acc.z += u.z; acc.w += u.w;
          }
          // float index 4m = (cc * 32 + l) * R + j0
          const int g = (4 * m) / R, j0 = (4 * m) % R;
          const int cc = g >> 5, l = g & 31;
          red_add4(W + ((size_t)J * TILE + 4 * l + cc) * R + j0, acc.x, acc.y, acc.z, acc.w);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&pempty[b]);
        pair_order_next(nt, I, J);
      }
      return;
    }
  }

  // ---------------- consumers
  const int ctid = threadIdx.x;            // 0 .. 32*NW-1
  constexpr int NCT = 32 * NW;
  constexpr int RH = C::PAIR ? R / 2 : 1;  // j-pairs per row
  int curI = -1;
  int I = I0, J = J0;
  int stage = 0, ysl = 0;
  uint32_t phase = 0, yphase = 0;
  bool ok = true;

  // scalar-path state
  A yj[4][R];
  A colacc[4][R];
  A rowacc[C::SLABS][C::NCHUNK];
  // pair-path state: column pairs over c, Y_J pairs over j, row pairs over j
  unsigned long long colp[2][R];
  unsigned long long yjp[4][RH];
  unsigned long long rowp[C::DEFER ? C::SLABS : 1][C::DEFER ? C::RPW : 1][RH];

  // Reduce this lane's row partials of slab s across the warp and add them to W_I.
  auto reduce_add_rows = [&](int Irow, int s, A (&vals)[C::RPW * R]) {
#pragma unroll
    for (int ch = 0; ch < C::NCHUNK; ++ch) {
      A v[C::V];
#pragma unroll
      for (int e = 0; e < C::V; ++e) v[e] = vals[ch * C::V + e];
      const A x = transpose_reduce<C::V>(v, lane);
      constexpr int DUP = 32 / C::V;
      if ((lane & (DUP - 1)) == 0) {
        const int idx = lane / DUP;
        const int k = idx / R, j = idx % R;
        const int row = s * C::ROWS + warp * C::RPW + ch * C::CHUNK + k;
        atomicAdd(&W[((size_t)Irow * TILE + row) * R + j], x);
      }
    }
  };

  auto flush_rows = [&](int Irow) {
    if constexpr (C::DEFER) {
#pragma unroll
      for (int s = 0; s < C::SLABS; ++s) {
        A vals[C::RPW * R];
#pragma unroll
        for (int k = 0; k < C::RPW; ++k)
#pragma unroll
          for (int jp = 0; jp < RH; ++jp) upk(rowp[s][k][jp], vals[k * R + 2 * jp], vals[k * R + 2 * jp + 1]);
        reduce_add_rows(Irow, s, vals);
      }
    } else {
      constexpr int DUP = 32 / C::V;         // lanes sharing one butterfly result
      if ((lane & (DUP - 1)) == 0) {
        const int idx = lane / DUP;           // value index within a chunk
        const int k = idx / R, j = idx % R;
#pragma unroll
        for (int s = 0; s < C::SLABS; ++s)
#pragma unroll
          for (int c = 0; c < C::NCHUNK; ++c) {
            const int row = s * C::ROWS + warp * C::RPW + c * C::CHUNK + k;
            atomicAdd(&W[((size_t)Irow * TILE + row) * R + j], rowacc[s][c]);
          }
      }
    }
  };

  // Every consumer warp runs the same sequence of named barriers whatever happens: a wait that
  // gives up only marks the warp as failed (no further waits, no work), so no barrier can hang.
  for (int64_t t = t0; t < t1; ++t) {
    if (I != curI) {
      if (curI >= 0) flush_rows(curI);
      named_bar_sync(1, NCT);
      if constexpr (C::PAIR) {
        unsigned long long* ys2 = reinterpret_cast<unsigned long long*>(ysm);
        for (int e = ctid; e < TILE * R; e += NCT) {
          const float y = Y[(size_t)I * TILE * R + e];
          ys2[e] = pk(y, y);
        }
      } else {
        for (int e = ctid; e < TILE * R; e += NCT) ysm[e] = Y[(size_t)I * TILE * R + e];
      }
      named_bar_sync(1, NCT);
      if constexpr (C::DEFER) {
#pragma unroll
        for (int s = 0; s < C::SLABS; ++s)
#pragma unroll
          for (int k = 0; k < C::RPW; ++k)
#pragma unroll
            for (int jp = 0; jp < RH; ++jp) rowp[s][k][jp] = 0ull;
      } else {
#pragma unroll
        for (int s = 0; s < C::SLABS; ++s)
#pragma unroll
          for (int c = 0; c < C::NCHUNK; ++c) rowacc[s][c] = A(0);
      }
      curI = I;
    }
    {
      if (ok && !mbar_wait(&fully[ysl], yphase)) { atomicOr(err, DEV_TIMEOUT); ok = false; }
      const A* yp = yjs + (size_t)ysl * (TILE * R) + (size_t)(4 * lane) * R;
      if constexpr (SW) {
        // swizzled slot: 16-byte chunk k of 32-float row v sits at chunk k ^ (v & 7)
        const unsigned char* slot = reinterpret_cast<const unsigned char*>(yjs) + (size_t)ysl * C::YJ_BYTES;
        if constexpr (R == 4) {
          const int v = lane >> 1;                       // rows 4l..4l+3 = chunks 4(l&1)..+3 of row v
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float4 t = *reinterpret_cast<const float4*>(
                slot + v * 128 + 16 * ((4 * (lane & 1) + c) ^ (v & 7)));
            yjp[c][0] = pk(t.x, t.y);
            yjp[c][1] = pk(t.z, t.w);
          }
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) {                  // rows 4l..4l+3 = the 8 chunks of row l
            const float4 t = *reinterpret_cast<const float4*>(slot + lane * 128 + 16 * (k ^ (lane & 7)));
            yjp[k >> 1][2 * (k & 1)] = pk(t.x, t.y);
            yjp[k >> 1][2 * (k & 1) + 1] = pk(t.z, t.w);
          }
        }
#pragma unroll
        for (int cp = 0; cp < 2; ++cp)
#pragma unroll
          for (int j = 0; j < R; ++j) colp[cp][j] = 0ull;
      } else if constexpr (C::PAIR) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int jp = 0; jp < RH; ++jp) yjp[c][jp] = pk(yp[c * R + 2 * jp], yp[c * R + 2 * jp + 1]);
#pragma unroll
        for (int cp = 0; cp < 2; ++cp)
#pragma unroll
          for (int j = 0; j < R; ++j) colp[cp][j] = 0ull;
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int j = 0; j < R; ++j) { yj[c][j] = yp[c * R + j]; colacc[c][j] = A(0); }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&emptyy[ysl]);
      if (++ysl == C::YJ_SLOTS) { ysl = 0; yphase ^= 1u; }
    }
#pragma unroll
    for (int s = 0; s < C::SLABS; ++s) {
      if (ok && !mbar_wait(&full[stage], phase)) { atomicOr(err, DEV_TIMEOUT); ok = false; }
      const TQ* slab = reinterpret_cast<const TQ*>(stages + (size_t)stage * SLAB_BYTES);
      A q[C::RPW][4];
#pragma unroll
      for (int k = 0; k < C::RPW; ++k) {
        if (ok) load4(slab + (size_t)(warp * C::RPW + k) * TILE + 4 * lane, q[k]);
        else q[k][0] = q[k][1] = q[k][2] = q[k][3] = A(0);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (++stage == nstage) { stage = 0; phase ^= 1u; }
      const int rbase = s * C::ROWS + warp * C::RPW;
      if constexpr (C::PAIR) {
        const unsigned long long* ys2 = reinterpret_cast<const unsigned long long*>(ysm);
        unsigned long long rloc[C::DEFER ? 1 : C::RPW][RH];
        if constexpr (!C::DEFER) {
#pragma unroll
          for (int k = 0; k < C::RPW; ++k)
#pragma unroll
            for (int jp = 0; jp < RH; ++jp) rloc[k][jp] = 0ull;
        }
#pragma unroll
        for (int k = 0; k < C::RPW; ++k) {
          const unsigned long long q01 = pk(q[k][0], q[k][1]);
          const unsigned long long q23 = pk(q[k][2], q[k][3]);
          // column contribution: (colacc[c][j], colacc[c+1][j]) += (q_c, q_c+1) * (y_j, y_j)
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const unsigned long long yy = ys2[(rbase + k) * R + j];
            colp[0][j] = ffma2(q01, yy, colp[0][j]);
            colp[1][j] = ffma2(q23, yy, colp[1][j]);
          }
          // row contribution: (v_j, v_j+1) += (q_c, q_c) * (Y_J[c][j], Y_J[c][j+1])
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const unsigned long long qq = pk(q[k][c], q[k][c]);
#pragma unroll
            for (int jp = 0; jp < RH; ++jp) {
              if constexpr (C::DEFER) rowp[s][k][jp] = ffma2(qq, yjp[c][jp], rowp[s][k][jp]);
              else rloc[k][jp] = ffma2(qq, yjp[c][jp], rloc[k][jp]);
            }
          }
        }
        if constexpr (!C::DEFER) {
          A vals[C::RPW * R];
#pragma unroll
          for (int k = 0; k < C::RPW; ++k)
#pragma unroll
            for (int jp = 0; jp < RH; ++jp) upk(rloc[k][jp], vals[k * R + 2 * jp], vals[k * R + 2 * jp + 1]);
#pragma unroll
          for (int ch = 0; ch < C::NCHUNK; ++ch) {
            A v[C::V];
#pragma unroll
            for (int e = 0; e < C::V; ++e) v[e] = vals[ch * C::V + e];
            rowacc[s][ch] += transpose_reduce<C::V>(v, lane);
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < C::RPW; ++k) {
          A yi[R];
#pragma unroll
          for (int j = 0; j < R; ++j) yi[j] = ysm[(rbase + k) * R + j];
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int j = 0; j < R; ++j) colacc[c][j] = fma(q[k][c], yi[j], colacc[c][j]);
        }
#pragma unroll
        for (int ch = 0; ch < C::NCHUNK; ++ch) {
          A v[C::V];
#pragma unroll
          for (int kk = 0; kk < C::CHUNK; ++kk) {
            const int k = ch * C::CHUNK + kk;
#pragma unroll
            for (int j = 0; j < R; ++j) {
              A acc = q[k][0] * yj[0][j];
              acc = fma(q[k][1], yj[1][j], acc);
              acc = fma(q[k][2], yj[2][j], acc);
              acc = fma(q[k][3], yj[3][j], acc);
              v[kk * R + j] = acc;
            }
          }
          rowacc[s][ch] += transpose_reduce<C::V>(v, lane);
        }
      }
    }
    // column contribution: each warp adds its partials for columns 4l..4l+3 of Y_J directly
    // (vector reductions in L2; no barrier between warps), or (CRED) hands them to the reducer
    if constexpr (C::CRED) {
      const int64_t k = t - t0;
      const int b = (int)(k % C::NPB);
      const uint32_t par = (uint32_t)(((k / C::NPB) & 1) ^ 1);
      if (ok && !mbar_wait(&pempty[b], par)) { atomicOr(err, DEV_TIMEOUT); ok = false; }
      if (ok) {
        A* pw = part + (size_t)b * (C::PART_BYTES / sizeof(A)) + (size_t)warp * TILE * R;
#pragma unroll
        for (int cp = 0; cp < 2; ++cp) {
          float lo[R], hi[R];
#pragma unroll
          for (int j = 0; j < R; ++j) upk(colp[cp][j], lo[j], hi[j]);
#pragma unroll
          for (int j = 0; j < R; j += 4) {
            *reinterpret_cast<float4*>(pw + ((2 * cp) * 32 + lane) * R + j) = make_float4(lo[j], lo[j + 1], lo[j + 2], lo[j + 3]);
            *reinterpret_cast<float4*>(pw + ((2 * cp + 1) * 32 + lane) * R + j) = make_float4(hi[j], hi[j + 1], hi[j + 2], hi[j + 3]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pfull[b]);
    } else {
      A* wj = W + ((size_t)J * TILE + 4 * lane) * R;
      if constexpr (C::PAIR) {
#pragma unroll
        for (int cp = 0; cp < 2; ++cp) {
          float lo[R], hi[R];
#pragma unroll
          for (int j = 0; j < R; ++j) upk(colp[cp][j], lo[j], hi[j]);
#pragma unroll
          for (int j = 0; j < R; j += 4) {
            red_add4(wj + (2 * cp) * R + j, lo[j], lo[j + 1], lo[j + 2], lo[j + 3]);
            red_add4(wj + (2 * cp + 1) * R + j, hi[j], hi[j + 1], hi[j + 2], hi[j + 3]);
          }
        }
      } else if constexpr (sizeof(A) == 4 && R == 1) {
        red_add4(wj, colacc[0][0], colacc[1][0], colacc[2][0], colacc[3][0]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int j = 0; j < R; ++j) atomicAdd(&wj[c * R + j], colacc[c][j]);
      }
    }
    pair_order_next(nt, I, J);
  }
  if (curI >= 0) flush_rows(curI);
}

// ------------------------------------------------------------------ host launcher
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// 2-D map of an FP32 n_pad x R row-major Y viewed as rows of 32 floats, box = one Y_J tile,
// 128-byte swizzle.  Maps are cached by (address, rows, R) (the solver reuses a few buffers);
// false when Y is not 16-byte aligned or the driver cannot encode one.
static bool y_swizzle_map(const void* Y, int n_pad, int R, CUtensorMap* out) {
  struct Entry { const void* y; int n_pad, R; CUtensorMap map; };
  static Entry cache[16];
  static int used = 0, next = 0;
  static std::mutex mu;   // contexts may be driven from different host threads
  if ((reinterpret_cast<uintptr_t>(Y) & 15u) != 0) return false;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i)
    if (cache[i].y == Y && cache[i].n_pad == n_pad && cache[i].R == R) { *out = cache[i].map; return true; }
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t gdim[2] = {32, (cuuint64_t)n_pad * R / 32};
  const cuuint64_t gstride[1] = {128};
  const cuuint32_t box[2] = {32, (cuuint32_t)(TILE * R / 32)};
  const cuuint32_t estride[2] = {1, 1};
  CUtensorMap m;
  if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(Y), gdim, gstride, box, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  cache[next] = Entry{Y, n_pad, R, m};
  next = (next + 1) % 16;
  if (used < 16) ++used;
  *out = m;
  return true;
}

template <typename TQ, int R, int NW, bool SW>
static xm_status launch_t(xm_ctx* ctx, const TQ* tiles, const DeviceQ& q, const void* Y, void* W,
                          const int* skip, cudaStream_t st, const CUtensorMap& ymap) {
  using C = SweepCfg<TQ, R, NW, SW>;
  using A = typename C::A;
  // The shared-memory opt-in is an attribute of the kernel on each device: configure it once
  // per device (contexts on different devices may launch from different host threads).
  constexpr int MAX_DEVICES = 64;
  static std::mutex mu;
  static int nstage_dev[MAX_DEVICES] = {};
  if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
    return set_error(XM_EINVAL, "sweep: device %d out of range", ctx->device);
  int nstage_cfg;
  {
    std::lock_guard<std::mutex> lock(mu);
    nstage_cfg = nstage_dev[ctx->device];
    if (nstage_cfg == 0) {
      const size_t fixed = C::smem_bytes(0);
      int ns = (int)((ctx->smem_optin - fixed) / (SLAB_BYTES + 16));
      if (ns > 12) ns = 12;
      if (ns < 2) return set_error(XM_ECUDA, "sweep: not enough shared memory (%zu)", ctx->smem_optin);
      XM_CUDA_TRY(cudaFuncSetAttribute(qy_packed_kernel<TQ, R, NW, SW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::smem_bytes(ns)));
      nstage_dev[ctx->device] = nstage_cfg = ns;
    }
  }
  int grid = ctx->num_sms;
  if ((int64_t)grid > q.ntiles) grid = (int)q.ntiles;
  qy_packed_kernel<TQ, R, NW, SW><<<grid, C::THREADS, C::smem_bytes(nstage_cfg), st>>>(
      tiles, q.nt, q.ntiles, nstage_cfg, static_cast<const A*>(Y), static_cast<A*>(W),
      ctx->d_err, skip, ymap);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

template <typename TQ, int NW>
static xm_status dispatch_r(xm_ctx* ctx, const TQ* tiles, const DeviceQ& q, int R, const void* Y,
                            void* W, const int* skip, cudaStream_t st) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  constexpr bool f32 = sizeof(typename QT<TQ>::A) == 4;
  const bool sw = f32 && (R == 4 || R == 8) && y_swizzle_map(Y, q.n_pad, R, &m);
  switch (R) {
    case 1: return launch_t<TQ, 1, NW, false>(ctx, tiles, q, Y, W, skip, st, m);
    case 4:
      if constexpr (f32)
        if (sw) return launch_t<TQ, 4, NW, true>(ctx, tiles, q, Y, W, skip, st, m);
      return launch_t<TQ, 4, NW, false>(ctx, tiles, q, Y, W, skip, st, m);
    case 8:
      if constexpr (f32)
        if (sw) return launch_t<TQ, 8, NW, true>(ctx, tiles, q, Y, W, skip, st, m);
      return launch_t<TQ, 8, NW, false>(ctx, tiles, q, Y, W, skip, st, m);
    default: return set_error(XM_EINVAL, "sweep: padded width %d not in {1,4,8}", R);
  }
}

xm_status qy_launch(xm_ctx* ctx, const DeviceQ& q, int prec, int R, const void* Y, void* W,
                    const int* skip, cudaStream_t st) {
  if (q.ntiles == 0 && !q.fact) return XM_OK;
  switch (prec) {
    case XM_FP64:
      if (!q.q64) {
        // the factored operator (App. A in product form) stands in for the FP64 tiles
        if (q.fact) return qfact_apply(ctx, *q.fact, R, R, static_cast<const double*>(Y),
                                       static_cast<double*>(W), skip, st);
        return set_error(XM_EINVAL, "sweep: Q has no FP64 copy and no factored operator");
      }
      return dispatch_r<double, 8>(ctx, q.q64, q, R, Y, W, skip, st);
    case XM_FP32_BULK:
      if (!q.q32) return set_error(XM_EINVAL, "sweep: Q has no FP32 copy");
      return dispatch_r<float, 8>(ctx, q.q32, q, R, Y, W, skip, st);
    case XM_BF16Q_BULK:
      // tensor cores: Y in three BF16 digits against the BF16 tiles (xm_qy_tc.cu)
      return qy_tc_launch(ctx, q, R, static_cast<const float*>(Y), static_cast<float*>(W), skip, st);
    default:
      return set_error(XM_EINVAL, "sweep: unknown precision %d", prec);
  }
}

}  // namespace xm
