// Factored Q operator: Q Y without the dense Q (App. A's elimination kept in product form).
//
// Q = P - Bbar Sbar^{-1} Bbar^T (landmarks eliminated first, then the translations with t_0 = 0).
// For an n x r block Y (camera i owns rows 3i..3i+2) every term of Q Y is a sum over the
// observations, which makes Q Y the gradient of the least-squares SBA cost at the optimal
// translations and landmarks for the columns of Y (Prop. 1):
//   a_e   = u_e^T Y_i                                   (1 x r, observation e = (i, k))
//   m_k   = sum_{e in k} w_e a_e / d_k,  d_k = sum_{e in k} w_e       (landmark means)
//   b_j   = sum_{e in j} w_e (a_e - m_k)                (camera sums: Bbar^T Y, rows j >= 1)
//   t     = -Sbar^{-1} bbar,  t_0 = 0                   (the optimal translations)
//   tb_k  = sum_{e in k} w_e t_{i_e} / d_k              (landmark means of t)
//   (Q Y)_i = sum_{e in i} w_e u_e (a_e - m_k + t_i - tb_k)     (3 x r)
// The residual a_e - m_k + t_i - tb_k is the least-squares residual of Eq. 3 for the columns of
// Y.  Per product: four passes over the observations (two landmark-major, two camera-major, each
// in its own contiguous copy of (u, w)) and one packed symmetric sweep with -Sbar^{-1}, an
// (N-1)^2 matrix instead of the (3N)^2 of Q.  All arithmetic is FP64; every sum runs in a fixed
// order (reruns are bit-identical).
//
// Set-up: Sbar's Cholesky factor L (the camera block left after the landmark elimination), the
// triangular inverse X = L^{-1} and the tiles of 0 - X^T X = -Sbar^{-1}, all by the build's
// error-free digit-split products on the BF16 tensor cores (FP64-accurate).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "xm_internal.cuh"

namespace xm {

xm_status alloc_tiles(xm_ctx* ctx, DeviceQ& q, int N, unsigned mask);
void free_tiles(DeviceQ& q);

namespace {
struct Mem {
  void* p = nullptr;
  ~Mem() { if (p) cudaFree(p); }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};
int grid_of(size_t work, int threads, int num_sms, int per_sm = 8) {
  const size_t g = (work + threads - 1) / threads;
  return (int)std::max<size_t>(1, std::min(g, (size_t)num_sms * per_sm));
}
}  // namespace


// ------------------------------------------------------------------ kernels
// Observation pass kernels take the padded width R of Y (1, 4 or 8) and the used columns r.

__global__ void k_qf_gather(int64_t E, const int64_t* __restrict__ idx, const int32_t* __restrict__ other,
                            const double* __restrict__ ukp, const double* __restrict__ w,
                            double* __restrict__ u_out, double* __restrict__ w_out,
                            int32_t* __restrict__ other_out) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < E; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx[x];
    u_out[3 * x] = ukp[3 * e];
    u_out[3 * x + 1] = ukp[3 * e + 1];
    u_out[3 * x + 2] = ukp[3 * e + 2];
    w_out[x] = w[e];
    other_out[x] = other[e];
  }
}

// X = I (column-major m x m, zero elsewhere on entry)
__global__ void k_qf_eye(int m, double* __restrict__ X) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
    X[(size_t)j * m + j] = 1.0;
}

__global__ void k_qf_dinv(int M, const int64_t* __restrict__ loff, const double* __restrict__ lw,
                          double* __restrict__ dinv) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) d += lw[x];
    dinv[k] = d > 0.0 ? 1.0 / d : 0.0;
  }
}

// m_k = sum_{e in k} w_e u_e^T Y_{i_e} / d_k (one thread per landmark)
template <int R>
__global__ void k_qf_lmk_a(int M, int r, int ld, const int64_t* __restrict__ loff, const double* __restrict__ lu,
                           const double* __restrict__ lw, const int32_t* __restrict__ lc,
                           const double* __restrict__ dinv, const double* __restrict__ Y,
                           double* __restrict__ mk, const int* skip) {
  if (skip && *skip) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double acc[R];
#pragma unroll
    for (int j = 0; j < R; ++j) acc[j] = 0.0;
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) {
      const double* y = Y + (size_t)3 * lc[x] * ld;
      const double u0 = lu[3 * x], u1 = lu[3 * x + 1], u2 = lu[3 * x + 2], we = lw[x];
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (j < r) acc[j] += we * (u0 * y[j] + u1 * y[ld + j] + u2 * y[2 * ld + j]);
    }
    const double di = dinv[k];
#pragma unroll
    for (int j = 0; j < R; ++j) mk[(size_t)k * 8 + j] = acc[j] * di;
  }
}

// tb_k = sum_{e in k} w_e t_{i_e} / d_k, t_0 = 0, t_i = row i - 1 of the sweep output
template <int R>
__global__ void k_qf_lmk_t(int M, const int64_t* __restrict__ loff, const double* __restrict__ lw,
                           const int32_t* __restrict__ lc, const double* __restrict__ dinv,
                           const double* __restrict__ tt, double* __restrict__ tbk, const int* skip) {
  if (skip && *skip) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double acc[R];
#pragma unroll
    for (int j = 0; j < R; ++j) acc[j] = 0.0;
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) {
      const int i = lc[x];
      if (i == 0) continue;
      const double we = lw[x];
      const double* t = tt + (size_t)(i - 1) * R;
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] += we * t[j];
    }
    const double di = dinv[k];
#pragma unroll
    for (int j = 0; j < R; ++j) tbk[(size_t)k * 8 + j] = acc[j] * di;
  }
}

// One warp per camera: lanes stride over the camera's observations, then a fixed butterfly.
// OUT = false: b_i = sum w_e (a_e - m_k) into row i - 1 of the sweep input (i >= 1).
// OUT = true:  (Q Y)_i += sum w_e u_e (a_e - m_k + t_i - tb_k); t's row i - 1 is then cleared
//              for the next accumulating sweep.
template <int R, bool OUT>
__global__ void k_qf_cam(int N, int r, int ld, const int64_t* __restrict__ coff, const double* __restrict__ cu,
                         const double* __restrict__ cw, const int32_t* __restrict__ cl,
                         const double* __restrict__ Y, const double* __restrict__ mk,
                         const double* __restrict__ tbk, double* __restrict__ tt,
                         double* __restrict__ bb, double* __restrict__ W, const int* skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < N; i += warps) {
    double y[3][R], ti[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const bool on = j < r;
      y[0][j] = on ? Y[(size_t)(3 * i) * ld + j] : 0.0;
      y[1][j] = on ? Y[(size_t)(3 * i + 1) * ld + j] : 0.0;
      y[2][j] = on ? Y[(size_t)(3 * i + 2) * ld + j] : 0.0;
      ti[j] = (OUT && i > 0) ? tt[(size_t)(i - 1) * R + j] : 0.0;
    }
    double acc[OUT ? 3 : 1][R];
#pragma unroll
    for (int a = 0; a < (OUT ? 3 : 1); ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[a][j] = 0.0;
    for (int64_t x = coff[i] + lane; x < coff[i + 1]; x += 32) {
      const double u0 = cu[3 * x], u1 = cu[3 * x + 1], u2 = cu[3 * x + 2], we = cw[x];
      const double* m = mk + (size_t)cl[x] * 8;
      if constexpr (OUT) {
        const double* tb = tbk + (size_t)cl[x] * 8;
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const double rho = we * (u0 * y[0][j] + u1 * y[1][j] + u2 * y[2][j] - m[j] + ti[j] - tb[j]);
          acc[0][j] += u0 * rho;
          acc[1][j] += u1 * rho;
          acc[2][j] += u2 * rho;
        }
      } else {
#pragma unroll
        for (int j = 0; j < R; ++j) acc[0][j] += we * (u0 * y[0][j] + u1 * y[1][j] + u2 * y[2][j] - m[j]);
      }
    }
#pragma unroll
    for (int a = 0; a < (OUT ? 3 : 1); ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[a][j] = warp_sum(acc[a][j]);
    if (lane == 0) {
      if constexpr (OUT) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int j = 0; j < R; ++j)
            if (j < r) W[(size_t)(3 * i + a) * ld + j] += acc[a][j];
        if (i > 0)
#pragma unroll
          for (int j = 0; j < R; ++j) tt[(size_t)(i - 1) * R + j] = 0.0;
      } else if (i > 0) {
#pragma unroll
        for (int j = 0; j < R; ++j) bb[(size_t)(i - 1) * R + j] = acc[0][j];
      }
    }
  }
}

// ------------------------------------------------------------------ set-up and product
void qfact_release(QFact& f) {
  void* ptrs[] = {f.loff, f.coff, f.lu, f.lw, f.lc, f.cu, f.cw, f.cl, f.dinv, f.mk, f.tbk, f.bb, f.tt};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free_tiles(f.sinv);
  f = QFact();
}

xm_status qfact_build(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                      const double* ukp, const double* w, QFact& f) {
  auto tic = std::chrono::steady_clock::now();
  cudaStream_t st = ctx->stream;
  XM_TRY(validate_obs(ctx, N, M, E, cam, lmk, ukp, w));
  XM_TRY(check_connected(ctx, N, M, E, cam, lmk));
  f.N = N; f.M = M; f.E = E;
  const size_t Es = (size_t)std::max<int64_t>(E, 1), Ms = (size_t)std::max(M, 1);
  auto alloc = [&](void** p, size_t bytes) -> xm_status {
    XM_CUDA_TRY(cudaMalloc(p, bytes));
    f.bytes += bytes;
    return XM_OK;
  };
  XM_TRY(alloc((void**)&f.loff, sizeof(int64_t) * (Ms + 1)));
  XM_TRY(alloc((void**)&f.coff, sizeof(int64_t) * ((size_t)N + 1)));
  XM_TRY(alloc((void**)&f.lu, sizeof(double) * 3 * Es));
  XM_TRY(alloc((void**)&f.lw, sizeof(double) * Es));
  XM_TRY(alloc((void**)&f.lc, sizeof(int32_t) * Es));
  XM_TRY(alloc((void**)&f.cu, sizeof(double) * 3 * Es));
  XM_TRY(alloc((void**)&f.cw, sizeof(double) * Es));
  XM_TRY(alloc((void**)&f.cl, sizeof(int32_t) * Es));
  XM_TRY(alloc((void**)&f.dinv, sizeof(double) * Ms));
  XM_TRY(alloc((void**)&f.mk, sizeof(double) * 8 * Ms));
  XM_TRY(alloc((void**)&f.tbk, sizeof(double) * 8 * Ms));
  Mem lidx, cidx, S, d;
  XM_CUDA_TRY(cudaMalloc(&lidx.p, sizeof(int64_t) * Es));
  XM_CUDA_TRY(cudaMalloc(&cidx.p, sizeof(int64_t) * Es));
  if (M > 0) XM_TRY(obs_csr(ctx, E, lmk, M, f.loff, lidx.as<int64_t>()));
  else XM_CUDA_TRY(cudaMemsetAsync(f.loff, 0, sizeof(int64_t), st));
  XM_TRY(obs_csr(ctx, E, cam, N, f.coff, cidx.as<int64_t>()));
  if (E > 0) {
    const int g = grid_of((size_t)E, 256, ctx->num_sms);
    k_qf_gather<<<g, 256, 0, st>>>(E, lidx.as<int64_t>(), cam, ukp, w, f.lu, f.lw, f.lc);
    k_qf_gather<<<g, 256, 0, st>>>(E, cidx.as<int64_t>(), lmk, ukp, w, f.cu, f.cw, f.cl);
  }
  if (M > 0) k_qf_dinv<<<grid_of((size_t)M, 256, ctx->num_sms), 256, 0, st>>>(M, f.loff, f.lw, f.dinv);
  XM_CUDA_TRY(cudaGetLastError());
  const int m = N - 1;
  if (m >= 1) {
    // Cholesky factor of Sbar (camera 0 anchored), then X = L^{-1} and the tiles of -X^T X
    XM_CUDA_TRY(cudaMalloc(&S.p, sizeof(double) * (size_t)N * N));
    XM_CUDA_TRY(cudaMalloc(&d.p, sizeof(double) * Ms));
    XM_TRY(schur_S_factor(ctx, N, M, cam, w, f.coff, cidx.as<int64_t>(), f.loff, lidx.as<int64_t>(),
                          S.as<double>(), d.as<double>()));
    Mem X, Z;
    XM_CUDA_TRY(cudaMalloc(&X.p, sizeof(double) * (size_t)m * m));
    XM_CUDA_TRY(cudaMemsetAsync(X.p, 0, sizeof(double) * (size_t)m * m, st));
    k_qf_eye<<<grid_of((size_t)m, 256, ctx->num_sms), 256, 0, st>>>(m, X.as<double>());
    XM_CUDA_TRY(cudaGetLastError());
    XM_TRY(split_trsm(ctx, S.as<double>() + N + 1, N, X.as<double>(), m, m, m));
    // tiles of 0 - X^T X; q.n = m rows
    DeviceQ& q = f.sinv;
    q.N = 0;
    q.n = m;
    q.nt = (m + TILE - 1) / TILE;
    q.n_pad = q.nt * TILE;
    q.ntiles = tile_count(q.nt);
    q.mask = XM_STORE_FP64;
    XM_CUDA_TRY(cudaMalloc(&q.q64, sizeof(double) * (size_t)q.ntiles * TILE * TILE));
    f.bytes += sizeof(double) * (size_t)q.ntiles * TILE * TILE;
    XM_CUDA_TRY(cudaMalloc(&Z.p, sizeof(double) * (size_t)m * m));
    XM_CUDA_TRY(cudaMemsetAsync(Z.p, 0, sizeof(double) * (size_t)m * m, st));
    XM_TRY(split_update_pack(ctx, X.as<double>(), m, m, Z.as<double>(), q, q.q64));
    XM_TRY(alloc((void**)&f.bb, sizeof(double) * (size_t)q.n_pad * 8));
    XM_TRY(alloc((void**)&f.tt, sizeof(double) * (size_t)q.n_pad * 8));
    XM_CUDA_TRY(cudaMemsetAsync(f.bb, 0, sizeof(double) * (size_t)q.n_pad * 8, st));
    XM_CUDA_TRY(cudaMemsetAsync(f.tt, 0, sizeof(double) * (size_t)q.n_pad * 8, st));
  }
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  XM_TRY(check_device_error(ctx, "factored operator set-up"));
  f.t_setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - tic).count();
  return XM_OK;
}

template <int R>
static xm_status qfact_apply_t(xm_ctx* ctx, const QFact& f, int r, int ld, const double* Y, double* W,
                               const int* skip, cudaStream_t st) {
  const int gl = grid_of((size_t)std::max(f.M, 1), 128, ctx->num_sms, 16);
  const int gc = grid_of((size_t)f.N * 32, 256, ctx->num_sms, 16);
  if (f.M > 0)
    k_qf_lmk_a<R><<<gl, 128, 0, st>>>(f.M, r, ld, f.loff, f.lu, f.lw, f.lc, f.dinv, Y, f.mk, skip);
  if (f.N > 1) {
    k_qf_cam<R, false><<<gc, 256, 0, st>>>(f.N, r, ld, f.coff, f.cu, f.cw, f.cl, Y, f.mk, f.tbk, f.tt,
                                           f.bb, nullptr, skip);
    XM_CUDA_TRY(cudaGetLastError());
    XM_TRY(qy_launch(ctx, f.sinv, XM_FP64, R, f.bb, f.tt, skip, st));   // t = -Sbar^{-1} bbar
    if (f.M > 0)
      k_qf_lmk_t<R><<<gl, 128, 0, st>>>(f.M, f.loff, f.lw, f.lc, f.dinv, f.tt, f.tbk, skip);
  } else if (f.M > 0) {
    XM_CUDA_TRY(cudaMemsetAsync(f.tbk, 0, sizeof(double) * 8 * (size_t)f.M, st));
  }
  k_qf_cam<R, true><<<gc, 256, 0, st>>>(f.N, r, ld, f.coff, f.cu, f.cw, f.cl, Y, f.mk, f.tbk, f.tt, f.bb,
                                        W, skip);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

// W += Q Y for an FP64 Y whose first r columns are used, rows of ld doubles (W accumulates, like
// the dense sweep; the padded layout of the solver has ld = R).
xm_status qfact_apply(xm_ctx* ctx, const QFact& f, int r, int ld, const double* Y, double* W,
                      const int* skip, cudaStream_t st) {
  if (r == 1) return qfact_apply_t<1>(ctx, f, r, ld, Y, W, skip, st);
  if (r <= 4) return qfact_apply_t<4>(ctx, f, r, ld, Y, W, skip, st);
  return qfact_apply_t<8>(ctx, f, r, ld, Y, W, skip, st);
}

}  // namespace xm

struct xm_qfact {
  xm::QFact f;
};

using namespace xm;

extern "C" {

xm_status xm_qfact_create(xm_ctx* c, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                          const double* ukp, const double* w, xm_qfact** out) {
  if (!c || !out) return set_error(XM_EINVAL, "xm_qfact_create: NULL argument");
  *out = nullptr;
  if (N < 1 || M < 0 || E < 0) return set_error(XM_EINVAL, "xm_qfact_create: bad sizes");
  if (E > 0 && (!cam || !lmk || !ukp || !w)) return set_error(XM_EINVAL, "xm_qfact_create: NULL observations");
  if (N - 1 > 0 && !split_update_fits(N - 1, N - 1))
    return set_error(XM_EINVAL, "xm_qfact_create: N = %d beyond the tensor-core inverse's range", N);
  XM_CUDA_TRY(cudaSetDevice(c->device));
  xm_qfact* h = new xm_qfact();
  xm_status s = qfact_build(c, N, M, E, cam, lmk, ukp, w, h->f);
  if (s != XM_OK) {
    qfact_release(h->f);
    delete h;
    return s;
  }
  *out = h;
  return XM_OK;
}

xm_status xm_qy_factored(xm_ctx* c, const xm_qfact* f, int r, const double* Y, double* W) {
  if (!c || !f || !Y || !W) return set_error(XM_EINVAL, "xm_qy_factored: NULL argument");
  if (r < 1 || r > XM_MAX_RANK) return set_error(XM_EINVAL, "xm_qy_factored: r=%d not in [1, %d]", r, XM_MAX_RANK);
  XM_CUDA_TRY(cudaSetDevice(c->device));
  XM_CUDA_TRY(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)3 * f->f.N * r, c->stream));
  return qfact_apply(c, f->f, r, r, Y, W, nullptr, c->stream);
}

xm_status xm_qfact_info(const xm_qfact* f, int* N, int* M, int64_t* E, size_t* bytes, double* t_setup_s) {
  if (!f) return set_error(XM_EINVAL, "xm_qfact_info: NULL handle");
  if (N) *N = f->f.N;
  if (M) *M = f->f.M;
  if (E) *E = f->f.E;
  if (bytes) *bytes = f->f.bytes;
  if (t_setup_s) *t_setup_s = f->f.t_setup_s;
  return XM_OK;
}

xm_status xm_qfact_free(xm_ctx* c, xm_qfact* f) {
  if (!f) return XM_OK;
  if (c) cudaSetDevice(c->device);
  qfact_release(f->f);
  delete f;
  return XM_OK;
}

}  // extern "C"
