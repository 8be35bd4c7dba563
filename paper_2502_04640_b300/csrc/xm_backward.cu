// Adjoint of the certified optimum: gradients of a loss of the anchored blocks G_i = Y_0 Y_i^T
// (= s_i R_i at a tight optimum, Sec. 2.2) with respect to the lifted keypoints u_e and the
// weights w_e of every observation.
//
// Implicit differentiation of the first-order condition rgrad(Y) = 2 P_Y(Q Y - Lambda Y) = 0
// (Sec. 3): a perturbation Qdot moves the optimum by Ydot with Hess[Ydot] = -P_Y(2 Qdot Y), so
// with the adjoint lambda solving Hess[lambda] = P_Y(dL/dY) the loss changes by
// <dL/dQ, Qdot> with dL/dQ = -(lambda Y^T + Y lambda^T).  Q enters only through the bilinear
// forms a^T Q b, which equal sum_e w_e <e_a, e_b> at the optimal translations and landmarks of
// Prop. 1 (App. A elimination); by the envelope theorem their derivatives are
//   d(a^T Q b)/du_e = w_e (a_i e_b + b_i e_a),   d(a^T Q b)/dw_e = <e_a, e_b>,
// with e the residual u_e^T U_i + t_i - p_k of the least-squares fit for columns U = [Y, lambda].
//
// Device path:
//   1. FP64 gradient at Y (dual blocks Lambda of Sec. 3), dL/dY from dL/dG, tangent projection.
//   2. Hess[lambda] = g_L by conjugate gradients on the Q sweep: FP64 operator for prec FP64;
//      otherwise FP32 inner CG with FP64 residual refinement (mixed-precision iterative
//      refinement: each refinement step solves Hess[delta] = g_L - Hess64[lambda] in FP32).
//   3. The optimal residuals of the 2R columns [Y, lambda]: landmark means, camera sums, the
//      anchored translation solve with the Cholesky factor of Sbar, then the outputs.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "xm_internal.cuh"
#include "xm_ops.cuh"

namespace xm {

// dL/dY for G_i = Y_0 Y_i^T (i >= 1): dY_i = D_i^T Y_0, dY_0 = sum_i D_i Y_i.  D: N x 3 x 3
// row-major (entry 0 ignored).  The anchor row is the deterministic grid sum.
template <int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_adj_dY(int N, const double* __restrict__ Y, const double* __restrict__ D, double* __restrict__ X,
         double* partials, unsigned* counter) {
  double v[3 * R];
#pragma unroll
  for (int k = 0; k < 3 * R; ++k) v[k] = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 1 && i < N) {
    double y0[3][R], yi[3][R], d[3][3], x[3][R];
    load_block<double, double, R>(Y, 0, y0);
    load_block<double, double, R>(Y, i, yi);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) d[a][b] = D[(size_t)9 * i + 3 * a + b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        x[a][j] = d[0][a] * y0[0][j] + d[1][a] * y0[1][j] + d[2][a] * y0[2][j];
        v[a * R + j] = d[a][0] * yi[0][j] + d[a][1] * yi[1][j] + d[a][2] * yi[2][j];
      }
    store_block<double, double, R>(X, i, x);
  }
  grid_reduce<3 * R>(v, partials, counter, [&](double* t) {
    for (int k = 0; k < 3 * R; ++k) X[k] = t[k];
  });
}

// X <- P_Y(X) (tangent projection of Sec. 3); sc->dot = ||X||^2
template <int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_adj_proj(int N, const double* __restrict__ Y, double* __restrict__ X, Scal* sc, double* partials,
           unsigned* counter) {
  double v[1] = {0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double y[3][R], x[3][R], S[3][3], al;
    load_block<double, double, R>(Y, i, y);
    load_block<double, double, R>(X, i, x);
    dual_block<double, R>(x, y, i == 0, S, al);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        x[a][j] -= S[a][0] * y[0][j] + S[a][1] * y[1][j] + S[a][2] * y[2][j];
        s += x[a][j] * x[a][j];
      }
    store_block<double, double, R>(X, i, x);
    v[0] = s;
  }
  grid_reduce<1>(v, partials, counter, [&](double* t) { sc->dot = t[0]; });
}

// res = g_L - Hess[lambda] from the FP64 sweep Wd = Q lambda (Wd is reset to zero); the inner
// CG's right side Gin = -res in its storage type; sc->dot = ||res||^2
template <typename Ti, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_adj_resid(int N, const double* __restrict__ Y, double* __restrict__ Wd,
            const double* __restrict__ lam, const double* __restrict__ gL,
            const double* __restrict__ Lam, double* __restrict__ res, Ti* __restrict__ Gin,
            Scal* sc, double* partials, unsigned* counter) {
  double v[1] = {0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    hvp_block<double, R>(i, Y, Wd, lam, res, Lam);
    double h[3][R], g[3][R];
    load_block<double, double, R>(res, i, h);
    load_block<double, double, R>(gL, i, g);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        h[a][j] = g[a][j] - h[a][j];
        s += h[a][j] * h[a][j];
        Gin[(size_t)(3 * i + a) * R + j] = Ti(-h[a][j]);
      }
    store_block<double, double, R>(res, i, h);
    v[0] = s;
  }
  grid_reduce<1>(v, partials, counter, [&](double* t) { sc->dot = t[0]; });
}

// plain CG step length: alpha = <r,r> / <d, Hess d>; a non-positive curvature ends the solve
// (the operator is positive semi-definite at a certified optimum and the right side lies in
// its range)
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_cg_epi(int N, const T* __restrict__ Y, T* __restrict__ Wd, const T* __restrict__ delta,
         T* __restrict__ Hd, const double* __restrict__ Lam, Scal* sc, double* partials,
         unsigned* counter) {
  if (sc->done) return;
  double v[1] = {0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) v[0] = hvp_block<T, R>(i, Y, Wd, delta, Hd, Lam);
  grid_reduce<1>(v, partials, counter, [&](double* t) {
    sc->kappa = t[0];
    if (!(t[0] > 0.0)) { sc->done = 1; sc->reason = 1; return; }
    sc->alpha = sc->rr / t[0];
  });
}

template <typename Ti>
__global__ void k_axpy_to64(size_t total, const Ti* __restrict__ x, double* __restrict__ y) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    y[e] += double(x[e]);
}

// a_e = U_i^T u_e for the 2R columns U = [Y, lambda] of camera i
template <int R>
__device__ __forceinline__ void obs_proj(const double* __restrict__ Y, const double* __restrict__ lam,
                                         int i, const double* __restrict__ u, double (&a)[2 * R]) {
#pragma unroll
  for (int j = 0; j < R; ++j) {
    double s = 0.0, t = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s += Y[(size_t)(3 * i + c) * R + j] * u[c];
      t += lam[(size_t)(3 * i + c) * R + j] * u[c];
    }
    a[j] = s;
    a[R + j] = t;
  }
}

// m_k = sum_{e in k} w_e a_e / d_k   (M x 2R)
template <int R>
__global__ void k_adj_lmk_mean(int M, const int64_t* __restrict__ loff, const int64_t* __restrict__ lidx,
                               const int32_t* __restrict__ cam, const double* __restrict__ ukp,
                               const double* __restrict__ w, const double* __restrict__ dk,
                               const double* __restrict__ Y, const double* __restrict__ lam,
                               double* __restrict__ m) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double acc[2 * R];
#pragma unroll
    for (int c = 0; c < 2 * R; ++c) acc[c] = 0.0;
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) {
      const int64_t e = lidx[x];
      double a[2 * R];
      obs_proj<R>(Y, lam, cam[e], ukp + 3 * e, a);
#pragma unroll
      for (int c = 0; c < 2 * R; ++c) acc[c] += w[e] * a[c];
    }
    const double inv = dk[k] > 0.0 ? 1.0 / dk[k] : 0.0;
#pragma unroll
    for (int c = 0; c < 2 * R; ++c) m[(size_t)k * 2 * R + c] = acc[c] * inv;
  }
}

// b_j = sum_{e: cam_e = j} w_e (a_e - m_{k_e})   (column-major N x 2R: b[c N + j])
template <int R>
__global__ void k_adj_cam_sum(int N, const int64_t* __restrict__ coff, const int64_t* __restrict__ cidx,
                              const int32_t* __restrict__ lmk, const double* __restrict__ ukp,
                              const double* __restrict__ w, const double* __restrict__ Y,
                              const double* __restrict__ lam, const double* __restrict__ m,
                              double* __restrict__ b) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    double acc[2 * R];
#pragma unroll
    for (int c = 0; c < 2 * R; ++c) acc[c] = 0.0;
    for (int64_t x = coff[j]; x < coff[j + 1]; ++x) {
      const int64_t e = cidx[x];
      double a[2 * R];
      obs_proj<R>(Y, lam, j, ukp + 3 * e, a);
      const double* mk = m + (size_t)lmk[e] * 2 * R;
#pragma unroll
      for (int c = 0; c < 2 * R; ++c) acc[c] += w[e] * (a[c] - mk[c]);
    }
#pragma unroll
    for (int c = 0; c < 2 * R; ++c) b[(size_t)c * N + j] = acc[c];
  }
}

// p_k = m_k + sum_{e in k} w_e t_{i_e} / d_k;  e_e = a_e + t_i - p_k;
// dL/du_e = -2 w_e (Y_i e_lambda + lambda_i e_Y),  dL/dw_e = -2 <e_lambda, e_Y>
template <int R>
__global__ void k_adj_out(int M, const int64_t* __restrict__ loff, const int64_t* __restrict__ lidx,
                          int N, const int32_t* __restrict__ cam, const double* __restrict__ ukp,
                          const double* __restrict__ w, const double* __restrict__ dk,
                          const double* __restrict__ Y, const double* __restrict__ lam,
                          const double* __restrict__ m, const double* __restrict__ t,
                          double* __restrict__ d_u, double* __restrict__ d_w) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double p[2 * R];
#pragma unroll
    for (int c = 0; c < 2 * R; ++c) p[c] = 0.0;
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) {
      const int64_t e = lidx[x];
      const int i = cam[e];
#pragma unroll
      for (int c = 0; c < 2 * R; ++c) p[c] += w[e] * t[(size_t)c * N + i];
    }
    const double inv = dk[k] > 0.0 ? 1.0 / dk[k] : 0.0;
#pragma unroll
    for (int c = 0; c < 2 * R; ++c) p[c] = m[(size_t)k * 2 * R + c] + p[c] * inv;
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) {
      const int64_t e = lidx[x];
      const int i = cam[e];
      double a[2 * R];
      obs_proj<R>(Y, lam, i, ukp + 3 * e, a);
#pragma unroll
      for (int c = 0; c < 2 * R; ++c) a[c] += t[(size_t)c * N + i] - p[c];
      double gw = 0.0;
#pragma unroll
      for (int j = 0; j < R; ++j) gw += a[j] * a[R + j];
      const double we = w[e];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < R; ++j)
          s += Y[(size_t)(3 * i + c) * R + j] * a[R + j] + lam[(size_t)(3 * i + c) * R + j] * a[j];
        d_u[3 * e + c] = -2.0 * we * s;
      }
      d_w[e] = -2.0 * gw;
    }
  }
}

namespace {

struct Buf {
  void* p = nullptr;
  ~Buf() { if (p) cudaFree(p); }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

int grid_cap(size_t work, int threads, int num_sms) {
  size_t g = (work + threads - 1) / threads;
  const size_t cap = (size_t)num_sms * 8;
  return (int)std::max<size_t>(1, std::min(g, cap));
}

}  // namespace

template <int R>
static xm_status backward_impl(xm_ctx* ctx, const DeviceQ& q, const xm_opts& o, int r,
                               const double* Yin, int ldy, int M, int64_t E, const int32_t* cam,
                               const int32_t* lmk, const double* ukp, const double* w,
                               const double* dL_dG, double* d_u, double* d_w, double* lam_out,
                               xm_adj_info* info) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  cudaStream_t st = ctx->stream;
  const int N = q.N, n = q.n, n_pad = q.n_pad;
  const int nb_cam = (N + CAM_THREADS - 1) / CAM_THREADS;
  const bool fp64 = o.prec == XM_FP64;
  const size_t rows = (size_t)n_pad, vec64 = rows * R * sizeof(double);
  XM_TRY(validate_obs(ctx, N, M, E, cam, lmk, ukp, w));
  XM_TRY(ensure_partials(ctx, (size_t)std::max(nb_cam, 1) * 3 * R + 64));
  long launches = 0;
  xm_adj_info inf{};

  // ---- vectors (FP64: Y, G, Lam, g_L, lambda, res, Wd; inner: Y, G, eta, Heta, r, d, Hd, Wd)
  Buf bY, bG, bLam, bgL, blam, bres, bWd, bsc, bYi, bGi, beta, bHeta, br, bd, bHd, bWi;
  for (Buf* b : {&bY, &bG, &bgL, &blam, &bres, &bWd}) {
    XM_CUDA_TRY(cudaMalloc(&b->p, vec64));
    XM_CUDA_TRY(cudaMemsetAsync(b->p, 0, vec64, st));
  }
  XM_CUDA_TRY(cudaMalloc(&bLam.p, sizeof(double) * 9 * (size_t)N));
  XM_CUDA_TRY(cudaMalloc(&bsc.p, sizeof(Scal)));
  XM_CUDA_TRY(cudaMemsetAsync(bsc.p, 0, sizeof(Scal), st));
  Scal* sc = bsc.as<Scal>();
  Scal hs{};
  auto pull = [&]() -> xm_status {
    XM_CUDA_TRY(cudaMemcpyAsync(&hs, sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    return check_device_error(ctx, "xm_backward");
  };
  const size_t vin = rows * R * (fp64 ? sizeof(double) : sizeof(float));
  if (!fp64) {
    for (Buf* b : {&bYi, &bGi, &beta, &bHeta, &br, &bd, &bHd, &bWi}) {
      XM_CUDA_TRY(cudaMalloc(&b->p, vin));
      XM_CUDA_TRY(cudaMemsetAsync(b->p, 0, vin, st));
    }
  } else {
    for (Buf* b : {&bGi, &beta, &bHeta, &br, &bd, &bHd, &bWi}) {
      XM_CUDA_TRY(cudaMalloc(&b->p, vin));
      XM_CUDA_TRY(cudaMemsetAsync(b->p, 0, vin, st));
    }
  }
  k_repad<double, double><<<grid_cap(rows * R, 256, ctx->num_sms), 256, 0, st>>>(
      n, n_pad, Yin, ldy, bY.as<double>(), R);
  // the first r columns only: zero what lies beyond r (ldy may exceed r)
  if (ldy > r) {
    // k_repad copied min(ldy, R) columns; clear columns r..R-1
    for (int c = r; c < R; ++c)
      XM_CUDA_TRY(cudaMemset2DAsync(bY.as<double>() + c, sizeof(double) * R, 0, sizeof(double), n, st));
  }
  launches += 1;

  // ---- 1. FP64 gradient at Y (dual blocks), g_L = P_Y(dL/dY)
  XM_TRY(qy_launch(ctx, q, XM_FP64, R, bY.p, bWd.p, nullptr, st));
  ++inf.n_sweeps_fp64;
  k_grad_epi<double, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, bY.as<double>(), bWd.as<double>(),
                                                        bG.as<double>(), bLam.as<double>(), sc, 0,
                                                        ctx->d_partials, ctx->d_counter, ctx->d_err);
  k_adj_dY<R><<<nb_cam, CAM_THREADS, 0, st>>>(N, bY.as<double>(), dL_dG, bgL.as<double>(),
                                              ctx->d_partials, ctx->d_counter);
  k_adj_proj<R><<<nb_cam, CAM_THREADS, 0, st>>>(N, bY.as<double>(), bgL.as<double>(), sc,
                                                ctx->d_partials, ctx->d_counter);
  launches += 4;
  XM_CUDA_TRY(cudaGetLastError());
  XM_TRY(pull());
  const double gnorm = std::sqrt(hs.dot);
  inf.g_norm = gnorm;
  inf.grad_norm_Y = std::sqrt(hs.g2);

  // ---- 2. Hess[lambda] = g_L: CG, FP64 residual refinement around an FP32 inner solve
  const double target = o.grad_tol_rel * gnorm;
  xm_status result = XM_OK;
  double res = gnorm;
  if (gnorm > 0.0) {
    const void* Yinner = bY.p;
    if (!fp64) {
      k_cast<double, float><<<grid_cap(rows * R, 256, ctx->num_sms), 256, 0, st>>>(
          rows * R, bY.as<double>(), bYi.as<float>());
      ++launches;
      Yinner = bYi.p;
    }
    for (int it = 0;; ++it) {
      // res = g_L - Hess[lambda] (FP64 operator); lambda = 0 at it = 0 needs no sweep
      if (it > 0) {
        XM_TRY(qy_launch(ctx, q, XM_FP64, R, blam.p, bWd.p, nullptr, st));
        ++inf.n_sweeps_fp64;
        ++launches;
      }
      if (fp64)
        k_adj_resid<double, R><<<nb_cam, CAM_THREADS, 0, st>>>(
            N, bY.as<double>(), bWd.as<double>(), blam.as<double>(), bgL.as<double>(),
            bLam.as<double>(), bres.as<double>(), bGi.as<double>(), sc, ctx->d_partials,
            ctx->d_counter);
      else
        k_adj_resid<float, R><<<nb_cam, CAM_THREADS, 0, st>>>(
            N, bY.as<double>(), bWd.as<double>(), blam.as<double>(), bgL.as<double>(),
            bLam.as<double>(), bres.as<double>(), bGi.as<float>(), sc, ctx->d_partials,
            ctx->d_counter);
      ++launches;
      XM_CUDA_TRY(cudaGetLastError());
      XM_TRY(pull());
      res = std::sqrt(hs.dot);
      inf.n_refine = it;
      if (!std::isfinite(res)) { result = set_error(XM_ENUMERIC, "xm_backward: non-finite residual"); break; }
      if (res <= target) break;
      if (it >= std::max(1, o.max_polish)) {
        result = set_error(XM_ENOCONV, "xm_backward: adjoint residual %.3e of %.3e after %d refinements",
                           res, gnorm, it);
        break;
      }
      // inner solve Hess[delta] = res, eta = delta
      const double tol_in = fp64 ? std::max(target / res, 1e-15) : std::max(target / res, 1e-4);
      const int prec_in = fp64 ? XM_FP64 : XM_FP32_BULK;
      auto inner = [&](auto tag) -> xm_status {
        using Ti = decltype(tag);
        k_tcg_init<Ti, Ti, R><<<grid_cap(rows * R, CAM_THREADS, ctx->num_sms), CAM_THREADS, 0, st>>>(
            (int)rows, bGi.as<Ti>(), beta.as<Ti>(), bHeta.as<Ti>(), br.as<Ti>(), bd.as<Ti>(), sc,
            res * res, 0.0, o.max_tcg, 0.0, tol_in);
        ++launches;
        const int CH = 4;
        int done = 0;
        for (int j = 0; j < o.max_tcg && !done; j += CH) {
          for (int c = 0; c < CH; ++c) {
            XM_TRY(qy_launch(ctx, q, prec_in, R, bd.p, bWi.p, &sc->done, st));
            if (fp64) ++inf.n_sweeps_fp64; else ++inf.n_sweeps_fp32;
            k_cg_epi<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, (const Ti*)Yinner, bWi.as<Ti>(), bd.as<Ti>(),
                                                            bHd.as<Ti>(), bLam.as<double>(), sc,
                                                            ctx->d_partials, ctx->d_counter);
            k_tcg_update<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(
                N, (const Ti*)Yinner, beta.as<Ti>(), bHeta.as<Ti>(), br.as<Ti>(), bd.as<Ti>(),
                bHd.as<Ti>(), sc, ctx->d_partials, ctx->d_counter);
            k_tcg_dir<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, beta.as<Ti>(), br.as<Ti>(), bd.as<Ti>(),
                                                             sc, ctx->d_partials, ctx->d_counter);
            launches += 4;
          }
          XM_CUDA_TRY(cudaGetLastError());
          XM_CUDA_TRY(cudaMemcpyAsync(&hs.done, &sc->done, sizeof(int), cudaMemcpyDeviceToHost, st));
          XM_CUDA_TRY(cudaStreamSynchronize(st));
          done = hs.done;
        }
        XM_TRY(pull());
        inf.n_cg += hs.iters;
        k_axpy_to64<Ti><<<grid_cap(rows * R, 256, ctx->num_sms), 256, 0, st>>>(
            rows * R, beta.as<Ti>(), blam.as<double>());
        ++launches;
        XM_CUDA_TRY(cudaGetLastError());
        return XM_OK;
      };
      if (fp64) XM_TRY(inner(double{}));
      else XM_TRY(inner(float{}));
    }
  }
  inf.res_rel = gnorm > 0.0 ? res / gnorm : 0.0;
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  const auto t1 = clk::now();
  inf.t_lambda_s = std::chrono::duration<double>(t1 - t0).count();
  if (result != XM_OK && result != XM_ENOCONV) return result;

  // ---- 3. optimal residuals of [Y, lambda] and the output gradients
  {
    Buf loff, lidx, coff, cidx, S, dk, m, b;
    XM_CUDA_TRY(cudaMalloc(&loff.p, sizeof(int64_t) * ((size_t)M + 1)));
    XM_CUDA_TRY(cudaMalloc(&coff.p, sizeof(int64_t) * ((size_t)N + 1)));
    XM_CUDA_TRY(cudaMalloc(&lidx.p, sizeof(int64_t) * (size_t)std::max<int64_t>(E, 1)));
    XM_CUDA_TRY(cudaMalloc(&cidx.p, sizeof(int64_t) * (size_t)std::max<int64_t>(E, 1)));
    XM_CUDA_TRY(cudaMalloc(&S.p, sizeof(double) * (size_t)N * N));
    XM_CUDA_TRY(cudaMalloc(&dk.p, sizeof(double) * (size_t)std::max(M, 1)));
    XM_CUDA_TRY(cudaMalloc(&m.p, sizeof(double) * (size_t)std::max(M, 1) * 2 * R));
    XM_CUDA_TRY(cudaMalloc(&b.p, sizeof(double) * (size_t)N * 2 * R));
    XM_TRY(obs_csr(ctx, E, lmk, M, loff.as<int64_t>(), lidx.as<int64_t>()));
    XM_TRY(obs_csr(ctx, E, cam, N, coff.as<int64_t>(), cidx.as<int64_t>()));
    XM_TRY(schur_S_factor(ctx, N, M, cam, w, coff.as<int64_t>(), cidx.as<int64_t>(),
                          loff.as<int64_t>(), lidx.as<int64_t>(), S.as<double>(), dk.as<double>()));
    const int gl = grid_cap((size_t)M, 128, ctx->num_sms * 4);
    k_adj_lmk_mean<R><<<gl, 128, 0, st>>>(M, loff.as<int64_t>(), lidx.as<int64_t>(), cam, ukp, w,
                                          dk.as<double>(), bY.as<double>(), blam.as<double>(),
                                          m.as<double>());
    k_adj_cam_sum<R><<<grid_cap((size_t)N, 64, ctx->num_sms * 4), 64, 0, st>>>(
        N, coff.as<int64_t>(), cidx.as<int64_t>(), lmk, ukp, w, bY.as<double>(), blam.as<double>(),
        m.as<double>(), b.as<double>());
    XM_CUDA_TRY(cudaGetLastError());
    XM_TRY(schur_S_solve(ctx, N, S.as<double>(), b.as<double>(), 2 * R));
    k_adj_out<R><<<gl, 128, 0, st>>>(M, loff.as<int64_t>(), lidx.as<int64_t>(), N, cam, ukp, w,
                                     dk.as<double>(), bY.as<double>(), blam.as<double>(),
                                     m.as<double>(), b.as<double>(), d_u, d_w);
    launches += 3;
    XM_CUDA_TRY(cudaGetLastError());
    if (lam_out)
      k_repad<double, double><<<grid_cap((size_t)n * r, 256, ctx->num_sms), 256, 0, st>>>(
          n, n, blam.as<double>(), R, lam_out, r);
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    XM_TRY(check_device_error(ctx, "xm_backward"));
  }
  const auto t2 = clk::now();
  inf.t_resid_s = std::chrono::duration<double>(t2 - t1).count();
  inf.t_total_s = std::chrono::duration<double>(t2 - t0).count();
  inf.launches = launches;
  if (info) *info = inf;
  return result;
}

}  // namespace xm

using namespace xm;

extern "C" xm_status xm_backward(xm_ctx* c, const xm_qmat* q, const xm_opts* opts, int r,
                                 const double* Y, int ldy, int M, int64_t E, const int32_t* cam,
                                 const int32_t* lmk, const double* ukp, const double* w,
                                 const double* dL_dG, double* dL_dukp, double* dL_dw,
                                 double* lam_out, xm_adj_info* info) {
  if (!c || !q || !opts || !Y || !dL_dG || !dL_dukp || !dL_dw)
    return set_error(XM_EINVAL, "xm_backward: NULL argument");
  if (E > 0 && (!cam || !lmk || !ukp || !w)) return set_error(XM_EINVAL, "xm_backward: NULL observations");
  if (r < 3 || r > XM_MAX_RANK) return set_error(XM_EINVAL, "xm_backward: r=%d not in [3, %d]", r, XM_MAX_RANK);
  if (ldy < r) return set_error(XM_EINVAL, "xm_backward: ldy=%d < r=%d", ldy, r);
  if (M < 0 || E < 0) return set_error(XM_EINVAL, "xm_backward: negative size");
  const DeviceQ& d = q->d;
  if (!d.q64) return set_error(XM_EINVAL, "xm_backward: Q has no FP64 copy (residual refinement needs it)");
  if (opts->prec != XM_FP64 && !d.q32)
    return set_error(XM_EINVAL, "xm_backward: Q has no FP32 copy for the inner solve (use prec XM_FP64)");
  XM_CUDA_TRY(cudaSetDevice(c->device));
  if (r <= 4)
    return backward_impl<4>(c, d, *opts, r, Y, ldy, M, E, cam, lmk, ukp, w, dL_dG, dL_dukp, dL_dw,
                            lam_out, info);
  return backward_impl<8>(c, d, *opts, r, Y, ldy, M, E, cam, lmk, ukp, w, dL_dG, dL_dukp, dL_dw,
                          lam_out, info);
}
