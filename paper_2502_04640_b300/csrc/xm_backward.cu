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
//   2. Hess[lambda] = g_L by conjugate gradients on the Q sweep, preconditioned by
//      (Z + gamma Pi_Y)^-1 (Z the certificate matrix; an explicit FP32 inverse packed like Q and
//      applied by the same sweep, n <= 40000) or else by Z's per-camera 3 x 3 diagonal blocks,
//      projected onto the tangent space: FP64 operator for prec FP64; otherwise FP32 inner CG
//      with FP64 residual refinement (mixed-precision iterative refinement: each refinement
//      step solves Hess[delta] = g_L - Hess64[lambda] in FP32).
//   3. The optimal residuals of the 2R columns [Y, lambda]: landmark means, camera sums, the
//      anchored translation solve with the Cholesky factor of Sbar, then the outputs.

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <vector>

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
// CG's right side Gin = res in its storage type; sc->dot = ||res||^2
template <typename Ti, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_adj_resid(int N, const double* __restrict__ Y, double* __restrict__ Wd,
            const double* __restrict__ lam, const double* __restrict__ gL,
            const double* __restrict__ Lam, double* __restrict__ res, Ti* __restrict__ Gin,
            Scal* sc, double* partials, unsigned* counter) {
  double v[1] = {0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    hvp_block<double, R>(i, N, Y, Wd, lam, res, Lam, sc->mu);
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
        Gin[(size_t)(3 * i + a) * R + j] = Ti(h[a][j]);
      }
    store_block<double, double, R>(res, i, h);
    v[0] = s;
  }
  grid_reduce<1>(v, partials, counter, [&](double* t) { sc->dot = t[0]; });
}

// CG step length alpha = <r, z> / <p, Hess p> (z = M^-1 r); a non-positive curvature ends the
// solve (the operator is positive semi-definite at a certified optimum and the right side lies
// in its range)
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_cg_epi(int N, const T* __restrict__ Y, T* __restrict__ Wd, const T* __restrict__ delta,
         T* __restrict__ Hd, const double* __restrict__ Lam, Scal* sc, double* partials,
         unsigned* counter) {
  if (sc->done) return;
  double v[1] = {0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) v[0] = hvp_block<T, R, T>(i, N, Y, Wd, delta, Hd, Lam, sc->mu);
  grid_reduce<1>(v, partials, counter, [&](double* t) {
    sc->kappa = t[0];
    if (!(t[0] > 0.0)) { sc->done = 1; sc->reason = 1; return; }
    sc->alpha = sc->rz / t[0];
  });
}

// ---- block-Jacobi preconditioner of the Riemannian Hessian

// Per camera, Minv_i = (2 Z_ii)^-1 with Z_ii = Q_ii + diag(0, 0, dreg_i) - Lambda_i, the 3 x 3
// diagonal block of the certificate matrix (positive semi-definite at a certified optimum),
// eigenvalues clamped below at 1e-8 of the largest; the preconditioner is the tangent
// projection of the block-diagonal left multiplication, z_i = P_{Y_i}(Minv_i r_i).
__global__ void k_adj_precond(int N, const double* __restrict__ q64, int nt,
                              const double* __restrict__ Lam, double* __restrict__ Minv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double Z[3][3], V[3][3], d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      Z[a][b] = q_entry(q64, nt, 3 * i + a, 3 * i + b) - Lam[(size_t)9 * i + 3 * a + b];
  Z[2][2] += Lam[(size_t)9 * N + i];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a + 1; b < 3; ++b) { const double m = 0.5 * (Z[a][b] + Z[b][a]); Z[a][b] = m; Z[b][a] = m; }
  jacobi3<double>(Z, V, d);
  const double dmax = fmax(d[0], fmax(d[1], d[2]));
  double inv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) inv[k] = dmax > 0.0 ? 0.5 / fmax(d[k], 1e-8 * dmax) : 1.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      Minv[(size_t)9 * i + 3 * a + b] =
          V[a][0] * inv[0] * V[b][0] + V[a][1] * inv[1] * V[b][1] + V[a][2] * inv[2] * V[b][2];
}

// z_i = P_{Y_i}(Minv_i r_i)
template <int R>
__device__ __forceinline__ void precond_block(int i, const double (&y)[3][R], const double (&r)[3][R],
                                              const double* __restrict__ Minv, double (&z)[3][R]) {
  double M[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) M[a][b] = Minv[(size_t)9 * i + 3 * a + b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) z[a][j] = M[a][0] * r[0][j] + M[a][1] * r[1][j] + M[a][2] * r[2][j];
  double S[3][3], al;
  dual_block<double, R>(z, y, i == 0, S, al);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) z[a][j] -= S[a][0] * y[0][j] + S[a][1] * y[1][j] + S[a][2] * y[2][j];
}

// ---- gauge deflation
// The Hessian of the rank-r problem vanishes on the orbit directions N = {Y Omega : Omega skew}
// (f(Y O) = f(Y) for orthogonal O); the right side and Hess's range are orthogonal to N, so the
// CG residual and the preconditioned residual are kept orthogonal to N.  The projection of v
// onto N is Y Omega with skew(Y^T v) = (G Omega + Omega G) / 2, G = Y^T Y: in the eigenbasis W
// of G (eigenvalues g), Omega~_ab = 2 (W^T skew(Y^T v) W)_ab / (g_a + g_b).
// defl = [W (R x R row-major), g (R), threshold]; C = Y^T v (R x R, C[a R + b]).
template <int R>
__device__ __forceinline__ void omega_from_C(const double* C, const double* __restrict__ defl,
                                             double* __restrict__ Om) {
  const double* W = defl;
  const double* g = defl + R * R;
  const double thr = defl[R * R + R];
  double B[R][R], T[R][R];
  for (int a = 0; a < R; ++a)
    for (int b = 0; b < R; ++b) B[a][b] = 0.5 * (C[a * R + b] - C[b * R + a]);
  for (int a = 0; a < R; ++a)        // T = W^T B
    for (int b = 0; b < R; ++b) {
      double t = 0.0;
      for (int k = 0; k < R; ++k) t += W[k * R + a] * B[k][b];
      T[a][b] = t;
    }
  for (int a = 0; a < R; ++a)        // B~ = T W, then divide
    for (int b = 0; b < R; ++b) {
      double t = 0.0;
      for (int k = 0; k < R; ++k) t += T[a][k] * W[k * R + b];
      const double den = g[a] + g[b];
      B[a][b] = den > thr ? 2.0 * t / den : 0.0;
    }
  for (int a = 0; a < R; ++a)        // Omega = W B~ W^T
    for (int b = 0; b < R; ++b) {
      double t = 0.0;
      for (int k = 0; k < R; ++k)
        for (int l = 0; l < R; ++l) t += W[a * R + k] * B[k][l] * W[b * R + l];
      Om[a * R + b] = t;
    }
}

// per-camera share of C = Y^T v, in the element type C of y and v (FP32 in the FP32 inner solve:
// B300's FP64 pipe is narrow), handed to the FP64 grid reduction
template <int R, typename C = double>
__device__ __forceinline__ void yt_v(const C (&y)[3][R], const C (&v)[3][R], double (&c)[R * R]) {
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) c[a * R + b] = double(y[0][a] * v[0][b] + y[1][a] * v[1][b] + y[2][a] * v[2][b]);
}

// x = 0, r = b (tangent), C = Y^T r -> Om; resets the CG scalars
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_pcg_begin(int N, const T* __restrict__ Y, const T* __restrict__ b, T* __restrict__ x,
            T* __restrict__ r, const double* __restrict__ defl, double* __restrict__ Om, Scal* sc,
            int max_iters, double tol, double* partials, unsigned* counter) {
  double v[R * R];
#pragma unroll
  for (int k = 0; k < R * R; ++k) v[k] = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double y[3][R], rr[3][R];
    load_block<T, double, R>(Y, i, y);
    load_block<T, double, R>(b, i, rr);
    yt_v<R>(y, rr, v);
    zero_block<T, R>(x, i);
    store_block<T, double, R>(r, i, rr);
  }
  grid_reduce<R * R>(v, partials, counter, [&](double* t) {
    omega_from_C<R>(t, defl, Om);
    sc->done = 0; sc->iters = 0; sc->max_iters = max_iters; sc->reason = 0; sc->kappa_tol = tol;
  });
}

// x += alpha p, r -= alpha Hp (re-projected onto the tangent space), C = Y^T r -> Om
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_pcg_update(int N, const T* __restrict__ Y, T* __restrict__ x, T* __restrict__ r,
             const T* __restrict__ p, const T* __restrict__ Hp, const double* __restrict__ defl,
             double* __restrict__ Om, Scal* sc, double* partials, unsigned* counter) {
  if (sc->done) return;
  const double alpha = sc->alpha;
  double v[R * R];
#pragma unroll
  for (int k = 0; k < R * R; ++k) v[k] = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    using C = T;   // per-camera arithmetic in the inner solve's precision
    const C at = C(alpha);
    C y[3][R], xx[3][R], rr[3][R], pp[3][R], hp[3][R];
    load_block<T, C, R>(Y, i, y);
    load_block<T, C, R>(x, i, xx);
    load_block<T, C, R>(r, i, rr);
    load_block<T, C, R>(p, i, pp);
    load_block<T, C, R>(Hp, i, hp);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) { xx[a][j] += at * pp[a][j]; rr[a][j] -= at * hp[a][j]; }
    C S[3][3], al;
    dual_block<C, R>(rr, y, i == 0, S, al);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) rr[a][j] -= S[a][0] * y[0][j] + S[a][1] * y[1][j] + S[a][2] * y[2][j];
    yt_v<R, C>(y, rr, v);
    store_block<T, C, R>(x, i, xx);
    store_block<T, C, R>(r, i, rr);
  }
  grid_reduce<R * R>(v, partials, counter, [&](double* t) { omega_from_C<R>(t, defl, Om); });
}

// v -= Y Om (deflation); optionally also writes v in FP32 (n_pad x R, row-major) as the input
// of the dense preconditioner's sweep
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_deflate(int N, const T* __restrict__ Y, T* __restrict__ v, const double* __restrict__ Om,
          float* __restrict__ col, const Scal* sc) {
  if (sc->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double y[3][R], vv[3][R], O[R][R];
  load_block<T, double, R>(Y, i, y);
  load_block<T, double, R>(v, i, vv);
#pragma unroll
  for (int a = 0; a < R; ++a)
#pragma unroll
    for (int b = 0; b < R; ++b) O[a][b] = Om[a * R + b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < R; ++k) t += y[a][k] * O[k][j];
      vv[a][j] -= t;
      if (col) col[(size_t)(3 * i + a) * R + j] = float(vv[a][j]);
    }
  store_block<T, double, R>(v, i, vv);
}

// block-Jacobi preconditioner: z = P_Y(Minv r), C = Y^T z -> Om
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_precond_bj(int N, const T* __restrict__ Y, const T* __restrict__ r, T* __restrict__ z,
             const double* __restrict__ Minv, const double* __restrict__ defl, double* __restrict__ Om,
             Scal* sc, double* partials, unsigned* counter) {
  if (sc->done) return;
  double v[R * R];
#pragma unroll
  for (int k = 0; k < R * R; ++k) v[k] = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double y[3][R], rr[3][R], zz[3][R];
    load_block<T, double, R>(Y, i, y);
    load_block<T, double, R>(r, i, rr);
    precond_block<R>(i, y, rr, Minv, zz);
    yt_v<R>(y, zz, v);
    store_block<T, double, R>(z, i, zz);
  }
  grid_reduce<R * R>(v, partials, counter, [&](double* t) { omega_from_C<R>(t, defl, Om); });
}

// dense preconditioner, after the sweep with its inverse: z = P_Y(col / 2), C = Y^T z -> Om;
// col (the sweep's output, n_pad x R row-major) is zeroed for the next sweep's accumulation
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_precond_from_col(int N, const T* __restrict__ Y, float* __restrict__ col, T* __restrict__ z,
                   const double* __restrict__ defl, double* __restrict__ Om, Scal* sc,
                   double* partials, unsigned* counter) {
  if (sc->done) return;
  double v[R * R];
#pragma unroll
  for (int k = 0; k < R * R; ++k) v[k] = 0.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    using C = T;   // per-camera arithmetic in the inner solve's precision
    C y[3][R], zz[3][R];
    load_block<T, C, R>(Y, i, y);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        float* c = col + (size_t)(3 * i + a) * R + j;
        zz[a][j] = C(0.5) * C(*c);
        *c = 0.0f;
      }
    C S[3][3], al;
    dual_block<C, R>(zz, y, i == 0, S, al);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) zz[a][j] -= S[a][0] * y[0][j] + S[a][1] * y[1][j] + S[a][2] * y[2][j];
    yt_v<R, C>(y, zz, v);
    store_block<T, C, R>(z, i, zz);
  }
  grid_reduce<R * R>(v, partials, counter, [&](double* t) { omega_from_C<R>(t, defl, Om); });
}

// z -= Y Om (deflation); <r, r>, <r, z>; first call (init): p = z, r0; later: residual test and
// beta = <r, z>' / <r, z>
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_pcg_rz(int N, const T* __restrict__ Y, const T* __restrict__ r, T* __restrict__ z,
         T* __restrict__ p, const double* __restrict__ Om, int init, Scal* sc, double* partials,
         unsigned* counter) {
  if (sc->done) return;
  double v[2] = {0.0, 0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    using C = T;   // per-camera arithmetic in the inner solve's precision, sums in FP64
    C y[3][R], rr[3][R], zz[3][R], O[R][R];
    load_block<T, C, R>(Y, i, y);
    load_block<T, C, R>(r, i, rr);
    load_block<T, C, R>(z, i, zz);
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) O[a][b] = C(Om[a * R + b]);
    C s0 = C(0), s1 = C(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        C t = C(0);
#pragma unroll
        for (int k = 0; k < R; ++k) t += y[a][k] * O[k][j];
        zz[a][j] -= t;
        s0 += rr[a][j] * rr[a][j];
        s1 += rr[a][j] * zz[a][j];
      }
    v[0] = double(s0);
    v[1] = double(s1);
    store_block<T, C, R>(z, i, zz);
    if (init) store_block<T, C, R>(p, i, zz);
  }
  grid_reduce<2>(v, partials, counter, [&](double* t) {
    sc->rr = t[0];
    if (init) {
      sc->r0 = sqrt(t[0]); sc->rz = t[1];
      if (!(t[0] > 0.0) || !(t[1] > 0.0)) { sc->done = 1; sc->reason = 3; }
      return;
    }
    sc->iters += 1;
    if (sqrt(t[0]) <= sc->r0 * sc->kappa_tol) { sc->done = 1; sc->reason = 3; }
    else if (sc->iters >= sc->max_iters) { sc->done = 1; sc->reason = 4; }
    else if (!(t[1] > 0.0)) { sc->done = 1; sc->reason = 5; }
    else { sc->beta = t[1] / sc->rz; sc->rz = t[1]; }
  });
}

// dense Z + gamma Pi_Y (FP32, column-major n x n): Q + diag(dreg) - blockdiag(Lambda) +
// gamma Y G^+ Y^T, the preconditioner's matrix (Pi_Y = Y G^+ Y^T projects onto range(Y), the
// null space of Z at a certified optimum)
template <int R>
__global__ void k_dense_Z(int N, const double* __restrict__ q64, int nt, const double* __restrict__ Lam,
                          const double* __restrict__ Y, const double* __restrict__ Gp, double gamma,
                          float* __restrict__ Z) {
  const int n = 3 * N;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n), rr = (int)(e % n);
    double v = q_entry(q64, nt, rr, c);
    if (rr / 3 == c / 3) {
      const int i = rr / 3;
      v -= Lam[(size_t)9 * i + 3 * (rr % 3) + (c % 3)];
      if (rr == c && rr % 3 == 2) v += Lam[(size_t)9 * N + i];
    }
    double t = 0.0;
#pragma unroll
    for (int a = 0; a < R; ++a) {
      double u = 0.0;
#pragma unroll
      for (int b = 0; b < R; ++b) u += Gp[a * R + b] * Y[(size_t)c * R + b];
      t += Y[(size_t)rr * R + a] * u;
    }
    Z[e] = float(v + gamma * t);
  }
}

// p = z + beta p
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_pcg_dir(int N, const T* __restrict__ z, T* __restrict__ p, const Scal* sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int e = 3 * i * R; e < 3 * (i + 1) * R; ++e) p[e] = T(double(z[e]) + beta * double(p[e]));
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
  void reset() { if (p) cudaFree(p); p = nullptr; }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

int grid_cap(size_t work, int threads, int num_sms) {
  size_t g = (work + threads - 1) / threads;
  const size_t cap = (size_t)num_sms * 8;
  return (int)std::max<size_t>(1, std::min(g, cap));
}

}  // namespace

// cyclic Jacobi eigen-decomposition of a small symmetric m x m matrix (row-major):
// A = V diag(w) V^T, V's columns the eigenvectors
static void small_sym_eig(int m, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        tot += A[(size_t)i * m + j] * A[(size_t)i * m + j];
        if (i != j) off += A[(size_t)i * m + j] * A[(size_t)i * m + j];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double th = 0.5 * (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / apq;
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {   // A <- J^T A J
          const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
          A[(size_t)k * m + p] = c * akp - s * akq;
          A[(size_t)k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
          A[(size_t)p * m + k] = c * apk - s * aqk;
          A[(size_t)q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[(size_t)k * m + p], vkq = V[(size_t)k * m + q];
          V[(size_t)k * m + p] = c * vkp - s * vkq;
          V[(size_t)k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(m);
  for (int i = 0; i < m; ++i) w[i] = A[(size_t)i * m + i];
}

// Largest n for which the dense preconditioner is factored (n x n FP32: 6.4 GB at the limit);
// above it the block-Jacobi preconditioner is used.
constexpr int DENSE_PRECOND_MAX_N = 40000;

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
  XM_TRY(ensure_partials(ctx, (size_t)std::max(3 * nb_cam, ctx->num_sms * 4) * R * R + 64));
  long launches = 0;
  xm_adj_info inf{};

  // ---- vectors (FP64: Y, G, Lam, g_L, lambda, res, Wd; inner: Y, G, eta, Heta, r, d, Hd, Wd)
  Buf bY, bG, bLam, bMinv, bgL, blam, bres, bWd, bsc, bYi, bGi, beta, bHeta, br, bd, bHd, bWi;
  Buf bsmall, bZ, bcol, bcol2;
  struct TilesGuard { DeviceQ q; ~TilesGuard() { free_tiles(q); } } Pinv;
  for (Buf* b : {&bY, &bG, &bgL, &blam, &bres, &bWd}) {
    XM_CUDA_TRY(cudaMalloc(&b->p, vec64));
    XM_CUDA_TRY(cudaMemsetAsync(b->p, 0, vec64, st));
  }
  XM_CUDA_TRY(cudaMalloc(&bLam.p, sizeof(double) * lam_doubles(N)));
  XM_CUDA_TRY(cudaMalloc(&bMinv.p, sizeof(double) * 9 * (size_t)N));
  // small: G = Y^T Y | defl = [W, g, thr] | G^+ | Omega
  const int SM_G = 0, SM_DEFL = R * R, SM_GP = 2 * R * R + R + 1, SM_OM = 3 * R * R + R + 1;
  XM_CUDA_TRY(cudaMalloc(&bsmall.p, sizeof(double) * (4 * R * R + R + 1)));
  XM_CUDA_TRY(cudaMemsetAsync(bsmall.p, 0, sizeof(double) * (4 * R * R + R + 1), st));
  double* dsm = bsmall.as<double>();
  XM_CUDA_TRY(cudaMalloc(&bsc.p, sizeof(Scal)));
  XM_CUDA_TRY(cudaMemsetAsync(bsc.p, 0, sizeof(Scal), st));
  Scal* sc = bsc.as<Scal>();
  XM_CUDA_TRY(cudaMemcpyAsync(&sc->mu, &o.scale_reg, sizeof(double), cudaMemcpyHostToDevice, st));
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
  k_gram<double, R><<<std::max(1, std::min(nb_cam * 3, ctx->num_sms * 4)), CAM_THREADS, 0, st>>>(
      n_pad, bY.as<double>(), dsm + SM_G, ctx->d_partials, ctx->d_counter);
  launches += 5;
  XM_CUDA_TRY(cudaGetLastError());
  XM_TRY(pull());
  const double gnorm = std::sqrt(hs.dot);
  inf.g_norm = gnorm;
  inf.grad_norm_Y = std::sqrt(hs.g2);

  // ---- preconditioner data: deflation basis of the gauge directions, Pi_Y, gamma, Z's factor
  const auto tp0 = clk::now();
  {
    std::vector<double> G(R * R), gw, W, host(4 * R * R + R + 1, 0.0);
    XM_CUDA_TRY(cudaMemcpy(G.data(), dsm + SM_G, sizeof(double) * R * R, cudaMemcpyDeviceToHost));
    small_sym_eig(R, G, gw, W);
    double gmax = 0.0;
    for (double x : gw) gmax = std::max(gmax, x);
    for (int k = 0; k < R * R; ++k) host[SM_DEFL + k] = W[k];
    for (int k = 0; k < R; ++k) host[SM_DEFL + R * R + k] = gw[k];
    host[SM_DEFL + R * R + R] = 1e-12 * gmax;
    for (int a = 0; a < R; ++a)
      for (int b = 0; b < R; ++b) {
        double t = 0.0;
        for (int k = 0; k < R; ++k)
          if (gw[k] > 1e-10 * gmax) t += W[a * R + k] * W[b * R + k] / gw[k];
        host[SM_GP + a * R + b] = t;
      }
    XM_CUDA_TRY(cudaMemcpy(dsm + SM_DEFL, host.data() + SM_DEFL, sizeof(double) * (2 * R * R + R + 1),
                           cudaMemcpyHostToDevice));
    // gamma: the mean Frobenius norm of the dual blocks over sqrt(3), the curvature scale the
    // dense preconditioner gives to range(Y)
    std::vector<double> Lh((size_t)9 * N);
    XM_CUDA_TRY(cudaMemcpy(Lh.data(), bLam.p, sizeof(double) * 9 * N, cudaMemcpyDeviceToHost));
    double gsum = 0.0;
    for (int i = 0; i < N; ++i) {
      double f2 = 0.0;
      for (int k = 0; k < 9; ++k) f2 += Lh[(size_t)9 * i + k] * Lh[(size_t)9 * i + k];
      gsum += std::sqrt(f2);
    }
    const double gamma = gsum / (std::sqrt(3.0) * N) + 1e-300;
    inf.dense_precond = 0;
    if (n <= DENSE_PRECOND_MAX_N && gnorm > 0.0) {
      XM_CUDA_TRY(cudaMalloc(&bZ.p, sizeof(float) * (size_t)n * n));
      k_dense_Z<R><<<grid_cap((size_t)n * n, 256, ctx->num_sms * 4), 256, 0, st>>>(
          N, q.q64, q.nt, bLam.as<double>(), bY.as<double>(), dsm + SM_GP, gamma, bZ.as<float>());
      ++launches;
      XM_CUDA_TRY(cudaGetLastError());
      // Explicit inverse (this library's tensor-core SPD inverse, FP32 accuracy), packed into
      // FP32 upper-triangle tiles: applying it is then one Q.Y-style sweep per CG step, which
      // streams n^2/2 floats at the sweep's HBM rate, where triangular solves with a factor are
      // long chains of small dependent steps.  A preconditioner needs no more accuracy than
      // the FP32 inverse gives; a matrix that is not numerically positive definite falls back
      // to block Jacobi.
      const xm_status si = spd_inverse_f32(ctx, bZ.as<float>(), n, n, nullptr);
      if (si != XM_OK && si != XM_ENUMERIC) return si;
      launches += g_last_launches;
      if (si == XM_OK) {
        XM_TRY(alloc_tiles(ctx, Pinv.q, N, XM_STORE_FP32));
        XM_TRY(pack_dense_f32(ctx, Pinv.q, bZ.as<float>()));
        ++launches;
        const size_t colb = sizeof(float) * rows * R;
        XM_CUDA_TRY(cudaMalloc(&bcol.p, colb));
        XM_CUDA_TRY(cudaMalloc(&bcol2.p, colb));
        XM_CUDA_TRY(cudaMemsetAsync(bcol.p, 0, colb, st));
        XM_CUDA_TRY(cudaMemsetAsync(bcol2.p, 0, colb, st));
        inf.dense_precond = 1;
      }
      XM_CUDA_TRY(cudaStreamSynchronize(st));   // the packing has read the inverse
      bZ.reset();
    }
    if (!inf.dense_precond) {
      k_adj_precond<<<nb_cam, CAM_THREADS, 0, st>>>(N, q.q64, q.nt, bLam.as<double>(), bMinv.as<double>());
      ++launches;
      XM_CUDA_TRY(cudaGetLastError());
    }
    inf.gamma = gamma;
  }
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  inf.t_precond_s = std::chrono::duration<double>(clk::now() - tp0).count();
  const bool dense = inf.dense_precond != 0;

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
      const double res_prev = res;
      res = std::sqrt(hs.dot);
      inf.n_refine = it;
      if (!std::isfinite(res)) { result = set_error(XM_ENUMERIC, "xm_backward: non-finite residual"); break; }
      if (res <= target) break;
      // a pass that no longer halves the residual has reached the floor set by how stationary
      // Y is (Hess is singular along the gauge directions only at an exact critical point)
      if (it >= 2 && res > 0.5 * res_prev) {
        if (res > 1e-6 * gnorm)
          result = set_error(XM_ENOCONV, "xm_backward: adjoint residual stalled at %.3e of %.3e", res, gnorm);
        break;
      }
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
        const Ti* Yi = (const Ti*)Yinner;
        double* Om = dsm + SM_OM;
        const double* defl = dsm + SM_DEFL;
        // z = deflated, projected M^-1 r (r already deflated)
        auto precond = [&]() -> xm_status {
          if (dense) {
            XM_TRY(qy_launch(ctx, Pinv.q, XM_FP32_BULK, R, bcol.p, bcol2.p, &sc->done, st));
            ++launches;
            k_precond_from_col<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(
                N, Yi, bcol2.as<float>(), bHeta.as<Ti>(), defl, Om, sc, ctx->d_partials, ctx->d_counter);
          } else {
            k_precond_bj<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(
                N, Yi, br.as<Ti>(), bHeta.as<Ti>(), bMinv.as<double>(), defl, Om, sc, ctx->d_partials,
                ctx->d_counter);
          }
          ++launches;
          return XM_OK;
        };
        float* col = dense ? bcol.as<float>() : nullptr;
        k_pcg_begin<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, Yi, bGi.as<Ti>(), beta.as<Ti>(), br.as<Ti>(),
                                                          defl, Om, sc, o.max_tcg, tol_in,
                                                          ctx->d_partials, ctx->d_counter);
        k_deflate<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, Yi, br.as<Ti>(), Om, col, sc);
        XM_TRY(precond());
        k_pcg_rz<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, Yi, br.as<Ti>(), bHeta.as<Ti>(), bd.as<Ti>(), Om,
                                                        1, sc, ctx->d_partials, ctx->d_counter);
        launches += 3;
        XM_CUDA_TRY(cudaGetLastError());
        const int CH = 4;
        int done = 0;
        for (int j = 0; j < o.max_tcg && !done; j += CH) {
          for (int c = 0; c < CH; ++c) {
            XM_TRY(qy_launch(ctx, q, prec_in, R, bd.p, bWi.p, &sc->done, st));
            if (fp64) ++inf.n_sweeps_fp64; else ++inf.n_sweeps_fp32;
            k_cg_epi<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, Yi, bWi.as<Ti>(), bd.as<Ti>(), bHd.as<Ti>(),
                                                            bLam.as<double>(), sc, ctx->d_partials,
                                                            ctx->d_counter);
            k_pcg_update<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, Yi, beta.as<Ti>(), br.as<Ti>(), bd.as<Ti>(),
                                                               bHd.as<Ti>(), defl, Om, sc, ctx->d_partials,
                                                               ctx->d_counter);
            k_deflate<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, Yi, br.as<Ti>(), Om, col, sc);
            XM_TRY(precond());
            k_pcg_rz<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, Yi, br.as<Ti>(), bHeta.as<Ti>(), bd.as<Ti>(),
                                                            Om, 0, sc, ctx->d_partials, ctx->d_counter);
            k_pcg_dir<Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, bHeta.as<Ti>(), bd.as<Ti>(), sc);
            launches += 6;
          }
          XM_CUDA_TRY(cudaGetLastError());
          XM_CUDA_TRY(cudaMemcpyAsync(&hs.done, &sc->done, sizeof(int), cudaMemcpyDeviceToHost, st));
          XM_CUDA_TRY(cudaStreamSynchronize(st));
          done = hs.done;
        }
        XM_TRY(pull());
        inf.n_cg += hs.iters;
        if (o.verbose >= 1)
          fprintf(stderr, "[xm] adjoint pass %d: |res| %.3e (target %.3e) inner CG %d its, stop %d, "
                  "last curvature %.3e, inner |r| %.3e\n", it, res, target, hs.iters, hs.reason,
                  hs.kappa, std::sqrt(hs.rr));
        k_axpy_to64<Ti><<<grid_cap(rows * R, 256, ctx->num_sms), 256, 0, st>>>(
            rows * R, beta.as<Ti>(), blam.as<double>());
        // an FP32 correction is tangent at the FP32-rounded Y: keep lambda tangent at Y in FP64
        k_adj_proj<R><<<nb_cam, CAM_THREADS, 0, st>>>(N, bY.as<double>(), blam.as<double>(), sc,
                                                      ctx->d_partials, ctx->d_counter);
        launches += 2;
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
  if (!(opts->scale_reg >= 0.0) || !std::isfinite(opts->scale_reg))
    return set_error(XM_EINVAL, "xm_backward: scale_reg must be finite and >= 0");
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
