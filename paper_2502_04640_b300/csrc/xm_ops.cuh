// Per-camera and vector kernels of the solver (Sec. 3.2): gradient / Hessian epilogues with
// the closed-form dual blocks, tangent projection, polar retraction, truncated-CG updates with
// device-resident scalars, Lanczos helpers and rounding.  Layout: every n x r quantity is an
// n_pad x R row-major array (R = 4 or 8, unused columns zero), camera i owns rows 3i..3i+2.
#pragma once
#include "xm_internal.cuh"

namespace xm {

// Scalars of one RTR step, resident on the device (the tCG loop never waits for the host).
struct Scal {
  double f, g2, y2;          // objective, ||rgrad||^2, ||Y||^2 at the current point
  double fc, gc2, yc2;       // the same at the candidate point
  double Delta;              // trust-region radius
  double rr, r0, rz;         // <r, r>, ||r_0||, <r, M^-1 r> (preconditioned CG)
  double ee, ed, dd;         // <eta,eta>, <eta,delta>, <delta,delta>
  double kappa, alpha, beta; // curvature, step, CG coefficient
  double theta, kappa_tol;   // residual-based stop: ||r|| <= r0 min(r0^theta, kappa_tol)
  double g_eta, eta_Heta, eta2;  // model terms of the step
  double dot;                // generic reduction result
  double mu;                 // App. D scale-regularisation weight (0: plain Eq. 17 objective)
  double thr_min;            // floor of the residual stop: no tighter than the phase's tolerance
  double df;                 // f(candidate) - f(current) in difference form (RTR ratio test)
  int done, stop_after, iters, max_iters, reason, pad_;
};

// The dual-block arrays hold N row-major 3 x 3 blocks Lambda_i followed by N values
// dreg_i = 2 mu (x_i - 1), x_i = X_{3i+2,3i+2} = ||row 2 of Y_i||^2 (0 for the anchor): the
// diagonal of grad_X F of App. D's regulariser F(X) = mu sum_{i>=1} (x_i - 1)^2, which acts on
// the third row of every non-anchor block.  Z = Q + diag(dreg) - blockdiag(Lambda).
__host__ __device__ inline size_t lam_doubles(int N) { return (size_t)10 * N; }

constexpr int CAM_THREADS = 64;   // per-camera kernels: 10155 cameras -> 159 blocks

// ------------------------------------------------------------------ reductions
// Deterministic grid reduction of K per-thread values: block sums -> partials[b*K+k]; the last
// block to finish adds the partials in block order and thread 0 calls fin(total).
template <int K, typename Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[K], double* partials, unsigned* counter,
                                            Fin fin) {
  __shared__ double sh[K][CAM_THREADS / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) sh[k][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < CAM_THREADS / 32; ++w) s += sh[k][w];
      partials[(size_t)blockIdx.x * K + k] = s;
    }
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // every thread of the last block adds a fixed stride of the partials, then a fixed tree
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += static_cast<volatile double*>(partials)[(size_t)b * K + k];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      tot[k] = 0.0;
      for (int w = 0; w < CAM_THREADS / 32; ++w) tot[k] += sh[k][w];
    }
    fin(tot);
    *counter = 0u;
    __threadfence();
  }
}

// ------------------------------------------------------------------ small dense algebra
// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (Golub & Van Loan, Sec. 8.5):
// A = V diag(d) V^T, V orthogonal (columns = eigenvectors).
template <typename C>
__device__ __forceinline__ void jacobi3(C (&A)[3][3], C (&V)[3][3], C (&d)[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? C(1) : C(0);
  for (int sweep = 0; sweep < 12; ++sweep) {
    const C off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    const C diag = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
    if (off <= C(1e-30) + diag * (sizeof(C) == 8 ? C(1e-17) : C(1e-8))) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const C apq = A[p][q];
      if (fabs(apq) <= C(1e-300)) continue;
      const C tau = (A[q][q] - A[p][p]) / (C(2) * apq);
      const C t = (tau >= C(0) ? C(1) : C(-1)) / (fabs(tau) + sqrt(C(1) + tau * tau));
      const C c = C(1) / sqrt(C(1) + t * t), s = t * c;
      // A <- J^T A J with J = rotation in the (p, q) plane
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const C akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - s * akq;
        A[k][q] = s * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const C apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - s * aqk;
        A[q][k] = s * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const C vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
    }
  }
  d[0] = A[0][0]; d[1] = A[1][1]; d[2] = A[2][2];
}

template <typename C>
__device__ __forceinline__ C det3(const C (&A)[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// Closed-form dual block (Thm. 1 / App. C): Lambda = P_i(sym(X Y^T)) / alpha with
// alpha = ||Y||_F^2 / 3; P_i removes the trace except on the anchor (i = 0).
template <typename C, int R>
__device__ __forceinline__ void dual_block(const C (&X)[3][R], const C (&Y)[3][R], bool anchor,
                                          C (&L)[3][3], C& alpha) {
  C y2 = C(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) y2 += Y[a][j] * Y[a][j];
  alpha = y2 / C(3);
  C M[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      C s = C(0);
#pragma unroll
      for (int j = 0; j < R; ++j) s += X[a][j] * Y[b][j];
      M[a][b] = s;
    }
  const C tr3 = anchor ? C(0) : (M[0][0] + M[1][1] + M[2][2]) / C(3);
  const C inv = alpha > C(0) ? C(1) / alpha : C(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      L[a][b] = (C(0.5) * (M[a][b] + M[b][a]) - (a == b ? tr3 : C(0))) * inv;
}

template <typename T, typename C, int R>
__device__ __forceinline__ void load_block(const T* p, int i, C (&X)[3][R]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) X[a][j] = C(p[(size_t)(3 * i + a) * R + j]);
}
template <typename T, typename C, int R>
__device__ __forceinline__ void store_block(T* p, int i, const C (&X)[3][R]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) p[(size_t)(3 * i + a) * R + j] = T(X[a][j]);
}
template <typename T, int R>
__device__ __forceinline__ void zero_block(T* p, int i) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) p[(size_t)(3 * i + a) * R + j] = T(0);
}

// ------------------------------------------------------------------ gradient epilogue
// From W = Q Y: Lambda_i, rgrad_i = 2 (W_i - Lambda_i Y_i), f = <Y, W>, ||rgrad||^2, ||Y||^2
// (with App. D's regulariser: W_i + dreg_i e_3 e_3^T Y_i in place of W_i, f + F(X)).
// W is reset to zero for the next accumulating sweep.  Results go to (sc->f, g2, y2) or, with
// cand = 1, to (sc->fc, gc2, yc2).
// Camera i's share: Lambda_i (and dreg_i) into Lam, rgrad_i into G, W_i reset to zero;
// returns (f_i, ||rgrad_i||^2, ||Y_i||^2) in v.
// C: per-camera arithmetic type (FP64 in the grid-wide kernels whatever the storage type; the
// batched solver's FP32 bulk phase uses FP32).
template <typename T, int R, typename C = double>
__device__ __forceinline__ void grad_block(int i, int N, const T* __restrict__ Y, T* __restrict__ W,
                                           T* __restrict__ G, double* __restrict__ Lam, double mu,
                                           double (&v)[3]) {
  C y[3][R], w[3][R], L[3][3], alpha;
  load_block<T, C, R>(Y, i, y);
  load_block<T, C, R>(W, i, w);
  zero_block<T, R>(W, i);
  C fi = C(0), gi = C(0), yi = C(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) fi += y[a][j] * w[a][j];   // tr(Y^T Q Y)
  // App. D regulariser: f += mu (x_i - 1)^2, (Q + grad F) Y adds dreg_i * row 2 of Y_i
  C dreg = C(0);
  if (mu != 0.0 && i > 0) {
    C x2 = C(0);
#pragma unroll
    for (int j = 0; j < R; ++j) x2 += y[2][j] * y[2][j];
    dreg = C(2) * C(mu) * (x2 - C(1));
    fi += C(mu) * (x2 - C(1)) * (x2 - C(1));
#pragma unroll
    for (int j = 0; j < R; ++j) w[2][j] += dreg * y[2][j];
  }
  dual_block<C, R>(w, y, i == 0, L, alpha);
  C g[3][R];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      C ly = L[a][0] * y[0][j] + L[a][1] * y[1][j] + L[a][2] * y[2][j];
      g[a][j] = C(2) * (w[a][j] - ly);
      gi += g[a][j] * g[a][j];
      yi += y[a][j] * y[a][j];
    }
  store_block<T, C, R>(G, i, g);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Lam[(size_t)9 * i + 3 * a + b] = double(L[a][b]);
  Lam[(size_t)9 * N + i] = double(dreg);
  v[0] = double(fi); v[1] = double(gi); v[2] = double(yi);
}

template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_grad_epi(int N, const T* __restrict__ Y, T* __restrict__ W, T* __restrict__ G,
           double* __restrict__ Lam, Scal* sc, int cand, double* partials, unsigned* counter,
           int* err) {
  double v[3] = {0.0, 0.0, 0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) grad_block<T, R>(i, N, Y, W, G, Lam, sc->mu, v);
  grid_reduce<3>(v, partials, counter, [&](double* t) {
    if (!isfinite(t[0]) || !isfinite(t[1])) atomicOr(err, DEV_NUMERIC);
    if (cand) { sc->fc = t[0]; sc->gc2 = t[1]; sc->yc2 = t[2]; }
    else { sc->f = t[0]; sc->g2 = t[1]; sc->y2 = t[2]; }
  });
}

// ------------------------------------------------------------------ truncated CG
// Steihaug-Toint tCG (Absil et al. 2008, Alg. 11) on the model with Hessian 2 P_Y(Q d - Lambda d),
// optionally preconditioned (Conn, Gould and Toint's form): z = M^-1 r with the block-Jacobi
// preconditioner z_i = P_{Y_i}(Minv_i r_i), Minv_i = (2 (Q_ii + eps I))^-1; the trust region is
// then measured in the M-norm, whose <eta,M eta>, <eta,M delta>, <delta,M delta> follow by
// recurrences (no product with M).  Minv == nullptr: z = r, the plain method.

template <typename C, int R>
__device__ __forceinline__ void tcg_precond(int i, const C (&y)[3][R], const C (&r)[3][R],
                                            const double* __restrict__ Minv, C (&z)[3][R]) {
  if (!Minv) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) z[a][j] = r[a][j];
    return;
  }
  C M[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) M[a][b] = C(Minv[(size_t)9 * i + 3 * a + b]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) z[a][j] = M[a][0] * r[0][j] + M[a][1] * r[1][j] + M[a][2] * r[2][j];
  C S[3][3], al;
  dual_block<C, R>(z, y, i == 0, S, al);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) z[a][j] -= S[a][0] * y[0][j] + S[a][1] * y[1][j] + S[a][2] * y[2][j];
}

// eta = Heta = 0, r = G, z = M^-1 r, delta = -z; <r, r>, <r, z>
template <typename To, typename Ti, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_tcg_init(int N, const Ti* __restrict__ Y, const To* __restrict__ G, Ti* eta, Ti* Heta, Ti* r, Ti* z,
           Ti* delta, const double* __restrict__ Minv, Scal* sc, double Delta, int max_iters,
           double theta, double kappa_tol, double thr_min, double* partials, unsigned* counter) {
  using C = double;
  double v[2] = {0.0, 0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    C y[3][R], rr[3][R], zz[3][R], zero[3][R];
    load_block<Ti, C, R>(Y, i, y);
    load_block<To, C, R>(G, i, rr);
    tcg_precond<C, R>(i, y, rr, Minv, zz);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        v[0] += rr[a][j] * rr[a][j];
        v[1] += rr[a][j] * zz[a][j];
        zero[a][j] = C(0);
      }
    store_block<Ti, C, R>(r, i, rr);
    store_block<Ti, C, R>(z, i, zz);
    store_block<Ti, C, R>(eta, i, zero);
    store_block<Ti, C, R>(Heta, i, zero);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) zz[a][j] = -zz[a][j];
    store_block<Ti, C, R>(delta, i, zz);
  }
  grid_reduce<2>(v, partials, counter, [&](double* t) {
    sc->Delta = Delta;
    sc->rr = t[0];
    sc->rz = t[1];
    sc->r0 = sqrt(t[0]);
    sc->ee = 0.0; sc->ed = 0.0; sc->dd = t[1];
    sc->done = (t[0] > 0.0 && t[1] > 0.0) ? 0 : 1;
    sc->stop_after = 0; sc->iters = 0; sc->max_iters = max_iters; sc->reason = 0;
    sc->theta = theta; sc->kappa_tol = kappa_tol; sc->thr_min = thr_min;
  });
}

// Hd_i = 2 P_{Y_i}(Wd_i - Lambda_i d_i) for camera i (Wd_i is reset to zero for the next
// accumulating sweep); returns <d_i, Hd_i>.
// With App. D's regulariser the Euclidean Hessian adds, on row 2 of every non-anchor block,
// dreg_i d_i + 4 mu <y_i, d_i> y_i (row-2 vectors): the derivative of dreg_i y_i along d.
template <typename T, int R, typename C = double>
__device__ __forceinline__ double hvp_block(int i, int N, const T* __restrict__ Y, T* __restrict__ Wd,
                                            const T* __restrict__ delta, T* __restrict__ Hd,
                                            const double* __restrict__ Lam, double mu) {
  C y[3][R], w[3][R], d[3][R], L[3][3];
  load_block<T, C, R>(Y, i, y);
  load_block<T, C, R>(Wd, i, w);
  zero_block<T, R>(Wd, i);
  load_block<T, C, R>(delta, i, d);
  if (mu != 0.0 && i > 0) {
    const C dreg = C(Lam[(size_t)9 * N + i]);
    C yd = C(0);
#pragma unroll
    for (int j = 0; j < R; ++j) yd += y[2][j] * d[2][j];
#pragma unroll
    for (int j = 0; j < R; ++j) w[2][j] += dreg * d[2][j] + C(4) * C(mu) * yd * y[2][j];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) L[a][b] = C(Lam[(size_t)9 * i + 3 * a + b]);
  C A[3][R];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j)
      A[a][j] = C(2) * (w[a][j] - (L[a][0] * d[0][j] + L[a][1] * d[1][j] + L[a][2] * d[2][j]));
  C S[3][3], alpha;
  dual_block<C, R>(A, y, i == 0, S, alpha);
  C kap = C(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      A[a][j] -= S[a][0] * y[0][j] + S[a][1] * y[1][j] + S[a][2] * y[2][j];
      kap += d[a][j] * A[a][j];
    }
  store_block<T, C, R>(Hd, i, A);
  return double(kap);
}

// Hd = 2 P_Y(Wd - Lambda d); kappa = <d, Hd>; then decide the step (alpha, or tau to the
// trust-region boundary on negative curvature / when the CG step leaves the region).
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_hvp_epi(int N, const T* __restrict__ Y, T* __restrict__ Wd, const T* __restrict__ delta,
          T* __restrict__ Hd, const double* __restrict__ Lam, Scal* sc, double* partials,
          unsigned* counter) {
  if (sc->done) return;
  double v[1] = {0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) v[0] = hvp_block<T, R, T>(i, N, Y, Wd, delta, Hd, Lam, sc->mu);
  grid_reduce<1>(v, partials, counter, [&](double* t) {
    const double kap = t[0];
    sc->kappa = kap;
    const double D2 = sc->Delta * sc->Delta;
    const double a = kap > 0.0 ? sc->rz / kap : 0.0;
    if (!(kap > 0.0) || sc->ee + 2.0 * a * sc->ed + a * a * sc->dd >= D2) {
      const double disc = sc->ed * sc->ed + sc->dd * (D2 - sc->ee);
      sc->alpha = (-sc->ed + sqrt(disc > 0.0 ? disc : 0.0)) / sc->dd;
      sc->stop_after = 1;
      sc->reason = kap > 0.0 ? 2 : 1;
    } else {
      sc->alpha = a;
    }
  });
}

// eta += alpha d, Heta += alpha Hd, r += alpha Hd (re-projected), z = M^-1 r; residual test on
// ||r||, beta = <r, z>' / <r, z>; M-norm recurrences for <eta,M eta>, <eta,M d>, <d,M d>.
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_tcg_update(int N, const T* __restrict__ Y, T* eta, T* Heta, T* r, T* z, const T* __restrict__ delta,
             const T* __restrict__ Hd, const double* __restrict__ Minv, Scal* sc, double* partials,
             unsigned* counter) {
  if (sc->done) return;
  // per-camera arithmetic in the vectors' precision (B300's FP64 rate is 1/64 of its FP32 rate:
  // FP64 here had made the tCG epilogues slower than the sweep on the 2000-camera trajectory);
  // the reductions accumulate in FP64
  using C = T;
  const C alpha = C(sc->alpha);
  const bool stop = sc->stop_after != 0;
  double v[2] = {0.0, 0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    C e[3][R], he[3][R], d[3][R], hd[3][R];
    load_block<T, C, R>(eta, i, e);
    load_block<T, C, R>(Heta, i, he);
    load_block<T, C, R>(delta, i, d);
    load_block<T, C, R>(Hd, i, hd);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        e[a][j] += alpha * d[a][j];
        he[a][j] += alpha * hd[a][j];
      }
    store_block<T, C, R>(eta, i, e);
    store_block<T, C, R>(Heta, i, he);
    if (!stop) {
      C rr[3][R], y[3][R], zz[3][R];
      load_block<T, C, R>(r, i, rr);
      load_block<T, C, R>(Y, i, y);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < R; ++j) rr[a][j] += alpha * hd[a][j];
      C S[3][3], al;
      dual_block<C, R>(rr, y, i == 0, S, al);   // re-project r onto the tangent space
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < R; ++j) rr[a][j] -= S[a][0] * y[0][j] + S[a][1] * y[1][j] + S[a][2] * y[2][j];
      tcg_precond<C, R>(i, y, rr, Minv, zz);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          v[0] += double(rr[a][j]) * double(rr[a][j]);
          v[1] += double(rr[a][j]) * double(zz[a][j]);
        }
      store_block<T, C, R>(r, i, rr);
      store_block<T, C, R>(z, i, zz);
    }
  }
  grid_reduce<2>(v, partials, counter, [&](double* t) {
    sc->iters += 1;
    const double a = sc->alpha;
    sc->ee = sc->ee + 2.0 * a * sc->ed + a * a * sc->dd;   // <eta, M eta> after the step
    if (stop) { sc->done = 1; return; }
    const double rr_new = t[0], rz_new = t[1];
    const double rn = sqrt(rr_new);
    const double thr = fmax(sc->r0 * fmin(pow(sc->r0, sc->theta), sc->kappa_tol), sc->thr_min);
    if (rn <= thr) { sc->done = 1; sc->reason = 3; return; }
    if (sc->iters >= sc->max_iters) { sc->done = 1; sc->reason = 4; return; }
    if (!(rz_new > 0.0)) { sc->done = 1; sc->reason = 5; return; }
    const double beta = rz_new / sc->rz;
    sc->beta = beta;
    sc->ed = beta * (sc->ed + a * sc->dd);
    sc->dd = rz_new + beta * beta * sc->dd;
    sc->rz = rz_new;
    sc->rr = rr_new;
  });
}

// delta = -z + beta delta
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_tcg_dir(int N, const T* __restrict__ z, T* delta, const Scal* sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T b = T(beta);
  for (int e = 3 * i * R; e < 3 * (i + 1) * R; ++e) delta[e] = -z[e] + b * delta[e];
}

// model terms <grad, eta>, <eta, Heta>, ||eta||^2 after tCG
template <typename To, typename Ti, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_model_terms(int n_rows, const To* __restrict__ G, const Ti* __restrict__ eta,
              const Ti* __restrict__ Heta, Scal* sc, double* partials, unsigned* counter) {
  double v[3] = {0.0, 0.0, 0.0};
  const size_t total = (size_t)n_rows * R;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const double g = double(G[e]), x = double(eta[e]), h = double(Heta[e]);
    v[0] += g * x; v[1] += x * h; v[2] += x * x;
  }
  grid_reduce<3>(v, partials, counter, [&](double* t) {
    sc->g_eta = t[0]; sc->eta_Heta = t[1]; sc->eta2 = t[2];
  });
}

// ------------------------------------------------------------------ retraction
// Metric projection onto {sqrt(a) * (3 x r with orthonormal rows)}: A = Y_i + s Xi_i,
// polar(A) = (A A^T)^{-1/2} A, scale = (sum of singular values) / 3 (anchor: 1).
template <typename To, typename Ti, int R, typename C = double>
__device__ __forceinline__ void retract_block(int i, const To* __restrict__ Y, const Ti* __restrict__ Xi,
                                              double s, To* __restrict__ Yo) {
  C A[3][R];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j)
      A[a][j] = C(Y[(size_t)(3 * i + a) * R + j]) + C(s) * C(Xi[(size_t)(3 * i + a) * R + j]);
  // work with A / ||A||_F so that the 3x3 eigenproblem is scale free (blocks can shrink far
  // towards zero on the way to a scale-collapsed stationary point)
  C fro = C(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j) fro += A[a][j] * A[a][j];
  fro = sqrt(fro);
  const C ifro = fro > C(0) ? C(1) / fro : C(0);
  C M[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      C t = C(0);
#pragma unroll
      for (int j = 0; j < R; ++j) t += (A[a][j] * ifro) * (A[b][j] * ifro);
      M[a][b] = t;
    }
  C V[3][3], d[3];
  jacobi3<C>(M, V, d);
  C sq[3], isq[3];
  C ssum = C(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const C dk = d[k] > C(1e-30) ? d[k] : C(1e-30);   // eigenvalues of the unit-norm problem
    sq[k] = sqrt(dk);
    isq[k] = ifro / sq[k];                             // (A A^T)^{-1/2} = V diag(1/(|A| sqrt d)) V^T
    ssum += sq[k];
  }
  const C scale = i == 0 ? C(1) : fro * ssum / C(3);
  C P[3][3];   // scale * V diag(1/sqrt d) V^T
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      P[a][b] = scale * (V[a][0] * isq[0] * V[b][0] + V[a][1] * isq[1] * V[b][1] +
                         V[a][2] * isq[2] * V[b][2]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < R; ++j)
      Yo[(size_t)(3 * i + a) * R + j] = To(P[a][0] * A[0][j] + P[a][1] * A[1][j] + P[a][2] * A[2][j]);
}

template <typename To, typename Ti, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_retract(int N, const To* __restrict__ Y, const Ti* __restrict__ Xi, double s, To* __restrict__ Yo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) retract_block<To, Ti, R>(i, Y, Xi, s, Yo);
}

// ------------------------------------------------------------------ element-wise helpers
template <typename Ts, typename Td>
__global__ void k_cast(size_t total, const Ts* __restrict__ s, Td* __restrict__ d) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    d[e] = Td(s[e]);
}

// copy an n x rs row-major array into an n_rows x Rd padded one (zero fill), any types
template <typename Ts, typename Td>
__global__ void k_repad(int n, int n_rows, const Ts* __restrict__ s, int rs, Td* __restrict__ d,
                        int Rd) {
  const size_t total = (size_t)n_rows * Rd;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / Rd), col = (int)(e % Rd);
    d[e] = (row < n && col < rs) ? Td(s[(size_t)row * rs + col]) : Td(0);
  }
}

// Y <- Y Rot (R x R matrix in device memory), rows independent
template <int R>
__global__ void k_rotate(int n_rows, double* Y, const double* __restrict__ Rot) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  double y[R], o[R];
#pragma unroll
  for (int j = 0; j < R; ++j) y[j] = Y[(size_t)row * R + j];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < R; ++k) s += y[k] * Rot[k * R + j];
    o[j] = s;
  }
#pragma unroll
  for (int j = 0; j < R; ++j) Y[(size_t)row * R + j] = o[j];
}

// G = Y^T Y (R x R), deterministic
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_gram(int n_rows, const T* __restrict__ Y, double* out, double* partials, unsigned* counter) {
  double v[R * R];
#pragma unroll
  for (int k = 0; k < R * R; ++k) v[k] = 0.0;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n_rows;
       row += gridDim.x * blockDim.x) {
    double y[R];
#pragma unroll
    for (int j = 0; j < R; ++j) y[j] = double(Y[(size_t)row * R + j]);
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) v[a * R + b] += y[a] * y[b];
  }
  grid_reduce<R * R>(v, partials, counter, [&](double* t) {
    for (int k = 0; k < R * R; ++k) out[k] = t[k];
  });
}

// C = A^T B (R x R) for two n_rows x R row-major arrays, deterministic
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_cross(int n_rows, const T* __restrict__ A, const T* __restrict__ B, double* out, double* partials,
        unsigned* counter) {
  double v[R * R];
#pragma unroll
  for (int k = 0; k < R * R; ++k) v[k] = 0.0;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n_rows;
       row += gridDim.x * blockDim.x) {
    double a[R], b[R];
#pragma unroll
    for (int j = 0; j < R; ++j) { a[j] = double(A[(size_t)row * R + j]); b[j] = double(B[(size_t)row * R + j]); }
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int y = 0; y < R; ++y) v[x * R + y] += a[x] * b[y];
  }
  grid_reduce<R * R>(v, partials, counter, [&](double* t) {
    for (int k = 0; k < R * R; ++k) out[k] = t[k];
  });
}

// <a, b> over total elements (mixed types) -> *out
template <typename Ta, typename Tb>
__global__ void __launch_bounds__(CAM_THREADS)
k_dot(size_t total, const Ta* __restrict__ a, const Tb* __restrict__ b, double* out,
      double* partials, unsigned* counter) {
  double v[1] = {0.0};
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    v[0] += double(a[e]) * double(b[e]);
  grid_reduce<1>(v, partials, counter, [&](double* t) { *out = t[0]; });
}

// ------------------------------------------------------------------ Lanczos (FP64 vectors)
// w_i = Wz_i + dreg_i e_3 e_3^T v_i - Lambda_i v_i (Z v with Z = Q + diag(dreg) -
// blockdiag(Lambda), App. D; dreg = 0 without the regulariser); Wz reset to zero.
template <typename Tw, typename Tv = double>
__global__ void k_zv_epi(int N, Tw* __restrict__ Wz, const Tv* __restrict__ v,
                         const double* __restrict__ Lam, double* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x[3] = {double(v[3 * i]), double(v[3 * i + 1]), double(v[3 * i + 2])};
  const double dreg = Lam[(size_t)9 * N + i];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double lx = Lam[9 * i + 3 * a] * x[0] + Lam[9 * i + 3 * a + 1] * x[1] +
                      Lam[9 * i + 3 * a + 2] * x[2];
    w[3 * i + a] = double(Wz[3 * i + a]) - lx + (a == 2 ? dreg * x[2] : 0.0);
    Wz[3 * i + a] = Tw(0);
  }
}

// F(X) = mu sum_{i>=1} (x_i - 1)^2 and <grad F(X), X> = sum_i dreg_i x_i for the dual value of
// App. E (sc->dot, sc->kappa)
template <int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_reg_terms(int N, const double* __restrict__ Y, Scal* sc, double* partials, unsigned* counter) {
  double v[2] = {0.0, 0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > 0 && i < N) {
    double x2 = 0.0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const double t = Y[(size_t)(3 * i + 2) * R + j];
      x2 += t * t;
    }
    v[0] = sc->mu * (x2 - 1.0) * (x2 - 1.0);
    v[1] = 2.0 * sc->mu * (x2 - 1.0) * x2;
  }
  grid_reduce<2>(v, partials, counter, [&](double* t) { sc->dot = t[0]; sc->kappa = t[1]; });
}

// The Lanczos basis V (column-major, stride ld) is FP32 when the Z products are FP32 sweeps
// (orthogonality to ~1e-7 matches their accuracy; the per-element work then runs on the FP32
// pipes, B300's FP64 rate being ~2 FMA per clock per SM) and FP64 otherwise.  Working vectors
// (w), recurrence coefficients and Ritz values are FP64 in both cases.

// c[j] = <V_j, w> for the m columns of V; one block per column; also writes cf = float(c).
// w is given in the basis type (an FP32 copy of the FP64 working vector for an FP32 basis).
template <typename VT>
__global__ void k_gemv_t(int n, int m, const VT* __restrict__ V, size_t ld, const VT* __restrict__ w,
                         double* __restrict__ c, float* __restrict__ cf) {
  __shared__ double sh[8];
  for (int j = blockIdx.x; j < m; j += gridDim.x) {
    VT s = VT(0);
    const VT* col = V + (size_t)j * ld;
    for (int e = threadIdx.x; e < n; e += blockDim.x) s += col[e] * w[e];
    double sd = warp_sum(double(s));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = sd;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
      c[j] = t;
      if (cf) cf[j] = float(t);
    }
    __syncthreads();
  }
}

// w -= V c (m columns); cf = float(c) for an FP32 basis, c itself for an FP64 one
template <typename VT>
__global__ void k_gemv_n_sub(int n, int m, const VT* __restrict__ V, size_t ld, const double* __restrict__ c,
                             const float* __restrict__ cf, double* __restrict__ w) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    VT s = VT(0);
    if (sizeof(VT) == 4) {
      for (int j = 0; j < m; ++j) s += V[(size_t)j * ld + e] * VT(cf[j]);
    } else {
      for (int j = 0; j < m; ++j) s += V[(size_t)j * ld + e] * VT(c[j]);
    }
    w[e] -= double(s);
  }
}

// Partial sums of V c over column chunks: part[s][e] = sum_{j in chunk s} V[j][e] c_j (chunk s =
// columns [s*chunk, min(m, (s+1)*chunk)), one grid row per chunk), so that the product streams V
// with every SM busy; k_gemv_n_finish adds the chunks in a fixed order (deterministic).
template <typename VT>
__global__ void k_gemv_n_part(int n, int m, const VT* __restrict__ V, size_t ld,
                              const double* __restrict__ c, const float* __restrict__ cf, int chunk,
                              double* __restrict__ part) {
  const int j0 = blockIdx.y * chunk;
  const int j1 = min(m, j0 + chunk);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    VT s = VT(0);
    if (sizeof(VT) == 4) {
      for (int j = j0; j < j1; ++j) s += V[(size_t)j * ld + e] * VT(cf[j]);
    } else {
      for (int j = j0; j < j1; ++j) s += V[(size_t)j * ld + e] * VT(c[j]);
    }
    part[(size_t)blockIdx.y * n + e] = double(s);
  }
}
// w -= sum_s part[s] (chunks in order)
static __global__ void k_gemv_n_finish(int n, int S, const double* __restrict__ part, double* __restrict__ w) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int s = 0; s < S; ++s) t += part[(size_t)s * n + e];
    w[e] -= t;
  }
}

// w -= a[k] v_k + b[k-1] v_{k-1}  (coefficients read on the device)
template <typename VT>
__global__ void k_lanczos_3term(int n, double* __restrict__ w, const VT* __restrict__ vk,
                                const VT* __restrict__ vkm1, const double* alpha, const double* beta, int k) {
  const double a = alpha[k];
  const double b = (k > 0 && vkm1) ? beta[k - 1] : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    w[e] -= a * double(vk[e]) + (b != 0.0 ? b * double(vkm1[e]) : 0.0);
}

// dst = w / sqrt(*nrm2); *beta_out = sqrt(*nrm2)
template <typename VT>
__global__ void k_normalize(int n, const double* __restrict__ w, const double* nrm2, VT* __restrict__ dst,
                            double* beta_out) {
  const double b = sqrt(*nrm2);
  const double inv = b > 0.0 ? 1.0 / b : 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    dst[e] = VT(w[e] * inv);
  if (blockIdx.x == 0 && threadIdx.x == 0 && beta_out) *beta_out = b;
}

// column j of V (stride ld) from column j of a row-major n_rows x R array
template <typename VT, int R>
__global__ void k_col_from_rows(int n_rows, int j, const double* __restrict__ src, VT* __restrict__ col) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_rows; e += gridDim.x * blockDim.x)
    col[e] = VT(src[(size_t)e * R + j]);
}

// deterministic pseudo-random start vector (splitmix64 of (seed, index)), uniform in [-1, 1)
static __global__ void k_random_vec(int n, uint64_t seed, double* v) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(e + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[e] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

// ------------------------------------------------------------------ start point (Alg. 1)
// Camera i's block of [I_3, ..., I_3] padded to rank r (R stored columns), plus jitter times a
// splitmix64 uniform(-1, 1) fill of the columns 3..r-1 keyed by (seed, element index).
__device__ __forceinline__ void init_block(int i, int R, int r, double jitter, uint64_t seed, double* Y) {
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < R; ++j) {
      double v = (a == j) ? 1.0 : 0.0;
      if (j >= 3 && j < r && jitter != 0.0) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)((3 * i + a) * R + j + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v = jitter * ((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
      }
      Y[(size_t)(3 * i + a) * R + j] = v;
    }
}

// ------------------------------------------------------------------ rounding (Sec. 2.2)
// Per camera: Ubar_i = Yh_i^T (3 x 3), G_i = O0^T Ubar_i, s_i = ||G_i||_F / sqrt(3),
// R_i = SO(3) projection of G_i (SVD with determinant fix, Prop. 2); the anchor is (I, 1).
// Writes R (N x 9, row-major), s (N) and Yhat = [s_i R_i]^T (n_rows x 4, last column zero).
__device__ __forceinline__ void round_block(int i, const double* __restrict__ Yh,
                                            const double* __restrict__ O0, double* __restrict__ Rout,
                                            double* __restrict__ sout, double* __restrict__ Yhat) {
  double Rm[3][3], s;
  if (i == 0) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Rm[a][b] = a == b ? 1.0 : 0.0;
    s = 1.0;
  } else {
    double Ub[3][3], G[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Ub[a][b] = Yh[(size_t)(3 * i + b) * 4 + a];   // Yh_i^T
    double fro = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k) t += O0[3 * k + a] * Ub[k][b];
        G[a][b] = t;
        fro += t * t;
      }
    s = sqrt(fro / 3.0);
    // SVD via the eigen-decomposition of G^T G = V diag(sig^2) V^T, U = G V diag(1/sig)
    double M[3][3], V[3][3], d[3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k) t += G[k][a] * G[k][b];
        M[a][b] = t;
      }
    jacobi3<double>(M, V, d);
    double U[3][3];
    for (int k = 0; k < 3; ++k) {
      const double sig = sqrt(d[k] > 1e-300 ? d[k] : 1e-300);
      for (int a = 0; a < 3; ++a)
        U[a][k] = (G[a][0] * V[0][k] + G[a][1] * V[1][k] + G[a][2] * V[2][k]) / sig;
    }
    // the smallest singular direction takes the sign that makes det(R) = +1
    int kmin = 0;
    for (int k = 1; k < 3; ++k) if (d[k] < d[kmin]) kmin = k;
    const double sgn = det3<double>(U) * det3<double>(V) < 0.0 ? -1.0 : 1.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k) t += U[a][k] * (k == kmin ? sgn : 1.0) * V[b][k];
        Rm[a][b] = t;
      }
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      Rout[(size_t)9 * i + 3 * a + b] = Rm[a][b];
      Yhat[(size_t)(3 * i + b) * 4 + a] = s * Rm[a][b];
    }
  for (int b = 0; b < 3; ++b) Yhat[(size_t)(3 * i + b) * 4 + 3] = 0.0;
  sout[i] = s;
}

// G_i = s_i R_i (row-major 3 x 3) from the rounded Yhat (n_pad x 4 row-major, Yhat_i = G_i^T)
static __global__ void k_round_G(int N, const double* __restrict__ Yhat, double* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) G[(size_t)9 * i + 3 * a + b] = Yhat[(size_t)(3 * i + b) * 4 + a];
}

static __global__ void k_round(int N, const double* __restrict__ Yh, const double* __restrict__ O0,
                               double* __restrict__ Rout, double* __restrict__ sout,
                               double* __restrict__ Yhat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) round_block(i, Yh, O0, Rout, sout, Yhat);
}

}  // namespace xm
