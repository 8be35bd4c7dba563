// Solver driver: Alg. 1 (Riemannian staircase) around RTR-tCG (Sec. 3.2), the dual certificate
// of Thm. 1 with a Lanczos lambda_min, the escape of Thm. 2 and the rounding of Sec. 2.2.
// The host only takes per-step trust-region decisions; inside truncated CG the control flow
// (step length, boundary, negative curvature, residual test) runs on the device, so the host
// checks a done flag once per chunk of iterations.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "xm_ops.cuh"

namespace xm {

// ------------------------------------------------------------------ host linear algebra
// Cyclic Jacobi eigen-decomposition of a small symmetric matrix (Golub & Van Loan, Sec. 8.5),
// eigenvalues sorted in descending order, eigenvectors as the columns of V (row-major m x m).
static void sym_eig_desc(int m, std::vector<double> A, std::vector<double>& w,
                         std::vector<double>& V) {
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q) {
        const double a = A[(size_t)p * m + q];
        tot += a * a;
        if (p != q) off += a * a;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double tau = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < m; ++k) {
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
  std::vector<int> idx(m);
  for (int i = 0; i < m; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(),
            [&](int a, int b) { return A[(size_t)a * m + a] > A[(size_t)b * m + b]; });
  std::vector<double> V2((size_t)m * m);
  w.resize(m);
  for (int j = 0; j < m; ++j) {
    w[j] = A[(size_t)idx[j] * m + idx[j]];
    for (int k = 0; k < m; ++k) V2[(size_t)k * m + j] = V[(size_t)k * m + idx[j]];
  }
  V.swap(V2);
}

// Number of eigenvalues of the symmetric tridiagonal (a[0..k), b[0..k-1)) below x (Sturm).
static int sturm_count(int k, const double* a, const double* b, double x) {
  int c = 0;
  double q = a[0] - x;
  if (q < 0) ++c;
  for (int i = 1; i < k; ++i) {
    const double qq = (q == 0.0) ? 1e-300 : q;
    q = a[i] - x - b[i - 1] * b[i - 1] / qq;
    if (q < 0) ++c;
  }
  return c;
}

// j-th smallest eigenvalue (0-based) of the tridiagonal by bisection
static double tri_eig_bisect(int k, const double* a, const double* b, int j) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  const double span = std::max(std::fabs(lo), std::fabs(hi)) + 1e-300;
  for (int it = 0; it < 200 && hi - lo > 1e-16 * span; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(k, a, b, mid) > j) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Eigenvector of the tridiagonal for eigenvalue th by inverse iteration with a tridiagonal
// LU factorisation with partial pivoting.
static void tri_eigvec(int k, const double* a, const double* b, double th, std::vector<double>& s) {
  s.assign(k, 0.0);
  if (k == 1) { s[0] = 1.0; return; }
  double scale = 0.0;
  for (int i = 0; i < k; ++i) scale = std::max(scale, std::fabs(a[i]) + (i < k - 1 ? std::fabs(b[i]) : 0.0));
  const double sigma = th - 1e-13 * (scale + 1e-300);
  // factor (T - sigma I) = P L U with U upper triangular (bandwidth 2)
  std::vector<double> d(k), du(k), du2(k), l(k), dl(k);
  std::vector<char> piv(k, 0);
  for (int i = 0; i < k; ++i) { d[i] = a[i] - sigma; du[i] = i < k - 1 ? b[i] : 0.0; du2[i] = 0.0; }
  for (int i = 0; i < k - 1; ++i) dl[i] = b[i];
  for (int i = 0; i < k - 1; ++i) {
    if (std::fabs(d[i]) >= std::fabs(dl[i])) {
      const double f = d[i] != 0.0 ? dl[i] / d[i] : 0.0;
      l[i] = f;
      d[i + 1] -= f * du[i];
    } else {
      const double f = d[i] / dl[i];
      l[i] = f;
      piv[i] = 1;
      const double t = du[i];
      d[i] = dl[i];
      du[i] = d[i + 1];
      d[i + 1] = t - f * d[i + 1];
      if (i < k - 2) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du[i + 1];
      }
    }
  }
  for (int i = 0; i < k; ++i) if (d[i] == 0.0) d[i] = 1e-300;
  for (int i = 0; i < k; ++i) s[i] = 1.0 / std::sqrt((double)k) * ((i % 3) ? 1.0 : -0.7);
  for (int it = 0; it < 4; ++it) {
    for (int i = 0; i < k - 1; ++i) {
      if (piv[i]) { const double t = s[i]; s[i] = s[i + 1]; s[i + 1] = t - l[i] * s[i + 1]; }
      else s[i + 1] -= l[i] * s[i];
    }
    s[k - 1] /= d[k - 1];
    if (k > 1) s[k - 2] = (s[k - 2] - du[k - 2] * s[k - 1]) / d[k - 2];
    for (int i = k - 3; i >= 0; --i) s[i] = (s[i] - du[i] * s[i + 1] - du2[i] * s[i + 2]) / d[i];
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += s[i] * s[i];
    nrm = std::sqrt(nrm);
    for (int i = 0; i < k; ++i) s[i] /= nrm;
  }
}

// ------------------------------------------------------------------ the solver
// Block-Jacobi preconditioner of the tCG, per camera: B_i = 2 Q_ii and Minv_i = B_i^-1 with the
// eigenvalues of Q_ii (positive semidefinite) clamped below at 1e-6 of the largest; N x 9 each.
template <typename TQ>
__global__ void k_tcg_precond_blocks(int N, const TQ* __restrict__ q64, int nt, double* __restrict__ Minv,
                                     double* __restrict__ B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double A[3][3], V[3][3], d[3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) A[a][b] = q_entry(q64, nt, 3 * i + a, 3 * i + b);
  jacobi3<double>(A, V, d);
  const double dmax = fmax(d[0], fmax(d[1], d[2]));
  double e[3];
  for (int k = 0; k < 3; ++k) e[k] = dmax > 0.0 ? fmax(d[k], 1e-6 * dmax) : 1.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double mi = 0.0, bb = 0.0;
      for (int k = 0; k < 3; ++k) {
        mi += V[a][k] * V[b][k] / (2.0 * e[k]);
        bb += V[a][k] * V[b][k] * (2.0 * e[k]);
      }
      Minv[(size_t)9 * i + 3 * a + b] = mi;
      B[(size_t)9 * i + 3 * a + b] = bb;
    }
}

// sc->dot = sum_i <Y_i, B_i Y_i> (the preconditioner's norm of the iterate, the trust region's scale)
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_bnorm(int N, const T* __restrict__ Y, const double* __restrict__ B, Scal* sc, double* partials,
        unsigned* counter) {
  double v[1] = {0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double y[3][R];
    load_block<T, double, R>(Y, i, y);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double m = B[(size_t)9 * i + 3 * a + b];
        for (int j = 0; j < R; ++j) v[0] += y[a][j] * m * y[b][j];
      }
  }
  grid_reduce<1>(v, partials, counter, [&](double* t) { sc->dot = t[0]; });
}

// Gradient epilogue of the RTR iterates: grad_block, plus the raw Q Y of the point saved to QY and,
// for a candidate Yc with reference Y (Yref, its Q Y in QYref), the change of the objective in
// difference form, sc->df = <Yc - Y, Q Yc + Q Y> + mu sum_{i>=1} (xc_i - x_i)(xc_i + x_i - 2)
// (Q symmetric; x_i = ||row 2 of Y_i||^2 as in the App. D term).  Its rounding error scales with
// |Yc - Y| instead of |Y|: near convergence f is a sum of terms many orders of magnitude above f
// itself, and the difference of two such sums is rounding noise once the predicted decrease is
// small (in FP64 too), which turns the trust-region ratio into noise.
template <typename T, int R>
__global__ void __launch_bounds__(CAM_THREADS)
k_grad_epi_rtr(int N, const T* __restrict__ Y, T* __restrict__ W, T* __restrict__ G,
               double* __restrict__ Lam, Scal* sc, int cand, const T* __restrict__ Yref,
               const T* __restrict__ QYref, T* __restrict__ QY, double* partials, unsigned* counter,
               int* err) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double y[3][R], w[3][R];
    load_block<T, double, R>(Y, i, y);
    load_block<T, double, R>(W, i, w);
    store_block<T, double, R>(QY, i, w);
    if (cand && Yref) {
      double yr[3][R], wr[3][R];
      load_block<T, double, R>(Yref, i, yr);
      load_block<T, double, R>(QYref, i, wr);
      double d = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int j = 0; j < R; ++j) d += (y[a][j] - yr[a][j]) * (w[a][j] + wr[a][j]);
      if (sc->mu != 0.0 && i > 0) {
        double xc = 0.0, xr = 0.0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
          xc += y[2][j] * y[2][j];
          xr += yr[2][j] * yr[2][j];
        }
        d += sc->mu * (xc - xr) * (xc + xr - 2.0);
      }
      v[3] = d;
    }
    double vg[3] = {0.0, 0.0, 0.0};
    grad_block<T, R>(i, N, Y, W, G, Lam, sc->mu, vg);
    v[0] = vg[0]; v[1] = vg[1]; v[2] = vg[2];
  }
  grid_reduce<4>(v, partials, counter, [&](double* t) {
    if (!isfinite(t[0]) || !isfinite(t[1])) atomicOr(err, DEV_NUMERIC);
    if (cand) { sc->fc = t[0]; sc->gc2 = t[1]; sc->yc2 = t[2]; sc->df = t[3]; }
    else { sc->f = t[0]; sc->g2 = t[1]; sc->y2 = t[2]; }
  });
}

// ------------------------------------------------------------------ LOBPCG certificate kernels
// Blocks of 4 vectors are n_pad x 4 row-major FP32 arrays (the sweep's layout for R = 4).

// Minv_i = inverse of the 3 x 3 diagonal block Z_ii = Q_ii - Lambda_i + dreg_i e3 e3^T of the
// certificate matrix, eigenvalues clamped at 1e-6 of the largest (block-Jacobi preconditioner).
template <typename TQ>
__global__ void k_zblock_precond(int N, const TQ* __restrict__ q64, int nt,
                                 const double* __restrict__ Lam, double* __restrict__ Minv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double A[3][3], V[3][3], d[3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      A[a][b] = q_entry(q64, nt, 3 * i + a, 3 * i + b) - 0.5 * (Lam[9 * i + 3 * a + b] + Lam[9 * i + 3 * b + a]);
  A[2][2] += Lam[(size_t)9 * N + i];
  jacobi3<double>(A, V, d);
  const double dmax = fmax(fabs(d[0]), fmax(fabs(d[1]), fabs(d[2])));
  double e[3];
  for (int k = 0; k < 3; ++k) e[k] = dmax > 0.0 ? fmax(d[k], 1e-6 * dmax) : 1.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double m = 0.0;
      for (int k = 0; k < 3; ++k) m += V[a][k] * V[b][k] / e[k];
      Minv[(size_t)9 * i + 3 * a + b] = m;
    }
}

// ZV_i = Wz_i - Lambda_i V_i + dreg_i e3 e3^T V_i for a 4-column block (Z V after the sweep
// Wz = Q V); Wz is reset to zero for the next accumulating sweep.
__global__ void k_zv4(int N, float* __restrict__ Wz, const float* __restrict__ V,
                      const double* __restrict__ Lam, float* __restrict__ ZV) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double x[3][4];
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 4; ++j) x[a][j] = V[(size_t)(3 * i + a) * 4 + j];
  const double dreg = Lam[(size_t)9 * N + i];
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < 4; ++j) {
      const double lx = Lam[9 * i + 3 * a] * x[0][j] + Lam[9 * i + 3 * a + 1] * x[1][j] +
                        Lam[9 * i + 3 * a + 2] * x[2][j];
      const size_t e = (size_t)(3 * i + a) * 4 + j;
      ZV[e] = float(double(Wz[e]) - lx + (a == 2 ? dreg * x[2][j] : 0.0));
      Wz[e] = 0.f;
    }
}

// R = ZX - X diag(theta); W = Minv R (per camera); out[j] = ||R_j||^2 (j = 0..3)
__global__ void __launch_bounds__(CAM_THREADS)
k_lob_resid(int N, const float* __restrict__ X, const float* __restrict__ ZX,
            const double* __restrict__ theta, const double* __restrict__ Minv, float* __restrict__ W,
            double* partials, unsigned* counter, double* out) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    double r[3][4];
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j < 4; ++j) {
        const size_t e = (size_t)(3 * i + a) * 4 + j;
        r[a][j] = double(ZX[e]) - theta[j] * double(X[e]);
        v[j] += r[a][j] * r[a][j];
      }
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j < 4; ++j) {
        double w = 0.0;
        for (int b = 0; b < 3; ++b) w += Minv[(size_t)9 * i + 3 * a + b] * r[b][j];
        W[(size_t)(3 * i + a) * 4 + j] = float(w);
      }
  }
  grid_reduce<4>(v, partials, counter, [&](double* t) {
    for (int j = 0; j < 4; ++j) out[j] = t[j];
  });
}

// c[d][j] = <Vd_d, B_j> for the nd deflation columns (column-major, stride ld) and the 4 columns
// of block B (c: nd x 4 row-major, nd <= 8)
template <typename VT>
__global__ void __launch_bounds__(CAM_THREADS)
k_lob_defl_coef(int nn, int nd, const VT* __restrict__ Vd, size_t ld, const float* __restrict__ B,
                double* partials, unsigned* counter, double* c) {
  double v[32];
  for (int k = 0; k < 32; ++k) v[k] = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gridDim.x * blockDim.x) {
    double b[4];
    for (int j = 0; j < 4; ++j) b[j] = B[(size_t)e * 4 + j];
    for (int d = 0; d < nd; ++d) {
      const double x = double(Vd[(size_t)d * ld + e]);
      for (int j = 0; j < 4; ++j) v[d * 4 + j] += x * b[j];
    }
  }
  grid_reduce<32>(v, partials, counter, [&](double* t) {
    for (int k = 0; k < 32; ++k) c[k] = t[k];
  });
}
// B -= Vd c (projection onto range(Y)^perp)
template <typename VT>
__global__ void k_lob_defl_apply(int nn, int nd, const VT* __restrict__ Vd, size_t ld,
                                 const double* __restrict__ c, float* __restrict__ B) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gridDim.x * blockDim.x)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int d = 0; d < nd; ++d) s += double(Vd[(size_t)d * ld + e]) * c[d * 4 + j];
      B[(size_t)e * 4 + j] -= float(s);
    }
}

// Gram blocks of S = [S0 S1 S2] (n x 12) and ZS: pair p < 6 is S_a^T S_b (a <= b), pair p >= 6
// is S_a^T ZS_b; blockIdx.y = p, partial sums per x-block (16 values), FP64 accumulation.
__device__ __constant__ int c_lob_pa[15] = {0, 0, 0, 1, 1, 2, 0, 0, 0, 1, 1, 1, 2, 2, 2};
__device__ __constant__ int c_lob_pb[15] = {0, 1, 2, 1, 2, 2, 0, 1, 2, 0, 1, 2, 0, 1, 2};
struct LobBlocks { const float* s[3]; const float* zs[3]; };
__global__ void __launch_bounds__(256)
k_lob_gram(int nn, LobBlocks B, double* __restrict__ part) {
  const int p = blockIdx.y;
  const float* A = B.s[c_lob_pa[p]];
  const float* C = p < 6 ? B.s[c_lob_pb[p]] : B.zs[c_lob_pb[p]];
  double acc[16];
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gridDim.x * blockDim.x) {
    const float4 a = *reinterpret_cast<const float4*>(A + (size_t)e * 4);
    const float4 c = *reinterpret_cast<const float4*>(C + (size_t)e * 4);
    const double av[4] = {a.x, a.y, a.z, a.w}, cv[4] = {c.x, c.y, c.z, c.w};
    for (int x = 0; x < 4; ++x)
      for (int y = 0; y < 4; ++y) acc[x * 4 + y] += av[x] * cv[y];
  }
  __shared__ double sh[16][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 16; ++k) {
    const double t = warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[threadIdx.x][w];
    part[((size_t)p * gridDim.x + blockIdx.x) * 16 + threadIdx.x] = t;
  }
}
// out[p][16] = sum over x-blocks of part (fixed order)
__global__ void k_lob_gram_finish(int nxb, const double* __restrict__ part, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 15 * 16) return;
  const int p = t / 16, k = t % 16;
  double s = 0.0;
  for (int x = 0; x < nxb; ++x) s += part[((size_t)p * nxb + x) * 16 + k];
  out[t] = s;
}

// Xo = S C, ZXo = ZS C, Po = S CP, ZPo = ZS CP (C, CP: 12 x 4 row-major, FP64)
__global__ void k_lob_update(int nn, LobBlocks B, const double* __restrict__ C,
                             const double* __restrict__ CP, float* __restrict__ Xo,
                             float* __restrict__ ZXo, float* __restrict__ Po, float* __restrict__ ZPo) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gridDim.x * blockDim.x) {
    double s[12], z[12];
    for (int b = 0; b < 3; ++b)
      for (int j = 0; j < 4; ++j) {
        s[b * 4 + j] = B.s[b][(size_t)e * 4 + j];
        z[b * 4 + j] = B.zs[b][(size_t)e * 4 + j];
      }
    for (int j = 0; j < 4; ++j) {
      double x = 0, zx = 0, pp = 0, zp = 0;
      for (int k = 0; k < 12; ++k) {
        x += s[k] * C[k * 4 + j];
        zx += z[k] * C[k * 4 + j];
        pp += s[k] * CP[k * 4 + j];
        zp += z[k] * CP[k * 4 + j];
      }
      Xo[(size_t)e * 4 + j] = float(x);
      ZXo[(size_t)e * 4 + j] = float(zx);
      Po[(size_t)e * 4 + j] = float(pp);
      ZPo[(size_t)e * 4 + j] = float(zp);
    }
  }
}

// 4-column block filled with the seeded uniform(-1, 1) sequence (rows >= n zero)
__global__ void k_lob_random(int nn, int n, uint64_t seed, float* __restrict__ X) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn * 4; e += gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(e + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    X[e] = (e / 4 < n) ? float((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0) : 0.f;
  }
}
// dst (n_pad FP64) = column j of the block
__global__ void k_lob_col(int nn, int j, const float* __restrict__ X, double* __restrict__ dst) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gridDim.x * blockDim.x)
    dst[e] = double(X[(size_t)e * 4 + j]);
}

struct Solver {
  xm_ctx* ctx;
  const DeviceQ& q;
  xm_opts o;
  cudaStream_t st;
  int N, n, n_pad, nb_cam;
  size_t vec_bytes;
  // vectors (n_pad x 8 elements of up to 8 bytes each)
  void *bY = nullptr, *bYc = nullptr, *bW = nullptr, *bWc = nullptr, *bG = nullptr,
       *bGc = nullptr, *bYin = nullptr, *bEta = nullptr, *bHeta = nullptr, *bR = nullptr,
       *bD = nullptr, *bHd = nullptr, *bWd = nullptr, *bY64 = nullptr, *bXi = nullptr,
       *bYh = nullptr, *bQY = nullptr, *bQYc = nullptr;   // Q Y of the RTR iterate / candidate
  double *Lam = nullptr, *Lamc = nullptr;
  double *pcMinv = nullptr, *pcB = nullptr;   // tCG preconditioner blocks (N x 9), or null
  void* bZ = nullptr;                         // tCG preconditioned residual
  Scal* d_sc = nullptr;
  Scal* h_sc = nullptr;
  double* d_small = nullptr;   // gram / rotation / O0 / scalar scratch (256 doubles)
  // Lanczos
  int kmax = 0;
  void* V = nullptr;   // Lanczos basis: FP32 or FP64 columns of n_pad (room for FP64)
  double *lw = nullptr, *lz = nullptr, *lalpha = nullptr, *lbeta = nullptr, *lc = nullptr,
         *lnrm = nullptr, *lritz = nullptr;
  float *lv32 = nullptr, *lW32 = nullptr, *lwf = nullptr, *lcf = nullptr;
  static constexpr int LPART_MAX = 64;   // column chunks of the reorthogonalisation product
  static constexpr int BULK_PLATEAU = 15; // outer steps without a halving of min ||rgrad||
  static constexpr int PRECOND_CAP_RUN = 3; // capped tCG solves in a row that switch on precond = 2
  // tCG iterations per step of the FP32 bulk phase (at most max_tcg): far from the optimum a
  // truncated inner solve is still a descent step and the trust region absorbs it; the long
  // inner solves of the late bulk (100-200 iterations) bought little.  A solve stopped here
  // counts as capped (cap_run) like one stopped at max_tcg.  The polish keeps max_tcg.
  static constexpr int BULK_TCG_CAP = 60;
  double* lpart = nullptr;               // LPART_MAX x n_pad partial sums
  int last_nd = 0;                       // deflation columns of the last certificate's basis
  // LOBPCG certificate: 12 blocks of n_pad x 4 floats, preconditioner, Gram partials, scalars
  float* lob = nullptr;
  double *lob_minv = nullptr, *lob_part = nullptr, *lob_small = nullptr;
  int lob_nxb = 0;
  // stats
  xm_info info{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t fev[2] = {nullptr, nullptr};   // tCG chunk flags: one chunk in flight ahead
  int* h_flags = nullptr;                     // pinned, 2 slots
  cudaStream_t cap_st = nullptr;              // side stream on which tCG chunks are captured
  bool use_graphs = true;                     // cleared if a capture ever fails
  double ms32 = 0, ms64 = 0;
  int n32 = 0, n64 = 0;
  long launches = 0;
  std::chrono::steady_clock::time_point t_start;
  bool timed_out = false;
  double ref_g = -1.0;   // ||rgrad|| at the start point of the solve (tolerance reference)
  double cur_g2 = 0.0;
  double carry_delta = 0.0;   // trust radius handed from a stalled bulk phase to the polish
  bool bulk_stalled = false;  // the last bulk phase stopped on stagnation (opts.bulk_stall)
  // bG holds the FP64 Riemannian gradient 2 Z Y at bY64 (set for the final certificate after an
  // FP64 gradient): Z's block on range(Y) then follows from Y^T G without a Z product
  bool g64_valid = false;

  Solver(xm_ctx* c, const DeviceQ& qq, const xm_opts& oo) : ctx(c), q(qq), o(oo), st(c->stream) {
    N = q.N; n = q.n; n_pad = q.n_pad;
    nb_cam = (N + CAM_THREADS - 1) / CAM_THREADS;
    vec_bytes = (size_t)n_pad * XM_MAX_RANK * sizeof(double);
  }
  ~Solver() {
    void* bufs[] = {bY, bYc, bW, bWc, bG, bGc, bYin, bEta, bHeta, bR, bD, bHd, bWd, bY64, bXi, bYh,
                    bQY, bQYc, bZ, Lam, Lamc, pcMinv, pcB, d_sc, d_small, V, lw, lz, lalpha, lbeta, lc, lnrm,
                    lritz, lv32, lW32, lwf, lcf, lpart, lob, lob_minv, lob_part, lob_small};
    for (void* p : bufs) if (p) cudaFree(p);
    if (h_sc) cudaFreeHost(h_sc);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (cudaEvent_t e : fev) if (e) cudaEventDestroy(e);
    if (h_flags) cudaFreeHost(h_flags);
    if (cap_st) cudaStreamDestroy(cap_st);
  }

  xm_status alloc() {
    void** vecs[] = {&bY, &bYc, &bW, &bWc, &bG, &bGc, &bYin, &bEta, &bHeta, &bR, &bD, &bHd, &bWd,
                     &bY64, &bXi, &bYh, &bQY, &bQYc, &bZ};
    for (void** p : vecs) {
      XM_CUDA_TRY(cudaMalloc(p, vec_bytes));
      XM_CUDA_TRY(cudaMemsetAsync(*p, 0, vec_bytes, st));
    }
    XM_CUDA_TRY(cudaMalloc(&Lam, sizeof(double) * lam_doubles(N)));
    XM_CUDA_TRY(cudaMalloc(&Lamc, sizeof(double) * lam_doubles(N)));
    XM_CUDA_TRY(cudaMemsetAsync(Lam, 0, sizeof(double) * lam_doubles(N), st));
    XM_CUDA_TRY(cudaMemsetAsync(Lamc, 0, sizeof(double) * lam_doubles(N), st));
    XM_CUDA_TRY(cudaMalloc(&d_sc, sizeof(Scal)));
    XM_CUDA_TRY(cudaMemsetAsync(d_sc, 0, sizeof(Scal), st));
    XM_CUDA_TRY(cudaMemcpyAsync(&d_sc->mu, &o.scale_reg, sizeof(double), cudaMemcpyHostToDevice, st));
    XM_CUDA_TRY(cudaMallocHost(&h_sc, sizeof(Scal)));
    XM_CUDA_TRY(cudaMalloc(&d_small, 256 * sizeof(double)));
    XM_CUDA_TRY(cudaMemsetAsync(d_small, 0, 256 * sizeof(double), st));
    XM_CUDA_TRY(cudaEventCreate(&ev0));
    XM_CUDA_TRY(cudaEventCreate(&ev1));
    for (cudaEvent_t& e : fev) XM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    XM_CUDA_TRY(cudaMallocHost(&h_flags, 2 * sizeof(int)));
    XM_CUDA_TRY(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
    XM_TRY(ensure_partials(ctx, (size_t)std::max(nb_cam, 1024) * 64));
    if (o.precond == 1) XM_TRY(enable_precond());
    return XM_OK;
  }

  // the tCG's block-Jacobi preconditioner: Q's 3 x 3 diagonal blocks from the FP64 tiles, else
  // the FP32 ones (a preconditioner)
  xm_status enable_precond() {
    if (pcMinv) return XM_OK;
    XM_CUDA_TRY(cudaMalloc(&pcMinv, sizeof(double) * 9 * (size_t)N));
    XM_CUDA_TRY(cudaMalloc(&pcB, sizeof(double) * 9 * (size_t)N));
    if (q.q64) k_tcg_precond_blocks<double><<<nb_cam, CAM_THREADS, 0, st>>>(N, q.q64, q.nt, pcMinv, pcB);
    else k_tcg_precond_blocks<float><<<nb_cam, CAM_THREADS, 0, st>>>(N, q.q32, q.nt, pcMinv, pcB);
    ++launches;
    XM_CUDA_TRY(cudaGetLastError());
    return XM_OK;
  }

  // Zero every work vector except the FP64 master iterate.  Called whenever the precision or
  // the padded width changes, so that no buffer is ever read through a stale reinterpretation.
  xm_status clear_vecs() {
    void* vecs[] = {bY, bYc, bW, bWc, bG, bGc, bYin, bEta, bHeta, bR, bD, bHd, bWd, bXi, bYh, bZ};
    for (void* p : vecs) XM_CUDA_TRY(cudaMemsetAsync(p, 0, vec_bytes, st));
    return XM_OK;
  }

  int grid_elems(size_t total) const {
    size_t g = (total + CAM_THREADS - 1) / CAM_THREADS;
    const size_t cap = (size_t)ctx->num_sms * 8;
    if (g > cap) g = cap;
    return (int)std::max<size_t>(g, 1);
  }
  int grid_gram() const { return std::max(1, std::min(nb_cam * 3, ctx->num_sms * 4)); }
  double* d_slot() { return d_small + 200; }

  bool over_time() {
    if (o.time_limit_s <= 0) return false;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (el > o.time_limit_s) timed_out = true;
    return timed_out;
  }

  xm_status pull_scalars() {
    XM_CUDA_TRY(cudaMemcpyAsync(h_sc, d_sc, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    return check_device_error(ctx, "solver");
  }

  // F(X) - <grad F(X), X> at the FP64 point Y64 (App. E dual value; 0 without regulariser)
  template <int R>
  xm_status reg_dual_terms(const double* Y64, double* out) {
    *out = 0.0;
    if (o.scale_reg == 0.0) return XM_OK;
    k_reg_terms<R><<<nb_cam, CAM_THREADS, 0, st>>>(N, Y64, d_sc, ctx->d_partials, ctx->d_counter);
    ++launches;
    XM_CUDA_TRY(cudaGetLastError());
    XM_TRY(pull_scalars());
    *out = h_sc->dot - h_sc->kappa;
    return XM_OK;
  }

  // one sweep; timed = bracket it with events (only for sweeps that always run)
  xm_status sweep(int prec, int R, const void* Yp, void* Wp, const int* skip, bool timed) {
    if (timed) XM_CUDA_TRY(cudaEventRecord(ev0, st));
    XM_TRY(qy_launch(ctx, q, prec, R, Yp, Wp, skip, st));
    ++launches;
    ++info.n_sweeps;
    if (prec == XM_FP64) ++info.n_sweeps_fp64;
    if (timed) {
      XM_CUDA_TRY(cudaEventRecord(ev1, st));
      XM_CUDA_TRY(cudaEventSynchronize(ev1));
      float ms = 0.f;
      XM_CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
      if (prec == XM_FP64) { ms64 += ms; ++n64; }
      else if (prec == XM_FP32_BULK && R == 4) { ms32 += ms; ++n32; }
    }
    return XM_OK;
  }

  // ---------------- gradient / objective at a point (W zero on entry, zero on exit)
  template <typename To, int R>
  // QYp: also save Q Y of this point (RTR iterates); Yref, QYref: a candidate's reference point
  // and its saved Q Y, for the objective change in difference form (sc->df)
  xm_status grad_at(int prec, void* Yp, void* Wp, void* Gp, double* L, int cand, bool timed,
                    void* QYp = nullptr, const void* Yref = nullptr, const void* QYref = nullptr) {
    XM_TRY(sweep(prec, R, Yp, Wp, nullptr, timed));
    if (QYp)
      k_grad_epi_rtr<To, R><<<nb_cam, CAM_THREADS, 0, st>>>(
          N, (const To*)Yp, (To*)Wp, (To*)Gp, L, d_sc, cand, (const To*)Yref, (const To*)QYref,
          (To*)QYp, ctx->d_partials, ctx->d_counter, ctx->d_err);
    else
      k_grad_epi<To, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, (const To*)Yp, (To*)Wp, (To*)Gp, L, d_sc,
                                                        cand, ctx->d_partials, ctx->d_counter,
                                                        ctx->d_err);
    ++launches;
    XM_CUDA_TRY(cudaGetLastError());
    return XM_OK;
  }

  // ---------------- RTR (Absil et al. 2008, Alg. 10) at fixed rank
  template <typename To, typename Ti, int R>
  xm_status rtr(int prec_grad, int prec_hvp, double tol_rel, int max_outer, bool bulk) {
    const size_t rows = (size_t)n_pad;
    XM_TRY(grad_at<To, R>(prec_grad, bY, bW, bG, Lam, 0, true, bQY));
    XM_TRY(pull_scalars());
    double f = h_sc->f, g2 = h_sc->g2;
    if (!std::isfinite(f) || !std::isfinite(g2)) return set_error(XM_ENUMERIC, "rtr: non-finite f");
    if (ref_g <= 0) ref_g = std::sqrt(g2);
    const double tol_abs = tol_rel * ref_g;
    // trust-region scale: ||Y|| in the tCG's norm (the preconditioner's B-norm when it is on)
    double ynorm2 = h_sc->y2;
    if (pcB) {
      k_bnorm<To, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, (const To*)bY, pcB, d_sc, ctx->d_partials,
                                                      ctx->d_counter);
      ++launches;
      XM_TRY(pull_scalars());
      ynorm2 = h_sc->dot;
    }
    double Delta_bar = std::sqrt(std::max(ynorm2, 1e-300));
    double Delta = Delta_bar / 8.0;
    if (!bulk && carry_delta > 0.0) Delta = std::min(carry_delta, Delta_bar);   // polish after a stall
    carry_delta = 0.0;
    if (bulk) bulk_stalled = false;
    const double eps_reg = std::is_same<To, float>::value ? 1e2 * 1.1920929e-07
                                                          : 1e3 * 2.220446049250313e-16;
    int rejects = 0;
    // BF16-tile Hessian products early in the FP32 bulk phase (opts.bf16_hvp_until)
    const bool bf16_early = bulk && prec_hvp == XM_FP32_BULK && o.bf16_hvp_until > 0.0 && q.q16;
    double best_f = f;   // bulk stagnation test (opts.bulk_stall > 0)
    int stall = 0;
    double g_halved = std::sqrt(g2);   // automatic hand-over (opts.bulk_stall < 0): the gradient
    int since_halved = 0;              // norm at its last halving, outer steps since then
    int cap_run = 0;                   // consecutive tCG solves stopped by the iteration cap
    // captured tCG chunks of this call, keyed by the (iterate, Lambda) buffers they read
    struct ChunkGraph { const void* yin; const double* lam; int prec; cudaGraphExec_t exec; };
    struct GraphCache {
      ChunkGraph e[2] = {{nullptr, nullptr, 0, nullptr}, {nullptr, nullptr, 0, nullptr}};
      int n = 0;
      cudaStream_t s = nullptr;
      void clear() {
        if (n > 0) cudaStreamSynchronize(s);   // no launch of these graphs still in flight
        for (int i = 0; i < n; ++i) cudaGraphExecDestroy(e[i].exec);
        n = 0;
      }
      ~GraphCache() { clear(); }
    } gcache;
    gcache.s = st;
    ChunkGraph* cg = gcache.e;
    int& ncg = gcache.n;
    for (int k = 0; k < max_outer; ++k) {
      if (std::sqrt(g2) <= tol_abs) break;
      if (over_time()) break;
      const int hvp = (bf16_early && std::sqrt(g2) > o.bf16_hvp_until * ref_g) ? XM_BF16Q_BULK : prec_hvp;
      const Ti* Yin;
      if (!std::is_same<To, Ti>::value) {
        k_cast<To, Ti><<<grid_elems(rows * R), CAM_THREADS, 0, st>>>(rows * R, (const To*)bY, (Ti*)bYin);
        ++launches;
        Yin = (const Ti*)bYin;
      } else {
        Yin = (const Ti*)bY;
      }
      const int tcg_cap = bulk ? std::min(o.max_tcg, BULK_TCG_CAP) : o.max_tcg;
      k_tcg_init<To, Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(
          N, Yin, (const To*)bG, (Ti*)bEta, (Ti*)bHeta, (Ti*)bR, (Ti*)bZ, (Ti*)bD, pcMinv, d_sc, Delta,
          tcg_cap, 1.0, 0.1, bulk ? 0.5 * tol_abs : 0.0, ctx->d_partials, ctx->d_counter);
      ++launches;
      XM_CUDA_TRY(cudaGetLastError());
      // Chunks of CH iterations; the host reads the done flag of chunk k-1 while chunk k is
      // already queued, so the device never waits for the host.  A chunk queued after the
      // device set done is a no-op (every kernel of the loop returns on done).  From the second
      // chunk on, a chunk is one CUDA graph (captured on a side stream, replayed on st): its
      // 4 CH kernels then start back to back without a host launch each.  The iterate and Lam
      // alternate between two buffers as steps are accepted, so at most two graphs per call.
      const int CH = 4;
      int done = 0, slot = 0;
      bool pending = false;
      auto launch_chunk = [&](cudaStream_t cst) -> xm_status {
        for (int c = 0; c < CH; ++c) {
          XM_TRY(qy_launch(ctx, q, hvp, R, bD, bWd, &d_sc->done, cst));
          k_hvp_epi<Ti, R><<<nb_cam, CAM_THREADS, 0, cst>>>(N, Yin, (Ti*)bWd, (const Ti*)bD, (Ti*)bHd,
                                                           Lam, d_sc, ctx->d_partials, ctx->d_counter);
          k_tcg_update<Ti, R><<<nb_cam, CAM_THREADS, 0, cst>>>(N, Yin, (Ti*)bEta, (Ti*)bHeta, (Ti*)bR,
                                                              (Ti*)bZ, (const Ti*)bD, (const Ti*)bHd,
                                                              pcMinv, d_sc, ctx->d_partials,
                                                              ctx->d_counter);
          k_tcg_dir<Ti, R><<<nb_cam, CAM_THREADS, 0, cst>>>(N, (const Ti*)bZ, (Ti*)bD, d_sc);
        }
        XM_CUDA_TRY(cudaGetLastError());
        return XM_OK;
      };
      auto chunk_exec = [&]() -> cudaGraphExec_t {
        for (int i = 0; i < ncg; ++i)
          if (cg[i].yin == Yin && cg[i].lam == Lam && cg[i].prec == hvp) return cg[i].exec;
        if (cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
          (void)cudaGetLastError();
          return nullptr;
        }
        const xm_status sc_ = launch_chunk(cap_st);
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cap_st, &g);
        cudaGraphExec_t ex = nullptr;
        if (sc_ != XM_OK || ee != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess)
          ex = nullptr;
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        if (!ex) return nullptr;
        if (ncg == 2) { cudaGraphExecDestroy(cg[0].exec); cg[0] = cg[1]; ncg = 1; }
        cg[ncg++] = ChunkGraph{Yin, Lam, hvp, ex};
        return ex;
      };
      xm_status chunk_status = XM_OK;
      for (int j = 0; j < tcg_cap && !done; j += CH) {
        cudaGraphExec_t ex = (j > 0 && use_graphs) ? chunk_exec() : nullptr;
        if (j > 0 && use_graphs && !ex) use_graphs = false;
        if (ex) {
          if (cudaGraphLaunch(ex, st) != cudaSuccess) {
            chunk_status = set_error(XM_ECUDA, "tCG chunk graph launch failed");
            break;
          }
        } else {
          chunk_status = launch_chunk(st);
          if (chunk_status != XM_OK) break;
        }
        launches += 4 * CH;
        XM_CUDA_TRY(cudaMemcpyAsync(&h_flags[slot], &d_sc->done, sizeof(int), cudaMemcpyDeviceToHost, st));
        XM_CUDA_TRY(cudaEventRecord(fev[slot], st));
        if (pending) {
          XM_CUDA_TRY(cudaEventSynchronize(fev[slot ^ 1]));
          done = h_flags[slot ^ 1];
        }
        pending = true;
        slot ^= 1;
      }
      XM_TRY(chunk_status);
      k_model_terms<To, Ti, R><<<grid_elems(rows * R), CAM_THREADS, 0, st>>>(
          (int)rows, (const To*)bG, (const Ti*)bEta, (const Ti*)bHeta, d_sc, ctx->d_partials,
          ctx->d_counter);
      k_retract<To, Ti, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, (const To*)bY, (const Ti*)bEta, 1.0,
                                                           (To*)bYc);
      launches += 2;
      XM_CUDA_TRY(cudaGetLastError());
      XM_TRY(grad_at<To, R>(prec_grad, bYc, bWc, bGc, Lamc, 1, true, bQYc, bY, bQY));
      XM_TRY(pull_scalars());
      ++info.n_outer;
      info.n_tcg += h_sc->iters;
      cap_run = h_sc->reason == 4 ? cap_run + 1 : 0;
      // one Hessian-vector sweep per tCG iteration (the sweeps of chunks queued after the
      // device stopped returned at once and are not counted)
      info.n_sweeps += h_sc->iters;
      if (prec_hvp == XM_FP64) info.n_sweeps_fp64 += h_sc->iters;
      const double fc = h_sc->fc;
      const double dfc = h_sc->df;   // f(Yc) - f(Y) in difference form
      const double model_dec = -(h_sc->g_eta + 0.5 * h_sc->eta_Heta);
      const double reg = std::max(1.0, std::fabs(f)) * eps_reg;
      const double rho = (-dfc + reg) / (model_dec + reg);
      const double en = std::sqrt(pcMinv ? h_sc->ee : h_sc->eta2);   // ||eta|| in the tCG's norm
      const bool finite = std::isfinite(fc) && std::isfinite(dfc);
      if (!finite || rho < 0.25) {
        // a quarter of the step actually taken when it stayed inside the region: the tCG's
        // interior solution is what failed, and shrinking from a radius it never reached only
        // repeats it (the FP32-HVP polish ran 200 iterations to the same rejected interior step
        // at every radius from 5e-2 down to 3e-6); for a boundary step en = Delta
        Delta = 0.25 * ((finite && en > 0.0) ? std::min(Delta, en) : Delta);
      } else if (rho > 0.75 && en >= Delta * (1.0 - 1e-6)) {
        Delta = std::min(2.0 * Delta, Delta_bar);
      }
      const bool accept = finite && rho > 0.1 && dfc <= reg;
      if (o.verbose >= 2)
        fprintf(stderr, "[xm] %s k=%d f=%.12e |g|=%.3e rho=%.3f Delta=%.3e tcg=%d(%d) %s\n",
                bulk ? "bulk" : "fp64", k, f, std::sqrt(g2), rho, Delta, h_sc->iters, h_sc->reason,
                accept ? "acc" : "rej");
      if (accept) {
        std::swap(bY, bYc); std::swap(bW, bWc); std::swap(bG, bGc); std::swap(Lam, Lamc);
        std::swap(bQY, bQYc);
        f = fc;
        g2 = h_sc->gc2;
        rejects = 0;
      } else {
        ++rejects;
      }
      if (Delta < 1e-12 * Delta_bar) break;
      if (bulk && (rejects >= 6 || Delta < 1e-7 * Delta_bar)) break;
      if (bulk && o.bulk_stall < 0) {
        // automatic: FP32 has reached its noise floor when the running minimum of the
        // gradient norm has not halved over BULK_PLATEAU outer steps (below 1e-6 of its start)
        // while the inner solves no longer reach their tolerance (the last PRECOND_CAP_RUN tCG
        // solves stopped at max_tcg); the FP64 polish takes over from there.  Where FP32 keeps
        // converging the minimum halves every few steps down to bulk_tol_rel
        const double gn = std::sqrt(g2);
        if (gn <= 0.5 * g_halved) { g_halved = gn; since_halved = 0; } else { ++since_halved; }
        if (since_halved >= BULK_PLATEAU && cap_run >= PRECOND_CAP_RUN && gn <= 1e-6 * ref_g) {
          carry_delta = Delta;
          bulk_stalled = true;
          break;
        }
      } else if (bulk && o.bulk_stall > 0) {
        // the FP32 objective has stopped improving beyond its own noise (the ratio test's
        // allowance reg): further FP32 steps only chase rounding, the FP64 polish takes over
        if (f < best_f - reg) { best_f = f; stall = 0; } else { ++stall; }
        if (stall >= o.bulk_stall && std::sqrt(g2) <= 1e-6 * ref_g) {
          // the polish continues from here: keep the trust radius the bulk phase found
          carry_delta = Delta;
          bulk_stalled = true;
          break;
        }
      }
      if (o.precond == 2 && !pcMinv && cap_run >= PRECOND_CAP_RUN && (q.q64 || q.q32)) {
        // adaptive: the Hessian is too ill-conditioned for max_tcg plain CG steps; precondition
        // every later tCG (this and the following RTR calls).  The chunk graphs captured the
        // unpreconditioned launches; the trust region moves to the B-norm, radius rescaled.
        gcache.clear();
        XM_TRY(enable_precond());
        k_bnorm<To, R><<<nb_cam, CAM_THREADS, 0, st>>>(N, (const To*)bY, pcB, d_sc, ctx->d_partials,
                                                        ctx->d_counter);
        ++launches;
        XM_TRY(pull_scalars());
        const double bar_b = std::sqrt(std::max(h_sc->dot, 1e-300));
        Delta *= bar_b / Delta_bar;
        Delta_bar = bar_b;
        if (o.verbose >= 1) fprintf(stderr, "[xm] tCG at its cap %d times: block-Jacobi preconditioner on\n", cap_run);
      }
    }
    info.f = f;
    cur_g2 = g2;
    return XM_OK;
  }

  // w = Z v (v, w: FP64 n_pad vectors), Z = Q - blockdiag(Lam)
  // w = Z v (Z = Q + diag(dreg) - blockdiag(Lam)) for a basis vector v of type VT (n_pad long)
  template <typename VT>
  xm_status zmul(int prec, const VT* v, double* w) {
    const int nn = n_pad;
    if (prec == XM_FP64) {
      const double* vd = reinterpret_cast<const double*>(v);
      if (sizeof(VT) != 8) {
        k_cast<VT, double><<<grid_elems(nn), CAM_THREADS, 0, st>>>((size_t)nn, v, lritz_tmp());
        ++launches;
        vd = lritz_tmp();
      }
      XM_TRY(sweep(XM_FP64, 1, vd, lz, nullptr, false));
      k_zv_epi<double, double><<<nb_cam, CAM_THREADS, 0, st>>>(N, lz, vd, Lam, w);
    } else {
      const float* vf = reinterpret_cast<const float*>(v);
      if (sizeof(VT) != 4) {
        k_cast<VT, float><<<grid_elems(nn), CAM_THREADS, 0, st>>>((size_t)nn, v, lv32);
        ++launches;
        vf = lv32;
      }
      XM_TRY(sweep(XM_FP32_BULK, 1, vf, lW32, nullptr, false));
      k_zv_epi<float, float><<<nb_cam, CAM_THREADS, 0, st>>>(N, lW32, vf, Lam, w);
    }
    ++launches;
    XM_CUDA_TRY(cudaGetLastError());
    return XM_OK;
  }
  double* lritz_tmp() { return lz + n_pad; }   // second half of the lz scratch

  // classical Gram-Schmidt pass of w against the first m columns of V (basis type VT)
  template <typename VT>
  xm_status reorth(double* w, int m) {
    if (m <= 0) return XM_OK;
    const int nn = n_pad;
    const VT* Vb = static_cast<const VT*>(V);
    const VT* wv;
    if (sizeof(VT) == 4) {
      k_cast<double, float><<<grid_elems(nn), CAM_THREADS, 0, st>>>((size_t)nn, w, lwf);
      ++launches;
      wv = reinterpret_cast<const VT*>(lwf);
    } else {
      wv = reinterpret_cast<const VT*>(w);
    }
    k_gemv_t<VT><<<std::min(m, ctx->num_sms * 8), 256, 0, st>>>(nn, m, Vb, nn, wv, lc, lcf);
    // w -= V c over a (row block, column chunk) grid of about 8 blocks per SM
    const int xb = (nn + 255) / 256;
    const int S = std::max(1, std::min({m, LPART_MAX, (ctx->num_sms * 8 + xb - 1) / xb}));
    const int chunk = (m + S - 1) / S;
    k_gemv_n_part<VT><<<dim3(xb, (m + chunk - 1) / chunk), 256, 0, st>>>(nn, m, Vb, nn, lc, lcf, chunk, lpart);
    k_gemv_n_finish<<<grid_elems(nn), CAM_THREADS, 0, st>>>(nn, (m + chunk - 1) / chunk, lpart, w);
    launches += 3;
    XM_CUDA_TRY(cudaGetLastError());
    return XM_OK;
  }

  // ---------------- Lanczos on Z restricted to range(Y)^perp (Thm. 1 certificate)
  // The basis is FP32 when the Z products are FP32 sweeps, FP64 otherwise.
  template <int R>
  xm_status certify(int r, int prec_z, double* lam_def, double* lam_max, double* lam_range,
                    int kcap_steps = 0) {
    if (prec_z == XM_FP64) return certify_t<R, double>(r, prec_z, lam_def, lam_max, lam_range, kcap_steps);
    if (kcap_steps == 0 && o.cert_lobpcg) {
      bool conv = false;
      XM_TRY(certify_lobpcg<R>(r, lam_def, lam_max, lam_range, &conv));
      if (conv) return XM_OK;
      if (o.verbose >= 1) fprintf(stderr, "[xm] LOBPCG certificate did not converge: Lanczos\n");
    }
    return certify_t<R, float>(r, prec_z, lam_def, lam_max, lam_range, kcap_steps);
  }

  // Rayleigh-Ritz on the active columns of S = [X W P] (nb blocks of 4) from the 15 Gram blocks
  // (SVQB: columns scaled to unit norm, near-dependent directions of S^T S dropped); C, CP:
  // 12 x 4 coefficients of the 4 smallest Ritz vectors and of their [W P] part; false when
  // fewer than 4 independent directions remain.
  static bool lob_rayleigh_ritz(const double* blk, int nb, double* C, double* CP, double* theta) {
    const int m = 4 * nb;
    auto gidx = [](int a, int b) { static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}}; return t[a][b]; };
    std::vector<double> G((size_t)m * m), H((size_t)m * m);
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b)
        for (int x = 0; x < 4; ++x)
          for (int y = 0; y < 4; ++y) {
            G[(size_t)(4 * a + x) * m + 4 * b + y] =
                a <= b ? blk[gidx(a, b) * 16 + x * 4 + y] : blk[gidx(b, a) * 16 + y * 4 + x];
            H[(size_t)(4 * a + x) * m + 4 * b + y] = blk[(6 + 3 * a + b) * 16 + x * 4 + y];
          }
    std::vector<double> Dn(m), Gn((size_t)m * m), Hn((size_t)m * m);
    double gmax = 0.0;
    for (int j = 0; j < m; ++j) gmax = std::max(gmax, G[(size_t)j * m + j]);
    for (int j = 0; j < m; ++j) {
      const double g = G[(size_t)j * m + j];
      Dn[j] = (g > 1e-20 * gmax && g > 0.0) ? 1.0 / std::sqrt(g) : 0.0;
    }
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        Gn[(size_t)a * m + b] = 0.5 * (G[(size_t)a * m + b] + G[(size_t)b * m + a]) * Dn[a] * Dn[b];
        Hn[(size_t)a * m + b] = 0.5 * (H[(size_t)a * m + b] + H[(size_t)b * m + a]) * Dn[a] * Dn[b];
      }
    std::vector<double> w, V;
    sym_eig_desc(m, Gn, w, V);
    std::vector<int> keep;
    for (int j = 0; j < m; ++j)
      if (w[j] > 1e-10 * w[0]) keep.push_back(j);
    const int k = (int)keep.size();
    if (k < 4) return false;
    std::vector<double> Bm((size_t)m * k);   // m x k: kept eigenvectors / sqrt(eigenvalue)
    for (int a = 0; a < m; ++a)
      for (int c = 0; c < k; ++c) Bm[(size_t)a * k + c] = V[(size_t)a * m + keep[c]] / std::sqrt(w[keep[c]]);
    std::vector<double> Hr((size_t)k * k, 0.0);
    for (int c = 0; c < k; ++c)
      for (int d = 0; d < k; ++d) {
        double t = 0.0;
        for (int a = 0; a < m; ++a)
          for (int b = 0; b < m; ++b) t += Bm[(size_t)a * k + c] * Hn[(size_t)a * m + b] * Bm[(size_t)b * k + d];
        Hr[(size_t)c * k + d] = t;
      }
    for (int c = 0; c < k; ++c)
      for (int d = c + 1; d < k; ++d) Hr[(size_t)c * k + d] = Hr[(size_t)d * k + c] = 0.5 * (Hr[(size_t)c * k + d] + Hr[(size_t)d * k + c]);
    std::vector<double> hw, HV;
    sym_eig_desc(k, Hr, hw, HV);   // descending: the 4 smallest are the last
    for (int i = 0; i < 48; ++i) { C[i] = 0.0; CP[i] = 0.0; }
    for (int j = 0; j < 4; ++j) {
      const int col = k - 1 - j;
      theta[j] = hw[col];
      for (int a = 0; a < m; ++a) {
        double t = 0.0;
        for (int c = 0; c < k; ++c) t += Bm[(size_t)a * k + c] * HV[(size_t)c * k + col];
        C[a * 4 + j] = Dn[a] * t;
        CP[a * 4 + j] = a >= 4 ? Dn[a] * t : 0.0;
      }
    }
    return true;
  }

  // Thm. 1 certificate with FP32 Z products by LOBPCG (Knyazev 2001) on Z restricted to
  // range(Y)^perp: blocks of 4 vectors (one R = 4 sweep per iteration), 3 x 3 block-Jacobi
  // preconditioner of Z, Rayleigh-Ritz in FP64.  lambda_max and the Rayleigh quotients on
  // range(Y) come from a 40-step Lanczos run.  Stops when the smallest Ritz pair's residual is
  // <= 1e-6 |lambda_max| (its Ritz value is then within that of lambda_min); *converged = false
  // after 300 iterations (the caller falls back to Lanczos).
  template <int R>
  xm_status certify_lobpcg(int r, double* lam_def, double* lam_max, double* lam_range, bool* converged) {
    *converged = false;
    auto tic = std::chrono::steady_clock::now();
    const double t_cert_before = info.t_cert_s;
    double ld_short = 0.0;
    XM_TRY(certify_t<R, float>(r, XM_FP32_BULK, &ld_short, lam_max, lam_range, 40));
    if (!q.q64 && !q.q32) return XM_OK;   // the preconditioner reads Q's diagonal blocks
    const int nn = n_pad, nd = last_nd;
    const float* Vd = static_cast<const float*>(V);
    const size_t blk = (size_t)nn * 4;
    if (!lob) {
      XM_CUDA_TRY(cudaMalloc(&lob, sizeof(float) * blk * 12));
      XM_CUDA_TRY(cudaMemsetAsync(lob, 0, sizeof(float) * blk * 12, st));
      XM_CUDA_TRY(cudaMalloc(&lob_minv, sizeof(double) * 9 * (size_t)N));
      lob_nxb = std::max(1, std::min((nn + 255) / 256, ctx->num_sms * 2));
      XM_CUDA_TRY(cudaMalloc(&lob_part, sizeof(double) * 15 * 16 * (size_t)lob_nxb));
      XM_CUDA_TRY(cudaMalloc(&lob_small, sizeof(double) * 512));
    }
    float *X = lob, *ZX = lob + blk, *W = lob + 2 * blk, *ZW = lob + 3 * blk, *P = lob + 4 * blk,
          *ZP = lob + 5 * blk, *X2 = lob + 6 * blk, *ZX2 = lob + 7 * blk, *P2 = lob + 8 * blk,
          *ZP2 = lob + 9 * blk, *Wz = lob + 10 * blk, *Zero = lob + 11 * blk;
    double* gram = lob_small;          // 15 x 16
    double* dC = lob_small + 240;      // 48
    double* dCP = lob_small + 288;     // 48
    double* dth = lob_small + 336;     // 4
    double* dnorm = lob_small + 344;   // 4
    double* dcoef = lob_small + 352;   // 32
    const int gv = grid_elems((size_t)nn);
    auto deflate = [&](float* B) {
      if (nd == 0) return;
      k_lob_defl_coef<float><<<gv, CAM_THREADS, 0, st>>>(nn, nd, Vd, nn, B, ctx->d_partials, ctx->d_counter, dcoef);
      k_lob_defl_apply<float><<<gv, CAM_THREADS, 0, st>>>(nn, nd, Vd, nn, dcoef, B);
      launches += 2;
    };
    auto zmul4 = [&](float* B, float* ZB) -> xm_status {
      XM_TRY(sweep(XM_FP32_BULK, 4, B, Wz, nullptr, false));
      k_zv4<<<nb_cam, CAM_THREADS, 0, st>>>(N, Wz, B, Lam, ZB);
      ++launches;
      return XM_OK;
    };
    std::vector<double> hblk(15 * 16 + 8);
    auto gram_rr = [&](float* S1, float* ZS1, float* S2, float* ZS2, int nb, double* theta, bool* ok) -> xm_status {
      LobBlocks Bk{{X, S1, S2}, {ZX, ZS1, ZS2}};
      k_lob_gram<<<dim3(lob_nxb, 15), 256, 0, st>>>(nn, Bk, lob_part);
      k_lob_gram_finish<<<1, 256, 0, st>>>(lob_nxb, lob_part, gram);
      launches += 2;
      XM_CUDA_TRY(cudaMemcpyAsync(hblk.data(), gram, sizeof(double) * 15 * 16, cudaMemcpyDeviceToHost, st));
      XM_CUDA_TRY(cudaMemcpyAsync(hblk.data() + 240, dnorm, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
      XM_CUDA_TRY(cudaStreamSynchronize(st));
      double C[48], CP[48];
      *ok = lob_rayleigh_ritz(hblk.data(), nb, C, CP, theta);
      if (!*ok) return XM_OK;
      XM_CUDA_TRY(cudaMemcpyAsync(dC, C, sizeof(C), cudaMemcpyHostToDevice, st));
      XM_CUDA_TRY(cudaMemcpyAsync(dCP, CP, sizeof(CP), cudaMemcpyHostToDevice, st));
      XM_CUDA_TRY(cudaMemcpyAsync(dth, theta, sizeof(double) * 4, cudaMemcpyHostToDevice, st));
      k_lob_update<<<gv, CAM_THREADS, 0, st>>>(nn, Bk, dC, dCP, X2, ZX2, P2, ZP2);
      ++launches;
      std::swap(X, X2); std::swap(ZX, ZX2); std::swap(P, P2); std::swap(ZP, ZP2);
      // the host copies above read C and CP before they go out of scope
      XM_CUDA_TRY(cudaStreamSynchronize(st));
      return XM_OK;
    };
    if (q.q64) k_zblock_precond<double><<<nb_cam, CAM_THREADS, 0, st>>>(N, q.q64, q.nt, Lam, lob_minv);
    else k_zblock_precond<float><<<nb_cam, CAM_THREADS, 0, st>>>(N, q.q32, q.nt, Lam, lob_minv);
    k_lob_random<<<gv, CAM_THREADS, 0, st>>>(nn, n, o.seed ^ 0x5DEECE66Dull, X);
    launches += 2;
    deflate(X);
    XM_TRY(zmul4(X, ZX));
    double theta[4] = {0, 0, 0, 0};
    bool ok = false;
    XM_TRY(gram_rr(Zero, Zero, Zero, Zero, 1, theta, &ok));   // orthonormal Ritz basis of span X
    if (!ok) return XM_OK;
    const double tol = 1e-6 * std::max(std::fabs(*lam_max), 1e-300);
    bool have_p = false;
    int it = 0;
    double rn0 = 0.0;
    for (it = 1; it <= 300; ++it) {
      k_lob_resid<<<nb_cam, CAM_THREADS, 0, st>>>(N, X, ZX, dth, lob_minv, W, ctx->d_partials, ctx->d_counter, dnorm);
      ++launches;
      deflate(W);
      XM_TRY(zmul4(W, ZW));
      XM_TRY(gram_rr(W, ZW, have_p ? P : Zero, have_p ? ZP : Zero, have_p ? 3 : 2, theta, &ok));
      rn0 = std::sqrt(std::max(hblk[240], 0.0));   // residual of the Ritz pair before this update
      ++info.n_lanczos;
      if (!ok) return XM_OK;
      if (rn0 <= tol) { *converged = true; break; }
      have_p = true;
      XM_CUDA_TRY(cudaGetLastError());
    }
    if (!*converged) return XM_OK;
    *lam_def = theta[0];
    // escape direction: the Ritz vector of theta_min (FP64)
    k_lob_col<<<gv, CAM_THREADS, 0, st>>>(nn, 0, X, lritz);
    ++launches;
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    info.lanczos_converged = 1;
    info.t_cert_s = t_cert_before + std::chrono::duration<double>(std::chrono::steady_clock::now() - tic).count();
    if (o.verbose >= 1)
      fprintf(stderr, "[xm] LOBPCG certificate: %d iterations, theta_min=%.6e residual=%.3e\n", it,
              theta[0], rn0);
    return XM_OK;
  }

  template <int R, typename VT>
  xm_status certify_t(int r, int prec_z, double* lam_def, double* lam_max, double* lam_range,
                      int kcap_steps) {
    auto tic = std::chrono::steady_clock::now();
    const int nn = n_pad;
    const int nd_max = XM_MAX_RANK;
    if (!V) {
      kmax = std::max(10, std::min(o.lanczos_max, n));
      XM_CUDA_TRY(cudaMalloc(&V, sizeof(double) * (size_t)nn * (nd_max + kmax + 1)));   // room for FP64
      XM_CUDA_TRY(cudaMalloc(&lw, sizeof(double) * nn));
      XM_CUDA_TRY(cudaMemsetAsync(lw, 0, sizeof(double) * nn, st));
      XM_CUDA_TRY(cudaMalloc(&lz, sizeof(double) * 2 * (size_t)nn));
      XM_CUDA_TRY(cudaMalloc(&lritz, sizeof(double) * nn));
      XM_CUDA_TRY(cudaMalloc(&lpart, sizeof(double) * (size_t)LPART_MAX * nn));
      XM_CUDA_TRY(cudaMalloc(&lalpha, sizeof(double) * (kmax + 1)));
      XM_CUDA_TRY(cudaMalloc(&lbeta, sizeof(double) * (kmax + 1)));
      XM_CUDA_TRY(cudaMalloc(&lc, sizeof(double) * (nd_max + kmax + 2)));
      XM_CUDA_TRY(cudaMalloc(&lcf, sizeof(float) * (nd_max + kmax + 2)));
      XM_CUDA_TRY(cudaMalloc(&lnrm, sizeof(double) * 2));
      XM_CUDA_TRY(cudaMalloc(&lv32, sizeof(float) * nn));
      XM_CUDA_TRY(cudaMalloc(&lW32, sizeof(float) * nn));
      XM_CUDA_TRY(cudaMalloc(&lwf, sizeof(float) * nn));
      XM_CUDA_TRY(cudaMemsetAsync(lz, 0, sizeof(double) * 2 * (size_t)nn, st));
      XM_CUDA_TRY(cudaMemsetAsync(lritz, 0, sizeof(double) * nn, st));
      XM_CUDA_TRY(cudaMemsetAsync(lW32, 0, sizeof(float) * nn, st));
    }
    VT* Vb = static_cast<VT*>(V);
    const int gv = grid_elems((size_t)nn);
    // orthonormal basis of range(Y) from the Gram matrix (first r columns)
    k_gram<double, R><<<grid_gram(), CAM_THREADS, 0, st>>>(nn, (const double*)bY64, d_small,
                                                           ctx->d_partials, ctx->d_counter);
    ++launches;
    std::vector<double> gram(R * R);
    XM_CUDA_TRY(cudaMemcpyAsync(gram.data(), d_small, sizeof(double) * R * R, cudaMemcpyDeviceToHost, st));
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> gr((size_t)r * r), ew, EV;
    for (int a = 0; a < r; ++a) for (int b = 0; b < r; ++b) gr[(size_t)a * r + b] = gram[a * R + b];
    sym_eig_desc(r, gr, ew, EV);
    int nd = 0;
    std::vector<double> rot((size_t)R * R, 0.0);   // R x R: column j = E_j / sqrt(w_j)
    for (int j = 0; j < r; ++j)
      if (ew[j] > 1e-10 * ew[0]) {
        for (int a = 0; a < r; ++a) rot[(size_t)a * R + nd] = EV[(size_t)a * r + j] / std::sqrt(ew[j]);
        ++nd;
      }
    // V[:, j] = Y rot[:, j] for j < nd, through a row-major staging copy in bXi
    XM_CUDA_TRY(cudaMemcpyAsync(bXi, bY64, sizeof(double) * (size_t)nn * R, cudaMemcpyDeviceToDevice, st));
    XM_CUDA_TRY(cudaMemcpyAsync(d_small + 64, rot.data(), sizeof(double) * R * R, cudaMemcpyHostToDevice, st));
    k_rotate<R><<<(nn + 127) / 128, 128, 0, st>>>(nn, (double*)bXi, d_small + 64);
    ++launches;
    for (int j = 0; j < nd; ++j) {
      k_col_from_rows<VT, R><<<gv, CAM_THREADS, 0, st>>>(nn, j, (const double*)bXi, Vb + (size_t)j * nn);
      ++launches;
    }
    last_nd = nd;
    // Rayleigh quotients of Z on range(Y): Vd^T Z Vd (nd x nd).  With the FP64 gradient at hand,
    // Vd^T Z Vd = rot^T (Y^T G / 2) rot in FP64 (G = 2 Z Y, App. D's term included); otherwise
    // one Z product per basis vector in the certificate's precision.
    std::vector<double> zr((size_t)nd * nd, 0.0);
    if (g64_valid && nd > 0) {
      k_cross<double, R><<<grid_gram(), CAM_THREADS, 0, st>>>(nn, (const double*)bY64, (const double*)bG,
                                                              d_small, ctx->d_partials, ctx->d_counter);
      ++launches;
      std::vector<double> yg(R * R);
      XM_CUDA_TRY(cudaMemcpyAsync(yg.data(), d_small, sizeof(double) * R * R, cudaMemcpyDeviceToHost, st));
      XM_CUDA_TRY(cudaStreamSynchronize(st));
      for (int j = 0; j < nd; ++j)
        for (int l = 0; l < nd; ++l) {
          double acc = 0.0;
          for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b)
              acc += rot[(size_t)a * R + j] * 0.5 * yg[a * R + b] * rot[(size_t)b * R + l];
          zr[(size_t)j * nd + l] = acc;
        }
    }
    for (int j = 0; j < nd && !g64_valid; ++j) {
      XM_TRY(zmul<VT>(prec_z, Vb + (size_t)j * nn, lw));
      const VT* wv = reinterpret_cast<const VT*>(lw);
      if (sizeof(VT) == 4) {
        k_cast<double, float><<<gv, CAM_THREADS, 0, st>>>((size_t)nn, lw, lwf);
        ++launches;
        wv = reinterpret_cast<const VT*>(lwf);
      }
      k_gemv_t<VT><<<nd, 256, 0, st>>>(nn, nd, Vb, nn, wv, lc, nullptr);
      ++launches;
      std::vector<double> cj(nd);
      XM_CUDA_TRY(cudaMemcpyAsync(cj.data(), lc, sizeof(double) * nd, cudaMemcpyDeviceToHost, st));
      XM_CUDA_TRY(cudaStreamSynchronize(st));
      for (int l = 0; l < nd; ++l) zr[(size_t)j * nd + l] = cj[l];
    }
    if (nd > 0) {
      for (int a = 0; a < nd; ++a) for (int b = a + 1; b < nd; ++b) {
        const double m = 0.5 * (zr[(size_t)a * nd + b] + zr[(size_t)b * nd + a]);
        zr[(size_t)a * nd + b] = zr[(size_t)b * nd + a] = m;
      }
      std::vector<double> zw, zv;
      sym_eig_desc(nd, zr, zw, zv);
      *lam_range = zw[nd - 1];
    } else {
      *lam_range = 0.0;
    }
    // start vector (FP64 working vector, then normalised into the basis)
    k_random_vec<<<gv, CAM_THREADS, 0, st>>>(n, o.seed, lw);
    XM_CUDA_TRY(cudaMemsetAsync(lw + n, 0, sizeof(double) * (nn - n), st));
    ++launches;
    XM_TRY(reorth<VT>(lw, nd));
    k_dot<double, double><<<gv, CAM_THREADS, 0, st>>>((size_t)nn, lw, lw, lnrm, ctx->d_partials, ctx->d_counter);
    k_normalize<VT><<<gv, CAM_THREADS, 0, st>>>(nn, lw, lnrm, Vb + (size_t)nd * nn, nullptr);
    launches += 2;
    std::vector<double> ha(kmax + 1), hb(kmax + 1), s;
    int K = 0;
    double th_min = 0, th_max = 0;
    bool conv = false, met = false;
    const int kcap = std::min(kcap_steps > 0 ? std::min(kcap_steps, kmax) : kmax, n - nd);
    for (int k = 0; k < kcap; ++k) {
      const VT* vk = Vb + (size_t)(nd + k) * nn;
      const VT* vkm1 = k > 0 ? Vb + (size_t)(nd + k - 1) * nn : nullptr;
      XM_TRY(zmul<VT>(prec_z, vk, lw));
      k_dot<VT, double><<<gv, CAM_THREADS, 0, st>>>((size_t)nn, vk, lw, lalpha + k, ctx->d_partials, ctx->d_counter);
      k_lanczos_3term<VT><<<gv, CAM_THREADS, 0, st>>>(nn, lw, vk, vkm1, lalpha, lbeta, k);
      launches += 2;
      XM_TRY(reorth<VT>(lw, nd + k + 1));
      XM_TRY(reorth<VT>(lw, nd + k + 1));
      k_dot<double, double><<<gv, CAM_THREADS, 0, st>>>((size_t)nn, lw, lw, lnrm, ctx->d_partials, ctx->d_counter);
      k_normalize<VT><<<gv, CAM_THREADS, 0, st>>>(nn, lw, lnrm, Vb + (size_t)(nd + k + 1) * nn, lbeta + k);
      launches += 2;
      XM_CUDA_TRY(cudaGetLastError());
      ++info.n_lanczos;
      K = k + 1;
      if ((K % 10) == 0 || K == kcap) {
        XM_CUDA_TRY(cudaMemcpyAsync(ha.data(), lalpha, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
        XM_CUDA_TRY(cudaMemcpyAsync(hb.data(), lbeta, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
        XM_CUDA_TRY(cudaStreamSynchronize(st));
        th_min = tri_eig_bisect(K, ha.data(), hb.data(), 0);
        th_max = tri_eig_bisect(K, ha.data(), hb.data(), K - 1);
        tri_eigvec(K, ha.data(), hb.data(), th_min, s);
        const double res = std::fabs(hb[K - 1] * s[K - 1]);
        const double scale = std::max(std::fabs(th_max), std::fabs(th_min)) + 1e-300;
        met = res <= o.lanczos_tol * scale || hb[K - 1] <= 1e-14 * scale || K == n - nd;
        if (met || K == kcap) {
          conv = true;
          break;
        }
      }
    }
    if (!conv && K > 0) {
      XM_CUDA_TRY(cudaMemcpyAsync(ha.data(), lalpha, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
      XM_CUDA_TRY(cudaMemcpyAsync(hb.data(), lbeta, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
      XM_CUDA_TRY(cudaStreamSynchronize(st));
      th_min = tri_eig_bisect(K, ha.data(), hb.data(), 0);
      th_max = tri_eig_bisect(K, ha.data(), hb.data(), K - 1);
      tri_eigvec(K, ha.data(), hb.data(), th_min, s);
    }
    info.lanczos_converged = (met || K == 0) ? 1 : 0;
    // Ritz vector of theta_min -> lritz (k_gemv_n_sub subtracts: lritz = -V s; the sign of an
    // eigenvector is irrelevant)
    if (K > 0) {
      std::vector<float> sf(K);
      for (int j = 0; j < K; ++j) sf[j] = float(s[j]);
      XM_CUDA_TRY(cudaMemcpyAsync(lc, s.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st));
      XM_CUDA_TRY(cudaMemcpyAsync(lcf, sf.data(), sizeof(float) * K, cudaMemcpyHostToDevice, st));
      XM_CUDA_TRY(cudaMemsetAsync(lritz, 0, sizeof(double) * nn, st));
      k_gemv_n_sub<VT><<<gv, CAM_THREADS, 0, st>>>(nn, K, Vb + (size_t)nd * nn, nn, lc, lcf, lritz);
      ++launches;
    }
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    *lam_def = th_min;
    *lam_max = th_max;
    info.t_cert_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - tic).count();
    return XM_OK;
  }

  // ---------------- rounding (Sec. 2.2) and the Eq. 18 / App. E numbers
  template <int R>
  xm_status round_and_eval(int r, double* R_out, double* s_out, double* G_out) {
    const int nn = n_pad;
    k_gram<double, R><<<grid_gram(), CAM_THREADS, 0, st>>>(nn, (const double*)bY64, d_small,
                                                           ctx->d_partials, ctx->d_counter);
    ++launches;
    std::vector<double> gram(R * R);
    XM_CUDA_TRY(cudaMemcpyAsync(gram.data(), d_small, sizeof(double) * R * R, cudaMemcpyDeviceToHost, st));
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> gr((size_t)r * r), ew, EV;
    for (int a = 0; a < r; ++a) for (int b = 0; b < r; ++b) gr[(size_t)a * r + b] = gram[a * R + b];
    sym_eig_desc(r, gr, ew, EV);
    // Yh = Y V3 (n_pad x 4, last column zero): a rotation padded to R x R then truncated
    std::vector<double> rot((size_t)R * R, 0.0);
    for (int a = 0; a < r; ++a) for (int j = 0; j < 3 && j < r; ++j) rot[(size_t)a * R + j] = EV[(size_t)a * r + j];
    XM_CUDA_TRY(cudaMemcpyAsync(bXi, bY64, sizeof(double) * (size_t)nn * R, cudaMemcpyDeviceToDevice, st));
    XM_CUDA_TRY(cudaMemcpyAsync(d_small + 64, rot.data(), sizeof(double) * R * R, cudaMemcpyHostToDevice, st));
    k_rotate<R><<<(nn + 127) / 128, 128, 0, st>>>(nn, (double*)bXi, d_small + 64);
    k_repad<double, double><<<grid_elems((size_t)nn * 4), CAM_THREADS, 0, st>>>(nn, nn, (const double*)bXi, R,
                                                                          (double*)bYh, 4);
    launches += 2;
    // anchor block -> O0 = polar(Ubar_0), Ubar_0 = Yh_0^T
    double yh0[12];
    XM_CUDA_TRY(cudaMemcpyAsync(yh0, bYh, sizeof(double) * 12, cudaMemcpyDeviceToHost, st));
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> Ub(9), UtU(9), w3, V3;
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) Ub[a * 3 + b] = yh0[b * 4 + a];
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
      double t = 0; for (int k = 0; k < 3; ++k) t += Ub[k * 3 + a] * Ub[k * 3 + b];
      UtU[a * 3 + b] = t;
    }
    sym_eig_desc(3, UtU, w3, V3);
    double O0[9];   // Ub V diag(1/sig) V^T
    for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
      double t = 0;
      for (int k = 0; k < 3; ++k) {
        const double sig = std::sqrt(std::max(w3[k], 1e-300));
        double uk = 0; for (int m = 0; m < 3; ++m) uk += Ub[a * 3 + m] * V3[m * 3 + k];
        t += uk / sig * V3[b * 3 + k];
      }
      O0[a * 3 + b] = t;
    }
    XM_CUDA_TRY(cudaMemcpyAsync(d_small + 128, O0, sizeof(O0), cudaMemcpyHostToDevice, st));
    double* Rd = (double*)bXi;                  // N x 9 scratch (9N <= 8 n_pad doubles)
    double* sd = Lamc;                          // N scratch
    XM_CUDA_TRY(cudaMemsetAsync(bYc, 0, vec_bytes, st));
    k_round<<<nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)bYh, d_small + 128, Rd, sd, (double*)bYc);
    ++launches;
    XM_CUDA_TRY(cudaGetLastError());
    if (G_out) {   // G_i = s_i R_i: the rounded block of camera i, as Yhat holds it (Yhat_i = G_i^T)
      k_round_G<<<nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)bYc, G_out);
      ++launches;
    }
    if (R_out) XM_CUDA_TRY(cudaMemcpyAsync(R_out, Rd, sizeof(double) * 9 * N, cudaMemcpyDeviceToDevice, st));
    if (s_out) XM_CUDA_TRY(cudaMemcpyAsync(s_out, sd, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    // rho_hat = f(Yhat) in FP64
    XM_CUDA_TRY(cudaMemsetAsync(bWc, 0, vec_bytes, st));
    XM_TRY(sweep(XM_FP64, 4, bYc, bWc, nullptr, false));
    k_dot<double, double><<<grid_elems((size_t)nn * 4), CAM_THREADS, 0, st>>>(
        (size_t)nn * 4, (const double*)bYc, (const double*)bWc, d_slot(), ctx->d_partials,
        ctx->d_counter);
    ++launches;
    double rho_hat = 0;
    XM_CUDA_TRY(cudaMemcpyAsync(&rho_hat, d_slot(), sizeof(double), cudaMemcpyDeviceToHost, st));
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    XM_CUDA_TRY(cudaMemsetAsync(bWc, 0, vec_bytes, st));
    if (o.scale_reg != 0.0) {   // + F(Xhat) = mu sum (s_i^2 - 1)^2 (App. D)
      k_reg_terms<4><<<nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)bYc, d_sc, ctx->d_partials,
                                                     ctx->d_counter);
      ++launches;
      XM_CUDA_TRY(cudaGetLastError());
      XM_TRY(pull_scalars());
      rho_hat += h_sc->dot;
    }
    info.rho_hat = rho_hat;
    return XM_OK;
  }
};

// ------------------------------------------------------------------ staircase driver
template <typename F4, typename F8>
static xm_status with_R(int R, F4 f4, F8 f8) {
  return R == 4 ? f4() : f8();
}

// Alg. 1's start [I_3, ..., I_3] padded to rank r with zero columns, plus jitter * u in columns
// 3..r-1, u uniform in [-1, 1) from splitmix64 of (seed, element index).
__global__ void k_init_identity(int N, int R, int r, double jitter, uint64_t seed, double* Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) init_block(i, R, r, jitter, seed, Y);
}

__global__ void k_set_col(int n, int n_rows, int R, int col, const double* v, double* Xi) {
  const size_t total = (size_t)n_rows * R;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / R), c = (int)(e % R);
    Xi[e] = (c == col && row < n) ? v[row] : 0.0;
  }
}

static double suboptimality(double rho_hat, double rho) {
  return (rho_hat - rho) / (1.0 + std::fabs(rho_hat) + std::fabs(rho));
}

xm_status solve_impl(xm_ctx* ctx, const DeviceQ& q, const xm_opts& o, int r_in, const double* Y0,
                     double* Y_out, double* R_out, double* s_out, double* G_out, xm_info* out_info,
                     bool certify_only, double* Lambda_out, double* v_out) {
  Solver S(ctx, q, o);
  S.t_start = std::chrono::steady_clock::now();
  XM_TRY(S.alloc());
  cudaStream_t st = ctx->stream;
  const int N = q.N, n = q.n, nn = q.n_pad;
  const bool fp64_mode = o.prec == XM_FP64;
  const int prec_hvp = o.prec == XM_BF16Q_BULK ? XM_BF16Q_BULK : (fp64_mode ? XM_FP64 : XM_FP32_BULK);
  const int prec_z = fp64_mode ? XM_FP64 : XM_FP32_BULK;

  int r = Y0 ? r_in : o.r0;
  int R = r <= 4 ? 4 : 8;
  // initial point (FP64, n_pad x R)
  if (Y0) {
    k_repad<double, double><<<S.grid_elems((size_t)nn * R), CAM_THREADS, 0, st>>>(
        n, nn, Y0, r_in, (double*)S.bY64, R);
    XM_CUDA_TRY(cudaMemsetAsync(S.bXi, 0, S.vec_bytes, st));
    // make it feasible: retract with a zero step
    XM_TRY(with_R(R,
        [&] { k_retract<double, double, 4><<<S.nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)S.bY64, (const double*)S.bXi, 0.0, (double*)S.bYc); return XM_OK; },
        [&] { k_retract<double, double, 8><<<S.nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)S.bY64, (const double*)S.bXi, 0.0, (double*)S.bYc); return XM_OK; }));
    XM_CUDA_TRY(cudaMemcpyAsync(S.bY64, S.bYc, sizeof(double) * (size_t)nn * R, cudaMemcpyDeviceToDevice, st));
    S.launches += 2;
  } else {
    k_init_identity<<<S.nb_cam, CAM_THREADS, 0, st>>>(N, R, r, o.init_jitter, o.seed, (double*)S.bY64);
    ++S.launches;
    if (o.init_jitter != 0.0 && r > 3) {
      // make the jittered start feasible: retraction with a zero step
      XM_CUDA_TRY(cudaMemsetAsync(S.bXi, 0, S.vec_bytes, st));
      XM_TRY(with_R(R,
          [&] { k_retract<double, double, 4><<<S.nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)S.bY64, (const double*)S.bXi, 0.0, (double*)S.bYc); return XM_OK; },
          [&] { k_retract<double, double, 8><<<S.nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)S.bY64, (const double*)S.bXi, 0.0, (double*)S.bYc); return XM_OK; }));
      XM_CUDA_TRY(cudaMemcpyAsync(S.bY64, S.bYc, sizeof(double) * (size_t)nn * R, cudaMemcpyDeviceToDevice, st));
      ++S.launches;
    }
  }
  XM_CUDA_TRY(cudaGetLastError());

  double lam_def = 0, lam_max = 0, lam_range = 0;
  bool certified = false;
  xm_status result = XM_OK;
  for (;;) {
    const size_t elems = (size_t)nn * R;
    XM_TRY(S.clear_vecs());
    // ---- local optimisation at rank r
    bool quick_escape = false;
    if (certify_only) {
      XM_CUDA_TRY(cudaMemcpyAsync(S.bY, S.bY64, sizeof(double) * elems, cudaMemcpyDeviceToDevice, st));
      XM_TRY(with_R(R, [&] { return S.grad_at<double, 4>(XM_FP64, S.bY, S.bW, S.bG, S.Lam, 0, false); },
                       [&] { return S.grad_at<double, 8>(XM_FP64, S.bY, S.bW, S.bG, S.Lam, 0, false); }));
      XM_TRY(S.pull_scalars());
      S.info.f = S.h_sc->f;
      S.cur_g2 = S.h_sc->g2;
    } else if (fp64_mode) {
      XM_CUDA_TRY(cudaMemcpyAsync(S.bY, S.bY64, sizeof(double) * elems, cudaMemcpyDeviceToDevice, st));
      XM_TRY(with_R(R,
          [&] { return S.rtr<double, double, 4>(XM_FP64, XM_FP64, o.grad_tol_rel, o.max_outer, false); },
          [&] { return S.rtr<double, double, 8>(XM_FP64, XM_FP64, o.grad_tol_rel, o.max_outer, false); }));
      XM_CUDA_TRY(cudaMemcpyAsync(S.bY64, S.bY, sizeof(double) * elems, cudaMemcpyDeviceToDevice, st));
    } else {
      // bulk FP32 phase
      k_cast<double, float><<<S.grid_elems(elems), CAM_THREADS, 0, st>>>(elems, (const double*)S.bY64, (float*)S.bY);
      ++S.launches;
      XM_TRY(with_R(R,
          [&] { return S.rtr<float, float, 4>(XM_FP32_BULK, prec_hvp, o.bulk_tol_rel, o.max_outer, true); },
          [&] { return S.rtr<float, float, 8>(XM_FP32_BULK, prec_hvp, o.bulk_tol_rel, o.max_outer, true); }));
      k_cast<float, double><<<S.grid_elems(elems), CAM_THREADS, 0, st>>>(elems, (const float*)S.bY, (double*)S.bY64);
      ++S.launches;
      XM_CUDA_TRY(cudaGetLastError());
      // Quick certificate with the bulk-phase dual blocks: clearly negative curvature means the
      // rank-r point is a saddle of the SDP (Thm. 2) and an FP64 polish would be wasted.  After
      // a stagnation hand-over the gradient, hence the dual blocks, are too coarse for that
      // test; the FP64 certificate after the polish decides instead.
      if (r < o.r_max && !S.bulk_stalled) {
        // a short Krylov run suffices: strong negative curvature is an extreme eigenvalue
        XM_TRY(with_R(R, [&] { return S.certify<4>(r, XM_FP32_BULK, &lam_def, &lam_max, &lam_range, 60); },
                         [&] { return S.certify<8>(r, XM_FP32_BULK, &lam_def, &lam_max, &lam_range, 60); }));
        if (lam_def < -1e-4 * std::fabs(lam_max)) {
          if (o.verbose >= 1)
            fprintf(stderr, "[xm] rank %d: bulk f=%.12e lam_def=%.6e lam_max=%.6e escape without polish\n",
                    r, S.info.f, lam_def, lam_max);
          quick_escape = true;
        }
      }
      if (!quick_escape) {
        // FP64 polish: FP64 gradient and objective, FP32 Hessian-vector products
        XM_TRY(S.clear_vecs());
        // The widened FP32 iterate is feasible only to FP32 precision; project it back onto the
        // manifold in FP64 (retraction with a zero step) so the polish compares feasible points.
        XM_TRY(with_R(R,
            [&] { k_retract<double, double, 4><<<S.nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)S.bY64, (const double*)S.bXi, 0.0, (double*)S.bY); return XM_OK; },
            [&] { k_retract<double, double, 8><<<S.nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)S.bY64, (const double*)S.bXi, 0.0, (double*)S.bY); return XM_OK; }));
        ++S.launches;
        XM_TRY(with_R(R,
            [&] { return S.rtr<double, float, 4>(XM_FP64, XM_FP32_BULK, o.grad_tol_rel, o.max_polish, false); },
            [&] { return S.rtr<double, float, 8>(XM_FP64, XM_FP32_BULK, o.grad_tol_rel, o.max_polish, false); }));
        XM_CUDA_TRY(cudaMemcpyAsync(S.bY64, S.bY, sizeof(double) * elems, cudaMemcpyDeviceToDevice, st));
      }
    }
    // ---- certificate (FP64 Lambda from the last FP64 gradient)
    double gap = 0.0;
    bool stationary = false;
    if (!quick_escape) {
      // every path here ended with an FP64 gradient at bY64 (FP64 RTR, the FP64 polish, or the
      // certify-only gradient)
      S.g64_valid = true;
      const xm_status sc = with_R(R, [&] { return S.certify<4>(r, prec_z, &lam_def, &lam_max, &lam_range); },
                                     [&] { return S.certify<8>(r, prec_z, &lam_def, &lam_max, &lam_range); });
      S.g64_valid = false;
      XM_TRY(sc);
      // Thm. 1 needs a first-order critical point: with Lambda in closed form the duality gap
      // f - tr(Lambda_0) = <Y, Z Y> vanishes exactly there, so it is checked beside lambda_min.
      double L0g[9], regd = 0.0;
      XM_CUDA_TRY(cudaMemcpy(L0g, S.Lam, sizeof(L0g), cudaMemcpyDeviceToHost));
      XM_TRY(with_R(R, [&] { return S.reg_dual_terms<4>((const double*)S.bY64, &regd); },
                       [&] { return S.reg_dual_terms<8>((const double*)S.bY64, &regd); }));
      gap = S.info.f - (L0g[0] + L0g[4] + L0g[8] + regd);
      stationary = std::fabs(gap) <= 1e-6 * (1.0 + std::fabs(S.info.f));
    }
    const double tau = o.cert_tau_rel * std::max(std::fabs(lam_max), 1e-300);
    certified = !quick_escape && lam_def >= -tau && stationary;
    if (o.verbose >= 1 && !quick_escape)
      fprintf(stderr, "[xm] rank %d: f=%.12e |g|=%.3e gap=%.3e lam_def=%.6e lam_rng=%.3e lam_max=%.6e %s\n",
              r, S.info.f, std::sqrt(S.cur_g2), gap, lam_def, lam_range, lam_max,
              certified ? "CERTIFIED" : "escape");
    if (certified || certify_only) break;
    if (S.timed_out || (!quick_escape && lam_def >= -tau && !stationary)) { result = XM_ENOCONV; break; }
    if (r >= o.r_max) { result = XM_ENOTCERT; break; }
    // ---- escape (Thm. 2): into a null column of Y if one exists, else one rank up
    std::vector<double> gram(R * R);
    XM_TRY(with_R(R,
        [&] { k_gram<double, 4><<<S.grid_gram(), CAM_THREADS, 0, st>>>(nn, (const double*)S.bY64, S.d_small, ctx->d_partials, ctx->d_counter); return XM_OK; },
        [&] { k_gram<double, 8><<<S.grid_gram(), CAM_THREADS, 0, st>>>(nn, (const double*)S.bY64, S.d_small, ctx->d_partials, ctx->d_counter); return XM_OK; }));
    XM_CUDA_TRY(cudaMemcpyAsync(gram.data(), S.d_small, sizeof(double) * R * R, cudaMemcpyDeviceToHost, st));
    XM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> gr((size_t)r * r), ew, EV;
    for (int a = 0; a < r; ++a) for (int b = 0; b < r; ++b) gr[(size_t)a * r + b] = gram[a * R + b];
    sym_eig_desc(r, gr, ew, EV);
    int col;
    if (ew[r - 1] < 1e-12 * ew[0]) {
      std::vector<double> rot((size_t)R * R, 0.0);
      for (int a = 0; a < R; ++a) for (int b = 0; b < R; ++b)
        rot[(size_t)a * R + b] = (a < r && b < r) ? EV[(size_t)a * r + b] : (a == b ? 1.0 : 0.0);
      XM_CUDA_TRY(cudaMemcpyAsync(S.d_small + 64, rot.data(), sizeof(double) * R * R, cudaMemcpyHostToDevice, st));
      XM_TRY(with_R(R, [&] { k_rotate<4><<<(nn + 127) / 128, 128, 0, st>>>(nn, (double*)S.bY64, S.d_small + 64); return XM_OK; },
                       [&] { k_rotate<8><<<(nn + 127) / 128, 128, 0, st>>>(nn, (double*)S.bY64, S.d_small + 64); return XM_OK; }));
      col = r - 1;
    } else {
      const int Rn = (r + 1) <= 4 ? 4 : 8;
      if (Rn != R) {
        k_repad<double, double><<<S.grid_elems((size_t)nn * Rn), CAM_THREADS, 0, st>>>(nn, nn, (const double*)S.bY64, R, (double*)S.bYc, Rn);
        XM_CUDA_TRY(cudaMemcpyAsync(S.bY64, S.bYc, sizeof(double) * (size_t)nn * Rn, cudaMemcpyDeviceToDevice, st));
        R = Rn;
        XM_TRY(S.clear_vecs());
      }
      col = r;
      r += 1;
    }
    S.launches += 2;
    k_set_col<<<S.grid_elems((size_t)nn * R), CAM_THREADS, 0, st>>>(n, nn, R, col, S.lritz, (double*)S.bXi);
    // line search on f in the working precision (FP64 mode: FP64; mixed modes: FP32 sweeps of
    // the FP64-retracted points), against f at alpha = 0 in the same precision
    const bool ls64 = fp64_mode;
    const size_t ls_elems = (size_t)nn * R;
    auto f_at = [&](double a, double* fout) -> xm_status {
      XM_CUDA_TRY(cudaMemsetAsync(S.bWc, 0, S.vec_bytes, st));
      XM_TRY(with_R(R,
          [&] { k_retract<double, double, 4><<<S.nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)S.bY64, (const double*)S.bXi, a, (double*)S.bYh); return XM_OK; },
          [&] { k_retract<double, double, 8><<<S.nb_cam, CAM_THREADS, 0, st>>>(N, (const double*)S.bY64, (const double*)S.bXi, a, (double*)S.bYh); return XM_OK; }));
      ++S.launches;
      if (ls64) {
        XM_TRY(with_R(R, [&] { return S.grad_at<double, 4>(XM_FP64, S.bYh, S.bWc, S.bGc, S.Lamc, 1, false); },
                         [&] { return S.grad_at<double, 8>(XM_FP64, S.bYh, S.bWc, S.bGc, S.Lamc, 1, false); }));
      } else {
        XM_CUDA_TRY(cudaMemsetAsync(S.bYc, 0, S.vec_bytes, st));
        k_cast<double, float><<<S.grid_elems(ls_elems), CAM_THREADS, 0, st>>>(ls_elems, (const double*)S.bYh, (float*)S.bYc);
        ++S.launches;
        XM_TRY(with_R(R, [&] { return S.grad_at<float, 4>(XM_FP32_BULK, S.bYc, S.bWc, S.bGc, S.Lamc, 1, false); },
                         [&] { return S.grad_at<float, 8>(XM_FP32_BULK, S.bYc, S.bWc, S.bGc, S.Lamc, 1, false); }));
      }
      XM_TRY(S.pull_scalars());
      *fout = S.h_sc->fc;
      return XM_OK;
    };
    double f0 = 0.0;
    XM_TRY(f_at(0.0, &f0));
    bool moved = false;
    double alpha = 1.0;
    for (int h = 0; h <= 30; ++h, alpha *= 0.5) {
      double fa = 0.0;
      XM_TRY(f_at(alpha, &fa));
      if (fa < f0) {
        XM_CUDA_TRY(cudaMemcpyAsync(S.bY64, S.bYh, sizeof(double) * (size_t)nn * R, cudaMemcpyDeviceToDevice, st));
        moved = true;
        break;
      }
    }
    ++S.info.n_escapes;
    if (!moved) { result = XM_ENOTCERT; break; }
  }

  // ---- rounding, suboptimality
  XM_TRY(with_R(R, [&] { return S.round_and_eval<4>(r, R_out, s_out, G_out); },
                   [&] { return S.round_and_eval<8>(r, R_out, s_out, G_out); }));
  if (Lambda_out) XM_CUDA_TRY(cudaMemcpyAsync(Lambda_out, S.Lam, sizeof(double) * 9 * N, cudaMemcpyDeviceToDevice, st));
  if (v_out && S.lritz) XM_CUDA_TRY(cudaMemcpyAsync(v_out, S.lritz, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  if (Y_out) {
    k_repad<double, double><<<S.grid_elems((size_t)n * XM_MAX_RANK), CAM_THREADS, 0, st>>>(
        n, n, (const double*)S.bY64, R, Y_out, XM_MAX_RANK);
    ++S.launches;
  }
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  XM_TRY(check_device_error(ctx, "solve"));

  xm_info& I = S.info;
  I.rank = r;
  I.grad_norm = std::sqrt(S.cur_g2);
  I.lambda_min_deflated = lam_def;
  I.lambda_min = std::min(lam_def, lam_range);
  I.lambda_max = lam_max;
  I.certified = certified ? 1 : 0;
  // dual value tr(Lambda_0) (+ F(X) - <grad F(X), X> with App. D's regulariser, App. E)
  double L0[9], regd = 0.0;
  XM_CUDA_TRY(cudaMemcpy(L0, S.Lam, sizeof(L0), cudaMemcpyDeviceToHost));
  XM_TRY(with_R(R, [&] { return S.reg_dual_terms<4>((const double*)S.bY64, &regd); },
                   [&] { return S.reg_dual_terms<8>((const double*)S.bY64, &regd); }));
  I.dual = L0[0] + L0[4] + L0[8] + regd;
  double y2 = 0;
  {
    XM_TRY(with_R(R,
        [&] { k_gram<double, 4><<<S.grid_gram(), CAM_THREADS, 0, st>>>(nn, (const double*)S.bY64, S.d_small, ctx->d_partials, ctx->d_counter); return XM_OK; },
        [&] { k_gram<double, 8><<<S.grid_gram(), CAM_THREADS, 0, st>>>(nn, (const double*)S.bY64, S.d_small, ctx->d_partials, ctx->d_counter); return XM_OK; }));
    std::vector<double> g(R * R);
    XM_CUDA_TRY(cudaMemcpy(g.data(), S.d_small, sizeof(double) * R * R, cudaMemcpyDeviceToHost));
    for (int j = 0; j < R; ++j) y2 += g[j * R + j];
  }
  I.eta = suboptimality(I.rho_hat, I.f);
  const double lower = I.dual + std::min(0.0, I.lambda_min) * y2;
  I.eta_robust = suboptimality(I.rho_hat, lower);
  I.qy_ms_fp32 = S.n32 ? S.ms32 / S.n32 : 0.0;
  I.qy_ms_fp64 = S.n64 ? S.ms64 / S.n64 : 0.0;
  I.t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - S.t_start).count();
  g_last_launches = S.launches;
  g_last_sweeps = S.info.n_sweeps;
  if (out_info) *out_info = I;
  if (result == XM_ENOTCERT)
    return set_error(XM_ENOTCERT, "staircase stopped at rank %d without a certificate (lambda_min %.3e)", r, lam_def);
  if (result == XM_ENOCONV)
    return set_error(XM_ENOCONV, "not converged: time limit, or iteration caps hit before a stationary point");
  return XM_OK;
}

// ====================================================================================== ABI
xm_status build_Q(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                  const double* ukp, const double* w, unsigned mask, DeviceQ& out,
                  double* t_build);

xm_status check_opts(const DeviceQ& q, const xm_opts& o) {
  if (o.r0 < 1 || o.r0 > XM_MAX_RANK || o.r_max < o.r0 || o.r_max > XM_MAX_RANK)
    return set_error(XM_EINVAL, "opts: need 1 <= r0 <= r_max <= %d (r0=%d, r_max=%d)", XM_MAX_RANK,
                     o.r0, o.r_max);
  if (o.prec < XM_FP64 || o.prec > XM_BF16Q_BULK) return set_error(XM_EINVAL, "opts: bad prec %d", o.prec);
  if (!q.q64 && !q.fact)
    return set_error(XM_EINVAL, "solve: Q needs its FP64 copy (XM_STORE_FP64) or the factored operator");
  if (o.precond == 1 && !q.q64 && !q.q32)
    return set_error(XM_EINVAL, "opts: precond = 1 reads Q's diagonal blocks from its FP64 or FP32 tiles");
  if (o.prec != XM_FP64 && !q.q32) return set_error(XM_EINVAL, "solve: mixed precision needs XM_STORE_FP32");
  if (o.prec == XM_BF16Q_BULK && !q.q16) return set_error(XM_EINVAL, "solve: XM_BF16Q_BULK needs XM_STORE_BF16");
  if (o.max_outer < 1 || o.max_tcg < 1 || o.lanczos_max < 1)
    return set_error(XM_EINVAL, "opts: iteration caps must be positive");
  if (!(o.scale_reg >= 0.0) || !std::isfinite(o.scale_reg))
    return set_error(XM_EINVAL, "opts: scale_reg must be finite and >= 0 (got %g)", o.scale_reg);
  if (o.precond < 0 || o.precond > 2) return set_error(XM_EINVAL, "opts: precond must be 0, 1 or 2");
  if (o.cert_lobpcg != 0 && o.cert_lobpcg != 1) return set_error(XM_EINVAL, "opts: cert_lobpcg must be 0 or 1");
  if (!(o.bf16_hvp_until >= 0.0)) return set_error(XM_EINVAL, "opts: bf16_hvp_until must be >= 0");
  if (o.bf16_hvp_until > 0.0 && o.prec == XM_FP32_BULK && !q.q16)
    return set_error(XM_EINVAL, "solve: bf16_hvp_until > 0 needs XM_STORE_BF16");
  if (o.bulk_stall < -1 || o.bulk_stall > o.max_outer)
    return set_error(XM_EINVAL, "opts: bulk_stall must be -1 or in [0, max_outer] (got %d)", o.bulk_stall);
  return XM_OK;
}

template <typename T>
static xm_status qy_generic(xm_ctx* c, const DeviceQ& q, int prec, int r, const T* Y, T* W) {
  const int R = r == 1 ? 1 : (r <= 4 ? 4 : 8);
  cudaStream_t st = c->stream;
  T *Yp = nullptr, *Wp = nullptr;
  const size_t bytes = sizeof(T) * (size_t)q.n_pad * R;
  XM_CUDA_TRY(cudaMallocAsync(&Yp, bytes, st));
  XM_CUDA_TRY(cudaMallocAsync(&Wp, bytes, st));
  const int g = (int)std::min<size_t>(((size_t)q.n_pad * R + 255) / 256, (size_t)c->num_sms * 8);
  k_repad<T, T><<<g, 256, 0, st>>>(q.n, q.n_pad, Y, r, Yp, R);
  XM_CUDA_TRY(cudaMemsetAsync(Wp, 0, bytes, st));
  xm_status s = qy_launch(c, q, prec, R, Yp, Wp, nullptr, st);
  if (s == XM_OK) {
    const int g2 = (int)std::min<size_t>(((size_t)q.n * r + 255) / 256, (size_t)c->num_sms * 8);
    k_repad<T, T><<<std::max(g2, 1), 256, 0, st>>>(q.n, q.n, Wp, R, W, r);
  }
  cudaFreeAsync(Yp, st);
  cudaFreeAsync(Wp, st);
  XM_CUDA_TRY(cudaGetLastError());
  return s;
}

template <typename T>
static xm_status bench_generic(xm_ctx* c, const DeviceQ& q, int prec, int r, int iters, double* ms_mean,
                               double* ms_min) {
  const int R = r == 1 ? 1 : (r <= 4 ? 4 : 8);
  cudaStream_t st = c->stream;
  T *Yp = nullptr, *Wp = nullptr;
  const size_t bytes = sizeof(T) * (size_t)q.n_pad * R;
  XM_CUDA_TRY(cudaMalloc(&Yp, bytes));
  XM_CUDA_TRY(cudaMalloc(&Wp, bytes));
  std::vector<T> hy((size_t)q.n_pad * R, T(0));
  for (int i = 0; i < q.n; ++i)
    for (int j = 0; j < r; ++j) hy[(size_t)i * R + j] = T(((i * 7 + j * 13) % 17) - 8) / T(8);
  xm_status s = XM_OK;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double tot = 0.0, mn = 1e30;
  if (cudaMemcpyAsync(Yp, hy.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    s = set_error(XM_ECUDA, "bench: copy failed");
  for (int it = -3; it < iters && s == XM_OK; ++it) {
    cudaMemsetAsync(Wp, 0, bytes, st);
    cudaEventRecord(e0, st);
    s = qy_launch(c, q, prec, R, Yp, Wp, nullptr, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (it >= 0) { tot += ms; mn = std::min(mn, (double)ms); }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaFree(Yp);
  cudaFree(Wp);
  if (s != XM_OK) return s;
  XM_TRY(check_device_error(c, "sweep benchmark"));
  if (ms_mean) *ms_mean = iters > 0 ? tot / iters : 0.0;
  if (ms_min) *ms_min = mn;
  return XM_OK;
}
}  // namespace xm

using namespace xm;
extern "C" {

xm_status xm_qy(xm_ctx* c, const xm_qmat* q, int prec, int r, const void* Y, void* W) {
  if (!c || !q || !Y || !W) return set_error(XM_EINVAL, "xm_qy: NULL argument");
  if (r < 1 || r > XM_MAX_RANK) return set_error(XM_EINVAL, "xm_qy: r=%d not in [1, %d]", r, XM_MAX_RANK);
  XM_CUDA_TRY(cudaSetDevice(c->device));
  if (prec == XM_FP64) return qy_generic<double>(c, q->d, prec, r, (const double*)Y, (double*)W);
  return qy_generic<float>(c, q->d, prec, r, (const float*)Y, (float*)W);
}

xm_status xm_bench_qy(xm_ctx* c, const xm_qmat* q, int prec, int r, int iters, double* ms_mean,
                      double* ms_min) {
  if (!c || !q || iters < 0) return set_error(XM_EINVAL, "xm_bench_qy: bad argument");
  if (r < 1 || r > XM_MAX_RANK) return set_error(XM_EINVAL, "xm_bench_qy: r=%d", r);
  XM_CUDA_TRY(cudaSetDevice(c->device));
  if (prec == XM_FP64) return bench_generic<double>(c, q->d, prec, r, iters, ms_mean, ms_min);
  return bench_generic<float>(c, q->d, prec, r, iters, ms_mean, ms_min);
}

long xm_last_launch_count(void) { return g_last_launches; }

xm_status xm_solve(xm_ctx* c, const xm_qmat* q, const xm_opts* opts, int r_in, const double* Y0,
                   double* Y_out, double* R_out, double* s_out, double* G_out, xm_info* info) {
  if (!c || !q) return set_error(XM_EINVAL, "xm_solve: NULL context or Q");
  xm_opts o;
  if (opts) o = *opts; else xm_default_opts(&o);
  if (Y0 && (r_in < 1 || r_in > XM_MAX_RANK)) return set_error(XM_EINVAL, "xm_solve: r_in=%d", r_in);
  if (Y0 && r_in > o.r_max) o.r_max = r_in;
  XM_TRY(check_opts(q->d, o));
  XM_CUDA_TRY(cudaSetDevice(c->device));
  return solve_impl(c, q->d, o, r_in, Y0, Y_out, R_out, s_out, G_out, info, false, nullptr, nullptr);
}

xm_status xm_certify(xm_ctx* c, const xm_qmat* q, const xm_opts* opts, int r, const double* Y,
                     double* Lambda_out, double* v_out, xm_info* info) {
  if (!c || !q || !Y) return set_error(XM_EINVAL, "xm_certify: NULL argument");
  if (r < 1 || r > XM_MAX_RANK) return set_error(XM_EINVAL, "xm_certify: r=%d", r);
  xm_opts o;
  if (opts) o = *opts; else xm_default_opts(&o);
  o.r0 = r;
  o.r_max = r;
  XM_TRY(check_opts(q->d, o));
  XM_CUDA_TRY(cudaSetDevice(c->device));
  return solve_impl(c, q->d, o, r, Y, nullptr, nullptr, nullptr, nullptr, info, true, Lambda_out, v_out);
}

xm_status xm_pipeline_host(xm_ctx* c, int N, int M, int64_t E, const int32_t* cam_h,
                           const int32_t* lmk_h, const double* ukp_h, const double* w_h,
                           const xm_opts* opts, double* R_h, double* s_h, xm_info* info) {
  if (!c || !cam_h || !lmk_h || !ukp_h || !w_h || !R_h || !s_h || E < 0 || N < 1)
    return set_error(XM_EINVAL, "xm_pipeline_host: bad argument");
  xm_opts o;
  if (opts) o = *opts; else xm_default_opts(&o);
  XM_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  unsigned mask = XM_STORE_FP64;
  if (o.prec != XM_FP64) mask |= XM_STORE_FP32;
  if (o.prec == XM_BF16Q_BULK || (o.prec == XM_FP32_BULK && o.bf16_hvp_until > 0.0)) mask |= XM_STORE_BF16;
  int32_t *cam = nullptr, *lmk = nullptr;
  double *ukp = nullptr, *w = nullptr, *R = nullptr, *s = nullptr;
  auto cleanup = [&]() {
    if (cam) cudaFree(cam);
    if (lmk) cudaFree(lmk);
    if (ukp) cudaFree(ukp);
    if (w) cudaFree(w);
    if (R) cudaFree(R);
    if (s) cudaFree(s);
  };
  auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaSuccess;
  const size_t Ez = (size_t)(E > 0 ? E : 1);
  e = cudaMalloc(&cam, sizeof(int32_t) * Ez);
  if (e == cudaSuccess) e = cudaMalloc(&lmk, sizeof(int32_t) * Ez);
  if (e == cudaSuccess) e = cudaMalloc(&ukp, sizeof(double) * 3 * Ez);
  if (e == cudaSuccess) e = cudaMalloc(&w, sizeof(double) * Ez);
  if (e == cudaSuccess) e = cudaMalloc(&R, sizeof(double) * 9 * (size_t)N);
  if (e == cudaSuccess) e = cudaMalloc(&s, sizeof(double) * (size_t)N);
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(cam, cam_h, sizeof(int32_t) * E, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(lmk, lmk_h, sizeof(int32_t) * E, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(ukp, ukp_h, sizeof(double) * 3 * E, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && E > 0) e = cudaMemcpyAsync(w, w_h, sizeof(double) * E, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    cleanup();
    return set_error(e == cudaErrorMemoryAllocation ? XM_ENOMEM : XM_ECUDA, "xm_pipeline_host: %s",
                     cudaGetErrorString(e));
  }
  xm_qmat* q = nullptr;
  xm_status stt = xm_build_Q(c, N, M, E, cam, lmk, ukp, w, mask, &q);
  xm_info inf{};
  if (stt == XM_OK) {
    stt = xm_solve(c, q, &o, 0, nullptr, nullptr, R, s, nullptr, &inf);
    inf.t_build_s = q->t_build_s;
    if (stt == XM_OK || stt == XM_ENOTCERT) {
      cudaError_t e2 = cudaMemcpyAsync(R_h, R, sizeof(double) * 9 * N, cudaMemcpyDeviceToHost, st);
      if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(s_h, s, sizeof(double) * N, cudaMemcpyDeviceToHost, st);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
      if (e2 != cudaSuccess) stt = set_error(XM_ECUDA, "xm_pipeline_host: %s", cudaGetErrorString(e2));
    }
    xm_free_Q(c, q);
  }
  cleanup();
  inf.t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return stt;
}

}  // extern "C"
