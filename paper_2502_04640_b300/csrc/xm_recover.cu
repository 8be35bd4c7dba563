// Translations and landmarks of the rounded solution (Eq. 7) and the XM^2 re-run (Sec. 5).
//
// For fixed rotations and scales the SBA cost of Eq. 3 is a linear least-squares problem in
// (t, p) with t_0 = 0 (the anchor): with a_e = s_i R_i u_e, the landmark normal equations give
// p_k = (sum_e w_e (a_e + t_i)) / d_k, and eliminating them leaves Sbar tbar = -bbar on the
// anchored camera block (App. A), b_j = sum_{e: cam_e = j} w_e (a_e - m_k), m_k the weighted
// landmark mean of a.  All sums run in observation order (deterministic), in FP64.
//
// XM^2 drops the tenth of the measurements whose Eq. 3 terms w_e ||a_e + t_i - p_k||^2 are the
// largest (ties broken by the lower index) and solves again on the rest.  When the cut splits the
// view graph, the second solve runs on the component with the most cameras (ties: the one with
// the lowest camera index), anchored at its lowest-index camera; cameras and landmarks outside
// it are reported with zero rotation, scale, translation and position.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

#include "xm_internal.cuh"

namespace xm {

xm_status build_Q(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                  const double* ukp, const double* w, unsigned mask, DeviceQ& out, double* t_build);
void free_tiles(DeviceQ& q);
xm_status solve_impl(xm_ctx* ctx, const DeviceQ& q, const xm_opts& o, int r_in, const double* Y0,
                     double* Y_out, double* R_out, double* s_out, double* G_out, xm_info* out_info,
                     bool certify_only, double* Lambda_out, double* v_out);
xm_status check_opts(const DeviceQ& q, const xm_opts& o);

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

// a_e = s_i R_i u_e (R row-major 3 x 3)
__device__ __forceinline__ void transformed(const double* __restrict__ R, const double* __restrict__ s,
                                            int i, const double* __restrict__ u, double (&a)[3]) {
  const double* Ri = R + 9 * (size_t)i;
  const double si = s[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) a[c] = si * (Ri[3 * c] * u[0] + Ri[3 * c + 1] * u[1] + Ri[3 * c + 2] * u[2]);
}

// m_k = sum_{e in k} w_e a_e / d_k (0 for a landmark without observations)
__global__ void k_rec_lmk_mean(int M, const int64_t* __restrict__ loff, const int64_t* __restrict__ lidx,
                               const int32_t* __restrict__ cam, const double* __restrict__ ukp,
                               const double* __restrict__ w, const double* __restrict__ dk,
                               const double* __restrict__ R, const double* __restrict__ s,
                               double* __restrict__ m) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) {
      const int64_t e = lidx[x];
      double a[3];
      transformed(R, s, cam[e], ukp + 3 * e, a);
      for (int c = 0; c < 3; ++c) acc[c] += w[e] * a[c];
    }
    const double inv = dk[k] > 0.0 ? 1.0 / dk[k] : 0.0;
    for (int c = 0; c < 3; ++c) m[(size_t)3 * k + c] = acc[c] * inv;
  }
}

// b_j = sum_{e: cam_e = j} w_e (a_e - m_{k_e}), column-major N x 3
__global__ void k_rec_cam_sum(int N, const int64_t* __restrict__ coff, const int64_t* __restrict__ cidx,
                              const int32_t* __restrict__ lmk, const double* __restrict__ ukp,
                              const double* __restrict__ w, const double* __restrict__ R,
                              const double* __restrict__ s, const double* __restrict__ m,
                              double* __restrict__ b) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t x = coff[j]; x < coff[j + 1]; ++x) {
      const int64_t e = cidx[x];
      double a[3];
      transformed(R, s, j, ukp + 3 * e, a);
      const double* mk = m + (size_t)3 * lmk[e];
      for (int c = 0; c < 3; ++c) acc[c] += w[e] * (a[c] - mk[c]);
    }
    for (int c = 0; c < 3; ++c) b[(size_t)c * N + j] = acc[c];
  }
}

// p_k = m_k + sum_{e in k} w_e t_{i_e} / d_k; res2_e = w_e ||a_e + t_i - p_k||^2
__global__ void k_rec_out(int M, const int64_t* __restrict__ loff, const int64_t* __restrict__ lidx, int N,
                          const int32_t* __restrict__ cam, const double* __restrict__ ukp,
                          const double* __restrict__ w, const double* __restrict__ dk,
                          const double* __restrict__ R, const double* __restrict__ s,
                          const double* __restrict__ m, const double* __restrict__ t,
                          double* __restrict__ p_out, double* __restrict__ res2) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double pk[3] = {0.0, 0.0, 0.0};
    for (int64_t x = loff[k]; x < loff[k + 1]; ++x) {
      const int64_t e = lidx[x];
      const int i = cam[e];
      for (int c = 0; c < 3; ++c) pk[c] += w[e] * t[(size_t)c * N + i];
    }
    const bool seen = dk[k] > 0.0;
    const double inv = seen ? 1.0 / dk[k] : 0.0;
    for (int c = 0; c < 3; ++c) pk[c] = seen ? m[(size_t)3 * k + c] + pk[c] * inv : 0.0;
    if (p_out)
      for (int c = 0; c < 3; ++c) p_out[(size_t)3 * k + c] = pk[c];
    if (res2)
      for (int64_t x = loff[k]; x < loff[k + 1]; ++x) {
        const int64_t e = lidx[x];
        const int i = cam[e];
        double a[3];
        transformed(R, s, i, ukp + 3 * e, a);
        double q = 0.0;
        for (int c = 0; c < 3; ++c) {
          const double r = a[c] + t[(size_t)c * N + i] - pk[c];
          q += r * r;
        }
        res2[e] = w[e] * q;
      }
  }
}

__global__ void k_rec_t_rows(int N, const double* __restrict__ tcol, double* __restrict__ t_out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x)
    for (int c = 0; c < 3; ++c) t_out[(size_t)3 * j + c] = tcol[(size_t)c * N + j];
}

// out[j] = in[idx[j]] for the kept measurements
__global__ void k_gather_obs(int64_t Ek, const int64_t* __restrict__ idx, const int32_t* __restrict__ cam,
                             const int32_t* __restrict__ lmk, const double* __restrict__ ukp,
                             const double* __restrict__ w, int32_t* __restrict__ cam2,
                             int32_t* __restrict__ lmk2, double* __restrict__ ukp2, double* __restrict__ w2) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < Ek;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx[j];
    cam2[j] = cam[e];
    lmk2[j] = lmk[e];
    for (int c = 0; c < 3; ++c) ukp2[3 * j + c] = ukp[3 * e + c];
    w2[j] = w[e];
  }
}

// dst[map[j] * width + c] = src[j * width + c]: results of a re-indexed sub-problem written
// back to the rows of the full problem (the caller zeroes the rows nothing maps to)
__global__ void k_scatter_rows(int rows, int width, const int32_t* __restrict__ map,
                               const double* __restrict__ src, double* __restrict__ dst) {
  const int64_t total = (int64_t)rows * width;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = x / width;
    dst[(int64_t)map[j] * width + (x - j * width)] = src[x];
  }
}

// Connected components of the camera-landmark graph of the kept measurements (vertices: N
// cameras, then M landmarks), by union-find on the host.  in_comp[i] = 1 for the cameras of the
// component with the most cameras; ties go to the component of the lowest camera index.
static void largest_component(int N, int M, int64_t E, const std::vector<int32_t>& cam,
                              const std::vector<int32_t>& lmk, const std::vector<unsigned char>& keep,
                              std::vector<unsigned char>& in_comp) {
  std::vector<int> parent((size_t)N + M);
  std::iota(parent.begin(), parent.end(), 0);
  auto find = [&](int v) {
    while (parent[v] != v) { parent[v] = parent[parent[v]]; v = parent[v]; }
    return v;
  };
  for (int64_t e = 0; e < E; ++e) {
    if (!keep[e]) continue;
    const int a = find(cam[e]), b = find(N + lmk[e]);
    if (a != b) parent[std::max(a, b)] = std::min(a, b);
  }
  std::vector<int> count((size_t)N + M, 0);
  for (int i = 0; i < N; ++i) ++count[find(i)];
  const int most = *std::max_element(count.begin(), count.end());
  int best = -1;
  for (int i = 0; i < N && best < 0; ++i)
    if (count[find(i)] == most) best = find(i);
  in_comp.assign(N, 0);
  for (int i = 0; i < N; ++i) in_comp[i] = find(i) == best;
}

static xm_status recover_impl(xm_ctx* c, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                              const double* ukp, const double* w, const double* R, const double* s,
                              double* t_out, double* p_out, double* res2_out) {
  cudaStream_t st = c->stream;
  XM_TRY(validate_obs(c, N, M, E, cam, lmk, ukp, w));
  Buf loff, lidx, coff, cidx, S, dk, m, b;
  XM_CUDA_TRY(cudaMalloc(&loff.p, sizeof(int64_t) * ((size_t)M + 1)));
  XM_CUDA_TRY(cudaMalloc(&coff.p, sizeof(int64_t) * ((size_t)N + 1)));
  XM_CUDA_TRY(cudaMalloc(&lidx.p, sizeof(int64_t) * (size_t)std::max<int64_t>(E, 1)));
  XM_CUDA_TRY(cudaMalloc(&cidx.p, sizeof(int64_t) * (size_t)std::max<int64_t>(E, 1)));
  XM_CUDA_TRY(cudaMalloc(&S.p, sizeof(double) * (size_t)N * N));
  XM_CUDA_TRY(cudaMalloc(&dk.p, sizeof(double) * (size_t)std::max(M, 1)));
  XM_CUDA_TRY(cudaMalloc(&m.p, sizeof(double) * 3 * (size_t)std::max(M, 1)));
  XM_CUDA_TRY(cudaMalloc(&b.p, sizeof(double) * 3 * (size_t)N));
  XM_TRY(obs_csr(c, E, lmk, M, loff.as<int64_t>(), lidx.as<int64_t>()));
  XM_TRY(obs_csr(c, E, cam, N, coff.as<int64_t>(), cidx.as<int64_t>()));
  XM_TRY(schur_S_factor(c, N, M, cam, w, coff.as<int64_t>(), cidx.as<int64_t>(), loff.as<int64_t>(),
                        lidx.as<int64_t>(), S.as<double>(), dk.as<double>()));
  const int gl = grid_cap((size_t)std::max(M, 1), 128, c->num_sms * 4);
  k_rec_lmk_mean<<<gl, 128, 0, st>>>(M, loff.as<int64_t>(), lidx.as<int64_t>(), cam, ukp, w, dk.as<double>(),
                                     R, s, m.as<double>());
  k_rec_cam_sum<<<grid_cap((size_t)N, 64, c->num_sms * 4), 64, 0, st>>>(
      N, coff.as<int64_t>(), cidx.as<int64_t>(), lmk, ukp, w, R, s, m.as<double>(), b.as<double>());
  XM_CUDA_TRY(cudaGetLastError());
  XM_TRY(schur_S_solve(c, N, S.as<double>(), b.as<double>(), 3));
  k_rec_out<<<gl, 128, 0, st>>>(M, loff.as<int64_t>(), lidx.as<int64_t>(), N, cam, ukp, w, dk.as<double>(), R, s,
                                m.as<double>(), b.as<double>(), p_out, res2_out);
  if (t_out) k_rec_t_rows<<<grid_cap((size_t)N, 128, c->num_sms), 128, 0, st>>>(N, b.as<double>(), t_out);
  XM_CUDA_TRY(cudaGetLastError());
  XM_CUDA_TRY(cudaStreamSynchronize(st));
  return check_device_error(c, "xm_recover_tp");
}

}  // namespace xm

using namespace xm;

extern "C" xm_status xm_recover_tp(xm_ctx* c, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                                   const double* ukp, const double* w, const double* R, const double* s,
                                   double* t_out, double* p_out, double* res2_out) {
  if (!c || !R || !s) return set_error(XM_EINVAL, "xm_recover_tp: NULL argument");
  if (N < 1 || M < 0 || E < 0) return set_error(XM_EINVAL, "xm_recover_tp: bad sizes");
  if (E > 0 && (!cam || !lmk || !ukp || !w)) return set_error(XM_EINVAL, "xm_recover_tp: NULL observations");
  XM_CUDA_TRY(cudaSetDevice(c->device));
  return recover_impl(c, N, M, E, cam, lmk, ukp, w, R, s, t_out, p_out, res2_out);
}

extern "C" xm_status xm_solve_xm2(xm_ctx* c, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                                  const double* ukp, const double* w, const xm_opts* opts, double drop_frac,
                                  double* R_out, double* s_out, double* t_out, double* p_out,
                                  unsigned char* keep_out, xm_info* info_first, xm_info* info_second) {
  if (!c || !opts || !R_out || !s_out) return set_error(XM_EINVAL, "xm_solve_xm2: NULL argument");
  if (!(drop_frac >= 0.0 && drop_frac < 1.0)) return set_error(XM_EINVAL, "xm_solve_xm2: drop_frac not in [0, 1)");
  if (N < 1 || M < 0 || E < 1) return set_error(XM_EINVAL, "xm_solve_xm2: bad sizes");
  XM_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = c->stream;
  const unsigned mask = XM_STORE_FP64 | (opts->prec == XM_FP64 ? 0u : XM_STORE_FP32) |
                        (opts->prec == XM_BF16Q_BULK ? XM_STORE_BF16 : 0u);
  // ---- first solve
  Buf res2;
  XM_CUDA_TRY(cudaMalloc(&res2.p, sizeof(double) * (size_t)E));
  {
    DeviceQ q;
    xm_status sb = build_Q(c, N, M, E, cam, lmk, ukp, w, mask, q, nullptr);
    if (sb != XM_OK) { free_tiles(q); return sb; }
    xm_status so = check_opts(q, *opts);
    if (so != XM_OK) { free_tiles(q); return so; }
    xm_status s1 = solve_impl(c, q, *opts, 0, nullptr, nullptr, R_out, s_out, nullptr, info_first, false, nullptr,
                              nullptr);
    free_tiles(q);
    if (s1 != XM_OK && s1 != XM_ENOTCERT && s1 != XM_ENOCONV) return s1;
  }
  XM_TRY(recover_impl(c, N, M, E, cam, lmk, ukp, w, R_out, s_out, nullptr, nullptr, res2.as<double>()));
  // ---- keep rule: drop floor(drop_frac E) largest terms, ties by the lower index
  std::vector<double> h(E);
  XM_CUDA_TRY(cudaMemcpy(h.data(), res2.p, sizeof(double) * (size_t)E, cudaMemcpyDeviceToHost));
  const int64_t k = (int64_t)std::floor(drop_frac * (double)E);
  std::vector<unsigned char> keep(E, 1);
  if (k > 0) {
    std::vector<int64_t> order(E);
    std::iota(order.begin(), order.end(), int64_t(0));
    auto before = [&](int64_t a, int64_t b2) { return h[a] > h[b2] || (h[a] == h[b2] && a < b2); };
    std::nth_element(order.begin(), order.begin() + (k - 1), order.end(), before);
    for (int64_t j = 0; j < k; ++j) keep[order[j]] = 0;
  }
  // ---- the kept view graph may have split: solve on its largest component
  std::vector<int32_t> hc(E), hl(E);
  XM_CUDA_TRY(cudaMemcpy(hc.data(), cam, sizeof(int32_t) * (size_t)E, cudaMemcpyDeviceToHost));
  XM_CUDA_TRY(cudaMemcpy(hl.data(), lmk, sizeof(int32_t) * (size_t)E, cudaMemcpyDeviceToHost));
  std::vector<unsigned char> in_comp;
  largest_component(N, M, E, hc, hl, keep, in_comp);
  std::vector<int32_t> cmap(N, -1), cidx, lmap(M, -1), lidx;
  for (int i = 0; i < N; ++i)
    if (in_comp[i]) { cmap[i] = (int32_t)cidx.size(); cidx.push_back(i); }
  std::vector<int64_t> kept;
  kept.reserve(E - k);
  for (int64_t e = 0; e < E; ++e) {
    keep[e] = keep[e] && in_comp[hc[e]];
    if (!keep[e]) continue;
    kept.push_back(e);
    if (lmap[hl[e]] < 0) lmap[hl[e]] = 0;
  }
  for (int j = 0; j < M; ++j)
    if (lmap[j] >= 0) { lmap[j] = (int32_t)lidx.size(); lidx.push_back(j); }
  const bool split = (int)cidx.size() < N;
  const int N2 = (int)cidx.size(), M2 = split ? (int)lidx.size() : M;
  if (keep_out) XM_CUDA_TRY(cudaMemcpy(keep_out, keep.data(), (size_t)E, cudaMemcpyHostToDevice));
  const int64_t Ek = (int64_t)kept.size();
  // ---- second solve on the kept measurements (re-indexed when the graph split)
  Buf idx, cam2, lmk2, ukp2, w2;
  XM_CUDA_TRY(cudaMalloc(&idx.p, sizeof(int64_t) * (size_t)std::max<int64_t>(Ek, 1)));
  XM_CUDA_TRY(cudaMalloc(&cam2.p, sizeof(int32_t) * (size_t)std::max<int64_t>(Ek, 1)));
  XM_CUDA_TRY(cudaMalloc(&lmk2.p, sizeof(int32_t) * (size_t)std::max<int64_t>(Ek, 1)));
  XM_CUDA_TRY(cudaMalloc(&ukp2.p, sizeof(double) * 3 * (size_t)std::max<int64_t>(Ek, 1)));
  XM_CUDA_TRY(cudaMalloc(&w2.p, sizeof(double) * (size_t)std::max<int64_t>(Ek, 1)));
  XM_CUDA_TRY(cudaMemcpyAsync(idx.p, kept.data(), sizeof(int64_t) * (size_t)Ek, cudaMemcpyHostToDevice, st));
  k_gather_obs<<<grid_cap((size_t)std::max<int64_t>(Ek, 1), 256, c->num_sms), 256, 0, st>>>(
      Ek, idx.as<int64_t>(), cam, lmk, ukp, w, cam2.as<int32_t>(), lmk2.as<int32_t>(), ukp2.as<double>(),
      w2.as<double>());
  XM_CUDA_TRY(cudaGetLastError());
  Buf dcidx, dlidx, R2, s2b, t2, p2;
  if (split) {
    std::vector<int32_t> hc2(Ek), hl2(Ek);
    for (int64_t j = 0; j < Ek; ++j) { hc2[j] = cmap[hc[kept[j]]]; hl2[j] = lmap[hl[kept[j]]]; }
    XM_CUDA_TRY(cudaMemcpy(cam2.p, hc2.data(), sizeof(int32_t) * (size_t)Ek, cudaMemcpyHostToDevice));
    XM_CUDA_TRY(cudaMemcpy(lmk2.p, hl2.data(), sizeof(int32_t) * (size_t)Ek, cudaMemcpyHostToDevice));
    XM_CUDA_TRY(cudaMalloc(&dcidx.p, sizeof(int32_t) * (size_t)N2));
    XM_CUDA_TRY(cudaMalloc(&dlidx.p, sizeof(int32_t) * (size_t)std::max(M2, 1)));
    XM_CUDA_TRY(cudaMemcpy(dcidx.p, cidx.data(), sizeof(int32_t) * (size_t)N2, cudaMemcpyHostToDevice));
    XM_CUDA_TRY(cudaMemcpy(dlidx.p, lidx.data(), sizeof(int32_t) * (size_t)M2, cudaMemcpyHostToDevice));
    XM_CUDA_TRY(cudaMalloc(&R2.p, sizeof(double) * 9 * (size_t)N2));
    XM_CUDA_TRY(cudaMalloc(&s2b.p, sizeof(double) * (size_t)N2));
    XM_CUDA_TRY(cudaMalloc(&t2.p, sizeof(double) * 3 * (size_t)N2));
    XM_CUDA_TRY(cudaMalloc(&p2.p, sizeof(double) * 3 * (size_t)std::max(M2, 1)));
  }
  double* Rs = split ? R2.as<double>() : R_out;
  double* ss = split ? s2b.as<double>() : s_out;
  xm_status s2;
  {
    DeviceQ q;
    xm_status sb = build_Q(c, N2, M2, Ek, cam2.as<int32_t>(), lmk2.as<int32_t>(), ukp2.as<double>(),
                           w2.as<double>(), mask, q, nullptr);
    if (sb != XM_OK) { free_tiles(q); return sb; }
    s2 = solve_impl(c, q, *opts, 0, nullptr, nullptr, Rs, ss, nullptr, info_second, false, nullptr, nullptr);
    free_tiles(q);
    if (s2 != XM_OK && s2 != XM_ENOTCERT && s2 != XM_ENOCONV) return s2;
  }
  if (!split) {
    if (t_out || p_out)
      XM_TRY(recover_impl(c, N, M, Ek, cam2.as<int32_t>(), lmk2.as<int32_t>(), ukp2.as<double>(),
                          w2.as<double>(), R_out, s_out, t_out, p_out, nullptr));
  } else {
    const bool want_tp = t_out || p_out;
    if (want_tp)
      XM_TRY(recover_impl(c, N2, M2, Ek, cam2.as<int32_t>(), lmk2.as<int32_t>(), ukp2.as<double>(),
                          w2.as<double>(), Rs, ss, t2.as<double>(), p2.as<double>(), nullptr));
    // rows outside the solved component: zero rotation, scale, translation and position
    XM_CUDA_TRY(cudaMemsetAsync(R_out, 0, sizeof(double) * 9 * (size_t)N, st));
    XM_CUDA_TRY(cudaMemsetAsync(s_out, 0, sizeof(double) * (size_t)N, st));
    const int gsc = grid_cap((size_t)9 * N2, 256, c->num_sms);
    k_scatter_rows<<<gsc, 256, 0, st>>>(N2, 9, dcidx.as<int32_t>(), Rs, R_out);
    k_scatter_rows<<<gsc, 256, 0, st>>>(N2, 1, dcidx.as<int32_t>(), ss, s_out);
    if (t_out) {
      XM_CUDA_TRY(cudaMemsetAsync(t_out, 0, sizeof(double) * 3 * (size_t)N, st));
      k_scatter_rows<<<gsc, 256, 0, st>>>(N2, 3, dcidx.as<int32_t>(), t2.as<double>(), t_out);
    }
    if (p_out) {
      XM_CUDA_TRY(cudaMemsetAsync(p_out, 0, sizeof(double) * 3 * (size_t)M, st));
      if (M2 > 0)
        k_scatter_rows<<<grid_cap((size_t)3 * M2, 256, c->num_sms), 256, 0, st>>>(
            M2, 3, dlidx.as<int32_t>(), p2.as<double>(), p_out);
    }
    XM_CUDA_TRY(cudaGetLastError());
    XM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (s2 != XM_OK) return set_error(s2, "xm_solve_xm2: the second solve ended with status %d", (int)s2);
  return XM_OK;
}
