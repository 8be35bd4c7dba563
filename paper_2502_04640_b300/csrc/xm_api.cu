// C ABI: context, error reporting and Q handles.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "xm_internal.cuh"

namespace xm {

static thread_local char g_err[1024] = "";
long g_last_launches = 0;
long g_last_sweeps = 0;

xm_status set_error(xm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

xm_status check_device_error(xm_ctx* ctx, const char* where) {
  XM_CUDA_TRY(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                              ctx->stream));
  XM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const int e = *ctx->h_err;
  if (e == 0) return XM_OK;
  XM_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  if (e & DEV_BAD_INDEX) return set_error(XM_EINVAL, "%s: observation index out of range", where);
  if (e & DEV_BAD_VALUE) return set_error(XM_EINVAL, "%s: weight <= 0 or non-finite input", where);
  if (e & DEV_TIMEOUT) return set_error(XM_ETIMEOUT, "%s: a bounded device wait gave up", where);
  if (e & DEV_NUMERIC) return set_error(XM_ENUMERIC, "%s: NaN/Inf produced", where);
  return set_error(XM_ECUDA, "%s: device error word %d", where, e);
}

xm_status ensure_partials(xm_ctx* ctx, size_t nd) {
  if (nd <= ctx->partials_cap) return XM_OK;
  if (ctx->d_partials) cudaFree(ctx->d_partials);
  ctx->d_partials = nullptr;
  ctx->partials_cap = 0;
  XM_CUDA_TRY(cudaMalloc(&ctx->d_partials, nd * sizeof(double)));
  ctx->partials_cap = nd;
  return XM_OK;
}

xm_status build_Q(xm_ctx* ctx, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                  const double* ukp, const double* w, unsigned mask, DeviceQ& out,
                  double* t_build);
xm_status alloc_tiles(xm_ctx* ctx, DeviceQ& q, int N, unsigned mask);
void free_tiles(DeviceQ& q);
xm_status pack_dense(xm_ctx* ctx, DeviceQ& q, const double* Qd);
xm_status unpack_dense(xm_ctx* ctx, const DeviceQ& q, double* Qd);

// Self-check of the bounded waits (xm_selftest_wait): thread 0 initialises an mbarrier for one
// arrival, optionally arrives on it, and waits for phase 0 with at most `polls` polls.  No copy
// or transaction count is attached to the barrier, so a wait that gives up leaves nothing in
// flight; the barrier is invalidated before the CTA exits.
static __global__ void k_selftest_wait(int* err, long long polls, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive(&bar);
    if (!mbar_wait(&bar, 0, polls)) atomicOr(err, DEV_TIMEOUT);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
  }
}

}  // namespace xm

using namespace xm;

extern "C" {

xm_status xm_selftest_wait(xm_ctx* c, long long polls, int arrive) {
  if (!c) return set_error(XM_EINVAL, "xm_selftest_wait: NULL context");
  if (polls < 1 || polls > WAIT_LIMIT)
    return set_error(XM_EINVAL, "xm_selftest_wait: polls=%lld not in [1, %lld]", polls, WAIT_LIMIT);
  XM_CUDA_TRY(cudaSetDevice(c->device));
  k_selftest_wait<<<1, 32, 0, c->stream>>>(c->d_err, polls, arrive ? 1 : 0);
  XM_CUDA_TRY(cudaGetLastError());
  return check_device_error(c, "xm_selftest_wait");
}

int xm_abi_version(void) { return XM_ABI_VERSION; }

const char* xm_last_error(void) { return xm::g_err; }

void xm_default_opts(xm_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->r0 = 4;
  o->r_max = XM_MAX_RANK;
  o->prec = XM_FP32_BULK;
  o->grad_tol_rel = 1e-11;
  o->bulk_tol_rel = 1e-9;
  o->cert_tau_rel = 1e-6;
  o->max_outer = 300;
  o->max_tcg = 200;
  o->max_polish = 20;
  o->lanczos_max = 800;
  o->lanczos_tol = 1e-8;
  o->time_limit_s = 0.0;
  o->seed = 12345;
  o->verbose = 0;
  o->init_jitter = 0.1;
  o->scale_reg = 0.0;
  o->precond = 2;
  o->bulk_stall = -1;
  o->cert_lobpcg = 1;
  o->bf16_hvp_until = 0.0;
}

xm_status xm_create(xm_ctx** out, int device, void* stream) {
  if (!out) return set_error(XM_EINVAL, "xm_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  XM_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev)
    return set_error(XM_EINVAL, "xm_create: device %d not in [0, %d)", device, ndev);
  XM_CUDA_TRY(cudaSetDevice(device));
  cudaDeviceProp prop;
  XM_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
  if (prop.major < 10)
    return set_error(XM_ECUDA, "xm_create: device %d (sm_%d%d) is not a Blackwell GPU", device,
                     prop.major, prop.minor);
  xm_ctx* c = new xm_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  c->num_sms = prop.multiProcessorCount;
  c->smem_optin = prop.sharedMemPerBlockOptin;
  cudaError_t e = cudaMalloc(&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_counter, 64 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_counter, 0, 64 * sizeof(unsigned));
  if (e != cudaSuccess) {
    xm_destroy(c);
    return set_error(XM_ECUDA, "xm_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return XM_OK;
}

void xm_destroy(xm_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->d_err) cudaFree(c->d_err);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->d_counter) cudaFree(c->d_counter);
  if (c->d_partials) cudaFree(c->d_partials);
  delete c;
}

xm_status xm_sync(xm_ctx* c) {
  if (!c) return set_error(XM_EINVAL, "xm_sync: NULL context");
  XM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return check_device_error(c, "xm_sync");
}

xm_status xm_build_Q(xm_ctx* c, int N, int M, int64_t E, const int32_t* cam, const int32_t* lmk,
                     const double* ukp, const double* w, unsigned mask, xm_qmat** out) {
  if (!c || !out) return set_error(XM_EINVAL, "xm_build_Q: NULL context or output");
  *out = nullptr;
  if (N < 1 || M < 0 || E < 0) return set_error(XM_EINVAL, "xm_build_Q: N=%d M=%d E=%lld", N, M, (long long)E);
  mask &= XM_STORE_ALL | XM_STORE_FACTORED;
  if (mask == 0) return set_error(XM_EINVAL, "xm_build_Q: empty store mask");
  if (E > 0 && (!cam || !lmk || !ukp || !w)) return set_error(XM_EINVAL, "xm_build_Q: NULL array");
  if ((int64_t)3 * N > (1 << 20)) return set_error(XM_EINVAL, "xm_build_Q: N=%d too large", N);
  XM_CUDA_TRY(cudaSetDevice(c->device));
  xm_qmat* q = new xm_qmat();
  xm_status st = build_Q(c, N, M, E, cam, lmk, ukp, w, mask, q->d, &q->t_build_s);
  if (st != XM_OK) {
    free_tiles(q->d);
    delete q;
    return st;
  }
  *out = q;
  return XM_OK;
}

xm_status xm_qmat_from_dense(xm_ctx* c, int N, const double* Q, unsigned mask, xm_qmat** out) {
  if (!c || !out || !Q || N < 1) return set_error(XM_EINVAL, "xm_qmat_from_dense: bad argument");
  if ((mask & XM_STORE_ALL) == 0) return set_error(XM_EINVAL, "xm_qmat_from_dense: empty mask");
  *out = nullptr;
  XM_CUDA_TRY(cudaSetDevice(c->device));
  xm_qmat* q = new xm_qmat();
  xm_status st = alloc_tiles(c, q->d, N, mask & XM_STORE_ALL);
  if (st == XM_OK) st = pack_dense(c, q->d, Q);
  if (st == XM_OK) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = set_error(XM_ECUDA, "xm_qmat_from_dense: %s", cudaGetErrorString(e));
  }
  if (st != XM_OK) {
    free_tiles(q->d);
    delete q;
    return st;
  }
  *out = q;
  return XM_OK;
}

xm_status xm_qmat_to_dense(xm_ctx* c, const xm_qmat* q, double* Q_out) {
  if (!c || !q || !Q_out) return set_error(XM_EINVAL, "xm_qmat_to_dense: bad argument");
  XM_CUDA_TRY(cudaSetDevice(c->device));
  XM_TRY(unpack_dense(c, q->d, Q_out));
  XM_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return XM_OK;
}

xm_status xm_qmat_dims(const xm_qmat* q, int* N, int* n, unsigned* mask) {
  if (!q) return set_error(XM_EINVAL, "xm_qmat_dims: NULL handle");
  if (N) *N = q->d.N;
  if (n) *n = q->d.n;
  if (mask) *mask = q->d.mask;
  return XM_OK;
}

xm_status xm_set_build_mode(xm_ctx* c, int mode) {
  if (!c) return set_error(XM_EINVAL, "xm_set_build_mode: NULL context");
  if (mode != XM_BUILD_AUTO && mode != XM_BUILD_FP64 && mode != XM_BUILD_SPLIT_BF16)
    return set_error(XM_EINVAL, "xm_set_build_mode: unknown mode %d", mode);
  c->build_mode = mode;
  return XM_OK;
}

xm_status xm_qmat_build_info(const xm_qmat* q, int* path, double* t_update_s) {
  if (!q) return set_error(XM_EINVAL, "xm_qmat_build_info: NULL handle");
  if (path) *path = q->d.build_path;
  if (t_update_s) *t_update_s = q->d.t_update_s;
  return XM_OK;
}

xm_status xm_free_Q(xm_ctx* c, xm_qmat* q) {
  if (!q) return XM_OK;
  if (c) {
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
  }
  free_tiles(q->d);
  delete q;
  return XM_OK;
}

}  // extern "C"
