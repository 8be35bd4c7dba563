// xm_qy_noalloc: the single-sweep entry point without any device allocation.
//
// xm_qy pads Y and W to the tile layout in buffers it allocates on every call.  Some callers
// cannot have a library allocate device memory: applications whose memory is entirely owned by
// their own pool allocator (a framework that reserved nearly all of HBM up front and accounts
// for every byte), and latency-bound loops in which the implicit synchronisation and
// unpredictable latency of an allocation are not acceptable.  This variant keeps the padded
// operands in one fixed, file-scope device array instead.
//
// The array lives on every GPU that loads this library until the process exits.  Its device
// address is looked up once per device, on the first call made on that device (with that
// device current); make that first call before any stream capture.  All calls share the array
// and it keeps the previous call's contents, so the padded W is cleared on every call; two
// calls whose work overlaps on the GPU (different streams or contexts) race on it.  The
// looked-up address is kept for the life of the process: after cudaDeviceReset on a device
// (which also invalidates every context, stream and Q handle made on it) this entry point must
// not be used on that device again.
#include <algorithm>
#include <mutex>

#include "xm_internal.cuh"

namespace xm {

// copy an n x rs row-major array into an n_rows x Rd padded one (zero fill)
template <typename T>
static __global__ void k_noalloc_repad(int n, int n_rows, const T* __restrict__ s, int rs,
                                       T* __restrict__ d, int Rd) {
  const size_t total = (size_t)n_rows * Rd;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / Rd), col = (int)(e % Rd);
    d[e] = (row < n && col < rs) ? s[(size_t)row * rs + col] : T(0);
  }
}

// 4 MiB: room for the padded Y and W of the 10155-camera workload in every precision up to
// r = 8 in FP64 (2 * 30592 * 8 * 8 bytes = 3.9 MB).
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[MAX_DEVICES] = {};
}  // namespace

// Device address of the scratch array on the current device (looked up once per device).
static xm_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= MAX_DEVICES)
    return set_error(XM_EINVAL, "xm_qy_noalloc: device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return set_error(XM_ECUDA, "xm_qy_noalloc: cudaGetSymbolAddress failed on device %d: %s",
                       device, cudaGetErrorString(e));
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return XM_OK;
}

template <typename T>
static xm_status qy_noalloc(xm_ctx* c, const DeviceQ& q, int prec, int r, const T* Y, T* W) {
  const int R = r == 1 ? 1 : (r <= 4 ? 4 : 8);
  const size_t bytes = sizeof(T) * (size_t)q.n_pad * R;   // one padded operand
  if (2 * bytes > NOALLOC_SCRATCH_BYTES)
    return set_error(XM_EINVAL,
                     "xm_qy_noalloc: padded Y and W need %zu bytes, above the fixed %zu-byte "
                     "scratch (n = %d, r = %d); use xm_qy",
                     2 * bytes, NOALLOC_SCRATCH_BYTES, q.n, r);
  void* base = nullptr;
  XM_TRY(noalloc_scratch(c->device, &base));
  T* Yp = static_cast<T*>(base);
  T* Wp = reinterpret_cast<T*>(static_cast<unsigned char*>(base) + ((bytes + 255) & ~size_t(255)));
  cudaStream_t st = c->stream;
  const int g = (int)std::min<size_t>(((size_t)q.n_pad * R + 255) / 256, (size_t)c->num_sms * 8);
  k_noalloc_repad<T><<<g, 256, 0, st>>>(q.n, q.n_pad, Y, r, Yp, R);   // writes every padded element
  XM_CUDA_TRY(cudaMemsetAsync(Wp, 0, bytes, st));                // the sweep accumulates into W
  XM_TRY(qy_launch(c, q, prec, R, Yp, Wp, nullptr, st));
  const int g2 = (int)std::min<size_t>(((size_t)q.n * r + 255) / 256, (size_t)c->num_sms * 8);
  k_noalloc_repad<T><<<g2 > 0 ? g2 : 1, 256, 0, st>>>(q.n, q.n, Wp, R, W, r);
  XM_CUDA_TRY(cudaGetLastError());
  return XM_OK;
}

}  // namespace xm

using namespace xm;

extern "C" xm_status xm_qy_noalloc(xm_ctx* c, const xm_qmat* q, int prec, int r, const void* Y,
                                   void* W) {
  if (!c || !q || !Y || !W) return set_error(XM_EINVAL, "xm_qy_noalloc: NULL argument");
  if (r < 1 || r > XM_MAX_RANK)
    return set_error(XM_EINVAL, "xm_qy_noalloc: r=%d not in [1, %d]", r, XM_MAX_RANK);
  XM_CUDA_TRY(cudaSetDevice(c->device));
  if (prec == XM_FP64) return qy_noalloc<double>(c, q->d, prec, r, (const double*)Y, (double*)W);
  return qy_noalloc<float>(c, q->d, prec, r, (const float*)Y, (float*)W);
}
