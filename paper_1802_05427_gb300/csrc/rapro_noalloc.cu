// Allocation-free receive: rapro_receive_subframe_noalloc and rapro_noalloc_status.
//
// Some callers cannot allocate device memory at the moment they receive a subframe:
// real-time slot loops that must never wait on an allocator (the receiver has a fixed
// per-slot deadline and cudaMalloc may synchronise the device or take milliseconds),
// processes whose device memory is owned by another framework's pool, and deployments
// that forbid run-time allocation altogether.  For them this entry point needs no plan
// and allocates nothing: the channel-estimate scratch that rapro_receive_subframe keeps
// in its plan lives here in a fixed, file-scope device array instead, and the LMMSE
// weights travel in the kernel parameters.
//
// The array (kNoAllocScratchBytes) is part of the library's device image: every GPU that
// loads the library holds it until the process exits.  All calls share it and it keeps
// the last call's contents, so calls that overlap on the GPU (different streams, or
// different host threads on the same device) race on it.
#include <cmath>
#include <complex>
#include <mutex>

#include "rapro_internal.h"

namespace rapro {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;     // 32 MiB of channel estimate
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_h[kNoAllocScratchBytes / sizeof(float2)];
static __device__ __align__(256) int g_noalloc_status;

struct DeviceScratch {
  float2* h = nullptr;
  int* status = nullptr;
  cudaError_t err = cudaSuccess;
};
DeviceScratch g_scratch[kMaxDevices];
std::once_flag g_once[kMaxDevices];

// Once per device, with that device current: the device addresses of the arrays (their
// names are host-side stand-ins in host code) and the kernels' shared-memory limits.
const DeviceScratch& device_scratch(int dev) {
  std::call_once(g_once[dev], [dev] {
    DeviceScratch& s = g_scratch[dev];
    s.err = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.h), g_noalloc_h);
    if (s.err == cudaSuccess) s.err = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.status), g_noalloc_status);
    if (s.err == cudaSuccess) s.err = prepare_detect(dev);
    if (s.err == cudaSuccess) s.err = prepare_estimate(dev);
  });
  return g_scratch[dev];
}

// FP64 weights of one block of n <= LMMSE_SMALL_MAX subcarriers with the plan's builder,
// in stack storage, rounded to complex64.
bool small_weights(const rapro_params& p, int n, float2* w) {
  std::complex<double> work[weights_fp64_work(LMMSE_SMALL_MAX)];
  double wd[2 * LMMSE_SMALL_MAX * LMMSE_SMALL_MAX];
  if (!weights_fp64_into(p, n, work, wd)) return false;
  for (int e = 0; e < n * n; ++e) w[e] = make_float2(float(wd[2 * e]), float(wd[2 * e + 1]));
  return true;
}

rapro_status reject(rapro_status s, const char* msg) {
  set_error(msg);
  return s;
}

}  // namespace
}  // namespace rapro

using namespace rapro;

extern "C" rapro_status rapro_receive_subframe_noalloc(const rapro_params* p, const rapro_c32* y_pilot,
                                                       const rapro_c32* pilots, const rapro_c32* y_data,
                                                       rapro_c32* x_eq, uint8_t* labels, float* llr,
                                                       int32_t* info, rapro_stream stream) {
  rapro_status s = rapro_params_validate(p);
  if (s != RAPRO_OK) return s;
  if (!y_pilot || !pilots || !y_data || !x_eq)
    return reject(RAPRO_ERR_INVALID_ARG, "y_pilot, pilots, y_data and x_eq must not be NULL");
  if (p->pilot_layout != RAPRO_PILOT_ORTHOGONAL)
    return reject(RAPRO_ERR_UNSUPPORTED, "the allocation-free receive reads the orthogonal pilot layout only");
  if (half_precision(*p))
    return reject(RAPRO_ERR_UNSUPPORTED, "the allocation-free receive runs the FP32 path only (precision = FP32)");
  if (p->subblock > LMMSE_SMALL_MAX)
    return reject(RAPRO_ERR_UNSUPPORTED, "the allocation-free receive needs subblock <= 32");
  const int T = p->n_pilot_sym, D = p->n_sym / p->n_pilot_sym - 1;
  const size_t h_bytes = size_t(T) * p->K * p->M * p->n_sc * sizeof(float2);
  if (h_bytes > kNoAllocScratchBytes)
    return reject(RAPRO_ERR_INVALID_ARG,
                  "n_pilot_sym*K*M*n_sc*8 bytes exceeds the 32 MiB scratch of the allocation-free receive");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return reject(RAPRO_ERR_INVALID_ARG, "device index out of range");
  const DeviceScratch& ds = device_scratch(dev);
  if (ds.err != cudaSuccess) return cuda_fail(ds.err, "allocation-free receive set-up");

  const int B = p->subblock, tail = p->n_sc % p->subblock, nb = (p->n_sc + B - 1) / B;
  float2 w_main[LMMSE_SMALL_MAX * LMMSE_SMALL_MAX], w_tail[LMMSE_SMALL_MAX * LMMSE_SMALL_MAX];
  if (!small_weights(*p, B, w_main) || (tail && !small_weights(*p, tail, w_tail)))
    return reject(RAPRO_ERR_NOT_POSDEF, "R_b + sigma2 I is not positive definite in FP64");

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The status word only has to start at zero; the estimate is fully rewritten below.
  // The detector reads it on entry and leaves every output untouched if the estimator
  // recorded a timeout (its rows of the scratch would hold the previous call's estimate).
  if ((e = cudaMemsetAsync(ds.status, 0, sizeof(int), st)) != cudaSuccess)
    return cuda_fail(e, "clear status word");
  const float2* yp = reinterpret_cast<const float2*>(y_pilot);
  const float2* pil = reinterpret_cast<const float2*>(pilots);
  e = launch_ls_lmmse_small_raw(w_main, w_tail, B, tail, nb, T * p->K * p->M, p->M, p->n_sc, yp, pil,
                                ds.h, ds.status, st);
  if (e != cudaSuccess) return cuda_fail(e, "LS+LMMSE kernel launch");
  const DetTiles tiles = make_det_tiles(p->K, D);
  e = launch_detect_raw(tiles, T, p->K, p->M, p->n_sc, D, p->qam_bits, float(p->sigma2), ds.status, ds.h,
                        reinterpret_cast<const float2*>(y_data), reinterpret_cast<float2*>(x_eq), labels, llr,
                        info, st);
  if (e != cudaSuccess) return cuda_fail(e, "detection kernel launch");
  return RAPRO_OK;
}

extern "C" rapro_status rapro_noalloc_status(int reset, int* status_out, rapro_stream stream) {
  if (!status_out) return reject(RAPRO_ERR_INVALID_ARG, "status_out must not be NULL");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return reject(RAPRO_ERR_INVALID_ARG, "device index out of range");
  const DeviceScratch& ds = device_scratch(dev);
  if (ds.err != cudaSuccess) return cuda_fail(ds.err, "allocation-free receive set-up");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int v = 0;
  if ((e = cudaMemcpyAsync(&v, ds.status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "read status word");
  if (reset && (e = cudaMemsetAsync(ds.status, 0, sizeof(int), st)) != cudaSuccess)
    return cuda_fail(e, "clear status word");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  *status_out = v;
  return RAPRO_OK;
}
