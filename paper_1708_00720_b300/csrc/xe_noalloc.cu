// Allocation-free entry point: xe_correlate_noalloc (declared in include/xengine.h).
//
// Some callers cannot allocate device memory: a host framework that owns
// every device allocation through its own pool, or a real-time stream
// processor that reserves all of its memory at start-up and must not call
// cudaMalloc / cudaFree while observing (those calls can synchronise the
// device and stall the stream).  This entry point serves them.  It runs the
// same e4m3 tensor-core X-engine as xe_correlate, but its scratch memory (the
// int32 integration buffer and the device error word) lives in a file-scope
// __device__ array of fixed size, so it allocates nothing.
//
// The array is defined once in this library and every GPU that loads the
// library keeps it until the process exits.  All calls share it: a call
// overwrites the integration buffer before it adds to it, and calls whose GPU
// work overlaps (for example on two streams) race on it.  The error word is
// sticky: kernels OR their timeout codes into it and only
// xe_correlate_noalloc_check reads and clears it, so a timeout of any call
// since the last check is reported there.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "xengine.h"
#include "xe_kernels.h"

namespace {

// Largest output this entry point accepts: n_chan * n_input (n_input + 1) / 2
// complex visibilities (2^21 = 2,097,152; e.g. 512 inputs x 15 channels or
// 256 inputs x 63 channels).  The scratch holds them as int32 pairs (16 MiB)
// behind a 256-byte header whose first word is the device error word.
constexpr long long kMaxPairs = 1LL << 21;
constexpr size_t kHeaderBytes = 256;
constexpr size_t kScratchBytes = kHeaderBytes + static_cast<size_t>(kMaxPairs) * 8;
constexpr int kMaxDevices = 64;
constexpr int kLaunchNtime = 32768;                 // exact-float32 bound of one launch
constexpr long long kMaxSamplesCI32 = 16777215;
constexpr long long kMaxSamplesCF32 = 131072;
constexpr unsigned long long kWaitTimeoutNs = 2000000000ull;

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_xe_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.  The cache is not refreshed
// after cudaDeviceReset, which unloads the module: the entry points must not
// be used across a reset of the device.
xe_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return XE_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_xe_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return XE_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return XE_OK;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

}  // namespace

extern "C" XE_API xe_status xe_correlate_noalloc(const uint8_t* d_gulp, int ntime, int n_chan,
                                                 int n_input, xe_out out_type, void* d_vis,
                                                 void* stream) {
  // ---- argument checks (nothing is enqueued when one fails)
  if (!d_vis || ntime < 0 || n_chan < 1 || n_input < 16 || n_input > 8192) return XE_ERR_INVALID_ARG;
  if (out_type != XE_OUT_CI32 && out_type != XE_OUT_CF32) return XE_ERR_INVALID_ARG;
  if (!d_gulp && ntime > 0) return XE_ERR_INVALID_ARG;
  if (n_input % 16 != 0) return XE_ERR_ALIGNMENT;
  if ((ntime > 0 && (reinterpret_cast<uintptr_t>(d_gulp) & 15u) != 0) ||
      (reinterpret_cast<uintptr_t>(d_vis) & 7u) != 0)
    return XE_ERR_ALIGNMENT;
  const long long nbl = static_cast<long long>(n_input) * (n_input + 1) / 2;
  const long long pairs = nbl * n_chan;
  if (pairs > kMaxPairs) return XE_ERR_SHAPE;  // beyond the fixed scratch
  if (ntime > (out_type == XE_OUT_CF32 ? kMaxSamplesCF32 : kMaxSamplesCI32)) return XE_ERR_ACCUM_BOUND;
  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return XE_ERR_CUDA;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return XE_ERR_CUDA;
  if (major != 10 || minor != 3) return XE_ERR_DEVICE_UNSUPPORTED;

  void* scratch = nullptr;
  xe_status st = scratch_address(&scratch);
  if (st != XE_OK) return st;
  int* d_err = static_cast<int*>(scratch);
  int32_t* d_acc = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(scratch) + kHeaderBytes);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t out_bytes = static_cast<size_t>(pairs) * 8;

  // The error word is not cleared here: it collects the timeouts of every
  // call until xe_correlate_noalloc_check reads it.
  if (ntime == 0) return cudaMemsetAsync(d_vis, 0, out_bytes, s) == cudaSuccess ? XE_OK : XE_ERR_CUDA;

  EncodeTiledFn enc = encode_fn();
  if (!enc) return XE_ERR_CUDA;
  const size_t row_bytes = static_cast<size_t>(n_chan) * static_cast<size_t>(n_input);
  const int nt = (n_input + 127) / 128;
  for (int t0 = 0; t0 < ntime; t0 += kLaunchNtime) {
    const int T = (ntime - t0) < kLaunchNtime ? (ntime - t0) : kLaunchNtime;
    const uint8_t* slice = d_gulp + static_cast<size_t>(t0) * row_bytes;
    CUtensorMap map, map_j;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(n_input), static_cast<cuuint64_t>(n_chan),
                          static_cast<cuuint64_t>(T)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(n_input), static_cast<cuuint64_t>(row_bytes)};
    cuuint32_t box[3] = {128, 1, 128};       // I tiles, 128-byte swizzle
    cuuint32_t box_j[3] = {64, 1, 128};      // half J tiles, 64-byte swizzle
    cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(slice), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&map_j, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(slice), dims, strides, box_j, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return XE_ERR_CUDA;
    xe::TcParams prm;
    prm.N = n_input;
    prm.C = n_chan;
    prm.nt = nt;
    prm.units = 0;  // set by the launcher
    prm.nks = 4 * ((T + 127) / 128);
    prm.accumulate = t0 > 0 ? 1 : 0;  // the first launch overwrites the scratch accumulator
    prm.acc = d_acc;
    prm.err = d_err;
    prm.timeout_ns = kWaitTimeoutNs;
    prm.split_ws = nullptr;  // no scratch for time slices here: leftover units run whole
    prm.split_parts = 0;
    int kernels = 0;
    if (xe::launch_xcorr_pair(1, &map, &map_j, prm, sms, s, &kernels) != cudaSuccess) return XE_ERR_CUDA;
  }
  cudaError_t e = (out_type == XE_OUT_CI32)
                      ? cudaMemcpyAsync(d_vis, d_acc, out_bytes, cudaMemcpyDeviceToDevice, s)
                      : xe::launch_emit_cf32(d_acc, static_cast<float*>(d_vis), pairs, s);
  return e == cudaSuccess ? XE_OK : XE_ERR_CUDA;
}

extern "C" XE_API xe_status xe_correlate_noalloc_check(void* stream) {
  void* scratch = nullptr;
  xe_status st = scratch_address(&scratch);
  if (st != XE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return XE_ERR_CUDA;
  int err = 0;
  // a synchronous copy into this stack variable: the runtime stages it, this
  // library allocates nothing
  if (cudaMemcpy(&err, scratch, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return XE_ERR_CUDA;
  if (err == 0) return XE_OK;
  if (cudaMemset(scratch, 0, sizeof(int)) != cudaSuccess) return XE_ERR_CUDA;
  return (err & xe::kErrBounds) ? XE_ERR_DEVICE_INDEX : XE_ERR_TIMEOUT;
}
