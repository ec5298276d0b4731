// C-ABI of the X-engine (declared in include/xengine.h): plan objects,
// host-side argument checks, tensor-map encoding and kernel launches.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "xengine.h"
#include "xe_kernels.h"

namespace {

constexpr int kTcMaxLaunchNtime = 32768;   // exact-float32 bound of one tcgen05 launch
constexpr long long kMaxSamplesCI32 = 16777215;  // 128 * T < 2^31
constexpr long long kMaxSamplesCF32 = 131072;    // 128 * T <= 2^24
constexpr unsigned long long kWaitTimeoutNs = 2000000000ull;  // 2 s per device wait

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Looked up once per process; plans may be created from several threads.
EncodeTiledFn get_encode_fn() {
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

struct xe_plan {
  int device = 0;
  int N = 0, C = 0, max_ntime = 0;
  xe_operand op = XE_OPERAND_FP8_E4M3;
  xe_out out_type = XE_OUT_CI32;
  long long nbl = 0;            // baselines per channel
  long long n_pairs = 0;        // C * nbl complex values
  int32_t* d_acc = nullptr;     // [C][nbl][2]
  int* d_err = nullptr;         // device error word
  int2* d_split = nullptr;      // scratch of the time-sliced leftover units (tensor-core operands)
  int num_sms = 0;
  long long samples = 0;
  long long launches = 0;
  std::string last_error;
  // host end-to-end path (allocated on first use)
  uint8_t* d_stage = nullptr;
  size_t stage_bytes = 0;
  float* d_vis_f = nullptr;
  cudaStream_t s_copy = nullptr, s_comp = nullptr;
};

namespace {

xe_status cuda_fail(xe_plan* p, cudaError_t e, const char* what) {
  if (p) {
    p->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return XE_ERR_CUDA;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Encode the tensor map of one gulp slice: uint8 {N, C, T}, box
// {box_x inputs, 1 channel, box_t samples}, shared-memory swizzle of
// swizzle_bytes (128 or 64).
xe_status encode_gulp_map(xe_plan* p, const uint8_t* gulp, int T, unsigned box_x, unsigned box_t, int swizzle_bytes,
                          CUtensorMap* map) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc) {
    p->last_error = "cuTensorMapEncodeTiled entry point unavailable";
    return XE_ERR_CUDA;
  }
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(p->N), static_cast<cuuint64_t>(p->C),
                        static_cast<cuuint64_t>(T)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(p->N),
                           static_cast<cuuint64_t>(p->N) * static_cast<cuuint64_t>(p->C)};
  cuuint32_t box[3] = {box_x, 1, box_t};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(gulp), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[96];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (CUresult %d)", static_cast<int>(r));
    p->last_error = buf;
    return XE_ERR_CUDA;
  }
  return XE_OK;
}

}  // namespace

// Tiled uint8 tensor map of rank 3 or 4 (no interleave, OOB reads as zeros),
// shared with the beamformer.
bool xe::encode_tensor_u8(CUtensorMap* map, const void* base, int rank, const unsigned long long* dims,
                          const unsigned long long* strides, const unsigned* box, int swizzle_bytes) {
  EncodeTiledFn enc = get_encode_fn();
  if (!enc || rank < 1 || rank > 5) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], estr[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    estr[i] = 1;
    if (i + 1 < rank) st[i] = strides[i];
  }
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, static_cast<cuuint32_t>(rank), const_cast<void*>(base), d, st, bx,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// Enqueue the correlation of one gulp (already validated) on `stream` into
// the int32 accumulator `acc` ([C][N(N+1)/2][2]): the plan's own, or the
// caller's visibility buffer for a one-gulp integration.
xe_status enqueue_correlate(xe_plan* p, const uint8_t* d_gulp, int ntime, int accumulate,
                            cudaStream_t stream, int32_t* acc) {
  if (ntime == 0) {
    if (!accumulate) {
      cudaError_t e = cudaMemsetAsync(acc, 0, static_cast<size_t>(p->n_pairs) * 8, stream);
      if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemsetAsync");
    }
    return XE_OK;
  }
  const size_t row_bytes = static_cast<size_t>(p->C) * static_cast<size_t>(p->N);
  if (p->op == XE_OPERAND_INT32_CUDACORE) {
    cudaError_t e = xe::launch_xcorr_cudacore(d_gulp, ntime, p->C, p->N, acc, accumulate, p->d_err, stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudacore launch");
    ++p->launches;
    return XE_OK;
  }
  const int eb = (p->op == XE_OPERAND_FP8_E4M3) ? 1 : 2;
  const int nt = (p->N + 127) / 128;
  const unsigned rows = eb == 1 ? 128u : 64u;   // samples per pipeline stage (one TMA box)
  for (int t0 = 0; t0 < ntime; t0 += kTcMaxLaunchNtime) {
    const int T = (ntime - t0) < kTcMaxLaunchNtime ? (ntime - t0) : kTcMaxLaunchNtime;
    CUtensorMap map, map_j;
    const uint8_t* slice = d_gulp + static_cast<size_t>(t0) * row_bytes;
    xe_status st = encode_gulp_map(p, slice, T, 128, rows, 128, &map);       // I tiles
    if (st == XE_OK) st = encode_gulp_map(p, slice, T, 64, rows, 64, &map_j);  // half J tiles
    if (st != XE_OK) return st;
    xe::TcParams prm;
    prm.N = p->N;
    prm.C = p->C;
    prm.nt = nt;
    prm.units = 0;  // set by the launcher
    prm.nks = static_cast<int>((T + rows - 1) / rows * (rows / 32));   // whole stages of 32-sample steps
    prm.accumulate = (accumulate || t0 > 0) ? 1 : 0;
    prm.acc = acc;
    prm.err = p->d_err;
    prm.timeout_ns = kWaitTimeoutNs;
    prm.split_ws = p->d_split;
    prm.split_parts = 0;  // set by the launcher
    int kernels = 0;
    cudaError_t e = xe::launch_xcorr_pair(eb, &map, &map_j, prm, p->num_sms, stream, &kernels);
    p->launches += kernels;
    if (e != cudaSuccess) return cuda_fail(p, e, "tcgen05 launch");
  }
  return XE_OK;
}

long long integration_bound(const xe_plan* p) {
  return p->out_type == XE_OUT_CF32 ? kMaxSamplesCF32 : kMaxSamplesCI32;
}

// Common argument checks of the correlate calls.
xe_status check_correlate(xe_plan* p, const void* gulp, int ntime, int accumulate) {
  if (!p || ntime < 0 || (accumulate != 0 && accumulate != 1)) return XE_ERR_INVALID_ARG;
  if (!gulp && ntime > 0) return XE_ERR_INVALID_ARG;  // an empty gulp is never dereferenced
  if (ntime > p->max_ntime) return XE_ERR_SHAPE;
  const long long base = accumulate ? p->samples : 0;
  if (base + ntime > integration_bound(p)) return XE_ERR_ACCUM_BOUND;
  return XE_OK;
}

}  // namespace

extern "C" {

const char* xe_version(void) { return "xengine-b300 0.1 (sm_103a)"; }

const char* xe_status_string(xe_status s) {
  switch (s) {
    case XE_OK: return "ok";
    case XE_ERR_INVALID_ARG: return "invalid argument";
    case XE_ERR_ALIGNMENT: return "misaligned pointer or n_input not a multiple of 16";
    case XE_ERR_SHAPE: return "size exceeds the plan";
    case XE_ERR_ACCUM_BOUND: return "integration would exceed the exact-accumulation bound";
    case XE_ERR_NOMEM: return "device allocation failed";
    case XE_ERR_CUDA: return "CUDA error";
    case XE_ERR_DEVICE_UNSUPPORTED: return "device is not sm_103 (B300)";
    case XE_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    case XE_ERR_BUSY: return "resource busy";
    case XE_ERR_DEVICE_INDEX: return "device index outside its buffer (debug build)";
  }
  return "unknown status";
}

const char* xe_plan_last_error(xe_plan_t plan) { return plan ? plan->last_error.c_str() : ""; }

xe_status xe_plan_create(xe_plan_t* out, int n_input, int n_chan, int max_ntime, xe_operand op,
                         xe_out out_type) {
  if (!out) return XE_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_input < 16 || n_input > 8192 || n_chan < 1 || max_ntime < 1) return XE_ERR_INVALID_ARG;
  if (op != XE_OPERAND_FP8_E4M3 && op != XE_OPERAND_FP16 && op != XE_OPERAND_INT32_CUDACORE)
    return XE_ERR_INVALID_ARG;
  if (out_type != XE_OUT_CI32 && out_type != XE_OUT_CF32) return XE_ERR_INVALID_ARG;
  if (n_input % 16 != 0) return XE_ERR_ALIGNMENT;
  const long long nt = (n_input + 127) / 128;
  if (static_cast<long long>(n_chan) * nt * (nt + 1) / 2 > 0x7FFFFFFFLL) return XE_ERR_INVALID_ARG;
  if (static_cast<long long>(max_ntime) * n_chan * n_input > (1LL << 40)) return XE_ERR_INVALID_ARG;

  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return XE_ERR_CUDA;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return XE_ERR_CUDA;
  if (major != 10 || minor != 3) return XE_ERR_DEVICE_UNSUPPORTED;

  xe_plan* p = new (std::nothrow) xe_plan();
  if (!p) return XE_ERR_NOMEM;
  p->device = dev;
  p->N = n_input;
  p->C = n_chan;
  p->max_ntime = max_ntime;
  p->op = op;
  p->out_type = out_type;
  p->nbl = static_cast<long long>(n_input) * (n_input + 1) / 2;
  p->n_pairs = p->nbl * n_chan;
  p->num_sms = sms;
  if (cudaMalloc(&p->d_acc, static_cast<size_t>(p->n_pairs) * 8) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return XE_ERR_NOMEM;
  }
  if (cudaMalloc(&p->d_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->d_acc);
    delete p;
    return XE_ERR_NOMEM;
  }
  if (op != XE_OPERAND_INT32_CUDACORE &&
      cudaMalloc(&p->d_split, xe::split_workspace_bytes(p->num_sms)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p->d_acc);
    cudaFree(p->d_err);
    delete p;
    return XE_ERR_NOMEM;
  }
  cudaError_t e1 = cudaMemset(p->d_acc, 0, static_cast<size_t>(p->n_pairs) * 8);
  cudaError_t e2 = cudaMemset(p->d_err, 0, sizeof(int));
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    cudaFree(p->d_acc);
    cudaFree(p->d_err);
    if (p->d_split) cudaFree(p->d_split);
    delete p;
    return XE_ERR_CUDA;
  }
  *out = p;
  return XE_OK;
}

xe_status xe_plan_destroy(xe_plan_t p) {
  if (!p) return XE_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  cudaFree(p->d_acc);
  cudaFree(p->d_err);
  if (p->d_split) cudaFree(p->d_split);
  if (p->d_stage) cudaFree(p->d_stage);
  if (p->d_vis_f) cudaFree(p->d_vis_f);
  if (p->s_copy) cudaStreamDestroy(p->s_copy);
  if (p->s_comp) cudaStreamDestroy(p->s_comp);
  cudaSetDevice(cur);
  delete p;
  return XE_OK;
}

xe_status xe_unpack(xe_plan_t p, const uint8_t* d_packed, int8_t* d_ci8, int ntime, void* stream) {
  if (!p || !d_packed || !d_ci8 || ntime < 0) return XE_ERR_INVALID_ARG;
  if (ntime > p->max_ntime) return XE_ERR_SHAPE;
  if (!aligned16(d_packed) || !aligned16(d_ci8)) return XE_ERR_ALIGNMENT;
  const long long n = static_cast<long long>(ntime) * p->C * p->N;
  cudaError_t e = xe::launch_unpack(d_packed, d_ci8, n, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(p, e, "unpack launch");
  if (n > 0) ++p->launches;
  return XE_OK;
}

xe_status xe_correlate(xe_plan_t p, const uint8_t* d_gulp, int ntime, int accumulate, void* stream) {
  xe_status st = check_correlate(p, d_gulp, ntime, accumulate);
  if (st != XE_OK) return st;
  if (ntime > 0 && !aligned16(d_gulp)) return XE_ERR_ALIGNMENT;
  st = enqueue_correlate(p, d_gulp, ntime, accumulate, static_cast<cudaStream_t>(stream), p->d_acc);
  if (st != XE_OK) return st;
  p->samples = (accumulate ? p->samples : 0) + ntime;
  return XE_OK;
}

xe_status xe_correlate_batch(int n, const xe_plan_t* plans, const uint8_t* const* d_gulps, const int* ntime,
                             const int* accumulate, void* stream) {
  if (n < 1 || n > xe::kMaxBatch || !plans || !d_gulps || !ntime || !accumulate) return XE_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return XE_ERR_CUDA;
  for (int k = 0; k < n; ++k) {
    xe_plan* p = plans[k];
    if (!p || p->op != XE_OPERAND_FP8_E4M3 || p->device != dev) return XE_ERR_INVALID_ARG;
    for (int q = 0; q < k; ++q)
      if (plans[q] == p) return XE_ERR_INVALID_ARG;   // one plan, one accumulator: once per batch
    xe_status st = check_correlate(p, d_gulps[k], ntime[k], accumulate[k]);
    if (st != XE_OK) return st;
    if (ntime[k] > kTcMaxLaunchNtime) return XE_ERR_SHAPE;   // one launch per problem
    if (ntime[k] > 0 && !aligned16(d_gulps[k])) return XE_ERR_ALIGNMENT;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  xe::BatchProblem probs[xe::kMaxBatch];
  int m = 0, max_ctas = 0;
  for (int k = 0; k < n; ++k) {
    xe_plan* p = plans[k];
    if (ntime[k] == 0) {   // nothing to correlate: as xe_correlate does
      xe_status st = enqueue_correlate(p, d_gulps[k], 0, accumulate[k], s, p->d_acc);
      if (st != XE_OK) return st;
      continue;
    }
    xe::BatchProblem& b = probs[m++];
    xe_status st = encode_gulp_map(p, d_gulps[k], ntime[k], 128, 128, 128, &b.ti);
    if (st == XE_OK) st = encode_gulp_map(p, d_gulps[k], ntime[k], 64, 128, 64, &b.tj);
    if (st != XE_OK) return st;
    b.prm.N = p->N;
    b.prm.C = p->C;
    b.prm.nt = (p->N + 127) / 128;
    b.prm.units = 0;
    b.prm.nks = (ntime[k] + 127) / 128 * 4;   // whole stages of four 32-sample steps
    b.prm.accumulate = accumulate[k];
    b.prm.acc = p->d_acc;
    b.prm.err = p->d_err;
    b.prm.timeout_ns = kWaitTimeoutNs;
    b.prm.split_ws = nullptr;
    b.prm.split_parts = 0;
    max_ctas = p->num_sms;
  }
  if (m > 0) {
    int kernels = 0;
    cudaError_t e = xe::launch_xcorr_batch(probs, m, max_ctas, s, &kernels);
    if (e != cudaSuccess) return cuda_fail(plans[0], e, "batched tcgen05 launch");
  }
  for (int k = 0; k < n; ++k) {
    xe_plan* p = plans[k];
    p->samples = (accumulate[k] ? p->samples : 0) + ntime[k];
    if (ntime[k] > 0) ++p->launches;
  }
  return XE_OK;
}

xe_status xe_correlate_emit(xe_plan_t p, const uint8_t* d_gulp, int ntime, void* d_vis, void* stream) {
  if (!p || !d_vis) return XE_ERR_INVALID_ARG;
  if (p->out_type != XE_OUT_CI32) return XE_ERR_INVALID_ARG;
  if (ntime < 0 || ntime > p->max_ntime) return ntime < 0 ? XE_ERR_INVALID_ARG : XE_ERR_SHAPE;
  if (!d_gulp && ntime > 0) return XE_ERR_INVALID_ARG;
  if (ntime > integration_bound(p)) return XE_ERR_ACCUM_BOUND;
  if ((reinterpret_cast<uintptr_t>(d_vis) & 7u) != 0) return XE_ERR_ALIGNMENT;
  if (ntime > 0 && !aligned16(d_gulp)) return XE_ERR_ALIGNMENT;
  return enqueue_correlate(p, d_gulp, ntime, 0, static_cast<cudaStream_t>(stream), static_cast<int32_t*>(d_vis));
}

xe_status xe_integrate(xe_plan_t p, void* d_vis, void* stream) {
  if (!p || !d_vis) return XE_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_vis) & 7u) != 0) return XE_ERR_ALIGNMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (p->out_type == XE_OUT_CI32) {
    e = cudaMemcpyAsync(d_vis, p->d_acc, static_cast<size_t>(p->n_pairs) * 8, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemcpyAsync");
  } else {
    e = xe::launch_emit_cf32(p->d_acc, static_cast<float*>(d_vis), p->n_pairs, s);
    if (e != cudaSuccess) return cuda_fail(p, e, "emit launch");
    ++p->launches;
  }
  return XE_OK;
}

xe_status xe_reset(xe_plan_t p, void* stream) {
  if (!p) return XE_ERR_INVALID_ARG;
  cudaError_t e = cudaMemsetAsync(p->d_acc, 0, static_cast<size_t>(p->n_pairs) * 8,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemsetAsync");
  p->samples = 0;
  return XE_OK;
}

xe_status xe_samples_integrated(xe_plan_t p, long long* out) {
  if (!p || !out) return XE_ERR_INVALID_ARG;
  *out = p->samples;
  return XE_OK;
}

xe_status xe_plan_launch_count(xe_plan_t p, long long* out) {
  if (!p || !out) return XE_ERR_INVALID_ARG;
  *out = p->launches;
  return XE_OK;
}

xe_status xe_plan_check(xe_plan_t p) {
  if (!p) return XE_ERR_INVALID_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaDeviceSynchronize");
  int err = 0;
  e = cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemcpy");
  if (err != 0) {
    char buf[96];
    const bool index = (err & xe::kErrBounds) != 0;
    snprintf(buf, sizeof buf, index ? "device index check failed (code 0x%x)" : "device wait timed out (code 0x%x)",
             err);
    p->last_error = buf;
    cudaMemset(p->d_err, 0, sizeof(int));
    return index ? XE_ERR_DEVICE_INDEX : XE_ERR_TIMEOUT;
  }
  return XE_OK;
}

xe_status xe_correlate_host(xe_plan_t p, const uint8_t* h_gulp, int ntime, int accumulate, void* h_vis) {
  xe_status st = check_correlate(p, h_gulp, ntime, accumulate);
  if (st != XE_OK) return st;
  if (!h_vis) return XE_ERR_INVALID_ARG;
  const size_t row_bytes = static_cast<size_t>(p->C) * static_cast<size_t>(p->N);
  const size_t need = row_bytes * static_cast<size_t>(p->max_ntime);
  cudaError_t e;
  if (!p->s_copy) {
    if ((e = cudaStreamCreateWithFlags(&p->s_copy, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(p, e, "cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&p->s_comp, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(p, e, "cudaStreamCreate");
  }
  if (p->stage_bytes < need) {
    if (p->d_stage) cudaFree(p->d_stage);
    p->d_stage = nullptr;
    p->stage_bytes = 0;
    if (cudaMalloc(&p->d_stage, need) != cudaSuccess) {
      cudaGetLastError();
      return XE_ERR_NOMEM;
    }
    p->stage_bytes = need;
  }
  if (p->out_type == XE_OUT_CF32 && !p->d_vis_f) {
    if (cudaMalloc(&p->d_vis_f, static_cast<size_t>(p->n_pairs) * 8) != cudaSuccess) {
      cudaGetLastError();
      return XE_ERR_NOMEM;
    }
  }
  // Slices of the gulp: copy slice k+1 while slice k is correlated.
  const int slice = ntime <= 2048 ? (ntime > 0 ? ntime : 1) : 2048;
  const long long base = accumulate ? p->samples : 0;
  int k = 0;
  for (int t0 = 0; t0 < ntime; t0 += slice, ++k) {
    const int T = (ntime - t0) < slice ? (ntime - t0) : slice;
    const size_t off = static_cast<size_t>(t0) * row_bytes;
    e = cudaMemcpyAsync(p->d_stage + off, h_gulp + off, static_cast<size_t>(T) * row_bytes,
                        cudaMemcpyHostToDevice, p->s_copy);
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemcpyAsync H2D");
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(p, e, "cudaEventCreate");
    cudaEventRecord(ev, p->s_copy);
    cudaStreamWaitEvent(p->s_comp, ev, 0);
    cudaEventDestroy(ev);
    st = enqueue_correlate(p, p->d_stage + off, T, (accumulate || t0 > 0) ? 1 : 0, p->s_comp, p->d_acc);
    if (st != XE_OK) return st;
  }
  if (ntime == 0) {
    st = enqueue_correlate(p, p->d_stage, 0, accumulate, p->s_comp, p->d_acc);
    if (st != XE_OK) return st;
  }
  const size_t out_bytes = static_cast<size_t>(p->n_pairs) * 8;
  if (p->out_type == XE_OUT_CI32) {
    e = cudaMemcpyAsync(h_vis, p->d_acc, out_bytes, cudaMemcpyDeviceToHost, p->s_comp);
  } else {
    e = xe::launch_emit_cf32(p->d_acc, p->d_vis_f, p->n_pairs, p->s_comp);
    if (e == cudaSuccess) {
      ++p->launches;
      e = cudaMemcpyAsync(h_vis, p->d_vis_f, out_bytes, cudaMemcpyDeviceToHost, p->s_comp);
    }
  }
  if (e != cudaSuccess) return cuda_fail(p, e, "cudaMemcpyAsync D2H");
  if ((e = cudaStreamSynchronize(p->s_comp)) != cudaSuccess) return cuda_fail(p, e, "cudaStreamSynchronize");
  p->samples = base + ntime;
  return XE_OK;
}

}  // extern "C"
