// Internal interface between the C-ABI layer (xe_api.cu) and the kernels.
// Not installed; the public interface is include/xengine.h.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace xe {

// Parameters of one tcgen05 X-engine launch.
struct TcParams {
  int N;                  // inputs
  int C;                  // channels
  int nt;                 // 128-input tiles per side, ceil(N / 128)
  int units;              // channels x pair units (set by the launcher)
  int nks;                // 32-sample steps, whole pipeline stages, T <= 32768
  int accumulate;         // 1: add into acc; 0: overwrite
  int32_t* acc;           // [C][N (N + 1) / 2][2] int32 accumulator
  int* err;               // device error word (bit mask of timed-out waits)
  unsigned long long timeout_ns;  // bound on every device-side wait
  int2* split_ws;         // split_workspace_bytes(max_ctas) of scratch for time-sliced units, or nullptr
  int split_parts;        // parts per time-sliced leftover unit, 0: none (set by the launcher)
  long long acc_pairs;    // int2 elements of acc, C N (N + 1) / 2 (set by the launcher)
  long long ws_pairs;     // int2 elements of split_ws (set by the launcher)
};

// Error-word bit of the debug build (XE_DEBUG_CHECKS): a kernel computed a
// global index outside its buffer; the access was skipped.
constexpr int kErrBounds = 1 << 9;

// Scratch of the time-sliced leftover units of one launch on at most
// max_ctas CTAs: one slot per CTA pair, one 128 x 128 int2 tile per CTA.
inline size_t split_workspace_bytes(int max_ctas) {
  return static_cast<size_t>(max_ctas / 2) * 2 * 128 * 128 * sizeof(int2);
}

// Tensor-core X-engine on pairs of CTAs, operand width eb (1: e4m3, 2:
// float16).  Both maps view the gulp as uint8 {N, C, T}: tmap_i with box
// {128, 1, R} and the 128-byte swizzle, tmap_j with box {64, 1, R} and the
// 64-byte swizzle, R = 128 time rows for e4m3 and 64 for float16.
// prm.nks must be a multiple of 4 (e4m3) or 2 (float16) 32-sample steps;
// prm.units and prm.split_parts are set here; the grid is at most max_ctas
// CTAs (an even number).  With prm.split_ws, units left over after the last
// full round are cut along time over all clusters and summed by a second,
// small kernel; *kernels receives the number of kernels launched (1 or 2).
int tc8_smem_bytes(int eb);
cudaError_t launch_xcorr_pair(int eb, const CUtensorMap* tmap_i, const CUtensorMap* tmap_j, const TcParams& prm,
                              int max_ctas, cudaStream_t stream, int* kernels);

// Several independent problems (e.g. the gulps of several streams) in ONE
// launch of the e4m3 pair kernel: the grid runs the concatenation of their
// pair units.  Each problem has its own maps (as for launch_xcorr_pair), N,
// C, nks (one launch: T <= 32768), accumulate flag, accumulator and error
// word; split_ws must be nullptr (leftover units run whole).  At most
// kMaxBatch problems; *kernels = 1 on success.
constexpr int kMaxBatch = 8;
struct BatchProblem {
  CUtensorMap ti, tj;
  TcParams prm;
};
cudaError_t launch_xcorr_batch(const BatchProblem* probs, int n, int max_ctas, cudaStream_t stream,
                               int* kernels);

// Plain CUDA-core correlator (int8 dot products into int32), the baseline.
cudaError_t launch_xcorr_cudacore(const uint8_t* gulp, int T, int C, int N, int32_t* acc,
                                  int accumulate, int* err, cudaStream_t stream);

// Index check of a global access in the debug build (XE_DEBUG_CHECKS):
// element p of an n-element buffer at base.  Outside it, the check sets
// kErrBounds in *err and the caller skips the access; in the normal build
// it is always true and compiles away.
template <typename E>
__device__ __forceinline__ bool debug_in_bounds(const E* p, const E* base, long long n, int* err) {
#ifdef XE_DEBUG_CHECKS
  const long long i = p - base;
  if (i < 0 || i >= n) {
    atomicOr(err, kErrBounds);
    return false;
  }
#else
  (void)p; (void)base; (void)n; (void)err;
#endif
  return true;
}

// 4+4 -> 8+8 unpack of n packed samples (n % 16 == 0 not required).
cudaError_t launch_unpack(const uint8_t* packed, int8_t* out, long long n, cudaStream_t stream);

// Emit the int32 accumulator as float pairs (exact integers).
cudaError_t launch_emit_cf32(const int32_t* acc, float* out, long long n_pairs,
                             cudaStream_t stream);

// Gain calibration (xe_calib.cu): persistent grid size; scratch bytes for
// that grid; one pass (two launches) that computes chi^2 (if chisq !=
// nullptr, float64 out), the gradient (if grad != nullptr, scaled by *scale
// or 1), or both; and out = (*scale) * in.
int calib_grid_ctas(int N, int C);
size_t calib_scratch_bytes(int N, int C, int ctas);
cudaError_t launch_calib(const float* g, const float* model, const float* vobs, const float* w, int N, int C,
                         int ctas, int include_autos, void* scratch, double* chisq, const double* scale,
                         float* grad, cudaStream_t stream);
cudaError_t launch_calib_scale(const float* in, const double* scale, long long n, float* out, cudaStream_t stream);

// Tiled uint8 tensor map of the given rank (dims innermost first, strides in
// bytes of dims 1 .. rank-1), shared-memory swizzle of 0, 64 or 128 bytes,
// OOB reads as zeros; false if encoding failed.
bool encode_tensor_u8(CUtensorMap* map, const void* base, int rank, const unsigned long long* dims,
                      const unsigned long long* strides, const unsigned* box, int swizzle_bytes);

// Beamformer (xe_beam.cu).
struct BeamParams {
  int N, C, B;            // inputs, channels, beams
  int S;                  // 64-input stages, ceil(N / 64)
  int T;                  // samples in this launch
  int tiles;              // 128-sample time tiles, ceil(T / 128)
  const uint16_t* wt;     // [C][S][2][2B][64] float16 weights, K-major 128-byte-swizzled operand tiles
  const float* bias;      // [C][2B] 8 * (sum of each operand row)
  float* out;             // [T][C][B] complex64
  int* err;               // device error word
  unsigned long long timeout_ns;
  int map4;               // 1: the raw map is 4-D {64, T, S, C} (box {64, 128, 4, 1}); 0: 3-D {N, C, T}
                          // (box {64, 1, 128}); both with the 64-byte shared-memory swizzle
};
int beam_smem_bytes(int S, int B);
int beam_threads();
cudaError_t launch_beam(const CUtensorMap* tmap, const BeamParams& prm, int grid, cudaStream_t stream);
int beam_w_group(int B);   // stages of weights per bulk copy
cudaError_t launch_beam_weights(const float* w, int N, int C, int B, int S, uint16_t* wt, float* bias,
                                cudaStream_t stream);

// Beamformer for B <= 16 beams and N <= 512 inputs (xe_beam8.cu): operand
// A = the voltages as biased e4m3 bytes in tensor memory (a time sample per
// lane), operand B = the weights as four e4m3 terms per float16 coefficient,
// resident in shared memory per channel.  The raw map views the gulp as
// uint8 {N, C, T} with box {128, 1, 128} and the 128-byte swizzle.
struct Beam8Params {
  int N, C, B;            // inputs, channels, beams
  int S;                  // 128-input stages, ceil(N / 128) (<= 4)
  int T;                  // samples in this launch
  int tiles;              // 128-sample time tiles, ceil(T / 128)
  const uint8_t* wa;      // [C][S][re, im][128 rows][128 K bytes] e4m3 operand-B images as shared memory holds
                          // them (128-byte swizzle; row 4 o + k: term k of output o)
  const float* osc;       // [C] 2^9 / sigma_c
  const float* bias;      // [C][32] 8 * (sum of each output row's coefficients)
  float* out;             // [T][C][B] complex64
  int* err;               // device error word
  unsigned long long timeout_ns;
};
int beam8_smem_bytes();
cudaError_t launch_beam8(const CUtensorMap* tmap, const Beam8Params& prm, int grid, cudaStream_t stream);
// Weights [C][B][N] complex64 -> sigma [C], osc [C], bias [C][32] and the A images.
cudaError_t launch_beam8_weights(const float* w, int N, int C, int B, int S, uint8_t* wa, float* sigma, float* osc,
                                 float* bias, cudaStream_t stream);

}  // namespace xe
