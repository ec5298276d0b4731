// Plain CUDA-core X-engine: the comparison baseline for the tensor-core path.
//
// Same result as the tcgen05 kernel (exact int32 visibilities, packed lower
// triangle), computed with int8 4-way dot products (dp4a) on the CUDA cores:
// two time samples of one input are packed as the int8 word
//   w(t) = [a(t), b(t), a(t+1), b(t+1)]
// and the rotated word of an I-side input as
//   r(t) = [b(t), -a(t), b(t+1), -a(t+1)],
// so that dp4a(w_i, w_j) adds a_i a_j + b_i b_j (Re) and dp4a(r_i, w_j) adds
// b_i a_j - a_i b_j (Im) over two samples.
//
// Tiling: one CTA of 128 threads per (channel, 64 x 64 input block pair
// I >= J); each thread owns 4 I rows x 8 J columns in registers (64 int32
// accumulators), so one pass over a time pair loads 16 words (four 128-bit
// shared-memory loads, one wavefront each) for 64 dp4a.  64-sample chunks
// are read with 128-bit global loads one chunk ahead and unpacked into
// shared memory rows padded to 68 words (conflict-free 128-bit stores).
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_kernels.h"

namespace xe {
namespace cc {

constexpr int kBlk = 64;       // inputs per block side
constexpr int kChunk = 64;     // time samples per chunk
constexpr int kPairs = kChunk / 2;
constexpr int kThreads = 128;
constexpr int kRow = kBlk + 4; // words per shared-memory row (one time pair)

__device__ __forceinline__ void tri_decode(int p, int& bi, int& bj) {
  int i = static_cast<int>((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  bi = i;
  bj = p - i * (i + 1) / 2;
}

// Sign-extend the eight nibbles of four packed samples into int8 lanes.
__device__ __forceinline__ uint32_t sext_hi(uint32_t w) {
  const uint32_t h = (w >> 4) & 0x0F0F0F0Fu;
  return h | ((h & 0x08080808u) * 0x1Eu);
}
__device__ __forceinline__ uint32_t sext_lo(uint32_t w) {
  const uint32_t l = w & 0x0F0F0F0Fu;
  return l | ((l & 0x08080808u) * 0x1Eu);
}

// Interleave the parts of four inputs at times t (A0 re, B0 im) and t + 1
// (A1, B1) into four words [A0_k, B0_k, A1_k, B1_k].
__device__ __forceinline__ void interleave(uint32_t A0, uint32_t B0, uint32_t A1, uint32_t B1,
                                           uint32_t* out) {
  const uint32_t p = __byte_perm(A0, B0, 0x5140), q = __byte_perm(A1, B1, 0x5140);
  const uint32_t p2 = __byte_perm(A0, B0, 0x7362), q2 = __byte_perm(A1, B1, 0x7362);
  out[0] = __byte_perm(p, q, 0x5410);
  out[1] = __byte_perm(p, q, 0x7632);
  out[2] = __byte_perm(p2, q2, 0x5410);
  out[3] = __byte_perm(p2, q2, 0x7632);
}

__global__ void __launch_bounds__(kThreads)
xcorr_cudacore_kernel(const uint8_t* __restrict__ x, int T, int C, int N,
                      int32_t* __restrict__ acc, int accumulate, int* err) {
  __shared__ __align__(16) uint32_t si[kPairs][kRow];   // I words
  __shared__ __align__(16) uint32_t sr[kPairs][kRow];   // I rotated words
  __shared__ __align__(16) uint32_t sj[kPairs][kRow];   // J words

  int bi, bj;
  tri_decode(blockIdx.x, bi, bj);
  const int tid = threadIdx.x;
  // unpack role: half the threads bring in I, half J; thread lt takes the
  // 16-input chunk lq of time pairs lp and lp + 16
  const bool jside = tid >= 64;
  const int lt = tid & 63;
  const int lp = lt >> 2;
  const int lq = lt & 3;
  const int in0 = (jside ? bj : bi) * kBlk + lq * 16;
  const bool in_ok = in0 < N;      // N % 16 == 0: a 16-input chunk is all in or all out
  // compute role: I rows 4 ti + a, J columns 4 tj + b and 32 + 4 tj + b
  const int ti = tid >> 3, tj = tid & 7;
  const long long nbl = static_cast<long long>(N) * (N + 1) / 2;

  for (int c = blockIdx.y; c < C; c += gridDim.y) {
    int re[4][8], im[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) re[a][b] = im[a][b] = 0;

    // samples t0 + 2 lp (+1) and t0 + 2 lp + 32 (+1) of this thread's chunk
    auto load = [&](int t0, uint4 (&v)[4]) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int t = t0 + 2 * lp + (k & 1) + (k >> 1) * kPairs;
        v[k] = make_uint4(0, 0, 0, 0);
        if (in_ok && t < T)
          v[k] = __ldg(reinterpret_cast<const uint4*>(x + (static_cast<size_t>(t) * C + c) * N + in0));
      }
    };

    uint4 v[4];
    load(0, v);
    for (int t0 = 0; t0 < T; t0 += kChunk) {
      // unpack the prefetched chunk into shared memory
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = lp + h * (kPairs / 2);
        const uint32_t w0[4] = {v[2 * h].x, v[2 * h].y, v[2 * h].z, v[2 * h].w};
        const uint32_t w1[4] = {v[2 * h + 1].x, v[2 * h + 1].y, v[2 * h + 1].z, v[2 * h + 1].w};
        uint32_t* dst = jside ? &sj[p][lq * 16] : &si[p][lq * 16];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t A0 = sext_hi(w0[k]), B0 = sext_lo(w0[k]);
          const uint32_t A1 = sext_hi(w1[k]), B1 = sext_lo(w1[k]);
          uint32_t o[4];
          interleave(A0, B0, A1, B1, o);
          *reinterpret_cast<uint4*>(dst + 4 * k) = make_uint4(o[0], o[1], o[2], o[3]);
          if (!jside) {
            uint32_t r[4];
            interleave(B0, __vsub4(0u, A0), B1, __vsub4(0u, A1), r);
            *reinterpret_cast<uint4*>(&sr[p][lq * 16 + 4 * k]) = make_uint4(r[0], r[1], r[2], r[3]);
          }
        }
      }
      __syncthreads();
      if (t0 + kChunk < T) load(t0 + kChunk, v);
#pragma unroll 2
      for (int p = 0; p < kPairs; ++p) {
        const uint4 wi = *reinterpret_cast<const uint4*>(&si[p][ti * 4]);
        const uint4 wr = *reinterpret_cast<const uint4*>(&sr[p][ti * 4]);
        const uint4 wj0 = *reinterpret_cast<const uint4*>(&sj[p][tj * 4]);
        const uint4 wj1 = *reinterpret_cast<const uint4*>(&sj[p][32 + tj * 4]);
        const int ai[4] = {static_cast<int>(wi.x), static_cast<int>(wi.y), static_cast<int>(wi.z),
                           static_cast<int>(wi.w)};
        const int ar[4] = {static_cast<int>(wr.x), static_cast<int>(wr.y), static_cast<int>(wr.z),
                           static_cast<int>(wr.w)};
        const int aj[8] = {static_cast<int>(wj0.x), static_cast<int>(wj0.y), static_cast<int>(wj0.z),
                           static_cast<int>(wj0.w), static_cast<int>(wj1.x), static_cast<int>(wj1.y),
                           static_cast<int>(wj1.z), static_cast<int>(wj1.w)};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            re[a][b] = __dp4a(ai[a], aj[b], re[a][b]);
            im[a][b] = __dp4a(ar[a], aj[b], im[a][b]);
          }
      }
      __syncthreads();
    }

    // write the lower-triangle part of this thread's 4 x 8 block
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int gi = bi * kBlk + ti * 4 + a;
      if (gi >= N) continue;
      int32_t* row = acc + 2 * (static_cast<long long>(c) * nbl + static_cast<long long>(gi) * (gi + 1) / 2);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int gj = bj * kBlk + (b >> 2) * 32 + tj * 4 + (b & 3);
        if (gj > gi) continue;
        int2* dst = reinterpret_cast<int2*>(row + 2 * gj);
        if (!debug_in_bounds(dst, reinterpret_cast<int2*>(acc), C * nbl, err)) continue;
        if (accumulate) {
          const int2 o = *dst;
          *dst = make_int2(o.x + re[a][b], o.y + im[a][b]);
        } else {
          *dst = make_int2(re[a][b], im[a][b]);
        }
      }
    }
  }
}

}  // namespace cc

cudaError_t launch_xcorr_cudacore(const uint8_t* gulp, int T, int C, int N, int32_t* acc,
                                  int accumulate, int* err, cudaStream_t stream) {
  const int nb = (N + cc::kBlk - 1) / cc::kBlk;
  const int npairs = nb * (nb + 1) / 2;
  dim3 grid(npairs, C < 65535 ? C : 65535);
  cc::xcorr_cudacore_kernel<<<grid, cc::kThreads, 0, stream>>>(gulp, T, C, N, acc, accumulate, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- unpack
// 4+4 -> 8+8: out[2k] = real, out[2k+1] = imaginary part of packed[k].
__global__ void unpack_kernel(const uint8_t* __restrict__ in, int8_t* __restrict__ out, long long n) {
  const long long nvec = n / 16;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long v = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; v < nvec; v += stride) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(in) + v);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    uint32_t o[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t A = cc::sext_hi(ws[k]), B = cc::sext_lo(ws[k]);
      o[2 * k] = __byte_perm(A, B, 0x5140);      // samples 0,1 of this word
      o[2 * k + 1] = __byte_perm(A, B, 0x7362);  // samples 2,3
    }
    uint4* dst = reinterpret_cast<uint4*>(out) + 2 * v;
    dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
    dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
  }
  // tail (n % 16 samples), one sample per thread
  for (long long k = nvec * 16 + blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < n; k += stride) {
    const int b = in[k];
    out[2 * k] = static_cast<int8_t>(static_cast<int8_t>(b & 0xF0) >> 4);
    out[2 * k + 1] = static_cast<int8_t>(static_cast<int8_t>((b & 0x0F) << 4) >> 4);
  }
}

// SMs of the current device (grids of the element-wise kernels are capped
// at a few waves of resident CTAs; grid-stride loops cover the rest).
static long long current_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 1;
  }
  return sms;
}

cudaError_t launch_unpack(const uint8_t* packed, int8_t* out, long long n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n / 16 + 255) / 256;
  if (blocks < 1) blocks = 1;
  const long long cap = current_sms() * 32;   // 8 resident 256-thread CTAs per SM, 4 waves
  if (blocks > cap) blocks = cap;
  unpack_kernel<<<static_cast<int>(blocks), 256, 0, stream>>>(packed, out, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ emit cf32
// One (re, im) pair per thread: the output only needs 8-byte alignment.
__global__ void emit_cf32_kernel(const int2* __restrict__ acc, float2* __restrict__ out, long long n_pairs) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < n_pairs; k += stride) {
    const int2 a = acc[k];
    out[k] = make_float2(static_cast<float>(a.x), static_cast<float>(a.y));
  }
}

cudaError_t launch_emit_cf32(const int32_t* acc, float* out, long long n_pairs, cudaStream_t stream) {
  if (n_pairs <= 0) return cudaSuccess;
  long long blocks = (n_pairs + 255) / 256;
  const long long cap = current_sms() * 16;
  if (blocks > cap) blocks = cap;
  emit_cf32_kernel<<<static_cast<int>(blocks), 256, 0, stream>>>(
      reinterpret_cast<const int2*>(acc), reinterpret_cast<float2*>(out), n_pairs);
  return cudaGetLastError();
}

}  // namespace xe
