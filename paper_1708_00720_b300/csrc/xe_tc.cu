// tcgen05 X-engine: per-channel Hermitian correlation of 4+4-bit complex
// voltages on the fifth-generation tensor cores (sm_103a).
//
// What it computes (the linear-algebra module of the paper's section "Back
// end" applied to the samples of section "Packet capture implementation"):
//   V_c[i][j] = sum_t x[t][c][i] conj(x[t][c][j]),  i >= j,
// accumulated into an int32 buffer laid out [C][N(N+1)/2][2] (packed lower
// triangle, row-major, (re, im) pairs).
//
// Formulation.  With x = a + ib, Re V = sum(a_i a_j + b_i b_j) and
// Im V = sum(b_i a_j - a_i b_j).  Each 32-sample step of a 128 x 128 tile
// pair (I, J) issues four MMAs over planar operands (re and im planes of the
// I and J tiles, time along K):
//   D_re += A_re(I) B_re(J)^T + A_im(I) B_im(J)^T
//   D_im += A_im(I) B_re(J)^T - A_re(I) B_im(J)^T     (negate-B bit)
//
// Operand encoding ("biased subnormal").  A signed nibble v in [-8, 7] is
// stored as the byte u = v + 8 = nibble XOR 8 (one lop3 per 4 samples).  As
// an e4m3 bit pattern 0x00..0x0F is exactly u * 2^-9 (subnormals and the
// first binade are evenly spaced), and as an f16 bit pattern it is u * 2^-24,
// so every product is an exact integer multiple of 2^-18 (e4m3) or 2^-48
// (f16).  The bias is removed exactly in the epilogue from per-input sums of
// u kept by the unpack warps:
//   Re V = D_re - 8 (P_i + Q_i + P_j + Q_j) + 128 T'
//   Im V = D_im + 8 (P_i - Q_i) - 8 (P_j - Q_j)
// where P, Q are the sums of the biased real / imaginary parts and T' the
// number of processed samples (the time tail is zero-filled by TMA; a zero
// byte is a zero sample and enters D, P, Q and T' consistently).
//
// Exactness.  Every partial sum of D_re is at most 2 * 15 * 15 = 450 units per
// sample in magnitude, so it is an exact float32 integer while 450 T' <= 2^24,
// i.e. T' <= 37282 samples; the host splits longer gulps into launches of at
// most 32768 samples that add into the int32 accumulator.
//
// Data path per CTA (one persistent CTA per SM, 512 threads):
//   warp 0       TMA producer: raw 32 x 128-byte time x input tiles -> smem
//   warp 1       MMA issuer (one thread): 4 tcgen05.mma per step
//   warps 4..11  unpack, two groups of four warps taking alternate steps:
//                raw tile -> biased operand planes (MN-major, 128-byte
//                swizzle) + per-input sums
//   warps 12..15 epilogue: tcgen05.ld of D, bias removal, staging through
//                shared memory, coalesced int32 accumulate
// Accumulators are double-buffered in TMEM (2 x 256 columns) so a unit's
// epilogue overlaps the next unit's MMAs.  All waits are bounded; on timeout
// the kernel records an error code and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_kernels.h"
#include "xe_ptx.cuh"

namespace xe {
namespace tc {

constexpr int kTile = 128;           // inputs per tile side (MMA M and N)
constexpr int kStep = 32;            // time samples per pipeline step
constexpr int kRawTile = kStep * kTile;  // 4096 bytes of raw samples
#ifndef XE_TC_UNPACK_GROUPS
#define XE_TC_UNPACK_GROUPS 2
#endif
// Unpack warps form groups of four; group g converts the 32-sample steps
// whose index is g modulo the number of groups, so consecutive steps are
// unpacked concurrently.
constexpr int kUnpackGroups = XE_TC_UNPACK_GROUPS;
constexpr int kUnpackWarp0 = 4;
constexpr int kUnpackWarps = 4 * kUnpackGroups;
constexpr int kEpiWarp0 = kUnpackWarp0 + kUnpackWarps;  // a multiple of 4: one warp per TMEM lane quadrant
constexpr int kEpiThreads = 128;
constexpr int kThreads = 32 * (kEpiWarp0 + 4);
constexpr int kEpiStagePitch = 33;  // int2 per staged row (32 + 1 pad)
constexpr int kTmemCols = 512;       // 2 accumulator stages x (128 re + 128 im)

#ifndef XE_TC_RAW_STAGES_F8
#define XE_TC_RAW_STAGES_F8 12
#endif
#ifndef XE_TC_OP_STAGES_F8
#define XE_TC_OP_STAGES_F8 4
#endif

template <int EB>  // operand bytes per element: 1 = e4m3, 2 = f16
struct Cfg {
  // Raw tiles in flight cover the L2/HBM latency of the TMA loads; operand
  // stages decouple the unpack warps from the tensor pipe.
  static constexpr int kRawStages = EB == 1 ? XE_TC_RAW_STAGES_F8 : 8;
  static constexpr int kOpStages = EB == 1 ? XE_TC_OP_STAGES_F8 : 3;
  static constexpr int kPlane = kStep * kTile * EB;   // one re or im plane of one tile
  static constexpr int kOpStage = 4 * kPlane;         // I re, I im, J re, J im
  static constexpr int kRawStage = 2 * kRawTile;      // I raw, J raw
  static constexpr int kOpBytes = kOpStages * kOpStage;
  static constexpr int kRawBytes = kRawStages * kRawStage;
  static constexpr int kSumsBytes = 2 * 4 * kTile * 4;  // 2 stages x {P_I,Q_I,P_J,Q_J}[128] int
  static constexpr int kEpiBytes = 4 * 32 * kEpiStagePitch * 8;  // per-warp 32 x 32 int2 staging
  static constexpr int kBarOffset = kOpBytes + kRawBytes + kSumsBytes + kEpiBytes;
  static constexpr int kNumBars = 2 * kRawStages + 2 * kOpStages + 2 + 2 + 2 + 2 + 1;
  static_assert(kBarOffset + kNumBars * 8 + 16 + 1024 <= 227 * 1024, "shared memory budget");
  static constexpr int kSmemBytes = kBarOffset + kNumBars * 8 + 16 + 1024;  // + align slack
};

enum ErrCode : int {
  kErrWaitRawFull = 1 << 0,
  kErrWaitRawEmpty = 1 << 1,
  kErrWaitOpFull = 1 << 2,
  kErrWaitOpEmpty = 1 << 3,
  kErrWaitAccFull = 1 << 4,
  kErrWaitAccEmpty = 1 << 5,
  kErrWaitSumsFull = 1 << 6,
  kErrWaitSumsEmpty = 1 << 7,
  kErrWaitFinal = 1 << 8,
};

struct SmemPtrs {
  uint8_t* op;        // [Cfg::kOpStages][4][kPlane]
  uint8_t* raw;       // [Cfg::kRawStages][2][kRawTile]
  int* sums;          // [2][4][kTile]
  int2* epi;          // [4 warps][32][kEpiStagePitch]
  uint64_t* raw_full; uint64_t* raw_empty;
  uint64_t* op_full;  uint64_t* op_empty;
  uint64_t* acc_full; uint64_t* acc_empty;
  uint64_t* sums_full; uint64_t* sums_empty;
  uint64_t* final_bar;
  uint32_t* tmem_slot;
  int* abort_flag;
};

template <int EB>
__device__ __forceinline__ SmemPtrs carve(uint8_t* base) {
  using C = Cfg<EB>;
  SmemPtrs p;
  p.op = base;
  p.raw = base + C::kOpBytes;
  p.sums = reinterpret_cast<int*>(base + C::kOpBytes + C::kRawBytes);
  p.epi = reinterpret_cast<int2*>(base + C::kOpBytes + C::kRawBytes + C::kSumsBytes);
  uint64_t* b = reinterpret_cast<uint64_t*>(base + C::kBarOffset);
  p.raw_full = b; b += C::kRawStages;
  p.raw_empty = b; b += C::kRawStages;
  p.op_full = b; b += C::kOpStages;
  p.op_empty = b; b += C::kOpStages;
  p.acc_full = b; b += 2;
  p.acc_empty = b; b += 2;
  p.sums_full = b; b += 2;
  p.sums_empty = b; b += 2;
  p.final_bar = b; b += 1;
  p.tmem_slot = reinterpret_cast<uint32_t*>(b);
  p.abort_flag = reinterpret_cast<int*>(b) + 1;
  return p;
}

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                              volatile int* abort_flag) {
  const uint32_t a = smem_u32(bar);
  if (mbar_try_wait(a, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait(a, parity)) return true;
    if (*abort_flag) return false;
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void fail(const SmemPtrs& s, int* err, int code) {
  atomicExch(s.abort_flag, 1);
  atomicOr(err, code);
}

// Unit u -> (channel, I tile, J tile) with I >= J, row-major over the tile triangle.
__device__ __forceinline__ void decode_unit(int u, int npairs, int& c, int& bi, int& bj) {
  c = u / npairs;
  int p = u - c * npairs;
  int i = static_cast<int>((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  bi = i;
  bj = p - i * (i + 1) / 2;
}

__device__ __forceinline__ uint4 lds128(const void* p) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void sts128(void* p, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};"
               ::"r"(smem_u32(p)), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// Biased parts of four packed samples: byte k of the result is
// (nibble XOR 8) of sample k, i.e. v + 8 in 0..15.
__device__ __forceinline__ uint32_t biased_re(uint32_t w) {
  return ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
}
__device__ __forceinline__ uint32_t biased_im(uint32_t w) {
  return (w & 0x0F0F0F0Fu) ^ 0x08080808u;
}

// Byte offset, inside one operand plane, of the 16-byte chunk holding inputs
// [16 q, 16 q + 16) (e4m3) or [8 q, 8 q + 8) (f16) at time row k.  Layout:
// MN-major, 128-byte swizzle: [col block of 128 bytes][32 rows][128 bytes],
// the 16-byte chunk index XOR-ed with (row mod 8).
template <int EB>
__device__ __forceinline__ uint32_t plane_chunk_offset(int k, int q) {
  const int blk = q >> 3, ch = q & 7;
  return static_cast<uint32_t>(blk * (kStep * 128) + k * 128 + ((ch ^ (k & 7)) << 4));
}

struct UnpackSums {
  uint32_t b_re[4], b_im[4];    // byte lanes: 16 inputs, <= 17 rows before overflow
  uint32_t h_re[8], h_im[8];    // 16-bit lanes: pairs of inputs (k, k+2) per word
  __device__ __forceinline__ void zero_bytes() {
#pragma unroll
    for (int k = 0; k < 4; ++k) b_re[k] = b_im[k] = 0u;
  }
  __device__ __forceinline__ void zero() {
    zero_bytes();
#pragma unroll
    for (int k = 0; k < 8; ++k) h_re[k] = h_im[k] = 0u;
  }
  __device__ __forceinline__ void add(const uint4& re, const uint4& im) {
    b_re[0] += re.x; b_re[1] += re.y; b_re[2] += re.z; b_re[3] += re.w;
    b_im[0] += im.x; b_im[1] += im.y; b_im[2] += im.z; b_im[3] += im.w;
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h_re[2 * k] += b_re[k] & 0x00FF00FFu;
      h_re[2 * k + 1] += (b_re[k] >> 8) & 0x00FF00FFu;
      h_im[2 * k] += b_im[k] & 0x00FF00FFu;
      h_im[2 * k + 1] += (b_im[k] >> 8) & 0x00FF00FFu;
    }
    zero_bytes();
  }
  // Add this thread's partial sums for inputs [16 q, 16 q + 16) into P[], Q[].
  __device__ __forceinline__ void publish(int* P, int* Q, int q) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // word k holds inputs 4k..4k+3 as bytes 0..3; h[2k] = (byte0, byte2), h[2k+1] = (byte1, byte3)
      const int i0 = 16 * q + 4 * k;
      atomicAdd(&P[i0 + 0], static_cast<int>(h_re[2 * k] & 0xFFFFu));
      atomicAdd(&P[i0 + 2], static_cast<int>(h_re[2 * k] >> 16));
      atomicAdd(&P[i0 + 1], static_cast<int>(h_re[2 * k + 1] & 0xFFFFu));
      atomicAdd(&P[i0 + 3], static_cast<int>(h_re[2 * k + 1] >> 16));
      atomicAdd(&Q[i0 + 0], static_cast<int>(h_im[2 * k] & 0xFFFFu));
      atomicAdd(&Q[i0 + 2], static_cast<int>(h_im[2 * k] >> 16));
      atomicAdd(&Q[i0 + 1], static_cast<int>(h_im[2 * k + 1] & 0xFFFFu));
      atomicAdd(&Q[i0 + 3], static_cast<int>(h_im[2 * k + 1] >> 16));
    }
  }
};

// Unpack one raw 16-byte chunk (16 inputs at one time row) into the re / im
// operand planes and the running sums.
template <int EB>
__device__ __forceinline__ void unpack_chunk(const uint8_t* raw_tile, uint8_t* plane_re,
                                             uint8_t* plane_im, int row, int q, UnpackSums& sums) {
  const uint4 w = lds128(raw_tile + row * 128 + q * 16);
  uint4 re, im;
  re.x = biased_re(w.x); re.y = biased_re(w.y); re.z = biased_re(w.z); re.w = biased_re(w.w);
  im.x = biased_im(w.x); im.y = biased_im(w.y); im.z = biased_im(w.z); im.w = biased_im(w.w);
  sums.add(re, im);
  if constexpr (EB == 1) {
    const uint32_t off = plane_chunk_offset<1>(row, q);
    sts128(plane_re + off, re);
    sts128(plane_im + off, im);
  } else {
    // f16: each byte u becomes the 16-bit pattern u (a subnormal, u * 2^-24)
    uint4 r0, r1, i0, i1;
    r0.x = __byte_perm(re.x, 0u, 0x4140); r0.y = __byte_perm(re.x, 0u, 0x4342);
    r0.z = __byte_perm(re.y, 0u, 0x4140); r0.w = __byte_perm(re.y, 0u, 0x4342);
    r1.x = __byte_perm(re.z, 0u, 0x4140); r1.y = __byte_perm(re.z, 0u, 0x4342);
    r1.z = __byte_perm(re.w, 0u, 0x4140); r1.w = __byte_perm(re.w, 0u, 0x4342);
    i0.x = __byte_perm(im.x, 0u, 0x4140); i0.y = __byte_perm(im.x, 0u, 0x4342);
    i0.z = __byte_perm(im.y, 0u, 0x4140); i0.w = __byte_perm(im.y, 0u, 0x4342);
    i1.x = __byte_perm(im.z, 0u, 0x4140); i1.y = __byte_perm(im.z, 0u, 0x4342);
    i1.z = __byte_perm(im.w, 0u, 0x4140); i1.w = __byte_perm(im.w, 0u, 0x4342);
    const uint32_t off0 = plane_chunk_offset<2>(row, 2 * q);
    const uint32_t off1 = plane_chunk_offset<2>(row, 2 * q + 1);
    sts128(plane_re + off0, r0);
    sts128(plane_re + off1, r1);
    sts128(plane_im + off0, i0);
    sts128(plane_im + off1, i1);
  }
}

template <int EB>
__global__ void __launch_bounds__(kThreads, 1)
xcorr_tc_kernel(const __grid_constant__ CUtensorMap tmap, TcParams prm) {
  using C = Cfg<EB>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const SmemPtrs s = carve<EB>(base);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int npairs = prm.nt * (prm.nt + 1) / 2;
  const int nks = prm.nks;
  const uint64_t lim = prm.timeout_ns;
  volatile int* abort_flag = s.abort_flag;

  // ---- set-up: barriers, TMEM, zeroed sums
  if (tid == 0) {
    for (int k = 0; k < C::kRawStages; ++k) {
      mbar_init(&s.raw_full[k], 1);
      mbar_init(&s.raw_empty[k], 4);   // one elected lane per unpack warp of a group
    }
    for (int k = 0; k < C::kOpStages; ++k) {
      mbar_init(&s.op_full[k], 4);
      mbar_init(&s.op_empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&s.acc_full[k], 1);
      mbar_init(&s.acc_empty[k], 4);
      mbar_init(&s.sums_full[k], 4 * kUnpackGroups);
      mbar_init(&s.sums_empty[k], 4);
    }
    mbar_init(s.final_bar, 1);
    *s.abort_flag = 0;
    mbar_fence_init();
    tma_prefetch_desc(&tmap);
  }
  for (int k = tid; k < 2 * 4 * kTile; k += kThreads) s.sums[k] = 0;
  if (warp == 0) {
    tmem_alloc<kTmemCols>(s.tmem_slot);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_slot;

  if (warp == 0) {
    // ================================================= TMA producer
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < prm.units && ok; u += gridDim.x) {
        int c, bi, bj;
        decode_unit(u, npairs, c, bi, bj);
        const bool diag = (bi == bj);
        for (int ks = 0; ks < nks; ++ks, ++it) {
          const int st = it % C::kRawStages;
          const uint32_t ph = (it / C::kRawStages) & 1;
          if (!wait_or_abort(&s.raw_empty[st], ph ^ 1, lim, abort_flag)) {
            fail(s, prm.err, kErrWaitRawEmpty);
            ok = false;
            break;
          }
          uint8_t* dst = s.raw + st * C::kRawStage;
          mbar_arrive_expect_tx(&s.raw_full[st], diag ? kRawTile : 2 * kRawTile);
          tma_load_3d(dst, &tmap, &s.raw_full[st], bi * kTile, c, ks * kStep);
          if (!diag) tma_load_3d(dst + kRawTile, &tmap, &s.raw_full[st], bj * kTile, c, ks * kStep);
        }
      }
      // wait for the copies still in flight (normally all consumed already)
      for (int k = 0; k < C::kRawStages && k < it; ++k) {
        const int last = it - 1 - k;
        mbar_wait(&s.raw_full[last % C::kRawStages], (last / C::kRawStages) & 1, lim);
      }
    }
  } else if (warp == 1) {
    // ================================================= MMA issuer
    if (lane == 0) {
      int it = 0, ui = 0;
      bool ok = true;
      constexpr uint32_t fmt = 0;  // e4m3 for kind::f8f6f4, f16 for kind::f16
      constexpr uint32_t id_pos = idesc_mn(kTile, kTile, fmt, false);
      constexpr uint32_t id_neg = idesc_mn(kTile, kTile, fmt, true);
      for (int u = blockIdx.x; u < prm.units && ok; u += gridDim.x, ++ui) {
        int c, bi, bj;
        decode_unit(u, npairs, c, bi, bj);
        const bool diag = (bi == bj);
        const int as = ui & 1;
        if (!wait_or_abort(&s.acc_empty[as], ((ui >> 1) & 1) ^ 1, lim, abort_flag)) {
          fail(s, prm.err, kErrWaitAccEmpty);
          break;
        }
        tc_fence_after();
        const uint32_t d_re = tmem + as * 256;
        const uint32_t d_im = d_re + 128;
        for (int ks = 0; ks < nks; ++ks, ++it) {
          const int st = it % C::kOpStages;
          const uint32_t ph = (it / C::kOpStages) & 1;
          if (!wait_or_abort(&s.op_full[st], ph, lim, abort_flag)) {
            fail(s, prm.err, kErrWaitOpFull);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t op = smem_u32(s.op + st * C::kOpStage);
          const uint32_t a_re = op, a_im = op + C::kPlane;
          const uint32_t b_re = diag ? a_re : op + 2 * C::kPlane;
          const uint32_t b_im = diag ? a_im : op + 3 * C::kPlane;
          if constexpr (EB == 1) {
            const uint32_t acc0 = ks > 0 ? 1u : 0u;
            mma_f8f6f4(d_re, sdesc_mn_sw128(a_re, 4096, 1024), sdesc_mn_sw128(b_re, 4096, 1024), id_pos, acc0);
            mma_f8f6f4(d_re, sdesc_mn_sw128(a_im, 4096, 1024), sdesc_mn_sw128(b_im, 4096, 1024), id_pos, 1u);
            mma_f8f6f4(d_im, sdesc_mn_sw128(a_im, 4096, 1024), sdesc_mn_sw128(b_re, 4096, 1024), id_pos, acc0);
            mma_f8f6f4(d_im, sdesc_mn_sw128(a_re, 4096, 1024), sdesc_mn_sw128(b_im, 4096, 1024), id_neg, 1u);
          } else {
            // f16: K = 16 per instruction, two halves of the 32-row step;
            // column blocks of 64 inputs are kStep*128 = 4096 bytes apart.
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint32_t o = h * 16 * 128;
              const uint32_t acc0 = (ks > 0 || h > 0) ? 1u : 0u;
              mma_f16(d_re, sdesc_mn_sw128(a_re + o, 4096, 1024), sdesc_mn_sw128(b_re + o, 4096, 1024), id_pos, acc0);
              mma_f16(d_re, sdesc_mn_sw128(a_im + o, 4096, 1024), sdesc_mn_sw128(b_im + o, 4096, 1024), id_pos, 1u);
              mma_f16(d_im, sdesc_mn_sw128(a_im + o, 4096, 1024), sdesc_mn_sw128(b_re + o, 4096, 1024), id_pos, acc0);
              mma_f16(d_im, sdesc_mn_sw128(a_re + o, 4096, 1024), sdesc_mn_sw128(b_im + o, 4096, 1024), id_neg, 1u);
            }
          }
          mma_commit(&s.op_empty[st]);
        }
        if (!ok) break;
        mma_commit(&s.acc_full[as]);
      }
      // drain: every MMA issued so far has completed once this barrier fires
      mma_commit(s.final_bar);
      if (!mbar_wait(s.final_bar, 0, lim)) atomicOr(prm.err, kErrWaitFinal);
    }
  } else if (warp >= kUnpackWarp0 && warp < kUnpackWarp0 + kUnpackWarps) {
    // ================================================= unpack
    const int grp = (warp - kUnpackWarp0) >> 2;
    const int ut = tid - (kUnpackWarp0 + 4 * grp) * 32;
    const int q = ut & 7;         // 16-input column chunk
    const int r0 = ut >> 3;       // rows r0 and r0 + 16 of each 32-row step
    int it = 0, ui = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < prm.units && ok; u += gridDim.x, ++ui) {
      int c, bi, bj;
      decode_unit(u, npairs, c, bi, bj);
      const bool diag = (bi == bj);
      UnpackSums sI, sJ;
      sI.zero();
      sJ.zero();
      int since_flush = 0;
      for (int ks = 0; ks < nks; ++ks, ++it) {
        if (it % kUnpackGroups != grp) continue;
        const int rst = it % C::kRawStages, ost = it % C::kOpStages;
        if (!wait_or_abort(&s.raw_full[rst], (it / C::kRawStages) & 1, lim, abort_flag)) {
          fail(s, prm.err, kErrWaitRawFull);
          ok = false;
          break;
        }
        if (!wait_or_abort(&s.op_empty[ost], ((it / C::kOpStages) & 1) ^ 1, lim, abort_flag)) {
          fail(s, prm.err, kErrWaitOpEmpty);
          ok = false;
          break;
        }
        const uint8_t* raw = s.raw + rst * C::kRawStage;
        uint8_t* op = s.op + ost * C::kOpStage;
        unpack_chunk<EB>(raw, op, op + C::kPlane, r0, q, sI);
        unpack_chunk<EB>(raw, op, op + C::kPlane, r0 + 16, q, sI);
        if (!diag) {
          unpack_chunk<EB>(raw + kRawTile, op + 2 * C::kPlane, op + 3 * C::kPlane, r0, q, sJ);
          unpack_chunk<EB>(raw + kRawTile, op + 2 * C::kPlane, op + 3 * C::kPlane, r0 + 16, q, sJ);
        }
        // each lane makes its operand writes visible to the tensor core, the
        // warp converges, and one lane arrives for all 32
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&s.op_full[ost]);
          mbar_arrive(&s.raw_empty[rst]);
        }
        if (++since_flush == 8) {  // 16 rows per 8 steps: byte lanes stay <= 240
          sI.flush();
          sJ.flush();
          since_flush = 0;
        }
      }
      if (!ok) break;
      sI.flush();
      sJ.flush();
      const int as = ui & 1;
      if (!wait_or_abort(&s.sums_empty[as], ((ui >> 1) & 1) ^ 1, lim, abort_flag)) {
        fail(s, prm.err, kErrWaitSumsEmpty);
        break;
      }
      int* sums = s.sums + as * 4 * kTile;
      sI.publish(sums + 0 * kTile, sums + 1 * kTile, q);
      if (!diag) sJ.publish(sums + 2 * kTile, sums + 3 * kTile, q);
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.sums_full[as]);
    }
  } else if (warp >= kEpiWarp0) {
    // ================================================= epilogue
    // The loop never exits early: after an abort it only skips work, so the
    // named barrier below is reached the same number of times by all four
    // epilogue warps.
    const int quad = warp & 3;          // TMEM lane quadrant this warp may access
    const int r = quad * 32 + lane;     // accumulator row = input offset within I
    const float scale = (EB == 1) ? 262144.0f : 281474976710656.0f;  // 2^18, 2^48
    const int T_pad = nks * kStep;
    const long long nbl = static_cast<long long>(prm.N) * (prm.N + 1) / 2;
    bool ok = true;
    int ui = 0;
    for (int u = blockIdx.x; u < prm.units; u += gridDim.x, ++ui) {
      int c, bi, bj;
      decode_unit(u, npairs, c, bi, bj);
      const bool diag = (bi == bj);
      const int as = ui & 1;
      const uint32_t par = (ui >> 1) & 1;
      if (ok && !wait_or_abort(&s.acc_full[as], par, lim, abort_flag)) {
        fail(s, prm.err, kErrWaitAccFull);
        ok = false;
      }
      if (ok && !wait_or_abort(&s.sums_full[as], par, lim, abort_flag)) {
        fail(s, prm.err, kErrWaitSumsFull);
        ok = false;
      }
      ok = __all_sync(0xFFFFFFFFu, ok);
      int* sums = s.sums + as * 4 * kTile;
      if (ok) {
        tc_fence_after();
        const int* PJ = diag ? sums : sums + 2 * kTile;
        const int* QJ = diag ? sums + kTile : sums + 3 * kTile;
        const int Pi = sums[r], Qi = sums[kTile + r];
        const int row_re = -8 * (Pi + Qi) + 128 * T_pad;
        const int row_im = 8 * (Pi - Qi);
        const uint32_t t_row = tmem + (static_cast<uint32_t>(quad * 32) << 16) + as * 256;
        int2* stg = s.epi + quad * 32 * kEpiStagePitch;
        const long long chan_base = static_cast<long long>(c) * nbl;
#pragma unroll 1
        for (int cc = 0; cc < kTile; cc += 32) {
          uint32_t vre[32], vim[32];
          tmem_ld32(t_row + cc, vre);
          tmem_ld32(t_row + 128 + cc, vim);
          tmem_ld_wait();
          // this lane's row, 32 columns -> staging row `lane`
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const int jl = cc + k;
            const int dre = __float2int_rn(__uint_as_float(vre[k]) * scale);
            const int dim = __float2int_rn(__uint_as_float(vim[k]) * scale);
            stg[lane * kEpiStagePitch + k] =
                make_int2(dre + row_re - 8 * (PJ[jl] + QJ[jl]), dim + row_im - 8 * (PJ[jl] - QJ[jl]));
          }
          __syncwarp();
          // row by row: 32 lanes write 32 consecutive baselines (256 bytes)
          const int gj = bj * kTile + cc + lane;
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const int gr = bi * kTile + quad * 32 + rr;
            if (gr < prm.N && gj <= gr && gj < prm.N) {
              const int2 v = stg[rr * kEpiStagePitch + lane];
              int2* dst = reinterpret_cast<int2*>(prm.acc) + chan_base +
                          static_cast<long long>(gr) * (gr + 1) / 2 + gj;
              if (prm.accumulate) {
                const int2 o = *dst;
                *dst = make_int2(o.x + v.x, o.y + v.y);
              } else {
                *dst = v;
              }
            }
          }
          __syncwarp();
        }
        tc_fence_before();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.acc_empty[as]);
      // every epilogue thread has read the column sums: clear this stage
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
      sums[r] = 0;
      sums[kTile + r] = 0;
      sums[2 * kTile + r] = 0;
      sums[3 * kTile + r] = 0;
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.sums_empty[as]);
    }
  }

  // ---- tear-down: all MMAs have drained (issuer waited on final_bar)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc<kTmemCols>(tmem);
}

}  // namespace tc

int tc_smem_bytes(int eb) {
  return eb == 1 ? tc::Cfg<1>::kSmemBytes : tc::Cfg<2>::kSmemBytes;
}

int tc_threads() { return tc::kThreads; }

cudaError_t launch_xcorr_tc(int eb, const CUtensorMap* tmap, const TcParams& prm, int grid,
                            cudaStream_t stream) {
  const int smem = tc_smem_bytes(eb);
  cudaError_t e;
  if (eb == 1) {
    e = cudaFuncSetAttribute(tc::xcorr_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc::xcorr_tc_kernel<1><<<grid, tc::kThreads, smem, stream>>>(*tmap, prm);
  } else {
    e = cudaFuncSetAttribute(tc::xcorr_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc::xcorr_tc_kernel<2><<<grid, tc::kThreads, smem, stream>>>(*tmap, prm);
  }
  return cudaGetLastError();
}

}  // namespace xe
