// Phase-and-sum beamformer with time along the MMA's N dimension, for up to
// 16 beams and 512 inputs (the DRX pipeline's beamformer, section "LWA
// Sevilleta implementation", which works on the 4+4-bit samples):
//   y[t][c][b] = sum_i w[c][b][i] x[t][c][i].
//
// Per channel, Y^T (2B x T) = W' X'^T as a real product: output row o = 2b
// (Re y_b) has the coefficient Re w on the real part of x_i and -Im w on its
// imaginary part, row 2b + 1 (Im y_b) has Im w and Re w.  Time runs along
// the MMA's N (128 samples per unit), so one tcgen05 MMA does
// 128 x 128 x 32 multiply-adds; with time along M (weights as the N = 2B
// side) an MMA did only 128 x 32 x 16 at nearly the same issue cost.
//
// Operands, e4m3 (kind::f8f6f4), both exact:
//  * voltages (operand B, shared memory, K-major, 128-byte swizzle): the
//    nibble v in [-8, 7] becomes u = v + 8 = nibble XOR 8, whose e4m3 bit
//    pattern is exactly u * 2^-9 (as in the X-engine);
//  * weights (operand A, tensor memory): the float16-rounded coefficients,
//    scaled by a per-channel power of two sigma so that the largest has
//    magnitude in [128, 256), are split into four e4m3 terms,
//    v = t0 + t1 2^-4 + t2 2^-8 + t3 2^-12, each term the residual so far
//    truncated toward zero to four significant bits (or, below 2^-6, to the
//    e4m3 subnormal grid 2^-9).  Every term takes at least four bit
//    positions, so three already hold a float16 value exactly while they stay
//    above the subnormal grid: every coefficient of at least 2^-18 of the
//    channel's largest is exact, and any other errs by less than 2^-21 / sigma
//    (below 2^-28 of the largest).  The M = 128 rows are
//    row 32 q + 8 k + m = term k of output o = 8 q + m.
// Accumulators are float32; the epilogue forms
//   y_o = (D_o0 + 2^-4 D_o1 + 2^-8 D_o2 + 2^-12 D_o3) 2^9 / sigma - 8 sum_K coef,
// one tcgen05.ld.16x256b giving each thread terms 0, 1 (lanes m, m + 8) and a
// second one terms 2, 3 (lanes m + 16, m + 24) of the same output.
//
// Work: a unit is (channel, 128-sample time tile); each CTA of the persistent
// grid takes a contiguous range of units, so it changes channel at most a
// few times; the channel's weights (at most 128 rows x 1024 K bytes, 256
// TMEM columns) are loaded into tensor memory when the channel changes,
// after the last MMA of the previous channel has completed.
// Per CTA (448 threads):
//   warp 0       TMA of raw tiles [128 samples][128 inputs] (16 KB, 128-byte
//                swizzle), one per stage of 128 inputs
//   warp 1       MMA issuer (one thread): 8 MMAs per stage, D double-buffered
//   warps 2-9    unpack: 16-byte chunks of the raw tile -> re and im e4m3
//                bytes of operand B (re of inputs 64a..64a+63 at K bytes
//                0-63 of atom a, im at 64-127)
//   warps 10-13  epilogue (TMEM lane quadrant = warp mod 4): weight loads
//                into tensor memory, term combination, complex64 rows
// Every wait is bounded; on timeout the kernel records an error and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_kernels.h"
#include "xe_ptx.cuh"

namespace xe {
namespace b8 {

constexpr int kTile = 128;                    // time samples per unit (MMA N)
constexpr int kStageIn = 128;                 // inputs per stage
constexpr int kRawStage = kTile * kStageIn;   // 16 KB: [128 t][128 inputs], 128-byte swizzle
constexpr int kAtom = kTile * 128;            // 16 KB: [128 t][128 K bytes], K-major, 128-byte swizzle
constexpr int kOpStage = 2 * kAtom;           // K = 256 bytes per stage
constexpr int kRaw = 3;
constexpr int kOp = 4;
constexpr int kRows = 128;                    // MMA M: 4 terms x up to 32 outputs
constexpr int kMaxStages = 4;                 // weights: 64 columns per stage in [0, 256) of tensor memory
constexpr int kD0 = 256;                      // accumulators: [256, 384) and [384, 512)
constexpr int kRawWarp = 0, kMmaWarp = 1, kUnpackWarp0 = 2, kUnpackWarps = 8;
constexpr int kEpiWarp0 = kUnpackWarp0 + kUnpackWarps;
constexpr int kThreads = 32 * (kEpiWarp0 + 4);
constexpr int kNumBars = 2 * kRaw + 2 * kOp + 2 + 2 + 1 + 1;
constexpr int kSmemBytes = kOp * kOpStage + kRaw * kRawStage + kNumBars * 8 + 16 + 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
static_assert(kMaxStages * 64 <= kD0, "weight columns below the accumulators");

enum ErrCode : int {
  kErrRawFull = 1 << 0, kErrRawEmpty = 1 << 1, kErrOpFull = 1 << 2, kErrOpEmpty = 1 << 3,
  kErrAccFull = 1 << 4, kErrAccEmpty = 1 << 5, kErrAFull = 1 << 6, kErrFinal = 1 << 7,
};

struct Smem {
  uint8_t* op;     // [kOp][2 atoms][128 t][128 K bytes]
  uint8_t* raw;    // [kRaw][128 t][128 bytes]
  uint64_t *raw_full, *raw_empty, *op_full, *op_empty, *acc_full, *acc_empty, *a_full, *fin;
  uint32_t* tmem_slot;
  int* abort_flag;
};

__device__ __forceinline__ Smem carve(uint8_t* base) {
  Smem s;
  s.op = base;
  s.raw = base + kOp * kOpStage;
  uint64_t* b = reinterpret_cast<uint64_t*>(s.raw + kRaw * kRawStage);
  s.raw_full = b; b += kRaw;
  s.raw_empty = b; b += kRaw;
  s.op_full = b; b += kOp;
  s.op_empty = b; b += kOp;
  s.acc_full = b; b += 2;
  s.acc_empty = b; b += 2;
  s.a_full = b; b += 1;
  s.fin = b; b += 1;
  s.tmem_slot = reinterpret_cast<uint32_t*>(b);
  s.abort_flag = reinterpret_cast<int*>(b) + 1;
  return s;
}

__device__ __forceinline__ void fail(const Smem& s, int* err, int code) {
  atomicExch(s.abort_flag, 1);
  atomicOr(err, code);
}

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

// D += A B^T, A (128 rows x K = 32 e4m3) in tensor memory, B K-major in shared memory.
__device__ __forceinline__ void mma_f8_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}"
               ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

// K-major operand, 128-byte swizzle: 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= 1ull << 16;
  d |= static_cast<uint64_t>(1024 >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

// 16 lanes x 8 columns, 4 times along the columns: thread i gets lanes
// base + i / 4 (regs 4 j, 4 j + 1) and base + i / 4 + 8 (4 j + 2, 4 j + 3)
// at columns 8 j + 2 (i % 4) and 8 j + 2 (i % 4) + 1.
__device__ __forceinline__ void tmem_ld_16x256b_x4(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// 32 lanes x 16 consecutive columns: thread `lane` writes row (quadrant base + lane).
__device__ __forceinline__ void tmem_st_32x32b_x16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// One channel's weight rows (this warp's TMEM lane quadrant) into tensor memory.
__device__ __forceinline__ void load_weights(uint32_t tmem, int quad, int lane, const uint8_t* wa, int c,
                                             int kbytes) {
  const int row = 32 * quad + lane;
  const uint4* src = reinterpret_cast<const uint4*>(wa + (static_cast<long long>(c) * kRows + row) * kbytes);
  const uint32_t t_row = tmem + (static_cast<uint32_t>(32 * quad) << 16);
  for (int cc = 0; cc < kbytes / 64; ++cc) {
    uint32_t r[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 v = __ldg(src + 4 * cc + k);
      r[4 * k] = v.x;
      r[4 * k + 1] = v.y;
      r[4 * k + 2] = v.z;
      r[4 * k + 3] = v.w;
    }
    tmem_st_32x32b_x16(t_row + 16 * cc, r);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
beam8_kernel(const __grid_constant__ CUtensorMap tmap, const Beam8Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Smem s = carve(base);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long units = static_cast<long long>(p.C) * p.tiles;
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  const int S = p.S;                 // stages of 128 inputs, at most kMaxStages
  const int kbytes = 256 * S;        // K bytes per weight row
  const uint64_t lim = p.timeout_ns;
  volatile int* abort_flag = s.abort_flag;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kRaw; ++i) {
      mbar_init(&s.raw_full[i], 1);
      mbar_init(&s.raw_empty[i], kUnpackWarps);
    }
    for (int i = 0; i < kOp; ++i) {
      mbar_init(&s.op_full[i], kUnpackWarps);
      mbar_init(&s.op_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.acc_full[i], 1);
      mbar_init(&s.acc_empty[i], 4);
    }
    mbar_init(s.a_full, 4);
    mbar_init(s.fin, 1);
    *s.abort_flag = 0;
    mbar_fence_init();
    tma_prefetch_desc(&tmap);
  }
  if (warp == kMmaWarp) {
    tmem_alloc<512>(s.tmem_slot);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_slot;

  if (warp == kRawWarp) {
    // ------------------------------------------------------------ raw producer
    if (lane == 0) {
      int h = 0;
      bool ok = true;
      for (long long u = u0; u < u1 && ok; ++u) {
        const int c = static_cast<int>(u / p.tiles), t0 = static_cast<int>(u % p.tiles) * kTile;
        for (int st = 0; st < S; ++st, ++h) {
          const int rs = h % kRaw;
          if (h >= kRaw && !wait_or_abort(&s.raw_empty[rs], ((h / kRaw) & 1) ^ 1, lim, abort_flag)) {
            if (!*abort_flag) fail(s, p.err, kErrRawEmpty);
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&s.raw_full[rs], kRawStage);
          tma_load_3d(s.raw + rs * kRawStage, &tmap, &s.raw_full[rs], st * kStageIn, c, t0);
        }
      }
      // every copy issued has landed before the CTA may exit
      for (int k = h - 1; k >= 0 && k >= h - kRaw; --k)
        mbar_wait(&s.raw_full[k % kRaw], static_cast<uint32_t>((k / kRaw) & 1), lim);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // e4m3 x e4m3 -> f32, A from tensor memory, B K-major; M = 128, N = 128.
      // Descriptors are one base per operand slot plus compile-time offsets
      // and the slot and its phase are counters: the tensor core's
      // instruction queue is short, so scalar work between MMAs shows.
      constexpr uint32_t idesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
      constexpr uint32_t kSlotDesc = kOpStage >> 4, kAtomDesc = kAtom >> 4;   // descriptor address units
      const uint64_t desc0 = sdesc_k_sw128(smem_u32(s.op));
      int j = 0, wl = 0, os = 0;
      uint32_t oph = 0;                     // phase of operand slot os
      int prev_c = -1;
      bool ok = true;
      for (long long u = u0; u < u1 && ok; ++u, ++j) {
        const int c = static_cast<int>(u / p.tiles);
        if (c != prev_c) {   // this channel's weights are in tensor memory
          if (!wait_or_abort(s.a_full, wl & 1, lim, abort_flag)) {
            if (!*abort_flag) fail(s, p.err, kErrAFull);
            break;
          }
          ++wl;
          prev_c = c;
        }
        const int ab = j & 1;
        if (j >= 2 && !wait_or_abort(&s.acc_empty[ab], ((j >> 1) - 1) & 1, lim, abort_flag)) {
          if (!*abort_flag) fail(s, p.err, kErrAccEmpty);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + kD0 + 128 * ab;
        for (int st = 0; st < S; ++st) {
          if (!wait_or_abort(&s.op_full[os], oph, lim, abort_flag)) {
            if (!*abort_flag) fail(s, p.err, kErrOpFull);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t bd = desc0 + static_cast<uint64_t>(kSlotDesc * os);
          const uint32_t a0 = tmem + 64 * st;
          const uint32_t acc_first = st > 0 ? 1u : 0u;
#pragma unroll
          for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              mma_f8_tmem_a(d, a0 + 32 * a + 8 * ks, bd + kAtomDesc * a + 2 * ks, idesc,
                            (a | ks) != 0 ? 1u : acc_first);
          mma_commit(&s.op_empty[os]);
          if (++os == kOp) {
            os = 0;
            oph ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(&s.acc_full[ab]);
      }
      // all MMAs of this thread have completed before tensor memory is freed
      mma_commit(s.fin);
      if (!mbar_wait(s.fin, 0, lim)) atomicOr(p.err, kErrFinal);
    }
  } else if (warp < kEpiWarp0) {
    // ------------------------------------------------------------ unpack
    // Per stage each warp converts 16 time rows: 8 rows x 4 chunks per pass
    // (rows r0 .. r0 + 7 in lanes 0-7 of each quarter: distinct swizzle
    // phases, so the 16-byte loads and stores are conflict-free).
    const int w8 = warp - kUnpackWarp0;
    int h = 0;
    bool ok = true;
    for (long long u = u0; u < u1 && ok; ++u) {
      for (int st = 0; st < S; ++st, ++h) {
        const int rs = h % kRaw, os = h % kOp;
        if (!wait_or_abort(&s.raw_full[rs], (h / kRaw) & 1, lim, abort_flag)) {
          if (!*abort_flag) fail(s, p.err, kErrRawFull);
          ok = false;
          break;
        }
        if (h >= kOp && !wait_or_abort(&s.op_empty[os], ((h / kOp) & 1) ^ 1, lim, abort_flag)) {
          if (!*abort_flag) fail(s, p.err, kErrOpEmpty);
          ok = false;
          break;
        }
        const uint8_t* raw = s.raw + rs * kRawStage;
        uint8_t* op = s.op + os * kOpStage;
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
          const int r = 16 * w8 + 8 * (pass & 1) + (lane & 7);   // time row
          const int jc = 4 * (pass >> 1) + (lane >> 3);           // 16-input chunk of the stage
          const int ph = r & 7;
          const uint4 x = *reinterpret_cast<const uint4*>(raw + r * 128 + ((jc ^ ph) << 4));
          uint4 re, im;
          re.x = ((x.x >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
          re.y = ((x.y >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
          re.z = ((x.z >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
          re.w = ((x.w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
          im.x = (x.x & 0x0F0F0F0Fu) ^ 0x08080808u;
          im.y = (x.y & 0x0F0F0F0Fu) ^ 0x08080808u;
          im.z = (x.z & 0x0F0F0F0Fu) ^ 0x08080808u;
          im.w = (x.w & 0x0F0F0F0Fu) ^ 0x08080808u;
          const int q = jc & 3;
          uint8_t* row = op + (jc >> 2) * kAtom + (r >> 3) * 1024 + ph * 128;
          *reinterpret_cast<uint4*>(row + ((q ^ ph) << 4)) = re;
          *reinterpret_cast<uint4*>(row + (((4 + q) ^ ph) << 4)) = im;
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&s.op_full[os]);
          mbar_arrive(&s.raw_empty[rs]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int m = lane >> 2, o = 8 * quad + m;   // this thread's output row
    const int R = 2 * p.B;
    int j = 0;
    bool ok = true;
    if (u0 < u1) {
      load_weights(tmem, quad, lane, p.wa, static_cast<int>(u0 / p.tiles), kbytes);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(s.a_full);
    }
    for (long long u = u0; u < u1 && ok; ++u, ++j) {
      const int c = static_cast<int>(u / p.tiles), t0 = static_cast<int>(u % p.tiles) * kTile;
      const int ab = j & 1;
      if (!wait_or_abort(&s.acc_full[ab], (j >> 1) & 1, lim, abort_flag)) {
        if (!*abort_flag) fail(s, p.err, kErrAccFull);
        ok = false;
        break;
      }
      tc_fence_after();
      if (u + 1 < u1 && static_cast<int>((u + 1) / p.tiles) != c) {
        // every MMA of this channel has completed: the next channel's weights
        load_weights(tmem, quad, lane, p.wa, c + 1, kbytes);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(s.a_full);
        tc_fence_after();
      }
      const float osc = p.osc[c];
      const float bias = o < R ? p.bias[c * 32 + o] : 0.f;
      float* out_c = p.out + static_cast<long long>(c) * R + o;
      const long long row_stride = static_cast<long long>(p.C) * R;
      const uint32_t t_lo = tmem + (static_cast<uint32_t>(32 * quad) << 16) + kD0 + 128 * ab;
      const uint32_t t_hi = t_lo + (16u << 16);
#pragma unroll 1
      for (int ch = 0; ch < 4; ++ch) {
        uint32_t lo[16], hi[16];
        tmem_ld_16x256b_x4(t_lo + 32 * ch, lo);   // terms 0 (lane m) and 1 (lane m + 8)
        tmem_ld_16x256b_x4(t_hi + 32 * ch, hi);   // terms 2 (lane m + 16) and 3 (lane m + 24)
        tmem_ld_wait();
        if (o < R) {
#pragma unroll
          for (int blk = 0; blk < 4; ++blk)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              float v = __uint_as_float(hi[4 * blk + 2 + e]) * 0.000244140625f;       // 2^-12
              v = __fmaf_rn(__uint_as_float(hi[4 * blk + e]), 0.00390625f, v);         // 2^-8
              v = __fmaf_rn(__uint_as_float(lo[4 * blk + 2 + e]), 0.0625f, v);         // 2^-4
              v += __uint_as_float(lo[4 * blk + e]);
              const int t = t0 + 32 * ch + 8 * blk + 2 * (lane & 3) + e;
              if (t < p.T) out_c[t * row_stride] = __fmaf_rn(v, osc, -bias);
            }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.acc_empty[ab]);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc<512>(tmem);
  }
}

// ------------------------------------------------------------------ weights
// Float16 rounding of a weight component, as the operand precision.
__device__ __forceinline__ float f16r(float x) { return __half2float(__float2half_rn(x)); }

// Coefficient of output row o (o = 2b: Re y_b, o = 2b + 1: Im y_b) on the
// real (part 0) or imaginary (part 1) component of input i.
__device__ __forceinline__ float coef(const float2* w, int N, int B, int c, int o, int i, int part) {
  const float2 v = w[(static_cast<long long>(c) * B + (o >> 1)) * N + i];
  const float wr = f16r(v.x), wi = f16r(v.y);
  if ((o & 1) == 0) return part == 0 ? wr : -wi;
  return part == 0 ? wi : wr;
}

// Largest |coefficient| of each channel -> sigma (a power of two putting it
// in [128, 256)); one block of 256 threads per channel.
__global__ void beam8_scale_kernel(const float2* __restrict__ w, int N, int C, int B, float* __restrict__ sigma,
                                   float* __restrict__ osc) {
  __shared__ float red[256];
  const int c = blockIdx.x;
  float mx = 0.f;
  for (int k = threadIdx.x; k < B * N; k += 256) {
    const float2 v = w[static_cast<long long>(c) * B * N + k];
    mx = fmaxf(mx, fmaxf(fabsf(f16r(v.x)), fabsf(f16r(v.y))));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int e = 0;
    if (red[0] > 0.f) frexpf(red[0], &e);   // red[0] in [2^(e-1), 2^e)
    const float sg = ldexpf(1.f, 8 - e);    // largest * sigma in [128, 256)
    sigma[c] = red[0] > 0.f ? sg : 1.f;
    osc[c] = red[0] > 0.f ? ldexpf(1.f, 9 - (8 - e)) : 512.f;   // 2^9 / sigma
  }
}

// bias[c][o] = 8 * sum over K of the row's coefficients (float64 sum).
__global__ void beam8_bias_kernel(const float2* __restrict__ w, int N, int C, int B, float* __restrict__ bias) {
  const int idx = blockIdx.x * 256 + threadIdx.x;
  if (idx >= C * 32) return;
  const int c = idx / 32, o = idx % 32;
  double acc = 0.0;
  if (o < 2 * B)
    for (int i = 0; i < N; ++i) acc += static_cast<double>(coef(w, N, B, c, o, i, 0)) + coef(w, N, B, c, o, i, 1);
  bias[idx] = static_cast<float>(8.0 * acc);
}

// The next weight term: x truncated toward zero to four significant bits,
// or to the e4m3 subnormal grid 2^-9 below 2^-6.
__device__ __forceinline__ float term4(float x) {
  if (fabsf(x) >= 0.015625f) return __uint_as_float(__float_as_uint(x) & 0xFFF00000u);
  return copysignf(floorf(fabsf(x) * 512.f) * 0.001953125f, x);
}

// e4m3 bit pattern of a term4 value: four significant bits in the normal
// range 2^-6 <= |x| < 256, or a multiple of 2^-9 below it.
__device__ __forceinline__ uint32_t e4m3_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t sgn = (u >> 31) << 7;
  const float a = fabsf(x);
  if (a < 0.015625f) return sgn | static_cast<uint32_t>(a * 512.f);   // subnormal: m 2^-9, m < 8 (exact)
  const int e = static_cast<int>((u >> 23) & 0xFF) - 127;             // -6 .. 8
  return sgn | (static_cast<uint32_t>(e + 7) << 3) | ((u >> 20) & 7u);
}

// Operand A images: [C][128 rows][2 Npad K bytes]; one thread per 4 K bytes.
__global__ void beam8_image_kernel(const float2* __restrict__ w, int N, int C, int B, int S,
                                   const float* __restrict__ sigma, uint32_t* __restrict__ wa) {
  const int kw = 64 * S;   // 32-bit words per row
  const long long idx = blockIdx.x * 256LL + threadIdx.x;
  if (idx >= static_cast<long long>(C) * kRows * kw) return;
  const int wd = static_cast<int>(idx % kw);
  const int row = static_cast<int>((idx / kw) % kRows);
  const int c = static_cast<int>(idx / (static_cast<long long>(kw) * kRows));
  const int q = row >> 5, k = (row >> 3) & 3, o = 8 * q + (row & 7);
  uint32_t word = 0;
  if (o < 2 * B) {
    const float sg = sigma[c];
#pragma unroll
    for (int bt = 0; bt < 4; ++bt) {
      const int K = 4 * wd + bt;                  // K byte: stage K / 256, atom (K / 128) & 1
      const int kb = K & 127, part = kb >> 6;
      const int i = (K >> 8) * kStageIn + ((K >> 7) & 1) * 64 + (kb & 63);
      if (i >= N) continue;
      float r = coef(w, N, B, c, o, i, part) * sg;   // exact: a power-of-two scaling
      float t = term4(r);
      for (int kk = 0; kk < k; ++kk) {
        r = (r - t) * 16.f;                          // exact
        t = term4(r);
      }
      word |= e4m3_bits(t) << (8 * bt);
    }
  }
  wa[idx] = word;
}

}  // namespace b8

int beam8_smem_bytes() { return b8::kSmemBytes; }

cudaError_t launch_beam8(const CUtensorMap* tmap, const Beam8Params& prm, int grid, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(b8::beam8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       b8::kSmemBytes);
  if (e != cudaSuccess) return e;
  b8::beam8_kernel<<<grid, b8::kThreads, b8::kSmemBytes, stream>>>(*tmap, prm);
  return cudaGetLastError();
}

cudaError_t launch_beam8_weights(const float* w, int N, int C, int B, int S, uint8_t* wa, float* sigma, float* osc,
                                 float* bias, cudaStream_t stream) {
  const float2* w2 = reinterpret_cast<const float2*>(w);
  b8::beam8_scale_kernel<<<C, 256, 0, stream>>>(w2, N, C, B, sigma, osc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  b8::beam8_bias_kernel<<<(C * 32 + 255) / 256, 256, 0, stream>>>(w2, N, C, B, bias);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = static_cast<long long>(C) * b8::kRows * 64 * S;
  b8::beam8_image_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
      w2, N, C, B, S, sigma, reinterpret_cast<uint32_t*>(wa));
  return cudaGetLastError();
}

}  // namespace xe
