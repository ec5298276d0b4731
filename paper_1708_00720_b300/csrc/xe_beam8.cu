// Phase-and-sum beamformer for up to 16 beams and 512 inputs (the DRX
// pipeline's beamformer, section "LWA Sevilleta implementation", which works
// on the 4+4-bit samples):
//   y[t][c][b] = sum_i w[c][b][i] x[t][c][i].
//
// Per channel, Y (T x 2B) = X' W'^T as a real product: output o = 2b
// (Re y_b) has the coefficient Re w on the real part of x_i and -Im w on its
// imaginary part, o = 2b + 1 (Im y_b) has Im w and Re w.  One tcgen05 MMA
// (kind::f8f6f4, cta_group::1) does M = 128 samples x N = 128 weight rows x
// K = 32 bytes.
//
// Operands, e4m3, both exact:
//  * voltages (operand A, tensor memory): time sample t of a 128-sample unit
//    is TMEM lane t, so a thread copies its own raw row with no
//    transposition: the nibble v in [-8, 7] becomes u = v + 8 = nibble XOR 8,
//    whose e4m3 bit pattern is exactly u * 2^-9 (as in the X-engine); per
//    stage of 128 inputs the real parts fill K bytes 0-127 (columns 0-31)
//    and the imaginary parts K bytes 128-255 (columns 32-63);
//  * weights (operand B, shared memory, K-major with the 128-byte swizzle,
//    resident for as long as a CTA works on the channel): the float16-rounded
//    coefficients, scaled by a per-channel power of two sigma so that the
//    largest has magnitude in [128, 256), split into four e4m3 terms
//    v = t0 + t1 2^-4 + t2 2^-8 + t3 2^-12, each the residual so far
//    truncated toward zero to four significant bits (or, below 2^-6, to the
//    e4m3 subnormal grid 2^-9).  Every term takes at least four bit
//    positions, so three already hold a float16 value exactly while they stay
//    above the subnormal grid: every coefficient of at least 2^-18 of the
//    channel's largest is exact, and any other errs by less than 2^-21 / sigma
//    (below 2^-28 of the largest).  Weight row n = 4 o + k is term k of
//    output o (zero rows beyond 2B outputs), so D column 4 o + k holds it.
// Accumulators are float32; the epilogue forms
//   y_o = (D_o0 + 2^-4 D_o1 + 2^-8 D_o2 + 2^-12 D_o3) 2^9 / sigma - 8 sum_K coef.
//
// Why this way round.  Shared memory carries, per 128-input stage, the raw
// tile in (TMA) and out (unpack) and the tensor core's operand-B reads:
// 64 KB, against 96 KB when the voltages were the shared-memory operand
// (their unpacked copy was written and read again).
//
// Work: a unit is (channel, 128-sample time tile); each CTA of the
// persistent grid takes a contiguous range of units, so it changes channel
// at most a few times.  A channel's weights (S stages x 32 KB, pre-swizzled
// in global memory) arrive by one bulk copy when the last MMA of the
// previous channel has completed, issued by the MMA thread (the voltage
// producers carry on meanwhile).
// Per CTA (448 threads):
//   warp 0       TMA of raw tiles [128 samples][128 inputs] (16 KB, 128-byte
//                swizzle), one per stage
//   warp 1       MMA issuer (one thread): 8 MMAs per stage, D double-buffered;
//                at a channel change it waits for its own MMAs, copies the
//                channel's weights in (one bulk copy) and prefetches the
//                next channel's into L2
//   warps 2-9    unpack: TMEM lane quadrant warp % 4, half (warp - 2) / 4 of
//                the 16-byte chunks of each raw row -> tcgen05.st.32x32b
//   warps 10-13  epilogue (TMEM lane quadrant = warp mod 4): terms combined,
//                rows staged in shared memory, written as whole 128-byte lines
// Every wait is bounded; on timeout the kernel records an error and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_kernels.h"
#include "xe_ptx.cuh"

namespace xe {
namespace b8 {

constexpr int kTile = 128;                    // time samples per unit (MMA M)
constexpr int kStageIn = 128;                 // inputs per stage
constexpr int kRawStage = kTile * kStageIn;   // 16 KB: [128 t][128 inputs], 128-byte swizzle
constexpr int kAtom = 128 * 128;              // 16 KB: [128 weight rows][128 K bytes], K-major, 128-byte swizzle
constexpr int kWStage = 2 * kAtom;            // weights of one stage: K = 256 bytes (re part, im part)
// Raw stages: 4 or 5 stages, or an L2 prefetch 2 or 3 stages ahead,
// measured no faster than 3.
constexpr int kRaw = 3;
constexpr int kOp = 4;                        // voltage stages in tensor memory, 64 columns each
constexpr int kRows = 128;                    // MMA N: 4 terms x up to 32 outputs
constexpr int kMaxStages = 4;
constexpr int kD0 = 256;                      // accumulators: [256, 384) and [384, 512)
constexpr int kRawWarp = 0, kMmaWarp = 1, kUnpackWarp0 = 2, kUnpackWarps = 8;
constexpr int kEpiWarp0 = kUnpackWarp0 + kUnpackWarps;
constexpr int kThreads = 32 * (kEpiWarp0 + 4);
constexpr int kOutRow = 128;                  // staged output bytes per time row: 16 beams x complex64
constexpr int kStageOut = 4 * 32 * kOutRow;   // 16 KB: the epilogue warps' rows
constexpr int kNumBars = 2 * kRaw + 2 * kOp + 2 + 2 + 2 + 1;
constexpr int kSmemBytes = kMaxStages * kWStage + kRaw * kRawStage + kStageOut + kNumBars * 8 + 16 + 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
static_assert(kOp * 64 <= kD0, "voltage columns below the accumulators");

enum ErrCode : int {
  kErrRawFull = 1 << 0, kErrRawEmpty = 1 << 1, kErrOpFull = 1 << 2, kErrOpEmpty = 1 << 3,
  kErrAccFull = 1 << 4, kErrAccEmpty = 1 << 5, kErrWFull = 1 << 6, kErrFinal = 1 << 7, kErrWEmpty = 1 << 8,
};

struct Smem {
  uint8_t* w;      // [kMaxStages][2 atoms][128 rows][128 K bytes]  this channel's weights
  uint8_t* raw;    // [kRaw][128 t][128 bytes]
  uint8_t* out;    // [4 warps][32 rows][128 bytes]  epilogue staging
  uint64_t *raw_full, *raw_empty, *op_full, *op_empty, *acc_full, *acc_empty, *w_full, *w_empty, *fin;
  uint32_t* tmem_slot;
  int* abort_flag;
};

__device__ __forceinline__ Smem carve(uint8_t* base) {
  Smem s;
  s.w = base;
  s.raw = base + kMaxStages * kWStage;
  s.out = s.raw + kRaw * kRawStage;
  uint64_t* b = reinterpret_cast<uint64_t*>(s.out + kStageOut);
  s.raw_full = b; b += kRaw;
  s.raw_empty = b; b += kRaw;
  s.op_full = b; b += kOp;
  s.op_empty = b; b += kOp;
  s.acc_full = b; b += 2;
  s.acc_empty = b; b += 2;
  s.w_full = b; b += 1;
  s.w_empty = b; b += 1;
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

// 32 lanes x 16 consecutive columns: thread `lane` writes row (quadrant base + lane).
__device__ __forceinline__ void tmem_st_32x32b_x16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// L2 prefetch of a global range (no shared-memory destination).
__device__ __forceinline__ void bulk_prefetch_l2(const void* gmem_src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gmem_src), "r"(bytes) : "memory");
}

// Bulk copy global -> shared (no tensor map), completion on an mbarrier.
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(smem_dst)), "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Channel and time tile of consecutive units, advanced without a 64-bit
// division per unit.
struct UnitPos {
  int c, tile;
  __device__ __forceinline__ UnitPos(long long u, int tiles)
      : c(static_cast<int>(u / tiles)), tile(static_cast<int>(u % tiles)) {}
  __device__ __forceinline__ void next(int tiles) {
    if (++tile == tiles) {
      tile = 0;
      ++c;
    }
  }
};

__global__ void __launch_bounds__(kThreads, 1)
beam8_kernel(const __grid_constant__ CUtensorMap tmap, const Beam8Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Smem s = carve(base);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long units = static_cast<long long>(p.C) * p.tiles;
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  const int S = p.S;                          // stages of 128 inputs, at most kMaxStages
  const uint32_t wbytes = static_cast<uint32_t>(S) * kWStage;   // one channel's weights
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
    mbar_init(s.w_full, 1);
    mbar_init(s.w_empty, 1);
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
      UnitPos up(u0, p.tiles);
      for (long long u = u0; u < u1 && ok; ++u, up.next(p.tiles)) {
        const int c = up.c, t0 = up.tile * kTile;
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
      constexpr uint32_t idesc = (1u << 4) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
      constexpr uint32_t kWStageDesc = kWStage >> 4, kAtomDesc = kAtom >> 4;   // descriptor address units
      const uint64_t wdesc0 = sdesc_k_sw128(smem_u32(s.w));
      int j = 0, wl = 0, os = 0;
      uint32_t oph = 0;                     // phase of operand slot os
      int prev_c = -1;
      bool ok = true;
      UnitPos up(u0, p.tiles);
      for (long long u = u0; u < u1 && ok; ++u, ++j, up.next(p.tiles)) {
        const int c = up.c;
        if (c != prev_c) {
          // This thread loads the channel's weights: once the previous
          // channel's MMAs (which read the old ones) have completed, one bulk
          // copy; meanwhile the producers keep filling the voltage stages.
          if (prev_c >= 0) {
            mma_commit(s.w_empty);
            if (!wait_or_abort(s.w_empty, (wl - 1) & 1, lim, abort_flag)) {
              if (!*abort_flag) fail(s, p.err, kErrWEmpty);
              break;
            }
          }
          mbar_arrive_expect_tx(s.w_full, wbytes);
          bulk_load(s.w, p.wa + static_cast<long long>(c) * wbytes, wbytes, s.w_full);
          // the next channel of this CTA's range into L2 ahead of its copy
          if (u + (p.tiles - up.tile) < u1)
            bulk_prefetch_l2(p.wa + (static_cast<long long>(c) + 1) * wbytes, wbytes);
          if (!wait_or_abort(s.w_full, wl & 1, lim, abort_flag)) {
            if (!*abort_flag) fail(s, p.err, kErrWFull);
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
          const uint64_t bd = wdesc0 + static_cast<uint64_t>(kWStageDesc * st);
          const uint32_t a0 = tmem + 64 * os;
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
    // ------------------------------------------------------------ unpack -> tensor memory
    // Thread = TMEM lane = time row t of the unit (t = 32 quad + lane); this
    // warp converts chunks 4 hf .. 4 hf + 3 (inputs 64 hf .. 64 hf + 63) of
    // the row: real parts to columns 16 hf .. 16 hf + 15 of the stage,
    // imaginary parts to 32 + 16 hf .. 32 + 16 hf + 15.  Within a quarter
    // warp the rows have distinct swizzle phases: conflict-free loads.
    const int w8 = warp - kUnpackWarp0;
    const int quad = warp & 3, hf = w8 >> 2;
    const int t = 32 * quad + lane;
    const uint32_t lane_off = static_cast<uint32_t>(32 * quad) << 16;
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
        const uint8_t* row = s.raw + rs * kRawStage + t * 128;
        uint4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          v[q] = *reinterpret_cast<const uint4*>(row + (((4 * hf + q) ^ (t & 7)) << 4));
        uint32_t re[16], im[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t x[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            re[4 * q + k] = ((x[k] >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
            im[4 * q + k] = (x[k] & 0x0F0F0F0Fu) ^ 0x08080808u;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.raw_empty[rs]);   // the row is in registers
        if (h >= kOp && !wait_or_abort(&s.op_empty[os], ((h / kOp) & 1) ^ 1, lim, abort_flag)) {
          if (!*abort_flag) fail(s, p.err, kErrOpEmpty);
          ok = false;
          break;
        }
        const uint32_t ta = tmem + lane_off + 64 * os + 16 * hf;
        tmem_st_32x32b_x16(ta, re);
        tmem_st_32x32b_x16(ta + 32, im);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.op_full[os]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // Thread = TMEM lane = time row t; D column 4 o + k is term k of output o.
    const int quad = warp & 3;
    const int R = 2 * p.B;
    uint8_t* stage = s.out + quad * (32 * kOutRow);
    const int row_bytes = 8 * p.B;            // complex64 per beam
    int j = 0;
    bool ok = true;
    UnitPos up(u0, p.tiles);
    for (long long u = u0; u < u1 && ok; ++u, ++j, up.next(p.tiles)) {
      const int c = up.c, t0 = up.tile * kTile;
      const int ab = j & 1;
      if (!wait_or_abort(&s.acc_full[ab], (j >> 1) & 1, lim, abort_flag)) {
        if (!*abort_flag) fail(s, p.err, kErrAccFull);
        ok = false;
        break;
      }
      tc_fence_after();
      const float osc = p.osc[c];
      const uint32_t t_row = tmem + (static_cast<uint32_t>(32 * quad) << 16) + kD0 + 128 * ab;
      float y[32];
#pragma unroll
      for (int g = 0; g < 4; g += 2) {   // outputs 8 g .. 8 g + 15, two loads in flight
        uint32_t v[32], w[32];
        tmem_ld32(t_row + 32 * g, v);
        tmem_ld32(t_row + 32 * g + 32, w);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float a = __uint_as_float(v[4 * e + 3]) * 0.000244140625f;       // 2^-12
          a = __fmaf_rn(__uint_as_float(v[4 * e + 2]), 0.00390625f, a);     // 2^-8
          a = __fmaf_rn(__uint_as_float(v[4 * e + 1]), 0.0625f, a);         // 2^-4
          y[8 * g + e] = a + __uint_as_float(v[4 * e]);
          float b = __uint_as_float(w[4 * e + 3]) * 0.000244140625f;
          b = __fmaf_rn(__uint_as_float(w[4 * e + 2]), 0.00390625f, b);
          b = __fmaf_rn(__uint_as_float(w[4 * e + 1]), 0.0625f, b);
          y[8 * g + 8 + e] = b + __uint_as_float(w[4 * e]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.acc_empty[ab]);   // D read: the MMA may reuse it
      // this row's outputs, scaled and unbiased, into its staging row as
      // 16-byte chunks at position chunk XOR (row mod 8): the 32 rows of a
      // warp then spread over all banks (rows are 128 bytes apart)
      const float* bc = p.bias + c * 32;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 bv = *reinterpret_cast<const float4*>(bc + 4 * k);
        float4 val;
        val.x = __fmaf_rn(y[4 * k + 0], osc, -bv.x);
        val.y = __fmaf_rn(y[4 * k + 1], osc, -bv.y);
        val.z = __fmaf_rn(y[4 * k + 2], osc, -bv.z);
        val.w = __fmaf_rn(y[4 * k + 3], osc, -bv.w);
        *reinterpret_cast<float4*>(stage + lane * kOutRow + ((k ^ (lane & 7)) << 4)) = val;
      }
      __syncwarp();
      // the 32 rows of this warp, whole lines: lane k of each 8-lane group
      // writes 16 bytes of row 4 pass + lane / 8
      float* out_c = p.out + static_cast<long long>(c) * R;
      const long long row_stride = static_cast<long long>(p.C) * R;   // floats per time row of out
#pragma unroll 1
      for (int r0 = 0; r0 < 32; r0 += 4) {
        const int r = r0 + (lane >> 3), k16 = lane & 7;
        const int tg = t0 + 32 * quad + r;
        if (tg < p.T && 16 * k16 < row_bytes) {
          const float4 val = *reinterpret_cast<const float4*>(stage + r * kOutRow + ((k16 ^ (r & 7)) << 4));
          *reinterpret_cast<float4*>(out_c + tg * row_stride + 4 * k16) = val;
        }
      }
      __syncwarp();
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

// Operand B images, laid out as shared memory holds them: per channel
// [stage][re part, im part][128 rows][128 K bytes] with the 128-byte swizzle
// (16-byte chunk q of row n at position q XOR (n mod 8)); row n = 4 o + k
// holds term k of output o; K byte kb of a stage is input 128 stage + kb.
// One thread per 4 K bytes.
__global__ void beam8_image_kernel(const float2* __restrict__ w, int N, int C, int B, int S,
                                   const float* __restrict__ sigma, uint32_t* __restrict__ wa) {
  const long long idx = blockIdx.x * 256LL + threadIdx.x;
  if (idx >= static_cast<long long>(C) * S * 2 * kRows * 32) return;
  const int pw = static_cast<int>(idx & 31);                  // word of the 128-byte row (physical)
  const int n = static_cast<int>((idx >> 5) % kRows);
  const int part = static_cast<int>((idx >> 5) / kRows % 2);
  const int st = static_cast<int>((idx >> 5) / (2 * kRows) % S);
  const int c = static_cast<int>(idx / (32LL * kRows * 2 * S));
  const int o = n >> 2, k = n & 3;
  const int q = (pw >> 2) ^ (n & 7);                          // logical 16-byte chunk
  uint32_t word = 0;
  if (o < 2 * B) {
    const float sg = sigma[c];
#pragma unroll
    for (int bt = 0; bt < 4; ++bt) {
      const int i = st * kStageIn + 16 * q + 4 * (pw & 3) + bt;
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
  const long long n = static_cast<long long>(C) * S * 2 * b8::kRows * 32;
  b8::beam8_image_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
      w2, N, C, B, S, sigma, reinterpret_cast<uint32_t*>(wa));
  return cudaGetLastError();
}

}  // namespace xe
