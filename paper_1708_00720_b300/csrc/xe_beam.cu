// Phase-and-sum beamformer on 4+4-bit voltages (the DRX pipeline's GPU
// beamformer, section "LWA Sevilleta implementation", which works directly
// on the 4+4-bit samples):
//   y[t][c][b] = sum_i w[c][b][i] x[t][c][i]
//
// This file holds the beamformer's C ABI, which sends up to 16 beams over up
// to 512 inputs to the e4m3 kernel of xe_beam8.cu (voltages in tensor
// memory, weight terms resident in shared memory), and the float16 kernel
// below for every other shape.
//
// Per channel this is a complex matrix product Y (T x B) = X (T x N) W^T,
// written as one real product on the tcgen05 tensor cores (kind::f16):
//   [Y_re | Y_im] = [X_re | X_im] . [[ W_re,  W_im],
//                                    [-W_im,  W_re]]^T
// with M = 128 time samples per unit, N_mma = 2B output columns and
// K = 2 x 64 inputs per pipeline stage (a real-part atom and an
// imaginary-part atom of the operand).
//
// Operand encoding.  A voltage nibble v in [-8, 7] becomes u = v + 8 =
// nibble XOR 8, stored as the float16 bit pattern u, i.e. the subnormal
// u * 2^-24 (exact; one lop3 per 4 samples).  The weights are float16
// (normal).  So D = 2^-24 sum_k W'[n][k] u_k and
//   y_n = 2^24 D_n - 8 sum_k W'[n][k],
// one FFMA per output with a per-(channel, column) bias computed when the
// weights are set.  Padded inputs (N not a multiple of 64) have zero weights;
// samples past T are zero-filled by TMA and their rows are not written.
//
// Weights (operand B): K-major with the 128-byte swizzle: row r of an atom
// (64 float16 of K) at (r / 8) * 1024 + (r % 8) * 128, its 16-byte chunk j at
// position j XOR (r % 8); the descriptor start advances 32 bytes per K = 16
// step inside an atom.  The weights are stored in global memory already in
// this layout, one contiguous 2 x 2B x 128-byte block per (channel, stage),
// consecutive stages adjacent, so a group of stages is one bulk copy.
//
// Data path per CTA (persistent, contiguous range of (channel, time tile)
// units, 480 threads):
//   warp 0       raw producer: one TMA copy per 4 stages (128 samples x 256
//                inputs = 32 KB, laid out as four [128][64-byte] tiles with
//                the 64-byte swizzle)
//   warp 1       MMA issuer (one thread): 8 MMAs per stage, D double-buffered
//   warp 2       weight producer: one bulk copy per group of up to 4 stages
//   warps 3-10   unpack, two warps per tensor-memory lane quadrant: each
//                thread converts 32 inputs of its own time row and writes
//                them into operand A in tensor memory (tcgen05.st)
//   warps 11-14  epilogue: tcgen05.ld, bias, complex64 rows to global memory
// Operand A lives in tensor memory (lane = time row, column c = the float16
// pair k = 2c, 2c + 1; real parts in the stage's first 32 columns), so the
// 4-byte-per-sample operand never passes through shared memory, whose
// bandwidth it would otherwise saturate.  (A thread issues about one bulk
// copy per ~800 cycles, so copies are few and large, from two warps.)
// Every wait is bounded; on timeout the kernel records an error and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_kernels.h"
#include "xe_ptx.cuh"

namespace xe {
namespace bm {

constexpr int kTile = 128;                 // time samples per unit (MMA M)
constexpr int kChunk = 64;                 // inputs per K stage
constexpr int kSubStage = kTile * kChunk;  // 8 KB of raw bytes: [128 t][64 inputs], 64-byte swizzle
constexpr int kSub = 4;                    // K stages per raw copy
constexpr int kRawStage = kSub * kSubStage;   // 32 KB
constexpr int kRaw = 3;
constexpr int kOpMax = 7;                  // operand-A stages in tensor memory, 64 columns each
constexpr int kW = 2;
constexpr int kWResident = 96 * 1024;      // a channel's weights this small stay in shared memory
constexpr int kRawWarp = 0, kMmaWarp = 1, kWWarp = 2;
constexpr int kUnpackWarp0 = 3, kUnpackWarps = 8;        // two per TMEM lane quadrant
constexpr int kEpiWarp0 = kUnpackWarp0 + kUnpackWarps;   // 4 epilogue warps, one per TMEM lane quadrant
constexpr int kThreads = 32 * (kEpiWarp0 + 4);

enum ErrCode : int {
  kErrRawFull = 1 << 0, kErrRawEmpty = 1 << 1, kErrOpFull = 1 << 2, kErrOpEmpty = 1 << 3,
  kErrWFull = 1 << 4, kErrAccFull = 1 << 5, kErrAccEmpty = 1 << 6, kErrFinal = 1 << 7, kErrWEmpty = 1 << 8,
};

__host__ __device__ constexpr int w_stage_bytes(int B) { return 2 * (2 * B) * 128; }
// weights of up to 4 stages per bulk copy, at most 32 KB
__host__ __device__ constexpr int w_group(int B) {
  return w_stage_bytes(B) >= 32768 ? 1 : (32768 / w_stage_bytes(B) >= 4 ? 4 : 32768 / w_stage_bytes(B));
}
__host__ __device__ constexpr int w_slot_bytes(int B) { return w_group(B) * w_stage_bytes(B); }
// D occupies tensor-memory columns [0, 4B) (two accumulators of 2B); operand-A
// stages fill the rest of the 512 columns in 64-column steps.
__host__ __device__ constexpr int a_col0(int B) { return (4 * B + 63) / 64 * 64; }
__host__ __device__ constexpr int op_stages(int B) {
  return (512 - a_col0(B)) / 64 < kOpMax ? (512 - a_col0(B)) / 64 : kOpMax;
}
// Resident weights: one buffer with all S stages of a channel, loaded when the
// channel changes.  Otherwise: kW slots of w_group(B) stages, streamed.
__host__ __device__ constexpr bool w_resident(int S, int B) { return S * w_stage_bytes(B) <= kWResident; }
__host__ __device__ constexpr int w_region_bytes(int S, int B) {
  return w_resident(S, B) ? S * w_stage_bytes(B) : kW * w_slot_bytes(B);
}

struct Smem {
  uint8_t* w;      // resident: [S][w_stage_bytes]; streamed: [kW][w_slot_bytes]
  uint8_t* raw;    // [kRaw][kRawStage]
  uint64_t *raw_full, *raw_empty, *op_full, *op_empty, *w_full, *w_empty, *acc_full, *acc_empty, *fin;
  uint32_t* tmem_slot;
  int* abort_flag;
};

__host__ __device__ inline int smem_bytes(int S, int B) {
  return (w_region_bytes(S, B) + 1023) / 1024 * 1024 + kRaw * kRawStage + (2 * kRaw + 2 * kOpMax + 2 * kW + 5) * 8 +
         16 + 1024;
}

__device__ inline Smem carve(uint8_t* base, int S, int B) {
  Smem s;
  s.w = base;
  s.raw = s.w + (w_region_bytes(S, B) + 1023) / 1024 * 1024;
  uint64_t* b = reinterpret_cast<uint64_t*>(s.raw + kRaw * kRawStage);
  s.raw_full = b; b += kRaw;
  s.raw_empty = b; b += kRaw;
  s.op_full = b; b += kOpMax;
  s.op_empty = b; b += kOpMax;
  s.w_full = b; b += kW;
  s.w_empty = b; b += kW;
  s.acc_full = b; b += 2;
  s.acc_empty = b; b += 2;
  s.fin = b; b += 1;
  s.tmem_slot = reinterpret_cast<uint32_t*>(b);
  s.abort_flag = reinterpret_cast<int*>(b) + 1;
  return s;
}

// K-major, 128-byte-swizzle shared-memory descriptor (8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= 1ull << 16;                                     // leading byte offset: unused when swizzled
  d |= static_cast<uint64_t>(1024 >> 4) << 32;         // stride byte offset
  d |= 1ull << 46;                                     // descriptor version for tcgen05
  d |= 2ull << 61;                                     // SWIZZLE_128B
  return d;
}
// kind::f16, D = f32, A = B = f16, both K-major.
__host__ __device__ constexpr uint32_t idesc_k_f16(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// D += A B^T with A (128 rows x K = 16) in tensor memory: lane = row, column c
// holds the float16 pair (k = 2c, 2c + 1) in its (low, high) halves.
__device__ __forceinline__ void mma_f16_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
               ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* smem_dst, const void* desc, uint64_t* bar, int x, int y, int z,
                                            int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cta.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];"
      ::"r"(smem_u32(smem_dst)), "l"(reinterpret_cast<uint64_t>(desc)), "r"(smem_u32(bar)), "r"(x), "r"(y),
        "r"(z), "r"(w)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// 32 lanes x 16 consecutive 32-bit columns: thread `lane` writes row (lane
// quadrant base + lane).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
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

// Position in a ring of n barrier-guarded slots: the slot, the parity of the
// slot's current fill, and whether every slot has been used once (from then on
// a producer must wait for the previous use of its slot to be released).
struct Ring {
  int n, slot = 0;
  uint32_t phase = 0;
  bool wrapped = false;
  __device__ explicit Ring(int n_) : n(n_) {}
  __device__ __forceinline__ void next() {
    if (++slot == n) {
      slot = 0;
      phase ^= 1u;
      wrapped = true;
    }
  }
};

__device__ __forceinline__ void fail(const Smem& s, int* err, int code) {
  atomicExch(s.abort_flag, 1);
  atomicOr(err, code);
}

// Four samples (one 32-bit word of raw bytes) -> biased float16 bit patterns:
// re0 = (u_re(s0), u_re(s1)), re1 = (u_re(s2), u_re(s3)); same for im.
__device__ __forceinline__ void unpack4(uint32_t x, uint32_t& re0, uint32_t& re1, uint32_t& im0, uint32_t& im1) {
  const uint32_t hi = ((x >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
  const uint32_t lo = (x & 0x0F0F0F0Fu) ^ 0x08080808u;
  re0 = __byte_perm(hi, 0u, 0x4140);
  re1 = __byte_perm(hi, 0u, 0x4342);
  im0 = __byte_perm(lo, 0u, 0x4140);
  im1 = __byte_perm(lo, 0u, 0x4342);
}

__global__ void __launch_bounds__(kThreads, 1)
beam_kernel(const __grid_constant__ CUtensorMap tmap, const BeamParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Smem s = carve(base, p.S, p.B);
  const int R = 2 * p.B;                 // MMA N: real then imaginary output columns
  const int kOp = op_stages(p.B), acol0 = a_col0(p.B);
  const bool resident = w_resident(p.S, p.B);
  const int wbytes = w_stage_bytes(p.B);
  const int gw = resident ? p.S : w_group(p.B);   // stages per weight copy
  const int wslot = resident ? 0 : w_slot_bytes(p.B);
  const int SS = (p.S + kSub - 1) / kSub;    // raw copies per unit
  const int G = (p.S + gw - 1) / gw;         // weight copies per unit (streamed)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long units = static_cast<long long>(p.C) * p.tiles;
  const long long u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  const uint64_t lim = p.timeout_ns;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kRaw; ++i) {
      mbar_init(&s.raw_full[i], 1);
      mbar_init(&s.raw_empty[i], kUnpackWarps);
    }
    for (int i = 0; i < kOpMax; ++i) {
      mbar_init(&s.op_full[i], kUnpackWarps);
      mbar_init(&s.op_empty[i], 1);
    }
    for (int i = 0; i < kW; ++i) {
      mbar_init(&s.w_full[i], 1);
      mbar_init(&s.w_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&s.acc_full[i], 1);
      mbar_init(&s.acc_empty[i], 4);
    }
    mbar_init(s.fin, 1);
    *s.abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc<512>(s.tmem_slot);   // D: columns [0, 4B); operand-A stages above a_col0(B)
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_slot;

  if (warp == kRawWarp) {
    // ------------------------------------------------------------ raw producer
    if (lane == 0) {
      tma_prefetch_desc(&tmap);
      long long h = 0;
      Ring rr(kRaw);
      for (long long u = u0; u < u1; ++u) {
        const int c = static_cast<int>(u / p.tiles), t0 = static_cast<int>(u % p.tiles) * kTile;
        bool ok = true;
        for (int ss = 0; ss < SS; ++ss, ++h, rr.next()) {
          const int rs = rr.slot;
          if (rr.wrapped && !wait_or_abort(&s.raw_empty[rs], rr.phase ^ 1u, lim, s.abort_flag)) {
            if (!*s.abort_flag) fail(s, p.err, kErrRawEmpty);
            ok = false;
            break;
          }
          uint8_t* dst = s.raw + rs * kRawStage;
          if (p.map4) {
            mbar_arrive_expect_tx(&s.raw_full[rs], kRawStage);
            tma_load_4d(dst, &tmap, &s.raw_full[rs], 0, t0, ss * kSub, c);
          } else {
            const int nsub = min(kSub, p.S - ss * kSub);
            mbar_arrive_expect_tx(&s.raw_full[rs], nsub * kSubStage);
            for (int k = 0; k < nsub; ++k)
              tma_load_3d(dst + k * kSubStage, &tmap, &s.raw_full[rs], (ss * kSub + k) * kChunk, c, t0);
          }
        }
        if (!ok) break;
      }
      // every copy issued has landed before the CTA may exit
      for (long long k = h - 1; k >= 0 && k >= h - kRaw; --k)
        mbar_wait(&s.raw_full[k % kRaw], static_cast<uint32_t>((k / kRaw) & 1), lim);
    }
  } else if (warp == kWWarp) {
    // ------------------------------------------------------------ weight producer
    // Streamed: G copies per unit into kW slots.  Resident: one copy of the
    // whole channel into the single buffer whenever the channel changes
    // (the MMA thread releases it after the last stage of a channel).
    if (lane == 0) {
      long long v = 0;
      int prev_c = -1;
      Ring wr(resident ? 1 : kW);
      for (long long u = u0; u < u1; ++u) {
        const int c = static_cast<int>(u / p.tiles);
        if (resident && c == prev_c) continue;
        prev_c = c;
        bool ok = true;
        for (int gi = 0; gi < G; ++gi, ++v, wr.next()) {
          const int ws = wr.slot;
          if (wr.wrapped && !wait_or_abort(&s.w_empty[ws], wr.phase ^ 1u, lim, s.abort_flag)) {
            if (!*s.abort_flag) fail(s, p.err, kErrWEmpty);
            ok = false;
            break;
          }
          const int nst = min(gw, p.S - gi * gw);
          mbar_arrive_expect_tx(&s.w_full[ws], nst * wbytes);
          bulk_load(s.w + ws * wslot, p.wt + (static_cast<long long>(c) * p.S + gi * gw) * (wbytes / 2),
                    nst * wbytes, &s.w_full[ws]);
        }
        if (!ok) break;
      }
      const int nslot = resident ? 1 : kW;
      for (long long k = v - 1; k >= 0 && k >= v - nslot; --k)
        mbar_wait(&s.w_full[resident ? 0 : k % kW], static_cast<uint32_t>((k / nslot) & 1), lim);
    }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_k_f16(kTile, R);
      long long j = 0;
      bool ok = true;
      int prev_c = -1;
      Ring opr(kOp), wr(resident ? 1 : kW);
      for (long long u = u0; u < u1 && ok; ++u, ++j) {
        const int ab = static_cast<int>(j & 1);
        if (j >= 2 && !wait_or_abort(&s.acc_empty[ab], static_cast<uint32_t>((j / 2 - 1) & 1), lim, s.abort_flag)) {
          if (!*s.abort_flag) fail(s, p.err, kErrAccEmpty);
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + static_cast<uint32_t>(ab * R);
        const int c = static_cast<int>(u / p.tiles);
        const bool new_chan = c != prev_c;
        const bool last_of_chan = u + 1 == u1 || static_cast<int>((u + 1) / p.tiles) != c;
        prev_c = c;
        for (int st = 0; st < p.S; ++st, opr.next()) {
          const int os = opr.slot;
          const int ws = wr.slot;
          const bool need_w = resident ? (st == 0 && new_chan) : (st % gw == 0);
          if (need_w && !wait_or_abort(&s.w_full[ws], wr.phase, lim, s.abort_flag)) {
            if (!*s.abort_flag) fail(s, p.err, kErrWFull);
            ok = false;
            break;
          }
          if (!wait_or_abort(&s.op_full[os], opr.phase, lim, s.abort_flag)) {
            if (!*s.abort_flag) fail(s, p.err, kErrOpFull);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = tmem + static_cast<uint32_t>(acol0 + 64 * os);
          const uint32_t w0 = smem_u32(s.w + ws * wslot + (st % gw) * wbytes);
#pragma unroll
          for (int at = 0; at < 2; ++at)
#pragma unroll
            for (int k = 0; k < 4; ++k)
              mma_f16_tmem_a(d, a0 + 32 * at + 8 * k, sdesc_k_sw128(w0 + at * (R * 128) + 32 * k), idesc,
                             (st | at | k) != 0 ? 1u : 0u);
          mma_commit(&s.op_empty[os]);
          const bool w_done = resident ? (st == p.S - 1 && last_of_chan) : (st % gw == gw - 1 || st == p.S - 1);
          if (w_done) {   // these weights are no longer needed
            mma_commit(&s.w_empty[ws]);
            wr.next();
          }
        }
        if (!ok) break;
        mma_commit(&s.acc_full[ab]);
      }
      // all MMAs of this thread have completed before TMEM is freed
      mma_commit(s.fin);
      if (!mbar_wait(s.fin, 0, lim)) atomicOr(p.err, kErrFinal);
    }
  } else if (warp < kEpiWarp0) {
    // ------------------------------------------------------------ unpack
    // warp -> TMEM lane quadrant q (rows 32 q .. 32 q + 31) and half h of a
    // stage's 64 inputs; each thread converts 32 inputs of its own row.
    const int q = warp & 3, hf = (warp - kUnpackWarp0) / 4;
    const int t = 32 * q + lane;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(32 * q) << 16);
    Ring rr(kRaw), opr(kOp);
    bool ok = true;
    for (long long u = u0; u < u1 && ok; ++u) {
      for (int ss = 0; ss < SS && ok; ++ss, rr.next()) {
        const int rs = rr.slot;
        if (!wait_or_abort(&s.raw_full[rs], rr.phase, lim, s.abort_flag)) {
          if (!*s.abort_flag) fail(s, p.err, kErrRawFull);
          ok = false;
          break;
        }
        const int nsub = min(kSub, p.S - ss * kSub);
        for (int sub = 0; sub < nsub; ++sub, opr.next()) {
          const int os = opr.slot;
          if (opr.wrapped && !wait_or_abort(&s.op_empty[os], opr.phase ^ 1u, lim, s.abort_flag)) {
            if (!*s.abort_flag) fail(s, p.err, kErrOpEmpty);
            ok = false;
            break;
          }
          // row t of the 64-byte-swizzled tile: 16-byte chunk c sits at c XOR ((t >> 1) & 3)
          const uint8_t* row = s.raw + rs * kRawStage + sub * kSubStage + t * kChunk;
          const int sw = (t >> 1) & 3;
          const uint4 x0 = *reinterpret_cast<const uint4*>(row + (((2 * hf) ^ sw) << 4));
          const uint4 x1 = *reinterpret_cast<const uint4*>(row + (((2 * hf + 1) ^ sw) << 4));
          uint32_t re[16], im[16];
          unpack4(x0.x, re[0], re[1], im[0], im[1]);
          unpack4(x0.y, re[2], re[3], im[2], im[3]);
          unpack4(x0.z, re[4], re[5], im[4], im[5]);
          unpack4(x0.w, re[6], re[7], im[6], im[7]);
          unpack4(x1.x, re[8], re[9], im[8], im[9]);
          unpack4(x1.y, re[10], re[11], im[10], im[11]);
          unpack4(x1.z, re[12], re[13], im[12], im[13]);
          unpack4(x1.w, re[14], re[15], im[14], im[15]);
          const uint32_t a = lane_base + static_cast<uint32_t>(acol0 + 64 * os + 16 * hf);
          tmem_st16(a, re);          // real parts: K columns 0 .. 31 of the stage
          tmem_st16(a + 32, im);     // imaginary parts: K columns 32 .. 63
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&s.op_full[os]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.raw_empty[rs]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                  // TMEM lane quadrant of this warp
    long long j = 0;
    for (long long u = u0; u < u1; ++u, ++j) {
      const int ab = static_cast<int>(j & 1);
      if (!wait_or_abort(&s.acc_full[ab], static_cast<uint32_t>((j / 2) & 1), lim, s.abort_flag)) {
        if (!*s.abort_flag) fail(s, p.err, kErrAccFull);
        break;
      }
      tc_fence_after();
      const int c = static_cast<int>(u / p.tiles), t = static_cast<int>(u % p.tiles) * kTile + 32 * q + lane;
      const float* bias = p.bias + static_cast<long long>(c) * R;
      float4* dst = reinterpret_cast<float4*>(p.out + (static_cast<long long>(t) * p.C + c) * p.B * 2);
      const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(ab * R);
      for (int b0 = 0; b0 < p.B; b0 += 16) {
        uint32_t re[16], im[16];
        const int nb = p.B - b0 < 16 ? p.B - b0 : 16;   // B is a multiple of 8
        tmem_ld16(taddr + b0, re);
        tmem_ld16(taddr + p.B + b0, im);
        tmem_ld_wait();
        if (t < p.T) {
#pragma unroll
          for (int k = 0; k < 16; k += 2) {
            if (k < nb) {
              float4 v;
              v.x = fmaf(__uint_as_float(re[k]), 16777216.0f, -bias[b0 + k]);
              v.y = fmaf(__uint_as_float(im[k]), 16777216.0f, -bias[p.B + b0 + k]);
              v.z = fmaf(__uint_as_float(re[k + 1]), 16777216.0f, -bias[b0 + k + 1]);
              v.w = fmaf(__uint_as_float(im[k + 1]), 16777216.0f, -bias[p.B + b0 + k + 1]);
              dst[(b0 + k) >> 1] = v;
            }
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

// Weights -> operand tiles and biases.  One thread per (channel, column n,
// input i): column n < B is the real output of beam n (W' = Re w on the
// real-part atom, -Im w on the imaginary-part atom), column B + b the
// imaginary output of beam b (Im w, Re w).
__global__ void beam_weights_kernel(const float2* __restrict__ w, int N, int C, int B, int S,
                                    uint16_t* __restrict__ wt) {
  const int R = 2 * B, Np = S * kChunk;
  const long long idx = blockIdx.x * 256LL + threadIdx.x;
  if (idx >= static_cast<long long>(C) * R * Np) return;
  const int i = static_cast<int>(idx % Np);
  const int n = static_cast<int>((idx / Np) % R);
  const int c = static_cast<int>(idx / (static_cast<long long>(Np) * R));
  const int b = n < B ? n : n - B;
  float2 v = make_float2(0.f, 0.f);
  if (i < N) v = w[(static_cast<long long>(c) * B + b) * N + i];
  const float on_re = n < B ? v.x : v.y;    // multiplies the real part of x
  const float on_im = n < B ? -v.y : v.x;   // multiplies the imaginary part of x
  const int st = i / kChunk, kk = i % kChunk;
  const int off = (n >> 3) * 1024 + (n & 7) * 128 + ((((kk >> 3) ^ (n & 7)) << 4)) + (kk & 7) * 2;
  uint8_t* blk = reinterpret_cast<uint8_t*>(wt) + (static_cast<long long>(c) * S + st) * w_stage_bytes(B);
  *reinterpret_cast<uint16_t*>(blk + off) = __half_as_ushort(__float2half_rn(on_re));
  *reinterpret_cast<uint16_t*>(blk + R * 128 + off) = __half_as_ushort(__float2half_rn(on_im));
}

// bias[c][n] = 8 * (sum over the column's operand values), from the rounded
// float16 values, summed in float64.
__global__ void beam_bias_kernel(const uint16_t* __restrict__ wt, int C, int B, int S, float* __restrict__ bias) {
  const int R = 2 * B;
  const long long idx = blockIdx.x * 256LL + threadIdx.x;
  if (idx >= static_cast<long long>(C) * R) return;
  const int n = static_cast<int>(idx % R), c = static_cast<int>(idx / R);
  double acc = 0.0;
  for (int st = 0; st < S; ++st) {
    const uint8_t* blk = reinterpret_cast<const uint8_t*>(wt) + (static_cast<long long>(c) * S + st) * w_stage_bytes(B);
    for (int at = 0; at < 2; ++at)
      for (int kk = 0; kk < kChunk; ++kk) {
        const int off = (n >> 3) * 1024 + (n & 7) * 128 + ((((kk >> 3) ^ (n & 7)) << 4)) + (kk & 7) * 2;
        acc += static_cast<double>(__half2float(__ushort_as_half(*reinterpret_cast<const uint16_t*>(blk + at * R * 128 + off))));
      }
  }
  bias[idx] = static_cast<float>(8.0 * acc);
}

}  // namespace bm

int beam_smem_bytes(int S, int B) { return bm::smem_bytes(S, B); }
int beam_w_group(int B) { return bm::w_group(B); }
int beam_threads() { return bm::kThreads; }

cudaError_t launch_beam(const CUtensorMap* tmap, const BeamParams& prm, int grid, cudaStream_t stream) {
  const int smem = bm::smem_bytes(prm.S, prm.B);
  cudaError_t e = cudaFuncSetAttribute(bm::beam_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  bm::beam_kernel<<<grid, bm::kThreads, smem, stream>>>(*tmap, prm);
  return cudaGetLastError();
}

cudaError_t launch_beam_weights(const float* w, int N, int C, int B, int S, uint16_t* wt, float* bias,
                                cudaStream_t stream) {
  const long long n = static_cast<long long>(C) * 2 * B * S * bm::kChunk;
  bm::beam_weights_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
      reinterpret_cast<const float2*>(w), N, C, B, S, wt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long nb = static_cast<long long>(C) * 2 * B;
  bm::beam_bias_kernel<<<static_cast<unsigned>((nb + 255) / 256), 256, 0, stream>>>(wt, C, B, S, bias);
  return cudaGetLastError();
}

}  // namespace xe

// ------------------------------------------------------------------ C ABI
#include <new>
#include <string>

#include "xengine.h"

struct xe_beam {
  int N = 0, C = 0, B = 0, S = 0, max_ntime = 0;
  int num_sms = 0;
  bool weights_set = false;
  // the e4m3 kernel (xe_beam8.cu) when B <= 16 and N <= 512, else the float16 one
  bool e4m3 = false;
  int S8 = 0;                   // 128-input stages of the e4m3 kernel
  uint16_t* d_wt = nullptr;     // float16 kernel: operand tiles
  float* d_bias = nullptr;      // [C][2B] (float16 kernel) or [C][32] (e4m3 kernel)
  uint8_t* d_wa = nullptr;      // e4m3 kernel: weight-term images (operand B)
  float* d_sigma = nullptr;     // e4m3 kernel: per-channel weight scale
  float* d_osc = nullptr;       // e4m3 kernel: 2^9 / sigma
  int* d_err = nullptr;
  long long launches = 0;
  std::string last_error;
};

namespace {
constexpr unsigned long long kBeamTimeoutNs = 2000000000ull;
bool aligned_to(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// One gulp through the e4m3 kernel (validated arguments).
xe_status form_e4m3(xe_beam* b, const uint8_t* d_gulp, int ntime, float* d_out, cudaStream_t stream) {
  CUtensorMap map;
  const unsigned long long dims[3] = {static_cast<unsigned long long>(b->N), static_cast<unsigned long long>(b->C),
                                      static_cast<unsigned long long>(ntime)};
  const unsigned long long strides[2] = {static_cast<unsigned long long>(b->N),
                                         static_cast<unsigned long long>(b->N) * b->C};
  const unsigned box[3] = {128, 1, 128};
  if (!xe::encode_tensor_u8(&map, d_gulp, 3, dims, strides, box, 128)) {
    b->last_error = "cuTensorMapEncodeTiled failed";
    return XE_ERR_CUDA;
  }
  xe::Beam8Params prm;
  prm.N = b->N;
  prm.C = b->C;
  prm.B = b->B;
  prm.S = b->S8;
  prm.T = ntime;
  prm.tiles = (ntime + 127) / 128;
  prm.wa = b->d_wa;
  prm.osc = b->d_osc;
  prm.bias = b->d_bias;
  prm.out = d_out;
  prm.err = b->d_err;
  prm.timeout_ns = kBeamTimeoutNs;
  const long long units = static_cast<long long>(b->C) * prm.tiles;
  const int grid = static_cast<int>(units < b->num_sms ? units : b->num_sms);
  const cudaError_t e = xe::launch_beam8(&map, prm, grid, stream);
  if (e != cudaSuccess) {
    b->last_error = std::string("beam launch: ") + cudaGetErrorString(e);
    return XE_ERR_CUDA;
  }
  ++b->launches;
  return XE_OK;
}
}  // namespace

extern "C" {

XE_API xe_status xe_beam_create(xe_beam_t* out, int n_input, int n_chan, int n_beam, int max_ntime) {
  if (!out) return XE_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_input < 1 || n_input > 65536 || n_chan < 1 || max_ntime < 1 || n_beam < 8 || n_beam > 64 ||
      n_beam % 8 != 0)
    return XE_ERR_INVALID_ARG;
  if (n_input % 16 != 0) return XE_ERR_ALIGNMENT;   // TMA row stride: a multiple of 16 bytes
  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return XE_ERR_CUDA;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (major != 10 || minor != 3) return XE_ERR_DEVICE_UNSUPPORTED;
  xe_beam* b = new (std::nothrow) xe_beam();
  if (!b) return XE_ERR_NOMEM;
  b->N = n_input;
  b->C = n_chan;
  b->B = n_beam;
  b->S = (n_input + 63) / 64;
  b->max_ntime = max_ntime;
  b->num_sms = sms;
  b->e4m3 = n_beam <= 16 && n_input <= 512;
  b->S8 = (n_input + 127) / 128;
  bool ok = true;
  if (b->e4m3) {
    ok = cudaMalloc(&b->d_wa, static_cast<size_t>(n_chan) * 128 * 256 * b->S8) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_sigma, static_cast<size_t>(n_chan) * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_osc, static_cast<size_t>(n_chan) * sizeof(float)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_bias, static_cast<size_t>(n_chan) * 32 * sizeof(float)) == cudaSuccess;
  } else {
    const size_t wt_bytes = static_cast<size_t>(n_chan) * b->S * xe::bm::w_stage_bytes(n_beam);
    ok = cudaMalloc(&b->d_wt, wt_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_bias, static_cast<size_t>(n_chan) * 2 * n_beam * sizeof(float)) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&b->d_err, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMemset(b->d_err, 0, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFree(b->d_wt);
    cudaFree(b->d_bias);
    cudaFree(b->d_wa);
    cudaFree(b->d_sigma);
    cudaFree(b->d_osc);
    cudaFree(b->d_err);
    delete b;
    return XE_ERR_NOMEM;
  }
  *out = b;
  return XE_OK;
}

XE_API xe_status xe_beam_destroy(xe_beam_t b) {
  if (!b) return XE_OK;
  cudaDeviceSynchronize();
  cudaFree(b->d_wt);
  cudaFree(b->d_bias);
  cudaFree(b->d_wa);
  cudaFree(b->d_sigma);
  cudaFree(b->d_osc);
  cudaFree(b->d_err);
  delete b;
  return XE_OK;
}

XE_API xe_status xe_beam_set_weights(xe_beam_t b, const float* d_w, void* stream) {
  if (!b || !d_w) return XE_ERR_INVALID_ARG;
  if (!aligned_to(d_w, 8)) return XE_ERR_ALIGNMENT;
  const cudaError_t e =
      b->e4m3 ? xe::launch_beam8_weights(d_w, b->N, b->C, b->B, b->S8, b->d_wa, b->d_sigma, b->d_osc, b->d_bias,
                                           static_cast<cudaStream_t>(stream))
                : xe::launch_beam_weights(d_w, b->N, b->C, b->B, b->S, b->d_wt, b->d_bias,
                                          static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    b->last_error = "weight conversion launch failed";
    return XE_ERR_CUDA;
  }
  b->weights_set = true;
  return XE_OK;
}

XE_API xe_status xe_beam_form(xe_beam_t b, const uint8_t* d_gulp, int ntime, float* d_out, void* stream) {
  if (!b || ntime < 0 || ntime > b->max_ntime || !b->weights_set) return XE_ERR_INVALID_ARG;
  if (ntime == 0) return XE_OK;
  if (!d_gulp || !d_out) return XE_ERR_INVALID_ARG;
  if (!aligned_to(d_gulp, 16) || !aligned_to(d_out, 16)) return XE_ERR_ALIGNMENT;
  if (b->e4m3) return form_e4m3(b, d_gulp, ntime, d_out, static_cast<cudaStream_t>(stream));
  CUtensorMap map;
  const bool map4 = b->N % 64 == 0;   // whole 64-input chunks: one copy per 4 stages
  bool enc;
  if (map4) {
    // {64 inputs of a chunk, time, chunk, channel}: box {64, 128, 4, 1} lands as four [128][64] tiles
    const unsigned long long dims[4] = {64, static_cast<unsigned long long>(ntime),
                                        static_cast<unsigned long long>(b->S), static_cast<unsigned long long>(b->C)};
    const unsigned long long strides[3] = {static_cast<unsigned long long>(b->N) * b->C, 64,
                                           static_cast<unsigned long long>(b->N)};
    const unsigned box[4] = {64, 128, 4, 1};
    enc = xe::encode_tensor_u8(&map, d_gulp, 4, dims, strides, box, 64);
  } else {
    const unsigned long long dims[3] = {static_cast<unsigned long long>(b->N), static_cast<unsigned long long>(b->C),
                                        static_cast<unsigned long long>(ntime)};
    const unsigned long long strides[2] = {static_cast<unsigned long long>(b->N),
                                           static_cast<unsigned long long>(b->N) * b->C};
    const unsigned box[3] = {64, 1, 128};
    enc = xe::encode_tensor_u8(&map, d_gulp, 3, dims, strides, box, 64);
  }
  if (!enc) {
    b->last_error = "cuTensorMapEncodeTiled failed";
    return XE_ERR_CUDA;
  }
  xe::BeamParams prm;
  prm.N = b->N;
  prm.C = b->C;
  prm.B = b->B;
  prm.S = b->S;
  prm.T = ntime;
  prm.tiles = (ntime + 127) / 128;
  prm.wt = b->d_wt;
  prm.bias = b->d_bias;
  prm.out = d_out;
  prm.err = b->d_err;
  prm.timeout_ns = kBeamTimeoutNs;
  prm.map4 = map4 ? 1 : 0;
  const long long units = static_cast<long long>(b->C) * prm.tiles;
  const int grid = static_cast<int>(units < b->num_sms ? units : b->num_sms);
  const cudaError_t e = xe::launch_beam(&map, prm, grid, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    b->last_error = std::string("beam launch: ") + cudaGetErrorString(e);
    return XE_ERR_CUDA;
  }
  ++b->launches;
  return XE_OK;
}

XE_API xe_status xe_beam_check(xe_beam_t b) {
  if (!b) return XE_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return XE_ERR_CUDA;
  int err = 0;
  if (cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return XE_ERR_CUDA;
  if (err) {
    b->last_error = "device wait timed out (code " + std::to_string(err) + ")";
    cudaMemset(b->d_err, 0, sizeof(int));
    return XE_ERR_TIMEOUT;
  }
  return XE_OK;
}

XE_API const char* xe_beam_last_error(xe_beam_t b) { return b ? b->last_error.c_str() : ""; }

}  // extern "C"
