// tcgen05 X-engine, e4m3 operands, operand A fed from tensor memory.
//
// Computes, like every X-engine path here (the linear-algebra module of the
// paper's section "Back end" applied to the 4+4-bit samples of section
// "Packet capture implementation"),
//   V_c[i][j] = sum_t x[t][c][i] conj(x[t][c][j]),   i >= j,
// into an int32 accumulator [C][N(N+1)/2][2] (packed lower triangle).
//
// Why this layout.  On sm_103 the tensor core reads shared-memory operands
// through the same data pipe as ld/st.shared.  A 128 x 128 x 32 e4m3 MMA with
// both operands in shared memory needs about one pipe-width of bytes per
// clock by itself, so every byte the unpack warps move through shared memory
// steals tensor-core time.  Here the I tile (operand A) never touches the
// shared-memory operand path: it is transposed in registers and written to
// tensor memory with tcgen05.st; only the J tile (operand B) is staged in
// shared memory.  Per 32-sample step of a 128 x 128 tile pair the pipe moves
// ~32 KB instead of ~56 KB.
//
// Per step (32 samples) of a unit (channel c, 128-input tiles I >= J):
//  * TMA loads the raw 32 x 128-byte time x input tiles of I and J into
//    shared memory with the 128-byte swizzle.
//  * A side (one warp per TMEM lane quadrant): ldmatrix.x4.trans reads a
//    32-time x 16-input block as 16-bit pairs, four byte permutes regroup it
//    so that each 32-bit word holds four samples of one input, the nibbles
//    are split into biased e4m3 bytes (u = v + 8, exactly u * 2^-9) and
//    tcgen05.st.16x256b writes the re and im planes (K = 32 bytes per row).
//    Input 16g + 2p goes to TMEM lane 16g + p and input 16g + 2p + 1 to lane
//    16g + p + 8; the four samples of a word follow a fixed permutation of
//    time within the step (kappa below).
//  * B side: the J raw tile is split into biased re / im planes in shared
//    memory (MN-major, 128-byte swizzle), time row t stored at K row
//    kappa(t) so both operands agree on the order of K.
//  * MMA (one thread): D_re += A_re B_re^T + A_im B_im^T,
//                      D_im += A_im B_re^T - A_re B_im^T   (negate-B bit).
//  * Epilogue: D (single buffer, 256 TMEM columns) is drained through a
//    swizzled 128 KB shared staging buffer, the bias is removed exactly from
//    per-input sums of u, and rows are written coalesced to the accumulator:
//      Re V = D_re - 8 (P_i + Q_i + P_j + Q_j) + 128 T'
//      Im V = D_im + 8 (P_i - Q_i) - 8 (P_j - Q_j).
// Exactness: all partial sums of D stay below 450 T' <= 2^24 for T' <= 37282;
// the host splits longer gulps into launches of at most 32768 samples.  The
// number of 32-sample steps per launch is a multiple of 4 (TMA zero-fills the
// padding, which enters D, the sums and T' consistently).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_kernels.h"
#include "xe_ptx.cuh"

namespace xe {
namespace tc8 {

constexpr int kTile = 128;
constexpr int kStep = 32;                 // samples per MMA step (K = 32 e4m3)
constexpr int kSteps = 4;                 // steps per pipeline stage (128 samples)
constexpr int kRawSub = kStep * kTile;    // 4096 bytes: one step of one raw tile
constexpr int kRawTile = kSteps * kRawSub;  // 16 KB TMA box: 128 time rows x 128 inputs
constexpr int kPlane = kStep * kTile;     // one e4m3 plane (re or im) of one tile, one step
#ifndef XE_TC8_RAW_STAGES
#define XE_TC8_RAW_STAGES 2
#endif
#ifndef XE_TC8_OP_STAGES
#define XE_TC8_OP_STAGES 3
#endif
// Synchronisation happens once per stage of 4 steps: the tensor core's
// instruction queue holds only a few MMAs, so every barrier check or commit
// between MMAs costs issue bubbles, and each warp's wait-wake latency is a
// few hundred cycles.  Per stage the MMA thread issues 16 MMAs and one commit.
constexpr int kRawStages = XE_TC8_RAW_STAGES;
constexpr int kOpStages = XE_TC8_OP_STAGES;
// A warp that issues a TMA tile load is held for roughly 750 cycles per
// instruction on this part, whatever the box size, so raw tiles move in 16 KB
// boxes (one per stage) issued by two producer warps: warp 0 for I, warp 2 for J.
// Warp roles.  Warp w issues from SM sub-partition w % 4; the A-side and
// epilogue warps need one warp per TMEM lane quadrant (w % 4), and the MMA
// warp's sub-partition (1) carries one B-side warp instead of two.
//   0: TMA I tiles   1: MMA issuer   2: TMA J tiles   4-7: A side
//   3, 8, 10-15: B side   9: idle   16-19: epilogue
constexpr int kAWarp0 = 4;                // 4 A-side warps, one per TMEM lane quadrant
constexpr int kBWarps = 8;
constexpr int kEpiWarp0 = 16;             // 4 epilogue warps, one per quadrant
constexpr int kThreads = 32 * (kEpiWarp0 + 4);
// B-side warp -> its index 0..7, -1 for other roles
__device__ __forceinline__ int b_ordinal(int w) {
  return w == 3 ? 0 : (w == 8 ? 1 : (w >= 10 && w < 16 ? w - 8 : -1));
}
constexpr int kStageArrivals = 4 + kBWarps;   // A and B warps, once per stage
constexpr int kTmemCols = 512;
constexpr int kTmemA0 = 256;              // A stages: 64 columns each (4 steps x (re 8 + im 8))
constexpr int kTmemAStage = 16 * kSteps;

constexpr int kOpStage = kSteps * 2 * kPlane;   // B planes of 4 steps: [step][re, im][kPlane]
constexpr int kRawStage = 2 * kRawTile;         // I box, J box
constexpr int kOpBytes = kOpStages * kOpStage;
constexpr int kRawBytes = kRawStages * kRawStage;
constexpr int kStageBytes = 4 * 32 * 32 * 8;    // per epilogue warp: 32 rows x 32 int2
constexpr int kSumsBytes = 2 * 4 * kTile * 4 + 2 * kTile * 4 + kTile * 4;
// 2 slots x {P_I,Q_I,P_J,Q_J}, column corrections, per-row triangle offsets
constexpr int kBarOffset = kOpBytes + kRawBytes + kStageBytes + kSumsBytes;
constexpr int kNumBars = 2 * kRawStages + 2 * kOpStages + 2 + 2 + 2 + 1;
constexpr int kSmemBytes = kBarOffset + kNumBars * 8 + 16 + 1024;
static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
static_assert(kTmemA0 + kTmemAStage * kOpStages <= kTmemCols, "tensor memory budget");

enum ErrCode : int {
  kErrWaitRawFull = 1 << 0, kErrWaitRawEmpty = 1 << 1, kErrWaitOpFull = 1 << 2,
  kErrWaitOpEmpty = 1 << 3, kErrWaitAccFull = 1 << 4, kErrWaitAccEmpty = 1 << 5,
  kErrWaitSumsFull = 1 << 6, kErrWaitSumsEmpty = 1 << 7, kErrWaitFinal = 1 << 8,
};

struct Smem {
  uint8_t* op;     // [kOpStages][kSteps][2][kPlane]  B planes
  uint8_t* raw;    // [kRawStages][2][kRawTile]
  int2* stage;     // [4 warps][32 rows][32], column index XOR row
  int* sums;       // [2][4][128]
  float* colcorr;  // [2][128]: per-column bias corrections of the current unit (re, im)
  int* rowoff;     // [128]: packed-triangle offset i (i + 1) / 2 of each accumulator row's input i
  uint64_t *raw_full, *raw_empty, *op_full, *op_empty;
  uint64_t *acc_full, *acc_empty, *sums_full, *sums_empty, *final_bar;
  uint32_t* tmem_slot;
  int* abort_flag;
};

__device__ __forceinline__ Smem carve(uint8_t* base) {
  Smem p;
  p.op = base;
  p.raw = base + kOpBytes;
  p.stage = reinterpret_cast<int2*>(base + kOpBytes + kRawBytes);
  p.sums = reinterpret_cast<int*>(base + kOpBytes + kRawBytes + kStageBytes);
  p.colcorr = reinterpret_cast<float*>(p.sums + 2 * 4 * kTile);
  p.rowoff = reinterpret_cast<int*>(p.colcorr + 2 * kTile);
  uint64_t* b = reinterpret_cast<uint64_t*>(base + kBarOffset);
  p.raw_full = b; b += kRawStages;
  p.raw_empty = b; b += kRawStages;
  p.op_full = b; b += kOpStages;
  p.op_empty = b; b += kOpStages;
  p.acc_full = b; b += 1;
  p.acc_empty = b; b += 1;
  p.sums_full = b; b += 2;
  p.sums_empty = b; b += 2;
  p.final_bar = b; b += 1;
  p.tmem_slot = reinterpret_cast<uint32_t*>(b);
  p.abort_flag = reinterpret_cast<int*>(b) + 1;
  return p;
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

__device__ __forceinline__ void fail(const Smem& s, int* err, int code) {
  atomicExch(s.abort_flag, 1);
  atomicOr(err, code);
}

__device__ __forceinline__ void decode_unit(int u, int npairs, int& c, int& bi, int& bj) {
  c = u / npairs;
  const int p = u - c * npairs;
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
__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t& d0, uint32_t& d1, uint32_t& d2,
                                              uint32_t& d3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3) : "r"(addr) : "memory");
}
// .x2: the re plane (8 columns) and the im plane (the next 8) of one step in
// one instruction
__device__ __forceinline__ void tmem_st_16x256b_x2(uint32_t taddr, uint32_t r0, uint32_t r1, uint32_t r2,
                                                   uint32_t r3, uint32_t r4, uint32_t r5, uint32_t r6,
                                                   uint32_t r7) {
  asm volatile("tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               ::"r"(taddr), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(r4), "r"(r5), "r"(r6), "r"(r7)
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void mma_f8_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}"
               ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ uint32_t biased_re(uint32_t w) { return ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u; }
__device__ __forceinline__ uint32_t biased_im(uint32_t w) { return (w & 0x0F0F0F0Fu) ^ 0x08080808u; }
__device__ __forceinline__ int byte_sum(uint32_t w) { return static_cast<int>(__dp4a(w, 0x01010101u, 0u)); }

// K row of time sample t within a 32-sample step (the order the A-side
// register transpose produces): t = 8a + 2j + b  ->  8j + 2a + b.
__device__ __forceinline__ int kappa(int t) { return 8 * ((t & 7) >> 1) + 2 * (t >> 3) + (t & 1); }

// Byte offset of 16-byte chunk q of row k in a 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw128(int k, int q) {
  return static_cast<uint32_t>(k * 128 + ((q ^ (k & 7)) << 4));
}

// Accumulator row (TMEM lane) -> input offset inside the I tile.
__device__ __forceinline__ int lane_to_input(int L) {
  const int r = L & 15;
  return (L & ~15) + (r < 8 ? 2 * r : 2 * (r - 8) + 1);
}

// Per-thread sums of the biased J-side parts of 16 inputs (byte lanes,
// flushed into 16-bit lanes before they can overflow).
struct BSums {
  uint32_t b_re[4], b_im[4], h_re[8], h_im[8];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 4; ++k) b_re[k] = b_im[k] = 0u;
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
      b_re[k] = b_im[k] = 0u;
    }
  }
  __device__ __forceinline__ void publish(int* P, int* Q, int q) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
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

__global__ void __launch_bounds__(kThreads, 1)
xcorr_tc8_kernel(const __grid_constant__ CUtensorMap tmap, TcParams prm) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const Smem s = carve(base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npairs = prm.nt * (prm.nt + 1) / 2;
  const int nks = prm.nks;
  const uint64_t lim = prm.timeout_ns;
  volatile int* abort_flag = s.abort_flag;

  if (tid == 0) {
    for (int k = 0; k < kRawStages; ++k) {
      mbar_init(&s.raw_full[k], 2);   // the I-tile producer and the J-tile producer
      mbar_init(&s.raw_empty[k], kStageArrivals);
    }
    for (int k = 0; k < kOpStages; ++k) {
      mbar_init(&s.op_full[k], kStageArrivals);
      mbar_init(&s.op_empty[k], 1);
    }
    mbar_init(s.acc_full, 1);
    mbar_init(s.acc_empty, 4);
    for (int k = 0; k < 2; ++k) {
      mbar_init(&s.sums_full[k], kStageArrivals);
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

  if (warp == 0 || warp == 2) {
    // ====================================================== TMA producers
    if (lane == 0) {
      const int tile = warp >> 1;               // 0: I tiles, 1: J tiles
      int rit = 0;                              // raw stage counter (4 steps each)
      bool ok = true;
      for (int u = blockIdx.x; u < prm.units && ok; u += gridDim.x) {
        int c, bi, bj;
        decode_unit(u, npairs, c, bi, bj);
        const bool diag = (bi == bj);
        for (int ks = 0; ks < nks; ks += kSteps, ++rit) {
          const int st = rit % kRawStages;
          if (!wait_or_abort(&s.raw_empty[st], ((rit / kRawStages) & 1) ^ 1, lim, abort_flag)) {
            fail(s, prm.err, kErrWaitRawEmpty);
            ok = false;
            break;
          }
          uint8_t* dst = s.raw + st * kRawStage + tile * kRawTile;
          if (tile == 0) {
            mbar_arrive_expect_tx(&s.raw_full[st], kRawTile);
            tma_load_3d(dst, &tmap, &s.raw_full[st], bi * kTile, c, ks * kStep);
          } else if (!diag) {
            mbar_arrive_expect_tx(&s.raw_full[st], kRawTile);
            tma_load_3d(dst, &tmap, &s.raw_full[st], bj * kTile, c, ks * kStep);
          } else {
            mbar_arrive(&s.raw_full[st]);    // diagonal unit: the I tile serves both operands
          }
        }
      }
      // wait for the copies still in flight (normally all consumed already)
      for (int k = rit - 1; k >= 0 && k > rit - 1 - kRawStages; --k)
        mbar_wait(&s.raw_full[k % kRawStages], (k / kRawStages) & 1, lim);
    }
  } else if (warp == 1) {
    // ====================================================== MMA issuer
    if (lane == 0) {
      int sit = 0, ui = 0;
      bool ok = true;
      // A from tensor memory (K-major), B MN-major; e4m3 x e4m3 -> f32, M = N = 128
      constexpr uint32_t id_pos = (1u << 4) | (1u << 16) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
      constexpr uint32_t id_neg = id_pos | (1u << 14);
      const uint32_t d_re = tmem, d_im = tmem + 128;
      for (int u = blockIdx.x; u < prm.units && ok; u += gridDim.x, ++ui) {
        if (!wait_or_abort(s.acc_empty, (ui & 1) ^ 1, lim, abort_flag)) {
          fail(s, prm.err, kErrWaitAccEmpty);
          break;
        }
        tc_fence_after();
        for (int ks = 0; ks < nks; ks += kSteps, ++sit) {
          const int st = sit % kOpStages;
          if (!wait_or_abort(&s.op_full[st], (sit / kOpStages) & 1, lim, abort_flag)) {
            fail(s, prm.err, kErrWaitOpFull);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = tmem + kTmemA0 + kTmemAStage * st;
          const uint32_t op = smem_u32(s.op + st * kOpStage);
#pragma unroll
          for (int sub = 0; sub < kSteps; ++sub) {
            const uint32_t a_re = a0 + 16 * sub, a_im = a_re + 8;
            const uint32_t b = op + sub * 2 * kPlane;
            const uint64_t b_re = sdesc_mn_sw128(b, 4096, 1024);
            const uint64_t b_im = sdesc_mn_sw128(b + kPlane, 4096, 1024);
            const uint32_t acc0 = (ks + sub) > 0 ? 1u : 0u;
            mma_f8_tmem_a(d_re, a_re, b_re, id_pos, acc0);
            mma_f8_tmem_a(d_re, a_im, b_im, id_pos, 1u);
            mma_f8_tmem_a(d_im, a_im, b_re, id_pos, acc0);
            mma_f8_tmem_a(d_im, a_re, b_im, id_neg, 1u);
          }
          mma_commit(&s.op_empty[st]);
        }
        if (!ok) break;
        mma_commit(s.acc_full);
      }
      mma_commit(s.final_bar);
      if (!mbar_wait(s.final_bar, 0, lim)) atomicOr(prm.err, kErrWaitFinal);
    }
  } else if (warp >= kAWarp0 && warp < kAWarp0 + 4) {
    // ====================================================== A side -> TMEM
    const int quad = warp & 3;                 // TMEM lane quadrant of this warp
    const int pj = lane >> 2;                  // input pair of this lane within a chunk
    int sit = 0, ui = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < prm.units && ok; u += gridDim.x, ++ui) {
      int aP[2][2] = {{0, 0}, {0, 0}}, aQ[2][2] = {{0, 0}, {0, 0}};  // [chunk h][input 2p + e]
      // byte-lane partial sums (8 samples <= 15 per add and stage step: <= 240
      // per lane after two stages), folded into aP / aQ every second stage
      uint32_t bP[2][2] = {{0u, 0u}, {0u, 0u}}, bQ[2][2] = {{0u, 0u}, {0u, 0u}};
      int since_fold = 0;
      for (int ks = 0; ks < nks; ks += kSteps, ++sit) {
        const int rst = sit % kRawStages, ost = sit % kOpStages;
        if (!wait_or_abort(&s.raw_full[rst], (sit / kRawStages) & 1, lim, abort_flag)) {
          fail(s, prm.err, kErrWaitRawFull);
          ok = false;
          break;
        }
        if (!wait_or_abort(&s.op_empty[ost], ((sit / kOpStages) & 1) ^ 1, lim, abort_flag)) {
          fail(s, prm.err, kErrWaitOpEmpty);
          ok = false;
          break;
        }
        const uint32_t rawI_s = smem_u32(s.raw + rst * kRawStage);
        const uint32_t ta0 = tmem + kTmemA0 + kTmemAStage * ost;
#pragma unroll
        for (int sub = 0; sub < kSteps; ++sub) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int ch = 2 * quad + h;
            uint32_t d0, d1, d2, d3;
            ldsm_x4_trans(rawI_s + sub * kRawSub + sw128(lane, ch), d0, d1, d2, d3);
            const uint32_t w0 = __byte_perm(d0, d1, 0x6420), w1 = __byte_perm(d2, d3, 0x6420);
            const uint32_t w2 = __byte_perm(d0, d1, 0x7531), w3 = __byte_perm(d2, d3, 0x7531);
            const uint32_t re0 = biased_re(w0), re1 = biased_re(w1), re2 = biased_re(w2), re3 = biased_re(w3);
            const uint32_t im0 = biased_im(w0), im1 = biased_im(w1), im2 = biased_im(w2), im3 = biased_im(w3);
            bP[h][0] += re0 + re1;
            bP[h][1] += re2 + re3;
            bQ[h][0] += im0 + im1;
            bQ[h][1] += im2 + im3;
            const uint32_t ta = ta0 + (static_cast<uint32_t>(32 * quad + 16 * h) << 16) + 16 * sub;
            tmem_st_16x256b_x2(ta, re0, re1, re2, re3, im0, im1, im2, im3);
          }
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&s.op_full[ost]);
          mbar_arrive(&s.raw_empty[rst]);
        }
        if (++since_fold == 2 || ks + kSteps >= nks) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              aP[h][e] += byte_sum(bP[h][e]);
              aQ[h][e] += byte_sum(bQ[h][e]);
              bP[h][e] = bQ[h][e] = 0u;
            }
          since_fold = 0;
        }
      }
      if (!ok) break;
      // the four lanes sharing an input pair hold disjoint samples
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          aP[h][e] += __shfl_xor_sync(0xFFFFFFFFu, aP[h][e], 1);
          aP[h][e] += __shfl_xor_sync(0xFFFFFFFFu, aP[h][e], 2);
          aQ[h][e] += __shfl_xor_sync(0xFFFFFFFFu, aQ[h][e], 1);
          aQ[h][e] += __shfl_xor_sync(0xFFFFFFFFu, aQ[h][e], 2);
        }
      const int slot = ui & 1;
      if (!wait_or_abort(&s.sums_empty[slot], ((ui >> 1) & 1) ^ 1, lim, abort_flag)) {
        fail(s, prm.err, kErrWaitSumsEmpty);
        break;
      }
      int* sums = s.sums + slot * 4 * kTile;
      if ((lane & 3) == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int i = 16 * (2 * quad + h) + 2 * pj + e;
            sums[i] = aP[h][e];            // each I input is owned by exactly one lane
            sums[kTile + i] = aQ[h][e];
          }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.sums_full[slot]);
    }
  } else if (b_ordinal(warp) >= 0) {
    // ====================================================== B side -> shared planes
    const int ut = b_ordinal(warp) * 32 + lane;  // 0..255
    const int q = ut & 7, row = ut >> 3;       // 16-input chunk, time row within each step
    const uint32_t off = sw128(kappa(row), q); // K row kappa(row) of the B planes
    int sit = 0, ui = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < prm.units && ok; u += gridDim.x, ++ui) {
      int c, bi, bj;
      decode_unit(u, npairs, c, bi, bj);
      const bool diag = (bi == bj);
      BSums sJ;
      sJ.zero();
      int since_flush = 0;
      for (int ks = 0; ks < nks; ks += kSteps, ++sit) {
        const int rst = sit % kRawStages, ost = sit % kOpStages;
        if (!wait_or_abort(&s.raw_full[rst], (sit / kRawStages) & 1, lim, abort_flag)) {
          fail(s, prm.err, kErrWaitRawFull);
          ok = false;
          break;
        }
        if (!wait_or_abort(&s.op_empty[ost], ((sit / kOpStages) & 1) ^ 1, lim, abort_flag)) {
          fail(s, prm.err, kErrWaitOpEmpty);
          ok = false;
          break;
        }
        const uint8_t* rawJ = s.raw + rst * kRawStage + (diag ? 0 : kRawTile);
        uint8_t* opB = s.op + ost * kOpStage;
#pragma unroll
        for (int sub = 0; sub < kSteps; ++sub) {
          const uint4 w = lds128(rawJ + sub * kRawSub + sw128(row, q));
          uint4 re, im;
          re.x = biased_re(w.x); re.y = biased_re(w.y); re.z = biased_re(w.z); re.w = biased_re(w.w);
          im.x = biased_im(w.x); im.y = biased_im(w.y); im.z = biased_im(w.z); im.w = biased_im(w.w);
          sJ.add(re, im);
          uint8_t* b = opB + sub * 2 * kPlane;
          sts128(b + off, re);
          sts128(b + kPlane + off, im);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&s.op_full[ost]);
          mbar_arrive(&s.raw_empty[rst]);
        }
        if (++since_flush == 4) {  // 16 rows per 4 stages: byte lanes stay <= 240
          sJ.flush();
          since_flush = 0;
        }
      }
      if (!ok) break;
      sJ.flush();
      const int slot = ui & 1;
      if (!wait_or_abort(&s.sums_empty[slot], ((ui >> 1) & 1) ^ 1, lim, abort_flag)) {
        fail(s, prm.err, kErrWaitSumsEmpty);
        break;
      }
      int* sums = s.sums + slot * 4 * kTile;
      if (!diag) sJ.publish(sums + 2 * kTile, sums + 3 * kTile, q);
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.sums_full[slot]);
    }
  } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {
    // ====================================================== epilogue
    // Never leaves the unit loop early (the named barriers below must be
    // reached equally often by all four warps); after an abort it only
    // skips work.
    const int quad = warp & 3;
    const int L = 32 * quad + lane;                 // TMEM lane = accumulator row
    const int il = lane_to_input(L);                // input offset of that row in I
    const int T_pad = nks * kStep;
    const long long nbl = static_cast<long long>(prm.N) * (prm.N + 1) / 2;
    int2* stg = s.stage + quad * 32 * 32;
    bool ok = true;
    int ui = 0;
    for (int u = blockIdx.x; u < prm.units; u += gridDim.x, ++ui) {
      int c, bi, bj;
      decode_unit(u, npairs, c, bi, bj);
      const bool diag = (bi == bj);
      const int slot = ui & 1;
      if (ok && !wait_or_abort(&s.sums_full[slot], (ui >> 1) & 1, lim, abort_flag)) {
        fail(s, prm.err, kErrWaitSumsFull);
        ok = false;
      }
      int* sums = s.sums + slot * 4 * kTile;
      const int* PI = sums;
      const int* QI = sums + kTile;
      const int* PJ = diag ? sums : sums + 2 * kTile;
      const int* QJ = diag ? sums + kTile : sums + 3 * kTile;
      // Bias removal: every correction is a multiple of 8 below 2^27 and the
      // corrected value an integer below 2^23, so one FFMA per value is exact.
      if (ok) {
        s.colcorr[L] = static_cast<float>(-8 * (PJ[L] + QJ[L]));
        s.colcorr[kTile + L] = static_cast<float>(-8 * (PJ[L] - QJ[L]));
      }
      {
        // this warp's 32 rows: packed-triangle row offsets (N <= 8192 fits int)
        const int gi = bi * kTile + il;
        s.rowoff[L] = gi < prm.N ? gi * (gi + 1) / 2 : 0;
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (ok && !wait_or_abort(s.acc_full, ui & 1, lim, abort_flag)) {
        fail(s, prm.err, kErrWaitAccFull);
        ok = false;
      }
      ok = __all_sync(0xFFFFFFFFu, ok);
      bool released = false;
      if (ok) {
        tc_fence_after();
        const float row_re = static_cast<float>(-8 * (PI[il] + QI[il]) + 128 * T_pad);
        const float row_im = static_cast<float>(8 * (PI[il] - QI[il]));
        const uint32_t t_row = tmem + (static_cast<uint32_t>(32 * quad) << 16);
        const long long chan_base = static_cast<long long>(c) * nbl;
#pragma unroll 1
        for (int cc = 0; cc < kTile; cc += 32) {
          uint32_t vre[32], vim[32];
          tmem_ld32(t_row + cc, vre);
          tmem_ld32(t_row + 128 + cc, vim);
          tmem_ld_wait();
          if (cc == kTile - 32) {
            // all of D is in registers: the MMA warp may start the next unit
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(s.acc_empty);
            released = true;
          }
          // this lane's row -> staging row `lane` (column index XOR lane)
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float cre = s.colcorr[cc + k], cim = s.colcorr[kTile + cc + k];
            const int re = __float2int_rn(__fmaf_rn(__uint_as_float(vre[k]), 262144.0f, row_re + cre));
            const int im = __float2int_rn(__fmaf_rn(__uint_as_float(vim[k]), 262144.0f, row_im + cim));
            stg[lane * 32 + (k ^ lane)] = make_int2(re, im);
          }
          __syncwarp();
          // 32 rows x 32 baselines: each row is 256 contiguous bytes of the accumulator
          const int gj = bj * kTile + cc + lane;
          const int* ro = s.rowoff + 32 * quad;
          int2* accj = reinterpret_cast<int2*>(prm.acc) + chan_base + gj;
          // a tile pair strictly below the diagonal and inside N needs no checks
          const bool full = bi > bj && bi * kTile + kTile <= prm.N;
          if (full && !prm.accumulate) {
#pragma unroll 4
            for (int r = 0; r < 32; ++r) accj[ro[r]] = stg[r * 32 + (lane ^ r)];
          } else if (full) {
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
              const int2 v = stg[r * 32 + (lane ^ r)];
              int2* dst = accj + ro[r];
              const int2 o = *dst;
              *dst = make_int2(o.x + v.x, o.y + v.y);
            }
          } else {
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
              const int gi = bi * kTile + lane_to_input(32 * quad + r);
              if (gi < prm.N && gj <= gi && gj < prm.N) {
                const int2 v = stg[r * 32 + (lane ^ r)];
                int2* dst = accj + ro[r];
                if (prm.accumulate) {
                  const int2 o = *dst;
                  *dst = make_int2(o.x + v.x, o.y + v.y);
                } else {
                  *dst = v;
                }
              }
            }
          }
          __syncwarp();
        }
      }
      if (!released) {
        __syncwarp();
        if (lane == 0) mbar_arrive(s.acc_empty);
      }
      // all four warps are done with this slot's sums and column corrections
      asm volatile("bar.sync 1, 128;" ::: "memory");
      sums[L] = 0;
      sums[kTile + L] = 0;
      sums[2 * kTile + L] = 0;
      sums[3 * kTile + L] = 0;
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.sums_empty[slot]);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc<kTmemCols>(tmem);
}

}  // namespace tc8

int tc8_smem_bytes() { return tc8::kSmemBytes; }

cudaError_t launch_xcorr_tc8(const CUtensorMap* tmap, const TcParams& prm, int grid, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(tc8::xcorr_tc8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc8::kSmemBytes);
  if (e != cudaSuccess) return e;
  tc8::xcorr_tc8_kernel<<<grid, tc8::kThreads, tc8::kSmemBytes, stream>>>(*tmap, prm);
  return cudaGetLastError();
}

}  // namespace xe
