// tcgen05 X-engine, e4m3 or float16 operands: pairs of CTAs on one M = 256
// MMA.
//
// Computes, like every X-engine path here (the linear-algebra module of the
// paper's section "Back end" applied to the 4+4-bit samples of section
// "Packet capture implementation"),
//   V_c[i][j] = sum_t x[t][c][i] conj(x[t][c][j]),   i >= j,
// into an int32 accumulator [C][N(N+1)/2][2] (packed lower triangle).
//
// Why this layout.  On sm_103 the tensor core reads shared-memory operands
// through the same data pipe as ld/st.shared, and the unpack warps compete
// with the MMA issuer for issue slots.  Two measures cut that traffic:
//  * operand A (the I tile) never touches shared memory: it is transposed in
//    registers and written to tensor memory with tcgen05.st;
//  * the two CTAs of a cluster run one tcgen05.mma.cta_group::2 per step:
//    M = 256 rows (128 I inputs in each CTA's tensor memory), N = 128 J
//    inputs of which each CTA holds 64 rows of operand B in its own shared
//    memory.  Both CTAs share one J tile, so each unpacks and stores only
//    half of it and its tensor core reads only half of B from local shared
//    memory.  Each CTA's 128 x 128 accumulator lives in its own TMEM.
// Per 32-sample e4m3 step the tensor core of one SM reads ~8 KB of operand B
// from its shared memory instead of ~16 KB, and the B unpack per SM halves.
//
// Work: a pair unit is (channel c, J tile, I tile of CTA 0, I tile of
// CTA 1).  The lower-triangle tile pairs (I >= J) of a channel are grouped
// by J column two at a time; the odd one out of a column, (nt-1, j), is
// computed as its transpose (I = j, J = nt-1) next to the last diagonal tile
// and written back conjugated and transposed.  If the count is still odd,
// CTA 1 repeats its partner's tile and writes nothing.  Units left over after
// the last full round of clusters are cut along time (see "schedule" below)
// and their slices summed by split_combine_kernel.
//
// Both operand widths share the design (template parameter EB): a stage is
// 128 K bytes per operand row, i.e. 4 steps of 32 samples as e4m3 (one
// K = 32 MMA per product and step) or 2 steps as float16 (u as the subnormal
// u * 2^-24, two K = 16 MMAs per product and step).
//
// Per step (32 samples) of a unit:
//  * TMA loads the raw time x input tile of I (128-byte rows, 128-byte
//    swizzle) and this CTA's half of J (64-byte rows, 64-byte swizzle) into
//    shared memory; J is skipped when I == J.
//  * A side (two warps per TMEM lane quadrant, one per 16-input chunk):
//    ldmatrix.x4.trans reads a 32-time x 16-input block as 16-bit pairs,
//    four byte permutes regroup it so that each 32-bit word holds four
//    samples of one input, the nibbles become biased e4m3 bytes
//    (u = v + 8, exactly u * 2^-9) and tcgen05.st.16x256b writes the re and
//    im planes.  Input 16g + 2p goes to row 16g + p and input 16g + 2p + 1 to
//    row 16g + p + 8; the samples of a word follow a fixed permutation of
//    time within the step, the same on both operands.
//  * B side (four warps): e4m3 operand B is MN-major with the 64-byte
//    swizzle, which is the raw half-J tile's own layout (a K row = 64
//    contiguous input bytes), so each thread unpacks 16-byte chunks in place
//    (biased re and im bytes at the same N positions) and stores them in K
//    row kappa(t), the A side's K position of time t: no transposition.
//    float16 operand B is K-major with the 128-byte swizzle (64 rows x 128
//    bytes per plane and stage), transposed like the A side, rows ordered
//    like the A rows.
//  * MMA (one thread of CTA 0): D_re += A_re B_re^T + A_im B_im^T,
//                               D_im += A_im B_re^T - A_re B_im^T
//    (negate-B bit); commits are multicast to both CTAs.
//  * Epilogue (each CTA): D (single buffer, 256 TMEM columns) is copied out
//    per 32-column chunk (three chunks to shared staging, one to registers),
//    D_re first and then D_im, each half released to the MMA as soon as it
//    is read (the next unit's real-part MMAs of its first stages run while
//    D_im is still being read); then the bias is removed exactly from per-input
//    sums of u (the column sums of the other half of J are read from the
//    partner's shared memory) and rows are written coalesced to the
//    accumulator (8 staged rows read before their stores, row and column
//    values shuffled from the lanes holding them, diagonal tiles by 32 x 32
//    blocks: unchecked below the diagonal, skipped above it):
//      Re V = D_re - 8 (P_i + Q_i + P_j + Q_j) + 128 T'
//      Im V = D_im + 8 (P_i - Q_i) - 8 (P_j - Q_j).
// Exactness: all partial sums of D stay below 450 T' <= 2^24 for T' <= 37282;
// the host splits longer gulps into launches of at most 32768 samples.  A
// launch covers whole stages (TMA zero-fills the padding, which enters D, the
// sums and T' consistently).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "xe_kernels.h"
#include "xe_ptx.cuh"

namespace xe {
namespace tc8 {

constexpr int kTile = 128;
constexpr int kHalf = 64;                 // J inputs whose B rows one CTA of the pair holds
constexpr int kStep = 32;                 // samples per step (one K = 32 e4m3 MMA, two K = 16 f16 MMAs)
constexpr int kRawSub = kStep * kTile;    // 4096 bytes: one step of one raw tile
#ifndef XE_TC8_RAW_STAGES
#define XE_TC8_RAW_STAGES 2
#endif
#ifndef XE_TC8_OP_STAGES
#define XE_TC8_OP_STAGES 4
#endif
// Synchronisation happens once per stage: the tensor core's instruction
// queue holds only a few MMAs, so every barrier check or commit between MMAs
// costs issue bubbles.  Per stage the MMA thread issues 16 MMAs and one
// commit: 4 steps (128 samples) of e4m3, 2 steps (64 samples) of f16, the
// same 128 K bytes per operand row.  A warp that issues a TMA tile load is
// held for roughly 750 cycles per instruction, so raw tiles move in one box
// per stage and producer warp.
constexpr int kRawStages = XE_TC8_RAW_STAGES;
constexpr int kOpStages = XE_TC8_OP_STAGES;
constexpr int kPlane = kHalf * 128;             // 8 KB: 64 rows x 128 K bytes, K-major
constexpr int kOpStage = 2 * kPlane;            // re plane, im plane
constexpr int kOpBytes = kOpStages * kOpStage;
constexpr int kStageBufs = 3;                   // accumulator chunks staged per epilogue warp
constexpr int kStageRow = 33;                   // words per staged row (padded: conflict-free both ways)
constexpr int kStageChunk = 32 * kStageRow;     // one 32 x 32 chunk of one half (re or im)
constexpr int kStageBytes = 4 * 2 * kStageBufs * kStageChunk * 4;  // per warp: re chunks, then im chunks
constexpr int kBWarpsSums = 4;                  // B-side warps, each with its own partial sums of J
// P_I, Q_I (128 each), then per B-side warp P_J, Q_J (64 each) of this CTA's
// half of J; the column sums are the sums over those warps
constexpr int kSlotInts = 2 * kTile + kBWarpsSums * 2 * kHalf;
constexpr int kSumsBytes = 2 * kSlotInts * 4 + 2 * kTile * 4 + 2 * kTile * 4;
// 2 slots of sums, column corrections (re, im), row and column triangle offsets
constexpr int kNumBars = 2 * kRawStages + 2 * kOpStages + 3 + 2 + 2 + 1;
constexpr int kCtlBytes = 64;   // after the barriers: TMEM address, abort flag, schedule

// Operand width EB (1: e4m3, 2: f16) sets the samples per stage and the raw tiles.
template <int EB>
struct Geo {
  static constexpr int kSteps = EB == 1 ? 4 : 2;        // 32-sample steps per stage
  static constexpr int kRawTile = kSteps * kRawSub;     // TMA box: stage rows x 128 inputs
  static constexpr int kRawHalf = kRawTile / 2;         // TMA box: stage rows x this CTA's 64 J inputs
  static constexpr int kRawStage = kRawTile + kRawHalf; // I box (128-byte rows), half J box (64-byte rows)
  static constexpr int kRawBytes = kRawStages * kRawStage;
  static constexpr int kBarOffset = kOpBytes + kRawBytes + kStageBytes + kSumsBytes;
  static constexpr int kSmemBytes = kBarOffset + kNumBars * 8 + kCtlBytes + 1024;
  static_assert(kSmemBytes <= 227 * 1024, "shared memory budget");
  static_assert(kOpBytes % 1024 == 0 && kRawStage % 1024 == 0, "swizzled tiles need 1024-byte alignment");
};

// Warp roles.  Warp w issues from SM sub-partition w % 4; the A-side and
// epilogue warps need their warp index = TMEM lane quadrant (mod 4).
//   0: TMA I tiles   1: MMA issuer (CTA 0)   2: TMA J tiles
//   4-7, 12-15: A side (quadrant w % 4, chunk (w >> 3) & 1)
//   3, 8, 10, 11: B side   9: second stage forwarder (CTA 1), idle in CTA 0
//   16-19: epilogue
constexpr int kEpiWarp0 = 16;
constexpr int kThreads = 32 * (kEpiWarp0 + 4);
constexpr int kAWarps = 8;
constexpr int kBWarps = 4;
constexpr int kStageArrivals = kAWarps + kBWarps;   // per CTA and stage
static_assert(kBWarpsSums == kBWarps, "one partial-sum block per B-side warp");
constexpr int kTmemCols = 512;
constexpr int kTmemA0 = 256;              // A stages: 64 columns each (128 K bytes of re and of im)
constexpr int kTmemAStage = 64;
static_assert(kTmemA0 + kTmemAStage * kOpStages <= kTmemCols, "tensor memory budget");

__device__ __forceinline__ bool is_a_warp(int w) { return (w >= 4 && w < 8) || (w >= 12 && w < 16); }
__device__ __forceinline__ int b_ordinal(int w) {
  return w == 3 ? 0 : (w == 8 ? 1 : (w == 10 ? 2 : (w == 11 ? 3 : -1)));
}

enum ErrCode : int {
  kErrWaitRawFull = 1 << 0, kErrWaitRawEmpty = 1 << 1, kErrWaitOpFull = 1 << 2,
  kErrWaitOpEmpty = 1 << 3, kErrWaitAccFull = 1 << 4, kErrWaitAccEmpty = 1 << 5,
  kErrWaitSumsFull = 1 << 6, kErrWaitSumsEmpty = 1 << 7, kErrWaitFinal = 1 << 8,
};

struct Smem {
  uint8_t* op;     // [kOpStages][re, im][8 KB]  B planes (this CTA's half): e4m3 128 K rows x 64 N
                   // bytes (MN-major), float16 64 N rows x 128 K bytes (K-major)
  uint8_t* raw;    // [kRawStages][I: kRawTile | J half: kRawHalf]  (Geo<EB>)
  int* stage;      // [4 warps][re, im][kStageBufs][32 rows][kStageRow]
  int* sums;       // [2][kSlotInts]
  float* colcorr;  // [2][128]: per-column bias corrections of the current unit (re, im)
  int* rowoff;     // [128]: packed-triangle offset i (i + 1) / 2 of each accumulator row's input i
  int* coloff;     // [128]: the same for each accumulator column's input j
  uint64_t *raw_full, *raw_empty, *op_full, *op_empty;
  uint64_t *acc_full, *acc_empty, *acc_empty_im, *sums_full, *sums_empty, *final_bar;
  uint32_t* tmem_slot;
  int* abort_flag;
  int* sched;      // schedule header and tail items (item_at)
};

template <int EB>
__device__ __forceinline__ Smem carve(uint8_t* base) {
  using G = Geo<EB>;
  Smem p;
  p.op = base;
  p.raw = base + kOpBytes;
  p.stage = reinterpret_cast<int*>(base + kOpBytes + G::kRawBytes);
  p.sums = reinterpret_cast<int*>(base + kOpBytes + G::kRawBytes + kStageBytes);
  p.colcorr = reinterpret_cast<float*>(p.sums + 2 * kSlotInts);
  p.rowoff = reinterpret_cast<int*>(p.colcorr + 2 * kTile);
  p.coloff = p.rowoff + kTile;
  uint64_t* b = reinterpret_cast<uint64_t*>(base + G::kBarOffset);
  p.raw_full = b; b += kRawStages;
  p.raw_empty = b; b += kRawStages;
  p.op_full = b; b += kOpStages;
  p.op_empty = b; b += kOpStages;
  p.acc_full = b; b += 1;
  p.acc_empty = b; b += 1;
  p.acc_empty_im = b; b += 1;
  p.sums_full = b; b += 2;
  p.sums_empty = b; b += 2;
  p.final_bar = b; b += 1;
  p.tmem_slot = reinterpret_cast<uint32_t*>(b);
  p.abort_flag = reinterpret_cast<int*>(b) + 1;
  p.sched = reinterpret_cast<int*>(b) + 2;
  return p;
}

// ------------------------------------------------------------ cluster helpers
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared::cluster address of the same object in CTA `cta` of this cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(cta));
  return r;
}
// Arrive (release, cluster scope) on the barrier at this offset in CTA `cta`.
__device__ __forceinline__ void arrive_at(uint64_t* bar, uint32_t cta) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(peer_addr(bar, cta))
               : "memory");
}
// Arrive without release semantics: for signals that publish no memory
// writes (the arriving thread only finished reading), so the arrival does not
// wait for the thread's outstanding global stores.
__device__ __forceinline__ void arrive_relaxed_at(uint64_t* bar, uint32_t cta) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(peer_addr(bar, cta))
               : "memory");
}
__device__ __forceinline__ int ld_peer(const int* p, uint32_t cta) {
  int v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(peer_addr(p, cta)) : "memory");
  return v;
}
// One test of the phase with cluster-scope acquire (arrivals may come from
// the partner CTA), parked by the hardware up to the suspend hint.
__device__ __forceinline__ bool try_wait_c(uint32_t bar_addr, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(bar_addr), "r"(parity), "r"(0x989680u) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                              volatile int* abort_flag) {
  const uint32_t a = smem_u32(bar);
  if (try_wait_c(a, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (try_wait_c(a, parity)) return true;
    if (*abort_flag) return false;
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void fail(const Smem& s, int* err, int code) {
  atomicExch(s.abort_flag, 1);
  atomicOr(err, code);
}

// ----------------------------------------------------------- tcgen05 (pair)
__device__ __forceinline__ void mma2_f8_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}"
               ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma2_f16_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                                uint32_t idesc, uint32_t accumulate) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
               ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate));
}
// Completion of this thread's earlier MMAs arrives on `bar` in both CTAs.
__device__ __forceinline__ void commit2(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
               ::"r"(smem_u32(bar)), "h"(static_cast<uint16_t>(3)) : "memory");
}
// L2 prefetch of one tile of a 3-D tensor (no shared-memory destination).
__device__ __forceinline__ void tma_prefetch_3d(const void* desc, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];"
               ::"l"(reinterpret_cast<uint64_t>(desc)), "r"(x), "r"(y), "r"(z)
               : "memory");
}
// The raw-tile producers prefetch the tile kPrefetch stages ahead into L2,
// so a copy waits for L2 rather than DRAM (e4m3 lwa: 1.035 -> 0.961 ms at two
// stages ahead; with the leaner MMA issue loop one stage ahead is a little
// better, 0.914 -> 0.907 ms; three, four or eight stages ahead, or
// prefetching into the next unit, measured no better).
constexpr int kPrefetch = 1;
// MN-major operand, 64-byte swizzle: K rows of 64 bytes (64 e4m3 values
// along N, one swizzle atom wide), 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sdesc_mn_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= 1ull << 16;                                     // leading byte offset: one atom along N, unused
  d |= static_cast<uint64_t>(512 >> 4) << 32;          // stride byte offset: next 8 K rows
  d |= 1ull << 46;                                     // descriptor version for tcgen05
  d |= 4ull << 61;                                     // SWIZZLE_64B
  return d;
}
// K-major operand, 128-byte swizzle: 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= 1ull << 16;                                     // leading byte offset: unused when swizzled
  d |= static_cast<uint64_t>(1024 >> 4) << 32;         // stride byte offset
  d |= 1ull << 46;                                     // descriptor version for tcgen05
  d |= 2ull << 61;                                     // SWIZZLE_128B
  return d;
}

// -------------------------------------------------------------- work units
// Pair units per channel for nt tiles per side (see the file comment).
__host__ __device__ inline int pairs_per_channel(int nt) {
  int p = 0;
  for (int j = 0; j < nt - 1; ++j) p += (nt - j) >> 1;
  const int e = 1 + (nt - 1) / 2;  // last column: diagonal tile + transposed odd ones out
  return p + (e + 1) / 2;
}

struct Unit {
  int c, ti, tj;   // channel, this CTA's I tile, the pair's J tile
  bool transposed; // computed block is the transpose of the lower-triangle tile (tj, ti)
  bool write;      // false: duplicate of the partner's tile, kept off the output
};

__device__ __forceinline__ Unit decode_unit(int u, int per_chan, int nt, int rank) {
  Unit t;
  t.c = u / per_chan;
  int e = u - t.c * per_chan;
  t.transposed = false;
  t.write = true;
  for (int j = 0; j < nt - 1; ++j) {
    const int np = (nt - j) >> 1;
    if (e < np) {
      t.ti = j + 2 * e + rank;
      t.tj = j;
      return t;
    }
    e -= np;
  }
  const int ne = 1 + (nt - 1) / 2;
  int k = 2 * e + rank;
  if (k >= ne) {  // odd count: repeat the partner's tile
    k = 2 * e;
    t.write = false;
  }
  t.tj = nt - 1;
  if (k == 0) {
    t.ti = nt - 1;
  } else {  // odd one out of column j = ((nt-1) & 1) + 2 (k-1), i.e. tile (nt-1, j)
    t.ti = ((nt - 1) & 1) + 2 * (k - 1);
    t.transposed = true;
  }
  return t;
}

// ------------------------------------------------------------ schedule
// Cluster cl runs the pair units cl, cl + ncl, ... of the R = units / ncl
// full rounds.  The L = units % ncl units left over would keep L clusters
// busy for a whole unit more while the rest idle, so each is cut along time
// into q = ncl / L nearly equal parts (stages [S i / q, S (i + 1) / q) of its
// S, i < q), and cluster cl < q L takes part cl % q of leftover unit cl / q:
// one part per cluster, since a second one would wait for the first one's
// accumulator to be drained.  A part is reduced like a unit of its own (its
// own sums of u and sample count T') and its exact integer block is stored,
// in the epilogue's usual write pattern, into the cluster's workspace slot
// (one 128 x 128 int2 tile per CTA: row a = accumulator row of the output
// tile in lane order, column b = input offset in the tile).
// split_combine_kernel then adds the q parts of each leftover unit and
// writes the sum as a unit's epilogue would.  All sums are integer, so their
// order does not matter.
constexpr int kMinPartSamples = 1024;        // shortest part worth its own epilogue
constexpr int kSplitTile = kTile * kTile;    // int2 per CTA and workspace slot

struct Item {
  int p;        // problem of the launch
  int u;        // pair unit of that problem
  int k0, k1;   // its 32-sample steps [k0, k1)
  int lo;       // leftover unit index of a part, else -1
};

// One launch: the problems it correlates (one for a plan's call, up to
// kMaxBatch for a batched call), their maps and the concatenation of their
// pair units (problem k owns global units [prefix[k], prefix[k + 1])).
// Passed as a __grid_constant__ parameter, so the tensor maps stay in
// parameter space as TMA requires of a map it is given by address.
struct ProbDev {
  int32_t* acc;          // [C][N (N + 1) / 2][2]
  int* err;              // device error word of the problem's plan
  long long acc_pairs;   // int2 elements of acc (debug index checks)
  int N, nt, per_chan, nks, accumulate;
};
// NP: table size, 1 for a plan's own launch (every index a constant) or
// kMaxBatch for a batched launch.
template <int NP>
struct PairLaunch {
  CUtensorMap ti[NP];   // I tiles: box {128, 1, rows}, 128-byte swizzle
  CUtensorMap tj[NP];   // half J tiles: box {64, 1, rows}, 64-byte swizzle
  ProbDev p[NP];
  int prefix[NP + 1];
  int nprob, units, split_parts;
  int2* split_ws;              // time-sliced leftover units (one problem only), or nullptr
  long long ws_pairs;
  unsigned long long timeout_ns;
};
static_assert(sizeof(PairLaunch<kMaxBatch>) <= 4096, "kernel parameter space");
static_assert(alignof(CUtensorMap) >= 64, "tensor maps in parameter space need 64-byte alignment");

// A wait gave up: stop every role of this CTA and record the code in every
// problem's error word (the launch's results are all in doubt).
template <int NP>
__device__ __forceinline__ void fail_all(const Smem& s, const PairLaunch<NP>& L, int code) {
  atomicExch(s.abort_flag, 1);
  for (int k = 0; k < (NP == 1 ? 1 : L.nprob); ++k) atomicOr(L.p[k].err, code);
}

// Schedule of this cluster in shared memory: {items, R, cl, ncl, nks} and
// then the item after the R full rounds, if any, as {u, k0, k1, lo} (u a
// global unit; k1 = -1: the whole unit).  nks and the parts belong to a
// single-problem launch; a batched launch has no parts.
constexpr int kSchedInts = 5 + 4;
static_assert((2 + kSchedInts) * 4 <= kCtlBytes, "control words after the barriers");
__device__ inline void fill_sched(int* sc, int units, int cl, int ncl, int nks, int steps, int q) {
  const int R = units / ncl, L = units - R * ncl, S = nks / steps;
  int n = 0;
  int* t = sc + 5;
  if (q == 0 && cl < L) {
    t[0] = R * ncl + cl; t[1] = 0; t[2] = -1; t[3] = -1;
    n = 1;
  } else if (q > 0 && cl < q * L) {
    const int l = cl / q, i = cl - l * q;
    t[0] = R * ncl + l; t[1] = S * i / q * steps; t[2] = S * (i + 1) / q * steps; t[3] = l;
    n = 1;
  }
  sc[0] = R + n;
  sc[1] = R;
  sc[2] = cl;
  sc[3] = ncl;
  sc[4] = nks;
}

// Item i of this cluster (the schedule is read from shared memory each time:
// registers are scarce in every warp role), with its problem.
template <int NP>
__device__ __forceinline__ Item item_at(const int* sc, int i, const PairLaunch<NP>& L) {
  Item w;
  const int R = sc[1];
  int g;
  if (i < R) {
    g = sc[2] + i * sc[3];
    w.k0 = 0;
    w.k1 = -1;
    w.lo = -1;
  } else {
    g = sc[5];
    w.k0 = sc[6];
    w.k1 = sc[7];
    w.lo = sc[8];
  }
  int p = 0;
  if constexpr (NP > 1)
    while (p + 1 < L.nprob && g >= L.prefix[p + 1]) ++p;
  w.p = p;
  w.u = g - L.prefix[p];
  if (w.k1 < 0) w.k1 = L.p[p].nks;
  return w;
}

// Parts q per leftover unit (0: run the leftover units whole).
__host__ inline int split_parts(long long units, long long clusters, int nks, int steps) {
  const long long L = units % clusters;
  if (L == 0) return 0;
  long long min_part = kMinPartSamples / (steps * kStep);
  if (min_part < 1) min_part = 1;
  long long q = clusters / L;
  if (q > (nks / steps) / min_part) q = (nks / steps) / min_part;
  return q >= 2 ? static_cast<int>(q) : 0;
}

// ------------------------------------------------------------------ unpack
__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t& d0, uint32_t& d1, uint32_t& d2,
                                              uint32_t& d3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(d0), "=r"(d1), "=r"(d2), "=r"(d3) : "r"(addr) : "memory");
}
__device__ __forceinline__ void sts64(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.u32 [%0], {%1,%2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
               : "memory");
  return v;
}
// .x2: the re plane (8 columns) and the im plane (the next 8) of one step
__device__ __forceinline__ void tmem_st_16x256b_x2(uint32_t taddr, uint32_t r0, uint32_t r1, uint32_t r2,
                                                   uint32_t r3, uint32_t r4, uint32_t r5, uint32_t r6,
                                                   uint32_t r7) {
  asm volatile("tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               ::"r"(taddr), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(r4), "r"(r5), "r"(r6), "r"(r7)
               : "memory");
}
// .x4: the re plane (16 columns = 32 float16 of K) and the im plane of one step
__device__ __forceinline__ void tmem_st_16x256b_x4(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile("tcgen05.st.sync.aligned.16x256b.x4.b32 [%0], "
               "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                 "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
               : "memory");
}
// Release a raw stage as soon as this warp's loads from it have returned:
// the XOR reads every loaded register (so the loads have completed), the
// empty asm keeps it ahead of the arrive, and lane 0 arrives for the warp.
template <int NW>
__device__ __forceinline__ void release_raw_after_loads(const uint32_t* words, uint64_t* bar, int lane) {
  uint32_t dep = 0;
#pragma unroll
  for (int k = 0; k < NW; ++k) dep ^= words[k];
  asm volatile("" ::"r"(dep));
  __syncwarp();
  if (lane == 0) mbar_arrive(bar);
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t biased_re(uint32_t w) { return ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u; }
__device__ __forceinline__ uint32_t biased_im(uint32_t w) { return (w & 0x0F0F0F0Fu) ^ 0x08080808u; }
__device__ __forceinline__ int byte_sum(uint32_t w) { return static_cast<int>(__dp4a(w, 0x01010101u, 0u)); }

// Byte offset of 16-byte chunk q of row k in a 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw128(int k, int q) {
  return static_cast<uint32_t>(k * 128 + ((q ^ (k & 7)) << 4));
}

// Accumulator row -> input offset inside its 128-input tile (the A side's
// lane order; also the column order of the float16 kernel's B operand).
__device__ __forceinline__ int lane_to_input(int L) {
  const int r = L & 15;
  return (L & ~15) + (r < 8 ? 2 * r : 2 * (r - 8) + 1);
}
// Its inverse: the accumulator row that holds input offset i.
__device__ __forceinline__ int input_to_lane(int i) {
  const int r = i & 15;
  return (i & ~15) + ((r & 1) ? 8 + (r >> 1) : (r >> 1));
}
// Accumulator column -> input offset inside the J tile.  The e4m3 kernel's
// B operand is MN-major in the raw tile's own input order (column n is input
// n); the float16 kernel's is K-major in the A side's lane order.
template <int EB>
__device__ __forceinline__ int col_to_input(int L) {
  if constexpr (EB == 1) return L;
  else return lane_to_input(L);
}
// K position, within a 32-sample step, of the sample at time t of that step
// on the A side (the order in which the transposing loads deliver the
// samples; operand B follows it): kappa(t) = 8 ((t mod 8) / 2) + 2 (t / 8) + t mod 2.
__device__ __forceinline__ int kappa(int t) { return 8 * ((t & 7) >> 1) + 2 * (t >> 3) + (t & 1); }

// One 32-time x 16-input block of a raw tile (four 8x8 16-bit matrices read
// transposed by ldmatrix) -> biased e4m3 words of the two
// inputs 2p, 2p+1 (p = lane / 4): re0, re1 / im0, im1 hold 8 samples of
// input 2p, re2, re3 / im2, im3 those of input 2p+1 (K bytes 8 (lane % 4)
// to 8 (lane % 4) + 7 of the step).  Byte-lane sums go to bP / bQ.
struct Words {
  uint32_t re0, re1, re2, re3, im0, im1, im2, im3;
};
__device__ __forceinline__ Words unpack_words(const uint32_t (&d)[4], uint32_t (&bP)[2], uint32_t (&bQ)[2]) {
  const uint32_t d0 = d[0], d1 = d[1], d2 = d[2], d3 = d[3];
  const uint32_t w0 = __byte_perm(d0, d1, 0x6420), w1 = __byte_perm(d2, d3, 0x6420);
  const uint32_t w2 = __byte_perm(d0, d1, 0x7531), w3 = __byte_perm(d2, d3, 0x7531);
  Words o;
  o.re0 = biased_re(w0); o.re1 = biased_re(w1); o.re2 = biased_re(w2); o.re3 = biased_re(w3);
  o.im0 = biased_im(w0); o.im1 = biased_im(w1); o.im2 = biased_im(w2); o.im3 = biased_im(w3);
  bP[0] += o.re0 + o.re1;
  bP[1] += o.re2 + o.re3;
  bQ[0] += o.im0 + o.im1;
  bQ[1] += o.im2 + o.im3;
  return o;
}

// Four biased bytes -> two words of two float16 bit patterns each (u as the
// subnormal u * 2^-24): (b0, b1) and (b2, b3).
__device__ __forceinline__ uint32_t f16_lo(uint32_t w) { return __byte_perm(w, 0u, 0x4140); }
__device__ __forceinline__ uint32_t f16_hi(uint32_t w) { return __byte_perm(w, 0u, 0x4342); }

// Per-lane sums of the biased parts of inputs 2p + e: byte lanes (at most
// 4 x 30 per stage) folded into ints every second stage.
struct PairSums {
  uint32_t bP[2], bQ[2];
  int P[2], Q[2];
  __device__ __forceinline__ void zero() {
    bP[0] = bP[1] = bQ[0] = bQ[1] = 0u;
    P[0] = P[1] = Q[0] = Q[1] = 0;
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      P[e] += byte_sum(bP[e]);
      Q[e] += byte_sum(bQ[e]);
      bP[e] = bQ[e] = 0u;
    }
  }
  // the four lanes sharing an input pair hold disjoint samples
  __device__ __forceinline__ void reduce() {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      P[e] += __shfl_xor_sync(0xFFFFFFFFu, P[e], 1);
      P[e] += __shfl_xor_sync(0xFFFFFFFFu, P[e], 2);
      Q[e] += __shfl_xor_sync(0xFFFFFFFFu, Q[e], 1);
      Q[e] += __shfl_xor_sync(0xFFFFFFFFu, Q[e], 2);
    }
  }
};

// One 32-column chunk of one half (re or im) of this lane's accumulator row,
// as raw float32 bits, into row `lane` of a staging chunk: the quickest way
// to get D out of tensor memory.  The bias is removed after D is released.
// Rows of 33 words keep both the row-wise stores here and the column-wise
// reads of the write-out free of bank conflicts, with immediate offsets.
__device__ __forceinline__ void stage_raw(int* buf, const uint32_t (&v)[32], int lane) {
  int* w = buf + lane * kStageRow;
#pragma unroll
  for (int k = 0; k < 32; ++k) w[k] = static_cast<int>(v[k]);
}

// Staged value (row r, column k) of a chunk: real part, imaginary part.
__device__ __forceinline__ int2 staged(const int* chunk, int r, int k) {
  return make_int2(chunk[r * kStageRow + k], chunk[kStageBufs * kStageChunk + r * kStageRow + k]);
}

// The MMAs of one operand stage for the real half of D (WHICH & 1) and/or its
// imaginary half (WHICH & 2):
//   D_re += A_re B_re^T + A_im B_im^T,   D_im += A_im B_re^T - A_re B_im^T.
// A from tensor memory (stage columns at a0), B in shared memory (descriptor
// bd of the stage's re plane): e4m3 MN-major (K rows of 64 bytes, bit 16 of
// the instruction descriptor), float16 K-major; M = 256 (pair), N = 128.
template <int EB, int WHICH>
__device__ __forceinline__ void stage_mmas(uint32_t d_re, uint32_t d_im, uint32_t a0, uint64_t bd,
                                           uint32_t acc_first) {
  constexpr uint32_t id_pos =
      (1u << 4) | ((128u >> 3) << 17) | ((256u >> 4) << 24) | (EB == 1 ? (1u << 16) : 0u);
  constexpr uint32_t id_neg = id_pos | (1u << 14);
  constexpr uint32_t kPlaneDesc = kPlane >> 4;   // descriptor address units
  if constexpr (EB == 1) {
    // per step: A columns re 8 | im 8, B K rows 32 (2048 bytes)
#pragma unroll
    for (int sub = 0; sub < Geo<EB>::kSteps; ++sub) {
      const uint32_t a_re = a0 + 16 * sub, a_im = a_re + 8;
      const uint64_t b_re = bd + 128 * sub, b_im = bd + kPlaneDesc + 128 * sub;
      const uint32_t acc0 = sub > 0 ? 1u : acc_first;
      if constexpr ((WHICH & 1) != 0) {
        mma2_f8_tmem_a(d_re, a_re, b_re, id_pos, acc0);
        mma2_f8_tmem_a(d_re, a_im, b_im, id_pos, 1u);
      }
      if constexpr ((WHICH & 2) != 0) {
        mma2_f8_tmem_a(d_im, a_im, b_re, id_pos, acc0);
        mma2_f8_tmem_a(d_im, a_re, b_im, id_neg, 1u);
      }
    }
  } else {
    // per step: A columns re 16 | im 16 (two K = 16 halves of 8 each),
    // B K bytes 64 (two halves of 32)
#pragma unroll
    for (int sub = 0; sub < Geo<EB>::kSteps; ++sub)
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const uint32_t a_re = a0 + 32 * sub + 8 * kk, a_im = a_re + 16;
        const uint64_t b_re = bd + 4 * sub + 2 * kk, b_im = bd + kPlaneDesc + 4 * sub + 2 * kk;
        const uint32_t acc0 = (sub + kk) > 0 ? 1u : acc_first;
        if constexpr ((WHICH & 1) != 0) {
          mma2_f16_tmem_a(d_re, a_re, b_re, id_pos, acc0);
          mma2_f16_tmem_a(d_re, a_im, b_im, id_pos, 1u);
        }
        if constexpr ((WHICH & 2) != 0) {
          mma2_f16_tmem_a(d_im, a_im, b_re, id_pos, acc0);
          mma2_f16_tmem_a(d_im, a_re, b_im, id_neg, 1u);
        }
      }
  }
}

// Bias removal of one staged value: D holds sums of products of u * 2^-9
// (e4m3) or u * 2^-24 (f16) values; every correction is a multiple of 8
// below 2^27 and the corrected value an integer below 2^23, so one FFMA per
// value is exact.
template <int EB>
__device__ __forceinline__ int2 unbias(int2 raw, float rre, float rim, float cre, float cim) {
  constexpr float kScale = EB == 1 ? 262144.0f : 281474976710656.0f;   // 2^18, 2^48
  return make_int2(__float2int_rn(__fmaf_rn(__int_as_float(raw.x), kScale, rre + cre)),
                   __float2int_rn(__fmaf_rn(__int_as_float(raw.y), kScale, rim + cim)));
}

template <int EB, int NP>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
xcorr_tc8_kernel(const __grid_constant__ PairLaunch<NP> L) {
  using G = Geo<EB>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  const Smem s = carve<EB>(base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const uint32_t peer = rank ^ 1u;
  const int cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const uint64_t lim = L.timeout_ns;
  volatile int* abort_flag = s.abort_flag;

  if (tid == 0) {
    for (int k = 0; k < kRawStages; ++k) {
      mbar_init(&s.raw_full[k], 2);   // the I-tile producer and the J-tile producer
      mbar_init(&s.raw_empty[k], kStageArrivals);
    }
    for (int k = 0; k < kOpStages; ++k) {
      // own producers; in CTA 0 also the forwarded completion of CTA 1's stage
      mbar_init(&s.op_full[k], kStageArrivals + (rank == 0 ? 1 : 0));
      mbar_init(&s.op_empty[k], 1);
    }
    mbar_init(s.acc_full, 1);
    mbar_init(s.acc_empty, 8);       // both CTAs' epilogue warps (used in CTA 0): D_re read
    mbar_init(s.acc_empty_im, 8);    // the same for D_im
    for (int k = 0; k < 2; ++k) {
      mbar_init(&s.sums_full[k], kAWarps + 2 * kBWarps);  // own A and B warps, partner's B warps
      mbar_init(&s.sums_empty[k], 8);                     // own and partner's epilogue warps
    }
    mbar_init(s.final_bar, 1);
    *s.abort_flag = 0;
    fill_sched(s.sched, L.units, cl, ncl, L.p[0].nks, G::kSteps, L.split_parts);
    mbar_fence_init();
    for (int k = 0; k < (NP == 1 ? 1 : L.nprob); ++k) {
      tma_prefetch_desc(&L.ti[k]);
      tma_prefetch_desc(&L.tj[k]);
    }
  }
  // partial-sum blocks a kernel never writes (the float16 B side keeps its
  // sums in the first block) must read as zero
  for (int k = tid; k < 2 * kSlotInts; k += kThreads) s.sums[k] = 0;
  if (warp == 0) {
    // one warp of each CTA of the pair allocates together: same columns in both
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(s.tmem_slot)), "n"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();   // both CTAs' barriers and tensor memory exist before any remote access
  tc_fence_after();
  const uint32_t tmem = *s.tmem_slot;

  if (warp == 0 || warp == 2) {
    // ====================================================== TMA producers
    if (lane == 0) {
      const int tile = warp >> 1;               // 0: I tiles, 1: J tiles
      int rit = 0;                              // raw stage counter (4 steps each)
      bool ok = true;
      for (int it = 0; it < s.sched[0] && ok; ++it) {
        const Item w = item_at(s.sched, it, L);
        const Unit t = decode_unit(w.u, L.p[w.p].per_chan, L.p[w.p].nt, rank);
        const bool own_diag = (t.ti == t.tj);
        for (int ks = w.k0; ks < w.k1; ks += G::kSteps, ++rit) {
          const int st = rit % kRawStages;
          if (!wait_or_abort(&s.raw_empty[st], ((rit / kRawStages) & 1) ^ 1, lim, abort_flag)) {
            fail_all(s, L, kErrWaitRawEmpty);
            ok = false;
            break;
          }
          uint8_t* dst = s.raw + st * G::kRawStage + tile * G::kRawTile;
          const int kp = ks + kPrefetch * G::kSteps;   // the stage to prefetch into L2
          if (tile == 0) {
            mbar_arrive_expect_tx(&s.raw_full[st], G::kRawTile);
            tma_load_3d(dst, &L.ti[w.p], &s.raw_full[st], t.ti * kTile, t.c, ks * kStep);
            if (kp < w.k1) tma_prefetch_3d(&L.ti[w.p], t.ti * kTile, t.c, kp * kStep);
          } else if (!own_diag) {
            mbar_arrive_expect_tx(&s.raw_full[st], G::kRawHalf);
            tma_load_3d(dst, &L.tj[w.p], &s.raw_full[st], t.tj * kTile + kHalf * static_cast<int>(rank), t.c,
                        ks * kStep);
            if (kp < w.k1)
              tma_prefetch_3d(&L.tj[w.p], t.tj * kTile + kHalf * static_cast<int>(rank), t.c, kp * kStep);
          } else {
            mbar_arrive(&s.raw_full[st]);    // the I tile serves as J
          }
        }
      }
      // wait for the copies still in flight (normally all consumed already)
      for (int k = rit - 1; k >= 0 && k > rit - 1 - kRawStages; --k)
        mbar_wait(&s.raw_full[k % kRawStages], (k / kRawStages) & 1, lim);
    }
  } else if ((warp == 1 || warp == 9) && rank == 1) {
    // ====================================================== stage forwarders (CTA 1)
    // A release at cluster scope costs the arriving thread ~1100 cycles
    // (measured), so CTA 1's producers arrive on their local barrier and two
    // threads, in warps 1 and 9, tell CTA 0 that CTA 1's half of a stage is
    // ready: warp 1 forwards the even stages, warp 9 the odd ones.  One
    // forwarder was busy 93 % of the kernel and paced the stages.
    if (lane == 0) {
      const int fwd = warp == 9 ? 1 : 0;
      int sit = 0;
      bool ok = true;
      for (int it = 0; it < s.sched[0] && ok; ++it) {
        const Item w = item_at(s.sched, it, L);
        for (int ks = w.k0; ks < w.k1; ks += G::kSteps, ++sit) {
          if ((sit & 1) != fwd) continue;
          const int st = sit % kOpStages;
          if (!wait_or_abort(&s.op_full[st], (sit / kOpStages) & 1, lim, abort_flag)) {
            fail_all(s, L, kErrWaitOpFull);
            ok = false;
            break;
          }
          arrive_at(&s.op_full[st], 0);
        }
      }
    }
  } else if (warp == 1) {
    // ====================================================== MMA issuer (CTA 0)
    // The tensor core's instruction queue is short, so the issuing thread's
    // scalar work between MMAs shows: descriptors are one base per operand
    // slot plus compile-time offsets, and the slot and its phase are
    // counters (a probe: 79 -> 69 cycles per MMA).
    if (lane == 0) {
      int ui = 0, st = 0;
      uint32_t ph = 0;                            // phase of operand slot st
      bool ok = true;
      constexpr uint32_t kSlotDesc = kOpStage >> 4;   // descriptor address units
      const uint64_t desc0 = EB == 1 ? sdesc_mn_sw64(smem_u32(s.op)) : sdesc_k_sw128(smem_u32(s.op));
      const uint32_t d_re = tmem, d_im = tmem + 128;
      for (int it = 0; it < s.sched[0] && ok; ++it, ++ui) {
        const Item w = item_at(s.sched, it, L);
        const uint32_t free_par = (ui & 1) ^ 1;
        // D is released in two halves.  Once the epilogue has read D_re, the
        // real-part MMAs of the operand stages already resident (up to the
        // whole ring) are issued while it still reads D_im; their imaginary
        // parts follow the second release.
        const int nst = (w.k1 - w.k0 + G::kSteps - 1) / G::kSteps;
        const int head = nst < kOpStages ? nst : kOpStages;
        if (!wait_or_abort(s.acc_empty, free_par, lim, abort_flag)) {
          fail_all(s, L, kErrWaitAccEmpty);
          break;
        }
        tc_fence_after();
        {
          int sh = st;
          uint32_t phh = ph;
          for (int p = 0; p < head; ++p) {
            if (!wait_or_abort(&s.op_full[sh], phh, lim, abort_flag)) {
              fail_all(s, L, kErrWaitOpFull);
              ok = false;
              break;
            }
            tc_fence_after();
            stage_mmas<EB, 1>(d_re, d_im, tmem + kTmemA0 + kTmemAStage * sh,
                              desc0 + static_cast<uint64_t>(kSlotDesc * sh), p == 0 ? 0u : 1u);
            if (++sh == kOpStages) {
              sh = 0;
              phh ^= 1u;
            }
          }
        }
        if (!ok) break;
        if (!wait_or_abort(s.acc_empty_im, free_par, lim, abort_flag)) {
          fail_all(s, L, kErrWaitAccEmpty);
          break;
        }
        tc_fence_after();
        for (int p = 0; p < head; ++p) {
          stage_mmas<EB, 2>(d_re, d_im, tmem + kTmemA0 + kTmemAStage * st,
                            desc0 + static_cast<uint64_t>(kSlotDesc * st), p == 0 ? 0u : 1u);
          commit2(&s.op_empty[st]);
          if (++st == kOpStages) {
            st = 0;
            ph ^= 1u;
          }
        }
        for (int ks = w.k0 + head * G::kSteps; ks < w.k1; ks += G::kSteps) {
          if (!wait_or_abort(&s.op_full[st], ph, lim, abort_flag)) {
            fail_all(s, L, kErrWaitOpFull);
            ok = false;
            break;
          }
          tc_fence_after();
          stage_mmas<EB, 3>(d_re, d_im, tmem + kTmemA0 + kTmemAStage * st,
                            desc0 + static_cast<uint64_t>(kSlotDesc * st), 1u);
          commit2(&s.op_empty[st]);
          if (++st == kOpStages) {
            st = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        commit2(s.acc_full);
      }
      commit2(s.final_bar);
    }
  } else if (is_a_warp(warp)) {
    // ====================================================== A side -> TMEM
    const int quad = warp & 3;                 // TMEM lane quadrant of this warp
    const int h = (warp >> 3) & 1;             // which 16-input chunk of the quadrant
    const int ch = 2 * quad + h;
    const int pj = lane >> 2;                  // input pair of this lane within the chunk
    const uint32_t lane_off = static_cast<uint32_t>(32 * quad + 16 * h) << 16;
    int sit = 0, ui = 0;
    bool ok = true;
    for (int it = 0; it < s.sched[0] && ok; ++it, ++ui) {
      const Item w = item_at(s.sched, it, L);
      PairSums ps;
      ps.zero();
      int since_fold = 0;
      for (int ks = w.k0; ks < w.k1; ks += G::kSteps, ++sit) {
        const int rst = sit % kRawStages, ost = sit % kOpStages;
        if (!wait_or_abort(&s.raw_full[rst], (sit / kRawStages) & 1, lim, abort_flag)) {
          fail_all(s, L, kErrWaitRawFull);
          ok = false;
          break;
        }
        // the four transposing loads first (their latencies overlap), while
        // the MMA may still hold the operand stage
        const uint32_t rawI_s = smem_u32(s.raw + rst * G::kRawStage);
        uint32_t dv[G::kSteps][4];
#pragma unroll
        for (int sub = 0; sub < G::kSteps; ++sub)
          ldsm_x4_trans(rawI_s + sub * kRawSub + sw128(lane, ch), dv[sub][0], dv[sub][1], dv[sub][2], dv[sub][3]);
        // the raw stage goes back to the TMA producers before this warp waits
        // for its operand slot (raw tiles arrive with L2 latency; two raw
        // stages leave little slack)
        release_raw_after_loads<4 * G::kSteps>(&dv[0][0], &s.raw_empty[rst], lane);
        if (!wait_or_abort(&s.op_empty[ost], ((sit / kOpStages) & 1) ^ 1, lim, abort_flag)) {
          fail_all(s, L, kErrWaitOpEmpty);
          ok = false;
          break;
        }
        const uint32_t ta0 = tmem + kTmemA0 + kTmemAStage * ost + lane_off;
#pragma unroll
        for (int sub = 0; sub < G::kSteps; ++sub) {
          const Words w = unpack_words(dv[sub], ps.bP, ps.bQ);
          if constexpr (EB == 1) {
            tmem_st_16x256b_x2(ta0 + 16 * sub, w.re0, w.re1, w.re2, w.re3, w.im0, w.im1, w.im2, w.im3);
          } else {
            // float16: re K 0-15 | re K 16-31 | im K 0-15 | im K 16-31, 8 columns each;
            // a thread's first four samples go to the first K half, the next four to the second
            const uint32_t r[16] = {f16_lo(w.re0), f16_hi(w.re0), f16_lo(w.re2), f16_hi(w.re2),
                                    f16_lo(w.re1), f16_hi(w.re1), f16_lo(w.re3), f16_hi(w.re3),
                                    f16_lo(w.im0), f16_hi(w.im0), f16_lo(w.im2), f16_hi(w.im2),
                                    f16_lo(w.im1), f16_hi(w.im1), f16_lo(w.im3), f16_hi(w.im3)};
            tmem_st_16x256b_x4(ta0 + 32 * sub, r);
          }
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.op_full[ost]);
        if (++since_fold == 2 || ks + G::kSteps >= w.k1) {
          ps.fold();
          since_fold = 0;
        }
      }
      if (!ok) break;
      ps.reduce();
      const int slot = ui & 1;
      if (!wait_or_abort(&s.sums_empty[slot], ((ui >> 1) & 1) ^ 1, lim, abort_flag)) {
        fail_all(s, L, kErrWaitSumsEmpty);
        break;
      }
      int* sl = s.sums + slot * kSlotInts;
      if ((lane & 3) == 0) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int i = 16 * ch + 2 * pj + e;   // each I input is owned by exactly one lane
          sl[i] = ps.P[e];
          sl[kTile + i] = ps.Q[e];
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s.sums_full[slot]);
    }
  } else if (EB == 1 && b_ordinal(warp) >= 0) {
    // ====================================================== B side (e4m3) -> MN-major planes
    // Operand B is MN-major with the 64-byte swizzle: K row k of a step
    // holds this CTA's 64 J inputs as 64 contiguous bytes, which is the raw
    // half-J tile's own layout.  Unpacking is therefore element-wise: each
    // thread takes one 16-byte chunk (16 inputs) of one time row per step,
    // splits every byte into its biased re and im bytes and stores both at
    // the same N positions of K row kappa(t), the A side's K position of
    // that time.  No transposition, one 16-byte load and two 16-byte stores
    // per chunk.
    const int g = b_ordinal(warp);
    const int tau = 32 * g + lane;
    const int t32 = tau >> 2;                          // time row of this thread within each step
    const int cl = (tau & 3) ^ ((t32 >> 1) & 3);       // its 16-input chunk (physical chunk tau & 3 of row t32)
    const int kr = kappa(t32);                         // K row of that time within the step
    const uint32_t wr_off = static_cast<uint32_t>(kr * 64 + ((cl ^ ((kr >> 1) & 3)) << 4));
    const uint32_t rdJ = static_cast<uint32_t>(t32 * 64 + ((tau & 3) << 4));
    // when I == J the half comes from the I tile (128-byte rows, 128-byte swizzle)
    const uint32_t rdI = static_cast<uint32_t>(t32 * 128 + (((4 * static_cast<int>(rank) + cl) ^ (t32 & 7)) << 4));
    int sit = 0, ui = 0;
    bool ok = true;
    for (int it = 0; it < s.sched[0] && ok; ++it, ++ui) {
      const Item w = item_at(s.sched, it, L);
      const Unit t = decode_unit(w.u, L.p[w.p].per_chan, L.p[w.p].nt, rank);
      const bool own_diag = (t.ti == t.tj);
      // sums of the biased parts of the chunk's 16 inputs: byte lanes (at most
      // 4 x 4 x 15 = 240 between folds), then 16-bit lanes ([2k]: bytes 0 and
      // 2 of word k, [2k + 1]: bytes 1 and 3; at most 15 T / 32 per thread)
      uint32_t bP[4] = {0u, 0u, 0u, 0u}, bQ[4] = {0u, 0u, 0u, 0u};
      uint32_t hP[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u}, hQ[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
      int since_fold = 0;
      for (int ks = w.k0; ks < w.k1; ks += G::kSteps, ++sit) {
        const int rst = sit % kRawStages, ost = sit % kOpStages;
        if (!wait_or_abort(&s.raw_full[rst], (sit / kRawStages) & 1, lim, abort_flag)) {
          fail_all(s, L, kErrWaitRawFull);
          ok = false;
          break;
        }
        const uint32_t raw_s = smem_u32(s.raw + rst * G::kRawStage);
        const uint32_t src = own_diag ? raw_s + rdI : raw_s + G::kRawTile + rdJ;
        const uint32_t sstep = own_diag ? kRawSub : kRawSub / 2;
        uint4 v[G::kSteps];
#pragma unroll
        for (int sub = 0; sub < G::kSteps; ++sub) v[sub] = lds128(src + sub * sstep);
        release_raw_after_loads<4 * G::kSteps>(&v[0].x, &s.raw_empty[rst], lane);
        if (!wait_or_abort(&s.op_empty[ost], ((sit / kOpStages) & 1) ^ 1, lim, abort_flag)) {
          fail_all(s, L, kErrWaitOpEmpty);
          ok = false;
          break;
        }
        const uint32_t dst = smem_u32(s.op + ost * kOpStage) + wr_off;
#pragma unroll
        for (int sub = 0; sub < G::kSteps; ++sub) {
          const uint32_t x[4] = {v[sub].x, v[sub].y, v[sub].z, v[sub].w};
          uint32_t re[4], im[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            re[k] = biased_re(x[k]);
            im[k] = biased_im(x[k]);
            bP[k] += re[k];
            bQ[k] += im[k];
          }
          sts128(dst + sub * (32 * 64), re[0], re[1], re[2], re[3]);
          sts128(dst + kPlane + sub * (32 * 64), im[0], im[1], im[2], im[3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.op_full[ost]);
        if (++since_fold == 4 || ks + G::kSteps >= w.k1) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            hP[2 * k] += bP[k] & 0x00FF00FFu;
            hP[2 * k + 1] += (bP[k] >> 8) & 0x00FF00FFu;
            hQ[2 * k] += bQ[k] & 0x00FF00FFu;
            hQ[2 * k + 1] += (bQ[k] >> 8) & 0x00FF00FFu;
            bP[k] = bQ[k] = 0u;
          }
          since_fold = 0;
        }
      }
      if (!ok) break;
      // The 8 lanes of a warp that share a chunk differ by XOR 4, 9 and 18.
      // Two levels in 16-bit lanes (at most 4 x 15 T / 32 < 2^16 for T <=
      // 32768), then the values in 32 bits and the last level.
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        hP[k] += __shfl_xor_sync(0xFFFFFFFFu, hP[k], 4);
        hQ[k] += __shfl_xor_sync(0xFFFFFFFFu, hQ[k], 4);
        hP[k] += __shfl_xor_sync(0xFFFFFFFFu, hP[k], 9);
        hQ[k] += __shfl_xor_sync(0xFFFFFFFFu, hQ[k], 9);
      }
      int P[16], Q[16];   // input 4k + b of the chunk
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        P[4 * k + 0] = static_cast<int>(hP[2 * k] & 0xFFFFu);
        P[4 * k + 1] = static_cast<int>(hP[2 * k + 1] & 0xFFFFu);
        P[4 * k + 2] = static_cast<int>(hP[2 * k] >> 16);
        P[4 * k + 3] = static_cast<int>(hP[2 * k + 1] >> 16);
        Q[4 * k + 0] = static_cast<int>(hQ[2 * k] & 0xFFFFu);
        Q[4 * k + 1] = static_cast<int>(hQ[2 * k + 1] & 0xFFFFu);
        Q[4 * k + 2] = static_cast<int>(hQ[2 * k] >> 16);
        Q[4 * k + 3] = static_cast<int>(hQ[2 * k + 1] >> 16);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        P[e] += __shfl_xor_sync(0xFFFFFFFFu, P[e], 18);
        Q[e] += __shfl_xor_sync(0xFFFFFFFFu, Q[e], 18);
      }
      const int slot = ui & 1;
      if (!wait_or_abort(&s.sums_empty[slot], ((ui >> 1) & 1) ^ 1, lim, abort_flag)) {
        fail_all(s, L, kErrWaitSumsEmpty);
        break;
      }
      int* sl = s.sums + slot * kSlotInts + 2 * kTile + g * 2 * kHalf;   // this warp's block
      if (lane < 4) {   // lane c holds chunk c (lane >> 3 == 0)
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          sl[16 * lane + e] = P[e];
          sl[kHalf + 16 * lane + e] = Q[e];
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&s.sums_full[slot]);
        arrive_at(&s.sums_full[slot], peer);   // the partner's epilogue reads this half too
      }
    }
  } else if (EB == 2 && b_ordinal(warp) >= 0) {
    // ====================================================== B side (float16) -> K-major planes
    const int g = b_ordinal(warp);             // 16-input chunk within this CTA's half of J
    const int q = 4 * static_cast<int>(rank) + g;  // the same chunk within the J tile
    const int pj = lane >> 2;
    const int n0 = 16 * g + pj;                // B rows of inputs 2 pj and 2 pj + 1: n0, n0 + 8
    const int kq = lane & 3;                   // 8-byte K segment of each step
    int sit = 0, ui = 0;
    bool ok = true;
    for (int it = 0; it < s.sched[0] && ok; ++it, ++ui) {
      const Item w = item_at(s.sched, it, L);
      const Unit t = decode_unit(w.u, L.p[w.p].per_chan, L.p[w.p].nt, rank);
      const bool own_diag = (t.ti == t.tj);
      PairSums ps;
      ps.zero();
      int since_fold = 0;
      for (int ks = w.k0; ks < w.k1; ks += G::kSteps, ++sit) {
        const int rst = sit % kRawStages, ost = sit % kOpStages;
        if (!wait_or_abort(&s.raw_full[rst], (sit / kRawStages) & 1, lim, abort_flag)) {
          fail_all(s, L, kErrWaitRawFull);
          ok = false;
          break;
        }
        // this CTA's 64 J inputs: 64-byte rows of the half tile (chunk g at
        // g XOR ((t >> 1) & 3) in row t), or chunk q of the I tile when I == J
        const uint32_t raw_s = smem_u32(s.raw + rst * G::kRawStage);
        const uint32_t rowJ = own_diag ? raw_s + sw128(lane, q)
                                       : raw_s + G::kRawTile + lane * 64 + ((g ^ ((lane >> 1) & 3)) << 4);
        const uint32_t subJ = own_diag ? kRawSub : kRawSub / 2;
        uint32_t dv[G::kSteps][4];
#pragma unroll
        for (int sub = 0; sub < G::kSteps; ++sub)
          ldsm_x4_trans(rowJ + sub * subJ, dv[sub][0], dv[sub][1], dv[sub][2], dv[sub][3]);
        release_raw_after_loads<4 * G::kSteps>(&dv[0][0], &s.raw_empty[rst], lane);
        if (!wait_or_abort(&s.op_empty[ost], ((sit / kOpStages) & 1) ^ 1, lim, abort_flag)) {
          fail_all(s, L, kErrWaitOpEmpty);
          ok = false;
          break;
        }
        const uint32_t opB = smem_u32(s.op + ost * kOpStage);
#pragma unroll
        for (int sub = 0; sub < G::kSteps; ++sub) {
          const Words w = unpack_words(dv[sub], ps.bP, ps.bQ);
          // K-major rows n0 and n0 + 8 (same swizzle phase), the same K
          // positions as the A side
          const int kb0 = 64 * sub + 8 * kq, kb1 = kb0 + 32;
          const uint32_t o0 = static_cast<uint32_t>(n0 * 128 + (((kb0 >> 4) ^ (n0 & 7)) << 4) + (kb0 & 15));
          const uint32_t o1 = static_cast<uint32_t>(n0 * 128 + (((kb1 >> 4) ^ (n0 & 7)) << 4) + (kb1 & 15));
          sts64(opB + o0, f16_lo(w.re0), f16_hi(w.re0));
          sts64(opB + o1, f16_lo(w.re1), f16_hi(w.re1));
          sts64(opB + o0 + 8 * 128, f16_lo(w.re2), f16_hi(w.re2));
          sts64(opB + o1 + 8 * 128, f16_lo(w.re3), f16_hi(w.re3));
          sts64(opB + kPlane + o0, f16_lo(w.im0), f16_hi(w.im0));
          sts64(opB + kPlane + o1, f16_lo(w.im1), f16_hi(w.im1));
          sts64(opB + kPlane + o0 + 8 * 128, f16_lo(w.im2), f16_hi(w.im2));
          sts64(opB + kPlane + o1 + 8 * 128, f16_lo(w.im3), f16_hi(w.im3));
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.op_full[ost]);
        if (++since_fold == 2 || ks + G::kSteps >= w.k1) {
          ps.fold();
          since_fold = 0;
        }
      }
      if (!ok) break;
      ps.reduce();
      const int slot = ui & 1;
      if (!wait_or_abort(&s.sums_empty[slot], ((ui >> 1) & 1) ^ 1, lim, abort_flag)) {
        fail_all(s, L, kErrWaitSumsEmpty);
        break;
      }
      int* sl = s.sums + slot * kSlotInts + 2 * kTile;
      if ((lane & 3) == 0) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int j = 16 * g + 2 * pj + e;    // input offset within this CTA's half
          sl[j] = ps.P[e];
          sl[kHalf + j] = ps.Q[e];
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&s.sums_full[slot]);
        arrive_at(&s.sums_full[slot], peer);   // the partner's epilogue reads this half too
      }
    }
  } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {
    // ====================================================== epilogue
    // Never leaves the unit loop early (the named barriers below must be
    // reached equally often by all four warps); after an abort it only
    // skips work.
    const int quad = warp & 3;
    const int lr = 32 * quad + lane;                 // TMEM lane = accumulator row; also a column index
    const int il = lane_to_input(lr);                // input offset of row lr in its tile
    const int jl = col_to_input<EB>(lr);             // input offset of column lr in its tile
    int* const sre = s.stage + quad * 2 * kStageBufs * kStageChunk;   // this warp's staged real parts
    int* const sim = sre + kStageBufs * kStageChunk;                   // and imaginary parts
    bool ok = true;
    int ui = 0;
    for (int it = 0; it < s.sched[0]; ++it, ++ui) {
      const Item w = item_at(s.sched, it, L);
      const ProbDev& P = L.p[w.p];
      const Unit t = decode_unit(w.u, P.per_chan, P.nt, rank);
      const long long nbl = static_cast<long long>(P.N) * (P.N + 1) / 2;
      const int T_pad = (w.k1 - w.k0) * kStep;
      const int slot = ui & 1;
      if (ok && !wait_or_abort(&s.sums_full[slot], (ui >> 1) & 1, lim, abort_flag)) {
        fail_all(s, L, kErrWaitSumsFull);
        ok = false;
      }
      const int* sl = s.sums + slot * kSlotInts;
      float row_re = 0.f, row_im = 0.f;
      if (ok) {
        // bias corrections of this lane's row and of column lr (see unbias)
        row_re = static_cast<float>(-8 * (sl[il] + sl[kTile + il]) + 128 * T_pad);
        row_im = static_cast<float>(8 * (sl[il] - sl[kTile + il]));
        // column lr is J input jl; its half (lr / 64) is held by CTA lr / 64,
        // whose B-side warps each left partial sums in a block of their own
        const uint32_t holder = static_cast<uint32_t>(lr >> 6);
        const int jo = jl - kHalf * static_cast<int>(holder);
        const int* pq = sl + 2 * kTile;
        int pjv = 0, qjv = 0;
#pragma unroll
        for (int b = 0; b < kBWarps; ++b) {
          const int* blk = pq + b * 2 * kHalf;
          pjv += holder == rank ? blk[jo] : ld_peer(blk + jo, holder);
          qjv += holder == rank ? blk[kHalf + jo] : ld_peer(blk + kHalf + jo, holder);
        }
        s.colcorr[lr] = static_cast<float>(-8 * (pjv + qjv));
        s.colcorr[kTile + lr] = static_cast<float>(-8 * (pjv - qjv));
      }
      if (w.lo < 0) {
        // packed-triangle offsets of row lr's and column lr's inputs (N <= 8192 fits int)
        const int gi = t.ti * kTile + il, gj = t.tj * kTile + jl;
        s.rowoff[lr] = gi < P.N ? gi * (gi + 1) / 2 : 0;
        s.coloff[lr] = gj < P.N ? gj * (gj + 1) / 2 : 0;
      } else {
        // a part: rows of the compact workspace tile, in accumulator-row
        // order (a transposed part's rows are J inputs: row input_to_lane(jl))
        s.rowoff[lr] = lr * kTile;
        s.coloff[lr] = input_to_lane(jl) * kTile;
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (lane == 0) {   // this slot's own sums and the partner's half of J have been read
        arrive_relaxed_at(&s.sums_empty[slot], rank);
        arrive_relaxed_at(&s.sums_empty[slot], peer);
      }
      if (ok && !wait_or_abort(s.acc_full, ui & 1, lim, abort_flag)) {
        fail_all(s, L, kErrWaitAccFull);
        ok = false;
      }
      ok = __all_sync(0xFFFFFFFFu, ok);
      bool released = false;
      if (ok && t.write) {
        tc_fence_after();
        const uint32_t t_row = tmem + (static_cast<uint32_t>(32 * quad) << 16);
        // D leaves tensor memory first, D_re and then D_im, each released as
        // soon as it is read (the MMA starts the next unit's real parts in
        // between): chunks 0-2 (32 columns each) as raw bits into shared
        // staging, chunk 3 into registers (vb: re, va: im).  The bias removal
        // and global writes run while the MMA works on the next unit.
        uint32_t va[32], vb[32];
        tmem_ld32(t_row, va);
        tmem_ld32(t_row + 32, vb);
        tmem_ld_wait();
        stage_raw(sre, va, lane);
        stage_raw(sre + kStageChunk, vb, lane);
        tmem_ld32(t_row + 64, va);
        tmem_ld32(t_row + 96, vb);
        tmem_ld_wait();
        // D_re is in registers and staging: release it before staging chunk 2
        tc_fence_before();
        __syncwarp();
        if (lane == 0) arrive_relaxed_at(s.acc_empty, 0);
        stage_raw(sre + 2 * kStageChunk, va, lane);
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
          tmem_ld32(t_row + 128 + 32 * b, va);
          tmem_ld_wait();
          if (b < kStageBufs) stage_raw(sim + kStageChunk * b, va, lane);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) arrive_relaxed_at(s.acc_empty_im, 0);
        released = true;
        // a part goes to its workspace slot (stored, never added): the tile's
        // first column input then lands on column 0
        const int accumulate = w.lo < 0 ? P.accumulate : 0;
        int2* const acc =
            w.lo < 0 ? reinterpret_cast<int2*>(P.acc) + static_cast<long long>(t.c) * nbl
                     : L.split_ws + (static_cast<long long>(2 * cl + rank) * kSplitTile -
                                       (t.transposed ? t.ti : t.tj) * kTile);
        // the buffer written, for the debug build's index checks
        const int2* const wbase = w.lo < 0 ? reinterpret_cast<const int2*>(P.acc) : L.split_ws;
        const long long wlen = w.lo < 0 ? P.acc_pairs : L.ws_pairs;
        // a tile strictly below the diagonal and inside N needs no checks
        const bool full = !t.transposed && t.ti > t.tj && t.ti * kTile + kTile <= P.N;
        // A diagonal tile inside N, by 32 x 32 blocks: this warp's rows are
        // inputs [32 quad, 32 quad + 32) of the tile and column chunk b holds
        // inputs [32 b, 32 b + 32), so chunks b < quad lie wholly below the
        // diagonal (written without checks), b > quad wholly above it
        // (nothing to write) and only b == quad needs the per-element test.
        const bool diag_in = !t.transposed && t.ti == t.tj && t.ti * kTile + kTile <= P.N;
        const bool tfull = t.transposed && t.tj * kTile + kTile <= P.N;
        const int gI = t.ti * kTile + il;           // this lane's row input
        const int* ro = s.rowoff + 32 * quad;
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
          const int cc = 32 * b;
          const int* sb = sre + (b == 3 ? 0 : b) * kStageChunk;
          if (b == 3) {  // buffer 0 has been written out: chunk 3 goes there
            __syncwarp();
            stage_raw(sre, vb, lane);
            stage_raw(sim, va, lane);
          }
          __syncwarp();
          if (diag_in && b > quad) {
            // above the diagonal: nothing of this chunk is written
          } else if (!t.transposed) {
            // 32 rows x 32 baselines: each row is 256 contiguous bytes (lanes
            // permuted); row r's corrections come from lane r
            const int gj = t.tj * kTile + col_to_input<EB>(cc + lane);
            const float cre = s.colcorr[cc + lane], cim = s.colcorr[kTile + cc + lane];
            int2* accj = acc + gj;
            const bool unchecked = full || (diag_in && b < quad);
            if (unchecked && !accumulate) {
              // row r's offset comes from lane r by shuffle, and the staged
              // values of 8 rows are read before their 8 stores
              const int rof = ro[lane];
#pragma unroll 1
              for (int r0 = 0; r0 < 32; r0 += 8) {
                int2 sv[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) sv[q] = staged(sb, r0 + q, lane);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                  const int r = r0 + q;
                  const float rre = __shfl_sync(0xFFFFFFFFu, row_re, r), rim = __shfl_sync(0xFFFFFFFFu, row_im, r);
                  int2* dst = accj + __shfl_sync(0xFFFFFFFFu, rof, r);
                  if (debug_in_bounds(dst, wbase, wlen, P.err)) *dst = unbias<EB>(sv[q], rre, rim, cre, cim);
                }
              }
            } else if (unchecked) {
#pragma unroll 4
              for (int r = 0; r < 32; ++r) {
                const float rre = __shfl_sync(0xFFFFFFFFu, row_re, r), rim = __shfl_sync(0xFFFFFFFFu, row_im, r);
                const int2 v = unbias<EB>(staged(sb, r, lane), rre, rim, cre, cim);
                int2* dst = accj + ro[r];
                if (debug_in_bounds(dst, wbase, wlen, P.err)) {
                  const int2 o = *dst;
                  *dst = make_int2(o.x + v.x, o.y + v.y);
                }
              }
            } else {
#pragma unroll 4
              for (int r = 0; r < 32; ++r) {
                const float rre = __shfl_sync(0xFFFFFFFFu, row_re, r), rim = __shfl_sync(0xFFFFFFFFu, row_im, r);
                const int gi = t.ti * kTile + lane_to_input(32 * quad + r);
                if (gi < P.N && gj <= gi) {
                  const int2 v = unbias<EB>(staged(sb, r, lane), rre, rim, cre, cim);
                  int2* dst = accj + ro[r];
                  if (!debug_in_bounds(dst, wbase, wlen, P.err)) continue;
                  if (accumulate) {
                    const int2 o = *dst;
                    *dst = make_int2(o.x + v.x, o.y + v.y);
                  } else {
                    *dst = v;
                  }
                }
              }
            }
          } else {
            // transposed block: column cc + k is output row j, this lane's row
            // input gI < j its column; the 32 lanes write 32 consecutive
            // inputs of that row, conjugated
            int2* acci = acc + gI;
            // column k's corrections, output-row offset and presence are held
            // by lane k and broadcast by shuffles: read per k from shared
            // memory between the stores, they made this loop three times
            // slower than the row-wise one
            const float ccre = s.colcorr[cc + lane], ccim = s.colcorr[kTile + cc + lane];
            const int cco = s.coloff[cc + lane];
            const unsigned colok =
                tfull ? 0xFFFFFFFFu
                      : __ballot_sync(0xFFFFFFFFu, t.tj * kTile + col_to_input<EB>(cc + lane) < P.N);
            if (!accumulate) {
#pragma unroll 8
              for (int k = 0; k < 32; ++k) {
                const float cre = __shfl_sync(0xFFFFFFFFu, ccre, k), cim = __shfl_sync(0xFFFFFFFFu, ccim, k);
                const int co = __shfl_sync(0xFFFFFFFFu, cco, k);
                if ((colok >> k) & 1u) {
                  const int2 v = unbias<EB>(staged(sb, lane, k), row_re, row_im, cre, cim);
                  int2* dst = acci + co;
                  if (debug_in_bounds(dst, wbase, wlen, P.err)) *dst = make_int2(v.x, -v.y);
                }
              }
            } else {
#pragma unroll 8
              for (int k = 0; k < 32; ++k) {
                const float cre = __shfl_sync(0xFFFFFFFFu, ccre, k), cim = __shfl_sync(0xFFFFFFFFu, ccim, k);
                const int co = __shfl_sync(0xFFFFFFFFu, cco, k);
                if ((colok >> k) & 1u) {
                  const int2 v = unbias<EB>(staged(sb, lane, k), row_re, row_im, cre, cim);
                  int2* dst = acci + co;
                  if (debug_in_bounds(dst, wbase, wlen, P.err)) {
                    const int2 o = *dst;
                    *dst = make_int2(o.x + v.x, o.y - v.y);
                  }
                }
              }
            }
          }
        }
        __syncwarp();
      }
      if (!released) {
        // nothing (more) to read from D for this unit
        if (ok) tc_fence_after();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          arrive_relaxed_at(s.acc_empty, 0);
          arrive_relaxed_at(s.acc_empty_im, 0);
        }
      }
      // all four warps are done with colcorr, rowoff, coloff and staging
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
  }

  // Teardown: every MMA of the pair has completed (both CTAs' tensor memory
  // and shared memory are read by it) before either CTA frees or leaves.
  if (warp == 1 && lane == 0) {
    if (!mbar_wait(s.final_bar, 0, lim))
      for (int k = 0; k < (NP == 1 ? 1 : L.nprob); ++k) atomicOr(L.p[k].err, kErrWaitFinal);
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols));
  }
}

// Sum of the time-sliced parts of the leftover units.  Block (x, y): x =
// leftover unit l (x / 2) and CTA rank of its pair (x % 2), y = group of 8
// accumulator rows of that CTA's tile; each warp takes one row.  The q parts
// of unit l are in the workspace slots of clusters l q .. l q + q - 1.
struct CombineParams {
  int N, nt, per_chan, units, ncl, q, accumulate;
  int32_t* acc;
  const int2* ws;
  long long acc_pairs, ws_pairs;   // element counts, for the debug build's index checks
  int* err;
};

__global__ void __launch_bounds__(256) split_combine_kernel(const CombineParams p) {
  const int l = blockIdx.x >> 1, rank = blockIdx.x & 1;
  const Unit t = decode_unit(p.units - p.units % p.ncl + l, p.per_chan, p.nt, rank);
  if (!t.write) return;
  // the output tile: rows Rt * 128 + lane_to_input(a), columns Ct * 128 + b, j <= i < N
  const int Rt = t.transposed ? t.tj : t.ti, Ct = t.transposed ? t.ti : t.tj;
  const int a = 8 * blockIdx.y + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int gi = Rt * kTile + lane_to_input(a);
  if (gi >= p.N) return;
  int2* orow = reinterpret_cast<int2*>(p.acc) + static_cast<long long>(t.c) * p.N * (p.N + 1) / 2 + gi * (gi + 1) / 2;
  int sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
  for (int c = l * p.q; c < (l + 1) * p.q; ++c) {
    const int2* src = p.ws + static_cast<long long>(2 * c + rank) * kSplitTile + a * kTile;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!debug_in_bounds(src + lane + 32 * k, p.ws, p.ws_pairs, p.err)) continue;
      const int2 v = src[lane + 32 * k];
      sx[k] += v.x;
      sy[k] += v.y;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int gj = Ct * kTile + lane + 32 * k;
    if (gj > gi) break;
    int2* d = orow + gj;
    if (!debug_in_bounds(d, reinterpret_cast<const int2*>(p.acc), p.acc_pairs, p.err)) continue;
    if (p.accumulate) {
      const int2 o = *d;
      *d = make_int2(o.x + sx[k], o.y + sy[k]);
    } else {
      *d = make_int2(sx[k], sy[k]);
    }
  }
}

}  // namespace tc8

int tc8_smem_bytes(int eb) { return eb == 1 ? tc8::Geo<1>::kSmemBytes : tc8::Geo<2>::kSmemBytes; }

namespace {
// Clusters (pairs of SMs) of the pair kernel that can be resident at once,
// asked once per process and operand width.
template <int EB, int NP>
int resident_clusters() {
  static int n = -1;
  if (n < 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(tc8::kThreads, 1, 1);
    cfg.dynamicSmemBytes = tc8::Geo<EB>::kSmemBytes;
    int r = 0;
    if (cudaOccupancyMaxActiveClusters(&r, tc8::xcorr_tc8_kernel<EB, NP>, &cfg) != cudaSuccess || r < 1) {
      cudaGetLastError();
      r = 0;
    }
    n = r;
  }
  return n;
}

// Problem k of a launch description from a plan's parameters.
template <int NP>
void set_problem(tc8::PairLaunch<NP>& L, int k, const CUtensorMap& ti, const CUtensorMap& tj, const TcParams& prm) {
  L.ti[k] = ti;
  L.tj[k] = tj;
  tc8::ProbDev& d = L.p[k];
  d.acc = prm.acc;
  d.err = prm.err;
  d.acc_pairs = static_cast<long long>(prm.C) * prm.N * (prm.N + 1) / 2;
  d.N = prm.N;
  d.nt = prm.nt;
  d.per_chan = tc8::pairs_per_channel(prm.nt);
  d.nks = prm.nks;
  d.accumulate = prm.accumulate;
}

template <int EB, int NP>
cudaError_t launch_table(tc8::PairLaunch<NP>& L, long long units, int max_ctas, cudaStream_t stream,
                         long long* clusters_out) {
  constexpr int smem = tc8::Geo<EB>::kSmemBytes;
  cudaError_t e =
      cudaFuncSetAttribute(tc8::xcorr_tc8_kernel<EB, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (units > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  L.units = static_cast<int>(units);
  long long clusters = max_ctas / 2;
  const int res = resident_clusters<EB, NP>();
  if (res > 0 && res < clusters) clusters = res;
  if (units < clusters) clusters = units;
  if (clusters < 1) clusters = 1;
  *clusters_out = clusters;
  L.split_parts = L.split_ws ? tc8::split_parts(units, clusters, L.p[0].nks, tc8::Geo<EB>::kSteps) : 0;
  tc8::xcorr_tc8_kernel<EB, NP><<<static_cast<int>(2 * clusters), tc8::kThreads, smem, stream>>>(L);
  return cudaGetLastError();
}

template <int EB>
cudaError_t launch_pair(const CUtensorMap* tmap_i, const CUtensorMap* tmap_j, TcParams prm, int max_ctas,
                        cudaStream_t stream, int* kernels) {
  *kernels = 0;
  tc8::PairLaunch<1> L = {};
  L.nprob = 1;
  set_problem(L, 0, *tmap_i, *tmap_j, prm);
  const long long units = static_cast<long long>(prm.C) * L.p[0].per_chan;
  L.prefix[0] = 0;
  L.prefix[1] = static_cast<int>(units < 0x7FFFFFFFLL ? units : 0x7FFFFFFFLL);
  L.split_ws = prm.split_ws;
  L.ws_pairs = prm.split_ws ? static_cast<long long>(split_workspace_bytes(max_ctas) / sizeof(int2)) : 0;
  L.timeout_ns = prm.timeout_ns;
  long long clusters = 0;
  cudaError_t e = launch_table<EB, 1>(L, units, max_ctas, stream, &clusters);
  if (e != cudaSuccess) return e;
  *kernels = 1;
  if (L.split_parts > 0) {
    tc8::CombineParams q;
    q.N = prm.N;
    q.nt = prm.nt;
    q.per_chan = L.p[0].per_chan;
    q.units = L.units;
    q.ncl = static_cast<int>(clusters);
    q.q = L.split_parts;
    q.accumulate = prm.accumulate;
    q.acc = prm.acc;
    q.ws = prm.split_ws;
    q.acc_pairs = L.p[0].acc_pairs;
    q.ws_pairs = L.ws_pairs;
    q.err = prm.err;
    const int Lft = static_cast<int>(units % clusters);
    tc8::split_combine_kernel<<<dim3(2 * Lft, tc8::kTile / 8), 256, 0, stream>>>(q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *kernels = 2;
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_xcorr_pair(int eb, const CUtensorMap* tmap_i, const CUtensorMap* tmap_j, const TcParams& prm,
                              int max_ctas, cudaStream_t stream, int* kernels) {
  return eb == 1 ? launch_pair<1>(tmap_i, tmap_j, prm, max_ctas, stream, kernels)
                 : launch_pair<2>(tmap_i, tmap_j, prm, max_ctas, stream, kernels);
}

cudaError_t launch_xcorr_batch(const BatchProblem* probs, int n, int max_ctas, cudaStream_t stream, int* kernels) {
  *kernels = 0;
  if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
  tc8::PairLaunch<kMaxBatch> L = {};
  L.nprob = n;
  long long units = 0;
  for (int k = 0; k < n; ++k) {
    if (probs[k].prm.split_ws != nullptr || probs[k].prm.nks > 32768 / tc8::kStep) return cudaErrorInvalidValue;
    set_problem(L, k, probs[k].ti, probs[k].tj, probs[k].prm);
    L.prefix[k] = static_cast<int>(units);
    units += static_cast<long long>(probs[k].prm.C) * L.p[k].per_chan;
    if (units > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  }
  L.prefix[n] = static_cast<int>(units);
  L.split_ws = nullptr;
  L.ws_pairs = 0;
  L.timeout_ns = probs[0].prm.timeout_ns;
  long long clusters = 0;
  cudaError_t e = launch_table<1, kMaxBatch>(L, units, max_ctas, stream, &clusters);
  if (e == cudaSuccess) *kernels = 1;
  return e;
}

}  // namespace xe
