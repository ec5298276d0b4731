// Gain calibration on the X-engine's visibilities: weighted chi^2 and its
// hand-written adjoint.
//
//   r_ij = V_ij - g_i conj(g_j) C_ij           (packed lower triangle, i >= j)
//   chi2 = sum_c sum_{i>=j} w_ij |r_ij|^2
//   grad_k = dchi2/dRe g_k + i dchi2/dIm g_k = 2 dchi2/d conj(g_k)
//          = -2 [ sum_{j<=k} w_kj r_kj g_j conj(C_kj) + sum_{i>=k} w_ik conj(r_ik) g_i C_ik ]
//
// One pass over the triangle (calib_pass_kernel) computes the partial sums of
// chi^2, of the gradient, or of both: HBM-bound (each baseline's V and C, 8
// bytes each, and w, 4 bytes, are read once).  A small second kernel
// (calib_combine_kernel) adds the partials in a fixed order.  Per-baseline
// terms are float32.  chi^2 is summed in float32 with a compensation term
// (TwoSum, Knuth) per thread, across the warp and over the warps' partials
// in calib_combine_kernel; float64 is used only for the final sum of that
// kernel's 8 warp totals.  The gradient is summed in
// float32.  Every summation order is fixed by the problem size and the grid,
// so both results are deterministic.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "xe_kernels.h"

namespace xe {
namespace cal {

// Work decomposition.  Channel c's triangle is cut into 64 x 64 tiles (band
// b of rows [64 b, 64 b + 64), stripe s of columns [64 s, 64 s + 64), s <= b);
// a row segment (c, b, s, i) is row i of tile (b, s).  All segments, in the
// order (c, b, s, i), are split into equal contiguous ranges, one per warp
// of a persistent grid, so every warp streams the same number of bytes.  In
// this order the tiles of one band, which share the memory lines where a
// row crosses from one stripe to the next, are streamed by neighbouring
// warps at the same time, so those lines are fetched from HBM once.
constexpr int kStripe = 64;   // columns per segment; lane owns j0 = 64 s + lane and j1 = j0 + 32
// Defaults measured best on B300 for 512 inputs x 128 channels: 16 warps per
// CTA, two CTAs per SM (64 registers), groups of two segments, two groups in
// flight per warp.
#ifndef XE_CAL_WARPS
#define XE_CAL_WARPS 16
#endif
#ifndef XE_CAL_GROUP
#define XE_CAL_GROUP 2
#endif
#ifndef XE_CAL_RING
#define XE_CAL_RING 2
#endif
#ifndef XE_CAL_MINB
#define XE_CAL_MINB 2
#endif
constexpr int kWarps = XE_CAL_WARPS;
constexpr int kThreads = kWarps * 32;
constexpr int kGroup = XE_CAL_GROUP;   // segments per group (one transposed warp reduction): 2 or 4
constexpr int kRing = XE_CAL_RING;     // groups in a warp's shared-memory ring
constexpr int kMinBlocks = XE_CAL_MINB;
static_assert(kGroup == 2 || kGroup == 4, "group of 2 or 4 segments");

__host__ __device__ __forceinline__ long long band_prefix(long long b) {
  return 32 * b * (b + 1);   // segments of bands 0 .. b-1 of one channel (all but the last band are full)
}

struct Geometry {
  int N, C, S, W;      // inputs, channels, stripes (= bands) per channel, warps in the grid
  int T;               // tiles per channel, S (S + 1) / 2
  long long nbl;       // baselines per channel, N (N + 1) / 2
  long long P, L;      // segments per channel, in total
  int sparse;          // more warps than segments: some warps have none
  __host__ __device__ long long begin(long long w) const { return L * w / W; }   // warp w: [begin(w), begin(w+1))
  __host__ __device__ int warp_of(long long x) const { return static_cast<int>(((x + 1) * W - 1) / L); }
};

struct Scratch {
  float2* chi_part;    // [W]   chi^2 per warp: float32 sum and its compensation
  float2* row_part;    // [C][S][N] row sums per (stripe, row)
  float2* col_part;    // [C T + W][64] column sums of warp w for tile gt (= c T + tile) at row w + gt
                       // (unique: a later warp never touches an earlier tile)
  int2* tile_w;        // [C T] first and last warp that computed a row of tile gt
};

// Asynchronous 8- and 4-byte global -> shared copies (cp.async, L1-cached),
// issued only where pred is non-zero.
__device__ __forceinline__ void cp_async8(uint32_t smem, const void* gmem, int pred) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p cp.async.ca.shared.global [%0], [%1], 8;\n}\n" ::"r"(smem),
      "l"(gmem), "r"(pred)
      : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t smem, const void* gmem, int pred) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p cp.async.ca.shared.global [%0], [%1], 4;\n}\n" ::"r"(smem),
      "l"(gmem), "r"(pred)
      : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kPending) : "memory");
}

// One row segment in shared memory: V, C, w of its 64 columns and g_i.
struct Seg {
  float2 v[kStripe];
  float2 m[kStripe];
  float w[kStripe];
  float2 gi;
  float2 pad;
};

// Tile position shared by both cursors: channel c, band b, stripe s, row i,
// and the end of the band's rows.
struct TilePos {
  int c, b, s, i, bend;
  // Moves to the next tile; returns true when the channel changed.
  __device__ __forceinline__ bool next_tile(const Geometry& G) {
    bool chan = false;
    if (++s > b) {
      s = 0;
      if (++b == G.S) {
        b = 0;
        ++c;
        chan = true;
      }
      bend = min(b * kStripe + kStripe, G.N);
    }
    i = b * kStripe;
    return chan;
  }
  __device__ __forceinline__ long long tile(const Geometry& G) const {
    return static_cast<long long>(c) * G.T + b * (b + 1) / 2 + s;
  }
};

__device__ __forceinline__ TilePos decode(long long x, const Geometry& G) {
  TilePos t;
  t.c = static_cast<int>(x / G.P);
  const long long rem = x - static_cast<long long>(t.c) * G.P;
  int b = 0;
  while (b + 1 < G.S && band_prefix(b + 1) <= rem) ++b;
  const int rows = min(kStripe, G.N - b * kStripe);
  const int o = static_cast<int>(rem - band_prefix(b));
  t.b = b;
  t.s = o / rows;
  t.i = b * kStripe + (o - t.s * rows);
  t.bend = b * kStripe + rows;
  return t;
}

// Terms of one baseline (row i, column j) for one lane:
//   r = V - g_i C conj(g_j);  chi += w |r|^2;
//   rowt += -w r g_j conj(C)  (belongs to g_i);  col += -w conj(r) g_i C  (belongs to g_j).
template <bool kChi, bool kGrad>
__device__ __forceinline__ void baseline_terms(float2 v, float2 m, float wt, float2 gi, float2 gj, float& chi,
                                               float2& rowt, float2& col) {
  const float amx = fmaf(gi.x, m.x, -gi.y * m.y);     // a = g_i C
  const float amy = fmaf(gi.x, m.y, gi.y * m.x);
  const float rx = fmaf(-amx, gj.x, fmaf(-amy, gj.y, v.x));
  const float ry = fmaf(-amy, gj.x, fmaf(amx, gj.y, v.y));
  const float wrx = wt * rx, wry = wt * ry;
  if (kChi) chi = fmaf(wrx, rx, fmaf(wry, ry, chi));
  if (kGrad) {
    const float bx = fmaf(gj.x, m.x, gj.y * m.y);     // b = g_j conj(C)
    const float by = fmaf(gj.y, m.x, -gj.x * m.y);
    rowt.x = fmaf(-wrx, bx, fmaf(wry, by, rowt.x));
    rowt.y = fmaf(-wrx, by, fmaf(-wry, bx, rowt.y));
    col.x = fmaf(-wrx, amx, fmaf(-wry, amy, col.x));
    col.y = fmaf(-wrx, amy, fmaf(wry, amx, col.y));
  }
}

// Sum of 2 row values over the warp, transposed: afterwards lanes 16t ..
// 16t+15 hold the sum of x[t] over all 32 lanes.
__device__ __forceinline__ float reduce2(float x0, float x1, int lane) {
  const bool hi = lane & 16;
  float z = (hi ? x1 : x0) + __shfl_xor_sync(0xFFFFFFFFu, hi ? x0 : x1, 16);
  z += __shfl_xor_sync(0xFFFFFFFFu, z, 8);
  z += __shfl_xor_sync(0xFFFFFFFFu, z, 4);
  z += __shfl_xor_sync(0xFFFFFFFFu, z, 2);
  z += __shfl_xor_sync(0xFFFFFFFFu, z, 1);
  return z;
}

// Sum of 4 row values over the warp, transposed: afterwards lanes 8t .. 8t+7
// hold the sum of x[t] over all 32 lanes.
__device__ __forceinline__ float reduce4(float x0, float x1, float x2, float x3, int lane) {
  const bool hi = lane & 16;
  const float k0 = hi ? x2 : x0, k1 = hi ? x3 : x1;
  const float s0 = hi ? x0 : x2, s1 = hi ? x1 : x3;
  const float y0 = k0 + __shfl_xor_sync(0xFFFFFFFFu, s0, 16);
  const float y1 = k1 + __shfl_xor_sync(0xFFFFFFFFu, s1, 16);
  const bool b8 = lane & 8;
  float z = (b8 ? y1 : y0) + __shfl_xor_sync(0xFFFFFFFFu, b8 ? y0 : y1, 8);
  z += __shfl_xor_sync(0xFFFFFFFFu, z, 4);
  z += __shfl_xor_sync(0xFFFFFFFFu, z, 2);
  z += __shfl_xor_sync(0xFFFFFFFFu, z, 1);
  return z;
}

// Compensated float32 sum (Knuth's TwoSum): after add(x), s + c equals the
// exact sum of everything added, up to the rounding of c's own additions.
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
  }
  // this lane's (s, c) plus the partner lane's at XOR distance o
  __device__ __forceinline__ void add_lane(int o) {
    const float ps = __shfl_xor_sync(0xFFFFFFFFu, s, o), pc = __shfl_xor_sync(0xFFFFFFFFu, c, o);
    c += pc;
    add(ps);
  }
};

template <bool kChi, bool kGrad, bool kW>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
calib_pass_kernel(const float2* __restrict__ g, const float2* __restrict__ model, const float2* __restrict__ vobs,
                  const float* __restrict__ wts, Geometry G, int include_autos, Scratch sc) {
  __shared__ Seg ring[kWarps][kRing * kGroup];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.x * kWarps + warp;
  const long long x_begin = G.begin(w), x_end = G.begin(w + 1);
  const int n = static_cast<int>(x_end - x_begin);
  const uint32_t ring_base = static_cast<uint32_t>(__cvta_generic_to_shared(ring[warp]));

  // ---- issue side: cp.async of each segment's V, C, w (the lane's two
  // columns) and g_i (lane 0), walking the segments with its own cursor.
  TilePos ip = decode(x_begin, G);
  int ioff = ip.i * (ip.i + 1) / 2 + ip.s * kStripe;   // element of (row i, column 64 s) within the channel
  const float2* vc = vobs + static_cast<long long>(ip.c) * G.nbl;
  const float2* mc = model + static_cast<long long>(ip.c) * G.nbl;
  const float* wc = kW ? wts + static_cast<long long>(ip.c) * G.nbl : nullptr;
  const float2* gci = g + static_cast<long long>(ip.c) * G.N;

  // Below the diagonal (s < b) all 64 columns of a segment are present; only
  // the diagonal tiles need per-column predicates.
  auto issue_seg = [&](int slot) {
    const uint32_t sb = ring_base + slot * static_cast<uint32_t>(sizeof(Seg));
    const float2* pv = vc + ioff + lane;
    const float2* pm = mc + ioff + lane;
    int a0 = 1, a1 = 1;
    if (ip.s == ip.b) {
      const int j0 = ip.s * kStripe + lane, j1 = j0 + 32;
      a0 = j0 < G.N && j0 <= ip.i && (j0 != ip.i || include_autos);
      a1 = j1 < G.N && j1 <= ip.i && (j1 != ip.i || include_autos);
    }
    cp_async8(sb + offsetof(Seg, v) + 8 * lane, pv, a0);
    cp_async8(sb + offsetof(Seg, v) + 8 * lane + 256, pv + 32, a1);
    cp_async8(sb + offsetof(Seg, m) + 8 * lane, pm, a0);
    cp_async8(sb + offsetof(Seg, m) + 8 * lane + 256, pm + 32, a1);
    if (kW) {
      const float* pw = wc + ioff + lane;
      cp_async4(sb + offsetof(Seg, w) + 4 * lane, pw, a0);
      cp_async4(sb + offsetof(Seg, w) + 4 * lane + 128, pw + 32, a1);
    }
    cp_async8(sb + offsetof(Seg, gi), gci + ip.i, lane == 0);
    if (++ip.i < ip.bend) {          // next row of the tile: its row starts i elements later
      ioff += ip.i;
    } else {
      if (ip.next_tile(G)) {
        vc += G.nbl;
        mc += G.nbl;
        if (kW) wc += G.nbl;
        gci += G.N;
      }
      ioff = ip.i * (ip.i + 1) / 2 + ip.s * kStripe;
    }
  };
  auto issue_group = [&](int grp) {
    const int slot0 = (grp % kRing) * kGroup;
    if ((grp + 1) * kGroup <= n) {
#pragma unroll
      for (int r = 0; r < kGroup; ++r) issue_seg(slot0 + r);
    } else {
      for (int r = 0; grp * kGroup + r < n; ++r) issue_seg(slot0 + r);
    }
    cp_async_commit();
  };

#pragma unroll
  for (int q = 0; q < kRing; ++q) issue_group(q);

  // ---- compute side
  TilePos cp = decode(x_begin, G);
  float2* rpc = sc.row_part + (static_cast<long long>(cp.c) * G.S + cp.s) * G.N;   // row_part of (c, s)
  long long col_gt = cp.tile(G);
  // column accumulators (columns j0 = 64 s + lane, j1 = j0 + 32) of the tile being computed
  float2 col0 = make_float2(0.f, 0.f), col1 = make_float2(0.f, 0.f);
  float2 gj0 = make_float2(0.f, 0.f), gj1 = make_float2(0.f, 0.f);
  auto load_gj = [&]() {
    const int j0 = cp.s * kStripe + lane, j1 = j0 + 32;
    const float2* gc = g + static_cast<long long>(cp.c) * G.N;
    gj0 = j0 < G.N ? gc[j0] : make_float2(0.f, 0.f);
    gj1 = j1 < G.N ? gc[j1] : make_float2(0.f, 0.f);
  };
  if (n > 0) load_gj();
  CompSum chi_acc;

  const int groups = (n + kGroup - 1) / kGroup;
  for (int grp = 0; grp < groups; ++grp) {
    cp_async_wait<kRing - 1>();
    __syncwarp();
    float rre[kGroup], rim[kGroup], chi_g[kGroup];
    float2* rdst[kGroup];
#pragma unroll
    for (int r = 0; r < kGroup; ++r) {
      rre[r] = rim[r] = chi_g[r] = 0.f;
      rdst[r] = nullptr;
      if (grp * kGroup + r < n) {                  // warp-uniform
        const Seg& sl = ring[warp][(grp % kRing) * kGroup + r];
        const float2 gi = sl.gi;
        float2 rowt = make_float2(0.f, 0.f);
        if (cp.s < cp.b) {
          baseline_terms<kChi, kGrad>(sl.v[lane], sl.m[lane], kW ? sl.w[lane] : 1.0f, gi, gj0, chi_g[r], rowt,
                                      col0);
          baseline_terms<kChi, kGrad>(sl.v[lane + 32], sl.m[lane + 32], kW ? sl.w[lane + 32] : 1.0f, gi, gj1,
                                      chi_g[r], rowt, col1);
        } else {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int jl = h * 32 + lane, j = cp.s * kStripe + jl;
            const bool a = j < G.N && j <= cp.i && (j != cp.i || include_autos);
            const float2 v = a ? sl.v[jl] : make_float2(0.f, 0.f);
            const float2 m = a ? sl.m[jl] : make_float2(0.f, 0.f);
            const float wt = a ? (kW ? sl.w[jl] : 1.0f) : 0.f;
            baseline_terms<kChi, kGrad>(v, m, wt, gi, h ? gj1 : gj0, chi_g[r], rowt, h ? col1 : col0);
          }
        }
        rre[r] = rowt.x;
        rim[r] = rowt.y;
        rdst[r] = rpc + cp.i;
        if (kGrad && lane == 0) {
          if (cp.i == cp.b * kStripe) sc.tile_w[col_gt].x = w;
          if (cp.i == cp.bend - 1) sc.tile_w[col_gt].y = w;
        }
        if (++cp.i == cp.bend) {                   // the tile is done: flush its column sums
          if (kGrad) {
            float2* dst = sc.col_part + (w + col_gt) * kStripe;
            dst[lane] = col0;
            dst[lane + 32] = col1;
            col0 = col1 = make_float2(0.f, 0.f);
          }
          cp.next_tile(G);
          rpc = sc.row_part + (static_cast<long long>(cp.c) * G.S + cp.s) * G.N;
          col_gt = cp.tile(G);
          if (grp * kGroup + r + 1 < n) load_gj();
        }
      }
    }
    if (kChi) {
      float t = chi_g[0];
#pragma unroll
      for (int r = 1; r < kGroup; ++r) t += chi_g[r];
      chi_acc.add(t);
    }
    if (kGrad) {
      if constexpr (kGroup == 4) {
        const float sre = reduce4(rre[0], rre[1], rre[2], rre[3], lane);
        const float sim = reduce4(rim[0], rim[1], rim[2], rim[3], lane);
        const int t = lane >> 3;
        float2* d = t == 0 ? rdst[0] : t == 1 ? rdst[1] : t == 2 ? rdst[2] : rdst[3];
        if ((lane & 7) == 0 && d) *d = make_float2(sre, sim);
      } else {
        const float sre = reduce2(rre[0], rre[1], lane);
        const float sim = reduce2(rim[0], rim[1], lane);
        float2* d = (lane >> 4) ? rdst[1] : rdst[0];
        if ((lane & 15) == 0 && d) *d = make_float2(sre, sim);
      }
    }
    __syncwarp();                                  // every lane is done with this group's slots
    issue_group(grp + kRing);
  }
  cp_async_wait<0>();
  // a range that ends inside a tile leaves that tile's column sums unflushed
  if (kGrad && n > 0 && cp.i != cp.b * kStripe) {
    float2* dst = sc.col_part + (w + col_gt) * kStripe;
    dst[lane] = col0;
    dst[lane + 32] = col1;
  }
  if (kChi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) chi_acc.add_lane(o);
    if (lane == 0) sc.chi_part[w] = make_float2(chi_acc.s, chi_acc.c);
  }

}

// grad[c][k] = 2 scale (row sums over the stripes s <= k / 64, then the
// column sums of every warp that touched a tile (b, k / 64), b ascending and
// warps ascending within a tile), in that fixed order; one thread per entry.
// The pass kernel records each tile's first and last warp; the loads of up to
// 8 row partials and of up to 4 warps x 4 tiles of column partials are
// issued together (absent ones as zeros, which leave the sum unchanged).  The
// last block also sums the per-warp chi^2 partials.
__global__ void __launch_bounds__(256)
calib_combine_kernel(Geometry G, Scratch sc, const double* __restrict__ scale, float2* __restrict__ grad,
                     double* __restrict__ chisq) {
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (grad && t < static_cast<long long>(G.C) * G.N) {
    const int c = static_cast<int>(t / G.N), k = static_cast<int>(t - static_cast<long long>(c) * G.N);
    const int sk = k / kStripe, jl = k - sk * kStripe;
    const float2* rp = sc.row_part + static_cast<long long>(c) * G.S * G.N + k;
    float2 acc = make_float2(0.f, 0.f);
    for (int s0 = 0; s0 <= sk; s0 += 8) {
      float2 p[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) p[q] = s0 + q <= sk ? __ldcg(rp + static_cast<long long>(s0 + q) * G.N) : make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        acc.x += p[q].x;
        acc.y += p[q].y;
      }
    }
    const long long gt0 = static_cast<long long>(c) * G.T + sk;   // tile (b, sk) is gt0 + b (b + 1) / 2
    for (int b0 = sk; b0 < G.S; b0 += 4) {
      int2 tw[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        tw[u] = b0 + u < G.S ? __ldcg(sc.tile_w + gt0 + (b0 + u) * (b0 + u + 1) / 2) : make_int2(0, -1);
      float2 p[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long gt = gt0 + (b0 + u) * (b0 + u + 1) / 2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int w = tw[u].x + q;
          // a warp with no segments (only when the grid has more warps than segments) wrote nothing
          const bool has = w <= tw[u].y && (!G.sparse || G.begin(w) != G.begin(w + 1));
          p[u][q] = has ? __ldcg(sc.col_part + (w + gt) * kStripe + jl) : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc.x += p[u][q].x;
          acc.y += p[u][q].y;
        }
        const long long gt = gt0 + (b0 + u) * (b0 + u + 1) / 2;
        for (int w = tw[u].x + 4; w <= tw[u].y; ++w) {   // tiles spread over more than 4 warps
          if (G.sparse && G.begin(w) == G.begin(w + 1)) continue;
          const float2 e = __ldcg(sc.col_part + (w + gt) * kStripe + jl);
          acc.x += e.x;
          acc.y += e.y;
        }
      }
    }
    const float f = 2.0f * (scale ? static_cast<float>(*scale) : 1.0f);
    grad[t] = make_float2(f * acc.x, f * acc.y);
  }
  if (chisq && blockIdx.x == gridDim.x - 1) {
    // The per-warp (sum, compensation) pairs are added with the same
    // compensated float32 sum, per thread and across each warp; float64
    // appears only in the last step, over the 8 warps' pairs (B300's float64
    // rate is a small fraction of its float32 rate: converting every pair
    // here cost ~5 us of one SM).
    __shared__ float2 red[8];
    CompSum acc;
    for (int q0 = threadIdx.x; q0 < G.W; q0 += 8 * 256) {
      float2 p[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) p[u] = q0 + u * 256 < G.W ? __ldcg(sc.chi_part + q0 + u * 256) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        acc.c += p[u].y;
        acc.add(p[u].x);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc.add_lane(o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(acc.s, acc.c);
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) r += static_cast<double>(red[q].x) + static_cast<double>(red[q].y);
      *chisq = r;
    }
  }
}

// out[k] = scale * in[k] over n complex values.
__global__ void scale_kernel(const float2* __restrict__ in, const double* __restrict__ scale, long long n,
                             float2* __restrict__ out) {
  const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  const float f = static_cast<float>(*scale);
  const float2 x = in[t];
  out[t] = make_float2(f * x.x, f * x.y);
}

inline Geometry geometry(int N, int C, int ctas) {
  Geometry G;
  G.N = N;
  G.C = C;
  G.S = (N + kStripe - 1) / kStripe;
  G.W = ctas * kWarps;
  G.T = G.S * (G.S + 1) / 2;
  G.nbl = static_cast<long long>(N) * (N + 1) / 2;
  G.P = band_prefix(G.S - 1) + static_cast<long long>(G.S) * (N - (G.S - 1) * kStripe);
  G.L = G.P * C;
  G.sparse = G.L < G.W;
  return G;
}

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Byte offsets of the scratch regions (chi partials, row partials, column
// partials) and the total.
inline void layout(const Geometry& G, size_t off[4], size_t* total) {
  size_t o = 0;
  off[0] = o; o = align256(o + sizeof(float2) * G.W);
  off[1] = o; o = align256(o + sizeof(float2) * static_cast<size_t>(G.C) * G.S * G.N);
  off[2] = o; o = align256(o + sizeof(float2) * kStripe * (static_cast<size_t>(G.C) * G.T + G.W));
  off[3] = o; o = align256(o + sizeof(int2) * static_cast<size_t>(G.C) * G.T);
  *total = o;
}

inline Scratch carve(void* base, const Geometry& G) {
  size_t off[4], total;
  layout(G, off, &total);
  char* b = static_cast<char*>(base);
  Scratch sc;
  sc.chi_part = reinterpret_cast<float2*>(b + off[0]);
  sc.row_part = reinterpret_cast<float2*>(b + off[1]);
  sc.col_part = reinterpret_cast<float2*>(b + off[2]);
  sc.tile_w = reinterpret_cast<int2*>(b + off[3]);
  return sc;
}

template <bool kChi, bool kGrad, bool kW>
cudaError_t launch(const float2* g, const float2* m, const float2* v, const float* w, const Geometry& G, int ctas,
                   int include_autos, const Scratch& sc, cudaStream_t stream) {
  calib_pass_kernel<kChi, kGrad, kW><<<ctas, kThreads, 0, stream>>>(g, m, v, w, G, include_autos, sc);
  return cudaGetLastError();
}

template <bool kChi, bool kGrad>
cudaError_t launch_w(const float2* g, const float2* m, const float2* v, const float* w, const Geometry& G, int ctas,
                     int include_autos, const Scratch& sc, cudaStream_t stream) {
  return w ? launch<kChi, kGrad, true>(g, m, v, w, G, ctas, include_autos, sc, stream)
           : launch<kChi, kGrad, false>(g, m, v, w, G, ctas, include_autos, sc, stream);
}

}  // namespace cal

int calib_grid_ctas(int N, int C) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cal::calib_pass_kernel<true, true, true>,
                                                    cal::kThreads, 0) != cudaSuccess)
    return 0;
  const long long full = static_cast<long long>(sms) * (per_sm > 0 ? per_sm : 1);
  const long long L = cal::geometry(N, C, 1).L;
  const long long ctas = L / cal::kWarps < full ? L / cal::kWarps : full;   // every warp gets >= 1 segment
  return static_cast<int>(ctas > 0 ? ctas : 1);
}

size_t calib_scratch_bytes(int N, int C, int ctas) {
  size_t off[4], total;
  cal::layout(cal::geometry(N, C, ctas), off, &total);
  return total;
}

cudaError_t launch_calib(const float* g, const float* model, const float* vobs, const float* w, int N, int C,
                         int ctas, int include_autos, void* scratch, double* chisq, const double* scale,
                         float* grad, cudaStream_t stream) {
  const cal::Geometry G = cal::geometry(N, C, ctas);
  const cal::Scratch sc = cal::carve(scratch, G);
  const float2* g2 = reinterpret_cast<const float2*>(g);
  const float2* m2 = reinterpret_cast<const float2*>(model);
  const float2* v2 = reinterpret_cast<const float2*>(vobs);
  float2* gr = reinterpret_cast<float2*>(grad);
  cudaError_t e;
  if (chisq && grad) e = cal::launch_w<true, true>(g2, m2, v2, w, G, ctas, include_autos, sc, stream);
  else if (chisq) e = cal::launch_w<true, false>(g2, m2, v2, w, G, ctas, include_autos, sc, stream);
  else e = cal::launch_w<false, true>(g2, m2, v2, w, G, ctas, include_autos, sc, stream);
  if (e != cudaSuccess) return e;
  const long long entries = grad ? static_cast<long long>(C) * N : 1;
  cal::calib_combine_kernel<<<static_cast<unsigned>((entries + 255) / 256), 256, 0, stream>>>(G, sc, scale, gr, chisq);
  return cudaGetLastError();
}

cudaError_t launch_calib_scale(const float* in, const double* scale, long long n, float* out, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  cal::scale_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
      reinterpret_cast<const float2*>(in), scale, n, reinterpret_cast<float2*>(out));
  return cudaGetLastError();
}

}  // namespace xe

// ------------------------------------------------------------------ C ABI
#include <new>

#include "xengine.h"

struct xe_calib {
  int N = 0, C = 0;
  int ctas = 0;   // persistent grid of the pass kernel
  void* scratch = nullptr;
};

namespace {
bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

xe_status check_inputs(xe_calib_t c, const float* g, const float* model, const float* vobs, const float* w,
                       int include_autos) {
  if (!c || !g || !model || !vobs || (include_autos != 0 && include_autos != 1)) return XE_ERR_INVALID_ARG;
  if (!aligned(g, 8) || !aligned(model, 8) || !aligned(vobs, 8) || !aligned(w, 4)) return XE_ERR_ALIGNMENT;
  return XE_OK;
}
}  // namespace

extern "C" {

XE_API xe_status xe_calib_create(xe_calib_t* out, int n_input, int n_chan) {
  if (!out) return XE_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_input < 1 || n_input > 8192 || n_chan < 1 || n_chan > (1 << 20)) return XE_ERR_INVALID_ARG;
  if (static_cast<long long>(n_chan) * n_input * (n_input + 1) / 2 > (1LL << 40)) return XE_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return XE_ERR_CUDA;
  xe_calib* c = new (std::nothrow) xe_calib();
  if (!c) return XE_ERR_NOMEM;
  c->N = n_input;
  c->C = n_chan;
  c->ctas = xe::calib_grid_ctas(n_input, n_chan);
  if (c->ctas <= 0) {
    cudaGetLastError();
    delete c;
    return XE_ERR_CUDA;
  }
  if (cudaMalloc(&c->scratch, xe::calib_scratch_bytes(n_input, n_chan, c->ctas)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return XE_ERR_NOMEM;
  }
  *out = c;
  return XE_OK;
}

XE_API xe_status xe_calib_destroy(xe_calib_t c) {
  if (!c) return XE_OK;
  cudaDeviceSynchronize();
  cudaFree(c->scratch);
  delete c;
  return XE_OK;
}

XE_API xe_status xe_calib_chisq(xe_calib_t c, const float* d_g, const float* d_model, const float* d_vobs,
                                const float* d_w, int include_autos, double* d_chisq, void* stream) {
  const xe_status st = check_inputs(c, d_g, d_model, d_vobs, d_w, include_autos);
  if (st != XE_OK) return st;
  if (!d_chisq) return XE_ERR_INVALID_ARG;
  if (!aligned(d_chisq, 8)) return XE_ERR_ALIGNMENT;
  return xe::launch_calib(d_g, d_model, d_vobs, d_w, c->N, c->C, c->ctas, include_autos, c->scratch, d_chisq, nullptr,
                          nullptr, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? XE_OK
             : XE_ERR_CUDA;
}

XE_API xe_status xe_calib_grad(xe_calib_t c, const float* d_g, const float* d_model, const float* d_vobs,
                               const float* d_w, int include_autos, const double* d_scale, float* d_grad,
                               void* stream) {
  const xe_status st = check_inputs(c, d_g, d_model, d_vobs, d_w, include_autos);
  if (st != XE_OK) return st;
  if (!d_grad) return XE_ERR_INVALID_ARG;
  if (!aligned(d_grad, 8) || !aligned(d_scale, 8)) return XE_ERR_ALIGNMENT;
  return xe::launch_calib(d_g, d_model, d_vobs, d_w, c->N, c->C, c->ctas, include_autos, c->scratch, nullptr, d_scale,
                          d_grad, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? XE_OK
             : XE_ERR_CUDA;
}

XE_API xe_status xe_calib_chisq_grad(xe_calib_t c, const float* d_g, const float* d_model, const float* d_vobs,
                                     const float* d_w, int include_autos, double* d_chisq, float* d_grad,
                                     void* stream) {
  const xe_status st = check_inputs(c, d_g, d_model, d_vobs, d_w, include_autos);
  if (st != XE_OK) return st;
  if (!d_chisq || !d_grad) return XE_ERR_INVALID_ARG;
  if (!aligned(d_chisq, 8) || !aligned(d_grad, 8)) return XE_ERR_ALIGNMENT;
  return xe::launch_calib(d_g, d_model, d_vobs, d_w, c->N, c->C, c->ctas, include_autos, c->scratch, d_chisq, nullptr,
                          d_grad, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? XE_OK
             : XE_ERR_CUDA;
}

XE_API xe_status xe_calib_scale(xe_calib_t c, const float* d_in, const double* d_scale, float* d_out,
                                void* stream) {
  if (!c || !d_in || !d_scale || !d_out) return XE_ERR_INVALID_ARG;
  if (!aligned(d_in, 8) || !aligned(d_scale, 8) || !aligned(d_out, 8)) return XE_ERR_ALIGNMENT;
  return xe::launch_calib_scale(d_in, d_scale, static_cast<long long>(c->C) * c->N, d_out,
                                static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? XE_OK
             : XE_ERR_CUDA;
}

}  // extern "C"
