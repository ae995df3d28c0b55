// BF16 tensor-core network (pass 1) on tcgen05: each CTA takes a contiguous run of 32x4-cell
// tiles of the torus, then chunks of tiles from a shared pool. A tile's one-cell halo of the six
// sensor channels comes into shared memory by one TMA box copy (cp.async where the halo wraps
// around the torus). Every thread builds its cell's row of the 128 x 64 BF16 input tile straight
// from that stage (the rotation-ordered 3x3 neighbourhood, K index 6*rank + channel, a constant
// 1 at K = 54 that carries the layer-1 bias) and takes its own E, I and flow denominator from
// it; after one CTA barrier the stage is free and the next tile's copy overlaps this tile's
// network. The genome nets run on the tensor cores with FP32 accumulation in TMEM: one
// 128 x H x 64 MMA for layer 1 (both operands in shared memory; the genome's BF16 blob arrives
// by one bulk copy when it changes), tanh in the epilogue with the BF16 hidden tile written back
// into the consumed TMEM columns, one 128 x 16 x H MMA for layer 2 that reads its A operand from
// TMEM. A tile with several genomes runs one round per genome (the rows of other genomes are
// computed and discarded); a cell's actuator epilogue (communication, invest/liquidate,
// exploration, flow quotient) runs in registers in the round that computes its outputs.
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include "coral_internal.cuh"
#include "epilogue.cuh"
#include "tc_ptx.cuh"

namespace coral {

namespace {

constexpr int kThreads = 128;
constexpr int kCtasPerSm = 6;                             // 6 x 64 of the 512 TMEM columns, 80 registers
constexpr int kTileW = 32, kTileH = kThreads / kTileW;   // thread q: cell (q % kTileW, q / kTileW)
constexpr int kHaloW = kTileW + 2, kHaloH = kTileH + 2;
constexpr int kHaloCells = kHaloW * kHaloH;
// TMEM columns of a CTA: layer 1's FP32 accumulators in 0..H-1; the BF16 hidden tile is
// written over its first H/2 columns; layer 2's accumulators in kD2Col..kD2Col+15
constexpr uint32_t kTmemCols = 64;
constexpr uint32_t kD2Col = 32;
constexpr long long kWaitCycles = 4000000000LL;           // about 2 s of SM clock
// Work split: each CTA first takes a contiguous run of about half its share of the tiles
// (neighbouring tiles share halo rows in L2 and usually a genome); the remaining tiles form a
// pool of kChunk-tile chunks that CTAs claim with one atomic each as they finish, so CTAs
// whose tiles hold more genomes (more rounds) no longer set the kernel's end. Measured on the
// 4096^2 world: runs of 3/8 to 5/8 of the share are equally fast, 3/4 is 3% and 7/8 10%
// slower, chunks of 8 tiles 1.3% slower than 4.
constexpr int kStaticNum = 1, kStaticDen = 2;
constexpr int kChunk = 4;
// C' sums in fixed point: every float in [2^-3, 1) is a multiple of 2^-26 and C' lies in
// (0.26, 0.74), so C' * 2^26 is an exact integer and the sums are exact, independent of which
// CTA took which tile (and so of the order in which the pool was claimed).
constexpr float kCFix = 67108864.0f;                      // 2^26

// shared memory layout, offsets from a 1024-byte aligned base
constexpr int kOffA = 0;                                  // 128 x 128 B: input tile, then hidden tile
constexpr int kOffW = 16384;                              // genome blob (<= 10368 B at H = 64)
// stage: float32 [6 channels][6 rows][40 columns], halo column hx at 3 + hx (the TMA box starts
// 4 cells left of the tile so its x coordinate stays 16-byte aligned). One buffer: it is free
// again once every thread has built its input row and taken its own E, I and flow denominator
// from it, so the next tile's copy overlaps the current tile's network rounds.
constexpr int kStageW = kTileW + 8, kStageCh = kStageW * kHaloH;  // 240 floats per channel
constexpr int kStageBytes = 6 * kStageCh * 4;             // 5760
constexpr int kOffStage = kOffW + 10368;                  // 128-byte aligned
constexpr int kOffG = kOffStage + kStageBytes;            // int32 [128]
constexpr int kOffMisc = kOffG + 512;                     // mbarrier, TMEM slot, flags
constexpr int kSmemBytes = kOffMisc + 128 + 1024;         // + alignment slack

// C' * 2^26 as an integer from the float's bits: C' lies in (0.26, 0.74), so its exponent is
// 2^-2 or 2^-1 and the value is the 24-bit significand shifted left by 1 or 2 (exact; integer
// operations instead of a float-to-int conversion on the special-function pipe).
__device__ __forceinline__ int cfix(float c) {
  const uint32_t b = __float_as_uint(c);
  return (int)(((b & 0x7FFFFFu) | 0x800000u) << ((b >> 23) - 124u));
}

// Exact float -> double by moving the bits (rebias the exponent, shift the significand), for
// normal floats; returns false in `special` for zero, subnormal, infinite or NaN inputs, which
// the caller converts on the FP64 pipe instead.
__device__ __forceinline__ double f2d_bits(float f, bool& special) {
  const uint32_t b = __float_as_uint(f), a = b & 0x7FFFFFFFu;
  special |= (a - 0x00800000u) >= 0x7F000000u;
  return __hiloint2double((int)(((a >> 3) + 0x38000000u) | (b & 0x80000000u)), (int)(b << 29));
}

// v in [-1, n + tile) folded onto [0, n): one conditional step when the torus side is at least
// the halo's (small), else a full modulo.
__device__ __forceinline__ int fold(int v, int n, bool small) {
  if (small) {
    v %= n;
    return v < 0 ? v + n : v;
  }
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

// Stage-index offset (dy * kStageW + dx) of kernel ranks 1..8 for rotation r, one signed byte
// per rank (rank p in bits 8(p-1)..8p-1).
__host__ __device__ constexpr unsigned long long stage_offsets(int r) {
  unsigned long long v = 0;
  for (int p = 1; p < 9; ++p) {
    const int o = (2 * r + rank_delta(p)) & 7;
    const int dx = (int)((0x1A9u >> (2 * o)) & 3u) - 1, dy = (int)((0x1A90u >> (2 * o)) & 3u) - 1;
    v |= (unsigned long long)(uint8_t)(int8_t)(dy * kStageW + dx) << (8 * (p - 1));
  }
  return v;
}

// Starts the asynchronous copy (cp.async, for tiles whose halo wraps around the torus) of a
// tile's halo of the six contiguous sensor planes into a stage buffer: warp w copies row
// segments w, w+4, ... (one per channel and halo row); lane l copies halo columns l and l + 32.
__device__ __forceinline__ void issue_halo(const StepArgs& a, int x0, int y0, uint32_t dst) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool wraps = y0 == 0 || y0 - 1 + kHaloH > a.H;
  const bool small_h = a.H < kHaloH, small_w = a.W < kHaloW;
  const int col_a = fold(x0 - 1 + lane, a.W, small_w);
  const int col_b = fold(x0 + 31 + lane, a.W, small_w);
  static_assert(kHaloW <= 64 && (6 * kHaloH) % (kThreads / 32) == 0, "halo copy layout");
#pragma unroll
  for (int k = 0; k < 6 * kHaloH / (kThreads / 32); ++k) {
    const int sgm = warp + k * (kThreads / 32);
    const int ch = sgm / kHaloH, hy = sgm - ch * kHaloH;
    const int gy = wraps ? fold(y0 - 1 + hy, a.H, small_h) : y0 - 1 + hy;
    const long long off = (long long)ch * a.N + (long long)gy * a.P;
    const float* row = a.cur.E + off;
    const uint32_t d = dst + 4u * (uint32_t)(ch * kStageCh + hy * kStageW + 3);
    if (lane < kHaloW) tc::cp_async4(d + 4u * lane, row + col_a);
    if (lane + 32 < kHaloW) tc::cp_async4(d + 4u * (32 + lane), row + col_b);
  }
  tc::cp_async_commit();
}

// Warp-level FMA evaluation of one genome's net for the rows of this warp given in `rows`
// (the small-genome path): for each such row in turn, the 32 lanes compute the hidden units
// lane and lane + 32 (with one layer, H = 0: lanes 0..9 the ten outputs) from the row's BF16
// input (shared memory, the MMA's input tile) and the
// genome's BF16 blob (global memory: W1 rows, W2 rows, b2, the layout the MMA reads), with the
// MMA path's arithmetic: BF16 operands, FP32 sums, tanh.approx hidden values rounded to BF16;
// the ten layer-2 sums are reduced over the warp. Returns this lane's row outputs (before the
// output tanh, b2 added) in zo when its row is in `rows`.
template <int H>
__device__ __forceinline__ void fma_round(unsigned rows, uint32_t tile_s, const uint8_t* blob, int warp, int lane,
                                          float (&zo)[kOut]) {
  constexpr int N1 = H ? H : 16;
  while (rows) {
    const int lr = __ffs(rows) - 1;
    rows &= rows - 1;
    const int row = warp * 32 + lr;
    const uint32_t xrow = tile_s + (uint32_t)row * 128u;
    // output (H = 0) or hidden units u0 = lane, u1 = lane + 32 of layer 1
    const int u0 = lane, u1 = lane + 32;
    const bool has0 = u0 < (H ? H : kOut), has1 = H > 32 && u1 < H;
    float acc0 = 0.0f, acc1 = 0.0f;
#pragma unroll 1
    for (int p = 0; p < 8; ++p) {                     // not unrolled: few registers on this rare path
      uint32_t xw[4];
      asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];"
                   : "=r"(xw[0]), "=r"(xw[1]), "=r"(xw[2]), "=r"(xw[3])
                   : "r"(xrow + ((((uint32_t)p ^ (uint32_t)row) & 7u) << 4)));
      float x[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        x[2 * i] = __uint_as_float(xw[i] << 16);
        x[2 * i + 1] = __uint_as_float(xw[i] & 0xFFFF0000u);
      }
      if (has0) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(blob + u0 * 128 + (((p ^ u0) & 7) << 4)));
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc0 = fmaf(x[2 * i], __uint_as_float(ww[i] << 16), acc0);
          acc0 = fmaf(x[2 * i + 1], __uint_as_float(ww[i] & 0xFFFF0000u), acc0);
        }
      }
      if (has1) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(blob + u1 * 128 + (((p ^ u1) & 7) << 4)));
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc1 = fmaf(x[2 * i], __uint_as_float(ww[i] << 16), acc1);
          acc1 = fmaf(x[2 * i + 1], __uint_as_float(ww[i] & 0xFFFF0000u), acc1);
        }
      }
    }
    if constexpr (H == 0) {
#pragma unroll
      for (int o = 0; o < kOut; ++o) {
        const float z = __shfl_sync(0xffffffffu, acc0, o);
        if (lane == lr) zo[o] = z;
      }
    } else {
      // hidden values as the MMA's A operand holds them: tanh, rounded to BF16
      const float h0 = has0 ? __uint_as_float(tc::pack_bf16x2(0.0f, tc::tanh_approx(acc0)) & 0xFFFF0000u) : 0.0f;
      const float h1 = has1 ? __uint_as_float(tc::pack_bf16x2(0.0f, tc::tanh_approx(acc1)) & 0xFFFF0000u) : 0.0f;
      const uint8_t* w2 = blob + N1 * 128;
#pragma unroll
      for (int o = 0; o < kOut; ++o) {
        float part = 0.0f;
        if (has0) {
          const uint16_t b = __ldg(reinterpret_cast<const unsigned short*>(
              w2 + o * 128 + ((((u0 >> 3) ^ o) & 7) << 4) + ((u0 & 7) << 1)));
          part = h0 * __uint_as_float((uint32_t)b << 16);
        }
        if (has1) {
          const uint16_t b = __ldg(reinterpret_cast<const unsigned short*>(
              w2 + o * 128 + ((((u1 >> 3) ^ o) & 7) << 4) + ((u1 & 7) << 1)));
          part = fmaf(h1, __uint_as_float((uint32_t)b << 16), part);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == lr) zo[o] = part + __ldg(reinterpret_cast<const float*>(w2 + 16 * 128) + o);
      }
    }
  }
}

// One CTA's share of pass 1 for one world: CTA `cta` of `ncta` takes a contiguous run of tiles,
// then pool chunks (see kStaticNum); its partial sums go to a.part1[cta]. tmap: TMA descriptor (use_tma != 0) or unused.
// kH: the hidden size (0 = one layer), a compile-time constant so that the per-chunk loops and
// the layer-2 branch are resolved by the compiler; one instantiation per supported size.
// kFma: the instantiation with the warp-level FMA path for small genomes (fma_round), used
// when a.fma_cutoff > 0; the default instantiation has none of its code.
template <int kH, bool kFma>
__device__ __forceinline__ void pass1_bf16_body(const StepArgs& a, const CUtensorMap* tmap, const int use_tma,
                                                const int cta, const int ncta) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_s = tc::smem_u32(smem_raw);
  const uint32_t base_s = (raw_s + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_s - raw_s);
  int32_t* sG = reinterpret_cast<int32_t*>(base + kOffG);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + kOffMisc);
  uint64_t* w_bar = reinterpret_cast<uint64_t*>(base + kOffMisc + 96);    // bulk copy of a genome blob
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + kOffMisc + 8);
  unsigned* ballots = reinterpret_cast<unsigned*>(base + kOffMisc + 16);      // [2][4] pending rows
  uint64_t* halo_bar = reinterpret_cast<uint64_t*>(base + kOffMisc + 48);     // the stage's TMA barrier
  unsigned* match = reinterpret_cast<unsigned*>(base + kOffMisc + 64);        // [4] rows of the staged genome
  int* claim_s = reinterpret_cast<int*>(base + kOffMisc + 80);                // [2] pool chunks claimed by thread 0
  __shared__ long long red_s[4][4];
  __shared__ long long red_c[4];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lx = tid % kTileW, ly = tid / kTileW;     // this thread's cell within a tile
  const int W = a.W, Hh = a.H;
  constexpr int H = kH;
  constexpr int N1 = H ? H : 16;
  const uint32_t w_s = base_s + kOffW;
  const uint32_t a_s = base_s + kOffA;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::mbar_init(w_bar, 1);
    tc::mbar_init(halo_bar, 1);
    tc::fence_barrier_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t idesc1 = tc::idesc_bf16_f32(128, N1);
  const uint32_t idesc2 = tc::idesc_bf16_f32(128, 16);
  uint32_t phase = 0, w_phase = 0;

  if (lane == 0) {                                    // this warp's fixed-point sums of C'
#pragma unroll
    for (int k = 0; k < 4; ++k) red_s[warp][k] = 0;
  }
  int accX = 0;
  bool timed_out = false;                             // the CTA agreed to stop (a wait ran out)
  bool bad = false;                                   // one of this thread's waits ran out
  int staged = -1;                                    // genome whose blob is in shared memory
  int rb = 0;                                         // ballot buffer the next round reads
  const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (Hh + kTileH - 1) / kTileH;
  const int n_tiles = tiles_x * tiles_y;
  // this CTA's contiguous run, then chunks of the pool [pool0, n_tiles)
  const int per = (int)((long long)n_tiles * kStaticNum / kStaticDen / ncta);
  const int pool0 = per * ncta;
  // the pool chunk claimed as number q: its first tile, or -1 when the pool is used up
  auto chunk_first = [&](int q) { return q < (n_tiles - pool0 + kChunk - 1) / kChunk ? pool0 + q * kChunk : -1; };
  int cur = cta * per, run_end = cur + per;
  if (per == 0) {                                     // small world: the pool only
    if (tid == 0) claim_s[0] = atomicAdd(a.sched, 1);
    __syncthreads();
    cur = chunk_first(claim_s[0]);
    run_end = cur < 0 ? -1 : min(cur + kChunk, n_tiles);
    __syncthreads();                                  // claim_s[0] is written again below
  }
  int g_next = -1, r_next = 0;
  uint32_t halo_phase = 0;                            // parity of halo_bar
  bool tma_pending = false;                           // a TMA copy into the stage is in flight
  // A tile's halo comes by one TMA box copy when it does not wrap around the torus, else by
  // cp.async; the choice is uniform per tile.
  auto tma_tile = [&](int x0, int y0) {
    return use_tma && x0 >= 4 && x0 + kTileW + 4 <= W && y0 >= 1 && y0 + kTileH + 1 <= Hh;
  };
  // next tile: halo copy started, genome and rotation of this thread's cell loaded
  auto prefetch = [&](int x0, int y0) {
    const uint32_t dst = base_s + kOffStage;
    if (tma_tile(x0, y0)) {
      if (tid == 0) {
        tc::fence_proxy_async();                       // earlier generic accesses of the buffer
        tc::mbar_expect_tx(halo_bar, kStageBytes);
        tc::tma_load_3d(dst, tmap, x0 - 4, y0 - 1, 0, halo_bar);
      }
      tma_pending = true;
    } else {
      issue_halo(a, x0, y0, dst);
    }
    g_next = -1;
    r_next = 0;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx < W && gy < Hh) {
      const int jn = gy * a.P + gx;
      g_next = __ldg(a.cur.G + jn);
      r_next = a.rotation ? (int)__ldg(a.cur.R + jn) : 0;
    }
  };
  int ty = cur < 0 ? 0 : cur / tiles_x, tx = cur < 0 ? 0 : cur - ty * tiles_x;   // running tile coordinates
  if (cur >= 0) prefetch(tx * kTileW, ty * kTileH);
  int cacc[4] = {0, 0, 0, 0};             // fixed-point partials of up to 16 tiles (< 2^31), then into red_s
  // adds the partials of this warp's 32 threads (64-bit integers) to its row of red_s
  auto flush = [&]() {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      long long v = cacc[k];
#pragma unroll
      for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) red_s[warp][k] += v;
      cacc[k] = 0;
    }
  };
  int ntile = 0;
  int it = 0;                                         // tile count: parity selects claim_s
  int reserved = -2;                                  // thread 0: pool chunk claimed ahead (-2: none)

  while (cur >= 0) {
    const int x0 = tx * kTileW, y0 = ty * kTileH;
    // the next tile: the next one of this run, or the first of a newly claimed pool chunk
    // (claimed now, read after the input-tile barrier; two slots, so that a slow thread still
    // reading the last claim never sees it overwritten)
    const bool claim = cur + 1 >= run_end;
    if (tid == 0) {
      // the atomic is issued one tile ahead of the claim, so its latency is not waited for
      if (reserved == -2 && cur + 2 >= run_end) reserved = atomicAdd(a.sched, 1);
      if (claim) {
        claim_s[it & 1] = reserved;
        reserved = -2;
      }
    }
    const int gx = x0 + lx, gy = y0 + ly;
    const bool valid = gx < W && gy < Hh;
    const long long j = (long long)gy * a.P + gx;
    const int g = g_next, r = r_next;
    // this tile's halo: every thread waits on the TMA barrier itself; a cp.async tile needs
    // the CTA barrier to see the other threads' copies
    if (tma_tile(x0, y0)) {
      if (tc::mbar_wait(halo_bar, halo_phase, kWaitCycles)) {
        halo_phase ^= 1u;
        tma_pending = false;
      } else {
        bad = true;                                   // the copy may still land: waited for at exit
      }
    } else {
      tc::cp_async_wait_all();
      __syncthreads();
    }
    sG[tid] = g;
    const float* stage = reinterpret_cast<const float*>(base + kOffStage);
    // this cell's input row, straight from the stage: chunk p = the 6 BF16 channels of kernel
    // rank p (p < 8) and a spare word with rank 8's channels (p < 3) or the bias 1.0 (p = 3);
    // 128-byte swizzle. Rows of cells outside the grid get what the stage holds there and are
    // discarded.
    {
      const uint32_t row_s = a_s + tid * 128;
      const uint32_t t7 = tid & 7;
      const int sc = (ly + 1) * kStageW + lx + 4;
      const unsigned long long offs = r == 0 ? stage_offsets(0) : r == 1 ? stage_offsets(1)
                                    : r == 2 ? stage_offsets(2) : stage_offsets(3);
      const float* s8 = stage + sc + (int)(int8_t)(uint8_t)(offs >> 56);
      const uint32_t w8[3] = {tc::pack_bf16x2(s8[0], s8[kStageCh]), tc::pack_bf16x2(s8[2 * kStageCh], s8[3 * kStageCh]),
                              tc::pack_bf16x2(s8[4 * kStageCh], s8[5 * kStageCh])};
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const float* sp = stage + sc + (p == 0 ? 0 : (int)(int8_t)(uint8_t)(offs >> (8 * (p - 1))));
        const uint32_t w4 = p < 3 ? w8[p] : (p == 3 ? 0x3F80u : 0u);
        tc::sts128(row_s + (((uint32_t)p ^ t7) << 4), tc::pack_bf16x2(sp[0], sp[kStageCh]),
                   tc::pack_bf16x2(sp[2 * kStageCh], sp[3 * kStageCh]), tc::pack_bf16x2(sp[4 * kStageCh], sp[5 * kStageCh]),
                   w4);
      }
    }
    // this cell's E and I and the FP64 sum S of its 4 neighbours' I (N, E, S, W), rounded once
    float Ec, Ic, Sf;
    {
      const int sc = (ly + 1) * kStageW + lx + 4;      // this cell in the stage layout
      const float* sI = stage + kStageCh;
      Ec = stage[sc];
      Ic = sI[sc];
      // the four neighbours' I in double precision: exact bit moves unless a value is zero,
      // subnormal or not finite somewhere in the warp (then the FP64 conversions)
      const float iN = sI[sc - kStageW], iE = sI[sc + 1], iS = sI[sc + kStageW], iW = sI[sc - 1];
      bool sp = false;
      const double dN = f2d_bits(iN, sp), dE = f2d_bits(iE, sp), dS = f2d_bits(iS, sp), dW = f2d_bits(iW, sp);
      if (__any_sync(0xffffffffu, sp))
        Sf = (float)((double)iN + (double)iE + (double)iS + (double)iW);
      else
        Sf = (float)(dN + dE + dS + dW);
    }
    bool done = g < 0;
    rb ^= 1;                                          // the last round's buffer is free again
    {
      const unsigned b = __ballot_sync(0xffffffffu, !done);   // first round's pending rows
      if (lane == 0) ballots[4 * rb + warp] = b;
      const unsigned m = __ballot_sync(0xffffffffu, !done && g == staged);   // rows of the staged genome
      if (lane == 0) match[warp] = m;
    }
    tc::fence_proxy_async();                          // input rows for the MMA; stage reads before the next copy
    if (__syncthreads_or(bad)) {                      // input tile and the first ballots visible
      timed_out = true;
      break;
    }
    int nxt = cur + 1, nxt_end = run_end;
    if (claim) {
      nxt = chunk_first(claim_s[it & 1]);
      nxt_end = nxt < 0 ? -1 : min(nxt + kChunk, n_tiles);
    }
    if (nxt >= 0) {
      if (claim) {
        ty = nxt / tiles_x;
        tx = nxt - ty * tiles_x;
      } else if (++tx == tiles_x) {
        tx = 0;
        ++ty;
      }
      prefetch(tx * kTileW, ty * kTileH);
    }
    // actuator epilogue and pass-1 stores of this thread's cell, in the round that finishes it
    auto finish = [&](const float* act, const float* zo) {
      CellOut o;
      actuator_epilogue<true>(a, act, zo, Ec, Ic, Sf, r, o);
      store_pass1(a, j, o);
#pragma unroll
      for (int k = 0; k < 4; ++k) cacc[k] += cfix(o.C[k]);
      accX += o.xdir != kNoExplore ? 1 : 0;
    };
    if (valid && g < 0) {                             // empty cell: all actuators at zero
      const float zr[kOut] = {};
      finish(zr, zr);
    }
    // One tensor-core round per genome present in the tile: first the genome whose blob is
    // already staged, if the tile has cells of it, then the first pending row's genome.
    // The input tile in shared memory survives the rounds (the hidden tile lives in TMEM), so
    // it is built once per tile. Each round publishes the rows still pending after it in the
    // other ballot buffer before its hidden-tile barrier, so a single-genome tile costs two CTA
    // barriers (input tile, hidden tile); a later round starts with one more, after which the
    // last round's TMEM columns and b2 may be overwritten. The MMAs' completion is awaited by
    // every thread on the mbarrier, not through a CTA barrier.
    bool first_round = true;
    while (true) {
      const uint4 bl = *reinterpret_cast<const uint4*>(ballots + 4 * rb);
      const int first = bl.x ? __ffs(bl.x) - 1 : bl.y ? 31 + __ffs(bl.y) : bl.z ? 63 + __ffs(bl.z)
                      : bl.w ? 95 + __ffs(bl.w) : -1;
      int gs = first < 0 ? -1 : sG[first];
      if (first_round) {                              // the staged genome first: no restaging
        const uint4 mt = *reinterpret_cast<const uint4*>(match);
        if (mt.x | mt.y | mt.z | mt.w) gs = staged;
      }
      if (gs < 0) break;
      // a later round of a tile: every thread has read the last round's layer-2 outputs (TMEM)
      // and b2 (shared memory) before the new layer-1 MMA or the restaging overwrites them
      if (!first_round) {
        tc::fence_proxy_async();                      // b2 reads before a bulk copy over them
        if (__syncthreads_or(bad)) {
          timed_out = true;
          break;
        }
      }
      const bool restage = staged != gs;
      const bool mine = !done && g == gs;
      {
        const unsigned b = __ballot_sync(0xffffffffu, !done && !mine);   // pending after this round
        if (lane == 0) ballots[4 * (rb ^ 1) + warp] = b;
      }
      if constexpr (kFma) {
        // a later round whose genome has at most fma_cutoff rows in the tile: those rows by
        // warp-level FMA, no tensor-core round (the count's barrier publishes the ballots)
        if (!first_round) {
          const int cnt = __syncthreads_count(mine);
          if (cnt <= a.fma_cutoff) {
            const int gsafe = (unsigned)gs < (unsigned)a.capacity ? gs : 0;
            float zo[kOut];
            fma_round<H>(__ballot_sync(0xffffffffu, mine), a_s, a.nets16 + (long long)gsafe * a.blob_bytes, warp,
                         lane, zo);
            if (mine) {
              float act[kOut];
#pragma unroll
              for (int o = 0; o < kOut; ++o) act[o] = tc::tanh_approx(zo[o]);
              finish(act, zo);
              done = true;
            }
            rb ^= 1;
            continue;                                 // the next round starts with a CTA barrier
          }
        }
      }
      if constexpr (H == 0) {                         // no hidden-tile barrier: this one publishes
        if (__syncthreads_or(bad)) {                  // the ballots before the next round reads them
          timed_out = true;
          break;
        }
      }
      if (tid == 0) {
        tc::tc_fence_after();
        if (restage) {                                // this genome's BF16 blob, one bulk copy
          // an out-of-range GenomeIndex (loaded, reported as invalid, not yet read back) runs
          // slot 0's net instead of reading outside the genome table
          const int gsafe = (unsigned)gs < (unsigned)a.capacity ? gs : 0;
          tc::mbar_expect_tx(w_bar, (uint32_t)a.blob_bytes);
          tc::bulk_load(w_s, a.nets16 + (long long)gsafe * a.blob_bytes, (uint32_t)a.blob_bytes, w_bar);
          if (!tc::mbar_wait(w_bar, w_phase, kWaitCycles)) bad = true;
        }
        const uint64_t ad = tc::sdesc_sw128(a_s), bd = tc::sdesc_sw128(w_s);
#pragma unroll
        for (int k = 0; k < 4; ++k) tc::mma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc1, k > 0);
        tc::mma_commit(mbar);
      }
      if (!tc::mbar_wait(mbar, phase, kWaitCycles)) bad = true;
      phase ^= 1;
      tc::tc_fence_after();
      if constexpr (H == 0) {
        float v[16];
        tc::tmem_ld16(t_lane, v);
        tc::tmem_wait_ld();
        if (mine) {
          float act[kOut];
#pragma unroll
          for (int o = 0; o < kOut; ++o) act[o] = tc::tanh_approx(v[o]);
          finish(act, v);
        }
      } else {
        // hidden layer: tanh, packed to BF16 and written over the consumed layer-1 columns of
        // this thread's TMEM lane (BF16 column pair c holds hidden units 2c, 2c + 1): the
        // layer-2 A operand. Chunk c16's 8 packed columns lie inside the 16 columns it was
        // loaded from or an earlier chunk's. The store is warp-wide; rows of other genomes
        // store values that only their discarded layer-2 outputs use.
#pragma unroll
        for (int c16 = 0; c16 < N1 / 16; ++c16) {
          float v[16];
          tc::tmem_ld16(t_lane + c16 * 16, v);
          tc::tmem_wait_ld();
          uint32_t pk[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) pk[i] = tc::pack_bf16x2(tc::tanh_approx(v[2 * i]), tc::tanh_approx(v[2 * i + 1]));
          tc::tmem_st8(t_lane + c16 * 8, pk);
        }
        tc::tmem_wait_st();
        tc::tc_fence_before();
        if (__syncthreads_or(bad)) {
          timed_out = true;
          break;
        }
        if (tid == 0) {
          tc::tc_fence_after();
          const uint64_t bd = tc::sdesc_sw128(w_s + bf16_w2_off(H));
#pragma unroll
          for (int k = 0; k < N1 / 16; ++k) tc::mma_bf16_ts(tmem + kD2Col, tmem + 8 * k, bd + 2 * k, idesc2, k > 0);
          tc::mma_commit(mbar);
        }
        if (!tc::mbar_wait(mbar, phase, kWaitCycles)) bad = true;
        phase ^= 1;
        tc::tc_fence_after();
        float v[16];
        tc::tmem_ld16(t_lane + kD2Col, v);
        tc::tmem_wait_ld();
        if (restage) {                                // the blob's bytes seen by this thread too
          if (!tc::mbar_wait(w_bar, w_phase, kWaitCycles)) bad = true;
        }
        if (mine) {
          const float* b2 = reinterpret_cast<const float*>(base + kOffW + bf16_b2_off(H));
          float act[kOut];
#pragma unroll
          for (int o = 0; o < kOut; ++o) {
            v[o] += b2[o];
            act[o] = tc::tanh_approx(v[o]);
          }
          finish(act, v);
        }
      }
      tc::tc_fence_before();
      if (restage) {
        staged = gs;
        w_phase ^= 1u;
      }
      if (mine) done = true;
      first_round = false;
      rb ^= 1;
    }
    if (timed_out) break;
    if (++ntile == 16) {
      ntile = 0;
      flush();
    }
    cur = nxt;
    run_end = nxt_end;
    ++it;
  }
  tc::cp_async_wait_all();                            // no copy may land after the CTA exits
  if (tid == 0 && tma_pending) tc::mbar_wait(halo_bar, halo_phase, kWaitCycles);

  flush();
  int ex = accX;
#pragma unroll
  for (int off = 16; off; off >>= 1) ex += __shfl_xor_sync(0xffffffffu, ex, off);
  if (lane == 0) red_c[warp] = ex;
  tc::tc_fence_before();
  if (__syncthreads_or(bad || timed_out) && tid == 0) atomicCAS(a.status, 0, (int)CORAL_E_TIMEOUT);
  if (tid == 0) {
    Partial p = {};
    long long cs[4] = {0, 0, 0, 0};
    for (int w = 0; w < 4; ++w) {
      for (int k = 0; k < 4; ++k) cs[k] += red_s[w][k];
      p.c[0] += red_c[w];
    }
    // exact in FP64 (integers below 2^53 times a power of two), and so are the FP64 sums of
    // these partials: the totals do not depend on the order of the partials
    for (int k = 0; k < 4; ++k) p.s[2 + k] = (double)cs[k] / (double)kCFix;
    a.part1[cta] = p;
    // the pool is free again for the next launch: the last CTA to finish resets its counters
    __threadfence();
    if (atomicAdd(a.sched + 1, 1) == ncta - 1) {
      a.sched[0] = 0;
      a.sched[1] = 0;
      __threadfence();
    }
  }
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <int kH, bool kFma>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    k_pass1_bf16(const __grid_constant__ StepArgs a, const __grid_constant__ CUtensorMap tmap, const int use_tma) {
  pass1_bf16_body<kH, kFma>(a, &tmap, use_tma, blockIdx.x, gridDim.x);
}

template <int kH, bool kFma>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_pass1_bf16_batch(const __grid_constant__ BatchTable bt,
                                                                          const int parity) {
  __shared__ StepArgs sa;
  const int w = bt.cta_world1[blockIdx.x];
  copy_args_to_shared(&sa, &bt.args[parity * bt.n + w]);
  // this world's TMA descriptor lives in global memory (written by the host): thread 0, which
  // issues the copies, orders it for the tensor-map proxy before the first use
  const CUtensorMap* tm = bt.tmaps + parity * bt.n + w;
  const int use_tma = bt.tma_ok[w];
  if (use_tma && threadIdx.x == 0) tc::fence_tensormap_acquire(tm);
  __syncthreads();
  pass1_bf16_body<kH, kFma>(sa, tm, use_tma, blockIdx.x - bt.world_first1[w], bt.world_ctas1[w]);
}

// A wait that must run out: nothing arrives on the barrier. Same bounded wait, error report
// and TMEM release as the tensor-core kernel's timeout path.
__global__ void __launch_bounds__(128) k_selftest_wait(long long max_cycles, int* status) {
  __shared__ uint64_t bar;
  __shared__ uint32_t slot;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&slot, 32);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  bool ok = true;
  if (threadIdx.x == 0) ok = tc::mbar_wait(&bar, 0, max_cycles);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicCAS(status, 0, (int)CORAL_E_TIMEOUT);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(slot, 32);
  }
}

// Special-function unit throughput probe: eight independent tanh.approx.f32 chains per thread
// (the instruction the hidden and output activations use); sink is written only if the chains
// end on an impossible value, which keeps them live.
__global__ void __launch_bounds__(256) k_sfu_probe(int iters, float* sink) {
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = 0.25f + 1e-3f * (float)(threadIdx.x + 37 * k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = tc::tanh_approx(v[k]);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  if (s == 12345.5f) sink[blockIdx.x] = s;
}

}  // namespace

cudaError_t launch_sfu_probe(int blocks, int iters, float* sink, cudaStream_t st) {
  k_sfu_probe<<<blocks, 256, 0, st>>>(iters, sink);
  return cudaGetLastError();
}

cudaError_t launch_selftest_wait(long long max_cycles, int* status, cudaStream_t st) {
  k_selftest_wait<<<1, 128, 0, st>>>(max_cycles, status);
  return cudaGetLastError();
}

size_t pass1_bf16_smem() { return kSmemBytes; }

namespace {
// the kernel instantiations, indexed by hidden size / 16 (0, 16, 32, 48, 64)
using P1Fn = void (*)(StepArgs, CUtensorMap, int);
using P1BFn = void (*)(BatchTable, int);
// [FMA small-genome path off / on][hidden size / 16]
const P1Fn kP1[2][5] = {{k_pass1_bf16<0, false>, k_pass1_bf16<16, false>, k_pass1_bf16<32, false>,
                         k_pass1_bf16<48, false>, k_pass1_bf16<64, false>},
                        {k_pass1_bf16<0, true>, k_pass1_bf16<16, true>, k_pass1_bf16<32, true>,
                         k_pass1_bf16<48, true>, k_pass1_bf16<64, true>}};
const P1BFn kP1B[2][5] = {{k_pass1_bf16_batch<0, false>, k_pass1_bf16_batch<16, false>, k_pass1_bf16_batch<32, false>,
                           k_pass1_bf16_batch<48, false>, k_pass1_bf16_batch<64, false>},
                          {k_pass1_bf16_batch<0, true>, k_pass1_bf16_batch<16, true>, k_pass1_bf16_batch<32, true>,
                           k_pass1_bf16_batch<48, true>, k_pass1_bf16_batch<64, true>}};
int hidden_index(int hidden) { return (hidden >= 0 && hidden <= 64 && hidden % 16 == 0) ? hidden / 16 : -1; }
}  // namespace

long long pass1_bf16_tiles(int W, int H) {
  return (long long)((W + kTileW - 1) / kTileW) * ((H + kTileH - 1) / kTileH);
}

int pass1_bf16_grid(int sms) {
  int dev = 0, major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major != 10) return 0;                                  // tcgen05 needs the sm_100 family
  int per_sm = kCtasPerSm, max_regs = 0, static_smem = 0;
  for (int k = 0; k < 10; ++k) {
    const void* fn = reinterpret_cast<const void*>(kP1[k / 5][k % 5]);
    int n = 0;
    cudaFuncAttributes fa;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kThreads, kSmemBytes) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    if (n < per_sm) per_sm = n;
    if (fa.numRegs > max_regs) max_regs = fa.numRegs;
    if ((int)fa.sharedSizeBytes > static_smem) static_smem = (int)fa.sharedSizeBytes;
  }
  // Residency is bounded by TMEM (kCtasPerSm x 64 of 512 columns) and by the register and
  // shared-memory budgets the kernels were compiled for, which allow kCtasPerSm (the occupancy
  // query does not count the shared-memory carveout the launch asks for).
  if (per_sm < kCtasPerSm) {
    int smem_sm = 0, regs_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    const int by_smem = smem_sm / (kSmemBytes + static_smem + 1024);
    const int by_regs = max_regs > 0 ? regs_sm / (max_regs * kThreads) : 0;
    const int est = by_smem < by_regs ? by_smem : by_regs;
    if (est > per_sm) per_sm = est;
  }
  if (per_sm > kCtasPerSm) per_sm = kCtasPerSm;
  if (per_sm < 1) return 0;
  const int g = per_sm * sms;
  return g > kMaxPartials ? kMaxPartials : g;
}

cudaError_t prepare_pass1_bf16_batch() {
  for (int k = 0; k < 10; ++k) {
    const void* fn = reinterpret_cast<const void*>(kP1B[k / 5][k % 5]);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_pass1_bf16_batch(const BatchTable& b, int parity, int grid, int hidden, bool fma,
                                    cudaStream_t st) {
  const int k = hidden_index(hidden);
  if (k < 0) return cudaErrorInvalidValue;
  kP1B[fma ? 1 : 0][k]<<<grid, kThreads, kSmemBytes, st>>>(b, parity);
  return cudaGetLastError();
}

cudaError_t launch_pass1_bf16(const StepArgs& a, const CUtensorMap* tmap, cudaStream_t st, int grid) {
  const int k = hidden_index(a.hidden);
  if (k < 0) return cudaErrorInvalidValue;
  CUtensorMap m;
  if (tmap)
    m = *tmap;
  else
    memset(&m, 0, sizeof(m));
  kP1[a.fma_cutoff > 0 ? 1 : 0][k]<<<grid, kThreads, kSmemBytes, st>>>(a, m, tmap ? 1 : 0);
  return cudaGetLastError();
}

bool encode_sensor_tmap(CUtensorMap* map, const float* E, int W, int H, int P) {
  // rows (pitch P) must be a multiple of 16 bytes; the torus must hold the 40-wide box and 6 rows
  if ((P & 3) != 0 || W < kStageW || H < kHaloH) return false;
  if ((reinterpret_cast<uintptr_t>(E) & 15) != 0) return false;
  // looked up once (a function-local static: thread-safe initialisation)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, 6};
  const cuuint64_t strides[2] = {(cuuint64_t)P * 4, (cuuint64_t)P * (cuuint64_t)H * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kStageW, (cuuint32_t)kHaloH, 6};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(E), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace coral
