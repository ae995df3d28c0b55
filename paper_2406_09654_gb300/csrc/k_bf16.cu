// BF16 tensor-core network (pass 1) on tcgen05. Each CTA (128 threads) walks a contiguous run
// of 32x8-cell tiles of the torus; every thread owns two cells of a tile (rows w and w + 4 of
// the tile for warp w, column = lane), so the tile is two 128-row MMA operands. While a tile is
// processed, the next tile's one-cell halo of the six sensor channels is copied into shared
// memory with cp.async. Per tile: BF16 records (6 channels of a halo cell in 16 bytes) are
// built once; each cell assembles its 128 x 64 input row (the rotation-ordered 3x3
// neighbourhood, K index 6*rank + channel, a constant 1 at K = 54 that carries the layer-1
// bias) in the 128-byte swizzled layout; one thread issues the layer-1 MMAs (128 x H x 64 per
// half, FP32 accumulation in TMEM columns [64h, 64h + H)) and waits on an mbarrier (bounded);
// the epilogue applies tanh, packs BF16 over the consumed input rows, the layer-2 MMAs
// (128 x 16 x H) reuse the TMEM columns, and the actuator epilogue (communication,
// invest/liquidate, exploration, flow quotient) writes the pass-1 buffers. A tile with several
// genomes runs one round per genome (rows of other genomes are computed and discarded).
#include <math.h>

#include "coral_internal.cuh"
#include "epilogue.cuh"
#include "tc_ptx.cuh"

namespace coral {

namespace {

constexpr int kThreads = 128;
constexpr int kCtasPerSm = 3;
constexpr int kHalves = 2;                                // cells per thread / MMA operands per tile
constexpr int kTileW = 32, kTileH = 4 * kHalves;          // 32 x 8 cells
constexpr int kHaloW = kTileW + 2, kHaloH = kTileH + 2;   // 34 x 10
constexpr int kHaloCells = kHaloW * kHaloH;               // 340
constexpr int kSegments = 6 * kHaloH;                     // channel x halo-row segments
constexpr int kSegPerWarp = kSegments / (kThreads / 32);  // 15
constexpr uint32_t kTmemCols = 128;                       // half h: columns [64h, 64h + 64)
constexpr long long kWaitCycles = 4000000000LL;           // about 2 s of SM clock

// shared memory layout, offsets from a 1024-byte aligned base
constexpr int kOffA = 0;                                  // 2 x (128 x 128 B): input, then hidden tile
constexpr int kOffW = 32768;                              // genome blob (<= 10368 B)
constexpr int kStageBytes = 8192;                         // float32 [6][340], two buffers
constexpr int kOffStage = kOffW + 11264;
constexpr int kOffRec = kOffStage + 2 * kStageBytes;      // 340 x 16 B BF16 cell records
constexpr int kOffG = kOffRec + kHaloCells * 16;          // int32 [256]
constexpr int kOffSeg = kOffG + 1024;                     // int64 [4][15] segment offsets
constexpr int kOffMisc = kOffSeg + 8 * kSegments;         // mbarrier, TMEM slot, flags, ballots
constexpr int kSmemBytes = kOffMisc + 128 + 1024;         // + alignment slack

static_assert(kStageBytes >= 6 * kHaloCells * 4, "stage buffer too small");
static_assert(kSegments % (kThreads / 32) == 0, "segments must split evenly over the warps");

// v in [-1, n + tile) folded onto [0, n): one conditional step when the torus side is at least
// the halo's (small = false), else a full modulo.
__device__ __forceinline__ int fold(int v, int n, bool small) {
  if (small) {
    v %= n;
    return v < 0 ? v + n : v;
  }
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

// Record-index offset (dy * 34 + dx) of kernel ranks 1..8 for rotation r, one signed byte per
// rank (rank p in bits 8(p-1)..8p-1), from the same octant tables as the FP32 path.
__host__ __device__ constexpr unsigned long long rank_offsets(int r) {
  unsigned long long v = 0;
  for (int p = 1; p < 9; ++p) {
    const int o = (2 * r + rank_delta(p)) & 7;
    const int dx = (int)((0x1A9u >> (2 * o)) & 3u) - 1, dy = (int)((0x1A90u >> (2 * o)) & 3u) - 1;
    v |= (unsigned long long)(uint8_t)(int8_t)(dy * kHaloW + dx) << (8 * (p - 1));
  }
  return v;
}

// Starts the asynchronous copy of a tile's 34 x 10 halo of the six contiguous sensor planes into
// a stage buffer [6][10][34] floats: warp w copies segments w, w+4, ... (one per channel and
// halo row; seg[k] = channel * N + halo-row * W of its k-th segment); lane l copies column l,
// lanes 0 and 1 also columns 32 and 33 (col_a / col_b: their wrapped grid columns).
__device__ __forceinline__ void issue_halo(const StepArgs& a, int y0, int col_a, int col_b, uint32_t dst,
                                           const long long* seg) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool wraps = y0 == 0 || y0 - 1 + kHaloH > a.H;
  const long long row0 = (long long)(y0 - 1) * a.W;
  const bool small_h = a.H < kHaloH;
#pragma unroll 5
  for (int k = 0; k < kSegPerWarp; ++k) {
    const int sgm = warp + k * (kThreads / 32);
    const int ch = sgm / kHaloH, hy = sgm - ch * kHaloH;
    const long long off = wraps ? (long long)ch * a.N + (long long)fold(y0 - 1 + hy, a.H, small_h) * a.W
                                : seg[k] + row0;
    const float* row = a.cur.E + off;
    const uint32_t d = dst + 4u * (uint32_t)(ch * kHaloCells + hy * kHaloW);
    tc::cp_async4(d + 4u * lane, row + col_a);
    if (lane < 2) tc::cp_async4(d + 4u * (32 + lane), row + col_b);
  }
  tc::cp_async_commit();
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_pass1_bf16(const StepArgs a) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_s = tc::smem_u32(smem_raw);
  const uint32_t base_s = (raw_s + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_s - raw_s);
  int32_t* sG = reinterpret_cast<int32_t*>(base + kOffG);
  long long* sSeg = reinterpret_cast<long long*>(base + kOffSeg);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + kOffMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + kOffMisc + 8);
  int* wgenome = reinterpret_cast<int*>(base + kOffMisc + 12);
  unsigned* ballots = reinterpret_cast<unsigned*>(base + kOffMisc + 32);    // [8]
  __shared__ double red_s[4][4];
  __shared__ long long red_c[4];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = a.W, Hh = a.H;
  const int H = a.hidden;
  const int N1 = H ? H : 16;
  const uint32_t rec_s = base_s + kOffRec;
  const uint32_t w_s = base_s + kOffW;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    tc::fence_barrier_init();
    *wgenome = -1;
  }
  if (tid < kSegments) {
    const int w = tid % 4, k = tid / 4, ch = tid / kHaloH, hy = tid - ch * kHaloH;
    sSeg[w * kSegPerWarp + k] = (long long)ch * a.N + (long long)hy * W;    // segment tid = w + 4k
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t idesc1 = tc::idesc_bf16_f32(128, N1);
  const uint32_t idesc2 = tc::idesc_bf16_f32(128, 16);
  const long long* seg = sSeg + warp * kSegPerWarp;
  uint32_t phase = 0;

  double accC[4] = {0, 0, 0, 0};
  long long accX = 0;
  float cacc[4] = {0, 0, 0, 0};           // FP32 partials of up to 8 tiles, then into accC
  int ntile = 0;
  bool timed_out = false;
  const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (Hh + kTileH - 1) / kTileH;
  const int n_tiles = tiles_x * tiles_y;
  // a contiguous run of tiles per CTA: neighbouring tiles share halo rows (L2) and genomes
  const int per = (n_tiles + gridDim.x - 1) / gridDim.x;
  const int t_begin = blockIdx.x * per;
  const int t_end = t_begin + per < n_tiles ? t_begin + per : n_tiles;
  const bool small_w = W < kHaloW;

  int g_next[kHalves], r_next[kHalves];
  // next tile: halo copy started; genome and rotation of this thread's cells loaded
  auto prefetch = [&](int tile, uint32_t dst) {
    const int ty = tile / tiles_x;
    const int x0 = (tile - ty * tiles_x) * kTileW, y0 = ty * kTileH;
    issue_halo(a, y0, fold(x0 - 1 + lane, W, small_w), fold(x0 + 31 + lane, W, small_w), dst, seg);
    const int gx = x0 + lane;
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
      const int gy = y0 + 4 * h + warp;
      g_next[h] = -1;
      r_next[h] = 0;
      if (gx < W && gy < Hh) {
        const int jn = gy * W + gx;
        g_next[h] = __ldg(a.cur.G + jn);
        r_next[h] = a.rotation ? (int)__ldg(a.cur.R + jn) : 0;
      }
    }
  };
  if (t_begin < t_end) prefetch(t_begin, base_s + kOffStage);

  int buf = 0;
  for (int tile = t_begin; tile < t_end; ++tile, buf ^= 1) {
    const int ty = tile / tiles_x;
    const int x0 = (tile - ty * tiles_x) * kTileW, y0 = ty * kTileH;
    const int gx = x0 + lane;
    int g[kHalves], r[kHalves], hc[kHalves];
    bool valid[kHalves], done[kHalves];
    long long j[kHalves];
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
      const int gy = y0 + 4 * h + warp;
      valid[h] = gx < W && gy < Hh;
      j[h] = (long long)gy * W + gx;
      g[h] = g_next[h];
      r[h] = r_next[h];
      hc[h] = (4 * h + warp + 1) * kHaloW + (lane + 1);
      done[h] = g[h] < 0;
      sG[h * kThreads + tid] = g[h];
    }
    tc::cp_async_wait_all();
    __syncthreads();                                  // this tile's halo is in stage[buf]
    if (tile + 1 < t_end) prefetch(tile + 1, base_s + kOffStage + (buf ^ 1) * kStageBytes);
    const float* stage = reinterpret_cast<const float*>(base + kOffStage + buf * kStageBytes);
    // BF16 records: the 6 channels of each halo cell in one 16-byte slot
    for (int c = tid; c < kHaloCells; c += kThreads) {
      const float* s = stage + c;
      tc::sts128(rec_s + c * 16, tc::pack_bf16x2(s[0], s[kHaloCells]),
                 tc::pack_bf16x2(s[2 * kHaloCells], s[3 * kHaloCells]),
                 tc::pack_bf16x2(s[4 * kHaloCells], s[5 * kHaloCells]), 0u);
    }
    __syncthreads();
    float act[kHalves][kOut], zo[kHalves][kOut];
#pragma unroll
    for (int h = 0; h < kHalves; ++h)
#pragma unroll
      for (int o = 0; o < kOut; ++o) act[h][o] = zo[h][o] = 0.0f;
    // one tensor-core round per genome present in the tile (the first pending row's genome)
    while (true) {
#pragma unroll
      for (int h = 0; h < kHalves; ++h) {
        const unsigned b = __ballot_sync(0xffffffffu, !done[h]);
        if (lane == 0) ballots[h * 4 + warp] = b;
      }
      __syncthreads();
      int first = -1;
#pragma unroll
      for (int w = 0; w < 2 * 4; ++w) {
        const unsigned bw = ballots[w];
        if (first < 0 && bw) first = w * 32 + __ffs(bw) - 1;
      }
      const int gs = first < 0 ? -1 : sG[first];
      if (gs < 0) break;
      if (*wgenome != gs) {                           // stage this genome's BF16 blob
        const uint4* src = reinterpret_cast<const uint4*>(a.nets16 + (long long)gs * a.blob_bytes);
        const int n16 = a.blob_bytes >> 4;             // <= 648 = 6 x 108 per thread slot
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          uint4 v[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int i = tid + (3 * part + k) * kThreads;
            if (i < n16) v[k] = __ldg(src + i);
          }
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int i = tid + (3 * part + k) * kThreads;
            if (i < n16) tc::sts128(w_s + i * 16, v[k].x, v[k].y, v[k].z, v[k].w);
          }
        }
      }
      // input rows: 9 records in kernel-rank order, 1.0 at K = 54, swizzled
#pragma unroll
      for (int h = 0; h < kHalves; ++h) {
        uint32_t wv[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) wv[i] = 0u;
        if (valid[h]) {
          const uint32_t c_s = rec_s + hc[h] * 16;
          uint4 rc = tc::lds128(c_s);
          wv[0] = rc.x; wv[1] = rc.y; wv[2] = rc.z;
          const unsigned long long offs = r[h] == 0 ? rank_offsets(0) : r[h] == 1 ? rank_offsets(1)
                                        : r[h] == 2 ? rank_offsets(2) : rank_offsets(3);
#pragma unroll
          for (int p = 1; p < 9; ++p) {
            const int off = (int)(int8_t)(uint8_t)(offs >> (8 * (p - 1)));
            rc = tc::lds128(c_s + off * 16);
            wv[3 * p] = rc.x; wv[3 * p + 1] = rc.y; wv[3 * p + 2] = rc.z;
          }
          wv[27] = 0x3F80u;                  // bf16 1.0 at K = 54 (layer-1 bias), 0 at K = 55
        }
        const uint32_t row_s = base_s + kOffA + h * 16384 + tid * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c)
          tc::sts128(row_s + ((c ^ (tid & 7)) << 4), wv[4 * c], wv[4 * c + 1], wv[4 * c + 2], wv[4 * c + 3]);
      }
      tc::fence_proxy_async();
      __syncthreads();
      bool ok = true;
      if (tid == 0) {          // one thread issues and waits; the others park at the barrier
        *wgenome = gs;
        tc::tc_fence_after();
        const uint64_t bd = tc::sdesc_sw128(w_s);
#pragma unroll
        for (int h = 0; h < kHalves; ++h) {
          const uint64_t ad = tc::sdesc_sw128(base_s + kOffA + h * 16384);
#pragma unroll
          for (int k = 0; k < 4; ++k) tc::mma_bf16(tmem + 64 * h, ad + 2 * k, bd + 2 * k, idesc1, k > 0);
        }
        tc::mma_commit(mbar);
        ok = tc::mbar_wait(mbar, phase, kWaitCycles);
      }
      phase ^= 1;
      if (__syncthreads_or(!ok)) { timed_out = true; break; }
      tc::tc_fence_after();
      bool mine[kHalves];
#pragma unroll
      for (int h = 0; h < kHalves; ++h) mine[h] = !done[h] && g[h] == gs;
      if (H == 0) {
#pragma unroll
        for (int h = 0; h < kHalves; ++h) {
          float v[16];
          tc::tmem_ld16(t_lane + 64 * h, v);
          tc::tmem_wait_ld();
          if (mine[h]) {
#pragma unroll
            for (int o = 0; o < kOut; ++o) {
              zo[h][o] = v[o];
              act[h][o] = tc::tanh_approx(v[o]);
            }
          }
        }
      } else {
        // hidden layer: tanh, BF16, written over this row of the (consumed) input tile
#pragma unroll
        for (int h = 0; h < kHalves; ++h) {
          const uint32_t row_s = base_s + kOffA + h * 16384 + tid * 128;
          for (int c16 = 0; c16 < N1 / 16; ++c16) {
            float v[16];
            tc::tmem_ld16(t_lane + 64 * h + c16 * 16, v);
            tc::tmem_wait_ld();
            if (mine[h]) {
              uint32_t pk[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) pk[i] = tc::pack_bf16x2(tc::tanh_approx(v[2 * i]), tc::tanh_approx(v[2 * i + 1]));
              tc::sts128(row_s + (((2 * c16) ^ (tid & 7)) << 4), pk[0], pk[1], pk[2], pk[3]);
              tc::sts128(row_s + (((2 * c16 + 1) ^ (tid & 7)) << 4), pk[4], pk[5], pk[6], pk[7]);
            }
          }
        }
        tc::fence_proxy_async();
        tc::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
          tc::tc_fence_after();
          const uint64_t bd = tc::sdesc_sw128(w_s + bf16_w2_off(H));
#pragma unroll
          for (int h = 0; h < kHalves; ++h) {
            const uint64_t ad = tc::sdesc_sw128(base_s + kOffA + h * 16384);
            for (int k = 0; k < N1 / 16; ++k) tc::mma_bf16(tmem + 64 * h, ad + 2 * k, bd + 2 * k, idesc2, k > 0);
          }
          tc::mma_commit(mbar);
          ok = tc::mbar_wait(mbar, phase, kWaitCycles);
        }
        phase ^= 1;
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        tc::tc_fence_after();
        const float* b2 = reinterpret_cast<const float*>(base + kOffW + bf16_b2_off(H));
#pragma unroll
        for (int h = 0; h < kHalves; ++h) {
          float v[16];
          tc::tmem_ld16(t_lane + 64 * h, v);
          tc::tmem_wait_ld();
          if (mine[h]) {
#pragma unroll
            for (int o = 0; o < kOut; ++o) {
              zo[h][o] = v[o] + b2[o];
              act[h][o] = tc::tanh_approx(zo[h][o]);
            }
          }
        }
      }
      tc::tc_fence_before();
#pragma unroll
      for (int h = 0; h < kHalves; ++h)
        if (mine[h]) done[h] = true;
    }
    if (timed_out) break;
    // actuator epilogue and pass-1 stores
    const float* sI = stage + kHaloCells;
#pragma unroll
    for (int h = 0; h < kHalves; ++h) {
      if (!valid[h]) continue;
      CellOut o;
      const int c = hc[h];
      const double S = (double)sI[c - kHaloW] + (double)sI[c + 1] + (double)sI[c + kHaloW] + (double)sI[c - 1];
      actuator_epilogue<true>(a, act[h], zo[h], stage[c], sI[c], S, r[h], o);
      store_pass1(a, j[h], o);
#pragma unroll
      for (int k = 0; k < 4; ++k) cacc[k] += o.C[k];
      accX += o.xdir != kNoExplore ? 1 : 0;
    }
    if (++ntile == 4) {
      ntile = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        accC[k] += (double)cacc[k];
        cacc[k] = 0.0f;
      }
    }
  }
  tc::cp_async_wait_all();                            // no copy may land after the CTA exits

  if (timed_out && tid == 0) atomicCAS(a.status, 0, (int)CORAL_E_TIMEOUT);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = accC[k] + (double)cacc[k];
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    accC[k] = v;
  }
  long long ex = accX;
#pragma unroll
  for (int off = 16; off; off >>= 1) ex += __shfl_xor_sync(0xffffffffu, ex, off);
  accX = ex;
  if (lane == 0) {
    for (int k = 0; k < 4; ++k) red_s[warp][k] = accC[k];
    red_c[warp] = accX;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    Partial p = {};
    for (int w = 0; w < 4; ++w) {
      for (int k = 0; k < 4; ++k) p.s[2 + k] += red_s[w][k];
      p.c[0] += red_c[w];
    }
    a.part1[blockIdx.x] = p;
  }
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

size_t pass1_bf16_smem() { return kSmemBytes; }

int pass1_bf16_grid(int sms) {
  int dev = 0, major = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major != 10) return 0;                                  // tcgen05 needs the sm_100 family
  if (cudaFuncSetAttribute(k_pass1_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess ||
      cudaFuncSetAttribute(k_pass1_bf16, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass1_bf16, kThreads, kSmemBytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // Residency is bounded by TMEM (kCtasPerSm x 128 of 512 columns) and by the register and
  // shared-memory budgets the kernel was compiled for, which allow kCtasPerSm.
  if (per_sm < kCtasPerSm) {
    int smem_sm = 0, regs_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_pass1_bf16) == cudaSuccess) {
      const int by_smem = smem_sm / (kSmemBytes + (int)fa.sharedSizeBytes + 1024);
      const int by_regs = regs_sm / (fa.numRegs * kThreads);
      int est = by_smem < by_regs ? by_smem : by_regs;
      if (est > per_sm) per_sm = est;
    }
  }
  if (per_sm > kCtasPerSm) per_sm = kCtasPerSm;
  if (per_sm < 1) return 0;
  const int g = per_sm * sms;
  return g > kMaxPartials ? kMaxPartials : g;
}

cudaError_t launch_pass1_bf16(const StepArgs& a, cudaStream_t st, int grid) {
  k_pass1_bf16<<<grid, kThreads, kSmemBytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace coral
