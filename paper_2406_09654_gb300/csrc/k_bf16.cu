// BF16 tensor-core network (pass 1) on tcgen05: each CTA takes 32x4-cell tiles of the torus,
// stages the tile plus a one-cell halo of the six sensor channels in shared memory, builds the
// 128 x 64 BF16 input tile (the rotation-ordered 3x3 neighbourhood of every cell, K index
// 6*rank + channel, a constant 1 at K = 54 that carries the layer-1 bias), and runs the genome
// nets on the tensor cores with FP32 accumulation in TMEM: one 128 x H x 64 MMA for layer 1,
// tanh in the epilogue, one 128 x 16 x H MMA for layer 2. A tile with several genomes runs one
// round per genome (the rows of other genomes are computed and discarded). The actuator
// epilogue (communication, invest/liquidate, exploration, flow quotient) follows in registers.
#include <math.h>

#include "coral_internal.cuh"
#include "epilogue.cuh"
#include "tc_ptx.cuh"

namespace coral {

namespace {

constexpr int kThreads = 128;
constexpr int kTileW = 32, kTileH = 4;
constexpr int kHaloW = kTileW + 2, kHaloH = kTileH + 2;
constexpr int kHaloCells = kHaloW * kHaloH;               // 204
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kL2Col = 64;                           // TMEM column of the layer-2 accumulator
constexpr long long kWaitCycles = 4000000000LL;           // about 2 s of SM clock

// shared memory layout, offsets from a 1024-byte aligned base
constexpr int kOffA = 0;                                  // 128 rows x 128 B input tile
constexpr int kOffA2 = 16384;                             // 128 rows x 128 B hidden tile
constexpr int kOffW = 32768;                              // genome blob (<= 10368 B)
constexpr int kOffStage = kOffW + 11264;                  // float32 [6][204]
constexpr int kOffRec = kOffStage + 4928;                 // 204 x 16 B BF16 cell records
constexpr int kOffG = kOffRec + kHaloCells * 16;          // int32 [128]
constexpr int kOffMisc = kOffG + 512;                     // mbarrier, TMEM slot, flags
constexpr int kSmemBytes = kOffMisc + 128 + 1024;         // + alignment slack

__device__ __forceinline__ int modp(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__global__ void __launch_bounds__(kThreads, 4) k_pass1_bf16(const StepArgs a) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_s = tc::smem_u32(smem_raw);
  const uint32_t base_s = (raw_s + 1023u) & ~1023u;
  uint8_t* base = smem_raw + (base_s - raw_s);
  float* stage = reinterpret_cast<float*>(base + kOffStage);
  int32_t* sG = reinterpret_cast<int32_t*>(base + kOffG);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + kOffMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + kOffMisc + 8);
  int* wgenome = reinterpret_cast<int*>(base + kOffMisc + 12);
  int* sel = reinterpret_cast<int*>(base + kOffMisc + 16);
  unsigned* ballots = reinterpret_cast<unsigned*>(base + kOffMisc + 20);
  __shared__ double red_s[4][4];
  __shared__ long long red_c[4];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W = a.W, Hh = a.H;
  const long long N = a.N;
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
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t idesc1 = tc::idesc_bf16_f32(128, N1);
  const uint32_t idesc2 = tc::idesc_bf16_f32(128, 16);
  uint32_t phase = 0;

  double accC[4] = {0, 0, 0, 0};
  long long accX = 0;
  bool timed_out = false;
  const int tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (Hh + kTileH - 1) / kTileH;
  const long long n_tiles = (long long)tiles_x * tiles_y;

  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int x0 = (int)(tile % tiles_x) * kTileW, y0 = (int)(tile / tiles_x) * kTileH;
    // 1. tile + halo of the six sensor channels, float32, wrap-around
    for (int i = tid; i < 6 * kHaloCells; i += kThreads) {
      const int ch = i / kHaloCells, c = i - ch * kHaloCells;
      const int hy = c / kHaloW, hx = c - hy * kHaloW;
      const long long n = (long long)modp(y0 - 1 + hy, Hh) * W + modp(x0 - 1 + hx, W);
      const float* plane = ch == 0 ? a.cur.E : (ch == 1 ? a.cur.I : a.cur.C + (long long)(ch - 2) * N);
      stage[i] = __ldg(plane + n);
    }
    const int gx = x0 + lane, gy = y0 + warp;
    const bool valid = gx < W && gy < Hh;
    const long long j = (long long)gy * W + gx;
    int g = -1, r = 0;
    if (valid) {
      g = __ldg(a.cur.G + j);
      r = a.rotation ? (int)__ldg(a.cur.R + j) : 0;
    }
    sG[tid] = g;
    __syncthreads();
    // 2. BF16 records: 6 channels of each halo cell in one 16-byte slot
    for (int c = tid; c < kHaloCells; c += kThreads) {
      const float* s = stage + c;
      tc::sts128(rec_s + c * 16, tc::pack_bf16x2(s[0], s[kHaloCells]),
                 tc::pack_bf16x2(s[2 * kHaloCells], s[3 * kHaloCells]),
                 tc::pack_bf16x2(s[4 * kHaloCells], s[5 * kHaloCells]), 0u);
    }
    __syncthreads();
    // 3. this cell's input row: 9 records in kernel-rank order, 1.0 at K = 54, swizzled
    const int hc = (warp + 1) * kHaloW + (lane + 1);
    {
      uint32_t wv[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) wv[i] = 0u;
      if (valid) {
        uint4 rc = tc::lds128(rec_s + hc * 16);
        wv[0] = rc.x; wv[1] = rc.y; wv[2] = rc.z;
#pragma unroll
        for (int p = 1; p < 9; ++p) {
          int dx, dy;
          octant_offset((2 * r + rank_delta(p)) & 7, dx, dy);
          rc = tc::lds128(rec_s + (hc + dy * kHaloW + dx) * 16);
          wv[3 * p] = rc.x; wv[3 * p + 1] = rc.y; wv[3 * p + 2] = rc.z;
        }
        wv[27] = 0x3F80u;                    // bf16 1.0 at K = 54 (layer-1 bias), 0 at K = 55
      }
      const uint32_t row_s = base_s + kOffA + tid * 128;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        tc::sts128(row_s + ((c ^ (tid & 7)) << 4), wv[4 * c], wv[4 * c + 1], wv[4 * c + 2], wv[4 * c + 3]);
      tc::fence_proxy_async();
    }
    // 4. one tensor-core round per genome present in the tile
    bool done = g < 0;
    float act[kOut], zo[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) act[o] = zo[o] = 0.0f;
    while (true) {
      const unsigned b = __ballot_sync(0xffffffffu, !done);
      if (lane == 0) ballots[warp] = b;
      __syncthreads();
      if (tid == 0) {
        int first = -1;
        for (int w = 0; w < 4 && first < 0; ++w)
          if (ballots[w]) first = w * 32 + __ffs(ballots[w]) - 1;
        *sel = first < 0 ? -1 : sG[first];
      }
      __syncthreads();
      const int gs = *sel;
      if (gs < 0) break;
      if (*wgenome != gs) {                                      // stage this genome's BF16 blob
        const uint4* src = reinterpret_cast<const uint4*>(a.nets16 + (long long)gs * a.blob_bytes);
        for (int i = tid; i < a.blob_bytes / 16; i += kThreads) {
          const uint4 v = __ldg(src + i);
          tc::sts128(w_s + i * 16, v.x, v.y, v.z, v.w);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) *wgenome = gs;
      }
      if (tid == 0) {
        tc::tc_fence_after();
        const uint64_t ad = tc::sdesc_sw128(base_s + kOffA), bd = tc::sdesc_sw128(w_s);
#pragma unroll
        for (int k = 0; k < 4; ++k) tc::mma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc1, k > 0);
        tc::mma_commit(mbar);
      }
      bool ok = tc::mbar_wait(mbar, phase, kWaitCycles);
      phase ^= 1;
      if (__syncthreads_or(!ok)) { timed_out = true; break; }
      tc::tc_fence_after();
      const bool mine = !done && g == gs;
      if (H == 0) {
        float v[16];
        tc::tmem_ld16(t_lane, v);
        tc::tmem_wait_ld();
        if (mine) {
#pragma unroll
          for (int o = 0; o < kOut; ++o) {
            zo[o] = v[o];
            act[o] = tc::tanh_approx(v[o]);
          }
        }
      } else {
        const uint32_t row2 = base_s + kOffA2 + tid * 128;
        for (int c16 = 0; c16 < N1 / 16; ++c16) {
          float v[16];
          tc::tmem_ld16(t_lane + c16 * 16, v);
          tc::tmem_wait_ld();
          if (mine) {
            uint32_t pk[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) pk[i] = tc::pack_bf16x2(tc::tanh_approx(v[2 * i]), tc::tanh_approx(v[2 * i + 1]));
            tc::sts128(row2 + (((2 * c16) ^ (tid & 7)) << 4), pk[0], pk[1], pk[2], pk[3]);
            tc::sts128(row2 + (((2 * c16 + 1) ^ (tid & 7)) << 4), pk[4], pk[5], pk[6], pk[7]);
          }
        }
        tc::fence_proxy_async();
        tc::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
          tc::tc_fence_after();
          const uint64_t ad = tc::sdesc_sw128(base_s + kOffA2), bd = tc::sdesc_sw128(w_s + bf16_w2_off(H));
          for (int k = 0; k < N1 / 16; ++k) tc::mma_bf16(tmem + kL2Col, ad + 2 * k, bd + 2 * k, idesc2, k > 0);
          tc::mma_commit(mbar);
        }
        ok = tc::mbar_wait(mbar, phase, kWaitCycles);
        phase ^= 1;
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        tc::tc_fence_after();
        float v[16];
        tc::tmem_ld16(t_lane + kL2Col, v);
        tc::tmem_wait_ld();
        if (mine) {
          const float* b2 = reinterpret_cast<const float*>(base + kOffW + bf16_b2_off(H));
#pragma unroll
          for (int o = 0; o < kOut; ++o) {
            zo[o] = v[o] + b2[o];
            act[o] = tc::tanh_approx(zo[o]);
          }
        }
      }
      tc::tc_fence_before();
      if (mine) done = true;
    }
    if (timed_out) break;
    // 5. actuator epilogue and pass-1 stores
    CellOut o;
    o.C[0] = o.C[1] = o.C[2] = o.C[3] = 0.0f;
    o.xdir = kNoExplore;
    if (valid) {
      const float* sI = stage + kHaloCells;
      const double S = (double)sI[hc - kHaloW] + (double)sI[hc + 1] + (double)sI[hc + kHaloW] + (double)sI[hc - 1];
      actuator_epilogue(a, act, zo, stage[hc], sI[hc], S, r, o);
      store_pass1(a, j, o);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float s = warp_sum(valid ? o.C[k] : 0.0f);
      if (lane == 0) accC[k] += (double)s;
    }
    const int ex = warp_sum_i(valid && o.xdir != kNoExplore ? 1 : 0);
    if (lane == 0) accX += ex;
    __syncthreads();   // stage / records / tiles are rewritten by the next tile
  }

  if (timed_out && tid == 0) atomicCAS(a.status, 0, (int)CORAL_E_TIMEOUT);
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
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10) return 0;                                  // tcgen05 needs sm_100 family
  if (cudaFuncSetAttribute(k_pass1_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass1_bf16, kThreads, kSmemBytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (per_sm > 4) per_sm = 4;                                 // 4 x 128 TMEM columns per SM
  if (per_sm < 1) return 0;
  const int g = per_sm * sms;
  return g > kMaxPartials ? kMaxPartials : g;
}

cudaError_t launch_pass1_bf16(const StepArgs& a, cudaStream_t st, int grid) {
  k_pass1_bf16<<<grid, kThreads, kSmemBytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace coral
