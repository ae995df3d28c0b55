// Genome table kernels: CPPN -> dense nets (HyperNEAT), FP32 / BF16 packing, radiation
// (mutation and merge of CPPN genomes with slot allocation), and the stable counting sort of
// cells by GenomeIndex.
#include <cuda_bf16.h>
#include <math.h>

#include "coral_internal.cuh"

namespace coral {

namespace {

// ---------------------------------------------------------------------------------------
// CPPN (Section "System Design": small CPPNs generate the weights and biases of the dense
// net). Five inputs (x1, y1, x2, y2, 1), hidden sin / gauss / tanh, linear output.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float cppn_eval(const float* g, float x1, float y1, float x2, float y2) {
  float z[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    z[k] = g[5 * k] * x1 + g[5 * k + 1] * y1 + g[5 * k + 2] * x2 + g[5 * k + 3] * y2 + g[5 * k + 4];
  return g[15] * sinf(z[0]) + g[16] * expf(-z[1] * z[1]) + g[17] * tanhf(z[2]);
}

__device__ __forceinline__ float layer_x(int i, int n) {
  return n == 1 ? 0.0f : -1.0f + 2.0f * (float)i / (float)(n - 1);
}

// One block per listed slot; writes the slot's FP32 record (internal layout).
__global__ void __launch_bounds__(256) k_cppn(GenomeArgs g, const int32_t* slots, const int* n_dev,
                                             int n_host) {
  const int n = n_dev ? *n_dev : n_host;
  const int H = g.hidden;
  __shared__ float gs[kGenes];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int slot = slots ? slots[i] : i;
    __syncthreads();
    if (threadIdx.x < kGenes) gs[threadIdx.x] = g.genes[(long long)slot * kGenes + threadIdx.x];
    __syncthreads();
    float* rec = g.nets32 + (long long)slot * g.net_stride;
    const float s1 = rsqrtf((float)kIn);
    if (H == 0) {
      for (int c = threadIdx.x; c < kOut * 56; c += blockDim.x) {
        const int o = c / 56, i2 = c % 56;
        rec[c] = i2 < kIn ? s1 * cppn_eval(gs, layer_x(i2, kIn), -1.0f, layer_x(o, kOut), 1.0f) : 0.0f;
      }
      for (int c = threadIdx.x; c < 12; c += blockDim.x)
        rec[net32_b1(0) + c] = c < kOut ? s1 * cppn_eval(gs, 0.0f, 0.0f, layer_x(c, kOut), 1.0f) : 0.0f;
      continue;
    }
    const float s2 = rsqrtf((float)H);
    for (int c = threadIdx.x; c < H * 56; c += blockDim.x) {
      const int h = c / 56, i2 = c % 56;
      rec[c] = i2 < kIn ? s1 * cppn_eval(gs, layer_x(i2, kIn), -1.0f, layer_x(h, H), 0.0f) : 0.0f;
    }
    for (int c = threadIdx.x; c < ((H + 3) & ~3); c += blockDim.x)
      rec[net32_b1(H) + c] = c < H ? s1 * cppn_eval(gs, 0.0f, 0.0f, layer_x(c, H), 0.0f) : 0.0f;
    for (int c = threadIdx.x; c < H * 12; c += blockDim.x) {
      const int h = c / 12, o = c % 12;
      rec[net32_w2t(H) + c] = o < kOut ? s2 * cppn_eval(gs, layer_x(h, H), 0.0f, layer_x(o, kOut), 1.0f) : 0.0f;
    }
    for (int c = threadIdx.x; c < 12; c += blockDim.x)
      rec[net32_b2(H) + c] = c < kOut ? s2 * cppn_eval(gs, 0.0f, 0.0f, layer_x(c, kOut), 1.0f) : 0.0f;
  }
}

// Direct nets in the public dense layout -> internal FP32 records (slots 0..n-1).
__global__ void __launch_bounds__(256) k_dense_pack(GenomeArgs g, const float* dense, int n) {
  const int H = g.hidden;
  const int nf = dense_floats(H);
  for (int slot = blockIdx.x; slot < n; slot += gridDim.x) {
    const float* src = dense + (long long)slot * nf;
    float* rec = g.nets32 + (long long)slot * g.net_stride;
    for (int c = threadIdx.x; c < g.net_stride; c += blockDim.x) rec[c] = 0.0f;
    __syncthreads();
    const int rows = H ? H : kOut;
    for (int c = threadIdx.x; c < rows * kIn; c += blockDim.x) rec[(c / kIn) * 56 + c % kIn] = src[c];
    const float* b1 = src + rows * kIn;
    for (int c = threadIdx.x; c < rows; c += blockDim.x) rec[net32_b1(H) + c] = b1[c];
    if (H) {
      const float* w2 = b1 + H;   // [10][H]
      for (int c = threadIdx.x; c < kOut * H; c += blockDim.x) {
        const int o = c / H, h = c % H;
        rec[net32_w2t(H) + h * 12 + o] = w2[c];
      }
      const float* b2 = w2 + kOut * H;
      for (int c = threadIdx.x; c < kOut; c += blockDim.x) rec[net32_b2(H) + c] = b2[c];
    }
    __syncthreads();
  }
}

// Internal FP32 record -> public dense layout (one slot).
__global__ void k_read_dense(GenomeArgs g, int slot, float* dst) {
  const int H = g.hidden;
  const float* rec = g.nets32 + (long long)slot * g.net_stride;
  const int rows = H ? H : kOut;
  for (int c = threadIdx.x; c < rows * kIn; c += blockDim.x) dst[c] = rec[(c / kIn) * 56 + c % kIn];
  float* b1 = dst + rows * kIn;
  for (int c = threadIdx.x; c < rows; c += blockDim.x) b1[c] = rec[net32_b1(H) + c];
  if (H) {
    float* w2 = b1 + H;
    for (int c = threadIdx.x; c < kOut * H; c += blockDim.x) w2[c] = rec[net32_w2t(H) + (c % H) * 12 + c / H];
    float* b2 = w2 + kOut * H;
    for (int c = threadIdx.x; c < kOut; c += blockDim.x) b2[c] = rec[net32_b2(H) + c];
  }
}

// Byte offset of element (row, k) in a 128-byte-row K-major tile whose 16-byte chunks are
// XOR-swizzled by (row & 7): the layout the tensor cores read with 128-byte swizzling.
__device__ __forceinline__ int swz(int row, int k) {
  return row * 128 + ((((k >> 3) ^ row) & 7) << 4) + ((k & 7) << 1);
}

// Internal FP32 record -> BF16 tensor-core blob (round to nearest even).
__global__ void __launch_bounds__(256) k_bf16_pack(GenomeArgs g, const int32_t* slots, const int* n_dev,
                                                  int n_host) {
  const int n = n_dev ? *n_dev : n_host;
  const int H = g.hidden;
  const int n1 = bf16_n1(H);
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int slot = slots ? slots[i] : i;
    const float* rec = g.nets32 + (long long)slot * g.net_stride;
    uint8_t* blob = g.nets16 + (long long)slot * g.blob_bytes;
    const int rows1 = H ? H : kOut;
    for (int c = threadIdx.x; c < n1 * 64; c += blockDim.x) {
      const int row = c >> 6, k = c & 63;
      float v = 0.0f;
      const int i = bf16_kslot_input(k);
      if (row < rows1 && i >= 0) v = i < kIn ? rec[row * 56 + i] : rec[net32_b1(H) + row];
      *reinterpret_cast<__nv_bfloat16*>(blob + swz(row, k)) = __float2bfloat16_rn(v);
    }
    if (H) {
      uint8_t* w2 = blob + bf16_w2_off(H);
      for (int c = threadIdx.x; c < 16 * 64; c += blockDim.x) {
        const int o = c >> 6, k = c & 63;
        const float v = (o < kOut && k < H) ? rec[net32_w2t(H) + k * 12 + o] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(w2 + swz(o, k)) = __float2bfloat16_rn(v);
      }
      float* b2 = reinterpret_cast<float*>(blob + bf16_b2_off(H));
      for (int c = threadIdx.x; c < 16; c += blockDim.x) b2[c] = c < kOut ? rec[net32_b2(H) + c] : 0.0f;
    }
  }
}

__global__ void k_validate(const int32_t* G, const uint8_t* R, int W, long long N, int P, int cap, int* status) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N;
       j += (long long)gridDim.x * blockDim.x) {
    if ((int)(j % P) >= W) continue;                  // row padding
    if ((G && (G[j] < 0 || G[j] >= cap)) || (R && R[j] > 3)) atomicCAS(status, 0, (int)CORAL_E_INVALID);
  }
}

// ---------------------------------------------------------------------------------------
// Radiation (Fig. 1 C: radiation of the substrate mutates CPPN genomes; Section "System
// Design": mutation and crossover operators of NEAT applied via the physics).
// ---------------------------------------------------------------------------------------
constexpr int kRadThreads = 256;
constexpr int kRadPerThread = 8;
constexpr int kRadTile = kRadThreads * kRadPerThread;

struct Hit {
  bool hit, mut, merge;
  int32_t g, gp;
  uint32_t bits;
};

// Global cell id (y * W + x over the world) of pitched cell j of the own rows.
__device__ __forceinline__ long long global_id(const RadiationArgs& r, long long j) {
  const long long l = j - r.j0;
  return r.gid0 + (l / r.P) * r.W + l % r.P;
}

__device__ __forceinline__ Hit radiation_hit(const RadiationArgs& r, long long j) {
  Hit h = {false, false, false, 0, -1, 0};
  if ((int)(j % r.P) >= r.W) return h;                // row padding
  const uint32_t cell = (uint32_t)global_id(r, j);
  const uint32_t cap = (uint32_t)r.g.capacity;
  if ((uint32_t)r.G[j] >= cap) return h;              // invalid GenomeIndex: never a parent
  if (r.thr_mut) h.mut = draw(cell, r.step, 0, 0, r.world, r.seed).x < r.thr_mut;
  if (r.thr_merge) {
    const uint4 w = draw(cell, r.step, 1, 0, r.world, r.seed);
    if (w.x < r.thr_merge) {
      const int x = (int)(j % r.P), y = (int)(j / r.P);
      int dx, dy;
      octant_offset(2 * (int)(w.y & 3u), dx, dy);     // von Neumann N, E, S, W
      const long long n = (long long)wrap(y + dy, r.H) * r.P + wrap(x + dx, r.W);
      const int32_t gp = r.G[n];
      if (gp != r.G[j] && (uint32_t)gp < cap) {
        h.merge = true;
        h.gp = gp;
        h.bits = w.z;
      }
    }
  }
  h.hit = h.mut || h.merge;
  if (h.hit) h.g = r.G[j];
  return h;
}

// Exclusive block scan of one int per thread (blockDim = kRadThreads).
__device__ __forceinline__ int block_exscan(int v, int& total) {
  __shared__ int warp_tot[kRadThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  int before = 0;
  total = 0;
  for (int i = 0; i < kRadThreads / 32; ++i) {
    if (i < w) before += warp_tot[i];
    total += warp_tot[i];
  }
  __syncthreads();
  return before + inc - v;
}

__global__ void __launch_bounds__(kRadThreads) k_rad_count(RadiationArgs r) {
  const long long base = r.j0 + (long long)blockIdx.x * kRadTile + (long long)threadIdx.x * kRadPerThread;
  int nh = 0, nm = 0, ng = 0;
  uint32_t mask = 0;
  for (int i = 0; i < kRadPerThread; ++i) {
    const long long j = base + i;
    if (j >= r.j0 + r.n_own) break;
    const Hit h = radiation_hit(r, j);
    nh += h.hit;
    nm += h.mut;
    ng += h.merge;
    mask |= (uint32_t)h.hit << i;
  }
  r.hitmask[(long long)blockIdx.x * kRadThreads + threadIdx.x] = (uint8_t)mask;
  int tot;
  block_exscan(nh, tot);
  int tm, tg;
  block_exscan(nm, tm);
  block_exscan(ng, tg);
  if (threadIdx.x == 0) {
    r.blockcnt[blockIdx.x] = tot;
    if (tm) atomicAdd(&r.counters[3], tm);
    if (tg) atomicAdd(&r.counters[4], tg);
  }
}

// Exclusive scan of n ints by one block (fixed order); total into *total.
__global__ void __launch_bounds__(1024) k_scan(const int32_t* in, int32_t* out, long long n, int* total) {
  __shared__ int part[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long b0 = 0; b0 < n; b0 += 1024LL * 16) {
    // each thread owns 16 consecutive entries of this chunk
    const long long s = b0 + (long long)threadIdx.x * 16;
    int loc = 0;
    for (int i = 0; i < 16; ++i)
      if (s + i < n) loc += in[s + i];
    part[threadIdx.x] = loc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += t;
      __syncthreads();
    }
    int run = carry + part[threadIdx.x] - loc;
    for (int i = 0; i < 16; ++i)
      if (s + i < n) {
        const int v = in[s + i];
        out[s + i] = run;
        run += v;
      }
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// Writes the hits in cell order. The counting pass left each thread's hit bits in the mask, so
// only hit cells (about p_mut + p_merge of them) draw their Philox numbers again here.
__global__ void __launch_bounds__(kRadThreads) k_rad_emit(RadiationArgs r) {
  const long long base = r.j0 + (long long)blockIdx.x * kRadTile + (long long)threadIdx.x * kRadPerThread;
  uint32_t mask = r.hitmask[(long long)blockIdx.x * kRadThreads + threadIdx.x];
  int tot;
  int pos = r.blockoff[blockIdx.x] + block_exscan(__popc(mask), tot);
  while (mask) {
    const int i = __ffs(mask) - 1;
    mask &= mask - 1;
    const Hit h = radiation_hit(r, base + i);
    if (pos < r.max_hits) {
      r.hits[pos] = make_int4((int)global_id(r, base + i), h.g, h.merge ? h.gp : -1, (h.mut ? 1 : 0) | (h.merge ? 2 : 0));
      r.hitbits[pos] = h.bits;
    }
    ++pos;
  }
}

// Marks the slots that own at least one cell (flag[g] = 1). Each block collects the slots of
// its contiguous range of cells in a shared bitmap (one shared-memory OR per distinct slot of a
// warp's 32 cells), then writes one global flag per slot it saw: genomes occupy blobs, so a few
// stores per block instead of one per cell on a handful of hot lines.
constexpr int kLiveThreads = 256;
constexpr int kLiveMaxWords = 2048;                 // bitmap of up to 65,536 slots
__global__ void __launch_bounds__(kLiveThreads) k_live(const int32_t* G, long long N, int cap, int32_t* flag) {
  __shared__ uint32_t bits[kLiveMaxWords];
  const int words = (cap + 31) >> 5;
  for (int i = threadIdx.x; i < words; i += kLiveThreads) bits[i] = 0;
  __syncthreads();
  const long long per = (N + gridDim.x - 1) / gridDim.x;
  const long long j0 = (long long)blockIdx.x * per;
  const long long j1 = j0 + per < N ? j0 + per : N;
  for (long long b = j0; b < j1; b += kLiveThreads) {
    const long long j = b + threadIdx.x;
    const int g = j < j1 ? G[j] : -1;
    const unsigned m = __match_any_sync(0xffffffffu, g);
    if (g >= 0 && g < cap && (threadIdx.x & 31) == __ffs(m) - 1) atomicOr(&bits[g >> 5], 1u << (g & 31));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < words; i += kLiveThreads) {
    uint32_t w = bits[i];
    while (w) {
      const int k = __ffs(w) - 1;
      w &= w - 1;
      flag[32 * i + k] = 1;
    }
  }
}

// Slots without cells fall back to one store per cell when the bitmap would not fit.
__global__ void k_live_plain(const int32_t* G, long long N, int cap, int32_t* flag) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
    const int g = G[j];
    if (g >= 0 && g < cap) flag[g] = 1;
  }
}

// Free slots (flag 0) in increasing order and the live count, in two passes over blocks of
// 1024 consecutive slots: per-block counts, then each block's free slots compacted in order at
// the offset of the blocks before it.
constexpr int kFreeBlock = 1024;
__global__ void __launch_bounds__(kFreeBlock) k_free_count(RadiationArgs r) {
  __shared__ int wf[32], wl[32];
  const int sl = blockIdx.x * kFreeBlock + threadIdx.x;
  const int c = sl < r.g.capacity ? r.count[sl] : -1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = __popc(__ballot_sync(0xffffffffu, c == 0)), l = __popc(__ballot_sync(0xffffffffu, c > 0));
  if (lane == 0) {
    wf[w] = f;
    wl[w] = l;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tf = 0, tl = 0;
    for (int i = 0; i < 32; ++i) {
      tf += wf[i];
      tl += wl[i];
    }
    r.blockcnt[blockIdx.x] = tf;
    r.blockoff[blockIdx.x] = tl;           // live slots of this block
  }
}

__global__ void __launch_bounds__(kFreeBlock) k_free_emit(RadiationArgs r) {
  __shared__ int wf[32];
  __shared__ int base;
  const int sl = blockIdx.x * kFreeBlock + threadIdx.x;
  const int c = sl < r.g.capacity ? r.count[sl] : -1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, c == 0);
  if (lane == 0) wf[w] = __popc(b);
  if (threadIdx.x == 0) {
    int off = 0;
    for (int i = 0; i < (int)blockIdx.x; ++i) off += r.blockcnt[i];
    base = off;
    if (blockIdx.x == 0) {                 // totals: free slots and live slots
      int tf = 0, tl = 0;
      for (int i = 0; i < (int)gridDim.x; ++i) {
        tf += r.blockcnt[i];
        tl += r.blockoff[i];
      }
      r.counters[1] = tf;
      r.counters[5] = tl;
    }
  }
  __syncthreads();
  int before = base;
  for (int i = 0; i < w; ++i) before += wf[i];
  if (c == 0) r.freelist[before + __popc(b & ((1u << lane) - 1))] = sl;
}

__global__ void __launch_bounds__(128) k_rad_assign(RadiationArgs r) {
  const int nh = r.counters[0];
  const int nf = r.counters[1];
  int na = nh < nf ? nh : nf;
  if (na > r.max_hits) na = r.max_hits;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na; i += gridDim.x * blockDim.x) {
    const int4 h = r.hits[i];
    const int slot = r.freelist[i];
    float c[kGenes];
    const float* gp = r.g.genes + (long long)h.y * kGenes;
#pragma unroll
    for (int k = 0; k < kGenes; ++k) c[k] = gp[k];
    if (h.w & 2) {
      const uint32_t bits = r.hitbits[i];
      const float* gq = r.g.genes + (long long)h.z * kGenes;
#pragma unroll
      for (int k = 0; k < kGenes; ++k)
        if ((bits >> k) & 1u) c[k] = gq[k];
    }
    if (h.w & 1) {
      uint32_t u[20];
#pragma unroll
      for (int sub = 0; sub < 5; ++sub) {
        const uint4 w = draw((uint32_t)h.x, r.step, 2, sub, r.world, r.seed);
        u[4 * sub] = w.x; u[4 * sub + 1] = w.y; u[4 * sub + 2] = w.z; u[4 * sub + 3] = w.w;
      }
#pragma unroll
      for (int k = 0; k < kGenes / 2; ++k) {
        // Box-Muller (Box & Muller, 1958) on two open-interval uniforms
        const float rr = sqrtf(-2.0f * logf(uniform01f(u[2 * k])));
        float sn, cs;
        sincospif(2.0f * uniform01f(u[2 * k + 1]), &sn, &cs);
        c[2 * k] += r.sigma * (rr * cs);
        c[2 * k + 1] += r.sigma * (rr * sn);
      }
    }
    float* dst = r.g.genes + (long long)slot * kGenes;
#pragma unroll
    for (int k = 0; k < kGenes; ++k) dst[k] = c[k];
    r.g.parent[slot] = h.y;
    const long long l = (long long)h.x - r.gid0;             // the hit cell in this grid, if own
    if (l >= 0 && l < r.n_own / r.P * r.W) r.G[r.j0 + (l / r.W) * r.P + l % r.W] = slot;
    r.newslots[i] = slot;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    r.counters[2] = na;
    coral_stats* s = r.rec;
    s->n_mut = r.counters[3];
    s->n_merge = r.counters[4];
    s->n_born = na;
    s->n_skipped = nh - na;
    s->n_live = r.counters[5] + na;
  }
}

// ---------------------------------------------------------------------------------------
// Bucketing: stable counting sort of cell ids by GenomeIndex, as least-significant-digit
// passes of stable 256-bucket counting sorts.
// ---------------------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortTile = 4096;
constexpr int kSortItems = kSortTile / kSortThreads;    // keys per thread
static_assert(kSortThreads == 256, "one thread per digit value in the scatter's offsets");
// Element layout of a block's tile in the histogram, scatter and run kernels: warp w owns the
// contiguous range [w * 512, w * 512 + 512) of the tile; in item c, lane l holds element
// w * 512 + 32 c + l. Every thread loads its 16 keys before it uses any of them, so a warp
// has 16 coalesced 128-byte loads in flight instead of one.
__device__ __forceinline__ long long sort_elem0(int lane, int w) {
  return (long long)blockIdx.x * kSortTile + w * (kSortItems * 32) + lane;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const int32_t* __restrict__ keys, long long N,
                                                          int shift, int32_t* hist, int nblk) {
  __shared__ int h[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long e0 = sort_elem0(lane, w);
  int d[kSortItems];
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    const long long j = e0 + 32 * c;
    d[c] = j < N ? (__ldg(keys + j) >> shift) & 255 : 256;
  }
  h[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    // one shared-memory add per distinct digit of the warp (genomes come in runs)
    const unsigned m = __match_any_sync(0xffffffffu, d[c]);
    if (d[c] < 256 && lane == __ffs(m) - 1) atomicAdd(&h[d[c]], __popc(m));
  }
  __syncthreads();
  hist[(long long)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Keys per digit value: block d sums row d of the [256][nblk] block histograms.
__global__ void __launch_bounds__(256) k_digit_totals(const int32_t* hist, int nblk, int32_t* totals) {
  __shared__ int ws[8];
  int v = 0;
  for (int b = threadIdx.x; b < nblk; b += 256) v += hist[(long long)blockIdx.x * nblk + b];
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < 8; ++i) t += ws[i];
    totals[blockIdx.x] = t;
  }
}

// Exclusive scan of the histograms in digit-major order, one block per digit value: row d
// starts at the keys of smaller digits and runs over the blocks in order (in place). Each
// thread takes 4 consecutive entries, so a row of up to 4096 blocks is one pass.
__global__ void __launch_bounds__(1024) k_digit_scan(int32_t* hist, int nblk, const int32_t* totals) {
  __shared__ int wsum[32];
  __shared__ int base_s;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w == 0) {
    int v = 0;
    for (int d = lane; d < (int)blockIdx.x; d += 32) v += totals[d];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) base_s = v;
  }
  __syncthreads();
  int carry = base_s;
  int32_t* row = hist + (long long)blockIdx.x * nblk;
  for (int c0 = 0; c0 < nblk; c0 += 4 * 1024) {
    const int b0 = c0 + 4 * threadIdx.x;
    int v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = b0 + i < nblk ? row[b0 + i] : 0;
    const int sum = v[0] + v[1] + v[2] + v[3];
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int before = carry, tot = 0;
    for (int i = 0; i < 32; ++i) {
      const int s = wsum[i];
      if (i < w) before += s;
      tot += s;
    }
    int run = before + inc - sum;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (b0 + i < nblk) row[b0 + i] = run;
      run += v[i];
    }
    carry += tot;
    __syncthreads();                                  // wsum is rewritten by the next chunk
  }
}

// Keys per slot from the sorted keys: each block takes a contiguous chunk; a run of equal keys
// inside it adds (last - c0 + 1) at its last element and -(first - c0) at its first, so each
// slot receives the total length of its runs with two atomics per run and chunk.
__global__ void __launch_bounds__(kSortThreads) k_count_runs(const int32_t* __restrict__ sk, long long N, int cap,
                                                           int32_t* count) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long c0 = (long long)blockIdx.x * kSortTile;
  const long long c1 = c0 + kSortTile < N ? c0 + kSortTile : N;
  const long long e0 = sort_elem0(lane, w);
  int k[kSortItems];
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    const long long j = e0 + 32 * c;
    k[c] = j < c1 ? __ldg(sk + j) : -1;
  }
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    const long long j = e0 + 32 * c;
    // neighbours in the sorted order: the adjacent lanes, or memory at the warp's edges
    int prev = __shfl_up_sync(0xffffffffu, k[c], 1);
    int next = __shfl_down_sync(0xffffffffu, k[c], 1);
    if (lane == 0 && j > c0 && j < c1) prev = __ldg(sk + j - 1);
    if (lane == 31 && j + 1 < c1) next = __ldg(sk + j + 1);
    const int key = k[c];
    if (j >= c1 || key < 0 || key >= cap) continue;
    const bool head = j == c0 || prev != key;
    const bool tail = j == c1 - 1 || next != key;
    if (head && tail) atomicAdd(&count[key], 1);
    else if (head) atomicAdd(&count[key], -(int)(j - c0));
    else if (tail) atomicAdd(&count[key], (int)(j - c0 + 1));
  }
}

// One stable 256-bucket pass. Each warp ranks its own contiguous 512 keys (a running count
// per digit value in its row of shared memory), then thread t turns digit t's per-warp counts
// into start positions after the block's offset for that digit: two CTA barriers per block.
// kVal: values come from vin (later passes); else the value is the key's index (first pass).
// Three blocks per SM (80 registers: ranks packed two per register).
template <bool kVal>
__global__ void __launch_bounds__(kSortThreads, 3) k_sort_scatter(const int32_t* __restrict__ kin,
                                                                const int32_t* __restrict__ vin, int32_t* kout,
                                                                int32_t* vout, long long N, int shift,
                                                                const int32_t* off, int nblk) {
  __shared__ int wc[kSortThreads / 32][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long e0 = sort_elem0(lane, w);
  int key[kSortItems], val[kSortItems];
  uint32_t rank[kSortItems / 2];                      // ranks (< 512) of items 2i, 2i+1 in 16-bit halves
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    const long long j = e0 + 32 * c;
    const bool ok = j < N;
    key[c] = ok ? __ldg(kin + j) : 0;
    if (kVal) val[c] = ok ? __ldg(vin + j) : 0;
  }
  for (int i = lane; i < 256; i += 32) wc[w][i] = 0;
  __syncwarp();
  const unsigned lower = (1u << lane) - 1u;
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    const int d = e0 + 32 * c < N ? (key[c] >> shift) & 255 : 256;
    const unsigned m = __match_any_sync(0xffffffffu, d);
    const int before = d < 256 ? wc[w][d] : 0;
    const uint32_t rk = (uint32_t)(before + __popc(m & lower));
    if (c & 1) rank[c >> 1] |= rk << 16;
    else rank[c >> 1] = rk;
    __syncwarp();
    if (d < 256 && lane == __ffs(m) - 1) wc[w][d] = before + __popc(m);
    __syncwarp();
  }
  __syncthreads();
  {
    int acc = off[(long long)threadIdx.x * nblk + blockIdx.x];
#pragma unroll
    for (int i = 0; i < kSortThreads / 32; ++i) {
      const int t = wc[i][threadIdx.x];
      wc[i][threadIdx.x] = acc;
      acc += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kSortItems; ++c) {
    if (e0 + 32 * c < N) {
      const int pos = wc[w][(key[c] >> shift) & 255] + (int)((rank[c >> 1] >> (16 * (c & 1))) & 0xFFFFu);
      kout[pos] = key[c];
      vout[pos] = kVal ? val[c] : (int)(e0 + 32 * c);
    }
  }
}

// NEAT compatibility distance of fixed-topology genomes: 0.4 * mean |g_a - g_b| (18 genes).
__global__ void k_genome_distances(const float* genes, const int32_t* slots, int n, float* out) {
  const long long pair = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pair >= (long long)n * n) return;
  const int i = (int)(pair / n), k = (int)(pair - (long long)i * n);
  const float* a = genes + (long long)slots[i] * kGenes;
  const float* b = genes + (long long)slots[k] * kGenes;
  float acc = 0.0f;
#pragma unroll
  for (int g = 0; g < kGenes; ++g) acc += fabsf(a[g] - b[g]);
  out[pair] = 0.4f * (acc / (float)kGenes);
}

// Philox4x32-10 on the device for listed counters and keys: the same function the radiation
// kernels draw from (known-answer test hook).
__global__ void __launch_bounds__(256) k_philox(const uint4* ctr, const uint2* key, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], key[i].x, key[i].y);
}

}  // namespace

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, cudaStream_t st) {
  k_philox<<<(n + 255) / 256, 256, 0, st>>>(reinterpret_cast<const uint4*>(ctr), reinterpret_cast<const uint2*>(key),
                                            reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}

cudaError_t launch_genome_distances(const float* genes, const int32_t* slots, int n, float* out, cudaStream_t st) {
  const long long pairs = (long long)n * n;
  k_genome_distances<<<(int)((pairs + 255) / 256), 256, 0, st>>>(genes, slots, n, out);
  return cudaGetLastError();
}

int radiation_blocks(long long N) { return (int)((N + kRadTile - 1) / kRadTile); }
int radiation_threads() { return kRadThreads; }
int bucket_blocks(long long N) { return (int)((N + kSortTile - 1) / kSortTile); }

cudaError_t launch_cppn_generate(const GenomeArgs& g, const int32_t* slots, const int* n_dev, int n_host,
                                 cudaStream_t st) {
  const int grid = n_dev ? 512 : (n_host < 1 ? 1 : (n_host > 4096 ? 4096 : n_host));
  k_cppn<<<grid, 256, 0, st>>>(g, slots, n_dev, n_host);
  return cudaGetLastError();
}

cudaError_t launch_dense_pack(const GenomeArgs& g, const float* dense, int n, cudaStream_t st) {
  k_dense_pack<<<n < 4096 ? n : 4096, 256, 0, st>>>(g, dense, n);
  return cudaGetLastError();
}

cudaError_t launch_bf16_pack(const GenomeArgs& g, const int32_t* slots, const int* n_dev, int n_host,
                             cudaStream_t st) {
  const int grid = n_dev ? 512 : (n_host < 1 ? 1 : (n_host > 4096 ? 4096 : n_host));
  k_bf16_pack<<<grid, 256, 0, st>>>(g, slots, n_dev, n_host);
  return cudaGetLastError();
}

cudaError_t launch_read_dense(const GenomeArgs& g, int slot, float* dst, cudaStream_t st) {
  k_read_dense<<<1, 256, 0, st>>>(g, slot, dst);
  return cudaGetLastError();
}

cudaError_t launch_validate_state(const int32_t* G, const uint8_t* R, int W, int H, int P, int cap, int* status,
                                  cudaStream_t st) {
  k_validate<<<1024, 256, 0, st>>>(G, R, W, (long long)H * P, P, cap, status);
  return cudaGetLastError();
}

cudaError_t launch_radiation_scan(const RadiationArgs& r, cudaStream_t st) {
  const int nblk = radiation_blocks(r.n_own);
  cudaError_t e;
  if ((e = cudaMemsetAsync(r.count, 0, sizeof(int32_t) * r.g.capacity, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(r.counters, 0, sizeof(int) * 8, st)) != cudaSuccess) return e;
  if (r.g.capacity <= 32 * kLiveMaxWords)
    k_live<<<1024, kLiveThreads, 0, st>>>(r.G + r.j0, r.n_own, r.g.capacity, r.count);
  else
    k_live_plain<<<1024, 256, 0, st>>>(r.G + r.j0, r.n_own, r.g.capacity, r.count);
  k_rad_count<<<nblk, kRadThreads, 0, st>>>(r);
  k_scan<<<1, 1024, 0, st>>>(r.blockcnt, r.blockoff, nblk, &r.counters[0]);
  k_rad_emit<<<nblk, kRadThreads, 0, st>>>(r);
  return cudaGetLastError();
}

cudaError_t launch_radiation_apply(const RadiationArgs& r, cudaStream_t st) {
  cudaError_t e;
  {
    // blockcnt / blockoff are free again once the hits are emitted; the slot passes reuse them
    RadiationArgs f = r;
    const int fblk = (r.g.capacity + kFreeBlock - 1) / kFreeBlock;
    k_free_count<<<fblk, kFreeBlock, 0, st>>>(f);
    k_free_emit<<<fblk, kFreeBlock, 0, st>>>(f);
  }
  k_rad_assign<<<64, 128, 0, st>>>(r);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_cppn_generate(r.g, r.newslots, &r.counters[2], 0, st)) != cudaSuccess) return e;
  return launch_bf16_pack(r.g, r.newslots, &r.counters[2], 0, st);
}

cudaError_t launch_radiation(const RadiationArgs& r, cudaStream_t st) {
  cudaError_t e = launch_radiation_scan(r, st);
  return e != cudaSuccess ? e : launch_radiation_apply(r, st);
}

namespace {
// FP64 totals of a cell range: each block sums a contiguous chunk (doubles, a fixed tree), one
// partial per block and plane; block 0 of a second launch adds the partials in block order.
constexpr int kTotBlocks = 256;
__global__ void __launch_bounds__(256) k_row_totals(const float* E, long long N, long long j0, long long n,
                                                    double* part) {
  __shared__ double red[256];
  const long long per = (n + kTotBlocks - 1) / kTotBlocks;
  const long long c0 = j0 + (long long)blockIdx.x * per;
  const long long c1 = c0 + per < j0 + n ? c0 + per : j0 + n;
  for (int p = 0; p < 6; ++p) {
    double s = 0.0;
    for (long long j = c0 + threadIdx.x; j < c1; j += 256) s += (double)E[(long long)p * N + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[p * kTotBlocks + blockIdx.x] = red[0];
    __syncthreads();
  }
}
__global__ void k_row_totals_final(const double* part, double* out) {
  const int p = threadIdx.x;
  if (p < 6) {
    double s = 0.0;
    for (int b = 0; b < kTotBlocks; ++b) s += part[p * kTotBlocks + b];
    out[p] = s;
  }
}
}  // namespace

cudaError_t launch_row_totals(const float* E, long long N, long long j0, long long n, double* out, cudaStream_t st) {
  // out must have room for 6 + 6 * kTotBlocks doubles: the partials follow the six totals
  k_row_totals<<<kTotBlocks, 256, 0, st>>>(E, N, j0, n, out + 6);
  k_row_totals_final<<<1, 32, 0, st>>>(out + 6, out);
  return cudaGetLastError();
}

cudaError_t launch_bucket(const SortArgs& a, cudaStream_t st) {
  const int nblk = bucket_blocks(a.N);
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.count, 0, sizeof(int32_t) * a.capacity, st)) != cudaSuccess) return e;
  int passes = 1;
  while (passes < 4 && (1LL << (8 * passes)) < (long long)a.capacity) ++passes;
  const int32_t* kin = a.keys_in;
  const int32_t* vin = nullptr;
  for (int p = 0; p < passes; ++p) {
    int32_t* kout = (p & 1) ? a.k1 : a.k0;
    int32_t* vout = (p + 1 == passes) ? a.perm : ((p & 1) ? a.v1 : a.v0);
    k_sort_hist<<<nblk, kSortThreads, 0, st>>>(kin, a.N, 8 * p, a.hist, nblk);
    k_digit_totals<<<256, 256, 0, st>>>(a.hist, nblk, a.totals);
    k_digit_scan<<<256, 1024, 0, st>>>(a.hist, nblk, a.totals);
    if (vin)
      k_sort_scatter<true><<<nblk, kSortThreads, 0, st>>>(kin, vin, kout, vout, a.N, 8 * p, a.hist, nblk);
    else
      k_sort_scatter<false><<<nblk, kSortThreads, 0, st>>>(kin, vin, kout, vout, a.N, 8 * p, a.hist, nblk);
    kin = kout;
    vin = vout;
  }
  k_count_runs<<<nblk, kSortThreads, 0, st>>>(kin, a.N, a.capacity, a.count);   // kin: sorted keys
  return cudaGetLastError();
}

}  // namespace coral
