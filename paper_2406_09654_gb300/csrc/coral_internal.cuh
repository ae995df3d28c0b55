// Internal declarations of the GB300 substrate-step library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/coral.h"

namespace coral {

constexpr int kIn = 54;        // 9 kernel offsets x 6 sensor channels
constexpr int kOut = 10;       // com0..3, invest, liquidate, explore0..3
constexpr int kGenes = 18;     // CPPN genes
constexpr int kRing = 4096;    // stats ring length (steps)
constexpr int kMaxPartials = 8192;
constexpr uint8_t kNoExplore = 4;

// ---- FP32 net layout in device memory (one record per genome slot) ------------------------
// hidden = 0: W[10][56] (columns 54,55 zero), b[12]
// hidden = H: W1[H][56], b1[H rounded to 4], W2T[H][12] (hidden-major, 10 used), b2[12]
__host__ __device__ inline int dense_floats(int H) {   // public dense layout length
  return H ? H * kIn + H + kOut * H + kOut : kOut * kIn + kOut;
}
__host__ __device__ inline int net32_b1(int H) { return (H ? H : kOut) * 56; }
__host__ __device__ inline int net32_w2t(int H) { return net32_b1(H) + ((H + 3) & ~3); }
__host__ __device__ inline int net32_b2(int H) { return net32_w2t(H) + H * 12; }
__host__ __device__ inline int net32_stride(int H) {
  int n = H ? net32_b2(H) + 12 : net32_b1(0) + 12;
  return (n + 15) & ~15;
}

// ---- BF16 tensor-core net blob (one per slot; byte image of the shared-memory operands) --
// [0, n1*128)         W1 (or W for hidden = 0): n1 rows of 64 bf16 (K-major, 128-byte rows,
//                     16-byte chunks XOR-swizzled by row & 7). K slot k = 8p + c holds input
//                     (rank p, channel c) for p < 8, c < 6; the spare slots 8p + 6, 8p + 7 of
//                     p = 0, 1, 2 hold rank 8's channels 2p, 2p + 1; slot 30 holds the layer-1
//                     bias (the A operand carries 1.0 there); every other slot is zero. Each
//                     16-byte chunk of an input row is then one cell record (6 channels of
//                     one neighbour) plus one word of rank 8 / bias.
// [n1*128, +2048)     W2: 16 rows x 64 bf16 (10 used), same swizzle; absent for hidden = 0.
// then                b2 (or nothing for hidden = 0): 16 float32.
__host__ __device__ inline int bf16_n1(int H) { return H ? H : 16; }
// Input index (6 * rank + channel) held by K slot k of the tensor-core input row, 54 for the
// bias slot, -1 for a zero slot.
__host__ __device__ inline int bf16_kslot_input(int k) {
  const int p = k >> 3, c = k & 7;
  if (c < 6) return 6 * p + c;
  if (p < 3) return 48 + 2 * p + (c - 6);
  return k == 30 ? kIn : -1;
}
__host__ __device__ inline int bf16_w2_off(int H) { return bf16_n1(H) * 128; }
__host__ __device__ inline int bf16_b2_off(int H) { return H ? bf16_w2_off(H) + 16 * 128 : bf16_w2_off(H); }
__host__ __device__ inline int bf16_blob_bytes(int H) {
  int n = H ? bf16_b2_off(H) + 64 : bf16_w2_off(H);
  return (n + 127) & ~127;
}

// Packed state of one cell in host transfers: E, I, C0..C3 float32, G int32, R uint8.
constexpr int kStateBytesPerCell = 6 * 4 + 4 + 1;

struct Planes {     // the six sensor planes are contiguous: I = E + N, C = E + 2N
  float* E;
  float* I;
  float* C;        // 4 planes of N floats
  int32_t* G;
  uint8_t* R;
};

// Pass-1 record of one cell, 16 bytes (one vector store / load):
//   x = keep: E1 minus what the cell sends along infrastructure
//   y = I1:   infrastructure after invest / liquidate
//   z = q:    k_flow * E1 / S (FP64 denominator), what each neighbour gets per unit of I_t
//   w = xamt: exploration amount (0 when not exploring)
struct Pass1Bufs {
  float4* rec;     // [N]
  uint8_t* xdir;   // exploration direction 0..3 (N,E,S,W) or kNoExplore
};

struct Partial {   // per-block partial sums of one step (FP64), fixed-order combined
  double s[6];     // E, I, C0..C3
  long long c[2];  // explore, takeover
};

// Planes are pitched: row y starts at cell y * P, P = W rounded up to a multiple of 4 (rows of
// 16-byte aligned floats for TMA and vector loads); the P - W padding cells of a row are never
// part of the torus (G = -1, R = 0, floats 0). N = H * P is the plane length.
__host__ __device__ inline int row_pitch(int W) { return (W + 3) & ~3; }

constexpr int kFmaCutoffMax = 128;   // the FMA small-genome cutoff: at most a whole tile

struct __align__(8) StepArgs {
  int W, H;
  long long N;                  // H * P
  int P;                        // row pitch in cells
  int hidden;
  int rotation;
  float k_inv, k_liq, k_exp, k_flow;
  int is_day;
  float e_day, e_night;
  Planes cur, nxt;
  Pass1Bufs p1;
  const float* nets32;
  int net_stride;
  const uint8_t* nets16;
  int blob_bytes;
  Partial* part1;   // written by pass 1 (C sums, explore count)
  Partial* part2;   // written by pass 2 (E, I sums, takeover count)
  int* status;
  int day_period;
  int capacity;     // genome slots: a GenomeIndex outside [0, capacity) acts as "no genome"
  const long long* step_dev;   // batched stepping: this world's step index on the device (day/night
                               // is taken from it); NULL: use is_day
  int* sched;                  // BF16 pass 1's tile pool: [0] next chunk, [1] CTAs done (both 0
                               // between launches: the last CTA of a launch resets them)
  int fma_cutoff;              // BF16 pass 1: a later genome round of a tile with at most this many
                               // cells runs on the warp-level FMA path (0: never)
};

// Batched stepping of many worlds (same hidden size, BF16 path): the CTAs of each launch are
// split among the worlds (contiguous CTA ranges), every CTA works on one world only.
struct BatchTable {
  int n;                          // worlds
  const StepArgs* args;           // [2][n]: parity p = batch step count & 1
  const int* cta_world1;          // pass 1: world of each CTA
  const int* world_first1;        //   first CTA of each world
  const int* world_ctas1;         //   CTAs of each world
  const int* cta_world2;          // pass 2: same
  const int* world_first2;
  const int* world_ctas2;
  coral_stats* const* rings;      // [n] stats rings
  long long* steps;               // [n] step index of each world (advanced by the stats kernel)
  const CUtensorMap* tmaps;       // [2][n] TMA descriptors of the worlds' sensor planes (parity p:
                                  // the buffer args[p][w] reads), written by the host before use
  const int* tma_ok;              // [n] the world has descriptors (rows a multiple of 16 bytes)
};

// ---- Philox4x32-10 (Salmon et al., SC'11), written for the device -----------------------
__host__ __device__ inline uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ inline uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = mulhi32(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = mulhi32(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Counter (cell, step, stream << 24 | sub, world), key = seed.
__device__ inline uint4 draw(uint32_t cell, uint32_t step, uint32_t stream, uint32_t sub,
                             uint32_t world, unsigned long long seed) {
  return philox4x32_10(make_uint4(cell, step, (stream << 24) | (sub & 0xFFFFFFu), world),
                       (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ inline float uniform01f(uint32_t u) {  // ((u >> 8) + 0.5) * 2^-24, exact
  return ((float)(u >> 8) + 0.5f) * 5.9604644775390625e-8f;
}

// ---- torus helpers -----------------------------------------------------------------------
__device__ inline int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Kernel rank p (1..8) -> octant offset from forward: 0, +1, -1, +2, -2, +3, -3, +4.
__host__ __device__ constexpr int rank_delta(int p) {
  return p == 1 ? 0 : p == 2 ? 1 : p == 3 ? -1 : p == 4 ? 2 : p == 5 ? -2 : p == 6 ? 3 : p == 7 ? -3 : 4;
}

// Octant o (0..7 clockwise from north: N, NE, E, SE, S, SW, W, NW) -> (dx, dy), north being
// the row above; the offsets are packed two bits per octant as (d + 1).
__host__ __device__ inline void octant_offset(int o, int& dx, int& dy) {
  dx = (int)((0x1A9u >> (2 * o)) & 3u) - 1;
  dy = (int)((0x1A90u >> (2 * o)) & 3u) - 1;
}

// Explore logit k -> quarter turns clockwise from the forward direction (fwd, right, left, back):
// 0, 1, 3, 2, which is the Gray code of k (two integer operations, no table).
__host__ __device__ constexpr int explore_turn(int k) { return k ^ (k >> 1); }

// ---- reductions: FP32 within a warp (32 cells), FP64 above ------------------------------
__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- launchers (defined in the .cu files) -----------------------------------------------
cudaError_t launch_pass1_fp32(const StepArgs& a, cudaStream_t st, int grid);
// tmap: TMA descriptor of the current state's six sensor planes as a W x H x 6 float tensor
// (box 40 x 6 x 6), or NULL when the grid does not allow it (then cp.async copies the halos).
cudaError_t launch_pass1_bf16(const StepArgs& a, const CUtensorMap* tmap, cudaStream_t st, int grid);
// Encodes that descriptor for planes starting at E (returns false when TMA cannot be used).
bool encode_sensor_tmap(CUtensorMap* map, const float* E, int W, int H, int P);
cudaError_t launch_pass2(const StepArgs& a, cudaStream_t st, int grid);
cudaError_t launch_stats(const StepArgs& a, int n_part1, int n_part2, long long t,
                         coral_stats* ring, cudaStream_t st);
// Copies one world's step arguments to shared memory (called by every thread of the block,
// followed by a barrier), so the kernel body reads them with shared loads.
__device__ __forceinline__ void copy_args_to_shared(StepArgs* dst, const StepArgs* src) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(StepArgs) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

cudaError_t prepare_pass1_bf16_batch();   // kernel attributes, once before any capture
cudaError_t launch_pass1_bf16_batch(const BatchTable& b, int parity, int grid, int hidden, bool fma,
                                    cudaStream_t st);
cudaError_t launch_pass2_batch(const BatchTable& b, int parity, int grid, cudaStream_t st);
cudaError_t launch_stats_batch(const BatchTable& b, cudaStream_t st);
int pass1_fp32_grid(int sms);
cudaError_t launch_selftest_wait(long long max_cycles, int* status, cudaStream_t st);
// blocks x 256 threads, each 8 x iters tanh.approx.f32 evaluations; sink: [blocks] floats
cudaError_t launch_sfu_probe(int blocks, int iters, float* sink, cudaStream_t st);
int pass1_bf16_grid(int sms);
int pass2_grid(int sms);
size_t pass1_bf16_smem();
long long pass1_bf16_tiles(int W, int H);   // tensor-core pass-1 tiles of a W x H world

struct GenomeArgs {
  int hidden;
  int capacity;
  float* genes;       // [cap][18]
  int32_t* parent;    // [cap]
  float* nets32;      // [cap][net_stride]
  int net_stride;
  uint8_t* nets16;    // [cap][blob_bytes]
  int blob_bytes;
};
cudaError_t launch_cppn_generate(const GenomeArgs& g, const int32_t* slots, const int* n_dev,
                                 int n_host, cudaStream_t st);
cudaError_t launch_dense_pack(const GenomeArgs& g, const float* dense, int n, cudaStream_t st);
cudaError_t launch_bf16_pack(const GenomeArgs& g, const int32_t* slots, const int* n_dev,
                             int n_host, cudaStream_t st);
cudaError_t launch_read_dense(const GenomeArgs& g, int slot, float* dst, cudaStream_t st);
// ctr [n][4], key [n][2], out [n][4] device arrays (16- and 8-byte aligned)
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n, cudaStream_t st);
cudaError_t launch_genome_distances(const float* genes, const int32_t* slots, int n, float* out, cudaStream_t st);
// G and R of the W x H torus in planes of pitch P (padding cells not checked)
cudaError_t launch_validate_state(const int32_t* G, const uint8_t* R, int W, int H, int P, int cap,
                                  int* status, cudaStream_t st);

struct RadiationArgs {
  int W, H;
  long long N;                // H * P
  int P;                      // row pitch in cells
  int32_t* G;                 // current state's G (rewritten in place for the children)
  // the cells radiation acts on: the whole rows [j0, j0 + n_own) of G (pitched indices, j0 a
  // multiple of P; padding cells skipped), whose global cell ids (y * W + x: the Philox counter
  // and the hit order) start at gid0; the whole grid (0, N, 0) unless the substrate is one row
  // slab of a larger world
  long long j0, n_own, gid0;
  GenomeArgs g;
  uint32_t thr_mut, thr_merge;
  float sigma;
  uint32_t world;
  unsigned long long seed;
  uint32_t step;
  // scratch
  int32_t* count;             // [cap]: 1 for slots that own a cell, else 0
  uint8_t* hitmask;           // [nblk * kRadThreads]: hit bits of each thread's 8 cells
  int32_t* blockcnt;          // [max(nblk, slot blocks)]: hits per block, then free slots per block
  int32_t* blockoff;          // [max(nblk, slot blocks)]: hit offsets, then live slots per block
  int4* hits;                 // [max_hits] (cell, parent, partner or -1, flags)
  uint32_t* hitbits;          // [max_hits]
  int max_hits;
  int32_t* freelist;          // [cap]
  int32_t* newslots;          // [cap]
  int* counters;              // [8]: n_hits, n_free, n_assigned, n_mut, n_merge, n_live
  coral_stats* rec;           // stats record of this step
};
cudaError_t launch_radiation(const RadiationArgs& r, cudaStream_t st);
// The two halves of launch_radiation for a row slab: the scan leaves the liveness flags of the
// own cells in r.count and the hits (global cell ids, in cell order) in r.hits / r.hitbits with
// their count in r.counters[0]; the apply takes global liveness flags in r.count and the global
// hit list in r.hits / r.hitbits / r.counters[0] (with the event counts in r.counters[3..4]),
// assigns the lowest free slots to the hits in order, writes the children and the G of the own
// cells among them, and regenerates the new slots' nets.
cudaError_t launch_radiation_scan(const RadiationArgs& r, cudaStream_t st);
cudaError_t launch_radiation_apply(const RadiationArgs& r, cudaStream_t st);
// FP64 totals (E, I, C0..C3) of cells [j0, j0 + n) of the six contiguous sensor planes at E,
// fixed order, into out[6] (device)
cudaError_t launch_row_totals(const float* E, long long N, long long j0, long long n, double* out, cudaStream_t st);
int radiation_blocks(long long N);
int radiation_threads();   // threads per radiation block (one hit-mask byte each)

struct SortArgs {
  const int32_t* keys_in;     // [N]
  long long N;
  int capacity;
  int32_t* count;             // [cap] output
  int32_t* perm;              // [N] output
  int32_t* k0; int32_t* v0;   // ping-pong scratch [N]
  int32_t* k1; int32_t* v1;
  int32_t* hist;              // [256 * nblk]
  int32_t* totals;            // [256]: keys per digit value of the current pass
};
cudaError_t launch_bucket(const SortArgs& a, cudaStream_t st);
int bucket_blocks(long long N);

}  // namespace coral
