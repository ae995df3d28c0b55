// Plain FP32 per-cell network (pass 1), physics stencil (pass 2) and the per-step FP64 totals.
#include <math.h>

#include "coral_internal.cuh"
#include "epilogue.cuh"

namespace coral {

namespace {

constexpr int kP1Threads = 128;
constexpr int kP2Threads = 256;

__device__ __forceinline__ void load6(const Planes& s, long long n, long long N, float* dst) {
  dst[0] = __ldg(s.E + n);
  dst[1] = __ldg(s.I + n);
#pragma unroll
  for (int c = 0; c < 4; ++c) dst[2 + c] = __ldg(s.C + (long long)c * N + n);
}

// Sums one value per thread into a per-warp FP64 accumulator held by lane 0.
__device__ __forceinline__ void warp_accumulate(float v, double& acc) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) acc += (double)v;
}

// Combines the lane-0 accumulators of all warps of the block in warp order.
template <int NS, int NC>
__device__ void block_partial(const double (&s)[NS], const long long (&c)[NC], Partial* out,
                              int s_first, int c_first, int slot) {
  __shared__ double ss[32][6];
  __shared__ long long sc[32][2];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < NS; ++k) ss[w][k] = s[k];
    for (int k = 0; k < NC; ++k) sc[w][k] = c[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial p = {};
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      for (int k = 0; k < NS; ++k) p.s[s_first + k] += ss[i][k];
      for (int k = 0; k < NC; ++k) p.c[c_first + k] += sc[i][k];
    }
    out[slot] = p;
  }
}

// One thread per cell: gather the rotation-ordered 3x3 neighbourhood of the six sensor
// channels straight from the SoA planes, run the FP32 net with FMA, apply the actuators.
__global__ void __launch_bounds__(kP1Threads, 4) k_pass1_fp32(const StepArgs a) {
  const int W = a.W, H = a.H, P = a.P;
  const long long N = a.N;
  double accC[4] = {0, 0, 0, 0};
  long long accX[1] = {0};
  const long long stride = (long long)gridDim.x * kP1Threads;
  for (long long base = (long long)blockIdx.x * kP1Threads; base < N; base += stride) {
    const long long j = base + threadIdx.x;
    const int y = (int)(j / P), x = (int)(j - (long long)y * P);
    const bool valid = j < N && x < W;               // row padding is not part of the torus
    CellOut o;
    o.C[0] = o.C[1] = o.C[2] = o.C[3] = 0.0f;
    o.xdir = kNoExplore;
    if (valid) {
      const int r = a.rotation ? (int)a.cur.R[j] : 0;
      float in[kIn];
      load6(a.cur, j, N, in);
#pragma unroll
      for (int p = 1; p < 9; ++p) {
        int dx, dy;
        octant_offset((2 * r + rank_delta(p)) & 7, dx, dy);
        const long long n = (long long)wrap(y + dy, H) * P + wrap(x + dx, W);
        load6(a.cur, n, N, in + 6 * p);
      }
      const int gj = a.cur.G[j];
      // an out-of-range GenomeIndex (loaded, reported as invalid) runs slot 0's net
      const float* net = a.nets32 + (long long)((unsigned)gj < (unsigned)a.capacity ? gj : 0) * a.net_stride;
      float act[kOut], zo[kOut];
      if (a.hidden == 0) {
#pragma unroll
        for (int oo = 0; oo < kOut; ++oo) {
          const float4* w = reinterpret_cast<const float4*>(net + oo * 56);
          float acc = __ldg(net + net32_b1(0) + oo);
#pragma unroll
          for (int q = 0; q < 13; ++q) {
            const float4 w4 = __ldg(w + q);
            acc = fmaf(w4.x, in[4 * q], acc);
            acc = fmaf(w4.y, in[4 * q + 1], acc);
            acc = fmaf(w4.z, in[4 * q + 2], acc);
            acc = fmaf(w4.w, in[4 * q + 3], acc);
          }
          const float4 w4 = __ldg(w + 13);
          acc = fmaf(w4.x, in[52], acc);
          acc = fmaf(w4.y, in[53], acc);
          zo[oo] = acc;
          act[oo] = tanhf(acc);
        }
      } else {
        const int Hd = a.hidden;
        const float* b1 = net + net32_b1(Hd);
        const float* w2t = net + net32_w2t(Hd);
        const float* b2 = net + net32_b2(Hd);
        float acc2[kOut];
#pragma unroll
        for (int oo = 0; oo < kOut; ++oo) acc2[oo] = __ldg(b2 + oo);
        for (int k = 0; k < Hd; ++k) {
          const float4* w = reinterpret_cast<const float4*>(net + k * 56);
          float acc = __ldg(b1 + k);
#pragma unroll
          for (int q = 0; q < 13; ++q) {
            const float4 w4 = __ldg(w + q);
            acc = fmaf(w4.x, in[4 * q], acc);
            acc = fmaf(w4.y, in[4 * q + 1], acc);
            acc = fmaf(w4.z, in[4 * q + 2], acc);
            acc = fmaf(w4.w, in[4 * q + 3], acc);
          }
          const float4 w4 = __ldg(w + 13);
          acc = fmaf(w4.x, in[52], acc);
          acc = fmaf(w4.y, in[53], acc);
          const float h = tanhf(acc);
          const float4* u = reinterpret_cast<const float4*>(w2t + k * 12);
          const float4 u0 = __ldg(u), u1 = __ldg(u + 1), u2 = __ldg(u + 2);
          acc2[0] = fmaf(u0.x, h, acc2[0]);
          acc2[1] = fmaf(u0.y, h, acc2[1]);
          acc2[2] = fmaf(u0.z, h, acc2[2]);
          acc2[3] = fmaf(u0.w, h, acc2[3]);
          acc2[4] = fmaf(u1.x, h, acc2[4]);
          acc2[5] = fmaf(u1.y, h, acc2[5]);
          acc2[6] = fmaf(u1.z, h, acc2[6]);
          acc2[7] = fmaf(u1.w, h, acc2[7]);
          acc2[8] = fmaf(u2.x, h, acc2[8]);
          acc2[9] = fmaf(u2.y, h, acc2[9]);
        }
#pragma unroll
        for (int oo = 0; oo < kOut; ++oo) {
          zo[oo] = acc2[oo];
          act[oo] = tanhf(acc2[oo]);
        }
      }
      // FP64 flow denominator: I_t of the von Neumann neighbours (kernel ranks 1, 4, 5, 8).
      const double S = (double)in[7] + (double)in[25] + (double)in[31] + (double)in[49];
      actuator_epilogue(a, act, zo, in[0], in[1], (float)S, r, o);
      store_pass1(a, j, o);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) warp_accumulate(valid ? o.C[k] : 0.0f, accC[k]);
    const int ex = warp_sum_i(valid && o.xdir != kNoExplore ? 1 : 0);
    if ((threadIdx.x & 31) == 0) accX[0] += ex;
  }
  block_partial<4, 1>(accC, accX, a.part1, 2, 0, blockIdx.x);
}

// Day or night for this step (batched stepping reads the step index from the device).
__device__ __forceinline__ bool is_day_now(const StepArgs& a) {
  if (!a.step_dev) return a.is_day != 0;
  const long long t = *a.step_dev;
  return (t % a.day_period) * 2 < a.day_period;
}

// Pass 2: exploration resolve and takeover, energy flow, day/night. Each thread resolves 4
// consecutive cells of one pitched row (16-byte loads and stores; the last chunk of a row holds
// the row's padding when the width is not a multiple of 4: its padding cells keep G = -1, R = 0
// and get E = I = 0). CTA `cta` of `ncta` strides over the chunks, partial sums to a.part2[cta].
__device__ __forceinline__ void pass2_body(const StepArgs& a, const int cta, const int ncta) {
  const int W = a.W, H = a.H, P = a.P;
  const int cpr = P >> 2;                       // chunks per row
  const int n_chunks = cpr * H;
  const bool day = is_day_now(a);
  double acc[2] = {0, 0};
  long long accT[1] = {0};
  const int stride = ncta * kP2Threads;
  for (int base = cta * kP2Threads; base < n_chunks; base += stride) {
    const int c = base + threadIdx.x;
    const bool valid = c < n_chunks;
    float e_sum = 0.0f, i_sum = 0.0f;
    int takes = 0;
    if (valid) {
      const int y = c / cpr;
      const int x = (c - y * cpr) << 2;
      const int nv = min(4, W - x);                             // torus cells of this chunk
      const int j = y * P + x;
      const int jn = (y == 0 ? H - 1 : y - 1) * P + x;          // same columns, row above
      const int js = (y == H - 1 ? 0 : y + 1) * P + x;          // row below
      const int jw = y * P + (x == 0 ? W - 1 : x - 1);          // west of the first cell
      const int je = y * P + (x + 4 >= W ? 0 : x + 4);          // east of the last torus cell
      float4 rc[4];                                             // keep, I1, q, xamt
      float2 rn[4], rs[4];                                      // the rows above and below: q, xamt
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        rc[k] = a.p1.rec[j + k];
        rn[k] = *reinterpret_cast<const float2*>(&a.p1.rec[jn + k].z);
        rs[k] = *reinterpret_cast<const float2*>(&a.p1.rec[js + k].z);
      }
      const float4 It = *reinterpret_cast<const float4*>(a.cur.I + j);
      const uint32_t dc = *reinterpret_cast<const uint32_t*>(a.p1.xdir + j);
      const uint32_t dN = *reinterpret_cast<const uint32_t*>(a.p1.xdir + jn);
      const uint32_t dS = *reinterpret_cast<const uint32_t*>(a.p1.xdir + js);
      const int4 Gc = *reinterpret_cast<const int4*>(a.cur.G + j);
      const uint32_t Rc = *reinterpret_cast<const uint32_t*>(a.cur.R + j);
      const uint8_t dW = a.p1.xdir[jw], dE = a.p1.xdir[je];
      const float2 wq = *reinterpret_cast<const float2*>(&a.p1.rec[jw].z);
      const float2 eq = *reinterpret_cast<const float2*>(&a.p1.rec[je].z);
      const float xaW = wq.y, xaE = eq.y, qW = wq.x, qE = eq.x;
      float vI1[4], vxa[4], vkp[4], vq[4], vxaN[4], vxaS[4], vqN[4], vqS[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        vkp[k] = rc[k].x; vI1[k] = rc[k].y; vq[k] = rc[k].z; vxa[k] = rc[k].w;
        vqN[k] = rn[k].x; vxaN[k] = rn[k].y; vqS[k] = rs[k].x; vxaS[k] = rs[k].y;
      }
      const float vIt[4] = {It.x, It.y, It.z, It.w};
      const int vG[4] = {Gc.x, Gc.y, Gc.z, Gc.w};
      float oE[4], oI[4];
      int oG[4];
      uint32_t oR = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= nv) {                                          // row padding keeps its values
          oE[k] = 0.0f;
          oI[k] = 0.0f;
          oG[k] = vG[k];
          oR |= ((Rc >> (8 * k)) & 0xFFu) << (8 * k);
          continue;
        }
        const bool last = k == nv - 1;                          // its east neighbour is past the chunk
        // neighbours of cell x+k in N, E, S, W order: direction byte, amount, flow quotient
        const uint32_t nd[4] = {(dN >> (8 * k)) & 0xFFu,
                                !last ? (dc >> (8 * (k + 1))) & 0xFFu : (uint32_t)dE,
                                (dS >> (8 * k)) & 0xFFu,
                                k > 0 ? (dc >> (8 * (k - 1))) & 0xFFu : (uint32_t)dW};
        const float na[4] = {vxaN[k], !last ? vxa[k < 3 ? k + 1 : 3] : xaE, vxaS[k], k > 0 ? vxa[k - 1] : xaW};
        const float nq[4] = {vqN[k], !last ? vq[k < 3 ? k + 1 : 3] : qE, vqS[k], k > 0 ? vq[k - 1] : qW};
        float I2 = vI1[k] - vxa[k];
        float best = -INFINITY;
        int bd = -1;
#pragma unroll
        for (int D = 0; D < 4; ++D) {
          if (nd[D] == (uint32_t)((D + 2) & 3)) {
            I2 += na[D];
            if (na[D] > best) { best = na[D]; bd = D; }
          }
        }
        const bool take = bd >= 0 && best > vI1[k];
        int g = vG[k];
        uint32_t r = (Rc >> (8 * k)) & 0xFFu;
        if (take) {
          const int nb = bd == 0 ? jn + k : (bd == 2 ? js + k : (bd == 1 ? (!last ? j + k + 1 : je) : (k > 0 ? j + k - 1 : jw)));
          g = a.cur.G[nb];
          r = bd == 0 ? nd[0] : (bd == 1 ? nd[1] : (bd == 2 ? nd[2] : nd[3]));
          ++takes;
        }
        const float inflow = ((nq[0] + nq[1]) + nq[2]) + nq[3];
        const float E2 = vkp[k] + vIt[k] * inflow;
        oE[k] = day ? E2 + a.e_day : E2 - a.e_night * E2;
        oI[k] = I2;
        oG[k] = g;
        oR |= r << (8 * k);
        e_sum += oE[k];
        i_sum += oI[k];
      }
      *reinterpret_cast<float4*>(a.nxt.E + j) = make_float4(oE[0], oE[1], oE[2], oE[3]);
      *reinterpret_cast<float4*>(a.nxt.I + j) = make_float4(oI[0], oI[1], oI[2], oI[3]);
      *reinterpret_cast<int4*>(a.nxt.G + j) = make_int4(oG[0], oG[1], oG[2], oG[3]);
      *reinterpret_cast<uint32_t*>(a.nxt.R + j) = oR;
    }
    warp_accumulate(e_sum, acc[0]);
    warp_accumulate(i_sum, acc[1]);
    const int tk = warp_sum_i(takes);
    if ((threadIdx.x & 31) == 0) accT[0] += tk;
  }
  block_partial<2, 1>(acc, accT, a.part2, 0, 1, cta);
}

__global__ void __launch_bounds__(kP2Threads) k_pass2_x4(const __grid_constant__ StepArgs a) {
  pass2_body(a, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kP2Threads) k_pass2_batch(const __grid_constant__ BatchTable bt, const int parity) {
  __shared__ StepArgs a;
  const int w = bt.cta_world2[blockIdx.x];
  copy_args_to_shared(&a, &bt.args[parity * bt.n + w]);
  __syncthreads();
  pass2_body(a, blockIdx.x - bt.world_first2[w], bt.world_ctas2[w]);
}

// Fixed-order FP64 combination of the block partials into the stats ring.
__global__ void __launch_bounds__(256) k_stats(const Partial* p1, int n1, const Partial* p2, int n2,
                                              long long t, coral_stats* ring) {
  __shared__ double ss[256][6];
  __shared__ long long sc[256][2];
  double s[6] = {0, 0, 0, 0, 0, 0};
  long long c[2] = {0, 0};
  for (int i = threadIdx.x; i < n1; i += 256) {
    for (int k = 2; k < 6; ++k) s[k] += p1[i].s[k];
    c[0] += p1[i].c[0];
  }
  for (int i = threadIdx.x; i < n2; i += 256) {
    s[0] += p2[i].s[0];
    s[1] += p2[i].s[1];
    c[1] += p2[i].c[1];
  }
  for (int k = 0; k < 6; ++k) ss[threadIdx.x][k] = s[k];
  sc[threadIdx.x][0] = c[0];
  sc[threadIdx.x][1] = c[1];
  __syncthreads();
  for (int h = 128; h; h >>= 1) {
    if ((int)threadIdx.x < h) {
      for (int k = 0; k < 6; ++k) ss[threadIdx.x][k] += ss[threadIdx.x + h][k];
      sc[threadIdx.x][0] += sc[threadIdx.x + h][0];
      sc[threadIdx.x][1] += sc[threadIdx.x + h][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    coral_stats r;
    r.step = t;
    r.sum_E = ss[0][0];
    r.sum_I = ss[0][1];
    for (int k = 0; k < 4; ++k) r.sum_C[k] = ss[0][2 + k];
    r.n_explore = sc[0][0];
    r.n_takeover = sc[0][1];
    r.n_live = -1;
    r.n_mut = r.n_merge = r.n_born = r.n_skipped = 0;
    ring[t % kRing] = r;
  }
}

// Batched totals: block w combines world w's partials (pass-1 and pass-2 CTA counts of that
// world) into its ring at its device step index, then advances the step index.
__global__ void __launch_bounds__(256) k_stats_batch(const __grid_constant__ BatchTable bt, const int parity) {
  const int w = blockIdx.x;
  const StepArgs& a = bt.args[parity * bt.n + w];
  __shared__ double ss[256][6];
  __shared__ long long sc[256][2];
  double s[6] = {0, 0, 0, 0, 0, 0};
  long long c[2] = {0, 0};
  const int n1 = bt.world_ctas1[w], n2 = bt.world_ctas2[w];
  for (int i = threadIdx.x; i < n1; i += 256) {
    for (int k = 2; k < 6; ++k) s[k] += a.part1[i].s[k];
    c[0] += a.part1[i].c[0];
  }
  for (int i = threadIdx.x; i < n2; i += 256) {
    s[0] += a.part2[i].s[0];
    s[1] += a.part2[i].s[1];
    c[1] += a.part2[i].c[1];
  }
  for (int k = 0; k < 6; ++k) ss[threadIdx.x][k] = s[k];
  sc[threadIdx.x][0] = c[0];
  sc[threadIdx.x][1] = c[1];
  __syncthreads();
  for (int h = 128; h; h >>= 1) {
    if ((int)threadIdx.x < h) {
      for (int k = 0; k < 6; ++k) ss[threadIdx.x][k] += ss[threadIdx.x + h][k];
      sc[threadIdx.x][0] += sc[threadIdx.x + h][0];
      sc[threadIdx.x][1] += sc[threadIdx.x + h][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long t = bt.steps[w];
    coral_stats r;
    r.step = t;
    r.sum_E = ss[0][0];
    r.sum_I = ss[0][1];
    for (int k = 0; k < 4; ++k) r.sum_C[k] = ss[0][2 + k];
    r.n_explore = sc[0][0];
    r.n_takeover = sc[0][1];
    r.n_live = -1;
    r.n_mut = r.n_merge = r.n_born = r.n_skipped = 0;
    bt.rings[w][t % kRing] = r;
    bt.steps[w] = t + 1;
  }
}

int occupancy_grid(const void* fn, int threads, size_t smem, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  int g = per_sm * sms;
  return g > kMaxPartials ? kMaxPartials : g;
}

}  // namespace

int pass1_fp32_grid(int sms) { return occupancy_grid((const void*)k_pass1_fp32, kP1Threads, 0, sms); }
int pass2_grid(int sms) { return occupancy_grid((const void*)k_pass2_x4, kP2Threads, 0, sms); }

cudaError_t launch_pass1_fp32(const StepArgs& a, cudaStream_t st, int grid) {
  k_pass1_fp32<<<grid, kP1Threads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pass2(const StepArgs& a, cudaStream_t st, int grid) {
  k_pass2_x4<<<grid, kP2Threads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pass2_batch(const BatchTable& b, int parity, int grid, cudaStream_t st) {
  k_pass2_batch<<<grid, kP2Threads, 0, st>>>(b, parity);
  return cudaGetLastError();
}

cudaError_t launch_stats_batch(const BatchTable& b, cudaStream_t st) {
  k_stats_batch<<<b.n, 256, 0, st>>>(b, 0);
  return cudaGetLastError();
}

cudaError_t launch_stats(const StepArgs& a, int n1, int n2, long long t, coral_stats* ring,
                         cudaStream_t st) {
  k_stats<<<1, 256, 0, st>>>(a.part1, n1, a.part2, n2, t, ring);
  return cudaGetLastError();
}

}  // namespace coral
