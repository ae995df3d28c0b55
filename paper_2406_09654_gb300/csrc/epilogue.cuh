// Actuator epilogue shared by both network paths: from the ten activated actuator values of a
// cell to its pass-1 outputs (Section "Experiment").
#pragma once

#include "coral_internal.cuh"

namespace coral {

struct CellOut {
  float C[4];
  float keep, q, I1, xamt;
  uint8_t xdir;
};

// a[0..3] com, a[4] invest, a[5] liquidate, a[6..9] explore (fwd, right, left, back);
// z[6..9]: pre-activations of the explore actuators (tanh is strictly increasing, so the
// maximal actuator and its sign are read off z, where saturated outputs cannot tie).
// E, I: the cell's state; Sf: the sum of I_t over its 4 von Neumann neighbours, summed in FP64
// and rounded once to float32 (Sf > 0 exactly when the sum is > 0); r: rotation.
// kFast: hardware exp / reciprocal / reciprocal-square-root approximations (relative error
// ~1e-6, far inside the BF16 path's tolerance); otherwise the accurate library functions.
template <bool kFast = false>
__device__ __forceinline__ void actuator_epilogue(const StepArgs& p, const float* a, const float* z,
                                                  float E, float I, float Sf, int r, CellOut& o) {
  // Communication: normalised by max(1, ||a0..3||) and passed through a sigmoid.
  const float n2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3];
  if (kFast) {
    // sigmoid(x) = (1 + tanh(x / 2)) / 2 with the hardware tanh (relative error < 2^-10.9)
    const float inv = n2 > 1.0f ? rsqrtf(n2) : 1.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float t;
      asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * (a[k] * inv)));
      o.C[k] = fmaf(0.5f, t, 0.5f);
    }
  } else {
    const float nrm = fmaxf(1.0f, sqrtf(n2));
#pragma unroll
    for (int k = 0; k < 4; ++k) o.C[k] = 1.0f / (1.0f + expf(-(a[k] / nrm)));
  }
  // Invest moves inv*E into infrastructure, liquidate moves liq*I back into energy.
  const float inv = p.k_inv * fmaxf(a[4], 0.0f);
  const float liq = p.k_liq * fmaxf(a[5], 0.0f);
  const float E1 = E - inv * E + liq * I;
  const float I1 = I + inv * E - liq * I;
  // Exploration toward the maximal explore actuator (first maximum on ties).
  int k = 0;
  float zm = z[6], m = a[6];
  if (z[7] > zm) { k = 1; zm = z[7]; m = a[7]; }
  if (z[8] > zm) { k = 2; zm = z[8]; m = a[8]; }
  if (z[9] > zm) { k = 3; zm = z[9]; m = a[9]; }
  const bool go = (zm > 0.0f) && (I1 > 0.0f);
  o.xdir = go ? (uint8_t)((r + explore_turn(k)) & 3) : kNoExplore;
  o.xamt = go ? p.k_exp * m * I1 : 0.0f;
  o.I1 = I1;
  // Energy flow along infrastructure: the cell keeps (1 - k_flow) E1 when it has somewhere
  // to send, and each neighbour j receives I_t(j) * q with q = k_flow E1 / S.
  const bool send = Sf > 0.0f;
  o.keep = send ? E1 - p.k_flow * E1 : E1;
  o.q = send ? (kFast ? __fdividef(p.k_flow * E1, Sf) : (p.k_flow * E1) / Sf) : 0.0f;
}

__device__ __forceinline__ void store_pass1(const StepArgs& p, long long j, const CellOut& o) {
#pragma unroll
  for (int k = 0; k < 4; ++k) p.nxt.C[(long long)k * p.N + j] = o.C[k];
  p.p1.rec[j] = make_float4(o.keep, o.I1, o.q, o.xamt);
  p.p1.xdir[j] = o.xdir;
}

}  // namespace coral
