// C ABI of the substrate-step library: substrate lifetime, device memory ownership, loads and
// reads, and the per-step launch sequence. Declarations and contracts: include/coral.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "coral_internal.cuh"

using namespace coral;

// Host-to-host job stepping (coral_step_jobs): two input and two output staging buffers of
// one packed state each, a copy-in and a copy-out stream, and the events that order them with
// the substrate's stream. Created at the first call.
struct JobPipe {
  uint8_t* in[2] = {};
  uint8_t* out[2] = {};
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t h2d_done[2] = {}, in_free[2] = {}, out_ready[2] = {}, out_free[2] = {};
  bool ready = false;
};

struct coral_substrate {
  coral_params p;
  int W = 0, H = 0;
  int P = 0;                    // row pitch of the planes in cells (W rounded up to a multiple of 4)
  long long N = 0;              // plane length H * P
  long long NL = 0;             // torus cells W * H
  int cap = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 0;
  std::vector<void*> allocs;
  Planes st[2] = {};
  int cur = 0;
  CUtensorMap tmap[2];          // TMA descriptors of the two state buffers' sensor planes
  bool tmap_ok = false;
  Pass1Bufs p1 = {};
  GenomeArgs g = {};
  bool genomes_loaded = false;
  bool has_cppn = false;
  Partial* part1 = nullptr;
  int* sched = nullptr;         // pass 1's tile pool counters
  Partial* part2 = nullptr;
  coral_stats* ring = nullptr;
  int* status = nullptr;
  // radiation scratch
  int32_t* count = nullptr;
  uint8_t* hitmask = nullptr;
  int32_t* blockcnt = nullptr;
  int32_t* blockoff = nullptr;
  int4* hits = nullptr;
  uint32_t* hitbits = nullptr;
  int32_t* freelist = nullptr;
  int32_t* newslots = nullptr;
  int* counters = nullptr;
  // bucketing scratch (allocated at the first coral_read_perm)
  int32_t* sort_buf = nullptr;
  long long t = 0;
  int grid1 = 0, grid2 = 0;
  int fma_cutoff = 0;           // BF16 pass 1: FMA path for later genome rounds of at most this many cells
  JobPipe jobs;
  // row slab of a larger world (coral_slab_set): own rows [row_lo, row_hi), global id of the
  // first own cell; radiation then runs through coral_slab_radiation_scan / _apply
  bool slab = false;
  int row_lo = 0, row_hi = 0;
  long long gid0 = 0;
  double* totals_buf = nullptr;  // coral_slab_totals: 6 totals + per-block partials
  std::string err;
};

namespace {

thread_local std::string g_err = "no error";

int fail(coral_substrate* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  g_err = msg;
  return code;
}

int cuda_fail(coral_substrate* s, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(s, e == cudaErrorMemoryAllocation ? CORAL_E_OOM : CORAL_E_CUDA, m);
}

#define CK(s, call)                                        \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
  } while (0)

template <typename T>
cudaError_t dalloc(coral_substrate* s, T** p, size_t count) {
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, count * sizeof(T) + 256);
  if (e != cudaSuccess) return e;
  s->allocs.push_back(d);
  *p = reinterpret_cast<T*>(d);
  return cudaSuccess;
}

void free_all(coral_substrate* s) {
  for (void* d : s->allocs) cudaFree(d);
  s->allocs.clear();
}

// Radiation hit threshold of a probability (reading R2): a cell is hit iff its 32-bit Philox
// word is below floor(p * 2^32), capped at 2^32 - 1 (p * 2^32 is exact in double precision).
uint32_t hit_threshold(double p) {
  const double t = floor(p * 4294967296.0);
  return t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
}

bool valid_hidden(int h) { return h == 0 || h == 16 || h == 32 || h == 48 || h == 64; }

StepArgs step_args(const coral_substrate* s) {
  StepArgs a = {};
  a.W = s->W;
  a.H = s->H;
  a.N = s->N;
  a.P = s->P;
  a.hidden = s->p.hidden;
  a.rotation = s->p.rotation;
  a.k_inv = s->p.k_inv;
  a.k_liq = s->p.k_liq;
  a.k_exp = s->p.k_exp;
  a.k_flow = s->p.k_flow;
  a.is_day = ((s->t % s->p.day_period) * 2 < s->p.day_period) ? 1 : 0;
  a.e_day = s->p.e_day;
  a.e_night = s->p.e_night;
  a.cur = s->st[s->cur];
  a.nxt = s->st[s->cur ^ 1];
  a.p1 = s->p1;
  a.nets32 = s->g.nets32;
  a.net_stride = s->g.net_stride;
  a.nets16 = s->g.nets16;
  a.blob_bytes = s->g.blob_bytes;
  a.part1 = s->part1;
  a.part2 = s->part2;
  a.status = s->status;
  a.day_period = s->p.day_period;
  a.capacity = s->cap;
  a.step_dev = nullptr;
  a.sched = s->sched;
  a.fma_cutoff = s->fma_cutoff;
  return a;
}

// Pageable host memory (not pinned, not registered): a 2-D copy to or from it goes row by row
// through the driver's staging buffers, so the planes are copied as one contiguous block and
// re-pitched on the device instead.
bool pageable(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeUnregistered;
}

// The spare state buffer (the one the next step writes in full) serves as the packed staging
// area between steps: its E plane holds N >= W * H floats. Afterwards its row padding is set
// back to zero (the padding of every float plane is zero; the totals sum over pitched rows).
cudaError_t host_to_pitched(coral_substrate* s, void* dst, const void* src, size_t es) {
  const size_t W = (size_t)s->W, H = (size_t)s->H, P = (size_t)s->P;
  float* spare = s->st[s->cur ^ 1].E;
  cudaError_t e = cudaMemcpyAsync(spare, src, es * W * H, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpy2DAsync(dst, es * P, spare, es * W, es * W, H, cudaMemcpyDeviceToDevice, s->stream);
  return e;
}

cudaError_t pitched_to_host(coral_substrate* s, void* dst, const void* src, size_t es) {
  const size_t W = (size_t)s->W, H = (size_t)s->H, P = (size_t)s->P;
  float* spare = s->st[s->cur ^ 1].E;
  cudaError_t e = cudaMemcpy2DAsync(spare, es * W, src, es * P, es * W, H, cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, spare, es * W * H, cudaMemcpyDeviceToHost, s->stream);
  return e;
}

cudaError_t restore_spare_padding(coral_substrate* s) {
  const size_t W = (size_t)s->W, H = (size_t)s->H, P = (size_t)s->P;
  float* spare = s->st[s->cur ^ 1].E;
  // the staging area is the E plane's first W * H floats: zero them where they cover padding
  return cudaMemset2DAsync(spare + W, 4 * P, 0, 4 * (P - W), H, s->stream);
}

cudaMemcpyKind kind_in(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

int check_status(coral_substrate* s) {
  int st = 0;
  CK(s, cudaStreamSynchronize(s->stream));
  CK(s, cudaMemcpy(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    CK(s, cudaMemset(s->status, 0, sizeof(int)));
    return fail(s, st, st == CORAL_E_INVALID ? "invalid value found on the device (G outside [0, capacity) or R > 3)"
                                             : "device-side error");
  }
  return CORAL_OK;
}

}  // namespace

extern "C" {

int32_t coral_net_floats(int32_t hidden) { return dense_floats(hidden); }

int coral_params_default(coral_params* p) {
  if (!p) return fail(nullptr, CORAL_E_INVALID, "params is NULL");
  memset(p, 0, sizeof(*p));
  p->hidden = 0;
  p->path = CORAL_NET_FP32_PERCELL;
  p->k_inv = 0.1f;
  p->k_liq = 0.1f;
  p->k_exp = 0.5f;
  p->k_flow = 0.2f;
  p->e_day = 0.005f;
  p->e_night = 0.005f;
  p->day_period = 200;
  p->rotation = 1;
  p->radiation_every = 0;
  p->p_mut = 0.0;
  p->p_merge = 0.0;
  p->sigma_mut = 0.05f;
  p->world = 0;
  p->seed = 0;
  return CORAL_OK;
}

int coral_substrate_create(const coral_params* p, int32_t width, int32_t height, int32_t genome_capacity,
                           void* cuda_stream, coral_substrate** out) {
  if (!p || !out) return fail(nullptr, CORAL_E_INVALID, "NULL argument");
  *out = nullptr;
  if (width < 3 || height < 3) return fail(nullptr, CORAL_E_INVALID, "width and height must be >= 3");
  if ((long long)row_pitch(width) * height >= (1LL << 31))
    return fail(nullptr, CORAL_E_INVALID, "width (rounded up to a multiple of 4) * height must be < 2^31");
  if (genome_capacity < 1 || genome_capacity > (1 << 24))
    return fail(nullptr, CORAL_E_INVALID, "genome_capacity must be in [1, 2^24]");
  if (!valid_hidden(p->hidden)) return fail(nullptr, CORAL_E_INVALID, "hidden must be 0, 16, 32, 48 or 64");
  if (p->path != CORAL_NET_FP32_PERCELL && p->path != CORAL_NET_BF16_GROUPED)
    return fail(nullptr, CORAL_E_INVALID, "unknown path");
  if (p->day_period < 1) return fail(nullptr, CORAL_E_INVALID, "day_period must be >= 1");
  if (p->radiation_every < 0) return fail(nullptr, CORAL_E_INVALID, "radiation_every must be >= 0");
  if (!(p->p_mut >= 0.0 && p->p_mut <= 1.0) || !(p->p_merge >= 0.0 && p->p_merge <= 1.0))
    return fail(nullptr, CORAL_E_INVALID, "p_mut and p_merge must be in [0, 1]");
  coral_substrate* s = nullptr;
  try {
    s = new coral_substrate();
  } catch (...) {
    return fail(nullptr, CORAL_E_OOM, "host allocation failed");
  }
  s->p = *p;
  s->W = width;
  s->H = height;
  s->P = row_pitch(width);
  s->N = (long long)height * s->P;
  s->NL = (long long)width * height;
  s->cap = genome_capacity;
  s->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  int rc = CORAL_OK;
  do {
    cudaError_t e;
    if ((e = cudaGetDevice(&s->device)) != cudaSuccess) { rc = cuda_fail(s, e, "cudaGetDevice"); break; }
    if ((e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device)) != cudaSuccess) {
      rc = cuda_fail(s, e, "cudaDeviceGetAttribute");
      break;
    }
    const long long N = s->N;
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
      // the six sensor planes are contiguous (E, I, C0..C3, N floats each): plane c = E + c * N
      ok &= dalloc(s, &s->st[b].E, 6 * N) == cudaSuccess;
      if (ok) {
        s->st[b].I = s->st[b].E + N;
        s->st[b].C = s->st[b].E + 2 * N;
      }
      ok &= dalloc(s, &s->st[b].G, N) == cudaSuccess;
      ok &= dalloc(s, &s->st[b].R, N) == cudaSuccess;
    }
    ok = ok && dalloc(s, &s->p1.rec, N) == cudaSuccess && dalloc(s, &s->p1.xdir, N) == cudaSuccess;
    s->g.hidden = p->hidden;
    s->g.capacity = genome_capacity;
    s->g.net_stride = net32_stride(p->hidden);
    s->g.blob_bytes = bf16_blob_bytes(p->hidden);
    ok = ok && dalloc(s, &s->g.genes, (size_t)genome_capacity * kGenes) == cudaSuccess &&
         dalloc(s, &s->g.parent, (size_t)genome_capacity) == cudaSuccess &&
         dalloc(s, &s->g.nets32, (size_t)genome_capacity * s->g.net_stride) == cudaSuccess &&
         dalloc(s, &s->g.nets16, (size_t)genome_capacity * s->g.blob_bytes) == cudaSuccess;
    ok = ok && dalloc(s, &s->part1, kMaxPartials) == cudaSuccess && dalloc(s, &s->part2, kMaxPartials) == cudaSuccess &&
         dalloc(s, &s->ring, kRing) == cudaSuccess && dalloc(s, &s->status, 4) == cudaSuccess &&
         dalloc(s, &s->sched, 2) == cudaSuccess;
    const int nblk = radiation_blocks(N);
    // per-block counts of the hit passes (cells) and of the free-slot passes (slots)
    const int nbc = std::max(nblk, (genome_capacity + 1023) / 1024);
    ok = ok && dalloc(s, &s->count, genome_capacity) == cudaSuccess && dalloc(s, &s->blockcnt, nbc) == cudaSuccess &&
         dalloc(s, &s->blockoff, nbc) == cudaSuccess && dalloc(s, &s->hits, genome_capacity) == cudaSuccess &&
         dalloc(s, &s->hitbits, genome_capacity) == cudaSuccess &&
         dalloc(s, &s->freelist, genome_capacity) == cudaSuccess &&
         dalloc(s, &s->newslots, genome_capacity) == cudaSuccess && dalloc(s, &s->counters, 8) == cudaSuccess &&
         dalloc(s, &s->hitmask, (size_t)nblk * radiation_threads()) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      rc = fail(s, CORAL_E_OOM, "device allocation failed");
      break;
    }
    // row padding: G = -1 (no genome), R = 0, floats 0, in both state buffers; loads and reads
    // copy the torus columns only, and the kernels keep the padding as it is
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      if ((e = cudaMemset(s->st[b].E, 0, sizeof(float) * 6 * N)) == cudaSuccess &&
          (e = cudaMemset(s->st[b].G, 0xFF, sizeof(int32_t) * N)) == cudaSuccess)
        e = cudaMemset(s->st[b].R, 0, (size_t)N);
    }
    if (e != cudaSuccess ||
        (e = cudaMemset(s->status, 0, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(s->sched, 0, 2 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(s->ring, 0, kRing * sizeof(coral_stats))) != cudaSuccess ||
        (e = cudaMemset(s->g.parent, 0xFF, sizeof(int32_t) * genome_capacity)) != cudaSuccess ||
        (e = cudaMemset(s->g.genes, 0, sizeof(float) * kGenes * genome_capacity)) != cudaSuccess ||
        (e = cudaMemset(s->g.nets32, 0, sizeof(float) * s->g.net_stride * (size_t)genome_capacity)) != cudaSuccess ||
        (e = cudaMemset(s->g.nets16, 0, (size_t)s->g.blob_bytes * genome_capacity)) != cudaSuccess) {
      rc = cuda_fail(s, e, "cudaMemset");
      break;
    }
    s->grid1 = p->path == CORAL_NET_BF16_GROUPED ? pass1_bf16_grid(s->sms) : pass1_fp32_grid(s->sms);
    if (p->path == CORAL_NET_BF16_GROUPED)
      s->tmap_ok = encode_sensor_tmap(&s->tmap[0], s->st[0].E, width, height, s->P) &&
                   encode_sensor_tmap(&s->tmap[1], s->st[1].E, width, height, s->P);
    s->grid2 = pass2_grid(s->sms);
    if (s->grid1 < 1) {
      rc = fail(s, CORAL_E_CUDA, "the BF16 tensor-core kernel cannot be launched on this device");
      break;
    }
    // small worlds: no more CTAs than units of work (pass-1 tiles; pass-2 chunks of 4 cells,
    // 256 per CTA), so that CTAs without work do not pay for their setup every step
    if (p->path == CORAL_NET_BF16_GROUPED)
      s->grid1 = (int)std::min<long long>(s->grid1, pass1_bf16_tiles(width, height));
    s->grid2 = (int)std::min<long long>(s->grid2, (N + 1023) / 1024);
  } while (0);
  if (rc != CORAL_OK) {
    free_all(s);
    delete s;
    return rc;
  }
  *out = s;
  return CORAL_OK;
}

int coral_substrate_destroy(coral_substrate* s) {
  if (!s) return CORAL_OK;
  cudaStreamSynchronize(s->stream);
  JobPipe& jp = s->jobs;
  for (cudaStream_t st : {jp.s_in, jp.s_out})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (int b = 0; b < 2; ++b)
    for (cudaEvent_t ev : {jp.h2d_done[b], jp.in_free[b], jp.out_ready[b], jp.out_free[b]})
      if (ev) cudaEventDestroy(ev);
  free_all(s);
  delete s;
  return CORAL_OK;
}

int coral_set_fma_cutoff(coral_substrate* s, int32_t cells) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (cells < 0 || cells > kFmaCutoffMax) return fail(s, CORAL_E_INVALID, "cells must be in [0, 128]");
  s->fma_cutoff = cells;
  return CORAL_OK;
}

int coral_state_load(coral_substrate* s, const float* E, const float* I, const float* C, const int32_t* G,
                     const uint8_t* R, int src_on_device) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  const Planes& d = s->st[s->cur];
  const cudaMemcpyKind k = kind_in(src_on_device);
  const size_t W = (size_t)s->W, H = (size_t)s->H, P = (size_t)s->P, NP = (size_t)s->N;
  // packed rows of W cells in, pitched rows of P cells on the device (the padding untouched)
  const bool host_pageable =
      !src_on_device && (pageable(E) || pageable(I) || pageable(C) || pageable(G) || pageable(R));
  const bool stage = host_pageable && P != W;
  auto plane_in = [&](void* dst, const void* src, size_t es) -> int {
    if (!src) return CORAL_OK;
    if (stage) {
      CK(s, host_to_pitched(s, dst, src, es));
    } else if (host_pageable) {                     // rows unpadded: one contiguous copy
      CK(s, cudaMemcpyAsync(dst, src, es * W * H, k, s->stream));
    } else {
      CK(s, cudaMemcpy2DAsync(dst, es * P, src, es * W, es * W, H, k, s->stream));
    }
    return CORAL_OK;
  };
  int rc;
  if ((rc = plane_in(d.E, E, 4)) || (rc = plane_in(d.I, I, 4))) return rc;
  for (size_t c = 0; c < 4 && C; ++c)
    if ((rc = plane_in(d.C + c * NP, C + c * W * H, 4))) return rc;
  if ((rc = plane_in(d.G, G, 4)) || (rc = plane_in(d.R, R, 1))) return rc;
  if (stage) CK(s, restore_spare_padding(s));
  if (G || R)
    CK(s, launch_validate_state(G ? d.G : nullptr, R ? d.R : nullptr, s->W, s->H, s->P, s->cap, s->status, s->stream));
  // host sources may be pinned: the copies must finish before the caller regains the buffers
  if (!src_on_device) CK(s, cudaStreamSynchronize(s->stream));
  s->t = 0;
  return CORAL_OK;
}

int coral_genome_table_load(coral_substrate* s, int32_t n, const float* genes, const float* dense,
                            int src_on_device) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (n < 1 || n > s->cap) return fail(s, CORAL_E_INVALID, "n must be in [1, genome_capacity]");
  if (!genes && !dense) return fail(s, CORAL_E_INVALID, "need CPPN genes or dense nets");
  const cudaMemcpyKind k = kind_in(src_on_device);
  CK(s, cudaMemsetAsync(s->g.genes, 0, sizeof(float) * kGenes * (size_t)s->cap, s->stream));
  CK(s, cudaMemsetAsync(s->g.parent, 0xFF, sizeof(int32_t) * (size_t)s->cap, s->stream));
  CK(s, cudaMemsetAsync(s->g.nets32, 0, sizeof(float) * s->g.net_stride * (size_t)s->cap, s->stream));
  CK(s, cudaMemsetAsync(s->g.nets16, 0, (size_t)s->g.blob_bytes * s->cap, s->stream));
  if (genes) {
    CK(s, cudaMemcpyAsync(s->g.genes, genes, sizeof(float) * kGenes * (size_t)n, k, s->stream));
    if (!src_on_device) CK(s, cudaStreamSynchronize(s->stream));
    s->has_cppn = true;
  } else {
    const size_t bytes = sizeof(float) * coral_net_floats(s->p.hidden) * (size_t)n;
    float* tmp = nullptr;
    CK(s, cudaMallocAsync((void**)&tmp, bytes, s->stream));
    cudaError_t e = cudaMemcpyAsync(tmp, dense, bytes, k, s->stream);
    if (e == cudaSuccess) e = launch_dense_pack(s->g, tmp, n, s->stream);
    if (e == cudaSuccess) e = launch_bf16_pack(s->g, nullptr, nullptr, n, s->stream);
    cudaFreeAsync(tmp, s->stream);
    if (e == cudaSuccess && !src_on_device) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "dense net load");
    s->has_cppn = false;
  }
  s->genomes_loaded = true;
  return CORAL_OK;
}

int coral_cppn_generate_weights(coral_substrate* s, const int32_t* slots, int32_t n) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (!s->has_cppn) return fail(s, CORAL_E_STATE, "no CPPN genes loaded");
  if (n < 0 || n > s->cap) return fail(s, CORAL_E_INVALID, "n must be in [0, genome_capacity]");
  if (n == 0) return CORAL_OK;
  int32_t* dslots = nullptr;
  if (slots) {
    for (int i = 0; i < n; ++i)
      if (slots[i] < 0 || slots[i] >= s->cap) return fail(s, CORAL_E_INVALID, "slot id out of range");
    CK(s, cudaMemcpyAsync(s->newslots, slots, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s->stream));
    dslots = s->newslots;
  }
  CK(s, launch_cppn_generate(s->g, dslots, nullptr, n, s->stream));
  CK(s, launch_bf16_pack(s->g, dslots, nullptr, n, s->stream));
  if (slots) CK(s, cudaStreamSynchronize(s->stream));   // the host slot list is consumed
  return CORAL_OK;
}

}  // extern "C"

namespace {

// Radiation arguments of the step that just ended (index t), over the substrate's own cells.
RadiationArgs radiation_args(coral_substrate* s, long long t) {
  RadiationArgs r = {};
  r.W = s->W;
  r.H = s->H;
  r.N = s->N;
  r.P = s->P;
  r.G = s->st[s->cur].G;
  r.j0 = s->slab ? (long long)s->row_lo * s->P : 0;
  r.n_own = s->slab ? (long long)(s->row_hi - s->row_lo) * s->P : s->N;
  r.gid0 = s->slab ? s->gid0 : 0;
  r.g = s->g;
  r.thr_mut = hit_threshold(s->p.p_mut);
  r.thr_merge = hit_threshold(s->p.p_merge);
  r.sigma = s->p.sigma_mut;
  r.world = s->p.world;
  r.seed = s->p.seed;
  r.step = (uint32_t)t;
  r.count = s->count;
  r.hitmask = s->hitmask;
  r.blockcnt = s->blockcnt;
  r.blockoff = s->blockoff;
  r.hits = s->hits;
  r.hitbits = s->hitbits;
  r.max_hits = s->cap;
  r.freelist = s->freelist;
  r.newslots = s->newslots;
  r.counters = s->counters;
  r.rec = s->ring + (t % kRing);
  return r;
}

// Enqueues one step; ev (4 events or NULL) is recorded before pass 1, after pass 1, after
// pass 2 and after the totals / radiation.
int enqueue_step(coral_substrate* s, cudaEvent_t* ev) {
  StepArgs a = step_args(s);
  if (ev) CK(s, cudaEventRecord(ev[0], s->stream));
  if (s->p.path == CORAL_NET_BF16_GROUPED)
    CK(s, launch_pass1_bf16(a, s->tmap_ok ? &s->tmap[s->cur] : nullptr, s->stream, s->grid1));
  else
    CK(s, launch_pass1_fp32(a, s->stream, s->grid1));
  if (ev) CK(s, cudaEventRecord(ev[1], s->stream));
  CK(s, launch_pass2(a, s->stream, s->grid2));
  if (ev) CK(s, cudaEventRecord(ev[2], s->stream));
  CK(s, launch_stats(a, s->grid1, s->grid2, s->t, s->ring, s->stream));
  s->cur ^= 1;
  if (!s->slab && s->p.radiation_every > 0 && (s->t + 1) % s->p.radiation_every == 0)
    CK(s, launch_radiation(radiation_args(s, s->t), s->stream));
  if (ev) CK(s, cudaEventRecord(ev[3], s->stream));
  ++s->t;
  return CORAL_OK;
}

int step_preconditions(coral_substrate* s, int32_t n_steps) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (n_steps < 0) return fail(s, CORAL_E_INVALID, "n_steps must be >= 0");
  if (!s->genomes_loaded) return fail(s, CORAL_E_STATE, "no genome table loaded");
  if (s->p.radiation_every > 0 && !s->has_cppn)
    return fail(s, CORAL_E_STATE, "radiation needs CPPN genomes (direct nets cannot mutate)");
  return CORAL_OK;
}

}  // namespace

extern "C" int coral_step(coral_substrate* s, int32_t n_steps) {
  int rc = step_preconditions(s, n_steps);
  if (rc) return rc;
  for (int i = 0; i < n_steps; ++i)
    if ((rc = enqueue_step(s, nullptr)) != CORAL_OK) return rc;
  return CORAL_OK;
}

namespace {

int jobs_setup(coral_substrate* s) {
  JobPipe& jp = s->jobs;
  if (jp.ready) return CORAL_OK;
  const size_t bytes = (size_t)kStateBytesPerCell * (size_t)s->NL;
  for (int b = 0; b < 2; ++b) {
    CK(s, dalloc(s, &jp.in[b], bytes));
    CK(s, dalloc(s, &jp.out[b], bytes));
  }
  CK(s, cudaStreamCreateWithFlags(&jp.s_in, cudaStreamNonBlocking));
  CK(s, cudaStreamCreateWithFlags(&jp.s_out, cudaStreamNonBlocking));
  for (int b = 0; b < 2; ++b)
    for (cudaEvent_t* ev : {&jp.h2d_done[b], &jp.in_free[b], &jp.out_ready[b], &jp.out_free[b]})
      CK(s, cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
  jp.ready = true;
  return CORAL_OK;
}

// Enqueues job k of coral_step_jobs (see the header): copy in on s_in, load + validate +
// steps + copy to the output staging buffer on the substrate's stream, copy out on s_out.
int enqueue_job(coral_substrate* s, int k, const void* src, void* dst, int32_t n_steps, int64_t t0) {
  JobPipe& jp = s->jobs;
  const int b = k & 1;
  const long long N = s->NL;                        // packed cells of a job's state
  const size_t bytes = (size_t)kStateBytesPerCell * (size_t)N;
  const size_t W = (size_t)s->W, H = (size_t)s->H, P = (size_t)s->P;
  if (k >= 2) CK(s, cudaStreamWaitEvent(jp.s_in, jp.in_free[b], 0));
  CK(s, cudaMemcpyAsync(jp.in[b], src, bytes, cudaMemcpyHostToDevice, jp.s_in));
  CK(s, cudaEventRecord(jp.h2d_done[b], jp.s_in));
  CK(s, cudaStreamWaitEvent(s->stream, jp.h2d_done[b], 0));
  {
    const Planes& d = s->st[s->cur];
    // the six float planes are 6H packed rows in, 6H pitched rows on the device
    CK(s, cudaMemcpy2DAsync(d.E, 4 * P, jp.in[b], 4 * W, 4 * W, 6 * H, cudaMemcpyDeviceToDevice, s->stream));
    CK(s, cudaMemcpy2DAsync(d.G, 4 * P, jp.in[b] + 24 * N, 4 * W, 4 * W, H, cudaMemcpyDeviceToDevice, s->stream));
    CK(s, cudaMemcpy2DAsync(d.R, P, jp.in[b] + 28 * N, W, W, H, cudaMemcpyDeviceToDevice, s->stream));
    CK(s, cudaEventRecord(jp.in_free[b], s->stream));
    CK(s, launch_validate_state(d.G, d.R, s->W, s->H, s->P, s->cap, s->status, s->stream));
  }
  s->t = t0;
  for (int i = 0; i < n_steps; ++i) {
    const int rc = enqueue_step(s, nullptr);
    if (rc != CORAL_OK) return rc;
  }
  if (k >= 2) CK(s, cudaStreamWaitEvent(s->stream, jp.out_free[b], 0));
  {
    const Planes& d = s->st[s->cur];
    CK(s, cudaMemcpy2DAsync(jp.out[b], 4 * W, d.E, 4 * P, 4 * W, 6 * H, cudaMemcpyDeviceToDevice, s->stream));
    CK(s, cudaMemcpy2DAsync(jp.out[b] + 24 * N, 4 * W, d.G, 4 * P, 4 * W, H, cudaMemcpyDeviceToDevice, s->stream));
    CK(s, cudaMemcpy2DAsync(jp.out[b] + 28 * N, W, d.R, P, W, H, cudaMemcpyDeviceToDevice, s->stream));
  }
  CK(s, cudaEventRecord(jp.out_ready[b], s->stream));
  CK(s, cudaStreamWaitEvent(jp.s_out, jp.out_ready[b], 0));
  CK(s, cudaMemcpyAsync(dst, jp.out[b], bytes, cudaMemcpyDeviceToHost, jp.s_out));
  CK(s, cudaEventRecord(jp.out_free[b], jp.s_out));
  return CORAL_OK;
}

}  // namespace

extern "C" int coral_step_jobs(coral_substrate* s, int32_t n_jobs, const void* const* host_in,
                               void* const* host_out, int32_t n_steps, int64_t t0) {
  int rc = step_preconditions(s, n_steps);
  if (rc) return rc;
  if (n_jobs < 0 || t0 < 0) return fail(s, CORAL_E_INVALID, "n_jobs and t0 must be >= 0");
  if (n_jobs == 0) return CORAL_OK;
  if (!host_in || !host_out) return fail(s, CORAL_E_INVALID, "NULL job buffer array");
  for (int k = 0; k < n_jobs; ++k)
    if (!host_in[k] || !host_out[k]) return fail(s, CORAL_E_INVALID, "NULL job buffer");
  if ((rc = jobs_setup(s)) != CORAL_OK) return rc;
  for (int k = 0; k < n_jobs && rc == CORAL_OK; ++k) rc = enqueue_job(s, k, host_in[k], host_out[k], n_steps, t0);
  // the caller regains its buffers only when no copy is in flight, also after an error
  cudaStreamSynchronize(s->jobs.s_in);
  cudaStreamSynchronize(s->stream);
  cudaStreamSynchronize(s->jobs.s_out);
  if (rc != CORAL_OK) return rc;
  return check_status(s);
}

extern "C" int coral_step_timed(coral_substrate* s, int32_t n_steps, float* step_ms, float* stage_ms) {
  int rc = step_preconditions(s, n_steps);
  if (rc) return rc;
  std::vector<cudaEvent_t> ev;
  try {
    ev.resize(4 * (size_t)n_steps);
  } catch (...) {
    return fail(s, CORAL_E_OOM, "host allocation failed");
  }
  int made = 0;
  for (; made < 4 * n_steps; ++made)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
  if (made < 4 * n_steps) rc = fail(s, CORAL_E_CUDA, "cudaEventCreate failed");
  for (int i = 0; rc == CORAL_OK && i < n_steps; ++i) rc = enqueue_step(s, &ev[4 * i]);
  if (rc == CORAL_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = fail(s, CORAL_E_CUDA, "sync failed");
  for (int i = 0; rc == CORAL_OK && i < n_steps; ++i) {
    float t0 = 0, t1 = 0, t2 = 0;
    cudaEventElapsedTime(&t0, ev[4 * i], ev[4 * i + 1]);
    cudaEventElapsedTime(&t1, ev[4 * i + 1], ev[4 * i + 2]);
    cudaEventElapsedTime(&t2, ev[4 * i + 2], ev[4 * i + 3]);
    if (step_ms) cudaEventElapsedTime(&step_ms[i], ev[4 * i], ev[4 * i + 3]);
    if (stage_ms) {
      stage_ms[3 * i] = t0;
      stage_ms[3 * i + 1] = t1;
      stage_ms[3 * i + 2] = t2;
    }
  }
  for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
  return rc;
}

extern "C" {

int coral_read_channels(coral_substrate* s, uint32_t mask, void* dst, size_t dst_bytes, int on_device) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (!dst) return fail(s, CORAL_E_INVALID, "dst is NULL");
  const long long N = s->NL, NP = s->N;
  size_t need = 0;
  for (int b = 0; b < 8; ++b)
    if (mask & (1u << b)) need += (b == 7) ? (size_t)N : (size_t)N * 4;
  if (dst_bytes < need) return fail(s, CORAL_E_CAPACITY, "dst_bytes too small for the selected planes");
  const Planes& d = s->st[s->cur];
  const cudaMemcpyKind k = kind_out(on_device);
  char* o = static_cast<char*>(dst);
  const void* src[8] = {d.E, d.I, d.C, d.C + NP, d.C + 2 * NP, d.C + 3 * NP, d.G, d.R};
  const size_t W = (size_t)s->W, H = (size_t)s->H, P = (size_t)s->P;
  const bool host_pageable = !on_device && pageable(dst);
  const bool stage = host_pageable && P != W;
  for (int b = 0; b < 8; ++b) {
    if (!(mask & (1u << b))) continue;
    const size_t es = (b == 7) ? 1 : 4;             // pitched rows on the device, packed rows out
    if (stage) {
      CK(s, pitched_to_host(s, o, src[b], es));
    } else if (host_pageable) {                     // rows unpadded: one contiguous copy
      CK(s, cudaMemcpyAsync(o, src[b], es * W * H, k, s->stream));
    } else {
      CK(s, cudaMemcpy2DAsync(o, es * W, src[b], es * P, es * W, H, k, s->stream));
    }
    o += es * (size_t)N;
  }
  if (stage) CK(s, restore_spare_padding(s));
  return check_status(s);
}

int coral_read_stats(coral_substrate* s, int64_t step_from, int32_t n, coral_stats* out) {
  if (!s || !out) return fail(s, CORAL_E_INVALID, "NULL argument");
  if (n < 0 || step_from < 0 || step_from + n > s->t || step_from < s->t - kRing)
    return fail(s, CORAL_E_INVALID, "requested steps are not in the stats ring");
  int rc = check_status(s);
  if (rc) return rc;
  for (int i = 0; i < n; ++i)
    CK(s, cudaMemcpy(out + i, s->ring + ((step_from + i) % kRing), sizeof(coral_stats), cudaMemcpyDeviceToHost));
  return CORAL_OK;
}

int coral_read_perm(coral_substrate* s, int32_t* dst_counts, int32_t* dst_perm) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  const long long N = s->NL;
  const int nblk = bucket_blocks(N);
  if (!s->sort_buf) {
    const size_t words = 6 * (size_t)N + 256 * (size_t)nblk + (size_t)s->cap + 256 + 64;
    CK(s, dalloc(s, &s->sort_buf, words));
  }
  // the torus cells' G packed (cell id y * W + x), then sorted; unpadded rows are packed already
  const int32_t* keys = s->st[s->cur].G;
  if (s->P != s->W) {
    int32_t* packed = s->sort_buf + 5 * (size_t)N + 256 * (size_t)nblk + (size_t)s->cap + 256;
    CK(s, cudaMemcpy2DAsync(packed, 4 * (size_t)s->W, s->st[s->cur].G, 4 * (size_t)s->P, 4 * (size_t)s->W,
                            (size_t)s->H, cudaMemcpyDeviceToDevice, s->stream));
    keys = packed;
  }
  SortArgs a = {};
  a.keys_in = keys;
  a.N = N;
  a.capacity = s->cap;
  a.k0 = s->sort_buf;
  a.v0 = a.k0 + N;
  a.k1 = a.v0 + N;
  a.v1 = a.k1 + N;
  a.perm = a.v1 + N;
  a.hist = a.perm + N;
  a.count = a.hist + 256 * (size_t)nblk;
  a.totals = a.count + s->cap;
  CK(s, launch_bucket(a, s->stream));
  if (dst_counts) CK(s, cudaMemcpyAsync(dst_counts, a.count, sizeof(int32_t) * s->cap, cudaMemcpyDeviceToHost, s->stream));
  if (dst_perm) CK(s, cudaMemcpyAsync(dst_perm, a.perm, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

int coral_read_genomes(coral_substrate* s, float* genes, int32_t* parent) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (genes) CK(s, cudaMemcpyAsync(genes, s->g.genes, sizeof(float) * kGenes * (size_t)s->cap, cudaMemcpyDeviceToHost, s->stream));
  if (parent) CK(s, cudaMemcpyAsync(parent, s->g.parent, sizeof(int32_t) * (size_t)s->cap, cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

int coral_read_weights(coral_substrate* s, int32_t slot, float* dst, size_t dst_floats) {
  if (!s || !dst) return fail(s, CORAL_E_INVALID, "NULL argument");
  if (slot < 0 || slot >= s->cap) return fail(s, CORAL_E_INVALID, "slot out of range");
  const int nf = coral_net_floats(s->p.hidden);
  if (dst_floats < (size_t)nf) return fail(s, CORAL_E_CAPACITY, "dst too small");
  float* tmp = nullptr;
  CK(s, cudaMallocAsync((void**)&tmp, sizeof(float) * nf, s->stream));
  cudaError_t e = launch_read_dense(s->g, slot, tmp, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, sizeof(float) * nf, cudaMemcpyDeviceToHost, s->stream);
  cudaFreeAsync(tmp, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "read weights");
  return check_status(s);
}

int coral_genome_distances(coral_substrate* s, const int32_t* slots, int32_t n, float* out) {
  if (!s || !slots || !out) return fail(s, CORAL_E_INVALID, "NULL argument");
  if (n < 1 || n > 4096) return fail(s, CORAL_E_INVALID, "n must be in [1, 4096]");
  for (int i = 0; i < n; ++i)
    if (slots[i] < 0 || slots[i] >= s->cap) return fail(s, CORAL_E_INVALID, "slot out of range");
  const size_t pairs = (size_t)n * n;
  void* tmp = nullptr;
  CK(s, cudaMallocAsync(&tmp, sizeof(int32_t) * n + sizeof(float) * pairs + 256, s->stream));
  int32_t* dslots = static_cast<int32_t*>(tmp);
  float* dout = reinterpret_cast<float*>(static_cast<char*>(tmp) + ((sizeof(int32_t) * n + 255) & ~(size_t)255));
  cudaError_t e = cudaMemcpyAsync(dslots, slots, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = launch_genome_distances(s->g.genes, dslots, n, dout, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(float) * pairs, cudaMemcpyDeviceToHost, s->stream);
  cudaFreeAsync(tmp, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "genome distances");
  return check_status(s);
}

int coral_set_step(coral_substrate* s, int64_t t) {
  if (!s || t < 0) return fail(s, CORAL_E_INVALID, "bad argument");
  s->t = t;
  return CORAL_OK;
}

int coral_get_step(const coral_substrate* s, int64_t* t) {
  if (!s || !t) return fail(nullptr, CORAL_E_INVALID, "NULL argument");
  *t = s->t;
  return CORAL_OK;
}

int coral_launch_config(const coral_substrate* s, int32_t* g1, int32_t* g2, int32_t* sms) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (g1) *g1 = s->grid1;
  if (g2) *g2 = s->grid2;
  if (sms) *sms = s->sms;
  return CORAL_OK;
}

int coral_selftest_wait_timeout(void* cuda_stream, int32_t wait_us, int32_t* status_out) {
  if (!status_out || wait_us < 1 || wait_us > 1000000) return fail(nullptr, CORAL_E_INVALID, "bad arguments");
  int dev = 0, major = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, CORAL_E_CUDA, "cudaGetDevice failed");
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (major != 10) return fail(nullptr, CORAL_E_INVALID, "needs an sm_100-family GPU (tensor memory)");
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (khz <= 0) khz = 2000000;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_selftest_wait((long long)khz * 1000LL / 1000000LL * wait_us, d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, d, sizeof(int), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail(nullptr, CORAL_E_CUDA, cudaGetErrorString(e));
  *status_out = v;
  return CORAL_OK;
}

int coral_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int32_t n) {
  if (!ctr || !key || !out) return fail(nullptr, CORAL_E_INVALID, "NULL argument");
  if (n < 1 || n > 65536) return fail(nullptr, CORAL_E_INVALID, "n must be in [1, 65536]");
  void* d = nullptr;
  const size_t b_ctr = 16 * (size_t)n, b_key = 8 * (size_t)n;
  cudaError_t e = cudaMalloc(&d, 2 * b_ctr + b_key);
  uint32_t* dc = static_cast<uint32_t*>(d);
  uint32_t* dout = dc + 4 * (size_t)n;
  uint32_t* dk = dout + 4 * (size_t)n;
  if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, b_ctr, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dk, key, b_key, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_philox(dc, dk, dout, n, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, b_ctr, cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail(nullptr, e == cudaErrorMemoryAllocation ? CORAL_E_OOM : CORAL_E_CUDA,
                                    std::string("philox: ") + cudaGetErrorString(e));
  return CORAL_OK;
}

int coral_measure_sfu_rate(void* cuda_stream, double* evals_per_s) {
  if (!evals_per_s) return fail(nullptr, CORAL_E_INVALID, "NULL argument");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(nullptr, CORAL_E_CUDA, "device query failed");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int blocks = 8 * sms, iters = 4096;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.0f;
  cudaError_t e = cudaMalloc(&sink, sizeof(float) * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = launch_sfu_probe(blocks, iters, sink, st);              // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = launch_sfu_probe(blocks, iters, sink, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return fail(nullptr, CORAL_E_CUDA, std::string("sfu probe: ") + cudaGetErrorString(e));
  *evals_per_s = (double)blocks * 256.0 * 8.0 * iters / (ms * 1e-3);
  return CORAL_OK;
}

int coral_slab_set(coral_substrate* s, int32_t row_lo, int32_t row_hi, int64_t global_cell0) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (row_lo < 1 || row_hi <= row_lo || row_hi > s->H - 1 || global_cell0 < 0)
    return fail(s, CORAL_E_INVALID, "own rows must satisfy 1 <= row_lo < row_hi <= height - 1, global_cell0 >= 0");
  if (global_cell0 + (long long)(row_hi - row_lo) * s->W > (1LL << 32))
    return fail(s, CORAL_E_INVALID, "global cell ids must stay below 2^32");
  s->slab = true;
  s->row_lo = row_lo;
  s->row_hi = row_hi;
  s->gid0 = global_cell0;
  return CORAL_OK;
}

int coral_copy_rows(coral_substrate* dst, int32_t dst_row, coral_substrate* src, int32_t src_row, int32_t n_rows) {
  if (!dst || !src) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  if (dst->W != src->W) return fail(dst, CORAL_E_INVALID, "substrates of different widths");
  if (dst->device != src->device) return fail(dst, CORAL_E_INVALID, "substrates on different devices");
  if (n_rows < 0 || dst_row < 0 || src_row < 0 || dst_row + n_rows > dst->H || src_row + n_rows > src->H)
    return fail(dst, CORAL_E_INVALID, "row range outside a substrate");
  if (n_rows == 0) return CORAL_OK;
  if (dst == src && dst_row < src_row + n_rows && src_row < dst_row + n_rows)
    return fail(dst, CORAL_E_INVALID, "overlapping row ranges");
  // order: the copies after src's enqueued work; src's later work after the copies
  cudaEvent_t ev = nullptr;
  CK(dst, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, src->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(dst->stream, ev, 0);
  const Planes& d = dst->st[dst->cur];
  const Planes& q = src->st[src->cur];
  const size_t P = (size_t)dst->P, rows = (size_t)n_rows;   // whole pitched rows, padding included
  for (int p = 0; p < 6 && e == cudaSuccess; ++p)
    e = cudaMemcpyAsync(d.E + (size_t)p * dst->N + dst_row * P, q.E + (size_t)p * src->N + src_row * P,
                        sizeof(float) * rows * P, cudaMemcpyDeviceToDevice, dst->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.G + dst_row * P, q.G + src_row * P, sizeof(int32_t) * rows * P, cudaMemcpyDeviceToDevice,
                        dst->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.R + dst_row * P, q.R + src_row * P, rows * P, cudaMemcpyDeviceToDevice, dst->stream);
  if (e == cudaSuccess && src->stream != dst->stream) {
    e = cudaEventRecord(ev, dst->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(src->stream, ev, 0);
  }
  cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(dst, e, "copy rows");
  return CORAL_OK;
}

int coral_slab_totals(coral_substrate* s, double* out) {
  if (!s || !out) return fail(s, CORAL_E_INVALID, "NULL argument");
  if (!s->totals_buf) CK(s, dalloc(s, &s->totals_buf, 6 + 6 * 256));
  // whole pitched rows: the padding's floats are 0
  const long long j0 = s->slab ? (long long)s->row_lo * s->P : 0;
  const long long n = s->slab ? (long long)(s->row_hi - s->row_lo) * s->P : s->N;
  CK(s, launch_row_totals(s->st[s->cur].E, s->N, j0, n, s->totals_buf, s->stream));
  CK(s, cudaMemcpyAsync(out, s->totals_buf, 6 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

int coral_slab_radiation_scan(coral_substrate* s, uint8_t* live, int32_t* hits, int32_t max_hits, int32_t* counts) {
  if (!s || !live || !counts || (max_hits > 0 && !hits)) return fail(s, CORAL_E_INVALID, "NULL argument");
  if (!s->slab) return fail(s, CORAL_E_STATE, "not a slab (coral_slab_set)");
  if (!s->has_cppn) return fail(s, CORAL_E_STATE, "radiation needs CPPN genomes");
  if (s->t < 1) return fail(s, CORAL_E_STATE, "no step has run yet");
  CK(s, launch_radiation_scan(radiation_args(s, s->t - 1), s->stream));
  int c[8];
  CK(s, cudaMemcpyAsync(c, s->counters, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
  std::vector<int32_t> flags(s->cap);
  CK(s, cudaMemcpyAsync(flags.data(), s->count, sizeof(int32_t) * s->cap, cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  const int listed = std::min(std::min(c[0], s->cap), std::max(max_hits, 0));
  std::vector<int4> h(listed > 0 ? listed : 1);
  std::vector<uint32_t> bits(listed > 0 ? listed : 1);
  if (listed > 0) {
    CK(s, cudaMemcpy(h.data(), s->hits, sizeof(int4) * listed, cudaMemcpyDeviceToHost));
    CK(s, cudaMemcpy(bits.data(), s->hitbits, sizeof(uint32_t) * listed, cudaMemcpyDeviceToHost));
  }
  for (int i = 0; i < listed; ++i) {
    int32_t* o = hits + 5 * (size_t)i;
    o[0] = h[i].x;
    o[1] = h[i].y;
    o[2] = h[i].z;
    o[3] = h[i].w;
    o[4] = (int32_t)bits[i];
  }
  for (int k = 0; k < s->cap; ++k) live[k] = flags[k] ? 1 : 0;
  counts[0] = c[0];
  counts[1] = c[3];
  counts[2] = c[4];
  counts[3] = listed;
  return check_status(s);
}

int coral_slab_radiation_apply(coral_substrate* s, const uint8_t* live_all, const int32_t* hits_all,
                               int32_t n_listed, const int32_t* counts_all) {
  if (!s || !live_all || !counts_all || (n_listed > 0 && !hits_all)) return fail(s, CORAL_E_INVALID, "NULL argument");
  if (!s->slab) return fail(s, CORAL_E_STATE, "not a slab (coral_slab_set)");
  if (s->t < 1) return fail(s, CORAL_E_STATE, "no step has run yet");
  if (n_listed < 0 || counts_all[0] < n_listed || counts_all[0] < 0)
    return fail(s, CORAL_E_INVALID, "hit counts inconsistent with the list");
  const int up = std::min(n_listed, s->cap);
  std::vector<int32_t> flags(s->cap);
  for (int k = 0; k < s->cap; ++k) flags[k] = live_all[k] ? 1 : 0;
  std::vector<int4> h(up > 0 ? up : 1);
  std::vector<uint32_t> bits(up > 0 ? up : 1);
  for (int i = 0; i < up; ++i) {
    const int32_t* q = hits_all + 5 * (size_t)i;
    if (q[1] < 0 || q[1] >= s->cap || q[2] < -1 || q[2] >= s->cap)
      return fail(s, CORAL_E_INVALID, "hit with a genome slot out of range");
    h[i] = make_int4(q[0], q[1], q[2], q[3]);
    bits[i] = (uint32_t)q[4];
  }
  int c[8] = {counts_all[0], 0, 0, counts_all[1], counts_all[2], 0, 0, 0};
  CK(s, cudaMemcpyAsync(s->count, flags.data(), sizeof(int32_t) * s->cap, cudaMemcpyHostToDevice, s->stream));
  if (up > 0) {
    CK(s, cudaMemcpyAsync(s->hits, h.data(), sizeof(int4) * up, cudaMemcpyHostToDevice, s->stream));
    CK(s, cudaMemcpyAsync(s->hitbits, bits.data(), sizeof(uint32_t) * up, cudaMemcpyHostToDevice, s->stream));
  }
  CK(s, cudaMemcpyAsync(s->counters, c, sizeof(c), cudaMemcpyHostToDevice, s->stream));
  RadiationArgs r = radiation_args(s, s->t - 1);
  r.max_hits = up;                       // only the listed hits can be assigned
  CK(s, launch_radiation_apply(r, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));   // the host vectors above are released on return
  return check_status(s);
}

int coral_sync(coral_substrate* s) {
  if (!s) return fail(nullptr, CORAL_E_INVALID, "NULL substrate");
  return check_status(s);
}

const char* coral_last_error(const coral_substrate* s) { return s ? s->err.c_str() : g_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batched stepping
// ---------------------------------------------------------------------------------------------
// Batched launches ask for this many times the CTAs per SM of their launch shape (see partition;
// on the 256-world batch 4, 8, 16 and 32 gave 11.7, 11.6, 11.2 and 11.0 ms per step, and 32
// 10.7 against 16's 10.9 ms once the batch had TMA halos).
constexpr int kOversubscribe = 32;

struct coral_batch {
  std::vector<coral_substrate*> worlds;
  cudaStream_t stream = nullptr;
  int sms = 0;
  int n = 0;
  void* dmem = nullptr;          // one device block for the tables
  StepArgs* d_args = nullptr;    // [2][n]
  int* d_part = nullptr;         // cta_world1 | first1 | ctas1 | cta_world2 | first2 | ctas2
  coral_stats** d_rings = nullptr;
  long long* d_steps = nullptr;
  CUtensorMap* d_tmaps = nullptr;  // [2][n]
  int* d_tma_ok = nullptr;         // [n]
  int cps1 = 6, cps2 = 3;        // CTAs per SM of pass 1 / pass 2
  int fma_cutoff = 0;            // pass 1's FMA small-genome cutoff for every world of the batch
  int grid1 = 0, grid2 = 0;
  int max_grid = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaEvent_t ev = nullptr;
  long long steps_done = 0;      // parity of the batch (world w's current buffer = cur0[w] ^ parity)
  std::vector<int> cur0;
  std::string err;
};

namespace {

int bfail(coral_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  g_err = m;
  return code;
}

#define BCK(b, call)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return bfail((b), e_ == cudaErrorMemoryAllocation ? CORAL_E_OOM : CORAL_E_CUDA, \
                                        std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Splits about `grid` CTAs among the worlds so that the largest work of one CTA is as small as
// possible: world i gets max(1, ceil(work[i] / T)) CTAs (at most kMaxPartials) for the smallest
// T whose total is at most max(grid, n). The launches ask for several times the CTAs that fit on the GPU at once
// (kOversubscribe), so the block scheduler fills the slots that CTAs of small worlds leave
// early, and the kernel ends when the average SM does. Fills cta_world [total], first [n],
// ctas [n]; returns the total.
int partition(const std::vector<long long>& work, int grid, std::vector<int>& cta_world, std::vector<int>& first,
              std::vector<int>& ctas) {
  const int n = (int)work.size();
  if (grid < n) grid = n;
  long long hi = 1;
  for (long long w : work) hi = std::max(hi, w);
  auto count = [&](long long T) {
    long long c = 0;
    for (long long w : work) c += std::max(1LL, (w + T - 1) / T);
    return c;
  };
  long long lo = 1;                                   // count(hi) = n <= grid
  while (lo < hi) {
    const long long mid = lo + (hi - lo) / 2;
    if (count(mid) <= grid) hi = mid;
    else lo = mid + 1;
  }
  ctas.assign(n, 1);
  for (int i = 0; i < n; ++i)   // one world's partial sums have kMaxPartials slots
    ctas[i] = (int)std::min<long long>(kMaxPartials, std::max(1LL, (work[i] + hi - 1) / hi));
  first.assign(n, 0);
  cta_world.clear();
  for (int i = 0; i < n; ++i) {
    first[i] = (int)cta_world.size();
    for (int k = 0; k < ctas[i]; ++k) cta_world.push_back(i);
  }
  return (int)cta_world.size();
}

BatchTable table_of(const coral_batch* b) {
  BatchTable t;
  t.n = b->n;
  t.args = b->d_args;
  const int g = b->max_grid;
  t.cta_world1 = b->d_part;
  t.world_first1 = b->d_part + g;
  t.world_ctas1 = b->d_part + g + b->n;
  t.cta_world2 = b->d_part + g + 2 * b->n;
  t.world_first2 = b->d_part + 2 * g + 2 * b->n;
  t.world_ctas2 = b->d_part + 2 * g + 3 * b->n;
  t.rings = b->d_rings;
  t.steps = b->d_steps;
  t.tmaps = b->d_tmaps;
  t.tma_ok = b->d_tma_ok;
  return t;
}

// Launch shapes for the current cps1 / cps2, partition tables and the two graphs.
int batch_configure(coral_batch* b) {
  std::vector<long long> tiles, cells;
  for (coral_substrate* s : b->worlds) {
    tiles.push_back(pass1_bf16_tiles(s->W, s->H));
    cells.push_back(s->N);
  }
  std::vector<int> cw1, f1, c1, cw2, f2, c2;
  b->grid1 = partition(tiles, b->cps1 * b->sms * kOversubscribe, cw1, f1, c1);
  b->grid2 = partition(cells, b->cps2 * b->sms * kOversubscribe, cw2, f2, c2);
  if (b->grid1 > b->max_grid || b->grid2 > b->max_grid) return bfail(b, CORAL_E_INVALID, "launch shape too large");
  for (int i = 0; i < b->n; ++i)
    if (c1[i] > kMaxPartials || c2[i] > kMaxPartials) return bfail(b, CORAL_E_INVALID, "too many CTAs for one world");
  std::vector<int> part(4 * (size_t)b->max_grid + 6 * (size_t)b->n, 0);
  const int g = b->max_grid;
  std::copy(cw1.begin(), cw1.end(), part.begin());
  std::copy(f1.begin(), f1.end(), part.begin() + g);
  std::copy(c1.begin(), c1.end(), part.begin() + g + b->n);
  std::copy(cw2.begin(), cw2.end(), part.begin() + g + 2 * b->n);
  std::copy(f2.begin(), f2.end(), part.begin() + 2 * g + 2 * b->n);
  std::copy(c2.begin(), c2.end(), part.begin() + 2 * g + 3 * b->n);
  BCK(b, cudaMemcpyAsync(b->d_part, part.data(), sizeof(int) * (2 * (size_t)g + 4 * (size_t)b->n), cudaMemcpyHostToDevice,
                         b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  BCK(b, prepare_pass1_bf16_batch());
  const BatchTable t = table_of(b);
  for (int p = 0; p < 2; ++p) {
    if (b->graph[p]) {
      cudaGraphExecDestroy(b->graph[p]);
      b->graph[p] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_pass1_bf16_batch(t, p, b->grid1, b->worlds[0]->p.hidden, b->fma_cutoff > 0, b->stream);
    if (e == cudaSuccess) e = launch_pass2_batch(t, p, b->grid2, b->stream);
    if (e == cudaSuccess) e = launch_stats_batch(t, b->stream);
    const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return bfail(b, CORAL_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->graph[p], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, CORAL_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  return CORAL_OK;
}

// Orders the batch stream after the worlds' streams, refreshes the device step indices.
int batch_enter(coral_batch* b) {
  for (coral_substrate* s : b->worlds) {
    BCK(b, cudaEventRecord(b->ev, s->stream));
    BCK(b, cudaStreamWaitEvent(b->stream, b->ev, 0));
  }
  std::vector<long long> t(b->n);
  for (int i = 0; i < b->n; ++i) t[i] = b->worlds[i]->t;
  BCK(b, cudaMemcpyAsync(b->d_steps, t.data(), sizeof(long long) * b->n, cudaMemcpyHostToDevice, b->stream));
  return CORAL_OK;
}

// Orders the worlds' streams after the batch stream; advances the worlds' bookkeeping.
int batch_leave(coral_batch* b, int n_steps) {
  BCK(b, cudaEventRecord(b->ev, b->stream));
  for (coral_substrate* s : b->worlds) {
    BCK(b, cudaStreamWaitEvent(s->stream, b->ev, 0));
    s->cur ^= (n_steps & 1);
    s->t += n_steps;
  }
  b->steps_done += n_steps;
  return CORAL_OK;
}

// The worlds' step arguments and TMA descriptors for both parities relative to their current
// buffers.
int batch_upload_args(coral_batch* b) {
  std::vector<StepArgs> args(2 * (size_t)b->n);
  std::vector<CUtensorMap> maps(2 * (size_t)b->n);
  std::vector<int> ok(b->n, 0);
  for (int p = 0; p < 2; ++p)
    for (int i = 0; i < b->n; ++i) {
      coral_substrate* s = b->worlds[i];
      const int save = s->cur;
      s->cur = save ^ p;
      StepArgs a = step_args(s);
      s->cur = save;
      a.step_dev = b->d_steps + i;
      a.fma_cutoff = b->fma_cutoff;
      args[(size_t)p * b->n + i] = a;
      if (s->tmap_ok) maps[(size_t)p * b->n + i] = s->tmap[save ^ p];
      else memset(&maps[(size_t)p * b->n + i], 0, sizeof(CUtensorMap));
      ok[i] = s->tmap_ok ? 1 : 0;
    }
  BCK(b, cudaMemcpyAsync(b->d_args, args.data(), sizeof(StepArgs) * args.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemcpyAsync(b->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemcpyAsync(b->d_tma_ok, ok.data(), sizeof(int) * ok.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  return CORAL_OK;
}

}  // namespace

extern "C" int coral_batch_create(coral_substrate* const* worlds, int32_t n, coral_batch** out) {
  if (!worlds || !out || n < 1) return bfail(nullptr, CORAL_E_INVALID, "bad arguments");
  *out = nullptr;
  coral_batch* b = nullptr;
  try {
    b = new coral_batch();
  } catch (...) {
    return bfail(nullptr, CORAL_E_OOM, "host allocation failed");
  }
  b->n = n;
  int rc = CORAL_OK;
  do {
    int dev = -1;
    for (int i = 0; i < n; ++i) {
      coral_substrate* s = worlds[i];
      if (!s) { rc = bfail(b, CORAL_E_INVALID, "NULL world"); break; }
      if (s->p.path != CORAL_NET_BF16_GROUPED) { rc = bfail(b, CORAL_E_INVALID, "batched worlds use the BF16 path"); break; }
      if (s->p.hidden != worlds[0]->p.hidden) { rc = bfail(b, CORAL_E_INVALID, "batched worlds share one hidden size"); break; }
      if (s->p.radiation_every > 0 && !s->has_cppn) {
        rc = bfail(b, CORAL_E_STATE, "radiation needs CPPN genomes (direct nets cannot mutate)");
        break;
      }
      if (s->slab) { rc = bfail(b, CORAL_E_INVALID, "row-slab substrates are not batched"); break; }
      if (!s->genomes_loaded) { rc = bfail(b, CORAL_E_STATE, "a world has no genome table"); break; }
      if (dev >= 0 && s->device != dev) { rc = bfail(b, CORAL_E_INVALID, "worlds on different devices"); break; }
      dev = s->device;
      b->worlds.push_back(s);
    }
    if (rc) break;
    b->sms = worlds[0]->sms;
    b->max_grid = std::max(6 * b->sms * kOversubscribe, n) + 8;
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    const size_t bytes = sizeof(StepArgs) * 2 * (size_t)n + 256 + sizeof(int) * (4 * (size_t)b->max_grid + 6 * (size_t)n) +
                         256 + sizeof(coral_stats*) * (size_t)n + 256 + sizeof(long long) * (size_t)n + 256 +
                         sizeof(CUtensorMap) * 2 * (size_t)n + 256 + sizeof(int) * (size_t)n + 256;
    if (e == cudaSuccess) e = cudaMalloc(&b->dmem, bytes);
    if (e != cudaSuccess) { rc = bfail(b, e == cudaErrorMemoryAllocation ? CORAL_E_OOM : CORAL_E_CUDA, cudaGetErrorString(e)); break; }
    char* p = static_cast<char*>(b->dmem);
    auto carve = [&](size_t nbytes) {
      char* q = p;
      p += (nbytes + 255) & ~(size_t)255;
      return q;
    };
    b->d_args = reinterpret_cast<StepArgs*>(carve(sizeof(StepArgs) * 2 * (size_t)n));
    b->d_part = reinterpret_cast<int*>(carve(sizeof(int) * (4 * (size_t)b->max_grid + 6 * (size_t)n)));
    b->d_rings = reinterpret_cast<coral_stats**>(carve(sizeof(coral_stats*) * (size_t)n));
    b->d_steps = reinterpret_cast<long long*>(carve(sizeof(long long) * (size_t)n));
    b->d_tmaps = reinterpret_cast<CUtensorMap*>(carve(sizeof(CUtensorMap) * 2 * (size_t)n));   // 256-byte aligned
    b->d_tma_ok = reinterpret_cast<int*>(carve(sizeof(int) * (size_t)n));
    std::vector<coral_stats*> rings(n);
    for (int i = 0; i < n; ++i) rings[i] = worlds[i]->ring;
    if ((e = cudaMemcpy(b->d_rings, rings.data(), sizeof(coral_stats*) * n, cudaMemcpyHostToDevice)) != cudaSuccess) {
      rc = bfail(b, CORAL_E_CUDA, cudaGetErrorString(e));
      break;
    }
    for (coral_substrate* s : b->worlds) cudaStreamSynchronize(s->stream);
    if ((rc = batch_upload_args(b)) != CORAL_OK) break;
    rc = batch_configure(b);
  } while (0);
  if (rc != CORAL_OK) {
    coral_batch_destroy(b);
    return rc;
  }
  *out = b;
  return CORAL_OK;
}

extern "C" int coral_batch_destroy(coral_batch* b) {
  if (!b) return CORAL_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int p = 0; p < 2; ++p)
    if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->dmem) cudaFree(b->dmem);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return CORAL_OK;
}

namespace {
// radiation = false: the graphs alone (the tuner's trial steps, which must leave the genome
// tables as they are).
int batch_run(coral_batch* b, int32_t n_steps, float* step_ms, bool radiation = true) {
  if (!b) return bfail(nullptr, CORAL_E_INVALID, "NULL batch");
  if (n_steps < 0) return bfail(b, CORAL_E_INVALID, "n_steps must be >= 0");
  if (n_steps == 0) return CORAL_OK;
  int rc = batch_upload_args(b);          // worlds may have been reloaded or stepped alone
  if (rc) return rc;
  if ((rc = batch_enter(b)) != CORAL_OK) return rc;
  std::vector<cudaEvent_t> ev;
  if (step_ms) {
    ev.resize(n_steps + 1);
    for (auto& e : ev) BCK(b, cudaEventCreate(&e));
    BCK(b, cudaEventRecord(ev[0], b->stream));
  }
  for (int i = 0; i < n_steps; ++i) {
    BCK(b, cudaGraphLaunch(b->graph[i & 1], b->stream));
    // radiation of the worlds whose step t = t0 + i ends an epoch: on the post-step state
    // (buffer cur ^ ((i + 1) & 1)), on the batch stream before the next step's graph
    for (coral_substrate* s : b->worlds) {
      const long long t = s->t + i;
      if (!radiation || s->p.radiation_every <= 0 || (t + 1) % s->p.radiation_every != 0) continue;
      const int save = s->cur;
      s->cur = save ^ ((i + 1) & 1);
      const RadiationArgs r = radiation_args(s, t);
      s->cur = save;
      BCK(b, launch_radiation(r, b->stream));
    }
    if (step_ms) BCK(b, cudaEventRecord(ev[i + 1], b->stream));
  }
  if ((rc = batch_leave(b, n_steps)) != CORAL_OK) return rc;
  if (step_ms) {
    BCK(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < n_steps; ++i) cudaEventElapsedTime(&step_ms[i], ev[i], ev[i + 1]);
    for (auto& e : ev) cudaEventDestroy(e);
  }
  return CORAL_OK;
}
}  // namespace

extern "C" int coral_batch_step(coral_batch* b, int32_t n_steps) { return batch_run(b, n_steps, nullptr); }

extern "C" int coral_batch_set_fma_cutoff(coral_batch* b, int32_t cells) {
  if (!b) return bfail(nullptr, CORAL_E_INVALID, "NULL batch");
  if (cells < 0 || cells > kFmaCutoffMax) return bfail(b, CORAL_E_INVALID, "cells must be in [0, 128]");
  const int old = b->fma_cutoff;
  b->fma_cutoff = cells;
  const int rc = batch_configure(b);                  // the graphs launch the matching kernel
  if (rc != CORAL_OK) b->fma_cutoff = old;
  return rc;
}

extern "C" int coral_batch_step_timed(coral_batch* b, int32_t n_steps, float* step_ms) {
  if (!step_ms) return bfail(b, CORAL_E_INVALID, "step_ms is NULL");
  return batch_run(b, n_steps, step_ms);
}

extern "C" int coral_batch_tune(coral_batch* b, int32_t trial_steps, int32_t* choice) {
  if (!b) return bfail(nullptr, CORAL_E_INVALID, "NULL batch");
  if (trial_steps < 1) return bfail(b, CORAL_E_INVALID, "trial_steps must be >= 1");
  const int cps1_0 = b->cps1, cps2_0 = b->cps2;
  // save every world's current state, step index and stats ring
  std::vector<void*> saved(b->n, nullptr);
  std::vector<long long> t0(b->n);
  std::vector<int> c0(b->n);
  auto release = [&]() {
    for (void* q : saved)
      if (q) cudaFree(q);
  };
  for (int i = 0; i < b->n; ++i) {
    coral_substrate* s = b->worlds[i];
    t0[i] = s->t;
    c0[i] = s->cur;
    const size_t bytes = (size_t)s->N * kStateBytesPerCell + sizeof(coral_stats) * kRing;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaMalloc(&saved[i], bytes);
    char* q = static_cast<char*>(saved[i]);
    const Planes& d = s->st[s->cur];
    if (e == cudaSuccess) e = cudaMemcpy(q, d.E, (size_t)s->N * 24, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q + (size_t)s->N * 24, d.G, (size_t)s->N * 4, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(q + (size_t)s->N * 28, d.R, (size_t)s->N, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(q + (size_t)s->N * kStateBytesPerCell, s->ring, sizeof(coral_stats) * kRing, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
      release();
      cudaGetLastError();
      return bfail(b, e == cudaErrorMemoryAllocation ? CORAL_E_OOM : CORAL_E_CUDA,
                   std::string("saving the states for tuning: ") + cudaGetErrorString(e));
    }
  }
  const int c1s[4] = {3, 4, 5, 6}, c2s[3] = {1, 2, 3};
  float best = 1e30f;
  int b1 = cps1_0, b2 = cps2_0, rc = CORAL_OK;
  std::vector<float> ms(trial_steps + 1);
  for (int i1 = 0; i1 < 4 && rc == CORAL_OK; ++i1)
    for (int i2 = 0; i2 < 3 && rc == CORAL_OK; ++i2) {
      b->cps1 = c1s[i1];
      b->cps2 = c2s[i2];
      if ((rc = batch_configure(b)) != CORAL_OK) break;
      if ((rc = batch_run(b, trial_steps + 1, ms.data(), false)) != CORAL_OK) break;
      float tot = 0;
      for (int k = 1; k <= trial_steps; ++k) tot += ms[k];
      if (tot < best) {
        best = tot;
        b1 = c1s[i1];
        b2 = c2s[i2];
      }
    }
  // the FMA small-genome cutoff at the chosen launch shape (the shapes are timed without it)
  const int fma_0 = b->fma_cutoff;
  int bf = fma_0;
  if (rc == CORAL_OK) {
    const int cuts[5] = {0, 1, 2, 4, 8};
    float best_f = 1e30f;
    b->cps1 = b1;
    b->cps2 = b2;
    for (int i = 0; i < 5 && rc == CORAL_OK; ++i) {
      b->fma_cutoff = cuts[i];
      if ((rc = batch_configure(b)) != CORAL_OK) break;
      if ((rc = batch_run(b, trial_steps + 1, ms.data(), false)) != CORAL_OK) break;
      float tot = 0;
      for (int k = 1; k <= trial_steps; ++k) tot += ms[k];
      if (tot < best_f) {
        best_f = tot;
        bf = cuts[i];
      }
    }
    if (rc == CORAL_OK) best = best_f;
  }
  // restore the states, step indices and stats rings, also after an error
  cudaError_t e = cudaStreamSynchronize(b->stream);
  for (int i = 0; i < b->n; ++i) {
    coral_substrate* s = b->worlds[i];
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    s->cur = c0[i];
    s->t = t0[i];
    const char* q = static_cast<const char*>(saved[i]);
    const Planes& d = s->st[s->cur];
    if (e == cudaSuccess) e = cudaMemcpy(d.E, q, (size_t)s->N * 24, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.G, q + (size_t)s->N * 24, (size_t)s->N * 4, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d.R, q + (size_t)s->N * 28, (size_t)s->N, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(s->ring, q + (size_t)s->N * kStateBytesPerCell, sizeof(coral_stats) * kRing, cudaMemcpyDeviceToDevice);
  }
  release();
  if (e != cudaSuccess && rc == CORAL_OK)
    rc = bfail(b, CORAL_E_CUDA, std::string("restoring the states after tuning: ") + cudaGetErrorString(e));
  if (rc != CORAL_OK) {
    // back to the launch shape the batch had before tuning
    b->cps1 = cps1_0;
    b->cps2 = cps2_0;
    b->fma_cutoff = fma_0;
    const std::string keep = b->err;
    batch_configure(b);
    b->err = keep;
    g_err = keep;
    return rc;
  }
  b->cps1 = b1;
  b->cps2 = b2;
  b->fma_cutoff = bf;
  if ((rc = batch_configure(b)) != CORAL_OK) return rc;
  if (choice) {
    choice[0] = b1;
    choice[1] = b2;
    choice[2] = (int32_t)(1000.0f * best / trial_steps);
    choice[3] = bf;
  }
  return CORAL_OK;
}
