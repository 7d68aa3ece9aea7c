// Batched elimination (step a7): many independent matrices of uneven N, one
// persistent launch.  Host side: inputs, offsets, the processing order and
// the launch; the arithmetic is k_batch in kernels.cuh.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/mpdet.h"
#include "batch_variants.h"
#include "kernelset.h"

using mpd::MpArr;

namespace mpd {
int batch_variants(int n, const BatchVariant** out) {
  // One list per supported limb count, built once (thread-safe static
  // initialisation): entry 0 is the kernel set's own kernel, then the extra
  // geometries compiled for that n.
  struct Table {
    int ns[9] = {4, 8, 16, 32, 64, 128, 256, 512, 1024};
    BatchVariant lists[9][8];
    int counts[9] = {0};
    Table() {
      for (int q = 0; q < 9; ++q) {
        const KernelSet* ks = kernel_set_for(ns[q]);
        if (!ks) continue;
        lists[q][0] = BatchVariant{ks->W, ks->G, ks->PW, ks->PG, ks->batch, ks->batch_blocks_per_sm};
        int c = 0;
        const BatchVariant* v = ns[q] == 16    ? batch_variants_n16(&c)
                                : ns[q] == 32  ? batch_variants_n32(&c)
                                : ns[q] == 64  ? batch_variants_n64(&c)
                                : ns[q] == 128 ? batch_variants_n128(&c)
                                               : nullptr;
        for (int i = 0; v && i < c && i < 7; ++i) lists[q][1 + i] = v[i];
        counts[q] = 1 + (v ? (c < 7 ? c : 7) : 0);
      }
    }
  };
  static const Table t;
  for (int q = 0; q < 9; ++q)
    if (t.ns[q] == n && t.counts[q] > 0) {
      *out = t.lists[q];
      return t.counts[q];
    }
  *out = nullptr;
  return 0;
}
}  // namespace mpd

struct mpdet_batch_ctx {
  int64_t count = 0, total = 0, total_d = 0, max_n = 0;
  // p, n: the kernels' frame; nu: the limbs of the precision asked for (pad = n - nu)
  int p = 0, n = 0, nu = 0, pad = 0, nsm = 0;
  int max_blocks = 0;  // blocks the per-block multiplier scratch Z is sized for
  cudaStream_t stream = nullptr;
  const mpd::KernelSet* ks = nullptr;
  // lane-geometry variant and resident blocks per SM of the persistent launch
  const mpd::BatchVariant* variants = nullptr;
  int nvariants = 0, variant = 0, bpsm = 0;
  std::vector<int> bpsm_max;  // occupancy limit per variant
  // CUDA graph of one factorisation (device outputs): captured on cap, replayed on stream
  bool graph = false;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int gkey_variant = -1, gkey_bpsm = -1;
  std::vector<int64_t> Ns, xoff, doff;
  MpArr X0{}, X{}, D{}, Z{};  // inputs as set, working copy, minors, per-block multipliers
  int64_t *dN = nullptr, *dxoff = nullptr, *ddoff = nullptr, *dzero = nullptr;
  int32_t* dorder = nullptr;
  int* dqueue = nullptr;
  void* stage = nullptr;
  size_t stage_bytes = 0;
  int64_t launches = 0;
};

static void free_arr(MpArr* a) {
  if (a->m) cudaFree(a->m);
  if (a->e) cudaFree(a->e);
  if (a->s) cudaFree(a->s);
  *a = MpArr{};
}

static bool alloc_arr(MpArr* a, int64_t count, int n, int pad) {
  if (count < 1) count = 1;
  a->pad = pad;
  return cudaMalloc(&a->m, (size_t)count * n * 4) == cudaSuccess && cudaMalloc(&a->e, (size_t)count * 8) == cudaSuccess &&
         cudaMalloc(&a->s, (size_t)count) == cudaSuccess;
}

extern "C" int mpdet_batch_free(mpdet_batch_t b) {
  if (!b) return MPDET_OK;
  free_arr(&b->X0);
  free_arr(&b->X);
  free_arr(&b->D);
  free_arr(&b->Z);
  cudaFree(b->dN);
  cudaFree(b->dxoff);
  cudaFree(b->ddoff);
  cudaFree(b->dzero);
  cudaFree(b->dorder);
  cudaFree(b->dqueue);
  if (b->stage) cudaFree(b->stage);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return MPDET_OK;
}

extern "C" int mpdet_batch_create(int64_t count, const int64_t* Ns, int32_t p_bits, void* cuda_stream, mpdet_batch_t* out) {
  if (!out || !Ns || count < 1 || count > (int64_t)1 << 30) return MPDET_EINVAL;
  *out = nullptr;
  int32_t n = 0;
  if (mpdet_geometry(p_bits, &n, nullptr, nullptr) != MPDET_OK) return MPDET_EINVAL;
  for (int64_t i = 0; i < count; ++i)
    if (Ns[i] < 1 || Ns[i] > 65536) return MPDET_EINVAL;
  mpdet_batch_t b = new (std::nothrow) mpdet_batch_ctx();
  if (!b) return MPDET_ENOMEM;
  b->count = count;
  b->nu = n;
  b->n = mpd::frame_limbs(n);
  b->p = 32 * b->n;
  b->pad = b->n - b->nu;
  n = b->n;
  b->stream = (cudaStream_t)cuda_stream;
  b->ks = mpd::kernel_set_for(n);
  b->Ns.assign(Ns, Ns + count);
  b->xoff.resize(count);
  b->doff.resize(count);
  for (int64_t i = 0; i < count; ++i) {
    b->xoff[i] = b->total;
    b->doff[i] = b->total_d;
    b->total += Ns[i] * Ns[i];
    b->total_d += Ns[i];
    b->max_n = std::max(b->max_n, Ns[i]);
  }
  // longest jobs first (greedy balance of the persistent blocks)
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return Ns[a] > Ns[c]; });
  int dev = 0;
  bool ok = cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
  if (ok) b->nvariants = mpd::batch_variants(n, &b->variants);
  ok = ok && b->nvariants >= 1;
  if (ok) {
    int mx = 1;
    for (int v = 0; v < b->nvariants; ++v) {
      b->bpsm_max.push_back(b->variants[v].blocks_per_sm());
      mx = std::max(mx, b->bpsm_max.back());
    }
    b->bpsm = b->bpsm_max[0];
    b->max_blocks = b->nsm * mx;
  }
  ok = ok && alloc_arr(&b->X0, b->total, n, b->pad) && alloc_arr(&b->X, b->total, n, b->pad) &&
       alloc_arr(&b->D, b->total_d, n, b->pad) && alloc_arr(&b->Z, (int64_t)b->max_blocks * b->max_n, n, b->pad);
  ok = ok && cudaMalloc(&b->dN, count * 8) == cudaSuccess && cudaMalloc(&b->dxoff, count * 8) == cudaSuccess &&
       cudaMalloc(&b->ddoff, count * 8) == cudaSuccess && cudaMalloc(&b->dzero, count * 8) == cudaSuccess &&
       cudaMalloc(&b->dorder, count * 4) == cudaSuccess && cudaMalloc(&b->dqueue, 16) == cudaSuccess;
  ok = ok && cudaMemcpy(b->dN, Ns, count * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(b->dxoff, b->xoff.data(), count * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(b->ddoff, b->doff.data(), count * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(b->dorder, order.data(), count * 4, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mpdet_batch_free(b);
    return MPDET_ENOMEM;
  }
  *out = b;
  return MPDET_OK;
}

static MpArr view(const MpArr& a, int64_t off, int n) {
  return MpArr{a.s + off, a.e + off, a.m + (size_t)off * n, a.pad};
}

static int stage_in(mpdet_batch_t b, const void* src, size_t bytes, const void** dev) {
  if (b->stage_bytes < bytes) {
    if (b->stage) cudaFree(b->stage);
    b->stage = nullptr;
    b->stage_bytes = 0;
    if (cudaMalloc(&b->stage, bytes) != cudaSuccess) return MPDET_ENOMEM;
    b->stage_bytes = bytes;
  }
  if (cudaMemcpyAsync(b->stage, src, bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) return MPDET_ECUDA;
  *dev = b->stage;
  return MPDET_OK;
}

static int finish(mpdet_batch_t b, int device_ptr) {
  if (cudaGetLastError() != cudaSuccess) return MPDET_ECUDA;
  if (!device_ptr && cudaStreamSynchronize(b->stream) != cudaSuccess) return MPDET_ECUDA;
  return MPDET_OK;
}

static int set_dense(mpdet_batch_t b, int64_t m, const void* A, int64_t ld, int device_ptr, int kind) {
  if (!b || m < 0 || m >= b->count || !A || ld < b->Ns[m]) return MPDET_EINVAL;
  const int64_t N = b->Ns[m];
  const void* src = A;
  if (!device_ptr) {
    int rc = stage_in(b, A, (size_t)((N - 1) * ld + N) * (kind == 0 ? 8 : 4), &src);
    if (rc) return rc;
  }
  if (b->ks->lift(src, kind, ld, N, view(b->X0, b->xoff[m], b->n), b->p, b->nsm, b->stream) != cudaSuccess)
    return MPDET_ECUDA;
  b->launches += 1;
  return finish(b, device_ptr);
}

extern "C" int mpdet_batch_set_f64(mpdet_batch_t b, int64_t m, const double* A, int64_t ld, int device_ptr) {
  return set_dense(b, m, A, ld, device_ptr, 0);
}

extern "C" int mpdet_batch_set_i32(mpdet_batch_t b, int64_t m, const int32_t* A, int64_t ld, int device_ptr) {
  return set_dense(b, m, A, ld, device_ptr, 1);
}

extern "C" int mpdet_batch_set_cauchy(mpdet_batch_t b, int64_t m, const double* x, const double* y, int device_ptr) {
  if (!b || m < 0 || m >= b->count || !x || !y) return MPDET_EINVAL;
  const int64_t N = b->Ns[m];
  const double *dx = x, *dy = y;
  if (!device_ptr) {
    const size_t nb = (size_t)N * 8;
    if (b->stage_bytes < 2 * nb) {
      if (b->stage) cudaFree(b->stage);
      b->stage = nullptr;
      b->stage_bytes = 0;
      if (cudaMalloc(&b->stage, 2 * nb) != cudaSuccess) return MPDET_ENOMEM;
      b->stage_bytes = 2 * nb;
    }
    if (cudaMemcpyAsync(b->stage, x, nb, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync((char*)b->stage + nb, y, nb, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
      return MPDET_ECUDA;
    dx = (const double*)b->stage;
    dy = (const double*)((char*)b->stage + nb);
  }
  if (b->ks->cauchy(dx, dy, N, view(b->X0, b->xoff[m], b->n), b->p, b->nsm, b->stream) != cudaSuccess)
    return MPDET_ECUDA;
  b->launches += 1;
  return finish(b, device_ptr);
}

// Copy matrix m's N_m * N_m numbers into the stored inputs (no synchronisation;
// a copy from pageable host memory returns once the source has been read).
static int copy_mp_in(mpdet_batch_t b, int64_t m, const mpdet_numv& A, int device_ptr) {
  const int64_t NN = b->Ns[m] * b->Ns[m];
  const MpArr v = view(b->X0, b->xoff[m], b->n);
  const cudaMemcpyKind k = device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (mpd::copy_numbers(v, b->n, A.sign, A.exp, A.limbs, b->nu, NN, true, k, b->stream) != cudaSuccess)
    return MPDET_ECUDA;
  return MPDET_OK;
}

extern "C" int mpdet_batch_set_mp(mpdet_batch_t b, int64_t m, mpdet_numv A, int device_ptr) {
  if (!b || m < 0 || m >= b->count || !A.sign || !A.exp || !A.limbs) return MPDET_EINVAL;
  const int rc = copy_mp_in(b, m, A, device_ptr);
  return rc ? rc : finish(b, device_ptr);
}

// One factorisation of the stored inputs: working copy, cleared queue and
// statuses, the persistent launch, and the outputs (kind: copy direction).
static int enqueue_factor(mpdet_batch_t b, cudaStream_t st, mpdet_numv minors, int64_t* zero_k, cudaMemcpyKind k) {
  const int n = b->n;
  // the stored inputs stay intact: eliminate a working copy
  if (cudaMemcpyAsync(b->X.m, b->X0.m, (size_t)b->total * n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->X.e, b->X0.e, (size_t)b->total * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->X.s, b->X0.s, (size_t)b->total, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(b->dqueue, 0, 16, st) != cudaSuccess || cudaMemsetAsync(b->dzero, 0, b->count * 8, st) != cudaSuccess)
    return MPDET_ECUDA;
  mpd::BatchDescHost bd{b->dN, b->dxoff, b->ddoff, b->dorder, b->dzero, b->dqueue, b->count, b->max_n};
  const int blocks = (int)std::min<int64_t>((int64_t)b->nsm * b->bpsm, b->count);
  if (b->variants[b->variant].launch(b->X, b->D, b->Z, bd, b->p, blocks, st) != cudaSuccess) return MPDET_ECUDA;
  if (mpd::copy_numbers(b->D, n, minors.sign, minors.exp, minors.limbs, b->nu, b->total_d, false, k, st) !=
          cudaSuccess ||
      (zero_k && cudaMemcpyAsync(zero_k, b->dzero, b->count * 8, k, st) != cudaSuccess))
    return MPDET_ECUDA;
  return MPDET_OK;
}

// Replay (capturing first when the outputs or the launch shape changed) the
// graph of one factorisation with device outputs.
static int graph_factor(mpdet_batch_t b, mpdet_numv minors, int64_t* zero_k) {
  const void* key[5] = {minors.limbs, minors.exp, minors.sign, zero_k, b->stream};
  bool same = b->gexec && b->gkey_variant == b->variant && b->gkey_bpsm == b->bpsm;
  for (int q = 0; q < 5 && same; ++q) same = key[q] == b->gkey[q];
  if (!same) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return MPDET_ECUDA;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MPDET_ECUDA;
    int rc = enqueue_factor(b, b->cap, minors, zero_k, cudaMemcpyDeviceToDevice);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
    if (rc || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return MPDET_ECUDA;
    }
    ce = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      b->gexec = nullptr;
      return MPDET_ECUDA;
    }
    for (int q = 0; q < 5; ++q) b->gkey[q] = key[q];
    b->gkey_variant = b->variant;
    b->gkey_bpsm = b->bpsm;
  }
  return cudaGraphLaunch(b->gexec, b->stream) == cudaSuccess ? MPDET_OK : MPDET_ECUDA;
}

extern "C" int mpdet_batch_factor(mpdet_batch_t b, mpdet_numv minors, int64_t* zero_k, int device_ptr) {
  if (!b) return MPDET_EINVAL;
  int rc = (b->graph && device_ptr)
               ? graph_factor(b, minors, zero_k)
               : enqueue_factor(b, b->stream, minors, zero_k, device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  if (rc) return rc;
  b->launches += 1;
  return finish(b, device_ptr);
}

extern "C" int mpdet_batch_tune(mpdet_batch_t b, int param, int value) {
  if (!b) return MPDET_EINVAL;
  switch (param) {
    case MPDET_BATCH_VARIANT:
      if (value < 0 || value >= b->nvariants) return MPDET_EINVAL;
      b->variant = value;
      b->bpsm = std::min(b->bpsm, b->bpsm_max[value]);
      return MPDET_OK;
    case MPDET_BATCH_BLOCKS_PER_SM:
      if (value < 1 || value > b->bpsm_max[b->variant]) return MPDET_EINVAL;
      b->bpsm = value;
      return MPDET_OK;
    case MPDET_BATCH_GRAPH:
      if (value != 0 && value != 1) return MPDET_EINVAL;
      b->graph = value == 1;
      return MPDET_OK;
    default:
      return MPDET_EINVAL;
  }
}

extern "C" int mpdet_batch_variant_info(mpdet_batch_t b, int32_t variant, int32_t* W, int32_t* G, int32_t* PW,
                                        int32_t* PG, int32_t* max_blocks_per_sm) {
  if (!b || variant < 0 || variant >= b->nvariants) return MPDET_EINVAL;
  const mpd::BatchVariant& v = b->variants[variant];
  if (W) *W = v.W;
  if (G) *G = v.G;
  if (PW) *PW = v.PW;
  if (PG) *PG = v.PG;
  if (max_blocks_per_sm) *max_blocks_per_sm = b->bpsm_max[variant];
  return MPDET_OK;
}

extern "C" int mpdet_batch_autotune(mpdet_batch_t b, int reps, int32_t* variant, int32_t* blocks_per_sm,
                                    double* best_ms, int32_t* candidates) {
  if (!b || reps < 1) return MPDET_EINVAL;
  const int v0 = b->variant, p0 = b->bpsm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return MPDET_ECUDA;
  }
  double best = 1e300;
  int bv = v0, bp = p0, ncand = 0, rc = MPDET_OK;
  mpdet_numv none{nullptr, nullptr, nullptr};
  for (int v = 0; v < b->nvariants && !rc; ++v) {
    // resident blocks per SM: the occupancy limit and its half (more blocks
    // hide latency, fewer balance the tail of uneven jobs better)
    const int mx = b->bpsm_max[v];
    const int cand[2] = {mx, std::max(1, mx / 2)};
    for (int c = 0; c < (cand[1] == cand[0] ? 1 : 2) && !rc; ++c) {
      b->variant = v;
      b->bpsm = cand[c];
      float ms = 0.f;
      if ((rc = enqueue_factor(b, b->stream, none, nullptr, cudaMemcpyDeviceToDevice))) break;  // warm-up
      if (cudaEventRecord(e0, b->stream) != cudaSuccess) { rc = MPDET_ECUDA; break; }
      for (int r = 0; r < reps && !rc; ++r) rc = enqueue_factor(b, b->stream, none, nullptr, cudaMemcpyDeviceToDevice);
      if (rc || cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = rc ? rc : MPDET_ECUDA;
        break;
      }
      b->launches += 1 + reps;
      ++ncand;
      if (ms / reps < best) {
        best = ms / reps;
        bv = v;
        bp = cand[c];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    b->variant = v0;
    b->bpsm = p0;
    return rc;
  }
  b->variant = bv;
  b->bpsm = bp;
  if (variant) *variant = bv;
  if (blocks_per_sm) *blocks_per_sm = bp;
  if (best_ms) *best_ms = best;
  if (candidates) *candidates = ncand;
  return MPDET_OK;
}

extern "C" int mpdet_batch(int64_t count, const int64_t* Ns, int32_t p_bits, const mpdet_numv* in,
                           mpdet_numv* minors_out, int64_t* status_out, int device_ptr, void* cuda_stream) {
  // sizes first: count bounds how far the pointer arrays may be read
  if (count < 1 || count > (int64_t)1 << 30 || !Ns || !in || !minors_out) return MPDET_EINVAL;
  for (int64_t m = 0; m < count; ++m)
    if (Ns[m] < 1 || Ns[m] > 65536) return MPDET_EINVAL;
  for (int64_t m = 0; m < count; ++m)
    if (!in[m].sign || !in[m].exp || !in[m].limbs || !minors_out[m].sign || !minors_out[m].exp ||
        !minors_out[m].limbs)
      return MPDET_EINVAL;
  mpdet_batch_t b = nullptr;
  int rc = mpdet_batch_create(count, Ns, p_bits, cuda_stream, &b);
  if (rc) return rc;
  // all inputs are enqueued without a wait in between; one synchronisation at the end
  for (int64_t m = 0; m < count && !rc; ++m) rc = copy_mp_in(b, m, in[m], device_ptr);
  const mpdet_numv none{nullptr, nullptr, nullptr};
  if (!rc) rc = enqueue_factor(b, b->stream, none, nullptr, cudaMemcpyDeviceToDevice);
  if (!rc) b->launches += 1;
  // matrix m's minors D_1..D_{N_m} sit at offset doff[m] of the batch's minors
  const cudaMemcpyKind k = device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const int n = b->n;
  for (int64_t m = 0; m < count && !rc; ++m) {
    const MpArr d = view(b->D, b->doff[m], n);
    const int64_t N = b->Ns[m];
    if (mpd::copy_numbers(d, n, minors_out[m].sign, minors_out[m].exp, minors_out[m].limbs, b->nu, N, false, k,
                          b->stream) != cudaSuccess)
      rc = MPDET_ECUDA;
  }
  if (!rc && status_out && cudaMemcpyAsync(status_out, b->dzero, count * 8, k, b->stream) != cudaSuccess)
    rc = MPDET_ECUDA;
  if (!rc && (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess)) rc = MPDET_ECUDA;
  if (rc) cudaStreamSynchronize(b->stream);
  mpdet_batch_free(b);
  return rc;
}

extern "C" int64_t mpdet_batch_launches(mpdet_batch_t b) { return b ? b->launches : -1; }
