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
#include "kernelset.h"

using mpd::MpArr;

struct mpdet_batch_ctx {
  int64_t count = 0, total = 0, total_d = 0, max_n = 0;
  int p = 0, n = 0, nsm = 0, blocks = 0;
  cudaStream_t stream = nullptr;
  const mpd::KernelSet* ks = nullptr;
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

static bool alloc_arr(MpArr* a, int64_t count, int n) {
  if (count < 1) count = 1;
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
  b->p = p_bits;
  b->n = n;
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
  b->blocks = b->nsm * b->ks->batch_blocks_per_sm();
  ok = ok && alloc_arr(&b->X0, b->total, n) && alloc_arr(&b->X, b->total, n) && alloc_arr(&b->D, b->total_d, n) &&
       alloc_arr(&b->Z, (int64_t)b->blocks * b->max_n, n);
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

static MpArr view(const MpArr& a, int64_t off, int n) { return MpArr{a.s + off, a.e + off, a.m + (size_t)off * n}; }

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

extern "C" int mpdet_batch_set_mp(mpdet_batch_t b, int64_t m, mpdet_numv A, int device_ptr) {
  if (!b || m < 0 || m >= b->count || !A.sign || !A.exp || !A.limbs) return MPDET_EINVAL;
  const int64_t NN = b->Ns[m] * b->Ns[m];
  const MpArr v = view(b->X0, b->xoff[m], b->n);
  const cudaMemcpyKind k = device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(v.m, A.limbs, (size_t)NN * b->n * 4, k, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(v.e, A.exp, (size_t)NN * 8, k, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(v.s, A.sign, (size_t)NN, k, b->stream) != cudaSuccess)
    return MPDET_ECUDA;
  return finish(b, device_ptr);
}

extern "C" int mpdet_batch_factor(mpdet_batch_t b, mpdet_numv minors, int64_t* zero_k, int device_ptr) {
  if (!b) return MPDET_EINVAL;
  const int n = b->n;
  cudaStream_t st = b->stream;
  // the stored inputs stay intact: eliminate a working copy
  if (cudaMemcpyAsync(b->X.m, b->X0.m, (size_t)b->total * n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->X.e, b->X0.e, (size_t)b->total * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->X.s, b->X0.s, (size_t)b->total, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(b->dqueue, 0, 16, st) != cudaSuccess || cudaMemsetAsync(b->dzero, 0, b->count * 8, st) != cudaSuccess)
    return MPDET_ECUDA;
  mpd::BatchDescHost bd{b->dN, b->dxoff, b->ddoff, b->dorder, b->dzero, b->dqueue, b->count, b->max_n};
  int blocks = (int)std::min<int64_t>(b->blocks, b->count);
  if (b->ks->batch(b->X, b->D, b->Z, bd, b->p, blocks, st) != cudaSuccess) return MPDET_ECUDA;
  b->launches += 1;
  const cudaMemcpyKind k = device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if ((minors.limbs && cudaMemcpyAsync(minors.limbs, b->D.m, (size_t)b->total_d * n * 4, k, st) != cudaSuccess) ||
      (minors.exp && cudaMemcpyAsync(minors.exp, b->D.e, (size_t)b->total_d * 8, k, st) != cudaSuccess) ||
      (minors.sign && cudaMemcpyAsync(minors.sign, b->D.s, (size_t)b->total_d, k, st) != cudaSuccess) ||
      (zero_k && cudaMemcpyAsync(zero_k, b->dzero, b->count * 8, k, st) != cudaSuccess))
    return MPDET_ECUDA;
  return finish(b, device_ptr);
}

extern "C" int64_t mpdet_batch_launches(mpdet_batch_t b) { return b ? b->launches : -1; }
