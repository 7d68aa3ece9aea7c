// Factorisation entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host framework that hands a plugin
// its buffers and forbids it to allocate device memory of its own (the
// framework owns the memory budget and its pools), and latency-bound loops
// that cannot afford an allocation or a pool growth in the middle of a step.
// For them mpdet_factor_noalloc runs the same elimination kernels as
// mpdet_factor but keeps every piece of working memory (the in-place matrix,
// the multipliers, the pivot reciprocal and the status words) in one
// statically sized device array that is part of the library image.  The
// caller provides only the input matrix and the output buffers.  The call
// reads the status words back to the host and synchronises its stream before
// it returns.
#include <cstring>
#include <mutex>

#include "../../include/mpdet.h"
#include "kernelset.h"

namespace {

constexpr size_t kScratchBytes = (size_t)MPDET_NOALLOC_SCRATCH_BYTES;

// The working memory.  Every GPU that loads the library holds this array
// until the process exits.  Host code must not use the symbol itself as an
// address (it names a host-side stand-in); the device address comes from
// cudaGetSymbolAddress, looked up once per device.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices];  // device address of g_scratch per device, nullptr until set up

size_t pad256(size_t b) { return (b + 255) / 256 * 256; }

// Scratch layout for N x N numbers of n limbs: matrix limbs, exponents,
// signs; N multipliers; one reciprocal; status words.
struct Layout {
  size_t x_m, x_e, x_s, z_m, z_e, z_s, r_m, r_e, r_s, status, zero_k, total;
};

Layout layout(int64_t N, int n) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += pad256(bytes);
    return at;
  };
  const size_t NN = (size_t)N * (size_t)N;
  L.x_m = take(NN * n * 4);
  L.x_e = take(NN * 8);
  L.x_s = take(NN);
  L.z_m = take((size_t)N * n * 4);
  L.z_e = take((size_t)N * 8);
  L.z_s = take((size_t)N);
  L.r_m = take((size_t)n * 4);
  L.r_e = take(8);
  L.r_s = take(1);
  L.status = take(16);
  L.zero_k = take(16);
  L.total = off;
  return L;
}

int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPDET_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return MPDET_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MPDET_ECUDA;
    }
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return MPDET_OK;
}

}  // namespace

extern "C" int mpdet_factor_noalloc(int64_t N, int32_t p_bits, uint32_t flags, mpdet_numv A, mpdet_numv minors,
                                    mpdet_numv lastcol, int64_t* zero_pivot_k, void* cuda_stream) {
  if (zero_pivot_k) *zero_pivot_k = 0;
  int32_t n = 0;
  if (N < 1 || mpdet_geometry(p_bits, &n, nullptr, nullptr) != MPDET_OK) return MPDET_EINVAL;
  if (mpd::frame_limbs(n) != n) return MPDET_EINVAL;  // a kernel family's own limb count only
  if (flags & ~(uint32_t)MPDET_LASTCOL) return MPDET_EINVAL;
  if (!A.sign || !A.exp || !A.limbs || !minors.sign || !minors.exp || !minors.limbs) return MPDET_EINVAL;
  const bool want_lastcol = (flags & MPDET_LASTCOL) != 0;
  if (want_lastcol && (!lastcol.sign || !lastcol.exp || !lastcol.limbs)) return MPDET_EINVAL;
  const Layout L = layout(N, n);
  if (L.total > kScratchBytes) return MPDET_ENOSCRATCH;  // above the static limit: use mpdet_create
  const mpd::KernelSet* ks = mpd::kernel_set_for(n);
  if (!ks) return MPDET_EINVAL;
  void* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MPDET_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  char* b = static_cast<char*>(base);
  mpd::MpArr X{reinterpret_cast<int8_t*>(b + L.x_s), reinterpret_cast<int64_t*>(b + L.x_e),
               reinterpret_cast<uint32_t*>(b + L.x_m)};
  mpd::MpArr Z{reinterpret_cast<int8_t*>(b + L.z_s), reinterpret_cast<int64_t*>(b + L.z_e),
               reinterpret_cast<uint32_t*>(b + L.z_m)};
  mpd::MpArr R{reinterpret_cast<int8_t*>(b + L.r_s), reinterpret_cast<int64_t*>(b + L.r_e),
               reinterpret_cast<uint32_t*>(b + L.r_m)};
  mpd::MpArr D{minors.sign, minors.exp, minors.limbs};
  int* status = reinterpret_cast<int*>(b + L.status);
  int64_t* zero_k = reinterpret_cast<int64_t*>(b + L.zero_k);
  const size_t NN = (size_t)N * (size_t)N;
  // The array keeps the previous call's contents: the status words start at
  // zero, the working matrix is overwritten by the input.
  cudaError_t e = cudaMemsetAsync(status, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(zero_k, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(X.m, A.limbs, NN * n * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(X.e, A.exp, NN * 8, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(X.s, A.sign, NN, cudaMemcpyDeviceToDevice, st);
  const int lc = want_lastcol ? 1 : 0;
  for (int64_t k = 0; k < N && e == cudaSuccess; ++k) {
    e = ks->pivot(X, N, k, D, R, status, zero_k, p_bits, st);
    if (e == cudaSuccess && k < N - 1) e = ks->mult(X, N, k, R, Z, status, p_bits, lc, st);
    if (e == cudaSuccess && k < N - 1) e = ks->update[1](X, mpd::upd_step(N, k, lc), Z, status, p_bits, nsm, st);
  }
  if (e == cudaSuccess && want_lastcol) {
    mpd::MpArr C{lastcol.sign, lastcol.exp, lastcol.limbs};
    if (N == 1) {  // C_11 = D_0 = 1
      uint32_t one[1024] = {0};
      one[n - 1] = 0x80000000u;
      int64_t e1 = 1;
      int8_t s0 = 0;
      e = cudaMemcpyAsync(C.m, one, (size_t)n * 4, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(C.e, &e1, 8, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(C.s, &s0, 1, cudaMemcpyHostToDevice, st);
    } else {
      mpd::MpArr F{D.s + (N - 2), D.e + (N - 2), D.m + (size_t)(N - 2) * n};
      e = ks->lastcol(X, N, F, C, 0, status, st);
    }
  }
  int hs[4] = {0};
  int64_t hz[2] = {0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs, status, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hz, zero_k, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MPDET_ECUDA;
  }
  if (zero_pivot_k) *zero_pivot_k = hz[0];
  return hs[0];
}
