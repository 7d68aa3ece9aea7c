// C-ABI layer of libmpdet: handle life cycle, argument checks, device buffers
// and the step loop of the elimination (Sec. 3 / Algorithm 1).  Every
// arithmetic step runs in the kernels of kernels.cuh; this file only moves
// data and enqueues launches.
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mpdet.h"
#include "kernelset.h"

using mpd::KernelSet;
using mpd::MpArr;
using mpd::UpdArgs;

namespace mpd {
const KernelSet* kernel_set_for(int n) {
  switch (n) {
    case 4: return kernel_set_w4_g1();
    case 8: return kernel_set_w8_g1();
    case 16: return kernel_set_w16_g1();
    case 32: return kernel_set_w16_g2();
    case 64: return kernel_set_w16_g4();
    case 128: return kernel_set_w16_g8();
    case 256: return kernel_set_w16_g16();
    case 512: return kernel_set_w16_g32();
    case 1024: return kernel_set_w32_g32();
    default: return nullptr;
  }
}

// Default register-budget variant of the Schur update per limb count.
int default_update_variant(int n) {
  (void)n;
  return 1;
}
}  // namespace mpd

struct mpdet_ctx {
  int64_t N = 0;
  // p, n: the frame the kernels work in (a kernel family's limb count);
  // pu, nu: the precision asked for (pu = 32 nu <= p), pad = n - nu
  int p = 0, n = 0, pu = 0, nu = 0, pad = 0;
  uint32_t flags = 0;
  cudaStream_t stream = nullptr;
  int device = 0, nsm = 0;
  const KernelSet* ks = nullptr;
  MpArr X{}, D{}, Z{}, R{}, T{};  // matrix, minors, multipliers, reciprocal, temp (N numbers)
  MpArr Z2{};                     // multipliers of odd steps under look-ahead (N numbers)
  MpArr S{};                      // adjoint: S = L, then X = A^-1 (N*N numbers, allocated on first use)
  void* xhost[3] = {nullptr, nullptr, nullptr};  // MPDET_HOSTMEM: host allocations behind X (limbs, exp, sign)
  int* status = nullptr;          // [0] code
  int64_t* zero_k = nullptr;
  void* stage = nullptr;  // device staging for host inputs
  size_t stage_bytes = 0;
  int64_t k_done = 0;
  int upd_variant = 1;
  int engine = 1;  // 1: tensor cores, pipelined (p = 512..2048; 4096..32768); 2: tensor cores, one role at a time; 0: IMAD
  // large-precision tensor engine: the multipliers' digits and the staged
  // products (allocated on first use)
  void* zd = nullptr;
  uint32_t* slab = nullptr;
  int64_t tc_min_rows = -1;  // shorter update launches take the IMAD kernel; -1: per precision
  // look-ahead: the side stream updates column k+1 and runs the pivot and the
  // multipliers of step k+1 while the handle's stream updates the rest of
  // step k on all SMs but la_reserve
  int lookahead = 1;
  int la_reserve = 4;
  // IMAD update geometry: 0 the kernel set's own, 1 / 2 32 limbs per lane
  // compiled for 4 / 3 blocks per SM (n = 64 .. 512); -1 per precision
  int upd_geom = -1;
  int kara = 0;  // 1: IMAD update products by one Karatsuba level (n >= 256)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_mult = nullptr, ev_rest = nullptr;
  bool have_matrix = false;
  char err[512] = {0};
  // instrumentation: kernel launches enqueued, and optional event pairs
  // around every Schur-update launch
  int64_t launches = 0;
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double upd_ms = 0.0;
  int64_t upd_launches = 0;
  double upd_products = 0.0;
};

static const char* g_static_err = "no handle";

static int fail(mpdet_t h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof h->err, fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CU(h, call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(h, MPDET_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// radii of the ball mode for count numbers (MPDET_BALL only)
static int alloc_rad(mpdet_t h, MpArr* a, int64_t count) {
  if (!(h->flags & MPDET_BALL)) return MPDET_OK;
  if (cudaMalloc(&a->rm, (size_t)count * 4) != cudaSuccess || cudaMalloc(&a->re, (size_t)count * 8) != cudaSuccess)
    return fail(h, MPDET_ENOMEM, "cudaMalloc radii");
  return MPDET_OK;
}

static int alloc_arr(mpdet_t h, MpArr* a, int64_t count) {
  int n = h->n;
  a->pad = h->pad;
  if (cudaMalloc(&a->m, (size_t)count * n * 4) != cudaSuccess) return fail(h, MPDET_ENOMEM, "cudaMalloc limbs");
  if (cudaMalloc(&a->e, (size_t)count * 8) != cudaSuccess) return fail(h, MPDET_ENOMEM, "cudaMalloc exp");
  if (cudaMalloc(&a->s, (size_t)count) != cudaSuccess) return fail(h, MPDET_ENOMEM, "cudaMalloc sign");
  return MPDET_OK;
}

static void free_arr(MpArr* a) {
  if (a->m) cudaFree(a->m);
  if (a->e) cudaFree(a->e);
  if (a->s) cudaFree(a->s);
  if (a->rm) cudaFree(a->rm);
  if (a->re) cudaFree(a->re);
  *a = MpArr{};
}

// radii set to 0 (value 0) or to unbounded, count numbers
static cudaError_t set_rad(MpArr a, int64_t count, bool unbounded, cudaStream_t st) {
  if (!a.rm || count <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.rm, unbounded ? 0xff : 0, (size_t)count * 4, st);
  if (e != cudaSuccess) return e;
  if (unbounded) {  // INT64_MAX = ff .. ff 7f (little endian)
    e = cudaMemsetAsync(a.re, 0xff, (size_t)count * 8, st);
    if (e != cudaSuccess) return e;
    return cudaMemset2DAsync(reinterpret_cast<char*>(a.re) + 7, 8, 0x7f, 1, (size_t)count, st);
  }
  e = cudaMemsetAsync(a.re, 0, (size_t)count * 8, st);  // INT64_MIN = 00 .. 00 80
  if (e != cudaSuccess) return e;
  return cudaMemset2DAsync(reinterpret_cast<char*>(a.re) + 7, 8, 0x80, 1, (size_t)count, st);
}

// The in-place array in page-locked host memory mapped into the device's
// address space (MPDET_HOSTMEM): the kernels read and write it in place.
static int alloc_arr_host(mpdet_t h, MpArr* a, int64_t count) {
  const size_t bytes[3] = {(size_t)count * h->n * 4, (size_t)count * 8, (size_t)count};
  void* hp[3] = {nullptr, nullptr, nullptr};
  void* dp[3] = {nullptr, nullptr, nullptr};
  for (int q = 0; q < 3; ++q) {
    if (cudaHostAlloc(&hp[q], bytes[q], cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
        cudaHostGetDevicePointer(&dp[q], hp[q], 0) != cudaSuccess) {
      cudaGetLastError();
      for (int r = 0; r <= q; ++r)
        if (hp[r]) cudaFreeHost(hp[r]);
      return fail(h, MPDET_ENOMEM, "cudaHostAlloc of %zu bytes", bytes[q]);
    }
  }
  h->xhost[0] = hp[0];
  h->xhost[1] = hp[1];
  h->xhost[2] = hp[2];
  *a = MpArr{(int8_t*)dp[2], (int64_t*)dp[1], (uint32_t*)dp[0], h->pad};
  return MPDET_OK;
}

// zero (+0) numbers: sign 0, exp INT64_MIN, limbs 0
static cudaError_t zero_arr(MpArr a, int64_t count, int n, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.m, 0, (size_t)count * n * 4, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.s, 0, (size_t)count, st);
  if (e != cudaSuccess) return e;
  // INT64_MIN = 0x8000000000000000: bytes 00 .. 00 80 (little endian); fill by a 2D memset of the top byte
  e = cudaMemsetAsync(a.e, 0, (size_t)count * 8, st);
  if (e != cudaSuccess) return e;
  return cudaMemset2DAsync(reinterpret_cast<char*>(a.e) + 7, 8, 0x80, 1, (size_t)count, st);
}

extern "C" int mpdet_geometry(int32_t p_bits, int32_t* n, int32_t* W, int32_t* G) {
  if (p_bits < 64 || p_bits > 32768 || (p_bits % 32) != 0) return MPDET_EINVAL;
  const KernelSet* ks = mpd::kernel_set_for(mpd::frame_limbs(p_bits / 32));
  if (!ks) return MPDET_EINVAL;
  if (n) *n = p_bits / 32;
  if (W) *W = ks->W;
  if (G) *G = ks->G;
  return MPDET_OK;
}

extern "C" int mpdet_create(int64_t N, int32_t p_bits, uint32_t flags, void* cuda_stream, mpdet_t* out) {
  if (!out) return MPDET_EINVAL;
  *out = nullptr;
  if (N < 1 || N > (int64_t)1 << 20) return MPDET_EINVAL;
  if (flags & ~(uint32_t)(MPDET_LASTCOL | MPDET_HOSTMEM | MPDET_BALL)) return MPDET_EINVAL;
  if (mpdet_geometry(p_bits, nullptr, nullptr, nullptr) != MPDET_OK) return MPDET_EINVAL;
  mpdet_t h = new (std::nothrow) mpdet_ctx();
  if (!h) return MPDET_ENOMEM;
  h->N = N;
  h->pu = p_bits;
  h->nu = p_bits / 32;
  h->n = mpd::frame_limbs(h->nu);
  h->p = 32 * h->n;
  h->pad = h->n - h->nu;
  h->flags = flags;
  h->stream = (cudaStream_t)cuda_stream;
  h->ks = mpd::kernel_set_for(h->n);
  h->upd_variant = mpd::default_update_variant(h->n);
  int rc = MPDET_OK;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    rc = MPDET_ECUDA;
  }
  if (rc == MPDET_OK) rc = (flags & MPDET_HOSTMEM) ? alloc_arr_host(h, &h->X, N * N) : alloc_arr(h, &h->X, N * N);
  if (rc == MPDET_OK) rc = alloc_arr(h, &h->D, N);
  if (rc == MPDET_OK) rc = alloc_arr(h, &h->Z, N);
  if (rc == MPDET_OK) rc = alloc_arr(h, &h->Z2, N);
  if (rc == MPDET_OK) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_mult, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_rest, cudaEventDisableTiming) != cudaSuccess)
      rc = MPDET_ECUDA;
  }
  if (rc == MPDET_OK) rc = alloc_arr(h, &h->T, N);
  if (rc == MPDET_OK) rc = alloc_arr(h, &h->R, 1);
  if (rc == MPDET_OK) rc = alloc_rad(h, &h->X, N * N);
  if (rc == MPDET_OK) rc = alloc_rad(h, &h->D, N);
  if (rc == MPDET_OK) rc = alloc_rad(h, &h->Z, N);
  if (rc == MPDET_OK) rc = alloc_rad(h, &h->Z2, N);
  if (rc == MPDET_OK) rc = alloc_rad(h, &h->T, N);
  if (rc == MPDET_OK) rc = alloc_rad(h, &h->R, 1);
  if (rc == MPDET_OK && cudaMalloc(&h->status, 16) != cudaSuccess) rc = MPDET_ENOMEM;
  if (rc == MPDET_OK && cudaMalloc(&h->zero_k, 16) != cudaSuccess) rc = MPDET_ENOMEM;
  if (rc == MPDET_OK && (cudaMemsetAsync(h->status, 0, 16, h->stream) != cudaSuccess ||
                         cudaMemsetAsync(h->zero_k, 0, 16, h->stream) != cudaSuccess ||
                         zero_arr(h->D, N, h->n, h->stream) != cudaSuccess ||
                         cudaStreamSynchronize(h->stream) != cudaSuccess))
    rc = MPDET_ECUDA;
  if (rc != MPDET_OK) {
    cudaGetLastError();
    mpdet_free(h);
    return rc;
  }
  *out = h;
  return MPDET_OK;
}

extern "C" int mpdet_free(mpdet_t h) {
  if (!h) return MPDET_OK;
  if (h->flags & MPDET_HOSTMEM) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->side) cudaStreamSynchronize(h->side);
    for (void* hp : h->xhost)
      if (hp) cudaFreeHost(hp);
    h->X.s = nullptr;
    h->X.e = nullptr;
    h->X.m = nullptr;  // its radii, if any, are device memory and freed below
  }
  free_arr(&h->X);
  free_arr(&h->D);
  free_arr(&h->Z);
  free_arr(&h->Z2);
  free_arr(&h->T);
  free_arr(&h->R);
  free_arr(&h->S);
  if (h->status) cudaFree(h->status);
  if (h->zero_k) cudaFree(h->zero_k);
  if (h->stage) cudaFree(h->stage);
  if (h->zd) cudaFree(h->zd);
  if (h->slab) cudaFree(h->slab);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->ev_mult) cudaEventDestroy(h->ev_mult);
  if (h->ev_rest) cudaEventDestroy(h->ev_rest);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  delete h;
  return MPDET_OK;
}

extern "C" const char* mpdet_last_error(mpdet_t h) { return h ? h->err : g_static_err; }

extern "C" int64_t mpdet_steps_done(mpdet_t h) { return h ? h->k_done : -1; }

static int stage_in(mpdet_t h, const void* src, size_t bytes, const void** dev) {
  if (h->stage_bytes < bytes) {
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    if (cudaMalloc(&h->stage, bytes) != cudaSuccess) return fail(h, MPDET_ENOMEM, "staging buffer of %zu bytes", bytes);
    h->stage_bytes = bytes;
  }
  CU(h, cudaMemcpyAsync(h->stage, src, bytes, cudaMemcpyHostToDevice, h->stream));
  *dev = h->stage;
  return MPDET_OK;
}

// reset factorisation state after a new matrix
static int reset_state(mpdet_t h) {
  CU(h, cudaMemsetAsync(h->status, 0, 16, h->stream));
  CU(h, cudaMemsetAsync(h->zero_k, 0, 16, h->stream));
  CU(h, zero_arr(h->D, h->N, h->n, h->stream));
  CU(h, set_rad(h->D, h->N, true, h->stream));       // minors not reached stay unbounded
  CU(h, set_rad(h->X, h->N * h->N, false, h->stream));  // inputs are exact unless a generator sets radii
  h->k_done = 0;
  h->have_matrix = true;
  return MPDET_OK;
}

static int finish_call(mpdet_t h, int device_ptr) {
  CU(h, cudaGetLastError());
  if (!device_ptr) CU(h, cudaStreamSynchronize(h->stream));
  return MPDET_OK;
}

static int set_dense(mpdet_t h, const void* A, int64_t ld, int device_ptr, int kind) {
  if (!h || !A || ld < h->N) return fail(h, MPDET_EINVAL, "set: bad argument");
  const void* src = A;
  if (!device_ptr) {
    size_t es = kind == 0 ? 8 : 4;
    // pack rows (ld may exceed N): stage the whole ld-strided block
    size_t bytes = (size_t)((h->N - 1) * ld + h->N) * es;
    int rc = stage_in(h, A, bytes, &src);
    if (rc) return rc;
  }
  int rc = reset_state(h);
  if (rc) return rc;
  CU(h, h->ks->lift(src, kind, ld, h->N, h->X, h->p, h->nsm, h->stream));
  h->launches += 1;
  return finish_call(h, device_ptr);
}

extern "C" int mpdet_set_f64(mpdet_t h, const double* A, int64_t ld, int device_ptr) {
  return set_dense(h, A, ld, device_ptr, 0);
}

extern "C" int mpdet_set_i32(mpdet_t h, const int32_t* A, int64_t ld, int device_ptr) {
  return set_dense(h, A, ld, device_ptr, 1);
}

// Numbers between a caller's buffer (pu bits: nu limbs each) and a device
// array of the handle (frame of n limbs each).
static int copy_arr(mpdet_t h, MpArr dst_dev, const mpdet_numv& src, int64_t count, int device_ptr, bool to_dev) {
  cudaMemcpyKind kind = device_ptr ? cudaMemcpyDeviceToDevice : (to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  CU(h, mpd::copy_numbers(dst_dev, h->n, src.sign, src.exp, src.limbs, h->nu, count, to_dev, kind, h->stream));
  return MPDET_OK;
}

extern "C" int mpdet_set_mp(mpdet_t h, mpdet_numv A, int device_ptr) {
  if (!h || !A.sign || !A.exp || !A.limbs) return fail(h, MPDET_EINVAL, "set_mp: null pointer");
  int rc = reset_state(h);
  if (rc) return rc;
  rc = copy_arr(h, h->X, A, h->N * h->N, device_ptr, true);
  if (rc) return rc;
  return finish_call(h, device_ptr);
}

extern "C" int mpdet_set_cauchy(mpdet_t h, const double* x, const double* y, int device_ptr) {
  if (!h || !x || !y) return fail(h, MPDET_EINVAL, "set_cauchy: null pointer");
  const double *dx = x, *dy = y;
  if (!device_ptr) {
    size_t nb = (size_t)h->N * 8;
    if (h->stage_bytes < 2 * nb) {
      if (h->stage) cudaFree(h->stage);
      h->stage = nullptr;
      h->stage_bytes = 0;
      if (cudaMalloc(&h->stage, 2 * nb) != cudaSuccess) return fail(h, MPDET_ENOMEM, "staging");
      h->stage_bytes = 2 * nb;
    }
    CU(h, cudaMemcpyAsync(h->stage, x, nb, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync((char*)h->stage + nb, y, nb, cudaMemcpyHostToDevice, h->stream));
    dx = (const double*)h->stage;
    dy = (const double*)((char*)h->stage + nb);
  }
  int rc = reset_state(h);
  if (rc) return rc;
  CU(h, h->ks->cauchy(dx, dy, h->N, h->X, h->p, h->nsm, h->stream));
  h->launches += 1;
  return finish_call(h, device_ptr);
}

static int next_event(mpdet_t h, cudaEvent_t* ev) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    CU(h, cudaEventCreate(&e));
    h->ev_pool.push_back(e);
  }
  *ev = h->ev_pool[h->ev_used++];
  return MPDET_OK;
}

// Default row threshold of the tensor engines per precision, from GB300
// measurements of whole eliminations: 64 rows at p = 2048 (twice the IMAD
// kernel's speed from about 64 rows on), at p = 1024 (with two tensor-memory
// buffers: 0.62 of the IMAD kernel's time at N = 2048, 0.92 at N = 512, 1.05
// at N = 1024, lastcol mode) and at p = 4096 .. 32768 (a launch of fewer rows
// fills less than half of a 128-row block, and the IMAD kernel takes the last
// steps); at p = 512 the IMAD kernel measured faster at every size (4.7 times
// at N = 2048), so it takes all launches there unless the threshold is set.
static int64_t tc_default_min_rows(int p) {
  return (p == 1024 || p == 2048 || mpd::tcl_supports(p)) ? 64 : INT64_MAX;
}

// Large-precision tensor engine (p = 4096 .. 32768) for an update launch of
// `rows` rows?  It reads and writes the array with plain loads and stores (its
// TMA copies read only its own digit buffer), so a host-resident array is
// served too.
static bool use_tcl(mpdet_t h, int64_t rows) {
  if (h->pad) return false;                 // it rounds at the frame's own precision only
  if (h->flags & MPDET_BALL) return false;  // radii are kept by the IMAD kernels
  const int64_t thr = h->tc_min_rows >= 0 ? h->tc_min_rows : tc_default_min_rows(h->p);
  return h->engine >= 1 && mpd::tcl_supports(h->p) && rows >= thr;
}

// Tensor engine for an update launch of `rows` rows?
static bool use_tc(mpdet_t h, int64_t rows) {
  if (h->flags & MPDET_HOSTMEM) return false;  // its TMA copies address device memory only
  if (h->pad) return false;                    // it rounds at the frame's own precision only
  if (h->flags & MPDET_BALL) return false;     // radii are kept by the IMAD kernels
  const int64_t thr = h->tc_min_rows >= 0 ? h->tc_min_rows : tc_default_min_rows(h->p);
  return h->engine >= 1 && mpd::tc_supports(h->p, h->engine == 1) && rows >= thr;
}

// Default IMAD update geometry per limb count (-1 resolved): the kernel
// set's own unless the wide one measured faster.
static int default_upd_geom(int n) {
  (void)n;
  return 0;
}

// The IMAD Schur-update kernel the handle uses.
static mpd::UpdateFn imad_update(mpdet_t h) {
  if (h->pad || (h->flags & MPDET_BALL)) return h->ks->update_ext;  // frame rounding or radii
  if (h->kara && h->ks->update_kara) return h->ks->update_kara;
  const int g = h->upd_geom >= 0 ? h->upd_geom : default_upd_geom(h->n);
  if (g > 0) {
    mpd::UpdateFn f = mpd::update_wide_for(h->n, g == 1 ? 4 : 3);
    if (f) return f;
  }
  return h->ks->update[h->upd_variant];
}

// Enqueue one rank-1 update launch of the array A on stream st: single
// columns on the column kernel, long launches on the tensor engine where it
// exists, the rest on the IMAD kernel.  nsm: SMs the launch may fill.
static int launch_update(mpdet_t h, MpArr A, const UpdArgs& a, MpArr Z, int nsm, cudaStream_t st) {
  if (a.nrows <= 0 || a.ncols <= 0) return MPDET_OK;
  if (a.ncols == 1) {
    CU(h, h->ks->update_col(A, a, Z, h->status, h->p, st));
  } else if (use_tcl(h, a.nrows)) {
    if (!h->zd) {
      const size_t zb = mpd::tcl_zd_bytes(h->N, h->p);
      if (cudaMalloc(&h->zd, zb) != cudaSuccess) return fail(h, MPDET_ENOMEM, "digit buffer of %zu bytes", zb);
      CU(h, cudaMemsetAsync(h->zd, 0, zb, st));
    }
    if (!h->slab && cudaMalloc(&h->slab, mpd::tcl_slab_bytes(h->nsm, h->p)) != cudaSuccess)
      return fail(h, MPDET_ENOMEM, "product slab of %zu bytes", mpd::tcl_slab_bytes(h->nsm, h->p));
    CU(h, mpd::update_tcl(A, a, Z, h->status, h->p, nsm, st, h->zd, h->slab));
    h->launches += 1;  // the digit kernel
  } else if (use_tc(h, a.nrows)) {
    CU(h, mpd::update_tc(A, a, Z, h->status, h->p, nsm, st, h->engine == 1 ? 1 : 0));
  } else {
    CU(h, imad_update(h)(A, a, Z, h->status, h->p, nsm, st));
  }
  h->launches += 1;
  return MPDET_OK;
}

// The same, bracketed by a profiling event pair when profiling is on (the
// Schur update is the dominant kernel; its algorithmic work is counted).
static int timed_update(mpdet_t h, const UpdArgs& a, MpArr Z, int nsm, cudaStream_t st) {
  if (a.nrows <= 0 || a.ncols <= 0) return MPDET_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->profile) {
    int rc = next_event(h, &e0);
    if (!rc) rc = next_event(h, &e1);
    if (rc) return rc;
    CU(h, cudaEventRecord(e0, st));
  }
  int rc = launch_update(h, h->X, a, Z, nsm, st);
  if (rc) return rc;
  if (h->profile) {
    CU(h, cudaEventRecord(e1, st));
    h->upd_launches += 1;
    h->upd_products += (double)a.nrows * (double)a.ncols;
  }
  return MPDET_OK;
}

// Steps k (0-based) in [k0, k1), one after the other on the handle's stream:
// pivot, multipliers, update.
static int run_steps_serial(mpdet_t h, int64_t k0, int64_t k1) {
  const int lastcol = (h->flags & MPDET_LASTCOL) ? 1 : 0;
  const int64_t N = h->N;
  for (int64_t k = k0; k < k1; ++k) {
    CU(h, h->ks->pivot(h->X, N, k, h->D, h->R, h->status, h->zero_k, h->p, h->stream));
    h->launches += 1;
    if (k < N - 1) {
      CU(h, h->ks->mult(h->X, N, k, h->R, h->Z, h->status, h->p, lastcol, h->stream));
      h->launches += 1;
      int rc = timed_update(h, mpd::upd_step(N, k, lastcol), h->Z, h->nsm, h->stream);
      if (rc) return rc;
    }
  }
  return MPDET_OK;
}

// Steps k in [k0, k1) with look-ahead.  Step k+1 needs only column k+1 of
// step k's update before its pivot and multipliers, so the side stream T
// updates that column first and runs pivot and multipliers of step k+1 while
// the handle's stream S updates the rest of step k.  Order:
//   T: [rest of k-1 done] column k+1 of step k, pivot k+1, multipliers k+1
//   S: [multipliers k done] the rest of step k
// Multipliers alternate between Z (even steps) and Z2 (odd steps), since
// those of step k+1 are written while the rest of step k still reads step
// k's.  The last step of the window updates all its columns on S, so a
// window ends in the same state as without look-ahead; so do the results,
// which are the same operations on the same operands.
static int run_steps_lookahead(mpdet_t h, int64_t k0, int64_t k1) {
  const int lastcol = (h->flags & MPDET_LASTCOL) ? 1 : 0;
  const int64_t N = h->N;
  cudaStream_t S = h->stream, T = h->side;
  const MpArr Zb[2] = {h->Z, h->Z2};
  const int nsm_rest = h->nsm > 4 * h->la_reserve ? h->nsm - h->la_reserve : h->nsm;
  int rc = MPDET_OK;
  CU(h, cudaEventRecord(h->ev_rest, S));  // T starts after everything enqueued so far
  CU(h, cudaStreamWaitEvent(T, h->ev_rest, 0));
  CU(h, h->ks->pivot(h->X, N, k0, h->D, h->R, h->status, h->zero_k, h->p, T));
  h->launches += 1;
  if (k0 < N - 1) {
    CU(h, h->ks->mult(h->X, N, k0, h->R, Zb[k0 & 1], h->status, h->p, lastcol, T));
    h->launches += 1;
  }
  CU(h, cudaEventRecord(h->ev_mult, T));
  for (int64_t k = k0; k < k1 && k < N - 1; ++k) {
    const MpArr Zk = Zb[k & 1];
    CU(h, cudaStreamWaitEvent(S, h->ev_mult, 0));  // multipliers of step k
    if (k + 1 < k1) {
      CU(h, cudaStreamWaitEvent(T, h->ev_rest, 0));  // rest of step k-1
      rc = launch_update(h, h->X, mpd::upd_next(N, k), Zk, h->nsm, T);
      if (rc) return rc;
      CU(h, h->ks->pivot(h->X, N, k + 1, h->D, h->R, h->status, h->zero_k, h->p, T));
      h->launches += 1;
      if (k + 1 < N - 1) {
        CU(h, h->ks->mult(h->X, N, k + 1, h->R, Zb[(k + 1) & 1], h->status, h->p, lastcol, T));
        h->launches += 1;
      }
      CU(h, cudaEventRecord(h->ev_mult, T));
      rc = timed_update(h, mpd::upd_rest(N, k, lastcol), Zk, nsm_rest, S);
      if (rc) return rc;
      CU(h, cudaEventRecord(h->ev_rest, S));
    } else {
      rc = timed_update(h, mpd::upd_step(N, k, lastcol), Zk, h->nsm, S);
      if (rc) return rc;
    }
  }
  CU(h, cudaEventRecord(h->ev_mult, T));  // S continues after all of T's work
  CU(h, cudaStreamWaitEvent(S, h->ev_mult, 0));
  return MPDET_OK;
}

// enqueue steps k (0-based) in [k0, k1)
static int run_steps(mpdet_t h, int64_t k0, int64_t k1) {
  if (k1 <= k0) return MPDET_OK;
  int rc = h->lookahead ? run_steps_lookahead(h, k0, k1) : run_steps_serial(h, k0, k1);
  if (rc) return rc;
  h->k_done = k1;
  return MPDET_OK;
}

extern "C" int mpdet_tune(mpdet_t h, int param, int value) {
  if (!h) return MPDET_EINVAL;
  switch (param) {
    case MPDET_TUNE_UPDATE_VARIANT:
      if (value < 0 || value >= KernelSet::kUpdateVariants) return fail(h, MPDET_EINVAL, "tune: variant %d", value);
      h->upd_variant = value;
      return MPDET_OK;
    case MPDET_TUNE_ENGINE:
      if (value < 0 || value > 2) return fail(h, MPDET_EINVAL, "tune: engine %d", value);
      h->engine = value;
      return MPDET_OK;
    case MPDET_TUNE_TC_MIN_ROWS:
      if (value < 0) return fail(h, MPDET_EINVAL, "tune: tc_min_rows %d", value);
      h->tc_min_rows = value;
      return MPDET_OK;
    case MPDET_TUNE_LOOKAHEAD:
      if (value < 0 || value > 1) return fail(h, MPDET_EINVAL, "tune: lookahead %d", value);
      h->lookahead = value;
      return MPDET_OK;
    case MPDET_TUNE_LOOKAHEAD_RESERVE:
      if (value < 0 || value > 64) return fail(h, MPDET_EINVAL, "tune: lookahead reserve %d", value);
      h->la_reserve = value;
      return MPDET_OK;
    case MPDET_TUNE_UPDATE_GEOMETRY:
      if (value < -1 || value > 2) return fail(h, MPDET_EINVAL, "tune: update geometry %d", value);
      h->upd_geom = value;
      return MPDET_OK;
    case MPDET_TUNE_KARATSUBA:
      if (value < 0 || value > 1) return fail(h, MPDET_EINVAL, "tune: karatsuba %d", value);
      if (value && !h->ks->update_kara) return fail(h, MPDET_EINVAL, "tune: no Karatsuba update below p = 8192");
      h->kara = value;
      return MPDET_OK;
    default:
      return fail(h, MPDET_EINVAL, "tune: unknown parameter %d", param);
  }
}

extern "C" int mpdet_profile(mpdet_t h, int enable) {
  if (!h) return MPDET_EINVAL;
  h->profile = enable != 0;
  h->ev_used = 0;
  h->upd_ms = 0.0;
  h->upd_launches = 0;
  h->upd_products = 0.0;
  return MPDET_OK;
}

extern "C" int mpdet_profile_read(mpdet_t h, double* update_ms, int64_t* update_launches, double* update_limb_macs,
                                  int64_t* launches) {
  if (!h) return MPDET_EINVAL;
  CU(h, cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
    float ms = 0.f;
    CU(h, cudaEventElapsedTime(&ms, h->ev_pool[i], h->ev_pool[i + 1]));
    h->upd_ms += ms;
  }
  h->ev_used = 0;
  if (update_ms) *update_ms = h->upd_ms;
  if (update_launches) *update_launches = h->upd_launches;
  if (update_limb_macs) *update_limb_macs = h->upd_products * (double)h->nu * (double)h->nu;
  if (launches) *launches = h->launches;
  return MPDET_OK;
}

extern "C" int mpdet_factor_range(mpdet_t h, int64_t k0, int64_t k1) {
  if (!h) return MPDET_EINVAL;
  if (!h->have_matrix) return fail(h, MPDET_ESTATE, "factor_range: no matrix set");
  if (k0 != h->k_done || k1 < k0 || k1 > h->N)
    return fail(h, MPDET_ESTATE, "factor_range: window [%lld, %lld) but %lld steps done", (long long)k0, (long long)k1,
                (long long)h->k_done);
  int rc = run_steps(h, k0, k1);
  if (rc) return rc;
  CU(h, cudaGetLastError());
  return MPDET_OK;
}

extern "C" int mpdet_status(mpdet_t h, int64_t* zero_pivot_k) {
  if (!h) return MPDET_EINVAL;
  int st[4] = {0};
  int64_t zk[2] = {0};
  CU(h, cudaMemcpyAsync(st, h->status, 16, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaMemcpyAsync(zk, h->zero_k, 16, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (zero_pivot_k) *zero_pivot_k = zk[0];
  if (st[0] == MPDET_EZEROPIVOT) return fail(h, MPDET_EZEROPIVOT, "zero pivot at k = %lld", (long long)zk[0]);
  if (st[0] == MPDET_EZERODIV) return fail(h, MPDET_EZERODIV, "normalised minors: l_N1 is zero");
  return st[0];
}

extern "C" int mpdet_get_minors(mpdet_t h, mpdet_numv out, int device_ptr) {
  if (!h) return MPDET_EINVAL;
  int rc = copy_arr(h, h->D, out, h->N, device_ptr, false);
  if (rc) return rc;
  return finish_call(h, device_ptr);
}

extern "C" int mpdet_factor(mpdet_t h, mpdet_numv det, mpdet_numv minors, int64_t* zero_pivot_k, int device_ptr) {
  if (!h) return MPDET_EINVAL;
  if (!h->have_matrix) return fail(h, MPDET_ESTATE, "factor: no matrix set");
  int rc = run_steps(h, h->k_done, h->N);
  if (rc) return rc;
  MpArr last{h->D.s + (h->N - 1), h->D.e + (h->N - 1), h->D.m + (size_t)(h->N - 1) * h->n, h->pad};
  rc = copy_arr(h, last, det, 1, device_ptr, false);
  if (rc) return rc;
  rc = copy_arr(h, h->D, minors, h->N, device_ptr, false);
  if (rc) return rc;
  rc = finish_call(h, device_ptr);
  if (rc) return rc;
  if (device_ptr) {
    if (zero_pivot_k) *zero_pivot_k = -1;  // unknown until mpdet_status
    return MPDET_OK;
  }
  return mpdet_status(h, zero_pivot_k);
}

extern "C" int mpdet_lastcol_minors(mpdet_t h, mpdet_numv out, int normalised, int device_ptr) {
  if (!h) return MPDET_EINVAL;
  if (!(h->flags & MPDET_LASTCOL)) return fail(h, MPDET_ESTATE, "lastcol_minors: handle created without MPDET_LASTCOL");
  if (!h->have_matrix || h->k_done != h->N) return fail(h, MPDET_ESTATE, "lastcol_minors: factorisation not complete");
  if (!device_ptr) {  // device mode: the kernels skip on a bad status, read later by mpdet_status
    int64_t zk = 0;
    int st = mpdet_status(h, &zk);
    if (st == MPDET_EZEROPIVOT) return fail(h, MPDET_EZEROPIVOT, "lastcol_minors: zero pivot at k = %lld", (long long)zk);
    if (st) return st;
  }
  const int64_t N = h->N;
  if (N == 1) {  // C_11 = D_0 = 1, delta_{1,1} = 1
    uint32_t* one = new uint32_t[h->nu]();
    one[h->nu - 1] = 0x80000000u;
    int8_t s = 0;
    int64_t e = 1;
    cudaMemcpyKind k = device_ptr ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    cudaError_t ce = cudaMemcpy(out.limbs, one, h->nu * 4, k);
    if (ce == cudaSuccess) ce = cudaMemcpy(out.exp, &e, 8, k);
    if (ce == cudaSuccess) ce = cudaMemcpy(out.sign, &s, 1, k);
    if (ce == cudaSuccess) ce = set_rad(h->T, 1, false, h->stream);  // exactly 1
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    delete[] one;
    if (ce != cudaSuccess) return fail(h, MPDET_ECUDA, "lastcol N=1 copy: %s", cudaGetErrorString(ce));
    return MPDET_OK;
  }
  MpArr F;
  if (normalised) {
    // F = RN(1 / l_N1) into R; status 7 if l_N1 == 0
    CU(h, h->ks->recip1(h->X, (N - 1) * N, h->R, h->status, MPDET_EZERODIV, h->stream));
    h->launches += 1;
    F = h->R;
  } else {
    F = mpd::arr_at(h->D, N - 2, h->n);
  }
  CU(h, h->ks->lastcol(h->X, N, F, h->T, normalised, h->status, h->stream));
  h->launches += 1;
  if (normalised && !device_ptr) {
    int sts[4] = {0};
    CU(h, cudaMemcpyAsync(sts, h->status, 16, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    if (sts[0] == MPDET_EZERODIV) {
      CU(h, cudaMemsetAsync(h->status, 0, 16, h->stream));
      return fail(h, MPDET_EZERODIV, "normalised minors: l_N1 is zero");
    }
  }
  int rc = copy_arr(h, h->T, out, N, device_ptr, false);
  if (rc) return rc;
  return finish_call(h, device_ptr);
}

extern "C" int mpdet_minor_series(mpdet_t h, mpdet_numv out, int normalised, int device_ptr) {
  if (!h || !out.sign || !out.exp || !out.limbs) return fail(h, MPDET_EINVAL, "minor_series: null pointer");
  if (!(h->flags & MPDET_LASTCOL)) return fail(h, MPDET_ESTATE, "minor_series: handle created without MPDET_LASTCOL");
  if (!h->have_matrix || h->k_done != h->N) return fail(h, MPDET_ESTATE, "minor_series: factorisation not complete");
  const int64_t N = h->N, total = N * (N + 1) / 2;
  MpArr dst{out.sign, out.exp, out.limbs, h->pad};
  MpArr tmp{};
  if (!device_ptr || h->pad) {  // host output or another limb count: a device frame buffer of the triangle
    int rc = alloc_arr(h, &tmp, total);
    if (rc) {
      free_arr(&tmp);
      return rc;
    }
    dst = tmp;
  }
  MpArr F = h->D;
  cudaError_t ce = cudaSuccess;
  if (normalised) {
    // R[r] = RN(1/l_r0) for every row (1/0 gives +0): column 0 of the array
    // gathered into T, reciprocals into Z2 (both free once the elimination is done)
    const size_t nb = (size_t)h->n * 4;
    ce = cudaMemcpy2DAsync(h->T.m, nb, h->X.m, (size_t)N * nb, nb, (size_t)N, cudaMemcpyDeviceToDevice, h->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpy2DAsync(h->T.e, 8, h->X.e, (size_t)N * 8, 8, (size_t)N, cudaMemcpyDeviceToDevice, h->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpy2DAsync(h->T.s, 1, h->X.s, (size_t)N, 1, (size_t)N, cudaMemcpyDeviceToDevice, h->stream);
    if (ce == cudaSuccess) {
      ce = h->ks->ops(3, N, h->T, h->T, h->Z2, h->p, h->nsm, h->stream);
      h->launches += 1;
    }
    F = h->Z2;
  }
  if (ce == cudaSuccess) {
    ce = h->ks->series(h->X, N, F, normalised ? 1 : 0, dst, h->nsm, h->stream);
    h->launches += 1;
  }
  int rc = ce == cudaSuccess ? MPDET_OK : fail(h, MPDET_ECUDA, "k_series: %s", cudaGetErrorString(ce));
  if (!rc && tmp.m) {
    rc = copy_arr(h, tmp, out, total, device_ptr, false);
    if (!rc) rc = finish_call(h, device_ptr);
  } else if (!rc) {
    rc = finish_call(h, 1);
  }
  if (tmp.m || tmp.e || tmp.s) {
    cudaStreamSynchronize(h->stream);
    free_arr(&tmp);
  }
  return rc;
}

extern "C" int mpdet_get_entries(mpdet_t h, int64_t count, const int64_t* idx, mpdet_numv out, int device_ptr) {
  if (!h || count < 0 || (count > 0 && (!idx || !out.sign || !out.exp || !out.limbs)))
    return fail(h, MPDET_EINVAL, "get_entries: bad argument");
  const int64_t NN = h->N * h->N;
  for (int64_t q = 0; q < count; ++q)
    if (idx[q] < 0 || idx[q] >= NN) return fail(h, MPDET_EINVAL, "get_entries: index %lld out of range", (long long)idx[q]);
  const cudaMemcpyKind k = device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t nb = (size_t)h->nu * 4;
  for (int64_t q = 0; q < count; ++q) {
    const int64_t i = idx[q];
    CU(h, cudaMemcpyAsync(out.limbs + (size_t)q * h->nu, h->X.m + (size_t)i * h->n + h->pad, nb, k, h->stream));
    CU(h, cudaMemcpyAsync(out.exp + q, h->X.e + i, 8, k, h->stream));
    CU(h, cudaMemcpyAsync(out.sign + q, h->X.s + i, 1, k, h->stream));
  }
  return finish_call(h, device_ptr);
}

extern "C" int mpdet_radii(mpdet_t h, int which, uint32_t* rad_mant, int64_t* rad_exp, int device_ptr) {
  if (!h || which < 0 || which > 2 || !rad_mant || !rad_exp) return fail(h, MPDET_EINVAL, "radii: bad argument");
  if (!(h->flags & MPDET_BALL)) return fail(h, MPDET_ESTATE, "radii: handle created without MPDET_BALL");
  const MpArr& a = which == 0 ? h->D : which == 1 ? h->T : h->X;
  const int64_t count = which == 2 ? h->N * h->N : h->N;
  const cudaMemcpyKind k = device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CU(h, cudaMemcpyAsync(rad_mant, a.rm, (size_t)count * 4, k, h->stream));
  CU(h, cudaMemcpyAsync(rad_exp, a.re, (size_t)count * 8, k, h->stream));
  return finish_call(h, device_ptr);
}

extern "C" int mpdet_get_mp(mpdet_t h, mpdet_numv out, int device_ptr) {
  if (!h) return MPDET_EINVAL;
  int rc = copy_arr(h, h->X, out, h->N * h->N, device_ptr, false);
  if (rc) return rc;
  return finish_call(h, device_ptr);
}

extern "C" int mpdet_resume(mpdet_t h, mpdet_numv A, mpdet_numv minors, int64_t k_done, int device_ptr) {
  if (!h || k_done < 0 || k_done > h->N) return fail(h, MPDET_EINVAL, "resume: bad argument");
  if (h->flags & MPDET_BALL) return fail(h, MPDET_ESTATE, "resume: a checkpoint carries no radii (ball mode)");
  int rc = reset_state(h);
  if (rc) return rc;
  rc = copy_arr(h, h->X, A, h->N * h->N, device_ptr, true);
  if (rc) return rc;
  if (k_done > 0) {
    rc = copy_arr(h, h->D, minors, k_done, device_ptr, true);
    if (rc) return rc;
  }
  h->k_done = k_done;
  return finish_call(h, device_ptr);
}

// ---------------------------------------------------------------------------
// Adjoint (step a8): log|det| and d log|det| / dA = A^-T.
// ---------------------------------------------------------------------------
extern "C" int mpdet_logabsdet_grad(mpdet_t h, const double* A, int64_t ld, double* logabs, int* sign, double* grad,
                                    double grad_scale, int device_ptr) {
  if (!h || !A || !logabs || !sign) return fail(h, MPDET_EINVAL, "logabsdet_grad: null argument");
  if (grad && !(h->flags & MPDET_LASTCOL)) return fail(h, MPDET_ESTATE, "logabsdet_grad: gradient needs MPDET_LASTCOL");
  int rc = set_dense(h, A, ld, device_ptr, 0);
  if (rc) return rc;
  rc = run_steps(h, 0, h->N);
  if (rc) return rc;
  int64_t zk = 0;
  int st = mpdet_status(h, &zk);
  const int64_t N = h->N, n = h->n;
  // det = D_N on the host: log|det| = ln(m / 2^p) + e ln 2 in binary64
  int8_t ds = 0;
  int64_t de = 0;
  uint32_t top[2] = {0, 0};
  CU(h, cudaMemcpyAsync(&ds, h->D.s + (N - 1), 1, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaMemcpyAsync(&de, h->D.e + (N - 1), 8, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaMemcpyAsync(top, h->D.m + (size_t)(N - 1) * n + (n - 2), 8, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (de == INT64_MIN) {
    *logabs = -HUGE_VAL;
    *sign = 0;
    if (st) return st;
    return grad ? fail(h, MPDET_EZERODIV, "logabsdet_grad: singular matrix (det = 0), no gradient") : MPDET_OK;
  }
  *sign = ds ? -1 : 1;
  *logabs = log((double)top[1] * 0x1p-32 + (double)top[0] * 0x1p-64) + (double)de * 0.69314718055994530942;
  if (st) return st;
  if (!grad) return MPDET_OK;
  if (!h->S.m && alloc_arr(h, &h->S, N * N)) return MPDET_ENOMEM;
  CU(h, h->ks->init_s(h->X, N, h->S, h->nsm, h->stream));
  h->launches += 1;
  for (int64_t k = N - 1; k >= 0; --k) {
    CU(h, h->ks->recip1(h->X, k * N + k, h->R, h->status, MPDET_EZERODIV, h->stream));
    CU(h, h->ks->rowscale(h->S, N, k, h->R, h->stream));
    h->launches += 2;
    if (k > 0) {  // Z[0..k) = U column k, rows above the diagonal
      CU(h, cudaMemcpy2DAsync(h->Z.m, (size_t)n * 4, h->X.m + (size_t)k * n, (size_t)N * n * 4, (size_t)n * 4, (size_t)k,
                              cudaMemcpyDeviceToDevice, h->stream));
      CU(h, cudaMemcpy2DAsync(h->Z.e, 8, h->X.e + k, (size_t)N * 8, 8, (size_t)k, cudaMemcpyDeviceToDevice, h->stream));
      CU(h, cudaMemcpy2DAsync(h->Z.s, 1, h->X.s + k, (size_t)N, 1, (size_t)k, cudaMemcpyDeviceToDevice, h->stream));
      const int rc = launch_update(h, h->S, mpd::upd_back(N, k), h->Z, h->nsm, h->stream);
      if (rc) return rc;
    }
  }
  double* g = grad;
  if (!device_ptr) {
    size_t bytes = (size_t)N * N * 8;
    if (h->stage_bytes < bytes) {
      if (h->stage) cudaFree(h->stage);
      h->stage = nullptr;
      h->stage_bytes = 0;
      if (cudaMalloc(&h->stage, bytes) != cudaSuccess) return fail(h, MPDET_ENOMEM, "gradient staging");
      h->stage_bytes = bytes;
    }
    g = (double*)h->stage;
  }
  CU(h, h->ks->to_f64(h->S, N, g, grad_scale, h->p, 1, h->nsm, h->stream));
  h->launches += 1;
  if (!device_ptr) CU(h, cudaMemcpyAsync(grad, g, (size_t)N * N * 8, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return mpdet_status(h, nullptr);
}

// Copy out A^-1 (N*N numbers, row-major) computed by the last
// mpdet_logabsdet_grad call with a gradient.
extern "C" int mpdet_get_inverse(mpdet_t h, mpdet_numv out, int device_ptr) {
  if (!h) return MPDET_EINVAL;
  if (!h->S.m) return fail(h, MPDET_ESTATE, "get_inverse: no gradient computed yet");
  int rc = copy_arr(h, h->S, out, h->N * h->N, device_ptr, false);
  if (rc) return rc;
  return finish_call(h, device_ptr);
}

// Element-wise arithmetic on device arrays (diagnostics and tests).
extern "C" int mpdet_ops(int op, int64_t count, int32_t p_bits, mpdet_numv a, mpdet_numv b, mpdet_numv out,
                         void* cuda_stream) {
  int32_t n = 0;
  if (op < 0 || op > 3 || count < 0 || mpdet_geometry(p_bits, &n, nullptr, nullptr) != MPDET_OK) return MPDET_EINVAL;
  if (!a.sign || !a.exp || !a.limbs || !b.sign || !b.exp || !b.limbs || !out.sign || !out.exp || !out.limbs)
    return MPDET_EINVAL;
  const int nf = mpd::frame_limbs(n), pad = nf - n;
  const KernelSet* ks = mpd::kernel_set_for(nf);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MPDET_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  MpArr A{a.sign, a.exp, a.limbs}, B{b.sign, b.exp, b.limbs}, O{out.sign, out.exp, out.limbs};
  MpArr F[3] = {};
  cudaError_t e = cudaSuccess;
  if (pad) {  // operands of another limb count go through frame copies
    for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
      F[q].pad = pad;
      const int64_t c = count > 0 ? count : 1;
      e = cudaMalloc(&F[q].m, (size_t)c * nf * 4);
      if (e == cudaSuccess) e = cudaMalloc(&F[q].e, (size_t)c * 8);
      if (e == cudaSuccess) e = cudaMalloc(&F[q].s, (size_t)c);
    }
    if (e == cudaSuccess)
      e = mpd::copy_numbers(F[0], nf, a.sign, a.exp, a.limbs, n, count, true, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = mpd::copy_numbers(F[1], nf, b.sign, b.exp, b.limbs, n, count, true, cudaMemcpyDeviceToDevice, st);
    A = F[0];
    B = F[1];
    O = F[2];
  }
  if (e == cudaSuccess) e = ks->ops(op, count, A, B, O, 32 * nf, nsm, st);
  if (e == cudaSuccess && pad)
    e = mpd::copy_numbers(O, nf, out.sign, out.exp, out.limbs, n, count, false, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (MpArr& f : F) {
    if (f.m) cudaFree(f.m);
    if (f.e) cudaFree(f.e);
    if (f.s) cudaFree(f.s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MPDET_ECUDA;
  }
  return MPDET_OK;
}
