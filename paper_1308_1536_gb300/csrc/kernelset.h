// Internal interface between the C-ABI layer and the per-(W, G) kernel
// instantiations.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpd {

// Structure-of-arrays view of numbers in device memory (n limbs each).
struct MpArr {
  int8_t* s;
  int64_t* e;
  uint32_t* m;
};

// Device pointers describing a batch of independent matrices.
struct BatchDescHost {
  const int64_t* N;
  const int64_t* xoff;
  const int64_t* doff;
  const int32_t* order;
  int64_t* zero_k;
  int* queue;
  int64_t count;
  int64_t max_n;
};

struct KernelSet {
  int W, G;
  // kind 0: double entries, 1: int32 entries
  cudaError_t (*lift)(const void* src, int kind, int64_t ld, int64_t N, MpArr X, int p, int nsm, cudaStream_t st);
  cudaError_t (*cauchy)(const double* x, const double* y, int64_t N, MpArr X, int p, int nsm, cudaStream_t st);
  cudaError_t (*pivot)(MpArr X, int64_t N, int64_t k, MpArr D, MpArr R, int* status, int64_t* zk, int p,
                       cudaStream_t st);
  cudaError_t (*mult)(MpArr X, int64_t N, int64_t k, MpArr R, MpArr Z, const int* status, int p, int lastcol,
                      cudaStream_t st);
  // Schur update, one entry per register budget: variant v is compiled for
  // at least 3 + v resident 128-thread blocks per SM
  static constexpr int kUpdateVariants = 4;
  cudaError_t (*update[kUpdateVariants])(MpArr X, int64_t N, int64_t k, MpArr Z, const int* status, int p,
                                         int lastcol, int nsm, cudaStream_t st);
  cudaError_t (*lastcol)(MpArr X, int64_t N, MpArr F, MpArr out, int normalised, const int* status,
                         cudaStream_t st);
  cudaError_t (*recip1)(MpArr src, int64_t idx, MpArr dst, int* status, int code, cudaStream_t st);
  // persistent batch kernel (blocks = resident blocks to launch)
  cudaError_t (*batch)(MpArr X, MpArr D, MpArr Z, const BatchDescHost& bd, int p, int blocks, cudaStream_t st);
  int (*batch_blocks_per_sm)();
  // element-wise arithmetic (diagnostics)
  cudaError_t (*ops)(int op, int64_t count, MpArr A, MpArr B, MpArr O, int p, int nsm, cudaStream_t st);
  // adjoint (back substitution X = U^-1 L and the binary64 gradient)
  cudaError_t (*usolve_update)(MpArr S, int64_t N, int64_t k, MpArr Z, const int* status, int p, int nsm,
                               cudaStream_t st);
  cudaError_t (*init_s)(MpArr X, int64_t N, MpArr S, int nsm, cudaStream_t st);
  cudaError_t (*rowscale)(MpArr S, int64_t N, int64_t k, MpArr R, cudaStream_t st);
  cudaError_t (*to_f64)(MpArr X, int64_t N, double* out, double scale, int p, int transpose, int nsm,
                        cudaStream_t st);
};

struct UpdArgs;  // kernels.cuh

// Tensor-core engine of the rank-1 update, p = 2048 only (tc_update.cu).
bool tc_supports(int p, int pipelined);
// pipelined = 1: warp-specialised kernel (tensor core, epilogue and subtraction overlap); 0: one role at a time
cudaError_t update_tc_p2048_step(MpArr X, int64_t N, int64_t k, MpArr Z, int* status, int p, int lastcol, int nsm,
                                 cudaStream_t st, int pipelined);
cudaError_t usolve_tc_p2048(MpArr S, int64_t N, int64_t k, MpArr Z, int* status, int p, int nsm, cudaStream_t st,
                            int pipelined);

// Kernel set for n = p/32 limbs, or nullptr if this n is not instantiated.
const KernelSet* kernel_set_for(int n);

// one translation unit per (W, G): inst_w<W>_g<G>.cu
#define MPD_DECLARE_SET(W, G) const KernelSet* kernel_set_w##W##_g##G();
MPD_DECLARE_SET(4, 1)
MPD_DECLARE_SET(8, 1)
MPD_DECLARE_SET(16, 1)
MPD_DECLARE_SET(16, 2)
MPD_DECLARE_SET(16, 4)
MPD_DECLARE_SET(16, 8)
MPD_DECLARE_SET(16, 16)
MPD_DECLARE_SET(16, 32)
MPD_DECLARE_SET(32, 32)
#undef MPD_DECLARE_SET

}  // namespace mpd
