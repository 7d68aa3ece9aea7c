// Internal interface between the C-ABI layer and the per-(W, G) kernel
// instantiations.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpd {

// Structure-of-arrays view of numbers in device memory (n limbs each).  pad:
// the precision is p = 32 (n - pad) bits; a precision whose limb count is not
// one of the kernel families' sizes is held in the next family's frame of n
// limbs, mantissa in the top n - pad limbs and the low pad limbs zero, and
// every operation rounds at that position (0: the whole frame).
// rm, re: the ball mode's radii (mantissa, exponent) of the same numbers,
// or null when the array carries none.
struct MpArr {
  int8_t* s;
  int64_t* e;
  uint32_t* m;
  int pad = 0;
  uint32_t* rm = nullptr;
  int64_t* re = nullptr;
};

// Numbers [off, off + count) of a, radii included (n limbs each).
inline MpArr arr_at(const MpArr& a, int64_t off, int n) {
  MpArr v{a.s + off, a.e + off, a.m + (size_t)off * n, a.pad};
  if (a.rm) {
    v.rm = a.rm + off;
    v.re = a.re + off;
  }
  return v;
}

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

// One rank-1 update launch (Alg. 1 step 2.2.2, and the adjoint's back
// substitution):
//   x_ij = RN(x_ij - RN(z_i * x_{brow,j})),   i in [row0, row0 + nrows),
// over the columns j = j0 + c + (c >= hole ? hw : 0), c in [0, ncols): a run
// of columns with at most one gap of hw columns (the pivot column in lastcol
// mode, and with look-ahead also column k+1, which a separate launch updates
// first).  z_i is Z[i].  step: the 0-based elimination step of the launch,
// or -1 for the back substitution.
struct UpdArgs {
  int64_t N, brow, row0, nrows;
  int64_t j0, hole, ncols;
  int64_t step;
  int hw;
};

// Every column of step k's Schur update: j > k, or j != k in lastcol mode
// (which also carries L's row segment j < k).
inline UpdArgs upd_step(int64_t N, int64_t k, int lastcol) {
  return lastcol ? UpdArgs{N, k, k + 1, N - k - 1, 0, k, N - 1, k, 1}
                 : UpdArgs{N, k, k + 1, N - k - 1, k + 1, INT64_MAX, N - k - 1, k, 0};
}
// Column k+1 of step k alone (k + 1 < N): all the next pivot and the next
// multipliers need.
inline UpdArgs upd_next(int64_t N, int64_t k) { return UpdArgs{N, k, k + 1, N - k - 1, k + 1, INT64_MAX, 1, k, 0}; }
// The rest of step k: j > k + 1, or j not in {k, k + 1} in lastcol mode.
inline UpdArgs upd_rest(int64_t N, int64_t k, int lastcol) {
  return lastcol ? UpdArgs{N, k, k + 1, N - k - 1, 0, k, N - 2, k, 2}
                 : UpdArgs{N, k, k + 1, N - k - 1, k + 2, INT64_MAX, N - k - 2, k, 0};
}
// Back substitution of the adjoint: rows [0, k), every column, pivot row k.
inline UpdArgs upd_back(int64_t N, int64_t k) { return UpdArgs{N, k, 0, k, 0, INT64_MAX, N, -1, 0}; }

typedef cudaError_t (*UpdateFn)(MpArr X, const UpdArgs& a, MpArr Z, const int* status, int p, int nsm,
                                cudaStream_t st);

// Schur update with 32 limbs per lane for n = 64 .. 512 (updwide_*.cu),
// compiled for at least minb (3 or 4) resident 128-thread blocks per SM, or
// nullptr: the wide alternative to a kernel set's own update geometry.
UpdateFn update_wide_a(int n, int minb);
UpdateFn update_wide_b(int n, int minb);
inline UpdateFn update_wide_for(int n, int minb) {
  UpdateFn f = update_wide_a(n, minb);
  return f ? f : update_wide_b(n, minb);
}

struct KernelSet {
  int W, G;
  int PW, PG;  // lane geometry of the pivot and the single reciprocal (PW * PG = W * G)
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
  cudaError_t (*update[kUpdateVariants])(MpArr X, const UpdArgs& a, MpArr Z, const int* status, int p, int nsm,
                                         cudaStream_t st);
  // the same for numbers held in a larger frame (MpArr::pad > 0) or with
  // radii (ball mode): the update[] kernels are compiled without either
  cudaError_t (*update_ext)(MpArr X, const UpdArgs& a, MpArr Z, const int* status, int p, int nsm, cudaStream_t st);
  // the update with its products by one Karatsuba level (n >= 256 only, else
  // null): the same bits, a tuning choice (MPDET_TUNE_KARATSUBA)
  cudaError_t (*update_kara)(MpArr X, const UpdArgs& a, MpArr Z, const int* status, int p, int nsm, cudaStream_t st) =
      nullptr;
  // single-column launch (a.ncols == 1), one group per row
  cudaError_t (*update_col)(MpArr X, const UpdArgs& a, MpArr Z, const int* status, int p, cudaStream_t st);
  cudaError_t (*lastcol)(MpArr X, int64_t N, MpArr F, MpArr out, int normalised, const int* status,
                         cudaStream_t st);
  cudaError_t (*recip1)(MpArr src, int64_t idx, MpArr dst, int* status, int code, cudaStream_t st);
  // last-column minors of every leading size (packed triangle of N(N+1)/2
  // numbers); F = D (unnormalised) or R[r] = RN(1/l_r0) (normalised)
  cudaError_t (*series)(MpArr X, int64_t N, MpArr F, int normalised, MpArr out, int nsm, cudaStream_t st);
  // persistent batch kernel (blocks = resident blocks to launch)
  cudaError_t (*batch)(MpArr X, MpArr D, MpArr Z, const BatchDescHost& bd, int p, int blocks, cudaStream_t st);
  int (*batch_blocks_per_sm)();
  // element-wise arithmetic (diagnostics)
  cudaError_t (*ops)(int op, int64_t count, MpArr A, MpArr B, MpArr O, int p, int nsm, cudaStream_t st);
  // adjoint (X = U^-1 L by back substitution with update[], and the binary64 gradient)
  cudaError_t (*init_s)(MpArr X, int64_t N, MpArr S, int nsm, cudaStream_t st);
  cudaError_t (*rowscale)(MpArr S, int64_t N, int64_t k, MpArr R, cudaStream_t st);
  cudaError_t (*to_f64)(MpArr X, int64_t N, double* out, double scale, int p, int transpose, int nsm,
                        cudaStream_t st);
};


// Tensor-core engine of the rank-1 update (tc_update.cu): p = 512, 1024, 2048
// with the warp-specialised kernel (pipelined = 1: tensor core, epilogue and
// subtraction overlap), p = 2048 one role at a time (pipelined = 0).  nsm: the
// SMs the launch may fill (one block each).
bool tc_supports(int p, int pipelined);
cudaError_t update_tc(MpArr X, const UpdArgs& a, MpArr Z, int* status, int p, int nsm, cudaStream_t st,
                      int pipelined);

// Tensor-core engine of the rank-1 update for p = 4096 .. 32768 (tc_large.cu):
// 8-bit digits of z against 4-bit digits of b, the multipliers' digits
// precomputed per launch into zd (tcl_zd_bytes(N, p) bytes), the staged
// products in slab (tcl_slab_bytes(nsm, p) bytes).  nsm: the SMs the launch
// may fill (one block each).
bool tcl_supports(int p);
size_t tcl_zd_bytes(int64_t N, int p);
size_t tcl_slab_bytes(int nsm, int p);
cudaError_t update_tcl(MpArr X, const UpdArgs& a, MpArr Z, int* status, int p, int nsm, cudaStream_t st, void* zd,
                       uint32_t* slab);

// Kernel set for n = p/32 limbs, or nullptr if this n is not instantiated.
const KernelSet* kernel_set_for(int n);

// Limbs of the frame that holds numbers of nu limbs (2 <= nu <= 1024): the
// smallest kernel family size >= nu (powers of two from 4).
inline int frame_limbs(int nu) {
  int nf = 4;
  while (nf < nu) nf *= 2;
  return nf;
}

// Copy count numbers between a caller's arrays (nu limbs per number) and a
// frame array of nf >= nu limbs per number, whose mantissas sit in the top nu
// limbs with the low nf - nu limbs zero.  to_frame: caller -> frame (the low
// limbs are cleared), else frame -> caller.  A null caller pointer skips that
// field.  Asynchronous on st.
inline cudaError_t copy_numbers(MpArr f, int nf, int8_t* s, int64_t* e, uint32_t* m, int nu, int64_t count,
                                bool to_frame, cudaMemcpyKind kind, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  cudaError_t r = cudaSuccess;
  const int pad = nf - nu;
  if (m) {
    if (pad == 0) {
      r = to_frame ? cudaMemcpyAsync(f.m, m, (size_t)count * nf * 4, kind, st)
                   : cudaMemcpyAsync(m, f.m, (size_t)count * nf * 4, kind, st);
    } else if (to_frame) {
      r = cudaMemset2DAsync(f.m, (size_t)nf * 4, 0, (size_t)pad * 4, (size_t)count, st);
      if (r == cudaSuccess)
        r = cudaMemcpy2DAsync(f.m + pad, (size_t)nf * 4, m, (size_t)nu * 4, (size_t)nu * 4, (size_t)count, kind, st);
    } else {
      r = cudaMemcpy2DAsync(m, (size_t)nu * 4, f.m + pad, (size_t)nf * 4, (size_t)nu * 4, (size_t)count, kind, st);
    }
  }
  if (r == cudaSuccess && e)
    r = to_frame ? cudaMemcpyAsync(f.e, e, (size_t)count * 8, kind, st) : cudaMemcpyAsync(e, f.e, (size_t)count * 8, kind, st);
  if (r == cudaSuccess && s)
    r = to_frame ? cudaMemcpyAsync(f.s, s, (size_t)count, kind, st) : cudaMemcpyAsync(s, f.s, (size_t)count, kind, st);
  return r;
}

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
