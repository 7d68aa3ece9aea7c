// Elimination kernels, templated on the slice width W and group size G
// (n = W*G limbs per number).  Each translation unit inst_*.cu instantiates
// one family of (W, G) and exports its launchers through a KernelSet.
//
// Matrix layout in HBM (one N x N array of numbers, row-major):
//   sign  int8   [N*N]
//   exp   int64  [N*N]
//   limbs uint32 [N*N][n]   (each number's n limbs contiguous, 16-byte aligned)
// A group of G lanes moves one number with uint4 loads of its slices.
#pragma once
#include <math_constants.h>

#include "ball.cuh"
#include "karatsuba.cuh"
#include "mpdev.cuh"
#include "kernelset.h"

namespace mpd {

// Per-group shared scratch for sub_round / recip_round (words).
template <int W, int G>
struct Scratch {
  static constexpr int n = W * G;
  static constexpr int words = ((n + 8 + 3) / 4) * 4 + 4;  // 16-byte multiple, odd-ish stride via +4
};

__device__ __forceinline__ int status_set(const int* status) { return *(volatile const int*)status; }

__host__ __device__ constexpr int upd_pad4(int w) { return (w + 3) / 4 * 4; }

// ---------------------------------------------------------------------------
// a1: exact lift of f64 / int32 entries.  value = (-1)^s * mant * 2^E with a
// mant of t significant bits becomes m = mant << (p - t), e = E + t; only the
// top two limbs of m can be non-zero (t <= 53).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void lift_u64(uint64_t mant, int64_t E, int& t_out, uint32_t& top1, uint32_t& top0) {
  int t = 64 - __clzll((long long)mant);
  uint64_t al = mant << (64 - t);  // top bit at bit 63
  top1 = (uint32_t)(al >> 32);
  top0 = (uint32_t)al;
  t_out = t;
  (void)E;
}

template <int W, int G>
__global__ void k_lift(const void* __restrict__ src, int kind, int64_t ld, int64_t N, MpArr X, int p) {
  constexpr int n = W * G;
  Grp<G> gp;
  const int64_t ngroups_total = (int64_t)gridDim.x * (blockDim.x / G);
  const int64_t grp0 = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
  for (int64_t idx = grp0; idx < N * N; idx += ngroups_total) {
    const int64_t i = idx / N, j = idx % N;
    uint64_t mant = 0;
    int64_t E = 0;
    int s = 0;
    if (kind == 0) {  // f64
      double v = reinterpret_cast<const double*>(src)[i * ld + j];
      uint64_t bits = (uint64_t)__double_as_longlong(v);
      s = (int)(bits >> 63);
      int be = (int)((bits >> 52) & 0x7ff);
      uint64_t fr = bits & ((1ull << 52) - 1);
      if (be == 0) {
        mant = fr;
        E = -1074;
      } else {
        mant = fr | (1ull << 52);
        E = be - 1075;
      }
    } else {  // int32
      int32_t v = reinterpret_cast<const int32_t*>(src)[i * ld + j];
      s = v < 0;
      mant = (uint64_t)(s ? -(int64_t)v : (int64_t)v);
      E = 0;
    }
    uint32_t L[W];
#pragma unroll
    for (int q = 0; q < W; ++q) L[q] = 0u;
    int8_t so = 0;
    int64_t eo = ZEXP;
    if (mant != 0) {
      int t;
      uint32_t t1, t0;
      lift_u64(mant, E, t, t1, t0);
      if (gp.g == G - 1) {
        L[W - 1] = t1;
        L[W - 2] = t0;
      }
      so = (int8_t)s;
      eo = E + t;
    }
    store_slice<W>(X.m + idx * n + gp.g * W, L);
    if (gp.g == 0) {
      X.s[idx] = so;
      X.e[idx] = eo;
    }
  }
}

// ---------------------------------------------------------------------------
// a1: Cauchy matrix A_ij = RN(1 / RN(x_i + y_j)), generated on the device.
// ---------------------------------------------------------------------------
template <int W, int G>
__device__ __forceinline__ void lift_f64_slice(const Grp<G>& gp, double v, int8_t& s, int64_t& e, uint32_t (&L)[W]) {
  uint64_t bits = (uint64_t)__double_as_longlong(v);
  int sg = (int)(bits >> 63);
  int be = (int)((bits >> 52) & 0x7ff);
  uint64_t fr = bits & ((1ull << 52) - 1);
  uint64_t mant = be ? (fr | (1ull << 52)) : fr;
  int64_t E = be ? (int64_t)be - 1075 : -1074;
#pragma unroll
  for (int q = 0; q < W; ++q) L[q] = 0u;
  if (mant == 0) {
    s = 0;
    e = ZEXP;
    return;
  }
  int t;
  uint32_t t1, t0;
  lift_u64(mant, E, t, t1, t0);
  if (gp.g == G - 1) {
    L[W - 1] = t1;
    L[W - 2] = t0;
  }
  s = (int8_t)sg;
  e = E + t;
}

template <int W, int G>
__global__ void k_cauchy(const double* __restrict__ x, const double* __restrict__ y, int64_t N, MpArr X, int p) {
  constexpr int n = W * G;
  constexpr int SW = Scratch<W, G>::words;
  extern __shared__ __align__(16) uint32_t smem[];
  Grp<G> gp;
  const int gib = threadIdx.x / G;
  uint32_t* buf = smem + gib * SW;
  // groups of one warp advance together so that the trip count is warp-uniform
  constexpr int GPW = 32 / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  const int64_t total = N * N;
  for (int64_t base = warp * GPW; base < total; base += nwarps * GPW) {
    int64_t idx = base + gp.lane / G;
    const bool active = idx < total;
    if (!active) idx = total - 1;
    const int64_t i = idx / N, j = idx % N;
    int8_t xs, ys;
    int64_t xe, ye;
    uint32_t XL[W], YL[W];
    lift_f64_slice<W, G>(gp, x[i], xs, xe, XL);
    lift_f64_slice<W, G>(gp, y[j], ys, ye, YL);
    // s = RN(x + y) = RN(x - (-y))
    sub_round<W, G>(gp, p, xs, xe, XL, (int8_t)(ys ^ (ye != ZEXP ? 1 : 0)), ye, YL, buf, X.pad);
    // ball mode: s = RN(x + y) of exact x, y; |s|_ for the reciprocal's radius
    const int pl = p - 32 * X.pad;
    Rad rs{}, los{};
    if (X.rm) {
      rs = ball_diff(pl, xe, rad_zero(), rad_zero());
      los = rad_mag<W, G>(gp, xe, XL, false);
    }
    uint32_t Mr[W];
    if (xe == ZEXP) {  // x_i + y_j == 0 has no reciprocal: divide a dummy, store +0
#pragma unroll
      for (int q = 0; q < W; ++q) XL[q] = 0u;
      if (gp.g == G - 1) XL[W - 1] = 0x80000000u;
    }
    const int adj = recip_round<W, G>(gp, XL, buf, Mr, X.pad);
    if (X.rm && active && gp.g == 0)
      rad_store(X.rm, X.re, idx, xe == ZEXP ? rad_zero() : ball_inv(pl, (int64_t)adj - xe, los, rs));
    if (active && xe != ZEXP) {
      store_slice<W>(X.m + idx * n + gp.g * W, Mr);
      if (gp.g == 0) {
        X.s[idx] = xs;
        X.e[idx] = (int64_t)adj - xe;
      }
    } else if (active) {  // x_i + y_j == 0: no reciprocal; mark by +0
      uint32_t Z[W];
#pragma unroll
      for (int q = 0; q < W; ++q) Z[q] = 0u;
      store_slice<W>(X.m + idx * n + gp.g * W, Z);
      if (gp.g == 0) {
        X.s[idx] = 0;
        X.e[idx] = ZEXP;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// a2: pivot of step k (0-based): D_k = RN(D_{k-1} * a_kk) (D_{-1} = 1),
// zero-pivot check, r_k = RN(1 / a_kk).  One warp; group 0 does the work.
// status[0]: 0 ok, MPDET_EZEROPIVOT once a zero pivot was met before the last
// step; *zero_k: 1-based index of the first zero pivot.
// ---------------------------------------------------------------------------
template <int W, int G>
__global__ void k_pivot(MpArr X, int64_t N, int64_t k, MpArr D, MpArr R, int* status, int64_t* zero_k, int p) {
  constexpr int n = W * G;
  constexpr int SW = Scratch<W, G>::words;
  __shared__ __align__(16) uint32_t sbuf[(32 / G) * SW];
  __shared__ __align__(16) uint32_t dprev[n];
  Grp<G> gp;
  const bool mine = threadIdx.x < G;  // group 0 of warp 0
  uint32_t* buf = sbuf + (threadIdx.x / G) * SW;
  const int64_t kk = k * N + k;
  uint32_t A[W];
  load_slice<W>(X.m + kk * n + gp.g * W, A);
  const int8_t as = X.s[kk];
  const int64_t ae = X.e[kk];
  // D_k
  uint32_t Dm[W];
  int8_t ds;
  int64_t de;
  if (k == 0) {
#pragma unroll
    for (int q = 0; q < W; ++q) Dm[q] = A[q];
    ds = as;
    de = ae;
  } else {
    for (int q = threadIdx.x; q < n; q += blockDim.x) dprev[q] = D.m[(k - 1) * n + q];
    __syncwarp();
    const int8_t ps = D.s[k - 1];
    const int64_t pe = D.e[k - 1];
    int adj = mul_round<W, G>(gp, A, dprev, Dm, X.pad);
    if (pe == ZEXP || ae == ZEXP) {
      ds = 0;
      de = ZEXP;
#pragma unroll
      for (int q = 0; q < W; ++q) Dm[q] = 0u;
    } else {
      ds = (int8_t)(ps ^ as);
      de = pe + ae + adj;
    }
  }
  if (mine) {
    store_slice<W>(D.m + k * n + gp.g * W, Dm);
    if (gp.g == 0) {
      D.s[k] = ds;
      D.e[k] = de;
    }
  }
  const bool already = status_set(status) != 0;
  const int pl = p - 32 * X.pad;
  if (X.rm) {  // ball mode: radius of D_k (unbounded once the elimination has stopped)
    const Rad ra = rad_load(X.rm, X.re, kk);
    const Rad my = rad_mag<W, G>(gp, ae, A, true);
    Rad rd;
    if (k == 0) {
      rd = ball_prod(pl, de, Rad{0x80000000u, 1}, rad_zero(), my, ra);  // D_0 = 1 exactly
    } else {
      const Rad mx = rad_mag_mem<W, G>(gp, D.e[k - 1], dprev, true);
      rd = ball_prod(pl, de, mx, rad_load(D.rm, D.re, k - 1), my, ra);
    }
    if (mine && gp.g == 0) rad_store(D.rm, D.re, k, already ? rad_unbounded() : rd);
  }
  if (ae == ZEXP && !already) {
    if (mine && gp.g == 0) {
      if (*zero_k == 0) *zero_k = k + 1;
      // MPDET_EZEROPIVOT with the 1-based step in the upper half, one store
      if (k < N - 1) *reinterpret_cast<volatile unsigned long long*>(status) = ((unsigned long long)(k + 1) << 32) | 4u;
    }
    return;
  }
  if (already || k == N - 1) return;
  uint32_t Mr[W];
  int adj = recip_round<W, G>(gp, A, buf, Mr, X.pad);
  Rad rr{};
  if (X.rm) rr = ball_inv(pl, (int64_t)adj - ae, rad_mag<W, G>(gp, ae, A, false), rad_load(X.rm, X.re, kk));
  if (mine) {
    store_slice<W>(R.m + gp.g * W, Mr);
    if (gp.g == 0) {
      R.s[0] = as;
      R.e[0] = (int64_t)adj - ae;
      if (X.rm) rad_store(R.rm, R.re, 0, rr);
    }
  }
}

// ---------------------------------------------------------------------------
// a3: multipliers z_i = RN(a_ik * r_k), i > k.  In lastcol mode the
// eliminated entry becomes l_ik = -z_ik (exact).
// ---------------------------------------------------------------------------
template <int W, int G>
__global__ void k_mult(MpArr X, int64_t N, int64_t k, MpArr R, MpArr Z, const int* status, int p, int lastcol) {
  constexpr int n = W * G;
  __shared__ __align__(16) uint32_t rm[n];
  if (status_set(status)) return;
  Grp<G> gp;
  for (int q = threadIdx.x; q < n; q += blockDim.x) rm[q] = R.m[q];
  __syncthreads();
  const int8_t rs = R.s[0];
  const int64_t re = R.e[0];
  const int gpb = blockDim.x / G;
  int64_t i = k + 1 + (int64_t)blockIdx.x * gpb + threadIdx.x / G;
  const bool active = i < N;
  if (!active) i = N - 1;
  const int64_t ik = i * N + k;
  uint32_t A[W], M[W];
  load_slice<W>(X.m + ik * n + gp.g * W, A);
  const int8_t as = X.s[ik];
  const int64_t ae = X.e[ik];
  int adj = mul_round<W, G>(gp, A, rm, M, X.pad);
  const bool zero = (ae == ZEXP);
  Rad rz{};
  if (X.rm)  // ball mode: z = RN(a_ik * r)
    rz = ball_prod(p - 32 * X.pad, zero ? ZEXP : ae + re + adj, rad_mag<W, G>(gp, ae, A, true),
                   rad_load(X.rm, X.re, ik), rad_mag_mem<W, G>(gp, re, rm, true), rad_load(R.rm, R.re, 0));
  if (zero) {
#pragma unroll
    for (int q = 0; q < W; ++q) M[q] = 0u;
  }
  if (active) {
    store_slice<W>(Z.m + i * n + gp.g * W, M);
    if (lastcol) store_slice<W>(X.m + ik * n + gp.g * W, M);
    if (gp.g == 0) {
      const int8_t zs = zero ? 0 : (int8_t)(as ^ rs);
      const int64_t ze = zero ? ZEXP : ae + re + adj;
      Z.s[i] = zs;
      Z.e[i] = ze;
      if (X.rm) rad_store(Z.rm, Z.re, i, rz);
      if (lastcol) {
        X.s[ik] = zero ? 0 : (int8_t)(zs ^ 1);
        X.e[ik] = ze;
        if (X.rm) rad_store(X.rm, X.re, ik, rz);  // l_ik = -z_ik: same radius
      }
    }
  }
}

// ---------------------------------------------------------------------------
// a4/a5 (and the adjoint's back substitution): rank-1 update
//   x_ij = RN(x_ij - RN(z_i * x_{brow,j}))
// for the rows and columns of an UpdArgs (kernelset.h).
// z_i is Z[i].  Block: GPB groups, each owning one column j and holding the
// pivot-row element x_{brow,j}'s slice in registers; the block walks rows
// [i0, i1) with the multipliers staged in shared memory (broadcast reads).
// ---------------------------------------------------------------------------
// An update launch stops once the elimination has: on any error, and on a
// zero pivot found at its own step or before.  A zero pivot of a later step
// does not stop it: with look-ahead the next step's pivot runs while this
// step's update does.  The pivot stores its 1-based step in the status word's
// upper half together with the code (one 64-bit store).
__device__ __forceinline__ bool upd_stopped(const int* status, const UpdArgs& a) {
  const unsigned long long w = *reinterpret_cast<volatile const unsigned long long*>(status);
  const int code = (int)(uint32_t)w;
  if (code == 0) return false;
  if (code != 4 || a.step < 0) return true;  // MPDET_EZEROPIVOT
  return (int64_t)(w >> 32) <= a.step + 1;
}

__device__ __forceinline__ int64_t upd_col(const UpdArgs& a, int64_t c) { return a.j0 + c + (c >= a.hole ? a.hw : 0); }

// EXT: the instantiation for precisions held in a larger frame (X.pad > 0)
// and for the ball mode's radii; the others round at the frame's end and keep
// no radii, so the hot path carries neither.  KARA: the products by one
// Karatsuba level (mul_round_kara, 3n words of scratch per group after the
// per-group scratch) instead of the schoolbook mul_round; the same bits.
template <int W, int G, int MINB, bool EXT, bool KARA = false>
__global__ void __launch_bounds__(128, MINB) k_update(MpArr X, UpdArgs a, MpArr Z, const int* status, int p,
                                                     int rows_per_cta) {
  constexpr int n = W * G;
  constexpr int SW = Scratch<W, G>::words;
  extern __shared__ __align__(16) uint32_t smem[];
  if (upd_stopped(status, a)) return;
  Grp<G> gp;
  const int64_t N = a.N;
  const int gpb = blockDim.x / G;
  const int gib = threadIdx.x / G;
  // shared layout (words, every region a multiple of 4 words = 16 bytes):
  //   z mantissas rows*n | z exponents 2*rows (+pad) | z signs rows bytes (+pad) | per-group scratch
  uint32_t* zbuf = smem;
  int64_t* ze_s = reinterpret_cast<int64_t*>(smem + rows_per_cta * n);
  int8_t* zs_s = reinterpret_cast<int8_t*>(smem + rows_per_cta * n + upd_pad4(2 * rows_per_cta));
  uint32_t* buf = smem + rows_per_cta * n + upd_pad4(2 * rows_per_cta) + upd_pad4((rows_per_cta + 3) / 4) + gib * SW;
  uint32_t* kscr = smem + rows_per_cta * n + upd_pad4(2 * rows_per_cta) + upd_pad4((rows_per_cta + 3) / 4) +
                   (blockDim.x / G) * SW + gib * (KARA ? 3 * n : 0);
  const int64_t ncols = a.ncols;
  const int64_t i0 = a.row0 + (int64_t)blockIdx.y * rows_per_cta;
  const int64_t rend = a.row0 + a.nrows;
  const int64_t i1 = (i0 + rows_per_cta < rend) ? i0 + rows_per_cta : rend;
  const int nr = (int)(i1 - i0);
  // stage multipliers
  for (int q = threadIdx.x; q < nr * n / 4; q += blockDim.x)
    reinterpret_cast<uint4*>(zbuf)[q] = reinterpret_cast<const uint4*>(Z.m + i0 * n)[q];
  for (int q = threadIdx.x; q < nr; q += blockDim.x) {
    ze_s[q] = Z.e[i0 + q];
    zs_s[q] = Z.s[i0 + q];
  }
  __syncthreads();
  int64_t c = (int64_t)blockIdx.x * gpb + gib;
  const bool active = c < ncols;
  if (!active) c = ncols - 1;
  const int64_t j = upd_col(a, c);
  // pivot-row element x_{brow,j}
  const int64_t kj = a.brow * N + j;
  uint32_t Bk[W];
  load_slice<W>(X.m + kj * n + gp.g * W, Bk);
  const int8_t bs = X.s[kj];
  const int64_t be = X.e[kj];
  const int pad = EXT ? X.pad : 0;
  const bool ball = EXT && X.rm != nullptr;
  const int pl = p - 32 * pad;
  Rad mb{}, rb{};
  if (ball) {  // ball mode: |b|^ and the radius of the pivot-row element
    mb = rad_mag<W, G>(gp, be, Bk, true);
    rb = rad_load(X.rm, X.re, kj);
  }
#pragma unroll 1
  for (int r = 0; r < nr; ++r) {
    const int64_t ij = (i0 + r) * N + j;
    uint32_t Xv[W], T[W];
    int8_t xs = X.s[ij];
    int64_t xe = X.e[ij];
    const int64_t zer = ze_s[r];
    Rad mz{};
    if (ball) mz = rad_mag_mem<W, G>(gp, zer, zbuf + r * n, true);
    int adj;
    if constexpr (KARA)
      adj = mul_round_kara<W, G>(gp, Bk, zbuf + r * n, T, kscr, pad);
    else
      adj = mul_round<W, G>(gp, Bk, zbuf + r * n, T, pad);
    load_slice<W>(X.m + ij * n + gp.g * W, Xv);
    const bool tz = (zer == ZEXP) || (be == ZEXP);
    const int8_t ts = tz ? 0 : (int8_t)(zs_s[r] ^ bs);
    const int64_t te = tz ? ZEXP : zer + be + adj;
    if (tz) {
#pragma unroll
      for (int q = 0; q < W; ++q) T[q] = 0u;
    }
    sub_round<W, G>(gp, p, xs, xe, Xv, ts, te, T, buf, pad);
    if (active) {
      store_slice<W>(X.m + ij * n + gp.g * W, Xv);
      if (gp.g == 0) {
        if (ball) {  // t = RN(z b), then x - t
          const Rad rt = ball_prod(pl, te, mz, rad_load(Z.rm, Z.re, i0 + r), mb, rb);
          rad_store(X.rm, X.re, ij, ball_diff(pl, xe, rad_load(X.rm, X.re, ij), rt));
        }
        X.s[ij] = xs;
        X.e[ij] = xe;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The same update for a single column (a.ncols == 1): one group per row, so
// that the column k+1 of a look-ahead step spreads over as many groups as it
// has rows instead of occupying one group per block.
// ---------------------------------------------------------------------------
template <int W, int G>
__global__ void k_update_col(MpArr X, UpdArgs a, MpArr Z, const int* status, int p) {
  constexpr int n = W * G;
  constexpr int SW = Scratch<W, G>::words;
  __shared__ __align__(16) uint32_t sbuf[(128 / G) * SW];
  if (upd_stopped(status, a)) return;
  Grp<G> gp;
  const int64_t N = a.N;
  const int64_t j = upd_col(a, 0);
  int64_t r = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
  const bool active = r < a.nrows;
  if (!active) r = a.nrows - 1;
  const int64_t i = a.row0 + r;
  const int64_t kj = a.brow * N + j, ij = i * N + j;
  uint32_t Bk[W], Xv[W], T[W];
  load_slice<W>(X.m + kj * n + gp.g * W, Bk);
  const int8_t bs = X.s[kj];
  const int64_t be = X.e[kj];
  int8_t xs = X.s[ij];
  int64_t xe = X.e[ij];
  const int64_t zer = Z.e[i];
  const int8_t zs = Z.s[i];
  Rad mb{}, mz{};
  if (X.rm) {
    mb = rad_mag<W, G>(gp, be, Bk, true);
    mz = rad_mag_mem<W, G>(gp, zer, Z.m + i * n, true);
  }
  const int adj = mul_round<W, G>(gp, Bk, Z.m + i * n, T, X.pad);
  load_slice<W>(X.m + ij * n + gp.g * W, Xv);
  const bool tz = (zer == ZEXP) || (be == ZEXP);
  const int8_t ts = tz ? 0 : (int8_t)(zs ^ bs);
  const int64_t te = tz ? ZEXP : zer + be + adj;
  if (tz) {
#pragma unroll
    for (int q = 0; q < W; ++q) T[q] = 0u;
  }
  sub_round<W, G>(gp, p, xs, xe, Xv, ts, te, T, sbuf + (threadIdx.x / G) * SW, X.pad);
  if (active) {
    store_slice<W>(X.m + ij * n + gp.g * W, Xv);
    if (gp.g == 0) {
      if (X.rm) {
        const int pl = p - 32 * X.pad;
        const Rad rt = ball_prod(pl, te, mz, rad_load(Z.rm, Z.re, i), mb, rad_load(X.rm, X.re, kj));
        rad_store(X.rm, X.re, ij, ball_diff(pl, xe, rad_load(X.rm, X.re, ij), rt));
      }
      X.s[ij] = xs;
      X.e[ij] = xe;
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint helpers.
// k_init_s: S = L from a lastcol elimination X (l_ij below the diagonal, 1 on
// it, +0 above).  k_rowscale: row k of S times the reciprocal R[0]:
// X_kc = RN(S_kc * r_k).  k_to_f64: G_ij = scale * RN64(X_ji), binary64 round
// to nearest even with subnormals (quantum 2^max(e-53, -1074)).
// ---------------------------------------------------------------------------
template <int W, int G>
__global__ void k_init_s(MpArr X, int64_t N, MpArr S) {
  constexpr int n = W * G;
  Grp<G> gp;
  const int64_t ngroups_total = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t idx = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; idx < N * N; idx += ngroups_total) {
    const int64_t i = idx / N, j = idx % N;
    uint32_t L[W];
    int8_t s = 0;
    int64_t e = ZEXP;
    if (j < i) {
      load_slice<W>(X.m + idx * n + gp.g * W, L);
      s = X.s[idx];
      e = X.e[idx];
    } else {
#pragma unroll
      for (int q = 0; q < W; ++q) L[q] = 0u;
      if (j == i) {
        if (gp.g == G - 1) L[W - 1] = 0x80000000u;
        e = 1;
      }
    }
    store_slice<W>(S.m + idx * n + gp.g * W, L);
    if (gp.g == 0) {
      S.s[idx] = s;
      S.e[idx] = e;
    }
  }
}

template <int W, int G>
__global__ void k_rowscale(MpArr S, int64_t N, int64_t k, MpArr R) {
  constexpr int n = W * G;
  __shared__ __align__(16) uint32_t rm[n];
  Grp<G> gp;
  for (int q = threadIdx.x; q < n; q += blockDim.x) rm[q] = R.m[q];
  __syncthreads();
  const int8_t rs = R.s[0];
  const int64_t re = R.e[0];
  int64_t c = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
  const bool active = c < N;
  if (!active) c = N - 1;
  const int64_t kc = k * N + c;
  uint32_t A[W], M[W];
  load_slice<W>(S.m + kc * n + gp.g * W, A);
  const int8_t as = S.s[kc];
  const int64_t ae = S.e[kc];
  const int adj = mul_round<W, G>(gp, A, rm, M, S.pad);
  if (active) {
    const bool zero = (ae == ZEXP) || (re == ZEXP);
    if (zero) {
#pragma unroll
      for (int q = 0; q < W; ++q) M[q] = 0u;
    }
    store_slice<W>(S.m + kc * n + gp.g * W, M);
    if (gp.g == 0) {
      S.s[kc] = zero ? 0 : (int8_t)(as ^ rs);
      S.e[kc] = zero ? ZEXP : ae + re + adj;
    }
  }
}

template <int W, int G>
__global__ void k_to_f64(MpArr Xs, int64_t N, double* __restrict__ out, double scale, int p, int transpose) {
  constexpr int n = W * G;
  static_assert(W >= 2, "the top two limbs live in one lane");
  Grp<G> gp;
  const int64_t ngroups_total = (int64_t)gridDim.x * (blockDim.x / G);
  constexpr int GPW = 32 / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  (void)ngroups_total;
  for (int64_t base = warp * GPW; base < N * N; base += nwarps * GPW) {
    int64_t idx = base + gp.lane / G;
    const bool active = idx < N * N;
    if (!active) idx = N * N - 1;
    const int64_t i = idx / N, j = idx % N;
    const int64_t src = transpose ? j * N + i : idx;
    uint32_t M[W];
    load_slice<W>(Xs.m + src * n + gp.g * W, M);
    const int8_t s = Xs.s[src];
    const int64_t e = Xs.e[src];
    // lower limbs (all but the top two) for the sticky bit
    bool low = false;
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (!(gp.g == G - 1 && q >= W - 2)) low |= (M[q] != 0u);
    const bool lowany = gp.ballot(low) != 0u;
    const uint64_t hi64 = ((uint64_t)gp.from(M[W - 1], G - 1) << 32) | gp.from(M[W - 2], G - 1);
    double v;
    if (e == ZEXP) v = 0.0;
    else if (e > 1100) v = s ? -CUDART_INF : CUDART_INF;
    else if (e < -1100) v = s ? -0.0 : 0.0;
    else {
      const int64_t q = (e - 53 < -1074) ? -1074 : e - 53;
      const int64_t t = (int64_t)p + q - e - (p - 64);  // right shift of hi64 (>= 11)
      const uint64_t K0 = t < 64 ? (hi64 >> t) : 0ull;
      const uint32_t rbit = (t - 1 < 64) ? (uint32_t)((hi64 >> (t - 1)) & 1ull) : 0u;
      const bool st = lowany || ((t - 1 < 64) ? (hi64 & ((1ull << (t - 1)) - 1ull)) != 0ull : hi64 != 0ull);
      const uint64_t K = K0 + ((rbit && (st || (K0 & 1ull))) ? 1ull : 0ull);
      v = ldexp((double)K, (int)q);
      if (s) v = -v;
    }
    if (active && gp.g == 0) out[idx] = v * scale;
  }
}

// ---------------------------------------------------------------------------
// a6: last-column minors.  out_j = RN(f * l_Nj) for j < N-1 (0-based), where
// f = D_{N-1} (signed minors C_jN) or f = RN(1/l_N1) (normalised minors,
// then out_0 = 1 exactly); out_{N-1} = D_{N-1} or RN(1/l_N1) respectively.
// F holds f (one number).  Threads: groups over j.
// ---------------------------------------------------------------------------
template <int W, int G>
__global__ void k_lastcol(MpArr X, int64_t N, MpArr F, MpArr out, int normalised, const int* status) {
  constexpr int n = W * G;
  __shared__ __align__(16) uint32_t fm[n];
  if (status_set(status)) return;  // zero pivot or zero l_N1: outputs are not defined
  Grp<G> gp;
  for (int q = threadIdx.x; q < n; q += blockDim.x) fm[q] = F.m[q];
  __syncthreads();
  const int8_t fs = F.s[0];
  const int64_t fe = F.e[0];
  const int gpb = blockDim.x / G;
  int64_t j = (int64_t)blockIdx.x * gpb + threadIdx.x / G;
  const bool active = j < N;
  if (!active) j = N - 1;
  const int64_t Nj = (N - 1) * N + j;
  uint32_t L[W], M[W];
  load_slice<W>(X.m + Nj * n + gp.g * W, L);
  const int8_t ls = X.s[Nj];
  const int64_t le = X.e[Nj];
  int adj = mul_round<W, G>(gp, L, fm, M, X.pad);
  Rad ml{}, mf{};
  if (X.rm) {
    ml = rad_mag<W, G>(gp, le, L, true);
    mf = rad_mag_mem<W, G>(gp, fe, fm, true);
  }
  int8_t os;
  int64_t oe;
  if (le == ZEXP || fe == ZEXP) {
    os = 0;
    oe = ZEXP;
#pragma unroll
    for (int q = 0; q < W; ++q) M[q] = 0u;
  } else {
    os = (int8_t)(ls ^ fs);
    oe = le + fe + adj;
  }
  if (j == N - 1) {  // C_NN = D_{N-1}; delta_{N,N} = RN(1/l_N1): both are f itself
#pragma unroll
    for (int q = 0; q < W; ++q) M[q] = fm[gp.g * W + q];
    os = fs;
    oe = fe;
  }
  if (normalised && j == 0) {  // delta_{N,1} = 1
#pragma unroll
    for (int q = 0; q < W; ++q) M[q] = 0u;
    if (gp.g == G - 1) M[W - 1] = 0x80000000u;
    os = 0;
    oe = 1;
  }
  if (active) {
    store_slice<W>(out.m + j * n + gp.g * W, M);
    if (gp.g == 0) {
      out.s[j] = os;
      out.e[j] = oe;
      if (X.rm) {  // C_jN = RN(D_{N-1} l_Nj); normalised: RN(l_Nj r), delta_1 = 1 exactly
        const int pl = (int)(32 * n) - 32 * X.pad;
        const Rad rf = rad_load(F.rm, F.re, 0), rl = rad_load(X.rm, X.re, Nj);
        Rad ro = normalised ? ball_prod(pl, oe, ml, rl, mf, rf) : ball_prod(pl, oe, mf, rf, ml, rl);
        if (j == N - 1) ro = rf;
        if (normalised && j == 0) ro = rad_zero();
        rad_store(out.rm, out.re, j, ro);
      }
    }
  }
}

// Series of last-column minors for every leading size (Sec. 3: the series
// of minor arrays for N = 2, 3, ...; at step n row n of L holds the minors of
// the n x n leading matrix up to a factor).  Row r of L (0-based) is final
// after step r, and the elimination of the leading (r+1) x (r+1) block is the
// same rounded sequence, so series r holds
//   C^(r+1)_{j,r} = RN(D_r * l_rj),  j < r;   C^(r+1)_{r,r} = D_r,
// with D_r the leading minor of size r (D[r-1]; D_0 = 1), or, normalised,
//   delta_j = RN(l_rj * R[r]),  0 < j < r;   delta_0 = 1;   delta_r = R[r],
// with R[r] = RN(1/l_r0) (+0 when l_r0 = 0: that series is then all +0).
// out is the packed triangle: series r at offset r(r+1)/2.  A zero pivot at
// step kz leaves D_kz.. = +0, so every later unnormalised series is +0.
// Grid-stride over the triangle; the trip count is uniform per block, so
// every lane takes part in the group shuffles of mul_round.
template <int W, int G>
__global__ void k_series(MpArr X, int64_t N, MpArr F, int normalised, MpArr out) {
  constexpr int n = W * G;
  Grp<G> gp;
  const int64_t total = N * (N + 1) / 2;
  const int gpb = blockDim.x / G;
  for (int64_t t0 = (int64_t)blockIdx.x * gpb; t0 < total; t0 += (int64_t)gridDim.x * gpb) {
    int64_t t = t0 + threadIdx.x / G;
    const bool active = t < total;
    if (!active) t = total - 1;
    int64_t r = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (r > 0 && r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    const int64_t j = t - r * (r + 1) / 2;
    const int64_t fi = normalised ? r : (r > 0 ? r - 1 : 0);
    const int64_t xj = r * N + j;
    uint32_t L[W], M[W];
    load_slice<W>(X.m + xj * n + gp.g * W, L);
    const int8_t ls = X.s[xj];
    const int64_t le = X.e[xj];
    const int8_t fs = F.s[fi];
    const int64_t fe = F.e[fi];
    const int adj = mul_round<W, G>(gp, L, F.m + fi * n, M, X.pad);
    int8_t os;
    int64_t oe;
    if (le == ZEXP || fe == ZEXP) {
      os = 0;
      oe = ZEXP;
#pragma unroll
      for (int q = 0; q < W; ++q) M[q] = 0u;
    } else {
      os = (int8_t)(ls ^ fs);
      oe = le + fe + adj;
    }
    const bool one = r == 0 || (normalised && j == 0 && fe != ZEXP);
    if (one) {  // C^(1)_{1,1} = D_0 = 1; delta_0 = 1
#pragma unroll
      for (int q = 0; q < W; ++q) M[q] = 0u;
      if (gp.g == G - 1) M[W - 1] = 0x80000000u;
      os = 0;
      oe = 1;
    } else if (j == r) {  // C^(r+1)_{r,r} = D_r; delta_r = RN(1/l_r0)
      load_slice<W>(F.m + fi * n + gp.g * W, M);
      os = fs;
      oe = fe;
    }
    if (active) {
      store_slice<W>(out.m + t * n + gp.g * W, M);
      if (gp.g == 0) {
        out.s[t] = os;
        out.e[t] = oe;
      }
    }
  }
}

// RN(1/src[idx]) into dst[0]; one warp, group 0.  Sets *status = code when
// src[idx] is zero.
template <int W, int G>
__global__ void k_recip1(MpArr src, int64_t idx, MpArr dst, int* status, int code) {
  constexpr int n = W * G;
  constexpr int SW = Scratch<W, G>::words;
  __shared__ __align__(16) uint32_t sbuf[(32 / G) * SW];
  Grp<G> gp;
  uint32_t A[W], M[W];
  load_slice<W>(src.m + idx * n + gp.g * W, A);
  const int8_t as = src.s[idx];
  const int64_t ae = src.e[idx];
  if (ae == ZEXP) {
    if (threadIdx.x == 0) *status = code;
    return;
  }
  int adj = recip_round<W, G>(gp, A, sbuf + (threadIdx.x / G) * SW, M, src.pad);
  Rad rr{};
  if (src.rm)
    rr = ball_inv((int)(32 * n) - 32 * src.pad, (int64_t)adj - ae, rad_mag<W, G>(gp, ae, A, false),
                  rad_load(src.rm, src.re, idx));
  if (threadIdx.x < G) {
    store_slice<W>(dst.m + gp.g * W, M);
    if (gp.g == 0) {
      dst.s[0] = as;
      dst.e[0] = (int64_t)adj - ae;
      if (src.rm) rad_store(dst.rm, dst.re, 0, rr);
    }
  }
}


// ---------------------------------------------------------------------------
// a7: batch.  One persistent launch factors many independent matrices of
// uneven N (det and leading minors; no pivoting, no L).  Each 128-thread
// block takes the next matrix from an atomic queue (the host orders it by
// decreasing N, so the longest jobs start first) and runs every step of its
// elimination with block barriers between the phases: pivot (warp 0),
// multipliers and the Schur update (all groups, flattened over the items).
// Z: per-block multiplier scratch of max_n numbers.
// ---------------------------------------------------------------------------
struct BatchDesc {
  const int64_t* N;      // size of matrix m
  const int64_t* xoff;   // first number of matrix m in X
  const int64_t* doff;   // first number of D_1 of matrix m in D
  const int32_t* order;  // processing order
  int64_t* zero_k;       // first zero pivot of matrix m (1-based), 0 if none
  int* queue;            // next position in order (zeroed before the launch)
  int64_t count;
  int64_t max_n;
};

// The pivot phase (one warp) runs in its own lane geometry (PW limbs per lane,
// PG lanes per number, PW * PG = n): the long division's serial chain per
// quotient limb shortens with the slice width, as in the single-matrix path.
template <int W, int G, int PW, int PG>
__global__ void __launch_bounds__(128, 4) k_batch(MpArr Xall, MpArr Dall, MpArr Zall, BatchDesc bd, int p) {
  constexpr int n = W * G;
  static_assert(PW * PG == n, "the pivot geometry holds the same numbers");
  constexpr int SW = Scratch<W, G>::words;
  constexpr int NG = 128 / G;  // groups per block
  constexpr int SBUF = NG * SW > (32 / PG) * SW ? NG * SW : (32 / PG) * SW;
  __shared__ __align__(16) uint32_t sbuf[SBUF];
  __shared__ __align__(16) uint32_t r_m[n];
  __shared__ int64_t r_e;
  __shared__ int8_t r_s;
  __shared__ int s_job, s_zero;
  Grp<G> gp;
  const int pad = Xall.pad;
  const int gid = threadIdx.x / G;
  uint32_t* buf = sbuf + gid * SW;
  MpArr Z{Zall.s + blockIdx.x * bd.max_n, Zall.e + blockIdx.x * bd.max_n, Zall.m + (size_t)blockIdx.x * bd.max_n * n};
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(bd.queue, 1);
    __syncthreads();
    const int job = s_job;
    __syncthreads();
    if (job >= bd.count) break;
    const int m = bd.order[job];
    const int64_t N = bd.N[m];
    MpArr X{Xall.s + bd.xoff[m], Xall.e + bd.xoff[m], Xall.m + (size_t)bd.xoff[m] * n};
    MpArr D{Dall.s + bd.doff[m], Dall.e + bd.doff[m], Dall.m + (size_t)bd.doff[m] * n};
    for (int64_t k = 0; k < N; ++k) {
      const int64_t kk = k * N + k;
      if (threadIdx.x < 32) {  // warp 0: pivot
        Grp<PG> pg;
        uint32_t A[PW], Dm[PW];
        load_slice<PW>(X.m + kk * n + pg.g * PW, A);
        const int8_t as = X.s[kk];
        const int64_t ae = X.e[kk];
        int8_t ds = as;
        int64_t de = ae;
        if (k == 0) {
#pragma unroll
          for (int q = 0; q < PW; ++q) Dm[q] = A[q];
        } else {
          const int adj = mul_round<PW, PG>(pg, A, D.m + (k - 1) * n, Dm, pad);
          const int8_t ps = D.s[k - 1];
          const int64_t pe = D.e[k - 1];
          if (pe == ZEXP || ae == ZEXP) {
            ds = 0;
            de = ZEXP;
#pragma unroll
            for (int q = 0; q < PW; ++q) Dm[q] = 0u;
          } else {
            ds = (int8_t)(ps ^ as);
            de = pe + ae + adj;
          }
        }
        if (threadIdx.x < PG) {
          store_slice<PW>(D.m + k * n + pg.g * PW, Dm);
          if (pg.g == 0) {
            D.s[k] = ds;
            D.e[k] = de;
          }
        }
        if (threadIdx.x == 0) s_zero = (ae == ZEXP);
        if (ae != ZEXP && k < N - 1) {  // warp-uniform: every lane read the same pivot
          uint32_t Mr[PW];
          const int adj = recip_round<PW, PG>(pg, A, sbuf + (threadIdx.x / PG) * SW, Mr, pad);
          if (threadIdx.x < PG) {
            store_slice<PW>(r_m + pg.g * PW, Mr);
            if (pg.g == 0) {
              r_s = as;
              r_e = (int64_t)adj - ae;
            }
          }
        }
      }
      __syncthreads();
      if (s_zero) {
        if (threadIdx.x == 0) bd.zero_k[m] = k + 1;
        // D_k is +0 already; D_{k+1}..D_N are +0 too
        for (int64_t q = k + 1 + threadIdx.x; q < N; q += blockDim.x) {
          D.s[q] = 0;
          D.e[q] = ZEXP;
          for (int l = 0; l < n; ++l) D.m[q * n + l] = 0u;
        }
        __syncthreads();
        break;
      }
      if (k == N - 1) break;
      if (threadIdx.x == 0) bd.zero_k[m] = 0;
      const int64_t R = N - k - 1;
      // multipliers z_i = RN(a_ik * r_k)
      for (int64_t t0 = 0; t0 < R; t0 += NG) {
        int64_t t = t0 + gid;
        const bool active = t < R;
        if (!active) t = R - 1;
        const int64_t i = k + 1 + t, ik = i * N + k;
        uint32_t A[W], M[W];
        load_slice<W>(X.m + ik * n + gp.g * W, A);
        const int adj = mul_round<W, G>(gp, A, r_m, M, pad);
        const int64_t ae = X.e[ik];
        if (active) {
          const bool zero = (ae == ZEXP);
          if (zero) {
#pragma unroll
            for (int q = 0; q < W; ++q) M[q] = 0u;
          }
          store_slice<W>(Z.m + i * n + gp.g * W, M);
          if (gp.g == 0) {
            Z.s[i] = zero ? 0 : (int8_t)(X.s[ik] ^ r_s);
            Z.e[i] = zero ? ZEXP : ae + r_e + adj;
          }
        }
      }
      __syncthreads();
      // Schur update of the trailing R x R block, items (i, j) flattened; the
      // group's item t = t0 + gid advances by NG, its row and column follow
      // without a division per item
      const int64_t items = R * R;
      int64_t ti = gid / R, tj = gid % R;
      for (int64_t t0 = 0; t0 < items; t0 += NG) {
        const bool active = t0 + gid < items;
        const int64_t i = k + 1 + (active ? ti : R - 1), j = k + 1 + (active ? tj : R - 1);
        tj += NG;
        while (tj >= R) {
          tj -= R;
          ++ti;
        }
        const int64_t kj = k * N + j, ij = i * N + j;
        uint32_t Bk[W], T[W], Xv[W];
        load_slice<W>(X.m + kj * n + gp.g * W, Bk);
        const int8_t bs = X.s[kj];
        const int64_t be = X.e[kj];
        const int64_t zer = Z.e[i];
        const int adj = mul_round<W, G>(gp, Bk, Z.m + i * n, T, pad);
        const bool tz = (zer == ZEXP) || (be == ZEXP);
        const int8_t ts = tz ? 0 : (int8_t)(Z.s[i] ^ bs);
        const int64_t te = tz ? ZEXP : zer + be + adj;
        if (tz) {
#pragma unroll
          for (int q = 0; q < W; ++q) T[q] = 0u;
        }
        load_slice<W>(X.m + ij * n + gp.g * W, Xv);
        int8_t xs = X.s[ij];
        int64_t xe = X.e[ij];
        sub_round<W, G>(gp, p, xs, xe, Xv, ts, te, T, buf, pad);
        if (active) {
          store_slice<W>(X.m + ij * n + gp.g * W, Xv);
          if (gp.g == 0) {
            X.s[ij] = xs;
            X.e[ij] = xe;
          }
        }
      }
      __syncthreads();
    }
  }
}


// ---------------------------------------------------------------------------
// Element-wise operations on arrays of numbers (diagnostics and tests of the
// arithmetic core): op 0: RN(a*b), 1: RN(a-b), 2: RN(a+b), 3: RN(1/a).
// ---------------------------------------------------------------------------
template <int W, int G>
__global__ void k_ops(int op, int64_t count, MpArr A, MpArr B, MpArr O, int p) {
  constexpr int n = W * G;
  constexpr int SW = Scratch<W, G>::words;
  constexpr int GPW = 32 / G;
  extern __shared__ __align__(16) uint32_t smem[];
  Grp<G> gp;
  uint32_t* buf = smem + (threadIdx.x / G) * SW;
  uint32_t* zb = smem + (blockDim.x / G) * SW + (threadIdx.x / G) * n;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t base = warp * GPW; base < count; base += nwarps * GPW) {
    int64_t idx = base + gp.lane / G;
    const bool active = idx < count;
    if (!active) idx = count - 1;
    uint32_t a[W], b[W], o[W];
    load_slice<W>(A.m + idx * n + gp.g * W, a);
    load_slice<W>(B.m + idx * n + gp.g * W, b);
    int8_t as = A.s[idx], bs = B.s[idx], os = 0;
    int64_t ae = A.e[idx], be = B.e[idx], oe = ZEXP;
    if (op == 0) {
      store_slice<W>(zb + gp.g * W, b);
      __syncwarp();
      const int adj = mul_round<W, G>(gp, a, zb, o, A.pad);
      __syncwarp();
      if (ae == ZEXP || be == ZEXP) {
#pragma unroll
        for (int q = 0; q < W; ++q) o[q] = 0u;
      } else {
        os = (int8_t)(as ^ bs);
        oe = ae + be + adj;
      }
    } else if (op == 1 || op == 2) {
      const int8_t bsx = (op == 2 && be != ZEXP) ? (int8_t)(bs ^ 1) : bs;  // a + b = a - (-b)
      sub_round<W, G>(gp, p, as, ae, a, bsx, be, b, buf, A.pad);
#pragma unroll
      for (int q = 0; q < W; ++q) o[q] = a[q];
      os = as;
      oe = ae;
    } else {
      const bool z = (ae == ZEXP);
      if (z) {  // no reciprocal of zero: divide a dummy, report +0
#pragma unroll
        for (int q = 0; q < W; ++q) a[q] = 0u;
        if (gp.g == G - 1) a[W - 1] = 0x80000000u;
      }
      const int adj = recip_round<W, G>(gp, a, buf, o, A.pad);
      if (z) {
#pragma unroll
        for (int q = 0; q < W; ++q) o[q] = 0u;
      } else {
        os = as;
        oe = (int64_t)adj - ae;
      }
    }
    if (active) {
      store_slice<W>(O.m + idx * n + gp.g * W, o);
      if (gp.g == 0) {
        O.s[idx] = os;
        O.e[idx] = oe;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <int W, int G>
struct Launch {
  static constexpr int n = W * G;
  static constexpr int SW = Scratch<W, G>::words;
  static constexpr int NT = 128;  // threads per block (4 warps)

  static cudaError_t lift(const void* src, int kind, int64_t ld, int64_t N, MpArr X, int p, int nsm, cudaStream_t st) {
    int64_t groups = N * N;
    int64_t blocks = (groups + NT / G - 1) / (NT / G);
    int64_t cap = (int64_t)nsm * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_lift<W, G><<<(unsigned)blocks, NT, 0, st>>>(src, kind, ld, N, X, p);
    return cudaGetLastError();
  }
  static cudaError_t cauchy(const double* x, const double* y, int64_t N, MpArr X, int p, int nsm, cudaStream_t st) {
    int64_t groups = N * N;
    int64_t blocks = (groups + NT / G - 1) / (NT / G);
    int64_t cap = (int64_t)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    size_t sm = (size_t)(NT / G) * SW * 4;
    cudaFuncSetAttribute(k_cauchy<W, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_cauchy<W, G><<<(unsigned)blocks, NT, sm, st>>>(x, y, N, X, p);
    return cudaGetLastError();
  }
  static cudaError_t pivot(MpArr X, int64_t N, int64_t k, MpArr D, MpArr R, int* status, int64_t* zk, int p,
                           cudaStream_t st) {
    k_pivot<W, G><<<1, 32, 0, st>>>(X, N, k, D, R, status, zk, p);
    return cudaGetLastError();
  }
  static cudaError_t mult(MpArr X, int64_t N, int64_t k, MpArr R, MpArr Z, const int* status, int p, int lastcol,
                          cudaStream_t st) {
    int64_t rows = N - k - 1;
    if (rows <= 0) return cudaSuccess;
    int64_t blocks = (rows + NT / G - 1) / (NT / G);
    k_mult<W, G><<<(unsigned)blocks, NT, 0, st>>>(X, N, k, R, Z, status, p, lastcol);
    return cudaGetLastError();
  }
  static size_t update_smem(int rows_per_cta, bool kara = false) {
    return (size_t)(rows_per_cta * n + upd_pad4(2 * rows_per_cta) + upd_pad4((rows_per_cta + 3) / 4) + (NT / G) * SW +
                    (kara ? (NT / G) * 3 * n : 0)) * 4;
  }
  template <int MINB, bool EXT = false, bool KARA = false>
  static cudaError_t update(MpArr X, const UpdArgs& a, MpArr Z, const int* status, int p, int nsm, cudaStream_t st) {
    const int64_t ncols = a.ncols;
    const int64_t rows = a.nrows;
    if (rows <= 0 || ncols <= 0) return cudaSuccess;
    const int gpb = NT / G;
    int64_t bx = (ncols + gpb - 1) / gpb;
    // rows per block: enough blocks for ~4 waves of 4 blocks per SM
    int64_t target = (int64_t)nsm * 16;
    int64_t by_needed = (target + bx - 1) / bx;
    int64_t rpc = (rows + by_needed - 1) / by_needed;
    int64_t rmax = 32;
    const size_t cap = KARA ? 112 * 1024 : 96 * 1024;
    while (rmax > 1 && update_smem((int)rmax, KARA) > cap) rmax /= 2;
    if (rpc > rmax) rpc = rmax;
    if (rpc < 1) rpc = 1;
    int64_t by = (rows + rpc - 1) / rpc;
    size_t sm = update_smem((int)rpc, KARA);
    cudaFuncSetAttribute(k_update<W, G, MINB, EXT, KARA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((unsigned)bx, (unsigned)by);
    k_update<W, G, MINB, EXT, KARA><<<grid, NT, sm, st>>>(X, a, Z, status, p, (int)rpc);
    return cudaGetLastError();
  }
  static cudaError_t update_col(MpArr X, const UpdArgs& a, MpArr Z, const int* status, int p, cudaStream_t st) {
    if (a.ncols != 1) return cudaErrorInvalidValue;
    if (a.nrows <= 0) return cudaSuccess;
    const int64_t blocks = (a.nrows + NT / G - 1) / (NT / G);
    k_update_col<W, G><<<(unsigned)blocks, NT, 0, st>>>(X, a, Z, status, p);
    return cudaGetLastError();
  }
  static cudaError_t init_s(MpArr X, int64_t N, MpArr S, int nsm, cudaStream_t st) {
    int64_t blocks = (N * N + NT / G - 1) / (NT / G);
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
    k_init_s<W, G><<<(unsigned)blocks, NT, 0, st>>>(X, N, S);
    return cudaGetLastError();
  }
  static cudaError_t rowscale(MpArr S, int64_t N, int64_t k, MpArr R, cudaStream_t st) {
    int64_t blocks = (N + NT / G - 1) / (NT / G);
    k_rowscale<W, G><<<(unsigned)blocks, NT, 0, st>>>(S, N, k, R);
    return cudaGetLastError();
  }
  static cudaError_t to_f64(MpArr X, int64_t N, double* out, double scale, int p, int transpose, int nsm,
                            cudaStream_t st) {
    int64_t blocks = (N * N + NT / G - 1) / (NT / G);
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
    k_to_f64<W, G><<<(unsigned)blocks, NT, 0, st>>>(X, N, out, scale, p, transpose);
    return cudaGetLastError();
  }
  static cudaError_t lastcol(MpArr X, int64_t N, MpArr F, MpArr out, int normalised, const int* status,
                             cudaStream_t st) {
    int64_t blocks = (N + NT / G - 1) / (NT / G);
    k_lastcol<W, G><<<(unsigned)blocks, NT, 0, st>>>(X, N, F, out, normalised, status);
    return cudaGetLastError();
  }
  static cudaError_t series(MpArr X, int64_t N, MpArr F, int normalised, MpArr out, int nsm, cudaStream_t st) {
    const int64_t total = N * (N + 1) / 2;
    int64_t blocks = (total + NT / G - 1) / (NT / G);
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
    k_series<W, G><<<(unsigned)blocks, NT, 0, st>>>(X, N, F, normalised, out);
    return cudaGetLastError();
  }
  static cudaError_t recip1(MpArr src, int64_t idx, MpArr dst, int* status, int code, cudaStream_t st) {
    k_recip1<W, G><<<1, 32, 0, st>>>(src, idx, dst, status, code);
    return cudaGetLastError();
  }
  template <int PW, int PG>
  static cudaError_t batch_p(MpArr X, MpArr D, MpArr Z, const BatchDescHost& h, int p, int blocks,
                             cudaStream_t st) {
    BatchDesc bd{h.N, h.xoff, h.doff, h.order, h.zero_k, h.queue, h.count, h.max_n};
    k_batch<W, G, PW, PG><<<blocks, 128, 0, st>>>(X, D, Z, bd, p);
    return cudaGetLastError();
  }
  template <int PW, int PG>
  static int batch_blocks_per_sm_p() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<W, G, PW, PG>, 128, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
  }
  static cudaError_t ops(int op, int64_t count, MpArr A, MpArr B, MpArr O, int p, int nsm, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + NT / G - 1) / (NT / G);
    if (blocks > (int64_t)nsm * 8) blocks = (int64_t)nsm * 8;
    size_t sm = (size_t)(NT / G) * (SW + n) * 4;
    cudaFuncSetAttribute(k_ops<W, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_ops<W, G><<<(unsigned)blocks, NT, sm, st>>>(op, count, A, B, O, p);
    return cudaGetLastError();
  }
  static KernelSet make() {
    KernelSet s;
    s.W = W;
    s.G = G;
    s.PW = W;
    s.PG = G;
    s.lift = &lift;
    s.cauchy = &cauchy;
    s.pivot = &pivot;
    s.mult = &mult;
    s.update[0] = &update<3>;
    s.update[1] = &update<4>;
    s.update[2] = &update<5>;
    s.update[3] = &update<6>;
    s.update_ext = &update<4, true>;
    if constexpr (W >= 16 && n >= 256) s.update_kara = &update<3, false, true>;
    s.update_col = &update_col;
    s.lastcol = &lastcol;
    s.recip1 = &recip1;
    s.series = &series;
    s.batch = &batch_p<W, G>;
    s.ops = &ops;
    s.init_s = &init_s;
    s.rowscale = &rowscale;
    s.to_f64 = &to_f64;
    s.batch_blocks_per_sm = &batch_blocks_per_sm_p<W, G>;
    return s;
  }
  // The same set with the pivot and the single reciprocal taken from the
  // family (PW, PG), PW * PG = n.  Both run one long division per launch on
  // one group, a serial chain whose length per quotient limb grows with the
  // slice width, so the narrowest slices (W = 4 while n <= 128) give the
  // shortest step.
  template <int PW, int PG>
  static KernelSet make_with_pivot() {
    static_assert(PW * PG == n, "the pivot family holds the same numbers");
    KernelSet s = make();
    s.PW = PW;
    s.PG = PG;
    s.pivot = &Launch<PW, PG>::pivot;
    s.recip1 = &Launch<PW, PG>::recip1;
    s.batch = &batch_p<PW, PG>;
    s.batch_blocks_per_sm = &batch_blocks_per_sm_p<PW, PG>;
    return s;
  }
};

}  // namespace mpd
