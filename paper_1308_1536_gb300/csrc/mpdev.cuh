// Device multiprecision arithmetic for the elimination kernels (sm_103a).
//
// Number format: x = (-1)^s * m * 2^(e-p), m in [2^(p-1), 2^p) held as
// n = p/32 little-endian uint32 limbs, e an int64; zero is s = 0, m = 0,
// e = INT64_MIN.  Every operation is the exact result rounded to nearest,
// ties to even, at p bits (the method works at one fixed precision
// throughout, Sec. 4.3).  A precision of fewer limbs than the frame the
// routines work in (n = W*G) keeps its mantissa in the top limbs of the frame
// with the low `pad` limbs zero (the same value with the same exponent); the
// routines then round at limb pad instead of limb 0 (round_frame).
//
// Work split: one number is owned by a GROUP of G consecutive lanes of a warp
// (G in {1,2,4,8,16,32}); lane g of the group holds the W-limb SLICE
// [g*W, (g+1)*W) of a mantissa in registers, n = G*W.  Carries between the
// slices are resolved with warp ballots (generate/propagate masks), never by
// serial hand-offs.  All shuffles and ballots are executed by all 32 lanes
// (groups take data-dependent decisions with selects, not branches), so the
// full-warp mask is always valid.
//
// Limb products: mul.wide.u32 (one 32x32->64 multiply on the IMAD pipe) with
// the low and high words folded into the accumulator by two add-with-carry
// chains.  On sm_103a mad.hi.u32 issues at half the rate of mad.lo.u32, so
// this split keeps the IMAD pipe at two slots per limb product and moves the
// additions to the ALU pipe.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpd {

constexpr int64_t ZEXP = INT64_MIN;
constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Carry-chain primitives.  Each is one PTX instruction; the carry flag lives
// between consecutive volatile statements of one chain.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t add_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t addc_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t addc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("addc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

__device__ __forceinline__ uint32_t sub_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t subc_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
// borrow of the chain as 0 or 1
__device__ __forceinline__ uint32_t borrow_out() {
  uint32_t r;
  asm volatile("subc.u32 %0, 0, 0;" : "=r"(r));
  return r & 1u;
}

// Group geometry for a lane.
template <int G>
struct Grp {
  int lane, g, base;
  __device__ __forceinline__ Grp() {
    lane = threadIdx.x & 31;
    g = lane & (G - 1);
    base = lane - g;
  }
  // bits of a warp ballot that belong to this group (bit g = lane g)
  __device__ __forceinline__ uint32_t bits(uint32_t ballot) const {
    if (G == 32) return ballot;
    return (ballot >> base) & (uint32_t)((1ull << G) - 1ull);
  }
  __device__ __forceinline__ uint32_t ballot(bool p) const { return bits(__ballot_sync(FULL, p)); }
  // value of v held by lane g' of this group
  __device__ __forceinline__ uint32_t from(uint32_t v, int gp) const { return __shfl_sync(FULL, v, base + gp); }
  __device__ __forceinline__ int64_t from64(int64_t v, int gp) const {
    return (int64_t)__shfl_sync(FULL, (unsigned long long)v, base + gp);
  }
};

// Carry-in mask of the slices given generate (carry out) and propagate (all
// ones) masks, plus an optional carry injected into slice 0.  Bit g of the
// result is the carry entering slice g; bit G is the carry out of the top.
// Adding the generate bits one place up into the propagate runs makes every
// run of propagating slices above a generating slice flip, which is exactly
// the set of slices the carry reaches (carry-lookahead by integer addition).
__device__ __forceinline__ uint64_t carry_mask(uint32_t gen, uint32_t prop, uint32_t inject) {
  uint64_t P = prop, Gm = gen;
  return (P + (Gm << 1) + inject) ^ P;
}

template <int W>
__device__ __forceinline__ bool all_ones(const uint32_t (&v)[W]) {
  uint32_t a = v[0];
#pragma unroll
  for (int i = 1; i < W; ++i) a &= v[i];
  return a == 0xffffffffu;
}

template <int W>
__device__ __forceinline__ bool any_set(const uint32_t (&v)[W]) {
  uint32_t a = v[0];
#pragma unroll
  for (int i = 1; i < W; ++i) a |= v[i];
  return a != 0;
}

// v += c (c in {0,1}) over W limbs; returns the carry out.
template <int W>
__device__ __forceinline__ uint32_t slice_inc(uint32_t (&v)[W], uint32_t c) {
  v[0] = add_cc(v[0], c);
#pragma unroll
  for (int i = 1; i < W; ++i) v[i] = addc_cc(v[i], 0u);
  return addc(0u, 0u);
}

// v -= c (c in {0,1}) over W limbs; returns the borrow out.
template <int W>
__device__ __forceinline__ uint32_t slice_dec(uint32_t (&v)[W], uint32_t c) {
  v[0] = sub_cc(v[0], c);
#pragma unroll
  for (int i = 1; i < W; ++i) v[i] = subc_cc(v[i], 0u);
  return borrow_out();
}

template <int W>
__device__ __forceinline__ bool all_zero(const uint32_t (&v)[W]) {
  return !any_set<W>(v);
}

// ---------------------------------------------------------------------------
// Slice loads and stores (n limbs per number, 16-byte aligned since W % 4 == 0)
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void load_slice(const uint32_t* __restrict__ src, uint32_t (&v)[W]) {
  static_assert(W % 4 == 0, "slices are loaded as uint4");
#pragma unroll
  for (int i = 0; i < W; i += 4) {
    uint4 q = *reinterpret_cast<const uint4*>(src + i);
    v[i] = q.x;
    v[i + 1] = q.y;
    v[i + 2] = q.z;
    v[i + 3] = q.w;
  }
}

template <int W>
__device__ __forceinline__ void store_slice(uint32_t* __restrict__ dst, const uint32_t (&v)[W]) {
#pragma unroll
  for (int i = 0; i < W; i += 4) *reinterpret_cast<uint4*>(dst + i) = make_uint4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}

// Limb bits [bp, bp+32) of an L-limb integer held in memory (generic
// pointer), zero outside [0, 32L).  bp may be negative.
__device__ __forceinline__ uint32_t funnel(const uint32_t* x, int bp, int L) {
  int q = bp >> 5;  // floor division (arithmetic shift)
  int r = bp & 31;
  uint32_t lo = (q >= 0 && q < L) ? x[q] : 0u;
  uint32_t hi = (q + 1 >= 0 && q + 1 < L) ? x[q + 1] : 0u;
  return r ? ((lo >> r) | (hi << (32 - r))) : lo;
}

// Any bit of this slice (holding limbs [first, first+W)) below bit index cut?
template <int W>
__device__ __forceinline__ bool any_below(const uint32_t (&v)[W], int first, int cut) {
  uint32_t a = 0;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    int lb = 32 * (first + i);
    uint32_t m = (cut >= lb + 32) ? 0xffffffffu : (cut <= lb ? 0u : ((1u << (cut - lb)) - 1u));
    a |= v[i] & m;
  }
  return a != 0;
}

// ---------------------------------------------------------------------------
// One row of a W x W schoolbook tile: T[r .. r+W+1] += x * b[0..W).
// T[r+W] holds 0 or 1 on entry (a previous carry); T[r+W+1] is written (set
// to the outgoing carry) when it lies inside the 2W-limb tile.
// ---------------------------------------------------------------------------
template <int W, int L>
__device__ __forceinline__ void mac_row(uint32_t (&T)[L], const uint32_t (&b)[W], uint32_t x, const int r) {
  uint32_t lo[W], hi[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    uint64_t t;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(t) : "r"(x), "r"(b[i]));
    lo[i] = (uint32_t)t;
    hi[i] = (uint32_t)(t >> 32);
  }
  T[r] = add_cc(T[r], lo[0]);
#pragma unroll
  for (int i = 1; i < W; ++i) T[r + i] = addc_cc(T[r + i], lo[i]);
  T[r + W] = addc(T[r + W], 0u);
  T[r + 1] = add_cc(T[r + 1], hi[0]);
#pragma unroll
  for (int i = 1; i < W; ++i) T[r + 1 + i] = addc_cc(T[r + 1 + i], hi[i]);
  if (r + W + 1 < L) T[r + W + 1] = addc(0u, 0u);
}

// ---------------------------------------------------------------------------
// Final rounding of a normalised frame mantissa.  M is this lane's slice of
// the n frame limbs holding the top bits of an exact result, rbit the next
// bit below them and st whether any bit below that is set.  The result keeps
// p = 32 (n - pad) bits: with pad = 0 the whole frame, with pad > 0 the top
// n - pad limbs (the numbers of a precision that is not a power of two of
// limbs live in the next power-of-two frame with their low pad limbs zero).
// Round to nearest, ties to even, at that position; the dropped limbs come
// out zero.  Returns 1 when the rounding carried out of the top (M is then
// 2^(32n - 1) and the exponent grows by one), else 0.  pad is uniform over
// the warp.
// ---------------------------------------------------------------------------
template <int W, int G>
__device__ __forceinline__ uint32_t round_frame(const Grp<G>& gp, uint32_t (&M)[W], uint32_t rbit, bool st,
                                                int pad) {
  uint32_t inc;
  if (pad == 0) {
    const uint32_t lsb = gp.from(M[0], 0) & 1u;
    inc = rbit & ((st ? 1u : 0u) | lsb);
  } else {
    // round limb pad - 1 (its top bit is the round bit), kept limbs from pad
    const int g = gp.g;
    uint32_t rl = 0u, kl = 0u;
    bool below = false;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const int l = g * W + q;
      if (l < pad - 1) below |= (M[q] != 0u);
      if (l == pad - 1) rl = M[q];
      if (l == pad) kl = M[q];
    }
    rl = gp.from(rl, (pad - 1) / W);
    kl = gp.from(kl, pad / W);
    const bool low = gp.ballot(below) != 0u;  // every lane votes: not inside a short-circuit
    const bool stk = st || rbit != 0u || (rl & 0x7fffffffu) != 0u || low;
    inc = (rl >> 31) & ((stk ? 1u : 0u) | (kl & 1u));
    // the increment enters at limb 0 and runs through the dropped limbs
    // (set to all ones) into limb pad
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (g * W + q < pad) M[q] = 0xffffffffu;
  }
  const uint32_t ones = gp.ballot(all_ones<W>(M));
  const uint64_t cm = carry_mask(0u, ones, inc);
  slice_inc<W>(M, (uint32_t)(cm >> gp.g) & 1u);
  const uint32_t ovf = (uint32_t)(cm >> G) & 1u;
  if (pad) {
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (gp.g * W + q < pad) M[q] = 0u;
  }
  if (ovf && gp.g == G - 1) M[W - 1] = 0x80000000u;  // all limbs wrapped to 0
  return ovf;
}

template <int W, int G>
__device__ __forceinline__ int round_product(const Grp<G>& gp, const uint32_t (&F)[W], uint32_t ltop, uint32_t sticky,
                                             uint32_t (&M)[W], int pad);

// ---------------------------------------------------------------------------
// Rounded product of two mantissas.
//   b: this lane's slice of the first mantissa (registers)
//   z: the second mantissa, n limbs in memory (shared or global; every lane
//      of the group reads all of it, so in shared memory it is a broadcast)
// Output: M = this lane's slice of RN_p(mb * mz) scaled to [2^(p-1), 2^p),
// and the exponent adjustment adj with e = ea + eb + adj (adj in {-1,0,1}).
//
// The 2n-limb product is formed by G blocks: at block B, lane g multiplies
// the W limbs z[B*W .. B*W+W) by its slice into a fresh 2W-limb tile T that
// starts with the pending upper half H (from block B-1) plus the finished
// lower half that lane g+1 passed down.  The lower half of T is passed to
// lane g-1; lane 0's lower halves are the product's low limbs, which only
// matter through the round bit and the sticky bit.  After G blocks lane g
// holds product limbs [n + g*W, n + g*W + W).
// ---------------------------------------------------------------------------
// The block loop of mul_round for wide slices (W >= 32): the W x W tile is
// formed S rows at a time in a window of W + S + 1 registers (absolute tile
// limbs [sS, sS + W + S] during rows sS .. sS + S - 1).  After each group of
// S rows the window's lowest S limbs are final: they go down one lane (into
// R, filled by rotation) and into lane 0's sticky bit, and the window moves
// up by S.  The unrolled body is S rows instead of W, which keeps the loop
// inside the instruction cache; the limbs computed are those of the full
// tile, in the same order.
template <int W, int G, int S>
__device__ __forceinline__ void mul_blocks_windowed(const Grp<G>& gp, const uint32_t (&b)[W], const uint32_t* z,
                                                    uint32_t (&H)[W], uint32_t (&R)[W], uint32_t& sticky,
                                                    uint32_t& ltop) {
  static_assert(W % S == 0 && S % 4 == 0, "window of whole uint4 groups");
#pragma unroll 1
  for (int B = 0; B < G; ++B) {
    uint32_t Tw[W + S + 1];
    Tw[0] = add_cc(H[0], R[0]);
#pragma unroll
    for (int i = 1; i < W; ++i) Tw[i] = addc_cc(H[i], R[i]);
    Tw[W] = addc(0u, 0u);
    const uint32_t* zb = z + B * W;
    uint32_t o = 0u;
#pragma unroll 1
    for (int s0 = 0; s0 < W; s0 += S) {
#pragma unroll
      for (int j = 0; j < S; j += 4) {
        uint4 q = *reinterpret_cast<const uint4*>(zb + s0 + j);
        mac_row<W>(Tw, b, q.x, j);
        mac_row<W>(Tw, b, q.y, j + 1);
        mac_row<W>(Tw, b, q.z, j + 2);
        mac_row<W>(Tw, b, q.w, j + 3);
      }
      // limbs s0 .. s0 + S - 1 of the tile are final: down one lane into the
      // top of R (R moves down by S), and into lane 0's sticky bit except
      // limb n - 1 of the product (the last tile's limb W - 1), kept whole
#pragma unroll
      for (int i = 0; i < W - S; ++i) R[i] = R[i + S];
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const uint32_t v = __shfl_down_sync(FULL, Tw[j], 1);
        R[W - S + j] = (gp.g == G - 1) ? 0u : v;
      }
      const bool last = (B == G - 1) && (s0 == W - S);
#pragma unroll
      for (int j = 0; j < S - 1; ++j) o |= Tw[j];
      if (last) ltop = Tw[S - 1];
      else o |= Tw[S - 1];
#pragma unroll
      for (int i = 0; i <= W; ++i) Tw[i] = Tw[i + S];
    }
    sticky |= o;
#pragma unroll
    for (int i = 0; i < W; ++i) H[i] = Tw[i];
  }
}

template <int W, int G>
__device__ __forceinline__ int mul_round(const Grp<G>& gp, const uint32_t (&b)[W], const uint32_t* z,
                                         uint32_t (&M)[W], int pad = 0) {
  uint32_t H[W], R[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    H[i] = 0u;
    R[i] = 0u;
  }
  uint32_t sticky = 0u, ltop = 0u;
  if constexpr (W >= 32) {
    mul_blocks_windowed<W, G, 8>(gp, b, z, H, R, sticky, ltop);
  } else {
#pragma unroll 1
  for (int B = 0; B < G; ++B) {
    uint32_t T[2 * W];
    T[0] = add_cc(H[0], R[0]);
#pragma unroll
    for (int i = 1; i < W; ++i) T[i] = addc_cc(H[i], R[i]);
    T[W] = addc(0u, 0u);
    const uint32_t* zb = z + B * W;
#pragma unroll
    for (int r = 0; r < W; r += 4) {
      uint4 q = *reinterpret_cast<const uint4*>(zb + r);
      mac_row<W>(T, b, q.x, r);
      mac_row<W>(T, b, q.y, r + 1);
      mac_row<W>(T, b, q.z, r + 2);
      mac_row<W>(T, b, q.w, r + 3);
    }
    // lower half goes down one lane (lane G-1 receives nothing)
#pragma unroll
    for (int i = 0; i < W; ++i) {
      uint32_t v = __shfl_down_sync(FULL, T[i], 1);
      R[i] = (gp.g == G - 1) ? 0u : v;
    }
    // lane 0: low limbs of the product (sticky), limb n-1 kept whole
    uint32_t o = 0u;
#pragma unroll
    for (int i = 0; i < W - 1; ++i) o |= T[i];
    if (B < G - 1) o |= T[W - 1];
    else ltop = T[W - 1];
    sticky |= o;
#pragma unroll
    for (int i = 0; i < W; ++i) H[i] = T[W + i];
  }
  }
  // upper half: F = H + R, carries across the slices
  uint32_t F[W];
  F[0] = add_cc(H[0], R[0]);
#pragma unroll
  for (int i = 1; i < W; ++i) F[i] = addc_cc(H[i], R[i]);
  uint32_t c = addc(0u, 0u);
  uint32_t gen = gp.ballot(c != 0u), prop = gp.ballot(all_ones<W>(F));
  uint32_t cin = (uint32_t)(carry_mask(gen, prop, 0u) >> gp.g) & 1u;
  slice_inc<W>(F, cin);
  return round_product<W, G>(gp, F, ltop, sticky, M, pad);
}

// Normalise and round an exact product of two normalised n-limb mantissas:
// F is this lane's slice of its upper n limbs, ltop (lane 0's value) its
// limb n - 1 and sticky (lane 0's value) the OR of limbs [0, n - 1).  The
// product has 2p or 2p - 1 bits; M receives RN_p scaled to [2^(p-1), 2^p) and
// the return value is the exponent adjustment (-1, 0 or +1).
template <int W, int G>
__device__ __forceinline__ int round_product(const Grp<G>& gp, const uint32_t (&F)[W], uint32_t ltop, uint32_t sticky,
                                             uint32_t (&M)[W], int pad) {
  // normalise: the product has 2p or 2p-1 bits
  uint32_t top = gp.from(F[W - 1], G - 1) >> 31;
  ltop = gp.from(ltop, 0);
  sticky = gp.from(sticky, 0);
  uint32_t prev = __shfl_up_sync(FULL, F[W - 1], 1);
  if (gp.g == 0) prev = ltop;
  uint32_t rbit, st;
  if (top) {
#pragma unroll
    for (int i = 0; i < W; ++i) M[i] = F[i];
    rbit = ltop >> 31;
    st = (ltop & 0x7fffffffu) | sticky;
  } else {
#pragma unroll
    for (int i = W - 1; i > 0; --i) M[i] = (F[i] << 1) | (F[i - 1] >> 31);
    M[0] = (F[0] << 1) | (prev >> 31);
    rbit = (ltop >> 30) & 1u;
    st = (ltop & 0x3fffffffu) | sticky;
  }
  const uint32_t ovf = round_frame<W, G>(gp, M, rbit, st != 0u, pad);
  return (top ? 0 : -1) + (int)ovf;
}

// ---------------------------------------------------------------------------
// RN_p(x - t) for x = (xs, xe, X) and t = (ts, te, T), slices in registers.
// buf: per-group scratch in shared memory, >= n + 8 words, 16-byte aligned.
// Result overwrites (xs, xe, X).
//
// The larger magnitude A is placed in a frame of n+3 limbs with two guard
// limbs below it; the smaller B is aligned into the frame; bits of B that
// fall below the frame are folded into the lowest frame bit (sticky jam).
// With 64 guard bits every rounding threshold of the result is an even frame
// integer, so A +- B_jammed rounds exactly like A +- B.  Exponent gaps of
// p+2 or more return A unchanged (B is below a quarter ulp of A).
// ---------------------------------------------------------------------------
template <int W, int G>
__device__ __forceinline__ void sub_round(const Grp<G>& gp, int p, int8_t& xs, int64_t& xe, uint32_t (&X)[W],
                                          int8_t ts, int64_t te, const uint32_t (&T)[W], uint32_t* buf,
                                          int pad = 0) {
  constexpr int n = W * G;
  const int g = gp.g;
  const int8_t tsn = (te == ZEXP) ? 0 : (int8_t)(ts ^ 1);  // -t
  // |x| vs |t|
  int lc = 0;
#pragma unroll
  for (int i = W - 1; i >= 0; --i)
    if (lc == 0 && X[i] != T[i]) lc = X[i] > T[i] ? 1 : -1;
  uint32_t gt = gp.ballot(lc > 0), lt = gp.ballot(lc < 0), df = gt | lt;
  int mcmp = df ? (((gt >> (31 - __clz(df))) & 1u) ? 1 : -1) : 0;
  int cmp = (xe != te) ? (xe > te ? 1 : -1) : mcmp;
  const bool swap = cmp < 0;
  uint32_t A[W], Bv[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    A[i] = swap ? T[i] : X[i];
    Bv[i] = swap ? X[i] : T[i];
  }
  const int64_t eA = swap ? te : xe, eB = swap ? xe : te;
  const int8_t sA = swap ? tsn : xs, sB = swap ? xs : tsn;
  const bool eff_sub = (sA != sB);
  // alignment distance, clamped (B == 0 aligns below the frame)
  int d;
  if (eB == ZEXP || eA == ZEXP) d = p + 72;
  else {
    int64_t d64 = eA - eB;
    d = (int)(d64 > (int64_t)(p + 72) ? (int64_t)(p + 72) : d64);
  }
  // Aligned B: frame limb f holds bits [32f + d - 64, ..) of B.  Fast path
  // (every group of the warp has d < 64, or B == 0): the shift stays within
  // two limbs and is done in registers with the next lane's first limbs.
  // Otherwise B goes through shared memory and the bits below the frame are
  // jammed into the sticky bit.
  uint32_t Y[W], y0, y1;
  const bool fastA = (eB == ZEXP) || (eA != ZEXP && eA - eB <= 63);
  if (__all_sync(FULL, fastA)) {
    const int da = (eB == ZEXP) ? 0 : d;
    const int q = da >> 5, r = da & 31;
    uint32_t n0 = __shfl_down_sync(FULL, Bv[0], 1), n1 = __shfl_down_sync(FULL, Bv[1], 1);
    if (g == G - 1) n0 = n1 = 0u;
    uint32_t Bx[W + 2];
#pragma unroll
    for (int i = 0; i < W; ++i) Bx[i] = Bv[i];
    Bx[W] = n0;
    Bx[W + 1] = n1;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const uint32_t lo = q ? Bx[i + 1] : Bx[i];
      const uint32_t hi = q ? Bx[i + 2] : Bx[i + 1];
      Y[i] = __funnelshift_r(lo, hi, r);
    }
    y0 = q ? __funnelshift_r(0u, Bv[0], r) : 0u;
    y1 = q ? __funnelshift_r(Bv[0], Bv[1], r) : __funnelshift_r(0u, Bv[0], r);
  } else {
    store_slice<W>(buf + g * W, Bv);
    if (g == G - 1) {
#pragma unroll
      for (int i = 0; i < 8; ++i) buf[n + i] = 0u;
    }
    __syncwarp();
    // sticky of B's bits below the frame (bit index d - 64 of B)
    const bool lost = gp.ballot(any_below<W>(Bv, g * W, d - 64)) != 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) Y[i] = funnel(buf, 32 * (2 + g * W + i) + d - 64, n);
    y0 = funnel(buf, d - 64, n) | (lost ? 1u : 0u);
    y1 = funnel(buf, 32 + d - 64, n);
    __syncwarp();
  }
  // S = A*2^64 +- Ybar  (two's complement for subtraction)
  const uint32_t inv = eff_sub ? 0xffffffffu : 0u;
#pragma unroll
  for (int i = 0; i < W; ++i) Y[i] ^= inv;
  y0 ^= inv;
  y1 ^= inv;
  // guard limbs (thread 0's), A's guard bits are zero
  uint32_t s0 = add_cc(y0, eff_sub ? 1u : 0u);
  uint32_t s1 = addc_cc(y1, 0u);
  uint32_t cg = addc(0u, 0u);
  uint32_t S[W];
  S[0] = add_cc(A[0], Y[0]);
#pragma unroll
  for (int i = 1; i < W; ++i) S[i] = addc_cc(A[i], Y[i]);
  uint32_t c = addc(0u, 0u);
  cg = gp.from(cg, 0);
  uint32_t gen = gp.ballot(c != 0u), prop = gp.ballot(all_ones<W>(S));
  uint64_t cm = carry_mask(gen, prop, cg);
  slice_inc<W>(S, (uint32_t)(cm >> g) & 1u);
  const uint32_t sx = eff_sub ? 0u : (uint32_t)(cm >> G) & 1u;  // frame limb n+2
  // top bit of the frame value
  int ltf = -1;
#pragma unroll
  for (int i = 0; i < W; ++i)
    if (S[i]) ltf = 2 + g * W + i;
  if (g == 0 && ltf < 0) ltf = s1 ? 1 : (s0 ? 0 : -1);
  uint32_t nzm = gp.ballot(ltf >= 0);
  // shuffles run on every lane (groups of one warp may disagree on sx / nzm)
  const int ht = nzm ? 31 - __clz(nzm) : 0;
  const int tf = (int)gp.from((uint32_t)ltf, ht);
  uint32_t mine = 0u;  // the limb value at frame index tf, held by lane ht
#pragma unroll
  for (int i = 0; i < W; ++i)
    if (2 + g * W + i == tf) mine = S[i];
  if (g == 0 && tf == 1) mine = s1;
  if (g == 0 && tf == 0) mine = s0;
  const uint32_t tl = gp.from(mine, ht);
  int topbit;
  bool zero = false;
  if (sx) topbit = 32 * (n + 2);
  else if (nzm == 0u) {
    topbit = 0;
    zero = true;
  } else {
    topbit = 32 * tf + 31 - __clz(tl);
  }
  // mantissa: output limb l takes frame bits [32l + sh, ..), sh = topbit-(p-1).
  // Fast path (every group of the warp has sh in [32, 65] or a zero result):
  // at most 32 bits of cancellation, the shift uses the neighbouring lanes'
  // edge limbs and the round and sticky bits lie in lane 0's guard limbs.
  const int sh = topbit - (p - 1);
  uint32_t Mo[W];
  uint32_t rbit = 0u;
  bool st = false;
  const bool fastN = zero || (sh >= 32 && sh <= 65);
  if (__all_sync(FULL, fastN)) {
    uint32_t prev = __shfl_up_sync(FULL, S[W - 1], 1);
    uint32_t next = __shfl_down_sync(FULL, S[0], 1);
    if (g == 0) prev = s1;
    if (g == G - 1) next = sx;
    const int q = sh >> 5, r = sh & 31;  // q in {1, 2}
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const uint32_t lo = (q == 1) ? (i == 0 ? prev : S[i - 1]) : S[i];
      const uint32_t hi = (q == 1) ? S[i] : (i == W - 1 ? next : S[i + 1]);
      Mo[i] = __funnelshift_r(lo, hi, r);
    }
    const uint64_t g64 = ((uint64_t)s1 << 32) | s0;
    const int rb = zero ? 40 : sh - 1;  // 31..64 (any in-range value for a zero result)
    uint32_t r0 = (rb < 64) ? (uint32_t)((g64 >> rb) & 1ull) : (S[0] & 1u);
    uint32_t t0 = (rb < 64) ? (uint32_t)((g64 & ((1ull << rb) - 1ull)) != 0ull) : (uint32_t)(g64 != 0ull);
    rbit = gp.from(r0, 0);
    st = gp.from(t0, 0) != 0u;
    if (zero) rbit = 0u;
  } else {
    // frame to shared memory
#pragma unroll
    for (int i = 0; i < W; ++i) buf[2 + g * W + i] = S[i];  // frame limbs 2..n+1 (8-byte offset: scalar stores)
    if (g == 0) {
      buf[0] = s0;
      buf[1] = s1;
    }
    if (g == G - 1) buf[n + 2] = sx;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < W; ++i) Mo[i] = funnel(buf, 32 * (g * W + i) + sh, n + 3);
    if (sh >= 1) {
      rbit = (funnel(buf, sh - 1, n + 3)) & 1u;
    }
    // sticky: frame bits below sh-1 (this lane's frame limbs, lane 0's guards)
    bool stl = any_below<W>(S, 2 + g * W, sh - 1);
    if (g == 0) {
      uint32_t gv[2] = {s0, s1};
      stl = stl || any_below<2>(gv, 0, sh - 1);
    }
    st = gp.ballot(stl && sh >= 2) != 0u;
    __syncwarp();
  }
  const uint32_t ovf = round_frame<W, G>(gp, Mo, rbit, st, pad);
  if (zero) {
    xs = 0;
    xe = ZEXP;
#pragma unroll
    for (int i = 0; i < W; ++i) X[i] = 0u;
  } else {
    xs = sA;
    xe = (int64_t)topbit + 1 + eA - p - 64 + ovf;
#pragma unroll
    for (int i = 0; i < W; ++i) X[i] = Mo[i];
  }
}

// ---------------------------------------------------------------------------
// Division of the two-limb u1*2^32 + u0 (u1 < d) by a normalised limb d
// (top bit set) with the precomputed reciprocal v = floor((2^64-1)/d) - 2^32,
// after Moller and Granlund, "Improved division by invariant integers"
// (IEEE Trans. Computers 60(2), 2011), Algorithm 4: one multiply, one
// multiply-low and two rarely taken corrections instead of a 64-by-32-bit
// software division.  Returns the quotient limb; r = the remainder.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t div21_preinv(uint32_t u1, uint32_t u0, uint32_t d, uint32_t v,
                                                          uint32_t& r) {
  const uint64_t s = (uint64_t)v * u1 + (((uint64_t)u1 << 32) | u0);  // modulo 2^64
  uint32_t q1 = (uint32_t)(s >> 32) + 1u;
  const uint32_t q0 = (uint32_t)s;
  uint32_t rr = u0 - q1 * d;
  if (rr > q0) {
    q1 -= 1u;
    rr += d;
  }
  if (rr >= d) {
    q1 += 1u;
    rr -= d;
  }
  r = rr;
  return q1;
}

__host__ __device__ __forceinline__ uint32_t div21_inverse(uint32_t d) {
  return (uint32_t)(~0ull / d - (1ull << 32));
}

// ---------------------------------------------------------------------------
// Correctly rounded reciprocal of a mantissa: RN_p(2^(2p-1) / m) scaled to
// [2^(p-1), 2^p).  V: this lane's slice of m (normalised, top bit set).
// qbuf: per-group shared scratch of >= n + 1 words.
// Returns adj with 1/x having exponent adj - e (x = m * 2^(e-p)).
//
// Schoolbook long division in base 2^32 (Knuth, TAOCP vol. 2, 4.3.1,
// Algorithm D) of 2^(2p) by m: one quotient limb per step from the top two
// remainder limbs (Theorem B: the estimate is at most two too large for a
// normalised divisor), a 2-limb test that leaves it at most one too large, a
// multiply-subtract, and an add-back when the estimate was too large.
// Quotient Q = floor(2^(2p)/m) lies in (2^p, 2^(p+1)]; RN rounds Q/2 with
// Q's last bit as round bit and the remainder as sticky.
//
// Per step the group exchanges one word per lane: each lane subtracts q times
// its slice of m from its slice of the shifted remainder with a word-sized
// running borrow (at most 2^32 - 1), passes that borrow word one lane up, and
// the one-bit borrows that remain are resolved with two ballots.  A lane whose
// own subtraction borrowed is left with a non-zero slice (W >= 2), so no lane
// passes on more than one bit.
// ---------------------------------------------------------------------------
template <int W, int G>
__device__ __forceinline__ int recip_round(const Grp<G>& gp, const uint32_t (&V)[W], uint32_t* qbuf, uint32_t (&M)[W],
                                           int pad = 0) {
  constexpr int n = W * G;
  static_assert(W >= 4, "the quotient test reads three limbs of the top slice");
  const int g = gp.g;
  uint32_t R[W];
#pragma unroll
  for (int i = 0; i < W; ++i) R[i] = 0u;
  if (g == G - 1) R[W - 1] = 1u;  // R = 2^(32(n-1)); the first shift makes it 2^p
  const uint32_t v1 = gp.from(V[W - 1], G - 1), v0 = gp.from(V[W - 2], G - 1);
  const uint32_t vinv = div21_inverse(v1);
#pragma unroll 1
  for (int j = n; j >= 0; --j) {
    // R' = R * 2^32 (n+1 limbs; limb n is rtop, limbs n-1 and n-2 are r1, r0)
    const uint32_t rtop = gp.from(R[W - 1], G - 1);
    const uint32_t r1 = gp.from(R[W - 2], G - 1), r0 = gp.from(R[W - 3], G - 1);
    uint32_t up = __shfl_up_sync(FULL, R[W - 1], 1);
    if (g == 0) up = 0u;
#pragma unroll
    for (int i = W - 1; i > 0; --i) R[i] = R[i - 1];
    R[0] = up;
    // quotient limb estimate: min(floor((rtop, r1) / v1), 2^32 - 1); the
    // remainder never exceeds m, so rtop <= v1
    uint32_t q, rh;
    bool rbig;
    if (rtop >= v1) {
      q = 0xffffffffu;
      const uint64_t t = (uint64_t)r1 + v1;  // (rtop, r1) - q * v1 with rtop = v1
      rh = (uint32_t)t;
      rbig = (t >> 32) != 0u;
    } else {
      q = div21_preinv(rtop, r1, v1, vinv, rh);
      rbig = false;
    }
    for (int it = 0; it < 2 && !rbig && (uint64_t)q * v0 > (((uint64_t)rh << 32) | r0); ++it) {
      q -= 1u;
      const uint64_t t = (uint64_t)rh + v1;
      rh = (uint32_t)t;
      rbig = (t >> 32) != 0u;
    }
    // D = R' - q * m: this slice with a running borrow word ...
    uint32_t D[W];
    uint32_t acc = 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const uint64_t t = (uint64_t)q * V[i] + acc;
      const uint32_t lo = (uint32_t)t;
      D[i] = R[i] - lo;
      acc = (uint32_t)(t >> 32) + (R[i] < lo ? 1u : 0u);
    }
    // ... minus the borrow word of the slice below ...
    uint32_t bin = __shfl_up_sync(FULL, acc, 1);
    if (g == 0) bin = 0u;
    const uint32_t atop = gp.from(acc, G - 1);
    D[0] = sub_cc(D[0], bin);
#pragma unroll
    for (int i = 1; i < W; ++i) D[i] = subc_cc(D[i], 0u);
    const uint32_t bo = borrow_out();
    // ... and the one-bit borrows rippling up through all-zero slices
    const uint64_t bm = carry_mask(gp.ballot(bo != 0u), gp.ballot(all_zero<W>(D)), 0u);
    slice_dec<W>(D, (uint32_t)(bm >> g) & 1u);
    const int64_t top = (int64_t)rtop - (int64_t)atop - (int64_t)((bm >> G) & 1u);
    const bool neg = top < 0;  // estimate one too large: add m back
    if (__any_sync(FULL, neg)) {
      uint32_t Vm[W];
#pragma unroll
      for (int i = 0; i < W; ++i) Vm[i] = neg ? V[i] : 0u;
      D[0] = add_cc(D[0], Vm[0]);
#pragma unroll
      for (int i = 1; i < W; ++i) D[i] = addc_cc(D[i], Vm[i]);
      uint32_t ac = addc(0u, 0u);
      uint64_t am = carry_mask(gp.ballot(ac != 0u), gp.ballot(all_ones<W>(D)), 0u);
      slice_inc<W>(D, (uint32_t)(am >> g) & 1u);
      if (neg) q -= 1u;
    }
#pragma unroll
    for (int i = 0; i < W; ++i) R[i] = D[i];
    if (g == 0) qbuf[j] = q;
  }
  const bool rnz = gp.ballot(any_set<W>(R)) != 0u;
  __syncwarp();
  const uint32_t qn = qbuf[n];
  if (qn >= 2u) {  // m = 2^(p-1): 1/x is a power of two
#pragma unroll
    for (int i = 0; i < W; ++i) M[i] = 0u;
    if (g == G - 1) M[W - 1] = 0x80000000u;
  }
#pragma unroll
  for (int i = 0; i < W; ++i) {
    int l = g * W + i;
    uint32_t v = (qbuf[l] >> 1) | (qbuf[l + 1] << 31);
    M[i] = (qn >= 2u) ? M[i] : v;
  }
  const uint32_t rbit = (qn >= 2u) ? 0u : (qbuf[0] & 1u);
  const uint32_t ovf = round_frame<W, G>(gp, M, rbit, rnz, pad);
  __syncwarp();
  return (qn >= 2u) ? 2 : 1 + (int)ovf;
}

}  // namespace mpd
