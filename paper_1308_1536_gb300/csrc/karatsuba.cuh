// Exact products of two mantissas for the comparison of schoolbook and one
// Karatsuba level on the IMAD engine's lane layout (the product of the rank-1
// update, Alg. 1 step 2.2.2, is exact before its rounding, so any exact
// multiplication scheme gives the same rounded result).
//
// Layout as in mpdev.cuh: a number of n = W*G limbs is held by a group of G
// lanes, lane g holding limbs [gW, gW + W); the second operand z is n limbs in
// memory that every lane of the group reads (a broadcast in shared memory).
#pragma once
#include "mpdev.cuh"

namespace mpd {

// ---------------------------------------------------------------------------
// Schoolbook exact product, the lane-systolic scheme of mul_round: at block B
// lane g adds the W x W tile z[BW, BW + W) * b_g to its running 2W-limb tile;
// the finished lower W limbs go down one lane, and lane 0's (product limbs
// [BW, BW + W)) are stored to lo[BW ..].  On return lane g holds the upper
// product limbs [n + gW, n + gW + W) in U; lo holds limbs [0, n).
// ---------------------------------------------------------------------------
template <int W, int G>
__device__ __forceinline__ void mul_full(const Grp<G>& gp, const uint32_t (&b)[W], const uint32_t* z, uint32_t* lo,
                                         uint32_t (&U)[W]) {
  static_assert(W % 4 == 0 && W <= 16, "tiles held whole in registers");
  uint32_t H[W], R[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    H[i] = 0u;
    R[i] = 0u;
  }
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
      const uint4 q = *reinterpret_cast<const uint4*>(zb + r);
      mac_row<W>(T, b, q.x, r);
      mac_row<W>(T, b, q.y, r + 1);
      mac_row<W>(T, b, q.z, r + 2);
      mac_row<W>(T, b, q.w, r + 3);
    }
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const uint32_t v = __shfl_down_sync(FULL, T[i], 1);
      R[i] = (gp.g == G - 1) ? 0u : v;
    }
    if (gp.g == 0) {
#pragma unroll
      for (int i = 0; i < W; i += 4)
        *reinterpret_cast<uint4*>(lo + B * W + i) = make_uint4(T[i], T[i + 1], T[i + 2], T[i + 3]);
    }
#pragma unroll
    for (int i = 0; i < W; ++i) H[i] = T[W + i];
  }
  U[0] = add_cc(H[0], R[0]);
#pragma unroll
  for (int i = 1; i < W; ++i) U[i] = addc_cc(H[i], R[i]);
  const uint32_t c = addc(0u, 0u);
  const uint64_t cm = carry_mask(gp.ballot(c != 0u), gp.ballot(all_ones<W>(U)), 0u);
  slice_inc<W>(U, (uint32_t)(cm >> gp.g) & 1u);
  __syncwarp();
}

// One pass of S (+ or -) V over the group's slices, V in registers; returns
// the carry (+1), borrow (-1) or 0 out of the top slice.  Subtraction is the
// two's-complement addition S + ~V + 1 with the 1 entering the bottom slice,
// so both run the same instructions and ballots (groups of one warp may
// differ in sub).
template <int W, int G>
__device__ __forceinline__ int slices_addsub(const Grp<G>& gp, uint32_t (&S)[W], const uint32_t (&V)[W], bool sub) {
  const uint32_t inv = sub ? 0xffffffffu : 0u;
  S[0] = add_cc(S[0], V[0] ^ inv);
#pragma unroll
  for (int i = 1; i < W; ++i) S[i] = addc_cc(S[i], V[i] ^ inv);
  const uint32_t o = addc(0u, 0u);
  const uint64_t cm = carry_mask(gp.ballot(o != 0u), gp.ballot(all_ones<W>(S)), sub ? 1u : 0u);
  slice_inc<W>(S, (uint32_t)(cm >> gp.g) & 1u);
  const int top = (int)((cm >> G) & 1u);
  return sub ? top - 1 : top;
}

// S += c for a small signed c (|c| <= 7) entering at the bottom limb of the
// group; returns the carry or borrow out of the top (signed).
template <int W, int G>
__device__ __forceinline__ int slices_add_small(const Grp<G>& gp, uint32_t (&S)[W], int c) {
  uint32_t V[W];
#pragma unroll
  for (int i = 0; i < W; ++i) V[i] = 0u;
  if (gp.g == 0) V[0] = (uint32_t)(c < 0 ? -c : c);
  return slices_addsub<W, G>(gp, S, V, c < 0);
}

template <int W>
__device__ __forceinline__ void load_w(const uint32_t* p, uint32_t (&v)[W]) {
#pragma unroll
  for (int i = 0; i < W; i += 4) {
    const uint4 q = *reinterpret_cast<const uint4*>(p + i);
    v[i] = q.x;
    v[i + 1] = q.y;
    v[i + 2] = q.z;
    v[i + 3] = q.w;
  }
}

// ---------------------------------------------------------------------------
// One Karatsuba level over the schoolbook half-products.  With n2 = n/2,
// X = 2^(32 n2), z = z0 + z1 X and b = b0 + b1 X:
//     z b = P0 + X (M - P0 - P2) + X^2 P2,
//     P0 = z0 b0,  P2 = z1 b1,  M = (z0 + z1)(b0 + b1).
// The sums s_z = z0 + z1 = s'_z + c_z X and s_b = s'_b + c_b X carry one bit
// each, so M = s'_z s'_b + X (c_z s'_b + c_b s'_z) + c_z c_b X^2.  The three
// n2 x n2 products run on all G lanes with slices of W2 = W/2 limbs (three
// quarter-size products: 3/4 of the schoolbook's limb products), and the
// result is assembled region by region (n2 limbs each; lane g holds limbs
// [g W2, g W2 + W2) of a region) with one ballot-resolved carry pass per
// operand.  Scratch (memory of the group, 16-byte aligned): lo0, lo2, lom:
// n2 limbs each (the half-products' lower halves), sz: n2 limbs (s'_z).
// Output as mul_full: lo = product limbs [0, n), U = this lane's slice of the
// upper n limbs in the W-limb layout.
// ---------------------------------------------------------------------------
template <int W, int G>
__device__ __forceinline__ void mul_full_kara(const Grp<G>& gp, const uint32_t (&b)[W], const uint32_t* z, uint32_t* lo,
                                              uint32_t* lo0, uint32_t* lo2, uint32_t* lom, uint32_t* sz,
                                              uint32_t (&U)[W]) {
  constexpr int W2 = W / 2, n = W * G, n2 = n / 2;
  static_assert(W2 % 4 == 0, "half slices of whole uint4 groups");
  const int g = gp.g;
  // b0 (limbs [0, n2)) and b1 (limbs [n2, n)) in half slices: lane g takes
  // limbs [g W2, g W2 + W2) of each from lane g/2 (b0) and G/2 + g/2 (b1)
  uint32_t b0[W2], b1[W2];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const uint32_t v0 = gp.from(b[i], g >> 1), v1 = gp.from(b[i], (G >> 1) + (g >> 1));
    if (i < W2) {
      if (!(g & 1)) {
        b0[i] = v0;
        b1[i] = v1;
      }
    } else if (g & 1) {
      b0[i - W2] = v0;
      b1[i - W2] = v1;
    }
  }
  // s'_b = b0 + b1 (registers), c_b
  uint32_t sb[W2];
#pragma unroll
  for (int i = 0; i < W2; ++i) sb[i] = b0[i];
  const int cb = slices_addsub<W2, G>(gp, sb, b1, false);
  // s'_z = z0 + z1 (memory), c_z
  uint32_t zs[W2], z1v[W2];
  load_w<W2>(z + g * W2, zs);
  load_w<W2>(z + n2 + g * W2, z1v);
  const int cz = slices_addsub<W2, G>(gp, zs, z1v, false);
#pragma unroll
  for (int i = 0; i < W2; i += 4) *reinterpret_cast<uint4*>(sz + g * W2 + i) = make_uint4(zs[i], zs[i + 1], zs[i + 2], zs[i + 3]);
  __syncwarp();
  // the three half-products
  uint32_t U0[W2], U2[W2], Um[W2];
  mul_full<W2, G>(gp, b0, z, lo0, U0);
  mul_full<W2, G>(gp, b1, z + n2, lo2, U2);
  mul_full<W2, G>(gp, sb, sz, lom, Um);
  __syncwarp();
  // region 0: P0's lower half, final
  uint32_t R[W2], V[W2];
  load_w<W2>(lo0 + g * W2, R);
#pragma unroll
  for (int i = 0; i < W2; i += 4) *reinterpret_cast<uint4*>(lo + g * W2 + i) = make_uint4(R[i], R[i + 1], R[i + 2], R[i + 3]);
  // region 1: P0_hi + M'_lo - P0_lo - P2_lo
  int c1 = 0;
#pragma unroll
  for (int i = 0; i < W2; ++i) V[i] = R[i];  // P0_lo
#pragma unroll
  for (int i = 0; i < W2; ++i) R[i] = U0[i];
  uint32_t T[W2];
  load_w<W2>(lom + g * W2, T);
  c1 += slices_addsub<W2, G>(gp, R, T, false);
  c1 += slices_addsub<W2, G>(gp, R, V, true);
  load_w<W2>(lo2 + g * W2, T);
  c1 += slices_addsub<W2, G>(gp, R, T, true);
  __syncwarp();
#pragma unroll
  for (int i = 0; i < W2; i += 4) *reinterpret_cast<uint4*>(lo + n2 + g * W2 + i) = make_uint4(R[i], R[i + 1], R[i + 2], R[i + 3]);
  // region 2: M'_hi + c_z s'_b + c_b s'_z - P0_hi - P2_hi + P2_lo + c1
  int c2 = 0;
#pragma unroll
  for (int i = 0; i < W2; ++i) {
    R[i] = Um[i];
    V[i] = cz ? sb[i] : 0u;
  }
  c2 += slices_addsub<W2, G>(gp, R, V, false);
#pragma unroll
  for (int i = 0; i < W2; ++i) V[i] = cb ? zs[i] : 0u;
  c2 += slices_addsub<W2, G>(gp, R, V, false);
  c2 += slices_addsub<W2, G>(gp, R, U0, true);
  c2 += slices_addsub<W2, G>(gp, R, U2, true);
  load_w<W2>(lo2 + g * W2, T);
  c2 += slices_addsub<W2, G>(gp, R, T, false);
  c2 += slices_add_small<W2, G>(gp, R, c1);  // every group of the warp runs the pass
  // region 3: P2_hi + c_z c_b + c2 (the product fits 2n limbs: no carry out)
  uint32_t Q[W2];
#pragma unroll
  for (int i = 0; i < W2; ++i) Q[i] = U2[i];
  slices_add_small<W2, G>(gp, Q, c2 + cz * cb);
  // regions 2 and 3 back into the W-limb layout: lane g takes limbs
  // [gW, gW + W) of the upper half, the half slices of lanes 2g, 2g + 1 of
  // region 2 (g < G/2) or of region 3 (g >= G/2)
  const int src = (2 * g) & (G - 1);
#pragma unroll
  for (int i = 0; i < W2; ++i) {
    const uint32_t r0 = gp.from(R[i], src), r1 = gp.from(R[i], src + 1);
    const uint32_t q0 = gp.from(Q[i], src), q1 = gp.from(Q[i], src + 1);
    U[i] = (g < G / 2) ? r0 : q0;
    U[W2 + i] = (g < G / 2) ? r1 : q1;
  }
  __syncwarp();
}

// RN_p of the product by one Karatsuba level: the exact product of
// mul_full_kara, then the same normalisation and rounding as mul_round
// (round_product).  Returns the exponent adjustment as mul_round does.
template <int W, int G>
__device__ __forceinline__ int mul_round_kara(const Grp<G>& gp, const uint32_t (&b)[W], const uint32_t* z,
                                              uint32_t (&M)[W], uint32_t* scratch, int pad = 0) {
  constexpr int n = W * G, n2 = n / 2;
  uint32_t* lo = scratch;  // n limbs
  uint32_t* lo0 = scratch + n;
  uint32_t* lo2 = lo0 + n2;
  uint32_t* lom = lo2 + n2;
  uint32_t* sz = lom + n2;
  uint32_t F[W];
  mul_full_kara<W, G>(gp, b, z, lo, lo0, lo2, lom, sz, F);
  // limb n - 1 whole, and the OR of limbs [0, n - 1), every lane its slice
  uint32_t o = 0u;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const int l = gp.g * W + i;
    if (l < n - 1) o |= lo[l];
  }
  const uint32_t sticky = gp.ballot(o != 0u) ? 1u : 0u;
  const uint32_t ltop = lo[n - 1];
  __syncwarp();
  return round_product<W, G>(gp, F, ltop, sticky, M, pad);
}

}  // namespace mpd
