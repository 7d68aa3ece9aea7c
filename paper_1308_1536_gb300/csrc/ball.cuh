// Radii of the ball mode: each value x~ of the elimination carries a radius
// rho with |x* - x~| <= rho, x* being what exact arithmetic gives at the same
// place (midpoint-radius intervals: the rigorous bounds the paper leaves to
// future work, Sec. 4.4).  A radius is m * 2^(e - 32) with m in [2^31, 2^32),
// or 0 (m = 0, e = INT64_MIN), or unbounded (e = INT64_MAX); every operation
// on radii rounds up (down where a lower bound is needed), in integer
// arithmetic, so the radii do not depend on the hardware.
//
// Rules (u~ the rounded result; hu = half an ulp of u~ at p bits,
// 2^(e_u - p - 1), 0 when u~ = 0; |x~|^ and |x~|_ bound |x~| from above and
// below from its top limb):
//   u~ = RN(x~ y~):   rho_u = ((hu + |x~|^ rho_y) + |y~|^ rho_x) + rho_x rho_y
//   u~ = RN(x~ - t~): rho_u = (hu + rho_x) + rho_t
//   u~ = RN(1/a~):    rho_u = hu + rho_a / (|a~|_ (|a~|_ - rho_a)),
//                     unbounded unless |a~|_ > rho_a
// The additions run in the order written (they round).
#pragma once
#include "mpdev.cuh"

namespace mpd {

struct Rad {
  uint32_t m;
  int64_t e;
};

constexpr int64_t RAD_INF = INT64_MAX;

__device__ __forceinline__ Rad rad_zero() { return Rad{0u, ZEXP}; }
__device__ __forceinline__ Rad rad_unbounded() { return Rad{0xffffffffu, RAD_INF}; }
__device__ __forceinline__ bool rad_isz(const Rad& a) { return a.m == 0u; }
__device__ __forceinline__ bool rad_isinf(const Rad& a) { return a.e == RAD_INF; }

// V * 2^E to a radius, rounded up (up) or down
__device__ __forceinline__ Rad rad_of(uint64_t V, int64_t E, bool up) {
  if (V == 0ull) return rad_zero();
  int t = 64 - __clzll((long long)V);
  uint64_t m;
  if (t <= 32) {
    m = V << (32 - t);
  } else {
    const int sh = t - 32;
    m = V >> sh;
    if (up && (V & ((1ull << sh) - 1ull))) m += 1ull;
    if (m >> 32) {
      m >>= 1;
      t += 1;
    }
  }
  return Rad{(uint32_t)m, E + t};
}

// b on the scale 2^(e_a - 63), rounded up; d = e_a - e_b >= 0
__device__ __forceinline__ uint64_t rad_scale_up(const Rad& b, int64_t d) {
  if (d <= 31) return (uint64_t)b.m << (31 - d);
  const int64_t sh = d - 31;
  if (sh >= 32) return 1ull;
  uint64_t v = (uint64_t)b.m >> sh;
  if ((uint64_t)b.m & ((1ull << sh) - 1ull)) v += 1ull;
  return v;
}

__device__ __forceinline__ Rad rad_sum(Rad a, Rad b) {
  if (rad_isinf(a) || rad_isinf(b)) return rad_unbounded();
  if (rad_isz(a)) return b;
  if (rad_isz(b)) return a;
  if (b.e > a.e) {
    const Rad t = a;
    a = b;
    b = t;
  }
  return rad_of(((uint64_t)a.m << 31) + rad_scale_up(b, a.e - b.e), a.e - 63, true);
}

__device__ __forceinline__ Rad rad_prod(const Rad& a, const Rad& b, bool up) {
  if (rad_isz(a) || rad_isz(b)) return rad_zero();
  if (rad_isinf(a) || rad_isinf(b)) return rad_unbounded();
  return rad_of((uint64_t)a.m * (uint64_t)b.m, a.e + b.e - 64, up);
}

__device__ __forceinline__ Rad rad_quot_up(const Rad& a, const Rad& b) {
  if (rad_isz(a)) return rad_zero();
  if (rad_isinf(a)) return rad_unbounded();
  const uint64_t num = (uint64_t)a.m << 32;
  uint64_t q = num / b.m;
  if (q * b.m != num) q += 1ull;
  return rad_of(q, a.e - b.e - 32, true);
}

// a - b rounded down; pos = false when a - b <= 0
__device__ __forceinline__ Rad rad_diff_down(const Rad& a, const Rad& b, bool& pos) {
  pos = false;
  if (rad_isinf(b) || rad_isz(a)) return rad_zero();
  if (rad_isz(b)) {
    pos = true;
    return a;
  }
  if (b.e > a.e) return rad_zero();
  const uint64_t A = (uint64_t)a.m << 31, B = rad_scale_up(b, a.e - b.e);
  if (B >= A) return rad_zero();
  pos = true;
  return rad_of(A - B, a.e - 63, false);
}

__device__ __forceinline__ Rad rad_half_ulp(int64_t e, int p) {
  return (e == ZEXP) ? rad_zero() : Rad{0x80000000u, e - p};
}

// Bounds of |x| for a number held by the group (slices A, exponent e):
// its top limb, plus one when any other limb is set (up).  Every lane of the
// warp must call it (a ballot); all lanes get the same result.
template <int W, int G>
__device__ __forceinline__ Rad rad_mag(const Grp<G>& gp, int64_t e, const uint32_t (&A)[W], bool up) {
  const uint32_t top = gp.from(A[W - 1], G - 1);
  uint32_t any = 0u;
#pragma unroll
  for (int i = 0; i < W; ++i)
    if (!(gp.g == G - 1 && i == W - 1)) any |= A[i];
  const bool rest = gp.ballot(any != 0u) != 0u;
  if (e == ZEXP) return rad_zero();
  return rad_of((uint64_t)top + ((up && rest) ? 1ull : 0ull), e - 32, up);
}

// The same for a number in memory (every lane of the group reads its slice).
template <int W, int G>
__device__ __forceinline__ Rad rad_mag_mem(const Grp<G>& gp, int64_t e, const uint32_t* m, bool up) {
  uint32_t A[W];
  load_slice<W>(m + gp.g * W, A);
  return rad_mag<W, G>(gp, e, A, up);
}

// Product rule: x, y with magnitudes bounded above by mx, my.
__device__ __forceinline__ Rad ball_prod(int p, int64_t eu, const Rad& mx, const Rad& rx, const Rad& my,
                                         const Rad& ry) {
  Rad r = rad_sum(rad_half_ulp(eu, p), rad_prod(mx, ry, true));
  r = rad_sum(r, rad_prod(my, rx, true));
  return rad_sum(r, rad_prod(rx, ry, true));
}

__device__ __forceinline__ Rad ball_diff(int p, int64_t eu, const Rad& rx, const Rad& rt) {
  return rad_sum(rad_sum(rad_half_ulp(eu, p), rx), rt);
}

// Reciprocal rule: lo = |a~|_ .
__device__ __forceinline__ Rad ball_inv(int p, int64_t eu, const Rad& lo, const Rad& ra) {
  bool pos = false;
  const Rad gap = rad_diff_down(lo, ra, pos);
  if (!pos) return rad_unbounded();
  return rad_sum(rad_half_ulp(eu, p), rad_quot_up(ra, rad_prod(lo, gap, false)));
}

__device__ __forceinline__ Rad rad_load(const uint32_t* rm, const int64_t* re, int64_t i) { return Rad{rm[i], re[i]}; }
__device__ __forceinline__ void rad_store(uint32_t* rm, int64_t* re, int64_t i, const Rad& r) {
  rm[i] = r.m;
  re[i] = r.e;
}

}  // namespace mpd
