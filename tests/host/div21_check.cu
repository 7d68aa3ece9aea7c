// Host check of the 2-by-1 limb division the pivot reciprocal uses
// (div21_preinv with div21_inverse, compiled for the CPU from the kernels'
// own header) against exact 64-by-32-bit division: divisors at the corners of
// the normalised range and random ones, dividends (u1, u0) with u1 < d at
// their extremes and random.  Prints the number of cases and of mismatches.
#include <cstdint>
#include <cstdio>

#include "../../paper_1308_1536_gb300/csrc/mpdev.cuh"

using mpd::div21_inverse;
using mpd::div21_preinv;

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint32_t rnd32() {  // splitmix64, upper half
  state += 0x9E3779B97F4A7C15ull;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return (uint32_t)((z ^ (z >> 31)) >> 32);
}

int main() {
  uint64_t cases = 0, bad = 0;
  auto check = [&](uint32_t u1, uint32_t u0, uint32_t d) {
    if (u1 >= d) return;
    const uint64_t u = ((uint64_t)u1 << 32) | u0;
    uint32_t r = 0;
    const uint32_t q = div21_preinv(u1, u0, d, div21_inverse(d), r);
    ++cases;
    if (q != (uint32_t)(u / d) || r != (uint32_t)(u % d)) {
      if (bad < 5) printf("mismatch u1=%08x u0=%08x d=%08x q=%08x r=%08x\n", u1, u0, d, q, r);
      ++bad;
    }
  };
  const uint32_t dc[] = {0x80000000u, 0x80000001u, 0x80000002u, 0xC0000000u, 0xFFFFFFFEu, 0xFFFFFFFFu,
                         0xAAAAAAAAu, 0x55555555u | 0x80000000u, 0x80008000u, 0xFFFF0000u};
  for (uint32_t d : dc) {
    const uint32_t u1s[] = {0u, 1u, d - 1u, d - 2u, d >> 1, (d >> 1) + 1u};
    const uint32_t u0s[] = {0u, 1u, 0xFFFFFFFFu, 0xFFFFFFFEu, 0x80000000u, d, d - 1u};
    for (uint32_t u1 : u1s)
      for (uint32_t u0 : u0s) check(u1, u0, d);
    for (int i = 0; i < 200000; ++i) check(rnd32() % d, rnd32(), d);
  }
  for (int i = 0; i < 4000000; ++i) {
    const uint32_t d = rnd32() | 0x80000000u;
    const uint32_t u1 = (i & 3) == 0 ? d - 1u - (rnd32() & 15u) : rnd32() % d;
    check(u1, rnd32(), d);
  }
  // every divisor with few significant bits below the top (the estimate's
  // correction steps are taken most often near these)
  for (uint32_t hi = 0; hi < (1u << 12); ++hi) {
    const uint32_t d = 0x80000000u | (hi << 19);
    check(d - 1u, 0xFFFFFFFFu, d);
    check(d - 1u, 0u, d);
    check(rnd32() % d, rnd32(), d);
  }
  printf("cases %llu mismatches %llu\n", (unsigned long long)cases, (unsigned long long)bad);
  return bad != 0;
}
