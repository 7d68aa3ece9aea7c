// Tensor-core engine for the rank-1 update at p = 4096 .. 32768 (n = 128 ..
// 1024 limbs): x_ij = RN(x_ij - RN(z_i * b_j)), b_j = x_{brow,j}.
//
// The exact product of two mantissas as a digit convolution on the 5th
// generation tensor cores (kind::f16: bf16 operands, fp32 accumulation),
// with digits of different sizes on the two sides so that a whole column
// sum, over every digit of z, stays exact in fp32:
//   z: KD = 4n balanced 8-bit digits e_s in [-128, 127] (the bytes of
//      m_z + 0x80..80, less 128); a normalised mantissa carries 1 out of its
//      top digit, so m_z = z' + 2^p with z' = sum e_s 256^s.
//   b: KB = 8n balanced 4-bit digits f_t in [-8, 7] (the nibbles of
//      m_b + 0x88..8, less 8) and the carry digit f_KB = 1: m_b = sum f_t 16^t.
// Then m_z m_b = sum_r c_r 16^r + 2^p m_b with the radix-16 column sums
//   c_r = sum_{2s + t = r} e_s f_t,
// at most KD terms in [-1016, 1024], so c_r lies in [-1016 KD, 1024 KD]: a
// window narrower than 2^23 at every n <= 1024, exact in fp32, and adding
// kMagic = 2^23 + 1016 KD puts it in [2^23, 2^24) where the fp32 bits are
// 0x4B000000 + (c_r + 1016 KD).  The MMA adds kMagic itself: one more K step
// per tile, issued after the digit steps, multiplies a constant A with ones
// in two columns by a constant B holding 2^23 and 1016 KD (both exact in
// bf16); every partial sum before it is an integer below 2^23 in magnitude,
// the final one lies in [2^23, 2^24), so all of them are exact.  The 2^p m_b
// term is added to the limbs by the epilogue.
//
// GEMM shape, per block of M = 128 rows i and one column j: D[i][r] =
// sum_k' A[i][k'] B[k'][r], K reversed (k' = KD - 1 - s):
//   A[i][k'] = e_{KD-1-k'}(z_i): precomputed per step (k_zdig) in global
//     memory, row-major, and streamed by TMA with 128-byte swizzle, 256
//     digits x 128 rows (four 16 KB boxes) per pipeline stage;
//   B[k'][r] = f_{r + 2k' - 2KD + 2}(b_j): its 8 x 8 core matrices (k-core
//     kc, n-core nc) depend only on d = nc + 2 kc, so one no-swizzle
//     descriptor with leading offset 256 and stride offset 128 bytes reads
//     them from a run of 78 distinct cores, kept in a sliding ring (below)
//     and built from b_j's digits.
// Lazy low half: only the positions r >= R0 = 8n - 256 are formed (the upper
// n limbs of the product and 32 limbs below them), in T = n/32 + 1 tiles of
// 256 positions, two tiles (all 512 tensor-memory columns) per pass.  The
// positions below contribute less than 2^19 units of limb n - 32 in
// magnitude; when bits [19, 992) of limbs n-32 .. n-2 hold both a one and a
// zero, neither those limbs' carry out nor the sticky bit depends on them (the
// sticky bit is then 1).  Otherwise the subtraction role recomputes that
// product exactly with the IMAD engine's mul_round.
//
// Roles (384 threads, one block per SM, persistent over a range of (row
// block, column) items):
//   warp 0       TMA producer of the A stages (2-stage ring of 16 MMA K steps)
//   warp 1       MMA issuer (one thread); the bias step last in each tile
//   warps 2-3    builders: b_j's balanced nibbles per column, the new B cores
//                of each stage
//   warps 4-7    epilogue: one thread per row drains the column sums of a pass
//                from tensor memory, forms the limbs (running carry) and
//                stores the product's upper n limbs in a global slab
//   warps 8-11   subtraction: lane groups round the staged product and
//                subtract it from x_ij (round_product, sub_round: the IMAD
//                engine's code), two slab buffers per block
// Every wait is bounded; a timeout sets MPDET_ETIMEOUT through the status
// word, every role drains, the block waits for its copies and MMAs in flight
// and frees its tensor memory.  Results are bit-identical to the IMAD engine.
#include <cuda.h>

#include "kernels.cuh"

namespace mpd {
namespace tcl {

constexpr int M = 128;       // rows per block (MMA M)
constexpr int NT = 256;      // positions per tile (MMA N)
// Stage geometry (in Cfg): KSPS MMA K steps of 16 digits per stage, STAGES
// stages in the ring; a stage's B window spans NCORE cores.  The B cores live
// in a sliding ring of RING = STAGES * NCORE cores plus a mirror of its first
// MIRROR = NCORE - 4 KSPS, so that every window is contiguous: within a pass
// each stage's window starts 4 KSPS cores after the previous one's (the next
// NCORE - 4 KSPS are shared), so a stage builds 4 KSPS new cores, the first
// stage of a pass all NCORE.  The window start advances by 4 KSPS per stage
// and by NCORE after a pass's last stage, so it is a multiple of 4 KSPS and a
// window runs at most MIRROR cores past the ring's end.  The builders of stage
// g wait for stage g - STAGES to complete, so stages g-STAGES+1 .. g-1 are the
// only ones in flight, and the cores stage g writes lie less than RING cores
// after the first core of stage g-STAGES+1's window: no core still to be read
// is overwritten.
constexpr int NTH = 384;
constexpr int LIMIT = 1 << 22;


template <int n>
struct Cfg {
  static constexpr int KD = 4 * n;          // 8-bit digits of z
  static constexpr int KB = 8 * n;          // 4-bit digits of b
  static constexpr int R0 = 8 * n - 256;    // lowest position formed
  static constexpr int T = n / 32 + 1;      // tiles of 256 positions
  static constexpr int NPASS = (T + 1) / 2;
  static constexpr int W = n <= 512 ? 16 : 32;
  static constexpr int G = n / W;
  static constexpr int NGRP = 128 / G;      // subtraction lane groups
  static constexpr int SW = Scratch<W, G>::words;
  static constexpr int OFFU = 8;            // index of u = 0 in the nibble arrays
  static constexpr int FL = KB / 2 + 16;    // entries per parity array
  static constexpr int kOff = 1016 * KD;
  static constexpr int KSPS = 16;                     // MMA K steps per stage
  static constexpr int STAGES = 2;                    // ring depth
  static constexpr int NCORE = (63 + 4 * KSPS + 15) / 16 * 16;  // B window (63 + 4 KSPS cores read)
  static constexpr int RING = STAGES * NCORE;
  static constexpr uint32_t A_BYTES = M * 16 * KSPS * 2;  // 128 rows x 16 KSPS digits: KSPS / 4 swizzle boxes
  static constexpr int MIRROR = NCORE - 4 * KSPS;
  static_assert(NCORE % (4 * KSPS) == 0, "window starts multiples of 4 KSPS");
  static constexpr uint32_t B_BYTES = (RING + MIRROR) * 128;
  static constexpr int OFF_A = 0;
  static constexpr int OFF_B = OFF_A + STAGES * (int)A_BYTES;
  static constexpr int OFF_F = OFF_B + (int)B_BYTES;                   // two bf16 parity arrays
  static constexpr int OFF_SCR = OFF_F + (2 * FL * 2 + 15) / 16 * 16;  // subtraction scratch
  static constexpr int OFF_META = OFF_SCR + NGRP * SW * 4;            // 2 x 128 x 32 bytes
  static constexpr int OFF_ONE = OFF_META + 2 * M * 32;  // A of the bias step: 2 k-cores x 16 m-cores
  static constexpr int OFF_BIAS = OFF_ONE + 4096;        // B of the bias step: 2 k-cores x 32 n-cores
  static constexpr int OFF_BAR = OFF_BIAS + 8192;
  static constexpr int SMEM = OFF_BAR + 8 * (3 * STAGES + 10);
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert((long long)KD * 2040 < (1ll << 23), "column sums exact with the magic bias");
  static_assert(OFF_ONE % 16 == 0 && OFF_BAR % 16 == 0, "alignment");
  // MMA K steps (16 reversed digits) that meet tile tau's positions
  // [rho, rho + 256): s from max(0, ceil((rho - KB) / 2)) to
  // min(KD - 1, floor((rho + 255) / 2))
  __host__ __device__ static constexpr int ks_lo(int tau) {
    return (KD - 1 - ((R0 + 256 * tau + 255) / 2 < KD - 1 ? (R0 + 256 * tau + 255) / 2 : KD - 1)) / 16;
  }
  __host__ __device__ static constexpr int ks_hi(int tau) {
    return (KD - 1 - (R0 + 256 * tau > KB ? (R0 + 256 * tau - KB + 1) / 2 : 0)) / 16 + 1;
  }
  __host__ __device__ static constexpr int ntile(int pi) { return 2 * pi + 1 < T ? 2 : 1; }
  // stages (16 KSPS reversed digits each) of pass pi: [sg_lo, sg_hi)
  __host__ __device__ static constexpr int sg_lo(int pi) {
    return (ntile(pi) == 2 && ks_lo(2 * pi + 1) < ks_lo(2 * pi) ? ks_lo(2 * pi + 1) : ks_lo(2 * pi)) / KSPS;
  }
  __host__ __device__ static constexpr int sg_hi(int pi) {
    return ((ntile(pi) == 2 && ks_hi(2 * pi + 1) > ks_hi(2 * pi) ? ks_hi(2 * pi + 1) : ks_hi(2 * pi)) + KSPS - 1) /
           KSPS;
  }
};

// Per (buffer, row) record the epilogue leaves for the subtraction role.
struct Meta {
  int64_t te;        // exponent of the exact product (before rounding), ZEXP if it is zero
  uint32_t ltop;     // limb n - 1
  uint32_t sticky;   // OR of the limbs below n - 1 (non-zero)
  int32_t ts;        // sign
  int32_t unsafe;    // the lazy low half could not decide: recompute exactly
  int64_t pad;
};
static_assert(sizeof(Meta) == 32, "meta record");

// slab reads bypass L1: the slab is written by other warps of the block
template <int W>
__device__ __forceinline__ void load_slice_cg(const uint32_t* src, uint32_t (&v)[W]) {
#pragma unroll
  for (int q = 0; q < W; q += 4) {
    const uint4 t = __ldcg(reinterpret_cast<const uint4*>(src + q));
    v[q] = t.x;
    v[q + 1] = t.y;
    v[q + 2] = t.z;
    v[q + 3] = t.w;
  }
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// UMMA shared-memory descriptor, no swizzle, K-major: lbo steps between core
// matrices along K, sbo along M / N.
// UMMA shared-memory descriptor of a K-major operand in the 128-byte swizzle
// layout: rows of 128 bytes, 8-row groups 1024 bytes apart (stride offset);
// a K step of 16 bf16 moves the start address by 32 bytes within the row.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < LIMIT && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
  return done != 0;
}

// named barrier 1 over the 64 builder threads; returns the OR of q over them
__device__ __forceinline__ bool bbar_or(bool q) {
  uint32_t r;
  __syncwarp();
  asm volatile("{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.or.pred b, 1, 64, a;\n selp.u32 %0, 1, 0, b;\n}"
               : "=r"(r)
               : "r"((uint32_t)q)
               : "memory");
  return r != 0;
}
__device__ __forceinline__ void bbar() {
  __syncwarp();
  asm volatile("bar.sync 1, 64;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
                 "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]),
                 "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]),
                 "+r"(v[30]), "+r"(v[31]));
}

// 32 columns without waiting: the registers are valid after tmem_wait(v)
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
// wait for this thread's tensor-memory loads; v is named so that no use of it
// moves above the wait
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
                 "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]),
                 "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]),
                 "+r"(v[30]), "+r"(v[31]));
}

// bf16 bits of a small integer (|e| <= 256: exact)
__device__ __forceinline__ uint32_t bfi(int e) { return __float_as_uint((float)e) >> 16; }

// ---------------------------------------------------------------------------
// A operand: balanced 8-bit digits of the multipliers z_i, i in [row0, row0 +
// nrows), as bf16, row-major: Zd[i][k'] holds digit s = KD - 1 - k' of z_i
// (rows i of the whole N-row array).  A TMA copy with 128-byte swizzle moves
// 64 digits of 128 rows into the layout the MMA reads (K-major, 128-byte
// swizzle).  One thread per row; the carry chain runs over the limbs.
// ---------------------------------------------------------------------------
template <int n>
__global__ void k_zdig(MpArr Z, int64_t N, int64_t row0, int64_t nrows, uint4* __restrict__ zd) {
  constexpr int KD = 4 * n;
  const int64_t i = row0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= row0 + nrows) return;
  const bool zero = Z.e[i] == ZEXP;
  const uint32_t* zm = Z.m + i * n;
  uint64_t cy = 0;
#pragma unroll 4
  for (int m = 0; m < n / 2; ++m) {
    // limbs 2m, 2m + 1: digits s = 8m .. 8m + 7, reversed k' = KD - 1 - s:
    // k-core KD/8 - 1 - m, element kk = 7 - (s - 8m)
    const uint2 w = zero ? make_uint2(0u, 0u) : *reinterpret_cast<const uint2*>(zm + 2 * m);
    uint64_t t0 = (uint64_t)w.x + 0x80808080u + cy;
    const uint32_t y0 = (uint32_t)t0;
    uint64_t t1 = (uint64_t)w.y + 0x80808080u + (t0 >> 32);
    const uint32_t y1 = (uint32_t)t1;
    cy = t1 >> 32;
    uint32_t h[8];  // h[q]: digit s = 8m + q
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      h[q] = __float_as_uint(__uint_as_float(0x4B000000u | ((y0 >> (8 * q)) & 255u)) - 8388736.0f) >> 16;
      h[q + 4] = __float_as_uint(__uint_as_float(0x4B000000u | ((y1 >> (8 * q)) & 255u)) - 8388736.0f) >> 16;
    }
    // element kk holds digit q = 7 - kk
    zd[i * (KD / 8) + (KD / 8 - 1 - m)] =
        make_uint4(h[7] | (h[6] << 16), h[5] | (h[4] << 16), h[3] | (h[2] << 16), h[1] | (h[0] << 16));
  }
}

template <int n>
__global__ void __launch_bounds__(NTH, 1) k_update_tcl(MpArr X, UpdArgs a, MpArr Z, int* status, int p,
                                                      uint32_t* __restrict__ slab,
                                                      const __grid_constant__ CUtensorMap tmz) {
  using C = Cfg<n>;
  constexpr int W = C::W, G = C::G;
  constexpr int STAGES = C::STAGES, KSPS = C::KSPS, NCORE = C::NCORE, RING = C::RING;
  constexpr uint32_t A_BYTES = C::A_BYTES;
  extern __shared__ __align__(1024) unsigned char sm[];
  if (upd_stopped(status, a)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the TMA destinations assume a 1024-byte aligned window: refuse
  // (MPDET_ECUDA) rather than copy elsewhere
  if (su32(sm) & 1023u) {
    if (tid == 0) atomicExch(status, 3);
    return;
  }
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::OFF_BAR);
  // [0, S) afull, [S, 2S) bfull, [2S, 3S) empty (S = STAGES); then tfull, tempty (tensor-memory
  // half 0), tempty1 (half 1), sfull x 2, sfree x 2, mdone, the tensor-memory address (u32) and
  // the error flag
  constexpr int S3 = 3 * STAGES;
  const uint32_t b_afull = su32(&bars[0]), b_bfull = su32(&bars[STAGES]), b_empty = su32(&bars[2 * STAGES]);
  const uint32_t b_tfull = su32(&bars[S3]), b_tempty = su32(&bars[S3 + 1]), b_tempty1 = su32(&bars[S3 + 2]);
  const uint32_t b_sfull = su32(&bars[S3 + 3]), b_sfree = su32(&bars[S3 + 5]), b_mdone = su32(&bars[S3 + 7]);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(&bars[S3 + 8]);
  volatile int* eflag = reinterpret_cast<volatile int*>(&bars[S3 + 9]);
  Meta* meta = reinterpret_cast<Meta*>(sm + C::OFF_META);
  uint16_t* F0 = reinterpret_cast<uint16_t*>(sm + C::OFF_F);  // f~(2u), u = index - OFFU
  uint16_t* F1 = F0 + C::FL;                                  // f~(2u + 1)

  const int64_t N = a.N;
  const int64_t ncols = a.ncols;
  const int64_t rend = a.row0 + a.nrows;
  const int64_t nb = (a.nrows + M - 1) / M;
  const int64_t items = nb * ncols;
  const int64_t q0 = items * blockIdx.x / gridDim.x, q1 = items * (blockIdx.x + 1) / gridDim.x;

  // ---- set-up --------------------------------------------------------------
  for (int q = tid; q < 2 * C::FL; q += NTH) F0[q] = 0;  // zero padding around the digits
  // the bias step: A rows (1, 1, 0, ...) in k-core 0; B rows 2^23 and 1016 KD
  // at every position in k-core 0; k-core 1 of both zero
  for (int q = tid; q < (4096 + 8192) / 16; q += NTH) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (q < 128) v.x = 0x3F803F80u;                                              // A: 1.0, 1.0
    else if (q >= 256 && q < 256 + 256) v.x = 0x4B00u | (bfi(C::kOff) << 16);    // B: 2^23, kOff
    reinterpret_cast<uint4*>(sm + C::OFF_ONE)[q] = v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_afull + 8 * s));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_bfull + 8 * s));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_empty + 8 * s));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_tfull));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(b_tempty));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(b_tempty1));
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(b_sfull + 8 * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(b_sfree + 8 * b));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_mdone));
    *eflag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ================= producer: A stages by TMA ==========================
    if (lane == 0) {
      int64_t g = 0;
      bool ok = true;
      for (int64_t q = q0; q < q1 && ok; ++q) {
        const int i0 = (int)(a.row0 + (q / ncols) * M);
        for (int pi = 0; pi < C::NPASS && ok; ++pi)
          for (int sg = C::sg_lo(pi); sg < C::sg_hi(pi); ++sg, ++g) {
            const int slot = (int)(g % STAGES);
            if (g >= STAGES && !wait_bar(b_empty + 8 * slot, (uint32_t)((g / STAGES - 1) & 1))) ok = false;
            if (!ok || *eflag) {
              ok = false;
              break;
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b_afull + 8 * slot),
                         "r"(A_BYTES)
                         : "memory");
            for (int bx = 0; bx < KSPS / 4; ++bx)
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                  "[%4];" ::"r"(su32(sm + C::OFF_A + slot * A_BYTES + 16384 * bx)),
                  "l"(reinterpret_cast<uint64_t>(&tmz)), "r"(16 * KSPS * sg + 64 * bx), "r"(i0), "r"(b_afull + 8 * slot)
                  : "memory");
          }
      }
      if (!ok) *eflag = 1;
      // no copy may still be writing shared memory at exit: the last copy of
      // each slot completes that slot's most recent phase
      for (int64_t s = g - 1; s >= 0 && s >= g - STAGES; --s)
        wait_bar(b_afull + 8 * (int)(s % STAGES), (uint32_t)((s / STAGES) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ================= MMA issuer =========================================
    if (lane == 0) {
      const uint32_t idesc =
          (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
      int64_t g = 0;
      int wpos = 0;                  // ring slot of the current stage's window
      int64_t uses0 = 0, uses1 = 0;  // passes that used tensor-memory half 0 / 1 so far
      bool ok = true;
      const uint64_t ad_one = desc(su32(sm + C::OFF_ONE), 2048, 128);
      const uint64_t bd_bias = desc(su32(sm + C::OFF_BIAS), 4096, 128);
      for (int64_t q = q0; q < q1 && ok; ++q)
        for (int pi = 0; pi < C::NPASS && ok; ++pi) {
          if (*eflag) {
            ok = false;
            break;
          }
          const int nt = C::ntile(pi);
          // a half is free once the epilogue has read the previous pass's
          // sums from it; the two halves are waited for separately, so that
          // the MMAs into half 0 start while half 1 is still being read
          bool started0 = false, started1 = false;
          for (int sg = C::sg_lo(pi); sg < C::sg_hi(pi); ++sg, ++g) {
            const int slot = (int)(g % STAGES);
            const uint32_t ph = (uint32_t)((g / STAGES) & 1);
            if (!wait_bar(b_afull + 8 * slot, ph) || !wait_bar(b_bfull + 8 * slot, ph) || *eflag) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t aS = su32(sm + C::OFF_A + slot * A_BYTES);
            const uint32_t bS = su32(sm + C::OFF_B + wpos * 128);
            wpos += sg + 1 < C::sg_hi(pi) ? 4 * KSPS : NCORE;
            if (wpos >= RING) wpos -= RING;
            for (int t = 0; t < nt; ++t) {
              const int tau = 2 * pi + t;
              const int lo = C::ks_lo(tau) > KSPS * sg ? C::ks_lo(tau) : KSPS * sg;
              const int hi = C::ks_hi(tau) < KSPS * sg + KSPS ? C::ks_hi(tau) : KSPS * sg + KSPS;
              bool& started = t ? started1 : started0;
              if (lo < hi && !started) {
                const int64_t u = t ? uses1 : uses0;
                if (u >= 1 && !wait_bar(t ? b_tempty1 : b_tempty, (uint32_t)((u - 1) & 1))) {
                  ok = false;
                  break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
              }
              for (int ks = lo; ks < hi; ++ks) {
                const uint32_t kl = (uint32_t)(ks - KSPS * sg);  // K step within the stage
                const uint64_t ad = desc_sw128(aS + 16384u * (kl >> 2) + 32u * (kl & 3u));
                const uint64_t bd = desc(bS + 128u * (32u * (uint32_t)t + 4u * kl), 256, 128);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, "
                    "p;\n}" ::"r"(tmem + (uint32_t)(NT * t)),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(started ? 1u : 0u));
                started = true;
              }
            }
            if (!ok) break;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                b_empty + 8 * slot));
          }
          if (!ok) break;
          // the bias step, last into each tile of the pass
          for (int t = 0; t < nt; ++t)
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, "
                "p;\n}" ::"r"(tmem + (uint32_t)(NT * t)),
                "l"(ad_one), "l"(bd_bias), "r"(idesc), "r"(1u));
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b_tfull));
          uses0 += 1;
          if (nt == 2) uses1 += 1;
        }
      if (!ok) *eflag = 1;
      // every MMA issued has completed before the tensor memory is freed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b_mdone));
      wait_bar(b_mdone, 0);
    }
    __syncwarp();
  } else if (warp < 4) {
    // ================= builders: B cores ==================================
    const int bt = tid - 64;
    int64_t g = 0;
    int wpos = 0;  // ring slot of the current stage's window
    bool stop = false;
    for (int64_t q = q0; q < q1 && !stop; ++q) {
      const int64_t kj = a.brow * N + upd_col(a, q % ncols);
      const bool bz = X.e[kj] == ZEXP;
      bbar();  // the previous column's cores are built: its digits may be replaced
      if (warp == 2) {
        // balanced nibbles: the nibbles of m_b + 0x88..8, less 8; lane l adds
        // its limbs [l LPL, (l + 1) LPL), carries across lanes by lookahead
        constexpr int LPL = n / 32;
        uint32_t y[LPL];
        const uint32_t* bm = X.m + kj * n + lane * LPL;
#pragma unroll
        for (int k = 0; k < LPL; k += 4) {
          const uint4 v = bz ? make_uint4(0u, 0u, 0u, 0u) : *reinterpret_cast<const uint4*>(bm + k);
          y[k] = v.x;
          y[k + 1] = v.y;
          y[k + 2] = v.z;
          y[k + 3] = v.w;
        }
        y[0] = add_cc(y[0], 0x88888888u);
#pragma unroll
        for (int k = 1; k < LPL; ++k) y[k] = addc_cc(y[k], 0x88888888u);
        const uint32_t c0 = addc(0u, 0u);
        const uint64_t cm = carry_mask(__ballot_sync(FULL, c0 != 0u), __ballot_sync(FULL, all_ones<LPL>(y)), 0u);
        slice_inc<LPL>(y, (uint32_t)(cm >> lane) & 1u);
#pragma unroll
        for (int k = 0; k < LPL; ++k) {
          const int L = lane * LPL + k;
          const uint32_t v = y[k];
          // nibble q of limb L is f~(8L + q): parity q & 1, u = 4L + (q >> 1)
          const uint32_t e0 = bfi((int)(v & 15u) - 8), e1 = bfi((int)((v >> 4) & 15u) - 8);
          const uint32_t e2 = bfi((int)((v >> 8) & 15u) - 8), e3 = bfi((int)((v >> 12) & 15u) - 8);
          const uint32_t e4 = bfi((int)((v >> 16) & 15u) - 8), e5 = bfi((int)((v >> 20) & 15u) - 8);
          const uint32_t e6 = bfi((int)((v >> 24) & 15u) - 8), e7 = bfi((int)(v >> 28) - 8);
          *reinterpret_cast<uint2*>(F0 + C::OFFU + 4 * L) = make_uint2(e0 | (e2 << 16), e4 | (e6 << 16));
          *reinterpret_cast<uint2*>(F1 + C::OFFU + 4 * L) = make_uint2(e1 | (e3 << 16), e5 | (e7 << 16));
        }
        if (lane == 31) F0[C::OFFU + C::KB / 2] = (uint16_t)bfi((int)((cm >> 32) & 1u));  // the carry digit f~(KB)
      }
      bbar();
      for (int pi = 0; pi < C::NPASS && !stop; ++pi) {
        const int nc0 = (C::R0 + 512 * pi) / 8;
        for (int sg = C::sg_lo(pi); sg < C::sg_hi(pi); ++sg, ++g) {
          const int slot = (int)(g % STAGES);
          bool bad = false;
          if (bt == 0 && g >= STAGES && !wait_bar(b_empty + 8 * slot, (uint32_t)((g / STAGES - 1) & 1))) bad = true;
          if (bbar_or(bad || *eflag != 0)) {
            stop = true;
            break;
          }
          // core d = d0 + dl of the window, row rr: f~(8d + rr + 2kk - 2KD + 2),
          // kk = 0..7, = F_{rr & 1}[u0 + kk] with u0 = 4d + (rr >> 1) - KD + 1;
          // the first stage of a pass builds the whole window, the others its
          // last 4 KSPS cores
          unsigned char* Bring = sm + C::OFF_B;
          const int d0 = nc0 + 4 * KSPS * sg;
          const int dl0 = sg == C::sg_lo(pi) ? 0 : NCORE - 4 * KSPS;
          for (int q2 = bt; q2 < (NCORE - dl0) * 8; q2 += 64) {
            const int dl = dl0 + (q2 >> 3), rr = q2 & 7;
            const int u0 = 4 * (d0 + dl) + (rr >> 1) - C::KD + 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (u0 + 7 >= 0 && u0 <= C::KB / 2) {
              const uint16_t* f = ((rr & 1) ? F1 : F0) + C::OFFU + u0;
              v = make_uint4((uint32_t)f[0] | ((uint32_t)f[1] << 16), (uint32_t)f[2] | ((uint32_t)f[3] << 16),
                             (uint32_t)f[4] | ((uint32_t)f[5] << 16), (uint32_t)f[6] | ((uint32_t)f[7] << 16));
            }
            int x = wpos + dl;
            if (x >= RING) x -= RING;
            *reinterpret_cast<uint4*>(Bring + x * 128 + rr * 16) = v;
            if (x < C::MIRROR) *reinterpret_cast<uint4*>(Bring + (x + RING) * 128 + rr * 16) = v;  // mirror
          }
          wpos += sg + 1 < C::sg_hi(pi) ? 4 * KSPS : NCORE;
          if (wpos >= RING) wpos -= RING;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // read by the tensor core
          bbar();
          if (bt == 0) arrive(b_bfull + 8 * slot);
        }
      }
    }
    if (stop) *eflag = 1;
  } else if (warp < 8) {
    // ================= epilogue: one thread per row =======================
    const int r = tid - 128;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const int64_t kOffL = (int64_t)C::kOff * 0x11111111ll;
    int64_t pg = 0, it = 0;
    bool ok = true;
    // b's limbs of a pass, a pass ahead: limbs L - n of the pass's 64 limbs
    // L = n - 32 + 64 pi .. n + 31 + 64 pi (zero below limb n), lane l
    // holding offsets l (word 0) and 32 + l (word 1); a chunk takes its four
    // by shuffles
    auto bload = [&](const uint32_t* bmp, const int pi, uint32_t& w0, uint32_t& w1) {
      const int k0 = 64 * pi - 32 + lane, k1 = 64 * pi + lane;
      w0 = k0 >= 0 && k0 < n ? __ldg(bmp + k0) : 0u;
      w1 = k1 < n ? __ldg(bmp + k1) : 0u;
    };
    uint32_t bw0 = 0, bw1 = 0;
    if (q0 < q1) bload(X.m + (a.brow * N + upd_col(a, q0 % ncols)) * n, 0, bw0, bw1);
    for (int64_t q = q0; q < q1 && ok; ++q, ++it) {
      const int64_t i0 = a.row0 + (q / ncols) * M;
      const int64_t j = upd_col(a, q % ncols);
      const int64_t i = i0 + r;
      const bool active = i < rend;
      const int64_t ze = active ? Z.e[i] : ZEXP;
      const int8_t zs = active ? Z.s[i] : (int8_t)0;
      const int64_t kj = a.brow * N + j;
      const int64_t be = X.e[kj];
      const int8_t bs = X.s[kj];
      const uint32_t* bm = X.m + kj * n;
      const bool used = ze != ZEXP && be != ZEXP;
      const int buf = (int)(it & 1);
      uint32_t* srow = slab + ((size_t)(blockIdx.x * 2 + buf) * M + r) * n;
      if (it >= 2) {
        bool okw = wait_bar(b_sfree + 8 * buf, (uint32_t)(((it - 2) >> 1) & 1));
        ok = __all_sync(FULL, okw);
        if (!ok) break;
      }
      int64_t acc = 0;
      uint32_t l0 = 0, orv = 0, andv = 0xffffffffu, ltop = 0;
      for (int pi = 0; pi < C::NPASS; ++pi, ++pg) {
        // the next pass's b limbs (the next item's first pass after the last)
        uint32_t bn0 = 0, bn1 = 0;
        if (pi + 1 < C::NPASS)
          bload(bm, pi + 1, bn0, bn1);
        else if (q + 1 < q1)
          bload(X.m + (a.brow * N + upd_col(a, (q + 1) % ncols)) * n, 0, bn0, bn1);
        bool okt = wait_bar(b_tfull, (uint32_t)(pg & 1)) && !*eflag;
        ok = __all_sync(FULL, okt);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int nch = 8 * C::ntile(pi);
        // chunk ch: 32 sums (4 limbs) whose fp32 bits are 0x4B000000 + u,
        // u = c_r + kOff; the next chunk's load is in flight meanwhile
        auto step = [&](const int ch, uint32_t(&cur)[32], uint32_t(&nxt)[32]) {
          tmem_wait(cur);
          if (ch + 1 < nch) tmem_ld32_async(tl + (uint32_t)(32 * (ch + 1)), nxt);
          const uint32_t bsrc = ch < 8 ? bw0 : bw1;
          uint32_t bl[4];
#pragma unroll
          for (int l4 = 0; l4 < 4; ++l4) bl[l4] = __shfl_sync(FULL, bsrc, (4 * ch + l4) & 31);
          if ((ch & 7) == 7) {  // a tile's sums are in registers: free its half of the tensor memory
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) arrive(ch == 7 ? b_tempty : b_tempty1);
          }
          const int L0 = n - 32 + 64 * pi + 4 * ch;  // first limb of the chunk
          uint32_t lim[4];
#pragma unroll
          for (int l4 = 0; l4 < 4; ++l4) {
            const uint32_t* w = cur + 8 * l4;
            // w0 + 16 w1 = u0 + 16 u1 + 17 * 0x4B000000, and 17 * 0x4B000000 =
            // 0xFB000000 mod 2^32: adding 0x05000000 leaves u0 + 16 u1 < 2^28
            const uint32_t a01 = w[0] + (w[1] << 4) + 0x05000000u, a23 = w[2] + (w[3] << 4) + 0x05000000u;
            const uint32_t a45 = w[4] + (w[5] << 4) + 0x05000000u, a67 = w[6] + (w[7] << 4) + 0x05000000u;
            const uint64_t sv = (uint64_t)a01 + ((uint64_t)a23 << 8) + ((uint64_t)a45 << 16) + ((uint64_t)a67 << 24);
            acc += (int64_t)sv - kOffL + (int64_t)bl[l4];  // and 2^p m_b from limb n on
            lim[l4] = (uint32_t)acc;
            acc >>= 32;
          }
          if (L0 >= n) {
            *reinterpret_cast<uint4*>(srow + (L0 - n)) = make_uint4(lim[0], lim[1], lim[2], lim[3]);
          } else {
#pragma unroll
            for (int l4 = 0; l4 < 4; ++l4) {
              const int L = L0 + l4;
              if (L == n - 32)
                l0 = lim[l4];
              else if (L < n - 1) {
                orv |= lim[l4];
                andv &= lim[l4];
              } else {
                ltop = lim[l4];
              }
            }
          }
        };
        uint32_t va[32], vb[32];
        tmem_ld32_async(tl, va);
#pragma unroll 1
        for (int ch = 0; ch < nch; ch += 2) {
          step(ch, va, vb);
          step(ch + 1, vb, va);
        }
        bw0 = bn0;
        bw1 = bn1;
      }
      if (!ok) break;
      const bool any1 = ((l0 >> 19) | orv) != 0u;
      const bool any0 = ((~l0 >> 19) | ~andv) != 0u;
      Meta& mt = meta[buf * M + r];
      mt.te = used ? ze + be : ZEXP;
      mt.ltop = ltop;
      mt.sticky = 1u;
      mt.ts = (int32_t)(zs ^ bs);
      mt.unsafe = (used && !(any1 && any0)) ? 1 : 0;
      __syncwarp();
      if (lane == 0) arrive(b_sfull + 8 * buf);
    }
    if (!ok) *eflag = 1;
  } else {
    // ================= subtraction: lane groups ===========================
    const int st = tid - 256;
    const Grp<G> gp;
    const int grp = st / G;
    uint32_t* scr = reinterpret_cast<uint32_t*>(sm + C::OFF_SCR) + grp * C::SW;
    int64_t it = 0;
    bool ok = true;
    for (int64_t q = q0; q < q1 && ok; ++q, ++it) {
      const int64_t i0 = a.row0 + (q / ncols) * M;
      const int64_t j = upd_col(a, q % ncols);
      const int64_t kj = a.brow * N + j;
      const int buf = (int)(it & 1);
      bool okw = wait_bar(b_sfull + 8 * buf, (uint32_t)((it >> 1) & 1)) && !*eflag;
      ok = __all_sync(FULL, okw);
      if (!ok) break;
      // a row's staged product and x_ij; with 16 limbs per lane the next row's
      // are loaded while this one is computed (registers allow it there)
      constexpr bool PREF = W <= 16;
      auto load_row = [&](const int rr, uint32_t(&f)[W], uint32_t(&x)[W], int8_t& xs_, int64_t& xe_) {
        const int64_t i = i0 + rr;
        const int64_t ij = (i < rend ? i : i0) * N + j;
        load_slice_cg<W>(slab + ((size_t)(blockIdx.x * 2 + buf) * M + rr) * n + gp.g * W, f);
        load_slice<W>(X.m + ij * n + gp.g * W, x);
        xs_ = X.s[ij];
        xe_ = X.e[ij];
      };
      uint32_t F[W], Xv[W];
      int8_t xs = 0;
      int64_t xe = 0;
      if constexpr (PREF) load_row(grp, F, Xv, xs, xe);
      for (int rr = grp; rr < M; rr += C::NGRP) {
        if constexpr (!PREF) load_row(rr, F, Xv, xs, xe);
        const int64_t i = i0 + rr;
        const bool active = i < rend;
        const bool more = rr + C::NGRP < M;  // the same for every group of the warp
        uint32_t Fn[PREF ? W : 1], Xn[PREF ? W : 1];
        int8_t xsn = 0;
        int64_t xen = 0;
        if constexpr (PREF) {
          if (more) load_row(rr + C::NGRP, Fn, Xn, xsn, xen);
        }
        const Meta mt = meta[buf * M + rr];
        const bool used = mt.te != ZEXP;
        uint32_t Mr[W];
        int adj = round_product<W, G>(gp, F, mt.ltop, mt.sticky, Mr, 0);
        const bool unsafe = active && used && mt.unsafe != 0;
        if (__any_sync(FULL, unsafe)) {  // exact product by the IMAD engine
          uint32_t Bk[W], Mu[W];
          load_slice<W>(X.m + kj * n + gp.g * W, Bk);
          const int adju = mul_round<W, G>(gp, Bk, Z.m + (active ? i : i0) * n, Mu, 0);
          if (unsafe) {
#pragma unroll
            for (int w = 0; w < W; ++w) Mr[w] = Mu[w];
            adj = adju;
          }
        }
        if (!used) {
#pragma unroll
          for (int w = 0; w < W; ++w) Mr[w] = 0u;
        }
        const int64_t ij = (active ? i : i0) * N + j;
        const int64_t te = used ? mt.te + adj : ZEXP;
        sub_round<W, G>(gp, p, xs, xe, Xv, used ? (int8_t)mt.ts : (int8_t)0, te, Mr, scr, 0);
        if (active) {
          store_slice<W>(X.m + ij * n + gp.g * W, Xv);
          if (gp.g == 0) {
            X.s[ij] = xs;
            X.e[ij] = xe;
          }
        }
        if constexpr (PREF) {
          if (more) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
              F[w] = Fn[w];
              Xv[w] = Xn[w];
            }
            xs = xsn;
            xe = xen;
          }
        }
      }
      __syncwarp();
      if (lane == 0) arrive(b_sfree + 8 * buf);
    }
    if (!ok) *eflag = 1;
  }
  if (tid == 0 && *eflag) atomicExch(status, 5);  // MPDET_ETIMEOUT
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace tcl

// cuTensorMapEncodeTiled through the runtime's entry-point query.
typedef CUresult (*EncodeTiledFnL)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFnL encode_tiled_l() {
  static const EncodeTiledFnL fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFnL>(f);
  }();
  return fn;
}

bool tcl_supports(int p) { return p == 4096 || p == 8192 || p == 16384 || p == 32768; }

size_t tcl_zd_bytes(int64_t N, int p) { return (size_t)N * (size_t)(p / 8) * 2; }
size_t tcl_slab_bytes(int nsm, int p) { return (size_t)nsm * 2 * tcl::M * (size_t)(p / 32) * 4; }

template <int n>
static cudaError_t launch_tcl(MpArr X, const UpdArgs& a, MpArr Z, int* status, int p, int nsm, cudaStream_t st,
                              void* zd, uint32_t* slab) {
  using C = tcl::Cfg<n>;
  // A operand of this launch's rows
  {
    const int64_t blocks = (a.nrows + 127) / 128;
    tcl::k_zdig<n><<<(unsigned)blocks, 128, 0, st>>>(Z, a.N, a.row0, a.nrows, reinterpret_cast<uint4*>(zd));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const EncodeTiledFnL enc = encode_tiled_l();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tm;
  // Zd[i][k']: KD digits per row; a box is 64 digits (128 bytes) x 128 rows,
  // written with the 128-byte swizzle the A descriptor names
  const cuuint64_t dims[2] = {(cuuint64_t)C::KD, (cuuint64_t)a.N};
  const cuuint64_t strides[1] = {(cuuint64_t)C::KD * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)tcl::M};
  const cuuint32_t es[2] = {1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, zd, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int64_t items = (a.nrows + tcl::M - 1) / tcl::M * a.ncols;
  const int64_t grid = items < nsm ? items : nsm;
  cudaError_t e = cudaFuncSetAttribute(tcl::k_update_tcl<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  tcl::k_update_tcl<n><<<(unsigned)grid, tcl::NTH, C::SMEM, st>>>(X, a, Z, status, p, slab, tm);
  return cudaGetLastError();
}

// Rank-1 update on the large-precision tensor engine.  zd: tcl_zd_bytes(N, p)
// bytes of device memory for the multipliers' digits; slab: tcl_slab_bytes(nsm,
// p) bytes for the staged products (one block per SM, at most nsm blocks).
cudaError_t update_tcl(MpArr X, const UpdArgs& a, MpArr Z, int* status, int p, int nsm, cudaStream_t st, void* zd,
                       uint32_t* slab) {
  if (a.nrows <= 0 || a.ncols <= 0) return cudaSuccess;
  switch (p) {
    case 4096: return launch_tcl<128>(X, a, Z, status, p, nsm, st, zd, slab);
    case 8192: return launch_tcl<256>(X, a, Z, status, p, nsm, st, zd, slab);
    case 16384: return launch_tcl<512>(X, a, Z, status, p, nsm, st, zd, slab);
    case 32768: return launch_tcl<1024>(X, a, Z, status, p, nsm, st, zd, slab);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mpd
