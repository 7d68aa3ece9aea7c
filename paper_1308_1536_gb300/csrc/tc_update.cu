// Tensor-core engine for the rank-1 update at p = 512, 1024, 2048 (n = 16, 32, 64 limbs).
//
// The exact 2p-bit product of two mantissas is a convolution of their 8-bit
// digits: c_r = sum_s z[s] * b[r - s], P = sum_r c_r 2^(8r).  Every c_r is a
// sum of at most 256 products of digits <= 255, so it is below 2^24 and exact
// in fp32; bf16 holds every digit exactly.  For a block of 128 rows i and one
// column j the c_r of all 128 products are one GEMM on the 5th-generation
// tensor cores: D[i][r] = sum_k A[i][k] * B[k][r] with A[i][k'] = z_i[255-k']
// (digits reversed along K) and B[k'][r] = b_j[r - 255 + k'], a Hankel matrix:
// its 8x8 core matrices depend only on (n-core + k-core), so 95 distinct cores
// (12 KB of shared memory) serve the whole 256 x 512 operand through one
// descriptor with equal leading and stride byte offsets.  D lives in tensor
// memory (4 tiles of 128 columns); each thread then owns one row, turns its
// 512 exact column sums into the 128-limb product with a running carry,
// rounds it to p bits (round to nearest even) and leaves it in shared memory,
// where the lane groups of the IMAD engine subtract it from x_ij with the same
// sub_round.  Results are bit-identical to the IMAD engine.
//
// tcgen05 use: one thread issues the MMAs (kind::f16, bf16 inputs, fp32
// accumulate, M = 128, N = 128, K = 16), tcgen05.commit signals an mbarrier
// per tile; every wait is bounded and reports MPDET_ETIMEOUT through the
// status word; the block always frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace mpd {
namespace tc {

constexpr int n = 64;      // limbs per number
constexpr int KD = 256;    // 8-bit digits per mantissa
constexpr int M = 128;     // rows per block (MMA M)
constexpr int NT = 128;    // output positions per tile (MMA N)
constexpr int TILES = 4;   // 512 output positions
constexpr int NCORE = 95;  // Hankel cores
constexpr int W = 16, G = 4;
constexpr int SW = Scratch<W, G>::words;
constexpr int RSTR = 68;   // words per staged row (16-byte aligned; 8 rows hit distinct bank quads)

// shared memory layout (bytes)
constexpr int OFF_A = 0;                        // 128 x 256 bf16 = 64 KB
constexpr int OFF_H = OFF_A + M * KD * 2;       // Hankel cores, 95 x 128 B
constexpr int OFF_T = OFF_H + 12288;            // rounded products, 128 x 68 words
constexpr int OFF_X = OFF_T + M * RSTR * 4;     // x_ij rows of the column, 128 x 68 words
constexpr int OFF_B = OFF_X + M * RSTR * 4;     // b_j limbs, 64 words
constexpr int OFF_TE = OFF_B + 256;             // 128 int64 exponents of t
constexpr int OFF_XE = OFF_TE + M * 8;          // 128 int64 exponents of x
constexpr int OFF_TS = OFF_XE + M * 8;          // 128 int8 signs of t, 128 multiplier flags
constexpr int OFF_XS = OFF_TS + 256;            // 128 int8 signs of x
constexpr int OFF_SCR = OFF_XS + 128;           // 32 groups x SW words
constexpr int OFF_BAR = OFF_SCR + 32 * SW * 4;  // mbarriers + tmem slot
constexpr int SMEM = OFF_BAR + 128;

__device__ __forceinline__ void cp16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g));
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  // no swizzle, K-major: LBO steps between core matrices along K, SBO along M/N
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool bar_wait(uint32_t addr, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(addr), "r"(phase));
  return done != 0;
}

// 32 columns of this warp's 32 lanes, without waiting: the registers are
// valid after tmem_wait(v).
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
// Wait for this thread's tensor-memory loads; v is named so that no use of
// it moves above the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
                 "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]),
                 "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]),
                 "+r"(v[30]), "+r"(v[31]));
}

// 8 columns of this warp's 32 lanes, waited for.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]));
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
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// bf16 of a digit 0..255 (exact): the bit pattern of (float)d >> 16
__device__ __forceinline__ uint16_t dbf(uint32_t d) { return (uint16_t)(__float_as_uint((float)d) >> 16); }

__global__ void __launch_bounds__(128, 1) k_update_tc(MpArr X, UpdArgs a, MpArr Z, int* status, int p, int col_chunk) {
  extern __shared__ __align__(1024) unsigned char sm[];
  if (upd_stopped(status, a)) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* sA = sm + OFF_A;
  unsigned char* sH = sm + OFF_H;
  uint32_t* sT = reinterpret_cast<uint32_t*>(sm + OFF_T);
  uint32_t* sX = reinterpret_cast<uint32_t*>(sm + OFF_X);
  uint32_t* sB = reinterpret_cast<uint32_t*>(sm + OFF_B);
  int64_t* sTe = reinterpret_cast<int64_t*>(sm + OFF_TE);
  int64_t* sXe = reinterpret_cast<int64_t*>(sm + OFF_XE);
  int8_t* sTs = reinterpret_cast<int8_t*>(sm + OFF_TS);
  int8_t* sXs = reinterpret_cast<int8_t*>(sm + OFF_XS);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);  // 4 tile barriers
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_BAR + 64);
  const int64_t N = a.N;
  const int64_t ncols = a.ncols;
  const int64_t i0 = a.row0 + (int64_t)blockIdx.y * M;
  const int64_t rend = a.row0 + a.nrows;
  const int64_t c0 = (int64_t)blockIdx.x * col_chunk;
  const int64_t c1 = (c0 + col_chunk < ncols) ? c0 + col_chunk : ncols;

  // ---- A: digits of the 128 multipliers, K reversed (k' = 255 - s) --------
  // core (k-core c, row-group g) at c*128 + g*4096, row r of the core at +16r
  {
    const int64_t i = i0 + tid;  // one row per thread
    const bool have = i < rend && Z.e[i < rend ? i : i0] != ZEXP;
    const uint32_t* zm = Z.m + (i < rend ? i : i0) * n;
    unsigned char* rowbase = sA + (tid >> 3) * 4096 + (tid & 7) * 16;
    for (int c = 0; c < 32; ++c) {
      // digits s = 255-8c .. 248-8c are bytes of limbs 63-2c (high 4) and 62-2c (low 4), reversed
      uint32_t hi = have ? zm[63 - 2 * c] : 0u, lo = have ? zm[62 - 2 * c] : 0u;
      uint32_t w0 = dbf(hi >> 24) | ((uint32_t)dbf((hi >> 16) & 255) << 16);
      uint32_t w1 = dbf((hi >> 8) & 255) | ((uint32_t)dbf(hi & 255) << 16);
      uint32_t w2 = dbf(lo >> 24) | ((uint32_t)dbf((lo >> 16) & 255) << 16);
      uint32_t w3 = dbf((lo >> 8) & 255) | ((uint32_t)dbf(lo & 255) << 16);
      *reinterpret_cast<uint4*>(rowbase + c * 128) = make_uint4(w0, w1, w2, w3);
    }
    sTs[M + tid] = have ? 1 : 0;  // multiplier present (non-zero, row in range)
  }
  if (tid == 0)
    for (int t = 0; t < TILES; ++t) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bars[t])));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
  Grp<G> gp;
  const int gid = tid / G;  // 32 groups
  uint32_t* scr = reinterpret_cast<uint32_t*>(sm + OFF_SCR) + gid * SW;
  const int8_t zsign = (i0 + tid < rend) ? Z.s[i0 + tid] : 0;
  const int64_t zexp = (i0 + tid < rend) ? Z.e[i0 + tid] : ZEXP;
  uint32_t phase = 0;
  bool ok = true;

  for (int64_t c = c0; c < c1 && ok; ++c) {
    const int64_t j = upd_col(a, c);
    const int64_t kj = a.brow * N + j;
    const int64_t be = X.e[kj];
    const int8_t bs = X.s[kj];
    // ---- stage b_j and the 128 x_ij of this column (cp.async) ---------------
    if (tid < 16) cp16(su32(sB) + 16 * tid, X.m + kj * n + 4 * tid);
    asm volatile("cp.async.commit_group;");
    {
      const int64_t i = i0 + tid;
      const int64_t ij = (i < rend ? i : i0) * N + j;
      sXs[tid] = X.s[ij];
      sXe[tid] = X.e[ij];
#pragma unroll
      for (int q = 0; q < 16; ++q) cp16(su32(sX + tid * RSTR) + 16 * q, X.m + ij * n + 4 * q);
    }
    asm volatile("cp.async.commit_group;");
    asm volatile("cp.async.wait_group 1;");  // b_j has landed (x_ij may still be in flight)
    __syncthreads();
    // ---- Hankel cores of b_j: H_d[nn][kk] = b[8d + nn + kk - 255] ----------
    {
      const unsigned char* bb = reinterpret_cast<const unsigned char*>(sB);  // little-endian digits
      for (int q = tid; q < NCORE * 8; q += 128) {  // one core row (8 bf16) per item
        const int d = q >> 3, nn = q & 7;
        const int base = 8 * d + nn - 255;  // digit index of kk = 0
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t h2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int idx = base + 2 * e + u;
            const uint32_t dg = (idx >= 0 && idx < KD && be != ZEXP) ? bb[idx] : 0u;
            h2[u] = dbf(dg);
          }
          w[e] = h2[0] | (h2[1] << 16);
        }
        *reinterpret_cast<uint4*>(sH + d * 128 + nn * 16) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // ---- MMAs: 4 tiles x 16 K-steps ----------------------------------------
    if (tid == 0) {
      for (int t = 0; t < TILES; ++t) {
        for (int ks = 0; ks < KD / 16; ++ks) {
          const uint64_t ad = desc(su32(sA) + ks * 256, 128, 4096);
          const uint64_t bd = desc(su32(sH) + (16 * t + 2 * ks) * 128, 128, 128);
          const uint32_t acc = ks > 0 ? 1u : 0u;
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                           tmem + (uint32_t)(t * NT)),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bars[t])));
      }
    }
    // ---- epilogue: thread = row; column sums -> 128 limbs -> RN to p bits --
    uint32_t up[64];  // limbs 64..127
    uint32_t l63 = 0, sticky = 0;
    uint64_t acc = 0;
    bool okc = true;
#pragma unroll
    for (int t = 0; t < TILES; ++t) {
      if (okc && !bar_wait(su32(&bars[t]), phase)) okc = false;
      okc = __all_sync(0xffffffffu, okc);  // warp-uniform: tcgen05.ld is warp-collective
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (okc) {
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {  // 32 columns = 8 limbs per chunk
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * NT + ch * 32), v);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint64_t c0v = __float2uint_rz(__uint_as_float(v[4 * q]));
            const uint64_t c1v = __float2uint_rz(__uint_as_float(v[4 * q + 1]));
            const uint64_t c2v = __float2uint_rz(__uint_as_float(v[4 * q + 2]));
            const uint64_t c3v = __float2uint_rz(__uint_as_float(v[4 * q + 3]));
            acc += c0v + (c1v << 8) + (c2v << 16) + (c3v << 24);
            const uint32_t limb = (uint32_t)acc;
            acc >>= 32;
            const int L = t * 32 + ch * 8 + q;
            if (L >= 64) up[L >= 64 ? L - 64 : 0] = limb;
            else if (L == 63) l63 = limb;
            else sticky |= limb;
          }
        }
      }
    }
    ok = __syncthreads_and(okc) != 0;
    if (!ok) break;
    // round (same rule as mul_round): product has 2p or 2p-1 bits
    {
      const uint32_t top = up[63] >> 31;
      uint32_t rbit, st;
      if (top) {
        rbit = l63 >> 31;
        st = (l63 & 0x7fffffffu) | sticky;
      } else {
#pragma unroll
        for (int q = 63; q > 0; --q) up[q] = (up[q] << 1) | (up[q - 1] >> 31);
        up[0] = (up[0] << 1) | (l63 >> 31);
        rbit = (l63 >> 30) & 1u;
        st = (l63 & 0x3fffffffu) | sticky;
      }
      uint32_t inc = rbit & ((st != 0u) | (up[0] & 1u));
      uint32_t carry = inc;
#pragma unroll
      for (int q = 0; q < 64; ++q) {
        const uint64_t s = (uint64_t)up[q] + carry;
        up[q] = (uint32_t)s;
        carry = (uint32_t)(s >> 32);
      }
      int adj = top ? 0 : -1;
      if (carry) {
        up[63] = 0x80000000u;
        adj += 1;
      }
      const bool tz = !sTs[M + tid] || be == ZEXP;
#pragma unroll
      for (int q = 0; q < 64; q += 4)
        *reinterpret_cast<uint4*>(sT + tid * RSTR + q) =
            tz ? make_uint4(0u, 0u, 0u, 0u) : make_uint4(up[q], up[q + 1], up[q + 2], up[q + 3]);
      sTe[tid] = tz ? ZEXP : zexp + be + adj;
      sTs[tid] = tz ? (int8_t)0 : (int8_t)(zsign ^ bs);
    }
    asm volatile("cp.async.wait_group 0;");  // x_ij rows have landed
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    // ---- x_ij = RN(x_ij - t_i) by lane groups (4 rows per group) ------------
#pragma unroll 1
    for (int rr = 0; rr < 4; ++rr) {
      const int r = gid + 32 * rr;
      const int64_t i = i0 + r;
      const bool active = i < rend;
      const int64_t ij = (active ? i : i0) * N + j;
      uint32_t Xv[W], T[W];
      load_slice<W>(sX + r * RSTR + gp.g * W, Xv);
      load_slice<W>(sT + r * RSTR + gp.g * W, T);
      int8_t xs = sXs[r];
      int64_t xe = sXe[r];
      sub_round<W, G>(gp, p, xs, xe, Xv, sTs[r], sTe[r], T, scr);
      if (active) {
        store_slice<W>(X.m + ij * n + gp.g * W, Xv);
        if (gp.g == 0) {
          X.s[ij] = xs;
          X.e[ij] = xe;
        }
      }
    }
    phase ^= 1u;
    __syncthreads();  // sT and sH are rewritten by the next column
  }
  if (!ok && tid == 0) atomicExch(status, 5);  // MPDET_ETIMEOUT
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}


// ---------------------------------------------------------------------------
// Row tiles.  The subtraction role's operands, x_ij of the next column and the
// staged product t, sit per warp of 32 rows in the layout a TMA copy with
// 128-byte swizzle writes: for NL >= 32 limbs [half of the row (128 bytes)]
// [row r of the warp][32 words], the 16-byte chunk c of each 128-byte line
// stored at chunk c ^ (r & 7); for NL = 16 [row][16 words] with 64-byte
// swizzle, chunk c at c ^ ((r >> 1) & 3).  Eight consecutive rows then hit
// eight different bank quads, so one thread per row reads or writes its row
// 16 bytes at a time without bank conflicts.  Tiles are 1024-byte aligned.
// ---------------------------------------------------------------------------
template <int NL>
struct RowT {
  static constexpr int TILE = 32 * NL * 4;  // bytes per warp tile
  unsigned char* tile;
  uint32_t r;  // row within the warp, 0..31
  __device__ __forceinline__ uint32_t off(int kk) const {  // byte offset of the row's 16-byte chunk kk
    if constexpr (NL >= 32)
      return (uint32_t)(kk >> 3) * 4096u + r * 128u + ((((uint32_t)kk & 7u) ^ (r & 7u)) << 4);
    else
      return r * 64u + ((((uint32_t)kk) ^ ((r >> 1) & 3u)) << 4);
  }
  __device__ __forceinline__ uint4 ld16(int kk) const { return *reinterpret_cast<const uint4*>(tile + off(kk)); }
  __device__ __forceinline__ void st16(int kk, uint4 v) const { *reinterpret_cast<uint4*>(tile + off(kk)) = v; }
  __device__ __forceinline__ uint32_t ld32(int i) const {
    return *reinterpret_cast<const uint32_t*>(tile + off(i >> 2) + ((uint32_t)(i & 3) << 2));
  }
};

// Round a staged exact product to p = 32 NL bits in place: T holds its upper NL
// limbs, l63 its limb NL - 1 and sticky the OR of the limbs below.  The product
// of two normalised mantissas has 2p or 2p - 1 bits; returns the exponent
// adjustment (-1, 0 or +1) as mul_round does.
template <int NL>
__device__ __forceinline__ int round_product(const RowT<NL>& T, uint32_t l63, uint32_t sticky) {
  uint32_t up[NL];
#pragma unroll
  for (int q = 0; q < NL; q += 4) {
    const uint4 v = T.ld16(q >> 2);
    up[q] = v.x;
    up[q + 1] = v.y;
    up[q + 2] = v.z;
    up[q + 3] = v.w;
  }
  const uint32_t top = up[NL - 1] >> 31;
  const uint32_t sft = 1u - top;  // a 2p - 1 bit product moves up one bit (no branch: lanes differ)
#pragma unroll
  for (int q = NL - 1; q > 0; --q) up[q] = __funnelshift_l(up[q - 1], up[q], sft);
  up[0] = __funnelshift_l(l63, up[0], sft);
  const uint32_t rbit = (l63 >> (31u - sft)) & 1u;
  const uint32_t st = (l63 & (0x7fffffffu >> sft)) | sticky;
  const uint32_t inc = rbit & ((st != 0u) | (up[0] & 1u));
  up[0] = add_cc(up[0], inc);
#pragma unroll
  for (int q = 1; q < NL; ++q) up[q] = addc_cc(up[q], 0u);
  const uint32_t ovf = addc(0u, 0u);
  if (ovf) up[NL - 1] = 0x80000000u;
#pragma unroll
  for (int q = 0; q < NL; q += 4) T.st16(q >> 2, make_uint4(up[q], up[q + 1], up[q + 2], up[q + 3]));
  return (top ? 0 : -1) + (int)ovf;
}

template <int NL>
__device__ __forceinline__ void copy_row(const RowT<NL>& src, uint32_t* out) {
#pragma unroll
  for (int q = 0; q < NL; q += 4) *reinterpret_cast<uint4*>(out + q) = src.ld16(q >> 2);
}

// The row of src into the row of out (nothing to do when they are the same).
template <int NL>
__device__ __forceinline__ void put_row(const RowT<NL>& src, const RowT<NL>& out) {
  if (src.tile == out.tile) return;
#pragma unroll
  for (int q = 0; q < NL; q += 4) out.st16(q >> 2, src.ld16(q >> 2));
}

// ---------------------------------------------------------------------------
// x_ij = RN(x_ij - t) for one row by one thread, the same rounding as
// sub_round: the larger magnitude A sits in a frame of NL + 2 limbs above two
// guard limbs, the smaller B is aligned into it (bits below the frame jammed
// into a sticky bit), then normalisation and round to nearest even.  No data
// crosses lanes.  sub_row handles the usual case in registers (exponent gap
// below 64, at most 32 bits cancelled) and hands the rest to
// sub_row_general, which recomputes from the unchanged operands with the
// frame in thread-local memory.
//   x, t: the row's x and t tiles;  out: the row's destination tile (t's
//   own: every read of an operand comes before the first write of the
//   result).  Returns the result's sign and exponent in rs, re.
// ---------------------------------------------------------------------------
template <int NL>
__device__ __noinline__ void sub_row_general(RowT<NL> xr, int8_t xs, int64_t xe, RowT<NL> tr, int8_t ts, int64_t te,
                                             RowT<NL> out, int8_t* rs_, int64_t* re_) {
  constexpr int p = 32 * NL;
  if (te == ZEXP) {  // x - 0
    put_row<NL>(xr, out);
    *rs_ = xs;
    *re_ = xe;
    return;
  }
  const int8_t tsn = (int8_t)(ts ^ 1);
  if (xe == ZEXP) {  // 0 - t
    put_row<NL>(tr, out);
    *rs_ = tsn;
    *re_ = te;
    return;
  }
  int cmp = (xe != te) ? (xe > te ? 1 : -1) : 0;
  if (cmp == 0) {
    for (int i = NL - 1; i >= 0; --i) {
      const uint32_t a = xr.ld32(i), b = tr.ld32(i);
      if (a != b) {
        cmp = a > b ? 1 : -1;
        break;
      }
    }
  }
  const bool swap = cmp < 0;
  const RowT<NL> A = swap ? tr : xr;
  const RowT<NL> B = swap ? xr : tr;
  const int64_t eA = swap ? te : xe, eB = swap ? xe : te;
  const int8_t sA = swap ? tsn : xs, sB = swap ? xs : tsn;
  const bool eff_sub = (sA != sB);
  const int64_t dd = eA - eB;
  if (dd >= p + 2) {  // B below a quarter ulp of A
    put_row<NL>(A, out);
    *rs_ = sA;
    *re_ = eA;
    return;
  }
  const uint32_t inv = eff_sub ? 0xffffffffu : 0u;
  const int d = (int)dd;
  // frame F = A * 2^64 +- (B aligned): frame limb f holds bits
  // [32 (f - 2) + d, +32) of B; the bits of B below the frame (index d - 64)
  // are jammed into the lowest frame bit
  uint32_t F[NL + 3];
  {
    const int q = (d - 64) >> 5, r = (d - 64) & 31;  // frame limb f holds B bits from 32 (f + q) + r
    bool lost = false;
    for (int k = 0; k < q && k < NL; ++k) lost = lost || B.ld32(k) != 0u;
    if (q >= 0 && q < NL && r) lost = lost || (B.ld32(q) & ((1u << r) - 1u)) != 0u;
    uint32_t Y[NL + 2];
    for (int f = 0; f < NL + 2; ++f) {
      const int k = f + q;
      const uint32_t lo = (k >= 0 && k < NL) ? B.ld32(k) : 0u;
      const uint32_t hi = (k + 1 >= 0 && k + 1 < NL) ? B.ld32(k + 1) : 0u;
      Y[f] = __funnelshift_r(lo, hi, r);
    }
    Y[0] |= lost ? 1u : 0u;
    F[0] = add_cc(Y[0] ^ inv, eff_sub ? 1u : 0u);
    F[1] = addc_cc(Y[1] ^ inv, 0u);
#pragma unroll
    for (int k = 0; k < NL; ++k) F[k + 2] = addc_cc(A.ld32(k), Y[k + 2] ^ inv);
    F[NL + 2] = addc(0u, 0u);
    if (eff_sub) F[NL + 2] = 0u;  // the carry out of A*2^64 + ~Y + 1
  }
  int topbit = -1;
  for (int k = NL + 2; k >= 0 && topbit < 0; --k)
    if (F[k]) topbit = 32 * k + 31 - __clz(F[k]);
  if (topbit < 0) {  // exact cancellation
#pragma unroll
    for (int q = 0; q < NL; q += 4) out.st16(q >> 2, make_uint4(0u, 0u, 0u, 0u));
    *rs_ = 0;
    *re_ = ZEXP;
    return;
  }
  const int sh = topbit - (p - 1);
  uint32_t M[NL];
  for (int l = 0; l < NL; ++l) M[l] = funnel(F, 32 * l + sh, NL + 3);
  const uint32_t rbit = (sh >= 1) ? (funnel(F, sh - 1, NL + 3) & 1u) : 0u;
  bool stl = false;
  if (sh >= 2) {
    const int cut = sh - 1;  // bits [0, cut)
    for (int k = 0; 32 * k < cut; ++k) {
      const uint32_t m = (cut >= 32 * k + 32) ? 0xffffffffu : ((1u << (cut - 32 * k)) - 1u);
      stl = stl || (F[k] & m) != 0u;
    }
  }
  const uint32_t inc = rbit & ((stl ? 1u : 0u) | (M[0] & 1u));
  M[0] = add_cc(M[0], inc);
#pragma unroll
  for (int l = 1; l < NL; ++l) M[l] = addc_cc(M[l], 0u);
  const uint32_t ovf = addc(0u, 0u);
  if (ovf) M[NL - 1] = 0x80000000u;  // every limb wrapped to 0
#pragma unroll
  for (int q = 0; q < NL; q += 4) out.st16(q >> 2, make_uint4(M[q], M[q + 1], M[q + 2], M[q + 3]));
  *rs_ = sA;
  *re_ = (int64_t)topbit + 1 + eA - p - 64 + (int64_t)ovf;
}

template <int NL>
__device__ __forceinline__ void sub_row(const RowT<NL>& xr, int8_t xs, int64_t xe, const RowT<NL>& tr, int8_t ts,
                                        int64_t te, const RowT<NL>& out, int8_t& rs, int64_t& re) {
  constexpr int p = 32 * NL;
  const int8_t tsn = (int8_t)(ts ^ 1);
  const bool tzero = te == ZEXP, xzero = xe == ZEXP;
  int cmp = (xe != te) ? (xe > te ? 1 : -1) : 0;
  if (!tzero && !xzero && cmp == 0) {
    for (int i = NL - 1; i >= 0; --i) {
      const uint32_t a = xr.ld32(i), b = tr.ld32(i);
      if (a != b) {
        cmp = a > b ? 1 : -1;
        break;
      }
    }
  }
  const bool swap = cmp < 0;
  const int64_t dd = swap ? te - xe : xe - te;
  if (tzero || xzero || dd >= p + 2) {  // x - 0, 0 - t, or the smaller below a quarter ulp of the larger
    const bool keep_x = tzero || (!xzero && !swap);
    put_row<NL>(keep_x ? xr : tr, out);
    rs = keep_x ? xs : tsn;
    re = keep_x ? xe : te;
    return;
  }
  if (dd >= 64) {
    sub_row_general<NL>(xr, xs, xe, tr, ts, te, out, &rs, &re);
    return;
  }
  const RowT<NL> A = swap ? tr : xr;
  const RowT<NL> B = swap ? xr : tr;
  const int64_t eA = swap ? te : xe;
  const int8_t sA = swap ? tsn : xs, sB = swap ? xs : tsn;
  const bool eff_sub = (sA != sB);
  const uint32_t inv = eff_sub ? 0xffffffffu : 0u;
  const int d = (int)dd;
  const int q = d >> 5, r = d & 31;
  uint32_t F[NL + 2];
  {
    uint32_t Bv[NL];
#pragma unroll
    for (int k = 0; k < NL; k += 4) {
      const uint4 v = B.ld16(k >> 2);
      Bv[k] = v.x;
      Bv[k + 1] = v.y;
      Bv[k + 2] = v.z;
      Bv[k + 3] = v.w;
    }
    // bits [32 (f - 2) + d, +32) of B: limb f - 2 + q shifted right by r with
    // the next one; Bq[i] = limb i - 2 + q of B (zero outside 0..NL-1)
    uint32_t Bq[NL + 3];
#pragma unroll
    for (int i = 0; i < NL + 3; ++i) {
      const uint32_t lo = (i - 2 >= 0 && i - 2 < NL) ? Bv[i - 2 >= 0 && i - 2 < NL ? i - 2 : 0] : 0u;
      const uint32_t hi = (i - 1 >= 0 && i - 1 < NL) ? Bv[i - 1 >= 0 && i - 1 < NL ? i - 1 : 0] : 0u;
      Bq[i] = q ? hi : lo;
    }
    uint32_t Y[NL + 2];
#pragma unroll
    for (int f = 0; f < NL + 2; ++f) Y[f] = __funnelshift_r(Bq[f], Bq[f + 1], r);
    F[0] = add_cc(Y[0] ^ inv, eff_sub ? 1u : 0u);
    F[1] = addc_cc(Y[1] ^ inv, 0u);
#pragma unroll
    for (int k = 0; k < NL; k += 4) {
      const uint4 a = A.ld16(k >> 2);
      F[k + 2] = addc_cc(a.x, Y[k + 2] ^ inv);
      F[k + 3] = addc_cc(a.y, Y[k + 3] ^ inv);
      F[k + 4] = addc_cc(a.z, Y[k + 4] ^ inv);
      F[k + 5] = addc_cc(a.w, Y[k + 5] ^ inv);
    }
  }
  uint32_t sx = addc(0u, 0u);
  if (eff_sub) sx = 0u;  // the carry out of A*2^64 + ~Y + 1
  int topbit = -1;
  if (sx) topbit = 32 * (NL + 2);
  else if (F[NL + 1]) topbit = 32 * (NL + 1) + 31 - __clz(F[NL + 1]);
  else if (F[NL]) topbit = 32 * NL + 31 - __clz(F[NL]);
  const int sh = topbit - (p - 1);
  if (topbit < 0 || sh < 32) {  // more than 32 bits cancelled
    sub_row_general<NL>(xr, xs, xe, tr, ts, te, out, &rs, &re);
    return;
  }
  // sh in [32, 65]: output limb l = frame bits [32 l + sh, +32), i.e. frame
  // limb l + q2 shifted right by r2 with the next one (limb NL + 2 is sx)
  const int q2 = sh >> 5, r2 = sh & 31;
  uint32_t Fq[NL + 1];
#pragma unroll
  for (int i = 0; i < NL + 1; ++i) {
    const uint32_t f3 = (i + 2 < NL + 2) ? F[i + 2 < NL + 2 ? i + 2 : 0] : sx;
    Fq[i] = (q2 == 1) ? F[i + 1] : f3;
  }
  uint32_t M[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) M[l] = __funnelshift_r(Fq[l], Fq[l + 1], r2);
  const uint64_t g64 = ((uint64_t)F[1] << 32) | F[0];
  const int rb = sh - 1;  // 31..64
  const uint32_t rbit = (rb < 64) ? (uint32_t)((g64 >> rb) & 1ull) : (F[2] & 1u);
  const uint32_t st = (rb < 64) ? (uint32_t)((g64 & ((1ull << rb) - 1ull)) != 0ull) : (uint32_t)(g64 != 0ull);
  const uint32_t inc = rbit & (st | (M[0] & 1u));
  M[0] = add_cc(M[0], inc);
#pragma unroll
  for (int l = 1; l < NL; ++l) M[l] = addc_cc(M[l], 0u);
  const uint32_t ovf = addc(0u, 0u);
  if (ovf) M[NL - 1] = 0x80000000u;  // every limb wrapped to 0
#pragma unroll
  for (int k = 0; k < NL; k += 4) out.st16(k >> 2, make_uint4(M[k], M[k + 1], M[k + 2], M[k + 3]));
  rs = sA;
  re = (int64_t)topbit + 1 + eA - p - 64 + (int64_t)ovf;
}

// ---------------------------------------------------------------------------
// Pipelined version: 12 warps in three roles so that the tensor core, the
// epilogue and the subtraction of consecutive columns overlap.
//   warps 0-3  (E): one thread per row; drain the four tensor-memory tiles of
//                   a column, form and round the product, stage it (2 buffers)
//   warps 4-7  (S): lane groups subtract the staged products from x_ij
//   warps 8-11 (P): build the Hankel cores of the next column (2 buffers);
//                   thread 256 issues the MMAs of each tile as soon as the
//                   epilogue has released that tile
// mbarriers: full[t] (MMA -> E), empty[t] (E -> MMA), hfree[b] (MMA -> P),
// tfull[b] (E -> S), tfree[b] (S -> E).  For a barrier that completes once
// per use, the parity awaited at its u-th completion is u & 1.  Every wait
// is bounded; a timeout sets MPDET_ETIMEOUT and all roles drain.
// ---------------------------------------------------------------------------
namespace pipe {
constexpr int NTH = 384;
constexpr int LIMIT = 1 << 22;

// Balanced digits.  The warp-specialised kernel writes both mantissas in
// digits e in [-128, 127] (e_s = d_s + c_s - 256 c_{s+1}, c_{s+1} = 1 when
// d_s + c_s >= 128); a normalised mantissa m then equals sum_s e_s 256^s +
// 256^KD.  With m' = m - 2^p for the multiplier z and b~ = b's balanced
// digits followed by the carry digit 1 at position KD (the value b itself),
//     z * b = z' * b~ + 2^p * b,
// the first term a digit convolution of KD + 1 positions per output, the
// second one more MMA K step per upper tile: a column of ones in A times b's
// raw digits d_j at output position KD + j.  Every column sum lies
// in [-4161536, 4194559]: at most 256 products in [-16256, 16384], or 255 of
// them and one with the carry digit when that digit is in the window, plus a
// raw digit of b (0..255) above position KD.  Adding
// kMagic puts it in [2^23, 2^24), where the fp32 spacing is 1, so the fp32
// result's bits are 0x4B000000 + u with u = sum + kMagic - 2^23 (kOff) in
// [0, 2^23): one FADD instead of a conversion on the XU pipe.  Four
// consecutive outputs w0..w3 (raw bits) form a limb as
//     (w0 + (w1 << 8)) + (w2 + (w3 << 8)) * 2^16        (32-bit inner sums)
// where w << 8 drops the exponent field mod 2^32 and neither inner sum wraps
// (u < 2^23), so the limb is sum_q u_q 2^(8q) + 0x4B000000 * 0x10001 and,
// less kOff * 0x01010101, the four sums' weighted total: kC removes both.
constexpr float kMagic = 12566528.0f;  // 2^23 + kOff
// The upper tiles (positions >= KD) receive kMagic from the MMA itself: the
// extra K step has ones in A's columns KD + 1 and KD + 2 and the bf16
// constants 2^23 and kOff = 255 * 2^14 (both exact) in B's rows 1 and 2.
// The extra K step is issued last, so the partial sums before it are below
// 2^23 in magnitude and the final one lies in [2^23, 2^24): all are exact
// fp32 integers, the accumulator holds the exact biased sum and the epilogue
// reads its bits without the FADD.
constexpr uint32_t kBias23 = 0x4B00u;   // bf16 2^23
constexpr uint32_t kBiasOff = 0x4A7Fu;  // bf16 4177920 = kOff
constexpr uint32_t kOff = 4177920u;
constexpr int64_t kC = 152833374535680ll;  // kOff * 0x01010101 + 0x4B000000 * 0x10001
static_assert((int64_t)kOff * 0x01010101ll + 0x4B000000ll * 0x10001ll == kC, "per-limb constant");

// bf16 bits of a small integer (|e| <= 256: exact)
__device__ __forceinline__ uint32_t dbfs(int e) { return __float_as_uint((float)e) >> 16; }

// Geometry for mantissas of KD 8-bit digits (NL = KD/4 limbs; p = 8 KD).
template <int KD_>
struct Cfg {
  static constexpr int KD = KD_;
  static constexpr int NL = KD / 4;                 // limbs
  static constexpr int TILES = 2 * KD / 128;        // 128-column tensor-memory tiles (2 KD positions)
  // Tensor-memory buffers: two where a column's tiles fill at most half of
  // the 512 columns (p = 512, 1024), so that the MMAs of column c + 1 run
  // while the epilogue drains column c; column c uses buffer c % TB, whose
  // tiles and full/empty barriers are slots (c % TB) TILES + t.
  static constexpr int TB = TILES <= 2 ? 2 : 1;
  static constexpr int TCOLS = TB * TILES * 128;    // allocated columns (a power of two >= 32)
  static constexpr int NCORE = 16 * TILES + KD / 8 - 1;  // Hankel cores
  static constexpr int HBYTES = (NCORE * 128 + 1023) / 1024 * 1024;
  static constexpr int TILE = RowT<NL>::TILE;       // bytes per 32-row tile (swizzled rows)
  // Output tile t (positions [128 t, 128 t + 128)) receives products only
  // from reversed K positions k' in [KD - 128 (t + 1), 2 KD - 1 - 128 t]
  // (b~ has digits 0..KD): the K steps outside are all-zero Hankel corners and
  // are not issued.  Neighbouring tiles with the same K range form one
  // M = 128, N = 256 MMA (half the operand reads per product of two N = 128).
  __host__ __device__ static constexpr int ks_lo(int t) { return (KD - 128 * (t + 1)) > 0 ? (KD - 128 * (t + 1)) / 16 : 0; }
  __host__ __device__ static constexpr int ks_hi(int t) { return (2 * KD - 128 * t) < KD ? (2 * KD - 128 * t) / 16 : KD / 16; }
  __host__ __device__ static constexpr bool merge(int t) {  // tile t and t + 1 in one MMA group
    return t + 1 < TILES && ks_lo(t) == ks_lo(t + 1) && ks_hi(t) == ks_hi(t + 1);
  }
  // A holds KA = KD + 16 digits per row: z's KD balanced digits (K reversed)
  // and one K step whose first position is 1, which multiplies b's raw
  // digits in the BX region (the 2^p * b term, one extra MMA per upper tile)
  static constexpr int KA = KD + 16;
  static constexpr int XT0 = KD / 128;                      // first tile holding positions >= KD
  static constexpr int XTN = TILES - XT0;                   // tiles with the extra MMA
  static constexpr int XBYTES = XTN * 16 * 256;             // per buffer: 16 n-cores x 2 k-cores per tile
  static constexpr int OFF_A = 0;                           // M x KA bf16
  static constexpr int OFF_H = OFF_A + M * KA * 2;          // 2 Hankel buffers
  static constexpr int OFF_BX = OFF_H + 2 * HBYTES;         // 2 extra-K B buffers
  static constexpr int OFF_B = OFF_BX + 2 * XBYTES;         // 2 x NL limbs of b_j
  static constexpr int OFF_T = (OFF_B + 2 * NL * 4 + 1023) / 1024 * 1024;  // 2 x 4 tiles: staged products
  static constexpr int OFF_TA = OFF_T + 2 * 4 * TILE;       // 2 x M x 2 words: limb NL - 1 and sticky
  static constexpr int OFF_TE = OFF_TA + 2 * M * 8;          // 2 x M int64
  static constexpr int OFF_TS = OFF_TE + 2 * M * 8;         // 2 x M int8
  static constexpr int OFF_X = (OFF_TS + 2 * M + 1023) / 1024 * 1024;  // 4 tiles: x_ij of the current column
  static constexpr int OFF_EB = OFF_X + 4 * TILE;            // bf16 balanced digits of b, KD + 1 (+ pad)
  static constexpr int OFF_BAR = OFF_EB + (KD + 8) * 2;     // barriers
  static constexpr int SMEM = OFF_BAR + 256;
  static_assert(NL % 16 == 0 && NL <= 64, "tensor engine covers p = 512, 1024, 2048");
  static_assert(TB * TILES <= 4 && TCOLS <= 512, "four full/empty barrier slots, 512 tensor-memory columns");
  static_assert(OFF_X % 1024 == 0 && OFF_T % 1024 == 0 && OFF_BX % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ void arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar));
}
// barrier 1 over the 96 Hankel builder threads, returning the OR of q over them
__device__ __forceinline__ bool pbar_or(bool q) {
  uint32_t r;
  __syncwarp();
  asm volatile("{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.or.pred b, 1, 96, a;\n selp.u32 %0, 1, 0, b;\n}"
               : "=r"(r)
               : "r"((uint32_t)q));
  return r != 0;
}
__device__ __forceinline__ void pbar() {
  __syncwarp();
  asm volatile("bar.sync 1, 96;");
}
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < LIMIT && !done; ++it)
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity));
  return done != 0;
}
}  // namespace pipe

template <int KD>
__global__ void __launch_bounds__(pipe::NTH, 1) k_update_tcp(MpArr X, UpdArgs a, MpArr Z, int* status, int p,
                                                            int col_chunk, const __grid_constant__ CUtensorMap tmx0,
                                                            const __grid_constant__ CUtensorMap tmx1) {
  using pipe::arrive;
  using pipe::wait_bar;
  using C = pipe::Cfg<KD>;
  constexpr int NL = C::NL, TILES = C::TILES, TILE = C::TILE;
  extern __shared__ __align__(1024) unsigned char sm[];
  if (upd_stopped(status, a)) return;
  const int tid = threadIdx.x, warp = tid >> 5;
  // the swizzled x tiles need a 1024-byte aligned window: refuse (MPDET_ECUDA)
  // rather than copy with a layout the readers do not expect
  if (su32(sm) & 1023u) {
    if (tid == 0) atomicExch(status, 3);
    return;
  }
  unsigned char* sA = sm + C::OFF_A;
  uint32_t* sBl = reinterpret_cast<uint32_t*>(sm + C::OFF_B);
  unsigned char* const sT = sm + C::OFF_T;  // [buffer][warp] tiles of staged products
  uint32_t* const sTa = reinterpret_cast<uint32_t*>(sm + C::OFF_TA);  // [buffer][row]: limb NL - 1, sticky
  int64_t* sTe = reinterpret_cast<int64_t*>(sm + C::OFF_TE);
  int8_t* sTs = reinterpret_cast<int8_t*>(sm + C::OFF_TS);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::OFF_BAR);
  // bars: 0-3 full, 4-7 empty, 8-9 hfree, 10-11 tfull, 12-13 tfree; slot 14: tmem address; 15: error
  // flag; 16 aready (E -> I: the multipliers' digits are in A); 19-20 hready (B -> I: a column's
  // Hankel cores and extra-K digits are built); 21-24 xfull (one per subtraction warp: its rows'
  // x_ij have arrived)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(&bars[14]);
  volatile int* eflag = reinterpret_cast<volatile int*>(&bars[15]);
  const uint32_t b_full = su32(&bars[0]), b_empty = su32(&bars[4]), b_hfree = su32(&bars[8]);
  const uint32_t b_tfull = su32(&bars[10]), b_tfree = su32(&bars[12]), b_hready = su32(&bars[19]),
                 b_xfull = su32(&bars[21]), b_aready = su32(&bars[16]);
  uint16_t* const sEb = reinterpret_cast<uint16_t*>(sm + C::OFF_EB);
  const int64_t N = a.N;
  const int64_t ncols = a.ncols;
  const int64_t i0 = a.row0 + (int64_t)blockIdx.y * M;
  const int64_t rend = a.row0 + a.nrows;
  const int64_t c0 = (int64_t)blockIdx.x * col_chunk;
  const int64_t c1 = (c0 + col_chunk < ncols) ? c0 + col_chunk : ncols;
  const int nc = (int)(c1 > c0 ? c1 - c0 : 0);
  auto colj = [&](int c) -> int64_t {
    const int64_t cc = c0 + c;
    return upd_col(a, cc);
  };

  // ---- set-up: barriers, tensor memory, zero Hankel corners ----------------
  // the Hankel cores outside the digit window are zero for every column
  static_assert(C::OFF_BX == C::OFF_H + 2 * C::HBYTES, "Hankel and extra-K buffers are contiguous");
  // ... and the extra K step's rows 1 and 2 hold 2^23 and kOff at every
  // position (its row 0, b's raw digits, is written per column)
  for (int q = tid; q < (2 * C::HBYTES + 2 * C::XBYTES) / 16; q += pipe::NTH) {
    const int o = q * 16 - 2 * C::HBYTES;  // byte offset in the extra-K buffers
    const bool krow = o >= 0 && (o & 255) < 128;  // a row of k-core 0
    reinterpret_cast<uint4*>(sm + C::OFF_H)[q] =
        krow ? make_uint4((uint32_t)pipe::kBias23 << 16, pipe::kBiasOff, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    for (int t = 0; t < 4; ++t) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_full + 8 * t));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b_empty + 8 * t), "r"(M));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_hfree + 8 * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b_tfull + 8 * b), "r"(M));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b_tfree + 8 * b), "r"(M));
    }
    for (int b = 0; b < 2; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_hready + 8 * b));
    for (int b = 0; b < 4; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_xfull + 8 * b));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b_aready), "r"(M));
    *eflag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(C::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  if (warp == 8) {
    // ================= I: MMA issuer, one thread =========================
    // waits until the builders have a column's Hankel cores in shared memory,
    // then issues its MMAs tile group by tile group as the epilogue releases
    // the tensor-memory tiles; tcgen05.commit signals each tile (full) and the
    // Hankel buffer (hfree)
    if ((tid & 31) == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
      const uint32_t idesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * NT) >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
      // descriptors of the first K step; a K step adds 256 bytes to A's start
      // address and two cores (256 bytes) to the Hankel operand's, a tile 16
      // cores (the address field counts 16-byte units and never carries out)
      const uint64_t ad0 = desc(su32(sA), 128, C::KA * 16);
      const uint64_t hd0 = desc(su32(sm + C::OFF_H), 128, 128);
      const uint64_t xd0 = desc(su32(sm + C::OFF_BX), 128, 256);
      const uint64_t adx = ad0 + (uint64_t)((KD / 16) * 16);  // the extra K step
      const bool aok = nc <= 0 || wait_bar(b_aready, 0);
      if (!aok) *eflag = 1;
      for (int c = 0; c < nc && aok; ++c) {
        const int hb = c & 1;
        const int tu = (c % C::TB) * TILES;  // this column's tile slots
        const uint64_t hd = hd0 + (uint64_t)(hb * (C::HBYTES >> 4));
        const uint64_t xd = xd0 + (uint64_t)(hb * (C::XBYTES >> 4));
        if (!wait_bar(b_hready + 8 * hb, (c >> 1) & 1) || *eflag) {
          *eflag = 1;
          break;
        }
        bool okm = true;
#pragma unroll
        for (int t = 0; t < TILES; ++t) {
          if (t > 0 && C::merge(t - 1)) continue;  // issued with tile t - 1
          const bool two = C::merge(t);
          if (okm && c >= C::TB) {  // the epilogue has drained the buffer's previous column
            const uint32_t par = (uint32_t)(c / C::TB - 1) & 1u;
            okm = wait_bar(b_empty + 8 * (tu + t), par);
            if (two) okm = okm && wait_bar(b_empty + 8 * (tu + t + 1), par);
          }
          if (!okm) continue;
          asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
          for (int ks = C::ks_lo(t); ks < C::ks_hi(t); ++ks)
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                    tmem + (uint32_t)((tu + t) * NT)),
                "l"(ad0 + (uint64_t)(ks * 16)), "l"(hd + (uint64_t)((16 * t + 2 * ks) * 8)), "r"(two ? idesc2 : idesc),
                "r"(ks > C::ks_lo(t) ? 1u : 0u));
          // 2^p * b: the extra K step for the tiles at or above position KD
#pragma unroll
          for (int u = t; u <= (two ? t + 1 : t); ++u)
            if (u >= C::XT0)
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                      tmem + (uint32_t)((tu + u) * NT)),
                  "l"(adx), "l"(xd + (uint64_t)((u - C::XT0) * 256)), "r"(idesc), "r"(1u));
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b_full + 8 * (tu + t)));
          if (two)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                b_full + 8 * (tu + t + 1)));
        }
        if (!okm) *eflag = 1;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b_hfree + 8 * hb));
        if (!okm) break;
      }
    }
    __syncwarp();
  } else if (warp > 8) {
    // ================= B: Hankel builders, warps 9-11 ====================
    // per column: b's limbs (sB), b's balanced digits (warp 9), the Hankel
    // cores of b~ and b's raw digits for the extra K step into the free
    // buffers, then hready
    const int bt = tid - 288;
    // b of the next column (limb bt and the exponent), loaded one column ahead
    uint32_t bl_n = 0u;
    int64_t be_n = ZEXP;
    if (nc > 0) {
      const int64_t kj = a.brow * N + colj(0);
      if (bt < NL) bl_n = X.m[kj * NL + bt];
      be_n = X.e[kj];
    }
    for (int c = 0; c < nc; ++c) {
      const int hb = c & 1;
      unsigned char* sH = sm + C::OFF_H + hb * C::HBYTES;
      uint32_t* sB = sBl + hb * NL;
      const uint32_t bl = bl_n;
      const bool bz = be_n == ZEXP;
      if (c + 1 < nc) {
        const int64_t kj = a.brow * N + colj(c + 1);
        if (bt < NL) bl_n = X.m[kj * NL + bt];
        be_n = X.e[kj];
      }
      bool bad = false;
      if (bt == 0 && c >= 2 && !wait_bar(b_hfree + 8 * hb, ((c - 2) >> 1) & 1)) bad = true;
      if (pipe::pbar_or(bad || *eflag != 0)) {
        *eflag = 1;
        break;
      }
      if (bt < NL) sB[bt] = bl;
      pipe::pbar();
      // raw digit d_{r - KD} at output position r of the upper tiles: core
      // (n-core (r % 128) / 8 of tile r / 128, k-core 0), row r % 8, element 0
      {
        unsigned char* bx = sm + C::OFF_BX + hb * C::XBYTES;
        const unsigned char* bb = reinterpret_cast<const unsigned char*>(sB);
        for (int r = 128 * C::XT0 + bt; r < 128 * TILES; r += 96) {
          const int j = r - KD;
          const uint16_t v = (j >= 0 && j < KD && !bz) ? (uint16_t)pipe::dbfs((int)bb[j]) : (uint16_t)0;
          *reinterpret_cast<uint16_t*>(bx + (r / 128 - C::XT0) * 4096 + ((r % 128) / 8) * 256 + (r % 8) * 16) = v;
        }
      }
      if (warp == 9) {
        // balanced digits of b: carries across lanes by carry lookahead (lane l
        // holds digits [l * DPL, (l + 1) * DPL)); the top carry is digit KD
        constexpr int DPL = KD / 32;
        const unsigned char* bb = reinterpret_cast<const unsigned char*>(sB);
        int f0 = 0, f1 = 1;
#pragma unroll
        for (int q = 0; q < DPL; ++q) {
          const int d = bb[bt * DPL + q];
          f0 = (d + f0) >= 128 ? 1 : 0;
          f1 = (d + f1) >= 128 ? 1 : 0;
        }
        const uint64_t cm = carry_mask(__ballot_sync(FULL, f0 != 0), __ballot_sync(FULL, f1 != 0 && f0 == 0), 0u);
        int cy = (int)((cm >> bt) & 1u);
#pragma unroll
        for (int q = 0; q < DPL; ++q) {
          const int t = (int)bb[bt * DPL + q] + cy;
          cy = t >= 128 ? 1 : 0;
          sEb[bt * DPL + q] = bz ? (uint16_t)0 : (uint16_t)pipe::dbfs(t - (cy << 8));
        }
        if (bt == 31) sEb[KD] = bz ? (uint16_t)0 : (uint16_t)pipe::dbfs((int)((cm >> 32) & 1u));
      }
      pipe::pbar();
      // core d, row nn holds b~[8 (d - KD/8) + nn + 1 .. + 8]: only cores
      // KD/8 - 1 .. KD/4 - 1 meet digits 0..KD; the others stay zero
      for (int q = bt; q < (KD / 8 + 1) * 8; q += 96) {
        const int d = KD / 8 - 1 + (q >> 3), nn = q & 7;
        const int base = 8 * d + nn - (KD - 1);
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          uint32_t h2[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int idx = base + 2 * e + u;
            h2[u] = (idx >= 0 && idx <= KD) ? (uint32_t)sEb[idx] : 0u;
          }
          w[e] = h2[0] | (h2[1] << 16);
        }
        *reinterpret_cast<uint4*>(sH + d * 128 + nn * 16) = make_uint4(w[0], w[1], w[2], w[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;");
      pipe::pbar();
      if (bt == 0) arrive(b_hready + 8 * hb);
    }
  } else if (warp < 4) {
    // ================= E: epilogue, one thread per row ====================
    // Forms each row's 2n-limb product z' * b~ + 2^p * b from the column's
    // 2 KD exact sums (32-column chunks, the next chunk loading while this
    // one is processed) and stages for the subtraction role its upper n
    // limbs, limb n - 1 and the OR of the limbs below (it rounds there).
    // Lazy low half: the carry chain starts at limb NL - 8 with a zero carry.
    // The sums below contribute less than 2^(32 (NL - 8) + 14) in magnitude,
    // so when bits [14, 224) of limbs NL-8 .. NL-2 hold both a one and a zero
    // they change neither those limbs' carry out nor the sticky bit (which is
    // then set); otherwise the warp reads the low chunks and adds their exact
    // carry.  The low tiles are released only after that decision.
    const int r = tid;
    const int8_t zsign = (i0 + r < rend) ? Z.s[i0 + r] : 0;
    const int64_t zexp = (i0 + r < rend) ? Z.e[i0 + r] : ZEXP;
    const bool have = zexp != ZEXP;
    {
      // A: the balanced digits of this row's multiplier (the top carry is the
      // 2^p of z = z' + 2^p), digit s at k' = KD - 1 - s: limb L's four digits
      // fill k' = KD - 4 - 4L .. KD - 1 - 4L; then the extra K step's 1 at
      // k' = KD and zeros after it.  Digits in [-128, 127] are unique, so they
      // are the bytes of z + (128, 128, ..., 128) in base 256, less 128: one
      // carry chain over the limbs instead of one over the digits.  The row's
      // limbs arrive by vector loads issued together.
      const uint32_t* zm = Z.m + (have ? i0 + r : i0) * NL;
      unsigned char* rowbase = sA + (r >> 3) * (C::KA * 16) + (r & 7) * 16;
      uint32_t f[NL];
#pragma unroll
      for (int q = 0; q < NL / 4; ++q) {
        const uint4 v = have ? *reinterpret_cast<const uint4*>(zm + 4 * q) : make_uint4(0u, 0u, 0u, 0u);
        f[4 * q] = v.x;
        f[4 * q + 1] = v.y;
        f[4 * q + 2] = v.z;
        f[4 * q + 3] = v.w;
      }
      f[0] = add_cc(f[0], 0x80808080u);
#pragma unroll
      for (int L = 1; L < NL; ++L) f[L] = addc_cc(f[L], 0x80808080u);
#pragma unroll
      for (int L = 0; L < NL; ++L) {
        uint32_t h[4];  // bf16 of byte q - 128: exact through fp32 (2^23 + byte, less 2^23 + 128)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          h[q] = __float_as_uint(__uint_as_float(0x4B000000u | ((f[L] >> (8 * q)) & 255u)) - 8388736.0f) >> 16;
        const int k0 = KD - 4 - 4 * L;
        *reinterpret_cast<uint2*>(rowbase + (k0 >> 3) * 128 + (k0 & 7) * 2) =
            make_uint2(h[3] | (h[2] << 16), h[1] | (h[0] << 16));
      }
      *reinterpret_cast<uint4*>(rowbase + (KD / 8) * 128) = make_uint4(0x3F803F80u, 0x3F80u, 0u, 0u);
      *reinterpret_cast<uint4*>(rowbase + (KD / 8 + 1) * 128) = make_uint4(0u, 0u, 0u, 0u);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A is read by the tensor core
      arrive(b_aready);
    }
    constexpr int NCH = 4 * TILES;    // chunks of 32 sums (8 limbs)
    constexpr int K0 = NL / 8 - 1;     // first chunk read: limbs NL - 8 .. NL - 1
    constexpr int T0 = K0 >> 2;        // its tile
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    // b's exponent and sign, loaded one column ahead
    int64_t be_n = ZEXP;
    int8_t bs_n = 0;
    if (nc > 0) {
      be_n = X.e[a.brow * N + colj(0)];
      bs_n = X.s[a.brow * N + colj(0)];
    }
    for (int c = 0; c < nc; ++c) {
      const int tb = c & 1;
      const int tu = (c % C::TB) * TILES;                          // this column's tile slots
      const uint32_t tc = tl + (uint32_t)(tu * NT);                // and its tensor memory
      const uint32_t fpar = (uint32_t)(c / C::TB) & 1u;            // parity of its full barriers
      const int64_t be = be_n;
      const int8_t bs = bs_n;
      if (c + 1 < nc) {
        be_n = X.e[a.brow * N + colj(c + 1)];
        bs_n = X.s[a.brow * N + colj(c + 1)];
      }
      const bool used = have && be != ZEXP;  // the row's product is used
      const RowT<NL> Tw{sT + (tb * 4 + warp) * TILE, (uint32_t)(tid & 31)};
      uint32_t l63 = 0, sticky = 0;
      int64_t acc = 0;
      bool okc = true;
      uint32_t va[32], vb[32];
      // tiles complete in issue order: tile T0 done means the ones below are too
      if (!wait_bar(b_full + 8 * (tu + T0), fpar)) okc = false;
      okc = __all_sync(0xffffffffu, okc) && !*eflag;
      okc = __all_sync(0xffffffffu, okc);
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (okc) tmem_ld32_async(tc + 32 * K0, va);
      // biased: the sums already carry kMagic (tiles from XT0 up)
      auto limbs8 = [&](const uint32_t* v, const int64_t* kv, uint32_t(&lim)[8], int64_t& ac, const bool biased) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          uint32_t u[4];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            u[j] = biased ? v[4 * q + j]
                          : __float_as_uint(__fadd_rn(__uint_as_float(v[4 * q + j]), pipe::kMagic));  // 0x4B000000 + u
          const uint32_t xl = u[0] + (u[1] << 8), yl = u[2] + (u[3] << 8);
          ac += (int64_t)((uint64_t)yl * 65536u + xl) + kv[q];
          lim[q] = (uint32_t)ac;
          ac >>= 32;
        }
      };
      auto release_low = [&]() {  // tiles below T0, and T0 when K0 is its last chunk
        asm volatile("tcgen05.fence::before_thread_sync;");
#pragma unroll
        for (int t = 0; t < T0; ++t) arrive(b_empty + 8 * (tu + t));
        if ((K0 & 3) == 3) arrive(b_empty + 8 * (tu + T0));
      };
      auto chunk = [&](const int k, uint32_t(&cur)[32], uint32_t(&nxt)[32]) {
        const bool upper = 8 * k >= NL;
        if (8 * k == NL && okc) {  // first upper chunk: the staging buffer must be free
          const bool okw = (c < 2) || wait_bar(b_tfree + 8 * tb, ((c - 2) >> 1) & 1);
          okc = __all_sync(0xffffffffu, okw);
        }
        const int64_t kv[8] = {-pipe::kC, -pipe::kC, -pipe::kC, -pipe::kC,
                               -pipe::kC, -pipe::kC, -pipe::kC, -pipe::kC};
        if (okc) tmem_wait(cur);
        if (okc && (k & 3) == 3 && k != K0) {  // the tile's last chunk is in registers: release it
          asm volatile("tcgen05.fence::before_thread_sync;");
          arrive(b_empty + 8 * (tu + (k >> 2)));
        }
        if (k + 1 < NCH && okc) {
          if (((k + 1) & 3) == 0) {
            bool okt = wait_bar(b_full + 8 * (tu + ((k + 1) >> 2)), fpar);
            okt = __all_sync(0xffffffffu, okt) && !*eflag;
            okc = __all_sync(0xffffffffu, okt);
            asm volatile("tcgen05.fence::after_thread_sync;");
          }
          if (okc) tmem_ld32_async(tc + (uint32_t)(32 * (k + 1)), nxt);
        }
        if (!okc) return;
        uint32_t lim[8];
        if ((k >> 2) >= C::XT0)
          limbs8(cur, kv, lim, acc, true);
        else
          limbs8(cur, kv, lim, acc, false);
        if (upper) {
          Tw.st16(2 * k - NL / 4, make_uint4(lim[0], lim[1], lim[2], lim[3]));
          Tw.st16(2 * k - NL / 4 + 1, make_uint4(lim[4], lim[5], lim[6], lim[7]));
          return;
        }
        // k == K0: limbs NL - 8 .. NL - 1 with a zero carry in
        const uint32_t lo7 = lim[1] | lim[2] | lim[3] | lim[4] | lim[5] | lim[6];
        const uint32_t hi7 = lim[1] & lim[2] & lim[3] & lim[4] & lim[5] & lim[6];
        const bool any1 = ((lim[0] >> 14) | lo7) != 0u;
        const bool any0 = ((~lim[0] >> 14) | ~hi7) != 0u;
        const bool unsafe = used && !(any1 && any0);
        l63 = lim[7];
        sticky = 1u;
        if (__any_sync(0xffffffffu, unsafe)) {
          // exact low part: limbs 0 .. NL - 9 and its carry into limb NL - 8
          int64_t ac2 = 0;
          uint32_t slo = 0;
          const int64_t kvl[8] = {-pipe::kC, -pipe::kC, -pipe::kC, -pipe::kC,
                                  -pipe::kC, -pipe::kC, -pipe::kC, -pipe::kC};
#pragma unroll 1
          for (int kk = 0; kk < K0; ++kk) {
            uint32_t w[32];
#pragma unroll
            for (int part = 0; part < 4; ++part) {
              uint32_t w8[8];
              tmem_ld8(tc + (uint32_t)(32 * kk + 8 * part), w8);
#pragma unroll
              for (int e = 0; e < 8; ++e) w[8 * part + e] = w8[e];
            }
            uint32_t l8[8];
            limbs8(w, kvl, l8, ac2, (kk >> 2) >= C::XT0);
            slo |= l8[0] | l8[1] | l8[2] | l8[3] | l8[4] | l8[5] | l8[6] | l8[7];
          }
          if (unsafe) {
            int64_t t = ac2;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              t += (int64_t)lim[q];
              lim[q] = (uint32_t)t;
              t >>= 32;
            }
            acc += t;
            l63 = lim[7];
            sticky = slo | lim[0] | lim[1] | lim[2] | lim[3] | lim[4] | lim[5] | lim[6];
          }
        }
        release_low();
      };
#pragma unroll 1
      for (int k = K0; k + 1 < NCH; k += 2) {
        chunk(k, va, vb);
        chunk(k + 1, vb, va);
      }
      chunk(NCH - 1, va, vb);  // NCH - K0 is odd: the last chunk is in va
      if (!okc) {  // warp-uniform
        *eflag = 1;
        break;
      }
      const bool tz = !have || be == ZEXP;
      sTa[(tb * M + r) * 2] = l63;
      sTa[(tb * M + r) * 2 + 1] = sticky;
      sTe[tb * M + r] = tz ? ZEXP : zexp + be;  // before rounding
      sTs[tb * M + r] = tz ? (int8_t)0 : (int8_t)(zsign ^ bs);
      arrive(b_tfull + 8 * tb);
    }
  } else {
    // ================= S: one thread per row subtracts ====================
    const int r = tid - 128;
    const int64_t i = i0 + r;
    const bool active = i < rend;
    const int64_t irow = active ? i : i0;
    const int w = warp - 4;
    unsigned char* const xtile = sm + C::OFF_X + w * TILE;
    const RowT<NL> Xr{xtile, (uint32_t)(tid & 31)};
    const uint32_t xbar = b_xfull + 8 * w;
    // The results replace the staged products in the warp's T tile and leave
    // by one TMA store per 128-byte half, unless the tile holds rows in
    // [rend, N) (back substitution), which are not this launch's to write:
    // then each thread stores its own row.
    const bool tma_out = rend >= N || i0 + 32 * w + 32 <= rend;
    auto store_tile = [&](const unsigned char* tile, const int64_t j) {
      const int row0 = (int)(i0 + 32 * w), col = (int)j;
      asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                       reinterpret_cast<uint64_t>(&tmx0)),
                   "r"(0), "r"(col), "r"(row0), "r"(su32(tile))
                   : "memory");
      if (NL > 32)
        asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                         reinterpret_cast<uint64_t>(&tmx1)),
                     "r"(0), "r"(col), "r"(row0), "r"(su32(tile + 4096))
                     : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    };
    // x_ij of a column for the warp's 32 rows: one TMA copy per 128-byte half
    // of the rows (rows beyond N read as zero), completing on the warp's xfull
    // barrier; sign and exponent into registers.  The tile's earlier generic
    // reads have returned their values before the warp reaches this point.
    auto fetch_x = [&](const int64_t j) {
      __syncwarp();
      if ((tid & 31) == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(xbar), "r"(TILE) : "memory");
        const int row0 = (int)(i0 + 32 * w), col = (int)j;
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
                su32(xtile)),
            "l"(reinterpret_cast<uint64_t>(&tmx0)), "r"(0), "r"(col), "r"(row0), "r"(xbar)
            : "memory");
        if (NL > 32)
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
                  su32(xtile + 4096)),
              "l"(reinterpret_cast<uint64_t>(&tmx1)), "r"(0), "r"(col), "r"(row0), "r"(xbar)
              : "memory");
      }
    };
    int8_t xs_n = 0;
    int64_t xe_n = ZEXP;
    int pending = -1;  // column whose copy is issued and not yet waited for
    if (nc > 0) {
      const int64_t j = colj(0);
      fetch_x(j);
      pending = 0;
      xs_n = X.s[irow * N + j];
      xe_n = X.e[irow * N + j];
    }
    for (int c = 0; c < nc; ++c) {
      const int tb = c & 1;
      const int64_t ij = irow * N + colj(c);
      const int8_t xs = xs_n;
      const int64_t xe = xe_n;
      bool okc = wait_bar(b_tfull + 8 * tb, (c >> 1) & 1);
      okc = okc && wait_bar(xbar, c & 1);
      okc = __all_sync(0xffffffffu, okc) && !*eflag;
      okc = __all_sync(0xffffffffu, okc);
      if (!okc) {
        *eflag = 1;
        break;
      }
      pending = -1;
      // the previous column's store has read its tile: the epilogue may
      // stage into that buffer again
      if (c > 0) {
        if ((tid & 31) == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncwarp();
        arrive(b_tfree + 8 * (tb ^ 1));
      }
      int8_t rs = 0;
      int64_t re = ZEXP;
      const RowT<NL> Tr{sT + (tb * 4 + w) * TILE, (uint32_t)(tid & 31)};
      if (active) {
        int64_t te = sTe[tb * M + r];
        if (te != ZEXP) te += round_product<NL>(Tr, sTa[(tb * M + r) * 2], sTa[(tb * M + r) * 2 + 1]);
        sub_row<NL>(Xr, xs, xe, Tr, sTs[tb * M + r], te, Tr, rs, re);
      }
      // x is no longer read: the next column's copy may start
      if (c + 1 < nc) {
        const int64_t j2 = colj(c + 1);
        fetch_x(j2);
        pending = c + 1;
        xs_n = X.s[irow * N + j2];
        xe_n = X.e[irow * N + j2];
      }
      if (tma_out) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the results, to the TMA store
        __syncwarp();
        if ((tid & 31) == 0) store_tile(Tr.tile, colj(c));
      } else if (active) {
        copy_row<NL>(Tr, X.m + ij * NL);
      }
      if (active) {
        X.s[ij] = rs;
        X.e[ij] = re;
      }
    }
    // no copy may still be writing this block's shared memory, and no store
    // reading it, at exit (after an early stop too); column c's copy
    // completes the barrier's phase c
    if ((tid & 31) == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (pending >= 0) wait_bar(xbar, pending & 1);
  }
  if (tid == 0 && *eflag) atomicExch(status, 5);  // MPDET_ETIMEOUT
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS));
}


}  // namespace tc

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point
// query (no link against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

// Tensor maps for the subtraction role's x copies: half h (128 bytes, or the
// whole 64-byte row at n = 16) of every number of the N x N array as a 3-D
// tensor (words, column, row); a box is 1 column x 32 rows, written with the
// swizzle RowT reads.
static cudaError_t x_tensor_maps(MpArr X, int64_t N, int nl, CUtensorMap (&tm)[2]) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const int d0 = nl < 32 ? nl : 32;
  for (int h = 0; h < 2; ++h) {
    const int hh = nl > 32 ? h : 0;
    const cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)N, (cuuint64_t)N};
    const cuuint64_t strides[2] = {(cuuint64_t)nl * 4, (cuuint64_t)N * nl * 4};
    const cuuint32_t box[3] = {(cuuint32_t)d0, 1, 32};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = enc(&tm[h], CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, X.m + 32 * hh, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, nl >= 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// Launch: 128-row blocks x column chunks sized to fill the SMs once.
cudaError_t update_tc(MpArr X, const UpdArgs& a, MpArr Z, int* status, int p, int nsm, cudaStream_t st,
                      int pipelined) {
  const int64_t ncols = a.ncols;
  if (a.nrows <= 0 || ncols <= 0) return cudaSuccess;
  const int64_t by = (a.nrows + tc::M - 1) / tc::M;
  int64_t bx = nsm / by;  // one wave: at most one block per SM
  if (bx > ncols) bx = ncols;
  if (bx < 1) bx = 1;
  const int64_t chunk = (ncols + bx - 1) / bx;
  bx = (ncols + chunk - 1) / chunk;
  dim3 grid((unsigned)bx, (unsigned)by);
  if (pipelined) {
    CUtensorMap tm[2];
    const cudaError_t e = x_tensor_maps(X, a.N, p / 32, tm);
    if (e != cudaSuccess) return e;
    switch (p) {
      case 512:
        cudaFuncSetAttribute(tc::k_update_tcp<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::pipe::Cfg<64>::SMEM);
        tc::k_update_tcp<64><<<grid, tc::pipe::NTH, tc::pipe::Cfg<64>::SMEM, st>>>(X, a, Z, status, p, (int)chunk, tm[0],
                                                                                       tm[1]);
        break;
      case 1024:
        cudaFuncSetAttribute(tc::k_update_tcp<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::pipe::Cfg<128>::SMEM);
        tc::k_update_tcp<128><<<grid, tc::pipe::NTH, tc::pipe::Cfg<128>::SMEM, st>>>(X, a, Z, status, p, (int)chunk, tm[0],
                                                                                       tm[1]);
        break;
      case 2048:
        cudaFuncSetAttribute(tc::k_update_tcp<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::pipe::Cfg<256>::SMEM);
        tc::k_update_tcp<256><<<grid, tc::pipe::NTH, tc::pipe::Cfg<256>::SMEM, st>>>(X, a, Z, status, p, (int)chunk, tm[0],
                                                                                       tm[1]);
        break;
      default:
        return cudaErrorInvalidValue;
    }
  } else {
    if (p != 2048) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(tc::k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM);
    tc::k_update_tc<<<grid, 128, tc::SMEM, st>>>(X, a, Z, status, p, (int)chunk);
  }
  return cudaGetLastError();
}

// True when the tensor engine covers p (the warp-specialised kernel: p = 512,
// 1024, 2048; the one-phase-at-a-time kernel: p = 2048).
bool tc_supports(int p, int pipelined) { return pipelined ? (p == 512 || p == 1024 || p == 2048) : p == 2048; }

}  // namespace mpd
