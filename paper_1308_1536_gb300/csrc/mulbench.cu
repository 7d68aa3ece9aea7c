// Rounded products RN_p(a_i * b_i) by the IMAD engine's schoolbook product
// (mul_round, the one the Schur update uses) or by one Karatsuba level over
// half-size schoolbook products (mul_round_kara), for measuring the two on
// the same operands (the paper's CPU runs use GMP's Karatsuba, Sec. 4.2 and
// Table 2).  Both give the same bits: the product is exact before it is
// rounded.
#include "../../include/mpdet.h"
#include "karatsuba.cuh"
#include "kernelset.h"

namespace mpd {

// One group per pair, every group computes its product `reps` times (the
// operands stay in shared memory and registers) and stores it once.
template <int W, int G, bool KARA>
__global__ void __launch_bounds__(128) k_mulbench(int64_t count, MpArr A, MpArr B, MpArr O, int reps) {
  constexpr int n = W * G;
  constexpr int NG = 128 / G;
  constexpr int SCR = KARA ? 3 * n : 0;  // lo (n) + three half lower halves + s'_z (2n)
  extern __shared__ __align__(16) uint32_t smem[];
  Grp<G> gp;
  const int gid = threadIdx.x / G;
  uint32_t* zb = smem + gid * (n + SCR);
  uint32_t* scr = zb + n;
  int64_t idx = (int64_t)blockIdx.x * NG + gid;
  const bool active = idx < count;
  if (!active) idx = count - 1;
  uint32_t a[W], M[W];
  load_slice<W>(A.m + idx * n + gp.g * W, a);
  uint32_t zv[W];
  load_slice<W>(B.m + idx * n + gp.g * W, zv);
  store_slice<W>(zb + gp.g * W, zv);
  __syncwarp();
  int adj = 0;
  uint32_t acc = 0u;
#pragma unroll 1
  for (int r = 0; r < reps; ++r) {
    if constexpr (KARA)
      adj = mul_round_kara<W, G>(gp, a, zb, M, scr, A.pad);
    else
      adj = mul_round<W, G>(gp, a, zb, M, A.pad);
    acc ^= M[0];  // keeps every repetition live
    a[0] ^= (acc & 0u);
  }
  const int8_t as = A.s[idx], bs = B.s[idx];
  const int64_t ae = A.e[idx], be = B.e[idx];
  const bool zero = ae == ZEXP || be == ZEXP;
  if (zero) {
#pragma unroll
    for (int q = 0; q < W; ++q) M[q] = 0u;
  }
  if (active) {
    store_slice<W>(O.m + idx * n + gp.g * W, M);
    if (gp.g == 0) {
      O.s[idx] = zero ? 0 : (int8_t)(as ^ bs);
      O.e[idx] = zero ? ZEXP : ae + be + adj;
    }
  }
}

template <int W, int G, bool KARA>
static cudaError_t launch_mulbench(int64_t count, MpArr A, MpArr B, MpArr O, int reps, cudaStream_t st) {
  constexpr int n = W * G;
  constexpr int NG = 128 / G;
  const size_t sm = (size_t)NG * (n + (KARA ? 3 * n : 0)) * 4;
  cudaError_t e = cudaFuncSetAttribute(k_mulbench<W, G, KARA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (count + NG - 1) / NG;
  k_mulbench<W, G, KARA><<<(unsigned)blocks, 128, sm, st>>>(count, A, B, O, reps);
  return cudaGetLastError();
}

}  // namespace mpd

extern "C" int mpdet_mulbench(int method, int64_t count, int32_t p_bits, mpdet_numv a, mpdet_numv b, mpdet_numv out,
                              int reps, void* cuda_stream, float* ms) {
  if ((method != 0 && method != 1) || count < 1 || count > (int64_t)1 << 30 || reps < 1 || reps > 1 << 20)
    return MPDET_EINVAL;
  if (p_bits != 8192 && p_bits != 16384 && p_bits != 32768) return MPDET_EINVAL;
  if (!a.sign || !a.exp || !a.limbs || !b.sign || !b.exp || !b.limbs || !out.sign || !out.exp || !out.limbs)
    return MPDET_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  mpd::MpArr A{a.sign, a.exp, a.limbs}, B{b.sign, b.exp, b.limbs}, O{out.sign, out.exp, out.limbs};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return MPDET_ECUDA;
  }
  cudaError_t e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    if (p_bits == 8192)
      e = method ? mpd::launch_mulbench<16, 16, true>(count, A, B, O, reps, st)
                 : mpd::launch_mulbench<16, 16, false>(count, A, B, O, reps, st);
    else if (p_bits == 16384)
      e = method ? mpd::launch_mulbench<16, 32, true>(count, A, B, O, reps, st)
                 : mpd::launch_mulbench<16, 32, false>(count, A, B, O, reps, st);
    else
      e = method ? mpd::launch_mulbench<32, 32, true>(count, A, B, O, reps, st)
                 : mpd::launch_mulbench<32, 32, false>(count, A, B, O, reps, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MPDET_ECUDA;
  }
  if (ms) *ms = t;
  return MPDET_OK;
}
