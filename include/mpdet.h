/*
 * mpdet — fixed-precision multiprecision Gaussian elimination on one GPU.
 *
 * Computes, for a real N x N matrix A held at p bits, the determinant, all N
 * top-left leading minors and the signed minors of the last column, by
 * Gaussian elimination without pivoting (Beliakov & Matiyasevich, Sec. 3 and
 * Algorithm 1, with the augmented matrix [A I] of Sec. 3 for the minors).
 *
 * Number format (every call): a number is
 *     x = (-1)^s * m * 2^(e - p),   2^(p-1) <= m < 2^p,
 * with m stored as n = p/32 little-endian uint32 limbs and e an int64; zero is
 * s = 0, m = 0, e = INT64_MIN (no -0, no infinities, no NaN).  Every operation
 * of the method is the exact result rounded to nearest, ties to even, at p
 * bits, in a fixed order:
 *     D_k  = RN(D_{k-1} * a_kk)          (D_0 = 1)     Alg. 1 step 2.1
 *     r_k  = RN(1 / a_kk)
 *     z_ik = RN(a_ik * r_k),        i > k              Alg. 1 step 2.2.1
 *     a_ij = RN(a_ij - RN(z_ik * a_kj)),  i, j > k     Alg. 1 step 2.2.2
 * and in MPDET_LASTCOL mode the same row operation on the identity block of
 * [A I], stored in A's strict lower triangle (Sec. 3, memory N^2 + O(N)):
 *     l_ij = RN(l_ij - RN(z_ik * l_kj)),  i > k, j < k;   l_ik = -z_ik.
 * Results are therefore bit-for-bit reproducible and independent of the
 * kernels' tiling.
 *
 * Arrays of numbers cross the ABI as mpdet_numv (structure of arrays):
 * count numbers, sign[count] int8, exp[count] int64, limbs[count * n] uint32
 * (number i's limbs at limbs[i*n .. i*n + n)).  Row-major for matrices.
 *
 * Pointers: with device_ptr = 0 an argument is host memory and the call is
 * synchronous (it returns after the results are in host memory).  With
 * device_ptr = 1 it is device memory of the handle's GPU (for instance a torch
 * CUDA tensor) and the call is asynchronous on the handle's stream: results
 * are valid after that stream synchronises, and errors found on the device
 * (zero pivots) are reported by mpdet_status.  Device buffers of numbers must
 * be 16-byte aligned.
 *
 * Ownership: the handle owns all of its device memory; caller buffers are
 * only read or written during the call (or, for device_ptr = 1, during the
 * stream work the call enqueues).
 *
 * Errors: every call returns a status code; nothing is thrown across the ABI.
 * mpdet_last_error gives a message for the last failing call on a handle.
 * After MPDET_EZEROPIVOT the handle stays usable (a new matrix may be set);
 * after MPDET_ECUDA it should be freed.
 */
#ifndef MPDET_H
#define MPDET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int8_t* sign;
  int64_t* exp;
  uint32_t* limbs;
} mpdet_numv;

typedef struct mpdet_ctx* mpdet_t;

enum {
  MPDET_OK = 0,
  MPDET_EINVAL = 1,      /* bad argument (size, precision, null pointer, state order) */
  MPDET_ENOMEM = 2,      /* device or host allocation failed */
  MPDET_ECUDA = 3,       /* a CUDA call failed; see mpdet_last_error */
  MPDET_EZEROPIVOT = 4,  /* exact zero pivot a_kk at k < N: elimination stopped */
  MPDET_ETIMEOUT = 5,    /* a bounded device wait gave up */
  MPDET_ESTATE = 6,      /* call out of order (e.g. minors before the factorisation) */
  MPDET_EZERODIV = 7,    /* normalised minors requested but l_N1 (hence C_1N) is zero */
  MPDET_ENOSCRATCH = 8   /* problem larger than mpdet_factor_noalloc's static working memory */
};

enum { MPDET_LASTCOL = 1, MPDET_HOSTMEM = 2, MPDET_BALL = 4 };

/* Create a handle for N x N matrices at p bits on the current CUDA device.
 * p must be a multiple of 32 with 64 <= p <= 32768 (n = p/32 limbs).  The
 * kernel families hold 4, 8, ..., 1024 limbs; any other n runs in the next
 * family's frame (mantissa in its top n limbs, the low limbs zero) with every
 * operation rounded at p bits, so the results are those of the p-bit format,
 * at the cost of the frame (p = 3072 costs as much as p = 4096).  Buffers
 * crossing the ABI always hold n = p/32 limbs per number.  flags: 0 or MPDET_LASTCOL (keep L for the
 * last-column minors, 1.5x the work: Sec. 3 counts it as twice the row
 * operations).  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Allocates (4n + 9) * N^2 bytes of device memory plus O(N n).
 * MPDET_HOSTMEM (may be combined with MPDET_LASTCOL): the N x N array lives
 * in page-locked host memory mapped into the GPU's address space instead
 * (cudaHostAlloc, mapped), which the kernels read and write in place; on a
 * Grace-Blackwell node the GPU reaches it coherently over NVLink-C2C.  This
 * is for matrices larger than the GPU's memory, such as the paper's
 * production size N = 12000 at 32768 bits (590 GB, Sec. 4.2 pages blocks
 * to disk for it).  Every update of a p-bit number reads and writes 8n + 18
 * bytes for n^2 limb multiply-accumulates, so at p >= 8192 the link keeps
 * up with the arithmetic.  At p = 512 .. 2048 the update then runs on the
 * IMAD engine (that tensor-core engine's TMA copies address device memory
 * only); at p = 4096 .. 32768 the tensor-core engine reads and writes the
 * array with plain loads and stores and serves it.  Results are
 * bit-identical to the device-resident array.
 * Errors: MPDET_EINVAL (N < 1, unsupported p, unknown flag, out == NULL),
 * MPDET_ENOMEM, MPDET_ECUDA. */
int mpdet_create(int64_t N, int32_t p_bits, uint32_t flags, void* cuda_stream, mpdet_t* out);

/* MPDET_BALL (may be combined with the other flags): ball mode, the rigorous
 * error bounds the paper leaves to future work (Sec. 4.4: interval
 * arithmetic, upper and lower bounds at every operation).  Every value of the
 * elimination is computed exactly as without the flag (the same bits) and
 * carries a radius rho with |x* - x~| <= rho, x* being the value exact
 * arithmetic gives at the same place of the elimination of the exact input.
 * A radius is m * 2^(e - 32) with m in [2^31, 2^32), or 0 (m = 0, e =
 * INT64_MIN), or unbounded (e = INT64_MAX: a pivot's ball held zero, or the
 * elimination stopped before that minor); radii are rounded up in integer
 * arithmetic by three rules (u~ the rounded result, hu = 2^(e_u - p - 1) half
 * its ulp, |x~|^ and |x~|_ bounds of |x~| from its top limb):
 *   RN(x y):   ((hu + |x~|^ rho_y) + |y~|^ rho_x) + rho_x rho_y
 *   RN(x - t): (hu + rho_x) + rho_t
 *   RN(1/a):   hu + rho_a / (|a~|_ (|a~|_ - rho_a))  (unbounded unless |a~|_ > rho_a)
 * Inputs lifted from doubles or integers, and numbers given at p bits, are
 * exact (radius 0); Cauchy entries carry the radii of RN(x+y) and RN(1/s).
 * The update runs on the IMAD engine in ball mode; it costs N^2 * 12 more
 * bytes.  mpdet_radii reads the radii.  Series, the adjoint and mpdet_resume
 * carry no radii. */

/* Set A from an N x N row-major double matrix with leading dimension ld >= N
 * (exact lift: every finite double is representable at p >= 64).  Resets the
 * factorisation.  A is the input of Algorithm 1.  Host input is staged
 * through a device buffer the handle keeps.  Errors: MPDET_EINVAL (NULL
 * handle or A, ld < N), MPDET_ENOMEM (staging buffer), MPDET_ECUDA. */
int mpdet_set_f64(mpdet_t h, const double* A, int64_t ld, int device_ptr);

/* Same for int32 entries (exact).  Errors as for mpdet_set_f64. */
int mpdet_set_i32(mpdet_t h, const int32_t* A, int64_t ld, int device_ptr);

/* Set A (the input of Algorithm 1) from N*N numbers already at p bits,
 * row-major (copied; must be canonical: normalised mantissa or the zero
 * encoding).  Resets the factorisation.  Errors: MPDET_EINVAL (NULL handle or
 * pointer), MPDET_ECUDA. */
int mpdet_set_mp(mpdet_t h, mpdet_numv A, int device_ptr);

/* Set the Cauchy matrix A_ij = RN(1 / RN(x_i + y_j)) generated on the device
 * (x, y: N doubles each).  The seeded stand-in for the paper's interpolating
 * matrices of eq. (det) and eq. (betaNew), which are nearly singular.
 * Errors: MPDET_EINVAL (NULL handle or pointer), MPDET_ENOMEM (staging of host
 * x, y), MPDET_ECUDA. */
int mpdet_set_cauchy(mpdet_t h, const double* x, const double* y, int device_ptr);

/* Run elimination steps k0+1 .. k1 (1-based; 0 <= k0 <= k1 <= N), asynchronous
 * on the handle's stream.  k0 must equal the number of steps already done
 * (windows run in order; a factorisation can be split to time it or to
 * checkpoint it with mpdet_get_mp / mpdet_get_minors).  Errors: MPDET_ESTATE
 * (no matrix, or k0 out of order), MPDET_EINVAL, MPDET_ECUDA. */
int mpdet_factor_range(mpdet_t h, int64_t k0, int64_t k1);

/* Finish the factorisation (all remaining steps) and return det = D_N (one
 * number) and the leading minors D_1..D_N (N numbers); either output may have
 * NULL pointers to skip it.  zero_pivot_k (may be NULL, host) receives the
 * 1-based index of the first exactly zero pivot or 0.
 * Returns MPDET_EZEROPIVOT when that pivot is at k < N (D_1..D_{k-1} are
 * valid, D_k..D_N are +0); a zero pivot at k = N only makes det = +0 and
 * returns MPDET_OK.  With device_ptr = 1 the outputs are device buffers, the
 * call does not synchronise and zero pivots are read with mpdet_status
 * (*zero_pivot_k is then -1).  The leading minors are the running products of
 * the pivots (Algorithm 1 step 2.1; Sec. 3: elimination without pivoting gives
 * every top-left minor at no extra cost).  Errors: MPDET_EINVAL (NULL handle),
 * MPDET_ESTATE (no matrix set), MPDET_EZEROPIVOT, MPDET_ETIMEOUT (a bounded
 * wait of the tensor engine gave up), MPDET_ECUDA. */
int mpdet_factor(mpdet_t h, mpdet_numv det, mpdet_numv minors, int64_t* zero_pivot_k, int device_ptr);

/* Synchronise the handle's stream and read the status of the last
 * factorisation: MPDET_OK, MPDET_EZEROPIVOT (zero_pivot_k as above),
 * MPDET_EZERODIV (normalised minors with l_N1 = 0, device mode) or
 * MPDET_ETIMEOUT; MPDET_EINVAL for a NULL handle, MPDET_ECUDA when the
 * stream's work failed. */
int mpdet_status(mpdet_t h, int64_t* zero_pivot_k);

/* Signed minors of the last column (eq. minorsdef):
 *     C_jN = (-1)^(j+N) det(A without row j and column N) = RN(D_{N-1} * l_Nj),
 *     C_NN = D_{N-1},
 * N numbers.  normalised != 0 returns delta_{N,j} = C_jN / C_1N (eq. minors),
 * formed as RN(l_Nj * RN(1/l_N1)) with delta_{N,1} = 1 exactly.
 * Needs MPDET_LASTCOL and a completed factorisation without a zero pivot
 * before step N.  Errors: MPDET_ESTATE, MPDET_EZERODIV (normalised with
 * l_N1 = 0).  With device_ptr = 1 nothing is synchronised: a zero pivot or
 * l_N1 = 0 leaves the outputs undefined and is reported by mpdet_status
 * (MPDET_EZEROPIVOT or MPDET_EZERODIV). */
int mpdet_lastcol_minors(mpdet_t h, mpdet_numv out, int normalised, int device_ptr);

/* Signed minors of the last column for every leading size n = 1..N from one
 * elimination: the series of minor arrays for N = 2, 3, ... that the paper's
 * application needs (Sec. 3: at step n, row n of L holds the minors of the
 * leading n x n matrix's last column up to a factor, so the series costs no
 * extra elimination work).  Row n of L is final after step n-1 and the
 * leading n x n block goes through the same rounded operations as a
 * standalone n x n matrix, so series n is bit-identical to
 * mpdet_lastcol_minors of that block:
 *     C^(n)_jn = RN(D_{n-1} * l_nj),  j < n;    C^(n)_nn = D_{n-1}  (D_0 = 1),
 * or with normalised != 0 the delta of eq. (minors) for every n:
 *     delta^(n)_j = RN(l_nj * RN(1/l_n1)),  1 < j < n;   delta^(n)_1 = 1;
 *     delta^(n)_n = RN(1/l_n1);   delta^(1)_1 = 1,
 * where a series with l_n1 = 0 (C_1n = 0, delta undefined) comes out all +0.
 * out: N(N+1)/2 numbers, series n at offset n(n-1)/2 (entries j = 1..n).
 * Needs MPDET_LASTCOL and a completed factorisation.  After a zero pivot at
 * step kz (D_kz = 0) the series 1..kz are valid; later unnormalised series
 * are +0 and later normalised ones undefined.
 * With device_ptr = 0 the call allocates a device buffer of the triangle for
 * its duration.  Errors: MPDET_EINVAL, MPDET_ESTATE, MPDET_ENOMEM, MPDET_ECUDA. */
int mpdet_minor_series(mpdet_t h, mpdet_numv out, int normalised, int device_ptr);

/* Copy count entries of the in-place N x N array (flat row-major indices
 * idx[q] = i*N + j, host array, 0 <= idx < N^2) into out (count numbers):
 * sampled reads of a large factorisation without copying it whole.
 * Errors: MPDET_EINVAL (bad index or pointer), MPDET_ECUDA. */
int mpdet_get_entries(mpdet_t h, int64_t count, const int64_t* idx, mpdet_numv out, int device_ptr);

/* Radii of the ball mode (MPDET_BALL): which = 0 those of D_1..D_N (N
 * radii), 1 those of the last mpdet_lastcol_minors result (N radii), 2 those
 * of the in-place N x N array (N^2 radii).  rad_mant[i], rad_exp[i]: radius
 * i is rad_mant * 2^(rad_exp - 32) (0 when rad_mant = 0; unbounded when
 * rad_exp = INT64_MAX).  Synchronous unless device_ptr = 1.  Errors:
 * MPDET_EINVAL, MPDET_ESTATE (no ball mode), MPDET_ECUDA. */
int mpdet_radii(mpdet_t h, int which, uint32_t* rad_mant, int64_t* rad_exp, int device_ptr);

/* Copy out the leading minors computed so far (D_1..D_N; entries of steps not
 * yet run are +0).  Errors: MPDET_EINVAL (NULL handle), MPDET_ECUDA. */
int mpdet_get_minors(mpdet_t h, mpdet_numv out, int device_ptr);

/* Copy out the in-place N x N array (U in the upper triangle including the
 * diagonal; in MPDET_LASTCOL mode L's strict lower part below it; otherwise
 * the strict lower part is unspecified), e.g. to checkpoint a window.
 * Errors: MPDET_EINVAL (NULL handle), MPDET_ECUDA. */
int mpdet_get_mp(mpdet_t h, mpdet_numv out, int device_ptr);

/* Restore a checkpoint: the in-place array after k_done steps and the
 * leading minors D_1..D_{k_done} (N numbers, later entries ignored).  The
 * next mpdet_factor_range must start at k0 = k_done; the rest of the
 * elimination is the same rounded sequence as an uninterrupted one.
 * Errors: MPDET_EINVAL (NULL handle, k_done outside 0..N), MPDET_ESTATE (ball
 * mode: a checkpoint carries no radii), MPDET_ECUDA. */
int mpdet_resume(mpdet_t h, mpdet_numv A, mpdet_numv minors, int64_t k_done, int device_ptr);

/* Steps completed so far (0..N); -1 for a NULL handle. */
int64_t mpdet_steps_done(mpdet_t h);

/* Tuning knobs (results are identical for every setting; only speed
 * changes).  MPDET_TUNE_UPDATE_VARIANT selects the register budget of the
 * IMAD Schur-update kernel: value v in 0..3 compiles it for at least 3 + v
 * resident 128-thread blocks per SM.  MPDET_TUNE_ENGINE selects how the
 * update forms its products: 1 (default) on the tensor cores as an exact
 * digit convolution where an engine exists for p: at p = 512, 1024, 2048
 * 8-bit digits of both operands, warp-specialised so that the tensor core,
 * the rounding and the subtraction overlap; at p = 4096, 8192, 16384, 32768
 * 8-bit digits of the multiplier against 4-bit digits of the pivot-row
 * element (every column sum exact in fp32 over the whole mantissa), only the
 * upper half of each product formed when the lower half cannot change its
 * rounding, else that product recomputed exactly; 2 the p = 2048 engine one
 * phase at a time (p = 2048 only); 0 with IMAD limb products everywhere
 * (always for a p that runs in a larger frame, and in ball mode).  The
 * large-precision engine allocates, on its first use by a handle, N p / 4
 * bytes for the multipliers' digits and 32 p bytes per SM for staged products.
 * MPDET_TUNE_TC_MIN_ROWS (value >= 0): an update launch
 * of fewer rows than this takes the IMAD kernel even when the tensor engine is
 * selected (its tiles are 128 rows high).  By default the threshold follows the
 * precision: 64 rows at p = 1024, 2048 and 4096 .. 32768, and the IMAD kernel
 * always at p = 512, where it measured faster at every size.  MPDET_TUNE_LOOKAHEAD:
 * 1 (default) overlaps the pivot and multipliers of step k+1 with the update
 * of step k: a second stream owned by the handle updates column k+1 first and
 * runs them while the handle's stream updates the other columns; 0 runs each
 * step's kernels one after another on the handle's stream.
 * MPDET_TUNE_LOOKAHEAD_RESERVE (0..64, default 4): SMs the update of the
 * other columns leaves free for that second stream.
 * MPDET_TUNE_UPDATE_GEOMETRY: lane geometry of the IMAD update kernel: 0 the
 * precision's own (16 limbs per lane below p = 32768), 1 or 2 32 limbs per
 * lane (p = 2048 .. 16384) compiled for 4 or 3 resident blocks per SM, -1
 * (default) the one measured fastest for the precision.
 * MPDET_TUNE_KARATSUBA: 1 forms the IMAD update's products by one Karatsuba
 * level over three half-size schoolbook products (p = 8192, 16384, 32768;
 * the product is exact before it is rounded, so the bits are the same), 0
 * (default) the schoolbook product.  Ignored in ball mode and for
 * precisions held in a larger frame.
 * Errors: MPDET_EINVAL. */
enum {
  MPDET_TUNE_UPDATE_VARIANT = 1,
  MPDET_TUNE_ENGINE = 2,
  MPDET_TUNE_TC_MIN_ROWS = 3,
  MPDET_TUNE_LOOKAHEAD = 4,
  MPDET_TUNE_LOOKAHEAD_RESERVE = 5,
  MPDET_TUNE_UPDATE_GEOMETRY = 6,
  MPDET_TUNE_KARATSUBA = 7
};
int mpdet_tune(mpdet_t h, int param, int value);

/* Instrumentation (not part of the computation).  mpdet_profile(h, 1)
 * brackets every later Schur-update launch (step 2.2.2, the dominant kernel)
 * with a CUDA event pair on the handle's stream and resets the counters;
 * mpdet_profile(h, 0) stops.  mpdet_profile_read synchronises the stream and
 * returns the summed device time of those launches (ms), their number, their
 * algorithmic work in limb multiply-accumulates (products * n^2) and the
 * total number of kernels this handle has enqueued since creation.  Any
 * output pointer may be NULL.  Errors: MPDET_EINVAL (NULL handle),
 * MPDET_ECUDA. */
int mpdet_profile(mpdet_t h, int enable);
int mpdet_profile_read(mpdet_t h, double* update_ms, int64_t* update_launches, double* update_limb_macs,
                       int64_t* launches);

/* Factorisation that allocates no memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory, such as
 * host frameworks that give a plugin its buffers and forbid it allocations of
 * its own (the framework owns the memory budget), and latency-bound loops
 * that cannot take an allocation mid-step.
 *
 * It runs the same kernels and the same rounded operations as mpdet_factor
 * (results are bit-identical), with all working memory (the in-place matrix,
 * the multipliers, the reciprocal, the status words) in one static device
 * array of MPDET_NOALLOC_SCRATCH_BYTES bytes inside the library, which every
 * GPU that loads the library holds until the process exits.  That bounds the
 * problem size: N^2 (4n + 9) + N (4n + 9) + 4n + ~2.5 KB of padding <= 16 MiB
 * with n = p/32 (about N <= 478 at p = 512, N <= 251 at p = 2048); larger
 * problems return MPDET_ENOSCRATCH and should use mpdet_create.
 *
 * p must be one of the kernel families' sizes (a power of two, 128 <= p <=
 * 32768); other precisions return MPDET_EINVAL.
 *
 * Arguments (all device memory of the current device, 16-byte aligned):
 *   A       N*N numbers, row-major, read only (copied into the scratch);
 *   minors  N numbers, receives D_1..D_N (D_N = det);
 *   lastcol N numbers, receives C_1N..C_NN when flags has MPDET_LASTCOL
 *           (may be NULL pointers otherwise).
 * zero_pivot_k (host, may be NULL) and the return value are as for
 * mpdet_factor.  The call is enqueued on cuda_stream; it copies the status
 * words to the host and synchronises that stream before it returns.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call uses the same array and the array keeps the
 * previous call's contents; the call clears what has to start at zero.
 * Calls that overlap on the GPU (other threads or streams, another device's
 * calls excepted) race on the array and give undefined results.
 * Errors: MPDET_EINVAL, MPDET_ENOSCRATCH, MPDET_ECUDA, MPDET_EZEROPIVOT. */
#define MPDET_NOALLOC_SCRATCH_BYTES (16u << 20)
int mpdet_factor_noalloc(int64_t N, int32_t p_bits, uint32_t flags, mpdet_numv A, mpdet_numv minors,
                         mpdet_numv lastcol, int64_t* zero_pivot_k, void* cuda_stream);

/* ---- Adjoint (step a8) ----------------------------------------------------
 * All (N-1) x (N-1) minors are partial derivatives of the determinant (Sec.
 * 3, the Strassen argument), so d log|det| / dA = A^-T = C / det (cofactor
 * matrix over the determinant).  mpdet_logabsdet_grad lifts the binary64
 * matrix A (N x N, row-major, leading dimension ld) exactly to p bits, runs
 * the elimination in MPDET_LASTCOL mode (L A = U), returns log|det| and the
 * sign (host scalars; log|det| = ln(m/2^p) + e ln 2 in binary64; a zero
 * determinant gives -inf and sign 0) and, when grad != NULL, solves
 * X = U^-1 L = A^-1 at p bits by back substitution from the bottom row up:
 *     X_kc = RN(S_kc * RN(1/u_kk)), all c;  S_ic = RN(S_ic - RN(u_ik X_kc)), i < k
 * (S = L initially), and writes grad[i*N + j] = grad_scale * RN64(X_ji)
 * (binary64, nearest even, subnormals included).  Nothing is kept between
 * calls but the buffers: the factor is recomputed, not stored.
 * The handle must be created with MPDET_LASTCOL when grad != NULL.
 * device_ptr applies to A and grad; the call synchronises.
 * Errors: MPDET_EZEROPIVOT (zero pivot before N: no elimination without
 * pivoting), MPDET_EZERODIV (det = 0 and a gradient was asked for),
 * MPDET_ESTATE, MPDET_EINVAL, MPDET_ENOMEM, MPDET_ECUDA. */
int mpdet_logabsdet_grad(mpdet_t h, const double* A, int64_t ld, double* logabs, int* sign, double* grad,
                         double grad_scale, int device_ptr);

/* A^-1 (N*N numbers) from the last mpdet_logabsdet_grad call with a
 * gradient (before the binary64 rounding).  Errors: MPDET_ESTATE. */
int mpdet_get_inverse(mpdet_t h, mpdet_numv out, int device_ptr);

/* ---- Batches (step a7): many independent matrices of uneven N ------------
 * The paper needs the minors for a whole series of sizes N = 2, 3, ... and for
 * parameter sweeps (Sec. 1, Sec. 3); a batch factors many such matrices in
 * one persistent launch: 128-thread blocks take matrices from an atomic queue
 * ordered by decreasing N and run all of each matrix's steps (det and leading
 * minors; no L).  Every matrix's results equal mpdet_factor's bit for bit.
 *
 * mpdet_batch_create: count matrices of sizes Ns[0..count) (host) at p bits;
 *   allocates 2 sum(N_i^2) + sum(N_i) numbers plus per-block scratch.
 * mpdet_batch_set_*: input of matrix m (as mpdet_set_*); kept by the handle.
 *   Every matrix must be set before the first mpdet_batch_factor.
 * mpdet_batch_factor: eliminates a working copy of the stored inputs (one
 *   device-to-device copy and one persistent launch); minors receives
 *   sum(N_i) numbers, matrix m's D_1..D_{N_m} first at offset
 *   N_0 + .. + N_{m-1}; zero_k (count int64, may be NULL) the 1-based first
 *   zero pivot of each matrix or 0 (a zero pivot before N_m stops that
 *   matrix: its later minors are +0).  device_ptr as for mpdet_factor.
 * mpdet_batch_launches: kernels enqueued by the handle so far.
 * Errors: MPDET_EINVAL, MPDET_ENOMEM, MPDET_ECUDA. */
typedef struct mpdet_batch_ctx* mpdet_batch_t;
int mpdet_batch_create(int64_t count, const int64_t* Ns, int32_t p_bits, void* cuda_stream, mpdet_batch_t* out);
int mpdet_batch_set_f64(mpdet_batch_t b, int64_t m, const double* A, int64_t ld, int device_ptr);
int mpdet_batch_set_i32(mpdet_batch_t b, int64_t m, const int32_t* A, int64_t ld, int device_ptr);
int mpdet_batch_set_cauchy(mpdet_batch_t b, int64_t m, const double* x, const double* y, int device_ptr);
int mpdet_batch_set_mp(mpdet_batch_t b, int64_t m, mpdet_numv A, int device_ptr);
int mpdet_batch_factor(mpdet_batch_t b, mpdet_numv minors, int64_t* zero_k, int device_ptr);
int64_t mpdet_batch_launches(mpdet_batch_t b);

/* One-shot batch: create, set, factor and free in one call.  count matrices
 * of sizes Ns[0..count) at p bits, matrix m given as N_m * N_m numbers in[m]
 * (row-major, canonical); its leading minors D_1..D_{N_m} go to minors_out[m]
 * (N_m numbers) and the 1-based index of its first zero pivot (0 if none) to
 * status_out[m] (count int64, may be NULL).  device_ptr applies to every
 * buffer (all host or all device memory of the current device).  The device
 * memory of the batch is allocated and freed inside the call, which
 * synchronises cuda_stream; repeated factorisations of the same sizes should
 * keep a handle from mpdet_batch_create instead.  Results equal
 * mpdet_batch_factor's (and mpdet_factor's) bit for bit.
 * Errors: MPDET_EINVAL, MPDET_ENOMEM, MPDET_ECUDA. */
int mpdet_batch(int64_t count, const int64_t* Ns, int32_t p_bits, const mpdet_numv* in, mpdet_numv* minors_out,
                int64_t* status_out, int device_ptr, void* cuda_stream);

/* Batch tuning (results are bit-identical for every setting; only speed
 * changes).  The persistent kernel exists in several lane geometries per
 * precision: variant v runs the multipliers and the Schur update with W
 * limbs per lane and G lanes per number, the pivot with PW x PG
 * (mpdet_batch_variant_info; variant 0 is the default), and is launched with
 * a chosen number of resident blocks per SM (1 .. the occupancy limit).
 * mpdet_batch_tune params:
 *   MPDET_BATCH_VARIANT        value = variant index;
 *   MPDET_BATCH_BLOCKS_PER_SM  value = resident blocks per SM;
 *   MPDET_BATCH_GRAPH          1: mpdet_batch_factor with device outputs
 *     replays a CUDA graph of the whole factorisation (working copy, the
 *     persistent launch, the output copies), captured on the first call and
 *     again whenever the output pointers or the launch shape change; 0 (the
 *     default) enqueues the operations one by one.
 * mpdet_batch_autotune times every variant at its occupancy limit and at half
 * of it (reps factorisations each after one warm-up, CUDA events on the
 * batch's stream, on the stored inputs; synchronous), keeps the fastest and
 * returns it (any output pointer may be NULL): the variant, the blocks per
 * SM, its time per factorisation in ms and the number of candidates timed.
 * Every matrix must be set first.  Errors: MPDET_EINVAL, MPDET_ECUDA. */
enum { MPDET_BATCH_VARIANT = 1, MPDET_BATCH_BLOCKS_PER_SM = 2, MPDET_BATCH_GRAPH = 3 };
int mpdet_batch_tune(mpdet_batch_t b, int param, int value);
int mpdet_batch_variant_info(mpdet_batch_t b, int32_t variant, int32_t* W, int32_t* G, int32_t* PW, int32_t* PG,
                             int32_t* max_blocks_per_sm);
int mpdet_batch_autotune(mpdet_batch_t b, int reps, int32_t* variant, int32_t* blocks_per_sm, double* best_ms,
                         int32_t* candidates);
int mpdet_batch_free(mpdet_batch_t b);

/* Element-wise arithmetic of the kernels on device arrays of count numbers
 * (diagnostics and tests of the arithmetic core; the method's rounding rules):
 * op 0: out = RN(a*b), 1: RN(a-b), 2: RN(a+b), 3: RN(1/a) (b ignored; 1/0
 * gives +0).  All pointers are device memory; synchronises cuda_stream.
 * Errors: MPDET_EINVAL, MPDET_ECUDA. */
int mpdet_ops(int op, int64_t count, int32_t p_bits, mpdet_numv a, mpdet_numv b, mpdet_numv out, void* cuda_stream);

/* Schoolbook against Karatsuba (the paper's CPU runs use GMP, whose Karatsuba
 * multiply grows about 2.8x per doubling of the precision against 3.95x for
 * the GPU's schoolbook one, Sec. 4.2, Tables 1 and 2).  out[i] = RN(a[i] * b[i])
 * at p bits for count pairs (device memory of the current device, 16-byte
 * aligned), by the IMAD engine's lane-systolic schoolbook product (method 0,
 * the one the Schur update uses) or by one Karatsuba level over three
 * half-size schoolbook products (method 1); both give the same bits (the
 * product is exact before it is rounded).  Each product is formed reps times
 * on operands held on chip, so that *ms (the device time of the launch, CUDA
 * events on cuda_stream; may be NULL) measures the multiplication.  p = 8192,
 * 16384 or 32768.  Synchronises cuda_stream.  Errors: MPDET_EINVAL,
 * MPDET_ECUDA. */
int mpdet_mulbench(int method, int64_t count, int32_t p_bits, mpdet_numv a, mpdet_numv b, mpdet_numv out, int reps,
                   void* cuda_stream, float* ms);

/* Failure-detection self-test (the paper has no counterpart).  Every wait of
 * the kernels' hand-offs polls an mbarrier a bounded number of times and, when
 * the bound runs out, reports MPDET_ETIMEOUT through the handle's status word
 * and returns instead of hanging the GPU.  This call runs one such bounded
 * wait (at most `limit` polls, limit >= 1) in a one-block kernel on
 * cuda_stream, on a barrier that nothing completes (arrive = 0) or that the
 * block completes itself (arrive != 0, the control), and synchronises.
 * Returns MPDET_ETIMEOUT when the wait ran out, MPDET_OK when it completed;
 * the context stays usable either way.  Errors: MPDET_EINVAL, MPDET_ENOMEM,
 * MPDET_ECUDA. */
int mpdet_selftest_timeout(int32_t limit, int arrive, void* cuda_stream);

/* Release the handle and its device or host memory (NULL is accepted);
 * returns MPDET_OK. */
int mpdet_free(mpdet_t h);

/* Message for the last failing call on h (static string when h == NULL). */
const char* mpdet_last_error(mpdet_t h);

/* Limb count and slice geometry chosen for p: n = p/32, and the frame the
 * kernels hold a number in: W limbs per lane, G lanes per number (W * G >= n,
 * equal when n is a kernel family's size); returns MPDET_EINVAL for an
 * unsupported p. */
int mpdet_geometry(int32_t p_bits, int32_t* n, int32_t* W, int32_t* G);

#ifdef __cplusplus
}
#endif

#endif /* MPDET_H */
