// Dirichlet DST-I on the tensor cores (sm_103a: tcgen05 MMA, TMEM accumulators,
// bulk asynchronous copies).
//
// Step (b) of Eq. (3.3) is diagonal in L_h's eigenbasis; on a Dirichlet grid
// that basis is the orthonormal DST-I S (Sec. 3.1, L_h = V_h D_h V_h^{-1}), and
// the 2D transform of a slice is Y = S_y X S_x.  For sizes whose n + 1 is not a
// power of two it is a dense product.  Here it runs as split-BF16 products on
// the tensor cores with an exact float32 accumulation:
//
//  * every row of the left operand (a data row, or a row of S) is scaled by a
//    power of two 2^e with max|x| < 2^e and cut into k digits of 7 bits,
//    x = 2^e sum_{i=0}^{k-1} d_i 2^{-7(i+1)} (balanced digits, |d_0| <= 128,
//    |d_i| <= 64 for i > 0, rounded to nearest at the last one); every digit
//    is an integer, so it is exact in bf16.  The data rows carry one exponent
//    each, S one exponent for the whole matrix;
//  * the product of two digit matrices over K <= 1024 is a sum of integers of
//    at most 1024 * 128 * 128 = 2^24 in magnitude: the float32 accumulator of
//    the tensor core holds it exactly.  Pairs of one weight share an
//    accumulator while their bounds add up to at most 2^24 (tc_groups);
//  * the pairs (i, j) with i + j < k are summed with weights 2^{-7(i+j+2)} in
//    double-float (float hi + float lo) held in TMEM, then scaled by
//    2^{e_row + e_S} and rounded once to float64.
//
// The truncation leaves a relative error of about 2^{-7k} (k = 6: 2^{-42}), so
// the transform meets tolerances far below the float32 floor; the digit count
// follows the plan's tolerance.
//
// Two passes give the 2D transform: T_s = (X_s S_x)^T, then Y_s = (T_s S_y)^T.
// Each pass is C = A B^T with A = the slice rows (K contiguous) and B = S (its
// rows K contiguous; S is symmetric); the epilogue writes C transposed within
// each slice, which makes its stores coalesced (consecutive TMEM lanes are
// consecutive output addresses).
//
// Operand layout in global memory ("packed"): the split kernel writes every
// 128-row x 64-K tile as the 16 KB image the MMA reads from shared memory,
// K-major without swizzle: 8x8 core matrices of 128 contiguous bytes, the
// core matrix of row group g and K group c at byte (8 g + c) * 128.  One bulk
// copy moves a tile; no tensor map is needed.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <climits>
#include <cstring>
#include <string>

#include "common.cuh"
#include "dst_digits.cuh"
#include "tc_ptx.cuh"
#include "plan.h"

namespace {

using namespace expd_tc;

constexpr int TC_BM = 128;                          // rows per tile (TMEM lanes)
constexpr int TC_BK = 64;                           // K per stage (bf16: 128 bytes per row)
constexpr int TC_TILE_ELEMS = TC_BM * TC_BK;        // 8192 bf16 per packed operand tile (128 rows)
constexpr int TC_TILE_BYTES = TC_TILE_ELEMS * 2;    // 16 KB
constexpr int TC_NACC = 2;                          // accumulator buffers of BN columns
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // every wait gives up after 2 s

// Tile shapes: BN = 128 output columns per tile (the default) or 64 (twice the
// tiles, for transforms too small to give every SM a 128-column tile; a
// plan selects it with EXPD_KF_DST_N64).  A stage holds SK 128 x 64 A tiles
// and SK BN x 64 B tiles; TMEM holds acc[0], acc[1], hi and lo, BN columns each.
// SK: 64-K tile pairs per stage -- 2 for the 128-column tiles (one 32 KB A
// image and one 32 KB B image of 128 K, eight MMAs per stage: half the stage
// hand-offs of the copy and MMA threads per MMA; their B tiles are contiguous
// along K and their K-tile count is even), 1 for the 64-column tiles.
template <int BN, int SK = 1>
struct TcShape {
    static constexpr int B_BYTES = BN * TC_BK * 2;
    static constexpr int STAGE_BYTES = SK * (TC_TILE_BYTES + B_BYTES);
    static constexpr int STAGES = SK == 2 ? 3 : (BN == 128 ? 6 : 8);
    static constexpr int TMEM_COLS = 4 * BN;
    // drain warps: BN / 32 per TMEM lane quarter, 32 columns each (warp 0
    // copies, warp 1 issues the MMAs, warps 2.. drain); enough warps that one's
    // TMEM loads overlap another's double-float sums
    static constexpr int EPI = BN / 8;
    static constexpr int THREADS = 32 * (2 + EPI);
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 256 + 1024;
    // kind::f16 instruction descriptor: D float32 (bits 4-5 = 1), A and B bf16
    // (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit
    // 17, M >> 4 at bit 24.
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(TC_BM >> 4) << 24);
};
static_assert(TcShape<64>::SMEM <= 232448 && TcShape<128, 2>::SMEM <= 232448, "stage ring within 227 KB");

struct TcArgs {
    const uint16_t* A;        // packed digit slices of the rows: [nsl][rows/128][KB][8192]
    const uint16_t* B;        // packed digit slices of S:         [nsl][N/128][KB][8192]
    const int* ea;            // [rows] row exponents of A
    int eb;                   // exponent of S: max|S| < 2^eb (one for all its rows)
    double* out;              // [rows / R][N][R]: C transposed within each slice
    long long a_slice;        // elements per digit slice of A (rows * K)
    long long b_slice;        // elements per digit slice of B (N padded to whole 128-row tiles, times K)
    int rows, R, N, KB;       // rows (multiple of 128), rows per slice, columns, K / 64
    int npairs, ngroups;
    unsigned char pi[32], pj[32];  // digit pair (i, j), 0-based, most significant first
    // pairs gstart[q] .. gstart[q+1]-1 share one float32 accumulator (the sum of
    // their products stays within 2^24); gw[q] = i + j of the group's pairs
    unsigned char gstart[33], gw[32];
    int* err;                 // set to 1 when a pipeline wait gave up
    const volatile int* cancel;  // mapped host word: nonzero asks every wait to give up at once
    // folded transforms: a second product of the same shape (A2 B2^T, the odd
    // rows of S against the differences), and the output column map: column c
    // of product q goes to output column c * ocs + q of Nout
    const uint16_t* A2;
    const uint16_t* B2;
    int nprob, ocs, Nout;
};

// The waits of the issuing threads: one try inline (the phase is usually
// complete already), the bounded loop of mbar_wait only when it is not.
__device__ __forceinline__ bool mbar_wait_fast(uint32_t bar, uint32_t parity, const volatile int* abort,
                                               const volatile int* cancel);

// Waits for the phase of the given parity; gives up after TC_WAIT_NS, when
// another role of the CTA has given up (abort != 0) or when the host cancels
// the call (cancel != 0, read from mapped host memory every 1024 tries);
// ignore_abort (the clean-up waits) heeds neither flag, only the time limit.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort,
                                       const volatile int* cancel, bool ignore_abort = false) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (!ignore_abort && *abort) return false;
            if (!ignore_abort && cancel && (it & 1023) == 0 && *cancel) return false;
            if (globaltimer() - t0 > TC_WAIT_NS) return false;
        }
    }
}

__device__ __forceinline__ bool mbar_wait_fast(uint32_t bar, uint32_t parity, const volatile int* abort,
                                               const volatile int* cancel) {
    return mbar_try_wait(bar, parity) || mbar_wait(bar, parity, abort, cancel);
}

// 16-column variants for the drain (half the registers of the 32-column forms)
__device__ __forceinline__ void tm_ld16x3(uint32_t ta, uint32_t th, uint32_t tl, uint32_t (&a)[16], uint32_t (&h)[16],
                                          uint32_t (&l)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%48];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%49];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47}, [%50];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]), "=r"(h[7]), "=r"(h[8]), "=r"(h[9]), "=r"(h[10]), "=r"(h[11]), "=r"(h[12]), "=r"(h[13]), "=r"(h[14]), "=r"(h[15]), "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]), "=r"(l[7]), "=r"(l[8]), "=r"(l[9]), "=r"(l[10]), "=r"(l[11]), "=r"(l[12]), "=r"(l[13]), "=r"(l[14]), "=r"(l[15])
        : "r"(ta), "r"(th), "r"(tl)
        : "memory");
}
__device__ __forceinline__ void tm_ld16x2(uint32_t th, uint32_t tl, uint32_t (&h)[16], uint32_t (&l)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%33];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]), "=r"(h[7]), "=r"(h[8]), "=r"(h[9]), "=r"(h[10]), "=r"(h[11]), "=r"(h[12]), "=r"(h[13]), "=r"(h[14]), "=r"(h[15]), "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]), "=r"(l[7]), "=r"(l[8]), "=r"(l[9]), "=r"(l[10]), "=r"(l[11]), "=r"(l[12]), "=r"(l[13]), "=r"(l[14]), "=r"(l[15])
        : "r"(th), "r"(tl)
        : "memory");
}
__device__ __forceinline__ void tm_ld16(uint32_t ta, uint32_t (&a)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15])
        : "r"(ta)
        : "memory");
}
__device__ __forceinline__ void tm_st16x2(uint32_t th, uint32_t tl, const uint32_t (&h)[16], const uint32_t (&l)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%1], {%18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33};\n\t"
        "tcgen05.wait::st.sync.aligned;"
        :
        : "r"(th), "r"(tl), "r"(h[0]), "r"(h[1]), "r"(h[2]), "r"(h[3]), "r"(h[4]), "r"(h[5]), "r"(h[6]), "r"(h[7]), "r"(h[8]), "r"(h[9]), "r"(h[10]), "r"(h[11]), "r"(h[12]), "r"(h[13]), "r"(h[14]), "r"(h[15]), "r"(l[0]), "r"(l[1]), "r"(l[2]), "r"(l[3]), "r"(l[4]), "r"(l[5]), "r"(l[6]), "r"(l[7]), "r"(l[8]), "r"(l[9]), "r"(l[10]), "r"(l[11]), "r"(l[12]), "r"(l[13]), "r"(l[14]), "r"(l[15])
        : "memory");
}

// ------------------------------------------------------------ split rows ----
// float value of a small integer d (|d| < 2^22) without the conversion unit:
// 1.5 * 2^23 + d has d in its low mantissa bits
__device__ __forceinline__ uint32_t bf16_of_int(int d) {
    return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
}

// Eight rows of K float64 values (row r at in + r lda) per CTA of 256 threads
// (K a multiple of 64, rows a multiple of 8): first every warp finds its row's exponent e
// (max|x| < 2^e, or fixed_e for every row unless it is INT_MIN) into ex[r]
// (when ex is given); then thread t splits chunk t / 8 (eight values) of row
// t % 8 into nsl balanced 7-bit digits of x 2^{-e}, digit 0 the most
// significant.  The eight rows of a chunk form one 128-byte row of 8x8 core
// matrices in the packed layout and a warp covers four consecutive core
// matrices, so every digit slice is written in contiguous 512-byte runs.  All
// arithmetic is on the binary64 encoding (integer operations); a row holding a
// non-finite value gets NaN digits.
__global__ void __launch_bounds__(256) split_rows_kernel(const double* __restrict__ in, long long rows, int K,
                                                         long long lda, int nsl, uint16_t* __restrict__ out,
                                                         long long slice_elems, int* __restrict__ ex, int fixed_e) {
    __shared__ int se[8], sbad[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long r0 = (long long)blockIdx.x * 8;
    {
        const long long r = r0 + warp;
        int e = 0, bad = 0;
        if (r < rows) {
            const double2* x = reinterpret_cast<const double2*>(in + r * lda);
            unsigned long long mx = 0;
            for (int c = lane; c < (K >> 1); c += 32) {
                const double2 v = __ldg(x + c);
                mx = max(mx, (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull);
                mx = max(mx, (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            bad = (mx >> 52) == 2047;
            e = fixed_e != INT_MIN ? fixed_e : digit_row_exponent(mx);
            if (lane == 0 && ex) ex[r] = bad ? 0 : e;
        }
        if (lane == 0) {
            se[warp] = e;
            sbad[warp] = bad;
        }
    }
    __syncthreads();
    const int rr = threadIdx.x & 7;
    const long long r = r0 + rr;
    if (r >= rows) return;
    const int e = se[rr];
    const bool bad = sbad[rr] != 0;
    const double2* x = reinterpret_cast<const double2*>(in + r * lda);
    const int KB = K >> 6;
    const unsigned long long off = digit_offset(nsl);
    const int nch = K >> 3;  // chunks of 8 values (16 bytes of bf16 per digit slice)
    for (int c = threadIdx.x >> 3; c < nch; c += 32) {
        unsigned long long Y[8];
        unsigned neg = 0;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const double2 v = __ldg(x + 4 * c + h);
            unsigned n0, n1;
            Y[2 * h] = digit_magnitude((unsigned long long)__double_as_longlong(v.x), e, nsl, &n0);
            Y[2 * h + 1] = digit_magnitude((unsigned long long)__double_as_longlong(v.y), e, nsl, &n1);
            neg |= (n0 << (2 * h)) | (n1 << (2 * h + 1));
        }
        // the 8 values' 16 bytes of each digit slice (same 8x8 core matrix row)
        uint16_t* o = out + packed_offset(r, 8 * c, KB);
#pragma unroll
        for (int t = 0; t < 8; ++t) Y[t] += off;
        for (int i = nsl - 1; i >= 0; --i) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                int d = digit_at(Y[t], i, nsl);
                if ((neg >> t) & 1u) d = -d;
                const uint32_t hb = bad ? 0x7FC0u : bf16_of_int(d);
                w[t >> 1] |= hb << (16 * (t & 1));
            }
            *reinterpret_cast<uint4*>(o + (long long)i * slice_elems) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Folded rows for the symmetric half of the DST-I: S[j][n-1-k] = (-1)^j S[j][k]
// (sin(pi (j+1)(n-k)/(n+1)) = (-1)^j sin(pi (j+1)(k+1)/(n+1))), so output j of
// a row x is sum_{k < n/2} S[j][k] (x_k + (-1)^j x_{n-1-k}) for even n.  Eight
// rows of n float64 values per CTA: the row exponent e over all n values (as
// split_rows_kernel), then thread t takes chunk t / 8 (eight values, k =
// 8c..8c+7) of row t % 8 and its mirror (x_{n-1-k}), cuts both into digits with
// the row's exponent and writes the digit sums (to u) and differences (to v):
// integers with |d_0| <= 256 and |d_i| <= 128, exact in bf16; a product of
// n/2 of them with S's digits sums to at most (n/2) 256 128 = 2^24 for n =
// 1024, the bound of the unfolded product, so the same accumulator groups
// hold them exactly.
//
// STAGED: the CTA's rows come into shared memory by one bulk copy each (row
// stride n + 2 values, so that the eight rows a warp reads in the digit pass
// fall on distinct banks) and both passes read them there: every value leaves
// HBM once, with the CTA's whole 64 KB (n = 1024) in flight at a time.
// Otherwise (rows too long to stage) both passes read global memory.  Both
// read 16-byte vectors: the rows start 16-byte aligned (the caller checks).
template <bool STAGED>
__global__ void __launch_bounds__(256) split_fold_kernel(const double* __restrict__ in, long long rows, int n,
                                                         int nsl, uint16_t* __restrict__ out_u,
                                                         uint16_t* __restrict__ out_v, long long slice_elems,
                                                         int* __restrict__ ex, int* __restrict__ err) {
    __shared__ int se[8], sbad[8];
    __shared__ __align__(8) uint64_t sbar;
    extern __shared__ __align__(16) double srows[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long r0 = (long long)blockIdx.x * 8;
    const int stride = n + 2;
    auto row = [&](int rr) -> const double* { return STAGED ? srows + (size_t)rr * stride : in + (r0 + rr) * n; };
    if constexpr (STAGED) {
        const uint32_t bar = smem_u32(&sbar);
        const int nr = (int)min(8LL, rows - r0);
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(bar, (uint32_t)(nr * n * 8));
            for (int i = 0; i < nr; ++i) bulk_g2s(smem_u32(srows + (size_t)i * stride), in + (r0 + i) * n, (uint32_t)n * 8u, bar);
        }
        __syncthreads();
        // a copy that has not landed after 2 s: flagged, the CTA leaves
        bool done = mbar_try_wait(bar, 0);
        if (!done) {
            const uint64_t t0 = globaltimer();
            for (uint32_t it = 1; !done; ++it) {
                done = mbar_try_wait(bar, 0);
                if (!done && (it & 63) == 0 && globaltimer() - t0 > TC_WAIT_NS) break;
            }
        }
        if (!__syncthreads_and(done)) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            return;
        }
    }
    {
        const long long r = r0 + warp;
        int e = 0, bad = 0;
        if (r < rows) {
            const double2* x = reinterpret_cast<const double2*>(row(warp));
            unsigned long long mx = 0;
            for (int c = lane; c < (n >> 1); c += 32) {
                const double2 v = x[c];
                mx = max(mx, (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull);
                mx = max(mx, (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            bad = (mx >> 52) == 2047;
            e = digit_row_exponent(mx);
            if (lane == 0 && ex) ex[r] = bad ? 0 : e;
        }
        if (lane == 0) {
            se[warp] = e;
            sbad[warp] = bad;
        }
    }
    __syncthreads();
    const int rr = threadIdx.x & 7;
    const long long r = r0 + rr;
    if (r >= rows) return;
    const int e = se[rr];
    const bool bad = sbad[rr] != 0;
    const double* x = row(rr);
    const int K = n >> 1, KB = K >> 6;
    const unsigned long long off = digit_offset(nsl);
    const int nch = K >> 3;
    for (int c = threadIdx.x >> 3; c < nch; c += 32) {
        unsigned long long Y[8], Z[8];
        unsigned neg = 0, negz = 0;
        const double2* xa = reinterpret_cast<const double2*>(x + 8 * c);
        const double2* xb = reinterpret_cast<const double2*>(x + n - 8 * c - 8);  // x_{n-1-k} for k = 8c+7 .. 8c
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const double2 v = xa[h], w = xb[h];
            unsigned n0, n1, m0, m1;
            Y[2 * h] = digit_magnitude((unsigned long long)__double_as_longlong(v.x), e, nsl, &n0);
            Y[2 * h + 1] = digit_magnitude((unsigned long long)__double_as_longlong(v.y), e, nsl, &n1);
            neg |= (n0 << (2 * h)) | (n1 << (2 * h + 1));
            // w.x = x_{n-8c-8+2h} pairs with k = 8c + 7 - 2h, w.y with k = 8c + 6 - 2h
            Z[7 - 2 * h] = digit_magnitude((unsigned long long)__double_as_longlong(w.x), e, nsl, &m0);
            Z[6 - 2 * h] = digit_magnitude((unsigned long long)__double_as_longlong(w.y), e, nsl, &m1);
            negz |= (m0 << (7 - 2 * h)) | (m1 << (6 - 2 * h));
        }
        uint16_t* ou = out_u + packed_offset(r, 8 * c, KB);
        uint16_t* ov = out_v + packed_offset(r, 8 * c, KB);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            Y[t] += off;
            Z[t] += off;
        }
        for (int i = nsl - 1; i >= 0; --i) {
            uint32_t wu[4] = {0u, 0u, 0u, 0u}, wv[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                int d = digit_at(Y[t], i, nsl);
                if ((neg >> t) & 1u) d = -d;
                int dz = digit_at(Z[t], i, nsl);
                if ((negz >> t) & 1u) dz = -dz;
                const uint32_t hu = bad ? 0x7FC0u : bf16_of_int(d + dz);
                const uint32_t hv = bad ? 0x7FC0u : bf16_of_int(d - dz);
                wu[t >> 1] |= hu << (16 * (t & 1));
                wv[t >> 1] |= hv << (16 * (t & 1));
            }
            *reinterpret_cast<uint4*>(ou + (long long)i * slice_elems) = make_uint4(wu[0], wu[1], wu[2], wu[3]);
            *reinterpret_cast<uint4*>(ov + (long long)i * slice_elems) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
    }
}

// f 2^E as a float64 from the float's encoding (integer operations); false
// when f is zero, subnormal, non-finite or the result leaves the normal range
__device__ __forceinline__ bool f32_scaled_to_f64(float f, int E, double* out) {
    const uint32_t u = __float_as_uint(f);
    const int ex = (int)((u >> 23) & 0xFFu);
    if (ex == 0 || ex == 255) return false;
    const int ne = ex - 127 + 1023 + E;
    if (ne < 1 || ne > 2046) return false;
    *out = __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | ((unsigned long long)ne << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
    return true;
}

// zeros, non-finite values, range edges
__device__ __noinline__ double scaled_sum_edge(float hi, float lo, int E) { return ldexp((double)hi + (double)lo, E); }

// (hi + lo) 2^E rounded once to float64: both terms scaled exactly, one add
__device__ __forceinline__ double scaled_sum(float hi, float lo, int E) {
    double dh, dl;
    const bool okh = f32_scaled_to_f64(hi, E, &dh) || hi == 0.0f;
    const bool okl = f32_scaled_to_f64(lo, E, &dl) || lo == 0.0f;
    if (okh && okl) return (hi == 0.0f ? 0.0 : dh) + (lo == 0.0f ? 0.0 : dl);
    return scaled_sum_edge(hi, lo, E);
}

// ---------------------------------------------------------- MMA kernel ----
// Persistent: each CTA takes tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// (column tile fastest, so the CTAs running together share their A tiles in
// L2).  Per tile and digit pair, K / 64 stages of one A and one B tile flow
// through a TC_STAGES-deep ring: warp 0 (one lane) issues their bulk copies,
// warp 1 (one lane) the four K = 16 MMAs per stage into accumulator buffer
// group % 2 (a group: digit pairs of one weight whose products sum exactly in
// float32), and warps 2..9 drain the finished buffer into the double-float sum
// in TMEM while the next group accumulates.  After a tile's last group the
// drain warps write the float64 result.
template <int BN, int SK>
__global__ void __launch_bounds__(TcShape<BN, SK>::THREADS, 1) dst_mma_kernel(const __grid_constant__ TcArgs a) {
    typedef TcShape<BN, SK> SH;
    constexpr int TC_STAGES = SH::STAGES;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (size_t)TC_STAGES * SH::STAGE_BYTES);
    // full[s], empty[s], accf[b], acce[b], drain
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(TC_STAGES + s); };
    auto accf = [&](int b) { return bar0 + 8u * (uint32_t)(2 * TC_STAGES + b); };
    auto acce = [&](int b) { return bar0 + 8u * (uint32_t)(2 * TC_STAGES + TC_NACC + b); };
    const uint32_t drain = bar0 + 8u * (uint32_t)(2 * TC_STAGES + 2 * TC_NACC);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES + 2 * TC_NACC + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < TC_NACC; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), SH::EPI);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tc_alloc(smem_u32(tmem_slot), SH::TMEM_COLS);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int nct = a.N / BN;
    const int npc = a.nprob * nct;  // tiles per row tile: the products' column tiles
    const long long ntiles = (long long)(a.rows / TC_BM) * npc;
    const int KB = a.KB;

    if (warp == 0) {
        if (lane == 0) {
            // ---- copies ----
            uint32_t it = 0, cph = 0;  // stages issued; the ring's current stage and phase
            int cs = 0;
            const uint32_t sm0 = smem_u32(sm);
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const long long rt = t / npc;
                const int pc_ = (int)(t - rt * npc), q = pc_ / nct, ct = pc_ - q * nct;
                // B: packed 128-row tiles; a 64-column tile is the lower or
                // upper half (row groups 0-7 or 8-15: the first or second 8 KB)
                const long long boff = (long long)(ct * BN / 128) * KB * TC_TILE_ELEMS + (long long)((ct * BN) % 128) * TC_BK;
                const uint16_t* Aq = q ? a.A2 : a.A;
                const uint16_t* Bq = q ? a.B2 : a.B;
                for (int p = 0; p < a.npairs && ok; ++p) {
                    const uint16_t* Ab = Aq + a.pi[p] * a.a_slice + rt * KB * TC_TILE_ELEMS;
                    const uint16_t* Bb = Bq + a.pj[p] * a.b_slice + boff;
                    for (int kb = 0; kb < KB; kb += SK, ++it) {
                        if (!mbar_wait_fast(empty(cs), cph ^ 1u, abort_flag, a.cancel)) {
                            ok = false;
                            break;
                        }
                        // SK consecutive K tiles: contiguous in the packed images
                        const uint32_t st = sm0 + (uint32_t)cs * SH::STAGE_BYTES, fb = full(cs);
                        mbar_arrive_expect_tx(fb, SH::STAGE_BYTES);
                        bulk_g2s(st, Ab + (long long)kb * TC_TILE_ELEMS, SK * TC_TILE_BYTES, fb);
                        bulk_g2s(st + SK * TC_TILE_BYTES, Bb + (long long)kb * TC_TILE_ELEMS, SK * SH::B_BYTES, fb);
                        if (++cs == TC_STAGES) {
                            cs = 0;
                            cph ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(a.err, 1);
            }
            // copies still in flight land before the CTA leaves: the last one
            // issued into each stage completes that stage's phase
            for (uint32_t q = it > (uint32_t)TC_STAGES ? it - TC_STAGES : 0u; q < it; ++q)
                mbar_wait(full((int)(q % TC_STAGES)), (q / TC_STAGES) & 1u, abort_flag, nullptr, true);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMAs ----
            uint32_t it = 0, pc = 0, cph = 0;
            int cs = 0;
            const uint64_t desc0 = smem_desc(smem_u32(sm));  // stage 0's A tile; other stages by address
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int g = 0; g < a.ngroups && ok; ++g, ++pc) {
                    const int b = (int)(pc % TC_NACC);
                    if (!mbar_wait(acce(b), ((pc / TC_NACC) & 1u) ^ 1u, abort_flag, a.cancel)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(b * BN);
                    for (int p = a.gstart[g]; p < a.gstart[g + 1] && ok; ++p) {
                        const bool first = p == a.gstart[g];
                        for (int kb = 0; kb < KB; kb += SK, ++it) {
                            if (!mbar_wait_fast(full(cs), cph, abort_flag, a.cancel)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            // descriptors of the stage's A and B tiles; 16 bf16 of K =
                            // two core matrices = 256 bytes = 16 in the address field
                            const uint64_t da = desc0 + (uint64_t)(cs * (SH::STAGE_BYTES >> 4));
                            const uint64_t db = da + (uint64_t)((SK * TC_TILE_BYTES) >> 4);
#pragma unroll
                            for (int j = 0; j < SK; ++j)
#pragma unroll
                                for (int q = 0; q < TC_BK / 16; ++q)
                                    tc_mma(d, da + (uint64_t)(j * (TC_TILE_BYTES >> 4)) + 16u * q,
                                           db + (uint64_t)(j * (SH::B_BYTES >> 4)) + 16u * q, SH::IDESC,
                                           !first || (kb | j | q) != 0);
                            tc_commit(empty(cs));
                            if (++cs == TC_STAGES) {
                                cs = 0;
                                cph ^= 1u;
                            }
                        }
                    }
                    if (ok) tc_commit(accf(b));
                }
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(a.err, 1);
            }
            // every MMA issued has completed before TMEM is released
            tc_commit(drain);
            mbar_wait(drain, 0u, abort_flag, nullptr, true);
        }
    } else {
        // ---- drain and output (warps 2..): TMEM lane quarter warp % 4, columns
        // 32 (warp - 2) / 4 .. + 31; the double-float sums in TMEM columns
        // 2 BN .. 4 BN - 1 ----
        const int lq = warp & 3, half = (warp - 2) >> 2;
        const uint32_t tl = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(half * 32);
        const uint32_t thi = tl + 2u * BN, tlo = tl + 3u * BN;
        uint32_t pc = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const long long rt = t / npc;
            const int pc_ = (int)(t - rt * npc), q = pc_ / nct, ct = pc_ - q * nct;
            for (int g = 0; g < a.ngroups && ok; ++g, ++pc) {
                const int b = (int)(pc % TC_NACC);
                // every lane waits; the warp goes on only together (the TMEM
                // loads and stores below are warp-collective)
                if (!__all_sync(0xffffffffu, mbar_wait(accf(b), (pc / TC_NACC) & 1u, abort_flag, a.cancel))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // weight 2^{-7(i+j+2)} of the group's pairs (digits are 0-based)
                const float wsc = __int_as_float((127 - 7 * (a.gw[g] + 2)) << 23);
                const uint32_t tacc = tl + (uint32_t)(b * BN);
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {  // two 16-column halves of the warp's 32 columns
                    uint32_t v[16], h[16], l[16];
                    if (g == 0) {
                        tm_ld16(tacc + 16u * c, v);
                    } else {
                        tm_ld16x3(tacc + 16u * c, thi + 16u * c, tlo + 16u * c, v, h, l);
                    }
                    if (c == 1) {  // the accumulator buffer is free for the group after next
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acce(b));
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float w = __fmul_rn(__uint_as_float(v[e]), wsc);  // exact: a power of two
                        if (g == 0) {
                            h[e] = __float_as_uint(w);
                            l[e] = 0u;
                        } else {
                            // (hi, lo) += w: two-sum, error into lo, renormalise
                            const float hi = __uint_as_float(h[e]), lo = __uint_as_float(l[e]);
                            const float sm_ = __fadd_rn(hi, w);
                            const float bb = __fsub_rn(sm_, hi);
                            const float er = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm_, bb)), __fsub_rn(w, bb));
                            const float l1 = __fadd_rn(lo, er);
                            const float h1 = __fadd_rn(sm_, l1);
                            h[e] = __float_as_uint(h1);
                            l[e] = __float_as_uint(__fsub_rn(l1, __fsub_rn(h1, sm_)));
                        }
                    }
                    tm_st16x2(thi + 16u * c, tlo + 16u * c, h, l);
                }
            }
            if (!ok) break;
            // ---- output: C[row][col] = (hi + lo) 2^{ea[row] + eb}, transposed within the slice ----
            const long long row = rt * TC_BM + lq * 32 + lane;
            const long long slc = row / a.R;
            const int rin = (int)(row - slc * a.R);
            const int E = a.ea[row] + a.eb;
            const long long ostep = (long long)a.ocs * a.R;
            double* o = a.out + slc * (long long)a.R * a.Nout + (long long)(ct * BN + half * 32) * ostep +
                        (long long)q * a.R + rin;
#pragma unroll 1
            for (int c = 0; c < 2; ++c) {
                uint32_t h[16], l[16];
                tm_ld16x2(thi + 16u * c, tlo + 16u * c, h, l);
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    o[(long long)(16 * c + e) * ostep] = scaled_sum(__uint_as_float(h[e]), __uint_as_float(l[e]), E);
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(a.err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tc_dealloc(tmem, SH::TMEM_COLS);
    }
}

}  // namespace

// ------------------------------------------------------------------ host ----
namespace {

expd_status tc_dalloc(expd_plan p, void** ptr, size_t bytes, const char* what) {
    *ptr = nullptr;
    cudaError_t e = plan_malloc(p, ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return expd_fail(EXPD_ERR_OOM, std::string("cudaMalloc failed for ") + what + " (" + std::to_string(bytes) +
                                           " bytes): " + cudaGetErrorString(e));
    }
    p->bytes += bytes;
    return EXPD_OK;
}

expd_status split_rows(expd_plan p, const double* in, long long rows, int K, long long lda, uint16_t* out,
                       long long slice_elems, int* ex, int fixed_e, cudaStream_t s) {
    const int nsl = p->tc_nsl;
    // the kernel reads 16-byte vectors: every row starts 16-byte aligned
    if (reinterpret_cast<uintptr_t>(in) % 16 != 0 || lda % 2 != 0 || K % 2 != 0)
        return expd_fail(EXPD_ERR_INVALID_ARG, "digit split: rows must start 16-byte aligned");
    KProf kp(p, s, EXPD_K_DST_SPLIT, (double)rows * K * (8.0 + 2.0 * nsl) + 4.0 * rows, 0.0);
    split_rows_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(in, rows, K, lda, nsl, out, slice_elems, ex, fixed_e);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

// rows of n values -> digit sums (u) and differences (v) of mirrored halves
expd_status split_fold(expd_plan p, const double* in, long long rows, int n, uint16_t* out_u, uint16_t* out_v,
                       long long slice_elems, int* ex, cudaStream_t s) {
    const int nsl = p->tc_nsl;
    KProf kp(p, s, EXPD_K_DST_SPLIT, (double)rows * n * (8.0 + 2.0 * nsl) + 4.0 * rows, 0.0);
    if (reinterpret_cast<uintptr_t>(in) % 16 != 0 || n % 2 != 0)
        return expd_fail(EXPD_ERR_INVALID_ARG, "folded digit split: rows must start 16-byte aligned");
    const unsigned grid = (unsigned)((rows + 7) / 8);
    const size_t staged = (size_t)8 * (n + 2) * sizeof(double);
    if (staged <= 232448 - 1024) {
        EXPD_CUDA_TRY(smem_allow((const void*)split_fold_kernel<true>, staged));
        split_fold_kernel<true><<<grid, 256, staged, s>>>(in, rows, n, nsl, out_u, out_v, slice_elems, ex, p->tc_err);
    } else {
        split_fold_kernel<false><<<grid, 256, 0, s>>>(in, rows, n, nsl, out_u, out_v, slice_elems, ex, p->tc_err);
    }
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

// out (transposed within slices of R rows) = A B^T over the plan's digit pairs;
// folded (A2, B2 given): out's even columns A B^T, its odd ones A2 B2^T, each
// product N = K wide with digit sums of twice the unfolded bound (kbound = 2 K)
expd_status mma_pass(expd_plan p, const uint16_t* A, const int* ea, long long rows, int R, const uint16_t* B,
                     int eb, int N, int K, double* out, cudaStream_t s, const uint16_t* A2 = nullptr,
                     const uint16_t* B2 = nullptr) {
    TcArgs a = {};
    const bool fold = A2 != nullptr;
    a.A = A;
    a.B = B;
    a.A2 = fold ? A2 : A;
    a.B2 = fold ? B2 : B;
    a.nprob = fold ? 2 : 1;
    a.ocs = fold ? 2 : 1;
    a.Nout = fold ? 2 * N : N;
    a.ea = ea;
    a.eb = eb;
    a.out = out;
    a.a_slice = rows * K;
    a.b_slice = digit_rows(N) * K;
    a.rows = (int)rows;
    a.R = R;
    a.N = N;
    a.KB = K / TC_BK;
    const int nsl = p->tc_nsl;
    int np = 0, ng = 0;
    tc_groups(nsl, fold ? 2 * K : K, &np, &ng, a.pi, a.pj, a.gstart, a.gw);
    a.npairs = np;
    a.ngroups = ng;
    a.err = p->tc_err;
    a.cancel = p->cancel_dev;
    const int bn = (p->kernel_flags & EXPD_KF_DST_N64) || N % 128 != 0 ? 64 : 128;
    const long long ntiles = (rows / TC_BM) * (N / bn) * a.nprob;
    const int grid = (int)std::min<long long>(ntiles, (long long)p->sm_count);
    KProf kp(p, s, EXPD_K_DST_TC, a.nprob * 2.0 * nsl * ((double)rows * K + (double)N * K) + 8.0 * rows * a.Nout,
             a.nprob * 2.0 * np * (double)rows * N * K);
    if (bn == 64) {
        EXPD_CUDA_TRY(smem_allow((const void*)dst_mma_kernel<64, 1>, TcShape<64>::SMEM));
        dst_mma_kernel<64, 1><<<grid, TcShape<64>::THREADS, TcShape<64>::SMEM, s>>>(a);
    } else {
        // N = K in every pass (the products are square), so a 128-column tile
        // means K a multiple of 128: an even K-tile count, two per stage
        if (a.KB % 2 != 0) return expd_fail(EXPD_ERR_INVALID_ARG, "tensor-core DST: odd K-tile count for 128-column tiles");
        EXPD_CUDA_TRY(smem_allow((const void*)dst_mma_kernel<128, 2>, TcShape<128, 2>::SMEM));
        dst_mma_kernel<128, 2><<<grid, TcShape<128, 2>::THREADS, TcShape<128, 2>::SMEM, s>>>(a);
    }
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

// smallest e with sqrt(2 / (n + 1)) < 2^e: a bound on every entry of the
// orthonormal DST-I matrix of size n
int dst_exponent(int n) {
    int e;
    frexp(std::sqrt(2.0 / (n + 1)), &e);  // 2^(e-1) <= v < 2^e
    return e;
}

int tc_slices_for(double tol) {
    // digits of 7 bits; the transform's relative error is about 2^{-7 k}
    // times a small factor (the host emulation measures below 4, on rows of
    // uneven scale), kept 2^3 below the tolerance
    const double bits = -std::log2(std::max(tol, 1e-30)) + 3.0;
    return std::min(7, std::max(3, (int)std::ceil(bits / 7.0)));
}

}  // namespace

bool dst_tc_eligible(expd_plan p) {
    if (p->bc != EXPD_BC_DIRICHLET || p->fast_dst || p->ndim != 2 || p->precision != EXPD_PREC_MIXED) return false;
    if (p->kernel_flags & EXPD_KF_DST_FP64) return false;
    auto ok = [](int n) { return n % TC_BM == 0 && n <= 1024; };
    return ok(p->NX) && ok(p->NY);
}

void dst_tc_layout(expd_plan p) {
    p->tc_nsl = tc_slices_for(p->tol);
    // the symmetric half of S (even sizes; EXPD_DST_FOLD=0 keeps the full products)
    const char* fo = getenv("EXPD_DST_FOLD");
    p->tc_fold = !(fo && strcmp(fo, "0") == 0) && p->NX % 128 == 0 && p->NY % 128 == 0;
    const double per_slice = (double)p->tc_nsl * p->M * 2.0;
    p->tc_chunk = (int)std::max(1.0, std::min((double)p->Ns, std::floor(2147483648.0 / per_slice)));
}

size_t dst_tc_bytes(expd_plan p) {
    const size_t nx = p->NX, ny = p->NY, nsl = p->tc_nsl;
    return nsl * (nx * nx + ny * ny) * 2 + (nx + ny) * 4 + nsl * (size_t)p->tc_chunk * p->M * 2 +
           (size_t)p->tc_chunk * std::max(nx, ny) * 4 + 256;
}

expd_status dst_tc_setup(expd_plan p, cudaStream_t s) {
    const int NX = p->NX, NY = p->NY, nsl = p->tc_nsl;
    expd_status st = tc_dalloc(p, reinterpret_cast<void**>(&p->tc_S), (size_t)nsl * ((size_t)NX * NX + (size_t)NY * NY) * 2,
                               "DST digit slices");
    if (st == EXPD_OK)
        st = tc_dalloc(p, reinterpret_cast<void**>(&p->tc_pack), (size_t)nsl * p->tc_chunk * p->M * 2, "digit slices");
    if (st == EXPD_OK)
        st = tc_dalloc(p, reinterpret_cast<void**>(&p->tc_ex),
                       ((size_t)NX + NY + (size_t)p->tc_chunk * std::max(NX, NY)) * 4 + 256, "digit exponents");
    if (st != EXPD_OK) return st;
    p->tc_err = p->tc_ex + NX + NY + (size_t)p->tc_chunk * std::max(NX, NY);
    EXPD_CUDA_TRY(cudaMemsetAsync(p->tc_err, 0, sizeof(int), s));
    // digits of S_x and S_y with one exponent per matrix: |S| <= sqrt(2/(n+1)) < 2^e;
    // folded: of the even rows' and the odd rows' first halves (S_e, S_o: n/2 x
    // n/2 each, rows 2c and 2c + 1 of S at stride 2n)
    p->tc_eSx = dst_exponent(NX);
    p->tc_eSy = dst_exponent(NY);
    for (int d = 0; d < 2 && st == EXPD_OK; ++d) {
        const int n = d == 0 ? NX : NY;
        const double* S = d == 0 ? p->Sx : p->Sy;
        uint16_t* out = p->tc_S + (d == 0 ? 0 : (size_t)nsl * NX * NX);
        const int e = d == 0 ? p->tc_eSx : p->tc_eSy;
        if (p->tc_fold) {
            // a digit slice of S_e or S_o holds whole 128-row tiles: h rows
            // padded to a multiple of 128 (h = 192, 320, 448 leave a half
            // tile), so that one digit's last tile does not reach into the
            // next digit's slice; 2 nsl padded slices fit the n^2 nsl of
            // the unfolded layout
            const long long h = n / 2, sl = digit_rows(h) * h;
            st = split_rows(p, S, h, (int)h, 2LL * n, out, sl, nullptr, e, s);
            if (st == EXPD_OK) st = split_rows(p, S + n, h, (int)h, 2LL * n, out + (size_t)nsl * sl, sl, nullptr, e, s);
        } else {
            st = split_rows(p, S, n, n, n, out, (long long)n * n, nullptr, e, s);
        }
    }
    if (st != EXPD_OK) return st;
    EXPD_CUDA_TRY(cudaStreamSynchronize(s));
    return EXPD_OK;
}

// Y[s] = S_y X[s] S_x for ns slices [NY][NX]; tmp holds tc_chunk slices.
expd_status dst2_tc(expd_plan p, const double* X, double* Y, int ns, double* tmp, cudaStream_t s) {
    const int NX = p->NX, NY = p->NY, nsl = p->tc_nsl;
    const long long M = p->M;
    const uint16_t* Sxd = p->tc_S;
    const uint16_t* Syd = p->tc_S + (size_t)nsl * NX * NX;
    int* exA = p->tc_ex + NX + NY;
    // one pass: rows of n values (r of them, R per slice) -> out transposed within slices
    auto pass = [&](const double* in, long long r, int R, int n, const uint16_t* Sd, int eS, double* out) {
        if (!p->tc_fold) {
            expd_status st = split_rows(p, in, r, n, n, p->tc_pack, r * n, exA, INT_MIN, s);
            return st == EXPD_OK ? mma_pass(p, p->tc_pack, exA, r, R, Sd, eS, n, n, out, s) : st;
        }
        const int h = n / 2;
        uint16_t* u = p->tc_pack;
        uint16_t* v = p->tc_pack + (size_t)nsl * r * h;
        expd_status st = split_fold(p, in, r, n, u, v, r * h, exA, s);
        return st == EXPD_OK ? mma_pass(p, u, exA, r, R, Sd, eS, h, h, out, s, v, Sd + (size_t)nsl * digit_rows(h) * h)
                             : st;
    };
    for (int b0 = 0; b0 < ns; b0 += p->tc_chunk) {
        const int cs = std::min(p->tc_chunk, ns - b0);
        const double* x = X + (long long)b0 * M;
        double* y = Y + (long long)b0 * M;
        // pass 1: rows of X (cs*NY rows of NX), T[s] = (X[s] S_x)^T, [NX][NY]
        expd_status st = pass(x, (long long)cs * NY, NY, NX, Sxd, p->tc_eSx, tmp);
        // pass 2: rows of T (cs*NX rows of NY), Y[s] = (T[s] S_y)^T, [NY][NX]
        if (st == EXPD_OK) st = pass(tmp, (long long)cs * NX, NX, NY, Syd, p->tc_eSy, y);
        if (st != EXPD_OK) return st;
    }
    return EXPD_OK;
}

// Reports (and clears) a pipeline wait of a tensor-core kernel (the DST, the
// time kernel) that gave up.
expd_status dst_tc_check(expd_plan p, cudaStream_t s) {
    int* words[2] = {p->tc_dst ? p->tc_err : nullptr, p->tt_err};
    for (int w = 0; w < 2; ++w) {
        if (!words[w]) continue;
        int h = 0;
        EXPD_CUDA_TRY(cudaMemcpyAsync(&h, words[w], sizeof(int), cudaMemcpyDeviceToHost, s));
        EXPD_CUDA_TRY(cudaStreamSynchronize(s));
        if (!h) continue;
        EXPD_CUDA_TRY(cudaMemsetAsync(words[w], 0, sizeof(int), s));
        const char* what = w == 0 ? "tensor-core DST" : "tensor-core time kernel";
        // a wait that gave up because the call was cancelled, or one that ran
        // out of time; the results are invalid either way
        if (p->call_cancelled || p->cancel_req.exchange(0)) {
            if (p->cancel_host) *p->cancel_host = 0;
            p->call_cancelled = 1;
            return expd_fail(EXPD_ERR_CANCELLED, std::string(what) + ": cancelled in flight (results invalid)");
        }
        return expd_fail(EXPD_ERR_TIMEOUT, std::string(what) + ": a pipeline wait gave up after 2 s (results invalid)");
    }
    return EXPD_OK;
}
