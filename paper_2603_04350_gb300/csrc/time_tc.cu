// Time direction of the hot path on the tensor cores: real time columns
// (Dirichlet and Neumann grids, whose eigen-coefficients are real) with the
// float32 preconditioner on float64 storage, windows of at most 128 slices.
//
// For one mode m the preconditioner solve of Eq. (3.3) / Eq. (4.5) is
//     Step (a)  Y_k = sum_n y_n e^{+2 pi i kn/Ns},   y_n = alpha^(n/Ns) q_n,
//     Step (b)  Z_k = Y_k / d_k,  d_k = one - sum_j c_j(m) lambda_k^j,
//     Step (c)  s_n = sum_k Z_k e^{-2 pi i kn/Ns} / (Ns alpha^(n/Ns)),
// with q the residual combination of Eq. (3.2).  The column is real, so Y is
// conjugate-symmetric and Steps (a) and (c) are two real matrix products with
// one constant matrix W (rows f = 2k, 2k+1: cos and sin of 2 pi kn/Ns for
// 0 < k < Ns/2; row 0 the mean; row 1 the alternating row (-1)^n when Ns is
// even) and its transpose:
//     Y[m][f] = sum_n y[m][n] W[f][n],     s[m][n] ~ sum_f w_f Z[m][f] W[f][n]
// (w_f = 2 for the pairs, 1 for the mean and the alternating row).  For a tile
// of 128 consecutive modes both are tcgen05 MMAs with M = 128 (a mode per TMEM
// lane), K and N at most 128:
//   * the data operand lives in TMEM: the thread owning a lane forms its
//     mode's combination slice by slice (direct coalesced loads: a warp reads
//     32 consecutive modes of a slice), keeps the raw values in the
//     accumulator columns, and writes the fp16 digits to the operand columns;
//   * W and W^T sit in shared memory for the CTA's lifetime (K-major, no
//     swizzle, 8 x 8 core matrices);
//   * every operand is two fp16 digits, x = hi + lo, after a power-of-two
//     scale of the row (the constant matrices: 2^14) that puts its largest
//     magnitude in [2^14, 2^15): both digits are normal numbers, x is held to
//     2^-22 relative, and the four digit pairs accumulated in float32 give the
//     product to about 2^-21 -- the float32 preconditioner's accuracy (the
//     float32 FFTs it replaces round at 2^-24 per butterfly over eight to
//     sixteen passes);
//   * Step (b) runs in the drain of the first product, per lane (the real and
//     imaginary parts of a frequency are neighbouring columns), from a shared
//     table of lambda_k^j.
// Two pipelines of eight warps share a CTA (one CTA per SM: W and W^T take
// 128 KB of shared memory), each with its own 256 TMEM columns (operand 128,
// accumulator 128), so one tile's loads overlap the other's products and
// drains.  Waits on MMA completion give up after 2 s and set an error word.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dd.cuh"
#include "plan.h"
#include "tc_ptx.cuh"
#include "time_args.cuh"

namespace {

using namespace expd_time;
using namespace expd_tc;

constexpr int TT_M = 128;                        // modes per tile: the TMEM lanes
constexpr int TT_KMAX = 128;                     // largest window
constexpr int TT_PIPES = 2;                      // tiles in flight per CTA
constexpr int TT_PT = 256;                       // threads per pipeline: two per mode
constexpr int TT_THREADS = TT_PIPES * TT_PT;
constexpr int TT_DIG_BYTES = TT_KMAX * TT_KMAX * 2;  // one fp16 digit of a 128 x 128 matrix (32 KB)
constexpr int TT_SBO = 16 * 128;                 // next 8-row group: sixteen core matrices along K
constexpr int TT_LAMP_ROWS = 65;                 // lambda_k^j for k < 64, row 64 the alternating frequency
constexpr unsigned long long TT_WAIT_NS = 2000000000ull;

// Table image (device buffer and the prefix of shared memory, byte offsets)
constexpr int TT_OFF_W = 0;                                     // W: digit 0, digit 1
constexpr int TT_OFF_WT = 2 * TT_DIG_BYTES;                     // W^T: digit 0, digit 1
constexpr int TT_OFF_LAMP = 4 * TT_DIG_BYTES;                   // float2 [65][6]
constexpr int TT_OFF_GAM = TT_OFF_LAMP + TT_LAMP_ROWS * 6 * 8;  // float [128] Gamma_alpha (0 past the window)
constexpr int TT_OFF_OSC = TT_OFF_GAM + TT_KMAX * 4;            // float [128] 1 / (Ns alpha^(n/Ns))
constexpr int TT_OFF_TRIG = TT_OFF_OSC + TT_KMAX * 4;             // float2 [6][64] (cos, sin)(2 pi k n/Ns)
constexpr int TT_TAB_BYTES = TT_OFF_TRIG + 6 * 64 * 8;
// shared memory only
constexpr int TT_OFF_MAX = TT_TAB_BYTES;                        // float [pipe][half][128] row maxima
constexpr int TT_OFF_ACC = TT_OFF_MAX + TT_PIPES * 2 * TT_M * 4;  // double2 [pipe][lane quarter][128] partials
constexpr int TT_OFF_BAR = TT_OFF_ACC + TT_PIPES * 4 * TT_KMAX * 16;  // mbarriers [2], TMEM slot
constexpr int TT_SMEM_USED = TT_OFF_BAR + 32;
constexpr size_t TT_SMEM = (size_t)TT_SMEM_USED + 1024;         // + alignment of the dynamic base
static_assert(TT_TAB_BYTES % 16 == 0 && TT_OFF_LAMP % 16 == 0 && TT_OFF_ACC % 16 == 0 && TT_OFF_TRIG % 16 == 0,
              "16-byte regions");
static_assert(TT_SMEM <= 232448, "one CTA per SM within 227 KB");

struct TtArgs {
    TimeArgs a;
    const unsigned char* tab;  // the table image (TT_TAB_BYTES)
    int* err;                  // set to 1 when a wait on an MMA gave up
    int NF, KT;                // columns of Step (a)'s product; the window rounded up to 16
    float alpha;               // the identity form's factor (IDENT)
};

// byte offset of element (r, k) of digit d of a 128 x 128 K-major operand image
EXPD_HD int tt_elem_offset(int d, int r, int k) {
    return d * TT_DIG_BYTES + (r >> 3) * TT_SBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void pipe_sync(int id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }

// barrier of one pipeline that also returns the AND of v over its threads
__device__ __forceinline__ bool pipe_and(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, 256, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id)
        : "memory");
    return r != 0;
}

__device__ __noinline__ bool tt_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0 && globaltimer() - t0 > TT_WAIT_NS) return false;
    }
}

// 1/x to the hardware approximation (within one ulp): the divisions of
// Step (b) at the float32 preconditioner's accuracy
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Exact float -> double by integer operations on the encodings for normal
// floats (the exponent rebiased, the fraction widened); zeros, subnormals,
// infinities and NaN through f64_from_f32
__device__ __forceinline__ double f64_of_f32_fast(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e - 1u < 254u)
        return __hiloint2double((int)((u & 0x80000000u) | (((u & 0x7FFFFFFFu) >> 3) + (896u << 20))), (int)(u << 29));
    return f64_from_f32(f);
}

// 2^(15 - e) for a row whose largest magnitude mx satisfies 2^(e-1) <= mx < 2^e:
// the scaled row lies within 2^15; zero and non-finite maxima take 1 (the
// non-finite values themselves reach the output)
__device__ __forceinline__ float digit_scale(float mx) {
    if (!(mx > 0.0f) || !(mx < INFINITY)) return 1.0f;
    const int e = (int)((__float_as_uint(mx) >> 23) & 0xFFu) - 126;
    const int se = min(127, max(-126, 15 - e));
    return __int_as_float((se + 127) << 23);
}

// eight values times a power of two, cut into fp16 digit pairs packed two per
// 32-bit word (the even K index in the low half)
__device__ __forceinline__ void split8(const uint32_t (&v)[8], float sc, uint32_t (&hi)[4], uint32_t (&lo)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float a = __uint_as_float(v[2 * i]) * sc, b = __uint_as_float(v[2 * i + 1]) * sc;
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi[i] = *reinterpret_cast<const uint32_t*>(&h);
        lo[i] = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// Sums of a[0..7] over the warp's 32 lanes: three exchange rounds leave lane l
// with slice index ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1),
// two more complete the sum; returns it (valid in every lane)
template <typename T>
__device__ __forceinline__ T warp_sum8(const T (&a)[8], int lane) {
    T b[4], c[2];
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = (u16 ? a[4 + i] : a[i]) + __shfl_xor_sync(0xffffffffu, u16 ? a[i] : a[4 + i], 16);
#pragma unroll
    for (int i = 0; i < 2; ++i) c[i] = (u8 ? b[2 + i] : b[i]) + __shfl_xor_sync(0xffffffffu, u8 ? b[i] : b[2 + i], 8);
    T d = (u4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, u4 ? c[0] : c[1], 4);
    d += __shfl_xor_sync(0xffffffffu, d, 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
}

// One product: D = A B^T over `ksteps` K-steps of 16, A the two digits in TMEM
// (columns a .. a + 63: hi, a + 64 ..: lo), B the two digits at shared address
// sb (hi) and sb + TT_DIG_BYTES (lo); all four digit pairs (the tensor pipe
// has room to spare: the kernel is bound by its loads and drains).
__device__ __forceinline__ void tt_product(uint32_t d, uint32_t a, uint32_t sb, int ksteps, uint32_t idesc) {
#pragma unroll 1
    for (int q = 0; q < ksteps; ++q) {
        const uint64_t b0 = kmajor_desc(sb + 256u * q, 128u, TT_SBO);
        const uint64_t b1 = kmajor_desc(sb + TT_DIG_BYTES + 256u * q, 128u, TT_SBO);
        tc_mma_ts(d, a + 8u * q, b0, idesc, q > 0 ? 1u : 0u);
        tc_mma_ts(d, a + 8u * q, b1, idesc, 1u);
        tc_mma_ts(d, a + 64u + 8u * q, b0, idesc, 1u);
        tc_mma_ts(d, a + 64u + 8u * q, b1, idesc, 1u);
    }
}

// float32 value of a float64 in float's normal range by integer operations on
// its encoding (rounded half away from zero in magnitude); magnitudes below
// 2^-126 flush to signed zero, larger ones than float's range take the
// rounding conversion (to infinity)
__device__ __forceinline__ float f32_of_f64_fast(double v) {
    const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
    const uint32_t e = (hi >> 20) & 0x7FFu;
    if (e - 897u > 253u) return e < 897u ? __uint_as_float(hi & 0x80000000u) : f32_ftz_from_f64(v);
    // (hi << 3 | lo >> 29): the exponent's low eight bits over 23 fraction bits;
    // the float exponent e - 896 is those eight bits with the top one flipped
    const uint32_t f = __funnelshift_l(lo, hi, 3);
    return __uint_as_float(((hi & 0x80000000u) | ((f ^ 0x40000000u) & 0x7FFFFFFFu)) + ((lo >> 28) & 1u));
}

// LOWQ: the Krylov operator R_s X without right-hand side, its combination in
// float32 from the iterate rounded to float32; otherwise the combination
// F + sigR R_s X in float64, rounded to float32 before Step (a).  ORDER: the
// BDF order s (the lookback of R_s and the degree of d_k).
//
// IDENT (with LOWQ, an unshifted Step (b) and s < Ns): R_s differs from the
// alpha-circulant matrix P of Eq. (3.3) only in the wrap-around terms, R_s =
// P + alpha W with (W X)_n = sum_{j > n} c_j X_{n-j+Ns} nonzero in the first s
// slices, so P^{-1} R_s X = X + alpha P^{-1} (W X).  Step (a) of the s-slice
// vector W X is s terms per frequency (a table of the first s rows of the
// DFT), the first product is skipped, X is read once (by the output pass, which
// reads it for the Krylov dot anyway), and the rounding of the preconditioner
// enters the output scaled by alpha.
template <bool LOWQ, bool IDENT, int ORDER>
__global__ void __launch_bounds__(TT_THREADS, 1) time_kernel_tc(const __grid_constant__ TtArgs ta) {
    const TimeArgs& A = ta.a;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
    const float2* lamp = reinterpret_cast<const float2*>(sm + TT_OFF_LAMP);
    float* gamf = reinterpret_cast<float*>(sm + TT_OFF_GAM);
    const float* oscp = reinterpret_cast<const float*>(sm + TT_OFF_OSC);
    const float2* trig = reinterpret_cast<const float2*>(sm + TT_OFF_TRIG);
    float* smax = reinterpret_cast<float*>(sm + TT_OFF_MAX);
    double2* sacc = reinterpret_cast<double2*>(sm + TT_OFF_ACC);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + TT_OFF_BAR);
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + TT_OFF_BAR + 16);

    const int tid = threadIdx.x, pipe = tid / TT_PT, ptid = tid - pipe * TT_PT;
    const int wp = ptid >> 5, lane = tid & 31, lq = wp & 3, half = wp >> 2;
    const int m = lq * 32 + lane;  // mode within the tile = TMEM lane

    // ---- constants (independent of the previous kernel) ----
    {
        const uint4* src = reinterpret_cast<const uint4*>(ta.tab);
        uint4* dst = reinterpret_cast<uint4*>(sm);
        for (int i = tid; i < TT_TAB_BYTES / 16; i += TT_THREADS) dst[i] = src[i];
    }
    // per-slice partials: every warp adds into its own slots (one lane per
    // slice), summed in a fixed order at the end, so the partials -- and the
    // Krylov solvers that read them -- do not depend on timing
    for (int i = tid; i < TT_PIPES * 4 * TT_KMAX; i += TT_THREADS) sacc[i] = make_double2(0.0, 0.0);
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // W and W^T are read by the MMAs
    if (tid < 32) {
        tc_alloc(smem_u32(slot), 512);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    // the float32 combination's factor sigR Gamma_n (LOWQ), in place of Gamma
    if (LOWQ)
        for (int i = tid; i < TT_KMAX; i += TT_THREADS) gamf[i] *= (float)A.sigR;
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t tA = tmem + 256u * pipe, tD = tA + 128u;  // operand, accumulator (lane 0)
    const uint32_t lanes = (uint32_t)(lq * 32) << 16;
    const uint32_t wA = tA + lanes, wD = tD + lanes;          // this warp's lanes
    const uint32_t bar = smem_u32(&bars[pipe]);
    const int bid = 1 + pipe;
    pdl_wait();

    const int Ns = A.Ns, KT = ta.KT, NF = ta.NF;
    const long long Mcol = A.Mcol;
    const long long ntiles = (Mcol + TT_M - 1) / TT_M;
    const int GN = KT >> 3, GF = NF >> 3;  // 8-column groups (even counts)
    const int gn0 = half * (GN >> 1), gn1 = gn0 + (GN >> 1);
    const int gf0 = half * (GF >> 1), gf1 = gf0 + (GF >> 1);
    const int fsl = min(Ns, A.f_slices);
    const uint32_t idesc1 = (1u << 4) | ((uint32_t)(NF >> 3) << 17) | ((uint32_t)(TT_M >> 4) << 24);
    const uint32_t idesc2 = (1u << 4) | ((uint32_t)(KT >> 3) << 17) | ((uint32_t)(TT_M >> 4) << 24);
    const uint32_t sW = smem_u32(sm + TT_OFF_W), sWT = smem_u32(sm + TT_OFF_WT);
    const float one = (float)(1.0 - A.dshift);
    const float sgR = (float)A.sigR;
    double* X = const_cast<double*>(static_cast<const double*>(A.X));
    const double* F = static_cast<const double*>(A.F);
    double* out = static_cast<double*>(A.out);
    float* sout = static_cast<float*>(A.sout);
    const bool xload = IDENT || A.accum || (LOWQ && A.norms == 2);  // the output pass reads X
    uint32_t ph = 0;
    bool pending = false, ok = true;

    for (long long t = (long long)blockIdx.x * TT_PIPES + pipe; t < ntiles; t += (long long)gridDim.x * TT_PIPES) {
        const long long mg = t * TT_M + m;
        const bool mv = mg < Mcol;
        float cp[ORDER + 1];
        dd cs[ORDER + 1];  // the float64 coefficients as double-float (the accurate combination)
#pragma unroll
        for (int j = 1; j <= ORDER; ++j) {
            cp[j] = mv ? A.C32[(long long)(j - 1) * Mcol + mg] : 0.0f;
            if (!LOWQ) cs[j] = dd_from_f64(mv ? A.C64[(long long)(j - 1) * Mcol + mg] : 0.0);
        }

        const bool xr = X && mv, fr = !LOWQ && F && mv;

        // ---- IDENT: the wrap-around vector y_n = sum_{j=n+1..s} c_j X_{n-j+Ns}
        // (n < s) times sigR Gamma_n, from the window's last s slices ----
        float yv[ORDER];
        if constexpr (IDENT) {
            float xw[ORDER];  // X_{Ns-s} .. X_{Ns-1} rounded to float32
#pragma unroll
            for (int j = 0; j < ORDER; ++j)
                xw[j] = X && mv ? f32_of_f64_fast(X[(long long)(Ns - ORDER + j) * Mcol + mg]) : 0.0f;
#pragma unroll
            for (int n = 0; n < ORDER; ++n) {
                float acc = 0.0f;
#pragma unroll
                for (int j = n + 1; j <= ORDER; ++j) acc = fmaf(cp[j], xw[ORDER + n - j], acc);
                yv[n] = acc * gamf[n];
            }
        }
        float s1 = 1.0f;
        if constexpr (!IDENT) {
        // ---- Step (a) input: the combination of Eq. (3.2) times Gamma_alpha,
        // slice by slice (this thread: groups gn0..gn1-1), raw floats into the
        // accumulator columns; a warp reads 32 consecutive modes of a slice, the
        // next group's loads in flight while a group is formed ----
        float vmax = 0.0f;
        {
            const int nb = gn0 * 8;
            dd wd[ORDER];     // X_{n-1}, ..., X_{n-ORDER} as double-float (zero before slice 0)
            float wf[ORDER];  // the same rounded to float32 (LOWQ)
#pragma unroll
            for (int j = 0; j < ORDER; ++j) {
                const int n = nb - 1 - j;
                const double x = xr && n >= 0 && n < Ns ? X[(long long)n * Mcol + mg] : 0.0;
                if (LOWQ) wf[j] = f32_of_f64_fast(x);
                else wd[j] = dd_from_f64(x);
            }
            const double* xp = X + (long long)nb * Mcol + mg;
            const double* fp = LOWQ ? nullptr : F + (long long)nb * Mcol + mg;
            double nx[8], nf[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                nx[i] = xr && nb + i < Ns ? xp[(long long)i * Mcol] : 0.0;
                if (!LOWQ) nf[i] = fr && nb + i < fsl ? fp[(long long)i * Mcol] : 0.0;
            }
#pragma unroll 1
            for (int g = gn0; g < gn1; ++g) {
                const int n0 = 8 * g;
                double cx[8], cf[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    cx[i] = nx[i];
                    if (!LOWQ) cf[i] = nf[i];
                }
                xp += 8 * Mcol;
                if (!LOWQ) fp += 8 * Mcol;
                if (g + 1 < gn1) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        nx[i] = xr && n0 + 8 + i < Ns ? xp[(long long)i * Mcol] : 0.0;
                        if (!LOWQ) nf[i] = fr && n0 + 8 + i < fsl ? fp[(long long)i * Mcol] : 0.0;
                    }
                }
                uint32_t vb[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float val;
                    if constexpr (LOWQ) {
                        const float xf = f32_of_f64_fast(cx[i]);
                        float q = xf;
#pragma unroll
                        for (int j = 1; j <= ORDER; ++j) q = fmaf(-cp[j], wf[j - 1], q);
#pragma unroll
                        for (int j = ORDER - 1; j > 0; --j) wf[j] = wf[j - 1];
                        wf[0] = xf;
                        val = q * gamf[n0 + i];  // sigR Gamma_n
                    } else {
                        // F_n + sigR (X_n - sum_j c_j X_{n-j}) in double-float on
                        // the float32 pipe (GB300's float64 rate is 1/64 of it):
                        // the terms to 2^-48 relative, so the cancellation of a
                        // small residual keeps its float32 rounding
                        if (X) {
                            const dd xd = dd_from_f64(cx[i]);
                            dd rx = xd;
#pragma unroll
                            for (int j = 1; j <= ORDER; ++j) rx = rx - cs[j] * wd[j - 1];
                            const dd q = dd_from_f64(cf[i]) + rx * sgR;
#pragma unroll
                            for (int j = ORDER - 1; j > 0; --j) wd[j] = wd[j - 1];
                            wd[0] = xd;
                            val = (q.hi + q.lo) * gamf[n0 + i];
                        } else {
                            val = f32_of_f64_fast(cf[i]) * gamf[n0 + i];  // the right-hand side alone
                        }
                    }
                    // slices past the window and modes past the grid give zero
                    // (their loads are zero, Gamma beyond Ns is zero)
                    vmax = fmaxf(vmax, fabsf(val));
                    vb[i] = __float_as_uint(val);
                }
                tm_st8(wD + 8u * g, vb);
            }
        }
        smax[(pipe * 2 + half) * TT_M + m] = vmax;
        tm_wait_st();
        tc_fence_before();
        pipe_sync(bid);
        tc_fence_after();
        s1 = digit_scale(fmaxf(vmax, smax[(pipe * 2 + (half ^ 1)) * TT_M + m]));
#pragma unroll 1
        for (int g = gn0; g < gn1; ++g) {
            uint32_t v[8], hi[4], lo[4];
            tm_ld8(wD + 8u * g, v);
            split8(v, s1, hi, lo);
            tm_st4(wA + 4u * g, hi);
            tm_st4(wA + 64u + 4u * g, lo);
        }
        tm_wait_st();
        tc_fence_before();
        ok = pipe_and(bid, ok);
        if (!ok) break;
        if (ptid == 0) {
            tc_fence_after();
            tt_product(tD, tA, sW, KT >> 4, idesc1);
            tc_commit(bar);
            pending = true;
        }
        const bool w1 = tt_wait(bar, ph);
        ph ^= 1u;
        if (ptid == 0 && w1) pending = false;
        ok = pipe_and(bid, w1);
        if (!ok) break;
        tc_fence_after();

        }  // !IDENT

        // ---- Step (b), in place in the accumulator columns: Z_f = w_f Y_f / d_k ----
        const float k1 = (1.0f / 16384.0f) / s1;  // a power of two: 2^-14 / s1 (s1 <= 2^113)
        float zmax = 0.0f;
#pragma unroll 1
        for (int g = gf0; g < gf1; ++g) {
            uint32_t v[8];
            if constexpr (!IDENT) tm_ld8(wD + 8u * g, v);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = 4 * g + i;
                float yr, yi;
                if constexpr (IDENT) {
                    // Step (a) of the s-slice vector: the mean, the alternating
                    // frequency and the pairs as s-term sums
                    yr = 0.0f;
                    yi = 0.0f;
                    if (k == 0) {
#pragma unroll
                        for (int n = 0; n < ORDER; ++n) {
                            yr += yv[n];
                            yi += (n & 1) ? -yv[n] : yv[n];
                        }
                    } else if (2 * k < Ns) {
#pragma unroll
                        for (int n = 0; n < ORDER; ++n) {
                            const float2 tr = trig[n * 64 + k];
                            yr = fmaf(yv[n], tr.x, yr);
                            yi = fmaf(yv[n], tr.y, yi);
                        }
                    }
                } else {
                    yr = __uint_as_float(v[2 * i]) * k1;
                    yi = __uint_as_float(v[2 * i + 1]) * k1;
                }
                float zr = 0.0f, zi = 0.0f;
                if (k == 0) {
                    // the mean (real d_0) and, for even Ns, the alternating frequency (row 64)
                    float d0 = one, dn = one;
#pragma unroll
                    for (int j = 1; j <= ORDER; ++j) {
                        d0 = fmaf(-cp[j], lamp[j - 1].x, d0);
                        dn = fmaf(-cp[j], lamp[64 * 6 + j - 1].x, dn);
                    }
                    zr = yr * rcp_approx(d0);
                    zi = (Ns & 1) ? 0.0f : yi * rcp_approx(dn);
                } else if (2 * k < Ns) {
                    float dr = one, di = 0.0f;
#pragma unroll
                    for (int j = 1; j <= ORDER; ++j) {
                        const float2 l = lamp[k * 6 + j - 1];
                        dr = fmaf(-cp[j], l.x, dr);
                        di = fmaf(-cp[j], l.y, di);
                    }
                    // 2 y / d = 2 y conj(d) / |d|^2
                    const float inv = 2.0f * rcp_approx(fmaf(dr, dr, di * di));
                    zr = fmaf(yr, dr, yi * di) * inv;
                    zi = fmaf(yi, dr, -yr * di) * inv;
                }
                zmax = fmaxf(zmax, fmaxf(fabsf(zr), fabsf(zi)));
                v[2 * i] = __float_as_uint(zr);
                v[2 * i + 1] = __float_as_uint(zi);
            }
            tm_st8(wD + 8u * g, v);
        }
        smax[(pipe * 2 + half) * TT_M + m] = zmax;
        tm_wait_st();
        pipe_sync(bid);
        const float s2 = digit_scale(fmaxf(zmax, smax[(pipe * 2 + (half ^ 1)) * TT_M + m]));
#pragma unroll 1
        for (int g = gf0; g < gf1; ++g) {
            uint32_t v[8], hi[4], lo[4];
            tm_ld8(wD + 8u * g, v);
            split8(v, s2, hi, lo);
            tm_st4(wA + 4u * g, hi);
            tm_st4(wA + 64u + 4u * g, lo);
        }
        tm_wait_st();
        tc_fence_before();
        ok = pipe_and(bid, ok);
        if (!ok) break;
        if (ptid == 0) {
            tc_fence_after();
            tt_product(tD, tA, sWT, NF >> 4, idesc2);
            tc_commit(bar);
            pending = true;
        }
        const bool w2 = tt_wait(bar, ph);
        ph ^= 1u;
        if (ptid == 0 && w2) pending = false;
        ok = pipe_and(bid, w2);
        if (!ok) break;
        tc_fence_after();

        // ---- Step (c) output: s_n = z_n / (Ns alpha^(n/Ns)), update and partials ----
        const float k2 = (1.0f / 16384.0f) / s2;
        const long long ob = (long long)(gn0 * 8) * Mcol + mg;
        // X again where the output needs it (the update, the Krylov dot), one
        // group of slices ahead
        double xnx[8];
        auto xload8 = [&](int g, double (&d)[8]) {
            const long long gb = ob + (long long)(8 * (g - gn0)) * Mcol;
#pragma unroll
            for (int i = 0; i < 8; ++i) d[i] = xload && mv && 8 * g + i < Ns ? X[gb + (long long)i * Mcol] : 0.0;
        };
        xload8(gn0, xnx);
#pragma unroll 1
        for (int g = gn0; g < gn1; ++g) {
            const int n0 = 8 * g;
            double xo[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) xo[i] = xnx[i];
            if (g + 1 < gn1) xload8(g + 1, xnx);
            uint32_t v[8];
            tm_ld8(wD + 8u * g, v);
            const long long gb = ob + (long long)(8 * (g - gn0)) * Mcol;
            float a8[8], b8[8];  // norms 2: float32 products of the float32 output
            double r8[8];        // the output widened to float64 (zero outside the grid)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int n = n0 + i;
                const bool in = n < Ns && mv;
                float sa = (__uint_as_float(v[i]) * k2) * oscp[n];
                const float xf = LOWQ && (IDENT || A.norms == 2) ? f32_of_f64_fast(xo[i]) : 0.0f;
                if constexpr (IDENT) sa = fmaf(ta.alpha, sa, sgR * xf);  // sigR X + alpha P^{-1} (sigR W X)
                a8[i] = in ? sa * sa : 0.0f;
                b8[i] = LOWQ && A.norms == 2 && in ? xf * sa : 0.0f;
                r8[i] = 0.0;
                if (in) {
                    const double res = f64_of_f32_fast(sa);
                    const long long idx = gb + (long long)i * Mcol;
                    r8[i] = res;
                    if (A.accum) {
                        const double xn = xo[i] + res;
                        X[idx] = xn;
                        if (sout) sout[idx] = sa;
                        xo[i] = xn;
                    } else {
                        out[idx] = res;
                    }
                }
            }
            if (A.norms == 1) {
                // the fixed point's float64 norms (||s_n||^2, ||X_n + s_n||^2)
                double er[8], ex[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    er[i] = r8[i] * r8[i];
                    ex[i] = A.accum && n0 + i < Ns && mv ? xo[i] * xo[i] : 0.0;
                }
                const double sa_ = warp_sum8(er, lane), sb_ = warp_sum8(ex, lane);
                if ((lane & 3) == 0) {
                    const int n = n0 + ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                    double2& acc = sacc[(pipe * 4 + lq) * TT_KMAX + n];
                    acc.x += sa_;
                    acc.y += sb_;
                }
            } else if (A.norms == 2) {
                const float sa_ = warp_sum8(a8, lane), sb_ = warp_sum8(b8, lane);
                if ((lane & 3) == 0) {
                    const int n = n0 + ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                    double2& acc = sacc[(pipe * 4 + lq) * TT_KMAX + n];
                    acc.x += f64_from_f32(sa_);
                    acc.y += f64_from_f32(sb_);
                }
            }
        }
        // the accumulator columns are read before the next tile's stores
        tc_fence_before();
    }
    if (!ok && ptid == 0) atomicExch(ta.err, 1);
    // an MMA group whose completion a wait missed finishes before TMEM is released
    if (ptid == 0 && pending) tt_wait(bar, ph);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (A.norms)
        for (int n = tid; n < Ns; n += TT_THREADS) {
            double2 v = make_double2(0.0, 0.0);
            for (int w = 0; w < TT_PIPES * 4; ++w) {
                v.x += sacc[w * TT_KMAX + n].x;
                v.y += sacc[w * TT_KMAX + n].y;
            }
            A.partial[(size_t)n * gridDim.x + blockIdx.x] = v;
        }
    if (tid < 32) tc_dealloc(tmem, 512);
}

}  // namespace

// ------------------------------------------------------------------ host ----
bool time_tc_eligible(expd_plan p) {
    return p->realcol && p->precision == EXPD_PREC_MIXED && p->Ns >= 1 && p->Ns <= TT_KMAX && !p->no_tc_time;
}

size_t time_tc_bytes(expd_plan p) { return time_tc_eligible(p) ? (size_t)TT_TAB_BYTES + 16 : 0; }

// W (rows f, columns n) and W^T scaled by 2^14 as two fp16 digits each, the
// lambda powers, Gamma_alpha and the output scale; an error word after them.
expd_status time_tc_setup(expd_plan p, cudaStream_t s) {
    if (!time_tc_eligible(p)) return EXPD_OK;
    const int Ns = p->Ns;
    std::vector<unsigned char> img((size_t)TT_TAB_BYTES + 16, 0);
    auto put = [&](int base, int r, int k, double v) {
        const double x = 16384.0 * v;
        const __half hi = __float2half_rn((float)x);
        const __half lo = __float2half_rn((float)(x - (double)__half2float(hi)));
        memcpy(&img[(size_t)base + tt_elem_offset(0, r, k)], &hi, 2);
        memcpy(&img[(size_t)base + tt_elem_offset(1, r, k)], &lo, 2);
    };
    for (int n = 0; n < Ns; ++n) {
        auto both = [&](int f, double v) {
            put(TT_OFF_W, f, n, v);
            put(TT_OFF_WT, n, f, v);
        };
        both(0, 1.0);
        if (Ns % 2 == 0) both(1, (n & 1) ? -1.0 : 1.0);
        for (int k = 1; 2 * k < Ns; ++k) {
            const double th = 2.0 * M_PI * (double)(((long long)k * n) % Ns) / Ns;
            both(2 * k, cos(th));
            both(2 * k + 1, sin(th));
        }
    }
    const double ar = pow(p->alpha, 1.0 / Ns);
    std::vector<float2> lam((size_t)TT_LAMP_ROWS * 6, make_float2(0.f, 0.f));
    for (int k = 0; k < TT_LAMP_ROWS; ++k) {
        // rows k < 64: lambda_k = alpha^(1/Ns) e^{2 pi i k/Ns}; row 64: lambda_{Ns/2} = -alpha^(1/Ns)
        const std::complex<double> l = k < 64 ? std::polar(ar, 2.0 * M_PI * k / Ns) : std::complex<double>(-ar, 0.0);
        std::complex<double> pw = 1.0;
        for (int j = 1; j <= 6; ++j) {
            pw *= l;
            lam[(size_t)k * 6 + j - 1] = make_float2((float)pw.real(), (float)pw.imag());
        }
    }
    memcpy(&img[TT_OFF_LAMP], lam.data(), lam.size() * sizeof(float2));
    std::vector<float> g(TT_KMAX, 0.f), o(TT_KMAX, 0.f);
    for (int n = 0; n < Ns; ++n) {
        const double gm = pow(p->alpha, (double)n / Ns);
        g[n] = (float)gm;
        o[n] = (float)(1.0 / ((double)Ns * gm));
    }
    std::vector<float2> tr((size_t)6 * 64, make_float2(0.f, 0.f));
    for (int n = 0; n < 6; ++n)
        for (int k = 1; k < 64 && 2 * k < Ns; ++k) {
            const double th = 2.0 * M_PI * (double)(((long long)k * n) % Ns) / Ns;
            tr[(size_t)n * 64 + k] = make_float2((float)cos(th), (float)sin(th));
        }
    memcpy(&img[TT_OFF_TRIG], tr.data(), tr.size() * sizeof(float2));
    memcpy(&img[TT_OFF_GAM], g.data(), g.size() * 4);
    memcpy(&img[TT_OFF_OSC], o.data(), o.size() * 4);
    void* d = nullptr;
    cudaError_t e = plan_malloc(p, &d, img.size());
    if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMalloc(tensor-core time tables)", __FILE__, __LINE__);
    p->bytes += img.size();
    p->tt_tab = d;
    p->tt_err = reinterpret_cast<int*>(static_cast<unsigned char*>(d) + TT_TAB_BYTES);
    e = cudaMemcpyAsync(d, img.data(), img.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMemcpyAsync(tensor-core time tables)", __FILE__, __LINE__);
    return EXPD_OK;
}

template <int ORDER>
static void (*pick_tc_kernel(bool lowq, bool ident))(TtArgs) {
    if (!lowq) return time_kernel_tc<false, false, ORDER>;
    return ident ? time_kernel_tc<true, true, ORDER> : time_kernel_tc<true, false, ORDER>;
}

expd_status time_tc_launch(expd_plan p, TimeArgs& a, cudaStream_t s) {
    TtArgs t;
    t.a = a;
    t.tab = static_cast<const unsigned char*>(p->tt_tab);
    t.err = p->tt_err;
    t.KT = (p->Ns + 15) & ~15;
    t.NF = (p->Ns + (p->Ns & 1) + 15) & ~15;
    const bool lowq = !a.F && !a.NL;
    const long long ntiles = (p->Mcol + TT_M - 1) / TT_M;
    long long grid = std::min<long long>(p->sm_count, (ntiles + TT_PIPES - 1) / TT_PIPES);
    if (a.norms) grid = std::min<long long>(grid, p->partial_cap);
    grid = std::max<long long>(grid, 1);
    // the identity form for the unshifted Krylov operator (s < Ns)
    const bool ident = lowq && a.dshift == 0.0 && p->order < p->Ns;
    t.alpha = (float)p->alpha;
    void (*kern)(TtArgs) = nullptr;
    switch (p->order) {
        case 1: kern = pick_tc_kernel<1>(lowq, ident); break;
        case 2: kern = pick_tc_kernel<2>(lowq, ident); break;
        case 3: kern = pick_tc_kernel<3>(lowq, ident); break;
        case 4: kern = pick_tc_kernel<4>(lowq, ident); break;
        case 5: kern = pick_tc_kernel<5>(lowq, ident); break;
        case 6: kern = pick_tc_kernel<6>(lowq, ident); break;
        default: return expd_fail(EXPD_ERR_UNSUPPORTED, "tensor-core time kernel: BDF order outside 1..6");
    }
    EXPD_CUDA_TRY(smem_allow((const void*)kern, TT_SMEM));
    const double ffrac = (double)a.f_slices / p->Ns;
    const double per = (a.X ? 8.0 : 0.0) + (a.F ? 8.0 * ffrac : 0.0) + 8.0 + (a.accum && a.sout ? 4.0 : 0.0);
    // digit-pair products executed: four per element of each of the two products
    const double fl = 4.0 * 2.0 * 2.0 * (double)t.NF * t.KT * (double)(ntiles * TT_M);
    KProf kp(p, s, EXPD_K_TIME_TC, per * p->Ns * (double)p->Mcol, fl);
    EXPD_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(TT_THREADS), TT_SMEM, s, t));
    p->time_grid_used = (int)grid;
    return EXPD_OK;
}
