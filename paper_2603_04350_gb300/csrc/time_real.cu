// Time direction of the hot path on real time columns (Dirichlet grids, whose
// eigen-coefficients are real): the operation of the shared-memory time kernel
// in time_kernel.cu -- residual of Eq. (3.2), the alpha-circulant solve of
// Eq. (3.3) / Eq. (4.5) in Steps (a)-(c), update and per-slice norms -- laid
// out for real columns, with the FFT length fixed at compile time for the
// windows the workloads use (L = 64..1024; other lengths take the same kernel
// with the length read at run time).
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "dd.cuh"
#include "plan.h"
#include "time_args.cuh"
#include "time_column.cuh"
#include "time_fold.cuh"

namespace {

using namespace expd_time;

// Real time columns (Dirichlet grids).  A CTA owns a tile of TR = 16
// consecutive modes and every one of its 8 warps solves two of them as one
// complex column (precond_column_pair: the FFT work of one column for two).
// The tile is stored real, [TR][P] with an odd column stride P, so the
// coalesced row-wise loads and stores (a warp covers 128-byte row segments of
// two slices) and the per-column sweeps are both free of bank conflicts; the
// FFT buffers use the swizzled index map padi<2>.  An operator application
// without right-hand side and N (R_s X for the Krylov solvers) forms its
// residual combination in the preconditioner's precision when that is float32
// (the combination is rounded to float32 before Step (a) in any case); with a
// right-hand side (the residual the fixed point and the refinement rely on) it
// stays in the storage precision ST.  Per-slice partials only when A.norms:
// (||s_n||^2, ||X_n + s_n||^2) for the fixed point's update (norms = 1), or,
// with the float32 preconditioner, (||out_n||^2, <X_n, out_n>) for the Krylov
// solvers (norms = 2; the second only without right-hand side).  Tiles arrive
// by asynchronous copies, all of a thread's elements in flight at once.
constexpr int TIME_REAL_COLS = 2 * EXPD_TIME_COLS;

// Byte offsets of the real kernel's shared-memory regions, each 16-byte aligned
// (the host sizes the launch with the same struct).
template <typename PT, typename ST>
struct RealSmem {
    size_t w, tw, twp, lam, chirp, bp, bm, acc, x, r, gam, gamf, total;
    EXPD_HD static size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }
    EXPD_HD RealSmem(int Ns, int L, int bluestein, int norms) {
        const size_t c = sizeof(typename cplx<PT>::t);
        const int P = Ns | 1;
        size_t o = 0;
        w = o;     o = up16(o + (size_t)EXPD_TIME_COLS * L * c);
        tw = o;    o = up16(o + (size_t)((L >> 1) + 1) * c);
        twp = o;   o = up16(o + (size_t)twp_entries(L) * 2 * c);
        lam = o;   o = up16(o + (size_t)Ns * c);
        chirp = o; o = up16(o + (bluestein ? (size_t)Ns * c : 0));
        bp = o;    o = up16(o + (bluestein ? (size_t)L * c : 0));
        bm = o;    o = up16(o + (bluestein ? (size_t)L * c : 0));
        acc = o;   o = up16(o + (norms ? (size_t)Ns * 16 : 0));
        x = o;     o = up16(o + (size_t)TIME_REAL_COLS * P * sizeof(ST));
        r = o;     o = up16(o + (size_t)TIME_REAL_COLS * P * sizeof(ST));

        gam = o;   o = up16(o + 2 * (size_t)Ns * sizeof(ST));
        gamf = o;  o = up16(o + 2 * (size_t)Ns * sizeof(float));
        total = o;
    }
};

template <typename PT, typename ST, int LOG2L>
__global__ void __launch_bounds__(32 * EXPD_TIME_COLS, sizeof(PT) == 8 ? 2 : 3) time_kernel_real(TimeArgs A) {
    typedef typename cplx<PT>::t PT2;
    constexpr int TR = TIME_REAL_COLS;
    const int Ns = A.Ns, L = LOG2L > 0 ? (1 << LOG2L) : A.L;
    const int P = Ns | 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RealSmem<PT, ST> lay(Ns, L, A.bluestein, A.norms);
    PT2* sW = reinterpret_cast<PT2*>(smem_raw + lay.w);          // [NW][L]
    PT2* tw = reinterpret_cast<PT2*>(smem_raw + lay.tw);         // [L/2]
    TwPair<PT2>* twp = reinterpret_cast<TwPair<PT2>*>(smem_raw + lay.twp);  // per-pass twiddle pairs
    PT2* lam = reinterpret_cast<PT2*>(smem_raw + lay.lam);       // [Ns]
    PT2* chirp = reinterpret_cast<PT2*>(smem_raw + lay.chirp);   // [Ns]  (Bluestein)
    PT2* bp = reinterpret_cast<PT2*>(smem_raw + lay.bp);         // [L]   (Bluestein)
    PT2* bm = reinterpret_cast<PT2*>(smem_raw + lay.bm);         // [L]   (Bluestein)
    double2* sAcc = reinterpret_cast<double2*>(smem_raw + lay.acc);  // [Ns] (norms)
    ST* sX = reinterpret_cast<ST*>(smem_raw + lay.x);            // [TR][P]
    ST* sR = reinterpret_cast<ST*>(smem_raw + lay.r);            // [TR][P]
    ST* gam = reinterpret_cast<ST*>(smem_raw + lay.gam);         // [Ns]
    ST* osc = gam + Ns;                                          // [Ns]
    float* gamf = reinterpret_cast<float*>(smem_raw + lay.gamf); // [Ns]
    float* oscf = gamf + Ns;                                     // [Ns]
    // Operator launches without right-hand side (lowq) leave the residual
    // region free: it holds the float copy of X and the float output, and the
    // float64 output goes to the X region (X is dead once converted)
    float* xf = reinterpret_cast<float*>(sR);                    // [TR][P] (lowq)
    float* rf = xf + (size_t)TR * P;                             // [TR][P] (lowq)

    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < (L >> 1); i += nth) tw[i] = static_cast<const PT2*>(A.tw)[i];
    for (int i = tid; i < Ns; i += nth) {
        lam[i] = static_cast<const PT2*>(A.lam)[i];
        gam[i] = static_cast<const ST*>(A.gam)[i];
        osc[i] = static_cast<const ST*>(A.osc)[i];
        gamf[i] = A.gam32[i];
        oscf[i] = A.osc32[i];
        if (A.norms) sAcc[i] = make_double2(0.0, 0.0);
        if (A.bluestein) chirp[i] = static_cast<const PT2*>(A.chirp)[i];
    }
    if (A.bluestein)
        for (int i = tid; i < L; i += nth) {
            bp[i] = static_cast<const PT2*>(A.bplus)[i];
            bm[i] = static_cast<const PT2*>(A.bminus)[i];
        }
    __syncthreads();
    if (LOG2L > 0 && A.bluestein) {
        // the per-pass twiddle pairs of the folded passes, from the table above
        for (int h = L >> 2; h >= 1; h >>= 2)
            for (int k = tid; k < h; k += nth) {
                TwPair<PT2> tp;
                tp.w4 = tw[k * (L / (4 * h))];
                tp.w2 = tw[k * (L / (2 * h))];
                twp[twp_offset(L, h) + k] = tp;
            }
    }
    pdl_wait();
    __syncthreads();

    const int lane = tid & 31, warp = tid >> 5;
    const long long Mcol = A.Mcol;
    const ST bdt = (ST)A.bdt, sigR = (ST)A.sigR;
    const ST* X = static_cast<const ST*>(A.X);
    const ST* F = static_cast<const ST*>(A.F);
    // float32 combination: preconditioner in float32, no right-hand side, no N
    const bool lowq = std::is_same<PT, float>::value && std::is_same<ST, double>::value && !A.F && !A.NL;
    const PT one = (PT)(1.0 - A.dshift);
    for (long long tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const long long m0 = tile * TR;
        // ---- coalesced load of the tile: asynchronous copies, every one of a
        // thread's elements in flight at once (a warp covers 128-byte row
        // segments of two slices); zero-filled past the last mode and past the
        // right-hand side's nonzero slices ----
        for (int idx = tid; idx < Ns * TR; idx += nth) {
            const int n = idx / TR, c = idx - n * TR;
            const long long m = m0 + c;
            const bool valid = m < Mcol;
            const long long g = (long long)n * Mcol + (valid ? m : 0);
            if (X) cp_async_elem<(int)sizeof(ST)>(&sX[c * P + n], X + g, valid);
            else sX[c * P + n] = (ST)0;
            if (F) cp_async_elem<(int)sizeof(ST)>(&sR[c * P + n], F + g, valid && n < A.f_slices);
            else if (!lowq) sR[c * P + n] = (ST)0;
        }
        cp_async_wait_all();
        // N (nonlinear Dirichlet plans) and the float copy, each thread on the
        // elements it copied
        for (int idx = tid; idx < Ns * TR; idx += nth) {
            const int n = idx / TR, c = idx - n * TR;
            const long long m = m0 + c;
            if (A.NL && m < Mcol)
                sR[c * P + n] = fma(bdt, ldnl<ST, true>(A.NL, (long long)n * Mcol + m, A.nl_f32).x, sR[c * P + n]);
            // the float32 combination reads the iterate once converted (integer
            // rounding of the binary64 encoding, off the float64 pipe;
            // magnitudes below 2^-126 flush to zero)
            if (lowq) xf[c * P + n] = f32_ftz_from_f64((double)sX[c * P + n]);
        }
        __syncthreads();

        // ---- two columns per warp ----
        const int ca = 2 * warp;
        const long long ma = m0 + ca, mb = ma + 1;
        if (ma < Mcol && A.precond) {
            const bool hasb = mb < Mcol;
            ST csa[7], csb[7];
            PT cpa[7], cpb[7];
            csa[0] = csb[0] = (ST)0;
            cpa[0] = cpb[0] = (PT)0;
#pragma unroll
            for (int j = 1; j <= 6; ++j) {
                csa[j] = j <= A.order ? coef<ST>(A, j, ma) : (ST)0;
                cpa[j] = j <= A.order ? coef<PT>(A, j, ma) : (PT)0;
                csb[j] = j <= A.order && hasb ? coef<ST>(A, j, mb) : csa[j];
                cpb[j] = j <= A.order && hasb ? coef<PT>(A, j, mb) : cpa[j];
            }
            PT2* w = sW + (size_t)warp * L;
            const ST* xa = sX + (size_t)ca * P;
            const ST* xb = xa + P;
            // the combination's right-hand side, and the output (lowq: X region)
            const ST* qra = sR + (size_t)ca * P;
            const ST* qrb = qra + P;
            ST* ra = (lowq ? sX : sR) + (size_t)ca * P;
            ST* rb = ra + P;
            const int pos_shift = A.bluestein ? 0 : 1;  // radix-2 windows take bit-reversed positions
            // Bluestein windows at a compile-time length: the pointwise chirp
            // and kernel-spectrum steps fold into the FFT passes (bl_dif / bl_dit)
            const bool fold = LOG2L > 0 && A.bluestein;
            for (int n = lane; n < Ns; n += 32) {
                const int pos = padi<2>(pos_shift ? (int)bitrev(n, A.log2L) : n);
                PT2 val;
                if (lowq) {
                    // q = sigR (X_n - sum_j c_j X_{n-j}) in float32 (coefficients in
                    // the preconditioner's table)
                    const float* xfa = xf + (size_t)ca * P;
                    const float* xfb = xfa + P;
                    float qa = xfa[n], qb = hasb ? xfb[n] : 0.0f;
#pragma unroll
                    for (int j = 1; j <= 6; ++j) {
                        if (j <= A.order && j <= n) {
                            qa = fmaf(-(float)cpa[j], xfa[n - j], qa);
                            if (hasb) qb = fmaf(-(float)cpb[j], xfb[n - j], qb);
                        }
                    }
                    const float sg = (float)A.sigR * gamf[n];
                    val = cvt2<PT2>(make_float2(qa * sg, qb * sg));
                } else {
                    ST qa = qra[n], qb = hasb ? qrb[n] : (ST)0;
                    if (X) {
                        ST rxa = xa[n], rxb = hasb ? xb[n] : (ST)0;
#pragma unroll
                        for (int j = 1; j <= 6; ++j) {
                            if (j <= A.order && j <= n) {
                                rxa = fma(-csa[j], xa[n - j], rxa);
                                if (hasb) rxb = fma(-csb[j], xb[n - j], rxb);
                            }
                        }
                        qa = fma(sigR, rxa, qa);
                        qb = fma(sigR, rxb, qb);
                    }
                    if constexpr (std::is_same<PT, float>::value) {
                        // the accurate combination rounded to float32, then Gamma_alpha in float32
                        val = make_float2(f32_ftz_from_f64((double)qa) * gamf[n], f32_ftz_from_f64((double)qb) * gamf[n]);
                    } else {
                        val = cvt2<PT2>(c2(qa * gam[n], qb * gam[n]));
                    }
                }
                w[pos] = fold ? cmul(val, chirp[n]) : val;
            }
            if (fold) {
                const int half = L >> 1;
                for (int k = Ns + lane; k < half; k += 32) w[padi<2>(k)] = c2((PT)0, (PT)0);
                EXPD_SYNCWARP();
                // Step (a): chirp-z convolution; on exit w[k] c_k = L Y_k for k < Ns
                if constexpr (LOG2L > 0) {
                    bl_dif<PT2, LOG2L, -1>(w, twp, bp, lane);
                    bl_dit<PT2, LOG2L, +1>(w, twp, lane);
                }
                // Step (b) on two real columns at once (precond_column_pair), the
                // Step (a) output chirp folded into the reads and Step (c)'s input
                // chirp into the writes
                PT c1[7], c2v[7];
#pragma unroll
                for (int j = 1; j <= 6; ++j) {
                    c1[j] = j <= A.order ? cpa[j] : (PT)0;
                    c2v[j] = j <= A.order ? cpb[j] : (PT)0;
                }
                const PT hf = (PT)0.5;
                for (int k = lane; k <= Ns / 2; k += 32) {
                    const int kk = k == 0 ? 0 : Ns - k;
                    const PT2 av = cmul(w[padi<2>(k)], chirp[k]), bv = cmul(w[padi<2>(kk)], chirp[kk]);
                    const PT2 y1 = c2(hf * (av.x + bv.x), hf * (av.y - bv.y));
                    const PT2 y2 = c2(hf * (av.y + bv.y), hf * (bv.x - av.x));
                    const PT2 z1 = cdiv(y1, precond_divisor<PT, PT2, PT>(lam[k], c1, A.order, one));
                    const PT2 z2 = cdiv(y2, precond_divisor<PT, PT2, PT>(lam[k], c2v, A.order, one));
                    const PT2 wk = cmulc(c2(z1.x - z2.y, z1.y + z2.x), chirp[k]);
                    const PT2 wkk = cmulc(c2(z1.x + z2.y, z2.x - z1.y), chirp[kk]);
                    w[padi<2>(k)] = wk;
                    if (kk != k) w[padi<2>(kk)] = wkk;
                }
                for (int k = Ns + lane; k < half; k += 32) w[padi<2>(k)] = c2((PT)0, (PT)0);
                EXPD_SYNCWARP();
                // Step (c): the inverse DFT by chirp-z; the output chirp below
                if constexpr (LOG2L > 0) {
                    bl_dif<PT2, LOG2L, -1>(w, twp, bm, lane);
                    bl_dit<PT2, LOG2L, +1>(w, twp, lane);
                }
            } else {
                EXPD_SYNCWARP();
                precond_column_pair<PT, PT2, 2, LOG2L>(w, Ns, L, A.log2L, A.bluestein, tw, lam, chirp, bp, bm, cpa, cpb,
                                                       A.order, lane, 32, one);
            }
            for (int n = lane; n < Ns; n += 32) {
                PT2 v = w[padi<2>(pos_shift ? (int)bitrev(n, A.log2L) : n)];
                if (fold) v = cmulc(v, chirp[n]);
                if constexpr (std::is_same<PT, float>::value) {
                    // output scale in float32, widened exactly by integer operations
                    const float sa = v.x * oscf[n], sb = v.y * oscf[n];
                    if (lowq && A.norms == 2) {
                        rf[(size_t)ca * P + n] = sa;
                        if (hasb) rf[(size_t)(ca + 1) * P + n] = sb;
                    }
                    if constexpr (std::is_same<ST, double>::value) {
                        ra[n] = f64_from_f32(sa);
                        if (hasb) rb[n] = f64_from_f32(sb);
                    } else {
                        ra[n] = (ST)sa;
                        if (hasb) rb[n] = (ST)sb;
                    }
                } else {
                    ra[n] = (ST)v.x * osc[n];
                    if (hasb) rb[n] = (ST)v.y * osc[n];
                }
            }
        } else if (ma < Mcol) {
            // no preconditioner: out = F + bdt N + sigR R_s X in ST
            const bool hasb = mb < Mcol;
            for (int c = ca; c < ca + 2 && (c == ca || hasb); ++c) {
                const long long mc = m0 + c;
                ST cs[7];
#pragma unroll
                for (int j = 1; j <= 6; ++j) cs[j] = j <= A.order ? coef<ST>(A, j, mc) : (ST)0;
                const ST* xc = sX + (size_t)c * P;
                ST* rc = sR + (size_t)c * P;
                for (int n = lane; n < Ns; n += 32) {
                    ST q = rc[n];
                    if (X) {
                        ST rx = xc[n];
#pragma unroll
                        for (int j = 1; j <= 6; ++j)
                            if (j <= A.order && j <= n) rx = fma(-cs[j], xc[n - j], rx);
                        q = fma(sigR, rx, q);
                    }
                    rc[n] = q;
                }
            }
        }
        __syncthreads();

        // ---- coalesced write-back; per-element norm terms into sR / sX ----
        for (int idx = tid; idx < Ns * TR; idx += nth) {
            const int n = idx / TR, c = idx - n * TR;
            const long long mm = m0 + c;
            ST e_r = (ST)0, e_x = (ST)0;
            if (mm < Mcol) {
                const long long g = (long long)n * Mcol + mm;
                const ST res = lowq ? sX[c * P + n] : sR[c * P + n];
                if (A.accum) {
                    const ST xn = sX[c * P + n] + res;
                    const_cast<ST*>(X)[g] = xn;
                    if (A.sout) static_cast<float*>(A.sout)[g] = (float)res;
                    if (A.norms) {
                        e_r = res * res;
                        e_x = xn * xn;
                    }
                } else {
                    static_cast<ST*>(A.out)[g] = res;
                    if (A.norms == 1) e_r = res * res;
                }
            }
            if (A.norms == 1) {
                sR[c * P + n] = e_r;
                sX[c * P + n] = e_x;
            } else if (std::is_same<PT, float>::value && A.norms == 2) {
                // Krylov partials (||out||^2, <X, out>) from float32 products of
                // float32 values (the float64 output is the exact widening of
                // the float one; with a right-hand side it is rounded back
                // exactly): their rounding, ~2^-24 relative and random, is far
                // below the orthogonal part of out the solver extracts.  The
                // per-element products go to float scratch: xf / rf (lowq) or
                // the X region (free once the column phase is done)
                float fr = 0.0f, fx = 0.0f;
                if (mm < Mcol) {
                    const float r32 = lowq ? rf[c * P + n] : f32_rn_from_f64((double)sR[c * P + n]);
                    fr = r32 * r32;
                    if (lowq) fx = xf[c * P + n] * r32;
                }
                float* pr = lowq ? rf : reinterpret_cast<float*>(sX);
                float* px = lowq ? xf : reinterpret_cast<float*>(sX) + (size_t)TR * P;
                pr[c * P + n] = fr;
                px[c * P + n] = fx;
            }
        }
        __syncthreads();
        if (A.norms == 1) {
            for (int n = tid; n < Ns; n += nth) {
                ST a = (ST)0, b = (ST)0;
                for (int c = 0; c < TR; ++c) {
                    a += sR[c * P + n];
                    b += sX[c * P + n];
                }
                sAcc[n].x += (double)a;
                sAcc[n].y += (double)b;
            }
            __syncthreads();
        } else if (std::is_same<PT, float>::value && A.norms == 2) {
            const float* pr = lowq ? rf : reinterpret_cast<const float*>(sX);
            const float* px = lowq ? xf : reinterpret_cast<const float*>(sX) + (size_t)TR * P;
            for (int n = tid; n < Ns; n += nth) {
                float a = 0.0f, b = 0.0f;
                for (int c = 0; c < TR; ++c) {
                    a += pr[c * P + n];
                    b += px[c * P + n];
                }
                sAcc[n].x += f64_from_f32(a);
                sAcc[n].y += f64_from_f32(b);
            }
            __syncthreads();
        }
    }
    if (A.norms)
        for (int n = tid; n < Ns; n += nth) A.partial[(size_t)n * gridDim.x + blockIdx.x] = sAcc[n];
}

template <typename PT, typename ST, int LOG2L>
expd_status launch_time_real(expd_plan p, TimeArgs& a, cudaStream_t s) {
    const TimeTables& t = std::is_same<PT, float>::value ? p->t32 : p->t64;
    const TimeTables& ts = std::is_same<ST, float>::value ? p->t32 : p->t64;
    a.gam = ts.gam;
    a.osc = ts.osc;
    a.gam32 = static_cast<const float*>(p->t32.gam);
    a.osc32 = static_cast<const float*>(p->t32.osc);
    a.lam = t.lam;
    a.tw = t.tw;
    a.chirp = t.chirp;
    a.bplus = t.bplus;
    a.bminus = t.bminus;
    a.L = t.L;
    a.log2L = t.log2L;
    a.bluestein = t.bluestein;
    a.ntiles = (p->Mcol + TIME_REAL_COLS - 1) / TIME_REAL_COLS;
    const size_t smem = RealSmem<PT, ST>(p->Ns, t.L, t.bluestein, a.norms).total;
    auto kern = time_kernel_real<PT, ST, LOG2L>;
    EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    int per_sm = 1;
    EXPD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * EXPD_TIME_COLS, smem));
    long long grid = (long long)p->sm_count * std::max(per_sm, 1);
    grid = std::min<long long>(grid, std::max<long long>(a.ntiles, 1));
    if (a.norms) grid = std::min<long long>(grid, p->partial_cap);
    const double esz = sizeof(ST);
    const double nlsz = a.nl_f32 ? 4.0 : 8.0;
    const double ffrac = (double)a.f_slices / p->Ns;
    const double per = (a.X ? esz : 0.0) + (a.F ? esz * ffrac : 0.0) + (a.NL ? nlsz : 0.0) + esz +
                       (a.accum && a.sout ? 4.0 : 0.0);
    const double lg = (double)t.log2L;
    const double fl_col = (a.precond ? (t.bluestein ? 4.0 : 2.0) * 5.0 * t.L * lg / 2.0 + 8.0 * p->order * p->Ns : 0.0) +
                          2.0 * p->order * p->Ns;
    const int cls = sizeof(ST) == 4 ? EXPD_K_TIME32 : EXPD_K_TIME;
    KProf kp(p, s, cls, per * p->Ns * (double)p->Mcol, fl_col * (double)p->Mcol);
    EXPD_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(32 * EXPD_TIME_COLS), smem, s, a));
    p->time_grid_used = (int)grid;
    return EXPD_OK;
}


// the FFT length as a compile-time constant where the workloads need it
template <typename PT, typename ST>
expd_status launch_for_length(expd_plan p, TimeArgs& a, cudaStream_t s) {
    const TimeTables& t = std::is_same<PT, float>::value ? p->t32 : p->t64;
    switch (t.log2L) {
        case 6: return launch_time_real<PT, ST, 6>(p, a, s);
        case 7: return launch_time_real<PT, ST, 7>(p, a, s);
        case 8: return launch_time_real<PT, ST, 8>(p, a, s);
        case 9: return launch_time_real<PT, ST, 9>(p, a, s);
        case 10: return launch_time_real<PT, ST, 10>(p, a, s);
        default: return launch_time_real<PT, ST, 0>(p, a, s);
    }
}

}  // namespace

// Real columns with float64 (st32 = 0) or float32 (st32 = 1) storage and the
// float32 (f32 = 1) or float64 preconditioner.
expd_status time_real_launch(expd_plan p, TimeArgs& a, int f32, int st32, cudaStream_t s) {
    if (st32) return launch_for_length<float, float>(p, a, s);
    return f32 ? launch_for_length<float, double>(p, a, s) : launch_for_length<double, double>(p, a, s);
}
