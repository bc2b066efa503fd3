// Time direction of the hot path on complex time columns (periodic grids,
// whose half-spectrum eigen-coefficients are complex; complex states): the
// operation of the generic shared-memory time kernel in time_kernel.cu --
// residual of Eq. (3.2), the alpha-circulant solve of Eq. (3.3) / Eq. (4.5)
// in Steps (a)-(c), update and per-slice norms -- with the FFT length fixed at
// compile time for the windows the workloads use (L = 64..1024; other
// lengths take the same kernel with the length read at run time).  Bluestein
// windows fold their chirps into the first and last radix passes
// (time_fold.cuh), the FFT buffers use the swizzled index map padi<2>, and the
// tiles arrive by asynchronous copies.
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

// One warp per complex column, C columns per CTA: 8, or 12 for double-float
// storage (16-byte elements leave room for one CTA per SM only, so a wider
// CTA is what adds resident warps).  The tiles are column-major with the odd
// column stride P = Ns | 1, so the coalesced row-wise copies (consecutive
// lanes on consecutive columns) and the per-column sweeps are both free of
// bank conflicts.
template <typename PT, typename ST, int TC_COLS>
struct CplxSmem {
    size_t w, tw, twp, lam, chirp, bp, bm, acc, x, r, nl, gam, wgt, total;
    EXPD_HD static size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }
    // nl_async: N arrives by asynchronous copies into a tile of its own
    EXPD_HD CplxSmem(int Ns, int L, int bluestein, int nl_async) {
        typedef typename cplx<PT>::t PT2;
        typedef typename cplx<ST>::t ST2;
        const size_t c = sizeof(PT2), sc = sizeof(ST2);
        const int P = Ns | 1;
        size_t o = 0;
        w = o;     o = up16(o + (size_t)TC_COLS * L * c);
        tw = o;    o = up16(o + (size_t)((L >> 1) + 1) * c);
        twp = o;   o = up16(o + (size_t)twp_entries(L) * 2 * c);
        lam = o;   o = up16(o + (size_t)Ns * c);
        chirp = o; o = up16(o + (bluestein ? (size_t)Ns * c : 0));
        bp = o;    o = up16(o + (bluestein ? (size_t)L * c : 0));
        bm = o;    o = up16(o + (bluestein ? (size_t)L * c : 0));
        acc = o;   o = up16(o + (size_t)Ns * sc);
        x = o;     o = up16(o + (size_t)TC_COLS * P * sc);
        r = o;     o = up16(o + (size_t)TC_COLS * P * sc);
        nl = o;    o = up16(o + (nl_async ? (size_t)TC_COLS * P * sc : 0));
        gam = o;   o = up16(o + 2 * (size_t)Ns * sizeof(ST));
        wgt = o;   o = up16(o + (size_t)TC_COLS * sizeof(ST));
        total = o;
    }
};

// whether N's elements have the storage type ST2 (then they are copied with the tile)
template <typename ST>
EXPD_HD bool nl_copyable(const TimeArgs& A) {
    if (!A.NL) return false;
    if (std::is_same<ST, dd>::value) return true;
    return std::is_same<ST, float>::value ? A.nl_f32 != 0 : A.nl_f32 == 0;
}

template <typename PT, typename ST, int LOG2L, int C>
__global__ void __launch_bounds__(32 * C, C == 8 ? (sizeof(ST) == 4 ? 3 : 2) : 1) time_kernel_cplx(TimeArgs A) {
    typedef typename cplx<PT>::t PT2;
    typedef typename cplx<ST>::t ST2;
    const int Ns = A.Ns, L = LOG2L > 0 ? (1 << LOG2L) : A.L;
    const int P = Ns | 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // N in the storage type (float32 N with float32 storage, double-float N
    // with double-float storage, float64 N with float64 storage) is copied
    // asynchronously with the tile; any other N is read element by element
    const bool nl_async = nl_copyable<ST>(A);
    const CplxSmem<PT, ST, C> lay(Ns, L, A.bluestein, nl_async);
    PT2* sW = reinterpret_cast<PT2*>(smem_raw + lay.w);          // [C][L]
    PT2* tw = reinterpret_cast<PT2*>(smem_raw + lay.tw);         // [L/2]
    TwPair<PT2>* twp = reinterpret_cast<TwPair<PT2>*>(smem_raw + lay.twp);
    PT2* lam = reinterpret_cast<PT2*>(smem_raw + lay.lam);       // [Ns]
    PT2* chirp = reinterpret_cast<PT2*>(smem_raw + lay.chirp);   // [Ns]  (Bluestein)
    PT2* bp = reinterpret_cast<PT2*>(smem_raw + lay.bp);         // [L]   (Bluestein)
    PT2* bm = reinterpret_cast<PT2*>(smem_raw + lay.bm);         // [L]   (Bluestein)
    ST2* sAcc = reinterpret_cast<ST2*>(smem_raw + lay.acc);      // [Ns]
    ST2* sX = reinterpret_cast<ST2*>(smem_raw + lay.x);          // [C][P]
    ST2* sR = reinterpret_cast<ST2*>(smem_raw + lay.r);          // [C][P]
    ST2* sN = reinterpret_cast<ST2*>(smem_raw + lay.nl);         // [C][P] (nl_async)
    ST* gam = reinterpret_cast<ST*>(smem_raw + lay.gam);         // [Ns]
    ST* osc = gam + Ns;                                          // [Ns]
    ST* sWgt = reinterpret_cast<ST*>(smem_raw + lay.wgt);        // [C] norm weight of each column

    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < (L >> 1); i += nth) tw[i] = static_cast<const PT2*>(A.tw)[i];
    for (int i = tid; i < Ns; i += nth) {
        lam[i] = static_cast<const PT2*>(A.lam)[i];
        gam[i] = static_cast<const ST*>(A.gam)[i];
        osc[i] = static_cast<const ST*>(A.osc)[i];
        sAcc[i] = c2((ST)0, (ST)0);
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
    const ST2* X = static_cast<const ST2*>(A.X);
    const ST2* F = static_cast<const ST2*>(A.F);
    const ST2* NLc = static_cast<const ST2*>(A.NL);
    const PT one = (PT)(1.0 - A.dshift);
    const bool fold = LOG2L > 0 && A.bluestein;
    const int pos_shift = A.bluestein ? 0 : 1;  // radix-2 windows take bit-reversed positions
    for (long long tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const long long m0 = tile * C;
        // ---- the tile by asynchronous copies (zero-filled past the last mode
        // and past the right-hand side's nonzero slices), then N, each thread
        // on the elements it copied ----
        for (int idx = tid; idx < Ns * C; idx += nth) {
            const int n = idx / C, c = idx - n * C;
            const long long m = m0 + c;
            const bool valid = m < Mcol;
            const long long g = (long long)n * Mcol + (valid ? m : 0);
            if (X) cp_async_elem<(int)sizeof(ST2)>(&sX[c * P + n], X + g, valid);
            else sX[c * P + n] = c2((ST)0, (ST)0);
            if (F) cp_async_elem<(int)sizeof(ST2)>(&sR[c * P + n], F + g, valid && n < A.f_slices);
            else sR[c * P + n] = c2((ST)0, (ST)0);
            if (nl_async) cp_async_elem<(int)sizeof(ST2)>(&sN[c * P + n], NLc + g, valid);
        }
        cp_async_wait_all();
        if (A.NL) {
            for (int idx = tid; idx < Ns * C; idx += nth) {
                const int n = idx / C, c = idx - n * C;
                const long long m = m0 + c;
                if (m < Mcol) {
                    const ST2 v = nl_async ? sN[c * P + n] : ldnl<ST, false>(A.NL, (long long)n * Mcol + m, A.nl_f32);
                    ST2 r = sR[c * P + n];
                    r.x = fma(bdt, v.x, r.x);
                    r.y = fma(bdt, v.y, r.y);
                    sR[c * P + n] = r;
                }
            }
        }
        if (tid < C) {
            const long long m = m0 + tid;
            sWgt[tid] = m < Mcol ? mode_weight<ST>(m, A.KX, A.NX, A.realcol) : (ST)0;
        }
        __syncthreads();

        // ---- one warp per column ----
        const long long m = m0 + warp;
        if (m < Mcol) {
            ST cs[7];
            PT cp[7];
            cs[0] = (ST)0;
            cp[0] = (PT)0;
#pragma unroll
            for (int j = 1; j <= 6; ++j) {
                cs[j] = j <= A.order ? coef<ST>(A, j, m) : (ST)0;
                cp[j] = j <= A.order ? coef<PT>(A, j, m) : (PT)0;
            }
            PT2* w = sW + (size_t)warp * L;
            const ST2* xc = sX + (size_t)warp * P;
            ST2* rc = sR + (size_t)warp * P;
            // residual-type combination q_n in ST, then Gamma_alpha
            for (int n = lane; n < Ns; n += 32) {
                ST2 q = rc[n];
                if (X) {
                    ST2 rx = xc[n];
#pragma unroll
                    for (int j = 1; j <= 6; ++j) {
                        if (j <= A.order && j <= n) rx = sub_cx(rx, cs[j], xc[n - j]);
                    }
                    q.x = fma(sigR, rx.x, q.x);
                    q.y = fma(sigR, rx.y, q.y);
                }
                if (!A.precond) {
                    rc[n] = q;
                } else {
                    const PT2 val = cvt2<PT2>(cscale(q, gam[n]));
                    const int pos = padi<2>(pos_shift ? (int)bitrev(n, A.log2L) : n);
                    w[pos] = fold ? cmul(val, chirp[n]) : val;
                }
            }
            if (A.precond) {
                if (fold) {
                    const int half = L >> 1;
                    for (int k = Ns + lane; k < half; k += 32) w[padi<2>(k)] = c2((PT)0, (PT)0);
                    EXPD_SYNCWARP();
                    // Step (a): chirp-z convolution; on exit w[k] c_k = L Y_k for k < Ns
                    if constexpr (LOG2L > 0) {
                        bl_dif<PT2, LOG2L, -1>(w, twp, bp, lane);
                        bl_dit<PT2, LOG2L, +1>(w, twp, lane);
                    }
                    // Step (b), the output chirp of Step (a) on the read and the
                    // input chirp of Step (c) on the write
                    for (int k = lane; k < Ns; k += 32) {
                        const PT2 y = cmul(w[padi<2>(k)], chirp[k]);
                        const PT2 z = cdiv(y, precond_divisor<PT, PT2, PT>(lam[k], cp, A.order, one));
                        w[padi<2>(k)] = cmulc(z, chirp[k]);
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
                    precond_column<PT, PT2, PT, 2>(w, Ns, L, A.log2L, A.bluestein, tw, lam, chirp, bp, bm, cp,
                                                   A.order, lane, 32, one);
                }
                for (int n = lane; n < Ns; n += 32) {
                    PT2 v = w[padi<2>(pos_shift ? (int)bitrev(n, A.log2L) : n)];
                    if (fold) v = cmulc(v, chirp[n]);
                    rc[n] = cscale(cvt2<ST2>(v), osc[n]);
                }
            }
        }
        __syncthreads();

        // ---- coalesced write-back; per-element norm terms into sX ----
        for (int idx = tid; idx < Ns * C; idx += nth) {
            const int n = idx / C, c = idx - n * C;
            const long long mm = m0 + c;
            ST2 nrm = c2((ST)0, (ST)0);
            if (mm < Mcol) {
                const long long g = (long long)n * Mcol + mm;
                const ST2 res = sR[c * P + n];
                const ST wgt = sWgt[c];
                nrm.x = wgt * fma(res.x, res.x, res.y * res.y);
                if (A.accum) {
                    const ST2 xn = cadd(sX[c * P + n], res);
                    stcol<ST, false>(const_cast<void*>(A.X), g, xn);
                    nrm.y = wgt * fma(xn.x, xn.x, xn.y * xn.y);
                    if (A.sout) stcol<float, false>(A.sout, g, cvt2<float2>(res));
                } else {
                    stcol<ST, false>(A.out, g, res);
                }
            }
            sX[c * P + n] = nrm;
        }
        __syncthreads();
        for (int n = tid; n < Ns; n += nth) {
            ST a = (ST)0, b = (ST)0;
            for (int c = 0; c < C; ++c) {
                a += sX[c * P + n].x;
                b += sX[c * P + n].y;
            }
            sAcc[n].x += a;
            sAcc[n].y += b;
        }
        __syncthreads();
    }
    for (int n = tid; n < Ns; n += nth)
        A.partial[(size_t)n * gridDim.x + blockIdx.x] = make_double2((double)sAcc[n].x, (double)sAcc[n].y);
}

template <typename PT, typename ST, int LOG2L, int TC_COLS>
expd_status launch_time_cplx(expd_plan p, TimeArgs& a, cudaStream_t s) {
    const TimeTables& t = std::is_same<PT, float>::value ? p->t32 : p->t64;
    const TimeTables& ts = std::is_same<ST, float>::value ? p->t32 : p->t64;
    a.gam = std::is_same<ST, dd>::value ? p->gamdd : ts.gam;
    a.osc = std::is_same<ST, dd>::value ? p->oscdd : ts.osc;
    a.lam = t.lam;
    a.tw = t.tw;
    a.chirp = t.chirp;
    a.bplus = t.bplus;
    a.bminus = t.bminus;
    a.L = t.L;
    a.log2L = t.log2L;
    a.bluestein = t.bluestein;
    a.ntiles = (p->Mcol + TC_COLS - 1) / TC_COLS;
    const size_t smem = CplxSmem<PT, ST, TC_COLS>(p->Ns, t.L, t.bluestein, nl_copyable<ST>(a)).total;
    auto kern = time_kernel_cplx<PT, ST, LOG2L, TC_COLS>;
    EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    int per_sm = 1;
    EXPD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * TC_COLS, smem));
    long long grid = (long long)p->sm_count * std::max(per_sm, 1);
    grid = std::min<long long>(grid, std::max<long long>(a.ntiles, 1));
    grid = std::min<long long>(grid, p->partial_cap);
    const double esz = 2.0 * sizeof(ST);
    const double nlsz = 2.0 * (std::is_same<ST, dd>::value ? 8.0 : (a.nl_f32 ? 4.0 : 8.0));
    const double ffrac = (double)a.f_slices / p->Ns;
    const double per = (a.X ? esz : 0.0) + (a.F ? esz * ffrac : 0.0) + (a.NL ? nlsz : 0.0) + esz +
                       (a.accum && a.sout ? 8.0 : 0.0);
    const double lg = (double)t.log2L;
    const double fl_col = (a.precond ? (t.bluestein ? 4.0 : 2.0) * 5.0 * t.L * lg + 8.0 * p->order * p->Ns : 0.0) +
                          4.0 * p->order * p->Ns;
    const int cls = std::is_same<ST, float>::value ? EXPD_K_TIME32
                    : std::is_same<ST, dd>::value  ? EXPD_K_TIMEDD
                                                   : EXPD_K_TIME;
    KProf kp(p, s, cls, per * p->Ns * (double)p->Mcol, fl_col * (double)p->Mcol);
    EXPD_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(32 * TC_COLS), smem, s, a));
    p->time_grid_used = (int)grid;
    return EXPD_OK;
}

template <typename PT, typename ST, int C>
expd_status launch_cplx_for_length(expd_plan p, TimeArgs& a, cudaStream_t s) {
    const TimeTables& t = std::is_same<PT, float>::value ? p->t32 : p->t64;
    switch (t.log2L) {
        case 6: return launch_time_cplx<PT, ST, 6, C>(p, a, s);
        case 7: return launch_time_cplx<PT, ST, 7, C>(p, a, s);
        case 8: return launch_time_cplx<PT, ST, 8, C>(p, a, s);
        case 9: return launch_time_cplx<PT, ST, 9, C>(p, a, s);
        case 10: return launch_time_cplx<PT, ST, 10, C>(p, a, s);
        default: return launch_time_cplx<PT, ST, 0, C>(p, a, s);
    }
}

}  // namespace

size_t time_cplx_smem_bytes(expd_plan p, int st) {
    const TimeTables& t = st ? p->t32 : p->t64;
    // (eight columns, N copied with the tile: the largest eight-column layout)
    if (st == 1) return CplxSmem<float, float, 8>(p->Ns, t.L, t.bluestein, 1).total;
    if (st == 2) return CplxSmem<float, dd, 8>(p->Ns, t.L, t.bluestein, 1).total;
    return CplxSmem<double, double, 8>(p->Ns, t.L, t.bluestein, 1).total;
}

// Complex columns with real coefficient tables: st = 1 float32 storage with
// the float32 preconditioner, st = 2 double-float storage with the float32
// preconditioner, st = 0 float64 storage with the float64 preconditioner.
expd_status time_cplx_launch(expd_plan p, TimeArgs& a, int st, cudaStream_t s) {
    if (st == 1) return launch_cplx_for_length<float, float, 8>(p, a, s);
    if (st == 2) {
        const TimeTables& t = p->t32;
        if (CplxSmem<float, dd, 12>(p->Ns, t.L, t.bluestein, 1).total <= 227 * 1024)
            return launch_cplx_for_length<float, dd, 12>(p, a, s);
        return launch_cplx_for_length<float, dd, 8>(p, a, s);
    }
    return launch_cplx_for_length<double, double, 8>(p, a, s);
}
