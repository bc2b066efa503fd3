// Time direction of the hot path, register-resident variant: the same
// operation as the shared-memory time kernel (residual of Eq. (3.2), the
// alpha-circulant solve of Eq. (3.3) / Eq. (4.5) in Steps (a)-(c), update and
// per-slice norms), for power-of-two windows with the float32 preconditioner.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "dd.cuh"
#include "plan.h"
#include "time_args.cuh"

using expd_time::TimeArgs;

namespace {

using namespace expd_time;

// Register-resident variant for power-of-two windows NS in {16, 32, 64} with the
// float32 preconditioner.  A group of G consecutive lanes owns one spatial
// mode's time column; lane g of the group holds slices n = G j + g, j < R = NS/G,
// in registers.  Loads and stores are coalesced across the groups of a warp
// (consecutive modes), and the length-NS transforms factor as NS = G x R:
//   forward  Y[k1 + R k2] = sum_g w^(g k2)_G  w^(g k1)_NS  sum_j w^(j k1)_R y[G j + g]
// (R-point FFT in registers, twiddle, G-point FFT across the lanes by
// shuffles), and the inverse runs the same factors backwards.  The residual's
// sliding window of the previous `order` iterates comes from the neighbouring
// lanes by shuffles.  Per-slice norms are reduced over the warp's groups with a
// transpose-reduce and over the CTA in shared memory.
constexpr int REG_THREADS = 128;
// Lanes per column.  float32 storage: 4 (measured faster than 8 lanes with 8
// slices each, whose third cross-lane stage costs more than the occupancy it
// buys).  16-byte elements (double-float, float64) with Ns = 64: 8 lanes, 80
// registers, six CTAs per SM (the double-float sweep's time kernel 54 -> 41 us
// on 256^2 x 64: its loads need the extra warps in flight).
template <int NS, typename ST>
constexpr int reg_lanes() { return (NS >= 64 && sizeof(ST) >= 8) ? 8 : 4; }
constexpr int reg_min_blocks(int G) { return G == 8 ? 6 : 4; }

__device__ __forceinline__ float2 shfl_c(float2 v, int lane) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, lane), __shfl_sync(0xffffffffu, v.y, lane));
}
__device__ __forceinline__ float2 shfl_xor_c(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ double2 shfl_c(double2 v, int lane) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, lane), __shfl_sync(0xffffffffu, v.y, lane));
}
__device__ __forceinline__ dd shfl_c(dd v, int lane) {
    return dd(__shfl_sync(0xffffffffu, v.hi, lane), __shfl_sync(0xffffffffu, v.lo, lane));
}
__device__ __forceinline__ dd2 shfl_c(dd2 v, int lane) { return c2(shfl_c(v.x, lane), shfl_c(v.y, lane)); }


// Columns of the register kernel for a fixed order ORD (1..6), or ORD = 0 for
// the plan's order read at run time (at most 6).  ADV: complex a_j E^j
// (advection); otherwise real.
template <int NS, int G, typename ST, bool REAL, bool ADV, int ORD, int PER, bool XF>
__device__ __forceinline__ void reg_columns(const TimeArgs& A, unsigned char* stage_raw,
                                            const float2* tw, const float2* wfull, const float2* lamp, const ST* gam,
                                            const ST* osc, float (&accs)[PER], float (&accx)[PER]) {
    typedef typename cplx<ST>::t ST2;
    typedef typename std::conditional<REAL, ST, ST2>::type SE;
    constexpr int R = NS / G;
    constexpr int LOGR = ilog2_ct(R), LOGG = ilog2_ct(G);
    constexpr int COLS = REG_THREADS / G;         // columns per CTA
    constexpr int WG = 32 / G;                    // groups per warp
    constexpr int V = R < WG ? WG : R;            // transpose-reduce width (padded)
    constexpr int JM = ORD ? ORD : 6;             // largest order this body handles
    constexpr int NWIN = (G - 1 + JM) / G + 1;    // iterate window (slots j, j-1, ..)
    constexpr int ESZ = (int)sizeof(SE);
    static_assert(PER == V / WG, "per-lane reduction slots");
    const int tid = threadIdx.x, lane = tid & 31;
    const int g = lane & (G - 1);        // slice residue of this lane
    const int gl0 = lane & ~(G - 1);     // first lane of the group
    const long long Mcol = A.Mcol;
    const ST bdt = (ST)A.bdt, sigR = (ST)A.sigR;
    const int order = ORD ? ORD : A.order;
    const float one = (float)(1.0 - A.dshift);
    const int k2R = (int)bitrev((unsigned)g, LOGG) * R;  // spectral block of this lane
    // staging slots [slot][thread]: X, then N(u), then F on the slots j < RF
    // only (F is zero from slice f_slices on)
    const int RF = A.F ? min(R, (A.f_slices + G - 1) / G) : 0;
    // XF: the iterate comes from A.X32 in float32 (staged as such) and X + s
    // goes to A.X
    typedef typename std::conditional<REAL, float, float2>::type XE32;
    typedef typename std::conditional<XF, XE32, SE>::type XS;
    constexpr int XSZ = (int)sizeof(XS);
    const bool hasX = XF || A.X != nullptr;
    XS* stage_x = reinterpret_cast<XS*>(stage_raw);
    SE* stage = reinterpret_cast<SE*>(stage_raw + (hasX ? (size_t)R * REG_THREADS * XSZ : 0));
    const int sn = 0, sf = sn + (A.NL ? R : 0);
    const void* xsrc = XF ? A.X32 : A.X;
    auto ldx = [&](int j) -> ST2 {
        if constexpr (XF) {
            if constexpr (REAL) return c2(ST(stage_x[j * REG_THREADS + tid]), (ST)0);
            else return cvt2<ST2>(stage_x[j * REG_THREADS + tid]);
        } else {
            return ldcol<ST, REAL>(stage_x, j * REG_THREADS + tid);
        }
    };
    for (long long base = (long long)blockIdx.x * COLS; base < Mcol; base += (long long)gridDim.x * COLS) {
        const long long m = base + (tid / G);
        const bool valid = m < Mcol;
        const long long mm = valid ? m : 0;
        typedef typename std::conditional<ADV, ST2, ST>::type CS;
        typedef typename std::conditional<ADV, float2, float>::type CP;
        CS cs[JM + 1];
        CP cp[JM + 1];
#pragma unroll
        for (int j = 1; j <= JM; ++j) {
            cs[j] = (valid && j <= order) ? coef<CS>(A, j, mm) : coef_zero<CS>();
            cp[j] = (valid && j <= order) ? coef<CP>(A, j, mm) : coef_zero<CP>();
        }
        const float wgt = valid ? (float)mode_weight<float>(mm, A.KX, A.NX, A.realcol) : 0.0f;
        // ---- stage the column slices: every load of the tile in flight at once ----
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const long long gi = (long long)(G * j + g) * Mcol + mm;
            if (hasX) cp_async_elem<XSZ>(&stage_x[j * REG_THREADS + tid], static_cast<const XS*>(xsrc) + gi, valid);
            if (A.NL) cp_async_elem<ESZ>(&stage[(sn + j) * REG_THREADS + tid], static_cast<const SE*>(A.NL) + gi, valid);
            if (j < RF)  // zero-filled beyond the right-hand side's nonzero slices
                cp_async_elem<ESZ>(&stage[(sf + j) * REG_THREADS + tid], static_cast<const SE*>(A.F) + gi,
                                   valid && G * j + g < A.f_slices);
        }
        cp_async_wait_all();  // each thread reads back only its own elements
        // ---- residual q_n for n = G j + g, times Gamma_alpha ----
        float2 w[R];
        ST2 xw[NWIN];  // xw[d] = iterate at slot j - d of this lane
#pragma unroll
        for (int d = 0; d < NWIN; ++d) xw[d] = c2((ST)0, (ST)0);
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int n = G * j + g;
            ST2 q = c2((ST)0, (ST)0);
#pragma unroll
            for (int d = NWIN - 1; d >= 1; --d) xw[d] = xw[d - 1];
            xw[0] = c2((ST)0, (ST)0);
            if (hasX) xw[0] = ldx(j);
            if (j < RF) q = ldcol<ST, REAL>(stage, (sf + j) * REG_THREADS + tid);
            if (A.NL) {
                const ST2 v = ldcol<ST, REAL>(stage, (sn + j) * REG_THREADS + tid);
                q.x = fma(bdt, v.x, q.x);
                q.y = fma(bdt, v.y, q.y);
            }
            if (hasX) {
                ST2 rx = xw[0];
#pragma unroll
                for (int i = 1; i <= JM; ++i) {
                    if (ORD || i <= order) {  // warp-uniform
                        // x at slice n - i lives in lane (g - i) mod G at slot j - (g' + i) / G
                        const int gs = (g - i) & (G - 1);
                        const int dsend = (g + i) / G;  // what this lane sends, as a source
                        ST2 send = xw[0];
#pragma unroll
                        for (int d = 1; d < NWIN; ++d)
                            if (dsend == d) send = xw[d];
                        ST2 xv = shfl_c(send, gl0 + gs);
                        if (n - i < 0) xv = c2((ST)0, (ST)0);  // before the window: in F
                        rx = sub_cx(rx, cs[i], xv);
                    }
                }
                q.x = fma(sigR, rx.x, q.x);
                q.y = fma(sigR, rx.y, q.y);
            }
            w[j] = cvt2<float2>(cscale(q, gam[n]));
        }
        // ---- Step (a): Y[k1 + R k2] = sum_n y_n e^{+2 pi i kn/NS} ----
        reg_fft_dif<R, G, +1>(w, tw);  // slot p: k1 = bitrev_R(p)
#pragma unroll
        for (int p = 0; p < R; ++p) {
            const int k1 = (int)bitrev((unsigned)p, LOGR);
            if (p != 0) w[p] = cmul(w[p], wfull[g * k1]);
        }
        // DIF across the group's lanes: the lower lane of a pair keeps a + b,
        // the upper one (a - b) w; the last stage's twiddle is 1
#pragma unroll
        for (int h = G / 2; h >= 1; h >>= 1) {
            const bool up = (g & h) != 0;
            const float sg = up ? -1.0f : 1.0f;
            const float2 tw2 = up ? wfull[(g & (h - 1)) * (NS / (2 * h))] : make_float2(1.0f, 0.0f);
#pragma unroll
            for (int p = 0; p < R; ++p) {
                const float2 o = shfl_xor_c(w[p], h);
                const float2 t = make_float2(fmaf(sg, w[p].x, o.x), fmaf(sg, w[p].y, o.y));
                w[p] = h > 1 ? cmul(t, tw2) : t;
            }
        }
        // ---- Step (b): divide by d_k = 1 - sum_j cp_j lambda_k^j ----
        // (lambda_k^j from the CTA's table; d_k is the scheme's characteristic
        // polynomial at |z| = alpha^(1/Ns) < 1, bounded away from 0 and infinity
        // for the zero-stable BDF-s, so |d_k|^2 lies in the range where the
        // approximate reciprocal is within 2 ulp)
#pragma unroll
        for (int p = 0; p < R; ++p) {
            const int k = (int)bitrev((unsigned)p, LOGR) + k2R;
            float2 d = make_float2(one, 0.0f);
#pragma unroll
            for (int j = 1; j <= JM; ++j)
                if (ORD || j <= order) d = sub_cx(d, cp[j], lamp[(j - 1) * NS + k]);
            const float inv = __fdividef(1.0f, fmaf(d.x, d.x, d.y * d.y));
            w[p] = cscale(cmulc(w[p], d), inv);
        }
        // ---- Step (c): z_n = sum_k Z_k e^{-2 pi i kn/NS} ----
        // DIT across the group's lanes: the upper lane of a pair applies its
        // twiddle before the exchange, then lower = a + b w, upper = a - b w
#pragma unroll
        for (int h = 1; h < G; h <<= 1) {
            const bool up = (g & h) != 0;
            const float sg = up ? -1.0f : 1.0f;
            float2 tw2 = up ? wfull[(g & (h - 1)) * (NS / (2 * h))] : make_float2(1.0f, 0.0f);
            tw2.y = -tw2.y;
#pragma unroll
            for (int p = 0; p < R; ++p) {
                const float2 v = h > 1 ? cmul(w[p], tw2) : w[p];
                const float2 o = shfl_xor_c(v, h);
                w[p] = make_float2(fmaf(sg, v.x, o.x), fmaf(sg, v.y, o.y));
            }
        }
#pragma unroll
        for (int p = 0; p < R; ++p) {
            const int k1 = (int)bitrev((unsigned)p, LOGR);
            if (p != 0) w[p] = cmulc(w[p], wfull[g * k1]);
        }
        reg_fft_dit<R, G, -1>(w, tw);  // slot j: z_{G j + g}
        // ---- update (or output) and per-element norm terms ----
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int n = G * j + g;
            const ST2 sv = cscale(cvt2<ST2>(w[j]), osc[n]);
            const long long gi = (long long)n * Mcol + mm;
            float ns = 0.0f, nx = 0.0f;
            if (valid) {
                if (A.accum) {
                    const ST2 xn = cadd(ldx(j), sv);
                    stcol<ST, REAL>(const_cast<void*>(A.X), gi, xn);
                    const float2 xf = cvt2<float2>(xn);
                    nx = wgt * fmaf(xf.x, xf.x, xf.y * xf.y);
                } else {
                    stcol<ST, REAL>(A.out, gi, sv);
                }
                const float2 sf = cvt2<float2>(sv);
                if (A.sout) stcol<float, REAL>(A.sout, gi, sf);
                ns = wgt * fmaf(sf.x, sf.x, sf.y * sf.y);
            }
            w[j] = make_float2(ns, nx);
        }
        // ---- transpose-reduce over the warp's groups (lane bits >= LOGG) ----
        float vs[V], vx[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            vs[i] = i < R ? w[i].x : 0.0f;
            vx[i] = i < R ? w[i].y : 0.0f;
        }
#pragma unroll
        for (int st = 0; st < 5 - LOGG; ++st) {
            const int off = 16 >> st, len = (V / 2) >> st;
            const bool upper = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < len; ++i) {
                // lanes with this bit clear keep slots [0, len), the others [len, 2 len)
                const float ss = upper ? vs[i] : vs[i + len], sk = upper ? vs[i + len] : vs[i];
                const float xs = upper ? vx[i] : vx[i + len], xk = upper ? vx[i + len] : vx[i];
                vs[i] = sk + __shfl_xor_sync(0xffffffffu, ss, off);
                vx[i] = xk + __shfl_xor_sync(0xffffffffu, xs, off);
            }
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            accs[i] += vs[i];
            accx[i] += vx[i];
        }
    }
}

template <int NS, int G, typename ST, bool REAL, bool ADV, int ORD, bool XF>
__global__ void __launch_bounds__(REG_THREADS, reg_min_blocks(G)) time_reg_kernel(TimeArgs A) {
    typedef typename cplx<ST>::t ST2;
    typedef typename std::conditional<REAL, ST, ST2>::type SE;
    constexpr int R = NS / G;
    constexpr int WG = 32 / G;
    constexpr int V = R < WG ? WG : R;
    constexpr int PER = V / WG;
    constexpr int NW = REG_THREADS / 32;
    // staging of this thread's X, N(u) and F elements: [slot][thread]
    extern __shared__ __align__(16) unsigned char stage_raw[];
    __shared__ float2 tw[NS / 2];    // exp(-2 pi i k/NS)
    __shared__ float2 wfull[NS];     // exp(+2 pi i k/NS)
    __shared__ float2 lamp[6 * NS];  // lambda_k^j, j = 1..6
    __shared__ ST gam[NS], osc[NS];
    __shared__ float red[NW][2][NS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane & (G - 1);
    for (int i = tid; i < NS / 2; i += REG_THREADS) {
        const float2 t = static_cast<const float2*>(A.tw)[i];
        tw[i] = t;
        wfull[i] = make_float2(t.x, -t.y);
        wfull[i + NS / 2] = make_float2(-t.x, t.y);
    }
    for (int i = tid; i < NS; i += REG_THREADS) {
        const float2 l = static_cast<const float2*>(A.lam)[i];
        float2 pw = l;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            lamp[j * NS + i] = pw;
            pw = cmul(pw, l);
        }
        gam[i] = static_cast<const ST*>(A.gam)[i];
        osc[i] = static_cast<const ST*>(A.osc)[i];
    }
    for (int i = tid; i < NW * 2 * NS; i += REG_THREADS) (&red[0][0][0])[i] = 0.0f;
    pdl_wait();  // the iterate and N(u) come from the previous kernels
    __syncthreads();
    float accs[PER], accx[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) accs[i] = accx[i] = 0.0f;
    reg_columns<NS, G, ST, REAL, ADV, ORD, PER, XF>(A, stage_raw, tw, wfull, lamp, gam, osc, accs, accx);
    // lane (group c, residue g) holds slots j = c * PER + i of slice G j + g
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int j = (lane / G) * PER + i;
        if (j < R) {
            red[warp][0][G * j + g] = accs[i];
            red[warp][1][G * j + g] = accx[i];
        }
    }
    __syncthreads();
    for (int n = tid; n < NS; n += REG_THREADS) {
        float a = 0.0f, b = 0.0f;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            a += red[q][0][n];
            b += red[q][1][n];
        }
        A.partial[(size_t)n * gridDim.x + blockIdx.x] = make_double2((double)a, (double)b);
    }
}

template <int NS, typename ST, bool REAL, bool ADV>
expd_status launch_reg(expd_plan p, TimeArgs& a, cudaStream_t s) {
    const TimeTables& ts = std::is_same<ST, float>::value ? p->t32 : p->t64;
    a.gam = std::is_same<ST, dd>::value ? p->gamdd : ts.gam;
    a.osc = std::is_same<ST, dd>::value ? p->oscdd : ts.osc;
    a.lam = p->t32.lam;
    a.tw = p->t32.tw;
    constexpr bool DDS = std::is_same<ST, dd>::value;
    const bool xf = DDS && a.X32 != nullptr;  // iterate read in float32 (double-float storage only)
    if (a.X32 && !DDS) return expd_fail(EXPD_ERR_INVALID_ARG, "a float32 iterate input needs double-float storage");
    constexpr int G = reg_lanes<NS, ST>();
    constexpr int cols = REG_THREADS / G;
    long long grid = (p->Mcol + cols - 1) / cols;
    if (grid > p->partial_cap) grid = p->partial_cap;
    const double esz = (REAL ? 1.0 : 2.0) * sizeof(ST);
    const double xsz = xf ? (REAL ? 4.0 : 8.0) : esz;  // the iterate's element as read
    const bool hasX = a.X != nullptr;
    const double ffrac = (double)a.f_slices / p->Ns;  // F is read only where it can be nonzero
    const double per = (hasX ? xsz : 0.0) + (a.F ? esz * ffrac : 0.0) + (a.NL ? esz : 0.0) + esz +
                       (a.sout ? (REAL ? 4.0 : 8.0) : 0.0);  // N stored like X
    const double fl_col = 2.0 * 5.0 * NS * ilog2(NS) + 8.0 * p->order * NS + 4.0 * p->order * NS;
    const int cls = sizeof(ST) == 4 ? EXPD_K_TIME32 : DDS ? EXPD_K_TIMEDD : EXPD_K_TIME;
    KProf kp(p, s, cls, per * NS * (double)p->Mcol, fl_col * (double)p->Mcol);
    constexpr int R = NS / G;
    const int RF = a.F ? std::min(R, (a.f_slices + G - 1) / G) : 0;  // F slots that can be nonzero
    const size_t smem = std::max<size_t>(
        (size_t)(hasX ? R : 0) * REG_THREADS * (size_t)xsz + (size_t)((a.NL ? R : 0) + RF) * REG_THREADS * (size_t)esz,
        (size_t)REG_THREADS * (size_t)esz);
    // order 1 (exponential Euler) has a kernel of its own; the others share one
    auto kern = p->order == 1 ? time_reg_kernel<NS, G, ST, REAL, ADV, 1, false> : time_reg_kernel<NS, G, ST, REAL, ADV, 0, false>;
    if constexpr (DDS) {
        if (xf) kern = p->order == 1 ? time_reg_kernel<NS, G, ST, REAL, ADV, 1, true> : time_reg_kernel<NS, G, ST, REAL, ADV, 0, true>;
    }
    EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    EXPD_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(REG_THREADS), smem, s, a));
    p->time_grid_used = (int)grid;
    return EXPD_OK;
}

template <typename ST, bool REAL, bool ADV>
expd_status launch_reg_ns(expd_plan p, TimeArgs& a, cudaStream_t s) {
    switch (p->Ns) {
        case 16: return launch_reg<16, ST, REAL, ADV>(p, a, s);
        case 32: return launch_reg<32, ST, REAL, ADV>(p, a, s);
        case 64: return launch_reg<64, ST, REAL, ADV>(p, a, s);
    }
    return expd_fail(EXPD_ERR_UNSUPPORTED, "register time kernel needs Ns in {16, 32, 64}");
}

}  // namespace

bool time_reg_usable(expd_plan p) { return (p->Ns == 16 || p->Ns == 32 || p->Ns == 64) && !p->no_reg_time; }

expd_status time_reg_launch(expd_plan p, TimeArgs& a, int st, cudaStream_t s) {
    if (st == 1)
        return p->realcol ? launch_reg_ns<float, true, false>(p, a, s)
               : p->adv   ? launch_reg_ns<float, false, true>(p, a, s)
                          : launch_reg_ns<float, false, false>(p, a, s);
    if (st == 2)
        return p->realcol ? launch_reg_ns<dd, true, false>(p, a, s)
               : p->adv   ? launch_reg_ns<dd, false, true>(p, a, s)
                          : launch_reg_ns<dd, false, false>(p, a, s);
    return p->realcol ? launch_reg_ns<double, true, false>(p, a, s)
           : p->adv   ? launch_reg_ns<double, false, true>(p, a, s)
                      : launch_reg_ns<double, false, false>(p, a, s);
}
