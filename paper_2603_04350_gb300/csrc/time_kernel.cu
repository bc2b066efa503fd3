// Time direction of the hot path, in L_h's eigenbasis where every spatial mode m
// decouples into one column of Ns time values.  One fused kernel computes, per
// column,
//
//   q_n  = F_n + bdt*NL_n + sigR*(X_n - sum_{j=1..s, n-j>=0} a_j E_m^j X_{n-j})
//          (the all-at-once residual f_s + beta dt N(v) - R_s v of Eq. (3.2),
//           or R_s X for the GMRES operator; float64)
//   s    = (R_s^alpha)^{-1} q by Eq. (3.3) / Eq. (4.5):
//          Step (a)  Y_k = sum_n alpha^(n/Ns) q_n e^{+2 pi i kn/Ns}
//          Step (b)  Z_k = Y_k / (1 - sum_j a_j (lambda_k E_m)^j),
//                    lambda_k = alpha^(1/Ns) e^{2 pi i k/Ns}  (Sec. 2, Sec. 4)
//          Step (c)  s_n = alpha^(-n/Ns) (1/Ns) sum_k Z_k e^{-2 pi i kn/Ns}
//   X   += s (Richardson update, Eq. (3.2) / Eq. (4.4)) or out = s
//
// and accumulates per-slice norms of s and of the updated X.
//
// Layout: the eigen arrays are [Ns][Mcol] (slice-major).  A CTA owns a tile of
// EXPD_TIME_COLS consecutive modes and all Ns slices: the tile is loaded with
// coalesced reads along the mode index into shared memory, each warp then
// transforms one column in shared memory (radix-2 FFT for power-of-two Ns,
// Bluestein's chirp-z with a power-of-two length otherwise), and the tile is
// written back coalesced.  On Dirichlet grids the columns are real and one warp
// solves two of them as one complex column (precond_column_pair: the FFT work
// of one column for two).  The grid is a multiple of the SM count and loops
// over tiles in a fixed order, so the per-slice norm partials are deterministic.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include <type_traits>

#include "common.cuh"
#include "dd.cuh"
#include "plan.h"
#include "time_args.cuh"
#include "time_column.cuh"

namespace {

using namespace expd_time;

// PT: precision of steps (a)-(c); ST: precision of the stored state, the
// right-hand side and the residual arithmetic (float32 sweeps never touch the
// float64 pipe, whose rate on GB300 is 1/64 of float32).
template <typename PT, typename ST, bool REAL, bool ADV>
__global__ void __launch_bounds__(32 * EXPD_TIME_COLS, 3) time_kernel(TimeArgs A) {
    typedef typename cplx<PT>::t PT2;
    typedef typename cplx<ST>::t ST2;
    constexpr int C = EXPD_TIME_COLS;
    const int Ns = A.Ns, L = A.L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // ---- shared-memory carve-up (C even keeps every region 16-byte aligned) ----
    // tiles are column-major with a padded column stride P = Ns + 1, so the
    // per-column phase (a warp walking one column) is free of bank conflicts
    const int P = Ns + 1;
    ST2* sAcc = reinterpret_cast<ST2*>(smem_raw);             // [Ns + 1]
    ST2* sX = sAcc + (Ns + 1);                                 // [C][P]
    ST2* sR = sX + (size_t)P * C;                              // [C][P]
    ST* sWgt = reinterpret_cast<ST*>(sR + (size_t)P * C);     // [C] norm weight of each column
    PT2* sW = reinterpret_cast<PT2*>(sWgt + 2 * C);           // [C][L]
    PT2* tw = sW + (size_t)C * L;                              // [L/2]
    PT2* lam = tw + ((L >> 1) + 1);                            // [Ns]
    PT2* chirp = lam + (Ns + 1);                               // [Ns]   (Bluestein)
    PT2* bp = chirp + (A.bluestein ? Ns + 1 : 0);              // [L]
    PT2* bm = bp + (A.bluestein ? L : 0);                      // [L]
    ST* gam = reinterpret_cast<ST*>(bm + (A.bluestein ? L : 0));  // [Ns]
    ST* osc = gam + Ns;                                        // [Ns]

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
    pdl_wait();
    __syncthreads();

    const int lane = tid & 31, warp = tid >> 5;
    const long long Mcol = A.Mcol;
    const ST bdt = (ST)A.bdt, sigR = (ST)A.sigR;
    for (long long tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const long long m0 = tile * C;
        // ---- coalesced load of the tile: X and the additive right-hand side ----
        for (int idx = tid; idx < Ns * C; idx += nth) {
            const int n = idx / C, c = idx - n * C;
            const long long m = m0 + c;
            ST2 x = c2((ST)0, (ST)0), r = c2((ST)0, (ST)0);
            if (m < Mcol) {
                const long long g = (long long)n * Mcol + m;
                if (A.X) x = ldcol<ST, REAL>(A.X, g);
                if (A.F && n < A.f_slices) r = ldcol<ST, REAL>(A.F, g);
                if (A.NL) {
                    const ST2 v = ldnl<ST, REAL>(A.NL, g, A.nl_f32);
                    r.x = fma(bdt, v.x, r.x);
                    r.y = fma(bdt, v.y, r.y);
                }
            }
            sX[c * P + n] = x;
            sR[c * P + n] = r;
        }
        if (tid < C) {
            const long long m = m0 + tid;
            sWgt[tid] = m < Mcol ? mode_weight<ST>(m, A.KX, A.NX, A.realcol) : (ST)0;
        }
        __syncthreads();

        if (REAL && !ADV && A.precond) {
            // ---- real columns (Dirichlet): one warp per two columns, packed as
            // one complex column (precond_column_pair) ----
            const int ca = 2 * warp;
            const long long ma = m0 + ca, mb = ma + 1;
            if (ca < C && ma < Mcol) {
                const bool hasb = ca + 1 < C && mb < Mcol;
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
                const ST2* xa = sX + (size_t)ca * P;
                ST2* ra = sR + (size_t)ca * P;
                auto qcol = [&](const ST2* xc, const ST2* rc, const ST* cs, int n) {
                    ST2 q = rc[n];
                    if (A.X) {
                        ST2 rx = xc[n];
#pragma unroll
                        for (int j = 1; j <= 6; ++j) {
                            if (j <= A.order && j <= n) rx = sub_cx(rx, cs[j], xc[n - j]);
                        }
                        q.x = fma(sigR, rx.x, q.x);
                    }
                    return q.x;
                };
                for (int n = lane; n < Ns; n += 32) {
                    const ST qa = qcol(xa, ra, csa, n);
                    const ST qb = hasb ? qcol(xa + P, ra + P, csb, n) : (ST)0;
                    w[A.bluestein ? n : (int)bitrev(n, A.log2L)] = cvt2<PT2>(cscale(c2(qa, qb), gam[n]));
                }
                EXPD_SYNCWARP();
                precond_column_pair<PT, PT2>(w, Ns, L, A.log2L, A.bluestein, tw, lam, chirp, bp, bm, cpa, cpb,
                                             A.order, lane, 32, (PT)(1.0 - A.dshift));
                for (int n = lane; n < Ns; n += 32) {
                    const ST2 v = cscale(cvt2<ST2>(w[A.bluestein ? n : (int)bitrev(n, A.log2L)]), osc[n]);
                    ra[n] = c2(v.x, (ST)0);
                    if (hasb) ra[P + n] = c2(v.y, (ST)0);
                }
            }
        } else {
        // ---- one warp per column ----
        const long long m = m0 + warp;
        if (warp < C && m < Mcol) {
            // a_j E_m^j from the plan's tables (no float64 arithmetic here)
            typedef typename std::conditional<ADV, ST2, ST>::type CS;
            typedef typename std::conditional<ADV, PT2, PT>::type CP;
            CS cs[7];
            CP cp[7];
            cs[0] = coef_zero<CS>();
            cp[0] = coef_zero<CP>();
#pragma unroll
            for (int j = 1; j <= 6; ++j) {
                cs[j] = j <= A.order ? coef<CS>(A, j, m) : coef_zero<CS>();
                cp[j] = j <= A.order ? coef<CP>(A, j, m) : coef_zero<CP>();
            }
            PT2* w = sW + (size_t)warp * L;
            const ST2* xc = sX + (size_t)warp * P;
            ST2* rc = sR + (size_t)warp * P;
            // residual-type combination q_n in ST, then Gamma_alpha
            for (int n = lane; n < Ns; n += 32) {
                ST2 q = rc[n];
                if (A.X) {
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
                    w[A.bluestein ? n : (int)bitrev(n, A.log2L)] = cvt2<PT2>(cscale(q, gam[n]));
                }
            }
            if (A.precond) {
                EXPD_SYNCWARP();
                precond_column<PT, PT2, CP>(w, Ns, L, A.log2L, A.bluestein, tw, lam, chirp, bp, bm, cp, A.order, lane,
                                            32, (PT)(1.0 - A.dshift));
                for (int n = lane; n < Ns; n += 32) {
                    const ST2 v = cvt2<ST2>(w[A.bluestein ? n : (int)bitrev(n, A.log2L)]);
                    rc[n] = cscale(v, osc[n]);
                }
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
                    stcol<ST, REAL>(const_cast<void*>(A.X), g, xn);
                    nrm.y = wgt * fma(xn.x, xn.x, xn.y * xn.y);
                    if (A.sout) stcol<float, REAL>(A.sout, g, cvt2<float2>(res));
                } else {
                    stcol<ST, REAL>(A.out, g, res);
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

// Per-slice totals over the time kernel's CTAs: block n sums slice n's
// partials in a fixed order (four independent strided accumulators per thread,
// a shuffle tree, then the warps in order), so the totals are deterministic.
// The totals go to device memory (for the device-side stopping test) and to
// host-mapped memory (the host loop reads them there without a copy).
__global__ void __launch_bounds__(256) reduce_kernel(const double2* __restrict__ partial, int grid,
                                                     double2* __restrict__ slice_tot, double2* host_tot) {
    __shared__ double2 red[8];
    pdl_wait();
    const int n = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double2* src = partial + (size_t)n * grid;
    double a[4] = {0, 0, 0, 0}, b[4] = {0, 0, 0, 0};
    int g = threadIdx.x;
    for (; g + 3 * 256 < grid; g += 4 * 256) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const double2 v = src[g + u * 256];
            a[u] += v.x;
            b[u] += v.y;
        }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {
        if (g + u * 256 < grid) {
            const double2 v = src[g + u * 256];
            a[u] += v.x;
            b[u] += v.y;
        }
    }
    double x = (a[0] + a[1]) + (a[2] + a[3]), y = (b[0] + b[1]) + (b[2] + b[3]);
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) red[warp] = make_double2(x, y);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int w = 0; w < 8; ++w) {
            t.x += red[w].x;
            t.y += red[w].y;
        }
        slice_tot[n] = t;
        if (host_tot) host_tot[n] = t;
    }
}

size_t time_smem_bytes(int Ns, int L, int bluestein, size_t pt2, size_t st) {
    const int C = EXPD_TIME_COLS;
    size_t b = (size_t)(Ns + 1) * 2 * st + 2 * (size_t)(Ns + 1) * C * 2 * st + 2 * (size_t)C * st;
    b += (size_t)C * L * pt2 + (size_t)((L >> 1) + 1) * pt2 + (size_t)(Ns + 1) * pt2;
    if (bluestein) b += (size_t)(Ns + 1) * pt2 + 2 * (size_t)L * pt2;
    b += 2 * (size_t)Ns * st;
    return b;
}

template <typename PT, typename ST, bool REAL, bool ADV>
expd_status launch_time(expd_plan p, TimeArgs& a, cudaStream_t s) {
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
    const size_t smem = time_smem_bytes(p->Ns, t.L, t.bluestein, sizeof(typename cplx<PT>::t), sizeof(ST));
    auto kern = time_kernel<PT, ST, REAL, ADV>;
    EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    const double esz = (REAL ? 1.0 : 2.0) * sizeof(ST);
    const double nlsz = (REAL ? 1.0 : 2.0) * (a.nl_f32 ? 4.0 : 8.0);
    const double ffrac = (double)a.f_slices / p->Ns;
    const double per = (a.X ? esz : 0.0) + (a.F ? esz * ffrac : 0.0) + (a.NL ? nlsz : 0.0) + esz;
    const double lg = (double)t.log2L;
    const double fl_col = (a.precond ? (t.bluestein ? 4.0 : 2.0) * 5.0 * t.L * lg + 8.0 * p->order * p->Ns : 0.0) +
                          4.0 * p->order * p->Ns;
    const int cls = sizeof(ST) == 4 ? EXPD_K_TIME32 : std::is_same<ST, dd>::value ? EXPD_K_TIMEDD : EXPD_K_TIME;
    KProf kp(p, s, cls, per * p->Ns * (double)p->Mcol, fl_col * (double)p->Mcol);
    EXPD_CUDA_TRY(launch_pdl(kern, dim3(p->time_grid), dim3(32 * EXPD_TIME_COLS), smem, s, a));
    p->time_grid_used = p->time_grid;
    return EXPD_OK;
}

template <typename T2, typename T>
void* upload(expd_plan p, const std::vector<std::complex<double>>& v, cudaStream_t s, size_t& bytes, expd_status& st) {
    std::vector<T2> h(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        h[i].x = (T)v[i].real();
        h[i].y = (T)v[i].imag();
    }
    void* d = nullptr;
    cudaError_t e = plan_malloc(p, &d, h.size() * sizeof(T2) + 16);
    if (e != cudaSuccess) {
        st = expd_cuda_fail(e, "cudaMalloc(time table)", __FILE__, __LINE__);
        return nullptr;
    }
    bytes += h.size() * sizeof(T2) + 16;
    e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = expd_cuda_fail(e, "cudaMemcpyAsync(time table)", __FILE__, __LINE__);
    return d;
}

template <typename T2, typename T>
expd_status build_tables(expd_plan p, TimeTables& t, cudaStream_t s) {
    const TimeTablesHost h = time_tables_host(p->Ns, p->alpha);
    t.L = h.L;
    t.log2L = h.log2L;
    t.bluestein = h.bluestein;
    expd_status st = EXPD_OK;
    t.tw = upload<T2, T>(p, h.tw, s, p->bytes, st);
    if (st == EXPD_OK) t.lam = upload<T2, T>(p, h.lam, s, p->bytes, st);
    if (st == EXPD_OK && t.bluestein) t.chirp = upload<T2, T>(p, h.chirp, s, p->bytes, st);
    if (st == EXPD_OK && t.bluestein) t.bplus = upload<T2, T>(p, h.bplus, s, p->bytes, st);
    if (st == EXPD_OK && t.bluestein) t.bminus = upload<T2, T>(p, h.bminus, s, p->bytes, st);
    if (st != EXPD_OK) return st;
    // Gamma_alpha and the output scale in this table's precision
    std::vector<T> g(h.gamma.size()), o(h.gamma.size());
    const double extra = h.bluestein ? 1.0 / ((double)h.L * (double)h.L) : 1.0;
    for (size_t n = 0; n < g.size(); ++n) {
        g[n] = (T)h.gamma[n];
        o[n] = (T)(extra / ((double)p->Ns * h.gamma[n]));
    }
    for (int k = 0; k < 2; ++k) {
        void** dst = k == 0 ? &t.gam : &t.osc;
        const std::vector<T>& src = k == 0 ? g : o;
        cudaError_t e = plan_malloc(p, dst, src.size() * sizeof(T));
        if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMalloc(gamma)", __FILE__, __LINE__);
        p->bytes += src.size() * sizeof(T);
        e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMemcpyAsync(gamma)", __FILE__, __LINE__);
    }
    return EXPD_OK;
}

}  // namespace

expd_status time_tables_build(expd_plan p, cudaStream_t s) {
    expd_status st = build_tables<double2, double>(p, p->t64, s);
    if (st != EXPD_OK) return st;
    st = build_tables<float2, float>(p, p->t32, s);
    if (st != EXPD_OK) return st;
    int grid = 0;
    st = time_grid_for(p, &grid);
    if (st != EXPD_OK) return st;
    p->time_grid = grid;
    p->partial_cap = std::max(grid, p->sm_count * 8);
    cudaError_t e = plan_malloc(p, reinterpret_cast<void**>(&p->partial), (size_t)p->partial_cap * p->Ns * sizeof(double2));
    if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMalloc(partial)", __FILE__, __LINE__);
    p->bytes += (size_t)p->partial_cap * p->Ns * sizeof(double2);
    return EXPD_OK;
}

expd_status time_grid_for(expd_plan p, int* grid_out) {
    // a multiple of the SM count, as many CTAs as fit, never more than tiles
    const long long ntiles = (p->Mcol + EXPD_TIME_COLS - 1) / EXPD_TIME_COLS;
    int L = 1;
    while (L < p->Ns) L <<= 1;
    const int blue = (L != p->Ns);
    if (blue) {
        L = 1;
        while (L < 2 * p->Ns - 1) L <<= 1;
    }
    int per_sm = 1;
    const size_t smem64 = time_smem_bytes(p->Ns, L, blue, sizeof(double2), sizeof(double));
    if (smem64 > 227 * 1024) return expd_fail(EXPD_ERR_UNSUPPORTED, "time window too long for shared memory");
    // the float32-sweep variant (the most frequent launch) sets the grid
    const size_t smem = time_smem_bytes(p->Ns, L, blue, sizeof(float2), sizeof(float));
    auto kern = p->realcol ? time_kernel<float, float, true, false> : time_kernel<float, float, false, false>;
    EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    EXPD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * EXPD_TIME_COLS, smem));
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)p->sm_count * per_sm;
    if (grid > ntiles) grid = ntiles;
    *grid_out = (int)grid;
    return EXPD_OK;
}

void time_tables_free(expd_plan p) {
    TimeTables* ts[2] = {&p->t64, &p->t32};
    for (TimeTables* t : ts) {
        for (void* b : {t->gam, t->osc, t->lam, t->tw, t->chirp, t->bplus, t->bminus}) plan_free(p, b);
        *t = TimeTables();
    }
}

expd_status time_apply(expd_plan p, const TimeOp& op, cudaStream_t s) {
    TimeArgs a;
    a.X = op.X;
    a.F = op.F;
    a.NL = op.NL;
    a.out = op.out;
    a.nl_f32 = op.nl_f32;
    a.bdt = op.bdt;
    a.sigR = op.sigR;
    a.precond = op.precond;
    a.accum = op.accum;
    a.Mcol = p->Mcol;
    a.Ns = p->Ns;
    a.order = p->order;
    a.C64 = p->C64;
    a.C32 = p->C32;
    a.Cdd = static_cast<const dd*>(p->Cdd);
    a.KX = p->KX;
    a.NX = p->NX;
    a.realcol = p->realcol;
    a.ntiles = (p->Mcol + EXPD_TIME_COLS - 1) / EXPD_TIME_COLS;
    a.partial = p->partial;
    a.sout = op.accum ? op.sout : nullptr;
    a.X32 = op.X32;
    a.dshift = op.dshift;
    a.f_slices = op.f_slices < 0 ? p->Ns : op.f_slices;
    a.norms = op.accum ? 1 : 0;
    p->dots_fused = 0;
    // the Krylov partials come from the real-column kernel (Dirichlet grids)
    // (float32 preconditioner on float64 storage: its scratch layout, time_real.cu)
    if (op.dots && !op.accum && op.precond && op.f32 && !op.st32 && p->realcol && !op.stdd && !p->no_real_time) {
        a.norms = 2;
        p->dots_fused = 1;
    }
    // power-of-two windows up to 64 with the float32 preconditioner: register kernel
    const bool reg = op.precond && op.f32 && (p->Ns == 16 || p->Ns == 32 || p->Ns == 64) && !p->no_reg_time;
    // (double-float storage included: with the right-hand side staged only on
    // its nonzero slices, 16-byte X and N elements measured 60 us against 96 us
    // for the shared-memory kernel on 256^2 x 64)
    if (reg && op.stdd) return time_reg_launch(p, a, 2, s);
    if (op.X32) return expd_fail(EXPD_ERR_INVALID_ARG, "a float32 iterate input needs the register time kernel");
    if (reg) {
        if (op.st32) {
            if (op.NL && !op.nl_f32) return expd_fail(EXPD_ERR_INVALID_ARG, "float32 storage needs float32 N");
            return time_reg_launch(p, a, 1, s);
        }
        if (!op.NL || !op.nl_f32) return time_reg_launch(p, a, 0, s);
    }
    // real columns, float32 preconditioner on float64 storage, Ns <= 128:
    // Steps (a) and (c) as tensor-core products (time_tc.cu)
    // (sigR exact in float32: the kernel's double-float combination scales by it)
    if (p->realcol && p->tt_tab && op.precond && op.f32 && !op.st32 && !op.stdd && !op.NL &&
        (double)(float)op.sigR == op.sigR)
        return time_tc_launch(p, a, s);
    if (p->realcol && !op.stdd && !p->no_real_time) {
        if (op.st32) {
            if (!op.f32) return expd_fail(EXPD_ERR_INVALID_ARG, "float32 storage needs the float32 preconditioner");
            if (op.NL && !op.nl_f32) return expd_fail(EXPD_ERR_INVALID_ARG, "float32 storage needs float32 N");
            return time_real_launch(p, a, 1, 1, s);
        }
        return time_real_launch(p, a, op.f32 ? 1 : 0, 0, s);
    }
    // complex columns with real coefficients: the fixed-length kernel (when its
    // tables fit one CTA's shared memory; the generic kernel otherwise)
    const int cst = op.stdd ? 2 : op.st32 ? 1 : 0;
    if (!p->realcol && !p->adv && !p->no_cplx_time && time_cplx_smem_bytes(p, cst) <= 227 * 1024) {
        if (op.stdd) {
            if (!op.f32) return expd_fail(EXPD_ERR_INVALID_ARG, "double-float storage needs the float32 preconditioner");
            return time_cplx_launch(p, a, 2, s);
        }
        if (op.st32) {
            if (!op.f32) return expd_fail(EXPD_ERR_INVALID_ARG, "float32 storage needs the float32 preconditioner");
            if (op.NL && !op.nl_f32) return expd_fail(EXPD_ERR_INVALID_ARG, "float32 storage needs float32 N");
            return time_cplx_launch(p, a, 1, s);
        }
        if (!op.f32) return time_cplx_launch(p, a, 0, s);
    }
    if (op.stdd) {
        if (!op.f32) return expd_fail(EXPD_ERR_INVALID_ARG, "double-float storage needs the float32 preconditioner");
        return p->realcol ? launch_time<float, dd, true, false>(p, a, s)
               : p->adv   ? launch_time<float, dd, false, true>(p, a, s)
                          : launch_time<float, dd, false, false>(p, a, s);
    }
    if (op.st32) {
        if (!op.f32) return expd_fail(EXPD_ERR_INVALID_ARG, "float32 storage needs the float32 preconditioner");
        if (op.NL && !op.nl_f32) return expd_fail(EXPD_ERR_INVALID_ARG, "float32 storage needs float32 N");
        return p->realcol ? launch_time<float, float, true, false>(p, a, s)
               : p->adv   ? launch_time<float, float, false, true>(p, a, s)
                          : launch_time<float, float, false, false>(p, a, s);
    }
    if (op.f32)
        return p->realcol ? launch_time<float, double, true, false>(p, a, s)
               : p->adv   ? launch_time<float, double, false, true>(p, a, s)
                          : launch_time<float, double, false, false>(p, a, s);
    return p->realcol ? launch_time<double, double, true, false>(p, a, s)
           : p->adv   ? launch_time<double, double, false, true>(p, a, s)
                      : launch_time<double, double, false, false>(p, a, s);
}

expd_status time_reduce(expd_plan p, cudaStream_t s) {
    const int grid = p->time_grid_used > 0 ? p->time_grid_used : p->time_grid;
    KProf kp(p, s, EXPD_K_REDUCE, 16.0 * grid * p->Ns, 2.0 * grid * p->Ns);
    double2* slice_tot = reinterpret_cast<double2*>(p->redout + 8);
    EXPD_CUDA_TRY(launch_pdl(reduce_kernel, dim3(p->Ns), dim3(256), 0, s, (const double2*)p->partial, grid, slice_tot,
                             reinterpret_cast<double2*>(p->redhost_dev)));
    return EXPD_OK;
}
