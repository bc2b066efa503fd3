// Argument block and element helpers shared by the time-direction kernels
// (the shared-memory kernel and the register-resident one live in separate
// translation units so that they compile in parallel).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "dd.cuh"
#include "plan.h"

namespace expd_time {

struct TimeArgs {
    const void* X;
    const void* F;
    const void* NL;
    void* out;
    void* sout;  // optional float32 copy of the update (accum mode)
    const void* X32;  // register kernel, double-float storage: the iterate read from float32 (X written)
    double dshift;  // Step (b) divisor (1 - dshift) - sum_j c_j lambda^j
    int f_slices;   // F is zero from this slice on
    int nl_f32;
    double bdt, sigR;
    int precond, accum;
    long long Mcol;
    int Ns, order;
    const double* C64;  // [order][Mcol] a_j E_m^j
    const float* C32;
    const dd* Cdd;
    int KX, NX, realcol;
    const void* gam;  // [Ns] in the storage precision ST
    const void* osc;  // [Ns] in the storage precision ST
    const float* gam32;  // [Ns] float32 copies (residuals formed in float32)
    const float* osc32;
    int norms;        // per-slice partials: 0 none, 1 (||s||^2, ||X + s||^2) for the fixed point,
                      // 2 (||out||^2, <X, out>) for the Krylov solvers
    const void* lam;  // PT2 tables
    const void* tw;
    const void* chirp;
    const void* bplus;
    const void* bminus;
    int L, log2L, bluestein;
    long long ntiles;
    double2* partial;  // [Ns][gridDim.x]
};

// Loads and stores of one time-column element in the storage precision ST.
template <typename ST, bool REAL>
__device__ __forceinline__ typename cplx<ST>::t ldcol(const void* p, long long i) {
    typedef typename cplx<ST>::t ST2;
    if (REAL) return c2(static_cast<const ST*>(p)[i], (ST)0);
    return static_cast<const ST2*>(p)[i];
}
template <typename ST, bool REAL>
__device__ __forceinline__ void stcol(void* p, long long i, typename cplx<ST>::t v) {
    typedef typename cplx<ST>::t ST2;
    if (REAL) static_cast<ST*>(p)[i] = v.x;
    else static_cast<ST2*>(p)[i] = v;
}
template <typename ST, bool REAL>
__device__ __forceinline__ typename cplx<ST>::t ldnl(const void* p, long long i, int f32) {
    typedef typename cplx<ST>::t ST2;
    if (std::is_same<ST, dd>::value) return ldcol<ST, REAL>(p, i);  // double-float N
    if (REAL) return c2(f32 ? (ST) static_cast<const float*>(p)[i] : (ST) static_cast<const double*>(p)[i], (ST)0);
    if (f32) {
        const float2 v = static_cast<const float2*>(p)[i];
        return c2((ST)v.x, (ST)v.y);
    }
    const double2 v = static_cast<const double2*>(p)[i];
    return c2((ST)v.x, (ST)v.y);
}


// a_j E_m^j: real tables, or (with advection) complex tables of the same
// layout with (Re, Im) pairs
template <typename T>
__device__ __forceinline__ T coef(const TimeArgs& A, int j, long long m);
template <>
__device__ __forceinline__ double2 coef<double2>(const TimeArgs& A, int j, long long m) {
    return reinterpret_cast<const double2*>(A.C64)[(long long)(j - 1) * A.Mcol + m];
}
template <>
__device__ __forceinline__ float2 coef<float2>(const TimeArgs& A, int j, long long m) {
    return reinterpret_cast<const float2*>(A.C32)[(long long)(j - 1) * A.Mcol + m];
}
template <>
__device__ __forceinline__ dd2 coef<dd2>(const TimeArgs& A, int j, long long m) {
    return reinterpret_cast<const dd2*>(A.Cdd)[(long long)(j - 1) * A.Mcol + m];
}
template <>
__device__ __forceinline__ double coef<double>(const TimeArgs& A, int j, long long m) {
    return A.C64[(long long)(j - 1) * A.Mcol + m];
}
template <>
__device__ __forceinline__ float coef<float>(const TimeArgs& A, int j, long long m) {
    return A.C32[(long long)(j - 1) * A.Mcol + m];
}
template <>
__device__ __forceinline__ dd coef<dd>(const TimeArgs& A, int j, long long m) {
    return A.Cdd[(long long)(j - 1) * A.Mcol + m];
}

// Asynchronous global -> shared copy of one element (4, 8 or 16 bytes); a
// source size of 0 fills the destination with zeros (columns past the end).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? BYTES : 0;
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES), "r"(n)
                     : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename ST>
__device__ __forceinline__ ST mode_weight(long long m, int KX, int NX, int realcol) {
    // real columns, or the full spectrum of a complex state (KX = NX): every
    // mode stands for itself
    if (realcol || KX == NX) return (ST)1;
    const int kx = (int)(m % KX);
    return (kx == 0 || 2 * kx == NX) ? (ST)1 : (ST)2;
}

}  // namespace expd_time

// Register-resident time kernel for power-of-two windows Ns in {16, 32, 64}
// with the float32 preconditioner; st = 1 for float32 storage, 2 for
// double-float, 0 for float64.
expd_status time_reg_launch(expd_plan p, expd_time::TimeArgs& a, int st, cudaStream_t s);

// Real-column time kernel (Dirichlet grids; time_real.cu): float32 (f32 = 1)
// or float64 preconditioner, float32 (st32 = 1) or float64 storage.
expd_status time_real_launch(expd_plan p, expd_time::TimeArgs& a, int f32, int st32, cudaStream_t s);
// Complex-column time kernel (periodic grids and complex states without a
// complex symbol; time_cplx.cu): st = 1 float32 storage, 2 double-float
// storage (both with the float32 preconditioner), 0 float64 throughout;
// and the shared memory it needs for the plan's window.
expd_status time_cplx_launch(expd_plan p, expd_time::TimeArgs& a, int st, cudaStream_t s);
size_t time_cplx_smem_bytes(expd_plan p, int st);
// Tensor-core time kernel (time_tc.cu): real columns, float32 preconditioner,
// float64 storage, Ns <= 128, no N term; the plan's tables from time_tc_setup.
expd_status time_tc_launch(expd_plan p, expd_time::TimeArgs& a, cudaStream_t s);
