// Digits and operand layout of the tensor-core DST (dst_tc.cu), shared by the
// device kernels and the host self-test.
//
// A row of float64 values with max|x| < 2^e is written as
//   x = 2^e sum_{i=0}^{nsl-1} d_i 2^{-7(i+1)}   (up to a rounding at the last digit)
// with balanced 7-bit digits: d_0 in [-128, 128], d_i in [-64, 64] for i > 0.
// The digits are integers of at most 8 significant bits, exact in bf16, and
// the sum of 1024 products of two of them stays within 2^24 (exact in float32).
#pragma once

#include <stdint.h>

#include "common.cuh"

// Row exponent e from the largest |x| as its binary64 encoding (sign cleared):
// max|x| < 2^e.  Non-finite maxima are flagged by the caller (exponent 2047).
EXPD_HD int digit_row_exponent(unsigned long long maxbits) {
    const int E = (int)(maxbits >> 52);
    return E == 0 ? -1022 : E - 1022;
}

// |x| 2^{7 nsl - e}, rounded half up to an integer (at most 2^{7 nsl}), from
// the binary64 encoding of x; *neg receives the sign.
EXPD_HD unsigned long long digit_magnitude(unsigned long long b, int e, int nsl, unsigned* neg) {
    const int E = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
    const int sh = (E ? E - 1075 : -1074) - e + 7 * nsl;
    *neg = (unsigned)(b >> 63);
    if (sh >= 0) return m << sh;
    const int s = -sh;
    return s >= 64 ? 0ull : (((m >> (s - 1)) + 1ull) >> 1);
}

// Next digit from the least significant end: i > 0 takes a balanced digit in
// [-64, 63] and carries; i == 0 takes what is left (0..128).
EXPD_HD int digit_next(unsigned long long* Y, int i) {
    if (i == 0) return (int)*Y;
    int d = (int)(*Y & 127ull);
    *Y >>= 7;
    if (d >= 64) {
        d -= 128;
        *Y += 1ull;
    }
    return d;
}

// The offset that turns the balanced lower digits into standard base-128
// digits: adding 64 at every lower digit position makes digit i (i > 0) of
// Y + offset equal d_i + 64 in [0, 127] with no carries, and leaves the top
// digit d_0 as the quotient by 128^(nsl-1).
EXPD_HD unsigned long long digit_offset(int nsl) {
    unsigned long long off = 0;
    for (int p = 0; p < nsl - 1; ++p) off |= 64ull << (7 * p);
    return off;
}

// Digit i of Yo = Y + digit_offset(nsl): the same value repeated digit_next
// calls give for digit i, without their carry chain.
EXPD_HD int digit_at(unsigned long long Yo, int i, int nsl) {
    const int sh = 7 * (nsl - 1 - i);
    return i == 0 ? (int)(Yo >> sh) : (int)((Yo >> sh) & 127ull) - 64;
}

// Element offset of (row r, column k) of a packed operand with KB tiles of
// 64 K per 128-row tile: tile (r / 128, k / 64) of 8192 elements, inside it
// the 8x8 core matrix of row group (r % 128) / 8 and K group (k % 64) / 8 at
// element (8 g + c) * 64, row r % 8 at 8 (r % 8), column k % 8.
EXPD_HD long long packed_offset(long long r, int k, int KB) {
    return ((r >> 7) * KB + (k >> 6)) * 8192 + ((((r & 127) >> 3) * 8 + ((k & 63) >> 3)) * 64) + (r & 7) * 8 + (k & 7);
}

// Rows of a packed operand rounded up to whole 128-row tiles: the extent of
// one digit slice (a last, partly filled tile still takes its full 16 KB per
// 64-K step, so slices of fewer rows would overlap the next digit's tiles)
EXPD_HD long long digit_rows(long long n) { return (n + 127) / 128 * 128; }

// Shared-memory matrix descriptor of a K-major operand without swizzle
// (tcgen05): start address >> 4 (bits 0-13), leading-dimension byte offset
// >> 4 = the next core matrix along K, 128 B (bits 16-29), stride-dimension
// byte offset >> 4 = the next 8-row group, 1024 B (bits 32-45), descriptor
// version 1 (bit 46), base offset 0, swizzle mode 0 (bits 61-63).
EXPD_HD uint64_t smem_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46);
}

// The digit pairs (i, j), i + j < nsl, most significant first, cut into groups
// of one weight whose products sum exactly in float32: |d_0| <= 128 and
// |d_i| <= 64 otherwise, so a pair's K products sum to at most K |d_i| |d_j|,
// and a group holds pairs while those bounds add up to at most 2^24.  Within a
// weight the pairs with a leading digit come first.
inline void tc_groups(int nsl, int K, int* np, int* ng, unsigned char* pi, unsigned char* pj, unsigned char* gstart,
               unsigned char* gw) {
    auto bound = [&](int i, int j) { return (long long)K * (i ? 64 : 128) * (j ? 64 : 128); };
    int n = 0, q = 0;
    for (int g = 0; g < nsl; ++g) {
        int order[16], m = 0;
        order[m++] = 0;
        if (g > 0) order[m++] = g;
        for (int i = 1; i < g; ++i) order[m++] = i;
        long long sum = 0;
        for (int k = 0; k < m; ++k) {
            const int i = order[k], j = g - i;
            const long long b = bound(i, j);
            if (k == 0 || sum + b > (1LL << 24)) {
                gstart[q] = (unsigned char)n;
                gw[q] = (unsigned char)g;
                ++q;
                sum = 0;
            }
            sum += b;
            pi[n] = (unsigned char)i;
            pj[n] = (unsigned char)j;
            ++n;
        }
    }
    gstart[q] = (unsigned char)n;
    *np = n;
    *ng = q;
}
