// od_arith.cuh -- exact IEEE binary64 arithmetic on the integer pipes.
//
// GB300 runs FP64 at a small fraction of its FP32/INT32 rate (measured on
// the pool: DADD ~0.5 Tops/s, DDIV ~0.07 Tops/s for the whole GPU, against
// ~19 Tops/s IMAD and ~36 Tops/s FADD), so the Jacobi update
// (((((W+E)+S)+N)+D)+U)/6 is bound by the FP64 pipe, not by HBM.  These
// routines compute the SAME correctly rounded binary64 results with integer
// instructions, so a kernel can move work off the FP64 pipe without changing
// a single bit.  Both are written from the definition of IEEE 754 binary64
// round-to-nearest-even; inputs outside the fast domain (zero, subnormal,
// negative, infinite, NaN, or results that could leave the normal range) go
// to the ordinary IEEE operation, so every input gives the IEEE result.
//
// od_div6(s): s / 6.  With s = M * 2^(e-1075), M in [2^52, 2^53), the
//   quotient's significand is N/3 for N = 2M (M >= 3*2^51) or N = 4M
//   (otherwise), which lies in [2^52, 2^53).  N/3 = floor(N/3) + r/3 with
//   r = N mod 3, so the exact quotient is never a rounding tie: r = 2 rounds
//   up, r = 0 or 1 rounds down.  floor(N/3) is the high half of
//   N * ceil(2^65/3) shifted right once (the classical multiply-by-reciprocal
//   division by a constant, Granlund & Montgomery, PLDI 1994), exact for
//   every 64-bit N.
//
// od_add(a, b): a + b for positive normal a, b.  Align the smaller
//   significand to the larger with two guard bits and a sticky bit, add,
//   renormalise a carry, round to nearest even; a rounding carry into 2^53
//   propagates into the exponent field by the final addition.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define OD_HD __host__ __device__ __forceinline__
#else
#define OD_HD inline
#endif

namespace od {

constexpr uint64_t kFrac = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kHid = 0x0010000000000000ull;
constexpr uint64_t kSign = 0x8000000000000000ull;

OD_HD uint64_t f64_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
#endif
}

OD_HD double f64_from(uint64_t u) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double x;
    memcpy(&x, &u, 8);
    return x;
#endif
}

OD_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// IEEE operations (the fallback and the reference)
OD_HD double ieee_add(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dadd_rn(a, b);
#else
    volatile double r = a + b;
    return r;
#endif
}

OD_HD double ieee_div(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __ddiv_rn(a, b);
#else
    volatile double r = a / b;
    return r;
#endif
}

// s / 6.0, correctly rounded (see header).
OD_HD double div6(double s) {
    const uint64_t b = f64_bits(s);
    const uint32_t es = (uint32_t)(b >> 52) & 0x7FFu;
    if (es < 4u || es == 0x7FFu) return ieee_div(s, 6.0);
    const uint64_t M = (b & kFrac) | kHid;
    const bool big = M >= (3ull << 51);
    const uint64_t N = big ? (M << 1) : (M << 2);
    const uint64_t Q0 = mulhi64(N, 0xAAAAAAAAAAAAAAABull) >> 1;  // floor(N/3)
    const uint32_t r = (uint32_t)N - 3u * (uint32_t)Q0;          // N mod 3
    const uint64_t Q = Q0 + (r == 2u ? 1u : 0u);
    const uint64_t er = (uint64_t)(es - (big ? 2u : 3u));        // >= 1: normal
    return f64_from((b & kSign) | (((er - 1u) << 52) + Q));
}

// a + b, correctly rounded (see header).
OD_HD double add(double a, double b) {
    uint64_t A = f64_bits(a), B = f64_bits(b);
    // fast domain: both positive normal with biased exponent <= 2045
    const uint64_t lo = kHid, span = 0x7FD0000000000000ull - kHid;
    if (!((A - lo) < span && (B - lo) < span)) return ieee_add(a, b);
    if (A < B) {
        const uint64_t t = A;
        A = B;
        B = t;
    }
    const uint32_t ea = (uint32_t)(A >> 52), eb = (uint32_t)(B >> 52);
    const uint32_t d = ea - eb;
    const uint64_t ma = ((A & kFrac) | kHid) << 2;  // [2^54, 2^55)
    const uint64_t mb = ((B & kFrac) | kHid) << 2;
    uint64_t mbs, sticky;
    if (d < 64u) {
        mbs = mb >> d;
        sticky = (mbs << d) != mb ? 1u : 0u;
    } else {
        mbs = 0;
        sticky = 1;
    }
    uint64_t S = ma + mbs;  // [2^54, 2^56)
    uint32_t e = ea;
    if (S >> 55) {
        sticky |= S & 1u;
        S >>= 1;
        e += 1;
    }
    const uint64_t lsb = (S >> 2) & 1u, g = (S >> 1) & 1u, rs = (S & 1u) | sticky;
    const uint64_t Mt = (S >> 2) + (g & (rs | lsb));  // [2^52, 2^53]
    return f64_from(((uint64_t)(e - 1u) << 52) + Mt);
}

}  // namespace od
