// od_arith.cuh -- exact IEEE binary64 arithmetic on the integer pipes.
//
// GB300 runs FP64 at a small fraction of its FP32/INT32 rate (measured on
// GB300: DADD ~0.5 Tops/s, DDIV ~0.07 Tops/s for the whole GPU, against
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

// x << s and x >> s for a shift of at most 31: on the device two 32-bit
// funnel shifts instead of a general 64-bit shift.  The shift counts below
// are at most 11 whenever their result is used (the domain checks send every
// other case to the IEEE fallback); a larger count only yields a discarded
// value, the same on host and device.
OD_HD uint64_t shl31(uint64_t x, uint32_t s) {
    s &= 31u;
#if defined(__CUDA_ARCH__)
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    return ((uint64_t)__funnelshift_l(lo, hi, s) << 32) | (uint64_t)(lo << s);
#else
    return x << s;
#endif
}

OD_HD uint64_t shr31(uint64_t x, uint32_t s) {
    s &= 31u;
#if defined(__CUDA_ARCH__)
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    return ((uint64_t)(hi >> s) << 32) | (uint64_t)__funnelshift_r(lo, hi, s);
#else
    return x >> s;
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

// ---------------------------------------------------------------- chains
//
// A chain of additions keeps its partial sum unpacked: value = m * 2^(e-1075)
// with m in [2^52, 2^53) and biased exponent e, i.e. exactly the binary64
// number the IEEE sum would have produced, minus the packing.  Every step is
// still rounded to 53 bits, so the chain reproduces the IEEE sequence bit for
// bit.  The chain accepts only operands in its domain: positive with biased
// exponent in [4, 2040] (so no partial sum of up to six such operands can
// overflow, and s/6 of the total stays normal); callers fall back to IEEE
// operations when any operand is outside it.

struct Unpacked {
    uint64_t m;  // significand with the hidden bit, [2^52, 2^53)
    uint32_t e;  // biased exponent
};

// Unpack x; returns false when x is outside the chain's domain.
OD_HD bool unpack_chain(double x, Unpacked &u) {
    const uint64_t b = f64_bits(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    u.e = hi >> 20;  // includes the sign bit: negative x gives e >= 2048
    u.m = (b & kFrac) | kHid;
    return u.e - 4u <= 2036u;
}

OD_HD double pack_chain(const Unpacked &u) { return f64_from(((uint64_t)(u.e - 1u) << 52) + u.m); }

// a + b rounded to nearest even, both in the chain's domain.  Both
// significands are scaled by 2^10 inside a 64-bit word; the bits of the
// smaller one that fall off the word are folded into bit 0 (a sticky bit),
// which is enough for the round-to-nearest-even decision because the guard
// field's half-way pattern has bit 0 clear.  No branches.
OD_HD Unpacked add_chain(const Unpacked &a, const Unpacked &b) {
    const bool swap = b.e > a.e;
    const uint32_t e = swap ? b.e : a.e;
    const uint32_t d0 = swap ? b.e - a.e : a.e - b.e;
    const uint32_t d = d0 < 63u ? d0 : 63u;
    const uint64_t big10 = (swap ? b.m : a.m) << 10;
    const uint64_t small10 = (swap ? a.m : b.m) << 10;
    const uint64_t B = small10 >> d;
    const uint64_t sticky = (B << d) != small10 ? 1u : 0u;
    const uint64_t S = (big10 + B) | sticky;  // < 2^64
    const uint32_t c = (uint32_t)(S >> 63);   // carry into a new binade
    const uint32_t sh = 10u + c;
    const uint64_t M0 = S >> sh;
    const uint32_t rem = (uint32_t)S & ((1u << sh) - 1u);
    const uint32_t half = 1u << (sh - 1u);
    // round to nearest even (bitwise, no short-circuit branches)
    const uint32_t up = (uint32_t)(rem > half) | ((uint32_t)(rem == half) & (uint32_t)M0 & 1u);
    const uint64_t M = M0 + up;
    const uint32_t carry = (uint32_t)(M >> 53);  // rounding carried into 2^53
    Unpacked r;
    r.m = M >> carry;                             // 2^53 -> 2^52
    r.e = e + c + carry;
    return r;
}

// s / 6 for s in the chain's range (exponent >= 4): see div6.
OD_HD double div6_chain(const Unpacked &s) {
    const uint32_t big = (uint32_t)(s.m >= (3ull << 51));
    const uint64_t N = shl31(s.m, 2u - big);
    const uint64_t Q0 = mulhi64(N, 0xAAAAAAAAAAAAAAABull) >> 1;
    const uint32_t r = (uint32_t)N - 3u * (uint32_t)Q0;
    const uint64_t Q = Q0 + (r >> 1);
    const uint64_t er = (uint64_t)(s.e - 3u + big);
    return f64_from(((er - 1u) << 52) + Q);
}

// ---------------------------------------------------------------- window chain
//
// A cheaper chain when its operands are close in magnitude.  All K+1
// operands are aligned once to a common 64-bit fixed-point window: with
// emax the largest biased exponent, operand t becomes m_t << (8 - (emax -
// e_t)), so the largest operands put their hidden bit at bit 60 and -- when
// every exponent lies within 8 of emax -- no operand loses a bit.  Each add is
// then a plain 64-bit add followed by rounding the partial sum to 53
// significant bits at its own binade (position p = msb - 52, 0..11), exactly
// as the IEEE add would; nothing below the window is ever dropped, so no
// sticky bit is needed.  The value of a window word W is W * 2^(emax - 1083).

OD_HD uint32_t clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return (uint32_t)__clz((int)x);
#else
    return x ? (uint32_t)__builtin_clz(x) : 32u;
#endif
}

// Round W (whose top set bit is at 52 + p, p in [0, 11]) to 53 significant
// bits, nearest even; returns p.  With the p dropped bits r, half = 2^(p-1)
// and the kept lowest bit l, adding half - 1 + l and truncating rounds up
// exactly when r > half, or r == half and l == 1 (ties to even); for p = 0
// nothing is dropped and the added amount, masked to p bits, is 0.
OD_HD uint32_t round_window(uint64_t &W) {
    const uint32_t hi = (uint32_t)(W >> 32), lo = (uint32_t)W;
    const uint32_t p = 11u - clz32(hi);           // hi >= 2^20
    const uint32_t mask = (1u << p) - 1u;
    const uint32_t bias = ((mask >> 1) + ((lo >> p) & 1u)) & mask;  // half - 1 + l (0 when p = 0)
    W = (W + bias) & ~(uint64_t)mask;
    return p;
}

// First K adds of x[0..K] in the window; ok = false when an operand is not
// positive, has a biased exponent outside [4, 2040], or lies more than 8
// binades below the largest.  Returns the rounded window word and sets
// emax and p (the last rounding position).
template <int K>
OD_HD uint64_t window_chain(const double *x, bool &ok, uint32_t &emax, uint32_t &p) {
    uint32_t e[K + 1];
    uint64_t m[K + 1];
    uint32_t lo_e = 0xFFFFFFFFu, hi_e = 0;
#pragma unroll
    for (int t = 0; t <= K; ++t) {
        const uint64_t b = f64_bits(x[t]);
        e[t] = (uint32_t)(b >> 52);  // includes the sign bit: negative -> >= 2048
        m[t] = (b & kFrac) | kHid;
        lo_e = e[t] < lo_e ? e[t] : lo_e;
        hi_e = e[t] > hi_e ? e[t] : hi_e;
    }
    ok = (lo_e - 4u <= 2036u) & (hi_e - 4u <= 2036u) & (hi_e - lo_e <= 8u);
    emax = hi_e;
    uint64_t W = shl31(m[0], 8u - (hi_e - e[0]));
    p = 0;
#pragma unroll
    for (int t = 1; t <= K; ++t) {
        W += shl31(m[t], 8u - (hi_e - e[t]));
        p = round_window(W);
    }
    return W;
}

// The window word as a binary64 (53 significant bits at position p).
OD_HD double pack_window(uint64_t W, uint32_t emax, uint32_t p) {
    const uint64_t M = shr31(W, p);                       // [2^52, 2^53)
    const uint64_t E = (uint64_t)(emax - 8u + p);         // biased exponent
    return f64_from(((E - 1u) << 52) + M);
}

// s / 6 of the window value (see div6), s's exponent emax - 8 + p >= 4.
OD_HD double div6_window(uint64_t W, uint32_t emax, uint32_t p) {
    Unpacked u;
    u.m = shr31(W, p);
    u.e = emax - 8u + p;
    return div6_chain(u);
}

// ---------------------------------------------------------------- update

// s / 6 on the integer pipes without a branch; ok = false when s is outside
// [2^-1019, inf) in magnitude (zero, subnormal results, inf, NaN), where the
// caller must use the IEEE division instead.
OD_HD double div6_fast(double s, bool &ok) {
    const uint64_t b = f64_bits(s);
    const uint32_t es = (uint32_t)(b >> 52) & 0x7FFu;
    ok = es - 4u <= 2042u;
    const uint64_t M = (b & kFrac) | kHid;
    const uint32_t big = (uint32_t)(M >= (3ull << 51));
    const uint64_t N = shl31(M, 2u - big);
    const uint64_t Q0 = mulhi64(N, 0xAAAAAAAAAAAAAAABull) >> 1;
    const uint32_t r = (uint32_t)N - 3u * (uint32_t)Q0;  // 0, 1 or 2
    const uint64_t Q = Q0 + (r >> 1);                      // round up iff r == 2
    const uint64_t er = (uint64_t)(es - 3u + big);
    return f64_from((b & kSign) | (((er - 1u) << 52) + Q));
}

// The Jacobi update (((((W+E)+S)+N)+D)+U)/6 in binary64 round-to-nearest,
// as IEEE operations (the reference form, and the fallback of the fast one).
template <bool INT_DIV>
OD_HD double jacobi_update_ieee(double W, double E, double S, double N, double D, double U) {
    double s = ieee_add(W, E);
    s = ieee_add(s, S);
    s = ieee_add(s, N);
    s = ieee_add(s, D);
    s = ieee_add(s, U);
    if (INT_DIV) return div6(s);
    return ieee_div(s, 6.0);
}

// The same update with its operations placed by AM, never changing a bit:
//   AM = 0  every add and the division as IEEE operations (FP64 pipe)
//   AM = 1  IEEE adds, division by 6 on the integer pipes
//   AM = 1+k, k = 1..5: the first k adds in the integer window chain, the
//           remaining 5-k as IEEE adds, the division on the integer pipes.
// Branch-free: ok = false when an operand or the sum left the integer
// routines' domain (for the window: operands more than 8 binades apart,
// zero, negative, tiny or huge); the result is then garbage and the caller
// recomputes the cell with jacobi_update_ieee (a rare path kept out of the
// hot loop).
template <int AM>
OD_HD double jacobi_update_fast(double W, double E, double S, double N, double D, double U, bool &ok) {
    constexpr int K = AM > 1 ? AM - 1 : 0;
    if constexpr (AM == 0) {
        ok = true;
        return jacobi_update_ieee<false>(W, E, S, N, D, U);
    } else if constexpr (K == 0) {
        double s = ieee_add(W, E);
        s = ieee_add(s, S);
        s = ieee_add(s, N);
        s = ieee_add(s, D);
        s = ieee_add(s, U);
        return div6_fast(s, ok);
    } else {
        const double x[6] = {W, E, S, N, D, U};
        bool good;
        uint32_t emax, p;
        const uint64_t Wd = window_chain<K>(x, good, emax, p);
        if constexpr (K == 5) {
            ok = good;
            return div6_window(Wd, emax, p);
        } else {
            double s = pack_window(Wd, emax, p);
#pragma unroll
            for (int t = K + 1; t <= 5; ++t) s = ieee_add(s, x[t]);
            bool okd;
            const double v = div6_fast(s, okd);
            ok = good & okd;
            return v;
        }
    }
}

// Complete update in mode AM for every input (fast form, IEEE fallback).
template <int AM>
OD_HD double jacobi_update(double W, double E, double S, double N, double D, double U) {
    bool ok;
    const double v = jacobi_update_fast<AM>(W, E, S, N, D, U, ok);
    return ok ? v : jacobi_update_ieee<false>(W, E, S, N, D, U);
}

// The update with its LAST KT adds (KT = 1 or 2) in the window chain and the
// division by 6 taken straight from the window word: the first 5-KT adds are
// IEEE operations (FP64 pipe), their sum s joins the remaining operands in the
// window, and the rounded window value is divided without being packed into
// a double and unpacked again.  ok = false when the window's domain is left.
template <int KT>
OD_HD double jacobi_update_tail(double W, double E, double S, double N, double D, double U, bool &ok) {
    static_assert(KT == 1 || KT == 2, "one or two adds in the tail");
    double s = ieee_add(W, E);
    s = ieee_add(s, S);
    s = ieee_add(s, N);
    bool good;
    uint32_t emax, p;
    uint64_t Wd;
    if constexpr (KT == 1) {
        const double x[2] = {ieee_add(s, D), U};
        Wd = window_chain<1>(x, good, emax, p);
    } else {
        const double x[3] = {s, D, U};
        Wd = window_chain<2>(x, good, emax, p);
    }
    ok = good;
    return div6_window(Wd, emax, p);
}

template <int KT>
OD_HD double jacobi_update_tail_checked(double W, double E, double S, double N, double D, double U) {
    bool ok;
    const double v = jacobi_update_tail<KT>(W, E, S, N, D, U, ok);
    return ok ? v : jacobi_update_ieee<false>(W, E, S, N, D, U);
}

// ---------------------------------------------------------------- 2D update
//
// The paper's own application: the 5-point update (((W+E)+S)+N)/4.  Division
// by 4 is an exact power-of-two scaling: for a normal result it only lowers
// the exponent by two, which the integer pipes do in one subtraction.

// s / 4 by the exponent; ok = false when s is zero, subnormal, infinite, NaN
// or so small that s/4 would be subnormal (biased exponent < 3).
OD_HD double div4_fast(double s, bool &ok) {
    const uint64_t b = f64_bits(s);
    const uint32_t es = (uint32_t)(b >> 52) & 0x7FFu;
    ok = es - 3u <= 2043u;
    return f64_from(b - (2ull << 52));
}

template <bool INT_DIV>
OD_HD double jacobi2d_update_ieee(double W, double E, double S, double N) {
    double s = ieee_add(W, E);
    s = ieee_add(s, S);
    s = ieee_add(s, N);
    if (INT_DIV) {
        bool ok;
        const double v = div4_fast(s, ok);
        if (ok) return v;
    }
    return ieee_div(s, 4.0);
}

// Same placement modes as jacobi_update_fast (the chain takes at most the
// three adds there are); ok = false sends the cell to jacobi2d_update_ieee.
template <int AM>
OD_HD double jacobi2d_update_fast(double W, double E, double S, double N, bool &ok) {
    constexpr int K0 = AM > 1 ? AM - 1 : 0;
    constexpr int K = K0 > 3 ? 3 : K0;
    if constexpr (AM == 0) {
        ok = true;
        return jacobi2d_update_ieee<false>(W, E, S, N);
    } else if constexpr (K == 0) {
        double s = ieee_add(W, E);
        s = ieee_add(s, S);
        s = ieee_add(s, N);
        return div4_fast(s, ok);
    } else {
        const double x[4] = {W, E, S, N};
        bool good;
        uint32_t emax, p;
        const uint64_t Wd = window_chain<K>(x, good, emax, p);
        double s = pack_window(Wd, emax, p);
#pragma unroll
        for (int t = K + 1; t <= 3; ++t) s = ieee_add(s, x[t]);
        bool okd;
        const double v = div4_fast(s, okd);
        ok = good & okd;
        return v;
    }
}

template <int AM>
OD_HD double jacobi2d_update(double W, double E, double S, double N) {
    bool ok;
    const double v = jacobi2d_update_fast<AM>(W, E, S, N, ok);
    return ok ? v : jacobi2d_update_ieee<false>(W, E, S, N);
}

// The 2D update with its last KT adds (1 or 2) in the window; the division
// by 4 lowers the window value's exponent by two as it is packed (the window
// domain keeps the quotient normal).
template <int KT>
OD_HD double jacobi2d_update_tail(double W, double E, double S, double N, bool &ok) {
    static_assert(KT == 1 || KT == 2, "one or two adds in the tail");
    const double s = ieee_add(W, E);
    bool good;
    uint32_t emax, p;
    uint64_t Wd;
    if constexpr (KT == 1) {
        const double x[2] = {ieee_add(s, S), N};
        Wd = window_chain<1>(x, good, emax, p);
    } else {
        const double x[3] = {s, S, N};
        Wd = window_chain<2>(x, good, emax, p);
    }
    ok = good;
    return pack_window(Wd, emax - 2u, p);
}

template <int KT>
OD_HD double jacobi2d_update_tail_checked(double W, double E, double S, double N) {
    bool ok;
    const double v = jacobi2d_update_tail<KT>(W, E, S, N, ok);
    return ok ? v : jacobi2d_update_ieee<false>(W, E, S, N);
}

// Run-time dispatch of the 2D update (tests): 0..4 head modes, 5 / 6 the
// tail form with one / two window adds.
OD_HD double jacobi2d_update_mode(int am, const double *x) {
    switch (am) {
        case 0: return jacobi2d_update<0>(x[0], x[1], x[2], x[3]);
        case 1: return jacobi2d_update<1>(x[0], x[1], x[2], x[3]);
        case 2: return jacobi2d_update<2>(x[0], x[1], x[2], x[3]);
        case 3: return jacobi2d_update<3>(x[0], x[1], x[2], x[3]);
        case 5: return jacobi2d_update_tail_checked<1>(x[0], x[1], x[2], x[3]);
        case 6: return jacobi2d_update_tail_checked<2>(x[0], x[1], x[2], x[3]);
        default: return jacobi2d_update<4>(x[0], x[1], x[2], x[3]);
    }
}

// Run-time dispatch of jacobi_update (tests): 0..6 head modes, 7 / 8 the
// tail form with one / two window adds.
OD_HD double jacobi_update_mode(int am, const double *x) {
    switch (am) {
        case 7: return jacobi_update_tail_checked<1>(x[0], x[1], x[2], x[3], x[4], x[5]);
        case 8: return jacobi_update_tail_checked<2>(x[0], x[1], x[2], x[3], x[4], x[5]);
        case 0: return jacobi_update<0>(x[0], x[1], x[2], x[3], x[4], x[5]);
        case 1: return jacobi_update<1>(x[0], x[1], x[2], x[3], x[4], x[5]);
        case 2: return jacobi_update<2>(x[0], x[1], x[2], x[3], x[4], x[5]);
        case 3: return jacobi_update<3>(x[0], x[1], x[2], x[3], x[4], x[5]);
        case 4: return jacobi_update<4>(x[0], x[1], x[2], x[3], x[4], x[5]);
        case 5: return jacobi_update<5>(x[0], x[1], x[2], x[3], x[4], x[5]);
        default: return jacobi_update<6>(x[0], x[1], x[2], x[3], x[4], x[5]);
    }
}

}  // namespace od
