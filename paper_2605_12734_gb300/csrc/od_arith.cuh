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

// ---------------------------------------------------------------- anchored window
//
// The window chain above aligns each cell's operands to the largest of them,
// which costs a maximum over their exponents and a relative shift per
// operand.  When the whole field lies within a few binades -- a Jacobi field
// never leaves the range of its initial values and boundary (the maximum
// principle) -- one window can be anchored for every cell instead.  With a
// base exponent E0, an operand with biased exponent e in [E0, E0+7] is
// exactly the integer F = m << (e - E0) in units of 2^(E0-1075) (m its 53-bit
// significand), so F < 2^60 and a sum of up to six such integers is exact in
// 64 bits.  Each add of the chain is a 64-bit integer add followed by
// rounding the partial sum to 53 significant bits at its own binade, exactly
// as the IEEE add would round it; the division by 6 reads the rounded word.
// An operand outside [E0, E0+7] (zero, subnormal, negative, infinite, NaN, or
// just outside the window) sends the cell to the IEEE form (ok = false).
// E0 only decides how many cells take the fast form: any E0 in [4, 2037]
// gives the IEEE result for every input (the quotient's exponent stays
// normal and below the infinities, and an infinite or NaN operand still
// reads as outside the window).  The anchors chosen below lie in
// [kAnchorMin, kAnchorMax], which leaves room for E0 + 1.

constexpr uint32_t kAnchorMin = 4u, kAnchorMax = 2030u;

// Integer and FP32 helpers with one meaning on host and device.  On the
// device the multiply-adds are written as PTX mad instructions: with `one`
// a register whose value (1) the compiler cannot see, an add becomes an
// IMAD on the FMA pipe instead of an IADD on the integer ALU pipe, which the
// exact arithmetic below would otherwise saturate.  On the host they are the
// plain integer operations.
OD_HD uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
#else
    return a * b + c;
#endif
}

OD_HD uint64_t mad_wide_u(uint32_t a, uint32_t b, uint64_t c) {
#if defined(__CUDA_ARCH__)
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
#else
    return (uint64_t)a * b + c;
#endif
}

// a * b + c with a and b signed 32-bit (the product sign-extended)
OD_HD uint64_t mad_wide_s(int32_t a, int32_t b, uint64_t c) {
#if defined(__CUDA_ARCH__)
    uint64_t d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
#else
    return (uint64_t)((int64_t)a * (int64_t)b) + c;
#endif
}

// 1 << s, 0 for s >= 32 (PTX shl clamps its count; the host matches it)
OD_HD uint32_t pow2_u32(uint32_t s) {
#if defined(__CUDA_ARCH__)
    uint32_t d;
    asm("shl.b32 %0, 1, %1;" : "=r"(d) : "r"(s));
    return d;
#else
    return s < 32u ? 1u << s : 0u;
#endif
}

OD_HD float f32_from(uint32_t u) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float x;
    memcpy(&x, &u, 4);
    return x;
#endif
}

OD_HD uint32_t f32_bits(float x) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t u;
    memcpy(&u, &x, 4);
    return u;
#endif
}

// (a + b) - b in binary32 round-to-nearest-even, both operations rounded
// (never contracted or reassociated)
OD_HD float f32_add_sub(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fsub_rn(__fadd_rn(a, b), b);
#else
    volatile float s = a + b;
    volatile float r = s - b;
    return r;
#endif
}

// F += F(x): x's window word m * 2^sh (m its 53-bit significand, sh =
// e - E0) added into F as two multiply-adds by 2^sh, low word then high
// word.  nE0s = -(E0 << 20).  hb = hi - (E0 << 20) carries (e - E0) in its
// bits 20..30 and the top fraction bits below; x lies in the window exactly
// when hb < 2^23 (a negative x carries its sign bit into hb, a zero or
// subnormal x makes it wrap), so the caller ORs every hb into chk and tests
// chk < 2^23 once.  Out of the window F is meaningless (the caller discards
// the cell's fast result), and so it is on the host, which computes the
// same words.
OD_HD void anchor_acc(uint64_t &F, uint32_t &chk, double x, uint32_t nE0s, uint32_t one) {
    const uint64_t b = f64_bits(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t hb = mad_lo(hi, one, nE0s);
    chk |= hb;
    const uint32_t p2 = pow2_u32(hb >> 20);
    const uint32_t mh = (hb & 0x000FFFFFu) | 0x00100000u;  // high significand word with the hidden bit
    const uint64_t t = mad_wide_u(lo, p2, F);
    F = ((uint64_t)mad_lo(mh, p2, (uint32_t)(t >> 32)) << 32) | (uint32_t)t;
}

OD_HD bool anchored_ok(uint32_t chk) { return chk < 0x00800000u; }

// Round F, a sum of at least two window words (so its top set bit lies at
// 52 + d with d = 11 - c in [1, 10], c = clz(hi)), to 53 significant bits,
// nearest even; returns c.  Only F's low 23 bits x take part (d < 23): the
// binary32 sum (2^23 + x) + 2^(23+d) lies in [2^(23+d), 2^(24+d)], where
// binary32 numbers are 2^d apart, so the addition rounds 2^23 + x to a
// multiple of 2^d, nearest even, exactly as the rounding to 53 bits needs
// (the kept part's last bit is x's bit d), and subtracting 2^(23+d) again
// is exact.  F then moves by the difference of the two binary32 words.
OD_HD uint32_t round_acc(uint64_t &F, uint32_t one) {
    const uint32_t c = clz32((uint32_t)(F >> 32));
    const uint32_t mb = mad_lo(c, 0xFF800000u, 161u << 23);         // binary32 2^(23+d): exponent 150 + d
    const uint32_t fb = ((uint32_t)F & 0x007FFFFFu) | 0x4B000000u;  // binary32 2^23 + x
    const uint32_t hb = f32_bits(f32_add_sub(f32_from(fb), f32_from(mb)));
    F = mad_wide_s((int32_t)(hb - fb), (int32_t)one, F);
    return c;
}

// (x+1)/3 rounded down for x < 2^62: the high half of x * ceil(2^64/3)
// equals floor(x/3) for every x < 2^63 (its error, 2x/(3*2^64), stays below
// the distance 1/3 from x/3 to the next integer), and adding the constant
// once more turns x into x+1.
OD_HD uint64_t div3_up1(uint64_t x) {
    const uint64_t C = 0x5555555555555556ull;
    return mulhi64(x + 1u, C);
}

// s/6 correctly rounded, for the window word F of s as its last rounding
// left it: c = clz(hi) before that rounding, d = 11 - c >= 2, and F a
// multiple of 2^d in [2^(52+d), 2^(53+d)] -- the top end when the rounding
// carried into the next binade.  As in div6: the quotient's significand is
// N/3 for N = 2M or 4M (M = F >> d, N = 2M when M >= 3*2^51), N/3 is never a
// tie, and rounding it to nearest is floor((N+1)/3).  N = F >> (d - 2 + big)
// is exact because F's d low bits are zero.  The two bits of F below and at
// its expected top position, h = hi >> (30 - c), are 2 or 3 (big when 3);
// a carried F = 2^(53+d) reads h = 4 and is big too, which is right: its
// significand is 2^52 one binade up, whose N = 4 * 2^52 = F >> (d - 1).
// The result's biased exponent is E0 + d - 3 + big.
OD_HD double div6_anchored(uint64_t F, uint32_t c, uint32_t E0) {
    const uint32_t hi = (uint32_t)(F >> 32);
    const uint32_t big = (hi >> (30u - c)) >= 3u ? 1u : 0u;  // M >= 3*2^51, or a carried F
    const uint32_t sh = 9u - c + big;             // d - 2 + big
    const uint64_t Q = div3_up1(shr31(F, sh));    // [2^52, 2^53]; 2^53 carries into the exponent
    const uint32_t em1 = E0 + 7u - c + big;       // biased exponent - 1
    return f64_from(((uint64_t)mad_lo(em1, 1u << 20, (uint32_t)(Q >> 32)) << 32) | (uint32_t)Q);
}

// s/4 exactly (2D): the significand M = F >> d keeps its bits and the
// exponent drops by two: biased exponent E0 + d - 2.  A last rounding that
// carried into the next binade leaves M = 2^53, and the packing's addition
// carries it into the exponent field.
OD_HD double div4_anchored(uint64_t F, uint32_t c, uint32_t E0) {
    const uint64_t M = shr31(F, 11u - c);
    return f64_from(((uint64_t)mad_lo(E0 + 8u - c, 1u << 20, (uint32_t)(M >> 32)) << 32) | (uint32_t)M);
}

// The 3D update with its first NF adds (0..3) on the FP64 pipe and the rest
// in the anchored window, the division from the window word.  ok = false
// when the FP64 partial sum or a later operand leaves the window (or, with
// NF = 3, when the window sum is below 2^54 so that d = 1).  `one` must be 1
// (see mad_lo).
template <int NF>
OD_HD double jacobi_update_anchored(double W, double E, double S, double N, double D, double U, uint32_t E0,
                                    bool &ok, uint32_t one = 1u) {
    static_assert(NF >= 0 && NF <= 3, "zero to three adds on the FP64 pipe");
    const double x[6] = {W, E, S, N, D, U};
    double s = x[0];
#pragma unroll
    for (int t = 1; t <= NF; ++t) s = ieee_add(s, x[t]);
    const uint32_t nE0s = 0u - (E0 << 20);
    uint64_t F = 0;
    uint32_t chk = 0, c = 0;
    anchor_acc(F, chk, s, nE0s, one);
#pragma unroll
    for (int t = NF + 1; t <= 5; ++t) {
        anchor_acc(F, chk, x[t], nE0s, one);
        c = round_acc(F, one);
    }
    ok = anchored_ok(chk);
    if constexpr (NF == 3) ok = ok & (c <= 9u);
    return div6_anchored(F, c, E0);
}

// The 2D update (((W+E)+S)+N)/4 with its first NF adds (0..2) on the FP64
// pipe and the rest in the anchored window.
template <int NF>
OD_HD double jacobi2d_update_anchored(double W, double E, double S, double N, uint32_t E0, bool &ok,
                                      uint32_t one = 1u) {
    static_assert(NF >= 0 && NF <= 2, "zero to two adds on the FP64 pipe");
    const double x[4] = {W, E, S, N};
    double s = x[0];
#pragma unroll
    for (int t = 1; t <= NF; ++t) s = ieee_add(s, x[t]);
    const uint32_t nE0s = 0u - (E0 << 20);
    uint64_t F = 0;
    uint32_t chk = 0, c = 0;
    anchor_acc(F, chk, s, nE0s, one);
#pragma unroll
    for (int t = NF + 1; t <= 3; ++t) {
        anchor_acc(F, chk, x[t], nE0s, one);
        c = round_acc(F, one);
    }
    ok = anchored_ok(chk);
    return div4_anchored(F, c, E0);
}

// The anchor for a field whose largest value has bit pattern vmax (a
// positive double, or 0 when unknown).  The window [E0, E0+7] must hold the
// operands and the FP64 partial sum that joins them: up to twice the largest
// value with NF <= 1 (E0 = emax - 6: values down to 2^-6 of the largest stay
// in), up to three or four times it with NF = 2 or 3 (E0 = emax - 5).  A sum
// of three values near the top would otherwise leave the window whenever
// the field is locally above two thirds of its largest value.
OD_HD uint32_t anchor_for(uint64_t vmax, int nf) {
    const int64_t emax = (int64_t)(vmax >> 52) & 0x7FF;
    int64_t e0 = emax - (nf >= 2 ? 5 : 6);
    if (e0 < (int64_t)kAnchorMin) e0 = kAnchorMin;
    if (e0 > (int64_t)kAnchorMax) e0 = kAnchorMax;
    return (uint32_t)e0;
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

// The anchored forms with their IEEE fallback, and their run-time dispatch
// over the number of adds on the FP64 pipe (tests).
template <int NF>
OD_HD double jacobi_update_anchored_checked(const double *x, uint32_t E0) {
    bool ok;
    const double v = jacobi_update_anchored<NF>(x[0], x[1], x[2], x[3], x[4], x[5], E0, ok);
    return ok ? v : jacobi_update_ieee<false>(x[0], x[1], x[2], x[3], x[4], x[5]);
}

template <int NF>
OD_HD double jacobi2d_update_anchored_checked(const double *x, uint32_t E0) {
    bool ok;
    const double v = jacobi2d_update_anchored<NF>(x[0], x[1], x[2], x[3], E0, ok);
    return ok ? v : jacobi2d_update_ieee<false>(x[0], x[1], x[2], x[3]);
}

// The fast form alone, NaN where the cell would leave it (tests: how many
// cells take the fast form, and that every one of them is exact).
template <int NF>
OD_HD double jacobi_update_anchored_fast(const double *x, uint32_t E0) {
    bool ok;
    const double v = jacobi_update_anchored<NF>(x[0], x[1], x[2], x[3], x[4], x[5], E0, ok);
    return ok ? v : f64_from(0x7FF8000000000000ull);
}

template <int NF>
OD_HD double jacobi2d_update_anchored_fast(const double *x, uint32_t E0) {
    bool ok;
    const double v = jacobi2d_update_anchored<NF>(x[0], x[1], x[2], x[3], E0, ok);
    return ok ? v : f64_from(0x7FF8000000000000ull);
}

// nf 0..3 (3D) / 0..2 (2D): the checked form; nf + 4: the fast form alone.
OD_HD double jacobi_update_anchored_mode(int nf, const double *x, uint32_t E0) {
    switch (nf) {
        case 0: return jacobi_update_anchored_checked<0>(x, E0);
        case 1: return jacobi_update_anchored_checked<1>(x, E0);
        case 2: return jacobi_update_anchored_checked<2>(x, E0);
        case 3: return jacobi_update_anchored_checked<3>(x, E0);
        case 4: return jacobi_update_anchored_fast<0>(x, E0);
        case 5: return jacobi_update_anchored_fast<1>(x, E0);
        case 6: return jacobi_update_anchored_fast<2>(x, E0);
        default: return jacobi_update_anchored_fast<3>(x, E0);
    }
}

OD_HD double jacobi2d_update_anchored_mode(int nf, const double *x, uint32_t E0) {
    switch (nf) {
        case 0: return jacobi2d_update_anchored_checked<0>(x, E0);
        case 1: return jacobi2d_update_anchored_checked<1>(x, E0);
        case 2: return jacobi2d_update_anchored_checked<2>(x, E0);
        case 4: return jacobi2d_update_anchored_fast<0>(x, E0);
        case 5: return jacobi2d_update_anchored_fast<1>(x, E0);
        default: return jacobi2d_update_anchored_fast<2>(x, E0);
    }
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
