// fixed96.cuh -- exact sums of FP64 values in 96-bit two's-complement fixed point.
//
// The FP64 step's moment sums (sum f, sum f c, sum f |c|^2 over the 37 populations) are formed
// here on the integer pipe instead of with FP64 additions: on GB300 the FP64 pipe issues two
// instructions per clock per SM and binds the step, while 32-bit integer adds, shifts and logic run
// at a far higher rate. Each population f = m 2^(e - 1075) (m the 53-bit significand, e the biased
// exponent) is converted to the integer N = f / q with quantum q = 2^-80:
//   N = m << (e - 995)   for 2^-28 <= |f| < 16 (shift 0..31: exact, since every such f is a
//                        multiple of 2^-80);
//   N = m >> (995 - e)   for |f| < 2^-28 (truncated toward zero: error below q ~ 8e-25).
// Sums of such N are exact in 96 bits (|sum |c|^2 N| < 18 x 37 x 16 x 2^80 < 2^95). A sum is
// rounded to FP64 at the end (to_double48, correctly rounded), so the moments are at least as
// accurate as any FP64 summation order. Populations of magnitude >= 16, infinities and NaN are
// reported through the maximum exponent that to96 collects.
#pragma once

#include <cstdint>

namespace lbg {
namespace fx {

struct I96 {
    unsigned w0, w1, w2;  // value = w0 + 2^32 w1 + 2^64 (int)w2, in units of 2^-80
};

__device__ __forceinline__ I96 zero96() { return I96{0u, 0u, 0u}; }

__device__ __forceinline__ void add96(I96& a, const I96& b) {
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2)
        : "r"(b.w0), "r"(b.w1), "r"(b.w2));
}

__device__ __forceinline__ I96 plus96(I96 a, const I96& b) {
    add96(a, b);
    return a;
}

__device__ __forceinline__ I96 minus96(I96 a, const I96& b) {
    asm("sub.cc.u32 %0, %0, %3;\n\tsubc.cc.u32 %1, %1, %4;\n\tsubc.u32 %2, %2, %5;"
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2)
        : "r"(b.w0), "r"(b.w1), "r"(b.w2));
    return a;
}

// a * 2^K, K in 1..31 (no overflow for the magnitudes above)
template <int K>
__device__ __forceinline__ I96 shl96(const I96& a) {
    return I96{a.w0 << K, __funnelshift_l(a.w0, a.w1, K), __funnelshift_l(a.w1, a.w2, K)};
}

__device__ __forceinline__ I96 times2(const I96& a) { return shl96<1>(a); }
__device__ __forceinline__ I96 times3(const I96& a) { return plus96(shl96<1>(a), a); }
__device__ __forceinline__ I96 times4(const I96& a) { return shl96<2>(a); }
__device__ __forceinline__ I96 times9(const I96& a) { return plus96(shl96<3>(a), a); }

// N = f / 2^-80 as above; emax collects the largest biased exponent seen.
__device__ __forceinline__ I96 to96(double f, unsigned& emax) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(f);
    const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    const unsigned e = (hi >> 20) & 0x7FFu;
    emax = max(emax, e);
    const int s = (int)e - 995;
    unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | (e ? 0x100000u : 0u)) << 32) | lo;
    const unsigned rs = (unsigned)min(max(-s, 0), 63);  // right shift of tiny values
    m >>= rs;
    const unsigned k = (unsigned)min(max(s, 0), 31);    // left shift (>= 16 is clamped and flagged)
    const unsigned ml = (unsigned)m, mh = (unsigned)(m >> 32);
    I96 n{ml << k, __funnelshift_l(ml, mh, k), __funnelshift_l(mh, 0u, k)};
    // negative f: two's complement, (n xor -1) - (-1)
    const unsigned neg = (unsigned)((int)hi >> 31);
    n.w0 ^= neg;
    n.w1 ^= neg;
    n.w2 ^= neg;
    return minus96(n, I96{neg, neg, neg});
}

// The biased exponent limit of to96's exact range (|f| < 16).
constexpr unsigned EXP_LIMIT = 1026u;

// v in units of 2^-48 (i.e. 2^48 times the value v 2^-80) rounded to FP64 on the integer pipe, with
// no FP64 instruction: |v| is shifted so that its leading one lands on bit 63 of a 64-bit window,
// the window's leading 53 bits are rounded to nearest, ties to even (round bit: the next bit;
// sticky: the rest of the window and the bits of v shifted out below it), and sign, exponent and
// significand are assembled into the IEEE-754 bit pattern. The result is the correctly rounded
// value. Callers fold the 2^-48 scale into later arithmetic where it cancels.
__device__ __forceinline__ double to_double48(const I96& v) {
    const unsigned s = (unsigned)((int)v.w2 >> 31);
    const I96 m = minus96(I96{v.w0 ^ s, v.w1 ^ s, v.w2 ^ s}, I96{s, s, s});  // |v| < 2^95
    // the most significant nonzero word of |v| (x2) and the two words below it
    const bool t2 = m.w2 != 0u, t1 = m.w1 != 0u;
    const unsigned x2 = t2 ? m.w2 : (t1 ? m.w1 : m.w0);
    const unsigned x1 = t2 ? m.w1 : (t1 ? m.w0 : 0u);
    const unsigned x0 = t2 ? m.w0 : 0u;
    const int base = t2 ? 64 : (t1 ? 32 : 0);  // the bit of v that is bit 0 of x2
    const int z = __clz(x2);                   // 32 only for v = 0
    const unsigned lo = __funnelshift_l(x0, x1, z);
    const unsigned long long W = ((unsigned long long)__funnelshift_l(x1, x2, z) << 32) | lo;
    // t = the leading 53 bits and the round bit; x = 1 rounds up a set round bit (sticky or odd)
    const unsigned long long t = W >> 10;
    const unsigned sticky = (lo & 0x3FFu) | (x0 << (z & 31));  // x0 = 0 unless z < 32
    const unsigned long long x = (sticky != 0u ? 1ull : 0ull) | ((t >> 1) & 1ull);
    const unsigned long long sig = (t + x) >> 1;  // 53 bits (2^53 if rounding carried)
    // leading one of |v| at bit base + 31 - z, i.e. 2^(base - 1 - z) in units of 2^-48: biased
    // exponent base + 1022 - z; adding sig (implicit one at bit 52) to (exponent - 1) << 52 sets
    // the exponent field, and a rounding carry moves it up by one
    const unsigned long long e1 = (unsigned long long)(base + 1021 - z);
    const unsigned long long bits = ((e1 << 52) + sig) | ((unsigned long long)(s & 0x80000000u) << 32);
    return z == 32 ? 0.0 : __longlong_as_double((long long)bits);
}

}  // namespace fx
}  // namespace lbg
