// sl_rng.cuh -- device Wiener-increment generator.
//
// One standard normal pair per (seed, step, sample): Philox4x32-10 (Salmon,
// Moraes, Dror & Shaw, SC'11) on the counter (step, sample, 0, 0) with key
// (seed lo, seed hi); the four 32-bit words give two 52-bit integers
// x = (w0:w1) >> 12, (w2:w3) >> 12, mapped to u = (2x+1) 2^-53 in (0,1);
// Box-Muller z1 = r cos(2 pi u2), z2 = r sin(2 pi u2), r = sqrt(-2 ln u1).
// The paper draws one increment dW = sqrt(dt) z per sample, step and
// dimension, shared by all nodes and elements (Section 5.2).
//
// ln and sincospi are written out here (not CUDA's math library) so that
// every operation is an IEEE round-to-nearest add, multiply, fma, divide or
// square root in a fixed order; the intrinsics below are never contracted or
// reassociated, so the result is reproducible on any IEEE host.
//   ln x:   x = m 2^k, m in [sqrt(1/2), sqrt(2)) by an exact exponent split;
//           ln m = 2 atanh(t), t = (m-1)/(m+1), Taylor series of atanh(t)/t
//           in t^2 to degree 22 (|t| <= 0.1716); k ln 2 with a Cody-Waite
//           split constant (high part 21 bits, so k*hi is exact).
//   sincospi y, y in [0, 2]: y = j/2 + r exactly, |r| <= 1/4; Taylor series
//           of sin(pi r) and cos(pi r) to degree 19 / 18; quadrant identities.
#pragma once
#include <cstdint>

namespace sl {

struct Philox4x32 {
    static constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    static constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
    __device__ __forceinline__ static uint4 run(uint4 c, uint32_t k0, uint32_t k1)
    {
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
            const uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
            c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
            k0 += kW0;
            k1 += kW1;
        }
        return c;
    }
};

// ln 2 = kLn2Hi + kLn2Lo, kLn2Hi = 0x1.62e42p-1 (21 significant bits).
__device__ __forceinline__ double ln_unit(double x)
{
    constexpr double kLn2Hi = 0x1.62e42p-1;
    constexpr double kLn2Lo = 0x1.fdf473de6af28p-22;
    constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;
    // exact split of a positive normal double
    const unsigned long long bits = __double_as_longlong(x);
    int e = int((bits >> 52) & 0x7FF) - 1022;  // x = m 2^e, m in [1/2, 1)
    double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull);
    if (m < kSqrtHalf) {
        m = __dmul_rn(m, 2.0);
        e -= 1;
    }
    const double t = __ddiv_rn(__dadd_rn(m, -1.0), __dadd_rn(m, 1.0));
    const double s = __dmul_rn(t, t);
    double p = 1.0 / 23.0;
    p = __fma_rn(p, s, 1.0 / 21.0);
    p = __fma_rn(p, s, 1.0 / 19.0);
    p = __fma_rn(p, s, 1.0 / 17.0);
    p = __fma_rn(p, s, 1.0 / 15.0);
    p = __fma_rn(p, s, 1.0 / 13.0);
    p = __fma_rn(p, s, 1.0 / 11.0);
    p = __fma_rn(p, s, 1.0 / 9.0);
    p = __fma_rn(p, s, 1.0 / 7.0);
    p = __fma_rn(p, s, 1.0 / 5.0);
    p = __fma_rn(p, s, 1.0 / 3.0);
    p = __fma_rn(p, s, 1.0);
    const double lnm = __dmul_rn(__dmul_rn(t, p), 2.0);
    const double k = double(e);
    const double hi = __dmul_rn(k, kLn2Hi);
    const double lo = __dadd_rn(__dmul_rn(k, kLn2Lo), lnm);
    return __dadd_rn(hi, lo);
}

// (-1)^k pi^(2k+1)/(2k+1)! and (-1)^k pi^(2k)/(2k)!, k = 0..9, to nearest double.
__device__ __forceinline__ void sincospi_02(double y, double &sp, double &cp)
{
    constexpr double S[10] = {0x1.921fb54442d18p+1,  -0x1.4abbce625be53p+2, 0x1.466bc6775aae2p+1,
                              -0x1.32d2cce62bd86p-1, 0x1.50783487ee782p-4,  -0x1.e3074fde8871fp-8,
                              0x1.e8f434d018d63p-12, -0x1.6fadb9f155744p-16, 0x1.aaec32af93359p-21,
                              -0x1.8a404211f9547p-26};
    constexpr double Cc[10] = {0x1.0p+0,              -0x1.3bd3cc9be45dep+2, 0x1.03c1f081b5ac4p+2,
                               -0x1.55d3c7e3cbffap+0, 0x1.e1f506891babbp-3,  -0x1.a6d1f2a204a8cp-6,
                               0x1.f9d38a3763cc3p-10, -0x1.b6e24f44b128fp-14, 0x1.20c62c2f2d7f5p-18,
                               -0x1.2a0c591af8314p-23};
    const double j = rint(__dmul_rn(y, 2.0));
    const double r = __dadd_rn(y, -__dmul_rn(j, 0.5));
    const double r2 = __dmul_rn(r, r);
    double ps = S[9];
#pragma unroll
    for (int k = 8; k >= 0; --k) ps = __fma_rn(ps, r2, S[k]);
    const double s = __dmul_rn(ps, r);
    double pc = Cc[9];
#pragma unroll
    for (int k = 8; k >= 0; --k) pc = __fma_rn(pc, r2, Cc[k]);
    const int q = int(j) & 3;
    if (q == 0) {
        sp = s;
        cp = pc;
    } else if (q == 1) {
        sp = pc;
        cp = -s;
    } else if (q == 2) {
        sp = -s;
        cp = -pc;
    } else {
        sp = -pc;
        cp = s;
    }
}

// The two standard normals of (seed, step, sample, tag).
__device__ __forceinline__ double2 normal_pair(unsigned long long seed, uint32_t step, uint32_t sample,
                                               uint32_t tag)
{
    const uint4 w = Philox4x32::run(make_uint4(step, sample, tag, 0u), uint32_t(seed), uint32_t(seed >> 32));
    const unsigned long long x1 = ((static_cast<unsigned long long>(w.x) << 32) | w.y) >> 12;
    const unsigned long long x2 = ((static_cast<unsigned long long>(w.z) << 32) | w.w) >> 12;
    const double u1 = __dmul_rn(double(2ull * x1 + 1ull), 0x1p-53);  // exact
    const double u2 = __dmul_rn(double(2ull * x2 + 1ull), 0x1p-53);
    const double r = __dsqrt_rn(__dmul_rn(-2.0, ln_unit(u1)));
    double s, c;
    sincospi_02(__dmul_rn(2.0, u2), s, c);
    return make_double2(__dmul_rn(r, c), __dmul_rn(r, s));
}

}  // namespace sl
