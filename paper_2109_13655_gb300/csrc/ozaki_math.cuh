// The arithmetic of the FP64-accurate products from BF16 slices (ozaki.cu): the slicing of
// an FP64 value under a power-of-two scale, and the single rounding of the exact integer level
// sums back to FP64. Host and device code, so that the CPU tests exercise these functions
// against exact rational arithmetic.
//
// Slicing: with 2^e > |x| / 2 the largest magnitude sharing x's scale (e = ilogb of the
// largest |x|), V = floor(|x| 2^(56 - e - 1)) < 2^56 is cut into S = 8 fields of 7 bits,
// d_p = (V >> 7 (S - 1 - p)) & 127 with the sign of x: x = sign 2^(e+1) sum_p d_p 2^(-7 (p+1))
// + r with |r| < 2^(e + 1 - 56). Every d_p is an integer of at most 7 bits, exact in BF16.
//
// Levels: the product of slices p and q (counted from 1) carries the scale 2^(-7 (p + q)).
// With the level sums s_k of the products of level k = p + q (integers), the epilogues form
//   th = sum_{k=2..5} s_k 2^(7 (5 - k)),  tl = sum_{k=6..9} s_k 2^(7 (9 - k)),
// so that sum_k s_k 2^(-7 k) = th 2^-35 + tl 2^-63 = (th 2^28 + tl) 2^-63, and round that
// once to FP64 (oz_to_double).
#pragma once
#include <climits>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#endif

namespace cmsvd {

constexpr int OZ_S = 8;      // slices
constexpr int OZ_BITS = 7;   // bits per slice

OZ_HD uint64_t oz_bits(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}
OZ_HD double oz_from_bits(uint64_t b) {
    double x;
    memcpy(&x, &b, 8);
    return x;
}
OZ_HD int oz_clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// ilogb of a nonzero v from its exponent field (integer work; a subnormal counts as 2^-1023,
// an upper bound of its ilogb, which the slicing accepts as a scale)
OZ_HD int oz_ilogb(double v) { return (int)((oz_bits(v) >> 52) & 0x7ff) - 1023; }

// The S slices of x under the scale 2^(e+1), e >= ilogb(|x|) (see above).
OZ_HD void oz_slices(double x, int e, float (&d)[OZ_S]) {
    const uint64_t b = oz_bits(x);
    const int E = (int)((b >> 52) & 0x7ff);
    uint64_t m = b & ((1ull << 52) - 1);
    int Ee = E;
    if (E == 0) Ee = 1;
    else m |= 1ull << 52;
    // |x| = m 2^(Ee-1075); V = floor(|x| 2^(56-e-1)) = m >> (1075 - Ee + e + 1 - 56), below 2^56
    // since |x| < 2^(e+1); the shift is -3 for the largest value of a normal scale group
    const int sh = 1075 - Ee + e + 1 - OZ_BITS * OZ_S;
    const uint64_t V = ((b << 1) == 0 || sh >= 64) ? 0ull : (sh >= 0 ? (m >> sh) : (m << (-sh)));
    const float sg = (b >> 63) ? -1.f : 1.f;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int p = 0; p < OZ_S; ++p) d[p] = sg * (float)(int)((V >> (OZ_BITS * (OZ_S - 1 - p))) & 127ull);
}

// (th 2^-35 + tl 2^-63) 2^sc rounded once to the nearest double (ties to even), in integer
// operations only; results below the normal range flush to (signed) zero, above it to
// infinity. |th|, |tl| < 2^53.
OZ_HD double oz_to_double(long long th, long long tl, int sc) {
    const __int128 T = (__int128)th * (1ll << 28) + tl;   // value = T 2^(sc - 63), |T| < 2^82
    if (T == 0) return 0.0;
    const bool neg = T < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
    const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
    const int msb = hi ? 127 - oz_clz64(hi) : 63 - oz_clz64(lo);
    const int sh = msb - 52;
    uint64_t m;
    if (sh > 0) {
        m = (uint64_t)(a >> sh);
        const unsigned __int128 rem = a & ((((unsigned __int128)1) << sh) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
        if (rem > half || (rem == half && (m & 1))) ++m;
    } else {
        m = lo << (-sh);
    }
    int e = sh + sc - 63;   // value = m 2^e, m in [2^52, 2^53]
    if (m == (1ull << 53)) {
        m >>= 1;
        ++e;
    }
    const int field = e + 52 + 1023;
    const uint64_t sign = (uint64_t)neg << 63;
    if (field <= 0) return oz_from_bits(sign);
    if (field >= 2047) return oz_from_bits(sign | (0x7ffull << 52));
    return oz_from_bits(sign | ((uint64_t)field << 52) | (m & 0xfffffffffffffull));
}

}  // namespace cmsvd
