// Extended-range values ("XD") for the heuristic modes.
//
// IDP2 and UnionDP (Sec. 4) join plans of hundreds of relations, whose
// cardinalities leave binary64's range.  An XD value is m * 2^e with m = 0
// or 1 <= m < 2 and a 32-bit e:
//   mul: m = m_a * m_b (one rounded binary64 multiply), e = e_a + e_b,
//        then halve m (exactly) once if it reached 2;
//   add: with e_a >= e_b and d = e_a - e_b, m = m_a + m_b * 2^-d (one rounded
//        binary64 add; the second term is dropped for d > 60, which rounds
//        the same), e = e_a, then halve m once if it reached 2;
//   order: 0 first, then by e, then by m.
// Power-of-two scaling is exact, so every operation rounds as binary64 does
// on the same real values whenever binary64 would stay in its normal range.
#pragma once

#include <cstdint>

namespace mpdp {

struct alignas(16) XD {
    double m;
    int32_t e;
    int32_t pad;
};

__host__ __device__ __forceinline__ XD xd_zero() { return XD{0.0, 0, 0}; }

// 2^-d for 0 <= d <= 1022, exactly, from its bit pattern
__host__ __device__ __forceinline__ double pow2_neg(int d)
{
    const unsigned long long bits = (unsigned long long)(1023 - d) << 52;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double r;
    __builtin_memcpy(&r, &bits, sizeof(r));
    return r;
#endif
}

// c * 2^e2 for a finite c >= 0 (binary64 subnormals included)
__host__ __device__ __forceinline__ XD xd_make(double c, int32_t e2)
{
    if (c == 0.0) return xd_zero();
    unsigned long long bits;
#ifdef __CUDA_ARCH__
    bits = (unsigned long long)__double_as_longlong(c);
#else
    __builtin_memcpy(&bits, &c, sizeof(bits));
#endif
    int be = (int)((bits >> 52) & 0x7ff);
    if (be == 0) {  // subnormal: scale up by 2^64 first (exact)
        const double up = c * 18446744073709551616.0;
#ifdef __CUDA_ARCH__
        bits = (unsigned long long)__double_as_longlong(up);
#else
        __builtin_memcpy(&bits, &up, sizeof(bits));
#endif
        be = (int)((bits >> 52) & 0x7ff);
        e2 -= 64;
    }
    const unsigned long long mb = (bits & 0x000fffffffffffffull) | (1023ull << 52);
    double m;
#ifdef __CUDA_ARCH__
    m = __longlong_as_double((long long)mb);
#else
    __builtin_memcpy(&m, &mb, sizeof(m));
#endif
    return XD{m, e2 + be - 1023, 0};
}

__host__ __device__ __forceinline__ XD xd_mul(XD a, XD b)
{
    if (a.m == 0.0 || b.m == 0.0) return xd_zero();
#ifdef __CUDA_ARCH__
    double m = __dmul_rn(a.m, b.m);
#else
    double m = a.m * b.m;
#endif
    int32_t e = a.e + b.e;
    if (m >= 2.0) {
        m *= 0.5;
        e += 1;
    }
    return XD{m, e, 0};
}

__host__ __device__ __forceinline__ XD xd_add(XD a, XD b)
{
    if (a.m == 0.0) return b;
    if (b.m == 0.0) return a;
    if (a.e < b.e) {
        const XD t = a;
        a = b;
        b = t;
    }
    const long long d = (long long)a.e - (long long)b.e;
    double m = a.m;
    if (d <= 60) {
#ifdef __CUDA_ARCH__
        m = __dadd_rn(a.m, __dmul_rn(b.m, pow2_neg((int)d)));
#else
        m = a.m + b.m * pow2_neg((int)d);
#endif
    }
    int32_t e = a.e;
    if (m >= 2.0) {
        m *= 0.5;
        e += 1;
    }
    return XD{m, e, 0};
}

// a < b in the XD order
__host__ __device__ __forceinline__ bool xd_less(XD a, XD b)
{
    if (a.m == 0.0 || b.m == 0.0) return a.m == 0.0 && b.m != 0.0;
    if (a.e != b.e) return a.e < b.e;
    return a.m < b.m;
}

__host__ __device__ __forceinline__ bool xd_equal(XD a, XD b) { return a.m == b.m && (a.m == 0.0 || a.e == b.e); }

}  // namespace mpdp
