// Integer-exact scrambled Halton sampling (Appendix A.2 of the paper):
// radical inverses of 64-bit sequence indices evaluated with integer
// arithmetic only, divisions by the constant bases strength-reduced to a
// multiply-high and a shift (Granlund and Montgomery, PLDI 1994), and the
// full-screen enumeration of samples over pixels.
//
// Exactness: the value returned for base b, digit permutation pi and index i
// is floor(2^32 * phi_b(i)), phi_b(i) = sum_k pi(d_k) b^(-k-1). It is computed
// by Horner's rule from the most significant digit down,
//     y_n = 0,  y_k = floor((2^32 * pi(d_k) + y_(k+1)) / b),  result = y_0,
// which is exact because floor((a + x) / b) == floor((a + floor(x)) / b) for
// integers a, b. Digits are extracted least significant first and buffered
// in a 128-bit register pair (at most 115 bits for 64-bit indices and
// ceil(log2 b) bits per digit), so no local memory is touched.
#pragma once

#include "common.cuh"

namespace rtg {

// Multiply-high helpers usable on host and device.
RT_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}
RT_HD uint32_t umulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Division by a constant d >= 2 with the "N+1-bit magic" of Granlund and
// Montgomery: m = floor(2^N (2^l - d) / d) + 1, l = ceil(log2 d);
// q = (t + ((n - t) >> 1)) >> (l - 1), t = mulhi(m, n). Exact for all N-bit n.
struct Divisor {
    uint64_t m64;
    uint32_t m32;
    uint32_t d;
    uint32_t sh;   // l - 1
};

inline Divisor make_divisor(uint32_t d) {
    Divisor r{};
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    r.d = d;
    r.sh = l - 1;
    unsigned __int128 num = ((unsigned __int128)1 << 64) * (unsigned __int128)((1ull << l) - d);
    r.m64 = (uint64_t)(num / d) + 1;
    r.m32 = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    return r;
}

RT_HD uint64_t div64(uint64_t n, const Divisor &v) {
    uint64_t t = umulhi64(v.m64, n);
    return (t + ((n - t) >> 1)) >> v.sh;
}
RT_HD uint32_t div32(uint32_t n, const Divisor &v) {
    uint32_t t = umulhi32(v.m32, n);
    return (t + ((n - t) >> 1)) >> v.sh;
}

// Most base-b digits of a 64-bit index (b = 3: 3^40 < 2^64 < 3^41).
constexpr int kMaxDigits = 41;

// One Halton dimension: base, its divisor, digit scramble multiplier, the
// number of bits that hold one digit, and the digit weights
// w[k] = floor(2^64 / b^(k+1)) of the fixed-point evaluation.
struct HaltonDim {
    Divisor div;
    uint32_t f;     // pi(d) = (f * d) mod b
    uint32_t bits;  // ceil(log2 b)
    uint64_t w[kMaxDigits];
};

RT_HD uint32_t scramble_digit(uint32_t d, const HaltonDim &h) {
    uint32_t fd = h.f * d;
    return fd - div32(fd, h.div) * h.div.d;
}

// floor(2^32 * phi_b(i)) by Horner's rule (b > 2), exact for every index.
RT_HD uint32_t radical_inverse_horner(uint64_t i, const HaltonDim &h) {
    const uint32_t b = h.div.d;
    const uint32_t bits = h.bits;
    const uint64_t mask = (1ull << bits) - 1ull;
    uint64_t lo = 0, hi = 0;
    int n = 0;
    while (i >> 32) {
        uint64_t q = div64(i, h.div);
        uint64_t d = i - q * b;
        i = q;
        hi = (hi << bits) | (lo >> (64 - bits));
        lo = (lo << bits) | d;
        ++n;
    }
    uint32_t i32 = (uint32_t)i;
    while (i32) {
        uint32_t q = div32(i32, h.div);
        uint32_t d = i32 - q * b;
        i32 = q;
        hi = (hi << bits) | (lo >> (64 - bits));
        lo = (lo << bits) | d;
        ++n;
    }
    uint64_t y = 0;
    for (int k = 0; k < n; ++k) {
        uint32_t d = (uint32_t)(lo & mask);
        lo = (lo >> bits) | (hi << (64 - bits));
        hi >>= bits;
        uint64_t num = ((uint64_t)scramble_digit(d, h) << 32) + y;
        y = div64(num, h.div);
    }
    return (uint32_t)y;
}

// floor(2^32 * phi_b(i)) with the digit permutation of `h`.
//
// Fast path: the 64-bit fixed-point sum S = sum_k pi(d_k) w[k] with
// w[k] = floor(2^64 / b^(k+1)) under-estimates T = 2^64 phi_b(i) by
// T - S = sum_k pi(d_k) frac(2^64 / b^(k+1)) < n (b - 1) for n digits, and
// T < 2^64 so S cannot wrap. Hence floor(T / 2^32) = floor(S / 2^32)
// whenever (S mod 2^32) + n (b - 1) <= 2^32; otherwise (about one index in
// 2^32 / (n b)) the exact Horner evaluation decides. One digit costs a
// 32-bit multiply-high division, the scramble and one 64 x 32-bit
// multiply-add instead of two divisions and a 128-bit digit buffer.
RT_HD uint32_t radical_inverse(uint64_t i, const HaltonDim &h) {
    const uint32_t b = h.div.d;
    if (b == 2u) {
#ifdef __CUDA_ARCH__
        return __brev((uint32_t)i);
#else
        uint32_t x = (uint32_t)i, r = 0;
        for (int k = 0; k < 32; ++k) r |= ((x >> k) & 1u) << (31 - k);
        return r;
#endif
    }
    const uint64_t i_in = i;
    uint64_t S = 0;
    uint32_t n = 0;
    while (i >> 32) {
        uint64_t q = div64(i, h.div);
        uint32_t d = (uint32_t)(i - q * b);
        i = q;
        S += (uint64_t)scramble_digit(d, h) * h.w[n];
        ++n;
    }
    uint32_t i32 = (uint32_t)i;
    while (i32) {
        uint32_t q = div32(i32, h.div);
        uint32_t d = i32 - q * b;
        i32 = q;
        S += (uint64_t)scramble_digit(d, h) * h.w[n];
        ++n;
    }
    if ((uint64_t)(uint32_t)S + (uint64_t)n * (b - 1u) <= (1ull << 32)) return (uint32_t)(S >> 32);
    return radical_inverse_horner(i_in, h);
}

// FP32 sample value from the 32-bit fraction: (u >> 8) * 2^-24, exact.
RT_HD float u32_to_unit(uint32_t u) { return (float)(u >> 8) * 5.9604644775390625e-8f; }

// Full-screen enumeration (Appendix A.2): pixel (x, y) owns the indices
// i = i0 + j * 2^k 3^l with i mod 2^k = reverse_k(x), i mod 3^l =
// reverse3_l(y); i0 by the Chinese remainder theorem with precomputed
// idempotents e2 = 1 mod 2^k, 0 mod 3^l and e3 = 0 mod 2^k, 1 mod 3^l.
struct Enum {
    uint32_t k, l;        // 2^k >= W, 3^l >= H
    uint64_t p2, p3, period;  // 2^k, 3^l, 2^k 3^l
    uint64_t e2, e3;
    Divisor div_p3;       // division by 3^l (offset dimension 1)
    HaltonDim base3;      // unscrambled base 3
};

Enum make_enum(uint32_t W, uint32_t H);
HaltonDim make_dim(uint32_t base, uint32_t f);

RT_HD uint64_t pixel_base_index(const Enum &e, uint32_t x, uint32_t y) {
    uint64_t a = 0;
    for (uint32_t t = 0; t < e.k; ++t)
        if (x & (1u << t)) a |= 1ull << (e.k - 1 - t);
    uint64_t c = 0;
    uint32_t yy = y;
    for (uint32_t t = 0; t < e.l; ++t) {
        uint32_t d = yy % 3u;
        yy /= 3u;
        c = c * 3u + d;   // digit t of y becomes digit l-1-t of c
    }
    return (a * e.e2 + c * e.e3) % e.period;
}

// In-pixel offset dimensions 0 and 1 (unscrambled).
RT_HD uint32_t dim0_bits(const Enum &e, uint64_t i) {
    const uint32_t x = (uint32_t)(i >> e.k);
#ifdef __CUDA_ARCH__
    return __brev(x);
#else
    uint32_t r = 0;
    for (int k = 0; k < 32; ++k) r |= ((x >> k) & 1u) << (31 - k);
    return r;
#endif
}
RT_HD uint32_t dim1_bits(const Enum &e, uint64_t i) {
    uint64_t q = e.l ? div64(i, e.div_p3) : i;
    return radical_inverse(q, e.base3);
}

}  // namespace rtg
