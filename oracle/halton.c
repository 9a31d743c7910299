/*
 * Oracle: scrambled Halton sequence evaluated exactly (Appendix A.2) and the
 * full-screen sample enumeration it is used with (Appendix A.2, "samples are
 * enumerated over the full screen without tiling", 64-bit indices).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Definitions written out here:
 *   phi_b(i)   = sum_k pi_b(d_k(i)) b^(-k-1), d_k the base-b digits of i;
 *   pi_b(d)    = (f_b * d) mod b, a linear digit permutation with pi(0) = 0
 *                (the paper cites a scrambling it does not print; this is the
 *                linear-multiplier reading, with f_b drawn from SplitMix64);
 *   u32 value  = floor(2^32 * phi_b(i)), computed from the exact rational
 *                num / b^n with 128-bit integers (no rounding anywhere);
 *   FP32 value = (u32 >> 8) * 2^-24, exactly representable.
 * Divisions here are plain C '/' and '%': the oracle does not use the
 * strength-reduced division the paper describes; it checks it.
 */
#include "oracle.h"
#include <math.h>

static uint32_t g_primes[4096];
static int g_nprimes = 0;

static void init_primes(void) {
    if (g_nprimes) return;
    int n = 0;
    for (uint32_t c = 2; n < 4096; ++c) {
        int is_p = 1;
        for (uint32_t q = 2; q * q <= c; ++q)
            if (c % q == 0) { is_p = 0; break; }
        if (is_p) g_primes[n++] = c;
    }
    g_nprimes = n;
}

uint32_t or_prime(int dim) {
    init_primes();
    if (dim < 0 || dim >= g_nprimes) return 0;
    return g_primes[dim];
}

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): one generator step. */
uint64_t or_splitmix64(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Multiplier f_b of the linear digit scramble: state = seed + b, draw
 * 1 + z mod (b-1) until it is not 1 (base 2 stays unscrambled, f = 1). */
uint32_t or_scramble_factor(uint64_t seed, uint32_t b) {
    if (b <= 2) return 1;
    uint64_t st = seed + (uint64_t)b;
    for (;;) {
        uint64_t z = or_splitmix64(&st);
        uint32_t f = 1u + (uint32_t)(z % (uint64_t)(b - 1));
        if (f != 1u) return f;
    }
}

uint32_t or_radical_inverse_u32(uint32_t b, uint32_t f, uint64_t i) {
    unsigned __int128 num = 0, den = 1;
    while (i > 0) {
        uint64_t d = i % b;
        i = i / b;
        num = num * b + (unsigned __int128)((f * d) % b);
        den = den * b;
    }
    return (uint32_t)((num << 32) / den);
}

double or_u32_to_unit(uint32_t u) { return (double)(u >> 8) * 0x1p-24; }

/* Smallest k with 2^k >= W and smallest l with 3^l >= H. */
void or_enum_params(uint32_t W, uint32_t H, uint32_t *k, uint32_t *l,
                    uint64_t *p2, uint64_t *p3) {
    uint32_t kk = 0; uint64_t a = 1;
    while (a < W) { a *= 2; ++kk; }
    uint32_t ll = 0; uint64_t c = 1;
    while (c < H) { c *= 3; ++ll; }
    *k = kk; *l = ll; *p2 = a; *p3 = c;
}

/* The unique i in [0, 2^k 3^l) whose first Halton coordinate scaled by 2^k
 * has integer part x and whose second coordinate scaled by 3^l has integer
 * part y: i mod 2^k is x with its k bits reversed, i mod 3^l is y with its l
 * base-3 digits reversed; i itself is found by plain search. */
uint64_t or_pixel_base_index(uint32_t W, uint32_t H, uint32_t x, uint32_t y) {
    uint32_t k, l; uint64_t p2, p3;
    or_enum_params(W, H, &k, &l, &p2, &p3);
    uint64_t a = 0;
    for (uint32_t t = 0; t < k; ++t)
        if (x & (1u << t)) a |= 1ull << (k - 1 - t);
    uint64_t c = 0, yy = y;
    for (uint32_t t = 0; t < l; ++t) {  /* digit t of y goes to digit l-1-t */
        uint64_t d = yy % 3; yy /= 3;
        uint64_t pw = 1;
        for (uint32_t s = 0; s < l - 1 - t; ++s) pw *= 3;
        c += d * pw;
    }
    for (uint64_t m = 0; m < p2; ++m) {
        uint64_t i = c + m * p3;
        if (i % p2 == a) return i;
    }
    return UINT64_MAX; /* unreachable: 2^k and 3^l are coprime */
}

/* Sample value of dimension `dim` for sequence index `index`.
 * dim 0: phi_2(floor(i / 2^k)); dim 1: phi_3(floor(i / 3^l)) (the in-pixel
 * offset, unscrambled); dim >= 2: scrambled phi_{prime(dim)}(i). */
double or_sample_dim(uint64_t index, int dim, uint32_t k, uint32_t l,
                     const uint32_t *factors) {
    uint32_t u;
    if (dim == 0) {
        u = or_radical_inverse_u32(2, 1, index >> k);
    } else if (dim == 1) {
        uint64_t p3 = 1;
        for (uint32_t s = 0; s < l; ++s) p3 *= 3;
        u = or_radical_inverse_u32(3, 1, index / p3);
    } else {
        u = or_radical_inverse_u32(or_prime(dim), factors[dim], index);
    }
    return or_u32_to_unit(u);
}

void or_sample_dims_batch(const uint64_t *idx, int64_t n, int ndims,
                          uint32_t W, uint32_t H, uint64_t seed,
                          uint32_t *out) {
    uint32_t k, l; uint64_t p2, p3;
    or_enum_params(W, H, &k, &l, &p2, &p3);
    for (int64_t r = 0; r < n; ++r) {
        for (int d = 0; d < ndims; ++d) {
            uint32_t u;
            if (d == 0) u = or_radical_inverse_u32(2, 1, idx[r] >> k);
            else if (d == 1) u = or_radical_inverse_u32(3, 1, idx[r] / p3);
            else {
                uint32_t b = or_prime(d);
                u = or_radical_inverse_u32(b, or_scramble_factor(seed, b), idx[r]);
            }
            out[r * ndims + d] = u;
        }
    }
}
