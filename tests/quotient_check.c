/* Exhaustive check of the exact quotient from a correctly rounded reciprocal
 * (Markstein 1990): with r = RN(1/d), q0 = RN(a r), e = fma(-q0, d, a),
 * q1 = fma(e, r, q0), q1 must equal the IEEE quotient RN(a / d).
 *
 * Checked for every float significand of a (all 2^23 values), both signs, at
 * a few exponents (the sequence scales exactly with a power of two while the
 * values stay normal), for the divisors the integration's update divides by:
 * W + 1 for the integer weights 0..255, and truncation bands mu, and for
 * pseudo-random divisors (the projection's division by a voxel's depth Z,
 * with one reciprocal of Z shared by its two quotients).  Prints the
 * number of mismatches of the sequence and, as a control, of q0 alone.
 * Build: gcc -O2 -fopenmp -ffp-contract=off (float operations rounded one by
 * one; fmaf is the fused multiply-add). */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static float from_bits(uint32_t u)
{
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static void check(float d, int exponent, long long *bad, long long *bad_q0)
{
    volatile float one = 1.0f;
    const float r = one / d;
    long long b = 0, b0 = 0;
#pragma omp parallel for reduction(+ : b, b0) schedule(static)
    for (long long m = 0; m < (1LL << 23); ++m) {
        for (int sgn = 0; sgn < 2; ++sgn) {
            uint32_t u = (uint32_t)(127 + exponent) << 23 | (uint32_t)m;
            if (sgn) u |= 0x80000000u;
            const float a = from_bits(u);
            const float q0 = a * r;
            const float e = fmaf(-q0, d, a);
            const float q1 = fmaf(e, r, q0);
            const float want = a / d;
            b += memcmp(&q1, &want, 4) != 0;
            b0 += memcmp(&q0, &want, 4) != 0;
        }
    }
    *bad += b;
    *bad_q0 += b0;
}

/* argv[1]: how many pseudo-random divisors in [1/16, 16) (xorshift64, the
 * first four with significands next to all ones); argv[2..]: further
 * divisors (the mu values). */
int main(int argc, char **argv)
{
    long long bad = 0, bad_q0 = 0;
    const int exps[] = {-20, 0, 7};
    for (int d = 1; d <= 256; ++d)
        for (int k = 0; k < 3; ++k) check((float)d, exps[k], &bad, &bad_q0);
    const int n_random = argc > 1 ? atoi(argv[1]) : 0;
    uint64_t x = 88172645463325252ull;
    for (int t = 0; t < n_random; ++t) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        uint32_t mant = (uint32_t)(x & 0x7fffffu);
        if (t < 4) mant = 0x7fffffu - (uint32_t)t;
        const int ex = (int)((x >> 32) % 8) - 4;
        check(from_bits((uint32_t)(127 + ex) << 23 | mant), 0, &bad, &bad_q0);
    }
    for (int i = 2; i < argc; ++i)
        for (int k = 0; k < 3; ++k) check(strtof(argv[i], NULL), exps[k] - 10, &bad, &bad_q0);
    printf("%lld %lld\n", bad, bad_q0);
    return 0;
}
