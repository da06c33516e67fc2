/* Exhaustive check of the exact quotient from a correctly rounded reciprocal
 * (Markstein 1990): with r = RN(1/d), q0 = RN(a r), e = fma(-q0, d, a),
 * q1 = fma(e, r, q0), q1 must equal the IEEE quotient RN(a / d).
 *
 * Checked for every float significand of a (all 2^23 values), both signs, at
 * a few exponents (the sequence scales exactly with a power of two while the
 * values stay normal), for the divisors the integration's update divides by:
 * W + 1 for the integer weights 0..255, and truncation bands mu.  Prints the
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

int main(int argc, char **argv)
{
    long long bad = 0, bad_q0 = 0;
    const int exps[] = {-20, 0, 7};
    for (int d = 1; d <= 256; ++d)
        for (int k = 0; k < 3; ++k) check((float)d, exps[k], &bad, &bad_q0);
    for (int i = 1; i < argc; ++i)
        for (int k = 0; k < 3; ++k) check(strtof(argv[i], NULL), exps[k] - 10, &bad, &bad_q0);
    printf("%lld %lld\n", bad, bad_q0);
    return 0;
}
