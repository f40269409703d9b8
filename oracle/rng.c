/* Counter-based random numbers and Poisson draws - TEST INFRASTRUCTURE ONLY (part of the
 * oracle; see oracle.c's header for who may call it).
 *
 * Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3" (SC'11): a 4 x 32-bit counter and a 2 x 32-bit key; each of the ten rounds
 * multiplies words 0 and 2 by the two round multipliers, takes the high and low halves and
 * XORs the high halves with the other words and the round key; the key is bumped by the two
 * Weyl constants between rounds.
 *
 * Poisson(mu) pseudo-data, element i of a call (seed, offset): counters (i + offset lo, hi,
 * draw, 0) under key (seed lo, seed hi), four uniforms per counter, u = (m + 1/2) 2^-23 from the
 * top 23 bits of each word. mu < 10: the multiplication method (Knuth, TAOCP vol. 2, 3.4.1):
 * the smallest k with u_0 ... u_k <= exp(-mu). mu >= 10: Hormann's PTRS (W. Hormann, "The
 * transformed rejection method for generating Poisson random variables", Insurance:
 * Mathematics and Economics 12 (1993)), transformed rejection with a squeeze, in the step
 * order of that paper. Float steps are written one rounding at a time (compile with
 * -ffp-contract=off) and the acceptance test is evaluated in double.
 */
#include <math.h>
#include <stdint.h>

static void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t out0 = hi1 ^ c[1] ^ k0;
    const uint32_t out2 = hi0 ^ c[3] ^ k1;
    c[0] = out0;
    c[1] = lo1;
    c[2] = out2;
    c[3] = lo0;
}

/* ctr is replaced by Philox4x32-10(ctr, key) */
void orc_philox4x32_10(uint32_t ctr[4], const uint32_t key[2]) {
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        philox_round(ctr, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

typedef struct {
    uint32_t ctr_lo, ctr_hi, key[2], draw;
    uint32_t word[4];
    int used;
} orc_stream;

static float stream_uniform(orc_stream *s) {
    if (s->used == 4) {
        uint32_t c[4] = {s->ctr_lo, s->ctr_hi, s->draw, 0u};
        s->draw++;
        orc_philox4x32_10(c, s->key);
        for (int i = 0; i < 4; ++i) s->word[i] = c[i];
        s->used = 0;
    }
    const uint32_t m = s->word[s->used++] >> 9;
    return ((float)m + 0.5f) * (1.0f / 8388608.0f);
}

/* One PTRS trial for mean mu >= 10 with U uniform on (-1/2, 1/2) and V on (0, 1): the accepted
 * count k, or -1 when the pair is rejected. */
float orc_ptrs_step(float mu, float U, float V) {
    const float smu = sqrtf(mu);
    const float b = fmaf(2.53f, smu, 0.931f);
    const float a = fmaf(0.02483f, b, -0.059f);
    const float inv_alpha = 1.1239f + 1.1328f / (b - 3.4f);
    const float v_r = 0.9277f - 3.6224f / (b - 2.0f);
    const float us = 0.5f - fabsf(U);
    const float scaled = (2.0f * a) / us + b;
    const float k = floorf((scaled * U + mu) + 0.43f);
    if (us >= 0.07f && V <= v_r) return k;                 /* squeeze: immediate accept */
    if (k < 0.0f || (us < 0.013f && V > us)) return -1.0f; /* outside the hat */
    const double lhs = log((double)V) + log((double)inv_alpha) -
                       log((double)a / ((double)us * (double)us) + (double)b);
    const double rhs = -(double)mu + (double)k * log((double)mu) - lgamma((double)k + 1.0);
    return lhs <= rhs ? k : -1.0f;
}

/* orc_ptrs_step for n pairs */
void orc_ptrs_step_many(float mu, int64_t n, const float *U, const float *V, float *k) {
    for (int64_t i = 0; i < n; ++i) k[i] = orc_ptrs_step(mu, U[i], V[i]);
}

static float poisson_one(float mu, orc_stream *s) {
    if (!(mu > 0.0f)) return mu == 0.0f ? 0.0f : NAN;
    if (!(mu < 4194304.0f)) return NAN;
    if (mu < 10.0f) {
        const float limit = (float)exp(-(double)mu);
        float prod = 1.0f;
        for (int k = 0; k < 1000; ++k) {
            prod = prod * stream_uniform(s);
            if (prod <= limit) return (float)k;
        }
        return 1000.0f;
    }
    for (int it = 0; it < 1000; ++it) {
        const float U = stream_uniform(s) - 0.5f;
        const float V = stream_uniform(s);
        const float k = orc_ptrs_step(mu, U, V);
        if (k >= 0.0f) return k;
    }
    return rintf(mu);
}

/* out[i] ~ Poisson(mu[i]), i < n, element i on counters (i + offset, draw, 0, 0), key seed */
void orc_poisson_sample(int64_t n, const float *mu, uint64_t seed, uint64_t offset, float *out) {
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t c = (uint64_t)i + offset;
        orc_stream s;
        s.ctr_lo = (uint32_t)c;
        s.ctr_hi = (uint32_t)(c >> 32);
        s.key[0] = (uint32_t)seed;
        s.key[1] = (uint32_t)(seed >> 32);
        s.draw = 0;
        s.used = 4;
        out[i] = poisson_one(mu[i], &s);
    }
}
