/*
 * Drives every function of the C oracle on small seeded inputs, edge cases
 * included (no fragments, one pixel, J = 1..5, every flag set, rejected
 * inputs), so that a build with AddressSanitizer and UndefinedBehaviorSanitizer
 * checks the oracle's memory accesses and arithmetic.  Exit status 0 when
 * every call returned the expected status.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "wt_oracle.h"

static uint64_t state = 88172645463325252ull;
static double urand(void) { /* xorshift64 */
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return (double)(state >> 11) * (1.0 / 9007199254740992.0);
}

static int fail(const char *what, int got, int want) {
    fprintf(stderr, "%s returned %d, expected %d\n", what, got, want);
    return 1;
}

static int run(int64_t n, int64_t P, int J, uint32_t flags) {
    const int64_t C = (int64_t)1 << J;
    uint32_t *pixel = malloc(sizeof(uint32_t) * (size_t)(n + 1));
    float *z = malloc(sizeof(float) * (size_t)(n + 1)), *alpha = malloc(sizeof(float) * (size_t)(n + 1));
    float *r = malloc(sizeof(float) * (size_t)(n + 1)), *g = malloc(sizeof(float) * (size_t)(n + 1));
    float *b = malloc(sizeof(float) * (size_t)(n + 1));
    double *coeff = calloc((size_t)(P * C), sizeof(double)), *coeff2 = calloc((size_t)(P * C), sizeof(double));
    double *Ahat = malloc(sizeof(double) * (size_t)(n + 1)), *accum = malloc(sizeof(double) * (size_t)(P * 6));
    double *out = malloc(sizeof(double) * (size_t)(P * 4)), *out2 = malloc(sizeof(double) * (size_t)(P * 4));
    double *gout = malloc(sizeof(double) * (size_t)(P * 4)), *ga = malloc(sizeof(double) * (size_t)(n + 1));
    double *grgb = malloc(sizeof(double) * (size_t)(3 * n + 3)), *bg_img = malloc(sizeof(double) * (size_t)(P * 3));
    double *zlo = malloc(sizeof(double) * (size_t)P), *zhi = malloc(sizeof(double) * (size_t)P);
    double *zn = malloc(sizeof(double) * (size_t)(n + 1)), *Abar = malloc(sizeof(double) * (size_t)C);
    const double bg[3] = {0.2, 0.5, 0.8};
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        pixel[i] = (uint32_t)(urand() * (double)P);
        z[i] = (float)urand();
        alpha[i] = (float)(urand() * 0.95);
        r[i] = (float)urand();
        g[i] = (float)urand();
        b[i] = (float)urand();
    }
    for (int64_t i = 0; i < P * 4; ++i) gout[i] = urand() - 0.5;
    for (int64_t i = 0; i < P * 3; ++i) bg_img[i] = urand();
    int st;
    if ((st = wto_build(n, pixel, z, alpha, P, J, coeff)) != WTO_OK) bad |= fail("wto_build", st, WTO_OK);
    if ((st = wto_build_binned(n, pixel, z, alpha, P, J, coeff2)) != WTO_OK)
        bad |= fail("wto_build_binned", st, WTO_OK);
    wto_bin_values(coeff, J, Abar);
    (void)wto_recon(Abar, J, 0.37, 1);
    (void)wto_recon(Abar, J, 0.99, 0);
    (void)wto_psi(J - 1, 0, 0.3);
    (void)wto_Psi(J - 1, 0, 0.3);
    if ((st = wto_fragment_absorbance(n, pixel, z, alpha, P, J, flags, coeff, Ahat)) != WTO_OK)
        bad |= fail("wto_fragment_absorbance", st, WTO_OK);
    if ((st = wto_absorbance_at(n, pixel, z, P, J, flags, coeff, Ahat)) != WTO_OK)
        bad |= fail("wto_absorbance_at", st, WTO_OK);
    if ((st = wto_resolve(n, pixel, z, alpha, r, g, b, P, J, flags, coeff, bg, NULL, accum, out)) != WTO_OK)
        bad |= fail("wto_resolve", st, WTO_OK);
    if ((st = wto_resolve(n, pixel, z, alpha, r, g, b, P, J, flags, coeff, bg, bg_img, NULL, out2)) != WTO_OK)
        bad |= fail("wto_resolve (bg image)", st, WTO_OK);
    if ((st = wto_abuffer(n, pixel, z, alpha, r, g, b, P, bg, NULL, out2)) != WTO_OK)
        bad |= fail("wto_abuffer", st, WTO_OK);
    if ((st = wto_grad(n, pixel, z, alpha, r, g, b, P, J, flags, bg, NULL, gout, ga, grgb)) != WTO_OK)
        bad |= fail("wto_grad", st, WTO_OK);
    if ((st = wto_depth_bounds(n, pixel, z, alpha, P, zlo, zhi)) != WTO_OK)
        bad |= fail("wto_depth_bounds", st, WTO_OK);
    if ((st = wto_normalize_depth(n, pixel, z, P, zlo, zhi, zn)) != WTO_OK)
        bad |= fail("wto_normalize_depth", st, WTO_OK);
    if (n > 0) {
        /* rejected inputs: a pixel id past the image, then a NaN depth */
        const uint32_t keep = pixel[0];
        pixel[0] = (uint32_t)P;
        if ((st = wto_build(n, pixel, z, alpha, P, J, coeff)) != WTO_ERR_INPUT)
            bad |= fail("wto_build (bad pixel)", st, WTO_ERR_INPUT);
        pixel[0] = keep;
        z[0] = NAN;
        if ((st = wto_build(n, pixel, z, alpha, P, J, coeff)) != WTO_ERR_INPUT)
            bad |= fail("wto_build (NaN depth)", st, WTO_ERR_INPUT);
    }
    free(pixel); free(z); free(alpha); free(r); free(g); free(b); free(coeff); free(coeff2); free(Ahat);
    free(accum); free(out); free(out2); free(gout); free(ga); free(grgb); free(bg_img); free(zlo); free(zhi);
    free(zn); free(Abar);
    return bad;
}

int main(void) {
    int bad = 0;
    const uint32_t flag_sets[4] = {7u, 3u, 5u, 6u};
    for (int J = 1; J <= 5; ++J)
        for (int f = 0; f < 4; ++f) {
            bad |= run(0, 5, J, flag_sets[f]);
            bad |= run(1, 1, J, flag_sets[f]);
            bad |= run(300, 17, J, flag_sets[f]);
        }
    if (!bad) printf("oracle sanitizer run: ok\n");
    return bad;
}
