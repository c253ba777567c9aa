/*
 * FP64 CPU oracle for Wavelet Transparency (paper §2).  TEST INFRASTRUCTURE
 * ONLY: used by the tests, the smoke check and the CPU-baseline leg of the
 * benchmark; never by the product path.  This header is the oracle's own and
 * is not shared with the CUDA library.
 */
#ifndef WT_ORACLE_H
#define WT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { WTO_OK = 0, WTO_ERR_ARG = 1, WTO_ERR_INPUT = 3, WTO_ERR_NOMEM = 6 };

/* reading flags (same meaning as the library's, defined independently) */
enum { OAF_SELF_EXCLUDE = 1, OAF_INTERP_LINEAR = 2, OAF_RESOLVE_NORMALIZED = 4 };

double wto_psi(int n, int k, double x);
double wto_Psi(int n, int k, double x);

/* closed-form Haar coefficients (§2.3.1), coeff = P x 2^J, heap order */
int wto_build(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
              int64_t P, int J, double *coeff);
/* independent construction: exact bin averages + orthonormal Haar analysis */
int wto_build_binned(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
                     int64_t P, int J, double *coeff);
/* Haar series of one pixel evaluated at the C bin centres */
void wto_bin_values(const double *coeff, int J, double *Abar);
/* reconstruction at depth x from bin values (linear or staircase) */
double wto_recon(const double *Abar, int J, double x, int linear);
/* absorbance in front of every fragment (self term removed under OAF_SELF_EXCLUDE) */
int wto_fragment_absorbance(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
                            int64_t P, int J, uint32_t flags, const double *coeff, double *Ahat);
/* reconstruction A(z) at arbitrary (pixel, depth) queries */
int wto_absorbance_at(int64_t q, const uint32_t *pixel, const float *z, int64_t P, int J,
                      uint32_t flags, const double *coeff, double *Aout);
/* resolve + composite; accum = P x 6 {R',G',B',W',S,Amin} (nullable), out = P x 4 (nullable) */
int wto_resolve(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
                const float *r, const float *g, const float *b, int64_t P, int J, uint32_t flags,
                const double *coeff, const double *bg, const double *bg_img, double *accum, double *out);
/* exact sorted front-to-back composite */
int wto_abuffer(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
                const float *r, const float *g, const float *b, int64_t P,
                const double *bg, const double *bg_img, double *out);
/* analytic gradient of <gout, out> w.r.t. alpha (n) and rgb (n x 3) */
int wto_grad(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
             const float *r, const float *g, const float *b, int64_t P, int J, uint32_t flags,
             const double *bg, const double *bg_img, const double *gout,
             double *grad_alpha, double *grad_rgb);

/* §2.1 step 1: per-pixel depth bounds (min / max depth of the pixel's fragments) */
int wto_depth_bounds(int64_t n, const uint32_t *pixel, const float *z, const float *alpha, int64_t P,
                     double *zlo, double *zhi);
/* depth mapped into the pixel's bounds: (z - lo) / (hi - lo), 0 for an empty range */
int wto_normalize_depth(int64_t n, const uint32_t *pixel, const float *z, int64_t P, const double *zlo,
                        const double *zhi, double *z_out);

#ifdef __cplusplus
}
#endif
#endif
