/*
 * FP64 CPU oracle for Wavelet Transparency (Aizenshtein, Smal & McGuire,
 * "Wavelet Transparency", 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle and is
 * loaded by the test-suite, by the smoke check and by the CPU-baseline leg of
 * the benchmark.  The product path (the CUDA library and its Python binding)
 * never calls it, and it shares no code, header or constant table with that
 * path: every quantity here is re-derived from the paper's equations.
 *
 * Everything is plain, slow and literal:
 *   - coefficients are evaluated over ALL (n,k) pairs, not just the J+1 that
 *     are non-zero;
 *   - the reconstruction evaluates the Haar series term by term;
 *   - the self-term is removed by subtracting the fragment's own projection;
 *   - pixels are processed one at a time after a counting sort by pixel id.
 *
 * Notation (paper §2.2-§2.3): fragment i has opacity alpha_i, normalised depth
 * z_i (x_i in the paper) and colour c_i.  Its absorbance step is
 * a_i = -ln(1 - alpha_i) (the reading that makes a 25%-opaque plane give
 * v = 0.75 behind it, §1.2).  A(z) = sum_i a_i theta(z - z_i) (§2.2).
 * The Haar basis on [0,1) has phi_00 = 1 and
 * psi_{n,k}(x) = 2^{n/2} psi(2^n x - k), psi = +1 on [0,1/2), -1 on [1/2,1).
 * With J levels there are C = 2^J coefficients: index 0 holds chi_00 and
 * index 2^n + k holds X_{n,k} (n = 0..J-1, k = 0..2^n-1).
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes of the repository):
 *   R1 alpha is clamped to [0, 1-2^-20] and z to [0, 1-2^-24] before use.
 *   R2 "points on the subdivision" (§2.3.2) are the bin centres (m+1/2)/C;
 *      the reconstruction is the Haar approximation evaluated at the bin
 *      centres and linearly interpolated between them, held constant outside
 *      [c_0, c_{C-1}].  Without OAF_INTERP_LINEAR it is the plain staircase.
 *   R3 visibility at a fragment excludes the fragment's own step
 *      (OAF_SELF_EXCLUDE): v is the transmittance in front of the interface
 *      (§1.2, §2.2).
 *   R4 "accumulate ... modulated by the visibility function" (step 3, §2.1) is
 *      the normalised weighted resolve: rgb = (R/W)(1 - T) + bg T with
 *      R = sum c_i w_i, W = sum w_i, w_i = alpha_i v(z_i), T = exp(-sum a_i).
 *      Without OAF_RESOLVE_NORMALIZED it is the literal compositing sum of
 *      §2.2: rgb = sum c_i alpha_i v(z_i) + bg T.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "wt_oracle.h"

/* ---- R1: input conditioning ------------------------------------------- */

static double oa_alpha(float alpha)
{
    double a = (double)alpha;
    const double amax = 1.0 - ldexp(1.0, -20);
    if (!(a > 0.0)) return 0.0; /* also maps NaN to 0 (the caller rejects NaN) */
    if (a > amax) return amax;
    return a;
}

static double oa_depth(float z)
{
    double x = (double)z;
    const double zmax = 1.0 - ldexp(1.0, -24);
    if (!(x > 0.0)) return 0.0;
    if (x > zmax) return zmax;
    return x;
}

/* absorbance step of one interface: v drops by the factor (1 - alpha) */
static double oa_step(double alpha_c) { return -log1p(-alpha_c); }

/* ---- §2.3.1: Haar basis and the tent antiderivative -------------------- */

/* psi_{n,k}(x) = 2^{n/2} * (+1 on [0,1/2), -1 on [1/2,1)) in u = 2^n x - k */
static double oa_psi(int n, int k, double x)
{
    double u = ldexp(x, n) - (double)k;
    double s = pow(2.0, 0.5 * n);
    if (u >= 0.0 && u < 0.5) return s;
    if (u >= 0.5 && u < 1.0) return -s;
    return 0.0;
}

/* Psi_{n,k}(x) = 2^{-n/2} * (u on [0,1/2), 1-u on [1/2,1]), 0 elsewhere */
static double oa_Psi(int n, int k, double x)
{
    double u = ldexp(x, n) - (double)k;
    double s = pow(2.0, -0.5 * n);
    if (u >= 0.0 && u < 0.5) return s * u;
    if (u >= 0.5 && u <= 1.0) return s * (1.0 - u);
    return 0.0;
}

double wto_psi(int n, int k, double x) { return oa_psi(n, k, x); }
double wto_Psi(int n, int k, double x) { return oa_Psi(n, k, x); }

/* Closed-form coefficients of a single step a*theta(z - x) (§2.3.1):
 *   chi_00 = a (1 - x),  X_{n,k} = -a Psi_{n,k}(x),  all (n,k). */
static void oa_step_coeffs(double a, double x, int J, double *c)
{
    c[0] += a * (1.0 - x);
    for (int n = 0; n < J; ++n)
        for (int k = 0; k < (1 << n); ++k)
            c[(1 << n) + k] -= a * oa_Psi(n, k, x);
}

/* Haar series evaluated at x: chi_00 phi_00(x) + sum X_{n,k} psi_{n,k}(x) */
static double oa_series(const double *c, int J, double x)
{
    double s = c[0];
    for (int n = 0; n < J; ++n)
        for (int k = 0; k < (1 << n); ++k)
            s += c[(1 << n) + k] * oa_psi(n, k, x);
    return s;
}

/* R2: bin values at the subdivision points c_m = (m + 1/2)/C */
static void oa_bin_values(const double *c, int J, double *Abar)
{
    int C = 1 << J;
    for (int m = 0; m < C; ++m) Abar[m] = oa_series(c, J, (m + 0.5) / C);
}

/* R2: reconstruction at depth x from the bin values */
static double oa_recon(const double *Abar, int J, double x, int linear)
{
    int C = 1 << J;
    int m = (int)floor(x * C);
    if (m > C - 1) m = C - 1;
    if (m < 0) m = 0;
    if (!linear) return Abar[m];
    double pos = x * C - 0.5; /* position in units of bin centres */
    if (pos <= 0.0) return Abar[0];
    if (pos >= C - 1) return Abar[C - 1];
    int lo = (int)floor(pos);
    double t = pos - lo;
    return (1.0 - t) * Abar[lo] + t * Abar[lo + 1];
}

/* ---- grouping fragments by pixel (plain counting sort) ----------------- */

typedef struct {
    int64_t *start; /* P+1 */
    int64_t *idx;   /* n, fragment indices grouped by pixel, input order kept */
} oa_groups;

static int oa_group(int64_t n, const uint32_t *pixel, int64_t P, oa_groups *g)
{
    g->start = (int64_t *)calloc((size_t)P + 1, sizeof(int64_t));
    g->idx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!g->start || !g->idx) return WTO_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)pixel[i] >= P) return WTO_ERR_INPUT;
        g->start[pixel[i] + 1]++;
    }
    for (int64_t p = 0; p < P; ++p) g->start[p + 1] += g->start[p];
    int64_t *fill = (int64_t *)malloc((size_t)(P > 0 ? P : 1) * sizeof(int64_t));
    if (!fill) return WTO_ERR_NOMEM;
    memcpy(fill, g->start, (size_t)P * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) g->idx[fill[pixel[i]]++] = i;
    free(fill);
    return WTO_OK;
}

static void oa_ungroup(oa_groups *g)
{
    free(g->start);
    free(g->idx);
}

static int oa_check_inputs(int64_t n, const float *z, const float *alpha)
{
    for (int64_t i = 0; i < n; ++i)
        if (z[i] != z[i] || alpha[i] != alpha[i]) return WTO_ERR_INPUT;
    return WTO_OK;
}

/* ---- public: coefficient construction ---------------------------------- */

int wto_build(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
              int64_t P, int J, double *coeff)
{
    if (J < 1 || J > 24 || P < 0 || n < 0) return WTO_ERR_ARG;
    if (oa_check_inputs(n, z, alpha)) return WTO_ERR_INPUT;
    int C = 1 << J;
    memset(coeff, 0, (size_t)P * C * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)pixel[i] >= P) return WTO_ERR_INPUT;
        double a = oa_step(oa_alpha(alpha[i]));
        oa_step_coeffs(a, oa_depth(z[i]), J, coeff + (int64_t)pixel[i] * C);
    }
    return WTO_OK;
}

/* Independent second construction: the exact bin averages of A,
 *   Abar_m = C * integral over [m/C,(m+1)/C) of A = sum_{m_i<m} a_i + sum_{m_i=m} a_i (1-f_i),
 * followed by the orthonormal Haar analysis of that piecewise-constant
 * function (chi_00 = mean, X_{n,k} = 2^{n/2}/C (sum first half - sum second half)). */
int wto_build_binned(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
                     int64_t P, int J, double *coeff)
{
    if (J < 1 || J > 24 || P < 0 || n < 0) return WTO_ERR_ARG;
    if (oa_check_inputs(n, z, alpha)) return WTO_ERR_INPUT;
    int C = 1 << J;
    double *Abar = (double *)calloc((size_t)P * C, sizeof(double));
    if (!Abar) return WTO_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)pixel[i] >= P) { free(Abar); return WTO_ERR_INPUT; }
        double a = oa_step(oa_alpha(alpha[i]));
        double x = oa_depth(z[i]);
        double *A = Abar + (int64_t)pixel[i] * C;
        for (int m = 0; m < C; ++m) {
            double lo = (double)m / C, hi = (double)(m + 1) / C;
            /* C * measure of [max(x,lo), hi) */
            double cover = x <= lo ? 1.0 : (x >= hi ? 0.0 : (hi - x) * C);
            A[m] += a * cover;
        }
    }
    for (int64_t p = 0; p < P; ++p) {
        const double *A = Abar + p * C;
        double *c = coeff + p * C;
        double s = 0.0;
        for (int m = 0; m < C; ++m) s += A[m];
        c[0] = s / C;
        for (int n2 = 0; n2 < J; ++n2) {
            int width = C >> n2; /* bins under one psi_{n,k} */
            for (int k = 0; k < (1 << n2); ++k) {
                double d = 0.0;
                for (int m = 0; m < width; ++m)
                    d += (m < width / 2 ? 1.0 : -1.0) * A[k * width + m];
                c[(1 << n2) + k] = pow(2.0, 0.5 * n2) * d / C;
            }
        }
    }
    free(Abar);
    return WTO_OK;
}

void wto_bin_values(const double *coeff, int J, double *Abar) { oa_bin_values(coeff, J, Abar); }

double wto_recon(const double *Abar, int J, double x, int linear) { return oa_recon(Abar, J, x, linear); }

/* ---- per-fragment absorbance in front of each fragment ----------------- */

/* Ahat_i: reconstruction at z_i of the pixel's coefficients; with
 * OAF_SELF_EXCLUDE the fragment's own projection is subtracted first (R3).
 * scratch holds 2C doubles. */
static double oa_frag_absorbance(const double *Abar_pixel, int J, double a, double x,
                                 uint32_t flags, double *scratch)
{
    int C = 1 << J;
    int linear = (flags & OAF_INTERP_LINEAR) != 0;
    double full = oa_recon(Abar_pixel, J, x, linear);
    double self = 0.0;
    if (flags & OAF_SELF_EXCLUDE) {
        double *own = scratch, *ownbar = scratch + C;
        memset(own, 0, (size_t)C * sizeof(double));
        oa_step_coeffs(a, x, J, own);
        oa_bin_values(own, J, ownbar);
        self = oa_recon(ownbar, J, x, linear);
    }
    double r = full - self;
    return r > 0.0 ? r : 0.0;
}

int wto_fragment_absorbance(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
                            int64_t P, int J, uint32_t flags, const double *coeff, double *Ahat)
{
    if (J < 1 || J > 16) return WTO_ERR_ARG;
    if (oa_check_inputs(n, z, alpha)) return WTO_ERR_INPUT;
    int C = 1 << J;
    double *Abar = (double *)malloc((size_t)3 * C * sizeof(double));
    if (!Abar) return WTO_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)pixel[i] >= P) { free(Abar); return WTO_ERR_INPUT; }
        oa_bin_values(coeff + (int64_t)pixel[i] * C, J, Abar);
        double a = oa_step(oa_alpha(alpha[i]));
        Ahat[i] = oa_frag_absorbance(Abar, J, a, oa_depth(z[i]), flags, Abar + C);
    }
    free(Abar);
    return WTO_OK;
}

/* Visibility at arbitrary depths: Ahat(z) of the full reconstruction. */
int wto_absorbance_at(int64_t q, const uint32_t *pixel, const float *z, int64_t P, int J,
                      uint32_t flags, const double *coeff, double *Aout)
{
    if (J < 1 || J > 16) return WTO_ERR_ARG;
    int C = 1 << J;
    double *Abar = (double *)malloc((size_t)C * sizeof(double));
    if (!Abar) return WTO_ERR_NOMEM;
    for (int64_t i = 0; i < q; ++i) {
        if ((int64_t)pixel[i] >= P || z[i] != z[i]) { free(Abar); return WTO_ERR_INPUT; }
        oa_bin_values(coeff + (int64_t)pixel[i] * C, J, Abar);
        Aout[i] = oa_recon(Abar, J, oa_depth(z[i]), (flags & OAF_INTERP_LINEAR) != 0);
    }
    free(Abar);
    return WTO_OK;
}

/* ---- steps 3-4 (§2.1): resolve and composite --------------------------- */

static double oa_bg(const double *bg, const double *bg_img, int64_t p, int ch)
{
    return bg_img ? bg_img[p * 3 + ch] : bg[ch];
}

/* accum[p] = {R', G', B', W', S, Amin}: R', G', B', W' are the weighted sums
 * multiplied by exp(Amin) (Amin = smallest Ahat in the pixel), which leaves
 * R/W unchanged and keeps the largest weight away from underflow. */
int wto_resolve(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
                const float *r, const float *g, const float *b, int64_t P, int J, uint32_t flags,
                const double *coeff, const double *bg, const double *bg_img, double *accum, double *out)
{
    if (J < 1 || J > 16 || P < 0 || n < 0) return WTO_ERR_ARG;
    if (oa_check_inputs(n, z, alpha)) return WTO_ERR_INPUT;
    int C = 1 << J;
    oa_groups grp;
    int st = oa_group(n, pixel, P, &grp);
    if (st) { oa_ungroup(&grp); return st; }
    double *Abar = (double *)malloc((size_t)3 * C * sizeof(double));
    double *Ah = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!Abar || !Ah) { free(Abar); free(Ah); oa_ungroup(&grp); return WTO_ERR_NOMEM; }
    const float *col[3] = {r, g, b};
    for (int64_t p = 0; p < P; ++p) {
        oa_bin_values(coeff + p * C, J, Abar);
        double Amin = INFINITY, S = 0.0;
        for (int64_t q = grp.start[p]; q < grp.start[p + 1]; ++q) {
            int64_t i = grp.idx[q];
            double a = oa_step(oa_alpha(alpha[i]));
            Ah[q] = oa_frag_absorbance(Abar, J, a, oa_depth(z[i]), flags, Abar + C);
            if (Ah[q] < Amin) Amin = Ah[q];
            S += a;
        }
        if (!(Amin < INFINITY)) Amin = 0.0;
        double R[3] = {0, 0, 0}, W = 0.0;
        for (int64_t q = grp.start[p]; q < grp.start[p + 1]; ++q) {
            int64_t i = grp.idx[q];
            double w = oa_alpha(alpha[i]) * exp(-(Ah[q] - Amin));
            W += w;
            for (int ch = 0; ch < 3; ++ch) R[ch] += (double)col[ch][i] * w;
        }
        double T = exp(-S);
        if (accum) {
            double *A = accum + p * 6;
            A[0] = R[0]; A[1] = R[1]; A[2] = R[2]; A[3] = W; A[4] = S; A[5] = Amin;
        }
        if (out) {
            double *o = out + p * 4;
            for (int ch = 0; ch < 3; ++ch) {
                double bgc = oa_bg(bg, bg_img, p, ch);
                if (flags & OAF_RESOLVE_NORMALIZED)
                    o[ch] = W > 0.0 ? (R[ch] / W) * (1.0 - T) + bgc * T : bgc;
                else
                    o[ch] = R[ch] * exp(-Amin) + bgc * T;
            }
            o[3] = 1.0 - T;
        }
    }
    free(Abar);
    free(Ah);
    oa_ungroup(&grp);
    return WTO_OK;
}

/* ---- exact A-buffer: sort each pixel by depth and composite ------------ */

static const float *oa_sort_z;
static int oa_cmp_depth(const void *pa, const void *pb)
{
    int64_t ia = *(const int64_t *)pa, ib = *(const int64_t *)pb;
    double za = oa_depth(oa_sort_z[ia]), zb = oa_depth(oa_sort_z[ib]);
    if (za < zb) return -1;
    if (za > zb) return 1;
    return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

int wto_abuffer(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
                const float *r, const float *g, const float *b, int64_t P,
                const double *bg, const double *bg_img, double *out)
{
    if (P < 0 || n < 0) return WTO_ERR_ARG;
    if (oa_check_inputs(n, z, alpha)) return WTO_ERR_INPUT;
    oa_groups grp;
    int st = oa_group(n, pixel, P, &grp);
    if (st) { oa_ungroup(&grp); return st; }
    const float *col[3] = {r, g, b};
    oa_sort_z = z;
    for (int64_t p = 0; p < P; ++p) {
        int64_t s = grp.start[p], e = grp.start[p + 1];
        qsort(grp.idx + s, (size_t)(e - s), sizeof(int64_t), oa_cmp_depth);
        double T = 1.0, acc[3] = {0, 0, 0};
        for (int64_t q = s; q < e; ++q) {
            int64_t i = grp.idx[q];
            double al = oa_alpha(alpha[i]);
            for (int ch = 0; ch < 3; ++ch) acc[ch] += T * al * (double)col[ch][i];
            T *= (1.0 - al);
        }
        double *o = out + p * 4;
        for (int ch = 0; ch < 3; ++ch) o[ch] = acc[ch] + T * oa_bg(bg, bg_img, p, ch);
        o[3] = 1.0 - T;
    }
    oa_ungroup(&grp);
    return WTO_OK;
}

/* ---- adjoint of build + resolve + composite ---------------------------- */

/* Brute-force analytic gradient of L with dL/dout = gout (P x 4) with
 * respect to every fragment's alpha and colour.  Per pixel with k fragments:
 *   dL/dc_i   = gout_rgb (1-T)/W * w_i                       (normalised)
 *   dL/dw_i   = beta_i = sum_ch gout_ch (1-T)/W (c_i,ch - R_ch/W)
 *   dL/dAhat_i = gamma_i = -beta_i w_i
 *   dAhat_i/da_j = K(z_i, z_j) for j != i (the reconstruction at z_i of a unit
 *                  step at z_j; the self term is absent under R3) and
 *                  K(z_i, z_i) for j == i when the self term is kept
 *   dL/da_j   = sum_i gamma_i dAhat_i/da_j + dL/dT * (-T)
 *   dL/dalpha_j = beta_j exp(-Ahat_j) + dL/da_j / (1 - alpha_j)   (0 when clamped)
 * K is evaluated through the closed-form coefficients of a unit step, so this
 * is O(k^2) per pixel and independent of any fast summation. */
int wto_grad(int64_t n, const uint32_t *pixel, const float *z, const float *alpha,
             const float *r, const float *g, const float *b, int64_t P, int J, uint32_t flags,
             const double *bg, const double *bg_img, const double *gout,
             double *grad_alpha, double *grad_rgb)
{
    if (J < 1 || J > 12 || P < 0 || n < 0) return WTO_ERR_ARG;
    if (oa_check_inputs(n, z, alpha)) return WTO_ERR_INPUT;
    int C = 1 << J;
    int linear = (flags & OAF_INTERP_LINEAR) != 0;
    double *coeff = (double *)malloc((size_t)P * C * sizeof(double));
    if (!coeff) return WTO_ERR_NOMEM;
    int st = wto_build(n, pixel, z, alpha, P, J, coeff);
    if (st) { free(coeff); return st; }
    oa_groups grp;
    st = oa_group(n, pixel, P, &grp);
    if (st) { free(coeff); oa_ungroup(&grp); return st; }
    double *Abar = (double *)malloc((size_t)3 * C * sizeof(double));
    double *unit = (double *)malloc((size_t)C * sizeof(double));
    /* per-fragment scratch, indexed by position q in the grouped order */
    double *Ah = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *w = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *gam = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *bet = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *unitbar = (double *)malloc((size_t)(n > 0 ? n : 1) * C * sizeof(double));
    if (!Abar || !unit || !Ah || !w || !gam || !bet || !unitbar) {
        st = WTO_ERR_NOMEM;
        goto done;
    }
    const float *col[3] = {r, g, b};
    for (int64_t p = 0; p < P; ++p) {
        int64_t s = grp.start[p], e = grp.start[p + 1];
        if (e == s) continue;
        oa_bin_values(coeff + p * C, J, Abar);
        double Amin = INFINITY, S = 0.0;
        for (int64_t q = s; q < e; ++q) {
            int64_t i = grp.idx[q];
            double a = oa_step(oa_alpha(alpha[i]));
            Ah[q] = oa_frag_absorbance(Abar, J, a, oa_depth(z[i]), flags, Abar + C);
            if (Ah[q] < Amin) Amin = Ah[q];
            S += a;
            /* bin values of a unit step at z_i, for K(., z_i) */
            memset(unit, 0, (size_t)C * sizeof(double));
            oa_step_coeffs(1.0, oa_depth(z[i]), J, unit);
            oa_bin_values(unit, J, unitbar + (q - s) * C);
        }
        double R[3] = {0, 0, 0}, W = 0.0;
        for (int64_t q = s; q < e; ++q) {
            int64_t i = grp.idx[q];
            w[q] = oa_alpha(alpha[i]) * exp(-(Ah[q] - Amin));
            W += w[q];
            for (int ch = 0; ch < 3; ++ch) R[ch] += (double)col[ch][i] * w[q];
        }
        double T = exp(-S);
        const double *go = gout + p * 4;
        double dT = -go[3]; /* out.a = 1 - T */
        double u[3];
        for (int ch = 0; ch < 3; ++ch) {
            double bgc = oa_bg(bg, bg_img, p, ch);
            if (flags & OAF_RESOLVE_NORMALIZED) {
                if (W > 0.0) {
                    u[ch] = go[ch] * (1.0 - T) / W;
                    dT += go[ch] * (bgc - R[ch] / W);
                } else {
                    u[ch] = 0.0;
                }
            } else {
                u[ch] = go[ch] * exp(-Amin); /* d out / d R' */
                dT += go[ch] * bgc;
            }
        }
        for (int64_t q = s; q < e; ++q) {
            int64_t i = grp.idx[q];
            double bq = 0.0;
            for (int ch = 0; ch < 3; ++ch) {
                double centre = (flags & OAF_RESOLVE_NORMALIZED) && W > 0.0 ? R[ch] / W : 0.0;
                bq += u[ch] * ((double)col[ch][i] - centre);
                grad_rgb[i * 3 + ch] = u[ch] * w[q];
            }
            bet[q] = bq;
            gam[q] = -bq * w[q];
        }
        for (int64_t qj = s; qj < e; ++qj) {
            int64_t j = grp.idx[qj];
            double da = -T * dT;
            for (int64_t qi = s; qi < e; ++qi) {
                if (qi == qj && (flags & OAF_SELF_EXCLUDE)) continue;
                int64_t i = grp.idx[qi];
                da += gam[qi] * oa_recon(unitbar + (qj - s) * C, J, oa_depth(z[i]), linear);
            }
            /* the clamp of R1 is flat outside (0, 1-2^-20) */
            double al = (double)alpha[j];
            const double amax = 1.0 - ldexp(1.0, -20);
            if (al > 0.0 && al < amax)
                grad_alpha[j] = bet[qj] * exp(-(Ah[qj] - Amin)) + da / (1.0 - al);
            else
                grad_alpha[j] = 0.0;
        }
    }
done:
    free(Abar); free(unit); free(Ah); free(w); free(gam); free(bet); free(unitbar);
    free(coeff);
    oa_ungroup(&grp);
    return st;
}

/*
 * §2.1 step 1: the tight per-pixel depth bounds of the transparent surfaces,
 * taken literally as the smallest and largest depth of the pixel's fragments
 * (fragments with a NaN depth or opacity, or a pixel id outside the image,
 * are left out); +inf / -inf for a pixel without fragments.
 */
int wto_depth_bounds(int64_t n, const uint32_t *pixel, const float *z, const float *alpha, int64_t P,
                     double *zlo, double *zhi) {
    if (n < 0 || P < 1 || !zlo || !zhi || (n > 0 && (!pixel || !z || !alpha))) return WTO_ERR_ARG;
    for (int64_t p = 0; p < P; ++p) {
        zlo[p] = INFINITY;
        zhi[p] = -INFINITY;
    }
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)pixel[i] >= P || isnan(z[i]) || isnan(alpha[i])) continue;
        double d = (double)z[i];
        if (d < zlo[pixel[i]]) zlo[pixel[i]] = d;
        if (d > zhi[pixel[i]]) zhi[pixel[i]] = d;
    }
    return WTO_OK;
}

/*
 * Depth normalised into the pixel's bounds: (z - lo) / (hi - lo), so that the
 * nearest fragment sits at 0 and the farthest at 1; 0 when the pixel's range
 * is empty or not finite; NaN for a bad pixel id or a NaN depth.
 */
int wto_normalize_depth(int64_t n, const uint32_t *pixel, const float *z, int64_t P, const double *zlo,
                        const double *zhi, double *z_out) {
    if (n < 0 || P < 1 || !zlo || !zhi || (n > 0 && (!pixel || !z || !z_out))) return WTO_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)pixel[i] >= P || isnan(z[i])) {
            z_out[i] = NAN;
            continue;
        }
        double lo = zlo[pixel[i]], range = zhi[pixel[i]] - lo;
        z_out[i] = (range > 0.0 && isfinite(range)) ? ((double)z[i] - lo) / range : 0.0;
    }
    return WTO_OK;
}
