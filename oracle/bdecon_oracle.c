/*
 * bdecon_oracle.c -- plain, slow FP64 CPU oracle of the posterior-sampling
 * sweep of Bayesian deconvolution (Hendrix, Brown, Flanagan, Shepherd,
 * Saurabh, Presse: "Re-thinking Richardson-Lucy without Iteration Cutoffs:
 * Physically Motivated Bayesian Deconvolution", arXiv 2411.00991).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load or call this file.  It shares
 * no code, header, table or constant with the CUDA library; every quantity
 * is written out from its definition in the paper, single-threaded, in
 * double precision, without blocking, fusion or reordering beyond what the
 * definitions state.
 *
 * Model (Methods):
 *   Eq. 1-2  mu_n = sum_m K[n-m] rho_m, K the pixel-integrated PSF (true
 *            convolution of the object padded by the PSF radius, Fig. 5b).
 *   Eq. 3-6  l_n(mu) = log sum_{phi>=0} Normal(w_n; G_n phi + o_n, var_n)
 *                                  * Poisson(phi; mu_n).
 *   Eq. 7-8  Dirichlet prior on |F(rho)| / sum |F(rho)| with hyperparameter
 *            |OTF| / sum |OTF|, taken per P x P patch aligned with the
 *            sub-lattice (the paper's locality argument, "Parallelization
 *            Technique"), all frequencies included.
 *   Eq. 9    log posterior = sum_n l_n(mu_n) + sum_patches log prior.
 * Sampler (Results, Methods "Parallelization Technique", Fig. 5d): one
 * single-site Metropolis-Hastings step per object pixel per sweep,
 * systematic scan over sub-lattice classes, log-space Gaussian random walk
 * proposals keyed by Philox4x32-10 on (pixel, sweep, chain).
 * Optional burn-in adaptation of the proposal scale (not in the paper, which
 * leaves the proposal unstated): each pixel m has its own scale s_m, starting
 * at step; during burn-in sweeps only, after each update of m,
 * s_m <- s_m * exp(g_t (1 - a*)) if accepted, s_m * exp(-g_t a*) if not,
 * clamped to [1e-4, 4], with a* the problem's target acceptance rate and the
 * gain g_t = 0.5 / sqrt(t) of sweep t shrinking over burn-in, so that log s_m
 * settles where the pixel's acceptance rate is a*; after burn-in the scales
 * stay fixed and the chain is an ordinary Metropolis-Hastings chain.
 * Optional photon-count augmentation (the paper's completed likelihood,
 * Eq. 5): the photon counts phi_n are kept as variables and each sweep first
 * draws every phi_n from p(phi | w_n, mu_n), then updates rho against the
 * Poisson likelihood sum_n phi_n log mu_n - mu_n; the rho-marginal of the
 * augmented chain's target is Eq. 9.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#ifndef M_LN2
#define M_LN2 0.69314718055994530942
#endif

typedef struct {
    int H, W;            /* camera frame size                                  */
    int L;               /* PSF side (odd)                                     */
    int S;               /* sub-lattice stride = prior patch side (>= L)      */
    const double* w;     /* H*W ADU                                            */
    const double* gain;  /* H*W ADU per photon                                 */
    const double* offset;/* H*W ADU                                            */
    const double* var;   /* H*W ADU^2 (read-noise variance)                    */
    const double* psf;   /* L*L, non-negative, normalised here                 */
    uint64_t seed;
    int chain;
    double step;         /* sd of the log-space random walk                    */
    int burn_in;         /* sweeps t <= burn_in are not averaged               */
    int refresh_every;   /* recompute mu and spectra every this many sweeps    */
    double adapt_target; /* > 0: adapt the per-pixel proposal scale during
                            burn-in toward this acceptance rate               */
    int aug;             /* photon-count augmented sampler                     */
    int sub;             /* object lattice sub cells per camera pixel side (0/1:
                            the camera grid)                                  */
} or_problem;

#define OR_ADAPT_GAIN 0.5
#define OR_STEP_MIN 1e-4
#define OR_STEP_MAX 4.0

/* ------------------------------------------------------------------ RNG --
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * published multipliers and Weyl key increments.                           */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform on (0,1) from the top 23 bits: ((x >> 9) + 1/2) / 2^23.  The
 * numerator is an odd multiple of 1/2 below 2^23, so the value has at most
 * 24 significant bits and is exact in float as well as double.            */
double or_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) / 8388608.0;
}

/* The three numbers one proposal uses: a standard normal z (Box-Muller on
 * the first two uniforms) and the acceptance uniform u (third output).
 * Counter = (pixel index m, sweep t, chain, 0), key = seed split lo/hi.    */
void or_draw(uint64_t seed, uint32_t m, uint32_t t, uint32_t chain, double* z, double* u)
{
    uint32_t ctr[4] = {m, t, chain, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    double u0 = or_uniform(x[0]), u1 = or_uniform(x[1]);
    *z = sqrt(-2.0 * log(u0)) * cos(2.0 * M_PI * u1);
    *u = or_uniform(x[2]);
}

/* ------------------------------------------------------- likelihood ----- */
static double* g_lfact = NULL;
static long g_lfact_n = 0;

/* log(n!) from the C library's lgamma, memoised. */
static double lfact(long n)
{
    if (n >= g_lfact_n) {
        long nn = g_lfact_n ? g_lfact_n : 1024;
        while (nn <= n) nn *= 2;
        double* t = (double*)realloc(g_lfact, (size_t)nn * sizeof(double));
        if (!t) abort();
        for (long k = g_lfact_n; k < nn; ++k) t[k] = lgamma((double)k + 1.0);
        g_lfact = t;
        g_lfact_n = nn;
    }
    return g_lfact[n];
}

/* log of the phi-th summand of Eq. 6 without the phi-free constants:
 * -(w - G phi - o)^2 / (2 var) + phi log mu - log phi!                   */
static double summand(double w, double o, double G, double var, double lmu, long phi)
{
    double r = w - G * (double)phi - o;
    return -r * r / (2.0 * var) + (double)phi * lmu - lfact(phi);
}

/* Marginal log-likelihood of one pixel, Eq. 6 (the photon count phi summed
 * out): l(mu) = log sum_phi Normal(w; G phi + o, var) Poisson(phi; mu).
 * The summand is log-concave in phi, so the sum is taken outward from its
 * integer mode (found by hill climbing) until terms fall below 2^-60 of the
 * largest, in log-sum-exp form.  Requires mu > 0.                        */
double or_loglik(double w, double o, double G, double var, double mu)
{
    const double lmu = log(mu);
    double c = (w - o) / G;
    long phi = c > 0.0 ? (long)floor(c) : 0;
    double tm = summand(w, o, G, var, lmu, phi);
    for (;;) {
        double tu = summand(w, o, G, var, lmu, phi + 1);
        if (tu > tm) { ++phi; tm = tu; } else break;
    }
    for (;;) {
        if (phi == 0) break;
        double td = summand(w, o, G, var, lmu, phi - 1);
        if (td > tm) { --phi; tm = td; } else break;
    }
    const double cut = tm - 60.0 * M_LN2;
    double s = 1.0;
    for (long k = phi + 1;; ++k) {
        double t = summand(w, o, G, var, lmu, k);
        if (t < cut) break;
        s += exp(t - tm);
    }
    for (long k = phi - 1; k >= 0; --k) {
        double t = summand(w, o, G, var, lmu, k);
        if (t < cut) break;
        s += exp(t - tm);
    }
    return -0.5 * log(2.0 * M_PI * var) - mu + tm + log(s);
}

/* Draw a photon count from p(phi | w, mu) ∝ Normal(w; G phi + o, var)
 * Poisson(phi; mu) (the summands of Eq. 6, normalised) by inverse CDF: the
 * smallest phi whose cumulative weight, summed upward from the lowest
 * retained count, reaches u times the total.  Counts whose summand falls
 * below 2^-60 of the largest are dropped, as in or_loglik.               */
long or_sample_phi(double w, double o, double G, double var, double mu, double u)
{
    const double lmu = log(mu);
    double c = (w - o) / G;
    long phi = c > 0.0 ? (long)floor(c) : 0;
    double tm = summand(w, o, G, var, lmu, phi);
    for (;;) {
        double tu = summand(w, o, G, var, lmu, phi + 1);
        if (tu > tm) { ++phi; tm = tu; } else break;
    }
    for (;;) {
        if (phi == 0) break;
        double td = summand(w, o, G, var, lmu, phi - 1);
        if (td > tm) { --phi; tm = td; } else break;
    }
    const double cut = tm - 60.0 * M_LN2;
    long lo = phi, hi = phi;
    while (lo > 0 && summand(w, o, G, var, lmu, lo - 1) >= cut) --lo;
    while (summand(w, o, G, var, lmu, hi + 1) >= cut) ++hi;
    double Z = 0.0;
    for (long k = lo; k <= hi; ++k) Z += exp(summand(w, o, G, var, lmu, k) - tm);
    double acc = 0.0;
    for (long k = lo; k <= hi; ++k) {
        acc += exp(summand(w, o, G, var, lmu, k) - tm);
        if (acc >= u * Z) return k;
    }
    return hi;
}

/* The uniform of the photon-count draw of camera pixel n at sweep t: first
 * Philox output of counter (n, t, chain, 1).                              */
double or_phi_uniform(uint64_t seed, uint32_t n, uint32_t t, uint32_t chain)
{
    uint32_t ctr[4] = {n, t, chain, 1u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    or_philox4x32_10(ctr, key, x);
    return or_uniform(x[0]);
}

/* log of one pixel's completed likelihood (Eq. 5):
 * log Normal(w; G phi + o, var) + log Poisson(phi; mu).                   */
double or_logjoint_pixel(double w, double o, double G, double var, double mu, long phi)
{
    return -0.5 * log(2.0 * M_PI * var) + summand(w, o, G, var, log(mu), phi) - mu;
}

/* ------------------------------------------------------- convolution ---- */
/* Eq. 1-2: expected photons on camera pixel (a, b) from the padded object
 * rho of size (H+2R) x (W+2R): mu[a][b] = sum_{p,q} K[p][q] rho[a+2R-p][b+2R-q]
 * (a true convolution; K already integrated over the pixel area).        */
void or_convolve(const double* rho, int H, int W, const double* K, int L, double* mu)
{
    const int R = L / 2, Wo = W + 2 * R;
    for (int a = 0; a < H; ++a)
        for (int b = 0; b < W; ++b) {
            double s = 0.0;
            for (int p = 0; p < L; ++p)
                for (int q = 0; q < L; ++q)
                    s += K[p * L + q] * rho[(a + 2 * R - p) * Wo + (b + 2 * R - q)];
            mu[a * W + b] = s;
        }
}

/* ------------------------------------------------------------- prior ---- */
/* 2-D DFT of a ph x pw patch by its definition:
 * X[k][l] = sum_{u,v} x[u][v] exp(-2 pi i (k u / ph + l v / pw)).          */
void or_patch_dft(const double* x, int ld, int ph, int pw, double* re, double* im)
{
    for (int k = 0; k < ph; ++k)
        for (int l = 0; l < pw; ++l) {
            double sr = 0.0, si = 0.0;
            for (int u = 0; u < ph; ++u)
                for (int v = 0; v < pw; ++v) {
                    double th = 2.0 * M_PI * ((double)k * u / ph + (double)l * v / pw);
                    sr += x[u * ld + v] * cos(th);
                    si -= x[u * ld + v] * sin(th);
                }
            re[k * pw + l] = sr;
            im[k * pw + l] = si;
        }
}

/* Dirichlet hyperparameter of Eq. 8 for a ph x pw patch: the modulus of the
 * OTF (DFT of the normalised PSF, wrapped periodically onto the patch with
 * its centre at the origin), divided by its sum over all frequencies.    */
void or_alpha(const double* K, int L, int ph, int pw, double* alpha)
{
    const int R = L / 2, n = ph * pw;
    double* kw = (double*)calloc((size_t)n, sizeof(double));
    double* re = (double*)malloc((size_t)n * sizeof(double));
    double* im = (double*)malloc((size_t)n * sizeof(double));
    for (int p = 0; p < L; ++p)
        for (int q = 0; q < L; ++q) {
            int x = ((p - R) % ph + ph) % ph, y = ((q - R) % pw + pw) % pw;
            kw[x * pw + y] += K[p * L + q];
        }
    or_patch_dft(kw, pw, ph, pw, re, im);
    double tot = 0.0;
    for (int k = 0; k < n; ++k) {
        alpha[k] = hypot(re[k], im[k]);
        tot += alpha[k];
    }
    for (int k = 0; k < n; ++k) alpha[k] /= tot;
    free(kw); free(re); free(im);
}

/* log Dirichlet(|X| / sum|X|; alpha) without the constant log B(alpha), for
 * alpha summing to one (Eq. 7-8):
 *   sum_k (alpha_k - 1) log|X_k| + (n - 1) log sum_k |X_k|.               */
double or_log_prior_patch(const double* re, const double* im, const double* alpha, int n)
{
    double sa = 0.0, sm = 0.0;
    for (int k = 0; k < n; ++k) {
        double m = hypot(re[k], im[k]);
        sm += m;
        sa += (alpha[k] - 1.0) * log(m);
    }
    return sa + (double)(n - 1) * log(sm);
}

/* -------------------------------------------------- problem helpers ----- */
static void normalised_psf(const or_problem* P, double* K)
{
    double s = 0.0;
    for (int k = 0; k < P->L * P->L; ++k) s += P->psf[k];
    for (int k = 0; k < P->L * P->L; ++k) K[k] = P->psf[k] / s;
}

static int patch_len(int origin, int S, int n) { return (origin + S <= n) ? S : n - origin; }

/* Object lattice f times finer than the camera (f = sub; the paper's
 * Nyquist lattice, Methods after Eq. 6): camera pixel (a, b) integrates the
 * f x f lattice cells of its area (the A_n integral of Eq. 1), so
 *   mu[a][b] = sum_{p,q} Ke[p][q] rho[f a + Le-1-p][f b + Le-1-q]
 * with the effective kernel Ke = K (x) box_f of side Le = L + f - 1, K the
 * PSF on the lattice.  The object is (f H + L - 1) x (f W + L - 1).  f = 1
 * is the camera grid padded by R (Ke = K).                                 */
static int sub_of(const or_problem* P) { return P->sub > 1 ? P->sub : 1; }

static void obj_dims(const or_problem* P, int* Ho, int* Wo)
{
    const int f = sub_of(P);
    *Ho = f * P->H + P->L - 1;
    *Wo = f * P->W + P->L - 1;
}

void or_eff_kernel(const double* K, int L, int f, double* Ke)
{
    const int Le = L + f - 1;
    for (int p = 0; p < Le; ++p)
        for (int q = 0; q < Le; ++q) {
            double s = 0.0;
            for (int u = 0; u < f; ++u)
                for (int v = 0; v < f; ++v) {
                    const int pp = p - u, qq = q - v;
                    if (pp >= 0 && pp < L && qq >= 0 && qq < L) s += K[pp * L + qq];
                }
            Ke[p * Le + q] = s;
        }
}

/* Eq. 1 on the lattice: the expected image of the camera pixels. */
void or_expected(const double* rho, int H, int W, const double* Ke, int Le, int f, double* mu)
{
    const int Wo = f * (W - 1) + Le;
    for (int a = 0; a < H; ++a)
        for (int b = 0; b < W; ++b) {
            double s = 0.0;
            for (int p = 0; p < Le; ++p)
                for (int q = 0; q < Le; ++q)
                    s += Ke[p * Le + q] * rho[(f * a + Le - 1 - p) * Wo + (f * b + Le - 1 - q)];
            mu[a * W + b] = s;
        }
}

/* Sum of the patch log priors of Eq. 8 over all patches of rho. */
static double log_prior_all(const or_problem* P, const double* K, const double* rho)
{
    int Ho, Wo;
    obj_dims(P, &Ho, &Wo);
    const int S = P->S;
    double* re = (double*)malloc((size_t)S * S * sizeof(double));
    double* im = (double*)malloc((size_t)S * S * sizeof(double));
    double* al = (double*)malloc((size_t)S * S * sizeof(double));
    double tot = 0.0;
    for (int i0 = 0; i0 < Ho; i0 += S)
        for (int j0 = 0; j0 < Wo; j0 += S) {
            int ph = patch_len(i0, S, Ho), pw = patch_len(j0, S, Wo);
            or_patch_dft(rho + i0 * Wo + j0, Wo, ph, pw, re, im);
            or_alpha(K, P->L, ph, pw, al);
            tot += or_log_prior_patch(re, im, al, ph * pw);
        }
    free(re); free(im); free(al);
    return tot;
}

/* Likelihood part of Eq. 9: Eq. 6 summed over the camera pixels at the
 * expected image of rho (Eq. 1-2).                                        */
double or_log_likelihood(const or_problem* P, const double* rho)
{
    const int H = P->H, W = P->W, L = P->L, f = sub_of(P), Le = L + f - 1;
    double* K = (double*)malloc((size_t)L * L * sizeof(double));
    double* Ke = (double*)malloc((size_t)Le * Le * sizeof(double));
    double* mu = (double*)malloc((size_t)H * W * sizeof(double));
    normalised_psf(P, K);
    or_eff_kernel(K, L, f, Ke);
    or_expected(rho, H, W, Ke, Le, f, mu);
    double ll = 0.0;
    for (int n = 0; n < H * W; ++n)
        ll += or_loglik(P->w[n], P->offset[n], P->gain[n], P->var[n], mu[n]);
    free(K); free(Ke); free(mu);
    return ll;
}

/* Eq. 9: log posterior (up to the constant log B(alpha) terms) of rho. */
double or_log_posterior(const or_problem* P, const double* rho)
{
    double* K = (double*)malloc((size_t)P->L * P->L * sizeof(double));
    normalised_psf(P, K);
    double lp = log_prior_all(P, K, rho);
    free(K);
    return or_log_likelihood(P, rho) + lp;
}

/* Log of the augmented joint density p(w, phi, rho) (prior without B(alpha)):
 * sum_n log Normal(w_n; G phi_n + o_n, var_n) Poisson(phi_n; mu_n) + the
 * patch log priors.                                                         */
double or_log_joint(const or_problem* P, const double* rho, const double* phi)
{
    const int H = P->H, W = P->W, L = P->L, f = sub_of(P), Le = L + f - 1;
    double* K = (double*)malloc((size_t)L * L * sizeof(double));
    double* Ke = (double*)malloc((size_t)Le * Le * sizeof(double));
    double* mu = (double*)malloc((size_t)H * W * sizeof(double));
    normalised_psf(P, K);
    or_eff_kernel(K, L, f, Ke);
    or_expected(rho, H, W, Ke, Le, f, mu);
    double ll = 0.0;
    for (int n = 0; n < H * W; ++n)
        ll += or_logjoint_pixel(P->w[n], P->offset[n], P->gain[n], P->var[n], mu[n], (long)phi[n]);
    double lp = log_prior_all(P, K, rho);
    free(K); free(Ke); free(mu);
    return ll + lp;
}

/* Initial object: rho0_m = b0 exp(z_m / 10), b0 = max(0.1, mean_n (w_n - o_n) / G_n) / f^2,
 * z_m the Box-Muller normal of counter (m, 0, chain, 0) (sweep 0 is never a
 * sampling sweep).  The jitter keeps every patch spectrum coefficient away
 * from zero, where the Dirichlet density of Eq. 7 is singular.           */
void or_init(const or_problem* P, double* rho)
{
    int Ho, Wo;
    obj_dims(P, &Ho, &Wo);
    const int f = sub_of(P);
    double mc = 0.0;
    for (int n = 0; n < P->H * P->W; ++n) mc += (P->w[n] - P->offset[n]) / P->gain[n];
    mc /= (double)(P->H * P->W);
    /* a camera pixel collects f^2 lattice cells */
    double b0 = (mc > 0.1 ? mc : 0.1) / (double)(f * f);
    for (int m = 0; m < Ho * Wo; ++m) {
        double z, u;
        or_draw(P->seed, (uint32_t)m, 0u, (uint32_t)P->chain, &z, &u);
        rho[m] = b0 * exp(0.1 * z);
    }
}

/* ------------------------------------------------------------ sampler --- */
typedef struct {
    const or_problem* P;
    int R, Ho, Wo, S, npi, npj;
    int f, Le, Lc;    /* lattice cells per camera pixel side, effective
                         kernel side, camera window side                   */
    double* K;        /* normalised PSF                                   */
    double* Ke;       /* effective kernel K (x) box_f, Le*Le              */
    double* rho;      /* object, Ho*Wo                                    */
    double* mu;       /* expected image, H*W (kept incrementally)         */
    double** sre;     /* per patch spectrum (ph*pw)                       */
    double** sim;
    double** alpha;   /* per patch hyperparameter                         */
    double* tre;      /* scratch ph*pw                                    */
    double* tim;
    double* steps;    /* per-pixel proposal scale, Ho*Wo                  */
    double* phi;      /* photon counts, H*W (augmented sampler)           */
} chain_state;

static void cs_refresh(chain_state* c)
{
    const or_problem* P = c->P;
    or_expected(c->rho, P->H, P->W, c->Ke, c->Le, c->f, c->mu);
    for (int pi = 0; pi < c->npi; ++pi)
        for (int pj = 0; pj < c->npj; ++pj) {
            int i0 = pi * c->S, j0 = pj * c->S;
            int ph = patch_len(i0, c->S, c->Ho), pw = patch_len(j0, c->S, c->Wo);
            int p = pi * c->npj + pj;
            or_patch_dft(c->rho + i0 * c->Wo + j0, c->Wo, ph, pw, c->sre[p], c->sim[p]);
        }
}

static void cs_open(chain_state* c, const or_problem* P, const double* rho_in)
{
    c->P = P;
    c->R = P->L / 2;
    obj_dims(P, &c->Ho, &c->Wo);
    c->f = sub_of(P);
    c->Le = P->L + c->f - 1;
    c->Lc = (c->Le - 1) / c->f + 1;
    c->S = P->S;
    c->npi = (c->Ho + c->S - 1) / c->S;
    c->npj = (c->Wo + c->S - 1) / c->S;
    c->K = (double*)malloc((size_t)P->L * P->L * sizeof(double));
    normalised_psf(P, c->K);
    c->Ke = (double*)malloc((size_t)c->Le * c->Le * sizeof(double));
    or_eff_kernel(c->K, P->L, c->f, c->Ke);
    c->rho = (double*)malloc((size_t)c->Ho * c->Wo * sizeof(double));
    if (rho_in) memcpy(c->rho, rho_in, (size_t)c->Ho * c->Wo * sizeof(double));
    else or_init(P, c->rho);
    c->mu = (double*)malloc((size_t)P->H * P->W * sizeof(double));
    int np = c->npi * c->npj;
    c->sre = (double**)malloc((size_t)np * sizeof(double*));
    c->sim = (double**)malloc((size_t)np * sizeof(double*));
    c->alpha = (double**)malloc((size_t)np * sizeof(double*));
    for (int pi = 0; pi < c->npi; ++pi)
        for (int pj = 0; pj < c->npj; ++pj) {
            int ph = patch_len(pi * c->S, c->S, c->Ho), pw = patch_len(pj * c->S, c->S, c->Wo);
            int p = pi * c->npj + pj;
            c->sre[p] = (double*)malloc((size_t)ph * pw * sizeof(double));
            c->sim[p] = (double*)malloc((size_t)ph * pw * sizeof(double));
            c->alpha[p] = (double*)malloc((size_t)ph * pw * sizeof(double));
            or_alpha(c->K, P->L, ph, pw, c->alpha[p]);
        }
    c->tre = (double*)malloc((size_t)c->S * c->S * sizeof(double));
    c->tim = (double*)malloc((size_t)c->S * c->S * sizeof(double));
    c->steps = (double*)malloc((size_t)c->Ho * c->Wo * sizeof(double));
    for (int m = 0; m < c->Ho * c->Wo; ++m) c->steps[m] = P->step;
    c->phi = (double*)calloc((size_t)P->H * P->W, sizeof(double));
    cs_refresh(c);
}

static void cs_close(chain_state* c)
{
    int np = c->npi * c->npj;
    for (int p = 0; p < np; ++p) { free(c->sre[p]); free(c->sim[p]); free(c->alpha[p]); }
    free(c->sre); free(c->sim); free(c->alpha);
    free(c->K); free(c->Ke); free(c->rho); free(c->mu); free(c->tre); free(c->tim); free(c->steps); free(c->phi);
}

/* Likelihood and prior changes for replacing rho_m (m = (i, j)) by rho_new
 * in state c.  Returns 0 when the proposal is impossible (some mu'_n <= 0
 * or some spectrum coefficient exactly zero); on success the new spectrum
 * is left in c->tre / c->tim.                                             */
static int cs_delta(chain_state* c, int i, int j, double rho_new, double* dL, double* dP)
{
    const or_problem* P = c->P;
    const int H = P->H, W = P->W, S = c->S, f = c->f, Le = c->Le, Lc = c->Lc;
    const double delta = rho_new - c->rho[i * c->Wo + j];
    int ok = 1;
    /* Eq. 6 summed over the camera pixels that see object pixel (i, j):
     * rows a with 0 <= p = f a + Le-1-i < Le (a in [i/f - Lc + 1, i/f]), the
     * same for columns, weight Ke[p][q] (f = 1: a in [i-2R, i], K[a-i+2R]). */
    double l = 0.0;
    for (int a = i / f - (Lc - 1); a <= i / f; ++a) {
        const int p = f * a + Le - 1 - i;
        if (a < 0 || a >= H || p < 0 || p >= Le) continue;
        for (int b = j / f - (Lc - 1); b <= j / f; ++b) {
            const int q = f * b + Le - 1 - j;
            if (b < 0 || b >= W || q < 0 || q >= Le) continue;
            int n = a * W + b;
            double mu_old = c->mu[n];
            double mu_new = mu_old + delta * c->Ke[p * Le + q];
            if (!(mu_new > 0.0)) { ok = 0; continue; }
            if (P->aug)   /* completed likelihood: the phi-dependent Poisson part */
                l += c->phi[n] * (log(mu_new) - log(mu_old)) - (mu_new - mu_old);
            else
                l += or_loglik(P->w[n], P->offset[n], P->gain[n], P->var[n], mu_new)
                   - or_loglik(P->w[n], P->offset[n], P->gain[n], P->var[n], mu_old);
        }
    }
    /* Eq. 8 for the one patch containing (i, j): the DFT is linear, so the
     * new spectrum is the old one plus delta times the transform of a unit
     * impulse at the in-patch offset (u, v).                              */
    int pi = i / S, pj = j / S, u = i - pi * S, v = j - pj * S;
    int ph = patch_len(pi * S, S, c->Ho), pw = patch_len(pj * S, S, c->Wo);
    int p = pi * c->npj + pj;
    for (int k = 0; k < ph; ++k)
        for (int q = 0; q < pw; ++q) {
            double th = 2.0 * M_PI * ((double)k * u / ph + (double)q * v / pw);
            c->tre[k * pw + q] = c->sre[p][k * pw + q] + delta * cos(th);
            c->tim[k * pw + q] = c->sim[p][k * pw + q] - delta * sin(th);
            if (c->tre[k * pw + q] == 0.0 && c->tim[k * pw + q] == 0.0) ok = 0;
        }
    double pr = 0.0;
    if (ok)
        pr = or_log_prior_patch(c->tre, c->tim, c->alpha[p], ph * pw)
           - or_log_prior_patch(c->sre[p], c->sim[p], c->alpha[p], ph * pw);
    *dL = l;
    *dP = pr;
    return ok;
}

static void cs_accept(chain_state* c, int i, int j, double rho_new)
{
    const or_problem* P = c->P;
    const int H = P->H, W = P->W, S = c->S, f = c->f, Le = c->Le, Lc = c->Lc;
    const double delta = rho_new - c->rho[i * c->Wo + j];
    for (int a = i / f - (Lc - 1); a <= i / f; ++a) {
        const int p = f * a + Le - 1 - i;
        if (a < 0 || a >= H || p < 0 || p >= Le) continue;
        for (int b = j / f - (Lc - 1); b <= j / f; ++b) {
            const int q = f * b + Le - 1 - j;
            if (b < 0 || b >= W || q < 0 || q >= Le) continue;
            c->mu[a * W + b] += delta * c->Ke[p * Le + q];
        }
    }
    int pi = i / S, pj = j / S;
    int ph = patch_len(pi * S, S, c->Ho), pw = patch_len(pj * S, S, c->Wo);
    int p = pi * c->npj + pj;
    memcpy(c->sre[p], c->tre, (size_t)ph * pw * sizeof(double));
    memcpy(c->sim[p], c->tim, (size_t)ph * pw * sizeof(double));
    c->rho[i * c->Wo + j] = rho_new;
}

/* Likelihood and prior changes for one hypothetical update of rho (a state
 * given by the caller) at object pixel m to rho_new.  Returns 1 if the
 * proposal is possible.                                                    */
int or_delta(const or_problem* P, const double* rho, int m, double rho_new, double* dL, double* dP)
{
    chain_state c;
    cs_open(&c, P, rho);
    int i = m / c.Wo, j = m % c.Wo;
    int ok = cs_delta(&c, i, j, rho_new, dL, dP);
    cs_close(&c);
    return ok;
}

/* One update of object pixel m at sweep t evaluated from the given state
 * using only local quantities: mu on the pixel's PSF window by Eq. 1-2 and
 * the spectrum of the pixel's own patch by its DFT, so it costs O(L^4 + S^4)
 * whatever the frame size.  Outputs the accept decision, the proposed value,
 * dL and dP (0 and 0 when the proposal is impossible).  For the first class
 * of a sweep started from rho this is exactly what the sampler does.       */
int or_single_update(const or_problem* P, const double* rho, int m, int t, int* accept,
                     double* rho_new, double* dL, double* dP)
{
    const int H = P->H, W = P->W, L = P->L, S = P->S, f = sub_of(P), Le = L + f - 1, Lc = (Le - 1) / f + 1;
    int Ho, Wo;
    obj_dims(P, &Ho, &Wo);
    const int i = m / Wo, j = m % Wo;
    double* K = (double*)malloc((size_t)L * L * sizeof(double));
    double* Ke = (double*)malloc((size_t)Le * Le * sizeof(double));
    normalised_psf(P, K);
    or_eff_kernel(K, L, f, Ke);
    double z, u;
    or_draw(P->seed, (uint32_t)m, (uint32_t)t, (uint32_t)P->chain, &z, &u);
    const double rn = rho[m] * exp(P->step * z);
    const double delta = rn - rho[m];
    int ok = 1;
    double l = 0.0;
    for (int a = i / f - (Lc - 1); a <= i / f; ++a) {
        const int pa = f * a + Le - 1 - i;
        if (a < 0 || a >= H || pa < 0 || pa >= Le) continue;
        for (int b = j / f - (Lc - 1); b <= j / f; ++b) {
            const int qb = f * b + Le - 1 - j;
            if (b < 0 || b >= W || qb < 0 || qb >= Le) continue;
            double mu = 0.0;
            for (int p = 0; p < Le; ++p)
                for (int q = 0; q < Le; ++q)
                    mu += Ke[p * Le + q] * rho[(f * a + Le - 1 - p) * Wo + (f * b + Le - 1 - q)];
            const int n = a * W + b;
            const double mu_new = mu + delta * Ke[pa * Le + qb];
            if (!(mu_new > 0.0)) { ok = 0; continue; }
            l += or_loglik(P->w[n], P->offset[n], P->gain[n], P->var[n], mu_new)
               - or_loglik(P->w[n], P->offset[n], P->gain[n], P->var[n], mu);
        }
    }
    const int pi = i / S, pj = j / S, i0 = pi * S, j0 = pj * S;
    const int ph = patch_len(i0, S, Ho), pw = patch_len(j0, S, Wo), n = ph * pw;
    double* re = (double*)malloc((size_t)n * sizeof(double));
    double* im = (double*)malloc((size_t)n * sizeof(double));
    double* re2 = (double*)malloc((size_t)n * sizeof(double));
    double* im2 = (double*)malloc((size_t)n * sizeof(double));
    double* al = (double*)malloc((size_t)n * sizeof(double));
    double* x = (double*)malloc((size_t)n * sizeof(double));
    for (int uu = 0; uu < ph; ++uu)
        for (int vv = 0; vv < pw; ++vv) x[uu * pw + vv] = rho[(i0 + uu) * Wo + j0 + vv];
    or_patch_dft(x, pw, ph, pw, re, im);
    x[(i - i0) * pw + (j - j0)] = rn;
    or_patch_dft(x, pw, ph, pw, re2, im2);
    or_alpha(K, L, ph, pw, al);
    for (int k = 0; k < n; ++k)
        if (re2[k] == 0.0 && im2[k] == 0.0) ok = 0;
    const double pr = ok ? or_log_prior_patch(re2, im2, al, n) - or_log_prior_patch(re, im, al, n) : 0.0;
    *accept = ok && (log(u) < l + pr + P->step * z);
    *rho_new = rn;
    *dL = ok ? l : 0.0;
    *dP = pr;
    free(K); free(Ke); free(re); free(im); free(re2); free(im2); free(al); free(x);
    return ok;
}

/* Run sweeps t0+1 .. t0+T of one chain.
 *   rho_in    starting object (NULL: the initial object of or_init)
 *   order     0: raster order inside a class; 1: reversed (for the
 *             conditional-independence check)
 * Outputs (any may be NULL):
 *   rho_out   final object (Ho*Wo)           mu_out   final mu (H*W)
 *   sum_out   sum of rho over the sweeps t > burn_in of this run (Ho*Wo)
 *   n_sum     number of such sweeps
 *   trace     log posterior after each sweep (T)
 *   acc_log   1/0 accept decision of each pixel in each sweep (T*Ho*Wo)
 *   samples   rho after each sweep (T*Ho*Wo)
 *   n_acc     accepted updates in each sweep (T)
 * Per sweep: for class (u, v) in raster order of the in-patch offset, for
 * each pixel of the class: draw, propose rho' = rho exp(step z), accept iff
 * log u < dL + dP + step z (the last term is the Hastings ratio of the
 * log-space walk); after the sweep add rho to the sum if t > burn_in,
 * recompute mu and spectra from rho if t is a multiple of refresh_every,
 * and record the log posterior.                                             */
int or_run(const or_problem* P, int t0, int T, int order, const double* rho_in,
           double* rho_out, double* mu_out, double* sum_out, int* n_sum,
           double* trace, uint8_t* acc_log, double* samples, int64_t* n_acc,
           double* steps_out, double* phi_out)
{
    chain_state c;
    cs_open(&c, P, rho_in);
    const int Ho = c.Ho, Wo = c.Wo, S = c.S;
    if (sum_out) memset(sum_out, 0, (size_t)Ho * Wo * sizeof(double));
    int ns = 0;
    for (int tt = 1; tt <= T; ++tt) {
        const int t = t0 + tt;
        int64_t acc = 0;
        /* this sweep's adaptation factors (burn-in sweeps only) */
        const double gain = OR_ADAPT_GAIN / sqrt((double)t);
        const double up = exp(gain * (1.0 - P->adapt_target)), down = exp(-gain * P->adapt_target);
        if (P->aug)   /* step (1): the photon counts given the current mu */
            for (int n = 0; n < P->H * P->W; ++n)
                c.phi[n] = (double)or_sample_phi(P->w[n], P->offset[n], P->gain[n], P->var[n], c.mu[n],
                                                 or_phi_uniform(P->seed, (uint32_t)n, (uint32_t)t, (uint32_t)P->chain));
        for (int u = 0; u < S; ++u)
            for (int v = 0; v < S; ++v) {
                int ni = (Ho - 1 - u) / S + 1, nj = (Wo - 1 - v) / S + 1;
                if (u >= Ho || v >= Wo) continue;
                for (int qi = 0; qi < ni; ++qi)
                    for (int qj = 0; qj < nj; ++qj) {
                        int ri = order ? ni - 1 - qi : qi, rj = order ? nj - 1 - qj : qj;
                        int i = u + ri * S, j = v + rj * S, m = i * Wo + j;
                        double z, uu;
                        or_draw(P->seed, (uint32_t)m, (uint32_t)t, (uint32_t)P->chain, &z, &uu);
                        const double sm = c.steps[m];
                        double rho_new = c.rho[m] * exp(sm * z);
                        double dL, dP;
                        int ok = cs_delta(&c, i, j, rho_new, &dL, &dP);
                        int accept = ok && (log(uu) < dL + dP + sm * z);
                        if (accept) { cs_accept(&c, i, j, rho_new); ++acc; }
                        if (P->adapt_target > 0.0 && t <= P->burn_in) {
                            double sn = sm * (accept ? up : down);
                            c.steps[m] = sn < OR_STEP_MIN ? OR_STEP_MIN : sn > OR_STEP_MAX ? OR_STEP_MAX : sn;
                        }
                        if (acc_log) acc_log[(size_t)(tt - 1) * Ho * Wo + m] = (uint8_t)accept;
                    }
            }
        if (t > P->burn_in) {
            if (sum_out) for (int m = 0; m < Ho * Wo; ++m) sum_out[m] += c.rho[m];
            ++ns;
        }
        if (P->refresh_every > 0 && t % P->refresh_every == 0) cs_refresh(&c);
        if (trace) trace[tt - 1] = P->aug ? or_log_joint(P, c.rho, c.phi) : or_log_posterior(P, c.rho);
        if (samples) memcpy(samples + (size_t)(tt - 1) * Ho * Wo, c.rho, (size_t)Ho * Wo * sizeof(double));
        if (n_acc) n_acc[tt - 1] = acc;
    }
    if (rho_out) memcpy(rho_out, c.rho, (size_t)Ho * Wo * sizeof(double));
    if (mu_out) memcpy(mu_out, c.mu, (size_t)P->H * P->W * sizeof(double));
    if (steps_out) memcpy(steps_out, c.steps, (size_t)Ho * Wo * sizeof(double));
    if (phi_out) memcpy(phi_out, c.phi, (size_t)P->H * P->W * sizeof(double));
    if (n_sum) *n_sum = ns;
    cs_close(&c);
    return 0;
}
