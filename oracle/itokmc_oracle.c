/*
 * itokmc_oracle.c -- slow, plain FP64 CPU oracle of one Ito-KMC time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * constant generator with the CUDA library; both are written independently
 * from the same written specification (R. Marskar, "Stochastic and
 * self-consistent 3D modeling of streamer discharge trees with Kinetic Monte
 * Carlo", arXiv 2307.01797).
 *
 * Every function below follows the paper in the paper's order.  Where the
 * paper leaves a detail open (cell-centred indexing, tie-breaks, random-number
 * layout, particle boundary conditions ...) the reading adopted is stated at
 * the function.  Compile with -O2 -ffp-contract=off (no implicit contraction,
 * no fast-math) so that every floating-point operation is a single IEEE-754
 * round-to-nearest operation performed in the order written; fused
 * multiply-adds appear only as explicit fma() calls (one rounding each: the
 * series evaluations and the interpolation sums).
 *
 * Contents
 *   Philox4x32-10 counter RNG      (Salmon et al., SC'11)
 *   ora_log / ora_exp / sincos2pi  (argument reduction + series, own code)
 *   Poisson sampler                (inversion; PTRS of Hoermann 1993)
 *   normal sampler                 (ziggurat of Marsaglia & Tsang 2000)
 *   push      a1+a2  -- Sec. 4.2 (CIC interpolation), Sec. 4.3 (explicit
 *                       Euler-Maruyama, first equation), Eq. ito_kernel
 *   diffuse / advect -- the semi-implicit transport of Sec. 4.3 (Eq.
 *                       Xdagger, Eq. particle_kernel, Eq. Vk1); its field
 *                       solve is oracle/semi_implicit.py
 *   sort      a3     -- stable sort by cell ("spatial binning", Sec. 5.6)
 *   deposit   a4     -- Sec. 4.2 CIC deposition in int64 fixed point
 *   kmc       a6     -- Sec. 3.2.3 steps 1-8 (Cao et al. hybrid, eps = inf)
 *   products  a7     -- Sec. 4.4, Eq. w
 *   photons   a8     -- Sec. 4.5, Eq. photon_transport; Sec. 5.1 kappa(f)
 *   merge     a9     -- Sec. 4.6, Eq. weight_median
 * The field solve (a5) is oracle/poisson.py (numpy, exact separable solve).
 *
 * Built twice: plain (one thread) and with -fopenmp (the CPU baseline on
 * all host cores).  The OpenMP pragmas only spread the independent
 * iterations of the particle and cell loops over threads (each particle and
 * each cell draws from its own Philox stream; integer sums are atomic), so
 * both builds compute the same values; a build without -fopenmp ignores them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Parameters of one realization (single cubic grid).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n;            /* cells per axis                                 */
    int32_t ppc;          /* target particles per cell after merge (2^k)    */
    int32_t n_new;        /* max new computational particles per cell (64)  */
    int32_t n_crit;       /* critical-reaction threshold N_c (5)            */
    int32_t n_ssa;        /* max SSA steps per substep N_SSA (10)           */
    int32_t frac_bits;    /* fixed-point bits s per axis (10)               */
    double lo[3], hi[3];  /* domain corners, m                              */
    double dt;            /* time step, s                                   */
    double mu, D;         /* electron mobility m^2/Vs, diffusion m^2/s      */
    double alpha_A, alpha_B, eta; /* alpha(E)=A exp(-B/|E|) 1/m; eta 1/m    */
    double photon_ratio;  /* k_gamma / k_alpha (0 disables photons)         */
    double kappa_lo, kappa_hi; /* absorption coefficient range 1/m         */
    double eps;           /* Cao accuracy factor (INFINITY in the paper)    */
    uint64_t seed;        /* Philox key of this realization                 */
    uint32_t step;        /* step counter k (part of every Philox counter)  */
    uint32_t pad;
    double beta_ep;       /* electron-ion recombination coefficient m^3/s   */
    double beta_np;       /* ion-ion recombination coefficient m^3/s        */
    double mu_ion;        /* ion mobility m^2/Vs (mobile ions)              */
    double D_ion;         /* ion diffusion coefficient m^2/s (mobile ions)  */
} ora_params;

enum { TAG_INIT = 1, TAG_PUSH = 2, TAG_KMC = 3, TAG_PRODUCT = 4, TAG_PHOTON = 5,
       TAG_PUSH_POS = 6, TAG_PUSH_NEG = 7, TAG_PRODUCT_POS = 8, TAG_PRODUCT_NEG = 9 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  One round maps (c0,c1,c2,c3) with key        */
/* (k0,k1) to (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)); the */
/* key is bumped by the Weyl constants between rounds.                      */
/* ------------------------------------------------------------------------ */
void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A draw stream: key = seed, counter = (index, step, tag<<24|sub, block).   */
/* Words are consumed in order; a new block is generated when the previous  */
/* four words are used up.                                                  */
typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    int pos;
} ora_stream;

static void stream_init(ora_stream* s, uint64_t seed, uint32_t index, uint32_t step,
                        uint32_t tag, uint32_t sub)
{
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->ctr[0] = index;
    s->ctr[1] = step;
    s->ctr[2] = (tag << 24) | sub;
    s->ctr[3] = 0;
    s->pos = 4;
}

static uint32_t stream_u32(ora_stream* s)
{
    if (s->pos == 4) {
        ora_philox4x32_10(s->ctr, s->key, s->buf);
        s->ctr[3] += 1;
        s->pos = 0;
    }
    return s->buf[s->pos++];
}

/* Uniform in (0,1): 52 random bits k from two words, u = (2k+1) 2^-53,     */
/* exact in double, never 0 or 1.                                           */
static double stream_uniform(ora_stream* s)
{
    uint32_t a = stream_u32(s);
    uint32_t b = stream_u32(s);
    uint64_t k = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
    return (double)(2u * k + 1u) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* Elementary functions, written here so that CPU and GPU agree bit for bit */
/* (libm implementations differ in the last place).                         */
/*                                                                          */
/* log: x = 2^e m with m in [sqrt(1/2), sqrt(2)); s = (m-1)/(m+1);          */
/*      ln m = 2 atanh(s) = 2s + 2s z P(z), z = s^2, P = sum z^j/(2j+3)     */
/*      (series through s^21, |s| <= 0.1716); ln x = e ln2_hi + (e ln2_lo + */
/*      ln m), ln2 split Cody-Waite style so that e*ln2_hi is exact.        */
/* exp: n = rint(x/ln2), r = (x - n ln2_hi) - n ln2_lo, |r| <= 0.35;        */
/*      e^r by its Taylor series through r^13 (Horner), scaled by 2^n.      */
/* sincos2pi(u): angle 2 pi u = (q + f) pi/2 with q = rint(4u) and          */
/*      f = 4u - q in [-1/2, 1/2] exact; a = f pi/2, |a| <= pi/4; sin a and */
/*      cos a by Taylor series through a^17 / a^18; quadrant swap by q.     */
/* Only +, -, *, / and exact bit manipulation are used.                     */
/* ------------------------------------------------------------------------ */
/* ln2 split: HI = double(ln2) with its low 21 mantissa bits cleared (so    */
/* e*HI is exact for |e| < 2^21); LO = ln2 - HI rounded to double.          */
static const double ORA_LN2_HI = 6.93147180369123816490e-01;
static const double ORA_LN2_LO = 1.90821492927058770002e-10;

static double bits_to_double(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint64_t double_to_bits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }

double ora_log(double x)
{
    if (!(x > 0.0)) return (x == 0.0) ? -INFINITY : NAN;
    if (isinf(x)) return x;
    int e = 0;
    uint64_t b = double_to_bits(x);
    int bexp = (int)((b >> 52) & 0x7ff);
    if (bexp == 0) {                 /* subnormal: scale into normal range */
        x = x * 0x1p54;
        e = -54;
        b = double_to_bits(x);
        bexp = (int)((b >> 52) & 0x7ff);
    }
    e += bexp - 1023;
    double m = bits_to_double((b & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL); /* [1,2) */
    if (m > 1.41421356237309504880) { m = m * 0.5; e += 1; }
    double f = m - 1.0;              /* exact (Sterbenz) */
    double s = f / (2.0 + f);
    double z = s * s;
    double p = 1.0 / 21.0;
    p = fma(p, z, 1.0 / 19.0);
    p = fma(p, z, 1.0 / 17.0);
    p = fma(p, z, 1.0 / 15.0);
    p = fma(p, z, 1.0 / 13.0);
    p = fma(p, z, 1.0 / 11.0);
    p = fma(p, z, 1.0 / 9.0);
    p = fma(p, z, 1.0 / 7.0);
    p = fma(p, z, 1.0 / 5.0);
    p = fma(p, z, 1.0 / 3.0);
    double two_s = 2.0 * s;
    double lnm = fma(two_s, z * p, two_s);
    double de = (double)e;
    return de * ORA_LN2_HI + (de * ORA_LN2_LO + lnm);
}

double ora_exp(double x)
{
    if (x != x) return x;
    if (x > 709.78) return INFINITY;
    if (x < -745.2) return 0.0;
    double nd = rint(x * 1.44269504088896340736);   /* x / ln2 */
    double r = (x - nd * ORA_LN2_HI) - nd * ORA_LN2_LO;
    double p = 1.0 / 6227020800.0;                  /* 1/13! */
    p = fma(p, r, 1.0 / 479001600.0);                  /* 1/12! */
    p = fma(p, r, 1.0 / 39916800.0);                   /* 1/11! */
    p = fma(p, r, 1.0 / 3628800.0);                    /* 1/10! */
    p = fma(p, r, 1.0 / 362880.0);                     /* 1/9!  */
    p = fma(p, r, 1.0 / 40320.0);
    p = fma(p, r, 1.0 / 5040.0);
    p = fma(p, r, 1.0 / 720.0);
    p = fma(p, r, 1.0 / 120.0);
    p = fma(p, r, 1.0 / 24.0);
    p = fma(p, r, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    int n = (int)nd;
    if (n > 1023) {                                 /* 2^n overflows alone */
        return (p * 2.0) * bits_to_double((uint64_t)(n - 1 + 1023) << 52);
    }
    if (n < -1020) {                                /* subnormal result    */
        double scaled = p * bits_to_double((uint64_t)(n + 600 + 1023) << 52);
        return scaled * 0x1p-600;
    }
    return p * bits_to_double((uint64_t)(n + 1023) << 52);
}

void ora_sincos2pi(double u, double* s_out, double* c_out)
{
    double t = 4.0 * u;
    double q = rint(t);
    double f = t - q;
    double a = f * 1.57079632679489661923;          /* pi/2 */
    double z = a * a;
    double sp = -1.0 / 355687428096000.0;           /* -1/17! */
    sp = fma(sp, z, 1.0 / 1307674368000.0);            /* 1/15!  */
    sp = fma(sp, z, -1.0 / 6227020800.0);               /* 1/13!  */
    sp = fma(sp, z, 1.0 / 39916800.0);                 /* 1/11!  */
    sp = fma(sp, z, -1.0 / 362880.0);
    sp = fma(sp, z, 1.0 / 5040.0);
    sp = fma(sp, z, -1.0 / 120.0);
    sp = fma(sp, z, 1.0 / 6.0);
    double sa = fma(-a, z * sp, a);
    double cp = 1.0 / 6402373705728000.0;           /* 1/18! */
    cp = fma(cp, z, -1.0 / 20922789888000.0);           /* 1/16! */
    cp = fma(cp, z, 1.0 / 87178291200.0);              /* 1/14! */
    cp = fma(cp, z, -1.0 / 479001600.0);                /* 1/12! */
    cp = fma(cp, z, 1.0 / 3628800.0);
    cp = fma(cp, z, -1.0 / 40320.0);
    cp = fma(cp, z, 1.0 / 720.0);
    cp = fma(cp, z, -1.0 / 24.0);
    cp = fma(cp, z, 0.5);
    double ca = fma(-z, cp, 1.0);
    int qi = ((int)q) & 3;
    double s, c;
    switch (qi) {
    case 0: s = sa; c = ca; break;
    case 1: s = ca; c = -sa; break;
    case 2: s = -sa; c = -ca; break;
    default: s = -ca; c = sa; break;
    }
    *s_out = s;
    *c_out = c;
}

/* ------------------------------------------------------------------------ */
/* Poisson sampler P(mu) used by tau-leaping (Eq. tau_leaping).             */
/* mu <= 0: 0 with no draw.  mu < 10: inversion by sequential search (one   */
/* uniform).  mu >= 10: PTRS, transformed rejection with squeeze (W.        */
/* Hoermann, "The transformed rejection method for generating Poisson       */
/* random variables", Insurance: Math. & Econ. 12, 1993), two uniforms per  */
/* trial; log k! exact below 10, Stirling series through k^-7 above.        */
/* ------------------------------------------------------------------------ */
static double ora_logfact(int64_t k)
{
    if (k < 10) {
        double f = 1.0;
        for (int64_t i = 2; i <= k; ++i) f = f * (double)i;
        return ora_log(f);
    }
    double x = (double)k;
    double r = 1.0 / x;
    double r2 = r * r;
    double ser = 1.0 / 1680.0;
    ser = 1.0 / 1260.0 - r2 * ser;
    ser = 1.0 / 360.0 - r2 * ser;
    ser = 1.0 / 12.0 - r2 * ser;
    ser = r * ser;
    return (((x + 0.5) * ora_log(x) - x) + 0.91893853320467274178) + ser;
}

static int64_t ora_poisson(ora_stream* s, double mu)
{
    if (!(mu > 0.0)) return 0;
    if (mu < 10.0) {
        double u = stream_uniform(s);
        double p = ora_exp(-mu);
        double F = p;
        int64_t k = 0;
        while (u > F && k < 200) {
            k += 1;
            p = (p * mu) / (double)k;
            F = F + p;
        }
        return k;
    }
    double slam = sqrt(mu);
    double loglam = ora_log(mu);
    double b = 0.931 + 2.53 * slam;
    double a = -0.059 + 0.02483 * b;
    double invalpha = 1.1239 + 1.1328 / (b - 3.4);
    double vr = 0.9277 - 3.6224 / (b - 2.0);
    for (int it = 0; it < 1000000; ++it) {
        double U = stream_uniform(s) - 0.5;
        double V = stream_uniform(s);
        double us = 0.5 - fabs(U);
        double kd = floor(((((2.0 * a) / us) + b) * U + mu) + 0.43);
        if (us >= 0.07 && V <= vr) return (int64_t)kd;
        if (kd < 0.0 || (us < 0.013 && V > us)) continue;
        /* the acceptance test as one logarithm (Hoermann's form) */
        double lhs = ora_log((V * invalpha) / ((a / (us * us)) + b));
        double rhs = ((-mu) + kd * loglam) - ora_logfact((int64_t)kd);
        if (lhs <= rhs) return (int64_t)kd;
    }
    return -1;
}

/* Exported for the oracle's own pins: n Poisson draws from one stream.     */
void ora_poisson_draws(uint64_t seed, uint32_t index, uint32_t step, uint32_t tag, uint32_t sub,
                       double mu, int64_t n, int64_t* out)
{
    ora_stream s;
    stream_init(&s, seed, index, step, tag, sub);
    for (int64_t i = 0; i < n; ++i) out[i] = ora_poisson(&s, mu);
}

/* Exported: n uniforms from one stream (pins of the uniform map).          */
void ora_uniform_draws(uint64_t seed, uint32_t index, uint32_t step, uint32_t tag, uint32_t sub,
                       int64_t n, double* out)
{
    ora_stream s;
    stream_init(&s, seed, index, step, tag, sub);
    for (int64_t i = 0; i < n; ++i) out[i] = stream_uniform(&s);
}

/* ------------------------------------------------------------------------ */
/* Standard normals by the ziggurat method (G. Marsaglia and W. W. Tsang,   */
/* "The ziggurat method for generating random variables", J. Stat. Softw.   */
/* 5(8), 2000), 128 layers, base-strip parameters r = 3.442619855899 and    */
/* v = 9.91256303526217e-3 of that paper, with a 53-bit magnitude:          */
/* each attempt takes two words U = a 2^32 + b: layer i = U mod 128, sign  */
/* bit 7, magnitude m = U >> 11; x = m W_i is accepted at once if m < K_i,  */
/* else by the base-strip tail (i = 0, Marsaglia's tail method) or the      */
/* wedge test against exp(-x^2/2).  The tables come from the paper's setup  */
/* recurrence, evaluated with the project's own ln/exp and IEEE sqrt.       */
/* ------------------------------------------------------------------------ */
#define ZIG_R 3.442619855899
#define ZIG_V 9.91256303526217e-3
#define ZIG_M 9007199254740992.0            /* 2^53 */
static double zig_w[128], zig_f[128];
static uint64_t zig_k[128];
static int zig_ready = 0;

static void zig_init(void)
{
    double q = ZIG_V / ora_exp(-0.5 * ZIG_R * ZIG_R);
    zig_k[0] = (uint64_t)((ZIG_R / q) * ZIG_M);
    zig_k[1] = 0;
    zig_w[0] = q / ZIG_M;
    zig_w[127] = ZIG_R / ZIG_M;
    zig_f[0] = 1.0;
    zig_f[127] = ora_exp(-0.5 * ZIG_R * ZIG_R);
    double d = ZIG_R, t = ZIG_R;
    for (int i = 126; i >= 1; --i) {
        d = sqrt(-2.0 * ora_log(ZIG_V / d + ora_exp(-0.5 * d * d)));
        zig_k[i + 1] = (uint64_t)((d / t) * ZIG_M);
        t = d;
        zig_f[i] = ora_exp(-0.5 * d * d);
        zig_w[i] = d / ZIG_M;
    }
    zig_ready = 1;
}

static double ora_normal(ora_stream* s)
{
    if (!zig_ready) zig_init();
    for (int attempt = 0; attempt < 64; ++attempt) {
        uint32_t a = stream_u32(s);
        uint32_t b = stream_u32(s);
        uint64_t U = ((uint64_t)a << 32) | (uint64_t)b;
        int i = (int)(U & 127u);
        int neg = (int)((U >> 7) & 1u);
        uint64_t m = U >> 11;
        double x = (double)m * zig_w[i];
        if (m < zig_k[i]) return neg ? -x : x;
        if (i == 0) {                         /* tail beyond r */
            double xt, y;
            int tries = 0;
            do {
                xt = -ora_log(stream_uniform(s)) / ZIG_R;
                y = -ora_log(stream_uniform(s));
            } while (y + y < xt * xt && ++tries < 64);
            double v = ZIG_R + xt;
            return neg ? -v : v;
        }
        double u = stream_uniform(s);        /* wedge */
        if (zig_f[i] + u * (zig_f[i - 1] - zig_f[i]) < ora_exp(-0.5 * x * x)) return neg ? -x : x;
    }
    return 0.0;
}

/* Exported for the pins: n normals from one stream.                        */
void ora_normal_draws(uint64_t seed, uint32_t index, uint32_t step, uint32_t tag, uint32_t sub,
                      int64_t n, double* out)
{
    ora_stream s;
    stream_init(&s, seed, index, step, tag, sub);
    for (int64_t i = 0; i < n; ++i) out[i] = ora_normal(&s);
}

/* ------------------------------------------------------------------------ */
/* Grid helpers.  Cell-centred mesh: cell i spans [lo+i h, lo+(i+1) h], its  */
/* centre is lo+(i+1/2) h (the paper's x_i = i dx read as the centre index). */
/* Linear index (k n + j) n + i, x fastest.                                 */
/* ------------------------------------------------------------------------ */
static double cell_h(const ora_params* p, int ax) { return (p->hi[ax] - p->lo[ax]) / (double)p->n; }

static int64_t lin(const ora_params* p, int i, int j, int k)
{
    return ((int64_t)k * p->n + j) * p->n + i;
}

static int clampi(int i, int n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

/* (x-lo)/h in grid units: the quotient by the reciprocal r = 1/h with one   */
/* fused correction, q0 = d r, q = q0 + (d - q0 h) r (Markstein's step; both  */
/* fused operations are single IEEE roundings).                             */
static double grid_quot(const ora_params* p, int ax, double x)
{
    double h = cell_h(p, ax);
    double r = 1.0 / h;
    double d = x - p->lo[ax];
    double q0 = d * r;
    return fma(fma(-q0, h, d), r, q0);
}

/* CIC stencil along one axis: u = (x-lo)/h - 1/2, i0 = floor(u), f = u-i0; */
/* weights (1-f, f) on cells (i0, i0+1), indices folded onto [0, n-1].      */
static void cic_axis(const ora_params* p, int ax, double x, int* ia, int* ib, double* f_out)
{
    double u = grid_quot(p, ax, x) - 0.5;
    double fl = floor(u);
    int i0 = (int)fl;
    *f_out = u - fl;
    *ia = clampi(i0, p->n);
    *ib = clampi(i0 + 1, p->n);
}

/* Cell of a position known to lie in [lo, hi): floor((x-lo)/h), top-clamped. */
static int cell_axis(const ora_params* p, int ax, double x)
{
    int i = (int)floor(grid_quot(p, ax, x));
    return i > p->n - 1 ? p->n - 1 : (i < 0 ? 0 : i);
}

static int inside(const ora_params* p, const double X[3])
{
    for (int ax = 0; ax < 3; ++ax)
        if (!(X[ax] >= p->lo[ax] && X[ax] < p->hi[ax])) return 0;
    return 1;
}

/* Trilinear (CIC) interpolation of a cell-centred field at X (Sec. 4.2,     */
/* V_p = v(X_p), Sec. 3.1).  Sum order: z outer, y, x inner; weight product  */
/* (wx*wy)*wz, accumulated by fused multiply-add.                            */
static double interp(const ora_params* p, const double* F, const int ia[3], const int ib[3],
                     const double f[3])
{
    double wx[2] = { 1.0 - f[0], f[0] };
    double wy[2] = { 1.0 - f[1], f[1] };
    double wz[2] = { 1.0 - f[2], f[2] };
    int ix[2] = { ia[0], ib[0] }, iy[2] = { ia[1], ib[1] }, iz[2] = { ia[2], ib[2] };
    double acc = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a)
                acc = fma((wx[a] * wy[b]) * wz[c], F[lin(p, ix[a], iy[b], iz[c])], acc);
    return acc;
}

/* ------------------------------------------------------------------------ */
/* a1+a2: interpolate E and push (explicit Euler-Maruyama, Sec. 4.3 first   */
/* equation; Eq. ito_kernel; V_p = sgn(Z) mu E(X_p) with sgn = -1 for       */
/* electrons, Eq. Vk1).  Normals N_x, N_y, N_z by the ziggurat sampler, in  */
/* that order, from the stream (index = i, step, PUSH).                      */
/* x' = (x + ((-mu) E_x) dt) + sqrt(2 D dt) N_x.  A particle with            */
/* x' outside [lo, hi) on any axis leaves through the electrode / side face  */
/* and is removed; its weight is tallied (particle boundary condition: the   */
/* paper states removal for photons only; electrons are absorbed likewise).  */
/* cell_out[i] = new linear cell, or -1 if removed.                          */
/* ------------------------------------------------------------------------ */
/* The push of one species (Eq. ito_kernel with V = sgn(Z_s) mu_s E, Eq.     */
/* Vk1): cmu = sgn(Z_s) mu_s (electrons -mu, positive ions +mu_ion, negative */
/* ions -mu_ion), diffusion D_s, normals from the stream (i, step, tag).     */
static void push_species(const ora_params* p, double cmu, double D, uint32_t tag, int64_t np,
                         const double* x, const double* y, const double* z, const double* Ex,
                         const double* Ey, const double* Ez, double* xo, double* yo, double* zo,
                         int64_t* cell_out)
{
    double sdt = sqrt((2.0 * D) * p->dt);
    double nmu = cmu;
    if (!zig_ready) zig_init();
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < np; ++i) {
        double X[3] = { x[i], y[i], z[i] };
        int ia[3], ib[3];
        double f[3];
        for (int ax = 0; ax < 3; ++ax) cic_axis(p, ax, X[ax], &ia[ax], &ib[ax], &f[ax]);
        double Ep[3] = { interp(p, Ex, ia, ib, f), interp(p, Ey, ia, ib, f), interp(p, Ez, ia, ib, f) };
        ora_stream s;
        stream_init(&s, p->seed, (uint32_t)i, p->step, tag, 0);
        double N[3];
        for (int ax = 0; ax < 3; ++ax) N[ax] = ora_normal(&s);
        double Xn[3];
        for (int ax = 0; ax < 3; ++ax) Xn[ax] = (X[ax] + (nmu * Ep[ax]) * p->dt) + sdt * N[ax];
        xo[i] = Xn[0]; yo[i] = Xn[1]; zo[i] = Xn[2];
        if (inside(p, Xn))
            cell_out[i] = lin(p, cell_axis(p, 0, Xn[0]), cell_axis(p, 1, Xn[1]), cell_axis(p, 2, Xn[2]));
        else
            cell_out[i] = -1;
    }
}

/* Species 0 electrons, 1 positive ions, 2 negative ions. */
static void species_transport(const ora_params* p, int species, double* cmu, double* D, uint32_t* tag)
{
    if (species == 1) { *cmu = p->mu_ion; *D = p->D_ion; *tag = TAG_PUSH_POS; }
    else if (species == 2) { *cmu = -p->mu_ion; *D = p->D_ion; *tag = TAG_PUSH_NEG; }
    else { *cmu = -p->mu; *D = p->D; *tag = TAG_PUSH; }
}

void ora_push(const ora_params* p, int64_t np, const double* x, const double* y, const double* z,
              const double* Ex, const double* Ey, const double* Ez,
              double* xo, double* yo, double* zo, int64_t* cell_out)
{
    push_species(p, -p->mu, p->D, TAG_PUSH, np, x, y, z, Ex, Ey, Ez, xo, yo, zo, cell_out);
}

void ora_push_species(const ora_params* p, int32_t species, int64_t np, const double* x, const double* y,
                      const double* z, const double* Ex, const double* Ey, const double* Ez, double* xo,
                      double* yo, double* zo, int64_t* cell_out)
{
    double cmu, D;
    uint32_t tag;
    species_transport(p, species, &cmu, &D, &tag);
    push_species(p, cmu, D, tag, np, x, y, z, Ex, Ey, Ez, xo, yo, zo, cell_out);
}

/* ------------------------------------------------------------------------ */
/* Semi-implicit transport (Sec. 4.3, Eq. particle_kernel and Eq. Xdagger;   */
/* Sec. 4.7 steps 2, 4 and 5).  ora_diffuse: the diffusive advance           */
/* X+ = X + sqrt(2 D dt) N with the normals of ora_push (same stream, same   */
/* order), no removal (the charge density rho+ of Sec. 4.7 step 3 is         */
/* deposited at X+ with the folded stencil).  ora_advect: V = -mu E(X) with  */
/* the new field interpolated at the position X of the start of the step     */
/* (Eq. Vk1), X' = X+ + V dt, removal outside [lo, hi) as in ora_push.       */
/* ------------------------------------------------------------------------ */
void ora_diffuse(const ora_params* p, int64_t np, const double* x, const double* y, const double* z,
                 double* xd, double* yd, double* zd)
{
    double sdt = sqrt((2.0 * p->D) * p->dt);
    for (int64_t i = 0; i < np; ++i) {
        ora_stream s;
        stream_init(&s, p->seed, (uint32_t)i, p->step, TAG_PUSH, 0);
        double N[3];
        for (int ax = 0; ax < 3; ++ax) N[ax] = ora_normal(&s);
        xd[i] = x[i] + sdt * N[0];
        yd[i] = y[i] + sdt * N[1];
        zd[i] = z[i] + sdt * N[2];
    }
}

void ora_advect(const ora_params* p, int64_t np, const double* x, const double* y, const double* z,
                const double* xd, const double* yd, const double* zd,
                const double* Ex, const double* Ey, const double* Ez,
                double* xo, double* yo, double* zo, int64_t* cell_out)
{
    double nmu = -p->mu;
    for (int64_t i = 0; i < np; ++i) {
        double X[3] = { x[i], y[i], z[i] };
        int ia[3], ib[3];
        double f[3];
        for (int ax = 0; ax < 3; ++ax) cic_axis(p, ax, X[ax], &ia[ax], &ib[ax], &f[ax]);
        double Ep[3] = { interp(p, Ex, ia, ib, f), interp(p, Ey, ia, ib, f), interp(p, Ez, ia, ib, f) };
        double Xd[3] = { xd[i], yd[i], zd[i] };
        double Xn[3];
        for (int ax = 0; ax < 3; ++ax) Xn[ax] = Xd[ax] + (nmu * Ep[ax]) * p->dt;
        xo[i] = Xn[0]; yo[i] = Xn[1]; zo[i] = Xn[2];
        if (inside(p, Xn))
            cell_out[i] = lin(p, cell_axis(p, 0, Xn[0]), cell_axis(p, 1, Xn[1]), cell_axis(p, 2, Xn[2]));
        else
            cell_out[i] = -1;
    }
}

/* ------------------------------------------------------------------------ */
/* a3: stable sort by cell; removed particles (cell -1) dropped.  The        */
/* canonical order is (cell, previous array index).  Writes the permutation  */
/* and returns the number kept.  Written as a counting sort (a stable sort). */
/* ------------------------------------------------------------------------ */
int64_t ora_sort_by_cell(int64_t np, int64_t ncell, const int64_t* cell, int64_t* perm)
{
    int64_t* cnt = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    for (int64_t i = 0; i < np; ++i)
        if (cell[i] >= 0) cnt[cell[i] + 1] += 1;
    for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
    int64_t kept = cnt[ncell];
    for (int64_t i = 0; i < np; ++i)
        if (cell[i] >= 0) perm[cnt[cell[i]]++] = i;
    free(cnt);
    return kept;
}

/* ------------------------------------------------------------------------ */
/* a4: CIC deposition (Sec. 4.2, W_cic(x) = 1-|x|) in int64 fixed point.     */
/* Per axis a = floor(f 2^s) with f from cic_axis; axis weights (2^s - a, a) */
/* so the 8 contributions w*Ax*Ay*Az sum to w 2^(3s) exactly.  ne_fix is in  */
/* units of 2^-3s electrons per cell.  Xe[c] = sum of w over the particles   */
/* whose cell is c (the KMC state X_e of Sec. 3.2).                          */
/* ------------------------------------------------------------------------ */
void ora_deposit(const ora_params* p, int64_t np, const double* x, const double* y, const double* z,
                 const uint32_t* w, const int64_t* cell, int64_t* ne_fix, int64_t* Xe)
{
    int s = p->frac_bits;
    int64_t one = (int64_t)1 << s;
    double scale = (double)one;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < np; ++i) {
        double X[3] = { x[i], y[i], z[i] };
        int ia[3], ib[3];
        int64_t A[3][2];
        for (int ax = 0; ax < 3; ++ax) {
            double f;
            cic_axis(p, ax, X[ax], &ia[ax], &ib[ax], &f);
            int64_t a = (int64_t)floor(f * scale);
            A[ax][0] = one - a;
            A[ax][1] = a;
        }
        int ix[2] = { ia[0], ib[0] }, iy[2] = { ia[1], ib[1] }, iz[2] = { ia[2], ib[2] };
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int64_t v = (int64_t)w[i] * A[0][a] * A[1][b] * A[2][c];
#pragma omp atomic
                    ne_fix[lin(p, ix[a], iy[b], iz[c])] += v;
                }
#pragma omp atomic
        Xe[cell[i]] += (int64_t)w[i];
    }
}

/* ------------------------------------------------------------------------ */
/* a6: per-cell KMC, Sec. 3.2.3 steps 1-8 (Cao, Gillespie, Petzold 2005,     */
/* 2006) for the network of Table air_reactions.  State (X_e, X_+, X_-) =    */
/* electrons, positive and negative ions of the cell; reactions             */
/*   r=0 ionization     e -> 2e + M+    a0 = k_alpha X_e       nu = (+1,+1, 0) */
/*   r=1 attachment     e -> M-         a1 = k_eta X_e         nu = (-1, 0,+1) */
/*   r=2 photon         e -> e + gamma  a2 = k_gamma X_e       nu = ( 0, 0, 0) */
/*   r=3 e-ion recomb.  e + M+ -> 0     a3 = k_ep X_e X_+      nu = (-1,-1, 0) */
/*   r=4 ion-ion recomb M- + M+ -> 0    a4 = k_np X_+ X_-      nu = ( 0,-1,-1) */
/* with k_alpha = alpha(|E|) mu |E|, k_eta = eta mu |E|, k_gamma =           */
/* photon_ratio k_alpha (Sec. 5.1 structure) and k_ep = beta_ep / dV,        */
/* k_np = beta_np / dV (Sec. 5.1, dV = the cell volume); with beta = 0 the   */
/* last two never fire and the network is the first-order one.  Readings:   */
/* a reaction with a positive propensity is critical when it is within N_c  */
/* firings of exhausting a reactant (attachment: X_e < N_c; e-ion           */
/* recombination: min(X_e, X_+) < N_c; ion-ion: min(X_+, X_-) < N_c);       */
/* dt_c = -ln(u)/A_c; dt_nc from the eps formula over the reactant species  */
/* of the non-critical reactions, g_i = 2 for a species that is a reactant  */
/* of a second-order reaction with a positive coefficient (distinct         */
/* reactants, Cao et al. 2006), else 1 (infinite for eps = inf); the SSA    */
/* switch (A dtau <= 1, dtau = min(dt - tau, dt_nc)) is tested before the   */
/* critical time is drawn, as in the cited Cao et al. (2006) procedure --   */
/* testing it after a critical draw that did not fire would count critical  */
/* firings twice; a substep that leaves any count negative is rejected,     */
/* dt_nc = dtau/2 and step 5 is redone with fresh draws (the critical time  */
/* is kept); the SSA branch runs at most N_SSA events and advances tau by   */
/* the full dtau if the next event falls beyond it, else by the time of the */
/* last event.  Draws come from the stream (index = cell, step, KMC).       */
/* Outputs per cell: firings of each reaction.                              */
/* ------------------------------------------------------------------------ */
static const int kmc_nu[5][3] = { { +1, +1, 0 }, { -1, 0, +1 }, { 0, 0, 0 }, { -1, -1, 0 }, { 0, -1, -1 } };

static void kmc_props(const double kr[5], const int64_t X[3], double a[5])
{
    double xe = (double)X[0], xp = (double)X[1], xm = (double)X[2];
    a[0] = kr[0] * xe;
    a[1] = kr[1] * xe;
    a[2] = kr[2] * xe;
    a[3] = (kr[3] * xe) * xp;
    a[4] = (kr[4] * xp) * xm;
}

static int kmc_cell(const ora_params* p, ora_stream* s, const int64_t X0[3], const double kr[5],
                    int64_t fired[5])
{
    int64_t X[3] = { X0[0], X0[1], X0[2] };
    double dt = p->dt;
    double tau = 0.0;
    /* g_i: 2 for a reactant of a second-order reaction present in the network */
    double g[3] = { kr[3] > 0.0 ? 2.0 : 1.0, (kr[3] > 0.0 || kr[4] > 0.0) ? 2.0 : 1.0, kr[4] > 0.0 ? 2.0 : 1.0 };
    for (int r = 0; r < 5; ++r) fired[r] = 0;
    for (int guard = 0; guard < 100000; ++guard) {
        if (!(tau < dt)) return 0;
        double a[5];
        kmc_props(kr, X, a);
        double A = (((a[0] + a[1]) + a[2]) + a[3]) + a[4];
        if (!(A > 0.0)) return 0;
        /* step 1: partition by the firings left before a reactant runs out */
        int64_t L3 = X[0] < X[1] ? X[0] : X[1], L4 = X[1] < X[2] ? X[1] : X[2];
        int crit[5] = { 0, a[1] > 0.0 && X[0] < (int64_t)p->n_crit, 0, a[3] > 0.0 && L3 < (int64_t)p->n_crit,
                        a[4] > 0.0 && L4 < (int64_t)p->n_crit };
        /* step 2 */
        double Ac = 0.0;
        for (int r = 0; r < 5; ++r) if (crit[r]) Ac = Ac + a[r];
        /* step 4: non-critical step bound from eps (infinite for eps = inf) */
        double dtnc = INFINITY;
        if (!isinf(p->eps)) {
            /* reactant species of the non-critical reactions: the electrons */
            /* (ionization is never critical), the ions through the          */
            /* recombinations present in the network (beta > 0)             */
            int reactant[3] = { 1, (!crit[3] && kr[3] > 0.0) || (!crit[4] && kr[4] > 0.0), !crit[4] && kr[4] > 0.0 };
            for (int i = 0; i < 3; ++i) {
                if (!reactant[i]) continue;
                double xi = 0.0, sig2 = 0.0;
                for (int r = 0; r < 5; ++r) {
                    if (crit[r]) continue;
                    xi = xi + (double)kmc_nu[r][i] * a[r];
                    sig2 = sig2 + (double)(kmc_nu[r][i] * kmc_nu[r][i]) * a[r];
                }
                double num = (p->eps * (double)X[i]) / g[i];
                if (num < 1.0) num = 1.0;
                double t1 = (xi != 0.0) ? num / fabs(xi) : INFINITY;
                double t2 = (sig2 != 0.0) ? (num * num) / sig2 : INFINITY;
                double ti = t1 < t2 ? t1 : t2;
                if (ti < dtnc) dtnc = ti;
            }
        }
        /* step 3 is drawn lazily (only when a leap is taken) and kept across */
        /* rejections ("return to step 5").                                   */
        double dtc = -1.0;
        for (int rej = 0; rej < 10000; ++rej) {
            double rem = dt - tau;
            double dtau = dtnc < rem ? dtnc : rem;
            int64_t k[5] = { 0, 0, 0, 0, 0 };
            double adv;
            if (A * dtau <= 1.0) {
                /* step 6b exception, checked before the critical draw as in  */
                /* Cao et al. (2006): SSA on the whole network, at most N_SSA */
                /* events within dtau; tau advances by dtau if the next event */
                /* falls beyond it, else by the time of the last event.       */
                int64_t Xs[3] = { X[0], X[1], X[2] };
                double t = 0.0;
                for (int ev = 0; ev < p->n_ssa; ++ev) {
                    double as[5];
                    kmc_props(kr, Xs, as);
                    double As = (((as[0] + as[1]) + as[2]) + as[3]) + as[4];
                    if (!(As > 0.0)) { t = dtau; break; }
                    double dte = (-ora_log(stream_uniform(s))) / As;
                    if (t + dte > dtau) { t = dtau; break; }
                    t = t + dte;
                    double target = stream_uniform(s) * As, cum = 0.0;
                    int j = (as[3] > 0.0 || as[4] > 0.0) ? (as[4] > 0.0 ? 4 : 3) : 2;
                    for (int r = 0; r < 5; ++r) {
                        cum = cum + as[r];
                        if (cum > target) { j = r; break; }
                    }
                    k[j] += 1;
                    for (int i = 0; i < 3; ++i) Xs[i] += kmc_nu[j][i];
                }
                adv = t;
            } else {
                /* step 3: time to the next critical reaction */
                if (dtc < 0.0)
                    dtc = (Ac > 0.0) ? (-ora_log(stream_uniform(s))) / Ac : INFINITY;
                if (dtc < dtnc && dtc < rem) {
                    /* step 6a: one critical reaction fires, non-critical leap */
                    dtau = dtc;
                    double target = stream_uniform(s) * Ac, cum = 0.0;
                    int rc = -1, last = -1;
                    for (int r = 0; r < 5; ++r) {
                        if (!crit[r]) continue;
                        last = r;
                        cum = cum + a[r];
                        if (cum > target) { rc = r; break; }
                    }
                    if (rc < 0) rc = last;
                    k[rc] += 1;
                }
                /* step 6a/6b: non-critical tau-leap over dtau (Eq. tau_leaping) */
                for (int r = 0; r < 5; ++r)
                    if (!crit[r]) k[r] += ora_poisson(s, a[r] * dtau);
                adv = dtau;
            }
            int64_t Xn[3];
            for (int i = 0; i < 3; ++i)
                Xn[i] = X[i] + kmc_nu[0][i] * k[0] + kmc_nu[1][i] * k[1] + kmc_nu[3][i] * k[3] + kmc_nu[4][i] * k[4];
            if (Xn[0] < 0 || Xn[1] < 0 || Xn[2] < 0) {   /* step 7a: reject, halve, redo step 5 */
                dtnc = dtau * 0.5;
                continue;
            }
            /* step 7b: accept */
            for (int i = 0; i < 3; ++i) X[i] = Xn[i];
            for (int r = 0; r < 5; ++r) fired[r] += k[r];
            if (adv >= rem) tau = dt; else tau = tau + adv;
            goto next_substep;
        }
        return -1;
    next_substep:;
    }
    return -1;
}

/* Reaction frequencies from the cell-centred field (Sec. 5.1, LFA). */
static void rates_at(const ora_params* p, double ex, double ey, double ez, double kr[3])
{
    double Em = sqrt((ex * ex + ey * ey) + ez * ez);
    double ve = p->mu * Em;
    double alpha = (Em > 0.0) ? p->alpha_A * ora_exp(-(p->alpha_B / Em)) : 0.0;
    kr[0] = alpha * ve;
    kr[1] = p->eta * ve;
    kr[2] = p->photon_ratio * kr[0];
}

/* Recombination frequencies per pair: k = beta / dV (Sec. 5.1). */
static void recomb_rates(const ora_params* p, double* k_ep, double* k_np)
{
    double dV = (cell_h(p, 0) * cell_h(p, 1)) * cell_h(p, 2);
    *k_ep = p->beta_ep / dV;
    *k_np = p->beta_np / dV;
}

/* Npos, Nneg: the ion counts at the start of the chemistry (NULL: none);  */
/* n_ep, n_np: recombination firings (NULL: not wanted).  A cell runs when  */
/* it has electrons, or ions of both signs with ion-ion recombination on.  */
/* Returns 0, or -1 if some cell did not finish (iteration guard).          */
int ora_kmc(const ora_params* p, const int64_t* Xe, const int64_t* Npos, const int64_t* Nneg,
            const double* Ex, const double* Ey, const double* Ez, int64_t* n_ion, int64_t* n_att,
            int64_t* n_ph, int64_t* n_ep, int64_t* n_np)
{
    int64_t ncell = (int64_t)p->n * p->n * p->n;
    int status = 0;
    double k_ep, k_np;
    recomb_rates(p, &k_ep, &k_np);
#pragma omp parallel for schedule(dynamic, 4096) reduction(min : status)
    for (int64_t c = 0; c < ncell; ++c) {
        n_ion[c] = n_att[c] = n_ph[c] = 0;
        if (n_ep) n_ep[c] = 0;
        if (n_np) n_np[c] = 0;
        int64_t X[3] = { Xe[c], Npos ? Npos[c] : 0, Nneg ? Nneg[c] : 0 };
        if (X[0] <= 0 && !(k_np > 0.0 && X[1] > 0 && X[2] > 0)) continue;
        double kr[5];
        rates_at(p, Ex[c], Ey[c], Ez[c], kr);
        kr[3] = k_ep;
        kr[4] = k_np;
        ora_stream s;
        stream_init(&s, p->seed, (uint32_t)c, p->step, TAG_KMC, 0);
        int64_t fired[5];
        if (kmc_cell(p, &s, X, kr, fired) != 0) status = -1;
        n_ion[c] = fired[0]; n_att[c] = fired[1]; n_ph[c] = fired[2];
        if (n_ep) n_ep[c] = fired[3];
        if (n_np) n_np[c] = fired[4];
    }
    return status;
}

/* Exported for the oracle's pins: a single cell, given rates, X0 and a     */
/* stream index; returns the final X, firings in fired[3].                  */
int64_t ora_kmc_single(const ora_params* p, int64_t X0, double k_ion, double k_att, double k_ph,
                       uint32_t index, int64_t* fired)
{
    double kr[5] = { k_ion, k_att, k_ph, 0.0, 0.0 };
    int64_t X[3] = { X0, 0, 0 }, f[5];
    ora_stream s;
    stream_init(&s, p->seed, index, p->step, TAG_KMC, 0);
    if (kmc_cell(p, &s, X, kr, f) != 0) return -1;
    fired[0] = f[0]; fired[1] = f[1]; fired[2] = f[2];
    return X0 + fired[0] - fired[1];
}

/* Exported for the oracle's pins: one cell of the whole network (counts   */
/* X0 = (X_e, X_+, X_-), frequencies kr[5]) on stream (index, step, KMC);   */
/* the final counts in X[3], firings in fired[5].  Returns 0 or -1 (guard). */
int ora_kmc_network(const ora_params* p, const int64_t* X0, const double* kr, uint32_t index,
                    int64_t* X, int64_t* fired)
{
    ora_stream s;
    stream_init(&s, p->seed, index, p->step, TAG_KMC, 0);
    if (kmc_cell(p, &s, X0, kr, fired) != 0) return -1;
    for (int i = 0; i < 3; ++i) {
        X[i] = X0[i];
        for (int r = 0; r < 5; ++r) X[i] += kmc_nu[r][i] * fired[r];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a7 + a8: KMC-particle coupling (Sec. 4.4) and photons (Sec. 4.5).         */
/* Gain dN > 0 in cell c: m = min(dN, N_new) new particles, weight           */
/* dN div m (Eq. w), the remainder on the first; positions uniform in the    */
/* cell, x = lo + (i + u) h, stream (c, step, PRODUCT, slot j).  Loss L > 0: */
/* removed from the cell's existing particles by systematic integer          */
/* sampling over cumulative weights C_p (W = sum w): particle p loses        */
/* floor((C_p L + R)/W) - floor((C_{p-1} L + R)/W), R = (64-bit draw) mod W  */
/* from stream (c, step, PRODUCT, N_new) -- exact, unbiased (each physical   */
/* electron removed with probability L/W).  Photons: m = min(N_gamma, N_new) */
/* superphotons with the same weight rule; stream (c, step, PHOTON, j):     */
/* emission point (3 uniforms), kappa = K1 (K2/K1)^U (Sec. 5.1), r =         */
/* -ln(u)/kappa (exponential with parameter kappa), c_z = 2u-1, phi = 2 pi u,*/
/* c_xy = sqrt((1-c_z)(1+c_z)) (cos, sin); Y = Y0 + r c (Eq.                 */
/* photon_transport).  Y inside [lo,hi)^3: photoionization creates an        */
/* electron of the photon's weight at Y and an M+ in Y's cell; otherwise the */
/* photon is lost.  New particles are listed by (source cell, products then  */
/* photoelectrons, slot).                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double* x; double* y; double* z; uint32_t* w; int64_t* cell;
    int64_t n, cap;
} ora_plist;

static int plist_push(ora_plist* L, double x, double y, double z, uint64_t w, int64_t cell)
{
    if (L->n >= L->cap) return -1;
    if (w > 0xffffffffull) return -2;
    L->x[L->n] = x; L->y[L->n] = y; L->z[L->n] = z; L->w[L->n] = (uint32_t)w; L->cell[L->n] = cell;
    L->n += 1;
    return 0;
}

/* One superphoton of cell c, slot j (stream (c, step, PHOTON, j)):          */
/* emission point Y0 uniform in the cell, absorption coefficient kappa,      */
/* absorption distance r and unit direction dir.                             */
static void photon_sample(const ora_params* p, int64_t c, uint32_t j, const int ijk[3], double lnK,
                          double Y0[3], double* kappa_out, double* r_out, double dir[3])
{
    ora_stream s;
    stream_init(&s, p->seed, (uint32_t)c, p->step, TAG_PHOTON, j);
    for (int ax = 0; ax < 3; ++ax) {
        double u = stream_uniform(&s);
        Y0[ax] = p->lo[ax] + ((double)ijk[ax] + u) * cell_h(p, ax);
    }
    double kappa = p->kappa_lo * ora_exp(stream_uniform(&s) * lnK);
    double r = (-ora_log(stream_uniform(&s))) / kappa;
    double cz = 2.0 * stream_uniform(&s) - 1.0;
    double sphi, cphi;
    ora_sincos2pi(stream_uniform(&s), &sphi, &cphi);
    double st = sqrt((1.0 - cz) * (1.0 + cz));
    dir[0] = st * cphi;
    dir[1] = st * sphi;
    dir[2] = cz;
    *kappa_out = kappa;
    *r_out = r;
}

/* Exported for the pins: the photon draws of cells c (given as i,j,k) for  */
/* slots 0..m-1: Y0 (3m), kappa (m), r (m), dir (3m).                       */
void ora_photon_samples(const ora_params* p, int32_t i, int32_t j, int32_t k, int64_t m,
                        double* Y0, double* kappa, double* r, double* dir)
{
    int ijk[3] = { i, j, k };
    int64_t c = lin(p, i, j, k);
    double lnK = ora_log(p->kappa_hi / p->kappa_lo);
    for (int64_t q = 0; q < m; ++q)
        photon_sample(p, c, (uint32_t)q, ijk, lnK, Y0 + 3 * q, kappa + q, r + q, dir + 3 * q);
}

/* Particles: sorted canonical arrays (x,y,z,w,cell) of length np with       */
/* cell_start[ncell+1].  Weights w are updated in place for losses.          */
/* New particles are written to (nx..ncell_new) up to cap_new; returns their */
/* count, -1 if capacity is exceeded, -2 on weight overflow.                 */
/* Npos/Nneg are updated (+ionizations, +attachments, +photoionizations).    */
int64_t ora_products_photons(const ora_params* p, int64_t np, const double* x, const double* y,
                             const double* z, uint32_t* w, const int64_t* cell_start,
                             const int64_t* Xe, const int64_t* n_ion, const int64_t* n_att,
                             const int64_t* n_ph, const int64_t* n_ep, const int64_t* n_np,
                             int64_t* Npos, int64_t* Nneg,
                             double* nx, double* ny, double* nz, uint32_t* nw, int64_t* ncell_new,
                             int64_t cap_new, int64_t* lost_photon_weight, int64_t* nsrc, int32_t* nkind,
                             int32_t* nslot)
{
    (void)np; (void)x; (void)y; (void)z;
    int64_t ncell = (int64_t)p->n * p->n * p->n;
    ora_plist L = { nx, ny, nz, nw, ncell_new, 0, cap_new };
    int64_t lost = 0;
    double h[3] = { cell_h(p, 0), cell_h(p, 1), cell_h(p, 2) };
    double lnK = ora_log(p->kappa_hi / p->kappa_lo);
    for (int64_t c = 0; c < ncell; ++c) {
        int ci = (int)(c % p->n), cj = (int)((c / p->n) % p->n), ck = (int)(c / ((int64_t)p->n * p->n));
        int ijk[3] = { ci, cj, ck };
        int64_t ep = n_ep ? n_ep[c] : 0, npr = n_np ? n_np[c] : 0;
        int64_t dN = n_ion[c] - n_att[c] - ep;
        Npos[c] += n_ion[c] - ep - npr;
        Nneg[c] += n_att[c] - npr;
        if (dN > 0) {
            int64_t m = dN < p->n_new ? dN : p->n_new;
            int64_t wq = dN / m, rem = dN % m;
            for (int64_t j = 0; j < m; ++j) {
                ora_stream s;
                stream_init(&s, p->seed, (uint32_t)c, p->step, TAG_PRODUCT, (uint32_t)j);
                double P[3];
                for (int ax = 0; ax < 3; ++ax) {
                    double u = stream_uniform(&s);
                    P[ax] = p->lo[ax] + ((double)ijk[ax] + u) * h[ax];
                }
                int rc = plist_push(&L, P[0], P[1], P[2], (uint64_t)(wq + (j == 0 ? rem : 0)), c);
                if (rc) return rc;
                if (nsrc) { nsrc[L.n - 1] = c; nkind[L.n - 1] = 0; nslot[L.n - 1] = (int32_t)j; }
            }
        } else if (dN < 0) {
            uint64_t Ls = (uint64_t)(-dN);
            uint64_t W = (uint64_t)Xe[c];
            ora_stream s;
            stream_init(&s, p->seed, (uint32_t)c, p->step, TAG_PRODUCT, (uint32_t)p->n_new);
            uint32_t a = stream_u32(&s), b = stream_u32(&s);
            uint64_t R = (((uint64_t)a << 32) | b) % W;
            unsigned __int128 C = 0;
            for (int64_t q = cell_start[c]; q < cell_start[c + 1]; ++q) {
                unsigned __int128 before = (C * Ls + R) / W;
                C += w[q];
                unsigned __int128 after = (C * Ls + R) / W;
                w[q] = (uint32_t)(w[q] - (uint64_t)(after - before));
            }
        }
        if (n_ph[c] > 0) {
            int64_t G = n_ph[c];
            int64_t m = G < p->n_new ? G : p->n_new;
            int64_t wq = G / m, rem = G % m;
            for (int64_t j = 0; j < m; ++j) {
                int64_t wj = wq + (j == 0 ? rem : 0);
                double Y0[3], kappa, r, dir[3], Ya[3];
                photon_sample(p, c, (uint32_t)j, ijk, lnK, Y0, &kappa, &r, dir);
                for (int ax = 0; ax < 3; ++ax) Ya[ax] = Y0[ax] + r * dir[ax];
                if (inside(p, Ya)) {
                    int64_t dc = lin(p, cell_axis(p, 0, Ya[0]), cell_axis(p, 1, Ya[1]), cell_axis(p, 2, Ya[2]));
                    Npos[dc] += wj;
                    int rc = plist_push(&L, Ya[0], Ya[1], Ya[2], (uint64_t)wj, dc);
                    if (rc) return rc;
                    if (nsrc) { nsrc[L.n - 1] = c; nkind[L.n - 1] = 1; nslot[L.n - 1] = (int32_t)j; }
                } else {
                    lost += wj;
                }
            }
        }
    }
    *lost_photon_weight = lost;
    return L.n;
}

/* Mobile ions: the gain or loss dN of one ion species per cell (positive    */
/* ions n_ion - n_ep - n_np, negative ions n_att - n_np), with the electron  */
/* products' rules of Sec. 4.4 and the species' stream tag: a gain gives     */
/* m = min(dN, N_new) particles of weight dN div m (remainder on the first)  */
/* uniform in the cell, stream (c, step, tag, j); a loss is removed from the */
/* cell's ion particles by systematic integer sampling against X (the NGP    */
/* ion count of the last deposit), stream (c, step, tag, N_new).  The new    */
/* particles' source cell, kind (0) and slot go to nsrc / nkind / nslot.     */
/* Returns their count, -1 (capacity) or -2 (weight overflow).              */
int64_t ora_species_products(const ora_params* p, int32_t species, const int64_t* cell_start,
                             const int64_t* X, const int64_t* dNs, uint32_t* w, double* nx, double* ny,
                             double* nz, uint32_t* nw, int64_t* ncell_new, int64_t* nsrc, int32_t* nkind,
                             int32_t* nslot, int64_t cap_new)
{
    int64_t ncell = (int64_t)p->n * p->n * p->n;
    uint32_t tag = species == 2 ? TAG_PRODUCT_NEG : TAG_PRODUCT_POS;
    ora_plist L = { nx, ny, nz, nw, ncell_new, 0, cap_new };
    double h[3] = { cell_h(p, 0), cell_h(p, 1), cell_h(p, 2) };
    for (int64_t c = 0; c < ncell; ++c) {
        int ijk[3] = { (int)(c % p->n), (int)((c / p->n) % p->n), (int)(c / ((int64_t)p->n * p->n)) };
        int64_t dN = dNs[c];
        if (dN > 0) {
            int64_t m = dN < p->n_new ? dN : p->n_new;
            int64_t wq = dN / m, rem = dN % m;
            for (int64_t j = 0; j < m; ++j) {
                ora_stream s;
                stream_init(&s, p->seed, (uint32_t)c, p->step, tag, (uint32_t)j);
                double P[3];
                for (int ax = 0; ax < 3; ++ax) {
                    double u = stream_uniform(&s);
                    P[ax] = p->lo[ax] + ((double)ijk[ax] + u) * h[ax];
                }
                int rc = plist_push(&L, P[0], P[1], P[2], (uint64_t)(wq + (j == 0 ? rem : 0)), c);
                if (rc) return rc;
                nsrc[L.n - 1] = c; nkind[L.n - 1] = 0; nslot[L.n - 1] = (int32_t)j;
            }
        } else if (dN < 0) {
            uint64_t Ls = (uint64_t)(-dN);
            uint64_t W = (uint64_t)X[c];
            if (Ls > W) return -3;
            ora_stream s;
            stream_init(&s, p->seed, (uint32_t)c, p->step, tag, (uint32_t)p->n_new);
            uint32_t a = stream_u32(&s), b = stream_u32(&s);
            uint64_t R = (((uint64_t)a << 32) | b) % W;
            unsigned __int128 C = 0;
            for (int64_t q = cell_start[c]; q < cell_start[c + 1]; ++q) {
                unsigned __int128 before = (C * Ls + R) / W;
                C += w[q];
                unsigned __int128 after = (C * Ls + R) / W;
                w[q] = (uint32_t)(w[q] - (uint64_t)(after - before));
            }
        }
    }
    return L.n;
}

/* ------------------------------------------------------------------------ */
/* a9: superparticle merge/split per cell (Sec. 4.6).  The cell's list (its  */
/* surviving particles in canonical order, then its new particles in list    */
/* order) is split level by level, T = ppc leaves: a node of weight >= 2 is  */
/* split; the axis is that of the largest bounding-box extent (ties: lowest  */
/* axis); the node is stably sorted by that coordinate; the median p' is the */
/* first index with sum_{<p'} w + w_p' > sum_{>p'} w (Eq. weight_median,     */
/* read with p' >= 1); a physical median (w = 1) joins the lighter side      */
/* (tie: left); a superparticle median is split into left weight             */
/* ceil(W/2) - W_left and the rest, zero-weight parts dropped.  Each leaf    */
/* becomes one particle: weight sum, weight-averaged position summed in list */
/* order.  Leaves are emitted left to right.                                 */
/* ------------------------------------------------------------------------ */
typedef struct { double X[3]; uint64_t w; int64_t ord; } ora_mp;

static int cmp_axis;
static int cmp_mp(const void* A, const void* B)
{
    const ora_mp* a = (const ora_mp*)A;
    const ora_mp* b = (const ora_mp*)B;
    double xa = a->X[cmp_axis], xb = b->X[cmp_axis];
    if (xa < xb) return -1;
    if (xa > xb) return 1;
    return (a->ord < b->ord) ? -1 : (a->ord > b->ord);
}

/* Splits node [P, P+M) (array of M particles) into left/right arrays.      */
static void split_node(ora_mp* P, int64_t M, ora_mp* left, int64_t* nl, ora_mp* right, int64_t* nr)
{
    double lo[3], hi[3];
    for (int ax = 0; ax < 3; ++ax) { lo[ax] = P[0].X[ax]; hi[ax] = P[0].X[ax]; }
    for (int64_t q = 1; q < M; ++q)
        for (int ax = 0; ax < 3; ++ax) {
            if (P[q].X[ax] < lo[ax]) lo[ax] = P[q].X[ax];
            if (P[q].X[ax] > hi[ax]) hi[ax] = P[q].X[ax];
        }
    int axis = 0;
    double ext[3] = { hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2] };
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    for (int64_t q = 0; q < M; ++q) P[q].ord = q;       /* stability key */
    cmp_axis = axis;
    qsort(P, (size_t)M, sizeof(ora_mp), cmp_mp);
    uint64_t W = 0;
    for (int64_t q = 0; q < M; ++q) W += P[q].w;
    uint64_t C = 0;
    int64_t pm = M - 1;
    for (int64_t q = 0; q < M; ++q) {
        C += P[q].w;
        if (2 * C > W) { pm = q; break; }
    }
    uint64_t WL = C - P[pm].w;
    uint64_t WR = W - C;
    *nl = 0; *nr = 0;
    for (int64_t q = 0; q < pm; ++q) left[(*nl)++] = P[q];
    if (P[pm].w == 1) {
        if (WL <= WR) left[(*nl)++] = P[pm];
        else right[(*nr)++] = P[pm];
    } else {
        uint64_t a = (W + 1) / 2 - WL;
        uint64_t b = P[pm].w - a;
        if (a > 0) { ora_mp m = P[pm]; m.w = a; left[(*nl)++] = m; }
        if (b > 0) { ora_mp m = P[pm]; m.w = b; right[(*nr)++] = m; }
    }
    for (int64_t q = pm + 1; q < M; ++q) right[(*nr)++] = P[q];
}

/* a / b given r = 1/b: q0 = a r, q = q0 + (a - q0 b) r (one fused          */
/* correction, as for the grid quotient).                                   */
static double quot_r(double a, double b, double r)
{
    double q0 = a * r;
    return fma(fma(-q0, b, a), r, q0);
}

/* Merge one cell's list in[0..M) into at most T leaves written to out.     */
/* Returns the number of leaves.                                             */
static int64_t merge_cell(const ora_mp* in, int64_t M, int T, ora_mp* out)
{
    /* nodes stored as consecutive ranges in a work buffer; each split may   */
    /* add one particle, so capacity M + T suffices.                         */
    int64_t cap = M + T + 1;
    ora_mp* cur = (ora_mp*)malloc(sizeof(ora_mp) * (size_t)cap);
    ora_mp* nxt = (ora_mp*)malloc(sizeof(ora_mp) * (size_t)cap);
    ora_mp* tl = (ora_mp*)malloc(sizeof(ora_mp) * (size_t)cap);
    ora_mp* tr = (ora_mp*)malloc(sizeof(ora_mp) * (size_t)cap);
    int64_t* nb = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T + 1));
    int64_t* nb2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T + 1));
    memcpy(cur, in, sizeof(ora_mp) * (size_t)M);
    int nnodes = 1;
    nb[0] = 0; nb[1] = M;
    for (int level = 1; level < T; level *= 2) {
        int64_t fill = 0;
        int nn = 0;
        nb2[0] = 0;
        for (int d = 0; d < nnodes; ++d) {
            ora_mp* node = cur + nb[d];
            int64_t m = nb[d + 1] - nb[d];
            uint64_t W = 0;
            for (int64_t q = 0; q < m; ++q) W += node[q].w;
            if (W >= 2) {
                int64_t nl, nr;
                split_node(node, m, tl, &nl, tr, &nr);
                memcpy(nxt + fill, tl, sizeof(ora_mp) * (size_t)nl); fill += nl; nb2[++nn] = fill;
                memcpy(nxt + fill, tr, sizeof(ora_mp) * (size_t)nr); fill += nr; nb2[++nn] = fill;
            } else {
                memcpy(nxt + fill, node, sizeof(ora_mp) * (size_t)m); fill += m; nb2[++nn] = fill;
            }
        }
        ora_mp* t = cur; cur = nxt; nxt = t;
        int64_t* tb = nb; nb = nb2; nb2 = tb;
        nnodes = nn;
    }
    for (int d = 0; d < nnodes; ++d) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        uint64_t W = 0;
        for (int64_t q = nb[d]; q < nb[d + 1]; ++q) {
            double wd = (double)cur[q].w;
            sx = fma(wd, cur[q].X[0], sx);
            sy = fma(wd, cur[q].X[1], sy);
            sz = fma(wd, cur[q].X[2], sz);
            W += cur[q].w;
        }
        /* centroid: quotients by the reciprocal of W with one fused correction */
        double Wd = (double)W;
        double rw = 1.0 / Wd;
        out[d].X[0] = quot_r(sx, Wd, rw);
        out[d].X[1] = quot_r(sy, Wd, rw);
        out[d].X[2] = quot_r(sz, Wd, rw);
        out[d].w = W;
        out[d].ord = d;
    }
    free(cur); free(nxt); free(tl); free(tr); free(nb); free(nb2);
    return nnodes;
}

/* Merge/split every cell.  Input: canonical sorted list (existing then new  */
/* per cell, already grouped by cell: in_start[ncell+1]).  Zero-weight       */
/* particles are skipped.  Output arrays need capacity sum min(W_c, ppc).    */
/* Returns the count, or -1 on capacity, -2 on weight overflow.             */
int64_t ora_merge(const ora_params* p, const double* x, const double* y, const double* z,
                  const uint32_t* w, const int64_t* in_start,
                  double* ox, double* oy, double* oz, uint32_t* ow, int64_t* ocell, int64_t cap)
{
    int64_t ncell = (int64_t)p->n * p->n * p->n;
    int T = p->ppc;
    int64_t nout = 0;
    int64_t maxm = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t m = in_start[c + 1] - in_start[c];
        if (m > maxm) maxm = m;
    }
    ora_mp* buf = (ora_mp*)malloc(sizeof(ora_mp) * (size_t)(maxm + 1));
    ora_mp* leaves = (ora_mp*)malloc(sizeof(ora_mp) * (size_t)(T + 1));
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t M = 0;
        for (int64_t q = in_start[c]; q < in_start[c + 1]; ++q) {
            if (w[q] == 0) continue;
            buf[M].X[0] = x[q]; buf[M].X[1] = y[q]; buf[M].X[2] = z[q];
            buf[M].w = w[q]; buf[M].ord = M;
            M += 1;
        }
        if (M == 0) continue;
        int64_t nl = merge_cell(buf, M, T, leaves);
        for (int64_t d = 0; d < nl; ++d) {
            if (nout >= cap) { free(buf); free(leaves); return -1; }
            if (leaves[d].w > 0xffffffffull) { free(buf); free(leaves); return -2; }
            ox[nout] = leaves[d].X[0]; oy[nout] = leaves[d].X[1]; oz[nout] = leaves[d].X[2];
            ow[nout] = (uint32_t)leaves[d].w; ocell[nout] = c;
            nout += 1;
        }
    }
    free(buf); free(leaves);
    return nout;
}

/* Exported for the pins: merge one list (positions x,y,z, weights w) into  */
/* at most T leaves.  Returns the leaf count.                               */
int64_t ora_merge_list(int64_t M, const double* x, const double* y, const double* z,
                       const uint64_t* w, int32_t T, double* ox, double* oy, double* oz, uint64_t* ow)
{
    ora_mp* in = (ora_mp*)malloc(sizeof(ora_mp) * (size_t)(M + 1));
    ora_mp* out = (ora_mp*)malloc(sizeof(ora_mp) * (size_t)(T + 1));
    int64_t K = 0;
    for (int64_t q = 0; q < M; ++q) {
        if (w[q] == 0) continue;
        in[K].X[0] = x[q]; in[K].X[1] = y[q]; in[K].X[2] = z[q]; in[K].w = w[q]; in[K].ord = K;
        K += 1;
    }
    int64_t nl = (K > 0) ? merge_cell(in, K, T, out) : 0;
    for (int64_t d = 0; d < nl; ++d) {
        ox[d] = out[d].X[0]; oy[d] = out[d].X[1]; oz[d] = out[d].X[2]; ow[d] = out[d].w;
    }
    free(in); free(out);
    return nl;
}

/* Cell of each position (floor((x-lo)/h), top-clamped), or -1 outside       */
/* [lo, hi): the key by which an arbitrary particle list is put in canonical */
/* order (a stable sort by this key, ora_sort_by_cell).                      */
void ora_cells(const ora_params* p, int64_t np, const double* x, const double* y, const double* z,
               int64_t* cell)
{
    for (int64_t i = 0; i < np; ++i) {
        double X[3] = { x[i], y[i], z[i] };
        cell[i] = inside(p, X) ? lin(p, cell_axis(p, 0, X[0]), cell_axis(p, 1, X[1]), cell_axis(p, 2, X[2])) : -1;
    }
}

/* Exported for the pins of the grid arithmetic (no step calls it): for each */
/* coordinate x on axis ax, the quotient q = (x-lo)/h as grid_quot forms it, */
/* the cell of cell_axis, the folded CIC indices (ia, ib) and fraction f of  */
/* cic_axis, and the deposit's fixed-point weight a = floor(f 2^s).          */
void ora_grid_axis(const ora_params* p, int32_t ax, int64_t np, const double* x, double* q, int64_t* cell,
                   int64_t* ia, int64_t* ib, double* f, int64_t* a)
{
    double scale = (double)((int64_t)1 << p->frac_bits);
    for (int64_t i = 0; i < np; ++i) {
        int ja, jb;
        double fv;
        q[i] = grid_quot(p, ax, x[i]);
        cell[i] = cell_axis(p, ax, x[i]);
        cic_axis(p, ax, x[i], &ja, &jb, &fv);
        ia[i] = ja; ib[i] = jb; f[i] = fv;
        a[i] = (int64_t)floor(fv * scale);
    }
}

/* Exported for the pins of the interpolation (no step calls it): the CIC    */
/* interpolation of one cell-centred scalar field F at each point, exactly   */
/* as ora_push interpolates each component of E.                             */
void ora_interp_points(const ora_params* p, const double* F, int64_t np, const double* x, const double* y,
                       const double* z, double* out)
{
    for (int64_t i = 0; i < np; ++i) {
        double X[3] = { x[i], y[i], z[i] };
        int ia[3], ib[3];
        double f[3];
        for (int ax = 0; ax < 3; ++ax) cic_axis(p, ax, X[ax], &ia[ax], &ib[ax], &f[ax]);
        out[i] = interp(p, F, ia, ib, f);
    }
}

/* ------------------------------------------------------------------------ */
/* Initial electrons from Gaussian seeds (the initial conditions of Sec.    */
/* 5.1: electrons, or electron-ion pairs, seeded as Gaussian blobs).  The   */
/* density at the centre x_c of cell c is n(x_c) = sum_b A_b exp(-|x_c -    */
/* c_b|^2 / (2 s_b^2)) (squared distance summed x, y, z); the cell receives */
/* N_c ~ Poisson(n(x_c) dV) electrons, drawn from the stream (index = c,     */
/* step, INIT, sub 0) with the tau-leap's sampler, carried by m =           */
/* min(N_c, ppc) superparticles with the weight rule of Eq. w (N_c div m,   */
/* the remainder on the first), each uniform in the cell: three FP64        */
/* uniforms from the stream (c, step, INIT, 1 + slot), x = lo + (i + u) h.  */
/* Blob b seeds the realization real_b (or every one when real_b < 0); the  */
/* oracle seeds one realization, `real`.  Particles are written in          */
/* canonical order (cell, slot); counts[c] = N_c.  Returns the particle     */
/* count, or -1 if cap is exceeded, -2 if a weight exceeds 2^32 - 1.        */
/* ------------------------------------------------------------------------ */
int64_t ora_seed_blobs(const ora_params* p, int32_t nb, const double* centers, const double* sigma,
                       const double* peak, const int32_t* real_of_blob, int32_t real,
                       double* x, double* y, double* z, uint32_t* w, int64_t* cell, int64_t* counts, int64_t cap)
{
    int64_t ncell = (int64_t)p->n * p->n * p->n;
    double h[3] = { cell_h(p, 0), cell_h(p, 1), cell_h(p, 2) };
    double dV = (h[0] * h[1]) * h[2];
    int64_t np = 0;
    for (int64_t c = 0; c < ncell; ++c) {
        int ijk[3] = { (int)(c % p->n), (int)((c / p->n) % p->n), (int)(c / ((int64_t)p->n * p->n)) };
        double xc[3];
        for (int ax = 0; ax < 3; ++ax) xc[ax] = p->lo[ax] + ((double)ijk[ax] + 0.5) * h[ax];
        double dens = 0.0;
        for (int32_t b = 0; b < nb; ++b) {
            if (real_of_blob[b] >= 0 && real_of_blob[b] != real) continue;
            double d0 = xc[0] - centers[3 * b], d1 = xc[1] - centers[3 * b + 1], d2 = xc[2] - centers[3 * b + 2];
            double r2 = (d0 * d0 + d1 * d1) + d2 * d2;
            dens = dens + peak[b] * ora_exp(-r2 / (2.0 * sigma[b] * sigma[b]));
        }
        ora_stream s;
        stream_init(&s, p->seed, (uint32_t)c, p->step, TAG_INIT, 0);
        int64_t N = ora_poisson(&s, dens * dV);
        counts[c] = N;
        if (N <= 0) continue;
        int64_t m = N < p->ppc ? N : p->ppc;
        int64_t wq = N / m, rem = N % m;
        if (wq + rem > 0xffffffffll) return -2;
        for (int64_t j = 0; j < m; ++j) {
            if (np >= cap) return -1;
            ora_stream t;
            stream_init(&t, p->seed, (uint32_t)c, p->step, TAG_INIT, (uint32_t)(1 + j));
            double P[3];
            for (int ax = 0; ax < 3; ++ax) {
                double u = stream_uniform(&t);
                P[ax] = p->lo[ax] + ((double)ijk[ax] + u) * h[ax];
            }
            x[np] = P[0]; y[np] = P[1]; z[np] = P[2];
            w[np] = (uint32_t)(wq + (j == 0 ? rem : 0));
            cell[np] = c;
            np += 1;
        }
    }
    return np;
}

/* ------------------------------------------------------------------------ */
/* 0-D KMC ensembles (Sec. 3.2.4): n_real independent single cells, each    */
/* starting from X0 electrons in the field magnitude E_mag (rates as in the  */
/* spatial step: the field (0, 0, -E_mag)), advanced n_steps steps of dt,   */
/* realization m, step k drawing from the stream (key seed, index m, step   */
/* k, KMC).  X[m (n_steps + 1) + k] = electrons after k steps.  Returns 0,  */
/* or -1 if some cell hit the iteration guard.                               */
/* ------------------------------------------------------------------------ */
int ora_kmc0d(const ora_params* p, double E_mag, int64_t X0, int32_t n_real, int32_t n_steps, int64_t* X)
{
    double kr[5];
    rates_at(p, 0.0, 0.0, -E_mag, kr);
    kr[3] = kr[4] = 0.0;              /* the first-order network (no ion counts tracked) */
    int status = 0;
    for (int32_t m = 0; m < n_real; ++m) {
        int64_t x = X0;
        int64_t* out = X + (int64_t)m * (n_steps + 1);
        out[0] = x;
        for (int32_t k = 0; k < n_steps; ++k) {
            int64_t fired[5] = { 0, 0, 0, 0, 0 };
            if (x > 0) {
                int64_t X[3] = { x, 0, 0 };
                ora_stream s;
                stream_init(&s, p->seed, (uint32_t)m, (uint32_t)k, TAG_KMC, 0);
                if (kmc_cell(p, &s, X, kr, fired) != 0) status = -1;
            }
            x += fired[0] - fired[1];
            out[k + 1] = x;
        }
    }
    return status;
}
