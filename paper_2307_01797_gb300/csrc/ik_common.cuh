// ik_common.cuh -- device-side building blocks of libitokmc (sm_103a).
//
// Counter-based random numbers (Philox4x32-10, Salmon et al. SC'11), the
// uniform and normal maps, FP64 log/exp/sincos(2 pi u) written from their
// series so that every device agrees with any other IEEE-754 implementation
// of the same operation sequence, the Poisson sampler of the tau-leap, and
// grid helpers.  All translation units are compiled with -fmad=false: each
// FP64 expression below is evaluated as written, one rounding per operation.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ik {

// ---------------------------------------------------------------- parameters
// Kernel-argument copy of the configuration (one realization's grid; all
// realizations share it).
struct Params {
    int n, n3;              // cells per axis, cells per realization
    int R;                  // realizations
    int S;                  // particle species blocks: 1 (electrons), or 3 with mobile ions
    int B;                  // particle blocks S R: block b holds species b / R of realization b % R
    int log2n;
    int ppc, n_new, n_crit, n_ssa, frac_bits;
    int dep_win;            // largest shared deposit window (cells) a push block uses, <= DEP_WIN_MAX
    double lo[3], hi[3], h[3], rh[3];   // rh = 1/h
    double dt, mu, D, alpha_A, alpha_B, eta, photon_ratio, kappa_lo, kappa_hi, eps;
    double sdt;             // sqrt(2 D dt)
    double k_ep, k_np;      // recombination frequencies per pair, beta / dV (1/s)
    double E0;
    uint64_t seed0;
    uint32_t step;
    // graph-replayed steps read the step counter from device memory (the
    // last node of a step advances it); otherwise null and step is used
    const uint32_t* step_dev;
    // FP32 form constants (cell units)
    float f_drift;          // -mu dt / h   (multiplies E in V/m)
    float f_diff;           // sqrt(2 D dt) / h
    // per species (electrons, positive ions, negative ions): drift
    // coefficient sgn(Z) mu (V = cmu E), sqrt(2 D dt), the FP32 form's
    // cmu dt / h and sqrt(2 D dt) / h, and the push and product stream tags
    double cmu_sp[3], sdt_sp[3];
    float f_drift_sp[3], f_diff_sp[3];
    uint32_t push_tag_sp[3], prod_tag_sp[3];
};

constexpr int DEP_WIN_MAX = 2048;   // cells of the push's shared deposit window (16 KB)

enum : uint32_t {
    TAG_INIT = 1u, TAG_PUSH = 2u, TAG_KMC = 3u, TAG_PRODUCT = 4u, TAG_PHOTON = 5u,
    TAG_PUSH_POS = 6u, TAG_PUSH_NEG = 7u, TAG_PRODUCT_POS = 8u, TAG_PRODUCT_NEG = 9u
};

// Device error word bits (OR-ed by kernels, read by the host after a stage).
enum : uint32_t {
    DERR_CAPACITY = 1u, DERR_OVERFLOW = 2u, DERR_KMC = 4u, DERR_TIMEOUT = 8u, DERR_INTERNAL = 16u
};

// ---------------------------------------------------------------- Philox
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox10(u32x4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = u32x4{ hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0 };
    }
    return c;
}

// A draw stream (key = seed, counter = (index, step, tag<<24|sub, block));
// words are consumed in order, a block is generated every four words.
// (2k+1) 2^-53 for a 52-bit k, assembled from its bits with integer
// instructions (the value is exact: 2k+1 < 2^53).
__device__ __forceinline__ double u53(uint64_t k)
{
    const uint64_t m = 2ull * k + 1ull;
    const int p = 63 - __clzll((long long)m);            // leading bit, 0..52
    const uint64_t bits = ((uint64_t)(p - 53 + 1023) << 52) | ((m << (52 - p)) & 0x000fffffffffffffull);
    return __longlong_as_double((long long)bits);
}

struct Stream {
    uint32_t k0, k1, c0, c1, c2, blk;
    u32x4 buf;
    int pos;
    __device__ __forceinline__ Stream(uint64_t seed, uint32_t index, uint32_t step, uint32_t tag,
                                      uint32_t sub)
        : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), c0(index), c1(step),
          c2((tag << 24) | sub), blk(0), buf{0, 0, 0, 0}, pos(4) {}
    __device__ __forceinline__ uint32_t u32()
    {
        if (pos == 4) {
            buf = philox10(u32x4{ c0, c1, c2, blk }, k0, k1);
            ++blk;
            pos = 0;
        }
        const uint32_t v = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
        ++pos;
        return v;
    }
    // uniform on (0,1): k = 52 random bits, (2k+1) 2^-53 (exact)
    __device__ __forceinline__ double uniform()
    {
        const uint32_t a = u32();
        const uint32_t b = u32();
        const uint64_t k = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
        return u53(k);
    }
};

// The stream consumed two words at a time (the word order of Stream): pair
// k is words 2k, 2k+1; uniform() is the FP64 uniform of the next pair,
// uniform32() the FP32 uniform of its high word.
struct PairStream {
    uint32_t k0, k1, c0, c1, c2, blk;
    u32x4 buf;
    bool hi_half;                 // next pair is (buf.z, buf.w)
    __device__ __forceinline__ PairStream(uint64_t seed, uint32_t index, uint32_t step, uint32_t tag, uint32_t sub)
        : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), c0(index), c1(step), c2((tag << 24) | sub), blk(0),
          buf{ 0, 0, 0, 0 }, hi_half(false)
    {
        buf = philox10(u32x4{ c0, c1, c2, blk }, k0, k1);
        ++blk;
    }
    __device__ __forceinline__ void pair(uint32_t& a, uint32_t& b)
    {
        if (hi_half) {
            a = buf.z; b = buf.w;
            buf = philox10(u32x4{ c0, c1, c2, blk }, k0, k1);
            ++blk;
        } else {
            a = buf.x; b = buf.y;
        }
        hi_half = !hi_half;
    }
    __device__ __forceinline__ double uniform()
    {
        uint32_t a, b;
        pair(a, b);
        return u53((((uint64_t)a) << 20) | (uint64_t)(b >> 12));
    }
    __device__ __forceinline__ float uniform32();
};

// FP32 uniform on (0,1) from the high word of an FP64 uniform: its top 23
// bits k give (2k+1) 2^-24 (exact in FP32), the FP64 uniform to within an
// FP32 ulp.
__device__ __forceinline__ float uniform_f32(uint32_t v)
{
    return (float)(2u * (v >> 9) + 1u) * 0x1p-24f;
}

__device__ __forceinline__ float PairStream::uniform32()
{
    uint32_t a, b;
    pair(a, b);
    return uniform_f32(a);
}

// ---------------------------------------------------------------- FP64 math
// log: x = 2^e m, m in [1/sqrt2, sqrt2); s = (m-1)/(m+1);
// ln m = 2s + 2s z P(z), z = s^2, P(z) = sum_{j=0..9} z^j / (2j+3).
// ln x = e*LN2_HI + (e*LN2_LO + ln m); LN2_HI = ln2 with 21 low bits cleared.
__device__ __forceinline__ double dlog(double x)
{
    if (!(x > 0.0)) return (x == 0.0) ? -__longlong_as_double(0x7ff0000000000000ll) : __longlong_as_double(0x7ff8000000000000ll);
    if (x == __longlong_as_double(0x7ff0000000000000ll)) return x;
    int e = 0;
    uint64_t b = (uint64_t)__double_as_longlong(x);
    int bexp = (int)((b >> 52) & 0x7ff);
    if (bexp == 0) {
        x = x * 0x1p54;
        e = -54;
        b = (uint64_t)__double_as_longlong(x);
        bexp = (int)((b >> 52) & 0x7ff);
    }
    e += bexp - 1023;
    double m = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
    if (m > 1.41421356237309504880) { m = m * 0.5; e += 1; }
    const double f = m - 1.0;
    const double s = f / (2.0 + f);
    const double z = s * s;
    double p = 1.0 / 21.0;
    p = __fma_rn(p, z, 1.0 / 19.0);
    p = __fma_rn(p, z, 1.0 / 17.0);
    p = __fma_rn(p, z, 1.0 / 15.0);
    p = __fma_rn(p, z, 1.0 / 13.0);
    p = __fma_rn(p, z, 1.0 / 11.0);
    p = __fma_rn(p, z, 1.0 / 9.0);
    p = __fma_rn(p, z, 1.0 / 7.0);
    p = __fma_rn(p, z, 1.0 / 5.0);
    p = __fma_rn(p, z, 1.0 / 3.0);
    const double t = 2.0 * s;
    const double lnm = __fma_rn(t, z * p, t);
    const double de = (double)e;
    return de * 6.93147180369123816490e-01 + (de * 1.90821492927058770002e-10 + lnm);
}

// exp: n = rint(x / ln2), r = (x - n LN2_HI) - n LN2_LO, Taylor to r^13.
__device__ __forceinline__ double dexp(double x)
{
    if (x != x) return x;
    if (x > 709.78) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -745.2) return 0.0;
    const double nd = rint(x * 1.44269504088896340736);
    const double r = (x - nd * 6.93147180369123816490e-01) - nd * 1.90821492927058770002e-10;
    double p = 1.0 / 6227020800.0;
    p = __fma_rn(p, r, 1.0 / 479001600.0);
    p = __fma_rn(p, r, 1.0 / 39916800.0);
    p = __fma_rn(p, r, 1.0 / 3628800.0);
    p = __fma_rn(p, r, 1.0 / 362880.0);
    p = __fma_rn(p, r, 1.0 / 40320.0);
    p = __fma_rn(p, r, 1.0 / 5040.0);
    p = __fma_rn(p, r, 1.0 / 720.0);
    p = __fma_rn(p, r, 1.0 / 120.0);
    p = __fma_rn(p, r, 1.0 / 24.0);
    p = __fma_rn(p, r, 1.0 / 6.0);
    p = __fma_rn(p, r, 0.5);
    p = __fma_rn(p, r, 1.0);
    p = __fma_rn(p, r, 1.0);
    const int n = (int)nd;
    if (n > 1023) return (p * 2.0) * __longlong_as_double((long long)(n - 1 + 1023) << 52);
    if (n < -1020) {
        const double sc = p * __longlong_as_double((long long)(n + 600 + 1023) << 52);
        return sc * 0x1p-600;
    }
    return p * __longlong_as_double((long long)(n + 1023) << 52);
}

// sin and cos of 2 pi u: q = rint(4u), f = 4u - q, a = f pi/2, Taylor series
// of sin a through a^17 and cos a through a^18, quadrant by q mod 4.
__device__ __forceinline__ void dsincos2pi(double u, double* so, double* co)
{
    const double t = 4.0 * u;
    const double q = rint(t);
    const double f = t - q;
    const double a = f * 1.57079632679489661923;
    const double z = a * a;
    double sp = -1.0 / 355687428096000.0;
    sp = __fma_rn(sp, z, 1.0 / 1307674368000.0);
    sp = __fma_rn(sp, z, -1.0 / 6227020800.0);
    sp = __fma_rn(sp, z, 1.0 / 39916800.0);
    sp = __fma_rn(sp, z, -1.0 / 362880.0);
    sp = __fma_rn(sp, z, 1.0 / 5040.0);
    sp = __fma_rn(sp, z, -1.0 / 120.0);
    sp = __fma_rn(sp, z, 1.0 / 6.0);
    const double sa = __fma_rn(-a, z * sp, a);
    double cp = 1.0 / 6402373705728000.0;
    cp = __fma_rn(cp, z, -1.0 / 20922789888000.0);
    cp = __fma_rn(cp, z, 1.0 / 87178291200.0);
    cp = __fma_rn(cp, z, -1.0 / 479001600.0);
    cp = __fma_rn(cp, z, 1.0 / 3628800.0);
    cp = __fma_rn(cp, z, -1.0 / 40320.0);
    cp = __fma_rn(cp, z, 1.0 / 720.0);
    cp = __fma_rn(cp, z, -1.0 / 24.0);
    cp = __fma_rn(cp, z, 0.5);
    const double ca = __fma_rn(-z, cp, 1.0);
    switch (((int)q) & 3) {
    case 0: *so = sa; *co = ca; break;
    case 1: *so = ca; *co = -sa; break;
    case 2: *so = -sa; *co = -ca; break;
    default: *so = -ca; *co = sa; break;
    }
}

// ---------------------------------------------------------------- Poisson
// log k!: exact product below 10, Stirling series through k^-7 above.
__device__ __forceinline__ double dlogfact(int64_t k)
{
    if (k < 10) {
        double f = 1.0;
        for (int64_t i = 2; i <= k; ++i) f = f * (double)i;
        return dlog(f);
    }
    const double x = (double)k;
    const double r = 1.0 / x;
    const double r2 = r * r;
    double ser = 1.0 / 1680.0;
    ser = 1.0 / 1260.0 - r2 * ser;
    ser = 1.0 / 360.0 - r2 * ser;
    ser = 1.0 / 12.0 - r2 * ser;
    ser = r * ser;
    return (((x + 0.5) * dlog(x) - x) + 0.91893853320467274178) + ser;
}

// P(mu): 0 without a draw for mu <= 0; inversion by sequential search (one
// uniform) for mu < 10; PTRS transformed rejection (Hoermann 1993, two
// uniforms per trial) above.  Returns -1 if PTRS exhausts its trial limit.
static __device__ __noinline__ int64_t dpoisson(Stream& s, double mu)
{
    if (!(mu > 0.0)) return 0;
    if (mu < 10.0) {
        const double u = s.uniform();
        double p = dexp(-mu);
        double F = p;
        int64_t k = 0;
        while (u > F && k < 200) {
            k += 1;
            p = (p * mu) / (double)k;
            F = F + p;
        }
        return k;
    }
    const double slam = sqrt(mu);
    const double b = 0.931 + 2.53 * slam;
    const double a = -0.059 + 0.02483 * b;
    const double vr = 0.9277 - 3.6224 / (b - 2.0);
    // ln(mu) and 1/alpha serve only the slow test: formed on first use (the
    // same values, so the draws are unchanged)
    double loglam = 0.0, invalpha = 0.0;
    bool slow_ready = false;
    for (int it = 0; it < 1000000; ++it) {
        const double U = s.uniform() - 0.5;
        const double V = s.uniform();
        const double us = 0.5 - fabs(U);
        const double kd = floor(((((2.0 * a) / us) + b) * U + mu) + 0.43);
        if (us >= 0.07 && V <= vr) return (int64_t)kd;
        if (kd < 0.0 || (us < 0.013 && V > us)) continue;
        if (!slow_ready) {
            loglam = dlog(mu);
            invalpha = 1.1239 + 1.1328 / (b - 3.4);
            slow_ready = true;
        }
        // the acceptance test as one logarithm (Hoermann's form)
        const double lhs = dlog((V * invalpha) / ((a / (us * us)) + b));
        const double rhs = ((-mu) + kd * loglam) - dlogfact((int64_t)kd);
        if (lhs <= rhs) return (int64_t)kd;
    }
    return -1;
}

// ---------------------------------------------------------------- grid
__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

// CIC stencil along one axis for an absolute coordinate (FP64 form):
// u = (x - lo)/h - 1/2, i0 = floor(u), f = u - i0, indices folded to [0,n-1].
// (x-lo)/h in grid units: q0 = d r, q = q0 + (d - q0 h) r with r = 1/h (one
// fused correction; the same operations as the specification's).
__device__ __forceinline__ double grid_quot(double x, double lo, double h, double rh)
{
    // x - 0 is x itself (also for -0): a domain corner at 0 (uniform across
    // the launch) needs no subtraction on the FP64 pipe
    double d = x;
    if (__double_as_longlong(lo) != 0) d = x - lo;
    const double q0 = d * rh;
    return __fma_rn(__fma_rn(-q0, h, d), rh, q0);
}

// a / b given r = 1/b, with the same fused correction.
__device__ __forceinline__ double quot_r(double a, double b, double r)
{
    const double q0 = a * r;
    return __fma_rn(__fma_rn(-q0, b, a), r, q0);
}

__device__ __forceinline__ void cic_axis(double x, double lo, double h, double rh, int n, int& ia, int& ib,
                                         double& f)
{
    const double u = grid_quot(x, lo, h, rh) - 0.5;
    const double fl = floor(u);
    const int i0 = (int)fl;
    f = u - fl;
    ia = clampi(i0, n);
    ib = clampi(i0 + 1, n);
}

// Cell of a coordinate known to lie in [lo, hi): floor((x-lo)/h), clamped.
__device__ __forceinline__ int cell_axis(double x, double lo, double h, double rh, int n)
{
    const int i = (int)floor(grid_quot(x, lo, h, rh));
    return i > n - 1 ? n - 1 : (i < 0 ? 0 : i);
}

__device__ __forceinline__ uint64_t seed_of(const Params& P, int r) { return P.seed0 + (uint64_t)r; }
// The step counter of the Philox streams.
__device__ __forceinline__ uint32_t step_of(const Params& P) { return P.step_dev ? *P.step_dev : P.step; }

// Particle block b: species b / R, realization b % R (at most three species:
// two comparisons instead of a division).
__host__ __device__ __forceinline__ int species_of(const Params& P, int b) { return (b >= P.R) + (b >= 2 * P.R); }
__host__ __device__ __forceinline__ int phys_of(const Params& P, int b) { return b - species_of(P, b) * P.R; }

// ---------------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Inclusive segmented sum over runs of equal keys that are contiguous in
// lane order; returns true in the last lane of each run (which then holds
// the run total in v / c).
__device__ __forceinline__ bool warp_run_sum(uint32_t key, bool valid, unsigned long long& v,
                                             unsigned& c)
{
    const unsigned lane = lane_id();
    const unsigned full = 0xffffffffu;
    const uint32_t kprev = __shfl_up_sync(full, key, 1);
    const bool vprev = __shfl_up_sync(full, valid ? 1 : 0, 1);
    const bool head = (lane == 0) || !vprev || kprev != key || !valid;
    const unsigned heads = __ballot_sync(full, head);
    // segment start lane for this lane: highest head at or below lane
    const unsigned below = heads & (0xffffffffu >> (31 - lane));
    const int seg_start = 31 - __clz(below);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long ov = __shfl_up_sync(full, v, d);
        const unsigned oc = __shfl_up_sync(full, c, d);
        if ((int)lane - d >= seg_start) { v += ov; c += oc; }
    }
    const uint32_t knext = __shfl_down_sync(full, key, 1);
    const bool vnext = __shfl_down_sync(full, valid ? 1 : 0, 1);
    const bool tail = (lane == 31) || !vnext || knext != key;
    return valid && tail;
}

}  // namespace ik
