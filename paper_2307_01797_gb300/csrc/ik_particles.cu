// ik_particles.cu -- particle stages of the Ito-KMC step, FP64 form.
//
//   transport (a1-a4): pass 1 interpolates E (Sec. 4.2), pushes every
//     particle by explicit Euler-Maruyama (Sec. 4.3; v = -mu E, Eq. Vk1),
//     computes its new cell, deposits its CIC charge in int64 fixed point
//     (Sec. 4.2) and X_e, and counts per cell; a 3-channel cell scan gives
//     the new cell offsets; pass 2 moves every particle that stayed in its
//     cell straight to its final slot and a small kernel places the few that
//     changed cell.  The result is the stable order (cell, previous index).
//   rho: space charge snapshot and multigrid right-hand side.
//   KMC (a6): one thread per occupied cell, Sec. 3.2.3.
//   particles (a7-a9): loss removal and products (Sec. 4.4, Eq. w), photons
//     (Sec. 4.5, Eq. photon_transport), kd-tree merge/split (Sec. 4.6).
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "ik_common.cuh"
#include "ik_scan.cuh"
#include "ik_state.h"

namespace ik {

namespace {

__device__ __forceinline__ P64 ld_p64(const P64* p)
{
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    P64 r;
    r.x = a.x; r.y = a.y; r.z = b.x;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(b.y);
    r.cell = (uint32_t)bits;
    r.w = (uint32_t)(bits >> 32);
    return r;
}

__device__ __forceinline__ void st_p64(P64* p, const P64& v)
{
    const unsigned long long bits = (unsigned long long)v.cell | ((unsigned long long)v.w << 32);
    reinterpret_cast<double2*>(p)[0] = make_double2(v.x, v.y);
    reinterpret_cast<double2*>(p)[1] = make_double2(v.z, __longlong_as_double((long long)bits));
}

__device__ __forceinline__ E64 ld_e64(const E64* p)
{
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return E64{ a.x, a.y, b.x, b.y };
}

// Trilinear interpolation of the cell-centred field at (x,y,z); sum order z
// outer, y, x inner; weight (wx*wy)*wz.
// Cell quotients qd in [1/2, 2^31) split from their bits.  For such qd the
// stencil coordinate u = qd - 1/2 is exact (1/2 is a multiple of ulp(qd)),
// and so are floor(u), the fraction f = u - floor(u) = F 2^-sh and
// floor(f 2^s) = F >> (sh - s): the FP64 subtract / floor / convert
// sequence yields the same values, and these integer steps keep the FP64
// pipe (a small fraction of the FP32 rate on GB300) for the arithmetic
// that rounds.  qc = floor(qd) is the cell index.
struct QSplit {
    int qc, i0, sh;
    unsigned long long F;
};
__device__ __forceinline__ bool qsplit(double qd, QSplit& r)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(qd);
    const int e = (int)(b >> 52);                  // biased exponent (>= 2048 when negative)
    if (e < 1022 || e > 1053) return false;        // qd < 1/2, qd >= 2^31, negative, NaN
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1075 - e;                       // fraction bits of qd, 22..53
    const unsigned long long fb = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    r.qc = (int)(m >> sh);
    r.sh = sh;
    if (fb >= half) { r.i0 = r.qc; r.F = fb - half; }
    else { r.i0 = r.qc - 1; r.F = fb + half; }
    return true;
}
// F 2^-sh as a double (F < 2^sh, sh <= 53: exact).
__device__ __forceinline__ double qfrac(unsigned long long F, int sh)
{
    if (F == 0) return 0.0;
    const int pb = 63 - __clzll((long long)F);
    const unsigned long long mant = (F << (52 - pb)) & 0xfffffffffffffull;
    return __longlong_as_double((long long)(((unsigned long long)(pb - sh + 1023) << 52) | mant));
}
// cic_axis with the split above (the FP64 steps for qd < 1/2); g = 1 - f,
// exact: 2^sh - F is at most 2^sh, so (2^sh - F) 2^-sh is the same double
// as the FP64 subtraction 1 - f.
__device__ __forceinline__ void cic_axis_q(double x, double lo, double h, double rh, int n, int& ia, int& ib,
                                           double& f, double& g)
{
    const double qd = grid_quot(x, lo, h, rh);
    QSplit t;
    int i0;
    if (qsplit(qd, t)) {
        i0 = t.i0;
        f = qfrac(t.F, t.sh);
        g = t.F == 0 ? 1.0 : qfrac((1ull << t.sh) - t.F, t.sh);
    } else {
        const double u = qd - 0.5;
        const double fl = floor(u);
        i0 = (int)fl;
        f = u - fl;
        g = 1.0 - f;
    }
    ia = clampi(i0, n);
    ib = clampi(i0 + 1, n);
}
// x >= lo and x < hi by order-preserving integer keys (-0 taken as +0; a NaN
// fails one of the two tests, as in the FP64 comparisons).
__device__ __forceinline__ unsigned long long dkey(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    b = b == 0x8000000000000000ull ? 0ull : b;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ void interp_f64(const Params& P, const E64* __restrict__ E, const double X[3],
                                           double Ep[3])
{
    int ia[3], ib[3];
    double f[3], g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) cic_axis_q(X[a], P.lo[a], P.h[a], P.rh[a], P.n, ia[a], ib[a], f[a], g[a]);
    const double wx[2] = { g[0], f[0] }, wy[2] = { g[1], f[1] }, wz[2] = { g[2], f[2] };
    const int ix[2] = { ia[0], ib[0] }, iy[2] = { ia[1], ib[1] }, iz[2] = { ia[2], ib[2] };
    double ax = 0.0, ay = 0.0, az = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const double wgt = (wx[a] * wy[b]) * wz[c];
                const E64 e = ld_e64(E + ((size_t)iz[c] * P.n + iy[b]) * P.n + ix[a]);
                ax = __fma_rn(wgt, e.x, ax);
                ay = __fma_rn(wgt, e.y, ay);
                az = __fma_rn(wgt, e.z, az);
            }
    Ep[0] = ax; Ep[1] = ay; Ep[2] = az;
}

// Int64 CIC deposition of weight w at X into ne (one realization's block).
__device__ __forceinline__ void deposit_f64(const Params& P, unsigned long long* __restrict__ ne,
                                            const double X[3], uint32_t w)
{
    const long long one = 1ll << P.frac_bits;
    const double scale = (double)one;
    int ia[3], ib[3];
    long long A[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double f;
        cic_axis(X[a], P.lo[a], P.h[a], P.rh[a], P.n, ia[a], ib[a], f);
        const long long q = (long long)floor(f * scale);
        A[a][0] = one - q;
        A[a][1] = q;
    }
    const int ix[2] = { ia[0], ib[0] }, iy[2] = { ia[1], ib[1] }, iz[2] = { ia[2], ib[2] };
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const long long v = (long long)w * A[0][a] * A[1][b] * A[2][c];
                if (v) atomicAdd(ne + ((size_t)iz[c] * P.n + iy[b]) * P.n + ix[a], (unsigned long long)v);
            }
}

__device__ __forceinline__ int real_of(const Params& P, uint32_t g) { return (int)(g >> (3 * P.log2n)); }

// Sum over the warp, then one atomic by lane 0 (all lanes must call).
__device__ __forceinline__ void warp_add(unsigned long long* dst, unsigned long long v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// A slot in a shared counter for each calling lane: one atomic per group of
// converged lanes.
__device__ __forceinline__ unsigned long long warp_slot(unsigned long long* ctr)
{
    const unsigned mask = __activemask();
    const int leader = __ffs(mask) - 1;
    const unsigned lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if ((int)lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}
__device__ __forceinline__ unsigned warp_slot32(unsigned* ctr)
{
    const unsigned mask = __activemask();
    const int leader = __ffs(mask) - 1;
    const unsigned lane = threadIdx.x & 31;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(ctr, (unsigned)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// CIC stencil of one particle in fixed point: folded indices and axis
// weights (2^s - a, a).
struct Stencil {
    int ia[3], ib[3];
    uint32_t A[3][2];   // 2^s - a and a (s <= 10: a product of three fits 32 bits)
};

__device__ __forceinline__ void stencil_f32(const Params& P, const int id[3], const float o[3], Stencil& S)
{
    const int one = 1 << P.frac_bits, half = one >> 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int q = (int)floorf(o[a] * (float)one);   // exact: o in [0,1), power-of-two scale
        const int aa = (q + half) & (one - 1);
        const int i0 = id[a] - 1 + (q >= half ? 1 : 0);
        S.ia[a] = clampi(i0, P.n);
        S.ib[a] = clampi(i0 + 1, P.n);
        S.A[a][0] = one - aa;
        S.A[a][1] = aa;
    }
}

constexpr int DEP_WIN = DEP_WIN_MAX;

// Deposits the 8 fixed-point CIC contributions of every alive particle of the
// block.  The cells the block touches usually form a small box (particles are
// sorted by cell), so the contributions are first summed in a shared-memory
// window over that box and flushed with one global atomic per touched cell;
// blocks whose box is too large or spans realizations add directly.  The
// window keeps each 64-bit sum as two 32-bit words updated with native 32-bit
// shared atomics: the low word's atomic returns the old value, from which the
// carry into the high word follows exactly.  Integer sums: the result does
// not depend on the order.  The flush decodes window positions with
// multiplicative inverses ceil(2^32/e) formed once per block (exact for
// positions below 2^16).  SINGLE: one realization (no realization bounds).
// All threads of the block must call this.
template <bool SINGLE>
__device__ __forceinline__ void block_deposit(const Params& P, unsigned long long* __restrict__ ne, bool alive, int r,
                                              const Stencil& S, uint32_t w)
{
    constexpr int NK = SINGLE ? 6 : 8;
    __shared__ uint2 win[DEP_WIN];
    __shared__ int wred[TPB / 32][8];
    __shared__ int wfin[8];
    __shared__ uint32_t wdiv[2];
    const int BIG = 0x7fffffff;
    int v[8];
    if (alive) {
        v[0] = S.ia[0]; v[1] = S.ia[1]; v[2] = S.ia[2];
        v[3] = -S.ib[0]; v[4] = -S.ib[1]; v[5] = -S.ib[2];
        v[6] = r; v[7] = -r;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = BIG;
    }
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NK; ++k) v[k] = __reduce_min_sync(0xffffffffu, v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NK; ++k) wred[wid][k] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
        int m = BIG;
        if (lane < NK)
            for (int q = 0; q < TPB / 32; ++q) m = min(m, wred[q][lane]);
        const int l0 = __shfl_sync(0xffffffffu, m, 0), h0 = __shfl_sync(0xffffffffu, m, 3);
        const int l1 = __shfl_sync(0xffffffffu, m, 1), h1 = __shfl_sync(0xffffffffu, m, 4);
        if (lane < NK) wfin[lane] = m;
        if (lane == 0 && l0 != BIG) {
            const uint32_t e0 = (uint32_t)(-h0 - l0 + 1), e01 = e0 * (uint32_t)(-h1 - l1 + 1);
            wdiv[0] = e0 > 1 ? 0xffffffffu / e0 + 1u : 0u;
            wdiv[1] = e01 > 1 ? 0xffffffffu / e01 + 1u : 0u;
        }
    }
    __syncthreads();
    if (wfin[0] == BIG) return;                       // no alive particle in the block
    const int lo0 = wfin[0], lo1 = wfin[1], lo2 = wfin[2];
    const int e0 = -wfin[3] - lo0 + 1, e1 = -wfin[4] - lo1 + 1, e2 = -wfin[5] - lo2 + 1;
    const long long V = (long long)e0 * e1 * e2;
    const bool use = (SINGLE || wfin[6] == -wfin[7]) && V <= P.dep_win;
    const int ix[2] = { S.ia[0], S.ib[0] }, iy[2] = { S.ia[1], S.ib[1] }, iz[2] = { S.ia[2], S.ib[2] };
    if (!use) {
        if (alive) {
            unsigned long long* base = ne + (size_t)r * P.n3;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        const unsigned long long val = (unsigned long long)w * (S.A[0][a] * S.A[1][b] * S.A[2][c]);
                        if (val) atomicAdd(base + ((size_t)iz[c] * P.n + iy[b]) * P.n + ix[a], val);
                    }
        }
        return;
    }
    for (int t = threadIdx.x; t < (int)V; t += TPB) win[t] = make_uint2(0u, 0u);
    __syncthreads();
    if (alive) {
        uint32_t* wl = reinterpret_cast<uint32_t*>(win);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const unsigned long long val = (unsigned long long)w * (S.A[0][a] * S.A[1][b] * S.A[2][c]);
                    if (val) {
                        const int k = ((iz[c] - lo2) * e1 + (iy[b] - lo1)) * e0 + (ix[a] - lo0);
                        const uint32_t lo = (uint32_t)val;
                        const uint32_t old = atomicAdd(wl + 2 * k, lo);
                        const uint32_t hc = (uint32_t)(val >> 32) + (old + lo < old ? 1u : 0u);
                        if (hc) atomicAdd(wl + 2 * k + 1, hc);
                    }
                }
    }
    __syncthreads();
    const int rb = SINGLE ? 0 : wfin[6];
    unsigned long long* base = ne + (size_t)rb * P.n3 + ((size_t)lo2 * P.n + lo1) * P.n + lo0;
    const uint32_t m0 = wdiv[0], m01 = wdiv[1];
    const uint32_t e01 = (uint32_t)(e0 * e1);
    for (int t = threadIdx.x; t < (int)V; t += TPB) {
        const uint2 q = win[t];
        const unsigned long long val = ((unsigned long long)q.y << 32) | q.x;
        if (val) {
            const uint32_t zq = e01 > 1 ? __umulhi((uint32_t)t, m01) : (uint32_t)t;
            const uint32_t rem = (uint32_t)t - zq * e01;
            const uint32_t yq = e0 > 1 ? __umulhi(rem, m0) : rem;
            const uint32_t xq = rem - yq * (uint32_t)e0;
            atomicAdd(base + ((size_t)zq * P.n + yq) * P.n + xq, val);
        }
    }
}

// ------------------------------------------------------------------ normals
// Standard normals by the ziggurat method (Marsaglia & Tsang, J. Stat.
// Softw. 5(8), 2000), 128 layers, base strip r = 3.442619855899,
// v = 9.91256303526217e-3, 53-bit magnitudes: an attempt takes two words
// U = a 2^32 + b: layer i = U mod 128, sign bit 7, magnitude m = U >> 11;
// x = m W_i is accepted at once if m < K_i, else through the tail (i = 0) or
// the wedge test.  The tables follow the paper's setup recurrence with the
// library's ln/exp and IEEE sqrt (computed once per device by k_zig_init).
// The FP32 form takes the same words and the same integer decisions, and
// its rare paths use FP32 uniforms from the high words.
__device__ double g_zig_w[128], g_zig_f[128];
__device__ unsigned long long g_zig_k[128];
__device__ float g_zig_w32[128], g_zig_f32[128];   // W_i 2^29 (for the top 24 magnitude bits), F_i

constexpr double ZIG_R = 3.442619855899, ZIG_V = 9.91256303526217e-3, ZIG_M = 9007199254740992.0;

__global__ void k_zig_init()
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double q = ZIG_V / dexp(-0.5 * ZIG_R * ZIG_R);
    g_zig_k[0] = (unsigned long long)((ZIG_R / q) * ZIG_M);
    g_zig_k[1] = 0;
    g_zig_w[0] = q / ZIG_M;
    g_zig_w[127] = ZIG_R / ZIG_M;
    g_zig_f[0] = 1.0;
    g_zig_f[127] = dexp(-0.5 * ZIG_R * ZIG_R);
    double d = ZIG_R, t = ZIG_R;
    for (int i = 126; i >= 1; --i) {
        d = sqrt(-2.0 * dlog(ZIG_V / d + dexp(-0.5 * d * d)));
        g_zig_k[i + 1] = (unsigned long long)((d / t) * ZIG_M);
        t = d;
        g_zig_f[i] = dexp(-0.5 * d * d);
        g_zig_w[i] = d / ZIG_M;
    }
    for (int i = 0; i < 128; ++i) {
        g_zig_w32[i] = (float)(g_zig_w[i] * 536870912.0);   // 2^29
        g_zig_f32[i] = (float)g_zig_f[i];
    }
}

// m < 2^53 as a double, assembled from its bits (exact).
__device__ __forceinline__ double u53_exact(unsigned long long m)
{
    if (m == 0) return 0.0;
    const int p = 63 - __clzll((long long)m);
    const unsigned long long bits = ((unsigned long long)(p + 1023) << 52) | ((m << (52 - p)) & 0x000fffffffffffffull);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double znormal(PairStream& s)
{
    for (int attempt = 0; attempt < 64; ++attempt) {
        uint32_t a, b;
        s.pair(a, b);
        const unsigned long long U = ((unsigned long long)a << 32) | b;
        const int i = (int)(U & 127u);
        const bool neg = (U >> 7) & 1u;
        const unsigned long long m = U >> 11;
        const double x = u53_exact(m) * __ldg(g_zig_w + i);
        if (m < __ldg(g_zig_k + i)) return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
        if (i == 0) {
            double xt, y;
            int tries = 0;
            do {
                xt = -dlog(s.uniform()) / ZIG_R;
                y = -dlog(s.uniform());
            } while (y + y < xt * xt && ++tries < 64);
            const double v = ZIG_R + xt;
            return neg ? -v : v;
        }
        const double u = s.uniform();
        const double fi = __ldg(g_zig_f + i), fm = __ldg(g_zig_f + i - 1);
        if (fi + u * (fm - fi) < dexp(-0.5 * x * x)) return neg ? -x : x;
    }
    return 0.0;
}

__device__ __forceinline__ float znormal32(PairStream& s)
{
    for (int attempt = 0; attempt < 64; ++attempt) {
        uint32_t a, b;
        s.pair(a, b);
        const unsigned long long U = ((unsigned long long)a << 32) | b;
        const int i = (int)(U & 127u);
        const bool neg = (U >> 7) & 1u;
        const unsigned long long m = U >> 11;
        // the top 24 bits of the 53-bit magnitude: an exact 32-bit conversion
        const float x = __uint2float_rn((uint32_t)(m >> 29)) * __ldg(g_zig_w32 + i);
        if (m < __ldg(g_zig_k + i)) return neg ? -x : x;
        if (i == 0) {
            float xt, y;
            int tries = 0;
            do {
                xt = -logf(s.uniform32()) / (float)ZIG_R;
                y = -logf(s.uniform32());
            } while (y + y < xt * xt && ++tries < 64);
            const float v = (float)ZIG_R + xt;
            return neg ? -v : v;
        }
        const float u = s.uniform32();
        const float fi = __ldg(g_zig_f32 + i), fm = __ldg(g_zig_f32 + i - 1);
        if (fi + u * (fm - fi) < expf(-0.5f * x * x)) return neg ? -x : x;
    }
    return 0.f;
}

// ------------------------------------------------------------------ pass 1
__global__ void __launch_bounds__(TPB, 4) k_push_f64(
    Params P, const P64* __restrict__ A, P64* __restrict__ B, uint32_t* __restrict__ keyB, uint32_t N,
    const uint32_t* __restrict__ cell_start, const E64* __restrict__ E, int32_t* __restrict__ cnt_new,
    int32_t* __restrict__ in_cnt, int32_t* __restrict__ in_before, unsigned long long* __restrict__ Xe,
    unsigned long long* __restrict__ ne_fix, Mover* __restrict__ movers, uint32_t mover_cap,
    Counters* __restrict__ ctr, uint32_t* __restrict__ blk_stay, const uint32_t* __restrict__ Ndev)
{
    if (Ndev) N = *Ndev;                          // graph-replayed steps: the count of the current step
    const uint32_t i = blockIdx.x * TPB + threadIdx.x;
    bool alive = false, mover = false;
    uint32_t gnew = 0, w = 0;
    int rr = 0;
    Stencil S;
    if (i < N) {
        const P64 p = ld_p64(A + i);
        const uint32_t gold = p.cell;
        const int r = real_of(P, gold);              // particle block: species r / R, realization r % R
        rr = r;
        const int sp = species_of(P, r), rp = phys_of(P, r);
        const uint32_t idx = i - cell_start[(size_t)r * P.n3];
        const size_t ebase = (size_t)r * P.n3;
        w = p.w;
        const double X[3] = { p.x, p.y, p.z };
        double Ep[3];
        interp_f64(P, E + (size_t)rp * P.n3, X, Ep);
        PairStream s(seed_of(P, rp), idx, step_of(P), P.push_tag_sp[sp], 0);
        double Nn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) Nn[a] = znormal(s);
        const double nmu = P.cmu_sp[sp], sdt = P.sdt_sp[sp];   // electrons: -mu, sqrt(2 D dt)
        double Xn[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Xn[a] = (X[a] + (nmu * Ep[a]) * P.dt) + sdt * Nn[a];
            const unsigned long long kx = dkey(Xn[a]);
            inside = inside && kx >= dkey(P.lo[a]) && kx < dkey(P.hi[a]);
        }
        P64 q;
        q.x = Xn[0]; q.y = Xn[1]; q.z = Xn[2]; q.w = w;
        if (inside) {
            // one division per axis serves the cell index and the stencil
            int ic[3];
            const long long one = 1ll << P.frac_bits;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double qd = grid_quot(Xn[a], P.lo[a], P.h[a], P.rh[a]);
                QSplit t;
                int ci, i0;
                long long fq;
                if (qsplit(qd, t)) {
                    ci = t.qc;
                    i0 = t.i0;
                    fq = (long long)(t.F >> (t.sh - P.frac_bits));
                } else {
                    ci = (int)floor(qd);
                    const double u = qd - 0.5;
                    const double fl = floor(u);
                    i0 = (int)fl;
                    fq = (long long)floor((u - fl) * (double)one);
                }
                ic[a] = ci > P.n - 1 ? P.n - 1 : (ci < 0 ? 0 : ci);
                S.ia[a] = clampi(i0, P.n);
                S.ib[a] = clampi(i0 + 1, P.n);
                S.A[a][0] = (uint32_t)(one - fq);
                S.A[a][1] = (uint32_t)fq;
            }
            gnew = (uint32_t)(ebase + ((size_t)ic[2] * P.n + ic[1]) * P.n + ic[0]);
            alive = true;
            mover = gnew != gold;
            q.cell = gnew;
            keyB[i] = gnew | (mover ? KEY_MOVER : 0u);
            if (mover) {
                atomicAdd(in_cnt + gnew, 1);
                if (gold < gnew) atomicAdd(in_before + gnew, 1);
                const unsigned long long slot = warp_slot(&ctr->n_movers);
                if (slot < mover_cap) movers[slot] = Mover{ gnew, i };
                else atomicOr(&ctr->err, DERR_CAPACITY);
            }
        } else {
            q.cell = gold;
            keyB[i] = KEY_DEAD;
            atomicAdd(&ctr->outflow[r], (unsigned long long)w);
        }
        st_p64(B + i, q);
    }
    block_deposit<false>(P, ne_fix, alive, rr, S, w);
    unsigned long long v = alive ? (unsigned long long)w : 0ull;
    unsigned c = alive ? 1u : 0u;
    if (warp_run_sum(gnew, alive, v, c)) {
        atomicAdd(cnt_new + gnew, (int)c);
        atomicAdd(Xe + gnew, v);
    }
    const int nstay = __syncthreads_count(alive && !mover);
    if (threadIdx.x == 0) blk_stay[blockIdx.x] = (uint32_t)nstay;
}

// The advective substep of the semi-implicit transport (Sec. 4.3, Eq.
// particle_kernel), otherwise the FP64 push: B holds the diffused positions
// X+ on entry; the field (of the end of the step) is interpolated at the
// positions X of A and the particle moves from X+ by V dt, no normals drawn.
__global__ void __launch_bounds__(TPB, 4) k_advect_f64(
    Params P, const P64* __restrict__ A, P64* __restrict__ B, uint32_t* __restrict__ keyB, uint32_t N,
    const uint32_t* __restrict__ cell_start, const E64* __restrict__ E, int32_t* __restrict__ cnt_new,
    int32_t* __restrict__ in_cnt, int32_t* __restrict__ in_before, unsigned long long* __restrict__ Xe,
    unsigned long long* __restrict__ ne_fix, Mover* __restrict__ movers, uint32_t mover_cap,
    Counters* __restrict__ ctr, uint32_t* __restrict__ blk_stay)
{
    const uint32_t i = blockIdx.x * TPB + threadIdx.x;
    bool alive = false, mover = false;
    uint32_t gnew = 0, w = 0;
    int rr = 0;
    Stencil S;
    if (i < N) {
        const P64 p = ld_p64(A + i);
        const uint32_t gold = p.cell;
        const int r = real_of(P, gold);
        rr = r;
        const size_t ebase = (size_t)r * P.n3;
        w = p.w;
        const double X[3] = { p.x, p.y, p.z };
        double Ep[3];
        interp_f64(P, E + ebase, X, Ep);
        const P64 pd = ld_p64(B + i);
        const double Xd[3] = { pd.x, pd.y, pd.z };
        const double nmu = -P.mu;
        double Xn[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Xn[a] = Xd[a] + (nmu * Ep[a]) * P.dt;
            const unsigned long long kx = dkey(Xn[a]);
            inside = inside && kx >= dkey(P.lo[a]) && kx < dkey(P.hi[a]);
        }
        P64 q;
        q.x = Xn[0]; q.y = Xn[1]; q.z = Xn[2]; q.w = w;
        if (inside) {
            // one division per axis serves the cell index and the stencil
            int ic[3];
            const long long one = 1ll << P.frac_bits;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double qd = grid_quot(Xn[a], P.lo[a], P.h[a], P.rh[a]);
                QSplit t;
                int ci, i0;
                long long fq;
                if (qsplit(qd, t)) {
                    ci = t.qc;
                    i0 = t.i0;
                    fq = (long long)(t.F >> (t.sh - P.frac_bits));
                } else {
                    ci = (int)floor(qd);
                    const double u = qd - 0.5;
                    const double fl = floor(u);
                    i0 = (int)fl;
                    fq = (long long)floor((u - fl) * (double)one);
                }
                ic[a] = ci > P.n - 1 ? P.n - 1 : (ci < 0 ? 0 : ci);
                S.ia[a] = clampi(i0, P.n);
                S.ib[a] = clampi(i0 + 1, P.n);
                S.A[a][0] = (uint32_t)(one - fq);
                S.A[a][1] = (uint32_t)fq;
            }
            gnew = (uint32_t)(ebase + ((size_t)ic[2] * P.n + ic[1]) * P.n + ic[0]);
            alive = true;
            mover = gnew != gold;
            q.cell = gnew;
            keyB[i] = gnew | (mover ? KEY_MOVER : 0u);
            if (mover) {
                atomicAdd(in_cnt + gnew, 1);
                if (gold < gnew) atomicAdd(in_before + gnew, 1);
                const unsigned long long slot = warp_slot(&ctr->n_movers);
                if (slot < mover_cap) movers[slot] = Mover{ gnew, i };
                else atomicOr(&ctr->err, DERR_CAPACITY);
            }
        } else {
            q.cell = gold;
            keyB[i] = KEY_DEAD;
            atomicAdd(&ctr->outflow[r], (unsigned long long)w);
        }
        st_p64(B + i, q);
    }
    block_deposit<false>(P, ne_fix, alive, rr, S, w);
    unsigned long long v = alive ? (unsigned long long)w : 0ull;
    unsigned c = alive ? 1u : 0u;
    if (warp_run_sum(gnew, alive, v, c)) {
        atomicAdd(cnt_new + gnew, (int)c);
        atomicAdd(Xe + gnew, v);
    }
    const int nstay = __syncthreads_count(alive && !mover);
    if (threadIdx.x == 0) blk_stay[blockIdx.x] = (uint32_t)nstay;
}

// Exclusive scan over the pass-1 blocks of their stayer counts.
struct BlockScanOp {
    const uint32_t* blk;
    uint32_t* prefix;
    __device__ void load(uint64_t g, long long v[1]) const { v[0] = blk[g]; }
    __device__ void store(uint64_t g, const long long ex[1], const long long*) const { prefix[g] = (uint32_t)ex[0]; }
    __device__ void total(const long long*) const {}
};

// Cell scan: new offsets, stayer offsets, mover offsets.
struct TransportScanOp {
    const int32_t* cnt_new;
    const int32_t* in_cnt;
    const int32_t* in_before;
    uint32_t* new_start;
    int64_t* delta;
    uint32_t* in_off;
    uint64_t G;
    __device__ void load(uint64_t g, long long v[3]) const
    {
        const int cn = cnt_new[g], ic = in_cnt[g];
        v[0] = cn; v[1] = cn - ic; v[2] = ic;
    }
    __device__ void store(uint64_t g, const long long ex[3], const long long*) const
    {
        new_start[g] = (uint32_t)ex[0];
        delta[g] = ex[0] + in_before[g] - ex[1];
        in_off[g] = (uint32_t)ex[2];
    }
    __device__ void total(const long long t[3]) const
    {
        new_start[G] = (uint32_t)t[0];
        in_off[G] = (uint32_t)t[2];
    }
};

// ------------------------------------------------------------------ pass 2
__device__ __forceinline__ uint32_t block_excl_count(bool flag, uint32_t* total)
{
    __shared__ uint32_t wcnt[TPB / 32];
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    const uint32_t within = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wcnt[wid] = __popc(bal);
    __syncthreads();
    uint32_t pre = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < TPB / 32; ++k) {
        if (k < (int)wid) pre += wcnt[k];
        tot += wcnt[k];
    }
    if (total) *total = tot;
    return pre + within;
}

__global__ void __launch_bounds__(TPB) k_scatter_f64(const P64* __restrict__ B, P64* __restrict__ A,
                                                     const uint32_t* __restrict__ keyB, uint32_t N,
                                                     const uint32_t* __restrict__ blk_prefix,
                                                     const int64_t* __restrict__ delta, uint32_t cap,
                                                     Counters* __restrict__ ctr, const uint32_t* __restrict__ Ndev)
{
    if (Ndev) N = *Ndev;
    const uint32_t i = blockIdx.x * TPB + threadIdx.x;
    uint32_t k = KEY_DEAD;
    if (i < N) k = keyB[i];
    const bool stay = !(k & (KEY_DEAD | KEY_MOVER));
    const uint32_t rank = block_excl_count(stay, nullptr);
    if (stay) {
        const uint32_t g = k & KEY_MASK;
        const long long pos = (long long)blk_prefix[blockIdx.x] + rank + delta[g];
        if (pos >= 0 && pos < (long long)cap) st_p64(A + pos, ld_p64(B + i));
        else atomicOr(&ctr->err, DERR_INTERNAL);
    }
}

__global__ void k_mover_place(const Mover* __restrict__ movers, const Counters* __restrict__ ctr,
                              uint32_t mover_cap, const uint32_t* __restrict__ in_off,
                              int32_t* __restrict__ cursor, uint32_t* __restrict__ sorted)
{
    const uint32_t n = (uint32_t)min(ctr->n_movers, (unsigned long long)mover_cap);
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        const uint32_t g = movers[m].g;
        const uint32_t slot = in_off[g] + (uint32_t)atomicAdd(cursor + g, 1);
        if (slot < mover_cap) sorted[slot] = m;
    }
}

__global__ void k_mover_write_f64(const Mover* __restrict__ movers, const Counters* __restrict__ ctr,
                                  uint32_t mover_cap, const uint32_t* __restrict__ sorted,
                                  const uint32_t* __restrict__ in_off, const int32_t* __restrict__ in_cnt,
                                  const int32_t* __restrict__ in_before, const int32_t* __restrict__ cnt_new,
                                  const uint32_t* __restrict__ new_start, int32_t* __restrict__ cursor,
                                  const P64* __restrict__ B, P64* __restrict__ A)
{
    const uint32_t n = (uint32_t)min(ctr->n_movers, (unsigned long long)mover_cap);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const Mover mv = movers[sorted[s]];
        const uint32_t g = mv.g;
        const uint32_t b = in_off[g], e = b + (uint32_t)in_cnt[g];
        uint32_t rank = 0;
        for (uint32_t t = b; t < e && t < mover_cap; ++t) rank += movers[sorted[t]].i < mv.i;
        const uint32_t stay = (uint32_t)(cnt_new[g] - in_cnt[g]);
        const uint32_t pos = new_start[g] + rank + (rank >= (uint32_t)in_before[g] ? stay : 0u);
        if (pos < mover_cap && e <= mover_cap) st_p64(A + pos, ld_p64(B + mv.i));
        cursor[g] = 0;
    }
}

// ------------------------------------------------------------------ deposit only
__global__ void __launch_bounds__(TPB) k_deposit_f64(Params P, const P64* __restrict__ A, uint32_t N,
                                                     unsigned long long* __restrict__ Xe,
                                                     unsigned long long* __restrict__ ne_fix)
{
    const uint32_t i = blockIdx.x * TPB + threadIdx.x;
    bool alive = i < N;
    uint32_t g = 0, w = 0;
    if (alive) {
        const P64 p = ld_p64(A + i);
        g = p.cell;
        w = p.w;
        const double X[3] = { p.x, p.y, p.z };
        deposit_f64(P, ne_fix + (size_t)real_of(P, g) * P.n3, X, w);
    }
    unsigned long long v = alive ? (unsigned long long)w : 0ull;
    unsigned c = alive ? 1u : 0u;
    if (warp_run_sum(g, alive, v, c)) atomicAdd(Xe + g, v);
}

// ------------------------------------------------------------------ rho
// rho_fixed = 2^3s (N+ - N-) - ne_fix (units q_e 2^-3s per cell), its
// maximum modulus, and (rhs != nullptr) the FP64 multigrid right-hand side
// h^2 b, b = -rho/eps0 with the electrode potentials folded in (ghost
// 2 phi_b - phi_1 at z faces: -2 phi_b / h^2).
__global__ void k_rho(Params P, const int64_t* __restrict__ Npos, const int64_t* __restrict__ Nneg,
                      const unsigned long long* __restrict__ ne_fix, int64_t* __restrict__ rho,
                      double* __restrict__ rhs, uint64_t G, double qscale, double bc_top, double h2,
                      Counters* __restrict__ ctr)
{
    unsigned long long amax = 0;
    const bool mobile = P.S == 3;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < G; g += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long ne = ne_fix[g];
        long long rf;
        if (mobile) {
            // mobile ions: the CIC densities of the ion blocks, same units
            const unsigned long long np_ = ne_fix[G + g], nn_ = ne_fix[2 * G + g];
            if (ne >= (1ull << 62) || np_ >= (1ull << 62) || nn_ >= (1ull << 62)) atomicOr(&ctr->err, DERR_OVERFLOW);
            rf = ((long long)np_ - (long long)nn_) - (long long)ne;
        } else {
            const long long dq = Npos[g] - Nneg[g];
            const long long lim = 1ll << (62 - 3 * P.frac_bits);
            if (dq >= lim || dq <= -lim || ne >= (1ull << 62)) atomicOr(&ctr->err, DERR_OVERFLOW);
            rf = dq * (1ll << (3 * P.frac_bits)) - (long long)ne;
        }
        rho[g] = rf;
        const unsigned long long a = (unsigned long long)(rf < 0 ? -rf : rf);
        amax = a > amax ? a : amax;
        if (rhs) {
            const int k = (int)((g >> (2 * P.log2n)) & (uint64_t)(P.n - 1));
            double b = -((double)rf * qscale);
            if (k == P.n - 1) b = b - bc_top;
            rhs[g] = b * h2;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, amax, d);
        amax = o > amax ? o : amax;
    }
    if ((threadIdx.x & 31) == 0 && amax) atomicMax(&ctr->rho_absmax, amax);
}

// ------------------------------------------------------------------ KMC
// Sec. 3.2.3 for the network {e -> 2e + M+, e -> M-, e -> e + gamma}; the
// SSA switch is tested before the critical draw (Cao et al. 2006).  T is the
// arithmetic of the propensities, times and leaps: double (FP64 form, the
// specification's operation order) or float (mixed form; a float uniform is the top 23
// bits of the same stream's FP64 uniform, so both forms draw common random
// numbers; Poisson means at or above 2^22 are drawn in FP64).
template <class T> struct KT;
template <> struct KT<double> {
    static __device__ __forceinline__ double uni(Stream& s) { return s.uniform(); }
    static __device__ __forceinline__ double lg(double x) { return dlog(x); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    static __device__ __forceinline__ long long poisson(Stream& s, double mu) { return dpoisson(s, mu); }
};
template <> struct KT<float> {
    static __device__ __forceinline__ float uni(Stream& s)
    {
        const uint32_t a = s.u32();
        (void)s.u32();
        return uniform_f32(a);
    }
    static __device__ __forceinline__ float lg(float x) { return logf(x); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
    static __device__ long long poisson(Stream& s, float mu);
};

// FP32 Poisson: inversion below 10, PTRS (Hoermann 1993) up to 2^22, FP64 above.
__device__ long long KT<float>::poisson(Stream& s, float mu)
{
    if (!(mu > 0.0f)) return 0;
    if (mu >= 4194304.0f) return dpoisson(s, (double)mu);
    if (mu < 10.0f) {
        const float u = uni(s);
        float p = expf(-mu);
        float F = p;
        long long k = 0;
        while (u > F && k < 200) {
            k += 1;
            p = (p * mu) / (float)k;
            F = F + p;
        }
        return k;
    }
    const float slam = sqrtf(mu);
    const float loglam = logf(mu);
    const float b = 0.931f + 2.53f * slam;
    const float a = -0.059f + 0.02483f * b;
    const float invalpha = 1.1239f + 1.1328f / (b - 3.4f);
    const float vr = 0.9277f - 3.6224f / (b - 2.0f);
    for (int it = 0; it < 1000000; ++it) {
        const float U = uni(s) - 0.5f;
        const float V = uni(s);
        const float us = 0.5f - fabsf(U);
        const float kd = floorf(((((2.0f * a) / us) + b) * U + mu) + 0.43f);
        if (us >= 0.07f && V <= vr) return (long long)kd;
        if (kd < 0.0f || (us < 0.013f && V > us)) continue;
        const float lhs = logf((V * invalpha) / ((a / (us * us)) + b));
        const float rhs = ((-mu) + kd * loglam) - lgammaf(kd + 1.0f);
        if (lhs <= rhs) return (long long)kd;
    }
    return -1;
}

// Per-cell hybrid tau-leap/SSA of Cao et al. (2006), Sec. 3.2.3, over the
// counts X = (X_e, X_+, X_-) and the five reactions of Sec. 5.1's air table:
//   r=0 ionization      a = k_alpha X_e        nu = (+1, +1,  0)
//   r=1 attachment      a = k_eta X_e          nu = (-1,  0, +1)
//   r=2 photon emission a = k_gamma X_e        nu = ( 0,  0,  0)
//   r=3 e-ion recomb.   a = k_ep X_e X_+       nu = (-1, -1,  0)
//   r=4 ion-ion recomb. a = k_np X_+ X_-       nu = ( 0, -1, -1)
// A reaction is critical when it is within N_c firings of exhausting a
// reactant; the non-critical step bound takes eps X_i / g_i over the
// reactant species of the non-critical reactions, g_i = 2 for a reactant of
// a second-order reaction with a positive coefficient; the SSA switch
// (A dtau <= 1) is tested before the critical time is drawn; a substep that
// leaves a count negative is redone with half the step.  Sums are taken in
// reaction order and each operation rounds once (-fmad=false), so the FP64
// form is one fixed evaluation of these steps.
__device__ __forceinline__ int kmc_nu(int r, int i)
{
    // compile-time after unrolling: the stoichiometry table above
    return i == 0 ? (r == 0) - (r == 1) - (r == 3) : (i == 1 ? (r == 0) - (r == 3) - (r == 4) : (r == 1) - (r == 4));
}

// REC = false compiles the first-order network alone (reactions 0-2, only
// X_e enters): the same results as REC = true with k_ep = k_np = 0, whose
// extra terms are exact zeros, without their cost.
template <class T, bool REC>
__device__ __forceinline__ void kmc_props(const T kr[5], const long long X[3], T a[5])
{
    const T xe = (T)X[0];
    a[0] = kr[0] * xe;
    a[1] = kr[1] * xe;
    a[2] = kr[2] * xe;
    if constexpr (REC) {
        const T xp = (T)X[1], xm = (T)X[2];
        a[3] = (kr[3] * xe) * xp;
        a[4] = (kr[4] * xp) * xm;
    } else {
        a[3] = a[4] = (T)0;
    }
}

template <class T, bool REC>
__device__ T kmc_total(const T a[5])
{
    const T A = (a[0] + a[1]) + a[2];
    if constexpr (REC) return (A + a[3]) + a[4];
    return A;
}

template <class T, bool REC>
__device__ int kmc_cell(const Params& P, Stream& s, const long long X0[3], const T kr[5], long long fired[5])
{
    using K = KT<T>;
    constexpr int NR = REC ? 5 : 3;          // reactions that can fire
    constexpr int NS = REC ? 3 : 1;          // species that enter a propensity
    long long X[3] = { X0[0], X0[1], X0[2] };
    const T dt = (T)P.dt;
    const long long nc = (long long)P.n_crit;
    T tau = (T)0;
    const bool g2[3] = { REC && kr[3] > (T)0, REC && (kr[3] > (T)0 || kr[4] > (T)0), REC && kr[4] > (T)0 };
#pragma unroll
    for (int r = 0; r < 5; ++r) fired[r] = 0;
    for (int guard = 0; guard < 100000; ++guard) {
        if (!(tau < dt)) return 0;
        T a[5];
        kmc_props<T, REC>(kr, X, a);
        const T A = kmc_total<T, REC>(a);
        if (!(A > (T)0)) return 0;
        bool crit[5] = { false, a[1] > (T)0 && X[0] < nc, false, false, false };
        if constexpr (REC) {
            const long long L3 = X[0] < X[1] ? X[0] : X[1], L4 = X[1] < X[2] ? X[1] : X[2];
            crit[3] = a[3] > (T)0 && L3 < nc;
            crit[4] = a[4] > (T)0 && L4 < nc;
        }
        T Ac = (T)0;
#pragma unroll
        for (int r = 0; r < NR; ++r) if (crit[r]) Ac = Ac + a[r];
        T dtnc = K::inf();
        if (!isinf(P.eps)) {
            const bool reactant[3] = { true, REC && ((!crit[3] && kr[3] > (T)0) || (!crit[4] && kr[4] > (T)0)),
                                       REC && !crit[4] && kr[4] > (T)0 };
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                if (!reactant[i]) continue;
                T xi = (T)0, sig2 = (T)0;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (crit[r]) continue;
                    xi = xi + (T)kmc_nu(r, i) * a[r];
                    sig2 = sig2 + (T)(kmc_nu(r, i) * kmc_nu(r, i)) * a[r];
                }
                T num = (T)P.eps * (T)X[i];
                if (g2[i]) num = num * (T)0.5;          // num / g_i, exact for g_i = 2
                if (num < (T)1) num = (T)1;
                const T t1 = (xi != (T)0) ? num / (xi < (T)0 ? -xi : xi) : K::inf();
                const T t2 = (sig2 != (T)0) ? (num * num) / sig2 : K::inf();
                const T ti = t1 < t2 ? t1 : t2;
                if (ti < dtnc) dtnc = ti;
            }
        }
        T dtc = (T)-1;
        bool accepted = false;
        for (int rej = 0; rej < 10000 && !accepted; ++rej) {
            const T rem = dt - tau;
            T dtau = dtnc < rem ? dtnc : rem;
            long long k[5] = { 0, 0, 0, 0, 0 };
            T adv;
            if (A * dtau <= (T)1) {
                long long Xs[3] = { X[0], X[1], X[2] };
                T t = (T)0;
                for (int ev = 0; ev < P.n_ssa; ++ev) {
                    T as[5];
                    kmc_props<T, REC>(kr, Xs, as);
                    const T As = kmc_total<T, REC>(as);
                    if (!(As > (T)0)) { t = dtau; break; }
                    const T dte = (-K::lg(K::uni(s))) / As;
                    if (t + dte > dtau) { t = dtau; break; }
                    t = t + dte;
                    const T target = K::uni(s) * As;
                    T cum = (T)0;
                    int j = (REC && (as[3] > (T)0 || as[4] > (T)0)) ? (as[4] > (T)0 ? 4 : 3) : 2;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        cum = cum + as[r];
                        if (cum > target) { j = r; break; }
                    }
#pragma unroll
                    for (int r = 0; r < NR; ++r) k[r] += (j == r);
                    Xs[0] += (j == 0) - (j == 1) - (j == 3);
                    if constexpr (REC) {
                        Xs[1] += (j == 0) - (j == 3) - (j == 4);
                        Xs[2] += (j == 1) - (j == 4);
                    }
                }
                adv = t;
            } else {
                if (dtc < (T)0) dtc = (Ac > (T)0) ? (-K::lg(K::uni(s))) / Ac : K::inf();
                if (dtc < dtnc && dtc < rem) {
                    dtau = dtc;
                    const T target = K::uni(s) * Ac;
                    T cum = (T)0;
                    int rc = -1, last = -1;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        if (!crit[r]) continue;
                        last = r;
                        cum = cum + a[r];
                        if (cum > target) { rc = r; break; }
                    }
                    if (rc < 0) rc = last;
#pragma unroll
                    for (int r = 0; r < NR; ++r) k[r] += (rc == r);
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    if (crit[r]) continue;
                    const long long kk = K::poisson(s, a[r] * dtau);
                    if (kk < 0) return -1;
                    k[r] += kk;
                }
                adv = dtau;
            }
            const long long Xn0 = X[0] + k[0] - k[1] - k[3];
            if (Xn0 < 0) {
                dtnc = dtau * (T)0.5;
                continue;
            }
            if constexpr (REC) {
                const long long Xn1 = X[1] + k[0] - k[3] - k[4];
                const long long Xn2 = X[2] + k[1] - k[4];
                if (Xn1 < 0 || Xn2 < 0) {
                    dtnc = dtau * (T)0.5;
                    continue;
                }
                X[1] = Xn1; X[2] = Xn2;
            }
            X[0] = Xn0;
#pragma unroll
            for (int r = 0; r < NR; ++r) fired[r] += k[r];
            if (adv >= rem) tau = dt; else tau = tau + adv;
            accepted = true;
        }
        if (!accepted) return -1;
    }
    return -1;
}

// Cells with electrons -- or, with ion-ion recombination on, ions of both
// signs -- listed for the KMC (one thread per listed cell keeps the warps'
// lanes busy: the active cells are a small part of the grid); the other
// cells fire nothing.  The recombination blocks of the firings are touched
// only when their reaction is on.
// The ion counts of cell g: the NGP counts of the ion blocks' last deposit
// (mobile ions), else the per-cell counts.
__device__ __forceinline__ void ion_counts(const Params& P, const unsigned long long* __restrict__ Xe,
                                           const int64_t* __restrict__ Npos, const int64_t* __restrict__ Nneg,
                                           uint64_t G, uint64_t g, long long& xp, long long& xm)
{
    if (P.S == 3) { xp = (long long)Xe[G + g]; xm = (long long)Xe[2 * G + g]; }
    else { xp = (long long)Npos[g]; xm = (long long)Nneg[g]; }
}

__global__ void k_kmc_list(Params P, const unsigned long long* __restrict__ Xe, const int64_t* __restrict__ Npos,
                           const int64_t* __restrict__ Nneg, int64_t* __restrict__ fired,
                           int64_t* __restrict__ gain, uint64_t G, uint32_t* __restrict__ list,
                           Counters* __restrict__ ctr)
{
    const bool rec = P.k_ep > 0.0 || P.k_np > 0.0;
    const bool ion_only = P.k_np > 0.0;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < G; g += (uint64_t)gridDim.x * blockDim.x) {
        bool run = Xe[g] > 0;
        if (!run && ion_only) {
            long long xp, xm;
            ion_counts(P, Xe, Npos, Nneg, G, g, xp, xm);
            run = xp > 0 && xm > 0;
        }
        if (run) {
            list[warp_slot32(&ctr->n_kmc_cells)] = (uint32_t)g;
        } else {
            fired[g] = 0;
            fired[G + g] = 0;
            fired[2 * G + g] = 0;
            if (rec) {
                fired[3 * G + g] = 0;
                fired[4 * G + g] = 0;
            }
            for (int s = 0; s < P.S; ++s) gain[(uint64_t)s * G + g] = 0;
        }
    }
}

// Residency: four blocks of 128 threads per SM in the FP64 form and with
// recombination (<= 128 registers), five in the FP32 first-order form.
template <class T, bool REC>
__global__ void __launch_bounds__(128, (sizeof(T) == 8 || REC) ? 4 : 5) k_kmc(Params P, const unsigned long long* __restrict__ Xe, const E64* __restrict__ E,
                      const float4* __restrict__ E32, int64_t* __restrict__ fired, int64_t* __restrict__ gain,
                      int64_t* __restrict__ Npos, int64_t* __restrict__ Nneg, uint64_t G, const uint32_t* __restrict__ list,
                      uint32_t* __restrict__ pc_list, Counters* __restrict__ ctr)
{
    unsigned long long t_ion = 0, t_att = 0, t_ph = 0, t_ep = 0, t_np = 0, t_slots = 0;
    const uint64_t n = ctr->n_kmc_cells;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t tend = ((n + stride - 1) / stride) * stride;   // whole warps iterate together
    for (uint64_t t = t0; t < tend; t += stride) {
        if (t >= n) continue;
        const uint64_t g = list[t];
        long long f[5] = { 0, 0, 0, 0, 0 };
        long long xp = 0, xm = 0;
        if constexpr (REC) ion_counts(P, Xe, Npos, Nneg, G, g, xp, xm);
        const long long X0[3] = { (long long)Xe[g], xp, xm };
        T kr[5];
        kr[3] = (T)P.k_ep;
        kr[4] = (T)P.k_np;
        if constexpr (sizeof(T) == 8) {
            const E64 e = ld_e64(E + g);
            const double Em = e.m;
            const double ve = P.mu * Em;
            const double alpha = (Em > 0.0) ? P.alpha_A * dexp(-(P.alpha_B / Em)) : 0.0;
            kr[0] = alpha * ve;
            kr[1] = P.eta * ve;
            kr[2] = P.photon_ratio * kr[0];
        } else {
            const float Em = __ldg(E32 + g).w;
            const float ve = (float)P.mu * Em;
            const float alpha = (Em > 0.0f) ? (float)P.alpha_A * expf(-((float)P.alpha_B / Em)) : 0.0f;
            kr[0] = alpha * ve;
            kr[1] = (float)P.eta * ve;
            kr[2] = (float)P.photon_ratio * kr[0];
        }
        const int r = real_of(P, (uint32_t)g);
        const uint32_t c = (uint32_t)(g & (uint64_t)(P.n3 - 1));
        Stream s(seed_of(P, r), c, step_of(P), TAG_KMC, 0);
        if (kmc_cell<T, REC>(P, s, X0, kr, f) != 0) {
            atomicOr(&ctr->err, DERR_KMC);
            ctr->kmc_fail_cell = (unsigned)g;
        }
        // net gains of the cell's particle species (Sec. 4.4); the per-cell
        // ion counts when the ions are not particles
        gain[g] = (f[0] - f[1]) - f[3];
        if (P.S == 3) {
            gain[G + g] = (f[0] - f[3]) - f[4];
            gain[2 * G + g] = f[1] - f[4];
        } else {
            Npos[g] += (f[0] - f[3]) - f[4];
            Nneg[g] += f[1] - f[4];
        }
        if (f[2] > 0) {
            t_slots += (unsigned long long)(f[2] < P.n_new ? f[2] : P.n_new);
            pc_list[warp_slot32(&ctr->n_photo_cells)] = (uint32_t)g;
        }
        t_ion += (unsigned long long)f[0];
        t_att += (unsigned long long)f[1];
        t_ph += (unsigned long long)f[2];
        t_ep += (unsigned long long)f[3];
        t_np += (unsigned long long)f[4];
        fired[g] = f[0];
        fired[G + g] = f[1];
        fired[2 * G + g] = f[2];
        if constexpr (REC) {
            fired[3 * G + g] = f[3];
            fired[4 * G + g] = f[4];
        }
    }
    warp_add(&ctr->ion, t_ion);
    warp_add(&ctr->att, t_att);
    warp_add(&ctr->phot, t_ph);
    if constexpr (REC) {
        warp_add(&ctr->rec_ep, t_ep);
        warp_add(&ctr->rec_np, t_np);
    }
    warp_add(&ctr->photo_slots, t_slots);
}

// ------------------------------------------------------------------ 0-D KMC
// Independent single-cell realizations (Sec. 3.2.4): realization m starts
// from X0 electrons and advances nsteps steps of dt with the rates of the
// field magnitude Em (k_ion = alpha(Em) mu Em, k_att = eta mu Em, k_ph =
// photon_ratio k_ion), each step the per-cell KMC of the spatial model drawn
// from the stream (key seed0, index m, step k, KMC).  X[m (nsteps + 1) + k]
// holds the electrons after k steps.  The ensembles track no ion counts:
// the network is the first-order one (no recombination).
template <class T>
__global__ void k_kmc0d(Params P, double Em, long long X0, uint32_t nreal, int nsteps, long long* __restrict__ X,
                        Counters* __restrict__ ctr)
{
    T kr[5];
    kr[3] = kr[4] = (T)0;
    if constexpr (sizeof(T) == 8) {
        const double ve = P.mu * Em;
        const double alpha = (Em > 0.0) ? P.alpha_A * dexp(-(P.alpha_B / Em)) : 0.0;
        kr[0] = alpha * ve;
        kr[1] = P.eta * ve;
        kr[2] = P.photon_ratio * kr[0];
    } else {
        const float Ef = (float)Em;
        const float ve = (float)P.mu * Ef;
        const float alpha = (Ef > 0.0f) ? (float)P.alpha_A * expf(-((float)P.alpha_B / Ef)) : 0.0f;
        kr[0] = alpha * ve;
        kr[1] = (float)P.eta * ve;
        kr[2] = (float)P.photon_ratio * kr[0];
    }
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < nreal; m += gridDim.x * blockDim.x) {
        long long x = X0;
        long long* out = X + (size_t)m * (nsteps + 1);
        out[0] = x;
        for (int k = 0; k < nsteps; ++k) {
            long long f[5] = { 0, 0, 0, 0, 0 };
            if (x > 0) {
                const long long X3[3] = { x, 0, 0 };
                Stream s(P.seed0, m, (uint32_t)k, TAG_KMC, 0);
                if (kmc_cell<T, false>(P, s, X3, kr, f) != 0) atomicOr(&ctr->err, DERR_KMC);
            }
            x += f[0] - f[1];
            out[k + 1] = x;
        }
    }
}

// ------------------------------------------------------------------ loss
// Systematic integer removal of L = -dN electrons from the cell's particles
// in canonical order: particle p loses floor((C_p L + R)/W) -
// floor((C_{p-1} L + R)/W), R = (64-bit draw) mod W.
// Gp particle cells: each block's species loses from its own particles,
// against its own NGP count, with its own stream tag.
__global__ void k_loss(Params P, uint32_t* __restrict__ wbase, int wstride, const uint32_t* __restrict__ cs,
                       const unsigned long long* __restrict__ Xe, const int64_t* __restrict__ gain, uint64_t G)
{
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < G; g += (uint64_t)gridDim.x * blockDim.x) {
        const long long dN = gain[g];
        if (dN >= 0) continue;
        const unsigned long long L = (unsigned long long)(-dN);
        const unsigned long long W = Xe[g];
        const int blk = real_of(P, (uint32_t)g);
        const uint32_t c = (uint32_t)(g & (uint64_t)(P.n3 - 1));
        Stream s(seed_of(P, phys_of(P, blk)), c, step_of(P), P.prod_tag_sp[species_of(P, blk)], (uint32_t)P.n_new);
        const uint32_t a = s.u32(), b = s.u32();
        const unsigned long long R = (((unsigned long long)a << 32) | b) % W;
        if (W < (1ull << 32)) {
            // C <= W and L <= W: C L + R < 2^64, the same quotients in 64 bits
            unsigned long long C64 = 0;
            for (uint32_t q = cs[g]; q < cs[g + 1]; ++q) {
                uint32_t* wq = wbase + (size_t)q * wstride;
                const uint32_t w = *wq;
                const unsigned long long before = (C64 * L + R) / W;
                C64 += w;
                const unsigned long long after = (C64 * L + R) / W;
                *wq = (uint32_t)(w - (after - before));
            }
            continue;
        }
        unsigned __int128 C = 0;
        for (uint32_t q = cs[g]; q < cs[g + 1]; ++q) {
            const unsigned __int128 before = (C * L + R) / W;
            uint32_t* wq = wbase + (size_t)q * wstride;
            const uint32_t w = *wq;
            C += w;
            const unsigned __int128 after = (C * L + R) / W;
            *wq = (uint32_t)(w - (unsigned long long)(after - before));
        }
    }
}

// Offset in cell units, rounded to FP32 and kept in [0, 1).
__device__ __forceinline__ float clamp_off(double v)
{
    float f = (float)v;
    if (!(f >= 0.0f)) f = 0.0f;
    if (f >= 1.0f) f = 0x1.fffffep-1f;
    return f;
}
__device__ __forceinline__ float clamp_offf(float f)
{
    if (!(f >= 0.0f)) f = 0.0f;
    if (f >= 1.0f) f = 0x1.fffffep-1f;
    return f;
}

// ------------------------------------------------------------------ photons
// One superphoton (cell c, slot j): emission point, kappa, distance, direction.
__device__ __forceinline__ void photon_sample(const Params& P, uint64_t seed, uint32_t c, uint32_t j,
                                              const int ijk[3], double lnK, double Y0[3], double& r,
                                              double dir[3])
{
    Stream s(seed, c, step_of(P), TAG_PHOTON, j);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double u = s.uniform();
        Y0[a] = P.lo[a] + ((double)ijk[a] + u) * P.h[a];
    }
    const double kappa = P.kappa_lo * dexp(s.uniform() * lnK);
    r = (-dlog(s.uniform())) / kappa;
    const double cz = 2.0 * s.uniform() - 1.0;
    double sphi, cphi;
    dsincos2pi(s.uniform(), &sphi, &cphi);
    const double st = sqrt((1.0 - cz) * (1.0 + cz));
    dir[0] = st * cphi;
    dir[1] = st * sphi;
    dir[2] = cz;
}

// One warp per photon-emitting cell, one lane per superphoton slot.
__global__ void k_photons(Params P, int mixed, const int64_t* __restrict__ fired, uint64_t G,
                          const uint32_t* __restrict__ pc_list, Photo* __restrict__ photos, uint32_t photo_cap,
                          int32_t* __restrict__ photo_cnt, unsigned long long* __restrict__ photo_w,
                          int64_t* __restrict__ Npos, Counters* __restrict__ ctr)
{
    const unsigned lane = lane_id();
    const uint32_t ncells = ctr->n_photo_cells;
    unsigned long long t_abs = 0;
    const double lnK = dlog(P.kappa_hi / P.kappa_lo);
    for (uint32_t e = (blockIdx.x * blockDim.x + threadIdx.x) / 32; e < ncells; e += (gridDim.x * blockDim.x) / 32) {
        const uint64_t g = pc_list[e];
        const long long Gm = fired[2 * G + g];
        const int r = real_of(P, (uint32_t)g);
        const uint32_t c = (uint32_t)(g & (uint64_t)(P.n3 - 1));
        const int ijk[3] = { (int)(c & (uint32_t)(P.n - 1)), (int)((c >> P.log2n) & (uint32_t)(P.n - 1)),
                             (int)(c >> (2 * P.log2n)) };
        const long long m = Gm < P.n_new ? Gm : P.n_new;
        const long long wq = Gm / m, rem = Gm % m;
        const uint64_t seed = seed_of(P, r);
        for (long long j = lane; j < m; j += 32) {
            const long long wj = wq + (j == 0 ? rem : 0);
            bool inside = true;
            int ix, iy, iz;
            double Ya[3];
            if (mixed) {
                // FP32 in cell units from the source cell's corner; the same
                // draws as the FP64 form (top 23 bits of each uniform)
                Stream st(seed, c, step_of(P), TAG_PHOTON, (uint32_t)j);
                float Yc[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const uint32_t hw = st.u32();
                    (void)st.u32();
                    Yc[a] = uniform_f32(hw);
                }
                const uint32_t h4 = st.u32(); (void)st.u32();
                const uint32_t h5 = st.u32(); (void)st.u32();
                const uint32_t h6 = st.u32(); (void)st.u32();
                const uint32_t h7 = st.u32(); (void)st.u32();
                const float kappa = (float)P.kappa_lo * expf(uniform_f32(h4) * (float)lnK);
                const float rc = (-logf(uniform_f32(h5))) / kappa * (float)(1.0 / P.h[0]);
                const float cz = 2.0f * uniform_f32(h6) - 1.0f;
                float sphi, cphi;
                sincospif(2.0f * uniform_f32(h7), &sphi, &cphi);
                const float stt = sqrtf((1.0f - cz) * (1.0f + cz));
                const float dir[3] = { stt * cphi, stt * sphi, cz };
                int id[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float y = Yc[a] + rc * dir[a];
                    const float fl = floorf(y);
                    id[a] = ijk[a] + (int)fl;
                    Ya[a] = (double)clamp_off((double)(y - fl));
                    inside = inside && id[a] >= 0 && id[a] < P.n;
                }
                ix = id[0]; iy = id[1]; iz = id[2];
            } else {
                double Y0[3], rr, dir[3];
                photon_sample(P, seed, c, (uint32_t)j, ijk, lnK, Y0, rr, dir);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Ya[a] = Y0[a] + rr * dir[a];
                    inside = inside && (Ya[a] >= P.lo[a]) && (Ya[a] < P.hi[a]);
                }
                ix = inside ? cell_axis(Ya[0], P.lo[0], P.h[0], P.rh[0], P.n) : 0;
                iy = inside ? cell_axis(Ya[1], P.lo[1], P.h[1], P.rh[1], P.n) : 0;
                iz = inside ? cell_axis(Ya[2], P.lo[2], P.h[2], P.rh[2], P.n) : 0;
            }
            if (!inside) {
                atomicAdd(&ctr->lost[r], (unsigned long long)wj);
                continue;
            }
            if (wj > 0xffffffffll) atomicOr(&ctr->err, DERR_OVERFLOW);
            const uint32_t gd = (uint32_t)((size_t)r * P.n3 + ((size_t)iz * P.n + iy) * P.n + ix);
            if (P.S == 1) atomicAdd((unsigned long long*)(Npos + gd), (unsigned long long)wj);
            atomicAdd(photo_cnt + gd, 1);
            atomicAdd(photo_w + gd, (unsigned long long)wj);
            t_abs += (unsigned long long)wj;
            const unsigned long long slot = warp_slot(&ctr->n_photo);
            if (slot < photo_cap) {
                Photo ph;
                ph.x = Ya[0]; ph.y = Ya[1]; ph.z = Ya[2];   // offsets (mixed) or absolute (FP64)
                ph.g = gd; ph.src = c; ph.slot = (uint32_t)j; ph.w = (uint32_t)wj;
                photos[slot] = ph;
            } else {
                atomicOr(&ctr->err, DERR_CAPACITY);
            }
        }
    }
    warp_add(&ctr->absorbed_w, t_abs);
}

__global__ void k_photo_place(const Photo* __restrict__ photos, const Counters* __restrict__ ctr,
                              uint32_t photo_cap, const uint32_t* __restrict__ photo_off,
                              int32_t* __restrict__ cursor, uint32_t* __restrict__ sorted)
{
    const uint32_t n = (uint32_t)min(ctr->n_photo, (unsigned long long)photo_cap);
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        const uint32_t g = photos[m].g;
        const uint32_t slot = photo_off[g] + (uint32_t)atomicAdd(cursor + g, 1);
        if (slot < photo_cap) sorted[slot] = m;
    }
}

// ------------------------------------------------------------------ merge scan
// Per-warp scratch of the merge of one cell (all node arrays for T = ppc
// nodes, element lists for `cap` elements): byte offsets from the base.
struct MLayout {
    uint32_t cur, tmp, nW, nW2, nC, keys, nA, nB, nb, nb2, npm, nsh, nid, nid2, nnd, nax, nfl, bytes;
};
__host__ __device__ inline uint32_t ml_take(uint32_t& o, uint32_t bytes)
{
    const uint32_t r = o;
    o += (bytes + 15u) & ~15u;
    return r;
}
__host__ __device__ inline MLayout merge_layout(uint32_t cap, uint32_t T, uint32_t esize, uint32_t ksize)
{
    MLayout L;
    uint32_t o = 0;
    L.cur = ml_take(o, cap * esize);
    L.tmp = ml_take(o, cap * esize);
    L.nW = ml_take(o, T * 8);
    L.nW2 = ml_take(o, (T + 1) * 8);
    L.nC = ml_take(o, T * 8);
    L.keys = ml_take(o, cap * (ksize == 4 ? 8u : 16u));   // KeyW<K>
    L.nA = ml_take(o, T * 4);
    L.nB = ml_take(o, T * 4);
    L.nb = ml_take(o, (T + 1) * 4);
    L.nb2 = ml_take(o, (T + 1) * 4);
    L.npm = ml_take(o, T * 4);
    L.nsh = ml_take(o, T * 4);
    L.nid = ml_take(o, cap * 2);
    L.nid2 = ml_take(o, cap * 2);
    L.nnd = ml_take(o, T * 2);
    L.nax = ml_take(o, T);
    L.nfl = ml_take(o, T);
    L.bytes = o;
    return L;
}

// Merge tiers by list capacity M + ppc (a level adds at most one element
// per node): tier 0 and 1 in shared memory (warps per block NW0 / NW1),
// tier 2 in the global work area.
constexpr uint32_t MERGE_CAP0_MP32 = 96, MERGE_CAP0_MP = 96, MERGE_CAP1 = 256;
constexpr int MERGE_NW0 = 4, MERGE_NW1 = 4;
__host__ __device__ inline uint32_t merge_cap0(int esize) { return esize == 16 ? MERGE_CAP0_MP32 : MERGE_CAP0_MP; }

// Per particle cell: W = X + dN + photo weight -> min(W, ppc) leaves; photo
// offsets; work-area units (32 B) for tier-2 cells; the tier lists.  The
// photons of physical cell c are the electron block's photoelectrons and the
// positive-ion block's photo-ions (mobile ions); the photo offsets count
// them once, over the electron blocks.
struct MergeScanOp {
    const unsigned long long* Xe;
    const int64_t* gain;
    const unsigned long long* photo_w;
    const int32_t* photo_cnt;
    const uint32_t* cs;
    uint32_t* out_start;
    uint32_t* photo_off;
    uint64_t* work_off;
    uint32_t* small_list;     // non-empty cells of tier 0
    uint32_t* mid_list;       // ... tier 1
    uint32_t* big_list;       // ... tier 2
    uint32_t* list_n;         // [3]: lengths
    uint64_t G;               // particle cells
    uint64_t Gphys;           // physical cells (one block per realization)
    int ppc, n_new, esize, ksize;
    __device__ void load(uint64_t g, long long v[6]) const
    {
        const long long dN = gain[g];
        const uint64_t sp = (uint64_t)(g >= Gphys) + (uint64_t)(g >= 2 * Gphys), gph = g - sp * Gphys;
        const long long pw = sp <= 1 ? (long long)photo_w[gph] : 0, pc = sp <= 1 ? photo_cnt[gph] : 0;
        const long long W = (long long)Xe[g] + dN + pw;
        v[0] = W < ppc ? W : ppc;
        v[1] = sp == 0 ? pc : 0;
        const long long M = (long long)(cs[g + 1] - cs[g]) + (dN > 0 ? (dN < n_new ? dN : n_new) : 0) + pc;
        const long long S = M + ppc;
        const int tier = S <= (long long)merge_cap0(esize) ? 0 : (S <= MERGE_CAP1 ? 1 : 2);
        v[2] = (v[0] > 0 && tier == 2)
                   ? ((long long)merge_layout((uint32_t)S, (uint32_t)ppc, (uint32_t)esize, (uint32_t)ksize).bytes + 31) / 32
                   : 0;
        v[3] = (v[0] > 0 && tier == 0) ? 1 : 0;
        v[4] = (v[0] > 0 && tier == 1) ? 1 : 0;
        v[5] = (v[0] > 0 && tier == 2) ? 1 : 0;
    }
    __device__ void store(uint64_t g, const long long ex[6], const long long* v) const
    {
        out_start[g] = (uint32_t)ex[0];
        photo_off[g] = (uint32_t)ex[1];
        work_off[g] = (uint64_t)ex[2];
        if (v[3]) small_list[ex[3]] = (uint32_t)g;
        if (v[4]) mid_list[ex[4]] = (uint32_t)g;
        if (v[5]) big_list[ex[5]] = (uint32_t)g;
    }
    __device__ void total(const long long t[6]) const
    {
        out_start[G] = (uint32_t)t[0];
        photo_off[G] = (uint32_t)t[1];
        work_off[G] = (uint64_t)t[2];
        list_n[0] = (uint32_t)t[3];
        list_n[1] = (uint32_t)t[4];
        list_n[2] = (uint32_t)t[5];
    }
};

// ------------------------------------------------------------------ merge
struct MP32 {         // merge work element (mixed form: cell offsets)
    float x, y, z;
    uint32_t w;
};

struct MP {           // merge work element (FP64 form)
    double x, y, z;
    uint32_t w;
    uint32_t pad;
};

template <class E> struct EKey { using K = unsigned long long; };
template <> struct EKey<MP32> { using K = uint32_t; };

// A sort key beside its element's weight: the rank loop reads both with one
// vector load.
template <class K> struct __align__(sizeof(K) == 4 ? 8 : 16) KeyW {
    K k;
    uint32_t w;
};

// Order-preserving integer keys of coordinates: the tree compares keys with
// integer instructions (FP64 comparisons run at a small fraction of the FP32
// rate on GB300).  key(a) < key(b) iff a < b for all non-NaN values except
// that -0 sorts below +0 (positions never hold -0).
__device__ __forceinline__ uint32_t okey(float v)
{
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned long long okey(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ float okey_val(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ double okey_val(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

template <class E> struct ET;
template <> struct ET<MP> {
    using K = unsigned long long;
    using V = double;
    static __device__ __forceinline__ K key(const MP& e, int a) { return okey(a == 0 ? e.x : (a == 1 ? e.y : e.z)); }
    static __device__ __forceinline__ K wmin(K v)
    {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) { const K o = __shfl_xor_sync(0xffffffffu, v, d); v = o < v ? o : v; }
        return v;
    }
    static __device__ __forceinline__ K wmax(K v)
    {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) { const K o = __shfl_xor_sync(0xffffffffu, v, d); v = o > v ? o : v; }
        return v;
    }
};
template <> struct ET<MP32> {
    using K = uint32_t;
    using V = float;
    static __device__ __forceinline__ K key(const MP32& e, int a) { return okey(a == 0 ? e.x : (a == 1 ? e.y : e.z)); }
    static __device__ __forceinline__ K wmin(K v) { return __reduce_min_sync(0xffffffffu, v); }
    static __device__ __forceinline__ K wmax(K v) { return __reduce_max_sync(0xffffffffu, v); }
};

// Widest axis from key bounds (largest extent, ties to the lowest axis); the
// extent hi - lo is taken in the element's own precision.
template <class E>
__device__ __forceinline__ int widest_axis(const typename ET<E>::K lo[3], const typename ET<E>::K hi[3])
{
    using V = typename ET<E>::V;
    V ext[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ext[a] = okey_val(hi[a]) - okey_val(lo[a]);
    int axis = 0;
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    return axis;
}

// Minimum / maximum / sum over a group of contiguous lanes (a node's
// elements in one chunk of 32; gs = the group's first lane) by an inclusive
// segmented shuffle scan; the result is valid at the group's last lane.
// (Shuffles measured faster than the redux and match instructions for this
// pattern on GB300.)
template <class V, class Op>
__device__ __forceinline__ V grp_scan(int gs, V v, unsigned lane, Op op)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const V o = __shfl_up_sync(0xffffffffu, v, d);
        if ((int)lane - d >= gs) v = op(o, v);
    }
    return v;
}
template <class V>
__device__ __forceinline__ V grp_min(int gs, V v, unsigned lane)
{
    return grp_scan(gs, v, lane, [](V a, V b) { return a < b ? a : b; });
}
template <class V>
__device__ __forceinline__ V grp_max(int gs, V v, unsigned lane)
{
    return grp_scan(gs, v, lane, [](V a, V b) { return a > b ? a : b; });
}

constexpr uint8_t NO_SPLIT = 0xff;

// Merge/split of whole cells, one warp per cell, all nodes of a tree level
// at once.  The cell's list (existing particles with w > 0 in canonical
// order, then new ones in (source cell, products before photoelectrons,
// slot) order) is split level by level exactly as specified: every node of
// weight >= 2 is sorted stably along the widest axis of its bounding box
// (ties keep the node's current order), cut at the weighted median (first
// element with 2 C > W), a unit-weight median joins the lighter side (left
// on ties) and a heavier one is divided ceil(W/2) - W_L : rest.  Leaves are
// the nodes after log2(ppc) levels.  Per level the warp runs element-
// parallel passes (bounding boxes by group reductions carried across chunks
// of 32, a rank sort whose loop also gives each element's prefix weight and
// so the weighted median, a scatter into the next level's list) and node-
// parallel passes (axis, median bookkeeping).  GLOBAL: the scratch lives in
// the work area (cells too long for shared memory).
// Residency the registers are sized for: four blocks for the global tier,
// seven (mixed form, whose shared scratch allows eight) or five (FP64 form,
// held to five by its shared scratch) for the shared-memory tiers.
template <class E, bool GLOBAL>
__global__ void __launch_bounds__(128, GLOBAL ? 4 : (std::is_same<E, MP32>::value ? 7 : 5)) k_merge_lv(
    Params P, const P64* __restrict__ A, const P32* __restrict__ A32, const uint32_t* __restrict__ cs,
    const int64_t* __restrict__ gain, const Photo* __restrict__ photos, const uint32_t* __restrict__ photo_sorted,
    const uint32_t* __restrict__ photo_off, const uint32_t* __restrict__ out_start,
    const uint64_t* __restrict__ work_off, unsigned char* __restrict__ work, uint64_t work_cap,
    P64* __restrict__ out, P32* __restrict__ out32, uint32_t* __restrict__ cout, uint64_t Gphys, uint32_t cap,
    uint32_t photo_cap, const uint32_t* __restrict__ list, const uint32_t* __restrict__ list_n, int tier,
    uint32_t CAP, Counters* __restrict__ ctr)
{
    constexpr bool MX = std::is_same<E, MP32>::value;
    using K = typename EKey<E>::K;
    extern __shared__ __align__(16) unsigned char msm[];
    const unsigned lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int T = P.ppc;
    const uint32_t ncells = list_n[tier];
    unsigned long long t_cells = 0, t_el = 0, t_sq = 0, t_max = 0;
    for (uint32_t li = blockIdx.x * nw + wid; li < ncells; li += gridDim.x * nw) {
        const uint64_t g = list[li];                  // particle cell
        const int b = real_of(P, (uint32_t)g);
        const int sp = species_of(P, b), r = phys_of(P, b);
        const uint32_t c = (uint32_t)(g & (uint64_t)(P.n3 - 1));
        const long long dN = gain[g];
        const uint32_t e0 = cs[g], e1 = cs[g + 1];
        const uint32_t mprod = dN > 0 ? (uint32_t)(dN < P.n_new ? dN : P.n_new) : 0u;
        // the photons absorbed in this cell: photoelectrons of the electron
        // block and, with mobile ions, photo-ions of the positive-ion block
        const uint64_t ge = g - (uint64_t)sp * Gphys;
        const uint32_t p0 = sp <= 1 ? photo_off[ge] : 0u, np = sp <= 1 ? photo_off[ge + 1] - p0 : 0u;
        const uint32_t Mmax = (e1 - e0) + mprod + np;
        if ((uint64_t)p0 + np > photo_cap || out_start[g + 1] > cap) {
            if (lane == 0) atomicOr(&ctr->err, DERR_CAPACITY);
            continue;
        }
        MLayout L;
        unsigned char* base;
        if constexpr (GLOBAL) {
            L = merge_layout(Mmax + T, T, sizeof(E), sizeof(K));
            if (work_off[g] * 32 + L.bytes > work_cap * 32) {
                if (lane == 0) atomicOr(&ctr->err, DERR_CAPACITY);
                continue;
            }
            base = work + work_off[g] * 32;
        } else {
            if (Mmax + T > CAP) {
                if (lane == 0) atomicOr(&ctr->err, DERR_INTERNAL);
                continue;
            }
            L = merge_layout(CAP, T, sizeof(E), sizeof(K));
            base = msm + (size_t)wid * L.bytes;
        }
        E* cur = reinterpret_cast<E*>(base + L.cur);
        E* tmp = reinterpret_cast<E*>(base + L.tmp);
        unsigned long long* nW = reinterpret_cast<unsigned long long*>(base + L.nW);
        unsigned long long* nW2 = reinterpret_cast<unsigned long long*>(base + L.nW2);
        unsigned long long* nC = reinterpret_cast<unsigned long long*>(base + L.nC);
        KeyW<K>* keys = reinterpret_cast<KeyW<K>*>(base + L.keys);
        uint32_t* nA = reinterpret_cast<uint32_t*>(base + L.nA);
        uint32_t* nB = reinterpret_cast<uint32_t*>(base + L.nB);
        uint32_t* nb = reinterpret_cast<uint32_t*>(base + L.nb);
        uint32_t* nb2 = reinterpret_cast<uint32_t*>(base + L.nb2);
        uint32_t* npm = reinterpret_cast<uint32_t*>(base + L.npm);
        uint32_t* nsh = reinterpret_cast<uint32_t*>(base + L.nsh);
        uint16_t* nid = reinterpret_cast<uint16_t*>(base + L.nid);
        uint16_t* nid2 = reinterpret_cast<uint16_t*>(base + L.nid2);
        uint16_t* nnd = reinterpret_cast<uint16_t*>(base + L.nnd);
        uint8_t* nax = reinterpret_cast<uint8_t*>(base + L.nax);
        uint8_t* nfl = reinterpret_cast<uint8_t*>(base + L.nfl);

        // ---- gather: existing particles with w > 0 (canonical order)
        uint32_t M = 0;
        for (uint32_t b = e0; b < e1; b += 32) {
            const uint32_t q = b + lane;
            E e;
            bool ok = false;
            if (q < e1) {
                if constexpr (MX) {
                    const P32 p = A32[q];
                    e.x = p.ox; e.y = p.oy; e.z = p.oz; e.w = p.w;
                } else {
                    const P64 p = ld_p64(A + q);
                    e.x = p.x; e.y = p.y; e.z = p.z; e.w = p.w; e.pad = 0;
                }
                ok = e.w > 0;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (ok) cur[M + __popc(bal & ((1u << lane) - 1u))] = e;
            M += __popc(bal);
        }
        // photoelectrons ranked by (source cell, slot): keys staged in tmp
        unsigned long long* pkey = reinterpret_cast<unsigned long long*>(tmp);
        uint32_t n_lt = 0;
        for (uint32_t j = lane; j < np; j += 32) {
            const Photo& pj = photos[photo_sorted[p0 + j]];
            pkey[j] = ((unsigned long long)pj.src << 8) | pj.slot;
            n_lt += pj.src < c;
        }
        n_lt = __reduce_add_sync(0xffffffffu, n_lt);
        __syncwarp();
        for (uint32_t j = lane; j < np; j += 32) {
            const unsigned long long kj = pkey[j];
            uint32_t rank = 0;
            for (uint32_t k = 0; k < np; ++k) rank += pkey[k] < kj;
            const Photo pj = photos[photo_sorted[p0 + j]];
            E e;
            e.x = pj.x; e.y = pj.y; e.z = pj.z; e.w = pj.w;
            if constexpr (!MX) e.pad = 0;
            cur[M + (rank < n_lt ? rank : rank + mprod)] = e;
        }
        // products: uniform in the cell, the remainder on the first
        if (mprod) {
            const long long wq = dN / (long long)mprod, rem = dN % (long long)mprod;
            const int ijk[3] = { (int)(c & (uint32_t)(P.n - 1)), (int)((c >> P.log2n) & (uint32_t)(P.n - 1)),
                                 (int)(c >> (2 * P.log2n)) };
            for (uint32_t j = lane; j < mprod; j += 32) {
                Stream st(seed_of(P, r), c, step_of(P), P.prod_tag_sp[sp], j);
                E e;
                if constexpr (MX) {
                    // FP32 uniforms from the high words of the FP64 ones
                    float X[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        X[a] = uniform_f32(st.u32());
                        (void)st.u32();
                    }
                    e.x = X[0]; e.y = X[1]; e.z = X[2];
                } else {
                    double X[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) X[a] = P.lo[a] + ((double)ijk[a] + st.uniform()) * P.h[a];
                    e.x = X[0]; e.y = X[1]; e.z = X[2];
                }
                const long long wj = wq + (j == 0 ? rem : 0);
                if (wj > 0xffffffffll) atomicOr(&ctr->err, DERR_OVERFLOW);
                e.w = (uint32_t)wj;
                if constexpr (!MX) e.pad = 0;
                cur[M + n_lt + j] = e;
            }
        }
        M += mprod + np;
        if (lane == 0) {
            t_cells += 1; t_el += M; t_sq += (unsigned long long)M * M; t_max = M > t_max ? M : t_max;
            nb[0] = 0;
            nb[1] = M;
        }
        // root weight; the weights of later nodes follow from the splits
        unsigned long long wroot = 0;
        for (uint32_t j = lane; j < M; j += 32) {
            nid[j] = 0;
            wroot += cur[j].w;
        }
#pragma unroll
        for (int dd = 16; dd > 0; dd >>= 1) wroot += __shfl_xor_sync(0xffffffffu, wroot, dd);
        if (lane == 0) nW[0] = wroot;
        const bool w32 = wroot < (1ull << 31);
        uint32_t n = M;
        int nnodes = 1;
        __syncwarp();

        for (int level = 1; level < T; level *= 2) {
            // ---- bounding boxes and the split axis of every node (NO_SPLIT
            // below weight 2), taken where a node's box is complete: one node
            // per lane when the nodes are small (at most 4 elements on
            // average), else group reductions per chunk
            bool any_split = false;
            if (n <= 4u * (uint32_t)nnodes) {
                for (int d = lane; d < nnodes; d += 32) {
                    K lo[3], hi[3];
                    const E e0 = cur[nb[d]];
#pragma unroll
                    for (int a = 0; a < 3; ++a) { lo[a] = ET<E>::key(e0, a); hi[a] = lo[a]; }
                    for (uint32_t q = nb[d] + 1; q < nb[d + 1]; ++q) {
                        const E e = cur[q];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const K v = ET<E>::key(e, a);
                            lo[a] = v < lo[a] ? v : lo[a];
                            hi[a] = v > hi[a] ? v : hi[a];
                        }
                    }
                    const bool sp = nW[d] >= 2;
                    nax[d] = sp ? (uint8_t)widest_axis<E>(lo, hi) : NO_SPLIT;
                    any_split |= sp;
                }
            } else {
                // a node continuing from the previous chunk takes that chunk's
                // partial bounds (carried from its last lane); a node's axis
                // is taken by its last lane
                K clo[3] = { (K)~(K)0, (K)~(K)0, (K)~(K)0 }, chi[3] = { 0, 0, 0 };
                uint32_t cd = 0xffffffffu;
                for (uint32_t b0 = 0; b0 < n; b0 += 32) {
                    const uint32_t j = b0 + lane;
                    const bool ok = j < n;
                    const uint32_t d = ok ? nid[j] : 0xffffu;
                    // nodes are contiguous: the lane's group is its node's range
                    // within the chunk (the tail past n forms one more group)
                    const uint32_t g0 = ok ? nb[d] : n, g1 = ok ? nb[d + 1] : b0 + 32;
                    const int gs = (int)(g0 > b0 ? g0 - b0 : 0);
                    const bool fin = ok && g1 <= b0 + 32 && (int)lane == (int)(g1 - b0) - 1;
                    const bool cont = d == cd;
                    E e;
                    if (ok) e = cur[j];
                    else { e.x = 0; e.y = 0; e.z = 0; e.w = 0; }
                    K lo[3], hi[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const K v = ET<E>::key(e, a);
                        K mn = grp_min(gs, v, lane), mx = grp_max(gs, v, lane);
                        if (cont) {
                            mn = clo[a] < mn ? clo[a] : mn;
                            mx = chi[a] > mx ? chi[a] : mx;
                        }
                        lo[a] = mn;
                        hi[a] = mx;
                        clo[a] = __shfl_sync(0xffffffffu, mn, 31);
                        chi[a] = __shfl_sync(0xffffffffu, mx, 31);
                    }
                    if (fin) {
                        const bool sp = nW[d] >= 2;
                        nax[d] = sp ? (uint8_t)widest_axis<E>(lo, hi) : NO_SPLIT;
                        any_split |= sp;
                    }
                    cd = __shfl_sync(0xffffffffu, d, 31);
                }
            }
            // no node of weight >= 2: this and all further levels keep the list
            if (!__any_sync(0xffffffffu, any_split)) break;
            __syncwarp();
            for (uint32_t j = lane; j < n; j += 32) {
                const uint8_t a = nax[nid[j]];
                const E e = cur[j];
                keys[j] = KeyW<K>{ a == NO_SPLIT ? (K)0 : ET<E>::key(e, a), e.w };
            }
            __syncwarp();
            // ---- stable rank sort within each node (cur -> tmp), and the
            // weighted median: an element's rank counts the node's elements
            // placed before it, whose weights give its inclusive prefix
            // weight v in sorted order; the median is the element with
            // 2 v > W >= 2 (v - w)
            for (uint32_t j = lane; j < n; j += 32) {
                const uint32_t d = nid[j];
                const E ej = cur[j];
                if (nax[d] == NO_SPLIT) { tmp[j] = ej; continue; }
                const uint32_t s0 = nb[d], s1 = nb[d + 1];
                const K kj = keys[j].k;
                // one pass over the node (every lane of the node busy for the
                // same trip count): smaller keys, and equal keys placed before
                uint32_t rk = 0;
                unsigned long long v;
                if (w32) {
                    uint32_t pw = 0;
                    for (uint32_t k = s0; k < s1; ++k) {
                        const KeyW<K> q = keys[k];
                        const K kk = q.k;
                        const uint32_t wk = q.w;
                        const bool bf = (kk < kj) | ((kk == kj) & (k < j));
                        rk += bf;
                        pw += bf ? wk : 0u;
                    }
                    v = (unsigned long long)pw + ej.w;
                } else {
                    unsigned long long pw = 0;
                    for (uint32_t k = s0; k < s1; ++k) {
                        const KeyW<K> q = keys[k];
                        const K kk = q.k;
                        const uint32_t wk = q.w;
                        const bool bf = (kk < kj) | ((kk == kj) & (k < j));
                        rk += bf;
                        pw += bf ? (unsigned long long)wk : 0ull;
                    }
                    v = pw + ej.w;
                }
                tmp[s0 + rk] = ej;
                const unsigned long long W = nW[d];
                if (2ull * v > W && 2ull * (v - ej.w) <= W) {
                    npm[d] = rk;
                    nC[d] = v;
                }
            }
            __syncwarp();
            // ---- per node: median rule, child layout of the next level
            uint32_t ex_c = 0, nd_c = 0;
            for (int d0 = 0; d0 < nnodes; d0 += 32) {
                const int d = d0 + (int)lane;
                uint32_t extra = 0, cnt = 0, pm = 0, a = 0, b = 0;
                bool lm = false, rm = false, split = false;
                if (d < nnodes) {
                    split = nax[d] != NO_SPLIT;
                    cnt = split ? 2u : 1u;
                    if (split) {
                        pm = npm[d];
                        const unsigned long long W = nW[d], C = nC[d];
                        const uint32_t wm = tmp[nb[d] + pm].w;
                        const unsigned long long WL = C - wm, WR = W - C;
                        if (wm == 1) {
                            lm = WL <= WR;
                            rm = !lm;
                        } else {
                            const unsigned long long aa = (W + 1) / 2 - WL;
                            a = (uint32_t)aa;
                            b = (uint32_t)(wm - aa);
                            lm = a > 0;
                            rm = b > 0;
                        }
                        extra = (lm ? 1u : 0u) + (rm ? 1u : 0u) - 1u;
                    }
                }
                // both prefix counts in one word (each at most 64 per chunk)
                uint32_t pk = (cnt << 16) | extra;
#pragma unroll
                for (int k = 1; k < 32; k <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, pk, k);
                    if ((int)lane >= k) pk += y;
                }
                const uint32_t ie = pk & 0xffffu, ic = pk >> 16;
                if (d < nnodes) {
                    const uint32_t sh = ex_c + ie - extra, ndi = nd_c + ic - cnt;
                    nsh[d] = sh;
                    nnd[d] = (uint16_t)ndi;
                    // weights of the children: the left one holds the elements
                    // before the median and the median's left share
                    const unsigned long long Wd = nW[d];
                    if (split) {
                        const uint32_t wm = tmp[nb[d] + pm].w;
                        const unsigned long long wl = nC[d] - wm + (lm ? (wm == 1 ? 1ull : (unsigned long long)a) : 0ull);
                        nW2[ndi] = wl;
                        nW2[ndi + 1] = Wd - wl;
                    } else {
                        nW2[ndi] = Wd;
                    }
                    nA[d] = a;
                    nB[d] = b;
                    nfl[d] = (uint8_t)((lm ? 1 : 0) | (rm ? 2 : 0));
                    const uint32_t start = nb[d] + sh;
                    nb2[ndi] = start;
                    if (split) nb2[ndi + 1] = start + pm + (lm ? 1u : 0u);
                }
                ex_c += __shfl_sync(0xffffffffu, ie, 31);
                nd_c += __shfl_sync(0xffffffffu, ic, 31);
            }
            if (lane == 0) nb2[nd_c] = n + ex_c;
            __syncwarp();
            // ---- scatter into the next level's list
            for (uint32_t j = lane; j < n; j += 32) {
                const uint32_t d = nid[j];
                const uint32_t p = j - nb[d], start = nb[d] + nsh[d];
                const uint16_t nd = nnd[d];
                const E e = tmp[j];
                if (nax[d] == NO_SPLIT) {
                    cur[start + p] = e;
                    nid2[start + p] = nd;
                    continue;
                }
                const uint32_t pm = npm[d];
                const uint32_t lm = nfl[d] & 1u, rm = nfl[d] >> 1;
                if (p < pm) {
                    cur[start + p] = e;
                    nid2[start + p] = nd;
                } else if (p > pm) {
                    const uint32_t q = start + p + lm + rm - 1u;
                    cur[q] = e;
                    nid2[q] = (uint16_t)(nd + 1);
                } else {
                    if (lm) {
                        E l = e;
                        if (e.w != 1) l.w = nA[d];
                        cur[start + pm] = l;
                        nid2[start + pm] = nd;
                    }
                    if (rm) {
                        E rr = e;
                        if (e.w != 1) rr.w = nB[d];
                        cur[start + pm + lm] = rr;
                        nid2[start + pm + lm] = (uint16_t)(nd + 1);
                    }
                }
            }
            n += ex_c;
            nnodes = (int)nd_c;
            { uint32_t* t = nb; nb = nb2; nb2 = t; }
            { uint16_t* t = nid; nid = nid2; nid2 = t; }
            { unsigned long long* t = nW; nW = nW2; nW2 = t; }
            __syncwarp();
        }
        // ---- leaves: weight sum, weight-averaged position (list order)
        const uint32_t o0 = out_start[g];
        if ((uint32_t)nnodes != out_start[g + 1] - o0) {
            if (lane == 0) atomicOr(&ctr->err, DERR_INTERNAL);
        } else {
            for (int d = lane; d < nnodes; d += 32) {
                if constexpr (MX) {
                    // mixed form: a one-element leaf keeps its offsets; the
                    // weighted mean of a larger leaf is taken in FP32
                    const uint32_t q0 = nb[d], q1 = nb[d + 1];
                    P32 o;
                    if (q1 - q0 == 1) {
                        const E e = cur[q0];
                        o.ox = e.x; o.oy = e.y; o.oz = e.z; o.w = e.w;
                    } else {
                        float sx = 0.f, sy = 0.f, sz = 0.f;
                        unsigned long long Wl = 0;
                        for (uint32_t q = q0; q < q1; ++q) {
                            const E e = cur[q];
                            const float wf = (float)e.w;
                            sx = __fmaf_rn(wf, e.x, sx);
                            sy = __fmaf_rn(wf, e.y, sy);
                            sz = __fmaf_rn(wf, e.z, sz);
                            Wl += e.w;
                        }
                        if (Wl > 0xffffffffull) atomicOr(&ctr->err, DERR_OVERFLOW);
                        const float Wf = (float)Wl;
                        o.ox = clamp_offf(sx / Wf); o.oy = clamp_offf(sy / Wf); o.oz = clamp_offf(sz / Wf);
                        o.w = (uint32_t)Wl;
                    }
                    out32[o0 + d] = o;
                    cout[o0 + d] = (uint32_t)g;
                } else {
                    double sx = 0.0, sy = 0.0, sz = 0.0;
                    unsigned long long Wl = 0;
                    for (uint32_t q = nb[d]; q < nb[d + 1]; ++q) {
                        const E e = cur[q];
                        const double wd = (double)e.w;
                        sx = __fma_rn(wd, e.x, sx);
                        sy = __fma_rn(wd, e.y, sy);
                        sz = __fma_rn(wd, e.z, sz);
                        Wl += e.w;
                    }
                    if (Wl > 0xffffffffull) atomicOr(&ctr->err, DERR_OVERFLOW);
                    // quotients by the reciprocal of W with one fused correction
                    const double Wd = (double)Wl, rw = 1.0 / Wd;
                    P64 o;
                    o.x = quot_r(sx, Wd, rw); o.y = quot_r(sy, Wd, rw); o.z = quot_r(sz, Wd, rw);
                    o.cell = (uint32_t)g;
                    o.w = (uint32_t)Wl;
                    st_p64(out + o0 + d, o);
                }
            }
        }
        __syncwarp();
    }
    // workload counters, one atomic each per warp
    if (lane == 0 && t_cells) {
        atomicAdd(&ctr->merge_cells, t_cells);
        atomicAdd(&ctr->merge_elems, t_el);
        atomicAdd(&ctr->merge_elems2, t_sq);
        atomicMax(&ctr->merge_maxm, t_max);
    }
}

// ------------------------------------------------------------------ mixed form
// Positions are (cell, FP32 offset in cell units); the push, interpolation
// and normals run in FP32; the deposit stays exact int64 fixed point.
__device__ __forceinline__ void cic32(float o, int idx, int n, int& ia, int& ib, float& f)
{
    const bool up = o >= 0.5f;
    const int i0 = idx - 1 + (up ? 1 : 0);
    f = up ? o - 0.5f : o + 0.5f;
    ia = clampi(i0, n);
    ib = clampi(i0 + 1, n);
}

__device__ __forceinline__ void deposit32(const Params& P, unsigned long long* __restrict__ ne, const int id[3],
                                          const float o[3], uint32_t w)
{
    const int one = 1 << P.frac_bits, half = one >> 1;
    int ia[3], ib[3];
    long long A[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int q = (int)floorf(o[a] * (float)one);   // exact: o in [0,1), power-of-two scale
        const int aa = (q + half) & (one - 1);
        const int i0 = id[a] - 1 + (q >= half ? 1 : 0);
        ia[a] = clampi(i0, P.n);
        ib[a] = clampi(i0 + 1, P.n);
        A[a][0] = one - aa;
        A[a][1] = aa;
    }
    const int ix[2] = { ia[0], ib[0] }, iy[2] = { ia[1], ib[1] }, iz[2] = { ia[2], ib[2] };
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const long long v = (long long)w * A[0][a] * A[1][b] * A[2][c];
                if (v) atomicAdd(ne + ((size_t)iz[c] * P.n + iy[b]) * P.n + ix[a], (unsigned long long)v);
            }
}

// Pass 1 of the mixed form: interpolation (FP32, cell-relative offsets),
// push, new cell, fixed-point deposit, per-cell counts.  SINGLE: one
// realization (Philox key and counter index are kernel-wide).
template <bool SINGLE>
__global__ void __launch_bounds__(TPB, 4) k_push_f32(
    Params P, const P32* __restrict__ A, const uint32_t* __restrict__ cA, P32* __restrict__ B,
    uint32_t* __restrict__ keyB, uint32_t N, const uint32_t* __restrict__ cell_start,
    const float4* __restrict__ E32, int32_t* __restrict__ cnt_new, int32_t* __restrict__ in_cnt,
    int32_t* __restrict__ in_before, unsigned long long* __restrict__ Xe, unsigned long long* __restrict__ ne_fix,
    Mover* __restrict__ movers, uint32_t mover_cap, Counters* __restrict__ ctr, uint32_t* __restrict__ blk_stay,
    const uint32_t* __restrict__ Ndev)
{
    if (Ndev) N = *Ndev;
    const uint32_t i = blockIdx.x * TPB + threadIdx.x;
    bool alive = false, mover = false;
    uint32_t gnew = 0, w = 0;
    int rr = 0;
    Stencil S;
    if (i < N) {
        const P32 p = A[i];
        const uint32_t gold = __ldg(cA + i);
        const int r = SINGLE ? 0 : real_of(P, gold);      // particle block
        rr = r;
        const int sp = SINGLE ? 0 : species_of(P, r), rp = SINGLE ? 0 : phys_of(P, r);
        const uint32_t c = gold & (uint32_t)(P.n3 - 1);
        const int id[3] = { (int)(c & (uint32_t)(P.n - 1)), (int)((c >> P.log2n) & (uint32_t)(P.n - 1)),
                            (int)(c >> (2 * P.log2n)) };
        const uint32_t idx = SINGLE ? i : i - cell_start[(size_t)r * P.n3];
        const size_t ebase = SINGLE ? 0 : (size_t)r * P.n3;
        const size_t fbase = SINGLE ? 0 : (size_t)rp * P.n3;
        w = p.w;
        const float o[3] = { p.ox, p.oy, p.oz };
        int ia[3], ib[3];
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) cic32(o[a], id[a], P.n, ia[a], ib[a], f[a]);
        const float wx[2] = { 1.f - f[0], f[0] }, wy[2] = { 1.f - f[1], f[1] }, wz[2] = { 1.f - f[2], f[2] };
        const int ix[2] = { ia[0], ib[0] }, iy[2] = { ia[1], ib[1] }, iz[2] = { ia[2], ib[2] };
        float ex = 0.f, ey = 0.f, ez = 0.f;
#pragma unroll
        for (int cz = 0; cz < 2; ++cz)
#pragma unroll
            for (int by = 0; by < 2; ++by)
#pragma unroll
                for (int ax = 0; ax < 2; ++ax) {
                    const float wgt = __fmul_rn(__fmul_rn(wx[ax], wy[by]), wz[cz]);
                    const float4 e = __ldg(E32 + fbase + ((size_t)iz[cz] * P.n + iy[by]) * P.n + ix[ax]);
                    ex = __fmaf_rn(wgt, e.x, ex);
                    ey = __fmaf_rn(wgt, e.y, ey);
                    ez = __fmaf_rn(wgt, e.z, ez);
                }
        // the FP64 form's stream and words: the same ziggurat decisions, so
        // both forms draw common random numbers (equal to FP32 rounding)
        PairStream zs(SINGLE ? P.seed0 : seed_of(P, rp), idx, step_of(P), SINGLE ? TAG_PUSH : P.push_tag_sp[sp], 0);
        float nrm[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) nrm[a] = znormal32(zs);
        const float Ep[3] = { ex, ey, ez };
        float on[3];
        int idn[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float d = __fmaf_rn(P.f_drift_sp[sp], Ep[a], P.f_diff_sp[sp] * nrm[a]);
            float x = o[a] + d;
            const float fl = floorf(x);
            x -= fl;
            if (x >= 1.0f) x = 0x1.fffffep-1f;
            if (!(x >= 0.0f)) x = 0.0f;
            on[a] = x;
            idn[a] = id[a] + (int)fl;
            inside = inside && idn[a] >= 0 && idn[a] < P.n;
        }
        P32 q;
        q.ox = on[0]; q.oy = on[1]; q.oz = on[2]; q.w = w;
        B[i] = q;
        if (inside) {
            gnew = (uint32_t)(ebase + ((size_t)idn[2] * P.n + idn[1]) * P.n + idn[0]);
            alive = true;
            mover = gnew != gold;
            keyB[i] = gnew | (mover ? KEY_MOVER : 0u);
            stencil_f32(P, idn, on, S);
            if (mover) {
                atomicAdd(in_cnt + gnew, 1);
                if (gold < gnew) atomicAdd(in_before + gnew, 1);
                const unsigned long long slot = warp_slot(&ctr->n_movers);
                if (slot < mover_cap) movers[slot] = Mover{ gnew, i };
                else atomicOr(&ctr->err, DERR_CAPACITY);
            }
        } else {
            keyB[i] = KEY_DEAD;
            atomicAdd(&ctr->outflow[r], (unsigned long long)w);
        }
    }
    block_deposit<SINGLE>(P, ne_fix, alive, rr, S, w);
    unsigned long long v = alive ? (unsigned long long)w : 0ull;
    unsigned cc = alive ? 1u : 0u;
    if (warp_run_sum(gnew, alive, v, cc)) {
        atomicAdd(cnt_new + gnew, (int)cc);
        atomicAdd(Xe + gnew, v);
    }
    const int nstay = __syncthreads_count(alive && !mover);
    if (threadIdx.x == 0) blk_stay[blockIdx.x] = (uint32_t)nstay;
}

__global__ void __launch_bounds__(TPB) k_scatter_f32(const P32* __restrict__ B, P32* __restrict__ A,
                                                     uint32_t* __restrict__ cA, const uint32_t* __restrict__ keyB,
                                                     uint32_t N, const uint32_t* __restrict__ blk_prefix,
                                                     const int64_t* __restrict__ delta, uint32_t cap,
                                                     Counters* __restrict__ ctr, const uint32_t* __restrict__ Ndev)
{
    if (Ndev) N = *Ndev;
    const uint32_t i = blockIdx.x * TPB + threadIdx.x;
    uint32_t k = KEY_DEAD;
    if (i < N) k = keyB[i];
    const bool stay = !(k & (KEY_DEAD | KEY_MOVER));
    const uint32_t rank = block_excl_count(stay, nullptr);
    if (stay) {
        const uint32_t g = k & KEY_MASK;
        const long long pos = (long long)blk_prefix[blockIdx.x] + rank + delta[g];
        if (pos >= 0 && pos < (long long)cap) {
            A[pos] = B[i];
            cA[pos] = g;
        } else {
            atomicOr(&ctr->err, DERR_INTERNAL);
        }
    }
}

__global__ void k_mover_write_f32(const Mover* __restrict__ movers, const Counters* __restrict__ ctr,
                                  uint32_t mover_cap, const uint32_t* __restrict__ sorted,
                                  const uint32_t* __restrict__ in_off, const int32_t* __restrict__ in_cnt,
                                  const int32_t* __restrict__ in_before, const int32_t* __restrict__ cnt_new,
                                  const uint32_t* __restrict__ new_start, int32_t* __restrict__ cursor,
                                  const P32* __restrict__ B, P32* __restrict__ A, uint32_t* __restrict__ cA)
{
    const uint32_t n = (uint32_t)min(ctr->n_movers, (unsigned long long)mover_cap);
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const Mover mv = movers[sorted[s]];
        const uint32_t g = mv.g;
        const uint32_t b = in_off[g], e = b + (uint32_t)in_cnt[g];
        uint32_t rank = 0;
        for (uint32_t t = b; t < e && t < mover_cap; ++t) rank += movers[sorted[t]].i < mv.i;
        const uint32_t stay = (uint32_t)(cnt_new[g] - in_cnt[g]);
        const uint32_t pos = new_start[g] + rank + (rank >= (uint32_t)in_before[g] ? stay : 0u);
        if (pos < mover_cap && e <= mover_cap) {
            A[pos] = B[mv.i];
            cA[pos] = g;
        }
        cursor[g] = 0;
    }
}

__global__ void __launch_bounds__(TPB) k_deposit_f32(Params P, const P32* __restrict__ A,
                                                     const uint32_t* __restrict__ cA, uint32_t N,
                                                     unsigned long long* __restrict__ Xe,
                                                     unsigned long long* __restrict__ ne_fix)
{
    const uint32_t i = blockIdx.x * TPB + threadIdx.x;
    bool alive = i < N;
    uint32_t g = 0, w = 0;
    if (alive) {
        const P32 p = A[i];
        g = cA[i];
        w = p.w;
        const uint32_t c = g & (uint32_t)(P.n3 - 1);
        const int id[3] = { (int)(c & (uint32_t)(P.n - 1)), (int)((c >> P.log2n) & (uint32_t)(P.n - 1)),
                            (int)(c >> (2 * P.log2n)) };
        const float o[3] = { p.ox, p.oy, p.oz };
        deposit32(P, ne_fix + (size_t)real_of(P, g) * P.n3, id, o, w);
    }
    unsigned long long v = alive ? (unsigned long long)w : 0ull;
    unsigned c = alive ? 1u : 0u;
    if (warp_run_sum(g, alive, v, c)) atomicAdd(Xe + g, v);
}

int grid_for(uint64_t n, int tpb, int maxb = 152 * 16)
{
    const uint64_t b = (n + tpb - 1) / tpb;
    return (int)(b < 1 ? 1 : (b > (uint64_t)maxb ? (uint64_t)maxb : b));
}

}  // namespace

size_t scan_scratch_elems(uint64_t G, int C) { return (size_t)(scan_nblk(G) + 1) * C + C; }

// ---------------------------------------------------------------- launchers
// Ndev (graph-replayed steps): the particle count is read on the device and
// N is a bound on it that sizes the grids; otherwise N is the count.
void launch_transport(const Params& P, Dev& d, uint32_t N, cudaStream_t s, const uint32_t* Ndev)
{
    const uint64_t G = (uint64_t)P.B * P.n3;     // particle cells
    cudaMemsetAsync(d.cnt_new, 0, G * sizeof(int32_t), s);
    cudaMemsetAsync(d.in_cnt, 0, G * sizeof(int32_t), s);
    cudaMemsetAsync(d.in_before, 0, G * sizeof(int32_t), s);
    cudaMemsetAsync(d.Xe, 0, G * sizeof(unsigned long long), s);
    cudaMemsetAsync(d.ne_fix, 0, G * sizeof(unsigned long long), s);
    cudaMemsetAsync(d.ctr, 0, sizeof(Counters), s);
    const uint32_t nblk = (N + TPB - 1) / TPB;
    if (N == 0) return;
    ++g_launches;
    if (d.mixed) {
        auto k = P.B == 1 ? k_push_f32<true> : k_push_f32<false>;
        k<<<nblk, TPB, 0, s>>>(P, d.rA32, d.cellA32, d.rB32, d.keyB, N, d.cell_start, d.E32, d.cnt_new, d.in_cnt,
                               d.in_before, d.Xe, d.ne_fix, d.movers, d.mover_cap, d.ctr, d.blk_stay, Ndev);
    } else
        k_push_f64<<<nblk, TPB, 0, s>>>(P, d.recA, d.recB, d.keyB, N, d.cell_start, d.E, d.cnt_new, d.in_cnt,
                                         d.in_before, d.Xe, d.ne_fix, d.movers, d.mover_cap, d.ctr, d.blk_stay,
                                         Ndev);
}

// Semi-implicit transport (FP64 form), Sec. 4.7 steps 2 and 5: the
// diffusive substep X+ = X + sqrt(2 D dt) N into recB (the push's normals:
// the same stream and order), and the advective substep from X+ with the
// field of d.E, which also counts, keys and deposits like the push.
__global__ void __launch_bounds__(TPB) k_diffuse_f64(Params P, const P64* __restrict__ A, P64* __restrict__ B,
                                                     uint32_t N, const uint32_t* __restrict__ cell_start)
{
    const uint32_t i = blockIdx.x * TPB + threadIdx.x;
    if (i >= N) return;
    P64 p = ld_p64(A + i);
    const int r = real_of(P, p.cell);
    const uint32_t idx = i - cell_start[(size_t)r * P.n3];
    PairStream s(seed_of(P, r), idx, step_of(P), TAG_PUSH, 0);
    double Nn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Nn[a] = znormal(s);
    p.x = p.x + P.sdt * Nn[0];
    p.y = p.y + P.sdt * Nn[1];
    p.z = p.z + P.sdt * Nn[2];
    st_p64(B + i, p);
}

void launch_diffuse(const Params& P, Dev& d, uint32_t N, cudaStream_t s)
{
    if (N == 0) return;
    ++g_launches;
    k_diffuse_f64<<<(N + TPB - 1) / TPB, TPB, 0, s>>>(P, d.recA, d.recB, N, d.cell_start);
}

// Deposit (ne_fix, X_e) of the records of recB (the diffused positions).
void launch_deposit_B(const Params& P, Dev& d, uint32_t N, cudaStream_t s)
{
    const uint64_t G = (uint64_t)P.B * P.n3;
    cudaMemsetAsync(d.Xe, 0, G * sizeof(unsigned long long), s);
    cudaMemsetAsync(d.ne_fix, 0, G * sizeof(unsigned long long), s);
    if (N == 0) return;
    ++g_launches;
    k_deposit_f64<<<(N + TPB - 1) / TPB, TPB, 0, s>>>(P, d.recB, N, d.Xe, d.ne_fix);
}

void launch_advect(const Params& P, Dev& d, uint32_t N, cudaStream_t s)
{
    const uint64_t G = (uint64_t)P.B * P.n3;
    cudaMemsetAsync(d.cnt_new, 0, G * sizeof(int32_t), s);
    cudaMemsetAsync(d.in_cnt, 0, G * sizeof(int32_t), s);
    cudaMemsetAsync(d.in_before, 0, G * sizeof(int32_t), s);
    cudaMemsetAsync(d.Xe, 0, G * sizeof(unsigned long long), s);
    cudaMemsetAsync(d.ne_fix, 0, G * sizeof(unsigned long long), s);
    cudaMemsetAsync(d.ctr, 0, sizeof(Counters), s);
    if (N == 0) return;
    ++g_launches;
    k_advect_f64<<<(N + TPB - 1) / TPB, TPB, 0, s>>>(P, d.recA, d.recB, d.keyB, N, d.cell_start, d.E,
                                                          d.cnt_new, d.in_cnt, d.in_before, d.Xe, d.ne_fix,
                                                          d.movers, d.mover_cap, d.ctr, d.blk_stay);
}

void launch_transport_finish(const Params& P, Dev& d, uint32_t N, uint64_t G, cudaStream_t s, const uint32_t* Ndev)
{
    TransportScanOp op{ d.cnt_new, d.in_cnt, d.in_before, d.cell_start_B, d.delta, d.in_off, G };
    run_scan<3>(op, G, d.scan_blk, s);
    const uint32_t nblk = (N + TPB - 1) / TPB;
    if (N > 0) {
        BlockScanOp bop{ d.blk_stay, d.blk_prefix };
        run_scan<1>(bop, nblk, d.scan_blk + scan_scratch_elems(G, 3), s);
        const int mg = grid_for(N / 8 + 1, 256, 1024);
        g_launches += 3;
        if (d.mixed) {
            k_scatter_f32<<<nblk, TPB, 0, s>>>(d.rB32, d.rA32, d.cellA32, d.keyB, N, d.blk_prefix, d.delta,
                                               d.mover_cap, d.ctr, Ndev);
            k_mover_place<<<mg, 256, 0, s>>>(d.movers, d.ctr, d.mover_cap, d.in_off, d.cursor, d.mover_sorted);
            k_mover_write_f32<<<mg, 256, 0, s>>>(d.movers, d.ctr, d.mover_cap, d.mover_sorted, d.in_off, d.in_cnt,
                                                 d.in_before, d.cnt_new, d.cell_start_B, d.cursor, d.rB32, d.rA32,
                                                 d.cellA32);
        } else {
            k_scatter_f64<<<nblk, TPB, 0, s>>>(d.recB, d.recA, d.keyB, N, d.blk_prefix, d.delta, d.mover_cap,
                                               d.ctr, Ndev);
            k_mover_place<<<mg, 256, 0, s>>>(d.movers, d.ctr, d.mover_cap, d.in_off, d.cursor, d.mover_sorted);
            k_mover_write_f64<<<mg, 256, 0, s>>>(d.movers, d.ctr, d.mover_cap, d.mover_sorted, d.in_off, d.in_cnt,
                                                 d.in_before, d.cnt_new, d.cell_start_B, d.cursor, d.recB, d.recA);
        }
    }
    uint32_t* t = d.cell_start; d.cell_start = d.cell_start_B; d.cell_start_B = t;
}

void launch_deposit_only(const Params& P, Dev& d, uint32_t N, cudaStream_t s)
{
    const uint64_t G = (uint64_t)P.B * P.n3;
    cudaMemsetAsync(d.Xe, 0, G * sizeof(unsigned long long), s);
    cudaMemsetAsync(d.ne_fix, 0, G * sizeof(unsigned long long), s);
    if (N == 0) return;
    ++g_launches;
    if (d.mixed) k_deposit_f32<<<(N + TPB - 1) / TPB, TPB, 0, s>>>(P, d.rA32, d.cellA32, N, d.Xe, d.ne_fix);
    else k_deposit_f64<<<(N + TPB - 1) / TPB, TPB, 0, s>>>(P, d.recA, N, d.Xe, d.ne_fix);
}

// Time of the push kernel alone (ms per launch, median of reps) with the
// current parameters: it reads the records and writes only what the next
// transport stage writes again first (the autotuner's deposit-window trial).
float time_push(const Params& P, Dev& d, uint32_t N, cudaStream_t s, int reps)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = -1.f;
    for (int k = 0; k < reps; ++k) {
        cudaEventRecord(a, s);
        launch_transport(P, d, N, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (best < 0.f || ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// Sets *flag if a and b differ anywhere (the autotuner's check that every
// deposit window gives the same integer densities).
__global__ void k_diff_flag(const unsigned long long* __restrict__ a, const unsigned long long* __restrict__ b,
                            uint64_t n, unsigned int* __restrict__ flag)
{
    bool diff = false;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        diff |= a[i] != b[i];
    if (__any_sync(0xffffffffu, diff) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

void launch_diff_flag(const unsigned long long* a, const unsigned long long* b, uint64_t n, unsigned int* flag,
                      cudaStream_t s)
{
    ++g_launches;
    k_diff_flag<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(a, b, n, flag);
}

// Ziggurat tables, once per device (the same values for every handle).
void launch_zig_init(cudaStream_t s)
{
    static std::mutex mtx;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mtx);
    if (dev >= 0 && dev < 64 && done[dev]) return;
    ++g_launches;
    k_zig_init<<<1, 1, 0, s>>>();
    cudaStreamSynchronize(s);
    if (dev >= 0 && dev < 64) done[dev] = true;
}

void launch_rho(const Params& P, Dev& d, uint64_t G, cudaStream_t s)
{
    double qscale, bc_top;
    rhs_consts(P, qscale, bc_top);
    ++g_launches;
    // the fixed-point field form builds its right-hand side in the solve
    k_rho<<<grid_for(G, 256), 256, 0, s>>>(P, d.Npos, d.Nneg, d.ne_fix, d.rho, d.phi_F > 0 ? nullptr : d.lev[0].rhs,
                                          G, qscale, bc_top, P.h[2] * P.h[2], d.ctr);
}

// Largest |E| (FP64 field, or the FP32 copy of the mixed form) and largest
// fixed-point electron density over all cells, into m[0], m[1] (zeroed by
// the caller): the inputs of the adaptive step size.  Non-negative doubles
// order like their bit patterns, so an integer maximum serves both.
__global__ void k_step_maxima(const E64* __restrict__ E, const float4* __restrict__ E32,
                              const unsigned long long* __restrict__ ne, uint64_t G, unsigned long long* __restrict__ m)
{
    unsigned long long em = 0, nm = 0;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < G; g += (uint64_t)gridDim.x * blockDim.x) {
        const double e = E ? E[g].m : (double)__ldg(E32 + g).w;
        const unsigned long long b = (unsigned long long)__double_as_longlong(e > 0.0 ? e : 0.0);
        em = b > em ? b : em;
        const unsigned long long v = ne[g];
        nm = v > nm ? v : nm;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, em, d), b = __shfl_xor_sync(0xffffffffu, nm, d);
        em = a > em ? a : em;
        nm = b > nm ? b : nm;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(m, em);
        atomicMax(m + 1, nm);
    }
}

void launch_step_maxima(const Params& P, Dev& d, unsigned long long* m, cudaStream_t s)
{
    const uint64_t G = (uint64_t)P.R * P.n3;
    cudaMemsetAsync(m, 0, 2 * sizeof(unsigned long long), s);
    ++g_launches;
    k_step_maxima<<<grid_for(G, 256), 256, 0, s>>>(d.mixed ? nullptr : d.E, d.mixed ? d.E32 : nullptr, d.ne_fix, G, m);
}

void launch_kmc0d(const Params& P, bool mixed, double Em, long long X0, uint32_t nreal, int nsteps, long long* X,
                  Counters* ctr, cudaStream_t s)
{
    ++g_launches;
    const int blocks = grid_for(nreal, 128, 152 * 64);
    if (mixed) k_kmc0d<float><<<blocks, 128, 0, s>>>(P, Em, X0, nreal, nsteps, X, ctr);
    else k_kmc0d<double><<<blocks, 128, 0, s>>>(P, Em, X0, nreal, nsteps, X, ctr);
}

void launch_kmc(const Params& P, Dev& d, uint64_t G, cudaStream_t s)
{
    // The stage's own counters start from zero on every call (firing totals,
    // photon slots, the photon-cell and KMC-cell list lengths, and the
    // absorbed photon weight the particles stage adds after it): a KMC stage
    // run again without a transport stage between must not append to the
    // lists of the previous run, whose lengths are bounded by G only per call.
    static_assert(offsetof(Counters, n_kmc_cells) > offsetof(Counters, ion), "counter layout");
    cudaMemsetAsync(reinterpret_cast<char*>(d.ctr) + offsetof(Counters, ion), 0,
                    offsetof(Counters, n_kmc_cells) + sizeof(unsigned int) - offsetof(Counters, ion), s);
    // the merge's tier-0 list is free until the merge scan of this step
    g_launches += 2;
    k_kmc_list<<<grid_for(G, 256, 152 * 32), 256, 0, s>>>(P, d.Xe, d.Npos, d.Nneg, d.fired, d.gain, G, d.small_list,
                                                          d.ctr);
    const int nb = grid_for(G, 128, 152 * 64);
    const bool rec = P.k_ep > 0.0 || P.k_np > 0.0;
    if (d.mixed) {
        if (rec) k_kmc<float, true><<<nb, 128, 0, s>>>(P, d.Xe, d.E, d.E32, d.fired, d.gain, d.Npos, d.Nneg, G, d.small_list,
                                                       d.pc_list, d.ctr);
        else k_kmc<float, false><<<nb, 128, 0, s>>>(P, d.Xe, d.E, d.E32, d.fired, d.gain, d.Npos, d.Nneg, G, d.small_list,
                                                    d.pc_list, d.ctr);
    } else {
        if (rec) k_kmc<double, true><<<nb, 128, 0, s>>>(P, d.Xe, d.E, d.E32, d.fired, d.gain, d.Npos, d.Nneg, G, d.small_list,
                                                        d.pc_list, d.ctr);
        else k_kmc<double, false><<<nb, 128, 0, s>>>(P, d.Xe, d.E, d.E32, d.fired, d.gain, d.Npos, d.Nneg, G, d.small_list,
                                                     d.pc_list, d.ctr);
    }
}

// Part a: loss removal, photons, merge scan (offsets, output count, work).
// G: physical cells (photons); the loss and the merge scan run over the
// particle cells of every species block.
void launch_particles_a(const Params& P, Dev& d, uint64_t G, cudaStream_t s)
{
    const uint64_t Gp = (uint64_t)P.B * P.n3;
    cudaMemsetAsync(d.photo_cnt, 0, G * sizeof(int32_t), s);
    cudaMemsetAsync(d.photo_cursor, 0, G * sizeof(int32_t), s);
    cudaMemsetAsync(d.photo_w, 0, G * sizeof(unsigned long long), s);
    uint32_t* wbase = d.mixed ? reinterpret_cast<uint32_t*>(d.rA32) + 3 : reinterpret_cast<uint32_t*>(d.recA) + 7;
    const int wstride = d.mixed ? 4 : 8;
    ++g_launches;
    k_loss<<<grid_for(Gp, 128, 152 * 64), 128, 0, s>>>(P, wbase, wstride, d.cell_start, d.Xe, d.gain, Gp);
    if (P.photon_ratio > 0.0) {
        ++g_launches;
        k_photons<<<152 * 16, 256, 0, s>>>(P, d.mixed ? 1 : 0, d.fired, G, d.pc_list, d.photos, d.photo_cap,
                                            d.photo_cnt, d.photo_w, d.Npos, d.ctr);
    }
    MergeScanOp op{ d.Xe, d.gain, d.photo_w, d.photo_cnt, d.cell_start, d.out_start, d.photo_off, d.work_off,
                    d.small_list, d.mid_list, d.big_list, d.list_n, Gp, G, P.ppc, P.n_new,
                    d.mixed ? (int)sizeof(MP32) : (int)sizeof(MP), d.mixed ? 4 : 8 };
    run_scan<6>(op, Gp, d.scan_blk, s);
}


template <bool MX>
void launch_merge_tiers(const Params& P, Dev& d, uint64_t G, cudaStream_t s, const P64* A, const P32* A32, P64* out,
                        P32* out32, uint32_t* cout)
{
    using E = typename std::conditional<MX, MP32, MP>::type;
    using K = typename EKey<E>::K;
    const uint32_t cap0 = merge_cap0((int)sizeof(E));
    const MLayout L0 = merge_layout(cap0, P.ppc, sizeof(E), sizeof(K));
    const MLayout L1 = merge_layout(MERGE_CAP1, P.ppc, sizeof(E), sizeof(K));
    const size_t sm0 = (size_t)L0.bytes * MERGE_NW0, sm1 = (size_t)L1.bytes * MERGE_NW1;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_merge_lv<E, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    g_launches += 3;
    // tiers 1 and 2 (few, long cells) on the side stream beside tier 0
    cudaStream_t s12 = s;
    if (d.side) {
        cudaEventRecord(d.side_fork, s);
        cudaStreamWaitEvent(d.side, d.side_fork, 0);
        s12 = d.side;
    }
    k_merge_lv<E, false><<<152 * 8, MERGE_NW1 * 32, sm1, s12>>>(
        P, A, A32, d.cell_start, d.gain, d.photos, d.photo_sorted, d.photo_off, d.out_start, d.work_off, d.work,
        d.work_cap, out, out32, cout, (uint64_t)P.R * P.n3, d.mover_cap, d.photo_cap, d.mid_list, d.list_n, 1, MERGE_CAP1, d.ctr);
    k_merge_lv<E, true><<<152 * 4, 128, 0, s12>>>(
        P, A, A32, d.cell_start, d.gain, d.photos, d.photo_sorted, d.photo_off, d.out_start, d.work_off, d.work,
        d.work_cap, out, out32, cout, (uint64_t)P.R * P.n3, d.mover_cap, d.photo_cap, d.big_list, d.list_n, 2, 0, d.ctr);
    k_merge_lv<E, false><<<152 * 16, MERGE_NW0 * 32, sm0, s>>>(
        P, A, A32, d.cell_start, d.gain, d.photos, d.photo_sorted, d.photo_off, d.out_start, d.work_off, d.work,
        d.work_cap, out, out32, cout, (uint64_t)P.R * P.n3, d.mover_cap, d.photo_cap, d.small_list, d.list_n, 0, cap0, d.ctr);
    if (d.side) {
        cudaEventRecord(d.side_join, d.side);
        cudaStreamWaitEvent(s, d.side_join, 0);
    }
}

void launch_merges(const Params& P, Dev& d, uint64_t G, cudaStream_t s)
{
    if (d.mixed) {
        launch_merge_tiers<true>(P, d, G, s, nullptr, d.rA32, nullptr, d.rB32, d.cellB32);
        P32* t = d.rA32; d.rA32 = d.rB32; d.rB32 = t;
        uint32_t* tc = d.cellA32; d.cellA32 = d.cellB32; d.cellB32 = tc;
    } else {
        launch_merge_tiers<false>(P, d, G, s, d.recA, nullptr, d.recB, nullptr, nullptr);
        P64* t = d.recA; d.recA = d.recB; d.recB = t;
    }
}

// Part b (after the host has checked the output count and work size):
// photoelectron grouping and the merge/split itself.
void launch_particles_b(const Params& P, Dev& d, uint64_t G, cudaStream_t s)
{
    if (P.photon_ratio > 0.0) {
        ++g_launches;
        k_photo_place<<<grid_for(d.photo_cap, 256, 1024), 256, 0, s>>>(d.photos, d.ctr, d.photo_cap, d.photo_off,
                                                                      d.photo_cursor, d.photo_sorted);
    }
    launch_merges(P, d, (uint64_t)P.B * P.n3, s);
    uint32_t* u = d.cell_start; d.cell_start = d.out_start; d.out_start = u;
}

}  // namespace ik
