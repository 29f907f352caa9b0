// ik_field.cu -- field solve (a5): lap(phi) = -rho/eps0, E = -grad(phi).
//
// Sec. 4.3: finite-volume discretisation (the 3D standard stencil is the
// 7-point one) solved by geometric multigrid V-cycles with red-black
// Gauss-Seidel smoothing, exit at a relative residual of 1e-10.  Boundary
// conditions of Sec. 5.1: plane electrodes (Dirichlet, phi = 0 at z = lo,
// E0 L at z = hi; ghost 2 phi_b - phi_1) and homogeneous Neumann side faces
// (ghost = phi_1).  Cell-centred hierarchy down to 4^3: averaging
// restriction, trilinear cell-centred prolongation, and a one-block
// red-black solve at the bottom (the paper uses BiCGSTAB there).
//
// Two forms: FP64 V-cycles on the FP64 system, or FP32 V-cycles on the
// correction equation inside FP64 residual iterative refinement
// (phi += V32(b - A phi) until the FP64 residual meets the tolerance).
// Realizations are stacked (slowest index) and solved together; each has
// its own convergence test.  Norms are reduced in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/itokmc.h"
#include "ik_common.cuh"
#include "ik_state.h"

namespace ik {

namespace {

struct Geo {      // one level, all realizations
    int n, log2n, R;
    uint64_t cells;   // R n^3
};

__device__ __forceinline__ void decode(uint64_t t, int log2n, int& r, int& k, int& j, int& i)
{
    const int n = 1 << log2n;
    i = (int)(t & (uint64_t)(n - 1));
    j = (int)((t >> log2n) & (uint64_t)(n - 1));
    k = (int)((t >> (2 * log2n)) & (uint64_t)(n - 1));
    r = (int)(t >> (3 * log2n));
}

// Sum of interior neighbours and the diagonal count n_int + 2 n_D of the
// homogeneous operator at (k, j, i).
template <class T>
__device__ __forceinline__ T nbr_sum(const T* __restrict__ phi, uint64_t idx, int n, int i, int j, int k,
                                     int& diag)
{
    const uint64_t sy = (uint64_t)n, sz = (uint64_t)n * n;
    T s = 0;
    diag = 0;
    if (i > 0) { s = phi[idx - 1]; ++diag; }     // the sum starts at the first neighbour
    if (i < n - 1) { s += phi[idx + 1]; ++diag; }
    if (j > 0) { s += phi[idx - sy]; ++diag; }
    if (j < n - 1) { s += phi[idx + sy]; ++diag; }
    if (k > 0) { s += phi[idx - sz]; ++diag; } else diag += 2;
    if (k < n - 1) { s += phi[idx + sz]; ++diag; } else diag += 2;
    return s;
}

// diag as a T without a conversion instruction.
template <class T>
__device__ __forceinline__ T diag_val(int d)
{
    switch (d) {
    case 4: return (T)4;
    case 5: return (T)5;
    case 6: return (T)6;
    case 7: return (T)7;
    case 8: return (T)8;
    case 9: return (T)9;
    default: return (T)d;
    }
}

// 1/diag for the diagonal counts 1..8 (a multiply instead of a divide).
template <class T>
__device__ __forceinline__ T inv_diag(int d)
{
    switch (d) {
    case 4: return (T)(1.0 / 4.0);
    case 5: return (T)(1.0 / 5.0);
    case 6: return (T)(1.0 / 6.0);
    case 7: return (T)(1.0 / 7.0);
    case 8: return (T)(1.0 / 8.0);
    case 9: return (T)(1.0 / 9.0);
    default: return (T)1 / (T)d;
    }
}

template <class T>
__global__ void k_smooth(T* __restrict__ phi, const T* __restrict__ rhs, Geo G, int color)
{
    const uint64_t half = G.cells >> 1;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < half; t += (uint64_t)gridDim.x * blockDim.x) {
        // t enumerates (r, k, j, ih); i = 2 ih + parity
        const int n = G.n;
        const int ih = (int)(t & (uint64_t)(n / 2 - 1));
        const int j = (int)((t >> (G.log2n - 1)) & (uint64_t)(n - 1));
        const int k = (int)((t >> (2 * G.log2n - 1)) & (uint64_t)(n - 1));
        const uint64_t r = t >> (3 * G.log2n - 1);
        const int i = 2 * ih + ((j + k + color) & 1);
        const uint64_t idx = ((r * n + k) * n + j) * n + i;
        int diag;
        const T s = nbr_sum(phi, idx, n, i, j, k, diag);
        phi[idx] = (s - rhs[idx]) * inv_diag<T>(diag);
    }
}

// Residual at fine cells, averaged over the 8 children of each coarse cell
// into the coarse right-hand side.  Every level stores h^2 b (the multigrid
// systems are scaled by h^2), so the coarse value h_c^2 mean(r) is half the
// sum of the children's h_f^2 r = h_f^2 b - (neighbour sum - diag phi).
template <class T, class TC>
__global__ void k_resid_restrict(const T* __restrict__ phi, const T* __restrict__ rhs, TC* __restrict__ rhs_c,
                                 Geo Gc, int nf)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < Gc.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        int r, K, J, I;
        decode(t, Gc.log2n, r, K, J, I);
        T acc = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
            const uint64_t idx = (((uint64_t)r * nf + k) * nf + j) * nf + i;
            int diag;
            const T s = nbr_sum(phi, idx, nf, i, j, k, diag);
            acc += fma(diag_val<T>(diag), phi[idx], rhs[idx] - s);
        }
        rhs_c[t] = (TC)(acc * (T)0.5);
    }
}

// phi_f += trilinear cell-centred interpolation of the coarse correction:
// weights 3/4, 1/4 per axis written as (3 a + b) / 4 with fused multiply-
// adds (ghosts: Neumann e, Dirichlet -e, i.e. (3 a - a) / 4 in z).
template <class T>
__device__ __forceinline__ T prolong_at(const T* __restrict__ ec, int nc, int i, int j, int k)
{
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    int I2 = I + ((i & 1) ? 1 : -1), J2 = J + ((j & 1) ? 1 : -1), K2 = K + ((k & 1) ? 1 : -1);
    T sz = (T)1;
    if (I2 < 0 || I2 >= nc) I2 = I;
    if (J2 < 0 || J2 >= nc) J2 = J;
    if (K2 < 0 || K2 >= nc) { K2 = K; sz = (T)-1; }
    const int iz[2] = { K, K2 }, iy[2] = { J, J2 };
    T m[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        T q[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const T* row = ec + ((uint64_t)iz[c] * nc + iy[b]) * nc;
            q[b] = fma((T)3, row[I], row[I2]);
        }
        m[c] = fma((T)3, q[0], q[1]);
    }
    return fma((T)3, m[0], sz * m[1]) * (T)(1.0 / 64.0);
}

template <class T>
__global__ void k_prolong(T* __restrict__ phi_f, const T* __restrict__ e_c, Geo Gf)
{
    const int nc = Gf.n / 2;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < Gf.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        int r, k, j, i;
        decode(t, Gf.log2n, r, k, j, i);
        phi_f[t] += prolong_at(e_c + (uint64_t)r * nc * nc * nc, nc, i, j, k);
    }
}

// Bottom solve: one block per realization, red-black sweeps in shared memory.
template <class T>
__global__ void k_bottom(T* __restrict__ phi, const T* __restrict__ rhs, int n, int sweeps)
{
    extern __shared__ unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);
    T* b = s + n * n * n;
    const int cells = n * n * n;
    const uint64_t base = (uint64_t)blockIdx.x * cells;
    for (int c = threadIdx.x; c < cells; c += blockDim.x) { s[c] = phi[base + c]; b[c] = rhs[base + c]; }
    __syncthreads();
    for (int it = 0; it < sweeps; ++it) {
        for (int color = 0; color < 2; ++color) {
            for (int c = threadIdx.x; c < cells; c += blockDim.x) {
                const int i = c % n, j = (c / n) % n, k = c / (n * n);
                if (((i + j + k) & 1) != color) continue;
                int diag;
                const T sum = nbr_sum(s, (uint64_t)c, n, i, j, k, diag);
                s[c] = (sum - b[c]) * inv_diag<T>(diag);
            }
            __syncthreads();
        }
    }
    for (int c = threadIdx.x; c < cells; c += blockDim.x) phi[base + c] = s[c];
}

// FP64 residual, its squared norm per block (fixed order), and optionally
// the FP32 copy for the inner V-cycle.  A block covers items*256 cells of
// one realization.
constexpr int NORM_TPB = 256;

__global__ void __launch_bounds__(NORM_TPB) k_resid_norm(const double* __restrict__ phi, const double* __restrict__ rhs,
                                                         float* __restrict__ r32, Geo G,
                                                         double* __restrict__ part, int with_b, int items)
{
    __shared__ double red[NORM_TPB / 32][2];
    const uint64_t base = ((uint64_t)blockIdx.x * NORM_TPB) * items;
    double acc = 0.0, bacc = 0.0;
    for (int q = 0; q < items; ++q) {
        const uint64_t t = base + (uint64_t)q * NORM_TPB + threadIdx.x;
        if (t >= G.cells) break;
        int r, k, j, i;
        decode(t, G.log2n, r, k, j, i);
        int diag;
        const double s = nbr_sum(phi, t, G.n, i, j, k, diag);
        const double res = rhs[t] - (s - (double)diag * phi[t]);
        if (r32) r32[t] = (float)res;
        acc = __fma_rn(res, res, acc);
        if (with_b) bacc = __fma_rn(rhs[t], rhs[t], bacc);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, d);
        bacc += __shfl_xor_sync(0xffffffffu, bacc, d);
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = acc; red[threadIdx.x >> 5][1] = bacc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < NORM_TPB / 32; ++w) { a += red[w][0]; b += red[w][1]; }
        part[2 * (uint64_t)blockIdx.x] = a;
        part[2 * (uint64_t)blockIdx.x + 1] = b;
    }
}

// Per realization (one block each): fixed-order strided sums, then a fixed
// tree in shared memory -- the same result on every run.
__global__ void __launch_bounds__(256) k_norm_final(const double* __restrict__ part, int blocks_per_real, int R,
                                                    double* __restrict__ out)
{
    __shared__ double sa[256], sb[256];
    const int r = blockIdx.x;
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < blocks_per_real; q += 256) {
        a += part[2 * ((uint64_t)r * blocks_per_real + q)];
        b += part[2 * ((uint64_t)r * blocks_per_real + q) + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * r] = sa[0];
        out[2 * r + 1] = sb[0];
    }
}

__global__ void k_add_correction(double* __restrict__ phi, const float* __restrict__ e, uint64_t cells)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cells; t += (uint64_t)gridDim.x * blockDim.x)
        phi[t] += (double)e[t];
}

// ---- fixed-point potential (mixed field form)
// The potential is held as Phi = phi 2^F (int64) and the right-hand side as
// B = round(h^2 2^F b), so the residual h^2 2^F (b - A phi) = B - (sum of
// neighbours - diag Phi) is exact integer arithmetic (FP64 runs at a small
// fraction of the integer rate on GB300).  The FP32 residual r = R 2^-F / h^2
// feeds the FP32 correction V-cycles; squared norms are summed in FP32 per
// thread and FP64 across the block in a fixed order.
constexpr long long PHI_LIM = 1ll << 59;

__global__ void __launch_bounds__(NORM_TPB) k_resid_fixed(const long long* __restrict__ Phi,
                                                          const long long* __restrict__ B, float* __restrict__ r32,
                                                          Geo G, float sc, double* __restrict__ part, int with_b,
                                                          int items)
{
    __shared__ double red[NORM_TPB / 32][2];
    const uint64_t base = ((uint64_t)blockIdx.x * NORM_TPB) * items;
    float acc = 0.f, bacc = 0.f;
    bool bad = false;
    for (int q = 0; q < items; ++q) {
        const uint64_t t = base + (uint64_t)q * NORM_TPB + threadIdx.x;
        if (t >= G.cells) break;
        int r, k, j, i;
        decode(t, G.log2n, r, k, j, i);
        int diag;
        const long long s = nbr_sum(Phi, t, G.n, i, j, k, diag);
        const long long pc = Phi[t];
        bad |= pc >= PHI_LIM || pc <= -PHI_LIM;
        const long long b = B[t];
        const float res = __ll2float_rn(b - (s - (long long)diag * pc)) * sc;
        r32[t] = res;
        acc = __fmaf_rn(res, res, acc);
        if (with_b) {
            const float bf = __ll2float_rn(b) * sc;
            bacc = __fmaf_rn(bf, bf, bacc);
        }
    }
    double a = bad ? (double)INFINITY : (double)acc, bb = (double)bacc;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, d);
        bb += __shfl_xor_sync(0xffffffffu, bb, d);
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = a; red[threadIdx.x >> 5][1] = bb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < NORM_TPB / 32; ++w) { x += red[w][0]; y += red[w][1]; }
        part[2 * (uint64_t)blockIdx.x] = x;
        part[2 * (uint64_t)blockIdx.x + 1] = y;
    }
}

// Phi += round(e 2^F) for the FP32 correction e (volts).
__global__ void k_add_fixed(long long* __restrict__ Phi, const float* __restrict__ e, float scale, uint64_t cells)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cells; t += (uint64_t)gridDim.x * blockDim.x)
        Phi[t] += __float2ll_rn(e[t] * scale);
}

// E = -grad(phi) from the fixed-point potential: the neighbour differences
// are exact integers, scaled by 2^-F / 2h (FP64 into E64 and/or FP32 into E32).
__global__ void k_efield_fixed(const long long* __restrict__ Phi, E64* __restrict__ E, float4* __restrict__ E32,
                               Geo G, double sc, long long Phi_top)
{
    const float scf = (float)sc;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < G.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        int r, k, j, i;
        decode(t, G.log2n, r, k, j, i);
        const int n = G.n;
        const uint64_t sy = (uint64_t)n, sz = (uint64_t)n * n;
        const long long c = Phi[t];
        const long long xm = i > 0 ? Phi[t - 1] : c, xp = i < n - 1 ? Phi[t + 1] : c;
        const long long ym = j > 0 ? Phi[t - sy] : c, yp = j < n - 1 ? Phi[t + sy] : c;
        const long long zm = k > 0 ? Phi[t - sz] : -c, zp = k < n - 1 ? Phi[t + sz] : 2 * Phi_top - c;
        if (E) {
            const double ex = (double)(xm - xp) * sc, ey = (double)(ym - yp) * sc, ez = (double)(zm - zp) * sc;
            const double m = sqrt((ex * ex + ey * ey) + ez * ez);
            reinterpret_cast<double2*>(E + t)[0] = make_double2(ex, ey);
            reinterpret_cast<double2*>(E + t)[1] = make_double2(ez, m);
            if (E32) E32[t] = make_float4((float)ex, (float)ey, (float)ez, (float)m);
        } else {
            const float ex = __ll2float_rn(xm - xp) * scf, ey = __ll2float_rn(ym - yp) * scf,
                        ez = __ll2float_rn(zm - zp) * scf;
            E32[t] = make_float4(ex, ey, ez, sqrtf(ex * ex + ey * ey + ez * ez));
        }
    }
}

// B = round(b h^2 2^F) with b formed exactly as the FP64 right-hand side.
__global__ void k_rhs_fixed(const int64_t* __restrict__ rho, long long* __restrict__ B, Geo G, double qscale,
                            double bc_top, double bfix)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < G.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        const int k = (int)((t >> (2 * G.log2n)) & (uint64_t)(G.n - 1));
        double b = -((double)rho[t] * qscale);
        if (k == G.n - 1) b = b - bc_top;
        B[t] = __double2ll_rn(b * bfix);
    }
}

// Phi <- round(Phi 2^-sh) when the fixed-point scale is lowered.
__global__ void k_shift_fixed(long long* __restrict__ Phi, int sh, uint64_t cells)
{
    const long long half = 1ll << (sh - 1);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cells; t += (uint64_t)gridDim.x * blockDim.x)
        Phi[t] = (Phi[t] + half) >> sh;
}

// phi <- 2 phi - prev, prev <- the old phi (with no previous potential yet:
// prev <- phi only).
template <class T>
__global__ void k_extrapolate(T* __restrict__ phi, T* __restrict__ prev, uint64_t cells, bool have)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cells; t += (uint64_t)gridDim.x * blockDim.x) {
        const T v = phi[t];
        if (have) phi[t] = (v + v) - prev[t];
        prev[t] = v;
    }
}

__global__ void k_phi_to_double(const long long* __restrict__ Phi, double* __restrict__ out, double sc, uint64_t cells)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cells; t += (uint64_t)gridDim.x * blockDim.x)
        out[t] = (double)Phi[t] * sc;
}

template <class T>
__global__ void k_zero(T* __restrict__ a, uint64_t cells)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cells; t += (uint64_t)gridDim.x * blockDim.x)
        a[t] = (T)0;
}

// E = -grad(phi) by centred differences with the boundary ghosts, and |E|.
// FP64 form: everything in FP64 into E64.  Mixed form (E == nullptr): the
// differences of neighbouring potentials in FP64 (they cancel most digits),
// the scaling and |E| in FP32, into E32 only.
__global__ void k_efield(const double* __restrict__ phi, E64* __restrict__ E, float4* __restrict__ E32, Geo G,
                         double h, double phi_top)
{
    const float inv2h = (float)(1.0 / (2.0 * h));
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < G.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        int r, k, j, i;
        decode(t, G.log2n, r, k, j, i);
        const int n = G.n;
        const uint64_t sy = (uint64_t)n, sz = (uint64_t)n * n;
        const double c = phi[t];
        const double xm = i > 0 ? phi[t - 1] : c, xp = i < n - 1 ? phi[t + 1] : c;
        const double ym = j > 0 ? phi[t - sy] : c, yp = j < n - 1 ? phi[t + sy] : c;
        const double zm = k > 0 ? phi[t - sz] : -c, zp = k < n - 1 ? phi[t + sz] : 2.0 * phi_top - c;
        if (E) {
            const double ex = (xm - xp) / (2.0 * h), ey = (ym - yp) / (2.0 * h), ez = (zm - zp) / (2.0 * h);
            const double m = sqrt((ex * ex + ey * ey) + ez * ez);
            reinterpret_cast<double2*>(E + t)[0] = make_double2(ex, ey);
            reinterpret_cast<double2*>(E + t)[1] = make_double2(ez, m);
            if (E32) E32[t] = make_float4((float)ex, (float)ey, (float)ez, (float)m);
        } else {
            const float ex = (float)(xm - xp) * inv2h, ey = (float)(ym - yp) * inv2h, ez = (float)(zm - zp) * inv2h;
            E32[t] = make_float4(ex, ey, ez, sqrtf(ex * ex + ey * ey + ez * ez));
        }
    }
}

int gridsz(uint64_t n, int tpb) {
    uint64_t b = (n + tpb - 1) / tpb;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

Geo geo(const Dev& d, int l, int R)
{
    Geo g;
    g.n = d.lev[l].n;
    g.log2n = 0;
    while ((1 << g.log2n) < g.n) ++g.log2n;
    g.R = R;
    g.cells = (uint64_t)R * g.n * g.n * g.n;
    return g;
}

// ---------------------------------------------------------------------------
// The coarse end of the V-cycle (levels of at most 16^3 cells) in one launch:
// one block per realization runs pre-smoothing, residual restriction, the
// bottom sweeps, prolongation and post-smoothing level by level, with block
// barriers between the phases (the arrays are tiny and stay in cache).
constexpr int COARSE_N = 16;

struct CoarseLevels {
    int nlev;            // levels in the fused range, finest first
    int n[MAX_LEVELS];
    void* phi[MAX_LEVELS];
    void* rhs[MAX_LEVELS];
};

template <class T>
__device__ void blk_smooth(T* phi, const T* rhs, int n, int color)
{
    const int half = n * n * n / 2;
    for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int ih = t % (n / 2), j = (t / (n / 2)) % n, k = t / (n * n / 2);
        const int i = 2 * ih + ((j + k + color) & 1);
        const uint64_t idx = ((uint64_t)k * n + j) * n + i;
        int diag;
        const T sum = nbr_sum(phi, idx, n, i, j, k, diag);
        phi[idx] = (sum - rhs[idx]) * inv_diag<T>(diag);
    }
    __syncthreads();
}

template <class T>
__device__ void blk_resid_restrict(const T* phi, const T* rhs, T* rhs_c, int nf)
{
    const int nc = nf / 2;
    for (int t = threadIdx.x; t < nc * nc * nc; t += blockDim.x) {
        const int I = t % nc, J = (t / nc) % nc, K = t / (nc * nc);
        T acc = 0;
        for (int c = 0; c < 8; ++c) {
            const int i = 2 * I + (c & 1), j = 2 * J + ((c >> 1) & 1), k = 2 * K + (c >> 2);
            const uint64_t idx = ((uint64_t)k * nf + j) * nf + i;
            int diag;
            const T sum = nbr_sum(phi, idx, nf, i, j, k, diag);
            acc += fma(diag_val<T>(diag), phi[idx], rhs[idx] - sum);
        }
        rhs_c[t] = acc * (T)0.5;
    }
    __syncthreads();
}

template <class T>
__device__ void blk_prolong(T* phi_f, const T* e_c, int nf)
{
    const int nc = nf / 2;
    for (int t = threadIdx.x; t < nf * nf * nf; t += blockDim.x) {
        const int i = t % nf, j = (t / nf) % nf, k = t / (nf * nf);
        phi_f[t] += prolong_at(e_c, nc, i, j, k);
    }
    __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(1024) k_vcycle_coarse(CoarseLevels C, int nu1, int nu2, int bottom_sweeps)
{
    const int r = blockIdx.x;
    auto PHI = [&](int l) { return reinterpret_cast<T*>(C.phi[l]) + (uint64_t)r * C.n[l] * C.n[l] * C.n[l]; };
    auto RHS = [&](int l) { return reinterpret_cast<T*>(C.rhs[l]) + (uint64_t)r * C.n[l] * C.n[l] * C.n[l]; };
    const int L = C.nlev - 1;
    for (int l = 0; l < L; ++l) {
        for (int it = 0; it < nu1; ++it) {
            blk_smooth<T>(PHI(l), RHS(l), C.n[l], 0);
            blk_smooth<T>(PHI(l), RHS(l), C.n[l], 1);
        }
        blk_resid_restrict<T>(PHI(l), RHS(l), RHS(l + 1), C.n[l]);
        T* pc = PHI(l + 1);
        for (int t = threadIdx.x; t < C.n[l + 1] * C.n[l + 1] * C.n[l + 1]; t += blockDim.x) pc[t] = (T)0;
        __syncthreads();
    }
    for (int it = 0; it < bottom_sweeps; ++it) {
        blk_smooth<T>(PHI(L), RHS(L), C.n[L], 0);
        blk_smooth<T>(PHI(L), RHS(L), C.n[L], 1);
    }
    for (int l = L - 1; l >= 0; --l) {
        blk_prolong<T>(PHI(l), PHI(l + 1), C.n[l]);
        for (int it = 0; it < nu2; ++it) {
            blk_smooth<T>(PHI(l), RHS(l), C.n[l], 1);
            blk_smooth<T>(PHI(l), RHS(l), C.n[l], 0);
        }
    }
}

template <class T>
T* lphi(MGLevel& L);
template <>
double* lphi<double>(MGLevel& L) { return L.phi; }
template <>
float* lphi<float>(MGLevel& L) { return L.phi32; }
template <class T>
T* lrhs(MGLevel& L);
template <>
double* lrhs<double>(MGLevel& L) { return L.rhs; }
template <>
float* lrhs<float>(MGLevel& L) { return L.rhs32; }

template <class T>
void vcycle(Dev& d, int l, int R, int nu1, int nu2, cudaStream_t s)
{
    MGLevel& L = d.lev[l];
    const Geo G = geo(d, l, R);
    T* phi = lphi<T>(L);
    T* rhs = lrhs<T>(L);
    if (L.n <= COARSE_N && d.nlev - l >= 2) {
        CoarseLevels C{};
        C.nlev = d.nlev - l;
        for (int q = 0; q < C.nlev; ++q) {
            MGLevel& M = d.lev[l + q];
            C.n[q] = M.n;
            C.phi[q] = lphi<T>(M);
            C.rhs[q] = lrhs<T>(M);
        }
        ++g_launches;
        k_vcycle_coarse<T><<<R, 1024, 0, s>>>(C, nu1, nu2, 48);
        return;
    }
    if (l == d.nlev - 1) {
        const int cells = G.n * G.n * G.n;
        const size_t sm = 2 * sizeof(T) * cells;
        ++g_launches;
        k_bottom<T><<<R, 256, sm, s>>>(phi, rhs, G.n, 48);
        return;
    }
    const int tpb = 256;
    for (int it = 0; it < nu1; ++it) {
        ++g_launches;
        k_smooth<T><<<gridsz(G.cells / 2, tpb), tpb, 0, s>>>(phi, rhs, G, 0);
        ++g_launches;
        k_smooth<T><<<gridsz(G.cells / 2, tpb), tpb, 0, s>>>(phi, rhs, G, 1);
    }
    MGLevel& C = d.lev[l + 1];
    const Geo Gc = geo(d, l + 1, R);
    ++g_launches;
    k_resid_restrict<T, T><<<gridsz(Gc.cells, tpb), tpb, 0, s>>>(phi, rhs, lrhs<T>(C), Gc, G.n);
    ++g_launches;
    k_zero<T><<<gridsz(Gc.cells, tpb), tpb, 0, s>>>(lphi<T>(C), Gc.cells);
    vcycle<T>(d, l + 1, R, nu1, nu2, s);
    ++g_launches;
    k_prolong<T><<<gridsz(G.cells, tpb), tpb, 0, s>>>(phi, lphi<T>(C), G);
    for (int it = 0; it < nu2; ++it) {
        ++g_launches;
        k_smooth<T><<<gridsz(G.cells / 2, tpb), tpb, 0, s>>>(phi, rhs, G, 1);
        ++g_launches;
        k_smooth<T><<<gridsz(G.cells / 2, tpb), tpb, 0, s>>>(phi, rhs, G, 0);
    }
}


// ------------------------------------------------------------------ semi-implicit
// Variable-coefficient operator of the semi-implicit coupling (Sec. 4.3, Eq.
// poisson_simp): div(c grad phi) with c = 1 + sigma dt / eps0 per cell; the
// coefficient of an interior face is the mean of its two cells', a boundary
// face takes the cell's own (Neumann sides: no flux; Dirichlet electrodes:
// ghost 2 phi_b - phi_1, i.e. 2 c on the diagonal).  With c = 1 it is the
// operator above.  The systems are scaled by h^2 like the constant-
// coefficient ones.  Per level the face coefficients (fx, fy, fz: the +x,
// +y, +z face of each cell, 0 on the boundary), the diagonal and its
// inverse are formed once per solve (k_vc_faces), so a smoothing update is
// six fused multiply-adds and one multiply.
__global__ void k_vc_faces(const double* __restrict__ c, double* __restrict__ fx, double* __restrict__ fy,
                           double* __restrict__ fz, double* __restrict__ dg, double* __restrict__ idg, Geo G)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < G.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        int r, k, j, i;
        decode(t, G.log2n, r, k, j, i);
        const int n = G.n;
        const uint64_t sy = (uint64_t)n, sz = (uint64_t)n * n;
        const double ci = c[t];
        const double xm = i > 0 ? 0.5 * (c[t - 1] + ci) : 0.0, xp = i < n - 1 ? 0.5 * (ci + c[t + 1]) : 0.0;
        const double ym = j > 0 ? 0.5 * (c[t - sy] + ci) : 0.0, yp = j < n - 1 ? 0.5 * (ci + c[t + sy]) : 0.0;
        const double zm = k > 0 ? 0.5 * (c[t - sz] + ci) : 2.0 * ci, zp = k < n - 1 ? 0.5 * (ci + c[t + sz]) : 2.0 * ci;
        fx[t] = xp;
        fy[t] = yp;
        fz[t] = k < n - 1 ? zp : 0.0;
        const double d = ((((xm + xp) + ym) + yp) + zm) + zp;
        dg[t] = d;
        idg[t] = 1.0 / d;
    }
}

// Off-diagonal sum of the variable-coefficient operator at (k, j, i).
__device__ __forceinline__ double vcf_sum(const double* __restrict__ phi, const double* __restrict__ fx,
                                          const double* __restrict__ fy, const double* __restrict__ fz, uint64_t idx,
                                          int n, int i, int j, int k)
{
    const uint64_t sy = (uint64_t)n, sz = (uint64_t)n * n;
    double s = 0.0;
    if (i > 0) s = __fma_rn(fx[idx - 1], phi[idx - 1], s);
    if (i < n - 1) s = __fma_rn(fx[idx], phi[idx + 1], s);
    if (j > 0) s = __fma_rn(fy[idx - sy], phi[idx - sy], s);
    if (j < n - 1) s = __fma_rn(fy[idx], phi[idx + sy], s);
    if (k > 0) s = __fma_rn(fz[idx - sz], phi[idx - sz], s);
    if (k < n - 1) s = __fma_rn(fz[idx], phi[idx + sz], s);
    return s;
}

struct VCArrays {        // one level's operator (kernel argument)
    const double* fx;
    const double* fy;
    const double* fz;
    const double* dg;
    const double* idg;
};

__global__ void k_smooth_vc(double* __restrict__ phi, const double* __restrict__ rhs, VCArrays A, Geo G, int color)
{
    const uint64_t half = G.cells >> 1;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < half; t += (uint64_t)gridDim.x * blockDim.x) {
        const int n = G.n;
        const int ih = (int)(t & (uint64_t)(n / 2 - 1));
        const int j = (int)((t >> (G.log2n - 1)) & (uint64_t)(n - 1));
        const int k = (int)((t >> (2 * G.log2n - 1)) & (uint64_t)(n - 1));
        const uint64_t r = t >> (3 * G.log2n - 1);
        const int i = 2 * ih + ((j + k + color) & 1);
        const uint64_t idx = ((r * n + k) * n + j) * n + i;
        const double sum = vcf_sum(phi, A.fx, A.fy, A.fz, idx, n, i, j, k);
        phi[idx] = (sum - rhs[idx]) * A.idg[idx];
    }
}

// Residual h^2 (b - A phi) at fine cells, half the sum of 8 children into the
// coarse right-hand side (the convention of k_resid_restrict).
__global__ void k_resid_restrict_vc(const double* __restrict__ phi, const double* __restrict__ rhs, VCArrays A,
                                    double* __restrict__ rhs_c, Geo Gc, int nf)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < Gc.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        int r, K, J, I;
        decode(t, Gc.log2n, r, K, J, I);
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
            const uint64_t idx = (((uint64_t)r * nf + k) * nf + j) * nf + i;
            const double sum = vcf_sum(phi, A.fx, A.fy, A.fz, idx, nf, i, j, k);
            acc += rhs[idx] - __fma_rn(-A.dg[idx], phi[idx], sum);
        }
        rhs_c[t] = acc * 0.5;
    }
}

// Coarse coefficient: the mean of the 8 children.
__global__ void k_coef_restrict(const double* __restrict__ cf, double* __restrict__ cc, Geo Gc, int nf)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < Gc.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        int r, K, J, I;
        decode(t, Gc.log2n, r, K, J, I);
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
            acc += cf[(((uint64_t)r * nf + k) * nf + j) * nf + i];
        }
        cc[t] = acc * 0.125;
    }
}

// The coarse end of the variable-coefficient V-cycle (levels of at most 16^3
// cells) in one launch, one block per realization (as k_vcycle_coarse).
struct CoarseVC {
    int nlev;
    int n[MAX_LEVELS];
    double* phi[MAX_LEVELS];
    double* rhs[MAX_LEVELS];
    VCArrays A[MAX_LEVELS];
};

__device__ void blk_smooth_vc(double* phi, const double* rhs, const VCArrays& A, uint64_t off, int n, int color)
{
    const int half = n * n * n / 2;
    for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int ih = t % (n / 2), j = (t / (n / 2)) % n, k = t / (n * n / 2);
        const int i = 2 * ih + ((j + k + color) & 1);
        const uint64_t idx = ((uint64_t)k * n + j) * n + i;
        const double sum = vcf_sum(phi, A.fx + off, A.fy + off, A.fz + off, idx, n, i, j, k);
        phi[idx] = (sum - rhs[idx]) * A.idg[off + idx];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(512) k_vcycle_coarse_vc(CoarseVC C, int nu1, int nu2, int bottom_sweeps)
{
    const uint64_t r = blockIdx.x;
    auto cells = [&](int l) { return (uint64_t)C.n[l] * C.n[l] * C.n[l]; };
    const int L = C.nlev - 1;
    for (int l = 0; l < L; ++l) {
        const uint64_t off = r * cells(l);
        double* phi = C.phi[l] + off;
        const double* rhs = C.rhs[l] + off;
        for (int it = 0; it < nu1; ++it) {
            blk_smooth_vc(phi, rhs, C.A[l], off, C.n[l], 0);
            blk_smooth_vc(phi, rhs, C.A[l], off, C.n[l], 1);
        }
        const int nf = C.n[l], nc = nf / 2;
        const uint64_t offc = r * cells(l + 1);
        for (int t = threadIdx.x; t < nc * nc * nc; t += blockDim.x) {
            const int I = t % nc, J = (t / nc) % nc, K = t / (nc * nc);
            double acc = 0.0;
            for (int q = 0; q < 8; ++q) {
                const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + (q >> 2);
                const uint64_t idx = ((uint64_t)k * nf + j) * nf + i;
                const double sum = vcf_sum(phi, C.A[l].fx + off, C.A[l].fy + off, C.A[l].fz + off, idx, nf, i, j, k);
                acc += rhs[idx] - __fma_rn(-C.A[l].dg[off + idx], phi[idx], sum);
            }
            C.rhs[l + 1][offc + t] = acc * 0.5;
            C.phi[l + 1][offc + t] = 0.0;
        }
        __syncthreads();
    }
    {
        const uint64_t off = r * cells(L);
        for (int it = 0; it < bottom_sweeps; ++it) {
            blk_smooth_vc(C.phi[L] + off, C.rhs[L] + off, C.A[L], off, C.n[L], 0);
            blk_smooth_vc(C.phi[L] + off, C.rhs[L] + off, C.A[L], off, C.n[L], 1);
        }
    }
    for (int l = L - 1; l >= 0; --l) {
        const uint64_t off = r * cells(l);
        double* phi = C.phi[l] + off;
        const double* ec = C.phi[l + 1] + r * cells(l + 1);
        const int nf = C.n[l];
        for (int t = threadIdx.x; t < nf * nf * nf; t += blockDim.x) {
            const int i = t % nf, j = (t / nf) % nf, k = t / (nf * nf);
            phi[t] += prolong_at(ec, nf / 2, i, j, k);
        }
        __syncthreads();
        for (int it = 0; it < nu2; ++it) {
            blk_smooth_vc(phi, C.rhs[l] + off, C.A[l], off, nf, 1);
            blk_smooth_vc(phi, C.rhs[l] + off, C.A[l], off, nf, 0);
        }
    }
}

// Squared norms of the residual and of the right-hand side per realization
// (blockIdx.y): one partial pair per block in part[2 (r gridDim.x + x)],
// summed in a fixed order by k_norm_final, so the convergence test (and with
// it the cycle count and the potential) is the same on every run.  256
// threads per block.
__global__ void __launch_bounds__(256) k_resid_norm_vc(const double* __restrict__ phi, const double* __restrict__ rhs,
                                                       VCArrays A, Geo G, double* __restrict__ part)
{
    const uint64_t r = blockIdx.y;
    const uint64_t per = (uint64_t)G.n * G.n * G.n;
    double s0 = 0.0, s1 = 0.0;
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < per; u += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = r * per + u;
        int rr, k, j, i;
        decode(t, G.log2n, rr, k, j, i);
        const double sum = vcf_sum(phi, A.fx, A.fy, A.fz, t, G.n, i, j, k);
        const double res = rhs[t] - __fma_rn(-A.dg[t], phi[t], sum);
        s0 += res * res;
        s1 += rhs[t] * rhs[t];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    __shared__ double w0[8], w1[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { w0[wid] = s0; w1[wid] = s1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += w0[q]; b += w1[q]; }
        const uint64_t o = 2 * (r * gridDim.x + blockIdx.x);
        part[o] = a;
        part[o + 1] = b;
    }
}

// h^2 b = h^2 (-rho/eps0) with the top electrode term weighted by the
// boundary cell's coefficient.
__global__ void k_rhs_vc(const int64_t* __restrict__ rho, const double* __restrict__ c, double* __restrict__ rhs, Geo G,
                         double qscale, double bc_top, double h2)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < G.cells; t += (uint64_t)gridDim.x * blockDim.x) {
        int r, k, j, i;
        decode(t, G.log2n, r, k, j, i);
        double b = -((double)rho[t] * qscale);
        if (k == G.n - 1) b = b - c[t] * bc_top;
        rhs[t] = b * h2;
    }
}

// c = 1 + sigma dt / eps0, sigma = q_e mu n_e (Eq. conductivity) from the
// fixed-point CIC electron count.
__global__ void k_coef_from_ne(const unsigned long long* __restrict__ ne_fix, double* __restrict__ c, uint64_t cells,
                               double per_cell, double qmu, double dt_eps)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < cells; t += (uint64_t)gridDim.x * blockDim.x) {
        const double ne = ((double)ne_fix[t] * per_cell);
        const double sigma = qmu * ne;
        c[t] = 1.0 + sigma * dt_eps;
    }
}

}  // namespace

constexpr int MAX_REAL_NORM = 4096;

// Replays (capturing first if needed) the graph of kind k on stream s:
// k = 0: one FP64 V-cycle; k = 1: zero the FP32 correction, two FP32
// V-cycles.  The launches of a cycle depend only on the level pointers and
// the smoother counts, so one capture per (nu1, nu2) serves every solve.
// Launches directly when d.direct_cycles is set (a solve on per-call
// buffers, whose graphs could not be reused) or capture is not possible.
void run_cycles(Dev& d, int k, int R, int nu1, int nu2, cudaStream_t s)
{
    auto direct = [&]() {
        if (k == 0) {
            vcycle<double>(d, 0, R, nu1, nu2, s);
        } else {
            const Geo G0 = geo(d, 0, R);
            ++g_launches;
            k_zero<float><<<gridsz(G0.cells, 256), 256, 0, s>>>(d.lev[0].phi32, G0.cells);
            vcycle<float>(d, 0, R, nu1, nu2, s);
            vcycle<float>(d, 0, R, nu1, nu2, s);
        }
    };
    if (d.direct_cycles) {
        direct();
        return;
    }
    if (d.vgraph[k] && (d.vgraph_nu[k][0] != nu1 || d.vgraph_nu[k][1] != nu2)) {
        cudaGraphExecDestroy(d.vgraph[k]);
        d.vgraph[k] = nullptr;
    }
    if (!d.vgraph[k]) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            direct();
            return;
        }
        const unsigned long long l0 = g_launches.load();
        direct();
        const unsigned long long nk = g_launches.load() - l0;
        g_launches -= nk;                         // captured, not run
        if (cudaStreamEndCapture(s, &g) != cudaSuccess || !g ||
            cudaGraphInstantiate(&d.vgraph[k], g, 0) != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            d.vgraph[k] = nullptr;
            direct();
            return;
        }
        cudaGraphDestroy(g);
        d.vgraph_nu[k][0] = nu1;
        d.vgraph_nu[k][1] = nu2;
        d.vgraph_kernels[k] = nk;
    }
    g_launches += d.vgraph_kernels[k];
    cudaGraphLaunch(d.vgraph[k], s);
}

// precision: 0 FP64 V-cycles; 1 FP32 V-cycles in FP64 residual refinement;
// 2 FP32 V-cycles in fixed-point residual refinement (potential in units of
// 2^-phi_F V, right-hand side prepared by the charge kernel).  Returns 0 on
// convergence, ITOKMC_ERR_NOCONV (-6) if max_cycles is reached or the
// potential leaves the fixed-point range.
// Lowers the fixed-point potential's scale to F bits (F < d.phi_F): the
// potential and the kept previous one shifted right by the difference.
void lower_phi_scale(const Params& P, Dev& d, int F, cudaStream_t s)
{
    if (F >= d.phi_F) return;
    const Geo G0 = geo(d, 0, P.R);
    ++g_launches;
    k_shift_fixed<<<gridsz(G0.cells, 256), 256, 0, s>>>(reinterpret_cast<long long*>(d.lev[0].phi), d.phi_F - F,
                                                       G0.cells);
    if (d.phi_prev && d.have_prev) {
        ++g_launches;
        k_shift_fixed<<<gridsz(G0.cells, 256), 256, 0, s>>>(reinterpret_cast<long long*>(d.phi_prev), d.phi_F - F,
                                                           G0.cells);
    }
    d.phi_F = F;
}

int field_solve(const Params& P, Dev& d, int precision, double rtol, int nu1, int nu2, unsigned long long rho_absmax,
                int max_cycles, cudaStream_t s, int* cycles_out, double* rel_out, bool extrapolate)
{
    const int R = P.R;
    MGLevel& L0 = d.lev[0];
    const Geo G0 = geo(d, 0, R);
    const uint64_t per_real = G0.cells / R;
    const int items = (int)(per_real / NORM_TPB < 8 ? per_real / NORM_TPB : 8);
    const int nblk = (int)(G0.cells / ((uint64_t)NORM_TPB * items));
    const int bpr = nblk / R;
    double* h_norm = d.norm_host;       // 2 R doubles of host memory owned by the caller
    double bnorm[MAX_REAL_NORM];
    if (R > MAX_REAL_NORM) return -1;
    double worst = 0.0;
    int cyc = 0;
    int status = -6;
    const bool fixed = precision == 2;
    long long* Phi = reinterpret_cast<long long*>(L0.phi);
    long long* Bfix = reinterpret_cast<long long*>(L0.rhs);
    if (fixed) {
        // scale from a bound on |phi| (lowered only: the warm start is shifted)
        lower_phi_scale(P, d, phi_fixed_bits(phi_bound(P, rho_absmax)), s);
        double qscale, bc_top;
        rhs_consts(P, qscale, bc_top);
        ++g_launches;
        k_rhs_fixed<<<gridsz(G0.cells, 256), 256, 0, s>>>(d.rho, Bfix, G0, qscale, bc_top,
                                                         L0.h * L0.h * std::ldexp(1.0, d.phi_F));
    }
    // initial guess 2 phi_k - phi_{k-1} (the previous potential is kept)
    if (extrapolate && d.phi_prev) {
        ++g_launches;
        if (fixed)
            k_extrapolate<long long><<<gridsz(G0.cells, 256), 256, 0, s>>>(
                Phi, reinterpret_cast<long long*>(d.phi_prev), G0.cells, d.have_prev);
        else
            k_extrapolate<double><<<gridsz(G0.cells, 256), 256, 0, s>>>(
                L0.phi, reinterpret_cast<double*>(d.phi_prev), G0.cells, d.have_prev);
        d.have_prev = true;
    }
    const float rsc = (float)std::ldexp(1.0, -d.phi_F);
    const float esc = (float)std::ldexp(1.0, d.phi_F);
    // FP64 V-cycles: the residual norm only serves the convergence test, so
    // it is evaluated at cycle 0 and then at the cycle the observed
    // convergence factor predicts (refinement forms need the residual every
    // outer iteration as the right-hand side of the correction).
    int next_check = 0;
    double rho_est = 0.1, prev_rel = -1.0;
    int prev_cyc = 0;
    for (cyc = 0; cyc <= max_cycles; ++cyc) {
        if (precision == 0 && cyc < next_check && cyc < max_cycles) {
            run_cycles(d, 0, R, nu1, nu2, s);
            continue;
        }
        ++g_launches;
        if (fixed)
            k_resid_fixed<<<nblk, NORM_TPB, 0, s>>>(Phi, Bfix, L0.rhs32, G0, rsc, d.norm_part, cyc == 0, items);
        else
            k_resid_norm<<<nblk, NORM_TPB, 0, s>>>(L0.phi, L0.rhs, precision == 1 ? L0.rhs32 : nullptr, G0,
                                                   d.norm_part, cyc == 0, items);
        ++g_launches;
        k_norm_final<<<R, 256, 0, s>>>(d.norm_part, bpr, R, d.norm_out);
        cudaMemcpyAsync(h_norm, d.norm_out, 2 * R * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -3;
        worst = 0.0;
        bool done = true;
        for (int r = 0; r < R; ++r) {
            if (cyc == 0) bnorm[r] = h_norm[2 * r + 1];
            const double rn = std::sqrt(h_norm[2 * r]), bn = std::sqrt(bnorm[r]);
            const double rel = bn > 0.0 ? rn / bn : rn;
            if (rel > worst || !(rel == rel)) worst = rel;
            if (!(rn <= rtol * bn)) done = false;
        }
        if (done) { status = 0; break; }
        if (cyc == max_cycles || !std::isfinite(worst)) break;
        if (precision == 0) {
            if (prev_rel > 0.0 && worst > 0.0 && cyc > prev_cyc) {
                rho_est = std::pow(worst / prev_rel, 1.0 / (cyc - prev_cyc));
                rho_est = std::min(0.5, std::max(0.02, rho_est));
            }
            prev_rel = worst;
            prev_cyc = cyc;
            const double need = worst > 0.0 ? std::log(rtol / worst) / std::log(rho_est) : 1.0;
            next_check = cyc + std::max(1, (int)std::floor(need));
        }
        if (precision >= 1) {
            // inner solve of A e = r in FP32: two V-cycles per outer residual
            run_cycles(d, 1, R, nu1, nu2, s);
            ++g_launches;
            if (fixed)
                k_add_fixed<<<gridsz(G0.cells, 256), 256, 0, s>>>(Phi, L0.phi32, esc, G0.cells);
            else
                k_add_correction<<<gridsz(G0.cells, 256), 256, 0, s>>>(L0.phi, L0.phi32, G0.cells);
        } else {
            run_cycles(d, 0, R, nu1, nu2, s);
        }
    }
    if (cycles_out) *cycles_out = cyc;
    if (rel_out) *rel_out = worst;
    return status;
}

// The solve of field_solve with a fixed number of cycles and no host
// synchronisation, for steps replayed from a captured graph: the same
// launches (the fixed-point scale is kept: a step that needs a lower one is
// solved again by field_solve afterwards), then the residual and right-hand
// side norms of every realization in d.norm_out, which the host checks after
// the step.  cycles: V-cycles (FP64), or outer corrections of two FP32
// V-cycles each (refinement forms).
void field_solve_fixed(const Params& P, Dev& d, int precision, int nu1, int nu2, int cycles, cudaStream_t s)
{
    const int R = P.R;
    MGLevel& L0 = d.lev[0];
    const Geo G0 = geo(d, 0, R);
    const uint64_t per_real = G0.cells / R;
    const int items = (int)(per_real / NORM_TPB < 8 ? per_real / NORM_TPB : 8);
    const int nblk = (int)(G0.cells / ((uint64_t)NORM_TPB * items));
    const int bpr = nblk / R;
    const bool fixed = precision == 2;
    long long* Phi = reinterpret_cast<long long*>(L0.phi);
    long long* Bfix = reinterpret_cast<long long*>(L0.rhs);
    if (fixed) {
        double qscale, bc_top;
        rhs_consts(P, qscale, bc_top);
        ++g_launches;
        k_rhs_fixed<<<gridsz(G0.cells, 256), 256, 0, s>>>(d.rho, Bfix, G0, qscale, bc_top,
                                                         L0.h * L0.h * std::ldexp(1.0, d.phi_F));
    }
    if (d.phi_prev) {
        ++g_launches;
        if (fixed)
            k_extrapolate<long long><<<gridsz(G0.cells, 256), 256, 0, s>>>(
                Phi, reinterpret_cast<long long*>(d.phi_prev), G0.cells, d.have_prev);
        else
            k_extrapolate<double><<<gridsz(G0.cells, 256), 256, 0, s>>>(
                L0.phi, reinterpret_cast<double*>(d.phi_prev), G0.cells, d.have_prev);
        d.have_prev = true;
    }
    const float rsc = (float)std::ldexp(1.0, -d.phi_F);
    const float esc = (float)std::ldexp(1.0, d.phi_F);
    auto resid = [&](bool first) {
        ++g_launches;
        if (fixed)
            k_resid_fixed<<<nblk, NORM_TPB, 0, s>>>(Phi, Bfix, L0.rhs32, G0, rsc, d.norm_part, first, items);
        else
            k_resid_norm<<<nblk, NORM_TPB, 0, s>>>(L0.phi, L0.rhs, precision == 1 ? L0.rhs32 : nullptr, G0,
                                                   d.norm_part, first, items);
    };
    for (int c = 0; c < cycles; ++c) {
        if (precision == 0) {
            run_cycles(d, 0, R, nu1, nu2, s);
            continue;
        }
        resid(false);
        run_cycles(d, 1, R, nu1, nu2, s);
        ++g_launches;
        if (fixed)
            k_add_fixed<<<gridsz(G0.cells, 256), 256, 0, s>>>(Phi, L0.phi32, esc, G0.cells);
        else
            k_add_correction<<<gridsz(G0.cells, 256), 256, 0, s>>>(L0.phi, L0.phi32, G0.cells);
    }
    resid(true);
    ++g_launches;
    k_norm_final<<<R, 256, 0, s>>>(d.norm_part, bpr, R, d.norm_out);
}

__global__ void k_pack_field(const double* __restrict__ E3, E64* __restrict__ E, float4* __restrict__ E32, uint64_t G)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < G; t += (uint64_t)gridDim.x * blockDim.x) {
        const double ex = E3[t], ey = E3[G + t], ez = E3[2 * G + t];
        const double m = sqrt((ex * ex + ey * ey) + ez * ez);
        if (E) {
            reinterpret_cast<double2*>(E + t)[0] = make_double2(ex, ey);
            reinterpret_cast<double2*>(E + t)[1] = make_double2(ez, m);
        }
        if (E32) E32[t] = make_float4((float)ex, (float)ey, (float)ez, (float)m);
    }
}

// Field readback: from the FP64 field, or from the FP32 one (mixed form).
__global__ void k_unpack_field(const E64* __restrict__ E, const float4* __restrict__ E32, double* __restrict__ E3,
                               uint64_t G)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < G; t += (uint64_t)gridDim.x * blockDim.x) {
        if (E) {
            const E64 e = E[t];
            E3[t] = e.x; E3[G + t] = e.y; E3[2 * G + t] = e.z;
        } else {
            const float4 e = E32[t];
            E3[t] = e.x; E3[G + t] = e.y; E3[2 * G + t] = e.z;
        }
    }
}

void launch_pack_field(const Params& P, Dev& d, const double* E3, cudaStream_t s)
{
    const uint64_t G = (uint64_t)P.R * P.n3;
    ++g_launches;
    k_pack_field<<<gridsz(G, 256), 256, 0, s>>>(E3, d.E, d.E32, G);
}

void launch_unpack_field(const Params& P, Dev& d, double* E3, cudaStream_t s)
{
    const uint64_t G = (uint64_t)P.R * P.n3;
    ++g_launches;
    k_unpack_field<<<gridsz(G, 256), 256, 0, s>>>(d.E, d.E32, E3, G);
}

void launch_efield(const Params& P, Dev& d, cudaStream_t s) { launch_efield_to(P, d, s, d.E, d.E32); }

// E = -grad(phi) into the given FP64 and/or FP32 field arrays.
void launch_efield_to(const Params& P, Dev& d, cudaStream_t s, E64* E, float4* E32)
{
    const Geo G0 = geo(d, 0, P.R);
    const double phi_top = P.E0 * (P.hi[2] - P.lo[2]);
    ++g_launches;
    if (d.phi_F > 0)
        k_efield_fixed<<<gridsz(G0.cells, 256), 256, 0, s>>>(
            reinterpret_cast<const long long*>(d.lev[0].phi), E, E32, G0,
            std::ldexp(1.0, -d.phi_F) / (2.0 * d.lev[0].h), std::llrint(std::ldexp(phi_top, d.phi_F)));
    else
        k_efield<<<gridsz(G0.cells, 256), 256, 0, s>>>(d.lev[0].phi, E, E32, G0, d.lev[0].h, phi_top);
}

// The potential as FP64 volts into out (R n^3).
void launch_phi_to_double(const Params& P, Dev& d, double* out, cudaStream_t s)
{
    const Geo G0 = geo(d, 0, P.R);
    ++g_launches;
    k_phi_to_double<<<gridsz(G0.cells, 256), 256, 0, s>>>(reinterpret_cast<const long long*>(d.lev[0].phi), out,
                                                          std::ldexp(1.0, -d.phi_F), G0.cells);
}


// ------------------------------------------------------------------ semi-implicit solve
VCArrays vc_arrays(const Dev& d, int l)
{
    const VCLevel& V = d.vc[l];
    return VCArrays{ V.fx, V.fy, V.fz, V.dg, V.idg };
}

// One V-cycle of the variable-coefficient system from level l (RB-GS, the
// colour order of the constant-coefficient cycle); levels of at most 16^3
// cells run in the fused coarse kernel, whose coarsest level is relaxed by
// 48 sweep pairs.
static void vcycle_vc(const Dev& d, int l, int R, int nu1, int nu2, cudaStream_t s)
{
    const Geo G = geo(d, l, R);
    double* phi = d.lev[l].phi;
    const double* rhs = d.lev[l].rhs;
    const int tpb = 256;
    if (G.n <= COARSE_N && d.nlev - l >= 2) {
        CoarseVC C{};
        C.nlev = d.nlev - l;
        for (int q = 0; q < C.nlev; ++q) {
            C.n[q] = d.lev[l + q].n;
            C.phi[q] = d.lev[l + q].phi;
            C.rhs[q] = d.lev[l + q].rhs;
            C.A[q] = vc_arrays(d, l + q);
        }
        ++g_launches;
        k_vcycle_coarse_vc<<<R, 512, 0, s>>>(C, nu1, nu2, 48);
        return;
    }
    const VCArrays A = vc_arrays(d, l);
    auto sweep = [&](int color) {
        ++g_launches;
        k_smooth_vc<<<gridsz(G.cells / 2, tpb), tpb, 0, s>>>(phi, rhs, A, G, color);
    };
    for (int it = 0; it < nu1; ++it) { sweep(0); sweep(1); }
    const Geo Gc = geo(d, l + 1, R);
    g_launches += 3;
    k_resid_restrict_vc<<<gridsz(Gc.cells, tpb), tpb, 0, s>>>(phi, rhs, A, d.lev[l + 1].rhs, Gc, G.n);
    k_zero<double><<<gridsz(Gc.cells, tpb), tpb, 0, s>>>(d.lev[l + 1].phi, Gc.cells);
    vcycle_vc(d, l + 1, R, nu1, nu2, s);
    k_prolong<double><<<gridsz(G.cells, tpb), tpb, 0, s>>>(phi, d.lev[l + 1].phi, G);
    for (int it = 0; it < nu2; ++it) { sweep(1); sweep(0); }
}

// One variable-coefficient V-cycle from the graph of kind 2 (captured once
// per smoother pair: the operator arrays keep their addresses).
static void run_cycle_vc(Dev& d, int R, int nu1, int nu2, cudaStream_t s)
{
    const int k = 2;
    if (d.direct_cycles) { vcycle_vc(d, 0, R, nu1, nu2, s); return; }
    if (d.vgraph[k] && (d.vgraph_nu[k][0] != nu1 || d.vgraph_nu[k][1] != nu2)) {
        cudaGraphExecDestroy(d.vgraph[k]);
        d.vgraph[k] = nullptr;
    }
    if (!d.vgraph[k]) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            vcycle_vc(d, 0, R, nu1, nu2, s);
            return;
        }
        const unsigned long long l0 = g_launches.load();
        vcycle_vc(d, 0, R, nu1, nu2, s);
        const unsigned long long nk = g_launches.load() - l0;
        g_launches -= nk;
        if (cudaStreamEndCapture(s, &g) != cudaSuccess || !g ||
            cudaGraphInstantiate(&d.vgraph[k], g, 0) != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            d.vgraph[k] = nullptr;
            vcycle_vc(d, 0, R, nu1, nu2, s);
            return;
        }
        cudaGraphDestroy(g);
        d.vgraph_nu[k][0] = nu1;
        d.vgraph_nu[k][1] = nu2;
        d.vgraph_kernels[k] = nk;
    }
    g_launches += d.vgraph_kernels[k];
    cudaGraphLaunch(d.vgraph[k], s);
}

// Coefficients of the semi-implicit field (Sec. 4.7 step 1) into c0 from the
// electron deposit in d.ne_fix (the particles at the start of the step).
void launch_semi_coef(const Params& P, Dev& d, double* c0, cudaStream_t s)
{
    const Geo G0 = geo(d, 0, P.R);
    const double dV = P.h[0] * P.h[1] * P.h[2];
    const double per_cell = std::ldexp(1.0, -3 * P.frac_bits) / dV;
    ++g_launches;
    k_coef_from_ne<<<gridsz(G0.cells, 256), 256, 0, s>>>(d.ne_fix, c0, G0.cells, per_cell, 1.602176634e-19 * P.mu,
                                                          P.dt / 8.8541878128e-12);
}

// Semi-implicit field (Sec. 4.7 step 3, FP64 form): the level-0
// coefficients in d.vc[0].c (launch_semi_coef), restricted to the coarser
// levels, each level's face coefficients and diagonal, the right-hand side
// from d.rho (the charge of the diffused particles), FP64 V-cycles until
// ||r|| <= rtol ||b|| per realization, then E = -grad(phi) into d.E.  acc 2 R
// doubles of device scratch, acc_host its pinned mirror.  Returns 0, -6 (no
// convergence) or -3 (CUDA error).
int field_solve_vc(const Params& P, Dev& d, double* acc, double* acc_host, double rtol, int nu1, int nu2,
                   int max_cycles, cudaStream_t s, int* cycles_out, double* rel_out)
{
    const int R = P.R;
    const Geo G0 = geo(d, 0, R);
    const int tpb = 256;
    for (int l = 0; l + 1 < d.nlev; ++l) {
        const Geo Gc = geo(d, l + 1, R);
        ++g_launches;
        k_coef_restrict<<<gridsz(Gc.cells, tpb), tpb, 0, s>>>(d.vc[l].c, d.vc[l + 1].c, Gc, d.lev[l].n);
    }
    for (int l = 0; l < d.nlev; ++l) {
        const Geo G = geo(d, l, R);
        const VCLevel& V = d.vc[l];
        ++g_launches;
        k_vc_faces<<<gridsz(G.cells, tpb), tpb, 0, s>>>(V.c, V.fx, V.fy, V.fz, V.dg, V.idg, G);
    }
    double qscale, bc_top;
    rhs_consts(P, qscale, bc_top);
    ++g_launches;
    k_rhs_vc<<<gridsz(G0.cells, tpb), tpb, 0, s>>>(d.rho, d.vc[0].c, d.lev[0].rhs, G0, qscale, bc_top,
                                                    P.h[2] * P.h[2]);
    const VCArrays A0 = vc_arrays(d, 0);
    int cyc = 0, status = -6;
    double worst = 0.0;
    for (cyc = 0; cyc <= max_cycles; ++cyc) {
        g_launches += 2;
        const uint64_t per = G0.cells / (uint64_t)R;
        const dim3 ng((unsigned)gridsz(per, tpb), (unsigned)R);
        k_resid_norm_vc<<<ng, tpb, 0, s>>>(d.lev[0].phi, d.lev[0].rhs, A0, G0, d.norm_part);
        k_norm_final<<<R, 256, 0, s>>>(d.norm_part, (int)ng.x, R, acc);
        cudaMemcpyAsync(acc_host, acc, 2 * R * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -3;
        worst = 0.0;
        bool done = true;
        for (int r = 0; r < R; ++r) {
            const double rn = std::sqrt(acc_host[2 * r]), bn = std::sqrt(acc_host[2 * r + 1]);
            const double rel = bn > 0.0 ? rn / bn : rn;
            if (rel > worst || !(rel == rel)) worst = rel;
            if (!(rn <= rtol * bn)) done = false;
        }
        if (done) { status = 0; break; }
        if (cyc == max_cycles || !std::isfinite(worst)) break;
        run_cycle_vc(d, R, nu1, nu2, s);
    }
    if (cycles_out) *cycles_out = cyc;
    if (rel_out) *rel_out = worst;
    launch_efield_to(P, d, s, d.E, d.E32);
    return status;
}

}  // namespace ik

// ===========================================================================
// Field solve without device allocation (itokmc_field_solve_noalloc).
//
// Some callers cannot call cudaMalloc: a host program whose device memory
// belongs to another runtime's pool with a fixed budget, code that must not
// incur the implicit device synchronisation of cudaMalloc/cudaFree inside a
// latency-critical loop, or a plugin whose host forbids new device
// allocations.  For them the multigrid scratch (coarse levels, FP32 copies,
// right-hand side, norm partials and the packed field) lives in this
// file-scope device array, which every GPU that loads the library keeps
// until the process exits.  The caller passes the charge, the potential and
// the field buffers.
// ===========================================================================
namespace ik {
namespace {

constexpr size_t NOALLOC_BYTES = 16u << 20;     // 16 MiB: grids up to 64^3
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mtx;
constexpr int NOALLOC_MAX_DEV = 64;
void* g_noalloc_ptr[NOALLOC_MAX_DEV] = {};

// h^2 b with b = -rho/eps0 and the electrode potentials folded in (as the
// step does).
__global__ void k_rhs_from_rho(const int64_t* __restrict__ rho, double* __restrict__ rhs, int n, int log2n,
                               double qscale, double phi_top, double h)
{
    const uint64_t cells = (uint64_t)n * n * n;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < cells; g += (uint64_t)gridDim.x * blockDim.x) {
        const int k = (int)(g >> (2 * log2n));
        double b = -((double)rho[g] * qscale) / 8.8541878128e-12;
        if (k == n - 1) b = b - 2.0 * phi_top / (h * h);
        rhs[g] = b * (h * h);
    }
}

size_t carve(size_t& off, size_t bytes)
{
    const size_t at = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return at;
}

}  // namespace
}  // namespace ik

extern "C" int itokmc_field_solve_noalloc(const itokmc_config* cfg, const int64_t* rho, double* phi, double* E,
                                          int32_t* cycles_out, double* rel_out)
{
    using namespace ik;
    if (!cfg || !rho || !phi || !E) { set_global_error("field_solve_noalloc: NULL argument"); return ITOKMC_ERR_ARG; }
    const int n = cfg->n[0];
    if (cfg->n_realizations != 1 || cfg->n[1] != n || cfg->n[2] != n || n < 8 || (n & (n - 1))) {
        set_global_error("field_solve_noalloc: one realization on an n^3 grid, n a power of two >= 8");
        return ITOKMC_ERR_ARG;
    }
    if (n > ITOKMC_NOALLOC_MAX_N) {
        set_global_error("field_solve_noalloc: grid larger than ITOKMC_NOALLOC_MAX_N (64) cells per axis");
        return ITOKMC_ERR_ARG;
    }
    if ((cfg->precision != ITOKMC_FP64 && cfg->precision != ITOKMC_MIXED) ||
        (cfg->field_precision != -1 && cfg->field_precision != ITOKMC_FP64 && cfg->field_precision != ITOKMC_MIXED)) {
        set_global_error("field_solve_noalloc: precision must be ITOKMC_FP64 or ITOKMC_MIXED (field_precision also -1)");
        return ITOKMC_ERR_ARG;
    }
    const int fp = cfg->field_precision < 0 ? cfg->precision : cfg->field_precision;
    // FP64 V-cycles, or FP32 V-cycles inside FP64 residual refinement
    const int prec = fp == ITOKMC_MIXED ? 1 : 0;
    cudaStream_t s = (cudaStream_t)cfg->stream;
    // set-up once per device, with that device current: the device address
    // of the scratch array (its name is only a stand-in in host code)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEV) {
        cudaGetLastError();
        set_global_error("field_solve_noalloc: no current CUDA device");
        return ITOKMC_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mtx);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                set_global_error("field_solve_noalloc: cudaGetSymbolAddress of the scratch array failed");
                return ITOKMC_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    }
    // lay the hierarchy out in the scratch array
    Params P{};
    P.n = n; P.n3 = n * n * n; P.R = 1;
    while ((1 << P.log2n) < n) ++P.log2n;
    for (int a = 0; a < 3; ++a) {
        P.lo[a] = cfg->lo[a]; P.hi[a] = cfg->hi[a]; P.h[a] = (cfg->hi[a] - cfg->lo[a]) / n;
        P.rh[a] = 1.0 / P.h[a];
    }
    P.E0 = cfg->E0;
    P.frac_bits = cfg->frac_bits;
    Dev d;
    d.direct_cycles = true;            // no graph objects: nothing is instantiated per call
    size_t off = 0;
    int l = 0;
    for (int m = n; m >= 4 && l < MAX_LEVELS; m >>= 1, ++l) {
        MGLevel& L = d.lev[l];
        const size_t cells = (size_t)m * m * m;
        L.n = m;
        L.h = P.h[0] * (double)(n / m);
        L.phi = l == 0 ? phi : reinterpret_cast<double*>(base + carve(off, cells * sizeof(double)));
        L.rhs = reinterpret_cast<double*>(base + carve(off, cells * sizeof(double)));
        L.res = nullptr;
        L.phi32 = reinterpret_cast<float*>(base + carve(off, cells * sizeof(float)));
        L.rhs32 = reinterpret_cast<float*>(base + carve(off, cells * sizeof(float)));
    }
    d.nlev = l;
    d.norm_part = reinterpret_cast<double*>(base + carve(off, 2 * ((size_t)P.n3 / 256 + 16) * sizeof(double)));
    d.norm_out = reinterpret_cast<double*>(base + carve(off, 2 * sizeof(double)));
    d.E = reinterpret_cast<E64*>(base + carve(off, (size_t)P.n3 * sizeof(E64)));
    d.E32 = nullptr;
    if (off > NOALLOC_BYTES) {
        set_global_error("field_solve_noalloc: scratch layout exceeds the static array");
        return ITOKMC_ERR_ARG;
    }
    double norm_host[2];               // stack memory: no allocation
    d.norm_host = norm_host;
    const double dV = P.h[0] * P.h[1] * P.h[2];
    const double qscale = 1.602176634e-19 * ldexp(1.0, -3 * P.frac_bits) / dV;
    const double phi_top = P.E0 * (P.hi[2] - P.lo[2]);
    ++g_launches;
    k_rhs_from_rho<<<gridsz((uint64_t)P.n3, 256), 256, 0, s>>>(rho, d.lev[0].rhs, n, P.log2n, qscale, phi_top, P.h[0]);
    int cycles = 0;
    double rel = 0.0;
    const int st = field_solve(P, d, prec, cfg->mg_rtol, cfg->mg_nu1, cfg->mg_nu2, 0ull, cfg->mg_max_cycles, s, &cycles,
                               &rel);
    if (cycles_out) *cycles_out = cycles;
    if (rel_out) *rel_out = rel;
    if (st == -3) {
        set_global_error("field_solve_noalloc: CUDA error in the multigrid");
        return ITOKMC_ERR_CUDA;
    }
    launch_efield(P, d, s);
    const uint64_t G = (uint64_t)P.n3;
    ++g_launches;
    k_unpack_field<<<gridsz(G, 256), 256, 0, s>>>(d.E, nullptr, E, G);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_global_error("field_solve_noalloc: CUDA error");
        return ITOKMC_ERR_CUDA;
    }
    if (st != 0) {
        set_global_error("field_solve_noalloc: multigrid did not reach mg_rtol within mg_max_cycles");
        return ITOKMC_ERR_NOCONV;
    }
    return ITOKMC_OK;
}
