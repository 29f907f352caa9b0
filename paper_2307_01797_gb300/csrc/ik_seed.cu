// ik_seed.cu -- initial electrons from Gaussian seeds on the device
// (itokmc_seed_blobs, and itokmc_init when the configuration lists blobs).
//
// The paper starts its discharges from Gaussian seeds of electrons (or
// electron-ion pairs), Sec. 5.1.  Per cell c of realization r: the density
// at the cell centre n(x_c) = sum_b A_b exp(-|x_c - c_b|^2 / (2 s_b^2))
// (squared distance summed x, y, z; blob b counts for r when its
// realization is r or -1); N_c ~ Poisson(n(x_c) dV) from the stream
// (key seed0 + r, index c, step, INIT, sub 0) with the tau-leap's sampler;
// m = min(N_c, ppc) superparticles with the weight rule of Eq. w (N_c div m,
// the remainder on the first), slot j uniform in the cell from the stream
// (c, step, INIT, 1 + j): FP64 x = lo + (i + u) h from three FP64 uniforms;
// the mixed form takes the FP32 offsets from the high words of the same
// uniforms.  Pass 1 draws the counts, a cell scan places the cells, pass 2
// writes the particles in canonical order (cell, slot).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "ik_common.cuh"
#include "ik_handle.h"
#include "ik_scan.cuh"

namespace ik {
namespace {

struct SeedBlob {
    double c[3];
    double sigma, peak;
    int real;
    int pad;
};

__device__ __forceinline__ double seed_density(const Params& P, const SeedBlob* __restrict__ B, int nb, int r,
                                               const int ijk[3])
{
    double xc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) xc[a] = P.lo[a] + ((double)ijk[a] + 0.5) * P.h[a];
    double dens = 0.0;
    for (int b = 0; b < nb; ++b) {
        if (B[b].real >= 0 && B[b].real != r) continue;
        const double d0 = xc[0] - B[b].c[0], d1 = xc[1] - B[b].c[1], d2 = xc[2] - B[b].c[2];
        const double r2 = (d0 * d0 + d1 * d1) + d2 * d2;
        dens = dens + B[b].peak * dexp(-r2 / (2.0 * B[b].sigma * B[b].sigma));
    }
    return dens;
}

__global__ void k_seed_count(Params P, const SeedBlob* __restrict__ B, int nb, int64_t* __restrict__ cnt, uint64_t G,
                             Counters* __restrict__ ctr)
{
    const double dV = (P.h[0] * P.h[1]) * P.h[2];
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < G; g += (uint64_t)gridDim.x * blockDim.x) {
        const int r = (int)(g >> (3 * P.log2n));
        const uint32_t c = (uint32_t)(g & (uint64_t)(P.n3 - 1));
        const int ijk[3] = { (int)(c & (uint32_t)(P.n - 1)), (int)((c >> P.log2n) & (uint32_t)(P.n - 1)),
                             (int)(c >> (2 * P.log2n)) };
        const double mu = seed_density(P, B, nb, r, ijk) * dV;
        Stream s(seed_of(P, r), c, P.step, TAG_INIT, 0);
        const int64_t N = dpoisson(s, mu);
        if (N < 0) atomicOr(&ctr->err, DERR_KMC);
        const int64_t Nc = N > 0 ? N : 0;
        cnt[g] = Nc;
        if (Nc > 0) {
            const int64_t m = Nc < P.ppc ? Nc : P.ppc;
            if (Nc / m + Nc % m > 0xffffffffll) atomicOr(&ctr->err, DERR_OVERFLOW);
        }
    }
}

// Cell offsets of the seeded particles: min(N_c, ppc) per cell.
struct SeedScanOp {
    const int64_t* cnt;
    uint32_t* cell_start;
    uint64_t G;
    int ppc;
    __device__ void load(uint64_t g, long long v[1]) const
    {
        const long long N = cnt[g];
        v[0] = N < ppc ? N : ppc;
    }
    __device__ void store(uint64_t g, const long long ex[1], const long long*) const { cell_start[g] = (uint32_t)ex[0]; }
    __device__ void total(const long long t[1]) const { cell_start[G] = (uint32_t)t[0]; }
};

template <bool MX>
__global__ void k_seed_write(Params P, const int64_t* __restrict__ cnt, const uint32_t* __restrict__ cell_start,
                             uint32_t cap, P64* __restrict__ rec, P32* __restrict__ rec32, uint32_t* __restrict__ cell32,
                             int64_t* __restrict__ Npos, int neutral, uint64_t G)
{
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < G; g += (uint64_t)gridDim.x * blockDim.x) {
        const int64_t N = cnt[g];
        if (N <= 0) continue;
        if (neutral) Npos[g] += N;
        const int r = (int)(g >> (3 * P.log2n));
        const uint32_t c = (uint32_t)(g & (uint64_t)(P.n3 - 1));
        const int ijk[3] = { (int)(c & (uint32_t)(P.n - 1)), (int)((c >> P.log2n) & (uint32_t)(P.n - 1)),
                             (int)(c >> (2 * P.log2n)) };
        const int64_t m = N < P.ppc ? N : P.ppc;
        const int64_t wq = N / m, rem = N % m;
        const uint32_t base = cell_start[g];
        for (int64_t j = 0; j < m; ++j) {
            const uint32_t q = base + (uint32_t)j;
            if (q >= cap) break;
            Stream t(seed_of(P, r), c, P.step, TAG_INIT, (uint32_t)(1 + j));
            const uint32_t w = (uint32_t)(wq + (j == 0 ? rem : 0));
            if constexpr (MX) {
                P32 o;
                float X[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    X[a] = uniform_f32(t.u32());
                    (void)t.u32();
                }
                o.ox = X[0]; o.oy = X[1]; o.oz = X[2]; o.w = w;
                rec32[q] = o;
                cell32[q] = (uint32_t)g;
            } else {
                double X[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) X[a] = P.lo[a] + ((double)ijk[a] + t.uniform()) * P.h[a];
                P64 o;
                o.x = X[0]; o.y = X[1]; o.z = X[2]; o.cell = (uint32_t)g; o.w = w;
                rec[q] = o;
            }
        }
    }
}

int grid_of(uint64_t n) { const uint64_t b = (n + 255) / 256; return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b)); }

// Mobile ions: the ion blocks' cell offsets after the electrons' (G cells),
// and with pairs a positive ion at every seed electron's position and weight
// (records [N, 2N) copy [0, N), their cells shifted by the G cells of the
// electron blocks).
__global__ void k_seed_ions(const uint32_t* __restrict__ cs_e, uint32_t* __restrict__ cs, uint32_t N, uint64_t G,
                            int pairs, P64* __restrict__ rec, P32* __restrict__ rec32, uint32_t* __restrict__ cell32)
{
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, st = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = t0; g <= G; g += st) {
        cs[G + g] = pairs ? N + cs_e[g] : N;
        cs[2 * G + g] = pairs ? 2 * N : N;
    }
    if (!pairs) return;
    for (uint64_t i = t0; i < N; i += st) {
        if (rec) {
            P64 p = rec[i];
            p.cell = (uint32_t)(p.cell + G);
            rec[N + i] = p;
        } else {
            rec32[N + i] = rec32[i];
            cell32[N + i] = (uint32_t)(cell32[i] + G);
        }
    }
}

}  // namespace

// Seeds the particles of every realization (pass 1, scan, pass 2); the
// caller has validated the blobs.  Returns ITOKMC_OK or an error code.
int seed_blobs(itokmc_handle* h, const itokmc_seed_blob* blobs, int nb, int flags)
{
    HandleView v;
    int rc = handle_view(h, &v);
    if (rc) return rc;
    *v.stage = 0;
    Dev& d = *v.d;
    const Params& P = *v.P;
    const uint64_t G = v.G;
    std::vector<SeedBlob> hb((size_t)nb);
    for (int b = 0; b < nb; ++b) {
        for (int a = 0; a < 3; ++a) hb[b].c[a] = blobs[b].center[a];
        hb[b].sigma = blobs[b].sigma;
        hb[b].peak = blobs[b].peak;
        hb[b].real = blobs[b].realization;
        hb[b].pad = 0;
    }
    // the blob table in the photon list (scratch until the first step)
    if ((size_t)nb * sizeof(SeedBlob) > (size_t)d.photo_cap * sizeof(Photo))
        return handle_fail(h, ITOKMC_ERR_ARG, "seed_blobs: too many blobs");
    SeedBlob* dB = reinterpret_cast<SeedBlob*>(d.photos);
    int64_t* cnt = d.fired;                      // counts in the first G of the firing array
    cudaStream_t s = v.s;
    if (nb > 0 && cudaMemcpyAsync(dB, hb.data(), nb * sizeof(SeedBlob), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return handle_fail(h, ITOKMC_ERR_CUDA, "seed_blobs: copy");
    cudaMemsetAsync(d.ctr, 0, sizeof(Counters), s);
    g_launches += 1;
    k_seed_count<<<grid_of(G), 256, 0, s>>>(P, dB, nb, cnt, G, d.ctr);
    SeedScanOp op{ cnt, d.cell_start, G, P.ppc };
    run_scan<1>(op, G, d.scan_blk, s);
    uint32_t total = 0;
    unsigned err = 0;
    if (cudaMemcpyAsync(&total, d.cell_start + G, sizeof total, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&err, &d.ctr->err, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return handle_fail(h, ITOKMC_ERR_CUDA, "seed_blobs: count pass");
    if (err & DERR_OVERFLOW) return handle_fail(h, ITOKMC_ERR_OVERFLOW, "seed_blobs: a weight exceeds 2^32 - 1");
    if (err) return handle_fail(h, ITOKMC_ERR_KMC, "seed_blobs: Poisson sampler gave up");
    const bool mobile = P.S == 3, pairs = mobile && (flags & ITOKMC_SEED_NEUTRAL);
    if ((uint64_t)total * (pairs ? 2u : 1u) > v.cap)
        return handle_fail(h, ITOKMC_ERR_CAPACITY, "seed_blobs: more particles than particle_capacity");
    // the count model adds the pairs' ions to the positive-ion counts
    const int neutral_counts = (flags & ITOKMC_SEED_NEUTRAL) && !mobile;
    g_launches += 1;
    if (d.mixed)
        k_seed_write<true><<<grid_of(G), 256, 0, s>>>(P, cnt, d.cell_start, v.cap, nullptr, d.rA32, d.cellA32, d.Npos,
                                                      neutral_counts, G);
    else
        k_seed_write<false><<<grid_of(G), 256, 0, s>>>(P, cnt, d.cell_start, v.cap, d.recA, nullptr, nullptr, d.Npos,
                                                       neutral_counts, G);
    if (mobile) {
        g_launches += 1;
        // cs_e: the electron offsets [0, G]; the ion blocks' offsets go after
        // them in the same array (a copy of [0, G] is not needed: each thread
        // reads cs[g] before any thread writes index G + g' >= G, except g = G,
        // whose value N both writes keep)
        k_seed_ions<<<grid_of(G + 1), 256, 0, s>>>(d.cell_start, d.cell_start, total, G, pairs ? 1 : 0,
                                                    d.mixed ? nullptr : d.recA, d.rA32, d.cellA32);
    }
    // the firing counts were borrowed: no reaction has fired yet
    cudaMemsetAsync(d.fired, 0, 5 * G * sizeof(int64_t), s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return handle_fail(h, ITOKMC_ERR_CUDA, "seed_blobs: write pass");
    *v.N = total * (pairs ? 2u : 1u);
    return ITOKMC_OK;
}

}  // namespace ik

extern "C" int itokmc_seed_blobs(itokmc_handle* h, const itokmc_seed_blob* blobs, int32_t n_blobs, int32_t flags)
{
    if (!h) return ITOKMC_ERR_ARG;
    if (n_blobs < 0 || (n_blobs > 0 && !blobs)) return ik::handle_fail(h, ITOKMC_ERR_ARG, "seed_blobs: bad blob array");
    if (flags & ~ITOKMC_SEED_NEUTRAL) return ik::handle_fail(h, ITOKMC_ERR_ARG, "seed_blobs: unknown flag");
    for (int b = 0; b < n_blobs; ++b) {
        const itokmc_seed_blob& B = blobs[b];
        if (!(B.sigma > 0.0) || !(B.peak >= 0.0) || !(B.peak < 1e300) || B.realization < -1)
            return ik::handle_fail(h, ITOKMC_ERR_ARG, "seed_blobs: sigma > 0, 0 <= peak, realization >= -1");
        for (int a = 0; a < 3; ++a)
            if (!(B.center[a] == B.center[a]) || B.center[a] > 1e300 || B.center[a] < -1e300)
                return ik::handle_fail(h, ITOKMC_ERR_ARG, "seed_blobs: blob centre not finite");
    }
    return ik::seed_blobs(h, blobs, n_blobs, flags);
}
