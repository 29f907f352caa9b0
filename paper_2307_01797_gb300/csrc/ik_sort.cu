// ik_sort.cu -- stable LSD radix sort of (key, value) pairs and the particle
// upload that uses it: particles given in any order are placed in the
// canonical order (realization, cell, input order) with their cell offsets.
#include <cstdint>

#include "ik_common.cuh"
#include "ik_scan.cuh"
#include "ik_state.h"

namespace ik {

namespace {

constexpr int RS_TPB = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_TPB * RS_ROUNDS;
constexpr int RS_BINS = 256;

__global__ void __launch_bounds__(RS_TPB) k_rs_hist(const uint32_t* __restrict__ keys, uint32_t n, int shift,
                                                    uint32_t nblk, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[RS_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    for (int q = 0; q < RS_ROUNDS; ++q) {
        const uint64_t i = base + (uint64_t)q * RS_TPB + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

struct HistScanOp {
    const uint32_t* hist;
    uint32_t* off;
    __device__ void load(uint64_t g, long long v[1]) const { v[0] = hist[g]; }
    __device__ void store(uint64_t g, const long long ex[1], const long long*) const { off[g] = (uint32_t)ex[0]; }
    __device__ void total(const long long*) const {}
};

__global__ void __launch_bounds__(RS_TPB) k_rs_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                       uint32_t n, int shift, uint32_t nblk,
                                                       const uint32_t* __restrict__ off, uint32_t* __restrict__ kout,
                                                       uint32_t* __restrict__ vout)
{
    __shared__ uint32_t running[RS_BINS];
    __shared__ uint32_t wc[RS_TPB / 32][RS_BINS];
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    running[threadIdx.x] = 0;
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    for (int q = 0; q < RS_ROUNDS; ++q) {
        for (int w = 0; w < RS_TPB / 32; ++w) wc[w][threadIdx.x] = 0;
        __syncthreads();
        const uint64_t i = base + (uint64_t)q * RS_TPB + threadIdx.x;
        const bool ok = i < n;
        const uint32_t k = ok ? keys[i] : 0u;
        const uint32_t dg = ok ? ((k >> shift) & 0xffu) : 0x100u;   // 0x100: no digit
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rin = __popc(peers & ((1u << lane) - 1u));
        if (ok && rin == 0) wc[wid][dg] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pre = running[dg];
            for (unsigned w = 0; w < wid; ++w) pre += wc[w][dg];
            const uint32_t pos = off[(uint64_t)dg * nblk + blockIdx.x] + pre + rin;
            kout[pos] = k;
            vout[pos] = vals[i];
        }
        __syncthreads();
        uint32_t add = 0;
        for (int w = 0; w < RS_TPB / 32; ++w) add += wc[w][threadIdx.x];
        running[threadIdx.x] += add;
        __syncthreads();
    }
}

// Pack SoA input into records, compute global cells, validate.
__global__ void k_pack(Params P, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const uint32_t* __restrict__ w,
                       const int32_t* __restrict__ real, const int32_t* __restrict__ species, uint32_t n,
                       P64* __restrict__ out, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                       Counters* __restrict__ ctr)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double X[3] = { x[i], y[i], z[i] };
        const int r0 = real ? real[i] : 0, sp = species ? species[i] : 0;
        bool ok = r0 >= 0 && r0 < P.R && sp >= 0 && sp < P.S && w[i] > 0;
        const int r = sp * P.R + r0;             // particle block
        for (int a = 0; a < 3; ++a) ok = ok && X[a] >= P.lo[a] && X[a] < P.hi[a];
        uint32_t g = 0;
        if (ok) {
            const int ix = cell_axis(X[0], P.lo[0], P.h[0], P.rh[0], P.n);
            const int iy = cell_axis(X[1], P.lo[1], P.h[1], P.rh[1], P.n);
            const int iz = cell_axis(X[2], P.lo[2], P.h[2], P.rh[2], P.n);
            g = (uint32_t)((size_t)r * P.n3 + ((size_t)iz * P.n + iy) * P.n + ix);
        } else {
            atomicOr(&ctr->err, DERR_INTERNAL);
        }
        P64 p;
        p.x = X[0]; p.y = X[1]; p.z = X[2]; p.cell = g; p.w = w[i];
        out[i] = p;
        keys[i] = g;
        vals[i] = i;
    }
}

__global__ void k_gather(const P64* __restrict__ in, const uint32_t* __restrict__ perm, uint32_t n, P64* __restrict__ out)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) out[j] = in[perm[j]];
}

// Mixed form: (cell, FP32 offset in cell units) from the sorted FP64 records.
__global__ void k_gather32(Params P, const P64* __restrict__ in, const uint32_t* __restrict__ perm, uint32_t n,
                           P32* __restrict__ out, uint32_t* __restrict__ cout)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const P64 p = in[perm[j]];
        const uint32_t c = p.cell & (uint32_t)(P.n3 - 1);
        const int id[3] = { (int)(c & (uint32_t)(P.n - 1)), (int)((c >> P.log2n) & (uint32_t)(P.n - 1)),
                            (int)(c >> (2 * P.log2n)) };
        const double X[3] = { p.x, p.y, p.z };
        float o[3];
        for (int a = 0; a < 3; ++a) {
            float f = (float)(grid_quot(X[a], P.lo[a], P.h[a], P.rh[a]) - (double)id[a]);
            if (!(f >= 0.0f)) f = 0.0f;
            if (f >= 1.0f) f = 0x1.fffffep-1f;
            o[a] = f;
        }
        P32 q;
        q.ox = o[0]; q.oy = o[1]; q.oz = o[2]; q.w = p.w;
        out[j] = q;
        cout[j] = p.cell;
    }
}

// Particles per cell (keys are cells), for the offsets.
__global__ void k_count_keys(const uint32_t* __restrict__ keys, uint32_t n, int32_t* __restrict__ cnt)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        atomicAdd(cnt + keys[j], 1);
}

struct CountScanOp {
    const int32_t* cnt;
    uint32_t* cs;
    uint64_t G;
    __device__ void load(uint64_t g, long long v[1]) const { v[0] = cnt[g]; }
    __device__ void store(uint64_t g, const long long ex[1], const long long*) const { cs[g] = (uint32_t)ex[0]; }
    __device__ void total(const long long t[1]) const { cs[G] = (uint32_t)t[0]; }
};

int gsz(uint64_t n, int tpb)
{
    uint64_t b = (n + tpb - 1) / tpb;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp, uint32_t n,
                      int key_bits, cudaStream_t s, long long* blk_scratch, size_t)
{
    if (n == 0) return;
    const uint32_t nblk = (n + RS_TILE - 1) / RS_TILE;
    // histogram lives after the scan scratch region
    uint32_t* hist = reinterpret_cast<uint32_t*>(blk_scratch + scan_scratch_elems((uint64_t)RS_BINS * nblk, 1));
    uint32_t* off = hist + (size_t)RS_BINS * nblk;
    for (int shift = 0; shift < key_bits; shift += 8) {
        ++g_launches;
        k_rs_hist<<<nblk, RS_TPB, 0, s>>>(keys, n, shift, nblk, hist);
        HistScanOp op{ hist, off };
        run_scan<1>(op, (uint64_t)RS_BINS * nblk, blk_scratch, s);
        ++g_launches;
        k_rs_scatter<<<nblk, RS_TPB, 0, s>>>(keys, vals, n, shift, nblk, off, keys_tmp, vals_tmp);
        uint32_t* t = keys; keys = keys_tmp; keys_tmp = t;
        t = vals; vals = vals_tmp; vals_tmp = t;
    }
    // an odd number of passes leaves the result in the tmp buffers
    if (((key_bits + 7) / 8) & 1) {
        cudaMemcpyAsync(keys_tmp, keys, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals_tmp, vals, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
}

size_t radix_scratch_elems(uint32_t cap)
{
    const uint64_t nblk = (cap + RS_TILE - 1) / RS_TILE + 1;
    return scan_scratch_elems((uint64_t)RS_BINS * nblk, 1) + (size_t)RS_BINS * nblk + 16;
}

// x, y, z, w, real are device pointers (already staged).  `tmp64` holds n
// FP64 records during the sort.
void launch_set_particles(const Params& P, Dev& d, const double* x, const double* y, const double* z,
                          const uint32_t* w, const int32_t* real, const int32_t* species, uint32_t n, uint64_t G,
                          cudaStream_t s)
{
    uint32_t* keys = d.sort_tmp;
    uint32_t* vals = keys + d.mover_cap;
    uint32_t* kt = vals + d.mover_cap;
    uint32_t* vt = kt + d.mover_cap;
    cudaMemsetAsync(d.ctr, 0, sizeof(Counters), s);
    if (n > 0) {
        ++g_launches;
        P64* tmp64 = d.mixed ? reinterpret_cast<P64*>(d.work) + n : d.recB;   // staging sits at the start
        k_pack<<<gsz(n, 256), 256, 0, s>>>(P, x, y, z, w, real, species, n, tmp64, keys, vals, d.ctr);
        int bits = 1;
        while (bits < 32 && (1ull << bits) < G) ++bits;
        radix_sort_pairs(keys, vals, kt, vt, n, bits, s, d.scan_blk, 0);
        ++g_launches;
        if (d.mixed) k_gather32<<<gsz(n, 256), 256, 0, s>>>(P, tmp64, vals, n, d.rA32, d.cellA32);
        else k_gather<<<gsz(n, 256), 256, 0, s>>>(tmp64, vals, n, d.recA);
    }
    cudaMemsetAsync(d.cnt_new, 0, G * sizeof(int32_t), s);
    if (n > 0) {
        ++g_launches;
        k_count_keys<<<gsz(n, 256), 256, 0, s>>>(keys, n, d.cnt_new);
    }
    run_scan<1>(CountScanOp{ d.cnt_new, d.cell_start, G }, G, d.scan_blk, s);
}

}  // namespace ik
