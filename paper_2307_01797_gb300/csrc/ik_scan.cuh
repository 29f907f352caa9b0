// ik_scan.cuh -- multi-channel exclusive scan over a cell range (3 phases:
// per-block totals, scan of the block totals, per-block apply).  An Op
// supplies load(g, v[C]), store(g, excl[C], v[C]) and total(tot[C]).
// Deterministic (integer sums), no inter-block waits.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace ik {

extern std::atomic<unsigned long long> g_launches;

constexpr int SCAN_TPB = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_TPB * SCAN_ITEMS;

template <int C>
__device__ __forceinline__ void block_excl_scan(long long v[C], long long excl[C], long long tot[C])
{
    __shared__ long long wsum[32][C];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long inc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        long long x = v[c];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        inc[c] = x;
    }
    if (lane == 31) {
#pragma unroll
        for (int c = 0; c < C; ++c) wsum[wid][c] = inc[c];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            long long x = lane < nw ? wsum[lane][c] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += y;
            }
            if (lane < nw) wsum[lane][c] = x;   // inclusive over warps
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const long long wpre = wid ? wsum[wid - 1][c] : 0;
        excl[c] = wpre + inc[c] - v[c];
        tot[c] = wsum[nw - 1][c];
    }
    __syncthreads();
}

template <int C, class Op>
__global__ void __launch_bounds__(SCAN_TPB) k_scan_reduce(Op op, uint64_t G, long long* blk)
{
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    long long s[C];
#pragma unroll
    for (int c = 0; c < C; ++c) s[c] = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const uint64_t g = base + k;
        if (g < G) {
            long long v[C];
            op.load(g, v);
#pragma unroll
            for (int c = 0; c < C; ++c) s[c] += v[c];
        }
    }
    long long ex[C], tot[C];
    block_excl_scan<C>(s, ex, tot);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < C; ++c) blk[(uint64_t)blockIdx.x * C + c] = tot[c];
    }
}

// Single block: exclusive scan of nblk block totals in place; the grand
// totals go to blk[nblk*C + c].
template <int C>
__global__ void __launch_bounds__(1024) k_scan_blocks(long long* blk, int nblk)
{
    __shared__ long long carry[C];
    if (threadIdx.x < C) carry[threadIdx.x] = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += 1024) {
        const int b = base + threadIdx.x;
        long long v[C];
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = b < nblk ? blk[(uint64_t)b * C + c] : 0;
        long long ex[C], tot[C];
        block_excl_scan<C>(v, ex, tot);
        if (b < nblk) {
#pragma unroll
            for (int c = 0; c < C; ++c) blk[(uint64_t)b * C + c] = carry[c] + ex[c];
        }
        __syncthreads();
        if (threadIdx.x < C) carry[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x < C) blk[(uint64_t)nblk * C + threadIdx.x] = carry[threadIdx.x];
}

template <int C, class Op>
__global__ void __launch_bounds__(SCAN_TPB) k_scan_apply(Op op, uint64_t G, const long long* blk,
                                                          int nblk)
{
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS][C];
    long long s[C];
#pragma unroll
    for (int c = 0; c < C; ++c) s[c] = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const uint64_t g = base + k;
        if (g < G) op.load(g, v[k]);
        else {
#pragma unroll
            for (int c = 0; c < C; ++c) v[k][c] = 0;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) s[c] += v[k][c];
    }
    long long ex[C], tot[C];
    block_excl_scan<C>(s, ex, tot);
    long long run[C];
#pragma unroll
    for (int c = 0; c < C; ++c) run[c] = blk[(uint64_t)blockIdx.x * C + c] + ex[c];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const uint64_t g = base + k;
        if (g < G) op.store(g, run, v[k]);
#pragma unroll
        for (int c = 0; c < C; ++c) run[c] += v[k][c];
    }
    if (blockIdx.x == nblk - 1 && threadIdx.x == 0) {
        long long t[C];
#pragma unroll
        for (int c = 0; c < C; ++c) t[c] = blk[(uint64_t)nblk * C + c];
        op.total(t);
    }
}

// Scratch: nblk * C + C long longs.
inline int scan_nblk(uint64_t G) { return (int)((G + SCAN_TILE - 1) / SCAN_TILE); }

template <int C, class Op>
void run_scan(const Op& op, uint64_t G, long long* scratch, cudaStream_t s)
{
    const int nblk = scan_nblk(G) > 0 ? scan_nblk(G) : 1;
    g_launches += 3;
    k_scan_reduce<C, Op><<<nblk, SCAN_TPB, 0, s>>>(op, G, scratch);
    k_scan_blocks<C><<<1, 1024, 0, s>>>(scratch, nblk);
    k_scan_apply<C, Op><<<nblk, SCAN_TPB, 0, s>>>(op, G, scratch, nblk);
}

}  // namespace ik
