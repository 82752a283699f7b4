// batch_kernels.cuh -- ensembles of uneven domains: one persistent kernel per
// stage (hdiff, then vadv), both captured once into a CUDA graph by the plan.
//
// Work items: hdiff (member, tile, K-chunk) and vadv (member, 32 x BJ column
// block).  A fixed grid of resident CTAs pulls item numbers from an atomic
// counter (reset by the graph before each stage), so uneven members balance
// dynamically; the plan numbers the items longest-first.  Each item runs the
// same device code as a single-domain launch (hdiff_rs_item, vadv_columns),
// so a batched member's results equal its single-domain results with the
// same tile configuration, bit for bit.
#pragma once

#include "hdiff_rs.cuh"
#include "vadv_kernels.cuh"

namespace gtb {

template <typename T>
struct BatchHdiffMember {
    View<T> in, coeff, out;
    HdiffGeom g;
    int vec_ok;
    int item0;  // first item of this member
};

template <typename T>
struct BatchVadvMember {
    View<const T> us, wc, up, ut, uts;
    View<T> out;
    VadvGeom g;
    int blocks_x;  // column blocks along i
    int item0;
};

// Next item for the whole CTA (block-uniform), or -1 when the queue is empty.
__device__ __forceinline__ int next_item(int *counter, int n_items, int *slot) {
    if (threadIdx.x == 0 && threadIdx.y == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    const int item = *slot;
    __syncthreads();  // every thread has read it before it is overwritten
    return item < n_items ? item : -1;
}

// Last member whose first item is <= item (members are numbered by item0).
template <typename M>
__device__ __forceinline__ int member_of(const M *mem, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mem[mid].item0 <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// maps: per member its in tensor map, followed (CTMA) by its coeff tensor map.
template <typename T, int CPL, int W, int R, int STAGES, bool FIXED, bool CTMA>
__global__ void __launch_bounds__(32 * W)
    hdiff_batch_kernel(const CUtensorMap *__restrict__ maps, const BatchHdiffMember<T> *__restrict__ mem, int n_mem,
                       int n_items, int *counter) {
    constexpr int MPM = CTMA ? 2 : 1;
    __shared__ int slot;
    uint64_t *bars;
    unsigned char *base = hdiff_rs_smem<T, CPL, W, R, STAGES, CTMA>(&bars);
    for (;;) {
        const int item = next_item(counter, n_items, &slot);
        if (item < 0) break;
        const int m = member_of(mem, n_mem, item);
        const BatchHdiffMember<T> M = mem[m];
        const int local = item - M.item0;
        hdiff_rs_item<T, CPL, W, R, STAGES, true, FIXED, CTMA>(&maps[MPM * m], &maps[MPM * m + MPM - 1], M.in,
                                                                M.coeff, M.out, M.g, M.vec_ok, local % M.g.n_tiles,
                                                                local / M.g.n_tiles, base, bars);
    }
}

// scratch: per CTA a slice of (DPG ? 1 : 2) * k_max * 32*BJ values of N.
// Registers capped for 28 resident warps per SM: the member descriptor a persistent CTA
// loads from global memory (six field views and the geometry) stays in registers
// through the column solve, which left the kernel at 122 registers and 16 warps per
// SM; the column solve is latency-bound, and the ensemble's replay went 2.26 -> 2.09 ms
// with the cap despite the spills (capped for 24 or 32 warps: 2.15, 2.21 ms).  Column
// pairs (two double-float columns a thread) capped for 12 warps: 2.03 ms, against 2.25
// at 28 warps (1.2 KB of spills), 2.05 at 16 and 2.43 at 8.
// Each item's column tests its address runs against the member's storages before the
// first access (vadv_columns' CHK, as in the checked build), in every build: the test is
// a few instructions per item, and with it the compiler spills less of the solve's state
// (96 -> 72 bytes reloaded): the ensemble's vadv stage 1.68 -> 1.56 ms, the same bits.
template <typename T, typename N, int BJ>
__global__ void __launch_bounds__(32 * BJ, (is_pair<T>() ? 12 : 28) / BJ)
    vadv_batch_kernel(const BatchVadvMember<T> *__restrict__ mem, int n_mem, int n_items, int *counter,
                      N *__restrict__ scratch, size_t slice, int k_max) {
    constexpr int NT = 32 * BJ;
    constexpr bool DPG = vadv_dp_global<T, N>();
    __shared__ int slot;
    const int t = threadIdx.y * 32 + threadIdx.x;
    N *cpb = scratch + (size_t)blockIdx.x * slice;
    N *dpb = cpb + (size_t)k_max * NT;
    for (;;) {
        const int item = next_item(counter, n_items, &slot);
        if (item < 0) break;
        const int m = member_of(mem, n_mem, item);
        const BatchVadvMember<T> M = mem[m];
        const int local = item - M.item0;
        vadv_columns<T, N, BJ, DPG, vadv_yform<T, N>(), true, true>(M.us, M.wc, M.up, M.ut, M.uts, M.out, M.g,
                                                        local % M.blocks_x, local / M.blocks_x, cpb, dpb, NT, t,
                                                        false, threadIdx.x, threadIdx.y);
    }
}

}  // namespace gtb
