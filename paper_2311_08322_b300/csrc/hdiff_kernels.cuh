// hdiff_kernels.cuh -- horizontal diffusion (GT4Py paper, Sec. 3.1), one
// PARALLEL computation (Sec. 2.2) per K level:
//   lap = 4 in - (((in[i+1] + in[i-1]) + in[j+1]) + in[j-1])   on the tile plus a 1-ring
//   fx  = lap[i+1] - lap[i]  (0 where fx * (in[i+1] - in[i]) > 0),  fy likewise
//   out = in - coeff ((fx[i] - fx[i-1]) + (fy[j] - fy[j-1]))
//
// Mapping: one CTA owns a TI x TJ tile of (i,j) for a run of KC consecutive
// K levels.  Per level the (TI+4) x (TJ+4) input box (tile + 2-point halo,
// widened on the left so its first column is 16-byte aligned) is brought
// into shared memory by one TMA tiled load, STAGES levels ahead, each stage
// completing on its own mbarrier.  lap, fx and fy are temporaries (Sec. 2.2):
// they live in shared memory for one level and never reach HBM.  coeff is
// read and out written with 16-byte vector accesses when the layout allows.
#pragma once

#include "gtb_device.cuh"

namespace gtb {

template <typename T>
struct View {  // p points at compute-domain point (0,0,0); i stride is 1
    T *p;
    int64_t sj, sk;
};

struct HdiffGeom {
    int I, J, K;
    int tiles_i, tiles_j, n_tiles;
    int kc;          // K levels per work item
    int X0, Y0, Z0;  // tensor-map coordinate of box column/row 0 for tile (0,0), level 0
    int xs;          // box column of domain i = -2 (alignment shift, < 16/sizeof(T))
};

template <typename T, int TI, int TJ>
struct HdiffTile {
    static constexpr int kAlign = 16 / (int)sizeof(T);                                  // elements per 16 B
    static constexpr int BX = ((TI + 4 + kAlign - 1 + kAlign - 1) / kAlign) * kAlign;  // box width
    static constexpr int BY = TJ + 4;
    static constexpr int LX = TI + 2, LY = TJ + 2;  // lap region
    static constexpr int box_elems = BX * BY;
    static constexpr int box_bytes = box_elems * (int)sizeof(T);
    static constexpr int stage_stride = ((box_bytes + 127) / 128) * 128;
};

template <typename T, int TI, int TJ, int STAGES>
constexpr int hdiff_smem_bytes() {
    using G = HdiffTile<T, TI, TJ>;
    return STAGES * G::stage_stride + (G::LX * G::LY + (TI + 1) * TJ + TI * (TJ + 1)) * (int)sizeof(T) +
           STAGES * 8 + 128;
}

// Limiter test of the definition, fx * g > 0 (strict), evaluated as written.
template <typename T>
__device__ __forceinline__ T limit(T f, T g) {
    return (f * g > T(0)) ? T(0) : f;
}

template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T *p, T (&v)[VEC]) {
    if constexpr (VEC == 2 && sizeof(T) == 8) {
        const double2 x = *reinterpret_cast<const double2 *>(p);
        v[0] = x.x, v[1] = x.y;
    } else if constexpr (VEC == 4 && sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) v[e] = p[e];
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T *p, const T (&v)[VEC]) {
    if constexpr (VEC == 2 && sizeof(T) == 8) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    } else if constexpr (VEC == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) p[e] = v[e];
    }
}

// USE_TMA: input box via TMA (else cooperative loads into one stage).  VEC:
// elements per coeff/out access (16 B when the layout is aligned, else 1).
template <typename T, int TI, int TJ, int NT, int STAGES, bool USE_TMA, int VEC>
__global__ void __launch_bounds__(NT)
    hdiff_kernel(const __grid_constant__ CUtensorMap tmap, const View<T> in, const View<T> coeff,
                 const View<T> out, const HdiffGeom g) {
    using G = HdiffTile<T, TI, TJ>;
    constexpr int BX = G::BX;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    T *lap = reinterpret_cast<T *>(base + STAGES * G::stage_stride);
    T *fx = lap + G::LX * G::LY;  // [TJ][TI+1], column li <-> i = li - 1
    T *fy = fx + (TI + 1) * TJ;   // [TJ+1][TI], row lj <-> j = lj - 1
    uint64_t *bars = reinterpret_cast<uint64_t *>(fy + TI * (TJ + 1));

    const int tid = threadIdx.x;
    const int item = blockIdx.x;
    const int tile = item % g.n_tiles;
    const int kchunk = item / g.n_tiles;
    const int ti0 = (tile % g.tiles_i) * TI;
    const int tj0 = (tile / g.tiles_i) * TJ;
    const int k0 = kchunk * g.kc;
    const int nk = min(g.kc, g.K - k0);
    if (nk <= 0) return;
    const int ni_valid = min(TI, g.I - ti0);
    const int nj_valid = min(TJ, g.J - tj0);
    const int xs = g.xs;

    if (USE_TMA) {
        if (tid == 0) {
            prefetch_tensormap(&tmap);
            for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            for (int p = 0; p < STAGES && p < nk; ++p) {
                mbar_arrive_expect_tx(&bars[p], G::box_bytes);
                tma_load_3d(base + p * G::stage_stride, &tmap, &bars[p], g.X0 + ti0, g.Y0 + tj0, g.Z0 + k0 + p);
            }
        }
    }

    // output ownership in phase 3: VEC consecutive i per thread
    constexpr int GROUPS_I = TI / VEC;
    constexpr int ROWS_PER_PASS = NT / GROUPS_I;
    constexpr int PASSES = (TJ + ROWS_PER_PASS - 1) / ROWS_PER_PASS;
    static_assert(NT % GROUPS_I == 0, "thread count must cover whole tile rows");

    bool failed = false;
    for (int p = 0; p < nk; ++p) {
        const int k = k0 + p;
        const int s = USE_TMA ? (p % STAGES) : 0;
        const T *S = reinterpret_cast<const T *>(base + s * G::stage_stride);

        // coeff for this level, issued early to overlap with the stencil work
        T cf[PASSES][VEC];
#pragma unroll
        for (int q = 0; q < PASSES; ++q) {
            const int j = (tid / GROUPS_I) + q * ROWS_PER_PASS;
            const int i = (tid % GROUPS_I) * VEC;
            const T *cp = coeff.p + (int64_t)(ti0 + i) + (int64_t)(tj0 + j) * coeff.sj + (int64_t)k * coeff.sk;
            if (j < nj_valid && i + VEC <= ni_valid) {
                load_vec<T, VEC>(cp, cf[q]);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) cf[q][e] = (j < nj_valid && i + e < ni_valid) ? cp[e] : T(0);
            }
        }

        if (USE_TMA) {
            if (!mbar_wait(&bars[s], (p / STAGES) & 1)) failed = true;
        } else {
            // cooperative load of the box: rows j = tj0-2.., columns i = ti0-2..
            T *D = reinterpret_cast<T *>(base);
            for (int idx = tid; idx < G::box_elems; idx += NT) {
                const int bx = idx % BX, by = idx / BX;
                const int i = ti0 - 2 - xs + bx, j = tj0 - 2 + by;  // domain-relative
                T v = T(0);
                if (i >= -2 && i < g.I + 2 && j >= -2 && j < g.J + 2)
                    v = in.p[(int64_t)i + (int64_t)j * in.sj + (int64_t)k * in.sk];
                D[idx] = v;
            }
        }
        if (__syncthreads_or(failed)) break;

        // phase 1: Laplacian on the tile and its 1-ring
        for (int idx = tid; idx < G::LX * G::LY; idx += NT) {
            const int li = idx % G::LX, lj = idx / G::LX;  // lap(i = li-1, j = lj-1)
            const T *c = S + (lj + 1) * BX + (li + 1 + xs);
            const T sum = ((c[1] + c[-1]) + c[BX]) + c[-BX];
            lap[idx] = T(4) * c[0] - sum;
        }
        __syncthreads();
        // every thread is past phase 3 of level p-1: its stage may be refilled
        if (USE_TMA && tid == 0 && p >= 1 && p - 1 + STAGES < nk) {
            const int sp = (p - 1) % STAGES;
            mbar_arrive_expect_tx(&bars[sp], G::box_bytes);
            tma_load_3d(base + sp * G::stage_stride, &tmap, &bars[sp], g.X0 + ti0, g.Y0 + tj0,
                        g.Z0 + k - 1 + STAGES);
        }

        // phase 2: limited fluxes
        for (int idx = tid; idx < (TI + 1) * TJ; idx += NT) {
            const int li = idx % (TI + 1), j = idx / (TI + 1);  // fx(i = li-1, j)
            const T f = lap[(j + 1) * G::LX + li + 1] - lap[(j + 1) * G::LX + li];
            const T *c = S + (j + 2) * BX + (li + 1 + xs);  // in(i, j)
            fx[idx] = limit(f, c[1] - c[0]);
        }
        for (int idx = tid; idx < TI * (TJ + 1); idx += NT) {
            const int i = idx % TI, lj = idx / TI;  // fy(i, j = lj-1)
            const T f = lap[(lj + 1) * G::LX + i + 1] - lap[lj * G::LX + i + 1];
            const T *c = S + (lj + 1) * BX + (i + 2 + xs);  // in(i, j)
            fy[idx] = limit(f, c[BX] - c[0]);
        }
        __syncthreads();

        // phase 3: update and store
#pragma unroll
        for (int q = 0; q < PASSES; ++q) {
            const int j = (tid / GROUPS_I) + q * ROWS_PER_PASS;
            const int i = (tid % GROUPS_I) * VEC;
            if (j >= nj_valid || i >= ni_valid) continue;
            T r[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int ie = i + e;
                const T div = (fx[j * (TI + 1) + ie + 1] - fx[j * (TI + 1) + ie]) +
                              (fy[(j + 1) * TI + ie] - fy[j * TI + ie]);
                const T x = S[(j + 2) * BX + ie + 2 + xs];
                r[e] = x - cf[q][e] * div;
            }
            T *op = out.p + (int64_t)(ti0 + i) + (int64_t)(tj0 + j) * out.sj + (int64_t)k * out.sk;
            if (i + VEC <= ni_valid) {
                store_vec<T, VEC>(op, r);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (i + e < ni_valid) op[e] = r[e];
            }
        }
        if (!USE_TMA) __syncthreads();  // the box buffer is overwritten by the next level
    }

    if (USE_TMA && failed) {
        // a load never completed: wait (bounded) for the ones still in flight
        // so no TMA write lands after this CTA has released its shared memory
        if (tid == 0)
            for (int s = 0; s < STAGES; ++s) mbar_wait(&bars[s], 0), mbar_wait(&bars[s], 1);
        __syncthreads();
    }
}

}  // namespace gtb
