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
//
// Two arithmetic forms:
//  * hdiff_kernel: the definition in the storage type (binary32 or binary64).
//  * hdiff_fx_kernel (binary64 storage): B300's FP64 pipe issues ~1/60 of the
//    FP32/INT rate, so the Laplacian -> flux -> divergence chain, which only
//    adds and subtracts in with small integer weights, runs EXACTLY in int64
//    fixed point on the integer pipe.  Per tile level, E = the largest binary64
//    exponent in the box; every in becomes X = in * 2^(1078-E) truncated to an
//    integer (exact for |in| >= 2^(E-1026), absolute error < 2^(E-1078) below
//    that, i.e. < 2^-55 of the box maximum), so |X| < 2^56 and every
//    intermediate fits int64 (|D| < 64 max|X| < 2^62).  The limiter takes the
//    sign of the exact flux and the exact sign of in[i+1]-in[i] (from X, or
//    from the binary64 bit patterns when two inputs truncate alike).  Only
//    out = in - coeff*D stays on the FP64 pipe (one FMA per point).  A level
//    whose box holds inf/NaN or extreme exponents takes the binary64 phases.
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
    // temporaries: lap [LY][LX], fx [TJ][TI+1], fy [TJ+1][TI]
    static constexpr int tmp_elems = LX * LY + (TI + 1) * TJ + TI * (TJ + 1);
};

// FX: the fixed-point form adds an int64 copy of the box.
template <typename T, int TI, int TJ, int STAGES, bool FX>
constexpr int hdiff_smem_bytes() {
    using G = HdiffTile<T, TI, TJ>;
    return STAGES * G::stage_stride + G::tmp_elems * 8 + (FX ? G::box_elems * 8 : 0) + 64 * 4 + STAGES * 8 + 128;
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

// ------------------------------------------------------------- shared pieces
template <typename T, int TI, int TJ, int NT, int VEC>
struct HdiffCtx {
    using G = HdiffTile<T, TI, TJ>;
    static constexpr int GROUPS_I = TI / VEC;
    static constexpr int ROWS_PER_PASS = NT / GROUPS_I;
    static constexpr int PASSES = (TJ + ROWS_PER_PASS - 1) / ROWS_PER_PASS;
    static_assert(NT % GROUPS_I == 0, "thread count must cover whole tile rows");

    // coeff of this thread's outputs at level k (issued early to overlap the stencil)
    static __device__ __forceinline__ void load_coeff(T (&cf)[PASSES][VEC], const View<T> &coeff, int ti0, int tj0,
                                                      int k, int ni_valid, int nj_valid) {
        const int tid = threadIdx.x;
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
    }

    // binary-format phases (storage type arithmetic), temporaries in `tmp`
    static __device__ __forceinline__ void lap_phase(const T *S, T *lap, int xs) {
        for (int idx = threadIdx.x; idx < G::LX * G::LY; idx += NT) {
            const int li = idx % G::LX, lj = idx / G::LX;  // lap(i = li-1, j = lj-1)
            const T *c = S + (lj + 1) * G::BX + (li + 1 + xs);
            const T sum = ((c[1] + c[-1]) + c[G::BX]) + c[-G::BX];
            lap[idx] = T(4) * c[0] - sum;
        }
    }

    static __device__ __forceinline__ void flux_phase(const T *S, const T *lap, T *fx, T *fy, int xs) {
        for (int idx = threadIdx.x; idx < (TI + 1) * TJ; idx += NT) {
            const int li = idx % (TI + 1), j = idx / (TI + 1);  // fx(i = li-1, j)
            const T f = lap[(j + 1) * G::LX + li + 1] - lap[(j + 1) * G::LX + li];
            const T *c = S + (j + 2) * G::BX + (li + 1 + xs);  // in(i, j)
            fx[idx] = limit(f, c[1] - c[0]);
        }
        for (int idx = threadIdx.x; idx < TI * (TJ + 1); idx += NT) {
            const int i = idx % TI, lj = idx / TI;  // fy(i, j = lj-1)
            const T f = lap[(lj + 1) * G::LX + i + 1] - lap[lj * G::LX + i + 1];
            const T *c = S + (lj + 1) * G::BX + (i + 2 + xs);  // in(i, j)
            fy[idx] = limit(f, c[G::BX] - c[0]);
        }
    }

    template <typename DivF>
    static __device__ __forceinline__ void out_phase(const T *S, const T (&cf)[PASSES][VEC], const View<T> &out,
                                                     int ti0, int tj0, int k, int ni_valid, int nj_valid, int xs,
                                                     DivF update) {
        const int tid = threadIdx.x;
#pragma unroll
        for (int q = 0; q < PASSES; ++q) {
            const int j = (tid / GROUPS_I) + q * ROWS_PER_PASS;
            const int i = (tid % GROUPS_I) * VEC;
            if (j >= nj_valid || i >= ni_valid) continue;
            T r[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const T x = S[(j + 2) * G::BX + i + e + 2 + xs];
                r[e] = update(i + e, j, x, cf[q][e]);
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
    }
};

// Stage management shared by both kernels: TMA ring or cooperative loads.
template <typename T, int TI, int TJ, int NT, int STAGES, bool USE_TMA>
struct HdiffStager {
    using G = HdiffTile<T, TI, TJ>;
    unsigned char *base;
    uint64_t *bars;
    const CUtensorMap *map;
    int X, Y, Z0, nk;

    __device__ __forceinline__ void start() {
        if (!USE_TMA) return;
        if (threadIdx.x == 0) {
            prefetch_tensormap(map);
            for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int p = 0; p < STAGES && p < nk; ++p) issue(p);
    }
    __device__ __forceinline__ void issue(int p) {  // level p of the item into stage p % STAGES
        const int s = p % STAGES;
        mbar_arrive_expect_tx(&bars[s], G::box_bytes);
        tma_load_3d(base + s * G::stage_stride, map, &bars[s], X, Y, Z0 + p);
    }
    __device__ __forceinline__ const T *stage(int p) const {
        return reinterpret_cast<const T *>(base + (USE_TMA ? (p % STAGES) : 0) * G::stage_stride);
    }
    // make level p's box available; false if a TMA wait expired
    __device__ __forceinline__ bool acquire(int p, const View<T> &in, int ti0, int tj0, int k, int I, int J, int xs) {
        if (USE_TMA) return mbar_wait(&bars[p % STAGES], (p / STAGES) & 1);
        T *D = reinterpret_cast<T *>(base);
        for (int idx = threadIdx.x; idx < G::box_elems; idx += NT) {
            const int bx = idx % G::BX, by = idx / G::BX;
            const int i = ti0 - 2 - xs + bx, j = tj0 - 2 + by;  // domain-relative
            T v = T(0);
            if (i >= -2 && i < I + 2 && j >= -2 && j < J + 2)
                v = in.p[(int64_t)i + (int64_t)j * in.sj + (int64_t)k * in.sk];
            D[idx] = v;
        }
        return true;
    }
    // called after the first barrier of level p: every thread is done with level p-1
    __device__ __forceinline__ void refill_after(int p) {
        if (USE_TMA && threadIdx.x == 0 && p >= 1 && p - 1 + STAGES < nk) issue(p - 1 + STAGES);
    }
    __device__ __forceinline__ void drain_on_failure() {
        if (!USE_TMA) return;
        if (threadIdx.x == 0)
            for (int s = 0; s < STAGES; ++s) mbar_wait(&bars[s], 0), mbar_wait(&bars[s], 1);
        __syncthreads();
    }
};

// ------------------------------------------------------------- binary form
template <typename T, int TI, int TJ, int NT, int STAGES, bool USE_TMA, int VEC>
__global__ void __launch_bounds__(NT)
    hdiff_kernel(const __grid_constant__ CUtensorMap tmap, const View<T> in, const View<T> coeff,
                 const View<T> out, const HdiffGeom g) {
    using G = HdiffTile<T, TI, TJ>;
    using C = HdiffCtx<T, TI, TJ, NT, VEC>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    T *lap = reinterpret_cast<T *>(base + STAGES * G::stage_stride);
    T *fx = lap + G::LX * G::LY;  // [TJ][TI+1], column li <-> i = li - 1
    T *fy = fx + (TI + 1) * TJ;   // [TJ+1][TI], row lj <-> j = lj - 1
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + STAGES * G::stage_stride + G::tmp_elems * 8 + 64 * 4);

    const int tile = blockIdx.x % g.n_tiles, kchunk = blockIdx.x / g.n_tiles;
    const int ti0 = (tile % g.tiles_i) * TI, tj0 = (tile / g.tiles_i) * TJ;
    const int k0 = kchunk * g.kc;
    const int nk = min(g.kc, g.K - k0);
    if (nk <= 0) return;
    const int ni_valid = min(TI, g.I - ti0), nj_valid = min(TJ, g.J - tj0);
    const int xs = g.xs;

    HdiffStager<T, TI, TJ, NT, STAGES, USE_TMA> st{base, bars, &tmap, g.X0 + ti0, g.Y0 + tj0, g.Z0 + k0, nk};
    st.start();
    bool failed = false;
    for (int p = 0; p < nk; ++p) {
        const int k = k0 + p;
        T cf[C::PASSES][VEC];
        C::load_coeff(cf, coeff, ti0, tj0, k, ni_valid, nj_valid);
        if (!st.acquire(p, in, ti0, tj0, k, g.I, g.J, xs)) failed = true;
        if (__syncthreads_or(failed)) break;
        const T *S = st.stage(p);
        C::lap_phase(S, lap, xs);
        __syncthreads();
        st.refill_after(p);
        C::flux_phase(S, lap, fx, fy, xs);
        __syncthreads();
        C::out_phase(S, cf, out, ti0, tj0, k, ni_valid, nj_valid, xs, [&](int i, int j, T x, T c) {
            const T div = (fx[j * (TI + 1) + i + 1] - fx[j * (TI + 1) + i]) + (fy[(j + 1) * TI + i] - fy[j * TI + i]);
            return x - c * div;
        });
        if (!USE_TMA) __syncthreads();  // the box buffer is overwritten by the next level
    }
    if (failed) st.drain_on_failure();
}

// ------------------------------------------------------------- fixed-point form
// in -> X = trunc(in * 2^(1078 - E)) for the box's largest biased exponent E.
__device__ __forceinline__ int64_t to_fixed(double x, int E) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7FF);
    uint64_t m = b & 0x000FFFFFFFFFFFFFull;
    if (e) m |= 0x0010000000000000ull;
    else e = 1;  // subnormal: no implicit bit, exponent of the smallest normal
    const int sh = min(e - E + 3, 3);  // <= 3 for every value the scan covered
    uint64_t v;
    if (sh >= 0) v = m << sh;
    else v = (sh > -64) ? (m >> (-sh)) : 0ull;
    return (int64_t)b < 0 ? -(int64_t)v : (int64_t)v;
}

// D * 2^(E - 1078) rounded to nearest-even binary64 (E in [64, 2040], |D| < 2^62).
__device__ __forceinline__ double from_fixed(int64_t D, int E) {
    if (D == 0) return 0.0;
    const uint64_t sgn = (uint64_t)D & 0x8000000000000000ull;
    uint64_t a = D < 0 ? (uint64_t)(-D) : (uint64_t)D;
    const int lz = __clzll((long long)a);
    a <<= lz;  // leading one at bit 63
    uint64_t mant = a >> 11;
    const uint64_t rem = a & 0x7FFull;
    mant += (uint64_t)((rem > 0x400ull) | ((rem == 0x400ull) & (mant & 1ull)));
    const int64_t ebias = (int64_t)(63 - lz) + E - 55;  // biased exponent of the leading one
    return __longlong_as_double((long long)(sgn | (((uint64_t)(ebias - 1) << 52) + mant)));
}

// Exact sign of x1 - x0 for finite binary64 values (-0 == +0).
__device__ __forceinline__ int exact_dir(int64_t X1, int64_t X0, double x1, double x0) {
    if (X1 != X0) return X1 > X0 ? 1 : -1;
    const int64_t b1 = __double_as_longlong(x1), b0 = __double_as_longlong(x0);
    const int64_t k1 = b1 < 0 ? -(b1 & 0x7FFFFFFFFFFFFFFFll) : b1;
    const int64_t k0 = b0 < 0 ? -(b0 & 0x7FFFFFFFFFFFFFFFll) : b0;
    return (k1 > k0) - (k1 < k0);
}

__device__ __forceinline__ int64_t limit_fx(int64_t f, int dir) {
    return ((f > 0 && dir > 0) || (f < 0 && dir < 0)) ? 0 : f;
}

template <int TI, int TJ, int NT, int STAGES, bool USE_TMA, int VEC>
__global__ void __launch_bounds__(NT)
    hdiff_fx_kernel(const __grid_constant__ CUtensorMap tmap, const View<double> in, const View<double> coeff,
                    const View<double> out, const HdiffGeom g) {
    using T = double;
    using G = HdiffTile<T, TI, TJ>;
    using C = HdiffCtx<T, TI, TJ, NT, VEC>;
    constexpr int BX = G::BX;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    unsigned char *tmp = base + STAGES * G::stage_stride;
    int64_t *L = reinterpret_cast<int64_t *>(tmp);  // lap [LY][LX]
    int64_t *FX = L + G::LX * G::LY;                // [TJ][TI+1]
    int64_t *FY = FX + (TI + 1) * TJ;               // [TJ+1][TI]
    int64_t *X = FY + TI * (TJ + 1);                // box in fixed point [BY][BX]
    int *red = reinterpret_cast<int *>(X + G::box_elems);
    uint64_t *bars = reinterpret_cast<uint64_t *>(red + 64);
    // binary64 fallback views of the same temporaries
    double *lap = reinterpret_cast<double *>(L), *fx = reinterpret_cast<double *>(FX),
           *fy = reinterpret_cast<double *>(FY);

    const int tid = threadIdx.x;
    const int tile = blockIdx.x % g.n_tiles, kchunk = blockIdx.x / g.n_tiles;
    const int ti0 = (tile % g.tiles_i) * TI, tj0 = (tile / g.tiles_i) * TJ;
    const int k0 = kchunk * g.kc;
    const int nk = min(g.kc, g.K - k0);
    if (nk <= 0) return;
    const int ni_valid = min(TI, g.I - ti0), nj_valid = min(TJ, g.J - tj0);
    const int xs = g.xs;

    HdiffStager<T, TI, TJ, NT, STAGES, USE_TMA> st{base, bars, &tmap, g.X0 + ti0, g.Y0 + tj0, g.Z0 + k0, nk};
    st.start();
    bool failed = false;
    for (int p = 0; p < nk; ++p) {
        const int k = k0 + p;
        T cf[C::PASSES][VEC];
        C::load_coeff(cf, coeff, ti0, tj0, k, ni_valid, nj_valid);
        if (!st.acquire(p, in, ti0, tj0, k, g.I, g.J, xs)) failed = true;
        if (__syncthreads_or(failed)) break;
        const T *S = st.stage(p);

        // largest biased exponent over the columns the stencil reads (box columns xs .. xs+TI+3)
        unsigned emax = 0;
        for (int idx = tid; idx < G::BY * (TI + 4); idx += NT) {
            const int bx = idx % (TI + 4) + xs, by = idx / (TI + 4);
            const unsigned hi = (unsigned)__double2hiint(S[by * BX + bx]);
            emax = max(emax, (hi >> 20) & 0x7FFu);
        }
        emax = __reduce_max_sync(0xffffffffu, emax);
        if ((tid & 31) == 0) red[tid >> 5] = (int)emax;
        __syncthreads();
        st.refill_after(p);
        int E = 0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) E = max(E, red[w]);
        const bool fast = (E >= 64 && E <= 2040);

        if (fast) {
            for (int idx = tid; idx < G::BY * (TI + 4); idx += NT) {
                const int bx = idx % (TI + 4) + xs, by = idx / (TI + 4);
                X[by * BX + bx] = to_fixed(S[by * BX + bx], E);
            }
            __syncthreads();
            for (int idx = tid; idx < G::LX * G::LY; idx += NT) {
                const int li = idx % G::LX, lj = idx / G::LX;
                const int64_t *c = X + (lj + 1) * BX + (li + 1 + xs);
                L[idx] = 4 * c[0] - (((c[1] + c[-1]) + c[BX]) + c[-BX]);
            }
            __syncthreads();
            for (int idx = tid; idx < (TI + 1) * TJ; idx += NT) {
                const int li = idx % (TI + 1), j = idx / (TI + 1);  // fx(i = li-1, j)
                const int64_t f = L[(j + 1) * G::LX + li + 1] - L[(j + 1) * G::LX + li];
                const int o = (j + 2) * BX + (li + 1 + xs);  // in(i, j)
                FX[idx] = limit_fx(f, exact_dir(X[o + 1], X[o], S[o + 1], S[o]));
            }
            for (int idx = tid; idx < TI * (TJ + 1); idx += NT) {
                const int i = idx % TI, lj = idx / TI;  // fy(i, j = lj-1)
                const int64_t f = L[(lj + 1) * G::LX + i + 1] - L[lj * G::LX + i + 1];
                const int o = (lj + 1) * BX + (i + 2 + xs);  // in(i, j)
                FY[idx] = limit_fx(f, exact_dir(X[o + BX], X[o], S[o + BX], S[o]));
            }
            __syncthreads();
            C::out_phase(S, cf, out, ti0, tj0, k, ni_valid, nj_valid, xs, [&](int i, int j, double x, double c) {
                const int64_t D = (FX[j * (TI + 1) + i + 1] - FX[j * (TI + 1) + i]) + (FY[(j + 1) * TI + i] - FY[j * TI + i]);
                return fma(-c, from_fixed(D, E), x);
            });
        } else {
            C::lap_phase(S, lap, xs);
            __syncthreads();
            C::flux_phase(S, lap, fx, fy, xs);
            __syncthreads();
            C::out_phase(S, cf, out, ti0, tj0, k, ni_valid, nj_valid, xs, [&](int i, int j, double x, double c) {
                const double div = (fx[j * (TI + 1) + i + 1] - fx[j * (TI + 1) + i]) + (fy[(j + 1) * TI + i] - fy[j * TI + i]);
                return x - c * div;
            });
        }
        if (!USE_TMA) __syncthreads();  // the box buffer is overwritten by the next level
    }
    if (failed) st.drain_on_failure();
}

}  // namespace gtb
