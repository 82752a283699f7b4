// hdiff_kernels.cuh -- pieces shared by the hdiff kernels (GT4Py paper,
// Sec. 3.1, horizontal diffusion) and the vadv kernels:
//   * View / HdiffGeom: field views (pointer at the domain origin, i stride 1)
//     and the launch geometry of a tiled, K-chunked hdiff launch;
//   * 16-byte vector loads/stores;
//   * the exact int64 fixed-point form used for binary64 hdiff: B300's FP64
//     pipe issues ~1/60 of the FP32/INT rate, so the Laplacian -> flux ->
//     divergence chain, which only adds and subtracts its input with small
//     integer weights, runs exactly on the integer pipe.  Per strip, E = the
//     largest binary64 exponent among the values the stored outputs read;
//     every in becomes X = in * 2^(1078-E) truncated to an integer (exact for
//     |in| >= 2^(E-1026), error < 2^(E-1078), i.e. < 2^-55 of the strip's
//     largest input, below that), so |X| < 2^56 and every intermediate fits
//     int64 (|D| < 64 max|X| < 2^62).  The limiter takes the sign of the exact
//     flux and the exact sign of in[i+1]-in[i] (from X, or from the binary64
//     bit patterns when two inputs truncate alike).
#pragma once

#include "gtb_device.cuh"

namespace gtb {

template <typename T>
struct View {  // p points at compute-domain point (0,0,0); i stride is 1
    T *p;
    int64_t sj, sk;
    const void *lo = nullptr, *hi = nullptr;  // the storage's bytes [lo, hi) (null: not checked)
};

// Checked build (compiled with GTB_CHECKED: libgtb_checked.so).  Before its first
// access a kernel tests the first and the last element of each affine run of
// addresses it will touch (a column's levels, a strip's rows) against the storage
// the host declared for that field (shape and strides of its gtb_field); a run
// outside it sets the device error word to kDeviceErrBounds and the run is not
// accessed.  This is the build's stand-in for a memory sanitizer: it checks the
// kernels' own index arithmetic, not the caller's descriptors (the host validates
// those in every build).  In the default build the tests are compiled out, except
// in the batched column solve (vadv_batch_kernel), where they stay (see there).
constexpr int kDeviceErrBounds = 2;
#ifdef GTB_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// Whether elements a and b (the ends of a run) lie in v's storage (always true in the
// default build, and for views the host built without a storage range).
template <typename V, typename Q>
__device__ __forceinline__ bool in_storage(const View<V> &v, const Q *a, const Q *b) {
    if (!v.lo) return true;
    const char *lo = static_cast<const char *>(v.lo), *hi = static_cast<const char *>(v.hi);
    const char *x = reinterpret_cast<const char *>(a), *y = reinterpret_cast<const char *>(b);
    if (x >= lo && x + sizeof(Q) <= hi && y >= lo && y + sizeof(Q) <= hi) return true;
    atomicCAS(&g_device_error, 0, kDeviceErrBounds);
    return false;
}

struct HdiffGeom {
    int I, J, K;
    int tiles_i, tiles_j, n_tiles;
    int kc;          // K levels per work item
    int X0, Y0, Z0;  // tensor-map coordinate of box column/row 0 for tile (0,0), level 0
    int xs;          // box column of domain i = -2 (alignment shift, < 16/sizeof(T))
    int CX0, CY0, CZ0;  // coeff tensor-map coordinate of domain point (0,0,0) (coeff staged by TMA)
    int int_update;  // co-scheduled / fused producers: the update on the integer pipe (FixedF64T<true>::outx)
};

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

// Whether hdiff on an I x J domain reads in(i, j) (domain indices): the used
// Laplacians are those of [-1, I] x [0, J) (for fx) and [0, I) x [-1, J] (for
// fy), so the cells read are [-2, I+1] x [0, J), [-1, I] x [-1, J] and
// [0, I) x [-2, J+1]: the halo ring of width 2 minus three cells at each
// corner, whose contents the definition never uses.
__device__ __forceinline__ bool hdiff_reads(int i, int j, int I, int J) {
    if (i < -2 || i > I + 1 || j < -2 || j > J + 1) return false;
    const bool i_out = (i < -1 || i > I), j_out = (j < -1 || j > J);
    const bool i_in = (i >= 0 && i < I), j_in = (j >= 0 && j < J);
    return !((i_out && !j_in) || (j_out && !i_in));
}

// in -> X = trunc(in * 2^(1078 - E)) for the box's largest biased exponent E:
// the significand, pre-shifted by the 3 bits of headroom, shifted right by
// E - e (values above the scan's E, outside every stored output's reach, are
// clamped), then the sign applied.
__device__ __forceinline__ int64_t to_fixed(double x, int E) {
    const int hi = __double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const int eb = (hi >> 20) & 0x7FF;
    const unsigned mh = ((unsigned)hi & 0xFFFFFu) | (eb ? 0x100000u : 0u);  // subnormals: no implicit bit
    const uint64_t m3 = ((uint64_t)mh << 35) | ((uint64_t)lo << 3);
    const int r = min(max(E - max(eb, 1), 0), 63);
    const int64_t v = (int64_t)(m3 >> r);
    const int64_t sg = (int64_t)(hi >> 31);  // 0 or -1
    return (v ^ sg) - sg;
}

// D * 2^(E - 1078) rounded to nearest-even binary64 (E in [64, 2040], |D| < 2^62):
// the hardware int64 -> binary64 conversion rounds, the power of two is an
// exact exponent shift (the result stays normal in that range).
__device__ __forceinline__ double from_fixed(int64_t D, int E) {
    const double d = __ll2double_rn(D);
    const int hi = __double2hiint(d) + ((E - 1078) << 20);
    return D == 0 ? 0.0 : __hiloint2double(hi, __double2loint(d));
}

// The same value, bit for bit, computed on the integer pipe, for kernels whose
// FP64 pipe is the bottleneck (hdiff sharing SMs with the column solve): |D| has its leading
// one at bit msb; its top 53 bits form the significand m, the bits shifted out
// round it to nearest, ties to even (IEEE 754-2019, 4.3.1); the biased exponent
// is msb + 1023 + (E - 1078), always normal in that range.  The significand
// (implicit bit included) is added to the exponent field less one, so a
// rounding carry into bit 53 raises the exponent by itself.
__device__ __forceinline__ double from_fixed_int(int64_t D, int E) {
    if (D == 0) return 0.0;
    const uint64_t u = D < 0 ? 0ull - (uint64_t)D : (uint64_t)D;
    const int msb = 63 - __clzll((long long)u);
    const int sh = max(msb - 52, 0), ls = max(52 - msb, 0);
    uint64_t m = (u << ls) >> sh;
    const uint64_t rem = u & ((1ull << sh) - 1ull), half = sh ? 1ull << (sh - 1) : 1ull;
    m += (sh != 0) & ((rem > half) | ((rem == half) & (unsigned)(m & 1ull)));
    const uint64_t bits = ((uint64_t)(msb + E - 1078 + 1023 - 1) << 52) + m;
    return __longlong_as_double((long long)(bits | (D < 0 ? 0x8000000000000000ull : 0ull)));
}

// Exact sign of x1 - x0 for finite binary64 values (-0 == +0).
__device__ __forceinline__ int exact_dir(int64_t X1, int64_t X0, double x1, double x0) {
    if (X1 != X0) return X1 > X0 ? 1 : -1;
    const int64_t b1 = __double_as_longlong(x1), b0 = __double_as_longlong(x0);
    const int64_t k1 = b1 < 0 ? -(b1 & 0x7FFFFFFFFFFFFFFFll) : b1;
    const int64_t k0 = b0 < 0 ? -(b0 & 0x7FFFFFFFFFFFFFFFll) : b0;
    return (k1 > k0) - (k1 < k0);
}

}  // namespace gtb
