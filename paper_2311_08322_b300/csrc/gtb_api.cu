// gtb_api.cu -- the C ABI of libgtb (declared in include/gtb.h): argument
// validation (the run-time storage checks of the GT4Py paper, Sec. 3.1),
// domain deduction from field sizes and stencil reach (Sec. 2.2), TMA
// descriptor encoding and kernel dispatch.  Single translation unit: every
// kernel of the library is instantiated here.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "gtb.h"
#include "gtb_device.cuh"
#include "hdiff_kernels.cuh"
#include "hdiff_rs.cuh"
#include "vadv_kernels.cuh"
#include "adjoint_kernels.cuh"
#include "batch_kernels.cuh"
#include "fused_kernels.cuh"
#include "probe_kernels.cuh"

namespace gtb {

// ------------------------------------------------------------------ errors
static thread_local char t_err[512] = "";

static int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return code;
}

static int ok() {
    t_err[0] = 0;
    return GTB_OK;
}

static size_t dtype_size(int dt) { return dt == GTB_F64 ? 8 : dt == GTB_F32 ? 4 : 0; }

// ------------------------------------------------------------------ fields
struct Reach {  // points read/written outside the domain on each side
    int lo[3], hi[3];
};

static int check_field(const char *name, const gtb_field *f, int dtype) {
    if (!f) return fail(GTB_ERR_NULL, "%s: NULL field", name);
    if (!f->ptr) return fail(GTB_ERR_NULL, "%s: NULL data pointer", name);
    if (f->dtype != dtype) return fail(GTB_ERR_DTYPE, "%s: dtype %d differs from the call's dtype %d", name, f->dtype, dtype);
    if (f->reserved != 0) return fail(GTB_ERR_ARG, "%s: reserved must be 0", name);
    for (int d = 0; d < 3; ++d)
        if (f->shape[d] < 0 || f->shape[d] > (int64_t(1) << 31))
            return fail(GTB_ERR_EXTENT, "%s: bad shape[%d] = %lld", name, d, (long long)f->shape[d]);
    if (f->strides[0] != 1) return fail(GTB_ERR_LAYOUT, "%s: strides[0] must be 1 (i contiguous)", name);
    if (f->strides[1] < f->shape[0] || f->strides[2] < f->strides[1] * f->shape[1])
        return fail(GTB_ERR_LAYOUT, "%s: overlapping or negative strides (%lld, %lld)", name,
                    (long long)f->strides[1], (long long)f->strides[2]);
    if (reinterpret_cast<uintptr_t>(f->ptr) % dtype_size(dtype) != 0)
        return fail(GTB_ERR_LAYOUT, "%s: data pointer not aligned to its element size", name);
    return GTB_OK;
}

// Fold one field into the deduced domain (largest domain keeping its accesses inside).
static void shrink_domain(const gtb_field *f, const Reach &r, int64_t dom[3]) {
    for (int d = 0; d < 3; ++d) dom[d] = std::min(dom[d], f->shape[d] - f->origin[d] - r.hi[d]);
}

static int check_extent(const char *name, const gtb_field *f, const Reach &r, const int64_t dom[3]) {
    for (int d = 0; d < 3; ++d) {
        if (f->origin[d] - r.lo[d] < 0 || f->origin[d] + dom[d] + r.hi[d] > f->shape[d])
            return fail(GTB_ERR_EXTENT,
                        "%s: axis %d: origin %lld, domain %lld and stencil reach (-%d,+%d) leave the storage of extent %lld",
                        name, d, (long long)f->origin[d], (long long)dom[d], r.lo[d], r.hi[d], (long long)f->shape[d]);
    }
    return GTB_OK;
}

static void byte_range(const gtb_field *f, uintptr_t *lo, uintptr_t *hi) {
    const size_t es = dtype_size(f->dtype);
    *lo = reinterpret_cast<uintptr_t>(f->ptr);
    const int64_t last = (f->shape[0] > 0 && f->shape[1] > 0 && f->shape[2] > 0)
                             ? (f->shape[2] - 1) * f->strides[2] + (f->shape[1] - 1) * f->strides[1] + f->shape[0]
                             : 0;
    *hi = *lo + (uintptr_t)last * es;
}

static bool overlaps(const gtb_field *a, const gtb_field *b) {
    uintptr_t al, ah, bl, bh;
    byte_range(a, &al, &ah);
    byte_range(b, &bl, &bh);
    return al < bh && bl < ah;
}

static bool same_view(const gtb_field *a, const gtb_field *b) {
    return a->ptr == b->ptr && a->dtype == b->dtype && !memcmp(a->shape, b->shape, sizeof(a->shape)) &&
           !memcmp(a->strides, b->strides, sizeof(a->strides)) && !memcmp(a->origin, b->origin, sizeof(a->origin));
}

template <typename T>
static View<T> view_of(const gtb_field *f) {
    T *p = static_cast<T *>(f->ptr) + f->origin[0] + f->origin[1] * f->strides[1] + f->origin[2] * f->strides[2];
    View<T> v{p, f->strides[1], f->strides[2]};
    // the storage's bytes (for the kernels' address checks): its last element is
    // (shape - 1) along every axis
    int64_t last = -1;
    if (f->shape[0] > 0 && f->shape[1] > 0 && f->shape[2] > 0)
        last = (f->shape[0] - 1) + (f->shape[1] - 1) * f->strides[1] + (f->shape[2] - 1) * f->strides[2];
    const size_t es = dtype_size(f->dtype);
    v.lo = f->ptr;
    v.hi = static_cast<const char *>(f->ptr) + (last + 1) * (int64_t)es;
    return v;
}

static int resolve_domain(const int64_t *domain, int64_t dom[3]) {
    if (domain) {
        for (int d = 0; d < 3; ++d) {
            if (domain[d] < 0) return fail(GTB_ERR_EXTENT, "negative domain extent in axis %d", d);
            dom[d] = domain[d];
        }
    }
    for (int d = 0; d < 3; ++d)
        if (dom[d] < 0) dom[d] = 0;
        else if (dom[d] > (int64_t(1) << 30)) return fail(GTB_ERR_UNSUPPORTED, "domain extent too large in axis %d", d);
    return GTB_OK;
}

// ------------------------------------------------------------------ device helpers
static int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev;
}

static int sm_count() {
    static int cached[64] = {0};
    const int dev = current_device();
    if (dev < 64 && cached[dev]) return cached[dev];
    int n = 148;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (dev < 64) cached[dev] = n;
    return n;
}

// Raise a kernel's dynamic shared-memory limit once per (kernel, device).
static std::mutex g_prep_mu;
static std::unordered_map<const void *, unsigned long long> g_prep_done;  // device bit mask

template <typename K>
static cudaError_t prepare_kernel(K kernel, int smem_bytes) {
    const int dev = current_device();
    const void *key = reinterpret_cast<const void *>(kernel);
    std::lock_guard<std::mutex> lock(g_prep_mu);
    unsigned long long &mask = g_prep_done[key];
    if (dev < 64 && ((mask >> dev) & 1ull)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e == cudaSuccess && dev < 64) mask |= 1ull << dev;
    return e;
}

template <typename K>
static int resident_blocks(K kernel, int threads, int smem_bytes) {
    int nb = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem_bytes) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

// Whether a co-scheduled or fused launch fills the GPU (at least 85% of the CTAs it
// can hold at once): then its FP64 pipe is the bound and the producers' update goes
// to the integer pipe; a smaller grid is bound by the producers' per-level path and
// keeps the binary64 FMA.  Measured at K = 80, step: 256x256 (99% of capacity) 4%
// faster, 224x224 (76%) and below 6-15% slower; fused chain: 256x256 (86%) 2%,
// 512x512 5% faster, 240x240 (81%) even, 224x224 and below 6-14% slower.
// Capacity cached per (kernel, device).
static std::mutex g_fill_mu;
static std::unordered_map<const void *, std::vector<int>> g_fill_cap;  // per device: resident CTAs, 0 = unknown

template <typename K>
static int fills_gpu(K kernel, int threads, int smem_bytes, int64_t ctas) {
    const int dev = current_device();
    int cap = 0;
    {
        std::lock_guard<std::mutex> lock(g_fill_mu);
        std::vector<int> &v = g_fill_cap[reinterpret_cast<const void *>(kernel)];
        if ((int)v.size() <= dev) v.resize(dev + 1, 0);
        if (!v[dev]) v[dev] = resident_blocks(kernel, threads, smem_bytes) * sm_count();
        cap = v[dev];
    }
    return ctas * 20 >= (int64_t)cap * 17 ? 1 : 0;
}

static int launch_status(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GTB_ERR_LAUNCH, "%s: %s", what, cudaGetErrorString(e));
    return ok();
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// The column coefficients of vadv for beta_v and the face-velocity mode:
// a_k = bp * (-w_k/2) with w_k = s_k/2 (I-face average) or s_k (literal), so
// a_k = ka s_k with ka = (-bp/4) or (-bp/2); the explicit weights use bm.
static VadvGeom make_vadv_geom(const int64_t dom[3], bool literal, double dtr_stage, double beta_v) {
    VadvGeom g{};
    g.I = (int)dom[0], g.J = (int)dom[1], g.K = (int)dom[2];
    g.literal = literal ? 1 : 0;
    const double bp = 0.5 * (1.0 + beta_v), bm = 0.5 * (1.0 - beta_v);
    g.sym = (bp == bm) ? 1 : 0;
    g.dtr = dtr_stage;
    g.ka = (literal ? -0.5 : -0.25) * bp;
    g.kas = (literal ? -0.5 : -0.25) * bm;
    g.kg = g.kas - g.ka;
    int n = 0;
    const double m = std::frexp(-g.ka, &n);  // -ka = m 2^n, m in [0.5, 1)
    g.ka_pow2 = (m == 0.5 && n - 1 < 0 && n - 1 > -64) ? n - 1 : 0;
    return g;
}

// ------------------------------------------------------------------ hdiff
template <typename T>
struct HdiffCfg;
// Measured on B300 (row loop fully unrolled): binary64 fixed point runs best
// with 4 warps of 16 rows, binary32 with 8 warps of 8 rows (more resident
// warps to cover the latency chain of each row).
template <> struct HdiffCfg<double> {  // 64 x 64 tile, 4 warps of 16 rows, 2 columns per lane
    static constexpr int CPL = 2, W = 4, R = 16, STAGES = 2;
};
template <> struct HdiffCfg<float> {   // 128 x 64 tile, 8 warps of 8 rows, 4 columns per lane
    static constexpr int CPL = 4, W = 8, R = 8, STAGES = 2;
};
// coeff staged by TMA beside in (when coeff's layout allows a tensor map).  binary32:
// 128 x 32 tiles of 8 warps x 4 rows, 2 stages (72 KB).  Measured at 512x512x80
// (20-launch means, two input sets of 253 MB): 48.9 us, against 50.0 for 4 warps x 8
// rows, 49.7 for 8 x 4 with 3 stages, 52.0 for 4 x 4 with 3, 54.0 for 8 x 8 (128 x 64,
// 140 KB) and 56.4 for 4 x 8 with 3; 70.5 with coeff loaded row by row from global memory.
template <typename T>
struct HdiffCoeffTmaCfg;
template <> struct HdiffCoeffTmaCfg<float> {
    static constexpr bool kUse = true;
    static constexpr int CPL = 4, W = 8, R = 4, STAGES = 2;
};
template <> struct HdiffCoeffTmaCfg<double> {
    static constexpr bool kUse = false;
    static constexpr int CPL = 2, W = 4, R = 8, STAGES = 2;
};

template <typename T, bool TMA, typename C = HdiffCfg<T>, bool CTMA = false>
static int launch_hdiff_t(const CUtensorMap &map, const CUtensorMap &cmap, const View<T> &in, const View<T> &cf,
                          const View<T> &out, HdiffGeom g, int vec_ok, cudaStream_t st) {
    constexpr int STG = TMA ? C::STAGES : 1;
    // binary64: exact fixed-point lap/flux chain on the integer pipe; binary32: the definition
    constexpr bool FIXED = sizeof(T) == 8;
    constexpr int smem = hdiff_rs_smem_bytes<T, C::CPL, C::W, C::R, STG, CTMA>();
    constexpr int NT = 32 * C::W;
    auto kern = hdiff_rs_kernel<T, C::CPL, C::W, C::R, STG, TMA, FIXED, CTMA>;
    if (prepare_kernel(kern, smem) != cudaSuccess) return launch_status("hdiff: shared-memory attribute");
    static int slots_cache[64] = {0};
    const int dev = current_device();
    int slots = dev < 64 ? slots_cache[dev] : 0;
    if (!slots) {
        slots = resident_blocks(kern, NT, smem) * sm_count();
        if (dev < 64) slots_cache[dev] = slots;
    }
    // one wave of work items: split K so that tiles x chunks fills the resident slots
    const int chunks = std::max(1, std::min(g.K, slots / std::max(1, g.n_tiles)));
    g.kc = (g.K + chunks - 1) / chunks;
    const int items = g.n_tiles * ((g.K + g.kc - 1) / g.kc);
    kern<<<items, NT, smem, st>>>(map, cmap, in, cf, out, g, vec_ok);
    return launch_status("hdiff launch");
}

// TMA descriptor of coeff for (bx x by x 1) boxes whose corner is a tile's first domain
// point: the tile corner's i coordinate must start on a 16-byte boundary (every tile's
// does when the domain's first point does, tiles being multiples of 16 bytes wide).
// Sets g.CX0/CY0/CZ0; false when the layout, the alignment or the driver rules it out.
template <typename T>
static bool encode_coeff_map(const gtb_field *fc, int bx, int by, HdiffGeom &g, CUtensorMap &map) {
    const size_t es = sizeof(T);
    const uintptr_t base = reinterpret_cast<uintptr_t>(fc->ptr);
    const uintptr_t abase = base & ~uintptr_t(15);
    const int shift = (int)((base - abase) / es);
    constexpr int kAlign = 16 / (int)sizeof(T);
    const int x0 = (int)fc->origin[0] + shift;
    bool ok = encode_fn() != nullptr && (fc->strides[1] * es) % 16 == 0 && (fc->strides[2] * es) % 16 == 0 &&
              fc->strides[2] * es < (1ull << 40) && fc->shape[0] + shift < (1ll << 31) && x0 % kAlign == 0 &&
              (bx * (int)es) % 16 == 0;
    memset(&map, 0, sizeof(map));
    if (!ok) return false;
    g.CX0 = x0, g.CY0 = (int)fc->origin[1], g.CZ0 = (int)fc->origin[2];
    cuuint64_t gdim[3] = {(cuuint64_t)(fc->shape[0] + shift), (cuuint64_t)fc->shape[1], (cuuint64_t)fc->shape[2]};
    cuuint64_t gstride[2] = {(cuuint64_t)(fc->strides[1] * es), (cuuint64_t)(fc->strides[2] * es)};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(&map, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                             reinterpret_cast<void *>(abase), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// TMA descriptor of hdiff's input for a (bx x by x 1) box whose column 0 is
// domain i = -2 rounded down to 16 bytes: storage base rounded down to 16 B,
// pitches multiples of 16 B.  Sets g.X0/Y0/Z0 and the alignment shift g.xs;
// false (g.xs = 0) when the layout or the driver rules TMA out.
template <typename T>
static bool encode_in_map(const gtb_field *fin, int bx, int by, HdiffGeom &g, CUtensorMap &map) {
    const size_t es = sizeof(T);
    const uintptr_t base = reinterpret_cast<uintptr_t>(fin->ptr);
    const uintptr_t abase = base & ~uintptr_t(15);
    const int shift = (int)((base - abase) / es);
    constexpr int kAlign = 16 / (int)sizeof(T);
    bool tma = encode_fn() != nullptr && (fin->strides[1] * es) % 16 == 0 && (fin->strides[2] * es) % 16 == 0 &&
               fin->strides[2] * es < (1ull << 40) && fin->shape[0] + shift < (1ll << 31);
    memset(&map, 0, sizeof(map));
    if (tma) {
        const int xraw = (int)fin->origin[0] - 2 + shift;
        g.xs = xraw % kAlign;
        g.X0 = xraw - g.xs;
        g.Y0 = (int)fin->origin[1] - 2;
        g.Z0 = (int)fin->origin[2];
        cuuint64_t gdim[3] = {(cuuint64_t)(fin->shape[0] + shift), (cuuint64_t)fin->shape[1], (cuuint64_t)fin->shape[2]};
        cuuint64_t gstride[2] = {(cuuint64_t)(fin->strides[1] * es), (cuuint64_t)(fin->strides[2] * es)};
        cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = encode_fn()(&map, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                 3, reinterpret_cast<void *>(abase), gdim, gstride, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) tma = false;
    }
    if (!tma) g.xs = 0;
    return tma;
}

template <typename T, typename C>
static HdiffGeom hdiff_geom(const int64_t dom[3]) {
    using Tile = RsTile<T, C::CPL, C::W, C::R>;
    HdiffGeom g{};
    g.I = (int)dom[0], g.J = (int)dom[1], g.K = (int)dom[2];
    g.tiles_i = (g.I + Tile::TI - 1) / Tile::TI;
    g.tiles_j = (g.J + Tile::TJ - 1) / Tile::TJ;
    g.n_tiles = g.tiles_i * g.tiles_j;
    return g;
}

template <typename T>
static int run_hdiff(const gtb_field *fin, const gtb_field *fcf, const gtb_field *fout, const int64_t dom[3],
                     cudaStream_t st) {
    const View<T> in = view_of<T>(fin), cf = view_of<T>(fcf), out = view_of<T>(fout);
    const size_t es = sizeof(T);
    auto aligned = [&](const View<T> &v) {
        return reinterpret_cast<uintptr_t>(v.p) % 16 == 0 && (v.sj * es) % 16 == 0 && (v.sk * es) % 16 == 0;
    };
    CUtensorMap map, cmap;
    if constexpr (HdiffCoeffTmaCfg<T>::kUse) {
        // in and coeff both by TMA when both layouts allow it, out by vector stores
        using C = HdiffCoeffTmaCfg<T>;
        using Tile = RsTile<T, C::CPL, C::W, C::R, true>;
        HdiffGeom g = hdiff_geom<T, C>(dom);
        if (aligned(out) && encode_in_map<T>(fin, Tile::BX, Tile::BY, g, map) &&
            encode_coeff_map<T>(fcf, Tile::TI, Tile::TJ, g, cmap))
            return launch_hdiff_t<T, true, C, true>(map, cmap, in, cf, out, g, 1, st);
    }
    using C = HdiffCfg<T>;
    using Tile = RsTile<T, C::CPL, C::W, C::R>;
    HdiffGeom g = hdiff_geom<T, C>(dom);
    const bool tma = encode_in_map<T>(fin, Tile::BX, Tile::BY, g, map);
    const int vec = (aligned(cf) && aligned(out)) ? 1 : 0;
    return tma ? launch_hdiff_t<T, true>(map, map, in, cf, out, g, vec, st)
               : launch_hdiff_t<T, false>(map, map, in, cf, out, g, vec, st);
}

// ------------------------------------------------------------------ vadv
constexpr int kVadvMaxK = 448;

// A binary32 field as pairs of columns (fpair): its domain column 0 8-byte aligned and
// its strides even, so that column 2i starts a pair.
static bool pairs_fit(const gtb_field *f) {
    const View<float> v = view_of<float>(f);
    return reinterpret_cast<uintptr_t>(v.p) % 8 == 0 && v.sj % 2 == 0 && v.sk % 2 == 0;
}
template <typename C>
static View<C> pair_view(const gtb_field *f) {
    const View<float> v = view_of<float>(f);
    View<C> pv{reinterpret_cast<C *>(v.p), v.sj / 2, v.sk / 2};
    pv.lo = v.lo, pv.hi = v.hi;
    return pv;
}

// Double-float columns two per thread (packed binary32 pairs): I even and every field
// pair-aligned; the workspace and the kept factors keep the one-column layout.
template <int BJ>
static int launch_vadv_pairs(const gtb_field *const f[6], const VadvGeom &g, void *ws, cudaStream_t st, void *ws2,
                             void *rsave, bool packed) {
    VadvGeom gp = g;
    gp.I = g.I / 2;
    dfpair *w = static_cast<dfpair *>(ws);
    dfpair *w2 = ws2 ? static_cast<dfpair *>(ws2) : w + (size_t)gp.K * gp.I * gp.J;
    dim3 block(32, BJ), grid((gp.I + 31) / 32, (gp.J + BJ - 1) / BJ);
    auto kern = packed ? vadv_kernel<fpair, dfpair, BJ, false, true, kStatePacked> : vadv_kernel<fpair, dfpair, BJ, false, true>;
    kern<<<grid, block, 0, st>>>(pair_view<const fpair>(f[0]), pair_view<const fpair>(f[1]),
                                 pair_view<const fpair>(f[2]), pair_view<const fpair>(f[3]),
                                 pair_view<const fpair>(f[4]), pair_view<fpair>(f[5]), gp, w, w2,
                                 static_cast<dfpair *>(rsave));
    return launch_status("vadv launch");
}

// Workspace form: c' in ws and the second state array in ws2 (by default right after c'),
// 1/p_k in rsave when the factors are kept (the chained call's binary32 storage path).
// packed (double-float, no rsave): the column state in 48 bits (GTB_STATE48).
template <typename T, typename N, int BJ, bool WS>
static int launch_vadv_t(const gtb_field *const f[6], const VadvGeom &g, void *ws, cudaStream_t st,
                         void *ws2 = nullptr, void *rsave = nullptr, bool packed = false) {
    if constexpr (std::is_same<T, float>::value && std::is_same<N, df>::value && WS) {
        bool fit = g.I % 2 == 0;
        for (int q = 0; q < 6; ++q) fit = fit && pairs_fit(f[q]);
        if (fit) return launch_vadv_pairs<BJ>(f, g, ws, st, ws2, rsave, packed && !rsave);
    }
    constexpr bool DPG = vadv_dp_global<T, N>();
    auto kern = vadv_kernel<T, N, BJ, DPG, WS>;
    if constexpr (is_df<N>() && WS) {
        if (packed && !rsave) kern = vadv_kernel<T, N, BJ, DPG, WS, kStatePacked>;
    }
    const int smem = WS ? 0 : (int)(vadv_smem_per_col_level<T, N>() * g.K * 32 * BJ);
    if (!WS && prepare_kernel(kern, 227 * 1024) != cudaSuccess)
        return launch_status("vadv: shared-memory attribute");
    N *w = static_cast<N *>(ws);
    N *w2 = ws2 ? static_cast<N *>(ws2) : (WS ? w + (size_t)g.K * g.I * g.J : nullptr);
    dim3 block(32, BJ), grid((g.I + 31) / 32, (g.J + BJ - 1) / BJ);
    kern<<<grid, block, smem, st>>>(view_of<const T>(f[0]), view_of<const T>(f[1]), view_of<const T>(f[2]),
                                    view_of<const T>(f[3]), view_of<const T>(f[4]), view_of<T>(f[5]), g, w, w2,
                                    static_cast<N *>(rsave));
    return launch_status("vadv launch");
}

template <typename T, typename N>
static size_t vadv_ws_bytes(const int64_t dom[3]) {
    return (size_t)vadv_state_arrays<T, N>() * sizeof(N) * (size_t)dom[0] * (size_t)dom[1] * (size_t)dom[2];
}

// With a large enough workspace: column state in global memory (L2), two warps
// per block.  Without: column state in shared memory, two warps per block while
// it stays within 48 KB (several blocks per SM), else one.
template <typename T, typename N>
static int run_vadv_n(const gtb_field *const f[6], const VadvGeom &g, void *ws, size_t ws_bytes, cudaStream_t st,
                      bool packed = false) {
    const int64_t dom[3] = {g.I, g.J, g.K};
    if (ws && ws_bytes >= vadv_ws_bytes<T, N>(dom))
        return launch_vadv_t<T, N, 2, true>(f, g, ws, st, nullptr, nullptr, packed);
    const size_t per_col = vadv_smem_per_col_level<T, N>() * (size_t)g.K;
    if (per_col * 64 <= 48 * 1024) return launch_vadv_t<T, N, 2, false>(f, g, nullptr, st);
    return launch_vadv_t<T, N, 1, false>(f, g, nullptr, st);
}

static size_t vadv_ws_bytes_for(int dt, int prec, const int64_t dom[3]) {
    if (dt == GTB_F64) return vadv_ws_bytes<double, double>(dom);
    if (prec == GTB_PREC_F64) return vadv_ws_bytes<float, double>(dom);
    if (prec == GTB_PREC_DF) return vadv_ws_bytes<float, df>(dom);
    return vadv_ws_bytes<float, float>(dom);
}

// ------------------------------------------------------------------ adjoints
template <typename T, typename N, int BJ, bool WS, bool FACT = false>
static int launch_vadv_adj_t(const gtb_field *const f[6], const VadvGeom &g, int accumulate, int merge, void *ws,
                             cudaStream_t st) {
    auto kern = vadv_adj_kernel<T, N, BJ, WS, FACT>;
    const int smem = WS ? 0 : (int)(2 * sizeof(N) * g.K * 32 * BJ);
    if (!WS && prepare_kernel(kern, 227 * 1024) != cudaSuccess)
        return launch_status("vadv_adj: shared-memory attribute");
    auto ov = [&](const gtb_field *x) { return x ? view_of<T>(x) : View<T>{nullptr, 0, 0}; };
    dim3 block(32, BJ), grid((g.I + 31) / 32, (g.J + BJ - 1) / BJ);
    kern<<<grid, block, smem, st>>>(view_of<const T>(f[0]), view_of<const T>(f[1]), ov(f[2]), ov(f[3]), ov(f[4]),
                                    ov(f[5]), g, accumulate, merge, static_cast<N *>(ws));
    return launch_status("vadv_adj launch");
}

template <typename T, typename N>
static size_t vadv_adj_ws_bytes(const int64_t dom[3]) {
    return 2 * sizeof(N) * (size_t)dom[0] * (size_t)dom[1] * (size_t)dom[2];
}

template <typename T, typename N>
static int run_vadv_adj_n(const gtb_field *const f[6], const VadvGeom &g, int accumulate, int merge, void *ws,
                          size_t ws_bytes, bool factors, cudaStream_t st) {
    const int64_t dom[3] = {g.I, g.J, g.K};
    if (factors) return launch_vadv_adj_t<T, N, 2, true, true>(f, g, accumulate, merge, ws, st);
    if (ws && ws_bytes >= vadv_adj_ws_bytes<T, N>(dom)) return launch_vadv_adj_t<T, N, 2, true>(f, g, accumulate, merge, ws, st);
    const size_t per_col = 2 * sizeof(N) * (size_t)g.K;
    if (per_col * 64 <= 48 * 1024) return launch_vadv_adj_t<T, N, 2, false>(f, g, accumulate, merge, nullptr, st);
    return launch_vadv_adj_t<T, N, 1, false>(f, g, accumulate, merge, nullptr, st);
}

static size_t vadv_adj_ws_bytes_for(int dt, int prec, const int64_t dom[3]) {
    if (dt == GTB_F64) return vadv_adj_ws_bytes<double, double>(dom);
    if (prec == GTB_PREC_F64) return vadv_adj_ws_bytes<float, double>(dom);
    if (prec == GTB_PREC_DF) return vadv_adj_ws_bytes<float, df>(dom);
    return vadv_adj_ws_bytes<float, float>(dom);
}

template <typename T>
static int run_hdiff_adj(const gtb_field *fin, const gtb_field *fcf, const gtb_field *fob, const gtb_field *fib,
                         const gtb_field *fcb, int accumulate, const int64_t dom[3], cudaStream_t st) {
    constexpr int TI = 52, TJ = 20, NT = 256;
    auto kern = hdiff_adj_kernel<T, TI, TJ, NT>;
    constexpr int smem = hdiff_adj_smem_bytes<T, TI, TJ>();
    if (prepare_kernel(kern, smem) != cudaSuccess) return launch_status("hdiff_adj: shared-memory attribute");
    HadjGeom g{};
    g.I = (int)dom[0], g.J = (int)dom[1], g.K = (int)dom[2];
    g.tiles_i = (g.I + 4 + TI - 1) / TI;
    g.tiles_j = (g.J + 4 + TJ - 1) / TJ;
    g.accumulate_coeff_bar = accumulate;
    dim3 grid(g.tiles_i * g.tiles_j, g.K);
    kern<<<grid, NT, smem, st>>>(view_of<const T>(fin), view_of<const T>(fcf), view_of<const T>(fob), view_of<T>(fib),
                                 fcb ? view_of<T>(fcb) : View<T>{nullptr, 0, 0}, g);
    return launch_status("hdiff_adj launch");
}

template <typename T>
static int run_halo(const gtb_field *f, int hi, int hj, const int64_t dom[3], bool adjoint, cudaStream_t st) {
    const View<T> v = view_of<T>(f);
    const int64_t rows_full = std::min<int64_t>(dom[1], 2 * hj);
    const int64_t band = rows_full * dom[0] + (dom[1] - rows_full) * std::min<int64_t>(dom[0], 2 * hi);
    const int64_t n = adjoint ? band * dom[2] : (dom[0] + 2 * hi) * (dom[1] + 2 * hj) * dom[2];
    if (n == 0) return ok();
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, (int64_t)sm_count() * 16);
    if (adjoint)
        halo_periodic_adj_kernel<T><<<blocks, threads, 0, st>>>(v, (int)dom[0], (int)dom[1], (int)dom[2], hi, hj);
    else
        halo_periodic_kernel<T><<<blocks, threads, 0, st>>>(v, (int)dom[0], (int)dom[1], (int)dom[2], hi, hj);
    return launch_status(adjoint ? "halo_periodic_adj launch" : "halo_periodic launch");
}

// ------------------------------------------------------------------ fused hdiff -> vadv
// Column tile TI x TJ (TI*TJ/32 consumer warps) and PW producer warps per CTA,
// measured on B300: binary64 runs best with 32 x 2 tiles (1024 CTAs at 256 x 256,
// every column resident at once, as the FP64 column solve needs).  Binary32 storage
// does not use the fused kernel (run_chain32_n).
template <typename T>
struct FusedCfg;
template <> struct FusedCfg<double> { static constexpr int TI = 32, TJ = 2, PW = 2; };
constexpr int kFusedStages = 2, kFusedRing = 8;

// Workspace of the chained call: c', then 1/p when the factors are kept, then e
// when it cannot be parked in the output (all [K][I*J] arrays of N); for binary32
// storage then h itself (chain_h_layout), which goes through the workspace there.
template <typename T, typename N>
static size_t fused_state_bytes(const int64_t dom[3], bool save) {
    const size_t arr = sizeof(N) * (size_t)dom[0] * (size_t)dom[1] * (size_t)dom[2];
    return arr * ((vadv_dp_global<T, N>() ? 1 : 2) + (save ? 1 : 0));
}

// h of the binary32 chained call: rows padded to 32 values (128 bytes), the region
// 256-byte aligned after the state arrays.  Returns its byte offset; *bytes its size.
static size_t chain_h_layout(size_t state_bytes, const int64_t dom[3], int64_t *pitch, size_t *bytes) {
    *pitch = (dom[0] + 31) / 32 * 32;
    *bytes = sizeof(float) * (size_t)(*pitch) * (size_t)dom[1] * (size_t)dom[2];
    return (state_bytes + 255) / 256 * 256;
}

template <typename T, typename N>
static size_t fused_ws_bytes(const int64_t dom[3], bool save) {
    const size_t st = fused_state_bytes<T, N>(dom, save);
    if (sizeof(T) == 8) return st;
    int64_t pitch;
    size_t hb;
    return chain_h_layout(st, dom, &pitch, &hb) + hb;
}

static size_t fused_ws_bytes_for(int dt, int prec, const int64_t dom[3], bool save) {
    if (dt == GTB_F64) return fused_ws_bytes<double, double>(dom, save);
    if (prec == GTB_PREC_F64) return fused_ws_bytes<float, double>(dom, save);
    if (prec == GTB_PREC_DF) return fused_ws_bytes<float, df>(dom, save);
    return fused_ws_bytes<float, float>(dom, save);
}

template <typename T, typename N, bool TMA>
static int launch_fused_t(const CUtensorMap &map, const gtb_field *const f[6], const HdiffGeom &hg,
                          const VadvGeom &g, void *ws, bool save, cudaStream_t st) {
    using C = FusedCfg<T>;
    constexpr bool DPG = vadv_dp_global<T, N>();
    constexpr int STG = TMA ? kFusedStages : 1;
    using Lay = FusedLayout<T, C::TI, C::TJ, C::PW, STG, kFusedRing>;
    auto kern = hdiff_vadv_kernel<T, N, C::TI, C::TJ, C::PW, STG, kFusedRing, TMA, DPG>;
    if (prepare_kernel(kern, Lay::smem_bytes) != cudaSuccess) return launch_status("hdiff_vadv: shared-memory attribute");
    dim3 grid((g.I + C::TI - 1) / C::TI, (g.J + C::TJ - 1) / C::TJ);
    const size_t arr = (size_t)g.I * g.J * g.K;  // values of N per [K][I*J] array
    HdiffGeom hgl = hg;
    hgl.int_update = fills_gpu(kern, C::TI * C::TJ + 32 * C::PW, Lay::smem_bytes, (int64_t)grid.x * grid.y);
    kern<<<grid, C::TI * C::TJ + 32 * C::PW, Lay::smem_bytes, st>>>(
        map, view_of<const T>(f[0]), view_of<const T>(f[1]), view_of<const T>(f[2]), view_of<const T>(f[3]),
        view_of<const T>(f[4]), view_of<T>(f[5]), hgl, g, static_cast<N *>(ws),
        save ? static_cast<N *>(ws) + arr : nullptr, static_cast<N *>(ws) + (save ? 2 : 1) * arr);
    return launch_status("hdiff_vadv launch");
}

// f = {in, coeff, wcon, utens, utens_stage, utens_stage_out}
template <typename T, typename N>
static int run_fused_n(const gtb_field *const f[6], const VadvGeom &g, void *ws, bool save, cudaStream_t st) {
    using Tile = FusedTile<T, FusedCfg<T>::TI, FusedCfg<T>::TJ>;
    HdiffGeom hg{};
    hg.I = g.I, hg.J = g.J, hg.K = g.K;
    CUtensorMap map;
    const bool tma = encode_in_map<T>(f[0], Tile::BX, Tile::BY, hg, map);
    return tma ? launch_fused_t<T, N, true>(map, f, hg, g, ws, save, st)
               : launch_fused_t<T, N, false>(map, f, hg, g, ws, save, st);
}

// Binary32 storage: the chain as its two kernels back to back, h through the workspace.
// On B300 hdiff (coeff staged by TMA, bound by HBM) and the FP32-pipe column solve each
// run faster on their own than sharing SMs in one kernel (512x512x80, double-float:
// 49.9 + 218 us against 409 us).  f = {in, coeff, wcon, utens, utens_stage, out}.
template <typename N>
static int run_chain32_n(const gtb_field *const f[6], const VadvGeom &g, const int64_t dom[3], void *ws, bool save,
                         cudaStream_t st) {
    int64_t pitch;
    size_t hb;
    const size_t off = chain_h_layout(fused_state_bytes<float, N>(dom, save), dom, &pitch, &hb);
    const gtb_field hf{static_cast<unsigned char *>(ws) + off, GTB_F32, 0, {pitch, dom[1], dom[2]},
                       {1, pitch, pitch * dom[1]}, {0, 0, 0}};
    int rc;
    if ((rc = run_hdiff<float>(f[0], f[1], &hf, dom, st))) return rc;
    const gtb_field *fv[6] = {&hf, f[2], &hf, f[3], f[4], f[5]};  // u_stage = u_pos = h
    const size_t arr = (size_t)dom[0] * dom[1] * dom[2];
    N *w = static_cast<N *>(ws);
    return launch_vadv_t<float, N, 2, true>(fv, g, w, st, w + (save ? 2 : 1) * arr, save ? w + arr : nullptr);
}

// ------------------------------------------------------------------ co-scheduled step
// 32 x 2 column tile: 2 vadv (consumer) warps + 2 hdiff (producer) warps per CTA,
// at most 73 registers a thread so that 7 CTAs (every column of 256 x 256) are
// resident per SM.
constexpr int kPairBJ = 2, kPairPW = 2;

// fh = {in, coeff, hdiff_out}; fv = {u_stage, wcon, u_pos, utens, utens_stage, utens_stage_out}
template <typename T, typename N, bool TMA>
static int launch_pair_t(const CUtensorMap &map, const gtb_field *const fh[3], const gtb_field *const fv[6],
                         const HdiffGeom &hg, const VadvGeom &g, void *ws, cudaStream_t st) {
    constexpr bool DPG = vadv_dp_global<T, N>();
    constexpr int STG = TMA ? kFusedStages : 1;
    using Lay = FusedLayout<T, 32, kPairBJ, kPairPW, STG, 1>;
    auto kern = hdiff_vadv_pair_kernel<T, N, kPairBJ, kPairPW, STG, TMA, DPG>;
    if (prepare_kernel(kern, Lay::smem_bytes) != cudaSuccess) return launch_status("step: shared-memory attribute");
    dim3 grid((g.I + 31) / 32, (g.J + kPairBJ - 1) / kPairBJ);
    HdiffGeom hgl = hg;
    hgl.int_update = fills_gpu(kern, 32 * (kPairBJ + kPairPW), Lay::smem_bytes, (int64_t)grid.x * grid.y);
    kern<<<grid, 32 * (kPairBJ + kPairPW), Lay::smem_bytes, st>>>(
        map, view_of<const T>(fh[0]), view_of<const T>(fh[1]), view_of<T>(fh[2]), view_of<const T>(fv[0]),
        view_of<const T>(fv[1]), view_of<const T>(fv[2]), view_of<const T>(fv[3]), view_of<const T>(fv[4]),
        view_of<T>(fv[5]), hgl, g, static_cast<N *>(ws));
    return launch_status("step launch");
}

template <typename T, typename N>
static int run_pair_n(const gtb_field *const fh[3], const gtb_field *const fv[6], const VadvGeom &g, void *ws,
                      cudaStream_t st) {
    using Tile = FusedTile<T, 32, kPairBJ>;
    HdiffGeom hg{};
    hg.I = g.I, hg.J = g.J, hg.K = g.K;
    CUtensorMap map;
    const bool tma = encode_in_map<T>(fh[0], Tile::BX, Tile::BY, hg, map);
    return tma ? launch_pair_t<T, N, true>(map, fh, fv, hg, g, ws, st)
               : launch_pair_t<T, N, false>(map, fh, fv, hg, g, ws, st);
}

}  // namespace gtb

// ====================================================================== C ABI
using namespace gtb;

extern "C" int gtb_hdiff(const gtb_field *in, const gtb_field *coeff, const gtb_field *out, const int64_t *domain,
                         void *stream) {
    if (!in || !coeff || !out) return fail(GTB_ERR_NULL, "gtb_hdiff: NULL field");
    const int dt = in->dtype;
    if (!dtype_size(dt)) return fail(GTB_ERR_DTYPE, "gtb_hdiff: unknown dtype %d", dt);
    int rc;
    if ((rc = check_field("in", in, dt)) || (rc = check_field("coeff", coeff, dt)) ||
        (rc = check_field("out", out, dt)))
        return rc;
    const Reach r_in{{2, 2, 0}, {2, 2, 0}}, r0{{0, 0, 0}, {0, 0, 0}};
    int64_t dom[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
    if (!domain) {
        shrink_domain(in, r_in, dom);
        shrink_domain(coeff, r0, dom);
        shrink_domain(out, r0, dom);
    }
    if ((rc = resolve_domain(domain, dom))) return rc;
    if ((rc = check_extent("in", in, r_in, dom)) || (rc = check_extent("coeff", coeff, r0, dom)) ||
        (rc = check_extent("out", out, r0, dom)))
        return rc;
    if (overlaps(out, in)) return fail(GTB_ERR_ALIAS, "gtb_hdiff: out overlaps in");
    if (overlaps(out, coeff)) return fail(GTB_ERR_ALIAS, "gtb_hdiff: out overlaps coeff");
    if (dom[0] == 0 || dom[1] == 0 || dom[2] == 0) return ok();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return dt == GTB_F64 ? run_hdiff<double>(in, coeff, out, dom, st) : run_hdiff<float>(in, coeff, out, dom, st);
}

extern "C" int gtb_vadv(const gtb_field *u_stage, const gtb_field *wcon, const gtb_field *u_pos,
                        const gtb_field *utens, const gtb_field *utens_stage, const gtb_field *utens_stage_out,
                        double dtr_stage, double beta_v, int prec, unsigned flags, const int64_t *domain,
                        void *workspace, size_t workspace_bytes, void *stream) {
    const gtb_field *f[6] = {u_stage, wcon, u_pos, utens, utens_stage, utens_stage_out};
    static const char *names[6] = {"u_stage", "wcon", "u_pos", "utens", "utens_stage", "utens_stage_out"};
    for (int q = 0; q < 6; ++q)
        if (!f[q]) return fail(GTB_ERR_NULL, "gtb_vadv: NULL field %s", names[q]);
    const int dt = u_stage->dtype;
    if (!dtype_size(dt)) return fail(GTB_ERR_DTYPE, "gtb_vadv: unknown dtype %d", dt);
    int rc;
    for (int q = 0; q < 6; ++q)
        if ((rc = check_field(names[q], f[q], dt))) return rc;
    if (flags & ~(GTB_WCON_LITERAL | GTB_STATE48)) return fail(GTB_ERR_ARG, "gtb_vadv: unknown flags 0x%x", flags);
    if (prec < GTB_PREC_NATIVE || prec > GTB_PREC_DF) return fail(GTB_ERR_ARG, "gtb_vadv: unknown prec %d", prec);
    if ((flags & GTB_STATE48) && (dt != GTB_F32 || prec != GTB_PREC_DF))
        return fail(GTB_ERR_ARG, "gtb_vadv: GTB_STATE48 applies to GTB_F32 storage with GTB_PREC_DF");
    if (dt == GTB_F64 && prec != GTB_PREC_NATIVE)
        return fail(GTB_ERR_ARG, "gtb_vadv: FP64 storage computes in binary64 (prec must be GTB_PREC_NATIVE)");
    if (!(dtr_stage == dtr_stage) || !(beta_v == beta_v)) return fail(GTB_ERR_ARG, "gtb_vadv: NaN scalar");
    const bool literal = flags & GTB_WCON_LITERAL;
    const Reach r0{{0, 0, 0}, {0, 0, 0}}, rw{{0, 0, 0}, {literal ? 0 : 1, 0, 0}};
    int64_t dom[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
    if (!domain)
        for (int q = 0; q < 6; ++q) shrink_domain(f[q], q == 1 ? rw : r0, dom);
    if ((rc = resolve_domain(domain, dom))) return rc;
    for (int q = 0; q < 6; ++q)
        if ((rc = check_extent(names[q], f[q], q == 1 ? rw : r0, dom))) return rc;
    for (int q = 0; q < 5; ++q) {
        if (q == 4 && same_view(utens_stage_out, utens_stage)) continue;  // in place
        if (overlaps(utens_stage_out, f[q]))
            return fail(GTB_ERR_ALIAS, "gtb_vadv: utens_stage_out overlaps %s", names[q]);
    }
    // the shared-memory form holds K levels of column state per thread; a workspace lifts the limit
    if (dom[2] > kVadvMaxK && !(workspace && workspace_bytes >= vadv_ws_bytes_for(dt, prec, dom)))
        return fail(GTB_ERR_UNSUPPORTED, "gtb_vadv: K = %lld exceeds the limit %d without a workspace",
                    (long long)dom[2], kVadvMaxK);
    if (dom[0] == 0 || dom[1] == 0 || dom[2] == 0) return ok();

    const VadvGeom g = make_vadv_geom(dom, literal, dtr_stage, beta_v);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (workspace) {
        if (reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
            return fail(GTB_ERR_LAYOUT, "gtb_vadv: workspace must be 16-byte aligned");
        const gtb_field wsf{workspace, dt, 0, {(int64_t)(workspace_bytes / dtype_size(dt)), 1, 1},
                            {1, (int64_t)(workspace_bytes / dtype_size(dt)), (int64_t)(workspace_bytes / dtype_size(dt))},
                            {0, 0, 0}};
        for (int q = 0; q < 6; ++q)
            if (overlaps(&wsf, f[q])) return fail(GTB_ERR_ALIAS, "gtb_vadv: workspace overlaps %s", names[q]);
    }
    if (dt == GTB_F64) return run_vadv_n<double, double>(f, g, workspace, workspace_bytes, st);
    if (prec == GTB_PREC_F64) return run_vadv_n<float, double>(f, g, workspace, workspace_bytes, st);
    if (prec == GTB_PREC_DF)
        return run_vadv_n<float, df>(f, g, workspace, workspace_bytes, st, (flags & GTB_STATE48) != 0);
    return run_vadv_n<float, float>(f, g, workspace, workspace_bytes, st);
}

extern "C" size_t gtb_vadv_workspace_bytes(int dtype, int prec, const int64_t *domain) {
    if (!domain || !dtype_size(dtype) || prec < GTB_PREC_NATIVE || prec > GTB_PREC_DF) return 0;
    for (int d = 0; d < 3; ++d)
        if (domain[d] < 0) return 0;
    return vadv_ws_bytes_for(dtype, dtype == GTB_F64 ? GTB_PREC_NATIVE : prec, domain);
}

extern "C" int gtb_hdiff_vadv(const gtb_field *in, const gtb_field *coeff, const gtb_field *wcon,
                              const gtb_field *utens, const gtb_field *utens_stage, const gtb_field *utens_stage_out,
                              double dtr_stage, double beta_v, int prec, unsigned flags, const int64_t *domain,
                              void *workspace, size_t workspace_bytes, void *stream) {
    const gtb_field *f[6] = {in, coeff, wcon, utens, utens_stage, utens_stage_out};
    static const char *names[6] = {"in", "coeff", "wcon", "utens", "utens_stage", "utens_stage_out"};
    for (int q = 0; q < 6; ++q)
        if (!f[q]) return fail(GTB_ERR_NULL, "gtb_hdiff_vadv: NULL field %s", names[q]);
    const int dt = in->dtype;
    if (!dtype_size(dt)) return fail(GTB_ERR_DTYPE, "gtb_hdiff_vadv: unknown dtype %d", dt);
    int rc;
    for (int q = 0; q < 6; ++q)
        if ((rc = check_field(names[q], f[q], dt))) return rc;
    if (flags & ~(GTB_WCON_LITERAL | GTB_SAVE_FACTORS))
        return fail(GTB_ERR_ARG, "gtb_hdiff_vadv: unknown flags 0x%x", flags);
    const bool save = flags & GTB_SAVE_FACTORS;
    if (prec < GTB_PREC_NATIVE || prec > GTB_PREC_DF) return fail(GTB_ERR_ARG, "gtb_hdiff_vadv: unknown prec %d", prec);
    if (dt == GTB_F64 && prec != GTB_PREC_NATIVE)
        return fail(GTB_ERR_ARG, "gtb_hdiff_vadv: FP64 storage computes in binary64 (prec must be GTB_PREC_NATIVE)");
    if (!(dtr_stage == dtr_stage) || !(beta_v == beta_v)) return fail(GTB_ERR_ARG, "gtb_hdiff_vadv: NaN scalar");
    const bool literal = flags & GTB_WCON_LITERAL;
    const Reach r_in{{2, 2, 0}, {2, 2, 0}}, r0{{0, 0, 0}, {0, 0, 0}}, rw{{0, 0, 0}, {literal ? 0 : 1, 0, 0}};
    const Reach *reach[6] = {&r_in, &r0, &rw, &r0, &r0, &r0};
    int64_t dom[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
    if (!domain)
        for (int q = 0; q < 6; ++q) shrink_domain(f[q], *reach[q], dom);
    if ((rc = resolve_domain(domain, dom))) return rc;
    for (int q = 0; q < 6; ++q)
        if ((rc = check_extent(names[q], f[q], *reach[q], dom))) return rc;
    for (int q = 0; q < 5; ++q) {
        if (q == 4 && same_view(utens_stage_out, utens_stage)) continue;  // in place
        if (overlaps(utens_stage_out, f[q]))
            return fail(GTB_ERR_ALIAS, "gtb_hdiff_vadv: utens_stage_out overlaps %s", names[q]);
    }
    if (dom[0] == 0 || dom[1] == 0 || dom[2] == 0) return ok();
    const size_t need = fused_ws_bytes_for(dt, prec, dom, save);
    if (!workspace || workspace_bytes < need)
        return fail(GTB_ERR_ARG, "gtb_hdiff_vadv: a workspace of %zu bytes is required (got %zu)", need,
                    workspace ? workspace_bytes : (size_t)0);
    if (reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
        return fail(GTB_ERR_LAYOUT, "gtb_hdiff_vadv: workspace must be 16-byte aligned");
    {
        const int64_t n = (int64_t)(workspace_bytes / dtype_size(dt));
        const gtb_field wsf{workspace, dt, 0, {n, 1, 1}, {1, n, n}, {0, 0, 0}};
        for (int q = 0; q < 6; ++q)
            if (overlaps(&wsf, f[q])) return fail(GTB_ERR_ALIAS, "gtb_hdiff_vadv: workspace overlaps %s", names[q]);
    }
    const VadvGeom g = make_vadv_geom(dom, literal, dtr_stage, beta_v);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dt == GTB_F64) return run_fused_n<double, double>(f, g, workspace, save, st);
    if (prec == GTB_PREC_F64) return run_chain32_n<double>(f, g, dom, workspace, save, st);
    if (prec == GTB_PREC_DF) return run_chain32_n<df>(f, g, dom, workspace, save, st);
    return run_chain32_n<float>(f, g, dom, workspace, save, st);
}

extern "C" int gtb_step(const gtb_field *in, const gtb_field *coeff, const gtb_field *hdiff_out,
                        const gtb_field *u_stage, const gtb_field *wcon, const gtb_field *u_pos,
                        const gtb_field *utens, const gtb_field *utens_stage, const gtb_field *utens_stage_out,
                        double dtr_stage, double beta_v, int prec, unsigned flags, const int64_t *domain,
                        void *workspace, size_t workspace_bytes, void *stream) {
    const gtb_field *f[9] = {in, coeff, hdiff_out, u_stage, wcon, u_pos, utens, utens_stage, utens_stage_out};
    static const char *names[9] = {"in", "coeff", "hdiff_out", "u_stage", "wcon", "u_pos", "utens", "utens_stage",
                                   "utens_stage_out"};
    for (int q = 0; q < 9; ++q)
        if (!f[q]) return fail(GTB_ERR_NULL, "gtb_step: NULL field %s", names[q]);
    const int dt = in->dtype;
    if (!dtype_size(dt)) return fail(GTB_ERR_DTYPE, "gtb_step: unknown dtype %d", dt);
    int rc;
    for (int q = 0; q < 9; ++q)
        if ((rc = check_field(names[q], f[q], dt))) return rc;
    if (flags & ~(GTB_WCON_LITERAL | GTB_STATE48)) return fail(GTB_ERR_ARG, "gtb_step: unknown flags 0x%x", flags);
    if (prec < GTB_PREC_NATIVE || prec > GTB_PREC_DF) return fail(GTB_ERR_ARG, "gtb_step: unknown prec %d", prec);
    if (dt == GTB_F64 && prec != GTB_PREC_NATIVE)
        return fail(GTB_ERR_ARG, "gtb_step: FP64 storage computes in binary64 (prec must be GTB_PREC_NATIVE)");
    if ((flags & GTB_STATE48) && (dt != GTB_F32 || prec != GTB_PREC_DF))
        return fail(GTB_ERR_ARG, "gtb_step: GTB_STATE48 applies to GTB_F32 storage with GTB_PREC_DF");
    if (!(dtr_stage == dtr_stage) || !(beta_v == beta_v)) return fail(GTB_ERR_ARG, "gtb_step: NaN scalar");
    const bool literal = flags & GTB_WCON_LITERAL;
    const Reach r_in{{2, 2, 0}, {2, 2, 0}}, r0{{0, 0, 0}, {0, 0, 0}}, rw{{0, 0, 0}, {literal ? 0 : 1, 0, 0}};
    const Reach *reach[9] = {&r_in, &r0, &r0, &r0, &rw, &r0, &r0, &r0, &r0};
    int64_t dom[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
    if (!domain)
        for (int q = 0; q < 9; ++q) shrink_domain(f[q], *reach[q], dom);
    if ((rc = resolve_domain(domain, dom))) return rc;
    for (int q = 0; q < 9; ++q)
        if ((rc = check_extent(names[q], f[q], *reach[q], dom))) return rc;
    // hdiff_out overlaps nothing; utens_stage_out overlaps nothing but possibly utens_stage itself
    for (int q = 0; q < 9; ++q)
        if (q != 2 && overlaps(hdiff_out, f[q]))
            return fail(GTB_ERR_ALIAS, "gtb_step: hdiff_out overlaps %s", names[q]);
    for (int q = 0; q < 8; ++q) {
        if (q == 7 && same_view(utens_stage_out, utens_stage)) continue;  // in place
        if (q != 2 && overlaps(utens_stage_out, f[q]))
            return fail(GTB_ERR_ALIAS, "gtb_step: utens_stage_out overlaps %s", names[q]);
    }
    if (dom[0] == 0 || dom[1] == 0 || dom[2] == 0) return ok();
    const size_t need = vadv_ws_bytes_for(dt, prec, dom);
    if (!workspace || workspace_bytes < need)
        return fail(GTB_ERR_ARG, "gtb_step: a workspace of %zu bytes is required (got %zu)", need,
                    workspace ? workspace_bytes : (size_t)0);
    if (reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
        return fail(GTB_ERR_LAYOUT, "gtb_step: workspace must be 16-byte aligned");
    {
        const int64_t n = (int64_t)(workspace_bytes / dtype_size(dt));
        const gtb_field wsf{workspace, dt, 0, {n, 1, 1}, {1, n, n}, {0, 0, 0}};
        for (int q = 0; q < 9; ++q)
            if (overlaps(&wsf, f[q])) return fail(GTB_ERR_ALIAS, "gtb_step: workspace overlaps %s", names[q]);
    }
    const VadvGeom g = make_vadv_geom(dom, literal, dtr_stage, beta_v);
    const gtb_field *fh[3] = {in, coeff, hdiff_out};
    const gtb_field *fv[6] = {u_stage, wcon, u_pos, utens, utens_stage, utens_stage_out};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dt == GTB_F64) return run_pair_n<double, double>(fh, fv, g, workspace, st);
    // binary32 storage: hdiff is bound by HBM and the column solve by the FP32 pipe;
    // on B300 the two separate kernels back to back are faster than sharing SMs
    if ((rc = run_hdiff<float>(in, coeff, hdiff_out, dom, st))) return rc;
    if (prec == GTB_PREC_F64) return run_vadv_n<float, double>(fv, g, workspace, workspace_bytes, st);
    if (prec == GTB_PREC_DF)
        return run_vadv_n<float, df>(fv, g, workspace, workspace_bytes, st, (flags & GTB_STATE48) != 0);
    return run_vadv_n<float, float>(fv, g, workspace, workspace_bytes, st);
}

extern "C" size_t gtb_hdiff_vadv_workspace_bytes(int dtype, int prec, unsigned flags, const int64_t *domain) {
    if (!domain || !dtype_size(dtype) || prec < GTB_PREC_NATIVE || prec > GTB_PREC_DF) return 0;
    for (int d = 0; d < 3; ++d)
        if (domain[d] < 0) return 0;
    return fused_ws_bytes_for(dtype, dtype == GTB_F64 ? GTB_PREC_NATIVE : prec, domain, flags & GTB_SAVE_FACTORS);
}

extern "C" int gtb_device_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(GTB_ERR_LAUNCH, "gtb_device_status: %s", cudaGetErrorString(e));
    int flag = 0;
    e = cudaMemcpyFromSymbol(&flag, g_device_error, sizeof(int));
    if (e != cudaSuccess) return fail(GTB_ERR_LAUNCH, "gtb_device_status: %s", cudaGetErrorString(e));
    if (flag) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int));
        if (flag == kDeviceErrBounds)
            return fail(GTB_ERR_DEVICE, "a kernel's address run fell outside a field's storage");
        return fail(GTB_ERR_DEVICE, "a kernel's bounded wait expired");
    }
    return ok();
}

extern "C" int gtb_selftest_wait(long long limit_ns, int arrive, void *stream) {
    if (limit_ns <= 0 || limit_ns > (long long)kWaitLimitNs)
        return fail(GTB_ERR_ARG, "gtb_selftest_wait: limit %lld ns outside (0, %llu]", limit_ns, kWaitLimitNs);
    if (arrive != 0 && arrive != 1) return fail(GTB_ERR_ARG, "gtb_selftest_wait: arrive must be 0 or 1");
    selftest_wait_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((unsigned long long)limit_ns, arrive);
    return launch_status("gtb_selftest_wait launch");
}

extern "C" int gtb_probe_fp64_fma(int blocks, int iters, void *sink, void *stream) {
    if (blocks < 1 || blocks > (1 << 20) || iters < 1 || iters > (1 << 24))
        return fail(GTB_ERR_ARG, "gtb_probe_fp64_fma: blocks %d or iters %d out of range", blocks, iters);
    if (!sink) return fail(GTB_ERR_NULL, "gtb_probe_fp64_fma: NULL sink");
    if (reinterpret_cast<uintptr_t>(sink) % 8 != 0) return fail(GTB_ERR_LAYOUT, "gtb_probe_fp64_fma: sink not 8-byte aligned");
    fp64_fma_probe_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.999999, 1e-7,
                                                                                static_cast<double *>(sink));
    return launch_status("gtb_probe_fp64_fma launch");
}

extern "C" const char *gtb_last_error(void) { return t_err; }

#ifdef GTB_CHECKED
extern "C" const char *gtb_version(void) { return "gtb 0.2 sm_103a checked"; }
#else
extern "C" const char *gtb_version(void) { return "gtb 0.2 sm_103a"; }
#endif

// ====================================================================== allocation-free vadv
// gtb_vadv_noalloc: gtb_vadv with its workspace in a fixed device array of this
// library instead of caller memory (declared in include/gtb.h; the paper has no
// counterpart).  The array is a file-scope __device__ variable, so it exists
// on every GPU that loads the library, from load until exit, and no call ever
// allocates.  Host code cannot use the array's name as a device address: every
// call looks the address up with cudaGetSymbolAddress on the current device.
// The lookup allocates nothing and is not cached, so a context torn down and
// re-created (cudaDeviceReset by this or another library), in which the array
// may sit at another address, never receives a stale pointer.
namespace gtb {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_vadv_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array in the current device's context.
static int noalloc_scratch(void **ptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_vadv_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(GTB_ERR_LAUNCH, "gtb_vadv_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                    cudaGetErrorString(e));
    *ptr = p;
    return GTB_OK;
}

}  // namespace gtb

extern "C" int gtb_vadv_noalloc(const gtb_field *u_stage, const gtb_field *wcon, const gtb_field *u_pos,
                                const gtb_field *utens, const gtb_field *utens_stage,
                                const gtb_field *utens_stage_out, double dtr_stage, double beta_v, int prec,
                                unsigned flags, const int64_t *domain, void *stream) {
    const gtb_field *f[6] = {u_stage, wcon, u_pos, utens, utens_stage, utens_stage_out};
    for (int q = 0; q < 6; ++q)
        if (!f[q]) return fail(GTB_ERR_NULL, "gtb_vadv_noalloc: NULL field");
    // the domain the call will use: given, or deduced as gtb_vadv deduces it
    int64_t dom[3];
    if (domain) {
        for (int d = 0; d < 3; ++d) dom[d] = domain[d];
    } else {
        const bool literal = flags & GTB_WCON_LITERAL;
        for (int d = 0; d < 3; ++d) {
            dom[d] = INT64_MAX;
            for (int q = 0; q < 6; ++q)
                dom[d] = std::min(dom[d], f[q]->shape[d] - f[q]->origin[d] - ((q == 1 && d == 0 && !literal) ? 1 : 0));
            dom[d] = std::max<int64_t>(dom[d], 0);
        }
    }
    const size_t need = gtb_vadv_workspace_bytes(u_stage->dtype, prec, dom);
    if (need > kNoAllocScratchBytes)
        return fail(GTB_ERR_UNSUPPORTED,
                    "gtb_vadv_noalloc: domain %lldx%lldx%lld needs %zu bytes of scratch, above the fixed %zu-byte "
                    "array; use gtb_vadv with a caller workspace",
                    (long long)dom[0], (long long)dom[1], (long long)dom[2], need, kNoAllocScratchBytes);
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    // the workspace contents are never read before being written: nothing to clear
    return gtb_vadv(u_stage, wcon, u_pos, utens, utens_stage, utens_stage_out, dtr_stage, beta_v, prec, flags,
                    dom, scratch, kNoAllocScratchBytes, stream);
}

// ====================================================================== adjoints and halos
extern "C" int gtb_hdiff_adj(const gtb_field *in, const gtb_field *coeff, const gtb_field *out_bar,
                             const gtb_field *in_bar, const gtb_field *coeff_bar, unsigned flags,
                             const int64_t *domain, void *stream) {
    if (!in || !coeff || !out_bar || !in_bar) return fail(GTB_ERR_NULL, "gtb_hdiff_adj: NULL field");
    const int dt = in->dtype;
    if (!dtype_size(dt)) return fail(GTB_ERR_DTYPE, "gtb_hdiff_adj: unknown dtype %d", dt);
    int rc;
    if ((rc = check_field("in", in, dt)) || (rc = check_field("coeff", coeff, dt)) ||
        (rc = check_field("out_bar", out_bar, dt)) || (rc = check_field("in_bar", in_bar, dt)) ||
        (coeff_bar && (rc = check_field("coeff_bar", coeff_bar, dt))))
        return rc;
    if (flags & ~GTB_ADJ_ACCUMULATE) return fail(GTB_ERR_ARG, "gtb_hdiff_adj: unknown flags 0x%x", flags);
    const Reach r2{{2, 2, 0}, {2, 2, 0}}, r0{{0, 0, 0}, {0, 0, 0}};
    int64_t dom[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
    if (!domain) {
        shrink_domain(in, r2, dom);
        shrink_domain(coeff, r0, dom);
        shrink_domain(out_bar, r0, dom);
        shrink_domain(in_bar, r2, dom);
        if (coeff_bar) shrink_domain(coeff_bar, r0, dom);
    }
    if ((rc = resolve_domain(domain, dom))) return rc;
    if ((rc = check_extent("in", in, r2, dom)) || (rc = check_extent("coeff", coeff, r0, dom)) ||
        (rc = check_extent("out_bar", out_bar, r0, dom)) || (rc = check_extent("in_bar", in_bar, r2, dom)) ||
        (coeff_bar && (rc = check_extent("coeff_bar", coeff_bar, r0, dom))))
        return rc;
    const gtb_field *ins[3] = {in, coeff, out_bar};
    static const char *inames[3] = {"in", "coeff", "out_bar"};
    for (int q = 0; q < 3; ++q) {
        if (overlaps(in_bar, ins[q])) return fail(GTB_ERR_ALIAS, "gtb_hdiff_adj: in_bar overlaps %s", inames[q]);
        if (coeff_bar && overlaps(coeff_bar, ins[q]))
            return fail(GTB_ERR_ALIAS, "gtb_hdiff_adj: coeff_bar overlaps %s", inames[q]);
    }
    if (coeff_bar && overlaps(coeff_bar, in_bar)) return fail(GTB_ERR_ALIAS, "gtb_hdiff_adj: coeff_bar overlaps in_bar");
    if (dom[0] == 0 || dom[1] == 0 || dom[2] == 0) return ok();
    if (dom[2] > 65535) return fail(GTB_ERR_UNSUPPORTED, "gtb_hdiff_adj: K above 65535");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int acc = (flags & GTB_ADJ_ACCUMULATE) ? 1 : 0;
    return dt == GTB_F64 ? run_hdiff_adj<double>(in, coeff, out_bar, in_bar, coeff_bar, acc, dom, st)
                         : run_hdiff_adj<float>(in, coeff, out_bar, in_bar, coeff_bar, acc, dom, st);
}

extern "C" size_t gtb_vadv_adj_workspace_bytes(int dtype, int prec, const int64_t *domain) {
    if (!domain || !dtype_size(dtype) || prec < GTB_PREC_NATIVE || prec > GTB_PREC_DF) return 0;
    for (int d = 0; d < 3; ++d)
        if (domain[d] < 0) return 0;
    return vadv_adj_ws_bytes_for(dtype, dtype == GTB_F64 ? GTB_PREC_NATIVE : prec, domain);
}

extern "C" int gtb_vadv_adj(const gtb_field *wcon, const gtb_field *y_bar, const gtb_field *u_stage_bar,
                            const gtb_field *u_pos_bar, const gtb_field *utens_bar, const gtb_field *utens_stage_bar,
                            double dtr_stage, double beta_v, int prec, unsigned flags, const int64_t *domain,
                            void *workspace, size_t workspace_bytes, void *stream) {
    const gtb_field *f[6] = {wcon, y_bar, u_stage_bar, u_pos_bar, utens_bar, utens_stage_bar};
    static const char *names[6] = {"wcon", "y_bar", "u_stage_bar", "u_pos_bar", "utens_bar", "utens_stage_bar"};
    if (!wcon || !y_bar) return fail(GTB_ERR_NULL, "gtb_vadv_adj: NULL wcon or y_bar");
    const int dt = y_bar->dtype;
    if (!dtype_size(dt)) return fail(GTB_ERR_DTYPE, "gtb_vadv_adj: unknown dtype %d", dt);
    int rc;
    for (int q = 0; q < 6; ++q)
        if (f[q] && (rc = check_field(names[q], f[q], dt))) return rc;
    if (flags & ~(GTB_WCON_LITERAL | GTB_ADJ_ACCUMULATE | GTB_ADJ_FACTORS))
        return fail(GTB_ERR_ARG, "gtb_vadv_adj: unknown flags 0x%x", flags);
    const bool factors = flags & GTB_ADJ_FACTORS;
    if (prec < GTB_PREC_NATIVE || prec > GTB_PREC_DF) return fail(GTB_ERR_ARG, "gtb_vadv_adj: unknown prec %d", prec);
    if (dt == GTB_F64 && prec != GTB_PREC_NATIVE)
        return fail(GTB_ERR_ARG, "gtb_vadv_adj: FP64 storage computes in binary64 (prec must be GTB_PREC_NATIVE)");
    if (!(dtr_stage == dtr_stage) || !(beta_v == beta_v)) return fail(GTB_ERR_ARG, "gtb_vadv_adj: NaN scalar");
    const bool literal = flags & GTB_WCON_LITERAL;
    const Reach r0{{0, 0, 0}, {0, 0, 0}}, rw{{0, 0, 0}, {literal ? 0 : 1, 0, 0}};
    int64_t dom[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
    if (!domain)
        for (int q = 0; q < 6; ++q)
            if (f[q]) shrink_domain(f[q], q == 0 ? rw : r0, dom);
    if ((rc = resolve_domain(domain, dom))) return rc;
    for (int q = 0; q < 6; ++q)
        if (f[q] && (rc = check_extent(names[q], f[q], q == 0 ? rw : r0, dom))) return rc;
    const bool merge = u_stage_bar && u_pos_bar && same_view(u_stage_bar, u_pos_bar);
    for (int q = 2; q < 6; ++q) {
        if (!f[q]) continue;
        for (int r = 0; r < 6; ++r) {
            if (r == q || !f[r]) continue;
            if (merge && ((q == 2 && r == 3) || (q == 3 && r == 2))) continue;
            if (overlaps(f[q], f[r])) return fail(GTB_ERR_ALIAS, "gtb_vadv_adj: %s overlaps %s", names[q], names[r]);
        }
    }
    if (dom[2] > kVadvMaxK && !(workspace && workspace_bytes >= vadv_adj_ws_bytes_for(dt, prec, dom)))
        return fail(GTB_ERR_UNSUPPORTED, "gtb_vadv_adj: K = %lld exceeds the limit %d without a workspace",
                    (long long)dom[2], kVadvMaxK);
    if (workspace && reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
        return fail(GTB_ERR_LAYOUT, "gtb_vadv_adj: workspace must be 16-byte aligned");
    if (dom[0] == 0 || dom[1] == 0 || dom[2] == 0) return ok();
    if (factors && (!workspace || workspace_bytes < vadv_adj_ws_bytes_for(dt, prec, dom)))
        return fail(GTB_ERR_ARG, "gtb_vadv_adj: GTB_ADJ_FACTORS needs the forward's factors: a workspace of %zu bytes",
                    vadv_adj_ws_bytes_for(dt, prec, dom));
    if (workspace) {
        const int64_t n = (int64_t)(workspace_bytes / dtype_size(dt));
        const gtb_field wsf{workspace, dt, 0, {n, 1, 1}, {1, n, n}, {0, 0, 0}};
        for (int q = 0; q < 6; ++q)
            if (f[q] && overlaps(&wsf, f[q])) return fail(GTB_ERR_ALIAS, "gtb_vadv_adj: workspace overlaps %s", names[q]);
    }
    const VadvGeom g = make_vadv_geom(dom, literal, dtr_stage, beta_v);
    const int acc = (flags & GTB_ADJ_ACCUMULATE) ? 1 : 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dt == GTB_F64) return run_vadv_adj_n<double, double>(f, g, acc, merge, workspace, workspace_bytes, factors, st);
    if (prec == GTB_PREC_F64)
        return run_vadv_adj_n<float, double>(f, g, acc, merge, workspace, workspace_bytes, factors, st);
    if (prec == GTB_PREC_DF) return run_vadv_adj_n<float, df>(f, g, acc, merge, workspace, workspace_bytes, factors, st);
    return run_vadv_adj_n<float, float>(f, g, acc, merge, workspace, workspace_bytes, factors, st);
}

static int halo_common(const char *fn, const gtb_field *f, int hi, int hj, const int64_t *domain, int64_t dom[3]) {
    if (!f) return fail(GTB_ERR_NULL, "%s: NULL field", fn);
    int rc;
    if (!dtype_size(f->dtype)) return fail(GTB_ERR_DTYPE, "%s: unknown dtype %d", fn, f->dtype);
    if ((rc = check_field("field", f, f->dtype))) return rc;
    if (hi < 0 || hj < 0) return fail(GTB_ERR_ARG, "%s: negative halo width", fn);
    const Reach r{{hi, hj, 0}, {hi, hj, 0}};
    for (int d = 0; d < 3; ++d) dom[d] = INT64_MAX;
    if (!domain) shrink_domain(f, r, dom);
    if ((rc = resolve_domain(domain, dom))) return rc;
    if ((rc = check_extent("field", f, r, dom))) return rc;
    if ((dom[0] > 0 && hi > dom[0]) || (dom[1] > 0 && hj > dom[1]))
        return fail(GTB_ERR_UNSUPPORTED, "%s: halo wider than the domain", fn);
    return GTB_OK;
}

extern "C" int gtb_halo_periodic(const gtb_field *f, int hi, int hj, const int64_t *domain, void *stream) {
    int64_t dom[3];
    int rc = halo_common("gtb_halo_periodic", f, hi, hj, domain, dom);
    if (rc) return rc;
    if (dom[0] == 0 || dom[1] == 0 || dom[2] == 0) return ok();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return f->dtype == GTB_F64 ? run_halo<double>(f, hi, hj, dom, false, st) : run_halo<float>(f, hi, hj, dom, false, st);
}

extern "C" int gtb_halo_periodic_adj(const gtb_field *f, int hi, int hj, const int64_t *domain, void *stream) {
    int64_t dom[3];
    int rc = halo_common("gtb_halo_periodic_adj", f, hi, hj, domain, dom);
    if (rc) return rc;
    if (dom[0] == 0 || dom[1] == 0 || dom[2] == 0) return ok();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return f->dtype == GTB_F64 ? run_halo<double>(f, hi, hj, dom, true, st) : run_halo<float>(f, hi, hj, dom, true, st);
}

// ====================================================================== batched ensembles
struct gtb_plan {
    int device = 0, dtype = 0, prec = 0, n = 0;
    gtb_batch_config cfg{};
    int h_items = 0, v_items = 0, h_grid = 0, v_grid = 0;
    void *d_maps = nullptr, *d_hmem = nullptr, *d_vmem = nullptr, *d_scratch = nullptr;
    int *d_counters = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double points = 0;
};

namespace gtb {

static void plan_free(gtb_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_maps);
    cudaFree(p->d_hmem);
    cudaFree(p->d_vmem);
    cudaFree(p->d_scratch);
    cudaFree(p->d_counters);
    delete p;
}

// hdiff tile variants of the batched form: variant 0 is the single-domain
// configuration (so batched and single results agree bit for bit), variant 1
// the other warp/row split.  CTMA: binary32 members with coeff staged by TMA (the
// single-domain binary32 configuration); otherwise coeff is read from global memory
// (the binary64 configuration, and binary32 plans whose coeff layouts rule TMA out).
template <typename T, int V, bool CTMA = false>
struct BatchHCfg {
    using B = typename std::conditional<CTMA, HdiffCoeffTmaCfg<T>, HdiffCfg<T>>::type;
    static constexpr int CPL = B::CPL, STAGES = 2;
    static constexpr int W = V == 0 ? B::W : (B::W == 4 ? 8 : 4);
    static constexpr int R = V == 0 ? B::R : (B::W == 4 ? B::R / 2 : B::R * 2);
};

template <typename T, int V, bool CTMA>
static int batch_hdiff_launch_info(int ctas_per_sm, int *slots, void (**kern)(const CUtensorMap *, const BatchHdiffMember<T> *, int, int, int *), int *smem) {
    using C = BatchHCfg<T, V, CTMA>;
    constexpr bool FIXED = sizeof(T) == 8;
    constexpr int W = C::W;
    auto k = hdiff_batch_kernel<T, C::CPL, W, C::R, C::STAGES, FIXED, CTMA>;
    *smem = hdiff_rs_smem_bytes<T, C::CPL, W, C::R, C::STAGES, CTMA>();
    if (prepare_kernel(k, *smem) != cudaSuccess) return launch_status("batch: hdiff shared-memory attribute");
    int rb = resident_blocks(k, 32 * W, *smem);
    if (ctas_per_sm > 0) rb = std::min(rb, ctas_per_sm);
    *slots = rb * sm_count();
    *kern = k;
    return GTB_OK;
}

// The column-solve stage of a plan in storage type TV and arithmetic NV: members longest
// column first (so the queue ends with short items), their device table, per-CTA scratch,
// and the launch arguments (the stage is launched by cudaLaunchKernel inside the capture).
struct VadvStageLaunch {
    const void *func;
    void *vmem, *scratch;
    size_t slice;
    int n, items, k_max;
};

template <typename TV, typename NV, int BJ>
static int plan_vadv_stage(const gtb_member *mem, int n, bool literal, double dtr, double beta, int k_max, gtb_plan *P,
                           VadvStageLaunch *L) {
    std::vector<int> vorder(n);
    for (int q = 0; q < n; ++q) vorder[q] = q;
    std::stable_sort(vorder.begin(), vorder.end(), [&](int a, int b) { return mem[a].domain[2] > mem[b].domain[2]; });
    std::vector<BatchVadvMember<TV>> vm(n);
    constexpr bool PAIRS = is_pair<TV>();
    auto view = [](const gtb_field *f) {
        if constexpr (PAIRS) return pair_view<const fpair>(f);
        else return view_of<const TV>(f);
    };
    int vitems = 0;
    for (int r = 0; r < n; ++r) {
        const gtb_member &M = mem[vorder[r]];
        VadvGeom g = make_vadv_geom(M.domain, literal, dtr, beta);
        if (PAIRS) g.I /= 2;  // pairs of columns
        const int bx = (g.I + 31) / 32, by = (g.J + BJ - 1) / BJ;
        const View<const TV> h = view(&M.h);
        View<TV> out;
        if constexpr (PAIRS) out = pair_view<fpair>(&M.out);
        else out = view_of<TV>(&M.out);
        vm[r] = BatchVadvMember<TV>{h, view(&M.wcon), h, view(&M.utens), view(&M.utens_stage), out, g, bx, vitems};
        vitems += bx * by;
    }
    auto k = vadv_batch_kernel<TV, NV, BJ>;
    int rb = resident_blocks(k, 32 * BJ, 0);
    if (P->cfg.ctas_per_sm > 0) rb = std::min(rb, P->cfg.ctas_per_sm);
    P->v_items = vitems;
    P->v_grid = std::max(1, std::min(vitems, rb * sm_count()));
    const size_t slice = (size_t)vadv_state_arrays<TV, NV>() * k_max * 32 * BJ;
    cudaError_t e;
    if ((e = cudaMalloc(&P->d_vmem, sizeof(BatchVadvMember<TV>) * n)) ||
        (e = cudaMalloc(&P->d_scratch, sizeof(NV) * slice * P->v_grid)) ||
        (e = cudaMemcpy(P->d_vmem, vm.data(), sizeof(BatchVadvMember<TV>) * n, cudaMemcpyHostToDevice)))
        return fail(GTB_ERR_LAUNCH, "gtb_batch_plan: column-solve tables: %s", cudaGetErrorString(e));
    *L = VadvStageLaunch{reinterpret_cast<const void *>(k), P->d_vmem, P->d_scratch, slice, n, vitems, k_max};
    return GTB_OK;
}

// Members whose binary32 fields all fit column pairs (even I, pair-aligned fields).
static bool batch_pairs_fit(const gtb_member *mem, int n) {
    for (int q = 0; q < n; ++q) {
        const gtb_member &M = mem[q];
        if (M.domain[0] % 2 || !pairs_fit(&M.h) || !pairs_fit(&M.wcon) || !pairs_fit(&M.utens) ||
            !pairs_fit(&M.utens_stage) || !pairs_fit(&M.out))
            return false;
    }
    return true;
}

template <typename T, typename N, int V, int BJ, bool CTMA>
static int build_plan(const gtb_member *mem, int n, double dtr, double beta, unsigned flags, gtb_plan *P) {
    using C = BatchHCfg<T, V, CTMA>;
    constexpr int W = C::W;
    using Tile = RsTile<T, C::CPL, W, C::R, CTMA>;
    const size_t es = sizeof(T);
    constexpr int kAlign = 16 / (int)sizeof(T);
    constexpr int MPM = CTMA ? 2 : 1;  // tensor maps per member: in (and coeff)
    std::vector<CUtensorMap> maps(MPM * n);
    std::vector<BatchHdiffMember<T>> hm(n);
    int k_max = 1;
    double pts = 0;
    // hdiff members in the given order
    int hitems = 0;
    for (int q = 0; q < n; ++q) {
        const gtb_member &M = mem[q];
        const int64_t *d = M.domain;
        HdiffGeom g{};
        g.I = (int)d[0], g.J = (int)d[1], g.K = (int)d[2];
        g.tiles_i = (g.I + Tile::TI - 1) / Tile::TI;
        g.tiles_j = (g.J + Tile::TJ - 1) / Tile::TJ;
        g.n_tiles = g.tiles_i * g.tiles_j;
        g.kc = P->cfg.hdiff_levels > 0 ? std::min(P->cfg.hdiff_levels, g.K) : g.K;
        const uintptr_t base = reinterpret_cast<uintptr_t>(M.in.ptr), abase = base & ~uintptr_t(15);
        const int shift = (int)((base - abase) / es);
        const int xraw = (int)M.in.origin[0] - 2 + shift;
        g.xs = xraw % kAlign;
        g.X0 = xraw - g.xs;
        g.Y0 = (int)M.in.origin[1] - 2;
        g.Z0 = (int)M.in.origin[2];
        cuuint64_t gdim[3] = {(cuuint64_t)(M.in.shape[0] + shift), (cuuint64_t)M.in.shape[1], (cuuint64_t)M.in.shape[2]};
        cuuint64_t gstride[2] = {(cuuint64_t)(M.in.strides[1] * es), (cuuint64_t)(M.in.strides[2] * es)};
        cuuint32_t box[3] = {(cuuint32_t)Tile::BX, (cuuint32_t)Tile::BY, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        memset(&maps[MPM * q], 0, sizeof(CUtensorMap));
        CUresult r = encode_fn()(&maps[MPM * q], sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                 3, reinterpret_cast<void *>(abase), gdim, gstride, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(GTB_ERR_LAYOUT, "gtb_batch_plan: member %d: tensor-map encoding failed (%d)", q, (int)r);
        if (CTMA && !encode_coeff_map<T>(&M.coeff, Tile::TI, Tile::TJ, g, maps[MPM * q + 1]))
            return fail(GTB_ERR_LAYOUT, "gtb_batch_plan: member %d: coeff tensor map", q);
        const View<T> cf = view_of<T>(&M.coeff), out = view_of<T>(&M.h);
        auto aligned = [&](const View<T> &v) {
            return reinterpret_cast<uintptr_t>(v.p) % 16 == 0 && (v.sj * es) % 16 == 0 && (v.sk * es) % 16 == 0;
        };
        hm[q] = BatchHdiffMember<T>{view_of<T>(&M.in), cf, out, g, (aligned(cf) && aligned(out)) ? 1 : 0, hitems};
        hitems += g.n_tiles * ((g.K + g.kc - 1) / g.kc);
        k_max = std::max(k_max, g.K);
        pts += (double)g.I * g.J * g.K;
    }
    const bool literal = flags & GTB_WCON_LITERAL;
    void (*hk)(const CUtensorMap *, const BatchHdiffMember<T> *, int, int, int *);
    int hslots, hsmem, rc;
    if ((rc = batch_hdiff_launch_info<T, V, CTMA>(P->cfg.ctas_per_sm, &hslots, &hk, &hsmem))) return rc;
    P->h_items = hitems;
    P->h_grid = std::max(1, std::min(hitems, hslots));
    P->points = pts;
    VadvStageLaunch vl{};
    if constexpr (std::is_same<T, float>::value && std::is_same<N, df>::value) {
        rc = batch_pairs_fit(mem, n) ? plan_vadv_stage<fpair, dfpair, BJ>(mem, n, literal, dtr, beta, k_max, P, &vl)
                                     : plan_vadv_stage<T, N, BJ>(mem, n, literal, dtr, beta, k_max, P, &vl);
    } else {
        rc = plan_vadv_stage<T, N, BJ>(mem, n, literal, dtr, beta, k_max, P, &vl);
    }
    if (rc) return rc;
    cudaError_t e;
    if ((e = cudaMalloc(&P->d_maps, sizeof(CUtensorMap) * MPM * n)) || (e = cudaMalloc(&P->d_hmem, sizeof(BatchHdiffMember<T>) * n)) ||
        (e = cudaMalloc(&P->d_counters, 2 * sizeof(int))))
        return fail(GTB_ERR_LAUNCH, "gtb_batch_plan: device tables: %s", cudaGetErrorString(e));
    if ((e = cudaMemcpy(P->d_maps, maps.data(), sizeof(CUtensorMap) * MPM * n, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(P->d_hmem, hm.data(), sizeof(BatchHdiffMember<T>) * n, cudaMemcpyHostToDevice)))
        return fail(GTB_ERR_LAUNCH, "gtb_batch_plan: table upload: %s", cudaGetErrorString(e));
    // capture: reset the two queues, hdiff stage, vadv stage
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)))
        return fail(GTB_ERR_LAUNCH, "gtb_batch_plan: stream: %s", cudaGetErrorString(e));
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(P->d_counters, 0, 2 * sizeof(int), cs);
        hk<<<P->h_grid, 32 * W, hsmem, cs>>>(static_cast<const CUtensorMap *>(P->d_maps),
                                             static_cast<const BatchHdiffMember<T> *>(P->d_hmem), n, hitems, P->d_counters);
        int *vcounter = P->d_counters + 1;
        void *args[] = {&vl.vmem, &vl.n, &vl.items, &vcounter, &vl.scratch, &vl.slice, &vl.k_max};
        cudaLaunchKernel(vl.func, dim3(P->v_grid), dim3(32, BJ), args, 0, cs);
        e = cudaStreamEndCapture(cs, &P->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return fail(GTB_ERR_LAUNCH, "gtb_batch_plan: graph capture: %s", cudaGetErrorString(e));
    return GTB_OK;
}

template <typename T, typename N, int V, bool CTMA>
static int build_plan_bj(const gtb_member *mem, int n, double dtr, double beta, unsigned flags, gtb_plan *P) {
    switch (P->cfg.vadv_warps) {
    case 1: return build_plan<T, N, V, 1, CTMA>(mem, n, dtr, beta, flags, P);
    case 4: return build_plan<T, N, V, 4, CTMA>(mem, n, dtr, beta, flags, P);
    default: return build_plan<T, N, V, 2, CTMA>(mem, n, dtr, beta, flags, P);
    }
}

// Whether every member's coeff can be staged by TMA: its domain's first point on a
// 16-byte boundary and 16-byte pitches.
static bool batch_coeff_tma_ok(const gtb_member *mem, int n, size_t es) {
    for (int q = 0; q < n; ++q) {
        const gtb_field &c = mem[q].coeff;
        const uintptr_t first = reinterpret_cast<uintptr_t>(c.ptr) + (uintptr_t)c.origin[0] * es;
        if (first % 16 || (c.strides[1] * es) % 16 || (c.strides[2] * es) % 16) return false;
    }
    return true;
}

template <typename T, typename N>
static int build_plan_w(const gtb_member *mem, int n, double dtr, double beta, unsigned flags, gtb_plan *P) {
    if constexpr (HdiffCoeffTmaCfg<T>::kUse) {
        if (batch_coeff_tma_ok(mem, n, sizeof(T)))
            return P->cfg.hdiff_tile == 1 ? build_plan_bj<T, N, 1, true>(mem, n, dtr, beta, flags, P)
                                          : build_plan_bj<T, N, 0, true>(mem, n, dtr, beta, flags, P);
    }
    return P->cfg.hdiff_tile == 1 ? build_plan_bj<T, N, 1, false>(mem, n, dtr, beta, flags, P)
                                  : build_plan_bj<T, N, 0, false>(mem, n, dtr, beta, flags, P);
}

}  // namespace gtb

extern "C" int gtb_batch_plan(const gtb_member *members, int n, double dtr_stage, double beta_v, int prec,
                              unsigned flags, const gtb_batch_config *config, gtb_plan **plan) {
    if (!plan) return fail(GTB_ERR_NULL, "gtb_batch_plan: NULL plan");
    *plan = nullptr;
    if (!members || n <= 0) return fail(GTB_ERR_ARG, "gtb_batch_plan: no members");
    if (flags & ~GTB_WCON_LITERAL) return fail(GTB_ERR_ARG, "gtb_batch_plan: unknown flags 0x%x", flags);
    if (encode_fn() == nullptr) return fail(GTB_ERR_LAUNCH, "gtb_batch_plan: cuTensorMapEncodeTiled unavailable");
    const int dt = members[0].in.dtype;
    if (!dtype_size(dt)) return fail(GTB_ERR_DTYPE, "gtb_batch_plan: unknown dtype %d", dt);
    if (prec < GTB_PREC_NATIVE || prec > GTB_PREC_DF || (dt == GTB_F64 && prec != GTB_PREC_NATIVE))
        return fail(GTB_ERR_ARG, "gtb_batch_plan: bad prec %d for this dtype", prec);
    if (!(dtr_stage == dtr_stage) || !(beta_v == beta_v)) return fail(GTB_ERR_ARG, "gtb_batch_plan: NaN scalar");
    const bool literal = flags & GTB_WCON_LITERAL;
    const Reach r2{{2, 2, 0}, {2, 2, 0}}, r0{{0, 0, 0}, {0, 0, 0}}, rw{{0, 0, 0}, {literal ? 0 : 1, 0, 0}};
    int rc;
    for (int q = 0; q < n; ++q) {
        const gtb_member &M = members[q];
        const gtb_field *f[7] = {&M.in, &M.coeff, &M.h, &M.wcon, &M.utens, &M.utens_stage, &M.out};
        static const char *nm[7] = {"in", "coeff", "h", "wcon", "utens", "utens_stage", "out"};
        const Reach *rr[7] = {&r2, &r0, &r0, &rw, &r0, &r0, &r0};
        for (int d = 0; d < 3; ++d)
            if (M.domain[d] <= 0) return fail(GTB_ERR_EXTENT, "gtb_batch_plan: member %d: empty domain", q);
        if (M.domain[2] > kVadvMaxK) return fail(GTB_ERR_UNSUPPORTED, "gtb_batch_plan: member %d: K above %d", q, kVadvMaxK);
        for (int a = 0; a < 7; ++a) {
            if ((rc = check_field(nm[a], f[a], dt)) || (rc = check_extent(nm[a], f[a], *rr[a], M.domain))) {
                char msg[512];
                snprintf(msg, sizeof msg, "gtb_batch_plan: member %d: %s", q, gtb_last_error());
                return fail(rc, "%s", msg);
            }
        }
        const size_t es = dtype_size(dt);
        if ((M.in.strides[1] * es) % 16 || (M.in.strides[2] * es) % 16)
            return fail(GTB_ERR_LAYOUT, "gtb_batch_plan: member %d: in needs 16-byte pitches (TMA)", q);
        // outputs: h and out may not overlap any field of any member (out == utens_stage of its own member allowed)
        for (int b = 0; b < n; ++b) {
            const gtb_member &B = members[b];
            const gtb_field *g[7] = {&B.in, &B.coeff, &B.h, &B.wcon, &B.utens, &B.utens_stage, &B.out};
            for (int a = 0; a < 7; ++a) {
                if (b == q && (a == 2)) continue;  // h itself
                if (overlaps(&M.h, g[a])) return fail(GTB_ERR_ALIAS, "gtb_batch_plan: member %d: h overlaps a field of member %d", q, b);
            }
            for (int a = 0; a < 7; ++a) {
                if (b == q && (a == 6 || (a == 5 && same_view(&M.out, &M.utens_stage)))) continue;
                if (overlaps(&M.out, g[a])) return fail(GTB_ERR_ALIAS, "gtb_batch_plan: member %d: out overlaps a field of member %d", q, b);
            }
        }
    }
    gtb_plan *P = new gtb_plan();
    P->n = n, P->dtype = dt, P->prec = prec;
    cudaGetDevice(&P->device);
    if (config) P->cfg = *config;
    if (P->cfg.vadv_warps != 1 && P->cfg.vadv_warps != 2 && P->cfg.vadv_warps != 4) P->cfg.vadv_warps = 2;
    if (P->cfg.hdiff_tile != 1) P->cfg.hdiff_tile = 0;
    if (dt == GTB_F64) rc = build_plan_w<double, double>(members, n, dtr_stage, beta_v, flags, P);
    else if (prec == GTB_PREC_F64) rc = build_plan_w<float, double>(members, n, dtr_stage, beta_v, flags, P);
    else if (prec == GTB_PREC_DF) rc = build_plan_w<float, df>(members, n, dtr_stage, beta_v, flags, P);
    else rc = build_plan_w<float, float>(members, n, dtr_stage, beta_v, flags, P);
    if (rc) {
        plan_free(P);
        return rc;
    }
    *plan = P;
    return ok();
}

extern "C" int gtb_batch_run(const gtb_plan *plan, void *stream) {
    if (!plan || !plan->exec) return fail(GTB_ERR_NULL, "gtb_batch_run: NULL plan");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != plan->device) return fail(GTB_ERR_ARG, "gtb_batch_run: the plan belongs to device %d", plan->device);
    cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(GTB_ERR_LAUNCH, "gtb_batch_run: %s", cudaGetErrorString(e));
    return ok();
}

extern "C" int gtb_plan_info(const gtb_plan *plan, int64_t info[6]) {
    if (!plan || !info) return fail(GTB_ERR_NULL, "gtb_plan_info: NULL argument");
    info[0] = plan->h_items, info[1] = plan->v_items, info[2] = plan->h_grid, info[3] = plan->v_grid;
    info[4] = (int64_t)plan->points, info[5] = plan->n;
    return ok();
}

extern "C" int gtb_plan_destroy(gtb_plan *plan) {
    plan_free(plan);
    return GTB_OK;
}
