// hdiff_rs.cuh -- register-streaming hdiff (GT4Py paper Sec. 3.1, horizontal
// diffusion; one PARALLEL computation, Sec. 2.2):
//   lap = 4 in - (((in[i+1] + in[i-1]) + in[j+1]) + in[j-1])
//   fx  = lap[i+1] - lap[i], 0 where fx * (in[i+1] - in[i]) > 0;  fy likewise
//   out = in - coeff ((fx[i] - fx[i-1]) + (fy[j] - fy[j-1]))
//
// CTA = W warps on a TI x TJ tile (TI = 32*CPL columns, TJ = W*R rows) for a
// run of K levels.  Per level the tile box (+2 halo, left edge rounded down to
// 16 bytes) arrives by one TMA tiled load into a STAGES-deep mbarrier ring.
// Warp w owns rows [w*R, w*R+R) and all TI columns: lane l holds columns
// l*CPL .. l*CPL+CPL-1 and rolls down j keeping in, lap and fy of its columns
// in registers; the i-neighbours come from adjacent lanes by shuffles, and the
// two columns just outside the warp (i = -1 and i = TI) are computed once per
// strip by the warp itself (16 rows per side, one lane per row).  Temporaries
// never leave registers (Sec. 2.2 temporaries); one CTA barrier per level
// releases the stage.
//
// Arithmetic policies:
//   Native<T>  the definition in binary32 / binary64;
//   FixedF64   binary64 storage: the lap -> flux -> divergence chain in exact
//              int64 fixed point (integer pipe), one FP64 FMA per point for
//              out = in - coeff * D; a warp whose strip holds inf/NaN or
//              exponents outside [64, 2040] switches to Native<double>.
#pragma once

#include "hdiff_kernels.cuh"

namespace gtb {

template <typename T>
struct Native {
    using V = T;  // value type of in, lap, flux
    using Gd = T; // gradient in[i+1] - in[i]
    __device__ __forceinline__ V conv(T x) const { return x; }
    __device__ __forceinline__ V lap(V c, V e, V w, V n, V s) const { return T(4) * c - (((e + w) + n) + s); }
    __device__ __forceinline__ Gd grad(V x1, V x0, const T *, const T *) const { return x1 - x0; }
    __device__ __forceinline__ V limit(V f, Gd g) const { return (f * g > T(0)) ? T(0) : f; }
    // limit(f, grad(x1, x0, ...)) in one step; no ties to settle (kTies)
    static constexpr bool kTies = false;
    __device__ __forceinline__ V lim(V f, V x1, V x0, bool &) const { return limit(f, x1 - x0); }
    __device__ __forceinline__ T out(T in, T c, V D) const { return in - c * D; }
    __device__ __forceinline__ T outx(T in, V, T c, V D) const { return out(in, c, D); }
};

// ICVT: convert the flux divergence back to binary64 on the integer pipe
// (from_fixed_int) instead of the FP64 pipe (from_fixed); the same results.
template <bool ICVT>
struct FixedF64T {
    using V = int64_t;
    using Gd = int;
    int E;
    int iu = 0;  // ICVT: the update on the integer pipe (outx)
    __device__ __forceinline__ V conv(double x) const { return to_fixed(x, E); }
    __device__ __forceinline__ V lap(V c, V e, V w, V n, V s) const { return 4 * c - (((e + w) + n) + s); }
    // exact sign of in1 - in0; the binary64 values are read only when X1 == X0
    __device__ __forceinline__ Gd grad(V x1, V x0, const double *p1, const double *p0) const {
        if (x1 != x0) return x1 > x0 ? 1 : -1;
        return exact_dir(x1, x0, *p1, *p0);
    }
    __device__ __forceinline__ V limit(V f, Gd g) const { return ((f > 0 && g > 0) || (f < 0 && g < 0)) ? 0 : f; }
    // limit(f, grad(x1, x0, ...)) from the fixed-point values alone: f is zeroed where f
    // and d = X1 - X0 have the same strict sign (sign bits equal, d != 0; f = 0 stays 0).
    // Where X1 == X0 the binary64 values may still differ below the fixed point's unit:
    // tie is raised, and the caller settles the row with grad before using its fluxes.
    static constexpr bool kTies = true;
    __device__ __forceinline__ V lim(V f, V x1, V x0, bool &tie) const {
        const V d = x1 - x0;
        tie |= d == 0;
        return ((f ^ d) >= 0 && d != 0) ? V(0) : f;
    }
    __device__ __forceinline__ double out(double in, double c, V D) const {
        return fma(-c, ICVT ? from_fixed_int(D, E) : from_fixed(D, E), in);
    }
    // The update given in's fixed-point value X as well.  ICVT (the kernels whose FP64
    // pipe is the bottleneck) keeps it on the integer pipe: c D in units of the level's
    // fixed point 2^(E-1078), from the exact product of c's significand and D (at most
    // 115 bits) rounded to the unit, is subtracted from X and the result rounded once
    // to binary64.  X's truncation and the product's rounding add at most a unit each,
    // the size of the fixed point's own truncation (below 2^-54 of the level's largest
    // input).  A zero product returns in itself; |c| >= 1 or non-finite c (the product
    // could leave the int64 range) and levels with E > 1984 (the result's exponent
    // could overflow) take the binary64 FMA, and so does everything unless iu: the
    // integer form lengthens the producers' per-level path, which pays only when the
    // grid fills the GPU and the FP64 pipe is the bound.
    __device__ __forceinline__ double outx(double in, V X, double c, V D) const {
        if constexpr (ICVT) {
            const int hi = __double2hiint(c);
            const int ec = (hi >> 20) & 0x7FF;
            if (iu && ec <= 1022 && E <= 1984) {
                const uint64_t mc = ((uint64_t)((unsigned)hi & 0xFFFFFu) << 32 | (unsigned)__double2loint(c)) |
                                    (ec ? (1ull << 52) : 0ull);
                const uint64_t d = D < 0 ? 0ull - (uint64_t)D : (uint64_t)D;
                const uint64_t plo = mc * d, phi = __umul64hi(mc, d);  // mc d < 2^115
                const int sh = 1075 - max(ec, 1);                        // >= 53
                uint64_t r = 0;
                if (sh < 64) r = ((phi << (64 - sh)) | (plo >> sh)) + ((plo >> (sh - 1)) & 1ull);
                else if (sh == 64) r = phi + (plo >> 63);
                else if (sh < 116) r = (phi >> (sh - 64)) + ((phi >> (sh - 65)) & 1ull);
                if (r == 0) return in;
                const bool neg = (hi < 0) != (D < 0);
                return from_fixed_int(neg ? X + (int64_t)r : X - (int64_t)r, E);
            }
        }
        return out(in, c, D);
    }
};
using FixedF64 = FixedF64T<false>;

// Stage layout: the level's `in` box, then (CTMA) the tile's coeff block of TI x TJ
// values, which the same TMA transaction brings in (one mbarrier per stage).
template <typename T, int CPL, int W, int R, bool CTMA = false>
struct RsTile {
    static constexpr int TI = 32 * CPL, TJ = W * R;
    static constexpr int kAlign = 16 / (int)sizeof(T);
    static constexpr int BX = ((TI + 4 + kAlign - 1 + kAlign - 1) / kAlign) * kAlign;
    static constexpr int BY = TJ + 4;
    static constexpr int box_elems = BX * BY;
    static constexpr int box_bytes = box_elems * (int)sizeof(T);
    static constexpr int cf_offset = ((box_bytes + 127) / 128) * 128;
    static constexpr int cf_bytes = CTMA ? TI * TJ * (int)sizeof(T) : 0;
    static constexpr int tx_bytes = box_bytes + cf_bytes;
    static constexpr int stage_stride = ((cf_offset + cf_bytes + 127) / 128) * 128;
};

template <typename T, int CPL, int W, int R, int STAGES, bool CTMA = false>
constexpr int hdiff_rs_smem_bytes() {
    return STAGES * RsTile<T, CPL, W, R, CTMA>::stage_stride + STAGES * 8 + 128;
}

// One warp's R-row strip of one level.  S: the level's box; bx(ci) = ci+2+xs,
// by(cj) = cj+2 (tile-relative ci, cj).  cf: this lane's coeff rows.
template <typename T, int CPL, int R, int BX, typename P>
__device__ __forceinline__ void rs_strip(const P &pol, const T *S, int xs, int cj0, int ncols, int nrows,
                                         const T *cfp, int64_t cf_sj, T *op, int64_t out_sj, bool cf_vec,
                                         bool vec_ok) {
    using V = typename P::V;
    using Gd = typename P::Gd;
    const int lane = threadIdx.x & 31;
    const int ci0 = lane * CPL;
    auto at = [&](int ci, int cj) -> T { return S[(cj + 2) * BX + ci + 2 + xs]; };
    auto ptr = [&](int ci, int cj) -> const T * { return S + (cj + 2) * BX + ci + 2 + xs; };
    // this lane's CPL values of row cj: one 16-byte shared load when the box column is aligned
    const bool vsm = ((2 + xs) % CPL) == 0;
    auto row = [&](int cj, T (&v)[CPL]) {
        if (vsm) {
            load_vec<T, CPL>(ptr(ci0, cj), v);
        } else {
#pragma unroll
            for (int q = 0; q < CPL; ++q) v[q] = at(ci0 + q, cj);
        }
    };

    // ---- the two columns outside the warp: i = -1 (lanes 0-15) and i = TI (16-31)
    const int side = lane >> 4, er = lane & 15;
    const int eci = side ? 32 * CPL : -1;
    const int ecj = cj0 + min(er, R - 1);
    V ex_c = pol.conv(at(eci, ecj)), ex_u = pol.conv(at(eci, ecj - 1)), ex_d = pol.conv(at(eci, ecj + 1));
    const V e_lap = pol.lap(ex_c, pol.conv(at(eci + 1, ecj)), pol.conv(at(eci - 1, ecj)), ex_d, ex_u);
    // X of the outside column at strip row t (t in [-1, R]) for lane 0 (left) / lane 31 (right)
    auto edge_x = [&](int t) -> V {
        const V send = (t < 0) ? ex_u : (t >= R ? ex_d : ex_c);
        const int src = (lane < 16 ? 0 : 16) + max(0, min(t, R - 1));
        return __shfl_sync(0xffffffffu, send, src);
    };
    auto edge_lap = [&](int t) -> V { return __shfl_sync(0xffffffffu, e_lap, (lane < 16 ? 0 : 16) + t); };

    // ---- rolling state; strip row t <-> tile row cj0 + t
    V xa[CPL], xb[CPL], xc[CPL];  // X at rows t-1, t, t+1
    V lp[CPL], fyp[CPL];          // lap(t-1), fy(t-2)
    V nbL_prev = V(0), nbR_prev = V(0);  // X(c-1), X(c+1) at row t-1 for the outer columns
    {
        T ra[CPL], rb[CPL], rc[CPL];
        row(cj0 - 2, ra);
        row(cj0 - 1, rb);
        row(cj0, rc);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            xa[q] = pol.conv(ra[q]);
            xb[q] = pol.conv(rb[q]);
            xc[q] = pol.conv(rc[q]);
            lp[q] = V(0), fyp[q] = V(0);
        }
    }
    // coeff ring: at the top of iteration t, cf[0] .. cf[NCF-1] hold rows t-1 .. t+NCF-2
    // (16-byte loads when aligned); a row is loaded NCF iterations before its use.  The
    // binary64 strip's short fixed-point rows need the loads further ahead (measured on
    // B300 at 256x256x80: 55.7 us with 5 rows, 52.9 with 9, 54.9 with 11, 55.8 with 13)
    constexpr int NCF = sizeof(T) == 8 ? 9 : 5;
    auto load_cf = [&](int rw, T (&v)[CPL]) {
        if (rw >= 0 && rw < nrows) {
            const T *c = cfp + (int64_t)(cj0 + rw) * cf_sj;
            if (cf_vec && ncols == CPL) {
                load_vec<T, CPL>(c, v);
                return;
            }
#pragma unroll
            for (int q = 0; q < CPL; ++q) v[q] = q < ncols ? c[q] : T(0);
        } else {
#pragma unroll
            for (int q = 0; q < CPL; ++q) v[q] = T(0);
        }
    };
    T cf[NCF][CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) cf[0][q] = T(0), cf[1][q] = T(0);
#pragma unroll
    for (int i = 2; i < NCF; ++i) load_cf(i - 2, cf[i]);
    // iteration t computes lap(row t) for t = -1 .. R and emits out(row t-1) for t >= 1;
    // fully unrolled, so the rolling rows need no register moves
#pragma unroll
    for (int t = -1; t <= R; ++t) {
        // X neighbours in i at row t
        V up = __shfl_up_sync(0xffffffffu, xb[CPL - 1], 1);
        V dn = __shfl_down_sync(0xffffffffu, xb[0], 1);
        const V ex = edge_x(t);
        if (lane == 0) up = ex;
        if (lane == 31) dn = ex;
        V lc[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const V w = (q == 0) ? up : xb[q - 1];
            const V e = (q == CPL - 1) ? dn : xb[q + 1];
            lc[q] = pol.lap(xb[q], e, w, xc[q], xa[q]);
        }
        if (t >= 0) {
            // fy(row t-1) = lap(t) - lap(t-1), gradient in(t) - in(t-1)
            // the fluxes from the policy's fast limiter (lim); a tie anywhere in the warp
            // (fixed point only) recomputes the row's fluxes with the exact gradient sign
            bool tie = false;
            V fyc[CPL];
            auto fy_exact = [&]() {
#pragma unroll
                for (int q = 0; q < CPL; ++q)
                    fyc[q] = pol.limit(lc[q] - lp[q],
                                       pol.grad(xb[q], xa[q], ptr(ci0 + q, cj0 + t), ptr(ci0 + q, cj0 + t - 1)));
            };
#pragma unroll
            for (int q = 0; q < CPL; ++q) fyc[q] = pol.lim(lc[q] - lp[q], xb[q], xa[q], tie);
            if (t == 0 && P::kTies && __any_sync(0xffffffffu, tie)) fy_exact();
            if (t >= 1) {
                // output row j = t-1: fx(row j) from lap(t-1) (= lp) of this lane and its right neighbour
                const int j = t - 1;
                V lnext = __shfl_down_sync(0xffffffffu, lp[0], 1);
                const V el = edge_lap(j);
                if (lane == 31) lnext = el;
                V fx[CPL];
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const V ln = (q == CPL - 1) ? lnext : lp[q + 1];
                    const V xn = (q == CPL - 1) ? nbR_prev : xa[q + 1];
                    fx[q] = pol.lim(ln - lp[q], xn, xa[q], tie);
                }
                // fx(i = -1) = lap(0) - lap(-1), lane 0's (every lane evaluates it)
                bool tie0 = false;
                V fx0 = pol.lim(lp[0] - el, xa[0], nbL_prev, tie0);
                tie |= lane == 0 && tie0;
                if (P::kTies && __any_sync(0xffffffffu, tie)) {
                    fy_exact();
#pragma unroll
                    for (int q = 0; q < CPL; ++q) {
                        const V ln = (q == CPL - 1) ? lnext : lp[q + 1];
                        const V xn = (q == CPL - 1) ? nbR_prev : xa[q + 1];
                        fx[q] = pol.limit(ln - lp[q],
                                          pol.grad(xn, xa[q], ptr(ci0 + q + 1, cj0 + j), ptr(ci0 + q, cj0 + j)));
                    }
                    fx0 = pol.limit(lp[0] - el, pol.grad(xa[0], nbL_prev, ptr(0, cj0 + j), ptr(-1, cj0 + j)));
                }
                V fxw = __shfl_up_sync(0xffffffffu, fx[CPL - 1], 1);
                if (lane == 0) fxw = fx0;
                T r[CPL], xin[CPL];
                row(cj0 + j, xin);
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const V fwq = (q == 0) ? fxw : fx[q - 1];
                    const V D = (fx[q] - fwq) + (fyc[q] - fyp[q]);
                    r[q] = pol.out(xin[q], cf[0][q], D);
                }
                if (j < nrows) {
                    T *o = op + (int64_t)(cj0 + j) * out_sj;
                    if (vec_ok && ncols >= CPL) {
                        store_vec<T, CPL>(o, r);
                    } else {
#pragma unroll
                        for (int q = 0; q < CPL; ++q)
                            if (q < ncols) o[q] = r[q];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < CPL; ++q) fyp[q] = fyc[q];
        }
        T rn[CPL];
        if (t + 2 <= R + 1) row(cj0 + t + 2, rn);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            lp[q] = lc[q];
            xa[q] = xb[q];
            xb[q] = xc[q];
            if (t + 2 <= R + 1) xc[q] = pol.conv(rn[q]);
        }
        nbL_prev = up, nbR_prev = dn;
#pragma unroll
        for (int i = 0; i + 1 < NCF; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) cf[i][q] = cf[i + 1][q];
        load_cf(t + NCF - 1, cf[NCF - 1]);
    }
}

// One work item: tile `tile` of the launch geometry g, K-chunk `kchunk`.
// Block-uniform; the caller provides the shared-memory stages and barriers.
// CTMA (with USE_TMA): coeff arrives with each level's box by a second tiled
// TMA load (cmap, box TI x TJ at g.CX0 + ti0, g.CY0 + tj0, g.CZ0 + k) instead
// of being loaded from global memory row by row inside the strip.
template <typename T, int CPL, int W, int R, int STAGES, bool USE_TMA, bool FIXED, bool CTMA = false>
__device__ __forceinline__ void hdiff_rs_item(const CUtensorMap *tmap, const CUtensorMap *cmap, const View<T> &in,
                                              const View<T> &coeff, const View<T> &out, const HdiffGeom &g,
                                              int vec_ok, int tile, int kchunk, unsigned char *base,
                                              uint64_t *bars) {
    static_assert(!CTMA || USE_TMA, "coeff by TMA needs the TMA ring");
    using G = RsTile<T, CPL, W, R, CTMA>;
    constexpr int NT = 32 * W;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ti0 = (tile % g.tiles_i) * G::TI, tj0 = (tile / g.tiles_i) * G::TJ;
    const int k0 = kchunk * g.kc;
    const int nk = min(g.kc, g.K - k0);
    if (nk <= 0) return;
    const int xs = g.xs;
    const int cj0 = warp * R;
    const int nrows = max(0, min(R, g.J - tj0 - cj0));  // rows of this strip inside the domain
    const int ncols = max(0, min(CPL, g.I - ti0 - lane * CPL));

    // TMA ring: (re)initialised per item; no load is in flight between items
    auto issue = [&](int s, int k) {  // one level's box (and coeff block) into stage s
        mbar_arrive_expect_tx(&bars[s], G::tx_bytes);
        tma_load_3d(base + s * G::stage_stride, tmap, &bars[s], g.X0 + ti0, g.Y0 + tj0, g.Z0 + k);
        if constexpr (CTMA)
            tma_load_3d(base + s * G::stage_stride + G::cf_offset, cmap, &bars[s], g.CX0 + ti0, g.CY0 + tj0, g.CZ0 + k);
    };
    if (USE_TMA) {
        if (tid == 0) {
            prefetch_tensormap(tmap);
            if constexpr (CTMA) prefetch_tensormap(cmap);
            for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0)
            for (int p = 0; p < STAGES && p < nk; ++p) issue(p, k0 + p);
    }
    bool failed = false;
    for (int p = 0; p < nk; ++p) {
        const int k = k0 + p;
        const T *S = reinterpret_cast<const T *>(base + (USE_TMA ? (p % STAGES) : 0) * G::stage_stride);
        if (USE_TMA) {
            if (!mbar_wait(&bars[p % STAGES], (p / STAGES) & 1)) failed = true;
        } else {
            T *D = reinterpret_cast<T *>(base);
            for (int idx = tid; idx < G::box_elems; idx += NT) {
                const int bx = idx % G::BX, by = idx / G::BX;
                const int i = ti0 - 2 - xs + bx, j = tj0 - 2 + by;
                T v = T(0);
                if (i >= -2 && i < g.I + 2 && j >= -2 && j < g.J + 2) {
                    const T *q = in.p + (int64_t)i + (int64_t)j * in.sj + (int64_t)k * in.sk;
                    if (!kChecked || in_storage(in, q, q)) v = *q;
                }
                D[idx] = v;
            }
            __syncthreads();
        }
        if (__syncthreads_or(failed)) break;
        if (nrows > 0) {
            // this lane's coeff at tile row 0: the staged block (row pitch TI) or global memory
            const T *cfp = CTMA ? reinterpret_cast<const T *>(reinterpret_cast<const unsigned char *>(S) + G::cf_offset) +
                                      lane * CPL
                                : coeff.p + (int64_t)(ti0 + lane * CPL) + (int64_t)tj0 * coeff.sj + (int64_t)k * coeff.sk;
            const int64_t cf_sj = CTMA ? (int64_t)G::TI : coeff.sj;
            const int cf_vec = CTMA ? 1 : vec_ok;
            T *op = out.p + (int64_t)(ti0 + lane * CPL) + (int64_t)tj0 * out.sj + (int64_t)k * out.sk;
            // checked build: the strip's coeff and out rows inside their storages (else the warp skips it)
            bool run = true;
            if constexpr (kChecked) {
                bool ok = true;
                if (ncols > 0) {
                    const int64_t r0 = cj0, r1 = cj0 + nrows - 1;
                    ok = in_storage(out, op + r0 * out.sj, op + r1 * out.sj + (ncols - 1));
                    if (!CTMA) ok = ok && in_storage(coeff, cfp + r0 * cf_sj, cfp + r1 * cf_sj + (ncols - 1));
                }
                run = __all_sync(0xffffffffu, ok);
            }
            if (!run) {
            } else if constexpr (FIXED) {
                // largest biased exponent over the values the strip's stored outputs read:
                // rows cj0-2 .. cj0+nrows+1, columns -2 .. ntile+1 of the tile, restricted to the
                // cells the definition reads (never the storage padding beyond the halo or the
                // unread halo corners, whose contents are arbitrary)
                const int ntile = min(G::TI, g.I - ti0);
                const int wx = ntile + 4, wy = nrows + 4;
                // a strip at a corner of the domain first zeroes, in its copy of the box,
                // the halo cells that the definition never reads (their contents are arbitrary)
                if ((ti0 == 0 || ti0 + ntile == g.I) && (tj0 + cj0 == 0 || tj0 + cj0 + nrows == g.J)) {
                    if (lane < 12) {
                        const int c = lane / 3, e = lane % 3;
                        const int di = e == 2 ? -1 : -2, dj = e == 1 ? -1 : -2;
                        const int gi = (c & 1) ? g.I - 1 - di : di, gj = (c & 2) ? g.J - 1 - dj : dj;
                        const int cx = gi - ti0 + 2, cy = gj - tj0 - cj0 + 2;
                        if (cx >= 0 && cx < wx && cy >= 0 && cy < wy)
                            const_cast<T *>(S)[(cy + cj0) * G::BX + cx + xs] = T(0);
                    }
                    fence_proxy_async_shared();  // before the stage's next TMA refill
                    __syncwarp();
                }
                // the maximum of the exponent fields (hi word & 0x7FF00000, monotone in the
                // exponent): each lane its own columns of every row, 16-byte loads where the
                // box column allows; then the four columns outside the lanes' (-2, -1, TI, TI+1)
                unsigned em = 0;
                const int c0 = lane * CPL;
                const bool vsm = ((2 + xs) % CPL) == 0;
#pragma unroll
                for (int r = 0; r < R + 4; ++r) {
                    if (r < wy) {
                        const T *rp = S + (cj0 + r) * G::BX + c0 + 2 + xs;
                        T v[CPL];
                        if (vsm) {
                            load_vec<T, CPL>(rp, v);
                        } else {
#pragma unroll
                            for (int q = 0; q < CPL; ++q) v[q] = rp[q];
                        }
#pragma unroll
                        for (int q = 0; q < CPL; ++q)
                            if (c0 + q < wx - 2) em = max(em, (unsigned)__double2hiint(v[q]) & 0x7FF00000u);
                    }
                }
                for (int idx = lane; idx < 4 * wy; idx += 32) {
                    const int sd = idx & 3, c = sd < 2 ? sd - 2 : G::TI + sd - 2;
                    if (c < wx - 2) em = max(em, (unsigned)__double2hiint(S[(cj0 + (idx >> 2)) * G::BX + c + 2 + xs]) & 0x7FF00000u);
                }
                const int E = (int)(__reduce_max_sync(0xffffffffu, em) >> 20);
                if (E >= 64 && E <= 2040)
                    rs_strip<T, CPL, R, G::BX>(FixedF64{E}, S, xs, cj0, ncols, nrows, cfp, cf_sj, op, out.sj,
                                               cf_vec != 0, vec_ok != 0);
                else
                    rs_strip<T, CPL, R, G::BX>(Native<T>{}, S, xs, cj0, ncols, nrows, cfp, cf_sj, op, out.sj,
                                               cf_vec != 0, vec_ok != 0);
            } else {
                rs_strip<T, CPL, R, G::BX>(Native<T>{}, S, xs, cj0, ncols, nrows, cfp, cf_sj, op, out.sj,
                                           cf_vec != 0, vec_ok != 0);
            }
        }
        __syncthreads();  // every warp is done with this stage
        if (USE_TMA && tid == 0 && p + STAGES < nk) issue(p % STAGES, k + STAGES);
    }
    if (USE_TMA && failed) {
        if (tid == 0)
            for (int s = 0; s < STAGES; ++s) mbar_wait(&bars[s], 0), mbar_wait(&bars[s], 1);
        __syncthreads();
    }
}

template <typename T, int CPL, int W, int R, int STAGES, bool CTMA = false>
__device__ __forceinline__ unsigned char *hdiff_rs_smem(uint64_t **bars) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    *bars = reinterpret_cast<uint64_t *>(base + STAGES * RsTile<T, CPL, W, R, CTMA>::stage_stride);
    return base;
}

// Single domain: one CTA per (tile, K-chunk) item.
template <typename T, int CPL, int W, int R, int STAGES, bool USE_TMA, bool FIXED, bool CTMA = false>
__global__ void __launch_bounds__(32 * W)
    hdiff_rs_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap cmap,
                    const View<T> in, const View<T> coeff, const View<T> out, const HdiffGeom g, const int vec_ok) {
    uint64_t *bars;
    unsigned char *base = hdiff_rs_smem<T, CPL, W, R, STAGES, CTMA>(&bars);
    hdiff_rs_item<T, CPL, W, R, STAGES, USE_TMA, FIXED, CTMA>(&tmap, &cmap, in, coeff, out, g, vec_ok,
                                                               blockIdx.x % g.n_tiles, blockIdx.x / g.n_tiles, base,
                                                               bars);
}

}  // namespace gtb
