// fused_kernels.cuh -- hdiff feeding vadv in one kernel (the two stencils of
// the GT4Py paper, Sec. 3.1, chained as h = hdiff(in, coeff),
// utens_stage_out = vadv(u_stage = h, u_pos = h, utens, utens_stage, wcon);
// Sec. 2.2 leaves the backend free to fuse the computations it runs).  h is
// produced level by level inside the SM and consumed there: it is never
// written to memory.
//
// CTA = a TI x TJ tile of columns, all K levels, warp-specialised:
//   * TI*TJ/32 consumer warps, one thread per column (t -> i = t % TI,
//     j = t / TI): the column's forward elimination step of level m-1 as soon
//     as h_m is ready, then the back substitution (the FP64- or FP32-pipe
//     bound part);
//   * PW producer warps: per level the (TI+4) x (TJ+4) box of `in` arrives by
//     TMA (STAGES-deep ring); binary64 storage converts it to exact int64 fixed
//     point (the form of hdiff_rs: E = the largest exponent among the cells the
//     tile's outputs read; a level whose E leaves [64, 2040] uses the
//     definition in binary64; the result goes back to binary64 on the integer
//     pipe, leaving the FP64 pipe to the column solve), forms the Laplacian on
//     (TI+2) x (TJ+2) cells,
//     the limited fluxes and h of the tile into a RING-deep shared ring (the
//     integer-pipe bound part).  A squarer tile needs fewer halo cells per
//     column: (TI+4)(TJ+4)/(TI TJ) conversions, (TI+2)(TJ+2)/(TI TJ) Laplacians.
// The two sides meet only through the ring's full / empty mbarriers (bounded
// waits), so the producers run up to RING levels ahead and the consumers never
// wait on a block barrier.
// The column solve takes the system in the shifted unknown y = x + h (with
// beta_v = 0 the explicit terms then fold into the matrix) and runs the back
// substitution on z = x - h, so that h is not needed after the forward sweep:
//   e_k = (d'_k - 2h_k) - c'_k 2h_{k+1},   z_{K-1} = e_{K-1},
//   z_k = e_k - c'_k z_{k+1},              utens_stage_out_k = dtr z_k,
// the same unknowns as x_k - h_k of the Thomas solution, in a different
// rounding order (fused_consumer).  c'_k goes to the caller's workspace, e_k is
// parked in the output array (or in the workspace when the arithmetic type is
// wider than the storage type).
#pragma once

#include "hdiff_rs.cuh"
#include "vadv_kernels.cuh"

namespace gtb {

template <typename T, int TI, int TJ>
struct FusedTile {
    static_assert(TI == 8 || TI == 16 || TI == 32, "a warp covers whole rows of the tile");
    static_assert((TI * TJ) % 32 == 0, "whole consumer warps");
    static constexpr int kAlign = 16 / (int)sizeof(T);
    static constexpr int BX = ((TI + 4 + kAlign - 1 + kAlign - 1) / kAlign) * kAlign;  // box width (+ alignment)
    static constexpr int BY = TJ + 4;
    static constexpr int box_elems = BX * BY;
    static constexpr int box_bytes = box_elems * (int)sizeof(T);
    static constexpr int stage_stride = ((box_bytes + 127) / 128) * 128;
    static constexpr int XW = TI + 4, XH = TJ + 4;  // cells ci in [-2, TI+1], cj in [-2, TJ+1]
    static constexpr int LW = TI + 2, LH = TJ + 2;  // Laplacians li in [-1, TI], lj in [-1, TJ]
    static constexpr int NC = TI * TJ;              // columns = consumer threads
    static constexpr int CW = NC / 32;              // consumer warps
};

template <typename T, int TI, int TJ, int PW, int STAGES, int RING>
struct FusedLayout {
    using Tile = FusedTile<T, TI, TJ>;
    static constexpr int x_off = STAGES * Tile::stage_stride;
    static constexpr int l_off = x_off + Tile::XW * Tile::XH * 8;
    static constexpr int e_off = l_off + Tile::LW * Tile::LH * 8;  // per producer warp exponent maxima
    static constexpr int h_off = e_off + ((PW * 4 + 15) / 16) * 16;
    static constexpr int bar_off = h_off + ((RING * Tile::NC * (int)sizeof(T) + 7) / 8) * 8;
    static constexpr int bytes = bar_off + (STAGES + 2 * RING) * 8;
    static constexpr int smem_bytes = bytes + 128;  // + slack for the 128-byte base alignment
};

// Cells of one level's box, tile-relative (ci, cj).
template <typename T, typename V, int TI, int TJ, bool FIXED>
struct FusedCells {
    using Tile = FusedTile<T, TI, TJ>;
    const T *S;  // the TMA box: cell (ci, cj) at S[(cj+2)*BX + ci+2+xs]
    const V *X;  // fixed point: X[(cj+2)*XW + ci+2]; unused for the definition
    const V *L;  // Laplacian: L[(lj+1)*LW + li+1]
    int xs;
    __device__ __forceinline__ const T *sp(int ci, int cj) const { return S + (cj + 2) * Tile::BX + ci + 2 + xs; }
    __device__ __forceinline__ V x(int ci, int cj) const {
        if constexpr (FIXED) return X[(cj + 2) * Tile::XW + ci + 2];
        else return *sp(ci, cj);
    }
    __device__ __forceinline__ V lap(int li, int lj) const { return L[(lj + 1) * Tile::LW + li + 1]; }
};

// Barrier among the PW producer warps (named barrier 1; a warp barrier for one warp).
template <int PW>
__device__ __forceinline__ void producer_sync() {
    if constexpr (PW == 1) __syncwarp();
    else asm volatile("bar.sync 1, %0;" ::"n"(32 * PW) : "memory");
}

// The producers' level with policy P (FixedF64 or Native<T>): Laplacians into Lw
// (split over the producer threads, then a producer barrier), then h of the
// tile's points pt, pt + NPT, ... handed to em.put(level, point, value).
template <int TI, int TJ, int PW, typename P, typename C, typename T, typename Emit>
__device__ __forceinline__ void fused_hdiff_level(const P &pol, const C &c, typename P::V *Lw, int pt,
                                                  const T (&cf)[(TI * TJ + 32 * PW - 1) / (32 * PW)], int m,
                                                  const Emit &em) {
    using V = typename P::V;
    using Tile = FusedTile<T, TI, TJ>;
    constexpr int NPT = 32 * PW, PPT = (Tile::NC + NPT - 1) / NPT;
    static_assert(!P::kTies || Tile::NC % NPT == 0, "the tie vote needs every producer lane on every point");
    for_cells<Tile::LW, Tile::LH, NPT>(pt, [&](int idx, int la, int lb) {
        const int li = la - 1, lj = lb - 1;
        Lw[idx] = pol.lap(c.x(li, lj), c.x(li + 1, lj), c.x(li - 1, lj), c.x(li, lj + 1), c.x(li, lj - 1));
    });
    producer_sync<PW>();
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int p = pt + q * NPT;
        if (Tile::NC % NPT != 0 && p >= Tile::NC) break;
        const int ci = p % TI, cj = p / TI;
        const V x0 = c.x(ci, cj), l0 = c.lap(ci, cj);
        // the policy's fast limiter; a fixed-point tie anywhere in the warp recomputes
        // the cell's fluxes with the exact gradient sign (every lane is here: NC % NPT == 0)
        bool tie = false;
        V fxe = pol.lim(c.lap(ci + 1, cj) - l0, c.x(ci + 1, cj), x0, tie);
        V fxw = pol.lim(l0 - c.lap(ci - 1, cj), x0, c.x(ci - 1, cj), tie);
        V fyn = pol.lim(c.lap(ci, cj + 1) - l0, c.x(ci, cj + 1), x0, tie);
        V fys = pol.lim(l0 - c.lap(ci, cj - 1), x0, c.x(ci, cj - 1), tie);
        if (P::kTies && __any_sync(0xffffffffu, tie)) {
            fxe = pol.limit(c.lap(ci + 1, cj) - l0, pol.grad(c.x(ci + 1, cj), x0, c.sp(ci + 1, cj), c.sp(ci, cj)));
            fxw = pol.limit(l0 - c.lap(ci - 1, cj), pol.grad(x0, c.x(ci - 1, cj), c.sp(ci, cj), c.sp(ci - 1, cj)));
            fyn = pol.limit(c.lap(ci, cj + 1) - l0, pol.grad(c.x(ci, cj + 1), x0, c.sp(ci, cj + 1), c.sp(ci, cj)));
            fys = pol.limit(l0 - c.lap(ci, cj - 1), pol.grad(x0, c.x(ci, cj - 1), c.sp(ci, cj), c.sp(ci, cj - 1)));
        }
        const V D = (fxe - fxw) + (fyn - fys);
        em.put(m, p, pol.outx(*c.sp(ci, cj), x0, cf[q], D));
    }
}

// Where the producers put h: the shared ring of the chained kernel (a slot is
// acquired through its `empty` barrier and published through `full`), or a
// field in global memory (hdiff as a stencil of its own).
template <typename T>
struct RingEmit {
    T *H;
    uint64_t *full, *empty;
    int nc, ring;
    __device__ __forceinline__ bool acquire(int m) const {
        return m < ring || mbar_wait(&empty[m % ring], ((m / ring) - 1) & 1);
    }
    __device__ __forceinline__ void put(int m, int p, T v) const { H[(m % ring) * nc + p] = v; }
    __device__ __forceinline__ void publish(int m) const {
        __syncwarp();  // this warp's points of h are written
        if ((threadIdx.x & 31) == 0) mbar_arrive(&full[m % ring]);
    }
};

template <typename T>
struct GlobalEmit {
    View<T> out;
    int ti0, tj0, I, J, ti;
    __device__ __forceinline__ bool acquire(int) const { return true; }
    __device__ __forceinline__ void put(int m, int p, T v) const {
        const int i = ti0 + p % ti, j = tj0 + p / ti;
        if (i < I && j < J) {
            T *q = out.p + i + (int64_t)j * out.sj + (int64_t)m * out.sk;
            if (!kChecked || in_storage(out, q, q)) *q = v;
        }
    }
    __device__ __forceinline__ void publish(int) const {}
};

// The producer warps of a CTA (warps CW .. CW+PW-1): hdiff of the TI x TJ tile
// at (ti0, tj0), level by level, handed to `em`.  Shared memory: the TMA ring
// at `base`, then X, L and the exponent slots of the layout; barriers tbar.
template <typename T, int TI, int TJ, int PW, int STAGES, bool USE_TMA, typename Emit>
__device__ __forceinline__ void hdiff_producer(const CUtensorMap *tmap, const View<const T> &in,
                                               const View<const T> &coeff, const HdiffGeom &hg, int ti0, int tj0,
                                               unsigned char *base, int x_off, int l_off, int e_off, uint64_t *tbar,
                                               const Emit &em) {
    using Tile = FusedTile<T, TI, TJ>;
    constexpr bool FIX = sizeof(T) == 8;           // binary64 storage: exact fixed-point hdiff
    constexpr int NC = Tile::NC, CW = Tile::CW;
    constexpr int NPT = 32 * PW;                   // producer threads
    constexpr int NCELL = Tile::XW * Tile::XH;     // box cells
    constexpr int CPT = (NCELL + NPT - 1) / NPT;   // cells per producer thread
    constexpr int PPT = (NC + NPT - 1) / NPT;      // points per producer thread
    const int lane = threadIdx.x & 31, pw = (threadIdx.x >> 5) - CW, pt = pw * 32 + lane;
    const int I = hg.I, J = hg.J, K = hg.K;
    int64_t *Xs = reinterpret_cast<int64_t *>(base + x_off);
    unsigned char *Lraw = base + l_off;
    unsigned *es = reinterpret_cast<unsigned *>(base + e_off);
    const int xs = hg.xs;
    if (USE_TMA && pt == 0) {
        prefetch_tensormap(tmap);
        for (int p = 0; p < STAGES && p < K; ++p) {
            mbar_arrive_expect_tx(&tbar[p], Tile::box_bytes);
            tma_load_3d(base + p * Tile::stage_stride, tmap, &tbar[p], hg.X0 + ti0, hg.Y0 + tj0, hg.Z0 + p);
        }
    }
    // this thread's box cells (the same at every level): offset in the box, and
    // whether hdiff reads the cell (bit q of rmask)
    int coff[CPT];
    unsigned rmask = 0;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int idx = pt + q * NPT;
        const int ci = idx % Tile::XW - 2, cj = idx / Tile::XW - 2;
        coff[q] = (cj + 2) * Tile::BX + ci + 2 + xs;
        if (idx < NCELL && hdiff_reads(ti0 + ci, tj0 + cj, I, J)) rmask |= 1u << q;
    }
    // coeff of this thread's points, one level ahead
    const T *pcf[PPT];
    T cf_n[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int p = min(pt + q * NPT, NC - 1);
        pcf[q] = coeff.p + min(ti0 + p % TI, I - 1) + (int64_t)min(tj0 + p / TI, J - 1) * coeff.sj;
        // checked build: a point whose coeff column leaves the storage reads coeff = 0 instead
        if (kChecked && !in_storage(coeff, pcf[q], pcf[q] + (int64_t)(K - 1) * coeff.sk)) pcf[q] = nullptr;
        cf_n[q] = (!kChecked || pcf[q]) ? pcf[q][0] : T(0);
    }
    bool failed = false;
    for (int m = 0; m < K; ++m) {
        T cf[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            cf[q] = cf_n[q];
            if (m + 1 < K && (!kChecked || pcf[q])) cf_n[q] = pcf[q][(int64_t)(m + 1) * coeff.sk];
        }
        const int s = USE_TMA ? m % STAGES : 0;
        const T *S = reinterpret_cast<const T *>(base + s * Tile::stage_stride);
        if (USE_TMA) {
            if (!mbar_wait(&tbar[s], (m / STAGES) & 1)) failed = true;
        } else {
            T *D = reinterpret_cast<T *>(base);
            for (int idx = pt; idx < Tile::box_elems; idx += NPT) {
                const int bx = idx % Tile::BX, by = idx / Tile::BX;
                const int gi = ti0 - 2 + bx, gj = tj0 - 2 + by;
                T v = T(0);
                if (gi >= -2 && gi < I + 2 && gj >= -2 && gj < J + 2) {
                    const T *q = in.p + (int64_t)gi + (int64_t)gj * in.sj + (int64_t)m * in.sk;
                    if (!kChecked || in_storage(in, q, q)) v = *q;
                }
                D[idx] = v;
            }
            producer_sync<PW>();
        }
        // this thread's cells; binary64: the largest exponent among the cells read
        T v[CPT];
        unsigned emax = 0;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            v[q] = (pt + q * NPT < NCELL) ? S[coff[q]] : T(0);
            if constexpr (FIX)
                if ((rmask >> q) & 1u) emax = max(emax, ((unsigned)__double2hiint(v[q]) >> 20) & 0x7FFu);
        }
        emax = __reduce_max_sync(0xffffffffu, emax);
        // a wait that expired (this level's box, or the previous level's ring slot) is
        // published with the exponents, so that every producer warp leaves here together
        const bool wf = __any_sync(0xffffffffu, failed);
        if (lane == 0) es[pw] = wf ? 0xFFFFFFFFu : emax;
        producer_sync<PW>();
        unsigned E = 0;
#pragma unroll
        for (int q = 0; q < PW; ++q) E = max(E, es[q]);
        if (E == 0xFFFFFFFFu) {
            failed = true;
            break;
        }
        // every producer is past the previous level: its box stage can be refilled
        if (USE_TMA && pt == 0 && m >= 1 && m - 1 + STAGES < K) {
            const int sp = (m - 1) % STAGES;
            mbar_arrive_expect_tx(&tbar[sp], Tile::box_bytes);
            tma_load_3d(base + sp * Tile::stage_stride, tmap, &tbar[sp], hg.X0 + ti0, hg.Y0 + tj0,
                        hg.Z0 + m - 1 + STAGES);
        }
        const bool fixed = FIX && E >= 64 && E <= 2040;
        if constexpr (FIX) {
            if (fixed) {
#pragma unroll
                for (int q = 0; q < CPT; ++q)
                    if (pt + q * NPT < NCELL) Xs[pt + q * NPT] = to_fixed(v[q], (int)E);
            }
        }
        if (!em.acquire(m)) failed = true;
        bool done = false;
        if constexpr (FIX) {
            if (fixed) {
                producer_sync<PW>();  // X complete
                const FusedCells<T, int64_t, TI, TJ, true> c{S, Xs, reinterpret_cast<const int64_t *>(Lraw), xs};
                fused_hdiff_level<TI, TJ, PW>(FixedF64T<true>{(int)E, hg.int_update}, c, reinterpret_cast<int64_t *>(Lraw), pt, cf,
                                              m, em);
                done = true;
            }
        }
        if (!done) {
            const FusedCells<T, T, TI, TJ, false> c{S, nullptr, reinterpret_cast<const T *>(Lraw), xs};
            fused_hdiff_level<TI, TJ, PW>(Native<T>{}, c, reinterpret_cast<T *>(Lraw), pt, cf, m, em);
        }
        em.publish(m);
    }
    if (USE_TMA && failed && pt == 0)  // let the box loads in flight land before leaving
        for (int s = 0; s < STAGES; ++s) mbar_wait(&tbar[s], 0), mbar_wait(&tbar[s], 1);
}

// 2 h in the arithmetic type: exact.  Binary64 storage and arithmetic: the exponent
// field raised by one on the integer pipe (bit for bit the binary64 sum h + h: a
// subnormal h shifts its significand, 2 h past the largest finite value is infinity,
// infinities and NaN stay), which takes one of the chain's operations off the FP64
// pipe that bounds it.
template <typename N, typename T>
__device__ __forceinline__ N twice(T h) {
    return add2<N, T>(h, h);
}
template <>
__device__ __forceinline__ double twice<double, double>(double h) {
    const long long b = __double_as_longlong(h);
    const int e = (int)((b >> 52) & 0x7FF);
    const long long sign = b & (1ll << 63);
    if (e != 0 && e < 2046) return __longlong_as_double(b + (1ll << 52));
    if (e == 0) return __longlong_as_double(sign | ((b & 0x7FFFFFFFFFFFFFFFll) << 1));
    if (e == 2046) return __longlong_as_double(sign | 0x7FF0000000000000ll);
    return h;
}

// The consumer warps of hdiff_vadv_kernel: the vadv column solve of the tile's
// columns, level by level as the producers publish h.  With u_stage = u_pos = h
// the system of Sec. 3.1 is solved in the shifted unknown y = x + h (the explicit
// terms fold into the matrix when SYM, i.e. beta_v = 0):
//   A y = 2 dtr h_k + utens_k + utens_stage_k [+ g_k (h_k - h_{k-1}) + g_{k+1} (h_{k+1} - h_k)]
// with g = as - a, and the back substitution runs in z = x - h = y - 2h, the output
// over dtr: z_k = e_k - c'_k z_{k+1}, e_k = d'_k - 2h_k - c'_k 2h_{k+1}.  SYM gets a
// body of its own so that no FP64 instruction of the general case is issued.
// ws: c'_k ([k][j*I + i]); rsave: 1/p_k in the same layout, or null (the factors
// kept for the adjoint); ework: e_k when it is not parked in the output.
template <typename T, typename N, int TI, int TJ, int RING, bool DPG, bool SYM>
__device__ __forceinline__ void fused_consumer(const View<const T> &wc, const View<const T> &ut,
                                               const View<const T> &uts, const View<T> &out, const VadvGeom &g,
                                               N *__restrict__ ws, N *__restrict__ rsave, N *__restrict__ ework,
                                               const T *H, uint64_t *full, uint64_t *empty, int NC, int ti0, int tj0,
                                               int tid) {
    const int lane = tid & 31;
    const int I = g.I, J = g.J, K = g.K;
    const int ci = tid % TI, cj = tid / TI;
    const int i = ti0 + ci, j = tj0 + cj;
    const bool active = (i < I) && (j < J);
    const int ilim = g.literal ? I - 1 : I;  // last wcon column read (I-staggered unless literal)
    const int ic = min(i, I - 1), jc = min(j, J - 1), iw = min(i, ilim);
    const T *put = ut.p + ic + (int64_t)jc * ut.sj;
    const T *puts = uts.p + ic + (int64_t)jc * uts.sj;  // may alias po (in place)
    const T *pw = wc.p + iw + (int64_t)jc * wc.sj;
    const T *pw1 = wc.p + min(i + 1, ilim) + (int64_t)jc * wc.sj;
    T *po = out.p + ic + (int64_t)jc * out.sj;
    const size_t cstride = (size_t)I * J, cidx = (size_t)jc * I + ic;
    if constexpr (kChecked) {  // every level of the column inside every field's storage
        const int64_t kl = K - 1;
        const bool ok = in_storage(ut, put, put + kl * ut.sk) && in_storage(uts, puts, puts + kl * uts.sk) &&
                        in_storage(wc, pw, pw + kl * wc.sk) && in_storage(wc, pw1, pw1 + kl * wc.sk) &&
                        in_storage(out, po, po + kl * out.sk);
        // the warp leaves; the producers' waits on its ring slots then expire (bounded)
        if (!__all_sync(0xffffffffu, ok)) return;
    }
    N *cpb = ws;
    N *epb = ework;  // e_k when it is not parked in the output
    const bool row_end = (ci == TI - 1);  // wcon(i+1) is not held by the next lane
    const bool lit = g.literal != 0;

    const N dtr = num_const<N>(g.dtr);
    const N ka = num_const<N>(g.ka);
    const N kg = num_const<N>(g.kg);
    const N zero = num_const<N>(0.0);
    const int kexp = g.ka_pow2;

    N a_cur = zero, g_cur = zero, dpl_prev = zero, cp_prev = zero, dp_prev = zero, e_last = zero;

    // forward elimination step of level k; hk = h_k, hk1 = h_{k+1}, s_cur = 2 h_k,
    // s_nx = 2 h_{k+1} (each formed once, when its level arrives)
    auto vstep = [&](int k, bool has_next, T hk, T hk1, N s_cur, N s_nx, T utk, T utsk, T wk1, T w1k1) {
        N a_next = zero, g_next = zero, s_next = zero, dpl = zero;
        if (has_next) {
            N sface;
            if (lit) {
                sface = to_num<N, T>(wk1);
            } else {
                T hi = __shfl_down_sync(0xffffffffu, wk1, 1);
                if (row_end) hi = w1k1;
                sface = add2<N, T>(wk1, hi);
            }
            a_next = coef<N>(sface, ka, kexp);
            s_next = s_nx;
            if (!SYM) {
                g_next = kg * sface;
                dpl = add2<N, T>(hk1, -hk);  // h_{k+1} - h_k
            }
        }
        const N b = (dtr - a_cur) + a_next;
        N d = addx<N, T>(addx<N, T>(dtr * s_cur, utk), utsk);
        if (!SYM) {
            if (k > 0) d = d + g_cur * dpl_prev;
            if (has_next) d = d + g_next * dpl;
        }
        N p = b, num = d;
        if (k > 0) {
            p = b - a_cur * cp_prev;
            num = d - a_cur * dp_prev;
        }
        const N r = recip(p);
        const N cpk = (-a_next) * r, dpk = num * r;
        const N e = (dpk - s_cur) - cpk * s_next;  // s_K = 0 (c'_{K-1} = 0)
        if (active) {
            cpb[(size_t)k * cstride + cidx] = cpk;
            if (rsave) rsave[(size_t)k * cstride + cidx] = r;
            if (DPG) po[(int64_t)k * out.sk] = to_store<T, N>(e);
            else epb[(size_t)k * cstride + cidx] = e;
        }
        cp_prev = cpk, dp_prev = dpk, e_last = e;
        if (!SYM) dpl_prev = dpl, g_cur = g_next;
        a_cur = a_next;
    };

    // utens, utens_stage of level m-1 and wcon of level m, loaded one iteration ahead
    T ut_n = T(0), uts_n = T(0), w_n = T(0), w1_n = T(0);
    T h_prev = T(0);
    N h2_prev = zero;
    for (int m = 0; m < K; ++m) {
        const T ut_k = ut_n, uts_k = uts_n, w_m = w_n, w1_m = w1_n;
        // inputs read once: streaming loads (utens_stage may be the output array, whose
        // level-m element is stored only after this value was used)
        if (m + 1 < K) {
            w_n = ld_once(pw + (int64_t)(m + 1) * wc.sk);
            if (row_end) w1_n = ld_once(pw1 + (int64_t)(m + 1) * wc.sk);
        }
        ut_n = ld_once(put + (int64_t)m * ut.sk);
        uts_n = ld_once(puts + (int64_t)m * uts.sk);
        const int slot = m % RING;
        const bool ok = mbar_wait(&full[slot], (m / RING) & 1);
        if (!__all_sync(0xffffffffu, ok)) return;  // the producers gave up (device error word set)
        const T h = H[slot * NC + tid];
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        const N h2 = twice<N, T>(h);  // s_m = 2 h_m, exact
        if (m >= 1) vstep(m - 1, true, h_prev, h, h2_prev, h2, ut_k, uts_k, w_m, w1_m);
        h_prev = h, h2_prev = h2;
    }
    vstep(K - 1, false, h_prev, T(0), h2_prev, zero, ut_n, uts_n, T(0), T(0));

    // back substitution in z = x - h; levels in groups of BG, a group's inputs loaded
    // before the previous group's outputs are stored (distinct levels, distinct addresses).
    // Without kept factors the column state is dead once read: last reads are streaming
    // loads, and the warp drops the state lines it owns whole (its 32 lanes on 32
    // consecutive columns of one row, which needs TI a multiple of 32, all in the domain,
    // the line 128-byte aligned) from L2 without a write-back.  Kept factors (rsave)
    // stay: the adjoint reads c'_k and 1/p_k later.
    const bool drop = rsave == nullptr;
    const bool own = (TI % 32 == 0) && drop && __all_sync(0xffffffffu, active);
    const size_t c0 = __shfl_sync(0xffffffffu, cidx, 0);
    constexpr int kArrays = DPG ? 1 : 2;
    constexpr int kLines = (int)(32 * sizeof(N) / 128);
    auto ld_state = [&](const N *q) -> N { return drop ? ld_once(q) : *q; };
    N z = e_last;
    if (active) st_once(po + (int64_t)(K - 1) * out.sk, to_store<T, N>(dtr * z));
    constexpr int BG = 4;
    N eq[BG], cq[BG];
    auto load_group = [&](int k0) {
#pragma unroll
        for (int q = 0; q < BG; ++q) {
            const int k = k0 - q;
            if (k < 0) break;
            eq[q] = DPG ? to_num<N, T>(po[(int64_t)k * out.sk]) : ld_state(epb + (size_t)k * cstride + cidx);
            cq[q] = ld_state(cpb + (size_t)k * cstride + cidx);
        }
    };
    if (K >= 2) load_group(K - 2);
    for (int k0 = K - 2; k0 >= 0; k0 -= BG) {
        N ec[BG], cc[BG];
#pragma unroll
        for (int q = 0; q < BG; ++q) ec[q] = eq[q], cc[q] = cq[q];
        if (k0 - BG >= 0) load_group(k0 - BG);
#pragma unroll
        for (int q = 0; q < BG; ++q) {
            const int k = k0 - q;
            if (k < 0) break;
            z = ec[q] - cc[q] * z;
            if (active) st_once(po + (int64_t)k * out.sk, to_store<T, N>(dtr * z));
        }
        if constexpr (kLines >= 1) {
            if (own) {
                __syncwarp();
                if (lane < BG * kArrays * kLines) {
                    const int m = lane % kLines, arr = (lane / kLines) % kArrays, q = lane / (kLines * kArrays);
                    const int k = k0 - q;
                    if (k >= 0) {
                        const N *row = (arr == 0 ? cpb : epb) + (size_t)k * cstride + c0;
                        const unsigned char *line = reinterpret_cast<const unsigned char *>(row) + m * 128;
                        if ((reinterpret_cast<uintptr_t>(line) & 127) == 0) discard_l2_line(line);
                    }
                }
            }
        }
    }
}

// hdiff -> vadv of one tile: PW producer warps compute h level by level into a
// shared ring, the consumer warps (fused_consumer) solve the columns from it.
template <typename T, typename N, int TI, int TJ, int PW, int STAGES, int RING, bool USE_TMA, bool DPG>
__global__ void __launch_bounds__(TI * TJ + 32 * PW)
    hdiff_vadv_kernel(const __grid_constant__ CUtensorMap tmap, const View<const T> in, const View<const T> coeff,
                      const View<const T> wc, const View<const T> ut, const View<const T> uts, const View<T> out,
                      const HdiffGeom hg, const VadvGeom g, N *__restrict__ ws, N *__restrict__ rsave,
                      N *__restrict__ ework) {
    using Lay = FusedLayout<T, TI, TJ, PW, STAGES, RING>;
    using Tile = typename Lay::Tile;
    constexpr int NC = Tile::NC, CW = Tile::CW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    T *H = reinterpret_cast<T *>(base + Lay::h_off);  // H[slot][point]
    uint64_t *tbar = reinterpret_cast<uint64_t *>(base + Lay::bar_off);
    uint64_t *full = tbar + STAGES, *empty = full + RING;

    const int tid = threadIdx.x, w = tid >> 5;
    const int ti0 = blockIdx.x * TI, tj0 = blockIdx.y * TJ;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&tbar[s], 1);
        for (int s = 0; s < RING; ++s) mbar_init(&full[s], PW), mbar_init(&empty[s], CW);
        fence_mbar_init();
    }
    __syncthreads();  // the only block-wide barrier

    if (w >= CW) {
        hdiff_producer<T, TI, TJ, PW, STAGES, USE_TMA>(&tmap, in, coeff, hg, ti0, tj0, base, Lay::x_off, Lay::l_off,
                                                       Lay::e_off, tbar, RingEmit<T>{H, full, empty, NC, RING});
        return;
    }

    // ==================================================================== consumer warps
    if (g.sym)
        fused_consumer<T, N, TI, TJ, RING, DPG, true>(wc, ut, uts, out, g, ws, rsave, ework, H, full, empty, NC, ti0,
                                                      tj0, tid);
    else
        fused_consumer<T, N, TI, TJ, RING, DPG, false>(wc, ut, uts, out, g, ws, rsave, ework, H, full, empty, NC, ti0,
                                                       tj0, tid);
}

// One step of the benchmark's two stencils on their own fields, co-scheduled:
// per CTA, the producer warps run hdiff on the 32 x BJ tile (out = hout) while
// the BJ consumer warps run the vadv column solve of the same tile
// (vadv_columns, the code of gtb_vadv's workspace form: same results, bit for
// bit).  The binary64 hdiff runs on the integer pipe and the column solve on the
// FP64 pipe, so on B300 the two overlap inside every SM.  No data passes
// between the roles; the only block-wide barrier is the initial one.
template <typename T, typename N, int BJ, int PW, int STAGES, bool USE_TMA, bool DPG>
__global__ void __launch_bounds__(32 * (BJ + PW), 7 * 4 / (BJ + PW))
    hdiff_vadv_pair_kernel(const __grid_constant__ CUtensorMap tmap, const View<const T> in,
                           const View<const T> coeff, const View<T> hout, const View<const T> us,
                           const View<const T> wc, const View<const T> up, const View<const T> ut,
                           const View<const T> uts, const View<T> out, const HdiffGeom hg, const VadvGeom g,
                           N *__restrict__ ws) {
    using Lay = FusedLayout<T, 32, BJ, PW, STAGES, 1>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t *tbar = reinterpret_cast<uint64_t *>(base + Lay::bar_off);
    const int tid = threadIdx.x, w = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&tbar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();  // the only block-wide barrier
    const int ti0 = blockIdx.x * 32, tj0 = blockIdx.y * BJ;
    if (w >= BJ) {
        hdiff_producer<T, 32, BJ, PW, STAGES, USE_TMA>(&tmap, in, coeff, hg, ti0, tj0, base, Lay::x_off, Lay::l_off,
                                                       Lay::e_off, tbar,
                                                       GlobalEmit<T>{hout, ti0, tj0, hg.I, hg.J, 32});
        return;
    }
    const size_t cstride = (size_t)g.I * g.J;
    vadv_columns<T, N, BJ, DPG, vadv_yform<T, N>(), true>(us, wc, up, ut, uts, out, g, blockIdx.x, blockIdx.y, ws,
                                                    ws + (size_t)g.K * cstride, cstride, 0, true, tid & 31, w);
}

}  // namespace gtb
