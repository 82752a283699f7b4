// fused_kernels.cuh -- hdiff feeding vadv in one kernel (the two stencils of
// the GT4Py paper, Sec. 3.1, chained as h = hdiff(in, coeff),
// utens_stage_out = vadv(u_stage = h, u_pos = h, utens, utens_stage, wcon);
// Sec. 2.2 leaves the backend free to fuse the computations it runs).  h is
// produced level by level inside the SM and consumed there: it is never
// written to memory.
//
// CTA = a 32 x BJ block of columns, all K levels, warp-specialised:
//   * BJ consumer warps (lane = i, warp = j), one thread per column: the
//     column's forward elimination step of level m-1 as soon as h_m is ready,
//     then the back substitution (the FP64- or FP32-pipe bound part);
//   * one producer warp: per level the (32+4) x (BJ+4) box of `in` arrives by
//     TMA (STAGES-deep ring); binary64 storage converts it to exact int64 fixed
//     point (the form of hdiff_rs: E = the largest exponent among the cells the
//     block's outputs read; a level whose E leaves [64, 2040] uses the
//     definition in binary64), forms the Laplacian on (32+2) x (BJ+2) cells,
//     the limited fluxes and h of the BJ x 32 columns into a RING-deep shared
//     ring (the integer-pipe bound part).
// The two sides meet only through the ring's full / empty mbarriers (bounded
// waits), so the producer runs up to RING levels ahead and the consumers never
// wait on a block barrier.
// The back substitution runs on the shifted unknown z = x - h (u_pos = h), so
// that h is not needed after the forward sweep:
//   e_k = (d'_k - h_k) - c'_k h_{k+1},   z_{K-1} = e_{K-1},
//   z_k = e_k - c'_k z_{k+1},            utens_stage_out_k = dtr z_k,
// the same unknowns as x_k - h_k of the Thomas solution (a different rounding
// order than dtr (x_k - u_pos_k)).  c'_k goes to the caller's workspace, e_k is
// parked in the output array (or in the workspace when the arithmetic type is
// wider than the storage type).
#pragma once

#include "hdiff_rs.cuh"
#include "vadv_kernels.cuh"

namespace gtb {

template <typename T, int BJ, int STAGES, int RING>
struct FusedLayout {
    using Tile = RsTile<T, 1, BJ, 1>;           // 32 x BJ columns; box (32+4+align) x (BJ+4)
    static constexpr int XW = 36, XH = BJ + 4;  // fixed-point cells: columns -2..33, rows -2..BJ+1
    static constexpr int LW = 34, LH = BJ + 2;  // Laplacian cells: columns -1..32, rows -1..BJ
    static constexpr int x_off = STAGES * Tile::stage_stride;
    static constexpr int l_off = x_off + XW * XH * 8;
    static constexpr int h_off = l_off + LW * LH * 8;
    static constexpr int bar_off = h_off + ((RING * BJ * 32 * (int)sizeof(T) + 7) / 8) * 8;
    static constexpr int bytes = bar_off + (STAGES + 2 * RING) * 8;
    static constexpr int smem_bytes = bytes + 128;  // + slack for the 128-byte base alignment
};

// Cells of one level's box, tile-relative (ci, cj) with ci in [-2, 33], cj in [-2, BJ+1].
template <typename T, typename V, int BJ, bool FIXED>
struct FusedCells {
    const T *S;  // the TMA box: cell (ci, cj) at S[(cj+2)*BX + ci+2+xs]
    const V *X;  // fixed point: X[(cj+2)*36 + ci+2]; unused for the definition
    const V *L;  // Laplacian: L[(lj+1)*34 + li+1]
    int xs;
    static constexpr int BX = RsTile<T, 1, BJ, 1>::BX;
    __device__ __forceinline__ const T *sp(int ci, int cj) const { return S + (cj + 2) * BX + ci + 2 + xs; }
    __device__ __forceinline__ V x(int ci, int cj) const {
        if constexpr (FIXED) return X[(cj + 2) * 36 + ci + 2];
        else return *sp(ci, cj);
    }
    __device__ __forceinline__ V lap(int li, int lj) const { return L[(lj + 1) * 34 + li + 1]; }
};

// The producer warp's level with policy P (FixedF64 or Native<T>): Laplacians
// into Lw, then h of column `lane` in the BJ rows into hrow[r * 32 + lane].
template <int BJ, typename P, typename C, typename T>
__device__ __forceinline__ void fused_hdiff_level(const P &pol, const C &c, typename P::V *Lw, const T (&cf)[BJ],
                                                  T *hrow) {
    using V = typename P::V;
    const int lane = threadIdx.x & 31;
    for (int idx = lane; idx < 34 * (BJ + 2); idx += 32) {
        const int li = idx % 34 - 1, lj = idx / 34 - 1;
        Lw[idx] = pol.lap(c.x(li, lj), c.x(li + 1, lj), c.x(li - 1, lj), c.x(li, lj + 1), c.x(li, lj - 1));
    }
    __syncwarp();
    const int ci = lane;
#pragma unroll
    for (int cj = 0; cj < BJ; ++cj) {
        const V x0 = c.x(ci, cj), l0 = c.lap(ci, cj);
        const V fxe = pol.limit(c.lap(ci + 1, cj) - l0, pol.grad(c.x(ci + 1, cj), x0, c.sp(ci + 1, cj), c.sp(ci, cj)));
        const V fxw = pol.limit(l0 - c.lap(ci - 1, cj), pol.grad(x0, c.x(ci - 1, cj), c.sp(ci, cj), c.sp(ci - 1, cj)));
        const V fyn = pol.limit(c.lap(ci, cj + 1) - l0, pol.grad(c.x(ci, cj + 1), x0, c.sp(ci, cj + 1), c.sp(ci, cj)));
        const V fys = pol.limit(l0 - c.lap(ci, cj - 1), pol.grad(x0, c.x(ci, cj - 1), c.sp(ci, cj), c.sp(ci, cj - 1)));
        const V D = (fxe - fxw) + (fyn - fys);
        hrow[cj * 32 + lane] = pol.out(*c.sp(ci, cj), cf[cj], D);
    }
}

template <typename T, typename N, int BJ, int STAGES, int RING, bool USE_TMA, bool DPG>
__global__ void __launch_bounds__(32 * (BJ + 1))
    hdiff_vadv_kernel(const __grid_constant__ CUtensorMap tmap, const View<const T> in, const View<const T> coeff,
                      const View<const T> wc, const View<const T> ut, const View<const T> uts, const View<T> out,
                      const HdiffGeom hg, const VadvGeom g, N *__restrict__ ws) {
    using Lay = FusedLayout<T, BJ, STAGES, RING>;
    using Tile = typename Lay::Tile;
    constexpr bool FIX = sizeof(T) == 8;  // binary64 storage: exact fixed-point hdiff
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    T *H = reinterpret_cast<T *>(base + Lay::h_off);  // H[slot][row][lane]
    uint64_t *tbar = reinterpret_cast<uint64_t *>(base + Lay::bar_off);
    uint64_t *full = tbar + STAGES, *empty = full + RING;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int ti0 = blockIdx.x * 32, tj0 = blockIdx.y * BJ;
    const int I = g.I, J = g.J, K = g.K;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&tbar[s], 1);
        for (int s = 0; s < RING; ++s) mbar_init(&full[s], 1), mbar_init(&empty[s], BJ);
        fence_mbar_init();
    }
    __syncthreads();  // the only block-wide barrier

    if (w == BJ) {
        // ================================================================ producer warp
        int64_t *Xs = reinterpret_cast<int64_t *>(base + Lay::x_off);
        unsigned char *Lraw = base + Lay::l_off;
        const int xs = hg.xs;
        if (USE_TMA && lane == 0) {
            prefetch_tensormap(&tmap);
            for (int p = 0; p < STAGES && p < K; ++p) {
                mbar_arrive_expect_tx(&tbar[p], Tile::box_bytes);
                tma_load_3d(base + p * Tile::stage_stride, &tmap, &tbar[p], hg.X0 + ti0, hg.Y0 + tj0, hg.Z0 + p);
            }
        }
        // coeff of this lane's column in the BJ rows, one level ahead
        const int ic = min(ti0 + lane, I - 1);
        const T *pcf[BJ];
        T cf_n[BJ];
#pragma unroll
        for (int r = 0; r < BJ; ++r) {
            pcf[r] = coeff.p + ic + (int64_t)min(tj0 + r, J - 1) * coeff.sj;
            cf_n[r] = pcf[r][0];
        }
        bool failed = false;
        for (int m = 0; m < K; ++m) {
            T cf[BJ];
#pragma unroll
            for (int r = 0; r < BJ; ++r) {
                cf[r] = cf_n[r];
                if (m + 1 < K) cf_n[r] = pcf[r][(int64_t)(m + 1) * coeff.sk];
            }
            const int s = USE_TMA ? m % STAGES : 0;
            const T *S = reinterpret_cast<const T *>(base + s * Tile::stage_stride);
            if (USE_TMA) {
                if (!mbar_wait(&tbar[s], (m / STAGES) & 1)) failed = true;
            } else {
                T *D = reinterpret_cast<T *>(base);
                for (int idx = lane; idx < Tile::box_elems; idx += 32) {
                    const int bx = idx % Tile::BX, by = idx / Tile::BX;
                    const int gi = ti0 - 2 + bx, gj = tj0 - 2 + by;
                    T v = T(0);
                    if (gi >= -2 && gi < I + 2 && gj >= -2 && gj < J + 2)
                        v = in.p[(int64_t)gi + (int64_t)gj * in.sj + (int64_t)m * in.sk];
                    D[idx] = v;
                }
                __syncwarp();
            }
            if (__any_sync(0xffffffffu, failed)) break;
            bool fixed = false;
            int E = 0;
            if constexpr (FIX) {
                // largest exponent among the cells the block's outputs read
                unsigned emax = 0;
                for (int idx = lane; idx < 36 * (BJ + 4); idx += 32) {
                    const int ci = idx % 36 - 2, cj = idx / 36 - 2;
                    if (!hdiff_reads(ti0 + ci, tj0 + cj, I, J)) continue;
                    emax = max(emax, ((unsigned)__double2hiint(S[(cj + 2) * Tile::BX + ci + 2 + xs]) >> 20) & 0x7FFu);
                }
                E = (int)__reduce_max_sync(0xffffffffu, emax);
                fixed = (E >= 64 && E <= 2040);
                if (fixed) {
                    for (int idx = lane; idx < 36 * (BJ + 4); idx += 32) {
                        const int ci = idx % 36 - 2, cj = idx / 36 - 2;
                        Xs[idx] = to_fixed(S[(cj + 2) * Tile::BX + ci + 2 + xs], E);
                    }
                    __syncwarp();
                }
            }
            // the ring slot must have been consumed (level m - RING)
            const int slot = m % RING;
            if (m >= RING && !mbar_wait(&empty[slot], ((m / RING) - 1) & 1)) failed = true;
            if (__any_sync(0xffffffffu, failed)) break;
            T *hrow = H + slot * BJ * 32;
            bool done = false;
            if constexpr (FIX) {
                if (fixed) {
                    const FusedCells<T, int64_t, BJ, true> c{S, Xs, reinterpret_cast<const int64_t *>(Lraw), xs};
                    fused_hdiff_level<BJ>(FixedF64{E}, c, reinterpret_cast<int64_t *>(Lraw), cf, hrow);
                    done = true;
                }
            }
            if (!done) {
                const FusedCells<T, T, BJ, false> c{S, nullptr, reinterpret_cast<const T *>(Lraw), xs};
                fused_hdiff_level<BJ>(Native<T>{}, c, reinterpret_cast<T *>(Lraw), cf, hrow);
            }
            __syncwarp();  // h written and the box, X and L read by every lane
            if (lane == 0) {
                mbar_arrive(&full[slot]);
                if (USE_TMA && m + STAGES < K) {
                    mbar_arrive_expect_tx(&tbar[s], Tile::box_bytes);
                    tma_load_3d(base + s * Tile::stage_stride, &tmap, &tbar[s], hg.X0 + ti0, hg.Y0 + tj0,
                                hg.Z0 + m + STAGES);
                }
            }
        }
        if (USE_TMA && failed && lane == 0)  // let the box loads in flight land before leaving
            for (int s = 0; s < STAGES; ++s) mbar_wait(&tbar[s], 0), mbar_wait(&tbar[s], 1);
        return;
    }

    // ==================================================================== consumer warps
    const int i = ti0 + lane, j = tj0 + w;
    const bool active = (i < I) && (j < J);
    const int ilim = g.literal ? I - 1 : I;  // last wcon column read (I-staggered unless literal)
    const int ic = min(i, I - 1), jc = min(j, J - 1), iw = min(i, ilim);
    const T *put = ut.p + ic + (int64_t)jc * ut.sj;
    const T *puts = uts.p + ic + (int64_t)jc * uts.sj;  // may alias po (in place)
    const T *pw = wc.p + iw + (int64_t)jc * wc.sj;
    const T *pw1 = wc.p + min(i + 1, ilim) + (int64_t)jc * wc.sj;
    T *po = out.p + ic + (int64_t)jc * out.sj;
    const size_t cstride = (size_t)I * J, cidx = (size_t)jc * I + ic;
    N *cpb = ws;
    N *epb = ws + (size_t)K * cstride;  // e_k when it is not parked in the output
    const bool last_lane = (lane == 31);
    const bool lit = g.literal != 0;

    const N dtr = num_const<N>(g.dtr);
    const N ka = num_const<N>(g.ka);
    const N kas = num_const<N>(g.kas);
    const N zero = num_const<N>(0.0);
    const int kexp = g.ka_pow2;

    N dm = zero, a_cur = zero, as_cur = zero, cp_prev = zero, dp_prev = zero, e_last = zero;

    // forward elimination step of level k; hk = u_stage_k = u_pos_k, hk1 = u_stage_{k+1}
    auto vstep = [&](int k, bool has_next, T hk, T hk1, T utk, T utsk, T wk1, T w1k1) {
        N a_next = zero, as_next = zero, dpl = zero;
        if (has_next) {
            N sface;
            if (lit) {
                sface = to_num<N, T>(wk1);
            } else {
                T hi = __shfl_down_sync(0xffffffffu, wk1, 1);
                if (last_lane) hi = w1k1;
                sface = add2<N, T>(wk1, hi);
            }
            a_next = coef<N>(sface, ka, kexp);
            as_next = g.sym ? a_next : kas * sface;
            dpl = add2<N, T>(hk1, -hk);  // u_stage_{k+1} - u_stage_k
        }
        const N b = (dtr - a_cur) + a_next;
        N d = addx<N, T>(mulx<N, T>(dtr, hk), utk);
        d = addx<N, T>(d, utsk);
        if (k > 0) d = d - as_cur * dm;
        if (has_next) d = d + as_next * dpl;
        N p = b, num = d;
        if (k > 0) {
            p = b - a_cur * cp_prev;
            num = d - a_cur * dp_prev;
        }
        const N r = recip(p);
        const N cpk = (-a_next) * r, dpk = num * r;
        N e = addx<N, T>(dpk, -hk);
        if (has_next) e = e - mulx<N, T>(cpk, hk1);
        if (active) {
            cpb[(size_t)k * cstride + cidx] = cpk;
            if (DPG) po[(int64_t)k * out.sk] = to_store<T, N>(e);
            else epb[(size_t)k * cstride + cidx] = e;
        }
        cp_prev = cpk, dp_prev = dpk, e_last = e;
        dm = -dpl;
        a_cur = a_next, as_cur = as_next;
    };

    // utens, utens_stage of level m-1 and wcon of level m, loaded one iteration ahead
    T ut_n = T(0), uts_n = T(0), w_n = T(0), w1_n = T(0);
    T h_prev = T(0);
    for (int m = 0; m < K; ++m) {
        const T ut_k = ut_n, uts_k = uts_n, w_m = w_n, w1_m = w1_n;
        if (m + 1 < K) {
            w_n = pw[(int64_t)(m + 1) * wc.sk];
            if (last_lane) w1_n = pw1[(int64_t)(m + 1) * wc.sk];
        }
        ut_n = put[(int64_t)m * ut.sk];
        uts_n = puts[(int64_t)m * uts.sk];
        const int slot = m % RING;
        const bool ok = mbar_wait(&full[slot], (m / RING) & 1);
        if (!__all_sync(0xffffffffu, ok)) return;  // the producer gave up (device error word set)
        const T h = H[(slot * BJ + w) * 32 + lane];
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (m >= 1) vstep(m - 1, true, h_prev, h, ut_k, uts_k, w_m, w1_m);
        h_prev = h;
    }
    vstep(K - 1, false, h_prev, T(0), ut_n, uts_n, T(0), T(0));

    // back substitution in z = x - h
    if (active) {
        N z = e_last;
        po[(int64_t)(K - 1) * out.sk] = to_store<T, N>(dtr * z);
#pragma unroll 4
        for (int k = K - 2; k >= 0; --k) {
            const N ek = DPG ? to_num<N, T>(po[(int64_t)k * out.sk]) : epb[(size_t)k * cstride + cidx];
            z = ek - cpb[(size_t)k * cstride + cidx] * z;
            po[(int64_t)k * out.sk] = to_store<T, N>(dtr * z);
        }
    }
}

}  // namespace gtb
