// adjoint_kernels.cuh -- reverse-mode hdiff and vadv (the differentiation form
// of the GT4Py paper's two benchmark stencils, Sec. 3.1), and the periodic
// halo refresh used between chained steps together with its adjoint.
//
// vadv_adj: y = dtr (x - u_pos), A x = d, d = dtr u_pos + utens + utens_stage
// + E u_stage.  With A = L U (Thomas: U = (p_k, c_k), l_k = a_k / p_{k-1}) the
// transposed system A^T z = dtr y_bar is U^T v = dtr y_bar (forward sweep,
// v_k = (x_k + a_k v_{k-1}) / p_k since c_{k-1} = -a_k) then L^T z = v
// (backward sweep, z_k = v_k + c'_k z_{k+1} since l_{k+1} = -c'_k): the same
// two sweeps as the forward solve, run on the transposed factors.  Then
//   utens_bar = utens_stage_bar = z,  u_pos_bar = dtr (z - y_bar),
//   u_stage_bar_m = as_m (z_{m-1} + z_m) - as_{m+1} (z_m + z_{m+1})
// (E^T z with cs_{m-1} = -as_m; as_0 = as_K = 0).  With beta_v = 0 (as = a),
// E = dtr I - A and A^T z = dtr y_bar give u_stage_bar = dtr (z - y_bar) exactly:
// the backward sweep then reads neither wcon nor z's neighbours.
//
// hdiff_adj (gather form, one output point of in_bar per thread item, over
// the domain plus its 2-point ring): with q = coeff * out_bar on the domain
// (0 elsewhere) and the limiter's keep/zero decision recomputed from in,
//   gx(face) = keep * (q(i) - q(i+1)),  gy likewise,
//   lb(cell) = gx(i-1) - gx(i) + gy(j-1) - gy(j),
//   in_bar   = [domain] out_bar - (4 lb - lb(i+1) - lb(i-1) - lb(j+1) - lb(j-1)),
//   coeff_bar = -D * out_bar with D the forward flux divergence.
#pragma once

#include "vadv_kernels.cuh"

namespace gtb {

// ------------------------------------------------------------------ vadv adjoint
// One column's outputs after the adjoint solve, for beta_v = 0: E^T z = dtr (z - y_bar)
// makes u_stage_bar equal to u_pos_bar (their sum when merged), and utens_bar =
// utens_stage_bar = z.  The sweep runs on Z = z / dtr: Z_k = V_k + c'_k Z_{k+1}.  WANT_Z:
// a utens or utens_stage cotangent is asked for; ACC: add to the cotangent fields.
// Compile-time cases, so that no FP64 instruction of another case is issued.
template <typename T, typename N, bool WANT_Z, bool ACC>
__device__ __forceinline__ void vadv_adj_back_sym(const View<const T> &yb, const View<T> &usb, const View<T> &upb,
                                                  const View<T> &utb, const View<T> &utsb, const N *cpb, const N *vb,
                                                  size_t cstride, size_t cidx, const T *py, int K, int ic, int jc,
                                                  bool active, N dtr, bool merge_us_up) {
    auto store = [&](const View<T> &o, int k, N val) {
        if (!o.p || !active) return;
        T *q = o.p + ic + (int64_t)jc * o.sj + (int64_t)k * o.sk;
        if (ACC) *q = to_store<T, N>(to_num<N, T>(*q) + val);
        else *q = to_store<T, N>(val);
    };
    const N m = merge_us_up ? dtr + dtr : dtr;
    const N zero = num_const<N>(0.0);
    // levels in groups of G, each group's inputs loaded while the previous group is
    // computed: in binary64, with 5 FP64 operations per point, the sweep waits on memory
    // otherwise (the FP32-pipe forms are compute-bound: one level ahead)
    constexpr int G = std::is_same<N, double>::value ? 4 : 1;
    N vq[G], cq[G];
    T yq[G];
    auto load_group = [&](int k0) {  // levels k0, k0-1, ..., k0-G+1
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int k = k0 - q;
            if (k < 0) break;
            vq[q] = vb[(size_t)k * cstride + cidx];
            cq[q] = k < K - 1 ? cpb[(size_t)k * cstride + cidx] : zero;
            yq[q] = py[(int64_t)k * yb.sk];
        }
    };
    N Z1 = zero;  // Z_K = 0
    load_group(K - 1);
    for (int k0 = K - 1; k0 >= 0; k0 -= G) {
        N vc[G], cc[G];
        T yc[G];
#pragma unroll
        for (int q = 0; q < G; ++q) vc[q] = vq[q], cc[q] = cq[q], yc[q] = yq[q];
        if (k0 - G >= 0) load_group(k0 - G);
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int k = k0 - q;
            if (k < 0) break;
            const N Z = vc[q] + cc[q] * Z1;  // c'_{K-1} = 0
            if (WANT_Z) {
                const N z = dtr * Z;
                store(utb, k, z);
                store(utsb, k, z);
            }
            const N u = m * addx<N, T>(dtr * Z, -yc[q]);  // one FMA: dtr Z - y_bar
            store(usb, k, u);
            if (!merge_us_up) store(upb, k, u);
            Z1 = Z;
        }
    }
}

// FACT: the workspace holds the forward solve's factors, c'_k then 1/p_k (kept by
// gtb_hdiff_vadv with GTB_SAVE_FACTORS): the forward sweep reads them instead of
// refactorising A, and V_k overwrites 1/p_k in place.
template <typename T, typename N, int BJ, bool WS, bool FACT>
__global__ void __launch_bounds__(32 * BJ)
    vadv_adj_kernel(const View<const T> wc, const View<const T> yb, const View<T> usb, const View<T> upb,
                    const View<T> utb, const View<T> utsb, const VadvGeom g, const int accumulate,
                    const int merge_us_up, N *__restrict__ ws) {
    constexpr int NT = 32 * BJ;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
    const int i = blockIdx.x * 32 + tx, j = blockIdx.y * BJ + ty;
    const bool active = (i < g.I) && (j < g.J);
    const int ic = min(i, g.I - 1), jc = min(j, g.J - 1);
    const int ilim = g.literal ? g.I - 1 : g.I;  // last wcon column read (I-staggered unless literal)
    const int iw = min(i, ilim);
    const int K = g.K;

    N *cpb, *vb;
    size_t cstride, cidx;
    if (WS) {
        cstride = (size_t)g.I * g.J;
        cidx = (size_t)jc * g.I + ic;
        cpb = ws;
        vb = ws + (size_t)K * cstride;
    } else {
        cstride = NT;
        cidx = t;
        cpb = reinterpret_cast<N *>(smem_raw);
        vb = cpb + (size_t)K * NT;
    }
    const bool wr = WS ? active : true;

    const T *pw = wc.p + iw + (int64_t)jc * wc.sj;
    const T *pw1 = wc.p + min(i + 1, ilim) + (int64_t)jc * wc.sj;
    const T *py = yb.p + ic + (int64_t)jc * yb.sj;
    const bool last_lane = (tx == 31);
    const bool lit = g.literal != 0;
    if constexpr (kChecked) {  // every level of the column inside every field's storage
        const int64_t kl = K - 1;
        auto col = [&](const View<T> &v) {
            if (!v.p) return true;
            const T *q = v.p + ic + (int64_t)jc * v.sj;
            return in_storage(v, q, q + kl * v.sk);
        };
        bool ok = in_storage(yb, py, py + kl * yb.sk) && col(usb) && col(upb) && col(utb) && col(utsb);
        if (!FACT) ok = ok && in_storage(wc, pw, pw + kl * wc.sk) && in_storage(wc, pw1, pw1 + kl * wc.sk);
        if (!__all_sync(0xffffffffu, ok)) return;
    }

    const N dtr = num_const<N>(g.dtr);
    const N ka = num_const<N>(g.ka);
    const N kas = num_const<N>(g.kas);
    const N zero = num_const<N>(0.0);
    const int kexp = g.ka_pow2;

    // face-velocity sum from this lane's wcon(i) and, for the last lane, wcon(i+1) (warp-uniform call)
    auto face_of = [&](T lo, T hi_last) -> N {
        if (lit) return to_num<N, T>(lo);
        T hi = __shfl_down_sync(0xffffffffu, lo, 1);
        if (last_lane) hi = hi_last;
        return to_num<N, T>(lo) + to_num<N, T>(hi);
    };
    auto wload = [&](int m, T &lo, T &hi) {
        lo = pw[(int64_t)m * wc.sk];
        if (last_lane) hi = pw1[(int64_t)m * wc.sk];
    };

    // forward sweep, U^T v = dtr y_bar: (U^T v)_k = c_{k-1} v_{k-1} + p_k v_k, and with
    // v_{k-1} = u_{k-1} / p_{k-1} and c'_{k-1} = c_{k-1} / p_{k-1},
    //   v_k = u_k / p_k,   u_k = dtr y_bar_k - c'_{k-1} u_{k-1}:
    // once c' is known no a_k is needed (FACT reads no wcon).  Carried in units of dtr,
    // U = u / dtr and V = v / dtr.  Every input of level k+1 is loaded during level k.
    N cp_prev = zero, U_prev = zero;
    if constexpr (FACT) {
        // levels in groups of G, each group's inputs loaded while the previous group is
        // computed (V_k overwrites 1/p_k only after level k's group was read); binary64
        // only, as in the backward sweep
        constexpr int G = std::is_same<N, double>::value ? 4 : 1;
        T yq[G];
        N rq[G], cq[G];
        auto load_group = [&](int k0) {
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int k = k0 + q;
                if (k >= K) break;
                yq[q] = py[(int64_t)k * yb.sk];
                rq[q] = vb[(size_t)k * cstride + cidx];
                cq[q] = cpb[(size_t)k * cstride + cidx];
            }
        };
        load_group(0);
        for (int k0 = 0; k0 < K; k0 += G) {
            T yc[G];
            N rc[G], cc[G];
#pragma unroll
            for (int q = 0; q < G; ++q) yc[q] = yq[q], rc[q] = rq[q], cc[q] = cq[q];
            if (k0 + G < K) load_group(k0 + G);
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int k = k0 + q;
                if (k >= K) break;
                const N U = (k > 0) ? addx<N, T>(-(cp_prev * U_prev), yc[q]) : to_num<N, T>(yc[q]);
                if (wr) vb[(size_t)k * cstride + cidx] = U * rc[q];
                cp_prev = cc[q], U_prev = U;
            }
        }
    } else {
        N a_cur = zero;
        T y_n = py[0], w_n = T(0), w1_n = T(0);
        if (K > 1) wload(1, w_n, w1_n);
        for (int k = 0; k < K; ++k) {
            const T yk = y_n, wk1 = w_n, w1k1 = w1_n;
            if (k + 1 < K) y_n = py[(int64_t)(k + 1) * yb.sk];
            if (k + 2 < K) wload(k + 2, w_n, w1_n);
            N a_next = zero;
            if (k + 1 < K) a_next = coef<N>(face_of(wk1, w1k1), ka, kexp);
            const N b = (dtr - a_cur) + a_next;
            const N p = (k > 0) ? fms(b, a_cur, cp_prev) : b;
            const N r = recip(p);
            const N U = (k > 0) ? addx<N, T>(-(cp_prev * U_prev), yk) : to_num<N, T>(yk);
            const N cpk = (-a_next) * r;
            if (wr) {
                cpb[(size_t)k * cstride + cidx] = cpk;
                vb[(size_t)k * cstride + cidx] = U * r;
            }
            cp_prev = cpk, U_prev = U;
            a_cur = a_next;
        }
    }

    // backward sweep, L^T z = v: Z_k = V_k + c'_k Z_{k+1} (Z = z / dtr), and the outputs
    if (g.sym) {
        const bool want_z = utb.p || utsb.p;
        if (want_z) {
            if (accumulate)
                vadv_adj_back_sym<T, N, true, true>(yb, usb, upb, utb, utsb, cpb, vb, cstride, cidx, py, K, ic, jc,
                                                    active, dtr, merge_us_up);
            else
                vadv_adj_back_sym<T, N, true, false>(yb, usb, upb, utb, utsb, cpb, vb, cstride, cidx, py, K, ic, jc,
                                                     active, dtr, merge_us_up);
        } else {
            if (accumulate)
                vadv_adj_back_sym<T, N, false, true>(yb, usb, upb, utb, utsb, cpb, vb, cstride, cidx, py, K, ic, jc,
                                                     active, dtr, merge_us_up);
            else
                vadv_adj_back_sym<T, N, false, false>(yb, usb, upb, utb, utsb, cpb, vb, cstride, cidx, py, K, ic,
                                                      jc, active, dtr, merge_us_up);
        }
        return;
    }
    // general weights: u_stage_bar = E^T z, emitted for level m once z_{m-1} is known
    auto store = [&](const View<T> &o, int k, N val) {
        if (!o.p || !active) return;
        T *q = o.p + ic + (int64_t)jc * o.sj + (int64_t)k * o.sk;
        *q = accumulate ? to_store<T, N>(to_num<N, T>(*q) + val) : to_store<T, N>(val);
    };
    // carried from the previous (higher) level, so that nothing is formed or loaded twice:
    N Z1 = zero;               // Z_{k+1}
    N z1 = zero;               // z_{k+1}
    N zz1 = zero;              // z_{k+1} + z_{k+2}
    N y1 = zero;               // y_bar_{k+1}
    N as1 = zero, as2 = zero;  // as_{k+1}, as_{k+2} (as_K = 0)
    // level K-1's inputs, then each level's during the level above it
    N vb_n = vb[(size_t)(K - 1) * cstride + cidx], cp_n = zero;
    T yb_n = py[(int64_t)(K - 1) * yb.sk], wb_n = T(0), wb1_n = T(0);
    if (K - 1 > 0) wload(K - 1, wb_n, wb1_n);
    for (int k = K - 1; k >= 0; --k) {
        const N vk = vb_n, cpk = cp_n;
        const T ykr = yb_n, wk = wb_n, w1k = wb1_n;
        if (k > 0) {
            vb_n = vb[(size_t)(k - 1) * cstride + cidx];
            cp_n = cpb[(size_t)(k - 1) * cstride + cidx];
            yb_n = py[(int64_t)(k - 1) * yb.sk];
            if (k - 1 > 0) wload(k - 1, wb_n, wb1_n);
        }
        const N Z = (k == K - 1) ? vk : vk + cpk * Z1;
        const N z = dtr * Z;
        N ask = zero;
        if (k > 0) ask = kas * face_of(wk, w1k);
        const N yk = to_num<N, T>(ykr);
        store(utb, k, z);
        store(utsb, k, z);
        if (!merge_us_up) store(upb, k, dtr * (z - yk));
        const N zz = z + z1;  // z_k + z_{k+1}
        if (k + 1 < K) {      // u_stage_bar of level k+1
            const N usb1 = as1 * zz - as2 * zz1;
            // u_stage_bar and u_pos_bar as one field: level k+1 gets both
            store(usb, k + 1, merge_us_up ? usb1 + dtr * (z1 - y1) : usb1);
        }
        Z1 = Z, z1 = z, zz1 = zz, y1 = yk;
        as2 = as1, as1 = ask;
    }
    {  // level 0: as_0 = 0
        const N usb0 = -as2 * zz1;
        store(usb, 0, merge_us_up ? usb0 + dtr * (z1 - y1) : usb0);
    }
}

// ------------------------------------------------------------------ hdiff adjoint
template <typename T, int TI, int TJ>
struct HadjTile {
    // regions (tile-relative offsets of their first element)
    static constexpr int IX = TI + 6, IY = TJ + 6;   // in: tile +- 3
    static constexpr int QX = TI + 4, QY = TJ + 4;   // q, lap: tile +- 2
    static constexpr int GXX = TI + 3, GXY = TJ + 2; // x-faces: i in [-2, TI], rows tile +- 1
    static constexpr int GYX = TI + 2, GYY = TJ + 3; // y-faces: cols tile +- 1, j in [-2, TJ]
    static constexpr int LX = TI + 2, LY = TJ + 2;   // lb: tile +- 1 (kept in the q region)
    static constexpr int NF = GXX * GXY + GYX * GYY; // faces
    // slots of sizeof(T) bytes: in (binary64: or its fixed-point copy, in place), q then
    // lb, lap, face cotangents; then one keep byte per face
    static constexpr int slots = IX * IY + 2 * QX * QY + NF;
    static_assert(LX * LY <= QX * QY, "lb fits the q region");
};

template <typename T, int TI, int TJ>
constexpr int hdiff_adj_smem_bytes() {
    using H = HadjTile<T, TI, TJ>;
    return H::slots * (int)sizeof(T) + ((H::NF + 15) / 16) * 16 + 64;
}

struct HadjGeom {
    int I, J, K;
    int tiles_i, tiles_j;  // over the extended region [-2, I+2) x [-2, J+2)
    int accumulate_coeff_bar;
};

// Limiter decision of the definition, f * g > 0 (strict), taken from the signs:
// the product of two finite values is positive iff both are nonzero with equal
// signs (barring underflow of the product).
template <typename T>
__device__ __forceinline__ bool limited(T f, T g) {
    if constexpr (sizeof(T) == 8) {
        const int fh = __double2hiint(f), gh = __double2hiint(g);
        const bool fz = ((fh & 0x7FFFFFFF) | __double2loint(f)) == 0, gz = ((gh & 0x7FFFFFFF) | __double2loint(g)) == 0;
        return !fz && !gz && ((fh ^ gh) >= 0);
    } else {
        return f * g > T(0);
    }
}

// The adjoint of one tile (staged in shared memory by the caller, in the
// policy's value type V: in at tile +- 3 in S_x, q = coeff * out_bar at
// tile +- 2 in S_q) with the arithmetic of policy P: lap / limited_face / out_*.
//   faces:  keep = not (f * (in[+1] - in) > 0),  g = keep (q - q[+1])
//   lb      = (gx[i-1] - gx[i]) + (gy[j-1] - gy[j])      (cotangent of lap)
//   in_bar  = out_bar - (4 lb - sum of the 4 neighbours of lb)
//   coeff_bar = -D out_bar,  D = (fx[i] - fx[i-1]) + (fy[j] - fy[j-1]),  f = keep (lap[+1] - lap)
template <typename T, int TI, int TJ, int NT, typename P>
__device__ __forceinline__ void hdiff_adj_tile(const P &pol, typename P::V *S_x, typename P::V *S_q,
                                               unsigned char *S_keep, const View<const T> &in,
                                               const View<const T> &ob, const View<T> &ib, const View<T> &cb,
                                               const HadjGeom &g, int ti0, int tj0, int k) {
    using V = typename P::V;
    using H = HadjTile<T, TI, TJ>;
    V *S_lap = S_q + H::QX * H::QY;   // forward lap, same region as q
    V *S_gx = S_lap + H::QX * H::QY;  // x-face cotangents, faces i in [-2, TI], rows [-1, TJ]
    V *S_gy = S_gx + H::GXX * H::GXY; // y-face cotangents, cols [-1, TI], faces j in [-2, TJ]
    V *S_lb = S_q;                    // lap cotangents, tile +- 1 (q is dead by then)
    unsigned char *S_kx = S_keep, *S_ky = S_keep + H::GXX * H::GXY;
    const int tid = threadIdx.x, I = g.I, J = g.J;
    auto X = [&](int a, int b) -> V { return S_x[(a + 3) + (b + 3) * H::IX]; };  // tile-relative
    auto GIN = [&](int a, int b) -> const T * {  // the binary64 value, for exact ties
        return in.p + (ti0 + a) + (int64_t)(tj0 + b) * in.sj + (int64_t)k * in.sk;
    };
    for_cells<H::QX, H::QY, NT>(tid, [&](int idx, int ca, int cb_) {
        const int a = ca - 2, b = cb_ - 2;
        S_lap[idx] = pol.lap(X(a, b), X(a + 1, b), X(a - 1, b), X(a, b + 1), X(a, b - 1));
    });
    __syncthreads();
    auto LAP = [&](int a, int b) -> V { return S_lap[(a + 2) + (b + 2) * H::QX]; };
    auto Q = [&](int a, int b) -> V { return S_q[(a + 2) + (b + 2) * H::QX]; };
    // every face once: keep/zero from the forward values and its cotangent
    // (a face exists for domain-relative i in [-1, I-1], j in [0, J) in x, and likewise in y)
    for_cells<H::GXX, H::GXY, NT>(tid, [&](int idx, int ca, int cb_) {
        const int a = ca - 2, b = cb_ - 1;  // face between cells a and a+1, row b
        const int da = ti0 + a, db = tj0 + b;
        V gv = V(0);
        bool keep = false;
        if (da >= -1 && da <= I - 1 && db >= 0 && db < J) {
            keep = !pol.limited_face(LAP(a + 1, b) - LAP(a, b), X(a + 1, b), X(a, b), GIN(a + 1, b), GIN(a, b));
            if (keep) gv = Q(a, b) - Q(a + 1, b);
        }
        S_gx[idx] = gv;
        S_kx[idx] = keep;
    });
    for_cells<H::GYX, H::GYY, NT>(tid, [&](int idx, int ca, int cb_) {
        const int a = ca - 1, b = cb_ - 2;  // face between rows b and b+1, column a
        const int da = ti0 + a, db = tj0 + b;
        V gv = V(0);
        bool keep = false;
        if (da >= 0 && da < I && db >= -1 && db <= J - 1) {
            keep = !pol.limited_face(LAP(a, b + 1) - LAP(a, b), X(a, b + 1), X(a, b), GIN(a, b + 1), GIN(a, b));
            if (keep) gv = Q(a, b) - Q(a, b + 1);
        }
        S_gy[idx] = gv;
        S_ky[idx] = keep;
    });
    __syncthreads();
    auto GX = [&](int a, int b) -> V { return S_gx[(a + 2) + (b + 1) * H::GXX]; };
    auto GY = [&](int a, int b) -> V { return S_gy[(a + 1) + (b + 2) * H::GYX]; };
    for_cells<H::LX, H::LY, NT>(tid, [&](int idx, int ca, int cb_) {
        const int a = ca - 1, b = cb_ - 1;
        S_lb[idx] = (GX(a - 1, b) - GX(a, b)) + (GY(a, b - 1) - GY(a, b));
    });
    __syncthreads();
    auto LB = [&](int a, int b) -> V { return S_lb[(a + 1) + (b + 1) * H::LX]; };
    auto FX = [&](int a, int b) -> V {  // forward x-flux of face (a, a+1) in row b, 0 where limited
        return S_kx[(a + 2) + (b + 1) * H::GXX] ? LAP(a + 1, b) - LAP(a, b) : V(0);
    };
    auto FY = [&](int a, int b) -> V {
        return S_ky[(a + 1) + (b + 2) * H::GYX] ? LAP(a, b + 1) - LAP(a, b) : V(0);
    };
    for_cells<TI, TJ, NT>(tid, [&](int idx, int a, int b) {
        const int da = ti0 + a, db = tj0 + b;
        if (da < -2 || da >= I + 2 || db < -2 || db >= J + 2) return;
        const V tr = pol.lap(LB(a, b), LB(a + 1, b), LB(a - 1, b), LB(a, b + 1), LB(a, b - 1));
        const bool dom = da >= 0 && da < I && db >= 0 && db < J;
        const T *po = ob.p + da + (int64_t)db * ob.sj + (int64_t)k * ob.sk;
        T *pi = ib.p + da + (int64_t)db * ib.sj + (int64_t)k * ib.sk;
        if (kChecked && !(in_storage(ib, pi, pi) && (!dom || in_storage(ob, po, po)))) return;
        const T o = dom ? *po : T(0);
        *pi = o - pol.out_q(tr);
        if (cb.p && dom) {
            const T D = pol.out_in((FX(a, b) - FX(a - 1, b)) + (FY(a, b) - FY(a, b - 1)));
            T *c = cb.p + da + (int64_t)db * cb.sj + (int64_t)k * cb.sk;
            if (kChecked && !in_storage(cb, c, c)) return;
            *c = g.accumulate_coeff_bar ? *c - D * o : -D * o;
        }
    });
}

// The definition in the storage type.
template <typename T>
struct AdjNative {
    using V = T;
    __device__ __forceinline__ V lap(V c, V e, V w, V n, V s) const { return T(4) * c - (((e + w) + n) + s); }
    __device__ __forceinline__ bool limited_face(V f, V x1, V x0, const T *, const T *) const {
        return limited(f, x1 - x0);
    }
    __device__ __forceinline__ T out_q(V v) const { return v; }
    __device__ __forceinline__ T out_in(V v) const { return v; }
};

// Binary64 in exact int64 fixed point (the form of the forward kernels): in with
// scale Ein, q with scale Eq (converted when the tile is staged);
// every add and subtract exact, the limiter takes the exact signs (the binary64
// inputs are read back only when two cells truncate alike); the two outputs are
// rounded once each on the way back.
struct AdjFixed {
    using V = int64_t;
    int Ein, Eq;
    __device__ __forceinline__ V lap(V c, V e, V w, V n, V s) const { return 4 * c - (((e + w) + n) + s); }
    __device__ __forceinline__ bool limited_face(V f, V x1, V x0, const double *p1, const double *p0) const {
        const int gsign = x1 != x0 ? (x1 > x0 ? 1 : -1) : exact_dir(x1, x0, *p1, *p0);
        return (f > 0 && gsign > 0) || (f < 0 && gsign < 0);
    }
    __device__ __forceinline__ double out_q(V v) const { return from_fixed(v, Eq); }
    __device__ __forceinline__ double out_in(V v) const { return from_fixed(v, Ein); }
};

template <typename T, int TI, int TJ, int NT>
__global__ void __launch_bounds__(NT)
    hdiff_adj_kernel(const View<const T> in, const View<const T> coeff, const View<const T> ob, const View<T> ib,
                     const View<T> cb, const HadjGeom g) {
    using H = HadjTile<T, TI, TJ>;
    constexpr bool FIX = sizeof(T) == 8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *S_in = reinterpret_cast<T *>(smem_raw);  // in at tile (-3..TI+2, -3..TJ+2)
    T *S_q = S_in + H::IX * H::IY;              // q at tile (-2..TI+1, -2..TJ+1), then the rest
    unsigned char *S_keep = smem_raw + H::slots * sizeof(T);
    __shared__ unsigned s_e[NT / 32][4];

    const int tid = threadIdx.x;
    const int ti0 = (blockIdx.x % g.tiles_i) * TI - 2;  // domain-relative i of tile column 0
    const int tj0 = (blockIdx.x / g.tiles_i) * TJ - 2;
    const int k = blockIdx.y;
    const int I = g.I, J = g.J;

    // Staging by asynchronous element copies (every copy of the block in flight at once,
    // no register round trip): in on the cells the forward definition reads, coeff and
    // out_bar on the domain cells of the q box, zero-filled elsewhere (including the
    // unread halo corners).  out_bar lands in the Laplacian region, written only after
    // the staging.  Each thread copies the cells tid + c NT and reads back only those.
    constexpr int CI = (H::IX * H::IY + NT - 1) / NT, CQ = (H::QX * H::QY + NT - 1) / NT;
    T *S_ob = S_q + H::QX * H::QY;
    {
        int ca = tid % H::IX, cb_ = tid / H::IX;  // cell coordinates, stepped by NT
#pragma unroll
        for (int c = 0; c < CI; ++c) {
            const int idx = tid + c * NT;
            if (idx >= H::IX * H::IY) break;
            const int a = ti0 - 3 + ca, b = tj0 - 3 + cb_;
            bool rd = hdiff_reads(a, b, I, J);
            const T *src = rd ? in.p + a + (int64_t)b * in.sj + (int64_t)k * in.sk : in.p;
            if (kChecked && rd) rd = in_storage(in, src, src);
            cp_async_elem(S_in + idx, rd ? src : in.p, rd);
            ca += NT % H::IX, cb_ += NT / H::IX;
            if (ca >= H::IX) ca -= H::IX, ++cb_;
        }
    }
    {
        int ca = tid % H::QX, cb_ = tid / H::QX;
#pragma unroll
        for (int c = 0; c < CQ; ++c) {
            const int idx = tid + c * NT;
            if (idx >= H::QX * H::QY) break;
            const int a = ti0 - 2 + ca, b = tj0 - 2 + cb_;
            bool dom = a >= 0 && a < I && b >= 0 && b < J;
            const T *sc = dom ? coeff.p + a + (int64_t)b * coeff.sj + (int64_t)k * coeff.sk : coeff.p;
            const T *so = dom ? ob.p + a + (int64_t)b * ob.sj + (int64_t)k * ob.sk : ob.p;
            if (kChecked && dom) dom = in_storage(coeff, sc, sc) && in_storage(ob, so, so);
            cp_async_elem(S_q + idx, dom ? sc : coeff.p, dom);
            cp_async_elem(S_ob + idx, dom ? so : ob.p, dom);
            ca += NT % H::QX, cb_ += NT / H::QX;
            if (ca >= H::QX) ca -= H::QX, ++cb_;
        }
    }
    cp_async_wait_all();

    // in, and q = coeff * out_bar, of this thread's cells in registers until the tile's
    // scales are known
    T vin[CI], vq[CQ];
    unsigned ein = 0, eq = 0, qnz = 0, inz = 0;
#pragma unroll
    for (int c = 0; c < CI; ++c) {
        const int idx = tid + c * NT;
        const T v = idx < H::IX * H::IY ? S_in[idx] : T(0);
        vin[c] = v;
        if constexpr (FIX) {
            ein = max(ein, ((unsigned)__double2hiint(v) >> 20) & 0x7FFu);
            inz |= (unsigned)((__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll) != 0);
        }
    }
#pragma unroll
    for (int c = 0; c < CQ; ++c) {
        const int idx = tid + c * NT;
        const T v = idx < H::QX * H::QY ? S_q[idx] * S_ob[idx] : T(0);  // zero-filled off the domain
        vq[c] = v;
        if constexpr (FIX) {
            eq = max(eq, ((unsigned)__double2hiint(v) >> 20) & 0x7FFu);
            qnz |= (unsigned)((__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll) != 0);
        }
    }
    bool fixed = false;
    if constexpr (FIX) {
        ein = __reduce_max_sync(0xffffffffu, ein);
        eq = __reduce_max_sync(0xffffffffu, eq);
        qnz = __reduce_or_sync(0xffffffffu, qnz);
        inz = __reduce_or_sync(0xffffffffu, inz);
        if ((tid & 31) == 0)
            s_e[tid >> 5][0] = ein, s_e[tid >> 5][1] = eq, s_e[tid >> 5][2] = qnz, s_e[tid >> 5][3] = inz;
        __syncthreads();
        ein = eq = qnz = inz = 0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w)
            ein = max(ein, s_e[w][0]), eq = max(eq, s_e[w][1]), qnz |= s_e[w][2], inz |= s_e[w][3];
        // a field that is zero on the whole tile converts exactly at any scale
        if (ein == 0 && !inz) ein = 64;
        if (eq == 0 && !qnz) eq = 64;
        fixed = ein >= 64 && ein <= 2040 && eq >= 64 && eq <= 2040;
    }
    // stage the tile: fixed point straight from the registers, or the values themselves
#pragma unroll
    for (int c = 0; c < CI; ++c) {
        const int idx = tid + c * NT;
        if (idx >= H::IX * H::IY) break;
        if constexpr (FIX) {
            if (fixed) reinterpret_cast<int64_t *>(S_in)[idx] = to_fixed(vin[c], (int)ein);
            else S_in[idx] = vin[c];
        } else {
            S_in[idx] = vin[c];
        }
    }
#pragma unroll
    for (int c = 0; c < CQ; ++c) {
        const int idx = tid + c * NT;
        if (idx >= H::QX * H::QY) break;
        if constexpr (FIX) {
            if (fixed) reinterpret_cast<int64_t *>(S_q)[idx] = to_fixed(vq[c], (int)eq);
            else S_q[idx] = vq[c];
        } else {
            S_q[idx] = vq[c];
        }
    }
    __syncthreads();
    if constexpr (FIX) {
        if (fixed) {
            hdiff_adj_tile<T, TI, TJ, NT>(AdjFixed{(int)ein, (int)eq}, reinterpret_cast<int64_t *>(S_in),
                                          reinterpret_cast<int64_t *>(S_q), S_keep, in, ob, ib, cb, g, ti0, tj0, k);
            return;
        }
    }
    hdiff_adj_tile<T, TI, TJ, NT>(AdjNative<T>{}, S_in, S_q, S_keep, in, ob, ib, cb, g, ti0, tj0, k);
}

// ------------------------------------------------------------------ periodic halo
// Fill the hi-wide I halo and hj-wide J halo around the domain with the
// periodic continuation of the domain (corners included).
template <typename T>
__global__ void halo_periodic_kernel(const View<T> f, int I, int J, int K, int hi, int hj) {
    const int W = I + 2 * hi, H = J + 2 * hj;
    const int64_t n = (int64_t)W * H * K;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx % W) - hi, b = (int)((idx / W) % H) - hj, k = (int)(idx / ((int64_t)W * H));
        if (a >= 0 && a < I && b >= 0 && b < J) continue;
        const int sa = (a + I) % I, sb = (b + J) % J;
        T *dst = f.p + a + (int64_t)b * f.sj + (int64_t)k * f.sk;
        const T *src = f.p + sa + (int64_t)sb * f.sj + (int64_t)k * f.sk;
        if (kChecked && !(in_storage(f, dst, dst) && in_storage(f, src, src))) continue;
        *dst = *src;
    }
}

// Adjoint of the refresh: every domain point gathers the cotangents of the halo
// points that copied it (halo widths <= I, J, so each halo point maps to one
// domain point); the halo itself is left unchanged.  Only the band of domain
// points within hi (hj) of an edge receives anything, so the launch covers
// that band: its rows j < hj or j >= J-hj in full, and the first and last hi
// columns of the other rows.
template <typename T>
__global__ void halo_periodic_adj_kernel(const View<T> f, int I, int J, int K, int hi, int hj) {
    const int rows_full = min(J, 2 * hj);             // rows taken in full
    const int mid_rows = J - rows_full;               // rows of which only 2*hi edge columns count
    const int cols_edge = min(I, 2 * hi);
    const int64_t per_level = (int64_t)rows_full * I + (int64_t)mid_rows * cols_edge;
    const int64_t n = per_level * K;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(idx / per_level);
        int64_t r = idx % per_level;
        int a, b;
        if (r < (int64_t)rows_full * I) {
            const int rr = (int)(r / I);
            a = (int)(r % I);
            b = rr < hj ? rr : J - rows_full + rr;  // top hj rows, then the bottom ones
            if (rows_full < 2 * hj) b = rr;         // J < 2 hj: every row is full
        } else {
            r -= (int64_t)rows_full * I;
            const int cc = (int)(r % cols_edge);
            b = hj + (int)(r / cols_edge);
            a = cc < hi ? cc : I - cols_edge + cc;
            if (cols_edge < 2 * hi) a = cc;
        }
        T acc = T(0);
#pragma unroll
        for (int sa = -1; sa <= 1; ++sa)
#pragma unroll
            for (int sb = -1; sb <= 1; ++sb) {
                if (sa == 0 && sb == 0) continue;
                const int x = a + sa * I, y = b + sb * J;
                if (x >= -hi && x < I + hi && y >= -hj && y < J + hj && !(x >= 0 && x < I && y >= 0 && y < J)) {
                    const T *src = f.p + x + (int64_t)y * f.sj + (int64_t)k * f.sk;
                    if (!kChecked || in_storage(f, src, src)) acc += *src;
                }
            }
        T *dst = f.p + a + (int64_t)b * f.sj + (int64_t)k * f.sk;
        if (!kChecked || in_storage(f, dst, dst)) *dst += acc;
    }
}

}  // namespace gtb
