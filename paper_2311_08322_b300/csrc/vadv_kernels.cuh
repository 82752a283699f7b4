// vadv_kernels.cuh -- implicit vertical advection (GT4Py paper, Sec. 3.1):
// per (i,j) column a tridiagonal system assembled from the staggered vertical
// velocity, solved by a FORWARD elimination sweep followed by a BACKWARD
// substitution sweep (Sec. 2.2 iteration orders; the top and bottom levels are
// the specialised intervals).
//
// Mapping: one thread per column, 32 consecutive i per warp (coalesced loads
// of every level), K streamed.  The forward sweep keeps the eliminated
// coefficients c'_k and d'_k of its column in shared memory ([k][thread]
// layout, conflict-free); the backward sweep reads them back.  wcon(i+1) comes
// from the neighbouring lane by a warp shuffle, the last lane loading its own.
//
// T is the storage type, N the arithmetic type (double, float, or df =
// double-float on the FP32 pipe).
#pragma once

#include "gtb_device.cuh"
#include "hdiff_kernels.cuh"  // View

namespace gtb {

struct VadvGeom {
    int I, J, K;
    int literal;  // 1: face velocity wcon(i); 0: average of the I-faces i and i+1
    int sym;      // 1 when beta_v == 0 (explicit weights equal implicit ones)
    double dtr;   // dtr_stage
    double ka;    // a_k  = ka  * s_k  (s_k = wcon(i)+wcon(i+1), or wcon(i) when literal)
    double kas;   // as_k = kas * s_k;  c_{k-1} = -a_k, cs_{k-1} = -as_k
};

template <typename N> __device__ __forceinline__ N num_const(double c);
template <> __device__ __forceinline__ double num_const<double>(double c) { return c; }
template <> __device__ __forceinline__ float num_const<float>(double c) { return (float)c; }
template <> __device__ __forceinline__ df num_const<df>(double c) {
    const float hi = __double2float_rn(c);
    return df{hi, __double2float_rn(c - (double)hi)};
}

template <typename N, typename T> __device__ __forceinline__ N to_num(T x);
template <> __device__ __forceinline__ double to_num<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float to_num<float, float>(float x) { return x; }
template <> __device__ __forceinline__ double to_num<double, float>(float x) { return (double)x; }
template <> __device__ __forceinline__ df to_num<df, float>(float x) { return df_from(x); }

template <typename T, typename N> __device__ __forceinline__ T to_store(N x);
template <> __device__ __forceinline__ double to_store<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float to_store<float, float>(float x) { return x; }
template <> __device__ __forceinline__ float to_store<float, double>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ float to_store<float, df>(df x) { return df_to_float(x); }

// face-velocity sum s_m of level m for this lane's column (all lanes take part
// in the shuffle, so it is called warp-uniformly)
template <typename T, typename N>
__device__ __forceinline__ N face_sum(const T *__restrict__ wcol, const T *__restrict__ wcol_next, int64_t off,
                                      bool last_lane, int literal) {
    const T lo = wcol[off];
    if (literal) return to_num<N, T>(lo);
    T hi = __shfl_down_sync(0xffffffffu, lo, 1);
    if (last_lane) hi = wcol_next[off];
    return to_num<N, T>(lo) + to_num<N, T>(hi);
}

template <typename T, typename N, int BJ>
__global__ void __launch_bounds__(32 * BJ)
    vadv_kernel(const View<const T> us, const View<const T> wc, const View<const T> up, const View<const T> ut,
                const View<const T> uts, const View<T> out, const VadvGeom g) {
    constexpr int NT = 32 * BJ;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    N *cpb = reinterpret_cast<N *>(smem_raw);  // [K][NT]
    N *dpb = cpb + (size_t)g.K * NT;           // [K][NT]

    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
    const int i = blockIdx.x * 32 + tx, j = blockIdx.y * BJ + ty;
    const bool active = (i < g.I) && (j < g.J);
    const int ic = min(i, g.I - 1), jc = min(j, g.J - 1);
    const int iw = min(i, g.I);  // wcon is valid up to i = I (staggered)
    const int K = g.K;

    const T *__restrict__ pus = us.p + ic + (int64_t)jc * us.sj;
    const T *__restrict__ pup = up.p + ic + (int64_t)jc * up.sj;
    const T *__restrict__ put = ut.p + ic + (int64_t)jc * ut.sj;
    const T *puts = uts.p + ic + (int64_t)jc * uts.sj;  // may alias out (in place)
    const T *__restrict__ pw = wc.p + iw + (int64_t)jc * wc.sj;
    const T *__restrict__ pw1 = wc.p + min(i + 1, g.I) + (int64_t)jc * wc.sj;
    const bool last_lane = (tx == 31);

    const N dtr = num_const<N>(g.dtr);
    const N ka = num_const<N>(g.ka);
    const N kas = num_const<N>(g.kas);
    const N zero = num_const<N>(0.0);

    // level 0 state
    N us_prev = zero;
    N us_cur = to_num<N, T>(pus[0]);
    N a_cur = zero, as_cur = zero;  // a_0 = as_0 = 0
    N cp_prev = zero, dp_prev = zero;

#pragma unroll 2
    for (int k = 0; k < K; ++k) {
        const int64_t ok_us = (int64_t)k * us.sk;
        N us_next = zero, a_next = zero, as_next = zero;
        const bool has_next = (k + 1 < K);
        if (has_next) {
            us_next = to_num<N, T>(pus[ok_us + us.sk]);
            const N s = face_sum<T, N>(pw, pw1, (int64_t)(k + 1) * wc.sk, last_lane, g.literal);
            a_next = ka * s;
            as_next = g.sym ? a_next : kas * s;
        }
        const N c_cur = -a_next, cs_cur = -as_next;  // c_k = -a_{k+1}; zero at k = K-1
        const N b = (dtr - a_cur) - c_cur;
        N d = dtr * to_num<N, T>(pup[(int64_t)k * up.sk]) + to_num<N, T>(put[(int64_t)k * ut.sk]);
        d = d + to_num<N, T>(puts[(int64_t)k * uts.sk]);
        if (k > 0) d = d - as_cur * (us_prev - us_cur);
        if (has_next) d = d - cs_cur * (us_next - us_cur);

        N p, num;
        if (k == 0) {
            p = b;
            num = d;
        } else {
            p = b - a_cur * cp_prev;
            num = d - a_cur * dp_prev;
        }
        const N r = recip(p);
        const N cpk = c_cur * r, dpk = num * r;
        cpb[(size_t)k * NT + t] = cpk;
        dpb[(size_t)k * NT + t] = dpk;
        cp_prev = cpk, dp_prev = dpk;
        us_prev = us_cur, us_cur = us_next;
        a_cur = a_next, as_cur = as_next;
    }

    // backward substitution and output, utens_stage_out = dtr (x - u_pos)
    T *po = out.p + ic + (int64_t)jc * out.sj;
    N x = dp_prev;
    {
        const int k = K - 1;
        const N o = dtr * (x - to_num<N, T>(pup[(int64_t)k * up.sk]));
        if (active) po[(int64_t)k * out.sk] = to_store<T, N>(o);
    }
#pragma unroll 4
    for (int k = K - 2; k >= 0; --k) {
        x = dpb[(size_t)k * NT + t] - cpb[(size_t)k * NT + t] * x;
        const N o = dtr * (x - to_num<N, T>(pup[(int64_t)k * up.sk]));
        if (active) po[(int64_t)k * out.sk] = to_store<T, N>(o);
    }
}

template <typename N>
constexpr size_t vadv_smem_per_col_level() {
    return 2 * sizeof(N);
}

}  // namespace gtb
