// vadv_kernels.cuh -- implicit vertical advection (GT4Py paper, Sec. 3.1):
// per (i,j) column a tridiagonal system assembled from the staggered vertical
// velocity, solved by a FORWARD elimination sweep followed by a BACKWARD
// substitution sweep (Sec. 2.2 iteration orders; the top and bottom levels are
// the specialised intervals).
//
// Mapping: one thread per column, 32 consecutive i per warp (coalesced loads
// of every level), K streamed, inputs loaded one level ahead.  The forward sweep
// keeps the eliminated coefficient c'_k and the back-substitution term e_k of
// its column (vadv_columns_t) in shared memory ([k][thread] layout,
// conflict-free) or a workspace; the backward sweep reads them back.  wcon(i+1) comes
// from the neighbouring lane by a warp shuffle, the last lane loading its own.
//
// T is the storage type, N the arithmetic type (double, float, or df =
// double-float on the FP32 pipe).
#pragma once

#include <type_traits>

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
    double kg;    // kas - ka: the explicit-minus-implicit weight, zero when sym
    int ka_pow2;  // n < 0 when ka = -2^n exactly (a_k is then an exponent shift), else 0
};

// Two columns per thread: fpair storage (two binary32 columns) with dfpair arithmetic.
template <typename T>
__host__ __device__ constexpr bool is_pair() { return std::is_same<T, fpair>::value; }
// double-float arithmetic, one column or two per thread
template <typename N>
__host__ __device__ constexpr bool is_df() { return std::is_same<N, df>::value || std::is_same<N, dfpair>::value; }

template <typename N> __device__ __forceinline__ N num_const(double c);
template <> __device__ __forceinline__ double num_const<double>(double c) { return c; }
template <> __device__ __forceinline__ float num_const<float>(double c) { return (float)c; }
template <> __device__ __forceinline__ df num_const<df>(double c) {
    const float hi = __double2float_rn(c);
    return df{hi, __double2float_rn(c - (double)hi)};
}
template <> __device__ __forceinline__ dfpair num_const<dfpair>(double c) {
    const df d = num_const<df>(c);
    return dfpair{fp_splat(d.hi), fp_splat(d.lo)};
}

template <typename N, typename T> __device__ __forceinline__ N to_num(T x);
template <> __device__ __forceinline__ double to_num<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float to_num<float, float>(float x) { return x; }
template <> __device__ __forceinline__ double to_num<double, float>(float x) { return (double)x; }
template <> __device__ __forceinline__ df to_num<df, float>(float x) { return df_from(x); }
template <> __device__ __forceinline__ dfpair to_num<dfpair, fpair>(fpair x) { return dfpair{x, fp_zero()}; }

template <typename T, typename N> __device__ __forceinline__ T to_store(N x);
template <> __device__ __forceinline__ double to_store<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float to_store<float, float>(float x) { return x; }
template <> __device__ __forceinline__ float to_store<float, double>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ float to_store<float, df>(df x) { return df_to_float(x); }
template <> __device__ __forceinline__ fpair to_store<fpair, dfpair>(dfpair x) { return fp_add(x.hi, x.lo); }

// Mixed operations with a storage value b (binary32 storage and double-float
// arithmetic use the cheaper double-word x word forms; other pairs convert).
template <typename N, typename T> __device__ __forceinline__ N mulx(N a, T b) { return a * to_num<N, T>(b); }
template <> __device__ __forceinline__ df mulx<df, float>(df a, float b) { return a * b; }
template <> __device__ __forceinline__ dfpair mulx<dfpair, fpair>(dfpair a, fpair b) { return a * b; }
template <typename N, typename T> __device__ __forceinline__ N addx(N a, T b) { return a + to_num<N, T>(b); }
template <> __device__ __forceinline__ df addx<df, float>(df a, float b) { return a + b; }
template <> __device__ __forceinline__ dfpair addx<dfpair, fpair>(dfpair a, fpair b) { return a + b; }
// a + b of two storage values (exact for double-float)
template <typename N, typename T> __device__ __forceinline__ N add2(T a, T b) { return to_num<N, T>(a) + to_num<N, T>(b); }
template <> __device__ __forceinline__ df add2<df, float>(float a, float b) { return df_add2(a, b); }
template <> __device__ __forceinline__ dfpair add2<dfpair, fpair>(fpair a, fpair b) { return df_add2(a, b); }
// x - y z and x + y z: as written for binary64 and binary32 (contracted to one FMA),
// the fused double-word forms for double-float
template <typename N> __device__ __forceinline__ N fms(N x, N y, N z) { return x - y * z; }
template <> __device__ __forceinline__ df fms<df>(df x, df y, df z) { return df_fms(x, y, z); }
template <> __device__ __forceinline__ dfpair fms<dfpair>(dfpair x, dfpair y, dfpair z) { return df_fms(x, y, z); }
template <typename N> __device__ __forceinline__ N fma_n(N x, N y, N z) { return x + y * z; }
template <> __device__ __forceinline__ df fma_n<df>(df x, df y, df z) { return df_fma(x, y, z); }
template <> __device__ __forceinline__ dfpair fma_n<dfpair>(dfpair x, dfpair y, dfpair z) { return df_fma(x, y, z); }
// dtr v rounded to the storage type
template <typename T, typename N> __device__ __forceinline__ T scaled_store(N dtr, N v) { return to_store<T, N>(dtr * v); }
template <> __device__ __forceinline__ float scaled_store<float, df>(df dtr, df v) { return df_mul_to_float(dtr, v); }
template <> __device__ __forceinline__ fpair scaled_store<fpair, dfpair>(dfpair dtr, dfpair v) {
    return df_mul_to_float(dtr, v);
}
__device__ __forceinline__ fpair operator-(fpair a) { return fp_neg(a); }

// One slot of column state: the pair form keeps the scalar layout (two consecutive df).
template <typename N>
__device__ __forceinline__ void put_state(N *p, N v) {
    *p = v;
}
template <>
__device__ __forceinline__ void put_state<dfpair>(dfpair *p, dfpair v) {
    *reinterpret_cast<float4 *>(p) = make_float4(fp_x(v.hi), fp_x(v.lo), fp_y(v.hi), fp_y(v.lo));
}

// Double-float column state in 48 bits (GTB_STATE48; global workspace): the binary32
// high part and the top 16 bits of the low part (its sign, exponent and 7 leading
// fraction bits), i.e. a value within 2^-8 |lo| <= 2^-32 |v| of the computed one.
// c'_k and e_k of one level go together: their high parts in one slot of the first
// array (float2 per column, float4 per column pair), their low parts packed into one
// word per column of the second (uint32, uint2 per pair).
__device__ __forceinline__ unsigned lo16_pack(float a, float b) {  // top halves of a (low) and b (high)
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}
// bytes of one slot of the low-part array (the first array's slot is sizeof(N))
template <typename N>
__host__ __device__ constexpr int sq_lo_bytes() {
    return sizeof(N) / 2;
}
__device__ __forceinline__ void put_state_sq(df *h, df *l, size_t idx, df c, df e) {
    reinterpret_cast<float2 *>(h)[idx] = make_float2(c.hi, e.hi);
    reinterpret_cast<unsigned *>(l)[idx] = lo16_pack(c.lo, e.lo);
}
__device__ __forceinline__ void put_state_sq(dfpair *h, dfpair *l, size_t idx, dfpair c, dfpair e) {
    reinterpret_cast<float4 *>(h)[idx] = make_float4(fp_x(c.hi), fp_y(c.hi), fp_x(e.hi), fp_y(e.hi));
    reinterpret_cast<uint2 *>(l)[idx] =
        make_uint2(lo16_pack(fp_x(c.lo), fp_y(c.lo)), lo16_pack(fp_x(e.lo), fp_y(e.lo)));
}
// the last read of a slot pair (streaming loads)
__device__ __forceinline__ void get_state_sq(const df *h, const df *l, size_t idx, df &c, df &e) {
    const float2 v = __ldcs(reinterpret_cast<const float2 *>(h) + idx);
    const unsigned w = __ldcs(reinterpret_cast<const unsigned *>(l) + idx);
    c = df{v.x, __uint_as_float(w << 16)};
    e = df{v.y, __uint_as_float(w & 0xFFFF0000u)};
}
__device__ __forceinline__ fpair lo16_unpack(unsigned w) {
    return fpair{((unsigned long long)(w & 0xFFFF0000u) << 32) | (unsigned long long)(w << 16)};
}
__device__ __forceinline__ void get_state_sq(const dfpair *h, const dfpair *l, size_t idx, dfpair &c, dfpair &e) {
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(h) + idx);
    const uint2 w = __ldcs(reinterpret_cast<const uint2 *>(l) + idx);
    c = dfpair{fp_make(v.x, v.y), lo16_unpack(w.x)};
    e = dfpair{fp_make(v.z, v.w), lo16_unpack(w.y)};
}

// Inputs of one level k for this lane's column (loaded one level ahead of their use).
template <typename T>
struct Level {
    T ut, uts, us1, up1, w;  // utens_k, utens_stage_k, u_stage_{k+1}, u_pos_{k+1}, wcon_{k+1}(i)
    T w1;                    // wcon_{k+1}(i+1) (last lane only; others take it by shuffle);
                             // pairs: wcon_{k+1}(2i+2) in the low half, every lane
};

template <typename T>
__device__ __forceinline__ void load_level(Level<T> &L, int k, int K, const T *pup, const T *put, const T *puts,
                                           const T *pus, const T *pw, const T *pw1, int64_t sk_up, int64_t sk_ut,
                                           int64_t sk_uts, int64_t sk_us, int64_t sk_w, bool last_lane) {
    // every input value is read once (streaming loads); utens_stage may be the output
    // array itself, whose level-k element is stored only after its value was used
    if (k < K) {
        L.ut = ld_once(put + (int64_t)k * sk_ut);
        L.uts = ld_once(puts + (int64_t)k * sk_uts);
    }
    if (k + 1 < K) {
        L.us1 = ld_once(pus + (int64_t)(k + 1) * sk_us);
        L.up1 = ld_once(pup + (int64_t)(k + 1) * sk_up);
        L.w = ld_once(pw + (int64_t)(k + 1) * sk_w);
        if constexpr (is_pair<T>()) {
            // the one binary32 face value past the pair (pw1: its address; sk_w in pairs)
            const float *f = reinterpret_cast<const float *>(pw1) + (int64_t)(k + 1) * sk_w * 2;
            L.w1 = fpair{(unsigned long long)__float_as_uint(*f)};
        } else {
            if (last_lane) L.w1 = ld_once(pw1 + (int64_t)(k + 1) * sk_w);
        }
    }
}

// s * 2^n (n < 0) with a sign flip, exact for normal binary64 inputs: the
// exponent field is adjusted on the integer pipe; inputs that would leave the
// normal range take the FP64 multiply (mul_fp64: kept inside its branch).
__device__ __forceinline__ double scale_pow2(double s, double k, int n) {
    const int hi = __double2hiint(s), lo = __double2loint(s);
    const int e = (hi >> 20) & 0x7FF;
    if (e + n >= 1 && e < 2047) return __hiloint2double((hi + (n << 20)) ^ 0x80000000, lo);
    return mul_fp64(k, s);
}

template <typename N>
__device__ __forceinline__ N coef(N s, N k, int n) {
    return k * s;
}
template <>
__device__ __forceinline__ double coef<double>(double s, double k, int n) {
    return n ? scale_pow2(s, k, n) : mul_fp64(k, s);
}
// double-float: k = -2^n is exact in binary32, so scaling both parts is exact
template <>
__device__ __forceinline__ df coef<df>(df s, df k, int n) {
    return n ? df{__fmul_rn(s.hi, k.hi), __fmul_rn(s.lo, k.hi)} : k * s;
}
template <>
__device__ __forceinline__ dfpair coef<dfpair>(dfpair s, dfpair k, int n) {
    return n ? dfpair{fp_mul(s.hi, k.hi), fp_mul(s.lo, k.hi)} : k * s;
}

template <typename T, typename N>
__host__ __device__ constexpr bool vadv_dp_global() {
    return sizeof(T) == sizeof(N);
}

// The y back substitution (one FP64 operation per point fewer, one more array of
// state) where the column state is in global memory: binary64 arithmetic only,
// whose pipe bounds the solve.  In binary32 it is slower (memory-bound there) and
// the y - s cancellation costs accuracy.
template <typename T, typename N>
__host__ __device__ constexpr bool vadv_yform() {
    return vadv_dp_global<T, N>() && std::is_same<N, double>::value;
}

// Arrays of column state per point: c'_k, and s_k (y form) or e_k when it cannot
// be parked in the output.
template <typename T, typename N>
__host__ __device__ constexpr int vadv_state_arrays() {
    return (vadv_dp_global<T, N>() && !vadv_yform<T, N>()) ? 1 : 2;
}

template <typename T, typename N>
__host__ __device__ constexpr size_t vadv_smem_per_col_level() {
    return (vadv_dp_global<T, N>() ? 1 : 2) * sizeof(N);
}

// Where the forward sweep keeps its eliminated coefficients:
//  * shared memory, [K][block columns]: the K x 32 x BJ state caps the
//    resident warps per SM;
//  * a caller-provided global workspace, [K][I*J] (column id j*I + i,
//    coalesced along i), written and read back within a few microseconds, so
//    it lives in L2.  No shared memory is needed and the resident warps are
//    bounded by registers only: on B300 the FP64 recurrence runs at the
//    pipe's rate only with many warps per SM (one warp keeps about one FP64
//    instruction in flight), so this is the fast form;
//  * a per-CTA slice of global scratch, [K][block columns] (batched form).
// The caller passes the base, the stride between levels and this thread's
// column index; `wr` says whether this thread may write its slot (inactive
// threads alias a real column in a domain-indexed workspace).
// DPG: a term of the backward sweep is parked in the output array (same element
// size as N) and read back by the backward sweep from L2.
// YF (global state, binary64 arithmetic, DPG): the backward sweep runs on y itself,
// y_k = d'_k - c'_k y_{k+1}, out_k = dtr (y_k - s_k), with d'_k parked in the
// output and s_k kept in the second state array: one FP64 operation per point
// fewer than the e_k form below, for one more array of state.  The shared-memory
// form keeps e_k (one slot per column and level fewer, twice the resident CTAs).
// SYM (beta_v = 0): the explicit weights equal the implicit ones and the explicit
// terms vanish into the matrix (below); a separate body, so that no FP64 instruction
// of the general case is issued, even predicated off (the FP64 pipe is the bound).
// GST: the column state is in global memory (its last reads are streaming loads); else
// in shared memory.  rsave (global state only, or null): the forward sweep also stores
// 1/p_k there, [k][column] like c'; c' and 1/p_k are then the factors the adjoint reads
// (gtb_vadv_adj with GTB_ADJ_FACTORS), and c' is not dropped from L2.  SF, the width of
// a double-float solve's global state: kStateFull, or kStatePacked, 48 bits
// (put_state_sq: 12 bytes per column and level instead of 16, so that less of it
// overflows L2 while every column of the grid is in flight; no rsave).
constexpr int kStateFull = 0, kStatePacked = 1;
template <typename T, typename N, int BJ, bool DPG, bool YF, bool SYM, bool GST, bool CHK, int SF>
__device__ __forceinline__ void vadv_columns_t(const View<const T> &us, const View<const T> &wc, const View<const T> &up,
                                               const View<const T> &ut, const View<const T> &uts, const View<T> &out,
                                               const VadvGeom &g, int bx, int by, N *cpb, N *dpb, size_t cstride,
                                               size_t cidx_ws, bool ws_domain, int tx, int ty, N *rsave = nullptr) {
    static_assert(!YF || DPG, "the y form parks d'_k in the output");
    constexpr bool SQ = is_df<N>() && GST && SF == kStatePacked;  // 48-bit double-float state
    static_assert(!SQ || (!DPG && !YF), "48-bit state holds c' and e_k");
    const int i = bx * 32 + tx, j = by * BJ + ty;
    const bool active = (i < g.I) && (j < g.J);
    const int ic = min(i, g.I - 1), jc = min(j, g.J - 1);
    // wcon is read up to i = I (I-staggered faces), or up to I-1 with the literal face velocity
    const int ilim = g.literal ? g.I - 1 : g.I;
    // pairs (g.I counts them): the pair's own faces 2i, 2i+1 and, apart, face 2i+2 (<= 2 g.I)
    const int iw = is_pair<T>() ? ic : min(i, ilim);
    const int K = g.K;
    const size_t cidx = ws_domain ? (size_t)jc * g.I + ic : cidx_ws;
    const bool wr = ws_domain ? active : true;

    const T *pus = us.p + ic + (int64_t)jc * us.sj;
    const T *pup = up.p + ic + (int64_t)jc * up.sj;
    const T *put = ut.p + ic + (int64_t)jc * ut.sj;
    const T *puts = uts.p + ic + (int64_t)jc * uts.sj;  // may alias po (in place)
    const T *pw = wc.p + iw + (int64_t)jc * wc.sj;
    const T *pw1 = is_pair<T>()
                       ? reinterpret_cast<const T *>(reinterpret_cast<const float *>(wc.p + (int64_t)jc * wc.sj) +
                                                     min(2 * ic + 2, 2 * g.I - (g.literal ? 1 : 0)))
                       : wc.p + min(i + 1, ilim) + (int64_t)jc * wc.sj;
    T *po = out.p + ic + (int64_t)jc * out.sj;
    const bool last_lane = (tx == 31);
    const bool lit = g.literal != 0;
    if constexpr (CHK) {  // every level of the column inside every field's storage
        const int64_t kl = K > 0 ? K - 1 : 0;
        bool ok = in_storage(us, pus, pus + kl * us.sk) && in_storage(up, pup, pup + kl * up.sk) &&
                  in_storage(ut, put, put + kl * ut.sk) && in_storage(uts, puts, puts + kl * uts.sk) &&
                  in_storage(wc, pw, pw + kl * wc.sk) && in_storage(out, po, po + kl * out.sk);
        if constexpr (is_pair<T>()) {
            const float *f1 = reinterpret_cast<const float *>(pw1);
            ok = ok && in_storage(wc, f1, f1 + kl * wc.sk * 2);
        } else {
            ok = ok && in_storage(wc, pw1, pw1 + kl * wc.sk);
        }
        if (!__all_sync(0xffffffffu, ok)) return;
    }

    const N dtr = num_const<N>(g.dtr);
    const N ka = num_const<N>(g.ka);
    const N kg = num_const<N>(g.kg);
    const N zero = num_const<N>(0.0);
    const int kexp = g.ka_pow2;  // a = ka * s as an exact exponent shift when ka = -2^kexp

    // The system of Sec. 3.1, A x = d, with d_k = dtr u_pos_k + utens_k + utens_stage_k
    // + E_k and the explicit terms E_k = -as_k (us_{k-1} - us_k) + as_{k+1} (us_{k+1} - us_k),
    // solved in the shifted unknown y = x + u_stage (us).  Since
    //   dtr us_k - (A us)_k = -a_k (us_{k-1} - us_k) + a_{k+1} (us_{k+1} - us_k),
    // A y = dtr s_k + utens_k + utens_stage_k - g_k (us_{k-1} - us_k) + g_{k+1} (us_{k+1} - us_k)
    // with s = u_stage + u_pos and g = as - a (zero when beta_v = 0: the explicit terms then
    // vanish into the matrix).  The output is dtr (x - u_pos) = dtr (y - s): YF back-
    // substitutes y and keeps s; otherwise the back substitution runs in z = x - u_pos =
    // y - s, z_k = e_k - c'_k z_{k+1}, e_k = d'_k - s_k - c'_k s_{k+1}.  Exact algebra;
    // u_pos is not read again by the backward sweep.
#define GTB_LOAD(L, k) load_level<T>(L, k, K, pup, put, puts, pus, pw, pw1, up.sk, ut.sk, uts.sk, us.sk, wc.sk, last_lane)
    // level k's inputs in L0; level k+1's are loaded at the top of iteration k (one
    // level ahead: on B300 a deeper prefetch only costs registers, i.e. resident warps)
    Level<T> L0, L1;
    GTB_LOAD(L0, 0);

    T us_cur = ld_once(pus);
    N s_cur = add2<N, T>(us_cur, ld_once(pup));  // s_0
    N dpl_prev = zero;                     // u_stage_k - u_stage_{k-1} (general case only)
    N a_cur = zero, g_cur = zero;          // a_0 = g_0 = 0
    N cp_prev = zero, dp_prev = zero, e_last = zero;

    // double-float: two levels per iteration let the compiler interleave one level's
    // FP32-pipe assembly with the previous level's recurrence (same results); binary64
    // gains nothing from it (its pipe is saturated)
#pragma unroll(is_df<N>() ? 2 : 1)
    for (int k = 0; k < K; ++k) {
        GTB_LOAD(L1, k + 1);
        const bool has_next = (k + 1 < K);
        N a_next = zero, g_next = zero, s_next = zero, dpl = zero;
        if (has_next) {
            N sf;
            if (lit) {
                sf = to_num<N, T>(L0.w);
            } else if constexpr (is_pair<T>()) {
                // faces (2i, 2i+1) and (2i+1, 2i+2): the pair against itself shifted by one
                sf = add2<N, T>(L0.w, fpair{(L0.w.v >> 32) | (L0.w1.v << 32)});
            } else {
                T hi = __shfl_down_sync(0xffffffffu, L0.w, 1);
                if (last_lane) hi = L0.w1;
                sf = add2<N, T>(L0.w, hi);
            }
            a_next = coef<N>(sf, ka, kexp);
            s_next = add2<N, T>(L0.us1, L0.up1);
            if (!SYM) {
                g_next = kg * sf;
                dpl = add2<N, T>(L0.us1, -us_cur);  // u_stage_{k+1} - u_stage_k
                us_cur = L0.us1;
            }
        }
        const N b = (dtr - a_cur) + a_next;  // dtr - a_k - c_k with c_k = -a_{k+1}
        // d = dtr s + utens + utens_stage: double-float adds the two inputs exactly first
        N d;
        if constexpr (is_df<N>()) d = df_fma(add2<N, T>(L0.ut, L0.uts), dtr, s_cur);
        else d = addx<N, T>(addx<N, T>(dtr * s_cur, L0.ut), L0.uts);
        if (!SYM) {  // + g_k (us_k - us_{k-1}) + g_{k+1} (us_{k+1} - us_k)
            if (k > 0) d = d + g_cur * dpl_prev;
            if (has_next) d = d + g_next * dpl;
        }
        N p = b, num = d;
        if (k > 0) {
            p = fms(b, a_cur, cp_prev);  // as the adjoint refactorises it (kept factors match bit for bit)
            num = fms(d, a_cur, dp_prev);
        }
        const N r = recip(p);
        const N cpk = (-a_next) * r, dpk = num * r;
        if (!SQ && wr) put_state(cpb + (size_t)k * cstride + cidx, cpk);
        if (rsave && wr) put_state(rsave + (size_t)k * cstride + cidx, r);
        N ek;  // the backward sweep's term of level k: d'_k (YF) or e_k
        if constexpr (YF) {
            ek = dpk;
            if (active) po[(int64_t)k * out.sk] = to_store<T, N>(dpk);
            if (wr) put_state(dpb + (size_t)k * cstride + cidx, s_cur);
        } else {
            ek = fms(dpk - s_cur, cpk, s_next);  // s_K = 0 (c'_{K-1} = 0)
            if (DPG) {
                if (active) po[(int64_t)k * out.sk] = to_store<T, N>(ek);
            } else if constexpr (SQ) {
                if (wr) put_state_sq(cpb, dpb, (size_t)k * cstride + cidx, cpk, ek);
            } else if (wr) {
                put_state(dpb + (size_t)k * cstride + cidx, ek);
            }
        }
        cp_prev = cpk, dp_prev = dpk, e_last = ek;
        s_cur = s_next;
        if (!SYM) dpl_prev = dpl, g_cur = g_next;
        a_cur = a_next;
        L0 = L1;
    }
#undef GTB_LOAD

    // backward substitution, utens_stage_out = dtr (y - s) (YF) or dtr z.  Levels go in
    // groups of BG; a group's inputs (d'_k or e_k, c'_k, s_k) are loaded before the
    // previous group's outputs are stored (distinct levels, so distinct addresses: the
    // out stride in k is nonzero), so the loads overlap instead of each waiting behind a
    // store.
    auto result = [&](N v, N sk) -> T {
        if constexpr (YF) return to_store<T, N>(dtr * (v - sk));
        else return scaled_store<T, N>(dtr, v);
    };
    // (the column state's last reads and the final outputs: streaming accesses; a value
    // parked in the output array is read with a plain load before its element is stored)
    auto ld_state = [&](const N *q) -> N {
        if constexpr (GST) return ld_once(q);
        else return *q;
    };
    N z = e_last;  // y_{K-1} = d'_{K-1} (YF) or z_{K-1} = e_{K-1}
    if (active)
        st_once(po + (int64_t)(K - 1) * out.sk, result(z, YF ? ld_state(dpb + (size_t)(K - 1) * cstride + cidx) : zero));
    constexpr int BG = 4;
    N eq[BG], cq[BG], sq[BG];
    auto load_group = [&](int k0) {
#pragma unroll
        for (int q = 0; q < BG; ++q) {
            const int k = k0 - q;
            if (k < 0) break;
            if constexpr (SQ) {
                get_state_sq(cpb, dpb, (size_t)k * cstride + cidx, cq[q], eq[q]);
            } else {
                eq[q] = DPG ? to_num<N, T>(po[(int64_t)k * out.sk]) : ld_state(dpb + (size_t)k * cstride + cidx);
                cq[q] = ld_state(cpb + (size_t)k * cstride + cidx);
            }
            sq[q] = YF ? ld_state(dpb + (size_t)k * cstride + cidx) : zero;
        }
    };
    // Global state: once a group's values are consumed, its lines are dead and the warp
    // drops the ones it owns whole (its 32 columns present, the line 128-byte aligned)
    // from L2 without a write-back.  Arrays: c', and s (y form) or e_k (not parked).
    constexpr int kArrays = (YF || !DPG) ? 2 : 1;
    constexpr int kLines = (int)(32 * sizeof(N) / 128);  // lines per warp, level and array
    // lines per warp and level of the first array (c', or the high parts) and the second
    constexpr int kL0 = kLines, kL1 = SQ ? 32 * sq_lo_bytes<N>() / 128 : (kArrays == 2 ? kLines : 0);
    constexpr int kPer = kL0 + kL1;
    constexpr size_t kSlot1 = SQ ? (size_t)sq_lo_bytes<N>() : sizeof(N);
    const bool own = GST && __all_sync(0xffffffffu, ws_domain ? active : true);
    const bool keep_cp = rsave != nullptr;  // c' is a kept factor: not dropped
    const size_t c0 = __shfl_sync(0xffffffffu, cidx, 0);
    if (K >= 2) load_group(K - 2);
    for (int k0 = K - 2; k0 >= 0; k0 -= BG) {
        N ec[BG], cc[BG], sc[BG];
#pragma unroll
        for (int q = 0; q < BG; ++q) ec[q] = eq[q], cc[q] = cq[q], sc[q] = sq[q];
        if (k0 - BG >= 0) load_group(k0 - BG);
#pragma unroll
        for (int q = 0; q < BG; ++q) {
            const int k = k0 - q;
            if (k < 0) break;
            z = fms(ec[q], cc[q], z);
            if (active) st_once(po + (int64_t)k * out.sk, result(z, sc[q]));
        }
        if constexpr (GST && kLines >= 1) {
            if (own) {
                __syncwarp();
                const int e = tx;  // (level in group, array, line) handled by this lane
                if (e < BG * kPer) {
                    const int q = e / kPer, r = e % kPer;
                    const int arr = r < kL0 ? 0 : 1, m = arr ? r - kL0 : r;
                    const int k = k0 - q;
                    if (k >= 0 && !(arr == 0 && keep_cp)) {
                        const size_t slot = (size_t)k * cstride + c0;
                        const unsigned char *line =
                            (arr == 0 ? reinterpret_cast<const unsigned char *>(cpb + slot)
                                      : reinterpret_cast<const unsigned char *>(dpb) + slot * kSlot1) +
                            m * 128;
                        if ((reinterpret_cast<uintptr_t>(line) & 127) == 0) discard_l2_line(line);
                    }
                }
            }
        }
    }
}

// CHK: test the column's address runs before the first access (the checked build, and
// the batched solve in every build)
template <typename T, typename N, int BJ, bool DPG, bool YF, bool GST, bool CHK = kChecked, int SF = kStateFull>
__device__ __forceinline__ void vadv_columns(const View<const T> &us, const View<const T> &wc, const View<const T> &up,
                                             const View<const T> &ut, const View<const T> &uts, const View<T> &out,
                                             const VadvGeom &g, int bx, int by, N *cpb, N *dpb, size_t cstride,
                                             size_t cidx_ws, bool ws_domain, int tx, int ty, N *rsave = nullptr) {
    if (g.sym)
        vadv_columns_t<T, N, BJ, DPG, YF, true, GST, CHK, SF>(us, wc, up, ut, uts, out, g, bx, by, cpb, dpb, cstride, cidx_ws,
                                                ws_domain, tx, ty, rsave);
    else
        vadv_columns_t<T, N, BJ, DPG, YF, false, GST, CHK, SF>(us, wc, up, ut, uts, out, g, bx, by, cpb, dpb, cstride, cidx_ws,
                                                 ws_domain, tx, ty, rsave);
}

// Single domain: one CTA per 32 x BJ block of columns; WS selects a
// domain-indexed global workspace over shared memory: c' in ws, the second state
// array in ws2, and (rsave, or null) 1/p_k kept for the adjoint.
// Column pairs: registers capped for 28 resident warps per SM (72 a thread, a few
// spilled); their chains of dependent paired operations need the warps more than the
// registers (512x512x80 double-float: 213 us uncapped at 114 registers, 192 us capped).
// SF: the width of a double-float workspace state (kStatePacked: rsave must be null).
template <typename T, typename N, int BJ, bool DPG, bool WS, int SF = kStateFull>
__global__ void __launch_bounds__(32 * BJ, is_pair<T>() ? 28 / BJ : 1)
    vadv_kernel(const View<const T> us, const View<const T> wc, const View<const T> up, const View<const T> ut,
                const View<const T> uts, const View<T> out, const VadvGeom g, N *__restrict__ ws,
                N *__restrict__ ws2, N *__restrict__ rsave) {
    constexpr int NT = 32 * BJ;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int t = threadIdx.y * 32 + threadIdx.x;
    static_assert(WS || !is_pair<T>(), "column pairs keep their state in a workspace");
    if constexpr (WS) {
        const size_t cstride = (size_t)g.I * g.J;
        vadv_columns<T, N, BJ, DPG, vadv_yform<T, N>(), true, kChecked, SF>(
            us, wc, up, ut, uts, out, g, blockIdx.x, blockIdx.y, ws, ws2, cstride, 0, true, threadIdx.x, threadIdx.y,
            rsave);
    } else {
        N *cpb = reinterpret_cast<N *>(smem_raw);
        vadv_columns<T, N, BJ, DPG, false, false>(us, wc, up, ut, uts, out, g, blockIdx.x, blockIdx.y, cpb,
                                           cpb + (size_t)g.K * NT, NT, t, false, threadIdx.x, threadIdx.y);
    }
}

}  // namespace gtb
