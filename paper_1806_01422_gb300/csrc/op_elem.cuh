// Element kernels for F(u), J(u)w and J(u)^T v in d = 1, 2, 3 (arXiv:1806.01422,
// eqs. rhsvec, jacvec, jactransvec).  Each kernel reads the global (unique-node)
// inputs with the periodic scatter Q, computes one element-local result per
// element and writes it to an element-local buffer; the gather-scatter sum
// Q^T (and the 1/k multiplicity scaling for F and J) is done by the assembly
// kernel, which also applies the Runge-Kutta epilogue.
//
// Local results (see op_kernels.cuh for the matrices):
//   F :  f_c   = sum_j [ Sv_j U_c - U_j Dg_j U_c ]
//   J :  f_c   = sum_j [ Sv_j W_c - (W_j Dg_j U_c + U_j Dg_j W_c) ]
//   JT:  f_l   = sum_j Dd_j (Gv_j Z_l + U_j Z_l) - sum_c Z_c Dg_l U_c,   Z = v / k
// with Dg_j, Sv_j, Gv_j, Dd_j the 1D matrices applied along direction x_j.  Each
// bracket is one pass along direction j; in 3D the x and y passes write two
// partial-result tiles and the z pass adds them and writes the result.
#pragma once
#include "op_kernels.cuh"

namespace semk {

template <int D>
__host__ __device__ constexpr int tiles_per_elem(int op) {
    // inputs (U; U and W; U and Z) plus the partial results (F; F and A in 3D)
    return (op == OP_RHS ? D : 2 * D) + (D == 3 ? 2 : 1);
}

// 3D kernels that run their passes from one copy of the code (df3_body): the
// double-float ones (long unrolled passes) and FP32 with n >= 12 (register-bound
// with three unrolled copies).
template <typename T, int NP>
__host__ __device__ constexpr bool shared_pass3() {
    return std::is_same<T, dfloat>::value || (sizeof(T) == 4 && NP >= 12);
}

// FP32 F and J^T in 3D (the unrolled bodies): the y pass adds the x pass's partial
// tile in place, so one partial tile serves both, at one more barrier per
// component.  The results are the same bits (x part + y part, then the z part).  At
// n = 8, F's four tiles instead of five let five blocks of four elements share an
// SM instead of four; at every n the smaller shared-memory footprint leaves more of
// the SM's on-chip memory to L1, which caches the neighbouring elements' shared
// nodes of the tile gathers.  Measured per element pass: F at n = 6, 8, 10 gained
// 11 %, 6 % and 1 %, and lost 6 % at n = 4 (the barrier); J^T gained 9 % at n = 7
// and 8 % at n = 8, and lost 2 % at n = 9.  J keeps two partial tiles.
template <typename T, int NP>
__host__ __device__ constexpr bool one_partial3(int op) {
    return sizeof(T) == 4 && !shared_pass3<T, NP>() && NP >= 6 && (op == OP_RHS || (op == OP_JACT && NP <= 8));
}

// Shared-memory tiles per element of the (non-lean) 3D element kernels.
template <typename T, int NP>
__host__ __device__ constexpr int tiles3(int op) {
    return tiles_per_elem<3>(op) - (one_partial3<T, NP>(op) ? 1 : 0);
}

// ------------------------------------------------------------------ loaders
// FP64 form: tiles hold the input doubles.
// FP32 form: every input node is read as a float pair (hi, lo) -- either from the
// two FP32 planes of a sweep-internal state, or split from a caller's double
// with integer instructions (split_bits), which give the same pair -- and a tile
// of U (or W) holds U - U_ref formed as (hi - hi_ref) + (lo - lo_ref) in FP32,
// U_ref being the value at the element's first node.  The 1D matrices applied
// to U and W annihilate constants (Dhat 1 = 0), so gradients and viscous terms
// see only the small in-element variation and lose little to FP32
// cancellation; pointwise products add hi_ref back.  Z = v / k keeps hi only.
template <typename T>
struct RefSub {
    static constexpr bool on = sizeof(T) == 4;
};

template <typename T>
__device__ __forceinline__ T with_ref(T ref, T x) {
    if constexpr (RefSub<T>::on) return ref + x;
    else return x;
}

__device__ __forceinline__ void read_pair(const ElemArgs& a, const void* g, size_t i, float& hi, float& lo) {
    if (a.in_f2) {
        hi = __ldg((const float*)g + i);
        lo = __ldg((const float*)g + a.plane + i);
    } else {
        split_bits(__ldg((const double*)g + i), hi, lo);
    }
}

// 1/k for k = 2^nb sharing elements (exact)
template <typename T>
__device__ __forceinline__ T inv_mult(int nb) {
    return nb == 0 ? (T)1 : (nb == 1 ? (T)0.5 : (nb == 2 ? (T)0.25 : (T)0.125));
}

// x * 2^-nb (nb = 0..3) without an FP64 instruction: the exponent field is lowered with
// integer arithmetic, which is exact.  Zeros, subnormal results, infinities and NaNs (rare)
// take the multiply, which gives the same value.
__device__ __forceinline__ double scale_pow2_down(double x, int nb) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex > nb && ex != 0x7ff) return __longlong_as_double(b - ((long long)nb << 52));
    return x * inv_mult<double>(nb);
}

// Value stored in a tile for global node i: the input (FP64), U - U_ref (FP32), or
// v / k when scale_mult (nb = boundary count of the node, k = 2^nb).
template <typename T>
__device__ __forceinline__ T tile_value(const ElemArgs& a, const void* g, size_t i, bool scale_mult, int nb,
                                        float ref_hi, float ref_lo) {
    if constexpr (std::is_same<T, dfloat>::value) {
        // double input split exactly enough (|x - h - l| <= 2^-47 |x|) with integer
        // instructions; 1/k is a power of two
        float h, l;
        split_bits(__ldg((const double*)g + i), h, l);
        if (scale_mult) {
            const float s = inv_mult<float>(nb);
            h *= s;
            l *= s;
        }
        return dfloat(h, l);
    } else if constexpr (sizeof(T) == 8) {
        const double x = __ldg((const double*)g + i);
        return scale_mult ? scale_pow2_down(x, nb) : x;
    } else {
        if (scale_mult && a.in_f2) return __ldg((const float*)g + i) * inv_mult<float>(nb);   // hi plane only
        float hi, lo;
        read_pair(a, g, i, hi, lo);
        if (scale_mult) return hi * inv_mult<float>(nb);
        return __fadd_rn(__fsub_rn(hi, ref_hi), __fsub_rn(lo, ref_lo));
    }
}

// Tile entry of a double input x (FP64 and double-float forms), times 1/k for Z = v / k.
template <typename T>
__device__ __forceinline__ T tile_of_double(double x, bool scale_mult, int nb) {
    if constexpr (std::is_same<T, dfloat>::value) {
        float h, l;
        split_bits(x, h, l);
        if (scale_mult) {
            const float sc = inv_mult<float>(nb);
            h *= sc;
            l *= sc;
        }
        return dfloat(h, l);
    } else {
        return scale_mult ? scale_pow2_down(x, nb) : x;
    }
}

// Load component c of a global field into an element tile (d = 3): thread t of
// the element owns column (i, j) = (t % n, t / n) and walks k.  `scale_mult`
// multiplies each node by 1/k (k = elements sharing it), used for Z = v / k.
// Returns the reference value of the tile (0 unless FP32 and not Z).
template <typename T, int NP>
__device__ __forceinline__ T load3(T* tile, const void* g, int c, int ex, int ey, int ez, int t, bool valid,
                                   const ElemArgs& a, bool scale_mult) {
    using Tl = Tile<NP>;
    const int i = t % NP, j = t / NP;
    const int N = a.N, G = a.G;
    const int gx = wrap(ex * N + i, G), gy = wrap(ey * N + j, G);
    const int nbij = (int)(i == 0 || i == N) + (int)(j == 0 || j == N);
    float ref_hi = 0.f, ref_lo = 0.f;
    if (RefSub<T>::on && !scale_mult && valid) read_pair(a, g, gidx3(c, ez * N, ey * N, ex * N, G), ref_hi, ref_lo);
    // Index of node k of the column: its nodes are G^2 apart, and only node N of the last
    // element along z wraps to gz = 0.  32-bit arithmetic suffices (fewer than 2^31 unknowns).
    const unsigned G2 = (unsigned)G * (unsigned)G;
    const unsigned col = (((unsigned)c * G + (unsigned)(ez * N)) * G + gy) * G + gx;
    const unsigned zwrap = ez == a.E - 1 ? (unsigned)G * G2 : 0u;
    auto node = [&](int k) -> unsigned { return col + (unsigned)k * G2 - (k == NP - 1 ? zwrap : 0u); };
    if constexpr (RefSub<T>::on) {
        // FP32 form: issue every load of the column before the first conversion, so that
        // the gather's latency is paid once per column rather than once per node
        float hv[NP], lv[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            hv[k] = 0.f;
            lv[k] = 0.f;
            const unsigned idx = node(k);
            if (valid) {
                if (a.in_f2) {
                    hv[k] = __ldg((const float*)g + idx);
                    if (!scale_mult) lv[k] = __ldg((const float*)g + a.plane + idx);
                } else {
                    split_bits(__ldg((const double*)g + idx), hv[k], lv[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float v = scale_mult ? hv[k] * inv_mult<float>(nbij + (int)(k == 0 || k == N))
                                       : __fadd_rn(__fsub_rn(hv[k], ref_hi), __fsub_rn(lv[k], ref_lo));
            tile[(k * NP + j) * Tl::P + i] = valid ? v : 0.f;
        }
        return (T)ref_hi;
    } else {
        // double inputs: every load of the column first, then the conversions
        double xv[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) xv[k] = valid ? __ldg((const double*)g + node(k)) : 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k)
            tile[(k * NP + j) * Tl::P + i] = tile_of_double<T>(xv[k], scale_mult, nbij + (int)(k == 0 || k == N));
        return (T)ref_hi;
    }
}

// Load the three components of u (and of the second input) of a d = 3 element.
template <typename T, int NP>
__device__ __forceinline__ void load3_fields(T* const* sU, T* const* sV, const ElemArgs& a, int ex, int ey, int ez,
                                             int t, bool valid, T* rU, T* rV, bool v_is_z) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        rU[c] = load3<T, NP>(sU[c], a.u, c, ex, ey, ez, t, valid, a, false);
        if (sV) rV[c] = load3<T, NP>(sV[c], a.w, c, ex, ey, ez, t, valid, a, v_is_z);
    }
}

// d = 2: thread t owns row j = t and walks i.
template <typename T, int NP>
__device__ __forceinline__ T load2(T* tile, const void* g, int c, int ex, int ey, int t, bool valid,
                                   const ElemArgs& a, bool scale_mult) {
    using Tl = Tile<NP>;
    const int j = t;
    const int N = a.N, G = a.G;
    const int gy = wrap(ey * N + j, G);
    const int nbj = (int)(j == 0 || j == N);
    const size_t row = ((size_t)c * G + gy) * G;
    float ref_hi = 0.f, ref_lo = 0.f;
    if (RefSub<T>::on && !scale_mult && valid) read_pair(a, g, ((size_t)c * G + ey * N) * G + ex * N, ref_hi, ref_lo);
    if constexpr (RefSub<T>::on) {
        // every load of the row first, then the conversions (see load3)
        float hv[NP], lv[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            hv[i] = 0.f;
            lv[i] = 0.f;
            const size_t idx = row + wrap(ex * N + i, G);
            if (valid) {
                if (a.in_f2) {
                    hv[i] = __ldg((const float*)g + idx);
                    if (!scale_mult) lv[i] = __ldg((const float*)g + a.plane + idx);
                } else {
                    split_bits(__ldg((const double*)g + idx), hv[i], lv[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const float v = scale_mult ? hv[i] * inv_mult<float>(nbj + (int)(i == 0 || i == N))
                                       : __fadd_rn(__fsub_rn(hv[i], ref_hi), __fsub_rn(lv[i], ref_lo));
            tile[j * Tl::P + i] = valid ? v : 0.f;
        }
        return (T)ref_hi;
    } else {
        double xv[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) xv[i] = valid ? __ldg((const double*)g + row + wrap(ex * N + i, G)) : 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i)
            tile[j * Tl::P + i] = tile_of_double<T>(xv[i], scale_mult, nbj + (int)(i == 0 || i == N));
        return (T)ref_hi;
    }
}

// ================================================================== d = 3
// Line bases of thread t (n^2 threads per element):
//   x-line (j, k) = (t % n, t / n): base t*P,                stride 1
//   y-line (i, k) = (t % n, t / n): base (t/n)*S2 + t % n,   stride P
//   z-line (i, j) = (t % n, t / n): base (t/n)*P + t % n,    stride S2
// The z pass writes node (i, j, m) of the element-local result at m*n^2 + j*n + i,
// so a warp stores contiguous runs.

// One F pass along a direction: r = Sv x - Ud * (Dg x), x the line of U_c - ref.
template <typename T, int NP, int STRIDE>
__device__ __forceinline__ void rhs_pass(const OpMats<T, NP>& M, const T* sUc, const T* sUd, T rd, int base,
                                         T (&r)[NP]) {
    T x[NP], g[NP];
    ld_line<T, NP, STRIDE>(sUc, base, x);
    Pre<T, NP> p;
    pre_add<T, NP>(x, p);
    eo_apply<false, T, NP>(M.Dg, p, g);
    eo_apply<true, T, NP>(M.Sv, p, r);
#pragma unroll
    for (int m = 0; m < NP; ++m) r[m] = fma(-with_ref(rd, sUd[base + m * STRIDE]), g[m], r[m]);
}

// One J pass: r = Sv W_c - (W_d Dg U_c + U_d Dg W_c).
template <typename T, int NP, int STRIDE>
__device__ __forceinline__ void jac_pass(const OpMats<T, NP>& M, const T* sUc, const T* sWc, const T* sUd,
                                         const T* sWd, T ru, T rw, int base, T (&r)[NP]) {
    T x[NP], gw[NP], gu[NP];
    ld_line<T, NP, STRIDE>(sWc, base, x);
    Pre<T, NP> p;
    pre_add<T, NP>(x, p);
    eo_apply<false, T, NP>(M.Dg, p, gw);
    eo_apply<true, T, NP>(M.Sv, p, r);
    ld_line<T, NP, STRIDE>(sUc, base, x);
    eo_apply<false, T, NP>(M.Dg, x, gu);
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const int id = base + m * STRIDE;
        r[m] -= fma(with_ref(rw, sWd[id]), gu[m], with_ref(ru, sUd[id]) * gw[m]);
    }
}

// One J^T pass: r = Dd (Gv Z_l + U_d Z_l), plus -sum_c Z_c Dg U_c when d == l.
template <typename T, int NP, int STRIDE, int D>
__device__ __forceinline__ void jact_pass(const OpMats<T, NP>& M, T* const* sU, T* const* sZ, const T* rU,
                                          int l, int d, int base, T (&r)[NP]) {
    T z[NP], u[NP];
    ld_line<T, NP, STRIDE>(sZ[l], base, z);
#pragma unroll
    for (int m = 0; m < NP; ++m) u[m] = with_ref(rU[d], sU[d][base + m * STRIDE]);
    gvdd_apply<T, NP>(M.Gv, M.Dd, z, u, r);
    if (l == d) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            T x[NP], g[NP];
            ld_line<T, NP, STRIDE>(sU[c], base, x);
            eo_apply<false, T, NP>(M.Dg, x, g);
#pragma unroll
            for (int m = 0; m < NP; ++m) r[m] = fma(-sZ[c][base + m * STRIDE], g[m], r[m]);
        }
    }
}


template <typename T, int NP, int D>
__device__ __forceinline__ void jact_pass_rt(const OpMats<T, NP>& M, T* const* sU, T* const* sZ, const T* rU, int l,
                                             int d, int base, int stride, T (&r)[NP]);

// Run-time-stride versions of the passes, for the double-float kernels: one copy of
// a pass serves every direction (see jact_pass_rt).
template <typename T, int NP>
__device__ __forceinline__ void rhs_pass_rt(const OpMats<T, NP>& M, const T* sUc, const T* sUd, T rd, int base,
                                            int stride, T (&r)[NP]) {
    T x[NP], g[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) x[m] = sUc[base + m * stride];
    Pre<T, NP> p;
    pre_add<T, NP>(x, p);
    eo_apply<false, T, NP>(M.Dg, p, g);
    eo_apply<true, T, NP>(M.Sv, p, r);
#pragma unroll
    for (int m = 0; m < NP; ++m) r[m] = fma(-with_ref(rd, sUd[base + m * stride]), g[m], r[m]);
}

template <typename T, int NP>
__device__ __forceinline__ void jac_pass_rt(const OpMats<T, NP>& M, const T* sUc, const T* sWc, const T* sUd,
                                            const T* sWd, T ru, T rw, int base, int stride, T (&r)[NP]) {
    T x[NP], gw[NP], gu[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) x[m] = sWc[base + m * stride];
    Pre<T, NP> p;
    pre_add<T, NP>(x, p);
    eo_apply<false, T, NP>(M.Dg, p, gw);
    eo_apply<true, T, NP>(M.Sv, p, r);
#pragma unroll
    for (int m = 0; m < NP; ++m) x[m] = sUc[base + m * stride];
    eo_apply<false, T, NP>(M.Dg, x, gu);
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const int id = base + m * stride;
        r[m] -= fma(with_ref(rw, sWd[id]), gu[m], with_ref(ru, sUd[id]) * gw[m]);
    }
}

// d = 3 double-float element body: the three passes run from one copy of the pass
// code in a loop over directions; x and y write the partial tiles, z adds and stores.
template <typename T, int NP>
__device__ __forceinline__ void df3_body(const OpMats<T, NP>& M, const ElemArgs& a, int op, T* const* sU,
                                         T* const* sV, T* sF, T* sA, const T* rU, const T* rV, int e, int t,
                                         bool valid) {
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2;
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP) + (t / NP) * NP + t % NP;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            const int base = d == 0 ? xb : (d == 1 ? yb : zb);
            const int stride = d == 0 ? 1 : (d == 1 ? P : S2);
            const T* sUd = d == 0 ? sU[0] : (d == 1 ? sU[1] : sU[2]);
            T r[NP];
            if (op == OP_RHS) {
                rhs_pass_rt<T, NP>(M, sU[c], sUd, rU[d], base, stride, r);
            } else if (op == OP_JAC) {
                const T* sVd = d == 0 ? sV[0] : (d == 1 ? sV[1] : sV[2]);
                jac_pass_rt<T, NP>(M, sU[c], sV[c], sUd, sVd, rU[d], rV[d], base, stride, r);
            } else {
                jact_pass_rt<T, NP, 3>(M, sU, sV, rU, c, d, base, stride, r);
            }
            if (d < 2) {
                T* dst = d == 0 ? sF : sA;
#pragma unroll
                for (int m = 0; m < NP; ++m) dst[base + m * stride] = r[m];
                if (d == 1) __syncthreads();
            } else if (valid) {
#pragma unroll
                for (int m = 0; m < NP; ++m)
                    out[(size_t)c * NP * NP * NP + m * NP * NP] = to_out(r[m] + (sF[zb + m * S2] + sA[zb + m * S2]));
            }
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__device__ __forceinline__ void rhs3_body(const OpMats<T, NP>& M, const ElemArgs& a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP * NP, P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    constexpr bool ONE = one_partial3<T, NP>(OP_RHS);
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles3<T, NP>(OP_RHS) * S3;
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sF = sm + 3 * S3;
    T* sA = ONE ? sF : sm + 4 * S3;
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3];
    load3_fields<T, NP>(sU, nullptr, a, ex, ey, ez, t, valid, rU, nullptr, false);
    __syncthreads();
    pdl_trigger();
    if constexpr (shared_pass3<T, NP>()) {
        df3_body<T, NP>(M, a, OP_RHS, sU, sU, sF, sA, rU, rU, e, t, valid);
        return;
    }
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP) + (t / NP) * NP + t % NP;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        T r[NP];
        rhs_pass<T, NP, 1>(M, sU[c], sU[0], rU[0], xb, r);
        st_line<T, NP, 1>(sF, xb, r);
        if constexpr (ONE) {
            // partial tile F = x part + y part (the sum the z pass would form: same bits)
            __syncthreads();
            rhs_pass<T, NP, P>(M, sU[c], sU[1], rU[1], yb, r);
#pragma unroll
            for (int m = 0; m < NP; ++m) sF[yb + m * P] = sF[yb + m * P] + r[m];
            __syncthreads();
            rhs_pass<T, NP, S2>(M, sU[c], sU[2], rU[2], zb, r);
            if (valid) {
#pragma unroll
                for (int m = 0; m < NP; ++m) out[(size_t)c * NP * NP * NP + m * NP * NP] = to_out(r[m] + sF[zb + m * S2]);
            }
        } else {
            rhs_pass<T, NP, P>(M, sU[c], sU[1], rU[1], yb, r);
            st_line<T, NP, P>(sA, yb, r);
            __syncthreads();
            rhs_pass<T, NP, S2>(M, sU[c], sU[2], rU[2], zb, r);
            if (valid) {
#pragma unroll
                for (int m = 0; m < NP; ++m) out[(size_t)c * NP * NP * NP + m * NP * NP] = to_out(r[m] + (sF[zb + m * S2] + sA[zb + m * S2]));
            }
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__device__ __forceinline__ void jac3_body(const OpMats<T, NP>& M, const ElemArgs& a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP * NP, P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<3>(OP_JAC) * S3;
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sW[3] = {sm + 3 * S3, sm + 4 * S3, sm + 5 * S3};
    T* sF = sm + 6 * S3;
    T* sA = sm + 7 * S3;
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3], rW[3];
    load3_fields<T, NP>(sU, sW, a, ex, ey, ez, t, valid, rU, rW, false);
    __syncthreads();
    pdl_trigger();
    if constexpr (shared_pass3<T, NP>()) {
        df3_body<T, NP>(M, a, OP_JAC, sU, sW, sF, sA, rU, rW, e, t, valid);
        return;
    }
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP) + (t / NP) * NP + t % NP;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        T r[NP];
        jac_pass<T, NP, 1>(M, sU[c], sW[c], sU[0], sW[0], rU[0], rW[0], xb, r);
        st_line<T, NP, 1>(sF, xb, r);
        jac_pass<T, NP, P>(M, sU[c], sW[c], sU[1], sW[1], rU[1], rW[1], yb, r);
        st_line<T, NP, P>(sA, yb, r);
        __syncthreads();
        jac_pass<T, NP, S2>(M, sU[c], sW[c], sU[2], sW[2], rU[2], rW[2], zb, r);
        if (valid) {
#pragma unroll
            for (int m = 0; m < NP; ++m) out[(size_t)c * NP * NP * NP + m * NP * NP] = to_out(r[m] + (sF[zb + m * S2] + sA[zb + m * S2]));
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__device__ __forceinline__ void jact3_body(const OpMats<T, NP>& M, const ElemArgs& a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP * NP, P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    constexpr bool ONE = one_partial3<T, NP>(OP_JACT);
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles3<T, NP>(OP_JACT) * S3;
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sZ[3] = {sm + 3 * S3, sm + 4 * S3, sm + 5 * S3};
    T* sF = sm + 6 * S3;
    T* sA = ONE ? sF : sm + 7 * S3;
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3], rZ[3];
    load3_fields<T, NP>(sU, sZ, a, ex, ey, ez, t, valid, rU, rZ, true);
    __syncthreads();
    pdl_trigger();
    if constexpr (shared_pass3<T, NP>()) {
        df3_body<T, NP>(M, a, OP_JACT, sU, sZ, sF, sA, rU, rU, e, t, valid);
        return;
    }
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP) + (t / NP) * NP + t % NP;
#pragma unroll 1
    for (int l = 0; l < 3; ++l) {
        T r[NP];
        jact_pass<T, NP, 1, 3>(M, sU, sZ, rU, l, 0, xb, r);
        st_line<T, NP, 1>(sF, xb, r);
        if constexpr (ONE) {
            __syncthreads();
            jact_pass<T, NP, P, 3>(M, sU, sZ, rU, l, 1, yb, r);
#pragma unroll
            for (int m = 0; m < NP; ++m) sF[yb + m * P] = sF[yb + m * P] + r[m];
            __syncthreads();
            jact_pass<T, NP, S2, 3>(M, sU, sZ, rU, l, 2, zb, r);
            if (valid) {
#pragma unroll
                for (int m = 0; m < NP; ++m) out[(size_t)l * NP * NP * NP + m * NP * NP] = to_out(r[m] + sF[zb + m * S2]);
            }
        } else {
            jact_pass<T, NP, P, 3>(M, sU, sZ, rU, l, 1, yb, r);
            st_line<T, NP, P>(sA, yb, r);
            __syncthreads();
            jact_pass<T, NP, S2, 3>(M, sU, sZ, rU, l, 2, zb, r);
            if (valid) {
#pragma unroll
                for (int m = 0; m < NP; ++m) out[(size_t)l * NP * NP * NP + m * NP * NP] = to_out(r[m] + (sF[zb + m * S2] + sA[zb + m * S2]));
            }
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__global__ void rhs3_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    rhs3_body<T, NP>(M, a);
}

template <typename T, int NP>
__global__ void jac3_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    jac3_body<T, NP>(M, a);
}

template <typename T, int NP>
__global__ void jact3_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    jact3_body<T, NP>(M, a);
}

// FP64 with n = 8 (the order of the 3D workload): the same bodies with the registers
// capped so that more blocks share an SM.  Uncapped, F uses 136 registers per thread and
// one 256-thread block fits an SM (8 warps); capped at 128 (36 bytes of spill) two fit.
// J and J^T run blocks of 128 threads (two elements): capped at 170 registers, three
// blocks fit instead of two, with no spill.  The FP64 pipe is the bound; the extra warps
// hide its latency.
template <int NP>
__global__ void __launch_bounds__(256, 2) rhs3_f64_kernel(const __grid_constant__ OpMats<double, NP> M,
                                                          const ElemArgs a) {
    rhs3_body<double, NP>(M, a);
}

template <int NP>
__global__ void __launch_bounds__(128, 3) jac3_f64_kernel(const __grid_constant__ OpMats<double, NP> M,
                                                          const ElemArgs a) {
    jac3_body<double, NP>(M, a);
}

template <int NP>
__global__ void __launch_bounds__(128, 3) jact3_f64_kernel(const __grid_constant__ OpMats<double, NP> M,
                                                           const ElemArgs a) {
    jact3_body<double, NP>(M, a);
}

// ================================================================== d = 2
// n threads per element.  x-line j = t: base t*P, stride 1; y-line i = t: base t,
// stride P.  The x pass writes its part to a tile; the y pass adds it and writes
// node (i, m) of the element-local result at m*n + i (contiguous over a warp).
// Element e (thread t of the element, slot el of the block's shared memory) of a d = 2 F apply.
template <typename T, int NP>
__device__ __forceinline__ void rhs2_body(const OpMats<T, NP>& M, const ElemArgs& a, int e, int t, int el,
                                        bool valid, unsigned char* smem_raw) {
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<2>(OP_RHS) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sF = sm + 2 * S2;
    const int ex = e % a.E, ey = e / a.E;
    T rU[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) rU[c] = load2<T, NP>(sU[c], a.u, c, ex, ey, t, valid, a, false);
    __syncthreads();
    const int xb = t * P, yb = t;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 2 * (NP * NP) + t;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        T r[NP];
        rhs_pass<T, NP, 1>(M, sU[c], sU[0], rU[0], xb, r);
        st_line<T, NP, 1>(sF, xb, r);
        __syncthreads();
        rhs_pass<T, NP, P>(M, sU[c], sU[1], rU[1], yb, r);
        if (valid) {
#pragma unroll
            for (int m = 0; m < NP; ++m) out[(size_t)c * NP * NP + m * NP] = to_out(r[m] + sF[yb + m * P]);
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__global__ void rhs2_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int el = threadIdx.x / NP, t = threadIdx.x % NP;
    const int e = blockIdx.x * (blockDim.x / NP) + el;
    rhs2_body<T, NP>(M, a, e, t, el, e < a.nelem, smem_raw);
}

// Element e (thread t of the element, slot el of the block's shared memory) of a d = 2 J apply.
template <typename T, int NP>
__device__ __forceinline__ void jac2_body(const OpMats<T, NP>& M, const ElemArgs& a, int e, int t, int el,
                                        bool valid, unsigned char* smem_raw) {
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<2>(OP_JAC) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sW[2] = {sm + 2 * S2, sm + 3 * S2};
    T* sF = sm + 4 * S2;
    const int ex = e % a.E, ey = e / a.E;
    T rU[2], rW[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        rU[c] = load2<T, NP>(sU[c], a.u, c, ex, ey, t, valid, a, false);
        rW[c] = load2<T, NP>(sW[c], a.w, c, ex, ey, t, valid, a, false);
    }
    __syncthreads();
    const int xb = t * P, yb = t;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 2 * (NP * NP) + t;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        T r[NP];
        jac_pass<T, NP, 1>(M, sU[c], sW[c], sU[0], sW[0], rU[0], rW[0], xb, r);
        st_line<T, NP, 1>(sF, xb, r);
        __syncthreads();
        jac_pass<T, NP, P>(M, sU[c], sW[c], sU[1], sW[1], rU[1], rW[1], yb, r);
        if (valid) {
#pragma unroll
            for (int m = 0; m < NP; ++m) out[(size_t)c * NP * NP + m * NP] = to_out(r[m] + sF[yb + m * P]);
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__global__ void jac2_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int el = threadIdx.x / NP, t = threadIdx.x % NP;
    const int e = blockIdx.x * (blockDim.x / NP) + el;
    jac2_body<T, NP>(M, a, e, t, el, e < a.nelem, smem_raw);
}

// Element e (thread t of the element, slot el of the block's shared memory) of a d = 2 J^T apply.
template <typename T, int NP>
__device__ __forceinline__ void jact2_body(const OpMats<T, NP>& M, const ElemArgs& a, int e, int t, int el,
                                        bool valid, unsigned char* smem_raw) {
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<2>(OP_JACT) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sZ[2] = {sm + 2 * S2, sm + 3 * S2};
    T* sF = sm + 4 * S2;
    const int ex = e % a.E, ey = e / a.E;
    T rU[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        rU[c] = load2<T, NP>(sU[c], a.u, c, ex, ey, t, valid, a, false);
        load2<T, NP>(sZ[c], a.w, c, ex, ey, t, valid, a, true);
    }
    __syncthreads();
    const int xb = t * P, yb = t;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 2 * (NP * NP) + t;
#pragma unroll 1
    for (int l = 0; l < 2; ++l) {
        T r[NP];
        jact_pass<T, NP, 1, 2>(M, sU, sZ, rU, l, 0, xb, r);
        st_line<T, NP, 1>(sF, xb, r);
        __syncthreads();
        jact_pass<T, NP, P, 2>(M, sU, sZ, rU, l, 1, yb, r);
        if (valid) {
#pragma unroll
            for (int m = 0; m < NP; ++m) out[(size_t)l * NP * NP + m * NP] = to_out(r[m] + sF[yb + m * P]);
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__global__ void jact2_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int el = threadIdx.x / NP, t = threadIdx.x % NP;
    const int e = blockIdx.x * (blockDim.x / NP) + el;
    jact2_body<T, NP>(M, a, e, t, el, e < a.nelem, smem_raw);
}

// ================================================================== d = 2, one thread per (line, component)
// Double-float kernels are bound by latency, not by a pipe: a 2D grid has too few
// lines to hide the dependent chains of a compensated multiply-add.  These bodies
// give each output component its own thread (2n threads per element): thread
// (t, c) runs the x and y passes of component c, with one partial tile per
// component.  The per-thread work halves and the thread count doubles; the
// passes and the summation order are those of the bodies above.
template <typename T, int NP>
__device__ __forceinline__ void rhs2c_body(const OpMats<T, NP>& M, const ElemArgs& a, int e, int t, int c, int el,
                                         bool valid, unsigned char* smem_raw) {
    static_assert(!RefSub<T>::on, "component-parallel bodies assume no reference subtraction");
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * (tiles_per_elem<2>(OP_RHS) + 1) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sF = sm + (2 + c) * S2;
    const int ex = e % a.E, ey = e / a.E;
    const T ru0 = load2<T, NP>(sU[c], a.u, c, ex, ey, t, valid, a, false);
    (void)ru0;
    __syncthreads();
    const T rU[2] = {(T)0, (T)0};   // no reference subtraction in this form
    const int xb = t * P, yb = t;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 2 * (NP * NP) + (size_t)c * NP * NP + t;
    T r[NP];
    rhs_pass<T, NP, 1>(M, sU[c], sU[0], rU[0], xb, r);
    st_line<T, NP, 1>(sF, xb, r);
    __syncthreads();
    rhs_pass<T, NP, P>(M, sU[c], sU[1], rU[1], yb, r);
    if (valid) {
#pragma unroll
        for (int m = 0; m < NP; ++m) out[m * NP] = to_out(r[m] + sF[yb + m * P]);
    }
}

template <typename T, int NP>
__device__ __forceinline__ void jac2c_body(const OpMats<T, NP>& M, const ElemArgs& a, int e, int t, int c, int el,
                                         bool valid, unsigned char* smem_raw) {
    static_assert(!RefSub<T>::on, "component-parallel bodies assume no reference subtraction");
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * (tiles_per_elem<2>(OP_JAC) + 1) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sW[2] = {sm + 2 * S2, sm + 3 * S2};
    T* sF = sm + (4 + c) * S2;
    const int ex = e % a.E, ey = e / a.E;
    load2<T, NP>(sU[c], a.u, c, ex, ey, t, valid, a, false);
    load2<T, NP>(sW[c], a.w, c, ex, ey, t, valid, a, false);
    __syncthreads();
    const T rz = (T)0;
    const int xb = t * P, yb = t;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 2 * (NP * NP) + (size_t)c * NP * NP + t;
    T r[NP];
    jac_pass<T, NP, 1>(M, sU[c], sW[c], sU[0], sW[0], rz, rz, xb, r);
    st_line<T, NP, 1>(sF, xb, r);
    __syncthreads();
    jac_pass<T, NP, P>(M, sU[c], sW[c], sU[1], sW[1], rz, rz, yb, r);
    if (valid) {
#pragma unroll
        for (int m = 0; m < NP; ++m) out[m * NP] = to_out(r[m] + sF[yb + m * P]);
    }
}

// J^T pass with the line stride as a run-time value: the x and y passes of
// jact2c_body then share one copy of the code.  The fully unrolled double-float
// passes are long straight-line code, and two copies of them overflow the
// instruction cache once the warps of an SM drift apart.
template <typename T, int NP, int D>
__device__ __forceinline__ void jact_pass_rt(const OpMats<T, NP>& M, T* const* sU, T* const* sZ, const T* rU, int l,
                                             int d, int base, int stride, T (&r)[NP]) {
    T z[NP], u[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        z[m] = sZ[l][base + m * stride];
        u[m] = with_ref(rU[d], sU[d][base + m * stride]);
    }
    gvdd_apply<T, NP>(M.Gv, M.Dd, z, u, r);
    if (l == d) {
#pragma unroll 1
        for (int c = 0; c < D; ++c) {
            T x[NP], g[NP];
#pragma unroll
            for (int m = 0; m < NP; ++m) x[m] = sU[c][base + m * stride];
            eo_apply<false, T, NP>(M.Dg, x, g);
#pragma unroll
            for (int m = 0; m < NP; ++m) r[m] = fma(-sZ[c][base + m * stride], g[m], r[m]);
        }
    }
}

template <typename T, int NP>
__device__ __forceinline__ void jact2c_body(const OpMats<T, NP>& M, const ElemArgs& a, int e, int t, int l, int el,
                                          bool valid, unsigned char* smem_raw) {
    static_assert(!RefSub<T>::on, "component-parallel bodies assume no reference subtraction");
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * (tiles_per_elem<2>(OP_JACT) + 1) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sZ[2] = {sm + 2 * S2, sm + 3 * S2};
    T* sF = sm + (4 + l) * S2;
    const int ex = e % a.E, ey = e / a.E;
    load2<T, NP>(sU[l], a.u, l, ex, ey, t, valid, a, false);
    load2<T, NP>(sZ[l], a.w, l, ex, ey, t, valid, a, true);
    __syncthreads();
    const T rU[2] = {(T)0, (T)0};
    const int xb = t * P, yb = t;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 2 * (NP * NP) + (size_t)l * NP * NP + t;
#pragma unroll 1
    for (int d = 0; d < 2; ++d) {
        T r[NP];
        jact_pass_rt<T, NP, 2>(M, sU, sZ, rU, l, d, d ? yb : xb, d ? P : 1, r);
        if (d == 0) {
            st_line<T, NP, 1>(sF, xb, r);
            __syncthreads();
        } else if (valid) {
#pragma unroll
            for (int m = 0; m < NP; ++m) out[m * NP] = to_out(r[m] + sF[yb + m * P]);
        }
    }
}

// Block of epb elements: the first half of the block runs component 0 of every
// element, the second half component 1, so that a warp takes one branch of the
// J^T cross term (the launcher makes epb n a multiple of 32 where it can).
template <typename T, int NP>
__global__ void __launch_bounds__(256, 2) op2c_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a, int op) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int half = blockDim.x / 2;
    const int c = threadIdx.x >= half, r = threadIdx.x - c * half;
    const int el = r / NP, t = r % NP;
    const int e = blockIdx.x * (half / NP) + el;
    const bool valid = e < a.nelem;
    if (op == OP_RHS) rhs2c_body<T, NP>(M, a, e, t, c, el, valid, smem_raw);
    else if (op == OP_JAC) jac2c_body<T, NP>(M, a, e, t, c, el, valid, smem_raw);
    else jact2c_body<T, NP>(M, a, e, t, c, el, valid, smem_raw);
}

// ================================================================== d = 1
// One thread per element; everything in registers.
template <typename T, int NP>
__device__ __forceinline__ T load1(T (&x)[NP], const void* g, int e, const ElemArgs& a, bool scale_mult) {
    float ref_hi = 0.f, ref_lo = 0.f;
    if (RefSub<T>::on && !scale_mult) read_pair(a, g, wrap(e * a.N, a.G), ref_hi, ref_lo);
#pragma unroll
    for (int i = 0; i < NP; ++i)
        x[i] = tile_value<T>(a, g, wrap(e * a.N + i, a.G), scale_mult, (int)(i == 0 || i == a.N), ref_hi, ref_lo);
    return (T)ref_hi;
}

template <typename T, int NP>
__global__ void op1_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a, int op) {
    pdl_wait();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.nelem) return;
    T u[NP], f[NP];
    const T ru = load1<T, NP>(u, a.u, e, a, false);
    if (op == OP_RHS) {
        T g[NP];
        Pre<T, NP> p;
        pre_add<T, NP>(u, p);
        eo_apply<false, T, NP>(M.Dg, p, g);
        eo_apply<true, T, NP>(M.Sv, p, f);
#pragma unroll
        for (int m = 0; m < NP; ++m) f[m] = fma(-with_ref(ru, u[m]), g[m], f[m]);
    } else if (op == OP_JAC) {
        T w[NP], gu[NP], gw[NP];
        const T rw = load1<T, NP>(w, a.w, e, a, false);
        Pre<T, NP> p;
        pre_add<T, NP>(w, p);
        eo_apply<false, T, NP>(M.Dg, p, gw);
        eo_apply<true, T, NP>(M.Sv, p, f);
        eo_apply<false, T, NP>(M.Dg, u, gu);
#pragma unroll
        for (int m = 0; m < NP; ++m) f[m] -= fma(with_ref(rw, w[m]), gu[m], with_ref(ru, u[m]) * gw[m]);
    } else {
        T z[NP], uu[NP], gu[NP];
        load1<T, NP>(z, a.w, e, a, true);
#pragma unroll
        for (int m = 0; m < NP; ++m) uu[m] = with_ref(ru, u[m]);
        gvdd_apply<T, NP>(M.Gv, M.Dd, z, uu, f);
        eo_apply<false, T, NP>(M.Dg, u, gu);
#pragma unroll
        for (int m = 0; m < NP; ++m) f[m] = fma(-z[m], gu[m], f[m]);
    }
    auto* o = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * NP;
#pragma unroll
    for (int m = 0; m < NP; ++m) o[m] = to_out(f[m]);
}

}  // namespace semk
