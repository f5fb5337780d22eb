// Element kernels for F(u), J(u)w and J(u)^T v in d = 1, 2, 3 (arXiv:1806.01422,
// eqs. rhsvec, jacvec, jactransvec).  Each kernel reads the global (unique-node)
// inputs with the periodic scatter Q, computes one element-local result per
// element and writes it to an element-local buffer; the gather-scatter sum
// Q^T (and the 1/k multiplicity scaling for F and J) is done by the assembly
// kernel, which also applies the Runge-Kutta epilogue.
//
// Local results (see op_kernels.cuh for the matrices):
//   F :  f_c   = sum_j Dv_j Dg_j U_c - sum_j U_j Dg_j U_c
//   J :  f_c   = sum_j Dv_j Dg_j W_c - sum_j (W_j Dg_j U_c + U_j Dg_j W_c)
//   JT:  f_l   = sum_j Dd_j (Vz_j Z_l + U_j Z_l) - sum_c Z_c Dg_l U_c,  Z = v / k
// with Dg_j, Dv_j, Vz_j, Dd_j the 1D matrices applied along direction x_j.
#pragma once
#include "op_kernels.cuh"

namespace semk {

template <int D>
__host__ __device__ constexpr int tiles_per_elem(int op) {
    // F: U[d] + G (d-1) + F ; J: U[d] + W[d] + G (d-1) + F + A ; JT: U[d] + Z[d] + G (d-1) + F
    return op == OP_RHS ? (2 * D) : (op == OP_JAC ? (3 * D + 1) : (3 * D));
}

// ------------------------------------------------------------------ loaders
// In the FP32 form each element tile of U (and W) holds U - U_ref, with U_ref
// the value at the element's first node, formed in FP64 before rounding to
// FP32.  The 1D matrices annihilate constants (Dhat 1 = 0), so gradients see
// only the small in-element variation and lose far less to FP32 cancellation;
// pointwise products add U_ref back.  The FP64 form stores U itself (ref = 0).
template <typename T>
struct RefSub {
    static constexpr bool on = sizeof(T) == 4;
};

template <typename T>
__device__ __forceinline__ T with_ref(T ref, T x) {
    if constexpr (RefSub<T>::on) return ref + x;
    else return x;
}

// Load component c of a global field into an element tile (d = 3): thread t of
// the element owns column (i, j) = (t % n, t / n) and walks k.  `scale_mult`
// multiplies each node by 1/k (k = elements sharing it), used for Z = v / k.
// Returns the reference value subtracted from the tile (0 unless FP32 and not Z).
template <typename T, int NP>
__device__ __forceinline__ T load3(T* tile, const double* __restrict__ g, int c, int ex, int ey,
                                   int ez, int t, bool valid, const ElemArgs& a, bool scale_mult) {
    using Tl = Tile<NP>;
    const int i = t % NP, j = t / NP;
    const int N = a.N, G = a.G;
    const int gx = wrap(ex * N + i, G), gy = wrap(ey * N + j, G);
    const bool bij = (i == 0 || i == N), bj = (j == 0 || j == N);
    const T sij = scale_mult ? (T)((bij ? 0.5 : 1.0) * (bj ? 0.5 : 1.0)) : (T)1;
    double ref = 0.0;
    if (RefSub<T>::on && !scale_mult && valid) ref = __ldg(g + gidx3(c, ez * N, ey * N, ex * N, G));
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int gz = wrap(ez * N + k, G);
        T v = (T)0;
        if (valid) {
            const double x = __ldg(g + gidx3(c, gz, gy, gx, G));
            if (RefSub<T>::on && !scale_mult) {
                v = (T)(x - ref);
            } else {
                v = (T)x;
                if (scale_mult) v = v * sij * ((k == 0 || k == N) ? (T)0.5 : (T)1);
            }
        }
        tile[(k * NP + j) * Tl::P + i] = v;
    }
    return (T)ref;
}

// d = 2: thread t owns row j = t and walks i.
template <typename T, int NP>
__device__ __forceinline__ T load2(T* tile, const double* __restrict__ g, int c, int ex, int ey,
                                   int t, bool valid, const ElemArgs& a, bool scale_mult) {
    using Tl = Tile<NP>;
    const int j = t;
    const int N = a.N, G = a.G;
    const int gy = wrap(ey * N + j, G);
    const T sj = (scale_mult && (j == 0 || j == N)) ? (T)0.5 : (T)1;
    const size_t row = ((size_t)c * G + gy) * G;
    double ref = 0.0;
    if (RefSub<T>::on && !scale_mult && valid) ref = __ldg(g + ((size_t)c * G + ey * N) * G + ex * N);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const int gx = wrap(ex * N + i, G);
        T v = (T)0;
        if (valid) {
            const double x = __ldg(g + row + gx);
            if (RefSub<T>::on && !scale_mult) {
                v = (T)(x - ref);
            } else {
                v = (T)x;
                if (scale_mult) v = v * sj * ((i == 0 || i == N) ? (T)0.5 : (T)1);
            }
        }
        tile[j * Tl::P + i] = v;
    }
    return (T)ref;
}

// ================================================================== d = 3
// Line bases of thread t (n^2 threads per element):
//   x-line (j, k) = (t % n, t / n): base t*P,                stride 1
//   y-line (i, k) = (t % n, t / n): base (t/n)*S2 + t % n,   stride P
//   z-line (i, j) = (t % n, t / n): base (t/n)*P + t % n,    stride S2
template <typename T, int NP>
__global__ void rhs3_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP * NP, P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<3>(OP_RHS) * S3;
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sG0 = sm + 3 * S3;
    T* sG1 = sm + 4 * S3;
    T* sF = sm + 5 * S3;
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) rU[c] = load3<T, NP>(sU[c], a.u, c, ex, ey, ez, t, valid, a, false);
    __syncthreads();
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    T* out = reinterpret_cast<T*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP);
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        const T* sUc = sU[c];
        {   // x and y gradients of U_c
            T x[NP], g[NP];
            ld_line<T, NP, 1>(sUc, xb, x);
            eo_apply<T, NP>(M.Dg, x, g);
            st_line<T, NP, 1>(sG0, xb, g);
            ld_line<T, NP, P>(sUc, yb, x);
            eo_apply<T, NP>(M.Dg, x, g);
            st_line<T, NP, P>(sG1, yb, g);
        }
        __syncthreads();
        {   // z gradient, advection, z part of the viscous divergence
            T x[NP], gz[NP], f[NP];
            ld_line<T, NP, S2>(sUc, zb, x);
            eo_apply<T, NP>(M.Dg, x, gz);
            eo_apply<T, NP>(M.Dv, gz, f);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const int id = zb + m * S2;
                T adv = with_ref(rU[0], sU[0][id]) * sG0[id];
                adv = fma(with_ref(rU[1], sU[1][id]), sG1[id], adv);
                adv = fma(with_ref(rU[2], sU[2][id]), gz[m], adv);
                f[m] -= adv;
            }
            st_line<T, NP, S2>(sF, zb, f);
        }
        __syncthreads();
        {   // x part of the viscous divergence
            T g[NP], f[NP];
            ld_line<T, NP, 1>(sG0, xb, g);
            ld_line<T, NP, 1>(sF, xb, f);
            eo_apply_add<T, NP>(M.Dv, g, f);
            st_line<T, NP, 1>(sF, xb, f);
        }
        __syncthreads();
        {   // y part, then the element-local result
            T g[NP], f[NP];
            ld_line<T, NP, P>(sG1, yb, g);
            ld_line<T, NP, P>(sF, yb, f);
            eo_apply_add<T, NP>(M.Dv, g, f);
            if (valid) {
                T* o = out + (size_t)c * (NP * NP * NP) + (t / NP) * NP * NP + t % NP;
#pragma unroll
                for (int m = 0; m < NP; ++m) o[m * NP] = f[m];
            }
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__global__ void jac3_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP * NP, P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<3>(OP_JAC) * S3;
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sW[3] = {sm + 3 * S3, sm + 4 * S3, sm + 5 * S3};
    T* sG0 = sm + 6 * S3;
    T* sG1 = sm + 7 * S3;
    T* sF = sm + 8 * S3;
    T* sA = sm + 9 * S3;
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3], rW[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        rU[c] = load3<T, NP>(sU[c], a.u, c, ex, ey, ez, t, valid, a, false);
        rW[c] = load3<T, NP>(sW[c], a.w, c, ex, ey, ez, t, valid, a, false);
    }
    __syncthreads();
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    T* out = reinterpret_cast<T*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP);
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        {
            T x[NP], gw[NP], gu[NP], f[NP];
            // x: gradient of W_c to sG0, advection x-term to sF
            ld_line<T, NP, 1>(sW[c], xb, x);
            eo_apply<T, NP>(M.Dg, x, gw);
            st_line<T, NP, 1>(sG0, xb, gw);
            ld_line<T, NP, 1>(sU[c], xb, x);
            eo_apply<T, NP>(M.Dg, x, gu);
#pragma unroll
            for (int m = 0; m < NP; ++m)
                f[m] = -fma(with_ref(rW[0], sW[0][xb + m]), gu[m], with_ref(rU[0], sU[0][xb + m]) * gw[m]);
            st_line<T, NP, 1>(sF, xb, f);
            // y: gradient of W_c to sG1, advection y-term to sA
            ld_line<T, NP, P>(sW[c], yb, x);
            eo_apply<T, NP>(M.Dg, x, gw);
            st_line<T, NP, P>(sG1, yb, gw);
            ld_line<T, NP, P>(sU[c], yb, x);
            eo_apply<T, NP>(M.Dg, x, gu);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const int id = yb + m * P;
                f[m] = -fma(with_ref(rW[1], sW[1][id]), gu[m], with_ref(rU[1], sU[1][id]) * gw[m]);
            }
            st_line<T, NP, P>(sA, yb, f);
        }
        __syncthreads();
        {
            T x[NP], gw[NP], gu[NP], f[NP];
            ld_line<T, NP, S2>(sW[c], zb, x);
            eo_apply<T, NP>(M.Dg, x, gw);
            ld_line<T, NP, S2>(sU[c], zb, x);
            eo_apply<T, NP>(M.Dg, x, gu);
            eo_apply<T, NP>(M.Dv, gw, f);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const int id = zb + m * S2;
                const T adv = fma(with_ref(rW[2], sW[2][id]), gu[m], with_ref(rU[2], sU[2][id]) * gw[m]);
                f[m] = (f[m] - adv) + (sF[id] + sA[id]);
            }
            st_line<T, NP, S2>(sF, zb, f);
        }
        __syncthreads();
        {
            T g[NP], f[NP];
            ld_line<T, NP, 1>(sG0, xb, g);
            ld_line<T, NP, 1>(sF, xb, f);
            eo_apply_add<T, NP>(M.Dv, g, f);
            st_line<T, NP, 1>(sF, xb, f);
        }
        __syncthreads();
        {
            T g[NP], f[NP];
            ld_line<T, NP, P>(sG1, yb, g);
            ld_line<T, NP, P>(sF, yb, f);
            eo_apply_add<T, NP>(M.Dv, g, f);
            if (valid) {
                T* o = out + (size_t)c * (NP * NP * NP) + (t / NP) * NP * NP + t % NP;
#pragma unroll
                for (int m = 0; m < NP; ++m) o[m * NP] = f[m];
            }
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__global__ void jact3_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP * NP, P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<3>(OP_JACT) * S3;
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sZ[3] = {sm + 3 * S3, sm + 4 * S3, sm + 5 * S3};
    T* sG0 = sm + 6 * S3;
    T* sG1 = sm + 7 * S3;
    T* sF = sm + 8 * S3;
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        rU[c] = load3<T, NP>(sU[c], a.u, c, ex, ey, ez, t, valid, a, false);
        load3<T, NP>(sZ[c], a.w, c, ex, ey, ez, t, valid, a, true);
    }
    __syncthreads();
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    T* out = reinterpret_cast<T*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP);
#pragma unroll 1
    for (int l = 0; l < 3; ++l) {
        const T* sZl = sZ[l];
        {
            T z[NP], q[NP];
            // x: flux q_x = Vz Z_l + U_x Z_l
            ld_line<T, NP, 1>(sZl, xb, z);
            eo_apply<T, NP>(M.Vz, z, q);
#pragma unroll
            for (int m = 0; m < NP; ++m) q[m] = fma(with_ref(rU[0], sU[0][xb + m]), z[m], q[m]);
            st_line<T, NP, 1>(sG0, xb, q);
            if (l == 0) {  // reaction term along x: -sum_c Z_c Dg_x U_c
                T acc[NP], x[NP], g[NP];
#pragma unroll
                for (int m = 0; m < NP; ++m) acc[m] = (T)0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ld_line<T, NP, 1>(sU[c], xb, x);
                    eo_apply<T, NP>(M.Dg, x, g);
#pragma unroll
                    for (int m = 0; m < NP; ++m) acc[m] = fma(sZ[c][xb + m], g[m], acc[m]);
                }
#pragma unroll
                for (int m = 0; m < NP; ++m) acc[m] = -acc[m];
                st_line<T, NP, 1>(sF, xb, acc);
            }
            // y: flux q_y
            ld_line<T, NP, P>(sZl, yb, z);
            eo_apply<T, NP>(M.Vz, z, q);
#pragma unroll
            for (int m = 0; m < NP; ++m) q[m] = fma(with_ref(rU[1], sU[1][yb + m * P]), z[m], q[m]);
            st_line<T, NP, P>(sG1, yb, q);
            if (l == 1) {
                T acc[NP], x[NP], g[NP];
#pragma unroll
                for (int m = 0; m < NP; ++m) acc[m] = (T)0;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ld_line<T, NP, P>(sU[c], yb, x);
                    eo_apply<T, NP>(M.Dg, x, g);
#pragma unroll
                    for (int m = 0; m < NP; ++m) acc[m] = fma(sZ[c][yb + m * P], g[m], acc[m]);
                }
#pragma unroll
                for (int m = 0; m < NP; ++m) acc[m] = -acc[m];
                st_line<T, NP, P>(sF, yb, acc);
            }
        }
        __syncthreads();
        {   // z: flux, its divergence, and the z reaction term (l == 2)
            T z[NP], q[NP], f[NP];
            ld_line<T, NP, S2>(sZl, zb, z);
            eo_apply<T, NP>(M.Vz, z, q);
#pragma unroll
            for (int m = 0; m < NP; ++m) q[m] = fma(with_ref(rU[2], sU[2][zb + m * S2]), z[m], q[m]);
            eo_apply<T, NP>(M.Dd, q, f);
            if (l == 2) {
                T x[NP], g[NP];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ld_line<T, NP, S2>(sU[c], zb, x);
                    eo_apply<T, NP>(M.Dg, x, g);
#pragma unroll
                    for (int m = 0; m < NP; ++m) f[m] = fma(-sZ[c][zb + m * S2], g[m], f[m]);
                }
            } else {
#pragma unroll
                for (int m = 0; m < NP; ++m) f[m] += sF[zb + m * S2];
            }
            st_line<T, NP, S2>(sF, zb, f);
        }
        __syncthreads();
        {
            T q[NP], f[NP];
            ld_line<T, NP, 1>(sG0, xb, q);
            ld_line<T, NP, 1>(sF, xb, f);
            eo_apply_add<T, NP>(M.Dd, q, f);
            st_line<T, NP, 1>(sF, xb, f);
        }
        __syncthreads();
        {
            T q[NP], f[NP];
            ld_line<T, NP, P>(sG1, yb, q);
            ld_line<T, NP, P>(sF, yb, f);
            eo_apply_add<T, NP>(M.Dd, q, f);
            if (valid) {
                T* o = out + (size_t)l * (NP * NP * NP) + (t / NP) * NP * NP + t % NP;
#pragma unroll
                for (int m = 0; m < NP; ++m) o[m * NP] = f[m];
            }
        }
        __syncthreads();
    }
}

// ================================================================== d = 2
// n threads per element.  x-line j = t: base t*P, stride 1; y-line i = t: base t,
// stride P.  The last pass runs along y so that the element-local output of a
// warp is written in contiguous rows.
template <typename T, int NP>
__global__ void rhs2_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP, P = Tl::P, S2 = Tl::S2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<2>(OP_RHS) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sG1 = sm + 2 * S2;
    T* sF = sm + 3 * S2;
    const int ex = e % a.E, ey = e / a.E;
    T rU[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) rU[c] = load2<T, NP>(sU[c], a.u, c, ex, ey, t, valid, a, false);
    __syncthreads();
    const int xb = t * P, yb = t;
    T* out = reinterpret_cast<T*>(a.lvec) + (size_t)e * 2 * (NP * NP);
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        {
            T x[NP], g[NP];
            ld_line<T, NP, P>(sU[c], yb, x);
            eo_apply<T, NP>(M.Dg, x, g);
            st_line<T, NP, P>(sG1, yb, g);
        }
        __syncthreads();
        {
            T x[NP], gx[NP], f[NP];
            ld_line<T, NP, 1>(sU[c], xb, x);
            eo_apply<T, NP>(M.Dg, x, gx);
            eo_apply<T, NP>(M.Dv, gx, f);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const int id = xb + m;
                const T adv = fma(with_ref(rU[1], sU[1][id]), sG1[id], with_ref(rU[0], sU[0][id]) * gx[m]);
                f[m] -= adv;
            }
            st_line<T, NP, 1>(sF, xb, f);
        }
        __syncthreads();
        {
            T g[NP], f[NP];
            ld_line<T, NP, P>(sG1, yb, g);
            ld_line<T, NP, P>(sF, yb, f);
            eo_apply_add<T, NP>(M.Dv, g, f);
            if (valid) {
                T* o = out + (size_t)c * (NP * NP) + t;
#pragma unroll
                for (int m = 0; m < NP; ++m) o[m * NP] = f[m];
            }
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__global__ void jac2_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP, P = Tl::P, S2 = Tl::S2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<2>(OP_JAC) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sW[2] = {sm + 2 * S2, sm + 3 * S2};
    T* sG1 = sm + 4 * S2;
    T* sF = sm + 5 * S2;
    const int ex = e % a.E, ey = e / a.E;
    T rU[2], rW[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        rU[c] = load2<T, NP>(sU[c], a.u, c, ex, ey, t, valid, a, false);
        rW[c] = load2<T, NP>(sW[c], a.w, c, ex, ey, t, valid, a, false);
    }
    __syncthreads();
    const int xb = t * P, yb = t;
    T* out = reinterpret_cast<T*>(a.lvec) + (size_t)e * 2 * (NP * NP);
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        {
            T x[NP], gw[NP], gu[NP], f[NP];
            ld_line<T, NP, P>(sW[c], yb, x);
            eo_apply<T, NP>(M.Dg, x, gw);
            st_line<T, NP, P>(sG1, yb, gw);
            ld_line<T, NP, P>(sU[c], yb, x);
            eo_apply<T, NP>(M.Dg, x, gu);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const int id = yb + m * P;
                f[m] = -fma(with_ref(rW[1], sW[1][id]), gu[m], with_ref(rU[1], sU[1][id]) * gw[m]);
            }
            st_line<T, NP, P>(sF, yb, f);
        }
        __syncthreads();
        {
            T x[NP], gw[NP], gu[NP], f[NP];
            ld_line<T, NP, 1>(sW[c], xb, x);
            eo_apply<T, NP>(M.Dg, x, gw);
            ld_line<T, NP, 1>(sU[c], xb, x);
            eo_apply<T, NP>(M.Dg, x, gu);
            eo_apply<T, NP>(M.Dv, gw, f);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                const int id = xb + m;
                const T adv = fma(with_ref(rW[0], sW[0][id]), gu[m], with_ref(rU[0], sU[0][id]) * gw[m]);
                f[m] = (f[m] - adv) + sF[id];
            }
            st_line<T, NP, 1>(sF, xb, f);
        }
        __syncthreads();
        {
            T g[NP], f[NP];
            ld_line<T, NP, P>(sG1, yb, g);
            ld_line<T, NP, P>(sF, yb, f);
            eo_apply_add<T, NP>(M.Dv, g, f);
            if (valid) {
                T* o = out + (size_t)c * (NP * NP) + t;
#pragma unroll
                for (int m = 0; m < NP; ++m) o[m * NP] = f[m];
            }
        }
        __syncthreads();
    }
}

template <typename T, int NP>
__global__ void jact2_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int TPE = NP, P = Tl::P, S2 = Tl::S2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int el = threadIdx.x / TPE, t = threadIdx.x % TPE;
    const int e = blockIdx.x * (blockDim.x / TPE) + el;
    const bool valid = e < a.nelem;
    T* sm = reinterpret_cast<T*>(smem_raw) + (size_t)el * tiles_per_elem<2>(OP_JACT) * S2;
    T* sU[2] = {sm, sm + S2};
    T* sZ[2] = {sm + 2 * S2, sm + 3 * S2};
    T* sG1 = sm + 4 * S2;
    T* sF = sm + 5 * S2;
    const int ex = e % a.E, ey = e / a.E;
    T rU[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        rU[c] = load2<T, NP>(sU[c], a.u, c, ex, ey, t, valid, a, false);
        load2<T, NP>(sZ[c], a.w, c, ex, ey, t, valid, a, true);
    }
    __syncthreads();
    const int xb = t * P, yb = t;
    T* out = reinterpret_cast<T*>(a.lvec) + (size_t)e * 2 * (NP * NP);
#pragma unroll 1
    for (int l = 0; l < 2; ++l) {
        {   // y: flux q_y, and the y reaction term when l == 1
            T z[NP], q[NP];
            ld_line<T, NP, P>(sZ[l], yb, z);
            eo_apply<T, NP>(M.Vz, z, q);
#pragma unroll
            for (int m = 0; m < NP; ++m) q[m] = fma(with_ref(rU[1], sU[1][yb + m * P]), z[m], q[m]);
            st_line<T, NP, P>(sG1, yb, q);
            if (l == 1) {
                T acc[NP], x[NP], g[NP];
#pragma unroll
                for (int m = 0; m < NP; ++m) acc[m] = (T)0;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    ld_line<T, NP, P>(sU[c], yb, x);
                    eo_apply<T, NP>(M.Dg, x, g);
#pragma unroll
                    for (int m = 0; m < NP; ++m) acc[m] = fma(sZ[c][yb + m * P], g[m], acc[m]);
                }
#pragma unroll
                for (int m = 0; m < NP; ++m) acc[m] = -acc[m];
                st_line<T, NP, P>(sF, yb, acc);
            }
        }
        __syncthreads();
        {   // x: flux, its divergence, the x reaction term when l == 0
            T z[NP], q[NP], f[NP];
            ld_line<T, NP, 1>(sZ[l], xb, z);
            eo_apply<T, NP>(M.Vz, z, q);
#pragma unroll
            for (int m = 0; m < NP; ++m) q[m] = fma(with_ref(rU[0], sU[0][xb + m]), z[m], q[m]);
            eo_apply<T, NP>(M.Dd, q, f);
            if (l == 0) {
                T x[NP], g[NP];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    ld_line<T, NP, 1>(sU[c], xb, x);
                    eo_apply<T, NP>(M.Dg, x, g);
#pragma unroll
                    for (int m = 0; m < NP; ++m) f[m] = fma(-sZ[c][xb + m], g[m], f[m]);
                }
            } else {
#pragma unroll
                for (int m = 0; m < NP; ++m) f[m] += sF[xb + m];
            }
            st_line<T, NP, 1>(sF, xb, f);
        }
        __syncthreads();
        {
            T q[NP], f[NP];
            ld_line<T, NP, P>(sG1, yb, q);
            ld_line<T, NP, P>(sF, yb, f);
            eo_apply_add<T, NP>(M.Dd, q, f);
            if (valid) {
                T* o = out + (size_t)l * (NP * NP) + t;
#pragma unroll
                for (int m = 0; m < NP; ++m) o[m * NP] = f[m];
            }
        }
        __syncthreads();
    }
}

// ================================================================== d = 1
// One thread per element; everything in registers.
template <typename T, int NP>
__device__ __forceinline__ T load1(T (&x)[NP], const double* __restrict__ g, int e, const ElemArgs& a,
                                   bool scale_mult) {
    const double ref = (RefSub<T>::on && !scale_mult) ? __ldg(g + wrap(e * a.N, a.G)) : 0.0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const double v = __ldg(g + wrap(e * a.N + i, a.G));
        if (RefSub<T>::on && !scale_mult) {
            x[i] = (T)(v - ref);
        } else {
            x[i] = (T)v;
            if (scale_mult && (i == 0 || i == a.N)) x[i] *= (T)0.5;
        }
    }
    return (T)ref;
}

template <typename T, int NP>
__global__ void op1_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a, int op) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.nelem) return;
    T u[NP], f[NP];
    const T ru = load1<T, NP>(u, a.u, e, a, false);
    if (op == OP_RHS) {
        T g[NP];
        eo_apply<T, NP>(M.Dg, u, g);
        eo_apply<T, NP>(M.Dv, g, f);
#pragma unroll
        for (int m = 0; m < NP; ++m) f[m] = fma(-with_ref(ru, u[m]), g[m], f[m]);
    } else if (op == OP_JAC) {
        T w[NP], gu[NP], gw[NP];
        const T rw = load1<T, NP>(w, a.w, e, a, false);
        eo_apply<T, NP>(M.Dg, u, gu);
        eo_apply<T, NP>(M.Dg, w, gw);
        eo_apply<T, NP>(M.Dv, gw, f);
#pragma unroll
        for (int m = 0; m < NP; ++m) f[m] -= fma(with_ref(rw, w[m]), gu[m], with_ref(ru, u[m]) * gw[m]);
    } else {
        T z[NP], q[NP], gu[NP];
        load1<T, NP>(z, a.w, e, a, true);
        eo_apply<T, NP>(M.Vz, z, q);
#pragma unroll
        for (int m = 0; m < NP; ++m) q[m] = fma(with_ref(ru, u[m]), z[m], q[m]);
        eo_apply<T, NP>(M.Dd, q, f);
        eo_apply<T, NP>(M.Dg, u, gu);
#pragma unroll
        for (int m = 0; m < NP; ++m) f[m] = fma(-z[m], gu[m], f[m]);
    }
    T* o = reinterpret_cast<T*>(a.lvec) + (size_t)e * NP;
#pragma unroll
    for (int m = 0; m < NP; ++m) o[m] = f[m];
}

}  // namespace semk
