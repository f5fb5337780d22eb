// Element kernels of d = 3 with many points per direction (n >= 13): the same
// passes as rhs3/jac3/jact3 (op_elem.cuh) with fewer shared-memory tiles.  In
// FP64 this is what makes one element's tiles fit the 227 KB of an SM (with
// n = 16 the plain kernels would need 5 tiles of 16 x 16 x 17 doubles, 174 KB,
// for F and 8, 278 KB, for J and J^T); in FP32 it lets two blocks share an SM.
//
//  * One element per block (n^2 threads).
//  * F: the x and y passes accumulate into one partial tile (an extra barrier
//    between them) instead of two; 4 tiles (139 KB at n = 16).
//  * J and J^T: no partial tiles.  The x pass writes its line of the result to
//    the element-local output in global memory, the y pass adds its line to it
//    and the z pass adds the stored sum to its own line and writes the result.
//    The output of one element stays in L2 between the passes; __syncthreads
//    orders the global accesses of the block.  6 tiles (209 KB at n = 16).
//  * The sums are formed in the same order as in the plain kernels, (x + y) + z,
//    so FP64 results are the same bits.  (Double-float kernels add their
//    partial lines in FP64 here.)
#pragma once
#include "op_elem.cuh"

namespace semk {

template <typename T, int NP>
__host__ __device__ constexpr bool lean3() {
    return NP >= 13;
}

// Lean kernels for one operator: always from n = 13, and for the double-float J^T at
// n = 12.  Its eight 8-byte tiles per element take 120 KB there, which leaves one
// 144-thread block per SM (4.5 warps); the six lean tiles let two blocks share it, and
// J^T went from 8.0 to 9.6 GDOF/s at order 11.  At n = 10 the lean kernel measured slower
// (12.1 against 10.1 GDOF/s at order 9): three plain blocks already fit there.  (The lean
// double-float J needs 255 registers at n = 12, so J keeps the plain kernel.)
template <typename T, int NP>
__host__ __device__ constexpr bool lean3_op(int op) {
    return lean3<T, NP>() || (std::is_same<T, dfloat>::value && NP == 12 && op == OP_JACT);
}

// Whether any operator of (T, NP) uses the lean kernels (they are compiled only then).
template <typename T, int NP>
__host__ __device__ constexpr bool lean3_any() {
    return lean3<T, NP>() || (std::is_same<T, dfloat>::value && NP == 12);
}

template <int D>
__host__ __device__ constexpr int lean_tiles_per_elem(int op) {
    return op == OP_RHS ? D + 1 : 2 * D;
}

template <typename T, int NP>
__device__ __forceinline__ void df3_lean_body(const OpMats<T, NP>& M, const ElemArgs& a, int op, T* const* sU,
                                              T* const* sV, T* sF, const T* rU, const T* rV, int e, int t);

template <typename T, int NP>
__global__ void __launch_bounds__(NP * NP)
rhs3_lean_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int t = threadIdx.x;
    const int e = blockIdx.x;
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sF = sm + 3 * S3;
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) rU[c] = load3<T, NP>(sU[c], a.u, c, ex, ey, ez, t, true, a, false);
    __syncthreads();
    if constexpr (shared_pass3<T, NP>()) {
        df3_lean_body<T, NP>(M, a, OP_RHS, sU, sU, sF, rU, rU, e, t);
        return;
    }
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP) + (t / NP) * NP + t % NP;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        T r[NP];
        rhs_pass<T, NP, 1>(M, sU[c], sU[0], rU[0], xb, r);
        st_line<T, NP, 1>(sF, xb, r);
        __syncthreads();
        rhs_pass<T, NP, P>(M, sU[c], sU[1], rU[1], yb, r);
#pragma unroll
        for (int m = 0; m < NP; ++m) sF[yb + m * P] += r[m];
        __syncthreads();
        rhs_pass<T, NP, S2>(M, sU[c], sU[2], rU[2], zb, r);
#pragma unroll
        for (int m = 0; m < NP; ++m) out[(size_t)c * NP * NP * NP + m * NP * NP] = to_out(r[m] + sF[zb + m * S2]);
        __syncthreads();
    }
}

// Element-local output of element e, component c: node (i, j, k) at k n^2 + j n + i.
// x-line of thread t: (j, k) = (t % n, t / n), nodes i = m;  y-line: (i, k), nodes j = m;
// z-line: (i, j), nodes k = m.
template <typename T, int NP, typename O>
__device__ __forceinline__ void lean_out_x(O* o, int t, const T (&r)[NP]) {
    O* p = o + (t / NP) * NP * NP + (t % NP) * NP;   // n contiguous values, 16-byte aligned for n % 2 == 0
    if constexpr (sizeof(O) == 8 && NP % 2 == 0) {
#pragma unroll
        for (int m = 0; m < NP; m += 2) reinterpret_cast<double2*>(p)[m / 2] = make_double2(to_out(r[m]), to_out(r[m + 1]));
    } else {
#pragma unroll
        for (int m = 0; m < NP; ++m) p[m] = to_out(r[m]);
    }
}
template <typename T, int NP, typename O>
__device__ __forceinline__ void lean_add_y(O* o, int t, const T (&r)[NP]) {
    O* p = o + (t / NP) * NP * NP + (t % NP);
#pragma unroll
    for (int m = 0; m < NP; ++m) p[m * NP] += to_out(r[m]);
}
template <typename T, int NP, typename O>
__device__ __forceinline__ void lean_add_z(O* o, int t, const T (&r)[NP]) {
    O* p = o + (t / NP) * NP + (t % NP);
#pragma unroll
    for (int m = 0; m < NP; ++m) p[m * NP * NP] += to_out(r[m]);
}

// Double-float lean body: the three passes from one copy of the pass code (see
// df3_body); F keeps its partial sum in one tile, J and J^T in the output.
template <typename T, int NP>
__device__ __forceinline__ void df3_lean_body(const OpMats<T, NP>& M, const ElemArgs& a, int op, T* const* sU,
                                              T* const* sV, T* sF, const T* rU, const T* rV, int e, int t) {
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2;
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP);
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        auto* oc = out + (size_t)c * NP * NP * NP;
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            const int base = d == 0 ? xb : (d == 1 ? yb : zb);
            const int stride = d == 0 ? 1 : (d == 1 ? P : S2);
            const T* sUd = d == 0 ? sU[0] : (d == 1 ? sU[1] : sU[2]);
            T r[NP];
            if (op == OP_RHS) {
                rhs_pass_rt<T, NP>(M, sU[c], sUd, rU[d], base, stride, r);
                if (d == 0) {
#pragma unroll
                    for (int m = 0; m < NP; ++m) sF[base + m * stride] = r[m];
                } else if (d == 1) {
#pragma unroll
                    for (int m = 0; m < NP; ++m) sF[base + m * stride] += r[m];
                } else {
#pragma unroll
                    for (int m = 0; m < NP; ++m) oc[(t / NP) * NP + t % NP + m * NP * NP] = to_out(r[m] + sF[zb + m * S2]);
                }
            } else {
                if (op == OP_JAC) {
                    const T* sVd = d == 0 ? sV[0] : (d == 1 ? sV[1] : sV[2]);
                    jac_pass_rt<T, NP>(M, sU[c], sV[c], sUd, sVd, rU[d], rV[d], base, stride, r);
                } else {
                    jact_pass_rt<T, NP, 3>(M, sU, sV, rU, c, d, base, stride, r);
                }
                if (d == 0) lean_out_x<T, NP>(oc, t, r);
                else if (d == 1) lean_add_y<T, NP>(oc, t, r);
                else lean_add_z<T, NP>(oc, t, r);
            }
            __syncthreads();
        }
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(NP * NP)
jac3_lean_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int t = threadIdx.x;
    const int e = blockIdx.x;
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sW[3] = {sm + 3 * S3, sm + 4 * S3, sm + 5 * S3};
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3], rW[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        rU[c] = load3<T, NP>(sU[c], a.u, c, ex, ey, ez, t, true, a, false);
        rW[c] = load3<T, NP>(sW[c], a.w, c, ex, ey, ez, t, true, a, false);
    }
    __syncthreads();
    if constexpr (shared_pass3<T, NP>()) {
        df3_lean_body<T, NP>(M, a, OP_JAC, sU, sW, nullptr, rU, rW, e, t);
        return;
    }
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP);
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        auto* oc = out + (size_t)c * NP * NP * NP;
        T r[NP];
        jac_pass<T, NP, 1>(M, sU[c], sW[c], sU[0], sW[0], rU[0], rW[0], xb, r);
        lean_out_x<T, NP>(oc, t, r);
        __syncthreads();
        jac_pass<T, NP, P>(M, sU[c], sW[c], sU[1], sW[1], rU[1], rW[1], yb, r);
        lean_add_y<T, NP>(oc, t, r);
        __syncthreads();
        jac_pass<T, NP, S2>(M, sU[c], sW[c], sU[2], sW[2], rU[2], rW[2], zb, r);
        lean_add_z<T, NP>(oc, t, r);
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(NP * NP)
jact3_lean_kernel(const __grid_constant__ OpMats<T, NP> M, const ElemArgs a) {
    using Tl = Tile<NP>;
    constexpr int P = Tl::P, S2 = Tl::S2, S3 = Tl::S3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();
    const int t = threadIdx.x;
    const int e = blockIdx.x;
    T* sm = reinterpret_cast<T*>(smem_raw);
    T* sU[3] = {sm, sm + S3, sm + 2 * S3};
    T* sZ[3] = {sm + 3 * S3, sm + 4 * S3, sm + 5 * S3};
    const int ex = e % a.E, ey = (e / a.E) % a.E, ez = e / (a.E * a.E);
    T rU[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        rU[c] = load3<T, NP>(sU[c], a.u, c, ex, ey, ez, t, true, a, false);
        load3<T, NP>(sZ[c], a.w, c, ex, ey, ez, t, true, a, true);
    }
    __syncthreads();
    if constexpr (shared_pass3<T, NP>()) {
        df3_lean_body<T, NP>(M, a, OP_JACT, sU, sZ, nullptr, rU, rU, e, t);
        return;
    }
    const int xb = t * P, yb = (t / NP) * S2 + t % NP, zb = (t / NP) * P + t % NP;
    auto* out = reinterpret_cast<typename OutT<T>::type*>(a.lvec) + (size_t)e * 3 * (NP * NP * NP);
#pragma unroll 1
    for (int l = 0; l < 3; ++l) {
        auto* ol = out + (size_t)l * NP * NP * NP;
        T r[NP];
        jact_pass<T, NP, 1, 3>(M, sU, sZ, rU, l, 0, xb, r);
        lean_out_x<T, NP>(ol, t, r);
        __syncthreads();
        jact_pass<T, NP, P, 3>(M, sU, sZ, rU, l, 1, yb, r);
        lean_add_y<T, NP>(ol, t, r);
        __syncthreads();
        jact_pass<T, NP, S2, 3>(M, sU, sZ, rU, l, 2, zb, r);
        lean_add_z<T, NP>(ol, t, r);
    }
}

}  // namespace semk
