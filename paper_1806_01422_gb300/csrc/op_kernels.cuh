// Element kernels of the matrix-free spectral-element Burgers operators.
//
// Method (arXiv:1806.01422, Sec. 3.2-3.3): on every element the operator is a
// sequence of 1D contractions with an (N+1)x(N+1) matrix along one tensor
// direction at a time (sum factorisation, eqs. rhsvec / jacvec / jactransvec),
// pointwise products at the GLL nodes, and a sum over the elements sharing a
// node (gather-scatter / direct stiffness summation).
//
// Reformulation used here (exact up to rounding).  With GLL collocation the element mass B is diagonal and, on a
// uniform periodic grid, equal in every element that shares a node, so
//   F = M^-1 Q^T r(Qu)   ==   F(node) = (1/k) sum_{e sharing node} r_e / B
// with k the number of sharing elements (1, 2, 4 or 8).  Dividing the weak
// residual by B turns D_j^T B D_j into (W^-1 Dhat^T W) Dhat along direction j:
// every mass factor disappears into 1D matrices.  For the transpose, with
// zhat = v / k (so B z = zhat for z = M^-1 v):
//   (L^T z)_l = sum_j Dd_j [ Vz_j zhat_l + U_j zhat_l ] - sum_c zhat_c Dg_l U_c,
// Vz = nu (2/h) W Dhat W^-1, Dd = -(2/h) Dhat^T, Dg = (2/h) Dhat.
//
// Every 1D matrix here is centro-antisymmetric (A[n-1-i][n-1-j] = -A[i][j],
// because the GLL nodes are symmetric), so a contraction of a line of n values
// costs n^2/2 multiply-adds plus 2n adds (even-odd split) instead of n^2.
//
// Thread layout: one thread per grid line of an element.  A contraction pass
// along direction x, y or z lets each thread load its line from a padded
// shared-memory tile into registers, contract, and store.  d = 3 uses n^2
// threads per element, d = 2 uses n, d = 1 one thread per element.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace semk {

// Which operator an element kernel evaluates.
enum OpKind { OP_RHS = 0, OP_JAC = 1, OP_JACT = 2 };

// ---------------------------------------------------------------- even-odd matrices
// A centro-antisymmetric n x n matrix A is stored as
//   e[i][j] = (A[i][j] + A[i][n-1-j]) / 2   (j < H), e[i][H] = A[i][H] (odd n)
//   o[i][j] = (A[i][j] - A[i][n-1-j]) / 2   (j < H)
//   m[j]    =  A[H][j]                      (odd n: middle row, j < H)
// with H = n/2; then for i < H
//   y_i = a_i + b_i,  y_{n-1-i} = b_i - a_i,  a = e xe, b = o xo,
//   xe_j = x_j + x_{n-1-j} (xe_H = x_H), xo_j = x_j - x_{n-1-j},
// and for odd n y_H = m . xo.
template <typename T, int NP>
struct EOMat {
    static constexpr int H = NP / 2;
    static constexpr int HE = NP / 2 + (NP & 1);
    T e[H][HE];
    T o[H][H];
    T m[H];
};

template <typename T, int NP>
struct OpMats {
    EOMat<T, NP> Dg;  // (2/h) Dhat                       gradient
    EOMat<T, NP> Dv;  // -nu (2/h) W^-1 Dhat^T W           viscous divergence of a gradient (F, J)
    EOMat<T, NP> Vz;  // nu (2/h) W Dhat W^-1              viscous flux from zhat (J^T)
    EOMat<T, NP> Dd;  // -(2/h) Dhat^T                     divergence (J^T)
};

// y = A x
template <typename T, int NP>
__device__ __forceinline__ void eo_apply(const EOMat<T, NP>& A, const T (&x)[NP], T (&y)[NP]) {
    constexpr int H = NP / 2;
    T xe[H + (NP & 1)], xo[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        xe[j] = x[j] + x[NP - 1 - j];
        xo[j] = x[j] - x[NP - 1 - j];
    }
    if constexpr (NP & 1) xe[H] = x[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        T a = A.e[i][0] * xe[0];
#pragma unroll
        for (int j = 1; j < H + (NP & 1); ++j) a = fma(A.e[i][j], xe[j], a);
        T b = A.o[i][0] * xo[0];
#pragma unroll
        for (int j = 1; j < H; ++j) b = fma(A.o[i][j], xo[j], b);
        y[i] = a + b;
        y[NP - 1 - i] = b - a;
    }
    if constexpr (NP & 1) {
        T c = A.m[0] * xo[0];
#pragma unroll
        for (int j = 1; j < H; ++j) c = fma(A.m[j], xo[j], c);
        y[H] = c;
    }
}

// y += A x
template <typename T, int NP>
__device__ __forceinline__ void eo_apply_add(const EOMat<T, NP>& A, const T (&x)[NP], T (&y)[NP]) {
    T t[NP];
    eo_apply<T, NP>(A, x, t);
#pragma unroll
    for (int m = 0; m < NP; ++m) y[m] += t[m];
}

// ---------------------------------------------------------------- tile geometry
// Shared-memory tile of one scalar field of one element: rows of n values along
// x padded to an odd length P so that the line passes are free of (8-byte)
// bank conflicts.  Index of node (i, j, k): (k*n + j)*P + i.
template <int NP>
struct Tile {
    static constexpr int P = NP | 1;
    static constexpr int S2 = NP * P;        // 2D tile size / 3D z-stride
    static constexpr int S3 = NP * NP * P;   // 3D tile size
};

template <typename T, int NP, int STRIDE>
__device__ __forceinline__ void ld_line(const T* s, int base, T (&x)[NP]) {
#pragma unroll
    for (int m = 0; m < NP; ++m) x[m] = s[base + m * STRIDE];
}
template <typename T, int NP, int STRIDE>
__device__ __forceinline__ void st_line(T* s, int base, const T (&x)[NP]) {
#pragma unroll
    for (int m = 0; m < NP; ++m) s[base + m * STRIDE] = x[m];
}

// Launch-time arguments shared by the element kernels.
struct ElemArgs {
    const double* u;   // state at which the operator is evaluated (global, SoA)
    const double* w;   // second input: w for J, v for J^T (unused by F)
    void* lvec;        // output: element-local values, [elem][comp][n^d] (unpadded)
    int E, N, G;       // elements per direction, order, unique nodes per direction
    int nelem;         // E^d
};

// Global index of component c at unique node (gz, gy, gx) of a d-dimensional grid.
__device__ __forceinline__ size_t gidx3(int c, int gz, int gy, int gx, int G) {
    return (((size_t)c * G + gz) * G + gy) * G + gx;
}

__device__ __forceinline__ int wrap(int g, int G) { return g >= G ? g - G : g; }

}  // namespace semk
