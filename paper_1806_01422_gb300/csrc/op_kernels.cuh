// Element kernels of the matrix-free spectral-element Burgers operators.
//
// Method (arXiv:1806.01422, Sec. 3.2-3.3): on every element the operator is a
// sequence of 1D contractions with an (N+1)x(N+1) matrix along one tensor
// direction at a time (sum factorisation, eqs. rhsvec / jacvec / jactransvec),
// pointwise products at the GLL nodes, and a sum over the elements sharing a
// node (gather-scatter / direct stiffness summation).
//
// Reformulation used here (exact up to rounding).  With GLL collocation the
// element mass B is diagonal and, on a uniform periodic grid, equal in every
// element that shares a node, so
//   F = M^-1 Q^T r(Qu)   ==   F(node) = (1/k) sum_{e sharing node} r_e / B
// with k the number of sharing elements (1, 2, 4 or 8).  Dividing the weak
// residual by B turns the viscous term nu D_j^T B D_j along direction j into
// the 1D second-derivative matrix Sv = -nu (2/h)^2 W^-1 Dhat^T W Dhat, applied
// along j: every mass factor folds into 1D matrices.  For the transpose, with
// zhat = v / k (so B z = zhat for z = M^-1 v):
//   (L^T z)_l = sum_j Dd_j (Gv_j zhat_l + U_j zhat_l) - sum_c zhat_c Dg_l U_c,
// Gv = nu (2/h) W Dhat W^-1, Dd = -(2/h) Dhat^T, Dg = (2/h) Dhat: the viscous flux
// and the advective flux of J^T share one divergence contraction (Dd Gv is the
// viscous matrix -nu (2/h)^2 Dhat^T W Dhat W^-1).
//
// Dg, Dd and Gv are centro-antisymmetric (A[n-1-i][n-1-j] = -A[i][j], because the
// GLL nodes are symmetric) and Sv is centro-symmetric (a product of two such
// matrices), so a contraction of a line of n values costs n^2/2
// multiply-adds plus n adds, with the n pre-adds shared by every matrix
// applied to the same line (even-odd split).
//
// Thread layout: one thread per grid line of an element.  One pass per
// direction: each thread loads its line from a padded shared-memory tile,
// applies every 1D matrix the operator needs along that direction, forms the
// pointwise terms at the line's nodes and adds its part of the result.  d = 3
// uses n^2 threads per element, d = 2 uses n, d = 1 one thread per element.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "df64.cuh"

namespace semk {

// Which operator an element kernel evaluates.
enum OpKind { OP_RHS = 0, OP_JAC = 1, OP_JACT = 2 };

// ---------------------------------------------------------------- even-odd matrices
// An n x n matrix A with A[n-1-i][n-1-j] = sigma A[i][j] (sigma = -1: centro-
// antisymmetric, +1: centro-symmetric) is stored, with H = n/2, as
//   e[i][j] = (A[i][j] + A[i][n-1-j]) / 2   (j < H),  e[i][H] = A[i][H]  (odd n)
//   o[i][j] = (A[i][j] - A[i][n-1-j]) / 2   (j < H)
//   m[j]    =  A[H][j]                      (odd n: middle row, j <= H)
// Then with the pre-adds xe_j = x_j + x_{n-1-j} (xe_H = x_H), xo_j = x_j - x_{n-1-j}
// and a = e xe, b = o xo:   y_i = a_i + b_i  and
//   antisymmetric: y_{n-1-i} = b_i - a_i,  y_H = sum_{j<H} m_j xo_j  (odd n)
//   symmetric:     y_{n-1-i} = a_i - b_i,  y_H = sum_{j<H} m_j xe_j + m_H x_H.
template <typename T, int NP>
struct EOMat {
    static constexpr int H = NP / 2;
    static constexpr int HE = NP / 2 + (NP & 1);
    T e[H][HE];
    T o[H][H];
    T m[H + 1];
};

template <typename T, int NP>
struct OpMats {
    EOMat<T, NP> Dg;   // (2/h) Dhat                                antisymmetric: gradient
    EOMat<T, NP> Sv;   // -nu (2/h)^2 W^-1 Dhat^T W Dhat             symmetric: viscous term of F and J
    EOMat<T, NP> Gv;   // nu (2/h) W Dhat W^-1                       antisymmetric: viscous flux of J^T,
                       //   stored with its even and odd halves doubled (gvdd_apply)
    EOMat<T, NP> Dd;   // -(2/h) Dhat^T                              antisymmetric: divergence (J^T)
};

// Pre-added halves of one line.
template <typename T, int NP>
struct Pre {
    T xe[NP / 2 + (NP & 1)];
    T xo[NP / 2];
};

template <typename T, int NP>
__device__ __forceinline__ void pre_add(const T (&x)[NP], Pre<T, NP>& p) {
    constexpr int H = NP / 2;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        p.xe[j] = x[j] + x[NP - 1 - j];
        p.xo[j] = x[j] - x[NP - 1 - j];
    }
    if constexpr (NP & 1) p.xe[H] = x[H];
}

// y = A x for a centro-antisymmetric (SYM = false) or centro-symmetric (SYM = true) A.
// FP64: the odd-half chain starts from a, so it yields t = a + b with no multiply and
// no add, and the mirrored output is 2a - t (symmetric) or t - 2a (antisymmetric), one
// multiply-add: 9 instead of 10 operations per pair of outputs on the FP64 pipe (the
// bound of the FP64 kernels).  Exact up to rounding; the other compute types keep the
// two independent chains.
template <bool SYM, typename T, int NP>
__device__ __forceinline__ void eo_apply(const EOMat<T, NP>& A, const Pre<T, NP>& p, T (&y)[NP]) {
    constexpr int H = NP / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        T a = A.e[i][0] * p.xe[0];
#pragma unroll
        for (int j = 1; j < H + (NP & 1); ++j) a = fma(A.e[i][j], p.xe[j], a);
        if constexpr (std::is_same<T, double>::value) {
            T t = a;
#pragma unroll
            for (int j = 0; j < H; ++j) t = fma(A.o[i][j], p.xo[j], t);
            y[i] = t;
            y[NP - 1 - i] = SYM ? fma(2.0, a, -t) : fma(-2.0, a, t);
        } else {
            T b = A.o[i][0] * p.xo[0];
#pragma unroll
            for (int j = 1; j < H; ++j) b = fma(A.o[i][j], p.xo[j], b);
            y[i] = a + b;
            y[NP - 1 - i] = SYM ? a - b : b - a;
        }
    }
    if constexpr (NP & 1) {
        if constexpr (SYM) {
            T c = A.m[H] * p.xe[H];
#pragma unroll
            for (int j = 0; j < H; ++j) c = fma(A.m[j], p.xe[j], c);
            y[H] = c;
        } else {
            T c = A.m[0] * p.xo[0];
#pragma unroll
            for (int j = 1; j < H; ++j) c = fma(A.m[j], p.xo[j], c);
            y[H] = c;
        }
    }
}

// y = A x from the raw line.
template <bool SYM, typename T, int NP>
__device__ __forceinline__ void eo_apply(const EOMat<T, NP>& A, const T (&x)[NP], T (&y)[NP]) {
    Pre<T, NP> p;
    pre_add<T, NP>(x, p);
    eo_apply<SYM, T, NP>(A, p, y);
}

// r = Dd (Gv z + u z) along one line (the J^T flux and its divergence), with G2
// holding Gv's even and odd halves doubled (split_eo with scale 2; the middle row
// of odd n as is).  With a = G2.e ze and b = G2.o zo, Gv z has
// y_i = (a_i + b_i)/2 and y_{n-1-i} = (b_i - a_i)/2, so the pre-adds of
// q = Gv z + u z that Dd takes are
//   qe_i = b_i + u_i z_i + u_{n-1-i} z_{n-1-i},   qo_i = a_i + u_i z_i - u_{n-1-i} z_{n-1-i}
// and, for odd n, qe_H = y_H + u_H z_H.  Gv's reconstruction, the advective
// product and Dd's pre-adds fold into four multiply-adds per node pair, against
// two adds, two multiply-adds and two adds the other way round.
template <typename T, int NP>
__device__ __forceinline__ void gvdd_apply(const EOMat<T, NP>& G2, const EOMat<T, NP>& Dd, const T (&z)[NP],
                                           const T (&u)[NP], T (&r)[NP]) {
    constexpr int H = NP / 2;
    Pre<T, NP> pz, pq;
    pre_add<T, NP>(z, pz);
#pragma unroll
    for (int i = 0; i < H; ++i) {
        T a = G2.e[i][0] * pz.xe[0];
#pragma unroll
        for (int j = 1; j < H + (NP & 1); ++j) a = fma(G2.e[i][j], pz.xe[j], a);
        T b = G2.o[i][0] * pz.xo[0];
#pragma unroll
        for (int j = 1; j < H; ++j) b = fma(G2.o[i][j], pz.xo[j], b);
        pq.xe[i] = fma(u[NP - 1 - i], z[NP - 1 - i], fma(u[i], z[i], b));
        pq.xo[i] = fma(-u[NP - 1 - i], z[NP - 1 - i], fma(u[i], z[i], a));
    }
    if constexpr (NP & 1) {
        T c = G2.m[0] * pz.xo[0];
#pragma unroll
        for (int j = 1; j < H; ++j) c = fma(G2.m[j], pz.xo[j], c);
        pq.xe[H] = fma(u[H], z[H], c);
    }
    eo_apply<false, T, NP>(Dd, pq, r);
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

// ---------------------------------------------------------------- dependent launches
// Programmatic dependent launch (sm_90 and later): the element and assembly
// kernels are launched with the programmatic stream-serialization attribute, so
// a kernel's blocks may be scheduled while its predecessor in the stream is
// still finishing.  Every such kernel first waits until its predecessors have
// completed and their memory is visible (griddepcontrol.wait; immediate for a
// kernel launched the ordinary way), and signals once it no longer needs to keep
// its successor from starting (griddepcontrol.launch_dependents).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Process-wide switch of the attribute (on by default; sem_set_dependent_launch).
bool pdl_enabled();

// Launch kernel k with the programmatic stream-serialization attribute.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Element-local output type: the compute type, except double for double-float
// kernels (whose results go to the FP64 assembly).
template <typename T>
struct OutT {
    using type = T;
};
template <>
struct OutT<dfloat> {
    using type = double;
};

template <typename T>
__device__ __forceinline__ T to_out(T x) {
    return x;
}
// exact: h and l widen exactly and their sum has at most 48 significant bits
__device__ __forceinline__ double to_out(dfloat x) { return widen_bits(x.h) + widen_bits(x.l); }

// Matrix coefficient in the compute type (host).
template <typename T>
T to_coeff(double x) {
    return (T)x;
}
template <>
inline dfloat to_coeff<dfloat>(double x) {
    return dfloat_of(x);
}

// Launch-time arguments shared by the element kernels.
struct ElemArgs {
    const void* u;     // state at which the operator is evaluated (global, SoA)
    const void* w;     // second input: w for J, v for J^T (unused by F)
    void* lvec;        // output: element-local values, [elem][comp][n^d] (unpadded)
    int E, N, G;       // elements per direction, order, unique nodes per direction
    int nelem;         // E^d
    unsigned plane;    // unknowns per vector: offset of the lo plane of a float-pair input
    int in_f2;         // FP32 form: inputs are float-pair planes (1) or doubles (0)
};

// Global index of component c at unique node (gz, gy, gx) of a d-dimensional grid.
__device__ __forceinline__ size_t gidx3(int c, int gz, int gy, int gx, int G) {
    return (((size_t)c * G + gz) * G + gy) * G + gx;
}

__device__ __forceinline__ int wrap(int g, int G) { return g >= G ? g - G : g; }

}  // namespace semk
