// Gather-scatter assembly with the Runge-Kutta epilogue, the M-weighted misfit
// reduction, and small vector kernels.
//
// Assembly (Q^T, arXiv:1806.01422 Sec. 6.3 "local to global" accumulation):
// every unique periodic node g = (g_0, .., g_{d-1}) receives the element-local
// values of the 1, 2, 4 or 8 elements that share it.  Along each axis the owner
// element is e = g / N at local index i = g % N; when i == 0 the left
// neighbour (e - 1 mod E) also holds the node at local index N.  The
// contributions are summed in a fixed order (bit pattern of the "left" choice
// per axis), so the result is bitwise reproducible run to run.
#include <math.h>

#include "sem_internal.h"

namespace semk {

// FP64 work per unique node: (contributions - 1) adds, then per output one
// multiply and one fused multiply-add per source.  The FP64 pipe of GB300 issues
// two lanes per SM per clock, so everything else (the non-finite test on the
// exponent bits, the choice of contributions, the index arithmetic) stays on the
// integer pipes.
__device__ __forceinline__ bool nonfinite_bits(double v) {
    return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}

// The launch grid is (ceil(G / 128), G, d) for d = 2 and (ceil(G / 128), G, d G)
// for d = 3, so a thread finds its node without integer division (32-bit
// division and modulo issue conversion instructions on the FP64 pipe); the
// element index along an axis is a multiply-shift checked on the host.
template <typename T, int D>
__global__ void __launch_bounds__(128) assemble_kernel(const T* __restrict__ lvec, const AsmArgs a,
                                                       const Epi ep) {
    int g[3];
    int c;
    g[0] = blockIdx.x * blockDim.x + threadIdx.x;
    if (g[0] >= a.G) return;
    if (D == 1) {
        c = 0;
    } else if (D == 2) {
        g[1] = blockIdx.y;
        c = blockIdx.z;
    } else {
        g[1] = blockIdx.y;
        c = blockIdx.z / a.G;          // once per block: blockIdx.z < 3G
        g[2] = blockIdx.z - c * a.G;
    }
    unsigned idx = c * a.GD;
    {
        unsigned st = 1;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            idx += g[d] * st;
            st *= a.G;
        }
    }
    int npd = a.NP;
    if (D >= 2) npd *= a.NP;
    if (D >= 3) npd *= a.NP;
    int e0[3], e1[3], i0[3];
    int shmask = 0, nsh = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        e0[d] = (int)(((unsigned)g[d] * a.divN_mul) >> a.divN_shift);
        i0[d] = g[d] - e0[d] * a.N;
        e1[d] = e0[d] == 0 ? a.E - 1 : e0[d] - 1;
        if (i0[d] == 0) {
            shmask |= 1 << d;
            ++nsh;
        }
    }
    // contributions in a fixed order: combo = bit pattern of the "left neighbour" choices
    T sumT = (T)0;
    double sum = 0.0;
    bool first = true;
#pragma unroll
    for (int combo = 0; combo < (1 << D); ++combo) {
        if (combo & ~shmask) continue;
        unsigned el = 0, node = 0;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
            const bool bit = (combo >> d) & 1;
            el = el * a.E + (bit ? e1[d] : e0[d]);
            node = node * a.NP + (bit ? a.N : i0[d]);
        }
        const T v = lvec[((size_t)el * D + c) * (size_t)npd + node];
        if constexpr (sizeof(T) == 8) {
            sum = first ? (double)v : sum + (double)v;
        } else {
            sumT = first ? v : sumT + v;
        }
        first = false;
    }
    if constexpr (sizeof(T) != 8) sum = (double)sumT;
    // read every source before writing any output: an output may be a source (in place)
    double sv[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) sv[m] = m < ep.nsrc ? ep.src[m][idx] : 0.0;
    double ov[3];
    bool bad = false;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        if (o >= ep.nout) break;
        double v = ep.alpha_k[o][nsh] * sum;
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m < ep.nsrc) v = fma(ep.beta[o][m], sv[m], v);
        ov[o] = v;
        bad |= nonfinite_bits(v);
    }
#pragma unroll
    for (int o = 0; o < 3; ++o)
        if (o < ep.nout) ep.out[o][idx] = ov[o];
    if (bad && ep.nonfinite) atomicOr(ep.nonfinite, 1u);
}

// Multiply-shift for g / N on 0 <= g < G, verified exhaustively (G <= 65535).
static bool magic_div(int N, int G, unsigned& mul, int& shift) {
    for (shift = 16; shift <= 31; ++shift) {
        mul = (unsigned)(((1ull << shift) + N - 1) / N);
        bool ok = true;
        for (unsigned g = 0; g < (unsigned)G && ok; ++g)
            ok = (unsigned)(((unsigned long long)g * mul) >> shift) == g / (unsigned)N &&
                 (unsigned long long)g * mul < (1ull << 32);
        if (ok) return true;
    }
    return false;
}

cudaError_t launch_assemble(bool lvec_fp32, const void* lvec, const AsmArgs& a_in, const Epi& ep_in,
                            cudaStream_t s) {
    Epi ep = ep_in;
    for (int o = 0; o < 3; ++o)
        for (int k = 0; k < 4; ++k) ep.alpha_k[o][k] = a_in.scale_mult ? ep.alpha[o] / (double)(1 << k) : ep.alpha[o];
    AsmArgs a = a_in;
    if (a.G <= 0) return cudaSuccess;
    thread_local int cN = -1, cG = -1, cShift = 0;
    thread_local unsigned cMul = 0;
    if (a.N != cN || a.G != cG) {
        if (a.G > 65535 || !magic_div(a.N, a.G, cMul, cShift)) return cudaErrorInvalidValue;
        cN = a.N;
        cG = a.G;
    }
    a.divN_mul = cMul;
    a.divN_shift = cShift;
    const int threads = 128;
    dim3 grid((a.G + threads - 1) / threads, 1, 1);
    if (a.D == 2) {
        grid.y = a.G;
        grid.z = 2;
    } else if (a.D == 3) {
        grid.y = a.G;
        grid.z = 3 * a.G;
    }
#define SEMK_ASM(T, D) assemble_kernel<T, D><<<grid, threads, 0, s>>>((const T*)lvec, a, ep)
    if (lvec_fp32) {
        if (a.D == 1) SEMK_ASM(float, 1);
        else if (a.D == 2) SEMK_ASM(float, 2);
        else SEMK_ASM(float, 3);
    } else {
        if (a.D == 1) SEMK_ASM(double, 1);
        else if (a.D == 2) SEMK_ASM(double, 2);
        else SEMK_ASM(double, 3);
    }
#undef SEMK_ASM
    return cudaGetLastError();
}

// ------------------------------------------------------------------ objective
// J = 1/2 sum_c sum_g M_g (u - uo)^2 with M_g = (h/2)^d prod_axis mw[g_axis % N];
// lam = M (u - uo)  (eqs. ourcost and initadj).  Per-block partial sums use warp
// shuffles; the final sum runs in one block in a fixed order.
constexpr int OBJ_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

__global__ void __launch_bounds__(OBJ_THREADS) objective_kernel(const double* __restrict__ u,
                                                                const double* __restrict__ uo,
                                                                double* __restrict__ lam,
                                                                double* __restrict__ partials,
                                                                const ObjArgs a) {
    __shared__ double ws[OBJ_THREADS / 32];
    double acc = 0.0;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < a.ndof; idx += stride) {
        unsigned r = idx % a.GD;
        double m = a.scale;
        for (int d = 0; d < a.D; ++d) {
            const unsigned g = r % (unsigned)a.G;
            r /= (unsigned)a.G;
            m *= a.mw[g % (unsigned)a.N];
        }
        const double diff = u[idx] - uo[idx];
        const double l = m * diff;
        if (lam) lam[idx] = l;
        acc = fma(diff, l, acc);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < OBJ_THREADS / 32 ? ws[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(OBJ_THREADS) sum_partials_kernel(const double* __restrict__ p, int n,
                                                                   double* __restrict__ out,
                                                                   double factor) {
    __shared__ double ws[OBJ_THREADS / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += p[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < OBJ_THREADS / 32 ? ws[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) out[0] = factor * v;
    }
}

int objective_blocks(unsigned ndof) {
    unsigned b = (ndof + OBJ_THREADS - 1) / OBJ_THREADS;
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_objective(const double* u, const double* uo, double* lam, double* partials,
                             int nblocks, const ObjArgs& a, cudaStream_t s) {
    objective_kernel<<<nblocks, OBJ_THREADS, 0, s>>>(u, uo, lam, partials, a);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partials, int n, double* out, double factor,
                                cudaStream_t s) {
    sum_partials_kernel<<<1, OBJ_THREADS, 0, s>>>(partials, n, out, factor);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ vectors
__global__ void scale_kernel(double* __restrict__ out, const double* __restrict__ in, double alpha,
                             size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = alpha * in[i];
}

cudaError_t launch_scale(double* out, const double* in, double alpha, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 65535u * 16u) blocks = 65535u * 16u;
    scale_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, in, alpha, n);
    return cudaGetLastError();
}

}  // namespace semk
