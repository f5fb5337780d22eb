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

#include <atomic>
#include <type_traits>

#include "asm_epi.cuh"
#include "df64.cuh"
#include "sem_internal.h"

namespace semk {

// Per-axis sharing of a global node index g: owner element e0 = g / N at local
// index i0 = g % N, left neighbour e1; sh when the node is also e1's node N.
// The division is a multiply-shift checked on the host (32-bit division and
// modulo issue conversion instructions on the FP64 pipe).
struct AxisSplit {
    int e0, i0, e1;
    bool sh;
};

__device__ __forceinline__ AxisSplit axis_split(int g, const AsmArgs& a) {
    AxisSplit s;
    s.e0 = (int)(((unsigned)g * a.divN_mul) >> a.divN_shift);
    s.i0 = g - s.e0 * a.N;
    s.e1 = s.e0 == 0 ? a.E - 1 : s.e0 - 1;
    s.sh = s.i0 == 0;
    return s;
}

// Sum of the element-local values of component c at one global node, in the
// fixed order: x pairs first, then y, then z.
template <typename Acc, typename T, int D>
__device__ __forceinline__ Acc gather_node(const T* __restrict__ lvec, const AsmArgs& a, int c, unsigned npd,
                                           const AxisSplit& x, const AxisSplit& y, const AxisSplit& z) {
    auto L = [&](int ex, int ix, int ey, int iy, int ez, int iz) -> Acc {
        const unsigned el = ((unsigned)ez * a.E + ey) * a.E + ex;
        const unsigned node = ((unsigned)iz * a.NP + iy) * a.NP + ix;
        return lvec[((size_t)el * D + c) * npd + node];
    };
    Acc sum = L(x.e0, x.i0, y.e0, y.i0, z.e0, z.i0);
    if (x.sh) sum += L(x.e1, a.N, y.e0, y.i0, z.e0, z.i0);
    if (D >= 2 && y.sh) {
        Acc t = L(x.e0, x.i0, y.e1, a.N, z.e0, z.i0);
        if (x.sh) t += L(x.e1, a.N, y.e1, a.N, z.e0, z.i0);
        sum += t;
    }
    if (D >= 3 && z.sh) {
        Acc t = L(x.e0, x.i0, y.e0, y.i0, z.e1, a.N);
        if (x.sh) t += L(x.e1, a.N, y.e0, y.i0, z.e1, a.N);
        if (y.sh) {
            Acc t2 = L(x.e0, x.i0, y.e1, a.N, z.e1, a.N);
            if (x.sh) t2 += L(x.e1, a.N, y.e1, a.N, z.e1, a.N);
            t += t2;
        }
        sum += t;
    }
    return sum;
}

// Node rows (along y) per thread: in 3D each thread gathers and combines
// asm_rows(3) nodes with independent loads, which halves the number of blocks
// (each with a partly idle last warp when G is not a multiple of 32).
// Measured on GB300 this shortens the 3D assembly by about a sixth; four rows
// gained nothing, and in 2D one row per thread measured faster.
constexpr int ASM_ROWS_3D = 2;
__host__ __device__ constexpr int asm_rows(int D) { return D == 3 ? ASM_ROWS_3D : 1; }

// The launch grid is (ceil(G / 128), G, d) for d = 2 and
// (ceil(G / 128), ceil(G / R), d G) for d = 3 with R = asm_rows(3), so a
// thread finds its nodes without integer division.  The y and z coordinates are
// uniform over a block, so only the x sharing differs between the lanes of a
// warp: each thread issues the FP64 adds its nodes need and no predicated-off
// ones.  The numbers of epilogue outputs and sources are template parameters
// for the same reason.  A row past the end (G not a multiple of R) repeats the
// block's first row and stores nothing.
template <typename T, int D, int NOUT, int NSRC>
__global__ void __launch_bounds__(128) assemble_kernel(const T* __restrict__ lvec, const AsmArgs a,
                                                       const Epi ep) {
    pdl_wait();
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    if (gx >= a.G) return;
    constexpr int R = asm_rows(D);
    int gy0 = 0, gz = 0, c = 0;
    if (D == 2) {
        gy0 = blockIdx.y * R;
        c = blockIdx.z;
    } else if (D == 3) {
        gy0 = blockIdx.y * R;
        c = blockIdx.z / a.G;          // once per block: blockIdx.z < 3G
        gz = blockIdx.z - c * a.G;
    }
    const unsigned npd = D == 1 ? a.NP : (D == 2 ? a.NP * a.NP : a.NP * a.NP * a.NP);
    const AxisSplit none{0, 0, 0, false};
    const AxisSplit sx = axis_split(gx, a);
    const AxisSplit sz = D >= 3 ? axis_split(gz, a) : none;
    double sum[R];
    unsigned idx[R];
    int nsh[R];
    bool live[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        live[r] = r == 0 || gy0 + r < a.G;   // uniform over the block
        const int gy = live[r] ? gy0 + r : gy0;
        const AxisSplit sy = D >= 2 ? axis_split(gy, a) : none;
        sum[r] = gather_node<double, T, D>(lvec, a, c, npd, sx, sy, sz);
        nsh[r] = (int)sx.sh + (int)sy.sh + (int)sz.sh;
        idx[r] = c * a.GD + ((unsigned)gz * a.G + gy) * a.G + gx;
    }
    // read every source before writing any output: an output may be a source (in place)
    double sv[R][NSRC > 0 ? NSRC : 1];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int m = 0; m < NSRC; ++m) sv[r][m] = ep.src[m][idx[r]];
    double ov[R][NOUT];
    bool bad = false;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
        double ak[R], v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) ak[r] = pick4(ep.alpha_k[o], nsh[r]);
        epi_output<R, NSRC>(ep.key[o], v, ak, sum, ep.beta[o], sv, nsh);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            ov[r][o] = v[r];
            bad |= live[r] && nonfinite_bits(v[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (live[r])
#pragma unroll
            for (int o = 0; o < NOUT; ++o) ep.out[o][idx[r]] = ov[r][o];
    if (bad && ep.nonfinite) atomicOr(ep.nonfinite, 1u);
}

// FP32 form.  The element contributions are summed in FP32 (same order as
// above); the epilogue either widens the sum to a caller's double (plain apply,
// F2 = false, no sources) or runs in float-pair arithmetic on float-pair planes:
// out = alpha a + sum_m beta_m src_m with alpha, beta as float pairs.
struct EpiF2 {
    float* out[3];
    df alpha_k[3][4];
    const float* src[4];
    df beta[3][4];
    double* out_f64;
    unsigned plane;
    unsigned* nonfinite;
};

template <int D, int NOUT, int NSRC, bool F2>
__global__ void __launch_bounds__(128) assemble_f32_kernel(const float* __restrict__ lvec, const AsmArgs a,
                                                           const EpiF2 ep) {
    pdl_wait();
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    if (gx >= a.G) return;
    constexpr int R = asm_rows(D);
    int gy0 = 0, gz = 0, c = 0;
    if (D == 2) {
        gy0 = blockIdx.y * R;
        c = blockIdx.z;
    } else if (D == 3) {
        gy0 = blockIdx.y * R;
        c = blockIdx.z / a.G;
        gz = blockIdx.z - c * a.G;
    }
    const unsigned npd = D == 1 ? a.NP : (D == 2 ? a.NP * a.NP : a.NP * a.NP * a.NP);
    const AxisSplit none{0, 0, 0, false};
    const AxisSplit sx = axis_split(gx, a);
    const AxisSplit sz = D >= 3 ? axis_split(gz, a) : none;
    float sum[R];
    unsigned idx[R];
    int nsh[R];
    bool live[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        live[r] = r == 0 || gy0 + r < a.G;
        const int gy = live[r] ? gy0 + r : gy0;
        const AxisSplit sy = D >= 2 ? axis_split(gy, a) : none;
        sum[r] = gather_node<float, float, D>(lvec, a, c, npd, sx, sy, sz);
        nsh[r] = (int)sx.sh + (int)sy.sh + (int)sz.sh;
        idx[r] = c * a.GD + ((unsigned)gz * a.G + gy) * a.G + gx;
    }
    if constexpr (!F2) {
        // plain apply: alpha = 1, no sources; 1/k (F and J only) is an exact power of two
        bool bad = false;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int k = nsh[r];
            const float v = a.scale_mult ? sum[r] * (k == 0 ? 1.f : (k == 1 ? 0.5f : (k == 2 ? 0.25f : 0.125f)))
                                         : sum[r];
            if (live[r]) {
                ep.out_f64[idx[r]] = widen_bits(v);
                bad |= nonfinite_f(v);
            }
        }
        if (bad && ep.nonfinite) atomicOr(ep.nonfinite, 1u);
    } else {
        df sv[R][NSRC > 0 ? NSRC : 1];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int m = 0; m < NSRC; ++m) sv[r][m] = {ep.src[m][idx[r]], ep.src[m][ep.plane + idx[r]]};
        // every term, zero or not: skipping them by key (as the FP64 kernel does)
        // measured slower here, where the FP32 pipe has room to spare
        df ov[R][NOUT];
        bool bad = false;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int o = 0; o < NOUT; ++o) {
                df v = df_mul_f(pick4(ep.alpha_k[o], nsh[r]), sum[r]);
#pragma unroll
                for (int m = 0; m < NSRC; ++m) v = df_add(v, df_mul(ep.beta[o][m], sv[r][m]));
                ov[r][o] = v;
                bad |= live[r] && nonfinite_f(v.hi);
            }
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (live[r])
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    ep.out[o][idx[r]] = ov[r][o].hi;
                    ep.out[o][ep.plane + idx[r]] = ov[r][o].lo;
                }
        if (bad && ep.nonfinite) atomicOr(ep.nonfinite, 1u);
    }
}

// Row-wise FP32 assembly for d = 3 (used at n = 8).  The node kernel above
// spends most of its issue slots on per-node index arithmetic; here one warp owns
// a chunk of one grid row along x (component c, rows gy and gz, up to 32
// elements along x) and the index work is done once per row.
//  * Gather: lane l takes element ex = 32 chunk + l and loads its element-local
//    row (n floats, vector loads) from each (y, z) element pair that shares the
//    row (1, 2 or 4 of them); node N of the left neighbour's row comes from lane
//    l - 1 by a shuffle (lane 0 loads it).  Its N nodes are summed in the order
//    of gather_node, so the results are the node kernel's bits.
//  * Epilogue: the sums go through shared memory and the warp walks the row's
//    nodes in order, lane l taking nodes l, l + 32, .., so that the sources and
//    outputs are read and written with coalesced accesses.
constexpr int ROW_WARPS = 8;

template <int NP>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&v)[NP]) {
    static_assert(NP % 4 == 0, "vector loads of whole rows");
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p) + q);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}

template <int NP, int NOUT, int NSRC, bool F2>
__global__ void __launch_bounds__(32 * ROW_WARPS) assemble_rows_f32_kernel(const float* __restrict__ lvec,
                                                                           const AsmArgs a, const EpiF2 ep,
                                                                           int nchunk) {
    constexpr int N = NP - 1;
    constexpr unsigned NPD = NP * NP * NP;
    __shared__ float srow[ROW_WARPS][32 * N];
    pdl_wait();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned task = blockIdx.x * ROW_WARPS + warp;     // (c, gz, gy, chunk), chunk fastest
    if (task >= 3u * a.G * a.G * nchunk) return;            // whole warps only
    const int chunk = task % nchunk;
    unsigned rest = task / nchunk;
    const int gy = rest % a.G;
    rest /= a.G;
    const int gz = rest % a.G;
    const int c = rest / a.G;
    const AxisSplit sy = axis_split(gy, a), sz = axis_split(gz, a);
    const int ex = chunk * 32 + lane;
    const bool act = ex < a.E;
    const int exs = act ? ex : a.E - 1;                       // idle lanes re-read a valid row
    auto row = [&](int exx, int ey, int j, int ez, int k) -> const float* {
        const unsigned el = ((unsigned)ez * a.E + ey) * a.E + exx;
        return lvec + ((size_t)el * 3 + c) * NPD + (k * NP + j) * NP;
    };
    const int exl = chunk * 32 == 0 ? a.E - 1 : chunk * 32 - 1;   // left neighbour of lane 0
    float v00[NP], v10[NP], v01[NP], v11[NP];
    float l00, l10 = 0.f, l01 = 0.f, l11 = 0.f;
    load_row<NP>(row(exs, sy.e0, sy.i0, sz.e0, sz.i0), v00);
    float t0 = lane == 0 ? row(exl, sy.e0, sy.i0, sz.e0, sz.i0)[N] : 0.f;
    l00 = __shfl_up_sync(0xffffffffu, v00[N], 1);
    if (lane == 0) l00 = t0;
    if (sy.sh) {
        load_row<NP>(row(exs, sy.e1, N, sz.e0, sz.i0), v10);
        t0 = lane == 0 ? row(exl, sy.e1, N, sz.e0, sz.i0)[N] : 0.f;
        l10 = __shfl_up_sync(0xffffffffu, v10[N], 1);
        if (lane == 0) l10 = t0;
    }
    if (sz.sh) {
        load_row<NP>(row(exs, sy.e0, sy.i0, sz.e1, N), v01);
        t0 = lane == 0 ? row(exl, sy.e0, sy.i0, sz.e1, N)[N] : 0.f;
        l01 = __shfl_up_sync(0xffffffffu, v01[N], 1);
        if (lane == 0) l01 = t0;
        if (sy.sh) {
            load_row<NP>(row(exs, sy.e1, N, sz.e1, N), v11);
            t0 = lane == 0 ? row(exl, sy.e1, N, sz.e1, N)[N] : 0.f;
            l11 = __shfl_up_sync(0xffffffffu, v11[N], 1);
            if (lane == 0) l11 = t0;
        }
    }
    if (act) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            // gather_node's order: x pairs first, then the y pair, then the z pairs
            float sum = i == 0 ? v00[0] + l00 : v00[i];
            if (sy.sh) sum += i == 0 ? v10[0] + l10 : v10[i];
            if (sz.sh) {
                float t = i == 0 ? v01[0] + l01 : v01[i];
                if (sy.sh) t += i == 0 ? v11[0] + l11 : v11[i];
                sum += t;
            }
            srow[warp][lane * N + i] = sum;
        }
    }
    __syncwarp();
    const int nodes = min(32, a.E - chunk * 32) * N;
    const unsigned base = c * a.GD + ((unsigned)gz * a.G + gy) * a.G + chunk * 32 * N;
    const int nsh_yz = (int)sy.sh + (int)sz.sh;
    bool bad = false;
    if constexpr (!F2) {
        for (int q = lane; q < nodes; q += 32) {
            const float sum = srow[warp][q];
            const int nsh = nsh_yz + (int)(q % N == 0);
            const float v = a.scale_mult ? sum * (nsh == 0 ? 1.f : (nsh == 1 ? 0.5f : (nsh == 2 ? 0.25f : 0.125f)))
                                         : sum;
            ep.out_f64[base + q] = widen_bits(v);
            bad |= nonfinite_f(v);
        }
    } else {
        // batches of B nodes per lane: every source of the batch is read before any output is
        // written (an output may be a source, in place), so the loads of a batch overlap
        constexpr int B = NSRC >= 3 ? 2 : 4;
        for (int q0 = lane; q0 < nodes; q0 += 32 * B) {
            df sv[B][NSRC > 0 ? NSRC : 1];
            float sum[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int q = q0 + 32 * b;
                const bool live = q < nodes;
                sum[b] = live ? srow[warp][q] : 0.f;
#pragma unroll
                for (int m = 0; m < NSRC; ++m)
                    sv[b][m] = live ? df{ep.src[m][base + q], ep.src[m][ep.plane + base + q]} : df{0.f, 0.f};
            }
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int q = q0 + 32 * b;
                if (q >= nodes) break;
                const int nsh = nsh_yz + (int)(q % N == 0);
                df ov[NOUT];
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    df v = df_mul_f(pick4(ep.alpha_k[o], nsh), sum[b]);
#pragma unroll
                    for (int m = 0; m < NSRC; ++m) v = df_add(v, df_mul(ep.beta[o][m], sv[b][m]));
                    ov[o] = v;
                    bad |= nonfinite_f(v.hi);
                }
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    ep.out[o][base + q] = ov[o].hi;
                    ep.out[o][ep.plane + base + q] = ov[o].lo;
                }
            }
        }
    }
    if (bad && ep.nonfinite) atomicOr(ep.nonfinite, 1u);
}

template <int NP, int NOUT, int NSRC, bool F2>
cudaError_t launch_rows_f32(const float* lvec, const AsmArgs& a, const EpiF2& e2, cudaStream_t s) {
    const int nchunk = (a.E + 31) / 32;
    const unsigned tasks = 3u * a.G * a.G * nchunk;
    const unsigned blocks = (tasks + ROW_WARPS - 1) / ROW_WARPS;
    return launch_pdl(assemble_rows_f32_kernel<NP, NOUT, NSRC, F2>, dim3(blocks), dim3(32 * ROW_WARPS), 0, s, lvec,
                      a, e2, nchunk);
}

// The row kernel serves n = 8 (the vector loads need n a multiple of 4).  At n = 16 the
// node-per-thread kernel measured faster (the N = 15 FP32 gradient at 16^3 hexes went from
// 0.435 to 0.442 evaluations/s with it): with 16 elements per grid row, half of each warp's
// lanes idle in the row gather.

template <int NP>
cudaError_t dispatch_rows_f32(const float* lvec, const AsmArgs& a, const EpiF2& e2, int nout, int nsrc, bool f2,
                              cudaStream_t s) {
    if (!f2) return launch_rows_f32<NP, 1, 0, false>(lvec, a, e2, s);
#define SEMK_ROWS_NS(NO)                                                        \
    switch (nsrc) {                                                             \
        case 0: return launch_rows_f32<NP, NO, 0, true>(lvec, a, e2, s);        \
        case 1: return launch_rows_f32<NP, NO, 1, true>(lvec, a, e2, s);        \
        case 2: return launch_rows_f32<NP, NO, 2, true>(lvec, a, e2, s);        \
        case 3: return launch_rows_f32<NP, NO, 3, true>(lvec, a, e2, s);        \
        default: return launch_rows_f32<NP, NO, 4, true>(lvec, a, e2, s);       \
    }
    switch (nout) {
        case 1: SEMK_ROWS_NS(1)
        case 2: SEMK_ROWS_NS(2)
        default: SEMK_ROWS_NS(3)
    }
#undef SEMK_ROWS_NS
}

static std::atomic<bool> g_pdl{true};
bool pdl_enabled() { return g_pdl.load(std::memory_order_relaxed); }
void set_pdl(bool on) { g_pdl.store(on, std::memory_order_relaxed); }

static df df_of(double x) {
    df r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
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
    epi_prepare(ep, a_in.scale_mult);
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
        grid.y = (a.G + asm_rows(2) - 1) / asm_rows(2);
        grid.z = 2;
    } else if (a.D == 3) {
        grid.y = (a.G + asm_rows(3) - 1) / asm_rows(3);
        grid.z = 3 * a.G;
    }
    if (ep.nout < 1 || ep.nout > 3 || ep.nsrc < 0 || ep.nsrc > 4) return cudaErrorInvalidValue;
    cudaError_t err = cudaSuccess;
#define SEMK_ASM_NS(T, D, NO)                                                                          \
    switch (ep.nsrc) {                                                                                 \
        case 0: err = launch_pdl(assemble_kernel<T, D, NO, 0>, grid, dim3(threads), 0, s, (const T*)lvec, a, ep); break; \
        case 1: err = launch_pdl(assemble_kernel<T, D, NO, 1>, grid, dim3(threads), 0, s, (const T*)lvec, a, ep); break; \
        case 2: err = launch_pdl(assemble_kernel<T, D, NO, 2>, grid, dim3(threads), 0, s, (const T*)lvec, a, ep); break; \
        case 3: err = launch_pdl(assemble_kernel<T, D, NO, 3>, grid, dim3(threads), 0, s, (const T*)lvec, a, ep); break; \
        default: err = launch_pdl(assemble_kernel<T, D, NO, 4>, grid, dim3(threads), 0, s, (const T*)lvec, a, ep); break; \
    }
#define SEMK_ASM_NO(T, D)                           \
    switch (ep.nout) {                              \
        case 1: SEMK_ASM_NS(T, D, 1) break;         \
        case 2: SEMK_ASM_NS(T, D, 2) break;         \
        default: SEMK_ASM_NS(T, D, 3) break;        \
    }
    if (lvec_fp32) {
        if (!ep.f2) {
            // plain apply of the FP32 form: alpha = 1, one double output, no sources
            if (ep.nout != 1 || ep.nsrc != 0 || ep.alpha[0] != 1.0) return cudaErrorInvalidValue;
            EpiF2 e2{};
            e2.out_f64 = ep.out[0];
            e2.nonfinite = ep.nonfinite;
            if (a.D == 1) return launch_pdl(assemble_f32_kernel<1, 1, 0, false>, grid, dim3(threads), 0, s, (const float*)lvec, a, e2);
            if (a.D == 2) return launch_pdl(assemble_f32_kernel<2, 1, 0, false>, grid, dim3(threads), 0, s, (const float*)lvec, a, e2);
            if (a.NP == 8) return dispatch_rows_f32<8>((const float*)lvec, a, e2, 1, 0, false, s);
            return launch_pdl(assemble_f32_kernel<3, 1, 0, false>, grid, dim3(threads), 0, s, (const float*)lvec, a, e2);
        }
        EpiF2 e2{};
        for (int o = 0; o < 3; ++o) {
            e2.out[o] = (float*)ep.out[o];
            for (int k = 0; k < 4; ++k) e2.alpha_k[o][k] = df_of(ep.alpha_k[o][k]);
            for (int m = 0; m < 4; ++m) e2.beta[o][m] = df_of(ep.beta[o][m]);
        }
        for (int m = 0; m < 4; ++m) e2.src[m] = (const float*)ep.src[m];
        e2.plane = a.ndof;
        e2.nonfinite = ep.nonfinite;
#define SEMK_F2_NS(D, NO)                                                                                 \
    switch (ep.nsrc) {                                                                                    \
        case 0: err = launch_pdl(assemble_f32_kernel<D, NO, 0, true>, grid, dim3(threads), 0, s, (const float*)lvec, a, e2); break; \
        case 1: err = launch_pdl(assemble_f32_kernel<D, NO, 1, true>, grid, dim3(threads), 0, s, (const float*)lvec, a, e2); break; \
        case 2: err = launch_pdl(assemble_f32_kernel<D, NO, 2, true>, grid, dim3(threads), 0, s, (const float*)lvec, a, e2); break; \
        case 3: err = launch_pdl(assemble_f32_kernel<D, NO, 3, true>, grid, dim3(threads), 0, s, (const float*)lvec, a, e2); break; \
        default: err = launch_pdl(assemble_f32_kernel<D, NO, 4, true>, grid, dim3(threads), 0, s, (const float*)lvec, a, e2); break; \
    }
#define SEMK_F2_NO(D)                         \
    switch (ep.nout) {                        \
        case 1: SEMK_F2_NS(D, 1) break;       \
        case 2: SEMK_F2_NS(D, 2) break;       \
        default: SEMK_F2_NS(D, 3) break;      \
    }
        if (a.D == 3 && a.NP == 8) return dispatch_rows_f32<8>((const float*)lvec, a, e2, ep.nout, ep.nsrc, true, s);
        if (a.D == 1) { SEMK_F2_NO(1) }
        else if (a.D == 2) { SEMK_F2_NO(2) }
        else { SEMK_F2_NO(3) }
#undef SEMK_F2_NO
#undef SEMK_F2_NS
        return err != cudaSuccess ? err : cudaGetLastError();
    } else {
        if (a.D == 1) { SEMK_ASM_NO(double, 1) }
        else if (a.D == 2) { SEMK_ASM_NO(double, 2) }
        else { SEMK_ASM_NO(double, 3) }
    }
#undef SEMK_ASM_NO
#undef SEMK_ASM_NS
    return err != cudaSuccess ? err : cudaGetLastError();
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

// ------------------------------------------------------------------ FP32 form
// HI_ONLY: write the hi plane alone (an input the element kernels read as hi only, Z = v / k)
template <bool HI_ONLY>
__global__ void f64_to_f2_kernel(const double* __restrict__ in, float* __restrict__ out, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        float hi, lo;
        split_bits(in[i], hi, lo);
        out[i] = hi;
        if (!HI_ONLY) out[n + i] = lo;
    }
}

__global__ void f2_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = widen_bits(in[i]) + widen_bits(in[n + i]);
}

__global__ void scale_f2_kernel(float* __restrict__ out, const float* __restrict__ in, df alpha, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const df v = df_mul(alpha, df{in[i], in[n + i]});
        out[i] = v.hi;
        out[n + i] = v.lo;
    }
}

// J partial sums and lam = M (u - uo) for a float-pair state (FP64 arithmetic, once per gradient)
__global__ void __launch_bounds__(OBJ_THREADS) objective_f2_kernel(const float* __restrict__ u,
                                                                   const double* __restrict__ uo,
                                                                   float* __restrict__ lam,
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
        const double diff = (widen_bits(u[idx]) + widen_bits(u[a.ndof + idx])) - uo[idx];
        const double l = m * diff;
        float hi, lo;
        split_bits(l, hi, lo);
        lam[idx] = hi;
        lam[a.ndof + idx] = lo;
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

static unsigned grid_for(size_t n) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 152u * 64u) blocks = 152u * 64u;
    return (unsigned)(blocks ? blocks : 1);
}

cudaError_t launch_f64_to_f2(const double* in, float* out, size_t n, cudaStream_t s, bool hi_only) {
    if (!n) return cudaSuccess;
    if (hi_only)
        f64_to_f2_kernel<true><<<grid_for(n), 256, 0, s>>>(in, out, n);
    else
        f64_to_f2_kernel<false><<<grid_for(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_f2_to_f64(const float* in, double* out, size_t n, cudaStream_t s) {
    if (!n) return cudaSuccess;
    f2_to_f64_kernel<<<grid_for(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_scale_f2(float* out, const float* in, double alpha, size_t n, cudaStream_t s) {
    if (!n) return cudaSuccess;
    scale_f2_kernel<<<grid_for(n), 256, 0, s>>>(out, in, df_of(alpha), n);
    return cudaGetLastError();
}

cudaError_t launch_objective_f2(const float* u, const double* uo, float* lam, double* partials, int nblocks,
                                const ObjArgs& a, cudaStream_t s) {
    objective_f2_kernel<<<nblocks, OBJ_THREADS, 0, s>>>(u, uo, lam, partials, a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Krylov helpers
constexpr int MD_THREADS = 256;

int multidot_blocks(size_t n) {
    size_t b = (n + MD_THREADS * 4 - 1) / (MD_THREADS * 4);
    if (b > 608) b = 608;
    return (int)(b ? b : 1);
}

// partials[j * gridDim.x + block] = sum over the block's strided range of V_j[i] w[i]
__global__ void __launch_bounds__(MD_THREADS) multidot_kernel(const VecList V, int k,
                                                              const double* __restrict__ w, size_t n,
                                                              double* __restrict__ partials) {
    __shared__ double ws[MD_THREADS / 32];
    for (int j = 0; j < k; ++j) {
        double acc = 0.0;
        const double* __restrict__ vj = V.v[j];
        for (size_t i = blockIdx.x * (size_t)MD_THREADS + threadIdx.x; i < n; i += (size_t)gridDim.x * MD_THREADS)
            acc = fma(vj[i], w[i], acc);
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < MD_THREADS / 32 ? ws[threadIdx.x] : 0.0;
            v = warp_sum(v);
            if (threadIdx.x == 0) partials[(size_t)j * gridDim.x + blockIdx.x] = v;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) multidot_final(const double* __restrict__ partials, int nb,
                                                      double* __restrict__ out) {
    __shared__ double ws[8];
    const int j = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partials[(size_t)j * nb + b];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < 8 ? ws[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) out[j] = v;
    }
}

cudaError_t launch_multidot(const VecList& V, int k, const double* w, size_t n, double* partials, double* out,
                            cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    const int nb = multidot_blocks(n);
    multidot_kernel<<<nb, MD_THREADS, 0, s>>>(V, k, w, n, partials);
    multidot_final<<<k, 256, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

// partials[block] = sum over the block's range of (e_i / (atol + rtol max(|u0_i|, |u1_i|)))^2
__global__ void __launch_bounds__(MD_THREADS) wrms_kernel(const double* __restrict__ e, const double* __restrict__ u0,
                                                          const double* __restrict__ u1, double atol, double rtol,
                                                          size_t n, double* __restrict__ partials) {
    __shared__ double ws[MD_THREADS / 32];
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)MD_THREADS + threadIdx.x; i < n; i += (size_t)gridDim.x * MD_THREADS) {
        const double r = e[i] / (atol + rtol * fmax(fabs(u0[i]), fabs(u1[i])));
        acc = fma(r, r, acc);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < MD_THREADS / 32 ? ws[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

cudaError_t launch_wrms_sum(const double* e, const double* u0, const double* u1, double atol, double rtol, size_t n,
                            double* partials, double* out, cudaStream_t s) {
    const int nb = multidot_blocks(n);
    wrms_kernel<<<nb, MD_THREADS, 0, s>>>(e, u0, u1, atol, rtol, n, partials);
    multidot_final<<<1, 256, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

// w += sum_j (+-coef[j]) V_j; the sign is an operand modifier of the FMA (no extra FP64 multiply)
template <bool NEG>
__global__ void multiaxpy_kernel(double* __restrict__ w, const VecList V, int k, const double* __restrict__ coef,
                                 size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        double acc = w[i];
        for (int j = 0; j < k; ++j) acc = fma(NEG ? -coef[j] : coef[j], V.v[j][i], acc);
        w[i] = acc;
    }
}

cudaError_t launch_multiaxpy(double* w, const VecList& V, int k, const double* coef, double scale, size_t n,
                             cudaStream_t s) {
    if (k <= 0 || n == 0) return cudaSuccess;
    if (scale < 0) multiaxpy_kernel<true><<<grid_for(n), 256, 0, s>>>(w, V, k, coef, n);
    else multiaxpy_kernel<false><<<grid_for(n), 256, 0, s>>>(w, V, k, coef, n);
    return cudaGetLastError();
}

}  // namespace semk
