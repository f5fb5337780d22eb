// Batched instances: many independent 2D viscous-Burgers problems of uneven
// element counts and orders advanced together (one launch per operator pass).
//
// Element work is a static list of items (instance, first element, count,
// order); a persistent grid of blocks walks the list with a stride of the
// grid size, and each item runs the same element body as a single-instance
// launch, so every instance's result is bitwise equal to its standalone
// computation.  The gather-scatter sum walks a table of (instance, component,
// row) rows, one block per row.  The RK drivers of sem_api.cu run unchanged on
// the packed vectors; only the operator applies and the misfit differ.
#include <type_traits>

#include "asm_epi.cuh"
#include "op_launch.cuh"
#include "sem_internal.h"

namespace semk {

bool batch_np_supported(int np) { return np == 4 || np == 6 || np == 8 || np == 10; }

template <int NP>
void fill_opmats(void* dst, const double* mats) {
    OpMats<double, NP> M;
    split_eo<double, NP>(M.Dg, mats + 0 * NP * NP);
    split_eo<double, NP>(M.Sv, mats + 1 * NP * NP);
    split_eo<double, NP>(M.Gv, mats + 2 * NP * NP, 2.0);
    split_eo<double, NP>(M.Dd, mats + 3 * NP * NP);
    memcpy(dst, &M, sizeof(M));
}
template void fill_opmats<4>(void*, const double*);
template void fill_opmats<6>(void*, const double*);
template void fill_opmats<8>(void*, const double*);
template void fill_opmats<10>(void*, const double*);

size_t batch_elem_smem(int threads, int op) {
    // element slots: threads / NP plus one spare slot for a partial group of threads
    size_t best = 0;
    for (int np : {4, 6, 8, 10}) {
        const size_t tile = (size_t)np * (np | 1);
        const size_t slots = threads / np + 1;
        const size_t b = slots * tiles_per_elem<2>(op) * tile * sizeof(double);
        if (b > best) best = b;
    }
    return best;
}

template <int NP>
__device__ __forceinline__ void batch_item2(int op, const BatchDev& b, const BatchInst& in, const WorkItem& w,
                                            const double* u, const double* wv, double* lvec,
                                            unsigned char* smem) {
    const OpMats<double, NP>& M = *reinterpret_cast<const OpMats<double, NP>*>(b.mats + in.mats_off);
    ElemArgs a;
    a.u = u + in.off;
    a.w = wv ? wv + in.off : nullptr;
    a.lvec = lvec + in.loff;
    a.E = in.E;
    a.N = in.N;
    a.G = in.G;
    a.nelem = in.nelem;
    a.plane = 0;
    a.in_f2 = 0;
    // threads past the last whole element form a spare slot (never valid)
    const int el = threadIdx.x / NP, t = threadIdx.x % NP;
    const bool valid = el < w.ne;
    const int e = w.e0 + el;
    if (op == OP_RHS) rhs2_body<double, NP>(M, a, e, t, el, valid, smem);
    else if (op == OP_JAC) jac2_body<double, NP>(M, a, e, t, el, valid, smem);
    else jact2_body<double, NP>(M, a, e, t, el, valid, smem);
}

__global__ void batch_elem2_kernel(const BatchDev b, int op, const double* __restrict__ u,
                                   const double* __restrict__ wv, double* __restrict__ lvec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int it = blockIdx.x; it < b.nitems; it += gridDim.x) {
        const WorkItem w = b.items[it];
        const BatchInst& in = b.inst[w.inst];
        switch (w.np) {
            case 4: batch_item2<4>(op, b, in, w, u, wv, lvec, smem_raw); break;
            case 6: batch_item2<6>(op, b, in, w, u, wv, lvec, smem_raw); break;
            case 8: batch_item2<8>(op, b, in, w, u, wv, lvec, smem_raw); break;
            default: batch_item2<10>(op, b, in, w, u, wv, lvec, smem_raw); break;
        }
        __syncthreads();
    }
}

cudaError_t launch_batch_elem(const BatchDev& b, int op, const double* u, const double* w, double* lvec,
                              int threads, int blocks, size_t smem, cudaStream_t s) {
    if (b.nitems <= 0) return cudaSuccess;
    if (smem > 48 * 1024) {
        static thread_local size_t done[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        if (done[dev & 63] < smem) {
            cudaError_t e = cudaFuncSetAttribute(batch_elem2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)227 * 1024);
            if (e != cudaSuccess) return e;
            done[dev & 63] = 227 * 1024;
        }
    }
    batch_elem2_kernel<<<blocks, threads, smem, s>>>(b, op, u, w, lvec);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ assembly
// One block per (instance, component, row); the block walks the row's nodes.
template <int NOUT, int NSRC>
__global__ void __launch_bounds__(128) batch_asm2_kernel(const double* __restrict__ lvec, const BatchDev b,
                                                         const Epi ep) {
    const RowInfo r = b.rows[blockIdx.x];
    const BatchInst& in = b.inst[r.inst];
    const int E = in.E, N = in.N, NP = in.NP, G = in.G;
    const unsigned npd = (unsigned)NP * NP;
    const double* lv = lvec + in.loff;
    const int gy = r.gy, c = r.c;
    const int ey0 = (int)(((unsigned)gy * in.divN_mul) >> in.divN_shift);
    const int iy0 = gy - ey0 * N;
    const int ey1 = ey0 == 0 ? E - 1 : ey0 - 1;
    const bool shy = iy0 == 0;
    for (int gx = threadIdx.x; gx < G; gx += blockDim.x) {
        const int ex0 = (int)(((unsigned)gx * in.divN_mul) >> in.divN_shift);
        const int ix0 = gx - ex0 * N;
        const int ex1 = ex0 == 0 ? E - 1 : ex0 - 1;
        const bool shx = ix0 == 0;
        auto L = [&](int ex, int ix, int ey, int iy) -> double {
            return lv[((size_t)((unsigned)ey * E + ex) * 2 + c) * npd + (unsigned)iy * NP + ix];
        };
        double sum = L(ex0, ix0, ey0, iy0);
        if (shx) sum += L(ex1, N, ey0, iy0);
        if (shy) {
            double t = L(ex0, ix0, ey1, N);
            if (shx) t += L(ex1, N, ey1, N);
            sum += t;
        }
        const int nsh = (int)shx + (int)shy;
        const unsigned idx = in.off + c * in.GD + (unsigned)gy * G + gx;
        double sv[1][NSRC > 0 ? NSRC : 1];
#pragma unroll
        for (int m = 0; m < NSRC; ++m) sv[0][m] = ep.src[m][idx];
        double ov[NOUT];
        bool bad = false;
        const double s1[1] = {sum};
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            const double ak[1] = {pick4(ep.alpha_k[o], nsh)};
            double v[1];
            const int n1[1] = {nsh};
            epi_output<1, NSRC>(ep.key[o], v, ak, s1, ep.beta[o], sv, n1);
            ov[o] = v[0];
            bad |= nonfinite_bits(v[0]);
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) ep.out[o][idx] = ov[o];
        if (bad && ep.nonfinite) atomicOr(ep.nonfinite, 1u);
    }
}

cudaError_t launch_batch_assemble(const BatchDev& b, const double* lvec, int scale_mult, const Epi& ep_in,
                                  cudaStream_t s) {
    Epi ep = ep_in;
    epi_prepare(ep, scale_mult);
    if (b.nrows <= 0) return cudaSuccess;
    if (ep.nout < 1 || ep.nout > 3 || ep.nsrc < 0 || ep.nsrc > 4) return cudaErrorInvalidValue;
#define SEMK_BA_NS(NO)                                                                             \
    switch (ep.nsrc) {                                                                             \
        case 0: batch_asm2_kernel<NO, 0><<<b.nrows, 128, 0, s>>>(lvec, b, ep); break;             \
        case 1: batch_asm2_kernel<NO, 1><<<b.nrows, 128, 0, s>>>(lvec, b, ep); break;             \
        case 2: batch_asm2_kernel<NO, 2><<<b.nrows, 128, 0, s>>>(lvec, b, ep); break;             \
        case 3: batch_asm2_kernel<NO, 3><<<b.nrows, 128, 0, s>>>(lvec, b, ep); break;             \
        default: batch_asm2_kernel<NO, 4><<<b.nrows, 128, 0, s>>>(lvec, b, ep); break;            \
    }
    switch (ep.nout) {
        case 1: SEMK_BA_NS(1) break;
        case 2: SEMK_BA_NS(2) break;
        default: SEMK_BA_NS(3) break;
    }
#undef SEMK_BA_NS
    return cudaGetLastError();
}

// ------------------------------------------------------------------ misfit
__device__ __forceinline__ double bwarp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

__global__ void __launch_bounds__(128) batch_objective_rows(const double* __restrict__ u,
                                                            const double* __restrict__ uo,
                                                            double* __restrict__ lam, double* __restrict__ part,
                                                            const BatchDev b) {
    __shared__ double ws[4];
    const RowInfo r = b.rows[blockIdx.x];
    const BatchInst& in = b.inst[r.inst];
    const int gy = r.gy;
    const int ey = (int)(((unsigned)gy * in.divN_mul) >> in.divN_shift);
    const double my = in.mw[gy - ey * in.N];
    double acc = 0.0;
    for (int gx = threadIdx.x; gx < in.G; gx += blockDim.x) {
        const int ex = (int)(((unsigned)gx * in.divN_mul) >> in.divN_shift);
        const unsigned idx = in.off + r.c * in.GD + (unsigned)gy * in.G + gx;
        const double diff = u[idx] - uo[idx];
        // mass product in the single-instance order: (h/2)^2 w_x w_y
        const double l = ((in.scale * in.mw[gx - ex * in.N]) * my) * diff;
        if (lam) lam[idx] = l;
        acc = fma(diff, l, acc);
    }
    acc = bwarp_sum(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) part[blockIdx.x] = (ws[0] + ws[1]) + (ws[2] + ws[3]);
}

// J[k] = 1/2 sum of instance k's row partials (rows of an instance are contiguous), fixed order
__global__ void batch_objective_sum(const double* __restrict__ part, const int* __restrict__ row_start, int count,
                                    double* __restrict__ J, double* __restrict__ Jtot) {
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        double acc = 0.0;
        for (int r = row_start[k]; r < row_start[k + 1]; ++r) acc += part[r];
        J[k] = 0.5 * acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < count; ++k) t += J[k];
        *Jtot = t;
    }
}

cudaError_t launch_batch_objective(const BatchDev& b, const double* u, const double* uo, double* lam,
                                   double* row_partials, const int* row_start, int count, double* J,
                                   double* Jtot, cudaStream_t s) {
    if (b.nrows <= 0) return cudaSuccess;
    batch_objective_rows<<<b.nrows, 128, 0, s>>>(u, uo, lam, row_partials, b);
    batch_objective_sum<<<1, 256, 0, s>>>(row_partials, row_start, count, J, Jtot);
    return cudaGetLastError();
}

}  // namespace semk
