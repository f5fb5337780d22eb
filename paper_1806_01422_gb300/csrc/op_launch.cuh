// Launch configuration of the element kernels: split the host matrices into
// even/odd halves, size the block (elements per block x threads per element)
// and the dynamic shared memory, and dispatch on the runtime point count.
#pragma once
#include <algorithm>

#include "op_elem.cuh"
#include "op_elem_lean.cuh"
#include "sem_internal.h"

namespace semk {

// Even/odd halves of a centro-(anti)symmetric matrix (the storage is the same
// for both symmetries; the kernels apply the matching reconstruction), times
// scale (a power of two, so the scaling is exact); the middle row of odd n is
// never scaled.  J^T takes Gv with scale 2 (gvdd_apply).
template <typename T, int NP>
void split_eo(EOMat<T, NP>& M, const double* A, double scale = 1.0) {
    constexpr int H = NP / 2;
    for (int i = 0; i < H; ++i) {
        for (int j = 0; j < H; ++j) {
            M.e[i][j] = to_coeff<T>(0.5 * scale * (A[i * NP + j] + A[i * NP + (NP - 1 - j)]));
            M.o[i][j] = to_coeff<T>(0.5 * scale * (A[i * NP + j] - A[i * NP + (NP - 1 - j)]));
        }
        if (NP & 1) M.e[i][H] = to_coeff<T>(scale * A[i * NP + H]);
    }
    for (int j = 0; j <= H; ++j) M.m[j] = to_coeff<T>((NP & 1) ? A[H * NP + j] : 0.0);
}

constexpr int SMEM_TARGET = 100 * 1024;   // two blocks per SM fit in 227 KB
constexpr int NUM_SMS = 152;               // GB300: 2 dies x 76 SMs

// 2D double-float kernels run one thread per (line, component) (op2c_kernel)
template <typename T, int D>
__host__ __device__ constexpr bool comp_parallel() {
    return D == 2 && std::is_same<T, dfloat>::value;
}

template <typename T, int D, int NP>
size_t elem_smem_bytes(int op) {
    using Tl = Tile<NP>;
    const size_t tile = D == 3 ? Tl::S3 : (D == 2 ? Tl::S2 : 0);
    if (comp_parallel<T, D>()) return (size_t)(tiles_per_elem<D>(op) + 1) * tile * sizeof(T);
    if (D == 3 && lean3_op<T, NP>(op)) return (size_t)lean_tiles_per_elem<D>(op) * tile * sizeof(T);
    if constexpr (D == 3) return (size_t)tiles3<T, NP>(op) * tile * sizeof(T);
    return (size_t)tiles_per_elem<D>(op) * tile * sizeof(T);
}

template <typename T, int D, int NP>
cudaError_t launch_elem_np(int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    OpMats<T, NP> M;
    split_eo<T, NP>(M.Dg, mats + 0 * NP * NP);
    split_eo<T, NP>(M.Sv, mats + 1 * NP * NP);
    split_eo<T, NP>(M.Gv, mats + 2 * NP * NP, 2.0);
    split_eo<T, NP>(M.Dd, mats + 3 * NP * NP);
    if (a.nelem <= 0) return cudaSuccess;
    if constexpr (D == 1) {
        const int threads = 128;
        const int blocks = (a.nelem + threads - 1) / threads;
        return launch_pdl(op1_kernel<T, NP>, dim3(blocks), dim3(threads), 0, s, M, a, op);
    } else {
        constexpr int TPE = D == 3 ? NP * NP : (comp_parallel<T, D>() ? 2 * NP : NP);
        const bool lean = D == 3 && lean3_op<T, NP>(op);
        const size_t per = elem_smem_bytes<T, D, NP>(op);
        const int epb_max = lean ? 1 : std::max(1, std::min(256 / TPE, (int)(SMEM_TARGET / per)));
        // Balance the grid over the SMs: the fewest waves k of NUM_SMS blocks that
        // fit epb_max elements per block, then the smallest block that fills them.
        const int waves = (a.nelem + NUM_SMS * epb_max - 1) / (NUM_SMS * epb_max);
        int epb = (a.nelem + NUM_SMS * waves - 1) / (NUM_SMS * waves);
        epb = std::max(1, std::min(epb, epb_max));
        if constexpr (comp_parallel<T, D>()) {
            // warp-aligned halves: epb * n a multiple of 32 when that fits
            int g = 32, n = NP;
            while (n) { const int r = g % n; g = n; n = r; }
            const int step = 32 / g;
            const int up = (epb + step - 1) / step * step;
            if (up <= epb_max) epb = up;
        }
        const size_t smem = per * epb;
        if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
        const int threads = epb * TPE;
        const int blocks = (a.nelem + epb - 1) / epb;
        if constexpr (D == 3 && std::is_same<T, double>::value && NP == 8)
            if (threads > (op == OP_RHS ? 256 : 128)) return cudaErrorInvalidConfiguration;
        if constexpr (comp_parallel<T, D>()) {
            if (smem > 48 * 1024) {
                static thread_local unsigned long long done_c = 0;
                static thread_local size_t done_c_smem = 0;
                int dev = 0;
                cudaGetDevice(&dev);
                const unsigned long long bit = 1ull << (dev & 63);
                if (!(done_c & bit) || done_c_smem < smem) {
                    cudaError_t err = cudaFuncSetAttribute(op2c_kernel<T, NP>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (err != cudaSuccess) return err;
                    done_c |= bit;
                    done_c_smem = smem;
                }
            }
            return launch_pdl(op2c_kernel<T, NP>, dim3(blocks), dim3(threads), smem, s, M, a, op);
        }
        void (*k)(const OpMats<T, NP>, const ElemArgs);
        if constexpr (D == 3 && lean3<T, NP>())
            k = op == OP_RHS ? rhs3_lean_kernel<T, NP>
                             : (op == OP_JAC ? jac3_lean_kernel<T, NP> : jact3_lean_kernel<T, NP>);
        else if constexpr (D == 3 && lean3_any<T, NP>())
            k = lean ? jact3_lean_kernel<T, NP>   // lean3_op: J^T only
                     : (op == OP_RHS ? rhs3_kernel<T, NP> : jac3_kernel<T, NP>);
        else if constexpr (D == 3 && std::is_same<T, double>::value && NP == 8)
            k = op == OP_RHS ? rhs3_f64_kernel<NP> : (op == OP_JAC ? jac3_f64_kernel<NP> : jact3_f64_kernel<NP>);
        else if constexpr (D == 3)
            k = op == OP_RHS ? rhs3_kernel<T, NP> : (op == OP_JAC ? jac3_kernel<T, NP> : jact3_kernel<T, NP>);
        else
            k = op == OP_RHS ? rhs2_kernel<T, NP> : (op == OP_JAC ? jac2_kernel<T, NP> : jact2_kernel<T, NP>);
        if (smem > 48 * 1024) {
            // once per kernel, size and device (no API call in the launch path afterwards,
            // so launches can be recorded into a CUDA graph)
            static thread_local unsigned long long done[3][3] = {};
            static thread_local size_t done_smem[3][3] = {};
            int dev = 0;
            cudaGetDevice(&dev);
            const unsigned long long bit = 1ull << (dev & 63);
            if (!(done[op][0] & bit) || done_smem[op][0] < smem) {
                cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (err != cudaSuccess) return err;
                done[op][0] |= bit;
                done_smem[op][0] = smem;
            }
        }
        return launch_pdl(k, dim3(blocks), dim3(threads), smem, s, M, a);
    }
}

}  // namespace semk

// Explicit dispatch over the point counts LO..HI of one (T, D) pair.
#define SEMK_DISPATCH_CASE(T, D, NP) \
    case NP: return launch_elem_np<T, D, NP>(op, mats, a, s);
