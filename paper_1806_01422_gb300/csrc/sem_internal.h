// Internal interfaces between the C-ABI host code and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "op_kernels.cuh"

struct sem_ctx;

namespace semk {

// Element kernel launch for dimension D, compute type T, runtime point count
// np = N+1.  `mats` holds the four full np x np matrices Dg, Dv, Vz, Dd
// (row-major, in that order); the launcher splits them into even/odd halves.
template <typename T, int D>
cudaError_t launch_elem(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s);

// Largest supported point count per (D, T): limited by the shared-memory tiles.
int max_np(int D, bool fp32);

// --------------------------------------------------------------- assembly
// Epilogue of the gather-scatter sum: for each unique scalar node with
// assembled value a,  out[o] = alpha[o] a + sum_m beta[o][m] src[m]  (o < nout).
// The host fills alpha; the launcher folds the 1/k multiplicity of F and J
// into alpha_k[o][nsh] = alpha[o] / 2^nsh so the kernel spends one multiply.
struct Epi {
    double* out[3];
    double alpha[3];
    const double* src[4];
    double beta[3][4];
    int nout, nsrc;
    unsigned* nonfinite;  // set to 1 if any output is NaN/Inf (may be null)
    double alpha_k[3][4]; // filled by launch_assemble
};

struct AsmArgs {
    int D, E, N, G, NP;
    unsigned GD;       // G^D
    unsigned ndof;     // D * G^D
    int scale_mult;    // 1: multiply the sum by 1/k (F and J); 0: plain sum (J^T)
    unsigned divN_mul; // g / N == (g * divN_mul) >> divN_shift for every 0 <= g < G (set by launch_assemble)
    int divN_shift;
};

cudaError_t launch_assemble(bool lvec_fp32, const void* lvec, const AsmArgs& a, const Epi& ep,
                            cudaStream_t s);

// --------------------------------------------------------------- objective
struct ObjArgs {
    int D, N, G;
    unsigned GD, ndof;
    double mw[16];     // 1D assembled GLL weights by position i = g % N (i = 0 counts both neighbours)
    double scale;      // (h/2)^D
};
// partials[nblocks] <- per-block sums of (u-uo) M (u-uo); lam <- M (u-uo) if lam != null
cudaError_t launch_objective(const double* u, const double* uo, double* lam, double* partials,
                             int nblocks, const ObjArgs& a, cudaStream_t s);
// out[0] <- factor * sum(partials[0..n)) in a fixed order
cudaError_t launch_sum_partials(const double* partials, int n, double* out, double factor,
                                cudaStream_t s);
int objective_blocks(unsigned ndof);

// Read-only view of a handle's grid and tables (for entry points outside sem_api.cu).
struct HandleView {
    int dim, E, N, G, np, nelem;
    size_t ndof, lvec_elems;
    bool fp32;
    const double* mats;   // 4 x np x np element matrices
};
int handle_view(struct ::sem_ctx* h, HandleView* v);
void set_error(const char* msg);

// out <- alpha * in  (n doubles)
cudaError_t launch_scale(double* out, const double* in, double alpha, size_t n, cudaStream_t s);

}  // namespace semk
