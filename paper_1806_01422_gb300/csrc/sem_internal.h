// Internal interfaces between the C-ABI host code and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "op_kernels.cuh"

struct sem_ctx;

namespace semk {

// Element kernel launch for dimension D, compute type T, runtime point count
// np = N+1.  `mats` holds the four full np x np matrices Dg, Sv, Gv, Dd
// (row-major, in that order); the launcher splits them into even/odd halves.
template <typename T, int D>
cudaError_t launch_elem(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s);

// Tensor-core element kernels (d = 3, n = 16): tcgen05 with split TF32 operands for the
// FP32-bulk form (fp32), DMMA for FP64.  F only; err (may be null) is set to 1 if the
// kernel gave up waiting for its MMAs (its outputs are then NaN).
bool tc_supported(int dim, int np, int op, bool fp32);
cudaError_t launch_elem_tc(bool fp32, int op, const double* mats, const ElemArgs& a, unsigned* err, cudaStream_t s);

// Largest supported point count per (D, T): limited by the shared-memory tiles.
int max_np(int D, bool fp32);
void set_pdl(bool on);   // programmatic dependent launch of element and assembly kernels

// --------------------------------------------------------------- assembly
// Epilogue of the gather-scatter sum: for each unique scalar node with
// assembled value a,  out[o] = alpha[o] a + sum_m beta[o][m] src[m]  (o < nout).
// The host fills alpha; the launcher folds the 1/k multiplicity of F and J
// into alpha_k[o][nsh] = alpha[o] / 2^nsh so the kernel spends one multiply,
// and sets key[o]: bit m when beta[o][m] != 0, bit 4 when alpha_k[o][*] == 1.
// The FP64 assembly skips the zero terms and the unit multiply (both exact);
// the float-pair assembly of the FP32-bulk form computes every term.
struct Epi {
    double* out[3];
    double alpha[3];
    const double* src[4];
    double beta[3][4];
    int nout, nsrc;
    unsigned* nonfinite;  // set to 1 if any output is NaN/Inf (may be null)
    int f2;               // FP32 form: out/src are float-pair planes (lo plane at +ndof floats)
    double alpha_k[3][4]; // filled by launch_assemble
    unsigned key[3];      // filled by launch_assemble
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
    bool fp32;            // SEM_PREC_FP32_BULK: FP32 element kernels and float element-local values
    bool dfloat;          // SEM_PREC_FP64_DF: double-float element kernels, double element-local values
    bool batch;           // a handle of sem_batch_create (packed instances; no single-grid tables)
    const double* mats;   // 4 x np x np element matrices (null for batch handles)
};
int handle_view(struct ::sem_ctx* h, HandleView* v);
void set_error(const char* msg);

// --------------------------------------------------------------- batches
// Many independent 2D instances of uneven E and N packed into one vector:
// instance k owns unknowns [off, off + 2 G^2) in the single-instance layout.
struct BatchInst {
    int E, N, NP, G, nelem;
    unsigned off;             // first unknown of the instance in the packed vector
    unsigned GD;              // G^2
    unsigned long long loff;  // first value of the instance in the element-local buffer
    unsigned mats_off;        // byte offset of its OpMats<double, NP> in the matrix table
    unsigned divN_mul;        // g / N == (g * divN_mul) >> divN_shift on 0 <= g < G
    int divN_shift;
    double mw[16];            // assembled 1D GLL weights by position (misfit mass)
    double scale;             // (h/2)^2
};
struct WorkItem { int inst, e0, ne, np; };  // ne elements of one instance from element e0
struct RowInfo { int inst, c, gy; };        // one grid row of one component

struct BatchDev {
    const BatchInst* inst;
    const WorkItem* items;
    int nitems;
    const RowInfo* rows;
    int nrows;
    const unsigned char* mats;
};

// the batched element kernel: one persistent launch over all work items
cudaError_t launch_batch_elem(const BatchDev& b, int op, const double* u, const double* w, double* lvec,
                              int threads, int blocks, size_t smem, cudaStream_t s);
size_t batch_elem_smem(int threads, int op);   // shared memory for the largest supported order
bool batch_np_supported(int np);
cudaError_t launch_batch_assemble(const BatchDev& b, const double* lvec, int scale_mult, const Epi& ep,
                                  cudaStream_t s);
// per-instance misfit: J[k] = 1/2 (u - uo)^T M (u - uo) over instance k, total in *Jtot
cudaError_t launch_batch_objective(const BatchDev& b, const double* u, const double* uo, double* lam,
                                   double* row_partials, const int* row_start, int count, double* J,
                                   double* Jtot, cudaStream_t s);
template <int NP>
void fill_opmats(void* dst, const double* mats);   // even/odd split of the 4 element matrices (host)

// FP32-form conversions at the API boundary (integer instructions for the split).
// hi_only writes the hi plane alone, for an input the element kernels read as hi only
// (Z = v / k of J^T).
cudaError_t launch_f64_to_f2(const double* in, float* out, size_t n, cudaStream_t s, bool hi_only = false);
cudaError_t launch_f2_to_f64(const float* in, double* out, size_t n, cudaStream_t s);
// misfit with a float-pair state u and float-pair output lam (FP64 arithmetic)
cudaError_t launch_objective_f2(const float* u, const double* uo, float* lam, double* partials, int nblocks,
                                const ObjArgs& a, cudaStream_t s);
// out <- alpha * in for float-pair vectors (pair arithmetic)
cudaError_t launch_scale_f2(float* out, const float* in, double alpha, size_t n, cudaStream_t s);

// Krylov helpers (FP64): out[j] = <V_j, w> for j < k in one pass, fixed summation
// order (per-block partials, then one block per j); w <- w + sum_j coef[j] V_j with
// coef on the device (scale = +1 or -1, the sign of the update).  k <= KMAX.
constexpr int KMAX = 40;
struct VecList { const double* v[KMAX]; };
int multidot_blocks(size_t n);
cudaError_t launch_multidot(const VecList& V, int k, const double* w, size_t n, double* partials, double* out,
                            cudaStream_t s);
// out[0] = sum_i (e_i / (atol + rtol max(|u0_i|, |u1_i|)))^2 (fixed-order block reduction;
// partials: multidot_blocks(n) doubles)
cudaError_t launch_wrms_sum(const double* e, const double* u0, const double* u1, double atol, double rtol, size_t n,
                            double* partials, double* out, cudaStream_t s);
cudaError_t launch_multiaxpy(double* w, const VecList& V, int k, const double* coef, double scale, size_t n,
                             cudaStream_t s);

// out <- alpha * in  (n doubles)
cudaError_t launch_scale(double* out, const double* in, double alpha, size_t n, cudaStream_t s);

}  // namespace semk
