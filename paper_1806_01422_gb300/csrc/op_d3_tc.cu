// Launchers of the tensor-core element kernels (d = 3, n = 16; op_tc.cuh).
#include <cstring>

#include "op_tc.cuh"
#include "sem_internal.h"

namespace semk {

namespace {

// Raise the dynamic shared-memory limit of kernel k once per device and size.
template <typename K>
cudaError_t smem_limit(K k, size_t bytes, unsigned long long& done) {
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done |= bit;
    return e;
}

}  // namespace

bool tc_supported(int dim, int np, int op, bool fp32) {
    (void)fp32;
    return dim == 3 && np == 16 && op == OP_RHS;
}

cudaError_t launch_elem_tc(bool fp32, int op, const double* mats, const ElemArgs& a, unsigned* err, cudaStream_t s) {
    if (op != OP_RHS) return cudaErrorNotSupported;
    FullMats16 FM;
    std::memcpy(FM.Dg, mats + 0 * 256, sizeof(FM.Dg));
    std::memcpy(FM.Sv, mats + 1 * 256, sizeof(FM.Sv));
    std::memcpy(FM.Gv, mats + 2 * 256, sizeof(FM.Gv));
    std::memcpy(FM.Dd, mats + 3 * 256, sizeof(FM.Dd));
    if (a.nelem <= 0) return cudaSuccess;
    static thread_local unsigned long long done_f = 0, done_d = 0;
    if (fp32) {
        const size_t smem = TcRhsSmem::total;
        cudaError_t e = smem_limit(rhs3_tc_kernel, smem, done_f);
        if (e != cudaSuccess) return e;
        return launch_pdl(rhs3_tc_kernel, dim3(a.nelem), dim3(256), smem, s, FM, a, err);
    }
    const size_t smem = 4 * (size_t)Tile<16>::S3 * sizeof(double);
    cudaError_t e = smem_limit(rhs3_dmma_kernel, smem, done_d);
    if (e != cudaSuccess) return e;
    return launch_pdl(rhs3_dmma_kernel, dim3(a.nelem), dim3(256), smem, s, FM, a);
}

}  // namespace semk
