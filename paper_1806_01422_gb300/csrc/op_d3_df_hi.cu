// Element-kernel instantiations for d = 3 in double-float arithmetic, n = 13..16
// (the lean kernels of op_elem_lean.cuh).
#include "op_launch.cuh"

namespace semk {

cudaError_t launch_elem_df3_hi(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(dfloat, 3, 13)
        SEMK_DISPATCH_CASE(dfloat, 3, 14)
        SEMK_DISPATCH_CASE(dfloat, 3, 15)
        SEMK_DISPATCH_CASE(dfloat, 3, 16)
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace semk
