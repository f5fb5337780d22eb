// Element-kernel instantiations for d = 2 in double-float arithmetic (n = 2..16).
#include "op_launch.cuh"

namespace semk {

template <>
cudaError_t launch_elem<dfloat, 2>(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(dfloat, 2, 2)
        SEMK_DISPATCH_CASE(dfloat, 2, 3)
        SEMK_DISPATCH_CASE(dfloat, 2, 4)
        SEMK_DISPATCH_CASE(dfloat, 2, 5)
        SEMK_DISPATCH_CASE(dfloat, 2, 6)
        SEMK_DISPATCH_CASE(dfloat, 2, 7)
        SEMK_DISPATCH_CASE(dfloat, 2, 8)
        SEMK_DISPATCH_CASE(dfloat, 2, 9)
        SEMK_DISPATCH_CASE(dfloat, 2, 10)
        SEMK_DISPATCH_CASE(dfloat, 2, 11)
        SEMK_DISPATCH_CASE(dfloat, 2, 12)
        SEMK_DISPATCH_CASE(dfloat, 2, 13)
        SEMK_DISPATCH_CASE(dfloat, 2, 14)
        SEMK_DISPATCH_CASE(dfloat, 2, 15)
        SEMK_DISPATCH_CASE(dfloat, 2, 16)
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace semk
