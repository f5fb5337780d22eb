// Element-kernel instantiations for d = 3 in FP64 (point counts n = 2..16; n >= 13 runs
// the lean kernels of op_elem_lean.cuh, whose tiles fit the shared memory).
#include "op_launch.cuh"

namespace semk {

template <>
cudaError_t launch_elem<double, 3>(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(double, 3, 2)
        SEMK_DISPATCH_CASE(double, 3, 3)
        SEMK_DISPATCH_CASE(double, 3, 4)
        SEMK_DISPATCH_CASE(double, 3, 5)
        SEMK_DISPATCH_CASE(double, 3, 6)
        SEMK_DISPATCH_CASE(double, 3, 7)
        SEMK_DISPATCH_CASE(double, 3, 8)
        SEMK_DISPATCH_CASE(double, 3, 9)
        SEMK_DISPATCH_CASE(double, 3, 10)
        SEMK_DISPATCH_CASE(double, 3, 11)
        SEMK_DISPATCH_CASE(double, 3, 12)
        SEMK_DISPATCH_CASE(double, 3, 13)
        SEMK_DISPATCH_CASE(double, 3, 14)
        SEMK_DISPATCH_CASE(double, 3, 15)
        SEMK_DISPATCH_CASE(double, 3, 16)
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace semk
