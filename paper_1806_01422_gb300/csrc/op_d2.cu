// Element-kernel instantiations for d = 2 (point counts n = 2..16): FP64 and FP32.
#include "op_launch.cuh"

namespace semk {

template <>
cudaError_t launch_elem<double, 2>(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(double, 2, 2)
        SEMK_DISPATCH_CASE(double, 2, 3)
        SEMK_DISPATCH_CASE(double, 2, 4)
        SEMK_DISPATCH_CASE(double, 2, 5)
        SEMK_DISPATCH_CASE(double, 2, 6)
        SEMK_DISPATCH_CASE(double, 2, 7)
        SEMK_DISPATCH_CASE(double, 2, 8)
        SEMK_DISPATCH_CASE(double, 2, 9)
        SEMK_DISPATCH_CASE(double, 2, 10)
        SEMK_DISPATCH_CASE(double, 2, 11)
        SEMK_DISPATCH_CASE(double, 2, 12)
        SEMK_DISPATCH_CASE(double, 2, 13)
        SEMK_DISPATCH_CASE(double, 2, 14)
        SEMK_DISPATCH_CASE(double, 2, 15)
        SEMK_DISPATCH_CASE(double, 2, 16)
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_elem<float, 2>(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(float, 2, 2)
        SEMK_DISPATCH_CASE(float, 2, 3)
        SEMK_DISPATCH_CASE(float, 2, 4)
        SEMK_DISPATCH_CASE(float, 2, 5)
        SEMK_DISPATCH_CASE(float, 2, 6)
        SEMK_DISPATCH_CASE(float, 2, 7)
        SEMK_DISPATCH_CASE(float, 2, 8)
        SEMK_DISPATCH_CASE(float, 2, 9)
        SEMK_DISPATCH_CASE(float, 2, 10)
        SEMK_DISPATCH_CASE(float, 2, 11)
        SEMK_DISPATCH_CASE(float, 2, 12)
        SEMK_DISPATCH_CASE(float, 2, 13)
        SEMK_DISPATCH_CASE(float, 2, 14)
        SEMK_DISPATCH_CASE(float, 2, 15)
        SEMK_DISPATCH_CASE(float, 2, 16)
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace semk
