// Element-kernel instantiations for d = 1 (point counts n = 2..16): FP64, FP32 and
// double-float arithmetic.
#include "op_launch.cuh"

namespace semk {

template <>
cudaError_t launch_elem<double, 1>(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(double, 1, 2)
        SEMK_DISPATCH_CASE(double, 1, 3)
        SEMK_DISPATCH_CASE(double, 1, 4)
        SEMK_DISPATCH_CASE(double, 1, 5)
        SEMK_DISPATCH_CASE(double, 1, 6)
        SEMK_DISPATCH_CASE(double, 1, 7)
        SEMK_DISPATCH_CASE(double, 1, 8)
        SEMK_DISPATCH_CASE(double, 1, 9)
        SEMK_DISPATCH_CASE(double, 1, 10)
        SEMK_DISPATCH_CASE(double, 1, 11)
        SEMK_DISPATCH_CASE(double, 1, 12)
        SEMK_DISPATCH_CASE(double, 1, 13)
        SEMK_DISPATCH_CASE(double, 1, 14)
        SEMK_DISPATCH_CASE(double, 1, 15)
        SEMK_DISPATCH_CASE(double, 1, 16)
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_elem<float, 1>(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(float, 1, 2)
        SEMK_DISPATCH_CASE(float, 1, 3)
        SEMK_DISPATCH_CASE(float, 1, 4)
        SEMK_DISPATCH_CASE(float, 1, 5)
        SEMK_DISPATCH_CASE(float, 1, 6)
        SEMK_DISPATCH_CASE(float, 1, 7)
        SEMK_DISPATCH_CASE(float, 1, 8)
        SEMK_DISPATCH_CASE(float, 1, 9)
        SEMK_DISPATCH_CASE(float, 1, 10)
        SEMK_DISPATCH_CASE(float, 1, 11)
        SEMK_DISPATCH_CASE(float, 1, 12)
        SEMK_DISPATCH_CASE(float, 1, 13)
        SEMK_DISPATCH_CASE(float, 1, 14)
        SEMK_DISPATCH_CASE(float, 1, 15)
        SEMK_DISPATCH_CASE(float, 1, 16)
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_elem<dfloat, 1>(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(dfloat, 1, 2)
        SEMK_DISPATCH_CASE(dfloat, 1, 3)
        SEMK_DISPATCH_CASE(dfloat, 1, 4)
        SEMK_DISPATCH_CASE(dfloat, 1, 5)
        SEMK_DISPATCH_CASE(dfloat, 1, 6)
        SEMK_DISPATCH_CASE(dfloat, 1, 7)
        SEMK_DISPATCH_CASE(dfloat, 1, 8)
        SEMK_DISPATCH_CASE(dfloat, 1, 9)
        SEMK_DISPATCH_CASE(dfloat, 1, 10)
        SEMK_DISPATCH_CASE(dfloat, 1, 11)
        SEMK_DISPATCH_CASE(dfloat, 1, 12)
        SEMK_DISPATCH_CASE(dfloat, 1, 13)
        SEMK_DISPATCH_CASE(dfloat, 1, 14)
        SEMK_DISPATCH_CASE(dfloat, 1, 15)
        SEMK_DISPATCH_CASE(dfloat, 1, 16)
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace semk
