// Element-kernel instantiations for d = 3 in double-float arithmetic, n = 10..12.
#include "op_launch.cuh"

namespace semk {

cudaError_t launch_elem_df3_hi(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s);

cudaError_t launch_elem_df3_mid(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(dfloat, 3, 10)
        SEMK_DISPATCH_CASE(dfloat, 3, 11)
        SEMK_DISPATCH_CASE(dfloat, 3, 12)
        default: return launch_elem_df3_hi(np, op, mats, a, s);
    }
}

}  // namespace semk
