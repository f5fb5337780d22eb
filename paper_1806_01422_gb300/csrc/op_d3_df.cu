// Element-kernel instantiations for d = 3 in double-float arithmetic, n = 2..9
// (n = 10..12 and 13..16 in op_d3_df_mid.cu and op_d3_df_hi.cu, compiled in parallel).
#include "op_launch.cuh"

namespace semk {

cudaError_t launch_elem_df3_mid(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s);

template <>
cudaError_t launch_elem<dfloat, 3>(int np, int op, const double* mats, const ElemArgs& a, cudaStream_t s) {
    switch (np) {
        SEMK_DISPATCH_CASE(dfloat, 3, 2)
        SEMK_DISPATCH_CASE(dfloat, 3, 3)
        SEMK_DISPATCH_CASE(dfloat, 3, 4)
        SEMK_DISPATCH_CASE(dfloat, 3, 5)
        SEMK_DISPATCH_CASE(dfloat, 3, 6)
        SEMK_DISPATCH_CASE(dfloat, 3, 7)
        SEMK_DISPATCH_CASE(dfloat, 3, 8)
        SEMK_DISPATCH_CASE(dfloat, 3, 9)
        default: return launch_elem_df3_mid(np, op, mats, a, s);
    }
}

}  // namespace semk
