// Instantiations of the matvec pass P3 (z-forward, spectrum product, z-inverse) in complex FP64 for every line
// length and tile width, and its dispatcher.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int LN>
static int p3_width(const MatvecView<T>& mv, cudaStream_t st) {
    DDA_LOGW_SWITCH(mv.logW_z, (launch_p3<T, LN, LW>(mv, st)))
}

template <typename T> int pass3(const MatvecView<T>& mv, cudaStream_t st) {
    DDA_LOGN_SWITCH(ilog2(mv.g.Lz), (p3_width<T, LN>(mv, st)))
}

template int pass3<double>(const MatvecView<double>&, cudaStream_t);

}  // namespace dda
