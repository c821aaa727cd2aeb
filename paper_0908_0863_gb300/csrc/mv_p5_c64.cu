// Instantiations (complex FP32) of the matvec pass P5 (y-inverse + diagonal + compress) for every line
// length and tile width, and its dispatcher.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int LN>
static int p5_width(const MatvecView<T>& mv, const C<IO<T>>* p, C<IO<T>>* y, cudaStream_t st) {
    DDA_LOGW_SWITCH(mv.logW_y, (launch_p5<T, LN, LW>(mv, p, y, st)))
}

template <typename T> int pass5(const MatvecView<T>& mv, const C<IO<T>>* p, C<IO<T>>* y, cudaStream_t st) {
    DDA_LEN_SWITCH(mv.g.Ly, (p5_width<T, LN>(mv, p, y, st)))
}

template int pass5<float>(const MatvecView<float>&, const C<float>*, C<float>*, cudaStream_t);

}  // namespace dda
