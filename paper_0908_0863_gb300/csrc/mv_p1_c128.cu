// Instantiations (complex FP64) of the matvec pass P1 (expand + y-forward) for every line
// length and tile width, and its dispatcher.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int LN>
static int p1_width(const MatvecView<T>& mv, const C<IO<T>>* p, cudaStream_t st) {
    DDA_LOGW_SWITCH(mv.logW_y, (launch_p1<T, LN, LW>(mv, p, st)))
}

template <typename T> int pass1(const MatvecView<T>& mv, const C<IO<T>>* p, cudaStream_t st) {
    DDA_LEN_SWITCH(mv.g.Ly, (p1_width<T, LN>(mv, p, st)))
}

template int pass1<double>(const MatvecView<double>&, const C<double>*, cudaStream_t);

}  // namespace dda
