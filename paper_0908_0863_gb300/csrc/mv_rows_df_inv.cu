// Instantiations of the matvec pass P4 (x-inverse) in complex double-float
// (df.cuh) for every line length and tile width, and its dispatcher.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, bool INV> int pass_rows(const MatvecView<T>& mv, cudaStream_t st) {
    DDA_LEN_SWITCH(mv.g.Lx, (launch_rows<T, INV, LN>(mv, st)))
}

template int pass_rows<DF, true>(const MatvecView<DF>&, cudaStream_t);

}  // namespace dda
