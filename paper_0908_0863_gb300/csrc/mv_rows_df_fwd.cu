// Instantiations of the matvec pass P2 (x-forward) in complex double-float
// (df.cuh) for every line length and tile width, and its dispatcher (P4 is
// a translation unit of its own, so that the two compile in parallel).
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, bool INV> int pass_rows(const MatvecView<T>& mv, cudaStream_t st) {
    DDA_LEN_SWITCH(mv.g.Lx, (launch_rows<T, INV, LN>(mv, st)))
}

template int pass_rows<DF, false>(const MatvecView<DF>&, cudaStream_t);

}  // namespace dda
