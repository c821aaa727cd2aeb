// Instantiations of the matvec pass P3 (z-forward, spectrum product,
// z-inverse) for the 5 * 2^a lengths, complex double-float (df.cuh).
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st) {
    return launch_p3<T, N>(mv, st);
}

template int p3_len<DF, 40>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 80>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 160>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 320>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 640>(const MatvecView<DF>&, cudaStream_t);

}  // namespace dda
