// Instantiations of the matvec pass P3 (z-forward, spectrum product,
// z-inverse) for the power-of-two lengths, complex double-float (df.cuh).
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st) {
    return launch_p3<T, N>(mv, st);
}

template int p3_len<DF, 2>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 4>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 8>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 16>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 32>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 64>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 128>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 256>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 512>(const MatvecView<DF>&, cudaStream_t);
template int p3_len<DF, 1024>(const MatvecView<DF>&, cudaStream_t);

}  // namespace dda
