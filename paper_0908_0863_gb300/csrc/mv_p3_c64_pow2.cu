// Instantiations of the matvec pass P3 (z-forward, spectrum product,
// z-inverse) for the power-of-two lengths, complex FP32.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st) {
    return launch_p3<T, N>(mv, st);
}

template int p3_len<float, 2>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 4>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 8>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 16>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 32>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 64>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 128>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 256>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 512>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 1024>(const MatvecView<float>&, cudaStream_t);

}  // namespace dda
