// Instantiations of the matvec pass P3 (z-forward, spectrum product,
// z-inverse) for the 5 * 2^a lengths, complex FP32.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st) {
    return launch_p3<T, N>(mv, st);
}

template int p3_len<float, 40>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 80>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 160>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 320>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 640>(const MatvecView<float>&, cudaStream_t);

}  // namespace dda
