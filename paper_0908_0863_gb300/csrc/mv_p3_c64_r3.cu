// Instantiations of the matvec pass P3 (z-forward, spectrum product,
// z-inverse) for the 3 * 2^a lengths, complex FP32.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st) {
    return launch_p3<T, N>(mv, st);
}

template int p3_len<float, 24>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 48>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 96>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 192>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 384>(const MatvecView<float>&, cudaStream_t);
template int p3_len<float, 768>(const MatvecView<float>&, cudaStream_t);

}  // namespace dda
