// Instantiations of the matvec pass P3 (z-forward, spectrum product,
// z-inverse) for the 3 * 2^a lengths, complex FP64.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st) {
    return launch_p3<T, N>(mv, st);
}

template int p3_len<double, 24>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 48>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 96>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 192>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 384>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 768>(const MatvecView<double>&, cudaStream_t);

}  // namespace dda
