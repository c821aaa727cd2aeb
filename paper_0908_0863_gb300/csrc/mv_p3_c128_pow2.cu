// Instantiations of the matvec pass P3 (z-forward, spectrum product,
// z-inverse) for the power-of-two lengths, complex FP64.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st) {
    return launch_p3<T, N>(mv, st);
}

template int p3_len<double, 2>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 4>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 8>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 16>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 32>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 64>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 128>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 256>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 512>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 1024>(const MatvecView<double>&, cudaStream_t);

}  // namespace dda
