// Instantiations of the matvec pass P3 (z-forward, spectrum product,
// z-inverse) for the 5 * 2^a lengths, complex FP64.
#include "matvec_kernels.cuh"

namespace dda {

template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st) {
    return launch_p3<T, N>(mv, st);
}

template int p3_len<double, 40>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 80>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 160>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 320>(const MatvecView<double>&, cudaStream_t);
template int p3_len<double, 640>(const MatvecView<double>&, cudaStream_t);

}  // namespace dda
