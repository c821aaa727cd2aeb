// Device view of one context's matvec state and the launcher of its passes.
#pragma once

#include "common.cuh"
#include "profile.cuh"

namespace dda {

__device__ __forceinline__ int ilog2_dev(int n) { return 31 - __clz(n); }

template <typename T>
struct MatvecView {
    Geometry g;
    TargetView tv;
    const C<T>* ainv;   // [nmat][3] alpha^-1
    const C<T>* spec;   // [Hz][Hy][Hx][6], scaled by 1/(Lx Ly Lz)
    const C<T>* tw;     // twiddle table, kMaxLine entries
    C<T>* Ay;           // [3][P][Ly][K]
    C<T>* Bxy;          // [3][P][Ly][Lx]
    int logW_y, logW_x, logW_z;  // tile widths (lines per CTA) of the passes
    const int* status;  // optional: when *status != 0 every pass returns at once
    int conj;           // 1: compute conj(A conj(p)) = A^H p (A complex symmetric)
    PassProfiler* prof; // host object; when non-null and on, each pass is timed
};

template <typename T> void configure_matvec(MatvecView<T>& mv);
template <typename T> int launch_matvec(const MatvecView<T>& mv, const C<T>* p, C<T>* y, cudaStream_t st);

}  // namespace dda
