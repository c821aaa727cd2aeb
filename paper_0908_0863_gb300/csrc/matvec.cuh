// Device view of one context's matvec state and the launcher of its passes.
#pragma once

#include "common.cuh"
#include "profile.cuh"

namespace dda {

template <typename T>
struct MatvecView {
    Geometry g;
    TargetView tv;
    const C<T>* ainv;   // [nmat][3] alpha^-1
    const C<T>* spec;   // half spectrum (spec_index), scaled by 1/(Lx Ly Lz)
    const C<T>* tw;     // twiddle tables exp(-2 pi i m / 3072) then exp(-2 pi i m / 5120)
    C<T>* Ay;           // [slots][3][P][Ly][K] (x fastest)
    C<T>* Bxy;          // [slots][3][Ly][Lx][Pb] (z fastest, P of Pb used)
    int logW_y;         // log2 of the y lines (adjacent x columns) per CTA of P1 and P5
    int logW_z;         // log2 of the whole z columns per CTA of P3
    int logW_x;         // log2 of the x lines (consecutive z planes) per CTA of P2 and P4
    const int* status;  // optional: right-hand side b is skipped while
                        // status[b * status_stride] != 0
    int status_stride;  // ints between the status words of consecutive RHS
    int conj;           // 1: compute conj(A conj(p)) = A^H p (A complex symmetric)
    const C<T>* jac = nullptr;  // point-Jacobi: when set, y = S A S p with S = diag(jac[mat][axis])
    PassProfiler* prof; // host object; when non-null and on, each pass is timed
    // Batches: p and y hold nb right-hand sides of vstride elements each
    // ([nb][3][N_d]); the work arrays hold `slots` of them.  launch_matvec
    // runs the batch in chunks of at most `slots`; inside a launch, RHS
    // b0 + j uses work slot j.
    int nb = 1;
    int slots = 1;
    int b0 = 0;
    int64_t vstride = 0;
};

// status of right-hand side b (true: skip it)
template <typename T>
__device__ __forceinline__ bool rhs_done(const MatvecView<T>& mv, int b) {
    return mv.status && mv.status[(int64_t)b * mv.status_stride] != 0;
}

// default tile widths for the view's geometry
template <typename T> void configure_matvec(MatvecView<T>& mv);
// whether tile widths (log2 of lines per CTA of P1/P5, P3 and P2/P4) fit the
// launch limits (threads per block, shared memory) for this geometry
template <typename T> bool tiles_ok(const Geometry& g, int logW_y, int logW_z, int logW_x);
// p and y: [nb][3][N_d] vectors of C<IO<T>> (complex128 for the double-float product)
template <typename T> int launch_matvec(const MatvecView<T>& mv, const C<IO<T>>* p, C<IO<T>>* y, cudaStream_t st);

}  // namespace dda
