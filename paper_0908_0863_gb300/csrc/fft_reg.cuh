// Register-resident power-of-two line DFTs for the matvec passes (sm_103a).
//
// Each line of N = 2^LOGN points is owned by T = N/8 threads; thread t
// holds the eight "canonical" points t + T m (m = 0..7) in registers.  The
// Stockham autosort stages (radix 8, one radix 2 or 4 first when LOGN is
// not a multiple of 3) all read exactly these canonical points, so the
// first stage takes its inputs straight from global memory, every stage
// runs its butterflies in registers, and only the data exchange between two
// stages goes through shared memory (write at the Stockham output
// positions, read back the canonical points).  The last radix-8 stage writes
// its outputs to the canonical positions themselves, so the transform ends
// in registers in natural order: N = 512 costs two shared-memory exchanges.
// The length is a template parameter, so every stride, stage count and
// twiddle step is a compile-time constant.
//
// Shared-memory addresses come from a layout functor (line w, point p):
// RowLayout keeps each line contiguous (lines of the lattice that are
// contiguous in memory, threads t-fastest); ColLayout keeps point-major
// tiles of 2^logW lines side by side (strided lines of the lattice, threads
// w-fastest).  Their paddings make every exchange take the minimum number
// of shared-memory wavefronts for 8- and 16-byte elements at the tile
// shapes the passes use (checked by replaying each stage's access pattern
// for N = 16..1024).
//
// Lines shorter than 8 points (lattice edges of 1 or 2 sites) are done by
// one thread each in registers.  Twiddles come from the FP64 table
// tw[m] = exp(-2 pi i m / 1024) (rounded once for FP32), conjugated for the
// inverse; FP32 stages load one twiddle and form the other six as its
// powers.  Transforms are unnormalised.
#pragma once

#include "fft.cuh"

namespace dda {

template <int LOGN>
struct RowLayout {
    static constexpr int N = 1 << LOGN;
    static constexpr int ld = N + N / 16 + 1;
    __device__ __forceinline__ int operator()(int w, int p) const { return w * ld + p + (p >> 4); }
};
struct ColLayout {
    int logW;  // 2^logW lines per tile; one pad row after every 8 points
    __device__ __forceinline__ int operator()(int w, int p) const { return ((p + (p >> 3)) << logW) + w; }
};

__host__ __device__ inline int row_ld(int N) { return N + N / 16 + 1; }
// elements of a ColLayout tile of W lines of N points
__host__ __device__ inline int col_elems(int N, int W) { return (N + N / 8) * W; }

template <typename T, bool INV>
__device__ __forceinline__ C<T> twiddle(const C<T>* __restrict__ tw, int idx) {
    C<T> t = __ldg(tw + idx);
    if (INV) t.y = -t.y;
    return t;
}

// v[1..7] *= w^r with w = exp(-+ 2 pi i k / (8 Ns)), k = index of the butterfly
template <typename T, bool INV, int LOGNS>
__device__ __forceinline__ void twiddle8(C<T> (&v)[8], int k, const C<T>* __restrict__ tw) {
    constexpr int step = 10 - LOGNS - 3;
    if (sizeof(T) == 4) {
        const C<T> w1 = twiddle<T, INV>(tw, k << step);
        const C<T> w2 = cmul<T>(w1, w1), w3 = cmul<T>(w2, w1), w4 = cmul<T>(w2, w2);
        const C<T> w5 = cmul<T>(w4, w1), w6 = cmul<T>(w3, w3), w7 = cmul<T>(w4, w3);
        v[1] = cmul<T>(v[1], w1); v[2] = cmul<T>(v[2], w2); v[3] = cmul<T>(v[3], w3);
        v[4] = cmul<T>(v[4], w4); v[5] = cmul<T>(v[5], w5); v[6] = cmul<T>(v[6], w6);
        v[7] = cmul<T>(v[7], w7);
    } else {
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = cmul<T>(v[r], twiddle<T, INV>(tw, (r * k) << step));
    }
}

// read back the canonical points after an exchange
template <typename T, int LOGN, class Layout>
__device__ __forceinline__ void read_canonical(C<T> (&v)[8], const C<T>* __restrict__ sm, const Layout& L, int w,
                                               int t) {
    constexpr int Tn = 1 << (LOGN - 3);
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = sm[L(w, t + m * Tn)];
}

// radix-8 stages from Ns = 2^LOGNS on; the last one leaves the outputs on
// the canonical points
template <typename T, bool INV, int LOGN, int LOGNS, class Layout>
struct Radix8Stages {
    __device__ __forceinline__ static void run(C<T> (&v)[8], C<T>* __restrict__ sm, const Layout& L, int w, int t,
                                               const C<T>* __restrict__ tw) {
        constexpr int Ns = 1 << LOGNS;
        const int k = t & (Ns - 1);
        twiddle8<T, INV, LOGNS>(v, k, tw);
        dft8<T, INV>(v);
        if constexpr (LOGNS + 3 < LOGN) {
            const int base = ((t >> LOGNS) << (LOGNS + 3)) + k;
#pragma unroll
            for (int r = 0; r < 8; ++r) sm[L(w, base + r * Ns)] = v[r];
            __syncthreads();
            read_canonical<T, LOGN>(v, sm, L, w, t);
            __syncthreads();
            Radix8Stages<T, INV, LOGN, LOGNS + 3, Layout>::run(v, sm, L, w, t, tw);
        }
    }
};

// In-place DFT of one line held as v[m] = x[t + T m].  All threads of the
// CTA must call it together (it synchronises when it exchanges).
template <typename T, bool INV, int LOGN, class Layout>
__device__ __forceinline__ void fft_regs(C<T> (&v)[8], C<T>* __restrict__ sm, const Layout& L, int w, int t,
                                         const C<T>* __restrict__ tw) {
    if constexpr (LOGN <= 3) {  // a single stage: one thread holds the whole line
        if constexpr (LOGN == 1) dft2<T, INV>(v);
        else if constexpr (LOGN == 2) dft4<T, INV>(v);
        else dft8<T, INV>(v);
    } else {
        constexpr int Tn = 1 << (LOGN - 3);
        constexpr int first = LOGN % 3;
        // first stage (Ns = 1, no twiddles): outputs of butterfly j, point r
        // go to j R + r
        if constexpr (first == 1) {
            // butterflies j = t + q T (q < 4) read x[j + 4T r] = v[q + 4r]
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                C<T> b[2] = {v[q], v[q + 4]};
                dft2<T, INV>(b);
                sm[L(w, (t + q * Tn) * 2)] = b[0];
                sm[L(w, (t + q * Tn) * 2 + 1)] = b[1];
            }
        } else if constexpr (first == 2) {
            // butterflies j = t + q T (q < 2) read x[j + 2T r] = v[q + 2r]
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                C<T> b[4] = {v[q], v[q + 2], v[q + 4], v[q + 6]};
                dft4<T, INV>(b);
#pragma unroll
                for (int r = 0; r < 4; ++r) sm[L(w, (t + q * Tn) * 4 + r)] = b[r];
            }
        } else {
            dft8<T, INV>(v);
#pragma unroll
            for (int r = 0; r < 8; ++r) sm[L(w, t * 8 + r)] = v[r];
        }
        __syncthreads();
        read_canonical<T, LOGN>(v, sm, L, w, t);
        __syncthreads();
        Radix8Stages<T, INV, LOGN, (first == 0 ? 3 : first), Layout>::run(v, sm, L, w, t, tw);
    }
}

}  // namespace dda
