// Register-resident power-of-two line DFTs for the matvec passes (sm_103a).
//
// Each line of N = 2^logN points is owned by T = N/8 threads; thread t
// holds the eight "canonical" points t + T m (m = 0..7) in registers.  The
// Stockham autosort stages (radix 8, one radix 2 or 4 first when log2 N is
// not a multiple of 3) all read exactly these canonical points, so the
// first stage takes its inputs straight from global memory, every stage
// runs its butterflies in registers, and only the data exchange between two
// stages goes through shared memory (write at the Stockham output
// positions, read back the canonical points).  The last radix-8 stage writes
// its outputs to the canonical positions themselves, so the transform ends
// in registers in natural order: N = 512 costs two shared-memory exchanges.
//
// Shared-memory addresses come from a layout functor (line w, point p):
// RowLayout keeps each line contiguous (lines of the lattice that are
// contiguous in memory, threads t-fastest) with one pad slot per 32 points
// against bank conflicts; ColLayout keeps point-major tiles of W lines side
// by side (strided lines of the lattice, threads w-fastest).
//
// Lines shorter than 8 points (lattice edges of 1 or 2 sites) are done by
// one thread each in registers.  Twiddles come from the FP64 table
// tw[m] = exp(-2 pi i m / 1024) (rounded once for FP32), conjugated for
// the inverse; transforms are unnormalised.
#pragma once

#include "fft.cuh"

namespace dda {

// The paddings below make every exchange of fft_regs take the minimum
// number of shared-memory wavefronts for 8- and 16-byte elements at the
// tile shapes the passes use (checked by replaying the access pattern of
// each stage for N = 16..1024).
struct RowLayout {
    int ld;  // row_ld(N)
    __device__ __forceinline__ int operator()(int w, int p) const { return w * ld + p + (p >> 4); }
};
struct ColLayout {
    int W;   // lines per tile; one pad row after every 8 points
    __device__ __forceinline__ int operator()(int w, int p) const { return (p + (p >> 3)) * W + w; }
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

// In-place DFT of one line held as v[m] = x[t + T m].  All threads of the
// CTA must call it together (it synchronises when it exchanges).
template <typename T, bool INV, class Layout>
__device__ __forceinline__ void fft_regs(C<T> (&v)[8], C<T>* __restrict__ sm, const Layout& L, int w, int t,
                                         int logN, const C<T>* __restrict__ tw) {
    if (logN <= 3) {  // a single stage: one thread holds the whole line
        if (logN == 1) dft2<T, INV>(v);
        else if (logN == 2) dft4<T, INV>(v);
        else if (logN == 3) dft8<T, INV>(v);
        return;
    }
    const int logT = logN - 3, Tn = 1 << logT;
    int logNs = 0;
    const int first = logN % 3;
    // first stage (Ns = 1, no twiddles): radix 2 or 4 on the canonical points
    if (first == 1) {
        // butterflies j = t + q T (q < 4) read x[j + 4T r] = v[q + 4r]
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            C<T> b[2] = {v[q], v[q + 4]};
            dft2<T, INV>(b);
            v[q] = b[0];
            v[q + 4] = b[1];
        }
    } else if (first == 2) {
        // butterflies j = t + q T (q < 2) read x[j + 2T r] = v[q + 2r]
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            C<T> b[4] = {v[q], v[q + 2], v[q + 4], v[q + 6]};
            dft4<T, INV>(b);
            v[q] = b[0]; v[q + 2] = b[1]; v[q + 4] = b[2]; v[q + 6] = b[3];
        }
    } else {
        dft8<T, INV>(v);
    }
    // exchange after the first stage: outputs of butterfly j, point r go to
    // (j / Ns) Ns R + j % Ns + r Ns with Ns = 1, i.e. j R + r
    if (first == 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int r = 0; r < 2; ++r) sm[L(w, (t + q * Tn) * 2 + r)] = v[q + 4 * r];
        logNs = 1;
    } else if (first == 2) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) sm[L(w, (t + q * Tn) * 4 + r)] = v[q + 2 * r];
        logNs = 2;
    } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) sm[L(w, t * 8 + r)] = v[r];
        logNs = 3;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = sm[L(w, t + m * Tn)];
    __syncthreads();
    // radix-8 stages; thread t is butterfly j = t reading v[r] = x[t + T r]
    while (logNs < logN) {
        const int Ns = 1 << logNs;
        const int k = t & (Ns - 1);
        const int step = 10 - logNs - 3;   // twiddle exp(-2 pi i r k / (8 Ns))
        if (sizeof(T) == 4) {
            // FP32: one table load, the other six twiddles as its powers
            // (relative error a few ulp, far below the FP32 transform's own)
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
        dft8<T, INV>(v);
        if (logNs + 3 == logN) break;      // last stage: outputs land on t + T r
        const int base = ((t >> logNs) << (logNs + 3)) + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) sm[L(w, base + r * Ns)] = v[r];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = sm[L(w, t + m * Tn)];
        __syncthreads();
        logNs += 3;
    }
}

}  // namespace dda
