// Batched line DFTs on a shared-memory tile (sm_103a), for lines of 2^a or
// 3 * 2^a points.
//
// The 3D DFTs of the DDA matvec are done as ensembles of 1D line transforms
// (OpenDDA Sec. 3).  Here a CTA holds W lines of N points in shared memory,
// element (line w, point n) at buf[n * ld + w] (ld >= W, lines side by side
// so that strided lines of the lattice load with coalesced rows), and
// transforms all of them in place with the Stockham autosort scheme: each
// stage of radix R (8, with one 2 or 4 first when log2 N is not a multiple
// of 3) reads R points at stride N/R, twiddles, does a radix-R DFT in
// registers, and writes them at stride Ns (the product of the radices done
// so far), so that the result comes out in natural order without a
// bit-reversal pass.  Every thread owns V points per stage (V/R butterflies);
// the launch uses exactly W*N/V threads.  A stage reads everything into
// registers, synchronises, then writes, so one buffer suffices.
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / 3072) computed in FP64
// on the host (rounded once for the FP32 table); the inverse transform uses
// their conjugates.  Lines of N = 3 * 2^a points end with a radix-3 stage.
// Transforms are unnormalised.
#pragma once

#include "common.cuh"

namespace dda {

template <typename T, bool INV>
__device__ __forceinline__ C<T> rot90(C<T> a) {  // times -i (forward) or +i (inverse)
    return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft2(C<T>* v) {
    const C<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
}

// radix-4 by decimation in frequency; outputs in natural order
template <typename T, bool INV>
__device__ __forceinline__ void dft4(C<T>* v) {
    const C<T> c0 = cadd<T>(v[0], v[2]), c2 = csub<T>(v[0], v[2]);
    const C<T> c1 = cadd<T>(v[1], v[3]), c3 = rot90<T, INV>(csub<T>(v[1], v[3]));
    v[0] = cadd<T>(c0, c1);
    v[2] = csub<T>(c0, c1);
    v[1] = cadd<T>(c2, c3);
    v[3] = csub<T>(c2, c3);
}

// radix-8: one radix-2 decimation-in-frequency layer with the internal
// twiddles W8^r, then two radix-4 DFTs on the even and odd outputs
template <typename T, bool INV>
__device__ __forceinline__ void dft8(C<T>* v) {
    const T h = (T)0.70710678118654752440;  // 1/sqrt(2)
    C<T> a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = cadd<T>(v[r], v[r + 4]);
        b[r] = csub<T>(v[r], v[r + 4]);
    }
    // b1 *= W8^1, b2 *= W8^2, b3 *= W8^3 (conjugated for the inverse)
    if (INV) {
        b[1] = mk<T>((b[1].x - b[1].y) * h, (b[1].x + b[1].y) * h);
        b[3] = mk<T>((-b[3].x - b[3].y) * h, (b[3].x - b[3].y) * h);
    } else {
        b[1] = mk<T>((b[1].x + b[1].y) * h, (b[1].y - b[1].x) * h);
        b[3] = mk<T>((b[3].y - b[3].x) * h, (-b[3].x - b[3].y) * h);
    }
    b[2] = rot90<T, INV>(b[2]);
    dft4<T, INV>(a);
    dft4<T, INV>(b);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        v[2 * r] = a[r];
        v[2 * r + 1] = b[r];
    }
}

template <typename T, int R, bool INV>
__device__ __forceinline__ void dftR(C<T>* v) {
    if (R == 2) dft2<T, INV>(v);
    else if (R == 4) dft4<T, INV>(v);
    else dft8<T, INV>(v);
}

// One Stockham stage of radix R over the whole tile.
template <typename T, int V, int R, bool INV>
__device__ __forceinline__ void fft_stage(C<T>* __restrict__ buf, int ld, int logW, int N, int logNs,
                                          const C<T>* __restrict__ tw, int logTwStep) {
    constexpr int B = V / R;  // butterflies per thread
    const int NT = blockDim.x;
    const int tid = threadIdx.x;
    const int W = 1 << logW;
    const int NR = N / R;
    const int Ns = 1 << logNs;
    C<T> v[B][R];
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int g = tid + q * NT;
        const int w = g & (W - 1);
        const int j = g >> logW;
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = buf[(j + r * NR) * ld + w];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int g = tid + q * NT;
        const int w = g & (W - 1);
        const int j = g >> logW;
        const int k = j & (Ns - 1);
        if (logNs > 0) {
            // twiddle exp(-+ 2 pi i r k / (Ns R)) = tw[3 r k * 1024 / (Ns R)]
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C<T> t = __ldg(tw + ((3 * r * k) << logTwStep));
                if (INV) t.y = -t.y;
                v[q][r] = cmul<T>(v[q][r], t);
            }
        }
        dftR<T, R, INV>(v[q]);
        const int base = ((j >> logNs) << logNs) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(base + r * Ns) * ld + w] = v[q][r];
    }
    __syncthreads();
}

// The closing radix-3 stage of an N = 3M line (Ns = M): butterfly j < M
// twiddles x[j + M r] by exp(-+ 2 pi i j r / N) = tw[3072 j r / N] and
// transforms the three points in place.  W M butterflies over the CTA.
template <typename T, bool INV>
__device__ __forceinline__ void fft_stage3(C<T>* __restrict__ buf, int ld, int logW, int N,
                                           const C<T>* __restrict__ tw) {
    const int M = N / 3, W = 1 << logW, step = 3072 / N;
    const T h = (T)0.86602540378443864676;   // sqrt(3) / 2
    for (int g = threadIdx.x; g < W * M; g += blockDim.x) {
        const int w = g & (W - 1), j = g >> logW;
        C<T> t1 = __ldg(tw + j * step), t2 = __ldg(tw + 2 * j * step);
        if (INV) { t1.y = -t1.y; t2.y = -t2.y; }
        const C<T> a = buf[j * ld + w];
        const C<T> b = cmul<T>(buf[(j + M) * ld + w], t1), c = cmul<T>(buf[(j + 2 * M) * ld + w], t2);
        const C<T> s = cadd<T>(b, c), d = csub<T>(b, c);
        const C<T> m = mk<T>(a.x - (T)0.5 * s.x, a.y - (T)0.5 * s.y);
        const C<T> r = cscale<T>(rot90<T, INV>(d), h);
        buf[j * ld + w] = cadd<T>(a, s);
        buf[(j + M) * ld + w] = cadd<T>(m, r);
        buf[(j + 2 * M) * ld + w] = csub<T>(m, r);
    }
    __syncthreads();
}

// In-place DFT of the W = 2^logW lines of N points (N = 2^a, or 3 * 2^a with
// a >= 3) of a tile: the Stockham stages of the power-of-two factor, then
// the radix-3 stage.  tw: table of 3072 entries exp(-2 pi i m / 3072).
// Requires blockDim.x * V == W * N.
template <typename T, int V, bool INV>
__device__ __forceinline__ void fft_tile(C<T>* __restrict__ buf, int ld, int logW, int N,
                                         const C<T>* __restrict__ tw) {
    const int M = (N % 3) ? N : N / 3;
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    const int logMax = 10;  // log2 of the longest power-of-two line
    int logNs = 0;
    const int first = logM % 3;
    if (first == 1) {
        fft_stage<T, V, 2, INV>(buf, ld, logW, N, 0, tw, logMax - 1);
        logNs = 1;
    } else if (first == 2) {
        fft_stage<T, V, 4, INV>(buf, ld, logW, N, 0, tw, logMax - 2);
        logNs = 2;
    }
    while (logNs < logM) {
        fft_stage<T, V, 8, INV>(buf, ld, logW, N, logNs, tw, logMax - logNs - 3);
        logNs += 3;
    }
    if (M != N) fft_stage3<T, INV>(buf, ld, logW, N, tw);
}

}  // namespace dda
