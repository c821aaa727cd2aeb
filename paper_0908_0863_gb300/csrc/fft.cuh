// Batched line DFTs on a shared-memory tile (sm_103a), for lines of 2^a,
// 3 * 2^a or 5 * 2^a points.
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
// Twiddles come from the tables exp(-2 pi i m / 3072) and, after it,
// exp(-2 pi i m / 5120), computed in FP64 on the host (rounded once for
// FP32); the inverse transform uses their conjugates.  Lines of 3 * 2^a and
// 5 * 2^a points end with a radix-3 or radix-5 stage.  Transforms are
// unnormalised.
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

// The closing stage of an N = R M line (R = 3 or 5, Ns = M): butterfly j < M
// twiddles x[j + M r] by exp(-+ 2 pi i j r / N) and transforms the R points
// in place.  Twiddles: tw[3072 j r / N] for R = 3, tw[3072 + 5120 j r / N]
// for R = 5.  W M butterflies over the CTA.
template <typename T, int R, bool INV>
__device__ __forceinline__ void fft_stage_odd(C<T>* __restrict__ buf, int ld, int logW, int N,
                                              const C<T>* __restrict__ tw) {
    const int M = N / R, W = 1 << logW;
    const int off = R == 3 ? 0 : 3072, step = (R == 3 ? 3072 : 5120) / N;
    for (int g = threadIdx.x; g < W * M; g += blockDim.x) {
        const int w = g & (W - 1), j = g >> logW;
        C<T> x[R];
        x[0] = buf[j * ld + w];
#pragma unroll
        for (int r = 1; r < R; ++r) {
            C<T> t = __ldg(tw + off + j * r * step);
            if (INV) t.y = -t.y;
            x[r] = cmul<T>(buf[(j + r * M) * ld + w], t);
        }
        if constexpr (R == 3) {
            const T h = (T)0.86602540378443864676;   // sqrt(3) / 2
            const C<T> s = cadd<T>(x[1], x[2]), d = csub<T>(x[1], x[2]);
            const C<T> m = mk<T>(x[0].x - (T)0.5 * s.x, x[0].y - (T)0.5 * s.y);
            const C<T> rr = cscale<T>(rot90<T, INV>(d), h);
            x[0] = cadd<T>(x[0], s);
            x[1] = cadd<T>(m, rr);
            x[2] = csub<T>(m, rr);
        } else {
            const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
            const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
            const C<T> a1 = cadd<T>(x[1], x[4]), b1 = csub<T>(x[1], x[4]);
            const C<T> a2 = cadd<T>(x[2], x[3]), b2 = csub<T>(x[2], x[3]);
            const C<T> t1 = mk<T>(x[0].x + c1 * a1.x + c2 * a2.x, x[0].y + c1 * a1.y + c2 * a2.y);
            const C<T> t2 = mk<T>(x[0].x + c2 * a1.x + c1 * a2.x, x[0].y + c2 * a1.y + c1 * a2.y);
            const C<T> u1 = rot90<T, INV>(mk<T>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
            const C<T> u2 = rot90<T, INV>(mk<T>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
            x[0] = cadd<T>(x[0], cadd<T>(a1, a2));
            x[1] = cadd<T>(t1, u1);
            x[4] = csub<T>(t1, u1);
            x[2] = cadd<T>(t2, u2);
            x[3] = csub<T>(t2, u2);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(j + r * M) * ld + w] = x[r];
    }
    __syncthreads();
}

// In-place DFT of the W = 2^logW lines of N points (N = 2^a, or 3 * 2^a or
// 5 * 2^a with a >= 3) of a tile: the Stockham stages of the power-of-two
// factor, then the closing radix-3 or radix-5 stage.  tw: the tables
// exp(-2 pi i m / 3072) (3072 entries) and exp(-2 pi i m / 5120) (5120
// entries, after the first).  Requires blockDim.x * V == W * N.
template <typename T, int V, bool INV>
__device__ __forceinline__ void fft_tile(C<T>* __restrict__ buf, int ld, int logW, int N,
                                         const C<T>* __restrict__ tw) {
    const int R = (N % 3) == 0 ? 3 : (N % 5) == 0 ? 5 : 1;
    const int M = N / R;
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
    if (R == 3) fft_stage_odd<T, 3, INV>(buf, ld, logW, N, tw);
    else if (R == 5) fft_stage_odd<T, 5, INV>(buf, ld, logW, N, tw);
}

}  // namespace dda
