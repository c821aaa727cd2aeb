// Register-resident line DFTs for the matvec passes (sm_103a), for lines of
// N = 2^a, 3 * 2^a or 5 * 2^a (a >= 3) points.
//
// Each line of N >= 8 points is owned by T = N/8 threads; thread t holds
// the eight "canonical" points t + T m (m = 0..7) in registers.  The
// Stockham autosort stages of the power-of-two factor M (radix 8, one radix
// 2 or 4 first when log2 M is not a multiple of 3) all read exactly these
// canonical points (a radix-8 stage reads stride N/8 = T whatever N's other
// factor), so the first stage takes its inputs straight from global memory,
// every stage runs its butterflies in registers, and only the data exchange
// between two stages goes through shared memory (write at the Stockham
// output positions, read back the canonical points).  For N = 2^a the last
// radix-8 stage writes its outputs to the canonical positions themselves, so
// the transform ends in registers in natural order: N = 512 costs two
// shared-memory exchanges.  For N = R M (R = 3 or 5) the radix-R stage comes
// last (Ns = M): its butterfly j < M reads and writes the positions j + M r,
// r < R, so it runs in place in shared memory after the last radix-8
// exchange, and one more canonical read ends the transform.  The length is a template
// parameter, so every stride, stage count and twiddle step is a
// compile-time constant.
//
// A thread may carry NL lines at once (the three polarisation components of
// a z column): they share the twiddles, the addresses and the barriers of
// every exchange, line l using the shared-memory region sm + l * region.
//
// Pruning (the zero-padding of Sec. 3): the matvec's forward transforms see
// only the first half of each line nonzero (n < L/2 holds every input, since
// L >= 2n - 1 for n lattice points), and its inverse transforms keep only the
// first half of the outputs.  HALF_IN skips the work on the known zeros in
// the first stage; HALF_OUT computes only outputs m < 4 in the last radix-8
// stage of a power-of-two length (a 3 * 2^a or 5 * 2^a length computes all
// outputs).
//
// Shared-memory addresses come from a layout functor (line w, point p),
// which also provides the barrier of the exchanges: RowLayout keeps each
// line contiguous (lines of the lattice that are contiguous in memory,
// threads t-fastest) and RowGroupLayout does the same with a barrier per
// group of lines; ColLayoutT keeps point-major tiles of 2^logW lines side
// by side (strided lines of the lattice, threads w-fastest).
//
// Lines shorter than 8 points (lattice edges of 1 or 2 sites) are done by
// one thread each in registers.  Twiddles come from the FP64 table
// tw[m] = exp(-2 pi i m / 3072), m < 3072, followed by
// tw[3072 + m] = exp(-2 pi i m / 5120), m < 5120 (rounded once for FP32),
// conjugated for the inverse; FP32 stages load one twiddle per butterfly
// and form the others as its powers.  Transforms are unnormalised.
#pragma once

#include "fft.cuh"

namespace dda {

constexpr int kTwLen = 3072;   // first twiddle table: 3 * the longest power-of-two line
constexpr int kTw5Len = 5120;  // second one (lines of 5 * 2^a points), stored after the first

__host__ __device__ constexpr int log2c(int n) { return n <= 1 ? 0 : 1 + log2c(n / 2); }

// shape of the transform of one N-point line
template <int N>
struct Line {
    static constexpr int R = (N % 3) == 0 ? 3 : (N % 5) == 0 ? 5 : 1;   // closing radix (1: none)
    static constexpr bool ODD = R != 1;                                 // N = R M
    static constexpr int M = N / R;                   // power-of-two factor
    static constexpr int LOGM = log2c(M);
    static constexpr int T = N >= 8 ? N / 8 : 1;      // threads per line
    static constexpr int NV = N >= 8 ? 8 : N;         // points per thread
    // points per thread that can hold lattice sites (t + T m with m < NH):
    // an edge of n sites pads to N >= 2n - 1 (N even), so n <= N/2
    static constexpr int NH = N >= 8 ? 4 : (N / 2 > 0 ? N / 2 : 1);
    static_assert(!ODD || M >= 8, "3 * 2^a and 5 * 2^a lengths need a >= 3");
};

template <int N>
struct RowLayout {
    static constexpr int ld = N + N / 16 + 1;
    __device__ __forceinline__ int operator()(int w, int p) const { return w * ld + p + (p >> 4); }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
// RowLayout whose exchanges synchronise only a group of whole warps holding
// whole lines (named barrier `id` > 0 over `count` threads), so that the
// groups of a CTA progress independently; id 0 synchronises the CTA
template <int N>
struct RowGroupLayout {
    static constexpr int ld = N + N / 16 + 1;
    int id, count;
    __device__ __forceinline__ int operator()(int w, int p) const { return w * ld + p + (p >> 4); }
    __device__ __forceinline__ void sync() const {
        if (id == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
    }
};
// lines of N points per barrier group of RowGroupLayout: the fewest whole
// lines that fill whole warps
__host__ __device__ constexpr int row_group_lines(int N) {
    int g = 1;
    while (((N >= 8 ? N / 8 : 1) * g) % 32 != 0) g *= 2;
    return g;
}
// 2^LOGW lines per tile, one pad row after every 8 points; the width is a
// compile-time constant, so every exchange address folds into a constant
// offset from the thread's base
template <int LOGW>
struct ColLayoutT {
    __device__ __forceinline__ int operator()(int w, int p) const { return ((p + (p >> 3)) << LOGW) + w; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

__host__ __device__ constexpr int row_ld(int N) { return N + N / 16 + 1; }
// elements of a ColLayoutT tile of W lines of N points
__host__ __device__ constexpr int col_elems(int N, int W) { return (N + N / 8) * W; }

template <typename T, bool INV>
__device__ __forceinline__ C<T> twiddle(const C<T>* __restrict__ tw, int idx) {
    C<T> t = __ldg(tw + idx);
    if (INV) t.y = -t.y;
    return t;
}

// radix-8 DFT with inputs 4..7 known to be zero: the first layer of dft8
// degenerates to copies
template <typename T, bool INV>
__device__ __forceinline__ void dft8_half_in(C<T>* v) {
    const T h = (T)0.70710678118654752440;
    C<T> a[4] = {v[0], v[1], v[2], v[3]};
    C<T> b[4] = {v[0], v[1], v[2], v[3]};
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

// radix-8 DFT computing only outputs 0..3 (outputs 4..7 left unspecified)
template <typename T, bool INV>
__device__ __forceinline__ void dft8_half_out(C<T>* v) {
    const T h = (T)0.70710678118654752440;
    C<T> a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = cadd<T>(v[r], v[r + 4]);
        b[r] = csub<T>(v[r], v[r + 4]);
    }
    if (INV) {
        b[1] = mk<T>((b[1].x - b[1].y) * h, (b[1].x + b[1].y) * h);
        b[3] = mk<T>((-b[3].x - b[3].y) * h, (b[3].x - b[3].y) * h);
    } else {
        b[1] = mk<T>((b[1].x + b[1].y) * h, (b[1].y - b[1].x) * h);
        b[3] = mk<T>((b[3].y - b[3].x) * h, (-b[3].x - b[3].y) * h);
    }
    b[2] = rot90<T, INV>(b[2]);
    // outputs 0, 2 from the even radix-4 (its outputs 0, 1), 1, 3 from the odd
    const C<T> ca0 = cadd<T>(a[0], a[2]), ca2 = csub<T>(a[0], a[2]);
    const C<T> ca1 = cadd<T>(a[1], a[3]), ca3 = rot90<T, INV>(csub<T>(a[1], a[3]));
    const C<T> cb0 = cadd<T>(b[0], b[2]), cb2 = csub<T>(b[0], b[2]);
    const C<T> cb1 = cadd<T>(b[1], b[3]), cb3 = rot90<T, INV>(csub<T>(b[1], b[3]));
    v[0] = cadd<T>(ca0, ca1);
    v[2] = cadd<T>(ca2, ca3);
    v[1] = cadd<T>(cb0, cb1);
    v[3] = cadd<T>(cb2, cb3);
}

// v[1..7] *= w^r with w = exp(-+ 2 pi i k / (8 Ns)) for each of NL lines
// (table index 3 k 1024 / (8 Ns))
template <typename T, bool INV, int LOGNS, int NL>
__device__ __forceinline__ void twiddle8(C<T> (&v)[NL][8], int k, const C<T>* __restrict__ tw) {
    constexpr int step = 10 - LOGNS - 3;
    k *= 3;
    C<T> w[8];
    if (sizeof(T) == 4) {
        // FP32: one table load, the other six twiddles as its powers
        // (relative error a few ulp, far below the FP32 transform's own)
        w[1] = twiddle<T, INV>(tw, k << step);
        w[2] = cmul<T>(w[1], w[1]); w[3] = cmul<T>(w[2], w[1]); w[4] = cmul<T>(w[2], w[2]);
        w[5] = cmul<T>(w[4], w[1]); w[6] = cmul<T>(w[3], w[3]); w[7] = cmul<T>(w[4], w[3]);
    } else {
#pragma unroll
        for (int r = 1; r < 8; ++r) w[r] = twiddle<T, INV>(tw, (r * k) << step);
    }
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int r = 1; r < 8; ++r) v[l][r] = cmul<T>(v[l][r], w[r]);
}

// read back the canonical points after an exchange
template <typename T, int N, int NL, class Layout>
__device__ __forceinline__ void read_canonical(C<T> (&v)[NL][8], const C<T>* __restrict__ sm, int region,
                                               const Layout& L, int w, int t) {
    constexpr int Tn = N / 8;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int o = L(w, t + m * Tn);
#pragma unroll
        for (int l = 0; l < NL; ++l) v[l][m] = sm[l * region + o];
    }
}

// radix-3 DFT of (a, b, c), forward (exp(-2 pi i / 3)) or inverse
template <typename T, bool INV>
__device__ __forceinline__ void dft3(C<T>& a, C<T>& b, C<T>& c) {
    const T h = (T)0.86602540378443864676;   // sqrt(3) / 2
    const C<T> s = cadd<T>(b, c), d = csub<T>(b, c);
    const C<T> m = mk<T>(a.x - (T)0.5 * s.x, a.y - (T)0.5 * s.y);
    const C<T> r = cscale<T>(rot90<T, INV>(d), h);
    a = cadd<T>(a, s);
    b = cadd<T>(m, r);
    c = csub<T>(m, r);
}

// radix-5 DFT of x[0..4] in place, forward (exp(-2 pi i / 5)) or inverse
template <typename T, bool INV>
__device__ __forceinline__ void dft5(C<T> (&x)[5]) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;   // cos(2 pi/5), cos(4 pi/5)
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;    // sin(2 pi/5), sin(4 pi/5)
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

// After the last radix-8 stage of an N = R M line (R = 3 or 5) has written
// its outputs to the Stockham positions: the radix-R stage (Ns = M) in
// place in shared memory -- butterfly j < M twiddles x[j + M r] by
// exp(-+ 2 pi i j r / N) -- then the canonical read that ends the transform
// in registers.  Thread t takes the butterflies j = t, t + T, ... below M.
template <typename T, bool INV, int N, int NL, bool TAIL = true, class Layout>
__device__ __forceinline__ void odd_finish(C<T> (&v)[NL][8], C<T>* __restrict__ sm, int region,
                                           const Layout& L, int w, int t, const C<T>* __restrict__ tw) {
    constexpr int R = Line<N>::R, M = N / R, Tn = N / 8;
    constexpr int off = R == 3 ? 0 : kTwLen, step = (R == 3 ? kTwLen : kTw5Len) / N;
    constexpr int nq = (M + Tn - 1) / Tn;   // butterflies per thread (3 for R = 3, 2 for R = 5)
    // the twiddles depend on j only: loaded before the barrier, so their
    // latency overlaps the wait (FP32: one load per butterfly and its powers,
    // as in the radix-8 stages; FP64: every power from the table)
    C<T> wq[nq][R];
#pragma unroll
    for (int q = 0; q < nq; ++q) {
        const int j = t + q * Tn, jj = j < M ? j : 0;
        wq[q][0] = mk<T>(1, 0);
        if (sizeof(T) == 4) {
            wq[q][1] = twiddle<T, INV>(tw, off + jj * step);
#pragma unroll
            for (int r = 2; r < R; ++r) wq[q][r] = cmul<T>(wq[q][r - 1], wq[q][1]);
        } else {
#pragma unroll
            for (int r = 1; r < R; ++r) wq[q][r] = twiddle<T, INV>(tw, off + jj * r * step);
        }
    }
    L.sync();
#pragma unroll
    for (int q = 0; q < nq; ++q) {
        const int j = t + q * Tn;
        if (j < M) {
            const C<T>(&wr)[R] = wq[q];
            int o[R];
#pragma unroll
            for (int r = 0; r < R; ++r) o[r] = L(w, j + r * M);
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                C<T>* S = sm + l * region;
                C<T> x[R];
                x[0] = S[o[0]];
#pragma unroll
                for (int r = 1; r < R; ++r) x[r] = cmul<T>(S[o[r]], wr[r]);
                if constexpr (R == 3) {
                    dft3<T, INV>(x[0], x[1], x[2]);
                } else {
                    dft5<T, INV>(x);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) S[o[r]] = x[r];
            }
        }
    }
    L.sync();
    read_canonical<T, N, NL>(v, sm, region, L, w, t);
    if constexpr (TAIL) L.sync();
}

// radix-8 stages from Ns = 2^LOGNS on.  The last one of a 2^a line leaves
// the outputs on the canonical points; that of a 3 * 2^a or 5 * 2^a line
// writes them to shared memory for the closing radix-3 or radix-5 stage.
template <typename T, bool INV, int N, int LOGNS, int NL, bool HALF_OUT, class Layout, bool TAIL = true>
struct Radix8Stages {
    __device__ __forceinline__ static void run(C<T> (&v)[NL][8], C<T>* __restrict__ sm, int region,
                                               const Layout& L, int w, int t, const C<T>* __restrict__ tw) {
        constexpr int Ns = 1 << LOGNS, LOGM = Line<N>::LOGM;
        const int k = t & (Ns - 1);
        twiddle8<T, INV, LOGNS, NL>(v, k, tw);
        if constexpr (LOGNS + 3 < LOGM || Line<N>::ODD) {
#pragma unroll
            for (int l = 0; l < NL; ++l) dft8<T, INV>(v[l]);
            const int base = ((t >> LOGNS) << (LOGNS + 3)) + k;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int o = L(w, base + r * Ns);
#pragma unroll
                for (int l = 0; l < NL; ++l) sm[l * region + o] = v[l][r];
            }
            if constexpr (LOGNS + 3 < LOGM) {
                L.sync();
                read_canonical<T, N, NL>(v, sm, region, L, w, t);
                // the next stage writes shared memory again, unless it is
                // the last one of a 2^a line (registers only); then only a
                // caller that reuses the buffer (TAIL) needs the barrier
                if constexpr (TAIL || LOGNS + 6 < LOGM || Line<N>::ODD) L.sync();
                Radix8Stages<T, INV, N, LOGNS + 3, NL, HALF_OUT, Layout, TAIL>::run(v, sm, region, L, w, t, tw);
            } else {
                odd_finish<T, INV, N, NL, TAIL>(v, sm, region, L, w, t, tw);
            }
        } else {
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                if (HALF_OUT) dft8_half_out<T, INV>(v[l]);
                else dft8<T, INV>(v[l]);
            }
        }
    }
};

// In-place DFT of NL lines held as v[l][m] = x_l[t + T m].  All threads of
// the CTA must call it together (it synchronises when it exchanges).
// HALF_IN: inputs m >= 4 are zero.  HALF_OUT: only outputs m < 4 are needed.
// TAIL: the caller reuses the shared buffer afterwards, so the transform
// ends with a barrier after its last shared-memory read (false when nothing
// touches the buffer again, e.g. the kernel's last transform).
template <typename T, bool INV, int N, int NL, bool HALF_IN, bool HALF_OUT, bool TAIL = true, class Layout>
__device__ __forceinline__ void fft_lines(C<T> (&v)[NL][8], C<T>* __restrict__ sm, int region, const Layout& L,
                                          int w, int t, const C<T>* __restrict__ tw) {
    if constexpr (N <= 8 && !Line<N>::ODD) {  // a single stage: one thread holds the whole line
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            if constexpr (N == 2) dft2<T, INV>(v[l]);
            else if constexpr (N == 4) dft4<T, INV>(v[l]);
            else dft8<T, INV>(v[l]);
        }
    } else {
        constexpr int Tn = N / 8, LOGM = Line<N>::LOGM;
        constexpr int first = LOGM % 3;
        constexpr int L1 = first == 0 ? 3 : first;   // log2 of the first radix
        // first stage (Ns = 1, no twiddles): outputs of butterfly j, point r
        // go to j R + r
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            C<T>* S = sm + l * region;
            if constexpr (first == 1) {
                // butterflies j = t + q T (q < 4) read x[j + 4T r] = v[q + 4r]
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    C<T> b[2] = {v[l][q], HALF_IN ? v[l][q] : v[l][q + 4]};
                    if (!HALF_IN) dft2<T, INV>(b);
                    S[L(w, (t + q * Tn) * 2)] = b[0];
                    S[L(w, (t + q * Tn) * 2 + 1)] = b[1];
                }
            } else if constexpr (first == 2) {
                // butterflies j = t + q T (q < 2) read x[j + 2T r] = v[q + 2r]
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    C<T> b[4] = {v[l][q], v[l][q + 2], HALF_IN ? mk<T>(0, 0) : v[l][q + 4],
                                 HALF_IN ? mk<T>(0, 0) : v[l][q + 6]};
                    dft4<T, INV>(b);
#pragma unroll
                    for (int r = 0; r < 4; ++r) S[L(w, (t + q * Tn) * 4 + r)] = b[r];
                }
            } else {
                if (HALF_IN) dft8_half_in<T, INV>(v[l]);
                else dft8<T, INV>(v[l]);
#pragma unroll
                for (int r = 0; r < 8; ++r) S[L(w, t * 8 + r)] = v[l][r];
            }
        }
        if constexpr (L1 == LOGM) {
            // the first stage was the only power-of-two stage (N = 3 * 8, 5 * 8)
            odd_finish<T, INV, N, NL, TAIL>(v, sm, region, L, w, t, tw);
        } else {
            L.sync();
            read_canonical<T, N, NL>(v, sm, region, L, w, t);
            if constexpr (TAIL || L1 + 3 < LOGM || Line<N>::ODD) L.sync();
            Radix8Stages<T, INV, N, L1, NL, HALF_OUT, Layout, TAIL>::run(v, sm, region, L, w, t, tw);
        }
    }
}

// one line: v[m] = x[t + T m]
template <typename T, bool INV, int N, bool HALF_IN, bool HALF_OUT, bool TAIL = true, class Layout>
__device__ __forceinline__ void fft_regs(C<T> (&v)[8], C<T>* __restrict__ sm, const Layout& L, int w, int t,
                                         const C<T>* __restrict__ tw) {
    C<T>(&vv)[1][8] = *reinterpret_cast<C<T>(*)[1][8]>(&v);
    fft_lines<T, INV, N, 1, HALF_IN, HALF_OUT, TAIL>(vv, sm, 0, L, w, t, tw);
}

}  // namespace dda
