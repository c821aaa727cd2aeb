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
// Shared-memory addresses come from a layout object (line w, point p, and
// the exchange), which also provides the barrier of the exchanges:
// RowLayout keeps each line contiguous (lines of the lattice that are
// contiguous in memory, threads t-fastest) with a bank-conflict pad per
// exchange; ColLayoutT keeps point-major tiles of 2^logW lines side by side
// (strided lines of the lattice, threads w-fastest).
//
// Lines of 3 * 2^a and 5 * 2^a points can also use the wide mapping below
// (M/8 threads of 8R points per line; fft_wide), which needs one exchange
// fewer and no shared-memory closing stage; fft_line picks the mapping
// of Map<T, N>.
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

// ------------------------------------------------------------------------
// Wide mappings.  A line of N points is held by T threads (a power of two,
// so warps hold whole lines) with V points each, t + T m, m < V.  A
// Stockham stage of radix r reads x[j + (N/r) s] for butterfly j < N/r;
// when r divides V, N/r is a multiple of T and thread t takes the V/r
// butterflies j = t + T q, whose inputs are its own points m = q + (V/r) s.
// So the transform is one radix-V stage (each thread one V-point DFT of its
// own points), then stages of radices dividing V over the factor T, every
// stage on the thread's registers, with one shared-memory exchange between
// two stages; the last stage leaves the outputs in natural order on the
// thread's points.
//  * N = R M (R = 3 or 5, M = 2^a >= 8): V = 8R (a prime-factor 8 x R
//    DFT), T = M/8, then radix-8 stages and one radix 2 or 4.  Lines of
//    96, 160, 192 and 320 points need one exchange per transform, 384, 640
//    and 768 two.
//  * N = 2^a >= 128: V = 2^ceil(a/2), T = N/V <= V, then one radix-T stage:
//    one exchange for every length (the 8-point mapping needs two from 128
//    points on).
template <int N>
struct Wide {
    static constexpr bool ODD = Line<N>::ODD;
    static constexpr int R = Line<N>::R;
    static constexpr int V = ODD ? 8 * R : 1 << ((log2c(N) + 1) / 2);   // points per thread, first radix
    static constexpr int T = N / V;                                      // threads per line
    static constexpr int LOGT = log2c(T);
    static constexpr int NSTAGES = ODD ? (LOGT + 2) / 3 : 1;             // stages after the first
    // radix of stage i after the first
    __host__ __device__ static constexpr int radix(int i) {
        return ODD ? ((i < LOGT / 3) ? 8 : 1 << (LOGT % 3)) : T;
    }
    // exchange key of the first exchange: 0, or for a 2^k-point first stage
    // (k >= 4) kPow2Key + k, whose column-tile pad is p >> k
    static constexpr int KEY0 = (!ODD && V >= 16) ? 100 + log2c(V) : 0;
};

// thread mapping the x pass uses for N-point lines of element type C<T>: a
// wide one for 3 * 2^a and 5 * 2^a, and for complex64 2^a lines from 128
// points; eight points per thread otherwise (the complex128 passes are
// bound by the FP64 units, where the one-exchange 2^a form measured slower:
// 10.0 against 9.5 ms for P2 at 256^3)
template <typename T, int N>
struct Map {
    static constexpr bool WIDE = Line<N>::ODD || (N >= 128 && sizeof(T) == 4);
    static constexpr int T_ = WIDE ? Wide<N>::T : Line<N>::T;      // threads per line
    static constexpr int V = WIDE ? Wide<N>::V : 8;               // register slots per thread
    static constexpr int NV = WIDE ? Wide<N>::V : Line<N>::NV;    // points held (N < 8: N)
    static constexpr int NH = WIDE ? Wide<N>::V / 2 : Line<N>::NH; // points of the first half
};
// threads per N-point line of the 8-point mapping, for host code
__host__ __device__ constexpr int line_threads(int N) { return N >= 8 ? N / 8 : 1; }
// whether Map<T, N> (c128: complex128) is a wide mapping, its points and
// threads per line
__host__ __device__ constexpr bool map_wide(int N, bool c128) { return N % 3 == 0 || N % 5 == 0 || (N >= 128 && !c128); }
__host__ __device__ constexpr int wide_points(int N) {
    return (N % 3 == 0) ? 24 : (N % 5 == 0) ? 40 : 1 << ((log2c(N) + 1) / 2);
}
__host__ __device__ constexpr int map_threads(int N, bool c128) {
    return map_wide(N, c128) ? N / wide_points(N) : line_threads(N);
}

// Shared-memory layouts.  An address comes from at<KEY>(w, p) (line w,
// point p), where KEY is log2 of Ns of the stage that writes the exchange;
// the stage writes and the canonical read that follows use the same KEY,
// so each exchange may have a layout of its own.  sync() is the barrier of
// the exchanges.
//
// RowLayout keeps each line contiguous (lines of the lattice that are
// contiguous in memory, threads t-fastest).  An 8-byte access of 16 lanes
// (a half-warp) takes one shared-memory wavefront when its 16 words fall
// in 16 different banks (word mod 16).  The canonical read (16 consecutive
// points, or 8/T lines of T consecutive points) and the stage writes (points
// 8j + r, or runs of Ns) need different pads; the pad of exchange KEY is
//   word = p + c0 (p >> 3) + c1 (p >> 4) + c2 (p >> 6),
// with (c0, c1, c2) = (1, 0, 0) after the first stage and 0 after the
// others for lines of T <= 8 threads (line stride = T mod 2T, row_ld), and (0, 1, 0), (0, 2, 0)
// for Ns = 2 or 4, (0, 0, 8) for Ns = 8, 0 beyond, for T >= 16.  These make
// every exchange of every supported line (24 points and up) conflict-free
// under that rule.  With T a power of two each shift term splits into a
// per-thread part and a compile-time constant, so the pads cost no
// per-access arithmetic.
struct Pad { int c0, c1, c2; };
__host__ __device__ constexpr Pad row_pad(int T, int KEY) {
    return KEY >= 100 ? row_pad(T, 0)
         : T <= 8 ? (KEY == 0 ? Pad{1, 0, 0} : Pad{0, 0, 0})
                  : KEY == 0 ? Pad{0, 1, 0} : KEY <= 2 ? Pad{0, 2, 0} : KEY == 3 ? Pad{0, 0, 8} : Pad{0, 0, 0};
}
__host__ __device__ constexpr int pad_word(Pad c, int p) { return p + c.c0 * (p >> 3) + c.c1 * (p >> 4) + c.c2 * (p >> 6); }
// elements per line of a RowLayout buffer for lines of T threads, the
// line stride of every exchange: the widest padded line of any key, and
// for lines of T <= 8 threads rounded up to T mod 2T, so that the 16/T
// lines a half-warp touches fall in complementary banks
__host__ __device__ constexpr int row_ld(int N, int T) {
    int ld = 0;
    for (int k = 0; k <= 10; ++k) {
        const int l = pad_word(row_pad(T, k), N - 1) + 1;
        ld = l > ld ? l : ld;
    }
    return T >= 16 ? ld : ld + ((T - ld) % (2 * T) + 2 * T) % (2 * T);
}

template <int N, int T>
struct RowLayout {
    template <int KEY>
    __device__ __forceinline__ int at(int w, int p) const {
        return w * row_ld(N, T) + pad_word(row_pad(T, KEY), p);
    }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};
// 2^LOGW lines per tile, point-major (threads w-fastest, strided lines of
// the lattice), with a pad row after every 2^SH points: SH = 3, or after a
// first stage of 2^k points per thread in a wide mapping (key 100 + k)
// SH = k, since that stage writes points 2^k t + r.  (For the first
// exchange of the 8-point mapping of 2^a lines, whose radix-2 or -4 first
// stage writes at stride 2 or 4, a half-warp bank model finds shifts 1 or 2
// conflict-free; in P1 at 256-point lines the larger tiles they need
// measured slower, 0.0372 against 0.0340 ms, so SH stays 3.)  The width is
// a compile-time constant, so every exchange address folds into a constant
// offset from the thread's base.
template <int LOGW>
struct ColLayoutT {
    template <int KEY>
    __device__ __forceinline__ int at(int w, int p) const {
        constexpr int SH = KEY >= 100 ? KEY - 100 : 3;
        return ((p + (p >> SH)) << LOGW) + w;
    }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// elements of a ColLayoutT tile of W lines of N points with a pad row
// after every 2^SH points (SH = 3: the 8-point and the odd wide mappings)
__host__ __device__ constexpr int col_elems_sh(int N, int W, int SH) { return (N + (N >> SH)) * W; }
__host__ __device__ constexpr int col_elems(int N, int W) { return col_elems_sh(N, W, 3); }

template <typename T, bool INV>
__device__ __forceinline__ C<T> twiddle(const C<T>* __restrict__ tw, int idx) {
    C<T> t = ldg_c<T>(tw + idx);
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

// read back the canonical points after the exchange written with key KEY
template <typename T, int N, int NL, int KEY, class Layout>
__device__ __forceinline__ void read_canonical(C<T> (&v)[NL][8], const C<T>* __restrict__ sm, int region,
                                               const Layout& L, int w, int t) {
    constexpr int Tn = N / 8;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int o = L.template at<KEY>(w, t + m * Tn);
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
template <typename T, bool INV, int N, int NL, int KEY, bool TAIL = true, class Layout>
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
            for (int r = 0; r < R; ++r) o[r] = L.template at<KEY>(w, j + r * M);
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
    read_canonical<T, N, NL, KEY>(v, sm, region, L, w, t);
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
                const int o = L.template at<LOGNS>(w, base + r * Ns);
#pragma unroll
                for (int l = 0; l < NL; ++l) sm[l * region + o] = v[l][r];
            }
            if constexpr (LOGNS + 3 < LOGM) {
                L.sync();
                read_canonical<T, N, NL, LOGNS>(v, sm, region, L, w, t);
                // the next stage writes shared memory again, unless it is
                // the last one of a 2^a line (registers only); then only a
                // caller that reuses the buffer (TAIL) needs the barrier
                if constexpr (TAIL || LOGNS + 6 < LOGM || Line<N>::ODD) L.sync();
                Radix8Stages<T, INV, N, LOGNS + 3, NL, HALF_OUT, Layout, TAIL>::run(v, sm, region, L, w, t, tw);
            } else {
                odd_finish<T, INV, N, NL, LOGNS, TAIL>(v, sm, region, L, w, t, tw);
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
        constexpr int K1 = 0;                         // key of the first exchange
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
                    S[L.template at<K1>(w, (t + q * Tn) * 2)] = b[0];
                    S[L.template at<K1>(w, (t + q * Tn) * 2 + 1)] = b[1];
                }
            } else if constexpr (first == 2) {
                // butterflies j = t + q T (q < 2) read x[j + 2T r] = v[q + 2r]
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    C<T> b[4] = {v[l][q], v[l][q + 2], HALF_IN ? mk<T>(0, 0) : v[l][q + 4],
                                 HALF_IN ? mk<T>(0, 0) : v[l][q + 6]};
                    dft4<T, INV>(b);
#pragma unroll
                    for (int r = 0; r < 4; ++r) S[L.template at<K1>(w, (t + q * Tn) * 4 + r)] = b[r];
                }
            } else {
                if (HALF_IN) dft8_half_in<T, INV>(v[l]);
                else dft8<T, INV>(v[l]);
#pragma unroll
                for (int r = 0; r < 8; ++r) S[L.template at<K1>(w, t * 8 + r)] = v[l][r];
            }
        }
        if constexpr (L1 == LOGM) {
            // the first stage was the only power-of-two stage (N = 3 * 8, 5 * 8)
            odd_finish<T, INV, N, NL, K1, TAIL>(v, sm, region, L, w, t, tw);
        } else {
            L.sync();
            read_canonical<T, N, NL, K1>(v, sm, region, L, w, t);
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

__host__ __device__ constexpr int inv_mod(int a, int m) {
    int r = 1;
    while ((a * r) % m != 1 % m) ++r;
    return r;
}

// DFT of NC = 2^B R points in place (prime-factor form, gcd(2^B, R) = 1:
// input n at (R n1 + 2^B n2) mod NC, output k = e1 k1 + e2 k2 mod NC with
// e1 = R (R^-1 mod 2^B), e2 = 2^B (2^-B mod R); 2^B-point DFTs, then
// R-point DFTs, no twiddles)
template <typename T, bool INV, int R, int B>
__device__ __forceinline__ void dft_pfa(C<T> (&x)[R << B]) {
    if constexpr (B == 0) {
        if constexpr (R == 3) dft3<T, INV>(x[0], x[1], x[2]);
        else dft5<T, INV>(x);
    } else {
        constexpr int N1 = 1 << B, NC = R << B;
        constexpr int e1 = R * inv_mod(R % N1, N1), e2 = N1 * inv_mod(N1 % R, R);
        C<T> a[R][N1];
#pragma unroll
        for (int n2 = 0; n2 < R; ++n2) {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) a[n2][n1] = x[(R * n1 + N1 * n2) % NC];
            if constexpr (B == 1) dft2<T, INV>(a[n2]);
            else if constexpr (B == 2) dft4<T, INV>(a[n2]);
            else dft8<T, INV>(a[n2]);
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            C<T> b[R];
#pragma unroll
            for (int n2 = 0; n2 < R; ++n2) b[n2] = a[n2][k1];
            if constexpr (R == 3) dft3<T, INV>(b[0], b[1], b[2]);
            else dft5<T, INV>(b);
#pragma unroll
            for (int k2 = 0; k2 < R; ++k2) x[(e1 * k1 + e2 * k2) % NC] = b[k2];
        }
    }
}

// cos(2 pi n / V) for V = 16, 24, 32 or 40, from the first-quadrant
// values cos(2 pi a / V), a <= V/4, and the symmetries of the cosine
template <int V>
__host__ __device__ constexpr double cos_v(int n) {
    constexpr double q16[5] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173, 0.0};
    constexpr double q24[7] = {1.0, 0.96592582628906828675, 0.86602540378443864676, 0.70710678118654752440,
                               0.5, 0.25881904510252076235, 0.0};
    constexpr double q32[9] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                               0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                               0.19509032201612826785, 0.0};
    constexpr double q40[11] = {1.0, 0.98768834059513772620, 0.95105651629515357212, 0.89100652418836786236,
                                0.80901699437494742410, 0.70710678118654752440, 0.58778525229247312917,
                                0.45399049973954679156, 0.30901699437494742410, 0.15643446504023086901, 0.0};
    n %= V;
    if (n < 0) n += V;
    if (n > V / 2) n = V - n;
    const double sg = n > V / 4 ? -1.0 : 1.0;
    const int a = n > V / 4 ? V / 2 - n : n;
    return sg * (V == 16 ? q16[a] : V == 24 ? q24[a] : V == 32 ? q32[a] : q40[a]);
}
// exp(-+ 2 pi i n / V): forward -, inverse +
template <typename T, bool INV, int V>
__device__ __forceinline__ C<T> root_v(int n) {
    const double c = cos_v<V>(n), s = cos_v<V>(n - V / 4);   // sin = cos(. - pi/2)
    return mk<T>((T)c, INV ? (T)s : (T)-s);
}
// x exp(-+ 2 pi i e / V) for a compile-time e: quarter turns exactly, odd
// eighths with one scale, the rest as a complex product
template <typename T, bool INV, int V>
__device__ __forceinline__ C<T> cmul_root(C<T> x, int e) {
    e %= V;
    if (e < 0) e += V;
    if (e == 0) return x;
    if (4 * e == V) return rot90<T, INV>(x);
    if (2 * e == V) return mk<T>(-x.x, -x.y);
    if (4 * e == 3 * V) return rot90<T, !INV>(x);
    if ((8 * e) % V == 0) {   // (+-1 +- i) / sqrt(2)
        const T h = (T)0.70710678118654752440;
        const double cr = cos_v<V>(e), sr = INV ? cos_v<V>(e - V / 4) : -cos_v<V>(e - V / 4);
        const T c = (T)(cr > 0 ? 1.0 : -1.0), s = (T)(sr > 0 ? 1.0 : -1.0);
        return mk<T>((c * x.x - s * x.y) * h, (c * x.y + s * x.x) * h);
    }
    return cmul<T>(x, root_v<T, INV, V>(e));
}

// DFT of n = 2^k <= 32 points in place, natural order.  n > 8: Cooley-Tukey
// with n = n1 n2 (n1 = 4 for 16, 8 for 32), input index a + n1 b, output
// n2 c + d: n1 DFTs of n2 points over b, the twiddles exp(-+ 2 pi i a d / n),
// then n2 DFTs of n1 points over a.
template <typename T, bool INV, int n>
__device__ __forceinline__ void dft_p2(C<T> (&x)[n]) {
    if constexpr (n == 1) {
    } else if constexpr (n == 2) {
        dft2<T, INV>(x);
    } else if constexpr (n == 4) {
        dft4<T, INV>(x);
    } else if constexpr (n == 8) {
        dft8<T, INV>(x);
    } else {
        constexpr int n1 = n == 16 ? 4 : 8, n2 = n / n1;
        C<T> y[n1][n2];
#pragma unroll
        for (int a = 0; a < n1; ++a) {
#pragma unroll
            for (int b = 0; b < n2; ++b) y[a][b] = x[a + n1 * b];
            dft_p2<T, INV, n2>(y[a]);
#pragma unroll
            for (int d = 1; d < n2; ++d) y[a][d] = cmul_root<T, INV, n>(y[a][d], a * d);
        }
#pragma unroll
        for (int d = 0; d < n2; ++d) {
            C<T> z[n1];
#pragma unroll
            for (int a = 0; a < n1; ++a) z[a] = y[a][d];
            dft_p2<T, INV, n1>(z);
#pragma unroll
            for (int c = 0; c < n1; ++c) x[n2 * c + d] = z[c];
        }
    }
}

// The first stage of a wide mapping: the V-point DFT of the thread's own
// points (prime-factor 8 x R for V = 8R, Cooley-Tukey for V = 2^k).  With
// HALF_IN (inputs V/2.. zero): one radix-2 decimation-in-frequency layer,
// a = x and b = x W_V^n for n < V/2, then V/2-point DFTs of a (even outputs)
// and b (odd outputs).
template <typename T, bool INV, int N, bool HALF_IN>
__device__ __forceinline__ void wide_first(C<T> (&v)[Wide<N>::V]) {
    using W = Wide<N>;
    constexpr int V = W::V, H = V / 2, R = W::R;
    if constexpr (HALF_IN) {
        C<T> a[H], b[H];
#pragma unroll
        for (int n = 0; n < H; ++n) {
            a[n] = v[n];
            b[n] = cmul_root<T, INV, V>(v[n], n);
        }
        if constexpr (W::ODD) {
            dft_pfa<T, INV, R, 2>(a);
            dft_pfa<T, INV, R, 2>(b);
        } else {
            dft_p2<T, INV, H>(a);
            dft_p2<T, INV, H>(b);
        }
#pragma unroll
        for (int k = 0; k < H; ++k) {
            v[2 * k] = a[k];
            v[2 * k + 1] = b[k];
        }
    } else {
        if constexpr (W::ODD) dft_pfa<T, INV, R, 3>(v);
        else dft_p2<T, INV, V>(v);
    }
}

// stage I after the first (radix RDX = Wide<N>::radix(I), Ns = V RDX_0 ...)
// of a wide mapping and the ones after it.  On entry the registers hold the
// canonical points after the exchange; butterfly q (j = t + T q) reads
// v[q + (V/RDX) r] and twiddles it by exp(-+ 2 pi i (j mod Ns) r / (RDX Ns)).
template <typename T, bool INV, int N, int I, int NS, bool TAIL, class Layout>
__device__ __forceinline__ void wide_stages(C<T> (&v)[Wide<N>::V], C<T>* __restrict__ sm, const Layout& L, int w,
                                            int t, const C<T>* __restrict__ tw) {
    using W = Wide<N>;
    constexpr int R = W::R, Tn = W::T, V = W::V, RDX = W::radix(I), NQ = V / RDX;
    constexpr int off = R == 5 ? kTwLen : 0, TWN = R == 5 ? kTw5Len : kTwLen;
    constexpr int step = TWN / (RDX * NS);   // table entries per unit of k r
    constexpr bool LAST = I + 1 == W::NSTAGES;
    // The last stage has Ns = N / RDX > j, so k = t + T q and its twiddles
    // factor as exp(-+ 2 pi i t r / N) exp(-+ 2 pi i q r / V): the first
    // from the table once per thread, the second a compile-time constant.
    // The other stages take k = j mod Ns from the table per butterfly.
    // FP32 forms powers of one table value for r < 8 and takes w^(8g) from
    // the table for the radix-16 and -32 stages (at most four roundings, far
    // below the FP32 transform's own error); FP64 reads every power.
    C<T> wt[RDX];
    if constexpr (LAST) {
        wt[0] = mk<T>(1, 0);
        if (sizeof(T) == 4) {
            wt[1] = twiddle<T, INV>(tw, off + t * step);
#pragma unroll
            for (int r = 2; r < (RDX < 8 ? RDX : 8); ++r)
                wt[r] = (r & 1) ? cmul<T>(wt[r - 1], wt[1]) : cmul<T>(wt[r / 2], wt[r / 2]);
#pragma unroll
            for (int g = 8; g < RDX; g += 8) {
                wt[g] = twiddle<T, INV>(tw, off + t * g * step);
#pragma unroll
                for (int r = 1; r < 8; ++r) wt[g + r] = cmul<T>(wt[g], wt[r]);
            }
        } else {
#pragma unroll
            for (int r = 1; r < RDX; ++r) wt[r] = twiddle<T, INV>(tw, off + t * r * step);
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        C<T> x[RDX], wr[RDX];
        wr[0] = mk<T>(1, 0);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 1; r < RDX; ++r) {
                // the constant factor: for 2^a lines with its trivial angles
                // folded (cmul_root); for 3 * 2^a and 5 * 2^a lines as a
                // plain product, which ptxas schedules better there (the
                // 192-point inverse x pass measured 0.050 against 0.073 ms,
                // while the 512-point forward measured 0.107 against 0.122
                // the other way round)
                if constexpr (W::ODD) wr[r] = q == 0 ? wt[r] : cmul<T>(wt[r], root_v<T, INV, V>(q * r));
                else wr[r] = cmul_root<T, INV, V>(wt[r], q * r);
            }
        } else {
            const int k = (t + Tn * q) % NS;
            if (sizeof(T) == 4) {
                if constexpr (RDX > 1) wr[1] = twiddle<T, INV>(tw, off + k * step);
#pragma unroll
                for (int r = 2; r < RDX; ++r)
                    wr[r] = (r & 1) ? cmul<T>(wr[r - 1], wr[1]) : cmul<T>(wr[r / 2], wr[r / 2]);
            } else {
#pragma unroll
                for (int r = 1; r < RDX; ++r) wr[r] = twiddle<T, INV>(tw, off + k * r * step);
            }
        }
        x[0] = v[q];
#pragma unroll
        for (int r = 1; r < RDX; ++r) x[r] = cmul<T>(v[q + NQ * r], wr[r]);
        dft_p2<T, INV, RDX>(x);
#pragma unroll
        for (int r = 0; r < RDX; ++r) v[q + NQ * r] = x[r];
    }
    if constexpr (!LAST) {
        // exchange: butterfly j's output r goes to (j / Ns) Ns RDX + j mod Ns + r Ns
        constexpr int KEY = 3;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int j = t + Tn * q;
            const int base = (j / NS) * NS * RDX + j % NS;
#pragma unroll
            for (int r = 0; r < RDX; ++r) sm[L.template at<KEY>(w, base + r * NS)] = v[q + NQ * r];
        }
        L.sync();
#pragma unroll
        for (int m = 0; m < V; ++m) v[m] = sm[L.template at<KEY>(w, t + Tn * m)];
        if constexpr (TAIL || I + 2 < W::NSTAGES) L.sync();
        wide_stages<T, INV, N, I + 1, NS * RDX, TAIL>(v, sm, L, w, t, tw);
    }
}

// In-place DFT of one N-point line in its wide mapping: v[m] = x[t + T m],
// m < V.  All threads of the CTA call it together.  HALF_IN: inputs
// m >= V/2 (n >= N/2) are zero.  Outputs the caller never reads are dead
// code, so an inverse that keeps the first half needs no flag.  TAIL: the
// caller reuses the shared buffer afterwards (see fft_lines).
template <typename T, bool INV, int N, bool HALF_IN, bool TAIL = true, class Layout>
__device__ __forceinline__ void fft_wide(C<T> (&v)[Wide<N>::V], C<T>* __restrict__ sm, const Layout& L, int w,
                                         int t, const C<T>* __restrict__ tw) {
    using W = Wide<N>;
    constexpr int Tn = W::T, V = W::V, K0 = W::KEY0;
    wide_first<T, INV, N, HALF_IN>(v);
    if constexpr (W::NSTAGES > 0 && Tn > 1) {
        // exchange: the first stage's output r of thread t goes to t V + r
#pragma unroll
        for (int r = 0; r < V; ++r) sm[L.template at<K0>(w, t * V + r)] = v[r];
        L.sync();
#pragma unroll
        for (int m = 0; m < V; ++m) v[m] = sm[L.template at<K0>(w, t + Tn * m)];
        if constexpr (TAIL || W::NSTAGES > 1) L.sync();
        wide_stages<T, INV, N, 0, V, TAIL>(v, sm, L, w, t, tw);
    }
}

// one line in the mapping Map<T, N> chooses (v[m] = x[t + Map<T, N>::T_ m])
template <typename T, bool INV, int N, bool HALF_IN, bool HALF_OUT, bool TAIL = true, class Layout>
__device__ __forceinline__ void fft_line(C<T> (&v)[Map<T, N>::V], C<T>* __restrict__ sm, const Layout& L, int w,
                                         int t, const C<T>* __restrict__ tw) {
    if constexpr (Map<T, N>::WIDE) fft_wide<T, INV, N, HALF_IN, TAIL>(v, sm, L, w, t, tw);
    else fft_regs<T, INV, N, HALF_IN, HALF_OUT, TAIL>(v, sm, L, w, t, tw);
}

}  // namespace dda
