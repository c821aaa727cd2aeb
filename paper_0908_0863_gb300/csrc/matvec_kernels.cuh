// Kernels and per-length launchers of the pruned FFT matrix-vector product
// y = A p of the DDA (OpenDDA Sec. 3).  Each of the translation units
// mv_p1_*.cu, mv_p3_*.cu, mv_p5_*.cu and mv_rows_*.cu instantiates one pass for
// every line length (and tile width) and exposes its dispatcher; matvec.cu
// sequences the passes.
//
// Five stream-ordered passes over device arrays:
//   P1  expand + y-forward   compressed p -> Ay[3][P][Ly][K] (x fastest;  K*P lines per component;
//                            a thread gathers a site's three components together)
//   P2  x-forward            Ay -> Bxy[3][Ly][Lx][Pb] (z fastest)      (Ly*P lines, K nonzero inputs)
//   P3  z conv               per (ix, jy): z-forward of the 3 components (P nonzero
//                            inputs), the 3x3 spectrum product of Eqs. 6-8 with the
//                            signed mirror lookup, z-inverse keeping k < P, in place
//   P4  x-inverse            Bxy -> Ay, keeping i < K
//   P5  y-inverse + compress Ay -> y, keeping j < J, y = alpha^-1 p + conv for
//                            occupied sites (Sec. 4 zero storage)
// The line counts are the paper's pruned ones (Sec. 3, Table 2): forward
// y 3[K x P], x 3[J'' x P], z all K'' x J''; the inverse mirrors them.  The
// 1/(Lx Ly Lz) normalisation of the inverse DFT is folded into the stored
// spectrum.  Within each line, forward transforms skip the work on the
// zero half of their input and inverse transforms compute only the half of
// the output that is kept.
//
// Layout of the xy-transformed volume: every z line of Bxy is contiguous,
// and so is every z line of the half spectrum ([Hy][Hx][Hz][6]).  The z
// pass, which does most of the work (a forward and an inverse transform of
// every line, and the product), therefore runs small independent CTAs of a
// few whole columns each, so that while some wait for memory others
// compute.  The transpose between x-fastest Ay and z-fastest Bxy is done by
// P2 and P4 through shared memory, on tiles of Wz x lines of consecutive z.
//
// Batches: one launch of each pass covers up to `slots` right-hand sides
// that share the context's spectrum (vectors [nb][3][N_d], work arrays one
// per slot); a right-hand side whose solver status is no longer "running"
// is skipped block by block.  The slot is a grid coordinate of its own (no
// index division in the kernels); in P3 it is the fastest-varying one, so
// the CTAs of all right-hand sides that read one spectrum line run back to
// back and the line is fetched from HBM once.
//
// Every pass keeps its lines in registers (fft_reg.cuh): points are loaded
// from global memory straight into the registers of the first DFT stage and
// stored from the registers of the last, and only the exchanges between
// stages use shared memory.  Strided y lines (P1, P5) are processed W at a
// time, W adjacent columns so that each load and store touches W
// contiguous elements.  In P3 each thread carries the same column of all
// three components, so the spectrum product happens in registers between
// the forward and the inverse transforms; in P1 it gathers a site's three
// components with one occupancy and rank lookup.  Each kernel is compiled
// for every line length N (2^a up to 1024, 3 * 2^a from 24 to 768, 5 * 2^a
// from 40 to 640) and, for P1 and P5, every tile width (LOGW = 0..4 lines
// per CTA, log2), and picked at launch.
#pragma once

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "fft_reg.cuh"
#include "matvec.cuh"

namespace dda {



// P3 keeps 3 x 8 complex values per thread: at most 512 threads per CTA for
// complex64, 256 for complex128.  With the wide mapping (3 * 2^a, 5 * 2^a)
// a thread keeps one component's 8R points (24 or 40): at most 256.
template <typename T> __host__ __device__ constexpr int p3_max_threads(int N) {
    return wide_len(N) ? 256 : (sizeof(T) == 4 ? 512 : 256);
}
// threads of one z column in P3: its three components share the T = N/8
// threads of the 8-point mapping, or take 3 x M/8 in the wide one
__host__ __device__ constexpr int p3_col_threads(int N) { return wide_len(N) ? 3 * map_threads(N, false) : line_threads(N); }
// threads of one z line in P3 (what its shared-memory pads are laid out for)
__host__ __device__ constexpr int p3_line_threads(int N) { return wide_len(N) ? map_threads(N, false) : line_threads(N); }
// widest tiles the runtime widths of P3 (columns per CTA) and P2/P4 (z lines
// per CTA) may take, as log2
constexpr int kMaxLogR = 6;
constexpr int kMaxLogZ = 4;
// P2/P4 keep eight points of one row per thread: up to 1024 threads per CTA;
// with a wide mapping (3 * 2^a and 5 * 2^a rows: 24 or 40 points per
// thread; 2^a rows from 128 points: 16 or 32) up to 256, which leaves the
// registers for them
constexpr int kRowThreads = 1024;
constexpr int kRowThreadsWide = 256;
__host__ __device__ constexpr int rows_max_threads(int N, bool c128) { return map_wide(N, c128) ? kRowThreadsWide : kRowThreads; }

// P1 and P5 keep the eight points, their gather indices and (P5) the
// gathered entries of p in registers: at most 512 threads per CTA leave
// room for them (the complex64 P5 is held to two such CTAs per SM, which
// measured faster than one with no register cap).  They keep the 8-point
// mapping for 3 * 2^a and 5 * 2^a lines too: with 8R points per thread the
// gather's registers (P1 before, P5 beside the transform) cost more
// occupancy than the wide mapping saves.
constexpr int kYThreads = 512;

// elements of one slot of the work arrays
__host__ __device__ __forceinline__ int64_t ay_elems(const Geometry& g) { return 3LL * g.P * g.Ly * g.K; }
__host__ __device__ __forceinline__ int64_t bxy_elems(const Geometry& g) { return 3LL * g.Pb * g.Ly * g.Lx; }
// Element offsets inside one work slot of Bxy ([3][Ly][Lx][Pb], columns of
// P values at pitch Pb) and inside the half spectrum fit in 32 bits for
// every lattice the library accepts (edges <= 512: 3 Ly Lx Pb < 2^31,
// 6 Hy Hx Hz < 2^31).

// ---------------------------------------------------------------- P1
template <typename T, int N, int LOGW>
__global__ void __launch_bounds__(kYThreads) k_p1(MatvecView<T> mv, const C<IO<T>>* __restrict__ p) {
    // the three components of a site share its occupancy and rank lookup:
    // each thread gathers all three and transforms them as three lines
    const int j = blockIdx.z;                                  // batch slot
    const int b = mv.b0 + j;
    if (rhs_done(mv, b)) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
    constexpr int TL = Line<N>::T, nv = Line<N>::NV;
    const Geometry& g = mv.g;
    constexpr int W = 1 << LOGW, region = col_elems(N, W);
    const int w = threadIdx.x & (W - 1), t = threadIdx.x >> LOGW;
    const int i = blockIdx.x * W + w, kz = blockIdx.y;
    const C<IO<T>>* pb = p + (int64_t)b * mv.vstride;
    const int64_t s0 = (int64_t)kz * g.J * g.K + i;
    // the gather as two rounds of independent loads: first the occupancy and
    // rank words of the thread's sites, then their entries of p (three
    // components each).  Only the first half of the points can hold sites
    // (J <= N/2).
    constexpr int nh = Line<N>::NH;
    uint32_t word[nh], rbase[nh];
    const bool inx = i < g.K;
#pragma unroll
    for (int m = 0; m < nh; ++m) {
        const int n = t + m * TL;
        const bool in = inx && n < g.J;
        const int64_t q = (s0 + (int64_t)n * g.K) >> 5;
        word[m] = in ? __ldg(mv.tv.occ + q) : 0u;
        rbase[m] = in ? __ldg(mv.tv.rank + q) : 0u;
    }
    C<T> v[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 8; ++m) v[c][m] = mk<T>(0, 0);
#pragma unroll
    for (int m = 0; m < nh; ++m) {
        const int n = t + m * TL;
        const uint32_t bit = (uint32_t)((s0 + (int64_t)n * g.K) & 31);
        if ((word[m] >> bit) & 1u) {
            const int64_t r = rbase[m] + __popc(word[m] & ((1u << bit) - 1u));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[c][m] = from_io<T>(pb[c * g.nd + r]);
                if (mv.conj) v[c][m].y = -v[c][m].y;
            }
        }
    }
    if (mv.jac) {   // point-Jacobi: the product starts from S p
#pragma unroll
        for (int m = 0; m < nh; ++m) {
            const int n = t + m * TL;
            if (inx && n < g.J)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    v[c][m] = cmul<T>(v[c][m], mv.jac[material(mv.tv, s0 + (int64_t)n * g.K, c) * 3 + c]);
        }
    }
    fft_lines<T, false, N, 3, true, false, false>(v, sm, region, ColLayoutT<LOGW>{}, w, t, mv.tw);
    if (inx) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C<T>* out = mv.Ay + j * ay_elems(g) + ((int64_t)c * g.P + kz) * ((int64_t)g.K * N) + i;
#pragma unroll
            for (int m = 0; m < nv; ++m) out[(int64_t)(t + m * TL) * g.K] = v[c][m];
        }
    }
}

// ------------------------------------------------------- P2 / P4 (rows)
// One tile takes the x lines of Wz = 2^LOGZ consecutive z planes at one
// (component, y row): rows of K inputs in Ay (x fastest) and the same x
// positions of Wz consecutive z in the columns of Bxy (z fastest).  Threads
// run w-fastest (w = z offset, t = point slot), so each load or store of
// the column side touches Wz consecutive z values of one x (32 bytes and
// more), and the row side whole 32-byte sectors of Wz rows.  A CTA holds
// rows_groups(N, Wz, c128) tiles of consecutive z (more than one only for the
// wide mappings, whose few threads per line would otherwise make CTAs of a
// warp or less), each with its own region of shared memory.
// Forward (P2): Ay rows -> transform -> Bxy.  Inverse (P4): Bxy ->
// transform -> the first K outputs into Ay.  Grid: (z tiles, Ly, 3 nb).
__host__ __device__ constexpr int rows_groups(int N, int Wz, bool c128) {
    return map_wide(N, c128) && Wz * map_threads(N, c128) < 128 ? 128 / (Wz * map_threads(N, c128)) : 1;
}

// elements of one P2/P4 tile of Wz rows: the 8-point mapping's tile, or for
// a wide mapping one with the pad its exchanges use (after every V points
// for 2^a rows, every 8 for 3 * 2^a and 5 * 2^a rows)
__host__ __device__ constexpr int rows_tile_elems(int N, int Wz, bool c128) {
    return !map_wide(N, c128) ? col_elems(N, Wz) : col_elems_sh(N, Wz, wide_len(N) ? 3 : log2c(wide_points(N)));
}

template <typename T, bool INV, int N, int LOGZ>
__global__ void __launch_bounds__(rows_max_threads(N, sizeof(T) == 8)) k_rows(MatvecView<T> mv) {
    const int c = blockIdx.z % 3, j = blockIdx.z / 3;      // component, batch slot
    if (rhs_done(mv, mv.b0 + j)) return;
    extern __shared__ unsigned char smem_raw[];
    using MP = Map<T, N>;
    constexpr int TL = MP::T_, V = MP::V, nv = MP::NV, nh = MP::NH, Wz = 1 << LOGZ;
    constexpr int G = rows_groups(N, Wz, sizeof(T) == 8);
    const Geometry& g = mv.g;
    const int w = threadIdx.x & (Wz - 1), t = (threadIdx.x >> LOGZ) % TL, gi = (threadIdx.x >> LOGZ) / TL;
    C<T>* sm = reinterpret_cast<C<T>*>(smem_raw) + gi * rows_tile_elems(N, Wz, sizeof(T) == 8);
    const int y = blockIdx.y, z = (blockIdx.x * G + gi) * Wz + w;
    const bool ok = z < g.P;
    C<T>* row = mv.Ay + j * ay_elems(g) + ((c * g.P + (ok ? z : 0)) * g.Ly + y) * g.K;
    C<T>* col = mv.Bxy + j * bxy_elems(g) + (c * g.Ly + y) * g.Lx * g.Pb + (ok ? z : 0);
    C<T> v[V];
    if (!INV) {
#pragma unroll
        for (int m = 0; m < V; ++m) {
            const int n = t + m * TL;
            v[m] = (ok && m < nh && n < g.K) ? row[n] : mk<T>(0, 0);
        }
        fft_line<T, false, N, true, false, false>(v, sm, ColLayoutT<LOGZ>{}, w, t, mv.tw);
        if (ok) {
#pragma unroll
            for (int m = 0; m < nv; ++m) col[(t + m * TL) * g.Pb] = v[m];
        }
    } else {
#pragma unroll
        for (int m = 0; m < V; ++m) v[m] = (ok && m < nv) ? col[(t + m * TL) * g.Pb] : mk<T>(0, 0);
        fft_line<T, true, N, false, true, false>(v, sm, ColLayoutT<LOGZ>{}, w, t, mv.tw);
        if (ok) {
#pragma unroll
            for (int m = 0; m < nh; ++m) {   // i < K <= N/2: first half only
                const int n = t + m * TL;
                if (n < g.K) row[n] = v[m];
            }
        }
    }
}

// ---------------------------------------------------------------- P3
// Signs of the mirrored half for component m (xx, xy, xz, yy, yz, zz):
// Table 1 per axis, multiplied over the mirrored axes.
__device__ __forceinline__ int mirror_flip(int m, int fx, int fy, int fz) {
    switch (m) {
        case 1: return fx ^ fy;   // xy
        case 2: return fx ^ fz;   // xz
        case 4: return fy ^ fz;   // yz
        default: return 0;        // xx, yy, zz
    }
}

// the six spectrum components of one point (contiguous) with 16-byte loads
template <typename T>
__device__ __forceinline__ void load6(const C<T>* __restrict__ p, C<T> (&Y)[6]) {
    if (sizeof(T) == 4) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float4 f = __ldg(q + i);
            Y[2 * i] = mk<T>(f.x, f.y);
            Y[2 * i + 1] = mk<T>(f.z, f.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) Y[i] = ldg_c<T>(p + i);
    }
}

// row jy of the b-th row of CTAs: rows jy and Ly - jy read the same spectrum
// lines (mirror lookup), so they are visited back to back (0, 1, Ly-1, 2,
// Ly-2, ...) and the second read hits L2
__device__ __forceinline__ int p3_row(int b, int Ly) {
    const int q2 = (b + 1) >> 1;
    return b == 0 ? 0 : ((b & 1) ? q2 : Ly - q2);
}

// the spectrum product of Eqs. 6-8 at z point n of a column whose mirrored
// spectrum line (contiguous in z) starts at line (flips fx, fy of the x and
// y mirrors): one 48-byte load of the six components, the Table-1 signs,
// then (X0, X1, X2) <- Y (X0, X1, X2)
template <typename T, int N>
__device__ __forceinline__ void p3_product(const C<T>* __restrict__ line, bool ok, int fx, int fy, int n, C<T>& X0,
                                           C<T>& X1, C<T>& X2) {
    const int mz = n <= N / 2 ? n : N - n, fz = n > N / 2;
    C<T> Y[6];
    if (ok) {
        load6<T>(line + mz * 6, Y);
    } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) Y[q] = mk<T>(0, 0);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
        if (mirror_flip(q, fx, fy, fz)) { Y[q].x = -Y[q].x; Y[q].y = -Y[q].y; }
    const C<T> a = X0, b = X1, c = X2;
    X0 = cfma<T>(Y[2], c, cfma<T>(Y[1], b, cmul<T>(Y[0], a)));
    X1 = cfma<T>(Y[4], c, cfma<T>(Y[3], b, cmul<T>(Y[1], a)));
    X2 = cfma<T>(Y[5], c, cfma<T>(Y[4], b, cmul<T>(Y[2], a)));
}

// Line c of three held in registers, copied out and back with selects on the
// (CTA-uniform) index c, so that a loop over the lines needs no dynamically
// indexed register array.
template <typename T>
__device__ __forceinline__ void take_line(const C<T> (&v)[3][8], int c, C<T> (&u)[1][8]) {
#pragma unroll
    for (int m = 0; m < 8; ++m) u[0][m] = c == 0 ? v[0][m] : (c == 1 ? v[1][m] : v[2][m]);
}
template <typename T>
__device__ __forceinline__ void put_line(C<T> (&v)[3][8], int c, const C<T> (&u)[1][8]) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        if (c == 0) v[0][m] = u[0][m];
        else if (c == 1) v[1][m] = u[0][m];
        else v[2][m] = u[0][m];
    }
}

// R = 2^logW_z whole columns (x = xg R + w, row jy, batch slot j) per CTA,
// T = N/8 threads per column (thread t holds the points t + T m of the
// three components): z-forward DFTs of the P nonzero inputs, the spectrum
// product of Eqs. 6-8 with the signed mirror lookup of Sec. 3, z-inverse
// DFTs, and the store of k < P.  Grid: (nb, Lx / R, Ly).
template <typename T, int N>
__global__ void __launch_bounds__(p3_max_threads<T>(N)) k_p3(MatvecView<T> mv) {
    const int j = blockIdx.x;                                   // batch slot
    if (rhs_done(mv, mv.b0 + j)) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
    constexpr int TL = Line<N>::T, nv = Line<N>::NV;
    const Geometry& g = mv.g;
    const int t = threadIdx.x % TL, w = threadIdx.x / TL;
    const int ix = (blockIdx.y << mv.logW_z) + w, jy = p3_row(blockIdx.z, g.Ly);
    const bool ok = ix < g.Lx;
    const int comp = g.Ly * g.Lx * g.Pb;                        // stride between components
    C<T>* col = mv.Bxy + j * bxy_elems(g) + (jy * g.Lx + (ok ? ix : 0)) * g.Pb;
    C<T> v[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int n = t + m * TL;
            v[c][m] = (ok && m < Line<N>::NH && n < g.P) ? col[c * comp + n] : mk<T>(0, 0);
        }
    const int region = row_ld(N, TL) << mv.logW_z;
    if constexpr (sizeof(T) == 8 && !std::is_same<T, double>::value) {
        // double-float: one component at a time, in a loop that is not
        // unrolled, so that the kernel holds one line's transform instead of
        // three (unrolled, its instruction fetch limited it, not arithmetic)
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            C<T> u[1][8];
            take_line<T>(v, c, u);
            fft_lines<T, false, N, 1, true, false>(u, sm, region, RowLayout<N, TL>{}, w, t, mv.tw);
            put_line<T>(v, c, u);
        }
    } else {
        fft_lines<T, false, N, 3, true, false>(v, sm, region, RowLayout<N, TL>{}, w, t, mv.tw);
    }
    {
        const int my = jy <= g.Ly / 2 ? jy : g.Ly - jy, fy = jy > g.Ly / 2;
        const int mx = ix <= g.Lx / 2 ? ix : g.Lx - ix, fx = ix > g.Lx / 2;
        const C<T>* line = mv.spec + ((my * g.Hx + (ok ? mx : 0)) * g.Hz) * 6;
#pragma unroll
        for (int m = 0; m < nv; ++m)
            p3_product<T, N>(line, ok, fx, fy, t + m * TL, v[0][m], v[1][m], v[2][m]);
    }
    if constexpr (sizeof(T) == 8 && !std::is_same<T, double>::value) {
        // each transform but the last ends with a barrier after its last
        // shared-memory read, before the next one writes the buffer
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            C<T> u[1][8];
            take_line<T>(v, c, u);
            fft_lines<T, true, N, 1, false, true, true>(u, sm, region, RowLayout<N, TL>{}, w, t, mv.tw);
            put_line<T>(v, c, u);
        }
    } else {
        // nothing reuses the exchange buffers after the inverse
        fft_lines<T, true, N, 3, false, true, false>(v, sm, region, RowLayout<N, TL>{}, w, t, mv.tw);
    }
    if (ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < Line<N>::NH; ++m) {   // z < P <= N/2: first half only
                const int n = t + m * TL;
                if (n < g.P) col[c * comp + n] = v[c][m];
            }
    }
}

// The wide mapping of P3 (N = 3 * 2^a, 5 * 2^a): each component of a column
// is a line of T = M/8 threads of 8R points, so a CTA of R columns has
// 3 T R threads (line l = c + 3 w, thread t).  After the forward DFTs every
// line publishes its spectrum X_c in shared memory.  For the product the
// 3 T threads of a column take the mirror pairs (mz, N - mz), mz <= N/2,
// which share the spectrum entries of Eqs. 6-8: thread u reads the six
// components at mz once (six coalesced loads from the column's [6][Hz]
// lines), forms y = G X at both points and writes y back in place.  Table
// 1's sign of the (c, d) component under the mirror flips is f_c f_d, with
// f = -1 on a mirrored axis, so y_c = f_c sum_d G_cd (f_d X_d).  Then every
// thread reads its own line back, does the inverse DFT and stores k < P.
// Grid: (nb, Lx / R, Ly).
// (complex64: at most 128 registers, five 96-thread CTAs per SM, which
// measured fastest among 128, 136, 144, 160 and no cap)
template <typename T, int N>
__global__ void __launch_bounds__(p3_max_threads<T>(N)) __maxnreg__(sizeof(T) == 4 ? 128 : 255) k_p3w(MatvecView<T> mv) {
    static_assert(Line<N>::ODD, "k_p3w takes 3 * 2^a and 5 * 2^a columns (their spectrum lines are [6][Hz])");
    const int j = blockIdx.x;                                   // batch slot
    if (rhs_done(mv, mv.b0 + j)) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
    constexpr int TL = Wide<N>::T, V = Wide<N>::V, nh = V / 2;
    constexpr int KP = 10;                                      // key of the product exchange (no pad)
    const Geometry& g = mv.g;
    const int t = threadIdx.x % TL, l = threadIdx.x / TL;      // thread, line of the CTA
    const int c = l % 3, w = l / 3;                             // component, column of the CTA
    const int ix = (blockIdx.y << mv.logW_z) + w, jy = p3_row(blockIdx.z, g.Ly);
    const bool ok = ix < g.Lx;
    C<T>* col = mv.Bxy + j * bxy_elems(g) + c * (g.Ly * g.Lx * g.Pb) + (jy * g.Lx + (ok ? ix : 0)) * g.Pb;
    C<T> v[V];
#pragma unroll
    for (int m = 0; m < V; ++m) {
        const int n = t + m * TL;
        v[m] = (ok && m < nh && n < g.P) ? col[n] : mk<T>(0, 0);
    }
    const RowLayout<N, TL> L;
    fft_wide<T, false, N, true>(v, sm, L, l, t, mv.tw);
#pragma unroll
    for (int m = 0; m < V; ++m) sm[L.template at<KP>(l, t + m * TL)] = v[m];
    L.sync();
    {
        const int my = jy <= g.Ly / 2 ? jy : g.Ly - jy, fy = jy > g.Ly / 2;
        const int mx = ix <= g.Lx / 2 ? ix : g.Lx - ix, fx = ix > g.Lx / 2;
        const C<T>* line = mv.spec + ((my * g.Hx + (ok ? mx : 0)) * 6) * g.Hz;   // [6][Hz]
        const int u = c * TL + t;                               // thread of the column
        constexpr int NU = 3 * TL, NMZ = (N / 2 + NU) / NU;     // mz per thread (at most)
#pragma unroll
        for (int i = 0; i < NMZ; ++i) {
            const int mz = u + i * NU;
            if (mz > N / 2) break;
            C<T> G[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) G[q] = ok ? ldg_c<T>(line + q * g.Hz + mz) : mk<T>(0, 0);
            // the point mz (z not mirrored) and, unless mz is 0 or N/2, its
            // mirror N - mz (z mirrored)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && (mz == 0 || mz == N / 2)) break;
                const int n = h ? N - mz : mz, fz = h;
                const int o0 = L.template at<KP>(3 * w, n), o1 = L.template at<KP>(3 * w + 1, n),
                          o2 = L.template at<KP>(3 * w + 2, n);
                C<T> a = sm[o0], b = sm[o1], d = sm[o2];
                if (fx) a = mk<T>(-a.x, -a.y);
                if (fy) b = mk<T>(-b.x, -b.y);
                if (fz) d = mk<T>(-d.x, -d.y);
                C<T> y0 = cfma<T>(G[2], d, cfma<T>(G[1], b, cmul<T>(G[0], a)));
                C<T> y1 = cfma<T>(G[4], d, cfma<T>(G[3], b, cmul<T>(G[1], a)));
                C<T> y2 = cfma<T>(G[5], d, cfma<T>(G[4], b, cmul<T>(G[2], a)));
                if (fx) y0 = mk<T>(-y0.x, -y0.y);
                if (fy) y1 = mk<T>(-y1.x, -y1.y);
                if (fz) y2 = mk<T>(-y2.x, -y2.y);
                sm[o0] = y0;
                sm[o1] = y1;
                sm[o2] = y2;
            }
        }
    }
    L.sync();
#pragma unroll
    for (int m = 0; m < V; ++m) v[m] = sm[L.template at<KP>(l, t + m * TL)];
    L.sync();   // the inverse's first exchange writes the buffer
    // nothing reuses the exchange buffers after the inverse
    fft_wide<T, true, N, false, false>(v, sm, L, l, t, mv.tw);
    if (ok) {
#pragma unroll
        for (int m = 0; m < nh; ++m) {   // z < P <= N/2: first half only
            const int n = t + m * TL;
            if (n < g.P) col[n] = v[m];
        }
    }
}

// ---------------------------------------------------------------- P5
template <typename T, int N, int LOGW>
__global__ void __launch_bounds__(kYThreads, sizeof(T) == 4 ? 2 : 1) k_p5(MatvecView<T> mv, const C<IO<T>>* __restrict__ p, C<IO<T>>* __restrict__ y) {
    const int c = blockIdx.z % 3, j = blockIdx.z / 3;      // component, batch slot
    const int b = mv.b0 + j;
    if (rhs_done(mv, b)) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
    constexpr int TL = Line<N>::T, nv = Line<N>::NV;
    const Geometry& g = mv.g;
    constexpr int logW = LOGW, W = 1 << LOGW;
    const int w = threadIdx.x & (W - 1), t = threadIdx.x >> logW;
    const int i = blockIdx.x * W + w, kz = blockIdx.y;
    const bool ok = i < g.K;
    const C<T>* in = mv.Ay + j * ay_elems(g) + ((int64_t)c * g.P + kz) * ((int64_t)g.K * N) + (ok ? i : 0);
    C<T> v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int n = t + m * TL;
        v[m] = (ok && m < nv) ? in[(int64_t)n * g.K] : mk<T>(0, 0);
    }
    // the gather of the thread's sites (first half of the points, J <= N/2)
    // goes out before the transform, which does not depend on it: occupancy
    // and rank words, then the occupied entries of p
    const C<IO<T>>* pc = p + (int64_t)b * mv.vstride + (int64_t)c * g.nd;
    C<IO<T>>* yc = y + (int64_t)b * mv.vstride + (int64_t)c * g.nd;
    const int64_t s0 = (int64_t)kz * g.J * g.K + i;
    constexpr int nh = Line<N>::NH;
    uint32_t word[nh], rbase[nh];
#pragma unroll
    for (int m = 0; m < nh; ++m) {
        const int n = t + m * TL;
        const bool in = ok && n < g.J;
        const int64_t q = (s0 + (int64_t)n * g.K) >> 5;
        word[m] = in ? __ldg(mv.tv.occ + q) : 0u;
        rbase[m] = in ? __ldg(mv.tv.rank + q) : 0u;
    }
    C<IO<T>> pv[nh];
#pragma unroll
    for (int m = 0; m < nh; ++m) {
        const int n = t + m * TL;
        const uint32_t bit = (uint32_t)((s0 + (int64_t)n * g.K) & 31);
        rbase[m] += __popc(word[m] & ((1u << bit) - 1u));   // the site's rank
        word[m] = (word[m] >> bit) & 1u;                    // occupied?
        if (word[m]) pv[m] = pc[rbase[m]];
    }
    fft_regs<T, true, N, false, true, false>(v, sm, ColLayoutT<LOGW>{}, w, t, mv.tw);
    if (!ok) return;
#pragma unroll
    for (int m = 0; m < nh; ++m) {
        if (!word[m]) continue;
        const int64_t s = s0 + (int64_t)(t + m * TL) * g.K;
        const int mat = material(mv.tv, s, c);
        const C<T> a = mv.ainv[mat * 3 + c];
        C<T> q = from_io<T>(pv[m]);
        if (mv.conj) q.y = -q.y;
        C<T> out;
        if (mv.jac) {   // point-Jacobi: S (alpha^-1 S p + conv)
            const C<T> f = mv.jac[mat * 3 + c];
            out = cmul<T>(f, cfma<T>(a, cmul<T>(f, q), v[m]));
        } else {
            out = cfma<T>(a, q, v[m]);
        }
        if (mv.conj) out.y = -out.y;
        yc[rbase[m]] = to_io<T>(out);
    }
}

// largest power of two <= n (n >= 1), as its log
inline int floor_log2(int n) { int l = 0; while ((2 << l) <= n) ++l; return l; }

// Raises a kernel's dynamic shared-memory limit once per kernel and size
// (`done` is the launcher's own record), so that launches recorded into a
// CUDA graph make no attribute calls.
inline int set_smem(const void* fn, size_t bytes, std::atomic<size_t>& done) {
    if (bytes <= 48 * 1024 || bytes <= done.load(std::memory_order_relaxed)) return 0;
    DDA_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    size_t cur = done.load(std::memory_order_relaxed);
    while (cur < bytes && !done.compare_exchange_weak(cur, bytes)) {
    }
    return 0;
}

// ------------------------------------------------- per-length launchers
template <typename T, int N, int LOGW>
int launch_p1(const MatvecView<T>& mv, const C<IO<T>>* p, cudaStream_t st) {
    const Geometry& g = mv.g;
    constexpr int W = 1 << LOGW;
    const size_t sm = 3 * (size_t)col_elems(N, W) * sizeof(C<T>);
    static std::atomic<size_t> smem_set{0};
    if (int rc = set_smem((const void*)k_p1<T, N, LOGW>, sm, smem_set)) return rc;
    dim3 grid((g.K + W - 1) / W, g.P, mv.nb);
    k_p1<T, N, LOGW><<<grid, W * Line<N>::T, sm, st>>>(mv, p);
    DDA_LAUNCH_CHECK("P1 expand + y-forward");
    return 0;
}

// shared memory of a P2/P4 CTA of Wz rows
inline size_t rows_smem_elems(int N, int Wz, bool c128) { return (size_t)rows_groups(N, Wz, c128) * rows_tile_elems(N, Wz, c128); }

template <typename T, bool INV, int N, int LOGZ>
int launch_rows_w(const MatvecView<T>& mv, cudaStream_t st) {
    const Geometry& g = mv.g;
    constexpr bool c128 = sizeof(T) == 8;
    constexpr int Wz = 1 << LOGZ, G = rows_groups(N, Wz, c128), threads = G * Wz * Map<T, N>::T_;
    if constexpr (threads > rows_max_threads(N, c128)) {
        return fail(DDA_ERR_ARG, "x pass tile wider than a CTA");
    } else {
        const size_t sm = rows_smem_elems(N, Wz, c128) * sizeof(C<T>);
        static std::atomic<size_t> smem_set{0};
        if (int rc = set_smem((const void*)k_rows<T, INV, N, LOGZ>, sm, smem_set)) return rc;
        const dim3 grid((unsigned)((g.P + G * Wz - 1) / (G * Wz)), g.Ly, 3 * mv.nb);
        k_rows<T, INV, N, LOGZ><<<grid, threads, sm, st>>>(mv);
        DDA_LAUNCH_CHECK(INV ? "P4 x-inverse" : "P2 x-forward");
        return 0;
    }
}

template <typename T, bool INV, int N>
int launch_rows(const MatvecView<T>& mv, cudaStream_t st) {
    switch (mv.logW_x) {
        case 0: return launch_rows_w<T, INV, N, 0>(mv, st);
        case 1: return launch_rows_w<T, INV, N, 1>(mv, st);
        case 2: return launch_rows_w<T, INV, N, 2>(mv, st);
        case 3: return launch_rows_w<T, INV, N, 3>(mv, st);
        case 4: return launch_rows_w<T, INV, N, 4>(mv, st);
        default: return fail(DDA_ERR_ARG, "x pass tile width out of range");
    }
}

template <typename T, int N>
int launch_p3(const MatvecView<T>& mv, cudaStream_t st) {
    const Geometry& g = mv.g;
    const int R = 1 << mv.logW_z;
    const size_t sm = 3 * (size_t)R * row_ld(N, p3_line_threads(N)) * sizeof(C<T>);
    static std::atomic<size_t> smem_set{0};
    const dim3 grid(mv.nb, (g.Lx + R - 1) / R, g.Ly);
    if constexpr (Line<N>::ODD) {   // the wide z pass for 3 * 2^a and 5 * 2^a columns
        if (int rc = set_smem((const void*)k_p3w<T, N>, sm, smem_set)) return rc;
        k_p3w<T, N><<<grid, R * p3_col_threads(N), sm, st>>>(mv);
    } else {
        if (int rc = set_smem((const void*)k_p3<T, N>, sm, smem_set)) return rc;
        k_p3<T, N><<<grid, R * p3_col_threads(N), sm, st>>>(mv);
    }
    DDA_LAUNCH_CHECK("P3 z-forward, spectrum product, z-inverse");
    return 0;
}

template <typename T, int N, int LOGW>
int launch_p5(const MatvecView<T>& mv, const C<IO<T>>* p, C<IO<T>>* y, cudaStream_t st) {
    const Geometry& g = mv.g;
    constexpr int W = 1 << LOGW;
    const size_t sm = (size_t)col_elems(N, W) * sizeof(C<T>);
    static std::atomic<size_t> smem_set{0};
    if (int rc = set_smem((const void*)k_p5<T, N, LOGW>, sm, smem_set)) return rc;
    dim3 grid((g.K + W - 1) / W, g.P, 3 * mv.nb);
    k_p5<T, N, LOGW><<<grid, W * Line<N>::T, sm, st>>>(mv, p, y);
    DDA_LAUNCH_CHECK("P5 y-inverse + diagonal + compress");
    return 0;
}

// every line length the passes are compiled for: 2^a (a = 1..10), 3 * 2^a
// (a = 3..8) and 5 * 2^a (a = 3..7)
#define DDA_LEN_CASE(V, CALL) case V: { constexpr int LN = V; return CALL; }
#define DDA_LEN_SWITCH(len, CALL)                                                        \
    switch (len) {                                                                       \
        DDA_LEN_CASE(2, CALL) DDA_LEN_CASE(4, CALL) DDA_LEN_CASE(8, CALL)                \
        DDA_LEN_CASE(16, CALL) DDA_LEN_CASE(32, CALL) DDA_LEN_CASE(64, CALL)             \
        DDA_LEN_CASE(128, CALL) DDA_LEN_CASE(256, CALL) DDA_LEN_CASE(512, CALL)          \
        DDA_LEN_CASE(1024, CALL) DDA_LEN_CASE(24, CALL) DDA_LEN_CASE(48, CALL)           \
        DDA_LEN_CASE(96, CALL) DDA_LEN_CASE(192, CALL) DDA_LEN_CASE(384, CALL)           \
        DDA_LEN_CASE(768, CALL) DDA_LEN_CASE(40, CALL) DDA_LEN_CASE(80, CALL)            \
        DDA_LEN_CASE(160, CALL) DDA_LEN_CASE(320, CALL) DDA_LEN_CASE(640, CALL)          \
        default: return fail(DDA_ERR_ARG, "line length out of range");                   \
    }

#define DDA_LOGW_SWITCH(logW, CALL)                    \
    switch (logW) {                                    \
        case 0: { constexpr int LW = 0; return CALL; } \
        case 1: { constexpr int LW = 1; return CALL; } \
        case 2: { constexpr int LW = 2; return CALL; } \
        case 3: { constexpr int LW = 3; return CALL; } \
        case 4: { constexpr int LW = 4; return CALL; } \
        default: return fail(DDA_ERR_ARG, "tile width out of range"); \
    }

// widest tile (log2 lines per CTA) the strided passes are compiled for
constexpr int kMaxLogW = 4;

// per-pass dispatchers (one translation unit each)
template <typename T> int pass1(const MatvecView<T>& mv, const C<IO<T>>* p, cudaStream_t st);
template <typename T, bool INV> int pass_rows(const MatvecView<T>& mv, cudaStream_t st);
template <typename T> int pass3(const MatvecView<T>& mv, cudaStream_t st);
// P3 for one line length; each length group is instantiated in its own
// translation unit (mv_p3_*.cu)
template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st);
template <typename T> int pass5(const MatvecView<T>& mv, const C<IO<T>>* p, C<IO<T>>* y, cudaStream_t st);

}  // namespace dda
