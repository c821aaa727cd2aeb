// Kernels and per-length launchers of the pruned FFT matrix-vector product
// y = A p of the DDA (OpenDDA Sec. 3).  Each of the translation units
// mv_p1_*.cu, mv_p3_*.cu, mv_p5_*.cu and mv_rows.cu instantiates one pass for
// every line length (and tile width) and exposes its dispatcher; matvec.cu
// sequences the passes.
//
// Five stream-ordered passes over device arrays (x fastest everywhere):
//   P1  expand + y-forward   compressed p -> Ay[3][P][Ly][K]   (K*P lines per component;
//                            a thread gathers a site's three components together)
//   P2  x-forward            Ay -> Bxy[3][P][Ly][Lx]           (Ly*P lines, K nonzero inputs)
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
// Batches: one launch of each pass covers up to `slots` right-hand sides
// that share the context's spectrum (vectors [nb][3][N_d], work arrays one
// per slot); a right-hand side whose solver status is no longer "running"
// is skipped block by block.  The slot is a grid coordinate of its own (no
// index division in the kernels); in P3 it is the fastest-varying one, so
// the CTAs of all right-hand sides that read one spectrum tile run back to
// back and the tile is fetched from HBM once.
//
// Every pass keeps its lines in registers (fft_reg.cuh): points are loaded
// from global memory straight into the registers of the first DFT stage and
// stored from the registers of the last, and only the exchanges between
// stages use shared memory.  Strided lines (y, z) are processed W at a
// time, W adjacent columns so that each load and store touches W
// contiguous elements.  In P3 each thread carries the same column of all
// three components, so the spectrum product happens in registers between
// the forward and the inverse transforms; in P1 it gathers a site's three
// components with one occupancy and rank lookup.  Each kernel is compiled
// for every line length N (2^a up to 1024, 3 * 2^a from 24 to 768, 5 * 2^a
// from 40 to 640) and, for the strided passes, every tile width (LOGW =
// 0..4 lines per CTA, log2), and picked at launch, so all shared-memory
// addresses are compile-time offsets.
#pragma once

#include <algorithm>
#include <atomic>

#include "fft_reg.cuh"
#include "matvec.cuh"

namespace dda {


// P3 keeps 3 x 8 complex values per thread: 512 threads fit the register
// file for complex64, 256 for complex128
template <typename T> __host__ __device__ constexpr int p3_max_threads() { return sizeof(T) == 4 ? 512 : 256; }

// P1 and P5 keep the eight points, their gather indices and (P5) the
// gathered entries of p in registers: at most 512 threads per CTA leave
// room for them (the complex64 P5 is held to two such CTAs per SM, which
// measured faster than one with no register cap)
constexpr int kYThreads = 512;

// elements of one slot of the work arrays
__host__ __device__ __forceinline__ int64_t ay_elems(const Geometry& g) { return 3LL * g.P * g.Ly * g.K; }
__host__ __device__ __forceinline__ int64_t bxy_elems(const Geometry& g) { return 3LL * g.P * g.Ly * g.Lx; }

// ---------------------------------------------------------------- P1
template <typename T, int N, int LOGW>
__global__ void __launch_bounds__(kYThreads) k_p1(MatvecView<T> mv, const C<T>* __restrict__ p) {
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
    const C<T>* pb = p + (int64_t)b * mv.vstride;
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
                v[c][m] = pb[c * g.nd + r];
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
// Forward: rows of K inputs (Ay) -> Lx outputs (Bxy).  Inverse: rows of Lx
// inputs (Bxy) -> first K outputs (Ay).  2^logW_x rows per CTA.
template <typename T, bool INV, int N>
__global__ void __launch_bounds__(512) k_rows(MatvecView<T> mv) {
    const int j = blockIdx.y;                               // batch slot
    if (rhs_done(mv, mv.b0 + j)) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
    constexpr int TL = Line<N>::T, nv = Line<N>::NV;
    const Geometry& g = mv.g;
    const int t = threadIdx.x % TL, wl = threadIdx.x / TL;
    const int64_t nrows = 3LL * g.P * g.Ly;
    const int64_t row = ((int64_t)blockIdx.x << mv.logW_x) + wl;
    const bool ok = row < nrows;
    const int nin = INV ? N : g.K, nout = INV ? g.K : N;
    const C<T>* src = (INV ? mv.Bxy + j * bxy_elems(g) : mv.Ay + j * ay_elems(g)) + (ok ? row * (INV ? N : g.K) : 0);
    C<T>* dst = (INV ? mv.Ay + j * ay_elems(g) : mv.Bxy + j * bxy_elems(g)) + (ok ? row * (INV ? g.K : N) : 0);
    C<T> v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int n = t + m * TL;
        v[m] = (ok && m < nv && n < nin) ? src[n] : mk<T>(0, 0);
    }
    fft_regs<T, INV, N, !INV, INV, false>(v, sm, RowLayout<N>{}, wl, t, mv.tw);
    if (ok) {
#pragma unroll
        for (int m = 0; m < nv; ++m) {
            const int n = t + m * TL;
            if (n < nout) dst[n] = v[m];
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
        for (int i = 0; i < 6; ++i) Y[i] = __ldg(p + i);
    }
}

// row jy of the b-th tile row: rows jy and Ly - jy read the same spectrum
// rows (mirror lookup), so they are visited back to back (0, 1, Ly-1, 2,
// Ly-2, ...) and the second read hits L2
__device__ __forceinline__ int p3_row(int b, int Ly) {
    const int q2 = (b + 1) >> 1;
    return b == 0 ? 0 : ((b & 1) ? q2 : Ly - q2);
}

// the spectrum product of Eqs. 6-8 at z point n of the column whose mirrored
// spectrum row starts at spec (flips fx, fy of the x and y mirrors): one
// 48-byte load of the six components, the Table-1 signs, then
// (X0, X1, X2) <- Y (X0, X1, X2)
template <typename T, int N>
__device__ __forceinline__ void p3_product(const C<T>* __restrict__ spec, int64_t zstep, bool ok, int fx, int fy,
                                           int n, C<T>& X0, C<T>& X1, C<T>& X2) {
    const int mz = n <= N / 2 ? n : N - n, fz = n > N / 2;
    C<T> Y[6];
    if (ok) {
        load6<T>(spec + mz * zstep, Y);
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

// One tile of W columns (x = xt W + w, row jy, batch slot j) whose inputs v
// (the P nonzero z points of the three components, canonical order) are
// loaded: forward z DFTs, the spectrum product of Eqs. 6-8 with the signed
// mirror lookup of Sec. 3, inverse z DFTs, and the store of k < P.
template <typename T, int N, int LOGW>
__device__ __forceinline__ void p3_tile(const MatvecView<T>& mv, C<T>* sm, int j, int xt, int jy, C<T> (&v)[3][8]) {
    constexpr int TL = Line<N>::T, nv = Line<N>::NV;
    const Geometry& g = mv.g;
    constexpr int logW = LOGW, W = 1 << LOGW;
    const int w = threadIdx.x & (W - 1), t = threadIdx.x >> logW;
    const int ix = xt * W + w;
    const bool ok = ix < g.Lx;
    const ColLayoutT<LOGW> L{};
    constexpr int region = col_elems(N, W);
    const int64_t plane = (int64_t)g.Ly * g.Lx;   // stride between z planes of Bxy
    const int64_t comp = (int64_t)g.P * plane;    // stride between components
    C<T>* col = mv.Bxy + j * bxy_elems(g) + (int64_t)jy * g.Lx + (ok ? ix : 0);
    fft_lines<T, false, N, 3, true, false>(v, sm, region, L, w, t, mv.tw);
    {
        const int my = jy <= g.Ly / 2 ? jy : g.Ly - jy, fy = jy > g.Ly / 2;
        const int mx = ix <= g.Lx / 2 ? ix : g.Lx - ix, fx = ix > g.Lx / 2;
        const C<T>* spec = mv.spec + ((int64_t)my * g.Hx + (ok ? mx : 0)) * 6;
        const int64_t zstep = (int64_t)g.Hy * g.Hx * 6;
#pragma unroll
        for (int m = 0; m < nv; ++m)
            p3_product<T, N>(spec, zstep, ok, fx, fy, t + m * TL, v[0][m], v[1][m], v[2][m]);
    }
    // nothing reuses the exchange buffers after the inverse (the persistent
    // schedule synchronises twice before its next tile)
    fft_lines<T, true, N, 3, false, true, false>(v, sm, region, L, w, t, mv.tw);
    if (ok) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < Line<N>::NH; ++m) {   // z < P <= N/2: first half only
                const int n = t + m * TL;
                if (n < g.P) col[c * comp + n * plane] = v[c][m];
            }
    }
}

// one CTA per tile, inputs loaded from global memory
template <typename T, int N, int LOGW>
__global__ void __launch_bounds__(p3_max_threads<T>(), 1) k_p3(MatvecView<T> mv) {
    const int j = blockIdx.x, xt = blockIdx.y;                  // batch slot, column tile
    if (rhs_done(mv, mv.b0 + j)) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
    constexpr int TL = Line<N>::T, nv = Line<N>::NV;
    const Geometry& g = mv.g;
    constexpr int W = 1 << LOGW;
    const int w = threadIdx.x & (W - 1), t = threadIdx.x >> LOGW;
    const int jy = p3_row(blockIdx.z, g.Ly);
    const int ix = xt * W + w;
    const bool ok = ix < g.Lx;
    const int64_t plane = (int64_t)g.Ly * g.Lx, comp = (int64_t)g.P * plane;
    const C<T>* col = mv.Bxy + j * bxy_elems(g) + (int64_t)jy * g.Lx + (ok ? ix : 0);
    C<T> v[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int n = t + m * TL;
            v[c][m] = (ok && m < Line<N>::NH && n < g.P) ? col[c * comp + n * plane] : mk<T>(0, 0);
        }
    p3_tile<T, N, LOGW>(mv, sm, j, xt, jy, v);
}

// Persistent schedule: each CTA walks the tiles q = blockIdx.x, + gridDim.x,
// ... in the order of the per-tile grid (batch slot fastest, then column
// tile, then row), and while it transforms tile q the next one's input
// columns are already on their way into a shared-memory stage with cp.async
// (16-byte copies, no registers held), so the column loads of a tile no
// longer stall the SM.  Tiles must be whole (W <= Lx) and a stage row must
// be whole 16-byte copies (W * sizeof(C<T>) a multiple of 16).
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T, int N, int LOGW>
__global__ void __launch_bounds__(p3_max_threads<T>(), 1) k_p3p(MatvecView<T> mv, int stage_off) {
    extern __shared__ unsigned char smem_raw[];
    C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
    C<T>* stage = sm + stage_off;                                  // [3][P][W]
    constexpr int TL = Line<N>::T, nv = Line<N>::NV;
    const Geometry& g = mv.g;
    constexpr int W = 1 << LOGW;
    constexpr int per16 = 16 / (int)sizeof(C<T>), chunks = W / per16;   // 16-byte copies per stage row
    if constexpr (chunks == 0) {
        return;   // never launched: the host only picks this schedule for whole 16-byte stage rows
    } else {
    const int w = threadIdx.x & (W - 1), t = threadIdx.x >> LOGW;
    const int ntx = g.Lx / W;
    const int ntiles = mv.nb * ntx * g.Ly;
    const int64_t plane = (int64_t)g.Ly * g.Lx, comp = (int64_t)g.P * plane;
    const int rows = 3 * g.P;
    auto issue = [&](int q) {
        const int j = q % mv.nb, xt = (q / mv.nb) % ntx, jy = p3_row(q / (mv.nb * ntx), g.Ly);
        if (rhs_done(mv, mv.b0 + j)) return;
        const C<T>* base = mv.Bxy + j * bxy_elems(g) + (int64_t)jy * g.Lx + xt * W;
        for (int e = threadIdx.x; e < rows * chunks; e += blockDim.x) {
            const int row = e / chunks, ch = e - row * chunks;
            const int c = row / g.P, n = row - c * g.P;
            cp_async16(stage + row * W + ch * per16, base + c * comp + (int64_t)n * plane + ch * per16);
        }
    };
    int q = blockIdx.x;
    if (q < ntiles) issue(q);
    cp_async_commit();
    for (; q < ntiles; q += gridDim.x) {
        const int j = q % mv.nb, xt = (q / mv.nb) % ntx, jy = p3_row(q / (mv.nb * ntx), g.Ly);
        const bool skip = rhs_done(mv, mv.b0 + j);             // the same for the whole CTA
        cp_async_wait_all();
        __syncthreads();
        C<T> v[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int n = t + m * TL;
                v[c][m] = (!skip && m < nv && n < g.P) ? stage[(c * g.P + n) * W + w] : mk<T>(0, 0);
            }
        __syncthreads();                                         // the stage is free again
        if (q + (int)gridDim.x < ntiles) issue(q + gridDim.x);
        cp_async_commit();
        if (!skip) p3_tile<T, N, LOGW>(mv, sm, j, xt, jy, v);
    }
    cp_async_wait_all();
    }
}

// ---------------------------------------------------------------- P5
template <typename T, int N, int LOGW>
__global__ void __launch_bounds__(kYThreads, sizeof(T) == 4 ? 2 : 1) k_p5(MatvecView<T> mv, const C<T>* __restrict__ p, C<T>* __restrict__ y) {
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
    const C<T>* pc = p + (int64_t)b * mv.vstride + (int64_t)c * g.nd;
    C<T>* yc = y + (int64_t)b * mv.vstride + (int64_t)c * g.nd;
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
    C<T> pv[nh];
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
        C<T> q = pv[m];
        if (mv.conj) q.y = -q.y;
        C<T> out;
        if (mv.jac) {   // point-Jacobi: S (alpha^-1 S p + conv)
            const C<T> f = mv.jac[mat * 3 + c];
            out = cmul<T>(f, cfma<T>(a, cmul<T>(f, q), v[m]));
        } else {
            out = cfma<T>(a, q, v[m]);
        }
        if (mv.conj) out.y = -out.y;
        yc[rbase[m]] = out;
    }
}

// threads per line of N points
inline int threads_of(int N) { return N >= 8 ? N / 8 : 1; }

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
int launch_p1(const MatvecView<T>& mv, const C<T>* p, cudaStream_t st) {
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

template <typename T, bool INV, int N>
int launch_rows(const MatvecView<T>& mv, cudaStream_t st) {
    const Geometry& g = mv.g;
    const int64_t rows = 3LL * g.P * g.Ly;
    const int R = 1 << mv.logW_x;
    const size_t sm = (size_t)R * row_ld(N) * sizeof(C<T>);
    static std::atomic<size_t> smem_set{0};
    if (int rc = set_smem((const void*)k_rows<T, INV, N>, sm, smem_set)) return rc;
    const dim3 grid((unsigned)((rows + R - 1) / R), mv.nb);
    k_rows<T, INV, N><<<grid, R * Line<N>::T, sm, st>>>(mv);
    DDA_LAUNCH_CHECK(INV ? "P4 x-inverse" : "P2 x-forward");
    return 0;
}

// the persistent z pass applies: whole tiles, whole 16-byte stage copies,
// stage and exchange buffers within the shared-memory budget
template <typename T>
inline bool p3_persistent_ok(const Geometry& g, int logW) {
    const int W = 1 << logW;
    if (W > g.Lx || g.Lx % W || (W * (int)sizeof(C<T>)) % 16) return false;
    const size_t stage_off = (3 * (size_t)col_elems(g.Lz, W) + 1) & ~size_t(1);
    return (stage_off + 3ull * g.P * W) * sizeof(C<T>) <= 220 * 1024;
}

inline int sm_count() {
    static std::atomic<int> n{0};
    int v = n.load(std::memory_order_relaxed);
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        n.store(v, std::memory_order_relaxed);
    }
    return v;
}

template <typename T, int N, int LOGW>
int launch_p3(const MatvecView<T>& mv, cudaStream_t st) {
    const Geometry& g = mv.g;
    constexpr int W = 1 << LOGW;
    const int threads = W * Line<N>::T;
    if (mv.p3_sched == 1 && p3_persistent_ok<T>(g, LOGW)) {
        const int stage_off = (int)((3 * (size_t)col_elems(N, W) + 1) & ~size_t(1));
        const size_t sm = ((size_t)stage_off + 3ull * g.P * W) * sizeof(C<T>);
        static std::atomic<size_t> smem_set{0};
        if (int rc = set_smem((const void*)k_p3p<T, N, LOGW>, sm, smem_set)) return rc;
        static std::atomic<int> per_sm{0};
        int bps = per_sm.load(std::memory_order_relaxed);
        if (!bps) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_p3p<T, N, LOGW>, threads, sm) != cudaSuccess ||
                bps < 1)
                bps = 1;
            per_sm.store(bps, std::memory_order_relaxed);
        }
        const int64_t ntiles = (int64_t)mv.nb * (g.Lx / W) * g.Ly;
        const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sm_count() * bps);
        k_p3p<T, N, LOGW><<<grid, threads, sm, st>>>(mv, stage_off);
        DDA_LAUNCH_CHECK("P3 z-forward, spectrum product, z-inverse (persistent)");
        return 0;
    }
    const size_t sm = 3 * (size_t)col_elems(N, W) * sizeof(C<T>);
    static std::atomic<size_t> smem_set{0};
    if (int rc = set_smem((const void*)k_p3<T, N, LOGW>, sm, smem_set)) return rc;
    dim3 grid(mv.nb, (g.Lx + W - 1) / W, g.Ly);
    k_p3<T, N, LOGW><<<grid, threads, sm, st>>>(mv);
    DDA_LAUNCH_CHECK("P3 z-forward, spectrum product, z-inverse");
    return 0;
}

template <typename T, int N, int LOGW>
int launch_p5(const MatvecView<T>& mv, const C<T>* p, C<T>* y, cudaStream_t st) {
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
template <typename T> int pass1(const MatvecView<T>& mv, const C<T>* p, cudaStream_t st);
template <typename T, bool INV> int pass_rows(const MatvecView<T>& mv, cudaStream_t st);
template <typename T> int pass3(const MatvecView<T>& mv, cudaStream_t st);
// P3 for one line length (all tile widths); each length group is
// instantiated in its own translation unit (mv_p3_*.cu)
template <typename T, int N> int p3_len(const MatvecView<T>& mv, cudaStream_t st);
template <typename T> int pass5(const MatvecView<T>& mv, const C<T>* p, C<T>* y, cudaStream_t st);

}  // namespace dda
