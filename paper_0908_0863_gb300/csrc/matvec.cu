// The pruned FFT matrix-vector product y = A p of the DDA (OpenDDA Sec. 3).
//
// Five stream-ordered passes over device arrays (x fastest everywhere):
//   P1  expand + y-forward   compressed p -> Ay[3][P][Ly][K]   (K*P lines per component)
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
// spectrum.
#include "fft.cuh"
#include "matvec.cuh"

namespace dda {

namespace {

// ---------------------------------------------------------------- P1
template <typename T, int V>
__global__ void __launch_bounds__(512) k_expand_yfwd(MatvecView<T> mv, const C<T>* __restrict__ p) {
    extern __shared__ unsigned char smem_raw[];
    C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
    if (mv.status && *mv.status) return;
    const Geometry& g = mv.g;
    const int logW = mv.logW_y, W = 1 << logW, ld = W + 1;
    const int i0 = blockIdx.x * W, kz = blockIdx.y, c = blockIdx.z;
    const int logN = ilog2_dev(g.Ly), N = g.Ly;
    const C<T>* pc = p + (int64_t)c * g.nd;
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int n = e >> logW, w = e & (W - 1), i = i0 + w;
        C<T> val = mk<T>(0, 0);
        if (n < g.J && i < g.K) {
            const int64_t s = ((int64_t)kz * g.J + n) * g.K + i;
            if (occupied(mv.tv, s)) {
                val = pc[site_rank(mv.tv, s)];
                if (mv.conj) val.y = -val.y;
            }
        }
        buf[n * ld + w] = val;
    }
    __syncthreads();
    fft_tile<T, V, false>(buf, ld, logW, logN, mv.tw);
    C<T>* out = mv.Ay + ((int64_t)c * g.P + kz) * N * g.K;
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int n = e >> logW, w = e & (W - 1), i = i0 + w;
        if (i < g.K) out[(int64_t)n * g.K + i] = buf[n * ld + w];
    }
}

// ------------------------------------------------------- P2 / P4 (rows)
// Transforms W rows of length Lx.  Forward: rows of K inputs (Ay) -> Lx
// outputs (Bxy).  Inverse: rows of Lx inputs (Bxy) -> first K outputs (Ay).
template <typename T, int V, bool INV>
__global__ void __launch_bounds__(512) k_xrows(MatvecView<T> mv) {
    if (mv.status && *mv.status) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
    const Geometry& g = mv.g;
    const int logW = mv.logW_x, W = 1 << logW, ld = W + 1;
    const int N = g.Lx, logN = ilog2_dev(N);
    const int64_t nrows = 3LL * g.P * g.Ly;
    const int64_t r0 = (int64_t)blockIdx.x * W;
    const int nin = INV ? N : g.K;
    const C<T>* src = INV ? mv.Bxy : mv.Ay;
    C<T>* dst = INV ? mv.Ay : mv.Bxy;
    const int ldin = INV ? N : g.K, ldout = INV ? g.K : N;
    const int nout = INV ? g.K : N;
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int w = e >> logN, n = e & (N - 1);
        const int64_t row = r0 + w;
        C<T> val = mk<T>(0, 0);
        if (n < nin && row < nrows) val = src[row * ldin + n];
        buf[n * ld + w] = val;
    }
    __syncthreads();
    fft_tile<T, V, INV>(buf, ld, logW, logN, mv.tw);
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int w = e >> logN, n = e & (N - 1);
        const int64_t row = r0 + w;
        if (n < nout && row < nrows) dst[row * ldout + n] = buf[n * ld + w];
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

template <typename T, int V>
__global__ void __launch_bounds__(512) k_zconv(MatvecView<T> mv) {
    if (mv.status && *mv.status) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
    const Geometry& g = mv.g;
    const int logW = mv.logW_z, W = 1 << logW, ld = W + 1;
    const int N = g.Lz, logN = ilog2_dev(N);
    const int ix0 = blockIdx.x * W, jy = blockIdx.y;
    const int64_t plane = (int64_t)g.Ly * g.Lx;   // stride between z planes of Bxy
    const int64_t comp = (int64_t)g.P * plane;    // stride between components
    const int64_t base = (int64_t)jy * g.Lx + ix0;
    const int cstride = N * ld;
    for (int c = 0; c < 3; ++c) {
        for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
            const int n = e >> logW, w = e & (W - 1);
            C<T> val = mk<T>(0, 0);
            if (n < g.P && ix0 + w < g.Lx) val = mv.Bxy[c * comp + n * plane + base + w];
            buf[c * cstride + n * ld + w] = val;
        }
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) fft_tile<T, V, false>(buf + c * cstride, ld, logW, logN, mv.tw);
    // spectrum product (Eqs. 6-8) with the mirror lookup of Sec. 3
    const int my = jy <= g.Ly / 2 ? jy : g.Ly - jy;
    const int fy = jy > g.Ly / 2;
    const int64_t sm = (int64_t)g.Hz * g.Hy * g.Hx;
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int n = e >> logW, w = e & (W - 1);
        const int ix = ix0 + w;
        if (ix >= g.Lx) continue;
        const int mx = ix <= g.Lx / 2 ? ix : g.Lx - ix, fx = ix > g.Lx / 2;
        const int mz = n <= N / 2 ? n : N - n, fz = n > N / 2;
        const C<T>* S = mv.spec + ((int64_t)mz * g.Hy + my) * g.Hx + mx;
        C<T> Y[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            C<T> t = S[m * sm];
            if (mirror_flip(m, fx, fy, fz)) { t.x = -t.x; t.y = -t.y; }
            Y[m] = t;
        }
        const int o = n * ld + w;
        const C<T> X0 = buf[o], X1 = buf[cstride + o], X2 = buf[2 * cstride + o];
        buf[o] = cfma<T>(Y[2], X2, cfma<T>(Y[1], X1, cmul<T>(Y[0], X0)));
        buf[cstride + o] = cfma<T>(Y[4], X2, cfma<T>(Y[3], X1, cmul<T>(Y[1], X0)));
        buf[2 * cstride + o] = cfma<T>(Y[5], X2, cfma<T>(Y[4], X1, cmul<T>(Y[2], X0)));
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) fft_tile<T, V, true>(buf + c * cstride, ld, logW, logN, mv.tw);
    for (int c = 0; c < 3; ++c) {
        for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
            const int n = e >> logW, w = e & (W - 1);
            if (n < g.P && ix0 + w < g.Lx) mv.Bxy[c * comp + n * plane + base + w] = buf[c * cstride + n * ld + w];
        }
    }
}

// ---------------------------------------------------------------- P5
template <typename T, int V>
__global__ void __launch_bounds__(512) k_yinv_compress(MatvecView<T> mv, const C<T>* __restrict__ p,
                                                       C<T>* __restrict__ y) {
    if (mv.status && *mv.status) return;
    extern __shared__ unsigned char smem_raw[];
    C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
    const Geometry& g = mv.g;
    const int logW = mv.logW_y, W = 1 << logW, ld = W + 1;
    const int i0 = blockIdx.x * W, kz = blockIdx.y, c = blockIdx.z;
    const int N = g.Ly, logN = ilog2_dev(N);
    const C<T>* in = mv.Ay + ((int64_t)c * g.P + kz) * N * g.K;
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int n = e >> logW, w = e & (W - 1), i = i0 + w;
        buf[n * ld + w] = i < g.K ? in[(int64_t)n * g.K + i] : mk<T>(0, 0);
    }
    __syncthreads();
    fft_tile<T, V, true>(buf, ld, logW, logN, mv.tw);
    const C<T>* pc = p + (int64_t)c * g.nd;
    C<T>* yc = y + (int64_t)c * g.nd;
    for (int e = threadIdx.x; e < W * g.J; e += blockDim.x) {
        const int n = e >> logW, w = e & (W - 1), i = i0 + w;
        if (i >= g.K) continue;
        const int64_t s = ((int64_t)kz * g.J + n) * g.K + i;
        if (!occupied(mv.tv, s)) continue;
        const uint32_t r = site_rank(mv.tv, s);
        const C<T> a = mv.ainv[material(mv.tv, s, c) * 3 + c];
        C<T> pv = pc[r];
        if (mv.conj) pv.y = -pv.y;
        C<T> out = cfma<T>(a, pv, buf[n * ld + w]);
        if (mv.conj) out.y = -out.y;
        yc[r] = out;
    }
}

template <typename T> constexpr int vals_per_thread() { return sizeof(T) == 4 ? 16 : 8; }

// pick W (a power of two) for a tile of lines of length N: as wide as the
// row budget allows while the launch stays within 512 threads
inline int pick_logW(int N, int V, int want_bytes, int elt, int ncols) {
    int logW = 0;
    while ((1 << logW) * elt < want_bytes && (2 << logW) * N / V <= 512) ++logW;
    while (logW > 0 && (1 << (logW - 1)) >= ncols) --logW;   // no wider than the data
    while ((1 << logW) * N < V) ++logW;                       // at least one full thread
    return logW;
}

}  // namespace

template <typename T>
void configure_matvec(MatvecView<T>& mv) {
    constexpr int V = vals_per_thread<T>();
    const int elt = sizeof(C<T>);
    mv.logW_y = pick_logW(mv.g.Ly, V, 128, elt, mv.g.K);
    mv.logW_x = pick_logW(mv.g.Lx, V, 128, elt, 1 << 30);
    mv.logW_z = pick_logW(mv.g.Lz, V, 64, elt, mv.g.Lx);
    // the z tile holds three components: keep it within the shared-memory budget
    while (mv.logW_z > 0 && 3 * (size_t)mv.g.Lz * ((1 << mv.logW_z) + 1) * elt > 200 * 1024) --mv.logW_z;
    while (((1 << mv.logW_z) * mv.g.Lz) < V) ++mv.logW_z;
}

template <typename T>
static int set_smem(const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) {
        DDA_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    }
    return 0;
}

template <typename T>
int launch_matvec(const MatvecView<T>& mv, const C<T>* p, C<T>* y, cudaStream_t st) {
    constexpr int V = vals_per_thread<T>();
    const Geometry& g = mv.g;
    const int elt = sizeof(C<T>);
    const int dt = sizeof(T) == 8 ? 0 : 1;
    PassProfiler* pf = (mv.prof && mv.prof->on) ? mv.prof : nullptr;
    int rc;
    {   // P1
        const int W = 1 << mv.logW_y;
        const size_t sm = (size_t)g.Ly * (W + 1) * elt;
        if ((rc = set_smem<T>((const void*)k_expand_yfwd<T, V>, sm))) return rc;
        dim3 grid((g.K + W - 1) / W, g.P, 3);
        if (pf) pf->begin(dt, 0, st);
        k_expand_yfwd<T, V><<<grid, W * g.Ly / V, sm, st>>>(mv, p);
        DDA_LAUNCH_CHECK("P1 expand + y-forward");
        if (pf) pf->end(st);
    }
    {   // P2
        const int W = 1 << mv.logW_x;
        const size_t sm = (size_t)g.Lx * (W + 1) * elt;
        if ((rc = set_smem<T>((const void*)k_xrows<T, V, false>, sm))) return rc;
        const int64_t rows = 3LL * g.P * g.Ly;
        if (pf) pf->begin(dt, 1, st);
        k_xrows<T, V, false><<<(unsigned)((rows + W - 1) / W), W * g.Lx / V, sm, st>>>(mv);
        DDA_LAUNCH_CHECK("P2 x-forward");
        if (pf) pf->end(st);
    }
    {   // P3
        const int W = 1 << mv.logW_z;
        const size_t sm = 3 * (size_t)g.Lz * (W + 1) * elt;
        if ((rc = set_smem<T>((const void*)k_zconv<T, V>, sm))) return rc;
        dim3 grid(g.Lx / W > 0 ? g.Lx / W : 1, g.Ly);
        if (pf) pf->begin(dt, 2, st);
        k_zconv<T, V><<<grid, W * g.Lz / V, sm, st>>>(mv);
        DDA_LAUNCH_CHECK("P3 z-forward, spectrum product, z-inverse");
        if (pf) pf->end(st);
    }
    {   // P4
        const int W = 1 << mv.logW_x;
        const size_t sm = (size_t)g.Lx * (W + 1) * elt;
        if ((rc = set_smem<T>((const void*)k_xrows<T, V, true>, sm))) return rc;
        const int64_t rows = 3LL * g.P * g.Ly;
        if (pf) pf->begin(dt, 3, st);
        k_xrows<T, V, true><<<(unsigned)((rows + W - 1) / W), W * g.Lx / V, sm, st>>>(mv);
        DDA_LAUNCH_CHECK("P4 x-inverse");
        if (pf) pf->end(st);
    }
    {   // P5
        const int W = 1 << mv.logW_y;
        const size_t sm = (size_t)g.Ly * (W + 1) * elt;
        if ((rc = set_smem<T>((const void*)k_yinv_compress<T, V>, sm))) return rc;
        dim3 grid((g.K + W - 1) / W, g.P, 3);
        if (pf) pf->begin(dt, 4, st);
        k_yinv_compress<T, V><<<grid, W * g.Ly / V, sm, st>>>(mv, p, y);
        DDA_LAUNCH_CHECK("P5 y-inverse + diagonal + compress");
        if (pf) pf->end(st);
    }
    return 0;
}

template void configure_matvec<double>(MatvecView<double>&);
template void configure_matvec<float>(MatvecView<float>&);
template int launch_matvec<double>(const MatvecView<double>&, const C<double>*, C<double>*, cudaStream_t);
template int launch_matvec<float>(const MatvecView<float>&, const C<float>*, C<float>*, cudaStream_t);

}  // namespace dda
