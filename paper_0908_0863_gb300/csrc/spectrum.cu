// Green's-tensor spectrum of the level-three Toeplitz interaction matrix
// (OpenDDA Sec. 3, App. A, Table 1), built once per target in FP64.
//
// Section 1 of the embedding holds the six independent components
// t_m(i, j, k), m = xx, xy, xz, yy, yz, zz, of the interaction tensor at
// displacements 0 <= i < K, 0 <= j < J, 0 <= k < P (t = 0 at the origin, the
// diagonal being added in the matvec).  The Toeplitz-to-circulant conversion
// and the DFT are fused line by line: every line of n values is extended to
// length L by mirroring entries 1..n-1 to L-1..L-n+1 with the Table-1 sign
// of that axis (zeros in between), transformed, and only the first L/2 + 1
// outputs are kept -- first along x, then y, then z, so each later pass
// works on the already reduced array.  The stored half spectrum is scaled by
// 1/(Lx Ly Lz) (the iDFT normalisation of Sec. 3 step 4) and copied to
// complex64 for the mixed-precision matvec.
#include "fft.cuh"
#include "matvec.cuh"
#include "spectrum.cuh"

namespace dda {

namespace {

// Table 1, row = axis (x, y, z), column = component
__device__ __forceinline__ double table1_sign(int axis, int m) {
    // sign -1 when the component pairs the mirrored axis with another axis
    const int a[6] = {0, 0, 0, 1, 1, 2}, b[6] = {0, 1, 2, 1, 2, 2};
    return ((a[m] == axis) != (b[m] == axis)) ? -1.0 : 1.0;
}

// t_m at r = (i, j, k) != 0:
//   exp(ikr)/r^3 [ k^2 (r_a r_b - r^2 d_ab) + (ikr - 1)/r^2 (3 r_a r_b - r^2 d_ab) ]
__global__ void k_section1(Geometry g, double kw, double2* __restrict__ t1) {
    const int64_t n = g.nsites;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(s % g.K);
        const int j = (int)((s / g.K) % g.J);
        const int k = (int)(s / ((int64_t)g.K * g.J));
        const double x = i, y = j, z = k;
        const double r2 = x * x + y * y + z * z;
        double2 out[6];
        if (r2 == 0.0) {
            for (int m = 0; m < 6; ++m) out[m] = make_double2(0.0, 0.0);
        } else {
            const double r = sqrt(r2);
            double sn, cs;
            sincos(kw * r, &sn, &cs);
            const double inv_r3 = 1.0 / (r2 * r);
            const double2 e = make_double2(cs * inv_r3, sn * inv_r3);           // exp(ikr)/r^3
            const double2 f = make_double2(-1.0 / r2, kw * r / r2);             // (ikr - 1)/r^2
            const double rr[6] = {x * x, x * y, x * z, y * y, y * z, z * z};
            const int diag[6] = {1, 0, 0, 1, 0, 1};
            for (int m = 0; m < 6; ++m) {
                const double d = diag[m] ? r2 : 0.0;
                const double a = kw * kw * (rr[m] - d);
                const double b = 3.0 * rr[m] - d;
                const double2 inner = make_double2(a + f.x * b, f.y * b);
                out[m] = make_double2(e.x * inner.x - e.y * inner.y, e.x * inner.y + e.y * inner.x);
            }
        }
        for (int m = 0; m < 6; ++m) t1[m * n + s] = out[m];
    }
}

constexpr int kV = 8;

// x lines: rows of K values (t1 [6][P][J][K]) -> rows of Hx ([6][P][J][Hx])
__global__ void __launch_bounds__(512) k_tensor_x(Geometry g, int logW, const double2* __restrict__ tw,
                                                  const double2* __restrict__ in, double2* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int W = 1 << logW, ld = W + 1, N = g.Lx;
    const int64_t rows_per_m = (int64_t)g.P * g.J, nrows = 6 * rows_per_m;
    const int64_t r0 = (int64_t)blockIdx.x * W;
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int w = e / N, n = e - w * N;
        const int64_t row = r0 + w;
        double2 v = make_double2(0.0, 0.0);
        if (row < nrows) {
            const int m = (int)(row / rows_per_m);
            if (n < g.K) {
                v = in[row * g.K + n];
            } else if (n > N - g.K) {
                v = in[row * g.K + (N - n)];
                const double sg = table1_sign(0, m);
                v.x *= sg; v.y *= sg;
            }
        }
        buf[n * ld + w] = v;
    }
    __syncthreads();
    fft_tile<double, kV, false>(buf, ld, logW, N, tw);
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int w = e / N, n = e - w * N;
        const int64_t row = r0 + w;
        if (row < nrows && n < g.Hx) out[row * g.Hx + n] = buf[n * ld + w];
    }
}

// strided lines along y (axis 1) or z (axis 2) on arrays whose rows are Hx
// long.  in: [6][n_outer][n_line][Hx] slices -> out: [6][n_outer][H][Hx]
// (y pass: outer = P, line = J -> Hy; z pass: the line is the outermost
// index of [6][P][Hy][Hx] -> the z-line layout of spec_index).
template <int AXIS>
__global__ void __launch_bounds__(512) k_tensor_col(Geometry g, int logW, const double2* __restrict__ tw,
                                                    const double2* __restrict__ in, double2* __restrict__ out,
                                                    double scale, float2* __restrict__ out32) {
    extern __shared__ unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int W = 1 << logW, ld = W + 1;
    const int N = AXIS == 1 ? g.Ly : g.Lz;
    const int nline = AXIS == 1 ? g.J : g.P;
    const int H = AXIS == 1 ? g.Hy : g.Hz;
    const int x0 = blockIdx.x * W;
    const int outer = blockIdx.y;   // y pass: z plane k; z pass: row my
    const int m = blockIdx.z;
    // element (line point n, column x) of the input and output
    int64_t in_base, in_step, out_base, out_step;
    if (AXIS == 1) {
        in_base = (((int64_t)m * g.P + outer) * g.J) * g.Hx;
        in_step = g.Hx;
        out_base = (((int64_t)m * g.P + outer) * g.Hy) * g.Hx;
        out_step = g.Hx;
    } else {
        in_base = ((int64_t)m * g.P * g.Hy + outer) * g.Hx;
        in_step = (int64_t)g.Hy * g.Hx;
        out_base = ((int64_t)m * g.Hz * g.Hy + outer) * g.Hx;
        out_step = (int64_t)g.Hy * g.Hx;
    }
    const double sg = table1_sign(AXIS, m);
    for (int e = threadIdx.x; e < W * N; e += blockDim.x) {
        const int n = e >> logW, w = e & (W - 1), x = x0 + w;
        double2 v = make_double2(0.0, 0.0);
        if (x < g.Hx) {
            if (n < nline) {
                v = in[in_base + n * in_step + x];
            } else if (n > N - nline) {
                v = in[in_base + (N - n) * in_step + x];
                v.x *= sg; v.y *= sg;
            }
        }
        buf[n * ld + w] = v;
    }
    __syncthreads();
    fft_tile<double, kV, false>(buf, ld, logW, N, tw);
    for (int e = threadIdx.x; e < W * H; e += blockDim.x) {
        const int n = e >> logW, w = e & (W - 1), x = x0 + w;
        if (x >= g.Hx) continue;
        double2 v = buf[n * ld + w];
        v.x *= scale; v.y *= scale;
        if (AXIS == 1) {
            out[out_base + n * out_step + x] = v;
        } else {
            // final spectrum: every z line contiguous (spec_index), so the z
            // pass reads a column's line in one stream
            const int64_t o = spec_index(g, outer, x, n, m);
            out[o] = v;
            if (out32) out32[o] = make_float2((float)v.x, (float)v.y);
        }
    }
}

int pick_logW_rows(int N) {   // rows of length N, V = 8 values per thread, <= 512 threads
    int logW = 0;
    while ((1 << logW) * 16 < 128 && (2 << logW) * N / kV <= 512) ++logW;
    while ((1 << logW) * N < kV) ++logW;
    return logW;
}

int pick_logW_cols(int N, int ncols) {
    int logW = 0;
    while ((1 << logW) * 16 < 128 && (2 << logW) * N / kV <= 512) ++logW;
    while (logW > 0 && (1 << (logW - 1)) >= ncols) --logW;
    while ((1 << logW) * N < kV) ++logW;
    return logW;
}

int smem_attr(const void* fn, size_t bytes) {
    if (bytes > 48 * 1024)
        DDA_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return 0;
}

}  // namespace

size_t spectrum_scratch_elems(const Geometry& g) {
    const size_t a = 6ull * g.P * g.J * g.K;
    const size_t b = 6ull * g.P * g.J * g.Hx;
    const size_t c = 6ull * g.P * g.Hy * g.Hx;
    return std::max(a, std::max(b, c));
}

int build_spectrum(const Geometry& g, double k, const double2* tw, double2* s0, double2* s1,
                   double2* spec64, float2* spec32, cudaStream_t st) {
    int rc;
    // section 1
    {
        const int threads = 256;
        const int64_t blocks = std::min<int64_t>((g.nsites + threads - 1) / threads, 152 * 64);
        k_section1<<<(unsigned)blocks, threads, 0, st>>>(g, k, s0);
        DDA_LAUNCH_CHECK("tensor section 1");
    }
    // x lines
    {
        const int logW = pick_logW_rows(g.Lx), W = 1 << logW;
        const size_t sm = (size_t)g.Lx * (W + 1) * sizeof(double2);
        if ((rc = smem_attr((const void*)k_tensor_x, sm))) return rc;
        const int64_t rows = 6ll * g.P * g.J;
        k_tensor_x<<<(unsigned)((rows + W - 1) / W), W * g.Lx / kV, sm, st>>>(g, logW, tw, s0, s1);
        DDA_LAUNCH_CHECK("tensor x DFT");
    }
    // y lines
    {
        const int logW = pick_logW_cols(g.Ly, g.Hx), W = 1 << logW;
        const size_t sm = (size_t)g.Ly * (W + 1) * sizeof(double2);
        if ((rc = smem_attr((const void*)k_tensor_col<1>, sm))) return rc;
        dim3 grid((g.Hx + W - 1) / W, g.P, 6);
        k_tensor_col<1><<<grid, W * g.Ly / kV, sm, st>>>(g, logW, tw, s1, s0, 1.0, nullptr);
        DDA_LAUNCH_CHECK("tensor y DFT");
    }
    // z lines, scaled, with the complex64 copy
    {
        const int logW = pick_logW_cols(g.Lz, g.Hx), W = 1 << logW;
        const size_t sm = (size_t)g.Lz * (W + 1) * sizeof(double2);
        if ((rc = smem_attr((const void*)k_tensor_col<2>, sm))) return rc;
        dim3 grid((g.Hx + W - 1) / W, g.Hy, 6);
        const double scale = 1.0 / ((double)g.Lx * g.Ly * g.Lz);
        k_tensor_col<2><<<grid, W * g.Lz / kV, sm, st>>>(g, logW, tw, s0, spec64, scale, spec32);
        DDA_LAUNCH_CHECK("tensor z DFT");
    }
    return 0;
}

// the spectrum in the exported order [Hy][Hx][Hz][6] from the stored one
template <typename T>
__global__ void __launch_bounds__(256) k_spec_export(Geometry g, const C<T>* __restrict__ in, C<T>* __restrict__ out) {
    const int64_t n = 6LL * g.Hz * g.Hy * g.Hx;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e % 6);
        const int64_t r = e / 6;
        const int mz = (int)(r % g.Hz);
        const int64_t col = r / g.Hz;
        out[e] = in[spec_index(g, (int)(col / g.Hx), (int)(col % g.Hx), mz, q)];
    }
}

// the double-float copy of the spectrum: each double split into the nearest
// float and the rounded remainder
__global__ void __launch_bounds__(256) k_spec_to_df(const double2* __restrict__ in, cdf* __restrict__ out, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = in[e];
        cdf z;
        z.x = DF(v.x);
        z.y = DF(v.y);
        out[e] = z;
    }
}

int spectrum_to_df(const double2* in, cdf* out, size_t n, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    k_spec_to_df<<<blocks, 256, 0, st>>>(in, out, (int64_t)n);
    DDA_LAUNCH_CHECK("spectrum double-float copy");
    return 0;
}

int export_spectrum(const Geometry& g, const void* in, void* out, bool c128, cudaStream_t st) {
    const size_t ns = 6ull * g.Hz * g.Hy * g.Hx;
    if (!wide_len(g.Lz)) {   // stored in the exported order
        DDA_CUDA_TRY(cudaMemcpyAsync(out, in, ns * (c128 ? sizeof(double2) : sizeof(float2)),
                                     cudaMemcpyDeviceToDevice, st));
        return 0;
    }
    const unsigned blocks = (unsigned)std::min<size_t>((ns + 255) / 256, 152 * 16);
    if (c128) k_spec_export<double><<<blocks, 256, 0, st>>>(g, static_cast<const double2*>(in), static_cast<double2*>(out));
    else k_spec_export<float><<<blocks, 256, 0, st>>>(g, static_cast<const float2*>(in), static_cast<float2*>(out));
    DDA_LAUNCH_CHECK("spectrum export");
    return 0;
}

}  // namespace dda
