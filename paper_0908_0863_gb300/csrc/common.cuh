// Shared device/host helpers of the DDA CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/dda.h"
#include "df.cuh"

namespace dda {

// ------------------------------------------------------------ complex types
// complex128, complex64 and complex double-float (df.cuh)
template <typename T> struct cpx;
template <> struct cpx<double> { using t = double2; };
template <> struct cpx<float> { using t = float2; };
template <> struct cpx<DF> { using t = cdf; };
template <typename T> using C = typename cpx<T>::t;
// element type of the vectors a product of element type T reads and writes
// (the double-float product reads and writes complex128 vectors)
template <typename T> struct io_of { using t = T; };
template <> struct io_of<DF> { using t = double; };
template <typename T> using IO = typename io_of<T>::t;
template <typename T> __host__ __device__ __forceinline__ C<T> from_io(C<IO<T>> v) { return v; }
template <> __host__ __device__ __forceinline__ cdf from_io<DF>(double2 v) {
    cdf z;
    z.x = DF(v.x);
    z.y = DF(v.y);
    return z;
}
template <typename T> __host__ __device__ __forceinline__ C<IO<T>> to_io(C<T> v) { return v; }
template <> __host__ __device__ __forceinline__ double2 to_io<DF>(cdf v) {
    return make_double2(to_double(v.x), to_double(v.y));
}
// read-only cached load of one complex value
template <typename T> __device__ __forceinline__ C<T> ldg_c(const C<T>* p) { return __ldg(p); }
template <> __device__ __forceinline__ cdf ldg_c<DF>(const cdf* p) {
    const float4 f = __ldg(reinterpret_cast<const float4*>(p));
    cdf z;
    z.x = DF(f.x, f.y);
    z.y = DF(f.z, f.w);
    return z;
}

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T re, T im) { C<T> z; z.x = re; z.y = im; return z; }
template <typename T> __host__ __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __host__ __device__ __forceinline__ C<T> cmulc(C<T> a, C<T> b) {
    return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __host__ __device__ __forceinline__ C<T> cscale(C<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ C<T> cfma(C<T> a, C<T> b, C<T> acc) {
    return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}

// --------------------------------------------------------------- limits
constexpr int kTwEntries = 3072 + 5120;   // twiddle tables exp(-2 pi i m / 3072) and exp(-2 pi i m / 5120)
constexpr int kMaxEdge = 512;

// ------------------------------------------------------- error reporting
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define DDA_CUDA_TRY(expr)                                         \
    do {                                                           \
        cudaError_t e__ = (expr);                                  \
        if (e__ != cudaSuccess) return ::dda::cuda_fail(e__, #expr); \
    } while (0)

void note_launches(int64_t n);

// true for device or managed memory of any device; false for host memory,
// stale or foreign pointers (checked on the host before any launch)
bool is_device_ptr(const void* p);

// after every kernel launch: count it and turn a launch error into a status
#define DDA_LAUNCH_CHECK(what)                                           \
    do {                                                                 \
        ::dda::note_launches(1);                                         \
        cudaError_t e__ = cudaGetLastError();                            \
        if (e__ != cudaSuccess) return ::dda::cuda_fail(e__, what);      \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// -------------------------------------------------------- lattice geometry
struct Geometry {
    int K, J, P;          // lattice edges (x, y, z)
    int Lx, Ly, Lz;       // padded DFT lengths (padded_length)
    int Hx, Hy, Hz;       // stored half-spectrum extents L/2 + 1
    int Pb;               // pitch of the z columns of the xy-transformed volume (>= P)
    int64_t nsites;       // K J P
    int64_t nwords;       // occupancy words
    int64_t nd;           // occupied sites
    int nmat;             // materials
    int cbits;            // composition bits per field
    int cfields;          // fields per word
};

// lines of 3 * 2^a and 5 * 2^a points (the other supported lengths are 2^a)
__host__ __device__ constexpr bool wide_len(int N) { return N % 3 == 0 || N % 5 == 0; }

// Element of the half spectrum (my, mx, mz, component q): columns
// [Hy][Hx], every z line contiguous.  For z lines of 2^a points the six
// components of a point sit side by side ([Hz][6]: one 48-byte record per
// point, read whole by the z-pass thread that holds all three components);
// for 3 * 2^a and 5 * 2^a points, whose z pass gives each component its own
// threads, each component's line is contiguous ([6][Hz]).
__host__ __device__ __forceinline__ int64_t spec_index(const Geometry& g, int my, int mx, int mz, int q) {
    const int64_t col = ((int64_t)my * g.Hx + mx) * 6 * g.Hz;
    return col + (wide_len(g.Lz) ? (int64_t)q * g.Hz + mz : (int64_t)mz * 6 + q);
}

// circulant length of an n-point Toeplitz level: the smallest L >= 2n - 1
// (and >= 2) of the form 2^a, 3 * 2^a or 5 * 2^a (a >= 3 for the last two;
// Sec. 3: K'' = 2K - 1 + kf with kf chosen for a fast DFT)
inline int padded_length(int n) {
    const int need = 2 * n - 1 > 2 ? 2 * n - 1 : 2;
    int best = 0;
    for (int start : {2, 24, 40}) {
        int L = start;
        while (L < need) L *= 2;
        if (!best || L < best) best = L;
    }
    return best;
}
// Column pitch of the xy-transformed volume: P rounded up to a multiple of
// 8 elements, and to an odd multiple of 8 (so that the columns, read and
// written 64 or 128 bytes at a time across x by the x passes, do not start
// at a power-of-two stride)
inline int column_pitch(int P) {
    int p = (P + 7) / 8 * 8;
    if ((p / 8) % 2 == 0) p += 8;
    return p;
}
inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

// device view of the target for the expand / compress kernels
struct TargetView {
    const uint32_t* occ;     // occupancy words
    const uint32_t* rank;    // exclusive prefix count per word
    const uint32_t* comp;    // composition words or nullptr
    int cbits, cfields;
};

__device__ __forceinline__ bool occupied(const TargetView& t, int64_t s) {
    return (__ldg(t.occ + (s >> 5)) >> (s & 31)) & 1u;
}
__device__ __forceinline__ uint32_t site_rank(const TargetView& t, int64_t s) {
    const uint32_t w = __ldg(t.occ + (s >> 5));
    return __ldg(t.rank + (s >> 5)) + __popc(w & ((1u << (s & 31)) - 1u));
}
__device__ __forceinline__ int material(const TargetView& t, int64_t s, int axis) {
    if (t.comp == nullptr) return 0;
    const int64_t q = 3 * s + axis;
    const uint32_t w = __ldg(t.comp + q / t.cfields);
    return (w >> ((q % t.cfields) * t.cbits)) & ((1u << t.cbits) - 1u);
}

}  // namespace dda
