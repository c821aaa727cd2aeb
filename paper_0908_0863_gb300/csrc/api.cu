// C ABI of the library (include/dda.h): context set-up, the matvec, the
// solves with FP64 or mixed-precision iterative refinement (single and
// batched right-hand sides), and the observables and their permittivity
// gradients.  Host code only orchestrates; every step runs in the kernels
// of matvec.cu, spectrum.cu, target.cu and solver.cu.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "krylov.cuh"
#include "matvec.cuh"
#include "spectrum.cuh"
#include "target.cuh"

namespace dda {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};
static thread_local int64_t* t_capture_sink = nullptr;

// launches recorded into a CUDA graph are counted when the graph runs
void note_launches(int64_t n) {
    if (t_capture_sink) *t_capture_sink += n;
    else g_launches.fetch_add(n, std::memory_order_relaxed);
}
void capture_launches_into(int64_t* sink) { t_capture_sink = sink; }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int status, const std::string& msg) {
    g_last_error = msg;
    return status;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DDA_ERR_OOM : DDA_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// bump allocator over one device allocation
struct Arena {
    char* base = nullptr;
    size_t used = 0, cap = 0;
    template <typename X> X* take(size_t count) {
        used = (used + 255) & ~size_t(255);
        X* p = reinterpret_cast<X*>(base + used);
        used += count * sizeof(X);
        return p;
    }
};

__global__ void k_clear_tail(uint32_t* occ, int64_t nwords, int64_t nsites) {
    const int rem = (int)(nsites & 31);
    if (rem) occ[nwords - 1] &= (1u << rem) - 1u;
}

}  // namespace dda

using namespace dda;

// Solve workspace for `cap` right-hand sides of n = 3 N_d elements, in four
// groups that grow independently on demand (a larger batch, or the first
// batch in a precision): core vectors and per-RHS state, matvec work
// slots, FP64 Krylov vectors, complex64 Krylov vectors.
struct Space {
    int64_t n = 0;
    // core
    int cap_core = 0;
    void* mem_core = nullptr;
    void* pinned = nullptr;
    double2 *x64 = nullptr, *b64 = nullptr, *r64 = nullptr;   // [cap][n]
    RhsCtl* ctl = nullptr;        // device [cap]
    RhsCtl* hctl = nullptr;       // pinned [cap]
    KState *st64 = nullptr, *st32 = nullptr;     // device [cap]
    double2 *part64 = nullptr, *part32 = nullptr;
    KState* host = nullptr;       // pinned [cap]
    int* host_status = nullptr;   // pinned [2][cap]
    size_t bytes_core = 0;
    // matvec work: slots32 complex64 slots, or slots64 complex128 ones, in the same bytes
    int cap_work = 0;
    void* work = nullptr;
    int slots32 = 0, slots64 = 0;
    size_t bytes_work = 0;
    // Krylov vectors
    int cap64 = 0, cap32 = 0;
    void *mem64 = nullptr, *mem32 = nullptr;
    double2* v64[12] = {};
    float2* v32[12] = {};
    float2 *b32 = nullptr, *d32 = nullptr;   // inner right-hand side and solution
    size_t bytes64 = 0, bytes32 = 0;
    cudaStream_t capture = nullptr;   // graph capture stream
};

struct dda_ctx {
    Geometry g{};
    double k = 0.0;
    int device = 0;
    void* arena0 = nullptr;   // target, tables, spectrum
    void* arena1 = nullptr;   // adjoint / C_sca vectors
    int64_t bytes_fixed = 0;
    uint32_t *occ = nullptr, *rank = nullptr, *comp = nullptr;
    double2* ainv64 = nullptr;
    float2* ainv32 = nullptr;
    double2* jac64 = nullptr;    // point-Jacobi scale diag(A)^(-1/2) per material and axis
    float2* jac32 = nullptr;
    double2* spec64 = nullptr;
    float2* spec32 = nullptr;
    double2* tw64 = nullptr;
    float2* tw32 = nullptr;
    // the same tables for the double-float product (df.cuh)
    cdf *ainv_df = nullptr, *jac_df = nullptr, *spec_df = nullptr, *tw_df = nullptr;
    double2* xsec = nullptr;
    double2* msum = nullptr;  // per-material sums: block partials, then the sums
    double2* aux[3] = {};     // adjoint / C_sca work vectors (P, right-hand side, mu)
    double2* dainv64 = nullptr;  // d(alpha^-1)/d eps table of the last gradient call
    Space sp;
    // mixed precision, per Krylov method: smallest residual reduction an
    // inner solve aims at (0: none)
    std::array<double, DDA_MLBICGSTAB3 + 1> inner_rho{};
    int residual_dtype = DDA_C128DF;   // mixed precision: products of the true residuals
    MatvecView<double> mv64{};   // geometry, tables and tiles; work set per call
    MatvecView<float> mv32{};
    MatvecView<DF> mvdf{};
    PassProfiler prof;
};

namespace {

TargetView target_view(const dda_ctx* c) {
    TargetView t;
    t.occ = c->occ;
    t.rank = c->rank;
    t.comp = c->comp;
    t.cbits = c->g.cbits;
    t.cfields = c->g.cfields;
    return t;
}

int check_ctx(const dda_ctx* c) {
    if (!c) return fail(DDA_ERR_ARG, "null context");
    return 0;
}

int check_dev(const void* p, const char* what) {
    if (!p) return fail(DDA_ERR_ARG, std::string(what) + " is NULL");
    if (!is_device_ptr(p)) return fail(DDA_ERR_ARG, std::string(what) + " must be a device pointer");
    if (reinterpret_cast<uintptr_t>(p) % 16) return fail(DDA_ERR_ARG, std::string(what) + " must be 16-byte aligned");
    return 0;
}

constexpr int kMaxBatch = 4096;

// elements of one matvec work slot (Ay + Bxy)
size_t work_elems(const Geometry& g) { return 3ull * g.Ly * ((size_t)g.P * g.K + (size_t)g.Pb * g.Lx); }

int ensure_core(Space& sp, int nb) {
    if (sp.cap_core >= nb) return 0;
    if (sp.mem_core) { cudaFree(sp.mem_core); sp.mem_core = nullptr; }
    if (sp.pinned) { cudaFreeHost(sp.pinned); sp.pinned = nullptr; }
    sp.cap_core = 0;
    sp.bytes_core = 0;
    const size_t n = (size_t)sp.n, npart = (size_t)(kVecBlocks + nb) * kMaxRed;
    Arena probe;
    for (int i = 0; i < 3; ++i) probe.take<double2>(nb * n);
    probe.take<RhsCtl>(nb);
    probe.take<KState>(nb);
    probe.take<KState>(nb);
    probe.take<double2>(npart);
    probe.take<double2>(npart);
    Arena a;
    a.cap = probe.used + 256;
    cudaError_t e = cudaMalloc(&sp.mem_core, a.cap);
    if (e != cudaSuccess) { sp.mem_core = nullptr; return cuda_fail(e, "solve workspace"); }
    a.base = static_cast<char*>(sp.mem_core);
    sp.x64 = a.take<double2>(nb * n);
    sp.b64 = a.take<double2>(nb * n);
    sp.r64 = a.take<double2>(nb * n);
    sp.ctl = a.take<RhsCtl>(nb);
    sp.st64 = a.take<KState>(nb);
    sp.st32 = a.take<KState>(nb);
    sp.part64 = a.take<double2>(npart);
    sp.part32 = a.take<double2>(npart);
    const size_t hbytes = nb * (sizeof(RhsCtl) + sizeof(KState) + 2 * sizeof(int)) + 64;
    e = cudaMallocHost(&sp.pinned, hbytes);
    if (e != cudaSuccess) {
        cudaFree(sp.mem_core);
        sp.mem_core = nullptr;
        sp.pinned = nullptr;
        return cuda_fail(e, "pinned solver state");
    }
    std::memset(sp.pinned, 0, hbytes);
    char* h = static_cast<char*>(sp.pinned);
    sp.host = reinterpret_cast<KState*>(h);
    sp.hctl = reinterpret_cast<RhsCtl*>(h + nb * sizeof(KState));
    sp.host_status = reinterpret_cast<int*>(h + nb * (sizeof(KState) + sizeof(RhsCtl)));
    sp.cap_core = nb;
    sp.bytes_core = a.cap;
    return 0;
}

// work for nb complex64 slots; the complex128 products use the same bytes
// (at least one complex128 slot)
int ensure_work(Space& sp, const Geometry& g, int nb) {
    if (sp.cap_work >= nb) return 0;
    if (sp.work) { cudaFree(sp.work); sp.work = nullptr; }
    sp.cap_work = 0;
    sp.bytes_work = 0;
    const size_t w32 = work_elems(g) * sizeof(float2), w64 = work_elems(g) * sizeof(double2);
    const size_t bytes = std::max((size_t)nb * w32, w64);
    cudaError_t e = cudaMalloc(&sp.work, bytes);
    if (e != cudaSuccess) { sp.work = nullptr; return cuda_fail(e, "matvec work"); }
    sp.cap_work = nb;
    sp.slots32 = nb;
    sp.slots64 = (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, bytes / w64));
    sp.bytes_work = bytes;
    return 0;
}

int ensure_v64(Space& sp, int nb) {
    if (sp.cap64 >= nb) return 0;
    if (sp.mem64) { cudaFree(sp.mem64); sp.mem64 = nullptr; }
    sp.cap64 = 0;
    sp.bytes64 = 0;
    const size_t n = (size_t)sp.n;
    Arena probe;
    for (int i = 0; i < 12; ++i) probe.take<double2>(nb * n);
    Arena a;
    a.cap = probe.used + 256;
    cudaError_t e = cudaMalloc(&sp.mem64, a.cap);
    if (e != cudaSuccess) { sp.mem64 = nullptr; return cuda_fail(e, "FP64 Krylov vectors"); }
    a.base = static_cast<char*>(sp.mem64);
    for (int i = 0; i < 12; ++i) sp.v64[i] = a.take<double2>(nb * n);
    sp.cap64 = nb;
    sp.bytes64 = a.cap;
    return 0;
}

int ensure_v32(Space& sp, int nb) {
    if (sp.cap32 >= nb) return 0;
    if (sp.mem32) { cudaFree(sp.mem32); sp.mem32 = nullptr; }
    sp.cap32 = 0;
    sp.bytes32 = 0;
    const size_t n = (size_t)sp.n;
    Arena probe;
    for (int i = 0; i < 14; ++i) probe.take<float2>(nb * n);
    Arena a;
    a.cap = probe.used + 256;
    cudaError_t e = cudaMalloc(&sp.mem32, a.cap);
    if (e != cudaSuccess) { sp.mem32 = nullptr; return cuda_fail(e, "complex64 Krylov vectors"); }
    a.base = static_cast<char*>(sp.mem32);
    for (int i = 0; i < 12; ++i) sp.v32[i] = a.take<float2>(nb * n);
    sp.b32 = a.take<float2>(nb * n);
    sp.d32 = a.take<float2>(nb * n);
    sp.cap32 = nb;
    sp.bytes32 = a.cap;
    return 0;
}

void free_space(Space& sp) {
    if (sp.mem_core) cudaFree(sp.mem_core);
    if (sp.pinned) cudaFreeHost(sp.pinned);
    if (sp.work) cudaFree(sp.work);
    if (sp.mem64) cudaFree(sp.mem64);
    if (sp.mem32) cudaFree(sp.mem32);
    if (sp.capture) cudaStreamDestroy(sp.capture);
    sp = Space{};
}

// everything a solve of nb right-hand sides in this precision needs
int reserve(dda_ctx* c, int nb, int precision) {
    if (int rc = ensure_core(c->sp, nb)) return rc;
    if (int rc = ensure_work(c->sp, c->g, nb)) return rc;
    return precision == DDA_FP64 ? ensure_v64(c->sp, nb) : ensure_v32(c->sp, nb);
}

// matvec views over the workspace's work slots
MatvecView<double> view64(const dda_ctx* c, int nb) {
    MatvecView<double> m = c->mv64;
    m.slots = c->sp.slots64;
    m.Ay = static_cast<double2*>(c->sp.work);
    m.Bxy = m.Ay + (size_t)m.slots * 3ull * c->g.P * c->g.Ly * c->g.K;
    m.nb = nb;
    m.vstride = 3 * c->g.nd;
    m.status = nullptr;
    m.conj = 0;
    return m;
}
// the double-float product uses the complex128 work slots (16-byte elements)
MatvecView<DF> viewdf(const dda_ctx* c, int nb) {
    MatvecView<DF> m = c->mvdf;
    m.slots = c->sp.slots64;
    m.Ay = static_cast<cdf*>(c->sp.work);
    m.Bxy = m.Ay + (size_t)m.slots * 3ull * c->g.P * c->g.Ly * c->g.K;
    m.nb = nb;
    m.vstride = 3 * c->g.nd;
    m.status = nullptr;
    m.conj = 0;
    return m;
}
MatvecView<float> view32(const dda_ctx* c, int nb) {
    MatvecView<float> m = c->mv32;
    m.slots = c->sp.slots32;
    m.Ay = static_cast<float2*>(c->sp.work);
    m.Bxy = m.Ay + (size_t)m.slots * 3ull * c->g.P * c->g.Ly * c->g.K;
    m.nb = nb;
    m.vstride = 3 * c->g.nd;
    m.status = nullptr;
    m.conj = 0;
    return m;
}

KrylovWork<double> work64(const dda_ctx* c, int nb) {
    KrylovWork<double> w;
    w.n = c->sp.n;
    w.nb = nb;
    for (int i = 0; i < 12; ++i) w.v[i] = c->sp.v64[i];
    w.part = c->sp.part64;
    w.st = c->sp.st64;
    w.host = c->sp.host;
    w.host_status = c->sp.host_status;
    w.capture = c->sp.capture;
    return w;
}
KrylovWork<float> work32(const dda_ctx* c, int nb) {
    KrylovWork<float> w;
    w.n = c->sp.n;
    w.nb = nb;
    for (int i = 0; i < 12; ++i) w.v[i] = c->sp.v32[i];
    w.part = c->sp.part32;
    w.st = c->sp.st32;
    w.host = c->sp.host;
    w.host_status = c->sp.host_status;
    w.capture = c->sp.capture;
    return w;
}

// Tile widths chosen by dda_autotune, per lattice shape and dtype, for the
// whole process: later contexts of the same shape start with them.
std::mutex g_tiles_mu;
std::map<std::array<int, 4>, std::array<int, 4>> g_tiles;

std::array<int, 4> tile_key(const Geometry& g, int dtype) { return {g.K, g.J, g.P, dtype}; }

// The inner-solve target of the mixed precision chosen by
// dda_autotune_inner, per lattice shape and Krylov method, likewise.
std::map<std::array<int, 4>, double> g_inner;
constexpr int kInnerCandidates = 6;

template <typename T>
void apply_tiles(MatvecView<T>& m, const std::array<int, 4>& t) {
    m.logW_y = t[0];
    m.logW_z = t[1];
    m.logW_x = t[2];
}

int64_t context_bytes(const dda_ctx* c) {
    const Space& s = c->sp;
    return c->bytes_fixed + (int64_t)(s.bytes_core + s.bytes_work + s.bytes64 + s.bytes32);
}

}  // namespace

extern "C" {

const char* dda_last_error(void) { return g_last_error.c_str(); }

int dda_polarizability(int n, const double* m, double k, int rule, const double* khat, const double* e0,
                       double* alpha_out) {
    if (n < 1 || !m || !alpha_out) return fail(DDA_ERR_ARG, "dda_polarizability: bad arguments");
    const bool given_eps = (rule & DDA_POL_EPS) != 0;
    rule &= ~DDA_POL_EPS;
    if (rule < DDA_POL_CM || rule > DDA_POL_LDR) return fail(DDA_ERR_ARG, "dda_polarizability: unknown rule");
    if (rule == DDA_POL_LDR && (!khat || !e0)) return fail(DDA_ERR_ARG, "dda_polarizability: LDR needs khat and e0");
    if (!(k >= 0.0) || !std::isfinite(k)) return fail(DDA_ERR_ARG, "dda_polarizability: bad k");
    using cd = std::complex<double>;
    const double b1 = -1.8915316, b2 = 0.1648469, b3 = -1.7700004;
    double S = 0.0;
    if (rule == DDA_POL_LDR) {
        // S = sum_a (khat_a e_a)^2 with e complex; the real part is used
        cd s = 0.0;
        for (int a = 0; a < 3; ++a) {
            const cd t = khat[a] * cd(e0[2 * a], e0[2 * a + 1]);
            s += t * t;
        }
        S = s.real();
    }
    for (int q = 0; q < n; ++q) {
        const cd mm(m[2 * q], m[2 * q + 1]);
        const cd eps = given_eps ? mm : mm * mm;
        const cd acm = 3.0 / (4.0 * M_PI) * (eps - 1.0) / (eps + 2.0);
        cd a = acm;
        if (rule == DDA_POL_CMRR) {
            a = acm / (1.0 - cd(0.0, 2.0 / 3.0) * k * k * k * acm);
        } else if (rule == DDA_POL_LDR) {
            const cd corr = (b1 + eps * b2 + eps * b3 * S) * (k * k) - cd(0.0, 2.0 / 3.0) * (k * k * k);
            a = acm / (1.0 + acm * corr);
        }
        for (int c = 0; c < 3; ++c) {
            alpha_out[(q * 3 + c) * 2] = a.real();
            alpha_out[(q * 3 + c) * 2 + 1] = a.imag();
        }
    }
    return DDA_OK;
}

int dda_pack_occupancy(const uint8_t* mask, int64_t n_sites, uint32_t* bits, void* stream) {
    if (n_sites <= 0) return fail(DDA_ERR_ARG, "dda_pack_occupancy: n_sites must be > 0");
    if (!mask || !bits || !is_device_ptr(mask) || !is_device_ptr(bits))
        return fail(DDA_ERR_ARG, "dda_pack_occupancy: mask and bits must be device pointers");
    return launch_pack_occupancy(mask, n_sites, bits, as_stream(stream));
}

int dda_unpack_occupancy(const uint32_t* bits, int64_t n_sites, uint8_t* mask, void* stream) {
    if (n_sites <= 0) return fail(DDA_ERR_ARG, "dda_unpack_occupancy: n_sites must be > 0");
    if (!mask || !bits || !is_device_ptr(mask) || !is_device_ptr(bits))
        return fail(DDA_ERR_ARG, "dda_unpack_occupancy: mask and bits must be device pointers");
    return launch_unpack_occupancy(bits, n_sites, mask, as_stream(stream));
}

int dda_pack_composition(const uint8_t* materials, int64_t n_sites, int n_materials, uint32_t* bits, void* stream) {
    if (n_sites <= 0 || n_materials < 1 || n_materials > 256)
        return fail(DDA_ERR_ARG, "dda_pack_composition: bad sizes");
    if (!materials || !bits || !is_device_ptr(materials) || !is_device_ptr(bits))
        return fail(DDA_ERR_ARG, "dda_pack_composition: materials and bits must be device pointers");
    int bad = 0;
    if (int rc = launch_pack_composition(materials, n_sites, n_materials, bits, &bad, as_stream(stream))) return rc;
    if (bad) return fail(DDA_ERR_ARG, "dda_pack_composition: material index >= n_materials");
    return DDA_OK;
}

int dda_unpack_composition(const uint32_t* bits, int64_t n_sites, int n_materials, uint8_t* materials, void* stream) {
    if (n_sites <= 0 || n_materials < 1 || n_materials > 256)
        return fail(DDA_ERR_ARG, "dda_unpack_composition: bad sizes");
    if (!materials || !bits || !is_device_ptr(materials) || !is_device_ptr(bits))
        return fail(DDA_ERR_ARG, "dda_unpack_composition: materials and bits must be device pointers");
    return launch_unpack_composition(bits, n_sites, n_materials, materials, as_stream(stream));
}

void dda_free(dda_ctx* c) {
    if (!c) return;
    if (c->arena0) cudaFree(c->arena0);
    if (c->arena1) cudaFree(c->arena1);
    free_space(c->sp);
    delete c;
}

int dda_init_lattice(dda_ctx** out, const int32_t shape[3], const uint32_t* occupancy_bits,
                     const uint32_t* composition_bits, int n_materials, const double* alpha, double k,
                     void* stream) {
    if (!out) return fail(DDA_ERR_ARG, "dda_init_lattice: out is NULL");
    *out = nullptr;
    if (!shape || !occupancy_bits || !alpha) return fail(DDA_ERR_ARG, "dda_init_lattice: NULL argument");
    for (int a = 0; a < 3; ++a)
        if (shape[a] < 1 || shape[a] > kMaxEdge)
            return fail(DDA_ERR_ARG, "dda_init_lattice: each lattice edge must be in [1, 512]");
    if (n_materials < 1 || n_materials > 256) return fail(DDA_ERR_ARG, "dda_init_lattice: n_materials in [1, 256]");
    if (n_materials > 1 && !composition_bits)
        return fail(DDA_ERR_ARG, "dda_init_lattice: composition bits required when n_materials > 1");
    if (!(k > 0.0) || !std::isfinite(k)) return fail(DDA_ERR_ARG, "dda_init_lattice: k must be finite and > 0");
    for (int i = 0; i < n_materials * 6; ++i)
        if (!std::isfinite(alpha[i])) return fail(DDA_ERR_NAN, "dda_init_lattice: non-finite polarisability");
    for (int i = 0; i < n_materials * 3; ++i)
        if (alpha[2 * i] == 0.0 && alpha[2 * i + 1] == 0.0)
            return fail(DDA_ERR_ARG, "dda_init_lattice: zero polarisability");
    cudaStream_t st = as_stream(stream);
    dda_ctx* c = new dda_ctx();
    cudaGetDevice(&c->device);
    Geometry& g = c->g;
    g.K = shape[0]; g.J = shape[1]; g.P = shape[2];
    g.Lx = padded_length(g.K); g.Ly = padded_length(g.J); g.Lz = padded_length(g.P);
    g.Hx = g.Lx / 2 + 1; g.Hy = g.Ly / 2 + 1; g.Hz = g.Lz / 2 + 1;
    g.Pb = column_pitch(g.P);
    g.nsites = (int64_t)g.K * g.J * g.P;
    g.nwords = (g.nsites + 31) / 32;
    g.nmat = n_materials;
    g.cbits = dda::composition_bits(n_materials);
    g.cfields = 32 / g.cbits;
    c->k = k;
    const int64_t ncw = n_materials > 1 ? (3 * g.nsites + g.cfields - 1) / g.cfields : 0;
    const size_t nspec = 6ull * g.Hz * g.Hy * g.Hx;
    // ---- arena 0: target, tables, spectrum
    Arena a0;
    {
        Arena probe;  // sizing pass
        probe.take<uint32_t>(g.nwords);
        probe.take<uint32_t>(g.nwords);
        probe.take<uint32_t>(ncw);
        probe.take<uint32_t>(rank_scratch_words(g.nwords));
        probe.take<double2>(3 * (size_t)n_materials);
        probe.take<double2>(3 * (size_t)n_materials);
        probe.take<float2>(3 * (size_t)n_materials);
        probe.take<double2>(3 * (size_t)n_materials);
        probe.take<float2>(3 * (size_t)n_materials);
        probe.take<double2>(nspec);
        probe.take<float2>(nspec);
        probe.take<double2>(kTwEntries);
        probe.take<float2>(kTwEntries);
        probe.take<cdf>(3 * (size_t)n_materials);
        probe.take<cdf>(3 * (size_t)n_materials);
        probe.take<cdf>(nspec);
        probe.take<cdf>(kTwEntries);
        probe.take<double2>(xsec_scratch_elems());
        probe.take<double2>(material_sums_scratch_elems(g));
        probe.take<int>(4);
        a0.cap = probe.used + 256;
    }
    cudaError_t e = cudaMalloc(&c->arena0, a0.cap);
    if (e != cudaSuccess) { dda_free(c); return cuda_fail(e, "dda_init_lattice: allocation"); }
    a0.base = static_cast<char*>(c->arena0);
    c->occ = a0.take<uint32_t>(g.nwords);
    c->rank = a0.take<uint32_t>(g.nwords);
    c->comp = ncw ? a0.take<uint32_t>(ncw) : nullptr;
    uint32_t* rscratch = a0.take<uint32_t>(rank_scratch_words(g.nwords));
    c->ainv64 = a0.take<double2>(3 * (size_t)n_materials);
    c->ainv32 = a0.take<float2>(3 * (size_t)n_materials);
    c->dainv64 = a0.take<double2>(3 * (size_t)n_materials);
    c->jac64 = a0.take<double2>(3 * (size_t)n_materials);
    c->jac32 = a0.take<float2>(3 * (size_t)n_materials);
    c->spec64 = a0.take<double2>(nspec);
    c->spec32 = a0.take<float2>(nspec);
    c->tw64 = a0.take<double2>(kTwEntries);
    c->tw32 = a0.take<float2>(kTwEntries);
    c->ainv_df = a0.take<cdf>(3 * (size_t)n_materials);
    c->jac_df = a0.take<cdf>(3 * (size_t)n_materials);
    c->spec_df = a0.take<cdf>(nspec);
    c->tw_df = a0.take<cdf>(kTwEntries);
    c->xsec = a0.take<double2>(xsec_scratch_elems());
    c->msum = a0.take<double2>(material_sums_scratch_elems(g));
    int* flags = a0.take<int>(4);
    c->bytes_fixed = (int64_t)a0.cap;
    int rc = 0;
    auto bail = [&](int code) { dda_free(c); return code; };
    // ---- target bit fields
    if (cudaMemcpyAsync(c->occ, occupancy_bits, g.nwords * 4, cudaMemcpyDefault, st) != cudaSuccess)
        return bail(fail(DDA_ERR_ARG, "dda_init_lattice: cannot read occupancy bits"));
    k_clear_tail<<<1, 1, 0, st>>>(c->occ, g.nwords, g.nsites);
    if (ncw) {
        if (cudaMemcpyAsync(c->comp, composition_bits, ncw * 4, cudaMemcpyDefault, st) != cudaSuccess)
            return bail(fail(DDA_ERR_ARG, "dda_init_lattice: cannot read composition bits"));
    }
    if (cudaMemsetAsync(flags, 0, 4 * sizeof(int), st) != cudaSuccess) return bail(fail(DDA_ERR_CUDA, "memset"));
    if (ncw && (rc = launch_check_composition(c->comp, g.nsites, n_materials, flags, st))) return bail(rc);
    uint32_t* total = reinterpret_cast<uint32_t*>(flags + 1);
    if ((rc = launch_ranks(c->occ, g.nwords, c->rank, rscratch, total, st))) return bail(rc);
    int hflags[2] = {0, 0};
    if (cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return bail(fail(DDA_ERR_CUDA, "dda_init_lattice: rank scan failed"));
    if (hflags[0]) return bail(fail(DDA_ERR_ARG, "dda_init_lattice: material index >= n_materials"));
    g.nd = (int64_t)(uint32_t)hflags[1];
    if (g.nd == 0) return bail(fail(DDA_ERR_ARG, "dda_init_lattice: no occupied site"));
    // ---- alpha^-1 and twiddle tables (host FP64, a few hundred numbers)
    {
        std::vector<double2> ai(3 * n_materials), sj(3 * n_materials);
        std::vector<float2> af(3 * n_materials), sf(3 * n_materials);
        for (int i = 0; i < 3 * n_materials; ++i) {
            const std::complex<double> inv = 1.0 / std::complex<double>(alpha[2 * i], alpha[2 * i + 1]);
            ai[i] = make_double2(inv.real(), inv.imag());
            af[i] = make_float2((float)inv.real(), (float)inv.imag());
            const std::complex<double> sc = 1.0 / std::sqrt(inv);   // diag(A)^(-1/2), principal root
            sj[i] = make_double2(sc.real(), sc.imag());
            sf[i] = make_float2((float)sc.real(), (float)sc.imag());
        }
        std::vector<double2> t64(kTwEntries);
        std::vector<float2> t32(kTwEntries);
        for (int m = 0; m < kTwEntries; ++m) {
            // exp(-2 pi i m / 3072) for m < 3072, then exp(-2 pi i m' / 5120)
            const double ang = m < 3072 ? -2.0 * M_PI * (double)m / 3072.0 : -2.0 * M_PI * (double)(m - 3072) / 5120.0;
            t64[m] = make_double2(std::cos(ang), std::sin(ang));
            t32[m] = make_float2((float)t64[m].x, (float)t64[m].y);
        }
        // double-float copies (each double split into a float and the rounded remainder)
        auto split = [](const std::vector<double2>& v) {
            std::vector<cdf> out(v.size());
            for (size_t i = 0; i < v.size(); ++i) { out[i].x = DF(v[i].x); out[i].y = DF(v[i].y); }
            return out;
        };
        const std::vector<cdf> aidf = split(ai), sjdf = split(sj), twdf = split(t64);
        if (cudaMemcpyAsync(c->ainv_df, aidf.data(), aidf.size() * sizeof(cdf), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(c->jac_df, sjdf.data(), sjdf.size() * sizeof(cdf), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(c->tw_df, twdf.data(), twdf.size() * sizeof(cdf), cudaMemcpyHostToDevice, st))
            return bail(fail(DDA_ERR_CUDA, "dda_init_lattice: table upload"));
        if (cudaMemcpyAsync(c->ainv64, ai.data(), ai.size() * sizeof(double2), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(c->ainv32, af.data(), af.size() * sizeof(float2), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(c->jac64, sj.data(), sj.size() * sizeof(double2), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(c->jac32, sf.data(), sf.size() * sizeof(float2), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(c->tw64, t64.data(), kTwEntries * sizeof(double2), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(c->tw32, t32.data(), kTwEntries * sizeof(float2), cudaMemcpyHostToDevice, st) ||
            cudaStreamSynchronize(st))
            return bail(fail(DDA_ERR_CUDA, "dda_init_lattice: table upload"));
    }
    // ---- Green's-tensor spectrum (temporary build buffers)
    {
        const size_t ns = spectrum_scratch_elems(g);
        void* tmp = nullptr;
        e = cudaMalloc(&tmp, 2 * ns * sizeof(double2));
        if (e != cudaSuccess) return bail(cuda_fail(e, "dda_init_lattice: spectrum scratch"));
        double2* s0 = static_cast<double2*>(tmp);
        rc = build_spectrum(g, k, c->tw64, s0, s0 + ns, c->spec64, c->spec32, st);
        if (!rc) rc = spectrum_to_df(c->spec64, c->spec_df, nspec, st);
        cudaError_t e2 = cudaStreamSynchronize(st);
        cudaFree(tmp);
        if (rc) return bail(rc);
        if (e2 != cudaSuccess) return bail(cuda_fail(e2, "dda_init_lattice: spectrum build"));
    }
    // ---- adjoint / C_sca vectors, and the solve workspace for one
    // right-hand side in both precisions (3 + 3 + 10 complex128 and 12
    // complex64 vectors of 3 N_d, one matvec work slot)
    {
        const size_t n = 3 * (size_t)g.nd;
        Arena probe;
        for (int i = 0; i < 3; ++i) probe.take<double2>(n);
        Arena a1;
        a1.cap = probe.used + 256;
        e = cudaMalloc(&c->arena1, a1.cap);
        if (e != cudaSuccess) return bail(cuda_fail(e, "dda_init_lattice: adjoint vectors"));
        a1.base = static_cast<char*>(c->arena1);
        for (int i = 0; i < 3; ++i) c->aux[i] = a1.take<double2>(n);
        c->bytes_fixed += (int64_t)a1.cap;
        c->sp.n = (int64_t)n;
        if ((rc = ensure_core(c->sp, 1)) || (rc = ensure_work(c->sp, g, 1)) || (rc = ensure_v64(c->sp, 1)) ||
            (rc = ensure_v32(c->sp, 1)))
            return bail(rc);
        e = cudaStreamCreateWithFlags(&c->sp.capture, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(e, "dda_init_lattice: capture stream"));
    }
    // ---- matvec views (the work arrays are taken per call from the workspace)
    {
        const TargetView tv = target_view(c);
        MatvecView<double>& m = c->mv64;
        m.g = g; m.tv = tv; m.ainv = c->ainv64; m.spec = c->spec64; m.tw = c->tw64;
        m.status = nullptr; m.conj = 0; m.prof = &c->prof;
        configure_matvec<double>(m);
        MatvecView<float>& f = c->mv32;
        f.g = g; f.tv = tv; f.ainv = c->ainv32; f.spec = c->spec32; f.tw = c->tw32;
        f.status = nullptr; f.conj = 0; f.prof = &c->prof;
        configure_matvec<float>(f);
        MatvecView<DF>& d = c->mvdf;
        d.g = g; d.tv = tv; d.ainv = c->ainv_df; d.spec = c->spec_df; d.tw = c->tw_df;
        d.status = nullptr; d.conj = 0; d.prof = nullptr;
        configure_matvec<DF>(d);
        std::lock_guard<std::mutex> lock(g_tiles_mu);
        auto it = g_tiles.find(tile_key(g, DDA_C128));
        if (it != g_tiles.end()) apply_tiles(m, it->second);
        it = g_tiles.find(tile_key(g, DDA_C64));
        if (it != g_tiles.end()) apply_tiles(f, it->second);
        for (int mth = 0; mth <= DDA_MLBICGSTAB3; ++mth) {
            auto ir = g_inner.find(tile_key(g, -1 - mth));
            if (ir != g_inner.end()) c->inner_rho[mth] = ir->second;
        }
    }
    *out = c;
    return DDA_OK;
}

int dda_query(const dda_ctx* c, int64_t* n_dipoles, int32_t padded[3], int64_t* device_bytes) {
    if (int rc = check_ctx(c)) return rc;
    if (n_dipoles) *n_dipoles = c->g.nd;
    if (padded) { padded[0] = c->g.Lx; padded[1] = c->g.Ly; padded[2] = c->g.Lz; }
    if (device_bytes) *device_bytes = context_bytes(c);
    return DDA_OK;
}

int dda_profile(dda_ctx* c, int enable) {
    if (int rc = check_ctx(c)) return rc;
    c->prof.on = enable != 0;
    if (!enable) {
        int64_t n[10];
        double ms[10];
        c->prof.read(n, ms);
    }
    return DDA_OK;
}

int dda_profile_read(dda_ctx* c, int64_t* counts, double* ms) {
    if (int rc = check_ctx(c)) return rc;
    if (!counts || !ms) return fail(DDA_ERR_ARG, "dda_profile_read: NULL output");
    if (c->prof.read(counts, ms)) return fail(DDA_ERR_CUDA, "dda_profile_read: event wait failed");
    return DDA_OK;
}

int64_t dda_launch_count(void) { return launch_count(); }

int dda_site_ranks(const dda_ctx* c, uint32_t* rank, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (!rank || !is_device_ptr(rank)) return fail(DDA_ERR_ARG, "dda_site_ranks: rank must be a device pointer");
    return launch_site_ranks(target_view(c), c->g.nsites, rank, as_stream(stream));
}

int dda_tensor_spectrum(const dda_ctx* c, void* out, int dtype, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (int rc = check_dev(out, "dda_tensor_spectrum: out")) return rc;
    if (dtype != DDA_C128 && dtype != DDA_C64) return fail(DDA_ERR_ARG, "dda_tensor_spectrum: unknown dtype");
    const bool c128 = dtype == DDA_C128;
    if (int rc = export_spectrum(c->g, c128 ? (const void*)c->spec64 : (const void*)c->spec32, out, c128,
                                 as_stream(stream)))
        return rc;
    return DDA_OK;
}

int dda_matvec_batch(dda_ctx* c, int nb, const void* p, void* y, int dtype, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (nb < 1 || nb > kMaxBatch) return fail(DDA_ERR_ARG, "dda_matvec: nb must be in [1, 4096]");
    if (int rc = check_dev(p, "dda_matvec: p")) return rc;
    if (int rc = check_dev(y, "dda_matvec: y")) return rc;
    if (dtype != DDA_C128 && dtype != DDA_C64 && dtype != DDA_C128DF) return fail(DDA_ERR_ARG, "dda_matvec: unknown dtype");
    const size_t esize = dtype == DDA_C64 ? sizeof(float2) : sizeof(double2);
    const char *pb = static_cast<const char*>(p), *yb = static_cast<const char*>(y);
    const size_t span = (size_t)nb * 3 * c->g.nd * esize;
    if (pb < yb + span && yb < pb + span) return fail(DDA_ERR_ARG, "dda_matvec: p and y must not overlap");
    if (int rc = ensure_work(c->sp, c->g, nb)) return rc;
    cudaStream_t st = as_stream(stream);
    if (dtype == DDA_C128)
        return launch_matvec<double>(view64(c, nb), static_cast<const double2*>(p), static_cast<double2*>(y), st);
    if (dtype == DDA_C128DF)
        return launch_matvec<DF>(viewdf(c, nb), static_cast<const double2*>(p), static_cast<double2*>(y), st);
    return launch_matvec<float>(view32(c, nb), static_cast<const float2*>(p), static_cast<float2*>(y), st);
}

int dda_matvec(dda_ctx* c, const void* p, void* y, int dtype, void* stream) {
    return dda_matvec_batch(c, 1, p, y, dtype, stream);
}

int dda_tiles(dda_ctx* c, int dtype, int* tiles_out, const int* tiles_in) {
    if (int rc = check_ctx(c)) return rc;
    if (dtype != DDA_C128 && dtype != DDA_C64) return fail(DDA_ERR_ARG, "dda_tiles: unknown dtype");
    if (tiles_in) {
        const bool ok = tiles_in[3] == 0 &&
                        (dtype == DDA_C128 ? tiles_ok<double>(c->g, tiles_in[0], tiles_in[1], tiles_in[2])
                                           : tiles_ok<float>(c->g, tiles_in[0], tiles_in[1], tiles_in[2]));
        if (!ok) return fail(DDA_ERR_ARG, "dda_tiles: tile widths not launchable for this lattice");
        const std::array<int, 4> t{tiles_in[0], tiles_in[1], tiles_in[2], 0};
        if (dtype == DDA_C128) apply_tiles(c->mv64, t);
        else apply_tiles(c->mv32, t);
    }
    if (tiles_out) {
        if (dtype == DDA_C128) {
            tiles_out[0] = c->mv64.logW_y; tiles_out[1] = c->mv64.logW_z; tiles_out[2] = c->mv64.logW_x;
        } else {
            tiles_out[0] = c->mv32.logW_y; tiles_out[1] = c->mv32.logW_z; tiles_out[2] = c->mv32.logW_x;
        }
        tiles_out[3] = 0;
    }
    return DDA_OK;
}

int dda_autotune(dda_ctx* c, int dtype, int nb, int reps, double* pass_ms, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (dtype != DDA_C128 && dtype != DDA_C64) return fail(DDA_ERR_ARG, "dda_autotune: unknown dtype");
    if (nb < 1 || nb > kMaxBatch || reps < 1 || reps > 1000) return fail(DDA_ERR_ARG, "dda_autotune: bad nb or reps");
    if (int rc = ensure_work(c->sp, c->g, nb)) return rc;
    cudaStream_t st = as_stream(stream);
    const size_t esize = dtype == DDA_C128 ? sizeof(double2) : sizeof(float2);
    const size_t bytes = (size_t)nb * 3 * c->g.nd * esize;
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 2 * bytes);
    if (e != cudaSuccess) return cuda_fail(e, "dda_autotune: scratch vectors");
    // finite, nonzero data (every byte 0x3f) so the timed arithmetic is ordinary
    e = cudaMemsetAsync(buf, 0x3f, 2 * bytes, st);
    const bool was_on = c->prof.on;
    int64_t cnt[10];
    double ms[10];
    c->prof.read(cnt, ms);   // drop older records
    c->prof.on = true;
    const int d = dtype == DDA_C128 ? 0 : 1;
    auto current = [&]() {
        return dtype == DDA_C128
                   ? std::array<int, 4>{c->mv64.logW_y, c->mv64.logW_z, c->mv64.logW_x, 0}
                   : std::array<int, 4>{c->mv32.logW_y, c->mv32.logW_z, c->mv32.logW_x, 0};
    };
    auto set = [&](const std::array<int, 4>& t) {
        if (dtype == DDA_C128) apply_tiles(c->mv64, t);
        else apply_tiles(c->mv32, t);
    };
    auto valid = [&](const std::array<int, 4>& t) {
        return dtype == DDA_C128 ? tiles_ok<double>(c->g, t[0], t[1], t[2])
                                 : tiles_ok<float>(c->g, t[0], t[1], t[2]);
    };
    // one warm product, then reps timed ones; per-pass average milliseconds
    auto time_tiles = [&](double (&out)[5]) -> int {
        for (int r = 0; r <= reps; ++r) {
            if (r == 1) c->prof.read(cnt, ms);
            int rc = dtype == DDA_C128
                         ? launch_matvec<double>(view64(c, nb), static_cast<const double2*>(buf),
                                                 reinterpret_cast<double2*>(static_cast<char*>(buf) + bytes), st)
                         : launch_matvec<float>(view32(c, nb), static_cast<const float2*>(buf),
                                                reinterpret_cast<float2*>(static_cast<char*>(buf) + bytes), st);
            if (rc) return rc;
        }
        if (c->prof.read(cnt, ms)) return fail(DDA_ERR_CUDA, "dda_autotune: event wait failed");
        for (int q = 0; q < 5; ++q) out[q] = cnt[d * 5 + q] ? ms[d * 5 + q] / reps : 0.0;
        return 0;
    };
    int rc = e == cudaSuccess ? 0 : cuda_fail(e, "dda_autotune: fill");
    double best_ms[5] = {};
    if (!rc) rc = time_tiles(best_ms);
    const std::array<int, 4> initial = current();
    // P3's width (index 1), then P1/P5's (0), then P2/P4's (2), each over
    // two steps either side of the current one
    for (int a : {1, 0, 2}) {
        if (rc) break;
        std::array<int, 4> best = current();
        auto cost = [&](const double (&m)[5]) { return a == 1 ? m[2] : a == 0 ? m[0] + m[4] : m[1] + m[3]; };
        double best_cost = cost(best_ms);
        const std::array<int, 4> start = best;
        const int center = start[a];
        for (int cand = 0; cand < 5 && !rc; ++cand) {
            std::array<int, 4> t = start;
            t[a] = center - 2 + cand;
            if (t == start || t[a] < 0 || !valid(t)) continue;
            set(t);
            double m[5];
            rc = time_tiles(m);
            if (!rc && cost(m) < best_cost) {
                best_cost = cost(m);
                best = t;
                std::copy(m, m + 5, best_ms);
            }
        }
        set(best);
    }
    // Each step compared timings of separate runs.  Against that noise the
    // chosen and the initial settings are then timed alternately, three
    // rounds each, and the chosen ones are kept unless the median of the
    // initial ones is faster by more than 1%.
    if (!rc && current() != initial) {
        const std::array<int, 4> chosen = current();
        double tc[3], ti[3], mc[5] = {};
        for (int r = 0; r < 3 && !rc; ++r) {
            double m[5];
            set(chosen);
            rc = time_tiles(m);
            tc[r] = m[0] + m[1] + m[2] + m[3] + m[4];
            if (r == 0) std::copy(m, m + 5, mc);
            if (rc) break;
            set(initial);
            rc = time_tiles(m);
            ti[r] = m[0] + m[1] + m[2] + m[3] + m[4];
        }
        if (!rc) {
            std::sort(tc, tc + 3);
            std::sort(ti, ti + 3);
            if (ti[1] < 0.99 * tc[1]) {
                set(initial);
            } else {
                set(chosen);
                std::copy(mc, mc + 5, best_ms);
            }
        }
    }
    c->prof.on = was_on;
    cudaStreamSynchronize(st);
    cudaFree(buf);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tiles_mu);
        g_tiles[tile_key(c->g, dtype)] = current();
    }
    if (pass_ms) std::copy(best_ms, best_ms + 5, pass_ms);
    return DDA_OK;
}

int dda_reserve(dda_ctx* c, int nb, int precision) {
    if (int rc = check_ctx(c)) return rc;
    if (nb < 1 || nb > kMaxBatch) return fail(DDA_ERR_ARG, "dda_reserve: nb must be in [1, 4096]");
    if (precision != DDA_FP64 && precision != DDA_MIXED) return fail(DDA_ERR_ARG, "dda_reserve: unknown precision");
    return reserve(c, nb, precision);
}

int dda_incident_field(dda_ctx* c, const double* khat, const double* e0, void* einc, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (!khat || !e0) return fail(DDA_ERR_ARG, "dda_incident_field: NULL khat or e0");
    if (int rc = check_dev(einc, "dda_incident_field: einc")) return rc;
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(khat[i])) return fail(DDA_ERR_NAN, "dda_incident_field: non-finite khat");
    return launch_incident(target_view(c), c->g, c->k, khat, e0, static_cast<double2*>(einc), as_stream(stream));
}

static int map_status(int s) {
    switch (s) {
        case ST_CONVERGED: return DDA_OK;
        case ST_BREAKDOWN: return DDA_ERR_BREAKDOWN;
        case ST_NAN: return DDA_ERR_NAN;
        default: return DDA_ERR_NOT_CONVERGED;
    }
}

// the batch's return value: the most severe per-RHS status
static int worst_status(const int* st, int nb) {
    int w = DDA_OK;
    for (int b = 0; b < nb; ++b) {
        if (st[b] == DDA_ERR_NAN) return DDA_ERR_NAN;
        if (st[b] == DDA_ERR_BREAKDOWN) w = DDA_ERR_BREAKDOWN;
        else if (st[b] == DDA_ERR_NOT_CONVERGED && w == DDA_OK) w = DDA_ERR_NOT_CONVERGED;
    }
    return w;
}

// y = A x for the true residuals of the mixed refinement (x, y: the
// workspace's complex128 x and r vectors): double-float products
// (df.cuh, about 48 significant bits on the FP32 units) or FP64 ones, as
// set by dda_residual_dtype; right-hand sides whose control word is set are
// skipped when ctl is given
static int residual_product(dda_ctx* c, int nb, const RhsCtl* ctl, cudaStream_t st) {
    Space& sp = c->sp;
    if (c->residual_dtype == DDA_C128DF) {
        MatvecView<DF> m = viewdf(c, nb);
        if (ctl) { m.status = &ctl[0].skip; m.status_stride = kCtlInts; }
        return launch_matvec<DF>(m, sp.x64, sp.r64, st);
    }
    MatvecView<double> m = view64(c, nb);
    if (ctl) { m.status = &ctl[0].skip; m.status_stride = kCtlInts; }
    return launch_matvec<double>(m, sp.x64, sp.r64, st);
}

// Solves of nb right-hand sides in lock step (vectors [nb][3 N_d]); per-RHS
// results into inf[] and stat[].  Returns a non-solver error (ARG, CUDA,
// OOM) or 0.
static int solve_batch(dda_ctx* c, int nb, const void* einc, void* p, int method, int precision, double tol,
                       int max_iter, int use_x0, dda_solve_info* inf, int* stat, cudaStream_t st) {
    if (int rc = reserve(c, nb, precision)) return rc;
    const bool jacobi = (method & DDA_PRECOND_JACOBI) != 0;
    method &= 0xff;
    const TargetView tv = target_view(c);
    Space& sp = c->sp;
    const int64_t n = sp.n;
    const size_t bytes = (size_t)nb * n * sizeof(double2);
    DDA_CUDA_TRY(cudaMemcpyAsync(sp.b64, einc, bytes, cudaMemcpyDefault, st));
    if (use_x0) DDA_CUDA_TRY(cudaMemcpyAsync(sp.x64, p, bytes, cudaMemcpyDefault, st));
    for (int b = 0; b < nb; ++b) { inf[b] = dda_solve_info{}; stat[b] = DDA_ERR_NOT_CONVERGED; }
    std::vector<SolveResult> res(nb);
    std::vector<double> bn2(nb), rn2(nb);
    if (precision == DDA_FP64) {
        KrylovWork<double> w = work64(c, nb);
        MatvecView<double> m = view64(c, nb);
        const double2* rhs = sp.b64;
        if (jacobi) {
            // (S A S) y = S E, P = S y: the scaled right-hand side in r, the start y0 = S^-1 P0
            m.jac = c->jac64;
            DDA_CUDA_TRY(cudaMemcpyAsync(sp.r64, sp.b64, bytes, cudaMemcpyDeviceToDevice, st));
            if (int rc = launch_site_scale<double>(tv, c->g, c->jac64, sp.r64, nb, n, 0, st)) return rc;
            if (use_x0)
                if (int rc = launch_site_scale<double>(tv, c->g, c->jac64, sp.x64, nb, n, 1, st)) return rc;
            rhs = sp.r64;
        }
        if (int rc = krylov_solve<double>(method, m, w, rhs, sp.x64, use_x0 != 0, nullptr, tol, max_iter, st,
                                          res.data()))
            return rc;
        if (jacobi)
            if (int rc = launch_site_scale<double>(tv, c->g, c->jac64, sp.x64, nb, n, 0, st)) return rc;
        // true residuals with one FP64 product per right-hand side
        if (int rc = launch_matvec<double>(view64(c, nb), sp.x64, sp.r64, st)) return rc;
        if (int rc = residual_from_product(sp.b64, sp.r64, n, nb, nullptr, sp.part64, sp.st64, st)) return rc;
        if (int rc = read_tmp_slots(sp.st64, nb, sp.host, rn2.data(), st)) return rc;
        if (int rc = vec_norm2_c128(sp.b64, n, nb, sp.part64, sp.st64, st)) return rc;
        if (int rc = read_tmp_slots(sp.st64, nb, sp.host, bn2.data(), st)) return rc;
        for (int b = 0; b < nb; ++b) {
            stat[b] = map_status(res[b].status);
            inf[b].iterations = res[b].iterations;
            inf[b].matvecs = res[b].matvecs;
            inf[b].matvecs_fp64 = res[b].matvecs + 1;
            inf[b].rel_residual = std::sqrt(res[b].rel2);
            inf[b].rel_residual_true = bn2[b] > 0 ? std::sqrt(rn2[b] / bn2[b]) : 0.0;
        }
    } else {
        if (int rc = vec_norm2_c128(sp.b64, n, nb, sp.part64, sp.st64, st)) return rc;
        if (int rc = read_tmp_slots(sp.st64, nb, sp.host, bn2.data(), st)) return rc;
        if (use_x0) {
            if (int rc = residual_product(c, nb, nullptr, st)) return rc;
            if (int rc = residual_from_product(sp.b64, sp.r64, n, nb, nullptr, sp.part64, sp.st64, st)) return rc;
            if (int rc = read_tmp_slots(sp.st64, nb, sp.host, rn2.data(), st)) return rc;
            for (int b = 0; b < nb; ++b) inf[b].matvecs_fp64 += 1;
        } else {
            DDA_CUDA_TRY(cudaMemsetAsync(sp.x64, 0, bytes, st));
            DDA_CUDA_TRY(cudaMemcpyAsync(sp.r64, sp.b64, bytes, cudaMemcpyDeviceToDevice, st));
            rn2 = bn2;
        }
        std::vector<char> active(nb, 1);
        std::vector<int> stall(nb, 0);
        std::vector<double> best(nb);
        for (int b = 0; b < nb; ++b) {
            best[b] = rn2[b];
            if (!std::isfinite(bn2[b]) || !std::isfinite(rn2[b])) { stat[b] = DDA_ERR_NAN; active[b] = 0; }
        }
        RhsCtl* hc = sp.hctl;
        KrylovWork<float> w = work32(c, nb);
        while (true) {
            bool any = false;
            for (int b = 0; b < nb; ++b) {
                if (!active[b]) continue;
                const double rel = bn2[b] > 0 ? std::sqrt(rn2[b] / bn2[b]) : 0.0;
                inf[b].rel_residual = inf[b].rel_residual_true = rel;
                if (rel <= tol) { stat[b] = DDA_OK; active[b] = 0; }
                else if (inf[b].iterations >= max_iter) { stat[b] = DDA_ERR_NOT_CONVERGED; active[b] = 0; }
                else any = true;
            }
            if (!any) break;
            for (int b = 0; b < nb; ++b) {
                if (active[b]) {
                    const double rel = std::sqrt(rn2[b] / bn2[b]);
                    // inner target: enough to reach tol from here, not below what FP32
                    // sustains, and no finer than the context's per-solve reduction
                    double ti = std::max(0.3 * tol / rel, 1e-6);
                    if (c->inner_rho[method] > 0.0) ti = std::max(ti, c->inner_rho[method]);
                    hc[b].tol = std::min(0.5, ti);
                    hc[b].scale = 1.0 / std::sqrt(rn2[b]);
                    hc[b].mult = std::sqrt(rn2[b]);
                    hc[b].maxit = max_iter - inf[b].iterations;
                    hc[b].skip = 0;
                } else {
                    hc[b] = RhsCtl{0.0, 0.0, 0.0, 0, 1};
                }
            }
            DDA_CUDA_TRY(cudaMemcpyAsync(sp.ctl, hc, nb * sizeof(RhsCtl), cudaMemcpyHostToDevice, st));
            if (int rc = scale_to_c64(sp.r64, sp.ctl, sp.b32, n, nb, st)) return rc;
            MatvecView<float> m32 = view32(c, nb);
            if (jacobi) {   // inner solve of (S A S) d' = S r, d = S d'
                m32.jac = c->jac32;
                if (int rc = launch_site_scale<float>(tv, c->g, c->jac32, sp.b32, nb, n, 0, st)) return rc;
            }
            if (int rc = krylov_solve<float>(method, m32, w, sp.b32, sp.d32, false, sp.ctl, 0.0, 0, st, res.data()))
                return rc;
            if (jacobi)
                if (int rc = launch_site_scale<float>(tv, c->g, c->jac32, sp.d32, nb, n, 0, st)) return rc;
            // krylov_solve synchronised the stream: the controls may be rewritten
            bool changed = false;
            for (int b = 0; b < nb; ++b) {
                if (!active[b]) continue;
                inf[b].iterations += res[b].iterations;
                inf[b].matvecs += res[b].matvecs;
                if (res[b].status == ST_NAN) {
                    stat[b] = DDA_ERR_NAN;
                    active[b] = 0;
                    hc[b] = RhsCtl{0.0, 0.0, 0.0, 0, 1};
                    changed = true;
                }
            }
            if (changed)
                DDA_CUDA_TRY(cudaMemcpyAsync(sp.ctl, hc, nb * sizeof(RhsCtl), cudaMemcpyHostToDevice, st));
            if (int rc = axpy_from_c64(sp.x64, sp.ctl, sp.d32, n, nb, st)) return rc;
            // the residual product skips finished right-hand sides
            if (int rc = residual_product(c, nb, sp.ctl, st)) return rc;
            if (int rc = residual_from_product(sp.b64, sp.r64, n, nb, sp.ctl, sp.part64, sp.st64, st)) return rc;
            std::vector<double> rnew(nb);
            if (int rc = read_tmp_slots(sp.st64, nb, sp.host, rnew.data(), st)) return rc;
            for (int b = 0; b < nb; ++b) {
                if (!active[b]) continue;
                inf[b].matvecs_fp64 += 1;
                inf[b].refinements += 1;
                rn2[b] = rnew[b];
                if (!std::isfinite(rn2[b])) { stat[b] = DDA_ERR_NAN; active[b] = 0; continue; }
                if (rn2[b] < 0.25 * best[b]) {
                    best[b] = rn2[b];
                    stall[b] = 0;
                } else if (++stall[b] >= 3) {
                    inf[b].rel_residual = inf[b].rel_residual_true = std::sqrt(rn2[b] / bn2[b]);
                    stat[b] = res[b].status == ST_BREAKDOWN ? DDA_ERR_BREAKDOWN : DDA_ERR_NOT_CONVERGED;
                    active[b] = 0;
                    continue;
                }
                if (res[b].status == ST_BREAKDOWN && res[b].iterations == 0) {
                    inf[b].rel_residual = inf[b].rel_residual_true = std::sqrt(rn2[b] / bn2[b]);
                    stat[b] = DDA_ERR_BREAKDOWN;
                    active[b] = 0;
                }
            }
        }
    }
    DDA_CUDA_TRY(cudaMemcpyAsync(p, sp.x64, bytes, cudaMemcpyDefault, st));
    DDA_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

static int check_solve_args(const dda_ctx* c, int nb, const void* einc, const void* p, int method, int precision,
                            double tol, int max_iter) {
    if (int rc = check_ctx(c)) return rc;
    if (nb < 1 || nb > kMaxBatch) return fail(DDA_ERR_ARG, "dda_solve: nb must be in [1, 4096]");
    if (!einc || !p) return fail(DDA_ERR_ARG, "dda_solve: NULL einc or p");
    if ((method & ~(0xff | DDA_PRECOND_JACOBI)) || (method & 0xff) > DDA_MLBICGSTAB3)
        return fail(DDA_ERR_ARG, "dda_solve: unknown method");
    if (precision != DDA_FP64 && precision != DDA_MIXED) return fail(DDA_ERR_ARG, "dda_solve: unknown precision");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(DDA_ERR_ARG, "dda_solve: tol must be finite and > 0");
    if (max_iter < 1) return fail(DDA_ERR_ARG, "dda_solve: max_iter must be >= 1");
    return 0;
}

static void report(int status) {
    if (status == DDA_ERR_NOT_CONVERGED) set_error("dda_solve: not converged within max_iter");
    else if (status == DDA_ERR_BREAKDOWN) set_error("dda_solve: Krylov breakdown");
    else if (status == DDA_ERR_NAN) set_error("dda_solve: non-finite value");
}

int dda_solve_batch(dda_ctx* c, int nb, const void* einc, void* p, int method, int precision, double tol,
                    int max_iter, int use_x0, dda_solve_info* info, int* status, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (int rc = check_solve_args(c, nb, einc, p, method, precision, tol, max_iter)) return rc;
    std::vector<dda_solve_info> inf(nb);
    std::vector<int> stat(nb);
    if (int rc = solve_batch(c, nb, einc, p, method, precision, tol, max_iter, use_x0, inf.data(), stat.data(),
                             as_stream(stream)))
        return rc;
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int b = 0; b < nb; ++b) {
        inf[b].seconds = sec;
        if (info) info[b] = inf[b];
        if (status) status[b] = stat[b];
    }
    const int w = worst_status(stat.data(), nb);
    report(w);
    return w;
}

int dda_solve(dda_ctx* c, const void* einc, void* p, int method, int precision, double tol, int max_iter,
              int use_x0, dda_solve_info* info, void* stream) {
    return dda_solve_batch(c, 1, einc, p, method, precision, tol, max_iter, use_x0, info, nullptr, stream);
}

int dda_inner_tolerance(dda_ctx* c, int method, const double* rho_in, double* rho_out) {
    if (int rc = check_ctx(c)) return rc;
    if ((method & ~(0xff | DDA_PRECOND_JACOBI)) || (method & 0xff) > DDA_MLBICGSTAB3)
        return fail(DDA_ERR_ARG, "dda_inner_tolerance: unknown method");
    method &= 0xff;
    if (rho_in) {
        if (!(*rho_in >= 0.0 && *rho_in < 1.0)) return fail(DDA_ERR_ARG, "dda_inner_tolerance: rho must be in [0, 1)");
        c->inner_rho[method] = *rho_in;
    }
    if (rho_out) *rho_out = c->inner_rho[method];
    return DDA_OK;
}

int dda_residual_dtype(dda_ctx* c, const int* dtype_in, int* dtype_out) {
    if (int rc = check_ctx(c)) return rc;
    if (dtype_in) {
        if (*dtype_in != DDA_C128 && *dtype_in != DDA_C128DF)
            return fail(DDA_ERR_ARG, "dda_residual_dtype: DDA_C128 or DDA_C128DF");
        c->residual_dtype = *dtype_in;
    }
    if (dtype_out) *dtype_out = c->residual_dtype;
    return DDA_OK;
}

int dda_autotune_inner(dda_ctx* c, const void* einc, int method, double tol, int max_iter, double* rho_out,
                       double* ms_out, void* stream) {
    if (int rc = check_solve_args(c, 1, einc, einc, method, DDA_MIXED, tol, max_iter)) return rc;
    cudaStream_t st = as_stream(stream);
    const double cand[kInnerCandidates] = {0.0, 1e-4, 1e-3, 1e-2, 3e-2, 1e-1};
    const size_t bytes = 3 * c->g.nd * sizeof(double2);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "dda_autotune_inner: scratch solution");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int mth = method & 0xff;
    const double keep = c->inner_rho[mth];
    double best = -1.0, best_ms = 0.0;
    int rc = 0;
    for (int q = 0; q < kInnerCandidates && !rc; ++q) {
        c->inner_rho[mth] = cand[q];
        dda_solve_info info{};
        cudaEventRecord(e0, st);
        int status = dda_solve_batch(c, 1, einc, p, method, DDA_MIXED, tol, max_iter, 0, &info, nullptr, stream);
        cudaEventRecord(e1, st);
        if (status == DDA_ERR_ARG || status == DDA_ERR_CUDA || status == DDA_ERR_OOM) { rc = status; break; }
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = fail(DDA_ERR_CUDA, "dda_autotune_inner: event timing failed");
            break;
        }
        const double t = status == DDA_OK ? ms : -1.0;
        if (ms_out) ms_out[q] = t;
        // the first candidate (rho = 0, the default) is kept unless another
        // one is faster by more than 2% (single timings differ by about 1%)
        if (t > 0.0 && (best < 0.0 || t < (q > 0 && best == cand[0] ? 0.98 : 1.0) * best_ms)) {
            best = cand[q];
            best_ms = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(p);
    if (rc) { c->inner_rho[mth] = keep; return rc; }
    if (best < 0.0) {
        c->inner_rho[mth] = keep;
        return fail(DDA_ERR_NOT_CONVERGED, "dda_autotune_inner: no candidate converged");
    }
    c->inner_rho[mth] = best;
    {
        std::lock_guard<std::mutex> lock(g_tiles_mu);
        g_inner[tile_key(c->g, -1 - mth)] = best;
    }
    if (rho_out) *rho_out = best;
    return DDA_OK;
}

int dda_polarizability_derivative(int n, const double* m, double k, int rule, const double* khat, const double* e0,
                                  double* out) {
    const bool given_eps = (rule & DDA_POL_EPS) != 0;
    rule &= ~DDA_POL_EPS;
    if (n < 1 || !m || !out) return fail(DDA_ERR_ARG, "dda_polarizability_derivative: bad arguments");
    if (rule < DDA_POL_CM || rule > DDA_POL_LDR)
        return fail(DDA_ERR_ARG, "dda_polarizability_derivative: unknown rule");
    if (rule == DDA_POL_LDR && (!khat || !e0))
        return fail(DDA_ERR_ARG, "dda_polarizability_derivative: LDR needs khat and e0");
    using cd = std::complex<double>;
    double S = 0.0;
    if (rule == DDA_POL_LDR) {
        cd s = 0.0;
        for (int a = 0; a < 3; ++a) {
            const cd t = khat[a] * cd(e0[2 * a], e0[2 * a + 1]);
            s += t * t;
        }
        S = s.real();
    }
    const double b2 = 0.1648469, b3 = -1.7700004;
    for (int q = 0; q < n; ++q) {
        const cd mm(m[2 * q], m[2 * q + 1]);
        const cd eps = given_eps ? mm : mm * mm;
        if (eps == cd(1.0, 0.0)) return fail(DDA_ERR_ARG, "dda_polarizability_derivative: m = 1 (no polarisability)");
        // 1/alpha_CM = (4 pi/3)(eps + 2)/(eps - 1): derivative -4 pi/(eps - 1)^2;
        // radiative reaction adds a constant; LDR adds (b1 + eps b2 + eps b3 S) k^2
        cd d = -4.0 * M_PI / ((eps - 1.0) * (eps - 1.0));
        if (rule == DDA_POL_LDR) d += (b2 + b3 * S) * k * k;
        for (int c = 0; c < 3; ++c) {
            out[(q * 3 + c) * 2] = d.real();
            out[(q * 3 + c) * 2 + 1] = d.imag();
        }
    }
    return DDA_OK;
}

int dda_material_sums(dda_ctx* c, const void* v, double* out, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (!v || !out) return fail(DDA_ERR_ARG, "dda_material_sums: NULL argument");
    if (c->g.nmat > kMaxSumMaterials) return fail(DDA_ERR_ARG, "dda_material_sums: more than 32 materials");
    cudaStream_t st = as_stream(stream);
    const double2* vd = static_cast<const double2*>(v);
    if (!is_device_ptr(v)) {
        DDA_CUDA_TRY(cudaMemcpyAsync(c->aux[0], v, c->g.nd * sizeof(double2), cudaMemcpyHostToDevice, st));
        vd = c->aux[0];
    }
    if (int rc = launch_material_sums(target_view(c), c->g, vd, c->msum, st)) return rc;
    std::vector<double2> h(c->g.nmat);
    DDA_CUDA_TRY(cudaMemcpyAsync(h.data(), c->msum, c->g.nmat * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DDA_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < c->g.nmat; ++q) { out[2 * q] = h[q].x; out[2 * q + 1] = h[q].y; }
    return DDA_OK;
}

int dda_scattering_cross_section(dda_ctx* c, const void* p, double* out, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (!p || !out) return fail(DDA_ERR_ARG, "dda_scattering_cross_section: NULL argument");
    cudaStream_t st = as_stream(stream);
    const size_t bytes = 3 * c->g.nd * sizeof(double2);
    double2* P = c->aux[0];
    DDA_CUDA_TRY(cudaMemcpyAsync(P, p, bytes, cudaMemcpyDefault, st));
    MatvecView<double> m = view64(c, 1);
    if (int rc = launch_matvec<double>(m, P, c->aux[1], st)) return rc;        // A P
    m.conj = 1;
    if (int rc = launch_matvec<double>(m, P, c->aux[2], st)) return rc;        // A^H P
    if (int rc = launch_csca(target_view(c), c->g, c->k, c->ainv64, P, c->aux[1], c->aux[2], c->xsec, st)) return rc;
    double2 h;
    DDA_CUDA_TRY(cudaMemcpyAsync(&h, c->xsec + xsec_scratch_elems() - 1, sizeof(double2), cudaMemcpyDeviceToHost, st));
    DDA_CUDA_TRY(cudaStreamSynchronize(st));
    *out = 4.0 * M_PI * c->k * h.x;
    return DDA_OK;
}

int dda_gradient(dda_ctx* c, int which, const void* einc, const void* p, const double* dalpha_inv, int method,
                 int precision, double tol, int max_iter, void* grad, dda_solve_info* info, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (which != 0 && which != 1) return fail(DDA_ERR_ARG, "dda_gradient: which must be 0 (C_ext) or 1 (C_abs)");
    if (!p || !grad || !dalpha_inv || (which == 0 && !einc)) return fail(DDA_ERR_ARG, "dda_gradient: NULL argument");
    for (int i = 0; i < 6 * c->g.nmat; ++i)
        if (!std::isfinite(dalpha_inv[i])) return fail(DDA_ERR_NAN, "dda_gradient: non-finite derivative table");
    cudaStream_t st = as_stream(stream);
    const int64_t nd = c->g.nd;
    const size_t bytes = 3 * nd * sizeof(double2);
    double2 *P = c->aux[0], *rhs = c->aux[1], *mu = c->aux[2];
    DDA_CUDA_TRY(cudaMemcpyAsync(P, p, bytes, cudaMemcpyDefault, st));
    if (which == 0) DDA_CUDA_TRY(cudaMemcpyAsync(rhs, einc, bytes, cudaMemcpyDefault, st));
    DDA_CUDA_TRY(cudaMemcpyAsync(c->dainv64, dalpha_inv, 3 * c->g.nmat * sizeof(double2), cudaMemcpyHostToDevice, st));
    // adjoint right-hand side (in place for C_ext: conj(E))
    if (int rc = launch_adjoint_rhs(target_view(c), c->g, c->k, which, c->ainv64, rhs, P, rhs, st)) return rc;
    // one extra solve with A^T = A (the adjoint of a complex-symmetric system)
    dda_solve_info inf{};
    const int status = dda_solve(c, rhs, mu, method, precision, tol, max_iter, 0, &inf, stream);
    if (info) *info = inf;
    if (status == DDA_ERR_ARG || status == DDA_ERR_CUDA || status == DDA_ERR_OOM) return status;
    const bool dev_out = is_device_ptr(grad);
    double2* g = dev_out ? static_cast<double2*>(grad) : rhs;
    if (int rc = launch_gradient(target_view(c), c->g, c->k, which, c->dainv64, P, mu, g, st)) return rc;
    if (!dev_out) DDA_CUDA_TRY(cudaMemcpyAsync(grad, g, nd * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DDA_CUDA_TRY(cudaStreamSynchronize(st));
    return status;
}

int dda_cross_sections_batch(dda_ctx* c, int nb, const void* einc, const void* p, double* out, void* stream) {
    if (int rc = check_ctx(c)) return rc;
    if (nb < 1 || nb > kMaxBatch) return fail(DDA_ERR_ARG, "dda_cross_sections: nb must be in [1, 4096]");
    if (!einc || !p || !out) return fail(DDA_ERR_ARG, "dda_cross_sections: NULL argument");
    cudaStream_t st = as_stream(stream);
    const int64_t n = 3 * c->g.nd;
    const size_t bytes = (size_t)nb * n * sizeof(double2);
    const double2* E = static_cast<const double2*>(einc);
    const double2* P = static_cast<const double2*>(p);
    if (!is_device_ptr(einc) || !is_device_ptr(p))
        if (int rc = ensure_core(c->sp, nb)) return rc;
    if (!is_device_ptr(einc)) {
        DDA_CUDA_TRY(cudaMemcpyAsync(c->sp.b64, einc, bytes, cudaMemcpyHostToDevice, st));
        E = c->sp.b64;
    }
    if (!is_device_ptr(p)) {
        DDA_CUDA_TRY(cudaMemcpyAsync(c->sp.r64, p, bytes, cudaMemcpyHostToDevice, st));
        P = c->sp.r64;
    }
    // one reduction per right-hand side; each result is copied out before
    // the next one reuses the scratch (stream order)
    double2* h = reinterpret_cast<double2*>(c->sp.host);   // pinned, >= nb double2
    for (int b = 0; b < nb; ++b) {
        if (int rc = launch_cross_sections(target_view(c), c->g, c->k, c->ainv64, E + b * n, P + b * n, c->xsec, st))
            return rc;
        DDA_CUDA_TRY(cudaMemcpyAsync(h + b, c->xsec + xsec_scratch_elems() - 1, sizeof(double2),
                                     cudaMemcpyDeviceToHost, st));
    }
    DDA_CUDA_TRY(cudaStreamSynchronize(st));
    const double f = 4.0 * M_PI * c->k;
    for (int b = 0; b < nb; ++b) {
        out[3 * b] = f * h[b].x;
        out[3 * b + 1] = f * h[b].y;
        out[3 * b + 2] = out[3 * b] - out[3 * b + 1];
    }
    return DDA_OK;
}

int dda_cross_sections(dda_ctx* c, const void* einc, const void* p, double* out, void* stream) {
    return dda_cross_sections_batch(c, 1, einc, p, out, stream);
}

}  // extern "C"
