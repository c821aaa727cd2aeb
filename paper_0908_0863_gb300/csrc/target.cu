// Bit-fielded target description (OpenDDA Sec. 2) and the per-dipole
// set-up and observables on it: occupancy / composition packing, the rank
// (compressed index) of every site for the zero-storage vectors of Sec. 4,
// the incident field and the cross-section sums.
#include <mutex>

#include "target.cuh"

namespace dda {

namespace {

// ------------------------------------------------------------- occupancy
// one warp packs 32 consecutive sites into one word with a ballot: lane l
// holds site 32 w + l, which becomes bit l (least significant first)
__global__ void k_pack_occ(const uint8_t* __restrict__ mask, int64_t n, uint32_t* __restrict__ bits) {
    const int64_t nwords = (n + 31) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < (nwords << 5); s += stride) {
        const bool on = s < n && mask[s] != 0;
        const uint32_t word = __ballot_sync(0xffffffffu, on);
        if ((threadIdx.x & 31) == 0) bits[s >> 5] = word;
    }
}

__global__ void k_unpack_occ(const uint32_t* __restrict__ bits, int64_t n, uint8_t* __restrict__ mask) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += stride)
        mask[s] = (bits[s >> 5] >> (s & 31)) & 1u;
}

// ----------------------------------------------------------- composition
__global__ void k_pack_comp(const uint8_t* __restrict__ mats, int64_t nfields, int nmat, int b, int f,
                            uint32_t* __restrict__ bits, int* __restrict__ bad) {
    const int64_t nwords = (nfields + f - 1) / f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t wd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; wd < nwords; wd += stride) {
        uint32_t word = 0;
        for (int t = 0; t < f; ++t) {
            const int64_t q = wd * f + t;
            if (q >= nfields) break;
            const uint32_t v = mats[q];
            if (v >= (uint32_t)nmat) atomicExch(bad, 1);
            word |= (v & ((1u << b) - 1u)) << (t * b);
        }
        bits[wd] = word;
    }
}

__global__ void k_unpack_comp(const uint32_t* __restrict__ bits, int64_t nfields, int b, int f,
                              uint8_t* __restrict__ mats) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nfields; q += stride)
        mats[q] = (bits[q / f] >> ((q % f) * b)) & ((1u << b) - 1u);
}

// range check of a composition field array already packed
__global__ void k_check_comp(const uint32_t* __restrict__ bits, int64_t nfields, int b, int f, int nmat,
                             int* __restrict__ bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nfields; q += stride) {
        const uint32_t v = (bits[q / f] >> ((q % f) * b)) & ((1u << b) - 1u);
        if (v >= (uint32_t)nmat) atomicExch(bad, 1);
    }
}

// ------------------------------------------------------------------ ranks
// three-step exclusive scan of the per-word popcounts:
//   1) each block scans kScanTile words, writing local prefixes and the block total
//   2) one block scans the block totals
//   3) add each block's offset
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads) k_rank_local(const uint32_t* __restrict__ occ, int64_t nwords,
                                                             uint32_t* __restrict__ rank, uint32_t* __restrict__ block_sum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPerThread;
    uint32_t c[kScanPerThread];
    uint32_t mine = 0;
#pragma unroll
    for (int t = 0; t < kScanPerThread; ++t) {
        c[t] = base + t < nwords ? __popc(occ[base + t]) : 0;
        mine += c[t];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(mine, &tot);
#pragma unroll
    for (int t = 0; t < kScanPerThread; ++t) {
        if (base + t < nwords) rank[base + t] = run;
        run += c[t];
    }
    if (threadIdx.x == 0) block_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_rank_blocks(uint32_t* __restrict__ block_sum, int64_t nblocks,
                                                              uint32_t* __restrict__ total) {
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < nblocks; b0 += kScanThreads) {
        const int64_t b = b0 + threadIdx.x;
        const uint32_t v = b < nblocks ? block_sum[b] : 0;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, &tot);
        if (b < nblocks) block_sum[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_rank_add(uint32_t* __restrict__ rank, int64_t nwords, const uint32_t* __restrict__ block_off) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords; w += stride)
        rank[w] += block_off[w / kScanTile];
}

__global__ void k_site_ranks(TargetView tv, int64_t n, uint32_t* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += stride) out[s] = site_rank(tv, s);
}

// --------------------------------------------------------- incident field
__global__ void k_incident(TargetView tv, Geometry g, double kw, double kx, double ky, double kz, double2 e0,
                           double2 e1, double2 e2, double2* __restrict__ E) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.nsites; s += stride) {
        if (!occupied(tv, s)) continue;
        const int i = (int)(s % g.K), j = (int)((s / g.K) % g.J), k = (int)(s / ((int64_t)g.K * g.J));
        double sn, cs;
        sincos(kw * (kx * i + ky * j + kz * k), &sn, &cs);
        const double2 ph = make_double2(cs, sn);
        const uint32_t r = site_rank(tv, s);
        E[r] = cmul<double>(e0, ph);
        E[g.nd + r] = cmul<double>(e1, ph);
        E[2 * g.nd + r] = cmul<double>(e2, ph);
    }
}

// --------------------------------------------------------- cross sections
// per block partial sums of Im(E^* P) and [-Im(ainv) - 2/3 k^3] |P|^2 over
// sites; the final sum over blocks runs in a fixed order on one block
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

__global__ void __launch_bounds__(kRedThreads) k_xsec_partial(TargetView tv, Geometry g, double k3,
                                                              const double2* __restrict__ ainv,
                                                              const double2* __restrict__ E,
                                                              const double2* __restrict__ P,
                                                              double2* __restrict__ part) {
    double ext = 0.0, abs_ = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.nsites; s += stride) {
        if (!occupied(tv, s)) continue;
        const uint32_t r = site_rank(tv, s);
        for (int c = 0; c < 3; ++c) {
            const double2 e = E[c * g.nd + r], p = P[c * g.nd + r];
            ext += e.x * p.y - e.y * p.x;                       // Im(conj(e) p)
            const double2 a = ainv[material(tv, s, c) * 3 + c];
            abs_ += (-a.y - (2.0 / 3.0) * k3) * (p.x * p.x + p.y * p.y);
        }
    }
    __shared__ double se[kRedThreads], sa[kRedThreads];
    se[threadIdx.x] = ext;
    sa[threadIdx.x] = abs_;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            se[threadIdx.x] += se[threadIdx.x + o];
            sa[threadIdx.x] += sa[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(se[0], sa[0]);
}

__global__ void __launch_bounds__(kRedThreads) k_xsec_final(const double2* __restrict__ part, int n, double2* out) {
    __shared__ double se[kRedThreads], sa[kRedThreads];
    double e = 0.0, a = 0.0;
    for (int i = threadIdx.x; i < n; i += kRedThreads) {
        e += part[i].x;
        a += part[i].y;
    }
    se[threadIdx.x] = e;
    sa[threadIdx.x] = a;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            se[threadIdx.x] += se[threadIdx.x + o];
            sa[threadIdx.x] += sa[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = make_double2(se[0], sa[0]);
}

// C_sca as the exact pair sum of the radiated power,
//   C_sca = 4 pi k sum_j [ (2/3) k^3 |P_j|^2 + P_j^H sum_{l != j} Im(G_jl) P_l ],
// G = diag(alpha^-1) - A being the dipole field tensor.  With A complex
// symmetric, Im(G) P = Im(alpha^-1) P - (A P - A^H P) / (2i), so the sum
// needs the two products A P and A^H P and this per-site reduction.
__global__ void __launch_bounds__(kRedThreads) k_csca_partial(TargetView tv, Geometry g, double k3,
                                                              const double2* __restrict__ ainv,
                                                              const double2* __restrict__ P,
                                                              const double2* __restrict__ AP,
                                                              const double2* __restrict__ AhP,
                                                              double2* __restrict__ part) {
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.nsites; s += stride) {
        if (!occupied(tv, s)) continue;
        const uint32_t r = site_rank(tv, s);
        for (int c = 0; c < 3; ++c) {
            const int64_t i = c * g.nd + r;
            const double2 p = P[i];
            const double2 a = ainv[material(tv, s, c) * 3 + c];
            const double2 d = make_double2(AP[i].x - AhP[i].x, AP[i].y - AhP[i].y);
            // (A P - A^H P) / (2i) = (d.y - i d.x) / 2
            const double2 q = make_double2(0.5 * d.y, -0.5 * d.x);
            const double re = p.x * q.x + p.y * q.y;   // Re(conj(p) q)
            acc += ((2.0 / 3.0) * k3 + a.y) * (p.x * p.x + p.y * p.y) - re;
        }
    }
    __shared__ double sa[kRedThreads];
    sa[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sa[threadIdx.x] += sa[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sa[0], 0.0);
}

// right-hand side of the adjoint solve A mu = b (A complex symmetric):
//   C_abs: b_c = w_c conj(P_c), w_c = -Im(alpha^-1_c) - (2/3) k^3;   C_ext: b = conj(E)
__global__ void k_adjoint_rhs(TargetView tv, Geometry g, double k3, int which, const double2* __restrict__ ainv,
                              const double2* __restrict__ E, const double2* __restrict__ P,
                              double2* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.nsites; s += stride) {
        if (!occupied(tv, s)) continue;
        const uint32_t r = site_rank(tv, s);
        for (int c = 0; c < 3; ++c) {
            const int64_t i = c * g.nd + r;
            if (which == 1) {
                const double w = -ainv[material(tv, s, c) * 3 + c].y - (2.0 / 3.0) * k3;
                out[i] = make_double2(w * P[i].x, -w * P[i].y);
            } else {
                out[i] = make_double2(E[i].x, -E[i].y);
            }
        }
    }
}

// per-dipole gradient g_j = dC/dRe(eps_j) + i dC/dIm(eps_j) from P and the
// adjoint solution mu, with a'_jc = d(alpha^-1_jc)/d eps (the three axes of
// a dipole share eps_j):
//   S = sum_c mu_c a'_c P_c
//   C_abs: 4 pi k ( sum_c -|P_c|^2 Im a'_c - 2 Re S ,  sum_c -|P_c|^2 Re a'_c + 2 Im S )
//   C_ext: 4 pi k ( -Im S , -Re S )
__global__ void k_gradient(TargetView tv, Geometry g, double k, int which, const double2* __restrict__ dainv,
                           const double2* __restrict__ P, const double2* __restrict__ mu,
                           double2* __restrict__ grad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const double f = 4.0 * 3.14159265358979323846 * k;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.nsites; s += stride) {
        if (!occupied(tv, s)) continue;
        const uint32_t r = site_rank(tv, s);
        double2 S = make_double2(0.0, 0.0);
        double dx = 0.0, dy = 0.0;
        for (int c = 0; c < 3; ++c) {
            const int64_t i = c * g.nd + r;
            const double2 p = P[i], u = mu[i];
            const double2 d = dainv[material(tv, s, c) * 3 + c];
            const double2 t = cmul<double>(cmul<double>(u, d), p);
            S.x += t.x;
            S.y += t.y;
            const double ap = p.x * p.x + p.y * p.y;
            dx -= ap * d.y;
            dy -= ap * d.x;
        }
        if (which == 1) {
            dx -= 2.0 * S.x;
            dy += 2.0 * S.y;
        } else {
            dx = -S.y;
            dy = -S.x;
        }
        grad[r] = make_double2(f * dx, f * dy);
    }
}

inline unsigned grid_for(int64_t n, int threads) {
    const int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

int launch_pack_occupancy(const uint8_t* mask, int64_t n, uint32_t* bits, cudaStream_t st) {
    k_pack_occ<<<grid_for((n + 31) / 32 * 32, 256), 256, 0, st>>>(mask, n, bits);
    DDA_LAUNCH_CHECK("pack occupancy");
    return 0;
}

int launch_unpack_occupancy(const uint32_t* bits, int64_t n, uint8_t* mask, cudaStream_t st) {
    k_unpack_occ<<<grid_for(n, 256), 256, 0, st>>>(bits, n, mask);
    DDA_LAUNCH_CHECK("unpack occupancy");
    return 0;
}

// out-of-range flag of dda_pack_composition: one word per device, shared by
// all calls (calls that overlap on the GPU share it)
__device__ int g_pack_bad;

int launch_pack_composition(const uint8_t* mats, int64_t nsites, int nmat, uint32_t* bits, int* bad_host,
                            cudaStream_t st) {
    const int b = composition_bits(nmat), f = 32 / b;
    const int64_t nf = 3 * nsites;
    int* bad = nullptr;
    DDA_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void**>(&bad), g_pack_bad));
    DDA_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    k_pack_comp<<<grid_for((nf + f - 1) / f, 256), 256, 0, st>>>(mats, nf, nmat, b, f, bits, bad);
    DDA_LAUNCH_CHECK("pack composition");
    DDA_CUDA_TRY(cudaMemcpyAsync(bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    DDA_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int launch_unpack_composition(const uint32_t* bits, int64_t nsites, int nmat, uint8_t* mats, cudaStream_t st) {
    const int b = composition_bits(nmat), f = 32 / b;
    k_unpack_comp<<<grid_for(3 * nsites, 256), 256, 0, st>>>(bits, 3 * nsites, b, f, mats);
    DDA_LAUNCH_CHECK("unpack composition");
    return 0;
}

int launch_check_composition(const uint32_t* bits, int64_t nsites, int nmat, int* bad, cudaStream_t st) {
    const int b = composition_bits(nmat), f = 32 / b;
    k_check_comp<<<grid_for(3 * nsites, 256), 256, 0, st>>>(bits, 3 * nsites, b, f, nmat, bad);
    DDA_LAUNCH_CHECK("check composition");
    return 0;
}

size_t rank_scratch_words(int64_t nwords) { return (size_t)((nwords + kScanTile - 1) / kScanTile) + 1; }

int launch_ranks(const uint32_t* occ, int64_t nwords, uint32_t* rank, uint32_t* scratch, uint32_t* total,
                 cudaStream_t st) {
    const int64_t nblocks = (nwords + kScanTile - 1) / kScanTile;
    k_rank_local<<<(unsigned)nblocks, kScanThreads, 0, st>>>(occ, nwords, rank, scratch);
    DDA_LAUNCH_CHECK("rank local scan");
    k_rank_blocks<<<1, kScanThreads, 0, st>>>(scratch, nblocks, total);
    DDA_LAUNCH_CHECK("rank block scan");
    k_rank_add<<<grid_for(nwords, 256), 256, 0, st>>>(rank, nwords, scratch);
    DDA_LAUNCH_CHECK("rank offsets");
    return 0;
}

int launch_site_ranks(const TargetView& tv, int64_t n, uint32_t* out, cudaStream_t st) {
    k_site_ranks<<<grid_for(n, 256), 256, 0, st>>>(tv, n, out);
    DDA_LAUNCH_CHECK("site ranks");
    return 0;
}

int launch_incident(const TargetView& tv, const Geometry& g, double k, const double* khat, const double* e0,
                    double2* E, cudaStream_t st) {
    k_incident<<<grid_for(g.nsites, 256), 256, 0, st>>>(tv, g, k, khat[0], khat[1], khat[2],
                                                      make_double2(e0[0], e0[1]), make_double2(e0[2], e0[3]),
                                                      make_double2(e0[4], e0[5]), E);
    DDA_LAUNCH_CHECK("incident field");
    return 0;
}

size_t xsec_scratch_elems() { return kRedBlocks + 1; }

int launch_cross_sections(const TargetView& tv, const Geometry& g, double k, const double2* ainv,
                          const double2* E, const double2* P, double2* scratch, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, (g.nsites + kRedThreads - 1) / kRedThreads));
    k_xsec_partial<<<blocks, kRedThreads, 0, st>>>(tv, g, k * k * k, ainv, E, P, scratch);
    DDA_LAUNCH_CHECK("cross-section partial sums");
    k_xsec_final<<<1, kRedThreads, 0, st>>>(scratch, (int)blocks, scratch + kRedBlocks);
    DDA_LAUNCH_CHECK("cross-section final sum");
    return 0;
}

int launch_csca(const TargetView& tv, const Geometry& g, double k, const double2* ainv, const double2* P,
                const double2* AP, const double2* AhP, double2* scratch, cudaStream_t st) {
    const unsigned blocks =
        (unsigned)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, (g.nsites + kRedThreads - 1) / kRedThreads));
    k_csca_partial<<<blocks, kRedThreads, 0, st>>>(tv, g, k * k * k, ainv, P, AP, AhP, scratch);
    DDA_LAUNCH_CHECK("C_sca partial sums");
    k_xsec_final<<<1, kRedThreads, 0, st>>>(scratch, (int)blocks, scratch + kRedBlocks);
    DDA_LAUNCH_CHECK("C_sca final sum");
    return 0;
}

int launch_adjoint_rhs(const TargetView& tv, const Geometry& g, double k, int which, const double2* ainv,
                       const double2* E, const double2* P, double2* out, cudaStream_t st) {
    k_adjoint_rhs<<<grid_for(g.nsites, 256), 256, 0, st>>>(tv, g, k * k * k, which, ainv, E, P, out);
    DDA_LAUNCH_CHECK("adjoint right-hand side");
    return 0;
}

template <typename T>
__global__ void k_site_scale(TargetView tv, Geometry g, const C<T>* __restrict__ tab, C<T>* __restrict__ vec,
                             int64_t stride, int inverse) {
    vec += (int64_t)blockIdx.y * stride;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.nsites; s += step) {
        if (!occupied(tv, s)) continue;
        const uint32_t r = site_rank(tv, s);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C<T> f = tab[material(tv, s, c) * 3 + c];
            if (inverse) {
                const T d = f.x * f.x + f.y * f.y;
                f = mk<T>(f.x / d, -f.y / d);
            }
            C<T>& v = vec[(int64_t)c * g.nd + r];
            v = cmul<T>(v, f);
        }
    }
}

template <typename T>
int launch_site_scale(const TargetView& tv, const Geometry& g, const C<T>* tab, C<T>* vec, int nb, int64_t stride,
                      int inverse, cudaStream_t st) {
    const unsigned gx = std::max(1u, std::min(grid_for(g.nsites, 256), (unsigned)((1216 + nb - 1) / nb)));
    k_site_scale<T><<<dim3(gx, nb), 256, 0, st>>>(tv, g, tab, vec, stride, inverse);
    DDA_LAUNCH_CHECK("Jacobi scaling");
    return 0;
}

template int launch_site_scale<double>(const TargetView&, const Geometry&, const C<double>*, C<double>*, int, int64_t,
                                       int, cudaStream_t);
template int launch_site_scale<float>(const TargetView&, const Geometry&, const C<float>*, C<float>*, int, int64_t,
                                      int, cudaStream_t);

int launch_gradient(const TargetView& tv, const Geometry& g, double k, int which, const double2* dainv,
                    const double2* P, const double2* mu, double2* grad, cudaStream_t st) {
    k_gradient<<<grid_for(g.nsites, 256), 256, 0, st>>>(tv, g, k, which, dainv, P, mu, grad);
    DDA_LAUNCH_CHECK("permittivity gradient");
    return 0;
}

// ------------------------------------------------------ per-material sums
// Each thread sums the values of its sites into its own row of a shared
// [threads][nmat] table (no atomics), the block adds the rows in a fixed
// order and writes one partial per material, and one block adds the
// partials in block order: the same bits on every call.
constexpr int kSumThreads = 64;   // the [threads][32] table of double2 fits 32 KB
constexpr int kSumBlocks = 256;

size_t material_sums_scratch_elems(const Geometry&) { return (size_t)(kSumBlocks + 1) * kMaxSumMaterials; }

__global__ void __launch_bounds__(kSumThreads) k_material_partial(TargetView tv, Geometry g,
                                                                   const double2* __restrict__ v,
                                                                   double2* __restrict__ part) {
    __shared__ double2 acc[kSumThreads][kMaxSumMaterials];
    const int nm = g.nmat;
    for (int q = 0; q < nm; ++q) acc[threadIdx.x][q] = make_double2(0.0, 0.0);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < g.nsites; s += stride) {
        if (!occupied(tv, s)) continue;
        const double2 x = v[site_rank(tv, s)];
        double2& a = acc[threadIdx.x][material(tv, s, 0)];
        a.x += x.x;
        a.y += x.y;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nm; q += blockDim.x) {
        double2 t = make_double2(0.0, 0.0);
        for (int i = 0; i < kSumThreads; ++i) { t.x += acc[i][q].x; t.y += acc[i][q].y; }
        part[blockIdx.x * kMaxSumMaterials + q] = t;
    }
}

__global__ void k_material_final(const double2* __restrict__ part, int nblocks, int nm, double2* __restrict__ out) {
    for (int q = threadIdx.x; q < nm; q += blockDim.x) {
        double2 t = make_double2(0.0, 0.0);
        for (int b = 0; b < nblocks; ++b) { t.x += part[b * kMaxSumMaterials + q].x; t.y += part[b * kMaxSumMaterials + q].y; }
        out[q] = t;
    }
}

int launch_material_sums(const TargetView& tv, const Geometry& g, const double2* v, double2* scratch,
                         cudaStream_t st) {
    if (g.nmat > kMaxSumMaterials) return fail(DDA_ERR_ARG, "material sums: more than 32 materials");
    const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(kSumBlocks, (g.nsites + kSumThreads - 1) / kSumThreads));
    k_material_partial<<<nblocks, kSumThreads, 0, st>>>(tv, g, v, scratch + kMaxSumMaterials);
    DDA_LAUNCH_CHECK("material sums");
    k_material_final<<<1, kMaxSumMaterials, 0, st>>>(scratch + kMaxSumMaterials, nblocks, g.nmat, scratch);
    DDA_LAUNCH_CHECK("material sums final");
    return 0;
}

// ------------------------------------- rank scan without device allocation
// dda_occupancy_ranks_static runs the rank scan above with its per-block
// totals in this file-scope array instead of caller or context memory, so
// the call allocates nothing.  Every GPU that loads the library holds the
// array (16 KB) until the process exits.  It bounds the input at
// kStaticScanBlocks blocks of kScanTile words: 4096 * 4096 * 32 sites.
constexpr int kStaticScanBlocks = 4096;
__device__ __align__(256) uint32_t g_static_scan[kStaticScanBlocks];
constexpr int64_t kStaticScanMaxSites = (int64_t)kStaticScanBlocks * kScanTile * 32;

namespace {

// the device address of g_static_scan, looked up once per device (with that
// device current) on the first call made there
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
uint32_t* g_static_addr[kMaxDevices] = {};

int static_scan_address(uint32_t** out) {
    int dev = 0;
    DDA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(DDA_ERR_ARG, "dda_occupancy_ranks_static: device index >= 64");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scan);
        if (e != cudaSuccess) return cuda_fail(e, "dda_occupancy_ranks_static: cudaGetSymbolAddress");
        g_static_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_static_addr[dev];
    return 0;
}

// first scan step on the caller's (read-only) bit field: the padding bits
// beyond n_sites in the last word are masked here instead of cleared
__global__ void __launch_bounds__(kScanThreads) k_rank_local_masked(const uint32_t* __restrict__ occ, int64_t nwords,
                                                                    uint32_t last_mask, uint32_t* __restrict__ rank,
                                                                    uint32_t* __restrict__ block_sum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPerThread;
    uint32_t c[kScanPerThread];
    uint32_t mine = 0;
#pragma unroll
    for (int t = 0; t < kScanPerThread; ++t) {
        const int64_t w = base + t;
        c[t] = w < nwords ? __popc(occ[w] & (w == nwords - 1 ? last_mask : 0xffffffffu)) : 0;
        mine += c[t];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(mine, &tot);
#pragma unroll
    for (int t = 0; t < kScanPerThread; ++t) {
        if (base + t < nwords) rank[base + t] = run;
        run += c[t];
    }
    if (threadIdx.x == 0) block_sum[blockIdx.x] = tot;
}

}  // namespace

}  // namespace dda

extern "C" int dda_occupancy_ranks_static(const uint32_t* occupancy_bits, int64_t n_sites, uint32_t* word_rank,
                                          uint32_t* n_occupied, void* stream) {
    using namespace dda;
    if (n_sites <= 0) return fail(DDA_ERR_ARG, "dda_occupancy_ranks_static: n_sites must be > 0");
    if (n_sites > kStaticScanMaxSites)
        return fail(DDA_ERR_ARG, "dda_occupancy_ranks_static: n_sites above the static scratch limit of "
                                 "536870912 sites (4096 blocks of 4096 words)");
    if (!occupancy_bits || !word_rank || !n_occupied)
        return fail(DDA_ERR_ARG, "dda_occupancy_ranks_static: NULL pointer");
    if (!is_device_ptr(occupancy_bits) || !is_device_ptr(word_rank) || !is_device_ptr(n_occupied))
        return fail(DDA_ERR_ARG, "dda_occupancy_ranks_static: occupancy_bits, word_rank and n_occupied must be "
                                 "device pointers");
    uint32_t* scratch = nullptr;
    if (int rc = static_scan_address(&scratch)) return rc;
    const cudaStream_t st = as_stream(stream);
    const int64_t nwords = (n_sites + 31) / 32;
    const int64_t nblocks = (nwords + kScanTile - 1) / kScanTile;
    const int rem = (int)(n_sites & 31);
    const uint32_t last_mask = rem ? ((1u << rem) - 1u) : 0xffffffffu;
    // every entry of the scratch that the later steps read is written first
    // by this step, so nothing has to be cleared between calls
    k_rank_local_masked<<<(unsigned)nblocks, kScanThreads, 0, st>>>(occupancy_bits, nwords, last_mask, word_rank,
                                                                    scratch);
    DDA_LAUNCH_CHECK("static rank local scan");
    k_rank_blocks<<<1, kScanThreads, 0, st>>>(scratch, nblocks, n_occupied);
    DDA_LAUNCH_CHECK("static rank block scan");
    k_rank_add<<<grid_for(nwords, 256), 256, 0, st>>>(word_rank, nwords, scratch);
    DDA_LAUNCH_CHECK("static rank offsets");
    return DDA_OK;
}
