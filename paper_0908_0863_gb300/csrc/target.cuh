// Bit fields, ranks, incident field and cross-section sums (OpenDDA Sec. 2, 4).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace dda {

inline int composition_bits(int nmat) {
    int b = 1;
    while ((1 << b) < nmat) ++b;
    return b;
}

int launch_pack_occupancy(const uint8_t* mask, int64_t n, uint32_t* bits, cudaStream_t st);
int launch_unpack_occupancy(const uint32_t* bits, int64_t n, uint8_t* mask, cudaStream_t st);
// *bad_host = 1 when an index >= nmat was met (synchronises the stream)
int launch_pack_composition(const uint8_t* mats, int64_t nsites, int nmat, uint32_t* bits, int* bad_host,
                            cudaStream_t st);
int launch_unpack_composition(const uint32_t* bits, int64_t nsites, int nmat, uint8_t* mats, cudaStream_t st);
int launch_check_composition(const uint32_t* bits, int64_t nsites, int nmat, int* bad, cudaStream_t st);

// words of scratch launch_ranks needs (block totals)
size_t rank_scratch_words(int64_t nwords);
// rank[w] = occupied sites in words before w; *total = all occupied sites (device)
int launch_ranks(const uint32_t* occ, int64_t nwords, uint32_t* rank, uint32_t* scratch, uint32_t* total,
                 cudaStream_t st);
int launch_site_ranks(const TargetView& tv, int64_t n, uint32_t* out, cudaStream_t st);

int launch_incident(const TargetView& tv, const Geometry& g, double k, const double* khat, const double* e0,
                    double2* E, cudaStream_t st);

size_t xsec_scratch_elems();
// scratch[xsec_scratch_elems()-1] receives {sum Im(E^* P), sum [-Im ainv - 2/3 k^3] |P|^2}
int launch_cross_sections(const TargetView& tv, const Geometry& g, double k, const double2* ainv,
                          const double2* E, const double2* P, double2* scratch, cudaStream_t st);

// C_sca by the exact pair sum from P, A P and A^H P; the sum lands in
// scratch[xsec_scratch_elems()-1].x (without the 4 pi k factor)
int launch_csca(const TargetView& tv, const Geometry& g, double k, const double2* ainv, const double2* P,
                const double2* AP, const double2* AhP, double2* scratch, cudaStream_t st);
// which: 0 = C_ext, 1 = C_abs
int launch_adjoint_rhs(const TargetView& tv, const Geometry& g, double k, int which, const double2* ainv,
                       const double2* E, const double2* P, double2* out, cudaStream_t st);
int launch_gradient(const TargetView& tv, const Geometry& g, double k, int which, const double2* dainv,
                    const double2* P, const double2* mu, double2* grad, cudaStream_t st);

// out[q] = sum of v[rank(s)] over the occupied sites s of material q (axis
// x field), q < g.nmat <= kMaxSumMaterials; scratch: at least
// material_sums_scratch_elems(g) elements; out may alias scratch
constexpr int kMaxSumMaterials = 32;
size_t material_sums_scratch_elems(const Geometry& g);
int launch_material_sums(const TargetView& tv, const Geometry& g, const double2* v, double2* out, cudaStream_t st);

// Point-Jacobi scaling (Sec. 6): vec[b][c][rank(s)] *= tab[material(s, c)][c]
// (or /= with inverse) for every occupied site s and right-hand side b < nb
// (vectors of stride elements); tab = diag(A)^(-1/2) per material and axis
template <typename T>
int launch_site_scale(const TargetView& tv, const Geometry& g, const C<T>* tab, C<T>* vec, int nb, int64_t stride,
                      int inverse, cudaStream_t st);

}  // namespace dda
