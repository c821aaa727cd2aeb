// Green's-tensor half spectrum built once per target (OpenDDA Sec. 3).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace dda {

// complex elements of each of the two scratch buffers build_spectrum needs
size_t spectrum_scratch_elems(const Geometry& g);

// Section-1 tensor values -> fused T-to-c + DFT along x, y, z -> half
// spectrum in the layout of spec_index, scaled by 1/(Lx Ly Lz) (FP64 and
// complex64).
int build_spectrum(const Geometry& g, double k, const double2* tw, double2* s0, double2* s1,
                   double2* spec64, float2* spec32, cudaStream_t st);

// the double-float copy of n complex128 spectrum entries (df.cuh)
int spectrum_to_df(const double2* in, cdf* out, size_t n, cudaStream_t st);

// copies the stored spectrum (complex128 if c128, else complex64) to `out`
// in the exported order [Hy][Hx][Hz][6]
int export_spectrum(const Geometry& g, const void* in, void* out, bool c128, cudaStream_t st);

}  // namespace dda
