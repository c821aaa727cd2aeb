// Sequencing of the pruned FFT matrix-vector product y = A p (OpenDDA
// Sec. 3): tile configuration, batch chunking and the five passes, whose
// kernels live in matvec_kernels.cuh (one translation unit per pass).
#include "matvec_kernels.cuh"

namespace dda {

template <typename T>
bool tiles_ok(const Geometry& g, int logW_y, int logW_z, int logW_x) {
    const int elt = sizeof(C<T>);
    const int ty = line_threads(g.Ly), tz = p3_col_threads(g.Lz);
    if (logW_y < 0 || logW_z < 0 || logW_x < 0) return false;
    if (logW_y > kMaxLogW || logW_z > kMaxLogR || logW_x > kMaxLogZ) return false;
    if ((1 << logW_y) * ty > kYThreads || 3ull * col_elems(g.Ly, 1 << logW_y) * elt > 200 * 1024) return false;
    if ((1 << logW_z) * tz > p3_max_threads<T>(g.Lz) ||
        3ull * (1ull << logW_z) * row_ld(g.Lz, p3_line_threads(g.Lz)) * elt > 200 * 1024)
        return false;
    const bool c128 = sizeof(T) == 8;
    if (rows_groups(g.Lx, 1 << logW_x, c128) * (1 << logW_x) * map_threads(g.Lx, c128) > rows_max_threads(g.Lx, c128) ||
        rows_smem_elems(g.Lx, 1 << logW_x, c128) * elt > 200 * 1024)
        return false;
    return true;
}

template <typename T>
void configure_matvec(MatvecView<T>& mv) {
    const Geometry& g = mv.g;
    const int elt = sizeof(C<T>);
    const int ty = line_threads(g.Ly), tz = p3_col_threads(g.Lz);
    // P1/P5: W adjacent columns (64-byte rows)
    int wy = floor_log2(64 / elt);
    while (wy > 0 && (1 << wy) * ty > kYThreads) --wy;
    while (wy > 0 && 3ull * col_elems(g.Ly, 1 << wy) * elt > 200 * 1024) --wy;   // P1's three regions
    while (wy > 0 && (1 << (wy - 1)) >= g.K) --wy;          // no wider than the lattice
    // P3: the fewest whole columns per CTA that fill at least two warps
    // exactly (small independent CTAs, many per SM)
    int wz = 0;
    while (wz < kMaxLogR && (((1 << wz) * tz) < 64 || (((1 << wz) * tz) & 31)) &&
           (2 << wz) * tz <= p3_max_threads<T>(g.Lz) && (1 << wz) < g.Lx)
        ++wz;
    // P2/P4: 32 bytes of each column of Bxy per CTA (4 complex64 or 2
    // complex128 consecutive z lines): whole sectors with small CTAs, which
    // measured faster than 64- or 128-byte tiles with larger CTAs
    int wx = floor_log2(32 / elt);
    while (wx > 0 && !tiles_ok<T>(g, wy, wz, wx)) --wx;
    while (wx > 0 && (1 << (wx - 1)) >= g.P) --wx;
    mv.logW_y = wy;
    mv.logW_z = wz;
    mv.logW_x = wx;
}
template <typename T>
static int launch_chunk(const MatvecView<T>& mv, const C<IO<T>>* p, C<IO<T>>* y, cudaStream_t st) {
    const int dt = sizeof(T) == 8 ? 0 : 1;
    PassProfiler* pf = (mv.prof && mv.prof->on) ? mv.prof : nullptr;
    int rc;
    if (pf) pf->begin(dt, 0, st);
    if ((rc = pass1<T>(mv, p, st))) return rc;
    if (pf) { pf->end(st); pf->begin(dt, 1, st); }
    if ((rc = pass_rows<T, false>(mv, st))) return rc;
    if (pf) { pf->end(st); pf->begin(dt, 2, st); }
    if ((rc = pass3<T>(mv, st))) return rc;
    if (pf) { pf->end(st); pf->begin(dt, 3, st); }
    if ((rc = pass_rows<T, true>(mv, st))) return rc;
    if (pf) { pf->end(st); pf->begin(dt, 4, st); }
    if ((rc = pass5<T>(mv, p, y, st))) return rc;
    if (pf) pf->end(st);
    return 0;
}

template <typename T>
int launch_matvec(const MatvecView<T>& mv, const C<IO<T>>* p, C<IO<T>>* y, cudaStream_t st) {
    if (mv.nb < 1 || mv.slots < 1) return fail(DDA_ERR_ARG, "matvec: empty batch");
    for (int b0 = 0; b0 < mv.nb; b0 += mv.slots) {
        MatvecView<T> m = mv;
        m.b0 = b0;
        m.nb = mv.nb - b0 < mv.slots ? mv.nb - b0 : mv.slots;
        if (int rc = launch_chunk<T>(m, p, y, st)) return rc;
    }
    return 0;
}

template <typename T> int pass3(const MatvecView<T>& mv, cudaStream_t st) {
    DDA_LEN_SWITCH(mv.g.Lz, (p3_len<T, LN>(mv, st)))
}
template int pass3<double>(const MatvecView<double>&, cudaStream_t);
template int pass3<float>(const MatvecView<float>&, cudaStream_t);
template int pass3<DF>(const MatvecView<DF>&, cudaStream_t);

template void configure_matvec<double>(MatvecView<double>&);
template void configure_matvec<float>(MatvecView<float>&);
template void configure_matvec<DF>(MatvecView<DF>&);
template bool tiles_ok<double>(const Geometry&, int, int, int);
template bool tiles_ok<float>(const Geometry&, int, int, int);
template bool tiles_ok<DF>(const Geometry&, int, int, int);
template int launch_matvec<double>(const MatvecView<double>&, const C<double>*, C<double>*, cudaStream_t);
template int launch_matvec<float>(const MatvecView<float>&, const C<float>*, C<float>*, cudaStream_t);
template int launch_matvec<DF>(const MatvecView<DF>&, const C<double>*, C<double>*, cudaStream_t);

}  // namespace dda
