// Device-resident Krylov solvers (OpenDDA Sec. 4) and their vector kernels,
// for a batch of right-hand sides that share one matrix.
#pragma once

#include "common.cuh"
#include "matvec.cuh"

namespace dda {

// scalar slots of the device solver state
enum Slot {
    S_RHO = 0, S_RHO_OLD, S_ALPHA, S_BETA, S_OMEGA, S_SIGMA,  // BiCG / BiCGSTAB
    S_DELTA, S_EPS, S_XI, S_RHOQ, S_GAMMA_OLD, S_THETA_OLD, S_ETA, S_F,  // QMR
    S_NCP, S_NCQ,                                    // QMR: -(xi delta/eps), -(rho delta/eps)
    S_RHO_NEW, S_XI_NEW, S_TMP,
    S_TAU, S_THETA, S_CD,                            // TFQMR: tau, theta, theta^2 eta / alpha
    S_G1, S_G2, S_G3,                                // BiCGSTAB(ell): minimal-residual coefficients
    S_ML,                                            // ML(n)BiCGSTAB: M = Q^H dR (n x n, column j at
                                                     // S_ML + 3 j), then f = Q^H r (S_ML + 9), c
                                                     // (S_ML + 12), omega (S_ML + 15), oldest column (S_ML + 16)
    S_NSLOTS = S_ML + 17
};

// ST_RUN must stay 0: the matvec passes skip a right-hand side whose status
// word is nonzero
enum Status { ST_RUN = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_NAN = 3, ST_HALF = 4, ST_MAXIT = 5 };

// solver state of one right-hand side
struct KState {
    double2 s[S_NSLOTS];
    double bnorm2;   // ||b||^2
    double tol2;     // tol^2
    double rel2;     // last ||r||^2 / ||b||^2 (recurrence)
    int status;
    int iter;        // completed iterations
    int matvecs;
    int maxit;       // iteration cap of this right-hand side
};
static_assert(sizeof(KState) % sizeof(int) == 0, "status stride");
constexpr int kStateInts = (int)(sizeof(KState) / sizeof(int));

// per right-hand side controls of a batched solve (device array, one per RHS)
struct RhsCtl {
    double tol;     // Krylov stopping tolerance (<= 0: the solve leaves this RHS alone)
    double scale;   // refinement: complex64 right-hand side = scale * residual
    double mult;    // refinement: x += mult * correction (0: no update)
    int maxit;      // Krylov iteration cap
    int skip;       // refinement: 1 = leave this RHS's residual alone
};
static_assert(sizeof(RhsCtl) % sizeof(int) == 0, "skip stride");
constexpr int kCtlInts = (int)(sizeof(RhsCtl) / sizeof(int));

constexpr int kVecBlocks = 152 * 4;   // blocks of one vector kernel over the whole batch
constexpr int kVecThreads = 256;
constexpr int kVecUnroll = 4;         // elements per thread per grid step
constexpr int kMaxRed = 10;         // partial sums per block (BiCGSTAB(3)'s Gram entries: 9)

// blocks per right-hand side of the vector kernels: enough to cover n with
// one grid step, at most kVecBlocks in total over the batch, at least one
inline int vec_blocks(int64_t n, int nb) {
    const int64_t need = (n + (int64_t)kVecThreads * kVecUnroll - 1) / ((int64_t)kVecThreads * kVecUnroll);
    const int64_t share = (kVecBlocks + nb - 1) / nb;
    const int64_t g = need < share ? need : share;
    return g < 1 ? 1 : (int)g;
}

// Workspace of one solver precision: nb right-hand sides of n = 3 N_d
// elements each, every vector stored as [nb][n].
template <typename T>
struct KrylovWork {
    int64_t n = 0;
    int nb = 1;
    C<T>* v[12] = {};     // solver vectors
    double2* part = nullptr;  // [nb][vec_blocks(n, nb)][kMaxRed] partial sums
    KState* st = nullptr;     // [nb] device state
    KState* host = nullptr;   // [nb] pinned copy (results)
    int* host_status = nullptr;  // [2][nb] pinned status polls
    cudaStream_t capture = nullptr;  // non-blocking stream for graph capture (null: no graphs)
};

struct SolveResult {
    int status;
    int iterations;
    int matvecs;
    double rel2;
};

// Runs the Krylov solves A x_b = b_b of all ws.nb right-hand sides in
// precision T on device buffers ([nb][n] each).  Right-hand side b stops at
// ctl[b].tol after at most ctl[b].maxit iterations (ctl: device array; a
// tolerance <= 0 leaves the RHS untouched) or, when ctl is null, at tol
// after at most max_iter iterations.
//   mv: matvec of precision T; its batch fields are set here.
// The host polls the device status words every iteration, two iterations
// behind, and never blocks inside an iteration.  Iterations after the first
// are replayed from a CUDA graph when ws.capture is set and the pass
// profiler is off.  res: [nb].
template <typename T>
int krylov_solve(int method, MatvecView<T> mv, KrylovWork<T>& ws, const C<T>* b, C<T>* x, bool use_x0,
                 const RhsCtl* ctl, double tol, int max_iter, cudaStream_t st, SolveResult* res);

// ---- batched vector helpers of the refinement loop (nb right-hand sides
// of n elements, KState st_dev[nb], partial buffer part)
// r_b = b_b - r_b (r holds A x on entry) for RHS with ctl[b].skip == 0 (ctl
// may be null: all); ||r_b||^2 into st_dev[b].s[S_TMP].x
int residual_from_product(const double2* b, double2* r, int64_t n, int nb, const RhsCtl* ctl, double2* part,
                          KState* st_dev, cudaStream_t st);
// ||a_b||^2 into st_dev[b].s[S_TMP].x
int vec_norm2_c128(const double2* a, int64_t n, int nb, double2* part, KState* st_dev, cudaStream_t st);
// copies st_dev[b].s[S_TMP].x of every RHS to out[b] (host); synchronises the stream
int read_tmp_slots(const KState* st_dev, int nb, KState* host, double* out, cudaStream_t st);
// out32_b = (float)(r_b * ctl[b].scale)
int scale_to_c64(const double2* r, const RhsCtl* ctl, float2* out, int64_t n, int nb, cudaStream_t st);
// x_b += ctl[b].mult * (double)d_b where ctl[b].mult != 0
int axpy_from_c64(double2* x, const RhsCtl* ctl, const float2* d, int64_t n, int nb, cudaStream_t st);

// launch counting while a graph is captured: launches are added to *sink
// instead of the global count (null ends it)
void capture_launches_into(int64_t* sink);

}  // namespace dda
