// Device-resident Krylov solvers (OpenDDA Sec. 4) and their vector kernels.
#pragma once

#include "common.cuh"
#include "matvec.cuh"

namespace dda {

// scalar slots of the device solver state
enum Slot {
    S_RHO = 0, S_RHO_OLD, S_ALPHA, S_BETA, S_OMEGA, S_SIGMA,  // BiCG / BiCGSTAB
    S_DELTA, S_EPS, S_XI, S_RHOQ, S_GAMMA_OLD, S_THETA_OLD, S_ETA, S_F,  // QMR
    S_NCP, S_NCQ,                                    // QMR: -(xi delta/eps), -(rho delta/eps)
    S_RHO_NEW, S_XI_NEW, S_TMP, S_NSLOTS
};

enum Status { ST_RUN = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_NAN = 3, ST_HALF = 4 };

struct KState {
    double2 s[S_NSLOTS];
    double bnorm2;   // ||b||^2
    double tol2;     // tol^2
    double rel2;     // last ||r||^2 / ||b||^2 (recurrence)
    int status;
    int iter;        // completed iterations
    int matvecs;
};

constexpr int kVecBlocks = 152 * 4;
constexpr int kVecThreads = 256;
constexpr int kMaxRed = 4;

// Workspace of one solver precision (vectors of n = 3 N_d elements).
template <typename T>
struct KrylovWork {
    int64_t n;
    C<T>* v[12];          // solver vectors
    double2* part;        // [kVecBlocks][kMaxRed] partial sums
    KState* st;           // device state
};

struct SolveResult {
    int status;
    int iterations;
    int matvecs;
    double rel2;
};

// Runs one Krylov solve A x = b in precision T on device buffers.
//   x: in (start if use_x0) / out; b: right-hand side.  Both length n.
//   mv: matvec of precision T (its status pointer is set to ws.st->status).
// Host polls the device status every few iterations; never blocks on the
// device except for those polls.
template <typename T>
int krylov_solve(int method, MatvecView<T> mv, KrylovWork<T>& ws, const C<T>* b, C<T>* x, bool use_x0,
                 double tol, int max_iter, KState* host_state, cudaStream_t st, SolveResult* res);

// vector helpers used by the refinement loop and the API
int vec_norm2_c128(const double2* a, int64_t n, double2* part, KState* st_dev, double* out_host,
                   KState* host_state, cudaStream_t st);
// r = b - r  (r holds A x on entry), partial ||r||^2 reduced into st->s[S_TMP].x
int residual_from_product(const double2* b, double2* r, int64_t n, double2* part, KState* st_dev, cudaStream_t st);
// out32 = (float)(r * scale)
int scale_to_c64(const double2* r, double scale, float2* out, int64_t n, cudaStream_t st);
// x += scale * (double)d
int axpy_from_c64(double2* x, double scale, const float2* d, int64_t n, cudaStream_t st);
int vec_copy_c128(double2* dst, const double2* src, int64_t n, cudaStream_t st);
int reduce_into_slot(const double2* part, int nr, KState* st_dev, int slot, cudaStream_t st);

}  // namespace dda
