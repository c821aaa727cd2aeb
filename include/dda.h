/*
 * dda.h -- C ABI of the GB300 DDA hot path: the FFT-accelerated product of
 * the Discrete Dipole Approximation interaction matrix with a vector, the
 * Krylov solves built on it, the bit-fielded target description and the
 * cross sections (Mc Donald, Golden & Jennings, "OpenDDA: a novel
 * high-performance computational framework for the Discrete Dipole
 * Approximation", arXiv:0908.0863).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Units: Gaussian, lattice spacing d = 1, wavenumber k in units of 1/d.
 *   The system solved is  sum_l A_jl P_l = E_inc,j  with A_jj = alpha_j^-1
 *   and, for j != l, r = r_j - r_l,
 *   A_jl = exp(ikr)/r^3 [ k^2 (r r - r^2 I) + (ikr - 1)/r^2 (3 r r - r^2 I) ]
 *   (Eq. 1 with the dyadic product of Eq. 2; the SI prefactor k^2/eps0 and
 *   1/(4 pi) of the paper are absorbed into the unit of P).
 * Lattice: K x J x P sites along x, y, z; site (i, j, k) has linear index
 *   s = (k J + j) K + i, x fastest (App. A), and sits at r = (i, j, k).
 * Occupancy bit field (Sec. 2): uint32 words, site s -> word s >> 5,
 *   bit s & 31 (least significant first); ceil(KJP / 32) words.
 * Composition bit field (Sec. 2): b = max(1, ceil(log2 n_materials)) bits
 *   per field, floor(32 / b) whole fields per uint32 word (none straddles),
 *   field q = 3 s + axis (axis 0, 1, 2 = x, y, z) at word q / f, bit offset
 *   (q % f) * b.  NULL when n_materials == 1.
 * Compressed vectors (Sec. 4, zero storage): [3][N_d] complex, component
 *   major; entry n of each component belongs to the n-th occupied site in
 *   increasing s.  DDA_C128 = interleaved (re, im) doubles, DDA_C64 =
 *   interleaved floats.  Device buffers must be 16-byte aligned.
 * Streams: every call takes a cudaStream_t as void* (NULL = legacy default
 *   stream) and is stream ordered; a context serves one stream at a time
 *   (its scratch is shared by all its calls).
 * Batches: the *_batch entry points take nb right-hand sides that share the
 *   context's spectrum, stored back to back: [nb][3][N_d].  One launch of
 *   each matvec pass covers the whole batch (the batch extension of the
 *   paper's plan reuse, Sec. 5).
 * Ownership: the caller owns every buffer it passes; the context owns its
 *   device state (bit fields, ranks, Green's-tensor spectra, scratch and
 *   solver workspace), allocated by dda_init_lattice (workspace for one
 *   right-hand side in both precisions) and released by dda_free.  The
 *   workspace grows, once, when a call first needs more right-hand sides
 *   (or the first batch in a precision) than it holds; dda_reserve makes
 *   that allocation ahead of time.  Apart from that growth and the scratch
 *   dda_autotune takes and frees, no call allocates device memory.
 * Errors: every int-returning call returns a dda_status; on failure
 *   dda_last_error() gives a message (thread local).  Arguments are
 *   checked before any work is queued; a failed call leaves outputs
 *   unspecified and the context usable unless DDA_ERR_CUDA is returned.
 */
#ifndef DDA_H_
#define DDA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dda_ctx dda_ctx; /* opaque, library owned */

typedef enum {
    DDA_OK = 0,
    DDA_ERR_ARG = -1,            /* bad shape, pointer, size or option      */
    DDA_ERR_CUDA = -2,           /* a CUDA call failed                      */
    DDA_ERR_OOM = -3,            /* device allocation failed                */
    DDA_ERR_NOT_CONVERGED = -4,  /* max_iter reached; last iterate returned */
    DDA_ERR_BREAKDOWN = -5,      /* Krylov breakdown (a zero denominator)   */
    DDA_ERR_NAN = -6             /* non-finite value met                    */
} dda_status;

/* DDA_C128DF: complex128 vectors, the product computed in double-float
 * arithmetic (each real the unevaluated sum of two floats, about 48
 * significant bits, on the FP32 units; tables and spectrum split from the
 * FP64 ones).  A choice of this library for the true residuals of the
 * mixed-precision refinement (dda_residual_dtype); the paper computes in
 * double precision throughout. */
typedef enum { DDA_C128 = 0, DDA_C64 = 1, DDA_C128DF = 2 } dda_dtype;
/* Krylov schemes of Sec. 4 (products with A per iteration in brackets):
 * BiCG [2], BiCGSTAB [2], QMR with coupled two-term recurrences [2],
 * BiCG for complex-symmetric systems "BiCG_sym" [1], CG with the bilinear
 * form x^T y [1] (for a complex-symmetric A the same recurrence as
 * BiCG_sym), CGS [2], TFQMR [2; one iteration = two half-steps], QMR for
 * complex-symmetric systems "QMR_sym" [1] and the restarted, stabilised BiCG
 * "RBiCGSTAB" as BiCGSTAB(l), l = 1, 2, 3 [2 l; one iteration = one cycle of
 * l BiCG steps and a degree-l minimal-residual polynomial, with the stopping
 * test at the end of a cycle], and ML(n)BiCGSTAB (Yeung & Chan 1999), the
 * BiCGSTAB variant with n left Lanczos starting vectors, n = 1, 2, 3 [n + 1;
 * one iteration = one cycle, with the stopping test at its end; n = 1 is
 * BiCGSTAB].  Its starting vectors are r0 and n - 1 pseudo-random vectors
 * whose entry e of vector i is u1 + i u2, u1 and u2 being the first two
 * SplitMix64 outputs from the state i * 2^40 + e mapped to [-1, 1) as
 * (u >> 11) * 2^-52 - 1.  OR DDA_PRECOND_JACOBI into
 * the method for point-Jacobi preconditioning (Sec. 6), applied as the
 * symmetric scaling (S A S) y = S E_inc, P = S y, S = diag(alpha)^(1/2),
 * which keeps the matrix complex symmetric; the stopping test then applies
 * to the scaled residual. */
typedef enum {
    DDA_BICG = 0, DDA_BICGSTAB = 1, DDA_QMR = 2, DDA_BICG_SYM = 3, DDA_CG = 4, DDA_CGS = 5, DDA_TFQMR = 6,
    DDA_QMR_SYM = 7, DDA_RBICGSTAB1 = 8, DDA_RBICGSTAB2 = 9, DDA_RBICGSTAB3 = 10,
    DDA_MLBICGSTAB1 = 11, DDA_MLBICGSTAB2 = 12, DDA_MLBICGSTAB3 = 13
} dda_method;
#define DDA_PRECOND_JACOBI 0x100
typedef enum { DDA_FP64 = 0, DDA_MIXED = 1 } dda_precision;
typedef enum { DDA_POL_CM = 0, DDA_POL_CMRR = 1, DDA_POL_LDR = 2 } dda_polarizability_rule;
/* OR into the rule of dda_polarizability and dda_polarizability_derivative:
 * the input array holds the complex permittivities eps = m^2 instead of the
 * refractive indices m. */
#define DDA_POL_EPS 0x10

typedef struct {
    int iterations;           /* Krylov iterations (inner ones summed, mixed)   */
    int matvecs;              /* products with A in the working precision        */
    int matvecs_fp64;         /* FP64 products (mixed: true-residual products, double-float by default) */
    int refinements;          /* outer refinement steps (mixed), 0 for FP64      */
    double rel_residual;      /* last recurrence residual / ||E_inc||            */
    double rel_residual_true; /* ||E_inc - A P|| / ||E_inc||: FP64 product (mixed: the
                                 refinement's residual product, dda_residual_dtype) */
    double seconds;           /* wall time of the call                           */
} dda_solve_info;

/* ---------------------------------------------------------------- target */

/*
 * Polarisability of each material (host only, no GPU work).  Sec. 1 cites
 * the prescriptions without formulas; they are, with eps = m^2,
 *   CM   : a = (3 / 4pi) (eps - 1) / (eps + 2)
 *   CMRR : a_CM / (1 - (2/3) i k^3 a_CM)                  (Draine 1988)
 *   LDR  : a_CM / (1 + a_CM [(b1 + m^2 b2 + m^2 b3 S) k^2 - (2/3) i k^3]),
 *          b1 = -1.8915316, b2 = 0.1648469, b3 = -1.7700004,
 *          S = sum_a (khat_a e0_a)^2                      (Draine & Goodman 1993)
 * m: [n][2] (re, im), or eps itself when DDA_POL_EPS is OR'd into rule;
 * khat: unit propagation (LDR only, may be NULL otherwise); e0: [3][2]
 * polarisation (LDR only); alpha_out: [n][3][2], the same value on all
 * three axes.  Returns DDA_ERR_ARG for n < 1 or an unknown rule.
 */
int dda_polarizability(int n, const double* m, double k, int rule, const double* khat,
                       const double* e0, double* alpha_out);

/*
 * Pack a per-site occupancy mask into the occupancy bit field (Sec. 2;
 * kernel family (d)).  mask: device uint8[n_sites] (nonzero = occupied);
 * bits: device uint32[ceil(n_sites/32)], fully overwritten (padding bits 0).
 */
int dda_pack_occupancy(const uint8_t* mask, int64_t n_sites, uint32_t* bits, void* stream);

/* Inverse of dda_pack_occupancy: bits -> uint8 mask[n_sites] (0/1), device. */
int dda_unpack_occupancy(const uint32_t* bits, int64_t n_sites, uint8_t* mask, void* stream);

/*
 * Pack per-site, per-axis material indices into the composition bit field
 * (Sec. 2).  materials: device uint8[n_sites][3]; bits: device
 * uint32[ceil(3 n_sites / floor(32/b))].  Indices >= n_materials are
 * rejected on the device: the call then returns DDA_ERR_ARG.
 */
int dda_pack_composition(const uint8_t* materials, int64_t n_sites, int n_materials,
                         uint32_t* bits, void* stream);

/* Inverse of dda_pack_composition: bits -> uint8 materials[n_sites][3], device. */
int dda_unpack_composition(const uint32_t* bits, int64_t n_sites, int n_materials,
                           uint8_t* materials, void* stream);

/*
 * Build a context for one target and wavenumber (Sec. 2-3, App. A).
 *   shape:            {K, J, P}, each in [1, 512].
 *   occupancy_bits:   host or device, layout above.  At least one site occupied.
 *   composition_bits: host or device, or NULL when n_materials == 1.
 *   n_materials:      1..256.
 *   alpha:            host [n_materials][3][2] doubles: polarisability of
 *                     material q acting on axis c (from dda_polarizability or
 *                     the caller's own prescription); must be nonzero, finite.
 *   k:                wavenumber, > 0 and finite.
 * Allocates all device state, ranks the occupied sites (per-word popcount
 * and scan), evaluates the six independent Green's-tensor components on
 * section 1 of the embedding (displacements 0 <= i < K, 0 <= j < J,
 * 0 <= k < P) and transforms them with the fused Toeplitz-to-circulant
 * line DFTs of Sec. 3 (x, then y, then z; mirrored halves signed per
 * Table 1; only L/2 + 1 outputs of each length-L line kept), in FP64, with
 * a complex64 copy.  L per axis = the smallest length >= 2n - 1 of the form
 * 2^a, 3 * 2^a or 5 * 2^a (a >= 3 for the last two): the paper's
 * K'' = 2K - 1 + kf with kf chosen for a fast DFT; dda_query reports it.
 * Returns DDA_ERR_ARG (bad shape, pointers, no occupied site, material
 * index out of range), DDA_ERR_OOM, DDA_ERR_CUDA.  *out is NULL on failure.
 * The call synchronises the stream before returning.
 */
int dda_init_lattice(dda_ctx** out, const int32_t shape[3], const uint32_t* occupancy_bits,
                     const uint32_t* composition_bits, int n_materials, const double* alpha,
                     double k, void* stream);

/* Release every device resource of the context (NULL is a no-op). */
void dda_free(dda_ctx* ctx);

/*
 * Sizes of a context: occupied sites N_d, padded grid {Lx, Ly, Lz} and the
 * device bytes the context holds.  Any output pointer may be NULL.
 */
int dda_query(const dda_ctx* ctx, int64_t* n_dipoles, int32_t padded[3], int64_t* device_bytes);

/*
 * Compressed index of every site: rank[s] = number of occupied sites before
 * s (device uint32[KJP]), as the matvec uses it.  Diagnostic entry point
 * for the bit-exact tests of the occupancy kernels.
 */
int dda_site_ranks(const dda_ctx* ctx, uint32_t* rank, void* stream);

/*
 * Copy the stored half spectrum of the six tensor components, scaled by
 * 1 / (Lx Ly Lz): device complex [Ly/2+1][Lx/2+1][Lz/2+1][6] of the given
 * dtype (the storage order: z lines contiguous, components xx, xy, xz, yy,
 * yz, zz innermost).  Diagnostic entry point (parity of the init step).
 */
int dda_tensor_spectrum(const dda_ctx* ctx, void* out, int dtype, void* stream);

/* ------------------------------------------------------------ hot path */

/*
 * y = A p (Eq. 1) by the pruned FFT algorithm of Sec. 3: expand the
 * compressed vector (Sec. 4) into the K x J'' x P y-line array and
 * transform along y (K P lines), transform along x (J'' P lines), then per
 * z-line forward DFT, the 3 x 3 symmetric spectrum product of Eqs. 6-8
 * with the signed mirror lookup, and inverse DFT keeping k < P; inverse
 * along x keeping i < K, inverse along y keeping j < J, add alpha^-1 p and
 * compress.  p, y: device [3][N_d] complex of the given dtype; p and y may
 * not overlap.  DDA_C64 runs every step in complex FP32 with the complex64
 * spectrum; DDA_C128DF takes complex128 p and y and runs every step in
 * double-float arithmetic (relative error about 1e-13 against 1e-15 for
 * DDA_C128).  Returns DDA_ERR_ARG for NULL or host pointers.
 */
int dda_matvec(dda_ctx* ctx, const void* p, void* y, int dtype, void* stream);

/*
 * y_b = A p_b for nb right-hand sides (1 <= nb <= 4096) at once: p, y are
 * device [nb][3][N_d] complex of the given dtype and may not overlap.  Every
 * pass of dda_matvec runs once over the batch (in chunks when the work
 * space holds fewer complex128 slots than nb), reading the shared spectrum
 * once per tile for all right-hand sides.  Results equal nb calls of
 * dda_matvec bit for bit.  May grow the workspace (see Ownership).
 */
int dda_matvec_batch(dda_ctx* ctx, int nb, const void* p, void* y, int dtype, void* stream);

/*
 * Tile settings of the matvec passes for dtype DDA_C128 or DDA_C64, as host
 * int[4]: tiles[0] = log2 of the y lines (adjacent x columns) one CTA
 * transforms in P1/P5, tiles[1] = log2 of the whole z columns one CTA
 * transforms in P3, tiles[2] = log2 of the x lines (consecutive z planes)
 * one CTA transforms and transposes in P2/P4; tiles[3] is reserved and
 * must be 0.  tiles_in (may be NULL) sets them after checking the launch
 * limits (threads per block, shared memory; DDA_ERR_ARG when exceeded);
 * tiles_out (may be NULL) receives the current ones.  The settings only
 * regroup lines between CTAs: every line's arithmetic, and so every result
 * bit, is the same for all valid settings.
 */
int dda_tiles(dda_ctx* ctx, int dtype, int* tiles_out, const int* tiles_in);

/*
 * Autotune the tile settings of dtype on this context: starting from the
 * current ones, try P3 widths up to two steps either way of the current
 * one, then the same for P1/P5 and for P2/P4, timing `reps` batched
 * products of nb right-hand sides per candidate with CUDA events (after
 * one untimed product), and keep the fastest.  Last, against timing noise
 * between those steps, the chosen and the starting settings are timed
 * alternately three times each; the chosen ones stay unless the median
 * whole product of the starting ones is more than 1% faster.  The choice
 * is set on the context and remembered for the process: contexts created
 * later with the same lattice shape start with it.  pass_ms (host
 * double[5], may be NULL) receives the per-pass milliseconds of the chosen
 * widths.  Allocates (and frees) two scratch vectors of nb right-hand
 * sides; may grow the workspace to nb slots.  Synchronises the stream.
 */
int dda_autotune(dda_ctx* ctx, int dtype, int nb, int reps, double* pass_ms, void* stream);

/*
 * Mixed precision (DDA_MIXED): every inner complex64 solve aims at the
 * relative residual max(0.3 tol / rho_now, 1e-6, rho), rho_now being the
 * refinement's current relative residual: by default (rho = 0) one inner
 * solve reaches the final tolerance, a larger rho (in (0, 1)) stops each
 * inner solve after that reduction and lets the FP64 refinement take more
 * steps.  Each Krylov method has its own rho (a method that restarts
 * badly, such as QMR, loses by the extra refinements that suit BiCGSTAB);
 * method is a dda_method value (the Jacobi flag is ignored).  rho_in (host,
 * may be NULL) sets rho of that method, rho_out (host, may be NULL)
 * receives it.  DDA_ERR_ARG for an unknown method or rho outside [0, 1).
 * This is a choice of this library (the paper runs one precision only).
 */
int dda_inner_tolerance(dda_ctx* ctx, int method, const double* rho_in, double* rho_out);

/*
 * Products of the true residuals r = einc - A x in the mixed-precision
 * refinement (dda_solve, dda_solve_batch with DDA_MIXED): DDA_C128DF
 * (default: double-float products, about 48 significant bits, a few times
 * faster than FP64 on this GPU, whose FP64 rate is a small fraction of its
 * FP32 rate) or DDA_C128 (FP64 products).  The double-float product is
 * accurate to about 1e-13 relative to |A||x|, so residual tolerances down
 * to about 1e-11 behave as with FP64 products.  dtype_in (host, may be
 * NULL) sets the choice, dtype_out (host, may be NULL) receives it.  The
 * FP64 solves always use FP64 products.  DDA_ERR_ARG for another dtype.
 * This is a choice of this library (the paper runs one precision only).
 */
int dda_residual_dtype(dda_ctx* ctx, const int* dtype_in, int* dtype_out);

/*
 * Tune rho of dda_inner_tolerance for one method on this context: solve
 * A P = einc (host or device [3][N_d] complex128) in mixed precision to tol
 * with the given method for rho = 0, 1e-4, 1e-3, 1e-2, 3e-2 and 1e-1,
 * timing each solve with CUDA events, and keep the fastest that converged;
 * rho = 0 stays unless another candidate is faster by more than 2% (the
 * noise of one timing is about 1%).  The choice is set on the context for
 * that method and remembered for the process: contexts created later with
 * the same lattice shape start with it for that method.  rho_out (host, may
 * be NULL) receives it, ms_out (host double[6], may be NULL) the solve times
 * (-1: not converged).  Allocates and frees one scratch solution;
 * synchronises.  DDA_ERR_NOT_CONVERGED when no candidate converged.
 */
int dda_autotune_inner(dda_ctx* ctx, const void* einc, int method, double tol, int max_iter, double* rho_out,
                       double* ms_out, void* stream);

/*
 * Grow the solve workspace to hold nb right-hand sides (1 <= nb <= 4096)
 * for solves of the given precision, so that later calls with up to nb
 * right-hand sides allocate nothing.  Per right-hand side it holds 3
 * complex128 vectors of 3 N_d, one complex64 matvec work slot (2 for the
 * first) and 12 complex128 (DDA_FP64) or 14 complex64 (DDA_MIXED) Krylov
 * vectors; dda_query reports the total.  DDA_ERR_OOM when it does not fit.
 */
int dda_reserve(dda_ctx* ctx, int nb, int precision);

/*
 * Incident plane wave at the occupied sites: E_c = e0_c exp(i k khat . r),
 * r = (i, j, k) (phase origin at site 0).  khat: host unit vector[3];
 * e0: host [3][2]; einc: device [3][N_d] complex128.
 */
int dda_incident_field(dda_ctx* ctx, const double* khat, const double* e0, void* einc, void* stream);

/*
 * Solve A P = E_inc (Sec. 4) with BiCG, BiCGSTAB or QMR, unpreconditioned.
 *   einc, p: host or device [3][N_d] complex128.  p is read as the starting
 *            guess when use_x0 != 0, else the start is 0 (Sec. 6); on return
 *            it holds the last iterate.
 *   precision: DDA_FP64 runs everything in FP64.  DDA_MIXED runs an outer
 *            FP64 iterative refinement: r = E_inc - A P with the
 *            double-float (default) or FP64 product (dda_residual_dtype),
 *            an inner complex64 Krylov solve of A d = r / ||r||
 *            (complex64 products and vectors, FP64 inner products and
 *            scalars), P += ||r|| d, until ||r|| <= tol ||E_inc||.
 *   tol:      relative residual target (> 0); max_iter: cap on Krylov
 *             iterations (summed over inner solves for DDA_MIXED).
 *   info:     host, may be NULL.
 * Stopping rule: ||r||_2 <= tol ||E_inc||_2 on the recurrence residual
 * (BiCGSTAB also stops half way on ||s||); info->rel_residual_true is then
 * recomputed with one FP64 product (DDA_MIXED: it is the refinement's own
 * true residual).  Returns DDA_OK, DDA_ERR_NOT_CONVERGED
 * (max_iter reached, p = last iterate), DDA_ERR_BREAKDOWN, DDA_ERR_NAN,
 * DDA_ERR_ARG.  Synchronises the stream.
 */
int dda_solve(dda_ctx* ctx, const void* einc, void* p, int method, int precision, double tol,
              int max_iter, int use_x0, dda_solve_info* info, void* stream);

/*
 * dda_solve for nb right-hand sides with the same matrix (incidence
 * directions and polarisations of one target), solved in lock step: every
 * Krylov kernel and matvec pass covers all of them, each right-hand side
 * keeps its own scalars, stopping test and iteration count, and one that
 * has finished is skipped by all later kernels.  Iterations after the first
 * of each Krylov solve are replayed from a CUDA graph (unless dda_profile
 * is on).  In the mixed form each right-hand side has its own refinement
 * steps and inner tolerances.
 *   einc, p: host or device [nb][3][N_d] complex128 (as in dda_solve).
 *   info: host dda_solve_info[nb] or NULL; status: host int[nb] or NULL,
 *         each right-hand side's dda_status.
 * Returns DDA_ERR_ARG / CUDA / OOM for a failed call, else the most severe
 * per-right-hand-side status (NAN, then BREAKDOWN, then NOT_CONVERGED).
 * May grow the workspace (see Ownership).
 */
int dda_solve_batch(dda_ctx* ctx, int nb, const void* einc, void* p, int method, int precision, double tol,
                    int max_iter, int use_x0, dda_solve_info* info, int* status, void* stream);

/*
 * Cross sections with |E0| = 1 (Draine 1988; values only in Table 7):
 *   C_ext = 4 pi k sum_j Im(E_inc,j^* . P_j)
 *   C_abs = 4 pi k sum_j sum_c [-Im(alpha^-1_jc) - (2/3) k^3] |P_jc|^2
 *   C_sca = C_ext - C_abs.
 * einc, p: host or device [3][N_d] complex128; out: host double[3] =
 * {C_ext, C_abs, C_sca}.  FP64 reductions in a fixed order (deterministic).
 * Synchronises the stream.
 */
int dda_cross_sections(dda_ctx* ctx, const void* einc, const void* p, double* out, void* stream);

/* dda_cross_sections for nb right-hand sides: einc, p host or device
 * [nb][3][N_d] complex128, out host double[nb][3]. */
int dda_cross_sections_batch(dda_ctx* ctx, int nb, const void* einc, const void* p, double* out, void* stream);

/*
 * Occupancy rank scan that allocates no device memory.  This entry point
 * has no counterpart in the paper; it exists for callers that cannot call
 * cudaMalloc: code whose device memory all belongs to another framework's
 * pooling allocator, code that must not allocate once it is running (a
 * latency-bound service loop), or a host thread that does not own the
 * allocation policy of the process.  It computes what dda_init_lattice
 * computes internally: word_rank[w] = number of occupied sites in words
 * 0..w-1 of the occupancy bit field (so the compressed index of an occupied
 * site s is word_rank[s >> 5] + popcount(bits[s >> 5] & ((1 << (s & 31)) - 1)))
 * and *n_occupied = N_d.
 *   occupancy_bits: device uint32[ceil(n_sites/32)], layout above; read
 *                   only (padding bits past n_sites are ignored).
 *   word_rank:      device uint32[ceil(n_sites/32)], written.
 *   n_occupied:     device uint32[1], written.
 * A NULL pointer, or one that is not device (or managed) memory, returns
 * DDA_ERR_ARG before any work is queued.
 * The scan keeps its per-block totals in a 16 KB array inside the library
 * (a file-scope __device__ array, one per GPU, held until the process
 * exits), which limits n_sites to 536,870,912 (4096 x 4096 x 32); larger
 * inputs return DDA_ERR_ARG before any work is queued.  The first call on
 * a device looks up that array's device address (once per device, with
 * the device current); make that first call before any stream capture.
 * All calls share the array: each call writes every entry it later reads,
 * so no state carries over, but calls that overlap on the GPU (on
 * different streams or from different threads) race on it -- order them
 * on one stream.  Stream ordered; no synchronisation.
 */
int dda_occupancy_ranks_static(const uint32_t* occupancy_bits, int64_t n_sites, uint32_t* word_rank,
                               uint32_t* n_occupied, void* stream);

/* -------------------------------------------------------------- tracing */

/*
 * Per-pass timing of the matvec (the paper reports per-component times,
 * Sec. 6 and Tables 4 and 6).  enable != 0: every later product of this
 * context (dda_matvec and the products inside dda_solve) records a CUDA
 * event pair around each of its five passes on the calling stream;
 * enable == 0 stops and drops what was recorded.
 */
int dda_profile(dda_ctx* ctx, int enable);

/*
 * Wait for the recorded events and return, for dtype d (0 = complex128,
 * 1 = complex64) and pass q (0..4 = P1..P5 of dda_matvec), the launch
 * count counts[d*5 + q] and the summed device milliseconds ms[d*5 + q];
 * the records are then cleared.  counts, ms: host arrays of 10.
 */
int dda_profile_read(dda_ctx* ctx, int64_t* counts, double* ms);

/* Kernel launches issued by the library since it was loaded (all threads). */
int64_t dda_launch_count(void);

/* ------------------------------------------- observables and gradients */

/*
 * C_sca as the exact pair sum of the power the dipoles radiate (Draine
 * 1988; the paper prints only the values, Table 7), independent of C_ext
 * and C_abs: C_sca = 4 pi k sum_j [(2/3) k^3 |P_j|^2 + P_j^H sum_{l!=j}
 * Im(G_jl) P_l], with G = diag(alpha^-1) - A the dipole field tensor.  For
 * an exact solution C_ext = C_abs + C_sca (optical theorem).  Computed with
 * two FP64 products, A P and A^H P.  p: host or device [3][N_d] complex128;
 * out: host double[1].  Synchronises the stream.
 */
int dda_scattering_cross_section(dda_ctx* ctx, const void* p, double* out, void* stream);

/*
 * d(alpha^-1)/d eps for each material, eps = m^2, for the prescriptions of
 * dda_polarizability (host only): -4 pi/(eps - 1)^2 for CM and CMRR, plus
 * (b2 + b3 S) k^2 for LDR.  Same arguments and output layout as
 * dda_polarizability ([n][3][2]); DDA_ERR_ARG for m = 1.
 */
int dda_polarizability_derivative(int n, const double* m, double k, int rule, const double* khat,
                                  const double* e0, double* dalpha_inv_out);

/*
 * Per-material sums of a per-dipole complex field: out[q] = sum of v_j over
 * the occupied sites j whose composition field of axis x holds material q
 * (all dipoles are material 0 without composition bits).  With v =
 * dda_gradient's g this is the chain rule from per-dipole permittivities
 * to one permittivity per material, dC/deps_q (all dipoles of a material
 * share its eps).  The paper has no gradient; this is the last step of the
 * adjoint gradient of dda_gradient.
 *   v:   host or device [N_d] complex128, compressed order.
 *   out: host double[n_materials][2] (re, im).
 * At most 32 materials (DDA_ERR_ARG beyond).  Fixed summation order (the
 * same bits on every call).  Synchronises the stream.
 */
int dda_material_sums(dda_ctx* ctx, const void* v, double* out, void* stream);

/*
 * Gradient of C_ext (which = 0) or C_abs (which = 1) with respect to the
 * complex permittivity eps_j of every dipole, g_j = dC/dRe(eps_j) +
 * i dC/dIm(eps_j), the three axes of a dipole sharing eps_j.  Adjoint
 * method: one extra solve with the same matrix (A^T = A, Sec. 3), of
 * A mu = W conj(P) (C_abs, W = -Im(alpha^-1) - (2/3) k^3) or A mu = conj(E)
 * (C_ext), then per dipole S = sum_c mu_c a'_c P_c and
 *   C_abs: g = 4 pi k (sum_c -|P_c|^2 Im a'_c - 2 Re S) + i 4 pi k (sum_c -|P_c|^2 Re a'_c + 2 Im S)
 *   C_ext: g = 4 pi k (-Im S) + i 4 pi k (-Re S)
 * with a' from dalpha_inv.  Only P is needed from the forward solve; no
 * Krylov iterate is stored.
 *   einc: host or device [3][N_d] complex128 (read for which = 0 only).
 *   p: host or device [3][N_d] complex128, the solution of A P = E_inc.
 *   dalpha_inv: host [n_materials][3][2] (dda_polarizability_derivative).
 *   method, precision, tol, max_iter: of the adjoint solve (dda_solve).
 *   grad: host or device [N_d] complex128, compressed order.
 *   info: host, may be NULL (the adjoint solve's).
 * Returns the adjoint solve's status (DDA_OK, DDA_ERR_NOT_CONVERGED, ...);
 * grad is written in every case but DDA_ERR_ARG / DDA_ERR_CUDA / DDA_ERR_OOM.
 */
int dda_gradient(dda_ctx* ctx, int which, const void* einc, const void* p, const double* dalpha_inv, int method,
                 int precision, double tol, int max_iter, void* grad, dda_solve_info* info, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* dda_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DDA_H_ */
