// Device-resident Krylov solvers (OpenDDA Sec. 4): BiCG, BiCG_sym (and CG
// with the bilinear form, the same recurrence), BiCGSTAB, CGS, TFQMR, QMR
// with coupled two-term recurrences and QMR_sym, in the textbook forms the
// paper cites (Barrett et al. 1994; Sonneveld 1989; Freund 1992, 1993),
// BiCGSTAB(l) (Sleijpen & Fokkema 1993) and ML(n)BiCGSTAB (Yeung & Chan
// 1999)
// written for complex vectors: Hermitian products x^H y in BiCG, BiCGSTAB,
// CGS and TFQMR, bilinear x^T y in BiCG_sym, CG and the QMR Lanczos
// processes with A^T = A (the DDA matrix is complex symmetric, Sec. 3);
// A^H v is formed as conj(A conj(v)).  BiCG starts from the shadow residual
// conj(r0), BiCGSTAB, CGS and TFQMR from r0.  QMR_sym runs QMR's
// recurrences on the complex-symmetric Lanczos process, whose left and
// right Lanczos vectors coincide, so it needs one product per iteration.
//
// A solve runs a batch of right-hand sides with the same matrix in lock
// step: every vector kernel covers all of them (blockIdx.y selects the
// right-hand side), every scalar kernel runs one block per right-hand side,
// and each matvec launch transforms the whole batch against the one shared
// spectrum.  Each right-hand side has its own scalars and status word; once
// it has converged, broken down or used its iterations, all later kernels
// and the matvec passes skip its blocks.
//
// Every vector update is fused with the inner products that follow it;
// each block writes its partial sums and the scalar kernel adds them in a
// fixed order (deterministic) and runs the scalar recurrence on the
// device, so the host never waits inside an iteration.  Vector data may be
// complex64: the products are then formed in FP32, summed per thread with
// compensation and accumulated in FP64; all scalars are FP64.
#include <cmath>
#include <cstring>

#include "krylov.cuh"

namespace dda {

namespace {

// ------------------------------------------------------------- reductions
template <typename T>
struct DotAcc {
    // Per-thread sum of one inner product.  FP64 data: plain FP64 sum.
    // FP32 data: compensated (Kahan) FP32 sum, whose error does not grow
    // with the number of terms, converted to FP64 once at the end; the block
    // and grid reductions are FP64.  (FP64 adds inside the element loop cost
    // more than the loads on this GPU and hold back the next loads.)
    C<T> s, c;
    double2 hi;
    __device__ __forceinline__ void init() { s = mk<T>(0, 0); c = mk<T>(0, 0); hi = make_double2(0.0, 0.0); }
    __device__ __forceinline__ void add(C<T> v) {
        if (sizeof(T) == 8) {
            s = cadd<T>(s, v);
        } else {
            const C<T> y = csub<T>(v, c);
            const C<T> t = cadd<T>(s, y);
            c = csub<T>(csub<T>(t, s), y);
            s = t;
        }
    }
    __device__ __forceinline__ void flush() {
        hi.x = (double)s.x - (double)c.x;
        hi.y = (double)s.y - (double)c.y;
    }
};

// partial sums of this block into part (already offset to its right-hand side)
template <int NR>
__device__ __forceinline__ void block_partials(double2 (&a)[NR], double2* __restrict__ part) {
    __shared__ double2 sm[NR][kVecThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a[r].x += __shfl_down_sync(0xffffffffu, a[r].x, o);
            a[r].y += __shfl_down_sync(0xffffffffu, a[r].y, o);
        }
        if (lane == 0) sm[r][wid] = a[r];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            double2 t = make_double2(0.0, 0.0);
            for (int w = 0; w < kVecThreads / 32; ++w) { t.x += sm[r][w].x; t.y += sm[r][w].y; }
            part[blockIdx.x * kMaxRed + r] = t;
        }
    }
}

// all threads of a scalar block call this; every thread gets the sums of
// the nparts partials of its right-hand side
template <int NR>
__device__ __forceinline__ void final_sums(const double2* __restrict__ part, int nparts, double2 (&out)[NR]) {
    __shared__ double2 sm[NR][kVecThreads];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        double2 a = make_double2(0.0, 0.0);
        for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
            a.x += part[i * kMaxRed + r].x;
            a.y += part[i * kMaxRed + r].y;
        }
        sm[r][threadIdx.x] = a;
    }
    __syncthreads();
    for (int o = kVecThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                sm[r][threadIdx.x].x += sm[r][threadIdx.x + o].x;
                sm[r][threadIdx.x].y += sm[r][threadIdx.x + o].y;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) out[r] = sm[r][0];
}

__device__ __forceinline__ double2 dmul(double2 a, double2 b) { return cmul<double>(a, b); }
__device__ __forceinline__ double2 ddiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ bool is_zero(double2 a) { return a.x == 0.0 && a.y == 0.0; }
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

template <typename T>
__device__ __forceinline__ C<T> to_t(double2 a) { return mk<T>((T)a.x, (T)a.y); }
template <typename T>
__device__ __forceinline__ C<T> conjg(C<T> a) { return mk<T>(a.x, -a.y); }
template <typename T>
__device__ __forceinline__ C<T> norm2c(C<T> a) { return mk<T>(a.x * a.x + a.y * a.y, 0); }

// ---- batch addressing: vector kernels run a (blocks per RHS, nb) grid,
// scalar kernels an (nb) grid
template <typename P>
__device__ __forceinline__ P* rhs_vec(P* p, int64_t n) { return p + (int64_t)blockIdx.y * n; }
__device__ __forceinline__ double2* rhs_part(double2* part) {
    return part + (int64_t)blockIdx.y * gridDim.x * kMaxRed;
}

// Grid-strided loop over the n elements of this block's right-hand side,
// kVecUnroll per thread per step: the loads of all of them are issued
// before any is used, so every thread keeps several requests in flight.
template <typename Load, typename Op>
__device__ __forceinline__ void vec_loop(int64_t n, Load load, Op op) {
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; base < n; base += kVecUnroll * S) {
        decltype(load(base)) v[kVecUnroll];
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = base + u * S;
            if (i < n) v[u] = load(i);
        }
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = base + u * S;
            if (i < n) op(i, v[u]);
        }
    }
}

template <typename T> struct V1 { C<T> a; };
template <typename T> struct V2 { C<T> a, b; };
template <typename T> struct V3 { C<T> a, b, c; };
template <typename T> struct V4 { C<T> a, b, c, d; };
template <typename T> struct V6 { C<T> a, b, c, d, e, f; };
template <typename T, int K> struct VN { C<T> v[K]; };

// ---------------------------------------------------------------- common
// r = b - r (r = A x on entry when has_x0), x = 0 otherwise r = b; rt = r or
// conj(r).  partials: ||b||^2, ||r||^2, rt^H r
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_init(const C<T>* __restrict__ b, C<T>* __restrict__ x,
                                                      C<T>* __restrict__ r, C<T>* __restrict__ rt, int64_t n,
                                                      int has_x0, int conj_rt, double2* __restrict__ part) {
    b = rhs_vec(b, n); x = rhs_vec(x, n); r = rhs_vec(r, n);
    if (rt) rt = rhs_vec(rt, n);
    part = rhs_part(part);
    DotAcc<T> nb, nr, rr;
    nb.init(); nr.init(); rr.init();
    vec_loop(n, [&](int64_t i) { return V2<T>{b[i], has_x0 ? r[i] : mk<T>(0, 0)}; },
             [&](int64_t i, const V2<T>& q) {
                 const C<T> ri = has_x0 ? csub<T>(q.a, q.b) : q.a;
                 if (!has_x0) x[i] = mk<T>(0, 0);
                 r[i] = ri;
                 const C<T> ti = conj_rt ? conjg<T>(ri) : ri;
                 if (rt) rt[i] = ti;
                 nb.add(norm2c<T>(q.a));
                 nr.add(norm2c<T>(ri));
                 rr.add(cmul<T>(conjg<T>(ti), ri));
             });
    nb.flush(); nr.flush(); rr.flush();
    double2 a[3] = {nb.hi, nr.hi, rr.hi};
    block_partials<3>(a, part);
}

// ctl: per right-hand side tolerance and cap (device) or null for tol and
// max_iter; a tolerance <= 0 marks a right-hand side that this solve leaves
// alone.  kind: 1 = QMR Lanczos norms, 2 = TFQMR's tau
__global__ void __launch_bounds__(kVecThreads) k_init_scalar(KState* st, const double2* __restrict__ part,
                                                             int nparts, const RhsCtl* __restrict__ ctl,
                                                             double tol, int max_iter, int kind) {
    st += blockIdx.x;
    part += (int64_t)blockIdx.x * nparts * kMaxRed;
    double2 s[3];
    final_sums<3>(part, nparts, s);
    if (threadIdx.x != 0) return;
    const double tl = ctl ? ctl[blockIdx.x].tol : tol;
    const int maxit = ctl ? ctl[blockIdx.x].maxit : max_iter;
    st->iter = 0;
    st->matvecs = 0;
    st->maxit = maxit;
    st->bnorm2 = s[0].x;
    st->tol2 = tl * tl;
    for (int i = 0; i < S_NSLOTS; ++i) st->s[i] = make_double2(0.0, 0.0);
    st->status = ST_RUN;
    if (!(tl > 0.0)) { st->rel2 = 0.0; st->status = ST_CONVERGED; return; }
    if (!isfinite(s[0].x) || !isfinite(s[1].x)) { st->status = ST_NAN; return; }
    if (s[0].x == 0.0) { st->rel2 = 0.0; st->status = ST_CONVERGED; return; }
    st->rel2 = s[1].x / s[0].x;
    if (st->rel2 <= st->tol2) { st->status = ST_CONVERGED; return; }
    if (maxit < 1) { st->status = ST_MAXIT; return; }
    st->s[S_RHO] = s[2];
    if (kind == 2) st->s[S_TAU] = make_double2(sqrt(s[1].x), 0.0);
    if (kind == 3) {   // BiCGSTAB(ell): rho0 = 1, alpha = 0, omega = 1, the first cycle starts from -omega rho0
        st->s[S_RHO_OLD] = make_double2(-1.0, 0.0);
        st->s[S_OMEGA] = make_double2(1.0, 0.0);
    }
    if (kind == 1) {
        st->s[S_RHOQ] = make_double2(sqrt(s[1].x), 0.0);
        st->s[S_XI] = make_double2(sqrt(s[1].x), 0.0);
        st->s[S_GAMMA_OLD] = make_double2(1.0, 0.0);
        st->s[S_ETA] = make_double2(-1.0, 0.0);
    }
}

// end of an iteration: convergence or the iteration cap (true: stop here)
__device__ __forceinline__ bool end_of_iteration(KState* st, double rel2) {
    st->iter += 1;
    st->rel2 = rel2;
    if (!isfinite(rel2)) { st->status = ST_NAN; return true; }
    if (rel2 <= st->tol2) { st->status = ST_CONVERGED; return true; }
    if (st->iter >= st->maxit) { st->status = ST_MAXIT; return true; }
    return false;
}

// partial dot products: kind 0 = a^H b, kind 1 = a^T b
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_dot1(const KState* st, const C<T>* __restrict__ a0,
                                                      const C<T>* __restrict__ b0, int kind0, int64_t n,
                                                      double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    a0 = rhs_vec(a0, n); b0 = rhs_vec(b0, n); part = rhs_part(part);
    DotAcc<T> d0;
    d0.init();
    vec_loop(n, [&](int64_t i) { return V2<T>{a0[i], b0[i]}; },
             [&](int64_t, const V2<T>& q) { d0.add(cmul<T>(kind0 == 0 ? conjg<T>(q.a) : q.a, q.b)); });
    d0.flush();
    double2 a[1] = {d0.hi};
    block_partials<1>(a, part);
}

// partials t^H t and t^H s (BiCGSTAB's omega)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_dot_ts(const KState* st, const C<T>* __restrict__ t,
                                                        const C<T>* __restrict__ s, int64_t n,
                                                        double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    t = rhs_vec(t, n); s = rhs_vec(s, n); part = rhs_part(part);
    DotAcc<T> tt, ts;
    tt.init(); ts.init();
    vec_loop(n, [&](int64_t i) { return V2<T>{t[i], s[i]}; },
             [&](int64_t, const V2<T>& q) {
                 tt.add(norm2c<T>(q.a));
                 ts.add(cmul<T>(conjg<T>(q.a), q.b));
             });
    tt.flush(); ts.flush();
    double2 a[2] = {tt.hi, ts.hi};
    block_partials<2>(a, part);
}

// ---------------------------------------------------------------- BiCGSTAB
// p = r (first) or p = r + beta (p - omega v)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_bcs_p(const KState* st, const C<T>* __restrict__ r,
                                                       C<T>* __restrict__ p, const C<T>* __restrict__ v,
                                                       int64_t n, int first) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    r = rhs_vec(r, n); p = rhs_vec(p, n); v = rhs_vec(v, n);
    const C<T> beta = to_t<T>(st->s[S_BETA]), omega = to_t<T>(st->s[S_OMEGA]);
    if (first) {
        vec_loop(n, [&](int64_t i) { return V1<T>{r[i]}; }, [&](int64_t i, const V1<T>& q) { p[i] = q.a; });
    } else {
        vec_loop(n, [&](int64_t i) { return V3<T>{r[i], p[i], v[i]}; },
                 [&](int64_t i, const V3<T>& q) { p[i] = cfma<T>(beta, csub<T>(q.b, cmul<T>(omega, q.c)), q.a); });
    }
}

// s = r - alpha v; partial ||s||^2
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_bcs_s(const KState* st, const C<T>* __restrict__ r,
                                                       const C<T>* __restrict__ v, C<T>* __restrict__ s,
                                                       int64_t n, double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    r = rhs_vec(r, n); v = rhs_vec(v, n); s = rhs_vec(s, n); part = rhs_part(part);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    DotAcc<T> ns;
    ns.init();
    vec_loop(n, [&](int64_t i) { return V2<T>{r[i], v[i]}; },
             [&](int64_t i, const V2<T>& q) {
                 const C<T> si = csub<T>(q.a, cmul<T>(alpha, q.b));
                 s[i] = si;
                 ns.add(norm2c<T>(si));
             });
    ns.flush();
    double2 a[1] = {ns.hi};
    block_partials<1>(a, part);
}

// x += alpha p + omega s; r = s - omega t; partials ||r||^2, rt^H r.
// After a half-step convergence (status HALF) only x += alpha p.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_bcs_xr(const KState* st, C<T>* __restrict__ x,
                                                        const C<T>* __restrict__ p, const C<T>* __restrict__ s,
                                                        const C<T>* __restrict__ t, C<T>* __restrict__ r,
                                                        const C<T>* __restrict__ rt, int64_t n,
                                                        double2* __restrict__ part) {
    st += blockIdx.y;
    const int status = st->status;
    if (status != ST_RUN && status != ST_HALF) return;
    x = rhs_vec(x, n); p = rhs_vec(p, n); s = rhs_vec(s, n); t = rhs_vec(t, n);
    r = rhs_vec(r, n); rt = rhs_vec(rt, n); part = rhs_part(part);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]), omega = to_t<T>(st->s[S_OMEGA]);
    if (status == ST_HALF) {
        vec_loop(n, [&](int64_t i) { return V2<T>{x[i], p[i]}; },
                 [&](int64_t i, const V2<T>& q) { x[i] = cfma<T>(alpha, q.b, q.a); });
        return;
    }
    DotAcc<T> nr, rr;
    nr.init(); rr.init();
    vec_loop(n, [&](int64_t i) { return V6<T>{x[i], p[i], s[i], t[i], rt[i], mk<T>(0, 0)}; },
             [&](int64_t i, const V6<T>& q) {
                 x[i] = cfma<T>(omega, q.c, cfma<T>(alpha, q.b, q.a));
                 const C<T> ri = csub<T>(q.c, cmul<T>(omega, q.d));
                 r[i] = ri;
                 nr.add(norm2c<T>(ri));
                 rr.add(cmul<T>(conjg<T>(q.e), ri));
             });
    nr.flush(); rr.flush();
    double2 a[2] = {nr.hi, rr.hi};
    block_partials<2>(a, part);
}

// step: 0 = alpha from sigma, 1 = half-step check, 2 = omega, 3 = end of iteration
__global__ void __launch_bounds__(kVecThreads) k_bcs_scalar(KState* st, const double2* __restrict__ part,
                                                            int nparts, int step) {
    st += blockIdx.x;
    part += (int64_t)blockIdx.x * nparts * kMaxRed;
    if (step == 3 && st->status == ST_HALF) {
        if (threadIdx.x == 0) { st->status = ST_CONVERGED; st->iter += 1; st->rel2 = st->s[S_TMP].x; }
        return;
    }
    if (st->status != ST_RUN) return;
    double2 s[2];
    final_sums<2>(part, nparts, s);
    if (threadIdx.x != 0) return;
    if (step == 0) {
        st->matvecs += 1;
        const double2 sigma = s[0];
        if (!finite2(sigma)) { st->status = ST_NAN; return; }
        if (is_zero(sigma)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_ALPHA] = ddiv(st->s[S_RHO], sigma);
    } else if (step == 1) {
        const double rel2s = s[0].x / st->bnorm2;
        st->s[S_TMP] = make_double2(rel2s, 0.0);
        if (!isfinite(rel2s)) { st->status = ST_NAN; return; }
        if (rel2s <= st->tol2) st->status = ST_HALF;
    } else if (step == 2) {
        st->matvecs += 1;
        const double2 tt = s[0], ts = s[1];
        if (!finite2(tt) || !finite2(ts)) { st->status = ST_NAN; return; }
        if (tt.x == 0.0) { st->status = ST_BREAKDOWN; return; }
        st->s[S_OMEGA] = make_double2(ts.x / tt.x, ts.y / tt.x);
    } else {
        if (end_of_iteration(st, s[0].x / st->bnorm2)) return;
        const double2 rho_new = s[1];
        if (is_zero(st->s[S_OMEGA]) || is_zero(rho_new)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_BETA] = dmul(ddiv(rho_new, st->s[S_RHO]), ddiv(st->s[S_ALPHA], st->s[S_OMEGA]));
        st->s[S_RHO] = rho_new;
    }
}

// -------------------------------------------------------------------- BiCG
// p = r + beta p, pt = rt + conj(beta) pt (copies on the first step)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_bicg_p(const KState* st, const C<T>* __restrict__ r,
                                                        const C<T>* __restrict__ rt, C<T>* __restrict__ p,
                                                        C<T>* __restrict__ pt, int64_t n, int first) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    r = rhs_vec(r, n); rt = rhs_vec(rt, n); p = rhs_vec(p, n); pt = rhs_vec(pt, n);
    const C<T> beta = to_t<T>(st->s[S_BETA]);
    const C<T> cbeta = conjg<T>(beta);
    if (first) {
        vec_loop(n, [&](int64_t i) { return V2<T>{r[i], rt[i]}; },
                 [&](int64_t i, const V2<T>& q) { p[i] = q.a; pt[i] = q.b; });
    } else {
        vec_loop(n, [&](int64_t i) { return V4<T>{r[i], rt[i], p[i], pt[i]}; },
                 [&](int64_t i, const V4<T>& q) {
                     p[i] = cfma<T>(beta, q.c, q.a);
                     pt[i] = cfma<T>(cbeta, q.d, q.b);
                 });
    }
}

// x += alpha p; r -= alpha q; rt -= conj(alpha) qt; partials ||r||^2, rt^H r
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_bicg_update(const KState* st, C<T>* __restrict__ x,
                                                             const C<T>* __restrict__ p, const C<T>* __restrict__ q,
                                                             const C<T>* __restrict__ qt, C<T>* __restrict__ r,
                                                             C<T>* __restrict__ rt, int64_t n,
                                                             double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    x = rhs_vec(x, n); p = rhs_vec(p, n); q = rhs_vec(q, n); qt = rhs_vec(qt, n);
    r = rhs_vec(r, n); rt = rhs_vec(rt, n); part = rhs_part(part);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    const C<T> nalpha = mk<T>(-alpha.x, -alpha.y), ncalpha = mk<T>(-alpha.x, alpha.y);
    DotAcc<T> nr, rr;
    nr.init(); rr.init();
    vec_loop(n, [&](int64_t i) { return V6<T>{x[i], p[i], q[i], qt[i], r[i], rt[i]}; },
             [&](int64_t i, const V6<T>& u) {
                 x[i] = cfma<T>(alpha, u.b, u.a);
                 const C<T> ri = cfma<T>(nalpha, u.c, u.e);
                 const C<T> ti = cfma<T>(ncalpha, u.d, u.f);
                 r[i] = ri;
                 rt[i] = ti;
                 nr.add(norm2c<T>(ri));
                 rr.add(cmul<T>(conjg<T>(ti), ri));
             });
    nr.flush(); rr.flush();
    double2 a[2] = {nr.hi, rr.hi};
    block_partials<2>(a, part);
}

// BiCG for complex-symmetric A (Freund 1992; the paper's BiCG_sym, Sec. 4):
// x += alpha p; r -= alpha q; partials ||r||^2 and the bilinear r^T r
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cocg_update(const KState* st, C<T>* __restrict__ x,
                                                             const C<T>* __restrict__ p, const C<T>* __restrict__ q,
                                                             C<T>* __restrict__ r, int64_t n,
                                                             double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    x = rhs_vec(x, n); p = rhs_vec(p, n); q = rhs_vec(q, n); r = rhs_vec(r, n); part = rhs_part(part);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    const C<T> nalpha = mk<T>(-alpha.x, -alpha.y);
    DotAcc<T> nr, rr;
    nr.init(); rr.init();
    vec_loop(n, [&](int64_t i) { return V4<T>{x[i], p[i], q[i], r[i]}; },
             [&](int64_t i, const V4<T>& u) {
                 x[i] = cfma<T>(alpha, u.b, u.a);
                 const C<T> ri = cfma<T>(nalpha, u.c, u.d);
                 r[i] = ri;
                 nr.add(norm2c<T>(ri));
                 rr.add(cmul<T>(ri, ri));
             });
    nr.flush(); rr.flush();
    double2 a[2] = {nr.hi, rr.hi};
    block_partials<2>(a, part);
}

// step 0: alpha = rho / sigma (sigma = pt^H q for BiCG, p^T q for BiCG_sym);
// step 1: end of iteration.  mv: products per iteration (2 or 1)
__global__ void __launch_bounds__(kVecThreads) k_bicg_scalar(KState* st, const double2* __restrict__ part,
                                                             int nparts, int step, int mv) {
    st += blockIdx.x;
    part += (int64_t)blockIdx.x * nparts * kMaxRed;
    if (st->status != ST_RUN) return;
    double2 s[2];
    final_sums<2>(part, nparts, s);
    if (threadIdx.x != 0) return;
    if (step == 0) {
        st->matvecs += mv;
        const double2 sigma = s[0];
        if (!finite2(sigma)) { st->status = ST_NAN; return; }
        if (is_zero(sigma)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_ALPHA] = ddiv(st->s[S_RHO], sigma);
    } else {
        if (end_of_iteration(st, s[0].x / st->bnorm2)) return;
        const double2 rho_new = s[1];
        if (is_zero(rho_new)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_BETA] = ddiv(rho_new, st->s[S_RHO]);
        st->s[S_RHO] = rho_new;
    }
}

// --------------------------------------------------------------------- QMR
// v = vt / rho, w = wt / xi; partial w^T v
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_qmr_vw(const KState* st, const C<T>* __restrict__ vt,
                                                        const C<T>* __restrict__ wt, C<T>* __restrict__ v,
                                                        C<T>* __restrict__ w, int64_t n, double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    vt = rhs_vec(vt, n); wt = rhs_vec(wt, n); v = rhs_vec(v, n); w = rhs_vec(w, n); part = rhs_part(part);
    const T irho = (T)(1.0 / st->s[S_RHOQ].x), ixi = (T)(1.0 / st->s[S_XI].x);
    DotAcc<T> d;
    d.init();
    vec_loop(n, [&](int64_t i) { return V2<T>{vt[i], wt[i]}; },
             [&](int64_t i, const V2<T>& q) {
                 const C<T> vi = cscale<T>(q.a, irho), wi = cscale<T>(q.b, ixi);
                 v[i] = vi;
                 w[i] = wi;
                 d.add(cmul<T>(wi, vi));
             });
    d.flush();
    double2 a[1] = {d.hi};
    block_partials<1>(a, part);
}

// p = v - cp p, q = w - cq q (copies on the first step)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_qmr_pq(const KState* st, const C<T>* __restrict__ v,
                                                        const C<T>* __restrict__ w, C<T>* __restrict__ p,
                                                        C<T>* __restrict__ q, int64_t n, int first) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    v = rhs_vec(v, n); w = rhs_vec(w, n); p = rhs_vec(p, n); q = rhs_vec(q, n);
    const C<T> ncp = to_t<T>(st->s[S_NCP]), ncq = to_t<T>(st->s[S_NCQ]);
    if (first) {
        vec_loop(n, [&](int64_t i) { return V2<T>{v[i], w[i]}; },
                 [&](int64_t i, const V2<T>& u) { p[i] = u.a; q[i] = u.b; });
    } else {
        vec_loop(n, [&](int64_t i) { return V4<T>{v[i], w[i], p[i], q[i]}; },
                 [&](int64_t i, const V4<T>& u) {
                     p[i] = cfma<T>(ncp, u.c, u.a);
                     q[i] = cfma<T>(ncq, u.d, u.b);
                 });
    }
}

// vt = pt - beta v; wt = (A q) - beta w; partials ||vt||^2, ||wt||^2
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_qmr_vtwt(const KState* st, const C<T>* __restrict__ pt,
                                                          const C<T>* __restrict__ v, const C<T>* __restrict__ w,
                                                          C<T>* __restrict__ vt, C<T>* __restrict__ wt, int64_t n,
                                                          double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    pt = rhs_vec(pt, n); v = rhs_vec(v, n); w = rhs_vec(w, n); vt = rhs_vec(vt, n); wt = rhs_vec(wt, n);
    part = rhs_part(part);
    const C<T> beta = to_t<T>(st->s[S_BETA]);
    const C<T> nbeta = mk<T>(-beta.x, -beta.y);
    DotAcc<T> a, b;
    a.init(); b.init();
    vec_loop(n, [&](int64_t i) { return V4<T>{pt[i], v[i], w[i], wt[i]}; },
             [&](int64_t i, const V4<T>& u) {
                 const C<T> vi = cfma<T>(nbeta, u.b, u.a);
                 const C<T> wi = cfma<T>(nbeta, u.c, u.d);
                 vt[i] = vi;
                 wt[i] = wi;
                 a.add(norm2c<T>(vi));
                 b.add(norm2c<T>(wi));
             });
    a.flush(); b.flush();
    double2 s[2] = {a.hi, b.hi};
    block_partials<2>(s, part);
}

// d = eta p + f d; s = eta pt + f s; x += d; r -= s; partial ||r||^2
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_qmr_ds(const KState* st, const C<T>* __restrict__ p,
                                                        const C<T>* __restrict__ pt, C<T>* __restrict__ d,
                                                        C<T>* __restrict__ s, C<T>* __restrict__ x,
                                                        C<T>* __restrict__ r, int64_t n, int first,
                                                        double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    p = rhs_vec(p, n); pt = rhs_vec(pt, n); d = rhs_vec(d, n); s = rhs_vec(s, n);
    x = rhs_vec(x, n); r = rhs_vec(r, n); part = rhs_part(part);
    const C<T> eta = to_t<T>(st->s[S_ETA]);
    const T f = first ? (T)0 : (T)st->s[S_F].x;
    DotAcc<T> nr;
    nr.init();
    vec_loop(n,
             [&](int64_t i) {
                 return V6<T>{p[i], pt[i], first ? mk<T>(0, 0) : d[i], first ? mk<T>(0, 0) : s[i], x[i], r[i]};
             },
             [&](int64_t i, const V6<T>& u) {
                 const C<T> di = cadd<T>(cmul<T>(eta, u.a), cscale<T>(u.c, f));
                 const C<T> si = cadd<T>(cmul<T>(eta, u.b), cscale<T>(u.d, f));
                 d[i] = di;
                 s[i] = si;
                 x[i] = cadd<T>(u.e, di);
                 const C<T> ri = csub<T>(u.f, si);
                 r[i] = ri;
                 nr.add(norm2c<T>(ri));
             });
    nr.flush();
    double2 a[1] = {nr.hi};
    block_partials<1>(a, part);
}

// step 0: delta (+ p/q coefficients); 1: eps, beta; 2: rho, xi, theta,
// gamma, eta, f; 3: end of iteration
__global__ void __launch_bounds__(kVecThreads) k_qmr_scalar(KState* st, const double2* __restrict__ part,
                                                            int nparts, int step, int first, int sym) {
    st += blockIdx.x;
    part += (int64_t)blockIdx.x * nparts * kMaxRed;
    if (st->status != ST_RUN) return;
    double2 s[2];
    final_sums<2>(part, nparts, s);
    if (threadIdx.x != 0) return;
    if (step == 0) {
        const double rho = st->s[S_RHOQ].x, xi = st->s[S_XI].x;
        if (rho == 0.0 || xi == 0.0) { st->status = ST_BREAKDOWN; return; }
        const double2 delta = s[0];
        if (!finite2(delta)) { st->status = ST_NAN; return; }
        if (is_zero(delta)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_DELTA] = delta;
        if (!first) {
            const double2 q = ddiv(delta, st->s[S_EPS]);
            st->s[S_NCP] = make_double2(-xi * q.x, -xi * q.y);    // -(xi delta / eps)
            st->s[S_NCQ] = make_double2(-rho * q.x, -rho * q.y);  // -(rho delta / eps)
        }
    } else if (step == 1) {
        st->matvecs += 1;
        const double2 eps = s[0];
        if (!finite2(eps)) { st->status = ST_NAN; return; }
        if (is_zero(eps)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_EPS] = eps;
        const double2 beta = ddiv(eps, st->s[S_DELTA]);
        if (is_zero(beta)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_BETA] = beta;
    } else if (step == 2) {
        if (!sym) st->matvecs += 1;   // QMR's second product, A^T q
        const double rho_new = sqrt(s[0].x), xi_new = sqrt(s[1].x);
        const double2 beta = st->s[S_BETA];
        const double gamma_old = st->s[S_GAMMA_OLD].x;
        const double theta = rho_new / (gamma_old * hypot(beta.x, beta.y));
        const double gamma = 1.0 / sqrt(1.0 + theta * theta);
        if (gamma == 0.0 || !isfinite(theta)) { st->status = ST_BREAKDOWN; return; }
        // eta = -eta rho gamma^2 / (beta gamma_old^2)
        const double sc = -st->s[S_RHOQ].x * gamma * gamma / (gamma_old * gamma_old);
        const double2 e = ddiv(st->s[S_ETA], beta);
        st->s[S_ETA] = make_double2(sc * e.x, sc * e.y);
        const double tg = st->s[S_THETA_OLD].x * gamma;
        st->s[S_F] = make_double2(tg * tg, 0.0);
        st->s[S_RHO_NEW] = make_double2(rho_new, 0.0);
        st->s[S_XI_NEW] = make_double2(xi_new, 0.0);
        st->s[S_TMP] = make_double2(theta, gamma);
    } else {
        if (end_of_iteration(st, s[0].x / st->bnorm2)) return;
        st->s[S_RHOQ] = st->s[S_RHO_NEW];
        st->s[S_XI] = st->s[S_XI_NEW];
        st->s[S_THETA_OLD] = make_double2(st->s[S_TMP].x, 0.0);
        st->s[S_GAMMA_OLD] = make_double2(st->s[S_TMP].y, 0.0);
    }
}

// ----------------------------------------------------------------- QMR_sym
// v = vt / rho; partial v^T v
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_qs_v(const KState* st, const C<T>* __restrict__ vt,
                                                      C<T>* __restrict__ v, int64_t n, double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    vt = rhs_vec(vt, n); v = rhs_vec(v, n); part = rhs_part(part);
    const T irho = (T)(1.0 / st->s[S_RHOQ].x);
    DotAcc<T> d;
    d.init();
    vec_loop(n, [&](int64_t i) { return V1<T>{vt[i]}; },
             [&](int64_t i, const V1<T>& q) {
                 const C<T> vi = cscale<T>(q.a, irho);
                 v[i] = vi;
                 d.add(cmul<T>(vi, vi));
             });
    d.flush();
    double2 a[1] = {d.hi};
    block_partials<1>(a, part);
}

// p = v - (rho delta / eps) p (a copy on the first step)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_qs_p(const KState* st, const C<T>* __restrict__ v,
                                                      C<T>* __restrict__ p, int64_t n, int first) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    v = rhs_vec(v, n); p = rhs_vec(p, n);
    const C<T> ncp = to_t<T>(st->s[S_NCP]);
    if (first) {
        vec_loop(n, [&](int64_t i) { return V1<T>{v[i]}; }, [&](int64_t i, const V1<T>& u) { p[i] = u.a; });
    } else {
        vec_loop(n, [&](int64_t i) { return V2<T>{v[i], p[i]}; },
                 [&](int64_t i, const V2<T>& u) { p[i] = cfma<T>(ncp, u.b, u.a); });
    }
}

// vt = pt - beta v; partial ||vt||^2 in both slots the QMR scalar step reads
// (the norms of the right and the left Lanczos vectors, equal here)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_qs_vt(const KState* st, const C<T>* __restrict__ pt,
                                                       const C<T>* __restrict__ v, C<T>* __restrict__ vt, int64_t n,
                                                       double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    pt = rhs_vec(pt, n); v = rhs_vec(v, n); vt = rhs_vec(vt, n); part = rhs_part(part);
    const C<T> beta = to_t<T>(st->s[S_BETA]);
    const C<T> nbeta = mk<T>(-beta.x, -beta.y);
    DotAcc<T> a;
    a.init();
    vec_loop(n, [&](int64_t i) { return V2<T>{pt[i], v[i]}; },
             [&](int64_t i, const V2<T>& u) {
                 const C<T> vi = cfma<T>(nbeta, u.b, u.a);
                 vt[i] = vi;
                 a.add(norm2c<T>(vi));
             });
    a.flush();
    double2 s2[2] = {a.hi, a.hi};
    block_partials<2>(s2, part);
}

// --------------------------------------------------------------------- CGS
// u = r + beta q, p = u + beta (q + beta p) (copies of r on the first step)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cgs_up(const KState* st, const C<T>* __restrict__ r,
                                                        const C<T>* __restrict__ q, C<T>* __restrict__ u,
                                                        C<T>* __restrict__ p, int64_t n, int first) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    r = rhs_vec(r, n); q = rhs_vec(q, n); u = rhs_vec(u, n); p = rhs_vec(p, n);
    const C<T> beta = to_t<T>(st->s[S_BETA]);
    if (first) {
        vec_loop(n, [&](int64_t i) { return V1<T>{r[i]}; },
                 [&](int64_t i, const V1<T>& a) { u[i] = a.a; p[i] = a.a; });
    } else {
        vec_loop(n, [&](int64_t i) { return V3<T>{r[i], q[i], p[i]}; },
                 [&](int64_t i, const V3<T>& a) {
                     const C<T> ui = cfma<T>(beta, a.b, a.a);
                     u[i] = ui;
                     p[i] = cfma<T>(beta, cfma<T>(beta, a.c, a.b), ui);
                 });
    }
}

// q = u - alpha vh; uh = u + q; x += alpha uh
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cgs_q(const KState* st, const C<T>* __restrict__ u,
                                                       const C<T>* __restrict__ vh, C<T>* __restrict__ q,
                                                       C<T>* __restrict__ uh, C<T>* __restrict__ x, int64_t n) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    u = rhs_vec(u, n); vh = rhs_vec(vh, n); q = rhs_vec(q, n); uh = rhs_vec(uh, n); x = rhs_vec(x, n);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    const C<T> nalpha = mk<T>(-alpha.x, -alpha.y);
    vec_loop(n, [&](int64_t i) { return V3<T>{u[i], vh[i], x[i]}; },
             [&](int64_t i, const V3<T>& a) {
                 const C<T> qi = cfma<T>(nalpha, a.b, a.a);
                 const C<T> ui = cadd<T>(a.a, qi);
                 q[i] = qi;
                 uh[i] = ui;
                 x[i] = cfma<T>(alpha, ui, a.c);
             });
}

// r -= alpha qh; partials ||r||^2, rt^H r
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cgs_r(const KState* st, const C<T>* __restrict__ qh,
                                                       C<T>* __restrict__ r, const C<T>* __restrict__ rt, int64_t n,
                                                       double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    qh = rhs_vec(qh, n); r = rhs_vec(r, n); rt = rhs_vec(rt, n); part = rhs_part(part);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    const C<T> nalpha = mk<T>(-alpha.x, -alpha.y);
    DotAcc<T> nr, rr;
    nr.init(); rr.init();
    vec_loop(n, [&](int64_t i) { return V3<T>{qh[i], r[i], rt[i]}; },
             [&](int64_t i, const V3<T>& a) {
                 const C<T> ri = cfma<T>(nalpha, a.a, a.b);
                 r[i] = ri;
                 nr.add(norm2c<T>(ri));
                 rr.add(cmul<T>(conjg<T>(a.c), ri));
             });
    nr.flush(); rr.flush();
    double2 s2[2] = {nr.hi, rr.hi};
    block_partials<2>(s2, part);
}

// ------------------------------------------------------------------- TFQMR
// One iteration = the half-steps m = 2n (vector u0 = u_m, product Au0) and
// m = 2n + 1 (u1, Au1).  The update x += eta_m d_m of each half-step runs in
// the next vector kernel, after the scalar kernel has formed eta_m; when the
// bound test stops the iteration, the status HALF lets exactly that pending
// update through.

// d's coefficient theta_{m-1}^2 eta_{m-1} / alpha for the half-step at hand
template <typename T>
__device__ __forceinline__ C<T> tf_cd(const KState* st) {
    const double th = st->s[S_THETA].x;
    const double2 c = ddiv(st->s[S_ETA], st->s[S_ALPHA]);
    return to_t<T>(make_double2(th * th * c.x, th * th * c.y));
}

// u0 = r, d = 0
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_tf_init(const KState* st, const C<T>* __restrict__ r,
                                                         C<T>* __restrict__ u0, C<T>* __restrict__ d, int64_t n) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    r = rhs_vec(r, n); u0 = rhs_vec(u0, n); d = rhs_vec(d, n);
    vec_loop(n, [&](int64_t i) { return V1<T>{r[i]}; },
             [&](int64_t i, const V1<T>& a) { u0[i] = a.a; d[i] = mk<T>(0, 0); });
}

// u1 = u0 - alpha v
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_tf_u1(const KState* st, const C<T>* __restrict__ u0,
                                                       const C<T>* __restrict__ v, C<T>* __restrict__ u1, int64_t n) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    u0 = rhs_vec(u0, n); v = rhs_vec(v, n); u1 = rhs_vec(u1, n);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    const C<T> nalpha = mk<T>(-alpha.x, -alpha.y);
    vec_loop(n, [&](int64_t i) { return V2<T>{u0[i], v[i]}; },
             [&](int64_t i, const V2<T>& a) { u1[i] = cfma<T>(nalpha, a.b, a.a); });
}

// even half-step: w -= alpha Au0; d = u0 + cd d; partial ||w||^2
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_tf_even(const KState* st, C<T>* __restrict__ w,
                                                         const C<T>* __restrict__ Au0, const C<T>* __restrict__ u0,
                                                         C<T>* __restrict__ d, int64_t n, double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    w = rhs_vec(w, n); Au0 = rhs_vec(Au0, n); u0 = rhs_vec(u0, n); d = rhs_vec(d, n); part = rhs_part(part);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    const C<T> nalpha = mk<T>(-alpha.x, -alpha.y);
    const C<T> cd = tf_cd<T>(st);
    DotAcc<T> nw;
    nw.init();
    vec_loop(n, [&](int64_t i) { return V4<T>{w[i], Au0[i], u0[i], d[i]}; },
             [&](int64_t i, const V4<T>& a) {
                 const C<T> wi = cfma<T>(nalpha, a.b, a.a);
                 w[i] = wi;
                 d[i] = cfma<T>(cd, a.d, a.c);
                 nw.add(norm2c<T>(wi));
             });
    nw.flush();
    double2 s1[1] = {nw.hi};
    block_partials<1>(s1, part);
}

// x += eta d (the even half-step's update); then, unless the iteration has
// stopped, the odd half-step: w -= alpha Au1; d = u1 + cd d; partials
// ||w||^2, rt^H w
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_tf_odd(const KState* st, C<T>* __restrict__ x, C<T>* __restrict__ w,
                                                        const C<T>* __restrict__ Au1, const C<T>* __restrict__ u1,
                                                        C<T>* __restrict__ d, const C<T>* __restrict__ rt, int64_t n,
                                                        double2* __restrict__ part) {
    st += blockIdx.y;
    const int status = st->status;
    if (status != ST_RUN && status != ST_HALF) return;
    x = rhs_vec(x, n); w = rhs_vec(w, n); Au1 = rhs_vec(Au1, n); u1 = rhs_vec(u1, n); d = rhs_vec(d, n);
    rt = rhs_vec(rt, n); part = rhs_part(part);
    const C<T> eta = to_t<T>(st->s[S_ETA]);
    if (status == ST_HALF) {
        vec_loop(n, [&](int64_t i) { return V2<T>{x[i], d[i]}; },
                 [&](int64_t i, const V2<T>& a) { x[i] = cfma<T>(eta, a.b, a.a); });
        return;
    }
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    const C<T> nalpha = mk<T>(-alpha.x, -alpha.y);
    const C<T> cd = tf_cd<T>(st);
    DotAcc<T> nw, rw;
    nw.init(); rw.init();
    vec_loop(n, [&](int64_t i) { return V6<T>{x[i], w[i], Au1[i], u1[i], d[i], rt[i]}; },
             [&](int64_t i, const V6<T>& a) {
                 x[i] = cfma<T>(eta, a.e, a.a);
                 const C<T> wi = cfma<T>(nalpha, a.c, a.b);
                 w[i] = wi;
                 d[i] = cfma<T>(cd, a.e, a.d);
                 nw.add(norm2c<T>(wi));
                 rw.add(cmul<T>(conjg<T>(a.f), wi));
             });
    nw.flush(); rw.flush();
    double2 s2[2] = {nw.hi, rw.hi};
    block_partials<2>(s2, part);
}

// x += eta d (the odd half-step's update); then, unless the iteration has
// stopped, u0 = w + beta u1
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_tf_next(const KState* st, C<T>* __restrict__ x,
                                                         const C<T>* __restrict__ d, const C<T>* __restrict__ w,
                                                         const C<T>* __restrict__ u1, C<T>* __restrict__ u0,
                                                         int64_t n) {
    st += blockIdx.y;
    const int status = st->status;
    if (status != ST_RUN && status != ST_HALF) return;
    x = rhs_vec(x, n); d = rhs_vec(d, n); w = rhs_vec(w, n); u1 = rhs_vec(u1, n); u0 = rhs_vec(u0, n);
    const C<T> eta = to_t<T>(st->s[S_ETA]);
    if (status == ST_HALF) {
        vec_loop(n, [&](int64_t i) { return V2<T>{x[i], d[i]}; },
                 [&](int64_t i, const V2<T>& a) { x[i] = cfma<T>(eta, a.b, a.a); });
        return;
    }
    const C<T> beta = to_t<T>(st->s[S_BETA]);
    vec_loop(n, [&](int64_t i) { return V4<T>{x[i], d[i], w[i], u1[i]}; },
             [&](int64_t i, const V4<T>& a) {
                 x[i] = cfma<T>(eta, a.b, a.a);
                 u0[i] = cfma<T>(beta, a.d, a.c);
             });
}

// v = Au0 + beta (Au1 + beta v) (first: v = Au0); partial rt^H v
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_tf_v(const KState* st, const C<T>* __restrict__ Au0,
                                                      const C<T>* __restrict__ Au1, C<T>* __restrict__ v,
                                                      const C<T>* __restrict__ rt, int64_t n, int first,
                                                      double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    Au0 = rhs_vec(Au0, n); Au1 = rhs_vec(Au1, n); v = rhs_vec(v, n); rt = rhs_vec(rt, n); part = rhs_part(part);
    const C<T> beta = first ? mk<T>(0, 0) : to_t<T>(st->s[S_BETA]);
    DotAcc<T> sv;
    sv.init();
    vec_loop(n,
             [&](int64_t i) {
                 return V4<T>{Au0[i], first ? mk<T>(0, 0) : Au1[i], first ? mk<T>(0, 0) : v[i], rt[i]};
             },
             [&](int64_t i, const V4<T>& a) {
                 const C<T> vi = cfma<T>(beta, cfma<T>(beta, a.c, a.b), a.a);
                 v[i] = vi;
                 sv.add(cmul<T>(conjg<T>(a.d), vi));
             });
    sv.flush();
    double2 s1[1] = {sv.hi};
    block_partials<1>(s1, part);
}

// theta, c, tau, eta of half-step m from ||w||^2; true: the bound test stops
__device__ __forceinline__ bool tf_half(KState* st, double w2, int m) {
    const double theta = sqrt(w2) / st->s[S_TAU].x;
    const double c2 = 1.0 / (1.0 + theta * theta);
    const double tau = st->s[S_TAU].x * theta * sqrt(c2);
    const double2 alpha = st->s[S_ALPHA];
    st->s[S_THETA] = make_double2(theta, 0.0);
    st->s[S_TAU] = make_double2(tau, 0.0);
    st->s[S_ETA] = make_double2(c2 * alpha.x, c2 * alpha.y);
    const double rel2 = tau * tau * (m + 1) / st->bnorm2;
    st->rel2 = rel2;
    if (!isfinite(rel2)) { st->status = ST_NAN; return true; }
    if (rel2 <= st->tol2) { st->status = ST_HALF; return true; }
    return false;
}

// alpha = rho / sigma; false after a breakdown
__device__ __forceinline__ bool tf_alpha(KState* st, double2 sigma) {
    if (!finite2(sigma)) { st->status = ST_NAN; return false; }
    if (is_zero(sigma) || is_zero(st->s[S_RHO])) { st->status = ST_BREAKDOWN; return false; }
    st->s[S_ALPHA] = ddiv(st->s[S_RHO], sigma);
    return true;
}

// step 0: first alpha (after the first product); 1: after the even
// half-step; 2: after the odd one (rho, beta); 3: after the new v (alpha,
// end of the iteration)
__global__ void __launch_bounds__(kVecThreads) k_tf_scalar(KState* st, const double2* __restrict__ part,
                                                           int nparts, int step) {
    st += blockIdx.x;
    part += (int64_t)blockIdx.x * nparts * kMaxRed;
    if ((step == 2 || step == 3) && st->status == ST_HALF) {
        // the pending update of x has run: the iteration ends here
        if (threadIdx.x == 0) { st->status = ST_CONVERGED; st->iter += 1; }
        return;
    }
    if (st->status != ST_RUN) return;
    double2 s[2];
    final_sums<2>(part, nparts, s);
    if (threadIdx.x != 0) return;
    if (step == 0) {
        st->matvecs += 1;
        tf_alpha(st, s[0]);
    } else if (step == 1) {
        st->matvecs += 1;
        tf_half(st, s[0].x, 2 * st->iter);
    } else if (step == 2) {
        if (tf_half(st, s[0].x, 2 * st->iter + 1)) return;
        const double2 rho_new = s[1];
        if (!finite2(rho_new)) { st->status = ST_NAN; return; }
        if (is_zero(rho_new)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_BETA] = ddiv(rho_new, st->s[S_RHO]);
        st->s[S_RHO] = rho_new;
    } else {
        st->matvecs += 1;
        st->iter += 1;
        if (!tf_alpha(st, s[0])) return;
        if (st->iter >= st->maxit) st->status = ST_MAXIT;
    }
}

// ------------------------------------------------------------ BiCGSTAB(l)
// One iteration is a cycle of l BiCG steps building r_j = A^j r and
// u_j = A^j u (j <= l), then the minimal-residual step: the gamma_j that
// minimise ||r_0 - sum_j gamma_j r_j|| come from the l x l Gram system of
// r_1..r_l (solved in FP64 on the device; the same minimiser as the
// modified Gram-Schmidt of Sleijpen & Fokkema 1993), and
// x += sum gamma_j r_(j-1), r_0 -= sum gamma_j r_j, u_0 -= sum gamma_j u_j.
template <typename T>
struct BLVecs {
    C<T>* r[4];
    C<T>* u[4];
};

// u_i = r_i - beta u_i, i < CNT
template <typename T, int CNT>
__global__ void __launch_bounds__(kVecThreads) k_bl_u(const KState* st, BLVecs<T> w, int64_t n) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    const C<T>* r[CNT];
    C<T>* u[CNT];
#pragma unroll
    for (int i = 0; i < CNT; ++i) { r[i] = rhs_vec(w.r[i], n); u[i] = rhs_vec(w.u[i], n); }
    const C<T> beta = to_t<T>(st->s[S_BETA]);
    const C<T> nbeta = mk<T>(-beta.x, -beta.y);
    vec_loop(n,
             [&](int64_t k) {
                 VN<T, 2 * CNT> a;
#pragma unroll
                 for (int i = 0; i < CNT; ++i) { a.v[i] = r[i][k]; a.v[CNT + i] = u[i][k]; }
                 return a;
             },
             [&](int64_t k, const VN<T, 2 * CNT>& a) {
#pragma unroll
                 for (int i = 0; i < CNT; ++i) u[i][k] = cfma<T>(nbeta, a.v[CNT + i], a.v[i]);
             });
}

// r_i -= alpha u_(i+1), i < CNT; x += alpha u_0
template <typename T, int CNT>
__global__ void __launch_bounds__(kVecThreads) k_bl_r(const KState* st, BLVecs<T> w, C<T>* __restrict__ x,
                                                      int64_t n) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    C<T>* r[CNT];
    const C<T>* u[CNT + 1];
#pragma unroll
    for (int i = 0; i < CNT; ++i) r[i] = rhs_vec(w.r[i], n);
#pragma unroll
    for (int i = 0; i <= CNT; ++i) u[i] = rhs_vec(w.u[i], n);
    x = rhs_vec(x, n);
    const C<T> alpha = to_t<T>(st->s[S_ALPHA]);
    const C<T> nalpha = mk<T>(-alpha.x, -alpha.y);
    vec_loop(n,
             [&](int64_t k) {
                 VN<T, 2 * CNT + 2> a;
#pragma unroll
                 for (int i = 0; i < CNT; ++i) a.v[i] = r[i][k];
#pragma unroll
                 for (int i = 0; i <= CNT; ++i) a.v[CNT + i] = u[i][k];
                 a.v[2 * CNT + 1] = x[k];
                 return a;
             },
             [&](int64_t k, const VN<T, 2 * CNT + 2>& a) {
#pragma unroll
                 for (int i = 0; i < CNT; ++i) r[i][k] = cfma<T>(nalpha, a.v[CNT + i + 1], a.v[i]);
                 x[k] = cfma<T>(alpha, a.v[CNT], a.v[2 * CNT + 1]);
             });
}

// Gram entries of the minimal-residual step: c_i = r_i^H r_0 (i = 1..L),
// then G_ij = r_i^H r_j for 1 <= i <= j <= L, in that order
template <typename T, int L>
__global__ void __launch_bounds__(kVecThreads) k_bl_gram(const KState* st, BLVecs<T> w, int64_t n,
                                                         double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    constexpr int NR = L + L * (L + 1) / 2;
    const C<T>* r[L + 1];
#pragma unroll
    for (int i = 0; i <= L; ++i) r[i] = rhs_vec(w.r[i], n);
    part = rhs_part(part);
    DotAcc<T> acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q].init();
    vec_loop(n,
             [&](int64_t k) {
                 VN<T, L + 1> a;
#pragma unroll
                 for (int i = 0; i <= L; ++i) a.v[i] = r[i][k];
                 return a;
             },
             [&](int64_t, const VN<T, L + 1>& a) {
                 int q = 0;
#pragma unroll
                 for (int i = 1; i <= L; ++i) acc[q++].add(cmul<T>(conjg<T>(a.v[i]), a.v[0]));
#pragma unroll
                 for (int i = 1; i <= L; ++i)
#pragma unroll
                     for (int j = i; j <= L; ++j) acc[q++].add(cmul<T>(conjg<T>(a.v[i]), a.v[j]));
             });
    double2 out[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) { acc[q].flush(); out[q] = acc[q].hi; }
    block_partials<NR>(out, part);
}

// x += sum_j gamma_j r_(j-1); r_0 -= sum_j gamma_j r_j; u_0 -= sum_j gamma_j u_j;
// partials ||r_0||^2, rt^H r_0
template <typename T, int L>
__global__ void __launch_bounds__(kVecThreads) k_bl_fin(const KState* st, BLVecs<T> w, C<T>* __restrict__ x,
                                                        const C<T>* __restrict__ rt, int64_t n,
                                                        double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    C<T>* r[L + 1];
    C<T>* u[L + 1];
#pragma unroll
    for (int i = 0; i <= L; ++i) { r[i] = rhs_vec(w.r[i], n); u[i] = rhs_vec(w.u[i], n); }
    x = rhs_vec(x, n); rt = rhs_vec(rt, n); part = rhs_part(part);
    C<T> g[L + 1];
#pragma unroll
    for (int j = 1; j <= L; ++j) g[j] = to_t<T>(st->s[S_G1 + j - 1]);
    DotAcc<T> nr, rr;
    nr.init(); rr.init();
    vec_loop(n,
             [&](int64_t k) {
                 VN<T, 2 * L + 4> a;
#pragma unroll
                 for (int i = 0; i <= L; ++i) { a.v[i] = r[i][k]; a.v[L + 1 + i] = u[i][k]; }
                 a.v[2 * L + 2] = x[k];
                 a.v[2 * L + 3] = rt[k];
                 return a;
             },
             [&](int64_t k, const VN<T, 2 * L + 4>& a) {
                 C<T> xi = a.v[2 * L + 2], ri = a.v[0], ui = a.v[L + 1];
#pragma unroll
                 for (int j = 1; j <= L; ++j) {
                     xi = cfma<T>(g[j], a.v[j - 1], xi);
                     ri = csub<T>(ri, cmul<T>(g[j], a.v[j]));
                     ui = csub<T>(ui, cmul<T>(g[j], a.v[L + 1 + j]));
                 }
                 x[k] = xi;
                 r[0][k] = ri;
                 u[0][k] = ui;
                 nr.add(norm2c<T>(ri));
                 rr.add(cmul<T>(conjg<T>(a.v[2 * L + 3]), ri));
             });
    nr.flush(); rr.flush();
    double2 s2[2] = {nr.hi, rr.hi};
    block_partials<2>(s2, part);
}

// solves the Hermitian L x L system G g = c (G_ij for i <= j given, row i
// of the upper triangle first) by Gaussian elimination with partial
// pivoting; false when singular
__device__ bool bl_solve(int L, const double2* __restrict__ gram, double2* g) {
    double2 M[3][4];
    int q = L;
    for (int i = 0; i < L; ++i) M[i][L] = gram[i];
    for (int i = 0; i < L; ++i)
        for (int j = i; j < L; ++j) {
            const double2 v = gram[q++];
            M[i][j] = v;
            M[j][i] = make_double2(v.x, -v.y);
        }
    for (int c = 0; c < L; ++c) {
        int piv = c;
        for (int i = c + 1; i < L; ++i)
            if (hypot(M[i][c].x, M[i][c].y) > hypot(M[piv][c].x, M[piv][c].y)) piv = i;
        if (is_zero(M[piv][c])) return false;
        if (piv != c)
            for (int j = 0; j <= L; ++j) { const double2 t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
        for (int i = c + 1; i < L; ++i) {
            const double2 f = ddiv(M[i][c], M[c][c]);
            for (int j = c; j <= L; ++j) {
                const double2 t = dmul(f, M[c][j]);
                M[i][j] = make_double2(M[i][j].x - t.x, M[i][j].y - t.y);
            }
        }
    }
    for (int i = L - 1; i >= 0; --i) {
        double2 acc = M[i][L];
        for (int j = i + 1; j < L; ++j) {
            const double2 t = dmul(M[i][j], g[j]);
            acc = make_double2(acc.x - t.x, acc.y - t.y);
        }
        g[i] = ddiv(acc, M[i][i]);
        if (!finite2(g[i])) return false;
    }
    return true;
}

// step 0: beta (rho1 from the dot of step j > 0, or carried over for j = 0);
// 1: alpha; 2: the minimal-residual coefficients; 3: end of the cycle
__global__ void __launch_bounds__(kVecThreads) k_bl_scalar(KState* st, const double2* __restrict__ part,
                                                           int nparts, int step, int j, int ell) {
    st += blockIdx.x;
    part += (int64_t)blockIdx.x * nparts * kMaxRed;
    if (st->status != ST_RUN) return;
    double2 s[9];
    final_sums<9>(part, nparts, s);
    if (threadIdx.x != 0) return;
    if (step == 0) {
        const double2 rho1 = j == 0 ? st->s[S_RHO] : s[0];
        const double2 rho0 = st->s[S_RHO_OLD];
        if (!finite2(rho1)) { st->status = ST_NAN; return; }
        if (is_zero(rho0)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_BETA] = dmul(st->s[S_ALPHA], ddiv(rho1, rho0));
        st->s[S_RHO_OLD] = rho1;
    } else if (step == 1) {
        const double2 gam = s[0];
        if (!finite2(gam)) { st->status = ST_NAN; return; }
        if (is_zero(gam)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_ALPHA] = ddiv(st->s[S_RHO_OLD], gam);
    } else if (step == 2) {
        st->matvecs += 2 * ell;
        double2 g[3];
        if (!bl_solve(ell, s, g)) { st->status = ST_BREAKDOWN; return; }
        for (int q = 0; q < ell; ++q) st->s[S_G1 + q] = g[q];
        st->s[S_OMEGA] = g[ell - 1];
    } else {
        if (end_of_iteration(st, s[0].x / st->bnorm2)) return;
        const double2 om = st->s[S_OMEGA];
        if (is_zero(om)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_RHO] = s[1];                                     // rho1 of the next cycle's first step
        st->s[S_RHO_OLD] = dmul(make_double2(-om.x, -om.y), st->s[S_RHO_OLD]);
    }
}

// --------------------------------------------------------- ML(n)BiCGSTAB
// ML(n)BiCGSTAB (Yeung & Chan 1999) with n = NS left starting vectors
// Q = [r0, q_2, .., q_n].  Its residual at the end of cycle j is the unique
// vector r_j = (I - omega_j A) v_j with v_j = Omega_(j-1)(A) phi_j(A) r0,
// where phi_j (degree j n, phi_j(0) = 1) makes phi_j(A) r0 orthogonal to
// K_j(A^H, Q) and omega_j minimises ||r_j||.  It is computed here with the
// recurrences of induced dimension reduction (Sonneveld & van Gijzen 2008)
// on the same shadow space: n differences dR_i = -A dX_i of residuals, the
// n x n matrix M = Q^H dR and f = Q^H r, kept up to date as columns are
// replaced oldest first.  Per cycle, n steps with one product each build n
// new differences, then the closing step takes v = r - dR c with
// M c = f (so Q^H v = 0), t = A v, omega = t^H v / t^H t and
// r = v - omega t, which is r_j above.  Before the first cycle n
// minimal-residual steps provide the first differences.
template <typename T>
struct MLVecs {
    C<T>* dR[3];
    C<T>* dX[3];
    const C<T>* q[3];    // q[0] = r0 (per right-hand side); q[1], q[2] shared by all
};

// entry e of shadow vector i >= 1 (see include/dda.h): two SplitMix64
// outputs (Steele, Lea & Flood 2014) from the state i 2^40 + e
__device__ __forceinline__ uint64_t splitmix_out(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_ml_shadow(C<T>* __restrict__ q, int i, int64_t n) {
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += S) {
        const uint64_t st = ((uint64_t)i << 40) + (uint64_t)e;
        const uint64_t u1 = splitmix_out(st + 0x9E3779B97F4A7C15ull);
        const uint64_t u2 = splitmix_out(st + 2 * 0x9E3779B97F4A7C15ull);
        const double re = (double)(u1 >> 11) * 0x1p-52 - 1.0, im = (double)(u2 >> 11) * 0x1p-52 - 1.0;
        q[e] = mk<T>((T)re, (T)im);
    }
}

template <typename T, int NS>
__device__ __forceinline__ void ml_rows(const MLVecs<T>& w, int64_t n, const C<T>* (&q)[NS]) {
    q[0] = rhs_vec(w.q[0], n);
#pragma unroll
    for (int i = 1; i < NS; ++i) q[i] = w.q[i];
}

__device__ __forceinline__ int ml_oldest(const KState* st) { return (int)st->s[S_ML + 16].x; }

// start-up step k (minimal residual): with t = A r and omega = t^H r / t^H t,
// dX_k = omega r, dR_k = -omega t, x += dX_k, r += dR_k; partials Q^H dR_k,
// then Q^H r
template <typename T, int NS>
__global__ void __launch_bounds__(kVecThreads) k_ml_mr(const KState* st, MLVecs<T> w, C<T>* __restrict__ x,
                                                       C<T>* __restrict__ r, const C<T>* __restrict__ t, int k,
                                                       int64_t n, double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    const C<T>* q[NS];
    ml_rows<T, NS>(w, n, q);
    C<T>* dR = rhs_vec(w.dR[k], n);
    C<T>* dX = rhs_vec(w.dX[k], n);
    x = rhs_vec(x, n); r = rhs_vec(r, n); t = rhs_vec(t, n); part = rhs_part(part);
    const C<T> om = to_t<T>(st->s[S_ML + 15]);
    const C<T> nom = mk<T>(-om.x, -om.y);
    DotAcc<T> acc[2 * NS];
#pragma unroll
    for (int i = 0; i < 2 * NS; ++i) acc[i].init();
    vec_loop(n,
             [&](int64_t e) {
                 VN<T, NS + 3> a;
                 a.v[0] = r[e]; a.v[1] = t[e]; a.v[2] = x[e];
#pragma unroll
                 for (int i = 0; i < NS; ++i) a.v[3 + i] = q[i][e];
                 return a;
             },
             [&](int64_t e, const VN<T, NS + 3>& a) {
                 const C<T> dx = cmul<T>(om, a.v[0]), dr = cmul<T>(nom, a.v[1]);
                 const C<T> rn = cadd<T>(a.v[0], dr);
                 dX[e] = dx;
                 dR[e] = dr;
                 x[e] = cadd<T>(a.v[2], dx);
                 r[e] = rn;
#pragma unroll
                 for (int i = 0; i < NS; ++i) {
                     acc[i].add(cmul<T>(conjg<T>(a.v[3 + i]), dr));
                     acc[NS + i].add(cmul<T>(conjg<T>(a.v[3 + i]), rn));
                 }
             });
    double2 out[2 * NS];
#pragma unroll
    for (int i = 0; i < 2 * NS; ++i) { acc[i].flush(); out[i] = acc[i].hi; }
    block_partials<2 * NS>(out, part);
}

// inner step: dX_old = -sum_i c_i dX_i + omega (r - sum_i c_i dR_i), also
// written to dx (the column the host hands to the product)
template <typename T, int NS>
__global__ void __launch_bounds__(kVecThreads) k_ml_dx(const KState* st, MLVecs<T> w, const C<T>* __restrict__ r,
                                                       C<T>* __restrict__ dx, int64_t n) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    const C<T>* dR[NS];
    const C<T>* dX[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) { dR[i] = rhs_vec(w.dR[i], n); dX[i] = rhs_vec(w.dX[i], n); }
    C<T>* out = rhs_vec(w.dX[ml_oldest(st)], n);
    r = rhs_vec(r, n); dx = rhs_vec(dx, n);
    C<T> c[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) c[i] = to_t<T>(st->s[S_ML + 12 + i]);
    const C<T> om = to_t<T>(st->s[S_ML + 15]);
    vec_loop(n,
             [&](int64_t e) {
                 VN<T, 2 * NS + 1> a;
                 a.v[0] = r[e];
#pragma unroll
                 for (int i = 0; i < NS; ++i) { a.v[1 + i] = dR[i][e]; a.v[1 + NS + i] = dX[i][e]; }
                 return a;
             },
             [&](int64_t e, const VN<T, 2 * NS + 1>& a) {
                 C<T> v = a.v[0], d = mk<T>(0, 0);
#pragma unroll
                 for (int i = 0; i < NS; ++i) {
                     v = csub<T>(v, cmul<T>(c[i], a.v[1 + i]));
                     d = csub<T>(d, cmul<T>(c[i], a.v[1 + NS + i]));
                 }
                 const C<T> o = cfma<T>(om, v, d);
                 out[e] = o;
                 dx[e] = o;
             });
}

// inner step after u = A dx (dx = dX_old): dR_old = -u, r -= u, x += dx;
// partials Q^H dR_old
template <typename T, int NS>
__global__ void __launch_bounds__(kVecThreads) k_ml_dr(const KState* st, MLVecs<T> w, C<T>* __restrict__ x,
                                                       C<T>* __restrict__ r, const C<T>* __restrict__ u,
                                                       const C<T>* __restrict__ dX, int64_t n,
                                                       double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    const C<T>* q[NS];
    ml_rows<T, NS>(w, n, q);
    const int old = ml_oldest(st);
    C<T>* dR = rhs_vec(w.dR[old], n);
    dX = rhs_vec(dX, n);
    x = rhs_vec(x, n); r = rhs_vec(r, n); u = rhs_vec(u, n); part = rhs_part(part);
    DotAcc<T> acc[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) acc[i].init();
    vec_loop(n,
             [&](int64_t e) {
                 VN<T, NS + 4> a;
                 a.v[0] = u[e]; a.v[1] = r[e]; a.v[2] = x[e]; a.v[3] = dX[e];
#pragma unroll
                 for (int i = 0; i < NS; ++i) a.v[4 + i] = q[i][e];
                 return a;
             },
             [&](int64_t e, const VN<T, NS + 4>& a) {
                 const C<T> dr = mk<T>(-a.v[0].x, -a.v[0].y);
                 dR[e] = dr;
                 r[e] = cadd<T>(a.v[1], dr);
                 x[e] = cadd<T>(a.v[2], a.v[3]);
#pragma unroll
                 for (int i = 0; i < NS; ++i) acc[i].add(cmul<T>(conjg<T>(a.v[4 + i]), dr));
             });
    double2 out[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) { acc[i].flush(); out[i] = acc[i].hi; }
    block_partials<NS>(out, part);
}

// closing step: v = r - sum_i c_i dR_i
template <typename T, int NS>
__global__ void __launch_bounds__(kVecThreads) k_ml_v(const KState* st, MLVecs<T> w, const C<T>* __restrict__ r,
                                                      C<T>* __restrict__ v, int64_t n) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    const C<T>* dR[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) dR[i] = rhs_vec(w.dR[i], n);
    r = rhs_vec(r, n); v = rhs_vec(v, n);
    C<T> c[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) c[i] = to_t<T>(st->s[S_ML + 12 + i]);
    vec_loop(n,
             [&](int64_t e) {
                 VN<T, NS + 1> a;
                 a.v[0] = r[e];
#pragma unroll
                 for (int i = 0; i < NS; ++i) a.v[1 + i] = dR[i][e];
                 return a;
             },
             [&](int64_t e, const VN<T, NS + 1>& a) {
                 C<T> vv = a.v[0];
#pragma unroll
                 for (int i = 0; i < NS; ++i) vv = csub<T>(vv, cmul<T>(c[i], a.v[1 + i]));
                 v[e] = vv;
             });
}

// closing step after t = A v and omega: dR_old = v - r - omega t,
// dX_old = -sum_i c_i dX_i + omega v, r = v - omega t, x += dX_old;
// partials Q^H dR_old, ||r||^2
template <typename T, int NS>
__global__ void __launch_bounds__(kVecThreads) k_ml_fin(const KState* st, MLVecs<T> w, C<T>* __restrict__ x,
                                                        C<T>* __restrict__ r, const C<T>* __restrict__ v,
                                                        const C<T>* __restrict__ t, int64_t n,
                                                        double2* __restrict__ part) {
    st += blockIdx.y;
    if (st->status != ST_RUN) return;
    const C<T>* q[NS];
    ml_rows<T, NS>(w, n, q);
    const int old = ml_oldest(st);
    const C<T>* dX[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) dX[i] = rhs_vec(w.dX[i], n);
    C<T>* dRo = rhs_vec(w.dR[old], n);
    C<T>* dXo = rhs_vec(w.dX[old], n);
    x = rhs_vec(x, n); r = rhs_vec(r, n); v = rhs_vec(v, n); t = rhs_vec(t, n); part = rhs_part(part);
    C<T> c[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) c[i] = to_t<T>(st->s[S_ML + 12 + i]);
    const C<T> om = to_t<T>(st->s[S_ML + 15]);
    const C<T> nom = mk<T>(-om.x, -om.y);
    DotAcc<T> acc[NS + 1];
#pragma unroll
    for (int i = 0; i <= NS; ++i) acc[i].init();
    vec_loop(n,
             [&](int64_t e) {
                 VN<T, 2 * NS + 4> a;
                 a.v[0] = v[e]; a.v[1] = t[e]; a.v[2] = r[e]; a.v[3] = x[e];
#pragma unroll
                 for (int i = 0; i < NS; ++i) { a.v[4 + i] = dX[i][e]; a.v[4 + NS + i] = q[i][e]; }
                 return a;
             },
             [&](int64_t e, const VN<T, 2 * NS + 4>& a) {
                 const C<T> rn = cfma<T>(nom, a.v[1], a.v[0]);
                 const C<T> dr = csub<T>(rn, a.v[2]);
                 C<T> dx = cmul<T>(om, a.v[0]);
#pragma unroll
                 for (int i = 0; i < NS; ++i) dx = csub<T>(dx, cmul<T>(c[i], a.v[4 + i]));
                 dRo[e] = dr;
                 dXo[e] = dx;
                 r[e] = rn;
                 x[e] = cadd<T>(a.v[3], dx);
#pragma unroll
                 for (int i = 0; i < NS; ++i) acc[i].add(cmul<T>(conjg<T>(a.v[4 + NS + i]), dr));
                 acc[NS].add(norm2c<T>(rn));
             });
    double2 out[NS + 1];
#pragma unroll
    for (int i = 0; i <= NS; ++i) { acc[i].flush(); out[i] = acc[i].hi; }
    block_partials<NS + 1>(out, part);
}

// solves the general ns x ns system M c = f (M column-major at S_ML, f at
// S_ML + 9) by Gaussian elimination with partial pivoting; false when singular
__device__ bool ml_solve(const KState* st, int ns, double2* c) {
    double2 A[3][4];
    for (int i = 0; i < ns; ++i) {
        for (int j = 0; j < ns; ++j) A[i][j] = st->s[S_ML + 3 * j + i];
        A[i][ns] = st->s[S_ML + 9 + i];
    }
    for (int col = 0; col < ns; ++col) {
        int piv = col;
        for (int i = col + 1; i < ns; ++i)
            if (hypot(A[i][col].x, A[i][col].y) > hypot(A[piv][col].x, A[piv][col].y)) piv = i;
        if (is_zero(A[piv][col])) return false;
        if (piv != col)
            for (int j = 0; j <= ns; ++j) { const double2 tmp = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = tmp; }
        for (int i = col + 1; i < ns; ++i) {
            const double2 f = ddiv(A[i][col], A[col][col]);
            for (int j = col; j <= ns; ++j) {
                const double2 tmp = dmul(f, A[col][j]);
                A[i][j] = make_double2(A[i][j].x - tmp.x, A[i][j].y - tmp.y);
            }
        }
    }
    for (int i = ns - 1; i >= 0; --i) {
        double2 acc = A[i][ns];
        for (int j = i + 1; j < ns; ++j) {
            const double2 tmp = dmul(A[i][j], c[j]);
            acc = make_double2(acc.x - tmp.x, acc.y - tmp.y);
        }
        c[i] = ddiv(acc, A[i][i]);
        if (!finite2(c[i])) return false;
    }
    return true;
}

// step 0: omega of start-up step k from (t^H t, t^H r); 1: after start-up
// step k, M column k = partials, f = the next ns partials; 2: c = M^-1 f;
// 3: after an inner step, M column `oldest` = partials, f += them, the next
// column becomes the oldest; 4: omega from (t^H t, t^H v); 5: like 3, then
// the end of the cycle (ns + 1 products) with ||r||^2 from partial ns
__global__ void __launch_bounds__(kVecThreads) k_ml_scalar(KState* st, const double2* __restrict__ part,
                                                           int nparts, int step, int k, int ns) {
    st += blockIdx.x;
    part += (int64_t)blockIdx.x * nparts * kMaxRed;
    if (st->status != ST_RUN) return;
    double2 s[7];
    final_sums<7>(part, nparts, s);
    if (threadIdx.x != 0) return;
    if (step == 0 || step == 4) {
        const double2 tt = s[0], tv = s[1];
        if (!finite2(tt) || !finite2(tv)) { st->status = ST_NAN; return; }
        if (tt.x == 0.0) { st->status = ST_BREAKDOWN; return; }
        const double2 om = make_double2(tv.x / tt.x, tv.y / tt.x);
        if (is_zero(om)) { st->status = ST_BREAKDOWN; return; }
        st->s[S_ML + 15] = om;
    } else if (step == 1) {
        for (int i = 0; i < ns; ++i) {
            st->s[S_ML + 3 * k + i] = s[i];
            st->s[S_ML + 9 + i] = s[ns + i];
        }
        st->s[S_ML + 16] = make_double2(0.0, 0.0);
    } else if (step == 2) {
        double2 c[3];
        if (!ml_solve(st, ns, c)) { st->status = ST_BREAKDOWN; return; }
        for (int i = 0; i < ns; ++i) st->s[S_ML + 12 + i] = c[i];
    } else {
        const int old = ml_oldest(st);
        for (int i = 0; i < ns; ++i) {
            st->s[S_ML + 3 * old + i] = s[i];
            const double2 f = st->s[S_ML + 9 + i];
            st->s[S_ML + 9 + i] = make_double2(f.x + s[i].x, f.y + s[i].y);
        }
        st->s[S_ML + 16] = make_double2((double)((old + 1) % ns), 0.0);
        if (step == 5) {
            st->matvecs += ns + 1;
            end_of_iteration(st, s[ns].x / st->bnorm2);
        }
    }
}

// ------------------------------------------------------ refinement helpers
__global__ void __launch_bounds__(kVecThreads) k_norm2_c128(const double2* __restrict__ a, int64_t n,
                                                            double2* __restrict__ part) {
    a = rhs_vec(a, n); part = rhs_part(part);
    DotAcc<double> d;
    d.init();
    vec_loop(n, [&](int64_t i) { return V1<double>{a[i]}; },
             [&](int64_t, const V1<double>& q) { d.add(norm2c<double>(q.a)); });
    d.flush();
    double2 s[1] = {d.hi};
    block_partials<1>(s, part);
}

__global__ void __launch_bounds__(kVecThreads) k_resid(const double2* __restrict__ b, double2* __restrict__ r,
                                                       int64_t n, const RhsCtl* __restrict__ ctl,
                                                       double2* __restrict__ part) {
    if (ctl && ctl[blockIdx.y].skip) return;
    b = rhs_vec(b, n); r = rhs_vec(r, n); part = rhs_part(part);
    DotAcc<double> d;
    d.init();
    vec_loop(n, [&](int64_t i) { return V2<double>{b[i], r[i]}; },
             [&](int64_t i, const V2<double>& q) {
                 const double2 ri = csub<double>(q.a, q.b);
                 r[i] = ri;
                 d.add(norm2c<double>(ri));
             });
    d.flush();
    double2 s[1] = {d.hi};
    block_partials<1>(s, part);
}

// sum of the partials of each right-hand side into st[b].s[slot]
__global__ void __launch_bounds__(kVecThreads) k_slot(KState* st, const double2* __restrict__ part, int nparts,
                                                      int slot, const RhsCtl* __restrict__ ctl) {
    if (ctl && ctl[blockIdx.x].skip) return;
    st += blockIdx.x;
    part += (int64_t)blockIdx.x * nparts * kMaxRed;
    double2 s[1];
    final_sums<1>(part, nparts, s);
    if (threadIdx.x == 0) st->s[slot] = s[0];
}

__global__ void __launch_bounds__(kVecThreads) k_to_c64(const double2* __restrict__ r,
                                                        const RhsCtl* __restrict__ ctl,
                                                        float2* __restrict__ out, int64_t n) {
    const double sc = ctl[blockIdx.y].scale;
    r = rhs_vec(r, n); out = rhs_vec(out, n);
    vec_loop(n, [&](int64_t i) { return V1<double>{r[i]}; },
             [&](int64_t i, const V1<double>& q) {
                 out[i] = make_float2((float)(q.a.x * sc), (float)(q.a.y * sc));
             });
}

__global__ void __launch_bounds__(kVecThreads) k_axpy_c64(double2* __restrict__ x, const RhsCtl* __restrict__ ctl,
                                                          const float2* __restrict__ d, int64_t n) {
    const double sc = ctl[blockIdx.y].mult;
    if (sc == 0.0) return;
    x = rhs_vec(x, n); d = rhs_vec(d, n);
    vec_loop(n, [&](int64_t i) { return V1<double>{make_double2((double)d[i].x, (double)d[i].y)}; },
             [&](int64_t i, const V1<double>& q) {
                 x[i].x += sc * q.a.x;
                 x[i].y += sc * q.a.y;
             });
}

}  // namespace

// ------------------------------------------------------------- host loops
template <typename T>
static int run_matvec(MatvecView<T> mv, const C<T>* p, C<T>* y, int conj, cudaStream_t st) {
    mv.conj = conj;
    return launch_matvec<T>(mv, p, y, st);
}

// ML(n)BiCGSTAB vectors in the workspace: r = v[0], q_1 = r0 = v[1] (the
// shadow residual written by k_init), v = v[2], t = v[3], dR_i = v[4 + i],
// dX_i = v[7 + i], q_2 = v[10], q_3 = v[11] (first n elements, shared)
template <typename T>
static MLVecs<T> ml_vecs(KrylovWork<T>& ws) {
    C<T>** v = ws.v;
    return MLVecs<T>{{v[4], v[5], v[6]}, {v[7], v[8], v[9]}, {v[1], v[10], v[11]}};
}

// One cycle: the start-up steps (first cycle) or the ns inner steps, then
// the closing step with the stopping test.  Returns the kernels launched
// besides the matvec passes; rc receives a launch failure.
template <typename T, int NS>
static int64_t enqueue_ml(const MatvecView<T>& mv, KrylovWork<T>& ws, C<T>* x, int first, cudaStream_t st,
                          int& rc) {
    const int64_t n = ws.n;
    const int nb = ws.nb, gx = vec_blocks(n, nb);
    const dim3 G(gx, nb), B(kVecThreads);
    double2* part = ws.part;
    KState* ds = ws.st;
    C<T>** v = ws.v;
    C<T>*r = v[0], *vv = v[2], *t = v[3];
    const MLVecs<T> w = ml_vecs(ws);
    int64_t k = 0;
    rc = 0;
    if (first) {
        for (int q = 0; q < NS; ++q) {
            if ((rc = run_matvec<T>(mv, r, t, 0, st))) return k;
            k_dot_ts<T><<<G, B, 0, st>>>(ds, t, r, n, part);
            k_ml_scalar<<<nb, B, 0, st>>>(ds, part, gx, 0, q, NS);
            k_ml_mr<T, NS><<<G, B, 0, st>>>(ds, w, x, r, t, q, n, part);
            k_ml_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1, q, NS);
            k += 4;
        }
    } else {
        for (int q = 0; q < NS; ++q) {
            k_ml_scalar<<<nb, B, 0, st>>>(ds, part, gx, 2, 0, NS);
            k_ml_dx<T, NS><<<G, B, 0, st>>>(ds, w, r, vv, n);
            if ((rc = run_matvec<T>(mv, vv, t, 0, st))) return k;
            k_ml_dr<T, NS><<<G, B, 0, st>>>(ds, w, x, r, t, vv, n, part);
            k_ml_scalar<<<nb, B, 0, st>>>(ds, part, gx, 3, 0, NS);
            k += 4;
        }
    }
    k_ml_scalar<<<nb, B, 0, st>>>(ds, part, gx, 2, 0, NS);
    k_ml_v<T, NS><<<G, B, 0, st>>>(ds, w, r, vv, n);
    if ((rc = run_matvec<T>(mv, vv, t, 0, st))) return k;
    k_dot_ts<T><<<G, B, 0, st>>>(ds, t, vv, n, part);
    k_ml_scalar<<<nb, B, 0, st>>>(ds, part, gx, 4, 0, NS);
    k_ml_fin<T, NS><<<G, B, 0, st>>>(ds, w, x, r, vv, t, n, part);
    k_ml_scalar<<<nb, B, 0, st>>>(ds, part, gx, 5, 0, NS);
    k += 6;
    return k;
}

// the kernels of one iteration (first: the first iteration's variants)
template <typename T>
static int enqueue_iteration(int method, const MatvecView<T>& mv, KrylovWork<T>& ws, C<T>* x, int first,
                             cudaStream_t st) {
    const int64_t n = ws.n;
    const int nb = ws.nb, gx = vec_blocks(n, nb);
    const dim3 G(gx, nb), B(kVecThreads);
    double2* part = ws.part;
    KState* ds = ws.st;
    C<T>** v = ws.v;
    C<T>*r = v[0], *rt = v[1];
    int rc;
    int64_t k = 0;
    if (method == DDA_BICGSTAB) {
        C<T>*p = v[2], *vv = v[3], *s = v[4], *t = v[5];
        k_bcs_p<T><<<G, B, 0, st>>>(ds, r, p, vv, n, first);
        if ((rc = run_matvec<T>(mv, p, vv, 0, st))) return rc;
        k_dot1<T><<<G, B, 0, st>>>(ds, rt, vv, 0, n, part);
        k_bcs_scalar<<<nb, B, 0, st>>>(ds, part, gx, 0);
        k_bcs_s<T><<<G, B, 0, st>>>(ds, r, vv, s, n, part);
        k_bcs_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1);
        if ((rc = run_matvec<T>(mv, s, t, 0, st))) return rc;
        k_dot_ts<T><<<G, B, 0, st>>>(ds, t, s, n, part);
        k_bcs_scalar<<<nb, B, 0, st>>>(ds, part, gx, 2);
        k_bcs_xr<T><<<G, B, 0, st>>>(ds, x, p, s, t, r, rt, n, part);
        k_bcs_scalar<<<nb, B, 0, st>>>(ds, part, gx, 3);
        k = 9;
    } else if (method == DDA_BICG) {
        C<T>*p = v[2], *pt = v[3], *q = v[4], *qt = v[5];
        k_bicg_p<T><<<G, B, 0, st>>>(ds, r, rt, p, pt, n, first);
        if ((rc = run_matvec<T>(mv, p, q, 0, st))) return rc;
        if ((rc = run_matvec<T>(mv, pt, qt, 1, st))) return rc;
        k_dot1<T><<<G, B, 0, st>>>(ds, pt, q, 0, n, part);
        k_bicg_scalar<<<nb, B, 0, st>>>(ds, part, gx, 0, 2);
        k_bicg_update<T><<<G, B, 0, st>>>(ds, x, p, q, qt, r, rt, n, part);
        k_bicg_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1, 2);
        k = 5;
    } else if (method == DDA_BICG_SYM || method == DDA_CG) {
        // p = r + beta p (k_bcs_p with omega = 0), q = A p; CG with the
        // bilinear form runs this same recurrence
        C<T>*p = v[2], *q = v[3];
        k_bcs_p<T><<<G, B, 0, st>>>(ds, r, p, p, n, first);
        if ((rc = run_matvec<T>(mv, p, q, 0, st))) return rc;
        k_dot1<T><<<G, B, 0, st>>>(ds, p, q, 1, n, part);
        k_bicg_scalar<<<nb, B, 0, st>>>(ds, part, gx, 0, 1);
        k_cocg_update<T><<<G, B, 0, st>>>(ds, x, p, q, r, n, part);
        k_bicg_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1, 1);
        k = 5;
    } else if (method == DDA_CGS) {
        C<T>*u = v[2], *p = v[3], *q = v[4], *vh = v[5], *uh = v[6], *qh = v[7];
        k_cgs_up<T><<<G, B, 0, st>>>(ds, r, q, u, p, n, first);
        if ((rc = run_matvec<T>(mv, p, vh, 0, st))) return rc;
        k_dot1<T><<<G, B, 0, st>>>(ds, rt, vh, 0, n, part);
        k_bicg_scalar<<<nb, B, 0, st>>>(ds, part, gx, 0, 2);
        k_cgs_q<T><<<G, B, 0, st>>>(ds, u, vh, q, uh, x, n);
        if ((rc = run_matvec<T>(mv, uh, qh, 0, st))) return rc;
        k_cgs_r<T><<<G, B, 0, st>>>(ds, qh, r, rt, n, part);
        k_bicg_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1, 2);
        k = 6;
    } else if (method == DDA_TFQMR) {
        // w = r (v[0]), rt = r (v[1]); the first iteration's prologue ran in krylov_solve
        C<T>*w = v[0], *u0 = v[2], *u1 = v[3], *Au0 = v[4], *Au1 = v[5], *vv = v[6], *d = v[7];
        k_tf_u1<T><<<G, B, 0, st>>>(ds, u0, vv, u1, n);
        if ((rc = run_matvec<T>(mv, u1, Au1, 0, st))) return rc;
        k_tf_even<T><<<G, B, 0, st>>>(ds, w, Au0, u0, d, n, part);
        k_tf_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1);
        k_tf_odd<T><<<G, B, 0, st>>>(ds, x, w, Au1, u1, d, rt, n, part);
        k_tf_scalar<<<nb, B, 0, st>>>(ds, part, gx, 2);
        k_tf_next<T><<<G, B, 0, st>>>(ds, x, d, w, u1, u0, n);
        if ((rc = run_matvec<T>(mv, u0, Au0, 0, st))) return rc;
        k_tf_v<T><<<G, B, 0, st>>>(ds, Au0, Au1, vv, rt, n, 0, part);
        k_tf_scalar<<<nb, B, 0, st>>>(ds, part, gx, 3);
        k = 8;
    } else if (method >= DDA_RBICGSTAB1 && method <= DDA_RBICGSTAB3) {
        const int ell = method - DDA_RBICGSTAB1 + 1;
        BLVecs<T> w{{v[0], v[2], v[3], v[4]}, {v[5], v[6], v[7], v[8]}};
        for (int j = 0; j < ell; ++j) {
            if (j > 0) {
                k_dot1<T><<<G, B, 0, st>>>(ds, rt, w.r[j], 0, n, part);
                ++k;
            }
            k_bl_scalar<<<nb, B, 0, st>>>(ds, part, gx, 0, j, ell);
            if (j == 0) k_bl_u<T, 1><<<G, B, 0, st>>>(ds, w, n);
            else if (j == 1) k_bl_u<T, 2><<<G, B, 0, st>>>(ds, w, n);
            else k_bl_u<T, 3><<<G, B, 0, st>>>(ds, w, n);
            if ((rc = run_matvec<T>(mv, w.u[j], w.u[j + 1], 0, st))) return rc;
            k_dot1<T><<<G, B, 0, st>>>(ds, rt, w.u[j + 1], 0, n, part);
            k_bl_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1, j, ell);
            if (j == 0) k_bl_r<T, 1><<<G, B, 0, st>>>(ds, w, x, n);
            else if (j == 1) k_bl_r<T, 2><<<G, B, 0, st>>>(ds, w, x, n);
            else k_bl_r<T, 3><<<G, B, 0, st>>>(ds, w, x, n);
            if ((rc = run_matvec<T>(mv, w.r[j], w.r[j + 1], 0, st))) return rc;
            k += 5;
        }
        if (ell == 1) k_bl_gram<T, 1><<<G, B, 0, st>>>(ds, w, n, part);
        else if (ell == 2) k_bl_gram<T, 2><<<G, B, 0, st>>>(ds, w, n, part);
        else k_bl_gram<T, 3><<<G, B, 0, st>>>(ds, w, n, part);
        k_bl_scalar<<<nb, B, 0, st>>>(ds, part, gx, 2, 0, ell);
        if (ell == 1) k_bl_fin<T, 1><<<G, B, 0, st>>>(ds, w, x, rt, n, part);
        else if (ell == 2) k_bl_fin<T, 2><<<G, B, 0, st>>>(ds, w, x, rt, n, part);
        else k_bl_fin<T, 3><<<G, B, 0, st>>>(ds, w, x, rt, n, part);
        k_bl_scalar<<<nb, B, 0, st>>>(ds, part, gx, 3, 0, ell);
        k += 4;
    } else if (method >= DDA_MLBICGSTAB1 && method <= DDA_MLBICGSTAB3) {
        const int ns = method - DDA_MLBICGSTAB1 + 1;
        if (ns == 1) k = enqueue_ml<T, 1>(mv, ws, x, first, st, rc);
        else if (ns == 2) k = enqueue_ml<T, 2>(mv, ws, x, first, st, rc);
        else k = enqueue_ml<T, 3>(mv, ws, x, first, st, rc);
        if (rc) return rc;
    } else if (method == DDA_QMR_SYM) {
        C<T>*vt = v[1], *vv = v[3], *p = v[5], *pt = v[7], *d = v[8], *s = v[9];
        k_qs_v<T><<<G, B, 0, st>>>(ds, vt, vv, n, part);
        k_qmr_scalar<<<nb, B, 0, st>>>(ds, part, gx, 0, first, 1);
        k_qs_p<T><<<G, B, 0, st>>>(ds, vv, p, n, first);
        if ((rc = run_matvec<T>(mv, p, pt, 0, st))) return rc;
        k_dot1<T><<<G, B, 0, st>>>(ds, p, pt, 1, n, part);
        k_qmr_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1, first, 1);
        k_qs_vt<T><<<G, B, 0, st>>>(ds, pt, vv, vt, n, part);
        k_qmr_scalar<<<nb, B, 0, st>>>(ds, part, gx, 2, first, 1);
        k_qmr_ds<T><<<G, B, 0, st>>>(ds, p, pt, d, s, x, r, n, first, part);
        k_qmr_scalar<<<nb, B, 0, st>>>(ds, part, gx, 3, first, 1);
        k = 9;
    } else {
        C<T>*vt = v[1], *wt = v[2], *vv = v[3], *w = v[4], *p = v[5], *q = v[6], *pt = v[7], *d = v[8],
            *s = v[9];
        k_qmr_vw<T><<<G, B, 0, st>>>(ds, vt, wt, vv, w, n, part);
        k_qmr_scalar<<<nb, B, 0, st>>>(ds, part, gx, 0, first, 0);
        k_qmr_pq<T><<<G, B, 0, st>>>(ds, vv, w, p, q, n, first);
        if ((rc = run_matvec<T>(mv, p, pt, 0, st))) return rc;
        k_dot1<T><<<G, B, 0, st>>>(ds, q, pt, 1, n, part);
        k_qmr_scalar<<<nb, B, 0, st>>>(ds, part, gx, 1, first, 0);
        if ((rc = run_matvec<T>(mv, q, wt, 0, st))) return rc;   // A^T q = A q
        k_qmr_vtwt<T><<<G, B, 0, st>>>(ds, pt, vv, w, vt, wt, n, part);
        k_qmr_scalar<<<nb, B, 0, st>>>(ds, part, gx, 2, first, 0);
        k_qmr_ds<T><<<G, B, 0, st>>>(ds, p, pt, d, s, x, r, n, first, part);
        k_qmr_scalar<<<nb, B, 0, st>>>(ds, part, gx, 3, first, 0);
        k = 9;
    }
    note_launches(k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "krylov iteration");
    return 0;
}

// records one steady iteration into an executable graph; false: capture
// was not possible (the iteration then runs with plain launches)
template <typename T>
static bool capture_iteration(int method, const MatvecView<T>& mv, KrylovWork<T>& ws, C<T>* x,
                              cudaGraphExec_t* exec, int64_t* kernels) {
    if (!ws.capture) return false;
    if (cudaStreamBeginCapture(ws.capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int64_t sink = 0;
    capture_launches_into(&sink);
    const int rc = enqueue_iteration<T>(method, mv, ws, x, 0, ws.capture);
    capture_launches_into(nullptr);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ws.capture, &graph);
    bool ok = rc == 0 && e == cudaSuccess && graph != nullptr;
    if (ok && cudaGraphInstantiate(exec, graph, 0) != cudaSuccess) ok = false;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        set_error("");
        return false;
    }
    *kernels = sink;
    return true;
}

template <typename T>
int krylov_solve(int method, MatvecView<T> mv, KrylovWork<T>& ws, const C<T>* b, C<T>* x, bool use_x0,
                 const RhsCtl* ctl, double tol, int max_iter, cudaStream_t st, SolveResult* res) {
    const int64_t n = ws.n;
    const int nb = ws.nb, gx = vec_blocks(n, nb);
    mv.nb = nb;
    mv.vstride = n;
    mv.status = &ws.st->status;
    mv.status_stride = kStateInts;
    C<T>** v = ws.v;
    int rc;
    // ---- initial residual (status is not yet valid: use a status-free matvec)
    C<T>* r = v[0];
    if (use_x0) {
        MatvecView<T> m0 = mv;
        m0.status = nullptr;
        if ((rc = run_matvec<T>(m0, x, r, 0, st))) return rc;
    }
    C<T>* rt = v[1];  // shadow residual (BiCG, BiCGSTAB) or vt (QMR)
    // BiCG: shadow conj(r0); BiCG_sym: rho = r^T r = conj(r)^H r, the same start
    const int conj_rt = (method == DDA_BICG || method == DDA_BICG_SYM || method == DDA_CG) ? 1 : 0;
    k_init<T><<<dim3(gx, nb), kVecThreads, 0, st>>>(b, x, r, rt, n, use_x0 ? 1 : 0, conj_rt, ws.part);
    DDA_LAUNCH_CHECK("krylov init");
    const bool bl = method >= DDA_RBICGSTAB1 && method <= DDA_RBICGSTAB3;
    const int kind = (method == DDA_QMR || method == DDA_QMR_SYM) ? 1 : method == DDA_TFQMR ? 2 : bl ? 3 : 0;
    k_init_scalar<<<nb, kVecThreads, 0, st>>>(ws.st, ws.part, gx, ctl, tol, max_iter, kind);
    DDA_LAUNCH_CHECK("krylov init scalar");
    if (method == DDA_QMR) {  // vt = r (v[1]), wt = r (v[2])
        DDA_CUDA_TRY(cudaMemcpyAsync(v[2], r, nb * n * sizeof(C<T>), cudaMemcpyDeviceToDevice, st));
    }
    if (method >= DDA_MLBICGSTAB1 && method <= DDA_MLBICGSTAB3) {   // shadow vectors q_2 .. q_n
        for (int i = 1; i <= method - DDA_MLBICGSTAB1; ++i) {
            k_ml_shadow<T><<<kVecBlocks, kVecThreads, 0, st>>>(v[9 + i], i, n);
            DDA_LAUNCH_CHECK("ML(n)BiCGSTAB shadow vectors");
        }
    }
    if (bl) {  // u_0 = 0
        DDA_CUDA_TRY(cudaMemsetAsync(v[5], 0, nb * n * sizeof(C<T>), st));
    }
    if (method == DDA_TFQMR) {  // u0 = r, d = 0, Au0 = A u0, v = Au0, first alpha
        const dim3 G(gx, nb);
        MatvecView<T> m1 = mv;
        k_tf_init<T><<<G, kVecThreads, 0, st>>>(ws.st, r, v[2], v[7], n);
        DDA_LAUNCH_CHECK("tfqmr init");
        if ((rc = run_matvec<T>(m1, v[2], v[4], 0, st))) return rc;
        k_tf_v<T><<<G, kVecThreads, 0, st>>>(ws.st, v[4], v[5], v[6], rt, n, 1, ws.part);
        DDA_LAUNCH_CHECK("tfqmr first v");
        k_tf_scalar<<<nb, kVecThreads, 0, st>>>(ws.st, ws.part, gx, 0);
        DDA_LAUNCH_CHECK("tfqmr first alpha");
    }
    // ---- iterations, polling the status words two iterations behind
    cudaEvent_t ev[2];
    DDA_CUDA_TRY(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    DDA_CUDA_TRY(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    const bool graphs = ws.capture && !(mv.prof && mv.prof->on);
    cudaGraphExec_t exec = nullptr;
    int64_t graph_kernels = 0;
    bool have_graph = false;
    int it = 0;
    bool done = false;
    rc = 0;
    // every right-hand side stops on the device after its iteration cap; the
    // two extra rounds cover the polling lag
    int cap = max_iter;
    if (ctl) {
        // caps live on the device: bound the host loop by the largest one
        RhsCtl* hc = reinterpret_cast<RhsCtl*>(ws.host);   // pinned, nb * sizeof(KState) >= nb * sizeof(RhsCtl)
        DDA_CUDA_TRY(cudaMemcpyAsync(hc, ctl, nb * sizeof(RhsCtl), cudaMemcpyDeviceToHost, st));
        DDA_CUDA_TRY(cudaStreamSynchronize(st));
        cap = 0;
        for (int q = 0; q < nb; ++q) cap = hc[q].maxit > cap ? hc[q].maxit : cap;
    }
    while (it < cap + 2 && !done) {
        ++it;
        if (it == 1) {
            rc = enqueue_iteration<T>(method, mv, ws, x, 1, st);
        } else {
            if (it == 2 && graphs) have_graph = capture_iteration<T>(method, mv, ws, x, &exec, &graph_kernels);
            if (have_graph) {
                const cudaError_t e = cudaGraphLaunch(exec, st);
                if (e != cudaSuccess) rc = cuda_fail(e, "krylov graph launch");
                else note_launches(graph_kernels);
            } else {
                rc = enqueue_iteration<T>(method, mv, ws, x, 0, st);
            }
        }
        if (rc) break;
        // copy the status words of this iteration; check the ones two behind
        const int slot = it & 1;
        int* hst = ws.host_status + slot * nb;
        if (it >= 3) {
            const cudaError_t e = cudaEventSynchronize(ev[slot]);
            if (e != cudaSuccess) { rc = cuda_fail(e, "krylov poll"); break; }
            done = true;
            for (int q = 0; q < nb; ++q)
                if (hst[q] == ST_RUN) { done = false; break; }
        }
        cudaError_t e = cudaMemcpy2DAsync(hst, sizeof(int), &ws.st->status, sizeof(KState), sizeof(int), nb,
                                          cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[slot], st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "krylov status copy"); break; }
    }
    if (exec) cudaGraphExecDestroy(exec);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    DDA_CUDA_TRY(cudaMemcpyAsync(ws.host, ws.st, nb * sizeof(KState), cudaMemcpyDeviceToHost, st));
    DDA_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < nb; ++q) {
        res[q].status = ws.host[q].status;
        res[q].iterations = ws.host[q].iter;
        res[q].matvecs = ws.host[q].matvecs + (use_x0 ? 1 : 0);
        res[q].rel2 = ws.host[q].rel2;
    }
    return 0;
}

template int krylov_solve<double>(int, MatvecView<double>, KrylovWork<double>&, const C<double>*, C<double>*,
                                  bool, const RhsCtl*, double, int, cudaStream_t, SolveResult*);
template int krylov_solve<float>(int, MatvecView<float>, KrylovWork<float>&, const C<float>*, C<float>*, bool,
                                 const RhsCtl*, double, int, cudaStream_t, SolveResult*);

int residual_from_product(const double2* b, double2* r, int64_t n, int nb, const RhsCtl* ctl, double2* part,
                          KState* st_dev, cudaStream_t st) {
    const int gx = vec_blocks(n, nb);
    k_resid<<<dim3(gx, nb), kVecThreads, 0, st>>>(b, r, n, ctl, part);
    DDA_LAUNCH_CHECK("residual");
    k_slot<<<nb, kVecThreads, 0, st>>>(st_dev, part, gx, S_TMP, ctl);
    DDA_LAUNCH_CHECK("residual final");
    return 0;
}

int vec_norm2_c128(const double2* a, int64_t n, int nb, double2* part, KState* st_dev, cudaStream_t st) {
    const int gx = vec_blocks(n, nb);
    k_norm2_c128<<<dim3(gx, nb), kVecThreads, 0, st>>>(a, n, part);
    DDA_LAUNCH_CHECK("norm");
    k_slot<<<nb, kVecThreads, 0, st>>>(st_dev, part, gx, S_TMP, nullptr);
    DDA_LAUNCH_CHECK("norm final");
    return 0;
}

int read_tmp_slots(const KState* st_dev, int nb, KState* host, double* out, cudaStream_t st) {
    DDA_CUDA_TRY(cudaMemcpy2DAsync(&host[0].s[S_TMP], sizeof(KState), &st_dev[0].s[S_TMP], sizeof(KState),
                                   sizeof(double2), nb, cudaMemcpyDeviceToHost, st));
    DDA_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < nb; ++q) out[q] = host[q].s[S_TMP].x;
    return 0;
}

int scale_to_c64(const double2* r, const RhsCtl* ctl, float2* out, int64_t n, int nb, cudaStream_t st) {
    k_to_c64<<<dim3(vec_blocks(n, nb), nb), kVecThreads, 0, st>>>(r, ctl, out, n);
    DDA_LAUNCH_CHECK("to c64");
    return 0;
}

int axpy_from_c64(double2* x, const RhsCtl* ctl, const float2* d, int64_t n, int nb, cudaStream_t st) {
    k_axpy_c64<<<dim3(vec_blocks(n, nb), nb), kVecThreads, 0, st>>>(x, ctl, d, n);
    DDA_LAUNCH_CHECK("axpy c64");
    return 0;
}

}  // namespace dda
