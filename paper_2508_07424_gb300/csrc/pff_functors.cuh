// Prologue / epilogue / per-frequency functors of the spectral passes (see pff_kernels.cuh).
//
// Storage: symmetric tensors in Mandel form (xx, yy, [zz], sqrt2 yz, sqrt2 xz, sqrt2 xy), so
// the Frobenius product of Sec. 4.1 is a plain dot product and the stiffness C^r (Eq. (Crot))
// is a symmetric NS x NS matrix per grain. Field arrays are component-major [c][voxel].
#pragma once

#include <type_traits>

#include "pff_common.cuh"

namespace pff {

// Field words per voxel that a fused prologue / epilogue / pointwise functor reads plus writes: its
// algorithmic memory traffic in words of the field precision (the int32 grain id counts as one,
// per-grain tables are not counted). Functors state it as RW; 0 when they do not.
template <class F, class = void> struct rw_words_of { static constexpr int v = 0; };
template <class F> struct rw_words_of<F, std::void_t<decltype(F::RW)>> { static constexpr int v = F::RW; };
template <class F> constexpr int rw_words() { return rw_words_of<F>::v; }

template <typename T> __device__ __forceinline__ T degr(T phi, T k) {
    T a = (T)1 - phi;
    return a * a + k;  // g(phi) = (1 - phi)^2 + k, Sec. 2.1
}

// ================================ mechanics =====================================================
template <typename T, int NS>
struct MechBase {
    const T *Cm;        // [grain][NS][NS] Mandel stiffness (rotated, crack-scaled)
    const int *gid;
    const T *phi;       // damage at which the equilibrium is solved
    T k;
    long long N;
    bool skip_if_done;
    __device__ __forceinline__ void stress(long long v, const T *u, T *out) const {
        const T *C = Cm + (size_t)ldro(gid + v) * NS * NS;
        const T gp = degr(ldro(phi + v), k);
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            T s = 0;
#pragma unroll
            for (int b = 0; b < NS; ++b) s += C[a * NS + b] * u[b];
            out[a] = gp * s;
        }
    }
};

// s = g C : (f + x): the total stress of the current fluctuation; reduces |g C : f|^2.
template <typename T, int NS>
struct ProStressTotal : MechBase<T, NS> {
    static constexpr int NR = 1;
    static constexpr int RW = NS + 2;  // x; phi, gid
    const T *x;
    T f[NS];
    __device__ void eval(long long v, T *out, double *acc) const {
        T u[NS], sf[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) u[a] = f[a] + x[a * this->N + v];
        this->stress(v, u, out);
        this->stress(v, f, sf);
#pragma unroll
        for (int a = 0; a < NS; ++a) acc[0] += (double)sf[a] * (double)sf[a];
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->scale2 = t[0]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// ---- spectral tension/compression split (2D plane strain, isotropic lam, mu) ---------------------
// eps = (a, b, sqrt2 c) in Mandel form, eps_zz = 0. In-plane eigenvalues e1,2 = (a+b)/2 +- r,
// r = sqrt(((a-b)/2)^2 + c^2), eigenvectors at angle theta with cos 2theta = (a-b)/(2r),
// sin 2theta = c/r. psi+- = lam/2 <tr>+-^2 + mu sum <e_a>+-^2, sigma+- = lam <tr>+- I + 2 mu eps+-;
// the tangent uses the divided differences of <.>+- over the eigenvalue pairs.
template <typename T>
struct SplitState {
    T e1, e2, tr, C2, S2;  // eigenvalues, trace, cos 2theta, sin 2theta
};

template <typename T> __device__ __forceinline__ SplitState<T> split_eig(const T *em) {
    const T r2 = (T)0.70710678118654752440;
    const T a = em[0], b = em[1], c = em[2] * r2;
    const T d = (T)0.5 * (a - b);
    const T r = sqrt(d * d + c * c);
    SplitState<T> st;
    st.tr = a + b;
    st.e1 = (T)0.5 * st.tr + r;
    st.e2 = (T)0.5 * st.tr - r;
    if (r > (T)0) { st.C2 = d / r; st.S2 = c / r; }
    else { st.C2 = (T)1; st.S2 = (T)0; }
    return st;
}

template <typename T> __device__ __forceinline__ T pos_(T x) { return x > (T)0 ? x : (T)0; }
template <typename T> __device__ __forceinline__ T neg_(T x) { return x < (T)0 ? x : (T)0; }

// sigma+ and sigma- (Mandel) and psi+, psi- at eps (Mandel).
template <typename T>
__device__ __forceinline__ void split_sigma(const T *em, T lam, T mu, T *sp, T *sm, T &psp, T &psm) {
    const SplitState<T> q = split_eig(em);
    const T s2 = (T)1.41421356237309504880;
    // n1 n1 = 1/2 [1 + C2, S2; S2, 1 - C2], n2 n2 = 1/2 [1 - C2, -S2; -S2, 1 + C2]
    const T p1 = pos_(q.e1), p2 = pos_(q.e2), m1 = neg_(q.e1), m2 = neg_(q.e2);
    const T tp = pos_(q.tr), tm = neg_(q.tr);
    const T epxx = (T)0.5 * (p1 * ((T)1 + q.C2) + p2 * ((T)1 - q.C2));
    const T epyy = (T)0.5 * (p1 * ((T)1 - q.C2) + p2 * ((T)1 + q.C2));
    const T epxy = (T)0.5 * (p1 - p2) * q.S2;
    const T emxx = (T)0.5 * (m1 * ((T)1 + q.C2) + m2 * ((T)1 - q.C2));
    const T emyy = (T)0.5 * (m1 * ((T)1 - q.C2) + m2 * ((T)1 + q.C2));
    const T emxy = (T)0.5 * (m1 - m2) * q.S2;
    sp[0] = lam * tp + 2 * mu * epxx; sp[1] = lam * tp + 2 * mu * epyy; sp[2] = s2 * 2 * mu * epxy;
    sm[0] = lam * tm + 2 * mu * emxx; sm[1] = lam * tm + 2 * mu * emyy; sm[2] = s2 * 2 * mu * emxy;
    psp = (T)0.5 * lam * tp * tp + mu * (p1 * p1 + p2 * p2);
    psm = (T)0.5 * lam * tm * tm + mu * (m1 * m1 + m2 * m2);
}

// Directional derivative of sigma = g sigma+ + sigma- at eps along dm (both Mandel).
template <typename T>
__device__ __forceinline__ void split_tangent(const T *em, const T *dm, T lam, T mu, T g, T *out) {
    const SplitState<T> q = split_eig(em);
    const T r2 = (T)0.70710678118654752440, s2 = (T)1.41421356237309504880;
    const T c = sqrt(fmax((T)0, (T)0.5 * ((T)1 + q.C2)));
    const T sn = copysign(sqrt(fmax((T)0, (T)0.5 * ((T)1 - q.C2))), q.S2);
    const T dxx = dm[0], dyy = dm[1], dxy = dm[2] * r2;
    const T cs = c * sn, cc = c * c, ss = sn * sn;
    const T P11 = cc * dxx + 2 * cs * dxy + ss * dyy;
    const T P22 = ss * dxx - 2 * cs * dxy + cc * dyy;
    const T P12 = -cs * dxx + (cc - ss) * dxy + cs * dyy;
    const T trd = dxx + dyy;
    T res[3] = {0, 0, 0};
    for (int part = 0; part < 2; ++part) {
        const bool plus = part == 0;
        const T f1 = plus ? pos_(q.e1) : neg_(q.e1), f2 = plus ? pos_(q.e2) : neg_(q.e2);
        const T d1 = plus ? (T)(q.e1 > 0) : (T)(q.e1 < 0), d2 = plus ? (T)(q.e2 > 0) : (T)(q.e2 < 0);
        const T qq = (q.e1 == q.e2) ? d1 : (f1 - f2) / (q.e1 - q.e2);
        const T ht = plus ? (T)(q.tr > 0) : (T)(q.tr < 0);
        // DF = d1 P11 n1n1 + d2 P22 n2n2 + qq P12 (n1n2 + n2n1)
        const T Fxx = (T)0.5 * (d1 * P11 * ((T)1 + q.C2) + d2 * P22 * ((T)1 - q.C2)) - qq * P12 * q.S2;
        const T Fyy = (T)0.5 * (d1 * P11 * ((T)1 - q.C2) + d2 * P22 * ((T)1 + q.C2)) + qq * P12 * q.S2;
        const T Fxy = (T)0.5 * (d1 * P11 - d2 * P22) * q.S2 + qq * P12 * q.C2;
        const T w = plus ? g : (T)1;
        res[0] += w * (lam * ht * trd + 2 * mu * Fxx);
        res[1] += w * (lam * ht * trd + 2 * mu * Fyy);
        res[2] += w * (2 * mu * Fxy);
    }
    out[0] = res[0]; out[1] = res[1]; out[2] = s2 * res[2];
}

// s = sigma(f + x) with the split; reduces |sigma|^2 (the scale of the Newton stopping test).
template <typename T>
struct ProSplitStress {
    static constexpr int NR = 1;
    bool skip_if_done;
    const T *x, *phi, *lam, *mu;
    const int *gid;
    T k;
    T f[3];
    long long N;
    __device__ void eval(long long v, T *out, double *acc) const {
        T e[3], sp[3], sm[3], pp, pm;
#pragma unroll
        for (int a = 0; a < 3; ++a) e[a] = f[a] + x[a * N + v];
        const int g = gid[v];
        split_sigma(e, lam[g], mu[g], sp, sm, pp, pm);
        const T gp = degr(phi[v], k);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            out[a] = gp * sp[a] + sm[a];
            acc[0] += (double)out[a] * (double)out[a];
        }
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->scale2 = t[0]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// Newton CG direction p = r + beta p fused with s = K(eps_k) : p (tangent frozen at eps_k).
template <typename T>
struct ProSplitDir {
    static constexpr int NR = 0;
    bool skip_if_done;
    const T *r, *epsk, *phi, *lam, *mu;
    T *p;
    const int *gid;
    T k;
    const Scal *scr;
    long long N;
    __device__ void eval(long long v, T *out, double *) const {
        const T beta = (T)scr->beta;
        T u[3], e[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const size_t i = a * N + v;
            u[a] = r[i] + beta * p[i];
            p[i] = u[a];
            e[a] = epsk[i];
        }
        const int g = gid[v];
        split_tangent(e, u, lam[g], mu[g], degr(phi[v], k), out);
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// Frequency tables xi~ (Nyquist zeroed) per axis, in the field precision: x over the padded
// half-spectrum columns (zero on padding), y and z over the full axes.
template <typename R>
struct XiTab {
    const R *x, *y, *z;
    __device__ __forceinline__ void get(int kx, int ky, int kz, R &a, R &b, R &c) const {
        a = x[kx]; b = y[ky]; c = z[kz];
    }
};


__device__ __forceinline__ double inv_sqrt(double v) { return rsqrt(v); }
__device__ __forceinline__ float inv_sqrt(float v) { return rsqrtf(v); }

// Symmetric-strain Galerkin projection P^ = Gamma0(lambda0 = 0, mu0 = 1/2):
// P(tau) = t (x) n + n (x) t - (n . t) n (x) n, t = tau n, n = xi~/|xi~|; zero where xi~ = 0.
// On symmetric fields P(sigma) = 0 <=> G^ : sigma = 0 with G^ of Eq. (GFourier).
template <typename C, int NS>
struct OpProj {
    typedef typename real_of<C>::type R;
    bool skip_if_done;
    XiTab<R> xi;
    __device__ void apply(const Geom &g, int kx, int ky, int kz, const C *in, C *out) const {
        R xx, xy, xz;
        xi.get(kx, ky, kz, xx, xy, xz);
        const R q2 = xx * xx + xy * xy + xz * xz;
        if (q2 == (R)0) {
#pragma unroll
            for (int a = 0; a < NS; ++a) { out[a].x = 0; out[a].y = 0; }
            return;
        }
        const R iq = inv_sqrt(q2);
        const R n0 = xx * iq, n1 = xy * iq, n2 = xz * iq;
        const R r2 = (R)0.70710678118654752440, s2 = (R)1.41421356237309504880;
        if constexpr (NS == 3) {
            const R ax = in[0].x, ay = in[0].y, bx = in[1].x, by = in[1].y;
            const R cx = in[2].x * r2, cy = in[2].y * r2;
            const R t0x = ax * n0 + cx * n1, t0y = ay * n0 + cy * n1;
            const R t1x = cx * n0 + bx * n1, t1y = cy * n0 + by * n1;
            const R sx = t0x * n0 + t1x * n1, sy = t0y * n0 + t1y * n1;
            out[0].x = 2 * t0x * n0 - sx * n0 * n0; out[0].y = 2 * t0y * n0 - sy * n0 * n0;
            out[1].x = 2 * t1x * n1 - sx * n1 * n1; out[1].y = 2 * t1y * n1 - sy * n1 * n1;
            const R ox = t0x * n1 + t1x * n0 - sx * n0 * n1, oy = t0y * n1 + t1y * n0 - sy * n0 * n1;
            out[2].x = ox * s2; out[2].y = oy * s2;
        } else {
            R trx[3][3], tiy[3][3];
            const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const R w = a < 3 ? (R)1 : r2;
                trx[ii[a]][jj[a]] = trx[jj[a]][ii[a]] = in[a].x * w;
                tiy[ii[a]][jj[a]] = tiy[jj[a]][ii[a]] = in[a].y * w;
            }
            const R n[3] = {n0, n1, n2};
            R tx[3], ty[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                tx[i] = trx[i][0] * n[0] + trx[i][1] * n[1] + trx[i][2] * n[2];
                ty[i] = tiy[i][0] * n[0] + tiy[i][1] * n[1] + tiy[i][2] * n[2];
            }
            const R sx = tx[0] * n[0] + tx[1] * n[1] + tx[2] * n[2];
            const R sy = ty[0] * n[0] + ty[1] * n[1] + ty[2] * n[2];
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const int i = ii[a], j = jj[a];
                const R w = a < 3 ? (R)1 : s2;
                out[a].x = w * (tx[i] * n[j] + n[i] * tx[j] - sx * n[i] * n[j]);
                out[a].y = w * (ty[i] * n[j] + n[i] * ty[j] - sy * n[i] * n[j]);
            }
        }
    }
};

// r = -P[g C : (f + x)]; reduces <r, r>.
template <typename T, int NS>
struct EpiMechInit {
    static constexpr int NR = 1;
    static constexpr int RW = NS;  // r
    bool skip_if_done;
    T *r;
    long long N;
    __device__ void apply(long long v, const T *val, double *acc) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            const T ra = -val[a];
            r[a * N + v] = ra;
            acc[0] += (double)ra * (double)ra;
        }
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            sc->rr = t[0]; sc->rr0 = t[0]; sc->beta = 0.0; sc->alpha = 0.0; sc->first = 1; sc->iters = 0;
            if (!(t[0] <= sc->tol2 * sc->scale2)) sc->done = 0; else sc->done = 1;
            if (!isfinite(t[0])) { sc->flag |= FLAG_NONFINITE; sc->done = 1; }
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// q = A p; reduces <p, q> and sets alpha = rr / pq.
template <typename T, int NS>
struct EpiMechQ {
    static constexpr int NR = 1;
    bool skip_if_done;
    T *q;
    const T *p;
    long long N;
    __device__ void apply(long long v, const T *val, double *acc) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            q[a * N + v] = val[a];
            acc[0] += (double)p[a * N + v] * (double)val[a];
        }
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            sc->pq = t[0];
            if (!(t[0] > 0.0) || !isfinite(t[0])) { sc->flag |= FLAG_BREAKDOWN; sc->done = 1; }
            else sc->alpha = sc->rr / t[0];
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// x += alpha p, r -= alpha q; reduces <r, r>; beta, convergence and iteration cap.
template <typename T, int NS>
struct PwMechUpdate {
    static constexpr int NR = 1;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    T *x, *r;
    const T *p, *q;
    const Scal *scr;
    long long N;
    __device__ void apply(long long v, double *acc) const {
        const T al = (T)scr->alpha;
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            const size_t i = a * N + v;
            x[i] += al * p[i];
            const T rn = r[i] - al * q[i];
            r[i] = rn;
            acc[0] += (double)rn * (double)rn;
        }
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            const double rrn = t[0];
            sc->beta = rrn / sc->rr;
            sc->rr = rrn;
            sc->iters += 1;
            if (rrn <= sc->tol2 * sc->scale2 || sc->iters >= sc->max_iters) sc->done = 1;
            if (!isfinite(rrn)) { sc->flag |= FLAG_NONFINITE; sc->done = 1; }
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// ---- single-reduction CG (Chronopoulos-Gear) for the equilibrium ----------------------------
// Iteration i holds r_i, w_i = A r_i and the scalars alpha_i, beta_i. The first pass applies
//   p_i = r_i + beta_i p_{i-1},  s_i = w_i + beta_i s_{i-1},  x += alpha_i p_i,  r_{i+1} = r_i - alpha_i s_i
// and emits the stress of r_{i+1}; after the projection the last pass stores w_{i+1} = A r_{i+1}
// and reduces gamma = <r, r> and delta = <w, r> in one go:
//   beta_{i+1} = gamma_{i+1} / gamma_i,  alpha_{i+1} = gamma_{i+1} / (delta - beta_{i+1} gamma_{i+1} / alpha_i).
// The first pass after a restart runs with alpha = beta = 0 and only computes w_0.
template <typename T, int NS>
struct ProCGCG : MechBase<T, NS> {
    static constexpr int NR = 0;
    static constexpr int RW = 9 * NS + 2;  // r, p, w, s, x read; p, s, x, r written; phi, gid
    T *x, *r, *p, *s;
    const T *w;
    const Scal *scr;
    __device__ void eval(long long v, T *out, double *) const {
        const T al = (T)scr->alpha, be = (T)scr->beta;
        T rn[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            const size_t i = a * this->N + v;
            const T ri = ldro(r + i);
            const T pi = ri + be * ldro(p + i);
            const T si = ldro(w + i) + be * ldro(s + i);
            p[i] = pi;
            s[i] = si;
            x[i] = ldro(x + i) + al * pi;
            rn[a] = ri - al * si;
            r[i] = rn[a];
        }
        this->stress(v, rn, out);
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

template <typename T, int NS>
struct EpiCGCG {
    static constexpr int NR = 2;
    static constexpr int RW = 2 * NS;  // w written, r read
    bool skip_if_done;
    T *w;
    const T *r;
    long long N;
    // FP32 path (see x_inv_body): per-thread partial sums in FP32, over the thread's voxels
    static constexpr bool FACC = true;
    __device__ void apply_f(long long v, const T *val, float *acc) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            const size_t i = a * N + v;
            w[i] = val[a];
            const float rv = (float)ldro(r + i);
            acc[0] = fmaf(rv, rv, acc[0]);
            acc[1] = fmaf((float)val[a], rv, acc[1]);
        }
    }
    __device__ void apply(long long v, const T *val, double *acc) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            const size_t i = a * N + v;
            w[i] = val[a];
            const double rv = (double)ldro(r + i);
            acc[0] += rv * rv;
            acc[1] += (double)val[a] * rv;
        }
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            const double gamma = t[0], delta = t[1];
            sc->rr = gamma;
            // converged first: an exact solve leaves r = 0 and the next step would be 0 / 0
            if (isfinite(gamma) && gamma <= sc->tol2 * sc->scale2) {
                if (!sc->first) sc->iters += 1;
                sc->first = 0;
                sc->alpha = 0.0;
                sc->done = 1;
                return;
            }
            double beta, den;
            if (sc->first) { beta = 0.0; den = delta; }
            else { beta = gamma / sc->rz; den = delta - beta * gamma / sc->alpha; }
            if (!(den > 0.0) || !isfinite(den) || !isfinite(gamma)) {
                sc->flag |= isfinite(gamma) ? FLAG_BREAKDOWN : FLAG_NONFINITE;
                sc->done = 1;
                return;
            }
            if (!sc->first) sc->iters += 1;
            sc->first = 0;
            sc->alpha = gamma / den;
            sc->beta = beta;
            sc->rz = gamma;
            if (gamma <= sc->tol2 * sc->scale2 || gamma <= sc->eta2 * sc->rr0 || sc->iters >= sc->max_iters)
                sc->done = 1;
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// ---- FP64 residual of the FP32 path (mixed-precision iterative refinement) ----------------------
// The solution x is kept in FP64; each refinement pass evaluates the true equilibrium residual
// r = -P[g(phi) C : (f + x)] in FP64 (FP64 transforms, FP64 stiffness table), stores it in FP32 as
// the start of a CG on the correction, and the correction is added to x in FP64 afterwards.
template <int NS>
struct ProStressTotal64 {
    static constexpr int NR = 1;
    static constexpr int RW = 2 * NS + 2;  // x (double: two words), phi, gid
    bool skip_if_done;
    const double *Cm;   // [grain][NS][NS], FP64
    const int *gid;
    const float *phi;
    double k;
    const double *x;
    double f[NS];
    long long N;
    __device__ void eval(long long v, double *out, double *acc) const {
        const double *C = Cm + (size_t)ldro(gid + v) * NS * NS;
        const double gp = degr((double)ldro(phi + v), k);
        double u[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) u[a] = f[a] + ldro(x + a * N + v);
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            double su = 0.0, sf = 0.0;
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                su += C[a * NS + b] * u[b];
                sf += C[a * NS + b] * f[b];
            }
            out[a] = gp * su;
            acc[0] += gp * sf * gp * sf;
        }
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->scale2 = t[0]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// r = -P[s] from the FP64 pass, stored in FP32; reduces <r, r> in FP64 and starts the CG (as
// EpiMechInit).
template <int NS>
struct EpiMechInit64 {
    static constexpr int NR = 1;
    static constexpr int RW = NS;
    bool skip_if_done;
    float *r;
    long long N;
    __device__ void apply(long long v, const double *val, double *acc) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            r[a * N + v] = (float)(-val[a]);
            acc[0] += val[a] * val[a];
        }
    }
    typedef typename EpiMechInit<double, NS>::Fin Fin;
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// psi1 = 1/2 (f + x) : C : (f + x), the undegraded energy at unit load (Eq. (elas_Ener_rot)).
template <typename T, int NS>
struct PwPsi1 {
    static constexpr int NR = 0;
    static constexpr int RW = NS + 2;  // x, gid; psi1
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *Cm, *x;
    const int *gid;
    T *psi1;
    T f[NS];
    long long N;
    __device__ void apply(long long v, double *) const {
        const T *C = Cm + (size_t)gid[v] * NS * NS;
        T u[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) u[a] = f[a] + x[a * N + v];
        T e = 0;
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            T s = 0;
#pragma unroll
            for (int b = 0; b < NS; ++b) s += C[a * NS + b] * u[b];
            e += u[a] * s;
        }
        psi1[v] = (T)0.5 * e;
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// ================================ damage =========================================================
// Operator L v = a v - div(K grad v) with a = acoef[g] + hmul H and K = Ktab[g] (symmetric d x d,
// stored xx, yy, [zz, yz, xz], xy). Damage mode: acoef = Gc/l, hmul = 2, K = Gc l A (Eq. (gamFunct));
// crack-tip enrichment mode: acoef = 1, hmul = 0, K = l^2 A (Eqs. (damini), (daminiAni)).
template <typename T>
struct DmgCoef {
    const T *acoef;
    const T *Ktab;
    const int *gid;
    T hmul;
    const T *H;
    __device__ __forceinline__ T a(long long v) const {
        return ldro(acoef + ldro(gid + v)) + (hmul != (T)0 ? hmul * ldro(H + v) : (T)0);
    }
};

// Initialise a damage solve: H_E = max(E^2 psi1 + psi_ini, H^n) (Eq. (HistoryNumIni)) or, without
// history, E^2 psi1 + psi_ini; rhs = 2 H_E (or the enrichment source phi_disc). Emits the warm
// start x. Reduces sum H and |rhs|^2.
template <typename T>
struct ProDmgInit {
    static constexpr int NR = 2;
    static constexpr int RW = 5;  // psi1, psi_ini, H^n, x read; H_E written
    bool skip_if_done;
    int mode;            // 0: damage with history, 1: damage without history, 2: fixed rhs field
    double E;
    const T *psi1, *psi_ini, *Hprev;
    T *Hcur;
    const T *rhs_field;  // mode 2
    const T *x;
    double amean, bbar;
    double hmul;
    long long N;
    __device__ void eval(long long v, T *out, double *acc) const {
        double rhs;
        if (mode == 2) {
            rhs = (double)rhs_field[v];
        } else {
            const T drive = (T)(E * E) * psi1[v] + psi_ini[v];
            const T H = (mode == 0) ? (drive > Hprev[v] ? drive : Hprev[v]) : drive;
            Hcur[v] = H;
            acc[0] += (double)H;
            rhs = 2.0 * (double)H;
        }
        acc[1] += rhs * rhs;
        out[0] = x[v];
    }
    struct Fin {
        Scal *sc;
        double amean, bbar, hmul, invN;
        __device__ void operator()(const double *t) const {
            sc->abar = amean + hmul * t[0] * invN;
            sc->bbar = bbar;
            sc->scale2 = t[1];
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc, amean, bbar, hmul, 1.0 / (double)N}; }
};

// Start of a damage solve from an x whose div(K grad x) is kept (the previous solve of the same
// control search ended at this x): the history H_E and the rhs as in ProDmgInit, then the true
// residual r = b - (a x - div) and D(x) as in EpiDmgRes, without any transform.
template <typename T>
struct PwDmgInitKept {
    static constexpr int NR = 4;
    static constexpr int RW = 8;  // psi1, psi_ini, H^n, x, div, gid; H_E, r
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    int mode;  // 0: with history, 1: without
    double E;
    const T *psi1, *psi_ini, *Hprev;
    T *Hcur;
    DmgCoef<T> co;  // co.H is Hcur
    const T *x, *divx;
    T *r;
    double amean, bbar;
    long long N;
    __device__ void apply(long long v, double *acc) const {
        const T drive = (T)(E * E) * ldro(psi1 + v) + ldro(psi_ini + v);
        const T hp = ldro(Hprev + v);
        const T H = (mode == 0) ? (drive > hp ? drive : hp) : drive;
        Hcur[v] = H;
        const T xv = ldro(x + v), dv = ldro(divx + v);
        const T a0 = ldro(co.acoef + ldro(co.gid + v));
        const T Lx = (a0 + co.hmul * H) * xv - dv;
        const T b = (T)2 * H;
        const T rv = b - Lx;
        r[v] = rv;
        acc[0] += (double)H;
        acc[1] += (double)b * (double)b;
        acc[2] += (double)rv * (double)rv;
        acc[3] += 0.5 * (double)xv * ((double)a0 * (double)xv - (double)dv);
    }
    struct Fin {
        Scal *sc;
        double amean, bbar, hmul, invN;
        __device__ void operator()(const double *t) const {
            sc->abar = amean + hmul * t[0] * invN;
            sc->bbar = bbar;
            sc->scale2 = t[1];
            sc->D = t[3];
            sc->rr = t[2]; sc->rr0 = t[2]; sc->iters = 0; sc->first = 1; sc->beta = 0.0; sc->alpha = 0.0;
            if (t[2] <= sc->tol2 * sc->scale2) sc->done = 1;
            if (!isfinite(t[2])) { sc->flag |= FLAG_NONFINITE; sc->done = 1; }
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc, amean, bbar, (double)co.hmul, 1.0 / (double)N}; }
};

template <typename T>
struct ProField {
    static constexpr int NR = 0;
    static constexpr int RW = 1;
    bool skip_if_done;
    const T *f;
    __device__ void eval(long long v, T *out, double *) const { out[0] = f[v]; }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

template <typename C, int D>
struct OpGrad {  // 1 -> D: i xi~_a v^
    typedef typename real_of<C>::type R;
    bool skip_if_done;
    XiTab<R> xi;
    __device__ void apply(const Geom &g, int kx, int ky, int kz, const C *in, C *out) const {
        R xs[3];
        xi.get(kx, ky, kz, xs[0], xs[1], xs[2]);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            out[a].x = -xs[a] * in[0].y;
            out[a].y = xs[a] * in[0].x;
        }
    }
};

template <typename C, int D>
struct OpDiv {  // D -> 1: sum_a i xi~_a q^_a
    typedef typename real_of<C>::type R;
    bool skip_if_done;
    XiTab<R> xi;
    __device__ void apply(const Geom &g, int kx, int ky, int kz, const C *in, C *out) const {
        R xs[3];
        xi.get(kx, ky, kz, xs[0], xs[1], xs[2]);
        R ox = 0, oy = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            ox -= xs[a] * in[a].y;
            oy += xs[a] * in[a].x;
        }
        out[0].x = ox;
        out[0].y = oy;
    }
};

template <typename C>
struct OpPrec {  // v^ / (abar + bbar |xi~|^2)
    typedef typename real_of<C>::type R;
    bool skip_if_done;
    const Scal *scr;
    XiTab<R> xi;
    __device__ void apply(const Geom &g, int kx, int ky, int kz, const C *in, C *out) const {
        R a, b, c;
        xi.get(kx, ky, kz, a, b, c);
        const R s = (R)1 / ((R)scr->abar + (R)scr->bbar * (a * a + b * b + c * c));
        out[0].x = in[0].x * s;
        out[0].y = in[0].y * s;
    }
};

// ---- single-reduction PCG (Chronopoulos-Gear) for the damage operator -----------------------
// Iteration i holds r_i, u_i = M^-1 r_i, w_i = L u_i and alpha_i, beta_i. The first pass applies
//   p_i = u_i + beta_i p_{i-1},  s_i = w_i + beta_i s_{i-1},  x += alpha_i p_i,  r_{i+1} = r_i - alpha_i s_i
// and transforms r_{i+1}; the spectral pass forms u^ = M^-1 r^ and i xi~ u^ together (the
// preconditioner costs no transform of its own); the middle x pass stores u and forms the flux
// K grad u; the last pass stores w = a u - div(flux) and reduces gamma = <r, u>, delta = <w, u>
// and <r, r> at once:
//   beta_{i+1} = gamma_{i+1} / gamma_i,  alpha_{i+1} = gamma_{i+1} / (delta - beta_{i+1} gamma_{i+1} / alpha_i).
template <typename T>
struct ProPCGCG {
    static constexpr int NR = 0;
    static constexpr int RW = 10;  // u, p, w, s, r, x read; p, s, x, r written
    bool skip_if_done;
    T *x, *r, *p, *s;
    const T *u, *w;
    const Scal *scr;
    __device__ void eval(long long v, T *out, double *) const {
        const T al = (T)scr->alpha, be = (T)scr->beta;
        const T pi = ldro(u + v) + be * ldro(p + v);
        const T si = ldro(w + v) + be * ldro(s + v);
        const T rn = ldro(r + v) - al * si;
        p[v] = pi;
        s[v] = si;
        x[v] = ldro(x + v) + al * pi;
        r[v] = rn;
        out[0] = rn;
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

template <typename C, int D>
struct OpPrecGrad {  // r^ -> [u^ = r^ / (abar + bbar |xi~|^2), i xi~_a u^]
    typedef typename real_of<C>::type R;
    bool skip_if_done;
    const Scal *scr;
    XiTab<R> xi;
    __device__ void apply(const Geom &g, int kx, int ky, int kz, const C *in, C *out) const {
        R xs[3];
        xi.get(kx, ky, kz, xs[0], xs[1], xs[2]);
        const R q2 = xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2];
        const R sc = (R)1 / ((R)scr->abar + (R)scr->bbar * q2);
        const R ux = in[0].x * sc, uy = in[0].y * sc;
        out[0].x = ux;
        out[0].y = uy;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            out[1 + a].x = -xs[a] * uy;
            out[1 + a].y = xs[a] * ux;
        }
    }
};

template <typename T, int D>
struct MidFluxU {  // [u, grad u] -> store u, K grad u
    static constexpr int RW = 2;  // gid; u written
    bool skip_if_done;
    const T *Ktab;
    const int *gid;
    T *u;
    __device__ void apply(long long v, const T *in, T *out) const {
        u[v] = in[0];
        const T *K = Ktab + (size_t)ldro(gid + v) * 6;
        if constexpr (D == 2) {
            out[0] = K[0] * in[1] + K[2] * in[2];
            out[1] = K[2] * in[1] + K[1] * in[2];
        } else {
            out[0] = K[0] * in[1] + K[5] * in[2] + K[4] * in[3];
            out[1] = K[5] * in[1] + K[1] * in[2] + K[3] * in[3];
            out[2] = K[4] * in[1] + K[3] * in[2] + K[2] * in[3];
        }
    }
};

template <typename T> struct DmgCoef;

template <typename T>
struct EpiPCGCG {
    static constexpr int NR = 3;
    static constexpr int RW = 5;  // gid, H, u, r read; w written
    bool skip_if_done;
    const T *acoef;
    const int *gid;
    T hmul;
    const T *H;
    const T *u, *r;
    T *w;
    __device__ void apply(long long v, const T *val, double *acc) const {
        const T a = ldro(acoef + ldro(gid + v)) + (hmul != (T)0 ? hmul * ldro(H + v) : (T)0);
        const T uv = ldro(u + v);
        const T wv = a * uv - val[0];
        const double rv = (double)ldro(r + v);
        w[v] = wv;
        acc[0] += rv * (double)uv;
        acc[1] += (double)wv * (double)uv;
        acc[2] += rv * rv;
    }
    // FP32 path (see x_inv_body): per-thread partial sums in FP32, over the thread's voxels
    static constexpr bool FACC = true;
    __device__ void apply_f(long long v, const T *val, float *acc) const {
        const T a = ldro(acoef + ldro(gid + v)) + (hmul != (T)0 ? hmul * ldro(H + v) : (T)0);
        const T uv = ldro(u + v);
        const T wv = a * uv - val[0];
        const float rv = (float)ldro(r + v);
        w[v] = wv;
        acc[0] = fmaf(rv, (float)uv, acc[0]);
        acc[1] = fmaf((float)wv, (float)uv, acc[1]);
        acc[2] = fmaf(rv, rv, acc[2]);
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            const double gamma = t[0], delta = t[1];
            sc->rr = t[2];
            // converged first: an exact solve leaves r = 0 and the next step would be 0 / 0
            if (isfinite(t[2]) && t[2] <= sc->tol2 * sc->scale2) {
                if (!sc->first) sc->iters += 1;
                sc->first = 0;
                sc->alpha = 0.0;
                sc->done = 1;
                return;
            }
            double beta, den;
            if (sc->first) { beta = 0.0; den = delta; }
            else { beta = gamma / sc->rz; den = delta - beta * gamma / sc->alpha; }
            if (!(den > 0.0) || !isfinite(den) || !isfinite(t[2])) {
                sc->flag |= isfinite(t[2]) ? FLAG_BREAKDOWN : FLAG_NONFINITE;
                sc->done = 1;
                return;
            }
            if (!sc->first) sc->iters += 1;
            sc->first = 0;
            sc->alpha = gamma / den;
            sc->beta = beta;
            sc->rz = gamma;
            if (t[2] <= sc->tol2 * sc->scale2 || sc->iters >= sc->max_iters) sc->done = 1;
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

template <typename T, int D>
struct MidFlux {  // grad v -> K grad v
    static constexpr int RW = 1;  // gid
    bool skip_if_done;
    const T *Ktab;
    const int *gid;
    __device__ void apply(long long v, const T *in, T *out) const {
        const T *K = Ktab + (size_t)ldro(gid + v) * 6;
        if constexpr (D == 2) {
            out[0] = K[0] * in[0] + K[2] * in[1];
            out[1] = K[2] * in[0] + K[1] * in[1];
        } else {
            out[0] = K[0] * in[0] + K[5] * in[1] + K[4] * in[2];
            out[1] = K[5] * in[0] + K[1] * in[1] + K[3] * in[2];
            out[2] = K[4] * in[0] + K[3] * in[1] + K[2] * in[2];
        }
    }
};

// r = rhs - (a x - div); reduces <r, r> and, in damage mode, the dissipation functional of x,
// D(x) = sum Gc/(2l) x^2 + 1/2 x . (-div(Gc l A grad x)) (Eq. (CrackLenght_ani) by parts: the
// spectral divergence is minus the adjoint of the spectral gradient), from the same operator
// application.
template <typename T>
struct EpiDmgRes {
    static constexpr int NR = 2;
    static constexpr int RW = 6;  // x, gid, H, rhs; r, div
    bool skip_if_done;
    DmgCoef<T> co;
    const T *x;
    T *r;
    const T *rhs;
    T rhs_scale;
    T *divx;  // optional: keeps div(K grad x) for a later solve from the same x
    __device__ void apply(long long v, const T *val, double *acc) const {
        const T xv = x[v];
        const T Lx = co.a(v) * xv - val[0];
        const T rv = rhs_scale * rhs[v] - Lx;
        r[v] = rv;
        if (divx) divx[v] = val[0];
        acc[0] += (double)rv * (double)rv;
        const double a0 = (double)ldro(co.acoef + ldro(co.gid + v));  // Gc / l
        acc[1] += 0.5 * (double)xv * (a0 * (double)xv - (double)val[0]);
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            sc->D = t[1];
            sc->rr = t[0]; sc->rr0 = t[0]; sc->iters = 0; sc->first = 1; sc->beta = 0.0; sc->alpha = 0.0;
            if (t[0] <= sc->tol2 * sc->scale2) sc->done = 1;
            if (!isfinite(t[0])) { sc->flag |= FLAG_NONFINITE; sc->done = 1; }
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// Dissipation functional of a converged damage solve from its residual: with L x = b - r and
// L = a0 + hmul H - div(K grad) (a0 = Gc / l, K = Gc l A), the identity
// D(x) = sum a0/2 x^2 + 1/2 x . (-div(K grad x)) = 1/2 x . (b - r) - hmul/2 H x^2 holds exactly;
// r is the solver's recursively updated residual.
template <typename T>
struct PwDmgEnergy {
    static constexpr int NR = 1;
    static constexpr int RW = 5;  // x, r, rhs, H, gid
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    DmgCoef<T> co;
    const T *x, *r, *rhs;
    double rhs_scale;
    T *divx;  // optional: div(K grad x) = a x - (b - r), kept for a later solve from the same x
    __device__ void apply(long long v, double *acc) const {
        const double xv = (double)x[v];
        const double b_r = rhs_scale * (double)rhs[v] - (double)r[v];
        acc[0] += 0.5 * xv * b_r - 0.5 * (double)co.hmul * (double)co.H[v] * xv * xv;
        if (divx) divx[v] = (T)((double)co.a(v) * xv - b_r);
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->D = t[0]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// out = a v - div (one application of the operator, no reduction).
template <typename T>
struct EpiApply {
    static constexpr int NR = 0;
    static constexpr int RW = 4;  // v, gid, H; out
    bool skip_if_done;
    DmgCoef<T> co;
    const T *v_in;
    T *out;
    __device__ void apply(long long v, const T *val, double *) const { out[v] = co.a(v) * v_in[v] - val[0]; }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// plain store of one component.
template <typename T>
struct EpiStore {
    static constexpr int NR = 0;
    static constexpr int RW = 1;
    bool skip_if_done;
    T *out;
    __device__ void apply(long long v, const T *val, double *) const { out[v] = val[0]; }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// D = sum Gc (phi^2/(2l) + l/2 grad phi . A grad phi) and Gamma (same without Gc), Eqs.
// (CrackLenght_ani), (CrackLenghtreal).
template <typename T, int D>
struct EpiDiss {
    static constexpr int NR = 2;
    static constexpr int RW = 2;  // phi, gid
    bool skip_if_done;
    const T *phi;
    const T *GcTab, *Atab;
    const int *gid;
    double ell;
    __device__ void apply(long long v, const T *gr, double *acc) const {
        const int gg = gid[v];
        const T *A = Atab + (size_t)gg * 6;
        T q;
        if constexpr (D == 2) {
            q = gr[0] * (A[0] * gr[0] + A[2] * gr[1]) + gr[1] * (A[2] * gr[0] + A[1] * gr[1]);
        } else {
            q = gr[0] * (A[0] * gr[0] + A[5] * gr[1] + A[4] * gr[2]) +
                gr[1] * (A[5] * gr[0] + A[1] * gr[1] + A[3] * gr[2]) +
                gr[2] * (A[4] * gr[0] + A[3] * gr[1] + A[2] * gr[2]);
        }
        const T p = phi[v];
        const T dens = p * p / ((T)2 * (T)ell) + (T)0.5 * (T)ell * q;
        acc[0] += (double)(GcTab[gg] * dens);
        acc[1] += (double)dens;
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->D = t[0]; sc->Gamma = t[1]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

}  // namespace pff
