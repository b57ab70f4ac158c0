// Functors of the monolithic Newton-Raphson increment (Sec. 4.1, Eqs. (schemeSys)-(relax)).
//
// Unknowns q = (e, phi, E): the strain fluctuation at the actual load (Mandel, eps = E f + e),
// the damage and the load factor. A Newton vector is one array [e (NS x N) | phi (N)] plus the
// scalar E component, which the host keeps. Residuals (Eq. (aniSystem_CrackLength)):
//   R1 = P[g C : eps],  R2 = (Gc/l + 2H) phi - div(Gc l A grad phi) - 2H,  R3 = D(phi) - tau,
// H = max(psi_o + psi_ini, H^n) (without history: psi_o + psi_ini). Jacobian applied to
// (ve, vphi, vE) (Eq. (aniCrackLength_linearization)):
//   J1 = P[g C : (ve + f vE) + g'(phi) sigma_o vphi]
//   J2 = g'(phi) [drive >= H^n] sigma_o : (ve + f vE) + (Gc/l + 2H) vphi - div(Gc l A grad vphi)
//   J3 = sum Gc/l phi vphi - phi div(Gc l A grad vphi)          (by parts: + Gc l grad phi . A grad vphi)
// with sigma_o = C : eps the undamaged stress; ties of the history switch count as loading.
#pragma once

#include "pff_common.cuh"

namespace pff {

// The linearisation point: total strain eps = E f + e and damage phi (Mandel, per-grain C).
template <typename T, int NS>
struct NRPoint {
    const T *Cm;     // [grain][NS][NS] stiffness (rotated, crack-scaled), no degradation
    const int *gid;
    const T *e;      // [NS][N] fluctuation at the actual load
    const T *phi;    // [N]
    double E, f[NS], k;
    long long N;
    __device__ __forceinline__ void strain(long long v, double *ep) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) ep[a] = E * f[a] + (double)e[a * N + v];
    }
    __device__ __forceinline__ void stiff(long long v, const double *u, double *s) const {
        const T *C = Cm + (size_t)gid[v] * NS * NS;
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            double t = 0.0;
#pragma unroll
            for (int b = 0; b < NS; ++b) t += (double)C[a * NS + b] * u[b];
            s[a] = t;
        }
    }
};

// Mechanics prologue. Residual mode (vphi == nullptr): s = g C : eps, reduces |s|^2 (the scale
// of R1). Jacobian mode: s = g C : (ve + f vE) + g'(phi) sigma_o vphi.
template <typename T, int NS>
struct ProNRMech {
    static constexpr int NR = 1;
    bool skip_if_done;
    NRPoint<T, NS> q;
    const T *ve, *vphi;
    double vE;
    __device__ void eval(long long v, T *out, double *acc) const {
        double ep[NS], so[NS];
        q.strain(v, ep);
        q.stiff(v, ep, so);
        const double ph = (double)q.phi[v];
        const double g = (1.0 - ph) * (1.0 - ph) + q.k;
        if (!vphi) {
#pragma unroll
            for (int a = 0; a < NS; ++a) {
                const double s = g * so[a];
                out[a] = (T)s;
                acc[0] += s * s;
            }
            return;
        }
        double u[NS], cu[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) u[a] = (double)ve[a * q.N + v] + q.f[a] * vE;
        q.stiff(v, u, cu);
        const double gp = -2.0 * (1.0 - ph), dphi = (double)vphi[v];
#pragma unroll
        for (int a = 0; a < NS; ++a) out[a] = (T)(g * cu[a] + gp * so[a] * dphi);
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->scale2 = t[0]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// Store NS projected components, optionally negated; reduces |out|^2.
template <typename T, int NS>
struct EpiNRStore {
    static constexpr int NR = 1;
    bool skip_if_done;
    T *out;
    double sign;
    long long N;
    __device__ void apply(long long v, const T *val, double *acc) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            const double x = sign * (double)val[a];
            out[a * N + v] = (T)x;
            acc[0] += x * x;
        }
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->rr = t[0]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// Damage epilogue after div(K grad w) of w = phi (residual mode, vphi == nullptr) or w = vphi
// (Jacobian mode). Residual: out = -R2, reductions |R2|^2, |2H|^2, D(phi) (by parts), sum H.
// Jacobian: out = J2, reduction J3.
template <typename T, int NS>
struct EpiNRDmg {
    static constexpr int NR = 4;
    bool skip_if_done;
    NRPoint<T, NS> q;
    const T *acoef;             // Gc / l per grain
    const T *psi_ini, *Hprev;
    int history;
    const T *ve, *vphi;
    double vE;
    T *out;
    __device__ void apply(long long v, const T *val, double *acc) const {
        double ep[NS], so[NS];
        q.strain(v, ep);
        q.stiff(v, ep, so);
        double psi = 0.0;
#pragma unroll
        for (int a = 0; a < NS; ++a) psi += 0.5 * ep[a] * so[a];
        const double drive = psi + (double)psi_ini[v];
        const double hp = (double)Hprev[v];
        const double H = history ? (drive > hp ? drive : hp) : drive;
        const double ph = (double)q.phi[v];
        const double a0 = (double)acoef[q.gid[v]];
        const double dv = (double)val[0];
        if (!vphi) {
            const double R2 = (a0 + 2.0 * H) * ph - dv - 2.0 * H;
            out[v] = (T)(-R2);
            acc[0] += R2 * R2;
            acc[1] += 4.0 * H * H;
            acc[2] += 0.5 * ph * (a0 * ph - dv);
            acc[3] += H;
            return;
        }
        double J2 = (a0 + 2.0 * H) * (double)vphi[v] - dv;
        if (!history || drive >= hp) {
            double c = 0.0;
#pragma unroll
            for (int a = 0; a < NS; ++a) c += so[a] * ((double)ve[a * q.N + v] + q.f[a] * vE);
            J2 += -2.0 * (1.0 - ph) * c;
        }
        out[v] = (T)J2;
        acc[0] += a0 * ph * (double)vphi[v] - ph * dv;
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            sc->red[0] = t[0]; sc->red[1] = t[1]; sc->red[2] = t[2]; sc->red[3] = t[3];
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// Committed history of a converged Newton state: H = max(psi_o + psi_ini, H^n) (or the drive).
template <typename T, int NS>
struct PwNRHistory {
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    NRPoint<T, NS> q;
    const T *psi_ini, *Hprev;
    int history;
    T *Hout;
    __device__ void apply(long long v, double *) const {
        double ep[NS], so[NS];
        q.strain(v, ep);
        q.stiff(v, ep, so);
        double psi = 0.0;
#pragma unroll
        for (int a = 0; a < NS; ++a) psi += 0.5 * ep[a] * so[a];
        const double drive = psi + (double)psi_ini[v];
        const double hp = (double)Hprev[v];
        Hout[v] = (T)(history ? (drive > hp ? drive : hp) : drive);
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// Degraded energy norms of a strain change and of the strain (the stopping test of Eq.
// (errors_crack), as in the staggered solver): sum d:gC:d, sum eps:gC:eps, |dphi|^2, |phi|^2.
template <typename T, int NS>
struct PwNRErr {
    static constexpr int NR = 4;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    NRPoint<T, NS> q;           // at the new point
    const T *de, *dphi;         // the applied step (already scaled by the relaxation)
    double dE;
    __device__ void apply(long long v, double *acc) const {
        double ep[NS], se[NS], d[NS], sd[NS];
        q.strain(v, ep);
        q.stiff(v, ep, se);
#pragma unroll
        for (int a = 0; a < NS; ++a) d[a] = (double)de[a * q.N + v] + q.f[a] * dE;
        q.stiff(v, d, sd);
        const double ph = (double)q.phi[v];
        const double g = (1.0 - ph) * (1.0 - ph) + q.k;
        double ed = 0.0, ee = 0.0;
#pragma unroll
        for (int a = 0; a < NS; ++a) { ed += d[a] * sd[a]; ee += ep[a] * se[a]; }
        acc[0] += g * ed;
        acc[1] += g * ee;
        const double dp = (double)dphi[v];
        acc[2] += dp * dp;
        acc[3] += ph * ph;
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            sc->red[0] = t[0]; sc->red[1] = t[1]; sc->red[2] = t[2]; sc->red[3] = t[3];
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// ---- Newton vectors [e | phi] of length n = (NS + 1) N --------------------------------------------
template <typename T>
struct PwVDot {  // <a, b> and, when c is given, <c, d>
    static constexpr int NR = 2;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *a, *b, *c, *d;
    __device__ void apply(long long v, double *acc) const {
        acc[0] += (double)a[v] * (double)b[v];
        if (c) acc[1] += (double)c[v] * (double)d[v];
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->red[0] = t[0]; sc->red[1] = t[1]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

template <typename T>
struct PwVComb {  // out = ca a + cb b + cc c (b, c may be null)
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    T *out;
    const T *a, *b, *c;
    double ca, cb, cc;
    __device__ void apply(long long v, double *) const {
        double x = ca * (double)a[v];
        if (b) x += cb * (double)b[v];
        if (c) x += cc * (double)c[v];
        out[v] = (T)x;
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// Fixed pseudo-random shadow residual of BiCGSTAB: a 64-bit integer hash (splitmix64 finaliser)
// of the index, mapped to [-1, 1).
template <typename T>
struct PwVHash {
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    T *out;
    __device__ void apply(long long v, double *) const {
        unsigned long long z = (unsigned long long)v + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z = z ^ (z >> 31);
        out[v] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

}  // namespace pff
