/*
 * pff_rve.h -- C ABI of the GB300 (sm_103a) FFT phase-field-fracture RVE library.
 *
 * Method: effective toughness by FFT phase-field fracture under dissipation control
 * (Aranda & Segurado, arXiv 2508.07424). One RVE handle owns the device state of one periodic
 * voxel RVE: strain fluctuation, damage phi, history H, crack-tip-enrichment energy psi_ini, the
 * load factor E and the load curve. Every step of an increment runs in the library's CUDA kernels;
 * the host only drives scalar control (load-factor search, Anderson weights, stopping tests).
 *
 * Conventions
 *   - Voxel grid n[0] x n[1] x n[2] (nx, ny, nz), voxel size h = 1; 2D problems use dim = 2,
 *     nz = 1 and plane strain. Each used extent is a power of two in [4, 1024].
 *   - Host field buffers are row-major with x fastest: index = x + nx (y + ny z).
 *   - Symmetric tensors (strain, stress, the load direction f) are passed as the six tensor
 *     components (xx, yy, zz, yz, xz, xy) -- shear NOT doubled. 2D fields carry (xx, yy, xy).
 *   - All functions return an int status (RVE_OK = 0, negative on error). Calls on one handle
 *     are stream-ordered on the handle's CUDA stream; use one host thread per handle.
 *   - Ownership: the library copies every input buffer; the caller keeps ownership of its
 *     pointers. Device memory belongs to the handle and is released by rve_destroy.
 */
#ifndef PFF_RVE_H
#define PFF_RVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rve_s *rve_handle;

enum rve_status {
    RVE_OK = 0,
    RVE_EINVAL = -1,        /* bad argument: size, NULL pointer, unsupported combination */
    RVE_ENOMEM = -2,        /* device allocation failed */
    RVE_ESTATE = -3,        /* call out of order (e.g. step before set_microstructure) */
    RVE_ENOCONV = -4,       /* an iteration hit its cap; the handle rolls back to the last increment */
    RVE_ENOROOT = -5,       /* the dissipation constraint could not be bracketed */
    RVE_ETIMEOUT = -6,      /* a device-side wait gave up */
    RVE_ENOTFRACTURED = -7, /* effective_toughness before the fracture point was reached */
    RVE_ECUDA = -8,         /* a CUDA runtime call failed */
    RVE_EBREAKDOWN = -9,    /* CG breakdown (non-positive curvature) or a non-finite scalar */
};

enum { RVE_SPLIT_NONE = 0, RVE_SPLIT_SPECTRAL = 1 };
enum { RVE_FP64 = 0, RVE_FP32R = 1 };
enum { RVE_CRACK_NONE = 0, RVE_CRACK_CTE = 1, RVE_CRACK_CPFE = 2 };

/* Field identifiers for rve_get_field / rve_set_field. Sizes are n_vox doubles for scalar
 * fields and ns * n_vox for tensor fields (ns = 3 in 2D, 6 in 3D; component-major, tensor
 * components as above). */
enum {
    RVE_FIELD_PHI = 0,      /* committed damage phi                                     */
    RVE_FIELD_H = 1,        /* committed history H (Eq. (HistoryNumIni))                 */
    RVE_FIELD_PSI_INI = 2,  /* crack-tip enrichment energy psi_ini (Eq. (Enini))         */
    RVE_FIELD_EPS = 3,      /* committed total strain E (f + eps~1)            [tensor]  */
    RVE_FIELD_SIGMA = 4,    /* committed stress sigma = g(phi) C^r : eps       [tensor]  */
    RVE_FIELD_FLUCT1 = 5,   /* unit-load strain fluctuation eps~1              [tensor]  */
    RVE_FIELD_PSI1 = 6,     /* unit-load driving energy psi_o(f + eps~1)                 */
    RVE_FIELD_PHI_TRIAL = 7 /* output of the last damage solve (rve_damage_solve)        */
};

/* Solver configuration (rve_config_default fills every field). */
typedef struct {
    int dim;               /* 2 (plane strain) or 3 */
    int n[3];              /* grid; n[2] = 1 when dim = 2; dim = 3 takes n[2] = 1 for the one-voxel-thick
                              plates of Sec. 5 (six strain components, xi_z = 0) */
    double ell;            /* phase-field length l in voxels (Eq. (CrackLenght)) */
    double k_res;          /* residual stiffness k of g(phi) = (1 - phi)^2 + k (Sec. 2.1) */
    int split;             /* RVE_SPLIT_NONE (the paper's psi_o) or RVE_SPLIT_SPECTRAL */
    int precision;         /* RVE_FP64 or RVE_FP32R */
    int history;           /* 1: H = max(psi + psi_ini, H^n) (Eq. (HistoryNumIni)); 0: no history */
    double f[6];           /* load direction f of E_M = f E (Eq. (f_defintion)); default e_y (x) e_y */
    double tol_mech;       /* equilibrium: |P[sigma]| <= tol_mech |g C : f| */
    double tol_dmg;        /* damage CG: |r| <= tol_dmg |2H| */
    double tol_root;       /* control: |D - tau| <= tol_root tau */
    double tol_stag;       /* staggered fixed point: the three ratios of Eq. (errors_crack), the strain
                              change measured in the degraded energy norm sqrt(sum d : g C : d) */
    int max_mech_iters, max_dmg_iters, max_root_evals, max_stag_iters;
    int anderson_m;        /* Anderson memory of the staggered iteration (0 = plain) */
    double fracture_ratio; /* fracture point F: Sigma^F <= ratio * max Sigma (Sec. 4.2) */
    void *stream;          /* cudaStream_t to run on; NULL: the handle creates its own */
    int solver;            /* RVE_SOLVER_STAGGERED (default): staggered fixed point with the control
                              root search; RVE_SOLVER_NEWTON: the monolithic Newton-Raphson of Sec. 4.1
                              (Eqs. (schemeSys)-(relax)) with BiCGSTAB, FP64 only (RVE_EINVAL with
                              RVE_FP32R: BiCGSTAB on the coupled single-precision system broke down
                              before its tolerance), no split; the first increment
                              (E = 0) is staggered, since at E = 0 the Jacobian does not couple E to
                              the damage. Newton steps are capped by min(max_stag_iters, 50); in
                              rve_step_result, stag_iters counts Newton steps and mech_iters
                              BiCGSTAB iterations. Both solve the same equations (same converged
                              state). */
} rve_config;

enum { RVE_SOLVER_STAGGERED = 0, RVE_SOLVER_NEWTON = 1 };

/* Microstructure (Sec. 2.2, Sec. 4.3). All pointers are host pointers, copied. */
typedef struct {
    const int32_t *grain_id; /* [n_vox] grain of each voxel, 0 <= id < n_grains */
    int n_grains;
    const double *C_cubic;   /* [n_grains][3] lattice C1111, C1122, C1212 (tensor constants) */
    const double *R;         /* [n_grains][9] row-major rotation lattice -> sample (Eq. (Crot)) */
    const double *Gc;        /* [n_grains] local toughness Gc (Eq. (CrackLenght)) */
    const double *cleave_n;  /* [n_grains][3] weak-plane normal in lattice axes, or NULL */
    const double *beta;      /* [n_grains] cleavage weight of Eq. (PFFani), or NULL (= 0) */
    int crack_kind;          /* RVE_CRACK_NONE / _CTE (tips) / _CPFE (whole crack), Sec. 4.3 */
    int crack_row;           /* crack voxels: y = crack_row, x = crack_x0 .. crack_x0+crack_len-1 */
    int crack_x0, crack_len; /* (periodic in x; all z in 3D)                                    */
    double crack_phi_M;      /* phi_M of Eq. (damini) */
    double crack_stiffness;  /* stiffness multiplier of the crack voxels ("negligible stiffness") */
} rve_micro;

/* Result of one dissipation increment (Sec. 4.1-4.2). */
typedef struct {
    int n;              /* increment index (1-based) */
    double E;           /* load factor E^n of E_M = f E */
    double Sigma;       /* Sigma^n = <sigma> : f */
    double D;           /* dissipation functional D(phi^n) (Eq. (CrackLenght_ani)) */
    double Emec;        /* elastic energy E_mec (Eq. (elas_Ener_rot)) */
    double T;           /* load-curve area T^n (Eq. (ABC)), per unit volume */
    double Gamma;       /* crack surface Gamma(phi^n) (Eq. (CrackLenghtreal)) */
    double tau;         /* prescribed dissipation tau^n */
    int mech_iters, dmg_iters, root_evals, stag_iters;
    int fractured;      /* 1 once Sigma^n <= fracture_ratio * max Sigma */
    double stag_err;    /* final staggered error of Eq. (errors_crack) */
    int flags;          /* RVE_STEP_STAGNATED: accepted at the staggered noise floor (no improvement
                           for 20 iterations, error within 1000 x tol_stag); RVE_STEP_CUTBACK: the
                           staggered iteration failed and the increment was split into halves
                           (up to 4 levels), each committed as its own load-curve point; the
                           iteration counts then cover every attempt; RVE_STEP_UNCONVERGED: even
                           the deepest split did not converge and its last staggered iterate was
                           kept (the increment is still a point of D = tau^n) */
    double G_inst;      /* instantaneous energy release rate of Eq. (Gmed),
                           V (T^n - T^{n-1}) / (Gamma^n - Gamma^{n-1}), with T^0 = 0 and Gamma^0
                           the crack surface of the initial crack; NaN when Gamma did not change */
} rve_step_result;

enum { RVE_STEP_STAGNATED = 1, RVE_STEP_CUTBACK = 2, RVE_STEP_UNCONVERGED = 4 };

/* Committed scalar state (for checkpoints and state injection in tests). */
typedef struct {
    int n;
    double E, tau, T, Sigma, Sigma_max, tau0;
    int fractured;
    double D, Gamma;    /* D(phi^n) and Gamma(phi^n) of the committed state (D = tau0, Gamma of the
                           initial crack before the first increment) */
} rve_scalars;

void rve_config_default(rve_config *cfg);

/* Check a configuration without allocating anything: the checks rve_create makes before it
 * allocates (listed there). Returns RVE_OK or RVE_EINVAL (rve_strerror / the last-error message
 * says why for the grid-size rule). rve_server_submit runs it before it copies a request. */
int rve_config_validate(const rve_config *cfg);

/* Allocate the device state of one RVE. cfg is copied. Errors: RVE_EINVAL (grid not a power of
 * two in [4, 1024], dim/nz mismatch, grid too small for one warp per x-pass CTA, i.e.
 * (nx/4) * min(128/(nx/4), ny*nz/2) < 32, ell <= 0, unsupported precision), RVE_ENOMEM, RVE_ECUDA. */
int rve_create(const rve_config *cfg, rve_handle *out);

/* Upload the microstructure and build the per-grain tables: rotated stiffness C^r (Eq. (Crot)),
 * toughness Gc and cleavage tensor A_f (Eq. (PFFani)); crack voxels take crack_stiffness x C.
 * Then build the enriched initial crack (Eqs. (damini)/(daminiAni), (Enini)): phi_ini, psi_ini,
 * H^0 = psi_ini, tau^0 = D(phi_ini), E = Sigma = T = 0. Resets the load curve.
 * Errors: RVE_EINVAL (ids out of range, split with a non-isotropic grain), RVE_ECUDA. */
int set_microstructure(rve_handle h, const rve_micro *m);

/* One increment at constant dissipation rate (with cutback, see rve_step_result.flags):
 * tau^n = tau^{n-1} + dtau, then the staggered
 * solve of Eq. (SystemDisany) -- Fourier-Galerkin CG equilibrium at unit load, the smallest
 * E >= 0 with D(phi(E)) = tau^n, FFT-preconditioned CG for phi -- until the stopping test of
 * Eq. (errors_crack); then the history update, Sigma, E_mec and the trapezoid T^n (Eq. (ABC)).
 * out may be NULL. On RVE_ENOCONV / RVE_ENOROOT / RVE_EBREAKDOWN the committed state is left as
 * it was before the call. */
int step_dissipation(rve_handle h, double dtau, rve_step_result *out);

/* One dissipation increment of each of n handles (1 <= n <= 256, distinct), in lockstep: a host
 * thread per handle runs that handle's own control (staggered loop, control search, Anderson
 * mixing) exactly as step_dissipation does, while the iteration loops of the equilibrium and
 * damage solves of all handles are launched together, one kernel launch per pass serving every
 * handle (at most 16 per launch), until each handle's own solve has converged. Each handle's
 * results are bit-identical to stepping it alone with step_dissipation. dtau[i] > 0 per handle;
 * out (NULL or n records) receives the step results. The handles must share the grid, the
 * precision and the column tiles, use the staggered solver without the energy split and have
 * timing off (else RVE_EINVAL, nothing stepped). Returns RVE_OK when every increment succeeded,
 * else the status of the lowest-index handle that failed; the other handles' increments are
 * committed all the same. Blocks until all increments are done. Not from the paper: the batching
 * pattern of this library (many RVEs per launch). */
int rve_step_batch(rve_handle *hs, int n, const double *dtau, rve_step_result *out);

/* A lockstep group for callers that step handles from threads of their own (the request server):
 * each rve_step_in_group call runs one increment of h like step_dissipation, and while it runs,
 * its solve loops are launched together with those of the other handles of the group that are
 * stepping at the same time (opportunistic batching: a solve loop joins the running batch at its
 * next chunk of iterations and leaves it as soon as it has converged; an idle group starts once
 * every stepping handle has reached a loop or 200 us after the first one did; results stay
 * bit-identical to stepping alone). Handles of one group must share grid, precision and column
 * tiles and use the staggered solver without the split (RVE_EINVAL otherwise, checked per call
 * for the handle's own configuration). The group owns a coordinator thread and a stream; destroy it only when no
 * rve_step_in_group call on it is running. */
typedef struct rve_batch_group_s *rve_batch_group;
int rve_batch_group_create(rve_batch_group *out);
int rve_step_in_group(rve_handle h, rve_batch_group g, double dtau, rve_step_result *out);
int rve_batch_group_destroy(rve_batch_group g);

/* Effective toughness of Eqs. (JaviGc)/(ABC): G = V / A_g (T^F - 1/2 Sigma^F E^F), V = voxel
 * count, A_g = (nx - crack_len) (x nz in 3D). RVE_ENOTFRACTURED until the fracture point. */
int effective_toughness(rve_handle h, double *g_eff);

/* Toughness from the dissipation functional (Eq. (CrackLenght_ani)) instead of the load curve, the
 * measure Sec. 5.1 compares against it: (D(phi^F) - D(phi^0)) / A_g. Without history (variational
 * model) the two measures agree up to the trapezoid error and the change of the enrichment energy;
 * with history the load-curve measure is the one that counts the dissipated energy.
 * RVE_ENOTFRACTURED until the fracture point. */
int effective_toughness_functional(rve_handle h, double *g_eff);

/* Copy a device field to / from a host buffer of n doubles (see RVE_FIELD_*). Setting PHI, H or
 * FLUCT1 lets a caller inject a committed state; setting PHI also copies it to the trial field. */
int rve_get_field(rve_handle h, int field, double *host, size_t n);
int rve_set_field(rve_handle h, int field, const double *host, size_t n);
int rve_get_scalars(rve_handle h, rve_scalars *s);
int rve_set_scalars(rve_handle h, const rve_scalars *s);

/* Single steps of the increment, for step-level checks against a reference:
 *  rve_mech_solve:   unit-load equilibrium (Eq. (GFourier)) at the committed phi -> FLUCT1, PSI1.
 *  rve_damage_solve: phi(E) of (Gc/l + 2 H_E) phi - div(Gc l A grad phi) = 2 H_E with
 *                    H_E = max(E^2 psi1 + psi_ini, H) (Eqs. (SystemDisanyb), (HistoryNumIni)),
 *                    warm-started from PHI_TRIAL; writes PHI_TRIAL and returns D(phi(E)).
 *  rve_dissipation:  D and Gamma of a host damage field (Eqs. (CrackLenght_ani), (CrackLenghtreal)). */
int rve_mech_solve(rve_handle h, int *iters);
int rve_damage_solve(rve_handle h, double E, double *D, int *iters);
int rve_dissipation(rve_handle h, const double *phi_host, double *D, double *Gamma);

/* Checkpoint: serialise the committed state (fields + scalars + curve) to a host buffer.
 * Call with buf = NULL to query the size in *len. rve_load restores it bit-exactly. */
int rve_save(rve_handle h, void *buf, size_t *len);
int rve_load(rve_handle h, const void *buf, size_t len);

/* Per-kernel device timing (CUDA events around every launch while enabled; rve_timing_enable
 * with on = 1 also clears what was recorded). kind selects the launches summed:
 *   0 = the mechanics projection pass (y/z FFT + projection + inverse),
 *   1 = every column pass (k_axis: projection, damage gradient / divergence / preconditioner),
 *   2 = k_x_fwd, 3 = k_x_inv, 4 = k_x_mid (the x-axis passes with their fused pointwise work),
 *   5 = k_pointwise, 6 = all launches, 7 = the FP64 residual passes of the FP32 path's
 *   equilibrium refinement (x and column passes in FP64; not counted in kinds 0-3),
 *   8 / 9 = the forward / inverse x pass of the equilibrium CG iteration (single kernels,
 *   k_x_fwd with the direction-update prologue and k_x_inv with the CG epilogue; inside 2 / 3).
 * total_ms: summed event time; launches: count; bytes_per_launch: average algorithmic bytes
 * (half-spectrum components read and written over the nx/2 + 1 columns, plus the field words
 * the fused prologue / epilogue reads and writes per voxel); flops_per_launch: average FFT flops
 * (5 L log2 L per transformed line of L points, none for pointwise kernels). While timing is on,
 * solves launch one iteration at a time (no graphs, no launch past convergence). RVE_EINVAL for
 * an unknown kind. Not from the paper: measurement support of this implementation. */
int rve_timing_enable(rve_handle h, int on);
int rve_timing_get(rve_handle h, int kind, double *total_ms, long *launches, double *bytes_per_launch);
int rve_timing_get_flops(rve_handle h, int kind, double *total_ms, long *launches, double *bytes_per_launch,
                         double *flops_per_launch);

/* Number of kernels this handle launched so far. */
long rve_launch_count(rve_handle h);

/* Column tile widths (kx columns per CTA) of the y and z FFT passes that rve_create chose for this
 * handle (*cw_z = 0 when the grid has no z pass). rve_create measures the admissible widths on the
 * handle's own buffers once per device, grid, dimension and precision, and keeps the fastest in a
 * process-wide table and a cache file of lines "<key> <cw_y> <cw_z>": $PFF_TILE_CACHE, else
 * $XDG_CACHE_HOME/pff_gb300/tiles.txt, else ~/.cache/pff_gb300/tiles.txt (not written if none can
 * be created). PFF_TILE_TUNE=0 keeps the built-in widths, PFF_TILE_CW=<y>,<z> forces admissible
 * ones (<y> alone for grids without a z pass; inadmissible values are ignored). Every column is transformed by the same code whatever the width, so results do not
 * depend on the choice. Not from the paper: a tuning aid of this implementation. */
int rve_tile_config(rve_handle h, int *cw_y, int *cw_z);

int rve_destroy(rve_handle h);
/* Message of a status; for RVE_ENOCONV, RVE_ENOROOT, RVE_EBREAKDOWN and RVE_ECUDA it is the
 * last failure recorded on the calling thread (which stage failed, with its numbers). */
const char *rve_strerror(int status);

/* ---- serving: many RVE toughness solves on one GPU --------------------------------------------
 * A request is one RVE broken by dissipation increments (Sec. 4.1-4.2) until the fracture point
 * F or n_inc increments; its result carries the effective toughness of Eqs. (JaviGc)/(ABC) when
 * F was reached. Worker threads run admitted requests concurrently, each on its own handle and
 * CUDA stream, so the work of different RVEs overlaps on the device; admission is first come
 * first served under max_inflight slots and an HBM budget checked against rve_footprint_bytes
 * (a request larger than the budget runs alone). A failing request is retired with its status
 * and the others keep running. Times are seconds since rve_server_create. */
typedef struct rve_server_s *rve_server;

typedef struct {
    long id;                 /* the id given at submission */
    int status;              /* RVE_OK or the first error of the request */
    int fractured;           /* 1 if the fracture point was reached */
    int n_done;              /* increments completed */
    double toughness;        /* G_Ceff when fractured, NaN otherwise */
    double E_last, Sigma_last, T_last, Sigma_max;
    double t_submit, t_start, t_end;
    long voxel_updates;      /* sum over increments of (CG + PCG iterations) x voxels */
} rve_request_result;

/* Device bytes one handle with this configuration holds (estimate used for admission). */
size_t rve_footprint_bytes(const rve_config *cfg);
/* max_inflight in [1, 256]; hbm_budget_bytes: admission budget over concurrently held footprints. */
int rve_server_create(int max_inflight, size_t hbm_budget_bytes, rve_server *out);
/* cfg and m are copied (cfg->stream is ignored). n_inc >= 1, dtau > 0. */
int rve_server_submit(rve_server s, long id, const rve_config *cfg, const rve_micro *m, int n_inc, double dtau);
/* Collect up to max finished results; waits up to timeout_s seconds for at least one (0: poll). */
int rve_server_wait(rve_server s, rve_request_result *out, int max, double timeout_s, int *n_out);
int rve_server_stats(rve_server s, int *peak_inflight, size_t *peak_bytes, long *pending);
/* Lockstep batching of the requests of one size class (grid, precision; staggered solver without
 * the split) through a shared rve_batch_group: on, or off (the default: every request steps on its
 * own stream, concurrently with the others, with graph-launched solve loops). Results are the same
 * either way. Set it before submitting. */
int rve_server_set_batching(rve_server s, int on);
/* Finishes every submitted request, then joins the workers. */
int rve_server_destroy(rve_server s);

/* Allocation-free D(phi) and Gamma(phi), for callers that cannot allocate device memory when
 * they need the value (a framework that owns all device memory through its own pool, a
 * latency-critical loop that must not hit the implicit synchronisation of cudaMalloc/cudaFree,
 * an embedded caller with a fixed memory budget). The paper has no counterpart: it is a service
 * entry point of this library, computing the same values as rve_dissipation.
 *   All pointers are DEVICE pointers owned by the caller: grain_id [n_vox] (x fastest), each
 *   id in [0, n_grains) (an id outside that range reads no table entry and makes out NaN),
 *   Gc [n_grains], A [n_grains][6] (cleavage tensor of Eq. (PFFani); 3D order xx, yy, zz, yz,
 *   xz, xy; 2D uses slots 0, 1, 2 for xx, yy, xy), phi [n_vox]; out [2] receives D and Gamma.
 *   stream: cudaStream_t or NULL. The call is asynchronous on that stream.
 * Scratch: one fixed 8 MiB __device__ array inside the library, held by every GPU that loads it
 * until the process exits; nothing is allocated. Grids whose spectra and partial sums do not fit
 * (e.g. 2D grids of more than 512 x 512 voxels such as 1024 x 512, 3D above 32^3) return RVE_EINVAL with a message on
 * stderr; so do grids too small for one warp per x-pass CTA (as for rve_create). Extents are
 * powers of two from 4 to 1024; dim = 3 also takes plates one voxel thick (n[2] = 1), as
 * rve_create does.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) and
 * copies a small table of FFT twiddles into the library's constant memory, so
 * make that first call before any stream capture. All calls share the array: calls that
 * overlap on the GPU (different streams, different host threads) race and must be ordered by
 * the caller. Each call clears the parts of the array it relies on. */
int rve_dissipation_noalloc(int dim, const int n[3], double ell, int n_grains, const int32_t *grain_id,
                            const double *Gc, const double *A, const double *phi, double *out, void *stream);

/* Measured FP64 fused multiply-add rate of the current device, for the roofline of the FP64
 * path (the paper has no counterpart: a measurement helper of this library). Launches one
 * warm-up and one timed kernel of 8 blocks per SM x 256 threads, each thread running 8
 * independent chains of iters x 16 FMAs, timed with CUDA events on `stream` (cudaStream_t or
 * NULL); blocks until done. tflops receives 2 x FMAs / time in TFLOP/s, ms_out (optional) the
 * kernel time. Errors: RVE_EINVAL (iters < 1, tflops NULL), RVE_ECUDA. */
int rve_fp64_fma_rate(int iters, double *tflops, double *ms_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PFF_RVE_H */
