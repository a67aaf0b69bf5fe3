/*
 * ofdft.h -- C-ABI of the GB300 finite-temperature orbital-free DFT library.
 *
 * The library evaluates and minimises the free-energy functional of the
 * paper's orbital-free DFT method on a periodic real-space grid:
 *
 *   F[n] = F_s^TF[n;T] + F_s^vW[n] + F_0^NL[n;T]          (Eq. 1 and Eq. 2)
 *        + E_H[n] + E_loc[n] + E_xc[n] + E_ion
 *
 * with the finite-temperature Thomas-Fermi term through Fermi-Dirac integrals
 * and their inverse, the von Weizsaecker term, the nonlocal kinetic kernel
 * K(|G|) fixed by the finite-temperature Lindhard response at the mean valence
 * density (the F_0^NL part of Eq. 2), Perdew-Zunger LDA exchange-correlation
 * (Methods, "Numerical calculations for OFDFT and KSDFT"), Hartree, a local
 * pseudopotential through ion structure factors, and the Ewald ion-ion energy.
 * The density is found by direct minimisation over sqrt(n) at fixed electron
 * number (the "SCF iterations" of the Methods section, Table 2 caption).
 *
 * Units: Hartree atomic units (Ha, bohr).  Cubic cell of side L, n^3 grid.
 *
 * Layouts (all device arrays are plain cudaMalloc'd memory owned by the
 * caller unless stated otherwise):
 *   real field   double/float [n][n][n], index (ix*n + iy)*n + iz (z fastest),
 *                point r = (L/n)*(ix, iy, iz).
 *   half spectrum complex [n][n][n/2+1] (interleaved re, im), index
 *                (kx*n + ky)*(n/2+1) + kz; integer wave numbers m in FFT order
 *                (m = k for k < n/2, m = k - n otherwise), G = (2 pi/L) m.
 *   f~(G) = (1/N) sum_r f(r) exp(-i G.r), N = n^3.
 * Element type: double for OFDFT_FP64 plans, float for OFDFT_FP32 plans
 * (FP32 bulk arithmetic with FP64 reductions, FP64 line search).
 *
 * Errors: every call returns an ofdft_status; 0 is success.  On failure the
 * outputs are left unspecified unless the call says otherwise, and
 * ofdft_last_error() returns a message (thread-local, valid until the next
 * call on the same thread).  No call aborts the process or faults the GPU on
 * invalid arguments: arguments are validated on the host first.
 *
 * Streams: calls enqueue work on the given stream (0 = legacy default).
 * Calls that return host results synchronise that stream before returning.
 * A plan is not thread-safe: one plan, one stream at a time.
 */
#ifndef OFDFT_H
#define OFDFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OFDFT_OK = 0,
    OFDFT_ERR_INVALID = 1,        /* bad argument (size, pointer, option)          */
    OFDFT_ERR_CUDA = 2,           /* a CUDA runtime call failed                    */
    OFDFT_ERR_OOM = 3,            /* device allocation failed                      */
    OFDFT_ERR_NOT_CONVERGED = 4,  /* minimiser stopped before the tolerances       */
    OFDFT_ERR_TIMEOUT = 5,        /* a bounded device wait ran out                 */
    OFDFT_ERR_NAN = 6             /* a non-finite energy or density was produced   */
} ofdft_status;

typedef enum { OFDFT_FP64 = 0, OFDFT_FP32 = 1 } ofdft_precision;

/* Which terms of F enter (bit mask); OFDFT_TERMS_ALL is the full functional.
 * Switching terms off gives the paper's ablations, e.g. TF-only. */
enum {
    OFDFT_TERM_TF = 1, OFDFT_TERM_VW = 2, OFDFT_TERM_NL = 4, OFDFT_TERM_XC = 8,
    OFDFT_TERM_HARTREE = 16, OFDFT_TERM_LOC = 32, OFDFT_TERMS_ALL = 63
};

/* The cell.  Z points to host memory and is copied by ofdft_plan_create. */
typedef struct {
    double L;            /* cubic cell side, bohr (> 0)                                */
    int n;               /* grid points per side: even, 2,3,5-smooth, 8 <= n <= 512    */
    int n_ion;           /* number of ions (>= 1)                                      */
    const double* Z;     /* host [n_ion] valence charges (> 0); N_e = sum Z            */
    double rc;           /* Gaussian smoothing radius of the local ion potential, bohr */
    double T;            /* electron temperature, Ha (> 0)                             */
} ofdft_cell;

/* Functional options. */
typedef struct {
    int precision;       /* ofdft_precision                                            */
    int terms;           /* OFDFT_TERM_* mask                                          */
    double alpha;        /* exponent a of E_NL = int int n^a K n^a (0 < a < 1)         */
    int fd64;            /* FP32 plans: 1 inverts the Fermi-Dirac integral (eta and
                            I_3/2 / I_1/2 of the finite-T Thomas-Fermi term, Eq. 1) in
                            FP64 at every grid point, from the density value as stored;
                            0 (default) uses the FP32 fit.  FP64 plans always use FP64.
                            The FP64 inversion runs on the FP64 pipe and costs about
                            as much as the rest of an evaluation at 256^3.            */
} ofdft_opts;

/* Energies in Ha (per cell) and derived scalars. */
typedef struct {
    double F_TF, E_vW, E_NL, E_H, E_loc, E_xc, E_ion;
    double F_total;      /* sum of the seven terms above                               */
    double N_e;          /* integral of the density                                    */
    double mu;           /* chemical potential int v n / N_e, Ha                       */
    double residual;     /* (int n (v - mu)^2 / N_e)^(1/2), Ha                         */
} ofdft_energies;

/* Minimiser options (L-BFGS on sqrt(n), strong-Wolfe line search). */
typedef struct {
    double tol_F_per_ion; /* |dF|/N_ion below this for 3 consecutive iterations ...   */
    double tol_residual;  /* ... and residual below this, Ha (both >= 0; 0 is never
                             met, so the minimiser runs to max_iter)                   */
    int m;                /* L-BFGS memory (1..8)                                      */
    int max_iter;         /* iteration cap                                             */
    double c1, c2;        /* Wolfe constants (sufficient decrease, curvature)          */
} ofdft_min_opts;

typedef struct {
    ofdft_energies e;
    int iterations;
    int evaluations;      /* functional evaluations (incl. line-search trials)         */
    int status;           /* OFDFT_OK or OFDFT_ERR_NOT_CONVERGED                       */
} ofdft_result;

typedef struct ofdft_plan ofdft_plan;

/* Defaults: FP64, all terms, alpha = 1/2, fd64 = 0; tol 1e-6 Ha/ion, residual 1e-4 Ha,
 * m = 8, max_iter = 1000, c1 = 1e-4, c2 = 0.9. */
void ofdft_default_opts(ofdft_opts* opts);
void ofdft_default_min_opts(ofdft_min_opts* opts);

const char* ofdft_last_error(void);
const char* ofdft_version(void);

/*
 * Create a plan for one cell: validates the cell, allocates every device
 * workspace the plan needs (FFT spectra, gradient and L-BFGS history, kernel
 * table K(|G|), reduction scratch) on the current device, and builds the
 * nonlocal kernel table from the finite-T Lindhard function at the mean density
 * (the F_0^NL kernel "that depends only on the mean valence electron density",
 * Results after Eq. 2).  Ion positions are given later by
 * ofdft_structure_factor.  Enqueued on `stream`, which is synchronised before
 * return.  *out receives the plan; on error *out is NULL.
 */
int ofdft_plan_create(const ofdft_cell* cell, const ofdft_opts* opts, void* stream,
                      ofdft_plan** out);

/* Release a plan and its device memory.  NULL is accepted; calling it twice on
 * the same pointer is the caller's error (the pointer is freed by the first). */
void ofdft_plan_destroy(ofdft_plan* plan);

/* Bytes of device memory held by a plan for this cell and these options,
 * without allocating (for admission control).  Returns 0 on invalid input. */
size_t ofdft_plan_bytes(const ofdft_cell* cell, const ofdft_opts* opts);

/*
 * Ion structure factor S(G) = sum_I exp(-i G.R_I) (the reciprocal-space ion
 * density n_i(q) of the static structure factor definition, Methods) for the
 * positions `pos` [n_ion][3] (Cartesian, bohr; wrapped into [0, L)).  `pos` is
 * host memory when pos_on_device == 0, device memory otherwise.
 * Also builds, inside the plan, the local pseudopotential
 * V_loc(G) = (1/Omega) sum_I v~_I(G) exp(-i G.R_I) with
 * v~(G) = -4 pi Z exp(-G^2 rc^2/4)/G^2, v~(0) = pi Z rc^2, and the Ewald energy.
 * S_out: device half spectrum (element type of the plan) or NULL to skip it.
 * Must be called before any energy evaluation.  Synchronises `stream`.
 */
int ofdft_structure_factor(ofdft_plan* plan, const double* pos, int pos_on_device,
                           void* S_out, void* stream);

/*
 * One functional evaluation at density `rho` (device real field, element
 * type of the plan; not modified).  Writes the potential v = dF/dn to v_out
 * (device real field, may be NULL) and the energies to *e_out (host, may be
 * NULL).  v includes v_vW = -lap(sqrt n)/(2 sqrt n), with sqrt n floored at
 * 1e-10.  Synchronises `stream` when e_out is not NULL.
 */
int ofdft_energy_potential(ofdft_plan* plan, const void* rho, void* v_out,
                           ofdft_energies* e_out, void* stream);

/*
 * As ofdft_energy_potential, without a host round trip: the energies are
 * formed on the device and written to e_dev (device memory, 11 doubles in the
 * order of ofdft_energies: F_TF, E_vW, E_NL, E_H, E_loc, E_xc, E_ion, F_total,
 * N_e, mu, residual), stream-ordered after the potential.  Does not
 * synchronise `stream`; the caller reads e_dev after its own synchronisation
 * (e.g. to keep a sequence of evaluations queued on the GPU).  The caller owns
 * e_dev; the plan's internal reduction buffers are reused by the next call on
 * the plan, so calls on one plan are ordered on one stream.
 */
int ofdft_energy_potential_async(ofdft_plan* plan, const void* rho, void* v_out, double* e_dev,
                                 void* stream);

/*
 * Minimise F over n = N_e psi^2 / int psi^2 by L-BFGS with a strong-Wolfe line
 * search.  rho_io: device real field; on entry the initial density (or NULL
 * contents ignored when start_uniform != 0, which starts from the uniform
 * density N_e/Omega); on exit the converged density.  Returns
 * OFDFT_ERR_NOT_CONVERGED (and still writes rho_io and *r) when max_iter is
 * reached or the line search fails.  Deterministic for a fixed input, plan and
 * options.  Synchronises `stream`.
 */
int ofdft_minimize(ofdft_plan* plan, void* rho_io, int start_uniform,
                   const ofdft_min_opts* o, ofdft_result* r, void* stream);

/*
 * Electron-ion static structure factor on |q| shells (Methods, S_ab(q) for one
 * snapshot): for the k-th distinct nonzero integer m^2 present on the grid
 * (k = 0 .. n_shells-1, ascending),
 *   S_ei(q_k) = (1/sqrt(N_e N_i)) < Re[ n_e(G) S*(G) ] >_{|m|^2 = m2_k},
 * n_e(G) = Omega n~(G), averaged over every G of the shell (full sphere).
 * rho: device real field.  q_out, s_out: host [n_shells] (q in 1/bohr).
 * Requires ofdft_structure_factor first.  Synchronises `stream`.
 */
int ofdft_sei_shells(ofdft_plan* plan, const void* rho, int n_shells, double* q_out,
                     double* s_out, void* stream);

/*
 * Hellmann-Feynman forces on the ions at density rho (Methods: the molecular
 * dynamics that produces the structure factors moves the ions with these
 * forces).  At fixed n only the electron-ion energy E_loc and the ion-ion
 * Ewald energy depend on the positions, so
 *   F_I = -dE_loc/dR_I - dE_ion/dR_I
 *       = -Z_I sum_{G != 0} G Im[ conj(v~(G) n~(G) + (4 pi/Omega) exp(-G^2/4eta^2)/G^2 S_Z(G))
 *                                  exp(-i G.R_I) ]  +  (Ewald real-space pair forces),
 * v~ the Gaussian-smoothed Coulomb form factor per unit charge, S_Z the
 * charge-weighted structure factor, over the same G and with the same Ewald
 * splitting as the energy of ofdft_energy_potential, so F is the exact
 * derivative of that energy at fixed rho (and, at the minimum density, the
 * total force).  The local term drops out when OFDFT_TERM_LOC is off.
 * rho: device real field (plan precision).  forces_out: host double[n_ion * 3]
 * (hartree/bohr), ion-major.  Requires ofdft_structure_factor first (the
 * positions are those of the last call).  The first call builds and keeps a G
 * list on the device.  Synchronises `stream`.
 */
int ofdft_forces(ofdft_plan* plan, const void* rho, double* forces_out, void* stream);

/*
 * Pressure P = -dF/dOmega at density rho (Results: Table 1 and Fig. 3 report
 * the pressure of warm dense hydrogen), read as the derivative under a
 * homogeneous dilation L, R_I -> lambda L, lambda R_I, n(r) -> n(r/lambda)/lambda^3
 * at fixed T and N_e.  At the minimum density this is the derivative of the
 * minimised free energy at fixed fractional ion coordinates (ion-ion term
 * included; the ideal-gas pressure of moving ions is not).  Per term:
 *   TF, xc:  (1/Omega) int (n v - f)      vW: 2 E_vW / (3 Omega)
 *   Hartree, ion:  E / (3 Omega)
 *   loc:  (1/3) sum_G Re[n~* V_loc] c(G), c = 1 - G^2 rc^2/2 (G != 0), 3 (G = 0)
 *   NL:  -(1/3) sum_G |(n^a)~|^2 [(3 - 6a) K + dK/dlambda],
 * dK/dlambda the derivative of K(|G|/lambda; nbar/lambda^3), formed from kernel
 * tables at lambda = 1 +- 2e-3, 1 +- 1e-3 (Richardson) on the first call.
 * rho: device real field.  p_out: host double[8] = {TF, vW, NL, Hartree, loc,
 * xc, ion, total} in hartree/bohr^3.  Requires ofdft_structure_factor first.
 * Synchronises `stream`.
 */
int ofdft_pressure(ofdft_plan* plan, const void* rho, double* p_out, void* stream);

/* Ion dynamics (Methods, molecular dynamics). */
typedef struct {
    double dt;            /* time step, hbar/E_h (> 0)                                  */
    double T_ion;         /* Nose-Hoover temperature, Ha; <= 0 runs NVE                 */
    double tau;           /* thermostat period, hbar/E_h (> 0 with a thermostat);
                             thermostat mass Q = g T_ion tau^2, g = 3 N_i - 3           */
    int n_shells;         /* > 0: add S_ei and S_ii on that many |q| shells every step */
    ofdft_min_opts min;   /* electronic minimisation at every step                      */
} ofdft_md_opts;

typedef struct {
    double xi;            /* Nose-Hoover friction, 1/(hbar/E_h); carried between calls */
    double s;             /* its time integral (enters the conserved quantity)         */
    int steps_done;       /* out: steps completed by the last call                     */
} ofdft_md_thermostat;

typedef struct {
    double e_pot;         /* minimised free energy at the step's positions, Ha          */
    double kinetic;       /* ion kinetic energy, Ha                                      */
    double conserved;     /* e_pot + kinetic, + Q xi^2/2 + g T_ion s with a thermostat  */
    double xi;
    int evaluations;      /* functional evaluations of the step's minimisation          */
    int iterations;
} ofdft_md_frame;

/*
 * Born-Oppenheimer molecular dynamics of the ions (Methods: NVT with a
 * Nose-Hoover thermostat; the integrator is not printed).  Velocity Verlet
 * with one Nose-Hoover variable in the symmetric Trotter splitting
 *   NH(dt/2), v += dt F/(2m), x += dt v, [electrons], v += dt F/(2m), NH(dt/2),
 *   NH(h): xi += h (2K - g T)/(2Q); v *= exp(-xi h); s += xi h; xi += h (2K - g T)/(2Q),
 * time reversible, conserving frames[].conserved to O(dt^2).  At every step
 * the electrons are minimised (o->min) at the new positions starting from the
 * previous step's density, and the forces are those of ofdft_forces.  The
 * first call minimises at the initial positions (from the uniform density when
 * start_uniform != 0, else from rho_io).
 * rho_io: device density (plan precision), in/out.  pos_io, vel_io: host
 * double[n_ion * 3] (bohr, bohr/(hbar/E_h)); positions are kept in [0, L).
 * mass: host double[n_ion] (electron masses).  th_io: thermostat state, in/out.
 * frames: host [n_steps] or NULL.  With o->n_shells > 0, q_out (host
 * [n_shells], 1/bohr) receives the shells and the step's S_ei (as
 * ofdft_sei_shells) and S_ii(q) = <|S(G)|^2>_shell / N_i are ADDED to
 * sei_sum, sii_sum (host [n_shells]): the caller divides by the steps to get
 * the trajectory averages of S_ab (Methods).  On an error (e.g. a step whose
 * minimisation does not converge: OFDFT_ERR_NOT_CONVERGED) pos_io, vel_io and
 * th_io hold the last completed step and th_io->steps_done counts the steps.
 * Synchronises `stream`.
 */
int ofdft_md_run(ofdft_plan* plan, void* rho_io, int start_uniform, double* pos_io, double* vel_io,
                 const double* mass, const ofdft_md_opts* o, ofdft_md_thermostat* th_io, int n_steps,
                 ofdft_md_frame* frames, double* q_out, double* sei_sum, double* sii_sum, void* stream);

/*
 * Batched form: minimise `count` independent snapshots (one plan each, any mix
 * of grid sizes and precisions) concurrently.  `concurrency` host workers
 * (>= 1) each own a CUDA stream on the plans' device and take the next plan,
 * largest grid first, so the kernels and host round trips of different
 * snapshots overlap on the GPU.  rhos[i] is plan i's density buffer (as in
 * ofdft_minimize); results[i] receives its result.  Every plan must have had
 * ofdft_structure_factor called.  Returns OFDFT_OK when every snapshot
 * converged, OFDFT_ERR_NOT_CONVERGED when some did not (their results say
 * which), or the first other error.  Blocks until all are done.
 */
int ofdft_minimize_batch(ofdft_plan* const* plans, void* const* rhos, int count, int start_uniform,
                         const ofdft_min_opts* o, ofdft_result* results, int concurrency);

/*
 * FFT tile schedule of a plan: tile[0] = grid rows per block of the z passes,
 * tile[1] = columns per block of the y pass, tile[2] = of the x pass (each
 * 8..64 and within shared memory).  ofdft_autotune times a few evaluations
 * for each candidate schedule on this plan and keeps the fastest; the choice
 * is cached per (grid size, precision) for the process, so later plans of the
 * same size reuse it without timing.  Requires ofdft_structure_factor first.
 * tile (may be NULL) receives the chosen schedule; us_per_eval (may be NULL)
 * the measured evaluation time, or -1 when a cached schedule was reused.
 * ofdft_set_tiles installs a schedule directly: tile[0] in 8..64, tile[1] and
 * tile[2] powers of two in 8..64, and the blocks' shared memory within the
 * 227 KB a block may use; otherwise it returns OFDFT_ERR_INVALID and keeps the
 * old schedule.  The schedule changes launch shapes only, never results
 * beyond rounding order.  (Launch shape; no counterpart in the paper.)
 */
int ofdft_autotune(ofdft_plan* plan, void* stream, int* tile, double* us_per_eval);
int ofdft_set_tiles(ofdft_plan* plan, const int* tile);

/*
 * ofdft_sei_shells_static: the same electron-ion structure factor as
 * ofdft_sei_shells, for callers that must not allocate device memory while
 * they run (a host code with a fixed, externally managed memory budget, an
 * analysis hook called inside another program's time loop, or any process that
 * forbids allocation after start-up so that nothing can fail or fragment
 * mid-run).  The paper has no counterpart; this is a library-usage variant.
 *
 * It allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * routine.  Its temporaries live in one fixed device array of about 2.5 MB that
 * every GPU loading the library holds until the process exits.  That array
 * bounds the inputs: n even, 2,3,5-smooth, 8 <= n <= 64, 1 <= n_shells <= 256;
 * larger requests return OFDFT_ERR_INVALID with a message.
 *
 * Arguments (FP64, all device pointers except `stream`):
 *   rho [n^3] density (layout as above), pos [n_ion][3] Cartesian ion
 *   positions in bohr, L cell side, n_electrons the electron count used in the
 *   1/sqrt(N_e N_i) normalisation; outputs q_out [n_shells] (1/bohr) and
 *   s_out [n_shells], the k-th distinct nonzero |m|^2 shell in ascending order.
 * The call synchronises `stream` before returning.
 *
 * Every call looks up the array's device address in the context current on
 * the calling thread (a symbol lookup, which allocates nothing), so a caller
 * that switches contexts or resets the device still gets its own copy.
 * All calls on a device share its one array, so they run one at a time: a
 * process-wide lock per device is held from the first copy into the array to
 * the final synchronisation, also when the call fails after queuing work
 * (calls from other host threads wait for it).
 */
int ofdft_sei_shells_static(const double* rho, const double* pos, int n_ion, double L, int n,
                            double n_electrons, int n_shells, double* q_out, double* s_out,
                            void* stream);

/*
 * Per-kernel launch statistics (tracing).  The paper reports only wall times
 * (Tables 2 and 3); these counters attribute device time to the library's own
 * kernels.  Launch counts are always kept.  With timing enabled, every launch
 * of the plan is bracketed by CUDA events recorded on its launch stream and the
 * device time is accumulated per kernel name; this adds host work per launch
 * but no device synchronisation.  ofdft_profile_enable resets the counters.
 * ofdft_profile_read synchronises the plan's outstanding events, fills up to
 * `max` entries of `out` (host) and sets *count to the number of kernels seen.
 */
typedef struct {
    char name[32];
    long long launches;
    double total_ms;      /* device time, 0 unless timing was enabled */
    double bytes;         /* algorithmic DRAM bytes of those launches (inputs read
                             once, outputs written once)                       */
} ofdft_kernel_stat;

int ofdft_profile_enable(ofdft_plan* plan, int timing);
int ofdft_profile_read(ofdft_plan* plan, ofdft_kernel_stat* out, int max, int* count);

#ifdef __cplusplus
}
#endif
#endif /* OFDFT_H */
