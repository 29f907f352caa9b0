/*
 * itokmc.h -- C ABI of the GB300 Ito-KMC streamer step (libitokmc.so).
 *
 * One time step of the Ito-Kinetic-Monte-Carlo model of R. Marskar,
 * "Stochastic and self-consistent 3D modeling of streamer discharge trees
 * with Kinetic Monte Carlo" (arXiv 2307.01797), on a uniform cubic grid with
 * plane electrodes at z = lo_z (phi = 0) and z = hi_z (phi = E0 (hi_z-lo_z))
 * and homogeneous Neumann side faces.  The system solved is Eq. ito_poisson
 * (Sec. 4): particle transport Eq. ito_kernel, per-cell chemistry Eq. kmc,
 * field Eq. poisson with E = -grad phi.
 *
 * A step (itokmc_step) runs, on the handle's CUDA stream:
 *   a1  trilinear (CIC) interpolation of E to the particles      Sec. 4.2
 *   a2  explicit Euler-Maruyama push, v = -mu E                   Sec. 4.3
 *   a3  stable sort of the particles by cell
 *   a4  CIC deposition in int64 fixed point; X_e per cell         Sec. 4.2
 *   a6  per-cell KMC, Cao et al. hybrid tau-leap/SSA              Sec. 3.2.3
 *   a7  product particles (N_new = 64, Eq. w), loss removal       Sec. 4.4
 *   a8  photon emission and absorption (photoionization)          Sec. 4.5
 *   a9  kd-tree merge/split to ppc particles per cell             Sec. 4.6
 *   a5  geometric-multigrid Poisson solve for the next step's E   Sec. 4.3
 * The field is solved from the charge deposited in a4 together with the ion
 * counts before a6 (every reaction is charge neutral).
 *
 * Conventions (all entry points):
 *   - Every call returns 0 (ITOKMC_OK) or a negative ITOKMC_ERR_* code; no
 *     C++ exception crosses the ABI.  itokmc_last_error() gives the message.
 *     After ITOKMC_ERR_CUDA or ITOKMC_ERR_TIMEOUT the handle is poisoned:
 *     every later call except itokmc_last_error/itokmc_destroy returns
 *     ITOKMC_ERR_POISONED.
 *   - Units are SI.  Grid index (i, j, k) has linear cell index
 *     (k n + j) n + i (x fastest); cell i spans [lo + i h, lo + (i+1) h].
 *   - Realization r of an ensemble uses Philox key seed0 + r and owns cells
 *     r n^3 ... (r+1) n^3 - 1 of every per-cell array.
 *   - Host buffers are owned by the caller and are only read or written
 *     during the call.  Device memory is owned by the handle (allocated in
 *     itokmc_init through the caller's allocator, or cudaMallocAsync when
 *     none is given, and released by itokmc_destroy).
 *   - Calls are asynchronous on the handle's stream unless they return data
 *     to the host, in which case they synchronise that stream.
 */
#ifndef ITOKMC_H
#define ITOKMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define ITOKMC_OK 0
#define ITOKMC_ERR_ARG (-1)        /* invalid argument or configuration     */
#define ITOKMC_ERR_OOM (-2)        /* device allocation failed              */
#define ITOKMC_ERR_CUDA (-3)       /* a CUDA runtime call failed            */
#define ITOKMC_ERR_CAPACITY (-4)   /* particle capacity exceeded            */
#define ITOKMC_ERR_OVERFLOW (-5)   /* weight or fixed-point overflow        */
#define ITOKMC_ERR_NOCONV (-6)     /* multigrid did not reach its tolerance */
#define ITOKMC_ERR_TIMEOUT (-7)    /* a bounded device wait gave up         */
#define ITOKMC_ERR_POISONED (-8)   /* handle unusable after an earlier error */
#define ITOKMC_ERR_KMC (-9)        /* KMC iteration guard hit in some cell  */
#define ITOKMC_ERR_INTERNAL (-10)  /* a self-check of the library failed     */

/* ---- precision forms --------------------------------------------------- */
#define ITOKMC_FP64 0   /* FP64 positions/push/KMC, FP64 multigrid (parity) */
#define ITOKMC_MIXED 1  /* FP32 cell-relative positions, push and KMC,      */
                        /* int64 fixed-point deposit; the potential held in */
                        /* int64 fixed point, its residual formed exactly   */
                        /* and corrected by FP32 V-cycles until the FP64    */
                        /* tolerance holds; E evaluated in FP32             */

/* ---- field coupling of a step (itokmc_config.coupling) ----------------- */
#define ITOKMC_EXPLICIT 0       /* Euler-Maruyama push with the field of the  */
                                /* start of the step (Sec. 4.3, first form)   */
#define ITOKMC_SEMI_IMPLICIT 1  /* the paper's semi-implicit step (Sec. 4.3, */
                                /* Sec. 4.7 steps 1-5; FP64 form)             */

/* ---- memory kinds for host/device pointers ----------------------------- */
#define ITOKMC_HOST 0
#define ITOKMC_DEVICE 1

/* ---- fields readable with itokmc_read_densities ------------------------ */
#define ITOKMC_NE_FIX 0   /* int64 n^3: CIC electron density in units of     */
                          /* 2^-3s electrons per cell (as of the last a4)   */
#define ITOKMC_XE 1       /* int64 n^3: electrons per cell (NGP), last a4   */
#define ITOKMC_NPOS 2     /* int64 n^3: positive-ion count per cell         */
#define ITOKMC_NNEG 3     /* int64 n^3: negative-ion count per cell         */
#define ITOKMC_PHI 4      /* double n^3: potential, V (mixed form: its int64 */
                          /* fixed-point potential, converted)              */
#define ITOKMC_E 5        /* double 3 n^3: Ex block, Ey block, Ez block V/m */
                          /* (mixed form: the FP32 values the push uses)    */
#define ITOKMC_RHO 6      /* int64 n^3: space charge 2^3s (N+ - N-) - ne_fix*/
                          /* in units of q_e 2^-3s, as of the last a4       */
#define ITOKMC_FIRINGS 7  /* int64 5 n^3: ionizations, attachments, photon  */
                          /* emissions, e-ion and ion-ion recombinations of */
                          /* the last a6 (blocks of n^3)                    */

/* ---- stages runnable one at a time (itokmc_run_stage) ------------------ */
#define ITOKMC_STAGE_TRANSPORT 0  /* a1-a4: push, sort, deposit, X_e, rho   */
#define ITOKMC_STAGE_KMC 1        /* a6 with the current E                  */
#define ITOKMC_STAGE_PARTICLES 2  /* a7-a9: products, photons, merge/split  */
#define ITOKMC_STAGE_FIELD 3      /* a5 from the rho of the last a4          */

/* ---- initial seeds ------------------------------------------------------
 * A Gaussian seed of electrons (the initial conditions of Sec. 5.1): density
 * peak exp(-|x - center|^2 / (2 sigma^2)) per m^3.  realization: the
 * realization it seeds, or -1 for every realization. */
typedef struct itokmc_seed_blob {
    double center[3];          /* m                                          */
    double sigma;              /* m, > 0                                     */
    double peak;               /* electrons per m^3 at the centre, >= 0      */
    int32_t realization;       /* -1: all realizations                       */
    int32_t pad;
} itokmc_seed_blob;
#define ITOKMC_SEED_NEUTRAL 1  /* seed electron-ion pairs: N+ += N_c per cell */

typedef void* (*itokmc_alloc_fn)(size_t bytes, void* ctx);   /* device memory */
typedef void (*itokmc_free_fn)(void* ptr, void* ctx);

typedef struct itokmc_config {
    int32_t n[3];              /* cells per axis: equal powers of two >= 8   */
    int32_t n_realizations;    /* ensemble size R >= 1                       */
    double lo[3], hi[3];       /* domain corners (m); cells must be cubes    */
    double dt;                 /* time step (s)                              */
    uint64_t seed0;            /* realization r uses Philox key seed0 + r    */
    double mu, D;              /* electron mobility (m^2/Vs), diffusion m^2/s*/
    double alpha_A, alpha_B;   /* ionization alpha(E) = A exp(-B/|E|) (1/m)  */
    double eta;                /* attachment coefficient (1/m)               */
    double E0;                 /* applied field (V/m): phi(hi_z)=E0 L_z      */
    double photon_ratio;       /* k_gamma = photon_ratio k_alpha; 0 = off    */
    double kappa_lo, kappa_hi; /* absorption coefficient range (1/m)         */
    double eps;                /* Cao accuracy factor; INFINITY as in paper  */
    int32_t ppc;               /* particles per cell after merge (2^k <= 256)*/
    int32_t n_new;             /* max new particles per cell (64, <= 64)     */
    int32_t n_crit;            /* critical threshold N_c (5)                 */
    int32_t n_ssa;             /* max SSA events per substep N_SSA (10)      */
    int32_t frac_bits;         /* fixed-point bits s per axis (10, <= 10)    */
    int32_t precision;         /* ITOKMC_FP64 or ITOKMC_MIXED                */
    double mg_rtol;            /* stop when ||r||_2 <= mg_rtol ||b||_2       */
    int32_t mg_nu1, mg_nu2;    /* red-black Gauss-Seidel pre/post sweeps     */
    int32_t mg_max_cycles;     /* V-cycle limit (ITOKMC_ERR_NOCONV beyond)   */
    int32_t field_precision;   /* -1: as precision; else ITOKMC_FP64/MIXED   */
    int64_t particle_capacity; /* particles storable (all realizations)      */
    void* stream;              /* cudaStream_t to run on, or NULL (default)  */
    itokmc_alloc_fn alloc;     /* device allocator, or NULL: cudaMallocAsync */
    itokmc_free_fn free_fn;    /* matching free                              */
    void* alloc_ctx;           /* passed to alloc/free_fn                    */
    const itokmc_seed_blob* blobs; /* initial seeds sampled by itokmc_init   */
    int32_t n_blobs;           /* 0: no seeding (particles set by the caller)*/
    int32_t seed_flags;        /* 0 or ITOKMC_SEED_NEUTRAL                   */
    int32_t coupling;          /* ITOKMC_EXPLICIT or ITOKMC_SEMI_IMPLICIT     */
    int32_t dt_adapt;          /* 0: every step dt; 1: adaptive, dt the largest */
    double dt_min;             /* smallest adaptive step (s)                  */
    double cfl;                /* drift / diffusion bound (cells per step)    */
    double drt_factor;         /* dt <= drt eps0/sigma_max (explicit; 0: off) */
    double ion_factor;         /* k_ion(|E|max) dt <= ion_factor (0: off)     */
    double beta_ep, beta_np;   /* recombination coefficients (m^3/s), Sec. 5.1:
                                  k_ep = beta_ep / dV, k_np = beta_np / dV;
                                  0 (the defaults): the reaction is off       */
    int32_t mobile_ions;       /* 0: ions as per-cell counts; 1: positive and
                                  negative ions as Ito particles (explicit
                                  coupling only)                             */
    int32_t pad_ions;
    double mu_ion, D_ion;      /* ion mobility (m^2/Vs), diffusion (m^2/s)   */
    int32_t graph_step;        /* 1: replay steps from captured CUDA graphs  */
    int32_t pad_graph;         /* (explicit coupling, fixed dt; see below)   */
} itokmc_config;

typedef struct itokmc_stats {
    int64_t n_particles;       /* particles now (all realizations)           */
    int64_t step;              /* steps taken                                */
    int64_t n_movers;          /* particles that changed cell in the last a2 */
    int64_t outflow_weight;    /* electrons absorbed at faces, last step     */
    int64_t ionizations, attachments, photon_emissions; /* last a6          */
    int64_t photons_absorbed_weight, photons_lost_weight; /* last a8        */
    int64_t n_new_particles;   /* products + photoelectrons, last a7/a8      */
    int32_t mg_cycles;         /* V-cycles of the last field solve           */
    int32_t kmc_status;        /* 0, or ITOKMC_ERR_KMC                       */
    double mg_rel_residual;    /* ||r||/||b|| after the last field solve      */
    double ms_transport, ms_kmc, ms_particles, ms_field; /* last step (events)*/
    int64_t kernel_launches;   /* kernels launched by the library so far     */
    int64_t merge_cells, merge_elements, merge_elements_sq, merge_max_list; /* last a9 */
    double dt_last;            /* step size of the last step (s)             */
    int64_t recombinations_ep, recombinations_np; /* last a6                */
    int64_t outflow_ion_pos, outflow_ion_neg;     /* ion weight absorbed at the
                                                     faces, last step (mobile) */
    int64_t graph_steps;       /* steps replayed from captured graphs so far */
} itokmc_stats;

typedef struct itokmc_handle itokmc_handle;

/* Fills *cfg with the defaults of the paper's method (N_new 64, N_c 5,
 * N_SSA 10, eps = INFINITY, s = 10, rtol 1e-10, nu1 = nu2 = 2, 64 cycles,
 * FP64).  Grid, physics and capacity must still be set by the caller. */
int itokmc_config_defaults(itokmc_config* cfg);

/* Validates *cfg, allocates all device state for n_realizations x n^3 cells
 * and particle_capacity particles, zeroes it, and returns the handle in
 * *out.  No particles exist yet.  The configuration is the problem of Sec. 4
 * (Eq. ito_poisson): the electron drift-diffusion coefficients (mu, D) of
 * Eq. ito_kernel with v = -mu E (Eq. Vk1), the reaction network of Sec.
 * 3.2 and Table air_reactions over the counts (X_e, X_+, X_-): ionization,
 * attachment and photon emission (alpha(E), eta, k_gamma) and, with
 * beta_ep / beta_np > 0, electron-ion and ion-ion recombination
 * (propensities k_ep X_e X_+ and k_np X_+ X_-, k = beta / dV, Sec. 5.1;
 * cells with ions of both signs but no electrons then run the KMC too; the
 * field dependence of beta_ep through T_e is the caller's: it is one
 * constant here), the photon absorption range of
 * Sec. 5.1, the Cao et al. parameters N_c, N_SSA, eps of Sec. 3.2.3, the
 * particle budget of Sec. 4.4 (N_new) and Sec. 4.6 (ppc), and the electrode
 * and side boundary conditions of Sec. 5.1.  With n_blobs > 0 the initial
 * electrons are then sampled on the device from cfg->blobs
 * (itokmc_seed_blobs, with cfg->seed_flags), deposited, and the initial
 * field is solved (itokmc_solve_field); cfg->blobs is read during the call
 * only.  Errors: ERR_ARG (bad config or blobs), ERR_OOM, and those of
 * itokmc_seed_blobs and itokmc_solve_field. */
int itokmc_init(const itokmc_config* cfg, itokmc_handle** out);

/* Releases all device memory of the handle.  Always safe on a poisoned
 * handle; NULL is a no-op. */
int itokmc_destroy(itokmc_handle* h);

/* Replaces all particles.  x, y, z (double), w (uint32 weights = physical
 * electrons, >= 1) and realization (int32, may be NULL when R = 1) hold n
 * particles in any order, in host (mem = ITOKMC_HOST) or device memory.
 * These are the computational particles of Sec. 3.1 (position X_p, integer
 * weight w_p: the number of physical electrons a superparticle stands for,
 * Sec. 4.4).  Particles are stably sorted by (realization, cell), the
 * binning of Sec. 5.6; particles outside [lo, hi) are rejected with ERR_ARG.
 * ERR_CAPACITY if n > capacity. */
int itokmc_set_particles(itokmc_handle* h, const double* x, const double* y, const double* z,
                         const uint32_t* w, const int32_t* realization, int64_t n, int32_t mem);

/* As itokmc_set_particles, with the species of each particle (int32, NULL:
 * all electrons): 0 electrons, 1 positive ions, 2 negative ions (the ions as
 * Ito particles, Sec. 4.3 Eq. particle_kernel with sgn(Z_s); species 1 and 2
 * need mobile_ions = 1, else ERR_ARG).  Each species of each realization
 * is a particle block b = species R + realization with its own cells;
 * particles are sorted by (block, cell). */
int itokmc_set_particles_species(itokmc_handle* h, const double* x, const double* y, const double* z,
                                 const uint32_t* w, const int32_t* realization, const int32_t* species,
                                 int64_t n, int32_t mem);

/* Copies the particles (canonical order: by realization, cell, then the
 * order of the last sort/merge) into caller buffers of capacity cap.  Any
 * pointer may be NULL.  cell receives the linear cell index within the
 * realization; realization receives the particle block (with mobile ions,
 * species R + realization: blocks of electrons, positive, negative ions).  *n_out receives the particle count; ERR_CAPACITY if it
 * exceeds cap (nothing copied).  Synchronises the stream. */
int itokmc_read_particles(itokmc_handle* h, double* x, double* y, double* z, uint32_t* w,
                          int32_t* realization, int64_t* cell, int64_t cap, int64_t* n_out,
                          int32_t mem);

/* Replaces all particles by initial electrons sampled on the device from
 * Gaussian seeds (Sec. 5.1).  Per cell c of realization r: the density at
 * the cell centre n(x_c) = sum of the blobs that seed r; N_c ~ Poisson(n(x_c)
 * dV), drawn from the Philox stream (key seed0 + r, index c, the step
 * counter, tag INIT, sub 0) with the tau-leap's sampler (inversion below mean
 * 10, PTRS above); m = min(N_c, ppc) superparticles with the weight rule of
 * Eq. w (N_c div m, the remainder on the first); slot j uniform in the cell
 * from the stream (c, step, INIT, 1 + j): x = lo + (i + u) h from FP64
 * uniforms (the mixed form keeps the FP32 offsets from the high words of
 * the same uniforms).  Particles come out in canonical order (cell, slot).
 * flags: ITOKMC_SEED_NEUTRAL also adds N_c to the cell's positive ions.  The
 * field is not solved (call itokmc_solve_field).  Errors: ERR_ARG (NULL
 * blobs with n_blobs > 0, sigma <= 0, peak < 0, realization < -1, unknown
 * flags), ERR_CAPACITY, ERR_OVERFLOW (a weight above 2^32 - 1), ERR_CUDA. */
int itokmc_seed_blobs(itokmc_handle* h, const itokmc_seed_blob* blobs, int32_t n_blobs, int32_t flags);

/* Sets the ion counts (int64, R n^3 each; host or device).  ERR_ARG with
 * mobile ions (the ions are particles then; the counts read back by
 * itokmc_read_densities are their NGP counts). */
int itokmc_set_ions(itokmc_handle* h, const int64_t* npos, const int64_t* nneg, int32_t mem);

/* Sets E directly (double, three blocks Ex, Ey, Ez of R n^3 each), bypassing
 * the field solve: used to feed a given field to the next step or stage. */
int itokmc_set_field(itokmc_handle* h, const double* E, int32_t mem);

/* Re-deposits the current particles (a4) and solves the field (a5) from
 * them and the current ions: the initial field of a run.  ERR_NOCONV if the
 * multigrid stops at mg_max_cycles above tolerance. */
int itokmc_solve_field(itokmc_handle* h);

/* Graph-replayed steps (graph_step = 1): with the explicit coupling and a
 * fixed step size, once a host-driven step has measured the field solve's
 * cycle count and the buffers' use, every further step with headroom in
 * those buffers is one launch of a captured CUDA graph (cached per state of
 * the swapped device buffers): the particle count and the step counter are
 * read on the device, the field runs that many cycles beside the KMC and
 * particle stages, and after the step the host checks the error word, the
 * residual and the fixed-point scale (a field short of the tolerance is
 * solved further on the host; its next replays run more cycles).  Results
 * equal the host-driven step's for the same field; the stage timings of
 * replayed steps read 0. */

/* Adaptive step size (dt_adapt = 1).  The paper runs fixed steps and names
 * CFL- or physics-based dynamic time stepping as the way to use its
 * adjustable-accuracy chemistry (Sec. 4.7).  Before each step the step size
 * becomes dt 2^-j, j the smallest >= 0 for which it satisfies every active
 * bound, from the field that pushes the particles (its largest |E|) and the
 * densest cell of the last deposit: mu |E|max dt <= cfl h and 2 D dt <=
 * (cfl h)^2 (cfl > 0); dt <= drt_factor eps0 / (q_e mu n_max) with the
 * explicit coupling (drt_factor > 0; the dielectric relaxation time);
 * alpha(|E|max) mu |E|max dt <= ion_factor (ion_factor > 0).  It never goes
 * below the largest such step not under dt_min.  Power-of-two steps make the
 * choice depend only on which side of each bound the candidate falls.  The
 * Philox counters keep using the step index; itokmc_get_stats reports the
 * size of the last step.
 *
 * Advances nsteps full steps.  With coupling = ITOKMC_EXPLICIT (a1-a9 then
 * a5): particle transport by Eq. ito_kernel with the Euler-Maruyama update
 * of Sec. 4.3 (first equation) in the field of the start of the step,
 * deposition (Sec. 4.2), per-cell KMC (Sec. 3.2.3), products (Sec. 4.4),
 * photoionization (Sec. 4.5), merge/split (Sec. 4.6) and the Poisson solve
 * (Sec. 4.3) for the next step's field, overlapped with a6-a9.  With
 * ITOKMC_SEMI_IMPLICIT the time step of Sec. 4.7: the semi-implicit
 * transport stage of itokmc_transport_semi_implicit (conductivity, diffusive
 * substep, variable-coefficient solve for the field of the end of the step,
 * advective substep, sort, deposit) and then a6-a9 with that field; no
 * solve follows the step.  Errors: ERR_CAPACITY, ERR_OVERFLOW, ERR_NOCONV,
 * ERR_KMC, ERR_CUDA. */
int itokmc_step(itokmc_handle* h, int32_t nsteps);

/* Runs one stage (ITOKMC_STAGE_*) on the current state without advancing
 * the step counter; a full step is TRANSPORT, KMC, PARTICLES, FIELD and then
 * the counter advance (itokmc_advance_counter).  Order: TRANSPORT (or
 * itokmc_transport_semi_implicit) and FIELD may run at any time; KMC needs a
 * transport of the current particles and may be repeated on it (each run
 * applies its firings to the ion counts again); PARTICLES needs a KMC after
 * the last transport and changes the particles, so the next KMC needs a new
 * transport.  Setting, seeding or loading particles restarts the order.
 * Errors: ERR_ARG (unknown stage or out of order), and those of the stage. */
int itokmc_run_stage(itokmc_handle* h, int32_t stage);

/* Advances the step counter used in every Philox counter by one. */
int itokmc_advance_counter(itokmc_handle* h);

/* Semi-implicit transport stage (Sec. 4.3, Eq. particle_kernel, Eq. Xdagger,
 * Eq. poisson_simp, Eq. conductivity; Sec. 4.7 steps 1-5), the alternative
 * to ITOKMC_STAGE_TRANSPORT that removes the dielectric-relaxation limit of
 * the explicit push: conductivity sigma = q_e mu n_e from a CIC deposit of
 * the current particles; diffusive advance X+ = X + sqrt(2 D dt) N (the
 * push's normals); charge rho+ of the diffused particles; FP64 multigrid on
 * div[(1 + sigma dt / eps0) grad phi] = -rho+/eps0 (face coefficient: the
 * mean of the two cells'; boundary faces: the cell's own) to mg_rtol, E =
 * -grad(phi) into the handle's field; advective step X' = X+ - mu E(X) dt
 * with E at the start-of-step position X; then the stable sort, the deposit
 * and the charge of X' as in ITOKMC_STAGE_TRANSPORT.  FP64 form only
 * (ERR_ARG for the mixed form).  cycles_out / rel_out (may be NULL): the
 * V-cycles taken and the final relative residual.  Errors: ERR_ARG,
 * ERR_NOCONV, ERR_OVERFLOW, ERR_CAPACITY, ERR_CUDA. */
int itokmc_transport_semi_implicit(itokmc_handle* h, int32_t* cycles_out, double* rel_out);

/* ---- 0-D KMC ensembles ------------------------------------------------------
 * The paper compares KMC with the reaction rate equation on a single
 * well-mixed cell (Sec. 3.2.4, Fig. AvalancheAttachment): thousands of
 * independent realizations of the electron count under ionization,
 * attachment and photon emission at a fixed field.  itokmc_kmc0d advances
 * n_real such realizations on the device, one thread each, with the per-cell
 * KMC of the spatial step (Sec. 3.2.3, Cao et al. hybrid; cfg's n_crit,
 * n_ssa, eps, dt) and the rates of the field magnitude E_mag (V/m): k_ion =
 * alpha(E) mu E, k_att = eta mu E, k_ph = photon_ratio k_ion, in FP64
 * (cfg->precision = ITOKMC_FP64) or FP32 (ITOKMC_MIXED).  Realization m,
 * step k draws from the Philox stream (key seed0, index m, step k, tag KMC).
 *   X  int64 n_real x (n_steps + 1), row m = realization m: the electrons
 *      after k = 0 .. n_steps steps (X[m][0] = X0); host (mem =
 *      ITOKMC_HOST) or device (ITOKMC_DEVICE) memory of the caller.
 * Grid, particle and allocator fields of cfg are ignored; cfg->stream is
 * used.  Allocates a small counter block (and, for host output, a device
 * copy of X) for the call.  Returns ITOKMC_OK, ITOKMC_ERR_ARG, ITOKMC_ERR_OOM,
 * ITOKMC_ERR_KMC (a realization hit the iteration guard) or ITOKMC_ERR_CUDA;
 * the message is in itokmc_last_error(NULL).  Synchronises the stream. */
int itokmc_kmc0d(const itokmc_config* cfg, double E_mag, int64_t X0, int32_t n_real, int32_t n_steps, int64_t* X,
                 int32_t mem);

/* ---- checkpoints ----------------------------------------------------------
 * The paper's runs write checkpoint files from which a run restarts (Sec.
 * 5.6).  itokmc_save writes, at a step boundary, everything the next step
 * reads: the configuration it belongs to, the step counter and the smoother
 * counts in use, the particles in canonical order with the per-cell offsets,
 * the ion counts N+ and N-, the field E of the next step, the potential and
 * the previous potential (the next solve starts from their extrapolation),
 * the fixed-point exponent of the mixed potential, and the densities of the
 * last deposit (NE_FIX, XE, RHO, FIRINGS).  Every random draw is a Philox
 * counter of (seed, index, step, tag), so a handle that loads the file
 * continues bit for bit as the run that wrote it would have.
 *   itokmc_save  path: file to create or overwrite (host I/O, about
 *                R n^3 (128 + 8 FP64 | 56 mixed) bytes plus 32 (FP64) or
 *                20 (mixed) bytes per particle).  Synchronises the stream.
 *   itokmc_load  into a handle created with the same configuration (grid,
 *                realizations, form, physics, seed0, mg_rtol; the stream,
 *                allocator and a capacity of at least the saved particle
 *                count may differ).  Replaces the handle's state and sets its
 *                step counter and smoother counts from the file.
 * Errors: ERR_ARG (NULL path, unreadable or foreign file, another
 * configuration: the message names the first differing field),
 * ERR_CAPACITY (load: too many particles), ERR_CUDA. */
int itokmc_save(itokmc_handle* h, const char* path);
int itokmc_load(itokmc_handle* h, const char* path);

/* ---- autotuning ----------------------------------------------------------
 * The paper fixes no smoother counts; the multigrid cycle (Sec. 4.3:
 * V-cycles with red-black Gauss-Seidel smoothing) takes nu1 pre- and nu2
 * post-smoothing sweeps per level.  itokmc_autotune times the field solve
 * of the current charge (as left by itokmc_solve_field or the last step)
 * for each candidate pair (nu1, nu2) in {1,2,3} x {1,2,3}, each from a zero
 * potential (a solve of many cycles, which ranks the pairs by convergence
 * per unit time), twice, and keeps the fastest pair that converges in the
 * handle's configuration (mg_nu1, mg_nu2).  The potential and field
 * are restored afterwards, so the run continues as without the call; only
 * the number of V-cycles of later solves changes (the tolerance does not).
 * Then, with particles present, it times the push kernel of the current
 * particles (the transport's first kernel; its trial writes only what the
 * next transport writes again) for each deposit window in {0, 256, 512,
 * 1024, 2048} cells (three launches each, the fastest kept) and keeps the
 * fastest window.
 *   out  optional: the chosen pair, its time, and every candidate's time
 *        (ms, -1 if it did not converge).
 * Returns ITOKMC_OK, ITOKMC_ERR_NOCONV if no candidate converges, or
 * ITOKMC_ERR_CUDA.  Synchronises the stream. */
#define ITOKMC_TUNE_CANDIDATES 9
#define ITOKMC_TUNE_DEPOSIT 5
typedef struct itokmc_tuning {
    int32_t mg_nu1, mg_nu2;                          /* chosen pair            */
    double ms_field;                                 /* its field-solve time   */
    int32_t cycles;                                  /* its V-cycle count      */
    int32_t n_tried;
    int32_t nu_tried[ITOKMC_TUNE_CANDIDATES][2];
    double ms_tried[ITOKMC_TUNE_CANDIDATES];         /* -1: no convergence     */
    /* the push's deposit tile: the largest cell box a block of the push
     * deposits through its shared window (0: global atomics only); the
     * deposit is an integer sum, so the choice changes no result */
    int32_t dep_win;                                 /* chosen window (cells)  */
    int32_t n_dep_tried;
    int32_t dep_tried[ITOKMC_TUNE_DEPOSIT];          /* 0, 256, 512, 1024, 2048 */
    double ms_dep_tried[ITOKMC_TUNE_DEPOSIT];        /* push ms, -1: not timed  */
} itokmc_tuning;
int itokmc_autotune(itokmc_handle* h, itokmc_tuning* out);

/* Copies one field (ITOKMC_NE_FIX ...) of realization r (or all
 * realizations when r = -1) into host_out of the given size in bytes.
 * The densities are the mesh quantities of Sec. 4.2: the CIC deposit of the
 * particle weights (W_cic, in fixed point), the per-cell electron and ion
 * counts X_e, N+, N- of the KMC state (Sec. 3.2, Eq. kmc), the space charge
 * rho of Eq. poisson, and phi and E = -grad phi (Sec. 4.3).  ERR_ARG if
 * bytes is too small.  Synchronises the stream. */
int itokmc_read_densities(itokmc_handle* h, int32_t realization, int32_t which, void* host_out,
                          size_t bytes);

/* Fills *st with counters of the last step.  Synchronises the stream. */
int itokmc_get_stats(itokmc_handle* h, itokmc_stats* st);

/* Current particle count (all realizations).  Synchronises the stream. */
int itokmc_num_particles(itokmc_handle* h, int64_t* n_out);

/* Message of the last error on this handle ("" if none).  h may be NULL
 * for errors of itokmc_init. */
const char* itokmc_last_error(const itokmc_handle* h);

/* Library version string. */
const char* itokmc_version(void);

/* ---- measurement --------------------------------------------------------
 * The FP64 form is bound by the device's FP64 units (the interpolation,
 * push and quotient arithmetic of Sec. 4.2-4.3 in double precision), so its
 * roofline is taken against the FP64 arithmetic rate.  This call measures
 * that rate: 8 blocks of 256 threads per SM, each thread 8 independent
 * chains of 4096 fused multiply-adds in registers (2 FLOP each), best of
 * three timed launches on `stream` (a cudaStream_t, or NULL).  Allocates
 * 64 KB of device memory for the duration of the call.
 *   tflops_out  measured FP64 TFLOP/s;  ms_out (may be NULL) the best time.
 * Returns ITOKMC_OK, ITOKMC_ERR_ARG, ITOKMC_ERR_OOM or ITOKMC_ERR_CUDA (the
 * message in itokmc_last_error(NULL)).  Synchronises the stream. */
int itokmc_probe_fp64_peak(void* stream, double* tflops_out, double* ms_out);

/* ---- field solve without device allocation ------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- for instance a program whose device memory is
 * owned by another runtime's pool with a fixed budget, code that must avoid
 * the implicit device synchronisation of cudaMalloc/cudaFree, or a plugin
 * whose host forbids new device allocations.  It runs the same multigrid
 * field solve as itokmc_solve_field (a5) on caller memory and allocates
 * nothing: its scratch is a file-scope device array of 16 MiB inside the
 * library, which every GPU that loads the library keeps until the process
 * exits, so grids are limited to ITOKMC_NOALLOC_MAX_N cells per axis.
 *
 *   cfg     grid (n, lo, hi; one realization), E0, frac_bits, mg_rtol,
 *           mg_nu1/nu2, mg_max_cycles, precision/field_precision and
 *           stream; particle and allocator fields are ignored.  The field
 *           form is field_precision, or precision when that is -1:
 *           ITOKMC_FP64 runs FP64 V-cycles; ITOKMC_MIXED runs FP32 V-cycles
 *           inside FP64 residual refinement (an FP64 potential, not the
 *           fixed-point potential a handle of the mixed form keeps).  Any
 *           other value is ITOKMC_ERR_ARG before anything is launched.
 *           The V-cycles are launched directly on the stream (no graph is
 *           captured or instantiated).
 *   rho     device, int64 n^3: space charge in units of q_e 2^-3s per cell
 *           (the ITOKMC_RHO layout).
 *   phi     device, double n^3: initial guess on entry, potential on exit.
 *   E       device, double 3 n^3: Ex, Ey, Ez blocks on exit.
 *   cycles_out, rel_out  optional: V-cycles used, final ||r||/||b||.
 * Returns ITOKMC_OK, ITOKMC_ERR_ARG (NULL pointer, R != 1, n not a power of
 * two, n > ITOKMC_NOALLOC_MAX_N, or an unknown precision), ITOKMC_ERR_NOCONV
 * or ITOKMC_ERR_CUDA;
 * the message is in itokmc_last_error(NULL).  The first call on a device
 * looks up the scratch array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the one
 * scratch array and it keeps the last call's contents (the solve clears
 * what it needs), so calls that overlap on the GPU -- on two streams, or
 * from two threads -- race and must be serialised by the caller.  The call
 * synchronises cfg->stream before it returns. */
#define ITOKMC_NOALLOC_MAX_N 64
int itokmc_field_solve_noalloc(const itokmc_config* cfg, const int64_t* rho, double* phi, double* E,
                               int32_t* cycles_out, double* rel_out);

#ifdef __cplusplus
}
#endif
#endif /* ITOKMC_H */
