/*
 * grmhd.h -- C ABI of the GB300 GRMHD substep library (libgrmhd.so).
 *
 * One Runge-Kutta substep of the GRMHD method of "MHDuet: a high-order GRRMHD
 * code for CPU and GPU architectures" (arXiv 2510.13965) on ghosted,
 * vertex-centred grid patches:
 *   - CCZ4 spacetime right-hand side with 1+log slicing and the simplified
 *     Gamma-freezing shift (Sec. II A, evolution equations and gauge),
 *     4th-order centred / one-sided finite differences and Kreiss-Oliger
 *     dissipation (Sec. III B);
 *   - ideal-MHD balance laws with divergence cleaning (Sec. II B, MHD system),
 *     Lax-Friedrichs flux splitting, MP5 reconstruction and the flux formula
 *     Fhat = F^L + F^R (Sec. III C), fast-magnetosonic speed bound (appendix on
 *     characteristic speeds);
 *   - per-point conservative-to-primitive recovery, Kastaun's two Brent
 *     root finds with the EOS validity clamps and the error policy (appendix on
 *     the conversion from conserved to primitive fields);
 *   - the explicit RK4 stage combination (Sec. III A, Table RK4 explicit part).
 *
 * Conventions
 *   - All floating-point data are FP64.  Every compute step runs in the
 *     library's CUDA kernels (sm_103a); there is no CPU path.
 *   - Pointers marked "device" are CUDA device pointers owned by the caller;
 *     the library never frees them.  The library owns its context, the patch
 *     descriptors copied to the device, its scratch arrays and CUDA graphs.
 *   - Work is enqueued on the stream given at creation (a cudaStream_t passed
 *     as void*; NULL means the legacy default stream).  Calls return after
 *     enqueueing, except where a call says it synchronises.
 *   - Every function returns a grmhd_status: 0 on success, a negative code on
 *     failure.  Argument errors are detected on the host before any launch.
 *     Device-side failures (a fatal con2prim point, a non-finite state) are
 *     recorded in a device flag and reported by grmhd_sync_status.  No
 *     function aborts, traps or exits.
 *
 * Patch layout
 *   A patch has n[0] x n[1] x n[2] interior points and 3 ghost layers per side
 *   (the width of the KO / one-sided stencils and of the 6-point MP5 interface
 *   stencil).  Point (i, j, k), with i in [-3, n[0]+3) etc., sits at
 *   x0 + (i, j, k) * dx.  Arrays are field-major, x fastest:
 *       a[f][k + 3][j + 3][i + 3],  extents (n[2]+6, n[1]+6, px), px >= n[0]+6.
 *   Evolved fields (32): 0-5 gt_ij (xx xy xz yy yz zz), 6-11 At_ij, 12 chi,
 *   13 Khat, 14 Theta, 15-17 Gammahat^i, 18 alpha, 19-21 beta^i, 22 Dbar,
 *   23 DYebar, 24 taubar, 25-27 Sbar_i, 28-30 Bbar^i, 31 phibar
 *   (bar = densitized by sqrt(gamma)).
 *   Primitives (10): rho, eps, p, v^x, v^y, v^z (contravariant), W, Ye, T, c_s^2.
 *   Initial data (26): gamma_ij (6), K_ij (6), alpha, beta^i (3), rho, eps,
 *   v^i (3), B^i (3, not densitized), Ye, T.
 */
#ifndef GRMHD_H
#define GRMHD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GRMHD_NFIELDS 32
#define GRMHD_NPRIM 10
#define GRMHD_NID 26
#define GRMHD_NGHOST 3

typedef enum {
  GRMHD_OK = 0,
  GRMHD_ERR_ARG = -1,        /* invalid argument (checked on the host)          */
  GRMHD_ERR_CUDA = -2,       /* a CUDA runtime call failed                       */
  GRMHD_ERR_C2P_FATAL = -3,  /* a point hit a fatal con2prim policy branch        */
  GRMHD_ERR_TIMEOUT = -4,    /* a bounded device wait ran out                     */
  GRMHD_ERR_NONFINITE = -5,  /* a non-finite conserved state reached con2prim     */
  GRMHD_ERR_NOMEM = -6,      /* a library allocation failed                      */
  GRMHD_ERR_SIZE = -7        /* a patch exceeds a fixed maximum size             */
} grmhd_status;

/* Per-point con2prim status codes written to grmhd_patch_desc.status:
 *    0 ok; positive = corrections applied (bit mask): 1 atmosphere,
 *    2 eps clamped to the EOS range, 4 velocity limited to W_max, 8 Ye reset;
 *   -1 rho > rho_max, -2 eps > eps_max in a dense region, -3 W > W_max in a
 *   dense region, -4 Ye out of range in a dense region (the paper's fatal
 *   cases), -5 no bracketed root / non-finite input. */

/* Physical and numerical parameters.  Constants the paper leaves open
 * (kappa_2, damping and gauge constants, c_b, kappa_b, the error-policy
 * thresholds, the Brent stop rule) are inputs. */
typedef struct grmhd_params {
  double kappa_z, kappa_c, kappa_2; /* CCZ4 constraint damping                         */
  double eta;                       /* shift damping (beta_0 = 0, f_alpha = f_beta = 1) */
  double sigma_ko;                  /* Kreiss-Oliger strength sigma                     */
  double c_b, kappa_b;              /* divergence-cleaning speed and damping            */
  double gamma_th;                  /* ideal-gas adiabatic index                        */
  double K_atmo;                    /* polytropic K of the ideal-gas atmosphere         */
  double rho_atmo, rho_min, rho_low, rho_max;
  double alpha_bh, W_max;
  double eps_max;                   /* ideal-gas eps upper bound                        */
  double ye_min, ye_max, ye_atmo;
  double T_atmo;                    /* tabulated EOS: atmosphere temperature [MeV]      */
  double h0;                        /* lower bound of the specific enthalpy of the EOS  */
  double c2p_xtol;                  /* absolute part of the Brent stop rule             */
  int eos_kind;                     /* 0 ideal gas, 1 table, 2 hybrid (below)           */
  int bc;                           /* ghosts: 0 periodic, 1 linear extrapolation,
                                       2 frozen (the initial data's ghost values),
                                       3 mesh-refinement hierarchy (see below)          */
  int max_iter;                     /* Brent iteration cap per root find                */
  int rk;                           /* time integrator (Sec. III A): 0 RK4 (Table RK4),
                                       1 SSP-RK3 (Table RK3SSP), explicit parts          */
  /* Hybrid EOS (eos_kind 2; Sec. II B, piecewise-polytropic cold part plus a
   * thermal ideal gas):
   *   p = p_cold(rho) + (gamma_th - 1) rho (eps - eps_cold(rho)),
   *   p_cold = K_i rho^Gamma_i,  eps_cold = a_i + K_i rho^(Gamma_i - 1) / (Gamma_i - 1)
   * on piece i (rho_poly[i-1] < rho <= rho_poly[i]), K_0 = K_poly, a_0 = 0,
   * K_i and a_i fixed by continuity of p_cold and eps_cold at rho_poly.
   * eps is clamped to [eps_cold(rho), eps_max]; T is reported as 0; initial
   * data give eps (as for the ideal gas).  Requires 1 <= npoly <= 4,
   * gamma_poly[i] > 1, K_poly > 0, rho_poly[0..npoly-2] > 0 increasing;
   * unused entries are ignored. */
  int npoly;
  int reserved2;
  double K_poly;
  double rho_poly[3];
  double gamma_poly[4];
  /* LES gradient sub-grid-scale model (Sec. II B; Appendix "Large Eddy
   * Simulation techniques"): coefficients C_N, C_Y, C_T, C_M of the SGS terms
   * of D, DYe, S_i and B^i (the paper's default: C_M = 8, the others 0); all
   * zero: no LES terms.  With any nonzero, every pointwise MHD flux along d
   * gains alpha C xi sqrt(gamma) H^d (xi = gamma^{1/3} dx^2 / 24) before the
   * reconstruction.  The pressure derivatives are analytic for the ideal gas
   * and the hybrid EOS, and for eos_kind 1 those of the table's interpolant
   * (linear in eps between temperature nodes, bilinear in log10 rho and Ye).  grmhd_rhs_eval_static returns
   * GRMHD_ERR_ARG for any LES coefficient (its point values need scratch
   * memory); a patch context allocates LES_NAUX = 32 doubles per ghosted
   * point for them. */
  double les_c[4];
  /* A flux point whose rest-mass density is below les_rho_min gets no SGS
   * flux (0: everywhere).  The paper states no rule for low densities; in an
   * atmosphere the gradient model acts on an almost massless, magnetised
   * fluid and C_M = 8 drove a static star's atmosphere unstable within nine
   * steps, so rho_low (the error policy's low-density threshold) is the
   * natural setting. */
  double les_rho_min;
} grmhd_params;

/* Tabulated EOS: p, eps, c_s^2 on the nodes of a uniform (log10 rho,
 * log10 T[MeV], Ye) grid, rho fastest: node (ir, it, iy) is at
 * (iy * nt + it) * nr + ir.  Arrays are device pointers owned by the caller
 * and must stay valid while a context uses them. */
typedef struct grmhd_eos_table {
  int nr, nt, ny, reserved;
  double lr0, dlr, lt0, dlt, ye0, dye;
  const double* p;
  const double* eps;
  const double* cs2;
} grmhd_eos_table;

/* One patch.  U[0] holds U^n; U[1], U[2] hold RK stage values; U[3] holds the
 * RK4 accumulator.  All arrays are device pointers with the layout above.
 *
 * Mesh-refinement hierarchy (bc = 3; Sec. IV B, prolongation and
 * restriction, for a fixed hierarchy advanced without sub-cycling):
 *   - exactly one patch has level 0; its outer ghosts are extrapolated as for
 *     bc = 1;
 *   - a level-l patch has dx = dx_0 / 2^l and x0 on the level-l grid that
 *     starts at the level-0 x0 (x0 = x0_0 + o dx, o integer); patches of one
 *     level do not overlap; level-l point g coincides with level-(l-1) point
 *     g/2 when g is even and is the midpoint of (g-1)/2 and (g+1)/2 when odd;
 *   - a ghost point of a level-l patch (l >= 1) is copied from the interior of
 *     another level-l patch that holds it, else prolongated from the level-
 *     (l-1) patch whose interior holds floor(g/2): the paper's six-point
 *     Lagrange midpoint formula along every axis where g is odd (x, then y,
 *     then z), the coarse value along the others.  Levels are filled in order;
 *   - grmhd_init_patches returns GRMHD_ERR_ARG (with a message on stderr) when
 *     the layout breaks these rules or a fine ghost point is not covered. */
typedef struct grmhd_patch_desc {
  int n[3];
  int px;
  int level;
  int reserved;
  double x0[3];
  double dx;
  double* U[4];
  double* prim;
  int8_t* status;
} grmhd_patch_desc;

typedef struct grmhd_c2p_stats {
  long long points;      /* points processed                          */
  long long iterations;  /* Brent iterations summed over both solves  */
  long long corrected;   /* points with a positive status             */
  long long failed;      /* points with a negative status             */
} grmhd_c2p_stats;

typedef struct grmhd_ctx grmhd_ctx;

/* Version of this ABI (increases when a signature changes; 2 since
 * grmhd_rhs_eval_static gained dev_flags). */
int grmhd_abi_version(void);

/* Creates a context for npatch patches (init_patches).  Validates the
 * descriptors (sizes >= 4 per axis, px >= n[0]+6, 8-byte-aligned non-NULL
 * pointers, dx > 0), copies them to the device and allocates the library's
 * scratch (pointwise and interface fluxes: 63 doubles per ghosted point).
 * eos may be NULL when p->eos_kind == 0.  stream: cudaStream_t or NULL.
 * Returns GRMHD_ERR_ARG / GRMHD_ERR_NOMEM / GRMHD_ERR_CUDA on failure, with
 * *out set to NULL. */
int grmhd_init_patches(grmhd_ctx** out, const grmhd_params* p, int npatch, const grmhd_patch_desc* d,
                       const grmhd_eos_table* eos, void* stream);

/* Initial data -> evolved state in register U[0] of patch `patch`:
 * chi = det(gamma)^(-1/3), gt = chi gamma, Khat = K, At = chi (K_ij - gamma_ij K/3),
 * Theta = 0, conserved variables from the primitives (Sec. II B definitions),
 * phibar = 0, then Gammahat^i = gt^ij gt^kl d_l gt_jk with the centred 4th-order
 * derivative at interior points, then the ghost fill of all fields.
 * id: device array [26][n2+6][n1+6][px] (ghosts included). */
int grmhd_init_state(grmhd_ctx* ctx, int patch, const double* id);

/* Fills the 3-deep ghost zones of register `reg` (0..3) of every patch
 * (periodic copy or linear extrapolation, axis by axis; for bc = 3 the
 * hierarchy fill described at grmhd_patch_desc).  The hierarchy fill computes
 * the coarse x-midpoints once per coarse row in the library's pointwise-flux
 * scratch of the coarser patches, so it invalidates the fluxes of an earlier
 * grmhd_con2prim: call grmhd_con2prim after it, as the substep does. */
int grmhd_ghost_fill(grmhd_ctx* ctx, int reg);

/* con2prim at every point (ghosts included) of register `reg` of every patch
 * (appendix "Conversion from conserved to primitive fields": Kastaun's
 * bracket mu_+ from eq. f_mu_plus, the master-function root on (0, mu_+],
 * the EOS validity clamps and the error policy; the conserved definitions
 * inverted are Sec. II B eq. def_con2prim).  Also forms the pointwise MHD flux
 * vectors (eq. mhd_system) and fast speeds (appendix "Characteristic
 * structure", eq. fast_waves) that grmhd_rhs_eval reads.  Writes prim and status; where a correction fired, the conserved variables
 * of `reg` are recomputed from the corrected primitives.  If stats is
 * non-NULL the call synchronises the stream and fills it. */
int grmhd_con2prim(grmhd_ctx* ctx, int reg, grmhd_c2p_stats* stats);

/* Right-hand side L(U) of register `reg` at interior points (Sec. III,
 * eq. PDEequation, the semi-discrete operator of the method of lines): the
 * CCZ4 + gauge right-hand side of Sec. II A (eqs. system1 .. system3) with the
 * centred, one-sided and Kreiss-Oliger operators of Sec. III B, plus the MHD
 * flux difference of Sec. III C (eqs. flux_decomposition, LLF2, MP5_unal ..
 * MP5_dm4) and the geometric sources of eq. mhd_system, from the
 * primitives and pointwise fluxes of the last grmhd_con2prim call.  rhs[p] is a device array with
 * the patch layout (32 fields); ghost entries are not written. */
int grmhd_rhs_eval(grmhd_ctx* ctx, int reg, double* const* rhs);

/* Stage combination (unfused), interior points, with k = rhs[p]: the explicit
 * half of the IMEX scheme of Sec. III A (eq. eq_IMEX with no stiff part), with
 * the coefficients of Table RK4 (explicit RK4(4,4)) or Table RK3SSP (explicit
 * SSP-RK(3,3)).  RK4:
 *   stage 0: U[1] = U[0] + dt/2 k, U[3] = U[0] + dt/6 k
 *   stage 1: U[2] = U[0] + dt/2 k, U[3] += dt/3 k
 *   stage 2: U[1] = U[0] + dt k,   U[3] += dt/3 k
 *   stage 3: U[0] = U[3] + dt/6 k
 * SSP-RK3 (rk = 1):
 *   stage 0: U[1] = U[0] + dt k, U[2] = U[0] + dt/4 k, U[3] = U[0] + dt/6 k
 *   stage 1: U[2] += dt/4 k, U[3] += dt/6 k
 *   stage 2: U[0] = U[3] + 2 dt/3 k */
int grmhd_rk_update(grmhd_ctx* ctx, int stage, double dt, double* const* rhs);

/* One fused substep `stage` of the time integrator (Sec. III A, method of
 * lines with the explicit stages of Table RK4 / Table RK3SSP): ghost fill of
 * the stage input (Sec. IV B), con2prim (appendix on the conversion from
 * conserved to primitive fields), right-hand side L(U) (eq. PDEequation) and
 * the stage combination of grmhd_rk_update, without storing k.  RK4 (rk = 0): stages 0..3, inputs U[0],
 * U[1], U[2], U[1].  SSP-RK3 (rk = 1): stages 0..2, inputs U[0] (Y1), U[1]
 * (Y2 = U^n + dt k1), U[2] (Y3 = U^n + dt/4 k1 + dt/4 k2); U[3] accumulates
 * U^n + dt/6 (k1 + k2) and the last stage writes U^{n+1} = U[3] + 2 dt/3 k3
 * into U[0]. */
int grmhd_rhs_substep(grmhd_ctx* ctx, int stage, double dt);

/* One full step of the time integrator (Sec. III A: U^{n+1} from the stages
 * of eq. eq_IMEX with the explicit tableaux of Table RK4 / Table RK3SSP; four
 * fused substeps for RK4, three for SSP-RK3); with bc = 3, followed by grmhd_restrict(ctx, 0).  With
 * sub-cycling on (grmhd_set_subcycling), dt is the level-0 step and one call
 * advances level l by 2^l steps of dt / 2^l (see below). */
int grmhd_step(grmhd_ctx* ctx, double dt);

/* Sub-cycling in time on a hierarchy (bc = 3; Sec. IV C, "Sub-cycling in
 * time", the BOR scheme, with the dense output of Sec. III A).  With on != 0,
 * grmhd_step(ctx, dt0) advances level l recursively: one step of
 * dt_l = dt0 / 2^l of level l, then two steps of level l + 1 and the
 * restriction of level l + 1 into level l.  During a step of level l >= 1 its
 * ghost points are copied from same-level interiors of the same stage, or
 * prolongated (six-point Lagrange, as for bc = 3) from the parent's stage value
 *   Y = c_0 U^n + c_1 D_1 + c_2 D_2 + c_3 D_3 + c_4 J
 * formed at each coarse stencil point: D_m = dt^m d^m U/dt^m at the parent's
 * t^n from the derivatives of the dense output b_j(theta) (RK4: third-order
 * interpolator; SSP-RK3: second-order), J = 4 (k3 - k2) = dt^3 f_U U'' +
 * O(dt^4) (RK4 only), and c the fine RK stages expanded in the Taylor data of
 * the interpolant at the start of the fine step, keeping RK4's third-order
 * f_U U'' terms.  The first call allocates five (RK4) or three (SSP-RK3)
 * dense registers per patch on the levels that have a finer level and
 * synchronises.  Returns GRMHD_ERR_ARG (message in grmhd_last_error) when
 * bc != 3 or when a prolongation stencil of a level >= 2 leaves the interiors
 * of the next coarser level (the dense output exists only there); on = 0
 * returns to synchronous steps.  A graph captured while on replays sub-cycled
 * steps. */
int grmhd_set_subcycling(grmhd_ctx* ctx, int on);

/* Restriction of a hierarchy (bc = 3; a no-op otherwise): every interior
 * point of a level-l patch at even level-l coordinates g overwrites, for all
 * fields of register reg, the interior point g/2 of the level-(l-1) patch that
 * holds it (direct copy, the paper's restriction operator); finest level
 * first. */
int grmhd_restrict(grmhd_ctx* ctx, int reg);

/* Captures nsteps grmhd_step calls into a CUDA graph owned by the context
 * (replacing a previous one); grmhd_graph_launch replays it on the stream. */
int grmhd_capture_graph(grmhd_ctx* ctx, int nsteps, double dt);
int grmhd_graph_launch(grmhd_ctx* ctx);

/* Synchronises the stream and returns the worst device-side condition since
 * the last call (GRMHD_OK, GRMHD_ERR_C2P_FATAL or GRMHD_ERR_NONFINITE), then
 * clears it. */
int grmhd_sync_status(grmhd_ctx* ctx);

/* Launch granularity.  With on != 0 every seeder, con2prim, LES,
 * interface-flux and right-hand-side launch covers one patch (one launch per
 * patch and kernel kind, in patch order, on the same stream): the plain
 * per-patch form that the batched launches (one per kernel kind over all
 * patches, the default, on = 0) are measured against.  Results are bitwise
 * the same in both forms; ghost fills and restrictions stay batched. */
int grmhd_set_per_patch(grmhd_ctx* ctx, int on);

/* Threads per block of the con2prim, interface-flux and right-hand-side
 * kernels (each 64, 128 or 256; 128 at creation). */
int grmhd_set_block_sizes(grmhd_ctx* ctx, int bs_c2p, int bs_iflux, int bs_rhs);

/* Autotuner (no counterpart in the paper), three phases on this context's own
 * patches, each timed with CUDA events:
 *   1. threads per block of the con2prim, interface-flux and right-hand-side
 *      kernels (64, 128, 256), from reps fused stage-0 substeps per candidate;
 *   2. a tile shape per patch-size class (longest edge <= 16, 24, 32, 48, 64,
 *      96, 128, larger) and kernel kind, each candidate shape's kernel timed
 *      alone on the class's patches (reps launches): 0 linear chunks of the
 *      block size, 1 row segments, 2 boxes of 32 x 2 x bs/64, 3 of
 *      16 x 4 x bs/64, 4 of 8 x 8 x bs/64 points;
 *   3. for con2prim and the interface fluxes, a persistent pool of blocks
 *      (as many as are resident at once, each looping over the work items)
 *      or one block per work item, from whole substeps.
 * It overwrites the stage registers U[1] and U[3] and may apply con2prim
 * corrections to U[0], so call it before stepping or between steps; it
 * discards a captured graph (capture again afterwards).  chosen (3 ints, may
 * be NULL) receives the block sizes kept for con2prim, interface fluxes and
 * right-hand side; grmhd_get_schedule returns the rest.  Synchronises. */
int grmhd_autotune(grmhd_ctx* ctx, double dt, int reps, int* chosen);

/* The launch schedule: shapes[3 * p + k] is the tile shape (0..4, see
 * grmhd_autotune) of patch p for kernel kind k (0 con2prim, 1 interface
 * fluxes, 2 right-hand side); pers[k] (k = 0, 1; pers[2] must be 0: the
 * right-hand-side kernel has no persistent form) selects the persistent pool.
 * Either pointer may be NULL (unchanged).  Every schedule computes every
 * point with the same arithmetic, so results do not depend on it.  Setting
 * a schedule synchronises and discards a captured graph. */
int grmhd_set_schedule(grmhd_ctx* ctx, const int* shapes, const int* pers);
int grmhd_get_schedule(grmhd_ctx* ctx, int* shapes, int* pers);

/* Per-kernel timing with CUDA events recorded on the context's stream around
 * each eager launch (not inside graph capture).  grmhd_profile(ctx, 1)
 * discards old records and starts recording; grmhd_profile(ctx, 0) stops.
 * grmhd_profile_read synchronises the stream, writes the summed milliseconds
 * and launch counts per kernel kind (0 ghost fill, 1 con2prim + pointwise
 * fluxes, 2 interface fluxes, 3 right-hand side + RK epilogue, 4 unfused RK
 * update, 5 initial data, 6 seeder inference, 7 sub-cycling dense-output
 * record and its ghosts, 8 LES SGS fluxes) into ms[0..nkinds) and
 * count[0..nkinds), and
 * discards the records. */
int grmhd_profile(grmhd_ctx* ctx, int on);
int grmhd_profile_read(grmhd_ctx* ctx, double* ms, long long* count, int nkinds);

/* Number of kernel launches the context has enqueued so far. */
long long grmhd_launch_count(grmhd_ctx* ctx);

/* Last error message of the context (static storage, never NULL). */
const char* grmhd_last_error(grmhd_ctx* ctx);

/* Frees the context's own memory and graphs (not the caller's arrays). */
void grmhd_destroy(grmhd_ctx* ctx);

/* ---- con2prim on independent states (flat metric, alpha = 1) ------------ */

/* Conserved (D, DYe, tau, S_i, B^i, phi) per state from primitives
 * (rho, eps, p, v^i, W, Ye, T, cs2; eps and p are recomputed from (rho, T, Ye)
 * with the EOS when p->eos_kind == 1) and B^i.
 * prim: device [n][10]; B: device [n][3]; cons: device [n][10]. */
int grmhd_prim2con_flat(const grmhd_params* p, const grmhd_eos_table* eos, long long n, const double* prim,
                        const double* B, double* cons, void* stream);

/* con2prim of n states with a flat metric (the isolated recovery workload).
 * cons: device [n][10]; prim: device [n][10]; status: device [n];
 * iters: device [n] or NULL.  From 2^16 states on, the states are solved in
 * an order grouped by the binary exponent of B^2 / D (warps then hold states
 * of similar root-finder cost); the order is a counting sort on the device
 * into n + 128 ints of stream-ordered scratch (cudaMallocAsync on `stream`,
 * freed after the solve's launch; if it cannot be had, the given order is
 * used).  Every state's result is independent of the order, bit for bit. */
int grmhd_c2p_flat(const grmhd_params* p, const grmhd_eos_table* eos, long long n, const double* cons,
                   double* prim, int8_t* status, int32_t* iters, void* stream);

/* ---- sharding a hierarchy across ranks --------------------------------------
 *
 * The paper decomposes the grid into boxes owned by MPI ranks (Sec. IV A)
 * and exchanges ghost data between them.  Here each rank (one GPU) evolves a
 * subset of the patches of a fixed mesh-refinement hierarchy (bc = 3) and, per
 * Runge-Kutta substep, receives once the source points its ghost fill reads
 * from other ranks' patches.  A point a ghost task reads is resolved to its
 * source: an interior point of some patch, or a level-0 ghost point (filled
 * on the level-0 patch's rank first).  This needs a nested hierarchy: every
 * prolongation stencil of a level l >= 2 inside interiors of level l-1.
 * Restriction becomes one copy per coarse point from the finest interior
 * point that coincides with it (the cascade of direct copies in one step),
 * with one more exchange per step.  Results are bitwise those of one context
 * holding every patch.
 *
 * Protocol of one RK step on every rank (stages s = 0.., input register
 * reg(s) as for grmhd_rhs_substep):
 *   for each stage: grmhd_shard_ghost0(ctx, reg); for every peer: pack the
 *   ghost-phase send list from reg, exchange, unpack the receive list into
 *   reg; grmhd_rhs_substep(ctx, s, dt) (fills levels 1.. and advances the
 *   rank's own patches);
 *   then: pack the restriction send lists from register 0, exchange, unpack
 *   into register 0, grmhd_restrict(ctx, 0). */

/* Owner rank (0..nranks-1) of every patch: Morton order of the patch centres
 * (finest-level grid units), cut into nranks runs of about equal interior
 * point count.  Host only; d needs geometry (n, px, level, x0, dx) only. */
int grmhd_shard_partition(int npatch, const grmhd_patch_desc* d, int nranks, int* owner);

/* Exchange plan of rank `rank` for the hierarchy d partitioned by owner.
 * Host only.  role (npatch ints, may be NULL): 0 the rank holds no array of
 * the patch, 1 the rank evolves it, 2 mirror (the rank holds an array that
 * receives source points).  counts (4 nranks): for every peer q, the numbers
 * of points of [ghost-phase send to q, ghost-phase receive from q,
 * restriction send to q, restriction receive from q]; q = rank is a local
 * copy.  lists (may be NULL for a size query; cap ints): for q = 0.. in
 * order, the four lists as (patch, offset) int pairs, offset in the patch's
 * ghosted layout; a send list on rank q and the matching receive list on
 * rank r have the same length and order (the source of the i-th sent value
 * lands at the i-th received point).  GRMHD_ERR_ARG when the hierarchy is
 * not nested (message on stderr); GRMHD_ERR_SIZE when cap is too small. */
int grmhd_shard_plan(int npatch, const grmhd_patch_desc* d, const int* owner, int nranks, int rank, int* role,
                     long long* counts, int* lists, long long cap);

/* Context of rank `rank` over the whole hierarchy d (every patch described;
 * the arrays of patches with role 0 in the plan may be NULL and are never
 * touched).  Evolves only the rank's own patches; ghost tasks only for them;
 * restriction as composed copies into them.  Sub-cycling and grmhd_step are
 * not available on it (see the protocol above). */
int grmhd_init_shard(grmhd_ctx** out, const grmhd_params* p, int npatch, const grmhd_patch_desc* d, const int* owner,
                     int nranks, int rank, const grmhd_eos_table* eos, void* stream);

/* Outer-boundary extrapolation of the level-0 patch (register reg) if this
 * rank evolves it; nothing otherwise. */
int grmhd_shard_ghost0(grmhd_ctx* ctx, int reg);

/* Gather (pack) / scatter (unpack) of the 32 fields of register reg at n
 * points: pts device [n][2] ints (patch, offset), buf device [32][n] doubles
 * (field-major).  Enqueued on the context's stream. */
int grmhd_shard_pack(grmhd_ctx* ctx, int reg, const int* pts, long long n, double* buf);
int grmhd_shard_unpack(grmhd_ctx* ctx, int reg, const int* pts, long long n, const double* buf);

/* ---- FP64 peak probe ------------------------------------------------------ */

/* Measurement aid with no counterpart in the paper: one launch of
 * blocks_per_sm (1..8) blocks of 256 threads per SM, each thread running
 * `chains` (4, 8 or 16) independent FP64 fused multiply-add chains for iters
 * iterations (rounded up to a multiple of 4); chains = -4, -8 or -16 runs
 * addition chains instead (the FP64 instruction rate of adds).  *fmas
 * receives the thread-level FMAs (or additions) of the launch (2 FP64 flops
 * per FMA); the caller times the
 * launch on `stream` with CUDA events to measure the FP64 peak that the
 * right-hand-side kernels are compared with.  sink: a device array of at
 * least blocks_per_sm * (SM count) doubles, written only in a case that does
 * not occur (it keeps the arithmetic from being optimised away). */
int grmhd_dfma_probe(int blocks_per_sm, int chains, long long iters, double* sink, long long* fmas, void* stream);

/* ---- allocation-free right-hand side -------------------------------------- */

/* No counterpart in the paper; this is a service for callers that must not
 * have the library allocate device memory (an application whose device memory
 * all belongs to its own pool allocator, a code path that cannot afford the
 * device synchronisation cudaMalloc / cudaFree may imply, a host framework
 * that allows allocation only through its own allocator).
 *
 * Same result as grmhd_con2prim(ctx, reg, NULL) followed by
 * grmhd_rhs_eval(ctx, reg, &rhs) on a context holding this single patch: con2prim
 * on U[reg] (writing prim, status and the corrected conserved variables into
 * U[reg]) and L(U) into rhs (device, patch layout, ghost entries untouched).
 * U[reg] must already hold filled ghost zones; only U[reg], prim and status
 * of the descriptor are used.  eos may be NULL for the ideal gas.
 *
 * dev_flags: NULL, or a device int (4-byte aligned) that receives, in stream
 * order after the kernels, this call's device error bits: bit 0 a fatal
 * con2prim point (also in the status array), bit 1 a non-finite conserved
 * state met by con2prim.  A non-finite right-hand-side value that arises
 * from finite inputs is not detected.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine: its working
 * memory (pointwise and interface fluxes, descriptor, work list, flags) is a
 * file-scope static device array of about 27.7 MB that every GPU which loads
 * the library holds until the process exits.  The descriptor, rhs and the
 * work list reach that array through a set-up kernel's arguments, not through
 * copies from host memory.  Patches are limited to
 * px * (n[1]+6) * (n[2]+6) <= 54872 ghosted points (a 32^3 patch); larger ones
 * return GRMHD_ERR_SIZE before any work is enqueued.  The first call on a device
 * looks up the array's device address with that device current; make that
 * first call before any stream capture.  All calls on a device share the
 * array and it keeps the last call's contents, so calls that may overlap on
 * the GPU (two streams of one device) race and must be serialised by the
 * caller; calls on one stream are ordered.  Work is enqueued on `stream`. */
int grmhd_rhs_eval_static(const grmhd_params* p, const grmhd_patch_desc* d, const grmhd_eos_table* eos, int reg,
                          double* rhs, int* dev_flags, void* stream);

/* ---- learned con2prim seeder ----------------------------------------------
 *
 * Not part of the paper's method: a small network that supplies starting
 * guesses for the two Brent root finds of the con2prim appendix.  The FP64
 * root finder still polishes every state with the paper's stop rule, and a
 * guess that does not bracket the root falls back to the plain bracket, so
 * the seeder changes evaluation counts, not results.
 *
 * Network: multilayer perceptron 8 -> 64 -> 64 -> 64 -> 3 with ReLU on the
 * hidden layers.  Products run on the tensor cores with BF16 operands (inputs,
 * weights, hidden activations and back-propagated gradients rounded to BF16,
 * round to nearest even) and FP32 accumulation; biases, master weights and
 * the Adam moments are FP32.
 *
 * Parameter vector (GRMHD_SEEDER_NPARAMS floats): W1[8][64], b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], W4[64][3], b4[3]; W[k][j] multiplies
 * input k into unit j.  Normalisation vector (GRMHD_SEEDER_NNORM floats):
 * feature mean[8], feature scale[8], target mean[3], target scale[3]; the
 * network sees x = (f - mean) / scale and its output y maps to the target
 * y * scale + mean.
 *
 * Features f of a conserved state (flat metric; D, DYe, tau, S_i, B^i as in
 * the cons arrays of grmhd_c2p_flat), with q = tau / D, r = |S| / D,
 * b2 = |B|^2 / D (Kastaun's scalars of the con2prim appendix) and
 * Q = max(1 + q, 1e-30).  q, r, b2, Q and (1 + q - r)(1 + q + r) are formed in
 * FP64; the logarithms of those quantities are taken in FP32:
 *   f0 = log10 D,      f1 = DYe / D,      f2 = ln Q,
 *   f3 = ln max((1 + q - r)(1 + q + r), 1e-30),   f4 = r / Q,
 *   f5 = log10 max(b2, 1e-30),   f6 = S.B / (|S| |B|) (0 if S or B is 0),
 *   f7 = b2 / Q.
 * Targets t from the roots (mu_+, mu) and the Lorentz factor W at mu:
 *   t0 = ln(mu_+ sqrt(1 + r^2)),  t1 = ln(mu Q),  t2 = ln W
 * (corrections to the unmagnetised closed forms mu_+ = 1 / sqrt(h0^2 + r^2)
 * and mu (1 + q) = 1 - p / (rho h W^2), with h0 ~ 1).
 * Seeds from targets: mu_+ = exp(t0) / sqrt(1 + r^2), mu = exp(t1) / Q,
 * W = exp(t2).
 */
#define GRMHD_SEEDER_NPARAMS 9091
#define GRMHD_SEEDER_NNORM 22

typedef struct grmhd_seeder grmhd_seeder; /* opaque: weights, Adam state, scratch */

typedef struct {
  int batch;       /* samples per Adam step: a multiple of 128 in [128, 65536] */
  int epochs;      /* passes over the training set (floor(n / batch) steps each) */
  float lr;        /* learning rate at the first step ... */
  float lr_final;  /* ... decaying as a half cosine to this value at the last */
  float beta1, beta2, eps; /* Adam constants */
  int fit_norm;    /* 1: first set the normalisation to the training set's
                      per-channel mean and standard deviation */
} grmhd_train_cfg;

/* Creates a seeder on the current device: weights uniform in
 * +-sqrt(6 / fan_in) from a splitmix64 stream of `seed`, zero biases, identity
 * normalisation (mean 0, scale 1), zero Adam state.  Synchronous. */
int grmhd_seeder_create(grmhd_seeder** out, unsigned long long seed);

/* Host copies of the parameters and/or the normalisation (either may be NULL).
 * set resets the Adam state; both synchronise the device. */
int grmhd_seeder_set_params(grmhd_seeder* s, const float* params, const float* norm);
int grmhd_seeder_get_params(grmhd_seeder* s, float* params, float* norm);

/* Features f (device float [n][8]) of the conserved states cons (device
 * double [n][10], as grmhd_c2p_flat). */
int grmhd_seeder_features(long long n, const double* cons, float* f, void* stream);

/* Targets t (device float [n][3]) of the states cons (device double [n][10])
 * from their roots (device double [n][3], as written by grmhd_c2p_flat_seeded
 * without seeds). */
int grmhd_seeder_targets(long long n, const double* cons, const double* roots, float* t, void* stream);

/* Network output mapped to targets: t = net((f - mean) / scale) * scale + mean.
 * f: device float [n][8]; t: device float [n][3]. */
int grmhd_seeder_forward(grmhd_seeder* s, long long n, const float* f, float* t_out, void* stream);

/* Gradient of the loss L = mean over the n samples and 3 outputs of
 * (net(x) - (t - mean) / scale)^2 with respect to the parameter vector
 * (device float [GRMHD_SEEDER_NPARAMS]), and L itself (device double [1]).
 * Uses the same kernels as the training step.  1 <= n <= 65536. */
int grmhd_seeder_grad(grmhd_seeder* s, long long n, const float* f, const float* t, float* grad, double* loss,
                      void* stream);

/* One Adam step with the gradient grad (device float [GRMHD_SEEDER_NPARAMS]),
 * as step number `step` (>= 1; sets the bias corrections), learning rate lr. */
int grmhd_seeder_adam(grmhd_seeder* s, const float* grad, long long step, float lr, float beta1, float beta2,
                      float eps, void* stream);

/* Trains on n pairs (f: device float [n][8], t: device float [n][3]): every
 * step a forward and backward pass over one batch, partial gradients per
 * 128-sample tile summed in a fixed order, then Adam; batches walk through the
 * set in order.  The epoch's steps are captured once in a CUDA graph that is
 * launched `epochs` times on `stream`.  loss_hist (device double [epochs] or
 * NULL) receives each epoch's mean loss.  Resets the Adam state first; keeps
 * the current weights as the starting point. */
int grmhd_seeder_train(grmhd_seeder* s, long long n, const float* f, const float* t, const grmhd_train_cfg* cfg,
                       double* loss_hist, void* stream);

/* Seeds (device double [n][3]: mu_+, mu, W) for the conserved states cons
 * (device double [n][10]): features, network and the seed map in one kernel.
 * The network runs on the tcgen05 tensor cores: 128-sample tiles, BF16
 * operands in shared memory, FP32 accumulators in tensor memory. */
int grmhd_seeder_infer(grmhd_seeder* s, long long n, const double* cons, double* seeds, void* stream);

/* Synchronises the device and returns GRMHD_ERR_TIMEOUT when an inference
 * kernel of this seeder gave up waiting for its tensor-core products (each
 * wait is bounded; the kernel then frees its tensor memory and stops), else
 * GRMHD_OK; clears the condition. */
int grmhd_seeder_status(grmhd_seeder* s);

/* Test hook for the timeout path above (no counterpart in the paper).  With
 * polls > 0 the inference kernels of this seeder (grmhd_seeder_forward,
 * grmhd_seeder_infer and the seeds of a context's con2prim) issue no
 * tensor-core products, so each bounded wait for a product gives up after
 * `polls` polls with nothing in flight: the kernel records GRMHD_ERR_TIMEOUT
 * (grmhd_seeder_status, or grmhd_sync_status for a context's seeds), frees its
 * tensor memory and stops, leaving the outputs it did not reach unwritten.
 * A seeded con2prim still gives the plain results (every seed is checked
 * against the bracket).  polls = 0 restores normal operation. */
int grmhd_seeder_hold_products(grmhd_seeder* s, int polls);

void grmhd_seeder_destroy(grmhd_seeder* s);

/* Seeded con2prim in the substep of a patch context: with a seeder set,
 * every con2prim pass (grmhd_con2prim, grmhd_rhs_substep, grmhd_step and the
 * captured graphs recorded afterwards) first runs the network on every point
 * (features from the conserved variables and the metric: the network's
 * inputs are functions of Kastaun's invariants q, r^2 = S_i S^i / D^2,
 * B_i B^i / D and S_i B^i, so the flat-metric training applies) and then
 * con2prim from those seeds with bracket half-width delta, as in
 * grmhd_c2p_flat_seeded.  Atmosphere and non-finite points get no seed.  The
 * first call allocates the seed buffer (3 floats per ghosted point) and
 * synchronises; s = NULL returns to the plain brackets.  The seeder must
 * outlive its use by the context. */
int grmhd_set_seeder(grmhd_ctx* ctx, const grmhd_seeder* s, double delta);

/* grmhd_c2p_flat with optional seeds (device double [n][3] or NULL).  The
 * mu seed s gives the bracket [s (1 - delta), min(s (1 + delta), 1 / h0)]:
 * (a) when f_a < 0 at its upper end the bracket lies below mu_+ (f_a changes
 * sign once, at mu_+) and the master root is found on it without solving for
 * mu_+; (b) otherwise mu_+ is solved, from the bracket
 * [s_+ (1 - delta), s_+ (1 + delta)] of the mu_+ seed when f_a changes sign on
 * it, and the mu seed bracket is clipped to mu_+.  A seed bracket on which the
 * function keeps its sign (or a seed that is not finite and positive) falls
 * back to the plain bracket of that step; results agree with the plain solve
 * to the root finder's tolerance.  iters counts every evaluation of the
 * auxiliary and master functions.  roots (device double [n][3] or NULL)
 * receives (mu_+, mu, W at mu), zeros where a root find failed and mu_+ = 0
 * when it was not solved; seeded (device int8 [n] or NULL): bit 0 the mu_+
 * seed bracket was used, bit 1 the mu seed bracket, bit 2 mu_+ was not solved.
 * The third seed (W) is not used.  The processing order and its scratch are
 * those of grmhd_c2p_flat. */
int grmhd_c2p_flat_seeded(const grmhd_params* p, const grmhd_eos_table* eos, long long n, const double* cons,
                          const double* seeds, double delta, double* prim, int8_t* status, int32_t* iters,
                          double* roots, int8_t* seeded, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GRMHD_H */
