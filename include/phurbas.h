/*
 * phurbas.h - C ABI of the GB300 (sm_103a) particle right-hand-side library.
 *
 * The library evaluates the data-parallel hot path of the Phurbas meshless
 * Lagrangian MHD method (McNally, Maron & Mac Low, Paper II, arXiv:1110.0836):
 *   - strict fixed-radius neighbour sets, r_f,i = 2.3 lambda_i (Sec. 2, Sec. 2.1);
 *   - the local third-order interpolating moving-least-squares fit of rho, V,
 *     B and sigma (Sec. 2; Acknowledgements: interpolating fits), its
 *     derivatives, and the ideal-MHD Lagrangian time derivatives with bulk
 *     viscosity and diffusive div B correction (Sec. 2; App. A);
 *   - the second-order predictor-corrector step (Sec. 2, Sec. 4.2), with a
 *     mask of fixed-value particles (Sec. 3);
 *   - individual power-of-two time-step levels with the spatial limiter and
 *     the right-hand side of an active subset (Sec. 2, Sec. 2.1);
 *   - particle adaptivity: the void and clump scan and the deletion and
 *     creation of particles (Sec. 2, Sec. 2.1);
 *   - a hand-written adjoint of the fit + right-hand side (not in the paper).
 *
 * Conventions for every entry point:
 *   - Array arguments named pos, lambda, U, dudt, grad, hess, gbar, Ubar, xbar,
 *     zeta, eta, ws, status_word are DEVICE pointers owned by the caller.
 *     Layout is structure-of-arrays float64: pos [3][n], U [8][n] with field
 *     order (rho, Vx, Vy, Vz, Bx, By, Bz, sigma), sigma the internal energy
 *     density with P = (gamma - 1) sigma (reading of Sec. 2: the paper names
 *     sigma but defers the equation of state to Paper I).
 *   - Particle index i is the caller's index; internally particles are
 *     re-ordered by cell, and results are returned in the caller's order.
 *   - The library allocates no device memory: all scratch lives in the
 *     caller-provided workspace `ws` of `ws_bytes` bytes, whose size is given
 *     by phb_workspace_size.  Neighbour lists live in the workspace between
 *     calls; a workspace belongs to one plan.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and performs no host synchronisation, so call sequences
 *     can be captured into CUDA graphs.
 *   - Errors found on the host are returned as phb_status.  Errors found on
 *     the device are OR-ed as PHB_FLAG_* bits into *status_word (an int32 in
 *     device memory that the caller zeroes); read it after synchronising and
 *     map it with phb_check.  No call throws, traps or spins without bound.
 */
#ifndef PHURBAS_H
#define PHURBAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* phb_stream_t; /* same type as cudaStream_t */

typedef enum {
  PHB_OK = 0,
  PHB_ERR_INVALID_ARG = 1, /* null pointer, n <= 0, bad box/lambda range, r_f >= len/2 */
  PHB_ERR_WORKSPACE = 2,   /* ws_bytes smaller than phb_workspace_size */
  PHB_ERR_CUDA = 3,        /* a CUDA launch or memset failed */
  PHB_ERR_CAPACITY = 4,    /* neighbour list larger than plan.nbr_capacity */
  PHB_ERR_SKIN = 5,        /* predictor moved a particle by more than skin/2 */
  PHB_WARN_FIT = 6,        /* at least one fit was singular (its derivatives are 0) */
  PHB_ERR_TIMEOUT = 7,     /* reserved for a bounded device wait that gave up (never
                              returned: no kernel of this library waits on another) */
  PHB_ERR_NONFINITE = 8    /* a non-finite input or result was seen */
} phb_status;

/* Device status-word bits (OR-ed by kernels). */
#define PHB_FLAG_CAPACITY 0x01
#define PHB_FLAG_SKIN 0x02
#define PHB_FLAG_FIT_SINGULAR 0x04
#define PHB_FLAG_NONFINITE 0x08
#define PHB_FLAG_TIMEOUT 0x10 /* reserved: no kernel waits on another, so none sets it */
#define PHB_FLAG_LAMBDA_RANGE 0x20 /* a lambda outside the plan's [lambda_min, lambda_max] */
#define PHB_FLAG_BAD_INDEX 0x40    /* an active-subset index outside [0, n) (it was skipped) */

/* Periodic or open box [lo, lo + len) per axis.  On a periodic axis offsets
 * use the minimum image d - len * nearbyint(d / len).  Particles on an open
 * axis may lie anywhere; cells clamp them to the box. */
typedef struct {
  double lo[3];
  double len[3];
  int32_t periodic[3];
  int32_t pad_;
} phb_box;

typedef enum { PHB_FP64 = 0, PHB_FP32_MIXED = 1 } phb_precision;

/* Method parameters. */
typedef struct {
  double gamma;          /* adiabatic index, P = (gamma - 1) sigma */
  int32_t weight_kind;   /* MLS weight: 0 = (1 - s^2)^2 with s = |d| / r_f,i; 1 = unweighted */
  int32_t precision;     /* phb_precision */
  double cond_threshold; /* FP32_MIXED: fits whose conditioning estimate
                            exceeds this (0 = default 3e4) are redone in FP64.
                            Estimate: 19 x a LINPACK-style greedy estimate of
                            ||M_s^-1||_inf of the Jacobi-scaled 19x19 normal
                            matrix M_s (one forward and one back substitution
                            with the FP32 factor); it follows cond_2(M_s)
                            within a factor ~0.4-1.8 on the test sets */
  const double* zeta;    /* bulk viscosity per particle [n], or NULL for 0 */
  const double* eta;     /* div B diffusivity per particle [n], or NULL for 0 */
  const uint8_t* frozen; /* phb_pc_step only: device mask [n] (caller order) or
                            NULL.  A particle with frozen[i] != 0 keeps its
                            position and state through the step (the
                            fixed-value boundaries of the Sec. 3 tests); its
                            right-hand side is still evaluated and it stays a
                            neighbour of the others.  Read by no other call. */
  /* Coefficient laws added to zeta and eta (0 = off).  Sec. 2 says what the
   * two bulk-viscosity fields and the div B diffusion do, not their form; the
   * forms read here, with the fast-speed bound c = sqrt((gamma P + |B|^2)/rho):
   *   zeta_i += c_zeta_l lambda_i c_i + c_zeta_a lambda_i^2 max(0, -div V_i)
   *   eta_i  += c_eta lambda_i c_i
   * (grid-scale damping at the signal speed; damping that grows with
   * compression, as at shocks; div B diffusion at the resolution scale).
   * Every right-hand-side, adjoint and step call applies them. */
  double c_zeta_l;
  double c_zeta_a;
  double c_eta;
  /* FP32_MIXED only: one corrected semi-normal-equations step (Bjorck) after
   * the FP32 solve: residuals r_j = (U_j - U_i) - p(q_j).c recomputed from the
   * neighbour data, P^T W r accumulated and solved with the same factor, so
   * the coefficient error follows cond(A) = cond(M_s)^(1/2) rather than
   * cond(M_s).  It costs about one more fit.  The decision is per tile of
   * particles: refine = 0 refines a tile when any of its fits has a
   * conditioning estimate (as for cond_threshold) above refine_kappa (0 =
   * default 500; the fits of a jittered lattice stay below ~330, about 40% of
   * the fits of a density-sampled set lie above 500, and there even
   * well-conditioned fits leak the large linear coefficients of a steep
   * front into the quadratic ones); refine = 1 refines every tile; refine =
   * -1 never refines. */
  int32_t refine;
  /* Where the corrected step of refined tiles runs: 0 = by the set (a second
   * kernel over a queue of the refined tiles' fits when n x 96 B of FP32
   * records fit in the device's L2 and lambda varies - sets of one
   * resolution rarely refine and skip that launch - inside the tile
   * otherwise), 1 = the queue, 2 = inside the tile (other values: as 0).
   * Same results either way. */
  int32_t refine_schedule;
  double refine_kappa;
} phb_params;

/* A plan fixes the particle count, box, radius law and the cell grid.  The
 * caller fills the input fields and calls phb_plan_init, which fills the rest.
 * Every lambda passed later must lie in [lambda_min, lambda_max]. */
typedef struct {
  /* inputs */
  phb_box box;
  int64_t n;             /* number of particles */
  double rf_factor;      /* r_f,i = rf_factor * lambda_i (2.3 in the paper, Sec. 2) */
  double skin;           /* list radius = r_f,i + skin (0: exact lists) */
  double lambda_min;
  double lambda_max;
  int64_t nbr_capacity;  /* entries reserved for neighbour lists (sum of |N(i)|) */
  double cell_frac;      /* cell edge / (rf_factor*lambda_min + skin); 0 = default 1 */
  int32_t tile;          /* particles per fused-fit tile (64 or 128; 0 = default 128) */
  int32_t stage_cap;     /* neighbourhood records staged per tile (0 = default) */
  int32_t schedule;      /* fused fit: 0 = one CTA per tile in cell order; 1 = one CTA per
                            tile in descending-cost order (longest lists first) */
  int32_t ell_width;     /* neighbour search: list entries kept per particle in the
                            single-pass scratch (0 = default: 128, or 256 when
                            lambda_max > 1.26 lambda_min; longer lists are
                            searched again); 8 .. 1024 */
  /* filled by phb_plan_init */
  double cell[3];        /* cell edge per axis */
  int32_t ncell[3];      /* cells per axis (at most 1023) */
  int32_t nbrick[3];     /* 4x4x4-cell bricks per axis */
  int32_t hilbert_bits;  /* bricks are ordered along a 3-D Hilbert curve of this order */
  int32_t ntiles;        /* ceil(n / tile) */
  int64_t nkeys;         /* cell-key space: bricks * 64 */
  double screen_margin;  /* absolute distance margin of the FP32 neighbour screen */
  size_t ws_bytes;       /* workspace bytes needed for every operation */
  size_t ws_off[48];     /* byte offsets of the workspace regions (internal) */
} phb_plan;

/* Operations for phb_workspace_size. */
#define PHB_OP_ALL 0

/* Fill the derived fields of *plan.  Host only.  Returns PHB_ERR_INVALID_ARG
 * for n <= 0, non-positive lengths or lambda range, rf_factor <= 0, skin < 0,
 * or when the list radius of lambda_max reaches half a periodic box length. */
phb_status phb_plan_init(phb_plan* plan);

/* Workspace bytes needed by `op` under `plan` (0 for an invalid plan). */
size_t phb_workspace_size(const phb_plan* plan, int32_t op);

/* Parts of the workspace, for callers that size or inspect it by use. */
#define PHB_PART_COMMON 0  /* neighbour lists, fits, right-hand sides, levels, adaptivity:
                              every call other than the two below needs only this part */
#define PHB_PART_STEP 1    /* phb_pc_step's state and right-hand sides (after the common part) */
#define PHB_PART_ADJOINT 2 /* phb_rhs_adjoint's scratch (after the common part; overlays the
                              step part, the two are never used at the same time) */

/* Byte range [*begin, *end) of workspace part `part` under `plan`; a call that
 * uses the part needs ws_bytes >= *end.  Host only.  Returns 0, or 1 for an
 * invalid plan, part or NULL output. */
int phb_workspace_part(const phb_plan* plan, int32_t part, size_t* begin, size_t* end);

/* Text for a phb_status code (static storage). */
const char* phb_status_string(int32_t status);

/* Map a device status word (already copied to the host) to the most severe
 * phb_status it encodes. */
phb_status phb_check(int32_t status_word);

/* Sizes of the ABI structs as this library was compiled: out[0] =
 * sizeof(phb_box), out[1] = sizeof(phb_params), out[2] = sizeof(phb_plan),
 * for the first `count` (1..3) of them, so a binding can check its copy of
 * the layouts.  Host only, no device call.  Returns 0, or 1 for a NULL out or
 * a count outside 1..3. */
int phb_struct_sizes(int64_t* out, int32_t count);

/* Build the neighbour sets of all particles (Sec. 2; Sec. 2.1: strict,
 * fixed radius, not mutual, no iteration):
 *   N(i) = { j != i : ((dx*dx + dy*dy) + dz*dz) < r*r },  r = rf_factor*lambda_i + skin,
 * with d = pos_j - pos_i (minimum image on periodic axes), evaluated in FP64
 * in exactly this order without fused multiply-adds, so the sets are
 * bit-exact.  Bins particles into the plan's cell grid with a counting sort
 * (stable by caller index) and stores the lists in the workspace.  Device
 * errors: PHB_FLAG_CAPACITY when the lists exceed plan->nbr_capacity (lists
 * are then incomplete), PHB_FLAG_LAMBDA_RANGE.  pos [3][n], lambda [n]. */
phb_status phb_build_neighbors(const phb_plan* plan, const double* pos, const double* lambda,
                               void* ws, size_t ws_bytes, int32_t* status_word,
                               phb_stream_t stream);

/* Particle adaptivity scan (Sec. 2: particles are added to voids and deleted
 * from clumps so that every sphere of radius r_f stays well sampled; Sec.
 * 2.1: the void search measures distances from the points of a 9^3 grid to
 * the neighbour particles and drops every point found close to one).  The
 * thresholds are Paper I's and are readings here.  With the lists of the
 * last build (pos and lambda may have moved since, within the skin), for
 * every particle i, r = rf_factor lambda_i, h = r / 4, d_v = void_factor
 * lambda_i, d_c = clump_factor lambda_i:
 *   test points o_k = h (kx, ky, kz), kx, ky, kz in -4..4, grid index
 *   k = ((kx+4) 9 + (ky+4)) 9 + (kz+4), those with |o_k| < r - d_v; a point
 *   is covered when i or a particle of its r_f set lies closer than d_v;
 *   void_count[i] = uncovered points; best[i] = the uncovered point whose
 *   nearest particle is farthest (lowest k on ties), -1 if none;
 *   cand [3][n] = x_i + o_best (0 if none), the place for a new particle;
 *   clump[i] = 1 when a neighbour with a smaller index lies closer than d_c
 *   (of a too-close pair the larger index is the one to delete).
 * Distances that decide an output are FP64 in the order written, so the
 * outputs are exact.  All outputs device arrays in caller order, each may be
 * NULL.  0 < void_factor < rf_factor and 0 <= clump_factor < rf_factor, else
 * PHB_ERR_INVALID_ARG. */
phb_status phb_adapt_scan(const phb_plan* plan, const double* pos, const double* lambda,
                          double void_factor, double clump_factor, void* ws, size_t ws_bytes,
                          int32_t* void_count, int32_t* best, double* cand, int32_t* clump,
                          int32_t* status_word, phb_stream_t stream);

/* Particle deletion and creation from a phb_adapt_scan of the same state and
 * build (Sec. 2: particles are added in voids and deleted in clumps; how is
 * Paper I's, the readings here): a particle marked as a clump is deleted; a
 * surviving particle i with a void creates one particle at cand_i when that
 * point lies inside the box on every open axis, unless a neighbour j < i of
 * its r_f set creates one closer than void_factor lambda_i to it; the new
 * particle takes lambda_i and the second-order Taylor value of i's fit at
 * o = cand_i - x_i, U + sum_a (grad_a o_a + sum_b ((hess_ab / 2) o_a) o_b),
 * from grad [8][3][n] and hess [8][6][n] of phb_mls_derivs.  Outputs of
 * leading dimension cap (pos_out [3][cap], lambda_out [cap], U_out [8][cap],
 * origin [cap]): survivors in order (origin = old index), then the new
 * particles in parent order (origin = n + parent); m_out (device int64) is
 * the new count - above cap nothing past cap is written and
 * PHB_FLAG_CAPACITY is raised.  Inputs and outputs are device arrays in
 * caller order; the plan and its lists stay those of the old set. */
phb_status phb_adapt_apply(const phb_plan* plan, const double* pos, const double* lambda,
                           const double* U, const int32_t* best, const double* cand,
                           const int32_t* clump, const double* grad, const double* hess,
                           double void_factor, int64_t cap, double* pos_out, double* lambda_out,
                           double* U_out, int64_t* origin, int64_t* m_out, void* ws,
                           size_t ws_bytes, int32_t* status_word, phb_stream_t stream);

/* Put the caller's particle arrays into the library's storage order - the
 * cells of the last build along their Hilbert curve, members of a cell by
 * caller index - as a tree code keeps its particles in Peano-Hilbert order
 * (Sec. 2.1).  After the call particle i of pos, lambda and U is the one the
 * last build stored in slot i; the plan's lists already refer to the new
 * numbering (no rebuild needed), and later builds keep the order up to the
 * particles' drift, so the gathers from and scatters to the caller's arrays
 * read and write contiguous runs.  pos [3][n] and lambda [n] must hold the
 * values of the last phb_build_neighbors call (U [8][n] any); all three are
 * permuted in place through the workspace.  perm_out (device int32 [n], may
 * be NULL) receives the old index of each new index, for the caller's other
 * per-particle arrays (zeta, eta, frozen).  PHB_ERR_INVALID_ARG for NULL
 * arrays. */
phb_status phb_reorder(const phb_plan* plan, double* pos, double* lambda, double* U,
                       int32_t* perm_out, void* ws, size_t ws_bytes, int32_t* status_word,
                       phb_stream_t stream);

/* Copy the lists of the last phb_build_neighbors out in the caller's
 * numbering: off [n+1] (int64, device), idx [capacity] (int32, device) with
 * the neighbours of i at idx[off[i] .. off[i+1]) in increasing index order.
 * Returns PHB_ERR_CAPACITY (and writes nothing) when idx_capacity is too
 * small for the total, which is read from the device (synchronising). */
phb_status phb_export_neighbors(const phb_plan* plan, const void* ws, int64_t* off, int32_t* idx,
                                int64_t idx_capacity, phb_stream_t stream);

/* Total neighbour-list entries of the last build (synchronises). */
int64_t phb_neighbor_total(const phb_plan* plan, const void* ws, phb_stream_t stream);

/* MLS fit derivatives of all 8 fields (Sec. 2: local, third-order polynomial
 * moving least squares over N(i); interpolating: the constant term is U_i):
 * minimise sum_j w_j (p(q_j).c - (U_j - U_i))^2 with q_j = d_ij / lambda_i,
 * p = the 19 monomials of degree 1..3, w_j = (1 - |d_ij|^2 / r_f,i^2)^2.
 * grad [8][3][n]: dU/dx_a = c_a / lambda_i;  hess [8][6][n] (xx,xy,xz,yy,yz,zz,
 * may be NULL): c_ab / lambda_i^2, doubled on the diagonal.  fit_status [n]
 * (may be NULL): 0 ok, 1 singular (fewer than 19 neighbours or a failed
 * factorisation: derivatives 0), 2 solved in FP64 after FP32 routing.
 * Uses the lists of the last phb_build_neighbors; entries farther than r_f,i
 * (skin) are skipped. */
phb_status phb_mls_derivs(const phb_plan* plan, const phb_params* params, const double* pos,
                          const double* lambda, const double* U, void* ws, size_t ws_bytes,
                          double* grad, double* hess, int32_t* fit_status, int32_t* status_word,
                          phb_stream_t stream);

/* Ideal-MHD Lagrangian time derivatives (Sec. 2; App. A), mu_0 = 1:
 *   Drho/Dt   = -rho div V
 *   DV/Dt     = [-(gamma-1) grad sigma + (curl B) x B] / rho + zeta_i grad(div V)
 *   DB/Dt     = (B.grad) V - B div V + eta_i grad(div B)
 *   Dsigma/Dt = -gamma sigma div V + rho zeta_i (div V)^2
 * from the fused fit (as phb_mls_derivs) at every particle.  dudt [8][n].
 * dx/dt = V needs no call.  fit_status as in phb_mls_derivs. */
phb_status phb_mhd_rhs(const phb_plan* plan, const phb_params* params, const double* pos,
                       const double* lambda, const double* U, void* ws, size_t ws_bytes,
                       double* dudt, int32_t* fit_status, int32_t* status_word,
                       phb_stream_t stream);

/* One second-order predictor-corrector step in place (Sec. 2; read as Heun):
 *   Y^p = Y^n + dt F(Y^n);  Y^{n+1} = Y^n + dt/2 (F(Y^n) + F(Y^p)),
 * Y = (x, U), dx/dt = V, lambda unchanged.  Builds the neighbour lists once
 * at x^n with radius r_f + plan->skin and filters them at r_f for both
 * evaluations; if the predictor moves any particle by more than skin/2 it
 * sets PHB_FLAG_SKIN (the step used incomplete sets; rebuild with a larger
 * skin).  pos [3][n] and U [8][n] are updated in place. */
phb_status phb_pc_step(const phb_plan* plan, const phb_params* params, double* pos,
                       const double* lambda, double* U, double dt, void* ws, size_t ws_bytes,
                       int32_t* status_word, phb_stream_t stream);

/* phb_pc_step on HOST arrays: pos_in [3][n], lambda_in [n], U_in [8][n]
 * (caller order, page-locked for the copies to run asynchronously) are copied
 * to the workspace's step part, stepped as by phb_pc_step, and x^{n+1}, U^{n+1}
 * copied back to pos_out [3][n] and U_out [8][n] (host; they may be pos_in and
 * U_in).  The positions and lambda go first; U follows on a side stream (one
 * per device, made on first use and kept) while the neighbour lists are built,
 * and the stream waits for it before U is read; x^{n+1}, which needs only V^n
 * and V^p, is corrected right after the predictor and downloaded on the side
 * stream while the second right-hand side runs.  When U_out is page-locked
 * and mapped (cudaHostAlloc / cudaHostRegister memory under unified
 * addressing) in the FP32-mixed precision, the corrector's fused fit writes
 * U^{n+1} of its final fits straight to U_out wherever the 32 particles of a
 * warp have caller indices within 64 of each other (storage order,
 * phb_reorder), and the rest (fits routed to FP64 or queued for the corrected
 * step, frozen particles, scattered warps) follows by a kernel after the
 * step; otherwise U^{n+1} is copied back once at the end.  All of it is ordered on
 * `stream`: the outputs are valid once the stream has reached this point (a
 * synchronisation, an event).  Capturable in a CUDA graph after one eager
 * call.  The side stream and its events are shared by all calls on a device:
 * calls issued concurrently from several host threads must be serialised by
 * the caller.  Same results and status as phb_pc_step; PHB_ERR_INVALID_ARG
 * also for a NULL output. */
phb_status phb_pc_step_host(const phb_plan* plan, const phb_params* params, const double* pos_in,
                            const double* lambda_in, const double* U_in, double* pos_out,
                            double* U_out, double dt, void* ws, size_t ws_bytes,
                            int32_t* status_word, phb_stream_t stream);

/* Right-hand side of an active subset only (the individual time steps of
 * Sec. 2 / Sec. 2.1: at a substep only the particles whose step ends there
 * are evaluated).  Same result as phb_mhd_rhs at the listed particles, with
 * the lists of the last build; dudt [8][n] and fit_status [n] (may be NULL)
 * are written at the listed caller indices only.  active: device int32
 * [n_active] caller indices (duplicates are evaluated once; an index outside
 * [0, n) is skipped and sets PHB_FLAG_BAD_INDEX).  The FP32-mixed path reads
 * neighbours through the unstaged (global-memory) form of the fused fit; the
 * FP64 path is the same kernel as the full evaluation.  Every particle's
 * pos, lambda and U are still read (neighbours of active particles). */
phb_status phb_mhd_rhs_active(const phb_plan* plan, const phb_params* params, const double* pos,
                              const double* lambda, const double* U, const int32_t* active,
                              int64_t n_active, void* ws, size_t ws_bytes, double* dudt,
                              int32_t* fit_status, int32_t* status_word, phb_stream_t stream);

/* Individual power-of-two time-step levels (Sec. 2: steps independent of
 * the bulk velocity, spatial variation limited; Sec. 2.1: steps rounded
 * down to powers of two, the restriction sent from a particle to its
 * neighbours).  With the lists of the last build (filtered exactly at r_f),
 * for every particle: c_i = sqrt((gamma P_i + |B_i|^2) / rho_i), P = (gamma - 1)
 * sigma, dt_i = cfl lambda_i / c_i (FP64, no contraction); unlimited level
 * L0_i = the smallest L in [0, max_level] with dt_max / 2^L <= dt_i (or
 * max_level); then one limiter pass L_j = max(L0_j, max over i with j in N(i)
 * of L0_i - 1).  A particle of level L advances with dt_max / 2^L.
 * levels: device int32 [n], caller order.  dt_max > 0, cfl > 0,
 * 0 <= max_level <= 30, else PHB_ERR_INVALID_ARG; a non-positive density or
 * squared speed sets PHB_FLAG_NONFINITE. */
phb_status phb_timestep_levels(const phb_plan* plan, const phb_params* params, const double* pos,
                               const double* lambda, const double* U, double cfl, double dt_max,
                               int32_t max_level, void* ws, size_t ws_bytes, int32_t* levels,
                               int32_t* status_word, phb_stream_t stream);

/* Individual power-of-two time steps (Sec. 2: each particle has its own step,
 * independent of the bulk velocity; Sec. 2.1: rounded down to powers of two
 * and organised as GADGET's binary blocks), every particle advanced by the
 * second-order predictor-corrector (read as Heun).  The paper leaves the
 * scheme to GADGET; the readings implemented:
 *   - a synchronised step of dt_max is cut into 2^max_level substeps of
 *     delta = dt_max / 2^max_level; a particle of level L (levels from
 *     phb_timestep_levels) takes steps of m = 2^(max_level - L) substeps, all
 *     starting together at the synchronised time;
 *   - each particle keeps an anchor: its state (x0, U0) and F0 = dU/dt at the
 *     start of its current step; at substep time t its current state is the
 *     prediction (x0, U0) + (t - t0) (V0, F0), the predictor itself when its
 *     step ends at t;
 *   - at substep time t the particles whose step ends there are corrected:
 *     F = dU/dt at the current states of all particles (neighbour sets built
 *     at the current positions), x = x0 + (D/2)(V0 + V), U = U0 + (D/2)(F0 +
 *     F), D = m delta; dU/dt at the corrected states (the others still at
 *     their predictions) is their new anchor's F0.
 * With every particle on one level a synchronised step is the plain Heun step.
 * anchor: caller-owned device double [19][n], caller order: x0 [3], U0 [8],
 * F0 [8].  phb_block_begin fills it at a synchronised time from pos, U (one
 * full right-hand side); phb_block_substep(k) advances from substep k to
 * k + 1 (0 <= k < 2^max_level, in order): pos and U (in-out) become the
 * current states at t_{k+1}; after the last substep every particle is
 * synchronised at t + dt_max and the anchor continues into the next step
 * (levels may change there).  levels: device int32 [n]; a level outside
 * [0, max_level] is clamped and sets PHB_FLAG_BAD_INDEX.  0 <= max_level <=
 * 30 and dt_max > 0, else PHB_ERR_INVALID_ARG.  Uses the step part of the
 * workspace (PHB_PART_STEP) and rebuilds the plan's neighbour lists. */
phb_status phb_block_begin(const phb_plan* plan, const phb_params* params, const double* pos,
                           const double* lambda, const double* U, double* anchor, void* ws,
                           size_t ws_bytes, int32_t* status_word, phb_stream_t stream);
phb_status phb_block_substep(const phb_plan* plan, const phb_params* params, double* pos,
                             const double* lambda, double* U, double* anchor,
                             const int32_t* levels, int32_t k, int32_t max_level, double dt_max,
                             void* ws, size_t ws_bytes, int32_t* status_word, phb_stream_t stream);

/* Reverse-mode derivative of the fused fit + right-hand side (not in the
 * paper): given gbar = dL/d(dudt) [8][n], returns Ubar = dL/dU [8][n] and
 * xbar = dL/dpos [3][n] with the neighbour sets of the last build held fixed
 * and lambda treated as a constant.  Recomputes each factorisation (no stored
 * factors); contributions to neighbours are gathered through a reverse
 * neighbour list, so the result is deterministic.  FP64. */
phb_status phb_rhs_adjoint(const phb_plan* plan, const phb_params* params, const double* pos,
                           const double* lambda, const double* U, const double* gbar,
                           void* ws, size_t ws_bytes, double* Ubar, double* xbar,
                           int32_t* status_word, phb_stream_t stream);

/* Stored-factorisation variant of phb_rhs_adjoint (not in the paper; offered
 * to compare memory and time against recomputation).
 * phb_adjoint_record_bytes(plan): bytes of the per-particle record, 343
 * doubles per particle = the Jacobi-scaled Cholesky factor of the 19 x 19
 * normal matrix (190), its scaling (19), the fitted coefficients of the seven
 * fields V, B, sigma (7 x 19) and a singular flag, [343][n] in the
 * workspace's slot order.  0 for an invalid plan.
 * phb_adjoint_record: FP64 fits of every particle with the lists of the last
 * build; writes the record (device, caller-owned, >= record_bytes).
 * phb_rhs_adjoint_stored: the same result as phb_rhs_adjoint, starting from
 * a record made with the same plan, lists, pos, lambda and U (not checked;
 * a stale record gives wrong gradients).  Both return PHB_ERR_INVALID_ARG
 * for a NULL or too small record; otherwise as phb_rhs_adjoint. */
size_t phb_adjoint_record_bytes(const phb_plan* plan);
phb_status phb_adjoint_record(const phb_plan* plan, const phb_params* params, const double* pos,
                              const double* lambda, const double* U, void* ws, size_t ws_bytes,
                              double* record, size_t record_bytes, int32_t* status_word,
                              phb_stream_t stream);
phb_status phb_rhs_adjoint_stored(const phb_plan* plan, const phb_params* params,
                                  const double* pos, const double* lambda, const double* U,
                                  const double* gbar, void* ws, size_t ws_bytes,
                                  const double* record, size_t record_bytes, double* Ubar,
                                  double* xbar, int32_t* status_word, phb_stream_t stream);

/* Mode-amplitude diagnostic of the Kelvin-Helmholtz test (Sec. 3.4: the
 * growth of the unstable y-velocity mode measured by a discrete convolution
 * over the particles instead of a Fourier transform of gridded values):
 *   e_i = exp(-k |y~_i - y0|), y~ = y where y < ly / 2, ly - y elsewhere (a
 *   layer at y0 and its mirror image at ly - y0),
 *   s = sum_i Vy_i sin(k x_i) e_i,  c = sum_i Vy_i cos(k x_i) e_i,
 *   d = sum_i e_i^2,  M = 2 [ (s / d)^2 + (c / d)^2 ]^(1/2),
 * over all plan->n particles.  The paper's set-up: k = 4 pi, y0 = 1, ly = 4.
 * pos [3][n] and U [8][n] device arrays (any particle order); out: device
 * double [4] = (s, c, d, M).  FP64; the sums are formed in a fixed order, so
 * repeated calls give identical results.  k > 0, ly > 0 and finite y0, else
 * PHB_ERR_INVALID_ARG. */
phb_status phb_kh_mode_amplitude(const phb_plan* plan, const double* pos, const double* U, double k,
                                 double y0, double ly, void* ws, size_t ws_bytes, double* out,
                                 phb_stream_t stream);

/* Neighbour build + fused right-hand side (phb_build_neighbors followed by
 * phb_mhd_rhs) without any device allocation and without a caller workspace.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory where they need the right-hand side (a pool that forbids new
 * allocations, a framework that owns every device buffer, a loop that must
 * not block on the allocator).  The caller still passes pos, lambda, U, dudt,
 * fit_status (may be NULL) and status_word as in phb_mhd_rhs.
 *   - Scratch: one file-scope device array of phb_noalloc_scratch_bytes()
 *     (32 MiB) that every GPU which loads the library holds until exit.  A
 *     plan whose build-and-fit workspace (everything before the
 *     predictor-corrector regions) is larger returns PHB_ERR_WORKSPACE and
 *     launches nothing; with constant lambda this allows roughly 15,000
 *     particles.
 *   - Every call looks up the array's device address in the current context
 *     (cudaGetSymbolAddress, a host-side query), so the call stays valid after
 *     cudaDeviceReset and under any context.  The first call in a context
 *     also loads the library's device code there: make it before any stream
 *     capture.
 *   - Every call shares the array and leaves its contents behind; the kernels
 *     clear what must start at zero.  Calls that overlap on the GPU (other
 *     streams, other threads) race on the array: serialise them.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
phb_status phb_mhd_rhs_noalloc(const phb_plan* plan, const phb_params* params, const double* pos,
                               const double* lambda, const double* U, double* dudt,
                               int32_t* fit_status, int32_t* status_word, phb_stream_t stream);

/* Size in bytes of the scratch array used by phb_mhd_rhs_noalloc. */
size_t phb_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* PHURBAS_H */
