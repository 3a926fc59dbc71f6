/*
 * pdn.h - C ABI of the GB300 explicit impact step with partial
 * Dirichlet-Neumann (PDN) contact.
 *
 * Method: Guillamet, Quintanas-Corominas, Rivero, Houzeaux, Vazquez, Turon,
 * "Application of the partial Dirichlet-Neumann contact algorithm to simulate
 * low-velocity impact events on composite structures", Composites Part A
 * (2022), arXiv 2301.05552.  Section, equation and algorithm numbers below
 * refer to that paper.
 *
 * One library context owns one laminated plate (hex8 plies, zero-thickness
 * interface elements between plies of different angle), its lumped mass,
 * its damage history and one rigid spherical striker, all resident in the
 * memory of the current CUDA device.  Every per-step operation runs in the
 * library's CUDA kernels on the stream given at creation.
 *
 * Conventions for every call:
 *   - Units: mm, N, tonne, s, MPa.
 *   - Return value 0 on success, a negative PDN_E_* code on failure; the
 *     context's pdn_last_error() then holds a one-line message.  No C++
 *     exception crosses this interface.
 *   - Input arrays are owned by the caller and copied during the call;
 *     output arrays are owned by the caller and written during the call.
 *     Pointers are host pointers unless a parameter says otherwise.
 *   - Node and element ids are the caller's (0-based) numbering.
 *   - Nodal vector fields are structure-of-arrays: [3][n_nodes] doubles
 *     (all x, then all y, then all z).
 *   - Calls on one context are not thread-safe; distinct contexts are
 *     independent.
 */
#ifndef PDN_H
#define PDN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define PDN_OK 0
#define PDN_E_ARG (-1)           /* invalid argument, size or mesh */
#define PDN_E_CUDA (-2)          /* CUDA runtime error (message says which) */
#define PDN_E_OOM (-3)           /* device allocation failed */
#define PDN_E_NONFINITE (-4)     /* a nodal acceleration or displacement became NaN/Inf */
#define PDN_E_RELEASE_LIMIT (-5) /* a step still had adhesive contact nodes after
                                    max_release_iters repetitions (Algorithm 2) */
#define PDN_E_TIMEOUT (-6)       /* a bounded device wait gave up (the batched launch's
                                    grid barrier, the learned law's tensor-core wait) */
#define PDN_E_UNSTABLE (-7)      /* material/mesh gives no stable step (and, for the
                                    learned law, a snap-back length: pdn_surrogate.h) */
#define PDN_E_STATE (-8)         /* call out of order (e.g. step before set_impactor) */

/* Precision of the element force, damage and cohesive updates.  Nodal
 * displacement/velocity accumulation, the striker state and the contact gap
 * test are always FP64. */
#define PDN_FP64 0       /* element arithmetic in FP64 */
#define PDN_FP32_FORCE 1 /* element arithmetic in FP32, nodal integration in FP64 */

/* Fields for pdn_damage_field (one value per element, maximum over its
 * integration points). */
#define PDN_FIELD_D1 0   /* fibre damage max(d_FT, d_FC), per hex */
#define PDN_FIELD_D2 1   /* matrix damage max(d_MT, d_MC), per hex */
#define PDN_FIELD_D6 2   /* shear damage d_6, per hex */
#define PDN_FIELD_DCOH 3 /* interface damage threshold r_D (Algorithm 5), per interface element */
#define PDN_FIELD_PLASTIC 4 /* equivalent plastic shear strain, per hex */

/* Kernel ids for pdn_profile_kernels. */
#define PDN_K_CONTACT 0
#define PDN_K_HEX 1
#define PDN_K_COH 2
#define PDN_K_GATHER 3
#define PDN_K_TAIL 4
#define PDN_K_COUNT 5

typedef struct pdn_ctx pdn_ctx;

/* Mesh of one plate (Sec. 2, Sec. 3.2).  All arrays are copied.
 *   X         [3][n_nodes] reference coordinates (mm).
 *   hex       [n_hex][8] hex8 connectivity: bottom face counter-clockwise
 *             seen from +z, then the top face in the same order.
 *   coh       [n_coh][8] zero-thickness interface elements: the 4 nodes of the
 *             lower face, then the 4 coincident nodes of the upper face in the
 *             same order.  May be NULL when n_coh == 0.
 *   ply_of_hex [n_hex] ply index of each hex (0 <= ply < n_plies).
 *   ply_angle_deg [n_plies] fibre angle of each ply about +z (degrees); the
 *             material axes are fixed in the reference configuration.
 *   fixed     [n_nodes] constraint bits: 1 = x, 2 = y, 4 = z held at zero
 *             displacement (7 = clamped).  May be NULL (all free).
 *   surf      [n_surf] ids of the contact-surface (slave) nodes. */
typedef struct {
  int64_t n_nodes, n_hex, n_coh, n_surf;
  const double *X;
  const int32_t *hex;
  const int32_t *coh;
  const int8_t *ply_of_hex;
  const double *ply_angle_deg;
  int32_t n_plies; /* 1..64 */
  const uint8_t *fixed;
  const int32_t *surf;
} pdn_mesh_desc;

/* Ply and interface material (Table 1 layout; MPa, N/mm, t/mm^3).
 * Intralaminar law (Sec. 2.3.1, Algorithm 4): elastic constants, strengths,
 * fracture angle alpha0, fracture toughnesses, shear yield stress Sp and
 * hardening ratio Kp (hardening modulus Kp*G12).  Interface law (Sec. 2.3.2,
 * Algorithm 5): GIc, GIIc, strengths tauI, tauII, Benzeggagh-Kenane
 * exponent eta, penalty stiffness KI (mode I; the shear penalty follows as
 * KI (GIc/GIIc)(tauII/tauI)^2).  Strengths XT, YT, SL of each hex are scaled
 * by seeded factors uniform in [1 - spread, 1 + spread] (SplitMix64 of
 * seed ^ (4*element + k), k = 0, 1, 2). */
typedef struct {
  double rho, E1, E2, E3, nu12, nu13, nu23, G12, G13, G23;
  double XT, XC, YT, YC, SL, alpha0_deg;
  double GXT, GXC, GYT, GYC, GSL;
  double Sp, Kp;
  double GIc, GIIc, tauI, tauII, eta, KI;
  double spread;
  uint64_t seed;
} pdn_material;

/* Run options.
 *   precision       PDN_FP64 or PDN_FP32_FORCE.
 *   damage_on       1: intralaminar and interface damage laws active.
 *   plasticity_on   1: shear plasticity of Algorithm 4 active.
 *   max_release_iters  repetitions of a step allowed for releasing adhesive
 *                   contact nodes (Algorithm 2); 0 selects 8; a negative
 *                   value allows none (the first adhesive node is an error).
 *   phi             Tchamwa-Wielgosz parameter (Sec. 2.2.1); 1 = central
 *                   difference; 0 selects 1.
 *   dt              time step (s); 0 = dt_safety * min(dt_bulk, dt_coh).
 *   dt_safety       factor on the stable step; 0 selects 0.5.
 *   gravity         body acceleration (mm/s^2) on plate and striker.
 *   history_cap     number of per-step contact-force samples kept on the
 *                   device; 0 selects 1<<20.
 *   stream          cudaStream_t on which all work is issued (NULL = the
 *                   legacy default stream). */
typedef struct {
  int32_t precision;
  int32_t damage_on;
  int32_t plasticity_on;
  int32_t max_release_iters;
  double phi;
  double dt;
  double dt_safety;
  double gravity[3];
  int64_t history_cap;
  void *stream;
} pdn_options;

/* Counters and derived quantities of a context. */
typedef struct {
  double dt, dt_bulk, dt_coh;
  double time;
  double f_peak;           /* maximum contact force along the impact axis so far */
  int64_t step;            /* committed steps */
  int64_t n_active;        /* contact nodes at the last committed step */
  int64_t n_repeats;       /* step repetitions for node release so far */
  int64_t n_nodes, n_hex, n_coh, n_surf;
  int64_t device_bytes;    /* device memory held by the context */
  int32_t status;          /* sticky device status (PDN_OK or an error code) */
  int32_t precision;
  int32_t hex_variant;     /* element-kernel launch variant chosen by the autotuner:
                              0..3 hex kernel (interface kernel on a forked stream)
                              with an occupancy target of 4, 5, 6 or 3 blocks/SM;
                              4..7 one mixed hex + interface kernel with the same
                              targets (never chosen by the autotuner, which times
                              0..3).  The environment variable PDN_HEX_VARIANT
                              (0..7) fixes it instead (no timing, tune_ms 0) */
  int32_t sweep;           /* 0: separate element, interface and gather kernels; 1, 2, 3:
                              the column sweep (FP32 box hexes, flat interfaces, a plate
                              layered as a full grid of columns) with tiles of 16 x 8,
                              8 x 8 or 8 x 4 columns: one kernel evaluates the elements
                              layer by layer and updates every node inside a tile from
                              shared memory; only tile-boundary nodes go through the
                              element-force slots.  Planned by pdn_init_mesh only when the
                              environment variable PDN_SWEEP=1 is set there and the mesh
                              allows it (it measured slower than the separate kernels),
                              and kept by the first pdn_step while PDN_SWEEP=1 is still
                              set; a planned sweep keeps the interface elements
                              (coh_pairs 0) */
  int32_t coh_pairs;       /* 1, 2: interfaces evaluated as node pairs inside the gather (flat
                              interfaces, at most eight elements per node, no column sweep):
                              with Newton-Cotes points at the corners (Sec. 2.3.2) the
                              traction at a point depends only on the jump of the two
                              coincident nodes there, so the law is evaluated once per node
                              and each incident element's share added in CSR order, with
                              the same sums as the interface kernel; no interface kernel
                              runs; 2 where the node numbering is layered (blocks of
                              consecutive ids are node layers and a node's partner is the
                              same position in the next layer), so that the gather finds
                              the partner from the node id, 1 otherwise (a partner table).
                              0: interface elements (k_coh).  The environment
                              variable PDN_COH_PAIRS=0, read by pdn_init_mesh, keeps the
                              interface elements.  With 2, a node of an interface layer
                              owns 4 element-force slots instead of 8 (its interface
                              elements write none), unless PDN_SLOTS_COMPACT=0 is set at
                              pdn_init_mesh */
  int32_t reserved;
  double tune_ms[12];      /* mean time of an internal-force pass with each variant when
                              tuned (0 if not): entries 0..3 the hex variants with separate
                              kernels, entry 8 the column sweep (0 where none was planned);
                              the fastest is used.  Entries 4..7, 9..11 unused */
} pdn_info;

/* Create a context on the current CUDA device: validate and copy the mesh,
 * compute the lumped (row-sum) mass, the characteristic lengths and stable
 * steps (Sec. 2.3.1: dt = lc sqrt(rho/max Cij), lc = V^(1/3); Sec. 2.3.2:
 * dt_coh = sqrt(rho_bar/K) with rho_bar = rho * adjacent hex thickness), the
 * node-to-element CSR map used for the deterministic force gather, and
 * allocate all device state (displacement, velocity, history double buffers).
 * Initial state: d = v = 0, damage thresholds r = 1, plastic strain 0,
 * interface thresholds 0 (Algorithms 4, 5), and the acceleration a^0 of the
 * momentum equation at step 0 (Sec. 2.2.1; no contact at t^0): the gravity
 * acceleration on every free degree of freedom.  One internal-force pass runs
 * on the device for it.  On failure *out is NULL. */
int pdn_init_mesh(pdn_ctx **out, const pdn_mesh_desc *mesh, const pdn_material *mat,
                  const pdn_options *opt);

/* Set the rigid spherical striker (Sec. 2.2.2): radius (mm), mass (t),
 * centre (mm) and velocity (mm/s).  The striker moves only along the unit
 * vector of its initial velocity (its other degrees of freedom are held, as
 * in Sec. 3.2); a zero velocity selects -z.  Resets the contact force to 0. */
int pdn_set_impactor(pdn_ctx *ctx, double radius, double mass, const double centre[3],
                     const double velocity[3]);

/* Advance nsteps explicit steps (Algorithm 1 per step): striker RK4 update
 * with the previous contact force (Eq. rk4); contact detection and
 * projection of penetrated and still-active surface nodes onto the sphere
 * (Dirichlet condition, Sec. 2.1); hex8 and interface internal forces with
 * trial damage history; deterministic CSR gather; lumped-mass accelerations
 * with the contact reactions; release of adhesive nodes (f^c . n < 0,
 * Eq. anodes) with repetition of the step (Algorithm 2); Tchamwa-Wielgosz
 * update (Sec. 2.2.1).  A repetition evaluates again only the elements of the
 * released nodes and the nodes of those elements (everything else has the
 * same inputs as before and keeps its values); the environment variable
 * PDN_FULL_REPEAT=1, read by pdn_init_mesh, makes repetitions evaluate every
 * element and node, with the same results.  The kernels of a pass are
 * launched with programmatic dependent launch (each waits for the previous
 * grid before reading); PDN_PDL=0, read once per process, launches them
 * plainly, with the same results.  Returns after the work has completed on
 * the stream.
 * Errors: PDN_E_STATE without a striker, PDN_E_NONFINITE,
 * PDN_E_RELEASE_LIMIT (both sticky), PDN_E_CUDA. */
int pdn_step(pdn_ctx *ctx, int64_t nsteps);

/* Contact force of the striker on the plate (Sec. 2.2.2: f^e = sum_j f^c_j):
 * f_now[3] at the last committed step, *f_peak the largest component along
 * the impact axis so far, and history[k] (k < cap) the component along the
 * impact axis after step k+1.  Any output pointer may be NULL.  Returns the
 * number of history samples written (>= 0), or, when history is NULL, the
 * number of samples available; negative values are error codes. */
int64_t pdn_contact_force(pdn_ctx *ctx, double f_now[3], double *f_peak, double *history,
                          int64_t cap);

/* Damage field `which` (PDN_FIELD_*), one float per hex (or per interface
 * element for PDN_FIELD_DCOH): the maximum over the element's integration
 * points of the committed history.  n must equal the element count of the
 * field.  out is a device pointer when out_on_device != 0. */
int pdn_damage_field(pdn_ctx *ctx, int32_t which, float *out, int64_t n, int32_t out_on_device);

/* Committed state: displacement d and velocity v ([3][n_nodes], the
 * Tchamwa-Wielgosz velocity of Sec. 2.2.1) and imp[10] = striker centre[3],
 * velocity[3], contact force[3], time.  Any pointer may be NULL. */
int pdn_get_state(pdn_ctx *ctx, double *d, double *v, double *imp);

/* Install displacement and velocity ([3][n_nodes]; constrained degrees of
 * freedom are forced to zero) and recompute the acceleration from the
 * internal forces without contact, as at a restart.  History and contact
 * set are kept. */
int pdn_set_state(pdn_ctx *ctx, const double *d, const double *v);

/* Contact set of the last committed step: active[n_surf] (1 = in contact)
 * and the reaction magnitude lambda[n_surf] along each node's sphere normal
 * (0 where inactive).  Either pointer may be NULL. */
int pdn_get_contact(pdn_ctx *ctx, uint8_t *active, double *lambda);

/* Committed damage history, for checkpoints and for checks against another
 * solver of the same model.  hist [7][8][n_hex]: field f of Gauss point g of
 * hex e at (f*8 + g)*n_hex + e, fields rFT rFC rMT rMC gp12 gp13 pbar
 * (Algorithm 4: the four damage thresholds, the two plastic shear strains and
 * the equivalent plastic strain).  rD [4][n_coh]: threshold of Newton-Cotes
 * point p of interface element e at p*n_coh + e (Algorithm 5).  Both in the
 * element precision: float for PDN_FP32_FORCE, double for PDN_FP64.  Host
 * pointers owned by the caller; either may be NULL. */
int pdn_get_history(pdn_ctx *ctx, void *hist, void *rD);

/* Acceleration a^n of the committed step n ([3][n_nodes]): the lumped-mass
 * acceleration with the contact reactions of that step (Sec. 2.2.1, Eq.
 * anodes), 0 on constrained degrees of freedom -- the acceleration the next
 * step's Tchamwa-Wielgosz predictor uses.  The library keeps the predicted
 * velocity v' = v + dt a instead of a; the value returned is (v' - v)/dt,
 * equal to a up to FP64 rounding.  Host pointer owned by the caller. */
int pdn_get_acceleration(pdn_ctx *ctx, double *a);

/* Energy ledger at the committed state (Sec. 3.2 reports the energy-time
 * curves of the impact), evaluated on the device in FP64:
 *   out[0] kinetic energy of the plate, 1/2 sum_j m_j v_j . v_j with the
 *          velocity at the committed time level, v + dt/2 a (the stored
 *          velocity of the scheme is the central-difference one half a step
 *          back at phi = 1)
 *   out[1] kinetic energy of the striker, 1/2 M w . w
 *   out[2] energy stored in the hexes: sum over Gauss points of
 *          det J * 1/2 sigma : eps_e (ply axes; eps_e the Green strain minus the
 *          plastic shear strains; sigma the law's nominal stress at the
 *          committed history, Algorithm 4 -- the secant energy of the damaged
 *          material)
 *   out[3] energy stored in the interface elements: sum over Newton-Cotes
 *          points of 1/2 w tau . Delta (Algorithm 5 at the committed thresholds)
 *   out[4] work of gravity since the striker was set: sum_j m_j g . d_j +
 *          M g . (c - c_set)
 *   out[5] the striker's kinetic energy when it was set (pdn_set_impactor)
 * For a plate set in motion only by the striker, out[5] + out[4] - (out[0] +
 * out[1] + out[2] + out[3]) is the energy dissipated by damage, plasticity
 * and the time integrator: zero up to the integrator's error in an elastic
 * impact.  Units mJ (N mm).  Host pointer out[6]. */
int pdn_energies(pdn_ctx *ctx, double out[6]);

/* Nodal internal force f^i ([3][n_nodes]) at the committed state, computed
 * by the same element and gather kernels as a step, without advancing and
 * without changing the history. */
int pdn_internal_force(pdn_ctx *ctx, double *f_int);

/* Counters; see pdn_info. */
int pdn_get_info(pdn_ctx *ctx, pdn_info *info);

/* Advance nsteps steps launching each kernel directly (no graph) with CUDA
 * events around every launch on the context's stream, and return the mean
 * device time per launch of each kernel in ms_per_launch[PDN_K_COUNT] and
 * the launch counts in launches[PDN_K_COUNT] (either may be NULL).  The
 * steps are real steps of the simulation. */
int pdn_profile_kernels(pdn_ctx *ctx, int64_t nsteps, float *ms_per_launch, int64_t *launches);

/* Release all device memory of the context.  NULL is ignored. */
void pdn_destroy(pdn_ctx *ctx);

/* Largest mesh pdn_internal_force_noalloc accepts (its static scratch). */
#define PDN_NOALLOC_MAX_HEX 8192
#define PDN_NOALLOC_MAX_NODES 16384

/* Nodal internal force of a hex8 mesh for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is a library service.
 *
 * Who needs it: code that runs under a memory manager owning all device
 * memory (a framework's caching allocator, a fixed device-memory budget)
 * and must not call cudaMalloc/cudaFree itself, or that must avoid their
 * implicit device synchronisation in steady state.  Such a caller cannot
 * create a context (pdn_init_mesh allocates).  This call computes the same
 * quantity as pdn_internal_force, with the same element and gather kernels,
 * from caller buffers, and calls no allocating routine: its working memory
 * (element forces, slot positions, mirrors, trial history, control block,
 * about 10.8 MB) is a fixed array in device global memory that every device
 * loading this library holds until the process exits.
 *
 * Device pointers (all caller-owned): hex [n_hex][8] and ply_of_hex [n_hex]
 * as in pdn_mesh_desc (node ids in [0, n_nodes), ply ids in [0, n_plies));
 * X and d [3][n_nodes] FP64; history [7][8][n_hex] in the element precision
 * (float for PDN_FP32_FORCE, double for PDN_FP64: fields rFT rFC rMT rMC
 * gp12 gp13 pbar per Gauss point), read only, or NULL for the undamaged
 * state; csr_row [n_nodes+1] and csr_col [8 n_hex], the node -> element slot
 * map: csr_col[csr_row[j] .. csr_row[j+1]) lists 8*e + k for every hex e
 * whose local node k is j, in ascending order, so that csr_col is a
 * permutation of 0 .. 8 n_hex - 1; f_int [3][n_nodes] output.
 * Host pointers: mat, ply_angle_deg [n_plies].  stream is a cudaStream_t
 * (NULL = legacy default stream); the call only enqueues work on it.
 *
 * Errors: PDN_E_ARG (message from pdn_last_error(NULL)) when n_hex exceeds
 * PDN_NOALLOC_MAX_HEX, n_nodes exceeds PDN_NOALLOC_MAX_NODES, a pointer is
 * NULL or a parameter is invalid; PDN_E_CUDA on a launch failure.  Device
 * contents are not validated (out-of-range ids are the caller's fault).
 *
 * Every call looks up the device address of the scratch array in the
 * current context (cudaGetSymbolAddress, a host-side query), so a reset
 * device or another context on the same device gets its own array.  The
 * first call in a context loads the library's device code there; make it
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents; each call rewrites what it reads.  Calls whose work
 * overlaps on the GPU (several streams or host threads on one device) race
 * and must be serialised by the caller. */
int pdn_internal_force_noalloc(int64_t n_nodes, int64_t n_hex, const int32_t *hex, const int8_t *ply_of_hex,
                               const double *X, const double *d, const void *history, const int32_t *csr_row,
                               const int32_t *csr_col, const pdn_material *mat, const double *ply_angle_deg,
                               int32_t n_plies, int32_t precision, int32_t damage_on, int32_t plasticity_on,
                               double *f_int, void *stream);

/* Last error message of a context (never NULL); with ctx == NULL, the last
 * error of a failed pdn_init_mesh in this thread. */
const char *pdn_last_error(const pdn_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PDN_H */
