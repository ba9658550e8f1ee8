/*
 * lbib.h -- C ABI of the GB300 (sm_103a) lattice-Boltzmann / immersed-boundary
 * solver for red cells and adhesive carriers in a capillary.
 *
 * Method: Coclite, "Vascular journey and adhesion mechanics of micro-sized
 * carriers in narrow capillaries", arXiv 1907.00080.  One time step runs, on
 * the GPU, in this order:
 *   forces at X^n (bond springs Eq. adhFor, repulsion Eq. repFor, stretching
 *   Eq. strainFor, bending Eq. bendFor, enclosed area Eq. areaFor) ->
 *   IB shape functions (MLS with Roma weights on the nine nearest nodes,
 *   Sec. 2.2 / 2.3) -> spreading of the marker forces into the Guo body force
 *   (Eq. ForcingTerm) fused into the D2Q9 BGK collide-and-stream (Eqs. BGK,
 *   feq, GaussHermite, forcedBGK) -> interpolation of u^n to the markers
 *   (Sec. 2.3) -> kinematic advance (Eq. kinematicPos; forward Euler on the
 *   first step) -> bond rupture and formation at X^{n+1} (Sec. 2.2,
 *   wall-particle interaction).
 *
 * Units: lattice units throughout (dx = dt = 1, rho_0 = 1).  The lattice has
 * NX nodes along the periodic x axis and NY fluid rows y = 0..NY-1; with
 * LBIB_WALLS_Y_BOUNCEBACK the walls sit half a node outside, at y = -1/2 and
 * y = NY - 1/2 (half-way bounce-back); with LBIB_WALLS_ZOU_HE they are the
 * rows y = 0 and y = NY - 1 themselves (wet nodes: after streaming, the three
 * populations that would come from outside are rebuilt by Zou and He's
 * known-velocity condition from the wall's velocity, lbib_set_wall_velocity,
 * and the known ones; the populations' momentum is the wall velocity less the
 * node's Guo half-force, so the collision sees the wall velocity); with
 * LBIB_WALLS_NONE y is periodic as well.  Zou-He walls start from rest
 * (LBIB_INIT_REST) or from written populations, and take kinematic and
 * rigid-projected membranes only; the derivative forms refuse them.
 *
 * Conventions for every call:
 *  - every call returns an lbib_status; lbib_last_error() gives a message;
 *  - inputs are copied, the caller keeps ownership of every pointer it passes;
 *    the library owns all device state it allocates in lbib_create /
 *    lbib_add_membrane / lbib_set_receptors and frees it in lbib_destroy;
 *  - `on_device` = 1 means the pointer is CUDA device memory on the context's
 *    device, 0 means host memory;
 *  - work is enqueued on the context's stream; read-backs synchronise it;
 *  - a context is not thread-safe: one host thread drives it at a time;
 *  - after LBIB_E_NONFINITE the context is poisoned and lbib_step returns
 *    LBIB_E_STATE.
 */
#ifndef LBIB_H
#define LBIB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbib_ctx lbib_ctx;

typedef enum {
    LBIB_OK = 0,
    LBIB_E_INVALID = 1,   /* bad argument (null pointer, size, range)        */
    LBIB_E_CUDA = 2,      /* a CUDA runtime call failed                       */
    LBIB_E_OOM = 3,       /* device allocation failed                         */
    LBIB_E_TIMEOUT = 4,   /* a bounded device-side wait gave up               */
    LBIB_E_NONFINITE = 5, /* a marker position became NaN/Inf, or a spread
                             force (|w F| >= 64 lu per vertex and node) or a
                             repulsion magnitude (>= 1 per vertex and segment,
                             i.e. overlapping membranes) left the range of its
                             fixed-point accumulator (the value was clamped) */
    LBIB_E_STATE = 6      /* call not valid in the current state              */
} lbib_status;

/* Population storage.  All forms store the deviation d_i = f_i - w_i of each
 * population from its lattice weight (round-off reduction); the 16-bit forms
 * store d_i * 2^k with k chosen at creation and compute in FP32. */
typedef enum {
    LBIB_F64 = 0,
    LBIB_F32 = 1,
    LBIB_F32_STORE_F16 = 2,
    LBIB_F32_STORE_BF16 = 3
} lbib_precision;

typedef enum {
    LBIB_WALLS_NONE = 0,          /* periodic in x and y (e.g. shear-wave tests) */
    LBIB_WALLS_Y_BOUNCEBACK = 1,  /* half-way bounce-back walls in y            */
    LBIB_WALLS_ZOU_HE = 2         /* Zou-He known-velocity walls on the rows y = 0
                                     and y = NY - 1 (Sec. 2.1); see below      */
} lbib_walls;

typedef enum {
    LBIB_INIT_REST = 0,        /* f_i = w_i (rho = 1, u = 0)                        */
    LBIB_INIT_POISEUILLE = 1,  /* tau = 1 discrete Poiseuille fixed point of the
                                  body force along x (needs bounce-back walls)   */
    LBIB_INIT_COUETTE = 2      /* planar Couette flow between the walls moving at
                                  the velocities of lbib_set_wall_velocity (rest
                                  until they are set); the discrete fixed point
                                  at tau = 1 (needs bounce-back walls)            */
} lbib_init;

typedef enum {
    LBIB_MEMBRANE_KINEMATIC = 0,       /* Eq. kinematicPos with the interpolated velocity */
    LBIB_MEMBRANE_RIGID_PROJECTED = 1, /* same, velocity first projected on the
                                          least-squares rigid motion of the ring  */
    LBIB_MEMBRANE_DYNAMIC = 2,         /* dynamic IB, deformable particle (Sec. 2.4):
                                          Eqs. newtonSoft, verletPos, verletVel  */
    LBIB_MEMBRANE_DYNAMIC_RIGID = 3    /* dynamic IB, rigid particle (Sec. 2.4):
                                          Eqs. linearVelRig, angularVelRig      */
} lbib_kind;

typedef struct {
    int32_t nx, ny;          /* lattice size; nx, ny >= 4.  Any nx for FP64 and
                                FP32 (row tiles take odd nx; the persistent form
                                needs 16-byte rows: nx a multiple of 2 in FP64,
                                4 in FP32, 8 in 16-bit storage, else the default
                                tiling is row tiles); even nx for 16-bit storage */
    lbib_precision prec;
    lbib_init init;
} lbib_lattice;

/* Bond model (Sec. 2.2): spring sigma (y - y_eq) along ligand->receptor,
 * ligand point = centroid of its element, force split half/half to the two
 * element vertices.  Per step, at X^{n+1}: rupture first (if d >= d_break or
 * u < P_r(d)), then formation (ligands free after rupture, receptors free at the
 * start of the step, d < d_cut, first receptor in ascending id with
 * u < P_f(d); a receptor goes to the lowest ligand id), where
 *   P_f(d) = 1 - exp(-kf_dt * exp(-beta_f ((d - y_eq)/y_eq)^2)),
 *   P_r(d) = 1 - exp(-kr0_dt * exp( beta_r ((d - y_eq)/y_eq)^2)),
 * and u is the Philox4x64-10 draw for counter (step, ligand, receptor, tag)
 * (tag 0 formation, 1 rupture), key (seed, instance): u = (x0 >> 11) 2^-53. */
typedef struct {
    double d_cut, y_eq, sigma, kf_dt, kr0_dt, beta_f, beta_r, d_break;
    uint64_t seed, instance;
} lbib_bond_params;

/* Create a context.  tau: BGK relaxation time (Eq. BGK; nu = (tau - 1/2)/3).
 * body_force: uniform G_body (2 doubles) added to the spread IB force.
 * cuda_stream: a cudaStream_t to enqueue on, or NULL for a library-owned
 * stream.  Allocates the two population buffers (9 NX NY elements each).
 * Errors: LBIB_E_INVALID (sizes, odd nx with 16-bit storage, tau <= 1/2,
 * POISEUILLE without walls), LBIB_E_OOM, LBIB_E_CUDA. */
lbib_status lbib_create(const lbib_lattice* lattice, double tau, const double body_force[2],
                        lbib_walls walls, void* cuda_stream, lbib_ctx** out);

/* Add a closed membrane ring (Sec. 2.2): xy holds 2n doubles (x0,y0,x1,y1,..),
 * counter-clockwise, unwrapped x; the given shape is the stress-free state that
 * fixes the rest lengths l_0, rest angles theta_0 and rest area A_0.  Element k
 * joins vertices k and (k+1) mod n.  k_s, k_b, k_area: Eqs. strainFor, bendFor,
 * areaFor (p_ref = 1/3).  ligand_elems: local element ids carrying one ligand
 * each (NULL if n_ligands = 0).  Must precede the first lbib_step.
 * membrane_id_out may be NULL.  Errors: LBIB_E_INVALID, LBIB_E_STATE. */
lbib_status lbib_add_membrane(lbib_ctx* ctx, const double* xy, int32_t n, double k_s, double k_b,
                              double k_area, lbib_kind kind, const int32_t* ligand_elems,
                              int32_t n_ligands, int32_t* membrane_id_out);

/* Dynamic particles (kinds LBIB_MEMBRANE_DYNAMIC and LBIB_MEMBRANE_DYNAMIC_RIGID,
 * Sec. 2.4).  Per step, at X^n, from the populations f^n at the start of the
 * step (rho, u = (sum f e + G_body/2)/rho, p = (rho - 1)/3):
 *  - Eqs. hydroForP / hydroForNu on each element: (-p n + tau.n) l, with n the
 *    outward normal, p and grad u fitted by MLS (linear basis, Roma weights,
 *    3x3 nearest nodes in the fluid) at the probe c + 1.2 n, tau =
 *    nu (grad u + grad u^T), nu = (tau_LB - 1/2)/3; half to each end vertex;
 *  - the total vertex force is the membrane force plus this hydrodynamic force;
 *  - the fluid receives, instead of the membrane forces, the forcing term
 *    2 dV (u_p - U~) per vertex (direct forcing: u_p the particle velocity at
 *    the vertex, U~ the interpolated flow, dV half the two adjacent element
 *    lengths), spread with the IB shape functions.
 * After the collision the deformable particle moves each vertex by the
 * interpolated velocity plus F / (2 m_v) (m_v = rho_P A_0 / n) and takes the
 * second-order backward-difference velocity; the rigid one advances its
 * velocity and spin by the printed second-order update of F/m and M/I (m =
 * rho_P A_0, I = rho_P J_0 about the area centroid), translates and turns about
 * its area centroid.  Particles start at rest.  A rigid dynamic membrane has
 * at most 256 vertices.  The tangent, the adjoint and the slab decomposition refuse
 * contexts that hold one. */

/* Particle density over fluid density rho_P / rho of a dynamic membrane
 * (default 1.1, Sec. 3).  Must precede the first lbib_step.
 * Errors: LBIB_E_INVALID (not a dynamic membrane, rho_ratio <= 0 or not
 * finite), LBIB_E_STATE (after the first step). */
lbib_status lbib_set_particle_density(lbib_ctx* ctx, int32_t membrane_id, double rho_ratio);

/* Particle velocity u_p^n of each vertex of one dynamic membrane (2 doubles
 * per vertex, host memory): the backward-difference velocity of a deformable
 * particle, u + omega x r of a rigid one; zero before the first step.
 * Errors: LBIB_E_INVALID (not a dynamic membrane), LBIB_E_STATE (not finalised). */
lbib_status lbib_read_particle_velocity(lbib_ctx* ctx, int32_t membrane_id, double* uv);

/* Receptors: xy holds 2n doubles (fixed positions, typically one per wall
 * node at y = -1/2 or NY - 1/2).  Replaces any earlier set; all bonds are
 * cleared.  Must precede the first lbib_step.  Errors: LBIB_E_INVALID, LBIB_E_STATE. */
lbib_status lbib_set_receptors(lbib_ctx* ctx, const double* xy, int32_t n,
                               const lbib_bond_params* params);

/* Walls moving along x (the planar Couette flow of the cell-free-layer
 * adhesion study, Sec. 4): u_bottom, u_top are the x velocities of the walls
 * at y = -1/2 and y = NY - 1/2 (default 0).  A population bounced back at a
 * moving wall gains 2 w_i rho_w (e_i . u_w) / c_s^2 with rho_w = 1 (the
 * moving-wall bounce-back of Ladd 1994); with tau = 1 the linear profile
 * u(y) = u_bottom + (u_top - u_bottom)(y + 1/2)/NY is the discrete steady state.
 * Must precede the first lbib_step; it re-initialises the populations to the
 * context's initial state (with LBIB_INIT_COUETTE, the Couette flow of these
 * velocities) and, for FP16 storage, chooses the storage scale again.  The
 * tangent and the adjoint need resting walls.
 * Errors: LBIB_E_INVALID (no bounce-back walls, non-finite), LBIB_E_STATE
 * (after the first step). */
lbib_status lbib_set_wall_velocity(lbib_ctx* ctx, double u_bottom, double u_top);

/* Cut-off distance of the inter-membrane repulsion, Eq. repFor (default 2). */
lbib_status lbib_set_repulsion(lbib_ctx* ctx, double d_rep);

/* Advance n time steps (enqueued; replays captured CUDA graphs).  Errors from
 * launching are returned; device-side failures are reported by lbib_sync or
 * the next read. */
lbib_status lbib_step(lbib_ctx* ctx, int64_t n);

/* Wait for the context's stream and report device-side status. */
lbib_status lbib_sync(lbib_ctx* ctx);

/* Steps taken so far. */
int64_t lbib_step_count(const lbib_ctx* ctx);

/* rho^n, u^n of the last completed step (Sec. 2.1 moments with the Guo
 * half-force, Sec. 2.2), each NY*NX doubles, row-major (y, x).  Any pointer may
 * be NULL.  LBIB_E_STATE before the first step or after write_populations. */
lbib_status lbib_read_fields(lbib_ctx* ctx, double* rho, double* ux, double* uy, int on_device);

/* Pre-collision populations f^n at the current step, 9*NY*NX doubles laid out
 * [i][y][x] with the velocity order of Eq. GaussHermite. */
lbib_status lbib_read_populations(lbib_ctx* ctx, double* f, int on_device);

/* Replace the populations by f (same layout as lbib_read_populations). */
lbib_status lbib_write_populations(lbib_ctx* ctx, const double* f, int on_device);

/* Marker positions X^n (2 doubles per vertex, unwrapped x) of one membrane, or
 * of all membranes concatenated in creation order when membrane_id = -1. */
lbib_status lbib_read_markers(lbib_ctx* ctx, int32_t membrane_id, double* xy);

/* Overwrite X^n and X^{n-1} of all membranes (2*nv doubles each, host memory);
 * xy_prev may be NULL (then X^{n-1} = X^n).  The particle velocities and rigid
 * states of dynamic membranes are left as they are. */
lbib_status lbib_write_markers(lbib_ctx* ctx, const double* xy, const double* xy_prev);

/* Total Lagrangian force F^n and interpolated velocity U^n used by the last
 * step, 2 doubles per vertex (all membranes, host memory). */
lbib_status lbib_read_marker_forces(lbib_ctx* ctx, double* fxy);
lbib_status lbib_read_marker_velocity(lbib_ctx* ctx, double* uxy);

/* Current bonds as (ligand, receptor) pairs, ascending ligand id; at most cap
 * pairs are written, *n_out receives the number of bonds. */
lbib_status lbib_read_bonds(lbib_ctx* ctx, int32_t* ligand_ids, int32_t* receptor_ids,
                            int32_t cap, int32_t* n_out);

/* FP64 invariants: total mass sum_x sum_i f_i (Sec. 2.1) and, if areas is not
 * NULL, the enclosed area of each membrane (Eq. areaFor's Green area). */
lbib_status lbib_diagnostics(lbib_ctx* ctx, double* mass, double* areas);

/* ---------------------------------------------------------------- ensembles
 * A batch of independent simulations (e.g. a sweep over release positions,
 * capillary numbers and bond strengths on channels of different lengths)
 * advanced together, one CUDA graph launch per chunk of 16 steps.  The paper
 * runs its cases one by one; this is a throughput form only: every member
 * computes exactly what it computes alone with the same tiling (bitwise).
 * Two forms, chosen at creation:
 *  - batched (lbib_ensemble_form = 1): when all members share the precision,
 *    the walls and the form and shape of the fused kernel (lbib_set_tiling:
 *    the same row tiles (vec, ty), or the persistent form (npt, 0) with the
 *    same npt), and all have membranes but no dynamic particles, each time
 *    step is three launches for all members together: the force kernel over
 *    every member's force units, the fused kernel over every member's tiles
 *    (row tiles) or row segments (persistent form) and the advance kernel
 *    over every member's advance units (work lists over (member, unit) with
 *    per-member arguments in the launch parameters or in device memory);
 *  - graph of member graphs (form 0), for any other set of members: each
 *    member's captured time step is an independent child graph.
 *
 *   In the batched form the members are split into groups of at most 64
 *   (contiguous, about equal nodes); each group's launches form an
 *   independent branch of the chunk graph, so groups overlap on the GPU.
 *
 * lbib_ensemble_form: 1 batched, 0 graph of member graphs, -1 for NULL.
 * lbib_ensemble_set_groups: regroup a batched ensemble into `groups` groups
 *   (ceil(n / 64) <= groups <= n; ceil(n / 64) at creation) and recapture its
 *   graphs; waits for the ensemble's stream.  LBIB_E_STATE if not batched,
 *   LBIB_E_INVALID out of range.  Results do not depend on the grouping.
 * lbib_ensemble_groups: the groups in use (0 if not batched, -1 for NULL).
 * lbib_ensemble_profile_kernels: time the batched kernels alone, `reps`
 *   back-to-back launches of each kind over all groups, and return the mean
 *   ms per launch (a time step of the whole ensemble) of the force kernel,
 *   the fused kernel and the advance kernel in ms_per_launch[0..2] (CUDA
 *   events on the ensemble's stream).  The launches do not form time steps,
 *   so the members are left poisoned: profile a scratch ensemble.
 *   LBIB_E_STATE if not batched.
 * lbib_ensemble_launches_per_step: kernel launches per time step of the
 *   whole ensemble (3 per group in the batched form, the members' sum
 *   otherwise).
 *
 * lbib_ensemble_create: members are n distinct contexts on the current device
 *   (their set-up calls done; they are finalised here).  The ensemble takes
 *   ownership: lbib_ensemble_destroy destroys them; do not destroy them
 *   yourself.  cuda_stream may be NULL (the ensemble creates its own).
 *   Errors: LBIB_E_INVALID (NULL, duplicates, other device, poisoned member),
 *   or a member's finalisation error.
 * lbib_ensemble_step: enqueue n steps of every member on the ensemble's
 *   stream (asynchronous).  Do not step the members individually afterwards.
 * lbib_ensemble_sync: wait for the ensemble's stream and check every member's
 *   device status; call it before reading a member (lbib_ensemble_member
 *   returns the member's context for the lbib_read_* calls).
 * lbib_ensemble_write_state: every member's state in one call.  f[i]: member
 *   i's pre-collision populations (9*NY*NX doubles, the layout of
 *   lbib_write_populations), xy[i] / xy_prev[i]: its marker positions X^n
 *   and X^{n-1} (as lbib_write_markers; xy_prev NULL or xy_prev[i] NULL means
 *   X^{n-1} = X^n).  Any of f, xy, or an entry of them may be NULL (that part
 *   is left as it is).  Host buffers (on_device = 0; pinned memory lets the
 *   copies run at full speed) or device buffers (populations only;
 *   on_device = 1).  All copies and conversions go on the ensemble's
 *   stream, after its pending steps, and the call waits once for them: the
 *   buffers may be reused on return.  Errors: LBIB_E_INVALID, LBIB_E_STATE
 *   (a poisoned member), LBIB_E_OOM, LBIB_E_CUDA.
 * lbib_ensemble_read_markers: every member's marker positions (xy[i]: 2 nv_i
 *   doubles, host; NULL entries are skipped) after the pending steps, with
 *   one wait.  Errors: LBIB_E_INVALID, LBIB_E_CUDA.
 */
typedef struct lbib_ensemble lbib_ensemble;
lbib_status lbib_ensemble_create(lbib_ctx* const* members, int32_t n, void* cuda_stream, lbib_ensemble** out);
lbib_status lbib_ensemble_step(lbib_ensemble* ens, int64_t n);
lbib_status lbib_ensemble_sync(lbib_ensemble* ens);
int32_t lbib_ensemble_size(const lbib_ensemble* ens);
int32_t lbib_ensemble_form(const lbib_ensemble* ens);
lbib_status lbib_ensemble_set_groups(lbib_ensemble* ens, int32_t groups);
int32_t lbib_ensemble_groups(const lbib_ensemble* ens);
lbib_status lbib_ensemble_profile_kernels(lbib_ensemble* ens, int32_t reps, double* ms_per_launch);
int32_t lbib_ensemble_launches_per_step(const lbib_ensemble* ens);
lbib_status lbib_ensemble_write_state(lbib_ensemble* ens, const double* const* f, const double* const* xy,
                                      const double* const* xy_prev, int32_t on_device);
lbib_status lbib_ensemble_read_markers(lbib_ensemble* ens, double* const* xy);
lbib_ctx* lbib_ensemble_member(lbib_ensemble* ens, int32_t i);
const char* lbib_ensemble_last_error(const lbib_ensemble* ens);
void lbib_ensemble_destroy(lbib_ensemble* ens);

/* ---------------------------------------------------------------- tangent
 * Forward-mode (tangent-linear) derivative of an FP64 trajectory.  Along one
 * direction of the parameters -- dk_s and dk_b per membrane, dsigma (the bond
 * stiffness sigma of Eq. adhFor in lattice units) and the derivative of the
 * current marker positions (e.g. a release height) -- the derivative of the
 * marker positions is carried through every step with the step itself:
 * forces (Eqs. strainFor, bendFor, areaFor, repFor, adhFor), MLS/Roma shape
 * functions and spreading, the Guo-forced BGK collide-stream, interpolation
 * and BDF2.  Bond formation and rupture are events: the bonds of every step are
 * the primal run's, held fixed (the derivative of the path with that bond
 * history).  The paper has no derivative; this serves sensitivity studies
 * (adhesion and margination against k_s, k_b, sigma, release position).
 *
 * lbib_tangent_create: ctx must be LBIB_F64 without rigid-projected
 *   membranes (LBIB_E_INVALID otherwise); the tangent borrows the context
 *   (destroy the tangent first).  Allocates its own device buffers.
 * lbib_tangent_seed: set the direction: dks, dkb (nmem doubles each, host, or
 *   NULL = 0), dsigma, dxy / dxy_prev (2*nv doubles, host, the derivatives of
 *   X^n and X^{n-1}; NULL = 0, dxy_prev NULL = dxy); clears the derivative of
 *   the populations.
 * lbib_tangent_step: advance the context n steps together with the tangent
 *   (instead of lbib_step).
 * lbib_tangent_read: derivative of X^n (and X^{n-1}) into host arrays of
 *   2*nv doubles (either may be NULL); synchronises.
 */
typedef struct lbib_tangent lbib_tangent;
lbib_status lbib_tangent_create(lbib_ctx* ctx, lbib_tangent** out);
lbib_status lbib_tangent_seed(lbib_tangent* t, const double* dks, const double* dkb, double dsigma,
                              const double* dxy, const double* dxy_prev);
lbib_status lbib_tangent_step(lbib_tangent* t, int64_t n);
lbib_status lbib_tangent_read(lbib_tangent* t, double* dxy, double* dxy_prev);
void lbib_tangent_destroy(lbib_tangent* t);

/* ---------------------------------------------------------------- adjoint
 * Reverse-mode derivative of an FP64 trajectory: the transpose of the tangent
 * above, with the same bond history held fixed.  For a scalar J of the final
 * state (X^N, X^{N-1}, f^N) it returns, in one backward sweep, dJ/dk_s and
 * dJ/dk_b of every membrane, dJ/dsigma and dJ/d(X^0, X^{-1}, f^0) -- the
 * gradient with respect to all parameters at the cost of about one tangent
 * direction.  The paper has no derivative; this serves the same sensitivity
 * studies as the tangent when there are many parameters.
 *
 * Memory: the full step state (populations, X^n, X^{n-1}, bonds, receptor
 * occupancy, step counter) every `checkpoint_every` steps, plus a tape of one
 * segment (checkpoint_every copies of the populations, positions and bonds).
 * The backward sweep re-runs each segment from its checkpoint with the
 * context's own step (bit-identical to the recorded run) and then applies the
 * adjoint step to the tape in reverse order.
 *
 * Precision: the recorded run is the context's own, in any precision (e.g.
 * an FP32 forward run); the tape holds FP64 copies of its states, and the
 * adjoint arithmetic and every gradient are FP64.  The result is then the
 * derivative of the exact-arithmetic step along that trajectory.
 *
 * lbib_adjoint_create: ctx without rigid-projected membranes and with at
 *   least 5 vertices per membrane (LBIB_E_INVALID otherwise);
 *   checkpoint_every >= 1; LBIB_E_OOM if the tape does not fit.  The adjoint
 *   borrows the context (destroy the adjoint first).
 * lbib_adjoint_record: advance the context n >= 1 steps (instead of
 *   lbib_step) from its current state, keeping the checkpoints; replaces an
 *   earlier recording; synchronises and returns the step status.
 * lbib_adjoint_seed: dJ/dX^N and dJ/dX^{N-1} (2*nv doubles each, host, NULL =
 *   0) and dJ/df^N (9*NY*NX doubles, host, layout of lbib_read_populations,
 *   NULL = 0) at the end of the recording; clears the parameter gradients.
 *   LBIB_E_STATE before a recording.
 * lbib_adjoint_reverse: the backward sweep over the recorded steps; the
 *   context is left in the state the recording ended in.  LBIB_E_STATE unless
 *   seeded since the last sweep.  Synchronises.
 * lbib_adjoint_read: dJ/dX^0, dJ/dX^{-1} (2*nv doubles), dJ/dk_s, dJ/dk_b
 *   (nmem doubles), dJ/dsigma (1 double), dJ/df^0 (9*NY*NX doubles, layout of
 *   lbib_read_populations) into host arrays; any pointer may be NULL.  Here 0
 *   is the first recorded step.  Synchronises.
 * lbib_adjoint_recorded_steps: N of the last recording (0 before, -1 for NULL).
 */
typedef struct lbib_adjoint lbib_adjoint;
lbib_status lbib_adjoint_create(lbib_ctx* ctx, int32_t checkpoint_every, lbib_adjoint** out);
lbib_status lbib_adjoint_record(lbib_adjoint* adj, int64_t n);
lbib_status lbib_adjoint_seed(lbib_adjoint* adj, const double* xy_bar, const double* xy_prev_bar,
                              const double* f_bar);
lbib_status lbib_adjoint_reverse(lbib_adjoint* adj);
lbib_status lbib_adjoint_read(lbib_adjoint* adj, double* xy_bar, double* xy_prev_bar, double* ks_bar,
                              double* kb_bar, double* sigma_bar, double* f_bar);
int64_t lbib_adjoint_recorded_steps(const lbib_adjoint* adj);
void lbib_adjoint_destroy(lbib_adjoint* adj);

/* ---------------------------------------------------------------- x-slabs
 * One lattice decomposed into x-slabs (the domain decomposition a multi-GPU
 * run of a single lattice would use; here the slabs share one GPU).  Slab k
 * is an ordinary context of width W_k + 2 on the same rows: its columns 1 ..
 * W_k are the lattice's columns X_k .. X_k + W_k - 1 (X_0 = 0, X_{k+1} = X_k +
 * W_k), and columns 0 and W_k + 1 are ghost columns.  After each step the
 * ghost columns receive from the neighbouring slabs (a ring: x stays
 * periodic) the post-collision populations that stream into the slab, so that
 * every interior column evolves exactly as in the undivided lattice.  Ghost
 * columns hold no meaningful populations of their own: read-backs and
 * diagnostics of a slab include them, so use the interior columns only.
 *
 * lbib_slabs_create: 2 .. 16 contexts in order of x, with the same NY,
 *   precision, walls, wall velocities, tau, body force and CUDA stream, no
 *   membranes, all at the same step; the slabs object borrows them (destroy it
 *   first).  Initialise each slab's populations with those of the lattice's
 *   columns X_k - 1 .. X_k + W_k (periodic) before creating the object, or use
 *   an x-uniform initial state.  Exchanges the ghost columns once.  (FP16
 *   storage: each context picks its storage scale at creation from the body
 *   force, whose y component counts the width; the slabs match the undivided
 *   lattice bit for bit when their scale equals its scale, e.g. with a body
 *   force along x.)
 * lbib_slabs_step: n times, one step of every slab and the exchange (enqueued).
 * lbib_slabs_sync: synchronise and report the slabs' device-side status.
 * Errors: LBIB_E_INVALID (sizes, mismatched slabs, membranes), LBIB_E_STATE
 * (slabs at different steps, a poisoned slab), LBIB_E_CUDA. */
typedef struct lbib_slabs lbib_slabs;

/* Slabs in different processes (one slab per rank, e.g. one per GPU).  The
 * same decomposition with the exchange done by the caller: after every step
 * of its slab, a rank sends the faces that leave it and writes the faces that
 * enter it, then steps again.
 * lbib_slab_face: out = 1 copies the face that leaves `ctx` on `side` from its
 *   current post-collision buffer: side 0 (left) the first interior column's
 *   populations 3, 6, 7 (they stream to the left neighbour's ghost column
 *   W + 1), side 1 (right) the last interior column's populations 1, 5, 8
 *   (to the right neighbour's ghost column 0).  out = 0 writes the face that
 *   enters on `side`: side 0 the ghost column 0's populations 1, 5, 8 (from
 *   the left neighbour's right face), side 1 the ghost column W + 1's
 *   populations 3, 6, 7 (from the right neighbour's left face).  buf holds
 *   3 x NY stored elements ([3][NY], the context's storage type, see
 *   lbib_storage_bytes): host memory (on_device = 0; the call synchronises
 *   the stream) or device memory (on_device = 1; enqueued).  Lattice-only
 *   contexts.  Errors: LBIB_E_INVALID, LBIB_E_CUDA.
 * lbib_storage_bytes: bytes per stored population (8, 4 or 2). */
lbib_status lbib_slab_face(lbib_ctx* ctx, int32_t side, int32_t out, void* buf, int32_t on_device);
int32_t lbib_storage_bytes(const lbib_ctx* ctx);
lbib_status lbib_slabs_create(lbib_ctx* const* slabs, int32_t n, lbib_slabs** out);
lbib_status lbib_slabs_step(lbib_slabs* group, int64_t n);
lbib_status lbib_slabs_sync(lbib_slabs* group);
const char* lbib_slabs_last_error(const lbib_slabs* group);
void lbib_slabs_destroy(lbib_slabs* group);

/* Save and restore the full step state of a context (checkpoint / resume).
 * lbib_save writes to the file at `path`:
 *  - a header identifying the set-up;
 *  - the populations in the context's storage format;
 *  - X^n and X^{n-1};
 *  - the bonds and the receptor occupancy;
 *  - the repulsion boxes;
 *  - the step counter.
 * The file is in host byte order.
 * lbib_load restores such a file into a context built with the same set-up
 * (same lattice, precision, walls and wall velocities, body force, tau,
 * membranes, ligands, receptors and repulsion range; LBIB_E_INVALID
 * otherwise, with the context untouched).  It resets the per-step scratch.
 * It also clears a poisoned context: after LBIB_E_NONFINITE or
 * LBIB_E_TIMEOUT, loading a saved state lets lbib_step run again.  Stepping
 * on from a loaded state reproduces the original run bit for bit.  Both
 * synchronise the context's stream.
 * Errors: LBIB_E_INVALID (NULL, unreadable or unwritable file, not a saved
 * state, truncated, other set-up), LBIB_E_STATE (lbib_save on a poisoned
 * context), LBIB_E_CUDA. */
lbib_status lbib_save(lbib_ctx* ctx, const char* path);
lbib_status lbib_load(lbib_ctx* ctx, const char* path);

/* Observables of the margination and adhesion studies (Sec. 4) for every
 * membrane, reduced on the device in FP64 over the current markers.  out
 * receives 8 doubles per membrane (host memory, nmem * 8):
 *   [0], [1]  centroid (x, y) of the vertices (x unwrapped)
 *   [2], [3]  centroid velocity, mean of X^n - X^{n-1} (lattice units per
 *             step): [2] is the rolling / translation velocity u_roll of an
 *             adhering carrier, [3] the lateral velocity
 *   [4]       region of the centroid height h = (y + 1/2)/NY above the lower
 *             wall: 0 bulk (0.3 <= h <= 0.7), 1 intermediate (0.2 <= h < 0.3
 *             or 0.7 < h <= 0.8), 2 cell-free layer (h < 0.2 or h > 0.8)
 *   [5]       bonds held by the membrane's ligands (n_L)
 *   [6], [7]  lowest and highest vertex height above the lower wall (y + 1/2)
 * Synchronises.  Allocates a small device buffer on the first call. */
lbib_status lbib_membrane_observables(lbib_ctx* ctx, double* out);

/* Allocation-free FP64 mass of a population buffer the caller owns.  The
 * paper has no counterpart: this is a library service for callers that must not
 * allocate device memory at the time of the call, e.g. a monitor running between
 * steps on a thread where cudaMalloc/cudaFree would synchronise the device, or a
 * program whose memory pool has already reserved the device memory.
 *
 *  f       device pointer (current device) to 9*n_nodes doubles, any order of
 *          the values (e.g. the layout of lbib_read_populations); 8-byte aligned
 *  n_nodes 0 .. 7,456,540 (9*n_nodes <= 2^26); 0 gives mass 0
 *  mass    device pointer (current device) that receives sum_k f[k]
 *  stream  cudaStream_t to enqueue on (NULL: the legacy default stream)
 *
 * The sum runs in a fixed order (run-to-run deterministic).  It enqueues two
 * kernels and returns without synchronising.  Scratch: one fixed 32 KiB array
 * per device inside the library; its address is looked up on the first call
 * on each device (with that device current), so make that first call before
 * any stream capture.  Calls on one device that overlap in time (other streams
 * or host threads) race on the scratch: serialise them.
 * Errors: LBIB_E_INVALID for NULL or misaligned pointers, a pointer that is
 * not device memory of the current device, or n_nodes out of range (nothing is
 * launched); LBIB_E_CUDA if the scratch lookup or a launch fails.  No message
 * is kept (there is no context). */
lbib_status lbib_population_mass_noalloc(const double* f, int64_t n_nodes, double* mass, void* stream);

/* Form and tile shape of the fused collide-stream kernel.  Must precede the
 * first step; 0,0 picks the default: for F32 and 16-bit storage the
 * persistent form when the two population buffers exceed 128 MB, for 16-bit
 * storage also from 2^20 nodes on (segments of 512 nodes), else a row-tile
 * shape.
 *  ty in 1..16: row tiles, vec consecutive x nodes per thread and ty rows per
 *    block; vec divides NX, with vec in {1,2} (F64), {1,2,4} (F32), {2,4,8}
 *    (16-bit storage).
 *  ty = 0: persistent bulk-copy form, one or more CTAs per SM streaming row
 *    segments of 256*vec nodes through a 4-stage shared-memory pipeline;
 *    vec in {1,2} (F64), {1,2,4} (F32), {2,4,8} (16-bit); NX a multiple of
 *    16 bytes of storage (2, 4 or 8 nodes).
 * Errors: LBIB_E_INVALID for other shapes, LBIB_E_STATE after the first step.
 * The forms give bitwise identical results. */
lbib_status lbib_set_tiling(lbib_ctx* ctx, int32_t vec, int32_t ty);
lbib_status lbib_get_tiling(const lbib_ctx* ctx, int32_t* vec, int32_t* ty);

/* Profiling aid: launch only the fused collide-stream kernel `reps` times on
 * the context's stream (ping-pong between the two population buffers, with the
 * IB force of the last completed step frozen), bracketed by CUDA events, and
 * return the mean duration of one launch in milliseconds.  This advances the
 * populations without the Lagrangian part, so use it on a scratch context.
 * Errors: LBIB_E_STATE before the first step. */
lbib_status lbib_profile_fused(lbib_ctx* ctx, int32_t reps, double* ms_per_launch);

/* Profiling aid: launch each kernel of the time step `reps` times back to
 * back on the context's stream, each series bracketed by CUDA events, and
 * return the mean duration of one launch in ms_per_launch[0..2]:
 * [0] forces + IB weights + spreading, [1] fused collide-stream, [2]
 * interpolation + advance + bond kinetics (0 for the marker kernels of a
 * context without membranes).  The repeated launches leave the state
 * inconsistent (forces accumulate, markers and bonds move without the
 * fluid): use it on a scratch context.  Errors: LBIB_E_STATE before the
 * first step. */
lbib_status lbib_profile_kernels(lbib_ctx* ctx, int32_t reps, double* ms_per_launch);

/* Profiling aid: the hydrodynamic-stress kernel of the dynamic particles
 * launched `reps` times back to back on the context's stream (it only reads
 * the state and rewrites its own outputs); mean duration of one launch in
 * *ms_per_launch, 0 for a context without dynamic membranes.
 * Errors: LBIB_E_STATE before the first step. */
lbib_status lbib_profile_hydro(lbib_ctx* ctx, int32_t reps, double* ms_per_launch);

/* Number of kernels one time step launches (for launch accounting). */
int32_t lbib_kernels_per_step(const lbib_ctx* ctx);

/* Scale exponent k of the 16-bit storage (d_i * 2^k); 0 for F32/F64. */
int32_t lbib_storage_scale_exponent(const lbib_ctx* ctx);

const char* lbib_last_error(const lbib_ctx* ctx);
void lbib_destroy(lbib_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBIB_H */
