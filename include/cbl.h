/*
 * cbl.h -- C ABI of the GB300 (sm_103a) capillary-bridge library: one time step of the combined
 * multi-phase-field / lattice-Boltzmann method of Schiedung, Tegeler, Medvedev and Varnik,
 * "Simulation of Capillary-Driven Kinetics with Multi-Phase-Field and Lattice-Boltzmann Method"
 * (arXiv:1902.10432).
 *
 * The calls follow the paper's statement of the problem: set up the lattice and the solid bodies
 * given as phase fields (Sec. 3.1), initialise the fluid (Sec. 3.2), advance N time steps
 * (Sec. 3.2.1-3.3), read the fluid fields, read the per-body force and torque
 * (Sec. 3.2.2 Eq. solid_liquid_force, Sec. 3.2.3), read or move the bodies (Sec. 3.1.1).
 *
 * Conventions shared by every call:
 *  - Every call returns a cbl_status; nothing is thrown across the boundary. On failure
 *    cbl_last_error() describes the cause.
 *  - Lattice cells are indexed n = x + nx * (y + ny * z), periodic in all three axes; arrays of
 *    vectors are [cell][3].
 *  - Device memory is obtained only through the caller's cbl_allocator (NULL = cudaMalloc) and is
 *    released by cbl_destroy. Output buffers are owned by the caller.
 *  - Work is enqueued on the stream given in cbl_params; NULL makes the library create a
 *    non-blocking stream of its own (the legacy default stream cannot be captured into the CUDA
 *    graph that cbl_step replays). cbl_step returns before the work finishes; every cbl_read_* /
 *    cbl_get_* call synchronises that stream first. One context must not be used from two host
 *    threads at once.
 *  - Wrong call order (e.g. cbl_step before cbl_init_fluid) returns CBL_ERR_STATE.
 *  - Solid cells read back zero density and velocity.
 */
#ifndef CBL_H
#define CBL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cbl_ctx cbl_ctx; /* opaque, library-owned */

typedef enum {
  CBL_OK = 0,
  CBL_ERR_ARG = 1,         /* invalid argument (size, pointer, parameter out of range) */
  CBL_ERR_STATE = 2,       /* wrong call order, or a device-side consistency check failed */
  CBL_ERR_OOM = 3,         /* the allocator returned NULL */
  CBL_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  CBL_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
  CBL_ERR_UNSTABLE = 6,    /* NaN / Inf in the fluid mass, or a body update that was not finite */
  CBL_ERR_UNSUPPORTED = 7  /* feature not built (e.g. the fused pass for a precision other than FP32) */
} cbl_status;

/* Storage precision of the lattice-Boltzmann populations. Arithmetic is FP64 for CBL_FP64 and FP32
 * otherwise; the FP32 collision uses FP32 weights whose sum is exactly 1 (each within 2 ulp of w_i),
 * so that its equilibria add no mass (Sec. 3.2.1). CBL_FP16DEV stores h_i = f_i - w_i in binary16
 * (w_i rounded to binary16), halving the population bytes. Phase fields, body reductions and the
 * rigid-body integrator are FP64 in every mode. */
typedef enum { CBL_FP64 = 0, CBL_FP32 = 1, CBL_FP16DEV = 2 } cbl_prec;

typedef struct {
  void* (*alloc)(size_t bytes, void* user); /* device memory, >= 256-byte aligned, NULL on failure */
  void (*free)(void* ptr, void* user);
  void* user;
} cbl_allocator;

typedef struct {
  int nx, ny, nz;          /* lattice size, each >= 4 */
  int q;                   /* velocity set: 19 (D3Q19) or 27 (D3Q27, the set of Sec. 3.2.1) */
  double tau;              /* BGK relaxation time (Eq. lb_collision), > 0.5 */
  double G;                /* Shan-Chen coupling (Eq. benzi_force), paper: -5 */
  double rho0;             /* reference density of psi (Eq. mean_field_potential), paper: 1 */
  double ext_force[3];     /* uniform external force density on fluid cells (0 in the paper) */
  cbl_prec prec;
  int mpf_kinetics;        /* 1: Eq. sim_proc_phase_field_dynamics after advection (Sec. 3.3) */
  double mobility;         /* M_alpha_beta, paper: 1e-5 */
  double eta;              /* interface width, paper: 5 */
  double sigma_sf;         /* solid-fluid interface energy (not given in the paper) */
  double sigma_ss;         /* solid-solid interface energy (not given in the paper) */
  double e0;               /* repulsion strength (Eq. soild_solid_potential; not given) */
  double rc;               /* repulsion range, paper: 3 */
  int nrep;                /* repulsion exponent n, paper: 4 */
  double solid_threshold;  /* a cell is solid iff its fluid phase < this; paper: 0.05 */
  double member_threshold; /* a cell is a repulsion point of body B iff phi_B >= this */
  void* stream;            /* cudaStream_t (not the legacy default stream), or NULL */
} cbl_params;

/* Solid body. The shape gives the phi = 1/2 surface; the phase field is the profile
 * 1/2 - 1/2 sin(pi d / eta) of the signed distance d across |d| < eta/2 (Sec. 3.1). */
typedef struct {
  int shape;             /* 0 sphere, 1 box */
  double center[3];      /* lattice coordinates; cell centres sit on integers */
  double radius;         /* sphere */
  double half[3];        /* box half extents in the body frame */
  double quat[4];        /* initial orientation (w, x, y, z); zero = identity */
  double mass_density;   /* rho_alpha: M = rho_alpha * sum phi */
  double wetting_rho;    /* varrho_B: solid cells act as fluid of this density (Sec. 3.2.3) */
  int fixed;             /* 1: the body is held in place (forces are still reported); see cbl_set_bodies_fixed */
} cbl_body;

/* Create a context. Validates the parameters (CBL_ERR_ARG) and allocates the lattice arrays through
 * `alloc` (NULL = cudaMalloc; CBL_ERR_OOM if it fails). `out` receives the context, owned by the
 * caller until cbl_destroy. */
cbl_status cbl_create(const cbl_params* params, const cbl_allocator* alloc, cbl_ctx** out);

/* Add a solid body (before cbl_init_fluid). Its phase-field tile is allocated here. CBL_ERR_ARG for
 * a non-finite or out-of-range field (centre beyond 1e6, radius or half extents <= 0, mass density
 * <= 0, wetting density < 0). `body_id`
 * (may be NULL) receives the 0-based id. A body whose support (surface + eta/2) covers the whole
 * periodic length along an axis is infinite along it (the plates of the planar bridge, Sec. 2.1):
 * it turns only about that axis; the other angular-velocity components are held at zero. */
cbl_status cbl_add_body(cbl_ctx* ctx, const cbl_body* body, int* body_id);

/* Initialise the phase fields, obstacle flags (Sec. 3.2.2: solid iff fluid phase < threshold),
 * body mass, centre of mass and inertia, and the fluid: f = f_eq(rho, 0) with rho = rho_liquid
 * where liquid_mask_host[n] != 0 and rho_vapour elsewhere (mask may be NULL: all vapour).
 * The mask is a host array of nx*ny*nz bytes; it is copied to the device and expanded there. */
cbl_status cbl_init_fluid(cbl_ctx* ctx, double rho_liquid, double rho_vapour,
                          const unsigned char* liquid_mask_host);

/* Same, from per-cell density and velocity (host arrays of N and 3N doubles; u may be NULL).
 * CBL_ERR_ARG if a density is negative or not finite, or a velocity is not finite. */
cbl_status cbl_init_fluid_fields(cbl_ctx* ctx, const double* rho_host, const double* u_host);

/* Advance nsteps time steps (asynchronous on the context's stream). One step: pull streaming with
 * half-way moving-wall bounce-back and local mass correction (Sec. 3.2.2), moments and psi,
 * Shan-Chen force with wetting (Sec. 3.2.3), Guo-forced BGK collision (Sec. 3.2.1), per-body
 * momentum-exchange and adhesion force/torque in FP64, solid-solid repulsion (Sec. 3.1.2),
 * rigid-body update (Sec. 3.1.1), phase-field advection and kinetics (Sec. 3.1.1, 3.3), obstacle
 * flags with cover refill / uncover (Sec. 3.2.2). The density and velocity of the last step of
 * each call are kept for cbl_read_fields. */
cbl_status cbl_step(cbl_ctx* ctx, int nsteps);

/* Fields of the last completed step: rho (N), vel (3N, [cell][3]) as computed in that step's
 * collision, and the fluid phase 1 - sum_B phi_B (N). Any pointer may be NULL. on_device != 0:
 * the pointers are device pointers; otherwise host pointers. */
cbl_status cbl_read_fields(cbl_ctx* ctx, double* rho, double* vel, double* phi_fluid, int on_device);

/* Obstacle flags: solid (N bytes, 0/1) and owner body id (N int32, -1 on fluid). Host pointers. */
cbl_status cbl_read_flags(cbl_ctx* ctx, unsigned char* solid, int32_t* owner);

/* Post-collision populations of the current state as doubles, laid out [direction][cell] (q * N),
 * in this library's direction order (cbl_velocity_set): rest, +x, -x, +y, -y, +z, -z, then the edge
 * directions (+x+y), (-x-y), (+x-y), (-x+y), (+x+z), (-x-z), (+x-z), (-x+z), (+y+z), (-y-z), (+y-z),
 * (-y+z), and for D3Q27 the corners (+++), (---), (++-), (--+), (+-+), (-+-), (-++), (+--).
 * on_device != 0: `out` is a device pointer; otherwise a host pointer. */
cbl_status cbl_read_populations(cbl_ctx* ctx, double* out, int on_device);

/* The context's velocity set (Sec. 3.2.1): q (19 or 27), the directions c (host array q*3 ints,
 * may be NULL) and the weights w (host array q doubles, may be NULL), in the order of
 * cbl_read_populations. */
cbl_status cbl_velocity_set(cbl_ctx* ctx, int* q, int* c, double* w);

/* Dense phase field of one body (N doubles, host). */
cbl_status cbl_read_phi(cbl_ctx* ctx, int body, double* phi_host);

/* Per-body total force F (nb*3) and torque T (nb*3) of the last completed step, FP64, and, if parts
 * is not NULL, the parts (nb*18): momentum exchange F,T | Shan-Chen adhesion F,T | repulsion F,T.
 * Host pointers; any may be NULL. */
cbl_status cbl_read_body_forces(cbl_ctx* ctx, double* F, double* T, double* parts);

/* Mean per-body total force F (nb*3) and torque T (nb*3) over the steps since the last reset (FP64
 * running sums kept on the device by the rigid-body update, so a mean over many steps needs no host
 * read per step); *nsteps (may be NULL) receives that number of steps. reset != 0 starts the sums
 * anew after reading. Host pointers; F, T may be NULL. cbl_load and cbl_init_fluid start them at 0. */
cbl_status cbl_read_force_mean(cbl_ctx* ctx, double* F, double* T, long long* nsteps, int reset);

/* Body state (host arrays, nb*3 / nb*4 / nb / nb*9; any may be NULL): centre of mass, velocity,
 * angular velocity, orientation quaternion, mass, body-frame inertia. Returns CBL_ERR_UNSTABLE (with
 * the arrays filled) once a body update was not finite or moved a body by a lattice length or more
 * in one step: that body is then held at its last finite pose (device error bit 3). */
cbl_status cbl_get_bodies(cbl_ctx* ctx, double* X, double* V, double* W, double* Q, double* M,
                          double* I);

/* Move bodies without stepping the fluid: centres X (nb*3), orientations Q (nb*4; NULL keeps them),
 * velocities V and W (nb*3; NULL keeps them), host arrays. The phase fields are rebuilt from the
 * body shapes at the new poses (Sec. 3.1 profile), the obstacle flags recomputed, nodes that became
 * solid hand their populations to their fluid neighbours and nodes that became fluid start empty
 * (Sec. 3.2.2). A move whose surface displacement exceeds half a cell is carried out as a chain of
 * sub-moves of at most half a cell each (linear in X, normalised blend of Q along the shorter arc),
 * so every newly covered node has a fluid neighbour to receive its populations. Mass, inertia and
 * reference volumes are kept. CBL_ERR_ARG for a non-finite position or a zero quaternion. Not
 * part of the paper's method: it serves the learned-force surrogate. */
cbl_status cbl_move_bodies(cbl_ctx* ctx, const double* X, const double* Q, const double* V, const double* W);

/* Set body velocities (host arrays nb*3, either may be NULL). CBL_ERR_ARG for a non-finite value. */
cbl_status cbl_set_body_velocities(cbl_ctx* ctx, const double* V, const double* W);

/* Checkpoint (Sec. 3: the state between two steps is the populations, the phase fields, the
 * obstacle flags and the bodies). cbl_save writes every buffer that carries state from one step to
 * the next (both population buffers, flags, the last step's fields and forces, the body table, the
 * phase-field tiles, the boundary-cell list, the step counter) to the file `path`, after
 * synchronising the context's stream; CBL_ERR_STATE before cbl_init_fluid, CBL_ERR_ARG if the file
 * cannot be written. cbl_load restores such a file into a context that was created with the same
 * parameters, had the same bodies added (same shapes, so the same tiles; options that size the
 * tiles, such as "tile_tail", set the same way) and was not initialised: it takes the place of
 * cbl_init_fluid, and the restored state is the saved one bit for bit (later steps can differ from
 * the uninterrupted run only by the order of FP64 atomic sums, as two runs do). CBL_ERR_ARG for
 * a file of another version or of a different set-up, or a truncated file; CBL_ERR_STATE on an
 * initialised context. The file is native-endian and tied to this build. */
cbl_status cbl_save(cbl_ctx* ctx, const char* path);
cbl_status cbl_load(cbl_ctx* ctx, const char* path);

/* Hold or release bodies (host array of nb ints, 1 = held in place). A held body keeps its pose,
 * its V and omega are set to zero, and its forces are still reported; a released body starts from
 * rest. This is how the paper lets the liquid reach its equilibrium shape before the particles may
 * move (Sec. 4.3.2: t = 0 is the release). CBL_ERR_ARG for a NULL array, CBL_ERR_STATE before
 * cbl_init_fluid. Takes effect from the next cbl_step. */
cbl_status cbl_set_bodies_fixed(cbl_ctx* ctx, const int* fixed);

/* Fluid mass sum_x rho(x) over fluid cells in the last completed step, FP64. Returns
 * CBL_ERR_UNSTABLE if it is not finite or a body update was not finite (device error bit 3). */
cbl_status cbl_total_mass(cbl_ctx* ctx, double* mass);

/* Number of bodies, cells; device error word (0 = none; bit 0 tile overflow, bit 1 neighbour
 * list overflow, bit 2 lost refill, bit 3 a body update that was not finite, the body held). */
cbl_status cbl_info(cbl_ctx* ctx, int* nbodies, int64_t* ncells, int* device_error);

/* Phases of one step, in launch order, as reported by cbl_time_phases. */
#define CBL_NPHASES 9
/* 0 psi of the step: pull + density + psi (split pass), psi of the bodies' tiles (fused pass,
 * "lbm_variant" 1), the regions' edge cells and the tiles (accumulating pass, 2); 1 collision:
 * pull + force + collision + mass partials, bulk and next to a solid (the fused pass also computes
 * psi, the accumulating pass the next step's density); 2 solid-fluid force on the bodies (momentum
 * exchange and adhesion reaction, compensated sums into FP64 accumulators); 3 solid-solid repulsion,
 * 4 rigid-body update, 5 phase-field advection (three sweeps), 6 phase-field kinetics, 7 obstacle
 * flags, 8 cover refill, boundary-cell list and the end of the step (fluid mass, buffer flip). */

/* Run nsteps time steps launched kernel by kernel (not through the graph) with CUDA events recorded
 * on the context's stream between the phases, synchronise, and write the mean duration per step of
 * each phase in milliseconds to ms[CBL_NPHASES] (host array). The state advances by nsteps. */
cbl_status cbl_time_phases(cbl_ctx* ctx, int nsteps, double* ms);

/* Durations in milliseconds of the bulk collision kernel in the last min(n, 512, max) step-graph
 * replays of the last cbl_step call (oldest first; n = that call's steps), measured inside the
 * replayed graph by two event-record nodes on the kernel's stream that bracket its launch (option
 * "kernel_events" = 1, set before the step graph is built). ms: host array of `max` floats;
 * *count receives the number written. Synchronises the context's stream. CBL_ERR_STATE if the option
 * is off. */
cbl_status cbl_kernel_times(cbl_ctx* ctx, int max, float* ms, int* count);

/* Execution options (no effect on the results beyond rounding order):
 *   "lbm_variant"  how each step computes the density and psi that the Shan-Chen force needs
 *                  (Sec. 3.2.3: psi of the post-streaming density at every neighbour):
 *                  0 = split pass: a density kernel pulls every cell, then the collision kernel
 *                  pulls it again (default);
 *                  1 = fused pass: one kernel marches along z, producer warps compute psi of the
 *                  plane ahead into shared memory, consumer warps collide;
 *                  2 = accumulating pass: the collision kernel also sums the next step's density
 *                  from the post-collision values it stores (shared-memory exchange within regions
 *                  of 32 x acc_ty columns x acc_sz planes); the next step completes psi of the
 *                  regions' edge cells from the populations of their outside sources and of the
 *                  bodies' tiles from the populations. Each step pulls the populations once. A
 *                  batch (cbl_batch_*) runs its instances with the split pass;
 *   "fused_ty"     y extent of a fused block's consumer tile: 4 or 8 (default);
 *   "fused_tz"     z extent of a fused block (0 = derived from the SM count);
 *   "acc_ty"       y extent of an accumulating region: 8 (default) or 16;
 *   "acc_sz"       z extent of an accumulating region (0 = derived from the SM count: the fewest
 *                  planes that give two waves of resident blocks);
 *   "lbm_block_x"  x extent of the 128-thread blocks of the split kernels: 32 (default), 64, 128;
 *   "graph_branches" 1 (default) = with bodies, the collision of the fluid cells next to a solid,
 *                  the solid-fluid force pass and the solid-solid repulsion run on a second branch
 *                  of the step graph beside the bulk collision; 0 = one chain;
 *   "node_priority" 1 (default) = the step graph keeps the side branch's higher stream priority
 *                  on its kernel nodes (instantiated with cudaGraphInstantiateFlagUseNodePriority);
 *                  0 = all nodes at the same priority;
 *   "tile_tail"    cells of room (default 2.5, at most 64) between a body's phase-field support and
 *                  the halo of its tile, for the tail that the advection leaves behind a moving
 *                  body and that grows with the distance travelled; set before the first
 *                  cbl_add_body (CBL_ERR_STATE after). Results do not depend on it while no phi
 *                  above 1e-12 reaches the halo (device error bit 0 stays clear).
 *   "kernel_events" 1 = the step graph brackets the bulk collision with event-record nodes, read
 *                  back by cbl_kernel_times; 0 (default) = none.
 * Unknown keys return CBL_ERR_ARG. The captured step graph is rebuilt at the next cbl_step. */
cbl_status cbl_set_option(cbl_ctx* ctx, const char* key, double value);

/* The value in use of an execution option (keys as for cbl_set_option; "acc_sz" and "fused_tz"
 * report the derived extent when none was requested). CBL_ERR_ARG for an unknown key or a NULL
 * argument. */
cbl_status cbl_get_option(cbl_ctx* ctx, const char* key, double* value);

/* One lattice-Boltzmann time step that allocates nothing, for callers that cannot allocate device
 * memory (their memory belongs to another framework's pool, or their process must not call
 * cudaMalloc once running). The paper has no counterpart: this is plumbing, not method.
 * The step is the plain fluid part of cbl_step on a lattice without solid bodies: pull streaming,
 * psi, Shan-Chen force, Guo-forced BGK collision; FP32 populations, SoA [direction][cell] with a
 * stride of nx*ny*nz, in the direction order of cbl_read_populations. f_in and f_out are the
 * caller's device buffers (19 * nx*ny*nz floats each, not overlapping); mass_out (device, may be
 * NULL) receives the fluid mass of the step. The library cannot check the buffers' sizes or where
 * they live: too small a buffer, or a host pointer, is a memory fault on the GPU (the Python binding
 * checks them before the call). Scratch (psi, flags, mass slots) is a fixed set of device arrays
 * inside the library, sized for CBL_NOALLOC_MAX_CELLS cells and held on every GPU that loads the
 * library until the process exits; larger lattices return CBL_ERR_ARG. Each call looks up those
 * arrays with the calling device current and clears, on `stream`, the part it uses; the first call
 * on a device may load the library's device code, so make it before any stream capture. All calls
 * share the arrays: calls that overlap on the GPU (other streams, other threads) race. Work is
 * enqueued on `stream` (NULL = legacy default stream). Returns CBL_ERR_ARG for bad sizes,
 * non-finite parameters, NULL or overlapping buffers, CBL_ERR_CUDA if a CUDA call fails. */
#define CBL_NOALLOC_MAX_CELLS (1 << 20)
cbl_status cbl_lbm_step_noalloc(const float* f_in, float* f_out, int nx, int ny, int nz, double tau, double G,
                                double rho0, const double* ext_force, double* mass_out, void* stream);

/* Batches: advance many independent contexts (lattices of any size, each with its own bodies and
 * parameters) with one call; one captured CUDA graph holds one step of every instance.
 * Persistent mode (mode 1, the default when every instance has the same precision and velocity set
 * and uses the split pass): the step of all instances starts with ONE launch of a persistent kernel
 * that computes psi and then the bulk collision of every cell of every instance (Sec. 3.2.1, 3.2.3):
 * its grid is as large as the GPU holds resident blocks, each block takes work items (a tile of one
 * instance; tile shape from "tile", picked by the project's autotuner) from a device queue, and the
 * two phases are separated by a grid barrier whose wait is bounded (option "spin_limit", clock64
 * cycles, default ~2 s): a block that waits longer sets an error word and returns, and
 * cbl_batch_sync then returns CBL_ERR_TIMEOUT (that step's results are not valid; the contexts stay
 * usable). Each instance's remaining work (the cells next to a solid, the bodies, the phase fields,
 * flags and refill) follows on its own graph branch. Mode 0: one fork/join branch per instance with
 * its whole step. The contexts must be initialised (cbl_init_fluid), live on the current device
 * and outlive the batch; while in a batch they must not be stepped on their own. `stream` (may be
 * NULL: the library creates one) orders the batch's work. The batch itself allocates its instance
 * table and control block with cudaMalloc (a few kB). */
typedef struct cbl_batch cbl_batch;
cbl_status cbl_batch_create(cbl_ctx* const* ctxs, int n, void* stream, cbl_batch** out);
/* Advance every instance nsteps steps (asynchronous); the fields of the last step are kept. */
cbl_status cbl_batch_step(cbl_batch* batch, int nsteps);
/* Wait for the batch's stream; CBL_ERR_TIMEOUT if a grid-barrier wait of the persistent kernel ran
 * out since the last call (the error word is cleared). */
cbl_status cbl_batch_sync(cbl_batch* batch);
/* Batch options (synchronises, rebuilds the graphs): "mode" 0 or 1; "tile" 0..3, the persistent
 * kernel's tile of x * y * z cells: 32*4*1, 32*4*4 (default), 32*4*8, 64*2*4; "spin_limit" the
 * barrier wait limit in clock64 cycles (0 makes every wait run out at once: a test of the timeout
 * path). CBL_ERR_UNSUPPORTED for mode 1 over mixed precisions or velocity sets. */
cbl_status cbl_batch_set_option(cbl_batch* batch, const char* key, double value);
/* The batch's mode, tile shape, number of work items per phase and grid size (blocks). */
cbl_status cbl_batch_info(cbl_batch* batch, int* mode, int* tile, long long* items, int* grid);
cbl_status cbl_batch_destroy(cbl_batch* batch);

/* Force surrogate network (no counterpart in the paper's method: it stands in for the force
 * evaluation between full lattice-Boltzmann force evaluations). A multilayer perceptron
 * n_in -> hidden x n_hidden_layers -> n_out with tanh hidden units and a linear output; the built
 * configuration is 4 -> 64 -> 64 -> 64 -> 6 (inputs: gap, liquid volume, contact angle, radius ratio,
 * standardised by the caller; outputs: force and torque). Weights are used in bfloat16 with FP32
 * accumulation; an FP32 master copy is updated by Adam. Parameter layout (n = cbl_mlp_num_params
 * floats): for each layer W (out x in, row-major) then b (out). Device memory comes from cudaMalloc
 * (9,030 parameters, a few hundred kB). x, y, t are device pointers, [sample][feature] floats. */
typedef struct cbl_mlp cbl_mlp;
cbl_status cbl_mlp_create(int n_in, int hidden, int n_hidden_layers, int n_out, void* stream, cbl_mlp** out);
int64_t cbl_mlp_num_params(const cbl_mlp* mlp);
/* Set the FP32 master weights from a host array (resets Adam's moments), or read them back. */
cbl_status cbl_mlp_set_params(cbl_mlp* mlp, const float* params_host);
cbl_status cbl_mlp_get_params(cbl_mlp* mlp, float* params_host);
/* y = network(x) for n samples. */
cbl_status cbl_mlp_forward(cbl_mlp* mlp, const float* x, float* y, int n);
/* Add the gradient of the mean squared error over the n samples and 6 outputs to the internal
 * FP32 gradient; loss_host (may be NULL) receives the loss (synchronises the stream). */
cbl_status cbl_mlp_grad(cbl_mlp* mlp, const float* x, const float* t, int n, float* loss_host);
cbl_status cbl_mlp_read_grad(cbl_mlp* mlp, float* grad_host);
cbl_status cbl_mlp_zero_grad(cbl_mlp* mlp);
/* One Adam update of the master weights from the accumulated gradient, refresh the bfloat16
 * copy, clear the gradient. */
cbl_status cbl_mlp_adam_step(cbl_mlp* mlp, float lr, float beta1, float beta2, float eps);
cbl_status cbl_mlp_sync(cbl_mlp* mlp);
/* Advance nb rigid spheres `steps` semi-implicit Euler steps (dt = 1) under the network's pair forces
 * and torques plus a fixed per-body bias force, with the fluid frozen: the surrogate window of the
 * hybrid advance (no counterpart in the paper's method), all on the device in one launch. For every
 * step and bridged pair (i, j) (pairs: npairs * 2 body ids; VL: their bridge volumes), both sides
 * form the features in the pair frame (e_z from the body to its partner, minimum image over the
 * periodic box dims[3]): gap (r - R_i - R_j) sqrt(R* / V_L), cos_theta, R_i / R_j, V_L / R*^3 with
 * R* = 2 R_i R_j / (R_i + R_j); standardise them with norm = {x mean[4], x std[4], x min[4], x max[4],
 * y mean[6], y std[6]} (clipped to [min, max] first); run the network; and add force * 2 pi R* sigma
 * and torque * 2 pi R*^2 sigma, turned to the lattice frame, to body i. Then each body whose fixed[i]
 * is 0: V += (F + bias) / M, X += V (wrapped into the box), omega += T * Iinv (spheres: a scalar
 * inverse inertia). X, V, Wang (nb * 3, in/out), M, Iinv, R (nb), fixed (nb ints), bias (nb * 3),
 * pairs, VL are device pointers; dims and norm host pointers. nb <= 2048. CBL_ERR_ARG for bad sizes
 * or a non-finite or degenerate normalisation. Asynchronous on the network's stream. */
cbl_status cbl_mlp_advance(cbl_mlp* mlp, double* X, double* V, double* Wang, const double* M, const double* Iinv,
                           const double* R, const int* fixed, const double* bias, const int* pairs, const double* VL,
                           int nb, int npairs, int steps, const int* dims, double cos_theta, const float* norm,
                           double sigma);
cbl_status cbl_mlp_destroy(cbl_mlp* mlp);

/* Release every device allocation and the context. */
cbl_status cbl_destroy(cbl_ctx* ctx);

/* Human-readable description of the last failure on this context (never NULL). */
const char* cbl_last_error(const cbl_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* CBL_H */
