/*
 * galnb.h -- C ABI of the GB300 N-body/SPH interaction library.
 *
 * The calls follow the statement of the problem in Hirashima et al.,
 * "The First Star-by-star N-body/Hydrodynamics Simulation of Our Galaxy
 * Coupling with a Surrogate Model" (SC'25, arXiv 2510.23330):
 *   - particles carry position, velocity, mass and a per-particle softening
 *     (Sec. 3.5, Eq. 1 and the paragraph after it), an ID used to replace
 *     particles (Sec. 3.2, step 4) and, for gas, an internal energy;
 *   - positions are stored in FP64 and interactions are evaluated in FP32 on
 *     offsets relative to the receiving group (Sec. 4.3);
 *   - gravity is the softened pair force of Eq. 1 summed directly or by a
 *     Barnes-Hut tree with groups sharing one interaction list (Sec. 3.4,
 *     Sec. 5.2.2, 5.2.4);
 *   - SPH needs a kernel size, a density/pressure pass and a hydro-force pass
 *     (Sec. 5.2.5, Table 3, Table 4);
 *   - particles advance with the second-order leapfrog at a shared timestep
 *     (Sec. 3.2).
 *
 * Conventions shared by every call:
 *   - Return value: GNB_OK (0) or a negative GNB_E* code.  No call aborts or
 *     throws; gnb_last_error() gives a one-line reason for the last failure.
 *   - Ownership: the library copies every input into its own device arrays
 *     and never keeps a caller pointer.  Outputs are copied into caller
 *     buffers, in the caller's original particle order.
 *   - on_device: 0 means the pointers are host memory; 1 means they are
 *     device memory of the current CUDA device, readable on cfg.cuda_stream.
 *   - Streams: all device work of a context is issued on cfg.cuda_stream
 *     (NULL means the legacy default stream).  Every call returns only when
 *     its work has finished on that stream.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef GALNB_H
#define GALNB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GNB_OK 0
#define GNB_EINVAL (-1)    /* bad argument (null pointer, bad size, NaN position, ...) */
#define GNB_ENOMEM (-2)    /* device allocation failed */
#define GNB_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define GNB_ESTATE (-4)    /* call made in the wrong order (e.g. force before particles) */
#define GNB_ECAPACITY (-5) /* an internal list stayed over capacity after retries */
#define GNB_ETIMEOUT (-6)  /* a bounded device-side wait ran out */
#define GNB_EMISMATCH (-7) /* replacement IDs or count differ from the particles held */

/* Particle types (Sec. 1: stars and dark matter are collisionless, gas is SPH). */
#define GNB_STAR 0
#define GNB_GAS 1

/* Gravity modes of gnb_compute_gravity / gnb_step_kdk. */
#define GNB_GRAV_DIRECT 0  /* O(N^2) sum of Eq. 1 over all particles */
#define GNB_GRAV_TREE 1    /* Barnes-Hut group walk, particle-particle + particle-cell */
#define GNB_GRAV_NONE 2    /* no self-gravity (e.g. a supernova region evolved for 0.1 Myr) */

typedef struct gnb_ctx gnb_ctx;

/* Run parameters.  gnb_config_default() fills the defaults in brackets. */
typedef struct gnb_config {
    double G;          /* gravitational constant [1] */
    double theta;      /* opening angle of the Barnes-Hut test [0.5] */
    double gamma;      /* adiabatic index of the ideal-gas EOS [5/3] */
    double alpha_visc; /* artificial-viscosity coefficient [1] */
    int n_leaf;        /* a cell with more particles than this is split [16] */
    int n_group;       /* particles sharing one interaction list, n_g [64] */
    int n_ngb;         /* SPH neighbours, self included; only 64 is supported [64] */
    int multipole;     /* 0 = monopole, 1 = monopole + quadrupole [1] */
    double nfw_ms;     /* static NFW halo mass scale 4 pi rho_s r_s^3; 0 disables [0] */
    double nfw_rs;     /* NFW scale radius [8] */
    void *cuda_stream; /* cudaStream_t for all work; NULL = default stream [NULL] */
    int sph_variant;   /* SPH formulation [0]: 0 = density-energy, P_i = (gamma-1) rho_i u_i;
                          1 = pressure-energy: the density and pressure pass (Table 3) also
                          smooths P_i = (gamma-1) sum_j m_j u_j W_ij(h_i), and the pair force
                          uses (gamma-1)^2 u_i u_j / P_i and / P_j in place of P_i / rho_i^2
                          and P_j / rho_j^2 (a reading) */
} gnb_config;

/* Fields readable with gnb_get.  Element type and count in brackets; n is
 * the particle count, "gas" rows are ordered like the gas particles in the
 * caller's original order. */
enum gnb_field {
    GNB_F_X = 0, GNB_F_Y, GNB_F_Z,  /* position [double, n] */
    GNB_F_VX, GNB_F_VY, GNB_F_VZ,   /* velocity [float, n] */
    GNB_F_AX, GNB_F_AY, GNB_F_AZ,   /* total acceleration [float, n] */
    GNB_F_POT,                      /* self-gravity potential phi [float, n] */
    GNB_F_U,                        /* internal energy, 0 for stars [float, n] */
    GNB_F_DUDT,                     /* du/dt, 0 for stars [float, n] */
    GNB_F_RHO,                      /* SPH density, 0 for stars [float, n] */
    GNB_F_PRES,                     /* pressure ((gamma-1) rho u, or the smoothed pressure when
                                       sph_variant = 1), 0 for stars [float, n] */
    GNB_F_CS,                       /* sound speed, 0 for stars [float, n] */
    GNB_F_H2,                       /* squared kernel support h^2, 0 for stars [double, n] */
    GNB_F_KEY,                      /* Morton key of the last sort [uint64, n] */
    GNB_F_ORDER,                    /* original index of the particle at each sorted slot [int64, n] */
    GNB_F_NBR,                      /* neighbour lists: n_ngb original indices per gas particle,
                                       ascending [int64, n_gas * n_ngb] */
    GNB_F_NODES,                    /* tree nodes, breadth-first: 4 int64 per node
                                       (level, prefix, first, count) [int64, 4 * nodes] */
    GNB_F_GROUPS,                   /* groups: node index of each group, ascending first
                                       particle [int64, groups] */
    GNB_F_ID,                       /* particle IDs [int64, n] */
    GNB_F_AGRAV_X, GNB_F_AGRAV_Y, GNB_F_AGRAV_Z, /* self-gravity part of a [float, n] */
    GNB_F_LEVEL,                    /* timestep level k (step t_span 2^-k) of each particle's last step
                                       in gnb_integrate_hier [int32, n] */
    GNB_F_POT_EXT,                  /* potential of the static NFW halo, 0 when it is off [float, n] */
    GNB_F_NODE_LINKS,               /* links of the tree nodes, in GNB_F_NODES order: 3 int64 per node
                                       (first child or -1, children, parent or -1) [int64, 3 * nodes] */
    GNB_F_COUNT_
};

/* Counters readable with gnb_stats (int64 out[GNB_S_COUNT_]). */
enum gnb_stat {
    GNB_S_N = 0,        /* particles */
    GNB_S_NGAS,         /* gas particles */
    GNB_S_NODES,        /* gravity tree nodes */
    GNB_S_GROUPS,       /* gravity groups */
    GNB_S_NPP,          /* particle-particle interactions of the last gravity pass */
    GNB_S_NPC,          /* particle-cell interactions of the last gravity pass */
    GNB_S_GAS_NODES,    /* hydro tree nodes */
    GNB_S_KNN_PASSES,   /* kernel-size search passes of the last density call */
    GNB_S_NSYM,         /* entries of the symmetric SPH force lists */
    GNB_S_MAXLEVEL,     /* deepest tree level */
    GNB_S_COUNT_
};

/* Phases timed by gnb_phase_times (the timing convention of Sec. 4.3:
 * timers around each routine, here CUDA events on cfg.cuda_stream). */
enum gnb_phase {
    GNB_T_SORT = 0,     /* root box, Morton keys, radix sort, permutation */
    GNB_T_TREE,         /* octree, cell moments, groups */
    GNB_T_GRAVITY,      /* tree walk + particle-particle/particle-cell kernel (or direct sum) */
    GNB_T_EXTERNAL,     /* static halo and force assembly */
    GNB_T_HYDRO_TREE,   /* gas extraction and hydro tree */
    GNB_T_KNN,          /* kernel size + density/pressure */
    GNB_T_FORCE,        /* symmetric lists + hydro force */
    GNB_T_KDK,          /* kicks, drift, prediction */
    GNB_T_VOXELISE,     /* surrogate: region membership, voxelisation, standardisation */
    GNB_T_UNET,         /* surrogate: U-Net forward */
    GNB_T_REMAP,        /* surrogate: Gibbs remap and replacement */
    GNB_T_COUNT_
};

/* Fill cfg with the defaults listed in gnb_config. */
void gnb_config_default(gnb_config *cfg);

/* Create a context on the current CUDA device.  *out is set on success.
 * Errors: GNB_EINVAL (null or invalid cfg), GNB_ECUDA. */
int gnb_create(gnb_ctx **out, const gnb_config *cfg);

/* Replace the parameters of a context (same rules as gnb_create).  The
 * particles are kept; the tree and all forces must be recomputed.  Used to
 * choose n_group on the data (Sec. 5.2.4: the best n_g depends on the
 * hardware).  Errors: GNB_EINVAL. */
int gnb_set_config(gnb_ctx *ctx, const gnb_config *cfg);

/* Free a context and all its device memory (NULL is ignored). */
void gnb_destroy(gnb_ctx *ctx);

/* Load n particles (Sec. 3.5: position, mass, softening per particle;
 * Sec. 3.2: IDs).  Arrays are SoA of length n; u is read for gas only.
 * Positions are FP64 (Sec. 4.3), velocities and the other fields FP32.
 * Clears all derived state.  Errors: GNB_EINVAL (n < 1, null pointer,
 * non-finite position, type not in {0,1}, n_ngb > number of gas particles
 * when gas exists), GNB_ENOMEM, GNB_ECUDA. */
int gnb_set_particles(gnb_ctx *ctx, int64_t n, const int64_t *id, const uint8_t *type,
                      const double *x, const double *y, const double *z,
                      const float *vx, const float *vy, const float *vz,
                      const float *m, const float *eps, const float *u, int on_device);

/* Load n particles with the state a kick-drift-kick integration carries
 * from one step to the next (Sec. 3.1: the kick at the start of a step uses
 * the accelerations of the step's end): the arrays of gnb_set_particles,
 * plus the total acceleration ax, ay, az and du/dt (the fields GNB_F_AX,
 * GNB_F_AY, GNB_F_AZ and GNB_F_DUDT of a context) evaluated on this state
 * with gravity mode grav_mode, and optionally the squared kernel supports h2
 * (GNB_F_H2; 0 for stars; NULL: none), the kernel-size search's starting
 * radii.  A following gnb_step_kdk with the same mode kicks with the given
 * accelerations instead of evaluating the forces first; the other results
 * (gravity alone, potentials, density) are not current until the next force
 * evaluation.  All arrays are in the caller's order, host or device as
 * on_device says.  Errors: as gnb_set_particles, and GNB_EINVAL for a null
 * acceleration or du/dt array or an invalid mode.  If the call fails after
 * the particles were set, the context holds them without forces. */
int gnb_set_state(gnb_ctx *ctx, int64_t n, const int64_t *id, const uint8_t *type,
                  const double *x, const double *y, const double *z,
                  const float *vx, const float *vy, const float *vz,
                  const float *m, const float *eps, const float *u, const double *h2,
                  const float *ax, const float *ay, const float *az, const float *dudt,
                  int grav_mode, int on_device);

/* Sort particles along the Morton curve and build the octree, its cell
 * moments and the groups (Sec. 3.4, 5.2.2).  Errors: GNB_ESTATE (no
 * particles), GNB_ECUDA. */
int gnb_build_tree(gnb_ctx *ctx);

/* Self-gravity (Eq. 1) of every particle, plus the static NFW halo when
 * enabled; mode is GNB_GRAV_DIRECT or GNB_GRAV_TREE.  Builds the tree first
 * if needed.  Writes acceleration and potential.  Errors: GNB_EINVAL (mode),
 * GNB_ESTATE, GNB_ECUDA. */
int gnb_compute_gravity(gnb_ctx *ctx, int mode);

/* SPH kernel size (exact n_ngb nearest gas neighbours, Sec. 5.2.5), density
 * and pressure (Table 3 "density and pressure"; with sph_variant = 1 the
 * pressure is smoothed over the neighbours, see gnb_config).  Builds the tree
 * first if needed.  Errors: GNB_ESTATE, GNB_ECAPACITY (e.g. more than 64
 * particles tied at one neighbour distance), GNB_ECUDA. */
int gnb_compute_sph_density(gnb_ctx *ctx);

/* SPH pressure force, artificial viscosity and du/dt over the symmetric
 * neighbour sets (Table 3 "hydro force").  Adds the hydro acceleration to
 * the total acceleration.  Requires gnb_compute_sph_density since the last
 * change of positions.  Errors: GNB_ESTATE, GNB_ECUDA. */
int gnb_compute_sph_force(gnb_ctx *ctx);

/* Total force evaluation: sort and tree build, gravity (mode), NFW, SPH
 * density and force.  With GNB_GRAV_NONE (and in the integrators below with
 * that mode) the particles are sorted but the gravity tree is not built:
 * GNB_F_NODES and GNB_F_GROUPS then return GNB_ESTATE.  Errors: as the calls
 * above. */
int gnb_compute_forces(gnb_ctx *ctx, int gravity_mode);

/* nsteps kick-drift-kick leapfrog steps with shared timestep dt (Sec. 3.2):
 * half kick, drift (FP64 positions), full force evaluation with predicted
 * gas velocity and energy, half kick.  Forces at the start are computed
 * first if they are not current.  Errors: GNB_EINVAL (dt not finite,
 * nsteps < 0, mode), GNB_ESTATE, GNB_ECAPACITY, GNB_ECUDA. */
int gnb_step_kdk(gnb_ctx *ctx, double dt, int nsteps, int gravity_mode);

/* Supernova energy injection (Sec. 1: 10^51 erg per explosion; the injection
 * rule is a reading): thermal energy `energy` is added to the n_ngb gas
 * particles nearest to pos (ordered by FP64 d^2, then gas rank) with cubic
 * spline weights whose support is the distance to the n_ngb-th of them:
 * du_j = energy W_j / (m_j sum_k W_k).  info (may be NULL) receives
 * {sum of weights, energy actually added (FP64 sum of m du after rounding u
 * to FP32), support h, particles heated}.  Errors: GNB_EINVAL, GNB_ESTATE
 * (no particles or fewer gas particles than n_ngb), GNB_ECUDA. */
int gnb_inject_energy(gnb_ctx *ctx, const double pos[3], double energy, double info[4]);

/* Shared CFL timestep of the last SPH force pass (Sec. 1: the CFL condition
 * limits the hydro timestep): dt = courant * min_i h_i / vsig_i, vsig_i =
 * max_j (c_i + c_j - 3 min(w_ij, 0)).  Errors: GNB_EINVAL, GNB_ESTATE (no SPH
 * force at the current positions). */
int gnb_cfl_timestep(gnb_ctx *ctx, double courant, double *dt);

/* Plain small-timestep integration (the conventional integration of Sec. 3.2
 * and 5.3 that the surrogate replaces): kick-drift-kick steps of the CFL
 * timestep above, the last one shortened to end exactly at t_span, at most
 * max_steps steps.  t_done and steps_done (may be NULL) receive the time
 * covered and the steps taken.  Errors: GNB_EINVAL, GNB_ESTATE (no gas),
 * GNB_ECAPACITY, GNB_ECUDA. */
int gnb_integrate_cfl(gnb_ctx *ctx, double t_span, double courant, int max_steps, int gravity_mode,
                      double *t_done, int64_t *steps_done);

/* Plain integration with hierarchical (block) individual timesteps (Sec. 1:
 * every particle has its own timestep and is updated only when it ends, while
 * all particles are predicted and the tree is rebuilt at each step; the rules
 * are a reading).  The span is 2^(max_level+1) integer ticks; level k steps
 * t_span 2^-k.  A step starting at tick T takes the coarser of the gas
 * particle's CFL level (the coarsest k with t_span 2^-k <= courant h / vsig;
 * level 0 for other particles) and the coarsest level whose step divides T.
 * Each block step goes to the next tick at which a step ends, drifts all
 * particles there, predicts v and u of every particle from the force of its
 * last update (v + a (t - t_mid), t_mid the middle of its step), evaluates
 * all forces (gravity_mode as in gnb_compute_forces) at the predicted state
 * and kicks the particles whose step ends there; a particle whose CFL level
 * there is finer than its own is woken: its step is cut to end there (its
 * opening kick and drift are corrected) and it is kicked too.  All particles
 * end synchronised at t_span unless max_steps block steps come first (then
 * velocities are those of the particles' current half steps).
 * t_done (may be NULL) receives the time reached; info (may be NULL) {block
 * steps, particle updates after the start, wake-ups}.  The levels are read
 * with GNB_F_LEVEL.  Errors: GNB_EINVAL (t_span, courant, max_level outside
 * 1..40, max_steps < 0, mode), GNB_ESTATE (no particles or no gas, a pending
 * asynchronous surrogate batch), GNB_ECAPACITY (a gas particle's CFL step
 * at some block step is shorter than the finest level's: that block step
 * kicks nobody, so the particles stay within their steps), GNB_ECUDA. */
int gnb_integrate_hier(gnb_ctx *ctx, double t_span, double courant, int max_level, int max_steps, int gravity_mode,
                       double *t_done, int64_t info[3]);

/* Replace particles by ID (Sec. 3.2, step 4: the particles of a supernova
 * region, integrated elsewhere -- by the surrogate, by the plain small-step
 * integration, on another device or from a checkpoint -- are handed back and
 * overwrite the particles with the same IDs).  n particles in SoA arrays:
 * id, FP64 position, FP32 velocity and internal energy (u is read for gas
 * particles only; a particle keeps its type, mass and softening).  Every ID
 * must be held by exactly one particle of the context and appear once in
 * the input; the particles are checked first and written only if all pass,
 * so a rejected call changes nothing.  A region is the set of particles its
 * IDs name: membership is not re-tested against a cube, since particles
 * drift between hand-off and return.  Positions change, so trees and forces
 * must be recomputed.  on_device as in gnb_set_particles.
 * Errors: GNB_EINVAL (n < 1, null pointer, non-finite position),
 * GNB_ESTATE (no particles, a pending asynchronous surrogate batch),
 * GNB_EMISMATCH (an ID not held, held twice, or repeated in the input;
 * more particles than the context holds), GNB_ENOMEM, GNB_ECUDA. */
int gnb_replace_region(gnb_ctx *ctx, int64_t n, const int64_t *id, const double *x, const double *y,
                       const double *z, const float *vx, const float *vy, const float *vz, const float *u,
                       int on_device);

/* Copy one field into dst, which holds cap elements of the field's type.
 * Errors: GNB_EINVAL (field, cap too small, null dst), GNB_ESTATE (field
 * not computed yet), GNB_ECUDA. */
int gnb_get(gnb_ctx *ctx, int field, void *dst, int64_t cap, int on_device);

/* gnb_get of nf fields at once: field fields[k] into dst[k], which holds
 * cap[k] elements of its type; all host or all device as on_device says.
 * Every field is checked before any is copied; host copies are queued on
 * the context's stream and the call waits once for all of them.  Errors: as
 * gnb_get (nothing is copied then), and GNB_EINVAL for nf < 0 or a null
 * list with nf > 0. */
int gnb_get_fields(gnb_ctx *ctx, int nf, const int *fields, void *const *dst, const int64_t *cap, int on_device);

/* Checkpoint of the particle state (no counterpart in the paper, which
 * describes no checkpoints).  gnb_save writes to `path`, in the caller's
 * particle order: IDs, types, FP64 positions, velocities, masses, softening
 * lengths, internal energies, the squared kernel supports, and the results
 * of the last force evaluation (accelerations, potentials, du/dt, density,
 * pressure, sound speed) with flags saying which are current.  gnb_load
 * replaces the context's particles by the file's (as gnb_set_particles
 * does, so the caller order is the file's) and restores the supports and
 * the current results: gnb_step_kdk then continues with the same kicks, and
 * every field reads back equal to the saved context's, except GNB_F_NBR,
 * which needs a new kernel-size search.  Not saved: the hierarchical
 * integrator's step state and surrogate batches.  Errors: GNB_EINVAL (NULL,
 * a file that cannot be opened, read or written or is not a state file, or
 * invalid particles in it), GNB_ESTATE (gnb_save without particles or with
 * an asynchronous surrogate batch pending), GNB_EMISMATCH (the file's gas
 * count disagrees with its particle types), GNB_ENOMEM, GNB_ECUDA.  If
 * gnb_load fails after its particles were set, the context holds them
 * without the restored results. */
int gnb_save(gnb_ctx *ctx, const char *path);
int gnb_load(gnb_ctx *ctx, const char *path);

/* FP64 totals: out = {E_kin, E_pot (1/2 sum m phi), E_ext (sum m Phi_nfw),
 * E_th (sum m u over gas), P_x, P_y, P_z, L_x, L_y, L_z}.  Requires a force
 * evaluation at the current positions.  Errors: GNB_ESTATE, GNB_ECUDA. */
int gnb_diagnostics(gnb_ctx *ctx, double out[10]);

/* Counters of the last passes (enum gnb_stat).  Errors: GNB_EINVAL. */
int gnb_stats(gnb_ctx *ctx, int64_t out[GNB_S_COUNT_]);

/* Enable (1) or disable (0) the per-phase timers.  While enabled, every
 * call records a pair of CUDA events around each phase it runs.
 * Errors: GNB_EINVAL (null ctx). */
int gnb_set_timing(gnb_ctx *ctx, int enable);

/* Device time per phase (enum gnb_phase) in milliseconds, summed over the
 * calls since the last reset; calls[p] counts the timed occurrences and
 * *launches the kernels this library launched in the process since the last
 * reset (any of the three outputs may be NULL).  reset = 1 clears the sums
 * after reading.  Errors: GNB_EINVAL (null ctx). */
int gnb_phase_times(gnb_ctx *ctx, double out_ms[GNB_T_COUNT_], int64_t calls[GNB_T_COUNT_],
                    int64_t *launches, int reset);

/* ------------------------------------------------------------------------
 * Supernova surrogate: 3D U-Net (Sec. 3.3: a U-Net of 3D convolutions that
 * maps the gas around a supernova, voxelised on a 64^3 grid, to its state
 * 0.1 Myr later; MSE loss and Adam; trained at batch size 1).  The layer list
 * is a reading: `levels` levels of widths base, 2 base, ...; two 3^3
 * convolutions with zero padding and ReLU per level; 2^3 max-pool; 2^3
 * stride-2 transposed convolution; skip concatenated before the up-sampled
 * tensor; a 1^3 linear head.  Computation: BF16 operands on the tensor cores
 * with FP32 accumulation; FP32 master weights and Adam state.
 * Tensors are FP32 [batch][z][y][x][channel] (channels innermost).
 * Parameters are one FP32 array, layer by layer in the order enc0a, enc0b,
 * enc1a, ..., up(levels-2), dec(levels-2)a, dec(levels-2)b, ..., up0, dec0a,
 * dec0b, head; per layer W[taps][cin][cout] then b[cout], with the 27 taps of
 * a 3^3 convolution ordered (dz, dy, dx) over {-1,0,1}^3 with dx fastest and
 * the 8 taps of the transposed convolution t = 4 tz + 2 ty + tx. */
typedef struct gnb_unet gnb_unet;

/* Create a U-Net on the current device with zero parameters.  Supported:
 * 1 <= cin <= 16, 1 <= cout <= 8, base in {8, 16, 24, 32}, 2 <= levels <= 5,
 * grid divisible by 2^(levels-1) with at least 2 voxels at the coarsest level.
 * stream: cudaStream_t (NULL = default).  Errors: GNB_EINVAL, GNB_ENOMEM. */
int gnb_unet_create(gnb_unet **out, int cin, int cout, int base, int levels, int grid, void *stream);
void gnb_unet_destroy(gnb_unet *net);
/* Number of FP32 parameters (-1 for NULL). */
int64_t gnb_unet_num_params(const gnb_unet *net);
/* Copy the parameters out / in (set also resets the Adam state).
 * Errors: GNB_EINVAL, GNB_ECUDA. */
int gnb_unet_get_params(gnb_unet *net, float *dst, int on_device);
int gnb_unet_set_params(gnb_unet *net, const float *src, int on_device);
/* Checkpoint of a network (no counterpart in the paper, which describes no
 * checkpoints): gnb_unet_save writes the FP32 master parameters, Adam's two
 * moments and its step count to `path` (a 64-byte header, then three arrays
 * of gnb_unet_num_params floats); gnb_unet_load reads such a file into a
 * network of the same shape (cin, cout, base, levels, grid), after which
 * training continues exactly where the saved network stopped.  Errors:
 * GNB_EINVAL (NULL, a file that cannot be opened, read or written, or is not
 * a network checkpoint), GNB_EMISMATCH (another network shape), GNB_ECUDA. */
int gnb_unet_save(gnb_unet *net, const char *path);
int gnb_unet_load(gnb_unet *net, const char *path);
/* Gradients of the last gnb_unet_train_step (before its Adam update). */
int gnb_unet_get_grads(gnb_unet *net, float *dst, int on_device);
/* The FP32 output [batch][grid^3][cout] of the network's last forward pass,
 * first `batch` samples: gnb_unet_forward, gnb_unet_train_step, or the
 * prediction gnb_sn_surrogate_batch remapped from (its regions in the order
 * of `centers`).  Errors: GNB_EINVAL (batch < 1 or above the batch of the
 * largest pass so far, NULL), GNB_ECUDA. */
int gnb_unet_get_output(gnb_unet *net, int batch, float *dst, int on_device);
/* Tile autotuner of the tensor-core convolutions (the paper runs its network
 * on CPUs and has no counterpart): one forward pass of `batch` samples on the network's current
 * input buffer times every supported tile plan of each 3^3 layer (tile depth,
 * halo buffering, resident or streamed weights) on that layer's real tensors
 * and keeps the fastest for every later forward pass, including those of
 * gnb_sn_surrogate_batch; if the whole pass with the chosen plans is not
 * faster than with the built-in rule, the rule is kept.  out_ms (may be
 * NULL) receives the forward pass's time before and after.  Synchronises the
 * network's stream: do not call it during a stream capture.  Changing the
 * network's parameters keeps the plans.  Errors: GNB_EINVAL, GNB_ENOMEM,
 * GNB_ECUDA, GNB_ETIMEOUT. */
int gnb_unet_autotune(gnb_unet *net, int batch, double out_ms[2]);

/* A tensor the last forward pass stored, as FP32 [batch][g^3][C] (g the
 * grid of its level, C its channels), first `batch` samples.  Slots in the
 * order the forward pass writes them: 0 the BF16 network input (cin
 * channels), then for each level l = 0 .. levels-1 the outputs of enc l a
 * and enc l b and, below the coarsest level, the max-pooled tensor (level
 * l+1 grid); then for each decoder level l = levels-2 .. 0 the outputs of
 * up l (the transposed convolution), dec l a and dec l b.  Read them after
 * gnb_unet_forward: a training step reuses the dec l a buffers for
 * gradients.  With the gradients of gnb_unet_get_grads this lets
 * back-propagation be checked layer by layer on the activations the network
 * actually stored.  Errors: GNB_EINVAL (slot
 * out of range, batch, NULL), GNB_ENOMEM, GNB_ECUDA. */
int gnb_unet_get_activation(gnb_unet *net, int slot, int batch, float *dst, int on_device);
/* Convolution kernels of the 3^3 layers.  GNB_CONV_AUTO (the default): the
 * tcgen05 tensor-core kernel (TMA halo tiles, TMEM accumulators) wherever the
 * channel counts are multiples of 16 and its weights fit in shared memory,
 * the mma.sync implicit GEMM elsewhere; GNB_CONV_MMA_SYNC: the mma.sync
 * implicit GEMM for every layer.  Both compute the same products with FP32
 * accumulation.  A bounded device wait of the tensor-core kernel that runs out
 * makes the call return GNB_ETIMEOUT.  Errors: GNB_EINVAL. */
#define GNB_CONV_AUTO 0
#define GNB_CONV_MMA_SYNC 2
int gnb_unet_set_conv_impl(gnb_unet *net, int impl);
/* Inference: x [batch][grid^3][cin] -> y [batch][grid^3][cout] (FP32).
 * Errors: GNB_EINVAL, GNB_ENOMEM, GNB_ECUDA, GNB_ETIMEOUT. */
int gnb_unet_forward(gnb_unet *net, int batch, const float *x, float *y, int on_device);
/* One training step: forward, MSE against target, back-propagation and, if
 * lr > 0, one Adam step (beta1 0.9, beta2 0.999, eps 1e-8).  *loss (may be
 * NULL) receives the mean squared error before the update. */
int gnb_unet_train_step(gnb_unet *net, int batch, const float *x, const float *target, double lr,
                        double *loss, int on_device);

/* ------------------------------------------------------------------------
 * Surrogate coupling (Sec. 3.2-3.3).  A region r is the cube of side `side`
 * centred on centers[3r..3r+2] (host array); a gas particle belongs to the
 * first region containing it (|x - c|_inf <= side/2).  Grids have grid^3
 * voxels with centres lo + (i + 1/2) side/grid, x fastest.  Channels
 * (standardised network units; the scalings are a reading):
 *   z0 = log10(max(rho, 1e-4)) + 0.33, z1 = (log10(max(T, 10)) - 2) / 2,
 *   z2..z4 = v / 20,
 * with rho in the mass/length^3 units of the particles (Msun/pc^3), T in K
 * from T = u (gamma-1) mu m_H / k_B (mu = 0.6, u in (km/s)^2), v in km/s.
 * --------------------------------------------------------------------- */

/* Voxelise the gas of nreg regions (Sec. 3.3: SPH kernel convolution for the
 * density, Shepard averages for T and v; empty voxels get rho = 0, T = 10 K,
 * v = 0).  out: [nreg][grid^3][5] FP32.  Requires gnb_compute_sph_density
 * at the current positions.  Errors: GNB_EINVAL, GNB_ESTATE, GNB_ENOMEM,
 * GNB_ECUDA. */
int gnb_voxelise(gnb_ctx *ctx, int nreg, const double *centers, double side, int grid, float *out,
                 int on_device);

/* Replace the gas of each region by the same number of particles, keeping
 * IDs and masses (Sec. 3.2 step 4; Sec. 3.3: Gibbs sampling, mass conserved
 * by keeping the particle count), drawn from the predicted grid pred
 * [nreg][grid^3][5]: from the voxel of its old position each particle makes
 * `sweeps` Gibbs sweeps over x, y, z, each draw choosing a voxel on the
 * current line with probability proportional to 10^(z0 - 0.33) (FP64 CDF),
 * then a uniform offset in the voxel; u and v come from the chosen voxel.
 * Draw k of particle id uses U = (splitmix64(splitmix64(seed + id) + k) >> 11)
 * * 2^-53.  Positions change, so trees and forces must be recomputed.
 * Errors: GNB_EINVAL, GNB_ESTATE, GNB_ECUDA. */
int gnb_remap_regions(gnb_ctx *ctx, int nreg, const double *centers, double side, int grid,
                      const float *pred, uint64_t seed, int sweeps, int on_device);

/* Batched surrogate step for nreg supernova regions of uneven particle
 * counts: voxelise -> U-Net forward (net, which must predict 5 channels on
 * its own grid) -> Gibbs remap, as above, pipelined over region chunks (see
 * gnb_set_sn_chunks).  With use_graph = 1, a non-default stream and the
 * phase timers off, the whole batch (all streams) is captured into one CUDA
 * graph on the first call and replayed while the shapes stay the same.  Requires
 * gnb_compute_sph_density at the current positions.  Errors: GNB_EINVAL,
 * GNB_ESTATE, GNB_ENOMEM, GNB_ECUDA. */
int gnb_sn_surrogate_batch(gnb_ctx *ctx, gnb_unet *net, int nreg, const double *centers, double side,
                           uint64_t seed, int sweeps, int use_graph);

/* Asynchronous surrogate batch: the pool nodes' role in Sec. 3.2 (steps
 * 2-4), where the supernova regions are handed off, predicted while the
 * global integration goes on, and returned 0.1 Myr (50 global steps) later.
 * gnb_sn_async_submit takes a snapshot of the members of the nreg regions
 * (the same membership rule as gnb_voxelise) on the context's stream -- their
 * state, caller index and ID -- and then voxelises the snapshot, runs the
 * U-Net (net) and builds the remap's line sums on a second stream; it
 * returns without waiting.  The context's steps may run meanwhile.
 * gnb_sn_async_apply waits for that work and replaces every snapshot member,
 * found at its current position in the arrays by its caller index, exactly
 * as gnb_remap_regions would: sweeps Gibbs sweeps on the prediction starting
 * from the voxel of its snapshot position, with draws from (seed, ID); u
 * and v from the drawn voxel.  One batch can be pending per context; while
 * it is, gnb_set_particles, gnb_voxelise, gnb_remap_regions and
 * gnb_sn_surrogate_batch return GNB_ESTATE, and net must not be used.
 * Requires gnb_compute_sph_density at the current positions for the submit.
 * gnb_sn_async_pending returns 1 while a batch is pending, else 0.
 * Errors: GNB_EINVAL, GNB_ESTATE (a batch pending at submit, none at apply),
 * GNB_ENOMEM, GNB_ECUDA, GNB_ETIMEOUT (as gnb_unet_forward). */
int gnb_sn_async_submit(gnb_ctx *ctx, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                        int sweeps);
int gnb_sn_async_apply(gnb_ctx *ctx);
int gnb_sn_async_pending(const gnb_ctx *ctx);

/* Number of region chunks the batched surrogate step pipelines (1 to 16;
 * default 1, the stages in sequence): with k > 1 chunks, chunk i is
 * voxelised on the context's stream, goes through the U-Net on a second
 * stream and is remapped on a third, so the stages of different chunks can
 * overlap.  With the phase timers on, the step always runs its stages in
 * sequence.  Errors: GNB_EINVAL (chunks outside 1..16). */
int gnb_set_sn_chunks(gnb_ctx *ctx, int chunks);

/* Largest particle count accepted by gnb_morton_order_noalloc. */
#define GNB_NOALLOC_MAX_N 262144

/* Morton keys and space-filling-curve order of n particles without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory -- an application whose
 * device memory is owned by another allocator (a framework's caching pool
 * or a fixed arena), or a latency-sensitive loop in which cudaMalloc and
 * cudaFree would synchronise the device or could fail under memory
 * pressure.  It computes exactly what gnb_build_tree computes for the keys
 * (GNB_F_KEY) and the order (GNB_F_ORDER): root box, 63-bit keys, order by
 * (key, caller index).
 *
 * Scratch: one static device array of 6,424,320 bytes (6.13 MiB) inside
 * libgalnb.so; every GPU that loads the library holds it until the process
 * exits.  The first call on a device looks up the array's device address
 * (with that device current) and keeps it for the life of the process, so
 * make that first call before any stream capture, and do not call this
 * entry point on a device after cudaDeviceReset there (the array went away
 * with the context).  Every call reuses the same array and clears what must
 * start at zero itself; calls that overlap on the GPU (different streams or
 * host threads, same device) race and give wrong results, so the caller
 * must serialise them.  Every call waits for its own work on `stream` to
 * finish before it returns: it reads back a flag that marks a non-finite
 * position.  The call uses no cudaMalloc, cudaFree or allocating library
 * routine.
 *
 * x, y, z: device FP64 positions, n each, caller order.  keys: device
 * uint64[n], written with each particle's key in caller order.  order:
 * device int64[n], written with the caller index of the particle at each
 * sorted slot.  stream: cudaStream_t (NULL = default stream); the call
 * returns after its work on stream has finished.
 * Errors: GNB_EINVAL (n < 1 or n > GNB_NOALLOC_MAX_N, null pointer, or a
 * non-finite position -- keys and order are then not valid), GNB_ECUDA. */
int gnb_morton_order_noalloc(int64_t n, const double *x, const double *y, const double *z,
                             uint64_t *keys, int64_t *order, void *stream);

/* One-line description of the last error of ctx ("" if none; a static
 * string if ctx is NULL). */
const char *gnb_last_error(const gnb_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* GALNB_H */
