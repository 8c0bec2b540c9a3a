/*
 * mw.h -- C ABI of libmw, the GB300 (sm_103a) engine for the mW water model
 * of Molinero & Moore, "Water modeled as an intermediate element between
 * carbon and silicon".
 *
 * The model (Sec. II.A of the paper) is the Stillinger-Weber form
 *   E = sum_i sum_{j>i} phi2(r_ij) + sum_i sum_{j!=i} sum_{k>j} phi3(r_ij, r_ik, theta_jik)
 *   phi2(r)       = A eps [B (sig/r)^p - (sig/r)^q] exp(sig / (r - a sig))
 *   phi3(r,s,th)  = lam eps [cos th - cos th0]^2 exp(gam sig/(r - a sig)) exp(gam sig/(s - a sig))
 * with every term zero beyond r = a sig.  This library evaluates energy,
 * forces and virial over cell-list / Verlet neighbour lists in orthorhombic
 * periodic boxes and advances velocity-Verlet dynamics (Sec. II.B: 10 fs
 * step, Nose-Hoover thermostat with a 1 ps relaxation time), for one box or
 * for a batch of independent boxes, plus the adjoint of the forces for
 * force-matching fits of (lambda, epsilon, sigma) (the parameters Sec. II.D
 * tunes).
 *
 * Conventions for every call:
 *   - Units: Angstrom, fs, kcal/mol, g/mol, K; forces kcal/mol/A; velocities
 *     A/fs; pressure atm.
 *   - Every call returns an mw_status; nothing is thrown across the ABI.  On
 *     failure mw_last_error() holds a message for the calling thread.
 *   - Atoms of all boxes are concatenated box-major: box b owns the global
 *     atom indices [off_b, off_b + n_b), off_b = n_0 + ... + n_{b-1}.
 *     Per-atom vectors are AoS, 3 doubles (or floats) per atom.
 *   - Host pointers are owned by the caller and only read or written during
 *     the call.  "_dev" calls take device pointers that must stay valid until
 *     the call returns; they are enqueued on the system's stream and the
 *     call synchronises that stream before returning.
 *   - The library owns all its device buffers (allocated at create time and
 *     when a neighbour list must grow) and frees them in mw_system_destroy.
 *   - One mw_system must not be used from two threads at once.
 *   - Environment: MW_AUTOTUNE_CACHE (see mw_autotune); MW_GRAPH_NO_CONDITIONAL
 *     (any value) captures the graph engine's step without its conditional
 *     node - every kernel launches each step and the rebuild kernels return at
 *     once when not needed - for profilers that do not follow conditional
 *     graph nodes.
 */
#ifndef MW_H
#define MW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Potential parameters (Sec. II.A: A, B, p, q, gamma, a, theta0 of the SW
 * form; Sec. II.D: lambda = 23.15, epsilon = 6.189 kcal/mol,
 * sigma = 2.3925 A).  cos_theta0 = -1/3 is the reading of "theta0 = 109.47
 * deg" as the tetrahedral angle. */
typedef struct mw_params {
  double lambda, epsilon, sigma, a, gamma, A, B, cos_theta0;
  int p, q;
} mw_params;

typedef enum mw_status {
  MW_OK = 0,
  MW_EINVAL = 1,           /* bad argument (null pointer, size, non-finite input) */
  MW_EBOX = 2,             /* a box edge is shorter than 2 * (a sigma + skin) */
  MW_ENLIST_OVERFLOW = 3,  /* neighbour list wider than its allocation (recovered internally by mw_step) */
  MW_ENAN = 4,             /* non-finite force or velocity met during dynamics */
  MW_ELOST = 5,            /* a velocity component would move an atom > 1/4 of the shortest edge per step */
  MW_ETIMEOUT = 6,         /* a bounded device-side wait ran out (persistent engine) */
  MW_ECUDA = 7,            /* a CUDA runtime call failed */
  MW_ENOMEM = 8,           /* device or host allocation failed */
  MW_ESTATE = 9,           /* call out of order (e.g. forces before any state was set) */
  MW_EGRID = 10            /* mw_step_async/mw_sync only: an isobaric box shrank or grew out of its cell
                              grid; the run stopped after a whole step, the grid was laid out again and
                              the next call continues (mw_step does this by itself) */
} mw_status;

/* MW_NPT: isothermal-isobaric dynamics, a Nose-Hoover thermostat (T0, tau)
 * and an isotropic barostat (p_ext, tau_p) in the Martyna-Tobias-Klein form,
 * the paper's constant-pressure runs of Sec. II.B-C (1 atm; the box is
 * cubic or orthorhombic and scales by one factor in all three edges).  Each
 * box of a batch has its own barostat.  Conserved: ke + pe + Q xi^2/2 +
 * N_df kB T0 eta + p_ext V + pe_b^2/(2 W), with Q = N_df kB T0 tau^2 and
 * W = (N_df + 3) kB T0 tau_p^2. */
typedef enum mw_thermostat { MW_NVE = 0, MW_BERENDSEN = 1, MW_NOSE_HOOVER = 2, MW_NPT = 3 } mw_thermostat;

/* How mw_step launches work.  GRAPH: one kernel per phase, one step captured
 * in a CUDA graph and replayed.  PERSISTENT: one cooperative launch runs many
 * steps with grid-wide barriers between phases.  AUTO: the library picks
 * (the autotuner's choice when one was made, else PERSISTENT).  PLAIN: the
 * plain GPU path the others are measured against: every phase kernel
 * launched from the host every step (no graph, no persistent launch) and a
 * force kernel with one thread per atom looping over its leg pairs (leg
 * forces scattered with red.global, no lane groups, no shared-memory leg
 * table, no moment form); it is also the force kernel of mw_energy_forces
 * and mw_forces_async while selected.  One species only; the autotuner
 * never picks it.  For the one-box-per-launch baseline of a batch, step one
 * single-box system per box. */
typedef enum mw_engine { MW_ENGINE_AUTO = 0, MW_ENGINE_GRAPH = 1, MW_ENGINE_PERSISTENT = 2, MW_ENGINE_PLAIN = 3 } mw_engine;

/* Integrator settings for mw_step (Sec. II.B: dt = 10 fs, tau_T = 1 ps). */
typedef struct mw_integrator {
  double dt;                /* fs, > 0 */
  int thermostat;           /* mw_thermostat */
  double T0;                /* K, target temperature of every box ... */
  const double* T0_per_box; /* ... unless this host array of nbox targets is non-NULL */
  double tau;               /* fs, thermostat relaxation time (> 0 unless NVE) */
  double p_ext;             /* atm, target pressure (MW_NPT only) */
  double tau_p;             /* fs, barostat period (MW_NPT only, > 0) */
} mw_integrator;

/* Per-box thermodynamic snapshot at the end of the last completed step. */
typedef struct mw_thermo {
  int64_t step;       /* steps completed since the last mw_set_state */
  double pe, e2, e3;  /* potential energy and its two- and three-body parts, kcal/mol */
  double ke;          /* kinetic energy, kcal/mol */
  double temperature; /* K, 2 ke / (Ndf kB), Ndf = 3 n - 3 */
  double conserved;   /* ke + pe (+ Q xi^2/2 + Ndf kB T0 eta under Nose-Hoover and MW_NPT;
                         + p_ext V + pe_b^2/(2 W) under MW_NPT) */
  double pressure;    /* atm, (2 ke + tr W) / (3 V) */
  double virial[6];   /* xx yy zz xy xz yz, kcal/mol: sum over terms and legs of d_a F_b */
  double xi, eta;     /* Nose-Hoover thermostat velocity (1/fs) and position */
  int64_t rebuilds;   /* neighbour-list rebuilds of this box since mw_set_state */
  double volume;      /* A^3, the box during that step */
  double box[3];      /* A, its edges (they change only under MW_NPT) */
} mw_thermo;

typedef struct mw_info {
  int nbox;
  int n_total;
  int nbr_width;      /* slots per atom in the neighbour list */
  int max_count;      /* widest neighbour set at the last build */
  int ncell_total;    /* cells over all boxes */
  int engine;         /* engine mw_step used last (mw_engine) */
  int persistent_blocks, persistent_threads;
  double r_list;      /* a sigma + skin, A */
  int64_t npairs, ntriplets; /* legs r < a sigma (unordered pairs) and triplets at the last force call */
  int64_t rebuild_steps;     /* steps and force calls that rebuilt at least one box since mw_set_state */
  int64_t regrids;           /* cell grids laid out again because an MW_NPT box left its grid */
  int species;               /* species of the potential (1 unless mw_set_species set more) */
  int species_moments;       /* 1: the species table factors into leg weights and the moment kernel runs */
  int force_lanes;           /* launch shape of the per-phase force kernel: lanes per centre atom ... */
  int force_blocks_per_sm;   /* ... and the co-resident blocks per SM its register budget allows */
  int force_owner;           /* 1: owner-computes (two passes, no per-leg scatter); 0: red.global scatter */
  int pad_;
} mw_info;

typedef struct mw_system mw_system;

/* Fills *out with the mW parameters of Sec. II.A / II.D. */
mw_status mw_params_default(mw_params* out);

/* Creates a one-box system of n >= 2 atoms in the orthorhombic box
 * box[0..2] (A), every edge >= 2 (a sigma + skin).  mass in g/mol
 * (18.015 for water, Sec. II.C), skin >= 0 in A (Verlet-list skin; the
 * list is rebuilt once an atom has moved more than skin/2).  stream is a
 * cudaStream_t on which all work of this system is enqueued (it must
 * outlive the system); NULL makes the library create and own a
 * non-blocking stream.  Allocates device memory. */
mw_status mw_system_create(mw_system** out, int n, const double box[3], const mw_params* prm, double mass,
                           double skin, void* stream);

/* Creates a batch of nbox independent boxes: n[b] atoms (>= 2) in the box
 * box[3b..3b+2].  Same rules as mw_system_create per box. */
mw_status mw_batch_create(mw_system** out, int nbox, const int* n, const double* box, const mw_params* prm,
                          double mass, double skin, void* stream);

/* Frees every device and host resource of s (NULL is a no-op). */
mw_status mw_system_destroy(mw_system* s);

/* Sets positions x (n_total*3, required, any finite values: they are
 * wrapped into the box) and velocities v (n_total*3, or NULL for zero), host
 * arrays.  Resets the step counter and the thermostat (xi = eta = 0).  A
 * non-finite value (checked on the device, for host and device inputs alike)
 * gives MW_EINVAL and leaves the system without a state.
 * When the system already holds a state whose forces were evaluated, its
 * atom order and neighbour lists are kept: the arrays are copied to device
 * staging buffers by DMA and loaded through the kept order, and only boxes
 * with an atom more than skin/2 from its list position are marked for a
 * rebuild (not under MW_NPT).  With host velocities this path also makes the
 * force call at the new positions that the next step or energy call would
 * make, while the velocities are copied in (so it can return the errors of a
 * force call, MW_ENLIST_OVERFLOW and the like).  Otherwise the atoms take the caller's order
 * and every list is marked stale; page-locked host arrays (cudaMallocHost,
 * cudaHostAlloc, cudaHostRegister) are then read in place by the loading
 * kernel, pageable ones copied to staging first.  Either way the arrays are
 * read completely before the call returns, and the caller keeps them. */
mw_status mw_set_state(mw_system* s, const double* x, const double* v);
/* Same with device arrays. */
mw_status mw_set_state_dev(mw_system* s, const double* x_dev, const double* v_dev);

/* Copies the current positions (wrapped into [0, L)) and velocities to host
 * arrays of n_total*3 doubles in the caller's atom order; either may be NULL. */
mw_status mw_get_state(mw_system* s, double* x, double* v);
mw_status mw_get_state_dev(mw_system* s, double* x_dev, double* v_dev);

/* Unwrapped positions (host array of n_total*3 doubles, caller's order): the
 * wrapped position plus the periodic images each atom has crossed along each
 * axis since mw_set_state (which counts the images of the positions it was
 * given, so a position outside the box comes back as given).  For mean-square
 * displacements and the diffusion coefficient (Sec. II.C). */
mw_status mw_get_unwrapped(mw_system* s, double* x);

/* Replaces the potential parameters (the neighbour list is marked stale:
 * its radius a sigma + skin follows sigma). */
mw_status mw_set_params(mw_system* s, const mw_params* prm);

/* Several species (Sec. IV: mW with solutes of their own lambda, epsilon,
 * sigma; the SW family of Fig. 2 mixed).  table: nt^3 parameter sets, entry
 * (a, b, c) at index (a nt + b) nt + c; types: n_total species in [0, nt),
 * caller's atom order (host array, copied).  The pair term of atoms of
 * species a and b uses entry (a, b, b), which must equal (b, a, a) in
 * epsilon, sigma, a, A, B, p and q.  The three-body term of a centre of
 * species a with legs to species b and c uses lambda, epsilon and
 * cos_theta0 of entry (a, b, c), which must equal (a, c, b), and for each
 * leg the gamma, sigma and a of that leg's pair entry.  1 <= nt <=
 * MW_MAX_SPECIES; nt = 1 is mw_set_params(table[0]) (types unused).  The
 * list radius becomes the largest a sigma + skin.  One mass for all atoms.
 * When lambda epsilon of every (a, b, c) is h_ab h_ac (h_ab = sqrt(lambda
 * epsilon) of (a, b, b), to 1e-9 relative: geometric-mean mixing, a solute
 * with lambda = 0) and cos_theta0 depends on the centre's species alone, the
 * one-species moment kernel runs with per-leg constants; otherwise a kernel
 * that walks every leg pair of each centre (several times slower).  While
 * nt > 1, mw_step uses the graph engine and mw_energy_forces_vjp returns
 * MW_EINVAL.  Calling mw_set_params returns to one species. */
#define MW_MAX_SPECIES 8
mw_status mw_set_species(mw_system* s, int nt, const mw_params* table, const int* types);

/* Forces a cell binning + neighbour-list rebuild now; *max_count_out (may be
 * NULL) receives the widest neighbour set.  Grows the list if needed.
 * Defining passage: Sec. II.A, where every term of the energy vanishes beyond
 * r = a sigma, so the pair sum and the three-body sum over leg pairs (j, k)
 * of a centre i only need the atoms within a sigma of i; the list holds
 * every atom within a sigma + skin (the skin is a build choice, not in the
 * paper), cell-binned by a counting sort over cells at least that wide. */
mw_status mw_build_neighbors(mw_system* s, int* max_count_out);

/* Copies the neighbour sets of the last build, in the caller's atom order:
 * counts[n_total] and nbr[n_total*width] (host; entries beyond counts[i] are
 * left untouched; sets wider than width are truncated, counts stay exact).
 * Neighbour j of atom i is any atom with |d_ij|^2 < r_list^2 evaluated in
 * FP32 on the device, at the positions of the last build. */
mw_status mw_get_neighbors(mw_system* s, int* counts, int* nbr, int width);

/* Energy, forces and virial at the current positions (rebuilding the
 * neighbour list first if it is stale).  Defining passage: Sec. II.A, the
 * total energy E = sum over pairs of phi2 plus the sum over centres i and leg
 * pairs j < k of phi3 with the angle at i; forces F_i = -dE/dx_i; the virial
 * sum over terms and legs of d_a F_b is what the pressure tensor of the
 * surface-tension formula of Sec. II.C needs.  Host outputs, each may be NULL:
 * f[n_total*3] (kcal/mol/A), energy[nbox*3] = (E, E2, E3) per box,
 * virial[nbox*6].  Pair and triplet arithmetic is FP32; energy and virial
 * are reduced in FP64. */
mw_status mw_energy_forces(mw_system* s, double* f, double* energy, double* virial);

/* Device variant: x_dev (n_total*3 doubles, or NULL to keep the current
 * positions) replaces the positions first; f_dev receives n_total*3 floats;
 * energy_dev[nbox*3] and virial_dev[nbox*6] doubles; any output may be NULL. */
mw_status mw_energy_forces_dev(mw_system* s, const double* x_dev, float* f_dev, double* energy_dev,
                               double* virial_dev);

/* Enqueues one force evaluation (zero the forces, fused two- + three-body
 * kernel) at the current positions with the current neighbour list on the
 * system's stream and returns without synchronising; for timing the force
 * kernel on its own (the neighbour list is built first if it is stale). */
mw_status mw_forces_async(mw_system* s);

/* Advances every box nsteps velocity-Verlet steps.  Defining passage:
 * Sec. II.B, MD with a 10 fs step (5 fs for interfaces), Nose-Hoover
 * thermostat with a 1 ps relaxation time and barostat with 2.5 ps (MW_NPT);
 * the integrator is velocity Verlet (the paper names LAMMPS, whose default
 * it is).  On a system made by mw_batch_create this call is the batched
 * step: every box advances in the same launches (there is no separate
 * mw_batch_step).  last (may be NULL) receives nbox thermo records after the
 * final step.  Recovers internally
 * from neighbour-list overflow (grows the list and resumes the interrupted
 * step); returns MW_ENAN / MW_ELOST / MW_ETIMEOUT if dynamics broke down (the
 * state is then left at the failing step). */
mw_status mw_step(mw_system* s, const mw_integrator* integ, int nsteps, mw_thermo* last);

/* Enqueues nsteps steps on the system's stream and returns without waiting.
 * No overflow recovery happens here: a failure (list overflow, NaN, lost
 * atom) freezes the state at the failing step and is returned by the next
 * mw_sync (or any synchronising call). */
mw_status mw_step_async(mw_system* s, const mw_integrator* integ, int nsteps);

/* Waits for the system's stream; returns the device-side status of the work
 * enqueued so far. */
mw_status mw_sync(mw_system* s);

/* Checkpoint / resume.  A checkpoint is the exact engine state (64-bit box
 * fractions, FP32-pair velocities, image counters, the forces of the last
 * evaluation, atom ids and species in the current cell order, every box's
 * geometry and thermostat / barostat state, the step count, the
 * integrator), so a run resumed from it continues the saved trajectory as
 * an uninterrupted run would (to the run-to-run spread of the GPU's
 * unordered FP32 force sums; a plain mw_set_state restarts the thermostat).
 * mw_checkpoint_size gives the bytes of the caller-owned buffer that
 * mw_checkpoint_save fills.  mw_checkpoint_load requires a system with the
 * same atom counts, boxes and species, the same parameters (and species
 * table), mass and skin, and a blob from the same library build (structure
 * sizes are checked); MW_EINVAL otherwise.  The neighbour list is rebuilt
 * at the next step. */
mw_status mw_checkpoint_size(mw_system* s, size_t* bytes);
mw_status mw_checkpoint_save(mw_system* s, void* buf, size_t bytes);
mw_status mw_checkpoint_load(mw_system* s, const void* buf, size_t bytes);

/* Phase marks of the persistent engine (tracing): with cap > 0, block 0 of
 * each persistent launch records the SM clock (clock64, cycles) at up to 16
 * points of each of its first cap steps: 0 step start, 1 kick1 done, 2 its
 * grid barrier passed, 3 rebuild done, 4 force done, 5 its barrier passed,
 * 6 kick2 done, 7 the last barrier passed (on a launch's last step, which
 * ends without that barrier: block 0's arrival); on rebuild steps also 8
 * binning, 9 local scan, 10 scan offsets, 11 scatter, 12 copy-back, 13
 * neighbour lists done (each before its barrier); unused slots hold 0.
 * mw_get_phase_marks copies cap x 16 values of the last launch (host array).
 * cap = 0 turns the marks off (the default). */
mw_status mw_set_phase_marks(mw_system* s, int cap);
mw_status mw_get_phase_marks(mw_system* s, unsigned long long* out, int cap);

/* Limit (seconds, 0..60; default 2) of every device-side wait of the
 * persistent engine (its grid barriers).  A wait that runs out sets
 * MW_ETIMEOUT and the kernel returns; the state of the interrupted step is
 * then undefined (set a state again), the context stays usable.  A limit of
 * 0 makes the first barrier of the next persistent launch give up at once,
 * which is how the timeout path is tested without a GPU fault. */
mw_status mw_set_wait_limit(mw_system* s, double seconds);

/* Thermo records (nbox) of the last completed step, or of the state just set. */
mw_status mw_get_thermo(mw_system* s, mw_thermo* out);

/* Current edges of every box (nbox * 3 doubles, A): those given at creation
 * unless an MW_NPT run has scaled them.  Positions passed to mw_set_state are
 * taken in these boxes. */
mw_status mw_get_box(mw_system* s, double* box);

/* Adjoint of the forces at the current positions (no counterpart in the
 * paper, whose Sec. II.D tunes lambda, epsilon, sigma by scans).  Given
 * w = dL/dF (device, n_total*3 floats, caller's order), writes
 *   dL_dx_dev[n_total*3] (device floats) = sum_i w_i . dF_i/dx
 *                                         = -(H w), H the Hessian of E;
 *   dL_dtheta[nbox*3] (host doubles, may be NULL) = sum_i w_i . dF_i/d(lambda, epsilon, sigma)
 *   per box.
 * The forward leg and triplet quantities are recomputed, not stored.
 * The neighbour list must be current (call mw_energy_forces first). */
mw_status mw_energy_forces_vjp(mw_system* s, const float* dL_dF_dev, float* dL_dx_dev, double* dL_dtheta);

/* Selects the engine mw_step uses (mw_engine).  MW_ENGINE_PLAIN is refused
 * (MW_EINVAL) while several species are set, and mw_set_species refuses
 * several species while it is selected. */
mw_status mw_set_engine(mw_system* s, int engine);

/* Sets the neighbour-list width (slots per atom, >= 1) and marks the list
 * stale; a width too small is grown again on the next build.  The library's
 * own widths (at creation, on growth, after autotuning) are multiples of 32
 * slots, whole 128-byte lines per row. */
mw_status mw_set_nbr_width(mw_system* s, int width);

/* Sets the Verlet-list skin (A, >= 0): the list radius is a sigma + skin and
 * the list is rebuilt once an atom has moved more than skin/2.  A pure
 * performance parameter (results agree to round-off).  Fails with MW_EBOX if
 * a box edge would be shorter than 2 (a sigma + skin). */
mw_status mw_set_skin(mw_system* s, double skin);

/* Autotuner.  First the launch shape of the per-phase force kernel: each
 * shape (lanes per centre x register budget: 4 x 8, 2 x 8, 8 x 8 and 4 x 7
 * blocks per SM with red.global scatter, and 4 x 8 owner-computes; see
 * mw_set_force_shape) is timed over 10 force calls on the current state and
 * the fastest kept.  Then it runs `steps` steps for each candidate configuration
 * - engine (graph / persistent), skin (0.7x, 1x, 1.4x, 1.8x, 2.2x, 2.6x the
 * current one) and persistent grid size - each from the same saved state
 * (positions, velocities and thermostat state are restored exactly between
 * candidates and at the end), keeps the fastest by GPU time as the AUTO
 * engine and the skin, and writes it to *best_engine (may be NULL).  The
 * choice is cached per device name and system signature in the text file
 * named by the environment variable MW_AUTOTUNE_CACHE, when set.  The
 * persistent engine's force phase keeps its own shape (4 lanes per centre,
 * the register budget of the cooperative kernel). */
mw_status mw_autotune(mw_system* s, const mw_integrator* integ, int steps, int* best_engine);

/* Sets the launch shape of the per-phase force kernel: lanes per centre,
 * blocks per SM and the way the three-body force on a leg's partner reaches
 * it.  owner_computes = 0: the centre scatters it with red.global (shapes
 * 4/8, 2/8, 8/8, 4/7); 1: owner-computes in two passes (4/8 only): pass 1
 * stores each centre's moments and legs, pass 2 gives every atom the forces
 * of its own terms and of its neighbours' terms (from their moments), with no
 * per-leg scatter.  MW_EINVAL for a shape not built; selecting
 * owner-computes allocates its buffers (~150 B per atom).  Results agree to
 * rounding; the autotuner times all five. */
mw_status mw_set_force_shape(mw_system* s, int lanes_per_centre, int blocks_per_sm, int owner_computes);

mw_status mw_get_info(mw_system* s, mw_info* out);

/* Diagnostics: advances nsteps steps with every phase kernel launched on its
 * own (no graph) between CUDA events, and writes the mean GPU time per step
 * of each phase to ms_out[8] (ms): kick1 + drift + rebuild check, cell
 * binning, scan, scatter, copy-back, neighbour list, force, kick2 +
 * thermostat.  The rebuild phases return at once on steps without a rebuild,
 * so their mean includes those launches. */
mw_status mw_phase_times(mw_system* s, const mw_integrator* integ, int nsteps, double* ms_out);

/* Diagnostics: when on != 0 the force kernels count legs (pairs with
 * r < a sigma) and triplets into mw_info.npairs / .ntriplets (device atomics,
 * slower; the counts feed the roofline arithmetic). */
mw_status mw_set_count_terms(mw_system* s, int on);

/* ---- Structure analysis (Sec. II.C) -----------------------------------
 * Of the current positions.  Both calls first build the neighbour list at
 * these positions (so every pair within the list radius a sigma + skin is
 * seen; a pending half-kick is applied first and the forces are recomputed
 * before the next step), then count on the GPU.  Counts are per box,
 * row-major hist[box * nbins + bin], host arrays the caller owns.
 *
 * Pair histogram, the raw count behind g(r): the ordered pairs (i, j), i != j,
 * of one box with bin * dr <= r_ij < (bin + 1) * dr (minimum image, FP32
 * distance from the fixed-point positions).  g(r) in bin k is
 * hist[k] V / (N^2 4 pi r^2 dr) at the bin's centre r, and the coordination
 * number within R_c the sum of hist up to R_c divided by N.  Needs dr > 0,
 * 1 <= nbins <= 4096 and nbins * dr <= a sigma + skin (MW_EINVAL otherwise,
 * naming the radius: raise the skin with mw_set_skin to reach further). */
mw_status mw_pair_histogram(mw_system* s, double dr, int nbins, unsigned long long* hist);

/* Angle histogram, the raw count behind the angular distribution function:
 * for each atom k its nc nearest neighbours (2 <= nc <= 16), the angle
 * theta_ikj at k for every ordered pair i != j of them, binned over
 * [0, 180] degrees in nbins equal bins (180 itself in the last);
 * nc (nc - 1) counts per atom.  Fails with MW_EINVAL if an atom has fewer
 * than nc neighbours within the list radius (raise the skin). */
mw_status mw_angle_histogram(mw_system* s, int nc, int nbins, unsigned long long* hist);

/* ---- For callers that cannot allocate device memory ----------------------
 * The paper has no counterpart to this call; it exists for callers that may
 * not call cudaMalloc (an application that owns every device allocation, a
 * plugin inside a fixed memory pool, a process whose footprint is fixed up
 * front).  It computes what mw_energy_forces_dev computes, for ONE box of
 * n <= MW_NOALLOC_MAX_ATOMS atoms with at most MW_NOALLOC_MAX_CELLS cells
 * (box edge / (a sigma + skin), rounded down, multiplied over the three
 * axes) and at most MW_NOALLOC_MAX_WIDTH neighbours per atom within
 * a sigma + skin, and it allocates nothing: all scratch lives in one static
 * device array of MW_NOALLOC_SCRATCH_BYTES that every GPU loading this
 * library holds until the process exits.
 *   x_dev       device, n*3 doubles (A, AoS, caller's order; wrapped into the box)
 *   f_dev       device, n*3 floats out (kcal/mol/A), or NULL
 *   energy_dev  device, 3 doubles out: E, E2, E3 (kcal/mol), or NULL
 *   virial_dev  device, 6 doubles out: xx yy zz xy xz yz (kcal/mol), or NULL
 *   stream      cudaStream_t the work is enqueued on (NULL = legacy default);
 *               the call synchronises it before returning.
 * Larger inputs are rejected with MW_EINVAL (atoms or cells) or
 * MW_ENLIST_OVERFLOW (neighbours), with a message naming the limit; a
 * non-finite coordinate gives MW_EINVAL and leaves the outputs untouched.
 * Positions are converted exactly as mw_set_state converts them, so both
 * entry points see the same coordinates.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process (a cudaDeviceReset in between is not supported).  Every
 * call ends by reading a status word back and synchronising the stream, so
 * no call may be made on a stream that is being captured (MW_EINVAL).  Every
 * call reuses the same array: calls whose GPU work can overlap (e.g. on two
 * unordered streams) race and must not be made. */
#define MW_NOALLOC_MAX_ATOMS 16384
#define MW_NOALLOC_MAX_WIDTH 64
#define MW_NOALLOC_MAX_CELLS 16384
#define MW_NOALLOC_SCRATCH_BYTES (6u << 20)
mw_status mw_energy_forces_noalloc(int n, const double box[3], const mw_params* prm, double skin,
                                   const double* x_dev, float* f_dev, double* energy_dev, double* virial_dev,
                                   void* stream);

/* Message describing the last failure on the calling thread ("" if none). */
const char* mw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MW_H */
