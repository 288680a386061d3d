/*
 * md.h — C ABI of surfmd: constrained Langevin molecular dynamics on implicit
 * surfaces, one GB300 GPU (sm_103a).
 *
 * Method (Paquay & Kusters, "A method for molecular dynamics on curved
 * surfaces"):
 *   - Constrained Hamiltonian, Eq. (1); equations of motion Eqs. (2)-(4):
 *       dx/dt = p/m,  dp/dt = f - lambda * n,  n = grad g (unnormalised).
 *   - Algorithm 1 (RATTLE for particles on manifolds): a position half that
 *     solves for (x^{m+1}, lambda) by Newton iteration and a momentum half that
 *     solves for (p^{m+1}, mu) so that n(x^{m+1}) . p^{m+1} = 0.
 *   - Algorithm S1 (RATTLE with the Gronbech-Jensen/Farago Langevin form):
 *       f_r^{n+1} = sqrt(2 m kT / (tau dt)) * (r_x, r_y, r_z),  r ~ N(0,1)
 *       F^{m+1}   = [f^{m+1} - p^{m+1/2}/tau + (f_r^{n+1} + f_r^n)/2] / (1 + dt/(2 tau))
 *     followed by the momentum half of Algorithm 1 with F^{m+1}.
 *   - Pair potential: truncated and shifted Lennard-Jones, Eq. (S1); WCA is
 *     the cut at 2^{1/6} sigma (Section 3.2).
 *   - Harmonic bond V = k (r - r0)^2 (no factor 1/2) and the repulsive
 *     Lennard-Jones wall V_w (SI Section S3.2, virus capsid set-up).
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status (MD_OK = 0 or an MD_ERR_* code).
 *     md_last_error() returns a NUL-terminated description of the last
 *     failure on that handle (owned by the handle, valid until the next call).
 *   - Host arrays passed in are owned by the caller and are copied during the
 *     call; host arrays passed out are written during the call. Device
 *     pointers (the *_device variants) must point to memory on the handle's
 *     device and stay valid until the call returns.
 *   - The library owns every device buffer it allocates; md_destroy frees
 *     them. All GPU work is enqueued on the handle's stream (md_set_stream).
 *   - Per-particle arrays are in user order. In a batch (md_create_batch) the
 *     systems are concatenated in system order: system s owns particles
 *     [off_s, off_s + n_s), off_s = n_0 + ... + n_{s-1}.
 *   - Positions/velocities/forces are row-major [n][3] float64 (x, y, z of
 *     particle 0, then particle 1, ...).
 *   - Units are Lennard-Jones units (sigma, epsilon, m, tau_LJ).
 *
 * Error behaviour
 *   - Argument errors are detected on the host before any GPU work and return
 *     MD_ERR_INVALID_ARG with the state unchanged.
 *   - Errors raised inside kernels (Newton non-convergence, non-finite
 *     values, a particle leaving the cell grid) are latched in a device status
 *     word and reported by the next synchronising call (md_sync, md_get_state,
 *     md_forces, md_constraint_residual, md_observables). The status word is
 *     cleared when it is reported. The kernels never trap and never spin
 *     without a bound.
 */
#ifndef SURFMD_MD_H
#define SURFMD_MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MD_OK                  0
#define MD_ERR_INVALID_ARG     1  /* bad argument; nothing was changed            */
#define MD_ERR_CUDA            2  /* a CUDA runtime call failed                    */
#define MD_ERR_RATTLE_DIVERGED 3  /* Newton of Algorithm 1 missed the tolerance    */
#define MD_ERR_NONFINITE       4  /* NaN/Inf in a position or momentum             */
#define MD_ERR_OUT_OF_GRID     5  /* a particle left the cell grid of its system   */
#define MD_ERR_TIMEOUT         6  /* a bounded device-side wait ran out            */
#define MD_ERR_NO_DEVICE       7  /* no CUDA device is visible                     */
#define MD_ERR_NLIST_FULL      8  /* a particle had more neighbours than the Verlet
                                     list holds (md_set_neighbor_list)              */

/* Bits of the device status word (md_status); a set bit maps to the code
 * given beside it, lowest code first. */
#define MD_FLAG_RATTLE_DIVERGED 0x1u
#define MD_FLAG_NONFINITE       0x2u
#define MD_FLAG_OUT_OF_GRID     0x4u
#define MD_FLAG_TIMEOUT         0x8u

#define MD_MAX_TYPES 8

/* ---- surfaces g(x) = 0 ------------------------------------------------- */
/* The constraint function g and its unnormalised gradient n = grad g.
 *   PLANE      g = a(x-x0) + b(y-y0) + c(z-z0), p = (a, b, c)   (SI S3.1)
 *   SPHERE     g = |x-c|^2 - R^2,                p[0] = R        (Eq. 1 text)
 *   ELLIPSOID  g = sum_d (x_d-c_d)^2 / p[d]^2 - 1, p = semi-axes
 *   TORUS      g = (rho - R)^2 + (z-c_z)^2 - r^2, rho = |(x-c_x, y-c_y)|,
 *              p = (R, r); the connector form of SI S3.1 with its axis on z
 *   GAUSSIAN_BUMP  g = (z-c_z) - A exp(-rho^2 / (2 w^2)), p = (A, w); rho is
 *              taken with the minimum image in periodic x, y
 *   CYLINDER   g = sum_{d != axis} (x_d-c_d)^2 - R^2, p = (R, axis 0|1|2)
 *              (SI S3.1 with the axis coefficient 0 and the others 1)
 *   THYLAKOID  the composite of SI S3.1, p = (R_b, L_x, R_c, L_b): a bridge
 *              cylinder (radius R_b, length L_b) along x through (c_y, c_z),
 *              toroidal connectors (tube radius R_c) joining it to the face
 *              planes of two blocks at x = c_x -/+ (L_b/2 + R_c), each block
 *              a tube along z with a square section of side L_x + 2 R_c and
 *              corners rounded by quarter cylinders of radius R_c; needs
 *              periodic z and open x, y. A particle's piece is chosen where
 *              its half step starts and held for that solve.
 *   XY2D       no constraint: particles move in the plane z = c_z with the
 *              z components of force, noise and momentum dropped (the
 *              unconstrained 2D baseline of Section 3.1's performance
 *              comparison); needs periodic x and y; 2 degrees of freedom
 * The Newton stopping test works on |g| / |grad g|, a length, so one
 * tolerance means the same thing on every surface. */
typedef enum {
  MD_SURF_NONE = 0,
  MD_SURF_PLANE = 1,
  MD_SURF_SPHERE = 2,
  MD_SURF_ELLIPSOID = 3,
  MD_SURF_TORUS = 4,
  MD_SURF_GAUSSIAN_BUMP = 5,
  MD_SURF_CYLINDER = 6,
  MD_SURF_XY2D = 7,
  MD_SURF_THYLAKOID = 8
} md_surface_kind;

typedef struct md_surface {
  int32_t kind;      /* md_surface_kind                                    */
  int32_t reserved;  /* must be 0                                          */
  double center[3];  /* (x0, y0, z0) of the plane / centre of the others   */
  double p[4];       /* shape parameters, see above                        */
} md_surface;

/* ---- parameters of one system ------------------------------------------ */
#define MD_PREC_FP64  0  /* every step in float64                              */
#define MD_PREC_MIXED 1  /* float32 pair forces and noise; float64 state,
                            Newton solve, projection and position update      */

/* Pair potential forms, phi(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6], both 0
 * for r >= rcut:
 *   MD_PAIR_TRUNC_SHIFT    V = phi(r) - phi(rcut)                  (Eq. S1)
 *   MD_PAIR_LINEAR_SMOOTH  V = phi(r) - phi(rcut) - (r - rcut) phi'(rcut),
 *     the linearly smoothed potential of the SI energy-conservation study,
 *     whose energy and force are both continuous at rcut (the SI prints the
 *     linear term with a plus sign, under which the force would not vanish
 *     at rcut; the sign here is the one that gives the stated continuity). */
#define MD_PAIR_TRUNC_SHIFT 0
#define MD_PAIR_LINEAR_SMOOTH 1

#define MD_WALL_PLANES 0
#define MD_WALL_SPHERE 1

typedef struct md_params {
  double dt;            /* time step                                          */
  double kT;            /* thermal energy                                     */
  double gamma;         /* 1/tau, Langevin friction rate; 0 gives NVE          */
  double rattle_tol;    /* eta: stop when |g|/|grad g| < eta (length units)   */
  int32_t max_newton;   /* iteration cap of the position half (e.g. 30)        */
  int32_t frozen_normal;/* 1: keep n = grad g(x^m) in the Newton Jacobian     */
  int32_t precision;    /* MD_PREC_FP64 | MD_PREC_MIXED                        */
  int32_t ntypes;       /* 1..MD_MAX_TYPES                                     */
  double mass[MD_MAX_TYPES];
  double eps[MD_MAX_TYPES][MD_MAX_TYPES];    /* symmetric                    */
  double sigma[MD_MAX_TYPES][MD_MAX_TYPES];  /* symmetric                    */
  double rcut[MD_MAX_TYPES][MD_MAX_TYPES];   /* symmetric; 0 = no pair term  */
  double box_lo[3];     /* cell-grid bounds; periodic dims wrap at these      */
  double box_hi[3];     /* all zero: bounds derived from the surface          */
  int32_t periodic[3];  /* 1 = periodic along that axis                       */
  int32_t beads_per_mol;/* > 1: particles [k*B, (k+1)*B) of a system form one
                           linear chain with harmonic bonds between neighbours */
  double bond_k;        /* V = bond_k (r - bond_r0)^2                         */
  double bond_r0;
  int32_t exclude_intramol; /* 1: no pair term between beads of one molecule  */
  int32_t wall_enable;  /* 1: V_w on the unconstrained particles (wall_kind)  */
  double wall_lo_z, wall_hi_z, wall_eps, wall_sigma;
  uint64_t seed;        /* Philox key word 0 = low 32 bits of seed            */
  uint32_t replica;     /* Philox key word 1                                  */
  int32_t pair_form;    /* MD_PAIR_TRUNC_SHIFT or MD_PAIR_LINEAR_SMOOTH        */
  double cell_size;     /* 0: largest rcut (plus a 2^-12 relative margin)     */
  /* Capsid-model terms (SI Section S3.2); all zero: none.                  */
  double angle_k;       /* V_bend = angle_k (theta - angle_theta0)^2 on every
                           three consecutive beads i, j, k of a chain, theta
                           the angle at j between x_i - x_j and x_k - x_j
                           (pi for a straight chain); needs beads_per_mol >= 3 */
  double angle_theta0;
  int32_t bond_r0_mix;  /* 1: bond rest length 2^{1/6} sigma[t_i][t_j] / 2 from
                           the bonded beads' types (with sigma_ij = (sigma_i +
                           sigma_j)/2 this is the SI's 2^{1/6}(sigma_i +
                           sigma_j)/4); 0: bond_r0 for every bond            */
  int32_t wall_kind;    /* MD_WALL_PLANES: V_w at z = wall_lo_z and wall_hi_z;
                           MD_WALL_SPHERE: V_w(r - wall_radius) with r the
                           distance from wall_center, pushing outwards      */
  double wall_radius;
  double wall_center[3];
} md_params;

/* Per-system observables (Section 3.1: kT = 2K/N_dof with 2 degrees of
 * freedom per constrained and 3 per free particle; MSD closed forms of
 * SI Section S1.3). */
typedef struct md_obs {
  uint64_t step;
  int64_t n;
  int64_t ndof;
  double kinetic;          /* K = sum p^2 / 2m at the integer step            */
  double potential;        /* U: pair + bond + wall                           */
  double kT;               /* 2 K / ndof                                      */
  double max_g_over_gradg; /* max over constrained particles of |g|/|grad g|  */
  double max_n_dot_v;      /* max |n.v| / |n|                                 */
  double msd;              /* mean |x - x_ref|^2, x unwrapped                 */
  double r0_dot_rt;        /* mean (x_ref-c).(x-c)/R^2 (sphere), else 0      */
} md_obs;

typedef struct md_handle md_handle;

/* Library version, (major << 16) | minor. */
int md_version(void);

/* Create one system of n particles held on `surf` (kind MD_SURF_NONE: all
 * particles free). Allocates all device memory for n particles on the
 * current CUDA device. n = 0 is valid and gives a handle whose steps do
 * nothing. Returns MD_ERR_INVALID_ARG for inconsistent parameters, e.g.
 * dt <= 0, a periodic axis shorter than 3 cells, a bump without periodic x,y. */
int md_create(const md_surface* surf, const md_params* prm, int64_t n,
              md_handle** out);

/* Create nsys independent systems advanced together (ensembles of replicas).
 * surfs[s], prms[s], n_per_sys[s] describe system s. All systems must share
 * precision, ntypes, mass, eps, sigma, rcut, pair_form and cell_size; the
 * other fields may differ. Systems never interact. */
int md_create_batch(int32_t nsys, const md_surface* surfs, const md_params* prms,
                    const int64_t* n_per_sys, md_handle** out);

/* Enqueue all later GPU work on `cuda_stream` (a cudaStream_t, e.g. taken
 * from torch.cuda.current_stream().cuda_stream). NULL = the legacy stream. */
int md_set_stream(md_handle* h, void* cuda_stream);

/* Set the state at step counter step0. x: positions [n][3]; v: velocities
 * [n][3] (NULL = zero); type: [n] in [0, ntypes) (NULL = 0); mol: [n]
 * molecule ids for exclusions (NULL = derived from beads_per_mol);
 * constrained: [n] 0/1 (NULL = 1 where the system has a surface).
 * Each constrained x must satisfy |g|/|grad g| < 1e-6 (else
 * MD_ERR_INVALID_ARG); its velocity is projected on the tangent plane,
 * v <- v - (n.v / n.n) n, before p = m v is stored. The positions also
 * become the reference of md_obs.msd. The first md_step after this call
 * forms F^{step0} = f(x) - gamma p + f_r^{step0}, i.e. Algorithm S1 with no
 * noise average and no 1/(1+dt/2tau) factor on its first force. */
int md_set_state(md_handle* h, const double* x, const double* v,
                 const int32_t* type, const int32_t* mol,
                 const uint8_t* constrained, uint64_t step0);

/* As md_set_state, with x, v and the optional arrays in device memory. */
int md_set_state_device(md_handle* h, const double* d_x, const double* d_v,
                        const int32_t* d_type, const int32_t* d_mol,
                        const uint8_t* d_constrained, uint64_t step0);

/* Restore a checkpoint written by md_get_state: positions x^k, the
 * half-step momenta p^{k-1/2} and the step counter k. Types, molecules and
 * the constrained flags stay as last set. Because the noise is a pure
 * function of (seed, replica, particle, step), a restored run repeats the
 * uninterrupted trajectory bit for bit. */
int md_restore(md_handle* h, const double* x, const double* p_half,
               uint64_t step);

/* Advance every system by nsteps steps of Algorithm S1 (asynchronous: the
 * work is enqueued on the stream; kernel-side errors surface at the next
 * synchronising call). */
int md_step(md_handle* h, int64_t nsteps);

/* Tuning options (they change speed, not results beyond float rounding
 * order). MD_OPT_PAIR_LANES: lanes of a warp that share one particle in the
 * pair kernel: 1 (default: one thread per particle, a z-slab of bucket ranges
 * loaded at a time) or 2, 4, 8 (the 27 cells split over the lanes and the
 * partial forces combined by shuffles). A change takes effect at the next
 * md_step (the captured step is rebuilt). */
#define MD_OPT_PAIR_LANES 1
/* MD_OPT_PAIR_ORDER: 1 (default) = the pair kernel visits particles in a
 * spatial (Morton) order refreshed every 16 steps, so neighbouring threads
 * share cache lines; 0 = bucket order. */
#define MD_OPT_PAIR_ORDER 2
/* MD_OPT_ENGINE: 0 (default) = every step is one graph of five kernels over
 * the whole batch with the cell list in global memory; 1 = resident engine:
 * one persistent launch advances every system many steps, one CTA per
 * system at a time with the system's cell list and forces in shared memory
 * (x and p stay in global memory). Results are bit-identical to engine 0.
 * Needs pair interactions and systems small enough for one CTA's shared
 * memory (at most 65535 particles; about 46 bytes per particle plus 4 per
 * bucket in mixed precision, 78 in float64); md_set_option returns
 * MD_ERR_INVALID_ARG with the reason otherwise. md_step(n) then runs
 * ceil(n / MD_OPT_RESIDENT_STEPS) launches and rebuilds the global cell list
 * of the final positions once, and md_profile_step reports two entries:
 * "resident" (the launches, per step) and "rebuild" (per step of the call). */
#define MD_OPT_ENGINE 3
/* MD_OPT_RESIDENT_THREADS: threads per CTA of the resident engine: 0
 * (default) chooses per size class of the batch (systems grouped by the
 * CTAs their shared memory lets one SM hold; each class its own launch and
 * the CTA size that keeps the most warps resident), or a multiple of 32 in
 * 64..512 for every class. */
#define MD_OPT_RESIDENT_THREADS 4
/* MD_OPT_RESIDENT_STEPS: most steps one resident launch runs (1..100000,
 * default 256); longer md_step calls are split into several launches. */
#define MD_OPT_RESIDENT_STEPS 5
/* MD_OPT_PAIR_TILE: 0 (default) = the pair kernel runs one particle per
 * thread (or MD_OPT_PAIR_LANES lanes per particle); 8, 16 or 32 = cell-tiled:
 * each warp takes that many consecutive sorted particles, split at cell
 * boundaries; for each piece it copies the records of the home cell's
 * 27-cell stencil into shared memory once and the piece's particles share
 * the warp's lanes over that list (MD_OPT_PAIR_LANES and MD_OPT_PAIR_ORDER
 * are then unused). Pays where cells hold several particles (long cutoffs,
 * dense 3D systems); fewer particles per warp give more warps to small
 * systems. Only for handles whose buckets are the cell ids (grids of at most
 * max(2^20, 4N) cells; else MD_ERR_INVALID_ARG). Forces agree with the other
 * settings to float rounding (summation order differs). */
#define MD_OPT_PAIR_TILE 6
/* MD_OPT_NLIST_BUILDS (md_get_option only; waits for the stream): how many
 * times the Verlet list has been built since it was first switched on (by
 * the steps, and by md_set_state, md_restore and switching the list on). */
#define MD_OPT_NLIST_BUILDS 7
/* MD_OPT_SPIN_LIMIT: the one bounded wait on the device, the scan of the
 * bucket counters waiting for its predecessor tiles (decoupled look-back),
 * reads a predecessor's word at most `limit` times (0..2^31-1, default
 * 2^22). When the limit runs out the kernel latches MD_FLAG_TIMEOUT, gives its
 * tile a zero prefix (the cell list of that step is then wrong, every access
 * stays in bounds) and returns; the next synchronising call reports
 * MD_ERR_TIMEOUT and the next md_step rebuilds the cell list from the
 * positions before it steps. With 0 the wait gives up without reading, so a
 * scan of more than one tile (more than 8192 buckets) always times out. */
#define MD_OPT_SPIN_LIMIT 8
/* MD_OPT_PAIR_QUEUE (mixed precision with the Verlet list): 1 (default) = a
 * warp walks its particles' packed list entries as one sequence (their
 * records staged in shared memory a few chunks of 32 at a time), queues the
 * pairs near or inside the cutoff and evaluates 32 queued pairs at a time on
 * all lanes; 0 = each lane walks its particle's list alone. Both add every
 * particle's terms in list order with the same arithmetic: the same bits. */
#define MD_OPT_PAIR_QUEUE 9
/* MD_OPT_FUSED_REBUILD (Verlet-list step form): 1 (default) = the cell-list
 * and list rebuild of a step is one cooperative launch that returns at once
 * unless the rebuild flag is up (three launches per step: pair, integrate,
 * rebuild); 0 = five separate launches (bin, scan, scatter, bucket build,
 * list build), each returning at once without a rebuild. The same lists and
 * the same bits either way. Where a cooperative launch cannot be captured or
 * run, md_step falls back to the separate launches (md_get_option then
 * reads 0). */
#define MD_OPT_FUSED_REBUILD 10
/* MD_OPT_LIST_WARP (mixed precision with the Verlet list, MD_OPT_PAIR_QUEUE =
 * 1): particles per warp of the list walk, 32 (default), 16 or 8. The warp
 * walks its particles' lists as one sequence, 32 entries at a time, so long
 * lists (long cutoffs, dense systems) spread over more warps with fewer
 * particles each. The same bits for every setting. */
#define MD_OPT_LIST_WARP 11
/* MD_OPT_STORE_NOISE (mixed precision with the Verlet list): 1 (default) =
 * the integrator stores the unit normals xi^k it draws for step k (16 bytes
 * per particle) and the next step's force combination, which needs xi^k
 * again beside xi^(k+1), reads them instead of drawing them a second time;
 * 0 = both steps' normals are drawn every step. The stored values are the
 * ones the generator gives, so trajectories are the same bit for bit either
 * way. After md_set_state or md_restore (and after switching the option) the
 * first step draws both. */
#define MD_OPT_STORE_NOISE 12
/* Verlet neighbour list (the LAMMPS-style list the paper's simulations
 * ran with; the cell list is how it is built). With skin > 0 every pair
 * within r_c + skin is listed from the cell list, and the pair kernel walks
 * the list. Between builds each particle keeps its cell and its record
 * moves with it. When any particle has moved more than skin / 2 since the
 * last build, the same step rebuilds the cell list and the list, so every
 * pair within r_c is always listed and forces equal the cell-list path's to
 * float rounding (summation order). max_neighbors bounds the entries per
 * particle (4 bytes each); a build that needs more latches MD_ERR_NLIST_FULL
 * (reported by the next synchronising call; those forces miss pairs).
 * The handle's cell edge must be >= the largest cutoff + skin on every axis
 * with more than one cell (md_params.cell_size), else MD_ERR_INVALID_ARG.
 * skin <= 0 switches the list off. Used by the global engine (md_step,
 * md_forces); the resident engine keeps its own per-step cell lists.
 * Cost: one pair pass over about (r_c + skin)^d / r_c^d times the partners
 * in range. The rebuild kernels (cell list and list) are launched every
 * step and return at once unless a particle has moved skin / 2 (a graph
 * with a conditional rebuild node measured slower: the node and its gate
 * cost more than four early exits). */
int md_set_neighbor_list(md_handle* h, double skin, int32_t max_neighbors);
int md_set_option(md_handle* h, int32_t key, int64_t value);
int md_get_option(md_handle* h, int32_t key, int64_t* value);

/* Wait for the stream and report (then clear) the device status word. */
int md_sync(md_handle* h);

/* Device status bits (MD_FLAG_*) since the last report; synchronises. */
int md_status(md_handle* h, uint32_t* flags);

/* Read the state at the current step counter k: x^k, v^k = p^k/m (the
 * momentum half of step k is evaluated on demand from p^{k-1/2} and the
 * forces at x^k), p^{k-1/2} and k. Any output may be NULL. */
int md_get_state(md_handle* h, double* x, double* v, double* p_half,
                 uint64_t* step);

/* As md_get_state, outputs in device memory (any may be NULL). */
int md_get_state_device(md_handle* h, double* d_x, double* d_v, double* d_p_half);

/* Conservative force f = -grad V (pair + bond + wall) at the current
 * positions, [n][3], and the per-particle potential energy u [n] (pair and
 * bond energies split equally between the two particles). Either may be
 * NULL. In MD_PREC_MIXED the pair part is computed in float32. */
int md_forces(md_handle* h, double* f_out, double* u_out);

/* Constraint residuals at the current step (Section 2.2: g(x)=0 and
 * v.n = 0): max |g|/|grad g|, max |g| and max |n.v|/|n| over constrained
 * particles of all systems. */
int md_constraint_residual(md_handle* h, double* max_g_over_gradg,
                           double* max_abs_g, double* max_n_dot_v);

/* Observables of every system at the current step: out[nsys]. */
int md_observables(md_handle* h, md_obs* out, int32_t max_systems,
                   int32_t* n_written);

/* Counts: total particles, systems, current step. Any output may be NULL. */
int md_info(md_handle* h, int64_t* n, int32_t* nsys, uint64_t* step);

/* Advance nsteps steps launching each kernel of a step on its own (no
 * graph), timed with CUDA events on the handle's stream; kernel_ms[i] is the
 * mean duration of kernel i of a step (i < *n_kernels, names from
 * md_profile_kernel_name). Synchronises. The trajectory is the same as with
 * md_step. */
int md_profile_step(md_handle* h, int64_t nsteps, double* kernel_ms, int32_t max_kernels,
                    int32_t* n_kernels);
const char* md_profile_kernel_name(md_handle* h, int32_t i);

/* Number of kernel launches issued by the last md_step (or md_profile_step)
 * call. */
int md_last_launch_count(md_handle* h, int64_t* launches);

/* Diagnostics of the cell list (the index work of the pair step), for
 * tests. md_grid_info: grid of system `sys`: origin lo[3], cell edge cs[3],
 * cells per axis nc[3] and the id of its first cell (cell ids of system s
 * are base_s + cx + nc0 (cy + nc1 cz), cx = floor((x_wrapped - lo)/cs)).
 * hashed: 0 when a bucket is a cell id, else log2 of the bucket count.
 * md_cell_list: after the last step, sorted_ids[n] lists the particles
 * bucket by bucket, ascending id inside a bucket; sorted_cells[n] their cell
 * ids; bucket_start[nbucket + 1] the bucket ranges. Arrays may be NULL
 * (then only *nbucket is written). */
int md_grid_info(md_handle* h, int32_t sys, double lo[3], double cs[3], int32_t nc[3],
                 uint32_t* base, int32_t* hashed);
int md_cell_list(md_handle* h, uint32_t* sorted_ids, uint32_t* sorted_cells,
                 uint32_t* bucket_start, uint32_t* nbucket);

/* Forces of one system without allocating device memory. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate at
 * the point where they need forces, e.g. an application whose device memory
 * all belongs to its own pool allocator (nothing is left for the driver to
 * hand out), or a caller on a latency-critical path that must not wait on
 * the driver's allocator.
 * It computes f = -grad V (pair, bond and wall terms) and the per-particle
 * energy u at positions d_x, as md_forces does for a handle with the same
 * surface and parameters (within the force tolerance of md_forces: its cell
 * grid and bucket layout may differ, so float32 sums can differ in their
 * last bits), using a scratch array of about 11 MB that the library
 * reserves in device global memory when its device code is loaded (each
 * device that loads the library keeps it until the process exits).
 *   n <= 65536 particles (else MD_ERR_INVALID_ARG); cell grids larger than
 *   2^18 cells use 2^18 hashed buckets.
 *   d_x [n][3] float64, d_f [n][3] float64 (required); d_type, d_mol,
 *   d_constrained, d_u may be NULL (defaults of md_set_state). All pointers
 *   are device memory owned by the caller.
 *   cuda_stream: the stream to work on (NULL = legacy stream, which waits
 *   for every blocking stream of the context: pass a non-blocking stream when
 *   other threads work on the device at the same time). The call waits for
 *   the stream before it returns and reports a particle outside the grid as
 *   MD_ERR_OUT_OF_GRID.
 * The first call on a device resolves the scratch address on that device
 * (and loads the device code if it is not loaded yet); make that first call
 * before any stream capture. While another thread captures a CUDA graph in
 * relaxed or thread-local capture mode, a call on a non-blocking stream runs
 * and gives the same forces; a capture in global mode in another thread
 * forbids the call's synchronising copies (the runtime refuses them and
 * invalidates that capture). Every call shares the one array, which keeps the
 * last call's contents (each call resets what must start at zero): calls that
 * overlap on the GPU (other threads, other streams) race and must be
 * serialised by the caller. Errors of this entry point are read with
 * md_last_error(NULL). */
int md_forces_noalloc(const md_surface* surf, const md_params* prm, int64_t n,
                      const double* d_x, const int32_t* d_type, const int32_t* d_mol,
                      const uint8_t* d_constrained, double* d_f, double* d_u,
                      void* cuda_stream);

/* Diagnostic (no counterpart in the paper): runs on the current device the
 * float64 -> float32 (round to nearest, ties to even) and float32 -> float64
 * format conversions that the mixed-precision kernels perform with integer
 * operations on the IEEE 754 bit fields, so that they can be checked against
 * any IEEE 754 implementation.
 *   in [n] float64, out_f32 [n] = in rounded to float32, out_f64 [n] =
 *   out_f32 widened to float64; all three are host memory owned by the
 *   caller; n >= 0 (n = 0 does nothing).
 * Synchronous; allocates and frees its own device buffers. Errors are read
 * with md_last_error(NULL). */
int md_check_conversions(const double* in, int64_t n, float* out_f32, double* out_f64);

/* Diagnostic (no counterpart in the paper): measured fused multiply-add
 * throughput of the current device, the denominator of the arithmetic
 * rooflines. precision: MD_PREC_FP64 (float64 FMA) or MD_PREC_MIXED (float32
 * FMA). A kernel of 16 CTAs per SM, 256 threads each, runs 8 independent FMA
 * chains per thread; the best of `trials` (>= 1) launches timed with CUDA
 * events gives *fma_per_s (thread FMA instructions per second; 2 flops
 * each). Synchronous; allocates nothing. Errors: MD_ERR_INVALID_ARG for a
 * bad precision, trials or NULL output; MD_ERR_CUDA for a failed launch (read
 * with md_last_error(NULL)). */
int md_measure_fma_peak(int32_t precision, int32_t trials, double* fma_per_s);

/* Description of the last error on h (or of the last md_create failure
 * when h is NULL). Never NULL. */
const char* md_last_error(md_handle* h);

/* Free all device memory of the handle. NULL is ignored. */
void md_destroy(md_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* SURFMD_MD_H */
