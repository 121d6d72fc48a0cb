/*
 * rbc.h -- C ABI of the GB300 (sm_103a) library for the coupled lattice-
 * Boltzmann + rigid red-blood-cell time step of S. Melchionna, "A model for
 * red blood cells in simulations of large-scale blood flows" (2011).
 *
 * One time step h (lattice units, h = 1) advances
 *   - the plasma: D3Q19 BGK streaming and collision with the Hermite
 *     body-force term and a per-node relaxation time (Sec. 2.1,
 *     Eqs. streaming, lbe_discrete, chen_force, dens, vel, stresstensorLB);
 *   - the relaxation time set by the local hematocrit through the smoothed
 *     characteristic function of every cell (Sec. 2.4, Eq. enhance-viscosity);
 *   - the fluid-cell exchange through each cell's diffused shape function:
 *     smeared velocity / vorticity and the elongational torque sampled from
 *     the fluid (Sec. 2.2, Eqs. vel, vort, pheno_torque_diss), the reaction
 *     spread back as a force density (Sec. 2.2, body-force equation);
 *   - Gay-Berne cell-cell and cell-wall forces and torques found through a
 *     device-built cell list (Sec. 2.5, App. B);
 *   - the rigid-body update of every cell (App. A).
 *
 * Conventions.  Lattice node n = x + nx*(y + ny*z), x fastest.  Lattice
 * indices wrap on every axis; walls are solid nodes, and an axis declared
 * non-periodic must have solid end planes.  Quaternions are (w, x, y, z) and
 * map body to lab frame; angular velocities are body-frame.  All host
 * buffers are caller-owned; inputs are copied at rbc_init.
 *
 * Status codes: every function returning int returns one of RBC_OK or a
 * negative RBC_E* code and never aborts; rbc_last_error() describes the last
 * failure of a handle (or of the calling thread when the handle is NULL).
 * The library is single-GPU: it runs on the CUDA device current at rbc_init.
 */
#ifndef RBC_H
#define RBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RBC_OK 0
#define RBC_EINVAL (-1)    /* invalid argument, geometry or parameter */
#define RBC_ENOMEM (-2)    /* workspace too small, or a capacity exceeded */
#define RBC_ECUDA (-3)     /* a CUDA runtime call failed */
#define RBC_EUNSTABLE (-4) /* NaN, or |u| above the Mach guard */
#define RBC_ETIMEOUT (-5)  /* a bounded device wait ran out */

typedef struct rbc_handle rbc_handle;

/* Geometry of the lattice (Sec. 2.1).  solid: host array of nx*ny*nz bytes,
 * 1 = solid node, NULL = all fluid; copied at init.  The external force
 * density at a fluid node (x, y, z) is body_force + body_force_wave *
 * sin(2 pi y / ny) (lattice units): a uniform drive, plus the Kolmogorov
 * profile that sustains a shear flow in a fully periodic box.
 * Open boundaries (the paper drives vessels by an inlet velocity and an
 * outlet pressure, Sec. 4, citing the rules without giving them):
 * node_type (host, nx*ny*nz bytes, NULL = none; copied) marks fluid nodes
 * RBC_NODE_INLET or RBC_NODE_OUTLET.  Boundary nodes are not collided; each
 * pass sets their populations from the previous pass: an inlet node takes
 * f_eq(rho of its neighbour at z + 1, u_in) with u_in = inlet_umax (1 -
 * r^2 / inlet_radius^2) along +z, r the distance of (x, y) from
 * inlet_center; an outlet node takes f_eq(1, u_m) plus the non-equilibrium
 * part of its neighbour m at z - 1.  The neighbour is the node straight
 * across if fluid, else the first fluid one of x - 1, x + 1, y - 1, y + 1 on
 * that plane (oblique vessels).  Cells must stay clear of them. */
typedef struct {
    int nx, ny, nz;
    int periodic[3];
    const uint8_t *solid;
    double body_force[3];
    double body_force_wave[3];
    const uint8_t *node_type;
    double inlet_center[2], inlet_radius, inlet_umax;
} rbc_geometry;

#define RBC_NODE_INTERIOR 0
#define RBC_NODE_INLET 1
#define RBC_NODE_OUTLET 2

/* Initial cell state (Sec. 2.2: Gamma_i = (R_i, Q_i, V_i, Omega_i)).  Host
 * arrays, copied at init: pos 3n (inside the box), quat 4n (need not be
 * normalised), vel 3n or NULL (zero), omega_body 3n or NULL (zero).
 * force_ext, torque_ext: 3n each or NULL (zero), a constant external force
 * and torque (lab frame) on every cell, as the mobility tests of Sec. 3
 * push a single cell; they act like the Gay-Berne forces (they enter the
 * combined force and torque of App. A and are not part of the impulse
 * returned to the fluid) and are reported with them in rbc_cell_diag. */
typedef struct {
    int n;
    const double *pos;
    const double *quat;
    const double *vel;
    const double *omega_body;
    const double *force_ext;
    const double *torque_ext;
} rbc_cells;

/* Model parameters (paper values in brackets; rbc_default_params fills them).
 *   tau0, delta, kappa  Eq. enhance-viscosity [1, 2, 20]
 *   gamma_T, gamma_R    friction rates of App. A [0.1, 0.1]
 *   alpha_tt            elongational torque factor, Eq. pheno_torque_diss [0.04]
 *   eps0                Gay-Berne energy scale, Eq. gayberne [not given; 0.01]
 *   xi[3]               shape-function radii along the body axes [4, 4, 1.5]
 *   semi_axes[3]        Gay-Berne semi-axes (shape matrix S) [4, 4, 1.5]
 *   mass, inertia[3]    M and the diagonal body-frame I [10; 1000, 1000, 1000]
 *   sigma_min_wall      wall-RBC sigma_min (Sec. 2.5) [0.5]
 *   wall_radius         radius of the spherical wall particle [0.5]
 *   rho_floor           lower clamp of the reduced GB distance [0.75]
 *   r_cut, r_cut_wall   candidate radii of the cell-pair / cell-wall search;
 *                       0 derives the Gay-Berne range from the shape
 *   mach_max            |u| guard of the stability flag [0.3]
 *   bin_capacity        cells per cell-list bin [0 = 32]
 *   max_neighbors       candidate partners kept per cell [0 = 64]
 *   precision           storage of the populations (the paper does not fix
 *                       it; Sec. 2.1 keeps f_p per node): RBC_PREC_F32 keeps
 *                       d_p = f_p - w_p in FP32; RBC_PREC_F16 / RBC_PREC_BF16
 *                       keep s_p = d_p S / w_p in IEEE binary16 (S = 1024) /
 *                       bfloat16 (S = 1), halving the population bytes; the
 *                       collision arithmetic is FP32 in every case [F32]
 *   rounding            16-bit stores: RBC_ROUND_STOCHASTIC rounds up with
 *                       probability equal to the fraction of the gap covered
 *                       (six random bits per value from Philox4x32-10, counter
 *                       (node, pass, 0), key = seed), which keeps a steady
 *                       flow unbiased; binary16 then stores values below its
 *                       normal range (|f_p / w_p - 1| < 6e-8) as zero.
 *                       RBC_ROUND_NEAREST (ties to even, IEEE) is biased by
 *                       percents in slow steady flows [stochastic]
 *   seed                key of the stochastic rounding [0]
 *   node_list           dense layout only: lattice pass over a list of the
 *                       fluid nodes (one thread each, no work on solid nodes)
 *                       instead of whole staged rows: 1 always, -1 never, 0
 *                       when fewer than half the nodes are fluid
 *   layout              storage of the lattice fields [RBC_LAYOUT_AUTO]:
 *                       RBC_LAYOUT_DENSE keeps every node; RBC_LAYOUT_COMPACT
 *                       keeps, per lattice row (y, z), only the span of x
 *                       that a fluid node can reach through a link (the
 *                       hull of the fluid nodes of the nine neighbouring rows
 *                       widened by one, rounded out to 8 entries, or the
 *                       whole row when it wraps along x), in lattice order,
 *                       so the memory and the lattice pass's traffic follow
 *                       the fluid nodes of vessel geometries; requires solid
 *                       nodes and nx <= 32760 (RBC_EINVAL otherwise).
 *                       RBC_LAYOUT_AUTO takes the compact layout for lattices
 *                       with solid nodes where it stores at most 90 % of the
 *                       nodes.  The request server packs dense solves only.
 *   stream              cudaStream_t the library works on (NULL: one it
 *                       creates and owns). */
typedef struct {
    double tau0, delta, kappa;
    double gamma_T, gamma_R;
    double alpha_tt;
    double eps0;
    double xi[3];
    double semi_axes[3];
    double mass, inertia[3];
    double sigma_min_wall, wall_radius;
    double rho_floor;
    double r_cut, r_cut_wall;
    double mach_max;
    int bin_capacity;
    int max_neighbors;
    int precision;
    int rounding;
    uint64_t seed;
    int node_list;
    int layout;
    void *stream;
} rbc_params;

#define RBC_LAYOUT_AUTO 0
#define RBC_LAYOUT_DENSE 1
#define RBC_LAYOUT_COMPACT 2

#define RBC_PREC_F32 0
#define RBC_PREC_F16 1
#define RBC_PREC_BF16 2
#define RBC_ROUND_STOCHASTIC 0
#define RBC_ROUND_NEAREST 1

/* Running budgets (Sec. 2.2 conservation claims).  mass and p_fluid are the
 * zeroth and first moments of the stored populations over fluid nodes;
 * p_cells = sum_i M V_i; max_u = max |u| of the last lattice pass; power =
 * sum over fluid nodes of G_ext(x) . u(x), the work rate of the external
 * force on the velocity of the last pass (at a fixed drive it is inversely
 * proportional to the effective viscosity of the suspension). */
typedef struct {
    int64_t step;
    double mass;
    double p_fluid[3];
    double p_cells[3];
    double max_u;
    int64_t gb_clamps;
    int32_t unstable;
    int32_t overflow; /* bit 0 bin, bit 1 neighbour list, bit 2 shape box */
    double power;
} rbc_stats_t;

/* Fill *p with the paper's parameters (values above) and a NULL stream. */
void rbc_default_params(rbc_params *p);

/* Bytes of device workspace rbc_init needs for this problem (256-byte
 * aligned pieces).  Returns RBC_EINVAL for an invalid problem. */
int rbc_workspace_size(const rbc_geometry *geom, const rbc_cells *cells,
                       const rbc_params *params, size_t *bytes);

/* Validate the problem (at most 2^32 / 19 lattice nodes), carve the caller's device workspace (at least
 * rbc_workspace_size bytes, 256-byte aligned, owned by the caller and kept
 * alive until rbc_free), copy geometry and cells to the device, set the
 * fluid at rest (f = f^eq(rho = 1, u = 0)), capture one step as CUDA graphs
 * on params->stream and build the cell list and Gay-Berne forces of the
 * initial poses.  Synchronises that stream.  *out receives the
 * handle.  Errors: RBC_EINVAL, RBC_ENOMEM (workspace too small), RBC_ECUDA. */
int rbc_init(const rbc_geometry *geom, const rbc_cells *cells, const rbc_params *params,
             void *workspace, size_t workspace_bytes, rbc_handle **out);

/* Enqueue n coupled steps on the handle's stream and return without waiting
 * (Sec. 2, App. A).  One step: sampling, rigid update and spreading per cell
 * at the current poses (whose cell list and Gay-Berne forces are already
 * known), then the lattice pass, while the cell list and Gay-Berne forces of
 * the new poses are computed alongside it for the next step.  Returns
 * RBC_EUNSTABLE / RBC_ENOMEM if an earlier synchronising call saw the device
 * flags raised; RBC_EINVAL for n < 0. */
int rbc_step(rbc_handle *h, int64_t n);

/* Copy the fields of the last lattice pass to host buffers (any may be
 * NULL): rho[N] (Eq. dens), u[3N] node-major (Eq. vel), and per cell 13
 * doubles R(3) quat(4) V(3) Omega_body(3).  Solid nodes report rho = u = 0.
 * Synchronises the stream; returns RBC_EUNSTABLE if the guard tripped. */
int rbc_fields(rbc_handle *h, double *rho, double *u, double *cells_state);

/* Compute the budgets on the device and copy them to *out (synchronising). */
int rbc_stats(rbc_handle *h, rbc_stats_t *out);

/* Per cell 21 doubles of the last step: F_mech(3) tau_mech(3) (Gay-Berne
 * plus any external force and torque, lab frame), u~(3) omega~(3) (Eqs. vel, vort), T^S(3) (Eq.
 * pheno_torque_diss), J(3) L(3) (hydrodynamic linear and lab angular impulse
 * returned to the fluid).  Host buffer; synchronises. */
int rbc_cell_diag(rbc_handle *h, double *out);

/* Candidate partners of every cell at its current pose (the cell list is
 * rebuilt at rbc_init and at the end of every step): counts[n]
 * and lists[n*max_per_cell], each list sorted by partner index; partners are
 * the j != i with |R_i - R_j|^2 < r_cut^2 (minimum image along periodic
 * axes, FP64, no fused multiply-add).  Returns RBC_ENOMEM if a list is longer
 * than max_per_cell.  Host buffers; synchronises. */
int rbc_neighbors(rbc_handle *h, int *counts, int *lists, int max_per_cell);

/* Kernel timing.  rbc_set_timing(h, capacity) makes the next `capacity`
 * steps record CUDA events inside the step graph on the handle's stream:
 * before and after the per-cell kernel and after the lattice pass (capacity
 * 0 turns it off).  Timed steps run a second pair of step graphs with those
 * event-record nodes (captured at the first call with capacity > 0); a node
 * between two kernels delays the second by a few microseconds, so untimed
 * steps run graphs without them.  Synchronises.  rbc_kernel_times synchronises and returns for k = 0 (the
 * lattice pass, which runs alongside the next step's cell list, Gay-Berne
 * forces and shape lists) and k = 1 (the per-cell kernel: sampling, rigid
 * update and spreading) the summed milliseconds ms[k] and the number of
 * timed launches count[k], then clears them. */
int rbc_set_timing(rbc_handle *h, int capacity);
int rbc_kernel_times(rbc_handle *h, double ms[2], int64_t count[2]);

/* Autotuner of the lattice pass's launch shape (tiles per SM).  The
 * row-staged pass is persistent: its grid is CTAs-per-SM x SMs, each CTA
 * holding a ring of `stages` shared-memory buffers.  Without tuning the
 * runtime picks the shape from a cost model (fewest idle CTA slots in the
 * last wave; at most 2 CTAs per SM when cells run beside the pass).
 * rbc_autotune times every shape that fits (ring depth 2..4 x 1..4 CTAs per
 * SM), each in both graph orders of the step (the cell-list, Gay-Berne and
 * shape-list kernels launched before the lattice pass, so that they overlap
 * it, or after it), over steps_per_trial coupled steps after as many
 * warm-up steps, keeps the fastest, then with it times jointly the schedule
 * of the cell-side kernels: the spread of the cells' impulses in the
 * per-cell kernel or split off it into a kernel of its own (the next step's
 * cell-side kernels then start beside the spread, which only the lattice
 * pass waits for), both graph orders, and bounded grids of the shape-list
 * and Gay-Berne kernels (2-4 blocks per SM, grid-stride over the cells)
 * against one block per group of cells; then the particle-bin edge
 * (the candidate radius times 1, 1.25, 1.5 or 2: coarser grids scan fewer,
 * fuller bins; a grid that overflows a bin is dropped), and re-captures the
 * step graphs.  The trial steps are ordinary
 * steps of the solve (the state advances).  Synchronises.  out may be NULL. */
typedef struct {
    int stages, ctas_per_sm;     /* chosen shape (0, 0: the one-thread-per-node pass, nothing to tune) */
    double ms_per_step;          /* its time per coupled step */
    double default_ms_per_step;  /* time per step of the cost model's shape */
    int trials;                  /* shapes timed */
    int lattice_first;           /* chosen order: 1 = lattice pass before the side kernels */
    int wt_blocks_per_sm;        /* grid of the shape-list kernel, blocks per SM (0: one per 4 cells) */
    int gb_blocks_per_sm;        /* grid of the Gay-Berne kernel, blocks per SM (0: one per 4 cells) */
    double bin_scale;            /* chosen edge of the particle bins over the candidate radius (>= 1) */
    int split_spread;            /* 1: the spread runs as a kernel of its own beside the side kernels */
} rbc_tune_report;
int rbc_autotune(rbc_handle *h, int steps_per_trial, rbc_tune_report *out);

/* Step schedule set by hand (what rbc_autotune chooses besides the launch
 * shapes): split_spread != 0 runs the spread of the cells' impulses as a
 * kernel of its own, which the next step's cell-list, Gay-Berne and
 * shape-list kernels run beside (no effect without cells); lattice_first
 * != 0 captures the lattice pass before those kernels in the step graph.
 * Either schedule computes the same step (up to the order of the spread's
 * float atomics).  Re-captures the step graphs.  RBC_EINVAL while kernel
 * timing is active. */
int rbc_set_schedule(rbc_handle *h, int split_spread, int lattice_first);

/* Wall shear stress (the quantity Sec. 4 maps in the coronary geometry).
 * At every fluid node with a solid link neighbour the wall normal n is the
 * unit sum of its links that stay in the fluid (minus those into the
 * wall), and the wall shear stress is the traction of the stress on the
 * tangent plane, sigma n - (n . sigma n) n, with the sigma of Eq.
 * stresstensorLB (requires walls, and cells with alpha_tt != 0 or open
 * boundaries, for sigma to be computed).  rbc_wss_accumulate enqueues on the
 * handle's stream the addition of the current value to per-node sums;
 * rbc_wss synchronises and copies the node indices (node[k]) and the
 * time-averaged vectors (tau[3k..]) of up to max nodes, returning their
 * number in *n and the number of samples in *samples.  RBC_EINVAL without
 * walls or stress. */
int rbc_wss_accumulate(rbc_handle *h);
int rbc_wss(rbc_handle *h, int64_t *node, double *tau, int64_t max, int64_t *n, int64_t *samples);

/* Checkpoint and resume (the paper has no counterpart).  A checkpoint
 * holds what the next step reads: the populations of the last pass, its
 * velocity and stress fields, the cell state (R, q, V, Omega in FP64, the
 * cached-step flags), the step count, the pass counter that keys the
 * stochastic rounding and the clamp count; the cell list, the Gay-Berne
 * forces and the shape lists are rebuilt from the poses on load.
 * rbc_checkpoint_size gives its bytes; rbc_save synchronises and writes it
 * to a caller-owned host buffer; rbc_load restores it into a handle
 * initialised with the same problem (geometry, cells count, parameters,
 * storage and layout; RBC_EINVAL otherwise) and synchronises.  A resumed
 * run continues as the saved one would: bit for bit without cells, and with
 * cells up to the rounding order of the spreading's float atomics.  The
 * time averages of the server, of the wall shear stress and of the
 * cell-centre profile start again. */
int rbc_checkpoint_size(const rbc_handle *h, size_t *bytes);
int rbc_save(rbc_handle *h, void *buf, size_t bytes);
int rbc_load(rbc_handle *h, const void *buf, size_t bytes);

/* Failure detection of the staged lattice passes (the paper has no
 * counterpart).  Their producer / consumer pipeline waits on shared-memory
 * barriers, each wait bounded: past the bound the waiting warp raises a
 * timeout flag and leaves, the producer first waiting (with the default
 * bound) for every copy it has issued, so the kernel always returns and the
 * context stays usable; the next synchronising call (rbc_stats,
 * rbc_fields) returns RBC_ETIMEOUT.  rbc_set_wait_limit sets the bound in
 * clock64 cycles (0: the default, about 2 s) and, for tests of this path,
 * starve_batch >= 0 names a batch whose copies the producer never issues,
 * so that the consumers waiting for it run out of time (-1: none); the step
 * graphs are re-captured.  RBC_EINVAL when the solve's lattice pass is not
 * a staged one. */
int rbc_set_wait_limit(rbc_handle *h, int64_t cycles, int starve_batch);

/* Cell-centre profile: the near-wall hematocrit and cell-free layer that
 * Sec. 4 reports for vessels.  rbc_profile_accumulate enqueues on the
 * handle's stream the addition of the current cell centres to a histogram
 * of 1-lattice-unit bins along `axis` (0 x, 1 y, 2 z; bin k counts centres
 * with k <= R_axis < k + 1), as FP64 whole numbers (exact, independent of
 * order); a call with another axis first clears it.  rbc_profile
 * synchronises and copies the n_axis bins to counts[nbins] (nbins >= the box
 * along the axis, the rest zeroed) with the axis (-1: never accumulated)
 * and the number of samples; the time-averaged count of bin k is
 * counts[k] / samples.  RBC_EINVAL without cells. */
int rbc_profile_accumulate(rbc_handle *h, int axis);
int rbc_profile(rbc_handle *h, double *counts, int nbins, int *axis, int64_t *samples);

/* Kernel launches one rbc_step(h, 1) enqueues. */
int rbc_launches_per_step(const rbc_handle *h);

/* Storage layout of the handle's lattice fields (see rbc_params.layout):
 * *compact = 1 for the compact layout, *entries = stored entries per field
 * (lattice nodes when dense), *fluid = fluid nodes.  Any pointer may be
 * NULL. */
int rbc_layout(const rbc_handle *h, int *compact, int64_t *entries, int64_t *fluid);

/* The library's fluid-node indexing: the lattice index x + nx (y + ny z) of
 * every fluid node in the order of its storage entries, read back from the
 * device's row table and link words (compact) or node flags (dense).  Up to
 * max indices go to nodes (host); *count receives the number of fluid nodes.
 * Synchronises. */
int rbc_fluid_nodes(rbc_handle *h, int64_t *nodes, int64_t max, int64_t *count);

/* Size of the static device scratch of rbc_neighbors_noalloc, in ints
 * (4 MiB). */
#define RBC_NOALLOC_SCRATCH_INTS (1 << 20)

/* Candidate-partner lists of n cells without any device allocation and
 * without caller-provided scratch.  The paper has no counterpart: this is a
 * convenience for callers that cannot call cudaMalloc -- code running where
 * device memory is fully committed to buffers it does not own, or a host
 * that forbids allocation outside its own pool -- and so cannot lend the
 * workspace rbc_init needs.  It builds the lists rbc_neighbors reports after
 * a step: partners j != i with |R_i - R_j|^2 < r_cut^2 (minimum image along
 * periodic axes, FP64, no fused multiply-add), each list sorted by index.
 *   pos           device, 3n doubles, inside [0, n_axis) on every axis
 *   nx, ny, nz    box; periodic[3] host flags
 *   counts        device, n ints (out); lists device, n * max_per_cell ints
 *   max_per_cell  1..128; stream: cudaStream_t (NULL: legacy default)
 * Its scratch (an overflow flag, bin counts and 32 slots per bin of a grid
 * of bins no smaller than r_cut) is a static device array of
 * RBC_NOALLOC_SCRATCH_INTS ints that every GPU loading the library holds
 * until the process exits; boxes whose grid needs more return RBC_EINVAL.
 * All calls share that array, so calls that overlap on the GPU race and
 * must be serialised.  Every call looks up the array's address
 * (cudaGetSymbolAddress) on the current device, clears the counts it uses,
 * and ends by copying a flag back and synchronising the stream: never call
 * it on a stream that is being captured into a CUDA graph.  RBC_EINVAL for
 * a box whose grid of bins no smaller than r_cut needs more scratch than
 * the array holds; RBC_ENOMEM when a bin holds more than 32 cells or a list
 * exceeds max_per_cell; rbc_last_error(NULL) describes failures. */
int rbc_neighbors_noalloc(const double *pos, int n, int nx, int ny, int nz, const int periodic[3],
                          double r_cut, int *counts, int *lists, int max_per_cell, void *stream);

/* ------------------------------------------------------------------------
 * Request server: continuous batching of independent solves.
 *
 * Not a step of the paper's method: it serves many rheology / vessel solves
 * (the use Sec. 4 puts the model to) on one GPU.  Requests of different box
 * sizes, hematocrits and drives are queued and admitted as device memory and
 * slots free up (rbc_init runs on a worker thread).  Admitted solves of one
 * class -- storage type, walls, cells, stress output, shape box -- form a
 * pack that advances in ticks of tick_steps coupled steps captured as one
 * CUDA graph: each kernel of the step is launched once for all members of
 * the pack, over device tables of their arguments with per-solve block and
 * batch offsets (the lattice pass is one persistent launch over all their
 * row batches), followed by each member's budget reduction, which adds to
 * its time averages on the device.  Members join and leave between ticks;
 * the last (steps mod tick_steps) steps of a solve, and solves that cannot be packed
 * (no cells, or rows not a multiple of 16 bytes), run on a stream of their
 * own.  Device memory comes from one arena the caller lends: each admitted
 * solve takes rbc_workspace_size bytes of it (first fit) and returns them
 * when it finishes; each pack class takes a small table region.  Results are
 * the time-averaged budgets of each solve.
 * ------------------------------------------------------------------------ */
typedef struct rbc_server rbc_server;

typedef struct {
    rbc_geometry geom;     /* copied at submit */
    rbc_cells cells;       /* copied at submit */
    rbc_params params;     /* copied; params.stream is ignored (the server assigns one) */
    int64_t steps;         /* coupled steps to run (>= 1) */
    int64_t average_from;  /* samples (one per tick) at pass counts >= this are averaged */
    uint64_t tag;          /* caller's identifier, returned in the result */
    /* Final state of the solve, written when it finishes successfully,
     * before its result is queued (each may be NULL): out_rho[N], out_u[3N]
     * and out_cells[13 n] as rbc_fields, out_diag[21 n] as rbc_cell_diag.
     * Host buffers owned by the caller, who keeps them valid until the
     * result has come out of rbc_server_results. */
    double *out_rho, *out_u, *out_cells, *out_diag;
} rbc_request;

typedef struct {
    uint64_t tag;
    int32_t status;        /* RBC_OK or the error that ended the solve */
    int32_t pad;
    int64_t steps;         /* coupled steps run */
    int64_t samples;       /* samples in the averages */
    double mean_power;     /* time average of rbc_stats_t.power */
    double mean_p_fluid[3];
    double max_u;          /* largest max |u| over the samples */
    double t_submit, t_admit, t_done;  /* server clock (s since rbc_server_create) */
    uint64_t workspace_bytes;
} rbc_result;

/* Create a server on the current device.  arena: device memory (256-byte
 * aligned, caller-owned, kept alive until rbc_server_free) that the solves'
 * workspaces are carved from; max_active: solves advanced at once (1..256);
 * tick_steps: steps per launched tick (even, 2..100000).  The server creates
 * max_active streams. */
int rbc_server_create(void *arena, size_t arena_bytes, int max_active, int tick_steps, rbc_server **out);

/* Validate and queue a request (inputs copied).  RBC_EINVAL for an invalid
 * problem, RBC_ENOMEM if its workspace exceeds the whole arena. */
int rbc_server_submit(rbc_server *s, const rbc_request *r);

/* One non-blocking round: retire finished ticks, finish solves that are
 * done (their results become available), launch further ticks (at most two
 * in flight per solve), and admit queued requests in arrival order while a
 * slot and an arena block are free (requests that do not fit yet are passed
 * over by later ones).  Admission runs rbc_init, which synchronises only the
 * new solve's stream.  *active, *queued (may be NULL) receive the counts.
 * Returns the first error of a server-level CUDA call; errors of one solve
 * end that solve and go into its result. */
int rbc_server_poll(rbc_server *s, int *active, int *queued);

/* Move up to max finished results into out (oldest first); *n receives the
 * number written. */
int rbc_server_results(rbc_server *s, rbc_result *out, int max, int *n);

/* Seconds on the server clock. */
double rbc_server_clock(const rbc_server *s);

/* Finish or abandon all work, release every solve, stream and event (not
 * the arena).  NULL is ignored. */
void rbc_server_free(rbc_server *s);

/* Release the handle, its graphs, events and owned stream (not the caller's
 * workspace).  NULL is ignored. */
void rbc_free(rbc_handle *h);

/* Message of the last failure on h (h may be NULL: last failure of the
 * calling thread).  Valid until the next call on the same handle/thread. */
const char *rbc_last_error(const rbc_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* RBC_H */
