/*
 * oracle.h -- interface of the plain FP64 CPU oracle of the coupled
 * lattice-Boltzmann + rigid red-blood-cell time step (Melchionna,
 * "A model for red blood cells in simulations of large-scale blood flows").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes this
 * header or links this code; only the tests, the package's smoke check and
 * the CPU-baseline leg of the benchmark call it, through oracle/oracle.py.
 *
 * Conventions (all lattice units, time step h = 1):
 *   - lattice node n = x + nx*(y + ny*z), x fastest; indices always wrap,
 *     walls are solid nodes;
 *   - node-major field arrays: u[3*n + a], sigma[6*n + k] with
 *     k = xx, yy, zz, xy, xz, yz;
 *   - orientation matrices Q[3*a + b] = component a (lab) of body axis b,
 *     i.e. v_lab = Q v_body (Sec. 2.2);
 *   - quaternions (w, x, y, z), body -> lab.
 */
#ifndef RBC_ORACLE_H
#define RBC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    int periodic[3];
    const unsigned char *solid;   /* nx*ny*nz, 1 = solid; NULL = all fluid */
    double body_force[3];         /* external force density on fluid nodes */
    double tau0, delta, kappa;    /* Eq. enhance-viscosity */
    double gamma_T, gamma_R;      /* Eqs. pheno_force / pheno_torque, App. A */
    double alpha;                 /* Eq. pheno_torque_diss */
    double eps0;                  /* Eq. gayberne */
    double xi[3];                 /* shape-function radii (Sec. 2.2) */
    double semi_axes[3];          /* Gay-Berne shape matrix S (Sec. 2.5) */
    double mass, inertia[3];      /* M, diagonal body-frame I */
    double sigma_min_wall;        /* wall-RBC sigma_min (Sec. 2.5, last paragraph) */
    double wall_radius;           /* radius of a wall particle */
    double rho_floor;             /* lower clamp of the GB reduced distance */
    double r_cut, r_cut_wall;     /* candidate radii of cell-cell / cell-wall pairs */
    int ncells;
    const double *pos, *quat, *vel, *omega;  /* 3n, 4n, 3n (or NULL), 3n body frame (or NULL) */
    int storage;      /* population storage: ORC_STORE_EXACT, _F16 or _BF16 */
    int stochastic;   /* 16-bit storage: 1 = stochastic rounding, 0 = to nearest */
    unsigned long long seed;  /* key of the stochastic rounding's random numbers */
    double body_force_wave[3];  /* amplitude of a force density A sin(2 pi y / ny) on fluid nodes */
    /* open boundaries: node_type[N] (NULL = none) marks fluid nodes as
     * ORC_NODE_INLET (velocity inlet: u = inlet_umax (1 - r^2 / R^2) along
     * +z, r the distance of (x, y) from inlet_center, R = inlet_radius) or
     * ORC_NODE_OUTLET (pressure outlet, rho = 1) */
    const unsigned char *node_type;
    double inlet_center[2], inlet_radius, inlet_umax;
    /* constant external force and torque on every cell (lab frame, 3n each,
     * or NULL): the push of the mobility tests of Sec. 3 */
    const double *force_ext, *torque_ext;
} orc_config;

#define ORC_NODE_INTERIOR 0
#define ORC_NODE_INLET 1
#define ORC_NODE_OUTLET 2

/* Population storage of the reduced-precision variants: FP64 (exact), or the
 * deviation from the lattice weight, scaled per direction, rounded to IEEE
 * binary16 or to bfloat16 after every collision, to nearest
 * (orc_round_storage) or stochastically (orc_round_storage_sr with six bits
 * of orc_storage_bits per value). */
#define ORC_STORE_EXACT 0
#define ORC_STORE_F16 1
#define ORC_STORE_BF16 2

typedef struct orc_state orc_state;

/* Coupled solver. */
orc_state *orc_create(const orc_config *cfg);
void orc_destroy(orc_state *s);
void orc_step(orc_state *s, long nsteps);
long orc_step_count(const orc_state *s);
/* rho[N], u[3N] of the last lattice pass (solid nodes 0). */
void orc_fields(const orc_state *s, double *rho, double *u, double *sigma);
/* Per cell 18 doubles: R(3) Q(9) V(3) Omega_body(3). */
void orc_cells(const orc_state *s, double *out);
/* Per cell 21 doubles of the last step: F_mech(3) tau_mech_lab(3) u~(3)
 * omega~(3) T^S(3) J(3) L(3). */
void orc_diag(const orc_state *s, double *out);
/* mass, P_fluid(3), P_cells(3) of the current state and the work rate of
 * the external force, sum over fluid nodes of G_ext(x) . u(x) with u of the
 * last lattice pass (8 doubles). */
void orc_budget(const orc_state *s, double *out);
long orc_clamps(const orc_state *s);
/* Cell pairs i<j with |R_ij|^2 < r_cut^2 at the current positions, by brute
 * force; writes up to max pairs (2 ints each), returns the number found. */
long orc_neighbor_pairs(const orc_state *s, int *pairs, long max);
/* Fluid nodes in canonical lattice order (n = x + nx (y + ny z)
 * ascending); writes up to max, returns the number of fluid nodes. */
long orc_fluid_nodes(const orc_state *s, long *nodes, long max);
/* Overwrite the fluid outputs the next step samples (sampling pins). */
void orc_set_sampled_fields(orc_state *s, const double *u, const double *sigma);

/* Building blocks, exported for the pin tests. */
double orc_peskin(double r);
void orc_quat_to_Q(const double q[4], double Q[9]);
/* Shape of one body on the whole lattice: raw w, normalised delta, central
 * difference gradient Ddelta[3N]; returns the normalisation sum. */
double orc_shape_field(int nx, int ny, int nz, const unsigned char *solid,
                       const double R[3], const double Q[9], const double xi[3],
                       double *w, double *delta, double *Ddelta);
void orc_sample_cell(int nx, int ny, int nz, const unsigned char *solid,
                     const double *u, const double *sigma,
                     const double R[3], const double Q[9], const double xi[3], double alpha,
                     double ut[3], double wt[3], double TS[3]);
void orc_spread_cell(int nx, int ny, int nz, const unsigned char *solid,
                     const double R[3], const double Q[9], const double xi[3], double kappa,
                     const double J[3], const double L[3], double *G, double *theta);
/* One Gay-Berne pair, d = R_i - R_j.  Returns 1 if the reduced distance was
 * clamped, 0 otherwise. */
int orc_gb_pair(const double d[3], const double Ai[9], const double Aj[9],
                double sigma_min, double eps0, double rho_floor,
                double *u, double F[3], double tau_i[3], double tau_j[3]);
/* Half steps of the App. A integrator for one body (Q row-major 3x3). */
void orc_rigid_close(double V[3], double Om[3], const double Fc[3], const double Tc[3],
                     double M, const double I[3], double gT, double gR);
void orc_rigid_open(double R[3], double Q[9], double V[3], double Om[3],
                    const double Fc[3], const double Tc[3], double M, const double I[3],
                    double gT, double gR);
/* One D3Q19 lattice pass on a caller-provided population array f[19*N]
 * (post-collision in, post-collision out) with given force density G[3N]
 * (NULL = 0) and relaxation-time field tau[N]; writes rho, u, sigma. */
void orc_lb_pass(int nx, int ny, int nz, const unsigned char *solid, double *f,
                 const double *G, const double *tau, double *rho, double *u, double *sigma);
/* Round v to the storage format `kind` (ORC_STORE_F16: IEEE binary16,
 * ORC_STORE_BF16: bfloat16; to nearest, ties to even, overflow to infinity);
 * ORC_STORE_EXACT returns v. */
double orc_round_storage(int kind, double v);
/* Stochastic rounding of v to `kind` with random integer r < 2^bits: up
 * (away from zero) when the fraction of the gap covered plus (r + 1/2)/2^bits
 * reaches 1; saturates at the largest finite value. */
double orc_round_storage_sr(int kind, double v, unsigned r, int bits);
/* Philox4x32-10 block function (counter, key -> 128 random bits). */
void orc_philox4x32(const unsigned ctr[4], const unsigned key[2], unsigned out[4]);
/* The six random bits of speed slot `slot` (rank of the speed ordered by
 * (c_z, c_y, c_x)) at node n and step `step`. */
unsigned orc_storage_bits(unsigned long long seed, long step, long n, int slot);
/* Scale S of the stored deviation s_p = (f_p - w_p) S / w_p of `kind`. */
double orc_storage_scale(int kind);
/* Post-collision populations f[19*N] (solid nodes 0), direction-major. */
void orc_populations(const orc_state *s, double *f);
/* Replace the post-collision populations (then stored in the solver's
 * format), e.g. to start from a prescribed flow. */
void orc_set_populations(orc_state *s, const double *f);
/* Wall shear stress of the last lattice pass at every fluid node with a
 * solid link neighbour: n = number of such nodes (returned), node[k] their
 * indices, tau[3k..] the traction of the stress on the wall tangent plane,
 * sigma n - (n.sigma n) n, with n the unit vector sum of the links into the
 * fluid (minus the links to solid neighbours).  Writes up to max entries. */
long orc_wall_shear(const orc_state *s, long *node, double *tau, long max);
/* Velocities and weights in the order used above. */
void orc_lattice(int *c, double *w);

#ifdef __cplusplus
}
#endif
#endif
