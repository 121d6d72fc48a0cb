/*
 * oracle.c -- plain, slow FP64 CPU oracle of the coupled lattice-Boltzmann +
 * rigid red-blood-cell time step of S. Melchionna, "A model for red blood
 * cells in simulations of large-scale blood flows" (2011).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the yardstick the CUDA path is
 * checked against; it shares no code, header, table or constant with the
 * CUDA library and is never linked into it.  Only the tests, the package's
 * smoke check and the CPU-baseline leg of the benchmark execute it.
 *
 * Every function follows the paper's steps in the paper's order, in FP64,
 * single-threaded, with no blocking or fusion.  Where the paper is garbled or
 * silent the reading taken is stated in the comment of the function that
 * takes it.  Pins: every function here is checked by the -m "not gpu" tests
 * against closed forms, invariants or brute force (tests/test_oracle_*.py);
 * the per-cell sums of the Gay-Berne forces and torques, the wall-particle
 * set and the frame of the angular impulse by tests/test_oracle_mechanics.py.
 *
 * One coupled step (readings "explicit coupling" and "velocity-Verlet caching"):
 *   1. shapes of every cell at the current pose (Sec. 2.2);
 *   2. Gay-Berne forces and torques, cell-cell and cell-wall (Sec. 2.5, App. B);
 *   3. sampling of the fluid fields written by the previous lattice pass:
 *      smeared velocity and vorticity (Eqs. vel, vort) and the elongational
 *      torque (Eq. pheno_torque_diss);
 *   4. combined force and torque (App. A, step 5);
 *   5. rigid-body update: close the previous step (App. A steps 6-7), open
 *      this one (steps 1-4); record the hydrodynamic impulses J, L;
 *   6. spreading of the reaction -J, -L to the fluid as a force density G and
 *      of the smoothed characteristic function into the relaxation time
 *      (Sec. 2.2 last equation, Eq. enhance-viscosity);
 *   7. lattice pass: streaming (Eq. streaming) then BGK collision with the
 *      body-force term (Eqs. lbe_discrete, chen_force) and the moments
 *      (Eqs. dens, vel) and stress (Eq. stresstensorLB).
 */
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define NQ 19
#define H_STEP 1.0 /* time step h = 1 in lattice units (Sec. 3) */

/* D3Q19 discrete speeds in the order Sec. 2.1 lists them: the null speed,
 * the six first-neighbour speeds, the twelve second-neighbour speeds. */
static const int CV[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* Weights of Sec. 2.1: 1/3 for the null speed, 1/18 for first and 1/36 for
 * second neighbours. */
static double weight(int p)
{
    int c2 = CV[p][0] * CV[p][0] + CV[p][1] * CV[p][1] + CV[p][2] * CV[p][2];
    if (c2 == 0) return 1.0 / 3.0;
    if (c2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite(int p)
{
    for (int q = 0; q < NQ; q++)
        if (CV[q][0] == -CV[p][0] && CV[q][1] == -CV[p][1] && CV[q][2] == -CV[p][2]) return q;
    return -1;
}

void orc_lattice(int *c, double *w)
{
    for (int p = 0; p < NQ; p++) {
        for (int a = 0; a < 3; a++) c[3 * p + a] = CV[p][a];
        w[p] = weight(p);
    }
}

static int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

static long node_of(int nx, int ny, int nz, int x, int y, int z)
{
    return (long)wrap(x, nx) + (long)nx * ((long)wrap(y, ny) + (long)ny * wrap(z, nz));
}

static int is_solid(const unsigned char *solid, long n) { return solid != NULL && solid[n] != 0; }

/* ------------------------------------------------------------------------ */
/* Lattice Boltzmann pass (Sec. 2.1)                                         */
/* ------------------------------------------------------------------------ */

/*
 * f holds post-collision populations f*_p(x) of the previous pass.
 * Streaming, Eq. streaming: f_p(x + h c_p) = f*_p(x); when x + c_p is a solid
 * node the population is bounced back to x into the opposite direction
 * (halfway bounce-back at resting walls: the paper does not give its wall
 * rule).  Collision, Eq. lbe_discrete, at every fluid node:
 *   rho = sum_p f_p                                  (Eq. dens)
 *   rho u = sum_p f_p c_p + h/2 G                    (Eq. vel; G is a force
 *                                                     density, see below)
 *   f_p^eq = w_p rho [1 + u.c/c^2 + ((u.c)^2 - c^2 u^2)/(2c^4)]
 *   Df_p = (1 - h/(2T)) w_p [G.c/c^2 + ((G.c)(u.c) - c^2 G.u)/(2c^4)]
 *   f*_p = (1 - h/T) f_p + (h/T) f_p^eq + h Df_p
 *   sigma = -(1 - h/(2T)) sum_p c_p c_p (f_p - f_p^eq)  (Eq. stresstensorLB)
 * Readings: G is a force density (the rho of Eq. chen_force dropped) so that
 * sum_p Df_p c_p is the injected momentum; Df carries Guo's factor
 * (1 - h/(2T)), the scheme Eq. vel is cited from, so that the fluid gains
 * exactly h G per node and step; the stress carries the minus sign that
 * makes it +rho nu (du + du^T) with nu = c^2 (T - h/2).
 */
void orc_lb_pass(int nx, int ny, int nz, const unsigned char *solid, double *f,
                 const double *G, const double *tau, double *rho, double *u, double *sigma)
{
    const long N = (long)nx * ny * nz;
    const double c2 = 1.0 / 3.0; /* sound speed squared, D3Q19 */
    double *fs = (double *)calloc((size_t)NQ * N, sizeof(double));

    /* streaming */
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long n = node_of(nx, ny, nz, x, y, z);
                if (is_solid(solid, n)) continue;
                for (int p = 0; p < NQ; p++) {
                    long m = node_of(nx, ny, nz, x + CV[p][0], y + CV[p][1], z + CV[p][2]);
                    if (is_solid(solid, m))
                        fs[(long)opposite(p) * N + n] = f[(long)p * N + n];
                    else
                        fs[(long)p * N + m] = f[(long)p * N + n];
                }
            }

    /* collision */
    for (long n = 0; n < N; n++) {
        if (is_solid(solid, n)) {
            rho[n] = 0.0;
            for (int a = 0; a < 3; a++) u[3 * n + a] = 0.0;
            for (int k = 0; k < 6; k++) sigma[6 * n + k] = 0.0;
            for (int p = 0; p < NQ; p++) f[(long)p * N + n] = 0.0;
            continue;
        }
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int p = 0; p < NQ; p++) {
            double fp = fs[(long)p * N + n];
            r += fp;
            for (int a = 0; a < 3; a++) j[a] += fp * CV[p][a];
        }
        double g[3] = {0.0, 0.0, 0.0};
        if (G != NULL)
            for (int a = 0; a < 3; a++) g[a] = G[3 * n + a];
        double T = tau[n];
        double v[3];
        for (int a = 0; a < 3; a++) v[a] = (j[a] + 0.5 * H_STEP * g[a]) / r;
        double uu = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        double gu = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
        double Pneq[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int p = 0; p < NQ; p++) {
            double cu = CV[p][0] * v[0] + CV[p][1] * v[1] + CV[p][2] * v[2];
            double cg = CV[p][0] * g[0] + CV[p][1] * g[1] + CV[p][2] * g[2];
            double feq = weight(p) * r * (1.0 + cu / c2 + (cu * cu - c2 * uu) / (2.0 * c2 * c2));
            double df = (1.0 - H_STEP / (2.0 * T)) * weight(p) *
                        (cg / c2 + (cg * cu - c2 * gu) / (2.0 * c2 * c2));
            double fp = fs[(long)p * N + n];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) Pneq[a][b] += CV[p][a] * CV[p][b] * (fp - feq);
            f[(long)p * N + n] = (1.0 - H_STEP / T) * fp + (H_STEP / T) * feq + H_STEP * df;
        }
        double fac = -(1.0 - H_STEP / (2.0 * T));
        rho[n] = r;
        for (int a = 0; a < 3; a++) u[3 * n + a] = v[a];
        sigma[6 * n + 0] = fac * Pneq[0][0];
        sigma[6 * n + 1] = fac * Pneq[1][1];
        sigma[6 * n + 2] = fac * Pneq[2][2];
        sigma[6 * n + 3] = fac * Pneq[0][1];
        sigma[6 * n + 4] = fac * Pneq[0][2];
        sigma[6 * n + 5] = fac * Pneq[1][2];
    }
    free(fs);
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision population storage                                      */
/* ------------------------------------------------------------------------ */

/*
 * The paper keeps the populations f_p at every node (Sec. 2.1) and says
 * nothing about their storage format.  The reduced-precision variants store,
 * after each collision, the deviation from the lattice weight scaled per
 * direction,
 *     s_p = (f_p - w_p) S / w_p,        f_p = w_p + s_p w_p / S,
 * in a 16-bit floating-point format; the collision itself is done in full
 * precision.  Dividing by w_p gives all directions the same range
 * (s_p / S = f_p / w_p - 1).  For IEEE binary16 S = 2^10: its normal range
 * then reaches down to |f_p / w_p - 1| = 2^-24 and its largest finite value
 * 65504 up to |f_p / w_p - 1| < 64.  bfloat16 has the exponent range of FP32,
 * so S = 1.  Scaling by a power of two is exact.
 *
 * Two roundings are offered.  Round to nearest (ties to even) is biased in a
 * steady flow: the same node and direction round the same way step after
 * step, and the errors add up to a spurious force (a walled channel at
 * G = 1e-6 loses 2.5 % of its centre-line velocity with binary16, 15 % with
 * bfloat16).  Stochastic rounding rounds up with probability equal to the
 * fraction of the gap covered, so the error has zero mean; the random
 * numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC 2011), keyed by a seed and counted
 * by (node, step), six bits per stored value.
 */
double orc_storage_scale(int kind) { return kind == ORC_STORE_F16 ? 1024.0 : 1.0; }

/* Format parameters: stored mantissa bits, smallest normal exponent, largest
 * finite value. */
static void format_of(int kind, int *mant, int *emin, double *vmax)
{
    if (kind == ORC_STORE_F16) {
        *mant = 10;
        *emin = -14;
        *vmax = 65504.0;
    } else {
        *mant = 7;
        *emin = -126;
        *vmax = 3.3895313892515355e38;
    }
}

/* Spacing of the format's values around |v| (gradual underflow below
 * 2^emin). */
static double quantum(double v, int mant, int emin)
{
    int e;
    frexp(v, &e); /* |v| in [2^(e-1), 2^e) */
    int lead = e - 1;
    if (lead < emin) lead = emin;
    return ldexp(1.0, lead - mant);
}

/* To nearest, ties to even (nearbyint in the default rounding mode),
 * infinity past the largest finite value. */
double orc_round_storage(int kind, double v)
{
    if (kind == ORC_STORE_EXACT || v == 0.0 || !isfinite(v)) return v;
    int mant, emin;
    double vmax;
    format_of(kind, &mant, &emin, &vmax);
    double q = quantum(v, mant, emin);
    double r = nearbyint(v / q) * q;
    if (fabs(r) > vmax) return copysign(INFINITY, v);
    return r;
}

/* Stochastic rounding with `bits` random bits r: |v| lies between the format
 * values a <= |v| < a + q; the result is a + q when
 * (|v| - a)/q + (r + 1/2)/2^bits >= 1, else a, with the sign of v,
 * saturated at the largest finite value.  binary16 stores values below its
 * normal range (|v| < 2^-14, i.e. |f_p / w_p - 1| < 6e-8 after scaling) as
 * zero. */
double orc_round_storage_sr(int kind, double v, unsigned r, int bits)
{
    if (kind == ORC_STORE_EXACT || v == 0.0 || !isfinite(v)) return v;
    int mant, emin;
    double vmax;
    format_of(kind, &mant, &emin, &vmax);
    double m = fabs(v);
    if (kind == ORC_STORE_F16 && m < ldexp(1.0, emin)) return 0.0;
    double q = quantum(m, mant, emin);
    double t = m / q, fl = floor(t);
    double thr = ((double)r + 0.5) / ldexp(1.0, bits);
    double res = (t - fl + thr >= 1.0 ? fl + 1.0 : fl) * q;
    if (res > vmax) res = vmax;
    return copysign(res, v);
}

/* Philox4x32-10: ten rounds of the Philox S-box on a 128-bit counter with a
 * 64-bit key bumped by the Weyl constants between rounds (Salmon et al.,
 * Sec. 5). */
void orc_philox4x32(const unsigned ctr_in[4], const unsigned key_in[2], unsigned out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    for (int i = 0; i < 4; i++) out[i] = c[i];
}

/* Random-bit slot of a speed: its rank when the 19 speeds are ordered by
 * 9 (c_z + 1) + 3 (c_y + 1) + (c_x + 1), i.e. by (c_z, c_y, c_x). */
static int speed_slot(int p)
{
    int key = 9 * (CV[p][2] + 1) + 3 * (CV[p][1] + 1) + (CV[p][0] + 1), rank = 0;
    for (int q = 0; q < NQ; q++)
        if (9 * (CV[q][2] + 1) + 3 * (CV[q][1] + 1) + (CV[q][0] + 1) < key) rank++;
    return rank;
}

/* Six random bits of slot k at node n and step `step`: Philox4x32-10 of the
 * counter (n, step low word, step high word, 0) under the key (seed low
 * word, seed high word); slot k takes bits 6 (k mod 5) .. 6 (k mod 5) + 5 of
 * output word k / 5. */
unsigned orc_storage_bits(unsigned long long seed, long step, long n, int slot)
{
    unsigned ctr[4] = {(unsigned)n, (unsigned)((unsigned long long)step & 0xffffffffu),
                       (unsigned)((unsigned long long)step >> 32), 0u};
    unsigned key[2] = {(unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)};
    unsigned out[4];
    orc_philox4x32(ctr, key, out);
    return (out[slot / 5] >> (6 * (slot % 5))) & 63u;
}

/* Storage step of the reduced-precision variants on the post-collision
 * populations of every fluid node. */
static void store_populations(int kind, int stochastic, unsigned long long seed, long step, long N,
                              const unsigned char *solid, double *f)
{
    if (kind == ORC_STORE_EXACT) return;
    const double S = orc_storage_scale(kind);
    for (int p = 0; p < NQ; p++) {
        const double w = weight(p);
        const int slot = speed_slot(p);
        for (long n = 0; n < N; n++) {
            if (is_solid(solid, n)) continue;
            double x = (f[(long)p * N + n] - w) * S / w;
            double sp = stochastic ? orc_round_storage_sr(kind, x, orc_storage_bits(seed, step, n, slot), 6)
                                   : orc_round_storage(kind, x);
            f[(long)p * N + n] = w + sp * w / S;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Shape function (Sec. 2.2)                                                 */
/* ------------------------------------------------------------------------ */

/*
 * One-dimensional factor of the diffused shape function.  The printed
 * branches of Sec. 2.2 are garbled (discontinuous at |y|/xi = 1/2, negative
 * at the edge, not normalised, contradicting the normalisation the paper
 * states next); the paper cites Peskin for it, so this is Peskin's
 * four-point kernel with r = 2|y|/xi: the same support |y| <= xi, the same
 * 64-node support at xi = 2, and exactly normalised on the lattice at xi = 2.
 */
double orc_peskin(double r)
{
    r = fabs(r);
    if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) / 8.0;
    if (r <= 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) / 8.0;
    return 0.0;
}

void orc_quat_to_Q(const double q_in[4], double Q[9])
{
    double nrm = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / nrm, x = q_in[1] / nrm, y = q_in[2] / nrm, z = q_in[3] / nrm;
    Q[0] = 1.0 - 2.0 * (y * y + z * z);
    Q[1] = 2.0 * (x * y - w * z);
    Q[2] = 2.0 * (x * z + w * y);
    Q[3] = 2.0 * (x * y + w * z);
    Q[4] = 1.0 - 2.0 * (x * x + z * z);
    Q[5] = 2.0 * (y * z - w * x);
    Q[6] = 2.0 * (x * z - w * y);
    Q[7] = 2.0 * (y * z + w * x);
    Q[8] = 1.0 - 2.0 * (x * x + y * y);
}

typedef struct {
    int o[3], n[3]; /* box origin (unwrapped lattice coordinates) and size */
    long size;
    double *w, *d, *D; /* raw weight (0 at solid), normalised delta, gradient [3*size] */
    double S;
} shape_t;

static long box_index(const shape_t *sh, int i, int j, int k)
{
    return (long)i + (long)sh->n[0] * ((long)j + (long)sh->n[1] * k);
}

/*
 * Shape of a cell at pose (R, Q) on a bounding box of its support.
 *   y = Q^T (x - R)                      body coordinates (v_lab = Q v_body)
 *   w(x) = prod_alpha phi(2 y_alpha / xi_alpha)      (Sec. 2.2, reading above)
 *   delta(x) = w(x) / sum_fluid w         normalised over the fluid nodes, so
 *                                         that sum_x delta = 1 for any pose
 *                                         (the paper's normalisation holds
 *                                         only at xi = 2 and axis-aligned)
 *   Ddelta_b(x) = (delta(x+e_b) - delta(x-e_b))/2    lattice central difference
 * The box spans the axis-aligned hull of the support |y_alpha| <= xi_alpha
 * (half extent sum_alpha |Q_a alpha| xi_alpha) plus one node on every side,
 * so the gradient is complete.
 */
static void shape_compute(int nx, int ny, int nz, const unsigned char *solid,
                          const double R[3], const double Q[9], const double xi[3], shape_t *sh)
{
    for (int a = 0; a < 3; a++) {
        double e = 0.0;
        for (int b = 0; b < 3; b++) e += fabs(Q[3 * a + b]) * xi[b];
        int lo = (int)ceil(R[a] - e) - 1;
        int hi = (int)floor(R[a] + e) + 1;
        sh->o[a] = lo;
        sh->n[a] = hi - lo + 1;
    }
    sh->size = (long)sh->n[0] * sh->n[1] * sh->n[2];
    sh->w = (double *)calloc((size_t)sh->size, sizeof(double));
    sh->d = (double *)calloc((size_t)sh->size, sizeof(double));
    sh->D = (double *)calloc((size_t)sh->size * 3, sizeof(double));
    double S = 0.0;
    for (int k = 0; k < sh->n[2]; k++)
        for (int j = 0; j < sh->n[1]; j++)
            for (int i = 0; i < sh->n[0]; i++) {
                int X[3] = {sh->o[0] + i, sh->o[1] + j, sh->o[2] + k};
                long g = node_of(nx, ny, nz, X[0], X[1], X[2]);
                double w = 0.0;
                if (!is_solid(solid, g)) {
                    double r[3] = {X[0] - R[0], X[1] - R[1], X[2] - R[2]};
                    w = 1.0;
                    for (int b = 0; b < 3; b++) {
                        double y = Q[0 * 3 + b] * r[0] + Q[1 * 3 + b] * r[1] + Q[2 * 3 + b] * r[2];
                        w *= orc_peskin(2.0 * y / xi[b]);
                    }
                }
                sh->w[box_index(sh, i, j, k)] = w;
                S += w;
            }
    sh->S = S;
    for (long m = 0; m < sh->size; m++) sh->d[m] = S > 0.0 ? sh->w[m] / S : 0.0;
    for (int k = 0; k < sh->n[2]; k++)
        for (int j = 0; j < sh->n[1]; j++)
            for (int i = 0; i < sh->n[0]; i++) {
                int idx[3] = {i, j, k};
                long m = box_index(sh, i, j, k);
                for (int b = 0; b < 3; b++) {
                    int ip[3] = {idx[0], idx[1], idx[2]}, im[3] = {idx[0], idx[1], idx[2]};
                    ip[b] += 1;
                    im[b] -= 1;
                    double dp = ip[b] < sh->n[b] ? sh->d[box_index(sh, ip[0], ip[1], ip[2])] : 0.0;
                    double dm = im[b] >= 0 ? sh->d[box_index(sh, im[0], im[1], im[2])] : 0.0;
                    sh->D[3 * m + b] = 0.5 * (dp - dm);
                }
            }
}

static void shape_free(shape_t *sh)
{
    free(sh->w);
    free(sh->d);
    free(sh->D);
}

double orc_shape_field(int nx, int ny, int nz, const unsigned char *solid,
                       const double R[3], const double Q[9], const double xi[3],
                       double *w, double *delta, double *Ddelta)
{
    const long N = (long)nx * ny * nz;
    memset(w, 0, sizeof(double) * N);
    memset(delta, 0, sizeof(double) * N);
    memset(Ddelta, 0, sizeof(double) * 3 * N);
    shape_t sh;
    shape_compute(nx, ny, nz, solid, R, Q, xi, &sh);
    for (int k = 0; k < sh.n[2]; k++)
        for (int j = 0; j < sh.n[1]; j++)
            for (int i = 0; i < sh.n[0]; i++) {
                long m = box_index(&sh, i, j, k);
                long g = node_of(nx, ny, nz, sh.o[0] + i, sh.o[1] + j, sh.o[2] + k);
                w[g] += sh.w[m];
                delta[g] += sh.d[m];
                for (int b = 0; b < 3; b++) Ddelta[3 * g + b] += sh.D[3 * m + b];
            }
    double S = sh.S;
    shape_free(&sh);
    return S;
}

/* ------------------------------------------------------------------------ */
/* Sampling and spreading (Sec. 2.2)                                         */
/* ------------------------------------------------------------------------ */

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Vorticity omega = curl u by central differences at node (x, y, z); u is 0
 * at solid nodes (Sec. 2.1: the antisymmetric part has no kinetic form). */
static void vorticity(int nx, int ny, int nz, const double *u, int x, int y, int z, double om[3])
{
    long xp = node_of(nx, ny, nz, x + 1, y, z), xm = node_of(nx, ny, nz, x - 1, y, z);
    long yp = node_of(nx, ny, nz, x, y + 1, z), ym = node_of(nx, ny, nz, x, y - 1, z);
    long zp = node_of(nx, ny, nz, x, y, z + 1), zm = node_of(nx, ny, nz, x, y, z - 1);
    double dy_uz = 0.5 * (u[3 * yp + 2] - u[3 * ym + 2]);
    double dz_uy = 0.5 * (u[3 * zp + 1] - u[3 * zm + 1]);
    double dz_ux = 0.5 * (u[3 * zp + 0] - u[3 * zm + 0]);
    double dx_uz = 0.5 * (u[3 * xp + 2] - u[3 * xm + 2]);
    double dx_uy = 0.5 * (u[3 * xp + 1] - u[3 * xm + 1]);
    double dy_ux = 0.5 * (u[3 * yp + 0] - u[3 * ym + 0]);
    om[0] = dy_uz - dz_uy;
    om[1] = dz_ux - dx_uz;
    om[2] = dx_uy - dy_ux;
}

/*
 * Smeared fields of one cell (Eqs. vel, vort) and its elongational torque
 * (Eq. pheno_torque_diss):
 *   u~ = sum_x delta u,   omega~ = sum_x delta (curl u),
 *   T^S = alpha sum_x delta (sigma . n) x (x - R),   n = Ddelta/|Ddelta|.
 * Reading: n is the printed normalised gradient of delta.  It points inwards
 * (delta peaks at the centre), although the text calls it the outward
 * normal; with the outward normal the unit-normal field, whose long rims
 * carry the longest lever arms, turns a flat cell in shear away from the
 * extensional axis, against what Sec. 2.3 says the elongational part does
 * (align the cell with the principal stretching direction).  Nodes with
 * |Ddelta| = 0 have no normal and add nothing.
 */
static void sample_shape(int nx, int ny, int nz, const double *u, const double *sigma,
                         const shape_t *sh, const double R[3], double alpha,
                         double ut[3], double wt[3], double TS[3])
{
    for (int a = 0; a < 3; a++) ut[a] = wt[a] = TS[a] = 0.0;
    for (int k = 0; k < sh->n[2]; k++)
        for (int j = 0; j < sh->n[1]; j++)
            for (int i = 0; i < sh->n[0]; i++) {
                long m = box_index(sh, i, j, k);
                double d = sh->d[m];
                if (d == 0.0) continue;
                int X[3] = {sh->o[0] + i, sh->o[1] + j, sh->o[2] + k};
                long g = node_of(nx, ny, nz, X[0], X[1], X[2]);
                double om[3];
                vorticity(nx, ny, nz, u, X[0], X[1], X[2], om);
                for (int a = 0; a < 3; a++) {
                    ut[a] += d * u[3 * g + a];
                    wt[a] += d * om[a];
                }
                if (alpha != 0.0) {
                    const double *D = &sh->D[3 * m];
                    double nD = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
                    if (nD > 1e-12) {
                        double nh[3] = {D[0] / nD, D[1] / nD, D[2] / nD};
                        const double *s = &sigma[6 * g];
                        double S3[3][3] = {{s[0], s[3], s[4]}, {s[3], s[1], s[5]}, {s[4], s[5], s[2]}};
                        double t[3], r[3] = {X[0] - R[0], X[1] - R[1], X[2] - R[2]}, tx[3];
                        for (int a = 0; a < 3; a++) t[a] = S3[a][0] * nh[0] + S3[a][1] * nh[1] + S3[a][2] * nh[2];
                        cross(t, r, tx);
                        for (int a = 0; a < 3; a++) TS[a] += alpha * d * tx[a];
                    }
                }
            }
}

/*
 * Reaction of one cell on the fluid (Sec. 2.2, the body-force equation) and
 * its contribution to the relaxation time (Eq. enhance-viscosity):
 *   G(x) += -(J/h) delta(x) + 1/2 (L/h) x Ddelta(x)      at fluid nodes
 *   theta(x) += 1 - (1 - w(x))^kappa                     at fluid nodes
 * J, L are the hydrodynamic linear and (lab) angular impulses the cell took
 * this step.  Reading: the torque term's sign is the one that gives the fluid
 * -L (what the paper's angular-momentum argument states; with d/dx the
 * printed sign would give +L, i.e. the printed derivative is with respect to
 * the cell position).  theta uses the raw product w (peak 1/8, so theta ~ 0.93
 * inside), not the normalised delta, whose peak depends on xi.
 */
static void spread_shape(int nx, int ny, int nz, const shape_t *sh, double kappa,
                         const double J[3], const double L[3], double *G, double *theta)
{
    for (int k = 0; k < sh->n[2]; k++)
        for (int j = 0; j < sh->n[1]; j++)
            for (int i = 0; i < sh->n[0]; i++) {
                long m = box_index(sh, i, j, k);
                const double *D = &sh->D[3 * m];
                double d = sh->d[m];
                long g = node_of(nx, ny, nz, sh->o[0] + i, sh->o[1] + j, sh->o[2] + k);
                double Lh[3] = {L[0] / H_STEP, L[1] / H_STEP, L[2] / H_STEP}, LxD[3];
                cross(Lh, D, LxD);
                for (int a = 0; a < 3; a++) G[3 * g + a] += -(J[a] / H_STEP) * d + 0.5 * LxD[a];
                if (sh->w[m] > 0.0) theta[g] += 1.0 - pow(1.0 - sh->w[m], kappa);
            }
}

void orc_sample_cell(int nx, int ny, int nz, const unsigned char *solid,
                     const double *u, const double *sigma,
                     const double R[3], const double Q[9], const double xi[3], double alpha,
                     double ut[3], double wt[3], double TS[3])
{
    shape_t sh;
    shape_compute(nx, ny, nz, solid, R, Q, xi, &sh);
    sample_shape(nx, ny, nz, u, sigma, &sh, R, alpha, ut, wt, TS);
    shape_free(&sh);
}

void orc_spread_cell(int nx, int ny, int nz, const unsigned char *solid,
                     const double R[3], const double Q[9], const double xi[3], double kappa,
                     const double J[3], const double L[3], double *G, double *theta)
{
    shape_t sh;
    shape_compute(nx, ny, nz, solid, R, Q, xi, &sh);
    /* solid nodes carry delta = 0 but may carry a gradient; only fluid
     * nodes receive force */
    for (int k = 0; k < sh.n[2]; k++)
        for (int j = 0; j < sh.n[1]; j++)
            for (int i = 0; i < sh.n[0]; i++) {
                long g = node_of(nx, ny, nz, sh.o[0] + i, sh.o[1] + j, sh.o[2] + k);
                if (is_solid(solid, g)) {
                    long m = box_index(&sh, i, j, k);
                    sh.D[3 * m] = sh.D[3 * m + 1] = sh.D[3 * m + 2] = 0.0;
                    sh.w[m] = 0.0;
                }
            }
    spread_shape(nx, ny, nz, &sh, kappa, J, L, G, theta);
    shape_free(&sh);
}

/* ------------------------------------------------------------------------ */
/* Gay-Berne exclusion forces (Sec. 2.5, App. B)                             */
/* ------------------------------------------------------------------------ */

static void inverse3(const double A[9], double B[9])
{
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    B[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

static void matvec(const double A[9], const double v[3], double r[3])
{
    for (int a = 0; a < 3; a++) r[a] = A[3 * a] * v[0] + A[3 * a + 1] * v[1] + A[3 * a + 2] * v[2];
}

/* A = Q S^2 Q^T, Sec. 2.5 */
static void shape_matrix(const double Q[9], const double s[3], double A[9])
{
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += Q[3 * a + k] * s[k] * s[k] * Q[3 * b + k];
            A[3 * a + b] = acc;
        }
}

/*
 * Pair i, j with d = R_ij = R_i - R_j (the direction that makes the force on
 * i equal to -grad_{R_i} u, checked by finite differences):
 *   H = A_i + A_j, kappa = H^-1 R_ij, phi = 1/2 R^ . H^-1 . R^, sigma = phi^-1/2
 *   rho = (R - sigma + sigma_min) / sigma_min
 *   u = 4 eps0 (rho^-12 - rho^-6) + eps0 for rho <= 2^(1/6) else 0  (Eq. gayberne)
 *   du/dR = -24 eps0 (2 rho^-13 - rho^-7) / sigma_min
 *   du/dphi = -24 eps0 (2 rho^-13 - rho^-7) sigma^3 / (2 sigma_min)
 *   F_i = -du/dR R^ - (1/R^2) du/dphi [kappa - (kappa.R^) R^]     (Eq. forcegb)
 *   f_kappa = -(1/R^2) du/dphi kappa
 *   tau_i = (R_c - R_i) x f_kappa = (-A_i kappa) x f_kappa
 *   tau_j = (R_c - R_j) x (-f_kappa) = (-A_j kappa) x f_kappa        (lab frame)
 * Readings: f_kappa takes 1/R^2 (the printed 1/R breaks the paper's own
 * identity tau_i + tau_j = -R_ij x F_ij); the force on j at the contact point
 * R_c is -f_kappa, which is what makes that identity hold; the cutoff is the
 * positive branch rho <= 2^(1/6) (rho^6 <= 2 would drop deep overlaps);
 * rho below rho_floor is clamped to rho_floor (the paper leaves deep overlap
 * open; the clamp bounds the force and is counted).
 */
int orc_gb_pair(const double d[3], const double Ai[9], const double Aj[9],
                double sigma_min, double eps0, double rho_floor,
                double *u, double F[3], double tau_i[3], double tau_j[3])
{
    for (int a = 0; a < 3; a++) F[a] = tau_i[a] = tau_j[a] = 0.0;
    *u = 0.0;
    double H[9], Hi[9], kap[3];
    for (int k = 0; k < 9; k++) H[k] = Ai[k] + Aj[k];
    inverse3(H, Hi);
    double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double R = sqrt(R2);
    double Rh[3] = {d[0] / R, d[1] / R, d[2] / R};
    matvec(Hi, d, kap);
    double phi = 0.5 * (d[0] * kap[0] + d[1] * kap[1] + d[2] * kap[2]) / R2;
    double sigma = 1.0 / sqrt(phi);
    double rho = (R - sigma + sigma_min) / sigma_min;
    const double rho_cut = pow(2.0, 1.0 / 6.0);
    if (rho > rho_cut) return 0;
    int clamped = 0;
    if (rho < rho_floor) {
        rho = rho_floor;
        clamped = 1;
    }
    double r6 = pow(rho, -6.0), r12 = r6 * r6;
    *u = 4.0 * eps0 * (r12 - r6) + eps0;
    double core = 2.0 * pow(rho, -13.0) - pow(rho, -7.0);
    double dudR = -24.0 * eps0 * core / sigma_min;
    double dudphi = -24.0 * eps0 * core * sigma * sigma * sigma / (2.0 * sigma_min);
    double kR = kap[0] * Rh[0] + kap[1] * Rh[1] + kap[2] * Rh[2];
    double fk[3], Aik[3], Ajk[3];
    for (int a = 0; a < 3; a++) {
        F[a] = -dudR * Rh[a] - (dudphi / R2) * (kap[a] - kR * Rh[a]);
        fk[a] = -(dudphi / R2) * kap[a];
    }
    matvec(Ai, kap, Aik);
    matvec(Aj, kap, Ajk);
    for (int a = 0; a < 3; a++) {
        Aik[a] = -Aik[a];
        Ajk[a] = -Ajk[a];
    }
    cross(Aik, fk, tau_i);
    cross(Ajk, fk, tau_j);
    return clamped;
}

/* ------------------------------------------------------------------------ */
/* Rigid-body integrator (App. A)                                            */
/* ------------------------------------------------------------------------ */

/* Active right-handed rotation by angle t about body axis k. */
static void axis_rotation(int k, double t, double Rk[9])
{
    double c = cos(t), s = sin(t);
    for (int m = 0; m < 9; m++) Rk[m] = 0.0;
    int a = (k + 1) % 3, b = (k + 2) % 3;
    Rk[3 * k + k] = 1.0;
    Rk[3 * a + a] = c;
    Rk[3 * a + b] = -s;
    Rk[3 * b + a] = s;
    Rk[3 * b + b] = c;
}

/* Steps 6-7 of App. A: friction half step, then half kick with the combined
 * force (lab) and torque (body frame) evaluated at the new pose. */
void orc_rigid_close(double V[3], double Om[3], const double Fc[3], const double Tc[3],
                     double M, const double I[3], double gT, double gR)
{
    for (int a = 0; a < 3; a++) {
        Om[a] = exp(-gR * H_STEP / 2.0) * Om[a];
        V[a] = exp(-gT * H_STEP / 2.0) * V[a];
    }
    for (int a = 0; a < 3; a++) {
        V[a] = V[a] + H_STEP / (2.0 * M) * Fc[a];
        Om[a] = Om[a] + H_STEP / 2.0 * Tc[a] / I[a];
    }
}

/*
 * Steps 1-4 of App. A: half kick, friction half step, drift, and the five
 * sub-rotations about the body axes with angles h Omega_1/2, h Omega_2/2,
 * h Omega_3, h Omega_2/2, h Omega_1/2 (each angle from the current Omega).
 * Each sub-rotation R: pi = I Omega -> R^T pi, Q -> Q R.  Readings: the
 * friction of step 2 acts on the current momenta (the printed Omega_0, V_0
 * would undo step 1); Q maps body to lab and dQ/dt = Q [Omega]x (the printed
 * skew() is the transpose, which turns a cell against the fluid vorticity
 * it is coupled to).  Positions are not wrapped here.
 */
void orc_rigid_open(double R[3], double Q[9], double V[3], double Om[3],
                    const double Fc[3], const double Tc[3], double M, const double I[3],
                    double gT, double gR)
{
    for (int a = 0; a < 3; a++) {
        Om[a] = Om[a] + H_STEP / 2.0 * Tc[a] / I[a];
        V[a] = V[a] + H_STEP / (2.0 * M) * Fc[a];
    }
    for (int a = 0; a < 3; a++) {
        Om[a] = exp(-gR * H_STEP / 2.0) * Om[a];
        V[a] = exp(-gT * H_STEP / 2.0) * V[a];
    }
    for (int a = 0; a < 3; a++) R[a] = R[a] + H_STEP * V[a];
    const int axis[5] = {0, 1, 2, 1, 0};
    const double frac[5] = {0.5, 0.5, 1.0, 0.5, 0.5};
    for (int s = 0; s < 5; s++) {
        int k = axis[s];
        double t = frac[s] * H_STEP * Om[k];
        double Rk[9], pi[3], pr[3], Qn[9];
        axis_rotation(k, t, Rk);
        for (int a = 0; a < 3; a++) pi[a] = I[a] * Om[a];
        for (int a = 0; a < 3; a++) pr[a] = Rk[0 * 3 + a] * pi[0] + Rk[1 * 3 + a] * pi[1] + Rk[2 * 3 + a] * pi[2];
        for (int a = 0; a < 3; a++) Om[a] = pr[a] / I[a];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                Qn[3 * a + b] = Q[3 * a + 0] * Rk[0 * 3 + b] + Q[3 * a + 1] * Rk[1 * 3 + b] + Q[3 * a + 2] * Rk[2 * 3 + b];
        memcpy(Q, Qn, sizeof(Qn));
    }
}

/* ------------------------------------------------------------------------ */
/* Coupled solver                                                            */
/* ------------------------------------------------------------------------ */

struct orc_state {
    int nx, ny, nz, per[3];
    long N;
    unsigned char *solid;
    double gext[3], gwave[3];
    double tau0, delta, kappa, gT, gR, alpha, eps0, xi[3], a[3], M, I[3];
    double smin_w, r_w, rho_floor, rc, rcw;
    double *f, *rho, *U, *S, *G, *theta, *tau;
    long nw;
    double *wpos;
    int nc;
    double *R, *Q, *V, *Om, *Fc, *Tc;
    int *have_cache;
    double *Fm, *Tm, *ut, *wt, *TS, *J, *L;
    double *Fext, *Text; /* external force and torque per cell (lab), 3n each */
    long step, clamps;
    unsigned char *node_type; /* NULL: no open boundaries */
    double in_c[2], in_r, in_umax;
    double *fprev;
    int storage, stochastic;
    unsigned long long seed;
};

static double *dalloc(long n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

orc_state *orc_create(const orc_config *c)
{
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    s->nx = c->nx;
    s->ny = c->ny;
    s->nz = c->nz;
    for (int a = 0; a < 3; a++) s->per[a] = c->periodic[a];
    s->N = (long)c->nx * c->ny * c->nz;
    s->solid = (unsigned char *)calloc((size_t)s->N, 1);
    if (c->solid) memcpy(s->solid, c->solid, (size_t)s->N);
    for (int a = 0; a < 3; a++) {
        s->gext[a] = c->body_force[a];
        s->gwave[a] = c->body_force_wave[a];
        s->xi[a] = c->xi[a];
        s->a[a] = c->semi_axes[a];
        s->I[a] = c->inertia[a];
    }
    s->tau0 = c->tau0;
    s->delta = c->delta;
    s->kappa = c->kappa;
    s->gT = c->gamma_T;
    s->gR = c->gamma_R;
    s->alpha = c->alpha;
    s->eps0 = c->eps0;
    s->M = c->mass;
    s->smin_w = c->sigma_min_wall;
    s->r_w = c->wall_radius;
    s->rho_floor = c->rho_floor;
    s->rc = c->r_cut;
    s->rcw = c->r_cut_wall;
    s->storage = c->storage;
    s->node_type = NULL;
    if (c->node_type) {
        s->node_type = (unsigned char *)malloc((size_t)s->N);
        memcpy(s->node_type, c->node_type, (size_t)s->N);
        s->fprev = (double *)calloc((size_t)NQ * s->N, sizeof(double));
    }
    s->in_c[0] = c->inlet_center[0];
    s->in_c[1] = c->inlet_center[1];
    s->in_r = c->inlet_radius;
    s->in_umax = c->inlet_umax;
    s->stochastic = c->stochastic;
    s->seed = c->seed;

    long N = s->N;
    s->f = dalloc(NQ * N);
    s->rho = dalloc(N);
    s->U = dalloc(3 * N);
    s->S = dalloc(6 * N);
    s->G = dalloc(3 * N);
    s->theta = dalloc(N);
    s->tau = dalloc(N);
    /* initial state: f = f^eq(rho = 1, u = 0) = w_p at fluid nodes */
    for (long n = 0; n < N; n++) {
        if (s->solid[n]) continue;
        s->rho[n] = 1.0;
        for (int p = 0; p < NQ; p++) s->f[(long)p * N + n] = weight(p);
    }
    /* wall particles: solid nodes with at least one fluid node among their
     * lattice links (Sec. 2.5, last paragraph) */
    s->nw = 0;
    s->wpos = dalloc(3 * N);
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long n = node_of(s->nx, s->ny, s->nz, x, y, z);
                if (!s->solid[n]) continue;
                int wet = 0;
                for (int p = 1; p < NQ; p++)
                    if (!s->solid[node_of(s->nx, s->ny, s->nz, x + CV[p][0], y + CV[p][1], z + CV[p][2])]) wet = 1;
                if (wet) {
                    s->wpos[3 * s->nw] = x;
                    s->wpos[3 * s->nw + 1] = y;
                    s->wpos[3 * s->nw + 2] = z;
                    s->nw++;
                }
            }
    int nc = c->ncells;
    s->nc = nc;
    s->R = dalloc(3 * nc);
    s->Q = dalloc(9 * nc);
    s->V = dalloc(3 * nc);
    s->Om = dalloc(3 * nc);
    s->Fc = dalloc(3 * nc);
    s->Tc = dalloc(3 * nc);
    s->have_cache = (int *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int));
    s->Fm = dalloc(3 * nc);
    s->Tm = dalloc(3 * nc);
    s->ut = dalloc(3 * nc);
    s->wt = dalloc(3 * nc);
    s->TS = dalloc(3 * nc);
    s->J = dalloc(3 * nc);
    s->L = dalloc(3 * nc);
    s->Fext = dalloc(3 * nc);
    s->Text = dalloc(3 * nc);
    for (int k = 0; k < 3 * nc; k++) {
        if (c->force_ext) s->Fext[k] = c->force_ext[k];
        if (c->torque_ext) s->Text[k] = c->torque_ext[k];
    }
    for (int i = 0; i < nc; i++) {
        for (int a = 0; a < 3; a++) {
            s->R[3 * i + a] = c->pos[3 * i + a];
            s->V[3 * i + a] = c->vel ? c->vel[3 * i + a] : 0.0;
            s->Om[3 * i + a] = c->omega ? c->omega[3 * i + a] : 0.0;
        }
        orc_quat_to_Q(&c->quat[4 * i], &s->Q[9 * i]);
    }
    return s;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    free(s->node_type);
    free(s->fprev);
    free(s->solid);
    free(s->f);
    free(s->rho);
    free(s->U);
    free(s->S);
    free(s->G);
    free(s->theta);
    free(s->tau);
    free(s->wpos);
    free(s->R);
    free(s->Q);
    free(s->V);
    free(s->Om);
    free(s->Fc);
    free(s->Tc);
    free(s->have_cache);
    free(s->Fm);
    free(s->Tm);
    free(s->ut);
    free(s->wt);
    free(s->TS);
    free(s->J);
    free(s->L);
    free(s->Fext);
    free(s->Text);
    free(s);
}

/* Minimum image along periodic axes; positions live in [0, n). */
static void min_image(const orc_state *s, double d[3])
{
    const int n[3] = {s->nx, s->ny, s->nz};
    for (int a = 0; a < 3; a++) {
        if (!s->per[a]) continue;
        double L = (double)n[a];
        if (d[a] > 0.5 * L)
            d[a] -= L;
        else if (d[a] < -0.5 * L)
            d[a] += L;
    }
}

static double dist2(const double d[3])
{
    double r2 = d[0] * d[0];
    r2 = r2 + d[1] * d[1];
    r2 = r2 + d[2] * d[2];
    return r2;
}

/* Gay-Berne forces and torques (lab frame) on every cell: all cell pairs and
 * all cell-wall-particle pairs inside the candidate radii, by brute force.
 * A constant external force and torque on a cell (the push of the mobility
 * tests of Sec. 3) is counted with them: like the Gay-Berne forces it is a
 * non-hydrodynamic force, so it enters the combined force and torque of
 * App. A and not the impulse the cell returns to the fluid. */
static void mechanical_forces(orc_state *s)
{
    int nc = s->nc;
    double *A = dalloc(9 * nc);
    for (int i = 0; i < nc; i++) shape_matrix(&s->Q[9 * i], s->a, &A[9 * i]);
    for (int k = 0; k < 3 * nc; k++) {
        s->Fm[k] = s->Fext[k];
        s->Tm[k] = s->Text[k];
    }
    double smin_cc = sqrt(2.0 * (2.0 * pow(fmin(s->a[0], fmin(s->a[1], s->a[2])), 2.0)));
    for (int i = 0; i < nc; i++)
        for (int j = i + 1; j < nc; j++) {
            double d[3];
            for (int a = 0; a < 3; a++) d[a] = s->R[3 * i + a] - s->R[3 * j + a];
            min_image(s, d);
            if (!(dist2(d) < s->rc * s->rc)) continue;
            double u, F[3], ti[3], tj[3];
            s->clamps += orc_gb_pair(d, &A[9 * i], &A[9 * j], smin_cc, s->eps0, s->rho_floor, &u, F, ti, tj);
            for (int a = 0; a < 3; a++) {
                s->Fm[3 * i + a] += F[a];
                s->Fm[3 * j + a] -= F[a];
                s->Tm[3 * i + a] += ti[a];
                s->Tm[3 * j + a] += tj[a];
            }
        }
    /* wall particles: spheres of radius r_w, A_w = r_w^2 1, sigma_min = the
     * wall-RBC value of Sec. 2.5 */
    double Aw[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    Aw[0] = Aw[4] = Aw[8] = s->r_w * s->r_w;
    for (int i = 0; i < nc; i++)
        for (long w = 0; w < s->nw; w++) {
            double d[3];
            for (int a = 0; a < 3; a++) d[a] = s->R[3 * i + a] - s->wpos[3 * w + a];
            min_image(s, d);
            if (!(dist2(d) < s->rcw * s->rcw)) continue;
            double u, F[3], ti[3], tj[3];
            s->clamps += orc_gb_pair(d, &A[9 * i], Aw, s->smin_w, s->eps0, s->rho_floor, &u, F, ti, tj);
            for (int a = 0; a < 3; a++) {
                s->Fm[3 * i + a] += F[a];
                s->Tm[3 * i + a] += ti[a];
            }
        }
    free(A);
}

static void QT_vec(const double Q[9], const double v[3], double r[3])
{
    for (int a = 0; a < 3; a++) r[a] = Q[0 * 3 + a] * v[0] + Q[1 * 3 + a] * v[1] + Q[2 * 3 + a] * v[2];
}

/* External force density at fluid node n: uniform part plus the
 * Kolmogorov wave A sin(2 pi y / ny) (the driver of a shear flow in a
 * periodic box, reading "G_ext on fluid nodes only"). */
static void external_force(const orc_state *s, long n, double g[3])
{
    long y = (n / s->nx) % s->ny;
    double sw = sin(2.0 * M_PI * (double)y / (double)s->ny);
    for (int a = 0; a < 3; a++) g[a] = s->gext[a] + s->gwave[a] * sw;
}

/* Equilibrium of Sec. 2.1 for density r and velocity v. */
static double feq(int p, double r, const double v[3])
{
    const double c2 = 1.0 / 3.0;
    double cu = CV[p][0] * v[0] + CV[p][1] * v[1] + CV[p][2] * v[2];
    double uu = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    return weight(p) * r * (1.0 + cu / c2 + (cu * cu - c2 * uu) / (2.0 * c2 * c2));
}

/*
 * Open boundaries.  The paper drives its vessels by an inlet velocity and an
 * outlet pressure and cites, without giving, the boundary rules.  Reading:
 * boundary nodes are not collided; after each pass their post-collision
 * populations are set from the post-collision populations of the previous
 * pass (fprev), so that every node of the pass reads only the previous state:
 *   inlet node n:  f_p = f_p^eq(rho_d, u_in(x, y)), rho_d the density of the
 *                  downstream neighbour (bc_neighbour on z + 1; 1 if there
 *                  is none; the pressure floats at the inlet),
 *                  u_in = u_max (1 - r^2/R^2) z;
 *   outlet node n: f_p = f_p^eq(1, u_m) + [f_p(m) - f_p^eq(rho_m, u_m)],
 *                  m the upstream neighbour (bc_neighbour on z - 1) with its
 *                  density and velocity (rho = 1 with the neighbour's
 *                  non-equilibrium part carried over); f^eq(1, 0) if there
 *                  is none.
 * Their reported rho and u are the moments of the set populations, sigma 0.
 */
/* The neighbour a boundary node takes its state from, on the plane dz = +1
 * (inlet) or -1 (outlet): the node straight across if it is fluid, else the
 * first fluid one of (x-1, y), (x+1, y), (x, y-1), (x, y+1) on that plane
 * (a tilted vessel meets the plane obliquely); -1 if none is. */
static long bc_neighbour(const orc_state *s, int x, int y, int z, int dz)
{
    static const int off[5][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    for (int k = 0; k < 5; k++) {
        long m = node_of(s->nx, s->ny, s->nz, x + off[k][0], y + off[k][1], z + dz);
        if (!is_solid(s->solid, m)) return m;
    }
    return -1;
}

static void open_boundaries(orc_state *s)
{
    const int nx = s->nx, ny = s->ny;
    const long N = s->N, nxy = (long)nx * ny;
    for (long n = 0; n < N; n++) {
        const int t = s->node_type[n];
        if (t != ORC_NODE_INLET && t != ORC_NODE_OUTLET) continue;
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / nxy);
        double fb[NQ];
        if (t == ORC_NODE_INLET) {
            long d = bc_neighbour(s, x, y, z, 1);
            double rd = d < 0 ? 1.0 : 0.0;
            if (d >= 0)
                for (int p = 0; p < NQ; p++) rd += s->fprev[(long)p * N + d];
            double dx = x - s->in_c[0], dy = y - s->in_c[1];
            double r2 = (dx * dx + dy * dy) / (s->in_r * s->in_r);
            double v[3] = {0.0, 0.0, r2 < 1.0 ? s->in_umax * (1.0 - r2) : 0.0};
            for (int p = 0; p < NQ; p++) fb[p] = feq(p, rd, v);
        } else {
            long m = bc_neighbour(s, x, y, z, -1);
            if (m < 0) {
                const double zero[3] = {0.0, 0.0, 0.0};
                for (int p = 0; p < NQ; p++) fb[p] = feq(p, 1.0, zero);
            } else {
                double rm = 0.0, j[3] = {0.0, 0.0, 0.0};
                for (int p = 0; p < NQ; p++) {
                    double fp = s->fprev[(long)p * N + m];
                    rm += fp;
                    for (int a = 0; a < 3; a++) j[a] += fp * CV[p][a];
                }
                double v[3] = {j[0] / rm, j[1] / rm, j[2] / rm};
                for (int p = 0; p < NQ; p++) fb[p] = feq(p, 1.0, v) + (s->fprev[(long)p * N + m] - feq(p, rm, v));
            }
        }
        double r = 0.0, jj[3] = {0.0, 0.0, 0.0};
        for (int p = 0; p < NQ; p++) {
            s->f[(long)p * N + n] = fb[p];
            r += fb[p];
            for (int a = 0; a < 3; a++) jj[a] += fb[p] * CV[p][a];
        }
        s->rho[n] = r;
        for (int a = 0; a < 3; a++) s->U[3 * n + a] = jj[a] / r;
        for (int k = 0; k < 6; k++) s->S[6 * n + k] = 0.0;
    }
}

long orc_wall_shear(const orc_state *s, long *node, double *tau, long max)
{
    long cnt = 0;
    for (int z = 0; z < s->nz; z++)
        for (int y = 0; y < s->ny; y++)
            for (int x = 0; x < s->nx; x++) {
                long n = node_of(s->nx, s->ny, s->nz, x, y, z);
                if (s->solid[n]) continue;
                double nv[3] = {0.0, 0.0, 0.0};
                int any = 0;
                for (int p = 1; p < NQ; p++)
                    if (s->solid[node_of(s->nx, s->ny, s->nz, x + CV[p][0], y + CV[p][1], z + CV[p][2])]) {
                        any = 1;
                        for (int a = 0; a < 3; a++) nv[a] -= CV[p][a];
                    }
                if (!any) continue;
                double nn = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
                if (cnt < max) {
                    const double *sg = &s->S[6 * n];
                    double S3[3][3] = {{sg[0], sg[3], sg[4]}, {sg[3], sg[1], sg[5]}, {sg[4], sg[5], sg[2]}};
                    double t[3] = {0.0, 0.0, 0.0}, tn = 0.0;
                    if (nn > 0.0)
                        for (int a = 0; a < 3; a++) nv[a] /= nn;
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++) t[a] += S3[a][b] * nv[b];
                    for (int a = 0; a < 3; a++) tn += t[a] * nv[a];
                    node[cnt] = n;
                    for (int a = 0; a < 3; a++) tau[3 * cnt + a] = t[a] - tn * nv[a];
                }
                cnt++;
            }
    return cnt;
}

void orc_step(orc_state *s, long nsteps)
{
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const long N = s->N;
    const int nc = s->nc;
    const int n_[3] = {nx, ny, nz};
    for (long it = 0; it < nsteps; it++) {
        /* 1. shapes at the current poses */
        shape_t *sh = (shape_t *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(shape_t));
        for (int i = 0; i < nc; i++) shape_compute(nx, ny, nz, s->solid, &s->R[3 * i], &s->Q[9 * i], s->xi, &sh[i]);
        /* 2. mechanical forces */
        mechanical_forces(s);
        /* 3.-5. sampling, combined forces, integration */
        for (int i = 0; i < nc; i++) {
            double *R = &s->R[3 * i], *Q = &s->Q[9 * i], *V = &s->V[3 * i], *Om = &s->Om[3 * i];
            sample_shape(nx, ny, nz, s->U, s->S, &sh[i], R, s->alpha, &s->ut[3 * i], &s->wt[3 * i], &s->TS[3 * i]);
            /* App. A step 5: F^comb = F^mech + gamma_T M u~ (lab);
             * tau^comb = tau^mech + gamma_R I omega~, in the body frame, with
             * the elongational torque T^S added (Sec. 2.2 counts it in the
             * total hydrodynamic torque T = T^S + T^A) */
            double Fc[3], Tlab[3], Tb[3], wb[3], Tc[3];
            for (int a = 0; a < 3; a++) {
                Fc[a] = s->Fm[3 * i + a] + s->gT * s->M * s->ut[3 * i + a];
                Tlab[a] = s->Tm[3 * i + a] + s->TS[3 * i + a];
            }
            QT_vec(Q, Tlab, Tb);
            QT_vec(Q, &s->wt[3 * i], wb);
            for (int a = 0; a < 3; a++) Tc[a] = Tb[a] + s->gR * s->I[a] * wb[a];
            double V0[3] = {V[0], V[1], V[2]}, Om0[3] = {Om[0], Om[1], Om[2]};
            double c = s->have_cache[i] ? 1.0 : 0.5;
            if (s->have_cache[i]) orc_rigid_close(V, Om, Fc, Tc, s->M, s->I, s->gT, s->gR);
            /* open the next step; the momenta after the kick and friction
             * half steps (before the drift) give the impulses */
            for (int a = 0; a < 3; a++) {
                Om[a] = Om[a] + H_STEP / 2.0 * Tc[a] / s->I[a];
                V[a] = V[a] + H_STEP / (2.0 * s->M) * Fc[a];
            }
            for (int a = 0; a < 3; a++) {
                Om[a] = exp(-s->gR * H_STEP / 2.0) * Om[a];
                V[a] = exp(-s->gT * H_STEP / 2.0) * V[a];
            }
            /* hydrodynamic impulses: total momentum change minus the
             * mechanical impulse c h F^mech (c = 1/2 on the first step,
             * which has no closing half); angular part in the lab frame */
            double dpi[3], dL[3];
            for (int a = 0; a < 3; a++) {
                s->J[3 * i + a] = s->M * (V[a] - V0[a]) - c * H_STEP * s->Fm[3 * i + a];
                dpi[a] = s->I[a] * (Om[a] - Om0[a]);
            }
            matvec(Q, dpi, dL);
            for (int a = 0; a < 3; a++) s->L[3 * i + a] = dL[a] - c * H_STEP * s->Tm[3 * i + a];
            /* drift and rotation: the rest of orc_rigid_open with zero kick
             * and no friction (both were applied above) */
            {
                double zero[3] = {0.0, 0.0, 0.0};
                orc_rigid_open(R, Q, V, Om, zero, zero, s->M, s->I, 0.0, 0.0);
            }
            for (int a = 0; a < 3; a++) {
                if (!s->per[a]) continue;
                if (R[a] >= n_[a])
                    R[a] -= n_[a];
                else if (R[a] < 0.0)
                    R[a] += n_[a];
            }
            for (int a = 0; a < 3; a++) {
                s->Fc[3 * i + a] = Fc[a];
                s->Tc[3 * i + a] = Tc[a];
            }
            s->have_cache[i] = 1;
        }
        /* 6. spreading: force density and relaxation time */
        for (long n = 0; n < N; n++) {
            for (int a = 0; a < 3; a++) s->G[3 * n + a] = 0.0;
            s->theta[n] = 0.0;
        }
        for (int i = 0; i < nc; i++) spread_shape(nx, ny, nz, &sh[i], s->kappa, &s->J[3 * i], &s->L[3 * i], s->G, s->theta);
        for (long n = 0; n < N; n++) {
            if (s->solid[n]) {
                for (int a = 0; a < 3; a++) s->G[3 * n + a] = 0.0;
                s->tau[n] = s->tau0;
                continue;
            }
            double gx[3];
            external_force(s, n, gx);
            for (int a = 0; a < 3; a++) s->G[3 * n + a] += gx[a];
            /* Eq. enhance-viscosity with h = 1 */
            s->tau[n] = s->tau0 + s->delta * H_STEP * s->theta[n];
        }
        for (int i = 0; i < nc; i++) shape_free(&sh[i]);
        free(sh);
        /* 7. lattice pass */
        if (s->node_type) memcpy(s->fprev, s->f, sizeof(double) * NQ * (size_t)N);
        orc_lb_pass(nx, ny, nz, s->solid, s->f, s->G, s->tau, s->rho, s->U, s->S);
        if (s->node_type) open_boundaries(s);
        /* 8. storage of the post-collision populations (reduced-precision
         * variants only) */
        store_populations(s->storage, s->stochastic, s->seed, s->step, N, s->solid, s->f);
        s->step++;
    }
}

long orc_step_count(const orc_state *s) { return s->step; }

void orc_populations(const orc_state *s, double *f) { memcpy(f, s->f, sizeof(double) * NQ * (size_t)s->N); }

void orc_set_populations(orc_state *s, const double *f)
{
    memcpy(s->f, f, sizeof(double) * NQ * (size_t)s->N);
    for (long n = 0; n < s->N; n++)
        for (int p = 0; p < NQ; p++) {
            if (!is_solid(s->solid, n)) continue;
            s->f[(long)p * s->N + n] = 0.0;
        }
    /* a prescribed state is stored by rounding to nearest */
    store_populations(s->storage, 0, 0, 0, s->N, s->solid, s->f);
}
long orc_clamps(const orc_state *s) { return s->clamps; }

void orc_fields(const orc_state *s, double *rho, double *u, double *sigma)
{
    if (rho) memcpy(rho, s->rho, sizeof(double) * s->N);
    if (u) memcpy(u, s->U, sizeof(double) * 3 * s->N);
    if (sigma) memcpy(sigma, s->S, sizeof(double) * 6 * s->N);
}

void orc_set_sampled_fields(orc_state *s, const double *u, const double *sigma)
{
    if (u) memcpy(s->U, u, sizeof(double) * 3 * s->N);
    if (sigma) memcpy(s->S, sigma, sizeof(double) * 6 * s->N);
}

void orc_cells(const orc_state *s, double *out)
{
    for (int i = 0; i < s->nc; i++) {
        double *o = &out[18 * i];
        for (int a = 0; a < 3; a++) o[a] = s->R[3 * i + a];
        for (int k = 0; k < 9; k++) o[3 + k] = s->Q[9 * i + k];
        for (int a = 0; a < 3; a++) {
            o[12 + a] = s->V[3 * i + a];
            o[15 + a] = s->Om[3 * i + a];
        }
    }
}

void orc_diag(const orc_state *s, double *out)
{
    for (int i = 0; i < s->nc; i++) {
        double *o = &out[21 * i];
        for (int a = 0; a < 3; a++) {
            o[a] = s->Fm[3 * i + a];
            o[3 + a] = s->Tm[3 * i + a];
            o[6 + a] = s->ut[3 * i + a];
            o[9 + a] = s->wt[3 * i + a];
            o[12 + a] = s->TS[3 * i + a];
            o[15 + a] = s->J[3 * i + a];
            o[18 + a] = s->L[3 * i + a];
        }
    }
}

/* mass and momentum of the stored (post-collision) populations, and the
 * momentum of the cells */
void orc_budget(const orc_state *s, double *out)
{
    double m = 0.0, P[3] = {0.0, 0.0, 0.0}, Pc[3] = {0.0, 0.0, 0.0};
    for (long n = 0; n < s->N; n++) {
        if (s->solid[n]) continue;
        for (int p = 0; p < NQ; p++) {
            double fp = s->f[(long)p * s->N + n];
            m += fp;
            for (int a = 0; a < 3; a++) P[a] += fp * CV[p][a];
        }
    }
    for (int i = 0; i < s->nc; i++)
        for (int a = 0; a < 3; a++) Pc[a] += s->M * s->V[3 * i + a];
    double W = 0.0;
    for (long n = 0; n < s->N; n++) {
        if (s->solid[n]) continue;
        double g[3];
        external_force(s, n, g);
        for (int a = 0; a < 3; a++) W += g[a] * s->U[3 * n + a];
    }
    out[0] = m;
    for (int a = 0; a < 3; a++) {
        out[1 + a] = P[a];
        out[4 + a] = Pc[a];
    }
    out[7] = W;
}

/* Fluid nodes in canonical lattice order: n = x + nx (y + ny z) ascending,
 * i.e. z-major, then y, then x (the indexing a sparse store of the fluid
 * nodes keeps). */
long orc_fluid_nodes(const orc_state *s, long *nodes, long max)
{
    long k = 0;
    for (long n = 0; n < s->N; n++) {
        if (s->solid[n]) continue;
        if (k < max) nodes[k] = n;
        k++;
    }
    return k;
}

long orc_neighbor_pairs(const orc_state *s, int *pairs, long max)
{
    long np = 0;
    for (int i = 0; i < s->nc; i++)
        for (int j = i + 1; j < s->nc; j++) {
            double d[3];
            for (int a = 0; a < 3; a++) d[a] = s->R[3 * i + a] - s->R[3 * j + a];
            min_image(s, d);
            if (dist2(d) < s->rc * s->rc) {
                if (np < max) {
                    pairs[2 * np] = i;
                    pairs[2 * np + 1] = j;
                }
                np++;
            }
        }
    return np;
}
