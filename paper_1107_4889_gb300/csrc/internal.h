// internal.h -- device buffers of one solver instance and the kernel
// launchers the host runtime (api.cu) calls.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace rbc {

// Per-cell shape header (floats; integer fields stored bit-cast):
// Q[9] body->lab, base[3] = box origin - R, origin[3], dims[3], centre node, ok.
constexpr int kHdrWords = 20;

// Flags word indices (device int[8]).
enum { FLAG_UNSTABLE = 0, FLAG_OVERFLOW = 1, FLAG_TIMEOUT = 2 };
enum { OVF_BIN = 1, OVF_NBR = 2, OVF_BOX = 4 };

struct Dev {
    // lattice: planes of Np floats (N rounded up to 64), node n = x + nx*(y + ny*z)
    int nx, ny, nz, N;
    long long Np;
    int walls;          // any solid node
    float *pops[2];     // 19 planes: deviations d_p = f_p - w_p of post-collision populations
    float *U;           // 3 planes: velocity of the last lattice pass
    float *S;           // 6 planes (xx yy zz xy xz yz): stress of the last pass, or null
    float *G;           // 3 planes: force density accumulated by the cells (zeroed by the pass)
    float *theta;       // 1 plane: sum of smoothed characteristic functions (zeroed by the pass)
    float *rho;         // 1 plane: density for field output
    uint8_t *solid;     // N bytes or null
    uint32_t *links;    // N words or null: bit p (1..18) = node + c_p is solid, bit 31 = node is solid
    // cells (SoA FP64)
    int nc;
    double *R, *q, *V, *Om;  // 3n, 4n, 3n, 3n
    double *A;               // 6n shape tensors (xx yy zz xy xz yz)
    float *Rf, *Af;          // 3n, 6n FP32 copies of positions and shape tensors (prefilters)
    double *Fm, *Tm;         // 3n GB force, 3n GB torque (lab)
    int *have;               // n: cached combined force exists (not the first step)
    double *diag;            // 21n per-cell diagnostics of the last step
    float *hdr;              // kHdrWords per cell: shape header built by k_bin
    // shape lists written by k_weights, two buffers (step parity): per cell
    // up to sp_cap entries (lattice node, packed box coordinates) and
    // (w, dw/dx, dw/dy, dw/dz) where w or its gradient is non-zero, their
    // count and the normalisation S = sum w
    int sp_cap;
    int2 *sp_idx[2];         // n * sp_cap
    float4 *sp_val[2];       // n * sp_cap
    int *sp_cnt[2];          // n
    float *sp_S[2];          // n
    // cell list
    int nb[3], nbins, bin_cap;
    double bin_size[3];
    int *bin_count, *bin_cells, *cell_bin;
    int max_nbr;
    int *nbr, *nbr_count;
    // wall particles, binned in a grid of their own (bins >= the wall radius)
    int nw, wnb[3], nwbins;
    double wbin_size[3];
    int *wall_start;  // nwbins + 1
    int *wall_xyz;    // 3 * nw, bin-sorted
    // status
    int *flags;                     // 8 ints
    unsigned long long *clamps;     // 1
    double *budget_part;            // budget_blocks * 8
    double *budget_out;             // 16: mass, p_fluid(3), max|u|, NaN count, p_cells(3)
    int budget_blocks;
    // lattice pass launch: grid of the row-staged kernel (0: one thread per node)
    int lb_grid, lb_stages;
    int *lb_work;  // lattice-pass batch counter and finished-CTA count (zero between launches)
    int side_prio;  // launch priority of the side-stream kernels (the device's highest)
    size_t lb_smem;
};

struct Params {
    float gext[3];
    float tau0, delta, kappa, alpha;
    float mach2;
    float xi[3];
    double a2[3];
    double M, I[3], iM, iI[3], eT, eR, gT, gR;
    double eps0, smin_cc, smin_w, rw2, rho_floor, rho_cut, rc2, rcw2;
    int periodic[3];
    int box_max;  // largest shape box (nodes)
    int sup_cap;  // bound on the support nodes of one cell: prod_b (2 xi_b + sqrt 3 + 0.01)
    int box_dim;  // largest shape box edge (nodes)
};

// lb.cu
void prepare_lb(Dev &d);
void launch_lb(const Dev &d, const Params &p, int parity, cudaStream_t s);
void launch_rho(const Dev &d, int parity, cudaStream_t s);
void launch_budget(const Dev &d, const Params &p, int parity, cudaStream_t s);
int budget_blocks_for(int N);

// cells.cu
void launch_bin(const Dev &d, const Params &p, cudaStream_t s);
void launch_gb(const Dev &d, const Params &p, cudaStream_t s);
void launch_weights(const Dev &d, const Params &p, int buf, cudaStream_t s);
void launch_cells(const Dev &d, const Params &p, int buf, cudaStream_t s);
size_t cells_smem_bytes(const Params &p);
void prepare_cells(const Params &p);

}  // namespace rbc
