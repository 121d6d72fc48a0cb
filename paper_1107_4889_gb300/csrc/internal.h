// internal.h -- device buffers of one solver instance and the kernel
// launchers the host runtime (api.cu) calls.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct rbc_handle;

namespace rbc {

using rbc_handle_t = ::rbc_handle;

// Per-cell shape header (floats; integer fields stored bit-cast):
// Q[9] body->lab, base[3] = box origin - R, origin[3], dims[3], centre node, ok.
constexpr int kHdrWords = 20;

// Compact lattice pass: at most kMaxSegs row segments per batch, each
// described by kSegDescs int2 in the descriptor pool (nine upstream copies,
// (y, z), (c0 | c1 << 16, X0 | W << 16), (offset in the stage's planes, 0)).
constexpr int kMaxSegs = 16;
constexpr int kSegDescs = 12;

// Flags word indices (device int[8]).
enum { FLAG_UNSTABLE = 0, FLAG_OVERFLOW = 1, FLAG_TIMEOUT = 2 };
enum { OVF_BIN = 1, OVF_NBR = 2, OVF_BOX = 4 };

// Population storage (values of rbc_params.precision).
enum { PREC_F32 = 0, PREC_F16 = 1, PREC_BF16 = 2 };

struct Dev {
    // lattice: planes of Np floats (N rounded up to 64), node n = x + nx*(y + ny*z)
    int nx, ny, nz, N;
    long long Np;
    int walls;          // any solid node
    // 19 planes of post-collision populations: FP32 deviations d_p = f_p - w_p
    // (PREC_F32), or d_p / w_p scaled and rounded to binary16 / bfloat16
    int prec, stochastic;
    unsigned long long seed;  // key of the stochastic rounding's random numbers
    void *pops[2];
    // node-major vectors, so that the per-cell gathers and the spread take
    // one access per node
    float4 *U;          // Np: velocity of the last lattice pass (x, y, z, 0)
    float4 *S;          // Np: stress of the last pass, (xx yy zz xy) (its xz sits in U.w), or null
    float *Syz;         // Np: stress yz of the last pass, or null
    float4 *G;          // Np: force density (x, y, z) and sum of smoothed characteristic
                        // functions (w), accumulated by the cells, zeroed by the pass
    float *rho;         // 1 plane: density for field output
    uint8_t *solid;     // N bytes or null
    uint32_t *links;    // N words or null: bit p (1..18) = node + c_p is solid, bit 29 = inlet node,
                        // bit 30 = outlet node, bit 31 = node is solid
    uint32_t *fluid_list;  // node-list pass: the fluid nodes in lattice order, or null
    int nfluid;
    // Compact layout (walled lattices with solid rows or row segments).  Only
    // the entries of each lattice row (y, z) that a fluid node can reach
    // through a link are stored: the row's span [s_lo, s_hi) of x, the hull
    // of the fluid nodes of the nine rows (y + dy, z + dz) widened by one
    // node, rounded out to whole 32-byte sectors, or the whole row when that hull
    // wraps around x.  rows[y + ny z] = (offset of the row's first entry,
    // s_lo, s_hi, fluid x-range lo | hi << 16; lo > hi for a row without
    // fluid).  Every field array then holds M entries in lattice order plus
    // one entry `zero_entry` = M that nothing writes (a node without storage
    // reads u = 0 there).  Dense layout: entry = lattice node, rows null.
    int compact;
    int M, zero_entry;
    const int4 *rows;
    const int4 *lb_batches;  // compact lattice pass: (first descriptor in lb_pool, segments | entries << 8, bytes, 0)
    const int2 *lb_pool;     // per batch segment kSegDescs descriptors (nine upstream rows, position, window)
    int nbatches;
    // wall shear stress: wall-adjacent fluid nodes, unit normals into the
    // fluid (3 floats each), time sums of the tangential traction
    int nwss;
    int *wss_node;
    float *wss_n;
    double *wss_acc;
    // cells (SoA FP64)
    int nc;
    double *R, *q, *V, *Om;  // 3n, 4n, 3n, 3n
    double *A;               // 6n shape tensors (xx yy zz xy xz yz)
    float *Rf, *Af;          // 3n, 6n FP32 copies of positions and shape tensors (prefilters)
    double *Fm, *Tm;         // 3n GB force, 3n GB torque (lab), external force and torque included
    double *ext;             // 6n external force (3) and torque (3) per cell (lab), or null
    int *have;               // n: cached combined force exists (not the first step)
    double *diag;            // 21n per-cell diagnostics of the last step
    float *jl;               // 8n: J / S, L / 2S and a go flag of the step, from k_cells to k_spread
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
    double *budget_out;             // 16: mass, p_fluid(3), max|u|, NaN count, p_cells(3), work rate
    double *accum;                  // 8: time-average sums of a served solve (k_budget_final)
    double *profile;                // max(nx, ny, nz): cell-centre counts per 1-lu bin (k_profile)
    int budget_blocks;
    // lattice pass launch: grid of the row-staged kernel (0: one thread per node)
    int lb_grid, lb_stages;
    int *lb_work;  // lattice-pass batch counter and finished-CTA count (zero between launches)
    unsigned long long *lb_step;  // lattice passes done (advanced by the pass itself)
    int side_prio;  // launch priority of the side-stream kernels (the device's highest)
    int wt_grid = 0, gb_grid = 0;  // blocks of the shape-list and Gay-Berne launches (0: one per group)
    size_t lb_smem;
    int lb_stage_bytes;  // compact lattice pass: bytes of one stage (its largest batch)
    long long wait_cycles = 0;  // bound of the staged passes' mbarrier waits (0: the default, ~2 s)
    int starve_batch = -1;      // fault injection: a batch the staged passes never fill (-1: none)
};

struct Params {
    float gext[3];
    float gwave[3];  // amplitude of the force profile sin(2 pi y / ny)
    int wave;        // gwave != 0
    float in_c[2], in_ir2, in_umax;  // inlet profile: centre, 1 / radius^2, peak velocity
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

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (never
// lowers it: solves of different shapes may launch the same kernel from
// several threads).
void raise_smem_limit(const void *func, int bytes);

// lb.cu
int pop_bytes(int prec);  // bytes of one stored population
void prepare_lb(Dev &d);
int lb_shapes(const Dev &d, int *stages, int *ctas_per_sm, int max);  // staged-pass shapes to try
void set_lb_shape(Dev &d, int stages, int ctas_per_sm);
void launch_lb(const Dev &d, const Params &p, int parity, cudaStream_t s);
void launch_rho(const Dev &d, int parity, cudaStream_t s);
void launch_wss(const Dev &d, cudaStream_t s);
void launch_budget(const Dev &d, const Params &p, int parity, cudaStream_t s, bool accumulate = false,
                   long long from = 0);
int budget_blocks_for(int N);

// Packs of solves of one class (request server): device tables of per-solve
// kernel arguments; start[kind] (device, ninst + 1 ints) is the first block
// of each solve in the packed launch of that kind, blocks[kind] the total.
enum { PACK_CLEAR = 0, PACK_BIN = 1, PACK_GB = 2, PACK_WEIGHTS = 3, PACK_CELLS = 4, PACK_KINDS = 5 };
struct CellPackDesc {
    const void *tab;  // ninst CellPackEntry (cells.cu)
    const int *start[PACK_KINDS];
    int blocks[PACK_KINDS];
    int ninst;
};
struct LbPackDesc {
    const void *tab;     // ninst LbPackEntry (lb.cu)
    const int *bstart;   // ninst + 1: first batch of each solve
    int total, ninst;    // batches
    int *work;           // 2 ints, zero between launches
    int grid, stages, stage_bytes;
    size_t smem;
};

// lb.cu (packs)
size_t lb_pack_entry_bytes();
bool fill_lb_pack_entry(const Dev &d, const Params &p, void *out, int *nbatches, int *stage_bytes);
bool prepare_lb_pack(const Dev &d0, LbPackDesc &k);  // sets grid, stages, smem from stage_bytes, total
void launch_lb_packed(const Dev &d0, const LbPackDesc &k, int parity, cudaStream_t s);

// cells.cu
size_t cell_pack_entry_bytes();
int cell_pack_blocks(int nc, int nbins, int kind);
void fill_cell_pack_entry(const Dev &d, const Params &p, void *out);
void launch_cells_packed(const CellPackDesc &k, int buf, bool alpha, cudaStream_t s);
void launch_bin_packed(const CellPackDesc &k, int prio, cudaStream_t s);
void launch_gb_packed(const CellPackDesc &k, int prio, cudaStream_t s);
void launch_weights_packed(const CellPackDesc &k, const Params &p, int buf, int prio, cudaStream_t s);
void launch_bin(const Dev &d, const Params &p, cudaStream_t s);
void launch_profile(const Dev &d, int axis, cudaStream_t s);
void launch_gb(const Dev &d, const Params &p, cudaStream_t s);
void launch_weights(const Dev &d, const Params &p, int buf, cudaStream_t s);
// split: the per-cell kernel stops after the rigid update (J, L to d.jl)
// and launch_spread spreads them
void launch_cells(const Dev &d, const Params &p, int buf, cudaStream_t s, bool split = false);
void launch_spread(const Dev &d, const Params &p, int buf, cudaStream_t s);
size_t cells_smem_bytes(const Params &p);
void prepare_cells(const Params &p);

// api.cu, for the request server (serve.cu)
int capture_ticks(rbc_handle_t *h, int64_t steps, long long average_from, cudaGraphExec_t *out);
void advance_steps(rbc_handle_t *h, int64_t steps);
const Dev &handle_dev(const rbc_handle_t *h);
const Params &handle_params(const rbc_handle_t *h);
int read_accum(rbc_handle_t *h, double accum[8], int flags[8]);
void set_thread_error(const char *msg);

}  // namespace rbc
