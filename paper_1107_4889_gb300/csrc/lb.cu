// lb.cu -- the fused D3Q19 lattice pass and the lattice reductions.
//
// One thread per lattice node.  Populations are stored as FP32 deviations
// d_p = f_p - w_p from the lattice weights, one plane of Np floats per speed
// (x fastest), ping-ponged between two buffers.  The pass pulls the 19
// post-collision deviations of the previous pass from the upstream nodes
// (halfway bounce-back from solid upstream nodes), reads and clears the force
// density and the smoothed hematocrit the cells spread, collides, stores the
// 19 new deviations to its own node and writes u and sigma for the cells to
// sample.  Bytes per fluid node: 76 read + 76 write (populations), 16 read
// (G, theta), 12 written (u), 24 written (sigma when alpha != 0), plus the
// 16-byte clear of G and theta.
#include "internal.h"
#include "rbc_device.cuh"

namespace rbc {

namespace {

constexpr int kLbThreads = 256;

__device__ __forceinline__ int wrapm(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Collision (Sec. 2.1), in deviations.  With drho = sum d, j = sum c d:
//   rho = 1 + drho, u = (j + G/2) / rho                       (Eqs. dens, vel)
//   f_eq - w = w [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)]
//   Df = (1 - 1/2T) w [3 c.G + 4.5 (c.G)(c.u) - 1.5 G.u]       (Eq. chen_force,
//        force-density G, Guo's factor of the scheme Eq. vel comes from)
//   d* = d - (d - d_eq)/T + Df                                (Eq. lbe_discrete)
//   sigma = -(1 - 1/2T) sum c c (d - d_eq)                    (Eq. stresstensorLB)
template <bool WALLS, bool CELLS, bool SIGMA>
__global__ void __launch_bounds__(kLbThreads)
k_lb(const float *__restrict__ src, float *__restrict__ dst, const uint8_t *__restrict__ solid,
     float *__restrict__ G, float *__restrict__ th, float *__restrict__ U, float *__restrict__ S,
     int *__restrict__ flags, int nx, int ny, int nz, int N, long long Np, float gx0, float gy0,
     float gz0, float tau0, float delta, float mach2)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    if (WALLS && solid[n]) return;
    const int x = n % nx;
    const int t = n / nx;
    const int y = t % ny;
    const int z = t / ny;
    const int nxy = nx * ny;
    // upstream coordinates x - c
    const int xs[3] = {x, wrapm(x - 1, nx), wrapm(x + 1, nx)};        // c_x = 0, +1, -1
    const int ys[3] = {y * nx, wrapm(y - 1, ny) * nx, wrapm(y + 1, ny) * nx};
    const int zs[3] = {z * nxy, wrapm(z - 1, nz) * nxy, wrapm(z + 1, nz) * nxy};

    float d[kQ];
#pragma unroll
    for (int p = 0; p < kQ; ++p) {
        const int ix = cx(p) == 0 ? 0 : (cx(p) > 0 ? 1 : 2);
        const int iy = cy(p) == 0 ? 0 : (cy(p) > 0 ? 1 : 2);
        const int iz = cz(p) == 0 ? 0 : (cz(p) > 0 ? 1 : 2);
        const int s = xs[ix] + ys[iy] + zs[iz];
        if (WALLS && p != 0 && solid[s])
            d[p] = src[(long long)opp(p) * Np + n];
        else
            d[p] = src[(long long)p * Np + s];
    }

    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int p = 0; p < kQ; ++p) {
        drho += d[p];
        if (cx(p)) jx += cx(p) > 0 ? d[p] : -d[p];
        if (cy(p)) jy += cy(p) > 0 ? d[p] : -d[p];
        if (cz(p)) jz += cz(p) > 0 ? d[p] : -d[p];
    }
    float gx = gx0, gy = gy0, gz = gz0, T = tau0;
    if (CELLS) {
        gx += G[n];
        gy += G[Np + n];
        gz += G[2 * Np + n];
        T += delta * th[n];
        G[n] = 0.f;
        G[Np + n] = 0.f;
        G[2 * Np + n] = 0.f;
        th[n] = 0.f;
    }
    const float rho = 1.0f + drho;
    const float irho = 1.0f / rho;
    const float ux = (jx + 0.5f * gx) * irho;
    const float uy = (jy + 0.5f * gy) * irho;
    const float uz = (jz + 0.5f * gz) * irho;
    const float om = 1.0f / T;
    const float ff = 1.0f - 0.5f * om;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float gu = gx * ux + gy * uy + gz * uz;
    float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
    for (int p = 0; p < kQ; ++p) {
        const float cu = float(cx(p)) * ux + float(cy(p)) * uy + float(cz(p)) * uz;
        const float cg = float(cx(p)) * gx + float(cy(p)) * gy + float(cz(p)) * gz;
        const float w = wq(p);
        const float deq = w * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
        const float df = ff * w * (3.0f * cg + 4.5f * cg * cu - 1.5f * gu);
        const float neq = d[p] - deq;
        if (SIGMA) {
            if (cx(p)) pxx += neq;
            if (cy(p)) pyy += neq;
            if (cz(p)) pzz += neq;
            if (cx(p) && cy(p)) pxy += cx(p) * cy(p) > 0 ? neq : -neq;
            if (cx(p) && cz(p)) pxz += cx(p) * cz(p) > 0 ? neq : -neq;
            if (cy(p) && cz(p)) pyz += cy(p) * cz(p) > 0 ? neq : -neq;
        }
        dst[(long long)p * Np + n] = d[p] - om * neq + df;
    }
    U[n] = ux;
    U[Np + n] = uy;
    U[2 * Np + n] = uz;
    if (SIGMA) {
        S[n] = -ff * pxx;
        S[Np + n] = -ff * pyy;
        S[2 * Np + n] = -ff * pzz;
        S[3 * Np + n] = -ff * pxy;
        S[4 * Np + n] = -ff * pxz;
        S[5 * Np + n] = -ff * pyz;
    }
    if (!(rho > 0.0f) || !(usq <= mach2)) atomicOr(&flags[FLAG_UNSTABLE], 1);
}

__global__ void k_rho(const float *__restrict__ pops, const uint8_t *__restrict__ solid,
                      float *__restrict__ rho, int N, long long Np)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    if (solid && solid[n]) {
        rho[n] = 0.f;
        return;
    }
    float s = 0.f;
#pragma unroll
    for (int p = 0; p < kQ; ++p) s += pops[(long long)p * Np + n];
    rho[n] = s;  // rho - 1: the host adds 1 in FP64
}

// Budgets (Sec. 2.2 conservation claims): per block FP64 partial sums of the
// zeroth and first moments of the stored populations over fluid nodes, the
// max |u|^2 of the last pass and a NaN count; a single block then sums the
// partials in a fixed order and adds the cell momenta sum M V.
constexpr int kBudThreads = 256;

__global__ void __launch_bounds__(kBudThreads)
k_budget_nodes(const float *__restrict__ pops, const float *__restrict__ U,
               const uint8_t *__restrict__ solid, double *__restrict__ part, int N, long long Np)
{
    double m = 0.0, px = 0.0, py = 0.0, pz = 0.0, umax = 0.0, nan = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        if (solid && solid[n]) continue;
        float s = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int p = 0; p < kQ; ++p) {
            const float v = pops[(long long)p * Np + n];
            s += v;
            if (cx(p)) jx += cx(p) > 0 ? v : -v;
            if (cy(p)) jy += cy(p) > 0 ? v : -v;
            if (cz(p)) jz += cz(p) > 0 ? v : -v;
        }
        m += 1.0 + (double)s;
        px += jx;
        py += jy;
        pz += jz;
        const float ux = U[n], uy = U[Np + n], uz = U[2 * Np + n];
        const float u2 = ux * ux + uy * uy + uz * uz;
        if (!(u2 == u2) || !(s == s)) nan += 1.0;
        else if (u2 > umax) umax = u2;
    }
    __shared__ double sh[6][kBudThreads];
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = px;
    sh[2][threadIdx.x] = py;
    sh[3][threadIdx.x] = pz;
    sh[4][threadIdx.x] = umax;
    sh[5][threadIdx.x] = nan;
    __syncthreads();
    for (int w = kBudThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int k = 0; k < 6; ++k) {
                if (k == 4)
                    sh[k][threadIdx.x] = fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
                else
                    sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kBudThreads)
k_budget_final(const double *__restrict__ part, int nblocks, const double *__restrict__ V, int nc,
               double M, double *__restrict__ out)
{
    __shared__ double sh[9][kBudThreads];
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        for (int k = 0; k < 6; ++k) {
            const double v = part[b * 8 + k];
            acc[k] = k == 4 ? fmax(acc[k], v) : acc[k] + v;
        }
    }
    for (int i = threadIdx.x; i < nc; i += blockDim.x)
        for (int a = 0; a < 3; ++a) acc[6 + a] += M * V[3 * i + a];
    for (int k = 0; k < 9; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kBudThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 9; ++k)
                sh[k][threadIdx.x] = k == 4 ? fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w])
                                            : sh[k][threadIdx.x] + sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // mass, p_fluid (3), max |u|, NaN count, p_cells (3)
        for (int k = 0; k < 9; ++k) out[k] = k == 4 ? sqrt(sh[4][0]) : sh[k][0];
    }
}

}  // namespace

void launch_lb(const Dev &d, const Params &p, int parity, cudaStream_t s)
{
    const float *src = d.pops[parity];
    float *dst = d.pops[parity ^ 1];
    const int grid = (d.N + kLbThreads - 1) / kLbThreads;
    const bool cells = d.nc > 0, sig = d.S != nullptr, walls = d.walls != 0;
#define RBC_LB(W, C, S_)                                                                          \
    k_lb<W, C, S_><<<grid, kLbThreads, 0, s>>>(src, dst, d.solid, d.G, d.theta, d.U, d.S, d.flags, \
                                               d.nx, d.ny, d.nz, d.N, d.Np, p.gext[0], p.gext[1], \
                                               p.gext[2], p.tau0, p.delta, p.mach2)
    if (walls) {
        if (cells) {
            if (sig) RBC_LB(true, true, true); else RBC_LB(true, true, false);
        } else {
            if (sig) RBC_LB(true, false, true); else RBC_LB(true, false, false);
        }
    } else {
        if (cells) {
            if (sig) RBC_LB(false, true, true); else RBC_LB(false, true, false);
        } else {
            if (sig) RBC_LB(false, false, true); else RBC_LB(false, false, false);
        }
    }
#undef RBC_LB
}

void launch_rho(const Dev &d, int parity, cudaStream_t s)
{
    k_rho<<<(d.N + 255) / 256, 256, 0, s>>>(d.pops[parity], d.solid, d.rho, d.N, d.Np);
}

int budget_blocks_for(int N)
{
    int b = (N + kBudThreads * 8 - 1) / (kBudThreads * 8);
    return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

void launch_budget(const Dev &d, const Params &p, int parity, cudaStream_t s)
{
    k_budget_nodes<<<d.budget_blocks, kBudThreads, 0, s>>>(d.pops[parity], d.U, d.solid,
                                                           d.budget_part, d.N, d.Np);
    k_budget_final<<<1, kBudThreads, 0, s>>>(d.budget_part, d.budget_blocks, d.V, d.nc, p.M,
                                             d.budget_out);
}

}  // namespace rbc
