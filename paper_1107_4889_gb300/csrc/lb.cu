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
// (G, theta), 12 written (u), 24 written (sigma when alpha != 0), 4 read
// (link mask, walled lattices only), plus the 16-byte clear of G and theta.
#include "internal.h"
#include "rbc_device.cuh"

namespace rbc {

namespace {

constexpr int kLbThreads = 256;

// opposite speeds for run-time indices
__constant__ int kOppTab[kQ] = {opp(0),  opp(1),  opp(2),  opp(3),  opp(4),  opp(5),  opp(6),
                                opp(7),  opp(8),  opp(9),  opp(10), opp(11), opp(12), opp(13),
                                opp(14), opp(15), opp(16), opp(17), opp(18)};

__device__ __forceinline__ int wrapm(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

struct LbArgs {
    const float *src;
    float *dst;
    const uint32_t *links;
    float *G, *th, *U, *S;
    int *flags;
    int *work;  // [0] next batch, [1] CTAs done; both zero at launch, reset by the last CTA
    int nx, ny, nz, N;
    long long Np;
    float gx0, gy0, gz0, tau0, delta, mach2;
};

// Collision (Sec. 2.1) of node n = (x, y, z), in deviations, from its 19
// pulled deviations d, the link mask lk, and the force density / smoothed
// hematocrit sums read at the node.  With drho = sum d, j = sum c d:
//   rho = 1 + drho, u = (j + G/2) / rho                       (Eqs. dens, vel)
//   f_eq - w = w [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)]
//   Df = (1 - 1/2T) w [3 c.G + 4.5 (c.G)(c.u) - 1.5 G.u]       (Eq. chen_force,
//        force-density G, Guo's factor of the scheme Eq. vel comes from)
//   d* = d - (d - d_eq)/T + Df                                (Eq. lbe_discrete)
//   sigma = -(1 - 1/2T) sum c c (d - d_eq)                    (Eq. stresstensorLB)
// Stores d*, u, sigma, clears the node's G and theta, raises the stability
// flag, and at walls writes the reflected populations (halfway bounce-back):
// a population heading into a solid neighbour m comes back to this node in
// the opposite direction next pass, so it is stored in m's slot of that
// direction, from which this node pulls.  Each (slot, solid node) pair has
// exactly one writer.
template <bool WALLS, bool CELLS, bool SIGMA>
__device__ __forceinline__ void collide_node(const LbArgs &a, float (&d)[kQ], uint32_t lk, float gx, float gy,
                                             float gz, float T, int n, int x, int y, int z)
{
    const long long Np = a.Np;
    if (CELLS) {
        a.G[n] = 0.f;
        a.G[Np + n] = 0.f;
        a.G[2 * Np + n] = 0.f;
        a.th[n] = 0.f;
    }
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int p = 0; p < kQ; ++p) {
        drho += d[p];
        if (cx(p)) jx += cx(p) > 0 ? d[p] : -d[p];
        if (cy(p)) jy += cy(p) > 0 ? d[p] : -d[p];
        if (cz(p)) jz += cz(p) > 0 ? d[p] : -d[p];
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
        a.dst[(long long)p * Np + n] = d[p] - om * neq + df;
    }
    a.U[n] = ux;
    a.U[Np + n] = uy;
    a.U[2 * Np + n] = uz;
    if (SIGMA) {
        a.S[n] = -ff * pxx;
        a.S[Np + n] = -ff * pyy;
        a.S[2 * Np + n] = -ff * pzz;
        a.S[3 * Np + n] = -ff * pxy;
        a.S[4 * Np + n] = -ff * pxz;
        a.S[5 * Np + n] = -ff * pyz;
    }
    if (!(rho > 0.0f) || !(usq <= a.mach2)) atomicOr(&a.flags[FLAG_UNSTABLE], 1);
    if (WALLS && (lk & 0x7FFFEu)) {  // nodes next to a wall only
        const int nxy = a.nx * a.ny;
#pragma unroll 1
        for (int p = 1; p < kQ; ++p) {
            if (!((lk >> p) & 1u)) continue;
            const int xd = wrapm(x + cx(p), a.nx), yd = wrapm(y + cy(p), a.ny), zd = wrapm(z + cz(p), a.nz);
            // read back this thread's own store of d*_p
            a.dst[(long long)kOppTab[p] * Np + (xd + a.nx * yd + nxy * zd)] = a.dst[(long long)p * Np + n];
        }
    }
}

// One thread per node; the 19 upstream deviations are pulled straight from
// global memory (used when rows are not a multiple of 16 bytes).
template <bool WALLS, bool CELLS, bool SIGMA>
__global__ void __launch_bounds__(kLbThreads) k_lb(LbArgs a)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = n % nx;
    const int t = n / nx;
    const int y = t % ny;
    const int z = t / ny;
    const int nxy = nx * ny;
    // upstream coordinates x - c (index 1: c = +1, index 2: c = -1)
    const int xs[3] = {x, wrapm(x - 1, nx), wrapm(x + 1, nx)};
    const int ys[3] = {y * nx, wrapm(y - 1, ny) * nx, wrapm(y + 1, ny) * nx};
    const int zs[3] = {z * nxy, wrapm(z - 1, nz) * nxy, wrapm(z + 1, nz) * nxy};
    // Pull without any test: at a wall the upstream slot is a solid node's,
    // into which this node wrote its reflected population last pass.
    const uint32_t lk = WALLS ? a.links[n] : 0u;
    float d[kQ];
#pragma unroll
    for (int p = 0; p < kQ; ++p) {
        const int ix = cx(p) == 0 ? 0 : (cx(p) > 0 ? 1 : 2);
        const int iy = cy(p) == 0 ? 0 : (cy(p) > 0 ? 1 : 2);
        const int iz = cz(p) == 0 ? 0 : (cz(p) > 0 ? 1 : 2);
        d[p] = a.src[(long long)p * a.Np + (xs[ix] + ys[iy] + zs[iz])];
    }
    float gx = a.gx0, gy = a.gy0, gz = a.gz0, T = a.tau0;
    if (CELLS) {
        gx += a.G[n];
        gy += a.G[a.Np + n];
        gz += a.G[2 * a.Np + n];
        T += a.delta * a.th[n];
    }
    if (WALLS && (lk >> 31)) return;  // solid node: nothing to collide
    collide_node<WALLS, CELLS, SIGMA>(a, d, lk, gx, gy, gz, T, n, x, y, z);
}

// ---------------------------------------------------------------------------
// Row-staged lattice pass.  A row is the nx nodes at fixed (y, z).  Every
// CTA is persistent and claims batches of B consecutive y-rows at one z from
// a global counter (CTAs that start late, behind other kernels on their SM,
// take fewer).  A producer warp brings each batch into a ring of L.stages
// shared-memory
// buffers with asynchronous bulk copies: the upstream row of every speed
// (row (y - c_y, z - c_z) of plane p) plus the batch's own rows of G, theta
// and the link mask.  The copies complete on the stage's "full" mbarrier;
// the eight consumer warps wait on it, collide the batch, and each arrives
// on the stage's "empty" mbarrier, which the producer waits on before it
// refills the stage.  No CTA-wide barrier sits in the loop, so the copy
// issue never stalls the collision.  The bytes in flight are bounded by
// shared memory, not by registers; the x shift of the pull is an index into
// the staged row.  Needs nx * 4 bytes to be a multiple of 16 (bulk-copy
// granularity).  Every wait is bounded (kWaitCycles) and raises
// FLAG_TIMEOUT; the producer then waits for its copies in flight before the
// CTA exits.
// ---------------------------------------------------------------------------
constexpr int kStConsumers = 256;                 // collision threads (8 warps)
constexpr int kStThreads = kStConsumers + 32;     // + the producer warp
constexpr int kMaxStages = 4;
constexpr int kLbCtasWithCells = 2;
constexpr int kStageBytes = 24 * 1024;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Wait for phase `parity` of the mbarrier, for at most kWaitCycles; false on
// timeout (the caller raises the timeout flag).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

struct StageLayout {
    int B;        // rows per batch
    int planes;   // staged planes per row: 19 (+4 G, theta) (+1 links)
    int stage_floats;
    int stages;   // buffers in the ring (2 .. kMaxStages)
};

template <bool WALLS, bool CELLS, bool SIGMA>
__global__ void __launch_bounds__(kStThreads) k_lb_staged(LbArgs a, StageLayout L, int nbatches)
{
    extern __shared__ __align__(128) float sm[];
    __shared__ __align__(8) unsigned long long full[kMaxStages], empty[kMaxStages];
    __shared__ int s_batch[kMaxStages];
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int B = L.B, ns = L.stages;
    const int nyb = (ny + B - 1) / B;
    if (threadIdx.x == 0) {
        for (int k = 0; k < ns; ++k) {
            mbar_init(smem_addr(&full[k]), 1);
            mbar_init(smem_addr(&empty[k]), kStConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (threadIdx.x >= kStConsumers) {
        // Producer warp.  Batches are claimed from a global counter, so a CTA
        // that starts late (the SM was busy with another kernel) just does
        // fewer of them.  A batch is rows y0 .. y0 + nb - 1 at one z.  Staged
        // plane k, batch row b sits at stage + (k * B + b) * nx.  For a speed
        // p the upstream rows y - c_y are contiguous in plane p except where
        // they wrap in y, so each plane needs one copy, or two.  The batch id
        // goes to s_batch[stage] before the arrive that the consumers'
        // wait acquires; -1 tells them to stop.
        const int lane = threadIdx.x - kStConsumers;
        const uint32_t row_bytes = (uint32_t)nx * 4u;
        int it = 0;
        bool ok = true;
        for (;; ++it) {
            const int stage = it % ns;
            if (it >= ns && !mbar_wait(smem_addr(&empty[stage]), (uint32_t)((it / ns - 1) & 1))) {
                if (lane == 0) atomicOr(&a.flags[FLAG_TIMEOUT], 1);
                ok = false;
                break;
            }
            int batch = 0;
            if (lane == 0) batch = atomicAdd(&a.work[0], 1);
            batch = __shfl_sync(0xffffffffu, batch, 0);
            const uint32_t bar = smem_addr(&full[stage]);
            if (batch >= nbatches) {
                if (lane == 0) {
                    s_batch[stage] = -1;
                    mbar_arrive(bar);
                }
                break;
            }
            const int z = batch / nyb, y0 = (batch - z * nyb) * B;
            const int nb = min(B, ny - y0);
            if (lane == 0) {
                s_batch[stage] = batch;
                mbar_expect_tx(bar, (uint32_t)(L.planes * nb) * row_bytes);
            }
            __syncwarp();
            float *base = sm + (size_t)stage * L.stage_floats;
            for (int k = lane; k < L.planes; k += 32) {
                float *dst = base + (size_t)k * B * nx;
                if (k < kQ) {
                    const int zs = wrapm(z - cz(k), nz);
                    const float *plane = a.src + (long long)k * a.Np + (long long)zs * ny * nx;
                    const int ys = y0 - cy(k);  // first upstream row, may be -1 or run past ny
                    int b = 0;
                    while (b < nb) {
                        const int yr = wrapm(ys + b, ny);
                        const int run = min(nb - b, ny - yr);
                        bulk_g2s(smem_addr(dst + (size_t)b * nx), plane + (long long)yr * nx,
                                 (uint32_t)run * row_bytes, bar);
                        b += run;
                    }
                } else {
                    const long long off = ((long long)z * ny + y0) * nx;
                    const float *src;
                    if (CELLS && k < kQ + 3)
                        src = a.G + (long long)(k - kQ) * a.Np + off;
                    else if (CELLS && k == kQ + 3)
                        src = a.th + off;
                    else
                        src = reinterpret_cast<const float *>(a.links) + off;
                    bulk_g2s(smem_addr(dst), src, (uint32_t)nb * row_bytes, bar);
                }
            }
        }
        if (!ok) {
            // let the copies still in flight land before the CTA's memory goes away
            for (int j = it > ns ? it - ns : 0; j < it; ++j)
                mbar_wait(smem_addr(&full[j % ns]), (uint32_t)((j / ns) & 1));
        }
        // the last CTA out resets the counters for the next launch
        if (lane == 0 && atomicAdd(&a.work[1], 1) == (int)gridDim.x - 1) {
            a.work[0] = 0;
            a.work[1] = 0;
            __threadfence();
        }
        return;
    }

    // consumer warps
    const int lane = threadIdx.x & 31;
    const int plane_stride = B * nx;
    for (int it = 0;; ++it) {
        const int stage = it % ns;
        if (!mbar_wait(smem_addr(&full[stage]), (uint32_t)((it / ns) & 1))) {
            if (lane == 0) atomicOr(&a.flags[FLAG_TIMEOUT], 1);
            break;
        }
        const int batch = s_batch[stage];
        if (batch < 0) break;
        const float *st = sm + (size_t)stage * L.stage_floats;
        const int z = batch / nyb, y0 = (batch - z * nyb) * B;
        const int nb = min(B, ny - y0);
        for (int l = threadIdx.x; l < nb * nx; l += kStConsumers) {
            const int b = l / nx, x = l - b * nx;
            const int y = y0 + b;
            const int n = (y + ny * z) * nx + x;
            const float *row = st + (size_t)b * nx;
            const uint32_t lk =
                WALLS ? reinterpret_cast<const uint32_t *>(row)[(size_t)(kQ + (CELLS ? 4 : 0)) * plane_stride + x] : 0u;
            if (WALLS && (lk >> 31)) continue;
            const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
            float d[kQ];
#pragma unroll
            for (int p = 0; p < kQ; ++p) {
                const int xs = cx(p) == 0 ? x : (cx(p) > 0 ? xm : xp);
                d[p] = row[p * plane_stride + xs];
            }
            float gx = a.gx0, gy = a.gy0, gz = a.gz0, T = a.tau0;
            if (CELLS) {
                gx += row[(kQ + 0) * plane_stride + x];
                gy += row[(kQ + 1) * plane_stride + x];
                gz += row[(kQ + 2) * plane_stride + x];
                T += a.delta * row[(kQ + 3) * plane_stride + x];
            }
            collide_node<WALLS, CELLS, SIGMA>(a, d, lk, gx, gy, gz, T, n, x, y, z);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[stage]));  // this warp is done with the stage
    }
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

StageLayout stage_layout(const Dev &d)
{
    StageLayout L;
    L.planes = kQ + (d.nc > 0 ? 4 : 0) + (d.walls ? 1 : 0);
    const int row_floats = d.nx;
    // about kStageBytes per stage, whole rows, at most one y column of rows;
    // a multiple of the rows that fill the consumer threads when rows are short
    int B = kStageBytes / (L.planes * row_floats * 4);
    B = B < 1 ? 1 : (B > d.ny ? d.ny : B);
    if (row_floats < kStConsumers && B * row_floats > kStConsumers)
        B -= B % (kStConsumers / row_floats > 0 ? kStConsumers / row_floats : 1);
    L.B = B;
    L.stage_floats = L.planes * B * row_floats;
    L.stages = kMaxStages;
    return L;
}

bool staged_ok(const Dev &d)
{
    if (d.nx % 4 != 0) return false;  // rows must be whole 16-byte units
    const StageLayout L = stage_layout(d);
    return 2u * L.stage_floats * sizeof(float) <= 200u * 1024u;
}

// Ring depth: among 2 .. kMaxStages stages (each depth fixes how many CTAs
// fit on an SM), take the one whose last wave of batches leaves the fewest
// idle CTA slots: time ~ ceil(batches / (SMs * k)) * k for k CTAs per SM;
// ties go to the deeper ring.  With cells, at most kLbCtasWithCells CTAs per
// SM: the next step's cell-list, Gay-Berne and shape-list kernels run
// alongside the pass and need registers and shared memory on every SM.
template <bool W, bool C, bool S_>
void prepare_lb_t(Dev &d)
{
    d.lb_grid = 0;
    if (!staged_ok(d)) return;
    StageLayout L = stage_layout(d);
    const int nbatches = d.nz * ((d.ny + L.B - 1) / L.B);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long best_cost = -1;
    for (int ns = kMaxStages; ns >= 2; --ns) {
        const size_t smem = (size_t)ns * L.stage_floats * sizeof(float);
        if (smem > 200u * 1024u) continue;
        cudaFuncSetAttribute(k_lb_staged<W, C, S_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lb_staged<W, C, S_>, kStThreads, smem);
        if (d.nc > 0 && per_sm > kLbCtasWithCells) per_sm = kLbCtasWithCells;
        if (per_sm < 1) continue;
        const long long slots = (long long)sms * per_sm;
        const long long cost = ((nbatches + slots - 1) / slots) * per_sm;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            d.lb_stages = ns;
            d.lb_smem = smem;
            d.lb_grid = (int)(slots > nbatches ? nbatches : slots);
        }
    }
    if (d.lb_grid > 0)
        cudaFuncSetAttribute(k_lb_staged<W, C, S_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.lb_smem);
}

template <bool W, bool C, bool S_>
void launch_lb_t(const Dev &d, const LbArgs &a, cudaStream_t s)
{
    if (d.lb_grid > 0) {
        StageLayout L = stage_layout(d);
        L.stages = d.lb_stages;
        const int nbatches = d.nz * ((d.ny + L.B - 1) / L.B);
        k_lb_staged<W, C, S_><<<d.lb_grid, kStThreads, d.lb_smem, s>>>(a, L, nbatches);
    } else {
        k_lb<W, C, S_><<<(d.N + kLbThreads - 1) / kLbThreads, kLbThreads, 0, s>>>(a);
    }
}

void prepare_lb(Dev &d)
{
    const bool cells = d.nc > 0, sig = d.S != nullptr, walls = d.walls != 0;
    if (walls) {
        if (cells) {
            if (sig) prepare_lb_t<true, true, true>(d); else prepare_lb_t<true, true, false>(d);
        } else {
            if (sig) prepare_lb_t<true, false, true>(d); else prepare_lb_t<true, false, false>(d);
        }
    } else {
        if (cells) {
            if (sig) prepare_lb_t<false, true, true>(d); else prepare_lb_t<false, true, false>(d);
        } else {
            if (sig) prepare_lb_t<false, false, true>(d); else prepare_lb_t<false, false, false>(d);
        }
    }
}

void launch_lb(const Dev &d, const Params &p, int parity, cudaStream_t s)
{
    LbArgs a;
    a.src = d.pops[parity];
    a.dst = d.pops[parity ^ 1];
    a.links = d.links;
    a.G = d.G;
    a.th = d.theta;
    a.U = d.U;
    a.S = d.S;
    a.flags = d.flags;
    a.work = d.lb_work;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.N = d.N;
    a.Np = d.Np;
    a.gx0 = p.gext[0];
    a.gy0 = p.gext[1];
    a.gz0 = p.gext[2];
    a.tau0 = p.tau0;
    a.delta = p.delta;
    a.mach2 = p.mach2;
    const bool cells = d.nc > 0, sig = d.S != nullptr, walls = d.walls != 0;
    if (walls) {
        if (cells) {
            if (sig) launch_lb_t<true, true, true>(d, a, s); else launch_lb_t<true, true, false>(d, a, s);
        } else {
            if (sig) launch_lb_t<true, false, true>(d, a, s); else launch_lb_t<true, false, false>(d, a, s);
        }
    } else {
        if (cells) {
            if (sig) launch_lb_t<false, true, true>(d, a, s); else launch_lb_t<false, true, false>(d, a, s);
        } else {
            if (sig) launch_lb_t<false, false, true>(d, a, s); else launch_lb_t<false, false, false>(d, a, s);
        }
    }
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
