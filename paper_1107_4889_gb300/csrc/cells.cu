// cells.cu -- per-cell work of the coupled step.
//
//   k_bin    one thread per cell: cell-list bin (FP64 position / bin size),
//            slot in a fixed-capacity bin, and the shape tensor A = Q S^2 Q^T.
//   k_gb     one thread per cell: candidate partners from the 27 surrounding
//            bins (FP64 distance test without fused multiply-add, kept sorted
//            by partner index), Gay-Berne forces and torques over them and
//            over the wall particles binned in the same grid (Sec. 2.5,
//            App. B).  Each pair is evaluated once from each side, so every
//            cell sums its own force in a fixed order (no atomics).
//   k_cells  one CTA per cell: the cell's shape-function weights on a box
//            around its support staged in shared memory, sampling of the
//            fluid (Eqs. vel, vort, pheno_torque_diss) with a block
//            reduction, the rigid-body update by one thread (App. A), and the
//            spreading of the reaction force density and the smoothed
//            characteristic function to the lattice with atomics (Sec. 2.2,
//            Eq. enhance-viscosity).
#include "internal.h"
#include "rbc_device.cuh"

namespace rbc {

namespace {

constexpr int kBinThreads = 128;
constexpr int kGbThreads = 64;
constexpr int kCellThreads = 256;
constexpr int kMaxNbr = 128;

__global__ void __launch_bounds__(kBinThreads)
k_bin(const double *__restrict__ R, const double *__restrict__ q, double *__restrict__ A,
      int *__restrict__ cell_bin, int *__restrict__ bin_count, int *__restrict__ bin_cells,
      int *__restrict__ flags, int nc, int nb0, int nb1, int nb2, double bs0, double bs1,
      double bs2, int cap, double a20, double a21, double a22)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int nb[3] = {nb0, nb1, nb2};
    const double bs[3] = {bs0, bs1, bs2};
    int b[3];
    for (int a = 0; a < 3; ++a) {
        int k = (int)floor(R[3 * i + a] / bs[a]);
        b[a] = k < 0 ? 0 : (k >= nb[a] ? nb[a] - 1 : k);
    }
    const int bin = b[0] + nb0 * (b[1] + nb1 * b[2]);
    cell_bin[i] = bin;
    const int slot = atomicAdd(&bin_count[bin], 1);
    if (slot < cap)
        bin_cells[bin * cap + slot] = i;
    else
        atomicOr(&flags[FLAG_OVERFLOW], OVF_BIN);
    double qq[4] = {q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3]};
    const double in = 1.0 / sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
    for (int k = 0; k < 4; ++k) qq[k] *= in;
    double Q[9];
    quat_matrix(qq, Q);
    const double a2[3] = {a20, a21, a22};
    const Sym3 S = shape_tensor(Q, a2);
    double *o = &A[6 * i];
    o[0] = S.xx;
    o[1] = S.yy;
    o[2] = S.zz;
    o[3] = S.xy;
    o[4] = S.xz;
    o[5] = S.yz;
}

struct GbArgs {
    const double *R, *A;
    const int *cell_bin, *bin_count, *bin_cells;
    const int *wall_start, *wall_xyz;
    int *nbr, *nbr_count;
    double *Fm, *Tm;
    int *flags;
    unsigned long long *clamps;
    int nc, cap, maxn, nb[3], per[3];
    double L[3], rc2, rcw2, smin, smin_w, rw2, eps0, rho_floor, rho_cut;
};

// minimum image along periodic axes; positions live in [0, L)
__device__ __forceinline__ void min_image(double d[3], const int per[3], const double L[3])
{
    for (int a = 0; a < 3; ++a) {
        if (!per[a]) continue;
        if (d[a] > 0.5 * L[a])
            d[a] = __dsub_rn(d[a], L[a]);
        else if (d[a] < -0.5 * L[a])
            d[a] = __dadd_rn(d[a], L[a]);
    }
}

__device__ __forceinline__ double dist2_exact(const double d[3])
{
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ void bin_range(int b, int nb, int per, int &lo, int &hi)
{
    if (per) {
        lo = nb >= 3 ? -1 : 0;
        hi = nb >= 2 ? 1 : 0;
    } else {
        lo = b > 0 ? -1 : 0;
        hi = b < nb - 1 ? 1 : 0;
    }
}

__device__ __forceinline__ int wrap_bin(int b, int nb) { return b < 0 ? b + nb : (b >= nb ? b - nb : b); }

__global__ void __launch_bounds__(kGbThreads) k_gb(GbArgs g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nc) return;
    const double Ri[3] = {g.R[3 * i], g.R[3 * i + 1], g.R[3 * i + 2]};
    const double *ai = &g.A[6 * i];
    const Sym3 Ai{ai[0], ai[1], ai[2], ai[3], ai[4], ai[5]};
    const int bin = g.cell_bin[i];
    const int b[3] = {bin % g.nb[0], (bin / g.nb[0]) % g.nb[1], bin / (g.nb[0] * g.nb[1])};
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) bin_range(b[a], g.nb[a], g.per[a], lo[a], hi[a]);

    int lst[kMaxNbr];
    int cnt = 0;
    bool ovf = false;
    for (int oz = lo[2]; oz <= hi[2]; ++oz)
        for (int oy = lo[1]; oy <= hi[1]; ++oy)
            for (int ox = lo[0]; ox <= hi[0]; ++ox) {
                const int bb = wrap_bin(b[0] + ox, g.nb[0]) +
                               g.nb[0] * (wrap_bin(b[1] + oy, g.nb[1]) + g.nb[1] * wrap_bin(b[2] + oz, g.nb[2]));
                const int c = min(g.bin_count[bb], g.cap);
                for (int k = 0; k < c; ++k) {
                    const int j = g.bin_cells[bb * g.cap + k];
                    if (j == i) continue;
                    double d[3] = {__dsub_rn(Ri[0], g.R[3 * j]), __dsub_rn(Ri[1], g.R[3 * j + 1]),
                                   __dsub_rn(Ri[2], g.R[3 * j + 2])};
                    min_image(d, g.per, g.L);
                    if (!(dist2_exact(d) < g.rc2)) continue;
                    if (cnt >= g.maxn) {
                        ovf = true;
                        continue;
                    }
                    int pos = cnt++;
                    while (pos > 0 && lst[pos - 1] > j) {
                        lst[pos] = lst[pos - 1];
                        --pos;
                    }
                    lst[pos] = j;
                }
            }
    if (ovf) atomicOr(&g.flags[FLAG_OVERFLOW], OVF_NBR);
    g.nbr_count[i] = cnt;
    for (int k = 0; k < cnt; ++k) g.nbr[i * g.maxn + k] = lst[k];

    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    int clamped = 0;
    for (int k = 0; k < cnt; ++k) {
        const int j = lst[k];
        double d[3] = {__dsub_rn(Ri[0], g.R[3 * j]), __dsub_rn(Ri[1], g.R[3 * j + 1]),
                       __dsub_rn(Ri[2], g.R[3 * j + 2])};
        min_image(d, g.per, g.L);
        const double *aj = &g.A[6 * j];
        const Sym3 Aj{aj[0], aj[1], aj[2], aj[3], aj[4], aj[5]};
        gb_pair(d, Ai, Aj, g.smin, g.eps0, g.rho_floor, g.rho_cut, F, T, clamped);
    }
    if (g.wall_start != nullptr) {
        const Sym3 Aw{g.rw2, g.rw2, g.rw2, 0.0, 0.0, 0.0};
        int wlo[3], whi[3];
        for (int a = 0; a < 3; ++a) bin_range(b[a], g.nb[a], g.per[a], wlo[a], whi[a]);
        for (int oz = wlo[2]; oz <= whi[2]; ++oz)
            for (int oy = wlo[1]; oy <= whi[1]; ++oy)
                for (int ox = wlo[0]; ox <= whi[0]; ++ox) {
                    const int bb = wrap_bin(b[0] + ox, g.nb[0]) +
                                   g.nb[0] * (wrap_bin(b[1] + oy, g.nb[1]) + g.nb[1] * wrap_bin(b[2] + oz, g.nb[2]));
                    for (int w = g.wall_start[bb]; w < g.wall_start[bb + 1]; ++w) {
                        double d[3] = {Ri[0] - (double)g.wall_xyz[3 * w], Ri[1] - (double)g.wall_xyz[3 * w + 1],
                                       Ri[2] - (double)g.wall_xyz[3 * w + 2]};
                        min_image(d, g.per, g.L);
                        if (!(dist2_exact(d) < g.rcw2)) continue;
                        gb_pair(d, Ai, Aw, g.smin_w, g.eps0, g.rho_floor, g.rho_cut, F, T, clamped);
                    }
                }
    }
    for (int a = 0; a < 3; ++a) {
        g.Fm[3 * i + a] = F[a];
        g.Tm[3 * i + a] = T[a];
    }
    if (clamped) atomicAdd(g.clamps, (unsigned long long)clamped);
}

struct CellsArgs {
    double *R, *q, *V, *Om;
    const double *Fm, *Tm;
    int *have;
    double *diag;
    const float *U, *S;
    float *G, *theta;
    const uint8_t *solid;
    int *flags;
    int nx, ny, nz;
    long long Np;
    float two_over_xi[3], xi[3], kappa, alpha;
    double M, I[3], eT, eR, gT, gR, L[3];
    int per[3], box_max, box_dim;
};

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Sum NV per-thread values over the block: FP32 within a warp, FP64 across
// warps in a fixed order; the result lands in out[] (shared) for all threads.
template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], double (*red)[NV], double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if (lane == 0)
        for (int k = 0; k < NV; ++k) red[warp][k] = (double)v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

template <bool ALPHA>
__global__ void __launch_bounds__(kCellThreads) k_cells(CellsArgs a)
{
    extern __shared__ float sw[];  // shape weight w per box node (0 at solid nodes)
    __shared__ double sQd[9], sRd[3];
    __shared__ float sQ[9], sbase[3];
    __shared__ int so[3], sn[3], sbad;
    __shared__ double red[kCellThreads / 32][9];
    __shared__ double sums[9];
    __shared__ float sJ[3], sL[3], sU0[3];
    const int i = blockIdx.x;
    const int tid = threadIdx.x;

    if (tid == 0) {
        double qq[4] = {a.q[4 * i], a.q[4 * i + 1], a.q[4 * i + 2], a.q[4 * i + 3]};
        const double in = 1.0 / sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
        for (int k = 0; k < 4; ++k) qq[k] *= in;
        quat_matrix(qq, sQd);
        for (int k = 0; k < 9; ++k) sQ[k] = (float)sQd[k];
        // the box must have 1..box_dim nodes per axis and lie within one
        // period of the lattice on each side, so that a single wrap maps it
        // into the lattice; a cell that left the box or went non-finite is
        // flagged and skipped
        const int dims[3] = {a.nx, a.ny, a.nz};
        bool bad = false;
        for (int d = 0; d < 3; ++d) {
            const double Rd = a.R[3 * i + d];
            sRd[d] = Rd;
            double e = 0.0;
            for (int b = 0; b < 3; ++b) e += fabs(sQd[3 * d + b]) * (double)a.xi[b];
            if (!(fabs(Rd) < 1e7) || !(e < 1e7)) {
                bad = true;
                so[d] = 0;
                sn[d] = 1;
                continue;
            }
            const int lo = (int)ceil(Rd - e) - 1;
            const int hi = (int)floor(Rd + e) + 1;
            so[d] = lo;
            sn[d] = hi - lo + 1;
            sbase[d] = (float)((double)lo - Rd);
            if (sn[d] < 1 || sn[d] > a.box_dim || lo < -dims[d] || hi >= 2 * dims[d]) bad = true;
        }
        sbad = bad;
        if (sbad) atomicOr(&a.flags[FLAG_OVERFLOW], OVF_BOX);
        // reference velocity: u at the node nearest the centre.  Sum D delta
        // vanishes over the box, so subtracting a constant from u leaves the
        // vorticity sum unchanged in exact arithmetic and removes the FP32
        // cancellation of a nearly uniform flow.
        if (!bad) {
            int c[3];
            for (int d = 0; d < 3; ++d) c[d] = wrap1((int)floor(sRd[d] + 0.5), dims[d]);
            const long long gc = c[0] + (long long)a.nx * (c[1] + (long long)a.ny * c[2]);
            sU0[0] = a.U[gc];
            sU0[1] = a.U[a.Np + gc];
            sU0[2] = a.U[2 * a.Np + gc];
        }
    }
    __syncthreads();
    if (sbad) return;
    const int n0 = sn[0], n1 = sn[1], n01 = sn[0] * sn[1], vol = n01 * sn[2];
    const int nxy = a.nx * a.ny;

    // 1. weights w = prod_b phi(2 y_b / xi_b), y = Q^T (x - R) (Sec. 2.2)
    {
        float part[1] = {0.f};
        for (int m = tid; m < vol; m += blockDim.x) {
            const int i0 = m % n0, t = m / n0, i1 = t % n1, i2 = t / n1;
            const int g = wrap1(so[0] + i0, a.nx) + a.nx * wrap1(so[1] + i1, a.ny) + nxy * wrap1(so[2] + i2, a.nz);
            float w = 0.f;
            if (a.solid == nullptr || !a.solid[g]) {
                const float r0 = sbase[0] + (float)i0, r1 = sbase[1] + (float)i1, r2 = sbase[2] + (float)i2;
                w = 1.f;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float y = sQ[b] * r0 + sQ[3 + b] * r1 + sQ[6 + b] * r2;
                    w *= peskin4(y * a.two_over_xi[b]);
                }
            }
            sw[m] = w;
            part[0] += w;
        }
        __syncthreads();
        block_sum<1>(part, reinterpret_cast<double (*)[1]>(red), sums);
    }
    const double S = sums[0];
    __syncthreads();
    if (!(S > 0.0)) {
        if (tid == 0) atomicOr(&a.flags[FLAG_UNSTABLE], 2);
        return;
    }

    // 2. sampling: u~ = sum delta u, omega~ = sum delta curl u = -sum D delta x u
    //    (summation by parts of the central-difference curl), and
    //    T^S = alpha sum delta (sigma n) x (x - R), n = D delta / |D delta|
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float thr = (float)(1e-24 * S * S);
    for (int m = tid; m < vol; m += blockDim.x) {
        const int i0 = m % n0, t = m / n0, i1 = t % n1, i2 = t / n1;
        const float w0 = sw[m];
        const float Dx = 0.5f * ((i0 + 1 < n0 ? sw[m + 1] : 0.f) - (i0 > 0 ? sw[m - 1] : 0.f));
        const float Dy = 0.5f * ((i1 + 1 < n1 ? sw[m + n0] : 0.f) - (i1 > 0 ? sw[m - n0] : 0.f));
        const float Dz = 0.5f * ((i2 + 1 < sn[2] ? sw[m + n01] : 0.f) - (i2 > 0 ? sw[m - n01] : 0.f));
        if (w0 == 0.f && Dx == 0.f && Dy == 0.f && Dz == 0.f) continue;
        const int g = wrap1(so[0] + i0, a.nx) + a.nx * wrap1(so[1] + i1, a.ny) + nxy * wrap1(so[2] + i2, a.nz);
        const float ux = a.U[g], uy = a.U[a.Np + g], uz = a.U[2 * a.Np + g];
        acc[0] += w0 * ux;
        acc[1] += w0 * uy;
        acc[2] += w0 * uz;
        const float vx = ux - sU0[0], vy = uy - sU0[1], vz = uz - sU0[2];
        acc[3] -= Dy * vz - Dz * vy;
        acc[4] -= Dz * vx - Dx * vz;
        acc[5] -= Dx * vy - Dy * vx;
        if (ALPHA && w0 > 0.f) {
            const float nd2 = Dx * Dx + Dy * Dy + Dz * Dz;
            if (nd2 > thr) {
                const float inv = rsqrtf(nd2);
                const float nx = Dx * inv, ny = Dy * inv, nz = Dz * inv;
                const float sxx = a.S[g], syy = a.S[a.Np + g], szz = a.S[2 * a.Np + g];
                const float sxy = a.S[3 * a.Np + g], sxz = a.S[4 * a.Np + g], syz = a.S[5 * a.Np + g];
                const float tx = sxx * nx + sxy * ny + sxz * nz;
                const float ty = sxy * nx + syy * ny + syz * nz;
                const float tz = sxz * nx + syz * ny + szz * nz;
                const float r0 = sbase[0] + (float)i0, r1 = sbase[1] + (float)i1, r2 = sbase[2] + (float)i2;
                acc[6] += w0 * (ty * r2 - tz * r1);
                acc[7] += w0 * (tz * r0 - tx * r2);
                acc[8] += w0 * (tx * r1 - ty * r0);
            }
        }
    }
    block_sum<9>(acc, red, sums);

    // 3. rigid-body update (App. A) by one thread, FP64
    if (tid == 0) {
        const double iS = 1.0 / S;
        double ut[3], wt[3], TS[3], Fm[3], Tm[3], Fc[3], Tl[3], Tb[3], wb[3], Tc[3];
        for (int d = 0; d < 3; ++d) {
            ut[d] = sums[d] * iS;
            wt[d] = sums[3 + d] * iS;
            TS[d] = ALPHA ? (double)a.alpha * sums[6 + d] * iS : 0.0;
            Fm[d] = a.Fm[3 * i + d];
            Tm[d] = a.Tm[3 * i + d];
            Fc[d] = Fm[d] + a.gT * a.M * ut[d];
            Tl[d] = Tm[d] + TS[d];
        }
        const double *Q = sQd;
        for (int d = 0; d < 3; ++d) {
            Tb[d] = Q[d] * Tl[0] + Q[3 + d] * Tl[1] + Q[6 + d] * Tl[2];
            wb[d] = Q[d] * wt[0] + Q[3 + d] * wt[1] + Q[6 + d] * wt[2];
            Tc[d] = Tb[d] + a.gR * a.I[d] * wb[d];
        }
        double V[3], Om[3], V0[3], Om0[3];
        for (int d = 0; d < 3; ++d) {
            V0[d] = V[d] = a.V[3 * i + d];
            Om0[d] = Om[d] = a.Om[3 * i + d];
        }
        const bool have = a.have[i] != 0;
        if (have) {  // steps 6-7 of the previous step, with forces at this pose
            for (int d = 0; d < 3; ++d) {
                Om[d] *= a.eR;
                V[d] *= a.eT;
                V[d] += 0.5 * Fc[d] / a.M;
                Om[d] += 0.5 * Tc[d] / a.I[d];
            }
        }
        for (int d = 0; d < 3; ++d) {  // steps 1-2
            Om[d] += 0.5 * Tc[d] / a.I[d];
            V[d] += 0.5 * Fc[d] / a.M;
            Om[d] *= a.eR;
            V[d] *= a.eT;
        }
        const double c = have ? 1.0 : 0.5;
        double J[3], L[3], dp[3];
        for (int d = 0; d < 3; ++d) {
            J[d] = a.M * (V[d] - V0[d]) - c * Fm[d];
            dp[d] = a.I[d] * (Om[d] - Om0[d]);
        }
        for (int d = 0; d < 3; ++d) L[d] = Q[3 * d] * dp[0] + Q[3 * d + 1] * dp[1] + Q[3 * d + 2] * dp[2] - c * Tm[d];
        // step 3: drift
        double R[3];
        for (int d = 0; d < 3; ++d) {
            R[d] = sRd[d] + V[d];
            if (a.per[d]) {
                if (R[d] >= a.L[d])
                    R[d] -= a.L[d];
                else if (R[d] < 0.0)
                    R[d] += a.L[d];
            }
        }
        // step 4: sub-rotations about body axes 1, 2, 3, 2, 1 by h Om/2, h Om/2,
        // h Om, h Om/2, h Om/2; each turns pi = I Om by R^T and the frame by R
        double q[4] = {a.q[4 * i], a.q[4 * i + 1], a.q[4 * i + 2], a.q[4 * i + 3]};
        {
            const double in = 1.0 / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            for (int k = 0; k < 4; ++k) q[k] *= in;
        }
        const int ax[5] = {0, 1, 2, 1, 0};
        const double fr[5] = {0.5, 0.5, 1.0, 0.5, 0.5};
        for (int s = 0; s < 5; ++s) {
            const int k = ax[s];
            const double th = fr[s] * Om[k];
            double sh, ch;
            sincos(0.5 * th, &sh, &ch);
            double r[4] = {ch, 0.0, 0.0, 0.0};
            r[1 + k] = sh;
            const double w1 = q[0], x1 = q[1], y1 = q[2], z1 = q[3];
            const double w2 = r[0], x2 = r[1], y2 = r[2], z2 = r[3];
            q[0] = w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2;
            q[1] = w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2;
            q[2] = w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2;
            q[3] = w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2;
            double st, ct;
            sincos(th, &st, &ct);
            const int p1 = (k + 1) % 3, p2 = (k + 2) % 3;
            const double pi1 = a.I[p1] * Om[p1], pi2 = a.I[p2] * Om[p2];
            Om[p1] = (ct * pi1 + st * pi2) / a.I[p1];
            Om[p2] = (-st * pi1 + ct * pi2) / a.I[p2];
        }
        {
            const double in = 1.0 / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            for (int k = 0; k < 4; ++k) a.q[4 * i + k] = q[k] * in;
        }
        for (int d = 0; d < 3; ++d) {
            a.R[3 * i + d] = R[d];
            a.V[3 * i + d] = V[d];
            a.Om[3 * i + d] = Om[d];
        }
        a.have[i] = 1;
        double *o = &a.diag[21 * i];
        for (int d = 0; d < 3; ++d) {
            o[d] = Fm[d];
            o[3 + d] = Tm[d];
            o[6 + d] = ut[d];
            o[9 + d] = wt[d];
            o[12 + d] = TS[d];
            o[15 + d] = J[d];
            o[18 + d] = L[d];
            sJ[d] = (float)J[d];
            sL[d] = (float)L[d];
        }
    }
    __syncthreads();

    // 4. spreading (h = 1): G += -J delta + 1/2 L x D delta at fluid nodes;
    //    theta += 1 - (1 - w)^kappa where w > 0
    const float iS = (float)(1.0 / S);
    const float Jx = sJ[0], Jy = sJ[1], Jz = sJ[2];
    const float Lx = 0.5f * sL[0], Ly = 0.5f * sL[1], Lz = 0.5f * sL[2];
    for (int m = tid; m < vol; m += blockDim.x) {
        const int i0 = m % n0, t = m / n0, i1 = t % n1, i2 = t / n1;
        const float w0 = sw[m];
        const float Dx = 0.5f * ((i0 + 1 < n0 ? sw[m + 1] : 0.f) - (i0 > 0 ? sw[m - 1] : 0.f));
        const float Dy = 0.5f * ((i1 + 1 < n1 ? sw[m + n0] : 0.f) - (i1 > 0 ? sw[m - n0] : 0.f));
        const float Dz = 0.5f * ((i2 + 1 < sn[2] ? sw[m + n01] : 0.f) - (i2 > 0 ? sw[m - n01] : 0.f));
        if (w0 == 0.f && Dx == 0.f && Dy == 0.f && Dz == 0.f) continue;
        const int g = wrap1(so[0] + i0, a.nx) + a.nx * wrap1(so[1] + i1, a.ny) + nxy * wrap1(so[2] + i2, a.nz);
        if (a.solid != nullptr && a.solid[g]) continue;
        const float dl = w0 * iS, ex = Dx * iS, ey = Dy * iS, ez = Dz * iS;
        atomicAdd(&a.G[g], -Jx * dl + (Ly * ez - Lz * ey));
        atomicAdd(&a.G[a.Np + g], -Jy * dl + (Lz * ex - Lx * ez));
        atomicAdd(&a.G[2 * a.Np + g], -Jz * dl + (Lx * ey - Ly * ex));
        if (w0 > 0.f) atomicAdd(&a.theta[g], 1.0f - powf(1.0f - w0, a.kappa));
    }
}

}  // namespace

void launch_bin(const Dev &d, const Params &p, cudaStream_t s)
{
    if (d.nc == 0) return;
    cudaMemsetAsync(d.bin_count, 0, sizeof(int) * d.nbins, s);
    k_bin<<<(d.nc + kBinThreads - 1) / kBinThreads, kBinThreads, 0, s>>>(
        d.R, d.q, d.A, d.cell_bin, d.bin_count, d.bin_cells, d.flags, d.nc, d.nb[0], d.nb[1], d.nb[2],
        d.bin_size[0], d.bin_size[1], d.bin_size[2], d.bin_cap, p.a2[0], p.a2[1], p.a2[2]);
}

void launch_gb(const Dev &d, const Params &p, cudaStream_t s)
{
    if (d.nc == 0) return;
    GbArgs g;
    g.R = d.R;
    g.A = d.A;
    g.cell_bin = d.cell_bin;
    g.bin_count = d.bin_count;
    g.bin_cells = d.bin_cells;
    g.wall_start = d.nw > 0 ? d.wall_start : nullptr;
    g.wall_xyz = d.wall_xyz;
    g.nbr = d.nbr;
    g.nbr_count = d.nbr_count;
    g.Fm = d.Fm;
    g.Tm = d.Tm;
    g.flags = d.flags;
    g.clamps = d.clamps;
    g.nc = d.nc;
    g.cap = d.bin_cap;
    g.maxn = d.max_nbr;
    const int dims[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; ++a) {
        g.nb[a] = d.nb[a];
        g.per[a] = p.periodic[a];
        g.L[a] = (double)dims[a];
    }
    g.rc2 = p.rc2;
    g.rcw2 = p.rcw2;
    g.smin = p.smin_cc;
    g.smin_w = p.smin_w;
    g.rw2 = p.rw2;
    g.eps0 = p.eps0;
    g.rho_floor = p.rho_floor;
    g.rho_cut = p.rho_cut;
    k_gb<<<(d.nc + kGbThreads - 1) / kGbThreads, kGbThreads, 0, s>>>(g);
}

size_t cells_smem_bytes(const Params &p) { return sizeof(float) * (size_t)p.box_max; }

void launch_cells(const Dev &d, const Params &p, cudaStream_t s)
{
    if (d.nc == 0) return;
    CellsArgs a;
    a.R = d.R;
    a.q = d.q;
    a.V = d.V;
    a.Om = d.Om;
    a.Fm = d.Fm;
    a.Tm = d.Tm;
    a.have = d.have;
    a.diag = d.diag;
    a.U = d.U;
    a.S = d.S;
    a.G = d.G;
    a.theta = d.theta;
    a.solid = d.solid;
    a.flags = d.flags;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.Np = d.Np;
    for (int k = 0; k < 3; ++k) {
        a.xi[k] = p.xi[k];
        a.two_over_xi[k] = 2.0f / p.xi[k];
        a.I[k] = p.I[k];
        a.per[k] = p.periodic[k];
    }
    a.L[0] = d.nx;
    a.L[1] = d.ny;
    a.L[2] = d.nz;
    a.kappa = p.kappa;
    a.alpha = p.alpha;
    a.M = p.M;
    a.eT = p.eT;
    a.eR = p.eR;
    a.gT = p.gT;
    a.gR = p.gR;
    a.box_max = p.box_max;
    a.box_dim = p.box_dim;
    const size_t smem = cells_smem_bytes(p);
    if (d.S != nullptr)
        k_cells<true><<<d.nc, kCellThreads, smem, s>>>(a);
    else
        k_cells<false><<<d.nc, kCellThreads, smem, s>>>(a);
}

}  // namespace rbc
