// cells.cu -- per-cell work of the coupled step.
//
//   k_bin     one thread per cell: cell-list bin and slot (FP64 position / bin
//             size) and the shape tensor A = Q S^2 Q^T.
//   k_gb      one warp per cell, four cells per block: the 27 surrounding
//             bins are scanned by the lanes with the exact FP64 distance
//             test (no fused multiply-add), passing partners are compacted
//             with a ballot and ranked into a list sorted by partner index;
//             the block's threads then evaluate the queued Gay-Berne pairs
//             and wall particles one each (Sec. 2.5, App. B; the geometry and
//             u'(rho) in FP64, the force and torque vectors in FP32).  A
//             conservative FP32 reduced-distance test skips pairs that are
//             certainly outside the range.  Each pair is evaluated from both
//             sides: every cell sums its own force in FP64 in a fixed order,
//             without atomics.
//   k_weights one warp per cell: the cell's shape header and the shape-function
//             weights on its box staged in shared memory, written out as
//             the cell's shape list (node, w, D w) with the normalisation S;
//             built for the next pose while the lattice pass runs.
//   k_cells   one warp per cell: the fields sampled over the shape list
//             (Eqs. vel, vort, pheno_torque_diss), the rigid-body update
//             (App. A) with the hydrodynamic impulses, and the reaction
//             force density and smoothed characteristic function added
//             over the same list with atomics (Sec. 2.2, Eq.
//             enhance-viscosity); or, split, the last part as k_spread.
#include <algorithm>
#include <cstring>
#include <utility>

#include "internal.h"
#include "rbc_device.cuh"

namespace rbc {

namespace {

constexpr int kBinThreads = 32;  // FP64-bound: spread the warps over all SMs
constexpr int kGbWarps = 4;   // cells per block of the Gay-Berne kernel
constexpr int kGbQueue = 64;  // partners per cell (cells and wall particles) that may interact
constexpr int kMaxNbr = 128;

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ void quat_matrix_f(const float q[4], float Q[9])
{
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    Q[0] = 1.f - 2.f * (y * y + z * z);
    Q[1] = 2.f * (x * y - w * z);
    Q[2] = 2.f * (x * z + w * y);
    Q[3] = 2.f * (x * y + w * z);
    Q[4] = 1.f - 2.f * (x * x + z * z);
    Q[5] = 2.f * (y * z - w * x);
    Q[6] = 2.f * (x * z - w * y);
    Q[7] = 2.f * (y * z + w * x);
    Q[8] = 1.f - 2.f * (x * x + y * y);
}

// Launch with a scheduling priority (the side-stream kernels of the step
// take the device's highest, so that their blocks are dispatched ahead of
// the persistent lattice pass that runs beside them).
template <typename... Params, typename... Args>
void launch_prio(void (*kernel)(Params...), int grid, int block, size_t smem, cudaStream_t s, int prio,
                 Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// v[k] for a run-time k without local memory
template <int N>
__device__ __forceinline__ float pick(const float (&v)[N], int k)
{
    float r = v[0];
#pragma unroll
    for (int j = 1; j < N; ++j) r = k == j ? v[j] : r;
    return r;
}

// ---------------------------------------------------------------------------
// k_bin
// ---------------------------------------------------------------------------
struct BinArgs {
    const double *R, *q;
    double *A;
    float *Rf, *Af;
    int *cell_bin, *bin_count, *bin_cells, *flags;
    int nc, nb[3], cap;
    double bs[3], a2[3];
};

// One thread per cell.  Its loads come first and the bin's slot, returned by
// the atomic, is used last, so that the FP64 shape tensor is computed while
// the atomic is in flight.
__device__ __forceinline__ void bin_body(const BinArgs &g, int blk)
{
    const int i = blk * blockDim.x + threadIdx.x;
    if (i >= g.nc) return;
    double Rd[3], qq[4];
    for (int a = 0; a < 3; ++a) Rd[a] = g.R[3 * i + a];
    for (int k = 0; k < 4; ++k) qq[k] = g.q[4 * i + k];
    int b[3];
    for (int a = 0; a < 3; ++a) {
        int k = (int)floor(Rd[a] / g.bs[a]);
        b[a] = k < 0 ? 0 : (k >= g.nb[a] ? g.nb[a] - 1 : k);
    }
    const int bin = b[0] + g.nb[0] * (b[1] + g.nb[1] * b[2]);
    const int slot = atomicAdd(&g.bin_count[bin], 1);
    g.cell_bin[i] = bin;
    const double in = 1.0 / sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
    for (int k = 0; k < 4; ++k) qq[k] *= in;
    double Q[9];
    quat_matrix(qq, Q);
    const Sym3 S = shape_tensor(Q, g.a2);
    double *o = &g.A[6 * i];
    o[0] = S.xx;
    o[1] = S.yy;
    o[2] = S.zz;
    o[3] = S.xy;
    o[4] = S.xz;
    o[5] = S.yz;
    for (int a = 0; a < 3; ++a) g.Rf[3 * i + a] = (float)Rd[a];
    g.Af[6 * i] = (float)S.xx;
    g.Af[6 * i + 1] = (float)S.yy;
    g.Af[6 * i + 2] = (float)S.zz;
    g.Af[6 * i + 3] = (float)S.xy;
    g.Af[6 * i + 4] = (float)S.xz;
    g.Af[6 * i + 5] = (float)S.yz;
    if (slot < g.cap)
        g.bin_cells[bin * g.cap + slot] = i;
    else
        atomicOr(&g.flags[FLAG_OVERFLOW], OVF_BIN);
}

__global__ void __launch_bounds__(kBinThreads) k_bin(BinArgs g) { bin_body(g, blockIdx.x); }

// ---------------------------------------------------------------------------
// k_gb
// ---------------------------------------------------------------------------
struct GbArgs {
    const double *R, *A;
    const float *Rf, *Af;
    const int *cell_bin, *bin_count, *bin_cells;
    const int *wall_start, *wall_xyz;
    int *nbr, *nbr_count;
    double *Fm, *Tm;
    const double *ext;  // 6n external force and torque (lab), or null
    int *flags;
    unsigned long long *clamps;
    int nc, cap, maxn, nb[3], per[3];
    double L[3], rc2, rcw2, smin, smin_w, rw2, eps0, rho_floor, rho_cut;
    double ismin, ismin_w;  // 1 / sigma_min (cell pairs, cell-wall pairs)
    float rho_cut_f;  // FP32 prefilter bound (rho_cut with a safety margin)
    float rc_lo2, rc_hi2, rcw2_f, Lf[3];  // FP32 candidate band around r_cut, wall radius
    int wnb[3];                           // wall-particle grid
    float wbs[3];
};

// ---------------------------------------------------------------------------
// Gay-Berne pair (Sec. 2.5, App. B), d = R_i - R_j: the force on i and the
// lab-frame torque on i; returns true if the pair is inside the range.
//   kappa = (A_i + A_j)^-1 d, phi = (d.kappa) / (2 R^2), sigma = phi^-1/2,
//   rho = (R - sigma + sigma_min) / sigma_min, range rho <= 2^(1/6),
//   F_i = -u'(rho)/sigma_min d^ - (du/dphi / R^2) (kappa - (kappa.d^) d^),
//   du/dphi = u'(rho) sigma^3 / (2 sigma_min),
//   tau_i = (-A_i kappa) x f_kappa, f_kappa = -(du/dphi / R^2) kappa.
// rho below rho_floor is evaluated at rho_floor and counted.
// ---------------------------------------------------------------------------
// Precision: the geometry (d.kappa through the cofactors of A_i + A_j, R,
// sigma, rho) and u'(rho) in FP64, so the range test and the clamp count are
// exact and the two differences of nearly equal numbers (the gap R - sigma,
// and u'(rho) near the minimum of the potential) keep FP64 accuracy; kappa
// itself, the force and the torque vectors in FP32 (relative error ~1e-7;
// 9e-8 median, 2.4e-7 99th percentile for the force over random pairs in
// range).  F and T are this pair's
// contribution; the caller sums them per cell in FP64.  Ai_f: A_i in FP32
// (xx yy zz xy xz yz); ismin = 1 / sigma_min.
__device__ inline bool gb_pair_mixed(const double d[3], const Sym3 &Ai, const Sym3 &Aj, const float Ai_f[6],
                                     double smin, double ismin, double eps0, double rho_floor, double rho_cut,
                                     float F[3], float T[3], int &clamped)
{
    Sym3 H{Ai.xx + Aj.xx, Ai.yy + Aj.yy, Ai.zz + Aj.zz, Ai.xy + Aj.xy, Ai.xz + Aj.xz, Ai.yz + Aj.yz};
    // adj(H) (the cofactors), det H; d.kappa = d^T adj(H) d / det H, so
    // sigma = phi^-1/2 = R sqrt(2 det H / d^T adj(H) d) and R - sigma =
    // R (1 - s): one division and two square roots in FP64
    const double cxx = H.yy * H.zz - H.yz * H.yz;
    const double cyy = H.xx * H.zz - H.xz * H.xz;
    const double czz = H.xx * H.yy - H.xy * H.xy;
    const double cxy = H.xz * H.yz - H.xy * H.zz;
    const double cxz = H.xy * H.yz - H.xz * H.yy;
    const double cyz = H.xy * H.xz - H.xx * H.yz;
    const double det = H.xx * cxx + H.xy * cxy + H.xz * cxz;
    const double qa = cxx * d[0] * d[0] + cyy * d[1] * d[1] + czz * d[2] * d[2] +
                      2.0 * (cxy * d[0] * d[1] + cxz * d[0] * d[2] + cyz * d[1] * d[2]);
    const double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double R = sqrt(R2);
    const double sr = sqrt(2.0 * det / qa);
    const double sigma = R * sr;
    double rho = (R - sigma) * ismin + 1.0;
    if (rho > rho_cut) return false;
    if (rho < rho_floor) {
        rho = rho_floor;
        clamped++;
    }
    // kappa in FP32 from the FP64 cofactors (it only enters the force and
    // torque vectors)
    const float idetf = 1.0f / (float)det;
    // u'(rho) in FP64 too: 2 rho^-13 - rho^-7 cancels near the minimum of
    // the potential
    const double ir = 1.0 / rho;
    const double ir2 = ir * ir;
    const double ir6 = ir2 * ir2 * ir2;
    const double ir7 = ir6 * ir;
    const double ir13 = ir6 * ir7;
    const double dud = -24.0 * eps0 * (2.0 * ir13 - ir7);  // du/drho
    const float df[3] = {(float)d[0], (float)d[1], (float)d[2]};
    const float kf[3] = {((float)cxx * df[0] + (float)cxy * df[1] + (float)cxz * df[2]) * idetf,
                         ((float)cxy * df[0] + (float)cyy * df[1] + (float)cyz * df[2]) * idetf,
                         ((float)cxz * df[0] + (float)cyz * df[1] + (float)czz * df[2]) * idetf};
    const float Rf = (float)R, R2f = (float)R2;
    const float dudR = (float)(dud * ismin);
    const float dudphi = (float)(dud * sigma * sigma * sigma * (0.5 * ismin));
    const float iR = 1.0f / Rf;
    const float kR = (kf[0] * df[0] + kf[1] * df[1] + kf[2] * df[2]) * iR;
    const float g = dudphi / R2f;
    float fk[3];
    for (int a = 0; a < 3; ++a) {
        F[a] = -dudR * df[a] * iR - g * (kf[a] - kR * df[a] * iR);
        fk[a] = -g * kf[a];
    }
    const float Ak[3] = {Ai_f[0] * kf[0] + Ai_f[3] * kf[1] + Ai_f[4] * kf[2],
                         Ai_f[3] * kf[0] + Ai_f[1] * kf[1] + Ai_f[5] * kf[2],
                         Ai_f[4] * kf[0] + Ai_f[5] * kf[1] + Ai_f[2] * kf[2]};
    // (-A_i kappa) x f_kappa
    T[0] = -(Ak[1] * fk[2] - Ak[2] * fk[1]);
    T[1] = -(Ak[2] * fk[0] - Ak[0] * fk[2]);
    T[2] = -(Ak[0] * fk[1] - Ak[1] * fk[0]);
    return true;
}

__device__ __forceinline__ void min_image_f(float d[3], const int per[3], const float L[3])
{
    for (int a = 0; a < 3; ++a) {
        if (!per[a]) continue;
        if (d[a] > 0.5f * L[a])
            d[a] -= L[a];
        else if (d[a] < -0.5f * L[a])
            d[a] += L[a];
    }
}

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

// Reduced Gay-Berne distance in FP32 (no force): false only if the pair is
// certainly outside the range.  H = Ai + Aj as 6 floats (xx yy zz xy xz yz).
__device__ __forceinline__ bool gb_maybe_in_range(const float d[3], const float H[6], float smin, float cut)
{
    const float cxx = H[1] * H[2] - H[5] * H[5];
    const float cyy = H[0] * H[2] - H[4] * H[4];
    const float czz = H[0] * H[1] - H[3] * H[3];
    const float cxy = H[4] * H[5] - H[3] * H[2];
    const float cxz = H[3] * H[5] - H[4] * H[1];
    const float cyz = H[3] * H[4] - H[0] * H[5];
    const float det = H[0] * cxx + H[3] * cxy + H[4] * cxz;
    const float kx = cxx * d[0] + cxy * d[1] + cxz * d[2];
    const float ky = cxy * d[0] + cyy * d[1] + cyz * d[2];
    const float kz = cxz * d[0] + cyz * d[1] + czz * d[2];
    const float R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float phi = 0.5f * (d[0] * kx + d[1] * ky + d[2] * kz) / (det * R2);
    const float rho = (sqrtf(R2) - rsqrtf(phi) + smin) / smin;
    return !(rho > cut);
}

__device__ __forceinline__ void gb_body(const GbArgs &g, int blk)
{
    __shared__ int s_cand[kGbWarps][kMaxNbr];
    __shared__ int s_sort[kGbWarps][kMaxNbr];
    __shared__ int s_pre[kGbWarps][32], s_key[kGbWarps][32];
    __shared__ int s_q[kGbWarps][kGbQueue];  // partner j >= 0, or -1 - wall particle
    __shared__ int s_qpre[kGbWarps + 1];
    __shared__ double s_res[kGbWarps * kGbQueue][6];
    __shared__ int s_clamped;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = blk * kGbWarps + wid;
    if (threadIdx.x == 0) s_clamped = 0;
    int qn = 0;
    if (i < g.nc) {  // uniform across the warp
        const unsigned lt = (1u << lane) - 1u;
        const double Ri[3] = {g.R[3 * i], g.R[3 * i + 1], g.R[3 * i + 2]};
        const float Rif[3] = {g.Rf[3 * i], g.Rf[3 * i + 1], g.Rf[3 * i + 2]};
        const float *aif = &g.Af[6 * i];
        const float Aif[6] = {aif[0], aif[1], aif[2], aif[3], aif[4], aif[5]};
        const int bin = g.cell_bin[i];
        const int b[3] = {bin % g.nb[0], (bin / g.nb[0]) % g.nb[1], bin / (g.nb[0] * g.nb[1])};
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) bin_range(b[a], g.nb[a], g.per[a], lo[a], hi[a]);

        // 1. candidates.  The lanes read the counts of the (up to 27) neighbour
        //    bins at once and prefix-sum them, so the candidates are visited 32
        //    at a time.  The FP32 distance decides outside a band around r_cut;
        //    inside the band the exact FP64 test (no fused multiply-add)
        //    decides, so the partner sets are those of the FP64 test.
        const int bx = hi[0] - lo[0] + 1, by = hi[1] - lo[1] + 1, nbn = bx * by * (hi[2] - lo[2] + 1);
        int cnt = 0;
        {
            int my_bb = 0, my_c = 0;
            if (lane < nbn) {
                const int ox = lo[0] + lane % bx, oy = lo[1] + (lane / bx) % by, oz = lo[2] + lane / (bx * by);
                my_bb = wrap_bin(b[0] + ox, g.nb[0]) +
                        g.nb[0] * (wrap_bin(b[1] + oy, g.nb[1]) + g.nb[1] * wrap_bin(b[2] + oz, g.nb[2]));
                my_c = min(g.bin_count[my_bb], g.cap);
            }
            int incl = my_c;
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            s_pre[wid][lane] = incl - my_c;
            s_key[wid][lane] = my_bb;
            __syncwarp();
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int t = t0 + lane;
                bool pass = false;
                int j = -1;
                if (t < total) {
                    int k0 = 0, k1 = nbn - 1;  // last bin whose first candidate is <= t
                    while (k0 < k1) {
                        const int mid = (k0 + k1 + 1) >> 1;
                        if (s_pre[wid][mid] <= t) k0 = mid; else k1 = mid - 1;
                    }
                    j = g.bin_cells[s_key[wid][k0] * g.cap + (t - s_pre[wid][k0])];
                    // a slot holds a cell index only if this step's binning
                    // wrote it; the range test keeps anything else out
                    if (j != i && (unsigned)j < (unsigned)g.nc) {
                        float df[3] = {Rif[0] - g.Rf[3 * j], Rif[1] - g.Rf[3 * j + 1], Rif[2] - g.Rf[3 * j + 2]};
                        min_image_f(df, g.per, g.Lf);
                        const float r2f = df[0] * df[0] + df[1] * df[1] + df[2] * df[2];
                        if (r2f < g.rc_lo2) {
                            pass = true;
                        } else if (r2f <= g.rc_hi2) {
                            double d[3] = {__dsub_rn(Ri[0], g.R[3 * j]), __dsub_rn(Ri[1], g.R[3 * j + 1]),
                                           __dsub_rn(Ri[2], g.R[3 * j + 2])};
                            min_image(d, g.per, g.L);
                            pass = dist2_exact(d) < g.rc2;
                        }
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, pass);
                const int pos = cnt + __popc(m & lt);
                if (pass && pos < g.maxn) s_cand[wid][pos] = j;
                cnt += __popc(m);
            }
            __syncwarp();
        }
        if (cnt > g.maxn) {
            if (lane == 0) atomicOr(&g.flags[FLAG_OVERFLOW], OVF_NBR);
            cnt = g.maxn;
        }
        __syncwarp();
        // 2. rank sort by partner index (entries are distinct)
        for (int e = lane; e < cnt; e += 32) {
            const int v = s_cand[wid][e];
            int r = 0;
            for (int f = 0; f < cnt; ++f) r += s_cand[wid][f] < v;
            s_sort[wid][r] = v;
        }
        __syncwarp();
        for (int e = lane; e < cnt; e += 32) g.nbr[i * g.maxn + e] = s_sort[wid][e];
        if (lane == 0) g.nbr_count[i] = cnt;

        // 3. the partners the FP32 reduced distance cannot rule out, in index
        //    order, then the wall particles of the 27 wall bins around the
        //    cell (a grid of its own, bins no smaller than the wall radius)
        //    that pass the FP32 tests and the exact FP64 distance test
        for (int e0 = 0; e0 < cnt; e0 += 32) {
            const int e = e0 + lane;
            bool pass = false;
            int j = 0;
            if (e < cnt) {
                j = s_sort[wid][e];
                float df[3] = {Rif[0] - g.Rf[3 * j], Rif[1] - g.Rf[3 * j + 1], Rif[2] - g.Rf[3 * j + 2]};
                min_image_f(df, g.per, g.Lf);
                const float *ajf = &g.Af[6 * j];
                const float H[6] = {Aif[0] + ajf[0], Aif[1] + ajf[1], Aif[2] + ajf[2],
                                    Aif[3] + ajf[3], Aif[4] + ajf[4], Aif[5] + ajf[5]};
                pass = gb_maybe_in_range(df, H, (float)g.smin, g.rho_cut_f);
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            const int pos = qn + __popc(m & lt);
            if (pass && pos < kGbQueue) s_q[wid][pos] = j;
            qn += __popc(m);
        }
        if (g.wall_start != nullptr) {
            const float rw2f = (float)g.rw2;
            const float Hw[6] = {Aif[0] + rw2f, Aif[1] + rw2f, Aif[2] + rw2f, Aif[3], Aif[4], Aif[5]};
            int wb[3], wlo[3], whi[3];
            for (int a = 0; a < 3; ++a) {
                const int k = (int)floorf(Rif[a] / g.wbs[a]);
                wb[a] = k < 0 ? 0 : (k >= g.wnb[a] ? g.wnb[a] - 1 : k);
                bin_range(wb[a], g.wnb[a], g.per[a], wlo[a], whi[a]);
            }
            const int wx = whi[0] - wlo[0] + 1, wy = whi[1] - wlo[1] + 1, nwn = wx * wy * (whi[2] - wlo[2] + 1);
            int my_start = 0, my_c = 0;
            if (lane < nwn) {
                const int ox = wlo[0] + lane % wx, oy = wlo[1] + (lane / wx) % wy, oz = wlo[2] + lane / (wx * wy);
                const int bb = wrap_bin(wb[0] + ox, g.wnb[0]) +
                               g.wnb[0] * (wrap_bin(wb[1] + oy, g.wnb[1]) + g.wnb[1] * wrap_bin(wb[2] + oz, g.wnb[2]));
                my_start = g.wall_start[bb];
                my_c = g.wall_start[bb + 1] - my_start;
            }
            int incl = my_c;
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            __syncwarp();
            s_pre[wid][lane] = incl - my_c;
            s_key[wid][lane] = my_start;
            __syncwarp();
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int t = t0 + lane;
                bool pass = false;
                int w = 0;
                if (t < total) {
                    int k0 = 0, k1 = nwn - 1;
                    while (k0 < k1) {
                        const int mid = (k0 + k1 + 1) >> 1;
                        if (s_pre[wid][mid] <= t) k0 = mid; else k1 = mid - 1;
                    }
                    w = s_key[wid][k0] + (t - s_pre[wid][k0]);
                    const int wxp = g.wall_xyz[3 * w], wyp = g.wall_xyz[3 * w + 1], wzp = g.wall_xyz[3 * w + 2];
                    float df[3] = {Rif[0] - (float)wxp, Rif[1] - (float)wyp, Rif[2] - (float)wzp};
                    min_image_f(df, g.per, g.Lf);
                    if (df[0] * df[0] + df[1] * df[1] + df[2] * df[2] < g.rcw2_f &&
                        gb_maybe_in_range(df, Hw, (float)g.smin_w, g.rho_cut_f)) {
                        double d[3] = {Ri[0] - (double)wxp, Ri[1] - (double)wyp, Ri[2] - (double)wzp};
                        min_image(d, g.per, g.L);
                        pass = dist2_exact(d) < g.rcw2;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, pass);
                const int pos = qn + __popc(m & lt);
                if (pass && pos < kGbQueue) s_q[wid][pos] = -1 - w;
                qn += __popc(m);
            }
        }
        if (qn > kGbQueue) {
            if (lane == 0) atomicOr(&g.flags[FLAG_OVERFLOW], OVF_NBR);
            qn = kGbQueue;
        }
    }
    if (lane == 0) s_qpre[wid + 1] = qn;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_qpre[0] = 0;
        for (int c = 0; c < kGbWarps; ++c) s_qpre[c + 1] += s_qpre[c];
    }
    __syncthreads();
    // 4. the block's queue, all lanes busy: one Gay-Berne pair each (Sec.
    //    2.5, App. B), cells and wall particles alike: the geometry up to
    //    rho in FP64, the force law in FP32 (gb_pair_mixed); step 5 sums
    //    the pairs per cell in FP64
    const int P = s_qpre[kGbWarps];
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        int c = 0;
        while (c + 1 < kGbWarps && s_qpre[c + 1] <= e) ++c;
        const int ci = blk * kGbWarps + c;
        const int v = s_q[c][e - s_qpre[c]];
        float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
        int clamped = 0;
        const double *ai = &g.A[6 * ci];
        const Sym3 Ai{ai[0], ai[1], ai[2], ai[3], ai[4], ai[5]};
        const float *aif = &g.Af[6 * ci];
        const float Ai_f[6] = {aif[0], aif[1], aif[2], aif[3], aif[4], aif[5]};
        if (v >= 0) {
            double d[3] = {__dsub_rn(g.R[3 * ci], g.R[3 * v]), __dsub_rn(g.R[3 * ci + 1], g.R[3 * v + 1]),
                           __dsub_rn(g.R[3 * ci + 2], g.R[3 * v + 2])};
            min_image(d, g.per, g.L);
            const double *aj = &g.A[6 * v];
            const Sym3 Aj{aj[0], aj[1], aj[2], aj[3], aj[4], aj[5]};
            gb_pair_mixed(d, Ai, Aj, Ai_f, g.smin, g.ismin, g.eps0, g.rho_floor, g.rho_cut, F, T, clamped);
        } else {
            const int w = -1 - v;
            double d[3] = {g.R[3 * ci] - (double)g.wall_xyz[3 * w], g.R[3 * ci + 1] - (double)g.wall_xyz[3 * w + 1],
                           g.R[3 * ci + 2] - (double)g.wall_xyz[3 * w + 2]};
            min_image(d, g.per, g.L);
            const Sym3 Aw{g.rw2, g.rw2, g.rw2, 0.0, 0.0, 0.0};
            gb_pair_mixed(d, Ai, Aw, Ai_f, g.smin_w, g.ismin_w, g.eps0, g.rho_floor, g.rho_cut, F, T, clamped);
        }
        for (int a = 0; a < 3; ++a) {
            s_res[e][a] = (double)F[a];
            s_res[e][3 + a] = (double)T[a];
        }
        if (clamped) atomicAdd(&s_clamped, clamped);
    }
    __syncthreads();
    // 5. every cell sums its own entries in queue order (deterministic),
    //    starting from its external force and torque
    if (i < g.nc && lane < 6) {
        double acc = g.ext ? g.ext[6 * i + lane] : 0.0;
        for (int e = s_qpre[wid]; e < s_qpre[wid + 1]; ++e) acc += s_res[e][lane];
        if (lane < 3)
            g.Fm[3 * i + lane] = acc;
        else
            g.Tm[3 * i + lane - 3] = acc;
    }
    if (threadIdx.x == 0 && s_clamped) atomicAdd(g.clamps, (unsigned long long)s_clamped);
}

// Grid-stride over the groups of kGbWarps cells: a grid smaller than the
// group count leaves room on the SMs for the kernels running beside it.
__global__ void __launch_bounds__(32 * kGbWarps) k_gb(GbArgs g)
{
    const int groups = (g.nc + kGbWarps - 1) / kGbWarps;
    for (int b = blockIdx.x; b < groups; b += gridDim.x) {
        gb_body(g, b);
        __syncthreads();  // the next group reuses the block's shared memory
    }
}

// ---------------------------------------------------------------------------
// Shape lists
// ---------------------------------------------------------------------------
struct ShapeArgs {
    float *hdr;
    const double *R, *q;
    const uint8_t *solid;
    const float4 *U, *S;  // node-major velocity (+ stress xz in w), stress xx yy zz xy
    const float *Syz;     // node-major stress yz
    float4 *G;            // node-major force density and hematocrit sum
    int2 *sp_idx;
    float4 *sp_val;
    int *sp_cnt, *flags;
    float *sp_S;
    int sp_cap;
    int nx, ny, nz;
    long long Np;
    float two_over_xi[3], xi[3], kappa, alpha;
    int kappa_i;  // kappa when it is a whole number 1..64 (integer power), else 0
    int box_dim, sup_cap;
    int box_pad;  // shared words per warp of k_weights (weights_words)
    const int4 *rows;  // compact layout: row table (offset, s_lo, s_hi, fluid range); null when dense
    int zero_entry;    // compact layout: the entry nothing writes (u = sigma = 0)
};

// ---------------------------------------------------------------------------
// k_weights: shape header and shape list of one cell, one warp per cell.
// Header: Q (FP32, from the unit quaternion), the box spanning the
// axis-aligned hull of the support |y_b| <= xi_b (half extent
// sum_b |Q_ab| xi_b) plus one node per side, its corner relative to R
// (FP64 difference), the centre node and a validity flag.  The box must
// have 1..box_dim nodes per axis and lie within one period of the lattice
// on each side; a cell that left the box or went non-finite is flagged and
// skipped by the per-cell kernel.
// Weights w = prod_b phi(2 y_b / xi_b), y = Q^T (x - R) (Sec. 2.2), 0 at
// solid nodes, vanish outside the parallelepiped |y_b| < xi_b.  Per box row
// (i1, i2) the kernel solves the three slab constraints for the row's
// support interval along x (widened by 1e-3: nodes outside evaluate to 0)
// and evaluates w only there, one lane per support node, into a compact
// array (a row index per item replaces a search).  Per row it then visits
// the union of its own support widened by one node and the supports of its
// four neighbour rows -- every node where w or its central difference D w
// can be non-zero -- one lane per row walking x with w(x - 1), w(x), w(x + 1)
// in registers.  The list holds every visited node, in lattice order (z, y,
// x), with the lattice index, box coordinates (i0 | i1 << 10 | i2 << 20), w
// and D w (all four zero at the few visited nodes where they vanish); S is
// the sum of w over fluid nodes.
// Shared memory per warp (weights_words): row words (support lo | hi << 8 |
// first item << 16), visit words (same layout), the rows that have visit
// items (row | first item << 16, in row order), the compact weights and the
// row of every support item (16 bits).
// ---------------------------------------------------------------------------
constexpr int kWtWarps = 4;

int weights_words(const Params &p)
{
    return 3 * p.box_dim * p.box_dim + p.sup_cap + (p.sup_cap + 1) / 2;
}

// support interval [lo, hi] of box row (i1, i2) along x; lo > hi if empty.
// lim[b] = 2 / t[b] = xi_b and iq[b] = 1 / Q_xb are the cell's, computed once.
__device__ __forceinline__ void support_row(const float Q[9], const float bs[3], const float lim3[3],
                                            const float iq3[3], int n0, int i1, int i2, int &lo, int &hi)
{
    const float r1 = bs[1] + (float)i1, r2 = bs[2] + (float)i2;
    float flo = -1e30f, fhi = 1e30f;
    bool empty = false;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const float cb = Q[3 + b] * r1 + Q[6 + b] * r2;  // y_b without the x term
        const float lim = lim3[b];                          // |y_b| < xi_b
        if (fabsf(Q[b]) < 1e-7f) {
            empty |= fabsf(cb) >= lim * 1.0001f;
            continue;
        }
        const float iq = iq3[b];
        const float u1 = (-lim - cb) * iq, u2 = (lim - cb) * iq;
        flo = fmaxf(flo, fminf(u1, u2));
        fhi = fminf(fhi, fmaxf(u1, u2));
    }
    flo -= bs[0];
    fhi -= bs[0];
    if (empty || !(flo <= fhi)) {
        lo = 1;
        hi = 0;
        return;
    }
    lo = (int)fmaxf(ceilf(flo - 1e-3f), 0.0f);
    hi = (int)fminf(floorf(fhi + 1e-3f), (float)(n0 - 1));
}

__device__ __forceinline__ void weights_body(const ShapeArgs &a, int nc, int blk)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blk * kWtWarps + warp;
    if (i >= nc) return;
    const int rows_cap = a.box_dim * a.box_dim;
    unsigned *srow = reinterpret_cast<unsigned *>(smem + (size_t)warp * a.box_pad);
    unsigned *vrow = srow + rows_cap;
    unsigned *vne = vrow + rows_cap;
    float *wc = reinterpret_cast<float *>(vne + rows_cap);
    uint16_t *srowof = reinterpret_cast<uint16_t *>(wc + a.sup_cap);
    const float qm = lane < 4 ? (float)a.q[4 * i + lane] : 0.f;
    float qf[4], Q[9];
#pragma unroll
    for (int k = 0; k < 4; ++k) qf[k] = __shfl_sync(0xffffffffu, qm, k);
    quat_matrix_f(qf, Q);
    // the box along axis `lane` (lanes 0-2)
    int lo = 0, n = 1, ctr = 0;
    float base = 0.f;
    bool okl = true;
    if (lane < 3) {
        const int dim = lane == 0 ? a.nx : (lane == 1 ? a.ny : a.nz);
        const float q0 = lane == 0 ? Q[0] : (lane == 1 ? Q[3] : Q[6]);
        const float q1 = lane == 0 ? Q[1] : (lane == 1 ? Q[4] : Q[7]);
        const float q2 = lane == 0 ? Q[2] : (lane == 1 ? Q[5] : Q[8]);
        const float e = fabsf(q0) * a.xi[0] + fabsf(q1) * a.xi[1] + fabsf(q2) * a.xi[2];
        const double Rd = a.R[3 * i + lane];
        if (fabs(Rd) < 1e7 && e < 1e7f) {
            lo = (int)ceil(Rd - (double)e) - 1;
            const int hi = (int)floor(Rd + (double)e) + 1;
            n = hi - lo + 1;
            okl = !(n < 1 || n > a.box_dim || lo < -dim || hi >= 2 * dim);
            ctr = wrap1((int)floor(Rd + 0.5), dim);
            base = (float)((double)lo - Rd);
        } else {
            okl = false;
        }
    }
    bool ok = __all_sync(0xffffffffu, okl);
    int o[3], nn[3], cc[3];
    float bs[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        o[ax] = __shfl_sync(0xffffffffu, lo, ax);
        nn[ax] = __shfl_sync(0xffffffffu, n, ax);
        cc[ax] = __shfl_sync(0xffffffffu, ctr, ax);
        bs[ax] = __shfl_sync(0xffffffffu, base, ax);
    }
    const int n0 = nn[0], n1 = nn[1], n2 = nn[2], nrows = n1 * n2;
    const float inv1 = 1.0f / (float)n1;
    const float tq[3] = {a.two_over_xi[0], a.two_over_xi[1], a.two_over_xi[2]};
    float lim3[3], iq3[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        lim3[b] = 2.0f / tq[b];
        iq3[b] = fabsf(Q[b]) < 1e-7f ? 0.0f : 1.0f / Q[b];
    }
    // 1. support interval and first item of every row
    int stot = 0;
    if (ok) {
        for (int rb = 0; rb < nrows; rb += 32) {
            const int r = rb + lane;
            int slo = 1, shi = 0;
            if (r < nrows) {
                const int i2 = (int)(((float)r + 0.5f) * inv1), i1 = r - i2 * n1;
                support_row(Q, bs, lim3, iq3, n0, i1, i2, slo, shi);
            }
            const int len = slo <= shi ? shi - slo + 1 : 0;
            int incl = len;
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            const int first = stot + incl - len;
            if (r < nrows) srow[r] = (slo <= shi ? (unsigned)(slo | (shi << 8)) : 0xFFu) | ((unsigned)first << 16);
            if (first + len <= a.sup_cap)
                for (int k = 0; k < len; ++k) srowof[first + k] = (uint16_t)r;
            stot += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (stot > a.sup_cap) ok = false;
    }
    float *h = &a.hdr[kHdrWords * i];
    int *hi_ = reinterpret_cast<int *>(h);
    if (!ok) {
        if (lane == 0) {
            hi_[18] = 0;
            hi_[19] = 0;
            a.sp_cnt[i] = 0;
            a.sp_S[i] = 0.f;
            atomicOr(&a.flags[FLAG_OVERFLOW], OVF_BOX);
        }
        return;
    }
    __syncwarp();
    // 2. visit interval and first item of every row, and the list of the
    //    rows that have visit items (many box rows miss the cell)
    int vtot = 0, nne = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int rb = 0; rb < nrows; rb += 32) {
        const int r = rb + lane;
        int vlo = 1 << 20, vhi = -1;
        if (r < nrows) {
            const int i2 = (int)(((float)r + 0.5f) * inv1), i1 = r - i2 * n1;
            const int own = (int)(srow[r] & 0xFFFFu);
            if ((own & 0xFF) <= (own >> 8)) {
                vlo = (own & 0xFF) - 1;
                vhi = (own >> 8) + 1;
            }
            const int nb[4] = {i1 > 0 ? r - 1 : -1, i1 + 1 < n1 ? r + 1 : -1, i2 > 0 ? r - n1 : -1,
                               i2 + 1 < n2 ? r + n1 : -1};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (nb[k] < 0) continue;
                const int wk = (int)(srow[nb[k]] & 0xFFFFu);
                if ((wk & 0xFF) > (wk >> 8)) continue;
                vlo = min(vlo, wk & 0xFF);
                vhi = max(vhi, wk >> 8);
            }
            vlo = max(vlo, 0);
            vhi = min(vhi, n0 - 1);
        }
        const int len = vlo <= vhi ? vhi - vlo + 1 : 0;
        int incl = len;
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (r < nrows) vrow[r] = (len > 0 ? (unsigned)(vlo | (vhi << 8)) : 0xFFu) | ((unsigned)(vtot + incl - len) << 16);
        const unsigned ne = __ballot_sync(0xffffffffu, len > 0);
        if (len > 0) vne[nne + __popc(ne & lt)] = (unsigned)r | ((unsigned)(vtot + incl - len) << 16);
        nne += __popc(ne);
        vtot += __shfl_sync(0xffffffffu, incl, 31);
    }
    // 3. weights over the support items
    const int nxy = a.nx * a.ny;
    float part = 0.f;
    for (int t = lane; t < stot; t += 32) {
        const int r = srowof[t];
        const unsigned word = srow[r];
        const int i0 = (int)(word & 0xFFu) + (t - (int)(word >> 16));
        const int i2 = (int)(((float)r + 0.5f) * inv1), i1 = r - i2 * n1;
        const float r0 = bs[0] + (float)i0, r1 = bs[1] + (float)i1, r2 = bs[2] + (float)i2;
        float w = peskin4((Q[0] * r0 + Q[3] * r1 + Q[6] * r2) * tq[0]);
        if (w != 0.f) w *= peskin4((Q[1] * r0 + Q[4] * r1 + Q[7] * r2) * tq[1]);
        if (w != 0.f) w *= peskin4((Q[2] * r0 + Q[5] * r1 + Q[8] * r2) * tq[2]);
        if (w != 0.f && a.solid != nullptr &&
            a.solid[wrap1(o[0] + i0, a.nx) + a.nx * wrap1(o[1] + i1, a.ny) + nxy * wrap1(o[2] + i2, a.nz)])
            w = 0.f;
        wc[t] = w;
        part += w;
    }
    __syncwarp();
    // w at column x of the row with support word `word` (0xFF: empty); 0
    // outside the row's support
    auto W = [&](unsigned word, int x) -> float {
        const int slo = (int)(word & 0xFFu), shi = (int)((word >> 8) & 0xFFu);
        return (x >= slo && x <= shi) ? wc[(int)(word >> 16) + x - slo] : 0.f;
    };
    // 4. the visit items, one lane per item, so that consecutive lanes write
    //    consecutive list entries: the item's row is reached by walking the
    //    list of rows with items forward from the row of the previous
    //    round's last item.  This phase is 57 % of the kernel's instructions
    //    (per item five support words, seven weight lookups and the storage
    //    entry)
    int2 *sp_idx = a.sp_idx + (size_t)i * a.sp_cap;
    float4 *sp_val = a.sp_val + (size_t)i * a.sp_cap;
    const int vcount = min(vtot, a.sp_cap);
    int kstart = 0;
    for (int t0 = 0; t0 < vcount; t0 += 32) {
        const int t = t0 + lane;
        int k = kstart;
        if (t < vcount)
            while (k + 1 < nne && (int)(vne[k + 1] >> 16) <= t) ++k;
        kstart = __shfl_sync(0xffffffffu, k, 31);
        if (t >= vcount) continue;
        const int r = (int)(vne[k] & 0xFFFFu);
        const unsigned vw = vrow[r];
        const int x = (int)(vw & 0xFFu) + (t - (int)(vw >> 16));
        const int i2 = (int)(((float)r + 0.5f) * inv1), i1 = r - i2 * n1;
        const unsigned own = srow[r];
        const unsigned ym = i1 > 0 ? srow[r - 1] : 0xFFu, yp = i1 + 1 < n1 ? srow[r + 1] : 0xFFu;
        const unsigned zm = i2 > 0 ? srow[r - n1] : 0xFFu, zp = i2 + 1 < n2 ? srow[r + n1] : 0xFFu;
        // storage entry of column xw of this lattice row: dense, the node
        // index; compact, the row's offset + xw - s_lo inside the row's span
        // (every visited node is there: it lies within one node of a fluid
        // support node), the zero entry otherwise
        const int lrow = wrap1(o[1] + i1, a.ny) + a.ny * wrap1(o[2] + i2, a.nz);
        int ebase = a.nx * lrow, elo = 0, ehi = a.nx;
        if (a.rows) {
            const int4 rt = __ldg(&a.rows[lrow]);
            ebase = rt.x - rt.y;
            elo = rt.y;
            ehi = rt.z;
        }
        const int xw = wrap1(o[0] + x, a.nx);
        sp_idx[t] = make_int2(xw >= elo && xw < ehi ? ebase + xw : a.zero_entry, x | (i1 << 10) | (i2 << 20));
        sp_val[t] = make_float4(W(own, x), 0.5f * (W(own, x + 1) - W(own, x - 1)), 0.5f * (W(yp, x) - W(ym, x)),
                                0.5f * (W(zp, x) - W(zm, x)));
    }
    const int run = vtot;
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if (lane == 0) {
        for (int k = 0; k < 9; ++k) h[k] = Q[k];
        for (int ax = 0; ax < 3; ++ax) {
            h[9 + ax] = bs[ax];
            hi_[12 + ax] = o[ax];
            hi_[15 + ax] = nn[ax];
        }
        int centre = cc[0] + a.nx * (cc[1] + a.ny * cc[2]);
        if (a.rows) {
            const int4 rt = a.rows[cc[1] + a.ny * cc[2]];
            centre = cc[0] >= rt.y && cc[0] < rt.z ? rt.x + cc[0] - rt.y : a.zero_entry;
        }
        hi_[18] = centre;
        hi_[19] = 1;
        a.sp_cnt[i] = min(run, a.sp_cap);
        a.sp_S[i] = part;
        if (run > a.sp_cap) atomicOr(&a.flags[FLAG_OVERFLOW], OVF_BOX);
    }
}

// Grid-stride over the groups of kWtWarps cells (see k_gb).
__global__ void __launch_bounds__(32 * kWtWarps) k_weights(ShapeArgs a, int nc)
{
    const int groups = (nc + kWtWarps - 1) / kWtWarps;
    for (int b = blockIdx.x; b < groups; b += gridDim.x) {
        weights_body(a, nc, b);
        __syncwarp();  // the warp's next cell reuses its shared memory
    }
}

// ---------------------------------------------------------------------------
// Sampling over the cell's shape list (one warp per cell):
// S = sum w;  u~ S = sum w u;  omega~ S = -sum D w x (u - u_c)  (summation by
// parts of the central-difference curl; sum D w vanishes over the box, so
// the constant u_c = u at the centre node changes nothing in exact
// arithmetic and removes FP32 cancellation);  T^S S / alpha =
// sum w (sigma n) x (x - R), n = D w / |D w|  (Eqs. vel, vort,
// pheno_torque_diss).  Lane partial sums, then a fixed shuffle tree: every
// lane ends with the 9 sums.
// ---------------------------------------------------------------------------
// List entries per lane in flight.  Each entry's u and stress gathers issue
// together, after the list loads: two dependent memory round trips per
// group instead of three (the stress had been gathered after the velocity
// sums): tube step 1.173 -> 1.159 ms.  Four entries need 80 registers (six
// blocks per SM: 1.162 ms) or spill at 72 (1.208 ms).  The stress is
// gathered only where w > 0 (the torque's other entries, the rim of the
// list where only D w is non-zero, need u alone): 1.159 -> 1.142 ms.
constexpr int kIlp = 3;

// Sums over the entries part, part + parts, ... (in units of 32) of cell
// i's list: this warp's share when `parts` warps sample one cell.
template <bool ALPHA>
__device__ __forceinline__ void sample_sums(const ShapeArgs &a, int i, int n, float S, float (&acc)[9], int part,
                                            int parts)
{
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < 9; ++k) acc[k] = 0.f;
    if (n == 0) return;
    const float *hd = &a.hdr[kHdrWords * i];
    const int gc = reinterpret_cast<const int *>(hd)[18];
    const float4 uc = a.U[gc];
    const float uc0 = uc.x, uc1 = uc.y, uc2 = uc.z;
    const float b0 = hd[9], b1 = hd[10], b2 = hd[11];
    const float thr = 1e-24f * S * S;
    const int2 *idx = a.sp_idx + (size_t)i * a.sp_cap;
    const float4 *val = a.sp_val + (size_t)i * a.sp_cap;
    // kIlp independent entries per lane in flight: the list loads of all of
    // them, then all their gathers (u, and the stress where the torque
    // needs it), before any sum uses them
    for (int e0 = lane + 32 * part; e0 < n; e0 += 32 * parts * kIlp) {
        int2 ix[kIlp];
        float4 v[kIlp];
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            const int e = e0 + 32 * parts * j;
            ix[j] = e < n ? idx[e] : make_int2(gc, 0);
            v[j] = e < n ? val[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float4 u4[kIlp], s4[kIlp];
        float syz[kIlp];
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            const int g = ix[j].x;
            u4[j] = a.U[g];
            if (ALPHA) {
                s4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                syz[j] = 0.f;
                if (v[j].x > 0.f) {  // the torque needs the stress only where w > 0
                    s4[j] = a.S[g];
                    syz[j] = a.Syz[g];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            acc[0] += v[j].x * u4[j].x;
            acc[1] += v[j].x * u4[j].y;
            acc[2] += v[j].x * u4[j].z;
            const float vx = u4[j].x - uc0, vy = u4[j].y - uc1, vz = u4[j].z - uc2;
            acc[3] -= v[j].z * vz - v[j].w * vy;
            acc[4] -= v[j].w * vx - v[j].y * vz;
            acc[5] -= v[j].y * vy - v[j].z * vx;
            if (ALPHA) {
                const float d2 = v[j].y * v[j].y + v[j].z * v[j].z + v[j].w * v[j].w;
                if (!(v[j].x > 0.f && d2 > thr)) continue;
                const float inv = rsqrtf(d2);
                const float nx = v[j].y * inv, ny = v[j].z * inv, nz = v[j].w * inv;
                // sigma components: xx = s.x, yy = s.y, zz = s.z, xy = s.w, xz = u.w, yz
                const float tx = s4[j].x * nx + s4[j].w * ny + u4[j].w * nz;
                const float ty = s4[j].w * nx + s4[j].y * ny + syz[j] * nz;
                const float tz = u4[j].w * nx + syz[j] * ny + s4[j].z * nz;
                const int pk = ix[j].y;
                const float r0 = b0 + (float)(pk & 1023), r1 = b1 + (float)((pk >> 10) & 1023),
                            r2 = b2 + (float)(pk >> 20);
                acc[6] += v[j].x * (ty * r2 - tz * r1);
                acc[7] += v[j].x * (tz * r0 - tx * r2);
                acc[8] += v[j].x * (tx * r1 - ty * r0);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
}

// ---------------------------------------------------------------------------
// k_rigid: App. A, FP64, one thread per cell
// ---------------------------------------------------------------------------
struct RigidArgs {
    double *R, *q, *V, *Om;
    const double *Fm, *Tm;
    const float *hdr;
    int *have, *flags;
    double *diag;
    int nc;
    double L[3];
    int per[3];
    // FP32 constants; aT[c] = eT^2 - 1 (c = 1: previous step closed here)
    // or eT - 1 (c = 0: first step), aR likewise
    float M, I[3], iM, iI[3], eT, eR, gT, gR, alpha, aT[2], aR[2];
};


// App. A for one cell, run by the cell's warp.  The state (R, q, V, Omega)
// stays in FP64; the step's changes are computed in FP32 from forms without
// cancellation and added to it once in FP64 (FP64 runs at a small fraction
// of the FP32 rate on this part, so each FP64 value is handled by one lane:
// lanes 0-2 R and V, 3-5 Omega, 6-9 q, 10-15 F^mech and T^mech; the FP32
// work is the same in all lanes).  With b = 1 when the previous step is
// closed here (b = 1/2 on the first step), aT = eT^2 - 1 (eT - 1) and
// F^comb = F^mech + gamma_T M u~,
// T^comb = Q^T (T^mech + T^S) + gamma_R I Q^T omega~:
//   V'  - V0  = aT V0 + b eT F^comb / M                    (steps 6-7, 1-2)
//   Om' - Om0 = aR Om0 + b eR T^comb / I
//   J = M (V' - V0) - b F^mech
//     = M aT V0 + b (eT - 1) F^mech + b eT gamma_T M u~
//   L = Q I (Om' - Om0) - b T^mech
//     = Q I (aR Om0 + b eR gamma_R Q^T omega~) + b ((eR - 1) T^mech + eR T^S)
// The sub-rotations of step 4 (body axes 1, 2, 3, 2, 1 by h Om/2, h Om/2,
// h Om, h Om/2, h Om/2) turn q by r = (cos t/2, sin t/2 e_k) and the
// momenta pi = I Om about e_k by t; both are applied as increments,
// q r - q = q (r - 1) with cos(t/2) - 1 = -sin^2(t/2) / (1 + cos(t/2)),
// and cos t - 1 = -2 sin^2(t/2), sin t = 2 sin(t/2) cos(t/2).  The stored
// q has unit norm (rbc_init normalises it, every step renormalises), so
// |q + dq|^2 - 1 = e = 2 q.dq + dq.dq and the renormalised q is
// (q + dq)(1 + s), s = -e/2 + 3e^2/8.
// J and L are handed to `publish` as soon as they exist, before the
// sub-rotations (which only the stored state needs).  Returns false, with
// no update and without calling publish, when the cell has no valid shape
// box or S = 0.

template <typename Publish>
__device__ __forceinline__ bool rigid_update(const RigidArgs &a, int i, float Sf, const float (&sums)[9],
                                             Publish &&publish)
{
    const int lane = threadIdx.x & 31;
    const int ok = reinterpret_cast<const int *>(a.hdr)[kHdrWords * i + 19];
    if (!ok || !(Sf > 0.f)) {
        if (ok && lane == 0) atomicOr(&a.flags[FLAG_UNSTABLE], 2);
        return false;
    }
    double mine = 0.0, Rd = 0.0;
    if (lane < 3) {
        mine = a.V[3 * i + lane];
        Rd = a.R[3 * i + lane];
    } else if (lane < 6) {
        mine = a.Om[3 * i + lane - 3];
    } else if (lane < 10) {
        mine = a.q[4 * i + lane - 6];
    } else if (lane < 13) {
        mine = a.Fm[3 * i + lane - 10];
    } else if (lane < 16) {
        mine = a.Tm[3 * i + lane - 13];
    }
    const float mf = (float)mine;
    float V0[3], W0[3], qf[4], Fm[3], Tm[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        V0[d] = __shfl_sync(0xffffffffu, mf, d);
        W0[d] = __shfl_sync(0xffffffffu, mf, 3 + d);
        Fm[d] = __shfl_sync(0xffffffffu, mf, 10 + d);
        Tm[d] = __shfl_sync(0xffffffffu, mf, 13 + d);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) qf[k] = __shfl_sync(0xffffffffu, mf, 6 + k);
    float Q[9];
    quat_matrix_f(qf, Q);
    const float iS = 1.0f / Sf;
    const int c = a.have[i] != 0 ? 1 : 0;
    const float b = c ? 1.0f : 0.5f, aT = a.aT[c], aR = a.aR[c];
    float ut[3], wt[3], TS[3], Tl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        ut[d] = sums[d] * iS;
        wt[d] = sums[3 + d] * iS;
        TS[d] = a.alpha * sums[6 + d] * iS;
        Tl[d] = Tm[d] + TS[d];
    }
    float dV[3], dW[3], Lb[3], J[3], Lm[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float Fc = Fm[d] + a.gT * a.M * ut[d];
        const float Tb = Q[d] * Tl[0] + Q[3 + d] * Tl[1] + Q[6 + d] * Tl[2];
        const float wb = Q[d] * wt[0] + Q[3 + d] * wt[1] + Q[6 + d] * wt[2];
        const float Tc = Tb + a.gR * a.I[d] * wb;
        dV[d] = aT * V0[d] + b * a.eT * Fc * a.iM;
        dW[d] = aR * W0[d] + b * a.eR * Tc * a.iI[d];
        J[d] = a.M * aT * V0[d] + b * (a.eT - 1.0f) * Fm[d] + b * a.eT * a.gT * a.M * ut[d];
        Lb[d] = a.I[d] * (aR * W0[d] + b * a.eR * a.gR * wb);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        Lm[d] = Q[3 * d] * Lb[0] + Q[3 * d + 1] * Lb[1] + Q[3 * d + 2] * Lb[2] +
                b * ((a.eR - 1.0f) * Tm[d] + a.eR * TS[d]);
    publish(J, Lm);
    // step 4 in increments: dq accumulates q r - q, dW the momentum turns
    float Wf[3] = {W0[0] + dW[0], W0[1] + dW[1], W0[2] + dW[2]};
    float dq[4] = {0.f, 0.f, 0.f, 0.f};
    const int ax[5] = {0, 1, 2, 1, 0};
    const float fr[5] = {0.5f, 0.5f, 1.0f, 0.5f, 0.5f};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int k = ax[s];
        const float th = fr[s] * Wf[k];
        float sh, ch;
        sincosf(0.5f * th, &sh, &ch);
        const float cm1 = -sh * sh / (1.0f + ch);
        float r[4] = {cm1, 0.f, 0.f, 0.f};  // r - 1
        r[1 + k] = sh;
        const float w1 = qf[0] + dq[0], x1 = qf[1] + dq[1], y1 = qf[2] + dq[2], z1 = qf[3] + dq[3];
        dq[0] += w1 * r[0] - x1 * r[1] - y1 * r[2] - z1 * r[3];
        dq[1] += w1 * r[1] + x1 * r[0] + y1 * r[3] - z1 * r[2];
        dq[2] += w1 * r[2] - x1 * r[3] + y1 * r[0] + z1 * r[1];
        dq[3] += w1 * r[3] + x1 * r[2] - y1 * r[1] + z1 * r[0];
        const float st = 2.0f * sh * ch, ctm1 = -2.0f * sh * sh;
        const int p1 = (k + 1) % 3, p2 = (k + 2) % 3;
        const float pi1 = a.I[p1] * Wf[p1], pi2 = a.I[p2] * Wf[p2];
        const float d1 = (ctm1 * pi1 + st * pi2) * a.iI[p1];
        const float d2 = (ctm1 * pi2 - st * pi1) * a.iI[p2];
        Wf[p1] += d1;
        Wf[p2] += d2;
        dW[p1] += d1;
        dW[p2] += d2;
    }
    // FP64 state, one value per lane
    if (lane < 3) {
        const double V = mine + (double)pick(dV, lane);
        double R = Rd + V;  // step 3: drift
        if (a.per[lane]) {
            if (R >= a.L[lane])
                R -= a.L[lane];
            else if (R < 0.0)
                R += a.L[lane];
        }
        a.V[3 * i + lane] = V;
        a.R[3 * i + lane] = R;
    } else if (lane < 6) {
        a.Om[3 * i + lane - 3] = mine + (double)pick(dW, lane - 3);
    } else if (lane < 10) {
        const float e = 2.0f * (qf[0] * dq[0] + qf[1] * dq[1] + qf[2] * dq[2] + qf[3] * dq[3]) +
                        (dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2] + dq[3] * dq[3]);
        const float sc = e * (-0.5f + 0.375f * e);
        const int k = lane - 6;
        const float dk = pick(dq, k);
        a.q[4 * i + k] = mine + (double)(dk + (pick(qf, k) + dk) * sc);
    }
    // diagnostics: F^mech, tau^mech (FP64 copies), u~, omega~, T^S, J, L
    double *o = &a.diag[21 * i];
    if (lane >= 10 && lane < 16) {
        o[lane - 10] = mine;
    } else if (lane >= 16 && lane < 31) {
        const float v[15] = {ut[0], ut[1], ut[2], wt[0], wt[1], wt[2], TS[0], TS[1], TS[2],
                             J[0],  J[1],  J[2],  Lm[0], Lm[1], Lm[2]};
        o[6 + lane - 16] = (double)pick(v, lane - 16);
    }
    if (lane == 0) a.have[i] = 1;
    return true;
}


// ---------------------------------------------------------------------------
// k_cells: the per-cell part of the coupled step, one warp per cell.
//   1. sample the fields over the cell's shape list (sample_sums);
//   2. the rigid-body update and the hydrodynamic impulses J, L (App. A);
//   3. spread (h = 1) over the same list: G += -J delta + 1/2 L x D delta
//      (delta = w / S) and theta += 1 - (1 - w)^kappa where w > 0 (Sec.
//      2.2, Eq. enhance-viscosity), with atomics.
// A cell's spread writes only G and theta, which no sampling reads, so the
// cells of the kernel need no order among themselves.
// ---------------------------------------------------------------------------
// (1 - w)^kappa of Eq. enhance-viscosity: by squaring for a whole-number
// kappa (the paper's 20: five multiplications), powf otherwise
__device__ __forceinline__ float pow_kappa(float x, const ShapeArgs &a)
{
    if (a.kappa_i <= 0) return powf(x, a.kappa);
    float r = 1.0f, b = x;
    for (int e = a.kappa_i; e > 0; e >>= 1) {
        if (e & 1) r *= b;
        b *= b;
    }
    return r;
}

// At most 72 registers so that 7 blocks fit an SM: the kernel waits on
// memory and wants the warps (at 80 registers, 6 blocks per SM ran 3,650
// cells as two full waves and a last one of a single block; at 64, 8
// blocks, the stress sampling spilled and the channel step took 3 % longer).
constexpr int kCellBlocksPerSm = 7;

// One warp per cell samples the whole list, runs the rigid update and
// spreads; four cells per block, no barriers between warps (the single-solve
// and the packed kernels alike).  Twice as many cells in flight per SM as a
// two-warp form (each cell taking longer) that split the sampling and handed
// J and L from a rigid-update warp to a spreading warp: the tube step
// 1,239 -> 1,221 us, the channel 108.2 -> 105.7 us.
constexpr int kCellWarps = 4;

// Spread (step 3) of cell i over its list, with J / S and L / 2S in jl.
__device__ __forceinline__ void spread_list(const ShapeArgs &a, int i, int n, int lane, const float (&jl)[6])
{
    const float Jx = jl[0], Jy = jl[1], Jz = jl[2], Lx = jl[3], Ly = jl[4], Lz = jl[5];
    const int2 *idx = a.sp_idx + (size_t)i * a.sp_cap;
    const float4 *val = a.sp_val + (size_t)i * a.sp_cap;
    // few values are live in the spread: eight entries per lane in flight
    // (against four: tube step 1,221 -> 1,206 us, channel 105.5 -> 103.6 us)
    constexpr int kIlpSpread = 8;
    for (int e0 = lane; e0 < n; e0 += 32 * kIlpSpread) {
        int g[kIlpSpread];
        float4 v[kIlpSpread];
#pragma unroll
        for (int j = 0; j < kIlpSpread; ++j) {
            const int e = e0 + 32 * j;
            g[j] = e < n ? idx[e].x : -1;
            v[j] = e < n ? val[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kIlpSpread; ++j) {
            if (g[j] < 0) continue;
            atomicAdd(&a.G[g[j]], make_float4(-Jx * v[j].x + (Ly * v[j].w - Lz * v[j].z),
                                              -Jy * v[j].x + (Lz * v[j].y - Lx * v[j].w),
                                              -Jz * v[j].x + (Lx * v[j].z - Ly * v[j].y),
                                              v[j].x > 0.f ? 1.0f - pow_kappa(1.0f - v[j].x, a) : 0.f));
        }
    }
}

// Steps 1 and 2 of cell i, then step 3 here (SPREAD) or, for k_spread,
// J / S, L / 2S and the go flag to jl_out[8 i ..].
template <bool ALPHA, bool SPREAD = true>
__device__ __forceinline__ void cells_body(const ShapeArgs &a, const RigidArgs &ra, int nc, int i,
                                           float *jl_out = nullptr)
{
    if (i >= nc) return;  // uniform across the warp
    const int lane = threadIdx.x & 31;
    const int n = a.sp_cnt[i];
    const float S = a.sp_S[i];
    float sums[9];
    sample_sums<ALPHA>(a, i, n, S, sums, 0, 1);
    float jl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool go = false;
    auto publish = [&](const float (&J)[3], const float (&L)[3]) {
        go = n > 0;
        const float iS = go ? 1.0f / S : 0.f;
        for (int d = 0; d < 3; ++d) {
            jl[d] = J[d] * iS;
            jl[3 + d] = 0.5f * L[d] * iS;
        }
    };
    rigid_update(ra, i, S, sums, publish);
    if (!SPREAD) {
        if (lane < 6) jl_out[8 * i + lane] = pick(jl, lane);
        if (lane == 6) jl_out[8 * i + 6] = go ? 1.f : 0.f;
        return;
    }
    if (go) spread_list(a, i, n, lane, jl);
}

template <bool ALPHA, bool SPREAD>
__global__ void __launch_bounds__(32 * kCellWarps, kCellBlocksPerSm) k_cells(ShapeArgs a, RigidArgs ra, int nc,
                                                                             float *jl)
{
    cells_body<ALPHA, SPREAD>(a, ra, nc, blockIdx.x * kCellWarps + (int)(threadIdx.x >> 5), jl);
}

// The spread as a kernel of its own: only the lattice pass waits for it,
// the next step's cell list, Gay-Berne forces and shape lists run beside it.
__global__ void __launch_bounds__(32 * kCellWarps) k_spread(ShapeArgs a, const float *__restrict__ jl, int nc)
{
    const int i = blockIdx.x * kCellWarps + (int)(threadIdx.x >> 5);
    if (i >= nc || jl[8 * i + 6] == 0.f) return;
    const float v[6] = {jl[8 * i], jl[8 * i + 1], jl[8 * i + 2], jl[8 * i + 3], jl[8 * i + 4], jl[8 * i + 5]};
    spread_list(a, i, a.sp_cnt[i], (int)(threadIdx.x & 31), v);
}

ShapeArgs shape_args(const Dev &d, const Params &p, int buf)
{
    ShapeArgs a;
    a.hdr = d.hdr;
    a.R = d.R;
    a.q = d.q;
    a.solid = d.solid;
    a.U = d.U;
    a.S = d.S;
    a.Syz = d.Syz;
    a.G = d.G;
    a.sp_idx = d.sp_idx[buf];
    a.sp_val = d.sp_val[buf];
    a.sp_cnt = d.sp_cnt[buf];
    a.sp_S = d.sp_S[buf];
    a.sp_cap = d.sp_cap;
    a.flags = d.flags;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.Np = d.Np;
    for (int k = 0; k < 3; ++k) {
        a.two_over_xi[k] = 2.0f / p.xi[k];
        a.xi[k] = p.xi[k];
    }
    a.box_dim = p.box_dim;
    a.box_pad = weights_words(p);
    a.sup_cap = p.sup_cap;
    a.kappa = p.kappa;
    a.kappa_i = (p.kappa >= 1.0f && p.kappa <= 64.0f && p.kappa == floorf(p.kappa)) ? (int)p.kappa : 0;
    a.alpha = p.alpha;
    a.rows = d.compact ? d.rows : nullptr;
    a.zero_entry = d.zero_entry;
    return a;
}

}  // namespace

// ---------------------------------------------------------------------------
// Packed launches: one launch of each per-cell kernel over the cells of
// several solves (the request server's packs).  Block b belongs to the solve
// i with start[i] <= b < start[i + 1] (found by binary search) and runs the
// kernel body with the solve's arguments from the table and its local block
// index.
// ---------------------------------------------------------------------------
struct CellPackEntry {
    BinArgs bin;
    GbArgs gb;
    ShapeArgs shape[2];  // shape-list buffer 0 / 1
    RigidArgs rigid;
    int *bin_count;
    int nbins;
};

__device__ __forceinline__ int cell_pack_find(const int *start, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_binclear_packed(const CellPackEntry *tab, const int *start, int ninst)
{
    const int i = cell_pack_find(start, ninst, blockIdx.x);
    const int k = (blockIdx.x - start[i]) * blockDim.x + threadIdx.x;
    if (k < tab[i].nbins) tab[i].bin_count[k] = 0;
}

__global__ void __launch_bounds__(kBinThreads) k_bin_packed(const CellPackEntry *tab, const int *start, int ninst)
{
    const int i = cell_pack_find(start, ninst, blockIdx.x);
    bin_body(tab[i].bin, blockIdx.x - start[i]);
}

__global__ void __launch_bounds__(32 * kGbWarps) k_gb_packed(const CellPackEntry *tab, const int *start, int ninst)
{
    const int i = cell_pack_find(start, ninst, blockIdx.x);
    gb_body(tab[i].gb, blockIdx.x - start[i]);
}

__global__ void __launch_bounds__(32 * kWtWarps)
    k_weights_packed(const CellPackEntry *tab, const int *start, int ninst, int buf)
{
    const int i = cell_pack_find(start, ninst, blockIdx.x);
    weights_body(tab[i].shape[buf], tab[i].rigid.nc, blockIdx.x - start[i]);
}

template <bool ALPHA>
// The packed kernel reads each solve's arguments from the pack table: at
// the single-solve kernel's 72 registers it spilled 172 bytes; bounded at 5
// blocks per SM it does not (serving 4.75 -> 4.81 solves/s)
__global__ void __launch_bounds__(32 * kCellWarps, 5)
    k_cells_packed(const CellPackEntry *tab, const int *start, int ninst, int buf)
{
    const int i = cell_pack_find(start, ninst, blockIdx.x);
    cells_body<ALPHA>(tab[i].shape[buf], tab[i].rigid, tab[i].rigid.nc,
                       (blockIdx.x - start[i]) * kCellWarps + (int)(threadIdx.x >> 5));
}

static BinArgs bin_args(const Dev &d, const Params &p)
{
    BinArgs g;
    g.R = d.R;
    g.q = d.q;
    g.A = d.A;
    g.Rf = d.Rf;
    g.Af = d.Af;
    g.cell_bin = d.cell_bin;
    g.bin_count = d.bin_count;
    g.bin_cells = d.bin_cells;
    g.flags = d.flags;
    g.nc = d.nc;
    g.cap = d.bin_cap;
    for (int a = 0; a < 3; ++a) {
        g.nb[a] = d.nb[a];
        g.bs[a] = d.bin_size[a];
        g.a2[a] = p.a2[a];
    }
    return g;
}

// Cell-centre profile along one axis: every cell adds 1 to the 1-lattice-
// unit bin floor(R_axis) of its centre (positions live in [0, n_axis)).
// FP64 atomics of whole numbers: the sums are exact and independent of
// their order.
__global__ void k_profile(const double *__restrict__ R, int nc, int axis, int nbins, double *__restrict__ prof)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double r = R[3 * i + axis];
    if (!(r >= 0.0 && r < (double)nbins)) return;  // non-finite or outside: not counted
    atomicAdd(&prof[(int)r], 1.0);
}

void launch_profile(const Dev &d, int axis, cudaStream_t s)
{
    if (d.nc <= 0) return;
    const int nbins = axis == 0 ? d.nx : (axis == 1 ? d.ny : d.nz);
    k_profile<<<(d.nc + 255) / 256, 256, 0, s>>>(d.R, d.nc, axis, nbins, d.profile);
}

void launch_bin(const Dev &d, const Params &p, cudaStream_t s)
{
    if (d.nc == 0) return;
    cudaMemsetAsync(d.bin_count, 0, sizeof(int) * d.nbins, s);
    launch_prio(k_bin, (d.nc + kBinThreads - 1) / kBinThreads, kBinThreads, 0, s, d.side_prio, bin_args(d, p));
}

static GbArgs gb_args(const Dev &d, const Params &p)
{
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
    g.ext = d.ext;
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
    g.rho_cut_f = (float)(p.rho_cut * 1.001 + 1e-3);
    g.ismin = 1.0 / p.smin_cc;
    g.ismin_w = 1.0 / p.smin_w;
    g.Rf = d.Rf;
    g.Af = d.Af;
    // FP32 positions carry ~1e-7 relative error: outside a band of
    // 1e-3 + 2e-6 max(L) around r_cut the FP32 distance decides the same way
    // as the exact FP64 test
    const double band = 1e-3 + 2e-6 * (double)std::max(d.nx, std::max(d.ny, d.nz));
    const double rc = sqrt(p.rc2);
    g.rc_lo2 = (float)((rc - band) * (rc - band));
    g.rc_hi2 = (float)((rc + band) * (rc + band));
    g.rcw2_f = (float)(p.rcw2 * 1.0001 + 1e-3);
    for (int a = 0; a < 3; ++a) {
        g.Lf[a] = (float)dims[a];
        g.wnb[a] = d.wnb[a];
        g.wbs[a] = (float)d.wbin_size[a];
    }
    return g;
}

void launch_gb(const Dev &d, const Params &p, cudaStream_t s)
{
    if (d.nc == 0) return;
    const int groups = (d.nc + kGbWarps - 1) / kGbWarps;
    const int blocks = d.gb_grid > 0 && d.gb_grid < groups ? d.gb_grid : groups;
    launch_prio(k_gb, blocks, 32 * kGbWarps, 0, s, d.side_prio, gb_args(d, p));
}

size_t cells_smem_bytes(const Params &p) { return kWtWarps * (size_t)weights_words(p) * sizeof(float); }

void prepare_cells(const Params &p)
{
    raise_smem_limit((const void *)k_weights, (int)cells_smem_bytes(p));
    cudaFuncSetAttribute(k_weights, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

void launch_weights(const Dev &d, const Params &p, int buf, cudaStream_t s)
{
    if (d.nc == 0) return;
    const int groups = (d.nc + kWtWarps - 1) / kWtWarps;
    const int blocks = d.wt_grid > 0 && d.wt_grid < groups ? d.wt_grid : groups;
    launch_prio(k_weights, blocks, 32 * kWtWarps, cells_smem_bytes(p), s, d.side_prio, shape_args(d, p, buf), d.nc);
}

static RigidArgs rigid_args(const Dev &d, const Params &p)
{
    RigidArgs a;
    a.R = d.R;
    a.q = d.q;
    a.V = d.V;
    a.Om = d.Om;
    a.Fm = d.Fm;
    a.Tm = d.Tm;
    a.hdr = d.hdr;
    a.have = d.have;
    a.flags = d.flags;
    a.diag = d.diag;
    a.nc = d.nc;
    a.M = (float)p.M;
    a.iM = (float)p.iM;
    a.eT = (float)p.eT;
    a.eR = (float)p.eR;
    a.gT = (float)p.gT;
    a.gR = (float)p.gR;
    a.aT[0] = (float)(p.eT - 1.0);
    a.aT[1] = (float)((p.eT - 1.0) * (p.eT + 1.0));
    a.aR[0] = (float)(p.eR - 1.0);
    a.aR[1] = (float)((p.eR - 1.0) * (p.eR + 1.0));
    a.alpha = d.S != nullptr ? p.alpha : 0.0f;
    const int dims[3] = {d.nx, d.ny, d.nz};
    for (int k = 0; k < 3; ++k) {
        a.I[k] = (float)p.I[k];
        a.iI[k] = (float)p.iI[k];
        a.per[k] = p.periodic[k];
        a.L[k] = dims[k];
    }
    return a;
}

void launch_cells(const Dev &d, const Params &p, int buf, cudaStream_t s, bool split)
{
    if (d.nc == 0) return;
    const ShapeArgs a = shape_args(d, p, buf);
    const RigidArgs r = rigid_args(d, p);
    const int blocks = (d.nc + kCellWarps - 1) / kCellWarps;
    if (d.S != nullptr) {
        if (split)
            k_cells<true, false><<<blocks, 32 * kCellWarps, 0, s>>>(a, r, d.nc, d.jl);
        else
            k_cells<true, true><<<blocks, 32 * kCellWarps, 0, s>>>(a, r, d.nc, d.jl);
    } else {
        if (split)
            k_cells<false, false><<<blocks, 32 * kCellWarps, 0, s>>>(a, r, d.nc, d.jl);
        else
            k_cells<false, true><<<blocks, 32 * kCellWarps, 0, s>>>(a, r, d.nc, d.jl);
    }
}

void launch_spread(const Dev &d, const Params &p, int buf, cudaStream_t s)
{
    if (d.nc == 0) return;
    k_spread<<<(d.nc + kCellWarps - 1) / kCellWarps, 32 * kCellWarps, 0, s>>>(shape_args(d, p, buf), d.jl, d.nc);
}


// ---------------------------------------------------------------------------
// Packs (host side)
// ---------------------------------------------------------------------------
size_t cell_pack_entry_bytes() { return sizeof(CellPackEntry); }

int cell_pack_blocks(int nc, int nbins, int kind)
{
    switch (kind) {
    case PACK_CLEAR: return (nbins + 255) / 256;
    case PACK_BIN: return (nc + kBinThreads - 1) / kBinThreads;
    case PACK_GB: return (nc + kGbWarps - 1) / kGbWarps;
    case PACK_WEIGHTS: return (nc + kWtWarps - 1) / kWtWarps;
    default: return (nc + kCellWarps - 1) / kCellWarps;
    }
}

void fill_cell_pack_entry(const Dev &d, const Params &p, void *out)
{
    CellPackEntry e;
    std::memset(&e, 0, sizeof e);
    // the same argument structs the single-solve launches build
    e.bin = bin_args(d, p);
    e.gb = gb_args(d, p);
    e.shape[0] = shape_args(d, p, 0);
    e.shape[1] = shape_args(d, p, 1);
    e.rigid = rigid_args(d, p);
    e.bin_count = d.bin_count;
    e.nbins = d.nbins;
    std::memcpy(out, &e, sizeof e);
}

void launch_cells_packed(const CellPackDesc &k, int buf, bool alpha, cudaStream_t s)
{
    const CellPackEntry *tab = static_cast<const CellPackEntry *>(k.tab);
    if (alpha)
        k_cells_packed<true><<<k.blocks[PACK_CELLS], 32 * kCellWarps, 0, s>>>(tab, k.start[PACK_CELLS], k.ninst, buf);
    else
        k_cells_packed<false><<<k.blocks[PACK_CELLS], 32 * kCellWarps, 0, s>>>(tab, k.start[PACK_CELLS], k.ninst, buf);
}

void launch_bin_packed(const CellPackDesc &k, int prio, cudaStream_t s)
{
    const CellPackEntry *tab = static_cast<const CellPackEntry *>(k.tab);
    launch_prio(k_binclear_packed, k.blocks[PACK_CLEAR], 256, 0, s, prio, tab, k.start[PACK_CLEAR], k.ninst);
    launch_prio(k_bin_packed, k.blocks[PACK_BIN], kBinThreads, 0, s, prio, tab, k.start[PACK_BIN], k.ninst);
}

void launch_gb_packed(const CellPackDesc &k, int prio, cudaStream_t s)
{
    const CellPackEntry *tab = static_cast<const CellPackEntry *>(k.tab);
    launch_prio(k_gb_packed, k.blocks[PACK_GB], 32 * kGbWarps, 0, s, prio, tab, k.start[PACK_GB], k.ninst);
}

void launch_weights_packed(const CellPackDesc &k, const Params &p, int buf, int prio, cudaStream_t s)
{
    const CellPackEntry *tab = static_cast<const CellPackEntry *>(k.tab);
    launch_prio(k_weights_packed, k.blocks[PACK_WEIGHTS], 32 * kWtWarps, cells_smem_bytes(p), s, prio, tab,
                k.start[PACK_WEIGHTS], k.ninst, buf);
}

}  // namespace rbc
