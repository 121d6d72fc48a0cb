// lb.cu -- the fused D3Q19 lattice pass and the lattice reductions.
//
// One thread per lattice node.  Populations are stored as deviations
// d_p = f_p - w_p from the lattice weights, one plane of Np values per speed
// (x fastest), ping-ponged between two buffers: FP32 d_p, or in 16 bits
// (IEEE binary16 or bfloat16) the scaled deviation s_p = d_p S / w_p,
// rounded stochastically (or to nearest) on store; the collision is FP32
// either way.  The pass pulls the 19 post-collision values of the previous
// pass from the upstream nodes (halfway bounce-back from solid upstream
// nodes), reads and clears the force density and the smoothed hematocrit the
// cells spread, collides, stores the 19 new values to its own node and
// writes u and sigma for the cells to sample.  Bytes per fluid node with
// populations of e bytes: 19 e read + 19 e write, 16 read (G, theta), 12
// written (u), 24 written (sigma when alpha != 0), 4 read (link mask, walled
// lattices only), plus the 16-byte clear of G and theta.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "internal.h"
#include "rbc_device.cuh"

namespace rbc {

namespace {

constexpr int kLbThreads = 256;

__device__ __forceinline__ int wrapm(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

struct LbArgs {
    const void *src;  // populations of the previous pass (storage type St)
    void *dst;
    const uint32_t *links;
    const int4 *rows;  // compact layout: row table (internal.h), else null
    const int2 *pool;  // compact lattice pass: per batch segment, kSegDescs descriptors (produce_compact)
    float4 *G, *U, *S;  // node-major: force density + hematocrit sum, velocity (+ stress xz), stress xx yy zz xy
    float *Syz;         // node-major: stress yz
    int *flags;
    int *work;                 // [0] next batch, [1] CTAs done; zero at launch, reset by the last CTA
    unsigned long long *step;  // passes done: the counter of the rounding's random numbers
    int nx, ny, nz, N;
    long long Np;
    float gx0, gy0, gz0, tau0, delta, mach2;
    float wx, wy, wz;  // amplitude of the external force profile sin(2 pi y / ny)
    int wave;
    float in_cx, in_cy, in_ir2, in_umax;  // inlet profile
    uint32_t key0, key1;  // seed of the stochastic rounding
    int stochastic;
    long long wait_cycles;  // bound of the pipeline's mbarrier waits (clock64 cycles)
    int starve_batch;       // fault injection: this batch's copies are never issued (-1: none)
};

// Storage entry of the lattice node (x, y, z) (wrapped coordinates): the node
// itself in the dense layout; in the compact layout the offset of its row
// plus x - s_lo.  Only nodes inside a row's span are ever addressed: the
// fluid nodes, and the nodes a fluid node reaches through one link.
template <bool COMPACT>
__device__ __forceinline__ uint32_t entry_of(const LbArgs &a, int x, int y, int z)
{
    if (COMPACT) {
        const int4 rt = a.rows[y + a.ny * z];
        return (uint32_t)(rt.x + x - rt.y);
    }
    return (uint32_t)x + (uint32_t)a.nx * ((uint32_t)y + (uint32_t)a.ny * (uint32_t)z);
}

// Storage entry of the neighbour x + c_p of node (x, y, z): arithmetic in the
// dense layout; in the compact layout from the row base of (y + c_y, z + c_z)
// in rb (the node's nine neighbour-row bases), with x + c_x wrapped.
template <int P, bool COMPACT>
__device__ __forceinline__ uint32_t ghost_entry(const LbArgs &a, int x, int y, int z, const int *rb)
{
    const int xd = wrapm(x + cx(P), a.nx);
    if (COMPACT) return (uint32_t)(rb[(cy(P) + 1) + 3 * (cz(P) + 1)] + xd);
    return entry_of<false>(a, xd, wrapm(y + cy(P), a.ny), wrapm(z + cz(P), a.nz));
}

// ---------------------------------------------------------------------------
// Population storage.  FP32 keeps d_p itself.  The 16-bit formats keep
// s_p = d_p S / w_p: dividing by w_p gives every speed the same range
// (s_p / S = f_p / w_p - 1); binary16 takes S = 2^10, which keeps it out of
// its subnormal range down to |f_p / w_p - 1| = 2^-24 and allows up to 64;
// bfloat16 has FP32's exponent range and takes S = 1.
//
// Rounding to nearest is biased in a steady flow (a node and speed round the
// same way step after step and the errors add up to a spurious force), so
// by default the store rounds stochastically: up (away from zero) when the
// fraction of the gap covered plus (r + 1/2)/64 reaches 1, for six random
// bits r per value, saturating at the largest finite value.  The random
// bits of a node come from one Philox4x32-10 block (Salmon, Moraes, Dror,
// Shaw, SC 2011) with counter (node, pass low word, pass high word, 0) and
// the seed as key; speed p takes bits 6 (k mod 5) .. + 5 of word k / 5,
// k = rank of p when the speeds are ordered by (c_z, c_y, c_x).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int rnd_key(int p) { return 9 * (cz(p) + 1) + 3 * (cy(p) + 1) + (cx(p) + 1); }
__host__ __device__ constexpr int rnd_slot(int p)
{
    int r = 0;
    for (int q = 0; q < kQ; ++q) r += rnd_key(q) < rnd_key(p) ? 1 : 0;
    return r;
}
__host__ __device__ constexpr float iwq(int p) { return c2(p) == 0 ? 3.0f : (c2(p) == 1 ? 18.0f : 36.0f); }

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

template <int P>
__device__ __forceinline__ uint32_t rbits6(const uint4 &rb)
{
    constexpr int k = rnd_slot(P);
    const uint32_t w = k / 5 == 0 ? rb.x : (k / 5 == 1 ? rb.y : (k / 5 == 2 ? rb.z : rb.w));
    return (w >> (6 * (k % 5))) & 63u;
}

// binary16, stochastic: binary16 keeps 10 of FP32's 23 mantissa bits;
// adding 128 r + 64 to the 13 dropped bits carries into the kept ones
// exactly when the rounding goes up, and truncation (which saturates at
// 65504) finishes it.  Values below binary16's normal range (|x| < 2^-14,
// i.e. |f_p / w_p - 1| < 6e-8) are stored as zero.
__device__ __forceinline__ __half sr_half(float x, uint32_t r)
{
    const uint32_t u = __float_as_uint(x), mag = u & 0x7fffffffu;
    const __half h = __float2half_rz(__uint_as_float(u + (r << 7) + 64u));
    return mag >= 0x38800000u ? h : __ushort_as_half((unsigned short)0);
}

// bfloat16, stochastic: 16 dropped bits, 1024 r + 512 added, then the high
// half; finite inputs saturate at the largest finite value.
__device__ __forceinline__ __nv_bfloat16 sr_bf16(float x, uint32_t r)
{
    const uint32_t u = __float_as_uint(x), sign = u & 0x80000000u, mag = u & 0x7fffffffu;
    uint32_t y = mag + (r << 10) + 512u;
    if (mag < 0x7f800000u) y = min(y, 0x7f7fffffu);
    return __ushort_as_bfloat16((unsigned short)((sign | y) >> 16));
}

template <typename St>
struct Pop;
template <>
struct Pop<float> {
    static constexpr bool kRounds = false;
    template <int P>
    __device__ static __forceinline__ float get(float s) { return s; }
    template <int P>
    __device__ static __forceinline__ float put(float d, bool, const uint4 &) { return d; }
};
template <>
struct Pop<__half> {
    static constexpr bool kRounds = true;
    static constexpr float kS = 1024.0f;
    template <int P>
    __device__ static __forceinline__ float get(__half s) { return __half2float(s) * (wq(P) * (1.0f / kS)); }
    template <int P>
    __device__ static __forceinline__ __half put(float d, bool sr, const uint4 &rb)
    {
        const float x = d * (kS * iwq(P));
        return sr ? sr_half(x, rbits6<P>(rb)) : __float2half_rn(x);
    }
};
template <>
struct Pop<__nv_bfloat16> {
    static constexpr bool kRounds = true;
    template <int P>
    __device__ static __forceinline__ float get(__nv_bfloat16 s) { return __bfloat162float(s) * wq(P); }
    template <int P>
    __device__ static __forceinline__ __nv_bfloat16 put(float d, bool sr, const uint4 &rb)
    {
        const float x = d * iwq(P);
        return sr ? sr_bf16(x, rbits6<P>(rb)) : __float2bfloat16_rn(x);
    }
};

// compile-time loop over the speeds (the storage conversions take p as a
// template argument)
template <int P, int End, typename F>
__device__ __forceinline__ void for_speeds(F &&f)
{
    if constexpr (P < End) {
        f(std::integral_constant<int, P>{});
        for_speeds<P + 1, End>(f);
    }
}

// Collision (Sec. 2.1) of node n = (x, y, z), in deviations, from its 19
// pulled deviations d, the link mask lk, and the force density / smoothed
// hematocrit sums read at the node.  With drho = sum d, j = sum c d:
//   rho = 1 + drho, u = (j + G/2) / rho                       (Eqs. dens, vel)
//   f_eq - w = w [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2)]
//   Df = (1 - 1/2T) w [3 c.G + 4.5 (c.G)(c.u) - 1.5 G.u]       (Eq. chen_force,
//        force-density G, Guo's factor of the scheme Eq. vel comes from)
//   d* = d - (d - d_eq)/T + Df                                (Eq. lbe_discrete)
//   sigma = -(1 - 1/2T) sum c c (d - d_eq)                    (Eq. stresstensorLB)
// Stores d* (in the storage format, with streaming stores: a population is
// written once and read once per pass, and evicting it first keeps u, sigma,
// G and the shape lists in L2 for the per-cell kernel; `step` counts the
// stochastic rounding's random numbers), u, sigma, clears the node's G and
// theta, raises the
// stability flag, and at walls writes the reflected populations (halfway
// bounce-back): a population heading into a solid neighbour m comes back to
// this node in the opposite direction next pass, so it is stored in m's slot
// of that direction, from which this node pulls.  Each (slot, solid node)
// pair has exactly one writer; opposite speeds share a weight, so the stored
// value is written as it is, from the register that holds it, together with
// the node's own store of the pair.
// n is the node's storage entry; nd its lattice index (x + nx (y + ny z)),
// which keys the rounding's random numbers in either layout.  rb (compact
// layout only): the nine row bases of the node's row neighbourhood, entry of
// (x', y + dy, z + dz) = rb[(dy + 1) + 3 (dz + 1)] + x'.
template <typename St, bool WALLS, bool CELLS, bool SIGMA, bool COMPACT = false>
__device__ __forceinline__ void collide_node(const LbArgs &a, float (&d)[kQ], uint32_t lk, float gx, float gy,
                                             float gz, float T, uint32_t n, uint32_t nd, int x, int y, int z,
                                             unsigned long long step, const int *rb = nullptr)
{
    // element offsets fit 32 bits: the host keeps 19 Np below 2^32
    const uint32_t Np = (uint32_t)a.Np;
    St *dst = static_cast<St *>(a.dst);
    if (CELLS) a.G[n] = make_float4(0.f, 0.f, 0.f, 0.f);
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
    const float omc = 1.0f - om;
    const float ff = 1.0f - 0.5f * om;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float gu = gx * ux + gy * uy + gz * uz;
    const bool sr = Pop<St>::kRounds && a.stochastic != 0;
    uint4 rbits = make_uint4(0u, 0u, 0u, 0u);
    if (sr) rbits = philox4x32_10(make_uint4(nd, (uint32_t)step, (uint32_t)(step >> 32), 0u), a.key0, a.key1);
    // A speed p and its opposite q share |c.u|, |c.G| and the weight, so
    //   d_eq(p, q) = A +- B,  A = w [drho + rho (4.5 (c.u)^2 - 1.5 u^2)],
    //                         B = 3 w rho c.u,
    //   Df(p, q)   = C +- D,  C = (1 - 1/2T) w [4.5 (c.G)(c.u) - 1.5 G.u],
    //                         D = 3 (1 - 1/2T) w c.G,
    //   d*         = (1 - 1/T) d + d_eq / T + Df,
    // and the pair adds c c (d_p + d_q - 2A) to the stress.
    float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
    for_speeds<0, kQ>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        constexpr int q = opp(p);
        if constexpr (p == 0) {
            const float A = wq(0) * (drho - 1.5f * rho * usq);
            const float C = -1.5f * ff * wq(0) * gu;
            __stcs(&dst[n], Pop<St>::template put<0>(omc * d[0] + (om * A + C), sr, rbits));
        } else if constexpr (p < q) {
            const float cu = float(cx(p)) * ux + float(cy(p)) * uy + float(cz(p)) * uz;
            const float cg = float(cx(p)) * gx + float(cy(p)) * gy + float(cz(p)) * gz;
            const float w = wq(p);
            const float A = w * (drho + rho * (4.5f * cu * cu - 1.5f * usq));
            const float B = (3.0f * w) * rho * cu;
            const float fw = ff * w;
            const float C = fw * (4.5f * cg * cu - 1.5f * gu);
            const float D = 3.0f * fw * cg;
            const float P = om * A + C, M = om * B + D;
            const St vp = Pop<St>::template put<p>(omc * d[p] + (P + M), sr, rbits);
            const St vq = Pop<St>::template put<q>(omc * d[q] + (P - M), sr, rbits);
            __stcs(&dst[(uint32_t)p * Np + n], vp);
            __stcs(&dst[(uint32_t)q * Np + n], vq);
            if (WALLS) {
                // the solid neighbour x + c_p pulls nothing: its slot of q is
                // this node's next-pass population q (and likewise for q)
                if ((lk >> p) & 1u) dst[(uint32_t)q * Np + ghost_entry<p, COMPACT>(a, x, y, z, rb)] = vp;
                if ((lk >> q) & 1u) dst[(uint32_t)p * Np + ghost_entry<q, COMPACT>(a, x, y, z, rb)] = vq;
            }
            if (SIGMA) {
                const float ne = (d[p] + d[q]) - 2.0f * A;
                if (cx(p)) pxx += ne;
                if (cy(p)) pyy += ne;
                if (cz(p)) pzz += ne;
                if (cx(p) && cy(p)) pxy += cx(p) * cy(p) > 0 ? ne : -ne;
                if (cx(p) && cz(p)) pxz += cx(p) * cz(p) > 0 ? ne : -ne;
                if (cy(p) && cz(p)) pyz += cy(p) * cz(p) > 0 ? ne : -ne;
            }
        }
    });
    // the stress's six components ride in U.w (xz), S (xx yy zz xy) and Syz:
    // 36 bytes per node
    a.U[n] = make_float4(ux, uy, uz, SIGMA ? -ff * pxz : 0.f);
    if (SIGMA) {
        a.S[n] = make_float4(-ff * pxx, -ff * pyy, -ff * pzz, -ff * pxy);
        a.Syz[n] = -ff * pyz;
    }
    if (!(rho > 0.0f) || !(usq <= a.mach2)) atomicOr(&a.flags[FLAG_UNSTABLE], 1);
}

// Open-boundary node n = (x, y, z) (bit 29 of its link word: inlet, bit 30:
// outlet), not collided: its populations are set from the previous pass
// (the source buffer), as deviations from the weights,
//   inlet:  d_p = f_p^eq(rho_d, u_in) - w_p, rho_d the density of the
//           neighbour on z + 1 (bc_neighbour; 1 if none), u_in = u_max
//           (1 - r^2/R^2) z;
//   outlet: d_p = d_p(m) - w_p drho_m (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u^2),
//           m the neighbour on z - 1 with density 1 + drho_m and velocity
//           u, i.e. f^eq(1, u) plus the non-equilibrium part of m (d = 0,
//           f^eq(1, 0), if none);
// stored like any population (same rounding), with u their moments, sigma
// 0, and G, theta cleared.
// The neighbour a boundary node takes its state from, on the plane z + dz:
// straight across if fluid, else the first fluid one of the links
// (-1, 0, dz), (+1, 0, dz), (0, -1, dz), (0, +1, dz) (a tilted vessel meets
// the plane obliquely); -1 if none is.  lk holds the node's solid links.
// The result is the neighbour's storage entry.
template <bool COMPACT>
__device__ __forceinline__ long long bc_neighbour(const LbArgs &a, int x, int y, int z, int dz, uint32_t lk)
{
    const int off[5][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    for (int k = 0; k < 5; ++k) {
        int p = -1;
        for (int q = 1; q < kQ; ++q)
            if (cx(q) == off[k][0] && cy(q) == off[k][1] && cz(q) == dz) p = q;
        if (p < 0 || ((lk >> p) & 1u)) continue;
        return (long long)entry_of<COMPACT>(a, wrapm(x + off[k][0], a.nx), wrapm(y + off[k][1], a.ny),
                                            wrapm(z + dz, a.nz));
    }
    return -1;
}

template <typename St, bool CELLS, bool SIGMA, bool COMPACT = false>
__device__ __noinline__ void boundary_node(const LbArgs &a, uint32_t n, uint32_t nd, int x, int y, int z,
                                           uint32_t lk, unsigned long long step)
{
    const uint32_t Np = (uint32_t)a.Np;
    const St *src = static_cast<const St *>(a.src);
    St *dst = static_cast<St *>(a.dst);
    float d[kQ];
    if (lk & (1u << 29)) {
        const long long dl = bc_neighbour<COMPACT>(a, x, y, z, 1, lk);
        const uint32_t dn = (uint32_t)(dl < 0 ? 0 : dl);
        float drho = 0.f;
        if (dl >= 0)
            for_speeds<0, kQ>([&](auto pc) {
                constexpr int p = decltype(pc)::value;
                drho += Pop<St>::template get<p>(src[(uint32_t)p * Np + dn]);
            });
        const float rx = (float)x - a.in_cx, ry = (float)y - a.in_cy;
        const float r2 = (rx * rx + ry * ry) * a.in_ir2;
        const float uz = r2 < 1.0f ? a.in_umax * (1.0f - r2) : 0.0f;
        const float rho = 1.0f + drho;
        for_speeds<0, kQ>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            const float cu = float(cz(p)) * uz;
            d[p] = wq(p) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uz * uz));
        });
    } else {
        const long long ml = bc_neighbour<COMPACT>(a, x, y, z, -1, lk);
        const uint32_t m = (uint32_t)(ml < 0 ? 0 : ml);
        float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
        for_speeds<0, kQ>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            d[p] = ml < 0 ? 0.f : Pop<St>::template get<p>(src[(uint32_t)p * Np + m]);
            drho += d[p];
            jx += float(cx(p)) * d[p];
            jy += float(cy(p)) * d[p];
            jz += float(cz(p)) * d[p];
        });
        const float ir = 1.0f / (1.0f + drho);
        const float ux = jx * ir, uy = jy * ir, uz = jz * ir, usq = ux * ux + uy * uy + uz * uz;
        for_speeds<0, kQ>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            const float cu = float(cx(p)) * ux + float(cy(p)) * uy + float(cz(p)) * uz;
            d[p] -= wq(p) * drho * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * usq);
        });
    }
    const bool sr = Pop<St>::kRounds && a.stochastic != 0;
    uint4 rb = make_uint4(0u, 0u, 0u, 0u);
    if (sr) rb = philox4x32_10(make_uint4(nd, (uint32_t)step, (uint32_t)(step >> 32), 0u), a.key0, a.key1);
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
    for_speeds<0, kQ>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        dst[(uint32_t)p * Np + n] = Pop<St>::template put<p>(d[p], sr, rb);
        drho += d[p];
        jx += float(cx(p)) * d[p];
        jy += float(cy(p)) * d[p];
        jz += float(cz(p)) * d[p];
    });
    const float ir = 1.0f / (1.0f + drho);
    a.U[n] = make_float4(jx * ir, jy * ir, jz * ir, 0.f);
    if (SIGMA) {
        a.S[n] = make_float4(0.f, 0.f, 0.f, 0.f);
        a.Syz[n] = 0.f;
    }
    if (CELLS) a.G[n] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// External force density at row y: the uniform drive plus the Kolmogorov
// profile A sin(2 pi y / ny).
__device__ __forceinline__ void external_force(const LbArgs &a, int y, float &gx, float &gy, float &gz)
{
    gx = a.gx0;
    gy = a.gy0;
    gz = a.gz0;
    if (a.wave) {
        const float sw = sinpif(2.0f * (float)y / (float)a.ny);
        gx += a.wx * sw;
        gy += a.wy * sw;
        gz += a.wz * sw;
    }
}

template <typename St, bool WALLS, bool CELLS, bool SIGMA>
__device__ __forceinline__ void lb_node(const LbArgs &a, int n, unsigned long long step)
{
    const St *src = static_cast<const St *>(a.src);
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
    for_speeds<0, kQ>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        constexpr int ix = cx(p) == 0 ? 0 : (cx(p) > 0 ? 1 : 2);
        constexpr int iy = cy(p) == 0 ? 0 : (cy(p) > 0 ? 1 : 2);
        constexpr int iz = cz(p) == 0 ? 0 : (cz(p) > 0 ? 1 : 2);
        d[p] = Pop<St>::template get<p>(src[(uint32_t)p * (uint32_t)a.Np + (uint32_t)(xs[ix] + ys[iy] + zs[iz])]);
    });
    float gx, gy, gz, T = a.tau0;
    external_force(a, y, gx, gy, gz);
    if (CELLS) {
        const float4 g4 = a.G[n];
        gx += g4.x;
        gy += g4.y;
        gz += g4.z;
        T += a.delta * g4.w;
    }
    if (WALLS && (lk >> 31)) return;  // solid node: nothing to collide
    if (WALLS && (lk & 0x60000000u)) {
        boundary_node<St, CELLS, SIGMA>(a, (uint32_t)n, (uint32_t)n, x, y, z, lk, step);
        return;
    }
    collide_node<St, WALLS, CELLS, SIGMA>(a, d, lk, gx, gy, gz, T, (uint32_t)n, (uint32_t)n, x, y, z, step);
}

template <typename St, bool WALLS, bool CELLS, bool SIGMA>
__global__ void __launch_bounds__(kLbThreads) k_lb(LbArgs a)
{
    __shared__ unsigned long long s_step;
    if (threadIdx.x == 0) s_step = *a.step;
    __syncthreads();
    const unsigned long long step = s_step;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < a.N) lb_node<St, WALLS, CELLS, SIGMA>(a, n, step);
    // the last block out advances the pass counter
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.work[1], 1) == (int)gridDim.x - 1) {
            a.work[1] = 0;
            *a.step = step + 1;
            __threadfence();
        }
    }
}

// Node-list pass: one thread per fluid node of a sorted list (sparse vessel
// geometries, where whole rows would be mostly solid); the pull, collision
// and stores are those of the one-thread-per-node pass.
template <typename St, bool WALLS, bool CELLS, bool SIGMA>
__global__ void __launch_bounds__(kLbThreads) k_lb_list(LbArgs a, const uint32_t *__restrict__ list, int nf)
{
    __shared__ unsigned long long s_step;
    if (threadIdx.x == 0) s_step = *a.step;
    __syncthreads();
    const unsigned long long step = s_step;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf) lb_node<St, WALLS, CELLS, SIGMA>(a, (int)list[t], step);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.work[1], 1) == (int)gridDim.x - 1) {
            a.work[1] = 0;
            *a.step = step + 1;
            __threadfence();
        }
    }
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

// L2 policy for data touched once per pass: evicted first
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// bulk_g2s with an L2 cache policy
__device__ __forceinline__ void bulk_g2s_hint(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar,
                                              uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}

// Wait for phase `parity` of the mbarrier, for at most `limit` cycles; false
// on timeout (the caller raises the timeout flag).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitCycles)
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
        if (clock64() - t0 > limit) return false;
    }
}

struct StageLayout {
    int B;           // rows per batch
    int planes;      // staged planes per row: 19 populations (+4 G, theta) (+1 links)
    int pop_bytes;   // bytes of the 19 population planes of a stage
    int stage_bytes;
    int stages;      // buffers in the ring (2 .. kMaxStages)
};

// Producer side of one batch (rows y0 .. y0 + nb - 1 at one z of the
// lattice `a`): the warp issues the bulk copies of the staged planes into
// `base` (population plane k, batch row b at (k * B + b) * nx elements; the
// 4-byte planes after the 19 population planes), completing on `bar`.
template <typename St, bool CELLS>
__device__ __forceinline__ void produce_batch(const LbArgs &a, const StageLayout &L, int batch, unsigned char *base,
                                              uint32_t bar, int lane)
{
    const int nx = a.nx, ny = a.ny, nz = a.nz, B = L.B;
    const int nyb = (ny + B - 1) / B;
    const int z = batch / nyb, y0 = (batch - z * nyb) * B;
    const int nb = min(B, ny - y0);
    const St *src = static_cast<const St *>(a.src);
    const uint32_t prow_bytes = (uint32_t)nx * (uint32_t)sizeof(St), frow_bytes = (uint32_t)nx * 4u;
    if (lane == 0)
        mbar_expect_tx(bar, (uint32_t)(kQ * nb) * prow_bytes + (uint32_t)((L.planes - kQ) * nb) * frow_bytes);
    __syncwarp();
    St *pst = reinterpret_cast<St *>(base);
    float *fst = reinterpret_cast<float *>(base + L.pop_bytes);
    const uint64_t once = l2_evict_first();
    for (int k = lane; k < L.planes; k += 32) {
        if (k < kQ) {
            // the upstream rows y - c_y are contiguous in plane k except
            // where they wrap in y: one copy, or two
            St *dst = pst + (size_t)k * B * nx;
            const int zs = wrapm(z - cz(k), nz);
            const St *plane = src + (long long)k * a.Np + (long long)zs * ny * nx;
            const int ys = y0 - cy(k);  // first upstream row, may be -1 or run past ny
            int b = 0;
            while (b < nb) {
                const int yr = wrapm(ys + b, ny);
                const int run = min(nb - b, ny - yr);
                bulk_g2s_hint(smem_addr(dst + (size_t)b * nx), plane + (long long)yr * nx,
                              (uint32_t)run * prow_bytes, bar, once);
                b += run;
            }
        } else if (CELLS && k == kQ) {
            // G and the hematocrit sum: one float4 per node, B rows of nx
            const long long off = ((long long)z * ny + y0) * nx;
            bulk_g2s(smem_addr(fst), a.G + off, (uint32_t)nb * 4u * frow_bytes, bar);
        } else if (!(CELLS && k < kQ + 4)) {
            // the link words after the cell planes
            float *dst = fst + (size_t)(k - kQ) * B * nx;
            const long long off = ((long long)z * ny + y0) * nx;
            bulk_g2s(smem_addr(dst), reinterpret_cast<const float *>(a.links) + off, (uint32_t)nb * frow_bytes, bar);
        }
    }
}

// Consumer side of one batch: the 256 consumer threads take batch nodes
// l = t, t + 256, ... as (row b, column x) = (l / nx, l % nx), advanced
// without a division, and collide them from the staged rows.
template <typename St, bool WALLS, bool CELLS, bool SIGMA>
__device__ __forceinline__ void consume_batch(const LbArgs &a, const StageLayout &L, int batch,
                                              const unsigned char *base, unsigned long long step, int x_first,
                                              int b_first, int x_step, int b_step)
{
    const int nx = a.nx, ny = a.ny, B = L.B;
    const int nyb = (ny + B - 1) / B;
    const int z = batch / nyb, y0 = (batch - z * nyb) * B;
    const int nb = min(B, ny - y0);
    const int plane_stride = B * nx;
    const St *pst = reinterpret_cast<const St *>(base);
    const float *fst = reinterpret_cast<const float *>(base + L.pop_bytes);
    for (int b = b_first, x = x_first; b < nb;) {
        const int y = y0 + b;
        const uint32_t n = (uint32_t)((y + ny * z) * nx + x);
        const int bx = b, xx = x;
        x += x_step;
        b += b_step;
        if (x >= nx) {
            x -= nx;
            ++b;
        }
        const St *prow = pst + (size_t)bx * nx;
        const float *frow = fst + (size_t)bx * nx;
        const uint32_t lk =
            WALLS ? reinterpret_cast<const uint32_t *>(frow)[(size_t)(CELLS ? 4 : 0) * plane_stride + xx] : 0u;
        if (WALLS && (lk >> 31)) continue;
        if (WALLS && (lk & 0x60000000u)) {
            boundary_node<St, CELLS, SIGMA>(a, n, n, xx, y, z, lk, step);
            continue;
        }
        const int xm = xx == 0 ? nx - 1 : xx - 1, xp = xx == nx - 1 ? 0 : xx + 1;
        float d[kQ];
        for_speeds<0, kQ>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            const int xs = cx(p) == 0 ? xx : (cx(p) > 0 ? xm : xp);
            d[p] = Pop<St>::template get<p>(prow[p * plane_stride + xs]);
        });
        float gx, gy, gz, T = a.tau0;
        external_force(a, y, gx, gy, gz);
        if (CELLS) {
            const float4 g4 = reinterpret_cast<const float4 *>(fst)[(size_t)bx * nx + xx];
            gx += g4.x;
            gy += g4.y;
            gz += g4.z;
            T += a.delta * g4.w;
        }
        collide_node<St, WALLS, CELLS, SIGMA>(a, d, lk, gx, gy, gz, T, n, n, xx, y, z, step);
    }
}

template <typename St, bool WALLS, bool CELLS, bool SIGMA>
__global__ void __launch_bounds__(kStThreads) k_lb_staged(LbArgs a, StageLayout L, int nbatches)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long full[kMaxStages], empty[kMaxStages];
    __shared__ int s_batch[kMaxStages];
    __shared__ unsigned long long s_step;
    const int ns = L.stages;
    if (threadIdx.x == 0) {
        for (int k = 0; k < ns; ++k) {
            mbar_init(smem_addr(&full[k]), 1);
            mbar_init(smem_addr(&empty[k]), kStConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_step = *a.step;
    }
    __syncthreads();

    if (threadIdx.x >= kStConsumers) {
        // Producer warp.  Batches are claimed from a global counter, so a CTA
        // that starts late (the SM was busy with another kernel) just does
        // fewer of them.  The batch id goes to s_batch[stage] before the
        // arrive that the consumers' wait acquires; -1 tells them to stop.
        const int lane = threadIdx.x - kStConsumers;
        int it = 0;
        bool ok = true;
        unsigned issued = 0;  // stages whose last fill has copies issued
        for (;; ++it) {
            const int stage = it % ns;
            if (it >= ns && !mbar_wait(smem_addr(&empty[stage]), (uint32_t)((it / ns - 1) & 1), a.wait_cycles)) {
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
            if (lane == 0) s_batch[stage] = batch;
            if (batch == a.starve_batch) {  // fault injection: the stage never fills
                issued &= ~(1u << stage);
                continue;
            }
            issued |= 1u << stage;
            produce_batch<St, CELLS>(a, L, batch, smraw + (size_t)stage * L.stage_bytes, bar, lane);
        }
        if (!ok) {
            // let the copies still in flight land before the CTA's memory
            // goes away (with the full bound, whatever the pipeline's)
            for (int j = it > ns ? it - ns : 0; j < it; ++j)
                if ((issued >> (j % ns)) & 1u) mbar_wait(smem_addr(&full[j % ns]), (uint32_t)((j / ns) & 1));
        }
        // the last CTA out resets the counters for the next launch and
        // advances the pass counter (every CTA read it before its barrier)
        if (lane == 0) {
            __threadfence();
            if (atomicAdd(&a.work[1], 1) == (int)gridDim.x - 1) {
                a.work[0] = 0;
                a.work[1] = 0;
                *a.step = s_step + 1;
                __threadfence();
            }
        }
        return;
    }

    // consumer warps
    const int lane = threadIdx.x & 31;
    const unsigned long long step = s_step;
    const int nx = a.nx;
    const int x_first = threadIdx.x % nx, b_first = threadIdx.x / nx;
    const int x_step = kStConsumers % nx, b_step = kStConsumers / nx;
    for (int it = 0;; ++it) {
        const int stage = it % ns;
        if (!mbar_wait(smem_addr(&full[stage]), (uint32_t)((it / ns) & 1), a.wait_cycles)) {
            if (lane == 0) atomicOr(&a.flags[FLAG_TIMEOUT], 1);
            break;
        }
        const int batch = s_batch[stage];
        if (batch < 0) break;
        consume_batch<St, WALLS, CELLS, SIGMA>(a, L, batch, smraw + (size_t)stage * L.stage_bytes, step, x_first,
                                               b_first, x_step, b_step);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[stage]));  // this warp is done with the stage
    }
}

// ---------------------------------------------------------------------------
// Compact lattice pass (walled lattices in the compact layout).  The same
// persistent producer / consumer pipeline as the row-staged pass, over a
// table of batches built at set-up.  A batch is up to kMaxSegs row segments
// in lattice order: a segment is the fluid x-range [c0, c1] of one row (or
// of one run of a branched row, or a piece of a row) with its staged window
// [X0, X0 + W) = [c0 - 1, c1 + 1] rounded out to whole 32-byte sectors (the
// whole row when the row wraps along x); the windows of a batch fill one
// stage, the segment that overflows it being cut.  Rows without fluid are
// never visited: their entries are only the targets of the bounce-back
// writes of their fluid neighbours.  For every speed p the producer copies,
// per segment, the part of the upstream row (y - c_y, z - c_z) that lies in
// both the window and that row's span (one bulk copy each; span and window
// ends are whole sectors, so every copy starts and ends on a 16-byte
// boundary), plus the segment's own G / theta and link words.  Stage layout:
// [19][E] populations, [E] float4 G, [E] link words, E the batch's window
// entries; segment s's window column x sits at off_s + x - X0_s.  The
// consumer threads run over the E entries and collide the fluid nodes among
// them; a node pulls only from upstream entries inside the upstream row's
// span (every node one link away from a fluid node is stored), so the parts
// of a window outside a span are never read.
// ---------------------------------------------------------------------------
// Producer side of one compact batch.  The set-up precomputed, for every
// segment s and each of its nine upstream rows u = (dy + 1) + 3 (dz + 1)
// (the row (y + dy, z + dz) that the speeds with c_y = -dy, c_z = -dz pull
// from), the part of that row's span inside the window: its first entry and
// (window offset | entry count << 16); and per batch the bytes of all its
// copies.  The lanes take the batch's copies one each (speed plane k of
// segment s reads descriptor u(k) of that segment; G / theta and the link
// words read u = 4), so a segment's 20 or 21 copies go out in one pass of
// the warp.
// Upstream row of speed p among the nine (dy, dz) rows of a compact batch
// row, u = (dy + 1) + 3 (dz + 1) with (dy, dz) = (-c_y, -c_z), for a
// run-time p: four bits per speed in two 64-bit constants.
__host__ __device__ constexpr uint64_t upstream_bits(int first, int count)
{
    uint64_t v = 0;
    for (int p = first; p < first + count && p < kQ; ++p)
        v |= (uint64_t)((1 - cy(p)) + 3 * (1 - cz(p))) << (4 * (p - first));
    return v;
}
__device__ __forceinline__ int upstream_row(int p)
{
    constexpr uint64_t lo = upstream_bits(0, 16), hi = upstream_bits(16, 16);
    return (int)((p < 16 ? lo >> (4 * p) : hi >> (4 * (p - 16))) & 0xFu);
}

__device__ __forceinline__ void cp_async_4(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The producer's own copy of one batch's descriptors (pd[j], j < kSegDescs
// nb): asynchronous copies, so that they are in flight while the producer
// waits for a free stage and hold no registers meanwhile.  The caller waits
// for them (cp_async_wait_all, then __syncwarp: every lane reads entries
// that other lanes copied).
__device__ __forceinline__ void load_descs(const LbArgs &a, int4 bd, int lane, int2 *pd)
{
    const int nd = kSegDescs * (bd.y & 0xFF);
    for (int j = lane; j < nd; j += 32) cp_async_8(smem_addr(&pd[j]), a.pool + bd.x + j);
    cp_async_commit();
}

// Per segment s of a stage, rbs[s][..]: [0..8] base of upstream row u
// (entry of x' in that row = base + x'), [9] y, [10] z, [11] c0, [12] c1,
// [13] X0, [14] off_s, [15] off_s + W_s; written before the stage's arrive,
// read by the consumers.
constexpr int kSegWords = 16;
template <typename St, bool CELLS>
__device__ __forceinline__ void produce_compact(const LbArgs &a, int4 bd, const int2 *pd, unsigned char *base,
                                                uint32_t bar, int lane, int (*rbs)[kSegWords])
{
    const int nb = bd.y & 0xFF;
    const int total = (int)((uint32_t)bd.y >> 8);
    for (int j = lane; j < kSegDescs * nb; j += 32) {
        const int2 e = pd[j];
        const int b = j / kSegDescs, u = j - kSegDescs * b;
        int *rb = rbs[b];
        if (u < 9) {
            const int count = (int)((uint32_t)e.y >> 16), at = e.y & 0xFFFF;
            rb[u] = count > 0 ? e.x - at - (pd[kSegDescs * b + 10].y & 0xFFFF) : 0;
        } else if (u == 9) {
            rb[9] = e.x;
            rb[10] = e.y;
        } else if (u == 10) {
            rb[11] = e.x & 0xFFFF;
            rb[12] = (int)((uint32_t)e.x >> 16);
            rb[13] = e.y & 0xFFFF;
        } else {
            rb[14] = e.x;
            rb[15] = e.x + (int)((uint32_t)pd[kSegDescs * b + 10].y >> 16);
        }
    }
    __syncwarp();
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)bd.z);
    __syncwarp();
    // one copy per lane: copy k of segment s is speed plane k (k < 19),
    // whose upstream row is u = (1 - c_y) + 3 (1 - c_z), then G / theta
    // and the link words of the row itself (u = 4)
    constexpr int kCopies = kQ + (CELLS ? 2 : 1);
    const uint64_t once = l2_evict_first();
    const size_t pop_bytes = (size_t)kQ * total * sizeof(St);
    for (int j = lane; j < kCopies * nb; j += 32) {
        const int b = j / kCopies, k = j - b * kCopies;
        const int u = k < kQ ? upstream_row(k) : 4;
        const int2 e = pd[kSegDescs * b + u];
        const int count = (int)((uint32_t)e.y >> 16);
        if (count == 0) continue;
        const int at = pd[kSegDescs * b + 11].x + (e.y & 0xFFFF);  // stage column of the first entry
        if (k < kQ) {
            const St *g = static_cast<const St *>(a.src) + (size_t)k * (size_t)a.Np + (size_t)e.x;
            bulk_g2s_hint(smem_addr(base + ((size_t)k * total + at) * sizeof(St)), g,
                          (uint32_t)(count * (int)sizeof(St)), bar, once);
        } else if (CELLS && k == kQ) {
            bulk_g2s(smem_addr(base + pop_bytes + (size_t)at * sizeof(float4)), a.G + e.x,
                     (uint32_t)(count * (int)sizeof(float4)), bar);
        } else {
            bulk_g2s(smem_addr(base + pop_bytes + (CELLS ? (size_t)total * sizeof(float4) : 0) +
                               (size_t)at * sizeof(uint32_t)),
                     a.links + e.x, (uint32_t)(count * (int)sizeof(uint32_t)), bar);
        }
    }
}

template <typename St, bool CELLS, bool SIGMA>
__device__ __forceinline__ void consume_compact(const LbArgs &a, int4 bd, const unsigned char *base,
                                                unsigned long long step, const int (*rbs)[kSegWords])
{
    const int nx = a.nx, ny = a.ny;
    // threads run over the batch's window entries, whose segments start on
    // whole sectors, so that a warp's stores cover whole 32-byte sectors of
    // each plane
    const int total = (int)((uint32_t)bd.y >> 8);
    const size_t pop_bytes = (size_t)kQ * total * sizeof(St);
    const St *pst = reinterpret_cast<const St *>(base);
    const float4 *gst = reinterpret_cast<const float4 *>(base + pop_bytes);
    const uint32_t *lst =
        reinterpret_cast<const uint32_t *>(base + pop_bytes + (CELLS ? (size_t)total * sizeof(float4) : 0));
    int s = 0;
    for (int l = (int)threadIdx.x; l < total; l += kStConsumers) {
        while (l >= rbs[s][15]) ++s;  // the last segment ends at total
        const int *rb = rbs[s];
        const int x = rb[13] + l - rb[14];
        if (x < rb[11] || x > rb[12]) continue;
        const uint32_t lk = lst[l];
        if (lk >> 31) continue;
        const int y = rb[9], z = rb[10];
        const uint32_t n = (uint32_t)(rb[4] + x);
        const uint32_t nd = (uint32_t)x + (uint32_t)nx * ((uint32_t)y + (uint32_t)ny * (uint32_t)z);
        if (lk & 0x60000000u) {
            boundary_node<St, CELLS, SIGMA, true>(a, n, nd, x, y, z, lk, step);
            continue;
        }
        // window column of x - 1 / x + 1 relative to x (the neighbour across
        // a periodic x boundary lies in the same whole-row window)
        const int om = x == 0 ? nx - 1 : -1, op = x == nx - 1 ? 1 - nx : 1;
        float d[kQ];
        for_speeds<0, kQ>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            const int o = cx(p) == 0 ? 0 : (cx(p) > 0 ? om : op);
            d[p] = Pop<St>::template get<p>(pst[p * total + l + o]);
        });
        float gx, gy, gz, T = a.tau0;
        external_force(a, y, gx, gy, gz);
        if (CELLS) {
            const float4 g4 = gst[l];
            gx += g4.x;
            gy += g4.y;
            gz += g4.z;
            T += a.delta * g4.w;
        }
        collide_node<St, true, CELLS, SIGMA, true>(a, d, lk, gx, gy, gz, T, n, nd, x, y, z, step, rb);
    }
}

// Registers bounded so that the side kernels of the step find room beside
// the pass on every SM: 72 per thread for FP32 populations (the row-staged
// pass's count), 96 for the 16-bit ones (their decode and stochastic
// rounding need more)
template <typename St>
constexpr int compact_min_blocks() { return sizeof(St) == 4 ? 3 : 2; }

template <typename St, bool CELLS, bool SIGMA>
__global__ void __launch_bounds__(kStThreads, compact_min_blocks<St>())
    k_lb_compact(LbArgs a, const int4 *__restrict__ batches, int nbatches, int ns, int stage_bytes)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long full[kMaxStages], empty[kMaxStages];
    __shared__ int4 s_desc[kMaxStages];
    __shared__ int s_rb[kMaxStages][kMaxSegs][kSegWords];
    __shared__ __align__(8) int2 s_pd[kSegDescs * kMaxSegs];
    __shared__ unsigned long long s_step;
    if (threadIdx.x == 0) {
        for (int k = 0; k < ns; ++k) {
            mbar_init(smem_addr(&full[k]), 1);
            mbar_init(smem_addr(&empty[k]), kStConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_step = *a.step;
    }
    __syncthreads();

    if (threadIdx.x >= kStConsumers) {
        // producer warp: claims batches from the global counter (see
        // k_lb_staged) two ahead.  While the stage for batch i is still in
        // use it starts the copy of batch i's descriptors (its record came
        // in the round before), loads batch i + 1's record (claimed the
        // round before) and claims batch i + 2, so that all of it is in
        // flight during the wait and the bulk copies start as soon as the
        // stage is free; s_desc[stage].x = -1 tells the consumers to stop.
        const int lane = threadIdx.x - kStConsumers;
        int it = 0;
        bool ok = true;
        unsigned issued = 0;  // stages whose last fill has copies issued
        int claim = 0;
        if (lane == 0) claim = atomicAdd(&a.work[0], 1);
        int batch = __shfl_sync(0xffffffffu, claim, 0);
        int4 bd = make_int4(-1, 0, 0, 0);
        if (batch < nbatches) {
            bd = batches[batch];
            if (lane == 0) claim = atomicAdd(&a.work[0], 1);
        }
        for (;; ++it) {
            const int stage = it % ns;
            if (batch < nbatches) load_descs(a, bd, lane, s_pd);
            const int nbatch = __shfl_sync(0xffffffffu, claim, 0);
            int4 nbd = make_int4(-1, 0, 0, 0);
            if (batch < nbatches && nbatch < nbatches) {
                nbd = batches[nbatch];
                if (lane == 0) claim = atomicAdd(&a.work[0], 1);
            }
            const bool freed =
                it < ns || mbar_wait(smem_addr(&empty[stage]), (uint32_t)((it / ns - 1) & 1), a.wait_cycles);
            cp_async_wait_all();
            __syncwarp();
            if (!freed) {
                if (lane == 0) atomicOr(&a.flags[FLAG_TIMEOUT], 1);
                ok = false;
                break;
            }
            const uint32_t bar = smem_addr(&full[stage]);
            if (batch >= nbatches) {
                if (lane == 0) {
                    s_desc[stage] = make_int4(-1, 0, 0, 0);
                    mbar_arrive(bar);
                }
                break;
            }
            if (lane == 0) s_desc[stage] = bd;
            if (batch == a.starve_batch) {  // fault injection: the stage never fills
                issued &= ~(1u << stage);
            } else {
                issued |= 1u << stage;
                produce_compact<St, CELLS>(a, bd, s_pd, smraw + (size_t)stage * stage_bytes, bar, lane,
                                           s_rb[stage]);
            }
            __syncwarp();  // every lane has read s_pd before the next copy into it
            batch = nbatch < nbatches ? nbatch : nbatches;
            bd = nbd;
        }
        if (!ok) {
            // let the copies still in flight land before the CTA's memory
            // goes away (with the full bound, whatever the pipeline's)
            for (int j = it > ns ? it - ns : 0; j < it; ++j)
                if ((issued >> (j % ns)) & 1u) mbar_wait(smem_addr(&full[j % ns]), (uint32_t)((j / ns) & 1));
        }
        if (lane == 0) {
            __threadfence();
            if (atomicAdd(&a.work[1], 1) == (int)gridDim.x - 1) {
                a.work[0] = 0;
                a.work[1] = 0;
                *a.step = s_step + 1;
                __threadfence();
            }
        }
        return;
    }

    const int lane = threadIdx.x & 31;
    const unsigned long long step = s_step;
    for (int it = 0;; ++it) {
        const int stage = it % ns;
        if (!mbar_wait(smem_addr(&full[stage]), (uint32_t)((it / ns) & 1), a.wait_cycles)) {
            if (lane == 0) atomicOr(&a.flags[FLAG_TIMEOUT], 1);
            break;
        }
        const int4 bd = s_desc[stage];
        if (bd.x < 0) break;
        consume_compact<St, CELLS, SIGMA>(a, bd, smraw + (size_t)stage * stage_bytes, step, s_rb[stage]);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[stage]));
    }
}

// ---------------------------------------------------------------------------
// Packed lattice pass: one persistent launch over the lattices of several
// solves of one class (storage type, walls, cells, stress).  The solves'
// batches are numbered consecutively (bstart[i] = first batch of solve i);
// a producer that claims batch g finds its solve by binary search, copies
// the solve's arguments, layout and pass count into the stage's slot of
// shared memory and stages the rows as above; the consumers collide from
// that slot.  Stages are `stage_bytes` (the largest layout of the pack).
// The last CTA out resets the counters and advances every solve's pass
// counter.  `parity` swaps source and destination populations.
// ---------------------------------------------------------------------------
struct LbPackEntry {
    LbArgs a;  // populations of parity 0: src = pops[0], dst = pops[1]
    StageLayout L;
};

__device__ __forceinline__ int pack_find(const int *start, int n, int g)
{
    int lo = 0, hi = n - 1;  // largest i with start[i] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename St, bool WALLS, bool CELLS, bool SIGMA>
__global__ void __launch_bounds__(kStThreads)
    k_lb_staged_packed(const LbPackEntry *__restrict__ tab, const int *__restrict__ bstart, int ninst, int total,
                       int parity, int *work, int ns, int stage_bytes)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) unsigned long long full[kMaxStages], empty[kMaxStages];
    __shared__ int s_batch[kMaxStages];
    __shared__ LbPackEntry s_ent[kMaxStages];
    __shared__ unsigned long long s_step[kMaxStages];
    if (threadIdx.x == 0) {
        for (int k = 0; k < ns; ++k) {
            mbar_init(smem_addr(&full[k]), 1);
            mbar_init(smem_addr(&empty[k]), kStConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (threadIdx.x >= kStConsumers) {
        const int lane = threadIdx.x - kStConsumers;
        int it = 0;
        bool ok = true;
        for (;; ++it) {
            const int stage = it % ns;
            if (it >= ns && !mbar_wait(smem_addr(&empty[stage]), (uint32_t)((it / ns - 1) & 1))) {
                if (lane == 0) atomicOr(&tab[0].a.flags[FLAG_TIMEOUT], 1);
                ok = false;
                break;
            }
            int g = 0;
            if (lane == 0) g = atomicAdd(&work[0], 1);
            g = __shfl_sync(0xffffffffu, g, 0);
            const uint32_t bar = smem_addr(&full[stage]);
            if (g >= total) {
                if (lane == 0) {
                    s_batch[stage] = -1;
                    mbar_arrive(bar);
                }
                break;
            }
            const int inst = pack_find(bstart, ninst, g);
            // copy the solve's entry into the stage's slot (the stage is free)
            const int *srcw = reinterpret_cast<const int *>(&tab[inst]);
            int *dstw = reinterpret_cast<int *>(&s_ent[stage]);
            for (int w = lane; w < (int)(sizeof(LbPackEntry) / sizeof(int)); w += 32) dstw[w] = srcw[w];
            if (lane == 0) {
                s_batch[stage] = g - bstart[inst];
                s_step[stage] = *tab[inst].a.step;
            }
            __syncwarp();
            if (lane == 0 && parity) {
                const void *t = s_ent[stage].a.src;
                s_ent[stage].a.src = s_ent[stage].a.dst;
                s_ent[stage].a.dst = const_cast<void *>(t);
            }
            __syncwarp();
            produce_batch<St, CELLS>(s_ent[stage].a, s_ent[stage].L, s_batch[stage],
                                     smraw + (size_t)stage * stage_bytes, bar, lane);
        }
        if (!ok) {
            for (int j = it > ns ? it - ns : 0; j < it; ++j)
                mbar_wait(smem_addr(&full[j % ns]), (uint32_t)((j / ns) & 1));
        }
        if (lane == 0) {
            __threadfence();
            if (atomicAdd(&work[1], 1) == (int)gridDim.x - 1) {
                work[0] = 0;
                work[1] = 0;
                for (int k = 0; k < ninst; ++k) *tab[k].a.step += 1;
                __threadfence();
            }
        }
        return;
    }

    const int lane = threadIdx.x & 31;
    for (int it = 0;; ++it) {
        const int stage = it % ns;
        if (!mbar_wait(smem_addr(&full[stage]), (uint32_t)((it / ns) & 1))) {
            if (lane == 0) atomicOr(&tab[0].a.flags[FLAG_TIMEOUT], 1);
            break;
        }
        const int batch = s_batch[stage];
        if (batch < 0) break;
        const LbArgs &a = s_ent[stage].a;
        const int nx = a.nx;
        consume_batch<St, WALLS, CELLS, SIGMA>(a, s_ent[stage].L, batch, smraw + (size_t)stage * stage_bytes,
                                               s_step[stage], threadIdx.x % nx, threadIdx.x / nx, kStConsumers % nx,
                                               kStConsumers / nx);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty[stage]));
    }
}

// One entry per thread; non-fluid entries (solid byte, or link bit 31 in the
// compact layout) report 0.
template <typename St>
__global__ void k_rho(const void *__restrict__ pops_v, const uint8_t *__restrict__ solid,
                      const uint32_t *__restrict__ links, float *__restrict__ rho, int N, long long Np)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    if ((solid && solid[n]) || (links && (links[n] >> 31))) {
        rho[n] = 0.f;
        return;
    }
    const St *pops = static_cast<const St *>(pops_v);
    float s = 0.f;
    for_speeds<0, kQ>([&](auto pc) {
        constexpr int p = decltype(pc)::value;
        s += Pop<St>::template get<p>(pops[(long long)p * Np + n]);
    });
    rho[n] = s;  // rho - 1: the host adds 1 in FP64
}

// Budgets (Sec. 2.2 conservation claims): per block FP64 partial sums of the
// zeroth and first moments of the stored populations over fluid nodes, the
// max |u|^2 of the last pass and a NaN count; a single block then sums the
// partials in a fixed order and adds the cell momenta sum M V.
constexpr int kBudThreads = 256;

struct ForceArgs {
    float g[3], w[3];
    int nx, ny;
};

template <typename St>
__global__ void __launch_bounds__(kBudThreads)
k_budget_nodes(const void *__restrict__ pops_v, const float4 *__restrict__ U,
               const uint8_t *__restrict__ solid, double *__restrict__ part, int N, long long Np, ForceArgs fa)
{
    const St *pops = static_cast<const St *>(pops_v);
    double m = 0.0, px = 0.0, py = 0.0, pz = 0.0, umax = 0.0, nan = 0.0, work = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        if (solid && solid[n]) continue;
        float s = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
        for_speeds<0, kQ>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            const float v = Pop<St>::template get<p>(pops[(long long)p * Np + n]);
            s += v;
            if (cx(p)) jx += cx(p) > 0 ? v : -v;
            if (cy(p)) jy += cy(p) > 0 ? v : -v;
            if (cz(p)) jz += cz(p) > 0 ? v : -v;
        });
        m += 1.0 + (double)s;
        px += jx;
        py += jy;
        pz += jz;
        const float4 u4 = U[n];
        const float ux = u4.x, uy = u4.y, uz = u4.z;
        const float u2 = ux * ux + uy * uy + uz * uz;
        if (!(u2 == u2) || !(s == s)) nan += 1.0;
        else if (u2 > umax) umax = u2;
        // work rate of the external force (uniform + sin(2 pi y / ny) profile)
        const double sw = sinpi(2.0 * (double)((n / fa.nx) % fa.ny) / (double)fa.ny);
        work += ((double)fa.g[0] + (double)fa.w[0] * sw) * ux + ((double)fa.g[1] + (double)fa.w[1] * sw) * uy +
                ((double)fa.g[2] + (double)fa.w[2] * sw) * uz;
    }
    __shared__ double sh[7][kBudThreads];
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = px;
    sh[2][threadIdx.x] = py;
    sh[3][threadIdx.x] = pz;
    sh[4][threadIdx.x] = umax;
    sh[5][threadIdx.x] = nan;
    sh[6][threadIdx.x] = work;
    __syncthreads();
    for (int w = kBudThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int k = 0; k < 7; ++k) {
                if (k == 4)
                    sh[k][threadIdx.x] = fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
                else
                    sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) part[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// The same partial sums in the compact layout, one thread per stored entry
// (grid-stride, coalesced); an entry is fluid when bit 31 of its link word
// is clear.  The row of an entry -- its y, for the sin(2 pi y / ny) drive --
// is found by binary search over the row offsets, only when that drive is
// on.
template <typename St>
__global__ void __launch_bounds__(kBudThreads)
k_budget_entries(const void *__restrict__ pops_v, const float4 *__restrict__ U, const uint32_t *__restrict__ links,
                 const int4 *__restrict__ rows, double *__restrict__ part, int nrows, int M, long long Np,
                 ForceArgs fa)
{
    const St *pops = static_cast<const St *>(pops_v);
    const bool wave = fa.w[0] != 0.f || fa.w[1] != 0.f || fa.w[2] != 0.f;
    double m = 0.0, px = 0.0, py = 0.0, pz = 0.0, umax = 0.0, nan = 0.0, work = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < M; c += gridDim.x * blockDim.x) {
        if (links[c] >> 31) continue;
        float sacc = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
        for_speeds<0, kQ>([&](auto pc) {
            constexpr int p = decltype(pc)::value;
            const float v = Pop<St>::template get<p>(pops[(long long)p * Np + c]);
            sacc += v;
            if (cx(p)) jx += cx(p) > 0 ? v : -v;
            if (cy(p)) jy += cy(p) > 0 ? v : -v;
            if (cz(p)) jz += cz(p) > 0 ? v : -v;
        });
        m += 1.0 + (double)sacc;
        px += jx;
        py += jy;
        pz += jz;
        const float4 u4 = U[c];
        const float u2 = u4.x * u4.x + u4.y * u4.y + u4.z * u4.z;
        if (!(u2 == u2) || !(sacc == sacc)) nan += 1.0;
        else if (u2 > umax) umax = u2;
        double sw = 0.0;
        if (wave) {
            int lo = 0, hi = nrows - 1;  // last row whose first entry is <= c
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (rows[mid].x <= c) lo = mid; else hi = mid - 1;
            }
            sw = sinpi(2.0 * (double)(lo % fa.ny) / (double)fa.ny);
        }
        work += ((double)fa.g[0] + (double)fa.w[0] * sw) * u4.x + ((double)fa.g[1] + (double)fa.w[1] * sw) * u4.y +
                ((double)fa.g[2] + (double)fa.w[2] * sw) * u4.z;
    }
    __shared__ double sh[7][kBudThreads];
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = px;
    sh[2][threadIdx.x] = py;
    sh[3][threadIdx.x] = pz;
    sh[4][threadIdx.x] = umax;
    sh[5][threadIdx.x] = nan;
    sh[6][threadIdx.x] = work;
    __syncthreads();
    for (int w = kBudThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int k = 0; k < 7; ++k) {
                if (k == 4)
                    sh[k][threadIdx.x] = fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w]);
                else
                    sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 7) part[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// accum (optional, 8 doubles): time-average sums of a solve, added to when
// the pass counter has reached `from`: work rate, sample count, p_fluid
// (3), max |u| (a maximum), NaN count.
__global__ void __launch_bounds__(kBudThreads)
k_budget_final(const double *__restrict__ part, int nblocks, const double *__restrict__ V, int nc,
               double M, double *__restrict__ out, double *__restrict__ accum,
               const unsigned long long *__restrict__ step, long long from)
{
    __shared__ double sh[10][kBudThreads];
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        for (int k = 0; k < 6; ++k) {
            const double v = part[b * 8 + k];
            acc[k] = k == 4 ? fmax(acc[k], v) : acc[k] + v;
        }
        acc[9] += part[b * 8 + 6];
    }
    for (int i = threadIdx.x; i < nc; i += blockDim.x)
        for (int a = 0; a < 3; ++a) acc[6 + a] += M * V[3 * i + a];
    for (int k = 0; k < 10; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kBudThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 10; ++k)
                sh[k][threadIdx.x] = k == 4 ? fmax(sh[k][threadIdx.x], sh[k][threadIdx.x + w])
                                            : sh[k][threadIdx.x] + sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // mass, p_fluid (3), max |u|, NaN count, p_cells (3), work rate of the external force
        for (int k = 0; k < 10; ++k) out[k] = k == 4 ? sqrt(sh[4][0]) : sh[k][0];
        if (accum && (long long)*step >= from) {
            accum[0] += out[9];
            accum[1] += 1.0;
            for (int a = 0; a < 3; ++a) accum[2 + a] += out[1 + a];
            accum[5] = fmax(accum[5], out[4]);
            accum[6] += out[5];
        }
    }
}

}  // namespace

int pop_bytes(int prec) { return prec == PREC_F32 ? 4 : 2; }

// Stage layout of the row-staged pass: about kStageBytes per stage, whole
// rows, at most one y column of rows; a multiple of the rows that fill the
// consumer threads when rows are short.  A single solve with 16-bit
// populations or with cells stages at least 2 kStConsumers nodes (two per
// consumer thread) when that still leaves kWideMinBatches batches: the
// 64 x 64 x 256 channel with cells, coupled step 97.9 -> 96.2 us in FP32,
// 105.1 -> 101.3 us in binary16 (102.8 with three nodes per thread).  The
// packed passes of the request server (`packed`) keep about kStageBytes,
// since their small lattices need the batches (48 mixed requests: 4.87 ->
// 4.38 solves/s with two nodes per thread).
constexpr int kWideMinBatches = 1024;

StageLayout stage_layout(const Dev &d, bool packed)
{
    StageLayout L;
    L.planes = kQ + (d.nc > 0 ? 4 : 0) + (d.walls ? 1 : 0);
    const int es = pop_bytes(d.prec);
    const int row_bytes = d.nx * (kQ * es + (L.planes - kQ) * 4);
    int budget = kStageBytes;
    if ((es == 2 || d.nc > 0) && !packed) {
        const int wide = max(budget, 2 * kStConsumers * (row_bytes / d.nx));
        const int Bw = max(1, min(wide / row_bytes, d.ny));
        if ((long long)d.nz * ((d.ny + Bw - 1) / Bw) >= kWideMinBatches) budget = wide;
    }
    int B = budget / row_bytes;
    B = B < 1 ? 1 : (B > d.ny ? d.ny : B);
    if (d.nx < kStConsumers && B * d.nx > kStConsumers)
        B -= B % (kStConsumers / d.nx > 0 ? kStConsumers / d.nx : 1);
    L.B = B;
    L.pop_bytes = kQ * B * d.nx * es;
    L.stage_bytes = B * row_bytes;
    L.stages = kMaxStages;
    return L;
}

bool staged_ok(const Dev &d, bool packed)
{
    if (d.compact) return false;  // the compact pass has its own batches
    if ((d.nx * pop_bytes(d.prec)) % 16 != 0) return false;  // rows must be whole 16-byte units
    const StageLayout L = stage_layout(d, packed);
    return 2u * (unsigned)L.stage_bytes <= 200u * 1024u;
}

// Calls op.run<St, WALLS, CELLS, SIGMA>() for the instance's storage type and
// lattice.
template <class Op, typename St>
void dispatch_flags(const Dev &d, Op &op)
{
    const bool cells = d.nc > 0, sig = d.S != nullptr, walls = d.walls != 0;
    if (walls) {
        if (cells) {
            if (sig) op.template run<St, true, true, true>(); else op.template run<St, true, true, false>();
        } else {
            if (sig) op.template run<St, true, false, true>(); else op.template run<St, true, false, false>();
        }
    } else {
        if (cells) {
            if (sig) op.template run<St, false, true, true>(); else op.template run<St, false, true, false>();
        } else {
            if (sig) op.template run<St, false, false, true>(); else op.template run<St, false, false, false>();
        }
    }
}

template <class Op>
void dispatch(const Dev &d, Op &op)
{
    if (d.prec == PREC_F16)
        dispatch_flags<Op, __half>(d, op);
    else if (d.prec == PREC_BF16)
        dispatch_flags<Op, __nv_bfloat16>(d, op);
    else
        dispatch_flags<Op, float>(d, op);
}

// Ring depth: among 2 .. kMaxStages stages (each depth fixes how many CTAs
// fit on an SM), take the one whose last wave of batches leaves the fewest
// idle CTA slots: time ~ ceil(batches / (SMs * k)) * k for k CTAs per SM;
// ties go to the deeper ring.  With cells, at most kLbCtasWithCells CTAs per
// SM: the next step's cell-list, Gay-Berne and shape-list kernels run
// alongside the pass and need registers and shared memory on every SM.
struct PrepareOp {
    Dev &d;
    template <typename St, bool W, bool C, bool S_>
    void run()
    {
        d.lb_grid = 0;
        if constexpr (W) {
            if (d.compact) {
                prepare_compact<St, C, S_>();
                return;
            }
        }
        if (d.fluid_list || !staged_ok(d, false)) return;
        StageLayout L = stage_layout(d, false);
        const int nbatches = d.nz * ((d.ny + L.B - 1) / L.B);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        long long best_cost = -1;
        int best_per_sm = 0;
        raise_smem_limit((const void *)k_lb_staged<St, W, C, S_>, 200 * 1024);
        for (int ns = kMaxStages; ns >= 2; --ns) {
            const size_t smem = (size_t)ns * L.stage_bytes;
            if (smem > 200u * 1024u) continue;
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lb_staged<St, W, C, S_>, kStThreads, smem);
            if (d.nc > 0 && per_sm > kLbCtasWithCells) per_sm = kLbCtasWithCells;
            if (per_sm < 1) continue;
            const long long slots = (long long)sms * per_sm;
            const long long cost = ((nbatches + slots - 1) / slots) * per_sm;
            // on a tie, more CTAs per SM (their copies hide each other's
            // latency): with 48 KB stages one CTA of four stages ties with
            // two of two, and one CTA per SM left the channel's FP32 pass at
            // 43.6 us alone
            if (best_cost < 0 || cost < best_cost || (cost == best_cost && per_sm > best_per_sm)) {
                best_cost = cost;
                best_per_sm = per_sm;
                d.lb_stages = ns;
                d.lb_smem = smem;
                d.lb_grid = (int)(slots > nbatches ? nbatches : slots);
            }
        }
    }
    // compact pass: the same rule over its batch table and stage size
    template <typename St, bool C, bool S_>
    void prepare_compact()
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        raise_smem_limit((const void *)k_lb_compact<St, C, S_>, 200 * 1024);
        int best_per_sm = 0;
        for (int ns = kMaxStages; ns >= 2; --ns) {
            const size_t smem = (size_t)ns * d.lb_stage_bytes;
            if (smem > 200u * 1024u) continue;
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lb_compact<St, C, S_>, kStThreads, smem);
            if (d.nc > 0 && per_sm > kLbCtasWithCells) per_sm = kLbCtasWithCells;
            if (per_sm < 1) continue;
            // many more batches than CTA slots: the last wave costs little,
            // while CTAs per SM hide the copies' latency; take the most CTAs
            // per SM, then the deepest ring (the autotuner times the others)
            const long long slots = (long long)sms * per_sm;
            if (per_sm > best_per_sm) {
                best_per_sm = per_sm;
                d.lb_stages = ns;
                d.lb_smem = smem;
                d.lb_grid = (int)(slots > d.nbatches ? d.nbatches : slots);
            }
        }
    }
};

struct LaunchOp {
    const Dev &d;
    const LbArgs &a;
    cudaStream_t s;
    template <typename St, bool W, bool C, bool S_>
    void run()
    {
        if constexpr (W) {
            if (d.compact) {
                if (d.lb_grid > 0)
                    k_lb_compact<St, C, S_><<<d.lb_grid, kStThreads, d.lb_smem, s>>>(
                        a, d.lb_batches, d.nbatches, d.lb_stages, d.lb_stage_bytes);
                return;
            }
        }
        if (d.fluid_list) {
            const int g = (d.nfluid + kLbThreads - 1) / kLbThreads;
            if (g > 0) k_lb_list<St, W, C, S_><<<g, kLbThreads, 0, s>>>(a, d.fluid_list, d.nfluid);
        } else if (d.lb_grid > 0) {
            StageLayout L = stage_layout(d, false);
            L.stages = d.lb_stages;
            const int nbatches = d.nz * ((d.ny + L.B - 1) / L.B);
            k_lb_staged<St, W, C, S_><<<d.lb_grid, kStThreads, d.lb_smem, s>>>(a, L, nbatches);
        } else {
            k_lb<St, W, C, S_><<<(d.N + kLbThreads - 1) / kLbThreads, kLbThreads, 0, s>>>(a);
        }
    }
};

void prepare_lb(Dev &d)
{
    PrepareOp op{d};
    dispatch(d, op);
}

// Launch shapes of the row-staged pass the autotuner tries: every ring depth
// 2 .. kMaxStages whose stages fit, with 1 .. (what fits on an SM, at most
// 4) CTAs per SM.
struct ShapesOp {
    const Dev &d;
    int *stages, *ctas, max, n;
    template <typename St, bool W, bool C, bool S_>
    void run()
    {
        n = 0;
        const void *kern = (const void *)k_lb_staged<St, W, C, S_>;
        int stage_bytes = 0;
        if constexpr (W) {
            if (d.compact) {
                kern = (const void *)k_lb_compact<St, C, S_>;
                stage_bytes = d.lb_stage_bytes;
            }
        }
        if (!d.compact) {
            if (!staged_ok(d, false)) return;
            stage_bytes = stage_layout(d, false).stage_bytes;
        }
        raise_smem_limit(kern, 200 * 1024);
        for (int ns = 2; ns <= kMaxStages; ++ns) {
            const size_t smem = (size_t)ns * stage_bytes;
            if (smem > 200u * 1024u) continue;
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStThreads, smem);
            for (int c = 1; c <= per_sm && c <= 4 && n < max; ++c) {
                stages[n] = ns;
                ctas[n] = c;
                ++n;
            }
        }
    }
};

int lb_shapes(const Dev &d, int *stages, int *ctas, int max)
{
    ShapesOp op{d, stages, ctas, max, 0};
    dispatch(d, op);
    return op.n;
}

void set_lb_shape(Dev &d, int stages, int ctas_per_sm)
{
    if (d.lb_grid <= 0) return;
    int nbatches = d.nbatches, stage_bytes = d.lb_stage_bytes;
    if (!d.compact) {
        const StageLayout L = stage_layout(d, false);
        nbatches = d.nz * ((d.ny + L.B - 1) / L.B);
        stage_bytes = L.stage_bytes;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long slots = (long long)sms * ctas_per_sm;
    d.lb_stages = stages;
    d.lb_smem = (size_t)stages * stage_bytes;
    d.lb_grid = (int)(slots > nbatches ? nbatches : slots);
}

static LbArgs lb_args(const Dev &d, const Params &p, int parity)
{
    LbArgs a;
    a.src = d.pops[parity];
    a.dst = d.pops[parity ^ 1];
    a.links = d.links;
    a.rows = d.rows;
    a.pool = d.lb_pool;
    a.G = d.G;
    a.U = d.U;
    a.S = d.S;
    a.Syz = d.Syz;
    a.flags = d.flags;
    a.work = d.lb_work;
    a.step = d.lb_step;
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
    a.wx = p.gwave[0];
    a.wy = p.gwave[1];
    a.wz = p.gwave[2];
    a.wave = p.wave;
    a.in_cx = p.in_c[0];
    a.in_cy = p.in_c[1];
    a.in_ir2 = p.in_ir2;
    a.in_umax = p.in_umax;
    a.key0 = (uint32_t)(d.seed & 0xffffffffull);
    a.key1 = (uint32_t)(d.seed >> 32);
    a.stochastic = d.stochastic;
    a.wait_cycles = d.wait_cycles > 0 ? d.wait_cycles : kWaitCycles;
    a.starve_batch = d.starve_batch;
    return a;
}

void launch_lb(const Dev &d, const Params &p, int parity, cudaStream_t s)
{
    const LbArgs a = lb_args(d, p, parity);
    LaunchOp op{d, a, s};
    dispatch(d, op);
}

// ---------------------------------------------------------------------------
// Packs of lattices (request server)
// ---------------------------------------------------------------------------
size_t lb_pack_entry_bytes() { return sizeof(LbPackEntry); }

bool fill_lb_pack_entry(const Dev &d, const Params &p, void *out, int *nbatches, int *stage_bytes)
{
    if (!staged_ok(d, true)) return false;
    LbPackEntry e;
    std::memset(&e, 0, sizeof e);
    e.a = lb_args(d, p, 0);
    e.L = stage_layout(d, true);
    e.L.stages = 0;  // the pack's ring depth applies
    *nbatches = d.nz * ((d.ny + e.L.B - 1) / e.L.B);
    *stage_bytes = e.L.stage_bytes;
    std::memcpy(out, &e, sizeof e);
    return true;
}

// ring depth and grid of a pack's launch: the deepest ring (up to
// kMaxStages) of the pack's largest stage that fits, at most
// kLbCtasWithCells CTAs per SM when cells run beside the pass
struct PackPrepOp {
    const Dev &d0;
    LbPackDesc &k;
    template <typename St, bool W, bool C, bool S_>
    void run()
    {
        raise_smem_limit((const void *)k_lb_staged_packed<St, W, C, S_>, 200 * 1024);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        k.grid = 0;
        for (int ns = kMaxStages; ns >= 2 && k.grid == 0; --ns) {
            const size_t smem = (size_t)ns * k.stage_bytes;
            if (smem > 200u * 1024u) continue;
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lb_staged_packed<St, W, C, S_>, kStThreads, smem);
            if (d0.nc > 0 && per_sm > kLbCtasWithCells) per_sm = kLbCtasWithCells;
            if (per_sm < 1) continue;
            k.stages = ns;
            k.smem = smem;
            k.grid = std::min(sms * per_sm, k.total);
        }
    }
};

struct PackLaunchOp {
    const LbPackDesc &k;
    int parity;
    cudaStream_t s;
    template <typename St, bool W, bool C, bool S_>
    void run()
    {
        k_lb_staged_packed<St, W, C, S_><<<k.grid, kStThreads, k.smem, s>>>(
            static_cast<const LbPackEntry *>(k.tab), k.bstart, k.ninst, k.total, parity, k.work, k.stages,
            k.stage_bytes);
    }
};

bool prepare_lb_pack(const Dev &d0, LbPackDesc &k)
{
    PackPrepOp op{d0, k};
    dispatch(d0, op);
    return k.grid > 0;
}

void launch_lb_packed(const Dev &d0, const LbPackDesc &k, int parity, cudaStream_t s)
{
    PackLaunchOp op{k, parity, s};
    dispatch(d0, op);
}

// Density of every entry (rho - 1; 0 at non-fluid entries): N lattice nodes,
// or the M entries of the compact layout.
void launch_rho(const Dev &d, int parity, cudaStream_t s)
{
    const int n = d.compact ? d.M : d.N;
    const int g = (n + 255) / 256;
    const uint8_t *solid = d.compact ? nullptr : d.solid;
    const uint32_t *links = d.compact ? d.links : nullptr;
    if (d.prec == PREC_F16)
        k_rho<__half><<<g, 256, 0, s>>>(d.pops[parity], solid, links, d.rho, n, d.Np);
    else if (d.prec == PREC_BF16)
        k_rho<__nv_bfloat16><<<g, 256, 0, s>>>(d.pops[parity], solid, links, d.rho, n, d.Np);
    else
        k_rho<float><<<g, 256, 0, s>>>(d.pops[parity], solid, links, d.rho, n, d.Np);
}

// Wall shear stress: the traction sigma n of the last pass's stress on the
// wall's tangent plane, t - (t.n) n, added to the node's time sums.
__global__ void k_wss(const float4 *__restrict__ S, const float4 *__restrict__ U, const float *__restrict__ Syz,
                      const int *__restrict__ node, const float *__restrict__ nrm, double *__restrict__ acc, int nw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nw) return;
    const long long n = node[k];
    const float4 s0 = S[n];
    const float sxx = s0.x, syy = s0.y, szz = s0.z, sxy = s0.w, sxz = U[n].w, syz = Syz[n];
    const float nx = nrm[3 * k], ny = nrm[3 * k + 1], nz = nrm[3 * k + 2];
    const float tx = sxx * nx + sxy * ny + sxz * nz;
    const float ty = sxy * nx + syy * ny + syz * nz;
    const float tz = sxz * nx + syz * ny + szz * nz;
    const float tn = tx * nx + ty * ny + tz * nz;
    acc[3 * k] += (double)(tx - tn * nx);
    acc[3 * k + 1] += (double)(ty - tn * ny);
    acc[3 * k + 2] += (double)(tz - tn * nz);
}

void launch_wss(const Dev &d, cudaStream_t s)
{
    if (d.nwss > 0 && d.S)
        k_wss<<<(d.nwss + 255) / 256, 256, 0, s>>>(d.S, d.U, d.Syz, d.wss_node, d.wss_n, d.wss_acc, d.nwss);
}

int budget_blocks_for(int N)
{
    int b = (N + kBudThreads * 8 - 1) / (kBudThreads * 8);
    return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

void launch_budget(const Dev &d, const Params &p, int parity, cudaStream_t s, bool accumulate, long long from)
{
    ForceArgs fa;
    for (int k = 0; k < 3; ++k) {
        fa.g[k] = p.gext[k];
        fa.w[k] = p.gwave[k];
    }
    fa.nx = d.nx;
    fa.ny = d.ny;
    if (d.compact) {
        const int nrows = d.ny * d.nz;
        if (d.prec == PREC_F16)
            k_budget_entries<__half><<<d.budget_blocks, kBudThreads, 0, s>>>(
                d.pops[parity], d.U, d.links, d.rows, d.budget_part, nrows, d.M, d.Np, fa);
        else if (d.prec == PREC_BF16)
            k_budget_entries<__nv_bfloat16><<<d.budget_blocks, kBudThreads, 0, s>>>(
                d.pops[parity], d.U, d.links, d.rows, d.budget_part, nrows, d.M, d.Np, fa);
        else
            k_budget_entries<float><<<d.budget_blocks, kBudThreads, 0, s>>>(
                d.pops[parity], d.U, d.links, d.rows, d.budget_part, nrows, d.M, d.Np, fa);
    } else if (d.prec == PREC_F16)
        k_budget_nodes<__half><<<d.budget_blocks, kBudThreads, 0, s>>>(d.pops[parity], d.U, d.solid,
                                                                      d.budget_part, d.N, d.Np, fa);
    else if (d.prec == PREC_BF16)
        k_budget_nodes<__nv_bfloat16><<<d.budget_blocks, kBudThreads, 0, s>>>(d.pops[parity], d.U, d.solid,
                                                                             d.budget_part, d.N, d.Np, fa);
    else
        k_budget_nodes<float><<<d.budget_blocks, kBudThreads, 0, s>>>(d.pops[parity], d.U, d.solid,
                                                                     d.budget_part, d.N, d.Np, fa);
    k_budget_final<<<1, kBudThreads, 0, s>>>(d.budget_part, d.budget_blocks, d.V, d.nc, p.M, d.budget_out,
                                             accumulate ? d.accum : nullptr, d.lb_step, from);
}

}  // namespace rbc
